"""Failure detection without a GPU fault: a device wait that can never
complete gives up after its limit, latches LINVIEW_ETIMEOUT exactly as a view
pass does when a copy never lands, and leaves the context usable.  The wait
is on an mbarrier that nothing arrives on (no fault, no trap, no endless
loop); every pass bounds its waits the same way (limit 2 s)."""
import numpy as np
import pytest

import linview_inputs as li
from oracle import powers as op
from oracle.metrics import rel_frob

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def test_expired_wait_latches_timeout_and_context_stays_usable():
    from paper_1403_6968_gb300 import Program, check_bounded_wait, LinviewError, _lib
    limit = 20_000_000  # 20 ms
    waited = check_bounded_wait(limit)
    assert limit <= waited < 2_000_000_000, waited
    # bad limits are refused before any device work
    with pytest.raises(LinviewError) as e:
        check_bounded_wait(10)
    assert e.value.status == _lib.EINVAL
    # the context is intact: a program refreshes correctly afterwards
    n, k = 256, 4
    a = li.power_matrix(n, seed=3)
    prog = Program("power", [torch.from_numpy(a).cuda()], k=k, precision="f64")
    u, v = next(iter(li.lowrank_update_stream(n, 1, 1, seed=4)))
    prog.apply_delta(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda())
    prog.sync()
    ref = op.reeval_powers(a + u @ v.T, k)
    assert rel_frob(prog.read_view_host(2), ref[4]) <= 1e-10
