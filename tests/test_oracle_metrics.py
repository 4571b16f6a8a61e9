"""Pins of the error metric every parity test uses (oracle.metrics.rel_frob).

The values below are worked by hand from the definition
||x - ref||_F / ||ref||_F, so a swapped, zeroed or mis-normalised numerator or
denominator fails one of them.
"""
import math

import numpy as np

from oracle.metrics import rel_frob


def test_hand_computed_values():
    ref = np.array([[1.0, 2.0], [3.0, 5.0]])
    x = np.array([[1.0, 2.0], [3.0, 4.0]])
    # ||x - ref|| = 1, ||ref|| = sqrt(1 + 4 + 9 + 25) = sqrt(39)
    assert rel_frob(x, ref) == 1.0 / math.sqrt(39.0)
    # the metric is not symmetric: normalised by the second argument
    assert rel_frob(ref, x) == 1.0 / math.sqrt(30.0)
    # a 3-4-5 difference: ||(3, 4)|| = 5 against ||(3, 4)|| = 5
    assert rel_frob(np.array([6.0, 8.0]), np.array([3.0, 4.0])) == 1.0
    assert abs(rel_frob(np.array([[9.0, 0.0], [0.0, 0.0]]), np.array([[6.0, 8.0], [0.0, 0.0]]))
               - math.sqrt(9.0 + 64.0) / 10.0) < 1e-16


def test_identity_zero_and_scale():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((5, 7))
    assert rel_frob(a, a) == 0.0
    assert rel_frob(np.zeros(3), np.zeros(3)) == 0.0
    # zero reference: the absolute norm of the difference
    assert rel_frob(np.array([0.0, 2.0]), np.zeros(2)) == 2.0
    # invariant under a common scale, linear in the perturbation
    d = rng.standard_normal((5, 7)) * 1e-3
    e1 = rel_frob(a + d, a)
    assert abs(rel_frob(4.0 * (a + d), 4.0 * a) - e1) <= 1e-15 * e1 * 10
    assert abs(rel_frob(a + 2 * d, a) - 2 * e1) <= 1e-12


def test_fp64_accumulation_of_fp32_inputs():
    # FP32 inputs are promoted before the difference is taken: the difference
    # 2^-24 relative in one entry is not lost to FP32 rounding
    ref = np.ones(4, dtype=np.float32)
    x = ref.copy()
    x[0] = np.float32(1.0) + np.float32(2.0 ** -23)
    assert rel_frob(x, ref) == (2.0 ** -23) / 2.0
