"""Error metric used by every parity check (test infrastructure)."""
import numpy as np


def rel_frob(x, ref) -> float:
    """||x - ref||_F / ||ref||_F, accumulated in FP64 (0 if both are zero)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.linalg.norm(ref))
    num = float(np.linalg.norm(x - ref))
    if den == 0.0:
        return num
    return num / den
