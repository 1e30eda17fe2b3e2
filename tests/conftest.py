import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


def check_flagged_bounds(T_gpu, ref, tol=1e-5, t_min=1e-4):
    """Rays the oracle flags (a candidate inside a rounding band of a
    threshold, or T near T_min, where a float32 evaluation may decide either
    way) hold T_gpu within tol of the oracle's bounds [T_lo, T_hi] over taking
    or leaving each borderline candidate, or 0 where those bounds reach below
    T_min.  Returns the number of flagged rays."""
    import numpy as np
    T_gpu = np.asarray(T_gpu, np.float64)
    fl = ref["flags"] != 0
    lo, hi = ref["T_lo"], ref["T_hi"]
    inside = (T_gpu >= lo - tol) & (T_gpu <= hi + tol)
    snapped = (T_gpu == 0) & (lo < t_min + tol)
    bad = np.nonzero(fl & ~inside & ~snapped)[0]
    assert bad.size == 0, (bad[:10], T_gpu[bad[:10]], lo[bad[:10]], hi[bad[:10]])
    return int(fl.sum())


def visibility_range(ref, tol=1e-5, t_min=1e-4):
    """Per ray, the interval [lo, hi] that a correct float32 trace may
    return: the oracle's bounds widened by tol, reaching down to 0 where
    the lower bound lies below T_min (the trace may snap there).  For the
    consumers that are monotone in each ray's T (an average, Eq. 10's
    colour)."""
    import numpy as np
    lo = np.where(ref["T_lo"] < t_min + tol, 0.0, ref["T_lo"] - tol)
    return np.maximum(lo, 0.0), ref["T_hi"] + tol
