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
