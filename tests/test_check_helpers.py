"""The parity checkers that hold flagged rays to the oracle's bounds
(``conftest.check_flagged_bounds``, ``conftest.visibility_range``), CPU only:
they accept the oracle's own values and any value a float32 evaluation may
take (a borderline candidate taken or left out), and reject a value outside
the bounds, so a GPU test that uses them is not vacuous."""
import math

import numpy as np
import pytest

import scenes
from conftest import check_flagged_bounds, visibility_range


@pytest.fixture(scope="module")
def flagged(orc):
    sc = scenes.uniform_scene(600, 21, log_scale_mean=math.log(0.08))
    dirs = scenes.fibonacci_sphere(32)
    ro, rd, src = orc.dir_rays(sc["mean"], dirs, np.arange(600 * 32, dtype=np.int64))
    ref = orc.trace(sc, ro, rd, src)
    fl = ref["flags"] != 0
    assert fl.sum() >= 5
    return ref


def test_accepts_the_oracle_and_its_bounds(flagged):
    ref = flagged
    assert check_flagged_bounds(ref["T"], ref) == int((ref["flags"] != 0).sum())
    # either end of a flagged ray's bounds, snapped as the trace snaps
    for side in ("T_lo", "T_hi"):
        T = np.where(ref[side] < 1e-4, 0.0, ref[side])
        check_flagged_bounds(T, ref)
    lo, hi = visibility_range(ref)
    assert np.all(lo <= ref["T"]) and np.all(ref["T"] <= hi) and np.all(lo >= 0)


def test_rejects_values_outside_the_bounds(flagged):
    ref = flagged
    fl = np.nonzero((ref["flags"] != 0) & (ref["T_lo"] > 1e-3))[0]
    assert fl.size > 0
    r = fl[0]
    for bad in (ref["T_hi"][r] + 1e-4, ref["T_lo"][r] - 1e-4, 0.0):
        T = ref["T"].copy()
        T[r] = bad
        with pytest.raises(AssertionError):
            check_flagged_bounds(T, ref)
