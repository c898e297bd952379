"""FP32 parity over the workloads' full run lengths (the precision policy
keeps moments in FP32; rounding errors accumulate with the step count).
The tiled kernel with the merged schedule, as the benchmark runs it,
against FP64 oracle results stored by ``tests/golden/make_long_runs.py``
(a script that calls only the oracle and the seeded input module):

* the P_13 checkerboard of section 6.3, 512 x 512 on [0,7]^2,
  extrapolation boundaries, 462 steps and linear interpolation to t = 3.2;
* P_39 on the random scattering medium, 256 x 256 periodic, 200 steps.

Compared: R_0^0 on its whole grid; every component on a sub-lattice of its
own grid, pooled and one by one (``helpers.assert_parity``); every
component's whole-grid norm; and the same sub-lattices at intermediate step
counts (the error's growth with the run length)."""
import math
import os

import numpy as np
import pytest

from helpers import FLOOR_ULPS, UNIT_ROUNDOFF, assert_parity, check_dt, rel_l2
from paper_1211_2205_gb300 import capi, inputs

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.fail(f"missing stored oracle run {name}: run tests/golden/make_long_runs.py")
    return np.load(path)


def _check_against(g, final, snaps_got):
    """final: the GPU's full arrays [iy, ix] per component at the end;
    snaps_got: {step: list of coarse sub-lattices}."""
    ncomp = len(final)
    off, st = int(g["off"]), int(g["stride"])
    r00 = g["r00"]
    assert final[0].shape == r00.shape
    assert rel_l2([final[0]], [r00]) <= FP32_TOL
    got = [final[j][off::st, off::st] for j in range(ncomp)]
    ref = [g[f"c{j}"] for j in range(ncomp)]
    assert_parity(got, ref, FP32_TOL, "fp32", "final sub-lattice")
    # whole-grid norms, component by component
    norms = g["norms"]
    pooled = float(np.sqrt(np.sum(norms ** 2)))
    mine = np.array([math.sqrt(float(np.sum(np.asarray(u, dtype=np.float64) ** 2))) for u in final])
    bar = FP32_TOL * norms + FLOOR_ULPS["fp32"] * UNIT_ROUNDOFF["fp32"] * pooled
    assert np.all(np.abs(mine - norms) <= bar), int(np.argmax(np.abs(mine - norms) / bar))
    curve = {}
    for k in g["snap_steps"]:
        ref_k = [g[f"s{int(k)}_{j}"] for j in range(ncomp)]
        curve[int(k)] = assert_parity(snaps_got[int(k)], ref_k, FP32_TOL, "fp32", f"step {int(k)}")
    return curve


def _snap(s, so, ss):
    return [s.moments(j)[so::ss, so::ss] for j in range(s.ncomp)]


def test_checkerboard_p13_to_final_time():
    g = _load("long_checkerboard_p13.npz")
    p = inputs.checkerboard_p13()
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule="merged")
    assert s.kernel == "tiled"
    assert check_dt(s, p) == pytest.approx(float(g["dt"]), rel=1e-15)
    so, ss = int(g["snap_off"]), int(g["snap_stride"])
    snaps = {}
    for k in g["snap_steps"]:
        s.step(int(k) - s.steps_done)
        snaps[int(k)] = _snap(s, so, ss)
    s.advance_to(float(g["t_final"]))
    assert s.steps_done == int(g["steps_done"]) == 462
    final = [s.output(j) for j in range(s.ncomp)]
    s.close()
    _check_against(g, final, snaps)
    assert np.abs(final[0]).max() > 1e-2


def test_random_p39_two_hundred_steps():
    g = _load("long_random_p39_256.npz")
    p = inputs.random_p39(n=256)
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule="merged")
    assert s.kernel == "tiled"
    assert check_dt(s, p) == pytest.approx(float(g["dt"]), rel=1e-15)
    so, ss = int(g["snap_off"]), int(g["snap_stride"])
    snaps = {}
    for k in g["snap_steps"]:
        s.step(int(k) - s.steps_done)
        snaps[int(k)] = _snap(s, so, ss)
    s.step(p.nsteps - s.steps_done)
    assert s.steps_done == int(g["steps_done"]) == 200
    final = [s.moments(j) for j in range(s.ncomp)]
    s.close()
    _check_against(g, final, snaps)
