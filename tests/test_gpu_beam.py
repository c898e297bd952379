"""The beam test of section 6 on the GPU: the library's beam moments drive
the source (the oracle uses its own), the beam crosses the void and hits
the Henyey-Greenstein medium (Sigma_sl = 100 * 0.85^l, N + 1 decay
classes)."""
import math

import numpy as np
import pytest

from helpers import DT_RTOL, assert_parity
from oracle import pn_oracle as O
from paper_1211_2205_gb300 import capi, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,kernel,tol", [("fp64", "auto", 1e-12), ("fp32", "tiled", 1e-5)])
def test_beam_matches_oracle_through_the_interface(precision, kernel, tol):
    N, n = 9, 48
    p = inputs.beam(capi.direction_moments(N, 0.0, inputs.BEAM_ANGLE), n=n, precision=precision)
    po = inputs.beam(O.direction_moments(N, 0.0, inputs.BEAM_ANGLE), n=n, precision="fp64")
    s = capi.Stepper.from_problem(p, kernel=kernel, schedule="merged")
    o = O.solver_from_problem(po)                  # the oracle's own step size ...
    assert abs(s.dt - o.dt) <= DT_RTOL * o.dt      # ... equals the library's
    nsteps = int(math.ceil(0.5 / o.dt))            # the front passes x = 0.3 at t ~ 0.35
    s.step(nsteps)
    got = [s.moments(j) for j in range(s.ncomp)]
    o.run(nsteps)
    assert_parity(got, [u.T for u in o.U], tol, precision)


def test_full_size_beam_p39():
    """150 x 150, P_39, FP32 tiled kernel (the paper's run).  With the medium
    moved away the mass at t ~ 0.25 is t / sqrt(4 pi) times the source's
    and the centroid t/2 Omega_0 (exact for the scheme at any order); with
    the medium, at t ~ 0.6 the beam has entered it and the state is finite."""
    N, n = 39, 150
    y0 = capi.direction_moments(N, 0.0, inputs.BEAM_ANGLE)
    cell = (1.2 / n) ** 2
    # all void: mass and centroid are exact for the scheme
    v = capi.Stepper.from_problem(inputs.beam(y0, n=n, interface=10.0), kernel="tiled", schedule="merged")
    v.step(int(round(0.25 / v.dt)))
    t = v.time
    R = v.moments(0).astype(np.float64)
    X, Y = v.grid_coords(v.moment_info(0)["grid"])
    qbar = inputs.gaussian_paper(3.2e-4)
    fed = [float(qbar(0.0, *v.grid_coords(v.moment_info(j)["grid"])).sum()) * cell for j in range(3)]
    m = float(R.sum())
    assert m * cell == pytest.approx(t / math.sqrt(4 * math.pi) * fed[0], rel=1e-5)
    assert float((R * X).sum()) / m == pytest.approx(0.5 * t * math.cos(inputs.BEAM_ANGLE) * fed[1] / fed[0], rel=1e-4)
    assert float((R * Y).sum()) / m == pytest.approx(0.5 * t * math.sin(inputs.BEAM_ANGLE) * fed[2] / fed[0], rel=1e-4)
    v.close()
    # the paper's beam: into the medium by t = 0.6
    p = inputs.beam(y0, n=n, precision="fp32")
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule="merged")
    s.step(int(round(0.6 / s.dt)))
    _, _, bad = s.diagnostics()
    assert bad == 0
    R = s.moments(0)
    assert float(R[:, X[0] >= inputs.BEAM_INTERFACE].sum()) > 0.05 * float(R.sum())
