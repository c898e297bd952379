"""Moments of a unit beam (the source of the beam test, section 6): the
oracle's real harmonics against what fixes them -- closed forms of the
first orders, the addition theorem, and the recursion that defines the
flux matrices (Omega_x Y_i = sum_j Mx[i, j] Y_j for every row below the
truncation order) -- and the library's host function against the oracle."""
import math

import numpy as np
import pytest

from oracle import pn_oracle as O
from paper_1211_2205_gb300 import capi

DIRS = [(0.0, math.pi / 6), (0.3, 1.1), (-0.8, 4.0), (0.999, 2.5)]


@pytest.fixture(scope="module")
def built():
    """The library's host functions need libstarmap.so (compiled here, no GPU needed)."""
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("mu,phi", DIRS)
def test_first_moments_closed_form(mu, phi):
    y = O.direction_moments(3, mu, phi)
    s = math.sqrt(1 - mu * mu)
    assert y[0] == pytest.approx(1 / math.sqrt(4 * math.pi), rel=1e-15)
    assert y[1] == pytest.approx(math.sqrt(3 / (4 * math.pi)) * s * math.cos(phi), abs=1e-15)
    assert y[2] == pytest.approx(math.sqrt(3 / (4 * math.pi)) * s * math.sin(phi), abs=1e-15)


@pytest.mark.parametrize("phi", [0.0, math.pi / 6, 2.0])
def test_addition_theorem_in_the_plane(phi):
    """sum_m |Y_l^m|^2 = (2l + 1)/(4 pi); in the plane (mu = 0) the
    harmonics with l + m odd vanish, so the 2D moments alone carry it."""
    N = 39
    y = O.direction_moments(N, 0.0, phi)
    order = O.moment_orders(N)
    for l in range(N + 1):
        assert np.sum(y[order == l] ** 2) == pytest.approx((2 * l + 1) / (4 * math.pi), rel=1e-12)


@pytest.mark.parametrize("N", [5, 12, 39])
@pytest.mark.parametrize("mu,phi", DIRS)
def test_flux_matrices_reproduce_the_direction(N, mu, phi):
    Mx, My = O.pn_matrices(N)
    y = O.direction_moments(N, mu, phi)
    rows = O.moment_orders(N) < N
    s = math.sqrt(1 - mu * mu)
    np.testing.assert_allclose((Mx @ y)[rows], s * math.cos(phi) * y[rows], atol=1e-12)
    np.testing.assert_allclose((My @ y)[rows], s * math.sin(phi) * y[rows], atol=1e-12)


@pytest.mark.parametrize("N", [3, 9, 39])
@pytest.mark.parametrize("mu,phi", DIRS)
def test_library_matches_oracle(built, N, mu, phi):
    np.testing.assert_allclose(capi.direction_moments(N, mu, phi), O.direction_moments(N, mu, phi), atol=1e-14)


def test_library_rejects_bad_arguments(built):
    with pytest.raises(capi.StarmapError) as e:
        capi.direction_moments(3, 1.5, 0.0)
    assert e.value.code == capi.E_ARG


def _beam_centroid(U, coords, grid, cell):
    X, Y = coords[grid[0]]
    R = U[0]
    m = float(R.sum())
    return m * cell, float((R * X).sum()) / m, float((R * Y).sum()) / m


@pytest.mark.parametrize("N", [3, 9])
def test_oracle_beam_in_void(N):
    """The beam of section 6 with the medium moved out of the domain (all
    void), before the beam reaches the boundary:
    the source feeds R_0^0 at the rate Y_0^0 times its (sampled) mass, and
    the flux moments carry its centroid along Omega_0 at unit speed, so at
    time t the mass is t / sqrt(4 pi) times the source mass and the
    centroid t/2 Omega_0, each flux component scaled by the source mass
    sampled on its own grid relative to R_0^0's (summation by parts of the
    staggered differences, and the midpoint rule of the step is exact for
    the linearly growing flux: these hold for every N)."""
    from paper_1211_2205_gb300 import inputs
    p = inputs.beam(O.direction_moments(N, 0.0, inputs.BEAM_ANGLE), n=48, precision="fp64", interface=10.0)
    s = O.solver_from_problem(p)
    s.run(int(round(0.25 / s.dt)))                   # whole steps: the centroid grows as t^2
    t = s.t
    U = s.U
    cell = (1.2 / 48) ** 2
    mass, cx, cy = _beam_centroid(U, s.coords, s.grid, cell)
    qbar = inputs.gaussian_paper(3.2e-4)
    # the sampled source's mass on the grids of R_0^0, R_1^1 and I_1^1
    fed = [float(qbar(0.0, *s.coords[s.grid[j]]).sum()) * cell for j in range(3)]
    assert mass == pytest.approx(t / math.sqrt(4 * math.pi) * fed[0], rel=1e-12)
    assert cx == pytest.approx(0.5 * t * math.cos(inputs.BEAM_ANGLE) * fed[1] / fed[0], rel=1e-12)
    assert cy == pytest.approx(0.5 * t * math.sin(inputs.BEAM_ANGLE) * fed[2] / fed[0], rel=1e-12)
