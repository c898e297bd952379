"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: printed
values (the P_3 matrices of section 3), closed forms (Legendre roots, the
growth-factor matrix of eq. growth_factor), an independent construction
(quadrature projection of real spherical harmonics), invariants (mass
conservation, exact decay, mirror symmetry, linearity, finite speed) and the
paper's own experiments (second-order convergence of section 6.1, the
discrete L2-norm bound of section 6.2).
"""
import math
import os

import numpy as np
import pytest

from oracle import pn_oracle as O
from paper_1211_2205_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- matrices

def _paper_d(l, m):
    return math.sqrt((l - m) * (l - m - 1) / ((2 * l + 1) * (2 * l - 1)))


def _paper_f(l, m):
    return math.sqrt((l + m) * (l + m - 1) / ((2 * l + 1) * (2 * l - 1)))


def _eval_symbol(sym):
    sign = -1.0 if sym[0] == "-" else 1.0
    body = sym[1:]
    scale = 1.0
    if body.startswith("r2"):
        scale = math.sqrt(2.0)
        body = body[2:]
    name, rest = body.split("_")
    l, m = rest.split("^")
    fn = {"d": _paper_d, "f": _paper_f}[name]
    return sign * scale * fn(int(l), int(m))


def _load_p3():
    Mx = np.zeros((10, 10))
    My = np.zeros((10, 10))
    with open(os.path.join(GOLDEN, "p3_matrices.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            which, r, c, sym = line.split()
            M = Mx if which == "Mx" else My
            M[int(r) - 1, int(c) - 1] = 0.5 * _eval_symbol(sym)
    return Mx, My


def test_p3_matrices_match_printed():
    Mx_p, My_p = _load_p3()
    Mx, My = O.pn_matrices(3)
    np.testing.assert_allclose(Mx, Mx_p, atol=1e-14)
    np.testing.assert_allclose(My, My_p, atol=1e-14)


def test_p1_flux_normalisation():
    # R_0^0 = phi/sqrt(4 pi) and R_1^1 = sqrt(3/(4 pi)) J_x (section 3), so the
    # continuity equation d_t phi + div J = ... reads d_t R00 + (1/sqrt3) d_x R11.
    Mx, My = O.pn_matrices(1)
    assert Mx.shape == (3, 3)
    assert abs(Mx[0, 1] - 1 / math.sqrt(3)) < 1e-15
    assert abs(My[0, 2] - 1 / math.sqrt(3)) < 1e-15
    assert Mx[0, 2] == 0 and My[0, 1] == 0


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 13, 39])
def test_matrices_symmetric_sparse_counts(N):
    Mx, My = O.pn_matrices(N)
    n = (N + 1) * (N + 2) // 2
    assert Mx.shape == (n, n)
    assert np.max(np.abs(Mx - Mx.T)) < 1e-15
    assert np.max(np.abs(My - My.T)) < 1e-15
    assert (Mx != 0).sum(axis=1).max() <= 4
    assert (My != 0).sum(axis=1).max() <= 4


def test_lemma2_coupling_pattern():
    N = 9
    Mx, My = O.pn_matrices(N)
    moms = O.real_moments(N)
    for i, (ki, li, mi) in enumerate(moms):
        for j in np.nonzero(Mx[i])[0]:
            kj, lj, mj = moms[j]
            assert kj == ki and abs(lj - li) == 1 and abs(mj - mi) == 1
        for j in np.nonzero(My[i])[0]:
            kj, lj, mj = moms[j]
            assert kj != ki and abs(lj - li) == 1 and abs(mj - mi) == 1


def _real_harmonics(N, mu, phi):
    """Real harmonics of the real moments: sqrt2 N_l^m cos(m phi) P_l^m,
    sqrt2 N_l^m sin(m phi) P_l^m, N_l^0 P_l (P_l^m without the Condon-Shortley
    phase, consistent with R_1^1 ~ Omega_x, I_1^1 ~ Omega_y of section 3)."""
    from scipy.special import lpmv
    out = []
    for kind, l, m in O.real_moments(N):
        norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
        P = (-1) ** m * lpmv(m, l, mu)
        if m == 0:
            out.append(norm * P)
        elif kind == "R":
            out.append(math.sqrt(2) * norm * np.cos(m * phi) * P)
        else:
            out.append(math.sqrt(2) * norm * np.sin(m * phi) * P)
    return np.array(out)


@pytest.mark.parametrize("N", [3, 6, 11])
def test_matrices_equal_quadrature_projection(N):
    # Independent construction: (M_x)_ij = int Omega_x Y_i Y_j dOmega.
    nq = 2 * N + 6
    mu, w = np.polynomial.legendre.leggauss(nq)
    nphi = 4 * N + 8
    phi = 2 * math.pi * np.arange(nphi) / nphi
    MU, PHI = np.meshgrid(mu, phi, indexing="ij")
    W = np.outer(w, np.full(nphi, 2 * math.pi / nphi))
    Y = _real_harmonics(N, MU, PHI)
    s = np.sqrt(1 - MU ** 2)
    Ox, Oy = s * np.cos(PHI), s * np.sin(PHI)
    gram = np.einsum("iab,jab,ab->ij", Y, Y, W)
    np.testing.assert_allclose(gram, np.eye(len(Y)), atol=1e-12)
    Qx = np.einsum("iab,jab,ab->ij", Y, Y, W * Ox)
    Qy = np.einsum("iab,jab,ab->ij", Y, Y, W * Oy)
    Mx, My = O.pn_matrices(N)
    np.testing.assert_allclose(Mx, Qx, atol=1e-12)
    np.testing.assert_allclose(My, Qy, atol=1e-12)


@pytest.mark.parametrize("N", [1, 3, 5, 7, 13, 20, 39])
def test_slab_eigenvalues_are_legendre_roots(N):
    roots = np.sort(np.polynomial.legendre.legroots([0] * (N + 1) + [1]))
    ev = np.sort(np.linalg.eigvals(O.slab_matrix(N)).real)
    np.testing.assert_allclose(ev, roots, atol=1e-12)


@pytest.mark.parametrize("N,expected", [(5, 0.9324695142), (7, 0.9602898565),
                                        (13, 0.9862838087), (39, 0.9982377097)])
def test_lambda_max_is_largest_legendre_root(N, expected):
    root = np.max(np.polynomial.legendre.legroots([0] * (N + 1) + [1]))
    Mx, My = O.pn_matrices(N)
    assert abs(O.lambda_max(Mx) - root) < 1e-12
    assert abs(root - expected) < 1e-9
    # rotational invariance assumed in section 5.3
    assert abs(O.lambda_max(0.6 * Mx + 0.8 * My) - root) < 1e-11


@pytest.mark.parametrize("N,ax,n,expected,last_digit", [
    (5, (-1.0, 1.0, -1.0, 1.0), 64, 0.0167566, 1e-7),     # P_5 pulse, 64^2 on [-1,1]^2
    (13, (0.0, 7.0, 0.0, 7.0), 512, 0.0069310, 1e-7),     # P_13 checkerboard, 512^2 on [0,7]^2
    (39, (-1.0, 1.0, -1.0, 1.0), 1024, 9.7829e-4, 1e-8),  # P_39, 1024^2 on [-1,1]^2
    (7, (0.0, 7.0, 0.0, 7.0), 512, 0.0071186, 1e-7),      # P_7, 512^2 on [0,7]^2
])
def test_time_step_rule(N, ax, n, expected, last_digit):
    """dt = cn min(dx, dy) / lambda_max with cn = 0.5 (the reading of the
    section 4.5 rule): against the step sizes worked out by hand for the
    workloads (to their printed digits) and against the formula with
    lambda_max taken as the largest root of P_{N+1} (section 5.3), so a
    wrong spacing (n - 1 intervals, the domain's length) or a wrong
    eigenvalue fails."""
    Mx, _ = O.pn_matrices(N)
    dt = O.time_step(Mx, ax, (n, n), 0.5)
    root = float(np.max(np.real(np.polynomial.legendre.legroots([0] * (N + 1) + [1]))))
    assert abs(dt - 0.5 * (ax[1] - ax[0]) / n / root) <= 1e-14 * dt
    assert abs(dt - expected) <= 0.5 * last_digit


def test_time_step_takes_the_smaller_spacing():
    """On a grid with dx != dy the step follows the finer axis, whichever it
    is, and scales linearly with cn."""
    Mx, _ = O.pn_matrices(3)
    lam = O.lambda_max(Mx)
    assert O.time_step(Mx, (0.0, 2.0, 0.0, 1.0), (10, 20), 0.5) == pytest.approx(0.5 * 0.05 / lam, rel=1e-15)
    assert O.time_step(Mx, (0.0, 1.0, 0.0, 3.0), (40, 10), 0.5) == pytest.approx(0.5 * 0.025 / lam, rel=1e-15)
    assert O.time_step(Mx, (0.0, 1.0, 0.0, 1.0), (16, 16), 0.3) == pytest.approx(0.3 / 16 / lam, rel=1e-15)


def test_time_step_reproduces_the_papers_degrees_of_freedom():
    """Section 6.3: the P_5 checkerboard on a 100 x 100 grid of [0,7]^2 run to
    t = 3.2 has 18.3 million degrees of freedom in space, angle and time.
    With the step rule read as dt = 0.5 h / lambda_max and n = ceil(t / dt)
    steps, (n + 1) time levels of 21 moments on 10^4 cells give that figure
    to its printed digits; the reading without the 2D factor 1/2 (dt = h /
    (sqrt(2) lambda_max), the stability bound) does not."""
    Mx, _ = O.pn_matrices(5)
    dt = O.time_step(Mx, (0.0, 7.0, 0.0, 7.0), (100, 100), 0.5)
    steps = math.ceil(3.2 / dt - 1e-9)
    assert steps == 86
    assert round((steps + 1) * 21 * 100 * 100 / 1e5) / 10 == 18.3
    alt = O.time_step(Mx, (0.0, 7.0, 0.0, 7.0), (100, 100), 1 / math.sqrt(2))
    assert round((math.ceil(3.2 / alt - 1e-9) + 1) * 21 * 1e4 / 1e5) / 10 != 18.3


@pytest.mark.parametrize("N,counts", [(5, (6, 6, 6, 3)), (13, (28, 28, 28, 21)),
                                      (39, (210, 210, 210, 190)), (7, (10, 10, 10, 6))])
def test_grid_assignment_counts(N, counts):
    Mx, My = O.pn_matrices(N)
    grid = O.assign_grids(Mx, My)
    got = tuple(sum(1 for g in grid if g == want) for want in ((1, 1), (2, 1), (1, 2), (2, 2)))
    assert got == counts
    for (kind, l, m), g in zip(O.real_moments(N), grid):
        want = {("R", 0): (1, 1), ("R", 1): (2, 1), ("I", 1): (1, 2), ("I", 0): (2, 2)}[(kind, l % 2)]
        assert g == want


# ------------------------------------------------------------ E(c), algebra

def test_expm1div_against_high_precision():
    import mpmath
    mpmath.mp.dps = 50
    cs = np.concatenate([-np.logspace(-12, 2, 300), np.logspace(-12, 2, 300), [0.0, 2e-4, -2e-4]])
    got = O.expm1div(cs)
    for c, g in zip(cs, got):
        ref = mpmath.mpf(1) if c == 0 else mpmath.expm1(mpmath.mpf(c)) / mpmath.mpf(c)
        assert abs(g - float(ref)) <= 1e-12 * abs(float(ref))


def test_two_frozen_half_steps_equal_one_full_step():
    # Two exact sub-steps of dt/2 with frozen r equal one of dt (section 4.3):
    # a^2 = exp(-c dt) and (1 + a) b = dt E(-c dt), a = exp(-c dt/2), b = dt/2 E(-c dt/2).
    for c in [0.0, 1e-9, 1e-4, 0.3, 1.0, 10.0, 1e3]:
        for dt in [1e-3, 0.0167, 0.2]:
            a = math.exp(-c * dt / 2)
            b = dt / 2 * float(O.expm1div(-c * dt / 2))
            assert abs(a * a - math.exp(-c * dt)) < 1e-15
            full = dt * float(O.expm1div(-c * dt))
            # both sides carry E's own error, below 1e-12 by section 5.6
            assert abs((1 + a) * b - full) <= 1e-12 * full


# --------------------------------------------------- Fourier-mode evolution

def _p1_system():
    # section 4.5 model: d_t u^e + d_x u^o + c^e u^e = 0, d_t u^o + d_x u^e + c^o u^o = 0
    Mx = np.array([[0.0, 1.0], [1.0, 0.0]])
    return Mx, np.zeros((2, 2)), np.array([0, 1])


def _paper_growth_matrix(ce, co, dt, h, k):
    """eq. growth_factor as printed."""
    E = lambda c: 1.0 if c == 0 else math.expm1(c) / c
    de, do = math.exp(-0.5 * ce * dt), math.exp(-0.5 * co * dt)
    fe = -1j * dt / h * E(-0.5 * ce * dt) * math.sin(k * h / 2)
    fo = -1j * dt / h * E(-0.5 * co * dt) * math.sin(k * h / 2)
    return np.array([[de ** 2 + (de + 1) * fe * fo, do * (de + 1) * fe],
                     [(do + de ** 2) * fo + (de + 1) * fe * fo ** 2, do ** 2 + do * (de + 1) * fe * fo]])


@pytest.mark.parametrize("ce,co,kappa,steps", [(0.0, 0.0, 3, 7), (0.5, 2.0, 5, 4), (0.0, 30.0, 11, 3)])
def test_p1_growth_factor_printed(ce, co, kappa, steps):
    L, n = 2 * math.pi, 32
    Mx, My, order = _p1_system()
    h = L / n
    k = 2 * math.pi * kappa / L
    dt = 0.8 * h
    ae, ao = 0.7 - 0.2j, -0.3 + 0.9j
    ic = [(0, lambda t, x, y: (ae * np.exp(1j * k * x)).real),
          (1, lambda t, x, y: (ao * np.exp(1j * k * x)).real)]
    # sigma_a = c^e (order 0), sigma_a + sigma_s0 = c^o (order 1)
    s = O.StaggeredSolver(Mx, My, order, (0, L, 0, 1), (n, 1), ("periodic", "periodic"),
                          sigma_a=lambda t, x, y: ce + 0 * x,
                          sigma_s0=lambda t, x, y: (co - ce) + 0 * x, ic=ic, dt=dt)
    s.run(steps)
    G = np.linalg.matrix_power(_paper_growth_matrix(ce, co, dt, h, k), steps)
    a = G @ np.array([ae, ao])
    Xe = s.coords[s.grid[0]][0][:, 0]
    Xo = s.coords[s.grid[1]][0][:, 0]
    np.testing.assert_allclose(s.U[0][:, 0], (a[0] * np.exp(1j * k * Xe)).real, atol=1e-13)
    np.testing.assert_allclose(s.U[1][:, 0], (a[1] * np.exp(1j * k * Xo)).real, atol=1e-13)


def test_p1_stability_threshold():
    # Thm. 1: |lambda| <= 1 for dt < h; remark after it: dt = h, no decay and
    # k = pi/h give a double eigenvalue -1 with a Jordan block (linear growth).
    h = 0.1
    for r in [0.3, 0.7, 0.99]:
        for ce, co in [(0, 0), (0.1, 3.0), (5.0, 0.0)]:
            for k in np.linspace(0, math.pi / h, 37):
                ev = np.linalg.eigvals(_paper_growth_matrix(ce, co, r * h, h, k))
                assert np.max(np.abs(ev)) <= 1 + 1e-12
    # the oracle itself at dt = h shows the linear growth of the k = pi/h mode
    L, n = 2.0, 20
    hh = L / n
    Mx, My, order = _p1_system()
    amp = []
    for steps in (10, 20):
        ic = [(1, lambda t, x, y: np.cos(math.pi / hh * x))]
        s = O.StaggeredSolver(Mx, My, order, (0, L, 0, 1), (n, 1), ("periodic", "periodic"), ic=ic, dt=hh)
        s.run(steps)
        amp.append(np.max(np.abs(s.U[0])))
    assert amp[0] > 5 and abs(amp[1] / amp[0] - 2.0) < 1e-9


def _half_symbol(Mx, My, grid, parity_set, c, dt, Dx, Dy):
    n = Mx.shape[0]
    G = np.eye(n, dtype=np.complex128)
    for j in parity_set:
        a = math.exp(-c[j] * dt / 2)
        b = dt / 2 * (1.0 if c[j] == 0 else -math.expm1(-c[j] * dt / 2) / (c[j] * dt / 2))
        G[j, :] = 0
        G[j, j] = a
        for k in range(n):
            G[j, k] += -b * (Mx[j, k] * Dx + My[j, k] * Dy)
    return G


@pytest.mark.parametrize("system,N,kap,sig", [("pn2d", 3, (2, 5), (0.0, 0.0)),
                                               ("pn2d", 5, (7, 3), (0.2, 1.3)),
                                               ("slab", 7, (4, 0), (0.1, 2.0))])
def test_fourier_mode_evolution(system, N, kap, sig):
    """Discrete symbol of the step (section 4.5 generalised to the full
    system): u_j = Re(a_j exp(i k.x_j)) at each component's own points evolves
    by G = G^o G^e G^e G^o with D_x -> (2i/dx) sin(k_x dx/2)."""
    Mx, My, order = O.system_matrices(system, N)
    nx, ny = (24, 20) if system == "pn2d" else (32, 1)
    ax = (0.0, 1.5, -0.5, 0.5)
    kx = 2 * math.pi * kap[0] / (ax[1] - ax[0])
    ky = 2 * math.pi * kap[1] / (ax[3] - ax[2])
    amps = inputs.fourier_mode_ic(len(order), 7)
    ic = [(j, (lambda aj: (lambda t, x, y: (aj * np.exp(1j * (kx * x + ky * y))).real))(amps[j]))
          for j in range(len(order))]
    sa, ss = sig
    s = O.StaggeredSolver(Mx, My, order, ax, (nx, ny), ("periodic", "periodic"),
                          sigma_a=lambda t, x, y: sa + 0 * x, sigma_s0=lambda t, x, y: ss + 0 * x, ic=ic)
    steps = 5
    s.run(steps)
    dx, dy = s.h
    Dx = 2j / dx * math.sin(kx * dx / 2)
    Dy = 2j / dy * math.sin(ky * dy / 2)
    c = np.array([sa if l == 0 else sa + ss for l in order])
    Ge = _half_symbol(Mx, My, s.grid, s.even, c, s.dt, Dx, Dy)
    Go = _half_symbol(Mx, My, s.grid, s.odd, c, s.dt, Dx, Dy)
    G = Go @ Ge @ Ge @ Go
    a = np.linalg.matrix_power(G, steps) @ amps
    for j in range(len(order)):
        X, Y = s.coords[s.grid[j]]
        np.testing.assert_allclose(s.U[j], (a[j] * np.exp(1j * (kx * X + ky * Y))).real, atol=1e-12)


# ------------------------------------------------------------- invariants

def _random_ic(ncomp, seed, funcs=4):
    rng = inputs.SplitMix64(seed)
    ic = []
    for j in range(ncomp):
        coef = rng.uniforms(3) * 2 - 1
        ic.append((j, (lambda c: (lambda t, x, y: c[0] * np.exp(-((x - 0.3 * c[1]) ** 2 + (y - 0.2 * c[2]) ** 2) / 0.05)))(coef)))
    return ic


def test_mass_conserved_without_absorption():
    N = 5
    Mx, My, order = O.system_matrices("pn2d", N)
    ss = inputs.smooth_log_field(3, 4, -1, 1, (-1, 1, -1, 1))
    s = O.StaggeredSolver(Mx, My, order, (-1, 1, -1, 1), (24, 20), ("periodic", "periodic"),
                          sigma_a=lambda t, x, y: 0 * x, sigma_s0=ss, ic=_random_ic(len(order), 11))
    m0 = s.mass()
    s.run(30)
    assert abs(s.mass() - m0) <= 1e-13 * abs(m0)


def test_mass_decays_exactly_with_uniform_absorption():
    N = 3
    Mx, My, order = O.system_matrices("pn2d", N)
    sa = 0.7
    s = O.StaggeredSolver(Mx, My, order, (-1, 1, -1, 1), (16, 16), ("periodic", "periodic"),
                          sigma_a=lambda t, x, y: sa + 0 * x, sigma_s0=lambda t, x, y: 2.0 + 0 * x,
                          ic=_random_ic(len(order), 5))
    m0 = s.mass()
    s.run(25)
    assert abs(s.mass() - m0 * math.exp(-sa * 25 * s.dt)) <= 1e-13 * abs(m0)


@pytest.mark.parametrize("n", [(1, 1), (4, 3)])
@pytest.mark.parametrize("aniso", [False, True])
def test_homogeneous_state_follows_the_relaxation_ode(n, aniso):
    """A spatially constant state in a constant medium on a periodic grid
    (down to a single cell) has no differences, so every moment obeys its
    own relaxation ODE u' = -c_l u + q (section 2: c_0 = sigma_a, c_l =
    sigma_a + sigma_s0 - sigma_sl), whose exact solution the exponential
    sub-steps (eq. sub_step_solution) must reproduce after any number of
    steps: u(t) = e^(-c t) u(0) + q (1 - e^(-c t)) / c."""
    N = 4
    Mx, My, order = O.system_matrices("pn2d", N)
    sa, s0 = 0.8, 1.7
    fac = [0.6 ** l for l in range(N + 1)] if aniso else None
    rng = inputs.SplitMix64(41)
    u0 = rng.uniforms(len(order)) * 2 - 1
    q = {0: 0.9, 2: -0.4, 7: 0.25}
    s = O.StaggeredSolver(Mx, My, order, (0, 1, 0, 1), n, ("periodic", "periodic"),
                          sigma_a=lambda t, x, y: sa + 0 * x, sigma_s0=lambda t, x, y: s0 + 0 * x,
                          sl_factor=fac, sources=[(j, (lambda v: lambda t, x, y: v + 0 * x)(v)) for j, v in q.items()],
                          ic=[(j, (lambda v: lambda t, x, y: v + 0 * x)(u0[j])) for j in range(len(order))])
    s.run(7)
    t = 7 * s.dt
    for j in range(len(order)):
        l = int(order[j])
        c = sa if l == 0 else sa + s0 - (s0 * fac[l] if aniso else 0.0)
        e = math.exp(-c * t)
        want = e * u0[j] + q.get(j, 0.0) * (1.0 - e) / c
        np.testing.assert_allclose(s.U[j], want, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("bc", ["periodic", "extrapolation"])
def test_even_then_odd_pass_reach_one_point_of_odd_data(bc):
    """One full even pass followed by one full odd pass (the two passes of a
    merged step, which a temporally fused step would run per tile): every
    odd output at array index (i, j) of either odd grid depends on odd
    inputs only at indices i-1..i+1, j-1..j+1 (wrapped on a periodic axis,
    clamped at an extrapolation boundary), so a tile of odd outputs needs one
    point of odd halo on each side.  The bound is reached."""
    N = 4
    Mx, My, order = O.system_matrices("pn2d", N)
    n = (12, 10)
    rng = inputs.SplitMix64(77)
    s = O.StaggeredSolver(Mx, My, order, (0, 1.2, 0, 1.0), n, (bc, bc),
                          sigma_a=lambda t, x, y: 0.3 + 0 * x, sigma_s0=lambda t, x, y: 0.7 + 0 * x,
                          ic=_random_ic(len(order), 9))
    s._evaluate(0.0)
    base = [u.copy() for u in s.U]

    def even_then_odd(U):
        s.U = [u.copy() for u in U]
        dxU, dyU = s._differences(s.odd)
        s._half_step(s.even, dxU, dyU)
        s._half_step(s.even, dxU, dyU)
        dxU, dyU = s._differences(s.even)
        s._half_step(s.odd, dxU, dyU)
        s._half_step(s.odd, dxU, dyU)
        return [s.U[j].copy() for j in s.odd]

    def dist(a, b, d):
        m = n[d] + (1 if bc == "extrapolation" and d == 0 else 0)
        return min(abs(a - b), m - abs(a - b)) if bc == "periodic" else abs(a - b)

    ref = even_then_odd(base)
    reached = 0
    for k0 in s.odd[::3]:
        shape = base[k0].shape
        for (i0, j0) in ((6, 5), (0, 0), (shape[0] - 1, shape[1] - 1)):
            pert = [u.copy() for u in base]
            pert[k0][i0, j0] += 1.0 + rng.uniform()
            out = even_then_odd(pert)
            for got, want in zip(out, ref):
                for i, j in zip(*np.nonzero(np.abs(got - want) > 1e-14)):
                    assert dist(i, i0, 0) <= 1 and dist(j, j0, 1) <= 1, (k0, (i0, j0), (i, j))
                    reached = max(reached, max(dist(i, i0, 0), dist(j, j0, 1)))
    assert reached == 1


def test_symmetry_of_centred_gaussian():
    p = inputs.gaussian_p5(n=32, nsteps=20)
    s = O.solver_from_problem(p)
    s.run(p.nsteps)
    R = s.U[0]
    scale = np.max(np.abs(R))
    assert np.max(np.abs(R - R[::-1, :])) <= 1e-13 * scale
    assert np.max(np.abs(R - R[:, ::-1])) <= 1e-13 * scale
    assert np.max(np.abs(R - R.T)) <= 1e-13 * scale


def test_linearity_and_finite_speed():
    N = 3
    Mx, My, order = O.system_matrices("pn2d", N)
    n = 40
    cell = 1.0 / n

    def src(alpha):
        return [(0, lambda t, x, y: alpha * ((np.abs(x - 0.5 - 0.5 * cell) < 0.4 * cell) & (np.abs(y - 0.5 - 0.5 * cell) < 0.4 * cell)).astype(float))]

    runs = []
    for alpha in (1.0, -3.5):
        s = O.StaggeredSolver(Mx, My, order, (0, 1, 0, 1), (n, n), ("extrapolation", "periodic"),
                              sigma_a=lambda t, x, y: 0 * x, sigma_s0=lambda t, x, y: 0.5 + 0 * x,
                              sources=src(alpha))
        s.run(6)
        runs.append(s)
    for j in range(len(order)):
        scale = np.max(np.abs(runs[0].U[j])) + 1e-300
        np.testing.assert_allclose(runs[1].U[j], -3.5 * runs[0].U[j], rtol=0, atol=1e-14 * 3.5 * scale)
    R = runs[0].U[0]
    i0 = int(np.argmax(np.abs(R).sum(axis=1)))
    assert R[n // 2, n // 2] != 0
    # the source sits in cell (n/2, n/2); per step information moves at most
    # two cells (odd half, even pair, odd half), so cells further than 2*6+1 stay 0
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    far = np.maximum(np.abs(ii - n // 2), np.abs(jj - n // 2)) > 13
    assert np.all(R[far] == 0.0)
    assert i0 == n // 2


# ----------------------------------------------- the paper's experiments

def _mms_problem(n):
    """Section 6.1: P_3 on [0,1]^2, Sigma_a = t cos(2 pi y), Sigma_sl = 0.9^l,
    R_0^0 = e^-t sin^2(2 pi x), all other moments 0."""
    N = 3
    Mx, My, order = O.system_matrices("pn2d", N)
    sl = [0.9 ** l for l in range(N + 1)]
    sigma_a = lambda t, x, y: t * np.cos(2 * math.pi * y) + 0 * x
    exact = lambda t, x, y: math.exp(-t) * np.sin(2 * math.pi * x) ** 2 + 0 * y
    q0 = lambda t, x, y: -math.exp(-t) * np.sin(2 * math.pi * x) ** 2 + sigma_a(t, x, y) * exact(t, x, y)
    q1 = lambda t, x, y: (1 / math.sqrt(3)) * 2 * math.pi * math.exp(-t) * np.sin(4 * math.pi * x) + 0 * y
    s = O.StaggeredSolver(Mx, My, order, (0, 1, 0, 1), (n, n), ("periodic", "periodic"),
                          sigma_a=sigma_a, sigma_s0=lambda t, x, y: 1.0 + 0 * x, sl_factor=sl,
                          sources=[(0, q0), (1, q1)], ic=[(0, exact)], time_dependent=True)
    return s, exact


@pytest.mark.slow
def test_mms_second_order():
    """Section 6.1: observed orders between the successive resolutions 32,
    64, 128 and 256, in the L1, L2 and max norms of the error over all
    moments, all within [1.9, 2.1]."""
    errs = []
    for n in (32, 64, 128, 256):
        s, exact = _mms_problem(n)
        U = s.run_to(0.5)
        e = []
        for j in range(len(U)):
            X, Y = s.coords[s.grid[j]]
            ref = exact(0.5, X, Y) if j == 0 else 0 * X
            e.append(U[j] - ref)
        flat = np.concatenate([v.ravel() for v in e])
        errs.append((np.mean(np.abs(flat)), math.sqrt(np.mean(flat ** 2)), np.max(np.abs(flat))))
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(orders > 1.9) and np.all(orders < 2.1), orders


@pytest.mark.slow
def test_discrete_l2_norm_variation():
    """Section 6.2: P_5, void, periodic, Gaussian sigma = 1e-2; the discrete
    L2 norm varies by less than 0.02% on 100x100 and less on finer grids."""
    var = {}
    for n in (50, 100, 200):
        p = inputs.Problem(name="l2", N=5, ax=(-1, 1, -1, 1), n=(n, n), bc=("periodic", "periodic"),
                           sigma_a=lambda t, x, y: 0 * x, sigma_s0=lambda t, x, y: 0 * x,
                           ic=[(0, inputs.gaussian_paper(1e-2))])
        s = O.solver_from_problem(p)
        P0 = s.l2norm()
        worst = 0.0
        while s.t < 0.5 - 1e-12:
            s.step()
            worst = max(worst, abs(s.l2norm() / P0 - 1))
        var[n] = worst
    assert var[100] < 2e-4
    assert var[200] < var[100] < var[50]


@pytest.mark.parametrize("axis", [0, 1])
def test_extrapolation_equals_mirrored_periodic(axis):
    """Section 4.2: constant extrapolation of the components on cell-centred
    points is exact reflection.  With data even under the mirror x -> -x
    (R_l^m, m even and I_l^m, m odd are even; the others odd and zero on the
    mirror line), the extrapolation run on [0, L] equals the periodic run on
    [-L, L] restricted to [0, L] (and likewise in y)."""
    N = 4
    Mx, My, order = O.system_matrices("pn2d", N)
    n_half, n_other = 10, 8
    L = 1.0
    g = lambda a, b: np.exp(-((a - 0.35) ** 2 + (b - 0.1) ** 2) / 0.04) + 0.3 * np.exp(-((a - 0.8) ** 2) / 0.02)
    ss = lambda a, b: 1.0 + 0.5 * np.cos(3 * a) * np.sin(2 * b + 0.3)
    if axis == 0:
        mir = lambda f: (lambda t, x, y: f(np.abs(x), y))
        ax_e, n_e, bc_e = (0, L, -0.5, 0.5), (n_half, n_other), ("extrapolation", "periodic")
        ax_p, n_p = (-L, L, -0.5, 0.5), (2 * n_half, n_other)
        base = lambda f: (lambda t, x, y: f(x, y))
    else:
        mir = lambda f: (lambda t, x, y: f(np.abs(y), x))
        ax_e, n_e, bc_e = (-0.5, 0.5, 0, L), (n_other, n_half), ("periodic", "extrapolation")
        ax_p, n_p = (-0.5, 0.5, -L, L), (n_other, 2 * n_half)
        base = lambda f: (lambda t, x, y: f(y, x))
    kw = dict(sigma_a=lambda t, x, y: 0.2 + 0 * x)
    se = O.StaggeredSolver(Mx, My, order, ax_e, n_e, bc_e, sigma_s0=base(ss),
                           ic=[(0, base(g))], sources=[(0, base(g))], **kw)
    dt = se.dt
    sp = O.StaggeredSolver(Mx, My, order, ax_p, n_p, ("periodic", "periodic"), sigma_s0=mir(ss),
                           ic=[(0, mir(g))], sources=[(0, mir(g))], dt=dt, **kw)
    se.run(12)
    sp.run(12)
    for j in range(len(order)):
        Xe, Ye = se.coords[se.grid[j]]
        Xp, Yp = sp.coords[sp.grid[j]]
        # pick the periodic run's points that coincide with the extrapolation grid
        ce = (Xe, Ye)[axis]
        cp = (Xp, Yp)[axis]
        vals_p = {}
        for idx in np.ndindex(cp.shape):
            vals_p[(round(float(Xp[idx]), 9), round(float(Yp[idx]), 9))] = sp.U[j][idx]
        # the node at -L coincides with +L in the periodic run
        got, want = [], []
        for idx in np.ndindex(ce.shape):
            key = (round(float(Xe[idx]), 9), round(float(Ye[idx]), 9))
            if key not in vals_p:
                alt = list(key)
                alt[axis] = round(-alt[axis], 9)
                key = tuple(alt)
            got.append(se.U[j][idx])
            want.append(vals_p[key])
        scale = max(1e-300, np.max(np.abs(sp.U[0])))
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * scale)
