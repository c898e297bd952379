"""StaRMAP oracle: a plain, slow FP64 restatement of the staggered-grid P_N
scheme of Seibold & Frank, "StaRMAP -- A Second Order Staggered Grid Method
for Spherical Harmonics Moment Equations of Radiative Transfer"
(arXiv:1211.2205).

THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.
The product path (the CUDA library and its Python binding) never calls it,
and nothing here imports the product.  It shares no code, tables or
constants with the CUDA path.

Each function follows the passage cited in its docstring, in the paper's
order and notation, with no blocking, fusion or reordering:

* moment matrices from the recursion coefficients of section 3 and the
  real transformation S (eq. transformation);
* grid assignment by the nonzero patterns (eq. matrix_conditions, section 5.3);
* per-component 2D arrays of the sizes of section 5.2, boundary index
  vectors of section 5.3, half-grid differences (eq. central_differences);
* the exact sub-step (eq. sub_step_solution) with E(c) = (e^c - 1)/c
  (section 5.6), as the weighted sparse sum of section 5.5;
* the Strang composition O-E-E-O (eq. solution_operator_full_step) with the
  even differences computed once (section 5.8), material and sources at the
  half-step time, output by linear interpolation in time (section 5.8).

Readings where the paper is silent or garbled:

* time step: dt = cn * min(dx, dy) / lambda_max(Mx); cn already contains the
  2D factor 1/2 of section 4.5;
* the Taylor branch of E printed in section 5.6 is E(-c); E(c) itself is
  1 + c/2 + c^2/6 for |c| <= 2e-4, expm1(c)/c otherwise;
* Sigma_t0 = Sigma_a for the zeroth moment, Sigma_tl = Sigma_a + Sigma_s0 -
  Sigma_sl for l >= 1, and Sigma_sl = 0 (l >= 1) for isotropic scattering.
"""
from __future__ import annotations

import math
from collections import deque
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

SQRT2 = math.sqrt(2.0)


# ---------------------------------------------------------------------------
# Section 3: recursion coefficients of Omega * conj(Y_l^m)
# ---------------------------------------------------------------------------

def _root(num: float, den: float) -> float:
    q = num / den
    if q < 0.0:
        if q > -1e-300:
            return 0.0
        raise ValueError("negative radicand in recursion coefficient")
    return math.sqrt(q)


def coef_a(l, m): return _root((l - m + 1) * (l + m + 1), (2 * l + 3) * (2 * l + 1))
def coef_b(l, m): return _root((l - m) * (l + m), (2 * l + 1) * (2 * l - 1))
def coef_c(l, m): return _root((l + m + 1) * (l + m + 2), (2 * l + 3) * (2 * l + 1))
def coef_d(l, m): return _root((l - m) * (l - m - 1), (2 * l + 1) * (2 * l - 1))
def coef_e(l, m): return _root((l - m + 1) * (l - m + 2), (2 * l + 3) * (2 * l + 1))
def coef_f(l, m): return _root((l + m) * (l + m - 1), (2 * l + 1) * (2 * l - 1))


def complex_moments(N: int) -> List[Tuple[int, int]]:
    """Complex moments psi_l^m kept by the z-symmetry reduction (section 3):
    0 <= l <= N, -l <= m <= l, l + m even, ordered by l then m."""
    return [(l, m) for l in range(N + 1) for m in range(-l, l + 1) if (l + m) % 2 == 0]


def real_moments(N: int) -> List[Tuple[str, int, int]]:
    """Real moments in the order of eq. transformation:
    R_0^0, R_1^1, I_1^1, R_2^2, I_2^2, R_2^0, R_3^3, I_3^3, R_3^1, I_3^1, ..."""
    out = []
    for l in range(N + 1):
        for m in range(l, 0, -2):
            out.append(("R", l, m))
            out.append(("I", l, m))
        if l % 2 == 0:
            out.append(("R", l, 0))
    return out


def _legendre_derivative(l: int, m: int, x):
    """d^m/dx^m P_l(x), exact in rationals, from the explicit sum
    P_l(x) = 2^-l sum_k (-1)^k C(l, k) C(2l - 2k, l) x^(l - 2k)."""
    from fractions import Fraction
    total = Fraction(0)
    for k in range(l // 2 + 1):
        p = l - 2 * k
        if p < m:
            continue
        coef = Fraction((-1) ** k * math.comb(l, k) * math.comb(2 * l - 2 * k, l), 2 ** l)
        total += coef * Fraction(math.factorial(p), math.factorial(p - m)) * x ** (p - m)
    return total


def direction_moments(N: int, mu: float, phi: float) -> np.ndarray:
    """The real harmonic of every real moment (order of real_moments) at the
    direction (sqrt(1-mu^2) cos phi, sqrt(1-mu^2) sin phi, mu): the moments
    of a unit beam q = delta(Omega - Omega_0) (the beam test of section 6).
    Orthonormal, without the Condon-Shortley phase (R_1^1 ~ Omega_x, I_1^1 ~
    Omega_y, as the real moments of section 3):
        N_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
        P_l^m(mu) = (1 - mu^2)^(m/2) d^m/dmu^m P_l(mu)   (derivative exact),
        R_l^m = sqrt2 N_l^m P_l^m cos(m phi), I_l^m = sqrt2 N_l^m P_l^m sin(m phi),
        R_l^0 = N_l^0 P_l(mu)."""
    from fractions import Fraction
    x = Fraction(mu)
    st = math.sqrt(max(0.0, 1.0 - mu * mu))
    out = []
    for kind, l, m in real_moments(N):
        norm = math.sqrt((2 * l + 1) / (4 * math.pi) * float(Fraction(math.factorial(l - m), math.factorial(l + m))))
        P = st ** m * float(_legendre_derivative(l, m, x))
        if m == 0:
            out.append(norm * P)
        elif kind == "R":
            out.append(math.sqrt(2.0) * norm * P * math.cos(m * phi))
        else:
            out.append(math.sqrt(2.0) * norm * P * math.sin(m * phi))
    return np.array(out)


def complex_flux_matrices(N: int) -> Tuple[np.ndarray, np.ndarray]:
    """M_x^complex and M_y^complex of section 3 (including the 1/2 and i/2),
    read off eq. Pncomplex; terms of order N+1 are dropped (P_N closure)."""
    moms = complex_moments(N)
    idx = {lm: k for k, lm in enumerate(moms)}
    n = len(moms)
    Mx = np.zeros((n, n), dtype=np.complex128)
    My = np.zeros((n, n), dtype=np.complex128)
    for (l, m), row in idx.items():
        # (target l, target m, x-coefficient, y-coefficient) before 1/2, i/2
        terms = []
        if (l - 1, m - 1) in idx:
            c = coef_c(l - 1, m - 1)
            terms.append(((l - 1, m - 1), -c, c))
        if (l + 1, m - 1) in idx:
            d = coef_d(l + 1, m - 1)
            terms.append(((l + 1, m - 1), d, -d))
        if (l - 1, m + 1) in idx:
            e = coef_e(l - 1, m + 1)
            terms.append(((l - 1, m + 1), e, e))
        if (l + 1, m + 1) in idx:
            f = coef_f(l + 1, m + 1)
            terms.append(((l + 1, m + 1), -f, -f))
        for target, cx, cy in terms:
            col = idx[target]
            Mx[row, col] += 0.5 * cx
            My[row, col] += 0.5j * cy
    return Mx, My


def realification(N: int) -> np.ndarray:
    """The unitary matrix S of eq. transformation: u = S psi with
    R_l^0 = psi_l^0, R_l^m = (-1)^m/sqrt2 (psi_l^m + (-1)^m psi_l^-m),
    I_l^m = (-1)^m i/sqrt2 (psi_l^m - (-1)^m psi_l^-m)."""
    cidx = {lm: k for k, lm in enumerate(complex_moments(N))}
    real = real_moments(N)
    S = np.zeros((len(real), len(cidx)), dtype=np.complex128)
    for r, (kind, l, m) in enumerate(real):
        sgn = (-1.0) ** m
        if m == 0:
            S[r, cidx[(l, 0)]] = 1.0
        elif kind == "R":
            S[r, cidx[(l, m)]] += sgn / SQRT2
            S[r, cidx[(l, -m)]] += sgn * sgn / SQRT2
        else:
            S[r, cidx[(l, m)]] += 1j * sgn / SQRT2
            S[r, cidx[(l, -m)]] += -1j * sgn * sgn / SQRT2
    return S


def pn_matrices(N: int, zero_tol: float = 1e-13) -> Tuple[np.ndarray, np.ndarray]:
    """Real P_N matrices M^real = S M^complex S^-1 (section 3, eq.
    real_valued_pn_equations).  Returns (Mx, My) as dense FP64 arrays."""
    Mxc, Myc = complex_flux_matrices(N)
    S = realification(N)
    Sinv = np.linalg.inv(S)
    out = []
    for Mc in (Mxc, Myc):
        M = S @ Mc @ Sinv
        if np.max(np.abs(M.imag)) > 1e-12:
            raise AssertionError("real P_N matrix has an imaginary part")
        R = M.real.copy()
        R[np.abs(R) < zero_tol] = 0.0
        out.append(R)
    return out[0], out[1]


def moment_orders(N: int) -> np.ndarray:
    """Moment order l of each real component (par.mom_order, section 5.1)."""
    return np.array([l for (_, l, _) in real_moments(N)], dtype=np.int64)


def slab_matrix(N: int) -> np.ndarray:
    """Tridiagonal slab-geometry matrix M of eq. PN_slab:
    M[l, l+1] = (l+1)/(2l+1), M[l, l-1] = l/(2l+1)."""
    M = np.zeros((N + 1, N + 1))
    for l in range(N + 1):
        if l + 1 <= N:
            M[l, l + 1] = (l + 1) / (2 * l + 1)
        if l - 1 >= 0:
            M[l, l - 1] = l / (2 * l + 1)
    return M


def system_matrices(system: str, N: int):
    """(Mx, My, mom_order) for the 2D P_N system or the slab system (My = 0)."""
    if system == "pn2d":
        Mx, My = pn_matrices(N)
        return Mx, My, moment_orders(N)
    if system == "slab":
        M = slab_matrix(N)
        return M, np.zeros_like(M), np.arange(N + 1, dtype=np.int64)
    raise ValueError(system)


# ---------------------------------------------------------------------------
# Section 4.1 / 5.3: distribution of the components onto the staggered grids
# ---------------------------------------------------------------------------

def assign_grids(Mx: np.ndarray, My: np.ndarray) -> List[Tuple[int, int]]:
    """Index sets I11, I21, I12, I22 of eq. matrix_conditions, found as in
    section 5.3: component 1 goes to G11, then every nonzero of Mx (My)
    moves a neighbour to the grid staggered in x (y), until all are placed.
    Returns the grid code (gx, gy) in {1,2}^2 of every component."""
    n = Mx.shape[0]
    grid: List[Optional[Tuple[int, int]]] = [None] * n
    grid[0] = (1, 1)
    queue = deque([0])
    while queue:
        i = queue.popleft()
        gx, gy = grid[i]
        links = []
        for j in np.nonzero(Mx[i])[0].tolist() + np.nonzero(Mx[:, i])[0].tolist():
            links.append((j, (3 - gx, gy)))
        for j in np.nonzero(My[i])[0].tolist() + np.nonzero(My[:, i])[0].tolist():
            links.append((j, (gx, 3 - gy)))
        for j, want in links:
            if grid[j] is None:
                grid[j] = want
                queue.append(j)
            elif grid[j] != want:
                raise ValueError("coupling pattern admits no staggered placement")
    if any(g is None for g in grid):
        raise ValueError("component not reachable from component 1")
    return grid  # type: ignore[return-value]


def lambda_max(Mx: np.ndarray) -> float:
    """Largest eigenvalue magnitude of Mx (section 5.3, eigs(Mx,1,'lm'))."""
    return float(np.max(np.abs(np.linalg.eigvals(Mx))))


def time_step(Mx: np.ndarray, ax, n, cn: float) -> float:
    """dt = cn * min(dx, dy) / lambda_max (section 4.5 rules; reading)."""
    dx = (ax[1] - ax[0]) / n[0]
    dy = (ax[3] - ax[2]) / n[1]
    return cn * min(dx, dy) / lambda_max(Mx)


# ---------------------------------------------------------------------------
# Section 5.6: E(c) = (exp(c) - 1)/c
# ---------------------------------------------------------------------------

def expm1div(c):
    """E(c) with the Taylor branch for |c| <= 2e-4 (section 5.6)."""
    c = np.asarray(c, dtype=np.float64)
    small = np.abs(c) <= 2e-4
    safe = np.where(small, 1.0, c)
    return np.where(small, 1.0 + c / 2.0 + c * c / 6.0, np.expm1(safe) / safe)


# ---------------------------------------------------------------------------
# Sections 4.1-4.3, 5.2-5.8: the solver
# ---------------------------------------------------------------------------

Field = Callable[[float, np.ndarray, np.ndarray], np.ndarray]


class StaggeredSolver:
    """The staggered-grid scheme of section 4 with the data layout of
    section 5: one 2D array per component, indexed [ix, iy].

    Parameters mirror the ``par`` struct of section 5.1: matrices Mx, My,
    mom_order, domain ax = (xmin, xmax, ymin, ymax), cells n = (nx, ny),
    bc = ('periodic'|'extrapolation', ...), CFL number cn, material fields
    sigma_a(t, x, y), sigma_s0(t, x, y), optional anisotropic factors
    (Sigma_sl = sigma_s0 * sl_factor[l], l >= 1), sources as a list of
    (component, q(t, x, y)), initial conditions as (component, f(x, y))."""

    def __init__(self, Mx, My, mom_order, ax, n, bc, cn=0.5,
                 sigma_a: Field = None, sigma_s0: Field = None,
                 sl_factor: Optional[Sequence[float]] = None,
                 sources: Sequence[Tuple[int, Field]] = (),
                 ic: Sequence[Tuple[int, Field]] = (),
                 time_dependent: bool = False, dt: Optional[float] = None,
                 frozen: Sequence[int] = (), pre_odd: Optional[Callable] = None):
        self.Mx = np.asarray(Mx, dtype=np.float64)
        self.My = np.asarray(My, dtype=np.float64)
        self.order = np.asarray(mom_order)
        self.ncomp = self.Mx.shape[0]
        self.ax = tuple(float(v) for v in ax)
        self.n = (int(n[0]), int(n[1]))
        self.p = tuple(1 if b == "periodic" else 0 for b in bc)  # eq. periodicity_flags
        self.h = ((self.ax[1] - self.ax[0]) / self.n[0], (self.ax[3] - self.ax[2]) / self.n[1])
        self.dt = time_step(self.Mx, self.ax, self.n, cn) if dt is None else float(dt)
        self.grid = assign_grids(self.Mx, self.My)
        self.sigma_a = sigma_a if sigma_a is not None else (lambda t, x, y: 0.0 * x)
        self.sigma_s0 = sigma_s0 if sigma_s0 is not None else (lambda t, x, y: 0.0 * x)
        self.sl_factor = sl_factor
        self.sources = list(sources)
        self.time_dependent = time_dependent
        self.t = 0.0
        self.nsteps_done = 0
        # Closure extension (not in the paper): components that the even
        # half-steps leave alone, and a hook that sets them from the state
        # right before every odd half-step.
        self.frozen = set(int(j) for j in frozen)
        self.pre_odd = pre_odd

        # Section 4.1: even components live on G11 u G22, odd on G21 u G12.
        self.even = [j for j in range(self.ncomp) if self.grid[j] in ((1, 1), (2, 2)) and j not in self.frozen]
        self.odd = [j for j in range(self.ncomp) if self.grid[j] in ((2, 1), (1, 2))]

        # eq. grid11 / staggered_grids: coordinates of the four grids
        self.coords = {}
        for gx in (1, 2):
            for gy in (1, 2):
                xs = self._axis_points(0, gx)
                ys = self._axis_points(1, gy)
                X, Y = np.meshgrid(xs, ys, indexing="ij")
                self.coords[(gx, gy)] = (X, Y)

        # Section 5.3: boundary index vectors (0-based)
        self.extend = []
        for d in range(2):
            nd = self.n[d]
            if self.p[d] == 1:
                e1 = np.concatenate([np.arange(nd), [0]])          # wrap G_1 -> G_2
                e2 = np.concatenate([[nd - 1], np.arange(nd)])      # wrap G_2 -> G_1
            else:
                e1 = np.concatenate([[0], np.arange(nd), [nd - 1]])  # ghost copies
                e2 = np.arange(nd + 1)
            self.extend.append({1: e1, 2: e2})

        # Section 5.2: one array per component, of its grid's size
        self.U = [np.zeros(self.coords[self.grid[j]][0].shape) for j in range(self.ncomp)]
        for j, f in ic:
            X, Y = self.coords[self.grid[j]]
            self.U[j] = np.array(f(0.0, X, Y), dtype=np.float64) * np.ones_like(X)
        self._materials_at = None

    def _axis_points(self, d: int, g: int) -> np.ndarray:
        lo = self.ax[2 * d]
        h = self.h[d]
        nd = self.n[d]
        if g == 1:
            return lo + (np.arange(1, nd + 1) - 0.5) * h          # (i - 1/2) h, i = 1..n
        return lo + np.arange(self.p[d], nd + 1) * h              # i h, i = p..n

    # -- section 5.7: material parameters and sources at t + dt/2 --------
    def _evaluate(self, tm: float):
        self.decay = []
        self.ET = []
        sA = {}
        sS0 = {}
        for g, (X, Y) in self.coords.items():
            sA[g] = np.asarray(self.sigma_a(tm, X, Y), dtype=np.float64) * np.ones_like(X)
            sS0[g] = np.asarray(self.sigma_s0(tm, X, Y), dtype=np.float64) * np.ones_like(X)
        for j in range(self.ncomp):
            g = self.grid[j]
            l = int(self.order[j])
            if l == 0:
                c = sA[g]                                       # Sigma_t0 = Sigma_a
            else:
                ssl = 0.0 if self.sl_factor is None else sS0[g] * self.sl_factor[l]
                c = sA[g] + sS0[g] - ssl                        # Sigma_tl
            self.decay.append(c)
            self.ET.append(expm1div(-c * self.dt / 2.0))       # E(-c dt/2)
        self.Q: Dict[int, np.ndarray] = {}
        for j, q in self.sources:
            X, Y = self.coords[self.grid[j]]
            val = np.asarray(q(tm, X, Y), dtype=np.float64) * np.ones_like(X)
            self.Q[j] = self.Q.get(j, 0.0) + val
        self._materials_at = tm

    # -- eq. central_differences via section 5.4 -------------------------
    def _differences(self, comps):
        dxU, dyU = {}, {}
        for k in comps:
            gx, gy = self.grid[k]
            dxU[k] = np.diff(self.U[k][self.extend[0][gx], :], axis=0) / self.h[0]
            dyU[k] = np.diff(self.U[k][:, self.extend[1][gy]], axis=1) / self.h[1]
        return dxU, dyU

    # -- eq. sub_step_solution as the update of section 5.5 --------------
    def _half_step(self, comps, dxU, dyU):
        for j in comps:
            W = np.zeros_like(self.U[j])
            for k in np.nonzero(self.Mx[j])[0]:
                W -= self.Mx[j, k] * dxU[k]
            for k in np.nonzero(self.My[j])[0]:
                W -= self.My[j, k] * dyU[k]
            Q = self.Q.get(j, 0.0)
            self.U[j] = self.U[j] + self.dt / 2.0 * (W + Q - self.decay[j] * self.U[j]) * self.ET[j]

    # -- eq. solution_operator_full_step ---------------------------------
    def step(self, reuse_closure: bool = False):
        """One full step O_1/2 E E O_1/2 (eq. solution_operator_full_step).
        reuse_closure: skip the pre_odd hook before the first odd half (its
        values from the previous step's second half are kept: the two odd
        halves then form one merged odd pass with one closure evaluation)."""
        tm = self.t + self.dt / 2.0
        if self._materials_at is None or self.time_dependent:
            self._evaluate(tm)
        inputs_even = self.even + sorted(self.frozen)
        if self.pre_odd is not None and not reuse_closure:
            self.pre_odd(self)
        dxU, dyU = self._differences(inputs_even)
        self._half_step(self.odd, dxU, dyU)
        dxU, dyU = self._differences(self.odd)     # computed once for both even halves
        self._half_step(self.even, dxU, dyU)
        self._half_step(self.even, dxU, dyU)
        if self.pre_odd is not None:
            self.pre_odd(self)
        dxU, dyU = self._differences(inputs_even)
        self._half_step(self.odd, dxU, dyU)
        self.t += self.dt
        self.nsteps_done += 1

    def run(self, nsteps: int, merged_closure: bool = False):
        """nsteps full steps.  merged_closure: the closure hook is evaluated
        once per merged odd pass -- before the first odd half of the run and
        before every second odd half, whose values the next step's first
        odd half reuses (the schedule O_1/2 (E O)^(n-1) E O_1/2 with one
        evaluation before each odd pass)."""
        for k in range(int(nsteps)):
            self.step(reuse_closure=merged_closure and k > 0)

    def run_to(self, t_final: float) -> List[np.ndarray]:
        """Step until t_final lies in (t, t + dt]; return the solution at
        t_final by linear interpolation in time (section 5.8)."""
        if t_final <= self.t:
            return [u.copy() for u in self.U]
        while True:
            old = [u.copy() for u in self.U]
            t0 = self.t
            self.step()
            if t0 < t_final <= self.t + 1e-14 * max(1.0, abs(t_final)):
                lam = (t_final - t0) / self.dt
                return [(1.0 - lam) * a + lam * b for a, b in zip(old, self.U)]

    # -- diagnostics (eq. L2_norm, eq. discrete_L2_norm) ----------------
    def mass(self) -> float:
        return float(np.sum(self.U[0]) * self.h[0] * self.h[1])

    def l2norm(self) -> float:
        return float(math.sqrt(sum(float(np.sum(u * u)) for u in self.U) * self.h[0] * self.h[1]))


def solver_from_problem(problem, **over) -> StaggeredSolver:
    """Build a StaggeredSolver from an input-module Problem description."""
    Mx, My, order = system_matrices(problem.system, problem.N)
    kw = dict(sigma_a=problem.sigma_a, sigma_s0=problem.sigma_s0,
              sl_factor=problem.sigma_sl_factor, sources=problem.sources,
              ic=problem.ic, time_dependent=problem.time_dependent)
    kw.update(over)
    return StaggeredSolver(Mx, My, order, problem.ax, problem.n, problem.bc,
                           problem.cn, **kw)
