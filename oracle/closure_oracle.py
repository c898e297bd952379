"""FP64 oracle of the learned moment closure (not in the paper).

TEST INFRASTRUCTURE ONLY (tests/, the smoke check and bench.py's CPU legs).

The paper closes P_N by dropping every moment of order N+1 (eq. PN_slab and
the P_N matrices of section 3 truncate at l = N).  Its outlook (section 7)
names closures that add information at the highest order (FP_N, D_N); this
build replaces the zero truncation of P_7 by a per-cell multilayer perceptron
that predicts the order-8 moments from the local state:

* the closed system is the P_8 system of section 3 in which the even
  half-steps leave the nine order-8 components alone (R_8^{8,6,4,2,0} on G11,
  I_8^{8,6,4,2} on G22) and, right before every odd half-step, the network
  sets them from the current state -- so the order-7 rows see Mx/My entries
  of P_8 times predicted order-8 moments instead of zero;
* features at each cell centre (the points of G11): the 36 moments of order
  <= 7 averaged to the cell centre from their own staggered grid (two
  neighbours on G21 / G12, four on G22), divided by their RMS s, plus
  log(1 + sigma_a) and log(1 + sigma_s0); a cell whose largest moment
  magnitude is at most 1e-30 is empty: its moment features and s are 0;
* network: 38 -> 128 -> 128 -> 9, tanh hidden layers, linear output; the
  prediction is s * y (positively homogeneous in the moments, as the linear
  transport equation is);
* R_8^m are written at the cell centres, I_8^m at the G22 points as the mean
  of the four surrounding cell-centre predictions (boundary cells copied for
  extrapolation boundaries, wrapped for periodic ones);
* schedules: literal -- the network runs before every odd half-step;
  merged -- consecutive odd halves form one odd pass with one evaluation
  (StaggeredSolver.run(n, merged_closure=True)).

Functions here follow that definition step by step in FP64.  The learned
mapping itself has no counterpart in the paper: its parity is unpinned
beyond the pins in tests/test_closure_oracle.py (zero network = plain P_7,
finite-difference gradients, homogeneity, closed-form interpolation).
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import pn_oracle as O

N_BASE = 7
N_CLOSED = 8
N_FEAT_MOM = (N_BASE + 1) * (N_BASE + 2) // 2      # 36
N_OUT = N_CLOSED + 1                                 # 9 moments of order 8
N_IN = N_FEAT_MOM + 2                                # 38
HIDDEN = 128
EMPTY = 1e-30          # largest moment magnitude of an empty cell


def order8_components() -> List[int]:
    """Indices of the order-8 components in the P_8 real ordering."""
    return [j for j, (_, l, _) in enumerate(O.real_moments(N_CLOSED)) if l == N_CLOSED]


def to_cell_centres(s: O.StaggeredSolver, j: int) -> np.ndarray:
    """Component j averaged to the cell centres (points of G11), [nx, ny]."""
    U = s.U[j]
    gx, gy = s.grid[j]
    if gx == 2:        # nodes in x: mean of the two nodes around each centre
        E = U[s.extend[0][2], :]
        U = 0.5 * (E[:-1, :] + E[1:, :])
    if gy == 2:
        E = U[:, s.extend[1][2]]
        U = 0.5 * (E[:, :-1] + E[:, 1:])
    return U


def cell_centres_to_nodes(s: O.StaggeredSolver, C: np.ndarray) -> np.ndarray:
    """Cell-centre field [nx, ny] to the points of G22: mean of the four
    surrounding cells (boundary cells copied / wrapped as in section 4.2)."""
    E = C[s.extend[0][1], :]
    C2 = 0.5 * (E[:-1, :] + E[1:, :])
    E = C2[:, s.extend[1][1]]
    return 0.5 * (E[:, :-1] + E[:, 1:])


def features(s: O.StaggeredSolver, sigma_a_cc: np.ndarray, sigma_s0_cc: np.ndarray):
    """Network inputs X [M, 38] and scales [M] at the M = nx*ny cell centres,
    cell index = iy * nx + ix."""
    u = np.stack([to_cell_centres(s, j).T.ravel() for j in range(N_FEAT_MOM)], axis=1)
    empty = np.max(np.abs(u), axis=1) <= EMPTY
    scale = np.where(empty, 0.0, np.sqrt(np.mean(u * u, axis=1)))
    inv = np.where(empty, 0.0, 1.0 / np.where(empty, 1.0, scale))
    X = np.concatenate([u * inv[:, None],
                        np.log1p(sigma_a_cc.T.ravel())[:, None],
                        np.log1p(sigma_s0_cc.T.ravel())[:, None]], axis=1)
    return X, scale


def targets(s: O.StaggeredSolver) -> np.ndarray:
    """Order-8 moments of a P_N run (N >= 8) at the cell centres, [M, 9]."""
    return np.stack([to_cell_centres(s, j).T.ravel() for j in order8_components()], axis=1)


class MLP:
    """38 -> 128 -> 128 -> 9 perceptron with tanh hidden layers."""

    def __init__(self, params: Dict[str, np.ndarray]):
        self.p = {k: np.asarray(v, dtype=np.float64) for k, v in params.items()}

    @staticmethod
    def init(seed: int, scale_out: float = 1.0) -> "MLP":
        rng = np.random.default_rng(seed)
        p = {
            "W1": rng.normal(0, 1 / math.sqrt(N_IN), (HIDDEN, N_IN)),
            "b1": np.zeros(HIDDEN),
            "W2": rng.normal(0, 1 / math.sqrt(HIDDEN), (HIDDEN, HIDDEN)),
            "b2": np.zeros(HIDDEN),
            "W3": scale_out * rng.normal(0, 1 / math.sqrt(HIDDEN), (N_OUT, HIDDEN)),
            "b3": np.zeros(N_OUT),
        }
        return MLP(p)

    def forward(self, X: np.ndarray):
        p = self.p
        H1 = np.tanh(X @ p["W1"].T + p["b1"])
        H2 = np.tanh(H1 @ p["W2"].T + p["b2"])
        Y = H2 @ p["W3"].T + p["b3"]
        return Y, (X, H1, H2)

    def backward(self, cache, dY: np.ndarray) -> Dict[str, np.ndarray]:
        X, H1, H2 = cache
        p = self.p
        g = {"W3": dY.T @ H2, "b3": dY.sum(axis=0)}
        dZ2 = (dY @ p["W3"]) * (1.0 - H2 * H2)
        g["W2"] = dZ2.T @ H1
        g["b2"] = dZ2.sum(axis=0)
        dZ1 = (dZ2 @ p["W2"]) * (1.0 - H1 * H1)
        g["W1"] = dZ1.T @ X
        g["b1"] = dZ1.sum(axis=0)
        return g


def loss_and_grad(mlp: MLP, X: np.ndarray, T_scaled: np.ndarray):
    """Mean squared error over samples and outputs, and its gradient."""
    Y, cache = mlp.forward(X)
    R = Y - T_scaled
    M = X.shape[0]
    loss = float(np.sum(R * R) / (M * N_OUT))
    dY = 2.0 * R / (M * N_OUT)
    return loss, mlp.backward(cache, dY)


class Adam:
    """Adam (Kingma & Ba, 2015) on FP64 parameters."""

    def __init__(self, params: Dict[str, np.ndarray], lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in params.items()}
        self.v = {k: np.zeros_like(v) for k, v in params.items()}
        self.t = 0

    def step(self, params: Dict[str, np.ndarray], grads: Dict[str, np.ndarray]):
        self.t += 1
        for k in params:
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * grads[k]
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * grads[k] ** 2
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            params[k] -= self.lr * mh / (np.sqrt(vh) + self.eps)


def closure_hook(mlp: MLP, sigma_a_cc: np.ndarray, sigma_s0_cc: np.ndarray):
    """pre_odd hook of a P_8 StaggeredSolver: set the order-8 components from
    the network's prediction at the cell centres."""
    comps = order8_components()
    kinds = [k for (k, l, _) in O.real_moments(N_CLOSED) if l == N_CLOSED]

    def hook(s: O.StaggeredSolver):
        X, scale = features(s, sigma_a_cc, sigma_s0_cc)
        Y, _ = mlp.forward(X)
        P = Y * scale[:, None]
        nx, ny = s.n
        for k, (j, kind) in enumerate(zip(comps, kinds)):
            C = P[:, k].reshape(ny, nx).T                    # [nx, ny] at cell centres
            s.U[j] = C.copy() if kind == "R" else cell_centres_to_nodes(s, C)
    return hook


def closed_solver(problem, mlp: MLP, dt: Optional[float] = None) -> O.StaggeredSolver:
    """P_8 solver with the order-8 moments frozen in the even half-steps and
    set by the network before each odd half-step."""
    Mx, My, order = O.system_matrices("pn2d", N_CLOSED)
    s = O.StaggeredSolver(Mx, My, order, problem.ax, problem.n, problem.bc, problem.cn,
                          sigma_a=problem.sigma_a, sigma_s0=problem.sigma_s0,
                          sl_factor=problem.sigma_sl_factor, sources=problem.sources, ic=problem.ic,
                          time_dependent=problem.time_dependent, dt=dt, frozen=order8_components())
    X, Y = s.coords[(1, 1)]
    sa = np.asarray(problem.sigma_a(0.0, X, Y), dtype=np.float64) * np.ones_like(X)
    ss = np.asarray(problem.sigma_s0(0.0, X, Y), dtype=np.float64) * np.ones_like(X)
    s.pre_odd = closure_hook(mlp, sa, ss)
    return s
