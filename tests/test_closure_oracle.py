"""Pins of the closure oracle (CPU).  The learned mapping has no counterpart
in the paper; what is pinned is its arithmetic and its reduction to plain
P_7."""
import math

import numpy as np
import pytest

from oracle import closure_oracle as C
from oracle import pn_oracle as O
from paper_1211_2205_gb300 import inputs


def _problem(n=(20, 18), bc=("periodic", "extrapolation"), seed=4):
    ax = (0.0, 1.0, 0.0, 0.9)
    rng = inputs.SplitMix64(seed)
    return inputs.Problem(name="closure", N=7, ax=ax, n=n, bc=bc, precision="fp64",
                          sigma_a=inputs.piecewise_blocks(rng, 4, 0.0, 2.0, ax),
                          sigma_s0=inputs.piecewise_blocks(rng, 4, 0.5, 5.0, ax),
                          sources=[(0, inputs.gaussian_std(0.45, 0.4, 0.1))],
                          ic=[(0, inputs.gaussian_std(0.5, 0.5, 0.12)), (1, inputs.gaussian_std(0.3, 0.5, 0.1, 0.2))],
                          nsteps=6)


def test_order8_components_are_the_last_nine():
    comps = C.order8_components()
    assert comps == list(range(36, 45))
    kinds = [O.real_moments(8)[j][0] for j in comps]
    assert kinds == ["R", "I", "R", "I", "R", "I", "R", "I", "R"]


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("extrapolation", "extrapolation")])
def test_zero_network_reproduces_plain_p7(bc):
    p = _problem(bc=bc)
    mlp = C.MLP.init(1, scale_out=0.0)
    base = O.solver_from_problem(p)
    closed = C.closed_solver(p, mlp, dt=base.dt)
    base.run(p.nsteps)
    closed.run(p.nsteps)
    for j in range(36):
        np.testing.assert_allclose(closed.U[j], base.U[j], rtol=0, atol=1e-14 * np.max(np.abs(base.U[0])))
    for j in C.order8_components():
        assert not closed.U[j].any()


def test_nonzero_network_changes_only_through_order7():
    p = _problem()
    mlp = C.MLP.init(2, scale_out=0.3)
    base = O.solver_from_problem(p)
    closed = C.closed_solver(p, mlp, dt=base.dt)
    base.run(2)
    closed.run(2)
    # only the order-7 rows see the order-8 moments; the closed run differs
    # from plain P_7 but stays finite
    diff = max(float(np.max(np.abs(closed.U[j] - base.U[j]))) for j in range(36))
    assert diff > 0
    assert all(np.isfinite(closed.U[j]).all() for j in range(45))


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    mlp = C.MLP.init(3, scale_out=0.5)
    X = rng.normal(size=(7, C.N_IN))
    T = rng.normal(size=(7, C.N_OUT))
    loss, g = C.loss_and_grad(mlp, X, T)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        P = mlp.p[name]
        flat = P.reshape(-1)
        gflat = g[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = C.loss_and_grad(mlp, X, T)
            flat[idx] = old - h
            lm, _ = C.loss_and_grad(mlp, X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gflat[idx]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (name, idx)


def test_closure_is_positively_homogeneous():
    p = _problem()
    mlp = C.MLP.init(5, scale_out=0.4)
    s = C.closed_solver(p, mlp)
    s.run(1)
    X, Y = s.coords[(1, 1)]
    sa = p.sigma_a(0, X, Y)
    ss = p.sigma_s0(0, X, Y)
    hook = C.closure_hook(mlp, sa, ss)
    comps = C.order8_components()
    hook(s)
    ref = [s.U[j].copy() for j in comps]
    for j in range(36):
        s.U[j] *= 3.0         # positive scaling of every moment of order <= 7
    hook(s)
    for j, r in zip(comps, ref):
        np.testing.assert_allclose(s.U[j], 3.0 * r, rtol=1e-12, atol=1e-13 * np.max(np.abs(r)))


def test_cell_centre_interpolation_closed_form():
    # u = cos(k x) on a node axis averages to cos(k h / 2) cos(k x_c)
    Mx, My, order = O.system_matrices("pn2d", 3)
    n = 16
    L = 2.0
    k = 2 * math.pi * 3 / L
    for bc in ("periodic",):
        s = O.StaggeredSolver(Mx, My, order, (0, L, 0, L), (n, n), (bc, bc),
                              ic=[(j, lambda t, x, y: np.cos(k * x) * np.cos(k * y)) for j in range(10)])
        h = L / n
        Xc, Yc = s.coords[(1, 1)]
        expect = {(1, 1): 1.0, (2, 1): math.cos(k * h / 2), (1, 2): math.cos(k * h / 2),
                  (2, 2): math.cos(k * h / 2) ** 2}
        for j in range(10):
            got = C.to_cell_centres(s, j)
            np.testing.assert_allclose(got, expect[s.grid[j]] * np.cos(k * Xc) * np.cos(k * Yc), atol=1e-14)
        nodes = C.cell_centres_to_nodes(s, np.cos(k * Xc) * np.cos(k * Yc))
        X22, Y22 = s.coords[(2, 2)]
        np.testing.assert_allclose(nodes, math.cos(k * h / 2) ** 2 * np.cos(k * X22) * np.cos(k * Y22), atol=1e-14)


def test_adam_first_step_is_signed_learning_rate():
    params = {"w": np.array([1.0, -2.0, 0.5])}
    opt = C.Adam(params, lr=0.01)
    opt.step(params, {"w": np.array([3.0, -0.2, 0.0])})
    # bias-corrected first step: -lr * g / (|g| + eps)
    np.testing.assert_allclose(params["w"], [1.0 - 0.01, -2.0 + 0.01, 0.5], atol=1e-9)


def test_merged_closure_schedule_reuses_one_evaluation_per_odd_pass():
    """With the merged closure schedule the hook runs n + 1 times in n steps
    (literal: 2n); with a zero network both equal plain P_7."""
    p = _problem()
    calls = []
    mlp = C.MLP.init(3, scale_out=0.0)
    s = C.closed_solver(p, mlp)
    hook = s.pre_odd
    s.pre_odd = lambda st: (calls.append(st.t), hook(st))
    s.run(4, merged_closure=True)
    assert len(calls) == 5
    base = O.solver_from_problem(p, dt=s.dt)
    base.run(4)
    for j in range(36):
        np.testing.assert_allclose(s.U[j], base.U[j], rtol=0, atol=1e-14 * np.max(np.abs(base.U[0])))
    calls.clear()
    s.run(3)
    assert len(calls) == 6
