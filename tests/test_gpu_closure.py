"""GPU parity of the learned order-8 closure and of its network kernels
against the FP64 closure oracle.

The network runs with BF16 operands and FP32 accumulation; the oracle gets
the same BF16-rounded weights (and, for the plain network tests, the same
BF16-rounded inputs), so what remains is the rounding of the hidden
activations and of the backward intermediates to BF16: bar 1e-2 relative
per tensor.  The features, the node averaging and the coupling into the
P_8 step are plain FP32/FP64 arithmetic and are held to those precisions."""
import math

import numpy as np
import pytest

from helpers import DT_RTOL, assert_parity, check_dt, rel_l2
from oracle import closure_oracle as C
from oracle import pn_oracle as O
from paper_1211_2205_gb300 import capi, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BF16_TOL = 1e-2


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _params(seed, scale_out=1.0, bias=0.1):
    mlp = C.MLP.init(seed, scale_out=scale_out)
    rng = np.random.default_rng(seed + 1000)
    for k in ("b1", "b2", "b3"):
        mlp.p[k] = rng.normal(0, bias, mlp.p[k].shape)
    return capi.params_from_dict(mlp.p)


def _oracle_mlp(params32):
    """The oracle network with the GPU's BF16 weights (biases stay FP32)."""
    d = capi.params_to_dict(params32)
    for k in ("W1", "W2", "W3"):
        d[k] = bf16(d[k]).astype(np.float64)
    return C.MLP(d)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(got, ref):
    return float(np.linalg.norm(np.asarray(got, np.float64) - ref) / max(np.linalg.norm(ref), 1e-300))


@pytest.mark.parametrize("M", [1, 127, 1000])
def test_forward_matches_oracle(M):
    rng = np.random.default_rng(M)
    X = rng.normal(size=(M, C.N_IN)).astype(np.float32)
    params = _params(3)
    net = capi.Network(params)
    Xd, Yd = _dev(X), torch.full((M * C.N_OUT,), float("nan"), device="cuda")
    torch.cuda.synchronize()
    net.forward(Xd, M, Yd)
    net.sync()
    Y = Yd.cpu().numpy().reshape(M, C.N_OUT)
    ref, _ = _oracle_mlp(params).forward(bf16(X).astype(np.float64))
    assert np.isfinite(Y).all()
    assert _rel(Y, ref) <= BF16_TOL
    assert np.max(np.abs(Y - ref)) <= 3 * BF16_TOL * np.max(np.abs(ref))


ENGINES = ["mma_sync", "tcgen05"]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("Mall,B", [(1000, 700), (300, 128), (300, 129), (50, 1)])
def test_gradients_match_oracle(engine, Mall, B):
    """Loss and gradient of a minibatch given by an index list (700 of 1000
    samples: five full tiles and a ragged one; one whole tile; a tile and
    one sample; a single sample) against the oracle's backward with the
    same BF16 weights and inputs, on both engines (the tcgen05 kernel reads
    the activations MN-major for the weight gradients and takes the bias
    gradients from ones columns)."""
    rng = np.random.default_rng(11 + B)
    X = rng.normal(size=(Mall, C.N_IN)).astype(np.float32)
    T = rng.normal(size=(Mall, C.N_OUT)).astype(np.float32)
    idx = rng.permutation(Mall)[:B].astype(np.int32)
    params = _params(5, scale_out=0.7)
    net = capi.Network(params)
    net.set_engine(engine)
    g = torch.zeros(capi.MLP_PARAMS, device="cuda")
    loss = torch.zeros(1, device="cuda")
    Xd, Td, Id = _dev(X), _dev(T), _dev(idx)
    torch.cuda.synchronize()
    net.loss_grad(Xd, Td, B, g, loss, idx=Id)
    net.sync()
    got = capi.params_to_dict(g.cpu().numpy())
    ref_loss, ref = C.loss_and_grad(_oracle_mlp(params), bf16(X[idx]).astype(np.float64), T[idx].astype(np.float64))
    assert abs(float(loss.item()) - ref_loss) <= BF16_TOL * ref_loss
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert _rel(got[k], ref[k]) <= BF16_TOL, k


def test_engines_give_the_same_gradient():
    """The tcgen05 and mma.sync training kernels compute the same products of
    the same BF16 operands; only the FP32 summation order differs."""
    rng = np.random.default_rng(15)
    M = 3000
    X = _dev(rng.normal(size=(M, C.N_IN)).astype(np.float32))
    T = _dev(rng.normal(size=(M, C.N_OUT)).astype(np.float32))
    params = _params(8, scale_out=0.5)
    got = {}
    for engine in ENGINES:
        net = capi.Network(params)
        net.set_engine(engine)
        g = torch.zeros(capi.MLP_PARAMS, device="cuda")
        loss = torch.zeros(1, device="cuda")
        torch.cuda.synchronize()
        net.loss_grad(X, T, M, g, loss)
        net.sync()
        got[engine] = (g.cpu().numpy().astype(np.float64), float(loss.item()))
        net.close()
    (ga, la), (gb, lb) = got["mma_sync"], got["tcgen05"]
    assert abs(la - lb) <= 1e-4 * abs(la)
    da, db = capi.params_to_dict(ga), capi.params_to_dict(gb)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert _rel(db[k], da[k]) <= 2e-3, k


@pytest.mark.parametrize("engine", ENGINES)
def test_gradient_is_deterministic(engine):
    rng = np.random.default_rng(12)
    X = rng.normal(size=(900, C.N_IN)).astype(np.float32)
    T = rng.normal(size=(900, C.N_OUT)).astype(np.float32)
    net = capi.Network(_params(6))
    net.set_engine(engine)
    Xd, Td = _dev(X), _dev(T)
    g1 = torch.zeros(capi.MLP_PARAMS, device="cuda")
    g2 = torch.zeros(capi.MLP_PARAMS, device="cuda")
    torch.cuda.synchronize()
    net.loss_grad(Xd, Td, 900, g1)
    net.loss_grad(Xd, Td, 900, g2)
    net.sync()
    assert torch.equal(g1, g2)


@pytest.mark.parametrize("engine", ENGINES)
def test_adam_steps_match_oracle_optimizer(engine):
    """Three Adam steps on the GPU against the oracle's Adam fed with the
    GPU's own gradients (the optimiser arithmetic in isolation)."""
    rng = np.random.default_rng(13)
    X = rng.normal(size=(512, C.N_IN)).astype(np.float32)
    T = rng.normal(size=(512, C.N_OUT)).astype(np.float32)
    params = _params(7)
    net = capi.Network(params)
    net.set_engine(engine)
    ref = capi.params_to_dict(params)
    opt = C.Adam(ref, lr=2e-3)
    Xd, Td = _dev(X), _dev(T)
    g = torch.zeros(capi.MLP_PARAMS, device="cuda")
    torch.cuda.synchronize()
    for _ in range(3):
        net.loss_grad(Xd, Td, 512, g)
        net.sync()
        gd = capi.params_to_dict(g.cpu().numpy())
        net.train_step(Xd, Td, 512, 2e-3)
        net.sync()
        opt.step(ref, gd)
    assert net.steps == 3
    np.testing.assert_allclose(net.params, capi.params_from_dict(ref), rtol=0, atol=2e-6)


@pytest.mark.parametrize("engine", ENGINES)
def test_training_fits_a_teacher_network(engine):
    """Minibatch Adam on the GPU learns the map of another network."""
    rng = np.random.default_rng(14)
    M = 8192
    X = rng.normal(size=(M, C.N_IN)).astype(np.float32)
    teacher = C.MLP(capi.params_to_dict(_params(21, scale_out=1.0)))
    T = teacher.forward(X.astype(np.float64))[0].astype(np.float32)
    net = capi.Network(_params(22, scale_out=0.1))
    net.set_engine(engine)
    Xd, Td = _dev(X), _dev(T)
    loss = torch.zeros(1, device="cuda")
    torch.cuda.synchronize()
    net.loss_grad(Xd, Td, M, torch.zeros(capi.MLP_PARAMS, device="cuda"), loss)
    net.sync()
    first = float(loss.item())
    perm = _dev(np.concatenate([rng.permutation(M) for _ in range(40)]).astype(np.int32))
    B = 1024
    for it in range(320):
        net.train_step(Xd, Td, B, 3e-3, idx=perm[it * B:(it + 1) * B])
    net.loss_grad(Xd, Td, M, torch.zeros(capi.MLP_PARAMS, device="cuda"), loss)
    net.sync()
    assert float(loss.item()) < 0.2 * first


# ----------------------------------------------------------- closure in the step
def _closure_problem(n=(37, 29), bc=("periodic", "extrapolation"), precision="fp64", N=7, seed=31, nsteps=4):
    ax = (0.0, 1.1, 0.0, 1.1 * n[1] / n[0])
    rng = inputs.SplitMix64(seed)
    ncomp = (N + 1) * (N + 2) // 2
    ic = []
    for j in range(min(ncomp, 36)):
        c = rng.uniforms(3)
        ic.append((j, inputs.gaussian_std(0.2 + 0.7 * c[0], 0.2 + 0.5 * c[1], 0.12 + 0.1 * c[2],
                                          mass=(-1) ** j / (1 + j // 6))))
    return inputs.Problem(name="closure", N=N, ax=ax, n=n, bc=bc, precision=precision,
                          sigma_a=inputs.piecewise_blocks(rng, 4, 0.0, 2.0, ax),
                          sigma_s0=inputs.piecewise_blocks(rng, 4, 0.2, 4.0, ax),
                          sources=[(0, inputs.gaussian_std(0.5, 0.45, 0.1))], ic=ic, nsteps=nsteps)


def _state(s):
    return [s.moments(j) for j in range(s.ncomp)]


def _closed_dt(s, p):
    """The oracle's step size of the closed system (P_8's lambda_max, the
    rule of section 4.5), checked against the closure handle's."""
    Mx, _, _ = O.system_matrices("pn2d", C.N_CLOSED)
    d = O.time_step(Mx, p.ax, p.n, p.cn)
    assert abs(s.dt - d) <= DT_RTOL * d, (s.dt, d)
    return d


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("extrapolation", "extrapolation"),
                                ("periodic", "extrapolation")])
@pytest.mark.parametrize("precision,kernel", [("fp64", "gather"), ("fp32", "tiled")])
def test_samples_match_oracle_features_and_targets(bc, precision, kernel):
    """Features, scales and order-8 targets of a plain P_8 run (two steps)
    against the oracle's definitions on the oracle's own run."""
    p = _closure_problem(bc=bc, precision=precision, N=8, nsteps=2)
    s = capi.Stepper.from_problem(p, kernel=kernel)
    s.step(2)
    o = O.solver_from_problem(p, dt=check_dt(s, p))
    o.run(2)
    X0, Y0 = o.coords[(1, 1)]
    Xr, scale_r = C.features(o, p.sigma_a(0, X0, Y0), p.sigma_s0(0, X0, Y0))
    Tr = C.targets(o)
    M = p.n[0] * p.n[1]
    Xd = torch.empty(M * C.N_IN, device="cuda")
    Sd = torch.empty(M, device="cuda")
    Td = torch.empty(M * C.N_OUT, device="cuda")
    torch.cuda.synchronize()
    s.closure_samples(Xd, Sd, Td)
    s.sync()
    tol = 2e-6 if precision == "fp64" else 2e-5
    assert _rel(Sd.cpu().numpy(), scale_r) <= tol
    assert _rel(Xd.cpu().numpy().reshape(M, C.N_IN), Xr) <= tol
    assert _rel(Td.cpu().numpy().reshape(M, C.N_OUT), Tr / scale_r[:, None]) <= tol


@pytest.mark.parametrize("schedule", ["literal", "merged"])
@pytest.mark.parametrize("precision,kernel,tol", [("fp64", "gather", 1e-12), ("fp32", "tiled", 1e-5)])
def test_zero_network_is_plain_p7(precision, kernel, tol, schedule):
    """A network with zero output layer predicts zero order-8 moments: the
    closed run equals plain P_7 (oracle) with the same dt."""
    p = _closure_problem(precision=precision)
    s = capi.Stepper.from_problem(p, kernel=kernel, closure="mlp8", schedule=schedule)
    assert s.ncomp == 45
    params = _params(40)
    params[-(C.N_OUT * C.HIDDEN + C.N_OUT):] = 0.0          # W3 and b3
    s.set_closure(params)
    s.step(p.nsteps)
    got = _state(s)
    o = O.solver_from_problem(p, dt=_closed_dt(s, p))
    o.run(p.nsteps)
    assert_parity(got[:36], [u.T for u in o.U], tol, precision)
    for j in range(36, 45):
        assert not got[j].any()


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("extrapolation", "extrapolation")])
def test_closure_prediction_matches_oracle_hook(bc):
    """One odd pass of a closure handle sets the order-8 moments from the
    state before it; they match the oracle's closure on that same state."""
    p = _closure_problem(bc=bc, nsteps=3)
    params = _params(41, scale_out=0.6)
    s = capi.Stepper.from_problem(p, kernel="gather", closure="mlp8")
    s.set_closure(params)
    s.step(3)
    before = _state(s)
    s.run_pass(1, 0)
    after = _state(s)
    o = C.closed_solver(p, _oracle_mlp(params), dt=_closed_dt(s, p))
    for j in range(45):
        o.U[j] = before[j].T.copy()
    o.pre_odd(o)
    ref = [o.U[j].T for j in range(36, 45)]
    assert rel_l2(after[36:], ref) <= 2 * BF16_TOL
    assert max(float(np.max(np.abs(r))) for r in ref) > 0


@pytest.mark.parametrize("schedule", ["literal", "merged"])
@pytest.mark.parametrize("precision,kernel", [("fp64", "gather"), ("fp32", "tiled")])
def test_closed_run_matches_oracle(precision, kernel, schedule):
    """A closed run against the oracle's closed run (same closure schedule):
    the difference stays a small fraction of what the closure changes
    relative to plain P_7."""
    p = _closure_problem(precision=precision, nsteps=5)
    params = _params(42, scale_out=0.6)
    s = capi.Stepper.from_problem(p, kernel=kernel, closure="mlp8", schedule=schedule)
    s.set_closure(params)
    s.step(p.nsteps)
    got = _state(s)
    o = C.closed_solver(p, _oracle_mlp(params), dt=_closed_dt(s, p))
    o.run(p.nsteps, merged_closure=schedule == "merged")
    plain = O.solver_from_problem(p, dt=_closed_dt(s, p))
    plain.run(p.nsteps)
    ref = [u.T for u in o.U[:36]]
    effect = rel_l2([u.T for u in plain.U], ref)
    assert effect > 1e-6
    # the BF16 activations of the GPU network against the oracle's FP64 ones:
    # measured 0.8 % (literal) and 1.0 % (merged) of the closure's effect
    assert rel_l2(got[:36], ref) <= 0.02 * effect


def test_closure_errors():
    p = _closure_problem()
    with pytest.raises(capi.StarmapError) as e:
        capi.Stepper(N=5, ax=p.ax, n=p.n, closure="mlp8")
    assert e.value.code == capi.E_UNSUPPORTED
    s = capi.Stepper(N=7, ax=p.ax, n=p.n, closure="mlp8")
    with pytest.raises(capi.StarmapError) as e:
        s.step(1)
    assert e.value.code == capi.E_STATE
    with pytest.raises(ValueError):
        s.set_closure(np.zeros(10))
    bad = _params(1)
    bad[5] = np.nan
    with pytest.raises(capi.StarmapError) as e:
        s.set_closure(bad)
    assert e.value.code == capi.E_NONFINITE
    with pytest.raises(capi.StarmapError) as e:
        s.set_source(40, np.ones(p.n[0] * p.n[1]))
    assert e.value.code == capi.E_ARG
    plain = capi.Stepper(N=7, ax=p.ax, n=p.n)
    with pytest.raises(capi.StarmapError) as e:
        plain.set_closure(_params(1))
    assert e.value.code == capi.E_STATE


# ----------------------------------------------------------- tcgen05 engine
@pytest.mark.parametrize("M", [1, 127, 1000, 40000])
def test_tcgen05_forward_matches_oracle_and_mma_sync(M):
    """The tcgen05 network (TMEM accumulators, shared-memory operands) against
    the oracle with the same BF16 weights and inputs, and against the
    mma.sync network: the same per-element arithmetic up to the FP32
    summation order (an occasional hidden activation may round to the
    neighbouring BF16 value)."""
    rng = np.random.default_rng(100 + M)
    X = rng.normal(size=(M, C.N_IN)).astype(np.float32)
    params = _params(8)
    net = capi.Network(params)
    Xd = _dev(X)
    Yt = torch.full((M * C.N_OUT,), float("nan"), device="cuda")
    Ym = torch.full((M * C.N_OUT,), float("nan"), device="cuda")
    torch.cuda.synchronize()
    net.set_engine("tcgen05")
    net.forward(Xd, M, Yt)
    net.sync()
    net.set_engine("mma_sync")
    net.forward(Xd, M, Ym)
    net.sync()
    yt = Yt.cpu().numpy().reshape(M, C.N_OUT)
    ym = Ym.cpu().numpy().reshape(M, C.N_OUT)
    ref, _ = _oracle_mlp(params).forward(bf16(X).astype(np.float64))
    assert np.isfinite(yt).all()
    assert _rel(yt, ref) <= BF16_TOL
    assert _rel(yt, ym) <= 2e-3


@pytest.mark.parametrize("bc,n", [(("periodic", "periodic"), (150, 90)), (("extrapolation", "periodic"), (150, 90)),
                                  # one partial tile; exactly 32 whole tiles; 469 tiles over 118 CTAs (3-4 each,
                                  # so consumers and producers run uneven counts)
                                  (("periodic", "extrapolation"), (10, 7)), (("periodic", "periodic"), (64, 64)),
                                  (("extrapolation", "extrapolation"), (200, 300))])
def test_tcgen05_closure_prediction_matches_oracle_hook(bc, n):
    """The fused closure kernel's prediction of the order-8 moments against
    the oracle's hook on the same state: tile counts from one partial tile to
    several per CTA, each consumer group fed by its producer group."""
    p = _closure_problem(bc=bc, nsteps=3, n=n)
    params = _params(43, scale_out=0.6)
    s = capi.Stepper.from_problem(p, kernel="gather", closure="mlp8")
    s.set_closure(params)
    s.set_closure_engine("tcgen05")
    s.step(3)
    before = _state(s)
    s.run_pass(1, 0)
    after = _state(s)
    s.sync()
    o = C.closed_solver(p, _oracle_mlp(params), dt=_closed_dt(s, p))
    for j in range(45):
        o.U[j] = before[j].T.copy()
    o.pre_odd(o)
    ref = [o.U[j].T for j in range(36, 45)]
    assert rel_l2(after[36:], ref) <= 2 * BF16_TOL


def test_tcgen05_closure_prediction_full_size():
    """The closure workload's own size and launch configuration: one medium
    of the benchmark's closure runs (512 x 512, P_8 state after a few plain
    closed steps), the tcgen05 prediction of all nine order-8 moments on every
    cell against the oracle's hook on the same state."""
    p = inputs.closure_medium(100, n=512, N=7)
    p = inputs.Problem(**{**p.__dict__, "nsteps": 3})
    params = _params(45, scale_out=0.6)
    s = capi.Stepper.from_problem(p, kernel="tiled", closure="mlp8", schedule="merged")
    s.set_closure(params)
    s.set_closure_engine("tcgen05")
    s.step(3)
    before = _state(s)
    s.run_pass(1, 0)
    after = _state(s)
    s.sync()
    o = C.closed_solver(p, _oracle_mlp(params), dt=_closed_dt(s, p))
    for j in range(45):
        o.U[j] = before[j].T.astype(np.float64)
    o.pre_odd(o)
    ref = [o.U[j].T for j in range(36, 45)]
    assert rel_l2(after[36:], ref) <= 2 * BF16_TOL


def test_tcgen05_closed_run_matches_mma_sync_run():
    p = _closure_problem(precision="fp32", nsteps=6, n=(130, 70))
    params = _params(44, scale_out=0.6)
    runs = []
    for engine in ("mma_sync", "tcgen05"):
        s = capi.Stepper.from_problem(p, kernel="tiled", closure="mlp8", schedule="merged")
        s.set_closure(params)
        s.set_closure_engine(engine)
        s.step(p.nsteps)
        s.sync()
        runs.append(_state(s))
    plain = O.solver_from_problem(p, dt=_closed_dt(s, p))
    plain.run(p.nsteps)
    effect = rel_l2([u.T for u in plain.U], runs[0][:36])
    assert rel_l2(runs[1][:36], runs[0][:36]) <= 0.05 * effect


def test_input_noise_is_gaussian_and_reproducible():
    """Training-input noise: the first 36 inputs get N(0, sigma^2) noise from
    a counter-based stream (same seed, same noise), the two material inputs
    are copied exactly; in place gives the same result."""
    M, sigma = 200000, 0.1
    rng = np.random.default_rng(7)
    X = rng.normal(size=(M, C.N_IN)).astype(np.float32)
    net = capi.Network(_params(3))
    Xd = _dev(X)
    A = torch.empty_like(Xd)
    B = torch.empty_like(Xd)
    D = torch.empty_like(Xd)
    torch.cuda.synchronize()
    net.perturb_inputs(Xd, A, M, 36, sigma, 11)
    net.perturb_inputs(Xd, B, M, 36, sigma, 11)
    net.perturb_inputs(Xd, D, M, 36, sigma, 12)
    net.sync()
    a, b, d = A.cpu().numpy(), B.cpu().numpy(), D.cpu().numpy()
    assert np.array_equal(a, b) and not np.array_equal(a, d)
    assert np.array_equal(a[:, 36:], X[:, 36:])
    n = (a[:, :36].astype(np.float64) - X[:, :36]) / sigma
    k = n.size
    assert abs(n.mean()) < 5 / math.sqrt(k)
    assert abs(n.std() - 1.0) < 5e-3
    assert abs(np.mean(np.abs(n) < 1.0) - 0.682689) < 3e-3          # normal, not uniform or clipped
    assert abs(np.mean(np.abs(n) < 2.0) - 0.954500) < 2e-3
    assert abs(float(np.corrcoef(n[:, 0], n[:, 1])[0, 1])) < 0.02      # independent across columns
    # the definition: SplitMix64's finaliser of seed * golden + element
    # index, two 32-bit halves, Box-Muller (recomputed here in float64)
    mask = (1 << 64) - 1
    for e in (0, 1, 37, 38 * 1000 + 5, 38 * (M - 1) + 35):
        z = (11 * 0x9E3779B97F4A7C15 + e + 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z ^= z >> 31
        u1 = ((z >> 32) + 0.5) * 2.0 ** -32
        u2 = ((z & 0xFFFFFFFF) + 0.5) * 2.0 ** -32
        g = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
        m, c = divmod(e, C.N_IN)
        want = float(X[m, c]) + (sigma * g if c < 36 else 0.0)       # the material inputs stay exact
        assert abs(float(a[m, c]) - want) <= 2e-6 * (1 + abs(g)), e
    net.perturb_inputs(Xd, Xd, M, 36, sigma, 11)                      # in place
    net.sync()
    assert np.array_equal(Xd.cpu().numpy(), a)
    with pytest.raises(capi.StarmapError):
        net.perturb_inputs(Xd, A, M, 39, sigma, 1)


@pytest.mark.parametrize("schedule", ["literal", "merged"])
def test_closed_run_same_on_both_tile_heights(schedule):
    """The frozen order-8 outputs and the closure's inputs do not depend on
    the tile shape: a closed run on 64 x 5 tiles equals the one on 64 x 10
    tiles bit for bit."""
    p = _closure_problem(precision="fp32", nsteps=4, n=(130, 70), bc=("extrapolation", "periodic"))
    params = _params(45, scale_out=0.6)
    runs = []
    for kernel in ("tiled_tall", "tiled_short"):
        s = capi.Stepper.from_problem(p, kernel=kernel, closure="mlp8", schedule=schedule)
        assert s.tile_rows == (10 if kernel == "tiled_tall" else 5)
        s.set_closure(params)
        s.step(p.nsteps)
        s.sync()
        runs.append(_state(s))
        s.close()
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def test_epoch_shuffle_is_a_seeded_permutation():
    """The device-side epoch order: a permutation of range(count) (also for
    counts just above and below a power of four, where the cycle walk is
    longest or absent), the same for the same seed, another for another
    seed, and index[perm] when an index is given."""
    net = capi.Network(_params(3))
    for count in (1, 2, 3, 1000, 4096, 4097, 65535, 1 << 20):
        out = torch.empty(count, dtype=torch.int32, device="cuda")
        net.shuffle(None, count, 7, out)
        net.sync()
        a = out.cpu().numpy()
        assert np.array_equal(np.sort(a), np.arange(count)), count
        if count >= 1000:
            assert not np.array_equal(a, np.arange(count))
            # no long runs of neighbours: the order is scrambled
            assert np.mean(np.abs(np.diff(a.astype(np.int64))) == 1) < 0.01
    count = 1 << 16
    outs = []
    for seed in (5, 5, 6):
        out = torch.empty(count, dtype=torch.int32, device="cuda")
        net.shuffle(None, count, seed, out)
        net.sync()
        outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert np.mean(outs[0] == outs[2]) < 0.01
    index = torch.from_numpy(np.random.default_rng(1).permutation(10 * count)[:count].astype(np.int32)).cuda()
    out = torch.empty(count, dtype=torch.int32, device="cuda")
    net.shuffle(index, count, 5, out)
    net.sync()
    assert np.array_equal(out.cpu().numpy(), index.cpu().numpy()[outs[0]])
    with pytest.raises(capi.StarmapError) as e:
        net.shuffle(None, 10, 1, None)
    assert e.value.code == capi.E_ARG
    net.close()
