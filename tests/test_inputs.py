"""CPU tests of the seeded input generators (the workload recipes): the
SplitMix64 stream against its published reference outputs, and the ranges,
counts and determinism each workload's description states."""
import numpy as np

from paper_1211_2205_gb300 import inputs


def test_splitmix64_reference_outputs():
    """SplitMix64 (Steele, Lea & Flood 2014) seeded with 0: the first three
    outputs of the published reference generator."""
    r = inputs.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniforms_in_unit_interval():
    u = inputs.SplitMix64(5).uniforms(100000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    a, b = inputs.SplitMix64(5).uniforms(10), inputs.SplitMix64(6).uniforms(10)
    assert np.array_equal(a, u[:10]) and not np.array_equal(a, b)


def test_checkerboard_layout():
    """7 x 7 blocks, the centre block is the source (not absorbing), 11 of
    the 48 outer blocks absorbing, the same for the same seed."""
    f = inputs.checkerboard_layout(1211)
    assert f.shape == (7, 7) and f[3, 3] == 0
    assert int(f.sum()) == 11 and set(np.unique(f)) <= {0, 1}
    assert np.array_equal(f, inputs.checkerboard_layout(1211))
    assert not np.array_equal(f, inputs.checkerboard_layout(1212))
    p = inputs.checkerboard_p13(n=70)
    x = np.array([3.5, 0.5, 6.5])
    y = np.array([3.5, 0.5, 6.5])
    q = p.sources[0][1](0.0, x, y)
    assert q[0] == 1.0 and q[1] == 0.0 and q[2] == 0.0       # unit source in the centre block only
    sa, ss = p.sigma_a(0.0, x, y), p.sigma_s0(0.0, x, y)
    assert set(sa) <= {0.0, 10.0} and np.all((sa == 10.0) == (ss == 0.0))


def test_batched_instances():
    ps = [inputs.batched_instance(k) for k in range(256)]
    sizes = {p.n[0] for p in ps}
    assert all(p.n[0] == p.n[1] and p.n[0] in range(64, 513, 32) for p in ps)
    assert {p.N for p in ps} == {3, 5, 7, 9, 11, 13, 15}
    assert len(sizes) >= 12
    assert all(p.bc[0] == p.bc[1] for p in ps) and {p.bc[0] for p in ps} == {"periodic", "extrapolation"}
    assert all(p.precision == "fp32" and not p.ic for p in ps)
    x = np.linspace(0.01, 0.99, 41)
    X, Y = np.meshgrid(x, x)
    for p in ps[:16]:
        sa, ss = p.sigma_a(0.0, X, Y), p.sigma_s0(0.0, X, Y)
        assert sa.min() >= 0 and sa.max() <= 5 and ss.min() >= 0 and ss.max() <= 10
    q = inputs.batched_instance(7)
    assert q.N == ps[7].N and q.n == ps[7].n and q.bc == ps[7].bc


def test_random_p39_fields():
    """log10 sigma_s0 in [-1, 1] (bilinear interpolation of lattice values
    stays inside their range); the initial pulse has unit mass."""
    p = inputs.random_p39(n=64)
    r = inputs.SplitMix64(3)
    x, y = r.uniforms(5000) * 2 - 1, r.uniforms(5000) * 2 - 1
    s = p.sigma_s0(0.0, x, y)
    assert s.min() >= 0.1 - 1e-12 and s.max() <= 10 + 1e-9
    h = 2.0 / 400
    c = -1 + (np.arange(400) + 0.5) * h
    X, Y = np.meshgrid(c, c)
    assert abs(p.ic[0][1](0.0, X, Y).sum() * h * h - 1.0) < 1e-6


def test_closure_media_ranges():
    x = np.linspace(-0.99, 0.99, 57)
    X, Y = np.meshgrid(x, x)
    for seed in (0, 100, 200):
        p = inputs.closure_medium(seed, n=64)
        sa, ss = p.sigma_a(0.0, X, Y), p.sigma_s0(0.0, X, Y)
        assert sa.min() >= 0 and sa.max() <= 0.5
        assert ss.min() >= 0.1 - 1e-12 and ss.max() <= 10 + 1e-9
        assert p.t_final == 0.5 and p.bc == ("periodic", "periodic")
    assert not np.array_equal(inputs.closure_medium(0, n=64).sigma_a(0.0, X, Y),
                              inputs.closure_medium(1, n=64).sigma_a(0.0, X, Y))
