"""GPU parity of batched stepping: a batch of uneven FP32 2D P_N instances
(grid sizes, orders, boundaries, media) advanced by one graph launch per
step call must equal every instance stepped alone with the tiled kernel bit
for bit (the same tile code runs on the same data), and a seeded subset must
match the FP64 oracle within the FP32 bar."""
import numpy as np
import pytest

from helpers import assert_parity, oracle_run, rel_l2
from paper_1211_2205_gb300 import capi, inputs

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def _instance(k, nsteps=6):
    """Small uneven instances: several tile columns and rows with ragged
    tails, orders with and without a last odd order, both boundaries."""
    rng = inputs.SplitMix64(7000 + k)
    n = [40, 67, 96, 130, 70][k % 5]
    ny = n + [0, 3, -5][k % 3]
    N = [1, 3, 5, 8, 13, 15, 2][k % 7]
    bc = ["periodic", "extrapolation"][(k // 2) % 2]
    ax = (0.0, 1.0, 0.0, ny / n)
    cx, cy = 0.3 + 0.4 * rng.uniform(), 0.3 + 0.3 * rng.uniform()
    return inputs.Problem(
        name=f"batch_test_{k}", N=N, ax=ax, n=(n, ny), bc=(bc, "periodic" if k % 3 else bc), cn=0.5,
        precision="fp32", sigma_a=inputs.piecewise_blocks(rng, 6, 0.0, 5.0, ax),
        sigma_s0=inputs.piecewise_blocks(rng, 6, 0.0, 10.0, ax),
        sources=[(0, inputs.gaussian_std(cx, cy, 0.05))],
        ic=[(0, inputs.gaussian_std(cy, cx, 0.08))], nsteps=nsteps)


def _alone(p, schedule, steps_list):
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule=schedule)
    for n in steps_list:
        s.step(n)
    return [s.moments(j) for j in range(s.ncomp)]


@pytest.mark.parametrize("schedule", ["merged", "literal"])
def test_batch_equals_instances_alone(schedule):
    probs = [_instance(k) for k in range(14)]
    b = capi.Batch.from_problems(probs, schedule=schedule)
    assert len(b) == 14
    b.step(4)
    b.step(2)
    b.sync()
    for k, p in enumerate(probs):
        got = [b.instances[k].moments(j) for j in range(b.instances[k].ncomp)]
        ref = _alone(p, schedule, [4, 2])
        for j, (g, r) in enumerate(zip(got, ref)):
            assert np.array_equal(g, r), (k, j)
        assert b.instances[k].steps_done == 6
    b.close()


def test_batch_subset_matches_oracle():
    probs = [_instance(k) for k in range(7)]
    b = capi.Batch.from_problems(probs)
    b.step(6)
    b.sync()
    for k in (0, 2, 3, 5):
        inst = b.instances[k]
        got = [inst.moments(j) for j in range(inst.ncomp)]
        _, ref = oracle_run(probs[k], inst, nsteps=6)
        assert_parity(got, ref, FP32_TOL, "fp32", k)
    b.close()


def test_batch_picks_up_changed_instance_data():
    """Sources and material changed on an instance after the first step
    reach the batched kernel (its parameters are re-uploaded)."""
    probs = [_instance(k) for k in range(4)]
    b = capi.Batch.from_problems(probs)
    b.step(2)
    alone = capi.Stepper.from_problem(probs[1], kernel="tiled", schedule="merged")
    alone.step(2)
    for s in (b.instances[1], alone):
        X, Y = s.grid_coords(1)
        s.set_source(1, 0.5 * np.sin(3 * X) * np.cos(2 * Y))
        nx, ny, *_ = s.grid_info(0)
        s.set_material(0, np.full((ny, nx), 0.7), np.full((ny, nx), 2.0))
    b.step(3)
    alone.step(3)
    b.sync()
    for j in range(alone.ncomp):
        assert np.array_equal(b.instances[1].moments(j), alone.moments(j)), j
    b.close()


def test_full_size_batch_samples():
    """The 256-instance workload (grids 64^2..512^2, N in {3..15}): eight
    seeded instances equal their standalone runs bit for bit, and the
    smallest sampled one matches the oracle."""
    probs = [inputs.batched_instance(k, nsteps=3) for k in range(256)]
    b = capi.Batch.from_problems(probs)
    b.step(3)
    b.sync()
    rng = np.random.default_rng(256)
    picks = sorted(rng.choice(256, size=8, replace=False))
    for k in picks:
        inst = b.instances[k]
        ref = _alone(probs[k], "merged", [3])
        for j in range(0, inst.ncomp, max(1, inst.ncomp // 6)):
            assert np.array_equal(inst.moments(j), ref[j]), (k, j)
    small = min(picks, key=lambda k: probs[k].n[0] * (probs[k].N + 1) ** 2)
    inst = b.instances[small]
    got = [inst.moments(j) for j in range(inst.ncomp)]
    _, ref = oracle_run(probs[small], inst, nsteps=3)
    assert_parity(got, ref, FP32_TOL, "fp32")
    b.close()


def test_batch_rejects_unsupported_instances():
    ok = dict(N=3, ax=(0, 1, 0, 1), n=(32, 32))
    with pytest.raises(capi.StarmapError) as e:
        capi.Batch([ok, dict(ok, precision="fp64")])
    assert e.value.code == capi.E_UNSUPPORTED
    with pytest.raises(capi.StarmapError) as e:
        capi.Batch([dict(ok, N=7, closure="mlp8")])
    assert e.value.code == capi.E_UNSUPPORTED
    with pytest.raises(capi.StarmapError) as e:
        capi.Batch([dict(ok, system="slab", n=(32, 1))])
    assert e.value.code == capi.E_UNSUPPORTED


def test_autotuner_times_both_tile_heights_and_leaves_state_zero(monkeypatch):
    monkeypatch.setenv("STARMAP_TUNE_CACHE", "off")
    probs = [_instance(k) for k in range(6)]
    b = capi.Batch.from_problems(probs)                  # kernel "auto": tuned
    rows, tall, short = b.tile_rows()
    assert rows in (5, 10) and tall > 0 and short > 0
    assert (rows == 5) == (short < tall)
    r, strip, cached = b.tuning()
    assert r == rows and strip in (96, 192, 384) and not cached
    for inst in b.instances:
        assert inst.steps_done == 0 and inst.time == 0.0
    # the tuning steps left the state as loaded (zero before the problem data)
    alone = capi.Stepper.from_problem(probs[2], kernel="tiled", schedule="merged")
    b.step(3)
    alone.step(3)
    b.sync()
    for j in range(alone.ncomp):
        assert np.array_equal(b.instances[2].moments(j), alone.moments(j)), j
    forced = capi.Batch.from_problems(probs[:2], kernel="tiled_tall")
    assert forced.tile_rows() == (10, -1.0, -1.0)


def test_batch_mixing_long_and_short_tiles():
    """Instances whose tiles are long (N = 21, 27: single tiles dealt in
    strided runs) next to short ones (strips of tiles): each equals its
    standalone tiled run bit for bit, with both tile heights."""
    probs = [_instance(k, nsteps=4) for k in range(5)]
    for k, N in ((0, 21), (3, 27)):
        probs[k] = inputs.Problem(**{**probs[k].__dict__, "N": N})
    for kernel in ("tiled_tall", "tiled_short"):
        b = capi.Batch.from_problems(probs, schedule="merged", kernel=kernel)
        b.step(3)
        b.step(1)
        b.sync()
        for k, p in enumerate(probs):
            alone = capi.Stepper.from_problem(p, kernel=kernel, schedule="merged")
            alone.step(3)
            alone.step(1)
            inst = b.instances[k]
            for j in range(0, inst.ncomp, max(1, inst.ncomp // 8)):
                assert np.array_equal(inst.moments(j), alone.moments(j)), (kernel, k, j)
        b.close()


def test_autotuner_cache(tmp_path, monkeypatch):
    """The tuned choice is written to the cache file; a batch of the same
    shapes takes it from there (no timing) and steps the same way."""
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("STARMAP_TUNE_CACHE", str(path))
    probs = [_instance(k, nsteps=3) for k in range(3)]
    a = capi.Batch.from_problems(probs)
    rows, strip, cached = a.tuning()
    assert not cached and path.exists() and len(path.read_text().splitlines()) == 1
    b = capi.Batch.from_problems(probs)
    assert b.tuning() == (rows, strip, True)
    assert b.tile_rows() == (rows, -1.0, -1.0)
    for batch in (a, b):
        batch.step(3)
        batch.sync()
    for k in range(3):
        for j in range(a.instances[k].ncomp):
            assert np.array_equal(a.instances[k].moments(j), b.instances[k].moments(j)), (k, j)
    other = capi.Batch.from_problems(probs[:2])          # another signature: tuned again
    assert not other.tuning()[2]
    assert len(path.read_text().splitlines()) == 2
