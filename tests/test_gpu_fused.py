"""The temporally fused step (schedule "fused": each inner E_dt O_dt pair of
the merged schedule in one launch, even then odd update per tile).  Every
point sees the same arithmetic in the same order as the two-pass merged
schedule, so the results must be equal bit for bit; and against the FP64
oracle within the FP32 bar.  Every boundary combination, ragged grids, N
from 1 to 39, anisotropic scattering, sources, step counts with and
without an unfused inner step, and the benchmark configuration on a
window."""
import numpy as np
import pytest

from helpers import assert_parity, oracle_run
from paper_1211_2205_gb300 import capi, inputs
from test_gpu_parity import _random_problem

pytestmark = pytest.mark.gpu

BCS = [("periodic", "periodic"), ("extrapolation", "extrapolation"),
       ("periodic", "extrapolation"), ("extrapolation", "periodic")]


def _both(p, steps_calls, **kw):
    out = []
    for sched in ("merged", "fused"):
        s = capi.Stepper.from_problem(p, kernel="tiled", schedule=sched, **kw)
        for n in steps_calls:
            s.step(n)
        out.append([s.moments(j) for j in range(s.ncomp)])
        s.close()
    return out


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("N", [1, 2, 4, 7, 13])
def test_fused_equals_merged_bitwise(N, bc):
    """130 x 47: three 62-wide tiles (the last ragged) and ten 5-row tiles
    (the last ragged); 3 + 4 + 1 steps: fused pairs, an unfused inner step,
    a call without inner steps."""
    p = _random_problem(N, (130, 47), bc, "fp32", 700 + N, 8)
    merged, fused = _both(p, [3, 4, 1])
    for j, (a, b) in enumerate(zip(merged, fused)):
        assert np.array_equal(a, b), (j, float(np.max(np.abs(a - b))))


@pytest.mark.parametrize("n", [(1, 1), (2, 3), (3, 2), (7, 5), (62, 5), (63, 6), (64, 11)])
@pytest.mark.parametrize("bc", BCS)
def test_fused_small_and_edge_sized_grids(n, bc):
    """Grids of one tile, mostly outside the grid, and sizes at the tile
    edges (62 / 63 / 64 columns, 5 / 6 / 11 rows)."""
    p = _random_problem(3, n, bc, "fp32", 900 + 7 * n[0] + n[1], 5)
    merged, fused = _both(p, [5])
    for j, (a, b) in enumerate(zip(merged, fused)):
        assert np.array_equal(a, b), j


def test_fused_matches_oracle_with_sources_and_anisotropy():
    p = _random_problem(6, (75, 52), ("extrapolation", "periodic"), "fp32", 17, 9, aniso=True)
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule="fused")
    s.step(p.nsteps)
    got = [s.moments(j) for j in range(s.ncomp)]
    _, ref = oracle_run(p, s)
    assert_parity(got, ref, 1e-5, "fp32")


def test_fused_high_order():
    """P_39 (820 moments; the shared memory holds both machines' tables)."""
    p = _random_problem(39, (70, 24), ("periodic", "periodic"), "fp32", 39, 5)
    merged, fused = _both(p, [5])
    for j, (a, b) in enumerate(zip(merged, fused)):
        assert np.array_equal(a, b), j
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule="fused")
    s.step(5)
    _, ref = oracle_run(p, s)
    assert_parity([s.moments(j) for j in range(s.ncomp)], ref, 1e-5, "fp32")


def test_fused_bench_configuration_window():
    """P_39 FP32 1024^2 periodic (the benchmark workload), 6 steps: a
    window of every component equal to the merged schedule's bit for bit."""
    p = inputs.random_p39(nsteps=6)
    wins = []
    for sched in ("merged", "fused"):
        s = capi.Stepper.from_problem(p, kernel="tiled", schedule=sched)
        s.step(6)
        wins.append([s.moments_window(j, 600, 300, 70, 16) for j in range(s.ncomp)] +
                    [s.moments_window(j, 0, 1000, 40, 11) for j in range(0, s.ncomp, 7)])
        s.close()
    for j, (a, b) in enumerate(zip(*wins)):
        assert np.array_equal(a, b), j


def test_fused_material_change_and_advance_to():
    """Tables rebuilt after a material change reach the fused launch;
    interpolated output works on the fused schedule."""
    p = _random_problem(5, (90, 40), ("periodic", "extrapolation"), "fp32", 55, 6)
    runs = []
    for sched in ("merged", "fused"):
        s = capi.Stepper.from_problem(p, kernel="tiled", schedule=sched)
        s.step(3)
        nx, ny, *_ = s.grid_info(3)
        s.set_material(3, np.full((ny, nx), 0.4), np.full((ny, nx), 2.5))
        X, Y = s.grid_coords(1)
        s.set_source(1, 0.3 * np.cos(4 * X) * np.sin(3 * Y))
        s.advance_to(s.time + 5.5 * s.dt)
        runs.append([s.output(j) for j in range(s.ncomp)])
        s.close()
    for j, (a, b) in enumerate(zip(*runs)):
        assert np.array_equal(a, b), j


def test_fused_unsupported_configurations():
    p = _random_problem(7, (40, 40), ("periodic", "periodic"), "fp32", 5, 2)
    with pytest.raises(capi.StarmapError) as e:
        capi.Stepper.from_problem(p, kernel="tiled", schedule="fused", closure="mlp8")
    assert e.value.code == capi.E_UNSUPPORTED
    q = _random_problem(3, (40, 40), ("periodic", "periodic"), "fp64", 5, 2)
    with pytest.raises(capi.StarmapError) as e:
        capi.Stepper.from_problem(q, schedule="fused")
    assert e.value.code == capi.E_UNSUPPORTED
