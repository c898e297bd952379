"""The allocation-free diagnostics entry point against starmap_diagnostics.

starmap_diagnostics_noalloc is for callers that cannot allocate device
memory where they need the FP64 reductions; its partial sums sit in a
library-wide device array instead of cudaMalloc'ed scratch.  This test calls
it through the C ABI on every grid of a stepper's state, combines the grids
on the host, and checks the result against starmap_diagnostics, twice in a
row with the state changing in between (the shared array keeps the previous
call's contents)."""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _grid_layout(s, capi):
    """Per grid: (pointer of its first component, pitch, origin, component
    stride, nx, ny, number of components), from the C ABI's queries."""
    by_grid = {}
    for j in range(s.ncomp):
        info = s.moment_info(j)
        ptr, pitch, origin = s.device_ptr(j)
        by_grid.setdefault(info["grid"], []).append((ptr, pitch, origin, info["nx"], info["ny"]))
    out = {}
    esize = 4 if s.precision == "fp32" else 8
    for g, comps in by_grid.items():
        comps.sort()
        ptr, pitch, origin, nx, ny = comps[0]
        stride = (comps[1][0] - ptr) // esize if len(comps) > 1 else pitch * (ny + 2)
        out[g] = (ptr, pitch, origin, stride, nx, ny, len(comps))
    return out


def _noalloc_diagnostics(s, capi, out_dev, torch):
    L = capi.lib()
    cell = s.grid_info(0)[4] * s.grid_info(0)[5]
    prec = capi.FP32 if s.precision == "fp32" else capi.FP64
    mass, sq, bad = None, 0.0, 0.0
    s.sync()
    for g, (ptr, pitch, origin, stride, nx, ny, K) in sorted(_grid_layout(s, capi).items()):
        rc = L.starmap_diagnostics_noalloc(ctypes.c_void_p(ptr), prec, K, nx, ny, pitch, stride, origin, cell,
                                           ctypes.c_void_p(out_dev.data_ptr()), None)
        assert rc == capi.OK
        torch.cuda.synchronize()
        m, l2, nb = out_dev.cpu().tolist()
        if g == 0:
            mass = m
        sq += l2 * l2
        bad += nb
    return mass, math.sqrt(sq), bad


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_diagnostics_twice(precision):
    torch = pytest.importorskip("torch")
    from paper_1211_2205_gb300 import capi, inputs
    p = inputs.gaussian_p5(n=48, nsteps=0, precision=precision)
    p.sigma_a = lambda t, x, y: 0.3 + 0 * x
    s = capi.Stepper.from_problem(p, schedule="merged")
    out_dev = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    tol = 1e-12 if precision == "fp64" else 1e-6
    for call in range(2):
        s.step(3)
        ref_mass, ref_l2, ref_bad = s.diagnostics()
        mass, l2, bad = _noalloc_diagnostics(s, capi, out_dev, torch)
        assert bad == ref_bad == 0
        assert abs(mass - ref_mass) <= tol * abs(ref_mass)
        assert abs(l2 - ref_l2) <= tol * ref_l2


def test_noalloc_rejects_oversized_and_bad_layout():
    torch = pytest.importorskip("torch")
    from paper_1211_2205_gb300 import capi
    L = capi.lib()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(buf.data_ptr())
    optr = ctypes.c_void_p(out.data_ptr())
    rows_max = 1 << 26
    # more rows than the stated maximum
    assert L.starmap_diagnostics_noalloc(ptr, capi.FP64, 2, 4, rows_max, 4, 4 * rows_max, 0, 1.0, optr, None) == capi.E_ARG
    # pitch shorter than a row
    assert L.starmap_diagnostics_noalloc(ptr, capi.FP64, 1, 4, 2, 3, 8, 0, 1.0, optr, None) == capi.E_ARG
    # a row longer than the stated maximum, and a pitch beyond its maximum
    long_row = (1 << 24) + 1
    assert L.starmap_diagnostics_noalloc(ptr, capi.FP64, 1, long_row, 1, long_row, long_row, 0, 1.0,
                                         optr, None) == capi.E_ARG
    assert L.starmap_diagnostics_noalloc(ptr, capi.FP64, 1, 4, 2, (1 << 31) + 1, 1 << 40, 0, 1.0,
                                         optr, None) == capi.E_ARG
    assert L.starmap_diagnostics_noalloc(None, capi.FP64, 1, 4, 2, 4, 8, 0, 1.0, optr, None) == capi.E_ARG
    # a valid call on a small dense array
    buf.copy_(torch.arange(16, dtype=torch.float64))
    assert L.starmap_diagnostics_noalloc(ptr, capi.FP64, 2, 4, 2, 4, 8, 0, 0.5, optr, None) == capi.OK
    torch.cuda.synchronize()
    m, l2, bad = out.cpu().tolist()
    v = np.arange(16.0)
    assert abs(m - 0.5 * v[:8].sum()) < 1e-12
    assert abs(l2 - math.sqrt(0.5 * (v * v).sum())) < 1e-12
    assert bad == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_many_rows_with_nonfinite_values(precision):
    """More rows than partial-sum blocks (each block then reduces several
    rows), a padded layout with the first point away from the buffer's
    start, and planted NaN and Inf values: against sums taken on the host,
    on two calls in a row with different data."""
    torch = pytest.importorskip("torch")
    from paper_1211_2205_gb300 import capi
    L = capi.lib()
    ncomp, nx, ny, pitch = 3, 37, 500, 40
    stride, origin = pitch * (ny + 3), 2 * pitch + 1
    assert ncomp * ny > 1024
    dtype = torch.float64 if precision == "fp64" else torch.float32
    npdt = np.float64 if precision == "fp64" else np.float32
    prec = capi.FP64 if precision == "fp64" else capi.FP32
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    cell = 0.25
    rng = np.random.default_rng(1024)
    for call in range(2):
        host = np.full(origin + ncomp * stride, 1e30, dtype=npdt)     # padding: never read
        vals = rng.normal(size=(ncomp, ny, nx)).astype(npdt)
        planted = [(0, 7, 3, np.nan), (2, 411, 36, np.inf), (1, 250 + call, 0, -np.inf)]
        for k, y, x, v in planted:
            vals[k, y, x] = v
        for k in range(ncomp):
            for y in range(ny):
                host[origin + k * stride + y * pitch: origin + k * stride + y * pitch + nx] = vals[k, y]
        dev = torch.from_numpy(host).to(device="cuda", dtype=dtype)
        torch.cuda.synchronize()
        rc = L.starmap_diagnostics_noalloc(ctypes.c_void_p(dev.data_ptr()), prec, ncomp, nx, ny, pitch, stride,
                                           origin, cell, ctypes.c_void_p(out.data_ptr()), None)
        assert rc == capi.OK
        torch.cuda.synchronize()
        m, l2, bad = out.cpu().tolist()
        v = vals.astype(np.float64)
        fin = np.isfinite(v)
        assert bad == len(planted)
        want_m = cell * float(np.sum(np.where(fin[0], v[0], 0.0)))
        want_l2 = math.sqrt(cell * float(np.sum(np.where(fin, v * v, 0.0))))
        assert abs(m - want_m) <= 1e-12 * want_l2
        assert abs(l2 - want_l2) <= 1e-12 * want_l2
