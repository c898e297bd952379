"""Thin ctypes binding of the StaRMAP C ABI (include/starmap.h).

Argument marshalling only: every step of the method runs in libstarmap.so.
If the library has not been built, loading raises RuntimeError: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libstarmap.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "starmap.h")

OK = 0
E_ARG, E_CFL, E_NOMEM, E_CUDA, E_NONFINITE, E_TIMEOUT, E_STATE, E_UNSUPPORTED = -1, -2, -3, -4, -5, -6, -7, -8
E_GROWTH = -9
PERIODIC, EXTRAPOLATION = 0, 1
PN2D, SLAB = 0, 1
FP64, FP32 = 0, 1
SCHEDULE_LITERAL, SCHEDULE_MERGED, SCHEDULE_FUSED = 0, 1, 2
KERNEL_AUTO, KERNEL_GATHER, KERNEL_TILED, KERNEL_TILED_TALL, KERNEL_TILED_SHORT = 0, 1, 2, 3, 4
CLOSURE_NONE, CLOSURE_MLP8 = 0, 1
ENGINE_MMA_SYNC, ENGINE_TCGEN05 = 0, 1
MLP_INPUTS, MLP_HIDDEN, MLP_OUTPUTS, MLP_PARAMS = 38, 128, 9, 22665
FIELD_SIGMA_A, FIELD_SIGMA_S0, FIELD_SOURCE = 0, 1, 2


class StarmapError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"starmap error {code}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("system", ctypes.c_int),
        ("N", ctypes.c_int),
        ("ax", ctypes.c_double * 4),
        ("n", ctypes.c_int * 2),
        ("bc", ctypes.c_int * 2),
        ("cn", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("schedule", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p),
        ("closure", ctypes.c_int),
    ]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_fp = ctypes.POINTER(ctypes.c_float)
# int fn(void* user, int field, double t, int g, const double* x, const double* y, size_t count, double* out)
FieldFn = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_size_t,
                           ctypes.POINTER(ctypes.c_double))


def exported_functions() -> list:
    """Names of all functions declared in include/starmap.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(starmap_[a-z0-9_]+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def lib():
    """Load libstarmap.so (fails loudly if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libstarmap.so is not built (run __graft_entry__.build()); "
                           "there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    sig = {
        "starmap_config_default": (None, [ctypes.POINTER(Config)]),
        "starmap_host_matrices": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _ip, _ip, _dp]),
        "starmap_host_expm1div": (ctypes.c_int, [_dp, ctypes.c_size_t]),
        "starmap_batch_plan": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                              ctypes.c_size_t, ctypes.c_void_p]),
        "starmap_tiled_schedule": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                                  ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t,
                                                  ctypes.c_void_p]),
        "starmap_direction_moments": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                     _dp, ctypes.c_size_t]),
        "starmap_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(H)]),
        "starmap_destroy": (None, [H]),
        "starmap_last_error": (ctypes.c_char_p, [H]),
        "starmap_num_moments": (ctypes.c_int, [H]),
        "starmap_dt": (ctypes.c_double, [H]),
        "starmap_time": (ctypes.c_double, [H]),
        "starmap_steps_done": (ctypes.c_long, [H]),
        "starmap_kernel": (ctypes.c_int, [H]),
        "starmap_moment_info": (ctypes.c_int, [H, ctypes.c_int, _ip, _ip, _ip, _ip, _ip, _ip]),
        "starmap_grid_info": (ctypes.c_int, [H, ctypes.c_int, _ip, _ip, _dp, _dp, _dp, _dp]),
        "starmap_set_material": (ctypes.c_int, [H, ctypes.c_int, _dp, _dp, ctypes.c_size_t]),
        "starmap_set_scattering_factors": (ctypes.c_int, [H, _dp, ctypes.c_int]),
        "starmap_set_source": (ctypes.c_int, [H, ctypes.c_int, _dp, ctypes.c_size_t]),
        "starmap_set_moment": (ctypes.c_int, [H, ctypes.c_int, _dp, ctypes.c_size_t]),
        "starmap_set_time": (ctypes.c_int, [H, ctypes.c_double]),
        "starmap_clear": (ctypes.c_int, [H]),
        "starmap_step": (ctypes.c_int, [H, ctypes.c_long]),
        "starmap_set_health_check": (ctypes.c_int, [H, ctypes.c_long, ctypes.c_double]),
        "starmap_set_time_dependence": (ctypes.c_int, [H, FieldFn, ctypes.c_void_p, _ip, ctypes.c_int]),
        "starmap_health": (ctypes.c_int, [H, ctypes.POINTER(ctypes.c_long), _dp, _dp]),
        "starmap_health_verdict": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_long]),
        "starmap_advance_to": (ctypes.c_int, [H, ctypes.c_double]),
        "starmap_pass": (ctypes.c_int, [H, ctypes.c_int, ctypes.c_int]),
        "starmap_output": (ctypes.c_int, [H, ctypes.c_int, _dp, ctypes.c_size_t]),
        "starmap_moments": (ctypes.c_int, [H, ctypes.c_int, _dp, ctypes.c_size_t]),
        "starmap_moments_window": (ctypes.c_int, [H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, _dp, ctypes.c_size_t]),
        "starmap_diagnostics": (ctypes.c_int, [H, _dp, _dp, ctypes.POINTER(ctypes.c_long)]),
        "starmap_device_ptr": (ctypes.c_int, [H, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                              ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long)]),
        "starmap_state_bytes": (ctypes.c_size_t, [H]),
        "starmap_get_state": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_size_t]),
        "starmap_set_state": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_size_t]),
        "starmap_sync": (ctypes.c_int, [H]),
        "starmap_pack_rows": (ctypes.c_int, [H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                             ctypes.c_size_t]),
        "starmap_unpack_rows": (ctypes.c_int, [H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_size_t]),
        "starmap_selftest_bounded_wait": (ctypes.c_int, []),
        "starmap_diagnostics_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                       ctypes.c_int, ctypes.c_long, ctypes.c_long, ctypes.c_long,
                                                       ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
        "starmap_set_closure": (ctypes.c_int, [H, _fp, ctypes.c_size_t]),
        "starmap_closure_samples": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_size_t]),
        "starmap_mlp_create": (ctypes.c_int, [_fp, ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(H)]),
        "starmap_mlp_destroy": (None, [H]),
        "starmap_mlp_last_error": (ctypes.c_char_p, [H]),
        "starmap_mlp_get_params": (ctypes.c_int, [H, _fp, ctypes.c_size_t]),
        "starmap_mlp_set_params": (ctypes.c_int, [H, _fp, ctypes.c_size_t]),
        "starmap_mlp_forward": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
        "starmap_mlp_loss_grad": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]),
        "starmap_mlp_train_step": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_size_t, ctypes.c_float, ctypes.c_void_p]),
        "starmap_mlp_perturb_inputs": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                                      ctypes.c_int, ctypes.c_float, ctypes.c_ulonglong]),
        "starmap_debug_fail_allocation": (ctypes.c_int, [ctypes.c_int]),
        "starmap_mlp_shuffle": (ctypes.c_int, [H, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_ulonglong,
                                               ctypes.c_void_p]),
        "starmap_mlp_steps": (ctypes.c_long, [H]),
        "starmap_mlp_set_engine": (ctypes.c_int, [H, ctypes.c_int]),
        "starmap_set_closure_engine": (ctypes.c_int, [H, ctypes.c_int]),
        "starmap_batch_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(H)]),
        "starmap_batch_destroy": (None, [H]),
        "starmap_batch_last_error": (ctypes.c_char_p, [H]),
        "starmap_batch_count": (ctypes.c_int, [H]),
        "starmap_batch_instance": (H, [H, ctypes.c_int]),
        "starmap_batch_launches": (ctypes.c_long, [H, ctypes.c_long]),
        "starmap_batch_step": (ctypes.c_int, [H, ctypes.c_long]),
        "starmap_batch_tile_rows": (ctypes.c_int, [H, _dp, _dp]),
        "starmap_batch_tuning": (ctypes.c_int, [H, _ip, _ip, _ip]),
        "starmap_batch_sync": (ctypes.c_int, [H]),
        "starmap_mlp_sync": (ctypes.c_int, [H]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _addr(x) -> Optional[int]:
    """Device address of a tensor-like (``data_ptr()``) or an int; None stays NULL."""
    if x is None:
        return None
    return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)


def _params32(params) -> np.ndarray:
    a = np.ascontiguousarray(params, dtype=np.float32).ravel()
    if a.size != MLP_PARAMS:
        raise ValueError(f"closure network needs {MLP_PARAMS} parameters, got {a.size}")
    return a


def host_matrices(system: int, N: int):
    """Mx, My, grid per component, order per component, lambda_max (host math)."""
    L = lib()
    n = (N + 1) * (N + 2) // 2 if system == PN2D else N + 1
    Mx = np.zeros((n, n))
    My = np.zeros((n, n))
    grid = np.zeros(n, dtype=np.int32)
    order = np.zeros(n, dtype=np.int32)
    lam = ctypes.c_double()
    rc = L.starmap_host_matrices(system, N, n, _dptr(Mx), _dptr(My), grid.ctypes.data_as(_ip),
                                 order.ctypes.data_as(_ip), ctypes.byref(lam))
    if rc != OK:
        raise StarmapError(rc, L.starmap_last_error(None).decode())
    return Mx, My, grid, order, lam.value


def direction_moments(N: int, mu: float, phi: float) -> np.ndarray:
    """Moments of a unit beam in the direction (mu, phi): the real harmonic
    of every component of the 2D system (host math)."""
    L = lib()
    n = (N + 1) * (N + 2) // 2
    out = np.zeros(n)
    rc = L.starmap_direction_moments(PN2D, int(N), float(mu), float(phi), _dptr(out), n)
    if rc != OK:
        raise StarmapError(rc, L.starmap_last_error(None).decode())
    return out


def tiled_schedule(N: int, parity: int, frozen_top: bool = False, dx: float = 1.0, dy: float = 1.0):
    """The tiled kernel's schedule of one pass (host only): stages (S, 4)
    global components (input R, input I, output R, output I; -1 absent),
    coefficient rows (R, 16) and the finalised component per event."""
    L = lib()
    counts = np.zeros(3, dtype=np.int64)
    rc = L.starmap_tiled_schedule(int(N), int(parity), int(bool(frozen_top)), float(dx), float(dy),
                                  None, 0, None, 0, None, 0, counts.ctypes.data)
    if rc != OK:
        raise StarmapError(rc, L.starmap_last_error(None).decode())
    st = np.zeros((int(counts[0]), 4), dtype=np.int32)
    co = np.zeros((int(counts[1]), 16), dtype=np.float32)
    fi = np.zeros(int(counts[2]), dtype=np.int32)
    rc = L.starmap_tiled_schedule(int(N), int(parity), int(bool(frozen_top)), float(dx), float(dy),
                                  st.ctypes.data, st.shape[0], co.ctypes.data, co.shape[0], fi.ctypes.data,
                                  fi.size, counts.ctypes.data)
    if rc != OK:
        raise StarmapError(rc, L.starmap_last_error(None).decode())
    return st, co, fi


def batch_plan(tiles_x, tiles_y, cost, slots: int):
    """The batch's work-unit plan (host only): (items (I, 4): instance,
    first tile, tile count, tile stride; off (grid + 1,))."""
    L = lib()
    tx = np.ascontiguousarray(tiles_x, dtype=np.int32)
    ty = np.ascontiguousarray(tiles_y, dtype=np.int32)
    c = np.ascontiguousarray(cost, dtype=np.int32)
    counts = np.zeros(2, dtype=np.int64)
    rc = L.starmap_batch_plan(tx.ctypes.data, ty.ctypes.data, c.ctypes.data, int(tx.size), int(slots),
                              None, 0, None, 0, counts.ctypes.data)
    if rc != OK:
        raise StarmapError(rc, L.starmap_last_error(None).decode())
    items = np.zeros((int(counts[1]), 4), dtype=np.int32)
    off = np.zeros(int(counts[0]) + 1, dtype=np.int32)
    rc = L.starmap_batch_plan(tx.ctypes.data, ty.ctypes.data, c.ctypes.data, int(tx.size), int(slots),
                              items.ctypes.data, items.shape[0], off.ctypes.data, off.size, counts.ctypes.data)
    if rc != OK:
        raise StarmapError(rc, L.starmap_last_error(None).decode())
    return items, off


def debug_fail_allocation(n: int) -> int:
    """Make the n-th following device allocation of the library fail (0: off)."""
    return lib().starmap_debug_fail_allocation(int(n))


def selftest_bounded_wait() -> int:
    """Status of the bounded-wait self-test (E_TIMEOUT is the expected outcome)."""
    return lib().starmap_selftest_bounded_wait()


def health_verdict(l2_start: float, l2_end: float, t_span: float, q_l2: float, growth: float,
                   nonfinite: int = 0) -> int:
    """The library's health-check decision (OK, E_NONFINITE or E_GROWTH)."""
    return lib().starmap_health_verdict(float(l2_start), float(l2_end), float(t_span), float(q_l2),
                                        float(growth), int(nonfinite))


def host_expm1div(c) -> np.ndarray:
    L = lib()
    a = np.ascontiguousarray(np.array(c, dtype=np.float64).ravel())
    rc = L.starmap_host_expm1div(_dptr(a), a.size)
    if rc != OK:
        raise StarmapError(rc, "expm1div")
    return a


def make_config(N: int, ax, n, bc=("periodic", "periodic"), cn: float = 0.5, precision: str = "fp64",
                system: str = "pn2d", schedule: str = "literal", kernel: str = "auto", dt: float = 0.0,
                stream: Optional[int] = None, closure: str = "none") -> Config:
    """A starmap_config from keyword values (library defaults elsewhere)."""
    c = Config()
    lib().starmap_config_default(ctypes.byref(c))
    c.system = {"pn2d": PN2D, "slab": SLAB}[system]
    c.N = int(N)
    for i in range(4):
        c.ax[i] = float(ax[i])
    c.n[0], c.n[1] = int(n[0]), int(n[1])
    bmap = {"periodic": PERIODIC, "extrapolation": EXTRAPOLATION}
    c.bc[0], c.bc[1] = bmap[bc[0]], bmap[bc[1]]
    c.cn = float(cn)
    c.dt = float(dt)
    c.precision = {"fp64": FP64, "fp32": FP32}[precision]
    c.schedule = {"literal": SCHEDULE_LITERAL, "merged": SCHEDULE_MERGED, "fused": SCHEDULE_FUSED}[schedule]
    c.kernel = {"auto": KERNEL_AUTO, "gather": KERNEL_GATHER, "tiled": KERNEL_TILED, "tiled_tall": KERNEL_TILED_TALL,
                "tiled_short": KERNEL_TILED_SHORT}[kernel]
    c.cuda_stream = stream
    c.closure = {"none": CLOSURE_NONE, "mlp8": CLOSURE_MLP8}[closure]
    return c


class Stepper:
    """One StaRMAP stepper (a handle of the C ABI)."""

    def __init__(self, N: int, ax, n, bc=("periodic", "periodic"), cn: float = 0.5,
                 precision: str = "fp64", system: str = "pn2d", schedule: str = "literal",
                 kernel: str = "auto", dt: float = 0.0, stream: Optional[int] = None, closure: str = "none"):
        self._L = lib()
        c = make_config(N, ax, n, bc, cn, precision, system, schedule, kernel, dt, stream, closure)
        h = ctypes.c_void_p()
        rc = self._L.starmap_create(ctypes.byref(c), ctypes.byref(h))
        if rc != OK:
            raise StarmapError(rc, self._L.starmap_last_error(None).decode())
        self._h = h
        self._owned = True
        self.precision = precision
        self.config = c

    @classmethod
    def _borrow(cls, handle, precision: str) -> "Stepper":
        """View of a handle owned elsewhere (a batch instance)."""
        s = cls.__new__(cls)
        s._L = lib()
        s._h = ctypes.c_void_p(handle)
        s._owned = False
        s.precision = precision
        s.config = None
        return s

    # -- lifetime -------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                self._L.starmap_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != OK:
            raise StarmapError(rc, self._L.starmap_last_error(self._h).decode())

    # -- queries --------------------------------------------------------
    @property
    def ncomp(self) -> int:
        return self._L.starmap_num_moments(self._h)

    @property
    def dt(self) -> float:
        return self._L.starmap_dt(self._h)

    @property
    def time(self) -> float:
        return self._L.starmap_time(self._h)

    @property
    def steps_done(self) -> int:
        return self._L.starmap_steps_done(self._h)

    @property
    def kernel(self) -> str:
        """"gather" or "tiled" (either tile height)."""
        return "gather" if self._L.starmap_kernel(self._h) == KERNEL_GATHER else "tiled"

    @property
    def tile_rows(self) -> int:
        """Rows of the tiled kernel's tiles (10 or 5; 0 for the gather kernel)."""
        return {KERNEL_GATHER: 0, KERNEL_TILED_TALL: 10, KERNEL_TILED_SHORT: 5}[self._L.starmap_kernel(self._h)]

    def moment_info(self, j: int):
        v = [ctypes.c_int() for _ in range(6)]
        self._check(self._L.starmap_moment_info(self._h, j, *[ctypes.byref(x) for x in v]))
        l, m, im, g, nx, ny = [x.value for x in v]
        return dict(l=l, m=m, imag=bool(im), grid=g, nx=nx, ny=ny)

    def grid_info(self, g: int):
        nx, ny = ctypes.c_int(), ctypes.c_int()
        x0, y0, dx, dy = [ctypes.c_double() for _ in range(4)]
        self._check(self._L.starmap_grid_info(self._h, g, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(x0),
                                              ctypes.byref(y0), ctypes.byref(dx), ctypes.byref(dy)))
        return nx.value, ny.value, x0.value, y0.value, dx.value, dy.value

    def grid_coords(self, g: int) -> Tuple[np.ndarray, np.ndarray]:
        """(X, Y) arrays of shape (ny, nx) of the points of grid g."""
        nx, ny, x0, y0, dx, dy = self.grid_info(g)
        X = x0 + dx * np.arange(nx)
        Y = y0 + dy * np.arange(ny)
        return np.meshgrid(X, Y, indexing="xy")

    # -- problem data ---------------------------------------------------
    def set_material(self, g: int, sigma_a: np.ndarray, sigma_s0: np.ndarray):
        a = np.ascontiguousarray(sigma_a, dtype=np.float64).ravel()
        s = np.ascontiguousarray(sigma_s0, dtype=np.float64).ravel()
        self._check(self._L.starmap_set_material(self._h, g, _dptr(a), _dptr(s), a.size))

    def set_scattering_factors(self, factor):
        if factor is None:
            self._check(self._L.starmap_set_scattering_factors(self._h, None, 0))
        else:
            f = np.ascontiguousarray(factor, dtype=np.float64)
            self._check(self._L.starmap_set_scattering_factors(self._h, _dptr(f), f.size))

    def set_source(self, j: int, q: Optional[np.ndarray]):
        if q is None:
            self._check(self._L.starmap_set_source(self._h, j, None, 0))
        else:
            a = np.ascontiguousarray(q, dtype=np.float64).ravel()
            self._check(self._L.starmap_set_source(self._h, j, _dptr(a), a.size))

    def set_moment(self, j: int, u: np.ndarray):
        a = np.ascontiguousarray(u, dtype=np.float64).ravel()
        self._check(self._L.starmap_set_moment(self._h, j, _dptr(a), a.size))

    def clear(self):
        self._check(self._L.starmap_clear(self._h))

    def set_time(self, t: float):
        self._check(self._L.starmap_set_time(self._h, float(t)))

    # -- stepping -------------------------------------------------------
    def step(self, n: int = 1):
        self._check(self._L.starmap_step(self._h, int(n)))

    def set_health_check(self, every: int, growth: float = 1.05):
        """FP64 check after every `every` steps (0 = off); a failing span
        raises StarmapError (E_NONFINITE / E_GROWTH) with the state reset to
        the last span that passed."""
        self._check(self._L.starmap_set_health_check(self._h, int(every), float(growth)))

    def health(self):
        """(steps at the last span that passed, its L2 norm, the failed
        span's L2 norm or NaN)."""
        k = ctypes.c_long()
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self._L.starmap_health(self._h, ctypes.byref(k), ctypes.byref(a), ctypes.byref(b)))
        return k.value, a.value, b.value

    def set_time_dependence(self, problem):
        """Hand the library a callback that evaluates the problem's material
        and sources at any time (starmap_set_time_dependence): from then on
        every step samples them at its midpoint t + dt/2 (section 5.7) and
        runs as O_1/2 E E O_1/2.  None turns it off."""
        if problem is None:
            self._check(self._L.starmap_set_time_dependence(self._h, FieldFn(), None, None, 0))
            self._td = None
            return
        zero = lambda t, x, y: 0.0 * x                                  # noqa: E731
        sa = problem.sigma_a or zero
        ss = problem.sigma_s0 or zero
        src = {}
        for j, q in problem.sources:
            src.setdefault(j, []).append(q)

        def fn(user, field, t, g, x, y, count, out):
            try:
                X = np.ctypeslib.as_array(x, shape=(count,))
                Y = np.ctypeslib.as_array(y, shape=(count,))
                dst = np.ctypeslib.as_array(out, shape=(count,))
                if field == FIELD_SIGMA_A:
                    dst[:] = np.broadcast_to(sa(t, X, Y), X.shape)
                elif field == FIELD_SIGMA_S0:
                    dst[:] = np.broadcast_to(ss(t, X, Y), X.shape)
                else:
                    dst[:] = sum(np.broadcast_to(q(t, X, Y), X.shape) for q in src[field - FIELD_SOURCE])
                return 0
            except Exception:                   # the library turns this into E_ARG
                return 1

        cb = FieldFn(fn)
        comps = np.array(sorted(src), dtype=np.int32)
        self._check(self._L.starmap_set_time_dependence(self._h, cb, None,
                                                        comps.ctypes.data_as(_ip) if comps.size else None,
                                                        int(comps.size)))
        self._td = (cb, comps)                  # kept alive while the library holds the pointer

    def step_time_dependent(self, problem, n: int = 1):
        """n steps of a problem whose material or sources change in time,
        through the library's time dependence (see set_time_dependence)."""
        if getattr(self, "_td_problem", None) is not problem:
            self.set_time_dependence(problem)
            self._td_problem = problem
        self.step(n)

    def run_pass(self, parity: int, which: int):
        self._check(self._L.starmap_pass(self._h, int(parity), int(which)))

    def advance_to(self, t: float):
        self._check(self._L.starmap_advance_to(self._h, float(t)))

    def output(self, j: int) -> np.ndarray:
        info = self.moment_info(j)
        out = np.empty((info["ny"], info["nx"]))
        self._check(self._L.starmap_output(self._h, j, _dptr(out), out.size))
        return out

    def sync(self):
        self._check(self._L.starmap_sync(self._h))

    # -- read-out -------------------------------------------------------
    def moments(self, j: int) -> np.ndarray:
        info = self.moment_info(j)
        out = np.empty((info["ny"], info["nx"]))
        self._check(self._L.starmap_moments(self._h, j, _dptr(out), out.size))
        return out

    def moments_window(self, j: int, i0: int, k0: int, nx: int, ny: int) -> np.ndarray:
        out = np.empty((ny, nx))
        self._check(self._L.starmap_moments_window(self._h, j, i0, k0, nx, ny, _dptr(out), out.size))
        return out

    def diagnostics(self):
        m, l2 = ctypes.c_double(), ctypes.c_double()
        bad = ctypes.c_long()
        rc = self._L.starmap_diagnostics(self._h, ctypes.byref(m), ctypes.byref(l2), ctypes.byref(bad))
        if rc not in (OK, E_NONFINITE):
            self._check(rc)
        return m.value, l2.value, bad.value

    def device_ptr(self, j: int):
        p = ctypes.c_void_p()
        pitch, off = ctypes.c_long(), ctypes.c_long()
        self._check(self._L.starmap_device_ptr(self._h, j, ctypes.byref(p), ctypes.byref(pitch), ctypes.byref(off)))
        return p.value, pitch.value, off.value

    def pack_rows(self, g: int, y0: int, rows: int, buf: int, nbytes: int):
        """Rows [y0, y0 + rows) of every component of grid g into the buffer
        at address buf ([component][row][x], the run's precision)."""
        self._check(self._L.starmap_pack_rows(self._h, int(g), int(y0), int(rows), ctypes.c_void_p(buf),
                                              int(nbytes)))

    def unpack_rows(self, g: int, y0: int, rows: int, buf: int, nbytes: int):
        self._check(self._L.starmap_unpack_rows(self._h, int(g), int(y0), int(rows), ctypes.c_void_p(buf),
                                                int(nbytes)))

    def state_bytes(self) -> int:
        return self._L.starmap_state_bytes(self._h)

    def get_state(self) -> bytes:
        buf = ctypes.create_string_buffer(self.state_bytes())
        self._check(self._L.starmap_get_state(self._h, buf, len(buf)))
        return buf.raw

    def set_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        self._check(self._L.starmap_set_state(self._h, buf, len(data)))

    # -- learned closure -------------------------------------------------
    def set_closure(self, params):
        """Network of a closure handle from FP32 parameters (MLP_PARAMS values)."""
        a = _params32(params)
        self._check(self._L.starmap_set_closure(self._h, a.ctypes.data_as(_fp), a.size))

    def set_closure_engine(self, engine: str):
        """"mma_sync" or "tcgen05": tensor-core path of the closure network."""
        self._check(self._L.starmap_set_closure_engine(self._h, {"mma_sync": ENGINE_MMA_SYNC,
                                                                 "tcgen05": ENGINE_TCGEN05}[engine]))

    def closure_samples(self, X, scale, targets=None):
        """Network inputs X [M, 38], scales s [M] and (optionally) the
        order-8 moments divided by s, targets [M, 9], of the current state,
        written into caller-owned device buffers (torch tensors or
        addresses), M = n_x * n_y."""
        nx, ny, *_ = self.grid_info(0)
        self._check(self._L.starmap_closure_samples(self._h, _addr(X), _addr(scale), _addr(targets), nx * ny))

    # -- convenience: load an input-module Problem ---------------------------
    @classmethod
    def from_problem(cls, problem, t_eval: float = 0.0, **over) -> "Stepper":
        kw = dict(N=problem.N, ax=problem.ax, n=problem.n, bc=problem.bc, cn=problem.cn,
                  precision=problem.precision, system=problem.system)
        kw.update(over)
        s = cls(**kw)
        s.load_problem(problem, t_eval)
        return s

    def load_problem(self, problem, t_eval: float = 0.0, ic: bool = True, factors: bool = True):
        """Sample material, sources and initial conditions of a Problem at
        the points of each grid and upload them (factors: also the
        per-order scattering factors)."""
        if factors and problem.sigma_sl_factor is not None:
            self.set_scattering_factors(problem.sigma_sl_factor)
        for g in range(4):
            nx, ny, *_ = self.grid_info(g)
            if nx * ny == 0:
                continue
            X, Y = self.grid_coords(g)
            sa = np.broadcast_to(problem.sigma_a(t_eval, X, Y), X.shape) if problem.sigma_a else np.zeros_like(X)
            ss = np.broadcast_to(problem.sigma_s0(t_eval, X, Y), X.shape) if problem.sigma_s0 else np.zeros_like(X)
            self.set_material(g, sa, ss)
        acc = {}
        for j, q in problem.sources:
            X, Y = self.grid_coords(self.moment_info(j)["grid"])
            acc[j] = acc.get(j, 0.0) + np.broadcast_to(q(t_eval, X, Y), X.shape)
        for j, q in acc.items():
            self.set_source(j, q)
        if ic:
            for j, f in problem.ic:
                X, Y = self.grid_coords(self.moment_info(j)["grid"])
                self.set_moment(j, np.broadcast_to(f(0.0, X, Y), X.shape))


class Network:
    """The closure network on the device (starmap_mlp_t): inference, loss
    gradient and Adam training steps over caller-owned device buffers."""

    def __init__(self, params, stream: Optional[int] = None):
        self._L = lib()
        a = _params32(params)
        h = ctypes.c_void_p()
        rc = self._L.starmap_mlp_create(a.ctypes.data_as(_fp), a.size, stream, ctypes.byref(h))
        if rc != OK:
            raise StarmapError(rc, self._L.starmap_mlp_last_error(None).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.starmap_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != OK:
            raise StarmapError(rc, self._L.starmap_mlp_last_error(self._h).decode())

    @property
    def params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, dtype=np.float32)
        self._check(self._L.starmap_mlp_get_params(self._h, out.ctypes.data_as(_fp), out.size))
        return out

    @params.setter
    def params(self, p):
        a = _params32(p)
        self._check(self._L.starmap_mlp_set_params(self._h, a.ctypes.data_as(_fp), a.size))

    @property
    def steps(self) -> int:
        return self._L.starmap_mlp_steps(self._h)

    def set_engine(self, engine: str):
        """"mma_sync" or "tcgen05" for forward(), loss_grad() and train_step()."""
        self._check(self._L.starmap_mlp_set_engine(self._h, {"mma_sync": ENGINE_MMA_SYNC,
                                                             "tcgen05": ENGINE_TCGEN05}[engine]))

    def forward(self, X, M: int, Y):
        self._check(self._L.starmap_mlp_forward(self._h, _addr(X), int(M), _addr(Y)))

    def loss_grad(self, X, T, B: int, grad, loss=None, idx=None):
        self._check(self._L.starmap_mlp_loss_grad(self._h, _addr(X), _addr(T), _addr(idx), int(B), _addr(grad),
                                                  _addr(loss)))

    def train_step(self, X, T, B: int, lr: float, loss=None, idx=None):
        self._check(self._L.starmap_mlp_train_step(self._h, _addr(X), _addr(T), _addr(idx), int(B), float(lr),
                                                   _addr(loss)))

    def perturb_inputs(self, X, Xn, M: int, cols: int, sigma: float, seed: int):
        """Xn = X plus N(0, sigma^2) noise on the first cols inputs of each row."""
        self._check(self._L.starmap_mlp_perturb_inputs(self._h, _addr(X), _addr(Xn), int(M), int(cols),
                                                       float(sigma), int(seed) & 0xFFFFFFFFFFFFFFFF))

    def shuffle(self, index, count: int, seed: int, out):
        """out[i] = index[perm(i)] on the device (index None: perm(i)), perm a
        seeded pseudo-random permutation of range(count)."""
        self._check(self._L.starmap_mlp_shuffle(self._h, _addr(index), int(count),
                                                int(seed) & 0xFFFFFFFFFFFFFFFF, _addr(out)))

    def sync(self):
        self._check(self._L.starmap_mlp_sync(self._h))


def params_from_dict(p) -> np.ndarray:
    """Flatten {W1, b1, W2, b2, W3, b3} into the C ABI's parameter vector."""
    return np.concatenate([np.asarray(p[k], dtype=np.float32).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def params_to_dict(v) -> dict:
    """Inverse of params_from_dict (float64 arrays)."""
    v = np.asarray(v, dtype=np.float64)
    shapes = [("W1", (MLP_HIDDEN, MLP_INPUTS)), ("b1", (MLP_HIDDEN,)), ("W2", (MLP_HIDDEN, MLP_HIDDEN)),
              ("b2", (MLP_HIDDEN,)), ("W3", (MLP_OUTPUTS, MLP_HIDDEN)), ("b3", (MLP_OUTPUTS,))]
    out, o = {}, 0
    for k, shp in shapes:
        n = int(np.prod(shp))
        out[k] = v[o:o + n].reshape(shp).copy()
        o += n
    assert o == MLP_PARAMS
    return out


class Batch:
    """Independent FP32 2D P_N instances stepped together (starmap_batch_t):
    one graph launch per step call, a persistent kernel per pass."""

    def __init__(self, configs, stream: Optional[int] = None):
        """configs: list of dicts of make_config keywords (precision fp32)."""
        self._L = lib()
        arr = (Config * len(configs))()
        for i, kw in enumerate(configs):
            kw = dict(kw)
            kw.setdefault("precision", "fp32")
            arr[i] = make_config(**kw)
        if stream is not None:
            arr[0].cuda_stream = stream
        h = ctypes.c_void_p()
        rc = self._L.starmap_batch_create(arr, len(configs), ctypes.byref(h))
        if rc != OK:
            raise StarmapError(rc, self._L.starmap_batch_last_error(None).decode())
        self._h = h
        self._inst = [Stepper._borrow(self._L.starmap_batch_instance(h, i), "fp32") for i in range(len(configs))]

    @classmethod
    def from_problems(cls, problems, schedule: str = "merged", stream: Optional[int] = None,
                      kernel: str = "auto") -> "Batch":
        """kernel: "auto" (autotuned tile height), "tiled_tall" or "tiled_short"."""
        cfgs = [dict(N=p.N, ax=p.ax, n=p.n, bc=p.bc, cn=p.cn, precision="fp32", schedule=schedule,
                     kernel=kernel) for p in problems]
        b = cls(cfgs, stream=stream)
        for inst, p in zip(b.instances, problems):
            inst.load_problem(p)
        return b

    def close(self):
        if getattr(self, "_h", None):
            for s in self._inst:
                s._h = None
            self._L.starmap_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != OK:
            raise StarmapError(rc, self._L.starmap_batch_last_error(self._h).decode())

    @property
    def instances(self):
        return self._inst

    def __len__(self):
        return len(self._inst)

    def tile_rows(self):
        """(rows of the batch's tiles, autotuner ms/step with 10-row tiles, with 5-row tiles)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        rows = self._L.starmap_batch_tile_rows(self._h, ctypes.byref(a), ctypes.byref(b))
        return rows, a.value, b.value

    def tuning(self):
        """(tile rows, stages per strip, from the tuning cache)."""
        r, s, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self._L.starmap_batch_tuning(self._h, ctypes.byref(r), ctypes.byref(s), ctypes.byref(c)))
        return r.value, s.value, bool(c.value)

    def launches(self, nsteps: int) -> int:
        return self._L.starmap_batch_launches(self._h, int(nsteps))

    def step(self, n: int = 1):
        self._check(self._L.starmap_batch_step(self._h, int(n)))

    def sync(self):
        self._check(self._L.starmap_batch_sync(self._h))
