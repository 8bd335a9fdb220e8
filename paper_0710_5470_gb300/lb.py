"""Python binding of liblb.so (the C ABI of include/lb.h).

Argument marshalling only: every step of the lattice Boltzmann update runs in
the library's CUDA kernels.  There is no CPU fallback; importing this module
without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LB_LIBRARY selects another build of the library (e.g. the index-checked one)
LIB_PATH = os.environ.get("LB_LIBRARY") or os.path.join(_HERE, "_build", "liblb.so")

D2Q9, D3Q19 = 0, 1
EQUILIBRIUM, FORCING = 0, 1
F64, F32, F16DEV, BF16DEV = 0, 1, 2, 3
STORAGE_NAMES = {"f64": F64, "f32": F32, "f16dev": F16DEV, "bf16dev": BF16DEV}
STATUS = {0: "LB_OK", 1: "LB_EINVAL", 2: "LB_ENOMEM", 3: "LB_ECUDA", 4: "LB_EUNSTABLE", 5: "LB_ETIMEOUT",
          6: "LB_ESTATE"}


class LBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class lb_free_params(C.Structure):
    _fields_ = [("wp58", C.c_double), ("wt58", C.c_double), ("wxx58", C.c_double), ("B", C.c_double),
                ("D", C.c_double), ("F", C.c_double)]


OPTIMUM_FREE = dict(wp58=1 / 12, wt58=1 / 12, wxx58=-1 / 24, B=1 / 12, D=1 / 6, F=1 / 12)


class lb_params(C.Structure):
    _fields_ = [("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("a", C.c_double), ("b", C.c_double), ("T", C.c_double), ("kappa", C.c_double),
                ("tau", C.c_double), ("scheme", C.c_int), ("storage", C.c_int), ("rho_ref", C.c_double)]


class lb_stats(C.Structure):
    _fields_ = [("mass", C.c_double), ("momentum", C.c_double * 3), ("max_u", C.c_double),
                ("max_v", C.c_double), ("min_rho", C.c_double), ("max_rho", C.c_double),
                ("step", C.c_longlong), ("status", C.c_int), ("dP", C.c_double), ("max_du", C.c_double),
                ("du_steps", C.c_longlong)]


class lb_instance(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("T", C.c_double), ("kappa", C.c_double), ("tau", C.c_double),
                ("radius", C.c_double)]


class lb_binary_params(C.Structure):
    _fields_ = [("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("A", C.c_double),
                ("B", C.c_double), ("kappa", C.c_double),
                ("Gamma", C.c_double), ("tau", C.c_double), ("tau_phi", C.c_double), ("scheme", C.c_int),
                ("storage", C.c_int)]


class lb_binary_stats(C.Structure):
    _fields_ = [("mass", C.c_double), ("phi_total", C.c_double), ("momentum", C.c_double * 3),
                ("max_u", C.c_double), ("max_v", C.c_double), ("min_phi", C.c_double), ("max_phi", C.c_double),
                ("step", C.c_longlong), ("status", C.c_int)]


_lib = None

_DPTR = C.POINTER(C.c_double)
_SIGNATURES = {
    "lb_version": (C.c_char_p, []),
    "lb_last_error": (C.c_char_p, []),
    "lb_coexistence": (C.c_int, [C.c_double, C.c_double, C.c_double, _DPTR, _DPTR]),
    "lb_create": (C.c_int, [C.POINTER(lb_params), C.c_void_p, C.POINTER(C.c_void_p)]),
    "lb_population_bytes": (C.c_int, [C.POINTER(lb_params), C.POINTER(C.c_size_t)]),
    "lb_create_with_buffers": (C.c_int, [C.POINTER(lb_params), C.c_void_p, C.c_void_p, C.c_size_t,
                                         C.POINTER(C.c_void_p)]),
    "lb_destroy": (C.c_int, [C.c_void_p]),
    "lb_get_coexistence": (C.c_int, [C.c_void_p, _DPTR, _DPTR]),
    "lb_init_drops": (C.c_int, [C.c_void_p, C.c_int, _DPTR, _DPTR, C.c_double]),
    "lb_init_fields": (C.c_int, [C.c_void_p, _DPTR, _DPTR]),
    "lb_set_populations": (C.c_int, [C.c_void_p, _DPTR]),
    "lb_get_populations": (C.c_int, [C.c_void_p, _DPTR]),
    "lb_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lb_synchronize": (C.c_int, [C.c_void_p]),
    "lb_fields": (C.c_int, [C.c_void_p, _DPTR, _DPTR, _DPTR]),
    "lb_stats_get": (C.c_int, [C.c_void_p, C.POINTER(lb_stats)]),
    "lb_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_int)]),
    "lb_set_free_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lb_device_state": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_size_t)]),
    "lb_set_probes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lb_get_probes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lb_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "lb_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lb_debug_bounds": (C.c_int, [C.POINTER(C.c_int), C.POINTER(C.c_ulonglong)]),
    "lb_params_hash": (C.c_int, [C.POINTER(lb_params), C.POINTER(C.c_ulonglong)]),
    "lb_kernel_info": (C.c_int, [C.c_void_p, C.c_char_p, C.c_size_t, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 C.POINTER(C.c_int), C.POINTER(C.c_size_t), C.POINTER(C.c_int)]),
    "lb_batch_create": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.POINTER(lb_instance),
                                  C.c_void_p, C.POINTER(C.c_void_p)]),
    "lb_batch_destroy": (C.c_int, [C.c_void_p]),
    "lb_batch_init_drops": (C.c_int, [C.c_void_p, C.c_double]),
    "lb_batch_init_fields": (C.c_int, [C.c_void_p, C.c_int, _DPTR, _DPTR]),
    "lb_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lb_batch_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lb_batch_run_to_steady": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_longlong, C.c_longlong,
                                         C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    "lb_batch_set_reference": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double]),
    "lb_batch_set_band": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int]),
    "lb_batch_set_self_test": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int]),
    "lb_batch_last_check": (C.c_int, [C.c_void_p, _DPTR, _DPTR, _DPTR, _DPTR]),
    "lb_batch_fields": (C.c_int, [C.c_void_p, C.c_int, _DPTR, _DPTR]),
    "lb_batch_populations": (C.c_int, [C.c_void_p, C.c_int, _DPTR]),
    "lb_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                                C.POINTER(C.c_longlong)]),
    "lb_ws_create": (C.c_int, [C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "lb_ws_destroy": (C.c_int, [C.c_void_p]),
    "lb_ws_num_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong)]),
    "lb_ws_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lb_ws_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lb_ws_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "lb_ws_predict_sym": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "lb_ws_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                  C.POINTER(C.c_double), C.c_void_p]),
    "lb_ws_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                              C.c_float, C.c_int, _DPTR]),
    "lb_ws_features": (C.c_int, [C.c_int, C.c_int, _DPTR, C.c_double, C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.c_double, C.c_void_p]),
    "lb_ws_decode": (C.c_int, [C.c_int, C.c_int, _DPTR, C.c_double, C.c_double, C.c_void_p, _DPTR, _DPTR]),
    "lb_ws3_create": (C.c_int, [C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "lb_ws3_destroy": (C.c_int, [C.c_void_p]),
    "lb_ws3_num_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong)]),
    "lb_ws3_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lb_ws3_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lb_ws3_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "lb_ws3_predict_sym": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "lb_ws3_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.POINTER(C.c_double), C.c_void_p]),
    "lb_ws3_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                               C.c_int, C.c_float, C.c_int, _DPTR]),
    "lb_ws3_decode": (C.c_int, [C.c_int, C.c_int, C.c_int, _DPTR, C.c_double, C.c_double, C.c_void_p, _DPTR,
                                _DPTR]),
    "lb_field_stats_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_longlong,
                                         C.c_void_p, C.c_void_p]),
    "lb_fma_peak": (C.c_int, [C.c_int, C.c_int, _DPTR]),
    "lb_work_list": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                               C.POINTER(C.c_int)]),
    "lb_get_populations_box": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _DPTR]),
    "lb_binary_create": (C.c_int, [C.POINTER(lb_binary_params), C.c_void_p, C.POINTER(C.c_void_p)]),
    "lb_binary_destroy": (C.c_int, [C.c_void_p]),
    "lb_binary_init_fields": (C.c_int, [C.c_void_p, _DPTR, _DPTR, _DPTR]),
    "lb_binary_set_populations": (C.c_int, [C.c_void_p, _DPTR, _DPTR]),
    "lb_binary_get_populations": (C.c_int, [C.c_void_p, _DPTR, _DPTR]),
    "lb_binary_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lb_binary_synchronize": (C.c_int, [C.c_void_p]),
    "lb_binary_fields": (C.c_int, [C.c_void_p, _DPTR, _DPTR, _DPTR, _DPTR, _DPTR]),
    "lb_binary_stats_get": (C.c_int, [C.c_void_p, C.POINTER(lb_binary_stats)]),
}


def load_library(path: str | None = None):
    """Load liblb.so (built by paper_0710_5470_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_0710_5470_gb300.build.build())")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise LBError(status, load_library().lb_last_error().decode())


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DPTR)


def coexistence(a: float, b: float, T: float):
    """lb_coexistence: Maxwell densities (rho_l, rho_g) of the van der Waals fluid."""
    rl, rg = C.c_double(), C.c_double()
    _check(load_library().lb_coexistence(a, b, T, C.byref(rl), C.byref(rg)))
    return rl.value, rg.value


def field_stats_noalloc(rho_ptr: int, u_ptr: int, v_ptr: int, dim: int, n: int, out_ptr: int,
                        stream: int = 0):
    """lb_field_stats_noalloc on caller-owned device buffers (raw device
    pointers as ints); allocates nothing.  Writes 8 doubles at out_ptr."""
    _check(load_library().lb_field_stats_noalloc(C.c_void_p(rho_ptr), C.c_void_p(u_ptr), C.c_void_p(v_ptr),
                                                 int(dim), int(n), C.c_void_p(out_ptr),
                                                 C.c_void_p(stream) if stream else None))


def work_list(sms: int, ctas_per_sm: int, shape, tile=(32, 8)) -> np.ndarray:
    """lb_work_list: the D3Q19 step's CTA work list for a lattice (nx, ny, nz) on a GPU
    with `sms` SMs, as an int array of (x0, y0, z0, z1) rows in launch order (host only)."""
    nx, ny, nz = (int(v) for v in shape)
    n = C.c_int()
    lib = load_library()
    _check(lib.lb_work_list(sms, ctas_per_sm, nx, ny, nz, tile[0], tile[1], None, 0, C.byref(n)))
    out = np.empty((n.value, 4), dtype=np.int32)
    _check(lib.lb_work_list(sms, ctas_per_sm, nx, ny, nz, tile[0], tile[1], out.ctypes.data_as(C.c_void_p),
                            n.value, C.byref(n)))
    return out


F64_FMA_ITERS, F32_FMA_ITERS = 4000, 200000


def fma_peak(precision: int, iters: int | None = None) -> float:
    """lb_fma_peak: the GPU's FMA rate in TFLOP/s, precision 0 = float64, 1 = float32."""
    if iters is None:
        iters = F64_FMA_ITERS if precision == 0 else F32_FMA_ITERS
    out = C.c_double()
    _check(load_library().lb_fma_peak(int(precision), int(iters), C.byref(out)))
    return out.value


def params_hash(lattice: int, shape, a: float, b: float, T: float, kappa: float, tau: float,
                scheme: int = EQUILIBRIUM, storage: int = F64, rho_ref: float = 0.0) -> int:
    """lb_params_hash (host only)."""
    nx, ny, nz = (tuple(shape) + (1,))[:3] if len(shape) == 2 else tuple(shape)
    p = lb_params(lattice, nx, ny, nz, a, b, T, kappa, tau, scheme, storage, rho_ref)
    h = C.c_ulonglong()
    _check(load_library().lb_params_hash(C.byref(p), C.byref(h)))
    return h.value


def population_bytes(lattice: int, shape, a: float, b: float, T: float, kappa: float, tau: float,
                     scheme: int = EQUILIBRIUM, storage: int = F64, rho_ref: float = 0.0) -> int:
    """lb_population_bytes (host only): bytes of a context's two population buffers."""
    nx, ny, nz = (tuple(shape) + (1,))[:3] if len(shape) == 2 else tuple(shape)
    p = lb_params(lattice, nx, ny, nz, a, b, T, kappa, tau, scheme, storage, rho_ref)
    n = C.c_size_t()
    _check(load_library().lb_population_bytes(C.byref(p), C.byref(n)))
    return n.value


def debug_bounds():
    """lb_debug_bounds: (index checks compiled in, first recorded violation or 0)."""
    c, v = C.c_int(), C.c_ulonglong()
    _check(load_library().lb_debug_bounds(C.byref(c), C.byref(v)))
    return bool(c.value), v.value


def version() -> str:
    return load_library().lb_version().decode()


class Context:
    """One lattice (lb_create ... lb_destroy)."""

    def __init__(self, lattice: int, shape, a: float, b: float, T: float, kappa: float, tau: float,
                 scheme: int = EQUILIBRIUM, storage: int = F64, rho_ref: float = 0.0, stream=None,
                 buffer=None):
        """buffer: optional caller-owned device memory for the population buffers
        (lb_create_with_buffers), an object with data_ptr() and nbytes (a CUDA
        tensor) or a (device pointer, bytes) pair; kept referenced by the context."""
        lib = load_library()
        nx, ny, nz = (tuple(shape) + (1,))[:3] if len(shape) == 2 else tuple(shape)
        self.params = lb_params(lattice, nx, ny, nz, a, b, T, kappa, tau, scheme, storage, rho_ref)
        self.dim = 2 if lattice == D2Q9 else 3
        self.q = 9 if lattice == D2Q9 else 19
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        h = C.c_void_p()
        st = C.c_void_p(int(stream)) if stream else None
        self._buffer = buffer
        if buffer is None:
            _check(lib.lb_create(C.byref(self.params), st, C.byref(h)))
        else:
            ptr, nbytes = (buffer.data_ptr(), buffer.nbytes) if hasattr(buffer, "data_ptr") else buffer
            _check(lib.lb_create_with_buffers(C.byref(self.params), st, C.c_void_p(int(ptr)), int(nbytes),
                                              C.byref(h)))
        self._h = h
        self._lib = lib

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.lb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls
    def coexistence(self):
        rl, rg = C.c_double(), C.c_double()
        _check(self._lib.lb_get_coexistence(self._h, C.byref(rl), C.byref(rg)))
        return rl.value, rg.value

    def init_drops(self, centres, radii, width: float = 2.0):
        c = np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(-1))
        r = np.ascontiguousarray(np.asarray(radii, dtype=np.float64).reshape(-1))
        _check(self._lib.lb_init_drops(self._h, len(r), _dptr(c) if len(r) else None,
                                       _dptr(r) if len(r) else None, width))

    def init_fields(self, rho: np.ndarray, u: np.ndarray | None = None):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        _check(self._lib.lb_init_fields(self._h, _dptr(rho), _dptr(uu)))

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == self.q * self.n
        _check(self._lib.lb_set_populations(self._h, _dptr(f)))

    def get_populations(self) -> np.ndarray:
        out = np.empty((self.q,) + self.shape, dtype=np.float64)
        _check(self._lib.lb_get_populations(self._h, _dptr(out)))
        return out

    def get_populations_box(self, origin, size) -> np.ndarray:
        """lb_get_populations_box: float64 populations of the periodic box at
        origin (x0, y0[, z0]) with size (bx, by[, bz]); shape (Q, bz, by, bx)."""
        o = (tuple(origin) + (0,))[:3]
        b = (tuple(size) + (1,))[:3]
        out = np.empty((self.q, b[2], b[1], b[0]), dtype=np.float64)
        _check(self._lib.lb_get_populations_box(self._h, *(int(v) for v in o), *(int(v) for v in b), _dptr(out)))
        return out

    def step(self, n: int = 1):
        _check(self._lib.lb_step(self._h, int(n)))

    def synchronize(self):
        _check(self._lib.lb_synchronize(self._h))

    def fields(self, want_v: bool = True):
        rho = np.empty(self.shape, dtype=np.float64)
        u = np.empty((self.dim,) + self.shape, dtype=np.float64)
        v = np.empty((self.dim,) + self.shape, dtype=np.float64) if want_v else None
        _check(self._lib.lb_fields(self._h, _dptr(rho), _dptr(u), _dptr(v)))
        return rho, u, v

    def fields_into(self, rho: np.ndarray, u: np.ndarray | None = None, v: np.ndarray | None = None):
        """lb_fields into caller-provided float64 arrays (e.g. pinned host memory)."""
        for a, k in ((rho, 1), (u, self.dim), (v, self.dim)):
            assert a is None or (a.dtype == np.float64 and a.size == k * self.n and a.flags["C_CONTIGUOUS"])
        _check(self._lib.lb_fields(self._h, _dptr(rho), _dptr(u), _dptr(v)))

    def set_free_params(self, **kw):
        """lb_set_free_params with the given values (others at the optimum)."""
        vals = dict(OPTIMUM_FREE)
        unknown = set(kw) - set(vals)
        if unknown:
            raise TypeError(f"unknown free parameters {sorted(unknown)}")
        vals.update(kw)
        fp = lb_free_params(**vals)
        _check(self._lib.lb_set_free_params(self._h, C.byref(fp)))

    def clear_free_params(self):
        _check(self._lib.lb_set_free_params(self._h, None))

    def stats(self) -> dict:
        s = lb_stats()
        _check(self._lib.lb_stats_get(self._h, C.byref(s)))
        return {"mass": s.mass, "momentum": list(s.momentum)[: self.dim], "max_u": s.max_u, "max_v": s.max_v,
                "min_rho": s.min_rho, "max_rho": s.max_rho, "step": s.step, "status": s.status, "dP": s.dP,
                "max_du": s.max_du, "du_steps": s.du_steps}

    def set_probes(self, inside, outside):
        """lb_set_probes: (x, y[, z]) sites of the dP probes."""
        i = (C.c_int * 3)(*((tuple(int(v) for v in inside) + (0,))[:3]))
        o = (C.c_int * 3)(*((tuple(int(v) for v in outside) + (0,))[:3]))
        _check(self._lib.lb_set_probes(self._h, i, o))

    def probes(self):
        i, o = (C.c_int * 3)(), (C.c_int * 3)()
        _check(self._lib.lb_get_probes(self._h, i, o))
        return tuple(i), tuple(o)

    def get_state(self) -> bytes:
        """lb_get_state: header + raw population buffer."""
        n = C.c_size_t()
        _check(self._lib.lb_get_state(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(self._lib.lb_get_state(self._h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def set_state(self, state: bytes):
        """lb_set_state: import a state exported by a context with the same parameters."""
        buf = C.create_string_buffer(bytes(state), len(state))
        _check(self._lib.lb_set_state(self._h, buf, len(state)))

    def kernel_info(self) -> dict:
        """lb_kernel_info: launch form of the fused step kernel."""
        buf = C.create_string_buffer(128)
        tx, ty, th, ctas = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        sm = C.c_size_t()
        _check(self._lib.lb_kernel_info(self._h, buf, 128, C.byref(tx), C.byref(ty), C.byref(th), C.byref(sm),
                                        C.byref(ctas)))
        return {"form": buf.value.decode(), "tile": [tx.value, ty.value], "threads": th.value,
                "smem_bytes": sm.value, "ctas": ctas.value}

    def device_state(self):
        p, nb = C.c_void_p(), C.c_size_t()
        _check(self._lib.lb_device_state(self._h, C.byref(p), C.byref(nb)))
        return p.value, nb.value


class Batch:
    """Independent D2Q9 drop runs advanced together (lb_batch_*)."""

    def __init__(self, instances, a: float, b: float, scheme: int = EQUILIBRIUM, storage: int = F64, stream=None):
        lib = load_library()
        self.instances = [dict(d) for d in instances]
        arr = (lb_instance * len(instances))(*[lb_instance(d["nx"], d["ny"], d["T"], d["kappa"], d["tau"],
                                                              d.get("radius", 0.0)) for d in instances])
        h = C.c_void_p()
        st = C.c_void_p(int(stream)) if stream else None
        _check(lib.lb_batch_create(scheme, storage, a, b, len(instances), arr, st, C.byref(h)))
        self._h, self._lib, self.n = h, lib, len(instances)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init_drops(self, width: float = 2.0):
        _check(self._lib.lb_batch_init_drops(self._h, width))

    def init_fields(self, k: int, rho: np.ndarray, u: np.ndarray | None = None):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        _check(self._lib.lb_batch_init_fields(self._h, k, _dptr(rho), _dptr(uu)))

    def step(self, n: int = 1):
        _check(self._lib.lb_batch_step(self._h, int(n)))

    def autotune(self, steps: int = 10):
        tx, ty = C.c_int(), C.c_int()
        _check(self._lib.lb_batch_autotune(self._h, steps, C.byref(tx), C.byref(ty)))
        return tx.value, ty.value

    def run_to_steady(self, tol: float = 1e-10, every: int = 100, min_steps: int = 0, max_steps: int = 200000):
        steps = (C.c_longlong * self.n)()
        status = (C.c_int * self.n)()
        total = C.c_longlong()
        _check(self._lib.lb_batch_run_to_steady(self._h, tol, every, min_steps, max_steps, steps, status,
                                                C.byref(total)))
        return list(steps), list(status), total.value

    def set_reference(self, k: int, umax_ref: float, rho_max_ref: float = 0.0, rho_min_ref: float = 0.0):
        """Reference steady state of instance k for the reference test
        (lb_batch_set_reference); umax_ref = 0 clears it."""
        _check(self._lib.lb_batch_set_reference(self._h, k, float(umax_ref), float(rho_max_ref), float(rho_min_ref)))

    def set_band(self, band: float = 0.05, tol_rho: float = 1e-3, hold: int = 10):
        _check(self._lib.lb_batch_set_band(self._h, band, tol_rho, hold))

    def set_self_test(self, rtol_u: float = 1e-3, tol_rho: float = 1e-5, hold: int = 10):
        """lb_batch_set_self_test: steady once max|u| and the bulk densities settle
        (no reference values); rtol_u = 0 switches it off."""
        _check(self._lib.lb_batch_set_self_test(self._h, float(rtol_u), float(tol_rho), int(hold)))

    def last_check(self):
        """(max|du|, max|u|, max rho, min rho) per instance at its last check."""
        out = [np.empty(self.n, dtype=np.float64) for _ in range(4)]
        _check(self._lib.lb_batch_last_check(self._h, *(_dptr(a) for a in out)))
        return tuple(out)

    def fields(self, k: int):
        d = self.instances[k]
        rho = np.empty((d["ny"], d["nx"]), dtype=np.float64)
        u = np.empty((2, d["ny"], d["nx"]), dtype=np.float64)
        _check(self._lib.lb_batch_fields(self._h, k, _dptr(rho), _dptr(u)))
        return rho, u

    def populations(self, k: int):
        d = self.instances[k]
        f = np.empty((9, 1, d["ny"], d["nx"]), dtype=np.float64)
        _check(self._lib.lb_batch_populations(self._h, k, _dptr(f)))
        return f

    def info(self):
        tx, ty, sites, steps = C.c_int(), C.c_int(), C.c_longlong(), C.c_longlong()
        _check(self._lib.lb_batch_info(self._h, C.byref(tx), C.byref(ty), C.byref(sites), C.byref(steps)))
        return {"tile": (tx.value, ty.value), "sites": sites.value, "steps": steps.value}


def _fptr(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


class WarmStart:
    """The warm-start network (lb_ws_*): 4 periodic 3x3 conv layers, 5 -> 32 -> 32 -> 32 -> 3."""

    def __init__(self, seed: int = 0, stream=None):
        lib = load_library()
        h = C.c_void_p()
        st = C.c_void_p(int(stream)) if stream else None
        _check(lib.lb_ws_create(seed, st, C.byref(h)))
        self._h, self._lib = h, lib
        n = C.c_longlong()
        _check(lib.lb_ws_num_params(h, C.byref(n)))
        self.num_params = n.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lb_ws_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def get_params(self) -> np.ndarray:
        p = np.empty(self.num_params, dtype=np.float32)
        _check(self._lib.lb_ws_get_params(self._h, _fptr(p), p.size))
        return p

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(self._lib.lb_ws_set_params(self._h, _fptr(p), p.size))

    def forward(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        n, c, H, W = x.shape
        y = np.empty((n, 3, H, W), dtype=np.float32)
        _check(self._lib.lb_ws_forward(self._h, _fptr(x), n, H, W, _fptr(y)))
        return y

    def predict_sym(self, x: np.ndarray) -> np.ndarray:
        """lb_ws_predict_sym: symmetry-averaged prediction for one drop (5 x H x W)."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        c, H, W = x.shape
        y = np.empty((3, H, W), dtype=np.float32)
        _check(self._lib.lb_ws_predict_sym(self._h, _fptr(x), H, W, _fptr(y)))
        return y

    def loss_grad(self, x: np.ndarray, t: np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        n, c, H, W = x.shape
        loss = C.c_double()
        g = np.empty(self.num_params, dtype=np.float32)
        _check(self._lib.lb_ws_loss_grad(self._h, _fptr(x), _fptr(t), n, H, W, C.byref(loss), _fptr(g)))
        return loss.value, g

    def train(self, x: np.ndarray, t: np.ndarray, epochs: int, batch: int, lr: float, seed: int = 0):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        n, c, H, W = x.shape
        hist = np.zeros(epochs, dtype=np.float64)
        _check(self._lib.lb_ws_train(self._h, _fptr(x), _fptr(t), n, H, W, epochs, batch, lr, seed, _dptr(hist)))
        return hist


class WarmStart3(WarmStart):
    """The 3D warm-start network (lb_ws3_*): 4 periodic 3x3x3 conv layers, 5 -> 32 -> 32 -> 32 -> 4."""

    def __init__(self, seed: int = 0, stream=None):
        lib = load_library()
        h = C.c_void_p()
        st = C.c_void_p(int(stream)) if stream else None
        _check(lib.lb_ws3_create(seed, st, C.byref(h)))
        self._h, self._lib = h, lib
        n = C.c_longlong()
        _check(lib.lb_ws3_num_params(h, C.byref(n)))
        self.num_params = n.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lb_ws3_destroy(self._h)
            self._h = None

    def get_params(self) -> np.ndarray:
        p = np.empty(self.num_params, dtype=np.float32)
        _check(self._lib.lb_ws3_get_params(self._h, _fptr(p), p.size))
        return p

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(self._lib.lb_ws3_set_params(self._h, _fptr(p), p.size))

    def forward(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        n, c, D, H, W = x.shape
        y = np.empty((n, 4, D, H, W), dtype=np.float32)
        _check(self._lib.lb_ws3_forward(self._h, _fptr(x), n, D, H, W, _fptr(y)))
        return y

    def predict_sym(self, x: np.ndarray) -> np.ndarray:
        """lb_ws3_predict_sym: reflection-averaged prediction for one drop (5 x D x H x W)."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        c, D, H, W = x.shape
        y = np.empty((4, D, H, W), dtype=np.float32)
        _check(self._lib.lb_ws3_predict_sym(self._h, _fptr(x), D, H, W, _fptr(y)))
        return y

    def loss_grad(self, x: np.ndarray, t: np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        n, c, D, H, W = x.shape
        loss = C.c_double()
        g = np.empty(self.num_params, dtype=np.float32)
        _check(self._lib.lb_ws3_loss_grad(self._h, _fptr(x), _fptr(t), n, D, H, W, C.byref(loss), _fptr(g)))
        return loss.value, g

    def train(self, x: np.ndarray, t: np.ndarray, epochs: int, batch: int, lr: float, seed: int = 0):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        n, c, D, H, W = x.shape
        hist = np.zeros(epochs, dtype=np.float64)
        _check(self._lib.lb_ws3_train(self._h, _fptr(x), _fptr(t), n, D, H, W, epochs, batch, lr, seed,
                                      _dptr(hist)))
        return hist


def ws_features(rho_tanh: np.ndarray, rho_l: float, rho_g: float, T: float, kappa: float, tau: float, R: float):
    """lb_ws_features: the 5 input planes (float32) of one drop, 2D (ny, nx) or 3D (nz, ny, nx)."""
    r = np.ascontiguousarray(rho_tanh, dtype=np.float64)
    nx = r.shape[-1]
    rows = r.size // nx
    x = np.empty((5,) + r.shape, dtype=np.float32)
    _check(load_library().lb_ws_features(nx, rows, _dptr(r), rho_l, rho_g, T, kappa, tau, R, _fptr(x)))
    return x


def ws3_decode(rho_tanh: np.ndarray, rho_l: float, rho_g: float, y: np.ndarray):
    """lb_ws3_decode: predicted volumes -> rho (nz, ny, nx), u (3, nz, ny, nx)."""
    r = np.ascontiguousarray(rho_tanh, dtype=np.float64)
    nz, ny, nx = r.shape
    y = np.ascontiguousarray(y, dtype=np.float32)
    rho = np.empty((nz, ny, nx), dtype=np.float64)
    u = np.empty((3, nz, ny, nx), dtype=np.float64)
    _check(load_library().lb_ws3_decode(nx, ny, nz, _dptr(r), rho_l, rho_g, _fptr(y), _dptr(rho), _dptr(u)))
    return rho, u


def ws_decode(rho_tanh: np.ndarray, rho_l: float, rho_g: float, y: np.ndarray):
    """lb_ws_decode: predicted planes -> rho (ny, nx), u (2, ny, nx)."""
    r = np.ascontiguousarray(rho_tanh, dtype=np.float64)
    ny, nx = r.shape[-2:]
    y = np.ascontiguousarray(y, dtype=np.float32)
    rho = np.empty((ny, nx), dtype=np.float64)
    u = np.empty((2, ny, nx), dtype=np.float64)
    _check(load_library().lb_ws_decode(nx, ny, _dptr(r), rho_l, rho_g, _fptr(y), _dptr(rho), _dptr(u)))
    return rho, u


class BinaryContext:
    """One binary-fluid lattice (lb_binary_create ... lb_binary_destroy).

    shape (nx, ny) selects D2Q9, (nx, ny, nz) D3Q19; fields are (ny, nx) or
    (nz, ny, nx) arrays, populations (Q, ...)."""

    def __init__(self, shape, A: float, B: float, kappa: float, Gamma: float, tau: float, tau_phi: float,
                 scheme: int = EQUILIBRIUM, storage: int = F64, stream=None):
        lib = load_library()
        dims = [int(v) for v in shape]
        self.dim = len(dims)
        nx, ny, nz = (dims + [1])[:3]
        self.q = 9 if self.dim == 2 else 19
        self.params = lb_binary_params(D2Q9 if self.dim == 2 else D3Q19, nx, ny, nz, A, B, kappa, Gamma, tau,
                                       tau_phi, scheme, storage)
        self.shape = (ny, nx) if self.dim == 2 else (nz, ny, nx)
        self.n = nx * ny * nz
        h = C.c_void_p()
        st = C.c_void_p(int(stream)) if stream else None
        _check(lib.lb_binary_create(C.byref(self.params), st, C.byref(h)))
        self._h = h
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lb_binary_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init_fields(self, rho: np.ndarray, phi: np.ndarray, u: np.ndarray | None = None):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        assert rho.size == self.n and phi.size == self.n and (uu is None or uu.size == self.dim * self.n)
        _check(self._lib.lb_binary_init_fields(self._h, _dptr(rho), _dptr(phi), _dptr(uu)))

    def set_populations(self, f: np.ndarray, g: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.size == self.q * self.n and g.size == self.q * self.n
        _check(self._lib.lb_binary_set_populations(self._h, _dptr(f), _dptr(g)))

    def get_populations(self):
        f = np.empty((self.q,) + self.shape, dtype=np.float64)
        g = np.empty((self.q,) + self.shape, dtype=np.float64)
        _check(self._lib.lb_binary_get_populations(self._h, _dptr(f), _dptr(g)))
        return f, g

    def step(self, n: int = 1):
        _check(self._lib.lb_binary_step(self._h, int(n)))

    def synchronize(self):
        _check(self._lib.lb_binary_synchronize(self._h))

    def fields(self):
        """rho, phi, u (D, ...), v (D, ...), mu."""
        rho = np.empty(self.shape)
        phi = np.empty(self.shape)
        u = np.empty((self.dim,) + self.shape)
        v = np.empty((self.dim,) + self.shape)
        mu = np.empty(self.shape)
        _check(self._lib.lb_binary_fields(self._h, _dptr(rho), _dptr(phi), _dptr(u), _dptr(v), _dptr(mu)))
        return rho, phi, u, v, mu

    def stats(self) -> dict:
        s = lb_binary_stats()
        _check(self._lib.lb_binary_stats_get(self._h, C.byref(s)))
        return {"mass": s.mass, "phi_total": s.phi_total, "momentum": list(s.momentum), "max_u": s.max_u,
                "max_v": s.max_v, "min_phi": s.min_phi, "max_phi": s.max_phi, "step": s.step, "status": s.status}
