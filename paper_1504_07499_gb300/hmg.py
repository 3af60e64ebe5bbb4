"""Python binding of libhmg (include/hmg.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method itself: arrays are passed as raw pointers (numpy arrays
as host pointers, torch CUDA tensors as device pointers) and results come back in
caller-provided buffers.  The CUDA library must be built (``build.build()``);
importing a function that needs it raises if libhmg.so is missing -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhmg.so")

HMG_OK, HMG_PENDING = 0, 1
HMG_INVALID_ARG, HMG_OUT_OF_MEMORY, HMG_NOT_CONVERGED = -1, -2, -3
HMG_DIVERGED, HMG_CUDA_ERROR, HMG_BUSY, HMG_UNKNOWN_TICKET = -4, -5, -6, -7
HMG_FP64, HMG_FP32_BULK = 0, 1
HMG_SCHEME_EYRE_MILTON, HMG_SCHEME_BASIC, HMG_SCHEME_AUGMENTED_LAGRANGIAN = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "PENDING", -1: "INVALID_ARG", -2: "OUT_OF_MEMORY", -3: "NOT_CONVERGED",
                -4: "DIVERGED", -5: "CUDA_ERROR", -6: "BUSY", -7: "UNKNOWN_TICKET"}

# every symbol include/hmg.h declares
EXPORTS = ["hmg_version", "hmg_last_error", "hmg_create", "hmg_destroy", "hmg_voxelize", "hmg_solve",
           "hmg_solve_fields", "hmg_em_iterate", "hmg_equilibrium", "hmg_fft_forward", "hmg_fft_inverse",
           "hmg_solve_batch", "hmg_submit", "hmg_poll", "hmg_footprint", "hmg_trace_enable",
           "hmg_trace_read", "hmg_equilibrium_noalloc", "hmg_set_variant", "hmg_get_variant",
           "hmg_server_stats", "hmg_solve_scheme", "hmg_solve_polarization", "hmg_rsa", "hmg_rve",
           "hmg_submit_rve", "hmg_fp64_rate", "hmg_voxelize_mixed"]
HMG_NOALLOC_MAX_N = 64
KERNEL_KINDS = ["x_forward", "y_forward", "z_green", "y_inverse", "x_inverse", "eq_x", "eq_z", "other",
                "x_round", "fp64", "yxy"]


class hmg_sphere(C.Structure):
    _fields_ = [("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double), ("r", C.c_double)]


class hmg_info(C.Structure):
    _fields_ = [("iters", C.c_int * 3), ("iters_fp64", C.c_int * 3), ("eps_comp", C.c_double * 3),
                ("eps_eq", C.c_double * 3), ("seconds", C.c_double), ("fp64_rounds", C.c_int),
                ("status", C.c_int * 3)]

    def as_dict(self) -> dict:
        return dict(iters=list(self.iters), iters_fp64=list(self.iters_fp64), eps_comp=list(self.eps_comp),
                    eps_eq=list(self.eps_eq), seconds=self.seconds, fp64_rounds=self.fp64_rounds,
                    status=[STATUS_NAMES.get(s, s) for s in self.status])


class HmgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """The loaded libhmg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libhmg.so not built ({LIB_PATH}); run paper_1504_07499_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
        dp = C.POINTER(C.c_double)
        L.hmg_version.restype = C.c_char_p
        L.hmg_last_error.restype = C.c_char_p
        L.hmg_create.argtypes = [C.POINTER(vp), i, sz]
        L.hmg_destroy.argtypes = [vp]
        L.hmg_voxelize.argtypes = [vp, vp, sz, d, i, vp]
        L.hmg_voxelize_mixed.argtypes = [vp, vp, sz, vp, sz, d, i, vp]
        L.hmg_rsa.argtypes = [vp, C.c_uint64, i, d, C.c_longlong, vp, C.POINTER(i)]
        L.hmg_rve.argtypes = [vp, C.c_uint64, i, d, C.c_longlong, d, i, vp, vp, C.POINTER(i)]
        L.hmg_solve.argtypes = [vp, vp, i, d, d, d, d, i, i, dp, C.POINTER(hmg_info)]
        L.hmg_solve_fields.argtypes = [vp, vp, i, d, d, d, d, i, i, dp, C.POINTER(hmg_info), vp]
        L.hmg_solve_scheme.argtypes = [vp, vp, i, d, d, d, d, i, i, i, dp, C.POINTER(hmg_info), vp]
        L.hmg_solve_polarization.argtypes = [vp, vp, i, d, d, d, d, i, d, i, dp, C.POINTER(hmg_info), vp]
        L.hmg_em_iterate.argtypes = [vp, vp, i, d, d, d, dp, i, i, vp, dp]
        L.hmg_equilibrium.argtypes = [vp, vp, i, d, d, d, i, vp, dp, dp]
        L.hmg_fft_forward.argtypes = [vp, i, i, i, vp, vp]
        L.hmg_fft_inverse.argtypes = [vp, i, i, i, vp, vp]
        L.hmg_solve_batch.argtypes = [vp, i, C.POINTER(vp), C.POINTER(i), dp, d, i, i, dp, C.POINTER(hmg_info)]
        L.hmg_submit.argtypes = [vp, vp, i, d, d, d, d, i, C.POINTER(C.c_uint64)]
        L.hmg_poll.argtypes = [vp, C.c_uint64, dp, C.POINTER(hmg_info)]
        L.hmg_submit_rve.argtypes = [vp, C.c_uint64, i, d, d, i, d, d, d, d, i, C.POINTER(C.c_uint64)]
        L.hmg_equilibrium_noalloc.argtypes = [vp, i, d, d, d, vp, dp, dp]
        L.hmg_server_stats.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.hmg_fp64_rate.argtypes = [vp, dp]
        L.hmg_set_variant.argtypes = [vp, i, i]
        L.hmg_get_variant.argtypes = [vp, i, C.POINTER(C.c_int)]
        L.hmg_trace_enable.argtypes = [vp, i]
        L.hmg_trace_read.argtypes = [vp, i, dp, C.POINTER(C.c_longlong), dp]
        L.hmg_footprint.argtypes = [i, i]
        L.hmg_footprint.restype = sz
        for name in EXPORTS:
            if name not in ("hmg_version", "hmg_last_error", "hmg_footprint"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _ptr(a) -> int:
    """Raw address of a numpy array (host) or torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def _check(status: int, allow=(HMG_OK,)) -> int:
    if status not in allow:
        raise HmgError(status, lib().hmg_last_error().decode())
    return status


def _dbuf(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# --- C entry points ------------------------------------------------------------

def hmg_version() -> str:
    return lib().hmg_version().decode()


def hmg_last_error() -> str:
    return lib().hmg_last_error().decode()


def hmg_footprint(N: int, precision: int = HMG_FP32_BULK) -> int:
    return lib().hmg_footprint(N, precision)


def hmg_create(device: int = 0, budget: int = 0) -> int:
    h = C.c_void_p()
    _check(lib().hmg_create(C.byref(h), device, budget))
    return h.value


def hmg_destroy(ctx: int) -> None:
    _check(lib().hmg_destroy(ctx))


def hmg_voxelize(ctx: int, spheres, layer: float, N: int, phase_out) -> None:
    """spheres: (n, 4) float64 array (cx, cy, cz, r) or device tensor; phase_out: N^3 uint8."""
    n = spheres.shape[0]
    _check(lib().hmg_voxelize(ctx, _ptr(spheres), n, layer, N, _ptr(phase_out)))


def hmg_voxelize_mixed(ctx: int, spheres, cylinders, layer: float, N: int, phase_out) -> None:
    """spheres: (n, 4) (or None), cylinders: (m, 8) cx, cy, cz, ux, uy, uz, r, h (or None);
    host arrays or device tensors; phase_out: N^3 uint8."""
    ns = 0 if spheres is None else spheres.shape[0]
    nc = 0 if cylinders is None else cylinders.shape[0]
    _check(lib().hmg_voxelize_mixed(ctx, _ptr(spheres) if ns else None, ns, _ptr(cylinders) if nc else None, nc,
                                    layer, N, _ptr(phase_out)))


def hmg_rsa(ctx: int, seed: int, n: int, r: float, max_candidates: int = 400_000, spheres_out=None):
    """Device sphere placement; returns ((n, 4) spheres, generator) -- spheres_out (host
    array or device tensor of n x 4 doubles) is filled when given."""
    out = spheres_out if spheres_out is not None else np.empty((n, 4))
    gen = C.c_int(-1)
    _check(lib().hmg_rsa(ctx, seed, n, r, max_candidates, _ptr(out), C.byref(gen)))
    return out, gen.value


def hmg_rve(ctx: int, seed: int, n: int, r: float, layer: float, N: int, phase_out, spheres_out=None,
            max_candidates: int = 400_000):
    """Device sphere placement + voxelization into phase_out (N^3 bytes); returns the generator."""
    gen = C.c_int(-1)
    _check(lib().hmg_rve(ctx, seed, n, r, max_candidates, layer, N, _ptr(phase_out),
                         _ptr(spheres_out) if spheres_out is not None else None, C.byref(gen)))
    return gen.value


def hmg_solve(ctx: int, phase, N: int, k, tol: float, precision: int, max_iter: int = 0,
              allow=(HMG_OK,)):
    K = np.zeros(9)
    info = hmg_info()
    st = lib().hmg_solve(ctx, _ptr(phase), N, k[0], k[1], k[2], tol, precision, max_iter, _dbuf(K), C.byref(info))
    _check(st, allow)
    return K.reshape(3, 3), info.as_dict(), st


def hmg_solve_fields(ctx: int, phase, N: int, k, tol: float, precision: int, e_out, max_iter: int = 0,
                     allow=(HMG_OK,)):
    K = np.zeros(9)
    info = hmg_info()
    st = lib().hmg_solve_fields(ctx, _ptr(phase), N, k[0], k[1], k[2], tol, precision, max_iter, _dbuf(K),
                                C.byref(info), _ptr(e_out))
    _check(st, allow)
    return K.reshape(3, 3), info.as_dict(), st


def hmg_solve_scheme(ctx: int, phase, N: int, k, tol: float, precision: int, scheme: int, e_out=None,
                     max_iter: int = 0, allow=(HMG_OK,)):
    K = np.zeros(9)
    info = hmg_info()
    st = lib().hmg_solve_scheme(ctx, _ptr(phase), N, k[0], k[1], k[2], tol, precision, scheme, max_iter, _dbuf(K),
                                C.byref(info), _ptr(e_out) if e_out is not None else None)
    _check(st, allow)
    return K.reshape(3, 3), info.as_dict(), st


def hmg_solve_polarization(ctx: int, phase, N: int, k, tol: float, precision: int, beta: float, e_out=None,
                           max_iter: int = 0, allow=(HMG_OK,)):
    K = np.zeros(9)
    info = hmg_info()
    st = lib().hmg_solve_polarization(ctx, _ptr(phase), N, k[0], k[1], k[2], tol, precision, beta, max_iter,
                                      _dbuf(K), C.byref(info), _ptr(e_out) if e_out is not None else None)
    _check(st, allow)
    return K.reshape(3, 3), info.as_dict(), st


def hmg_em_iterate(ctx: int, phase, N: int, k, grad_Theta, precision: int, n_iter: int, e_inout):
    g = np.ascontiguousarray(grad_Theta, dtype=np.float64)
    eps = np.zeros(max(n_iter, 1))
    _check(lib().hmg_em_iterate(ctx, _ptr(phase), N, k[0], k[1], k[2], _dbuf(g), precision, n_iter,
                                _ptr(e_inout), _dbuf(eps)))
    return eps[:n_iter]


def hmg_equilibrium(ctx: int, phase, N: int, k, precision: int, e):
    eps = np.zeros(1)
    flux = np.zeros(3)
    _check(lib().hmg_equilibrium(ctx, _ptr(phase), N, k[0], k[1], k[2], precision, _ptr(e), _dbuf(eps),
                                 _dbuf(flux)))
    return float(eps[0]), flux


def hmg_equilibrium_noalloc(phase, N: int, k, e):
    """hmg_equilibrium (FP64) with static scratch, for callers that cannot allocate
    device memory; N <= HMG_NOALLOC_MAX_N; runs on the current device."""
    eps = np.zeros(1)
    flux = np.zeros(3)
    _check(lib().hmg_equilibrium_noalloc(_ptr(phase), N, k[0], k[1], k[2], _ptr(e), _dbuf(eps), _dbuf(flux)))
    return float(eps[0]), flux


def hmg_fft_forward(ctx: int, N: int, count: int, precision: int, x, X_out) -> None:
    _check(lib().hmg_fft_forward(ctx, N, count, precision, _ptr(x), _ptr(X_out)))


def hmg_fft_inverse(ctx: int, N: int, count: int, precision: int, X, x_out) -> None:
    _check(lib().hmg_fft_inverse(ctx, N, count, precision, _ptr(X), _ptr(x_out)))


def hmg_solve_batch(ctx: int, phases, N_list, k3, tol: float, precision: int, max_iter: int = 0,
                    allow=(HMG_OK,)):
    n = len(phases)
    ptrs = (C.c_void_p * n)(*[_ptr(p) for p in phases])
    Ns = (C.c_int * n)(*N_list)
    kk = np.ascontiguousarray(k3, dtype=np.float64).reshape(-1)
    K = np.zeros(9 * n)
    infos = (hmg_info * n)()
    st = lib().hmg_solve_batch(ctx, n, ptrs, Ns, _dbuf(kk), tol, precision, max_iter, _dbuf(K), infos)
    _check(st, allow)
    return K.reshape(n, 3, 3), [x.as_dict() for x in infos], st


def hmg_submit(ctx: int, phase, N: int, k, tol: float, precision: int) -> int:
    t = C.c_uint64()
    _check(lib().hmg_submit(ctx, _ptr(phase), N, k[0], k[1], k[2], tol, precision, C.byref(t)))
    return t.value


def hmg_submit_rve(ctx: int, seed: int, n: int, r: float, layer: float, N: int, k, tol: float,
                   precision: int) -> int:
    t = C.c_uint64()
    _check(lib().hmg_submit_rve(ctx, seed, n, r, layer, N, k[0], k[1], k[2], tol, precision, C.byref(t)))
    return t.value


def hmg_poll(ctx: int, ticket: int):
    """Returns (status, K 3x3 or None, info dict or None)."""
    K = np.zeros(9)
    info = hmg_info()
    st = lib().hmg_poll(ctx, ticket, _dbuf(K), C.byref(info))
    if st == HMG_PENDING:
        return st, None, None
    _check(st, (HMG_OK, HMG_NOT_CONVERGED, HMG_DIVERGED))
    return st, K.reshape(3, 3), info.as_dict()


def hmg_fp64_rate(ctx: int) -> float:
    """Measured FP64 FMA rate of the context's GPU (flop/s)."""
    r = np.zeros(1)
    _check(lib().hmg_fp64_rate(ctx, _dbuf(r)))
    return float(r[0])


def hmg_server_stats(ctx: int) -> dict:
    out = (C.c_longlong * 6)()
    _check(lib().hmg_server_stats(ctx, out))
    keys = ["submitted", "completed", "max_resident", "ticks", "graph_captures", "graph_launches"]
    return dict(zip(keys, [int(v) for v in out]))


def hmg_set_variant(ctx: int, N: int, variant: int) -> None:
    _check(lib().hmg_set_variant(ctx, N, variant))


def hmg_get_variant(ctx: int, N: int) -> int:
    v = C.c_int()
    _check(lib().hmg_get_variant(ctx, N, C.byref(v)))
    return v.value


def hmg_trace_enable(ctx: int, enable: bool) -> None:
    _check(lib().hmg_trace_enable(ctx, 1 if enable else 0))


def hmg_trace_read(ctx: int) -> dict:
    """{kind name: (total ms, launches, algorithmic bytes)} for every kernel kind."""
    out = {}
    for k, name in enumerate(KERNEL_KINDS):
        ms, n, b = np.zeros(1), C.c_longlong(), np.zeros(1)
        _check(lib().hmg_trace_read(ctx, k, _dbuf(ms), C.byref(n), _dbuf(b)))
        out[name] = (float(ms[0]), int(n.value), float(b[0]))
    return out


@dataclass
class Context:
    """Owns one hmg context; a thin convenience wrapper over the functions above."""
    device: int = 0
    budget: int = 0

    def __post_init__(self):
        self.handle = hmg_create(self.device, self.budget)

    def close(self):
        if getattr(self, "handle", None):
            hmg_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def voxelize(self, spheres, layer: float, N: int, out=None):
        sph = np.ascontiguousarray(spheres, dtype=np.float64) if not hasattr(spheres, "data_ptr") else spheres
        if out is None:
            out = np.empty((N, N, N), dtype=np.uint8)
        hmg_voxelize(self.handle, sph, layer, N, out)
        return out

    def solve(self, phase, k, tol=1e-8, precision=HMG_FP64, max_iter=0, allow=(HMG_OK,)):
        N = phase.shape[-1]
        return hmg_solve(self.handle, phase, N, k, tol, precision, max_iter, allow)
