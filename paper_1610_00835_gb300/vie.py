"""ctypes binding of libvie.so: the same names as the C ABI in include/vie.h.

Argument marshalling only: every numeric step runs in the library's CUDA
kernels.  There is no fallback; if the library is missing or no GPU is
present the calls raise.  Tensors may be CUDA tensors (used in place, work
queued on the current torch stream) or CPU tensors / numpy arrays (copied by
the library through its own device buffers).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

VIE_OK, VIE_ERR_INVALID_ARG, VIE_ERR_CUDA, VIE_ERR_OOM = 0, 1, 2, 3
VIE_ERR_NOT_CONVERGED, VIE_ERR_TIMEOUT, VIE_ERR_NONFINITE, VIE_ERR_UNSUPPORTED = 4, 5, 6, 7
STATUS_NAMES = {0: "VIE_OK", 1: "VIE_ERR_INVALID_ARG", 2: "VIE_ERR_CUDA", 3: "VIE_ERR_OOM",
                4: "VIE_ERR_NOT_CONVERGED", 5: "VIE_ERR_TIMEOUT", 6: "VIE_ERR_NONFINITE",
                7: "VIE_ERR_UNSUPPORTED"}
VIE_TAU_MARCH, VIE_TAU_CLOSED = 0, 1
VIE_PREC_FP32, VIE_PREC_FP64 = 0, 1
VIE_DISC_MIII, VIE_DISC_MII = 0, 1
VIE_OP_K_SIGMA_S, VIE_OP_I_MINUS_K, VIE_OP_A_RAW = 0, 1, 2
VIE_OPERATOR_OTF, VIE_OPERATOR_FP32, VIE_OPERATOR_BF16X3, VIE_OPERATOR_PAIRS32, VIE_OPERATOR_SYM32 = 0, 1, 2, 3, 4
VIE_OPERATOR_FMM = 5
VIE_KERNEL_AUTO, VIE_KERNEL_SYMMETRIC, VIE_KERNEL_DISPLACEMENT, VIE_KERNEL_GENERAL = 0, 1, 2, 3


class VieError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class vie_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int)]


class vie_opts(C.Structure):
    _fields_ = [("steps", C.c_int), ("tau_mode", C.c_int), ("precision", C.c_int),
                ("device", C.c_int), ("kernel", C.c_int), ("disc", C.c_int)]


class vie_gmres_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("restart", C.c_int), ("maxit", C.c_int),
                ("zero_x0", C.c_int), ("rhs_is_phi", C.c_int), ("time_apply", C.c_int),
                ("nrhs", C.c_int)]


class vie_report(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("converged", C.c_int),
                ("n_apply", C.c_int), ("relres", C.c_double), ("relres_est", C.c_double),
                ("t_total_ms", C.c_double), ("t_apply_ms", C.c_double),
                ("t_apply_kernel_ms", C.c_double), ("precond_iters", C.c_int),
                ("fell_back", C.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


# Every symbol include/vie.h declares, with its ctypes signature.
_vp = C.c_void_p
SIGNATURES = {
    "vie_default_opts": (None, [C.POINTER(vie_opts)]),
    "vie_default_gmres_opts": (None, [C.POINTER(vie_gmres_opts)]),
    "vie_create": (C.c_int, [C.POINTER(_vp), C.POINTER(vie_grid), _vp, _vp, C.POINTER(vie_opts)]),
    "vie_destroy": (C.c_int, [_vp]),
    "vie_apply": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, _vp]),
    "vie_solve_gmres": (C.c_int, [_vp, _vp, _vp, C.POINTER(vie_gmres_opts),
                                  C.POINTER(vie_report), _vp]),
    "ert_sweep": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, _vp, _vp]),
    "vie_get_diagonal": (C.c_int, [_vp, _vp, _vp]),
    "vie_get_kernel": (C.c_int, [_vp, C.POINTER(C.c_int)]),
    "vie_get_kernel_work": (C.c_int, [_vp, C.POINTER(C.c_double)]),
    "vie_last_error": (C.c_char_p, []),
    "vie_version": (C.c_char_p, []),
    "vie_kernel_launches": (C.c_ulonglong, []),
    "vie_assemble": (C.c_int, [_vp, C.c_int, _vp]),
    "vie_assemble_fmm": (C.c_int, [_vp, C.c_int, _vp]),
    "vie_batch_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(vie_grid),
                                   C.POINTER(_vp), C.POINTER(_vp), C.POINTER(vie_opts)]),
    "vie_batch_destroy": (C.c_int, [_vp]),
    "vie_batch_layout": (C.c_int, [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "vie_batch_apply": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, _vp]),
    "vie_batch_autotune": (C.c_int, [_vp, C.c_char_p, _vp]),
    "vie_batch_config": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "vie_unet_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, C.c_ulonglong, C.c_int]),
    "vie_unet_destroy": (C.c_int, [_vp]),
    "vie_unet_num_params": (C.c_int, [_vp, C.POINTER(C.c_longlong)]),
    "vie_unet_get_params": (C.c_int, [_vp, _vp]),
    "vie_unet_set_params": (C.c_int, [_vp, _vp]),
    "vie_unet_forward": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp]),
    "vie_unet_loss_grad": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _vp, C.POINTER(C.c_double), _vp]),
    "vie_release_memory": (C.c_int, []),
    "vie_unet_train_step": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, C.c_int, C.c_float,
                                      C.POINTER(C.c_double), _vp]),
    "vie_unet_save": (C.c_int, [_vp, C.c_char_p]),
    "vie_unet_load": (C.c_int, [_vp, C.c_char_p]),
    "vie_unet_train_state": (C.c_int, [_vp, C.POINTER(C.c_longlong)]),
    "vie_set_wait_limits": (C.c_int, [C.c_double, C.c_double]),
    "vie_unet_layer_io": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    "vie_check_device": (C.c_int, [_vp, _vp]),
    "vie_set_preconditioner": (C.c_int, [_vp, _vp, C.c_double]),
    "vie_set_preconditioner_on_diffusion": (C.c_int, [_vp, _vp, C.c_double, _vp]),
    "vie_set_fft_preconditioner": (C.c_int, [_vp, C.c_int, _vp]),
    "vie_fft_precondition": (C.c_int, [_vp, _vp, _vp, _vp]),
    "vie_set_diffusion_preconditioner": (C.c_int, [_vp, C.c_int, _vp]),
    "vie_diffusion_precondition": (C.c_int, [_vp, _vp, _vp, _vp]),
    "vie_apply_noalloc": (C.c_int, [C.c_int, C.c_int, _vp, _vp, C.c_int, _vp, _vp, _vp]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libvie.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libvie.so not found at {path}; run __graft_entry__.build()")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != VIE_OK:
        raise VieError(status, load().vie_last_error().decode())


def _ptr(x, dtype):
    """(pointer, keepalive) for a torch tensor or numpy array of `dtype`."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            want = {np.float64: torch.float64, np.float32: torch.float32}[dtype]
            if x.dtype != want:
                raise TypeError(f"expected {want}, got {x.dtype}")
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return C.c_void_p(x.data_ptr()), x
    except ImportError:
        pass
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array")
    return C.c_void_p(a.ctypes.data), a


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


@dataclass
class VieHandle:
    ptr: C.c_void_p
    dim: int
    n: int

    @property
    def N(self) -> int:
        return self.n ** self.dim

    def __del__(self):
        try:
            if self.ptr:
                vie_destroy(self)
        except Exception:
            pass


def vie_create(dim: int, n: int, sigma_t, sigma_s, steps: int = 64, tau_mode: int = VIE_TAU_MARCH,
               precision: int = VIE_PREC_FP32, device: int = 0,
               kernel: int = VIE_KERNEL_AUTO, disc: int = VIE_DISC_MIII) -> VieHandle:
    L = load()
    st = np.ascontiguousarray(np.asarray(sigma_t, dtype=np.float64).ravel())
    ss = np.ascontiguousarray(np.asarray(sigma_s, dtype=np.float64).ravel())
    g = vie_grid(dim, n)
    o = vie_opts(steps, tau_mode, precision, device, kernel, disc)
    h = C.c_void_p()
    _check(L.vie_create(C.byref(h), C.byref(g), C.c_void_p(st.ctypes.data),
                        C.c_void_p(ss.ctypes.data), C.byref(o)))
    return VieHandle(h, dim, n)


def vie_destroy(h: VieHandle) -> None:
    if h.ptr:
        _check(load().vie_destroy(h.ptr))
        h.ptr = C.c_void_p()


def vie_apply(h: VieHandle, op: int, g, y, nrhs: int = 1, stream=None) -> None:
    gp, _g = _ptr(g, np.float64)
    yp, _y = _ptr(y, np.float64)
    _check(load().vie_apply(h.ptr, op, gp, yp, nrhs, _stream(stream)))


def vie_assemble(h: VieHandle, mode: int, stream=None) -> None:
    _check(load().vie_assemble(h.ptr, mode, _stream(stream)))


def vie_assemble_fmm(h: VieHandle, order: int = 6, stream=None) -> None:
    _check(load().vie_assemble_fmm(h.ptr, order, _stream(stream)))


def vie_solve_gmres(h: VieHandle, f, U, rtol: float = 1e-6, restart: int = 64, maxit: int = 1000,
                    zero_x0: bool = True, rhs_is_phi: bool = False, time_apply: bool = False,
                    stream=None, raise_on_nonconvergence: bool = True, nrhs: int = 1):
    """One solve (returns its report as a dict), or nrhs > 1 solves in
    lockstep with f and U of nrhs * N values (returns a list of reports)."""
    fp, _f = _ptr(f, np.float64)
    up, _u = _ptr(U, np.float64)
    o = vie_gmres_opts(rtol, restart, maxit, int(zero_x0), int(rhs_is_phi), int(time_apply), int(nrhs))
    reps = (vie_report * max(1, int(nrhs)))()
    s = load().vie_solve_gmres(h.ptr, fp, up, C.byref(o), reps, _stream(stream))
    out = [r.as_dict() for r in reps] if nrhs > 1 else reps[0].as_dict()
    if s == VIE_ERR_NOT_CONVERGED and not raise_on_nonconvergence:
        return out
    _check(s)
    return out


def vie_apply_noalloc(dim: int, n: int, sigma_t, sigma_s, op: int, g, y, stream=None) -> None:
    """vie_apply without any device allocation; all arrays must be CUDA tensors."""
    sp, _s1 = _ptr(sigma_t, np.float64)
    qp, _s2 = _ptr(sigma_s, np.float64)
    gp, _g = _ptr(g, np.float64)
    yp, _y = _ptr(y, np.float64)
    _check(load().vie_apply_noalloc(dim, n, sp, qp, op, gp, yp, _stream(stream)))


@dataclass
class VieBatch:
    ptr: C.c_void_p
    ns: list
    offsets: list

    @property
    def total(self) -> int:
        return self.offsets[-1]

    def __del__(self):
        try:
            if self.ptr:
                vie_batch_destroy(self)
        except Exception:
            pass


def vie_batch_create(ns, sigma_t_list, sigma_s_list, device: int = 0, kernel: int = VIE_KERNEL_AUTO) -> VieBatch:
    L = load()
    count = len(ns)
    grids = (vie_grid * count)(*[vie_grid(2, int(n)) for n in ns])
    st = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel()) for a in sigma_t_list]
    ss = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel()) for a in sigma_s_list]
    pst = (_vp * count)(*[a.ctypes.data for a in st])
    pss = (_vp * count)(*[a.ctypes.data for a in ss])
    o = vie_opts(64, VIE_TAU_MARCH, VIE_PREC_FP32, device, kernel)
    b = C.c_void_p()
    _check(L.vie_batch_create(C.byref(b), count, grids, pst, pss, C.byref(o)))
    total = C.c_longlong()
    offs = (C.c_longlong * (count + 1))()
    _check(L.vie_batch_layout(b, C.byref(total), offs))
    return VieBatch(b, list(ns), [int(x) for x in offs])


def vie_batch_destroy(b: VieBatch) -> None:
    if b.ptr:
        _check(load().vie_batch_destroy(b.ptr))
        b.ptr = C.c_void_p()


def vie_batch_apply(b: VieBatch, op: int, g, y, nrhs: int = 1, stream=None) -> None:
    """g, y: [nrhs][total] packed FP64 (host arrays or device tensors)."""
    gp, _g = _ptr(g, np.float64)
    yp, _y = _ptr(y, np.float64)
    _check(load().vie_batch_apply(b.ptr, op, gp, yp, nrhs, _stream(stream)))


def vie_batch_autotune(b: VieBatch, cache_path=None, stream=None) -> tuple:
    path = cache_path.encode() if cache_path else None
    _check(load().vie_batch_autotune(b.ptr, path, _stream(stream)))
    return vie_batch_config(b)


def vie_batch_config(b: VieBatch) -> tuple:
    g, p = C.c_int(), C.c_int()
    _check(load().vie_batch_config(b.ptr, C.byref(g), C.byref(p)))
    return g.value, p.value


@dataclass
class VieUnet:
    ptr: C.c_void_p
    levels: int
    channels: int

    def __del__(self):
        try:
            if self.ptr:
                vie_unet_destroy(self)
        except Exception:
            pass


def vie_unet_create(levels: int = 4, channels: int = 32, seed: int = 0, device: int = 0) -> VieUnet:
    u = C.c_void_p()
    _check(load().vie_unet_create(C.byref(u), levels, channels, seed, device))
    return VieUnet(u, levels, channels)


def vie_unet_destroy(u: VieUnet) -> None:
    if u.ptr:
        _check(load().vie_unet_destroy(u.ptr))
        u.ptr = C.c_void_p()


def vie_unet_num_params(u: VieUnet) -> int:
    n = C.c_longlong()
    _check(load().vie_unet_num_params(u.ptr, C.byref(n)))
    return n.value


def vie_unet_get_params(u: VieUnet) -> np.ndarray:
    out = np.empty(vie_unet_num_params(u), dtype=np.float32)
    _check(load().vie_unet_get_params(u.ptr, C.c_void_p(out.ctypes.data)))
    return out


def vie_unet_set_params(u: VieUnet, params) -> None:
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != vie_unet_num_params(u):
        raise ValueError("parameter count mismatch")
    _check(load().vie_unet_set_params(u.ptr, C.c_void_p(a.ctypes.data)))


def vie_unet_forward(u: VieUnet, x, o, B: int, n: int, use_bf16: bool = False, stream=None) -> None:
    xp, _x = _ptr(x, np.float32)
    op, _o = _ptr(o, np.float32)
    _check(load().vie_unet_forward(u.ptr, xp, op, B, n, int(use_bf16), _stream(stream)))


def vie_unet_loss_grad(u: VieUnet, x, t, B: int, n: int, stream=None):
    xp, _x = _ptr(x, np.float32)
    tp, _t = _ptr(t, np.float32)
    g = np.empty(vie_unet_num_params(u), dtype=np.float32)
    loss = C.c_double()
    _check(load().vie_unet_loss_grad(u.ptr, xp, tp, B, n, C.c_void_p(g.ctypes.data), C.byref(loss),
                                     _stream(stream)))
    return loss.value, g


def vie_unet_train_step(u: VieUnet, x, t, B: int, n: int, lr: float, weights=None,
                        stream=None) -> float:
    xp, _x = _ptr(x, np.float32)
    tp, _t = _ptr(t, np.float32)
    wp, _w = _ptr(weights, np.float32) if weights is not None else (None, None)
    loss = C.c_double()
    _check(load().vie_unet_train_step(u.ptr, xp, tp, wp, B, n, lr, C.byref(loss), _stream(stream)))
    return loss.value


def vie_unet_save(u: VieUnet, path: str) -> None:
    _check(load().vie_unet_save(u.ptr, path.encode()))


def vie_unet_load(u: VieUnet, path: str) -> None:
    _check(load().vie_unet_load(u.ptr, path.encode()))


def vie_set_wait_limits(limit_ms: float = 1000.0, first_wait_ms: float = -1.0) -> None:
    """Bounds of the tensor-core kernels' device waits (process-wide)."""
    _check(load().vie_set_wait_limits(float(limit_ms), float(first_wait_ms)))


def vie_check_device(h: VieHandle, stream=None) -> None:
    """Synchronise and raise VieError(VIE_ERR_TIMEOUT) if a bounded wait gave up."""
    _check(load().vie_check_device(h.ptr, _stream(stream)))


def vie_unet_layer_io(u: VieUnet, layer: int, inp, out, stream=None) -> None:
    """Input (unless None) and output of one convolution from the latest forward."""
    ip, _i = _ptr(inp, np.float32) if inp is not None else (None, None)
    op, _o = _ptr(out, np.float32)
    _check(load().vie_unet_layer_io(u.ptr, int(layer), ip, op, _stream(stream)))


def vie_unet_train_state(u: VieUnet) -> int:
    """Adam steps taken so far (a checkpoint restores it)."""
    st = C.c_longlong(0)
    _check(load().vie_unet_train_state(u.ptr, C.byref(st)))
    return st.value


def vie_set_preconditioner_on_diffusion(h: VieHandle, u, s_ref: float = 5.0, stream=None) -> None:
    """The network as a correction of the diffusion preconditioner (None removes both)."""
    _check(load().vie_set_preconditioner_on_diffusion(h.ptr, u.ptr if u is not None else None, float(s_ref),
                                                      _stream(stream)))


def vie_set_preconditioner(h: VieHandle, u, s_ref: float = 5.0) -> None:
    _check(load().vie_set_preconditioner(h.ptr, u.ptr if u is not None else None, s_ref))


def vie_set_fft_preconditioner(h: VieHandle, enable: bool = True, stream=None) -> None:
    _check(load().vie_set_fft_preconditioner(h.ptr, int(bool(enable)), _stream(stream)))


def vie_fft_precondition(h: VieHandle, v, z, stream=None) -> None:
    vp, _v = _ptr(v, np.float64)
    zp, _z = _ptr(z, np.float64)
    _check(load().vie_fft_precondition(h.ptr, vp, zp, _stream(stream)))


def vie_set_diffusion_preconditioner(h: VieHandle, enable: bool = True, stream=None) -> None:
    _check(load().vie_set_diffusion_preconditioner(h.ptr, int(bool(enable)), _stream(stream)))


def vie_diffusion_precondition(h: VieHandle, v, z, stream=None) -> None:
    vp, _v = _ptr(v, np.float64)
    zp, _z = _ptr(z, np.float64)
    _check(load().vie_diffusion_precondition(h.ptr, vp, zp, _stream(stream)))


def ert_sweep(h: VieHandle, U, f, dirs, Phi, stream=None) -> None:
    up, _u = _ptr(U, np.float64)
    fp, _f = _ptr(f, np.float64)
    dp, _d = _ptr(dirs, np.float32)
    M = int(np.prod(dirs.shape[:-1])) if hasattr(dirs, "shape") else len(dirs) // h.dim
    pp, _p = _ptr(Phi, np.float32)
    _check(load().ert_sweep(h.ptr, up, fp, dp, M, pp, _stream(stream)))


def vie_get_diagonal(h: VieHandle, d, stream=None) -> None:
    dp, _d = _ptr(d, np.float64)
    _check(load().vie_get_diagonal(h.ptr, dp, _stream(stream)))


def vie_get_kernel(h: VieHandle) -> int:
    k = C.c_int()
    _check(load().vie_get_kernel(h.ptr, C.byref(k)))
    return k.value


def vie_get_kernel_work(h: VieHandle) -> float:
    w = C.c_double()
    _check(load().vie_get_kernel_work(h.ptr, C.byref(w)))
    return w.value


def vie_last_error() -> str:
    return load().vie_last_error().decode()


def vie_version() -> str:
    return load().vie_version().decode()


def vie_kernel_launches() -> int:
    return int(load().vie_kernel_launches())


def vie_release_memory() -> None:
    """Return the library's cached device buffers to CUDA (include/vie.h)."""
    _check(load().vie_release_memory())
