"""GB300 (sm_103a) implementation of the per-time-step hot path of the explicit
2k-order generalized-alpha method for isogeometric structural dynamics
(arXiv 2102.11536).

This module is a thin ctypes binding over libiga_galpha.so, whose C ABI is
declared in include/iga_galpha.h: it only marshals arguments. Every step of the
path runs in the library's CUDA kernels; there is no CPU fallback, and a missing
library raises at first use.

Device buffers are passed as torch CUDA tensors (float64, contiguous) or raw
integer device addresses.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libiga_galpha.so")
_LIB = None

OK, EINVAL, ENOMEM, ECUDA, ENOT_CONVERGED, ENUMERIC, EUNSTABLE, EGEOMETRY = range(8)
OP_FORMS = {"matrix_free": 0, "assembled": 1, "assembled_df": 2}
PRECONDS = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3, "banded": 4, "banded32": 5}
GUESSES = {"zero": 0, "prev": 1, "extrap": 2, "taylor": 3, "learned": 4}
NET_NPARAM = 1745


class IgaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("nquad", ctypes.c_int), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("precond", ctypes.c_int), ("op_form", ctypes.c_int), ("guess", ctypes.c_int),
                ("device", ctypes.c_int), ("stream", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("solves", ctypes.c_int), ("iters", ctypes.c_longlong),
                ("max_iters", ctypes.c_int), ("max_relres", ctypes.c_double), ("launches", ctypes.c_longlong),
                ("init_relres_sum", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib():
    """Load libiga_galpha.so (built by __graft_entry__.build() or paper_2102_11536_gb300.build)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError("libiga_galpha.so is not built (run __graft_entry__.build()); "
                          "there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    H = ctypes.c_void_p
    sig = {
        "iga_options_default": (None, [ctypes.POINTER(Options)]),
        "iga_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "iga_last_error": (ctypes.c_char_p, [H]),
        "iga_create": (ctypes.c_int, [ctypes.c_int, ip, ip, ctypes.POINTER(dp), dp, ctypes.POINTER(Options),
                                      ctypes.POINTER(H)]),
        "iga_destroy": (None, [H]),
        "iga_ndof": (ctypes.c_int, [H, ctypes.POINTER(ctypes.c_longlong)]),
        "iga_assemble": (ctypes.c_int, [H]),
        "iga_set_op_form": (ctypes.c_int, [H, ctypes.c_int]),
        "iga_set_precond": (ctypes.c_int, [H, ctypes.c_int]),
        "iga_set_guess": (ctypes.c_int, [H, ctypes.c_int]),
        "iga_set_tol": (ctypes.c_int, [H, ctypes.c_double, ctypes.c_int]),
        "iga_set_graphs": (ctypes.c_int, [H, ctypes.c_int]),
        "iga_set_barrier_limit": (ctypes.c_int, [H, ctypes.c_longlong]),
        "iga_apply_M": (ctypes.c_int, [H, ctypes.c_int, vp, vp]),
        "iga_apply_K": (ctypes.c_int, [H, ctypes.c_int, vp, vp]),
        "iga_apply_Pinv": (ctypes.c_int, [H, ctypes.c_int, vp, vp]),
        "iga_apply_Pinv_noalloc": (ctypes.c_int, [H, ctypes.c_int, vp, vp]),
        "iga_solve_M": (ctypes.c_int, [H, ctypes.c_int, vp, vp, ctypes.c_int, ip, dp]),
        "iga_galpha_params": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, dp, dp, dp]),
        "iga_cfl": (ctypes.c_int, [H, ctypes.c_double, ctypes.c_int, dp, dp]),
        "iga_state_init": (ctypes.c_int, [H, ctypes.c_int, vp, vp, vp]),
        "iga_step": (ctypes.c_int, [H, vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(Stats)]),
        "iga_step_host": (ctypes.c_int, [H, vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.POINTER(Stats)]),
        "iga_profile": (ctypes.c_int, [H, ctypes.c_int]),
        "iga_probe_fp64_fma": (ctypes.c_int, [ctypes.c_int, dp, dp]),
        "iga_profile_read": (ctypes.c_int, [H, dp, ctypes.POINTER(ctypes.c_longlong), dp, dp]),
        "iga_ws_collect": (ctypes.c_int, [H, ctypes.c_int]),
        "iga_ws_samples": (ctypes.c_int, [H, ip]),
        "iga_ws_train": (ctypes.c_int, [H, ctypes.c_int, ctypes.c_double, ctypes.c_ulonglong, dp]),
        "iga_ws_init_params": (ctypes.c_int, [H, ctypes.c_ulonglong]),
        "iga_ws_get_params": (ctypes.c_int, [H, vp]),
        "iga_ws_set_params": (ctypes.c_int, [H, vp]),
        "iga_ws_features": (ctypes.c_int, [H, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp]),
        "iga_net_forward": (ctypes.c_int, [ctypes.c_int] * 4 + [vp, vp, vp, vp, vp]),
        "iga_net_workspace_bytes": (ctypes.c_ulonglong, [ctypes.c_int] * 4),
        "iga_net_backward": (ctypes.c_int, [ctypes.c_int] * 4 + [vp, vp, vp, vp, vp, vp, ctypes.c_ulonglong, vp]),
        "iga_net_adam": (ctypes.c_int, [ctypes.c_int, vp, vp, vp, vp, ctypes.c_int, ctypes.c_double, vp]),
        "iga_set_band_config": (ctypes.c_int, [H, ctypes.c_int, ctypes.c_int]),
        "iga_band_df_tiny": (ctypes.c_int, [H, dp, dp]),
        "iga_set_damping": (ctypes.c_int, [H, ctypes.c_double, ctypes.c_double]),
        "iga_set_forcing": (ctypes.c_int, [H, ctypes.c_int, vp, dp, dp]),
        "iga_set_time": (ctypes.c_int, [H, ctypes.c_double]),
        "iga_get_time": (ctypes.c_int, [H, dp]),
        "iga_autotune": (ctypes.c_int, [H, ctypes.c_int, ctypes.c_int, ip, ip]),
        "iga_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(H), ctypes.POINTER(H)]),
        "iga_batch_destroy": (None, [H]),
        "iga_batch_last_error": (ctypes.c_char_p, [H]),
        "iga_batch_step": (ctypes.c_int, [H, ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double, dp, ctypes.c_int,
                                          ctypes.POINTER(Stats)]),
        "iga_batch_set_persistent": (ctypes.c_int, [H, ctypes.c_int]),
        "iga_batch_phase_times": (ctypes.c_int, [H, dp, ctypes.c_int]),
        "iga_batch_set_persistent_variant": (ctypes.c_int, [H, ctypes.c_int]),
        "iga_batch_persistent_variant": (ctypes.c_int, [H, ip, dp]),
        "iga_mp_layout": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ip, ip, ctypes.POINTER(dp), ctypes.POINTER(dp),
                                         ctypes.c_double, ip, ip, ctypes.POINTER(ctypes.c_longlong), ip,
                                         ctypes.POINTER(ctypes.c_longlong), ctypes.c_longlong]),
        "iga_mp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ip, ip, ctypes.POINTER(dp), ctypes.POINTER(dp),
                                         ctypes.c_double, ctypes.POINTER(Options), ctypes.POINTER(H)]),
        "iga_mp_info": (ctypes.c_int, [H, ip, ip, ctypes.POINTER(ctypes.c_longlong)]),
        "iga_mp_patch": (ctypes.c_int, [H, ctypes.c_int, ctypes.POINTER(H)]),
        "iga_mp_set_concurrent": (ctypes.c_int, [H, ctypes.c_int]),
        "iga_mp_patch_io": (ctypes.c_int, [H, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]),
        "iga_npoints": (ctypes.c_int, [H, ctypes.POINTER(ctypes.c_longlong), ip]),
        "iga_gauss_points": (ctypes.c_int, [H, vp, vp]),
        "iga_evaluate": (ctypes.c_int, [H, ctypes.c_int, vp, vp]),
        "iga_integrate": (ctypes.c_int, [H, ctypes.c_int, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def exported_symbols():
    """Names of the entry points this binding expects the library to export."""
    return ["iga_options_default", "iga_status_string", "iga_last_error", "iga_create", "iga_destroy",
            "iga_ndof", "iga_assemble", "iga_set_op_form", "iga_set_precond", "iga_set_guess", "iga_set_tol",
            "iga_apply_M", "iga_apply_K", "iga_apply_Pinv", "iga_solve_M", "iga_galpha_params", "iga_cfl",
            "iga_state_init", "iga_step", "iga_step_host", "iga_profile", "iga_profile_read",
            "iga_apply_Pinv_noalloc", "iga_probe_fp64_fma", "iga_set_graphs", "iga_ws_collect",
            "iga_ws_samples", "iga_ws_train", "iga_ws_init_params", "iga_ws_get_params", "iga_ws_set_params",
            "iga_ws_features", "iga_net_forward", "iga_net_workspace_bytes", "iga_net_backward", "iga_net_adam",
            "iga_set_band_config", "iga_band_df_tiny", "iga_autotune", "iga_batch_create", "iga_batch_destroy", "iga_batch_last_error",
            "iga_batch_step", "iga_set_damping", "iga_set_forcing", "iga_set_time", "iga_get_time",
            "iga_mp_layout", "iga_mp_create", "iga_mp_info", "iga_mp_patch", "iga_mp_patch_io", "iga_mp_set_concurrent", "iga_npoints", "iga_gauss_points", "iga_evaluate",
            "iga_integrate", "iga_set_barrier_limit", "iga_batch_set_persistent", "iga_batch_phase_times",
            "iga_batch_set_persistent_variant", "iga_batch_persistent_variant"]


def multipatch_layout(patches, tol=0.0):
    """Gluing of conforming patches (iga_mp_layout, host only; Sec. 5.1, def:mp_basis).
    patches: list of (degrees, knots, ctrl) as for Patch. Returns a dict with "lo", "hi"
    ((npatch, dim) index boxes, inclusive), "nglob", "n_adj" and "gid": per patch an integer
    array shaped like its box (last direction first), the global id of each function or -1."""
    import numpy as np
    L = lib()
    npatch = len(patches)
    dim = len(patches[0][0])
    deg = (ctypes.c_int * (npatch * dim))(*[int(p) for pt in patches for p in pt[0]])
    nk = (ctypes.c_int * (npatch * dim))(*[len(kn) for pt in patches for kn in pt[1]])
    kn_arrays = [np.ascontiguousarray(kn, dtype=np.float64) for pt in patches for kn in pt[1]]
    ct_arrays = [np.ascontiguousarray(pt[2], dtype=np.float64).reshape(-1) for pt in patches]
    dp = ctypes.POINTER(ctypes.c_double)
    kn_ptr = (dp * len(kn_arrays))(*[a.ctypes.data_as(dp) for a in kn_arrays])
    ct_ptr = (dp * npatch)(*[a.ctypes.data_as(dp) for a in ct_arrays])
    lo = (ctypes.c_int * (npatch * dim))()
    hi = (ctypes.c_int * (npatch * dim))()
    nglob = ctypes.c_longlong()
    nadj = ctypes.c_int()
    rc = L.iga_mp_layout(npatch, dim, deg, nk, kn_ptr, ct_ptr, tol, lo, hi, ctypes.byref(nglob), ctypes.byref(nadj),
                         None, 0)
    if rc != OK:
        raise IgaError(rc, "iga_mp_layout: " + L.iga_last_error(None).decode())
    lo_a = np.array(lo[:], dtype=int).reshape(npatch, dim)
    hi_a = np.array(hi[:], dtype=int).reshape(npatch, dim)
    sizes = [int(np.prod(hi_a[r] - lo_a[r] + 1)) for r in range(npatch)]
    gid = np.zeros(sum(sizes), dtype=np.int64)
    rc = L.iga_mp_layout(npatch, dim, deg, nk, kn_ptr, ct_ptr, tol, lo, hi, ctypes.byref(nglob), ctypes.byref(nadj),
                         gid.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), gid.size)
    if rc != OK:
        raise IgaError(rc, "iga_mp_layout: " + L.iga_last_error(None).decode())
    out, w = [], 0
    for r in range(npatch):
        out.append(gid[w:w + sizes[r]].reshape(list(reversed((hi_a[r] - lo_a[r] + 1).tolist()))))
        w += sizes[r]
    return {"lo": lo_a, "hi": hi_a, "nglob": int(nglob.value), "n_adj": int(nadj.value), "gid": out}


def fp64_fma_probe(device=0):
    """(TFLOP/s, nominal max SM clock GHz) of the FP64 FMA-chain probe on `device`."""
    tf = ctypes.c_double()
    ghz = ctypes.c_double()
    rc = lib().iga_probe_fp64_fma(device, ctypes.byref(tf), ctypes.byref(ghz))
    if rc != OK:
        raise IgaError(rc, "iga_probe_fp64_fma")
    return tf.value, ghz.value


PROFILE_CLASSES = {"off": 0, "mass": 1, "stiff": 2, "precond": 3, "mass_apply": 4, "band_mass": 5, "band_stiff": 6}


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):  # numpy array (host memory)
        return t.ctypes.data
    raise TypeError("expected a tensor, a numpy array or an integer address")


def _check_dev(t, n, name):
    if isinstance(t, int):
        return
    if getattr(t, "is_cuda", False) is not True:
        raise ValueError("%s must be a CUDA tensor" % name)
    import torch
    if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() < n:
        raise ValueError("%s must be a contiguous float64 tensor with at least %d elements" % (name, n))


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def _check_dev_typed(t, n, name, dtype):
    if isinstance(t, int):
        return
    import torch
    if getattr(t, "is_cuda", False) is not True or t.dtype != dtype or not t.is_contiguous() or t.numel() < n:
        raise ValueError("%s must be a contiguous CUDA %s tensor with at least %d elements" % (name, dtype, n))


def net_forward(shape, x, theta, act, y, nb=1, stream=None):
    """Warm-start network forward on an (n1, n2, n3) grid: x [nb][3][N] bfloat16,
    theta float32 [NET_NPARAM] -> act [nb][16][N] bfloat16, y [nb][N] float32."""
    import torch
    n1, n2, n3 = shape
    N = n1 * n2 * n3
    _check_dev_typed(x, nb * 3 * N, "x", torch.bfloat16)
    _check_dev_typed(theta, NET_NPARAM, "theta", torch.float32)
    _check_dev_typed(act, nb * 16 * N, "act", torch.bfloat16)
    _check_dev_typed(y, nb * N, "y", torch.float32)
    rc = lib().iga_net_forward(n1, n2, n3, nb, _ptr(x), _ptr(theta), _ptr(act), _ptr(y),
                               stream if stream is not None else _default_stream())
    if rc != OK:
        raise IgaError(rc, "iga_net_forward")


def net_workspace_bytes(shape, nb=1):
    n1, n2, n3 = shape
    return int(lib().iga_net_workspace_bytes(n1, n2, n3, nb))


def net_backward(shape, x, theta, act, dy, grad, work, nb=1, stream=None):
    """Gradient of sum(dy * y) with respect to theta (grad float32 [NET_NPARAM]);
    work: a uint8 CUDA tensor of at least net_workspace_bytes(shape, nb) bytes."""
    import torch
    n1, n2, n3 = shape
    N = n1 * n2 * n3
    _check_dev_typed(x, nb * 3 * N, "x", torch.bfloat16)
    _check_dev_typed(theta, NET_NPARAM, "theta", torch.float32)
    _check_dev_typed(act, nb * 16 * N, "act", torch.bfloat16)
    _check_dev_typed(dy, nb * N, "dy", torch.float32)
    _check_dev_typed(grad, NET_NPARAM, "grad", torch.float32)
    rc = lib().iga_net_backward(n1, n2, n3, nb, _ptr(x), _ptr(theta), _ptr(act), _ptr(dy), _ptr(grad), _ptr(work),
                                work.numel() * work.element_size(),
                                stream if stream is not None else _default_stream())
    if rc != OK:
        raise IgaError(rc, "iga_net_backward")


def net_adam(theta, grad, m, v, step, lr, stream=None):
    """One Adam update of float32 CUDA tensors theta, m, v from grad (step counts from 1)."""
    import torch
    n = theta.numel()
    for t, name in ((theta, "theta"), (grad, "grad"), (m, "m"), (v, "v")):
        _check_dev_typed(t, n, name, torch.float32)
    rc = lib().iga_net_adam(n, _ptr(theta), _ptr(grad), _ptr(m), _ptr(v), step, lr,
                            stream if stream is not None else _default_stream())
    if rc != OK:
        raise IgaError(rc, "iga_net_adam")


def galpha_params(k: int, rho: float):
    """(alpha, beta, gamma) lists of the method for order 2k (Sec. 4.1)."""
    a = (ctypes.c_double * k)()
    b = (ctypes.c_double * k)()
    g = (ctypes.c_double * k)()
    rc = lib().iga_galpha_params(k, rho, a, b, g)
    if rc != OK:
        raise IgaError(rc, "iga_galpha_params")
    return list(a), list(b), list(g)


class Patch:
    """One B-spline patch on the GPU (iga_create / iga_destroy)."""

    def __init__(self, degrees, knots, ctrl, nquad=0, tol=1e-10, max_iter=500, precond="fp64",
                 op_form="matrix_free", guess="zero", device=0, stream="current"):
        import numpy as np
        L = lib()
        self.d = len(degrees)
        opt = Options()
        L.iga_options_default(ctypes.byref(opt))
        opt.nquad, opt.tol, opt.max_iter = nquad, tol, max_iter
        opt.precond, opt.op_form, opt.guess = PRECONDS[precond], OP_FORMS[op_form], GUESSES[guess]
        opt.device = device
        opt.stream = _default_stream() if stream == "current" else stream
        deg = (ctypes.c_int * self.d)(*[int(p) for p in degrees])
        self._knots = [np.ascontiguousarray(k, dtype=np.float64) for k in knots]
        nk = (ctypes.c_int * self.d)(*[len(k) for k in self._knots])
        kp = (ctypes.POINTER(ctypes.c_double) * self.d)(
            *[k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for k in self._knots])
        c = np.ascontiguousarray(ctrl, dtype=np.float64)
        h = ctypes.c_void_p()
        rc = L.iga_create(self.d, deg, nk, kp, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          ctypes.byref(opt), ctypes.byref(h))
        if rc != OK:
            raise IgaError(rc, "iga_create: " + L.iga_last_error(None).decode())
        self.h = h
        n = ctypes.c_longlong()
        L.iga_ndof(h, ctypes.byref(n))
        self.N = int(n.value)
        # interior control points per direction (n1, n2, n3), i1 fastest
        self.shape = tuple([len(k) - int(p) - 3 for k, p in zip(self._knots, degrees)] + [1] * (3 - self.d))

    def _chk(self, rc, what):
        if rc != OK:
            raise IgaError(rc, "%s: %s" % (what, lib().iga_last_error(self.h).decode()))

    def close(self):
        if getattr(self, "_borrowed", False):  # a multi-patch system's patch: the system owns it
            self.h = None
            return
        if getattr(self, "h", None):
            lib().iga_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def assemble(self):
        self._chk(lib().iga_assemble(self.h), "iga_assemble")

    def set_op_form(self, form):
        self._chk(lib().iga_set_op_form(self.h, OP_FORMS[form]), "iga_set_op_form")

    def set_precond(self, prec):
        self._chk(lib().iga_set_precond(self.h, PRECONDS[prec]), "iga_set_precond")

    def set_guess(self, guess):
        self._chk(lib().iga_set_guess(self.h, GUESSES[guess]), "iga_set_guess")

    def set_graphs(self, on):
        """Replay one captured CUDA graph per step (device-side PCG loop) or use the host loop."""
        self._chk(lib().iga_set_graphs(self.h, 1 if on else 0), "iga_set_graphs")

    def set_tol(self, tol, max_iter=500):
        self._chk(lib().iga_set_tol(self.h, tol, max_iter), "iga_set_tol")

    def set_barrier_limit(self, polls):
        """Polls of the double-FP32 split's grid barrier before its wait gives up (< 0: default)."""
        self._chk(lib().iga_set_barrier_limit(self.h, int(polls)), "iga_set_barrier_limit")

    def apply_M(self, x, y, nvec=1):
        _check_dev(x, nvec * self.N, "x"); _check_dev(y, nvec * self.N, "y")
        self._chk(lib().iga_apply_M(self.h, nvec, _ptr(x), _ptr(y)), "iga_apply_M")

    def apply_K(self, x, y, nvec=1):
        _check_dev(x, nvec * self.N, "x"); _check_dev(y, nvec * self.N, "y")
        self._chk(lib().iga_apply_K(self.h, nvec, _ptr(x), _ptr(y)), "iga_apply_K")

    def apply_Pinv(self, x, y, nvec=1):
        _check_dev(x, nvec * self.N, "x"); _check_dev(y, nvec * self.N, "y")
        self._chk(lib().iga_apply_Pinv(self.h, nvec, _ptr(x), _ptr(y)), "iga_apply_Pinv")

    def apply_Pinv_noalloc(self, x, y, nvec=1):
        """iga_apply_Pinv_noalloc: the preconditioner with the library's fixed scratch
        (no device allocation at call time; nvec * N <= 1048576)."""
        _check_dev(x, nvec * self.N, "x"); _check_dev(y, nvec * self.N, "y")
        self._chk(lib().iga_apply_Pinv_noalloc(self.h, nvec, _ptr(x), _ptr(y)), "iga_apply_Pinv_noalloc")

    def solve_M(self, b, x, nvec=1, use_x0=False):
        _check_dev(b, nvec * self.N, "b"); _check_dev(x, nvec * self.N, "x")
        its = (ctypes.c_int * nvec)()
        rel = (ctypes.c_double * nvec)()
        self._chk(lib().iga_solve_M(self.h, nvec, _ptr(b), _ptr(x), int(use_x0), its, rel), "iga_solve_M")
        return list(its), list(rel)

    def npoints(self):
        """(Qt, [Q_a]): the Gauss points of the handle's quadrature."""
        qt = ctypes.c_longlong()
        q = (ctypes.c_int * 3)()
        self._chk(lib().iga_npoints(self.h, ctypes.byref(qt), q), "iga_npoints")
        return int(qt.value), list(q)[:self.d]

    def gauss_points(self, x=None, w=None):
        """Physical Gauss points x ([d][Qt]) and weights w |det DF| ([Qt]) into device tensors."""
        qt, _ = self.npoints()
        if x is not None:
            _check_dev(x, self.d * qt, "x")
        if w is not None:
            _check_dev(w, qt, "w")
        self._chk(lib().iga_gauss_points(self.h, _ptr(x) if x is not None else None,
                                         _ptr(w) if w is not None else None), "iga_gauss_points")

    def evaluate(self, U, g, nvec=1):
        """g = sum_i U_i B_i at the Gauss points ([nvec][N] -> [nvec][Qt], device)."""
        qt, _ = self.npoints()
        _check_dev(U, nvec * self.N, "U"); _check_dev(g, nvec * qt, "g")
        self._chk(lib().iga_evaluate(self.h, nvec, _ptr(U), _ptr(g)), "iga_evaluate")

    def integrate(self, g, b, nvec=1):
        """b_i = int g B_i by the handle's quadrature ([nvec][Qt] -> [nvec][N], device)."""
        qt, _ = self.npoints()
        _check_dev(g, nvec * qt, "g"); _check_dev(b, nvec * self.N, "b")
        self._chk(lib().iga_integrate(self.h, nvec, _ptr(g), _ptr(b)), "iga_integrate")

    def cfl(self, rho, iters=100):
        lam = ctypes.c_double()
        tc = ctypes.c_double()
        self._chk(lib().iga_cfl(self.h, rho, iters, ctypes.byref(lam), ctypes.byref(tc)), "iga_cfl")
        return lam.value, tc.value

    def state_init(self, k, U0, V0, state):
        _check_dev(U0, self.N, "U0"); _check_dev(V0, self.N, "V0"); _check_dev(state, 3 * k * self.N, "state")
        self._chk(lib().iga_state_init(self.h, k, _ptr(U0), _ptr(V0), _ptr(state)), "iga_state_init")

    def step(self, state, k, rho, dt, nsteps=1, stats=None):
        _check_dev(state, 3 * k * self.N, "state")
        st = stats if stats is not None else Stats()
        self._chk(lib().iga_step(self.h, _ptr(state), k, rho, dt, nsteps, ctypes.byref(st)), "iga_step")
        return st

    def profile(self, kernel_class):
        """Time every later launch of one kernel class ('mass', 'stiff', 'precond',
        'mass_apply' or 'off') with CUDA events on the handle's stream."""
        self._chk(lib().iga_profile(self.h, PROFILE_CLASSES[kernel_class]), "iga_profile")

    def profile_read(self):
        """(total_ms, launches, algorithmic_flops, algorithmic_bytes) since the last read."""
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        fl = ctypes.c_double()
        by = ctypes.c_double()
        self._chk(lib().iga_profile_read(self.h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl),
                                         ctypes.byref(by)), "iga_profile_read")
        return ms.value, n.value, fl.value, by.value

    # -- general model M U'' + C U' + K U = F ---------------------------------------
    def set_damping(self, aM, aK):
        """Rayleigh damping C = aM M + aK K."""
        self._chk(lib().iga_set_damping(self.h, aM, aK), "iga_set_damping")

    def set_forcing(self, G, omegas, phases):
        """F(t) = sum_m G[m] sin(omegas[m] t + phases[m]); G: device float64 tensor [nterm][N] (copied)."""
        n = len(omegas)
        if len(phases) != n:
            raise ValueError("one phase per frequency")
        if n:
            _check_dev(G, n * self.N, "G")
        om = (ctypes.c_double * max(n, 1))(*[float(v) for v in omegas])
        ph = (ctypes.c_double * max(n, 1))(*[float(v) for v in phases])
        self._chk(lib().iga_set_forcing(self.h, n, _ptr(G) if n else None, om, ph), "iga_set_forcing")

    def set_time(self, t):
        self._chk(lib().iga_set_time(self.h, t), "iga_set_time")

    def get_time(self):
        t = ctypes.c_double()
        self._chk(lib().iga_get_time(self.h, ctypes.byref(t)), "iga_get_time")
        return t.value

    # -- launch tuning ------------------------------------------------------------
    def set_band_config(self, threads=0, nv=0):
        """Band-product launch configuration (threads per block, vectors per thread; 0 = default)."""
        self._chk(lib().iga_set_band_config(self.h, threads, nv), "iga_set_band_config")

    def band_df_tiny(self):
        """(frac_m, frac_k): the share of an interior row's terms that the double-FP32
        products form as one FP32 multiply-add (iga_band_df_tiny)."""
        fm, fk = ctypes.c_double(), ctypes.c_double()
        self._chk(lib().iga_band_df_tiny(self.h, ctypes.byref(fm), ctypes.byref(fk)), "iga_band_df_tiny")
        return fm.value, fk.value

    def autotune(self, nvec=2, reps=5):
        """Time the band-product configurations on nvec vectors, keep the fastest; returns (threads, nv)."""
        t = ctypes.c_int()
        v = ctypes.c_int()
        self._chk(lib().iga_autotune(self.h, nvec, reps, ctypes.byref(t), ctypes.byref(v)), "iga_autotune")
        return t.value, v.value

    # -- learned warm start -------------------------------------------------------
    def ws_collect(self, capacity):
        """Record up to `capacity` (features, target) samples from later learned-guess steps."""
        self._chk(lib().iga_ws_collect(self.h, capacity), "iga_ws_collect")

    def ws_samples(self):
        n = ctypes.c_int()
        self._chk(lib().iga_ws_samples(self.h, ctypes.byref(n)), "iga_ws_samples")
        return n.value

    def ws_train(self, epochs, lr=1e-3, seed=0):
        """Adam over the recorded samples (cosine-decayed learning rate); returns the
        mean loss of every epoch."""
        out = (ctypes.c_double * epochs)()
        self._chk(lib().iga_ws_train(self.h, epochs, lr, seed, out), "iga_ws_train")
        return list(out)

    def ws_init_params(self, seed=0):
        self._chk(lib().iga_ws_init_params(self.h, seed), "iga_ws_init_params")

    def ws_get_params(self):
        import numpy as np
        out = np.empty(NET_NPARAM, dtype=np.float32)
        self._chk(lib().iga_ws_get_params(self.h, out.ctypes.data), "iga_ws_get_params")
        return out

    def ws_set_params(self, theta):
        import numpy as np
        th = np.ascontiguousarray(theta, dtype=np.float32)
        if th.size != NET_NPARAM:
            raise ValueError("expected %d parameters" % NET_NPARAM)
        self._chk(lib().iga_ws_set_params(self.h, th.ctypes.data), "iga_ws_set_params")

    def ws_features(self, k, b, b1, b2, z1, z2, x, E, scales):
        """Features of k solves (device tensors; b1, b2, z1, z2 are overwritten by the moved histories)."""
        import torch
        n = k * self.N
        for t, name in ((b, "b"), (b1, "b1"), (b2, "b2"), (z1, "z1"), (z2, "z2"), (E, "E")):
            _check_dev(t, n, name)
        _check_dev_typed(x, 3 * n, "x", torch.bfloat16)
        _check_dev(scales, 2 * k, "scales")
        self._chk(lib().iga_ws_features(self.h, k, _ptr(b), _ptr(b1), _ptr(b2), _ptr(z1), _ptr(z2), _ptr(x),
                                        _ptr(E), _ptr(scales)), "iga_ws_features")

    def step_host(self, state_host, k, rho, dt, nsteps=1, stats=None):
        """state_host: host buffer (numpy array or pinned CPU tensor) of 3k*N float64."""
        st = stats if stats is not None else Stats()
        self._chk(lib().iga_step_host(self.h, _ptr(state_host), k, rho, dt, nsteps, ctypes.byref(st)),
                  "iga_step_host")
        return st



class MultiPatch(Patch):
    """Conforming patches glued face to face as one system on the GPU (iga_mp_create; Sec. 5.1,
    5.4): vectors have length N in the global numbering of multipatch_layout, M and K are
    the sums of the patches' matrices, apply_Pinv is the additive Schwarz preconditioner
    (def:asp), and the step, solve and CFL calls of Patch work on it (host-driven loop).
    patches: list of (degrees, knots, ctrl) as for Patch; the options are shared."""

    def __init__(self, patches, tol_glue=0.0, nquad=0, tol=1e-10, max_iter=500, precond="fp64",
                 op_form="matrix_free", guess="zero", device=0, stream="current"):
        import numpy as np
        L = lib()
        npatch = len(patches)
        self.d = len(patches[0][0])
        opt = Options()
        L.iga_options_default(ctypes.byref(opt))
        opt.nquad, opt.tol, opt.max_iter = nquad, tol, max_iter
        opt.precond, opt.op_form, opt.guess = PRECONDS[precond], OP_FORMS[op_form], GUESSES[guess]
        opt.device = device
        opt.stream = _default_stream() if stream == "current" else stream
        dp = ctypes.POINTER(ctypes.c_double)
        deg = (ctypes.c_int * (npatch * self.d))(*[int(p) for pt in patches for p in pt[0]])
        self._knots = [np.ascontiguousarray(kn, dtype=np.float64) for pt in patches for kn in pt[1]]
        nk = (ctypes.c_int * (npatch * self.d))(*[len(kn) for kn in self._knots])
        kp = (dp * len(self._knots))(*[kn.ctypes.data_as(dp) for kn in self._knots])
        self._ctrl = [np.ascontiguousarray(pt[2], dtype=np.float64).reshape(-1) for pt in patches]
        cp = (dp * npatch)(*[c.ctypes.data_as(dp) for c in self._ctrl])
        h = ctypes.c_void_p()
        rc = L.iga_mp_create(npatch, self.d, deg, nk, kp, cp, tol_glue, ctypes.byref(opt), ctypes.byref(h))
        if rc != OK:
            raise IgaError(rc, "iga_mp_create: " + L.iga_last_error(None).decode())
        self.h = h
        n = ctypes.c_longlong()
        L.iga_ndof(h, ctypes.byref(n))
        self.N = int(n.value)
        self.shape = None  # no single grid
        npc, nadj, nloc = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        L.iga_mp_info(h, ctypes.byref(npc), ctypes.byref(nadj), ctypes.byref(nloc))
        self.npatch, self.n_adj, self.nloc = int(npc.value), int(nadj.value), int(nloc.value)

    def set_concurrent(self, on=True):
        """Run the patches of every operator on streams of their own (iga_mp_set_concurrent)."""
        self._chk(lib().iga_mp_set_concurrent(self.h, int(bool(on))), "iga_mp_set_concurrent")

    def patch(self, r):
        """Patch r's own handle (borrowed, a Patch over its box; valid while this system lives)."""
        ph = ctypes.c_void_p()
        self._chk(lib().iga_mp_patch(self.h, r, ctypes.byref(ph)), "iga_mp_patch")
        p = Patch.__new__(Patch)
        p.h, p.d, p.shape = ph, self.d, None
        n = ctypes.c_longlong()
        lib().iga_ndof(ph, ctypes.byref(n))
        p.N = int(n.value)
        p._borrowed = True
        return p

    def patch_gather(self, r, x, box, nvec=1):
        """box = R^(r) x (global [nvec][N] -> patch r's box [nvec][box size], device)."""
        self._chk(lib().iga_mp_patch_io(self.h, r, nvec, 0, _ptr(x), _ptr(box)), "iga_mp_patch_io")

    def patch_scatter_add(self, r, box, y, nvec=1):
        """y += R^(r)T box (patch r's box -> global, device)."""
        self._chk(lib().iga_mp_patch_io(self.h, r, nvec, 1, _ptr(box), _ptr(y)), "iga_mp_patch_io")

class Batch:
    """Independent patches advanced together, one CUDA graph launch per batch step
    (iga_batch_create / iga_batch_step). The Patch objects must outlive the batch."""

    def __init__(self, patches):
        self.patches = list(patches)
        arr = (ctypes.c_void_p * len(self.patches))(*[p.h.value for p in self.patches])
        b = ctypes.c_void_p()
        rc = lib().iga_batch_create(len(self.patches), arr, ctypes.byref(b))
        if rc != OK:
            raise IgaError(rc, "iga_batch_create")
        self.b = b

    def step(self, states, k, rho, dts, nsteps=1, stats=None):
        """states: device float64 tensors (3k*N_i each); dts: per-patch step sizes.
        Returns the per-patch Stats list (accumulated into `stats` if given)."""
        n = len(self.patches)
        if len(states) != n or len(dts) != n:
            raise ValueError("one state and one dt per patch")
        for st, p in zip(states, self.patches):
            _check_dev(st, 3 * k * p.N, "state")
        sp = (ctypes.c_void_p * n)(*[_ptr(t) for t in states])
        dt = (ctypes.c_double * n)(*[float(v) for v in dts])
        out = stats if stats is not None else [Stats() for _ in range(n)]
        arr = (Stats * n)(*out)
        rc = lib().iga_batch_step(self.b, sp, k, rho, dt, nsteps, arr)
        for i in range(n):
            ctypes.memmove(ctypes.addressof(out[i]), ctypes.addressof(arr[i]), ctypes.sizeof(Stats))
        res = out
        if rc != OK:
            raise IgaError(rc, "iga_batch_step: " + lib().iga_batch_last_error(self.b).decode())
        return res

    def set_persistent(self, on=True):
        """One persistent cooperative launch per batch step (iga_batch_set_persistent)."""
        rc = lib().iga_batch_set_persistent(self.b, int(bool(on)))
        if rc != OK:
            raise IgaError(rc, "iga_batch_set_persistent: " + lib().iga_batch_last_error(self.b).decode())

    PHASES = ("predictor", "K product", "PCG scalars", "preconditioner", "direction update", "M product",
              "x, r update", "stage update")

    def phase_times(self):
        """Milliseconds per phase kind of the last persistent step call (iga_batch_phase_times),
        as a dict keyed by Batch.PHASES."""
        ms = (ctypes.c_double * len(self.PHASES))()
        rc = lib().iga_batch_phase_times(self.b, ms, len(self.PHASES))
        if rc != OK:
            raise IgaError(rc, "iga_batch_phase_times: " + lib().iga_batch_last_error(self.b).decode())
        return dict(zip(self.PHASES, list(ms)))

    def set_persistent_variant(self, variant=-1):
        """Launch variant of the persistent step (iga_batch_set_persistent_variant): -1 chooses
        by timing the first steps, 0 or 1 forces one."""
        rc = lib().iga_batch_set_persistent_variant(self.b, int(variant))
        if rc != OK:
            raise IgaError(rc, "iga_batch_set_persistent_variant: " + lib().iga_batch_last_error(self.b).decode())

    def persistent_variant(self):
        """(variant in use or -1, (fastest timed ms of variant 0, of variant 1) or -1 each)."""
        v = ctypes.c_int(0)
        ms = (ctypes.c_double * 2)()
        rc = lib().iga_batch_persistent_variant(self.b, ctypes.byref(v), ms)
        if rc != OK:
            raise IgaError(rc, "iga_batch_persistent_variant: " + lib().iga_batch_last_error(self.b).decode())
        return v.value, (ms[0], ms[1])

    def close(self):
        if getattr(self, "b", None):
            lib().iga_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shard_patches(works, world):
    """Longest-processing-time partition of independent patches over `world` ranks:
    patches in decreasing order of estimated work go to the rank with the least work
    so far (ties to the lower rank). Returns one sorted index list per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(works)), key=lambda i: (-works[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += works[i]
    return [sorted(o) for o in out]


def patch_work(ndof, p):
    """Work estimate of one patch step: couplings of the assembled band, N (2p+1)^3."""
    return float(ndof) * (2 * p + 1) ** 3
