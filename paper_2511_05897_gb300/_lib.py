"""ctypes binding of libeaadc.so: the C entry points of include/eaadc.h under
the same names.  Argument marshalling only: every computation runs in the
CUDA library, and loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libeaadc.so")

EAADC_OK = 0
EAADC_ERR_ARG = -1
EAADC_ERR_ALLOC = -2
EAADC_ERR_CUDA = -3
EAADC_ERR_NOCONV = -4
EAADC_ERR_NONFINITE = -5
EAADC_ERR_TIMEOUT = -6
EAADC_ERR_STATE = -7
EAADC_FP64 = 0
EAADC_MIXED_BF16 = 1
EAADC_MIXED_BF16X3 = 2

EXPORTED = (
    "eaadc_version", "eaadc_init", "eaadc_build_canonical", "eaadc_state_info", "eaadc_sigma",
    "eaadc_sigma_host", "eaadc_diagonal", "eaadc_get_m11", "eaadc_davidson", "eaadc_get_eigvecs",
    "eaadc_destroy", "eaadc_last_error", "eaadc_ladder", "eaadc_kernel_launches",
    "eaadc_ladder_noalloc", "eaadc_build_states", "eaadc_ea_energies", "eaadc_eigh_sym", "eaadc_num_states",
    "eaadc_precond_load", "eaadc_precond_get", "eaadc_precond_pairs", "eaadc_mlp_forward", "eaadc_mlp_loss_grad",
    "eaadc_mlp_train_step", "eaadc_get_trace", "eaadc_set_build_precision",
)
MLP_FEATURES = 16
MLP_PARAMS = 136193


class EaadcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"eaadc status {status}: {msg}")
        self.status = status


class DavidsonOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("etol", C.c_double), ("maxit", C.c_int), ("max_sub", C.c_int),
                ("prec", C.c_int), ("refine", C.c_int), ("precond", C.c_int), ("trace", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.eaadc_version.restype = C.c_char_p
        L.eaadc_kernel_launches.restype = C.c_longlong
        L.eaadc_init.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, dp, dp, dp, C.c_int, vp]
        L.eaadc_build_canonical.argtypes = [vp, C.c_int, C.c_double]
        L.eaadc_state_info.argtypes = [vp, C.c_int, ip, ip, C.POINTER(C.c_longlong)]
        L.eaadc_sigma.argtypes = [vp, C.c_int, C.c_int, vp, vp, C.c_int, vp]
        L.eaadc_sigma_host.argtypes = [vp, C.c_int, C.c_int, dp, dp, C.c_int]
        L.eaadc_diagonal.argtypes = [vp, C.c_int, dp]
        L.eaadc_ladder.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp]
        L.eaadc_ladder_noalloc.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp]
        L.eaadc_build_states.argtypes = [vp, C.c_int, dp, dp, C.c_int, C.c_double, C.POINTER(DavidsonOpts)]
        L.eaadc_ea_energies.argtypes = [vp, C.POINTER(DavidsonOpts), dp, dp, dp, dp]
        L.eaadc_eigh_sym.argtypes = [C.c_int, vp, vp, vp, C.c_int, vp]
        L.eaadc_num_states.argtypes = [vp]
        fp = C.POINTER(C.c_float)
        L.eaadc_precond_load.argtypes = [vp, fp, C.c_size_t]
        L.eaadc_precond_get.argtypes = [vp, fp, C.c_size_t]
        L.eaadc_precond_pairs.argtypes = [vp, C.c_int, C.c_int, vp, vp, dp, vp, vp, vp, vp, vp, vp]
        L.eaadc_mlp_forward.argtypes = [vp, C.c_longlong, vp, vp, vp]
        L.eaadc_mlp_loss_grad.argtypes = [vp, C.c_int, ip, vp, vp, vp, vp, dp, fp, vp]
        L.eaadc_mlp_train_step.argtypes = [vp, C.c_int, ip, vp, vp, vp, vp, C.c_float, dp, vp]
        L.eaadc_get_trace.argtypes = [vp, C.c_int, ip, ip, dp, dp, dp]
        L.eaadc_set_build_precision.argtypes = [vp, C.c_int]
        L.eaadc_num_states.restype = C.c_int
        L.eaadc_get_m11.argtypes = [vp, C.c_int, dp]
        L.eaadc_davidson.argtypes = [vp, C.c_int, C.POINTER(DavidsonOpts), dp, dp, ip]
        L.eaadc_get_eigvecs.argtypes = [vp, C.c_int, dp]
        L.eaadc_destroy.argtypes = [vp]
        L.eaadc_destroy.restype = None
        L.eaadc_last_error.argtypes = [vp]
        L.eaadc_last_error.restype = C.c_char_p
        for name in EXPORTED:
            if name not in ("eaadc_version", "eaadc_destroy", "eaadc_last_error", "eaadc_kernel_launches",
                            "eaadc_num_states"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(ctx, st):
    if st != EAADC_OK:
        raise EaadcError(st, lib().eaadc_last_error(ctx).decode())


def eaadc_version():
    return lib().eaadc_version().decode()


def eaadc_kernel_launches():
    return int(lib().eaadc_kernel_launches())


def eaadc_last_error(ctx):
    return lib().eaadc_last_error(ctx).decode()


def eaadc_init(o, v, naux, eps_occ, eps_vir, B, device=0, stream=None):
    eo, ev, Bf = _f64(eps_occ), _f64(eps_vir), _f64(B)
    if eo.size != o or ev.size != v or Bf.size != naux * (o + v) ** 2:
        raise ValueError("array sizes do not match (o, v, naux)")
    ctx = C.c_void_p()
    st = lib().eaadc_init(C.byref(ctx), o, v, naux, _dp(eo), _dp(ev), _dp(Bf), device, stream)
    _check(None, st)
    return ctx


def eaadc_build_canonical(ctx, adc_order=3, x3=1.0):
    _check(ctx, lib().eaadc_build_canonical(ctx, adc_order, x3))


def eaadc_state_info(ctx, state=0):
    vp, npx, dim = C.c_int(), C.c_int(), C.c_longlong()
    _check(ctx, lib().eaadc_state_info(ctx, state, C.byref(vp), C.byref(npx), C.byref(dim)))
    return vp.value, npx.value, dim.value


def eaadc_sigma(ctx, state, nvec, x_ptr, sigma_ptr, prec=EAADC_FP64, stream=None):
    """Device pointers (ints, e.g. torch.Tensor.data_ptr()) of [nvec][dim] float64 buffers."""
    _check(ctx, lib().eaadc_sigma(ctx, state, nvec, C.c_void_p(x_ptr), C.c_void_p(sigma_ptr), prec, stream))


def eaadc_sigma_host(ctx, state, x, prec=EAADC_FP64, out=None):
    """Host arrays; out (optional, e.g. pinned memory) receives sigma."""
    x = _f64(x)
    nvec = 1 if x.ndim == 1 else x.shape[0]
    y = np.empty_like(x) if out is None else out
    if y.shape != x.shape or y.dtype != np.float64 or not y.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous float64 array shaped like x")
    _check(ctx, lib().eaadc_sigma_host(ctx, state, nvec, _dp(x), _dp(y), prec))
    return y


def eaadc_ladder(ctx, state, nvec, x_ptr, out_ptr, stream=None):
    """Device pointers: x [nvec][dim] float64, out [nvec][o][v][v] float32."""
    _check(ctx, lib().eaadc_ladder(ctx, state, nvec, C.c_void_p(x_ptr), C.c_void_p(out_ptr), stream))


def eaadc_ladder_noalloc(ctx, state, nvec, x_ptr, out_ptr, stream=None):
    """As eaadc_ladder, working in the library's fixed device array instead of
    allocating (for callers that cannot allocate device memory mid-run)."""
    _check(ctx, lib().eaadc_ladder_noalloc(ctx, state, nvec, C.c_void_p(x_ptr), C.c_void_p(out_ptr), stream))


def eaadc_set_build_precision(ctx, prec):
    """Precision of the amplitude ladder in the next state builds (EAADC_FP64 default)."""
    _check(ctx, lib().eaadc_set_build_precision(ctx, prec))


def eaadc_build_states(ctx, nstates, fno_thresh, naf_thresh, adc_order=3, x3=1.0, can_opts=None):
    """Per-state FNO/NAF truncated spaces from the nstates lowest canonical
    EA-ADC(2) roots; thresholds are scalars or per-state sequences (< 0 keeps all).
    can_opts: dict of Davidson options for the canonical ADC(2) solve, or None."""
    f = np.ascontiguousarray(np.broadcast_to(np.asarray(fno_thresh, dtype=np.float64), (nstates,)))
    n = np.ascontiguousarray(np.broadcast_to(np.asarray(naf_thresh, dtype=np.float64), (nstates,)))
    o = C.byref(DavidsonOpts(**_opts(can_opts))) if can_opts is not None else None
    _check(ctx, lib().eaadc_build_states(ctx, nstates, _dp(f), _dp(n), adc_order, x3, o))


def eaadc_ea_energies(ctx, opts=None):
    """Eq. 30 per state: dict of omega_uncorr, omega_corr, omega2_can, omega2_fno (hartree)."""
    nstates = max(eaadc_num_states(ctx), 1)
    out = {k: np.zeros(nstates) for k in ("omega_uncorr", "omega_corr", "omega2_can", "omega2_fno")}
    o = C.byref(DavidsonOpts(**_opts(opts))) if opts is not None else None
    _check(ctx, lib().eaadc_ea_energies(ctx, o, _dp(out["omega_uncorr"]), _dp(out["omega_corr"]),
                                        _dp(out["omega2_can"]), _dp(out["omega2_fno"])))
    return out


def eaadc_eigh_sym(n, a_ptr, w_ptr, v_ptr, device=0, stream=None):
    """Device pointers: a [n][n] float64 (read), w [n], v [n][n] (eigenvectors as columns)."""
    _check(None, lib().eaadc_eigh_sym(n, C.c_void_p(a_ptr), C.c_void_p(w_ptr), C.c_void_p(v_ptr), device, stream))


def _opts(d):
    base = dict(tol=1e-8, etol=1e-10, maxit=300, max_sub=40, prec=EAADC_FP64, refine=0, precond=0, trace=0)
    base.update(d)
    return base


def eaadc_diagonal(ctx, state=0):
    dim = eaadc_state_info(ctx, state)[2]
    out = np.empty(dim)
    _check(ctx, lib().eaadc_diagonal(ctx, state, _dp(out)))
    return out


def eaadc_get_m11(ctx, state=0):
    v = eaadc_state_info(ctx, state)[0]
    out = np.empty((v, v))
    _check(ctx, lib().eaadc_get_m11(ctx, state, _dp(out)))
    return out


def eaadc_num_states(ctx):
    return lib().eaadc_num_states(ctx)


def eaadc_davidson(ctx, nroots, tol=1e-6, etol=1e-10, maxit=200, max_sub=40, prec=EAADC_FP64, refine=1,
                   precond=0, trace=0):
    """Returns (omega[nstates, nroots], resnorm[nstates, nroots], iters[nstates], status)."""
    nstates = eaadc_num_states(ctx)
    opts = DavidsonOpts(tol, etol, maxit, max_sub, prec, refine, precond, trace)
    om = np.zeros((max(nstates, 1), nroots))
    rn = np.zeros((max(nstates, 1), nroots))
    it = np.zeros(max(nstates, 1), dtype=np.int32)
    st = lib().eaadc_davidson(ctx, nroots, C.byref(opts), _dp(om), _dp(rn),
                              it.ctypes.data_as(C.POINTER(C.c_int)))
    if st not in (EAADC_OK, EAADC_ERR_NOCONV):
        _check(ctx, st)
    return om, rn, it, st


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def eaadc_precond_load(ctx, weights):
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(ctx, lib().eaadc_precond_load(ctx, _fp(w), w.nbytes))


def eaadc_precond_get(ctx):
    w = np.empty(MLP_PARAMS, dtype=np.float32)
    _check(ctx, lib().eaadc_precond_get(ctx, _fp(w), w.nbytes))
    return w


def eaadc_precond_pairs(ctx, state, nvec, y_ptr, r_ptr, theta, ystar_ptr, feat_ptr, rr_ptr, base_ptr, target_ptr,
                        stream=None):
    """Device pointers (see include/eaadc.h); theta: host sequence of nvec Ritz values."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    vp_ = lambda p: C.c_void_p(p) if p else None  # noqa: E731
    _check(ctx, lib().eaadc_precond_pairs(ctx, state, nvec, vp_(y_ptr), vp_(r_ptr), _dp(th), vp_(ystar_ptr),
                                          vp_(feat_ptr), vp_(rr_ptr), vp_(base_ptr), vp_(target_ptr), stream))


def eaadc_mlp_forward(ctx, n, feat_ptr, m_ptr, stream=None):
    _check(ctx, lib().eaadc_mlp_forward(ctx, n, C.c_void_p(feat_ptr), C.c_void_p(m_ptr), stream))


def eaadc_mlp_loss_grad(ctx, segs, feat_ptr, rr_ptr, base_ptr, target_ptr, stream=None):
    sg = np.ascontiguousarray(segs, dtype=np.int32)
    L = np.zeros(1)
    g = np.empty(MLP_PARAMS, dtype=np.float32)
    _check(ctx, lib().eaadc_mlp_loss_grad(ctx, sg.size - 1, _ip(sg), C.c_void_p(feat_ptr), C.c_void_p(rr_ptr),
                                          C.c_void_p(base_ptr), C.c_void_p(target_ptr), _dp(L), _fp(g), stream))
    return float(L[0]), g


def eaadc_mlp_train_step(ctx, segs, feat_ptr, rr_ptr, base_ptr, target_ptr, lr, stream=None):
    sg = np.ascontiguousarray(segs, dtype=np.int32)
    L = np.zeros(1)
    _check(ctx, lib().eaadc_mlp_train_step(ctx, sg.size - 1, _ip(sg), C.c_void_p(feat_ptr), C.c_void_p(rr_ptr),
                                           C.c_void_p(base_ptr), C.c_void_p(target_ptr), C.c_float(lr), _dp(L),
                                           stream))
    return float(L[0])


def eaadc_get_trace(ctx, state=0):
    """(X [niters, nroots, dim], R [niters, nroots, dim], theta [niters, nroots]) of the last traced Davidson."""
    ni, nr = C.c_int(), C.c_int()
    _check(ctx, lib().eaadc_get_trace(ctx, state, C.byref(ni), C.byref(nr), None, None, None))
    dim = eaadc_state_info(ctx, state)[2]
    X = np.empty((ni.value, nr.value, dim))
    R = np.empty_like(X)
    th = np.empty((ni.value, nr.value))
    if ni.value * nr.value:
        _check(ctx, lib().eaadc_get_trace(ctx, state, C.byref(ni), C.byref(nr), _dp(X), _dp(R), _dp(th)))
    return X, R, th


def eaadc_get_eigvecs(ctx, state, nroots):
    dim = eaadc_state_info(ctx, state)[2]
    out = np.empty((nroots, dim))
    _check(ctx, lib().eaadc_get_eigvecs(ctx, state, _dp(out)))
    return out


def eaadc_destroy(ctx):
    lib().eaadc_destroy(ctx)
