"""ctypes marshalling for the FP64 oracle in ntf_oracle.c (test infrastructure only).

Arrays are numpy float64 (factors, core, tensors) and int32 (COO coordinates), C-order.
Functions that update blocks in place return new arrays instead and leave inputs alone.
"""
import ctypes as C

import numpy as np

from . import build as _build

_lib = None

_D = C.c_double
_P = C.c_void_p
_I64 = C.c_int64


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        sig = {
            "ntfo_gamma": (_D, [_D]),
            "ntfo_dbeta": (_D, [_D, _D, _D]),
            "ntfo_mu_apply": (None, [_I64, _P, _P, _P, _D, _D, _P]),
            "ntfo_chi1": (None, [_I64, _P, _P, _D, _P]),
            "ntfo_chi2": (None, [_I64, _P, _P, _D, _P]),
            "ntfo_cp_full": (None, [C.c_int, _P, C.c_int, _P, _P]),
            "ntfo_cp_objective": (_D, [C.c_int, _P, _P, C.c_int, _P, _D, _D, _D]),
            "ntfo_cp_contr": (None, [C.c_int, _P, _P, C.c_int, _P, C.c_int, _P]),
            "ntfo_cp_block_update": (None, [C.c_int, _P, _P, C.c_int, _P, C.c_int, _D, _D, _D, _P, _P]),
            "ntfo_cp_mu_sweep": (None, [C.c_int, _P, _P, C.c_int, _P, _D, _D, _D, _P]),
            "ntfo_tucker_jcomm_outer_extrap": (None, [C.c_int, _P, _P, _P, _P, _P, _P, _P, _D, _D, _D, C.c_int, _D, _D, _D,
                                                      _P]),
            "ntfo_tucker_mu_sweep_extrap": (None, [C.c_int, _P, _P, _P, _P, _P, _P, _P, _D, _D, _D, _D, _D, _D, _P]),
            "ntfo_cp_mu_sweep_extrap": (None, [C.c_int, _P, _P, C.c_int, _P, _P, _D, _D, _D, _D, _D, _D, _P]),
            "ntfo_cp_jcomm_outer": (None, [C.c_int, _P, _P, C.c_int, _P, _D, _D, _D, C.c_int, C.c_int, _P]),
            "ntfo_cp_jcomm_outer_extrap": (None, [C.c_int, _P, _P, C.c_int, _P, _P, _D, _D, _D, C.c_int, _D, _D, _D, _P]),
            "ntfo_cp_numden_rows": (None, [C.c_int, _P, _P, C.c_int, _P, _P, _P, C.c_int, _D, _D, _D,
                                           C.c_int, _P, _P, _P]),
            "ntfo_tucker_full": (None, [C.c_int, _P, _P, _P, _P, _P]),
            "ntfo_tucker_objective": (_D, [C.c_int, _P, _P, _P, _P, _P, _D, _D, _D]),
            "ntfo_tucker_core_contr": (None, [C.c_int, _P, _P, _P, _P, _P]),
            "ntfo_tucker_partial": (None, [C.c_int, _P, _P, _P, _P, C.c_int, _P]),
            "ntfo_tucker_factor_contr": (None, [C.c_int, _P, _P, _P, _P, _P, C.c_int, _P]),
            "ntfo_tucker_mu_sweep": (None, [C.c_int, _P, _P, _P, _P, _P, _D, _D, _D, C.c_int, _P]),
            "ntfo_tucker_jcomm_outer": (None, [C.c_int, _P, _P, _P, _P, _P, _D, _D, _D, C.c_int, C.c_int, _P]),
            "ntfo_coo_kl_objective": (_D, [C.c_int, _P, _I64, _P, _P, C.c_int, _P, _D]),
            "ntfo_coo_kl_jcomm_outer": (None, [C.c_int, _P, _I64, _P, _P, C.c_int, _P, _D, C.c_int, _P]),
            "ntfo_coo_kl_mu_sweep": (None, [C.c_int, _P, _I64, _P, _P, C.c_int, _P, _D, _P]),
            "ntfo_stable_perm": (None, [_I64, _P, _I64, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _dims(shape):
    return np.ascontiguousarray(np.asarray(shape, dtype=np.int64))


class _PtrArray:
    """Host array of pointers to a list of float64 numpy arrays (kept alive)."""

    def __init__(self, arrays):
        self.arrays = arrays
        self.c = (C.c_void_p * len(arrays))(*[a.ctypes.data for a in arrays])


def gamma(beta):
    return _load().ntfo_gamma(float(beta))


def dbeta(x, y, beta):
    return _load().ntfo_dbeta(float(x), float(y), float(beta))


def mu_apply(pre, num, den, beta, eps):
    pre, num, den = _f64(pre), _f64(num), _f64(den)
    out = np.empty_like(pre)
    _load().ntfo_mu_apply(pre.size, _ptr(pre), _ptr(num), _ptr(den), float(beta), float(eps), _ptr(out))
    return out


def chi1(Z, Zt, beta):
    Z, Zt = _f64(Z), _f64(Zt)
    out = np.empty_like(Z)
    _load().ntfo_chi1(Z.size, _ptr(Z), _ptr(Zt), float(beta), _ptr(out))
    return out


def chi2(Z, Zt, beta):
    Z, Zt = _f64(Z), _f64(Zt)
    out = np.empty_like(Z)
    _load().ntfo_chi2(Z.size, _ptr(Z), _ptr(Zt), float(beta), _ptr(out))
    return out


# ----------------------------------------------------------------------------- CP

def cp_full(shape, factors):
    fs = [_f64(a) for a in factors]
    R = fs[0].shape[1]
    out = np.empty(tuple(shape), dtype=np.float64)
    pa = _PtrArray(fs)
    _load().ntfo_cp_full(len(fs), _ptr(_dims(shape)), R, pa.c, _ptr(out))
    return out


def cp_objective(X, factors, beta, eps=1e-12, eps_x=1e-12):
    X = _f64(X)
    fs = [_f64(a) for a in factors]
    pa = _PtrArray(fs)
    return _load().ntfo_cp_objective(X.ndim, _ptr(_dims(X.shape)), _ptr(X), fs[0].shape[1], pa.c,
                                     float(beta), float(eps), float(eps_x))


def cp_contr(T, mats, n):
    """CPContr^(n)(T; {B^(m)}); mats[n] is ignored (pass any array of the right rows)."""
    T = _f64(T)
    fs = [_f64(a) for a in mats]
    R = fs[(n + 1) % len(fs)].shape[1]
    fs = [a if a.shape[1] == R else np.zeros((a.shape[0], R)) for a in fs]
    out = np.empty((T.shape[n], R))
    pa = _PtrArray(fs)
    _load().ntfo_cp_contr(T.ndim, _ptr(_dims(T.shape)), _ptr(T), R, pa.c, n, _ptr(out))
    return out


def cp_block_update(X, factors, n, beta, eps=1e-12, eps_x=1e-12):
    """Returns (new_factors, Num^(n), Den^(n)) for one block of Algorithm 1."""
    X = _f64(X)
    fs = [_f64(a).copy() for a in factors]
    R = fs[0].shape[1]
    num = np.empty((X.shape[n], R))
    den = np.empty((X.shape[n], R))
    pa = _PtrArray(fs)
    _load().ntfo_cp_block_update(X.ndim, _ptr(_dims(X.shape)), _ptr(X), R, pa.c, n, float(beta),
                                 float(eps), float(eps_x), _ptr(num), _ptr(den))
    return fs, num, den


def cp_mu_sweep(X, factors, beta, eps=1e-12, eps_x=1e-12):
    """One B-CoMM sweep.  Returns (new_factors, objective of the incoming iterate)."""
    X = _f64(X)
    fs = [_f64(a).copy() for a in factors]
    f = np.zeros(1)
    pa = _PtrArray(fs)
    _load().ntfo_cp_mu_sweep(X.ndim, _ptr(_dims(X.shape)), _ptr(X), fs[0].shape[1], pa.c, float(beta),
                             float(eps), float(eps_x), _ptr(f))
    return fs, float(f[0])


def cp_mu_sweep_extrap(X, factors, factors_prev, beta, alpha, cap=np.inf, delta=1e-12, eps=1e-12, eps_x=1e-12):
    """One extrapolated B-CoMM sweep.  Returns (new_factors, new_prev, objective of the
    incoming iterate)."""
    X = _f64(X)
    fs = [_f64(a).copy() for a in factors]
    ps = [_f64(a).copy() for a in factors_prev]
    f = np.zeros(1)
    pa, pp = _PtrArray(fs), _PtrArray(ps)
    _load().ntfo_cp_mu_sweep_extrap(X.ndim, _ptr(_dims(X.shape)), _ptr(X), fs[0].shape[1], pa.c, pp.c, float(beta),
                                    float(eps), float(eps_x), float(alpha), float(cap), float(delta), _ptr(f))
    return fs, ps, float(f[0])


def cp_jcomm_outer(X, factors, beta, L=1, eps=1e-12, eps_x=1e-12, max_blocks=-1):
    """One J-CoMM outer iteration.  Returns (new_factors, objective at the reference)."""
    X = _f64(X)
    fs = [_f64(a).copy() for a in factors]
    f = np.zeros(1)
    pa = _PtrArray(fs)
    _load().ntfo_cp_jcomm_outer(X.ndim, _ptr(_dims(X.shape)), _ptr(X), fs[0].shape[1], pa.c, float(beta),
                                float(eps), float(eps_x), int(L), int(max_blocks), _ptr(f))
    return fs, float(f[0])


def cp_jcomm_outer_extrap(X, factors, factors_prev, beta, alpha, cap=np.inf, delta=1e-12, L=1, eps=1e-12,
                          eps_x=1e-12):
    """One J-CoMM outer iteration from the extrapolated reference.  Returns (new_factors,
    new_prev, objective of the incoming iterate)."""
    X = _f64(X)
    fs = [_f64(a).copy() for a in factors]
    ps = [_f64(a).copy() for a in factors_prev]
    f = np.zeros(1)
    pa, pp = _PtrArray(fs), _PtrArray(ps)
    _load().ntfo_cp_jcomm_outer_extrap(X.ndim, _ptr(_dims(X.shape)), _ptr(X), fs[0].shape[1], pa.c, pp.c, float(beta),
                                       float(eps), float(eps_x), int(L), float(alpha), float(cap), float(delta), _ptr(f))
    return fs, ps, float(f[0])


def cp_numden_rows(X, recon, num_f, den_f, n, rows, beta, eps=1e-12, eps_x=1e-12):
    """Num/Den rows i_n in `rows` of one mode-n block update, entry by entry."""
    X = _f64(X)
    ar = [_f64(a) for a in recon]
    bn = [_f64(a) for a in num_f]
    bd = [_f64(a) for a in den_f]
    R = ar[0].shape[1]
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    num = np.empty((len(rows), R))
    den = np.empty((len(rows), R))
    pr, pn, pd = _PtrArray(ar), _PtrArray(bn), _PtrArray(bd)
    _load().ntfo_cp_numden_rows(X.ndim, _ptr(_dims(X.shape)), _ptr(X), R, pr.c, pn.c, pd.c, n,
                                float(beta), float(eps), float(eps_x), len(rows), _ptr(rows),
                                _ptr(num), _ptr(den))
    return num, den


# ------------------------------------------------------------------------- Tucker

def tucker_full(shape, core, factors):
    G = _f64(core)
    fs = [_f64(a) for a in factors]
    out = np.empty(tuple(shape))
    pa = _PtrArray(fs)
    _load().ntfo_tucker_full(len(fs), _ptr(_dims(shape)), _ptr(_dims(G.shape)), _ptr(G), pa.c, _ptr(out))
    return out


def tucker_objective(X, core, factors, beta, eps=1e-12, eps_x=1e-12):
    X, G = _f64(X), _f64(core)
    fs = [_f64(a) for a in factors]
    pa = _PtrArray(fs)
    return _load().ntfo_tucker_objective(X.ndim, _ptr(_dims(X.shape)), _ptr(X), _ptr(_dims(G.shape)),
                                         _ptr(G), pa.c, float(beta), float(eps), float(eps_x))


def tucker_core_contr(T, mats, core_shape):
    T = _f64(T)
    fs = [_f64(a) for a in mats]
    out = np.empty(tuple(core_shape))
    pa = _PtrArray(fs)
    _load().ntfo_tucker_core_contr(T.ndim, _ptr(_dims(T.shape)), _ptr(T), _ptr(_dims(core_shape)), pa.c,
                                   _ptr(out))
    return out


def tucker_partial(shape, core, factors, n):
    G = _f64(core)
    fs = [_f64(a) for a in factors]
    rest = int(np.prod(shape)) // shape[n]
    out = np.empty((G.shape[n], rest))
    pa = _PtrArray(fs)
    _load().ntfo_tucker_partial(len(fs), _ptr(_dims(shape)), _ptr(_dims(G.shape)), _ptr(G), pa.c, n, _ptr(out))
    return out


def tucker_factor_contr(T, core, factors, n):
    T, G = _f64(T), _f64(core)
    fs = [_f64(a) for a in factors]
    out = np.empty((T.shape[n], G.shape[n]))
    pa = _PtrArray(fs)
    _load().ntfo_tucker_factor_contr(T.ndim, _ptr(_dims(T.shape)), _ptr(T), _ptr(_dims(G.shape)), _ptr(G),
                                     pa.c, n, _ptr(out))
    return out


def tucker_mu_sweep(X, core, factors, beta, eps=1e-12, eps_x=1e-12, max_blocks=-1):
    X = _f64(X)
    G = _f64(core).copy()
    fs = [_f64(a).copy() for a in factors]
    f = np.zeros(1)
    pa = _PtrArray(fs)
    _load().ntfo_tucker_mu_sweep(X.ndim, _ptr(_dims(X.shape)), _ptr(X), _ptr(_dims(G.shape)), _ptr(G), pa.c,
                                 float(beta), float(eps), float(eps_x), int(max_blocks), _ptr(f))
    return G, fs, float(f[0])


def tucker_mu_sweep_extrap(X, core, factors, core_prev, factors_prev, beta, alpha, cap=np.inf, delta=1e-12,
                           eps=1e-12, eps_x=1e-12):
    """One extrapolated Tucker block-MM sweep.  Returns (core, factors, core_prev, factors_prev,
    objective of the incoming iterate)."""
    X = _f64(X)
    G = _f64(core).copy()
    Gp = _f64(core_prev).copy()
    fs = [_f64(a).copy() for a in factors]
    ps = [_f64(a).copy() for a in factors_prev]
    f = np.zeros(1)
    pa, pp = _PtrArray(fs), _PtrArray(ps)
    _load().ntfo_tucker_mu_sweep_extrap(X.ndim, _ptr(_dims(X.shape)), _ptr(X), _ptr(_dims(G.shape)), _ptr(G), pa.c,
                                        _ptr(Gp), pp.c, float(beta), float(eps), float(eps_x), float(alpha), float(cap),
                                        float(delta), _ptr(f))
    return G, fs, Gp, ps, float(f[0])


def tucker_jcomm_outer_extrap(X, core, factors, core_prev, factors_prev, beta, alpha, cap=np.inf, delta=1e-12, L=1,
                              eps=1e-12, eps_x=1e-12):
    """One Tucker J-CoMM outer iteration from the extrapolated reference.  Returns (core,
    factors, core_prev, factors_prev, objective of the incoming iterate)."""
    X = _f64(X)
    G = _f64(core).copy()
    Gp = _f64(core_prev).copy()
    fs = [_f64(a).copy() for a in factors]
    ps = [_f64(a).copy() for a in factors_prev]
    f = np.zeros(1)
    pa, pp = _PtrArray(fs), _PtrArray(ps)
    _load().ntfo_tucker_jcomm_outer_extrap(X.ndim, _ptr(_dims(X.shape)), _ptr(X), _ptr(_dims(G.shape)), _ptr(G), pa.c,
                                           _ptr(Gp), pp.c, float(beta), float(eps), float(eps_x), int(L), float(alpha),
                                           float(cap), float(delta), _ptr(f))
    return G, fs, Gp, ps, float(f[0])


def tucker_jcomm_outer(X, core, factors, beta, L=1, eps=1e-12, eps_x=1e-12, max_blocks=-1):
    X = _f64(X)
    G = _f64(core).copy()
    fs = [_f64(a).copy() for a in factors]
    f = np.zeros(1)
    pa = _PtrArray(fs)
    _load().ntfo_tucker_jcomm_outer(X.ndim, _ptr(_dims(X.shape)), _ptr(X), _ptr(_dims(G.shape)), _ptr(G),
                                    pa.c, float(beta), float(eps), float(eps_x), int(L), int(max_blocks),
                                    _ptr(f))
    return G, fs, float(f[0])


# ---------------------------------------------------------------------------- COO

def _coo_args(idx):
    ii = [np.ascontiguousarray(np.asarray(a, dtype=np.int32)) for a in idx]
    return ii, _PtrArray(ii)


def coo_kl_objective(shape, idx, vals, factors, eps=1e-12):
    ii, pi = _coo_args(idx)
    v = _f64(vals)
    fs = [_f64(a) for a in factors]
    pa = _PtrArray(fs)
    return _load().ntfo_coo_kl_objective(len(shape), _ptr(_dims(shape)), v.size, pi.c, _ptr(v),
                                         fs[0].shape[1], pa.c, float(eps))


def coo_kl_jcomm_outer(shape, idx, vals, factors, L=1, eps=1e-12):
    ii, pi = _coo_args(idx)
    v = _f64(vals)
    fs = [_f64(a).copy() for a in factors]
    f = np.zeros(1)
    pa = _PtrArray(fs)
    _load().ntfo_coo_kl_jcomm_outer(len(shape), _ptr(_dims(shape)), v.size, pi.c, _ptr(v), fs[0].shape[1],
                                    pa.c, float(eps), int(L), _ptr(f))
    return fs, float(f[0])


def coo_kl_mu_sweep(shape, idx, vals, factors, eps=1e-12):
    ii, pi = _coo_args(idx)
    v = _f64(vals)
    fs = [_f64(a).copy() for a in factors]
    f = np.zeros(1)
    pa = _PtrArray(fs)
    _load().ntfo_coo_kl_mu_sweep(len(shape), _ptr(_dims(shape)), v.size, pi.c, _ptr(v), fs[0].shape[1],
                                 pa.c, float(eps), _ptr(f))
    return fs, float(f[0])


def stable_perm(keys, K):
    k = np.ascontiguousarray(np.asarray(keys, dtype=np.int32))
    out = np.empty(k.size, dtype=np.int64)
    _load().ntfo_stable_perm(k.size, _ptr(k), int(K), _ptr(out))
    return out


__all__ = [n for n, v in dict(globals()).items()
           if callable(v) and not n.startswith("_") and getattr(v, "__module__", None) == __name__]
