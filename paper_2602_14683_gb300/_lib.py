"""ctypes binding of libntf (include/ntf.h).  Argument marshalling only: every step of
the computation runs in the library's CUDA kernels.  Tensors are torch CUDA tensors
(float32 data/factors/core, int32 COO coordinates, float64 objective scalars); PyTorch
provides device memory and streams.

If the library has not been built this module raises at import: there is no fallback.
"""
import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libntf.so")

NTF_OK = 0
STATUS = {0: "NTF_OK", -1: "NTF_ERR_ARG", -2: "NTF_ERR_BETA", -3: "NTF_ERR_SHAPE", -4: "NTF_ERR_OOM",
          -5: "NTF_ERR_NONFINITE", -6: "NTF_ERR_TIMEOUT", -7: "NTF_ERR_CUDA", -8: "NTF_ERR_UNSUPPORTED"}
NTF_DENSE, NTF_COO = 0, 1
NTF_CP, NTF_TUCKER = 0, 1
NTF_PREC_FP32, NTF_PREC_TF32, NTF_PREC_3XTF32 = 0, 1, 2
PRECISIONS = {"fp32": NTF_PREC_FP32, "tf32": NTF_PREC_TF32, "3xtf32": NTF_PREC_3XTF32}


class NtfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class Tensor(C.Structure):
    _fields_ = [("order", C.c_int), ("dims", C.POINTER(C.c_int64)), ("kind", C.c_int),
                ("values", C.c_void_p), ("idx", C.POINTER(C.c_void_p)), ("nnz", C.c_int64)]


class Job(C.Structure):
    _fields_ = [("model", C.c_int), ("method", C.c_int), ("precision", C.c_int), ("dims", C.c_int64 * 3),
                ("rank", C.c_int), ("core_dims", C.c_int64 * 3), ("beta", C.c_float), ("eps", C.c_double),
                ("rtol", C.c_double), ("max_iters", C.c_int), ("X", C.c_void_p), ("factors", C.c_void_p * 3),
                ("core", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int), ("iterations", C.c_int), ("objective", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("eps", C.c_double), ("eps_x", C.c_double), ("inner_L", C.c_int), ("precision", C.c_int),
                ("autotune", C.c_int), ("merge", C.c_int), ("cache", C.c_int)]


if not os.path.exists(LIB_PATH):
    raise ImportError("libntf.so is not built (%s); run paper_2602_14683_gb300.build.build()" % LIB_PATH)

_lib = C.CDLL(LIB_PATH)
_P = C.c_void_p
_sig = {
    "ntf_opts_default": (None, [C.POINTER(Opts)]),
    "ntf_ctx_create": (C.c_int, [C.POINTER(_P), C.c_int]),
    "ntf_ctx_destroy": (None, [_P]),
    "ntf_last_error": (C.c_char_p, [_P]),
    "ntf_launch_count": (C.c_int64, [_P]),
    "ntf_set_pass_timing": (C.c_int, [_P, C.c_int]),
    "ntf_pass_timing": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "ntf_device_status": (C.c_int, [_P, _P]),
    "ntf_debug_wait_limit": (C.c_int, [_P, C.c_int, C.c_int]),
    "ntf_cp_mu_sweep": (C.c_int, [_P, C.POINTER(Tensor), C.c_float, C.c_int, C.POINTER(_P), C.POINTER(Opts), _P, _P]),
    "ntf_cp_mu_sweep_extrap": (C.c_int, [_P, C.POINTER(Tensor), C.c_float, C.c_int, C.POINTER(_P), C.POINTER(_P),
                                         C.c_float, C.c_float, C.c_float, C.POINTER(Opts), _P, _P]),
    "ntf_cp_jcomm_outer_extrap": (C.c_int, [_P, C.POINTER(Tensor), C.c_float, C.c_int, C.POINTER(_P), C.POINTER(_P),
                                            C.c_float, C.c_float, C.c_float, C.POINTER(Opts), _P, _P]),
    "ntf_tucker_jcomm_outer_extrap": (C.c_int, [_P, C.POINTER(Tensor), C.c_float, C.POINTER(C.c_int64), _P,
                                                C.POINTER(_P), _P, C.POINTER(_P), C.c_float, C.c_float, C.c_float,
                                                C.POINTER(Opts), _P, _P]),
    "ntf_tucker_mu_sweep_extrap": (C.c_int, [_P, C.POINTER(Tensor), C.c_float, C.POINTER(C.c_int64), _P, C.POINTER(_P),
                                             _P, C.POINTER(_P), C.c_float, C.c_float, C.c_float, C.POINTER(Opts), _P,
                                             _P]),
    "ntf_tucker_mu_sweep": (C.c_int, [_P, C.POINTER(Tensor), C.c_float, C.POINTER(C.c_int64), _P, C.POINTER(_P),
                                      C.POINTER(Opts), _P, _P]),
    "ntf_jcomm_outer": (C.c_int, [_P, C.c_int, C.POINTER(Tensor), C.c_float, C.c_int, C.POINTER(C.c_int64), _P,
                                  C.POINTER(_P), C.POINTER(Opts), _P, _P]),
    "ntf_beta_div": (C.c_int, [_P, C.c_int, C.POINTER(Tensor), C.c_float, C.c_int, C.POINTER(C.c_int64), _P,
                               C.POINTER(_P), C.POINTER(Opts), _P, _P]),
    "ntf_coo_stable_perm": (C.c_int, [_P, _P, C.c_int64, C.c_int64, _P, _P]),
    "ntf_plan_cut": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int64), C.c_int, C.POINTER(C.c_int64),
                               C.POINTER(Opts), C.c_float, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "ntf_server_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int, C.c_size_t]),
    "ntf_server_submit": (C.c_int, [_P, C.POINTER(Job), C.POINTER(C.c_int64)]),
    "ntf_server_poll": (C.c_int, [_P, C.POINTER(Result), C.c_int, C.c_int]),
    "ntf_server_destroy": (None, [_P]),
    "ntf_batch_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int, C.c_size_t]),
    "ntf_batch_add": (C.c_int, [_P, C.POINTER(Job), C.POINTER(C.c_int64)]),
    "ntf_batch_tick": (C.c_int, [_P, C.c_int, C.c_int]),
    "ntf_batch_results": (C.c_int, [_P, C.POINTER(Result), C.c_int]),
    "ntf_batch_resident": (C.c_int, [_P]),
    "ntf_batch_destroy": (None, [_P]),
    "ntf_cp_beta_div_noalloc": (C.c_int, [C.POINTER(Tensor), C.c_float, C.c_int, C.POINTER(_P), C.c_double,
                                          C.c_double, _P, _P]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


class Context:
    """Owns an ntf_ctx (workspaces) bound to one CUDA device."""

    def __init__(self, device=0):
        h = _P()
        rc = _lib.ntf_ctx_create(C.byref(h), int(device))
        if rc != NTF_OK:
            raise NtfError(rc, "ntf_ctx_create(device=%d) failed" % device)
        self.h = h
        self.device = int(device)

    def close(self):
        if self.h:
            _lib.ntf_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self):
        return int(_lib.ntf_launch_count(self.h))

    def set_pass_timing(self, enable=True):
        self.check(_lib.ntf_set_pass_timing(self.h, 1 if enable else 0))

    def pass_timing(self):
        """(total milliseconds, number of fused-pass launches) since the last query."""
        ms = C.c_double()
        n = C.c_int64()
        self.check(_lib.ntf_pass_timing(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def device_status(self, stream=None):
        """Synchronizes the stream and raises NtfError(NTF_ERR_TIMEOUT) if a bounded
        device-side wait gave up since the last check."""
        self.check(_lib.ntf_device_status(self.h, _stream(stream)))

    def debug_wait_limit(self, polls=0, probe=False):
        """Testing aid: polls before a bounded wait gives up (0: built-in), and the timeout
        probe (every tensor-core pass aborts on a wait that runs out before it issues work)."""
        self.check(_lib.ntf_debug_wait_limit(self.h, int(polls), 1 if probe else 0))

    def check(self, rc):
        if rc != NTF_OK:
            raise NtfError(rc, _lib.ntf_last_error(self.h).decode(errors="replace"))


_contexts = {}


def default_context(device=None):
    if device is None:
        device = torch.cuda.current_device()
    if device not in _contexts:
        _contexts[device] = Context(device)
    return _contexts[device]


class Coo:
    """COO tensor: `idx` is a list of N int32 CUDA tensors (nnz each), `values` float32."""

    def __init__(self, shape, idx, values):
        self.shape = tuple(int(s) for s in shape)
        self.idx = [i.contiguous() for i in idx]
        self.values = values.contiguous()
        self.nnz = int(values.numel())


def _check_dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


class _Desc:
    """Keeps the C descriptor and the arrays it points to alive for one call."""

    def __init__(self, X):
        if isinstance(X, Coo):
            _check_dev(X.values, torch.float32, "values")
            for i in X.idx:
                _check_dev(i, torch.int32, "COO coordinates")
            self.dims = (C.c_int64 * len(X.shape))(*X.shape)
            self.idx = (C.c_void_p * len(X.idx))(*[i.data_ptr() for i in X.idx])
            self.t = Tensor(len(X.shape), self.dims, NTF_COO, X.values.data_ptr(), self.idx, X.nnz)
        else:
            _check_dev(X, torch.float32, "X")
            self.dims = (C.c_int64 * X.dim())(*X.shape)
            self.idx = None
            self.t = Tensor(X.dim(), self.dims, NTF_DENSE, X.data_ptr(), None, 0)


def _ptrs(tensors, name):
    for t in tensors:
        _check_dev(t, torch.float32, name)
    return (C.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])


CACHE_MODES = {"auto": 0, "none": 1, "bf16": 2}


def make_opts(eps=1e-12, eps_x=1e-12, inner_L=1, precision="fp32", autotune=False, merge=None, cache="auto"):
    """merge: None, or (a, b) cutting the modes of an order N >= 4 tensor into the runs
    [0, a), [a, b), [b, N) of the 3-way view.  cache: "auto", "none" or "bf16" (J-CoMM's
    reference-powered tensors at beta != 1 on the tensor-core passes)."""
    o = Opts()
    _lib.ntf_opts_default(C.byref(o))
    o.eps, o.eps_x, o.inner_L = float(eps), float(eps_x), int(inner_L)
    o.autotune = 1 if autotune else 0
    o.merge = 0 if merge is None else 16 * int(merge[0]) + int(merge[1])
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.cache = CACHE_MODES[cache] if isinstance(cache, str) else int(cache)
    return o


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _out_ptr(t):
    if t is None:
        return None
    _check_dev(t, torch.float64, "objective")
    return t.data_ptr()


def cp_mu_sweep(X, beta, factors, objective=None, ctx=None, stream=None, **opts):
    """One B-CoMM sweep (Algorithm 1); factors updated in place.  `objective` (float64
    CUDA tensor, 1 element) receives D_beta of the incoming iterate."""
    ctx = ctx or default_context()
    d = _Desc(X)
    fp = _ptrs(factors, "factors")
    o = make_opts(**opts)
    rank = int(factors[0].shape[1])
    ctx.check(_lib.ntf_cp_mu_sweep(ctx.h, C.byref(d.t), float(beta), rank, fp, C.byref(o),
                                   _out_ptr(objective), _stream(stream)))


def cp_mu_sweep_extrap(X, beta, factors, factors_prev, alpha, cap=float("inf"), delta=1e-12, objective=None,
                       ctx=None, stream=None, **opts):
    """One extrapolated B-CoMM sweep (dense 3-way CP): factors A^t -> A^(t+1) in place,
    factors_prev A^(t-1) -> A^t in place; `alpha` is this iteration's extrapolation weight,
    capped per block at cap / (||[A - Aprev]_+|| + delta).  `objective` receives D_beta of the
    incoming iterate."""
    ctx = ctx or default_context()
    d = _Desc(X)
    fp = _ptrs(factors, "factors")
    pp = _ptrs(factors_prev, "factors_prev")
    o = make_opts(**opts)
    rank = int(factors[0].shape[1])
    ctx.check(_lib.ntf_cp_mu_sweep_extrap(ctx.h, C.byref(d.t), float(beta), rank, fp, pp, float(alpha), float(cap),
                                          float(delta), C.byref(o), _out_ptr(objective), _stream(stream)))


def cp_jcomm_outer_extrap(X, beta, factors, factors_prev, alpha, cap=float("inf"), delta=1e-12, objective=None,
                          ctx=None, stream=None, **opts):
    """One J-CoMM outer iteration (dense 3-way CP) from the extrapolated reference
    max(A + alpha_n [A - Aprev]_+, eps); factors A^t -> new iterate, factors_prev -> A^t, in
    place.  `objective` receives D_beta of the incoming iterate."""
    ctx = ctx or default_context()
    d = _Desc(X)
    fp = _ptrs(factors, "factors")
    pp = _ptrs(factors_prev, "factors_prev")
    o = make_opts(**opts)
    rank = int(factors[0].shape[1])
    ctx.check(_lib.ntf_cp_jcomm_outer_extrap(ctx.h, C.byref(d.t), float(beta), rank, fp, pp, float(alpha), float(cap),
                                             float(delta), C.byref(o), _out_ptr(objective), _stream(stream)))


def tucker_mu_sweep_extrap(X, beta, core, factors, core_prev, factors_prev, alpha, cap=float("inf"), delta=1e-12,
                           objective=None, ctx=None, stream=None, **opts):
    """One extrapolated Tucker block-MM sweep: core / factors -> new iterate, core_prev /
    factors_prev -> the incoming iterate, in place."""
    ctx = ctx or default_context()
    d = _Desc(X)
    _check_dev(core, torch.float32, "core")
    _check_dev(core_prev, torch.float32, "core_prev")
    cd = (C.c_int64 * core.dim())(*core.shape)
    fp = _ptrs(factors, "factors")
    pp = _ptrs(factors_prev, "factors_prev")
    o = make_opts(**opts)
    ctx.check(_lib.ntf_tucker_mu_sweep_extrap(ctx.h, C.byref(d.t), float(beta), cd, C.c_void_p(core.data_ptr()), fp,
                                              C.c_void_p(core_prev.data_ptr()), pp, float(alpha), float(cap),
                                              float(delta), C.byref(o), _out_ptr(objective), _stream(stream)))


def tucker_jcomm_outer_extrap(X, beta, core, factors, core_prev, factors_prev, alpha, cap=float("inf"), delta=1e-12,
                              objective=None, ctx=None, stream=None, **opts):
    """One Tucker J-CoMM outer iteration from the extrapolated reference: core / factors ->
    new iterate, core_prev / factors_prev -> the incoming iterate, in place."""
    ctx = ctx or default_context()
    d = _Desc(X)
    _check_dev(core, torch.float32, "core")
    _check_dev(core_prev, torch.float32, "core_prev")
    cd = (C.c_int64 * core.dim())(*core.shape)
    fp = _ptrs(factors, "factors")
    pp = _ptrs(factors_prev, "factors_prev")
    o = make_opts(**opts)
    ctx.check(_lib.ntf_tucker_jcomm_outer_extrap(ctx.h, C.byref(d.t), float(beta), cd, C.c_void_p(core.data_ptr()),
                                                 fp, C.c_void_p(core_prev.data_ptr()), pp, float(alpha), float(cap),
                                                 float(delta), C.byref(o), _out_ptr(objective), _stream(stream)))


def nesterov_weights():
    """Extrapolation weights alpha_t = (a_(t-1) - 1) / a_t with a_0 = 1 and
    a_t = (1 + sqrt(1 + 4 a_(t-1)^2)) / 2 -- the accelerated-gradient momentum sequence of
    Beck and Teboulle (FISTA) -- for t = 1, 2, ... (alpha_1 = 0)."""
    import math
    a = 1.0
    while True:
        a_next = (1.0 + math.sqrt(1.0 + 4.0 * a * a)) / 2.0
        yield (a - 1.0) / a_next
        a = a_next


def tucker_mu_sweep(X, beta, core, factors, objective=None, ctx=None, stream=None, **opts):
    """One Tucker block-MM sweep (core, then factors); blocks updated in place."""
    ctx = ctx or default_context()
    d = _Desc(X)
    _check_dev(core, torch.float32, "core")
    cd = (C.c_int64 * core.dim())(*core.shape)
    fp = _ptrs(factors, "factors")
    o = make_opts(**opts)
    ctx.check(_lib.ntf_tucker_mu_sweep(ctx.h, C.byref(d.t), float(beta), cd, core.data_ptr(), fp, C.byref(o),
                                       _out_ptr(objective), _stream(stream)))


def jcomm_outer(X, beta, factors, core=None, objective=None, ctx=None, stream=None, **opts):
    """One J-CoMM outer iteration (Algorithm 2) for CP (core=None) or Tucker; blocks
    updated in place.  `objective` receives D_beta at the reference (incoming) iterate."""
    ctx = ctx or default_context()
    d = _Desc(X)
    fp = _ptrs(factors, "factors")
    o = make_opts(**opts)
    if core is None:
        rc = _lib.ntf_jcomm_outer(ctx.h, NTF_CP, C.byref(d.t), float(beta), int(factors[0].shape[1]), None, None,
                                  fp, C.byref(o), _out_ptr(objective), _stream(stream))
    else:
        _check_dev(core, torch.float32, "core")
        cd = (C.c_int64 * core.dim())(*core.shape)
        rc = _lib.ntf_jcomm_outer(ctx.h, NTF_TUCKER, C.byref(d.t), float(beta), 0, cd, core.data_ptr(), fp,
                                  C.byref(o), _out_ptr(objective), _stream(stream))
    ctx.check(rc)


def plan_cut(dims, rank=None, core_dims=None, beta=1.0, **opts):
    """(a, b): the runs [0, a), [a, b), [b, N) an order-N dense CP (rank) or Tucker (core_dims)
    problem is cut into (host-only planning, no device)."""
    n = len(dims)
    d = (C.c_int64 * n)(*dims)
    cd = (C.c_int64 * n)(*core_dims) if core_dims is not None else None
    a, b = C.c_int(), C.c_int()
    o = make_opts(**opts)
    model = NTF_CP if core_dims is None else NTF_TUCKER
    rc = _lib.ntf_plan_cut(model, n, d, int(rank or 0), cd, C.byref(o), float(beta), C.byref(a), C.byref(b))
    if rc != NTF_OK:
        raise NtfError(rc, "ntf_plan_cut failed")
    return a.value, b.value


def beta_div(X, beta, factors, core=None, out=None, ctx=None, stream=None, **opts):
    """D_beta(X, Xhat) in FP64; returns a 1-element float64 CUDA tensor (written on the
    stream, not synchronised)."""
    ctx = ctx or default_context()
    d = _Desc(X)
    fp = _ptrs(factors, "factors")
    o = make_opts(**opts)
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=factors[0].device)
    if core is None:
        rc = _lib.ntf_beta_div(ctx.h, NTF_CP, C.byref(d.t), float(beta), int(factors[0].shape[1]), None, None, fp,
                               C.byref(o), _out_ptr(out), _stream(stream))
    else:
        _check_dev(core, torch.float32, "core")
        cd = (C.c_int64 * core.dim())(*core.shape)
        rc = _lib.ntf_beta_div(ctx.h, NTF_TUCKER, C.byref(d.t), float(beta), 0, cd, core.data_ptr(), fp,
                               C.byref(o), _out_ptr(out), _stream(stream))
    ctx.check(rc)
    return out


def coo_stable_perm(keys, key_range, ctx=None, stream=None):
    """Stable permutation (int32) ordering `keys` (int32 CUDA tensor)."""
    ctx = ctx or default_context()
    _check_dev(keys, torch.int32, "keys")
    out = torch.empty_like(keys)
    ctx.check(_lib.ntf_coo_stable_perm(ctx.h, keys.data_ptr(), keys.numel(), int(key_range), out.data_ptr(),
                                       _stream(stream)))
    return out


def cp_beta_div_noalloc(X, beta, factors, out, eps=1e-12, eps_x=1e-12, stream=None):
    """Allocation-free dense CP objective (ntf_cp_beta_div_noalloc); `out` is a 1-element
    float64 CUDA tensor owned by the caller.  Returns the C status code."""
    d = _Desc(X)
    fp = _ptrs(factors, "factors")
    return _lib.ntf_cp_beta_div_noalloc(C.byref(d.t), float(beta), int(factors[0].shape[1]), fp, float(eps),
                                        float(eps_x), _out_ptr(out), _stream(stream))


def _job(X, beta, factors, core, method, rtol, max_iters, precision, eps):
    _check_dev(X, torch.float32, "X")
    for f in factors:
        _check_dev(f, torch.float32, "factors")
    j = Job()
    j.model = NTF_CP if core is None else NTF_TUCKER
    j.method = {"jcomm": 0, "block": 1}[method]
    j.precision = PRECISIONS[precision]
    for n in range(3):
        j.dims[n] = X.shape[n]
    if core is None:
        j.rank = factors[0].shape[1]
    else:
        _check_dev(core, torch.float32, "core")
        for n in range(3):
            j.core_dims[n] = core.shape[n]
        j.core = core.data_ptr()
    j.beta, j.eps, j.rtol, j.max_iters = float(beta), float(eps), float(rtol), int(max_iters)
    j.X = X.data_ptr()
    for n in range(3):
        j.factors[n] = factors[n].data_ptr()
    return j


def _results(buf, n):
    return [dict(id=buf[q].id, status=buf[q].status, iterations=buf[q].iterations, objective=buf[q].objective,
                 t_submit=buf[q].t_submit, t_admit=buf[q].t_admit, t_done=buf[q].t_done) for q in range(n)]


class Batch:
    """Launches shared by many small dense CP jobs (ntf_batch_*): add jobs made of CUDA
    tensors, tick, collect results.  Keeps every resident job's tensors alive until its
    result has been collected."""

    def __init__(self, device=0, capacity=1024, mem_budget_bytes=0):
        h = _P()
        rc = _lib.ntf_batch_create(C.byref(h), int(device), int(capacity), int(mem_budget_bytes))
        if rc != NTF_OK:
            raise NtfError(rc, "ntf_batch_create failed")
        self.h = h
        self._live = {}

    def add(self, X, beta, factors, method="jcomm", rtol=1e-6, max_iters=200, eps=1e-12):
        """Makes a job resident; returns its id, or None when it does not fit now."""
        j = _job(X, beta, factors, None, method, rtol, max_iters, "fp32", eps)
        jid = C.c_int64()
        rc = _lib.ntf_batch_add(self.h, C.byref(j), C.byref(jid))
        if rc == -4:
            return None
        if rc != NTF_OK:
            raise NtfError(rc, "ntf_batch_add failed")
        self._live[jid.value] = (X, factors)
        return jid.value

    def tick(self, iters=8, wait=True):
        rc = _lib.ntf_batch_tick(self.h, int(iters), 1 if wait else 0)
        if rc < 0:
            raise NtfError(rc, "ntf_batch_tick failed")
        return rc

    def results(self, max_results=4096):
        buf = (Result * max_results)()
        out = _results(buf, _lib.ntf_batch_results(self.h, buf, max_results))
        for r in out:
            self._live.pop(r["id"], None)
        return out

    def run(self, iters=8):
        """Ticks until every resident job has finished; returns all results."""
        out = []
        while self.tick(iters, wait=True) > 0:
            out += self.results()
        return out + self.results()

    def close(self):
        if self.h:
            _lib.ntf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (ntf_server_*): submit jobs made of CUDA tensors, poll
    results.  Keeps every submitted job's tensors alive until its result is polled."""

    def __init__(self, device=0, slots=8, mem_budget_bytes=0):
        h = _P()
        rc = _lib.ntf_server_create(C.byref(h), int(device), int(slots), int(mem_budget_bytes))
        if rc != NTF_OK:
            raise NtfError(rc, "ntf_server_create failed")
        self.h = h
        self._live = {}

    def submit(self, X, beta, factors, core=None, method="jcomm", rtol=1e-6, max_iters=200, precision="fp32",
               eps=1e-12):
        j = _job(X, beta, factors, core, method, rtol, max_iters, precision, eps)
        jid = C.c_int64()
        rc = _lib.ntf_server_submit(self.h, C.byref(j), C.byref(jid))
        if rc != NTF_OK:
            raise NtfError(rc, "ntf_server_submit failed")
        self._live[jid.value] = (X, factors, core)
        return jid.value

    def poll(self, wait_all=False, max_results=4096):
        buf = (Result * max_results)()
        n = _lib.ntf_server_poll(self.h, buf, max_results, 1 if wait_all else 0)
        if n < 0:
            raise NtfError(n, "ntf_server_poll failed")
        out = _results(buf, n)
        for r in out:
            self._live.pop(r["id"], None)
        return out

    def close(self):
        if self.h:
            _lib.ntf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def raw_library():
    """The loaded ctypes CDLL (for ABI-level tests)."""
    return _lib
