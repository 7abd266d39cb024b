"""Thin Python binding of the libkrr C ABI (``include/libkrr.h``).

Argument marshalling only: every step of every call runs in the CUDA library.
Arrays may be CUDA ``torch.Tensor``s (device pointers; calls are ordered on
the current torch stream, or the ``stream`` given) or NumPy arrays (host
pointers; the library stages them through device memory and synchronises).

Layouts follow the C ABI: X is (N, d) row-major float32; multi-column arrays
are column-major N x m, i.e. a contiguous (m, N) array (one row per column).
A one-dimensional (N,) array is the single-column case.

If ``libkrr.so`` is missing the loader raises: there is no fallback path.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libkrr.so")

KRR_OK, KRR_ERR_INVALID_ARG, KRR_ERR_CUDA, KRR_ERR_OOM, KRR_ERR_NONFINITE = 0, 1, 2, 3, 4
KRR_NOT_CONVERGED, KRR_ERR_BREAKDOWN, KRR_ERR_TIMEOUT, KRR_ERR_UNIMPLEMENTED = 5, 6, 7, 8
KRR_ERR_SIZE_LIMIT = 9
PRECISION = {"fp32": 0, "bf16": 1, "fp16": 2}


class KrrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


class krr_fgmres_opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_cycles", ctypes.c_int),
                ("tol", ctypes.c_double), ("delta", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("inner_maxit", ctypes.c_int),
                ("inner_prec", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("x0_given", ctypes.c_int)]


class krr_solve_info(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("cycles", ctypes.c_int), ("breakdowns", ctypes.c_int),
                ("relres_est", ctypes.c_double), ("relres_true", ctypes.c_double),
                ("time_ms", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class krr_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("product_launches", ctypes.c_int),
                ("product_ms", ctypes.c_double), ("product_pairs", ctypes.c_double),
                ("tensor_exponent_launches", ctypes.c_int)]


class krr_problem(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("B", ctypes.c_void_p), ("Xsol", ctypes.c_void_p),
                ("N", ctypes.c_int64), ("gamma", ctypes.c_float)]


_lib = None

_vp, _i64, _int, _f, _d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_double
_SIGNATURES = {
    "krr_create": ([ctypes.POINTER(_vp)], _int),
    "krr_destroy": ([_vp], _int),
    "krr_last_error": ([_vp], ctypes.c_char_p),
    "krr_status_string": ([_int], ctypes.c_char_p),
    "krr_version": ([], _int),
    "krr_fgmres_default_opts": ([ctypes.POINTER(krr_fgmres_opts)], None),
    "krr_kernel_mvp": ([_vp, _vp, _i64, _int, _f, _f, _vp, _int, _vp, _int, _vp], _int),
    "krr_kernel_mvp_rect": ([_vp, _vp, _i64, _vp, _i64, _int, _f, _vp, _int, _vp, _int, _vp], _int),
    "krr_cg_solve": ([_vp, _vp, _i64, _int, _f, _f, _vp, _vp, _d, _int, _int,
                      ctypes.POINTER(krr_solve_info), _vp], _int),
    "krr_fgmres_solve": ([_vp, _vp, _i64, _int, _f, _f, _vp, _int, _vp,
                          ctypes.POINTER(krr_fgmres_opts), ctypes.POINTER(krr_solve_info), _vp], _int),
    "krr_fcg_solve": ([_vp, _vp, _i64, _int, _f, _f, _vp, _int, _vp,
                       ctypes.POINTER(krr_fgmres_opts), ctypes.POINTER(krr_solve_info), _vp], _int),
    "krr_fgmres_solve_batched": ([_vp, ctypes.POINTER(krr_problem), _int, _int, _f, _int,
                                  ctypes.POINTER(krr_fgmres_opts), ctypes.POINTER(krr_solve_info),
                                  _vp], _int),
    "krr_mll_grad": ([_vp, _vp, _i64, _int, _f, _f, _vp, _int, ctypes.c_uint64,
                      ctypes.POINTER(krr_fgmres_opts), ctypes.POINTER(_d), ctypes.POINTER(_d),
                      _vp, ctypes.POINTER(krr_solve_info), _vp], _int),
    "krr_measure_alu_peaks": ([_vp, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_d),
                               _vp], _int),
    "krr_measure_rsqrt_rate": ([_vp, ctypes.POINTER(_d), _vp], _int),
    "krr_measure_half_rates": ([_vp, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_d), _vp], _int),
    "krr_profile_enable": ([_vp, _int], _int),
    "krr_set_option": ([_vp, _int, _int], _int),
    "krr_kernel_mvp_noalloc": ([_vp, _i64, _int, _f, _f, _vp, _int, _vp, _vp], _int),
    "krr_profile_read": ([_vp, ctypes.POINTER(krr_profile)], _int),
    "krr_selftest_wait_timeout": ([_vp, ctypes.c_longlong, _vp], _int),
    "krr_points_create": ([_vp, _vp, _i64, _int, _f, ctypes.POINTER(_vp), _vp], _int),
    "krr_kernel_mvp_points": ([_vp, _vp, _vp, _int, _f, _vp, _int, _vp], _int),
    "krr_points_destroy": ([_vp, _vp], _int),
    "krr_tune_save": ([_vp, ctypes.c_char_p], _int),
    "krr_tune_load": ([_vp, ctypes.c_char_p], _int),
}


def lib():
    """The loaded C library (raises if libkrr.so has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libkrr.so not found at {LIB_PATH}: build it with "
                              "paper_1408_1237_gb300.build.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def status_string(s):
    try:
        return lib().krr_status_string(int(s)).decode()
    except Exception:  # library not loadable: still give a readable code
        return f"status {s}"


def default_opts(**kw):
    o = krr_fgmres_opts()
    lib().krr_fgmres_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "inner_prec" and isinstance(v, str):
            v = PRECISION[v]
        setattr(o, k, v)
    return o


class Handle:
    """Owns a krr_handle (device workspace bound to the current CUDA device)."""

    def __init__(self):
        h = _vp()
        s = lib().krr_create(ctypes.byref(h))
        if s != KRR_OK:
            raise KrrError(s, "krr_create failed")
        self.h = h

    def close(self):
        if self.h:
            lib().krr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def check(self, s):
        if s not in (KRR_OK,):
            raise KrrError(s, lib().krr_last_error(self.h).decode())
        return s


_default = None


def default_handle():
    global _default
    if _default is None:
        _default = Handle()
    return _default


# ------------------------------------------------------------- marshalling
def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """Device or host pointer of a float32 contiguous array (None -> NULL)."""
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
        raise ValueError("array must be a contiguous numpy array or torch tensor")
    return a.ctypes.data


def _check_f32(a, name):
    if a is None:
        return
    dt = str(a.dtype)
    if dt not in ("float32", "torch.float32"):
        raise TypeError(f"{name} must be float32, got {dt}")


def _stream(stream, *arrays):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def _empty_like_cols(ref, m, N, dtype="float32"):
    shape = (N,) if m == 1 else (m, N)
    if _is_torch(ref):
        import torch
        return torch.empty(shape, dtype=getattr(torch, dtype), device=ref.device)
    return np.empty(shape, dtype=dtype)


def _cols(Q, N):
    if Q.ndim == 1:
        return 1
    if Q.shape[1] != N:
        raise ValueError(f"multi-column arrays are (m, N) column blocks; got {tuple(Q.shape)}")
    return Q.shape[0]


# ---------------------------------------------------------------- calls
def krr_kernel_mvp(X, Q, sigma, gamma, prec="fp32", out=None, handle=None, stream=None):
    """Y = (K_hat + gamma I) Q.  X (N, d); Q (N,) or (m, N); returns like Q."""
    h = handle or default_handle()
    _check_f32(X, "X")
    _check_f32(Q, "Q")
    N, d = X.shape
    m = _cols(Q, N)
    Y = out if out is not None else _empty_like_cols(Q, m, N)
    h.check(lib().krr_kernel_mvp(h.h, _ptr(X), N, d, sigma, gamma, _ptr(Q), m, _ptr(Y),
                                 PRECISION[prec], _stream(stream, X, Q, Y)))
    return Y


class Points:
    """A prepared point set (krr_points_create): products over it with
    krr_kernel_mvp_points run with no host synchronisation.  Close it (or use
    it as a context manager) before its handle."""

    def __init__(self, X, sigma, handle=None, stream=None):
        self.handle = handle or default_handle()
        _check_f32(X, "X")
        self.N, self.d = X.shape
        p = _vp()
        self.handle.check(lib().krr_points_create(self.handle.h, _ptr(X), self.N, self.d, sigma,
                                                  ctypes.byref(p), _stream(stream, X)))
        self.p = p

    def close(self):
        if self.p and self.handle.h:
            p, self.p = self.p, None
            self.handle.check(lib().krr_points_destroy(self.handle.h, p))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def krr_points_create(X, sigma, handle=None, stream=None):
    return Points(X, sigma, handle=handle, stream=stream)


def krr_kernel_mvp_points(points, Q, gamma, prec="fp32", out=None, stream=None):
    """Y = (K_hat + gamma I) Q over a prepared point set; Q and Y device
    tensors, (N,) or (m, N)."""
    _check_f32(Q, "Q")
    m = _cols(Q, points.N)
    Y = out if out is not None else _empty_like_cols(Q, m, points.N)
    points.handle.check(lib().krr_kernel_mvp_points(points.handle.h, points.p, _ptr(Q), m, gamma, _ptr(Y),
                                                    PRECISION[prec], _stream(stream, Q, Y)))
    return Y


def krr_kernel_mvp_rect(Xt, Xs, Q, sigma, prec="fp32", out=None, handle=None, stream=None):
    """Y = K_hat(Xt, Xs) Q (prediction product).  Q (Ns,) or (m, Ns)."""
    h = handle or default_handle()
    Nt, d = Xt.shape
    Ns = Xs.shape[0]
    m = _cols(Q, Ns)
    Y = out if out is not None else _empty_like_cols(Q, m, Nt)
    h.check(lib().krr_kernel_mvp_rect(h.h, _ptr(Xt), Nt, _ptr(Xs), Ns, d, sigma, _ptr(Q), m,
                                      _ptr(Y), PRECISION[prec], _stream(stream, Xt, Q, Y)))
    return Y


def krr_cg_solve(X, b, sigma, shift, tol=1e-6, maxit=1000, prec="fp32", x0=None,
                 handle=None, stream=None, raise_on_nonconv=False):
    """CG on (K_hat + shift I) x = b.  Returns (x FP64, info dict)."""
    h = handle or default_handle()
    N, d = X.shape
    if x0 is None:
        x = _empty_like_cols(b, 1, N, "float64")
        x[...] = 0
    else:
        x = x0
    info = krr_solve_info()
    s = lib().krr_cg_solve(h.h, _ptr(X), N, d, sigma, shift, _ptr(b), _ptr(x), tol, maxit,
                           PRECISION[prec], ctypes.byref(info), _stream(stream, X, b, x))
    if s != KRR_NOT_CONVERGED or raise_on_nonconv:
        h.check(s)
    return x, info.as_dict()


def krr_fgmres_solve(X, B, sigma, gamma, opts=None, out=None, handle=None, stream=None,
                     raise_on_nonconv=False):
    """FGMRES with the truncated-CG preconditioner.  B (N,) or (m, N) float32.
    Returns (Xsol FP64 like B, [info dict per column])."""
    h = handle or default_handle()
    N, d = X.shape
    m = _cols(B, N)
    Xsol = out if out is not None else _empty_like_cols(B, m, N, "float64")
    if opts is None:
        opts = default_opts()
    infos = (krr_solve_info * m)()
    s = lib().krr_fgmres_solve(h.h, _ptr(X), N, d, sigma, gamma, _ptr(B), m, _ptr(Xsol),
                               ctypes.byref(opts), infos, _stream(stream, X, B, Xsol))
    if s != KRR_NOT_CONVERGED or raise_on_nonconv:
        h.check(s)
    return Xsol, [i.as_dict() for i in infos]


def krr_fcg_solve(X, B, sigma, gamma, opts=None, out=None, handle=None, stream=None,
                  raise_on_nonconv=False):
    """Flexible CG with the truncated-CG preconditioner (opts.restart = the
    window of kept directions).  B (N,) or (m, N) float32.
    Returns (Xsol FP64 like B, [info dict per column])."""
    h = handle or default_handle()
    N, d = X.shape
    m = _cols(B, N)
    Xsol = out if out is not None else _empty_like_cols(B, m, N, "float64")
    if opts is None:
        opts = default_opts()
    infos = (krr_solve_info * m)()
    s = lib().krr_fcg_solve(h.h, _ptr(X), N, d, sigma, gamma, _ptr(B), m, _ptr(Xsol),
                            ctypes.byref(opts), infos, _stream(stream, X, B, Xsol))
    if s != KRR_NOT_CONVERGED or raise_on_nonconv:
        h.check(s)
    return Xsol, [i.as_dict() for i in infos]


def krr_fgmres_solve_batched(problems, d, sigma, m_rhs, opts=None, handle=None, stream=None,
                             with_info=True, raise_on_nonconv=False):
    """problems: list of dicts with device tensors X (N, d), B (m, N), Xsol (m, N), gamma."""
    h = handle or default_handle()
    arr = (krr_problem * len(problems))()
    for k, p in enumerate(problems):
        arr[k].X, arr[k].B, arr[k].Xsol = _ptr(p["X"]), _ptr(p["B"]), _ptr(p["Xsol"])
        arr[k].N = p["X"].shape[0]
        arr[k].gamma = p["gamma"]
    if opts is None:
        opts = default_opts()
    infos = (krr_solve_info * (len(problems) * m_rhs))() if with_info else None
    st = _stream(stream, problems[0]["X"]) if problems else None
    s = lib().krr_fgmres_solve_batched(h.h, arr, len(problems), d, sigma, m_rhs,
                                       ctypes.byref(opts), infos, st)
    if s != KRR_NOT_CONVERGED or raise_on_nonconv:
        h.check(s)
    return [i.as_dict() for i in infos] if with_info else None


def krr_mll_grad(X, y, sigma, gamma, n_probes=32, seed=0, opts=None, want_dX=True,
                 handle=None, stream=None):
    """Returns (dlogsigma, dloggamma, dX or None, [info dicts])."""
    h = handle or default_handle()
    N, d = X.shape
    ds, dg = ctypes.c_double(), ctypes.c_double()
    dX = None
    if want_dX:
        if _is_torch(X):
            import torch
            dX = torch.empty((N, d), dtype=torch.float32, device=X.device)
        else:
            dX = np.empty((N, d), dtype=np.float32)
    if opts is None:
        opts = default_opts()
    infos = (krr_solve_info * (1 + n_probes))()
    h.check(lib().krr_mll_grad(h.h, _ptr(X), N, d, sigma, gamma, _ptr(y), n_probes, seed,
                               ctypes.byref(opts), ctypes.byref(ds), ctypes.byref(dg), _ptr(dX),
                               infos, _stream(stream, X, y)))
    return ds.value, dg.value, dX, [i.as_dict() for i in infos]


def krr_measure_alu_peaks(handle=None, stream=None):
    """(ex2/s, scalar FFMA/s, FP32 lanes/s via FFMA2) on the current device."""
    h = handle or default_handle()
    a, b, c = _d(), _d(), _d()
    h.check(lib().krr_measure_alu_peaks(h.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                        stream))
    return a.value, b.value, c.value


def krr_measure_rsqrt_rate(handle=None, stream=None):
    """rsqrtf results per second on the current device."""
    h = handle or default_handle()
    a = _d()
    h.check(lib().krr_measure_rsqrt_rate(h.h, ctypes.byref(a), stream))
    return a.value


def krr_measure_half_rates(handle=None, stream=None):
    """(ex2.f16x2 values/s, ex2.bf16x2 values/s, mma.sync f16 FLOP/s) on the
    current device."""
    h = handle or default_handle()
    a, b, c = _d(), _d(), _d()
    h.check(lib().krr_measure_half_rates(h.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), stream))
    return a.value, b.value, c.value


def krr_selftest_wait_timeout(limit_clocks=4000, handle=None, stream=None):
    """Run a kernel whose bounded wait cannot complete (an mbarrier phase
    nothing arrives on) and give up after limit_clocks SM clocks; returns the
    status the library reports (KRR_ERR_TIMEOUT), without raising."""
    h = handle or default_handle()
    return lib().krr_selftest_wait_timeout(h.h, int(limit_clocks), stream)


KRR_OPT_TCGEN05 = 1
KRR_OPT_KERNEL = 2
KRR_OPT_AUTOTUNE = 3
KRR_OPT_SHARD_COUNT, KRR_OPT_SHARD_INDEX = 4, 5
KRR_OPT_HIGHD_TCGEN05 = 6
KRR_OPT_DIRECT_TENSOR = 7
KRR_KERNEL_GAUSSIAN, KRR_KERNEL_MATERN32 = 0, 1


def krr_set_option(option, value, handle=None):
    """Set a handle option (KRR_OPT_TCGEN05: the kernel of multi-column
    products' compact blocks, 0 mma.sync, 1 and 2 tcgen05, 3 automatic by
    precision and columns; KRR_OPT_KERNEL: the
    kernel function, KRR_KERNEL_GAUSSIAN or KRR_KERNEL_MATERN32, whose length
    scale h is then passed as sigma; KRR_OPT_AUTOTUNE: time the products'
    kernel variants and source splits on first use of each shape and keep
    the fastest; the others as documented in include/libkrr.h)."""
    h = handle or default_handle()
    h.check(lib().krr_set_option(h.h, int(option), int(value)))


def krr_tune_save(path, handle=None):
    """Write the handle's tuning results (kernel variant and split scale per
    product shape) to a text file."""
    h = handle or default_handle()
    h.check(lib().krr_tune_save(h.h, str(path).encode()))


def krr_tune_load(path, handle=None):
    """Read tuning results written by krr_tune_save (same SM count) into the
    handle, so that its products skip the timing."""
    h = handle or default_handle()
    h.check(lib().krr_tune_load(h.h, str(path).encode()))


def krr_profile_enable(enable=True, handle=None):
    h = handle or default_handle()
    h.check(lib().krr_profile_enable(h.h, 1 if enable else 0))


def krr_profile_read(handle=None):
    """dict(launches, product_launches, product_ms, product_pairs,
    tensor_exponent_launches); resets the timed list."""
    h = handle or default_handle()
    p = krr_profile()
    h.check(lib().krr_profile_read(h.h, ctypes.byref(p)))
    return {f: getattr(p, f) for f, _ in p._fields_}


def krr_kernel_mvp_noalloc(X, Q, sigma, gamma, out=None, stream=None):
    """The kernel product through the entry point that allocates no device
    memory (for callers that cannot allocate: processes whose memory pool
    belongs to another framework, latency-bound paths).  Device tensors only;
    N <= 16384, d <= 8, m <= 16.  Waits for the stream; refuses a capturing
    stream.  The output is allocated here, by the caller side, unless `out`
    is given."""
    N, d = X.shape
    m = _cols(Q, N)
    Y = out if out is not None else _empty_like_cols(Q, m, N)
    s = lib().krr_kernel_mvp_noalloc(_ptr(X), N, d, sigma, gamma, _ptr(Q), m, _ptr(Y),
                                     _stream(stream, X, Q, Y))
    if s != KRR_OK:
        raise KrrError(s, "krr_kernel_mvp_noalloc (limits: device arrays, N <= 16384, "
                          "d <= 8, m <= 16)")
    return Y
