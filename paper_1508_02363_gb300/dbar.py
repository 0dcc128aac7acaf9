"""ctypes binding of libdbar_gb300.so (include/dbar.h), argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module only
converts arguments.  Device buffers are passed as torch CUDA tensors (torch is
used for device memory and streams), host buffers as numpy arrays.  Importing
this module fails if the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdbar_gb300.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with `python -m paper_1508_02363_gb300.build`")
_lib = ctypes.CDLL(_LIB_PATH)

DBAR_OK, DBAR_EINVAL, DBAR_ENOMEM, DBAR_ENOCONV, DBAR_ETIMEOUT, DBAR_ECUDA, DBAR_EBUSY = range(7)
DBAR_FP64, DBAR_MIXED = 0, 1
DBAR_RESID_DOUBLE_FLOAT, DBAR_RESID_FP64 = 0, 1
DBAR_REG_TAYLOR, DBAR_REG_CONV = 0, 1
STATUS_NAMES = ["DBAR_OK", "DBAR_EINVAL", "DBAR_ENOMEM", "DBAR_ENOCONV", "DBAR_ETIMEOUT", "DBAR_ECUDA",
                "DBAR_EBUSY"]
EXPORTED = ["dbar_params_init", "dbar_last_error", "dbar_plan_create", "dbar_plan_destroy", "dbar_plan_info",
            "dbar_solve_cgo", "dbar_apply", "dbar_rhs", "dbar_m_from_S", "dbar_taylor", "dbar_fft2",
            "dbar_profile_nkinds", "dbar_profile_kind_name", "dbar_profile", "dbar_profile_read",
            "dbar_launch_count", "dbar_fft2_noalloc", "dbar_serve_create", "dbar_serve_submit",
            "dbar_serve_poll", "dbar_serve_wait", "dbar_serve_release", "dbar_serve_stats",
            "dbar_serve_inject_fault", "dbar_serve_destroy", "dbar_plan_tuning", "dbar_reflection",
            "dbar_ds2_potential", "dbar_plan_inject_wait_timeout", "dbar_solve_batches",
            "dbar_plan_row_tuning"]


class dbar_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_double), ("M", ctypes.c_int), ("prec", ctypes.c_int),
                ("restart", ctypes.c_int), ("max_iter", ctypes.c_int), ("tol", ctypes.c_double),
                ("zero_fill", ctypes.c_int), ("max_batch", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("resid_mode", ctypes.c_int), ("graphs", ctypes.c_int),
                ("autotune", ctypes.c_int), ("sstep", ctypes.c_int), ("iterated", ctypes.c_int),
                ("regularisation", ctypes.c_int), ("inner_M", ctypes.c_int), ("gauss_w", ctypes.c_double),
                ("mem_budget", ctypes.c_size_t), ("support_skip", ctypes.c_int), ("row_shape", ctypes.c_int),
                ("row_shape_plain", ctypes.c_int)]


class dbar_request(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_double), ("Q", ctypes.c_void_p), ("k_re", ctypes.c_double),
                ("k_im", ctypes.c_double), ("want_m", ctypes.c_int)]


class dbar_batch(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("Q", ctypes.c_void_p), ("nk", ctypes.c_int), ("k", ctypes.c_void_p),
                ("x0", ctypes.c_void_p), ("S_out", ctypes.c_void_p), ("m_out", ctypes.c_void_p),
                ("iters", ctypes.c_void_p), ("resid", ctypes.c_void_p), ("io_on_device", ctypes.c_int),
                ("status", ctypes.c_int)]


class dbar_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("cycles", ctypes.c_int),
                ("resid", ctypes.c_double), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("S", ctypes.c_void_p), ("m", ctypes.c_void_p)]


class DbarError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


_vp, _dp, _ip, _int, _dbl = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), \
    ctypes.c_int, ctypes.c_double
_lib.dbar_params_init.argtypes = [ctypes.POINTER(dbar_params), _int, _dbl]
_lib.dbar_params_init.restype = None
_lib.dbar_last_error.restype = ctypes.c_char_p
_lib.dbar_plan_create.argtypes = [ctypes.POINTER(dbar_params), ctypes.POINTER(_vp)]
_lib.dbar_plan_destroy.argtypes = [_vp]
_lib.dbar_plan_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t), _ip]
_lib.dbar_solve_cgo.argtypes = [_vp, _vp, _int, _dp, _vp, _vp, _vp, _ip, _dp, _int, _vp]
_lib.dbar_apply.argtypes = [_vp, _vp, _int, _dp, _vp, _vp, _int, _vp]
_lib.dbar_reflection.argtypes = [_vp, _vp, _int, _dp, _dbl, _dp, _ip, _dp, _int, _vp]
_lib.dbar_ds2_potential.argtypes = [_vp, _vp, _dbl, _int, _dp, _dp, _ip, _dp, _int, _vp]
_lib.dbar_rhs.argtypes = [_vp, _vp, _int, _dp, _vp, _vp]
_lib.dbar_m_from_S.argtypes = [_vp, _int, _vp, _vp, _vp]
_lib.dbar_taylor.argtypes = [_vp, _int, _vp, _dp, _int, _vp]
_lib.dbar_fft2.argtypes = [_vp, _int, _vp, _vp, _int, _int, _vp]
_lib.dbar_fft2_noalloc.argtypes = [_int, _int, _vp, _vp, _int, _int, _vp]
_lib.dbar_check_bounded_wait.argtypes = [_int, _int, _dp, _vp]
_lib.dbar_profile_nkinds.argtypes = []
_lib.dbar_profile_kind_name.argtypes = [_int]
_lib.dbar_profile_kind_name.restype = ctypes.c_char_p
_lib.dbar_profile.argtypes = [_vp, _int]
_lib.dbar_profile_read.argtypes = [_vp, _int, _dp, ctypes.POINTER(ctypes.c_longlong), _dp]
_lib.dbar_launch_count.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong)]
_lib.dbar_plan_inject_wait_timeout.argtypes = [_vp]
_lib.dbar_solve_batches.argtypes = [ctypes.POINTER(dbar_batch), _int, _vp]
_lib.dbar_plan_tuning.argtypes = [_vp, _ip, _dp, _ip, _dp]
_lib.dbar_plan_row_tuning.argtypes = [_vp, _ip, _dp]
_u64 = ctypes.c_uint64
_lib.dbar_serve_create.argtypes = [ctypes.POINTER(dbar_params), ctypes.c_size_t, ctypes.POINTER(_vp)]
_lib.dbar_serve_submit.argtypes = [_vp, ctypes.POINTER(dbar_request), ctypes.POINTER(_u64)]
_lib.dbar_serve_poll.argtypes = [_vp, _u64, ctypes.POINTER(dbar_result)]
_lib.dbar_serve_wait.argtypes = [_vp, _u64, ctypes.c_double, ctypes.POINTER(dbar_result)]
_lib.dbar_serve_release.argtypes = [_vp, _u64]
_lib.dbar_serve_stats.argtypes = [_vp, _dp, _dp, _dp, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]
_lib.dbar_serve_inject_fault.argtypes = [_vp]
_lib.dbar_serve_destroy.argtypes = [_vp]
for _f in EXPORTED:
    if _f not in ("dbar_params_init", "dbar_last_error", "dbar_profile_kind_name"):
        getattr(_lib, _f).restype = _int


def _check(st: int, allow=(DBAR_OK,)) -> int:
    if st not in allow:
        raise DbarError(st, _lib.dbar_last_error().decode())
    return st


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(x):
    """Device pointer of a torch tensor or host pointer of a numpy array."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


def _kbuf(k) -> np.ndarray:
    k = np.ascontiguousarray(np.asarray(k, dtype=np.complex128).ravel())
    return k.view(np.float64)


def dbar_params_init(N: int, L: float, **overrides) -> dbar_params:
    p = dbar_params()
    _lib.dbar_params_init(ctypes.byref(p), int(N), float(L))
    for key, v in overrides.items():
        if key == "prec" and isinstance(v, str):
            v = {"fp64": DBAR_FP64, "mixed": DBAR_MIXED}[v]
        if key == "resid_mode" and isinstance(v, str):
            v = {"double_float": DBAR_RESID_DOUBLE_FLOAT, "fp64": DBAR_RESID_FP64}[v]
        if key == "regularisation" and isinstance(v, str):
            v = {"taylor": DBAR_REG_TAYLOR, "conv": DBAR_REG_CONV}[v]
        setattr(p, key, v)
    return p


def dbar_last_error() -> str:
    return _lib.dbar_last_error().decode()


def dbar_plan_create(params: dbar_params) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(_lib.dbar_plan_create(ctypes.byref(params), ctypes.byref(h)))
    return h


def dbar_plan_destroy(plan) -> None:
    _check(_lib.dbar_plan_destroy(plan))


def dbar_plan_info(plan):
    b = ctypes.c_size_t()
    mb = ctypes.c_int()
    _check(_lib.dbar_plan_info(plan, ctypes.byref(b), ctypes.byref(mb)))
    return b.value, mb.value


def dbar_solve_cgo(plan, Q, k, S_out, m_out=None, iters=None, resid=None, io_on_device=None, stream=None,
                   x0=None) -> int:
    """Q, x0, S_out, m_out: numpy complex128 arrays (host) or torch complex128 CUDA tensors.
    x0 (optional): initial guess of S per k.  iters: numpy int32 [nk, 2]; resid:
    numpy float64 [nk].  Returns the status (DBAR_OK or DBAR_ENOCONV); other
    failures raise DbarError."""
    kb = _kbuf(k)
    nk = kb.size // 2
    if io_on_device is None:
        io_on_device = hasattr(Q, "data_ptr")
    ip = iters.ctypes.data_as(_ip) if iters is not None else None
    rp = resid.ctypes.data_as(_dp) if resid is not None else None
    st = _lib.dbar_solve_cgo(plan, _ptr(Q), nk, kb.ctypes.data_as(_dp), _ptr(x0), _ptr(S_out), _ptr(m_out), ip,
                             rp, int(bool(io_on_device)), _stream(stream))
    return _check(st, (DBAR_OK, DBAR_ENOCONV))


def dbar_solve_batches(batches, stream=None):
    """batches: list of dicts with keys plan (a Plan handle), Q, k, S_out and optionally
    m_out, x0, io_on_device (device tensors or host arrays as in dbar_solve_cgo).  Runs the
    batches of different plans concurrently (see include/dbar.h).  Returns (status,
    per-batch statuses, per-batch iters [nk, 2], per-batch resid [nk])."""
    arr = (dbar_batch * len(batches))()
    keep = []
    out_iters, out_resid = [], []
    for i, bt in enumerate(batches):
        kb = _kbuf(bt["k"])
        nk = kb.size // 2
        it = np.zeros((nk, 2), np.int32)
        rs = np.zeros(nk, np.float64)
        keep += [kb, it, rs]
        dev = bt.get("io_on_device", hasattr(bt["Q"], "data_ptr"))
        arr[i] = dbar_batch(bt["plan"].value if hasattr(bt["plan"], "value") else bt["plan"],
                            _ptr(bt["Q"]).value, nk, kb.ctypes.data, _ptr(bt.get("x0")).value if bt.get("x0") is not None
                            else None, _ptr(bt["S_out"]).value, _ptr(bt.get("m_out")).value
                            if bt.get("m_out") is not None else None, it.ctypes.data, rs.ctypes.data, int(bool(dev)), 0)
        out_iters.append(it)
        out_resid.append(rs)
    st = _lib.dbar_solve_batches(arr, len(batches), _stream(stream))
    status = _check(st, (DBAR_OK, DBAR_ENOCONV))
    return status, [arr[i].status for i in range(len(batches))], out_iters, out_resid


def dbar_check_bounded_wait(complete: bool, rounds: int, stream=None) -> float:
    """One bounded mbarrier wait on the device (see include/dbar.h); returns the
    kernel's seconds.  complete=False makes the wait run out: DbarError with
    status DBAR_ETIMEOUT."""
    sec = ctypes.c_double(0.0)
    _check(_lib.dbar_check_bounded_wait(int(bool(complete)), int(rounds), ctypes.byref(sec), _stream(stream)))
    return sec.value


def dbar_reflection(plan, Q, k, t: float = 0.0, q_on_device=None, stream=None):
    """r(k, t) for each k (numpy complex128), plus iters [nk, 2], resid [nk] and the status."""
    kb = _kbuf(k)
    nk = kb.size // 2
    if q_on_device is None:
        q_on_device = hasattr(Q, "data_ptr")
    if not q_on_device:
        Q = np.ascontiguousarray(np.asarray(Q, dtype=np.complex128))
    r = np.zeros(2 * nk, np.float64)
    iters = np.zeros((nk, 2), np.int32)
    resid = np.zeros(nk, np.float64)
    st = _lib.dbar_reflection(plan, _ptr(Q), nk, kb.ctypes.data_as(_dp), float(t), r.ctypes.data_as(_dp),
                              iters.ctypes.data_as(_ip), resid.ctypes.data_as(_dp), int(bool(q_on_device)),
                              _stream(stream))
    status = _check(st, (DBAR_OK, DBAR_ENOCONV))
    return r.view(np.complex128), iters, resid, status


def dbar_ds2_potential(plan, r, z, t: float = 0.0, r_on_device=None, stream=None):
    """q(z, t) at the points z (numpy complex128) from r(k, 0) on the plan's grid, plus
    iters [nz, 2], resid [nz] and the status."""
    zb = _kbuf(z)
    nz = zb.size // 2
    if r_on_device is None:
        r_on_device = hasattr(r, "data_ptr")
    if not r_on_device:
        r = np.ascontiguousarray(np.asarray(r, dtype=np.complex128))
    q = np.zeros(2 * nz, np.float64)
    iters = np.zeros((nz, 2), np.int32)
    resid = np.zeros(nz, np.float64)
    st = _lib.dbar_ds2_potential(plan, _ptr(r), float(t), nz, zb.ctypes.data_as(_dp), q.ctypes.data_as(_dp),
                                 iters.ctypes.data_as(_ip), resid.ctypes.data_as(_dp), int(bool(r_on_device)),
                                 _stream(stream))
    status = _check(st, (DBAR_OK, DBAR_ENOCONV))
    return q.view(np.complex128), iters, resid, status


def dbar_apply(plan, Q, k, S, AS, fp32: bool = False, stream=None) -> None:
    kb = _kbuf(k)
    _check(_lib.dbar_apply(plan, _ptr(Q), kb.size // 2, kb.ctypes.data_as(_dp), _ptr(S), _ptr(AS), int(fp32),
                           _stream(stream)))


def dbar_rhs(plan, Q, k, b, stream=None) -> None:
    kb = _kbuf(k)
    _check(_lib.dbar_rhs(plan, _ptr(Q), kb.size // 2, kb.ctypes.data_as(_dp), _ptr(b), _stream(stream)))


def dbar_m_from_S(plan, nk: int, S, m, stream=None) -> None:
    _check(_lib.dbar_m_from_S(plan, int(nk), _ptr(S), _ptr(m), _stream(stream)))


def dbar_taylor(plan, nk: int, S, M: int, fp32: bool = False, stream=None) -> np.ndarray:
    out = np.zeros((nk, M + 2), dtype=np.complex128)
    _check(_lib.dbar_taylor(plan, int(nk), _ptr(S), out.view(np.float64).ctypes.data_as(_dp), int(fp32),
                            _stream(stream)))
    return out


def dbar_fft2(plan, nk: int, x, y, sign: int, fp32: bool = False, stream=None) -> None:
    _check(_lib.dbar_fft2(plan, int(nk), _ptr(x), _ptr(y), int(sign), int(fp32), _stream(stream)))


def dbar_fft2_noalloc(N: int, nk: int, x, y, sign: int, fp32: bool = False, stream=None) -> None:
    """2-D DFT without any device allocation (library-owned 16 MiB scratch); see include/dbar.h."""
    _check(_lib.dbar_fft2_noalloc(int(N), int(nk), _ptr(x), _ptr(y), int(sign), int(fp32), _stream(stream)))


def dbar_profile_nkinds() -> int:
    return _lib.dbar_profile_nkinds()


def dbar_profile_kind_name(kind: int) -> str:
    return _lib.dbar_profile_kind_name(int(kind)).decode()


def dbar_profile(plan, enable: bool) -> None:
    _check(_lib.dbar_profile(plan, int(bool(enable))))


def dbar_profile_read(plan, kind: int):
    ms, n, by = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
    _check(_lib.dbar_profile_read(plan, int(kind), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by)))
    return ms.value, n.value, by.value


COLUMN_VARIANTS = 3
ROW_VARIANTS = 5


def dbar_plan_tuning(plan):
    """(column-pass tile variant in use, [ms per launch of each variant])."""
    v, ms = ctypes.c_int(), (ctypes.c_double * COLUMN_VARIANTS)()
    _check(_lib.dbar_plan_tuning(plan, ctypes.byref(v), ms, None, None))
    return v.value, list(ms)


def dbar_plan_row_tuning(plan, passes: str = "fused"):
    """passes "fused": (shape of the fused chain row pass, [ms per launch of each shape]),
    from dbar_plan_tuning; "plain": (shape of the row passes A and C, [ms per A + C pair of
    each shape]), from dbar_plan_row_tuning."""
    v, ms = ctypes.c_int(), (ctypes.c_double * ROW_VARIANTS)()
    if passes == "fused":
        _check(_lib.dbar_plan_tuning(plan, None, None, ctypes.byref(v), ms))
    elif passes == "plain":
        _check(_lib.dbar_plan_row_tuning(plan, ctypes.byref(v), ms))
    else:
        raise ValueError("passes must be 'fused' or 'plain'")
    return v.value, list(ms)


def dbar_plan_inject_wait_timeout(plan) -> None:
    """Test hook: the plan's next block-update launch cannot complete its first bulk-copy
    stage, so its bounded waits run out and the solve returns DBAR_ETIMEOUT."""
    _check(_lib.dbar_plan_inject_wait_timeout(plan))


def dbar_launch_count(plan) -> int:
    c = ctypes.c_longlong()
    _check(_lib.dbar_launch_count(plan, ctypes.byref(c)))
    return c.value


def profile_table(plan) -> dict:
    """{kind name: (ms, launches, algorithmic bytes)} for every kernel kind."""
    return {dbar_profile_kind_name(i): dbar_profile_read(plan, i) for i in range(dbar_profile_nkinds())}


class Plan:
    """Owning wrapper: Plan(N, L, M=2, prec='mixed', ...) -> .solve(Q, k)."""

    def __init__(self, N: int, L: float, **params):
        self.params = dbar_params_init(N, L, **params)
        self.N, self.L, self.M = N, L, self.params.M
        self.handle = dbar_plan_create(self.params)
        self.device_bytes, self.max_batch = dbar_plan_info(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            dbar_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, Q, k, want_m: bool = True, stream=None, x0=None):
        """Host in, host out: returns dict(S, m, iters, resid, status).  x0: optional
        initial guess of S ([nk, N, N] complex128), e.g. the S of an interrupted solve."""
        k = np.atleast_1d(np.asarray(k, dtype=np.complex128))
        nk, N = k.size, self.N
        Q = np.ascontiguousarray(np.asarray(Q, dtype=np.complex128).reshape(N, N))
        if x0 is not None:
            x0 = np.ascontiguousarray(np.asarray(x0, dtype=np.complex128).reshape(nk, N, N))
        S = np.zeros((nk, N, N), np.complex128)
        m = np.zeros((nk, N, N), np.complex128) if want_m else None
        iters = np.zeros((nk, 2), np.int32)
        resid = np.zeros(nk, np.float64)
        st = dbar_solve_cgo(self.handle, Q, k, S, m, iters, resid, io_on_device=False, stream=stream, x0=x0)
        return {"S": S, "m": m, "iters": iters, "resid": resid, "status": st}

    def solve_device(self, Q, k, S_out, m_out=None, stream=None, x0=None):
        """Device in, device out (torch complex128 CUDA tensors; x0 optional)."""
        k = np.atleast_1d(np.asarray(k, dtype=np.complex128))
        iters = np.zeros((k.size, 2), np.int32)
        resid = np.zeros(k.size, np.float64)
        st = dbar_solve_cgo(self.handle, Q, k, S_out, m_out, iters, resid, io_on_device=True, stream=stream, x0=x0)
        return {"iters": iters, "resid": resid, "status": st}


# ----------------------------------------------------------------------------- serving

def dbar_serve_create(params: dbar_params, mem_budget: int):
    h = ctypes.c_void_p()
    _check(_lib.dbar_serve_create(ctypes.byref(params), ctypes.c_size_t(int(mem_budget)), ctypes.byref(h)))
    return h


def dbar_serve_submit(srv, N: int, L: float, Q, k: complex, want_m: bool = False) -> int:
    Q = np.ascontiguousarray(np.asarray(Q, dtype=np.complex128).reshape(N, N))
    rq = dbar_request(int(N), float(L), Q.ctypes.data, float(np.real(k)), float(np.imag(k)), int(bool(want_m)))
    t = ctypes.c_uint64()
    _check(_lib.dbar_serve_submit(srv, ctypes.byref(rq), ctypes.byref(t)))
    return t.value


def _result_dict(res: dbar_result, N: int, copy: bool = True):
    def arr(p):
        if not p or not copy:
            return None
        buf = (ctypes.c_double * (2 * N * N)).from_address(p)
        return np.frombuffer(buf, dtype=np.float64).view(np.complex128).reshape(N, N).copy()
    return {"status": res.status, "iters": res.iters, "cycles": res.cycles, "resid": res.resid,
            "latency_ms": res.latency_ms, "queue_ms": res.queue_ms, "run_ms": res.run_ms,
            "S": arr(res.S), "m": arr(res.m)}


def dbar_serve_poll(srv, ticket: int, N: int, copy: bool = True):
    """None while the request runs; else its result (copy=False leaves S and m out)."""
    res = dbar_result()
    st = _check(_lib.dbar_serve_poll(srv, ticket, ctypes.byref(res)), (DBAR_OK, DBAR_EBUSY))
    return None if st == DBAR_EBUSY else _result_dict(res, N, copy)


def dbar_serve_wait(srv, ticket: int, N: int, timeout_s: float = -1.0, copy: bool = True):
    """Blocks until the request is done; copy=False leaves S and m out of the dict."""
    res = dbar_result()
    _check(_lib.dbar_serve_wait(srv, ticket, float(timeout_s), ctypes.byref(res)))
    return _result_dict(res, N, copy)


def dbar_serve_release(srv, ticket: int) -> None:
    _check(_lib.dbar_serve_release(srv, ticket))


def dbar_serve_stats(srv) -> dict:
    p50, p99, rate = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    done, pend = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.dbar_serve_stats(srv, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(rate), ctypes.byref(done),
                                 ctypes.byref(pend)))
    return {"p50_ms": p50.value, "p99_ms": p99.value, "solves_per_s": rate.value, "completed": done.value,
            "pending": pend.value}


def dbar_serve_inject_fault(srv) -> None:
    _check(_lib.dbar_serve_inject_fault(srv))


def dbar_serve_destroy(srv) -> None:
    _check(_lib.dbar_serve_destroy(srv))


class Server:
    """Continuous-batching CGO server: Server(mem_budget, **solver params)."""

    def __init__(self, mem_budget: int, **params):
        self.params = dbar_params_init(64, 1.0, **params)
        self.handle = dbar_serve_create(self.params, mem_budget)
        self._N = {}

    def submit(self, N: int, L: float, Q, k: complex, want_m: bool = False) -> int:
        t = dbar_serve_submit(self.handle, N, L, Q, k, want_m)
        self._N[t] = N
        return t

    def poll(self, ticket: int, copy: bool = True):
        return dbar_serve_poll(self.handle, ticket, self._N[ticket], copy)

    def wait(self, ticket: int, timeout_s: float = -1.0, release: bool = True, copy: bool = True):
        r = dbar_serve_wait(self.handle, ticket, self._N[ticket], timeout_s, copy)
        if release:
            self.release(ticket)
        return r

    def release(self, ticket: int) -> None:
        dbar_serve_release(self.handle, ticket)
        self._N.pop(ticket, None)

    def stats(self) -> dict:
        return dbar_serve_stats(self.handle)

    def inject_fault(self) -> None:
        dbar_serve_inject_fault(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            dbar_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
