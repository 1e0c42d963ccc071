"""Python binding of librnmf.so: randomized HALS NMF on GB300 (sm_103a).

Erichson, Mendible, Wihlborn, Kutz, "Randomized Nonnegative Matrix
Factorization" (arXiv:1711.02037): randomized QB (Section 2.3) followed by
compressed HALS sweeps (Section 3.2, Algorithm 1), plus deterministic HALS
(Section 3.1).  Every step runs in the CUDA library behind the C ABI declared
in include/rnmf.h; this module only marshals arguments (device pointers of
torch tensors, the current CUDA stream) and raises on a non-OK status.  There is
no CPU fallback: importing works without a GPU, but every compute call needs the
built library and a CUDA device.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librnmf.so")

PREC_FP32, PREC_BF16, PREC_SPLIT3 = 0, 1, 2
ORDER_CYCLIC, ORDER_SHUFFLED, ORDER_INTERLEAVED = 0, 1, 2
INIT_UNIFORM, INIT_SVD = 0, 1
SWEEP_FP32, SWEEP_SPLIT3 = 0, 1
_CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy
STATUS = {0: "RNMF_OK", 1: "RNMF_EINVAL", 2: "RNMF_ENOMEM", 3: "RNMF_ECUDA", 4: "RNMF_ENOTPD",
          5: "RNMF_ETIMEOUT", 6: "RNMF_ENOTIMPL"}

# name -> (restype, argtypes) of every entry point declared in include/rnmf.h
_i64, _int, _u64, _vp, _dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_double


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("gram_mode", ctypes.c_int), ("omega_dist", ctypes.c_int),
                ("track_every", ctypes.c_int), ("spin_limit", ctypes.c_longlong), ("alpha_W", ctypes.c_float),
                ("alpha_H", ctypes.c_float), ("beta_W", ctypes.c_float), ("beta_H", ctypes.c_float),
                ("pg_tol", ctypes.c_double), ("pg_every", ctypes.c_int), ("order", ctypes.c_int),
                ("order_seed", ctypes.c_uint64), ("init", ctypes.c_int), ("sweep_products", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("rel_err_hist", ctypes.POINTER(ctypes.c_double)), ("final_rel_err", ctypes.c_double),
                ("ms_qb", ctypes.c_float), ("ms_sweeps", ctypes.c_float), ("sweeps_done", ctypes.c_int),
                ("pg_ratio", ctypes.c_double), ("obj_hist", ctypes.POINTER(ctypes.c_double)),
                ("obj_half_hist", ctypes.POINTER(ctypes.c_double))]


class KernelProf(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class Problem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("k", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int), ("iters", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("instance", ctypes.c_uint32), ("W", ctypes.c_void_p),
                ("H", ctypes.c_void_p)]


class BatchStats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_float), ("tuned", ctypes.c_int), ("graph_kernels", ctypes.c_int),
                ("cluster_count", ctypes.c_int * 4), ("threads_small", ctypes.c_int), ("failed", ctypes.c_int),
                ("tune_ms", ctypes.c_float * 8)]


SIGNATURES = {
    "rnmf_create": (_int, [ctypes.POINTER(_vp), _int, _vp]),
    "rnmf_destroy": (_int, [_vp]),
    "rnmf_default_opts": (None, [ctypes.POINTER(Opts)]),
    "rnmf": (_int, [_vp, _vp, _i64, _i64, _i64, _int, _int, _int, _int, _u64, ctypes.POINTER(Opts), _vp, _vp,
                    ctypes.POINTER(Stats)]),
    "rnmf_host": (_int, [_vp, _vp, _i64, _i64, _i64, _int, _int, _int, _int, _u64, ctypes.POINTER(Opts), _vp,
                         _vp, ctypes.POINTER(Stats)]),
    "rnmf_hals": (_int, [_vp, _vp, _i64, _i64, _i64, _int, _int, _u64, ctypes.POINTER(Opts), _vp, _vp,
                         ctypes.POINTER(Stats)]),
    "rnmf_qb": (_int, [_vp, _vp, _i64, _i64, _i64, _int, _int, _u64, ctypes.POINTER(Opts), _vp, _vp]),
    "rnmf_sweeps": (_int, [_vp, _vp, _vp, _i64, _i64, _int, _int, _int, ctypes.POINTER(Opts), _vp, _vp, _vp, _vp,
                           _i64, ctypes.POINTER(Stats)]),
    "rnmf_sketch": (_int, [_vp, _vp, _i64, _i64, _i64, _vp, _int, _int, _int, _vp]),
    "rnmf_omega": (_int, [_vp, _i64, _int, _u64, _int, _vp]),
    "rnmf_init_factors": (_int, [_vp, _i64, _i64, _int, _u64, _vp, _vp]),
    "rnmf_rel_err": (_int, [_vp, _vp, _i64, _i64, _i64, _vp, _vp, _int, ctypes.POINTER(_dbl)]),
    "rnmf_qb_streamed": (_int, [_vp, _vp, _i64, _i64, _i64, _int, _int, _u64, ctypes.POINTER(Opts), _i64, _vp, _vp]),
    "rnmf_streamed": (_int, [_vp, _vp, _i64, _i64, _i64, _int, _int, _int, _int, _u64, ctypes.POINTER(Opts), _i64,
                             _vp, _vp, ctypes.POINTER(Stats)]),
    "rnmf_projected_gradient": (_int, [_vp, _vp, _vp, _i64, _i64, _int, _int, _vp, _vp, ctypes.POINTER(_dbl)]),
    "rnmf_ckpt_floats": (ctypes.c_size_t, [_i64, _i64, _int, _int, _int]),
    "rnmf_sweeps_fwd": (_int, [_vp, _vp, _vp, _i64, _i64, _int, _int, _int, ctypes.POINTER(Opts), _vp, _vp, _vp]),
    "rnmf_sweeps_bwd": (_int, [_vp, _vp, _vp, _i64, _i64, _int, _int, _int, ctypes.POINTER(Opts), _vp, _vp, _vp,
                               _vp, _vp, _vp]),
    "rnmf_dA": (_int, [_vp, _vp, _vp, _i64, _i64, _int, _vp]),
    "rnmf_rel_err_noalloc": (_int, [_vp, _vp, _i64, _i64, _i64, _vp, _vp, _int, ctypes.POINTER(_dbl)]),
    "rnmf_batched": (_int, [_vp, ctypes.POINTER(Problem), _int, ctypes.POINTER(Opts), ctypes.POINTER(_int),
                            ctypes.POINTER(BatchStats)]),
    "rnmf_batched_config": (_int, [_vp, _int, _int]),
    "rnmf_batched_rel_err": (_int, [_vp, ctypes.POINTER(Problem), _int, ctypes.POINTER(_dbl)]),
    "rnmf_set_scratch_limit": (_int, [_vp, ctypes.c_size_t]),
    "rnmf_scratch_bytes": (ctypes.c_size_t, [_vp]),
    "rnmf_last_error": (ctypes.c_char_p, [_vp]),
    "rnmf_kernel_launches": (ctypes.c_longlong, [_vp]),
    "rnmf_profile": (_int, [_vp, _int]),
    "rnmf_profile_read": (_int, [_vp, ctypes.POINTER(KernelProf), _int]),
}

_lib = None


class RnmfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load librnmf.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                               f"g.build()'` (or python -m paper_1711_02037_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().rnmf_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@dataclass
class RunStats:
    ms_qb: float = 0.0
    ms_sweeps: float = 0.0
    sweeps_done: int = 0
    final_rel_err: float = -1.0
    rel_err_hist: list = field(default_factory=list)
    pg_ratio: float = -1.0
    obj_hist: list = field(default_factory=list)       # f~ = ||B - W~ H||^2 after each sweep
    obj_half_hist: list = field(default_factory=list)  # f~ after each sweep's H half


def _torch():
    import torch
    return torch


class Context:
    """An rnmf_ctx bound to a CUDA device and (by default) torch's current stream."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1711_02037_gb300 needs a CUDA device (no CPU fallback)")
        torch.cuda.set_device(device)
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.device = device
        h = _vp()
        # torch's default stream is CUDA's legacy default stream (handle 0); pass it
        # as cudaStreamLegacy, since a NULL handle asks the library for a stream of
        # its own, which would not be ordered after torch's work on the default stream
        handle = stream.cuda_stream if stream.cuda_stream else _CUDA_STREAM_LEGACY
        self._check(lib().rnmf_create(ctypes.byref(h), device, _vp(handle)), None)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().rnmf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, h):
        if st != 0:
            msg = lib().rnmf_last_error(h).decode() if h else ""
            raise RnmfError(st, msg)

    def launches(self) -> int:
        return int(lib().rnmf_kernel_launches(self.h))

    def set_scratch_limit(self, nbytes: int):
        """Cap the device scratch this context may hold (0: no cap); calls that
        would need more raise RnmfError(RNMF_ENOMEM) before any work."""
        self._check(lib().rnmf_set_scratch_limit(self.h, int(nbytes)), self.h)

    def scratch_bytes(self) -> int:
        return int(lib().rnmf_scratch_bytes(self.h))

    def profile(self, on: bool):
        """Start (reset) or stop per-kernel-class event timing of this context's launches."""
        self._check(lib().rnmf_profile(self.h, 1 if on else 0), self.h)

    def profile_read(self) -> dict:
        """{kernel class: dict(launches, ms, bytes, flops)} of the launches timed so far."""
        buf = (KernelProf * 32)()
        n = lib().rnmf_profile_read(self.h, buf, 32)
        return {buf[i].name.decode(): dict(launches=buf[i].launches, ms=buf[i].ms, bytes=buf[i].bytes,
                                           flops=buf[i].flops) for i in range(n)}

    # ------------------------------------------------------------ helpers
    @staticmethod
    def _mat(A):
        torch = _torch()
        assert A.dtype == torch.float32 and A.is_cuda and A.dim() == 2 and A.stride(1) == 1
        return A.data_ptr(), A.shape[0], A.shape[1], A.stride(0)

    def _empty(self, *shape):
        torch = _torch()
        return torch.empty(*shape, dtype=torch.float32, device=f"cuda:{self.device}")

    @staticmethod
    def _stats_in(track_obj: bool, iters: int):
        """Stats with host arrays for the per-sweep compressed objective when asked for."""
        s = Stats()
        bufs = None
        if track_obj:
            bufs = ((ctypes.c_double * max(iters, 1))(), (ctypes.c_double * max(iters, 1))())
            s.obj_hist, s.obj_half_hist = bufs
        return s, bufs

    @staticmethod
    def _stats_out(s: Stats, hist_buf, ntrack, obj_bufs=None) -> RunStats:
        r = RunStats(s.ms_qb, s.ms_sweeps, s.sweeps_done, s.final_rel_err,
                     list(hist_buf[:ntrack]) if hist_buf is not None else [], s.pg_ratio)
        if obj_bufs is not None:
            r.obj_hist = list(obj_bufs[0][:s.sweeps_done])
            r.obj_half_hist = list(obj_bufs[1][:s.sweeps_done])
        return r

    # ------------------------------------------------------------ calls
    def rnmf(self, A, k: int, p: int, q: int, iters: int, seed: int = 0, precision: int = PREC_FP32,
             gram_mode: int = 0, omega_dist: int = 0, track_every: int = 0, spin_limit: int = 0, W=None, H=None,
             track_obj: bool = False, **penalties):
        """Randomized HALS (Algorithm 1). Returns (W, H, RunStats).  Extra options:
        alpha_W, alpha_H, beta_W, beta_H (Section 3.4), pg_tol, pg_every (Section 3.3
        stopping rule), order, order_seed (ORDER_SHUFFLED / ORDER_INTERLEAVED: the
        update orders of Section 3.2) and init (INIT_SVD: NNDSVD of the randomized
        SVD), see rnmf_opts.  track_obj: per-sweep compressed objective in
        RunStats.obj_hist / obj_half_hist."""
        a, m, n, lda = self._mat(A)
        W = self._empty(m, k) if W is None else W
        H = self._empty(k, n) if H is None else H
        o = default_opts(precision=precision, gram_mode=gram_mode, omega_dist=omega_dist,
                         track_every=track_every, spin_limit=spin_limit, **penalties)
        ntrack = iters // track_every if track_every > 0 else 0
        hist = (ctypes.c_double * max(ntrack, 1))()
        s, ob = self._stats_in(track_obj, iters)
        s.rel_err_hist = hist
        self._check(lib().rnmf(self.h, a, m, n, lda, k, p, q, iters, seed, ctypes.byref(o), W.data_ptr(),
                               H.data_ptr(), ctypes.byref(s)), self.h)
        return W, H, self._stats_out(s, hist, ntrack, ob)

    def rnmf_host(self, A_host, k: int, p: int, q: int, iters: int, seed: int = 0, precision: int = PREC_FP32,
                  gram_mode: int = 0, W_host=None, H_host=None, **options):
        """rnmf with A, W, H in host memory (numpy float32 arrays or CPU tensors, pinned or not)."""
        import numpy as np
        A_np = A_host.numpy() if hasattr(A_host, "numpy") else A_host
        assert A_np.dtype == np.float32 and A_np.strides[1] == 4
        m, n = A_np.shape
        lda = A_np.strides[0] // 4
        W_host = np.empty((m, k), np.float32) if W_host is None else W_host
        H_host = np.empty((k, n), np.float32) if H_host is None else H_host
        Wn = W_host.numpy() if hasattr(W_host, "numpy") else W_host
        Hn = H_host.numpy() if hasattr(H_host, "numpy") else H_host
        o = default_opts(precision=precision, gram_mode=gram_mode, **options)
        s = Stats()
        self._check(lib().rnmf_host(self.h, A_np.ctypes.data, m, n, lda, k, p, q, iters, seed, ctypes.byref(o),
                                    Wn.ctypes.data, Hn.ctypes.data, ctypes.byref(s)), self.h)
        return W_host, H_host, self._stats_out(s, None, 0)

    def hals(self, A, k: int, iters: int, seed: int = 0, track_every: int = 0, W=None, H=None, **penalties):
        """Deterministic HALS (Section 3.1; with penalties Section 3.4) from the same
        initial factors. Returns (W, H, RunStats)."""
        a, m, n, lda = self._mat(A)
        W = self._empty(m, k) if W is None else W
        H = self._empty(k, n) if H is None else H
        o = default_opts(track_every=track_every, **penalties)
        ntrack = iters // track_every if track_every > 0 else 0
        hist = (ctypes.c_double * max(ntrack, 1))()
        s = Stats()
        s.rel_err_hist = hist
        self._check(lib().rnmf_hals(self.h, a, m, n, lda, k, iters, seed, ctypes.byref(o), W.data_ptr(),
                                    H.data_ptr(), ctypes.byref(s)), self.h)
        return W, H, self._stats_out(s, hist, ntrack)

    def qb(self, A, l: int, q: int, seed: int = 0, precision: int = PREC_FP32, omega_dist: int = 0):
        """Randomized QB (Section 2.3). Returns (Q (m x l), Bt = B^T (n x l))."""
        a, m, n, lda = self._mat(A)
        Q = self._empty(m, l)
        Bt = self._empty(n, l)
        o = default_opts(precision=precision, omega_dist=omega_dist)
        self._check(lib().rnmf_qb(self.h, a, m, n, lda, l, q, seed, ctypes.byref(o), Q.data_ptr(), Bt.data_ptr()),
                    self.h)
        return Q, Bt

    def sweeps(self, Q, Bt, W, H, iters: int, Wt=None, gram_mode: int = 0, A=None, track_every: int = 0,
               track_obj: bool = False, **penalties):
        """Compressed HALS sweeps in place on W (m x k), H (k x n) and optional Wt (l x k)."""
        m, l = Q.shape
        n = Bt.shape[0]
        k = W.shape[1]
        o = default_opts(gram_mode=gram_mode, track_every=track_every, **penalties)
        ntrack = iters // track_every if track_every > 0 else 0
        hist = (ctypes.c_double * max(ntrack, 1))()
        s, ob = self._stats_in(track_obj, iters)
        s.rel_err_hist = hist
        a, lda = (A.data_ptr(), A.stride(0)) if A is not None else (None, n)
        self._check(lib().rnmf_sweeps(self.h, Q.data_ptr(), Bt.data_ptr(), m, n, l, k, iters, ctypes.byref(o),
                                      W.data_ptr(), H.data_ptr(), Wt.data_ptr() if Wt is not None else None, a, lda,
                                      ctypes.byref(s)), self.h)
        return W, H, self._stats_out(s, hist, ntrack, ob)

    def sweeps_fwd(self, Q, Bt, W, H, T: int, gram_mode: int = 0, checkpoint: bool = True):
        """T sweeps in place on W (m x k, W_init -> W_T) and H (k x n), W~ = Q^T W_init.
        Returns (W, H, ckpt) with ckpt the (T + 1) sweep-boundary states (or None)."""
        torch = _torch()
        m, l = Q.shape
        n, k = Bt.shape[0], W.shape[1]
        ck = None
        if checkpoint:
            ck = torch.empty(int(lib().rnmf_ckpt_floats(m, n, l, k, T)), dtype=torch.float32, device=Q.device)
        o = default_opts(gram_mode=gram_mode)
        self._check(lib().rnmf_sweeps_fwd(self.h, Q.data_ptr(), Bt.data_ptr(), m, n, l, k, T, ctypes.byref(o),
                                          W.data_ptr(), H.data_ptr(), ck.data_ptr() if ck is not None else None),
                    self.h)
        return W, H, ck

    def sweeps_bwd(self, Q, Bt, ckpt, dW, dH, T: int, gram_mode: int = 0):
        """Reverse pass of sweeps_fwd: returns (dBt (n x l), dW_init (m x k), dH_init (k x n))."""
        m, l = Q.shape
        n, k = Bt.shape[0], dW.shape[1]
        dBt, dW0, dH0 = self._empty(n, l), self._empty(m, k), self._empty(k, n)
        o = default_opts(gram_mode=gram_mode)
        self._check(lib().rnmf_sweeps_bwd(self.h, Q.data_ptr(), Bt.data_ptr(), m, n, l, k, T, ctypes.byref(o),
                                          ckpt.data_ptr(), dW.data_ptr(), dH.data_ptr(), dBt.data_ptr(),
                                          dW0.data_ptr(), dH0.data_ptr()), self.h)
        return dBt, dW0, dH0

    @staticmethod
    def _host(A_host):
        import numpy as np
        A_np = A_host.numpy() if hasattr(A_host, "numpy") else A_host
        assert A_np.dtype == np.float32 and A_np.strides[1] == 4
        return A_np, A_np.shape[0], A_np.shape[1], A_np.strides[0] // 4

    def qb_streamed(self, A_host, l: int, q: int, seed: int = 0, block_cols: int = 0, omega_dist: int = 0,
                    precision: int = PREC_FP32):
        """Column-blocked QB (Algorithm 2) of a host matrix. Returns device (Q, Bt)."""
        A_np, m, n, lda = self._host(A_host)
        Q, Bt = self._empty(m, l), self._empty(n, l)
        o = default_opts(omega_dist=omega_dist, precision=precision)
        self._check(lib().rnmf_qb_streamed(self.h, A_np.ctypes.data, m, n, lda, l, q, seed, ctypes.byref(o),
                                           block_cols, Q.data_ptr(), Bt.data_ptr()), self.h)
        return Q, Bt

    def rnmf_streamed(self, A_host, k: int, p: int, q: int, iters: int, seed: int = 0, block_cols: int = 0,
                      gram_mode: int = 0, W=None, H=None, track_obj: bool = False, **options):
        """rnmf with A in host memory, QB by column blocks (Algorithm 2). Returns (W, H, RunStats)."""
        A_np, m, n, lda = self._host(A_host)
        W = self._empty(m, k) if W is None else W
        H = self._empty(k, n) if H is None else H
        o = default_opts(gram_mode=gram_mode, **options)
        s, ob = self._stats_in(track_obj, iters)
        self._check(lib().rnmf_streamed(self.h, A_np.ctypes.data, m, n, lda, k, p, q, iters, seed, ctypes.byref(o),
                                        block_cols, W.data_ptr(), H.data_ptr(), ctypes.byref(s)), self.h)
        return W, H, self._stats_out(s, None, 0, ob)

    def projected_gradient(self, Q, Bt, W, H) -> float:
        """||grad^P||_F^2 of the compressed problem (Section 3.3) at (W, H)."""
        m, l = Q.shape
        n, k = Bt.shape[0], W.shape[1]
        out = ctypes.c_double()
        self._check(lib().rnmf_projected_gradient(self.h, Q.data_ptr(), Bt.data_ptr(), m, n, l, k, W.data_ptr(),
                                                  H.data_ptr(), ctypes.byref(out)), self.h)
        return out.value

    def dA(self, Q, dBt):
        """dL/dA = Q dL/dB for B = Q^T A (m x n)."""
        m, l = Q.shape
        n = dBt.shape[0]
        out = self._empty(m, n)
        self._check(lib().rnmf_dA(self.h, Q.data_ptr(), dBt.data_ptr(), m, n, l, out.data_ptr()), self.h)
        return out

    # ------------------------------------------------------------ batches
    @staticmethod
    def _problems(items):
        """items: list of dicts with A (m x n device tensor, row stride lda), k, p, q,
        iters, seed, instance, W (m x k), H (k x n)."""
        arr = (Problem * len(items))()
        for i, it in enumerate(items):
            A = it["A"]
            arr[i] = Problem(A.data_ptr(), A.shape[0], A.shape[1], A.stride(0), it["k"], it["p"], it["q"],
                             it["iters"], it.get("seed", 0), it.get("instance", 0), it["W"].data_ptr(),
                             it["H"].data_ptr())
        return arr

    def batched(self, items, gram_mode: int = 0, omega_dist: int = 0):
        """Runs every problem of `items` (see _problems); W and H are written in place.
        Returns (per-problem status list, stats dict)."""
        arr = self._problems(items)
        st = (ctypes.c_int * len(items))()
        bs = BatchStats()
        o = default_opts(gram_mode=gram_mode, omega_dist=omega_dist)
        self._check(lib().rnmf_batched(self.h, arr, len(items), ctypes.byref(o), st, ctypes.byref(bs)), self.h)
        return list(st), dict(ms=bs.ms, tuned=bs.tuned, graph_kernels=bs.graph_kernels,
                              cluster_count=list(bs.cluster_count), threads_small=bs.threads_small,
                              failed=bs.failed, tune_ms=list(bs.tune_ms))

    def batched_config(self, max_cluster: int = 0, threads_small: int = 0):
        self._check(lib().rnmf_batched_config(self.h, max_cluster, threads_small), self.h)

    def batched_rel_err(self, items) -> list:
        arr = self._problems(items)
        out = (ctypes.c_double * len(items))()
        self._check(lib().rnmf_batched_rel_err(self.h, arr, len(items), out), self.h)
        return list(out)

    def sketch(self, A, X, transpose: bool = False, form: int = PREC_FP32):
        """Y = A X (transpose False, X n x l) or Z = A^T X (transpose True, X m x l)."""
        a, m, n, lda = self._mat(A)
        l = X.shape[1]
        out = self._empty(n if transpose else m, l)
        self._check(lib().rnmf_sketch(self.h, a, m, n, lda, X.data_ptr(), l, 1 if transpose else 0, form,
                                      out.data_ptr()), self.h)
        return out

    def omega(self, n: int, l: int, seed: int = 0, dist: int = 0):
        Om = self._empty(n, l)
        self._check(lib().rnmf_omega(self.h, n, l, seed, dist, Om.data_ptr()), self.h)
        return Om

    def init_factors(self, m: int, n: int, k: int, seed: int = 0):
        W = self._empty(m, k)
        H = self._empty(k, n)
        self._check(lib().rnmf_init_factors(self.h, m, n, k, seed, W.data_ptr(), H.data_ptr()), self.h)
        return W, H

    def rel_err(self, A, W, H) -> float:
        a, m, n, lda = self._mat(A)
        out = ctypes.c_double()
        self._check(lib().rnmf_rel_err(self.h, a, m, n, lda, W.data_ptr(), H.data_ptr(), W.shape[1],
                                       ctypes.byref(out)), self.h)
        return out.value

    def rel_err_noalloc(self, A, W, H) -> float:
        """rel_err with the library's fixed device scratch: no device allocation
        (for callers whose device memory is all taken or who cannot take the
        synchronisation of an allocation).  Calls on one device must not overlap."""
        a, m, n, lda = self._mat(A)
        out = ctypes.c_double()
        self._check(lib().rnmf_rel_err_noalloc(self.h, a, m, n, lda, W.data_ptr(), H.data_ptr(), W.shape[1],
                                               ctypes.byref(out)), self.h)
        return out.value


# ---------------------------------------------------------------- autograd
def _sweeps_function():
    torch = _torch()

    class RHalsSweeps(torch.autograd.Function):
        """(W_T, H_T) after T compressed sweeps from (W_init, H_init) on B = Q^T A, Q fixed.

        Forward keeps the T + 1 sweep-boundary states; backward recomputes each
        sweep's products from its two boundary states and runs the reverse of
        the H-row and W~-column updates in the library (subgradient 0 at a
        clamp argument of exactly 0)."""

        @staticmethod
        def forward(fctx, A, Q, W0, H0, T, gram_mode, cx):
            Bt = cx.sketch(A, Q, transpose=True)
            W, H, ck = cx.sweeps_fwd(Q, Bt, W0.detach().clone(), H0.detach().clone(), T, gram_mode)
            fctx.save_for_backward(Q, Bt, ck)
            fctx.T, fctx.gram_mode, fctx.cx = T, gram_mode, cx
            return W, H

        @staticmethod
        def backward(fctx, gW, gH):
            Q, Bt, ck = fctx.saved_tensors
            m, k = Q.shape[0], gW.shape[1] if gW is not None else gH.shape[0]
            n = Bt.shape[0]
            gW = gW.contiguous() if gW is not None else torch.zeros(m, k, device=Q.device)
            gH = gH.contiguous() if gH is not None else torch.zeros(k, n, device=Q.device)
            dBt, dW0, dH0 = fctx.cx.sweeps_bwd(Q, Bt, ck, gW, gH, fctx.T, fctx.gram_mode)
            dA = fctx.cx.dA(Q, dBt) if fctx.needs_input_grad[0] else None
            return dA, None, dW0, dH0, None, None, None

    return RHalsSweeps


_FN = None


def rhals_sweeps(cx: Context, A, Q, W0, H0, T: int, gram_mode: int = 0):
    """Differentiable T compressed HALS sweeps: returns (W_T, H_T); gradients reach
    A (through B = Q^T A), W0 and H0.  All tensors float32, contiguous, on cx's device."""
    global _FN
    if _FN is None:
        _FN = _sweeps_function()
    return _FN.apply(A, Q, W0, H0, T, gram_mode, cx)
