"""Seeded synthetic inputs for randomized HALS NMF (test and benchmark infrastructure).

The generators live in ``synth.c`` (plain C, OpenMP) and are pure functions of
(seed, stream, instance, element index); see that file for the exact recipe.
This module only makes inputs; it contains none of the method's arithmetic and
is imported by the tests and the benchmark, never by the library itself.

Workloads (Section 4.4 synthetic experiments, and the differentiation and
batching workloads built on the same recipe) are described by ``Workload``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None

STREAM_W0, STREAM_H0, STREAM_NOISE, STREAM_MASK, STREAM_G, STREAM_SHAPES = 4, 5, 6, 7, 8, 9
DATA_SEED = 12345  # key of every generated data matrix
G_SEED = 2         # key of the cotangent G of the differentiation workload


def build(force: bool = False) -> str:
    """Compile libsynth.so in place (gcc, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        i64, u64, u32, i32, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_double
        vp = ctypes.c_void_p
        L.synth_philox4x32_10.argtypes = [vp, vp, vp]
        L.synth_ln_export.argtypes = [dbl]
        L.synth_ln_export.restype = dbl
        L.synth_sincos_2pi_export.argtypes = [dbl, vp, vp]
        L.synth_gaussian_f64.argtypes = [vp, i64, u64, u32, u32]
        L.synth_gaussian_f32.argtypes = [vp, i64, u64, u32, u32]
        L.synth_uniform_f64.argtypes = [vp, i64, u64, u32, u32]
        L.synth_factors.argtypes = [vp, vp, i64, i64, ctypes.c_int, ctypes.c_int, dbl, u64, u32]
        L.synth_lowrank_from_factors.argtypes = [vp, vp, vp, i64, i64, i64, ctypes.c_int, dbl, u64, u32]
        L.synth_uniform_int.argtypes = [vp, i64, i32, i32, u64, u32, u32]
        L.synth_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"] or a.ndim == 2
    return a.ctypes.data


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().synth_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def ln(x: float) -> float:
    return lib().synth_ln_export(float(x))


def sincos_2pi(u: float):
    c, s = ctypes.c_double(), ctypes.c_double()
    lib().synth_sincos_2pi_export(float(u), ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def gaussian(count: int, seed: int, stream: int, instance: int = 0, dtype=np.float64) -> np.ndarray:
    out = np.empty(count, dtype=dtype)
    if dtype == np.float64:
        lib().synth_gaussian_f64(_ptr(out), count, seed, stream, instance)
    else:
        lib().synth_gaussian_f32(_ptr(out), count, seed, stream, instance)
    return out


def uniform(count: int, seed: int, stream: int, instance: int = 0) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    lib().synth_uniform_f64(_ptr(out), count, seed, stream, instance)
    return out


def uniform_int(count: int, lo: int, hi: int, seed: int, stream: int, instance: int = 0) -> np.ndarray:
    out = np.empty(count, dtype=np.int32)
    lib().synth_uniform_int(_ptr(out), count, lo, hi, seed, stream, instance)
    return out


@dataclass(frozen=True)
class Workload:
    """One synthetic nonnegative input A = W0 H0 + sigma |z| and its rHALS settings."""
    name: str
    m: int
    n: int
    r: int            # rank of W0 H0
    k: int            # target rank
    p: int            # oversampling, l = k + p
    q: int            # power (subspace) iterations
    iters: int        # HALS sweeps
    sigma: float      # noise scale
    w0_exp: bool = False        # W0 ~ Exponential(1) instead of U[0,1)
    h0_zero_frac: float = 0.0   # fraction of H0 entries zeroed
    seed: int = 0               # rHALS seed: Omega from seed, W/H init from seed + 1
    instance: int = 0

    @property
    def l(self) -> int:
        return self.k + self.p


# The five workloads (synthetic stand-ins for Section 4.4's experiments).
SMALL = Workload("rhals_fp32_1000x500_k10", 1000, 500, 10, 10, 10, 2, 100, 0.01)
SCALE = Workload("rhals_fp32_50000x20000_k50", 50000, 20000, 50, 50, 20, 2, 200, 0.05)
PRECISION = Workload("rhals_bf16sketch_100000x50000_k100", 100000, 50000, 100, 100, 20, 2, 300, 0.02,
                     w0_exp=True, h0_zero_frac=0.3)
ADJOINT = Workload("adjoint_4096x2048_k16_T50", 4096, 2048, 16, 16, 10, 1, 50, 0.01)
ADJOINT_FD = Workload("adjoint_fd_64x32_k4_T5", 64, 32, 4, 4, 2, 1, 5, 0.01)


def factors(w: Workload):
    W0 = np.empty((w.m, w.r), np.float64)
    H0 = np.empty((w.r, w.n), np.float64)
    lib().synth_factors(_ptr(W0), _ptr(H0), w.m, w.n, w.r, int(w.w0_exp), w.h0_zero_frac, DATA_SEED,
                        w.instance)
    return W0, H0


def lowrank_into(out: np.ndarray, w: Workload, sigma: float | None = None, W0=None, H0=None) -> np.ndarray:
    """Fill the float32 (m x >=n) array ``out`` with A of workload ``w``."""
    assert out.dtype == np.float32 and out.ndim == 2 and out.shape[0] == w.m and out.shape[1] >= w.n
    assert out.strides[1] == 4
    if W0 is None:
        W0, H0 = factors(w)
    lda = out.strides[0] // 4
    s = w.sigma if sigma is None else sigma
    lib().synth_lowrank_from_factors(out.ctypes.data, _ptr(W0), _ptr(H0), w.m, w.n, lda, w.r, s,
                                     DATA_SEED, w.instance)
    return out


def lowrank(w: Workload, sigma: float | None = None) -> np.ndarray:
    out = np.empty((w.m, w.n), np.float32)
    return lowrank_into(out, w, sigma)


def cotangent(m: int, n: int) -> np.ndarray:
    """G ~ N(0,1) (m x n, float32) of the differentiation workload: key 2, stream 8."""
    return gaussian(m * n, G_SEED, STREAM_G, 0, np.float32).reshape(m, n)


def batch_workloads(count: int = 512, iters: int = 100, seed: int = 0):
    """Ragged batch: heights U{256..8192}, widths U{128..4096}, ranks U{4..32}; k = r, p = 10, q = 2."""
    ms = uniform_int(count, 256, 8192, DATA_SEED, STREAM_SHAPES, 0)
    ns = uniform_int(count, 128, 4096, DATA_SEED, STREAM_SHAPES, 1)
    rs = uniform_int(count, 4, 32, DATA_SEED, STREAM_SHAPES, 2)
    return [Workload(f"batch_{i}", int(ms[i]), int(ns[i]), int(rs[i]), int(rs[i]), 10, 2, iters, 0.01,
                     seed=seed, instance=i + 1) for i in range(count)]
