"""Host check of the double-float arithmetic (csrc/df.cuh) that the CholeskyQR
factorisation runs on the GPU.

The header compiles as plain C++ (its rounding steps map to ordinary float
operations with contraction off), so a small host program exercises the same
formulas: two million random operands over 2^-20 .. 2^20, each result compared
with the exact value in long double.  Bounds: a few units of 2^-48 (the format
carries about 48 significant bits), i.e. relative error < 2^-44 for add, mul,
c - a b, 1/x and sqrt(x); and a 120 x 120 Cholesky factor inverse, computed
in the kernel's order (right-looking factorisation, then the row sweep with
32-way split sums), within 2^-42 of the long-double inverse, relative to its
diagonal.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_1711_02037_gb300", "csrc", "df.cuh")

PROGRAM = r"""
#define __host__
#define __device__
#define __forceinline__ inline
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>
#include "df.cuh"
typedef long double LD;
static dfloat from(LD v) { float h = (float)v; return df_make(h, (float)(v - (LD)h)); }
static LD val(dfloat x) { return (LD)x.hi + (LD)x.lo; }
int main() {
    std::mt19937_64 g(1);
    std::uniform_real_distribution<double> U(-1, 1);
    double w[5] = {0, 0, 0, 0, 0};
    for (int it = 0; it < 2000000; ++it) {
        LD a = (LD)U(g) * std::pow(2.0L, (int)(U(g) * 20)), b = (LD)U(g) * std::pow(2.0L, (int)(U(g) * 20));
        LD c = (LD)U(g) * 4;
        dfloat A = from(a), B = from(b), C = from(c);
        LD av = val(A), bv = val(B), cv = val(C);
        w[0] = std::fmax(w[0], (double)(std::fabs(val(df_add(A, B)) - (av + bv)) / (std::fabs(av) + std::fabs(bv))));
        w[1] = std::fmax(w[1], (double)(std::fabs(val(df_mul(A, B)) - av * bv) / std::fabs(av * bv)));
        w[2] = std::fmax(w[2], (double)(std::fabs(val(df_fms(C, A, B)) - (cv - av * bv)) /
                                        (std::fabs(cv) + std::fabs(av * bv))));
        w[3] = std::fmax(w[3], (double)(std::fabs(val(df_recip(A)) - 1.0L / av) * std::fabs(av)));
        dfloat P = A.hi < 0 ? df_neg(A) : A;
        LD pv = val(P);
        w[4] = std::fmax(w[4], (double)(std::fabs(val(df_sqrt(P)) - std::sqrt(pv)) / std::sqrt(pv)));
    }
    // Cholesky factor inverse of a Gram with condition ~1e8, in the kernel's order
    const int c = 120, N = 2000;
    std::normal_distribution<double> nd;
    std::vector<LD> Y((size_t)N * c), G((size_t)c * c, 0);
    for (int j = 0; j < c; ++j) {
        LD sc = std::pow(10.0L, -4.0L * j / (c - 1));
        for (int r = 0; r < N; ++r) Y[(size_t)r * c + j] = (float)(nd(g) * (double)sc);
    }
    for (int r = 0; r < N; ++r)
        for (int i = 0; i < c; ++i)
            for (int j = 0; j < c; ++j) G[i * c + j] += Y[(size_t)r * c + i] * Y[(size_t)r * c + j];
    std::vector<LD> R(G), X((size_t)c * c, 0);
    for (int j = 0; j < c; ++j) {
        R[j * c + j] = std::sqrt(R[j * c + j]);
        for (int t = j + 1; t < c; ++t) R[j * c + t] /= R[j * c + j];
        for (int ii = j + 1; ii < c; ++ii)
            for (int tt = ii; tt < c; ++tt) R[ii * c + tt] -= R[j * c + ii] * R[j * c + tt];
    }
    for (int i = c - 1; i >= 0; --i) {
        X[i * c + i] = 1 / R[i * c + i];
        for (int jc = i + 1; jc < c; ++jc) {
            LD s = 0;
            for (int t = i + 1; t <= jc; ++t) s += R[i * c + t] * X[t * c + jc];
            X[i * c + jc] = -s / R[i * c + i];
        }
    }
    std::vector<dfloat> Gs((size_t)c * c), diag(c);
    for (int e = 0; e < c * c; ++e) Gs[e] = from(G[e]);
    for (int j = 0; j < c; ++j) {
        dfloat r = df_sqrt(Gs[j * c + j]);
        Gs[j * c + j] = r;
        dfloat dinv = df_recip(r);
        for (int t = j + 1; t < c; ++t) Gs[j * c + t] = df_mul(Gs[j * c + t], dinv);
        for (int ii = j + 1; ii < c; ++ii)
            for (int tt = ii; tt < c; ++tt) Gs[ii * c + tt] = df_fms(Gs[ii * c + tt], Gs[j * c + ii], Gs[j * c + tt]);
    }
    for (int i = 0; i < c; ++i) {
        diag[i] = df_recip(Gs[i * c + i]);
        Gs[i * c + i] = diag[i];
    }
    for (int i = c - 2; i >= 0; --i)
        for (int jc = i + 1; jc < c; ++jc) {
            dfloat part[32];
            for (int L = 0; L < 32; ++L) part[L] = df_make(0.f, 0.f);
            for (int t = i + 1; t <= jc; ++t) {
                const int L = (t - (i + 1)) % 32;
                part[L] = df_add(part[L], df_mul(Gs[i * c + t], Gs[jc * c + t]));
            }
            for (int o = 16; o > 0; o >>= 1) {
                dfloat nx[32];
                for (int L = 0; L < 32; ++L) nx[L] = df_add(part[L], part[L ^ o]);
                for (int L = 0; L < 32; ++L) part[L] = nx[L];
            }
            Gs[jc * c + i] = df_neg(df_mul(part[0], diag[i]));
        }
    double wi = 0;
    for (int i = 0; i < c; ++i)
        for (int j = i; j < c; ++j) {
            LD v = val(i == j ? Gs[i * c + i] : Gs[j * c + i]);
            wi = std::fmax(wi, (double)(std::fabs(v - X[i * c + j]) / std::fabs(X[j * c + j])));
        }
    printf("%.6e %.6e %.6e %.6e %.6e %.6e\n", w[0], w[1], w[2], w[3], w[4], wi);
    return 0;
}
"""


def test_double_float_arithmetic(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "df_check.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "df_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.dirname(HEADER), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    add, mul, fms, recip, sqrt_, inv = (float(v) for v in out)
    for name, err in (("add", add), ("mul", mul), ("fms", fms), ("recip", recip), ("sqrt", sqrt_)):
        assert err < 2.0 ** -44, (name, err)
    assert inv < 2.0 ** -42, inv
