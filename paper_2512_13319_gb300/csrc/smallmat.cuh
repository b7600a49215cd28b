// Register-resident small dense linear algebra for the scan kernels.
//
// Every routine takes compile-time sizes and is fully unrolled, so the
// operands live in registers.  Symmetric matrices are stored packed (upper
// triangle, row by row).  The (I + C J) inverse is a Gauss-Jordan elimination
// without row exchanges that reports whether every pivot was at least `tau`
// times the largest entry below it; callers redo the operation with the
// pivoted FP64 routine when it was not (or when the condition estimate is too
// large).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <type_traits>

#define MS_DEV __device__ __forceinline__

namespace ms {

template <int N>
struct Sym {
    static constexpr int SZ = N * (N + 1) / 2;
    // packed index of (i, j), either triangle
    __host__ __device__ static constexpr int at(int i, int j)
    {
        return i <= j ? (i * (2 * N - i + 1)) / 2 + (j - i) : (j * (2 * N - j + 1)) / 2 + (i - j);
    }
};

template <typename S> MS_DEV S sabs(S x) { return fabs(x); }
template <> MS_DEV float sabs<float>(float x) { return fabsf(x); }

// reciprocal of a Gauss-Jordan pivot: the hardware approximation in FP32
// (within 2 ulp; the pivot test and the condition estimate guard the
// elimination), the correctly rounded quotient in FP64
template <typename S> MS_DEV S pivot_rcp(S p) { return S(1) / p; }
template <> MS_DEV float pivot_rcp<float>(float p) { return __fdividef(1.0f, p); }

// FP32 with an even N: two adjacent output columns per paired multiply-add
// (one f32x2 instruction; the same operations and rounding as two FMAs)
template <int N, typename S>
constexpr bool use_ffma2 = std::is_same<S, float>::value && N % 2 == 0;

// c = a b  (N x N)
template <int N, typename S>
MS_DEV void mm(const S* a, const S* b, S* c)
{
    if constexpr (use_ffma2<N, S>) {
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; j += 2) {
                float2 s = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < N; ++k)
                    s = __ffma2_rn(make_float2(a[i * N + k], a[i * N + k]), make_float2(b[k * N + j], b[k * N + j + 1]),
                                   s);
                c[i * N + j] = s.x;
                c[i * N + j + 1] = s.y;
            }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) {
                S s = a[i * N] * b[j];
#pragma unroll
                for (int k = 1; k < N; ++k) s = fma(a[i * N + k], b[k * N + j], s);
                c[i * N + j] = s;
            }
    }
}

// c = a S  (S packed symmetric)
template <int N, typename S>
MS_DEV void m_sym(const S* a, const S* sp, S* c)
{
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            S s = a[i * N] * sp[Sym<N>::at(0, j)];
#pragma unroll
            for (int k = 1; k < N; ++k) s = fma(a[i * N + k], sp[Sym<N>::at(k, j)], s);
            c[i * N + j] = s;
        }
}

// c = S a  (S packed symmetric)
template <int N, typename S>
MS_DEV void sym_m(const S* sp, const S* a, S* c)
{
    if constexpr (use_ffma2<N, S>) {
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; j += 2) {
                float2 s = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float p = sp[Sym<N>::at(i, k)];
                    s = __ffma2_rn(make_float2(p, p), make_float2(a[k * N + j], a[k * N + j + 1]), s);
                }
                c[i * N + j] = s.x;
                c[i * N + j + 1] = s.y;
            }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) {
                S s = sp[Sym<N>::at(i, 0)] * a[j];
#pragma unroll
                for (int k = 1; k < N; ++k) s = fma(sp[Sym<N>::at(i, k)], a[k * N + j], s);
                c[i * N + j] = s;
            }
    }
}

// c = S1 S2 (both packed symmetric), general result
template <int N, typename S>
MS_DEV void sym_sym(const S* s1, const S* s2, S* c)
{
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            S s = s1[Sym<N>::at(i, 0)] * s2[Sym<N>::at(0, j)];
#pragma unroll
            for (int k = 1; k < N; ++k) s = fma(s1[Sym<N>::at(i, k)], s2[Sym<N>::at(k, j)], s);
            c[i * N + j] = s;
        }
}

// upper triangle of a b^T (known to be symmetric) plus an optional packed addend
template <int N, typename S>
MS_DEV void sym_abt_add(const S* a, const S* b, const S* add, S* out)
{
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i; j < N; ++j) {
            S s = add[Sym<N>::at(i, j)];
#pragma unroll
            for (int k = 0; k < N; ++k) s = fma(a[i * N + k], b[j * N + k], s);
            out[Sym<N>::at(i, j)] = s;
        }
}

// upper triangle of a^T b (known to be symmetric) plus a packed addend
template <int N, typename S>
MS_DEV void sym_atb_add(const S* a, const S* b, const S* add, S* out)
{
    if constexpr (use_ffma2<N, S>) {
        // the column pairs (j, j+1) that meet the upper triangle of row i
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = i & ~1; j < N; j += 2) {
                float2 s = make_float2(j >= i ? add[Sym<N>::at(i, j)] : 0.f, add[Sym<N>::at(i, j + 1)]);
#pragma unroll
                for (int k = 0; k < N; ++k)
                    s = __ffma2_rn(make_float2(a[k * N + i], a[k * N + i]), make_float2(b[k * N + j], b[k * N + j + 1]),
                                   s);
                if (j >= i) out[Sym<N>::at(i, j)] = s.x;
                out[Sym<N>::at(i, j + 1)] = s.y;
            }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = i; j < N; ++j) {
                S s = add[Sym<N>::at(i, j)];
#pragma unroll
                for (int k = 0; k < N; ++k) s = fma(a[k * N + i], b[k * N + j], s);
                out[Sym<N>::at(i, j)] = s;
            }
    }
}

// y = a x
template <int N, typename S>
MS_DEV void mv(const S* a, const S* x, S* y)
{
#pragma unroll
    for (int i = 0; i < N; ++i) {
        S s = a[i * N] * x[0];
#pragma unroll
        for (int k = 1; k < N; ++k) s = fma(a[i * N + k], x[k], s);
        y[i] = s;
    }
}

// y = a^T x + add
template <int N, typename S>
MS_DEV void mtv_add(const S* a, const S* x, const S* add, S* y)
{
    if constexpr (use_ffma2<N, S>) {
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            float2 s = make_float2(add[i], add[i + 1]);
#pragma unroll
            for (int k = 0; k < N; ++k)
                s = __ffma2_rn(make_float2(a[k * N + i], a[k * N + i + 1]), make_float2(x[k], x[k]), s);
            y[i] = s.x;
            y[i + 1] = s.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S s = add[i];
#pragma unroll
            for (int k = 0; k < N; ++k) s = fma(a[k * N + i], x[k], s);
            y[i] = s;
        }
    }
}

// Rectangular products for the low-rank update (row-major operands; FP32
// pairs two adjacent output columns per instruction when C is even).
// c (N x C) = S b, S packed symmetric N x N, b N x C
template <int N, int C, typename S>
MS_DEV void sym_mr(const S* sp, const S* b, S* c)
{
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if constexpr (std::is_same<S, float>::value && C % 2 == 0) {
#pragma unroll
            for (int j = 0; j < C; j += 2) {
                float2 s = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float p = sp[Sym<N>::at(i, k)];
                    s = __ffma2_rn(make_float2(p, p), make_float2(b[k * C + j], b[k * C + j + 1]), s);
                }
                c[i * C + j] = s.x;
                c[i * C + j + 1] = s.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                S s = S(0);
#pragma unroll
                for (int k = 0; k < N; ++k) s = fma(sp[Sym<N>::at(i, k)], b[k * C + j], s);
                c[i * C + j] = s;
            }
        }
    }
}

// c (R x C) = a^T b, a K x R, b K x C
template <int R, int K, int C, typename S>
MS_DEV void mtm(const S* a, const S* b, S* c)
{
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if constexpr (std::is_same<S, float>::value && C % 2 == 0) {
#pragma unroll
            for (int j = 0; j < C; j += 2) {
                float2 s = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < K; ++k)
                    s = __ffma2_rn(make_float2(a[k * R + r], a[k * R + r]), make_float2(b[k * C + j], b[k * C + j + 1]),
                                   s);
                c[r * C + j] = s.x;
                c[r * C + j + 1] = s.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                S s = S(0);
#pragma unroll
                for (int k = 0; k < K; ++k) s = fma(a[k * R + r], b[k * C + j], s);
                c[r * C + j] = s;
            }
        }
    }
}

// c (R x C) = base - a b, a R x K, b K x C (base may be null: c = a b)
template <int R, int K, int C, typename S>
MS_DEV void mm_sub(const S* base, const S* a, const S* b, S* c)
{
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if constexpr (std::is_same<S, float>::value && C % 2 == 0) {
#pragma unroll
            for (int j = 0; j < C; j += 2) {
                float2 s = base ? make_float2(base[r * C + j], base[r * C + j + 1]) : make_float2(0.f, 0.f);
                const float sg = base ? -1.f : 1.f;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float v = sg * a[r * K + k];
                    s = __ffma2_rn(make_float2(v, v), make_float2(b[k * C + j], b[k * C + j + 1]), s);
                }
                c[r * C + j] = s.x;
                c[r * C + j + 1] = s.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                S s = base ? base[r * C + j] : S(0);
                const S sg = base ? S(-1) : S(1);
#pragma unroll
                for (int k = 0; k < K; ++k) s = fma(sg * a[r * K + k], b[k * C + j], s);
                c[r * C + j] = s;
            }
        }
    }
}

// y = S x  (packed symmetric)
template <int N, typename S>
MS_DEV void sym_v(const S* sp, const S* x, S* y)
{
#pragma unroll
    for (int i = 0; i < N; ++i) {
        S s = sp[Sym<N>::at(i, 0)] * x[0];
#pragma unroll
        for (int k = 1; k < N; ++k) s = fma(sp[Sym<N>::at(i, k)], x[k], s);
        y[i] = s;
    }
}

template <int N, typename S>
MS_DEV S norm_inf(const S* a)
{
    S m = S(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        S s = S(0);
#pragma unroll
        for (int j = 0; j < N; ++j) s += sabs(a[i * N + j]);
        m = s > m ? s : m;
    }
    return m;
}

// Gauss-Jordan inverse of X (destroyed) into Y, diagonal pivots.  Returns
// true when each pivot was at least tau times the largest magnitude below it
// in its column (false also for zero / NaN pivots).
template <int N, typename S>
MS_DEV bool inv_diag_pivot(S* X, S* Y, S tau)
{
    bool ok = true;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) Y[i * N + j] = i == j ? S(1) : S(0);
#pragma unroll
    for (int c = 0; c < N; ++c) {
        const S p = X[c * N + c];
        S below = S(0);
#pragma unroll
        for (int r = c + 1; r < N; ++r) {
            S a = sabs(X[r * N + c]);
            below = a > below ? a : below;
        }
        ok = ok && (sabs(p) > tau * below) && (p != S(0));
        const S ip = pivot_rcp(p);
#pragma unroll
        for (int j = c + 1; j < N; ++j) X[c * N + j] *= ip;
#pragma unroll
        for (int j = 0; j < N; ++j) Y[c * N + j] *= ip;
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (r == c) continue;
            const S f = X[r * N + c];
#pragma unroll
            for (int j = c + 1; j < N; ++j) X[r * N + j] = fma(-f, X[c * N + j], X[r * N + j]);
#pragma unroll
            for (int j = 0; j < N; ++j) Y[r * N + j] = fma(-f, Y[c * N + j], Y[r * N + j]);
        }
    }
    return ok;
}

// Gauss-Jordan inverse with partial (row) pivoting; rows are exchanged with
// selects so that every index stays a compile-time constant.  Returns false
// for an exactly singular matrix.
template <int N, typename S>
MS_DEV bool inv_row_pivot(S* X, S* Y)
{
    bool ok = true;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) Y[i * N + j] = i == j ? S(1) : S(0);
#pragma unroll
    for (int c = 0; c < N; ++c) {
        int p = c;
        S best = sabs(X[c * N + c]);
#pragma unroll
        for (int r = c + 1; r < N; ++r) {
            S a = sabs(X[r * N + c]);
            if (a > best) { best = a; p = r; }
        }
#pragma unroll
        for (int r = c + 1; r < N; ++r) {
            const bool sw = (p == r);
#pragma unroll
            for (int j = c; j < N; ++j) {
                S a = X[c * N + j], b = X[r * N + j];
                X[c * N + j] = sw ? b : a;
                X[r * N + j] = sw ? a : b;
            }
#pragma unroll
            for (int j = 0; j < N; ++j) {
                S a = Y[c * N + j], b = Y[r * N + j];
                Y[c * N + j] = sw ? b : a;
                Y[r * N + j] = sw ? a : b;
            }
        }
        const S pv = X[c * N + c];
        ok = ok && (pv != S(0));
        const S ip = S(1) / pv;
#pragma unroll
        for (int j = c + 1; j < N; ++j) X[c * N + j] *= ip;
#pragma unroll
        for (int j = 0; j < N; ++j) Y[c * N + j] *= ip;
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (r == c) continue;
            const S f = X[r * N + c];
#pragma unroll
            for (int j = c + 1; j < N; ++j) X[r * N + j] = fma(-f, X[c * N + j], X[r * N + j]);
#pragma unroll
            for (int j = 0; j < N; ++j) Y[r * N + j] = fma(-f, Y[c * N + j], Y[r * N + j]);
        }
    }
    return ok;
}

}  // namespace ms
