// Conditional value-function elements and their associative combination.
//
// An element is the parameter tuple (A, b, C, eta, J) of the linear-affine
// conditional value function of Eq. (35),
//   V(phi; z) = 1/2 phi^T J phi - phi^T eta + 1/2 |z - A phi - b|^2_{C^-1},
// where phi is the state at the start of the reversed-time interval and z the
// state at its end.  C and J are symmetric and stored packed.
//
// combine(ei, ej) is the rule of Section 4.1 (Eq. 36) for ei on [s, gamma]
// followed by ej on [gamma, t].  apply(e, P) is the same rule when the right
// operand is a value function of one variable, V(z) = 1/2 z^T P z - v^T z
// (A = C = b = 0 for it), i.e. the combination with a suffix that already
// contains the terminal element a_T of Eq. (31); it also returns the
// closed-loop affine map (Section 3.5, Eq. 40-41) of the interval,
//   z*(phi) = E phi + g,  E = (I + C P)^-1 A,  g = (I + C P)^-1 (b + C v),
// which the RTS pass composes.
//
// Precision policy: the (I + C J) inverse runs in the element precision S
// with diagonal pivots.  When a pivot is small against its column
// (tau = 1/2) or the infinity-norm condition estimate |M| |M^-1| exceeds the
// threshold, (I + C J) is formed and inverted again in FP64 with row
// pivoting, and a device counter records it; the products around the inverse
// stay in S.
#pragma once
#include <type_traits>
#include "smallmat.cuh"

namespace mapk {

using ms::Sym;

template <int N, typename S>
struct Elem {
    static constexpr int NS = Sym<N>::SZ;
    static constexpr int NCOMP = N * N + 2 * N + 2 * NS;
    S A[N * N];
    S b[N];
    S C[NS];
    S eta[N];
    S J[NS];
};

// value function of one variable: 1/2 x^T P x - v^T x
template <int N, typename S>
struct Red {
    static constexpr int NS = Sym<N>::SZ;
    static constexpr int NCOMP = N + NS;
    S v[N];
    S P[NS];
};

// affine map x -> F x + c
template <int N, typename S>
struct Aff {
    static constexpr int NCOMP = N * N + N;
    S F[N * N];
    S c[N];
};

// A handle's device event words (unsigned long long): [0] combines whose
// inverse was recomputed in FP64, [1] singular pivots, [2] bounded waits that
// ran out, [3] grid-barrier arrivals of the single-launch solves, [4] device
// address of the handle's host-mapped error flags (0: none), [5] the counter
// of the wait self-test.
constexpr int STATS_WORDS = 8;
enum : int { EV_FP64 = 0, EV_SINGULAR = 1, EV_TIMEOUT = 2, EV_BARRIER = 3, EV_FLAGS = 4, EV_SELFTEST = 5 };

// Count event ev (EV_SINGULAR, EV_TIMEOUT) and raise the matching host-visible
// flag: the result of the launch is not valid, and the handle's next call
// returns the error (the flags live in mapped host memory, so the host reads
// them without a device synchronisation).
__device__ __forceinline__ void report_event(unsigned long long* stats, int ev)
{
    if (!stats) return;
    atomicAdd(stats + ev, 1ull);
    const unsigned long long a = *reinterpret_cast<volatile unsigned long long*>(stats + EV_FLAGS);
    if (a) {
        *(reinterpret_cast<volatile unsigned*>(a) + ev) = 1u;
        __threadfence_system();
    }
}

struct CombineCtx {
    float cond_max;                  // FP64 inverse when |M| |M^-1| exceeds this
    unsigned long long* stats;       // the event words above
};

template <int N, typename S>
__device__ __forceinline__ void set_identity(Elem<N, S>& e)
{
#pragma unroll
    for (int i = 0; i < N * N; ++i) e.A[i] = (i % (N + 1) == 0) ? S(1) : S(0);
#pragma unroll
    for (int i = 0; i < N; ++i) { e.b[i] = S(0); e.eta[i] = S(0); }
#pragma unroll
    for (int i = 0; i < Elem<N, S>::NS; ++i) { e.C[i] = S(0); e.J[i] = S(0); }
}

template <int N, typename S>
__device__ __forceinline__ void set_identity(Aff<N, S>& a)
{
#pragma unroll
    for (int i = 0; i < N * N; ++i) a.F[i] = (i % (N + 1) == 0) ? S(1) : S(0);
#pragma unroll
    for (int i = 0; i < N; ++i) a.c[i] = S(0);
}

// flat component access (the order is the SoA component order in memory)
template <int N, typename S>
__device__ __forceinline__ S& comp(Elem<N, S>& e, int i)
{
    constexpr int NS = Sym<N>::SZ;
    return i < N * N ? e.A[i]
         : i < N * N + N ? e.b[i - N * N]
         : i < N * N + N + NS ? e.C[i - N * N - N]
         : i < N * N + 2 * N + NS ? e.eta[i - N * N - N - NS]
         : e.J[i - N * N - 2 * N - NS];
}
template <int N, typename S>
__device__ __forceinline__ S& comp(Red<N, S>& r, int i) { return i < N ? r.v[i] : r.P[i - N]; }
template <int N, typename S>
__device__ __forceinline__ S& comp(Aff<N, S>& a, int i) { return i < N * N ? a.F[i] : a.c[i - N * N]; }

// SoA load/store: component i of item `idx` lives at base[i * stride + idx]
template <class T, typename S>
__device__ __forceinline__ void soa_load(const S* __restrict__ base, long stride, long idx, T& x)
{
#pragma unroll
    for (int i = 0; i < T::NCOMP; ++i) comp(x, i) = base[i * stride + idx];
}
template <class T, typename S>
__device__ __forceinline__ void soa_store(S* __restrict__ base, long stride, long idx, T& x)
{
#pragma unroll
    for (int i = 0; i < T::NCOMP; ++i) base[i * stride + idx] = comp(x, i);
}

template <int N, typename Sd, typename Ss>
__device__ __forceinline__ void convert(const Elem<N, Ss>& s, Elem<N, Sd>& d)
{
#pragma unroll
    for (int i = 0; i < N * N; ++i) d.A[i] = Sd(s.A[i]);
#pragma unroll
    for (int i = 0; i < N; ++i) { d.b[i] = Sd(s.b[i]); d.eta[i] = Sd(s.eta[i]); }
#pragma unroll
    for (int i = 0; i < Sym<N>::SZ; ++i) { d.C[i] = Sd(s.C[i]); d.J[i] = Sd(s.J[i]); }
}

// ---------------------------------------------------------------------------
// (I + C P) and its inverse.  Fast path: diagonal pivots in precision S, with
// the pivot test and the infinity-norm condition estimate.  Slow path (rare):
// in FP32 solves, first the same matrix with row pivoting in FP32, kept when
// its condition estimate is within cond_max; otherwise (and in FP64 solves)
// (I + C P) formed and inverted in FP64 with row pivoting.  Only the inverse
// is returned, the rest of the operation stays in S.  The slow path copies its
// inputs into a local buffer inside the branch, so the operands of the fast
// path stay in registers.
// ---------------------------------------------------------------------------
template <int N, typename S>
__device__ __noinline__ void inverse_I_plus_fp64(const S* buf, S* out, unsigned long long* stats,
                                                 float cond_max = 0.f)
{
    constexpr int NS = Sym<N>::SZ;
    if constexpr (std::is_same<S, float>::value) {
        if (cond_max > 0.f) {
            float M[N * N], Mi[N * N];
            ms::sym_sym<N, float>(buf, buf + NS, M);
#pragma unroll
            for (int i = 0; i < N; ++i) M[i * N + i] += 1.f;
            const float nM = ms::norm_inf<N, float>(M);
            if (ms::inv_row_pivot<N, float>(M, Mi)) {
                const float nMi = ms::norm_inf<N, float>(Mi);
                if (nM * nMi <= cond_max) {           // false for inf and NaN
#pragma unroll
                    for (int i = 0; i < N * N; ++i) out[i] = Mi[i];
                    return;
                }
            }
        }
    }
    double Cd[NS], Pd[NS], M[N * N], Mi[N * N];
#pragma unroll
    for (int i = 0; i < NS; ++i) { Cd[i] = double(buf[i]); Pd[i] = double(buf[NS + i]); }
    ms::sym_sym<N, double>(Cd, Pd, M);
#pragma unroll
    for (int i = 0; i < N; ++i) M[i * N + i] += 1.0;
    const bool ok = ms::inv_row_pivot<N, double>(M, Mi);
#pragma unroll
    for (int i = 0; i < N * N; ++i) out[i] = S(Mi[i]);
    if (stats) {
        atomicAdd(stats, 1ull);
        if (!ok) report_event(stats, EV_SINGULAR);
    }
}

template <int N, typename S>
__device__ __forceinline__ void inverse_I_plus(const S* Cp, const S* Pp, S* Mi, float cond_max,
                                               unsigned long long* stats)
{
    constexpr int NS = Sym<N>::SZ;
    S M[N * N];
    ms::sym_sym<N, S>(Cp, Pp, M);
#pragma unroll
    for (int i = 0; i < N; ++i) M[i * N + i] += S(1);
    const S nM = ms::norm_inf<N, S>(M);
    const bool ok = ms::inv_diag_pivot<N, S>(M, Mi, S(0.5));
    const S nMi = ms::norm_inf<N, S>(Mi);
    if (!(ok && float(nM) * float(nMi) <= cond_max)) {
        S buf[2 * NS], out[N * N];
#pragma unroll
        for (int i = 0; i < NS; ++i) { buf[i] = Cp[i]; buf[NS + i] = Pp[i]; }
        inverse_I_plus_fp64<N, S>(buf, out, stats, cond_max);
#pragma unroll
        for (int i = 0; i < N * N; ++i) Mi[i] = out[i];
    }
}

// core of e_i (x) e_j given Mi = (I + C_i J_j)^-1
template <int N, typename S>
__device__ __forceinline__ void combine_core(const Elem<N, S>& ei, const Elem<N, S>& ej,
                                             const S* Mi, Elem<N, S>& out)
{
    S T1[N * N], T2[N * N], T3[N * N], u[N], w[N];
    Elem<N, S> r;
    ms::mm<N, S>(Mi, ei.A, T3);                       // M^-1 A_i  (= (A_i^T M^-T)^T)
    ms::sym_v<N, S>(ej.J, ei.b, u);                   // J_j b_i
#pragma unroll
    for (int i = 0; i < N; ++i) u[i] = ej.eta[i] - u[i];
    ms::mtv_add<N, S>(T3, u, ei.eta, r.eta);          // eta_ij
    ms::sym_m<N, S>(ej.J, ei.A, T2);                  // J_j A_i
    ms::sym_atb_add<N, S>(T3, T2, ei.J, r.J);         // J_ij
    ms::mm<N, S>(ej.A, Mi, T1);                       // A_j M^-1
    ms::mm<N, S>(T1, ei.A, r.A);                      // A_ij
    ms::sym_v<N, S>(ei.C, ej.eta, u);                 // C_i eta_j
#pragma unroll
    for (int i = 0; i < N; ++i) u[i] += ei.b[i];
    ms::mv<N, S>(T1, u, w);
#pragma unroll
    for (int i = 0; i < N; ++i) r.b[i] = w[i] + ej.b[i];   // b_ij
    ms::m_sym<N, S>(T1, ei.C, T2);                    // A_j M^-1 C_i
    ms::sym_abt_add<N, S>(T2, ej.A, ej.C, r.C);       // C_ij
    out = r;
}

// out = ei (x) ej  (out may alias either operand)
template <int N, typename S>
__device__ __forceinline__ void combine(const Elem<N, S>& ei, const Elem<N, S>& ej,
                                        Elem<N, S>& out, const CombineCtx& ctx)
{
    S Mi[N * N];
    inverse_I_plus<N, S>(ei.C, ej.J, Mi, ctx.cond_max, ctx.stats);
    combine_core<N, S>(ei, ej, Mi, out);
}

// ---------------------------------------------------------------------------
// e (x) [P, v]: value-function update and the interval's closed-loop map
// ---------------------------------------------------------------------------
template <int N, typename S, bool ALPHA>
__device__ __forceinline__ void apply(const Elem<N, S>& e, Red<N, S>& p, S* E, S* g,
                                      const CombineCtx& ctx)
{
    S Mi[N * N];
    inverse_I_plus<N, S>(e.C, p.P, Mi, ctx.cond_max, ctx.stats);
    S Em[N * N], T4[N * N], u[N], w[N];
    ms::mm<N, S>(Mi, e.A, Em);                        // E = M^-1 A
    if (ALPHA) {
        ms::sym_v<N, S>(e.C, p.v, u);
#pragma unroll
        for (int i = 0; i < N; ++i) u[i] += e.b[i];
        ms::mv<N, S>(Mi, u, g);                       // g = M^-1 (b + C v)
#pragma unroll
        for (int i = 0; i < N * N; ++i) E[i] = Em[i];
    }
    ms::sym_m<N, S>(p.P, e.A, T4);                    // P A
    ms::sym_v<N, S>(p.P, e.b, u);                     // P b
#pragma unroll
    for (int i = 0; i < N; ++i) w[i] = p.v[i] - u[i];
    Red<N, S> r;
    ms::sym_atb_add<N, S>(Em, T4, e.J, r.P);          // A^T M^-T P A + J
    ms::mtv_add<N, S>(Em, w, e.eta, r.v);             // A^T M^-T (v - P b) + eta
    p = r;
}

// ---------------------------------------------------------------------------
// e (x) [P, v] when C = Gam Gam^T with Gam N x R (R < N): by the matrix
// inversion lemma
//   (I + C P)^-1 = I - Gam W Gam^T P,   W = (I_R + Gam^T P Gam)^-1,
// so with U = P Gam the closed-loop map is E = A - Gam W (U^T A),
// g = z - Gam W (U^T z) with z = b + Gam (Gam^T v), and (P (I + C P)^-1 =
// (I + P C)^-1 P, push-through)
//   P' = A^T (P E) + J,   v' = E^T (v - P b) + eta.
// The R x R matrix D = I + Gam^T P Gam is symmetric positive definite for a
// positive semidefinite P; it is inverted by Cholesky.  Returns false (and
// leaves p unchanged) when a Cholesky pivot is not positive or the
// infinity-norm condition estimate |D| |D^-1| exceeds cond_max (the same
// threshold as the general update's); the caller then takes the general
// update with its FP64 recomputation.
// ---------------------------------------------------------------------------
template <int N, int R, typename S, bool ALPHA>
__device__ __forceinline__ bool apply_lowrank(const Elem<N, S>& e, const S* Gam, Red<N, S>& p, S* E, S* g,
                                              float cond_max, S* Vout = nullptr)
{
    S U[N * R];                                       // U = P Gam
    ms::sym_mr<N, R, S>(p.P, Gam, U);
    S L[R * R], Li[R * R], W[R * R];                  // I + Gam^T U = L L^T,  W = L^-T L^-1
    bool ok = true;
#pragma unroll
    for (int j = 0; j < R; ++j) {
#pragma unroll
        for (int i = j; i < R; ++i) {
            S s = (i == j) ? S(1) : S(0);
#pragma unroll
            for (int q = 0; q < N; ++q) s = fma(Gam[q * R + i], U[q * R + j], s);
#pragma unroll
            for (int k = 0; k < j; ++k) s = fma(-L[i * R + k], L[j * R + k], s);
            if (i == j) {
                ok = ok && s > S(0);
                L[j * R + j] = sqrt(s > S(0) ? s : S(1));
                Li[j * R + j] = S(1) / L[j * R + j];
            } else {
                L[i * R + j] = s * Li[j * R + j];
            }
        }
    }
    if (!ok) return false;
    S nD = S(0);                                      // |D|_inf, D = L L^T
#pragma unroll
    for (int i = 0; i < R; ++i) {
        S row = S(0);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            S d = S(0);
#pragma unroll
            for (int k = 0; k <= (i < j ? i : j); ++k) d = fma(L[i * R + k], L[j * R + k], d);
            row += ms::sabs(d);
        }
        nD = row > nD ? row : nD;
    }
#pragma unroll
    for (int i = 0; i < R; ++i)                       // L^-1 (lower triangular)
#pragma unroll
        for (int j = 0; j < i; ++j) {
            S s = S(0);
#pragma unroll
            for (int k = j; k < i; ++k) s = fma(L[i * R + k], Li[k * R + j], s);
            Li[i * R + j] = -s * Li[i * R + i];
        }
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            S s = S(0);
#pragma unroll
            for (int k = i; k < R; ++k) s = fma(Li[k * R + i], Li[k * R + j], s);
            W[i * R + j] = s;
            W[j * R + i] = s;
        }
    S nW = S(0);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        S row = S(0);
#pragma unroll
        for (int j = 0; j < R; ++j) row += ms::sabs(W[i * R + j]);
        nW = row > nW ? row : nW;
    }
    if (!(float(nD) * float(nW) <= cond_max)) return false;
    S V[R * N], Em[N * N];                            // V = W (U^T A),  E = A - Gam V
    ms::mtm<R, N, N, S>(U, e.A, Em);                  // U^T A, temporarily
    ms::mm_sub<R, R, N, S>(nullptr, W, Em, V);
    if (Vout) {                                       // E = A - Gam V: the compact form of the map
#pragma unroll
        for (int q = 0; q < R * N; ++q) Vout[q] = V[q];
    }
    ms::mm_sub<N, R, N, S>(e.A, Gam, V, Em);
    if (ALPHA) {
        S t[R], z[N], t2[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            S s = S(0);
#pragma unroll
            for (int i = 0; i < N; ++i) s = fma(Gam[i * R + k], p.v[i], s);
            t[k] = s;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S s = e.b[i];
#pragma unroll
            for (int k = 0; k < R; ++k) s = fma(Gam[i * R + k], t[k], s);
            z[i] = s;
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            S s = S(0);
#pragma unroll
            for (int i = 0; i < N; ++i) s = fma(U[i * R + k], z[i], s);
            t[k] = s;
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            S s = S(0);
#pragma unroll
            for (int l = 0; l < R; ++l) s = fma(W[k * R + l], t[l], s);
            t2[k] = s;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S s = z[i];
#pragma unroll
            for (int k = 0; k < R; ++k) s = fma(-Gam[i * R + k], t2[k], s);
            g[i] = s;
        }
#pragma unroll
        for (int i = 0; i < N * N; ++i) E[i] = Em[i];
    }
    S PE[N * N], w[N];                                // P E,  w = v - P b
    ms::sym_m<N, S>(p.P, Em, PE);
    ms::sym_v<N, S>(p.P, e.b, w);
#pragma unroll
    for (int i = 0; i < N; ++i) w[i] = p.v[i] - w[i];
    Red<N, S> r;
    ms::sym_atb_add<N, S>(e.A, PE, e.J, r.P);         // A^T (P E) + J
    ms::mtv_add<N, S>(Em, w, e.eta, r.v);             // E^T w + eta
    p = r;
    return true;
}

// ---------------------------------------------------------------------------
// affine maps (Eq. 40-41): (F1, c1) o (F2, c2) = (F1 F2, F1 c2 + c1)
// ---------------------------------------------------------------------------
template <int N, typename S>
__device__ __forceinline__ void compose(const Aff<N, S>& a1, const Aff<N, S>& a2, Aff<N, S>& out)
{
    Aff<N, S> r;
    ms::mm<N, S>(a1.F, a2.F, r.F);
    ms::mv<N, S>(a1.F, a2.c, r.c);
#pragma unroll
    for (int i = 0; i < N; ++i) r.c[i] += a1.c[i];
    out = r;
}

template <int N, typename S>
__device__ __forceinline__ void affine_apply(const Aff<N, S>& a, const S* x, S* y)
{
    ms::mv<N, S>(a.F, x, y);
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] += a.c[i];
}

// FP32 Cholesky factor of a packed symmetric matrix (L lower, il = 1 / diag);
// false when a pivot is not positive
template <int N>
__device__ __forceinline__ bool chol_f32(const float* P, float* L, float* il)
{
    bool pd = true;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        float d = P[Sym<N>::at(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) d = fmaf(-L[j * N + k], L[j * N + k], d);
        pd = pd && d > 0.f;
        il[j] = rsqrtf(d > 0.f ? d : 1.f);
        L[j * N + j] = 1.f / il[j];
#pragma unroll
        for (int i = j + 1; i < N; ++i) {
            float s = P[Sym<N>::at(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) s = fmaf(-L[i * N + k], L[j * N + k], s);
            L[i * N + j] = s * il[j];
        }
    }
    return pd;
}

// x = (L L^T)^-1 r
template <int N>
__device__ __forceinline__ void chol_solve_f32(const float* L, const float* il, const float* r, float* x)
{
    float z[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float s = r[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s = fmaf(-L[i * N + k], z[k], s);
        z[i] = s * il[i];
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        float s = z[i];
#pragma unroll
        for (int k = i + 1; k < N; ++k) s = fmaf(-L[k * N + i], x[k], s);
        x[i] = s * il[i];
    }
}

// x = P^-1 v (the minimiser of a one-variable value function, Eq. 18 initial condition)
template <int N, typename S>
__device__ __forceinline__ bool red_argmin(const Red<N, S>& p, S* x)
{
    if constexpr (std::is_same<S, float>::value) {
        // FP32 Cholesky with iterative refinement on FP64 residuals v - P x: the
        // FP64 solution to within a few FP32 ulps once a correction falls below
        // 2^-22 of x (at most three rounds); otherwise the FP64 solve below
        float L[N * N], il[N], xf[N];
        if (chol_f32<N>(p.P, L, il)) {
            chol_solve_f32<N>(L, il, p.v, xf);
            bool conv = false;
#pragma unroll 1
            for (int it = 0; it < 3 && !conv; ++it) {
                float r[N], dx[N];
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    double s = double(p.v[i]);
#pragma unroll
                    for (int k = 0; k < N; ++k) s = fma(-double(p.P[Sym<N>::at(i, k)]), double(xf[k]), s);
                    r[i] = float(s);
                }
                chol_solve_f32<N>(L, il, r, dx);
                float nd = 0.f, nx = 0.f;
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    xf[i] += dx[i];
                    nd = fmaxf(nd, fabsf(dx[i]));
                    nx = fmaxf(nx, fabsf(xf[i]));
                }
                conv = nd <= 0x1p-22f * nx;
            }
            if (conv) {
#pragma unroll
                for (int i = 0; i < N; ++i) x[i] = xf[i];
                return true;
            }
        }
    }
    double M[N * N], v[N], xd[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        v[i] = double(p.v[i]);
#pragma unroll
        for (int j = 0; j < N; ++j) M[i * N + j] = double(p.P[Sym<N>::at(i, j)]);
    }
    // P is symmetric positive definite for an observable model with P0 > 0:
    // Cholesky (fixed indexing, one reciprocal per column); a non-positive
    // pivot falls back to Gauss-Jordan with row pivoting
    double L[N * N], il[N];
    bool pd = true;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        double d = M[j * N + j];
#pragma unroll
        for (int k = 0; k < j; ++k) d = fma(-L[j * N + k], L[j * N + k], d);
        pd = pd && d > 0.0;
        const double ljj = sqrt(d > 0.0 ? d : 1.0);
        il[j] = 1.0 / ljj;
#pragma unroll
        for (int i = j + 1; i < N; ++i) {
            double s = M[i * N + j];
#pragma unroll
            for (int k = 0; k < j; ++k) s = fma(-L[i * N + k], L[j * N + k], s);
            L[i * N + j] = s * il[j];
        }
    }
    bool ok = true;
    if (pd) {
        double z[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = v[i];
#pragma unroll
            for (int k = 0; k < i; ++k) s = fma(-L[i * N + k], z[k], s);
            z[i] = s * il[i];
        }
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
            double s = z[i];
#pragma unroll
            for (int k = i + 1; k < N; ++k) s = fma(-L[k * N + i], xd[k], s);
            xd[i] = s * il[i];
        }
    } else {
        double Mi[N * N];
        ok = ms::inv_row_pivot<N, double>(M, Mi);
        ms::mv<N, double>(Mi, v, xd);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = S(xd[i]);
    return ok;
}

}  // namespace mapk
