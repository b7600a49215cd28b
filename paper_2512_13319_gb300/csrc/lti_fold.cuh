// Folds and tile trees of a linear time-invariant model as linear functions
// of the observations.
//
// For an LTI model every element of the filter scan has the same (A, b, C, J)
// and eta_k = G y_k - Gr with G = dt H^T R^-1 (Section 4.2 elements).  In the
// combine (Eq. 36) the outputs A, C and J depend only on the A, C and J of the
// operands, while b and eta depend linearly on the operands' b and eta.  Hence:
//
// (1) The fold of K full steps of one thread,
//       e_{k0+K-1} (x) ... (x) e_{k0+1} (x) e_{k0},
//     has the same (A, C, J) for every thread, and its (b, eta) is
//       (b, eta) = (b0, eta0) + sum_i Gamma_i y_{k0+i},   Gamma_i: 2N x M.
//     k_lti_fold evaluates the same combine recursion once in FP64, carrying
//     the b/eta parts as affine functions of the observations: with the new
//     (later) element on the left and
//       Mi = (I + C_e J_acc)^-1,  Tb = A_acc Mi C_e,  Te = A_e^T Mi^T,
//     the update is
//       b   <- b + Tb eta + A_acc Mi b_e,
//       eta <- Te (eta - J_acc b_e) + G y_i - Gr,
//       A <- A_acc Mi A_e,  C <- A_acc Mi C_e A_acc^T + C_acc,  J <- A_e^T Mi^T J_acc A_e + J_e.
//
// (2) In the tree of a tile whose B*K steps are all before T, the two children
//     of a level-d node are folds of 2^d full threads, with the same (A_d,
//     C_d, J_d).  With Mi = (I + C_d J_d)^-1 the parent (later child i on the
//     left, earlier child j on the right) is
//       b   = X_d b_i + b_j + Y_d eta_j,       X_d = A_d Mi,  Y_d = A_d Mi C_d,
//       eta = eta_i + Z_d eta_j - W_d b_i,     Z_d = A_d^T Mi^T,  W_d = Z_d J_d,
//     and (A_d+1, C_d+1, J_d+1) is the combine of (A_d, C_d, J_d) with itself.
//
// The reduce and down-sweep kernels evaluate (1) and (2) with these constants
// (2 N M multiply-adds per step and 4 N^2 per tree node instead of a combine);
// tiles that reach past T keep the general per-step fold and tree.
#pragma once
#include "producers.cuh"
#include "coop.cuh"

namespace mapk {

// Layout of the constants (scalars of type S).  K-fold constants with packed
// symmetric C, J; the Gamma_i; then per tree level d = 0..LMAX the children's
// (A_d, C_d, J_d) as an element node of CoopLayout (full rows padded to P)
// followed by X_d, Y_d, Z_d, W_d (N x N row-major).
template <int N, int M, typename S>
struct FoldLayout {
    using CL = CoopLayout<N, S>;
    static constexpr int NS = Sym<N>::SZ;
    static constexpr int KMAX = 64, LMAX = 7;              // K <= 64, B <= 128
    static constexpr int oA = 0, oC = N * N, oJ = oC + NS, ob = oJ + NS, oe = ob + N;
    static constexpr int oG = (oe + N + 3) / 4 * 4;         // Gamma_i at oG + i * GS
    static constexpr int GS = 2 * N * M;                    // rows 0..N-1: b, rows N..2N-1: eta
    static constexpr int oL = (oG + KMAX * GS + 3) / 4 * 4; // level d at oL + d * LS
    static constexpr int LN = 3 * N * CL::P;                // (A_d, C_d, J_d) node part
    static constexpr int oX = LN, oY = LN + N * N, oZ = LN + 2 * N * N, oW = LN + 3 * N * N;
    static constexpr int LS = (LN + 4 * N * N + 3) / 4 * 4;
    // folds of r = 1 .. KMAX-1 steps (a thread that reaches T): per r the
    // constants A, C, J, b0, eta0 (HS scalars, packed as above) then Gamma_0..r-1
    static constexpr int oP = oL + (LMAX + 1) * LS;
    static constexpr int HS = (N * N + 2 * NS + 2 * N + 3) / 4 * 4;
    __host__ __device__ static constexpr int poff(int r) { return oP + (r - 1) * HS + GS * (r - 1) * r / 2; }
    static constexpr int TOTAL = oP + (KMAX - 1) * HS + GS * (KMAX - 1) * KMAX / 2;
};

// Plan-time helpers of k_lti_fold (FP64, plain loops: run once per model and
// geometry, so they are kept small rather than unrolled)
namespace fold_detail {

// c = a b (n x n, row-major)
__device__ inline void mm(int n, const double* a, const double* b, double* c)
{
#pragma unroll 1
    for (int i = 0; i < n; ++i)
#pragma unroll 1
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
#pragma unroll 1
            for (int k = 0; k < n; ++k) s += a[i * n + k] * b[k * n + j];
            c[i * n + j] = s;
        }
}

// c = a^T (n x n)
__device__ inline void tr(int n, const double* a, double* c)
{
#pragma unroll 1
    for (int i = 0; i < n; ++i)
#pragma unroll 1
        for (int j = 0; j < n; ++j) c[i * n + j] = a[j * n + i];
}

// y = a x
__device__ inline void mv(int n, const double* a, const double* x, double* y)
{
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
#pragma unroll 1
        for (int k = 0; k < n; ++k) s += a[i * n + k] * x[k];
        y[i] = s;
    }
}

// out = (I + c j)^-1 by Gauss-Jordan elimination with row pivoting; w: 2 n^2 scratch
__device__ inline void inv_I_plus(int n, const double* c, const double* j, double* out, double* w)
{
    double* X = w;
    mm(n, c, j, X);
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        X[i * n + i] += 1.0;
#pragma unroll 1
        for (int k = 0; k < n; ++k) out[i * n + k] = i == k ? 1.0 : 0.0;
    }
#pragma unroll 1
    for (int col = 0; col < n; ++col) {
        int piv = col;
#pragma unroll 1
        for (int r = col + 1; r < n; ++r)
            if (fabs(X[r * n + col]) > fabs(X[piv * n + col])) piv = r;
        if (piv != col) {
#pragma unroll 1
            for (int k = 0; k < n; ++k) {
                double t = X[col * n + k]; X[col * n + k] = X[piv * n + k]; X[piv * n + k] = t;
                t = out[col * n + k]; out[col * n + k] = out[piv * n + k]; out[piv * n + k] = t;
            }
        }
        const double p = X[col * n + col];
        const double ip = p != 0.0 ? 1.0 / p : 0.0;
#pragma unroll 1
        for (int k = 0; k < n; ++k) { X[col * n + k] *= ip; out[col * n + k] *= ip; }
#pragma unroll 1
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double f = X[r * n + col];
#pragma unroll 1
            for (int k = 0; k < n; ++k) {
                X[r * n + k] -= f * X[col * n + k];
                out[r * n + k] -= f * out[col * n + k];
            }
        }
    }
}

}  // namespace fold_detail

// One CTA of KMAX threads; thread j carries Gamma_j.  FP64 throughout.
template <int N, int M, typename S>
__global__ void __launch_bounds__(64)
k_lti_fold(const LtiParams<N, M, double> p, int K, int LB, S* __restrict__ out)
{
    using FL = FoldLayout<N, M, S>;
    using CL = CoopLayout<N, S>;
    namespace fd = fold_detail;
    constexpr int NN = N * N;
    // accumulated composite (Ac, Cc, Jc), per-step maps (Tb, Te), offsets,
    // the element's constants and thread-0 scratch
    __shared__ double Ac[NN], Cc[NN], Jc[NN], Tb[NN], Te[NN], ob[N], oe[N];
    __shared__ double Ae[NN], Ce[NN], Je[NN], be[N], Gm[N * M], Gr[N];
    __shared__ double Mi[NN], T1[NN], T2[NN], T3[NN], wk[2 * NN], u[N], w[N];
    const int j = threadIdx.x;
    if (j == 0) {
#pragma unroll 1
        for (int a = 0; a < N; ++a) {
#pragma unroll 1
            for (int c = 0; c < N; ++c) {
                Ae[a * N + c] = p.A[a * N + c];
                Ce[a * N + c] = p.C[Sym<N>::at(a, c)];
                Je[a * N + c] = p.J[Sym<N>::at(a, c)];
            }
            be[a] = p.b[a];
            Gr[a] = p.Gr[a];
        }
#pragma unroll 1
        for (int q = 0; q < N * M; ++q) Gm[q] = p.G[q];
#pragma unroll 1
        for (int q = 0; q < NN; ++q) { Ac[q] = Ae[q]; Cc[q] = Ce[q]; Jc[q] = Je[q]; }
#pragma unroll 1
        for (int a = 0; a < N; ++a) { ob[a] = be[a]; oe[a] = -Gr[a]; }
    }
    __syncthreads();
    double gb[N * M], ge[N * M];                  // Gamma_j (b rows, eta rows)
#pragma unroll 1
    for (int q = 0; q < N * M; ++q) { gb[q] = 0.0; ge[q] = j == 0 ? Gm[q] : 0.0; }
    // the r-step fold (r < K): constants by thread 0, Gamma_j by thread j < r
    auto write_partial = [&](int r) {
        S* pb = out + FL::poff(r);
        if (j == 0) {
#pragma unroll 1
            for (int q = 0; q < NN; ++q) pb[FL::oA + q] = S(Ac[q]);
#pragma unroll 1
            for (int a = 0; a < N; ++a) {
#pragma unroll 1
                for (int c = a; c < N; ++c) {
                    pb[FL::oC + Sym<N>::at(a, c)] = S(0.5 * (Cc[a * N + c] + Cc[c * N + a]));
                    pb[FL::oJ + Sym<N>::at(a, c)] = S(0.5 * (Jc[a * N + c] + Jc[c * N + a]));
                }
                pb[FL::ob + a] = S(ob[a]);
                pb[FL::oe + a] = S(oe[a]);
            }
        }
        if (j < r) {
            S* g = pb + FL::HS + j * FL::GS;
#pragma unroll 1
            for (int q = 0; q < N * M; ++q) { g[q] = S(gb[q]); g[N * M + q] = S(ge[q]); }
        }
    };
    if (K > 1) write_partial(1);
#pragma unroll 1
    for (int i = 1; i < K; ++i) {
        if (j == 0) {
            fd::inv_I_plus(N, Ce, Jc, Mi, wk);    // (I + C_e J_acc)^-1
            fd::mm(N, Ac, Mi, T1);                // A_acc Mi
            fd::mm(N, T1, Ce, Tb);                // Tb = A_acc Mi C_e
            fd::mm(N, Mi, Ae, T2);
            fd::tr(N, T2, Te);                    // Te = (Mi A_e)^T
            // offsets: b <- b + Tb eta + A_acc Mi b_e;  eta <- Te (eta - J_acc b_e) - Gr
            fd::mv(N, Jc, be, u);
#pragma unroll 1
            for (int a = 0; a < N; ++a) u[a] = oe[a] - u[a];
            fd::mv(N, Te, u, w);
            fd::mv(N, Tb, oe, u);
#pragma unroll 1
            for (int a = 0; a < N; ++a) { ob[a] += u[a]; oe[a] = w[a] - Gr[a]; }
            fd::mv(N, T1, be, u);
#pragma unroll 1
            for (int a = 0; a < N; ++a) ob[a] += u[a];
            // composite: A = A_acc Mi A_e, C = Tb A_acc^T + C_acc, J = Te J_acc A_e + J_e
            fd::mm(N, T1, Ae, T2);
            fd::tr(N, Ac, T3);
            fd::mm(N, Tb, T3, T1);
#pragma unroll 1
            for (int q = 0; q < NN; ++q) { Ac[q] = T2[q]; Cc[q] += T1[q]; }
            fd::mm(N, Jc, Ae, T2);
            fd::mm(N, Te, T2, T3);
#pragma unroll 1
            for (int q = 0; q < NN; ++q) Jc[q] = T3[q] + Je[q];
        }
        __syncthreads();
        if (j < i) {                              // earlier observations: old eta parts on the right
            double nb[N * M], ne[N * M];
#pragma unroll 1
            for (int a = 0; a < N; ++a)
#pragma unroll 1
                for (int c = 0; c < M; ++c) {
                    double sb = gb[a * M + c], se = 0.0;
#pragma unroll 1
                    for (int k = 0; k < N; ++k) {
                        sb += Tb[a * N + k] * ge[k * M + c];
                        se += Te[a * N + k] * ge[k * M + c];
                    }
                    nb[a * M + c] = sb;
                    ne[a * M + c] = se;
                }
#pragma unroll 1
            for (int q = 0; q < N * M; ++q) { gb[q] = nb[q]; ge[q] = ne[q]; }
        } else if (j == i) {
#pragma unroll 1
            for (int q = 0; q < N * M; ++q) { gb[q] = 0.0; ge[q] = Gm[q]; }
        }
        __syncthreads();
        if (i + 1 < K) write_partial(i + 1);
    }
    if (j < K) {
        S* g = out + FL::oG + j * FL::GS;
#pragma unroll 1
        for (int q = 0; q < N * M; ++q) { g[q] = S(gb[q]); g[N * M + q] = S(ge[q]); }
    }
    if (j != 0) return;
#pragma unroll 1
    for (int q = 0; q < NN; ++q) out[FL::oA + q] = S(Ac[q]);
#pragma unroll 1
    for (int a = 0; a < N; ++a) {
#pragma unroll 1
        for (int c = a; c < N; ++c) {
            out[FL::oC + Sym<N>::at(a, c)] = S(0.5 * (Cc[a * N + c] + Cc[c * N + a]));
            out[FL::oJ + Sym<N>::at(a, c)] = S(0.5 * (Jc[a * N + c] + Jc[c * N + a]));
        }
        out[FL::ob + a] = S(ob[a]);
        out[FL::oe + a] = S(oe[a]);
    }
    // tree levels: level d holds the constants of its children
#pragma unroll 1
    for (int d = 0; d <= LB && d <= FL::LMAX; ++d) {
        S* lv = out + FL::oL + d * FL::LS;
#pragma unroll 1
        for (int a = 0; a < N; ++a)
#pragma unroll 1
            for (int c = 0; c < CL::P; ++c) {
                const bool in = c < N;
                lv[CL::oA + a * CL::P + c] = in ? S(Ac[a * N + c]) : S(0);
                lv[CL::oC + a * CL::P + c] = in ? S(0.5 * (Cc[a * N + c] + Cc[c * N + a])) : S(0);
                lv[CL::oJ + a * CL::P + c] = in ? S(0.5 * (Jc[a * N + c] + Jc[c * N + a])) : S(0);
            }
        if (d == LB) break;
        // X = A Mi, Y = A Mi C, Z = (Mi A)^T, W = Z J with Mi = (I + C J)^-1
        fd::inv_I_plus(N, Cc, Jc, Mi, wk);
        fd::mm(N, Ac, Mi, T1);                    // X
        fd::mm(N, T1, Cc, Tb);                    // Y
        fd::mm(N, Mi, Ac, T2);
        fd::tr(N, T2, Te);                        // Z
        fd::mm(N, Te, Jc, T3);                    // W
#pragma unroll 1
        for (int q = 0; q < NN; ++q) {
            lv[FL::oX + q] = S(T1[q]);
            lv[FL::oY + q] = S(Tb[q]);
            lv[FL::oZ + q] = S(Te[q]);
            lv[FL::oW + q] = S(T3[q]);
        }
        // parent: A = X A, C = Y A^T + C, J = W A + J
        fd::mm(N, T1, Ac, T2);
        fd::tr(N, Ac, wk);
        fd::mm(N, Tb, wk, Mi);
        fd::mm(N, T3, Ac, wk + NN);
#pragma unroll 1
        for (int q = 0; q < NN; ++q) { Ac[q] = T2[q]; Cc[q] += Mi[q]; Jc[q] += wk[NN + q]; }
    }
}

// (b, eta) of one thread's K full steps from the constants (Gamma staged in
// shared memory at gam) and the observations y_{k0}..y_{k0+K-1}
template <int N, typename S, class Prod>
__device__ __forceinline__ void lti_linear_fold(const Prod& prod, const S* __restrict__ fold,
                                                const S* gam, int K, long k0, S* bq)
{
    constexpr int M = Prod::W;
    using FL = FoldLayout<N, M, S>;
    S ab[N], ae[N];
#pragma unroll
    for (int q = 0; q < N; ++q) { ab[q] = __ldg(fold + FL::ob + q); ae[q] = __ldg(fold + FL::oe + q); }
#pragma unroll 2
    for (int i = 0; i < K; ++i) {
        S row[M], g[FL::GS];
        prod.load1(k0 + i, row);
        const S* gi = gam + i * FL::GS;
        if constexpr (sizeof(S) == 4 && FL::GS % 4 == 0) {
#pragma unroll
            for (int q = 0; q < FL::GS; q += 4) {
                const float4 v = *reinterpret_cast<const float4*>(gi + q);
                g[q] = v.x; g[q + 1] = v.y; g[q + 2] = v.z; g[q + 3] = v.w;
            }
        } else if constexpr (sizeof(S) == 8 && FL::GS % 2 == 0) {
#pragma unroll
            for (int q = 0; q < FL::GS; q += 2) {
                const double2 v = *reinterpret_cast<const double2*>(gi + q);
                g[q] = v.x; g[q + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int q = 0; q < FL::GS; ++q) g[q] = gi[q];
        }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int c = 0; c < M; ++c) {
                ab[a] = fma(g[a * M + c], row[c], ab[a]);
                ae[a] = fma(g[(N + a) * M + c], row[c], ae[a]);
            }
    }
#pragma unroll
    for (int q = 0; q < N; ++q) { bq[q] = ab[q]; bq[N + q] = ae[q]; }
}

// The element of a thread whose first r < K steps are before T (the rest are
// identity padding): the r-step fold from its constants pb (FoldLayout::poff(r)
// block, staged in shared memory) and its observations yq (r rows of M, staged)
template <int N, int M, typename S>
__device__ __forceinline__ void lti_partial_fold_elem(const S* pb, const S* yq, int r, Elem<N, S>& G)
{
    using FL = FoldLayout<N, M, S>;
#pragma unroll
    for (int q = 0; q < N * N; ++q) G.A[q] = pb[FL::oA + q];
#pragma unroll
    for (int q = 0; q < Sym<N>::SZ; ++q) { G.C[q] = pb[FL::oC + q]; G.J[q] = pb[FL::oJ + q]; }
#pragma unroll
    for (int q = 0; q < N; ++q) { G.b[q] = pb[FL::ob + q]; G.eta[q] = pb[FL::oe + q]; }
#pragma unroll 4
    for (int i = 0; i < r; ++i) {
        const S* g = pb + FL::HS + i * FL::GS;
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int c = 0; c < M; ++c) {
                G.b[a] = fma(g[a * M + c], yq[i * M + c], G.b[a]);
                G.eta[a] = fma(g[(N + a) * M + c], yq[i * M + c], G.eta[a]);
            }
    }
}

// The full element of one thread's K full steps (constants + linear fold)
template <int N, typename S, class Prod>
__device__ __forceinline__ void lti_fold_elem(const Prod& prod, const S* __restrict__ fold, const S* gam,
                                              int K, long k0, Elem<N, S>& G)
{
    using FL = FoldLayout<N, Prod::W, S>;
#pragma unroll
    for (int q = 0; q < N * N; ++q) G.A[q] = __ldg(fold + FL::oA + q);
#pragma unroll
    for (int q = 0; q < Sym<N>::SZ; ++q) { G.C[q] = __ldg(fold + FL::oC + q); G.J[q] = __ldg(fold + FL::oJ + q); }
    S bq[2 * N];
    lti_linear_fold<N, S>(prod, fold, gam, K, k0, bq);
#pragma unroll
    for (int q = 0; q < N; ++q) { G.b[q] = bq[q]; G.eta[q] = bq[N + q]; }
}

// Up-sweep of a full tile's tree on the (b, eta) parts: bq holds 2B nodes of
// 2N scalars (tree levels as lvl_off), leaves stored by the caller; lv the
// level constants (FoldLayout level blocks, in shared memory).
template <int N, int M, typename S>
__device__ void lti_tree_up(S* bq, const S* lv)
{
    using FL = FoldLayout<N, M, S>;
    const int B = blockDim.x, t = threadIdx.x;
    const int LB = 31 - __clz(B);
    for (int d = 0; d < LB; ++d) {
        __syncthreads();
        const int cnt = B >> (d + 1);
        if (t < cnt) {
            const S* L = lv + d * FL::LS;
            const S* ci = bq + (2 * B - ((2 * B) >> d) + 2 * t + 1) * 2 * N;    // later child
            const S* cj = ci - 2 * N;                                           // earlier child
            S* par = bq + (2 * B - ((2 * B) >> (d + 1)) + t) * 2 * N;
            S bi[N], ei[N], bj[N], ej[N];
#pragma unroll
            for (int q = 0; q < N; ++q) { bi[q] = ci[q]; ei[q] = ci[N + q]; bj[q] = cj[q]; ej[q] = cj[N + q]; }
#pragma unroll
            for (int a = 0; a < N; ++a) {
                S sb = bj[a], se = ei[a];
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    sb = fma(L[FL::oX + a * N + k], bi[k], sb);
                    sb = fma(L[FL::oY + a * N + k], ej[k], sb);
                    se = fma(L[FL::oZ + a * N + k], ej[k], se);
                    se = fma(-L[FL::oW + a * N + k], bi[k], se);
                }
                par[a] = sb;
                par[N + a] = se;
            }
        }
    }
    __syncthreads();
}

// Down-sweep of a full tile's tree: the value function before every leaf
// (value nodes pre, 2B slots of CoopLayout::NR) from the prefix of the tile
// (stored by the caller at the root slot), with the left children's elements
// given by the level constants and the (b, eta) nodes of the up-sweep.
template <int N, int M, typename S>
__device__ void lti_tree_down(const S* bq, const S* lv, S* pre, S* scr_all, const CombineCtx& ctx,
                              Red<N, S>& out)
{
    using FL = FoldLayout<N, M, S>;
    using L = CoopLayout<N, S>;
    const int B = blockDim.x, LB = 31 - __clz(B);
    const int NL = L::NL, ng = B / NL, g = threadIdx.x / NL, r = threadIdx.x & (NL - 1);
    S* scr = scr_all + g * L::NSCR;
    auto lvl_off = [B](int d) { return 2 * B - ((2 * B) >> d); };
    for (int d = LB - 1; d >= 0; --d) {
        __syncthreads();
        const int cnt = B >> (d + 1);
        for (int base = 0; base < cnt; base += ng) {
            const int j = base + g;
            const bool act = j < cnt;
            if (__any_sync(0xffffffffu, act)) {
                const int jj = act ? j : base;
                const S* par = pre + (lvl_off(d + 1) + jj) * L::NR;
                S* lft = pre + (lvl_off(d) + 2 * jj) * L::NR;
                S* rgt = lft + L::NR;
                const S* lq = bq + (lvl_off(d) + 2 * jj) * 2 * N;         // left child's (b, eta)
                coop_apply_parts<N, S>(lv + d * FL::LS, lq, lq + N, par, rgt, scr, act, ctx);
                __syncwarp();
                if (act)
                    for (int i = r; i < L::NR; i += NL) lft[i] = par[i];
            }
        }
    }
    __syncthreads();
    node_load(pre + (long)threadIdx.x * L::NR, out);
}

// LTI tile-tree shared memory inside the element-tree area: value nodes, the
// (b, eta) nodes and the level constants (offsets in scalars)
template <int N, int M, typename S>
struct LtiTreeSmem {
    __host__ __device__ static constexpr int pre(int) { return 0; }
    __host__ __device__ static constexpr int bq(int B) { return 2 * B * CoopLayout<N, S>::NR; }
    __host__ __device__ static constexpr int lv(int B) { return (bq(B) + 2 * B * 2 * N + 3) / 4 * 4; }
    __host__ __device__ static constexpr int end(int B, int LB) { return lv(B) + (LB + 1) * FoldLayout<N, M, S>::LS; }
};

}  // namespace mapk
