// Folds, tile trees and thread prefixes of a linear time-invariant model as
// linear functions of the observations.
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
// (2) In the up-sweep of a tile whose threads hold full folds, the two children
//     of a level-d node are folds of 2^d threads with the same (A_d, C_d, J_d).
//     With Mi = (I + C_d J_d)^-1 the parent (later child i on the left, earlier
//     child j on the right) is
//       b   = X_d b_i + b_j + Y_d eta_j,       X_d = A_d Mi,  Y_d = A_d Mi C_d,
//       eta = eta_i + Z_d eta_j - W_d b_i,     Z_d = A_d^T Mi^T,  W_d = Z_d J_d,
//     and (A_d+1, C_d+1, J_d+1) is the combine of (A_d, C_d, J_d) with itself.
//
// (3) The exclusive prefix of thread s of such a tile, D_s = the fold of its
//     threads 0..s-1, has the (A, C, J) of s thread folds (table "pre") and a
//     (b, eta) that a down-sweep on (b, eta) alone computes: the right child
//     that starts at thread p = (2j+1) 2^d receives U (x) D, U its left sibling
//     (level-d constants) and D the prefix of its parent (p - 2^d threads):
//       b   = X_p b_U + Y_p eta_D + b_D,  eta = eta_U + Z_p eta_D - W_p b_U,
//     with Mi = (I + C_U J_D)^-1, X_p = A_D Mi, Y_p = X_p C_U, Z_p = (Mi A_U)^T
//     and W_p = Z_p J_D (table "co").  A thread then needs one combine of D_s
//     (the one-variable case of Eq. 36, which updates a value function) with the
//     tile's prefix.
//
// (4) The tiles 0..nt-2 of a scan are full, so their totals share the
//     (A_T, C_T, J_T) of B thread folds.  The value function before tile j,
//     (P_j, v_j), then has a data-independent P_j, from the prior's P_0 by the
//     P part of the one-variable combine (Eq. 36),
//       P_{j+1} = A_T^T P_j E_j + J_T,  E_j = (I + C_T P_j)^-1 A_T,
//     and v_{j+1} = E_j^T v_j + w_j with w_j = eta_j - E_j^T P_j b_j, (b_j,
//     eta_j) the tile's total.  P_j is computed for all j in parallel: the
//     elements of 2^e full tiles are obtained by doubling, and P_j applies those
//     of the set bits of j to P_0 (chunks of equally many full tiles are the
//     same element, so their order does not matter).  The kernels then fold the
//     affine maps v -> E_j^T v + w_j of the tiles before theirs instead of
//     combining tile totals.
//
// (5) Unrolling the tile recursions: with Pi(a, b) = E_a E_{a+1} ... E_{b-1}
//     (data-independent, a table for scans of at most PI_TILES tiles),
//       v_j = Pi(0, j)^T v_0 + sum_{i<j} Pi(i+1, j)^T w_i,
//     and on the RTS side the state at the end of tile j < nt - 1 is
//       x_end(j) = Pi(j+1, nt-1) x_L + sum_{i=j+1}^{nt-2} Pi(j+1, i) beta_i,
//     x_L the state at the start of the last tile and beta_i the offset of
//     full tile i's map (whose linear part is E_i: the composition of a tile's
//     closed-loop maps is the closed-loop map of its combined element).  Both
//     are sums of independent terms: a CTA's threads take one term each and
//     add them up, without a chain of compositions.
//
// All constants depend on the model, K, B and the number of tiles only.  The
// reduce and down-sweep kernels evaluate (1)-(4) with them: 2 N M
// multiply-adds per step and 4 N^2 per tree node instead of a combine.
#pragma once
#include <type_traits>
#include "producers.cuh"
#include "coop.cuh"

namespace mapk {

// Layout of the constants (scalars of type S).  K-fold constants with packed
// symmetric C, J; the Gamma_i; per tree level d = 0..LMAX the children's
// (A_d, C_d, J_d) as an element node of CoopLayout (full rows padded to P)
// followed by X_d, Y_d, Z_d, W_d (N x N row-major); the thread-prefix
// constants pre_s = (A, C, J) of s thread folds (s = 0..BMAX-1, C and J
// packed); the right-child coefficients co_p = (X, Y, Z, W)_p (p = 1..BMAX-1).
template <int N, int M, typename S>
struct FoldLayout {
    using CL = CoopLayout<N, S>;
    static constexpr int NS = Sym<N>::SZ;
    static constexpr int KMAX = 64, LMAX = 7, BMAX = 128;   // K <= 64, B <= 128
    static constexpr int oA = 0, oC = N * N, oJ = oC + NS, ob = oJ + NS, oe = ob + N;
    static constexpr int oG = (oe + N + 3) / 4 * 4;         // Gamma_i at oG + i * GS
    static constexpr int GS = 2 * N * M;                    // rows 0..N-1: b, rows N..2N-1: eta
    static constexpr int oL = (oG + KMAX * GS + 3) / 4 * 4; // level d at oL + d * LS
    static constexpr int LN = 3 * N * CL::P;                // (A_d, C_d, J_d) node part
    static constexpr int oX = LN, oY = LN + N * N, oZ = LN + 2 * N * N, oW = LN + 3 * N * N;
    static constexpr int LS = (LN + 4 * N * N + 3) / 4 * 4;
    static constexpr int PS = (N * N + 2 * NS + 3) / 4 * 4; // pre_s at oPre + s * PS: A, C, J
    static constexpr int oPre = oL + (LMAX + 1) * LS;
    static constexpr int CS = 4 * N * N;                    // co_p at oCo + p * CS: X, Y, Z, W
    static constexpr int oCo = oPre + BMAX * PS;
    static constexpr int TOTAL = oCo + BMAX * CS;
};

// Per-tile tables of item (4), in the fold buffer after FoldLayout::TOTAL
// (offsets in bytes): the FP64 (A, C, J) of 2^e full tiles (e < ELMAX, full
// N x N matrices), then P_j (packed, scalars of S) and F_j = E_j^T (N x N
// row-major) for j < nt, E_j in FP64, and for scans of at most PI_TILES tiles
// the products Pi(a, b) of consecutive tiles' closed-loop maps (item (5)) by
// rows (a) and their transposes by columns (b).
template <int N, int M, typename S>
struct TileTables {
    static constexpr int ELMAX = 24;                        // up to 2^24 tiles
    static constexpr int NN = N * N, NS = Sym<N>::SZ;
    __host__ __device__ static constexpr size_t al(size_t x) { return (x + 15) / 16 * 16; }
    __host__ __device__ static constexpr size_t tl_off() { return al(sizeof(S) * FoldLayout<N, M, S>::TOTAL); }
    __host__ __device__ static constexpr size_t p_off() { return tl_off() + sizeof(double) * ELMAX * 3 * NN; }
    __host__ __device__ static constexpr size_t f_off(long nt) { return p_off() + al(sizeof(S) * nt * NS); }
    // E_j in FP64, then (scans of at most PI_TILES tiles) the products
    // Pi(a, b) = E_a E_{a+1} ... E_{b-1}, 0 <= a <= b < nt, row a holding b = a..nt-1
    static constexpr long PI_TILES = 4 * 128 + 1;
    __host__ __device__ static constexpr size_t e_off(long nt) { return al(f_off(nt) + sizeof(S) * nt * NN); }
    __host__ __device__ static constexpr size_t pi_off(long nt) { return al(e_off(nt) + sizeof(double) * nt * NN); }
    __host__ __device__ static constexpr long pi_index(long nt, long a, long b) { return a * nt - a * (a - 1) / 2 + (b - a); }
    // then the transposes Q(b, a) = Pi(a, b)^T, row b holding a = 0..b
    __host__ __device__ static constexpr size_t qt_off(long nt) { return pi_off(nt) + sizeof(S) * (size_t)(nt * (nt + 1) / 2) * NN; }
    __host__ __device__ static constexpr long qt_index(long b, long a) { return b * (b + 1) / 2 + a; }
    __host__ __device__ static constexpr size_t bytes(long nt)
    {
        return pi_off(nt) + (nt <= PI_TILES ? 2 * sizeof(S) * (size_t)(nt * (nt + 1) / 2) * NN : 0);
    }
};

// Tile-level inputs of the linear-fold kernels: the fold constants, the tile
// tables P_j and F_j, the per-solve w_j (N scalars per tile, written by the
// reduce kernel) and, for scans with more than one group of tiles, the
// composed maps of the groups (Aff records)
template <typename S>
struct LtiTiles {
    const S* fold;
    const S* P;
    const S* F;
    S* w;
    S* gmaps;
    int co_smem;                    // the co table is staged in shared memory (LtiDownSmem)
    const S* pi;                    // tile-map products (item (5)), or nullptr beyond PI_TILES
    const S* qt;                    // their transposes by column (item (5))
};

// The co table is stored by tree level: level d holds the B / 2^(d+1) right
// children p = (2i+1) 2^d of a tile of B threads, component-major (component
// q of entry i at q * B / 2^(d+1) + i, the components X, Y, Z, W row-major),
// so that the threads of a down-sweep level read consecutive words.  Offset of
// level d in scalars; the table holds 4 N^2 (B - 1) scalars.
template <int N>
__host__ __device__ constexpr int lti_co_level(int B, int d)
{
    return 4 * N * N * (B - (B >> d));
}

// Plan-time helpers of the constant kernels (FP64; n is the state dimension,
// a compile-time size, and the loops unroll)
namespace fold_detail {

// c = a b (n x n, row-major)
template <int n>
__device__ inline void mm(const double* a, const double* b, double* c)
{
#pragma unroll
    for (int i = 0; i < n; ++i)
#pragma unroll
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < n; ++k) s += a[i * n + k] * b[k * n + j];
            c[i * n + j] = s;
        }
}

// c = a^T (n x n)
template <int n>
__device__ inline void tr(const double* a, double* c)
{
#pragma unroll
    for (int i = 0; i < n; ++i)
#pragma unroll
        for (int j = 0; j < n; ++j) c[i * n + j] = a[j * n + i];
}

// y = a x
template <int n>
__device__ inline void mv(const double* a, const double* x, double* y)
{
#pragma unroll
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) s += a[i * n + k] * x[k];
        y[i] = s;
    }
}

// out = (I + c j)^-1 by Gauss-Jordan elimination with row pivoting; w: 2 n^2 scratch
template <int n>
__device__ inline void inv_I_plus(const double* c, const double* j, double* out, double* w)
{
    double* X = w;
    mm<n>(c, j, X);
#pragma unroll
    for (int i = 0; i < n; ++i) {
        X[i * n + i] += 1.0;
#pragma unroll
        for (int k = 0; k < n; ++k) out[i * n + k] = i == k ? 1.0 : 0.0;
    }
#pragma unroll
    for (int col = 0; col < n; ++col) {
        int piv = col;
#pragma unroll
        for (int r = col + 1; r < n; ++r)
            if (fabs(X[r * n + col]) > fabs(X[piv * n + col])) piv = r;
        if (piv != col) {
#pragma unroll
            for (int k = 0; k < n; ++k) {
                double t = X[col * n + k]; X[col * n + k] = X[piv * n + k]; X[piv * n + k] = t;
                t = out[col * n + k]; out[col * n + k] = out[piv * n + k]; out[piv * n + k] = t;
            }
        }
        const double p = X[col * n + col];
        const double ip = p != 0.0 ? 1.0 / p : 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) { X[col * n + k] *= ip; out[col * n + k] *= ip; }
#pragma unroll
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double f = X[r * n + col];
#pragma unroll
            for (int k = 0; k < n; ++k) {
                X[r * n + k] -= f * X[col * n + k];
                out[r * n + k] -= f * out[col * n + k];
            }
        }
    }
}

// coefficients of the (b, eta) part of U (x) D (U the later operand):
// Mi = (I + C_U J_D)^-1, X = A_D Mi, Y = X C_U, Z = (Mi A_U)^T, W = Z J_D;
// wk: 4 n^2 scratch
template <int n>
__device__ inline void pair_coeffs(const double* AU, const double* CU, const double* AD, const double* JD,
                                   double* X, double* Y, double* Z, double* W, double* wk)
{
    double* Mi = wk;
    double* T = wk + n * n;
    inv_I_plus<n>(CU, JD, Mi, wk + 2 * n * n);
    mm<n>(AD, Mi, X);
    mm<n>(X, CU, Y);
    mm<n>(Mi, AU, T);
    tr<n>(T, Z);
    mm<n>(Z, JD, W);
}

// (A, C, J) of U (x) D from the coefficients of pair_coeffs:
// A = X A_U, C = Y A_D^T + C_D, J = W A_U + J_U; wk: n^2 scratch
template <int n>
__device__ inline void pair_acj(const double* AU, const double* JU, const double* AD, const double* CD,
                                const double* X, const double* Y, const double* W, double* Ao, double* Co,
                                double* Jo, double* wk)
{
    mm<n>(X, AU, Ao);
    tr<n>(AD, wk);
    mm<n>(Y, wk, Co);
    mm<n>(W, AU, Jo);
#pragma unroll
    for (int q = 0; q < n * n; ++q) { Co[q] += CD[q]; Jo[q] += JU[q]; }
}

// P <- A^T P (I + C P)^-1 A + J, symmetrised (full matrices); w: 4 n^2 scratch
template <int n>
__device__ inline void riccati(const double* A, const double* C, const double* J, double* P, double* w)
{
    double* Mi = w;
    double* T1 = w + n * n;
    double* T2 = w + 2 * n * n;
    inv_I_plus<n>(C, P, Mi, w + 3 * n * n);
    mm<n>(Mi, A, T1);                  // (I + C P)^-1 A
    mm<n>(P, T1, T2);                  // P (I + C P)^-1 A
#pragma unroll
    for (int i = 0; i < n; ++i)
#pragma unroll
        for (int j = 0; j < n; ++j) {
            double s = J[i * n + j];
#pragma unroll
            for (int k = 0; k < n; ++k) s += A[k * n + i] * T2[k * n + j];
            Mi[i * n + j] = s;
        }
#pragma unroll
    for (int i = 0; i < n; ++i)
#pragma unroll
        for (int j = 0; j < n; ++j) P[i * n + j] = 0.5 * (Mi[i * n + j] + Mi[j * n + i]);
}

}  // namespace fold_detail

// One CTA of KMAX threads; thread j carries Gamma_j.  FP64 throughout.  LB:
// log2 of the threads per tile (B = 2^LB <= BMAX); ne: the tile levels of
// item (4) to write (2^ne above every tile index).
template <int N, int M, typename S>
__global__ void __launch_bounds__(64)
k_lti_fold(const LtiParams<N, M, double> p, int K, int LB, int ne, S* __restrict__ out)
{
    using FL = FoldLayout<N, M, S>;
    using CL = CoopLayout<N, S>;
    namespace fd = fold_detail;
    constexpr int NN = N * N;
    // accumulated composite (Ac, Cc, Jc), per-step maps (Tb, Te), offsets,
    // the element's constants, thread-0 scratch and the tree levels' (A, C, J)
    __shared__ double Ac[NN], Cc[NN], Jc[NN], Tb[NN], Te[NN], ob[N], oe[N];
    __shared__ double Ae[NN], Ce[NN], Je[NN], be[N], Gm[N * M], Gr[N];
    __shared__ double Mi[NN], T1[NN], T2[NN], T3[NN], wk[4 * NN], u[N], w[N];
    __shared__ double LA[FL::LMAX + 1][NN], LC[FL::LMAX + 1][NN], LJ[FL::LMAX + 1][NN];
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
#pragma unroll 1
    for (int i = 1; i < K; ++i) {
        if (j == 0) {
            fd::inv_I_plus<N>(Ce, Jc, Mi, wk);    // (I + C_e J_acc)^-1
            fd::mm<N>(Ac, Mi, T1);                // A_acc Mi
            fd::mm<N>(T1, Ce, Tb);                // Tb = A_acc Mi C_e
            fd::mm<N>(Mi, Ae, T2);
            fd::tr<N>(T2, Te);                    // Te = (Mi A_e)^T
            // offsets: b <- b + Tb eta + A_acc Mi b_e;  eta <- Te (eta - J_acc b_e) - Gr
            fd::mv<N>(Jc, be, u);
#pragma unroll 1
            for (int a = 0; a < N; ++a) u[a] = oe[a] - u[a];
            fd::mv<N>(Te, u, w);
            fd::mv<N>(Tb, oe, u);
#pragma unroll 1
            for (int a = 0; a < N; ++a) { ob[a] += u[a]; oe[a] = w[a] - Gr[a]; }
            fd::mv<N>(T1, be, u);
#pragma unroll 1
            for (int a = 0; a < N; ++a) ob[a] += u[a];
            // composite: A = A_acc Mi A_e, C = Tb A_acc^T + C_acc, J = Te J_acc A_e + J_e
            fd::mm<N>(T1, Ae, T2);
            fd::tr<N>(Ac, T3);
            fd::mm<N>(Tb, T3, T1);
#pragma unroll 1
            for (int q = 0; q < NN; ++q) { Ac[q] = T2[q]; Cc[q] += T1[q]; }
            fd::mm<N>(Jc, Ae, T2);
            fd::mm<N>(Te, T2, T3);
#pragma unroll 1
            for (int q = 0; q < NN; ++q) Jc[q] = T3[q] + Je[q];
        }
        __syncthreads();
        if (j < i) {                              // earlier observations: old eta parts on the right
            double nb[N * M], nq[N * M];
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
                    nq[a * M + c] = se;
                }
#pragma unroll 1
            for (int q = 0; q < N * M; ++q) { gb[q] = nb[q]; ge[q] = nq[q]; }
        } else if (j == i) {
#pragma unroll 1
            for (int q = 0; q < N * M; ++q) { gb[q] = 0.0; ge[q] = Gm[q]; }
        }
        __syncthreads();
    }
    if (j < K) {
        S* g = out + FL::oG + j * FL::GS;
#pragma unroll 1
        for (int q = 0; q < N * M; ++q) { g[q] = S(gb[q]); g[N * M + q] = S(ge[q]); }
    }
    if (j == 0) {
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
            for (int q = 0; q < NN; ++q) { LA[d][q] = Ac[q]; LC[d][q] = Cc[q]; LJ[d][q] = Jc[q]; }
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
            fd::pair_coeffs<N>(Ac, Cc, Ac, Jc, T1, Tb, Te, T3, wk);   // X, Y, Z, W
#pragma unroll 1
            for (int q = 0; q < NN; ++q) {
                lv[FL::oX + q] = S(T1[q]);
                lv[FL::oY + q] = S(Tb[q]);
                lv[FL::oZ + q] = S(Te[q]);
                lv[FL::oW + q] = S(T3[q]);
            }
            fd::pair_acj<N>(Ac, Jc, Ac, Cc, T1, Tb, T3, T2, Mi, wk, wk + NN);
#pragma unroll 1
            for (int q = 0; q < NN; ++q) { Ac[q] = T2[q]; Cc[q] = Mi[q]; Jc[q] = wk[q]; }
        }
        // tile levels (item (4)): (Ac, Cc, Jc) now hold the full tile
        double* tl = reinterpret_cast<double*>(reinterpret_cast<char*>(out) + TileTables<N, M, S>::tl_off());
#pragma unroll 1
        for (int e = 0; e < ne; ++e) {
#pragma unroll 1
            for (int q = 0; q < NN; ++q) {
                tl[e * 3 * NN + q] = Ac[q];
                tl[e * 3 * NN + NN + q] = Cc[q];
                tl[e * 3 * NN + 2 * NN + q] = Jc[q];
            }
            if (e + 1 == ne) break;
            fd::pair_coeffs<N>(Ac, Cc, Ac, Jc, T1, Tb, Te, T3, wk);
            fd::pair_acj<N>(Ac, Jc, Ac, Cc, T1, Tb, T3, T2, Mi, wk, wk + NN);
#pragma unroll 1
            for (int q = 0; q < NN; ++q) { Ac[q] = T2[q]; Cc[q] = Mi[q]; Jc[q] = wk[q]; }
        }
    }
    __syncthreads();
    // thread prefixes, p = j and j + KMAX: pre_p = the fold of p threads (pre_0
    // the identity) and, for p > 0, co_p.  With 2^d the lowest set bit of p,
    // pre_p = (level-d node) (x) pre_{p - 2^d}; unrolled over the set bits of p
    // from the highest (earliest threads) down, pre_p is a product of at most
    // LB level nodes.  (A sequential recurrence pre_{p+1} = fold (x) pre_p
    // compounds its rounding errors from thread to thread and is unstable for
    // models whose interval elements are ill-conditioned.)
    const int B = 1 << LB;
#pragma unroll 1
    for (int p = j; p < B; p += FL::KMAX) {
        double pA[NN], pC[NN], pJ[NN], X[NN], Y[NN], Z[NN], W[NN], nA[NN], nC[NN], nJ[NN], pw[4 * NN];
#pragma unroll 1
        for (int q = 0; q < NN; ++q) {
            pA[q] = q % (N + 1) == 0 ? 1.0 : 0.0;
            pC[q] = 0.0;
            pJ[q] = 0.0;
        }
#pragma unroll 1
        for (int d = LB - 1; d >= 0; --d) {
            if (!((p >> d) & 1)) continue;
            fd::pair_coeffs<N>(LA[d], LC[d], pA, pJ, X, Y, Z, W, pw);
            fd::pair_acj<N>(LA[d], LJ[d], pA, pC, X, Y, W, nA, nC, nJ, pw);
#pragma unroll 1
            for (int q = 0; q < NN; ++q) { pA[q] = nA[q]; pC[q] = nC[q]; pJ[q] = nJ[q]; }
        }
        // co_p: the coefficients of the last (lowest-bit) product, p = (2i+1) 2^d
        // stored as entry i of level d (lti_co_level)
        if (p > 0) {
            const int d = __ffs(p) - 1, i = p >> (d + 1), cnt = B >> (d + 1);
            S* co = out + FL::oCo + lti_co_level<N>(B, d) + i;
#pragma unroll 1
            for (int q = 0; q < NN; ++q) {
                co[q * cnt] = S(X[q]);
                co[(NN + q) * cnt] = S(Y[q]);
                co[(2 * NN + q) * cnt] = S(Z[q]);
                co[(3 * NN + q) * cnt] = S(W[q]);
            }
        }
        S* pr = out + FL::oPre + p * FL::PS;
#pragma unroll 1
        for (int a = 0; a < N; ++a) {
#pragma unroll 1
            for (int c = 0; c < N; ++c) pr[a * N + c] = S(pA[a * N + c]);
#pragma unroll 1
            for (int c = a; c < N; ++c) {
                pr[NN + Sym<N>::at(a, c)] = S(0.5 * (pC[a * N + c] + pC[c * N + a]));
                pr[NN + FL::NS + Sym<N>::at(a, c)] = S(0.5 * (pJ[a * N + c] + pJ[c * N + a]));
            }
        }
    }
}

// Tile tables of item (4): thread j computes P_j and F_j = E_j^T from the
// tile levels (written by k_lti_fold) and the prior's P_0.  FP64 throughout.
template <int N, int M, typename S>
__global__ void __launch_bounds__(64)
k_lti_tiles(const Red<N, double> prior, int nt, int ne, S* __restrict__ out)
{
    using TT = TileTables<N, M, S>;
    namespace fd = fold_detail;
    constexpr int NN = N * N;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nt) return;
    const double* tl = reinterpret_cast<const double*>(reinterpret_cast<const char*>(out) + TT::tl_off());
    double P[NN], E[NN], w[5 * NN];
#pragma unroll 1
    for (int a = 0; a < N; ++a)
#pragma unroll 1
        for (int c = 0; c < N; ++c) P[a * N + c] = prior.P[Sym<N>::at(a, c)];
#pragma unroll 1
    for (int e = ne - 1; e >= 0; --e)
        if ((j >> e) & 1) fd::riccati<N>(tl + e * 3 * NN, tl + e * 3 * NN + NN, tl + e * 3 * NN + 2 * NN, P, w);
    fd::inv_I_plus<N>(tl + NN, P, w, w + NN);            // (I + C_T P_j)^-1
    fd::mm<N>(w, tl, E);                                   // E_j
    S* tp = reinterpret_cast<S*>(reinterpret_cast<char*>(out) + TT::p_off()) + (long)j * Sym<N>::SZ;
    S* tf = reinterpret_cast<S*>(reinterpret_cast<char*>(out) + TT::f_off(nt)) + (long)j * NN;
    double* te = reinterpret_cast<double*>(reinterpret_cast<char*>(out) + TT::e_off(nt)) + (long)j * NN;
#pragma unroll 1
    for (int q = 0; q < NN; ++q) te[q] = E[q];
#pragma unroll 1
    for (int a = 0; a < N; ++a) {
#pragma unroll 1
        for (int c = a; c < N; ++c) tp[Sym<N>::at(a, c)] = S(P[a * N + c]);
#pragma unroll 1
        for (int c = 0; c < N; ++c) tf[a * N + c] = S(E[c * N + a]);
    }
}

// Products of consecutive full tiles' closed-loop maps (item (5)): thread a
// writes Pi(a, b) = E_a ... E_{b-1} for b = a..nt-1 (Pi(a, a) = I), in the
// solve's precision.  Runs after k_lti_tiles, for nt <= PI_TILES.
template <int N, int M, typename S>
__global__ void __launch_bounds__(64)
k_lti_products(int nt, S* __restrict__ out)   // any block size
{
    using TT = TileTables<N, M, S>;
    constexpr int NN = N * N;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nt) return;
    const double* E = reinterpret_cast<const double*>(reinterpret_cast<const char*>(out) + TT::e_off(nt));
    S* pi = reinterpret_cast<S*>(reinterpret_cast<char*>(out) + TT::pi_off(nt));
    S* qt = reinterpret_cast<S*>(reinterpret_cast<char*>(out) + TT::qt_off(nt));
    // products in the solve's precision (the FP64 E_j rounded): the terms that
    // matter are short products, the long ones have decayed; registers, N is a
    // compile-time size
    S P[NN], En[NN];
#pragma unroll
    for (int q = 0; q < NN; ++q) {
        P[q] = q % (N + 1) == 0 ? S(1) : S(0);
        En[q] = S(E[(long)a * NN + q]);             // E_b, loaded one step ahead
    }
#pragma unroll 1
    for (int b = a; b < nt; ++b) {
        S* o = pi + TT::pi_index(nt, a, b) * NN;
        S* ot = qt + TT::qt_index(b, a) * NN;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            o[q] = S(P[q]);
            ot[q] = S(P[(q % N) * N + q / N]);
        }
        if (b + 1 == nt) break;
        S Eb[NN], Q[NN];                            // Pi(a, b + 1) = Pi(a, b) E_b
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            Eb[q] = En[q];
            if (b + 2 < nt) En[q] = S(E[(long)(b + 1) * NN + q]);
        }
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) {
                S acc = S(0);
#pragma unroll
                for (int k = 0; k < N; ++k) acc = fma(P[i * N + k], Eb[k * N + j], acc);
                Q[i * N + j] = acc;
            }
#pragma unroll
        for (int q = 0; q < NN; ++q) P[q] = Q[q];
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

// (b, eta) nodes of a tile's tree: level d (B / 2^d nodes) starts at scalar
// 2N (2B - 2B / 2^d), component-major (component c of node j at c B / 2^d + j).
__host__ __device__ constexpr int lti_node_level(int N2, int B, int d) { return N2 * (2 * B - ((2 * B) >> d)); }

// Up-sweep of a full tile's tree on the (b, eta) parts: bq holds the nodes
// (lti_node_level; leaves stored by the caller); lv the level constants
// (FoldLayout level blocks, in shared memory).
template <int N, int M, typename S>
__device__ void lti_tree_up(S* bq, const S* lv)
{
    using FL = FoldLayout<N, M, S>;
    const int B = blockDim.x, t = threadIdx.x;
    const int LB = 31 - __clz(B);
    for (int d = 0; d < LB; ++d) {
        __syncthreads();
        const int cnt = B >> (d + 1), nd = 2 * cnt;
        if (t < cnt) {
            const S* L = lv + d * FL::LS;
            const S* ch = bq + lti_node_level(2 * N, B, d);
            S* par = bq + lti_node_level(2 * N, B, d + 1);
            S bi[N], ei[N], bj[N], ej[N];       // later child 2t+1, earlier child 2t
#pragma unroll
            for (int q = 0; q < N; ++q) {
                bi[q] = ch[q * nd + 2 * t + 1];
                ei[q] = ch[(N + q) * nd + 2 * t + 1];
                bj[q] = ch[q * nd + 2 * t];
                ej[q] = ch[(N + q) * nd + 2 * t];
            }
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
                par[a * cnt + t] = sb;
                par[(N + a) * cnt + t] = se;
            }
        }
    }
    __syncthreads();
}

// Down-sweep of the tile's tree on the (b, eta) parts, in place over the
// up-sweep nodes bq (item (3) above): on return leaf t of bq holds the (b, eta)
// of the fold of threads 0..t-1 (zero for t = 0).  A left child takes its
// parent's prefix; the right child starting at thread p takes the left
// sibling's up-sweep value combined with it through co_p (co: the table in
// shared or global memory, lti_co_level layout).  Leaf t's prefix uses only
// the leaves before t.
template <int N, int M, typename S>
__device__ void lti_tree_down_linear(S* bq, const S* co)
{
    constexpr int NN = N * N;
    const int B = blockDim.x, t = threadIdx.x;
    const int LB = 31 - __clz(B);
    if (t < 2 * N) bq[lti_node_level(2 * N, B, LB) + t] = S(0);   // root: empty prefix
    for (int d = LB - 1; d >= 0; --d) {
        __syncthreads();
        const int cnt = B >> (d + 1), nd = 2 * cnt;
        if (t < cnt) {
            const S* par = bq + lti_node_level(2 * N, B, d + 1);
            S* lvl = bq + lti_node_level(2 * N, B, d);
            const S* c = co + lti_co_level<N>(B, d) + t;
            S bD[N], eD[N], bU[N], eU[N];
#pragma unroll
            for (int q = 0; q < N; ++q) {
                bD[q] = par[q * cnt + t];
                eD[q] = par[(N + q) * cnt + t];
                bU[q] = lvl[q * nd + 2 * t];
                eU[q] = lvl[(N + q) * nd + 2 * t];
            }
#pragma unroll
            for (int a = 0; a < N; ++a) {
                S sb = bD[a], se = eU[a];
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    sb = fma(c[(a * N + k) * cnt], bU[k], sb);
                    sb = fma(c[(NN + a * N + k) * cnt], eD[k], sb);
                    se = fma(c[(2 * NN + a * N + k) * cnt], eD[k], se);
                    se = fma(-c[(3 * NN + a * N + k) * cnt], bU[k], se);
                }
                lvl[a * nd + 2 * t + 1] = sb;
                lvl[(N + a) * nd + 2 * t + 1] = se;
            }
#pragma unroll
            for (int q = 0; q < N; ++q) {
                lvl[q * nd + 2 * t] = bD[q];
                lvl[(N + q) * nd + 2 * t] = eD[q];
            }
        }
    }
    __syncthreads();
}

// Value function before the first step of thread t of the tile: its prefix
// D_t (constants pre_t, (b, eta) from the down-sweep at dleaf) applied to the
// tile's prefix pin (one-variable combine, Eq. 36); thread 0 takes pin itself.
template <int N, int M, typename S>
__device__ __forceinline__ void lti_thread_value(const S* __restrict__ fold, const S (&dleaf)[2 * N],
                                                 const Red<N, S>& pin, const CombineCtx& ctx, Red<N, S>& X)
{
    using FL = FoldLayout<N, M, S>;
    X = pin;
    if (threadIdx.x == 0) return;
    const S* pr = fold + FL::oPre + threadIdx.x * FL::PS;
    Elem<N, S> D;
#pragma unroll
    for (int q = 0; q < N * N; ++q) D.A[q] = __ldg(pr + q);
#pragma unroll
    for (int q = 0; q < Sym<N>::SZ; ++q) { D.C[q] = __ldg(pr + N * N + q); D.J[q] = __ldg(pr + N * N + FL::NS + q); }
#pragma unroll
    for (int q = 0; q < N; ++q) { D.b[q] = dleaf[q]; D.eta[q] = dleaf[N + q]; }
    apply<N, S, false>(D, X, nullptr, nullptr, ctx);
}

// Shared memory of the linear-fold down-sweep kernels (offsets in scalars of
// S).  A work area at 0, reused in turn by the tile-prefix affine tree, the
// (b, eta) tree with the tile's prefix value node after it, the last tile's
// staged Gamma_i, and the tile's own affine tree; then the tree level
// constants (levels 0..LB-1) and, with co_smem, the co table (entries
// 0..B-1), both staged before the wait for the preceding kernel.
template <int N, int M, typename S>
struct LtiDownSmem {
    using FL = FoldLayout<N, M, S>;
    __host__ __device__ static constexpr int al(int x) { return (x + 3) / 4 * 4; }
    __host__ __device__ static constexpr int mx(int a, int b) { return a > b ? a : b; }
    __host__ __device__ static constexpr int lb(int B) { return B >= 128 ? 7 : B >= 64 ? 6 : B >= 32 ? 5 : B >= 16 ? 4 : 3; }
    __host__ __device__ static constexpr int bq(int) { return 0; }
    __host__ __device__ static constexpr int pin(int B) { return 2 * B * 2 * N; }
    __host__ __device__ static constexpr int lv(int B, int K)
    {
        return al(mx(mx(pin(B) + CoopLayout<N, S>::NR, K * FL::GS), 2 * B * CoopLayout<N, S>::NA));
    }
    __host__ __device__ static constexpr int co(int B, int K) { return lv(B, K) + al(lb(B) * FL::LS); }
    __host__ __device__ static constexpr size_t bytes(int B, int K, bool co_smem)
    {
        return sizeof(S) * (size_t)(co(B, K) + (co_smem ? B * FL::CS : 0));
    }
};

// Stage the level constants and (co_smem) the co table into shared memory;
// copies of 16-byte words (both tables start at multiples of 4 scalars)
template <int N, int M, typename S>
__device__ __forceinline__ void lti_stage_tables(const LtiTiles<S>& lt, int K, S* sm)
{
    using FL = FoldLayout<N, M, S>;
    using DS = LtiDownSmem<N, M, S>;
    using V = typename std::conditional<sizeof(S) == 4, float4, double2>::type;
    constexpr int W = 16 / sizeof(S);
    const int B = blockDim.x, t = threadIdx.x, LB = 31 - __clz(B);
    const V* src = reinterpret_cast<const V*>(lt.fold + FL::oL);
    V* dst = reinterpret_cast<V*>(sm + DS::lv(B, K));
    for (int q = t; q < (LB * FL::LS) / W; q += B) dst[q] = src[q];
    if (lt.co_smem) {
        src = reinterpret_cast<const V*>(lt.fold + FL::oCo);
        dst = reinterpret_cast<V*>(sm + DS::co(B, K));
        for (int q = t; q < ((B - 1) * FL::CS) / W; q += B) dst[q] = src[q];
    }
}

}  // namespace mapk
