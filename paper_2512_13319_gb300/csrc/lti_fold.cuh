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
// N x N matrices) and of the tree levels' children (LMAX + 1), then P_j (packed, scalars of S) and F_j = E_j^T (N x N
// row-major) for j < nt, and for scans of at most PI_TILES tiles
// the products Pi(a, b) of consecutive tiles' closed-loop maps (item (5)) by
// rows (a) and their transposes by columns (b).
template <int N, int M, typename S>
struct TileTables {
    static constexpr int ELMAX = 24;                        // up to 2^24 tiles
    static constexpr int NN = N * N, NS = Sym<N>::SZ;
    __host__ __device__ static constexpr size_t al(size_t x) { return (x + 15) / 16 * 16; }
    __host__ __device__ static constexpr size_t tl_off() { return al(sizeof(S) * FoldLayout<N, M, S>::TOTAL); }
    // tile levels e < ELMAX, then the tree levels d <= LMAX at ELMAX + d
    __host__ __device__ static constexpr size_t p_off()
    {
        return tl_off() + sizeof(double) * (ELMAX + FoldLayout<N, M, S>::LMAX + 1) * 3 * NN;
    }
    __host__ __device__ static constexpr size_t f_off(long nt) { return p_off() + al(sizeof(S) * nt * NS); }
    // then (scans of at most PI_TILES tiles) the products
    // Pi(a, b) = E_a E_{a+1} ... E_{b-1}, 0 <= a <= b < nt, row a holding b = a..nt-1
    static constexpr long PI_TILES = 4 * 128 + 1;
    __host__ __device__ static constexpr size_t pi_off(long nt) { return al(f_off(nt) + sizeof(S) * nt * NN); }
    __host__ __device__ static constexpr long pi_index(long nt, long a, long b) { return a * nt - a * (a - 1) / 2 + (b - a); }
    // then the transposes Q(b, a) = Pi(a, b)^T, row b holding a = 0..b
    __host__ __device__ static constexpr size_t qt_off(long nt) { return pi_off(nt) + sizeof(S) * (size_t)(nt * (nt + 1) / 2) * NN; }
    __host__ __device__ static constexpr long qt_index(long b, long a) { return b * (b + 1) / 2 + a; }
    // then the segment products G(c) = Pi(c, c + PI_SEG) (k_lti_segments)
    static constexpr int PI_SEG = 16;
    __host__ __device__ static constexpr size_t g_off(long nt)
    {
        return pi_off(nt) + al(2 * sizeof(S) * (size_t)(nt * (nt + 1) / 2) * NN);
    }
    __host__ __device__ static constexpr size_t bytes(long nt)
    {
        return nt <= PI_TILES ? g_off(nt) + sizeof(S) * (size_t)nt * NN : pi_off(nt);
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

// Plan-time helpers of the constant kernels, in FP64 and warp-cooperative: a
// whole warp calls each one with the same arguments, lane l computes entries
// l, l + 32, ... of the result, and a __syncwarp() at the end makes the result
// visible to every lane.  Matrices are n x n row-major (n a compile-time size);
// inputs may be in global or shared memory, outputs are in shared memory and
// never alias an input.  The FP64 pipe of an SM sub-partition takes a warp
// instruction at about the same cost however many of its lanes are active, so
// a product spread over the lanes (one entry per lane) issues n FP64
// instructions per lane-round instead of n^3 in one thread.
namespace fold_warp {

__device__ inline int lane() { return threadIdx.x & 31; }

// |x| ordering of finite FP64 values through their bit patterns (no FP64 op)
__device__ inline unsigned long long absbits(double x)
{
    return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
}

// c = a b
template <int n>
__device__ inline void mm(const double* a, const double* b, double* c)
{
    for (int q = lane(); q < n * n; q += 32) {
        const int i = q / n, j = q - i * n;
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) s = fma(a[i * n + k], b[k * n + j], s);
        c[q] = s;
    }
    __syncwarp();
}

// c = a b + d
template <int n>
__device__ inline void mm_add(const double* a, const double* b, const double* d, double* c)
{
    for (int q = lane(); q < n * n; q += 32) {
        const int i = q / n, j = q - i * n;
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) s = fma(a[i * n + k], b[k * n + j], s);
        c[q] = s + d[q];
    }
    __syncwarp();
}

// c = (a b)^T
template <int n>
__device__ inline void mm_t(const double* a, const double* b, double* c)
{
    for (int q = lane(); q < n * n; q += 32) {
        const int i = q / n, j = q - i * n;         // c[i][j] = (a b)[j][i]
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) s = fma(a[j * n + k], b[k * n + i], s);
        c[q] = s;
    }
    __syncwarp();
}

// c = a b^T
template <int n>
__device__ inline void mm_bt(const double* a, const double* b, double* c)
{
    for (int q = lane(); q < n * n; q += 32) {
        const int i = q / n, j = q - i * n;
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) s = fma(a[i * n + k], b[j * n + k], s);
        c[q] = s;
    }
    __syncwarp();
}

// dst = src (n x n)
template <int n>
__device__ inline void copy(const double* src, double* dst)
{
    for (int q = lane(); q < n * n; q += 32) dst[q] = src[q];
    __syncwarp();
}

// out = (I + c j)^-1 by Gauss-Jordan elimination with row pivoting on the
// augmented [I + c j | I]; X: n^2 scratch
template <int n>
__device__ inline void inv_I_plus(const double* c, const double* j, double* out, double* X)
{
    for (int q = lane(); q < n * n; q += 32) {
        const int i = q / n, k = q - i * n;
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < n; ++t) s = fma(c[i * n + t], j[t * n + k], s);
        if (i == k) s += 1.0;
        X[q] = s;
        out[q] = i == k ? 1.0 : 0.0;
    }
    __syncwarp();
    constexpr int E = 2 * n * n, R = (E + 31) / 32;
#pragma unroll 1
    for (int col = 0; col < n; ++col) {
        int piv = col;                              // first row of largest magnitude
        unsigned long long best = absbits(X[col * n + col]);
#pragma unroll
        for (int r = col + 1; r < n; ++r) {
            const unsigned long long v = absbits(X[r * n + col]);
            if (v > best) { best = v; piv = r; }
        }
        const double p = X[piv * n + col];
        const double ip = p != 0.0 ? 1.0 / p : 0.0;
        // rows col and piv swapped, row col scaled by ip, column col
        // eliminated from the other rows: all reads first, then all writes
        double nv[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int e = lane() + 32 * t;
            if (e < E) {
                const int r = e / (2 * n), k = e - r * 2 * n;
                const double* A = k < n ? X : out;
                const int kk = k < n ? k : k - n;
                const double pk = A[piv * n + kk] * ip;
                const int sr = r == piv ? col : r;
                nv[t] = r == col ? pk : fma(-X[sr * n + col], pk, A[sr * n + kk]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int e = lane() + 32 * t;
            if (e < E) {
                const int r = e / (2 * n), k = e - r * 2 * n;
                (k < n ? X : out)[r * n + (k < n ? k : k - n)] = nv[t];
            }
        }
        __syncwarp();
    }
}

// coefficients of the (b, eta) part of U (x) D (U the later operand):
// Mi = (I + C_U J_D)^-1, X = A_D Mi, Y = X C_U, Z = (Mi A_U)^T, W = Z J_D;
// wk: 2 n^2 scratch
template <int n>
__device__ inline void pair_coeffs(const double* AU, const double* CU, const double* AD, const double* JD,
                                   double* X, double* Y, double* Z, double* W, double* wk)
{
    double* Mi = wk;
    inv_I_plus<n>(CU, JD, Mi, wk + n * n);
    mm<n>(AD, Mi, X);
    mm<n>(X, CU, Y);
    mm_t<n>(Mi, AU, Z);
    mm<n>(Z, JD, W);
}

// (A, C, J) of U (x) D from the coefficients of pair_coeffs:
// A = X A_U, C = Y A_D^T + C_D, J = W A_U + J_U
template <int n>
__device__ inline void pair_acj(const double* AU, const double* JU, const double* AD, const double* CD,
                                const double* X, const double* Y, const double* W, double* Ao, double* Co,
                                double* Jo)
{
    mm<n>(X, AU, Ao);
    for (int q = lane(); q < n * n; q += 32) {
        const int i = q / n, j = q - i * n;
        double s = 0.0, u = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            s = fma(Y[i * n + k], AD[j * n + k], s);
            u = fma(W[i * n + k], AU[k * n + j], u);
        }
        Co[q] = s + CD[q];
        Jo[q] = u + JU[q];
    }
    __syncwarp();
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
    for (int q = lane(); q < n * n; q += 32) {
        const int i = q / n, j = q - i * n;
        double s = J[q];
#pragma unroll
        for (int k = 0; k < n; ++k) s = fma(A[k * n + i], T2[k * n + j], s);
        Mi[q] = s;
    }
    __syncwarp();
    for (int q = lane(); q < n * n; q += 32) {
        const int i = q / n, j = q - i * n;
        P[q] = 0.5 * (Mi[i * n + j] + Mi[j * n + i]);
    }
    __syncwarp();
}

}  // namespace fold_warp

// One warp, lane-parallel FP64 (fold_warp).  The K-step fold: its (A, C, J)
// and the per-step maps (Tb_i, Te_i) of item (1) forward; the Gamma_j then
// backward, Gamma_j = R_j (0; G) with R_j = U_{K-1} ... U_{j+1} and U_i the map
// (b, eta) -> (b + Tb_i eta, Te_i eta) of step i.  Then the tree levels of
// item (2) (also kept in FP64 for k_lti_tables) and the tile levels of item
// (4).  LB: log2 of the threads per tile (B = 2^LB <= BMAX); ne: the tile
// levels to write (2^ne above every tile index).
template <int N, int M, typename S>
__global__ void __launch_bounds__(32)
k_lti_fold(const LtiParams<N, M, double> p, int K, int LB, int ne, S* __restrict__ out)
{
    using FL = FoldLayout<N, M, S>;
    using CL = CoopLayout<N, S>;
    using TT = TileTables<N, M, S>;
    namespace fw = fold_warp;
    constexpr int NN = N * N;
    __shared__ double Ac[NN], Cc[NN], Jc[NN], Ae[NN], Ce[NN], Je[NN], Mi[NN], T1[NN], T2[NN], wk[2 * NN];
    __shared__ double X[NN], Y[NN], Z[NN], W[NN], Rb[2][NN], Re[2][NN];
    __shared__ double ob[N], oe[N], be[N], Gr[N], u[N], Gm[N * M];
    __shared__ double Tb[FL::KMAX][NN], Te[FL::KMAX][NN];
    const int l = fw::lane();
    double* tl = reinterpret_cast<double*>(reinterpret_cast<char*>(out) + TT::tl_off());
    for (int q = l; q < NN; q += 32) {
        const int a = q / N, c = q - a * N;
        Ae[q] = Ac[q] = p.A[q];
        Ce[q] = Cc[q] = p.C[Sym<N>::at(a, c)];
        Je[q] = Jc[q] = p.J[Sym<N>::at(a, c)];
    }
    for (int q = l; q < N * M; q += 32) Gm[q] = p.G[q];
    if (l < N) {
        be[l] = ob[l] = p.b[l];
        Gr[l] = p.Gr[l];
        oe[l] = -p.Gr[l];
    }
    __syncwarp();
#pragma unroll 1
    for (int i = 1; i < K; ++i) {
        fw::inv_I_plus<N>(Ce, Jc, Mi, wk);      // (I + C_e J_acc)^-1
        fw::mm<N>(Ac, Mi, T1);                  // A_acc Mi
        fw::mm<N>(T1, Ce, Tb[i]);               // Tb = A_acc Mi C_e
        fw::mm_t<N>(Mi, Ae, Te[i]);             // Te = (Mi A_e)^T
        // offsets: b <- b + Tb eta + A_acc Mi b_e;  eta <- Te (eta - J_acc b_e) - Gr
        if (l < N) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < N; ++k) s = fma(Jc[l * N + k], be[k], s);
            u[l] = oe[l] - s;
        }
        __syncwarp();
        double nb = 0.0, nq = 0.0;
        if (l < N) {
            double te = 0.0, tb = 0.0, tm = 0.0;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                te = fma(Te[i][l * N + k], u[k], te);
                tb = fma(Tb[i][l * N + k], oe[k], tb);
                tm = fma(T1[l * N + k], be[k], tm);
            }
            nb = ob[l] + tb + tm;
            nq = te - Gr[l];
        }
        // composite: A = A_acc Mi A_e, C = Tb A_acc^T + C_acc, J = Te J_acc A_e + J_e
        fw::mm<N>(T1, Ae, T2);                  // new A
        fw::mm_bt<N>(Tb[i], Ac, X);             // Tb A_acc^T
        fw::mm<N>(Jc, Ae, Y);
        fw::mm_add<N>(Te[i], Y, Je, Z);         // new J
        for (int q = l; q < NN; q += 32) {
            Ac[q] = T2[q];
            Cc[q] += X[q];
            Jc[q] = Z[q];
        }
        if (l < N) { ob[l] = nb; oe[l] = nq; }
        __syncwarp();
    }
    for (int q = l; q < NN; q += 32) {
        const int a = q / N, c = q - a * N;
        out[FL::oA + q] = S(Ac[q]);
        if (c >= a) {
            out[FL::oC + Sym<N>::at(a, c)] = S(0.5 * (Cc[a * N + c] + Cc[c * N + a]));
            out[FL::oJ + Sym<N>::at(a, c)] = S(0.5 * (Jc[a * N + c] + Jc[c * N + a]));
        }
    }
    if (l < N) {
        out[FL::ob + l] = S(ob[l]);
        out[FL::oe + l] = S(oe[l]);
    }
    // Gamma_j, j = K-1 down to 0: R_{K-1} = I, i.e. (Rb, Re) = (0, I), and
    // R_{j-1} = R_j U_j: Rb <- Tb_j + Rb Te_j, Re <- Re Te_j
    for (int q = l; q < NN; q += 32) {
        Rb[0][q] = 0.0;
        Re[0][q] = q % (N + 1) == 0 ? 1.0 : 0.0;
    }
    __syncwarp();
    int cur = 0;
#pragma unroll 1
    for (int j = K - 1; j >= 0; --j) {
        S* g = out + FL::oG + j * FL::GS;       // rows 0..N-1: Rb G, rows N..2N-1: Re G
        for (int q = l; q < 2 * N * M; q += 32) {
            const bool top = q < N * M;
            const int r = (top ? q : q - N * M) / M, c = (top ? q : q - N * M) % M;
            const double* Rm = top ? Rb[cur] : Re[cur];
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < N; ++k) s = fma(Rm[r * N + k], Gm[k * M + c], s);
            g[q] = S(s);
        }
        if (j == 0) break;
        for (int q = l; q < 2 * NN; q += 32) {
            const bool top = q < NN;
            const int qq = top ? q : q - NN, a = qq / N, c = qq - a * N;
            const double* Rm = top ? Rb[cur] : Re[cur];
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < N; ++k) s = fma(Rm[a * N + k], Te[j][k * N + c], s);
            (top ? Rb[cur ^ 1] : Re[cur ^ 1])[qq] = top ? Tb[j][qq] + s : s;
        }
        __syncwarp();
        cur ^= 1;
    }
    // tree levels: level d holds the constants of its children
#pragma unroll 1
    for (int d = 0; d <= LB && d <= FL::LMAX; ++d) {
        S* lv = out + FL::oL + d * FL::LS;
        double* lf = tl + (TT::ELMAX + d) * 3 * NN;
        for (int q = l; q < NN; q += 32) { lf[q] = Ac[q]; lf[NN + q] = Cc[q]; lf[2 * NN + q] = Jc[q]; }
        for (int q = l; q < N * CL::P; q += 32) {
            const int a = q / CL::P, c = q - a * CL::P;
            const bool in = c < N;
            lv[CL::oA + q] = in ? S(Ac[a * N + c]) : S(0);
            lv[CL::oC + q] = in ? S(0.5 * (Cc[a * N + c] + Cc[c * N + a])) : S(0);
            lv[CL::oJ + q] = in ? S(0.5 * (Jc[a * N + c] + Jc[c * N + a])) : S(0);
        }
        if (d == LB) break;
        fw::pair_coeffs<N>(Ac, Cc, Ac, Jc, X, Y, Z, W, wk);
        for (int q = l; q < NN; q += 32) {
            lv[FL::oX + q] = S(X[q]);
            lv[FL::oY + q] = S(Y[q]);
            lv[FL::oZ + q] = S(Z[q]);
            lv[FL::oW + q] = S(W[q]);
        }
        fw::pair_acj<N>(Ac, Jc, Ac, Cc, X, Y, W, T1, T2, Mi);
        for (int q = l; q < NN; q += 32) { Ac[q] = T1[q]; Cc[q] = T2[q]; Jc[q] = Mi[q]; }
        __syncwarp();
    }
    // tile levels (item (4)): (Ac, Cc, Jc) now hold the full tile
#pragma unroll 1
    for (int e = 0; e < ne; ++e) {
        for (int q = l; q < NN; q += 32) {
            tl[e * 3 * NN + q] = Ac[q];
            tl[e * 3 * NN + NN + q] = Cc[q];
            tl[e * 3 * NN + 2 * NN + q] = Jc[q];
        }
        if (e + 1 == ne) break;
        fw::pair_coeffs<N>(Ac, Cc, Ac, Jc, X, Y, Z, W, wk);
        fw::pair_acj<N>(Ac, Jc, Ac, Cc, X, Y, W, T1, T2, Mi);
        for (int q = l; q < NN; q += 32) { Ac[q] = T1[q]; Cc[q] = T2[q]; Jc[q] = Mi[q]; }
        __syncwarp();
    }
}

// Per-warp shared scratch of k_lti_tables
template <int N>
union LtiTablesWk {
    struct { double A[N * N], C[N * N], J[N * N], X[N * N], Y[N * N], Z[N * N], W[N * N], nA[N * N], nC[N * N],
             nJ[N * N], s[2 * N * N]; } pre;
    struct { double P[N * N], E[N * N], Mi[N * N], s[4 * N * N]; } tile;
};

// Thread-prefix tables of item (3), by one warp for p (0 <= p < B): pre_p =
// the fold of p threads (pre_0 the identity) and, for p > 0, co_p.  With 2^d
// the lowest set bit of p, pre_p = (level-d node) (x) pre_{p - 2^d}; unrolled
// over the set bits of p from the highest (earliest threads) down, pre_p is a
// product of at most LB level nodes (the FP64 levels that k_lti_fold wrote).
// (A sequential recurrence pre_{p+1} = fold (x) pre_p compounds its rounding
// errors from thread to thread and is unstable for models whose interval
// elements are ill-conditioned.)
template <int N, int M, typename S>
__device__ void lti_prefix_warp(int pidx, int LB, S* __restrict__ out, LtiTablesWk<N>& wk)
{
    using FL = FoldLayout<N, M, S>;
    using TT = TileTables<N, M, S>;
    namespace fw = fold_warp;
    constexpr int NN = N * N;
    auto& w = wk.pre;
    const int l = fw::lane(), B = 1 << LB;
    const double* tl = reinterpret_cast<const double*>(reinterpret_cast<const char*>(out) + TT::tl_off());
    for (int q = l; q < NN; q += 32) {
        w.A[q] = q % (N + 1) == 0 ? 1.0 : 0.0;
        w.C[q] = 0.0;
        w.J[q] = 0.0;
    }
    __syncwarp();
#pragma unroll 1
    for (int d = LB - 1; d >= 0; --d) {
        if (!((pidx >> d) & 1)) continue;
        const double* LA = tl + (TT::ELMAX + d) * 3 * NN;
        fw::pair_coeffs<N>(LA, LA + NN, w.A, w.J, w.X, w.Y, w.Z, w.W, w.s);
        fw::pair_acj<N>(LA, LA + 2 * NN, w.A, w.C, w.X, w.Y, w.W, w.nA, w.nC, w.nJ);
        fw::copy<N>(w.nA, w.A);
        fw::copy<N>(w.nC, w.C);
        fw::copy<N>(w.nJ, w.J);
    }
    // co_p: the coefficients of the last (lowest-bit) product, p = (2i+1) 2^d
    // stored as entry i of level d (lti_co_level)
    if (pidx > 0) {
        const int d = __ffs(pidx) - 1, i = pidx >> (d + 1), cnt = B >> (d + 1);
        S* co = out + FL::oCo + lti_co_level<N>(B, d) + i;
        for (int q = l; q < NN; q += 32) {
            co[q * cnt] = S(w.X[q]);
            co[(NN + q) * cnt] = S(w.Y[q]);
            co[(2 * NN + q) * cnt] = S(w.Z[q]);
            co[(3 * NN + q) * cnt] = S(w.W[q]);
        }
    }
    S* pr = out + FL::oPre + pidx * FL::PS;
    for (int q = l; q < NN; q += 32) {
        const int a = q / N, c = q - a * N;
        pr[q] = S(w.A[q]);
        if (c >= a) {
            pr[NN + Sym<N>::at(a, c)] = S(0.5 * (w.C[a * N + c] + w.C[c * N + a]));
            pr[NN + FL::NS + Sym<N>::at(a, c)] = S(0.5 * (w.J[a * N + c] + w.J[c * N + a]));
        }
    }
}

// Tile tables of item (4), by one warp for tile j: P_j and F_j = E_j^T from
// the tile levels (written by k_lti_fold) and the prior's P_0.  FP64.
template <int N, int M, typename S>
__device__ void lti_tile_warp(int j, const Red<N, double>& prior, int nt, int ne, S* __restrict__ out,
                              LtiTablesWk<N>& wk)
{
    using TT = TileTables<N, M, S>;
    namespace fw = fold_warp;
    constexpr int NN = N * N;
    auto& w = wk.tile;
    const int l = fw::lane();
    const double* tl = reinterpret_cast<const double*>(reinterpret_cast<const char*>(out) + TT::tl_off());
    for (int q = l; q < NN; q += 32) {
        const int a = q / N, c = q - a * N;
        w.P[q] = prior.P[Sym<N>::at(a, c)];
    }
    __syncwarp();
#pragma unroll 1
    for (int e = ne - 1; e >= 0; --e)
        if ((j >> e) & 1) fw::riccati<N>(tl + e * 3 * NN, tl + e * 3 * NN + NN, tl + e * 3 * NN + 2 * NN, w.P, w.s);
    fw::inv_I_plus<N>(tl + NN, w.P, w.Mi, w.s);           // (I + C_T P_j)^-1
    fw::mm<N>(w.Mi, tl, w.E);                               // E_j
    S* tp = reinterpret_cast<S*>(reinterpret_cast<char*>(out) + TT::p_off()) + (long)j * Sym<N>::SZ;
    S* tf = reinterpret_cast<S*>(reinterpret_cast<char*>(out) + TT::f_off(nt)) + (long)j * NN;
    for (int q = l; q < NN; q += 32) {
        const int a = q / N, c = q - a * N;
        if (c >= a) tp[Sym<N>::at(a, c)] = S(w.P[q]);
        tf[q] = S(w.E[c * N + a]);
    }
}

// The tables of items (3) and (4) side by side, one warp per item, four warps
// per block of 128 threads: blocks 0 .. B/4 - 1 (rounded up) take the thread
// prefixes p, the rest the tiles j, so that both spread over the SMs' FP64
// pipes at once.  Runs after k_lti_fold.
template <int N, int M, typename S>
__global__ void __launch_bounds__(128)
k_lti_tables(const Red<N, double> prior, int LB, int nt, int ne, S* __restrict__ out)
{
    constexpr int WPB = 4;
    __shared__ LtiTablesWk<N> wks[WPB];
    const int wi = threadIdx.x >> 5;
    const int B = 1 << LB, pre_blocks = (B + WPB - 1) / WPB;
    if (wi >= WPB) return;
    if ((int)blockIdx.x < pre_blocks) {
        const int pidx = blockIdx.x * WPB + wi;
        if (pidx < B) lti_prefix_warp<N, M, S>(pidx, LB, out, wks[wi]);    // warp-uniform
    } else {
        const int j = ((int)blockIdx.x - pre_blocks) * WPB + wi;
        if (j < nt) lti_tile_warp<N, M, S>(j, prior, nt, ne, out, wks[wi]);
    }
}

// Products of consecutive full tiles' closed-loop maps (item (5)),
// Pi(a, b) = E_a ... E_{b-1} for 0 <= a <= b < nt (Pi(a, a) = I), in the
// solve's precision (from the tile table F_j = E_j^T: the terms that matter
// are short products, the long ones have decayed).  A row's chain is cut into segments
// of PI_SEG tiles so that no thread walks more than about nt / PI_SEG + PI_SEG
// factors: k_lti_segments forms G(c) = Pi(c, c + PI_SEG), then thread (a, s)
// of k_lti_products starts from Pi(a, a + s PI_SEG) = G(a) G(a + PI_SEG) ...
// and walks the E_b of its segment.  Run after k_lti_tables, for nt <= PI_TILES.
namespace products_detail {
// E_j from F_j = E_j^T (the tile table in the solve's precision)
template <int N, typename S>
__device__ inline void load_E(const S* F, long j, S (&e)[N * N])
{
#pragma unroll
    for (int q = 0; q < N * N; ++q) e[q] = F[j * N * N + (q % N) * N + q / N];
}
template <int N, typename S>
__device__ inline void mul(S (&P)[N * N], const S (&F)[N * N])   // P <- P F
{
    S Q[N * N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            S acc = S(0);
#pragma unroll
            for (int k = 0; k < N; ++k) acc = fma(P[i * N + k], F[k * N + j], acc);
            Q[i * N + j] = acc;
        }
#pragma unroll
    for (int q = 0; q < N * N; ++q) P[q] = Q[q];
}
}  // namespace products_detail

template <int N, int M, typename S>
__global__ void __launch_bounds__(128)
k_lti_segments(int nt, S* __restrict__ out)   // thread c, any block size
{
    using TT = TileTables<N, M, S>;
    namespace pd = products_detail;
    constexpr int NN = N * N, L = TT::PI_SEG;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c + L > nt - 1) return;                 // G(c) uses E_c .. E_{c+L-1}, E_{nt-2} the last
    const S* E = reinterpret_cast<const S*>(reinterpret_cast<const char*>(out) + TT::f_off(nt));
    S* G = reinterpret_cast<S*>(reinterpret_cast<char*>(out) + TT::g_off(nt)) + (long)c * NN;
    S P[NN], En[NN];
    pd::load_E<N>(E, c, P);
    pd::load_E<N>(E, c + 1, En);                // one factor ahead
#pragma unroll 1
    for (int b = c + 1; b < c + L; ++b) {
        S Eb[NN];
#pragma unroll
        for (int q = 0; q < NN; ++q) Eb[q] = En[q];
        if (b + 1 < c + L) pd::load_E<N>(E, b + 1, En);
        pd::mul<N>(P, Eb);
    }
#pragma unroll
    for (int q = 0; q < NN; ++q) G[q] = P[q];
}

// thread (a, s): threadIdx.x / 8 + 4 blockIdx.y = a, threadIdx.x % 8 + 8 blockIdx.x = s
// (blocks of 32 threads)
template <int N, int M, typename S>
__global__ void __launch_bounds__(32)
k_lti_products(int nt, S* __restrict__ out)
{
    using TT = TileTables<N, M, S>;
    namespace pd = products_detail;
    constexpr int NN = N * N, L = TT::PI_SEG;
    const int a = blockIdx.y * 4 + (threadIdx.x >> 3), sg = blockIdx.x * 8 + (threadIdx.x & 7);
    const int b0 = a + sg * L;
    if (a >= nt || b0 > nt - 1) return;
    const int b1 = min(b0 + L, nt);             // this thread writes Pi(a, b), b0 <= b < b1
    const S* E = reinterpret_cast<const S*>(reinterpret_cast<const char*>(out) + TT::f_off(nt));
    const S* G = reinterpret_cast<const S*>(reinterpret_cast<const char*>(out) + TT::g_off(nt));
    S* pi = reinterpret_cast<S*>(reinterpret_cast<char*>(out) + TT::pi_off(nt));
    S* qt = reinterpret_cast<S*>(reinterpret_cast<char*>(out) + TT::qt_off(nt));
    S P[NN], Fn[NN];
#pragma unroll
    for (int q = 0; q < NN; ++q) P[q] = q % (N + 1) == 0 ? S(1) : S(0);
    // Pi(a, b0) = G(a) G(a + L) ... G(a + (sg - 1) L), the next factor loaded ahead
    if (sg > 0) {
#pragma unroll
        for (int q = 0; q < NN; ++q) Fn[q] = G[(long)a * NN + q];
    }
#pragma unroll 1
    for (int t = 0; t < sg; ++t) {
        S Ft[NN];
#pragma unroll
        for (int q = 0; q < NN; ++q) Ft[q] = Fn[q];
        if (t + 1 < sg) {
#pragma unroll
            for (int q = 0; q < NN; ++q) Fn[q] = G[(long)(a + (t + 1) * L) * NN + q];
        }
        pd::mul<N>(P, Ft);
    }
    if (b0 + 1 < b1) pd::load_E<N>(E, b0, Fn);
#pragma unroll 1
    for (int b = b0; b < b1; ++b) {
        S* o = pi + TT::pi_index(nt, a, b) * NN;
        S* ot = qt + TT::qt_index(b, a) * NN;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            o[q] = P[q];
            ot[q] = P[(q % N) * N + q / N];
        }
        if (b + 1 == b1) break;
        S Eb[NN];                                   // Pi(a, b + 1) = Pi(a, b) E_b
#pragma unroll
        for (int q = 0; q < NN; ++q) Eb[q] = Fn[q];
        if (b + 2 < b1) pd::load_E<N>(E, b + 1, Fn);
        pd::mul<N>(P, Eb);
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
