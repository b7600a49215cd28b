// Per-step tables of a linear time-invariant model and the single-launch RTS
// solve that reads them.
//
// For an LTI model every interval element has the same (A, b, C, J) and only
// eta_k = G y_k - Gr depends on the observations (Section 4.2 elements).  In
// the one-variable combine (Eq. 36) that moves the filter value function
// V_k(x) = 1/2 x^T P_k x - v_k^T x across interval k,
//   P_{k+1} = A^T P_k (I + C P_k)^-1 A + J,
//   v_{k+1} = E_k^T (v_k - P_k b) + eta_k,
// and in the closed-loop map of the RTS pass (Section 4.3, Eq. 40-42)
//   x_k = E_k x_{k+1} + g_k,  E_k = (I + C P_k)^-1 A,  g_k = (I + C P_k)^-1 (b + C v_k),
// the P_k recursion, and with it E_k and P_k b, do not depend on the data.
// They are evaluated once per model in FP64 (k_lti_steptab), and a solve runs
// only the data-dependent part of every step.  With (I + C P_k)^-1 = E_k A^-1:
//   forward (filter):    v_{k+1} = E_k^T v_k + o_k + G y_{k+1} - Gr,  o_k = -E_k^T P_k b
//   closed-loop offset:  g_k = E_k (A^-1 C v_k + A^-1 b)
//   backward (RTS):      x_k = E_k x_{k+1} + g_k.
// This is the same combine evaluated with its data-independent factors
// precomputed (as lti_fold.cuh does for folds and tile tables).
//
// P_k converges to the fixed point of the recursion (the stationary filter)
// geometrically.  The table holds the steps k < KT (KT = min(T + 1, a cap), so
// that a short scan has its every P_k up to P_T); when T >= KT, row kc stands
// for every later step, where kc is the first step from which every tabulated
// P_k agrees with the P of the uniform decomposition's last full tile to a
// relative tolerance of 2^-25 (FP32 solves: below the solve's own rounding)
// or 1e-12 (FP64 solves: three orders below their 1e-9 accuracy target, and
// above the rounding noise of the FP64 tables themselves) per entry
// (|dP_ab| <= tol sqrt(P_aa P_bb)).  When the
// table does not reach that point (slowly converging models) the solve keeps
// the per-step combine paths of scan.cuh.
//
// Every tabulated P_k is formed independently of the others from the FP64
// plan-time tables of lti_fold.cuh: the value function before tile j (P_j),
// the fold of s threads (pre_s) and the fold of i steps (f_i), with
// k = j B K + s K + i:  P_k = apply(f_i, apply(pre_s, P_j)).  Each apply, and
// the per-step constants, use the factor Z = R^-1 L^T (P = L L^T and
// R R^T = I + L^T C L, both Cholesky factors of symmetric positive definite
// matrices, the second with eigenvalues >= 1):
//   P (I + C P)^-1 = (P^-1 + C)^-1 = Z^T Z,   (I + C P)^-1 = I - C Z^T Z,
// so no pivoting is needed and every lane of a warp runs the same instructions.
//
// The solve (k_lti_scan) is a scan of affine maps.  A thread owns consecutive
// steps; its filter map v -> Psi v + W (Psi = Phi^T, Phi = E_{k0} ... E_{k0+K-1}
// the composition of its closed-loop maps, data-independent) and its RTS map
// x -> Phi x + beta compose over the threads of a tile and over the tiles.
// Only the offsets W and beta depend on the data.  Tiles whose threads all
// start after kc share Phi = Phi_inf, so the linear parts of every partial
// composition inside such a tile are powers Phi_inf^d (a plan-time table of
// B + 1 matrices) and the in-tile scans run on offsets alone (one N x N
// matrix-vector product per shuffle level).  The first tiles (before kc) take
// K_t = 16 / sizeof(S) steps per thread, read their per-step E_k (and P_k b)
// from shared memory (one bulk copy per tile) and compose full maps, as does
// the last tile.
#pragma once
#include "scan.cuh"

namespace mapk {

// Layout of the step-table buffer (offsets in bytes): a few counters, the
// FP64 element powers e^(2^l) (A, C, J as full N x N matrices; l < LPOW),
// the FP64 P_T of the last step and its inverse, the FP64 e^i (i < SMALL) and
// P_{SMALL j}, the FP64 maps of the tiles before kc, then per step k < KT: the row in the solve's
// precision S (E, o, mb, P b, P packed), E in FP64 and, for elements whose
// offset b depends on the held sample (b_k = Bb y_k + b0), -E_k^T P_k Bb
// (N x M in an N x N slot); and for the thread starts k = g K_t < KT the
// K_t-step maps Phi_g in S and in FP64.
template <int N, typename S>
struct StepTab {
    static constexpr int NN = N * N, NS = Sym<N>::SZ;
    static constexpr int oE = 0, oO = NN, oMB = NN + N, oPB = NN + 2 * N, oP = NN + 3 * N;
    static constexpr int RS = ((NN + 3 * N + NS) * (int)sizeof(S) + 15) / 16 * 16 / (int)sizeof(S);
    static constexpr int BMAX = 128, LPOW = 48;
    // steps per thread before kc: 16 bytes of a step's scalar per thread row
    // for N <= 6; for larger N the tiles before kc read their rows from
    // global memory and keep to 8 bytes
    static constexpr int KT_STEPS = (N <= 6 ? 16 : 8) / (int)sizeof(S);
    __host__ __device__ static constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
    __host__ __device__ static constexpr size_t pow_off() { return 256; }
    __host__ __device__ static constexpr size_t pref_off() { return al(pow_off() + sizeof(double) * LPOW * 3 * NN); }
    // e^i (i < SMALL) as full (A, C, J), and P_{SMALL j} (j <= cap / SMALL)
    static constexpr int SMALL = 64;
    __host__ __device__ static constexpr size_t pinv_off() { return al(pref_off() + sizeof(double) * NN); }
    __host__ __device__ static constexpr size_t small_off() { return al(pinv_off() + sizeof(double) * NN); }
    __host__ __device__ static constexpr size_t base_off() { return al(small_off() + sizeof(double) * SMALL * 3 * NN); }
    __host__ __device__ static constexpr long base_count(long kt) { return kt / SMALL + 1; }
    // FP64 maps of the tiles before kc (tiles of 128 threads x K_t steps)
    static constexpr int TILE_STEPS = 128 * KT_STEPS;
    __host__ __device__ static constexpr size_t tmap_off() { return al(base_off() + sizeof(double) * base_count(cap()) * NN); }
    __host__ __device__ static constexpr long tmap_count(long kt) { return kt / TILE_STEPS + 1; }
    __host__ __device__ static constexpr size_t rows_off() { return al(tmap_off() + sizeof(double) * tmap_count(cap()) * NN); }
    __host__ __device__ static constexpr size_t e64_off(long kt) { return al(rows_off() + sizeof(S) * kt * RS); }
    __host__ __device__ static constexpr size_t mk_off(long kt) { return al(e64_off(kt) + sizeof(double) * kt * NN); }
    __host__ __device__ static constexpr long phit_count(long kt) { return kt / KT_STEPS + 1; }
    __host__ __device__ static constexpr size_t phit_off(long kt) { return al(mk_off(kt) + sizeof(S) * kt * NN); }
    __host__ __device__ static constexpr size_t phit64_off(long kt) { return al(phit_off(kt) + sizeof(S) * phit_count(kt) * NN); }
    __host__ __device__ static constexpr size_t bytes(long kt) { return phit64_off(kt) + sizeof(double) * phit_count(kt) * NN; }
    // table length cap: the FP32 table converges within 2^-25 earlier
    __host__ __device__ static constexpr long cap() { return sizeof(S) == 4 ? 16384 : 32768; }
    __host__ __device__ static constexpr int log2_kt() { return KT_STEPS >= 4 ? 2 : KT_STEPS == 2 ? 1 : 0; }
    __host__ __device__ static constexpr int log2_tile() { return 7 + log2_kt(); }
};

namespace steptab_detail {

// lower Cholesky factor L of the symmetric positive definite M (full,
// row-major); false when a pivot is not positive
template <int N>
__device__ __forceinline__ bool chol(const double (&M)[N * N], double (&L)[N * N])
{
    bool ok = true;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        double d = M[j * N + j];
#pragma unroll
        for (int k = 0; k < j; ++k) d = fma(-L[j * N + k], L[j * N + k], d);
        ok = ok && d > 0.0;
        const double ljj = sqrt(d > 0.0 ? d : 1.0), il = 1.0 / ljj;
        L[j * N + j] = ljj;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (i < j) {
                L[i * N + j] = 0.0;
            } else if (i > j) {
                double s = M[i * N + j];
#pragma unroll
                for (int k = 0; k < j; ++k) s = fma(-L[i * N + k], L[j * N + k], s);
                L[i * N + j] = s * il;
            }
        }
    }
    return ok;
}

// Z = R^-1 L^T with P = L L^T and R R^T = I + L^T C L (P, C full symmetric)
template <int N>
__device__ __forceinline__ bool zfactor(const double (&P)[N * N], const double (&C)[N * N], double (&Z)[N * N])
{
    double L[N * N], CL[N * N], G[N * N], R[N * N];
    bool ok = chol<N>(P, L);
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = j; k < N; ++k) s = fma(C[i * N + k], L[k * N + j], s);
            CL[i * N + j] = s;
        }
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i; j < N; ++j) {
            double s = i == j ? 1.0 : 0.0;
#pragma unroll
            for (int k = i; k < N; ++k) s = fma(L[k * N + i], CL[k * N + j], s);
            G[i * N + j] = s;
            G[j * N + i] = s;
        }
    ok = chol<N>(G, R) && ok;
    // forward substitution R Z = L^T, column by column
    double ir[N];
#pragma unroll
    for (int i = 0; i < N; ++i) ir[i] = 1.0 / R[i * N + i];
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = L[c * N + i];              // (L^T)[i][c]
#pragma unroll
            for (int k = 0; k < i; ++k) s = fma(-R[i * N + k], Z[k * N + c], s);
            Z[i * N + c] = s * ir[i];
        }
    return ok;
}

template <int N>
__device__ __forceinline__ void load_full(const double* __restrict__ src, double (&dst)[N * N])
{
#pragma unroll
    for (int q = 0; q < N * N; ++q) dst[q] = __ldg(src + q);
}

// P <- A^T P (I + C P)^-1 A + J = (Z A)^T (Z A) + J for the element (A, C, J)
// stored at e (three full matrices)
template <int N>
__device__ __forceinline__ bool apply_p(const double* __restrict__ e, double (&P)[N * N])
{
    constexpr int NN = N * N;
    double A[NN], C[NN], Z[NN], ZA[NN];
    load_full<N>(e, A);
    load_full<N>(e + NN, C);
#pragma unroll
    for (int q = 0; q < NN; ++q) C[q] = 0.5 * (C[q] + C[(q % N) * N + q / N]);
    const bool ok = zfactor<N>(P, C, Z);
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < N; ++k) s = fma(Z[i * N + k], A[k * N + j], s);
            ZA[i * N + j] = s;
        }
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i; j < N; ++j) {
            double s = 0.5 * (__ldg(e + 2 * NN + i * N + j) + __ldg(e + 2 * NN + j * N + i));
#pragma unroll
            for (int k = 0; k < N; ++k) s = fma(ZA[k * N + i], ZA[k * N + j], s);
            P[i * N + j] = s;
            P[j * N + i] = s;
        }
    return ok;
}

// closed-loop map (I + Cf P)^-1 Af = Af - Cf Z^T (Z Af) of the fold (Af, Cf)
// stored at f (full matrices) for the value function P
template <int N>
__device__ __forceinline__ bool fold_map(const double* __restrict__ f, const double (&P)[N * N], double (&Phi)[N * N])
{
    constexpr int NN = N * N;
    double Af[NN], Cf[NN], Z[NN], ZA[NN], CZt[NN];
    load_full<N>(f, Af);
    load_full<N>(f + NN, Cf);
#pragma unroll
    for (int q = 0; q < NN; ++q) Cf[q] = 0.5 * (Cf[q] + Cf[(q % N) * N + q / N]);
    const bool ok = zfactor<N>(P, Cf, Z);
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double za = 0.0, cz = 0.0;
#pragma unroll
            for (int q = 0; q < N; ++q) {
                za = fma(Z[a * N + q], Af[q * N + c], za);
                cz = fma(Cf[a * N + q], Z[c * N + q], cz);
            }
            ZA[a * N + c] = za;
            CZt[a * N + c] = cz;
        }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double e = Af[a * N + c];
#pragma unroll
            for (int q = 0; q < N; ++q) e = fma(-CZt[a * N + q], ZA[q * N + c], e);
            Phi[a * N + c] = e;
        }
    return ok;
}

}  // namespace steptab_detail

// Per-warp shared scratch of the plan-time element kernels (fold_warp helpers:
// lane l holds entries l, l + 32, ... of each small FP64 matrix)
template <int N>
struct PowWk {
    double A[N * N], C[N * N], J[N * N], X[N * N], Y[N * N], Z[N * N], W[N * N], T1[N * N], T2[N * N],
        T3[N * N], P[N * N], wk[4 * N * N];
};

// e (x) e of a data-free element (A, C, J), in place (one warp)
template <int N>
__device__ inline void warp_double(PowWk<N>& w)
{
    namespace fw = fold_warp;
    constexpr int NN = N * N;
    fw::pair_coeffs<N>(w.A, w.C, w.A, w.J, w.X, w.Y, w.Z, w.W, w.wk);
    fw::pair_acj<N>(w.A, w.J, w.A, w.C, w.X, w.Y, w.W, w.T1, w.T2, w.T3);
    for (int q = fw::lane(); q < NN; q += 32) { w.A[q] = w.T1[q]; w.C[q] = w.T2[q]; w.J[q] = w.T3[q]; }
    __syncwarp();
}

// Element powers e^(2^l) of the data-free interval element e = (A, C, J)
// (Eq. 36 combine of an element with itself), for every l with
// 2^l <= max(T, KT), and P_T, the value function after all T steps (the
// powers of the set bits of T applied to P_0; powers of one element commute),
// and P_T^-1, with which the solve forms x_T = P_T^-1 v_T (Eq. 18).
// One warp, lane-parallel FP64 (the doublings are a chain in series).
template <int N, int M, typename S>
__global__ void __launch_bounds__(32)
k_step_powers(const LtiParams<N, M, double> p, const Red<N, double> prior, long T, long KT, char* __restrict__ tab)
{
    namespace fw = fold_warp;
    using ST = StepTab<N, S>;
    constexpr int NN = N * N;
    __shared__ PowWk<N> w;
    const int l0 = threadIdx.x;
    double* pw = reinterpret_cast<double*>(tab + ST::pow_off());
    for (int q = l0; q < NN; q += 32) {
        const int a = q / N, c = q % N;
        w.A[q] = p.A[q];
        w.C[q] = p.C[Sym<N>::at(a, c)];
        w.J[q] = p.J[Sym<N>::at(a, c)];
        w.P[q] = prior.P[Sym<N>::at(a, c)];
    }
    __syncwarp();
    const long top = T > KT ? T : KT;
#pragma unroll 1
    for (int l = 0; l < ST::LPOW && (1L << l) <= top; ++l) {
        double* o = pw + (long)l * 3 * NN;
        for (int q = l0; q < NN; q += 32) { o[q] = w.A[q]; o[NN + q] = w.C[q]; o[2 * NN + q] = w.J[q]; }
        if ((T >> l) & 1) fw::riccati<N>(w.A, w.C, w.J, w.P, w.wk);
        warp_double<N>(w);
    }
    double* pr = reinterpret_cast<double*>(tab + ST::pref_off());
    for (int q = l0; q < NN; q += 32) {
        pr[q] = w.P[q];
        w.T1[q] = w.P[q] - (q % (N + 1) == 0 ? 1.0 : 0.0);      // P_T - I
        w.T2[q] = q % (N + 1) == 0 ? 1.0 : 0.0;
    }
    __syncwarp();
    fw::inv_I_plus<N>(w.T1, w.T2, w.T3, w.wk);                  // (I + (P_T - I))^-1 = P_T^-1
    double* pi = reinterpret_cast<double*>(tab + ST::pinv_off());
    for (int q = l0; q < NN; q += 32) pi[q] = w.T3[q];
}

// e^i for i < SMALL (the combination of the powers of the set bits of i;
// e^0 is the neutral element A = I, C = J = 0), one warp each
template <int N, typename S>
__global__ void __launch_bounds__(128) k_step_small(char* __restrict__ tab)
{
    namespace fw = fold_warp;
    using ST = StepTab<N, S>;
    constexpr int NN = N * N;
    __shared__ PowWk<N> wks[4];
    PowWk<N>& w = wks[threadIdx.x >> 5];
    const int i = blockIdx.x * 4 + (threadIdx.x >> 5), l0 = fw::lane();
    if (i >= ST::SMALL) return;
    const double* pw = reinterpret_cast<const double*>(tab + ST::pow_off());
    for (int q = l0; q < NN; q += 32) {
        w.A[q] = q % (N + 1) == 0 ? 1.0 : 0.0;
        w.C[q] = 0.0;
        w.J[q] = 0.0;
    }
    __syncwarp();
#pragma unroll 1
    for (int l = 0; (i >> l) != 0; ++l) {
        if (!((i >> l) & 1)) continue;
        const double* u = pw + (long)l * 3 * NN;           // e^(2^l), the later operand
        for (int q = l0; q < NN; q += 32) { w.T1[q] = u[q]; w.T2[q] = u[NN + q]; w.T3[q] = u[2 * NN + q]; }
        __syncwarp();
        fw::pair_coeffs<N>(w.T1, w.T2, w.A, w.J, w.X, w.Y, w.Z, w.W, w.wk);
        fw::pair_acj<N>(w.T1, w.T3, w.A, w.C, w.X, w.Y, w.W, w.P, w.Z, w.wk);
        for (int q = l0; q < NN; q += 32) { w.A[q] = w.P[q]; w.C[q] = w.Z[q]; w.J[q] = w.wk[q]; }
        __syncwarp();
    }
    double* o = reinterpret_cast<double*>(tab + ST::small_off()) + (long)i * 3 * NN;
    for (int q = l0; q < NN; q += 32) { o[q] = w.A[q]; o[NN + q] = w.C[q]; o[2 * NN + q] = w.J[q]; }
}

// P_{SMALL j} for j <= (KT - 1) / SMALL: the powers of the set bits of SMALL j
// applied to P_0, one warp each
template <int N, typename S>
__global__ void __launch_bounds__(128) k_step_base(const Red<N, double> prior, long KT, char* __restrict__ tab)
{
    namespace fw = fold_warp;
    using ST = StepTab<N, S>;
    constexpr int NN = N * N;
    __shared__ PowWk<N> wks[4];
    PowWk<N>& w = wks[threadIdx.x >> 5];
    const long j = (long)blockIdx.x * 4 + (threadIdx.x >> 5);
    const int l0 = fw::lane();
    if (j * ST::SMALL >= KT) return;
    const double* pw = reinterpret_cast<const double*>(tab + ST::pow_off());
    for (int q = l0; q < NN; q += 32) w.P[q] = prior.P[Sym<N>::at(q / N, q % N)];
    __syncwarp();
    const long k = j * ST::SMALL;
#pragma unroll 1
    for (int l = 0; (k >> l) != 0; ++l)
        if ((k >> l) & 1) {
            const double* u = pw + (long)l * 3 * NN;
            for (int q = l0; q < NN; q += 32) { w.A[q] = u[q]; w.C[q] = u[NN + q]; w.J[q] = u[2 * NN + q]; }
            __syncwarp();
            fw::riccati<N>(w.A, w.C, w.J, w.P, w.wk);
        }
    double* o = reinterpret_cast<double*>(tab + ST::base_off()) + j * NN;
    for (int q = l0; q < NN; q += 32) o[q] = w.P[q];
}

// Optional held-sample dependence of the element offset: b_k = Bb y_k + b0
// (block and exact elements); Bb is N x M row-major.
template <int N, int M>
struct SampleOffset {
    int on;
    double Bb[N * M];
};

// One thread per tabulated step k < KT (FP64): P_k = e^(k mod SMALL) applied
// to P_{SMALL floor(k / SMALL)}, then the row of constants, -E_k^T P_k Bb
// when the offset depends on the sample, and for the first step of a thread of
// K_t steps (k = g K_t) the thread's composite closed-loop map
// Phi_g = (I + C_Kt P_k)^-1 A_Kt of the K_t-step element e^(K_t) (the
// composition of its K_t per-step maps: the closed-loop map of the combined
// element), and likewise for the first step of a tile of 128 x K_t steps the
// tile's map.  With check, every step whose P_k differs from P_T beyond tol
// raises meta[0] to k + 1; meta[1] counts non-positive Cholesky pivots.
template <int N, int M, typename S>
__global__ void __launch_bounds__(128)
k_lti_steptab(const LtiParams<N, M, double> p, long KT, int check, double tol,
              const SampleOffset<N, M> so, char* __restrict__ tab)
{
    namespace sd = steptab_detail;
    using ST = StepTab<N, S>;
    constexpr int NN = N * N, Kt = ST::KT_STEPS;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= KT) return;
    const double* pw = reinterpret_cast<const double*>(tab + ST::pow_off());
    unsigned long long* meta = reinterpret_cast<unsigned long long*>(tab);
    S* row = reinterpret_cast<S*>(tab + ST::rows_off()) + k * ST::RS;
    double* e64 = reinterpret_cast<double*>(tab + ST::e64_off(KT)) + k * NN;
    double P[NN];
    sd::load_full<N>(reinterpret_cast<const double*>(tab + ST::base_off()) + (k / ST::SMALL) * NN, P);
    bool ok = true;
    if (k % ST::SMALL)
        ok = sd::apply_p<N>(reinterpret_cast<const double*>(tab + ST::small_off()) + (k % ST::SMALL) * 3 * NN, P);
    // per-step constants from Z of (P, C): E = A - C Z^T (Z A), mb = b - C Z^T (Z b)
    double A[NN], C[NN], b[N], Z[NN], ZA[NN], CZt[NN];
#pragma unroll
    for (int q = 0; q < NN; ++q) {
        A[q] = p.A[q];
        C[q] = p.C[Sym<N>::at(q / N, q % N)];
    }
#pragma unroll
    for (int q = 0; q < N; ++q) b[q] = p.b[q];
    ok = sd::zfactor<N>(P, C, Z) && ok;
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double za = 0.0, cz = 0.0;
#pragma unroll
            for (int q = 0; q < N; ++q) {
                za = fma(Z[a * N + q], A[q * N + c], za);
                cz = fma(C[a * N + q], Z[c * N + q], cz);
            }
            ZA[a * N + c] = za;
            CZt[a * N + c] = cz;
        }
    double E[NN], Zb[N], Pb[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        double zb = 0.0, pb = 0.0;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            zb = fma(Z[a * N + q], b[q], zb);
            pb = fma(P[a * N + q], b[q], pb);
        }
        Zb[a] = zb;
        Pb[a] = pb;
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double e = A[a * N + c];
#pragma unroll
            for (int q = 0; q < N; ++q) e = fma(-CZt[a * N + q], ZA[q * N + c], e);
            E[a * N + c] = e;
            row[ST::oE + a * N + c] = S(e);
            e64[a * N + c] = e;
        }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        double mb = b[a], o = 0.0;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            mb = fma(-CZt[a * N + q], Zb[q], mb);
            o = fma(-E[q * N + a], Pb[q], o);
        }
        row[ST::oMB + a] = S(mb);
        row[ST::oO + a] = S(o);
        row[ST::oPB + a] = S(Pb[a]);
#pragma unroll
        for (int c = a; c < N; ++c) row[ST::oP + Sym<N>::at(a, c)] = S(P[a * N + c]);
    }
    if (so.on) {
        // -E^T P Bb: the sample's share of o_k
        S* mk = reinterpret_cast<S*>(tab + ST::mk_off(KT)) + k * NN;
        double PB[N * M];
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int c = 0; c < M; ++c) {
                double acc = 0.0;
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(P[a * N + q], so.Bb[q * M + c], acc);
                PB[a * M + c] = acc;
            }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int c = 0; c < M; ++c) {
                double acc = 0.0;
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(-E[q * N + a], PB[q * M + c], acc);
                mk[a * M + c] = S(acc);
            }
    }
    if (k % ST::TILE_STEPS == 0) {
        double Tm[NN];
        ok = sd::fold_map<N>(pw + (long)ST::log2_tile() * 3 * NN, P, Tm) && ok;
        double* tm = reinterpret_cast<double*>(tab + ST::tmap_off()) + (k / ST::TILE_STEPS) * NN;
#pragma unroll
        for (int q = 0; q < NN; ++q) tm[q] = Tm[q];
    }
    if (k % Kt == 0) {
        double Ph[NN];
        ok = sd::fold_map<N>(pw + (long)ST::log2_kt() * 3 * NN, P, Ph) && ok;
        S* ph = reinterpret_cast<S*>(tab + ST::phit_off(KT)) + (k / Kt) * NN;
        double* ph64 = reinterpret_cast<double*>(tab + ST::phit64_off(KT)) + (k / Kt) * NN;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            ph[q] = S(Ph[q]);
            ph64[q] = Ph[q];
        }
    }
    if (check) {
        double Pr[NN];
        sd::load_full<N>(reinterpret_cast<const double*>(tab + ST::pref_off()), Pr);
        bool conv = true;
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int c = 0; c < N; ++c)
                conv = conv && fabs(P[a * N + c] - Pr[a * N + c]) <= tol * sqrt(fabs(Pr[a * N + a] * Pr[c * N + c]));
        if (!conv) atomicMax(meta, (unsigned long long)(k + 1));
    }
    if (!ok) atomicAdd(meta + 1, 1ull);
}

// ---------------------------------------------------------------------------
// tables of the tiled scan (k_lti_scan), computed once kc is known
// ---------------------------------------------------------------------------
// Tiling: J_t tiles of B threads x K_t steps cover [0, J_t B K_t) (J_t B K_t
// >= kc), then tiles of B threads x K steps; tile j starts at
// s_j = j B K_t (j < J_t) or J_t B K_t + (j - J_t) B K.
struct ScanGeom {
    int B, K, Kt, Jt, nt;
    __host__ __device__ long start(int j) const
    {
        return j < Jt ? (long)j * B * Kt : (long)Jt * B * Kt + (long)(j - Jt) * B * K;
    }
    __host__ __device__ int steps(int j) const { return j < Jt ? Kt : K; }
};

// Layout of the scan buffer (offsets in bytes): the powers Phi_inf^d
// (d = 0..BMAX), the per-step E_k and o_k of the tiles before kc in the order
// of their shared-memory copy (component c of step i of thread t at
// (i CT + c) B + t), the tiles' offsets w_j and RTS maps, the measurement
// gain of the steps after kc (G, plus -E^T P Bb when the offset depends on the
// sample), the partial thread's map E_inf^nv of the last tile, the suffix
// products Q_t of the thread maps of the tiles before kc, then the tile
// tables of lti_fold.cuh (TileTables: F_j = E_j^T and the products Pi).
template <int N, int M, typename S>
struct ScanBuf {
    static constexpr int NN = N * N, BMAX = 128, NTMAX = 5 * BMAX;
    static constexpr int CT = NN + N;                         // E, o
    using ST = StepTab<N, S>;
    __host__ __device__ static constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
    __host__ __device__ static constexpr long jt_max() { return ST::cap() / (BMAX * ST::KT_STEPS) + 2; }
    __host__ __device__ static constexpr size_t pw_off() { return 0; }
    __host__ __device__ static constexpr size_t ttab_off() { return al(sizeof(S) * (BMAX + 1) * NN); }
    // record of a tile before kc: its per-step (E_k, o_k), then its threads'
    // maps Phi_t and suffix products Q_t (component q of thread t at q B + t)
    __host__ __device__ static constexpr size_t ttab_rec(int B, int Kt) { return (size_t)B * (Kt * CT + 2 * NN); }
    __host__ __device__ static constexpr size_t ttab_tile() { return ttab_rec(BMAX, ST::KT_STEPS); }
    __host__ __device__ static constexpr size_t w_off() { return al(ttab_off() + sizeof(S) * jt_max() * ttab_tile()); }
    __host__ __device__ static constexpr size_t taff_off() { return al(w_off() + sizeof(S) * NTMAX * N); }
    __host__ __device__ static constexpr size_t gs_off() { return al(taff_off() + sizeof(S) * NTMAX * (NN + N)); }
    __host__ __device__ static constexpr size_t ep_off() { return al(gs_off() + sizeof(S) * N * M); }
    // per thread of a tile before kc: Q_t = (Phi_{t+1} ... Phi_{B-1})^T
    __host__ __device__ static constexpr size_t qsuf_off() { return al(ep_off() + sizeof(S) * NN); }
    // powers M^d (d < NTMAX) of the map M = Phi_inf^B of a full tile after kc,
    // and its FP64 squares M^(2^l) (l < MSQ) they are formed from
    static constexpr int MSQ = 10;
    __host__ __device__ static constexpr size_t mp_off() { return al(qsuf_off() + sizeof(S) * jt_max() * BMAX * NN); }
    __host__ __device__ static constexpr size_t msq_off() { return al(mp_off() + sizeof(S) * NTMAX * NN); }
    // products Pi(a, b) of the tile maps among the tiles up to jt_max(), and
    // their transposes, entry (a, b) at a (jt_max() + 1) + b
    __host__ __device__ static constexpr long tp_count() { return (jt_max() + 1) * (jt_max() + 1); }
    __host__ __device__ static constexpr size_t tpi_off() { return al(msq_off() + sizeof(double) * MSQ * NN); }
    __host__ __device__ static constexpr size_t tqt_off() { return al(tpi_off() + sizeof(S) * tp_count() * NN); }
    __host__ __device__ static constexpr size_t tiles_off() { return al(tqt_off() + sizeof(S) * tp_count() * NN); }
    // the tile tables (TileTables: the tile maps F_j), without the products
    __host__ __device__ static constexpr size_t bytes() { return tiles_off() + TileTables<N, M, S>::pi_off(NTMAX); }
};

namespace scan_plan_detail {
// c = a b (FP64 N x N in shared memory), lanes of one warp: entry q by lane q % 32
template <int N>
__device__ inline void wmul(const double* a, const double* b, double* c)
{
    for (int q = threadIdx.x & 31; q < N * N; q += 32) {
        const int i = q / N, j = q - i * N;
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < N; ++k) s = fma(a[i * N + k], b[k * N + j], s);
        c[q] = s;
    }
    __syncwarp();
}
}  // namespace scan_plan_detail

// Phi_inf = E_kc^K (FP64, warp 0, binary powers), then Phi_inf^d for
// d = 0..B by doubling levels (Phi^d = Phi^(d - 2^l) Phi^(2^l), all d of a
// level at once), written in S.  Then the last tile's maps when it lies after
// kc: its thread tp holds the last nvp < K steps (threads after it none), so
// the state at thread tp's start is Ep x_T + beta_tp with Ep = E_kc^nvp, and
// the tile's RTS map matrix is Phi_inf^tp Ep (the matrix part of its entry in
// the tile RTS maps; the kernel adds the offset).  One CTA of 256 threads.
template <int N, typename S>
__global__ void __launch_bounds__(256) k_scan_powers(const double* __restrict__ e_kc, int K, int B, S* __restrict__ pw,
                                                     int tp, int nvp, S* __restrict__ ep, S* __restrict__ taff_last)
{
    namespace pd = scan_plan_detail;
    constexpr int NN = N * N;
    __shared__ double W[StepTab<N, S>::BMAX + 1][NN];
    __shared__ double X[NN], Y[NN], Z[NN];
    const int t = threadIdx.x;
    if (t < 32) {
        for (int q = t; q < NN; q += 32) {
            X[q] = __ldg(e_kc + q);                       // E^(2^bit)
            Y[q] = q % (N + 1) == 0 ? 1.0 : 0.0;          // accumulated power
        }
        __syncwarp();
        for (int e = K; e > 0; e >>= 1) {
            if (e & 1) {
                pd::wmul<N>(Y, X, Z);
                for (int q = t; q < NN; q += 32) Y[q] = Z[q];
                __syncwarp();
            }
            if (e > 1) {
                pd::wmul<N>(X, X, Z);
                for (int q = t; q < NN; q += 32) X[q] = Z[q];
                __syncwarp();
            }
        }
        for (int q = t; q < NN; q += 32) {
            W[0][q] = q % (N + 1) == 0 ? 1.0 : 0.0;
            W[1][q] = Y[q];
        }
    }
    __syncthreads();
    for (int l = 1; l < B; l <<= 1) {
        // d in (l, min(2l, B)] from W[d - l] W[l] (both known after the level before)
        const int cnt = (min(2 * l, B) - l) * NN;
        for (int e = t; e < cnt; e += blockDim.x) {
            const int d = l + 1 + e / NN, q = e % NN, i = q / N, jj = q - i * N;
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < N; ++k) s = fma(W[d - l][i * N + k], W[l][k * N + jj], s);
            W[d][q] = s;
        }
        __syncthreads();
    }
    for (int e = t; e < (B + 1) * NN; e += blockDim.x) pw[e] = S(W[e / NN][e % NN]);
    if (t < 32 && taff_last) {
        for (int q = t; q < NN; q += 32) {
            X[q] = __ldg(e_kc + q);
            Y[q] = q % (N + 1) == 0 ? 1.0 : 0.0;
        }
        __syncwarp();
        for (int e = nvp; e > 0; e >>= 1) {
            if (e & 1) {
                pd::wmul<N>(Y, X, Z);
                for (int q = t; q < NN; q += 32) Y[q] = Z[q];
                __syncwarp();
            }
            if (e > 1) {
                pd::wmul<N>(X, X, Z);
                for (int q = t; q < NN; q += 32) X[q] = Z[q];
                __syncwarp();
            }
        }
        pd::wmul<N>(W[tp], Y, Z);
        for (int q = t; q < NN; q += 32) {
            ep[q] = S(Y[q]);
            taff_last[q] = S(Z[q]);
        }
    }
}

// The squares M^(2^l), l < MSQ, of the map M = E_kc^(K B) of a full tile after
// kc (FP64, one warp, lane-parallel products)
template <int N>
__global__ void __launch_bounds__(32) k_scan_msq(const double* __restrict__ e_kc, int K, int B, int nsq,
                                                 double* __restrict__ sq)
{
    namespace pd = scan_plan_detail;
    constexpr int NN = N * N;
    __shared__ double X[NN], Y[NN], Z[NN];
    const int l = threadIdx.x;
    for (int q = l; q < NN; q += 32) {
        X[q] = __ldg(e_kc + q);
        Y[q] = q % (N + 1) == 0 ? 1.0 : 0.0;
    }
    __syncwarp();
    for (long e = (long)K * B; e; e >>= 1) {        // Y = E^(K B) by binary powering
        if (e & 1) {
            pd::wmul<N>(Y, X, Z);
            for (int q = l; q < NN; q += 32) Y[q] = Z[q];
            __syncwarp();
        }
        if (e > 1) {
            pd::wmul<N>(X, X, Z);
            for (int q = l; q < NN; q += 32) X[q] = Z[q];
            __syncwarp();
        }
    }
    for (int q = l; q < NN; q += 32) sq[q] = Y[q];
    __syncwarp();
    for (int i = 1; i < nsq; ++i) {
        pd::wmul<N>(sq + (i - 1) * NN, sq + (i - 1) * NN, Z);
        for (int q = l; q < NN; q += 32) sq[i * NN + q] = Z[q];
        __syncwarp();
    }
}

// Products Pi(a, b) = E_a ... E_{b-1} of the tile maps among the tiles up to
// J1 = min(Jt, nt - 1) (0 <= a <= b <= J1), the only ones the tile sums of the
// tiled scan read (the later tiles share one map and take its powers), with
// their transposes (entry (a, b) at a ld + b): one thread per pair, from the
// tile table F_j = E_j^T.
template <int N, int M, typename S>
__global__ void __launch_bounds__(128) k_scan_tprod(int nt, int J1, const char* __restrict__ tiles, int ld,
                                                   S* __restrict__ tpi, S* __restrict__ tqt)
{
    using TT = TileTables<N, M, S>;
    namespace pd = products_detail;
    constexpr int NN = N * N;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    // pair p -> (a, b) with b = a .. J1, rows a = 0 .. J1
    int a = 0, q = p;
    while (a <= J1 && q > J1 - a) {
        q -= J1 - a + 1;
        ++a;
    }
    if (a > J1) return;
    const int b = a + q;
    const S* F = reinterpret_cast<const S*>(tiles + TT::f_off(nt));
    S P[NN];
#pragma unroll
    for (int r = 0; r < NN; ++r) P[r] = r % (N + 1) == 0 ? S(1) : S(0);
#pragma unroll 1
    for (int j = a; j < b; ++j) {
        S E[NN];
        pd::load_E<N>(F, j, E);
        pd::mul<N>(P, E);
    }
    S* pi = tpi + ((long)a * ld + b) * NN;
    S* qt = tqt + ((long)a * ld + b) * NN;
#pragma unroll
    for (int r = 0; r < NN; ++r) {
        pi[r] = P[r];
        qt[r] = P[(r % N) * N + r / N];
    }
}

// M^d for d < nt from the squares, one warp per d (FP64, lane-parallel), in S
template <int N, typename S>
__global__ void __launch_bounds__(128) k_scan_mpow(const double* __restrict__ sq, int nsq, int nt, S* __restrict__ mp)
{
    namespace pd = scan_plan_detail;
    constexpr int NN = N * N;
    __shared__ double P[4][NN], Z[4][NN];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int d = blockIdx.x * 4 + w;
    if (d >= nt) return;                                    // warp-uniform
    for (int q = l; q < NN; q += 32) P[w][q] = q % (N + 1) == 0 ? 1.0 : 0.0;
    __syncwarp();
    for (int i = 0; i < nsq; ++i)
        if ((d >> i) & 1) {
            pd::wmul<N>(P[w], sq + i * NN, Z[w]);
            for (int q = l; q < NN; q += 32) P[w][q] = Z[w][q];
            __syncwarp();
        }
    for (int q = l; q < NN; q += 32) mp[(long)d * NN + q] = S(P[w][q]);
}

// Tile maps E_j (the composition of a tile's per-step closed-loop maps) as
// F_j = E_j^T in the tile tables: a tile before kc takes the closed-loop map
// of the element of its 128 K_t steps at its first step (the step tables'
// tile maps), a later tile Phi_inf^B.  The last tile's map is not used by the
// tile products.  One thread per entry.
template <int N, int M, typename S>
__global__ void __launch_bounds__(128)
k_scan_tilemaps(const double* __restrict__ tmap64, ScanGeom g, const S* __restrict__ pw, char* __restrict__ tiles)
{
    using TT = TileTables<N, M, S>;
    constexpr int NN = N * N;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)g.nt * NN) return;
    const int j = (int)(e / NN), q = (int)(e % NN), qt = (q % N) * N + q / N;
    S* F = reinterpret_cast<S*>(tiles + TT::f_off(g.nt)) + (long)j * NN;
    F[q] = j >= g.Jt || j == g.nt - 1 ? pw[(long)g.B * NN + qt] : S(__ldg(tmap64 + (long)j * NN + qt));
}

// Suffix products of the thread maps of each tile before kc (one CTA of B
// threads per tile, FP64): Q_t = (Phi_{t+1} ... Phi_{B-1})^T, Q_{B-1} = I.  The
// filter offset of such a tile is then w_j = sum_t Q_t W_t.  Inclusive suffix
// products S_t = Phi_t ... Phi_{B-1} by a Kogge-Stone scan in shared memory
// (S_t <- S_t S_{t+d}), then Q_t = S_{t+1}^T.
template <int N, typename S>
__global__ void __launch_bounds__(128)
k_scan_qsuf(const double* __restrict__ phit64, ScanGeom g, S* __restrict__ qsuf)
{
    constexpr int NN = N * N;
    extern __shared__ double qsm[];                      // 2 x 128 x NN
    auto buf = [&](int b2, int i) { return qsm + ((long)b2 * 128 + i) * NN; };
    const int j = blockIdx.x, t = threadIdx.x, B = g.B;
    if (j >= g.Jt || j == g.nt - 1 || B > 128) return;   // the last tile has no w_j (its maps may pass KT)
    int cur = 0;
    if (t < B)
        for (int q = 0; q < NN; ++q) buf(0, t)[q] = __ldg(phit64 + ((long)j * B + t) * NN + q);
    __syncthreads();
    for (int d = 1; d < B; d <<= 1) {
        if (t < B) {
            if (t + d < B) {
                for (int q = 0; q < NN; ++q) {
                    const int r = q / N, c = q % N;
                    double acc = 0.0;
                    for (int k = 0; k < N; ++k) acc = fma(buf(cur, t)[r * N + k], buf(cur, t + d)[k * N + c], acc);
                    buf(cur ^ 1, t)[q] = acc;
                }
            } else {
                for (int q = 0; q < NN; ++q) buf(cur ^ 1, t)[q] = buf(cur, t)[q];
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    if (t < B) {
        S* o = qsuf + ((long)j * B + t) * NN;
        for (int q = 0; q < NN; ++q) {
            const int r = q / N, c = q % N;
            o[q] = t + 1 < B ? S(buf(cur, t + 1)[c * N + r]) : (r == c ? S(1) : S(0));
        }
    }
}

// Records of the tiles before kc in the order of their shared-memory copy
// (ScanBuf::ttab_rec): per-step E_k and o_k, the thread maps Phi_t and the
// suffix products Q_t; zeros past the tables
template <int N, typename S>
__global__ void k_scan_ttab(const S* __restrict__ rows, const S* __restrict__ phit, const S* __restrict__ qsuf, long KT,
                            ScanGeom g, S* __restrict__ ttab)
{
    using ST = StepTab<N, S>;
    constexpr int NN = N * N, CT = NN + N;
    const long steps = (long)g.B * g.Kt * CT, per = steps + 2L * g.B * NN;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= per * g.Jt) return;
    const int j = (int)(e / per);
    const long r = e % per;
    S v = S(0);
    if (r < steps) {
        const int t = (int)(r % g.B), ic = (int)(r / g.B), i = ic / CT, c = ic % CT;
        const long k = (long)j * g.B * g.Kt + (long)t * g.Kt + i;
        if (k < KT) v = c < NN ? rows[k * ST::RS + ST::oE + c] : rows[k * ST::RS + ST::oO + (c - NN)];
    } else {
        const long r2 = r - steps;
        const int which = (int)(r2 / ((long)g.B * NN)), q = (int)((r2 % ((long)g.B * NN)) / g.B), t = (int)(r2 % g.B);
        const long th = (long)j * g.B + t;
        if (which == 0) {
            if (th * g.Kt < KT) v = phit[th * NN + q];
        } else {
            v = qsuf[th * NN + q];
        }
    }
    ttab[e] = v;
}

// measurement gain of the steps after kc: G + (-E^T P Bb of row kc)
template <int N, int M, typename S>
__global__ void k_scan_gs(const LtiParams<N, M, S> p, const S* __restrict__ mk_kc, int on, S* __restrict__ gs)
{
    for (int q = threadIdx.x; q < N * M; q += blockDim.x) gs[q] = p.G[q] + (on ? mk_kc[q] : S(0));
}

// ---------------------------------------------------------------------------
// the tiled-scan solve
// ---------------------------------------------------------------------------
template <int N, int M, typename S>
struct ScanArgs {
    const S* rows;          // step rows (StepTab)
    long kc;                // steps k >= kc read row kc
    const S* pw;            // Phi_inf^d, d = 0..B
    const S* ttab;          // per-step E_k, o_k of the tiles before kc
    const S* phit;          // K_t-step thread maps before kc
    S* w;                   // tile offsets of the filter maps
    S* taff;                // tile RTS maps
    const S* pi;            // tile-map products Pi(a, b) among the tiles up to Jt, entry a tld + b
    const S* qt;            // their transposes, entry a tld + b holding Pi(a, b)^T
    int tld;
    const S* gs;            // measurement gain of the steps after kc (with the sample's share of o)
    const S* mk;            // per-step -E_k^T P_k Bb (steps before kc; offsets depending on the sample)
    const S* ep;            // E_inf^nv of the last tile's partial thread
    const S* qsuf;          // suffix products of the thread maps of the tiles before kc
    const S* mp;            // M^d, M = Phi_inf^B the map of a full tile after kc
    const double* pinv;     // P_T^-1 (FP64)
    ScanGeom g;
    int has_b;              // b != 0: the A^-1 b term of g_k
    S AiC[N * N];           // A^-1 C
    S Aib[N];               // A^-1 b (b0 when the offset depends on the sample)
    S AiBb[N * M];          // A^-1 Bb
    S EAiC[N * N];          // E_inf A^-1 C, E_inf A^-1 b, E_inf A^-1 Bb (the steps after kc)
    S EAib[N];
    S EAiBb[N * M];
};

// shared memory of k_lti_scan (offsets in scalars): the composition area, the
// warp totals, the tile's observations, the per-step offsets g_k (staged
// states in the RTS phase; exchange area of the full-map compositions before
// that), then the powers Phi_inf^d (tiles after kc) or the per-step E_k, o_k
// (tiles before kc), then the mbarrier.  With STAGE false (FP64, and FP32
// state dimensions above 6, whose per-step data would not fit for a grid of
// co-resident tiles)
// the observations are read from global memory, the g_k and states go
// through x_out, and the tiles before kc read their rows from global memory:
// only the composition areas and the powers stay.
template <int N, int M, typename S>
struct ScanSmem {
    static constexpr int NN = N * N, NA = NN + N, CT = NN + N;
    static constexpr bool STAGE = N <= 6 && sizeof(S) == 4;
    __host__ __device__ static constexpr int al(int x) { return (x + 3) / 4 * 4; }
    __host__ __device__ static constexpr int red_size(int B) { return (B / 32) * (NA + N) + N; }
    __host__ __device__ static constexpr int wt(int B) { return al(red_size(B)); }
    __host__ __device__ static constexpr int ys(int B) { return al(wt(B) + 2 * (B / 32) * N + 2 * N); }
    __host__ __device__ static constexpr int gst(int B, int Kmax) { return al(ys(B) + (STAGE ? B * Kmax * M : 0)); }
    __host__ __device__ static constexpr int tabs(int B, int Kmax)
    {
        return al(gst(B, Kmax) + (STAGE && B * Kmax * N > B * NA ? B * Kmax * N : B * NA));
    }
    __host__ __device__ static constexpr int bar(int B, int K, int Kt)
    {
        // the tile kind with the larger footprint decides
        const int a = tabs(B, K) + (B + 1) * NN, c = tabs(B, Kt) + (STAGE ? B * (Kt * CT + 2 * NN) : 0);
        return al(a > c ? a : c);
    }
    __host__ __device__ static constexpr size_t bytes(int B, int K, int Kt) { return sizeof(S) * (size_t)bar(B, K, Kt) + 16; }
};

template <int N, typename S>
__device__ __forceinline__ void mat_vec(const S* __restrict__ Mx, const S* x, S* y)     // y = M x
{
#pragma unroll
    for (int a = 0; a < N; ++a) {
        S acc = S(0);
#pragma unroll
        for (int q = 0; q < N; ++q) acc = fma(Mx[a * N + q], x[q], acc);
        y[a] = acc;
    }
}
template <int N, typename S>
__device__ __forceinline__ void mat_tvec(const S* __restrict__ Mx, const S* x, S* y)    // y = M^T x
{
#pragma unroll
    for (int a = 0; a < N; ++a) {
        S acc = S(0);
#pragma unroll
        for (int q = 0; q < N; ++q) acc = fma(Mx[q * N + a], x[q], acc);
        y[a] = acc;
    }
}

// The maps of the B threads exchanged so that thread t holds thread B-1-t's
// map (scratch: B Aff records); ends with a barrier.  With the order of the
// threads reversed, block_aff_reduce and block_aff_end_states compose the
// filter maps in time order (the earlier map innermost).
template <int N, typename S>
__device__ __forceinline__ void reverse_maps(Aff<N, S>& H, S* scratch)
{
    constexpr int NA = Aff<N, S>::NCOMP;
    const int B = blockDim.x, t = threadIdx.x;
#pragma unroll
    for (int c = 0; c < NA; ++c) scratch[c * B + (B - 1 - t)] = comp(H, c);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NA; ++c) comp(H, c) = scratch[c * B + t];
    __syncthreads();
}

// N scalars of thread t moved to thread B-1-t; ends with a barrier
template <int N, typename S>
__device__ __forceinline__ void reverse_vec(S (&v)[N], S* scratch)
{
    const int B = blockDim.x, t = threadIdx.x;
#pragma unroll
    for (int c = 0; c < N; ++c) scratch[c * B + (B - 1 - t)] = v[c];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = scratch[c * B + t];
    __syncthreads();
}

// Tile sums of the tiled scan (item (5) of lti_fold.cuh) with the powers of
// the full-tile map after kc: every full tile j >= Jt has the map
// M = Phi_inf^B, so Pi(a, b) = M^(b - a) for Jt <= a <= b <= nt - 1, and a
// product reaching back before Jt splits as Pi(a, b) = Pi(a, Jt) M^(b - Jt).
// Only the products among the first Jt + 1 tiles come from the product tables;
// the rest read the power table M^d (one small table shared by every tile).
//
// The value function's v before tile `tile` (in vout, thread 0):
//   v_j = Pi(0, j)^T v_0 + sum_{i<j} Pi(i+1, j)^T w_i.
// Terms i = t - 1 + u B (i = -1: v_0); at most 5 per thread (nt <= 4 B + 1),
// their operands loaded first.
template <int N, typename S>
__device__ __forceinline__ void scan_tile_prefix(const S* __restrict__ qt, int ld, const S* __restrict__ mp,
                                                 const S* __restrict__ w, int tile, int Jt, const S (&v0)[N],
                                                 S* red, S (&vout)[N])
{
    constexpr int NN = N * N, UMAX = 5;
    const int t = threadIdx.x;
    if (tile == 0) {
#pragma unroll
        for (int a = 0; a < N; ++a) vout[a] = v0[a];
        return;
    }
    S v[N];
#pragma unroll
    for (int a = 0; a < N; ++a) v[a] = S(0);
    // a term before min(tile, Jt) goes through Pi(i+1, jb)^T with jb = min(tile, Jt),
    // then (M^(tile - jb))^T; a later one through (M^(tile-1-i))^T alone
    const int jb = min(tile, Jt);
    S Pl[NN];
    if (tile > jb) load_run_aligned<NN, S>(mp + (long)(tile - jb) * NN, Pl);
#pragma unroll 1
    for (int u = 0; u < UMAX; ++u) {
        const int i = t - 1 + u * (int)blockDim.x;
        if (i >= tile) break;
        S wv[N], p[N];
#pragma unroll
        for (int c = 0; c < N; ++c) wv[c] = i < 0 ? v0[c] : w[(long)i * N + c];
        S Q[NN];
        if (i < jb) {
            load_run_aligned<NN, S>(qt + ((long)(i + 1) * ld + jb) * NN, Q);    // Pi(i+1, jb)^T
            mat_vec<N, S>(Q, wv, p);
            if (tile > jb) {
                mat_tvec<N, S>(Pl, p, wv);
#pragma unroll
                for (int c = 0; c < N; ++c) p[c] = wv[c];
            }
        } else {
            load_run_aligned<NN, S>(mp + (long)(tile - 1 - i) * NN, Q);        // M^(tile-1-i)
            mat_tvec<N, S>(Q, wv, p);
        }
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] += p[c];
    }
    block_vec_sum<N, S>(v, red);
#pragma unroll
    for (int a = 0; a < N; ++a) vout[a] = v[a];
}

// The state at the end of tile `tile` (thread 0 writes it to xe; ends with a
// barrier): x_T for the last tile, else
//   x_end(j) = Pi(j+1, nt-1) x_L + sum_{i=j+1}^{nt-2} Pi(j+1, i) beta_i,
// x_L the last tile's map applied to x_T and beta_i the offset of tile i's map.
template <int N, typename S>
__device__ __forceinline__ void scan_tile_suffix(const S* __restrict__ pi, int ld, const S* __restrict__ mp,
                                                 const S* __restrict__ tile_aff, int tile, int nt, int Jt,
                                                 const S* xT, S* red, S* xe)
{
    constexpr int NN = N * N, NA = Aff<N, S>::NCOMP, UMAX = 5;
    const int t = threadIdx.x;
    if (tile + 1 == nt) {
        if (t == 0)
#pragma unroll
            for (int i = 0; i < N; ++i) xe[i] = xT[i];
        __syncthreads();
        return;
    }
    S v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = S(0);
    // a term past ib = max(tile + 1, Jt) goes through M^(i - ib), then, when
    // tile + 1 < ib, through Pi(tile+1, ib); an earlier one through Pi(tile+1, i)
    const int a0 = tile + 1, ib = min(max(a0, Jt), nt - 1);
    S Pf[NN];
    if (a0 < ib) load_run_aligned<NN, S>(pi + ((long)a0 * ld + ib) * NN, Pf);
#pragma unroll 1
    for (int uu = 0; uu < UMAX; ++uu) {
        const int i = a0 + t + uu * (int)blockDim.x;
        if (i >= nt) break;
        S u[N], p[N];
        if (i + 1 == nt) {
            Aff<N, S> a;
#pragma unroll
            for (int c = 0; c < NA; ++c) comp(a, c) = tile_aff[(long)i * NA + c];
            S x[N];
#pragma unroll
            for (int c = 0; c < N; ++c) x[c] = xT[c];
            affine_apply<N, S>(a, x, u);
        } else {
#pragma unroll
            for (int c = 0; c < N; ++c) u[c] = tile_aff[(long)i * NA + NN + c];
        }
        S Q[NN];
        if (i < ib) {
            load_run_aligned<NN, S>(pi + ((long)a0 * ld + i) * NN, Q);          // Pi(tile+1, i)
            mat_vec<N, S>(Q, u, p);
        } else {
            load_run_aligned<NN, S>(mp + (long)(i - ib) * NN, Q);               // M^(i - ib)
            mat_vec<N, S>(Q, u, p);
            if (a0 < ib) {
                mat_vec<N, S>(Pf, p, u);
#pragma unroll
                for (int c = 0; c < N; ++c) p[c] = u[c];
            }
        }
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] += p[c];
    }
    block_vec_sum<N, S>(v, red);
    if (t == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) xe[i] = v[i];
    __syncthreads();
}

// The tiled-scan solve, one CTA of 128 threads per tile, all tiles
// co-resident (cooperative launch), three phases separated by two grid
// barriers:
//   1. the thread's filter offset W (its map v -> Psi v + W from v = 0) and
//      the tile's offset w_j;
//   2. the tile prefix (tile tables), the thread start values, the per-step
//      filter with the closed-loop offsets g_k staged, the thread's RTS offset
//      and the tile's RTS map;
//   3. the tile suffix, the thread end states and the per-step RTS pass.
// HB: the element offset depends on the held sample, b_k = Bb y_k + b0
// (block and exact elements): o_k gains -E_k^T P_k Bb y_k (folded into the
// gain of the steps after kc) and g_k gains E_k A^-1 Bb y_k.
template <int N, typename S, class Prod, bool HB>
__global__ void __launch_bounds__(128, (N <= 6 ? 3 : 1))
k_lti_scan(const __grid_constant__ Prod prod, const Red<N, S> prior, S* __restrict__ filt_out, CombineCtx ctx,
           S* __restrict__ final_out, S* __restrict__ x_out, S* __restrict__ filtT_out, const GridSync gs,
           const __grid_constant__ ScanArgs<N, Prod::W, S> sa)
{
    if constexpr (Prod::LINEAR_FOLD) {
        constexpr int M = Prod::W, NN = N * N, NA = NN + N, CT = NN + N;
        using ST = StepTab<N, S>;
        using SM = ScanSmem<N, M, S>;
        constexpr bool STAGE = SM::STAGE;
        extern __shared__ __align__(16) unsigned char smem_raw[];
        S* sm = reinterpret_cast<S*>(smem_raw);
        const ScanGeom& g = sa.g;
        const int B = blockDim.x, t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = B >> 5;
        const int tile = blockIdx.x;
        const bool trans = tile < g.Jt;                    // before kc: K_t steps, tabulated E_k
        const bool last = tile + 1 == g.nt;
        const bool powers = !trans;                        // in-tile scans on offsets with Phi_inf^d
        const int Kj = g.steps(tile);
        const long s0 = g.start(tile);
        const long k0 = s0 + (long)t * Kj;
        const long T = prod.T;
        const int nv = (int)max(0L, min((long)Kj, T - k0));
        // the first thread with fewer than Kj steps (B: none); in the last tile
        // the threads after it have none
        const int tp = last ? (int)min((long)B, (T - s0) / Kj) : B;
        S* red = sm;
        S* wt = sm + SM::wt(B);
        S* ys = sm + SM::ys(B);
        S* gst = sm + SM::gst(B, Kj);                      // staged g_k / states, exchange area
        S* tb = sm + SM::tabs(B, Kj);                      // powers or per-step E_k, o_k
        unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + SM::bar(B, g.K, g.Kt));
        S* mine = STAGE ? gst + t * Kj * N : x_out + k0 * N;   // this thread's g_k, then states

        // ---- phase 1: observations and tables into shared memory, the
        // thread's filter offset W (map v -> Psi v + W from v = 0), the
        // tile's filter offset w_j
        // (rounded up to whole 16-byte words: both source tables and the shared
        // area are padded to them)
        const bool tcopy = STAGE || !trans;
        const unsigned tbytes =
            tcopy ? (unsigned)((sizeof(S) * (trans ? (size_t)B * (g.Kt * CT + 2 * NN) : (size_t)(B + 1) * NN) + 15) / 16 * 16)
                  : 0u;
        const long yoff = s0 * M;
        const long ycnt = STAGE ? (long)B * Kj * M : 0;
        // the tile's rows by one bulk copy: all of them for full tiles, the
        // whole 16-byte words before T for the last tile (the rest below)
        const long yhave = min(ycnt, T * M - yoff);
        const long ybulk = yhave * (long)sizeof(S) / 16 * 16 / (long)sizeof(S);
        if (t == 0) mbar_init(bar, 1);
        __syncthreads();
        if (t == 0) {
            mbar_arrive_expect_tx(bar, tbytes + (unsigned)(sizeof(S) * ybulk));
            if (ybulk > 0) bulk_copy_g2s(ys, prod.y + yoff, (unsigned)(sizeof(S) * ybulk), bar);
            if (tbytes)
                bulk_copy_g2s(tb, trans ? sa.ttab + (long)tile * B * (g.Kt * CT + 2 * NN) : sa.pw, tbytes, bar);
            // the power table that the tile prefix and suffix sums read after
            // the grid barriers (data-independent, the same for every tile): into L2 now
            if (tile == 0) bulk_prefetch_l2(sa.mp, (unsigned)(sizeof(S) * (size_t)g.nt * NN));
        }
        for (long q = ybulk + t; q < ycnt; q += B) ys[q] = q < yhave ? prod.y[yoff + q] : S(0);
        // constants of the steps after kc (row kc; only read by threads with steps)
        S Einf[NN], oinf[N];
        if (!trans && nv > 0) {
            const S* r = sa.rows + sa.kc * ST::RS;
#pragma unroll
            for (int q = 0; q < NN; ++q) Einf[q] = __ldg(r + ST::oE + q);
#pragma unroll
            for (int q = 0; q < N; ++q) oinf[q] = __ldg(r + ST::oO + q);
        }
        const bool ok = mbar_wait_bounded(bar, 0, MBAR_POLLS);
        if (!__syncthreads_and(ok)) {
            if (t == 0) report_event(ctx.stats, EV_TIMEOUT);
            mbar_wait_bounded(bar, 0, MBAR_POLLS);      // the copy may still be in flight
        }
        const S* yt = STAGE ? ys + t * Kj * M : prod.y + k0 * M;
        // step constants: E_k and o_k of step i of this thread
        auto step_E = [&](int i, S (&E)[NN]) {
            if (trans) {
                if constexpr (STAGE) {
#pragma unroll
                    for (int q = 0; q < NN; ++q) E[q] = tb[(i * CT + q) * B + t];
                } else {
                    const S* r = sa.rows + (k0 + i) * ST::RS + ST::oE;
#pragma unroll
                    for (int q = 0; q < NN; ++q) E[q] = __ldg(r + q);
                }
            } else {
#pragma unroll
                for (int q = 0; q < NN; ++q) E[q] = Einf[q];
            }
        };
        auto step_o = [&](int i, S (&o)[N]) {
            if (!trans) {
#pragma unroll
                for (int q = 0; q < N; ++q) o[q] = oinf[q];
            } else if constexpr (STAGE) {
#pragma unroll
                for (int q = 0; q < N; ++q) o[q] = tb[(i * CT + NN + q) * B + t];
            } else {
                const S* r = sa.rows + (k0 + i) * ST::RS + ST::oO;
#pragma unroll
                for (int q = 0; q < N; ++q) o[q] = __ldg(r + q);
            }
        };
        // v <- E^T v + o + G y_{k+1} - Gr
        // (the data term is formed apart from the recursion, so that its
        // shared-memory loads overlap the E^T v chain)
        auto fstep = [&](int i, const S (&E)[NN], S (&v)[N]) {
            S o[N], gy[N], nv2[N];
            step_o(i, o);
#pragma unroll
            for (int a = 0; a < N; ++a) {
                S acc = o[a] - prod.p.Gr[a];
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    S gc;
                    if constexpr (HB)
                        gc = trans ? prod.p.G[a * M + m] + __ldg(sa.mk + (k0 + i) * NN + a * M + m)
                                   : __ldg(sa.gs + a * M + m);
                    else
                        gc = prod.p.G[a * M + m];
                    acc = fma(gc, yt[i * M + m], acc);
                }
                gy[a] = acc;
            }
#pragma unroll
            for (int a = 0; a < N; ++a) {
                S acc = E[a] * v[0];
#pragma unroll
                for (int q = 1; q < N; ++q) acc = fma(E[q * N + a], v[q], acc);
                nv2[a] = acc + gy[a];
            }
#pragma unroll
            for (int a = 0; a < N; ++a) v[a] = nv2[a];
        };
        S W[N];
#pragma unroll
        for (int a = 0; a < N; ++a) W[a] = S(0);
#pragma unroll 1
        for (int i = 0; i < nv; ++i) {
            S E[NN];
            step_E(i, E);
            fstep(i, E, W);
        }
        // the thread's map matrix Phi (RTS direction; the filter map's is Phi^T)
        Aff<N, S> Fm;                                  // filter map (Psi, W) on the full-map path
        S We[N];                                       // exclusive in-tile filter offset (powers path)
        if (powers) {
            // warp-inclusive prefix of the offsets: W_l <- Psi^d W_{l-d} + W_l
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                S o[N], p[N];
#pragma unroll
                for (int a = 0; a < N; ++a) o[a] = __shfl_up_sync(0xffffffffu, W[a], d);
                if (lane >= d) {
                    mat_tvec<N, S>(tb + d * NN, o, p);
#pragma unroll
                    for (int a = 0; a < N; ++a) W[a] += p[a];
                }
            }
            if (lane == 31)
#pragma unroll
                for (int a = 0; a < N; ++a) wt[wid * N + a] = W[a];
            __syncthreads();
            S WP[N];                                   // composition of the warps before this one
#pragma unroll
            for (int a = 0; a < N; ++a) WP[a] = S(0);
            for (int w2 = 0; w2 < wid; ++w2) {
                S p[N];
                mat_tvec<N, S>(tb + 32 * NN, WP, p);
#pragma unroll
                for (int a = 0; a < N; ++a) WP[a] = p[a] + wt[w2 * N + a];
            }
            {
                S p[N];
                mat_tvec<N, S>(tb + (lane + 1) * NN, WP, p);
#pragma unroll
                for (int a = 0; a < N; ++a) W[a] += p[a];          // inclusive tile prefix
            }
#pragma unroll
            for (int a = 0; a < N; ++a) {
                const S up = __shfl_up_sync(0xffffffffu, W[a], 1);
                We[a] = lane == 0 ? WP[a] : up;
            }
            if (t == B - 1)
#pragma unroll
                for (int a = 0; a < N; ++a) sa.w[(long)tile * N + a] = W[a];
        } else {
            // full maps: Phi of this thread (table, or the product of its steps)
            if (nv == Kj && trans) {
                if constexpr (STAGE) {
#pragma unroll
                    for (int q = 0; q < NN; ++q) Fm.F[q] = tb[B * g.Kt * CT + q * B + t];
                } else {
#pragma unroll
                    for (int q = 0; q < NN; ++q) Fm.F[q] = __ldg(sa.phit + ((long)tile * B + t) * NN + q);
                }
            } else if (nv == Kj) {
#pragma unroll
                for (int q = 0; q < NN; ++q) Fm.F[q] = tb[NN + q];            // Phi_inf
            } else {
#pragma unroll
                for (int q = 0; q < NN; ++q) Fm.F[q] = q % (N + 1) == 0 ? S(1) : S(0);
#pragma unroll 1
                for (int i = 0; i < nv; ++i) {
                    S E[NN], F2[NN];
                    step_E(i, E);
                    ms::mm<N, S>(Fm.F, E, F2);
#pragma unroll
                    for (int q = 0; q < NN; ++q) Fm.F[q] = F2[q];
                }
            }
            // filter map: matrix Phi^T, offset W
            {
                S Ft[NN];
#pragma unroll
                for (int q = 0; q < NN; ++q) Ft[q] = Fm.F[(q % N) * N + q / N];
#pragma unroll
                for (int q = 0; q < NN; ++q) Fm.F[q] = Ft[q];
            }
#pragma unroll
            for (int a = 0; a < N; ++a) Fm.c[a] = W[a];
            if (!last) {
                // w_j = sum_t Q_t W_t (Q_t the plan-time suffix products)
                S Q[NN], p[N];
                if constexpr (STAGE) {
#pragma unroll
                    for (int q = 0; q < NN; ++q) Q[q] = tb[B * (g.Kt * CT + NN) + q * B + t];
                } else {
#pragma unroll
                    for (int q = 0; q < NN; ++q) Q[q] = __ldg(sa.qsuf + ((long)tile * B + t) * NN + q);
                }
                mat_vec<N, S>(Q, W, p);
                block_vec_sum<N, S>(p, red);
                if (t == 0)
#pragma unroll
                    for (int a = 0; a < N; ++a) sa.w[(long)tile * N + a] = p[a];
            }
        }
        grid_sync(gs, 1, ctx.stats);

        // ---- phase 2: tile prefix, thread start values, per-step filter,
        // thread RTS maps and the tile's RTS map
        S v[N];
        {
            S pv[N];
            scan_tile_prefix<N, S>(sa.qt, sa.tld, sa.mp, sa.w, tile, g.Jt, prior.v, red, pv);
            S* vt = wt + 2 * (B / 32) * N;
            if (t == 0)
#pragma unroll
                for (int a = 0; a < N; ++a) vt[a] = pv[a];
            __syncthreads();
            S vtile[N];
#pragma unroll
            for (int a = 0; a < N; ++a) vtile[a] = vt[a];
            if (powers) {
                S p[N];
                mat_tvec<N, S>(tb + t * NN, vtile, p);
#pragma unroll
                for (int a = 0; a < N; ++a) v[a] = p[a] + We[a];
            } else {
                // v at thread t's start = (F_{t-1} o ... o F_0)(v_tile): the end
                // states of the reversed sequence
                Aff<N, S> H = Fm;
                reverse_maps<N, S>(H, gst);
                S* xe = vt;                            // block_aff_end_states reads thread 0's copy
                S r[N];
                block_aff_end_states<N, S>(H, xe, red, r);
                reverse_vec<N, S>(r, gst);
#pragma unroll
                for (int a = 0; a < N; ++a) v[a] = r[a];
            }
        }
        // forward: g_k = E_k (A^-1 C v_k + A^-1 b_k) staged; v_{k+1} = E_k^T v_k + o_k + G y - Gr
#pragma unroll 1
        for (int i = 0; i < nv; ++i) {
            const long k = k0 + i;
            S E[NN];
            step_E(i, E);
            if (filt_out) {
                const S* r = sa.rows + min(k, sa.kc) * ST::RS;
#pragma unroll
                for (int a = 0; a < N; ++a) filt_out[k * Red<N, S>::NCOMP + a] = v[a];
#pragma unroll
                for (int q = 0; q < Sym<N>::SZ; ++q) filt_out[k * Red<N, S>::NCOMP + N + q] = __ldg(r + ST::oP + q);
            }
            S gk[N];
            if (!trans) {
                // steps after kc: g_k = (E_inf A^-1 C) v_k + E_inf A^-1 b_k with the
                // products formed once at plan time
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    S acc = sa.EAib[a];
#pragma unroll
                    for (int q = 0; q < N; ++q) acc = fma(sa.EAiC[a * N + q], v[q], acc);
                    if constexpr (HB)
#pragma unroll
                        for (int m = 0; m < M; ++m) acc = fma(sa.EAiBb[a * M + m], yt[i * M + m], acc);
                    gk[a] = acc;
                }
            } else {
                S u[N];
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    S acc = sa.Aib[a];
#pragma unroll
                    for (int q = 0; q < N; ++q) acc = fma(sa.AiC[a * N + q], v[q], acc);
                    if constexpr (HB)
#pragma unroll
                        for (int m = 0; m < M; ++m) acc = fma(sa.AiBb[a * M + m], yt[i * M + m], acc);
                    u[a] = acc;
                }
                mat_vec<N, S>(E, u, gk);
            }
            stage_state<N, S>(mine + i * N, gk);
            fstep(i, E, v);
        }
        S* xT = x_out + T * N;
        if (last && k0 < T && k0 + Kj >= T) {          // the value function at x_T and its minimiser
            Red<N, S> XT;
            const S* rT = sa.rows + min(T, sa.kc) * ST::RS;
#pragma unroll
            for (int a = 0; a < N; ++a) XT.v[a] = v[a];
#pragma unroll
            for (int q = 0; q < Sym<N>::SZ; ++q) XT.P[q] = __ldg(rT + ST::oP + q);
            if (final_out) aos_store(final_out, 0, XT);
            // x_T = P_T^-1 v_T with the plan-time FP64 inverse, accumulated in FP64
#pragma unroll
            for (int a = 0; a < N; ++a) {
                double acc = 0.0;
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(__ldg(sa.pinv + a * N + q), double(v[q]), acc);
                xT[a] = S(acc);
            }
            if (filtT_out)
#pragma unroll
                for (int q = 0; q < Red<N, S>::NCOMP; ++q) filtT_out[q] = comp(XT, q);
        }
        // backward over the thread's steps: z <- E_k z + g_k (staged in place when asked)
        auto back = [&](S (&z)[N], bool stage) {
#pragma unroll 1
            for (int i = nv - 1; i >= 0; --i) {
                S E[NN], nz[N];
                step_E(i, E);
                mat_vec<N, S>(E, z, nz);
#pragma unroll
                for (int a = 0; a < N; ++a) z[a] = nz[a] + mine[i * N + a];
                if (stage) stage_state<N, S>(mine + i * N, z);
            }
        };
        S beta[N];
#pragma unroll
        for (int a = 0; a < N; ++a) beta[a] = S(0);
        back(beta, false);
        S Be[N];                                       // exclusive in-tile RTS suffix offset (powers path)
        Aff<N, S> Rm;                                  // RTS map (full-map path)
        if (powers) {
            // warp-inclusive suffix: B_l <- B_l + Phi^d B_{l+d} over the
            // threads before tp (the partial thread of the last tile enters
            // through its start state, below)
            S Bs[N];
#pragma unroll
            for (int a = 0; a < N; ++a) Bs[a] = t < tp ? beta[a] : S(0);
            S* bp = wt + 2 * (B / 32) * N + N;         // beta of thread tp
            if (t == tp)
#pragma unroll
                for (int a = 0; a < N; ++a) bp[a] = beta[a];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                S o[N], p[N];
#pragma unroll
                for (int a = 0; a < N; ++a) o[a] = __shfl_down_sync(0xffffffffu, Bs[a], d);
                if (lane + d < 32) {
                    mat_vec<N, S>(tb + d * NN, o, p);
#pragma unroll
                    for (int a = 0; a < N; ++a) Bs[a] += p[a];
                }
            }
            S* bt = wt + (B / 32) * N;
            if (lane == 0)
#pragma unroll
                for (int a = 0; a < N; ++a) bt[wid * N + a] = Bs[a];
            __syncthreads();
            S BN[N];                                   // composition of the warps after this one
#pragma unroll
            for (int a = 0; a < N; ++a) BN[a] = S(0);
            for (int w2 = nw - 1; w2 > wid; --w2) {
                S p[N];
                mat_vec<N, S>(tb + 32 * NN, BN, p);
#pragma unroll
                for (int a = 0; a < N; ++a) BN[a] = bt[w2 * N + a] + p[a];
            }
            {
                S p[N];
                mat_vec<N, S>(tb + (32 - lane) * NN, BN, p);
#pragma unroll
                for (int a = 0; a < N; ++a) Bs[a] += p[a];         // inclusive tile suffix
            }
#pragma unroll
            for (int a = 0; a < N; ++a) {
                const S dn = __shfl_down_sync(0xffffffffu, Bs[a], 1);
                Be[a] = lane == 31 ? BN[a] : dn;
            }
            if (t == 0) {
                if (tp < B) {                          // + Phi_inf^tp beta_tp
                    S p[N];
                    mat_vec<N, S>(tb + tp * NN, bp, p);
#pragma unroll
                    for (int a = 0; a < N; ++a) Bs[a] += p[a];
                }
#pragma unroll
                for (int a = 0; a < N; ++a) sa.taff[(long)tile * NA + NN + a] = Bs[a];
            }
        } else {
            {
                S Ft[NN];                              // back to the RTS direction
#pragma unroll
                for (int q = 0; q < NN; ++q) Ft[q] = Fm.F[(q % N) * N + q / N];
#pragma unroll
                for (int q = 0; q < NN; ++q) Rm.F[q] = Ft[q];
            }
#pragma unroll
            for (int a = 0; a < N; ++a) Rm.c[a] = beta[a];
            Aff<N, S> H = Rm;
            __syncthreads();                           // the composition area is free
            block_aff_reduce<N, S>(H, red);
            if (t == 0) aos_store(sa.taff, (long)tile, H);
        }
        grid_sync(gs, 2, ctx.stats);

        // ---- phase 3: tile suffix, thread end states, per-step states, bulk store
        S x[N];
        {
            S* xe_sh = red + (B / 32) * (NA + N);
            scan_tile_suffix<N, S>(sa.pi, sa.tld, sa.mp, sa.taff, tile, g.nt, g.Jt, xT, red, xe_sh);
            if (powers) {
                // state at thread tp's start (tp = B: the tile's end state)
                S* xs = wt + 2 * (B / 32) * N;
                if (tp < B) {
                    if (t == 0) {
                        const S* bp = wt + 2 * (B / 32) * N + N;
                        S Ep[NN], xv[N], p[N];
#pragma unroll
                        for (int q = 0; q < NN; ++q) Ep[q] = __ldg(sa.ep + q);
#pragma unroll
                        for (int a = 0; a < N; ++a) xv[a] = xe_sh[a];
                        mat_vec<N, S>(Ep, xv, p);
#pragma unroll
                        for (int a = 0; a < N; ++a) xs[a] = p[a] + bp[a];
                    }
                    __syncthreads();
                } else {
                    xs = xe_sh;
                }
                S xe[N], p[N];
#pragma unroll
                for (int a = 0; a < N; ++a) xe[a] = xs[a];
                mat_vec<N, S>(tb + (tp - 1 - min(t, tp - 1)) * NN, xe, p);
#pragma unroll
                for (int a = 0; a < N; ++a) x[a] = t < tp ? p[a] + Be[a] : xe_sh[a];
            } else {
                block_aff_end_states<N, S>(Rm, xe_sh, red, x);
            }
        }
        back(x, true);                                 // x_k = E_k x_{k+1} + g_k, in place of g_k
        if constexpr (STAGE) {
            __syncthreads();
            const long base = s0 * N;
            const long cnt = min((long)B * Kj * N, T * N - base);
            long done = 0;
            if ((reinterpret_cast<uintptr_t>(x_out + base) & 15) == 0) {
                done = cnt * (long)sizeof(S) / 16 * 16 / (long)sizeof(S);
                if (t == 0 && done > 0) {
                    fence_proxy_async_smem();
                    bulk_copy_s2g(x_out + base, gst, (unsigned)(done * sizeof(S)));
                    bulk_commit_and_wait();
                }
            }
            for (long idx = done + t; idx < cnt; idx += B) x_out[base + idx] = gst[idx];
            __syncthreads();
        }
    }
}

}  // namespace mapk
