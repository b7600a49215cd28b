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
// the P_k recursion, and with it E_k, M_k C = (I + C P_k)^-1 C (symmetric),
// mb_k = (I + C P_k)^-1 b and o_k = -E_k^T P_k b, do not depend on the data.
// They are therefore evaluated once per model and geometry, in FP64 (the
// plan-time kernel k_lti_steptab), and a solve only runs the data-dependent
// part of every step:
//   g_k = MC_k v_k + mb_k,  v_{k+1} = E_k^T v_k + o_k + G y_{k+1} - Gr,
//   x_k = E_k x_{k+1} + g_k.
// This is the same combine evaluated with its data-independent factors
// precomputed, as lti_fold.cuh does for the folds and tile tables.
//
// P_k converges to the fixed point of the recursion (the stationary filter)
// geometrically.  The table holds the steps k < KT (KT = min(T + 1, a cap), so
// that a short scan has its every P_k up to P_T); when T >= KT, row kc stands
// for every later step, where kc is the first step
// from which every tabulated P_k agrees with the P of the scan's last full
// tile to a relative tolerance of 2^-25 (FP32 solves) or 1e-14 (FP64 solves)
// per entry (|dP_ab| <= tol sqrt(P_aa P_bb)): below the solve's own rounding.
// When the table does not reach that point (slowly converging models) the
// solve keeps the per-step Riccati path of scan.cuh.
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
#pragma once
#include "scan.cuh"

namespace mapk {

// Layout of the step-table buffer (offsets in bytes): a few counters, the
// FP64 pre_s (A, C, J; s < BMAX), the FP64 i-step folds (A, C, J; i <= KMAX)
// and the FP64 P_j of the tiles (all full N x N matrices), then the rows of
// the steps k < KT in the solve's precision S (E, MC packed, o, mb, P packed)
// and the composite maps Phi of the threads that start at k = g K < KT.
template <int N, typename S>
struct StepTab {
    static constexpr int NN = N * N, NS = Sym<N>::SZ;
    static constexpr int oE = 0, oMC = NN, oO = NN + NS, oMB = NN + NS + N, oP = NN + NS + 2 * N;
    static constexpr int RS = ((NN + 2 * NS + 2 * N) * (int)sizeof(S) + 15) / 16 * 16 / (int)sizeof(S);
    static constexpr int BMAX = 128, KMAX = 64;
    __host__ __device__ static constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
    __host__ __device__ static constexpr size_t pre_off() { return 256; }
    __host__ __device__ static constexpr size_t fold_off() { return al(pre_off() + sizeof(double) * BMAX * 3 * NN); }
    __host__ __device__ static constexpr size_t p64_off() { return al(fold_off() + sizeof(double) * (KMAX + 1) * 3 * NN); }
    __host__ __device__ static constexpr size_t rows_off(long nt) { return al(p64_off() + sizeof(double) * nt * NN); }
    __host__ __device__ static constexpr long phi_count(long kt) { return kt / 8 + 2; }
    __host__ __device__ static constexpr size_t phi_off(long nt, long kt) { return al(rows_off(nt) + sizeof(S) * kt * RS); }
    // then the same constants (E, MC, o, mb: WC components) warp-interleaved by
    // thread: component c of step i of thread g at ((g/32 K + i) WC + c) 32 + g%32,
    // so that a warp's load of one component of one step is one 128-byte line
    static constexpr int WC = NN + NS + 2 * N;
    __host__ __device__ static constexpr long wi_threads(long kt, int K) { return ((kt + K - 1) / K + 31) / 32 * 32; }
    __host__ __device__ static constexpr size_t wi_off(long nt, long kt)
    {
        return al(phi_off(nt, kt) + sizeof(S) * phi_count(kt) * NN);
    }
    __host__ __device__ static constexpr long wi_index(long g, int i, int c, int K)
    {
        return (((g >> 5) * K + i) * WC + c) * 32 + (g & 31);
    }
    __host__ __device__ static constexpr size_t bytes(long nt, long kt, int K)
    {
        return wi_off(nt, kt) + sizeof(S) * (size_t)wi_threads(kt, K) * K * WC;
    }
    // table length cap: the FP32 table converges within 2^-25 earlier
    static constexpr long cap() { return sizeof(S) == 4 ? 16384 : 32768; }
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
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = L[c * N + i];              // (L^T)[i][c]
#pragma unroll
            for (int k = 0; k < i; ++k) s = fma(-R[i * N + k], Z[k * N + c], s);
            Z[i * N + c] = s / R[i * N + i];
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

}  // namespace steptab_detail

// One thread per tabulated step k < KT (FP64): P_k from the tile, thread-prefix
// and i-step tables (see the top of this file), then the row of constants and,
// for the first step of a thread (k = g K), the thread's composite closed-loop
// map Phi_g = (I + C_K P_k)^-1 A_K of its K-step fold (the composition of its
// K per-step maps: the closed-loop map of the combined element).  With check,
// every step whose P_k differs from P_ref beyond tol raises meta[0] to k + 1;
// meta[1] counts non-positive Cholesky pivots.
template <int N, int M, typename S>
__global__ void __launch_bounds__(128)
k_lti_steptab(const LtiParams<N, M, double> p, int K, int B, int nt, long KT, int check, double tol,
              char* __restrict__ tab)
{
    namespace sd = steptab_detail;
    using ST = StepTab<N, S>;
    constexpr int NN = N * N;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= KT) return;
    const double* pre = reinterpret_cast<const double*>(tab + ST::pre_off());
    const double* fold = reinterpret_cast<const double*>(tab + ST::fold_off());
    const double* p64 = reinterpret_cast<const double*>(tab + ST::p64_off());
    unsigned long long* meta = reinterpret_cast<unsigned long long*>(tab);
    S* row = reinterpret_cast<S*>(tab + ST::rows_off(nt)) + k * ST::RS;
    const long L = (long)B * K;
    const int j = (int)(k / L), s = (int)((k % L) / K), i = (int)(k % K);
    double P[NN];
    sd::load_full<N>(p64 + (long)j * NN, P);
    bool ok = true;
    if (s > 0) ok = sd::apply_p<N>(pre + (long)s * 3 * NN, P) && ok;
    if (i > 0) ok = sd::apply_p<N>(fold + (long)i * 3 * NN, P) && ok;
    // per-step constants from Z of (P, C)
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
    // the row, and the same constants in the warp-interleaved copy
    S* wi = reinterpret_cast<S*>(tab + ST::wi_off(nt, KT));
    const long g = k / K;
    auto put = [&](int off, double val) {
        row[off] = S(val);
        wi[ST::wi_index(g, i, off, K)] = S(val);
    };
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double e = A[a * N + c];
#pragma unroll
            for (int q = 0; q < N; ++q) e = fma(-CZt[a * N + q], ZA[q * N + c], e);
            E[a * N + c] = e;
            put(ST::oE + a * N + c, e);
        }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int c = a; c < N; ++c) {
            double mc = 0.5 * (C[a * N + c] + C[c * N + a]);
#pragma unroll
            for (int q = 0; q < N; ++q) mc = fma(-CZt[a * N + q], CZt[c * N + q], mc);
            put(ST::oMC + Sym<N>::at(a, c), mc);
            row[ST::oP + Sym<N>::at(a, c)] = S(P[a * N + c]);
        }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        double mb = b[a], o = 0.0;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            mb = fma(-CZt[a * N + q], Zb[q], mb);
            o = fma(-E[q * N + a], Pb[q], o);
        }
        put(ST::oMB + a, mb);
        put(ST::oO + a, o);
    }
    if (i == 0) {
        // Phi_g = (I + C_K P)^-1 A_K = A_K - C_K Z_K^T (Z_K A_K)
        const double* fK = fold + (long)K * 3 * NN;
        double AK[NN], CK[NN], ZK[NN];
        sd::load_full<N>(fK, AK);
        sd::load_full<N>(fK + NN, CK);
#pragma unroll
        for (int q = 0; q < NN; ++q) CK[q] = 0.5 * (CK[q] + CK[(q % N) * N + q / N]);
        ok = sd::zfactor<N>(P, CK, ZK) && ok;
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int c = 0; c < N; ++c) {
                double za = 0.0, cz = 0.0;
#pragma unroll
                for (int q = 0; q < N; ++q) {
                    za = fma(ZK[a * N + q], AK[q * N + c], za);
                    cz = fma(CK[a * N + q], ZK[c * N + q], cz);
                }
                ZA[a * N + c] = za;
                CZt[a * N + c] = cz;
            }
        S* ph = reinterpret_cast<S*>(tab + ST::phi_off(nt, KT)) + (k / K) * NN;
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int c = 0; c < N; ++c) {
                double e = AK[a * N + c];
#pragma unroll
                for (int q = 0; q < N; ++q) e = fma(-CZt[a * N + q], ZA[q * N + c], e);
                ph[a * N + c] = S(e);
            }
    }
    if (check) {
        double Pr[NN];
        sd::load_full<N>(p64 + (long)(nt >= 2 ? nt - 2 : 0) * NN, Pr);
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
// single-launch RTS solve with the per-step tables
// ---------------------------------------------------------------------------
template <typename S>
struct TabArgs {
    const S* rows;      // step rows (StepTab)
    const S* phi;       // thread maps
    const S* wi;        // the rows warp-interleaved by thread (threads that start before kc)
    long kc;            // steps k >= kc read row kc
    long gc;            // threads g >= gc read map gc
};

// per-step constants of one table row
template <int N, typename S>
struct StepC {
    S E[N * N];
    S MC[Sym<N>::SZ];
    S o[N];
    S mb[N];
};

template <int N, typename S>
__device__ __forceinline__ void load_stepc(const S* __restrict__ row, StepC<N, S>& c)
{
    using ST = StepTab<N, S>;
#pragma unroll
    for (int q = 0; q < N * N; ++q) c.E[q] = __ldg(row + ST::oE + q);
#pragma unroll
    for (int q = 0; q < Sym<N>::SZ; ++q) c.MC[q] = __ldg(row + ST::oMC + q);
#pragma unroll
    for (int q = 0; q < N; ++q) {
        c.o[q] = __ldg(row + ST::oO + q);
        c.mb[q] = __ldg(row + ST::oMB + q);
    }
}

// step i of thread g from the warp-interleaved copy (coalesced over the warp)
template <int N, typename S>
__device__ __forceinline__ void load_stepc_wi(const S* __restrict__ wi, long g, int i, int K, StepC<N, S>& c)
{
    using ST = StepTab<N, S>;
    const S* p = wi + ST::wi_index(g, i, 0, K);
#pragma unroll
    for (int q = 0; q < N * N; ++q) c.E[q] = __ldg(p + (ST::oE + q) * 32);
#pragma unroll
    for (int q = 0; q < Sym<N>::SZ; ++q) c.MC[q] = __ldg(p + (ST::oMC + q) * 32);
#pragma unroll
    for (int q = 0; q < N; ++q) {
        c.o[q] = __ldg(p + (ST::oO + q) * 32);
        c.mb[q] = __ldg(p + (ST::oMB + q) * 32);
    }
}

template <int N, typename S>
__device__ __forceinline__ void load_stepE_wi(const S* __restrict__ wi, long g, int i, int K, S (&E)[N * N])
{
    using ST = StepTab<N, S>;
    const S* p = wi + ST::wi_index(g, i, 0, K);
#pragma unroll
    for (int q = 0; q < N * N; ++q) E[q] = __ldg(p + (ST::oE + q) * 32);
}

template <int N, typename S>
__device__ __forceinline__ void load_stepE(const S* __restrict__ row, S (&E)[N * N])
{
#pragma unroll
    for (int q = 0; q < N * N; ++q) E[q] = __ldg(row + StepTab<N, S>::oE + q);
}

// shared memory of k_lti_solve_tab (offsets in scalars): the (b, eta) nodes
// and the tile's prefix, the composition area, the tile's observations (bulk
// copy), the Gamma_i, two mbarriers, the level constants and the co table;
// after the thread prefixes the per-step g_k of every thread (K N scalars per
// thread, in the tile's output order) overwrite the level constants and the
// co table, and the RTS phase turns them into the states in place.
template <int N, int M, typename S>
struct TabSmem {
    using FL = FoldLayout<N, M, S>;
    using FS = FusedSmem<N, M, S>;
    __host__ __device__ static constexpr int gst(int B, int K) { return FS::lv(B, K); }
    __host__ __device__ static constexpr size_t bytes(int B, int K)
    {
        const int e = FS::co(B, K) + B * FL::CS, g = gst(B, K) + B * K * N;
        return sizeof(S) * (size_t)(e > g ? e : g);
    }
};

template <int N, typename S, class Prod>
__global__ void __launch_bounds__(128, (N <= 6 ? 3 : 1))
k_lti_solve_tab(const __grid_constant__ Prod prod, int K, const LtiTiles<S> lt, const Red<N, S> prior,
                S* __restrict__ tile_aff, S* __restrict__ filt_out, CombineCtx ctx, S* __restrict__ final_out,
                S* __restrict__ x_out, S* __restrict__ filtT_out, const GridSync gs, const TabArgs<S> tb)
{
    if constexpr (Prod::LINEAR_FOLD && N <= 6) {
        constexpr int M = Prod::W, NN = N * N, NS = Sym<N>::SZ;
        using FL = FoldLayout<N, M, S>;
        using FS = FusedSmem<N, M, S>;
        using ST = StepTab<N, S>;
        extern __shared__ __align__(16) unsigned char smem_raw[];
        S* sm = reinterpret_cast<S*>(smem_raw);
        const int B = blockDim.x, t = threadIdx.x;
        const int tile = blockIdx.x;
        const long gthr = (long)tile * B + t;
        const long k0 = gthr * K;
        const long T = prod.T;
        const bool last = tile + 1 == (int)gridDim.x;
        const S* fold = lt.fold;
        S* bq = sm + FS::bq(B);
        S* ps = sm + FS::pin(B);
        S* red = sm + FS::red(B);
        S* ys = sm + FS::ys(B);
        S* gam = sm + FS::gam(B, K);
        S* lv = sm + FS::lv(B, K);
        S* co = sm + FS::co(B, K);
        S* gst = sm + TabSmem<N, M, S>::gst(B, K);
        unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + FS::bar(B, K));

        // ---- phase 1: the tile's observations, per-thread folds, up-sweep, w_j
        const int LB = ilog2(B);
        const unsigned ybytes = last ? 0u : (unsigned)(sizeof(S) * (size_t)B * K * M);
        const unsigned lbytes = (unsigned)(sizeof(S) * (size_t)LB * FL::LS);
        const unsigned cbytes = (unsigned)(sizeof(S) * (size_t)(B - 1) * FL::CS);
        const unsigned gbytes = (unsigned)(sizeof(S) * (size_t)((K * FL::GS + 3) / 4 * 4));
        unsigned long long* bar_co = bar + 1;
        if (t == 0) {
            mbar_init(bar, 1);
            mbar_init(bar_co, 1);
        }
        __syncthreads();
        if (t == 0) {
            mbar_arrive_expect_tx(bar, ybytes + lbytes + gbytes);
            if (!last) bulk_copy_g2s(ys, prod.y + (long)tile * B * K * M, ybytes, bar);
            bulk_copy_g2s(lv, fold + FL::oL, lbytes, bar);
            bulk_copy_g2s(gam, fold + FL::oG, gbytes, bar);
            mbar_arrive_expect_tx(bar_co, cbytes);
            bulk_copy_g2s(co, fold + FL::oCo, cbytes, bar_co);
        }
        if (!last) {
            for (int q = t; q < NS; q += B) red[q] = lt.P[(long)tile * NS + q];
            for (int q = t; q < NN; q += B) red[NS + q] = lt.F[(long)tile * NN + q];
        }
        if (last) {
            const long base = (long)tile * B * K * M, have = T * M - base;
            for (long q = t; q < (long)B * K * M; q += B) ys[q] = q < have ? prod.y[base + q] : S(0);
        }
        const bool ok = mbar_wait_bounded(bar, 0, MBAR_POLLS);
        if (!__syncthreads_and(ok)) {
            if (t == 0 && ctx.stats) atomicAdd(ctx.stats + 2, 1ull);
            mbar_wait_bounded(bar, 0, MBAR_POLLS);
        }
        const S* yt = ys + t * K * M;
        S leaf[2 * N];
        if (!last || k0 + K <= T) {
#pragma unroll
            for (int q = 0; q < N; ++q) { leaf[q] = __ldg(fold + FL::ob + q); leaf[N + q] = __ldg(fold + FL::oe + q); }
#pragma unroll 2
            for (int i = 0; i < K; ++i) {
                const S* gi = gam + i * FL::GS;
#pragma unroll
                for (int a = 0; a < N; ++a)
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        leaf[a] = fma(gi[a * M + c], yt[i * M + c], leaf[a]);
                        leaf[N + a] = fma(gi[(N + a) * M + c], yt[i * M + c], leaf[N + a]);
                    }
            }
        } else {
#pragma unroll
            for (int c = 0; c < 2 * N; ++c) leaf[c] = S(0);
        }
#pragma unroll
        for (int c = 0; c < 2 * N; ++c) bq[c * B + t] = leaf[c];
        lti_tree_up<N, M, S>(bq, lv);
        if (!last && t == 0) {                     // w_j = eta_j - F_j P_j b_j
            const S* rq = bq + lti_node_level(2 * N, B, ilog2(B));
            S Pb[N];
#pragma unroll
            for (int a = 0; a < N; ++a) {
                S acc = S(0);
#pragma unroll
                for (int c = 0; c < N; ++c) acc = fma(red[Sym<N>::at(a, c)], rq[c], acc);
                Pb[a] = acc;
            }
#pragma unroll
            for (int a = 0; a < N; ++a) {
                S acc = rq[N + a];
#pragma unroll
                for (int c = 0; c < N; ++c) acc = fma(-red[NS + a * N + c], Pb[c], acc);
                lt.w[(long)tile * N + a] = acc;
            }
        }
        grid_sync(gs, 1, ctx.stats);

        // ---- phase 2: tile prefix, thread prefixes, per-step filter, tile map
        Red<N, S> pin, X;
        lti_tile_prefix_sum<N, S>(lt, tile, gridDim.x, prior, red, pin);
        if (t == 0) node_store(pin, ps);
        if (!mbar_wait_bounded(bar_co, 0, MBAR_POLLS) && ctx.stats && t == 0) atomicAdd(ctx.stats + 2, 1ull);
        lti_tree_down_linear<N, M, S>(bq, co);     // starts and ends with a barrier
        {
            Red<N, S> P;
            node_load(ps, P);
            S dl[2 * N];
#pragma unroll
            for (int c = 0; c < 2 * N; ++c) dl[c] = bq[c * B + t];
            if (k0 < T)
                lti_thread_value<N, M, S>(fold, dl, P, ctx, X);
            else
                X = P;
        }
        __syncthreads();                           // level constants and co table are dead: gst takes them
        const int nv = (int)max(0L, min((long)K, T - k0));   // this thread's steps before T
        const bool steady = k0 >= tb.kc;
        StepC<N, S> c;
        if (steady && nv > 0) load_stepc<N, S>(tb.rows + tb.kc * ST::RS, c);   // row kc exists when kc < T
        S* mine = gst + t * K * N;
        S v[N];
#pragma unroll
        for (int a = 0; a < N; ++a) v[a] = X.v[a];
        // forward: g_k = MC v_k + mb; v_{k+1} = E^T v_k + o + G y_{k+1} - Gr
        // (threads that start before kc read the interleaved rows, two steps
        // per iteration so that the next step's loads are in flight)
        auto fwd = [&](int i, const StepC<N, S>& c) {
            const long k = k0 + i;
            const S* row = tb.rows + min(k, tb.kc) * ST::RS;
            if (filt_out) {
#pragma unroll
                for (int a = 0; a < N; ++a) filt_out[k * Red<N, S>::NCOMP + a] = v[a];
#pragma unroll
                for (int q = 0; q < NS; ++q) filt_out[k * Red<N, S>::NCOMP + N + q] = __ldg(row + ST::oP + q);
            }
            S g[N], nvv[N];
#pragma unroll
            for (int a = 0; a < N; ++a) {
                S acc = c.mb[a];
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(c.MC[Sym<N>::at(a, q)], v[q], acc);
                g[a] = acc;
            }
#pragma unroll
            for (int a = 0; a < N; ++a) {
                S acc = c.o[a] - prod.p.Gr[a];
#pragma unroll
                for (int m = 0; m < M; ++m) acc = fma(prod.p.G[a * M + m], yt[i * M + m], acc);
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(c.E[q * N + a], v[q], acc);
                nvv[a] = acc;
            }
            stage_state<N, S>(mine + i * N, g);
#pragma unroll
            for (int a = 0; a < N; ++a) v[a] = nvv[a];
        };
        if (steady) {
#pragma unroll 1
            for (int i = 0; i < nv; ++i) fwd(i, c);
        } else {
            int i = 0;
#pragma unroll 1
            for (; i + 1 < nv; i += 2) {
                StepC<N, S> c0, c1;
                load_stepc_wi<N, S>(tb.wi, gthr, i, K, c0);
                load_stepc_wi<N, S>(tb.wi, gthr, i + 1, K, c1);
                fwd(i, c0);
                fwd(i + 1, c1);
            }
            if (i < nv) {
                load_stepc_wi<N, S>(tb.wi, gthr, i, K, c);
                fwd(i, c);
            }
        }
        S* xT = x_out + T * N;
        if (last && k0 < T && k0 + K >= T) {        // the value function at x_T and its minimiser
            Red<N, S> XT;
            const S* rT = tb.rows + min(T, tb.kc) * ST::RS;
#pragma unroll
            for (int a = 0; a < N; ++a) XT.v[a] = v[a];
#pragma unroll
            for (int q = 0; q < NS; ++q) XT.P[q] = __ldg(rT + ST::oP + q);
            if (final_out) aos_store(final_out, 0, XT);
            S xt[N];
            if (!red_argmin<N, S>(XT, xt) && ctx.stats) atomicAdd(ctx.stats + 1, 1ull);
#pragma unroll
            for (int a = 0; a < N; ++a) xT[a] = xt[a];
            if (filtT_out) {
#pragma unroll
                for (int q = 0; q < Red<N, S>::NCOMP; ++q) filtT_out[q] = comp(XT, q);
            }
        }
        // the thread's composite map x_{k0} = Phi x_{k0+nv} + beta: beta by
        // Horner over the staged g_k, Phi from the table (full threads) or the
        // product of the per-step E_k (the thread that reaches T)
        // backward over the thread's steps: z <- E_k z + g_k from the staged g_k,
        // the result optionally staged in place of g_k
        auto back = [&](S (&z)[N], bool stage) {
            auto one = [&](int i, const S (&E)[NN]) {
                S nz[N];
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    S acc = mine[i * N + a];
#pragma unroll
                    for (int q = 0; q < N; ++q) acc = fma(E[a * N + q], z[q], acc);
                    nz[a] = acc;
                }
#pragma unroll
                for (int a = 0; a < N; ++a) z[a] = nz[a];
                if (stage) stage_state<N, S>(mine + i * N, z);
            };
            if (steady) {
#pragma unroll 1
                for (int i = nv - 1; i >= 0; --i) one(i, c.E);
            } else {
                int i = nv - 1;
#pragma unroll 1
                for (; i >= 1; i -= 2) {
                    S E0[NN], E1[NN];
                    load_stepE_wi<N, S>(tb.wi, gthr, i, K, E0);
                    load_stepE_wi<N, S>(tb.wi, gthr, i - 1, K, E1);
                    one(i, E0);
                    one(i - 1, E1);
                }
                if (i == 0) {
                    S E0[NN];
                    load_stepE_wi<N, S>(tb.wi, gthr, 0, K, E0);
                    one(0, E0);
                }
            }
        };
        Aff<N, S> comp_t;
        set_identity(comp_t);
        back(comp_t.c, false);
        if (nv == K) {
            const S* ph = tb.phi + min(gthr, tb.gc) * NN;
#pragma unroll
            for (int q = 0; q < NN; ++q) comp_t.F[q] = __ldg(ph + q);
        } else {
#pragma unroll 1
            for (int i = 0; i < nv; ++i) {           // Phi <- Phi E_k
                S E[NN], F2[NN];
                load_stepE<N, S>(tb.rows + min(k0 + i, tb.kc) * ST::RS, E);
                ms::mm<N, S>(comp_t.F, E, F2);
#pragma unroll
                for (int q = 0; q < NN; ++q) comp_t.F[q] = F2[q];
            }
        }
        {
            Aff<N, S> H = comp_t;
            block_aff_reduce<N, S>(H, red);       // starts with shuffles, ends with a barrier
            if (t == 0) aos_store(tile_aff, (long)tile, H);
        }
        grid_sync(gs, 2, ctx.stats);

        // ---- phase 3: tile suffix, thread end states, per-step states, bulk store
        S* xe_sh = red + (B / 32) * (Aff<N, S>::NCOMP + N);
        lti_tile_suffix_sum<N, S>(lt, tile_aff, tile, gridDim.x, xT, red, xe_sh);
        S x[N];
        block_aff_end_states<N, S>(comp_t, xe_sh, red, x);
        back(x, true);                               // x_k = E_k x_{k+1} + g_k, in place of g_k
        __syncthreads();
        const int KN = K * N;
        const long base = (long)tile * B * KN;
        const long cnt = min((long)B * KN, T * N - base);
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

}  // namespace mapk
