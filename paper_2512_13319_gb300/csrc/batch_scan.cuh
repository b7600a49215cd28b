// Batched solve of many independent trajectories of one linear time-invariant
// model with the per-step tables of steptab.cuh.
//
// Every trajectory starts from the same prior, so its filter value function
// P at local step k is the tabulated P_k of the model (row min(k, kc)), and
// its solve is the affine recursion of steptab.cuh in v and x alone:
//   v_{k+1} = E_k^T v_k + o_k + G y_{k+1} - Gr,   g_k = E_k (A^-1 C v_k + A^-1 b),
//   x_k = E_k x_{k+1} + g_k,   x_L = P_L^-1 v_L.
// The trajectories are cut into chunks of CH steps (the last chunk of a
// trajectory takes the rest); the linear part of a chunk's filter and RTS maps
// is data-independent and depends only on the chunk's place in its trajectory
// (a table of the chunk maps before kc, one map for the chunks after).  Five
// data-parallel kernels, no barrier inside any of them:
//   A  (thread per chunk)       the chunk's filter offset W from v = 0;
//   B  (thread per trajectory)  the chunk start values, v <- Psi^T v + W in chunk order;
//   C  (thread per chunk)       the forward steps from the start value with g_k
//                               staged in the state rows; the last chunk also
//                               forms x_L and runs its backward steps; the
//                               other chunks their RTS offset beta (from 0);
//   D  (thread per trajectory)  the chunk end states, x <- Phi x + beta backwards;
//   E  (thread per chunk)       the backward steps from the end state.
#pragma once
#include <type_traits>

#include "handle.h"
#include "steptab.cuh"

namespace mapk {

template <int N, int M, typename S>
struct BatchArgs {
    const S* y;                        // (rows, M)
    S* x;                              // (rows + 1, N)
    const BatchTraj* traj;
    const int* chunk_traj;             // trajectory of each chunk
    int ntraj, nchunks;
    S* W;                              // per chunk, N each: filter offset, then start value
    S* V;
    S* Bt;                             // per chunk: RTS offset, then end state
    const S* rows;                     // StepTab rows
    long kc;
    const S* tm;                       // chunk maps (RTS direction) for local chunks < ntm; ntm-1: after kc
    int ntm;
    Red<N, S> prior;
    S AiC[N * N], Aib[N], G[N * M], Gr[N];
    CombineCtx ctx;
};

// The step constants of local step kl: E_kl and o_kl from row min(kl, kc);
// a chunk wholly after kc keeps row kc's in registers (steady)
template <int N, int M, typename S>
struct BatchStep {
    using ST = StepTab<N, S>;
    static constexpr int NN = N * N;
    S Einf[NN], oinf[N];
    __device__ __forceinline__ void init(const BatchArgs<N, M, S>& a)
    {
        const S* r = a.rows + a.kc * ST::RS;
#pragma unroll
        for (int q = 0; q < NN; ++q) Einf[q] = __ldg(r + ST::oE + q);
#pragma unroll
        for (int q = 0; q < N; ++q) oinf[q] = __ldg(r + ST::oO + q);
    }
    template <bool STEADY>
    __device__ __forceinline__ void E_of(const BatchArgs<N, M, S>& a, long kl, S (&E)[NN]) const
    {
        if constexpr (STEADY) {
#pragma unroll
            for (int q = 0; q < NN; ++q) E[q] = Einf[q];
        } else {
            const S* r = a.rows + min(kl, a.kc) * ST::RS + ST::oE;
#pragma unroll
            for (int q = 0; q < NN; ++q) E[q] = __ldg(r + q);
        }
    }
    // v <- E^T v + o + G y - Gr
    template <bool STEADY>
    __device__ __forceinline__ void fstep(const BatchArgs<N, M, S>& a, long kl, const S (&E)[NN], const S* yk,
                                          S (&v)[N]) const
    {
        const S* r = a.rows + min(kl, a.kc) * ST::RS + ST::oO;
        S nv[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S acc = (STEADY ? oinf[i] : __ldg(r + i)) - a.Gr[i];
#pragma unroll
            for (int m = 0; m < M; ++m) acc = fma(a.G[i * M + m], yk[m], acc);
#pragma unroll
            for (int q = 0; q < N; ++q) acc = fma(E[q * N + i], v[q], acc);
            nv[i] = acc;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = nv[i];
    }
};

template <int N, typename S>
__device__ __forceinline__ void load_vec(const S* p, S (&v)[N])
{
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i];
}
template <int N, typename S>
__device__ __forceinline__ void store_vec(S* p, const S (&v)[N])
{
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = v[i];
}

// A: filter offset of each chunk
template <int N, int M, typename S>
__global__ void __launch_bounds__(128) k_batch_a(const __grid_constant__ BatchArgs<N, M, S> a)
{
    using BS = BatchStep<N, M, S>;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.nchunks) return;
    const BatchTraj tr = a.traj[a.chunk_traj[c]];
    const long k0 = (long)(c - tr.c0) * BATCH_CH;
    const int nv = (int)min((long)BATCH_CH, tr.L - k0);
    BS bs;
    bs.init(a);
    S W[N];
#pragma unroll
    for (int i = 0; i < N; ++i) W[i] = S(0);
    auto run = [&](auto steady) {
        constexpr bool ST_ = decltype(steady)::value;
        const S* yc = a.y + (tr.row + k0) * M;
        S y0[M], y1[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            y0[m] = __ldg(yc + m);
            y1[m] = nv > 1 ? __ldg(yc + M + m) : S(0);
        }
#pragma unroll 1
        for (int s = 0; s < nv; ++s) {
            S E[N * N], y2[M];
#pragma unroll
            for (int m = 0; m < M; ++m) y2[m] = s + 2 < nv ? __ldg(yc + (s + 2) * M + m) : S(0);
            bs.template E_of<ST_>(a, k0 + s, E);
            bs.template fstep<ST_>(a, k0 + s, E, y0, W);
#pragma unroll
            for (int m = 0; m < M; ++m) { y0[m] = y1[m]; y1[m] = y2[m]; }
        }
    };
    if (k0 >= a.kc) run(std::true_type{}); else run(std::false_type{});
    store_vec<N, S>(a.W + (long)c * N, W);
}

// B: start value of each chunk (the prior's v at the first)
template <int N, int M, typename S>
__global__ void __launch_bounds__(128) k_batch_b(const __grid_constant__ BatchArgs<N, M, S> a)
{
    constexpr int NN = N * N;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.ntraj) return;
    const BatchTraj tr = a.traj[j];
    S v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = a.prior.v[i];
#pragma unroll 1
    for (int i = 0; i < tr.nc; ++i) {
        const int c = tr.c0 + i;
        store_vec<N, S>(a.V + (long)c * N, v);
        if (i + 1 == tr.nc) break;
        const S* Ph = a.tm + (long)min(i, a.ntm - 1) * NN;      // Psi = Phi^T
        S w[N], nv[N];
        load_vec<N, S>(a.W + (long)c * N, w);
#pragma unroll
        for (int r = 0; r < N; ++r) {
            S acc = w[r];
#pragma unroll
            for (int q = 0; q < N; ++q) acc = fma(__ldg(Ph + q * N + r), v[q], acc);
            nv[r] = acc;
        }
#pragma unroll
        for (int r = 0; r < N; ++r) v[r] = nv[r];
    }
}

// C: forward steps with g_k staged in the state rows; the last chunk of a
// trajectory forms x_L and runs its backward steps, the others their RTS offset
template <int N, int M, typename S>
__global__ void __launch_bounds__(128) k_batch_c(const __grid_constant__ BatchArgs<N, M, S> a)
{
    using BS = BatchStep<N, M, S>;
    using ST = StepTab<N, S>;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.nchunks) return;
    const BatchTraj tr = a.traj[a.chunk_traj[c]];
    const long k0 = (long)(c - tr.c0) * BATCH_CH;
    const int nv = (int)min((long)BATCH_CH, tr.L - k0);
    const bool lastc = c + 1 == tr.c0 + tr.nc;
    BS bs;
    bs.init(a);
    const bool steady = k0 >= a.kc;
    S v[N];
    load_vec<N, S>(a.V + (long)c * N, v);
    S* xr = a.x + (tr.row + k0) * N;
    auto fwd = [&](auto st_) {
        constexpr bool ST_ = decltype(st_)::value;
        const S* yc = a.y + (tr.row + k0) * M;
        S y0[M], y1[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            y0[m] = __ldg(yc + m);
            y1[m] = nv > 1 ? __ldg(yc + M + m) : S(0);
        }
#pragma unroll 1
        for (int s = 0; s < nv; ++s) {
            S E[N * N], y2[M], u[N], g[N];
#pragma unroll
            for (int m = 0; m < M; ++m) y2[m] = s + 2 < nv ? __ldg(yc + (s + 2) * M + m) : S(0);
            bs.template E_of<ST_>(a, k0 + s, E);
#pragma unroll
            for (int i = 0; i < N; ++i) {
                S acc = a.Aib[i];
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(a.AiC[i * N + q], v[q], acc);
                u[i] = acc;
            }
            mat_vec<N, S>(E, u, g);
            store_vec<N, S>(xr + (long)s * N, g);
            bs.template fstep<ST_>(a, k0 + s, E, y0, v);
#pragma unroll
            for (int m = 0; m < M; ++m) { y0[m] = y1[m]; y1[m] = y2[m]; }
        }
    };
    if (steady) fwd(std::true_type{}); else fwd(std::false_type{});
    S z[N];
    if (lastc) {
        // x_L = P_L^-1 v_L
        Red<N, S> X;
#pragma unroll
        for (int i = 0; i < N; ++i) X.v[i] = v[i];
        const S* rP = a.rows + min(tr.L, a.kc) * ST::RS + ST::oP;
#pragma unroll
        for (int q = 0; q < Sym<N>::SZ; ++q) X.P[q] = __ldg(rP + q);
        if (!red_argmin<N, S>(X, z)) report_event(a.ctx.stats, EV_SINGULAR);
        store_vec<N, S>(a.x + (tr.row + tr.L) * N, z);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) z[i] = S(0);
    }
    auto back = [&](auto st_) {
        constexpr bool ST_ = decltype(st_)::value;
        // the staged g of the next two steps are loaded ahead of the recursion
        S g0[N], g1[N];
        load_vec<N, S>(xr + (long)(nv - 1) * N, g0);
        if (nv > 1) load_vec<N, S>(xr + (long)(nv - 2) * N, g1);
#pragma unroll 1
        for (int s = nv - 1; s >= 0; --s) {
            S E[N * N], g2[N], nz[N];
            if (s >= 2) load_vec<N, S>(xr + (long)(s - 2) * N, g2);
            bs.template E_of<ST_>(a, k0 + s, E);
            mat_vec<N, S>(E, z, nz);
#pragma unroll
            for (int i = 0; i < N; ++i) z[i] = nz[i] + g0[i];
            if (lastc) store_vec<N, S>(xr + (long)s * N, z);
#pragma unroll
            for (int i = 0; i < N; ++i) { g0[i] = g1[i]; g1[i] = g2[i]; }
        }
    };
    if (steady) back(std::true_type{}); else back(std::false_type{});
    store_vec<N, S>(a.Bt + (long)c * N, z);           // beta, or the state at the last chunk's start
}

// D: end state of each chunk but the last, x <- Phi x + beta backwards
template <int N, int M, typename S>
__global__ void __launch_bounds__(128) k_batch_d(const __grid_constant__ BatchArgs<N, M, S> a)
{
    constexpr int NN = N * N;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.ntraj) return;
    const BatchTraj tr = a.traj[j];
    S xv[N];
    load_vec<N, S>(a.Bt + (long)(tr.c0 + tr.nc - 1) * N, xv);      // state at the last chunk's start
#pragma unroll 1
    for (int i = tr.nc - 2; i >= 0; --i) {
        const int c = tr.c0 + i;
        S b[N], nx[N];
        load_vec<N, S>(a.Bt + (long)c * N, b);
        store_vec<N, S>(a.Bt + (long)c * N, xv);                    // the chunk's end state
        const S* Ph = a.tm + (long)min(i, a.ntm - 1) * NN;
        mat_vec<N, S>(Ph, xv, nx);
#pragma unroll
        for (int r = 0; r < N; ++r) xv[r] = nx[r] + b[r];
    }
}

// E: backward steps of every chunk but the last from its end state
template <int N, int M, typename S>
__global__ void __launch_bounds__(128) k_batch_e(const __grid_constant__ BatchArgs<N, M, S> a)
{
    using BS = BatchStep<N, M, S>;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.nchunks) return;
    const BatchTraj tr = a.traj[a.chunk_traj[c]];
    if (c + 1 == tr.c0 + tr.nc) return;
    const long k0 = (long)(c - tr.c0) * BATCH_CH;
    BS bs;
    bs.init(a);
    S z[N];
    load_vec<N, S>(a.Bt + (long)c * N, z);
    S* xr = a.x + (tr.row + k0) * N;
    auto back = [&](auto st_) {
        constexpr bool ST_ = decltype(st_)::value;
        // the staged g of the next two steps are loaded ahead of the recursion
        S g0[N], g1[N];
        load_vec<N, S>(xr + (long)(BATCH_CH - 1) * N, g0);
        load_vec<N, S>(xr + (long)(BATCH_CH - 2) * N, g1);
#pragma unroll 1
        for (int s = BATCH_CH - 1; s >= 0; --s) {
            S E[N * N], g2[N], nz[N];
            if (s >= 2) load_vec<N, S>(xr + (long)(s - 2) * N, g2);
            bs.template E_of<ST_>(a, k0 + s, E);
            mat_vec<N, S>(E, z, nz);
#pragma unroll
            for (int i = 0; i < N; ++i) z[i] = nz[i] + g0[i];
            store_vec<N, S>(xr + (long)s * N, z);
#pragma unroll
            for (int i = 0; i < N; ++i) { g0[i] = g1[i]; g1[i] = g2[i]; }
        }
    };
    if (k0 >= a.kc) back(std::true_type{}); else back(std::false_type{});
}

// Chunk maps (RTS direction) for local chunks i < ntm: the closed-loop map of
// the element e^CH at P_{i CH} (the composition of the chunk's per-step maps);
// the last one (i CH >= kc) stands for every later chunk.  One thread each, FP64.
template <int N, typename S>
__global__ void __launch_bounds__(64) k_batch_chunk_maps(const char* __restrict__ tab, long KT, int ntm,
                                                         S* __restrict__ tm)
{
    namespace sd = steptab_detail;
    using ST = StepTab<N, S>;
    constexpr int NN = N * N;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntm) return;
    int lc = 0;
    while ((1 << lc) < BATCH_CH) ++lc;
    const long k = min((long)i * BATCH_CH, (KT - 1) / ST::SMALL * ST::SMALL);
    double P[NN], Ph[NN];
    sd::load_full<N>(reinterpret_cast<const double*>(tab + ST::base_off()) + (k / ST::SMALL) * NN, P);
    sd::fold_map<N>(reinterpret_cast<const double*>(tab + ST::pow_off()) + (long)lc * 3 * NN, P, Ph);
#pragma unroll
    for (int q = 0; q < NN; ++q) tm[(long)i * NN + q] = S(Ph[q]);
}

}  // namespace mapk
