// Persistent solve of a batch of independent trajectories: one launch for
// every model and every trajectory of the batch.
//
// Each trajectory of a linear time-invariant model starts from the model's
// prior, so its filter factor P at local step k is the model's tabulated P_k
// (row min(k, kc) of its step table, Section 4.2 elements and the Eq. 36
// one-variable combine evaluated once per model in FP64), and its solve is
// the affine part of the same combines (batch_persist.h):
//   filter  v_{k+1} = E_k^T v_k + o_k + G y_{k+1} - Gr,
//   RTS     x_k = E_k x_{k+1} + g_k,  g_k = E_k (A^-1 C v_k + A^-1 b),
//   x_L = P_L^-1 v_L (Eq. 18 initial condition; Section 4.3, Eq. 40-42).
//
// A CTA of B threads takes whole trajectories from a work counter, longest
// first, and switches on the model's (nx, ny) to a code path compiled for
// it.  A trajectory is cut into blocks of B * KB steps; thread t owns steps
// t KB .. t KB + KB - 1 of a block.
//   forward sweep, block by block: the block's observations into shared
//     memory (coalesced loads), each thread's filter map v -> Phi_t^T v + W_t
//     over its steps (W_t from v = 0; Phi_t the product of its E_k), the
//     block's inclusive scan of these maps (warp shuffles, then the warps'
//     totals) from the value at the block's start; the threads' start values
//     go to global scratch, the block's end value carries to the next block.
//   x_L = P_L^-1 v_L.
//   backward sweep, last block first: the observations again, each thread's
//     forward steps from its stored start value with the offsets g_k staged
//     in shared memory, its RTS map x -> Phi_t x + beta_t (beta_t from x = 0
//     over the staged g_k), the block's suffix scan of these maps from the
//     state at the block's end, the per-step states in place of the g_k, and
//     one coalesced store of the block's states.
// Threads past the end of a trajectory hold the identity map.  Nothing waits
// on another CTA: the work counter is the only shared state (the last CTA to
// finish resets it for the next launch), so the launch needs no co-residency.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/map_smoother.h"
#include "batch_persist.h"
#include "elements.cuh"

namespace mapk {

template <typename S>
struct BpArgs {
    const BpModel<S>* models;
    const BpItem* items;
    int nitems;
    int KB;                            // steps per thread (even)
    int Nmax, Mmax;                    // largest model dimensions (shared-memory layout)
    S* scr;                            // thread start values of the forward sweep
    unsigned* ctr;                     // [0] next item, [1] CTAs finished
};

namespace bp {

template <int N, typename S>
__device__ __forceinline__ void mvec(const S* A, const S* x, S* y)     // y = A x
{
#pragma unroll
    for (int a = 0; a < N; ++a) {
        S acc = A[a * N] * x[0];
#pragma unroll
        for (int q = 1; q < N; ++q) acc = fma(A[a * N + q], x[q], acc);
        y[a] = acc;
    }
}

template <int N, typename S>
__device__ __forceinline__ void mtvec(const S* A, const S* x, S* y)    // y = A^T x
{
#pragma unroll
    for (int a = 0; a < N; ++a) {
        S acc = A[a] * x[0];
#pragma unroll
        for (int q = 1; q < N; ++q) acc = fma(A[q * N + a], x[q], acc);
        y[a] = acc;
    }
}

template <int N, typename S>
__device__ __forceinline__ void mmul(const S* A, const S* Bm, S* C)   // C = A B
{
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            S acc = A[i * N] * Bm[j];
#pragma unroll
            for (int k = 1; k < N; ++k) acc = fma(A[i * N + k], Bm[k * N + j], acc);
            C[i * N + j] = acc;
        }
}

// A <- A E, one row at a time (row i of A E depends on row i of A only)
template <int N, typename S>
__device__ __forceinline__ void mul_right(S (&A)[N * N], const S (&E)[N * N])
{
#pragma unroll
    for (int i = 0; i < N; ++i) {
        S r[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            S acc = A[i * N] * E[j];
#pragma unroll
            for (int k = 1; k < N; ++k) acc = fma(A[i * N + k], E[k * N + j], acc);
            r[j] = acc;
        }
#pragma unroll
        for (int j = 0; j < N; ++j) A[i * N + j] = r[j];
    }
}

template <int N, typename S>
__device__ __forceinline__ void eye(S (&A)[N * N])
{
#pragma unroll
    for (int q = 0; q < N * N; ++q) A[q] = q % (N + 1) == 0 ? S(1) : S(0);
}

template <int C, typename S>
__device__ __forceinline__ void ld(const S* __restrict__ p, S (&v)[C])
{
#pragma unroll
    for (int q = 0; q < C; ++q) v[q] = __ldg(p + q);
}

// Rows of a block between global memory (cnt scalars, contiguous) and the
// per-thread layout of shared memory: scalar e of the block belongs to thread
// e / run and sits at e + e / run (one padding scalar after each thread's
// run, so that the threads' rows start in different banks).  inv = 1 / run:
// floor((e + 1/2) inv) is e / run exactly for the run lengths used here.
__device__ __forceinline__ int padded(int e, float inv)
{
    return e + (int)(((float)e + 0.5f) * inv);
}

// start bringing the whole 16-byte words of [p, p + bytes) into L2 (a later
// block's observations; nothing waits for it)
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes)
{
    const unsigned long long a = reinterpret_cast<unsigned long long>(p);
    const unsigned long long lo = (a + 15ull) & ~15ull, hi = (a + bytes) & ~15ull;
    if (hi > lo)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

template <typename S, int B>
__device__ __forceinline__ void stage_in(const S* __restrict__ g, int cnt, S* sm, float inv)
{
    constexpr int U = 4;
    int e = threadIdx.x;
    for (; e + (U - 1) * B < cnt; e += U * B) {
        S r[U];
#pragma unroll
        for (int u = 0; u < U; ++u) r[u] = __ldg(g + e + u * B);
#pragma unroll
        for (int u = 0; u < U; ++u) sm[padded(e + u * B, inv)] = r[u];
    }
    for (; e < cnt; e += B) sm[padded(e, inv)] = __ldg(g + e);
}

template <typename S, int B>
__device__ __forceinline__ void stage_out(S* __restrict__ g, int cnt, const S* sm, float inv)
{
    for (int e = threadIdx.x; e < cnt; e += B) g[e] = sm[padded(e, inv)];
}

// Inclusive scan of the threads' filter maps v -> Phi_t^T v + W_t in time
// order from vin, the value at the block's start.  Returns the thread's start
// value in vs and the block's end value in vin.  wsm: B/32 (N^2 + N) scalars,
// bc: N scalars of shared memory.
template <int N, typename S, int B>
__device__ __forceinline__ void scan_fwd(S (&Phi)[N * N], S (&W)[N], S (&vin)[N], S* wsm, S* bc, S (&vs)[N])
{
    constexpr int NN = N * N, NA = NN + N;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    // lanes (l - d, l] composed with (l - 2d, l - d]: v -> (P' Phi)^T v + Phi^T W' + W
    // (P' fetched one row at a time)
#pragma unroll 1
    for (int d = 1; d < 32; d <<= 1) {
        S W2[N], nP[NN];
#pragma unroll
        for (int a = 0; a < N; ++a) W2[a] = __shfl_up_sync(0xffffffffu, W[a], d);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S pr[N];
#pragma unroll
            for (int k = 0; k < N; ++k) pr[k] = __shfl_up_sync(0xffffffffu, Phi[i * N + k], d);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                S acc = pr[0] * Phi[j];
#pragma unroll
                for (int k = 1; k < N; ++k) acc = fma(pr[k], Phi[k * N + j], acc);
                nP[i * N + j] = acc;
            }
        }
        if (lane >= d) {
            S nw[N];
            mtvec<N, S>(Phi, W2, nw);
#pragma unroll
            for (int a = 0; a < N; ++a) W[a] += nw[a];
#pragma unroll
            for (int q = 0; q < NN; ++q) Phi[q] = nP[q];
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int q = 0; q < NN; ++q) wsm[wid * NA + q] = Phi[q];
#pragma unroll
        for (int a = 0; a < N; ++a) wsm[wid * NA + NN + a] = W[a];
    }
    __syncthreads();
    S vc[N];
#pragma unroll
    for (int a = 0; a < N; ++a) vc[a] = vin[a];
    for (int u = 0; u < wid; ++u) {
        S nv[N];
        mtvec<N, S>(wsm + u * NA, vc, nv);
#pragma unroll
        for (int a = 0; a < N; ++a) vc[a] = nv[a] + wsm[u * NA + NN + a];
    }
    S ve[N];
    mtvec<N, S>(Phi, vc, ve);
#pragma unroll
    for (int a = 0; a < N; ++a) {
        ve[a] += W[a];
        const S up = __shfl_up_sync(0xffffffffu, ve[a], 1);
        vs[a] = lane == 0 ? vc[a] : up;
    }
    if (t == B - 1)
#pragma unroll
        for (int a = 0; a < N; ++a) bc[a] = ve[a];
    __syncthreads();
#pragma unroll
    for (int a = 0; a < N; ++a) vin[a] = bc[a];
}

// Suffix scan of the threads' RTS maps x -> Phi_t x + beta_t from xin, the
// state at the block's end.  Returns the state at the end of the thread's
// steps in xe and the state at the block's start in xin.
template <int N, typename S, int B>
__device__ __forceinline__ void scan_bwd(S (&Phi)[N * N], S (&beta)[N], S (&xin)[N], S* wsm, S* bc, S (&xe)[N])
{
    constexpr int NN = N * N, NA = NN + N, NW = B / 32;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    // lanes [l, l + d) composed with [l + d, l + 2d): x -> (Phi P') x + Phi beta' + beta
    // (P' fetched one column at a time)
#pragma unroll 1
    for (int d = 1; d < 32; d <<= 1) {
        S b2[N], nP[NN];
#pragma unroll
        for (int a = 0; a < N; ++a) b2[a] = __shfl_down_sync(0xffffffffu, beta[a], d);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            S pc[N];
#pragma unroll
            for (int k = 0; k < N; ++k) pc[k] = __shfl_down_sync(0xffffffffu, Phi[k * N + j], d);
#pragma unroll
            for (int i = 0; i < N; ++i) {
                S acc = Phi[i * N] * pc[0];
#pragma unroll
                for (int k = 1; k < N; ++k) acc = fma(Phi[i * N + k], pc[k], acc);
                nP[i * N + j] = acc;
            }
        }
        if (lane + d < 32) {
            S nb[N];
            mvec<N, S>(Phi, b2, nb);
#pragma unroll
            for (int a = 0; a < N; ++a) beta[a] += nb[a];
#pragma unroll
            for (int q = 0; q < NN; ++q) Phi[q] = nP[q];
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NN; ++q) wsm[wid * NA + q] = Phi[q];
#pragma unroll
        for (int a = 0; a < N; ++a) wsm[wid * NA + NN + a] = beta[a];
    }
    __syncthreads();
    S xc[N];
#pragma unroll
    for (int a = 0; a < N; ++a) xc[a] = xin[a];
    for (int u = NW - 1; u > wid; --u) {
        S nx[N];
        mvec<N, S>(wsm + u * NA, xc, nx);
#pragma unroll
        for (int a = 0; a < N; ++a) xc[a] = nx[a] + wsm[u * NA + NN + a];
    }
    S xs[N];
    mvec<N, S>(Phi, xc, xs);
#pragma unroll
    for (int a = 0; a < N; ++a) {
        xs[a] += beta[a];
        const S dn = __shfl_down_sync(0xffffffffu, xs[a], 1);
        xe[a] = lane == 31 ? xc[a] : dn;
    }
    if (t == 0)
#pragma unroll
        for (int a = 0; a < N; ++a) bc[a] = xs[a];
    __syncthreads();
#pragma unroll
    for (int a = 0; a < N; ++a) xin[a] = bc[a];
}

// v <- E^T v + o - Gr + G y
template <int N, int M, typename S>
__device__ __forceinline__ void fstep(const S (&E)[N * N], const S (&o)[N], const S (&Gm)[N * M], const S* yk,
                                      S (&v)[N])
{
    S yv[M], nv[N];
#pragma unroll
    for (int m = 0; m < M; ++m) yv[m] = yk[m];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        S acc = o[a];
#pragma unroll
        for (int m = 0; m < M; ++m) acc = fma(Gm[a * M + m], yv[m], acc);
        S ev = E[a] * v[0];
#pragma unroll
        for (int q = 1; q < N; ++q) ev = fma(E[q * N + a], v[q], ev);
        nv[a] = acc + ev;
    }
#pragma unroll
    for (int a = 0; a < N; ++a) v[a] = nv[a];
}

// One trajectory (see the top of the file).
template <int N, int M, typename S, int B>
__device__ void traj(const BpArgs<S>& a, const BpModel<S>* __restrict__ md, const BpItem& it, S* sm)
{
    constexpr int NN = N * N;
    const int t = threadIdx.x;
    const int KB = a.KB;
    const long BS = (long)B * KB, L = it.L;
    const int nb = (int)((L + BS - 1) / BS);
    const S* __restrict__ y = md->y + it.row * M;
    S* __restrict__ x = md->x + it.row * N;
    S* __restrict__ scr = a.scr + it.scr;
    const long kc = md->kc;
    const S* __restrict__ rows = md->rows;
    const int RS = md->RS, oE = md->oE, oO = md->oO;
    const int yrun = KB * M, grun = KB * N;
    const float yinv = 1.0f / (float)yrun, ginv = 1.0f / (float)grun;
    S* ys = sm;
    S* gs = ys + B * (KB * a.Mmax + 1);
    S* wsm = gs + B * (KB * a.Nmax + 1);
    S* bc = wsm + (B / 32) * (a.Nmax * a.Nmax + a.Nmax);
    const S* yt = ys + t * (yrun + 1);                 // this thread's observation rows
    S* gt = gs + t * (grun + 1);                       // its offsets g_k, then states

    // step constants of local step k (rows before kc; row kc after)
    auto row_Eo = [&](long k, S (&E)[NN], S (&o)[N], const S (&gr)[N]) {
        const S* r = rows + min(k, kc) * RS;
        ld<NN, S>(r + oE, E);
#pragma unroll
        for (int q = 0; q < N; ++q) o[q] = __ldg(r + oO + q) - gr[q];
    };

    // ---- forward sweep
    S vin[N];
    ld<N, S>(md->v0, vin);
    for (int b = 0; b < nb; ++b) {
        const long b0 = (long)b * BS;
        const int cnt = (int)min(BS, L - b0);
        __syncthreads();                               // the block before is done with ys
        if (t == 0 && b + 1 < nb)                      // the next block's observations into L2
            prefetch_l2(y + (b0 + BS) * M, sizeof(S) * (size_t)min(BS, L - b0 - BS) * M);
        stage_in<S, B>(y + b0 * M, cnt * M, ys, yinv);
        __syncthreads();
        const long k0 = b0 + (long)t * KB;
        const int nv = max(0, min(KB, cnt - t * KB));
        S Phi[NN], W[N];
#pragma unroll
        for (int q = 0; q < N; ++q) W[q] = S(0);
        {
            S Gm[N * M], gr[N];
            ld<N * M, S>(md->G, Gm);
            ld<N, S>(md->Gr, gr);
            if (k0 >= kc) {
                S E[NN], o[N];
                ld<NN, S>(md->Einf, E);
#pragma unroll
                for (int q = 0; q < N; ++q) o[q] = __ldg(md->oinf + q) - gr[q];
#pragma unroll 1
                for (int i = 0; i < nv; ++i) fstep<N, M, S>(E, o, Gm, yt + i * M, W);
                if (nv == KB) {
                    ld<NN, S>(md->PhiK, Phi);
                } else {
                    eye<N, S>(Phi);
#pragma unroll 1
                    for (int i = 0; i < nv; ++i) mul_right<N, S>(Phi, E);
                }
            } else {
                eye<N, S>(Phi);
#pragma unroll 1
                for (int i = 0; i < nv; ++i) {
                    S E[NN], o[N];
                    row_Eo(k0 + i, E, o, gr);
                    fstep<N, M, S>(E, o, Gm, yt + i * M, W);
                    mul_right<N, S>(Phi, E);
                }
            }
        }
        S vs[N];
        scan_fwd<N, S, B>(Phi, W, vin, wsm, bc, vs);
        S* sp = scr + ((long)b * B + t) * N;
#pragma unroll
        for (int q = 0; q < N; ++q) sp[q] = vs[q];
    }

    // ---- x_L = P_L^-1 v_L
    if (t == 0) {
        Red<N, S> X;
#pragma unroll
        for (int q = 0; q < N; ++q) X.v[q] = vin[q];
        const S* rP = rows + min(L, kc) * RS + md->oP;
#pragma unroll
        for (int q = 0; q < Sym<N>::SZ; ++q) X.P[q] = __ldg(rP + q);
        S z[N];
        if (!red_argmin<N, S>(X, z)) report_event(md->stats, EV_SINGULAR);
#pragma unroll
        for (int q = 0; q < N; ++q) {
            x[L * N + q] = z[q];
            bc[q] = z[q];
        }
    }
    __syncthreads();
    S xin[N];
#pragma unroll
    for (int q = 0; q < N; ++q) xin[q] = bc[q];

    // ---- backward sweep
    for (int b = nb - 1; b >= 0; --b) {
        const long b0 = (long)b * BS;
        const int cnt = (int)min(BS, L - b0);
        __syncthreads();                               // the block after is stored, bc read
        if (t == 0 && b > 0)                           // the previous block's observations into L2
            prefetch_l2(y + (b0 - BS) * M, sizeof(S) * (size_t)BS * M);
        stage_in<S, B>(y + b0 * M, cnt * M, ys, yinv);
        __syncthreads();
        const long k0 = b0 + (long)t * KB;
        const int nv = max(0, min(KB, cnt - t * KB));
        const bool steady = k0 >= kc;
        S v[N];
        {
            const S* sp = scr + ((long)b * B + t) * N;
#pragma unroll
            for (int q = 0; q < N; ++q) v[q] = sp[q];
        }
        S Phi[NN];
        // forward over the thread's steps: g_k staged, v advanced
        {
            S Gm[N * M], gr[N];
            ld<N * M, S>(md->G, Gm);
            ld<N, S>(md->Gr, gr);
            if (steady) {
                S E[NN], o[N], Cm[NN], cb[N];
                ld<NN, S>(md->Einf, E);
#pragma unroll
                for (int q = 0; q < N; ++q) o[q] = __ldg(md->oinf + q) - gr[q];
                ld<NN, S>(md->EAiC, Cm);
                ld<N, S>(md->EAib, cb);
#pragma unroll 1
                for (int i = 0; i < nv; ++i) {
                    S g[N];
                    mvec<N, S>(Cm, v, g);
#pragma unroll
                    for (int q = 0; q < N; ++q) gt[i * N + q] = g[q] + cb[q];
                    fstep<N, M, S>(E, o, Gm, yt + i * M, v);
                }
                if (nv == KB) {
                    ld<NN, S>(md->PhiK, Phi);
                } else {
                    eye<N, S>(Phi);
#pragma unroll 1
                    for (int i = 0; i < nv; ++i) mul_right<N, S>(Phi, E);
                }
            } else {
                eye<N, S>(Phi);
                // steps before kc (A^-1 C and A^-1 b read from the model record, L1-resident)
#pragma unroll 1
                for (int i = 0; i < nv; ++i) {
                    S E[NN], o[N], u[N], g[N];
                    row_Eo(k0 + i, E, o, gr);
#pragma unroll
                    for (int a2 = 0; a2 < N; ++a2) {
                        S acc = __ldg(md->Aib + a2);
#pragma unroll
                        for (int q = 0; q < N; ++q) acc = fma(__ldg(md->AiC + a2 * N + q), v[q], acc);
                        u[a2] = acc;
                    }
                    mvec<N, S>(E, u, g);
#pragma unroll
                    for (int q = 0; q < N; ++q) gt[i * N + q] = g[q];
                    fstep<N, M, S>(E, o, Gm, yt + i * M, v);
                    mul_right<N, S>(Phi, E);
                }
            }
        }
        // backward over the thread's steps: z <- E_k z + g_k (states in place when asked)
        auto back = [&](S (&z)[N], bool store) {
            if (steady) {
                S E[NN];
                ld<NN, S>(md->Einf, E);
#pragma unroll 1
                for (int i = nv - 1; i >= 0; --i) {
                    S nz[N];
                    mvec<N, S>(E, z, nz);
#pragma unroll
                    for (int q = 0; q < N; ++q) z[q] = nz[q] + gt[i * N + q];
                    if (store)
#pragma unroll
                        for (int q = 0; q < N; ++q) gt[i * N + q] = z[q];
                }
            } else {
#pragma unroll 1
                for (int i = nv - 1; i >= 0; --i) {
                    S E[NN], nz[N];
                    ld<NN, S>(rows + min(k0 + i, kc) * RS + oE, E);
                    mvec<N, S>(E, z, nz);
#pragma unroll
                    for (int q = 0; q < N; ++q) z[q] = nz[q] + gt[i * N + q];
                    if (store)
#pragma unroll
                        for (int q = 0; q < N; ++q) gt[i * N + q] = z[q];
                }
            }
        };
        S beta[N];
#pragma unroll
        for (int q = 0; q < N; ++q) beta[q] = S(0);
        back(beta, false);
        S xe[N];
        scan_bwd<N, S, B>(Phi, beta, xin, wsm, bc, xe);
        back(xe, true);
        __syncthreads();
        stage_out<S, B>(x + b0 * N, cnt * N, gs, ginv);
    }
}

}  // namespace bp

// The persistent kernel: CTAs take trajectories from the work counter until
// none is left; the last CTA to finish resets the counter.
template <typename S, int B>
__global__ void __launch_bounds__(B, (sizeof(S) == 4 ? 384 : 256) / B) k_batch_persist(const __grid_constant__ BpArgs<S> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* sm = reinterpret_cast<S*>(smem_raw);
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.ctr, 1u);
        __syncthreads();
        const int i = s_item;
        __syncthreads();
        if (i >= a.nitems) break;
        const BpItem it = a.items[i];
        const BpModel<S>* md = a.models + it.model;
        switch (md->N * 8 + md->M) {
            case 2 * 8 + 1: bp::traj<2, 1, S, B>(a, md, it, sm); break;
            case 3 * 8 + 1: bp::traj<3, 1, S, B>(a, md, it, sm); break;
            case 4 * 8 + 2: bp::traj<4, 2, S, B>(a, md, it, sm); break;
            case 5 * 8 + 2: bp::traj<5, 2, S, B>(a, md, it, sm); break;
            case 6 * 8 + 3: bp::traj<6, 3, S, B>(a, md, it, sm); break;
            default: break;                            // rejected when the batch is created
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.ctr + 1, 1u) == gridDim.x - 1) {
            atomicExch(a.ctr, 0u);
            atomicExch(a.ctr + 1, 0u);
            __threadfence();
        }
    }
}

// ---- host side

bool bp_shape_supported(int N, int M)
{
    return (N == 2 && M == 1) || (N == 3 && M == 1) || (N == 4 && M == 2) || (N == 5 && M == 2) ||
           (N == 6 && M == 3);
}

size_t bp_smem_bytes(int prec, int B, int KB, int Nmax, int Mmax)
{
    const size_t es = prec == MAP_FP64 ? 8 : 4;
    const size_t sc = (size_t)B * (KB * Mmax + 1) + (size_t)B * (KB * Nmax + 1) +
                      (size_t)(B / 32) * (Nmax * Nmax + Nmax) + Nmax;
    return (es * sc + 15) / 16 * 16;
}

namespace {
template <typename S, int B>
void* bp_kernel()
{
    return reinterpret_cast<void*>(&k_batch_persist<S, B>);
}
void* bp_kernel_of(int prec, int B)
{
    if (prec == MAP_FP64) return B == 64 ? bp_kernel<double, 64>() : bp_kernel<double, 128>();
    return B == 64 ? bp_kernel<float, 64>() : bp_kernel<float, 128>();
}
}  // namespace

// CTAs of the kernel per SM with `smem` bytes of dynamic shared memory (0: it does not fit)
int bp_blocks_per_sm(int prec, int B, size_t smem)
{
    const void* k = bp_kernel_of(prec, B);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int dyn_max = optin - (int)fa.sharedSizeBytes;
    if (smem > (size_t)dyn_max) return 0;
    // the largest dynamic size once, so that every candidate geometry launches
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, B, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t bp_launch(int prec, int B, int grid, size_t smem, const void* models, const BpItem* items, int nitems,
                      int KB, int Nmax, int Mmax, void* scr, unsigned* ctr, cudaStream_t st)
{
    if (prec == MAP_FP64) {
        BpArgs<double> a{static_cast<const BpModel<double>*>(models), items, nitems, KB, Nmax, Mmax,
                         static_cast<double*>(scr), ctr};
        if (B == 64) k_batch_persist<double, 64><<<grid, 64, smem, st>>>(a);
        else k_batch_persist<double, 128><<<grid, 128, smem, st>>>(a);
    } else {
        BpArgs<float> a{static_cast<const BpModel<float>*>(models), items, nitems, KB, Nmax, Mmax,
                        static_cast<float*>(scr), ctr};
        if (B == 64) k_batch_persist<float, 64><<<grid, 64, smem, st>>>(a);
        else k_batch_persist<float, 128><<<grid, 128, smem, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace mapk
