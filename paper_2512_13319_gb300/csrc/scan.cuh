// Blocked associative scans (reduce, then down-sweep) for the filter
// (Section 3.3-3.4, Eq. 32) and the RTS pass (Section 3.5 and 4.3, Eq. 40-42).
//
// Work decomposition.  A tile of L = B*K consecutive steps is one CTA of B
// threads; thread t owns steps [k0, k0+K), k0 = (tile*B + t)*K, and builds
// its elements in registers from the per-step inputs.  Within a CTA the
// per-thread partials are scanned with a work-efficient up/down sweep
// (Blelloch) through shared memory.  Across tiles, every CTA of a down-sweep
// reduces the totals of the tiles before it (for the filter) or after it (for
// the RTS pass) itself: at most ceil(tile / B) totals per thread and one
// sub-warp tree, all CTAs at once, instead of a scan of the totals by one CTA
// between the kernels.  There are no inter-CTA waits anywhere: every
// dependency between tiles is a kernel boundary.
//
// Orientation.  Elements are stored in original-time order.  The filter value
// function of x_k, V(., tau_{T-k}) = e_{k-1} (x) ... (x) e_0 (x) a_T, is the
// original-time prefix with the later element on the LEFT of the combine.
// Every prefix that contains the terminal element a_T is a one-variable value
// function (A = C = b = 0), so the down-sweep and the per-step recursion use
// the cheaper `apply`.  The RTS pass composes the closed-loop maps
// x_k = E_k x_{k+1} + g_k from the last step backwards (an original-time
// suffix), starting from x_T = S_T^-1 v_T (Eq. 18 initial condition).
#pragma once
#include <cstdint>

#include "producers.cuh"
#include "coop.cuh"
#include "lti_fold.cuh"
#include "bulk.cuh"

namespace mapk {

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialisation may start while its predecessor on the stream still runs;
// pdl_wait() blocks until the predecessor grid has completed and its writes
// are visible, pdl_trigger() lets the successor grid launch.  Each kernel
// triggers only after its own pdl_wait(), so a kernel never starts before the
// kernel two launches back has completed.  Both are no-ops without the
// launch attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Level d of a tree over B leaves has B >> d nodes stored from lvl_off(B, d);
// all 2B - 1 nodes fit in 2B slots.
__device__ __forceinline__ int lvl_off(int B, int d) { return 2 * B - ((2 * B) >> d); }

__device__ __forceinline__ int ilog2(int B) { return 31 - __clz(B); }

// copy of cnt scalars (a multiple of 16 bytes, both ends 16-byte aligned) by
// all threads of the block, 16 bytes at a time
template <typename S>
__device__ __forceinline__ void block_copy16(S* __restrict__ dst, const S* __restrict__ src, long cnt)
{
    const long n16 = cnt * (long)sizeof(S) / 16;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (long i = threadIdx.x; i < n16; i += blockDim.x) d4[i] = s4[i];
}

// vectorised copy of a contiguous run of CNT scalars (16-byte aligned endpoints)
template <int CNT, typename S>
__device__ __forceinline__ void store_run(S* __restrict__ dst, const S* src)
{
    constexpr int V = 16 / sizeof(S);
    if (CNT % V == 0) {
#pragma unroll
        for (int i = 0; i < CNT; i += V) {
            if (sizeof(S) == 4)
                *reinterpret_cast<float4*>(dst + i) = make_float4(float(src[i]), float(src[i + 1]),
                                                                  float(src[i + 2]), float(src[i + 3]));
            else
                *reinterpret_cast<double2*>(dst + i) = make_double2(double(src[i]), double(src[i + 1]));
        }
    } else {
#pragma unroll
        for (int i = 0; i < CNT; ++i) dst[i] = src[i];
    }
}

template <int CNT, typename S>
__device__ __forceinline__ void load_run_aligned(const S* __restrict__ src, S* dst)
{
    constexpr int V = 16 / sizeof(S);
    if (CNT % V == 0) {
#pragma unroll
        for (int i = 0; i < CNT; i += V) {
            if (sizeof(S) == 4) {
                float4 q = *reinterpret_cast<const float4*>(src + i);
                dst[i] = S(q.x); dst[i + 1] = S(q.y); dst[i + 2] = S(q.z); dst[i + 3] = S(q.w);
            } else {
                double2 q = *reinterpret_cast<const double2*>(src + i);
                dst[i] = S(q.x); dst[i + 1] = S(q.y);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < CNT; ++i) dst[i] = src[i];
    }
}

// AoS (item-major) global <-> register struct
template <class Tp, typename S>
__device__ __forceinline__ void aos_store(S* __restrict__ base, long idx, Tp& x)
{
    S tmp[Tp::NCOMP];
#pragma unroll
    for (int i = 0; i < Tp::NCOMP; ++i) tmp[i] = comp(x, i);
    store_run<Tp::NCOMP, S>(base + idx * Tp::NCOMP, tmp);
}
template <class Tp, typename S>
__device__ __forceinline__ void aos_load(const S* __restrict__ base, long idx, Tp& x)
{
    S tmp[Tp::NCOMP];
    load_run_aligned<Tp::NCOMP, S>(base + idx * Tp::NCOMP, tmp);
#pragma unroll
    for (int i = 0; i < Tp::NCOMP; ++i) comp(x, i) = tmp[i];
}

// warp-interleaved layouts: per-thread items with the 32 lanes of a warp
// adjacent for every component, so that every access is one 128-byte line
__device__ __forceinline__ long wi_idx(long gthr, int c, int NC)
{
    return ((gthr >> 5) * NC + c) * 32 + (gthr & 31);
}
__device__ __forceinline__ long wis_idx(long gthr, int i, int c, int K, int NC)
{
    return (((gthr >> 5) * K + i) * NC + c) * 32 + (gthr & 31);
}
template <class Tp, typename S>
__device__ __forceinline__ void wi_store(S* __restrict__ base, long gthr, Tp& x)
{
#pragma unroll
    for (int c = 0; c < Tp::NCOMP; ++c) base[wi_idx(gthr, c, Tp::NCOMP)] = comp(x, c);
}
template <class Tp, typename S>
__device__ __forceinline__ void wi_load(const S* __restrict__ base, long gthr, Tp& x)
{
#pragma unroll
    for (int c = 0; c < Tp::NCOMP; ++c) comp(x, c) = base[wi_idx(gthr, c, Tp::NCOMP)];
}

// ---------------------------------------------------------------------------
// block-level trees over B = blockDim.x leaves, nodes in shared memory (slot
// i of the tree at nodes + i * NE), evaluated by sub-warp groups (coop.cuh)
// ---------------------------------------------------------------------------
// slot j of level d in a tree whose node slots are NODE scalars apart
template <int NODE, typename S>
__device__ __forceinline__ S* slotn(S* nodes, int B, int d, int j)
{
    return nodes + (long)(lvl_off(B, d) + j) * NODE;
}
// element trees: slots of CoopLayout::NE scalars
template <int N, typename S>
__device__ __forceinline__ S* slot(S* nodes, int B, int d, int j)
{
    return slotn<CoopLayout<N, S>::NE>(nodes, B, d, j);
}

// up-sweep: node(d+1, j) = node(d, 2j+1) (x) node(d, 2j); leaves stored by the caller
template <int N, typename S>
__device__ void coop_elem_up(S* nodes, S* scr_all, const CombineCtx& ctx)
{
    using L = CoopLayout<N, S>;
    const int B = blockDim.x, LB = ilog2(B);
    const int ng = B / L::NL, g = threadIdx.x / L::NL;
    S* scr = scr_all + g * L::NSCR;
    for (int d = 0; d < LB; ++d) {
        __syncthreads();
        const int cnt = B >> (d + 1);
        for (int base = 0; base < cnt; base += ng) {
            const int j = base + g;
            const bool act = j < cnt;
            if (__any_sync(0xffffffffu, act)) {
                const int jj = act ? j : base;
                coop_combine<N, S>(slot<N, S>(nodes, B, d, 2 * jj + 1), slot<N, S>(nodes, B, d, 2 * jj),
                                   slot<N, S>(nodes, B, d + 1, jj), scr, act, ctx);
            }
        }
    }
    __syncthreads();
}

// down-sweep: exclusive prefixes (value nodes, written over the element nodes)
// of all leaves from the prefix `pin` of the block (given by thread 0)
template <int N, typename S>
__device__ void coop_elem_down(S* nodes, S* scr_all, const Red<N, S>& pin, const CombineCtx& ctx,
                               Red<N, S>& out)
{
    using L = CoopLayout<N, S>;
    const int B = blockDim.x, LB = ilog2(B);
    const int NL = L::NL, ng = B / NL, g = threadIdx.x / NL, r = threadIdx.x & (NL - 1);
    S* scr = scr_all + g * L::NSCR;
    if (threadIdx.x == 0) node_store(pin, slot<N, S>(nodes, B, LB, 0));
    for (int d = LB - 1; d >= 0; --d) {
        __syncthreads();
        const int cnt = B >> (d + 1);
        for (int base = 0; base < cnt; base += ng) {
            const int j = base + g;
            const bool act = j < cnt;
            if (__any_sync(0xffffffffu, act)) {
                const int jj = act ? j : base;
                S* par = slot<N, S>(nodes, B, d + 1, jj);
                S* lft = slot<N, S>(nodes, B, d, 2 * jj);
                S* rgt = slot<N, S>(nodes, B, d, 2 * jj + 1);
                coop_apply<N, S>(lft, par, rgt, scr, act, ctx);
                __syncwarp();
                if (act)
                    for (int i = r; i < L::NR; i += NL) lft[i] = par[i];
            }
        }
    }
    __syncthreads();
    node_load(slot<N, S>(nodes, B, 0, threadIdx.x), out);
}

// ---------------------------------------------------------------------------
// ordered compositions of one affine map per thread (leaf t = thread t, leaf 0
// outermost) with warp shuffles: no shared-memory tree levels and only one or
// two block barriers
// ---------------------------------------------------------------------------
// Within a warp (Kogge-Stone): lane l ends with H_l o H_{l+1} o ... o H_31.
template <int N, typename S>
__device__ __forceinline__ void warp_aff_suffix(Aff<N, S>& H)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        Aff<N, S> G;
#pragma unroll
        for (int q = 0; q < N * N; ++q) G.F[q] = __shfl_down_sync(0xffffffffu, H.F[q], d);
#pragma unroll
        for (int q = 0; q < N; ++q) G.c[q] = __shfl_down_sync(0xffffffffu, H.c[q], d);
        if (lane + d < 32) compose<N, S>(H, G, H);
    }
}

// H_0 o H_1 o ... o H_{B-1}, returned in thread 0 (H is overwritten in the
// other threads).  red: B / 32 Aff records of shared memory.  Ends with a barrier.
template <int N, typename S>
__device__ __forceinline__ void block_aff_reduce(Aff<N, S>& H, S* red)
{
    constexpr int NA = Aff<N, S>::NCOMP;
    const int t = threadIdx.x, nw = blockDim.x >> 5;
    warp_aff_suffix<N, S>(H);
    if ((t & 31) == 0)
        for (int c = 0; c < NA; ++c) red[(t >> 5) * NA + c] = comp(H, c);
    __syncthreads();
    if (t == 0) {
        for (int w = 1; w < nw; ++w) {
            Aff<N, S> g;
            for (int c = 0; c < NA; ++c) comp(g, c) = red[w * NA + c];
            compose<N, S>(H, g, H);
        }
    }
    __syncthreads();
}

// The state at the END of every thread's steps, x_t = (H_{t+1} o ... o H_{B-1})(xe),
// from the state xe at the end of the block (read by thread 0 from xe_in).
// red: B / 32 Aff records followed by B / 32 states of shared memory.
// Ends with a barrier.
template <int N, typename S>
__device__ __forceinline__ void block_aff_end_states(const Aff<N, S>& H, const S* xe_in, S* red, S* x)
{
    constexpr int NA = Aff<N, S>::NCOMP;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
    S* ys = red + nw * NA;
    Aff<N, S> Sf = H;
    warp_aff_suffix<N, S>(Sf);             // lane l: H_l o ... o H_31 of its warp
    if (lane == 0)
        for (int c = 0; c < NA; ++c) red[w * NA + c] = comp(Sf, c);
    __syncthreads();
    if (t == 0) {                          // y_w: the state at the end of warp w
        S y[N];
#pragma unroll
        for (int i = 0; i < N; ++i) y[i] = xe_in[i];
        for (int ww = nw - 1; ww >= 0; --ww) {
#pragma unroll
            for (int i = 0; i < N; ++i) ys[ww * N + i] = y[i];
            if (ww == 0) break;
            Aff<N, S> g;
            for (int c = 0; c < NA; ++c) comp(g, c) = red[ww * NA + c];
            S z[N];
            affine_apply<N, S>(g, y, z);
#pragma unroll
            for (int i = 0; i < N; ++i) y[i] = z[i];
        }
    }
    __syncthreads();
    Aff<N, S> nx;                          // H_{l+1} o ... o H_31
#pragma unroll
    for (int q = 0; q < N * N; ++q) nx.F[q] = __shfl_down_sync(0xffffffffu, Sf.F[q], 1);
#pragma unroll
    for (int q = 0; q < N; ++q) nx.c[q] = __shfl_down_sync(0xffffffffu, Sf.c[q], 1);
    S y[N];
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] = ys[w * N + i];
    if (lane < 31)
        affine_apply<N, S>(nx, y, x);
    else
#pragma unroll
        for (int i = 0; i < N; ++i) x[i] = y[i];
    __syncthreads();
}


// shared memory of the element trees: 2B node slots + one scratch area per group
template <int N, typename S>
__host__ __device__ constexpr size_t tree_smem(int B)
{
    return sizeof(S) * ((size_t)2 * B * CoopLayout<N, S>::NE +
                        (size_t)(B / CoopLayout<N, S>::NL) * CoopLayout<N, S>::NSCR);
}
// shared memory of the affine trees: 2B node slots
template <int N, typename S>
__host__ __device__ constexpr size_t aff_tree_smem(int B)
{
    return sizeof(S) * (size_t)2 * B * CoopLayout<N, S>::NA;
}

template <int N, typename S>
__device__ __forceinline__ S* scratch_of(S* nodes)
{
    return nodes + (long)2 * blockDim.x * CoopLayout<N, S>::NE;
}

// ---------------------------------------------------------------------------
// tile prefixes and suffixes, computed by each CTA of a down-sweep
// ---------------------------------------------------------------------------
// Fold, in thread 0, of the totals first..last-1 (later on the left of the
// combine): thread t folds a contiguous run of at most ceil(count / B), the runs
// are reduced with the sub-warp tree (empty runs are the identity element,
// neutral on both sides of the combine).  Uses the element-tree area of
// `nodes`; ends with a barrier.
template <int N, typename S>
__device__ __forceinline__ void fold_totals(const S* __restrict__ totals, int first_all, int last_all, S* nodes,
                                            const CombineCtx& ctx, Elem<N, S>& out)
{
    const int B = blockDim.x, t = threadIdx.x;
    const int cnt = last_all - first_all;
    const int per = (cnt + B - 1) / B;
    const int first = first_all + min(cnt, t * per), last = min(last_all, first + per);
    Elem<N, S> F;
    if (first < last) {
        aos_load(totals, first, F);
        for (int i = first + 1; i < last; ++i) {
            Elem<N, S> g;
            aos_load(totals, i, g);
            combine<N, S>(g, F, F, ctx);
        }
    } else {
        set_identity(F);
    }
    node_store(F, slot<N, S>(nodes, B, 0, t));
    coop_elem_up<N, S>(nodes, scratch_of<N, S>(nodes), ctx);
    if (t == 0) node_load(slot<N, S>(nodes, B, ilog2(B), 0), out);
    __syncthreads();
}

// Tiles per group of the two-level prefix: groups of 4B tiles are reduced by
// k_group_totals when a scan has more than one group.
__host__ __device__ constexpr int prefix_group_tiles(int B) { return 4 * B; }

// Value function before tile `tile` (returned in thread 0): the fold of the
// totals of tiles 0..tile-1 applied to the prior.  With group totals
// (group_agg != nullptr) the fold is that of the groups before the tile's group
// followed by the tiles of its group before it, so that no thread folds more
// than ceil(groups / B) or 4 totals.
template <int N, typename S>
__device__ __forceinline__ void tile_prefix_of(const S* __restrict__ tile_agg, int tile, const Red<N, S>& prior,
                                               S* nodes, const CombineCtx& ctx, Red<N, S>& out,
                                               const S* __restrict__ group_agg = nullptr)
{
    const int t = threadIdx.x;
    if (tile == 0) {
        out = prior;
        return;
    }
    Elem<N, S> tot;
    if (!group_agg) {
        fold_totals<N, S>(tile_agg, 0, tile, nodes, ctx, tot);
    } else {
        const int G = prefix_group_tiles(blockDim.x), g = tile / G;
        Elem<N, S> ga, tb;
        if (g > 0) fold_totals<N, S>(group_agg, 0, g, nodes, ctx, ga);
        fold_totals<N, S>(tile_agg, g * G, tile, nodes, ctx, tb);
        if (t == 0) {
            if (g > 0)
                combine<N, S>(tb, ga, tot, ctx);
            else
                tot = tb;
        }
    }
    if (t == 0) {
        Red<N, S> P = prior;
        apply<N, S, false>(tot, P, nullptr, nullptr, ctx);
        out = P;
    }
}

// Totals of the groups of prefix_group_tiles(B) consecutive tiles (one CTA per
// group), for the two-level tile prefix of scans with many tiles
template <int N, typename S>
__global__ void __launch_bounds__(128)
k_group_totals(const S* __restrict__ tile_agg, int nt, S* __restrict__ group_agg, CombineCtx ctx)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* nodes = reinterpret_cast<S*>(smem_raw);
    pdl_wait();                            // tile totals of the reduce kernel
    pdl_trigger();
    const int G = prefix_group_tiles(blockDim.x), g = blockIdx.x;
    Elem<N, S> tot;
    fold_totals<N, S>(tile_agg, g * G, min(nt, (g + 1) * G), nodes, ctx, tot);
    if (threadIdx.x == 0) aos_store(group_agg, (long)g, tot);
}

// Linear-fold mode (lti_fold.cuh, item (4)): fold, in thread 0, of the affine
// tile maps m_i(v) = F_i v + w_i for i = first_all..last_all-1, the later map
// outermost.  Map i has F_i at F + i * fs and w_i at w + i * ws.  Thread t
// composes the t-th run of at most ceil(count / B) maps counted from the end;
// the runs are composed in thread order (block_aff_reduce, leaf 0 outermost).
// Uses the start of `nodes`; ends with a barrier.
template <int N, typename S>
__device__ __forceinline__ void fold_tile_maps(const S* __restrict__ F, int fs, const S* w, int ws,
                                               int first_all, int last_all, S* nodes, Aff<N, S>& out)
{
    const int B = blockDim.x, t = threadIdx.x;
    const int cnt = last_all - first_all, per = (cnt + B - 1) / B;
    const int hi = last_all - min(cnt, t * per), lo = max(first_all, hi - per);
    Aff<N, S> H;
    set_identity(H);
    for (int i = lo; i < hi; ++i) {          // H = m_i o H
        Aff<N, S> m;
#pragma unroll
        for (int q = 0; q < N * N; ++q) m.F[q] = __ldg(F + (long)i * fs + q);
#pragma unroll
        for (int q = 0; q < N; ++q) m.c[q] = w[(long)i * ws + q];   // written by other CTAs: no __ldg
        compose<N, S>(m, H, H);
    }
    block_aff_reduce<N, S>(H, nodes);
    if (t == 0) out = H;
}

// Linear-fold mode: value function before tile `tile` (returned in thread 0):
// P_tile from the tile tables, v_tile = (m_{tile-1} o ... o m_0)(v_0).  With
// group maps the fold is that of the groups before the tile's group followed
// by the maps of its group before it.
template <int N, typename S>
__device__ __forceinline__ void lti_tile_prefix(const LtiTiles<S>& lt, int tile, const Red<N, S>& prior, S* nodes,
                                                Red<N, S>& out)
{
    constexpr int NN = N * N, NA = Aff<N, S>::NCOMP;
    if (tile == 0) {
        out = prior;
        return;
    }
    Aff<N, S> H;
    if (!lt.gmaps) {
        fold_tile_maps<N, S>(lt.F, NN, lt.w, N, 0, tile, nodes, H);
    } else {
        const int G = prefix_group_tiles(blockDim.x), g = tile / G;
        Aff<N, S> hg, ht;
        if (g > 0) fold_tile_maps<N, S>(lt.gmaps, NA, lt.gmaps + NN, NA, 0, g, nodes, hg);
        fold_tile_maps<N, S>(lt.F, NN, lt.w, N, g * G, tile, nodes, ht);
        if (threadIdx.x == 0) {
            if (g > 0)
                compose<N, S>(ht, hg, H);
            else
                H = ht;
        }
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < Sym<N>::SZ; ++q) out.P[q] = lt.P[(long)tile * Sym<N>::SZ + q];
        affine_apply<N, S>(H, prior.v, out.v);
    }
}

// Sum over the CTA of one N-vector per thread, returned in thread 0.  red:
// B / 32 * N scalars of shared memory; ends with a barrier.
template <int N, typename S>
__device__ __forceinline__ void block_vec_sum(S* v, S* red)
{
    const int t = threadIdx.x, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] += __shfl_down_sync(0xffffffffu, v[i], d);
    if ((t & 31) == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) red[(t >> 5) * N + i] = v[i];
    __syncthreads();
    if (t == 0)
        for (int w = 1; w < nw; ++w)
#pragma unroll
            for (int i = 0; i < N; ++i) v[i] += red[w * N + i];
    __syncthreads();
}

// Linear-fold mode with the product table (item (5) of lti_fold.cuh): value
// function before tile `tile` (returned in thread 0), v_tile as a sum of
// independent terms.  red: B / 32 * N scalars of shared memory.
template <int N, typename S>
__device__ __forceinline__ void lti_tile_prefix_sum(const LtiTiles<S>& lt, int tile, int nt, const Red<N, S>& prior,
                                                    S* red, Red<N, S>& out)
{
    using TT = TileTables<N, 1, S>;                     // pi_index does not depend on M
    constexpr int NN = N * N;
    const int t = threadIdx.x;
    if (tile == 0) {
        out = prior;
        return;
    }
    S v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = S(0);
    // terms i = t - 1 + u B (i = -1: Pi(0, tile)^T v_0, else Pi(i+1, tile)^T w_i); at
    // most 5 per thread (tile <= 4B + 1): all their operands are loaded first
    // (16-byte loads of the table rows), then multiplied
    constexpr int UMAX = 5;
    if constexpr (N <= 6) {
        S Qm[UMAX][NN], wv[UMAX][N];
#pragma unroll
        for (int u = 0; u < UMAX; ++u) {
            const int i = t - 1 + u * (int)blockDim.x;
            const bool on = i < tile;
            const S* Q = lt.qt + TT::qt_index(tile, on ? i + 1 : 0) * NN;   // Pi(i+1, tile)^T
            load_run_aligned<NN, S>(Q, Qm[u]);
#pragma unroll
            for (int c = 0; c < N; ++c) wv[u][c] = !on ? S(0) : i < 0 ? prior.v[c] : lt.w[(long)i * N + c];
        }
#pragma unroll
        for (int u = 0; u < UMAX; ++u)
#pragma unroll
            for (int r = 0; r < N; ++r)
#pragma unroll
                for (int c = 0; c < N; ++c) v[r] = fma(Qm[u][r * N + c], wv[u][c], v[r]);
    } else {
        // larger matrices: one term at a time (registers)
#pragma unroll 1
        for (int u = 0; u < UMAX; ++u) {
            const int i = t - 1 + u * (int)blockDim.x;
            if (i >= tile) break;
            S Qm[NN], wv[N];
            load_run_aligned<NN, S>(lt.qt + TT::qt_index(tile, i + 1) * NN, Qm);
#pragma unroll
            for (int c = 0; c < N; ++c) wv[c] = i < 0 ? prior.v[c] : lt.w[(long)i * N + c];
#pragma unroll
            for (int r = 0; r < N; ++r)
#pragma unroll
                for (int c = 0; c < N; ++c) v[r] = fma(Qm[r * N + c], wv[c], v[r]);
        }
    }
    block_vec_sum<N, S>(v, red);
    if (t == 0) {
#pragma unroll
        for (int q = 0; q < Sym<N>::SZ; ++q) out.P[q] = lt.P[(long)tile * Sym<N>::SZ + q];
#pragma unroll
        for (int i = 0; i < N; ++i) out.v[i] = v[i];
    }
}

// Linear-fold mode with the product table: state at the end of tile `tile`
// (thread 0 writes it to xe), x_T for the last tile, else
// Pi(tile+1, nt-1) x_L + sum_{i=tile+1}^{nt-2} Pi(tile+1, i) beta_i with
// x_L = (last tile's map)(x_T) and beta_i the offset of tile i's map in
// tile_aff.  red: B / 32 * N scalars; ends with a barrier.
template <int N, typename S>
__device__ __forceinline__ void lti_tile_suffix_sum(const LtiTiles<S>& lt, const S* tile_aff, int tile, int nt,
                                                    const S* xT, S* red, S* xe)
{
    using TT = TileTables<N, 1, S>;
    constexpr int NN = N * N, NA = Aff<N, S>::NCOMP;
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
    // terms i = tile + 1 + t + u B (at most 5 per thread: nt <= 4B + 1): all
    // operands loaded first, then multiplied; i = nt - 1 is x_L
    constexpr int UMAX = 5;
    auto term = [&](int i, S (&u)[N]) {
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
    };
    if constexpr (N <= 6) {
        S Pm[UMAX][NN], uv[UMAX][N];
#pragma unroll
        for (int uu = 0; uu < UMAX; ++uu) {
            const int i = tile + 1 + t + uu * (int)blockDim.x;
            const bool on = i < nt;
            load_run_aligned<NN, S>(lt.pi + TT::pi_index(nt, tile + 1, on ? i : tile + 1) * NN, Pm[uu]);
            if (on) {
                term(i, uv[uu]);
            } else {
#pragma unroll
                for (int c = 0; c < N; ++c) uv[uu][c] = S(0);
            }
        }
#pragma unroll
        for (int uu = 0; uu < UMAX; ++uu)
#pragma unroll
            for (int r = 0; r < N; ++r)
#pragma unroll
                for (int c = 0; c < N; ++c) v[r] = fma(Pm[uu][r * N + c], uv[uu][c], v[r]);
    } else {
        // larger matrices: one term at a time (registers)
#pragma unroll 1
        for (int uu = 0; uu < UMAX; ++uu) {
            const int i = tile + 1 + t + uu * (int)blockDim.x;
            if (i >= nt) break;
            S Pm[NN], u[N];
            load_run_aligned<NN, S>(lt.pi + TT::pi_index(nt, tile + 1, i) * NN, Pm);
            term(i, u);
#pragma unroll
            for (int r = 0; r < N; ++r)
#pragma unroll
                for (int c = 0; c < N; ++c) v[r] = fma(Pm[r * N + c], u[c], v[r]);
        }
    }
    block_vec_sum<N, S>(v, red);
    if (t == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) xe[i] = v[i];
    __syncthreads();
}

// Linear-fold mode: composed maps of the groups of prefix_group_tiles(B) full
// tiles (one CTA per group), for scans with many tiles
template <int N, typename S>
__global__ void __launch_bounds__(128)
k_lti_group_maps(const LtiTiles<S> lt, int nfull)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* nodes = reinterpret_cast<S*>(smem_raw);
    pdl_wait();                            // w_j of the reduce kernel
    pdl_trigger();
    const int G = prefix_group_tiles(blockDim.x), g = blockIdx.x;
    Aff<N, S> H;
    fold_tile_maps<N, S>(lt.F, N * N, lt.w, N, g * G, min(nfull, (g + 1) * G), nodes, H);
    if (threadIdx.x == 0) aos_store(lt.gmaps, (long)g, H);
}

// State at the end of tile `tile`, written by thread 0 to the N scalars at
// `xe` (shared memory outside the affine-tree area): the closed-loop maps of
// tiles tile+1..nt-1 composed (thread runs, then the affine tree; a map takes
// the state at the end of its steps to the state at their start) and applied
// to x_T.  Uses the start of `nodes` (block_aff_reduce); ends with a barrier.
template <int N, typename S>
__device__ __forceinline__ void tile_suffix_state(const S* __restrict__ tile_aff, int tile, int nt,
                                                  const S* __restrict__ xT, S* nodes, S* xe)
{
    const int B = blockDim.x, t = threadIdx.x;
    const int cnt = nt - 1 - tile;
    if (cnt == 0) {
        if (t == 0)
            for (int i = 0; i < N; ++i) xe[i] = xT[i];
        __syncthreads();
        return;
    }
    const int per = (cnt + B - 1) / B;
    const int first = tile + 1 + min(cnt, t * per), last = min(nt, first + per);
    Aff<N, S> H;
    set_identity(H);
    for (int i = last - 1; i >= first; --i) {      // H = a_first o ... o a_last
        Aff<N, S> a;                               // written by other CTAs: no __ldg
        aos_load(tile_aff, i, a);
        compose<N, S>(a, H, H);
    }
    block_aff_reduce<N, S>(H, nodes);
    if (t == 0) {
        S x[N], y[N];
#pragma unroll
        for (int i = 0; i < N; ++i) x[i] = xT[i];
        affine_apply<N, S>(H, x, y);
#pragma unroll
        for (int i = 0; i < N; ++i) xe[i] = y[i];
    }
    __syncthreads();
}

// prior of a scan: the model's (v0, S0), or the terminal value function that a
// reversed scan's reduce kernel wrote to prior_dev
template <int N, typename S>
__device__ __forceinline__ Red<N, S> scan_prior(const Red<N, S>& prior, const S* __restrict__ prior_dev)
{
    Red<N, S> p = prior;
    if (prior_dev) aos_load(prior_dev, 0, p);
    return p;
}

// Tile of a down-sweep CTA: block 0 takes the last tile, block b > 0 tile
// b - 1.  The last tile's CTA (in linear-fold mode the one with the extra
// work before its wait) is then dispatched first and overlaps that work with
// the previous kernel.
__device__ __forceinline__ int down_tile() { return blockIdx.x == 0 ? gridDim.x - 1 : blockIdx.x - 1; }

// Exclusive prefix (value function before the thread's first step) of every
// thread of a tile from the tile's prefix `pin` (valid in thread 0): the
// tile's up-sweep over the per-thread aggregates and the down-sweep.
// With linear-fold constants (lt.fold != nullptr, lti_fold.cuh; the level
// constants and co table staged by lti_stage_tables) the tree runs on
// (b, eta) parts only: the leaves are the per-thread (b, eta) aggregates (2N
// components) that the reduce kernel left in thr_agg, or with use_leaf `leaf`
// (the last tile, see lti_last_tile_leaf), and every thread ends with one
// one-variable combine of its prefix with pin.
template <int N, typename S, class Prod>
__device__ __forceinline__ void tile_thread_prefix(const Prod& prod, int tile, int K, const S* __restrict__ thr_agg,
                                                   const Red<N, S>& pin, const LtiTiles<S>& lt,
                                                   bool use_leaf, const S (&leaf)[2 * N], S* nodes,
                                                   const CombineCtx& ctx, Red<N, S>& X,
                                                   const S* __restrict__ tree = nullptr)
{
    const int B = blockDim.x, t = threadIdx.x;
    const long gthr = (long)tile * B + t;
    if constexpr (Prod::LINEAR_FOLD && N <= 6) {
        if (lt.fold) {
            constexpr int M = Prod::W;
            using FL = FoldLayout<N, M, S>;
            using DS = LtiDownSmem<N, M, S>;
            S* bq = nodes + DS::bq(B);
            S* ps = nodes + DS::pin(B);
#pragma unroll
            for (int c = 0; c < 2 * N; ++c) bq[c * B + t] = use_leaf ? leaf[c] : thr_agg[wi_idx(gthr, c, 2 * N)];
            if (t == 0) node_store(pin, ps);
            lti_tree_up<N, M, S>(bq, nodes + DS::lv(B, K));
            lti_tree_down_linear<N, M, S>(bq, lt.co_smem ? nodes + DS::co(B, K) : lt.fold + FL::oCo);
            Red<N, S> P;
            node_load(ps, P);
            S dl[2 * N];
#pragma unroll
            for (int c = 0; c < 2 * N; ++c) dl[c] = bq[c * B + t];
            if (gthr * K < prod.T)
                lti_thread_value<N, M, S>(lt.fold, dl, P, ctx, X);
            else
                X = P;                          // no steps: the value is not used
            return;
        }
    }
    if (tree) {
        // the up-sweep tree that the reduce kernel built from the same leaves
        __syncthreads();                   // the tile prefix is done with the nodes
        block_copy16<S>(nodes, tree, (long)2 * B * CoopLayout<N, S>::NE);
        __syncthreads();
    } else {
        Elem<N, S> G;
        wi_load(thr_agg, gthr, G);
        node_store(G, slot<N, S>(nodes, B, 0, t));
        coop_elem_up<N, S>(nodes, scratch_of<N, S>(nodes), ctx);
    }
    coop_elem_down<N, S>(nodes, scratch_of<N, S>(nodes), pin, ctx, X);
}

// Linear-fold mode, last tile (which the reduce kernel does not cover), before
// the wait for the reduce kernel: the thread's leaf (b, eta) in registers.  A
// thread whose K steps are all before T takes the K-step linear fold; the
// others take zero, which only the prefixes of threads after them see (the
// thread that reaches T and those past it fold or skip their steps one by
// one).  Stages the Gamma_i in `nodes` (K * 2 N M scalars); ends with a barrier.
template <int N, typename S, class Prod>
__device__ __forceinline__ void lti_last_tile_leaf(const Prod& prod, int tile, int K, const S* __restrict__ fold,
                                                   S* nodes, S (&leaf)[2 * N])
{
    if constexpr (Prod::LINEAR_FOLD && N <= 6) {
        using FL = FoldLayout<N, Prod::W, S>;
        const int B = blockDim.x, t = threadIdx.x;
        const long k0 = ((long)tile * B + t) * K;
        for (int q = t; q < K * FL::GS; q += B) nodes[q] = fold[FL::oG + q];
        __syncthreads();
        if (k0 + K <= prod.T) {
            lti_linear_fold<N, S>(prod, fold, nodes, K, k0, leaf);
        } else {
#pragma unroll
            for (int c = 0; c < 2 * N; ++c) leaf[c] = S(0);
        }
        __syncthreads();
    }
}

// The thread of the last tile that holds step T-1 writes the value function
// at x_T (after its steps), its minimiser x_T and, if asked, its filter value.
template <int N, typename S>
__device__ __forceinline__ void write_final_if_last(long T, int tile, int K, const Red<N, S>& X, S* final_out,
                                                    S* xT_out, S* filtT_out, const CombineCtx& ctx)
{
    const long k0 = ((long)tile * blockDim.x + threadIdx.x) * K;
    if (!final_out || tile + 1 != (int)gridDim.x || k0 >= T || k0 + K < T) return;
    Red<N, S> P = X;
    aos_store(final_out, 0, P);
    S x[N];
    if (!red_argmin<N, S>(P, x)) report_event(ctx.stats, EV_SINGULAR);
#pragma unroll
    for (int i = 0; i < N; ++i) xT_out[i] = x[i];
    if (filtT_out) {
#pragma unroll
        for (int i = 0; i < Red<N, S>::NCOMP; ++i) filtT_out[i] = comp(P, i);
    }
}

// shared memory of k_filter_reduce_lti (offsets in scalars of S): the tile's
// inputs staged by one bulk copy, the Gamma_i, the tree level constants, the
// (b, eta) nodes, then the mbarrier of the copy
template <int N, int M, typename S>
struct LtiReduceSmem {
    __host__ __device__ static constexpr int al(int x) { return (x + 3) / 4 * 4; }
    __host__ __device__ static constexpr int gam(int B, int K) { return al(B * K * M); }
    __host__ __device__ static constexpr int lv(int B, int K) { return gam(B, K) + al(K * 2 * N * M); }
    __host__ __device__ static constexpr int bq(int B, int K, int LB)
    {
        return lv(B, K) + (LB + 1) * FoldLayout<N, M, S>::LS;
    }
    __host__ __device__ static constexpr int bar(int B, int K, int LB) { return bq(B, K, LB) + al(2 * B * 2 * N); }
    __host__ __device__ static constexpr size_t bytes(int B, int K, int LB)
    {
        return sizeof(S) * (size_t)bar(B, K, LB) + 16;
    }
};

// ---------------------------------------------------------------------------
// phase 1, linear time-invariant model: per-thread folds and tile totals of
// the full tiles 0 .. gridDim.x - 1 (every step before T), on the (b, eta)
// parts only (lti_fold.cuh).  The tile's inputs arrive in shared memory by one
// bulk copy; per thread K steps cost 2 N M multiply-adds and the tree 4 N^2
// per node.  The per-thread (b, eta) go to thr_agg (2N components,
// warp-interleaved); the tile's total enters only through its affine tile map,
// whose w_j goes to lt.w (item (4) of lti_fold.cuh).  A bulk copy that does not
// complete within the poll limit is counted in ctx.stats[2] and the tile is
// left unwritten.
// ---------------------------------------------------------------------------
template <int N, typename S, class Prod>
__global__ void __launch_bounds__(128, 3)
k_filter_reduce_lti(const __grid_constant__ Prod prod, int K, S* __restrict__ thr_agg, const LtiTiles<S> lt,
                    CombineCtx ctx)
{
    const S* __restrict__ fold = lt.fold;
    constexpr int M = Prod::W;
    using FL = FoldLayout<N, M, S>;
    using RS = LtiReduceSmem<N, M, S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* sm = reinterpret_cast<S*>(smem_raw);
    const int B = blockDim.x, t = threadIdx.x, LB = ilog2(B);
    const long gthr = (long)blockIdx.x * B + t;
    S* ys = sm;
    S* gam = sm + RS::gam(B, K);
    S* lv = sm + RS::lv(B, K);
    S* bq = sm + RS::bq(B, K, LB);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + RS::bar(B, K, LB));
    const unsigned bytes = (unsigned)(sizeof(S) * (size_t)B * K * M);
    pdl_wait();
    pdl_trigger();
    if (t == 0) mbar_init(bar, 1);
    __syncthreads();
    if (t == 0) {
        mbar_arrive_expect_tx(bar, bytes);
        bulk_copy_g2s(ys, prod.y + (long)blockIdx.x * B * K * M, bytes, bar);
    }
    for (int q = t; q < K * FL::GS; q += B) gam[q] = fold[FL::oG + q];
    for (int q = t; q < (LB + 1) * FL::LS; q += B) lv[q] = fold[FL::oL + q];
    bool ok = mbar_wait_bounded(bar, 0, MBAR_POLLS);
    if (!__syncthreads_and(ok)) {
        if (t == 0) report_event(ctx.stats, EV_TIMEOUT);
        mbar_wait_bounded(bar, 0, MBAR_POLLS);      // the copy may still be in flight
        return;
    }
    // (b, eta) of this thread's K steps: offsets + sum_i Gamma_i y_{k0+i}
    S v[2 * N];
#pragma unroll
    for (int q = 0; q < N; ++q) { v[q] = __ldg(fold + FL::ob + q); v[N + q] = __ldg(fold + FL::oe + q); }
    const S* yt = ys + t * K * M;
#pragma unroll 2
    for (int i = 0; i < K; ++i) {
        S row[M];
#pragma unroll
        for (int c = 0; c < M; ++c) row[c] = yt[i * M + c];
        const S* gi = gam + i * FL::GS;
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int c = 0; c < M; ++c) {
                v[a] = fma(gi[a * M + c], row[c], v[a]);
                v[N + a] = fma(gi[(N + a) * M + c], row[c], v[N + a]);
            }
    }
#pragma unroll
    for (int c = 0; c < 2 * N; ++c) {
        thr_agg[wi_idx(gthr, c, 2 * N)] = v[c];
        bq[c * B + t] = v[c];
    }
    lti_tree_up<N, M, S>(bq, lv);
    if (t == 0) {
        // w_j = eta_j - F_j P_j b_j (item (4) of lti_fold.cuh), F_j = E_j^T
        const S* rq = bq + (2 * B - 2) * 2 * N;
        const long j = blockIdx.x;
        S Pb[N];
#pragma unroll
        for (int a = 0; a < N; ++a) {
            S acc = S(0);
#pragma unroll
            for (int c = 0; c < N; ++c) acc = fma(lt.P[j * Sym<N>::SZ + Sym<N>::at(a, c)], rq[c], acc);
            Pb[a] = acc;
        }
#pragma unroll
        for (int a = 0; a < N; ++a) {
            S acc = rq[N + a];
#pragma unroll
            for (int c = 0; c < N; ++c) acc = fma(-lt.F[j * N * N + a * N + c], Pb[c], acc);
            lt.w[j * N + a] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// phase 1: per-thread fold and per-tile total of the filter elements
// ---------------------------------------------------------------------------
template <int N, typename S, class Prod>
__global__ void __launch_bounds__(128, (Prod::LINEAR_FOLD ? (N <= 6 ? 3 : 1) : (N <= 4 ? 3 : 1)))
k_filter_reduce(const __grid_constant__ Prod prod, int K, S* __restrict__ thr_agg,
                S* __restrict__ tile_agg, S* __restrict__ terminal_out, CombineCtx ctx, S* __restrict__ trees)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* nodes = reinterpret_cast<S*>(smem_raw);
    const int B = blockDim.x, t = threadIdx.x;
    const long gthr = (long)blockIdx.x * B + t;
    const long k0 = gthr * K;
    pdl_wait();
    pdl_trigger();
    if (terminal_out && blockIdx.x == 0 && t == 0) {
        Red<N, S> r;
        prod.terminal(r);
        aos_store(terminal_out, 0, r);
    }

    Elem<N, S> G;
    {
        S row[Prod::W];
        prod.load1(k0, row);
        prod.make(k0, row, G);
    }
#pragma unroll 1
    for (int i = 1; i < K; ++i) {
        S row[Prod::W];
        prod.load1(k0 + i, row);
        Elem<N, S> e;
        prod.make(k0 + i, row, e);
        combine<N, S>(e, G, G, ctx);
    }
    wi_store(thr_agg, gthr, G);
    node_store(G, slot<N, S>(nodes, B, 0, t));
    coop_elem_up<N, S>(nodes, scratch_of<N, S>(nodes), ctx);
    if (trees)                             // the tile's tree, for the down-sweep to reuse
        block_copy16<S>(trees + (long)blockIdx.x * 2 * B * CoopLayout<N, S>::NE, nodes,
                        (long)2 * B * CoopLayout<N, S>::NE);
    if (t == 0) {
        Elem<N, S> root;
        node_load(slot<N, S>(nodes, B, ilog2(B), 0), root);
        aos_store(tile_agg, (long)blockIdx.x, root);
    }
}

// The per-step part of the filter down-sweep for one thread: from the value
// function X before step k0, for each of its K steps (those before T) the
// filter value (filt_out), the one-variable combine with the step's element,
// the closed-loop map stored to Eg (compact (V, g) with low-rank noise) and the
// thread's composite map comp_t (x_{k0} = Phi x_{k0+K} + beta).  row_of(i, k,
// row) supplies the step's producer inputs.
template <int N, typename S, class Prod, class RowFn>
__device__ __forceinline__ void filter_steps(const Prod& prod, int K, long k0, long gthr, Red<N, S>& X,
                                             S* __restrict__ Eg, S* __restrict__ filt_out, const CombineCtx& ctx,
                                             Aff<N, S>& comp_t, RowFn row_of)
{
    const long T = prod.T;
    constexpr int NA = Aff<N, S>::NCOMP;
    set_identity(comp_t);
    // compact closed-loop maps: (V, g) instead of (E, g) when E = A - Gam V
    constexpr int NAC = ((N + 1) / 2) * N + N;
    bool compact = false;
    if constexpr (Prod::LOWRANK && !Prod::RESETS) compact = prod.p.lowrank != 0;
    S Vc[((N + 1) / 2) * N];
    // the factor Gam of the process noise in registers for the whole loop
    S gam[((N + 1) / 2) * N];
    if constexpr (Prod::LOWRANK) {
#pragma unroll
        for (int q = 0; q < ((N + 1) / 2) * N; ++q) gam[q] = prod.p.Gam[q];
    }
#pragma unroll 1
    for (int i = 0; i < K; ++i) {
        const long k = k0 + i;
        if (k < T) {
            if (filt_out) {
#pragma unroll
                for (int c = 0; c < Red<N, S>::NCOMP; ++c)
                    filt_out[k * Red<N, S>::NCOMP + c] = comp(X, c);
            }
            S row[Prod::W];
            row_of(i, k, row);
            Elem<N, S> e;
            prod.make(k, row, e);
            Aff<N, S> a;
            if (Prod::RESETS && prod.is_reset(k)) {
                // trajectory start: the previous trajectory ends at the argmin of X
#pragma unroll
                for (int j = 0; j < N * N; ++j) a.F[j] = S(0);
                if (!red_argmin<N, S>(X, a.c)) report_event(ctx.stats, EV_SINGULAR);
                apply<N, S, false>(e, X, nullptr, nullptr, ctx);
            } else {
                bool done = false;
                if constexpr (Prod::LOWRANK) {
                    if (prod.p.lowrank)
                        done = apply_lowrank<N, (N + 1) / 2, S, true>(e, gam, X, a.F, a.c, ctx.cond_max,
                                                                      compact ? Vc : nullptr);
                }
                if (!done) {
                    apply<N, S, true>(e, X, a.F, a.c, ctx);
                    if constexpr (Prod::LOWRANK && !Prod::RESETS) {
                        if (compact) {                 // V = Gam^+ (A - E), exact: A - E lies in range(Gam)
                            constexpr int R = (N + 1) / 2;
#pragma unroll
                            for (int q = 0; q < R; ++q)
#pragma unroll
                                for (int j = 0; j < N; ++j) {
                                    S sv = S(0);
#pragma unroll
                                    for (int l = 0; l < N; ++l)
                                        sv = fma(prod.p.Gpinv[q * N + l], e.A[l * N + j] - a.F[l * N + j], sv);
                                    Vc[q * N + j] = sv;
                                }
                        }
                    }
                }
            }
            if (compact) {
                // compact map (V, g), E = A - Gam V (linear model with low-rank noise)
                constexpr int R = (N + 1) / 2;
#pragma unroll
                for (int c = 0; c < R * N; ++c) Eg[wis_idx(gthr, i, c, K, NAC)] = Vc[c];
#pragma unroll
                for (int c = 0; c < N; ++c) Eg[wis_idx(gthr, i, R * N + c, K, NAC)] = a.c[c];
            } else {
#pragma unroll
                for (int c = 0; c < NA; ++c) Eg[wis_idx(gthr, i, c, K, NA)] = comp(a, c);
            }
            // x_{k0} = Phi x_{k+1} + beta:  beta += Phi g,  Phi = Phi E
            S tmp[N];
            ms::mv<N, S>(comp_t.F, a.c, tmp);
#pragma unroll
            for (int j = 0; j < N; ++j) comp_t.c[j] += tmp[j];
            S F2[N * N];
            ms::mm<N, S>(comp_t.F, a.F, F2);
#pragma unroll
            for (int j = 0; j < N * N; ++j) comp_t.F[j] = F2[j];
        }
    }
}

// ---------------------------------------------------------------------------
// phase 2: per-step filter values, closed-loop maps and their per-thread /
// per-tile compositions; the last CTA writes the value function at x_T
// ---------------------------------------------------------------------------
template <int N, typename S, class Prod>
__global__ void __launch_bounds__(128, (Prod::LINEAR_FOLD ? (N <= 6 ? 3 : 1) : (N <= 4 ? 3 : 1)))
k_filter_down(const __grid_constant__ Prod prod, int K, S* __restrict__ thr_agg,
              const S* __restrict__ tile_agg, const Red<N, S> prior, const S* __restrict__ prior_dev,
              S* __restrict__ Eg, S* __restrict__ thr_aff, S* __restrict__ tile_aff, S* __restrict__ filt_out,
              CombineCtx ctx, const LtiTiles<S> lt, S* __restrict__ final_out, S* __restrict__ xT_out,
              S* __restrict__ filtT_out, const S* __restrict__ group_agg, const S* __restrict__ trees)
{
    const S* __restrict__ fold = lt.fold;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* nodes = reinterpret_cast<S*>(smem_raw);
    const int B = blockDim.x, t = threadIdx.x;
    const int tile = down_tile();
    const long gthr = (long)tile * B + t;
    const long k0 = gthr * K;
    const long T = prod.T;

    const bool last_lti = fold && tile + 1 == (int)gridDim.x;
    S leaf[2 * N] = {};
    if constexpr (Prod::LINEAR_FOLD && N <= 6)
        if (fold) lti_stage_tables<N, Prod::W, S>(lt, K, nodes);
    if (last_lti) lti_last_tile_leaf<N, S>(prod, tile, K, fold, nodes, leaf);
    pdl_wait();                            // totals and aggregates of the reduce kernel
    pdl_trigger();
    Red<N, S> pin, X;
    if (fold)
        lti_tile_prefix<N, S>(lt, tile, prior, nodes, pin);
    else
        tile_prefix_of<N, S>(tile_agg, tile, scan_prior(prior, prior_dev), nodes, ctx, pin, group_agg);
    tile_thread_prefix<N, S>(prod, tile, K, thr_agg, pin, lt, last_lti, leaf, nodes, ctx, X,
                             trees && !fold ? trees + (long)tile * 2 * B * CoopLayout<N, S>::NE : nullptr);

    Aff<N, S> comp_t;
    filter_steps<N, S>(prod, K, k0, gthr, X, Eg, filt_out, ctx, comp_t,
                       [&](int, long k, S* row) { prod.load1(k, row); });
    write_final_if_last<N, S>(T, tile, K, X, final_out, xT_out, filtT_out, ctx);
    wi_store(thr_aff, gthr, comp_t);
    __syncthreads();                       // the filter trees are done with shared memory
    block_aff_reduce<N, S>(comp_t, nodes);
    if (t == 0) aos_store(tile_aff, (long)tile, comp_t);
}

// ---------------------------------------------------------------------------
// phase 2 of the two-filter smoother, forward part: per-step filter value
// functions (S_k, v_k), stored per thread and step (warp-interleaved)
// ---------------------------------------------------------------------------
template <int N, typename S, class Prod>
__global__ void __launch_bounds__(128, (N <= 6 ? 3 : 1))
k_filter_states(const __grid_constant__ Prod prod, int K, S* __restrict__ thr_agg,
                const S* __restrict__ tile_agg, const Red<N, S> prior, S* __restrict__ filt_ws,
                S* __restrict__ filt_out, CombineCtx ctx, const LtiTiles<S> lt,
                S* __restrict__ final_out, S* __restrict__ xT_out, S* __restrict__ filtT_out)
{
    const S* __restrict__ fold = lt.fold;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* nodes = reinterpret_cast<S*>(smem_raw);
    const int B = blockDim.x, t = threadIdx.x;
    const int tile = down_tile();
    const long gthr = (long)tile * B + t;
    const long k0 = gthr * K;
    const long T = prod.T;
    constexpr int NR = Red<N, S>::NCOMP;
    const bool last_lti = fold && tile + 1 == (int)gridDim.x;
    S leaf[2 * N] = {};
    if constexpr (Prod::LINEAR_FOLD && N <= 6)
        if (fold) lti_stage_tables<N, Prod::W, S>(lt, K, nodes);
    if (last_lti) lti_last_tile_leaf<N, S>(prod, tile, K, fold, nodes, leaf);
    pdl_wait();
    pdl_trigger();
    Red<N, S> pin, X;
    if (fold)
        lti_tile_prefix<N, S>(lt, tile, prior, nodes, pin);
    else
        tile_prefix_of<N, S>(tile_agg, tile, prior, nodes, ctx, pin);
    tile_thread_prefix<N, S>(prod, tile, K, thr_agg, pin, lt, last_lti, leaf, nodes, ctx, X);
#pragma unroll 1
    for (int i = 0; i < K; ++i) {
        const long k = k0 + i;
        if (k < T) {
#pragma unroll
            for (int c = 0; c < NR; ++c) filt_ws[wis_idx(gthr, i, c, K, NR)] = comp(X, c);
            if (filt_out) {
#pragma unroll
                for (int c = 0; c < NR; ++c) filt_out[k * NR + c] = comp(X, c);
            }
            S row[Prod::W];
            prod.load1(k, row);
            Elem<N, S> e;
            prod.make(k, row, e);
            bool done = false;
            if constexpr (Prod::LOWRANK) {
                if (prod.p.lowrank)
                    done = apply_lowrank<N, (N + 1) / 2, S, false>(e, prod.p.Gam, X, nullptr, nullptr, ctx.cond_max);
            }
            if (!done) apply<N, S, false>(e, X, nullptr, nullptr, ctx);
        }
    }
    write_final_if_last<N, S>(T, tile, K, X, final_out, xT_out, filtT_out, ctx);
}

// x = (S + L)^-1 (v + z) for symmetric positive definite S + L (Cholesky; a
// non-positive pivot falls back to Gauss-Jordan with row pivoting)
template <int N, typename S>
__device__ __forceinline__ void spd_combine_solve(const Red<N, S>& a, const Red<N, S>& b, S* x)
{
    S M[N * N], rhs[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        rhs[i] = a.v[i] + b.v[i];
#pragma unroll
        for (int j = 0; j < N; ++j) M[i * N + j] = a.P[Sym<N>::at(i, j)] + b.P[Sym<N>::at(i, j)];
    }
    S Lc[N * N];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        S d = M[j * N + j];
#pragma unroll
        for (int k = 0; k < j; ++k) d = fma(-Lc[j * N + k], Lc[j * N + k], d);
        ok = ok && d > S(0);
        const S ljj = sqrt(d > S(0) ? d : S(1));
        const S il = S(1) / ljj;
        Lc[j * N + j] = ljj;
#pragma unroll
        for (int i = j + 1; i < N; ++i) {
            S s = M[i * N + j];
#pragma unroll
            for (int k = 0; k < j; ++k) s = fma(-Lc[i * N + k], Lc[j * N + k], s);
            Lc[i * N + j] = s * il;
        }
    }
    if (ok) {
        S z[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S s = rhs[i];
#pragma unroll
            for (int k = 0; k < i; ++k) s = fma(-Lc[i * N + k], z[k], s);
            z[i] = s / Lc[i * N + i];
        }
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
            S s = z[i];
#pragma unroll
            for (int k = i + 1; k < N; ++k) s = fma(-Lc[k * N + i], x[k], s);
            x[i] = s / Lc[i * N + i];
        }
    } else {
        S Mi[N * N];
        ms::inv_row_pivot<N, S>(M, Mi);
        ms::mv<N, S>(Mi, rhs, x);
    }
}

// ---------------------------------------------------------------------------
// phase 2 of the two-filter smoother, backward part: per-step backward
// information (Lam_k, zeta_k) on x_k from y_{k+1}..y_T, combined with the
// forward filter: x*_k = (S_k + Lam_k)^-1 (v_k + zeta_k)  (Eq. 43 in
// information form).  Thread g' of this reversed scan covers the steps of
// forward thread g = nthr - 1 - g'; the scan's prior is the terminal value
// function that its reduce kernel wrote to prior_dev.
// ---------------------------------------------------------------------------
template <int N, typename S, class RProd>
__global__ void __launch_bounds__(128, (N <= 6 ? 3 : 1))
k_tf_down(const __grid_constant__ RProd prod, int K, const S* __restrict__ thr_agg,
          const S* __restrict__ tile_agg, const S* __restrict__ prior_dev, const S* __restrict__ filt_ws,
          S* __restrict__ x_out, CombineCtx ctx)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* nodes = reinterpret_cast<S*>(smem_raw);
    const int B = blockDim.x, t = threadIdx.x;
    const long gthr = (long)blockIdx.x * B + t;
    const long nthr = (long)gridDim.x * B;
    const long j0 = gthr * K;
    const long T = prod.T, Tpad = prod.Tpad;
    const long gf = nthr - 1 - gthr;            // forward thread with the same steps
    constexpr int NR = Red<N, S>::NCOMP;
    pdl_wait();
    Red<N, S> pin, X, zero;
#pragma unroll
    for (int c = 0; c < NR; ++c) comp(zero, c) = S(0);
    tile_prefix_of<N, S>(tile_agg, blockIdx.x, scan_prior(zero, prior_dev), nodes, ctx, pin);
    {
        Elem<N, S> G;
        wi_load(thr_agg, gthr, G);
        node_store(G, slot<N, S>(nodes, B, 0, t));
    }
    coop_elem_up<N, S>(nodes, scratch_of<N, S>(nodes), ctx);
    coop_elem_down<N, S>(nodes, scratch_of<N, S>(nodes), pin, ctx, X);
    // the block's steps are forward tile (gridDim.x - 1 - blockIdx.x); its states
    // are staged in shared memory (the tree is no longer needed) and stored coalesced
    __syncthreads();
    S* st = nodes;
    const int tf = B - 1 - t;
#pragma unroll 1
    for (int i = 0; i < K; ++i) {
        const long j = j0 + i;
        const long k = Tpad - 1 - j;
        S* xk = st + (tf * K + (K - 1 - i)) * N;
        if (k < T) {
            S row[RProd::W];
            prod.load1(j, row);
            Elem<N, S> e;
            prod.make(j, row, e);
            Red<N, S> Lam = X, F;
            Elem<N, S> e0 = e;
#pragma unroll
            for (int q = 0; q < Sym<N>::SZ; ++q) e0.J[q] = S(0);
#pragma unroll
            for (int q = 0; q < N; ++q) e0.eta[q] = S(0);
            apply<N, S, false>(e0, Lam, nullptr, nullptr, ctx);   // information from y_{k+1}..y_T
#pragma unroll
            for (int c = 0; c < NR; ++c) comp(F, c) = filt_ws[wis_idx(gf, K - 1 - i, c, K, NR)];
            S x[N];
            spd_combine_solve<N, S>(F, Lam, x);
#pragma unroll
            for (int q = 0; q < N; ++q) xk[q] = x[q];
#pragma unroll
            for (int q = 0; q < Sym<N>::SZ; ++q) X.P[q] = Lam.P[q] + e.J[q];
#pragma unroll
            for (int q = 0; q < N; ++q) X.v[q] = Lam.v[q] + e.eta[q];
        }
    }
    __syncthreads();
    const long base = (long)(gridDim.x - 1 - blockIdx.x) * B * K * N;
    const long lim = T * N;
    for (int idx = t; idx < B * K * N; idx += B)
        if (base + idx < lim) x_out[base + idx] = st[idx];
}

// shared-memory stride of one thread's staged states: its K states
// contiguous, so that the staged block is the tile's output block
__host__ __device__ __forceinline__ int rts_stage_stride(int K, int N) { return K * N; }

// x (N scalars) into shared memory, as 16-byte words when the row allows
template <int N, typename S>
__device__ __forceinline__ void stage_state(S* dst, const S* x)
{
    if constexpr (sizeof(S) == 4 && N % 4 == 0) {
#pragma unroll
        for (int q = 0; q < N; q += 4)
            *reinterpret_cast<float4*>(dst + q) = make_float4(x[q], x[q + 1], x[q + 2], x[q + 3]);
    } else if constexpr (sizeof(S) == 8 && N % 2 == 0) {
#pragma unroll
        for (int q = 0; q < N; q += 2) *reinterpret_cast<double2*>(dst + q) = make_double2(x[q], x[q + 1]);
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) dst[q] = x[q];
    }
}

// ---------------------------------------------------------------------------
// phase 3: per-step smoothed states x_k = E_k x_{k+1} + g_k
// ---------------------------------------------------------------------------
// form of the stored closed-loop maps: (E, g), or the compact (V, g) with
// E = A - Gam V for linear models with low-rank process noise
template <int N, typename S>
struct EgForm {
    static constexpr int R = (N + 1) / 2;
    int compact;
    S A[N * N];
    S Gam[N * R];
};

// The per-step part of the RTS pass for one thread: from the state x at the
// end of its steps, x_k = E_k x_{k+1} + g_k for its steps before T, backwards,
// each state staged at mine[i N] (the maps are loaded four steps ahead).
template <int N, typename S>
__device__ __forceinline__ void rts_steps(const S* __restrict__ Eg, int K, long k0, long gthr, long T,
                                          const EgForm<N, S>& form, S* x, S* mine)
{
    constexpr int NA = Aff<N, S>::NCOMP;
    constexpr int U = 4;                   // steps whose maps are loaded ahead of use
    if (form.compact) {
        // A and Gam in registers for the whole loop (form is kernel-parameter
        // memory reached through a reference)
        constexpr int RR = EgForm<N, S>::R;
        S fA[N * N], fG[N * RR];
#pragma unroll
        for (int q = 0; q < N * N; ++q) fA[q] = form.A[q];
#pragma unroll
        for (int q = 0; q < N * RR; ++q) fG[q] = form.Gam[q];
        // x_k = A x_{k+1} - Gam (V_k x_{k+1}) + g_k
        constexpr int R = EgForm<N, S>::R, NAC = R * N + N;
#pragma unroll 1
        for (int i0 = K - 1; i0 >= 0; i0 -= U) {
            S buf[U][NAC];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 - u;
                if (i >= 0 && k0 + i < T) {
#pragma unroll
                    for (int c = 0; c < NAC; ++c) buf[u][c] = Eg[wis_idx(gthr, i, c, K, NAC)];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 - u;
                if (i >= 0) {
                    if (k0 + i < T) {
                        S vx[R], y[N];
#pragma unroll
                        for (int q = 0; q < R; ++q) {
                            S acc = S(0);
#pragma unroll
                            for (int j = 0; j < N; ++j) acc = fma(buf[u][q * N + j], x[j], acc);
                            vx[q] = acc;
                        }
#pragma unroll
                        for (int r = 0; r < N; ++r) {
                            S acc = buf[u][R * N + r];
#pragma unroll
                            for (int q = 0; q < N; ++q) acc = fma(fA[r * N + q], x[q], acc);
#pragma unroll
                            for (int q = 0; q < R; ++q) acc = fma(-fG[r * R + q], vx[q], acc);
                            y[r] = acc;
                        }
#pragma unroll
                        for (int j = 0; j < N; ++j) x[j] = y[j];
                    }
                    stage_state<N, S>(mine + i * N, x);
                }
            }
        }
    } else {
#pragma unroll 1
        for (int i0 = K - 1; i0 >= 0; i0 -= U) {
            S buf[U][NA];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 - u;
                if (i >= 0 && k0 + i < T) {
#pragma unroll
                    for (int c = 0; c < NA; ++c) buf[u][c] = Eg[wis_idx(gthr, i, c, K, NA)];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 - u;
                if (i >= 0) {
                    if (k0 + i < T) {
                        S y[N];
#pragma unroll
                        for (int r = 0; r < N; ++r) {
                            S acc = buf[u][N * N + r];
#pragma unroll
                            for (int q = 0; q < N; ++q) acc = fma(buf[u][r * N + q], x[q], acc);
                            y[r] = acc;
                        }
#pragma unroll
                        for (int j = 0; j < N; ++j) x[j] = y[j];
                    }
                    stage_state<N, S>(mine + i * N, x);
                }
            }
        }
    }
}

template <int N, typename S>
__global__ void __launch_bounds__(128)
k_rts_down(const S* __restrict__ Eg, int K, const S* __restrict__ thr_aff, const S* __restrict__ tile_aff,
           const S* __restrict__ xT, long T, S* __restrict__ x_out, const __grid_constant__ EgForm<N, S> form)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* nodes = reinterpret_cast<S*>(smem_raw);
    const int B = blockDim.x, t = threadIdx.x;
    const long gthr = (long)blockIdx.x * B + t;
    const long k0 = gthr * K;
    pdl_wait();                            // maps and x_T of the previous kernel
    S* xe_sh = nodes + 2 * B * CoopLayout<N, S>::NA;   // staging area, free until the state loop
    tile_suffix_state<N, S>(tile_aff, blockIdx.x, gridDim.x, xT, nodes, xe_sh);
    S x[N];
    {
        Aff<N, S> a;
        wi_load(thr_aff, gthr, a);
        block_aff_end_states<N, S>(a, xe_sh, nodes, x);
    }
    // the states are staged past the affine tree and written out coalesced
    const int SP = rts_stage_stride(K, N);
    S* st = nodes + 2 * B * CoopLayout<N, S>::NA;
    S* mine = st + t * SP;
    rts_steps<N, S>(Eg, K, k0, gthr, T, form, x, mine);
    __syncthreads();
    // the staged block is the tile's block of x_out (x_T itself comes from the
    // filter kernel): one bulk copy of its 16-byte part, the rest by plain stores
    const int KN = K * N;
    const long base = (long)blockIdx.x * B * KN;
    const long cnt = min((long)B * KN, T * N - base);
    long done = 0;
    if ((reinterpret_cast<uintptr_t>(x_out + base) & 15) == 0) {
        done = cnt * (long)sizeof(S) / 16 * 16 / (long)sizeof(S);
        if (t == 0 && done > 0) {
            fence_proxy_async_smem();
            bulk_copy_s2g(x_out + base, st, (unsigned)(done * sizeof(S)));
            bulk_commit_and_wait();
        }
    }
    for (long idx = done + t; idx < cnt; idx += B) x_out[base + idx] = st[idx];
    __syncthreads();                       // the bulk copy has read the staged block
}

// shared memory of k_rts_down: the affine tree and the staged states
template <int N, typename S>
__host__ __device__ constexpr size_t rts_smem(int B, int K)
{
    return aff_tree_smem<N, S>(B) + sizeof(S) * (size_t)B * rts_stage_stride(K, N);
}

// ---------------------------------------------------------------------------
// single-launch solve of a linear time-invariant model (RTS smoother): the
// reduce, filter down-sweep and RTS phases of the three-kernel path in one
// cooperative launch of one CTA per tile, separated by two grid barriers
// ---------------------------------------------------------------------------
// Grid barrier state in global memory: arrivals and generation (both start at
// zero; the last arrival resets the count before it advances the generation).
// Grid barrier state: a 64-bit arrival counter that only grows, and the
// number of arrivals before this launch (kept by the host: every launch adds
// two barriers' worth, 2 x gridDim.x).  Barrier p of the launch (p = 1, 2)
// completes when the counter reaches base + p * gridDim.x, so nothing is
// reset and the last arrival releases the others by its own increment.
struct GridSync {
    unsigned long long* count;
    unsigned long long base;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

constexpr int GRID_SPINS = 1 << 25;         // bounded wait (about a second with the back-off)

// All CTAs of the (co-resident) grid reach barrier p; the global writes of
// each CTA before it are visible to all after it.  A wait that runs out counts
// in stats[2] and lets the CTA continue.
__device__ __forceinline__ void grid_sync(const GridSync& gs, int p, unsigned long long* stats,
                                          int spins = GRID_SPINS)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long target = gs.base + (unsigned long long)p * gridDim.x;
        __threadfence();
        atomicAdd(gs.count, 1ull);
        int n = 0;
        while (ld_acquire_u64(gs.count) < target) {
            if (++n > spins) {
                report_event(stats, EV_TIMEOUT);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
}

// shared memory of k_lti_solve (offsets in scalars): the (b, eta) nodes and
// the tile's prefix, the composition area of the shuffle reductions, the
// tile's observations (bulk copy), the Gamma_i, the bulk copy's mbarrier, the
// level constants and the co table; the RTS phase stages the states from 0.
template <int N, int M, typename S>
struct FusedSmem {
    using FL = FoldLayout<N, M, S>;
    __host__ __device__ static constexpr int al(int x) { return (x + 3) / 4 * 4; }
    __host__ __device__ static constexpr int lb(int B) { return B >= 128 ? 7 : B >= 64 ? 6 : B >= 32 ? 5 : 4; }
    __host__ __device__ static constexpr int bq(int) { return 0; }
    __host__ __device__ static constexpr int pin(int B) { return 2 * B * 2 * N; }
    __host__ __device__ static constexpr int red(int B) { return al(pin(B) + CoopLayout<N, S>::NR); }
    // the composition area also holds P_j and F_j during the first phase
    __host__ __device__ static constexpr int red_size(int B)
    {
        return (B / 32) * (Aff<N, S>::NCOMP + N) + N > Sym<N>::SZ + N * N ? (B / 32) * (Aff<N, S>::NCOMP + N) + N
                                                                          : Sym<N>::SZ + N * N;
    }
    __host__ __device__ static constexpr int ys(int B) { return al(red(B) + red_size(B)); }
    __host__ __device__ static constexpr int gam(int B, int K) { return al(ys(B) + B * K * M); }
    __host__ __device__ static constexpr int bar(int B, int K) { return al(gam(B, K) + K * FL::GS); }
    __host__ __device__ static constexpr int lv(int B, int K) { return bar(B, K) + 4; }
    __host__ __device__ static constexpr int co(int B, int K) { return lv(B, K) + al(lb(B) * FL::LS); }
    __host__ __device__ static constexpr int end(int B, int K) { return co(B, K) + B * FL::CS; }
    __host__ __device__ static constexpr int stage(int B) { return al(red_size(B)); }
    __host__ __device__ static constexpr size_t bytes(int B, int K)
    {
        const int e = end(B, K), r = stage(B) + B * K * N;
        return sizeof(S) * (size_t)(e > r ? e : r);
    }
};

template <int N, typename S, class Prod>
__global__ void __launch_bounds__(128, (N <= 6 ? 3 : 1))
k_lti_solve(const __grid_constant__ Prod prod, int K, const LtiTiles<S> lt, const Red<N, S> prior,
            S* __restrict__ Eg, S* __restrict__ tile_aff, S* __restrict__ filt_out, CombineCtx ctx,
            S* __restrict__ final_out, S* __restrict__ x_out, S* __restrict__ filtT_out,
            const __grid_constant__ EgForm<N, S> form, const GridSync gs)
{
    if constexpr (Prod::LINEAR_FOLD && N <= 6) {
        constexpr int M = Prod::W;
        using FL = FoldLayout<N, M, S>;
        using FS = FusedSmem<N, M, S>;
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
        unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + FS::bar(B, K));

        // ---- phase 1: the tile's observations, per-thread folds, up-sweep, w_j
        // bulk copies (one mbarrier phase): the tile's observations (full tiles),
        // the level constants, the co table and the Gamma_i (all 16-byte runs)
        const int LB = ilog2(B);
        const unsigned ybytes = last ? 0u : (unsigned)(sizeof(S) * (size_t)B * K * M);
        const unsigned lbytes = (unsigned)(sizeof(S) * (size_t)LB * FL::LS);
        const unsigned cbytes = (unsigned)(sizeof(S) * (size_t)(B - 1) * FL::CS);
        // (the Gamma_i rounded up to whole 16-byte words: the fold buffer holds
        // KMAX of them and the shared area is padded to 4 scalars)
        const unsigned gbytes = (unsigned)(sizeof(S) * (size_t)((K * FL::GS + 3) / 4 * 4));
        // the co table (needed only in phase 2) completes on a second mbarrier
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
        if (!last) {                               // P_j and F_j for w_j, in the composition area
            for (int q = t; q < Sym<N>::SZ; q += B) red[q] = lt.P[(long)tile * Sym<N>::SZ + q];
            for (int q = t; q < N * N; q += B) red[Sym<N>::SZ + q] = lt.F[(long)tile * N * N + q];
        }
        if (last) {                                // the last tile's observations up to T, zeros after
            const long base = (long)tile * B * K * M, have = T * M - base;
            for (long q = t; q < (long)B * K * M; q += B) ys[q] = q < have ? prod.y[base + q] : S(0);
        }
        const bool ok = mbar_wait_bounded(bar, 0, MBAR_POLLS);
        if (!__syncthreads_and(ok)) {
            if (t == 0) report_event(ctx.stats, EV_TIMEOUT);
            mbar_wait_bounded(bar, 0, MBAR_POLLS);  // the copy may still be in flight
        }
        S leaf[2 * N];
        if (!last || k0 + K <= T) {
#pragma unroll
            for (int q = 0; q < N; ++q) { leaf[q] = __ldg(fold + FL::ob + q); leaf[N + q] = __ldg(fold + FL::oe + q); }
            const S* yt = ys + t * K * M;
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
        lti_tree_up<N, M, S>(bq, lv);              // starts and ends with a barrier
        if (!last && t == 0) {                     // w_j = eta_j - F_j P_j b_j
            const S* rq = bq + lti_node_level(2 * N, B, ilog2(B));
            const long j = tile;
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
                for (int c = 0; c < N; ++c) acc = fma(-red[Sym<N>::SZ + a * N + c], Pb[c], acc);
                lt.w[j * N + a] = acc;
            }
        }
        grid_sync(gs, 1, ctx.stats);

        // ---- phase 2: tile prefix, thread prefixes, per-step filter, tile map
        Red<N, S> pin, X;
        lti_tile_prefix_sum<N, S>(lt, tile, gridDim.x, prior, red, pin);
        if (t == 0) node_store(pin, ps);
        if (!mbar_wait_bounded(bar_co, 0, MBAR_POLLS) && t == 0)
            report_event(ctx.stats, EV_TIMEOUT);   // the co table
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
        Aff<N, S> comp_t;
        const S* yt = ys + t * K * M;
        filter_steps<N, S>(prod, K, k0, gthr, X, Eg, filt_out, ctx, comp_t, [&](int i, long, S* row) {
#pragma unroll
            for (int c = 0; c < M; ++c) row[c] = yt[i * M + c];
        });
        S* xT = x_out + T * N;
        write_final_if_last<N, S>(T, tile, K, X, final_out, xT, filtT_out, ctx);
        {
            Aff<N, S> H = comp_t;
            __syncthreads();                       // the trees are done with shared memory
            block_aff_reduce<N, S>(H, red);
            if (t == 0) aos_store(tile_aff, (long)tile, H);
        }
        grid_sync(gs, 2, ctx.stats);

        // ---- phase 3: tile suffix, thread end states, per-step states, bulk store
        S* st = sm + FS::stage(B);
        S* xe_sh = red + (B / 32) * (Aff<N, S>::NCOMP + N);
        lti_tile_suffix_sum<N, S>(lt, tile_aff, tile, gridDim.x, xT, red, xe_sh);
        S x[N];
        block_aff_end_states<N, S>(comp_t, xe_sh, red, x);
        S* mine = st + t * rts_stage_stride(K, N);
        rts_steps<N, S>(Eg, K, k0, gthr, T, form, x, mine);
        __syncthreads();
        const int KN = K * N;
        const long base = (long)tile * B * KN;
        const long cnt = min((long)B * KN, T * N - base);
        long done = 0;
        if ((reinterpret_cast<uintptr_t>(x_out + base) & 15) == 0) {
            done = cnt * (long)sizeof(S) / 16 * 16 / (long)sizeof(S);
            if (t == 0 && done > 0) {
                fence_proxy_async_smem();
                bulk_copy_s2g(x_out + base, st, (unsigned)(done * sizeof(S)));
                bulk_commit_and_wait();
            }
        }
        for (long idx = done + t; idx < cnt; idx += B) x_out[base + idx] = st[idx];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// sequential baseline: the same elements and recursions evaluated by one
// thread in time order (information filter of Eq. 17 in discrete form, then
// the closed-loop maps backwards), no scan
// ---------------------------------------------------------------------------
template <int N, typename S, class Prod>
__global__ void __launch_bounds__(32)
k_sequential(const __grid_constant__ Prod prod, Red<N, S> prior, S* __restrict__ Eg,
             S* __restrict__ x_out, CombineCtx ctx)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const long T = prod.T;
    Red<N, S> X = prior;
    for (long k = 0; k < T; ++k) {
        S row[Prod::W];
        prod.load1(k, row);
        Elem<N, S> e;
        prod.make(k, row, e);
        Aff<N, S> a;
        apply<N, S, true>(e, X, a.F, a.c, ctx);
        aos_store(Eg, k, a);
    }
    S x[N];
    if (!red_argmin<N, S>(X, x)) report_event(ctx.stats, EV_SINGULAR);
#pragma unroll
    for (int j = 0; j < N; ++j) x_out[T * N + j] = x[j];
    for (long k = T - 1; k >= 0; --k) {
        Aff<N, S> a;
        aos_load(Eg, k, a);
        S y[N];
        affine_apply<N, S>(a, x, y);
#pragma unroll
        for (int j = 0; j < N; ++j) { x[j] = y[j]; x_out[k * N + j] = y[j]; }
    }
}

}  // namespace mapk
