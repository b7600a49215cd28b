// Blocked three-phase associative scans (reduce / scan of tile totals /
// down-sweep) for the filter (Section 3.3-3.4, Eq. 32) and the RTS pass
// (Section 3.5 and 4.3, Eq. 40-42).
//
// Work decomposition.  A tile of L = B*K consecutive steps is one CTA of B
// threads; thread t owns steps [k0, k0+K), k0 = (tile*B + t)*K, and builds
// its elements in registers from the per-step inputs.  Within a CTA the
// per-thread partials are scanned with a work-efficient up/down sweep
// (Blelloch) through shared memory; across tiles a single CTA scans the tile
// totals.  There are no inter-CTA waits anywhere: every dependency between
// tiles is a kernel boundary.
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
#include "producers.cuh"

namespace mapk {

// Level d of a tree over B leaves has B >> d nodes stored from lvl_off(B, d);
// all 2B - 1 nodes fit in 2B slots.
__device__ __forceinline__ int lvl_off(int B, int d) { return 2 * B - ((2 * B) >> d); }

__device__ __forceinline__ int ilog2(int B) { return 31 - __clz(B); }

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

// ---------------------------------------------------------------------------
// block-level trees in shared memory (component-major: sh[c * 2B + node])
// ---------------------------------------------------------------------------

// up-sweep over B filter partials; level 0 must be stored by the caller
template <int N, typename S>
__device__ void elem_tree_up(S* sh, int B, int t, const CombineCtx& ctx)
{
    const int LB = ilog2(B);
    const int st = 2 * B;
    for (int d = 0; d < LB; ++d) {
        __syncthreads();
        if (t < (B >> (d + 1))) {
            Elem<N, S> l, r;
            soa_load(sh, st, lvl_off(B, d) + 2 * t, l);
            soa_load(sh, st, lvl_off(B, d) + 2 * t + 1, r);
            combine<N, S>(r, l, r, ctx);               // later partial on the left
            soa_store(sh, st, lvl_off(B, d + 1) + t, r);
        }
    }
    __syncthreads();
}

// down-sweep: exclusive prefixes (one-variable value functions) of all leaves
// given the prefix `pin` of the whole block (held by thread 0)
template <int N, typename S>
__device__ void elem_tree_down(const S* sh, S* pr, int B, int t, const Red<N, S>& pin,
                               const CombineCtx& ctx, Red<N, S>& out)
{
    const int LB = ilog2(B);
    const int st = 2 * B;
    if (t == 0) {
        Red<N, S> p = pin;
        soa_store(pr, st, lvl_off(B, LB), p);
    }
    for (int d = LB - 1; d >= 0; --d) {
        __syncthreads();
        if (t < (B >> (d + 1))) {
            Red<N, S> p;
            Elem<N, S> l;
            soa_load(pr, st, lvl_off(B, d + 1) + t, p);
            soa_store(pr, st, lvl_off(B, d) + 2 * t, p);
            soa_load(sh, st, lvl_off(B, d) + 2 * t, l);
            apply<N, S, false>(l, p, nullptr, nullptr, ctx);
            soa_store(pr, st, lvl_off(B, d) + 2 * t + 1, p);
        }
    }
    __syncthreads();
    soa_load(pr, st, t, out);
}

// affine maps: node(d+1, t) = node(d, 2t) o node(d, 2t+1)  (a leaf maps the
// state at the END of its steps to the state at their START)
template <int N, typename S>
__device__ void aff_tree_up(S* sh, int B, int t)
{
    const int LB = ilog2(B);
    const int st = 2 * B;
    for (int d = 0; d < LB; ++d) {
        __syncthreads();
        if (t < (B >> (d + 1))) {
            Aff<N, S> l, r;
            soa_load(sh, st, lvl_off(B, d) + 2 * t, l);
            soa_load(sh, st, lvl_off(B, d) + 2 * t + 1, r);
            compose<N, S>(l, r, l);
            soa_store(sh, st, lvl_off(B, d + 1) + t, l);
        }
    }
    __syncthreads();
}

// suffix down-sweep: the state at the END of every leaf, given the state at
// the end of the block (held by thread 0)
template <int N, typename S>
__device__ void aff_tree_down(const S* sh, S* xs, int B, int t, const S* xend, S* out)
{
    const int LB = ilog2(B);
    const int st = 2 * B;
    if (t == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) xs[i * st + lvl_off(B, LB)] = xend[i];
    }
    for (int d = LB - 1; d >= 0; --d) {
        __syncthreads();
        if (t < (B >> (d + 1))) {
            S x[N], y[N];
#pragma unroll
            for (int i = 0; i < N; ++i) x[i] = xs[i * st + lvl_off(B, d + 1) + t];
#pragma unroll
            for (int i = 0; i < N; ++i) xs[i * st + lvl_off(B, d) + 2 * t + 1] = x[i];
            Aff<N, S> r;
            soa_load(sh, st, lvl_off(B, d) + 2 * t + 1, r);
            affine_apply<N, S>(r, x, y);
#pragma unroll
            for (int i = 0; i < N; ++i) xs[i * st + lvl_off(B, d) + 2 * t] = y[i];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = xs[i * st + t];
}

// ---------------------------------------------------------------------------
// phase 1: per-thread fold and per-tile total of the filter elements
// ---------------------------------------------------------------------------
template <int N, typename S, class Prod, int K>
__global__ void __launch_bounds__(256)
k_filter_reduce(const __grid_constant__ Prod prod, S* __restrict__ thr_agg,
                S* __restrict__ tile_agg, CombineCtx ctx)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* sh = reinterpret_cast<S*>(smem_raw);
    const int B = blockDim.x, t = threadIdx.x;
    const long gthr = (long)blockIdx.x * B + t;
    const long k0 = gthr * K;

    S rows[K * Prod::W];
    prod.template load<K>(k0, rows);
    Elem<N, S> G;
    prod.make(k0, rows, G);
#pragma unroll
    for (int i = 1; i < K; ++i) {
        Elem<N, S> e;
        prod.make(k0 + i, rows + i * Prod::W, e);
        combine<N, S>(e, G, G, ctx);
    }
    aos_store(thr_agg, gthr, G);
    soa_store(sh, 2 * B, t, G);
    elem_tree_up<N, S>(sh, B, t, ctx);
    if (t == 0) {
        Elem<N, S> root;
        soa_load(sh, 2 * B, lvl_off(B, ilog2(B)), root);
        aos_store(tile_agg, (long)blockIdx.x, root);
    }
}

// ---------------------------------------------------------------------------
// phase 2: one CTA scans the tile totals from the prior (Eq. 31 a_T)
// ---------------------------------------------------------------------------
template <int N, typename S>
__global__ void __launch_bounds__(256)
k_filter_tiles(const S* __restrict__ tile_agg, int nt, Red<N, S> prior,
               S* __restrict__ tile_pref, S* __restrict__ final_out, S* __restrict__ xT_out,
               S* __restrict__ filtT_out, CombineCtx ctx)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int B = blockDim.x, t = threadIdx.x;
    S* sh = reinterpret_cast<S*>(smem_raw);
    S* pr = sh + Elem<N, S>::NCOMP * 2 * B;
    const int per = (nt + B - 1) / B;
    const int first = t * per, last = min(nt, first + per);

    Elem<N, S> H;
    set_identity(H);
    for (int i = first; i < last; ++i) {
        Elem<N, S> g;
        aos_load(tile_agg, i, g);
        combine<N, S>(g, H, H, ctx);
    }
    soa_store(sh, 2 * B, t, H);
    elem_tree_up<N, S>(sh, B, t, ctx);
    Red<N, S> P;
    elem_tree_down<N, S>(sh, pr, B, t, prior, ctx, P);
    for (int i = first; i < last; ++i) {
        aos_store(tile_pref, i, P);
        Elem<N, S> g;
        aos_load(tile_agg, i, g);
        apply<N, S, false>(g, P, nullptr, nullptr, ctx);
    }
    if (t == B - 1) {
        // P is now the value function at the end of the last tile, i.e. at x_T
        aos_store(final_out, 0, P);
        S x[N];
        if (!red_argmin<N, S>(P, x) && ctx.stats) atomicAdd(ctx.stats + 1, 1ull);
#pragma unroll
        for (int i = 0; i < N; ++i) xT_out[i] = x[i];
        if (filtT_out) {
#pragma unroll
            for (int i = 0; i < Red<N, S>::NCOMP; ++i) filtT_out[i] = comp(P, i);
        }
    }
}

// ---------------------------------------------------------------------------
// phase 3: per-step filter values, closed-loop maps and their per-thread /
// per-tile compositions
// ---------------------------------------------------------------------------
template <int N, typename S, class Prod, int K>
__global__ void __launch_bounds__(256)
k_filter_down(const __grid_constant__ Prod prod, const S* __restrict__ thr_agg,
              const S* __restrict__ tile_pref, S* __restrict__ Eg, S* __restrict__ thr_aff,
              S* __restrict__ tile_aff, S* __restrict__ filt_out, CombineCtx ctx)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int B = blockDim.x, t = threadIdx.x;
    S* sh = reinterpret_cast<S*>(smem_raw);
    S* pr = sh + Elem<N, S>::NCOMP * 2 * B;
    const long gthr = (long)blockIdx.x * B + t;
    const long k0 = gthr * K;
    const long T = prod.T;

    S rows[K * Prod::W];
    prod.template load<K>(k0, rows);
    {
        Elem<N, S> G;
        aos_load(thr_agg, gthr, G);
        soa_store(sh, 2 * B, t, G);
    }
    elem_tree_up<N, S>(sh, B, t, ctx);
    Red<N, S> pin, X;
    if (t == 0) aos_load(tile_pref, (long)blockIdx.x, pin);
    elem_tree_down<N, S>(sh, pr, B, t, pin, ctx, X);

    Aff<N, S> comp_t;
    set_identity(comp_t);
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const long k = k0 + i;
        if (k < T) {
            if (filt_out) {
#pragma unroll
                for (int c = 0; c < Red<N, S>::NCOMP; ++c)
                    filt_out[k * Red<N, S>::NCOMP + c] = comp(X, c);
            }
            Elem<N, S> e;
            prod.make(k, rows + i * Prod::W, e);
            Aff<N, S> a;
            apply<N, S, true>(e, X, a.F, a.c, ctx);
            aos_store(Eg, k, a);
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
    aos_store(thr_aff, gthr, comp_t);
    __syncthreads();                       // trees above are done with shared memory
    soa_store(sh, 2 * B, t, comp_t);
    aff_tree_up<N, S>(sh, B, t);
    if (t == 0) {
        Aff<N, S> root;
        soa_load(sh, 2 * B, lvl_off(B, ilog2(B)), root);
        aos_store(tile_aff, (long)blockIdx.x, root);
    }
}

// ---------------------------------------------------------------------------
// phase 4: one CTA scans the tile maps backwards from x_T
// ---------------------------------------------------------------------------
template <int N, typename S>
__global__ void __launch_bounds__(256)
k_affine_tiles(const S* __restrict__ tile_aff, int nt, const S* __restrict__ xT,
               S* __restrict__ tile_xend)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int B = blockDim.x, t = threadIdx.x;
    S* sh = reinterpret_cast<S*>(smem_raw);
    S* xs = sh + Aff<N, S>::NCOMP * 2 * B;
    const int per = (nt + B - 1) / B;
    const int first = t * per, last = min(nt, first + per);

    Aff<N, S> H;
    set_identity(H);
    for (int i = last - 1; i >= first; --i) {      // H = a_first o ... o a_last
        Aff<N, S> a;
        aos_load(tile_aff, i, a);
        compose<N, S>(a, H, H);
    }
    soa_store(sh, 2 * B, t, H);
    aff_tree_up<N, S>(sh, B, t);
    S xe[N], x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) xe[i] = xT[i];
    aff_tree_down<N, S>(sh, xs, B, t, xe, x);
    for (int i = last - 1; i >= first; --i) {
#pragma unroll
        for (int j = 0; j < N; ++j) tile_xend[(long)i * N + j] = x[j];
        Aff<N, S> a;
        aos_load(tile_aff, i, a);
        S y[N];
        affine_apply<N, S>(a, x, y);
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] = y[j];
    }
}

// ---------------------------------------------------------------------------
// phase 5: per-step smoothed states x_k = E_k x_{k+1} + g_k
// ---------------------------------------------------------------------------
template <int N, typename S, int K>
__global__ void __launch_bounds__(256)
k_rts_down(const S* __restrict__ Eg, const S* __restrict__ thr_aff,
           const S* __restrict__ tile_xend, long T, S* __restrict__ x_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int B = blockDim.x, t = threadIdx.x;
    S* sh = reinterpret_cast<S*>(smem_raw);
    S* xs = sh + Aff<N, S>::NCOMP * 2 * B;
    const long gthr = (long)blockIdx.x * B + t;
    const long k0 = gthr * K;
    {
        Aff<N, S> a;
        aos_load(thr_aff, gthr, a);
        soa_store(sh, 2 * B, t, a);
    }
    aff_tree_up<N, S>(sh, B, t);
    S xe[N], x[N];
    if (t == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) xe[i] = tile_xend[(long)blockIdx.x * N + i];
    }
    aff_tree_down<N, S>(sh, xs, B, t, xe, x);
#pragma unroll
    for (int i = K - 1; i >= 0; --i) {
        const long k = k0 + i;
        if (k < T) {
            Aff<N, S> a;
            aos_load(Eg, k, a);
            S y[N];
            affine_apply<N, S>(a, x, y);
#pragma unroll
            for (int j = 0; j < N; ++j) { x[j] = y[j]; x_out[k * N + j] = y[j]; }
        }
    }
}

}  // namespace mapk
