// Launch sequences of the solver, templated on the state dimension N, the
// measurement dimension M and the precision S.  Included only by the
// inst_*.cu translation units, which instantiate the combinations compiled
// into the library.
#pragma once
#include <algorithm>
#include <mutex>

#include "handle.h"
#include "scan.cuh"
#include "steptab.cuh"
#include "batch_persist.h"

namespace mapk {

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

inline int ilog2_host(int x)
{
    int l = 0;
    while ((2 << l) <= x) ++l;
    return l;
}

template <int N, typename S>
struct Layout {
    size_t thr_agg, tile_agg, fin, Eg, thr_aff, tile_aff, filt_ws, term, group_agg, trees, total;
    // filt_ws (the forward filter values of the two-filter smoother) only when
    // two_filter; Eg (the closed-loop maps) always (RTS pass, sequential baseline);
    // trees (each tile's up-sweep tree, kept by the reduce kernel for the
    // down-sweep) only when asked (nonlinear models)
    static Layout make(long nthr, long nt, long Tpad, bool two_filter, bool trees = false)
    {
        const long B = nt > 0 ? nthr / nt : 0;
        using E = Elem<N, S>;
        using R = Red<N, S>;
        using A = Aff<N, S>;
        Layout l{};
        size_t o = 0;
        l.thr_agg = o;   o = align_up(o + sizeof(S) * E::NCOMP * nthr);
        l.tile_agg = o;  o = align_up(o + sizeof(S) * E::NCOMP * nt);
        l.fin = o;       o = align_up(o + sizeof(S) * R::NCOMP);
        l.Eg = o;        o = align_up(o + sizeof(S) * A::NCOMP * Tpad);
        l.thr_aff = o;   o = align_up(o + sizeof(S) * A::NCOMP * nthr);
        l.tile_aff = o;  o = align_up(o + sizeof(S) * A::NCOMP * nt);
        l.filt_ws = o;   o = align_up(o + (two_filter ? sizeof(S) * R::NCOMP * Tpad : 0));
        l.term = o;      o = align_up(o + sizeof(S) * R::NCOMP);
        const long ng = B > 0 ? (nt + prefix_group_tiles((int)B) - 1) / prefix_group_tiles((int)B) : 0;
        l.group_agg = o; o = align_up(o + sizeof(S) * E::NCOMP * ng);
        l.trees = o;     o = align_up(o + (trees ? sizeof(S) * 2 * CoopLayout<N, S>::NE * nthr : 0));
        l.total = o;
        return l;
    }
};

// Launch with optional programmatic stream serialisation (see pdl_wait in scan.cuh).
template <typename... KArgs, typename... Args>
inline void launch(void (*k)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, bool pdl,
                   Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

template <typename Kern>
inline cudaError_t allow_smem(Kern k, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

template <int N, typename S>
Red<N, S> prior_of(const map_smoother& h)
{
    Red<N, S> p;
    for (int i = 0; i < N; ++i) p.v[i] = S(h.consts.v0[i]);
    for (int i = 0; i < N; ++i)
        for (int j = i; j < N; ++j) p.P[Sym<N>::at(i, j)] = S(h.consts.S0[i * N + j]);
    return p;
}

template <int N, int M, typename S>
LtiParams<N, M, S> lti_params(const map_smoother& h)
{
    const SetupOut& c = h.consts;
    LtiParams<N, M, S> p;
    for (int i = 0; i < N * N; ++i) p.A[i] = S(c.A[i]);
    for (int i = 0; i < N; ++i) { p.b[i] = S(c.b[i]); p.Gr[i] = S(c.Gr[i]); }
    for (int i = 0; i < N; ++i)
        for (int j = i; j < N; ++j) {
            p.C[Sym<N>::at(i, j)] = S(c.C[i * N + j]);
            p.J[Sym<N>::at(i, j)] = S(c.J[i * N + j]);
        }
    for (int i = 0; i < N * M; ++i) p.G[i] = S(c.G[i]);
    constexpr int R = LtiParams<N, M, S>::R;
    p.lowrank = c.rank <= R;
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < R; ++k) {
            const bool in = k < c.rank && p.lowrank;
            p.Gam[i * R + k] = in ? S(c.Gam[i * N + k]) : S(0);
            p.Gpinv[k * N + i] = in ? S(c.Gpinv[k * N + i]) : S(0);
        }
    return p;
}

template <int N, typename S>
size_t rts_workspace(const map_smoother& h)
{
    return Layout<N, S>::make((long)h.nt * h.B, h.nt, h.Tpad, h.smoother == MAP_TWO_FILTER,
                              h.model != MAP_MODEL_LINEAR).total;
}

// CTAs of B threads of the filter kernels of `Prod` resident on one SM
template <int N, typename S, class Prod>
int rts_resident_blocks(int B)
{
    const size_t big = 200 * 1024;
    if (allow_smem(k_filter_reduce<N, S, Prod>, big) != cudaSuccess ||
        allow_smem(k_filter_down<N, S, Prod>, big) != cudaSuccess)
        return 1;
    int a = 1, b = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_filter_reduce<N, S, Prod>, B, tree_smem<N, S>(B));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &b, k_filter_down<N, S, Prod>, B, std::max(tree_smem<N, S>(B), aff_tree_smem<N, S>(B)));
    return std::max(1, std::min(a, b));
}

// Filter scan + RTS pass for the elements of `prod`; writes x_out (T+1, N).
// Three kernels: reduce (per-thread and per-tile totals), filter down-sweep
// (each CTA reduces the totals before its tile, then per-step values and

// Tile-level pointers of the linear-fold mode (lti_fold.cuh): the tables in
// the fold buffer, w_j in the tile-total area (unused by that mode otherwise)
// and the group maps in the group-total area
template <int N, typename S, class Prod>
LtiTiles<S> lti_tiles_of(const map_smoother& h, const S* fold, S* w, S* gmaps)
{
    LtiTiles<S> lt{};
    if constexpr (Prod::LINEAR_FOLD && N <= 6) {
        if (fold) {
            using TT = TileTables<N, Prod::W, S>;
            const char* base = reinterpret_cast<const char*>(fold);
            lt.fold = fold;
            lt.P = reinterpret_cast<const S*>(base + TT::p_off());
            lt.F = reinterpret_cast<const S*>(base + TT::f_off(h.nt));
            lt.w = w;
            lt.gmaps = gmaps;
            lt.pi = h.nt <= TT::PI_TILES ? reinterpret_cast<const S*>(base + TT::pi_off(h.nt)) : nullptr;
            lt.qt = h.nt <= TT::PI_TILES ? reinterpret_cast<const S*>(base + TT::qt_off(h.nt)) : nullptr;
            // the co table goes to shared memory when three CTAs per SM still fit
            lt.co_smem = LtiDownSmem<N, Prod::W, S>::bytes(h.B, h.K, true) <= 72 * 1024;
        }
    }
    return lt;
}

// closed-loop maps; the last CTA writes x_T), RTS pass (each CTA composes the
// maps after its tile, then the per-step states).  With linear-fold constants
// (fold != nullptr) the reduce kernel covers the full tiles 0..nt-2 on (b, eta)
// parts and the down-sweep's last CTA folds the last tile itself; when all
// tiles fit on the GPU at once the three phases run as one cooperative launch
// (k_lti_solve).
template <int N, typename S, class Prod>
map_status run_rts(map_smoother& h, const Prod& prod, S* x_out, S* filt_out, cudaStream_t st,
                   bool dev_prior = false, const S* fold = nullptr)
{
    using R = Red<N, S>;
    const int B = h.B, nt = h.nt, K = h.K;
    const long nthr = (long)nt * B;
    const bool keep_trees = h.model != MAP_MODEL_LINEAR;
    const Layout<N, S> L = Layout<N, S>::make(nthr, nt, h.Tpad, h.smoother == MAP_TWO_FILTER, keep_trees);
    S* thr_agg = reinterpret_cast<S*>(h.ws + L.thr_agg);
    S* tile_agg = reinterpret_cast<S*>(h.ws + L.tile_agg);
    S* fin = reinterpret_cast<S*>(h.ws + L.fin);
    S* Eg = reinterpret_cast<S*>(h.ws + L.Eg);
    S* thr_aff = reinterpret_cast<S*>(h.ws + L.thr_aff);
    S* tile_aff = reinterpret_cast<S*>(h.ws + L.tile_aff);
    // the reduce kernel keeps each tile's up-sweep tree for the down-sweep
    S* trees = keep_trees ? reinterpret_cast<S*>(h.ws + L.trees) : nullptr;
    const CombineCtx ctx{(float)h.cond_max, h.d_stats};
    const long T = h.T;
    S* xT = x_out + T * N;
    S* filtT = filt_out ? filt_out + T * R::NCOMP : (S*)nullptr;
    const bool lti = fold != nullptr;

    const size_t sh_reduce = tree_smem<N, S>(B);
    size_t sh_down = std::max(tree_smem<N, S>(B), aff_tree_smem<N, S>(B));
    const size_t sh_rts = rts_smem<N, S>(B, K);

    static std::once_flag once;
    cudaError_t e0 = cudaSuccess;
    std::call_once(once, [&] {
        const size_t big = 200 * 1024;
        e0 = allow_smem(k_filter_reduce<N, S, Prod>, big);
        if (e0 == cudaSuccess) e0 = allow_smem(k_filter_down<N, S, Prod>, big);
        if (e0 == cudaSuccess) e0 = allow_smem(k_rts_down<N, S>, big);
        if (e0 == cudaSuccess) e0 = allow_smem(k_group_totals<N, S>, big);
        if (e0 == cudaSuccess) e0 = allow_smem(k_lti_group_maps<N, S>, big);
    });
    if (e0 != cudaSuccess) return cuda_fail(h, e0, "cudaFuncSetAttribute");

    // the down-sweep and the RTS pass overlap their prologues with their
    // predecessor (PDL), except when per-phase events are recorded between them
    h.nev = 0;
    const bool pdl = !h.profile;
    auto mark = [&] { if (h.profile) cudaEventRecord(h.ev[h.nev++], st); };
    mark();
    // dev_prior: the prior comes from the producer's terminal() (device data)
    S* term = dev_prior ? reinterpret_cast<S*>(h.ws + L.term) : nullptr;
    bool first = true;                     // no PDL edge to whatever ran before the solve
    const int G = prefix_group_tiles(B);
    const int ng = (lti ? nt - 1 : nt) > G ? (nt + G - 1) / G : 0;
    S* group_agg = ng ? reinterpret_cast<S*>(h.ws + L.group_agg) : nullptr;
    const LtiTiles<S> lt = lti_tiles_of<N, S, Prod>(h, fold, tile_agg, group_agg);
    EgForm<N, S> form{};                     // how the filter stores the closed-loop maps
    if constexpr (Prod::LOWRANK && !Prod::RESETS) {
        form.compact = prod.p.lowrank;
        for (int i = 0; i < N * N; ++i) form.A[i] = prod.p.A[i];
        for (int i = 0; i < N * EgForm<N, S>::R; ++i) form.Gam[i] = prod.p.Gam[i];
    }
    if constexpr (Prod::LINEAR_FOLD && N <= 6) {
        if (lti) sh_down = LtiDownSmem<N, Prod::W, S>::bytes(B, K, lt.co_smem);
        // single cooperative launch when every tile's CTA can be resident at once
        // (one group of tiles, 16-byte aligned observations, no per-phase events)
        // (not under stream capture: the launch's grid-barrier base would be
        // fixed in the graph, while the arrival counter keeps growing)
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
            cudaGetLastError();
            cap = cudaStreamCaptureStatusActive;
        }
        const bool single = lti && lt.pi && !dev_prior && !h.profile && nt > 1 && nt - 1 <= G &&
                            cap == cudaStreamCaptureStatusNone && (reinterpret_cast<uintptr_t>(prod.y) & 15) == 0;
        if (single) {
            const size_t sh = FusedSmem<N, Prod::W, S>::bytes(B, K);
            if (h.fused < 0) {
                int nb = 0, sms = 0;
                h.fused = allow_smem(k_lti_solve<N, S, Prod>, sh) == cudaSuccess &&
                          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lti_solve<N, S, Prod>, B, sh) ==
                              cudaSuccess &&
                          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h.device) == cudaSuccess &&
                          (long)nb * sms >= nt;
                cudaGetLastError();
            }
            if (h.fused == 1) {
                const GridSync gs{h.d_stats + 3, h.bar_arrivals};
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(nt);
                cfg.blockDim = dim3(B);
                cfg.dynamicSmemBytes = sh;
                cfg.stream = st;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeCooperative;
                at[0].val.cooperative = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                cudaError_t e = cudaLaunchKernelEx(&cfg, k_lti_solve<N, S, Prod>, prod, K, lt, prior_of<N, S>(h),
                                                   Eg, tile_aff, filt_out, ctx, fin, x_out, filtT, form, gs);
                if (e == cudaSuccess) {
                    h.launches += 1;
                    h.path = MAP_PATH_SINGLE;
                    h.bar_arrivals += 2ull * (unsigned long long)nt;   // the launch's two grid barriers
                    return MAP_OK;
                }
                // the grid cannot be resident at once after all (e.g. another
                // context holds part of the GPU): the three-kernel pipeline instead
                cudaGetLastError();
                h.fused = 0;
            }
        }
    }
    if (!lti) {
        launch(k_filter_reduce<N, S, Prod>, nt, B, sh_reduce, st, false, prod, K, thr_agg, tile_agg, term, ctx,
               trees);
        first = false;
    } else if (nt > 1) {
        if constexpr (Prod::LINEAR_FOLD && N <= 6) {
            const size_t sh = LtiReduceSmem<N, Prod::W, S>::bytes(B, K, ilog2_host(B));
            static std::once_flag once_lti;
            cudaError_t e1 = cudaSuccess;
            std::call_once(once_lti, [&] { e1 = allow_smem(k_filter_reduce_lti<N, S, Prod>, 200 * 1024); });
            if (e1 != cudaSuccess) return cuda_fail(h, e1, "cudaFuncSetAttribute");
            launch(k_filter_reduce_lti<N, S, Prod>, nt - 1, B, sh, st, false, prod, K, thr_agg, lt, ctx);
            first = false;
        }
    }
    // scans with more than one group of tiles: group totals (group maps in
    // linear-fold mode) for the two-level tile prefix (the last tile's total
    // is not needed and may be absent)
    if (ng) {
        if (lti)
            launch(k_lti_group_maps<N, S>, ng, B, aff_tree_smem<N, S>(B), st, pdl && !first, lt, nt - 1);
        else
            launch(k_group_totals<N, S>, ng, B, tree_smem<N, S>(B), st, pdl && !first, (const S*)tile_agg, nt,
                   group_agg, ctx);
        first = false;
    }
    mark();
    launch(k_filter_down<N, S, Prod>, nt, B, sh_down, st, pdl && !first, prod, K, thr_agg, (const S*)tile_agg,
           prior_of<N, S>(h), (const S*)term, Eg, thr_aff, tile_aff, filt_out, ctx, lt, fin, xT, filtT,
           (const S*)group_agg, (const S*)trees);
    mark();
    h.launches += (!lti || nt > 1 ? 1 : 0) + (ng ? 1 : 0) + 2;
    h.path = MAP_PATH_PIPELINE;
    launch(k_rts_down<N, S>, nt, B, sh_rts, st, pdl, (const S*)Eg, K, (const S*)thr_aff, (const S*)tile_aff,
           (const S*)xT, T, x_out, form);
    mark();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
    return MAP_OK;
}

// Two-filter smoother (linear models): forward filter scan storing (S_k, v_k),
// backward information-filter scan of the flipped elements in reversed order,
// and the per-step combination x*_k = (S_k + Lam_k)^-1 (v_k + zeta_k).
template <int N, typename S, class Prod, class RProd>
map_status run_tf(map_smoother& h, const Prod& fprod, const RProd& rprod, S* x_out, S* filt_out,
                  cudaStream_t st, const S* fold = nullptr)
{
    using R = Red<N, S>;
    const int K = h.K;
    const int B = h.B, nt = h.nt;
    const long nthr = (long)nt * B;
    const Layout<N, S> L = Layout<N, S>::make(nthr, nt, h.Tpad, h.smoother == MAP_TWO_FILTER);
    S* thr_agg = reinterpret_cast<S*>(h.ws + L.thr_agg);
    S* tile_agg = reinterpret_cast<S*>(h.ws + L.tile_agg);
    S* fin = reinterpret_cast<S*>(h.ws + L.fin);
    S* filt_ws = reinterpret_cast<S*>(h.ws + L.filt_ws);
    S* term = reinterpret_cast<S*>(h.ws + L.term);
    const CombineCtx ctx{(float)h.cond_max, h.d_stats};
    const long T = h.T;
    S* xT = x_out + T * N;
    S* filtT = filt_out ? filt_out + T * R::NCOMP : (S*)nullptr;
    const bool lti = fold != nullptr;          // forward scan in linear-fold mode (see run_rts)
    const size_t sh_tree = tree_smem<N, S>(B);
    size_t sh_states = sh_tree;
    const size_t sh_tfd = std::max(sh_tree, sizeof(S) * (size_t)B * K * N);   // k_tf_down stages the states

    static std::once_flag once;
    cudaError_t e0 = cudaSuccess;
    std::call_once(once, [&] {
        const size_t big = 200 * 1024;
        e0 = allow_smem(k_filter_reduce<N, S, Prod>, big);
        if (e0 == cudaSuccess) e0 = allow_smem(k_filter_reduce<N, S, RProd>, big);
        if (e0 == cudaSuccess) e0 = allow_smem(k_filter_states<N, S, Prod>, big);
        if (e0 == cudaSuccess) e0 = allow_smem(k_tf_down<N, S, RProd>, big);
        if (e0 == cudaSuccess) e0 = allow_smem(k_lti_group_maps<N, S>, big);
    });
    if (e0 != cudaSuccess) return cuda_fail(h, e0, "cudaFuncSetAttribute");

    h.nev = 0;
    const bool pdl = !h.profile;
    auto mark = [&] { if (h.profile) cudaEventRecord(h.ev[h.nev++], st); };
    mark();
    bool first = true;
    // linear-fold mode: tile maps, and group maps when the forward scan has
    // more than one group of tiles (the general forward scan folds all totals)
    const int ng = lti && nt - 1 > prefix_group_tiles(B) ? (nt + prefix_group_tiles(B) - 1) / prefix_group_tiles(B) : 0;
    const LtiTiles<S> lt =
        lti_tiles_of<N, S, Prod>(h, fold, tile_agg, ng ? reinterpret_cast<S*>(h.ws + L.group_agg) : nullptr);
    if constexpr (Prod::LINEAR_FOLD && N <= 6)
        if (lti) sh_states = LtiDownSmem<N, Prod::W, S>::bytes(B, K, lt.co_smem);
    if (!lti) {
        launch(k_filter_reduce<N, S, Prod>, nt, B, sh_tree, st, false, fprod, K, thr_agg, tile_agg, (S*)nullptr,
               ctx, (S*)nullptr);
        first = false;
    } else if (nt > 1) {
        if constexpr (Prod::LINEAR_FOLD && N <= 6) {
            const size_t sh = LtiReduceSmem<N, Prod::W, S>::bytes(B, K, ilog2_host(B));
            static std::once_flag once_lti;
            cudaError_t e1 = cudaSuccess;
            std::call_once(once_lti, [&] { e1 = allow_smem(k_filter_reduce_lti<N, S, Prod>, 200 * 1024); });
            if (e1 != cudaSuccess) return cuda_fail(h, e1, "cudaFuncSetAttribute");
            launch(k_filter_reduce_lti<N, S, Prod>, nt - 1, B, sh, st, false, fprod, K, thr_agg, lt, ctx);
            first = false;
        }
    }
    if (ng) {
        launch(k_lti_group_maps<N, S>, ng, B, aff_tree_smem<N, S>(B), st, pdl && !first, lt, nt - 1);
        first = false;
    }
    mark();
    launch(k_filter_states<N, S, Prod>, nt, B, sh_states, st, pdl && !first, fprod, K, thr_agg,
           (const S*)tile_agg, prior_of<N, S>(h), filt_ws, filt_out, ctx, lt, fin, xT, filtT);
    mark();
    launch(k_filter_reduce<N, S, RProd>, nt, B, sh_tree, st, pdl, rprod, K, thr_agg, tile_agg, term, ctx,
           (S*)nullptr);
    mark();
    h.launches += (!lti || nt > 1 ? 1 : 0) + (ng ? 1 : 0) + 3;
    h.path = MAP_PATH_PIPELINE;
    launch(k_tf_down<N, S, RProd>, nt, B, sh_tfd, st, pdl, rprod, K, (const S*)thr_agg, (const S*)tile_agg,
           (const S*)term, (const S*)filt_ws, x_out, ctx);
    mark();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
    return MAP_OK;
}

// Sequential baseline on the same elements: one thread, time order.
template <int N, typename S, class Prod>
map_status run_sequential(map_smoother& h, const Prod& prod, S* x_out, cudaStream_t st)
{
    const Layout<N, S> L = Layout<N, S>::make((long)h.nt * h.B, h.nt, h.Tpad, h.smoother == MAP_TWO_FILTER);
    S* Eg = reinterpret_cast<S*>(h.ws + L.Eg);
    const CombineCtx ctx{(float)h.cond_max, h.d_stats};
    k_sequential<N, S, Prod><<<1, 32, 0, st>>>(prod, prior_of<N, S>(h), Eg, x_out, ctx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
    return MAP_OK;
}

// ---------------------------------------------------------------------------
// linear models
// ---------------------------------------------------------------------------
template <int N, int M, typename S>
FlipParams<N, M, S> flip_params(const map_smoother& h)
{
    const SetupOut& c = h.consts;
    FlipParams<N, M, S> p;
    for (int i = 0; i < N * N; ++i) p.A[i] = S(c.Phi[i]);
    for (int i = 0; i < N; ++i) { p.b[i] = S(c.beta[i]); p.Gr[i] = S(c.Gr[i]); }
    for (int i = 0; i < N; ++i)
        for (int j = i; j < N; ++j) {
            p.C[Sym<N>::at(i, j)] = S(0.5 * (c.Sigma[i * N + j] + c.Sigma[j * N + i]));
            p.J[Sym<N>::at(i, j)] = S(c.J[i * N + j]);
        }
    for (int i = 0; i < N * M; ++i) p.G[i] = S(c.G[i]);
    return p;
}

// Tiling and tables of the tiled-scan solve (k_lti_scan) once the
// stationary point kc of the step tables is known: J_t tiles of 128 threads x
// K_t steps up to kc, then tiles of 128 x K steps with the smallest K (8..64)
// for which every tile's CTA is resident at once and the tile products fit
// (at most 4 x 128 + 1 tiles).  Sets h.tab_ok when the solve can run.
template <int N, int M, typename S, bool HB>
map_status scan_plan(map_smoother& h, cudaStream_t st)
{
    using ST = StepTab<N, S>;
    using SB = ScanBuf<N, M, S>;
    using TT = TileTables<N, M, S>;
    auto kern = k_lti_scan<N, S, LtiProducer<N, M, S>, HB>;
    h.tab_ok = 0;
    if (!h.d_scan) return MAP_OK;
    constexpr int B = 128, Kt = ST::KT_STEPS;
    const long T = h.T, kc = h.tab_kc, KT = h.tab_kt, Lt = (long)B * Kt;
    const int Jt = (int)((kc + Lt - 1) / Lt);
    if (Jt > SB::jt_max() || ((long)Jt * Lt > KT && (long)Jt * Lt < T)) return MAP_OK;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h.device) != cudaSuccess) {
        cudaGetLastError();
        return MAP_OK;
    }
    int K = 0, nt = 0;
    for (int k = 8; k <= 64 && !K; ++k) {
        const long rest = T - (long)Jt * Lt;
        const long n = rest > 0 ? Jt + (rest + (long)B * k - 1) / ((long)B * k) : (T + Lt - 1) / Lt;
        if (n < 2 || n > SB::NTMAX) continue;
        const size_t sh = ScanSmem<N, M, S>::bytes(B, k, Kt);
        int nb = 0;
        if (allow_smem(kern, sh) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, B, sh) != cudaSuccess) {
            cudaGetLastError();
            return MAP_OK;
        }
        if ((long)nb * sms >= n) {
            K = k;
            nt = (int)n;
        }
    }
    if (!K) return MAP_OK;
    const ScanGeom g{B, K, Kt, Jt, nt};
    const S* rows = reinterpret_cast<const S*>(h.d_tab + ST::rows_off());
    const double* e64 = reinterpret_cast<const double*>(h.d_tab + ST::e64_off(KT));
    const S* mk = reinterpret_cast<const S*>(h.d_tab + ST::mk_off(KT));
    S* pw = reinterpret_cast<S*>(h.d_scan + SB::pw_off());
    S* ttab = reinterpret_cast<S*>(h.d_scan + SB::ttab_off());
    S* gsv = reinterpret_cast<S*>(h.d_scan + SB::gs_off());
    char* tiles = h.d_scan + SB::tiles_off();
    const long kr = std::min(kc, KT - 1);
    // the last tile, when after kc: its partial thread tp and that thread's steps
    const bool last_steady = nt - 1 >= Jt;
    const long rem = T - g.start(nt - 1);
    const int tp = (int)std::min<long>(B, rem / K), nvp = tp < B ? (int)(rem - (long)tp * K) : 0;
    S* taff = reinterpret_cast<S*>(h.d_scan + SB::taff_off());
    k_scan_powers<N, S><<<1, 256, 0, st>>>(e64 + kr * N * N, K, B, pw, tp, nvp,
                                          reinterpret_cast<S*>(h.d_scan + SB::ep_off()),
                                          last_steady ? taff + (long)(nt - 1) * (N * N + N) : nullptr);
    if (Jt > 0) {
        const size_t qsh = sizeof(double) * 2 * 128 * N * N;
        if (cudaError_t e = allow_smem(k_scan_qsuf<N, S>, qsh); e != cudaSuccess) return cuda_fail(h, e, "cudaFuncSetAttribute");
        k_scan_qsuf<N, S><<<Jt, 128, qsh, st>>>(reinterpret_cast<const double*>(h.d_tab + ST::phit64_off(KT)), g,
                                               reinterpret_cast<S*>(h.d_scan + SB::qsuf_off()));
    }
    if (Jt > 0 && ScanSmem<N, M, S>::STAGE) {
        const long cnt = (long)Jt * SB::ttab_rec(B, Kt);
        k_scan_ttab<N, S><<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(
            rows, reinterpret_cast<const S*>(h.d_tab + ST::phit_off(KT)),
            reinterpret_cast<const S*>(h.d_scan + SB::qsuf_off()), KT, g, ttab);
    }
    k_scan_gs<N, M, S><<<1, 32, 0, st>>>(lti_params<N, M, S>(h), mk + kr * N * N, HB ? 1 : 0, gsv);
    {
        // powers M^d (d < nt) of the full-tile map after kc for the tile sums
        double* msq = reinterpret_cast<double*>(h.d_scan + SB::msq_off());
        int nsq = 1;
        while ((1 << nsq) < nt) ++nsq;
        k_scan_msq<N><<<1, 32, 0, st>>>(e64 + kr * N * N, K, B, nsq, msq);
        k_scan_mpow<N, S><<<(unsigned)((nt + 3) / 4), 128, 0, st>>>(msq, nsq, nt,
                                                                  reinterpret_cast<S*>(h.d_scan + SB::mp_off()));
    }
    k_scan_tilemaps<N, M, S><<<(unsigned)(((long)nt * N * N + 127) / 128), 128, 0, st>>>(
        reinterpret_cast<const double*>(h.d_tab + ST::tmap_off()), g, pw, tiles);
    {
        // the tile-map products among the tiles up to Jt (the later ones take powers)
        const int J1 = std::min(Jt, nt - 1), np = (J1 + 1) * (J1 + 2) / 2;
        k_scan_tprod<N, M, S><<<(unsigned)((np + 127) / 128), 128, 0, st>>>(
            nt, J1, tiles, (int)(SB::jt_max() + 1), reinterpret_cast<S*>(h.d_scan + SB::tpi_off()),
            reinterpret_cast<S*>(h.d_scan + SB::tqt_off()));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "scan table kernel launch");
    h.sc_K = K;
    h.sc_Kt = Kt;
    h.sc_Jt = Jt;
    h.sc_nt = nt;
    h.tab_ok = 1;
    return MAP_OK;
}

// whether the stream is being captured into a graph (errors count as capturing)
inline bool capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return cap != cudaStreamCaptureStatusNone;
}

// the sample's share of the element offset (b_k = Bb y_k + b0) of block and
// exact elements; off for per-step elements
template <int N, int M>
SampleOffset<N, M> sample_offset(const map_smoother& h)
{
    SampleOffset<N, M> so{};
    so.on = h.disc >= MAP_BLOCK_EULER;
    for (int i = 0; i < N * M; ++i) so.Bb[i] = so.on ? h.consts.Bb[i] : 0.0;
    return so;
}

// Per-step tables (steptab.cuh) of an RTS solve of a linear time-invariant
// model and the tiled-scan plan, computed once per model (they depend on the
// model constants and T only): the element powers, every step's row, the
// stationary point kc (read back: a synchronisation, so never under stream
// capture), then the scan tables.  h.tab_ok tells whether the tiled scan can
// run; otherwise the solve keeps the other paths.
template <int N, int M, typename S, bool HB>
map_status table_plan(map_smoother& h, cudaStream_t st)
{
    using ST = StepTab<N, S>;
    if (!h.d_tab || h.tab_state || h.smoother != MAP_RTS || capturing(st)) return MAP_OK;
    h.tab_ok = 0;
    h.tab_state = 1;
    // rows of the steps k < KT; with T >= KT the convergence point kc, from
    // which row kc stands for every later step, must leave room for the
    // thread maps of the threads that reach it
    const long KT = std::min<long>(h.T + 1, ST::cap());
    const int check = h.T + 1 > KT;
    const double tol = sizeof(S) == 4 ? 0x1p-25 : 1e-12;
    unsigned long long meta[2] = {0, 0};
    cudaError_t e;
    if ((e = cudaMemsetAsync(h.d_tab, 0, sizeof(meta), st)) != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
    k_step_powers<N, M, S><<<1, 32, 0, st>>>(lti_params<N, M, double>(h), prior_of<N, double>(h), h.T, KT, h.d_tab);
    k_step_small<N, S><<<ST::SMALL / 4, 128, 0, st>>>(h.d_tab);
    const long nb = ST::base_count(KT);
    k_step_base<N, S><<<(unsigned)((nb + 3) / 4), 128, 0, st>>>(prior_of<N, double>(h), KT, h.d_tab);
    k_lti_steptab<N, M, S><<<(unsigned)((KT + 127) / 128), 128, 0, st>>>(
        lti_params<N, M, double>(h), KT, check, tol, sample_offset<N, M>(h), h.d_tab);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "step table kernel launch");
    if ((e = cudaMemcpyAsync(meta, h.d_tab, sizeof(meta), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(h, e, "step table read-back");
    const long kc = check ? (long)meta[0] : h.T;
    h.tab_conv = 0;
    if (meta[1] != 0 || (check && kc + 1 >= KT)) return MAP_OK;
    h.tab_kt = KT;
    h.tab_kc = kc;
    // E_inf (FP64, row kc) for the plan-time products of the solve's steady steps
    if ((e = cudaMemcpy(h.tab_einf, reinterpret_cast<const double*>(h.d_tab + ST::e64_off(KT)) + std::min(kc, KT - 1) * N * N,
                        sizeof(double) * N * N, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(h, e, "step table read-back");
    h.tab_conv = 1;
    return scan_plan<N, M, S, HB>(h, st);
}

// The tiled-scan solve (one cooperative launch) when its tables are ready;
// *ran is false when the other paths must run.
template <int N, int M, typename S, bool HB>
map_status run_scan(map_smoother& h, const LtiProducer<N, M, S>& prod, S* x_out, S* filt_out, cudaStream_t st,
                    bool* ran)
{
    using ST = StepTab<N, S>;
    using SB = ScanBuf<N, M, S>;
    using TT = TileTables<N, M, S>;
    using R = Red<N, S>;
    *ran = false;
    if (map_status s = table_plan<N, M, S, HB>(h, st); s != MAP_OK) return s;
    if (!h.tab_ok || h.profile || capturing(st)) return MAP_OK;
    if (ScanSmem<N, M, S>::STAGE && (reinterpret_cast<uintptr_t>(prod.y) & 15) != 0) return MAP_OK;
    constexpr int B = 128;
    const int snt = h.sc_nt;
    const long KT = h.tab_kt;
    ScanArgs<N, M, S> sa{};
    sa.g = ScanGeom{B, h.sc_K, h.sc_Kt, h.sc_Jt, snt};
    sa.rows = reinterpret_cast<const S*>(h.d_tab + ST::rows_off());
    sa.kc = h.tab_kc;
    sa.phit = reinterpret_cast<const S*>(h.d_tab + ST::phit_off(KT));
    sa.mk = reinterpret_cast<const S*>(h.d_tab + ST::mk_off(KT));
    sa.pw = reinterpret_cast<const S*>(h.d_scan + SB::pw_off());
    sa.ttab = reinterpret_cast<const S*>(h.d_scan + SB::ttab_off());
    sa.w = reinterpret_cast<S*>(h.d_scan + SB::w_off());
    sa.taff = reinterpret_cast<S*>(h.d_scan + SB::taff_off());
    sa.gs = reinterpret_cast<const S*>(h.d_scan + SB::gs_off());
    sa.ep = reinterpret_cast<const S*>(h.d_scan + SB::ep_off());
    sa.qsuf = reinterpret_cast<const S*>(h.d_scan + SB::qsuf_off());
    sa.mp = reinterpret_cast<const S*>(h.d_scan + SB::mp_off());
    sa.pinv = reinterpret_cast<const double*>(h.d_tab + ST::pinv_off());
    const char* tiles = h.d_scan + SB::tiles_off();
    sa.pi = reinterpret_cast<const S*>(h.d_scan + SB::tpi_off());
    sa.qt = reinterpret_cast<const S*>(h.d_scan + SB::tqt_off());
    sa.tld = (int)(SB::jt_max() + 1);
    const SetupOut& c = h.consts;
    sa.has_b = 0;
    for (int i = 0; i < N; ++i) sa.has_b |= c.b[i] != 0.0;
    for (int i = 0; i < N; ++i) {
        double ab = 0.0;
        for (int k = 0; k < N; ++k) ab += c.Phi[i * N + k] * c.b[k];
        sa.Aib[i] = S(ab);
        for (int j = 0; j < N; ++j) {
            double ac = 0.0;
            for (int k = 0; k < N; ++k) ac += c.Phi[i * N + k] * c.C[k * N + j];
            sa.AiC[i * N + j] = S(ac);
        }
        for (int j = 0; j < M; ++j) {
            double ab2 = 0.0;
            if (HB)
                for (int k = 0; k < N; ++k) ab2 += c.Phi[i * N + k] * c.Bb[k * M + j];
            sa.AiBb[i * M + j] = S(ab2);
        }
    }
    {
        // E_inf times those, with E_inf the FP64 closed-loop map of row kc
        const double* Einf = h.tab_einf;
        double AiC[N * N], Aib[N], AiBb[N * M];
        for (int i = 0; i < N; ++i) {
            double ab = 0.0;
            for (int k = 0; k < N; ++k) ab += c.Phi[i * N + k] * c.b[k];
            Aib[i] = ab;
            for (int j = 0; j < N; ++j) {
                double ac = 0.0;
                for (int k = 0; k < N; ++k) ac += c.Phi[i * N + k] * c.C[k * N + j];
                AiC[i * N + j] = ac;
            }
            for (int j = 0; j < M; ++j) {
                double ab2 = 0.0;
                if (HB)
                    for (int k = 0; k < N; ++k) ab2 += c.Phi[i * N + k] * c.Bb[k * M + j];
                AiBb[i * M + j] = ab2;
            }
        }
        for (int i = 0; i < N; ++i) {
            double eb = 0.0;
            for (int k = 0; k < N; ++k) eb += Einf[i * N + k] * Aib[k];
            sa.EAib[i] = S(eb);
            for (int j = 0; j < N; ++j) {
                double ec = 0.0;
                for (int k = 0; k < N; ++k) ec += Einf[i * N + k] * AiC[k * N + j];
                sa.EAiC[i * N + j] = S(ec);
            }
            for (int j = 0; j < M; ++j) {
                double eb2 = 0.0;
                for (int k = 0; k < N; ++k) eb2 += Einf[i * N + k] * AiBb[k * M + j];
                sa.EAiBb[i * M + j] = S(eb2);
            }
        }
    }
    const CombineCtx ctx{(float)h.cond_max, h.d_stats};
    const Layout<N, S> L = Layout<N, S>::make((long)h.nt * h.B, h.nt, h.Tpad, false);
    S* fin = reinterpret_cast<S*>(h.ws + L.fin);
    S* filtT = filt_out ? filt_out + h.T * R::NCOMP : (S*)nullptr;
    const GridSync gs{h.d_stats + EV_BARRIER, h.bar_arrivals};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(snt);
    cfg.blockDim = dim3(B);
    cfg.dynamicSmemBytes = ScanSmem<N, M, S>::bytes(B, h.sc_K, h.sc_Kt);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_lti_scan<N, S, LtiProducer<N, M, S>, HB>, prod, prior_of<N, S>(h),
                                       filt_out, ctx, fin, x_out, filtT, gs, sa);
    if (e != cudaSuccess) {
        // the grid cannot be resident at once after all: the other paths
        cudaGetLastError();
        h.tab_ok = 0;
        return MAP_OK;
    }
    h.launches += 1;
    h.path = MAP_PATH_TABLES;
    h.bar_arrivals += 2ull * (unsigned long long)snt;
    *ran = true;
    return MAP_OK;
}

// constants of the linear per-thread fold and the tile tables (lti_fold.cuh)
// for the current geometry, recomputed on `st` after a change of K, B or of
// the model; nullptr when the geometry is beyond their range (the kernels then
// fold step by step and combine tile totals)
template <int N, int M, typename S>
map_status lti_fold_consts(map_smoother& h, cudaStream_t st, const S** out)
{
    using FL = FoldLayout<N, M, S>;
    *out = nullptr;
    if constexpr (N > 6) return MAP_OK;        // the kernels take the linear fold for N <= 6
    int LB = 0;
    while ((2 << LB) <= h.B) ++LB;
    using TT = TileTables<N, M, S>;
    int ne = 1;                                // tile levels: 2^ne > nt - 1, the largest tile index
    while (ne < 31 && (1L << ne) <= (long)h.nt - 1) ++ne;
    if (!h.d_fold || h.K > FL::KMAX || LB > FL::LMAX || ne > TT::ELMAX ||
        TT::bytes(h.nt) > fold_bytes(N, M, sizeof(S), h.nt) ||
        LtiDownSmem<N, M, S>::bytes(h.B, h.K, false) > 200 * 1024 ||
        LtiReduceSmem<N, M, S>::bytes(h.B, h.K, LB) > 200 * 1024)
        return MAP_OK;
    if (h.fold_K != h.K || h.fold_B != h.B) {
        // one warp for the serial FP64 chains, then one warp per thread
        // prefix and per tile in one launch, four to a block so that they
        // spread over the SMs' FP64 pipes
        k_lti_fold<N, M, S><<<1, 32, 0, st>>>(lti_params<N, M, double>(h), h.K, LB, ne, static_cast<S*>(h.d_fold));
        k_lti_tables<N, M, S><<<((1 << LB) + 3) / 4 + (h.nt + 3) / 4, 128, 0, st>>>(
            prior_of<N, double>(h), LB, h.nt, ne, static_cast<S*>(h.d_fold));
        if (h.nt <= TT::PI_TILES) {
            const int segs = (h.nt + TT::PI_SEG - 1) / TT::PI_SEG;
            k_lti_segments<N, M, S><<<(h.nt + 127) / 128, 128, 0, st>>>(h.nt, static_cast<S*>(h.d_fold));
            k_lti_products<N, M, S><<<dim3((segs + 7) / 8, (h.nt + 3) / 4), 32, 0, st>>>(
                h.nt, static_cast<S*>(h.d_fold));
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(h, e, "fold constants kernel launch");
        h.fold_K = h.K;
        h.fold_B = h.B;
    }
    *out = static_cast<const S*>(h.d_fold);
    return MAP_OK;
}

// Two-filter smoother of a linear model (its own function so that the build
// can compile it in a separate translation unit, see inst_linear.cu)
template <int N, int M, typename S>
map_status solve_linear_tf(map_smoother& h, const void* y, void* x_out, void* filt_out, cudaStream_t st,
                           const S* fold)
{
    LtiProducer<N, M, S> prod;
    prod.y = static_cast<const S*>(y);
    prod.T = h.T;
    prod.p = lti_params<N, M, S>(h);
    RevFlipProducer<N, M, S> rprod;
    rprod.y = static_cast<const S*>(y);
    rprod.T = h.T;
    rprod.Tpad = h.Tpad;
    rprod.p = flip_params<N, M, S>(h);
    return run_tf<N, S>(h, prod, rprod, static_cast<S*>(x_out), static_cast<S*>(filt_out), st, fold);
}

// ---------------------------------------------------------------------------
// block and exact elements (MAP_BLOCK_EULER, MAP_RICCATI_EXACT): both offsets
// of the element depend on the interval's sample (BlockProducer), so they take
// the general combine path; dense output between the grid points
// ---------------------------------------------------------------------------
template <int N, int M, typename S>
BlockParams<N, M, S> block_params(const map_smoother& h)
{
    const SetupOut& c = h.consts;
    BlockParams<N, M, S> p;
    for (int i = 0; i < N * N; ++i) p.A[i] = S(c.A[i]);
    for (int i = 0; i < N; ++i) { p.b0[i] = S(c.b[i]); p.Gr[i] = S(c.Gr[i]); }
    for (int i = 0; i < N; ++i)
        for (int j = i; j < N; ++j) {
            p.C[Sym<N>::at(i, j)] = S(c.C[i * N + j]);
            p.J[Sym<N>::at(i, j)] = S(c.J[i * N + j]);
        }
    for (int i = 0; i < N * M; ++i) { p.Bb[i] = S(c.Bb[i]); p.G[i] = S(c.G[i]); }
    return p;
}

template <int N, int M, typename S>
map_status solve_linear_block(map_smoother& h, const void* y, void* x_out, void* filt_out, cudaStream_t st,
                              bool sequential)
{
    BlockProducer<N, M, S> prod;
    prod.y = static_cast<const S*>(y);
    prod.T = h.T;
    prod.p = block_params<N, M, S>(h);
    if (sequential) return run_sequential<N, S>(h, prod, static_cast<S*>(x_out), st);
    // A, C and J are the same for every interval: the tiled scan with the
    // per-step tables, with the sample's share of the offset
    LtiProducer<N, M, S> lp;
    lp.y = prod.y;
    lp.T = h.T;
    lp.p = lti_params<N, M, S>(h);
    bool ran = false;
    if (map_status s = run_scan<N, M, S, true>(h, lp, static_cast<S*>(x_out), static_cast<S*>(filt_out), st, &ran);
        s != MAP_OK || ran)
        return s;
    return run_rts<N, S>(h, prod, static_cast<S*>(x_out), static_cast<S*>(filt_out), st);
}

// one substep element of a block (dense output)
template <int N, int M, typename S>
struct SubParams {
    S A[N * N];
    S b[N];
    S C[Sym<N>::SZ];
    S J[Sym<N>::SZ];
    S G[N * M];
    S Gr[N];
};

// Dense output (Section 4.3 recovery between grid points), one thread per
// interval k: the filter value function at x_k (filt row k) is carried across
// the interval's substeps by the one-variable combine (Eq. 36, `apply`), whose
// closed-loop maps (Eq. 40-41) are kept in shared memory (ns of them per
// thread); then x_{k+1} is taken back through them.  Row k ns + j of out is
// the state at t_k + j dt / ns; row T ns is x_T.
template <int N, int M, typename S>
__global__ void __launch_bounds__(64)
k_dense_block(const S* __restrict__ y, const S* __restrict__ x, const S* __restrict__ filt, long T, int ns,
              const SubParams<N, M, S> p, S* __restrict__ out, CombineCtx ctx)
{
    constexpr int NN = N * N, NA = NN + N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* my = reinterpret_cast<S*>(smem_raw) + (long)threadIdx.x * ns * NA;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= T) return;
    Red<N, S> X;
#pragma unroll
    for (int q = 0; q < Red<N, S>::NCOMP; ++q) comp(X, q) = filt[k * Red<N, S>::NCOMP + q];
    Elem<N, S> e;
#pragma unroll
    for (int q = 0; q < NN; ++q) e.A[q] = p.A[q];
#pragma unroll
    for (int q = 0; q < Sym<N>::SZ; ++q) { e.C[q] = p.C[q]; e.J[q] = p.J[q]; }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        S se = -p.Gr[i];
#pragma unroll
        for (int j = 0; j < M; ++j) se = fma(p.G[i * M + j], y[k * M + j], se);
        e.b[i] = p.b[i];
        e.eta[i] = se;
    }
#pragma unroll 1
    for (int j = 0; j < ns; ++j) {
        S E[NN], g[N];
        apply<N, S, true>(e, X, E, g, ctx);
#pragma unroll
        for (int q = 0; q < NN; ++q) my[j * NA + q] = E[q];
#pragma unroll
        for (int q = 0; q < N; ++q) my[j * NA + NN + q] = g[q];
    }
    S z[N];
#pragma unroll
    for (int a = 0; a < N; ++a) z[a] = x[(k + 1) * N + a];
    // substep 0 is the grid point itself: its row is x_k as the solve gave it
#pragma unroll
    for (int a = 0; a < N; ++a) out[k * ns * N + a] = x[k * N + a];
#pragma unroll 1
    for (int j = ns - 1; j >= 1; --j) {
        S nz[N];
#pragma unroll
        for (int a = 0; a < N; ++a) {
            S acc = my[j * NA + NN + a];
#pragma unroll
            for (int q = 0; q < N; ++q) acc = fma(my[j * NA + a * N + q], z[q], acc);
            nz[a] = acc;
        }
#pragma unroll
        for (int a = 0; a < N; ++a) {
            z[a] = nz[a];
            out[(k * ns + j) * N + a] = nz[a];
        }
    }
    if (k == T - 1)
#pragma unroll
        for (int a = 0; a < N; ++a) out[T * ns * N + a] = x[T * N + a];
}

template <int N, int M, typename S>
map_status dense_linear(map_smoother& h, const void* y, const void* x, const void* filt, void* out, cudaStream_t st)
{
    if (h.disc != MAP_BLOCK_EULER) return fail(h, MAP_ERR_UNSUPPORTED, "dense output needs MAP_BLOCK_EULER elements");
    const SetupOut& c = h.consts;
    SubParams<N, M, S> p;
    for (int i = 0; i < N * N; ++i) p.A[i] = S(c.sA[i]);
    for (int i = 0; i < N; ++i) { p.b[i] = S(c.sb[i]); p.Gr[i] = S(c.sGr[i]); }
    for (int i = 0; i < N; ++i)
        for (int j = i; j < N; ++j) {
            p.C[Sym<N>::at(i, j)] = S(c.sC[i * N + j]);
            p.J[Sym<N>::at(i, j)] = S(c.sJ[i * N + j]);
        }
    for (int i = 0; i < N * M; ++i) p.G[i] = S(c.sG[i]);
    const int ns = h.substeps;
    const size_t per = sizeof(S) * (size_t)ns * (N * N + N);
    int threads = (int)std::min<size_t>(64, (200 * 1024) / per);
    if (threads < 1) return fail(h, MAP_ERR_SHAPE, "too many substeps for the dense output");
    const size_t sh = per * threads;
    cudaError_t e = allow_smem(k_dense_block<N, M, S>, sh);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaFuncSetAttribute");
    const CombineCtx ctx{(float)h.cond_max, h.d_stats};
    k_dense_block<N, M, S><<<(unsigned)((h.T + threads - 1) / threads), threads, sh, st>>>(
        static_cast<const S*>(y), static_cast<const S*>(x), static_cast<const S*>(filt), h.T, ns, p,
        static_cast<S*>(out), ctx);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "dense output kernel launch");
    return MAP_OK;
}

template <int N, int M, typename S>
map_status solve_linear(map_smoother& h, const void* y, void* x_out, void* filt_out, cudaStream_t st)
{
    if constexpr (N <= 6)
        if (h.disc >= MAP_BLOCK_EULER) return solve_linear_block<N, M, S>(h, y, x_out, filt_out, st, false);
    LtiProducer<N, M, S> prod;
    prod.y = static_cast<const S*>(y);
    prod.T = h.T;
    prod.p = lti_params<N, M, S>(h);
    if (h.smoother == MAP_RTS) {
        bool ran = false;
        if (map_status s = run_scan<N, M, S, false>(h, prod, static_cast<S*>(x_out), static_cast<S*>(filt_out), st,
                                                   &ran);
            s != MAP_OK || ran)
            return s;
    }
    const S* fold = nullptr;
    if (map_status s = lti_fold_consts<N, M, S>(h, st, &fold); s != MAP_OK) return s;
    if constexpr (N <= 6) if (h.smoother == MAP_TWO_FILTER) return solve_linear_tf<N, M, S>(h, y, x_out, filt_out, st, fold);
    return run_rts<N, S>(h, prod, static_cast<S*>(x_out), static_cast<S*>(filt_out), st, false, fold);
}

template <int N, int M, typename S>
map_status solve_linear_sequential(map_smoother& h, const void* y, void* x_out, cudaStream_t st)
{
    if constexpr (N <= 6)
        if (h.disc >= MAP_BLOCK_EULER) return solve_linear_block<N, M, S>(h, y, x_out, nullptr, st, true);
    LtiProducer<N, M, S> prod;
    prod.y = static_cast<const S*>(y);
    prod.T = h.T;
    prod.p = lti_params<N, M, S>(h);
    return run_sequential<N, S>(h, prod, static_cast<S*>(x_out), st);
}

// Many trajectories of one linear model concatenated with reset elements
// (SegLtiProducer).
template <int N, int M, typename S>
map_status solve_linear_seg(map_smoother& h, const void* y, const unsigned char* reset, void* x_out,
                            cudaStream_t st)
{
    SegLtiProducer<N, M, S> prod;
    prod.y = static_cast<const S*>(y);
    prod.reset = reset;
    prod.T = h.T;
    prod.p = lti_params<N, M, S>(h);
    for (int i = 0; i < N; ++i) {
        prod.v0[i] = S(h.consts.v0[i]);
        for (int j = i; j < N; ++j) prod.S0[Sym<N>::at(i, j)] = S(h.consts.S0[i * N + j]);
    }
    return run_rts<N, S>(h, prod, static_cast<S*>(x_out), nullptr, st);
}

// Discrete Onsager-Machlup cost of a trajectory of a linear model:
//   1/2 |x0 - m0|^2_{P0^-1} + sum_k 1/2 |x_k - A x_{k+1} - b|^2_{C^-1}
//   + sum_k 1/2 dt |y_{k+1} - H x_{k+1} - r|^2_{R^-1} + 1/2 dt T tr F
// (C^-1 = Q^-1 / dt for the Euler element).  FP64 accumulation.
template <int N, int M, typename S>
__global__ void k_cost_linear(const S* __restrict__ y, const S* __restrict__ x, long T,
                              LinCostParams<N, M> p, double* out)
{
    double acc = 0.0;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < T; k += (long)gridDim.x * blockDim.x) {
        double xk[N], x1[N], rr[N], e[M];
#pragma unroll
        for (int i = 0; i < N; ++i) { xk[i] = double(x[k * N + i]); x1[i] = double(x[(k + 1) * N + i]); }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = xk[i] - p.b[i];
#pragma unroll
            for (int j = 0; j < N; ++j) s -= p.A[i * N + j] * x1[j];
            rr[i] = s;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
#pragma unroll
            for (int j = 0; j < N; ++j) s += p.Cinv[i * N + j] * rr[j];
            acc += 0.5 * rr[i] * s;
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
            double s = double(y[k * M + i]) - p.r[i];
#pragma unroll
            for (int j = 0; j < N; ++j) s -= p.H[i * N + j] * x1[j];
            e[i] = s;
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
            double s = 0.0;
#pragma unroll
            for (int j = 0; j < M; ++j) s += p.Rinv[i * M + j] * e[j];
            acc += 0.5 * p.dt * e[i] * s;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double e0[N];
#pragma unroll
        for (int i = 0; i < N; ++i) e0[i] = double(x[i]) - p.m0[i];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
#pragma unroll
            for (int j = 0; j < N; ++j) s += p.S0[i * N + j] * e0[j];
            acc += 0.5 * e0[i] * s;
        }
        acc += 0.5 * p.dt * double(T) * p.trF;
    }
    // warp + block reduction, one atomic per block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(out, acc);
    }
}

template <int N, int M, typename S>
map_status cost_linear(map_smoother& h, const void* y, const void* x, double* d_cost, cudaStream_t st)
{
    LinCostParams<N, M> p;
    const SetupOut& c = h.consts;
    for (int i = 0; i < N * N; ++i) { p.A[i] = c.A[i]; p.S0[i] = c.S0[i]; p.Cinv[i] = c.Cinv[i]; }
    for (int i = 0; i < N; ++i) { p.b[i] = c.b[i]; p.m0[i] = h.m0[i]; }
    for (int i = 0; i < M * N; ++i) p.H[i] = h.H[i];
    for (int i = 0; i < M; ++i) p.r[i] = h.r[i];
    for (int i = 0; i < M * M; ++i) p.Rinv[i] = c.Rinv[i];
    p.dt = h.dt;
    p.trF = 0.0;
    for (int i = 0; i < N; ++i) p.trF += h.F[i * N + i];
    for (int i = 0; i < N * N; ++i) p.IA[i] = (i % (N + 1) == 0 ? 1.0 : 0.0) - c.A[i];
    cudaError_t e = cudaMemsetAsync(d_cost, 0, sizeof(double), st);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
    const int blocks = (int)std::min<long>(1024, (h.T + 255) / 256);
    k_cost_linear<N, M, S><<<std::max(blocks, 1), 256, 0, st>>>(static_cast<const S*>(y),
                                                                static_cast<const S*>(x), h.T, p, d_cost);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "cost kernel launch");
    return MAP_OK;
}

// ---------------------------------------------------------------------------
// gradient of a loss of the MAP trajectory w.r.t. theta = (F, log q, log r)
// (Euler elements: A = I - dt F, C = dt q Q0, R = r R0)
//  - MAP cost (envelope): d/dF = sum dt (C^-1 r_k) x_{k+1}^T + 1/2 dt T I,
//    d/dlogq = -1/2 sum r^T C^-1 r, d/dlogr = -1/2 sum dt e^T R^-1 e
//  - other losses: -d_theta [lambda^T grad_x M] at fixed x*, lambda:
//    d/dF = -sum dt ((C^-1 r) lambda_{k+1}^T + (C^-1 s) x_{k+1}^T),
//    d/dlogq = sum s^T C^-1 r, d/dlogr = sum dt (H lambda_{k+1})^T R^-1 e
// with r_k = x_k - A x_{k+1} - b, s_k = lambda_k - A lambda_{k+1},
// e_k = H x_{k+1} + r - y_{k+1}.  Per-step terms in S, FP64 accumulation.
// The residuals are formed as (x_k - x_{k+1}) + (I - A) x_{k+1} - b with
// I - A = dt F kept apart from the identity: A = I - dt F rounded to FP32
// would carry an error of one FP32 ulp of 1 in every step's residual, the same
// in every step, which the sum over T steps turns into a systematic error of
// dL/dF of order ulp(1) T |x|^2 / q.
// ---------------------------------------------------------------------------
template <int N, int M, typename S>
__global__ void __launch_bounds__(256)
k_grad_contract(const S* __restrict__ y, const S* __restrict__ x, const S* __restrict__ lam, long T,
                LinCostParams<N, M> p, double* __restrict__ out)
{
    constexpr int NG = N * N + 2;
    double acc[NG];
#pragma unroll
    for (int i = 0; i < NG; ++i) acc[i] = 0.0;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < T; k += (long)gridDim.x * blockDim.x) {
        S xk[N], x1[N], r[N], Cr[N], e[M], Re[M];
#pragma unroll
        for (int i = 0; i < N; ++i) { xk[i] = x[k * N + i]; x1[i] = x[(k + 1) * N + i]; }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S s = (xk[i] - x1[i]) - S(p.b[i]);
#pragma unroll
            for (int j = 0; j < N; ++j) s = fma(S(p.IA[i * N + j]), x1[j], s);
            r[i] = s;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S s = S(0);
#pragma unroll
            for (int j = 0; j < N; ++j) s = fma(S(p.Cinv[i * N + j]), r[j], s);
            Cr[i] = s;
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
            S s = S(p.r[i]) - y[k * M + i];
#pragma unroll
            for (int j = 0; j < N; ++j) s = fma(S(p.H[i * N + j]), x1[j], s);
            e[i] = s;
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
            S s = S(0);
#pragma unroll
            for (int j = 0; j < M; ++j) s = fma(S(p.Rinv[i * M + j]), e[j], s);
            Re[i] = s;
        }
        if (lam) {
            S lk[N], l1[N], sv[N], Cs[N], Hl[M];
#pragma unroll
            for (int i = 0; i < N; ++i) { lk[i] = lam[k * N + i]; l1[i] = lam[(k + 1) * N + i]; }
#pragma unroll
            for (int i = 0; i < N; ++i) {
                S s = lk[i] - l1[i];
#pragma unroll
                for (int j = 0; j < N; ++j) s = fma(S(p.IA[i * N + j]), l1[j], s);
                sv[i] = s;
            }
#pragma unroll
            for (int i = 0; i < N; ++i) {
                S s = S(0);
#pragma unroll
                for (int j = 0; j < N; ++j) s = fma(S(p.Cinv[i * N + j]), sv[j], s);
                Cs[i] = s;
            }
#pragma unroll
            for (int i = 0; i < M; ++i) {
                S s = S(0);
#pragma unroll
                for (int j = 0; j < N; ++j) s = fma(S(p.H[i * N + j]), l1[j], s);
                Hl[i] = s;
            }
#pragma unroll
            for (int a = 0; a < N; ++a)
#pragma unroll
                for (int b = 0; b < N; ++b)
                    acc[a * N + b] -= p.dt * double(Cr[a] * l1[b] + Cs[a] * x1[b]);
            S q = S(0), w = S(0);
#pragma unroll
            for (int i = 0; i < N; ++i) q = fma(sv[i], Cr[i], q);
#pragma unroll
            for (int i = 0; i < M; ++i) w = fma(Hl[i], Re[i], w);
            acc[N * N] += double(q);
            acc[N * N + 1] += p.dt * double(w);
        } else {
#pragma unroll
            for (int a = 0; a < N; ++a)
#pragma unroll
                for (int b = 0; b < N; ++b) acc[a * N + b] += p.dt * double(Cr[a] * x1[b]);
            S q = S(0), w = S(0);
#pragma unroll
            for (int i = 0; i < N; ++i) q = fma(r[i], Cr[i], q);
#pragma unroll
            for (int i = 0; i < M; ++i) w = fma(e[i], Re[i], w);
            acc[N * N] -= 0.5 * double(q);
            acc[N * N + 1] -= 0.5 * p.dt * double(w);
        }
    }
    __shared__ double part[NG][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        double v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) part[i][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < NG) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += part[threadIdx.x][w];
        atomicAdd(out + threadIdx.x, v);
    }
}

template <int N, int M, typename S>
map_status grad_linear(map_smoother& h, const void* y, const void* x, const void* dLdx, int flags,
                       double* dtheta, cudaStream_t st)
{
    LinCostParams<N, M> p;
    const SetupOut& c = h.consts;
    for (int i = 0; i < N * N; ++i) { p.A[i] = c.A[i]; p.S0[i] = c.S0[i]; p.Cinv[i] = c.Cinv[i]; }
    for (int i = 0; i < N; ++i) { p.b[i] = c.b[i]; p.m0[i] = h.m0[i]; }
    for (int i = 0; i < M * N; ++i) p.H[i] = h.H[i];
    for (int i = 0; i < M; ++i) p.r[i] = h.r[i];
    for (int i = 0; i < M * M; ++i) p.Rinv[i] = c.Rinv[i];
    p.dt = h.dt;
    p.trF = 0.0;
    for (int i = 0; i < N * N; ++i) p.IA[i] = h.dt * h.F[i];     // Euler element: I - A = dt F
    S* lam = nullptr;
    if (dLdx) {
        AdjProducer<N, S> prod;
        prod.d = static_cast<const S*>(dLdx);
        prod.T = h.T;
        for (int i = 0; i < N * N; ++i) prod.p.A[i] = S(c.A[i]);
        for (int i = 0; i < N; ++i)
            for (int j = i; j < N; ++j) {
                prod.p.C[Sym<N>::at(i, j)] = S(c.C[i * N + j]);
                prod.p.J[Sym<N>::at(i, j)] = S(c.J[i * N + j]);
                prod.p.S0[Sym<N>::at(i, j)] = S(c.S0[i * N + j]);
            }
        lam = static_cast<S*>(h.d_lam);
        map_status s = run_rts<N, S>(h, prod, lam, nullptr, st, true);
        if (s != MAP_OK) return s;
    }
    constexpr int NG = N * N + 2;
    cudaError_t e = cudaMemsetAsync(h.d_grad, 0, sizeof(double) * NG, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
    const int blocks = (int)std::max<long>(1, std::min<long>(2048, (h.T + 255) / 256));
    k_grad_contract<N, M, S><<<blocks, 256, 0, st>>>(static_cast<const S*>(y), static_cast<const S*>(x),
                                                     lam, h.T, p, h.d_grad);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "gradient kernel launch");
    double g[NG];
    if ((e = cudaMemcpyAsync(g, h.d_grad, sizeof(double) * NG, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(h, e, "gradient read-back");
    if (!dLdx) {
        for (int a = 0; a < N; ++a) g[a * N + a] += 0.5 * h.dt * double(h.T);   // divergence tr F
        if (flags & 1) {                                                        // log-normalisers
            g[N * N] += 0.5 * N * double(h.T);
            g[N * N + 1] += 0.5 * M * double(h.T);
        }
    }
    for (int i = 0; i < NG; ++i) dtheta[i] = g[i];
    return MAP_OK;
}

// bytes of the per-step tables of an RTS solve (steptab.cuh)
template <int N, typename S>
size_t step_table_bytes(const map_smoother& h)
{
    if (h.smoother != MAP_RTS) return 0;
    return StepTab<N, S>::bytes(std::min<long>(h.T + 1, StepTab<N, S>::cap()));
}

// bytes of the tiled-scan tables (steptab.cuh ScanBuf)
template <int N, int M, typename S>
size_t scan_table_bytes(const map_smoother& h)
{
    return h.smoother == MAP_RTS ? ScanBuf<N, M, S>::bytes() : 0;
}

// Record of this model for the persistent batch solve (batch_persist.cu):
// the step tables on the first call (not under stream capture), then the
// constants of the affine recursions of its trajectories with KB steps per
// thread, written to out (a host BpModel<S>).  MAP_ERR_UNSUPPORTED when the
// tables do not reach the stationary filter (the batch then keeps the
// segmented scan).
template <int N, int M, typename S>
map_status batch_model(map_smoother& h, void* out, int KB, cudaStream_t st)
{
    using ST = StepTab<N, S>;
    constexpr int NN = N * N;
    if (capturing(st)) return fail(h, MAP_ERR_UNSUPPORTED, "the first batch solve plans its tables: not under capture");
    if (map_status s = table_plan<N, M, S, false>(h, st); s != MAP_OK) return s;
    if (!h.tab_conv) return fail(h, MAP_ERR_UNSUPPORTED, "the step tables do not reach the stationary filter");
    BpModel<S> d{};
    d.N = N;
    d.M = M;
    d.RS = ST::RS;
    d.oE = ST::oE;
    d.oO = ST::oO;
    d.oP = ST::oP;
    d.kc = h.tab_kc;
    d.rows = reinterpret_cast<const S*>(h.d_tab + ST::rows_off());
    d.stats = h.d_stats;
    S row[ST::RS];
    cudaError_t e = cudaMemcpy(row, d.rows + d.kc * ST::RS, sizeof(row), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "step table read-back");
    for (int q = 0; q < NN; ++q) d.Einf[q] = row[ST::oE + q];
    for (int q = 0; q < N; ++q) d.oinf[q] = row[ST::oO + q];
    // FP64 products: E_inf^KB, A^-1 C, A^-1 b and their products with E_inf
    const double* E = h.tab_einf;
    const SetupOut& c = h.consts;
    double P[NN], T2[NN], AiC[NN], Aib[N];
    for (int q = 0; q < NN; ++q) P[q] = q % (N + 1) == 0 ? 1.0 : 0.0;
    for (int s = 0; s < KB; ++s) {
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                double acc = 0.0;
                for (int k = 0; k < N; ++k) acc += P[i * N + k] * E[k * N + j];
                T2[i * N + j] = acc;
            }
        for (int q = 0; q < NN; ++q) P[q] = T2[q];
    }
    for (int i = 0; i < N; ++i) {
        double ab = 0.0;
        for (int k = 0; k < N; ++k) ab += c.Phi[i * N + k] * c.b[k];
        Aib[i] = ab;
        for (int j = 0; j < N; ++j) {
            double ac = 0.0;
            for (int k = 0; k < N; ++k) ac += c.Phi[i * N + k] * c.C[k * N + j];
            AiC[i * N + j] = ac;
        }
    }
    for (int i = 0; i < N; ++i) {
        double eb = 0.0;
        for (int k = 0; k < N; ++k) eb += E[i * N + k] * Aib[k];
        d.EAib[i] = S(eb);
        d.Aib[i] = S(Aib[i]);
        for (int j = 0; j < N; ++j) {
            double ec = 0.0;
            for (int k = 0; k < N; ++k) ec += E[i * N + k] * AiC[k * N + j];
            d.EAiC[i * N + j] = S(ec);
            d.AiC[i * N + j] = S(AiC[i * N + j]);
        }
    }
    for (int q = 0; q < NN; ++q) d.PhiK[q] = S(P[q]);
    for (int q = 0; q < N * M; ++q) d.G[q] = S(c.G[q]);
    for (int q = 0; q < N; ++q) {
        d.Gr[q] = S(c.Gr[q]);
        d.v0[q] = S(c.v0[q]);
    }
    *static_cast<BpModel<S>*>(out) = d;
    return MAP_OK;
}

// State dimensions up to 6 get every path; larger ones (whose 5-tuples do not
// fit one thread's registers) the RTS solve, the cost and the sequential baseline.
template <int N, int M, typename S>
const Ops* linear_ops()
{
    if constexpr (N <= 6) {
        static const Ops ops{&rts_workspace<N, S>, &solve_linear<N, M, S>, &cost_linear<N, M, S>,
                             &solve_linear_sequential<N, M, S>, &grad_linear<N, M, S>,
                             &solve_linear_seg<N, M, S>, &rts_resident_blocks<N, S, LtiProducer<N, M, S>>,
                             &step_table_bytes<N, S>, &scan_table_bytes<N, M, S>, &dense_linear<N, M, S>,
                             &batch_model<N, M, S>};
        return &ops;
    } else {
        static const Ops ops{&rts_workspace<N, S>, &solve_linear<N, M, S>, &cost_linear<N, M, S>,
                             &solve_linear_sequential<N, M, S>, nullptr, nullptr,
                             &rts_resident_blocks<N, S, LtiProducer<N, M, S>>,
                             &step_table_bytes<N, S>, &scan_table_bytes<N, M, S>};
        return &ops;
    }
}

// ---------------------------------------------------------------------------
// nonlinear models: iterated linearisation (Section 4.4), each iteration one
// filter scan + RTS pass on the elements linearised at the previous estimate
// ---------------------------------------------------------------------------
template <int N, int M, typename S>
NlParams<N, M, S> nl_params(const map_smoother& h)
{
    NlParams<N, M, S> p;
    p.dt = S(h.dt);
    p.expm = h.disc == MAP_EXPM;
    for (int i = 0; i < N; ++i)
        for (int j = i; j < N; ++j) {
            p.C[Sym<N>::at(i, j)] = S(h.dt * h.consts.Q[i * N + j]);
            p.Q[Sym<N>::at(i, j)] = S(h.consts.Q[i * N + j]);
        }
    for (int i = 0; i < M; ++i) p.Rinv[i] = S(1.0 / h.R[i * M + i]);
    for (int i = 0; i < N * N; ++i) p.F[i] = S(h.F[i]);
    for (int i = 0; i < N; ++i) p.c[i] = S(h.c[i]);
    for (int i = 0; i < M * N; ++i) p.H[i] = S(h.H[i]);
    for (int i = 0; i < M; ++i) p.r[i] = S(h.r[i]);
    p.gamma = S(h.gamma);
    return p;
}

template <class Model, typename S>
map_status solve_nonlinear(map_smoother& h, const void* y, void* x_out, void* filt_out, cudaStream_t st)
{
    constexpr int N = Model::N, M = Model::M;
    NlProducer<Model, S> prod;
    prod.y = static_cast<const S*>(y);
    prod.T = h.T;
    prod.p = nl_params<N, M, S>(h);
    S* cur = static_cast<S*>(x_out);
    S* nxt = static_cast<S*>(h.d_xtmp);
    for (int it = 0; it < h.gn_iters; ++it) {
        prod.xbar = cur;
        const bool last = it + 1 == h.gn_iters;
        if (prod.p.expm && h.d_etab) {
            // the exact elements of this iteration, once, for both scan passes
            prod.etab = nullptr;
            k_exact_rows<Model, S><<<(unsigned)((h.T + 127) / 128), 128, 0, st>>>(prod, static_cast<S*>(h.d_etab));
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
            prod.etab = static_cast<const S*>(h.d_etab);
            h.launches += 1;
        }
        map_status s = run_rts<N, S>(h, prod, nxt, last ? static_cast<S*>(filt_out) : nullptr, st);
        if (s != MAP_OK) return s;
        std::swap(cur, nxt);
    }
    if (cur != x_out) {
        cudaError_t e = cudaMemcpyAsync(x_out, cur, sizeof(S) * (size_t)(h.T + 1) * N,
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync");
    }
    return MAP_OK;
}

template <class Model, typename S>
map_status solve_nonlinear_sequential(map_smoother& h, const void* y, void* x_out, cudaStream_t st)
{
    constexpr int N = Model::N, M = Model::M;
    NlProducer<Model, S> prod;
    prod.y = static_cast<const S*>(y);
    prod.T = h.T;
    prod.p = nl_params<N, M, S>(h);
    S* cur = static_cast<S*>(x_out);
    S* nxt = static_cast<S*>(h.d_xtmp);
    for (int it = 0; it < h.gn_iters; ++it) {
        prod.xbar = cur;
        map_status s = run_sequential<N, S>(h, prod, nxt, st);
        if (s != MAP_OK) return s;
        std::swap(cur, nxt);
    }
    if (cur != x_out) {
        cudaError_t e = cudaMemcpyAsync(x_out, cur, sizeof(S) * (size_t)(h.T + 1) * N,
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync");
    }
    return MAP_OK;
}

template <typename S>
const Ops* coord_turn_ops()
{
    static const Ops ops{&rts_workspace<5, S>, &solve_nonlinear<CtModel<S>, S>, nullptr,
                         &solve_nonlinear_sequential<CtModel<S>, S>, nullptr, nullptr,
                         &rts_resident_blocks<5, S, NlProducer<CtModel<S>, S>>};
    return &ops;
}

template <int N, int M, typename S>
const Ops* cubic_ops()
{
    static const Ops ops{&rts_workspace<N, S>, &solve_nonlinear<CubicModel<N, M, S>, S>, nullptr,
                         &solve_nonlinear_sequential<CubicModel<N, M, S>, S>, nullptr, nullptr,
                         &rts_resident_blocks<N, S, NlProducer<CubicModel<N, M, S>, S>>};
    return &ops;
}

}  // namespace mapk
