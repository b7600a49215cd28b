// C ABI of the parallel MAP smoother: argument checks, model set-up, workspace
// ownership and dispatch to the compiled (model, N, M, precision) instances.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "elements.cuh"
#include "handle.h"

namespace mapk {

template <int N, int M, typename S> const Ops* linear_ops();
template <typename S> const Ops* coord_turn_ops();
template <int N, int M, typename S> const Ops* cubic_ops();

#define MAP_LINEAR_SHAPES(X) X(2, 1) X(3, 1) X(4, 2) X(5, 2) X(6, 3) X(8, 4)
#define MAP_CUBIC_SHAPES(X) X(2, 2)

const Ops* find_ops(int model, int N, int M, int prec)
{
#define CASE_LIN(n, m)                                                        \
    if (N == n && M == m) return prec == MAP_FP32 ? linear_ops<n, m, float>() \
                                                  : linear_ops<n, m, double>();
#define CASE_CUB(n, m)                                                        \
    if (N == n && M == m) return prec == MAP_FP32 ? cubic_ops<n, m, float>()  \
                                                  : cubic_ops<n, m, double>();
    if (model == MAP_MODEL_LINEAR) { MAP_LINEAR_SHAPES(CASE_LIN) }
    if (model == MAP_MODEL_COORD_TURN && N == 5 && M == 2)
        return prec == MAP_FP32 ? coord_turn_ops<float>() : coord_turn_ops<double>();
    if (model == MAP_MODEL_CUBIC) { MAP_CUBIC_SHAPES(CASE_CUB) }
    return nullptr;
#undef CASE_LIN
#undef CASE_CUB
}

size_t elem_bytes(int prec) { return prec == MAP_FP32 ? 4 : 8; }

map_status fail(map_smoother& h, map_status s, const std::string& msg)
{
    h.err = msg;
    return s;
}

map_status cuda_fail(map_smoother& h, cudaError_t e, const char* where)
{
    h.err = std::string(where) + ": " + cudaGetErrorString(e);
    return MAP_ERR_CUDA;
}

map_status device_errors(map_smoother& h)
{
    if (!h.h_flags) return MAP_OK;
    volatile unsigned* f = h.h_flags;
    if (f[EV_TIMEOUT]) {
        f[EV_TIMEOUT] = 0;
        f[EV_SINGULAR] = 0;
        return fail(h, MAP_ERR_TIMEOUT,
                    "a bounded device wait (bulk copy or grid barrier) ran out in an earlier launch on this "
                    "handle: the results of that launch are not valid");
    }
    if (f[EV_SINGULAR]) {
        f[EV_SINGULAR] = 0;
        return fail(h, MAP_ERR_SINGULAR,
                    "a singular pivot in an earlier launch on this handle (a combine's FP64 inverse or the "
                    "terminal solve): the results of that launch are not valid");
    }
    return MAP_OK;
}

}  // namespace mapk

using namespace mapk;

namespace {

thread_local std::string g_create_error;

std::vector<double> copy_or(const double* p, size_t n, double fill = 0.0)
{
    std::vector<double> v(n, fill);
    if (p) std::memcpy(v.data(), p, n * sizeof(double));
    return v;
}

bool aligned16(const void* p) { return (reinterpret_cast<size_t>(p) & 15) == 0; }

void free_handle(map_smoother* h)
{
    if (!h) return;
    if (h->ws) cudaFree(h->ws);
    if (h->d_stats) cudaFree(h->d_stats);
    if (h->h_flags) cudaFreeHost(h->h_flags);
    if (h->d_y) cudaFree(h->d_y);
    if (h->d_x) cudaFree(h->d_x);
    if (h->d_xtmp) cudaFree(h->d_xtmp);
    if (h->d_etab) cudaFree(h->d_etab);
    if (h->d_cost) cudaFree(h->d_cost);
    if (h->d_lam) cudaFree(h->d_lam);
    if (h->d_grad) cudaFree(h->d_grad);
    if (h->d_fold) cudaFree(h->d_fold);
    if (h->d_tab) cudaFree(h->d_tab);
    if (h->d_scan) cudaFree(h->d_scan);
    if (h->d_setup) cudaFree(h->d_setup);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    delete h;
}

// Model set-up on the device (FP64) for the current parameters: the noise
// scales of the gradient parameters multiply W and R.
map_status run_setup(map_smoother* h)
{
    const int n = h->N, m = h->M, nw = h->NW;
    h->fold_K = 0;                     // linear-fold constants follow the model
    h->tab_state = 0;                  // and so do the per-step tables
    h->tab_conv = 0;
    h->tab_ok = 0;
    std::vector<double> W = h->W, R = h->R;
    for (double& w : W) w *= std::exp(h->logq);
    for (double& r : R) r *= std::exp(h->logr);
    std::vector<double> host;
    auto push = [&](const std::vector<double>& v) { host.insert(host.end(), v.begin(), v.end()); };
    push(h->F); push(h->c); push(h->L); push(W); push(h->H); push(h->r); push(R); push(h->m0);
    push(h->P0);
    const size_t nin = host.size();
    cudaError_t e;
    if (nin > (size_t)SETUP_IN_CAP) return fail(*h, MAP_ERR_SHAPE, "model too large for the set-up buffer");
    // one buffer for the handle's lifetime (inputs, then SetupOut), so that a
    // parameter update allocates nothing
    if (!h->d_setup &&
        (e = cudaMalloc(&h->d_setup, SETUP_IN_CAP * sizeof(double) + sizeof(SetupOut))) != cudaSuccess)
        return cuda_fail(*h, e, "cudaMalloc");
    SetupOut* d_out = reinterpret_cast<SetupOut*>(h->d_setup + SETUP_IN_CAP);
    if ((e = cudaMemcpy(h->d_setup, host.data(), nin * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(*h, e, "cudaMemcpy");
    const double* b = h->d_setup;
    SetupIn si{};
    // nonlinear models discretise per step in their producers: their set-up takes the Euler constants
    si.nx = n; si.ny = m; si.nw = nw;
    si.mode = h->model != MAP_MODEL_LINEAR && h->disc == MAP_EXPM ? MAP_EULER : h->disc;
    si.dt = h->dt; si.substeps = h->substeps;
    size_t o = 0;
    si.F = b + o; o += (size_t)n * n;
    si.c = b + o; o += n;
    si.L = b + o; o += (size_t)n * nw;
    si.W = b + o; o += (size_t)nw * nw;
    si.H = b + o; o += (size_t)m * n;
    si.r = b + o; o += m;
    si.R = b + o; o += (size_t)m * m;
    si.m0 = b + o; o += n;
    si.P0 = b + o;
    if ((e = launch_setup(si, d_out, 0)) != cudaSuccess)
        return cuda_fail(*h, e, "set-up kernel launch");
    if ((e = cudaMemcpy(&h->consts, d_out, sizeof(SetupOut), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(*h, e, "set-up kernel");
    return MAP_OK;
}

map_status create_impl(map_smoother* h, const map_problem_desc* d)
{
    if (!d) return fail(*h, MAP_ERR_INVALID_ARG, "desc is NULL");
    const int n = d->nx, m = d->ny, nw = d->nw;
    if (n < 1 || n > MAXN || m < 1 || m > MAXM || nw < 1 || nw > MAXN)
        return fail(*h, MAP_ERR_SHAPE, "nx, ny, nw must be in [1, 8]");
    if (d->T < 1) return fail(*h, MAP_ERR_SHAPE, "T must be >= 1");
    if (!(d->dt > 0.0) || !std::isfinite(d->dt)) return fail(*h, MAP_ERR_INVALID_ARG, "dt must be positive");
    if (d->precision != MAP_FP32 && d->precision != MAP_FP64)
        return fail(*h, MAP_ERR_INVALID_ARG, "unknown precision");
    if (d->discretisation < MAP_EULER || d->discretisation > MAP_RICCATI_EXACT)
        return fail(*h, MAP_ERR_INVALID_ARG, "unknown discretisation");
    if (d->discretisation >= MAP_BLOCK_EULER) {
        if (d->model != MAP_MODEL_LINEAR || d->smoother != MAP_RTS || n > 6)
            return fail(*h, MAP_ERR_UNSUPPORTED,
                        "block and exact elements are built for linear models with nx <= 6 and the RTS smoother");
        if (d->substeps < 0 || d->substeps > 64)
            return fail(*h, MAP_ERR_INVALID_ARG, "substeps must be in 1..64 (0 = 10)");
    }
    h->substeps = d->discretisation == MAP_BLOCK_EULER ? (d->substeps > 0 ? d->substeps : 10) : 1;
    if (d->smoother != MAP_RTS && d->smoother != MAP_TWO_FILTER)
        return fail(*h, MAP_ERR_INVALID_ARG, "unknown smoother");
    if (!d->L || !d->W || !d->R || !d->m0 || !d->P0)
        return fail(*h, MAP_ERR_INVALID_ARG, "L, W, R, m0 and P0 are required");
    const bool linear_like = d->model == MAP_MODEL_LINEAR || d->model == MAP_MODEL_CUBIC;
    if (linear_like && (!d->F || !d->H))
        return fail(*h, MAP_ERR_INVALID_ARG, "F and H are required for linear and cubic models");
    if (d->model == MAP_MODEL_COORD_TURN && (n != 5 || m != 2))
        return fail(*h, MAP_ERR_SHAPE, "the coordinated-turn model has nx = 5, ny = 2");
    if (d->model < MAP_MODEL_LINEAR || d->model > MAP_MODEL_CUBIC)
        return fail(*h, MAP_ERR_INVALID_ARG, "unknown model");
    if (d->model != MAP_MODEL_LINEAR && d->gn_iters < 1)
        return fail(*h, MAP_ERR_INVALID_ARG, "gn_iters must be >= 1 for nonlinear models");
    if (d->smoother == MAP_TWO_FILTER && (d->model != MAP_MODEL_LINEAR || n > 6))
        return fail(*h, MAP_ERR_UNSUPPORTED, "the two-filter smoother is built for linear models with nx <= 6");

    h->model = d->model; h->N = n; h->M = m; h->NW = nw;
    h->prec = d->precision; h->smoother = d->smoother;
    h->gn_iters = d->model == MAP_MODEL_LINEAR ? 1 : d->gn_iters;
    h->T = (long)d->T; h->dt = d->dt; h->gamma = d->gamma;
    h->cond_max = d->cond_max > 0 ? d->cond_max : 1e6;
    h->F = copy_or(d->F, (size_t)n * n);
    h->c = copy_or(d->c, n);
    h->L = copy_or(d->L, (size_t)n * nw);
    h->W = copy_or(d->W, (size_t)nw * nw);
    h->H = copy_or(d->H, (size_t)m * n);
    h->r = copy_or(d->r, m);
    h->R = copy_or(d->R, (size_t)m * m);
    h->m0 = copy_or(d->m0, n);
    h->P0 = copy_or(d->P0, (size_t)n * n);

    const Ops* ops = find_ops(h->model, n, m, h->prec);
    if (!ops) return fail(*h, MAP_ERR_SHAPE, "no compiled kernels for this (model, nx, ny, precision)");

    int disc = d->discretisation;
    if (disc == MAP_AUTO) {
        double nF = 0.0;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += std::fabs(h->F[i * n + j]);
            nF = std::max(nF, s);
        }
        disc = (h->model == MAP_MODEL_LINEAR && nF * h->dt > 0.05) ? MAP_EXPM : MAP_EULER;
    }
    h->disc = disc;

    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return cuda_fail(*h, e, "cudaGetDevice");

    if (map_status st = run_setup(h); st != MAP_OK) return st;
    if (h->consts.flags & SETUP_SINGULAR_R) return fail(*h, MAP_ERR_SINGULAR, "R is singular");
    if (h->consts.flags & SETUP_SINGULAR_P0) return fail(*h, MAP_ERR_SINGULAR, "P0 is singular");
    if (h->consts.flags & SETUP_SINGULAR_A) return fail(*h, MAP_ERR_SINGULAR, "the interval map A is singular");

    // launch geometry: the tile CTA's tree (2B nodes with full, row-padded
    // matrices, plus one scratch area per sub-warp group) must fit in shared memory
    const size_t es = elem_bytes(h->prec);
    const size_t V = 16 / es, P = (n + V - 1) / V * V;
    const size_t NE = 3 * n * P + 2 * P, NSCR = 3 * n * P + P, NL = n <= 2 ? 2 : n <= 4 ? 4 : 8;
    auto tree_bytes = [&](int b) { return es * (2 * (size_t)b * NE + (size_t)b / NL * NSCR); };
    int B = d->tile_threads > 0 ? d->tile_threads : 128;
    if (B < 32 || B > 128 || (B & (B - 1)))
        return fail(*h, MAP_ERR_INVALID_ARG, "tile_threads must be 32, 64 or 128");
    while (B > 32 && tree_bytes(B) > (d->tile_threads > 0 ? 200 : 100) * 1024) B /= 2;
    if (d->steps_per_thread < 0 || d->steps_per_thread > max_steps_per_thread(*h, B))
        return fail(*h, MAP_ERR_INVALID_ARG,
                    "steps_per_thread must be 0 (automatic) or 1.." + std::to_string(max_steps_per_thread(*h, B)));
    set_geometry(*h, d->steps_per_thread > 0 ? d->steps_per_thread : balanced_steps_per_thread(*h, B), B);

    h->ws_bytes = ops->workspace_bytes(*h);
    if ((e = cudaMalloc(&h->ws, h->ws_bytes)) != cudaSuccess) return cuda_fail(*h, e, "cudaMalloc workspace");
    // event words (counters, the grid barrier state of the single-launch
    // solves) and the host-mapped error flags whose device address word 4 holds
    if ((e = cudaMalloc(&h->d_stats, STATS_WORDS * sizeof(unsigned long long))) != cudaSuccess)
        return cuda_fail(*h, e, "cudaMalloc");
    if ((e = cudaMemset(h->d_stats, 0, STATS_WORDS * sizeof(unsigned long long))) != cudaSuccess)
        return cuda_fail(*h, e, "cudaMemset");
    if ((e = cudaHostAlloc(reinterpret_cast<void**>(&h->h_flags), 4 * sizeof(unsigned), cudaHostAllocMapped)) !=
        cudaSuccess)
        return cuda_fail(*h, e, "cudaHostAlloc");
    std::memset(h->h_flags, 0, 4 * sizeof(unsigned));
    {
        void* dflags = nullptr;
        if ((e = cudaHostGetDevicePointer(&dflags, h->h_flags, 0)) != cudaSuccess)
            return cuda_fail(*h, e, "cudaHostGetDevicePointer");
        const unsigned long long a = reinterpret_cast<uintptr_t>(dflags);
        if ((e = cudaMemcpy(h->d_stats + EV_FLAGS, &a, sizeof(a), cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(*h, e, "cudaMemcpy");
    }
    if ((e = cudaMalloc(&h->d_cost, sizeof(double))) != cudaSuccess) return cuda_fail(*h, e, "cudaMalloc");
    if (h->model != MAP_MODEL_LINEAR) {
        if ((e = cudaMalloc(&h->d_xtmp, (size_t)(h->T + 1) * n * es)) != cudaSuccess)
            return cuda_fail(*h, e, "cudaMalloc");
        // exact per-step elements: one row of (A, b, C) per step, formed once per
        // iteration (rows of whole 16-byte words)
        const size_t rs = ((size_t)(n * n + n + n * (n + 1) / 2) * es + 15) / 16 * 16;
        if (h->disc == MAP_EXPM && (e = cudaMalloc(&h->d_etab, (size_t)h->T * rs)) != cudaSuccess)
            return cuda_fail(*h, e, "cudaMalloc");
    } else {
        if ((e = cudaMalloc(&h->d_lam, (size_t)(h->T + 1) * n * es)) != cudaSuccess)
            return cuda_fail(*h, e, "cudaMalloc");
        if ((e = cudaMalloc(&h->d_grad, sizeof(double) * (n * n + 2))) != cudaSuccess)
            return cuda_fail(*h, e, "cudaMalloc");
        if ((e = cudaMalloc(&h->d_fold, fold_bytes(n, m, es, h->nt))) != cudaSuccess)
            return cuda_fail(*h, e, "cudaMalloc");
        const size_t tb = ops->tab_bytes ? ops->tab_bytes(*h) : 0;
        if (tb && (e = cudaMalloc(reinterpret_cast<void**>(&h->d_tab), tb)) != cudaSuccess)
            return cuda_fail(*h, e, "cudaMalloc");
        const size_t sb = tb && ops->scan_bytes ? ops->scan_bytes(*h) : 0;
        if (sb && ((e = cudaMalloc(reinterpret_cast<void**>(&h->d_scan), sb)) != cudaSuccess ||
                   (e = cudaMemset(h->d_scan, 0, sb)) != cudaSuccess))
            return cuda_fail(*h, e, "cudaMalloc");
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(*h, e, "create");
    return MAP_OK;
}

}  // namespace

void mapk::set_handle_free_error(const std::string& msg) { g_create_error = msg; }

bool mapk::geometry_fits(const map_smoother& h, int B)
{
    const size_t es = elem_bytes(h.prec);
    const size_t n = h.N, V = 16 / es, P = (n + V - 1) / V * V;
    const size_t NE = 3 * n * P + 2 * P, NSCR = 3 * n * P + P, NL = n <= 2 ? 2 : n <= 4 ? 4 : 8;
    return es * (2 * (size_t)B * NE + (size_t)B / NL * NSCR) <= 200 * 1024;
}

int mapk::max_steps_per_thread(const map_smoother& h, int B)
{
    // the RTS pass stages B*K states next to its affine tree in shared memory
    const size_t es = elem_bytes(h.prec);
    const size_t n = h.N, V = 16 / es, P = (n + V - 1) / V * V, NA = n * P + P;
    int kmax = 64;
    while (kmax > 1 && es * (2 * (size_t)B * NA + (size_t)B * ((kmax * n) | 1)) > 200 * 1024) --kmax;
    return kmax;
}

int mapk::balanced_steps_per_thread(const map_smoother& h, int B)
{
    // A tile of B*K steps is one CTA and all tiles of a launch run at once
    // when there are at most SMs x (resident CTAs per SM) of them.  K is the
    // smallest value in [KMIN, kmax] for which the tiles fill a whole number
    // of such waves: a partial last wave would run a few CTAs alone.
    constexpr int KMIN = 8, KMAX = 64;
    const Ops* ops = find_ops(h.model, h.N, h.M, h.prec);
    int sms = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h.device) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 1;
    }
    const int per_sm = ops && ops->resident_blocks ? ops->resident_blocks(B) : 1;
    const long wave = (long)sms * per_sm * B;
    const int kmax = std::max(KMIN, max_steps_per_thread(h, B));
    const long waves = std::max(1L, (h.T + wave * kmax - 1) / (wave * kmax));
    const long K = (h.T + waves * wave - 1) / (waves * wave);
    return (int)std::min<long>(kmax, std::max<long>(KMIN, K));
}

void mapk::set_geometry(map_smoother& h, int K, int B)
{
    h.K = K;
    h.B = B;
    const long L = (long)B * K;
    h.nt = (int)((h.T + L - 1) / L);
    h.Tpad = (long)h.nt * L;
}

map_status mapk::ensure_workspace(map_smoother& h, size_t bytes)
{
    if (bytes <= h.ws_bytes) return MAP_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && h.ws) e = cudaFree(h.ws);
    h.ws = nullptr;
    h.ws_bytes = 0;
    if (e == cudaSuccess) e = cudaMalloc(&h.ws, bytes);
    if (e != cudaSuccess) return cuda_fail(h, e, "workspace");
    h.ws_bytes = bytes;
    return MAP_OK;
}

map_status mapk::create_handle(map_smoother** out, const map_problem_desc* desc)
{
    return map_smoother_create(out, desc);
}

extern "C" {

map_status map_smoother_create(map_smoother** out, const map_problem_desc* desc)
{
    if (!out) {
        g_create_error = "out is NULL";
        return MAP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    map_smoother* h = new (std::nothrow) map_smoother();
    if (!h) {
        g_create_error = "out of host memory";
        return MAP_ERR_INVALID_ARG;
    }
    const map_status s = create_impl(h, desc);
    if (s != MAP_OK) {
        g_create_error = h->err;
        free_handle(h);
        return s;
    }
    *out = h;
    return MAP_OK;
}

map_status map_smoother_solve(map_smoother* h, const void* y, void* x_out, void* filt_out,
                              double* cost_out, void* stream)
{
    if (!h) { g_create_error = "handle is NULL"; return MAP_ERR_INVALID_ARG; }
    if (!y || !x_out) return fail(*h, MAP_ERR_INVALID_ARG, "y and x_out are required");
    if (!aligned16(y) || !aligned16(x_out) || (filt_out && !aligned16(filt_out)))
        return fail(*h, MAP_ERR_INVALID_ARG, "device arrays must be 16-byte aligned");
    if (map_status s = device_errors(*h); s != MAP_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Ops* ops = find_ops(h->model, h->N, h->M, h->prec);
    h->launches = 0;
    h->path = 0;
    map_status s = ops->solve(*h, y, x_out, filt_out, st);
    if (s != MAP_OK) return s;
    if (cost_out) {
        if (h->disc >= MAP_BLOCK_EULER)
            return fail(*h, MAP_ERR_UNSUPPORTED, "the MAP cost output is defined for per-step elements");
        if (h->consts.flags & SETUP_SINGULAR_C)
            return fail(*h, MAP_ERR_UNSUPPORTED, "the MAP cost needs an invertible process noise");
        if (!ops->cost) return fail(*h, MAP_ERR_UNSUPPORTED, "no cost kernel for this model");
        s = ops->cost(*h, y, x_out, h->d_cost, st);
        if (s != MAP_OK) return s;
        cudaError_t e = cudaMemcpyAsync(cost_out, h->d_cost, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(*h, e, "cost read-back");
        return device_errors(*h);
    }
    return MAP_OK;
}

map_status map_smoother_solve_sequential(map_smoother* h, const void* y, void* x_out, void* stream)
{
    if (!h) { g_create_error = "handle is NULL"; return MAP_ERR_INVALID_ARG; }
    if (!y || !x_out) return fail(*h, MAP_ERR_INVALID_ARG, "y and x_out are required");
    if (!aligned16(y) || !aligned16(x_out))
        return fail(*h, MAP_ERR_INVALID_ARG, "device arrays must be 16-byte aligned");
    if (map_status s = device_errors(*h); s != MAP_OK) return s;
    const Ops* ops = find_ops(h->model, h->N, h->M, h->prec);
    return ops->solve_sequential(*h, y, x_out, static_cast<cudaStream_t>(stream));
}

map_status map_smoother_dense(map_smoother* h, const void* y, const void* x, const void* filt, void* dense_out,
                              void* stream)
{
    if (!h) { g_create_error = "handle is NULL"; return MAP_ERR_INVALID_ARG; }
    if (!y || !x || !filt || !dense_out) return fail(*h, MAP_ERR_INVALID_ARG, "y, x, filt and dense_out are required");
    const Ops* ops = find_ops(h->model, h->N, h->M, h->prec);
    if (!ops->dense || h->disc != MAP_BLOCK_EULER)
        return fail(*h, MAP_ERR_UNSUPPORTED, "dense output needs a linear model with MAP_BLOCK_EULER elements");
    if (map_status s = device_errors(*h); s != MAP_OK) return s;
    return ops->dense(*h, y, x, filt, dense_out, static_cast<cudaStream_t>(stream));
}

map_status map_smoother_solve_host(map_smoother* h, const void* y_host, void* x_host, void* stream)
{
    if (!h) { g_create_error = "handle is NULL"; return MAP_ERR_INVALID_ARG; }
    if (!y_host || !x_host) return fail(*h, MAP_ERR_INVALID_ARG, "y_host and x_host are required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t es = elem_bytes(h->prec);
    const size_t ybytes = (size_t)h->T * h->M * es, xbytes = (size_t)(h->T + 1) * h->N * es;
    cudaError_t e;
    if (!h->d_y) {
        if ((e = cudaMalloc(&h->d_y, ybytes)) != cudaSuccess) return cuda_fail(*h, e, "cudaMalloc");
        if ((e = cudaMalloc(&h->d_x, xbytes)) != cudaSuccess) return cuda_fail(*h, e, "cudaMalloc");
    }
    if ((e = cudaMemcpyAsync(h->d_y, y_host, ybytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(*h, e, "cudaMemcpyAsync H2D");
    if (h->model != MAP_MODEL_LINEAR &&
        (e = cudaMemcpyAsync(h->d_x, x_host, xbytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(*h, e, "cudaMemcpyAsync H2D");
    map_status s = map_smoother_solve(h, h->d_y, h->d_x, nullptr, nullptr, stream);
    if (s != MAP_OK) return s;
    if ((e = cudaMemcpyAsync(x_host, h->d_x, xbytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(*h, e, "cudaMemcpyAsync D2H");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(*h, e, "cudaStreamSynchronize");
    return device_errors(*h);
}

map_status map_smoother_grad(map_smoother* h, const void* y, const void* x, const void* dL_dx, int flags,
                             double* dL_dtheta, void* stream)
{
    if (!h) { g_create_error = "handle is NULL"; return MAP_ERR_INVALID_ARG; }
    if (!y || !x || !dL_dtheta) return fail(*h, MAP_ERR_INVALID_ARG, "y, x and dL_dtheta are required");
    if (!aligned16(y) || !aligned16(x) || (dL_dx && !aligned16(dL_dx)))
        return fail(*h, MAP_ERR_INVALID_ARG, "device arrays must be 16-byte aligned");
    if (h->model != MAP_MODEL_LINEAR || h->disc != MAP_EULER)
        return fail(*h, MAP_ERR_UNSUPPORTED, "gradients need a linear model with Euler elements");
    if (h->consts.flags & (SETUP_SINGULAR_C | SETUP_SINGULAR_Q))
        return fail(*h, MAP_ERR_UNSUPPORTED, "gradients need an invertible process noise Q");
    const Ops* ops = find_ops(h->model, h->N, h->M, h->prec);
    if (!ops->grad) return fail(*h, MAP_ERR_UNSUPPORTED, "no gradient kernels for this state dimension");
    if (map_status s = device_errors(*h); s != MAP_OK) return s;
    if (map_status s = ops->grad(*h, y, x, dL_dx, flags, dL_dtheta, static_cast<cudaStream_t>(stream)); s != MAP_OK)
        return s;
    return device_errors(*h);               // the gradient read-back synchronised the stream
}

namespace {
// log det of the symmetric positive definite n x n matrix A (row-major) by
// Cholesky; false when a pivot is not positive
bool logdet_spd(int n, std::vector<double> A, double* out)
{
    double ld = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
        if (!(d > 0.0)) return false;
        const double l = std::sqrt(d);
        A[j * n + j] = l;
        ld += 2.0 * std::log(l);
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = s / l;
        }
    }
    *out = ld;
    return true;
}
}  // namespace

map_status map_smoother_log_normaliser(const map_smoother* h, double* out)
{
    if (!h || !out) return MAP_ERR_INVALID_ARG;
    map_smoother& hm = const_cast<map_smoother&>(*h);
    if (h->model != MAP_MODEL_LINEAR || h->disc != MAP_EULER)
        return fail(hm, MAP_ERR_UNSUPPORTED, "the log-normalisers are those of linear models with Euler elements");
    const int n = h->N, m = h->M, nw = h->NW;
    const double twopi = 2.0 * 3.14159265358979323846;
    std::vector<double> C((size_t)n * n, 0.0), R((size_t)m * m);
    const double cq = twopi * h->dt * std::exp(h->logq);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int a = 0; a < nw; ++a)
                for (int b = 0; b < nw; ++b) s += h->L[i * nw + a] * h->W[a * nw + b] * h->L[j * nw + b];
            C[i * n + j] = cq * s;
        }
    const double cr = twopi * std::exp(h->logr) / h->dt;
    for (int i = 0; i < m * m; ++i) R[i] = cr * h->R[i];
    double lc = 0.0, lr = 0.0;
    if (!logdet_spd(n, C, &lc)) return fail(hm, MAP_ERR_SINGULAR, "the process noise C = dt Q is not positive definite");
    if (!logdet_spd(m, R, &lr)) return fail(hm, MAP_ERR_SINGULAR, "R is not positive definite");
    *out = 0.5 * double(h->T) * (lc + lr);
    return MAP_OK;
}

map_status map_smoother_update(map_smoother* h, const double* F, double log_q, double log_r)
{
    if (!h) { g_create_error = "handle is NULL"; return MAP_ERR_INVALID_ARG; }
    if (!std::isfinite(log_q) || !std::isfinite(log_r))
        return fail(*h, MAP_ERR_INVALID_ARG, "log_q and log_r must be finite");
    if (F) std::memcpy(h->F.data(), F, sizeof(double) * h->N * h->N);
    h->logq = log_q;
    h->logr = log_r;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(*h, e, "cudaDeviceSynchronize");
    if (map_status st = run_setup(h); st != MAP_OK) return st;
    if (h->consts.flags & SETUP_SINGULAR_R) return fail(*h, MAP_ERR_SINGULAR, "R is singular");
    if (h->consts.flags & SETUP_SINGULAR_A) return fail(*h, MAP_ERR_SINGULAR, "the interval map A is singular");
    return MAP_OK;
}

map_status map_smoother_stats(map_smoother* h, unsigned long long out[3], int reset, void* stream)
{
    if (!h || !out) return MAP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(out, h->d_stats, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && reset) e = cudaMemsetAsync(h->d_stats, 0, 3 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(*h, e, "stats");
    return device_errors(*h);
}

map_status map_smoother_geometry(const map_smoother* h, int* K, int* B, int* tiles)
{
    if (!h || !K || !B || !tiles) return MAP_ERR_INVALID_ARG;
    const bool scan = h->path == MAP_PATH_TABLES && h->sc_nt > 0;
    *K = scan ? h->sc_K : h->K;
    *B = h->B;
    *tiles = scan ? h->sc_nt : h->nt;
    return MAP_OK;
}

map_status map_smoother_launches(const map_smoother* h, int* kernels)
{
    if (!h || !kernels) return MAP_ERR_INVALID_ARG;
    *kernels = h->launches;
    return MAP_OK;
}

map_status map_smoother_solve_path(const map_smoother* h, int* path)
{
    if (!h || !path) return MAP_ERR_INVALID_ARG;
    *path = h->path;
    return MAP_OK;
}

map_status map_smoother_profile(map_smoother* h, int enable)
{
    if (!h) return MAP_ERR_INVALID_ARG;
    if (enable && !h->ev[0]) {
        for (cudaEvent_t& e : h->ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return cuda_fail(*h, r, "cudaEventCreate");
        }
    }
    h->profile = enable != 0;
    h->nev = 0;
    return MAP_OK;
}

map_status map_smoother_phase_times(map_smoother* h, float* ms_out, int cap, int* n_out)
{
    if (!h || !ms_out || !n_out) return MAP_ERR_INVALID_ARG;
    *n_out = 0;
    if (h->nev < 2) return fail(*h, MAP_ERR_INVALID_ARG, "no profiled solve recorded");
    cudaError_t e = cudaEventSynchronize(h->ev[h->nev - 1]);
    if (e != cudaSuccess) return cuda_fail(*h, e, "cudaEventSynchronize");
    int n = 0;
    for (int i = 0; i + 1 < h->nev && n < cap; ++i, ++n) {
        e = cudaEventElapsedTime(ms_out + n, h->ev[i], h->ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(*h, e, "cudaEventElapsedTime");
    }
    *n_out = n;
    return MAP_OK;
}

void map_smoother_destroy(map_smoother* h) { free_handle(h); }

const char* map_smoother_last_error(const map_smoother* h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

int map_smoother_supported(int model, int nx, int ny, int precision)
{
    if (precision != MAP_FP32 && precision != MAP_FP64) return 0;
    return find_ops(model, nx, ny, precision) != nullptr;
}

const char* map_smoother_version(void) { return "0.1.0"; }

}  // extern "C"
