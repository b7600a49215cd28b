// Allocation-free solve for linear models (map_smoother_solve_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs where the device memory
// budget is fixed up front and every allocation is forbidden (a real-time
// control or tracking loop, an embedded service that pre-reserves all device
// memory, a plug-in whose host application owns the allocator).  This entry
// point serves them: it allocates nothing.  The per-solve workspace of the
// scan kernels lives in a file-scope __device__ array of NOALLOC_SCRATCH_BYTES
// (64 MiB), which every GPU that loads this library holds until the process
// exits; the model set-up uses two more small __device__ arrays.  The same
// kernels as map_smoother_solve run on that memory, so the results are the
// same.
//
// Set-up: every call, with the target device current, looks up the device
// addresses of the arrays with cudaGetSymbolAddress (a host-side name of a
// __device__ array is not a device address).  The lookup allocates nothing
// and is not cached, so the addresses stay right when the context is torn
// down and created again (cudaDeviceReset), which may move the module.  The
// first call on a device loads the module into the context; make it before
// any stream capture.
//
// Every call shares the arrays and they keep the contents of the last call:
// the three device counters (precision policy, bounded waits) are cleared at the start of each
// call; everything else is fully written before it is read.  Calls that
// overlap on the GPU (two streams, two host threads) race on the arrays and
// must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "elements.cuh"
#include "handle.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(64) << 20;
constexpr int SETUP_IN_DOUBLES = 8 * 8 * 4 + 8 * 5 + 8 * 8 * 2;   // F, L, W, H, R, P0 + vectors

static __device__ __align__(256) unsigned char g_scratch[NOALLOC_SCRATCH_BYTES];
static __device__ __align__(256) unsigned long long g_stats[mapk::STATS_WORDS];   // event words (no error flags)
static __device__ __align__(256) double g_setup_in[SETUP_IN_DOUBLES];
static __device__ __align__(256) mapk::SetupOut g_setup_out;

struct DeviceArrays {
    int device = 0;
    char* scratch = nullptr;
    unsigned long long* stats = nullptr;
    double* setup_in = nullptr;
    mapk::SetupOut* setup_out = nullptr;
};

// device addresses of the arrays on the current device
cudaError_t device_arrays(DeviceArrays& d)
{
    cudaError_t e = cudaGetDevice(&d.device);
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_scratch)) != cudaSuccess) return e;
    d.scratch = static_cast<char*>(p);
    if ((e = cudaGetSymbolAddress(&p, g_stats)) != cudaSuccess) return e;
    d.stats = static_cast<unsigned long long*>(p);
    if ((e = cudaGetSymbolAddress(&p, g_setup_in)) != cudaSuccess) return e;
    d.setup_in = static_cast<double*>(p);
    if ((e = cudaGetSymbolAddress(&p, g_setup_out)) != cudaSuccess) return e;
    d.setup_out = static_cast<mapk::SetupOut*>(p);
    return cudaSuccess;
}

// failures are reported through map_smoother_last_error(NULL)
map_status noalloc_fail(map_status s, const std::string& msg)
{
    mapk::set_handle_free_error(msg);
    return s;
}

std::vector<double> copy_or_zero(const double* p, size_t n)
{
    std::vector<double> v(n, 0.0);
    if (p) std::memcpy(v.data(), p, n * sizeof(double));
    return v;
}

}  // namespace

extern "C" map_status map_smoother_solve_noalloc(const map_problem_desc* d, const void* y, void* x_out,
                                                 void* stream)
{
    using namespace mapk;
    if (!d || !y || !x_out) return noalloc_fail(MAP_ERR_INVALID_ARG, "desc, y and x_out are required");
    if ((reinterpret_cast<size_t>(y) & 15) || (reinterpret_cast<size_t>(x_out) & 15))
        return noalloc_fail(MAP_ERR_INVALID_ARG, "device arrays must be 16-byte aligned");
    if (d->model != MAP_MODEL_LINEAR)
        return noalloc_fail(MAP_ERR_UNSUPPORTED, "the allocation-free solve supports linear models only");
    const int n = d->nx, m = d->ny, nw = d->nw;
    if (n < 1 || n > MAXN || m < 1 || m > MAXM || nw < 1 || nw > MAXN)
        return noalloc_fail(MAP_ERR_SHAPE, "nx, ny, nw must be in [1, 8]");
    if (d->T < 1) return noalloc_fail(MAP_ERR_SHAPE, "T must be >= 1");
    if (!(d->dt > 0.0) || !std::isfinite(d->dt)) return noalloc_fail(MAP_ERR_INVALID_ARG, "dt must be positive");
    if (d->precision != MAP_FP32 && d->precision != MAP_FP64)
        return noalloc_fail(MAP_ERR_INVALID_ARG, "unknown precision");
    if (d->discretisation < MAP_EULER || d->discretisation > MAP_AUTO)
        return noalloc_fail(MAP_ERR_INVALID_ARG, "unknown discretisation");
    if (d->smoother != MAP_RTS)
        return noalloc_fail(MAP_ERR_UNSUPPORTED, "the allocation-free solve uses the RTS smoother");
    if (!d->F || !d->H || !d->L || !d->W || !d->R || !d->m0 || !d->P0)
        return noalloc_fail(MAP_ERR_INVALID_ARG, "F, H, L, W, R, m0 and P0 are required");
    const Ops* ops = find_ops(MAP_MODEL_LINEAR, n, m, d->precision);
    if (!ops) return noalloc_fail(MAP_ERR_SHAPE, "no compiled kernels for this (nx, ny, precision)");

    DeviceArrays arr;
    cudaError_t e = device_arrays(arr);
    if (e != cudaSuccess)
        return noalloc_fail(MAP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // a handle on the stack: model and geometry as in map_smoother_create, the
    // workspace and counters in the __device__ arrays
    map_smoother h;
    h.device = arr.device;
    h.model = MAP_MODEL_LINEAR; h.N = n; h.M = m; h.NW = nw;
    h.prec = d->precision; h.smoother = MAP_RTS; h.gn_iters = 1;
    h.T = (long)d->T; h.dt = d->dt; h.cond_max = d->cond_max > 0 ? d->cond_max : 1e6;
    h.F = copy_or_zero(d->F, (size_t)n * n);
    h.c = copy_or_zero(d->c, n);
    h.L = copy_or_zero(d->L, (size_t)n * nw);
    h.W = copy_or_zero(d->W, (size_t)nw * nw);
    h.H = copy_or_zero(d->H, (size_t)m * n);
    h.r = copy_or_zero(d->r, m);
    h.R = copy_or_zero(d->R, (size_t)m * m);
    h.m0 = copy_or_zero(d->m0, n);
    h.P0 = copy_or_zero(d->P0, (size_t)n * n);
    int disc = d->discretisation;
    if (disc == MAP_AUTO) {
        double nF = 0.0;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += std::fabs(h.F[i * n + j]);
            nF = std::max(nF, s);
        }
        disc = nF * h.dt > 0.05 ? MAP_EXPM : MAP_EULER;
    }
    h.disc = disc;

    // model set-up on the device into the __device__ arrays
    std::vector<double> host;
    for (const std::vector<double>* v : {&h.F, &h.c, &h.L, &h.W, &h.H, &h.r, &h.R, &h.m0, &h.P0})
        host.insert(host.end(), v->begin(), v->end());
    if (host.size() > (size_t)SETUP_IN_DOUBLES) return noalloc_fail(MAP_ERR_SHAPE, "model too large");
    if ((e = cudaMemcpyAsync(arr.setup_in, host.data(), host.size() * sizeof(double),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return noalloc_fail(MAP_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    SetupIn si{};
    si.nx = n; si.ny = m; si.nw = nw; si.mode = disc; si.dt = h.dt;
    const double* b = arr.setup_in;
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
    if ((e = launch_setup(si, arr.setup_out, st)) != cudaSuccess)
        return noalloc_fail(MAP_ERR_CUDA, std::string("set-up kernel launch: ") + cudaGetErrorString(e));
    if ((e = cudaMemcpyAsync(&h.consts, arr.setup_out, sizeof(SetupOut), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return noalloc_fail(MAP_ERR_CUDA, std::string("set-up: ") + cudaGetErrorString(e));
    if (h.consts.flags & SETUP_SINGULAR_R) return noalloc_fail(MAP_ERR_SINGULAR, "R is singular");
    if (h.consts.flags & SETUP_SINGULAR_P0) return noalloc_fail(MAP_ERR_SINGULAR, "P0 is singular");
    if (h.consts.flags & SETUP_SINGULAR_A) return noalloc_fail(MAP_ERR_SINGULAR, "the interval map A is singular");

    // fixed geometry (unlike map_smoother_create, which balances K over the
    // resident CTAs and honours desc->tile_threads): K = 16 steps per thread,
    // B = 128 threads per tile (fewer when the trees do not fit), so that the
    // scratch bound is a simple function of T
    const size_t es = elem_bytes(h.prec);
    const size_t V = 16 / es, P = (n + V - 1) / V * V;
    const size_t NE = 3 * n * P + 2 * P, NSCR = 3 * n * P + P, NL = n <= 2 ? 2 : n <= 4 ? 4 : 8;
    auto tree_bytes = [&](int bb) { return es * (2 * (size_t)bb * NE + (size_t)bb / NL * NSCR); };
    int B = 128;
    while (B > 32 && tree_bytes(B) > 100 * 1024) B /= 2;
    h.B = B;
    h.K = 16;
    const long L = (long)h.B * h.K;
    h.nt = (int)((h.T + L - 1) / L);
    h.Tpad = (long)h.nt * L;
    const size_t fold_off = (ops->workspace_bytes(h) + 255) / 256 * 256;
    const size_t need = fold_off + fold_bytes(n, m, es, h.nt);
    if (need > NOALLOC_SCRATCH_BYTES)
        return noalloc_fail(MAP_ERR_SHAPE,
                            "T too large for the allocation-free scratch: needs " + std::to_string(need) +
                                " bytes, the __device__ array holds " + std::to_string(NOALLOC_SCRATCH_BYTES));
    h.ws = arr.scratch;
    h.d_fold = arr.scratch + fold_off;     // recomputed by every call (fold_K = 0)
    h.fold_K = 0;
    h.d_stats = arr.stats;
    // the counters and the grid-barrier arrival count (the stack handle starts at 0)
    if ((e = cudaMemsetAsync(arr.stats, 0, mapk::STATS_WORDS * sizeof(unsigned long long), st)) != cudaSuccess)
        return noalloc_fail(MAP_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const map_status s = ops->solve(h, y, x_out, nullptr, st);
    h.ws = nullptr;        // the stack handle owns nothing
    h.d_fold = nullptr;
    h.d_stats = nullptr;
    if (s != MAP_OK) return noalloc_fail(s, h.err);
    return MAP_OK;
}
