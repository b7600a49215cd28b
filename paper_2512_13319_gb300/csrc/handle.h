// Host-side handle of the C ABI and the per-instantiation entry points.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/map_smoother.h"
#include "setup.h"

struct map_smoother {
    // problem
    int model = 0, N = 0, M = 0, NW = 0, prec = 0, disc = 0, smoother = 0, gn_iters = 1;
    int substeps = 1;                  // Euler substeps per interval (MAP_BLOCK_EULER)
    long T = 0;
    double dt = 0, gamma = 0, cond_max = 1e6;
    int device = 0;
    std::vector<double> F, c, L, W, H, r, R, m0, P0;
    mapk::SetupOut consts{};           // FP64 model constants computed on the device
    // launch geometry
    int B = 128;                       // threads per tile CTA
    int K = 16;                        // steps per thread
    int nt = 0;                        // tiles
    long Tpad = 0;                     // nt * B * K
    // device memory owned by the handle
    char* ws = nullptr;
    size_t ws_bytes = 0;
    unsigned long long* d_stats = nullptr;  // event words (STATS_WORDS of them, elements.cuh)
    unsigned* h_flags = nullptr;       // host-mapped error flags raised by report_event (elements.cuh)
    void* d_y = nullptr;               // staging for the host-buffer entry point
    void* d_x = nullptr;
    void* d_xtmp = nullptr;            // Gauss-Newton ping-pong trajectory
    void* d_etab = nullptr;            // Gauss-Newton with exact per-step elements: (A, b, C) of every step
    double* d_cost = nullptr;
    void* d_lam = nullptr;             // adjoint trajectory (linear models)
    double* d_grad = nullptr;          // gradient accumulators
    void* d_fold = nullptr;            // linear-fold constants of K steps (linear models)
    double* d_setup = nullptr;         // set-up kernel inputs (SETUP_IN_CAP doubles), then its SetupOut
    int fold_K = 0, fold_B = 0;        // K and B they were computed for (0: stale)
    // per-step tables of linear time-invariant RTS solves (steptab.cuh)
    char* d_tab = nullptr;
    int tab_state = 0;                 // 0: stale (model set-up changed), 1: computed
    int tab_conv = 0;                  // the tables reached the stationary filter (kc valid)
    double tab_einf[64] = {};          // E of row kc in FP64 (N x N, N <= 8)
    int tab_ok = 0;                    // the tables reach the stationary filter: the table solve runs
    long tab_kt = 0, tab_kc = 0;
    // tiled-scan geometry of the table solve (steptab.cuh ScanGeom) and its buffer
    char* d_scan = nullptr;
    int sc_K = 0, sc_Kt = 0, sc_Jt = 0, sc_nt = 0;
    int fused = -1;                    // single-launch LTI solve fits co-resident (-1: not yet asked)
    int launches = 0;                  // kernels of the last solve
    int path = 0;                      // how its last scan ran (map_smoother_solve_path)
    unsigned long long bar_arrivals = 0;   // grid-barrier arrivals counted at d_stats[3] so far
    double logq = 0.0, logr = 0.0;     // noise scales of the gradient parameters
    // per-phase timing (map_smoother_profile)
    bool profile = false;
    cudaEvent_t ev[8] = {};
    int nev = 0;
    std::string err;
};

namespace mapk {

size_t elem_bytes(int prec);

// bytes of the linear-fold constants of an (n, m) linear model in scalars of
// es bytes: up to 64 steps per thread, 8 tree levels and the thread-prefix
// tables of up to 128 threads per tile, then the tile tables of nt tiles and,
// for at most 513 tiles, their products (the layouts of FoldLayout and
// TileTables in lti_fold.cuh)
inline size_t fold_bytes(int n, int m, size_t es, long nt)
{
    auto al = [](size_t x) { return (x + 15) / 16 * 16; };
    const int ns = n * (n + 1) / 2, V = 16 / (int)es, P = (n + V - 1) / V * V;
    const int oG = (n * n + 2 * ns + 2 * n + 3) / 4 * 4;
    const int oL = (oG + 64 * 2 * n * m + 3) / 4 * 4;
    const int LS = (3 * n * P + 4 * n * n + 3) / 4 * 4;
    const int PS = (n * n + 2 * ns + 3) / 4 * 4;
    const size_t consts = es * (size_t)(oL + 8 * LS + 128 * PS + 128 * 4 * n * n);
    const size_t tiles = al(consts) + sizeof(double) * (24 + 8) * 3 * n * n + al(es * nt * ns);
    const size_t pi = al(tiles + es * nt * n * n);
    return pi + (nt <= 4 * 128 + 1 ? al(2 * es * (size_t)(nt * (nt + 1) / 2) * n * n) + es * (size_t)nt * n * n : 0);
}

// Per-(model, N, M, precision) entry points, explicitly instantiated in the inst_*.cu files.
struct Ops {
    size_t (*workspace_bytes)(const map_smoother& h);
    map_status (*solve)(map_smoother& h, const void* y, void* x_out, void* filt_out, cudaStream_t st);
    map_status (*cost)(map_smoother& h, const void* y, const void* x, double* d_cost, cudaStream_t st);
    map_status (*solve_sequential)(map_smoother& h, const void* y, void* x_out, cudaStream_t st);
    map_status (*grad)(map_smoother& h, const void* y, const void* x, const void* dLdx, int flags,
                       double* dtheta, cudaStream_t st);
    map_status (*solve_seg)(map_smoother& h, const void* y, const unsigned char* reset, void* x_out,
                            cudaStream_t st);
    int (*resident_blocks)(int B);     // CTAs of the filter kernels per SM at B threads
    size_t (*tab_bytes)(const map_smoother& h) = nullptr;   // per-step table buffer (0: none)
    size_t (*scan_bytes)(const map_smoother& h) = nullptr;  // tiled-scan table buffer (0: none)
    map_status (*dense)(map_smoother& h, const void* y, const void* x, const void* filt, void* out,
                        cudaStream_t st) = nullptr;         // states between the grid points
    map_status (*batch_model)(map_smoother& h, void* out, int KB,
                              cudaStream_t st) = nullptr;   // BpModel<S> record for the persistent batch solve
};

// geometry (steps per thread K, threads per tile B) and its workspace bytes
void set_geometry(map_smoother& h, int K, int B);
// K for B threads per tile such that the tiles fill whole waves of resident CTAs
int balanced_steps_per_thread(const map_smoother& h, int B);
// largest K whose RTS staging fits shared memory at B threads per tile
int max_steps_per_thread(const map_smoother& h, int B);
bool geometry_fits(const map_smoother& h, int B);
map_status ensure_workspace(map_smoother& h, size_t bytes);
map_status create_handle(map_smoother** out, const map_problem_desc* desc);

const Ops* find_ops(int model, int N, int M, int prec);

map_status fail(map_smoother& h, map_status s, const std::string& msg);
// MAP_ERR_TIMEOUT / MAP_ERR_SINGULAR (and clears the flag) when an earlier
// launch on the handle raised its host-mapped error flag; MAP_OK otherwise
map_status device_errors(map_smoother& h);
// message returned by map_smoother_last_error(NULL) on this thread
void set_handle_free_error(const std::string& msg);
map_status cuda_fail(map_smoother& h, cudaError_t e, const char* where);

}  // namespace mapk
