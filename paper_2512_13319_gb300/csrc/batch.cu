// Batched solve: many independent trajectories of a few linear models.
//
// Trajectories of the same model are stored concatenated, one spare row
// between them.  Every trajectory starts from the model's prior, so the
// data-independent part of its solve (the filter's P_k and closed-loop maps)
// is that of the model's per-step tables at its local step: the chunked solve
// of batch_scan.cuh runs all trajectories of a model as five data-parallel
// kernels over chunks of its trajectories.  A model whose tables do not reach
// the stationary filter takes the segmented scan instead: the trajectories
// form one scan with the prior element at every trajectory start (see
// SegLtiProducer), its steps per thread K and threads per tile B chosen by
// timing the candidates (K = 8, 16 and the wave-filling K of each B) on the
// caller's first arrays (autotuning).  The per-model launches are captured once
// into a CUDA graph whose branches run concurrently; each later call with the
// same arrays is one graph launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "handle.h"

using namespace mapk;

struct map_batch {
    struct Group {
        int model = -1;
        map_smoother* h = nullptr;
        unsigned char* d_reset = nullptr;
        long y_rows = 0, x_rows = 0;
        int ntraj = 0;
        cudaStream_t stream = nullptr;
        cudaEvent_t done = nullptr;
        bool tuned = false;
        bool chunked = false;          // the chunked solve runs (tables converged)
        BatchPlan bp;
    };
    int nmodels = 0;
    std::vector<Group> groups;
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;
    std::string err;
};

namespace {

thread_local std::string g_batch_error;

map_status bfail(map_batch* b, map_status s, const std::string& m)
{
    if (b) b->err = m;
    g_batch_error = m;
    return s;
}

void destroy_batch(map_batch* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto& g : b->groups) {
        if (g.h) map_smoother_destroy(g.h);
        if (g.d_reset) cudaFree(g.d_reset);
        if (g.bp.traj) cudaFree(g.bp.traj);
        if (g.bp.chunk_traj) cudaFree(g.bp.chunk_traj);
        if (g.bp.W) cudaFree(g.bp.W);
        if (g.bp.V) cudaFree(g.bp.V);
        if (g.bp.Bt) cudaFree(g.bp.Bt);
        if (g.bp.tm) cudaFree(g.bp.tm);
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.done) cudaEventDestroy(g.done);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

// reset[pos[i]] = 1 for the start positions of trajectories 1..n-1
__global__ void k_mark_resets(const long long* __restrict__ pos, int n, unsigned char* __restrict__ reset)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) reset[pos[i]] = 1;
}

map_status solve_group(map_batch::Group& g, const void* y, void* x, cudaStream_t st)
{
    const Ops* ops = find_ops(g.h->model, g.h->N, g.h->M, g.h->prec);
    if (g.chunked) return ops->batch(*g.h, g.bp, y, x, st);
    return ops->solve_seg(*g.h, y, g.d_reset, x, st);
}

// device arrays of the chunked solve of one model: trajectories (first row,
// length, chunks), the trajectory of each chunk, per-chunk scratch and the
// chunk maps
map_status plan_chunks(map_batch::Group& g, const std::vector<long>& rows, const std::vector<long>& lens)
{
    std::vector<BatchTraj> tr(rows.size());
    std::vector<int> ct;
    for (size_t j = 0; j < rows.size(); ++j) {
        const int nc = (int)((lens[j] + BATCH_CH - 1) / BATCH_CH);
        tr[j] = BatchTraj{rows[j], lens[j], (int)ct.size(), nc};
        for (int i = 0; i < nc; ++i) ct.push_back((int)j);
    }
    BatchPlan& bp = g.bp;
    bp.ntraj = (int)tr.size();
    bp.nchunks = (int)ct.size();
    const size_t es = elem_bytes(g.h->prec), per = es * (size_t)g.h->N * bp.nchunks;
    bp.tm_cap = (int)(16384 * (es == 4 ? 1 : 2) / BATCH_CH + 2);
    cudaError_t e;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&bp.traj), sizeof(BatchTraj) * tr.size())) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&bp.chunk_traj), sizeof(int) * ct.size())) != cudaSuccess ||
        (e = cudaMalloc(&bp.W, per)) != cudaSuccess || (e = cudaMalloc(&bp.V, per)) != cudaSuccess ||
        (e = cudaMalloc(&bp.Bt, per)) != cudaSuccess ||
        (e = cudaMalloc(&bp.tm, es * (size_t)g.h->N * g.h->N * bp.tm_cap)) != cudaSuccess ||
        (e = cudaMemcpy(bp.traj, tr.data(), sizeof(BatchTraj) * tr.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(bp.chunk_traj, ct.data(), sizeof(int) * ct.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return MAP_ERR_CUDA;
    return MAP_OK;
}

// time the (K, B) candidates on the caller's arrays; keep the fastest
map_status autotune(map_batch* b, map_batch::Group& g, const void* y, void* x)
{
    const Ops* ops = find_ops(g.h->model, g.h->N, g.h->M, g.h->prec);
    struct Cand { int K, B; };
    std::vector<Cand> cands;
    for (int B : {32, 64, 128}) {       // the scan kernels are built for <= 128 threads
        if (!geometry_fits(*g.h, B)) continue;
        const int kb = balanced_steps_per_thread(*g.h, B);
        for (int K : {8, 16, kb})
            if (K != kb || (kb != 8 && kb != 16)) cands.push_back({K, B});
    }
    size_t need = 0;
    for (const Cand& c : cands) {
        set_geometry(*g.h, c.K, c.B);
        need = std::max(need, ops->workspace_bytes(*g.h));
    }
    if (map_status s = ensure_workspace(*g.h, need); s != MAP_OK) return bfail(b, s, g.h->err);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Cand pick = cands.front();
    for (const Cand& c : cands) {
        set_geometry(*g.h, c.K, c.B);
        if (map_status s = solve_group(g, y, x, g.stream); s != MAP_OK) return bfail(b, s, g.h->err);
        float tot = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, g.stream);
            if (map_status s = solve_group(g, y, x, g.stream); s != MAP_OK) return bfail(b, s, g.h->err);
            cudaEventRecord(e1, g.stream);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) return bfail(b, MAP_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            tot += ms;
        }
        if (tot < best) { best = tot; pick = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_geometry(*g.h, pick.K, pick.B);
    g.tuned = true;
    return MAP_OK;
}

}  // namespace

extern "C" {

map_status map_batch_create(map_batch** out, const map_problem_desc* models, int nmodels,
                            const int64_t* lengths, const int* model_of, int ntraj)
{
    if (!out || !models || !lengths || !model_of || nmodels < 1 || ntraj < 1)
        return bfail(nullptr, MAP_ERR_INVALID_ARG, "out, models, lengths and model_of are required");
    *out = nullptr;
    map_batch* b = new map_batch();
    b->nmodels = nmodels;
    for (int j = 0; j < ntraj; ++j) {
        if (model_of[j] < 0 || model_of[j] >= nmodels) {
            destroy_batch(b);
            return bfail(nullptr, MAP_ERR_INVALID_ARG, "model index out of range");
        }
        if (lengths[j] < 1) {
            destroy_batch(b);
            return bfail(nullptr, MAP_ERR_SHAPE, "every trajectory needs at least one interval");
        }
    }
    cudaError_t e;
    for (int m = 0; m < nmodels; ++m) {
        std::vector<long long> starts;
        std::vector<long> rows, lens;
        long pos = 0;
        int cnt = 0;
        for (int j = 0; j < ntraj; ++j) {
            if (model_of[j] != m) continue;
            if (cnt > 0) { starts.push_back(pos); pos += 1; }   // the inserted prior element
            rows.push_back(pos);
            lens.push_back((long)lengths[j]);
            pos += lengths[j];
            ++cnt;
        }
        if (cnt == 0) continue;
        if (models[m].model != MAP_MODEL_LINEAR || models[m].smoother != MAP_RTS || models[m].nx > 6) {
            destroy_batch(b);
            return bfail(nullptr, MAP_ERR_UNSUPPORTED, "batches hold linear models with nx <= 6 and the RTS smoother");
        }
        map_batch::Group g;
        g.model = m;
        g.ntraj = cnt;
        g.y_rows = pos;
        g.x_rows = pos + 1;
        map_problem_desc d = models[m];
        d.T = pos;
        map_status s = create_handle(&g.h, &d);
        if (s != MAP_OK) {
            const std::string msg = map_smoother_last_error(nullptr);
            destroy_batch(b);
            return bfail(nullptr, s, msg);
        }
        if ((e = cudaMalloc(&g.d_reset, (size_t)pos)) != cudaSuccess ||
            (e = cudaMemset(g.d_reset, 0, (size_t)pos)) != cudaSuccess) {
            b->groups.push_back(g);
            destroy_batch(b);
            return bfail(nullptr, MAP_ERR_CUDA, std::string("reset flags: ") + cudaGetErrorString(e));
        }
        if (!starts.empty()) {
            long long* d_pos = nullptr;
            e = cudaMalloc(&d_pos, sizeof(long long) * starts.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(d_pos, starts.data(), sizeof(long long) * starts.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) {
                k_mark_resets<<<(int)((starts.size() + 255) / 256), 256>>>(d_pos, (int)starts.size(), g.d_reset);
                e = cudaDeviceSynchronize();
            }
            if (d_pos) cudaFree(d_pos);
            if (e != cudaSuccess) {
                b->groups.push_back(g);
                destroy_batch(b);
                return bfail(nullptr, MAP_ERR_CUDA, std::string("reset flags: ") + cudaGetErrorString(e));
            }
        }
        const Ops* gops = find_ops(g.h->model, g.h->N, g.h->M, g.h->prec);
        if (gops && gops->batch && plan_chunks(g, rows, lens) != MAP_OK) {
            b->groups.push_back(g);
            destroy_batch(b);
            return bfail(nullptr, MAP_ERR_CUDA, "chunk tables of the batch");
        }
        cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
        b->groups.push_back(g);
    }
    cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    *out = b;
    return MAP_OK;
}

map_status map_batch_rows(const map_batch* b, int model, int64_t* y_rows, int64_t* x_rows)
{
    if (!b || !y_rows || !x_rows || model < 0 || model >= b->nmodels) return MAP_ERR_INVALID_ARG;
    *y_rows = 0;
    *x_rows = 0;
    for (const auto& g : b->groups)
        if (g.model == model) { *y_rows = g.y_rows; *x_rows = g.x_rows; }
    return MAP_OK;
}

map_status map_batch_solve(map_batch* b, const void* const* y, void* const* x, void* stream)
{
    if (!b || !y || !x) return bfail(b, MAP_ERR_INVALID_ARG, "b, y and x are required");
    for (const auto& g : b->groups)
        if (!y[g.model] || !x[g.model] || (reinterpret_cast<size_t>(y[g.model]) & 15) ||
            (reinterpret_cast<size_t>(x[g.model]) & 15))
            return bfail(b, MAP_ERR_INVALID_ARG, "every model with trajectories needs 16-byte aligned y and x");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    // first call: plan the chunked solve of every group, else autotune its
    // segmented scan (eager launches on its own stream)
    for (auto& g : b->groups)
        if (!g.tuned) {
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
                return bfail(b, MAP_ERR_CUDA, cudaGetErrorString(e));
            const Ops* ops = find_ops(g.h->model, g.h->N, g.h->M, g.h->prec);
            if (ops->batch && g.bp.traj) {
                const map_status s = ops->batch(*g.h, g.bp, y[g.model], x[g.model], g.stream);
                if (s == MAP_OK) {
                    g.chunked = true;
                    g.tuned = true;
                    if ((e = cudaStreamSynchronize(g.stream)) != cudaSuccess)
                        return bfail(b, MAP_ERR_CUDA, cudaGetErrorString(e));
                    continue;
                }
                if (s != MAP_ERR_UNSUPPORTED) return bfail(b, s, g.h->err);
            }
            if (map_status s = autotune(b, g, y[g.model], x[g.model]); s != MAP_OK) return s;
        }
    std::vector<const void*> key;
    for (const auto& g : b->groups) { key.push_back(y[g.model]); key.push_back(x[g.model]); }
    if (!b->exec || key != b->key) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return bfail(b, MAP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        cudaEventRecord(b->fork, b->cap);
        map_status s = MAP_OK;
        for (auto& g : b->groups) {
            cudaStreamWaitEvent(g.stream, b->fork, 0);
            if (s == MAP_OK) s = solve_group(g, y[g.model], x[g.model], g.stream);
            cudaEventRecord(g.done, g.stream);
            cudaStreamWaitEvent(b->cap, g.done, 0);
        }
        e = cudaStreamEndCapture(b->cap, &b->graph);
        if (s != MAP_OK) return bfail(b, s, "capture of the batch launches failed");
        if (e != cudaSuccess) return bfail(b, MAP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
            return bfail(b, MAP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        b->key = key;
    }
    if ((e = cudaGraphLaunch(b->exec, st)) != cudaSuccess)
        return bfail(b, MAP_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return MAP_OK;
}

map_status map_batch_tuning(const map_batch* b, int model, int* K, int* B)
{
    if (!b || !K || !B) return MAP_ERR_INVALID_ARG;
    *K = 0;
    *B = 0;
    for (const auto& g : b->groups)
        if (g.model == model) {
            *K = g.chunked ? BATCH_CH : g.h->K;        // chunked: steps per chunk, one thread each
            *B = g.chunked ? 128 : g.h->B;
        }
    return MAP_OK;
}

const char* map_batch_last_error(const map_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

void map_batch_destroy(map_batch* b) { destroy_batch(b); }

}  // extern "C"
