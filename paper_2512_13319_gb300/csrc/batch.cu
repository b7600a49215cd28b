// Batched solve: many independent trajectories of a few linear models.
//
// Trajectories of the same model are stored concatenated, one spare row
// between them.  Every trajectory starts from its model's prior, so the
// data-independent part of its solve (the filter's P_k and closed-loop maps)
// is that of the model's per-step tables at its local step.  When every
// model's tables reach the stationary filter, the whole batch is ONE launch of
// the persistent kernel of batch_persist.cu (all models, all trajectories,
// longest first), captured into a CUDA graph; its threads per CTA and steps
// per thread are chosen on the first call by timing the candidates on the
// caller's arrays (autotuning).  Otherwise every model takes the segmented
// scan: its trajectories form one scan with the prior element at every
// trajectory start (see SegLtiProducer), with its own autotuned (K, B), and the
// per-model launches are captured into one graph with concurrent branches.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "batch_persist.h"
#include "handle.h"

using namespace mapk;

struct map_batch {
    struct Group {
        int model = -1;
        map_smoother* h = nullptr;
        unsigned char* d_reset = nullptr;  // segmented scan: trajectory starts
        std::vector<long long> starts;
        long y_rows = 0, x_rows = 0;
        int ntraj = 0;
        cudaStream_t stream = nullptr;
        cudaEvent_t done = nullptr;
        bool tuned = false;
    };
    int nmodels = 0;
    int prec = MAP_FP32;
    std::vector<Group> groups;
    int mode = 0;                      // 0: not planned, 1: persistent kernel, 2: segmented scans
    // the persistent solve
    std::vector<BpItem> items;         // longest trajectory first
    std::vector<int> item_N;           // state dimension of each item's model
    std::vector<unsigned char> mrec;   // host BpModel<S> records, one per model
    size_t mrec_size = 0;
    void* d_models = nullptr;
    BpItem* d_items = nullptr;
    void* d_scr = nullptr;
    unsigned* d_ctr = nullptr;
    int KB = 0, B = 0, grid = 0, Nmax = 0, Mmax = 0;
    size_t smem = 0;
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
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.done) cudaEventDestroy(g.done);
    }
    if (b->d_models) cudaFree(b->d_models);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_scr) cudaFree(b->d_scr);
    if (b->d_ctr) cudaFree(b->d_ctr);
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

// the segmented scan's reset flags of one model (eager, synchronising)
map_status make_resets(map_batch* b, map_batch::Group& g)
{
    cudaError_t e;
    if ((e = cudaMalloc(&g.d_reset, (size_t)g.y_rows)) != cudaSuccess ||
        (e = cudaMemset(g.d_reset, 0, (size_t)g.y_rows)) != cudaSuccess)
        return bfail(b, MAP_ERR_CUDA, std::string("reset flags: ") + cudaGetErrorString(e));
    if (g.starts.empty()) return MAP_OK;
    long long* d_pos = nullptr;
    e = cudaMalloc(&d_pos, sizeof(long long) * g.starts.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(d_pos, g.starts.data(), sizeof(long long) * g.starts.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_mark_resets<<<(int)((g.starts.size() + 255) / 256), 256>>>(d_pos, (int)g.starts.size(), g.d_reset);
        e = cudaDeviceSynchronize();
    }
    if (d_pos) cudaFree(d_pos);
    if (e != cudaSuccess) return bfail(b, MAP_ERR_CUDA, std::string("reset flags: ") + cudaGetErrorString(e));
    return MAP_OK;
}

map_status solve_group(map_batch::Group& g, const void* y, void* x, cudaStream_t st)
{
    const Ops* ops = find_ops(g.h->model, g.h->N, g.h->M, g.h->prec);
    return ops->solve_seg(*g.h, y, g.d_reset, x, st);
}

// time the (K, B) candidates of a model's segmented scan on the caller's
// arrays; keep the fastest
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

// ---- the persistent solve

template <typename S>
void set_io(unsigned char* rec, const void* y, void* x)
{
    BpModel<S>* m = reinterpret_cast<BpModel<S>*>(rec);
    m->y = static_cast<const S*>(y);
    m->x = static_cast<S*>(x);
}

// the models' records for KB steps per thread (with the caller's arrays) and
// the items' scratch offsets for B KB steps per block, on the device
map_status bp_geometry(map_batch* b, int KB, int B, const void* const* y, void* const* x, cudaStream_t st)
{
    for (auto& g : b->groups) {
        const Ops* ops = find_ops(g.h->model, g.h->N, g.h->M, g.h->prec);
        unsigned char* rec = b->mrec.data() + (size_t)g.model * b->mrec_size;
        if (map_status s = ops->batch_model(*g.h, rec, KB, g.stream); s != MAP_OK) return bfail(b, s, g.h->err);
        if (b->prec == MAP_FP64) set_io<double>(rec, y[g.model], x[g.model]);
        else set_io<float>(rec, y[g.model], x[g.model]);
    }
    const long BS = (long)B * KB;
    long off = 0;
    for (size_t i = 0; i < b->items.size(); ++i) {
        b->items[i].scr = off;
        off += (b->items[i].L + BS - 1) / BS * B * b->item_N[i];
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->d_models, b->mrec.data(), b->mrec.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->d_items, b->items.data(), sizeof(BpItem) * b->items.size(), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return bfail(b, MAP_ERR_CUDA, std::string("batch records: ") + cudaGetErrorString(e));
    b->KB = KB;
    b->B = B;
    return MAP_OK;
}

cudaError_t bp_run(map_batch* b, cudaStream_t st)
{
    return bp_launch(b->prec, b->B, b->grid, b->smem, b->d_models, b->d_items, (int)b->items.size(), b->KB, b->Nmax,
                     b->Mmax, b->d_scr, b->d_ctr, st);
}

// Plan the persistent solve: every model's record (its step tables), then
// time the candidate geometries (threads per CTA B, steps per thread KB) on the
// caller's arrays and keep the fastest.  MAP_ERR_UNSUPPORTED when a model's
// tables do not reach the stationary filter.
map_status bp_plan(map_batch* b, const void* const* y, void* const* x, cudaStream_t st)
{
    const size_t es = b->prec == MAP_FP64 ? 8 : 4;
    b->mrec_size = b->prec == MAP_FP64 ? sizeof(BpModel<double>) : sizeof(BpModel<float>);
    b->mrec.assign(b->mrec_size * b->nmodels, 0);
    for (auto& g : b->groups) {
        const Ops* ops = find_ops(g.h->model, g.h->N, g.h->M, g.h->prec);
        if (!ops->batch_model || !bp_shape_supported(g.h->N, g.h->M)) return MAP_ERR_UNSUPPORTED;
        map_status s = ops->batch_model(*g.h, b->mrec.data() + (size_t)g.model * b->mrec_size, 8, g.stream);
        if (s == MAP_ERR_UNSUPPORTED) return s;
        if (s != MAP_OK) return bfail(b, s, g.h->err);
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    struct Cand { int B, KB; size_t smem; int grid; };
    std::vector<Cand> cands;
    size_t scr_need = 0;
    for (int B : {64, 128})
        for (int KB : {8, 12, 16}) {
            const size_t smem = bp_smem_bytes(b->prec, B, KB, b->Nmax, b->Mmax);
            const int occ = bp_blocks_per_sm(b->prec, B, smem);
            if (occ < 1) continue;
            const int grid = (int)std::min<long>((long)occ * nsm, (long)b->items.size());
            cands.push_back({B, KB, smem, grid});
            const long BS = (long)B * KB;
            size_t need = 0;
            for (size_t i = 0; i < b->items.size(); ++i)
                need += (size_t)((b->items[i].L + BS - 1) / BS) * B * b->item_N[i];
            scr_need = std::max(scr_need, need * es);
        }
    if (cands.empty()) return bfail(b, MAP_ERR_UNSUPPORTED, "no geometry of the persistent batch kernel fits");
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_models, b->mrec.size())) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&b->d_items), sizeof(BpItem) * b->items.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_scr, scr_need)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&b->d_ctr), 2 * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(b->d_ctr, 0, 2 * sizeof(unsigned))) != cudaSuccess)
        return bfail(b, MAP_ERR_CUDA, std::string("batch buffers: ") + cudaGetErrorString(e));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Cand pick = cands.front();
    for (const Cand& c : cands) {
        if (map_status s = bp_geometry(b, c.KB, c.B, y, x, st); s != MAP_OK) return s;
        b->smem = c.smem;
        b->grid = c.grid;
        float tot = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            if ((e = bp_run(b, st)) != cudaSuccess)
                return bfail(b, MAP_ERR_CUDA, std::string("batch kernel launch: ") + cudaGetErrorString(e));
            cudaEventRecord(e1, st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess)
                return bfail(b, MAP_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tot += ms;                // the first run warms up
        }
        if (tot < best) { best = tot; pick = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (map_status s = bp_geometry(b, pick.KB, pick.B, y, x, st); s != MAP_OK) return s;
    b->smem = pick.smem;
    b->grid = pick.grid;
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
    b->prec = models[0].precision;
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
    for (int m = 0; m < nmodels; ++m) {
        map_batch::Group g;
        long pos = 0;
        int cnt = 0;
        for (int j = 0; j < ntraj; ++j) {
            if (model_of[j] != m) continue;
            if (cnt > 0) { g.starts.push_back(pos); pos += 1; }   // the spare row (segmented scan: the prior element)
            b->items.push_back(BpItem{m, j, pos, (long)lengths[j], 0});
            b->item_N.push_back(models[m].nx);
            pos += lengths[j];
            ++cnt;
        }
        if (cnt == 0) continue;
        if (models[m].model != MAP_MODEL_LINEAR || models[m].smoother != MAP_RTS || models[m].nx > BP_NMAX) {
            destroy_batch(b);
            return bfail(nullptr, MAP_ERR_UNSUPPORTED, "batches hold linear models with nx <= 6 and the RTS smoother");
        }
        if (models[m].precision != b->prec) {
            destroy_batch(b);
            return bfail(nullptr, MAP_ERR_INVALID_ARG, "every model of a batch has the same precision");
        }
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
        b->Nmax = std::max(b->Nmax, g.h->N);
        b->Mmax = std::max(b->Mmax, g.h->M);
        cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
        b->groups.push_back(std::move(g));
    }
    // the persistent kernel's work list: longest trajectory first
    std::vector<size_t> ord(b->items.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t p, size_t q) { return b->items[p].L > b->items[q].L; });
    std::vector<BpItem> it2(ord.size());
    std::vector<int> n2(ord.size());
    for (size_t i = 0; i < ord.size(); ++i) {
        it2[i] = b->items[ord[i]];
        n2[i] = b->item_N[ord[i]];
    }
    b->items.swap(it2);
    b->item_N.swap(n2);
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
    std::vector<const void*> key;
    for (const auto& g : b->groups) { key.push_back(y[g.model]); key.push_back(x[g.model]); }
    // first call: plan the persistent solve, else every model's segmented scan
    // (eager launches, synchronising)
    if (b->mode == 0) {
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bfail(b, MAP_ERR_CUDA, cudaGetErrorString(e));
        const map_status s = bp_plan(b, y, x, st);
        if (s == MAP_OK) {
            b->mode = 1;
            b->key = key;
        } else if (s == MAP_ERR_UNSUPPORTED && b->err.empty()) {
            b->mode = 2;
            for (auto& g : b->groups) {
                if (map_status s2 = make_resets(b, g); s2 != MAP_OK) return s2;
                if (map_status s2 = autotune(b, g, y[g.model], x[g.model]); s2 != MAP_OK) return s2;
            }
        } else {
            return s;
        }
    }
    if (b->mode == 1) {
        if (key != b->key) {          // new arrays: the records' pointers (stream-ordered)
            for (auto& g : b->groups) {
                unsigned char* rec = b->mrec.data() + (size_t)g.model * b->mrec_size;
                if (b->prec == MAP_FP64) set_io<double>(rec, y[g.model], x[g.model]);
                else set_io<float>(rec, y[g.model], x[g.model]);
            }
            if ((e = cudaMemcpyAsync(b->d_models, b->mrec.data(), b->mrec.size(), cudaMemcpyHostToDevice, st)) !=
                cudaSuccess)
                return bfail(b, MAP_ERR_CUDA, std::string("batch records: ") + cudaGetErrorString(e));
            b->key = key;
        }
        if (!b->exec) {
            if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return bfail(b, MAP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
            const cudaError_t el = bp_run(b, b->cap);
            e = cudaStreamEndCapture(b->cap, &b->graph);
            if (el != cudaSuccess) return bfail(b, MAP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(el));
            if (e != cudaSuccess) return bfail(b, MAP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
            if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
                return bfail(b, MAP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        if ((e = cudaGraphLaunch(b->exec, st)) != cudaSuccess)
            return bfail(b, MAP_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
        return MAP_OK;
    }
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
    if (b->mode == 1) {                // the persistent kernel: steps per thread, threads per CTA
        *K = b->KB;
        *B = b->B;
        return MAP_OK;
    }
    for (const auto& g : b->groups)
        if (g.model == model && g.tuned) {
            *K = g.h->K;
            *B = g.h->B;
        }
    return MAP_OK;
}

const char* map_batch_last_error(const map_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

void map_batch_destroy(map_batch* b) { destroy_batch(b); }

int map_batch_persistent(const map_batch* b) { return b && b->mode == 1 ? 1 : 0; }

}  // extern "C"
