// FMA-throughput measurement (map_fma_peak): the denominators of the ALU
// rooflines of this library's kernels, measured on the GPU they run on rather
// than taken from unit counts and the maximum clock.
//
// Every thread runs CH independent multiply-add chains acc <- acc * a + b for
// `iters` rounds (a, b kernel arguments, so nothing folds at compile time;
// |a| < 1 keeps the values bounded).  The grid is 8 CTAs of 256 threads per
// SM (64 warps per SM, 16 per scheduler), so every FMA pipe sees enough
// independent instructions to issue back to back.  Kinds:
//   0  FP32 scalar FFMA
//   1  FP32 paired FMA (__ffma2_rn on float2: two FMAs per instruction)
//   2  FP64 DFMA
// The result of every chain feeds one store into a file-scope __device__ sink,
// guarded by a condition the values never meet, so the compiler keeps the work.
#include <cuda_runtime.h>

#include "../../include/map_smoother.h"

namespace {

constexpr int CH = 8;             // independent chains per thread
constexpr int THREADS = 256;
constexpr int CTAS_PER_SM = 8;

__device__ float g_sink32[THREADS];
__device__ double g_sink64[THREADS];

__device__ __forceinline__ float* sink_of(float) { return g_sink32; }
__device__ __forceinline__ double* sink_of(double) { return g_sink64; }

template <typename S>
__global__ void __launch_bounds__(THREADS) k_fma_chains(int iters, S a, S b)
{
    S acc[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) acc[i] = S(threadIdx.x) * S(1e-3) + S(i);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int i = 0; i < CH; ++i) acc[i] = fma(acc[i], a, b);
    }
    S s = S(0);
#pragma unroll
    for (int i = 0; i < CH; ++i) s += acc[i];
    if (s == S(-12345.0)) sink_of(s)[threadIdx.x] = s;
}

__global__ void __launch_bounds__(THREADS) k_fma2_chains(int iters, float a, float b)
{
    float2 acc[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) acc[i] = make_float2(float(threadIdx.x) * 1e-3f + float(i), float(i) - 0.5f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int i = 0; i < CH; ++i) acc[i] = __ffma2_rn(acc[i], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += acc[i].x + acc[i].y;
    if (s == -12345.0f) g_sink32[threadIdx.x] = s;
}

}  // namespace

extern "C" map_status map_fma_peak(int kind, int iters, double* flop_out, float* ms_out, void* stream)
{
    if (!flop_out || !ms_out || iters < 1 || kind < 0 || kind > 2) return MAP_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return MAP_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = sms * CTAS_PER_SM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return MAP_ERR_CUDA;
    }
    cudaEventRecord(e0, st);
    if (kind == 0)
        k_fma_chains<float><<<grid, THREADS, 0, st>>>(iters, 0.9999999f, 1e-7f);
    else if (kind == 1)
        k_fma2_chains<<<grid, THREADS, 0, st>>>(iters, 0.9999999f, 1e-7f);
    else
        k_fma_chains<double><<<grid, THREADS, 0, st>>>(iters, 0.9999999999, 1e-12);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return MAP_ERR_CUDA;
    const double fma_per_thread = double(iters) * 16.0 * CH * (kind == 1 ? 2.0 : 1.0);
    *flop_out = 2.0 * fma_per_thread * double(grid) * THREADS;
    *ms_out = ms;
    return MAP_OK;
}
