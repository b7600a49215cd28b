// Descriptors of the persistent batch solve (batch_persist.cuh): one model of
// a batch and one trajectory (work item).  Shared by the host code that fills
// them (solve_impl.cuh batch_model, batch.cu) and the kernel that reads them.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace mapk {

constexpr int BP_NMAX = 6;             // largest state dimension of a batch model

// One linear time-invariant model of a batch.  Every trajectory of the model
// starts from its prior, so the filter factor at local step k is the model's
// tabulated P_k (row min(k, kc) of its step table), and its solve is the
// affine recursion of the step tables in v and x alone:
//   v_{k+1} = E_k^T v_k + o_k + G y_{k+1} - Gr,   g_k = E_k (A^-1 C v_k + A^-1 b),
//   x_k = E_k x_{k+1} + g_k,   x_L = P_L^-1 v_L.
template <typename S>
struct BpModel {
    int N, M;                          // state and observation dimensions
    int RS, oE, oO, oP;                // step-table row stride and offsets (StepTab<N, S>)
    long kc;                           // stationary point: row kc stands for every later step
    const S* rows;                     // step-table rows (device)
    const S* y;                        // the model's observation rows (device, per solve)
    S* x;                              // the model's state rows (device, per solve)
    unsigned long long* stats;         // event words of the model's handle
    S Einf[BP_NMAX * BP_NMAX], oinf[BP_NMAX];      // row kc: E_inf, o_inf
    S PhiK[BP_NMAX * BP_NMAX];                     // E_inf^KB (KB steps per thread)
    S AiC[BP_NMAX * BP_NMAX], Aib[BP_NMAX];        // A^-1 C, A^-1 b
    S EAiC[BP_NMAX * BP_NMAX], EAib[BP_NMAX];      // E_inf A^-1 C, E_inf A^-1 b
    S G[BP_NMAX * BP_NMAX], Gr[BP_NMAX];           // G (N x M), G r
    S v0[BP_NMAX];                                 // the prior's information vector P0^-1 m0
};

// One trajectory: its model, first row in the model's arrays (y rows row ..
// row + L - 1, x rows row .. row + L), length and the offset of its share of
// the forward sweep's scratch (thread start values, ceil(L / (B KB)) B N scalars)
struct BpItem {
    int model;
    int traj;
    long row;
    long L;
    long scr;
};

// Host entry points of the persistent kernel (batch_persist.cu).  prec is
// MAP_FP32 or MAP_FP64, B the threads per CTA (64 or 128), KB the steps per
// thread (even); models points to device BpModel<S> records, items to the
// device work list (longest trajectory first), scr to the thread start values
// (sum over items of ceil(L / (B KB)) B N scalars), ctr to two zeroed words.
bool bp_shape_supported(int N, int M);
size_t bp_smem_bytes(int prec, int B, int KB, int Nmax, int Mmax);
int bp_blocks_per_sm(int prec, int B, size_t smem);
cudaError_t bp_launch(int prec, int B, int grid, size_t smem, const void* models, const BpItem* items, int nitems,
                      int KB, int Nmax, int Mmax, void* scr, unsigned* ctr, cudaStream_t st);

}  // namespace mapk
