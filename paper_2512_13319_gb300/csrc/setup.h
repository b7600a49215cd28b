// Shared host/device declarations of the model set-up kernel.
#pragma once
#include <cuda_runtime.h>

namespace mapk {

constexpr int MAXN = 8;
constexpr int MAXM = 8;
// doubles of the set-up inputs F, c, L, W, H, r, R, m0, P0 at the largest
// sizes (6 matrices and 3 vectors of order 8), rounded up
constexpr int SETUP_IN_CAP = 512;

enum SetupFlags { SETUP_SINGULAR_R = 1, SETUP_SINGULAR_P0 = 2, SETUP_SINGULAR_A = 4, SETUP_SINGULAR_Q = 8,
                  SETUP_SINGULAR_C = 16 };

// device pointers to FP64 row-major inputs
struct SetupIn {
    int nx, ny, nw, mode;
    int substeps;                      // block elements (mode 3)
    double dt;
    const double *F, *c, *L, *W, *H, *r, *R, *m0, *P0;
};

// FP64 outputs (full matrices, row-major, leading dimension = actual size)
struct SetupOut {
    double Q[MAXN * MAXN], Qinv[MAXN * MAXN];
    double A[MAXN * MAXN], b[MAXN], C[MAXN * MAXN], Cinv[MAXN * MAXN];
    double Rinv[MAXM * MAXM], G[MAXN * MAXM], Gr[MAXN], J[MAXN * MAXN];
    double S0[MAXN * MAXN], v0[MAXN];
    double Phi[MAXN * MAXN], beta[MAXN], Sigma[MAXN * MAXN];
    double Gam[MAXN * MAXN];           // C = Gam Gam^T, Gam n x rank (leading dimension n)
    double Gpinv[MAXN * MAXN];         // (Gam^T Gam)^-1 Gam^T, rank x n (leading dimension n)
    int rank;                          // numerical rank of C (pivoted Cholesky, relative 1e-13)
    int flags;
    // block and exact elements (modes 3, 4): b = Bb y + b and eta = G y - Gr are
    // affine in the interval's sample y; Bb = 0 for the other modes
    double Bb[MAXN * MAXM];
    // one substep element of mode 3 (dense output): A, b, C, J, and eta = sG (y - r)
    double sA[MAXN * MAXN], sb[MAXN], sC[MAXN * MAXN], sJ[MAXN * MAXN], sG[MAXN * MAXM], sGr[MAXN];
};

cudaError_t launch_setup(const SetupIn& in, SetupOut* d_out, cudaStream_t st);

// FP64 constants of the discrete cost of a linear model
template <int N, int M>
struct LinCostParams {
    double A[N * N], b[N], Cinv[N * N], H[M * N], r[M], Rinv[M * M], S0[N * N], m0[N];
    double IA[N * N];                  // I - A (dt F for the Euler element), formed in FP64
    double dt, trF;
};

}  // namespace mapk
