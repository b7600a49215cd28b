// Model set-up on the device, in FP64: turns the problem statement (F, c, L,
// W, H, r, R, m0, P0, dt) into the constant parts of the interval elements.
//
//   Q = L W L^T
//   Euler (Section 5.1, one explicit Euler step of Eq. 37 from A=I, b=C=0):
//       A = I - dt F,  b = -dt c,  C = dt Q
//   exact (constant coefficients, Eq. 37 rows A, b, C with J = eta = 0):
//       A = e^{-F dt},  C = int_0^dt e^{-F u} Q e^{-F^T u} du,
//       b = -int_0^dt e^{-F u} du c
//     from one block exponential of Z = [[-F dt, Q dt, -c dt], [0, F^T dt, 0], [0, 0, 0]]:
//       e^Z = [[A, G, b], [0, e^{F^T dt}, 0], [0, 0, 1]],  C = G A^T.
//     The exponential is a degree-24 Taylor polynomial of Z / 2^s with
//     |Z / 2^s|_1 <= 1/4, squared s times (scaling and squaring).
//   Measurement: Rinv = R^-1, G = dt H^T R^-1, J = G H, Gr = G r
//   Prior (terminal element a_T of Eq. 31): S0 = P0^-1, v0 = S0 m0
//   Forward transition of the element: Phi = A^-1, beta = -A^-1 b, Sigma = A^-1 C A^-T
//
// One CTA; matrices of order <= 2*8+1 live in shared memory.
#include <cuda_runtime.h>
#include "setup.h"

namespace mapk {

#define MAXD 17   // 2 * 8 + 1

struct SetupShared {
    double Z[MAXD * MAXD], E[MAXD * MAXD], T1[MAXD * MAXD], T2[MAXD * MAXD];
    double X[8 * 8], Y[8 * 8];
    double pivw[2 * MAXD * MAXD];
    int flag;
};

// c (n x p) = a (n x k) b (k x p), all threads
__device__ void bmm(const double* a, const double* b, double* c, int n, int k, int p)
{
    for (int e = threadIdx.x; e < n * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        double s = 0.0;
        for (int l = 0; l < k; ++l) s = fma(a[i * k + l], b[l * p + j], s);
        c[e] = s;
    }
    __syncthreads();
}

// inverse by Gauss-Jordan with partial pivoting, thread 0; returns false if singular
__device__ bool binv(const double* a, double* x, int n, double* w)
{
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        const int m = 2 * n;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < m; ++j) w[i * m + j] = j < n ? a[i * n + j] : (j - n == i ? 1.0 : 0.0);
        for (int c = 0; c < n && ok; ++c) {
            int p = c;
            for (int r = c + 1; r < n; ++r)
                if (fabs(w[r * m + c]) > fabs(w[p * m + c])) p = r;
            if (w[p * m + c] == 0.0) { ok = 0; break; }
            if (p != c)
                for (int j = 0; j < m; ++j) { double t = w[c * m + j]; w[c * m + j] = w[p * m + j]; w[p * m + j] = t; }
            const double d = 1.0 / w[c * m + c];
            for (int j = 0; j < m; ++j) w[c * m + j] *= d;
            for (int r = 0; r < n; ++r) {
                if (r == c) continue;
                const double f = w[r * m + c];
                for (int j = 0; j < m; ++j) w[r * m + j] -= f * w[c * m + j];
            }
        }
        if (ok)
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) x[i * n + j] = w[i * m + n + j];
    }
    __syncthreads();
    return ok != 0;
}

// E = exp(Z) for Z of order d (in shared memory), all threads
__device__ void bexpm(SetupShared& s, int d)
{
    __shared__ int sq;
    if (threadIdx.x == 0) {
        double nrm = 0.0;
        for (int j = 0; j < d; ++j) {
            double c = 0.0;
            for (int i = 0; i < d; ++i) c += fabs(s.Z[i * d + j]);
            nrm = c > nrm ? c : nrm;
        }
        int k = 0;
        while (nrm > 0.25) { nrm *= 0.5; ++k; }
        sq = k;
    }
    __syncthreads();
    const double sc = ldexp(1.0, -sq);
    for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
        s.Z[e] *= sc;
        s.E[e] = (e / d == e % d) ? 1.0 : 0.0;
        s.T1[e] = s.E[e];
    }
    __syncthreads();
    // Horner-free accumulation: term_k = term_{k-1} Z / k
    for (int k = 1; k <= 24; ++k) {
        bmm(s.T1, s.Z, s.T2, d, d, d);
        for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
            s.T1[e] = s.T2[e] / k;
            s.E[e] += s.T1[e];
        }
        __syncthreads();
    }
    for (int k = 0; k < sq; ++k) {
        bmm(s.E, s.E, s.T2, d, d, d);
        for (int e = threadIdx.x; e < d * d; e += blockDim.x) s.E[e] = s.T2[e];
        __syncthreads();
    }
}

__global__ void k_setup(SetupIn in, SetupOut* out)
{
    __shared__ SetupShared s;
    const int n = in.nx, m = in.ny, nw = in.nw;
    const double dt = in.dt;
    if (threadIdx.x == 0) s.flag = 0;
    __syncthreads();
    // Q = L W L^T
    bmm(in.L, in.W, s.T1, n, nw, nw);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        double acc = 0.0;
        for (int l = 0; l < nw; ++l) acc = fma(s.T1[i * nw + l], in.L[j * nw + l], acc);
        out->Q[e] = acc;
    }
    __syncthreads();
    if (in.mode == 0) {
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e / n, j = e % n;
            out->A[e] = (i == j ? 1.0 : 0.0) - dt * in.F[e];
            out->C[e] = dt * out->Q[e];
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) out->b[i] = -dt * in.c[i];
        __syncthreads();
    } else {
        const int d = 2 * n + 1;
        for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
            const int i = e / d, j = e % d;
            double z = 0.0;
            if (i < n && j < n) z = -in.F[i * n + j] * dt;
            else if (i < n && j < 2 * n) z = out->Q[i * n + (j - n)] * dt;
            else if (i < n && j == 2 * n) z = -in.c[i] * dt;
            else if (i >= n && i < 2 * n && j >= n && j < 2 * n) z = in.F[(j - n) * n + (i - n)] * dt;
            s.Z[e] = z;
        }
        __syncthreads();
        bexpm(s, d);
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e / n, j = e % n;
            out->A[e] = s.E[i * d + j];
            s.X[e] = s.E[i * d + n + j];          // G
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) out->b[i] = s.E[i * d + 2 * n];
        __syncthreads();
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e / n, j = e % n;
            double acc = 0.0;
            for (int l = 0; l < n; ++l) acc = fma(s.X[i * n + l], out->A[j * n + l], acc);
            s.Y[e] = acc;                         // G A^T
        }
        __syncthreads();
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e / n, j = e % n;
            out->C[e] = 0.5 * (s.Y[i * n + j] + s.Y[j * n + i]);
        }
        __syncthreads();
    }
    // measurement
    if (!binv(in.R, out->Rinv, m, s.pivw)) { if (threadIdx.x == 0) s.flag |= SETUP_SINGULAR_R; }
    __syncthreads();
    for (int e = threadIdx.x; e < n * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc = fma(in.H[l * n + i], out->Rinv[l * m + j], acc);
        out->G[e] = dt * acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc = fma(out->G[i * m + l], in.H[l * n + j], acc);
        s.Y[e] = acc;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc = fma(out->G[i * m + l], in.r[l], acc);
        out->Gr[i] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        out->J[e] = 0.5 * (s.Y[i * n + j] + s.Y[j * n + i]);
    }
    // prior
    if (!binv(in.P0, out->S0, n, s.pivw)) { if (threadIdx.x == 0) s.flag |= SETUP_SINGULAR_P0; }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < n; ++l) acc = fma(out->S0[i * n + l], in.m0[l], acc);
        out->v0[i] = acc;
    }
    __syncthreads();
    // forward transition
    if (!binv(out->A, out->Phi, n, s.pivw)) { if (threadIdx.x == 0) s.flag |= SETUP_SINGULAR_A; }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < n; ++l) acc = fma(out->Phi[i * n + l], out->b[l], acc);
        out->beta[i] = -acc;
    }
    bmm(out->Phi, out->C, s.T1, n, n, n);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        double acc = 0.0;
        for (int l = 0; l < n; ++l) acc = fma(s.T1[i * n + l], out->Phi[j * n + l], acc);
        out->Sigma[e] = acc;
    }
    __syncthreads();
    // Q^-1 and C^-1 when they exist (cost and gradient)
    if (!binv(out->Q, out->Qinv, n, s.pivw)) { if (threadIdx.x == 0) s.flag |= SETUP_SINGULAR_Q; }
    __syncthreads();
    if (!binv(out->C, out->Cinv, n, s.pivw)) { if (threadIdx.x == 0) s.flag |= SETUP_SINGULAR_C; }
    __syncthreads();
    // C = Gam Gam^T by outer-product Cholesky with diagonal pivoting: each
    // column takes the largest remaining diagonal; stop when it falls below
    // 1e-13 of the largest diagonal of C (the numerical rank)
    if (threadIdx.x == 0) {
        double* Rm = s.pivw;
        double dmax = 0.0;
        for (int e = 0; e < n * n; ++e) Rm[e] = out->C[e];
        for (int i = 0; i < n; ++i) dmax = fmax(dmax, Rm[i * n + i]);
        for (int e = 0; e < n * n; ++e) out->Gam[e] = 0.0;
        int rk = 0;
        for (; rk < n; ++rk) {
            int p = 0;
            for (int i = 1; i < n; ++i)
                if (Rm[i * n + i] > Rm[p * n + p]) p = i;
            const double d = Rm[p * n + p];
            if (!(d > 1e-13 * dmax) || dmax <= 0.0) break;
            const double sd = sqrt(d);
            for (int i = 0; i < n; ++i) out->Gam[i * n + rk] = Rm[i * n + p] / sd;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) Rm[i * n + j] -= out->Gam[i * n + rk] * out->Gam[j * n + rk];
        }
        out->rank = rk;
        // pseudo-inverse of Gam: (Gam^T Gam)^-1 Gam^T by Gauss-Jordan on the rank x rank Gram matrix
        double* Gm = s.pivw;                    // rk x rk, then its inverse beside it
        double* Gi = s.pivw + MAXN * MAXN;
        for (int a = 0; a < rk; ++a)
            for (int c = 0; c < rk; ++c) {
                double acc = 0.0;
                for (int i = 0; i < n; ++i) acc += out->Gam[i * n + a] * out->Gam[i * n + c];
                Gm[a * rk + c] = acc;
                Gi[a * rk + c] = a == c ? 1.0 : 0.0;
            }
        for (int col = 0; col < rk; ++col) {   // symmetric positive definite: no pivoting needed
            const double ip = 1.0 / Gm[col * rk + col];
            for (int c = 0; c < rk; ++c) { Gm[col * rk + c] *= ip; Gi[col * rk + c] *= ip; }
            for (int r = 0; r < rk; ++r) {
                if (r == col) continue;
                const double f = Gm[r * rk + col];
                for (int c = 0; c < rk; ++c) { Gm[r * rk + c] -= f * Gm[col * rk + c]; Gi[r * rk + c] -= f * Gi[col * rk + c]; }
            }
        }
        for (int e = 0; e < n * n; ++e) out->Gpinv[e] = 0.0;
        for (int a = 0; a < rk; ++a)
            for (int i = 0; i < n; ++i) {
                double acc = 0.0;
                for (int c = 0; c < rk; ++c) acc += Gi[a * rk + c] * out->Gam[i * n + c];
                out->Gpinv[a * n + i] = acc;
            }
        out->flags = s.flag;
    }
}

cudaError_t launch_setup(const SetupIn& in, SetupOut* d_out, cudaStream_t st)
{
    k_setup<<<1, 256, 0, st>>>(in, d_out);
    return cudaGetLastError();
}

}  // namespace mapk
