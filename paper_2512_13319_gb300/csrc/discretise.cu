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

#define MAXD 32   // 4 * 8 (exact elements); 2 * 8 + 1 for the exponential of mode 1

// working matrices of the block-element composition (mode 3)
struct BlockWork {
    double A[MAXN * MAXN], b0[MAXN], C[MAXN * MAXN], J[MAXN * MAXN];    // accumulated block
    double Bb[MAXN * MAXM], Gy[MAXN * MAXM], g0[MAXN];
    double An[MAXN * MAXN], b0n[MAXN], Cn[MAXN * MAXN], Jn[MAXN * MAXN];  // the next one
    double Bbn[MAXN * MAXM], Gyn[MAXN * MAXM], g0n[MAXN];
    double M[MAXN * MAXN], Mi[MAXN * MAXN], T1[MAXN * MAXN], T2[MAXN * MAXN], T3[MAXN * MAXN];
    double U[MAXN * MAXM], u[MAXN];
};

struct SetupShared {
    union {
        struct { double Z[MAXD * MAXD], E[MAXD * MAXD], T1[MAXD * MAXD], T2[MAXD * MAXD]; };
        BlockWork bw;
    };
    double X[8 * 8], Y[8 * 8];
    double HR[MAXN * MAXM], Wm[MAXN * MAXN];   // H^T R^-1 and H^T R^-1 H (modes 3, 4)
    double inw[6][2 * MAXN * MAXN];        // per-warp scratch of the stage-3 warps
    double Gam[MAXN * MAXN];
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

// |x| ordering of finite FP64 values through their bit patterns (no FP64 op)
__device__ inline unsigned long long absbits(double x)
{
    return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
}

// x = a^-1 (n x n, n <= MAXN) by Gauss-Jordan elimination with partial
// pivoting on [a | I], by the calling warp: lane l updates entries l, l + 32,
// ... of the augmented matrix, reading all of them before any is written.
// Returns false (the same on every lane) at a zero pivot, x then unwritten.
// w: 2 n^2 scratch.  (The FP64 pipe takes a warp instruction at about the
// same cost however many lanes are active, so the lanes share the work.)
__device__ bool winv(const double* a, double* x, int n, double* w)
{
    const int l = threadIdx.x & 31, m = 2 * n, E = n * m;
    for (int e = l; e < E; e += 32) {
        const int i = e / m, j = e - i * m;
        w[e] = j < n ? a[i * n + j] : (j - n == i ? 1.0 : 0.0);
    }
    __syncwarp();
    constexpr int R = (2 * MAXN * MAXN + 31) / 32;
    for (int c = 0; c < n; ++c) {
        int p = c;
        unsigned long long best = absbits(w[c * m + c]);
        for (int r = c + 1; r < n; ++r) {
            const unsigned long long v = absbits(w[r * m + c]);
            if (v > best) { best = v; p = r; }
        }
        const double piv = w[p * m + c];
        if (piv == 0.0) return false;
        const double d = 1.0 / piv;
        // rows c and p swapped, row c scaled, column c eliminated elsewhere
        double nv[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int e = l + 32 * t;
            if (e < E) {
                const int r = e / m, j = e - r * m;
                const double pk = w[p * m + j] * d;
                const int sr = r == p ? c : r;
                nv[t] = r == c ? pk : fma(-w[sr * m + c], pk, w[sr * m + j]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int e = l + 32 * t;
            if (e < E) w[e] = nv[t];
        }
        __syncwarp();
    }
    for (int e = l; e < n * n; e += 32) x[e] = w[(e / n) * m + n + e % n];
    __syncwarp();
    return true;
}

// C = Gam Gam^T by outer-product Cholesky with diagonal pivoting, by the
// calling warp: each column takes the largest remaining diagonal; stop when it
// falls below 1e-13 of the largest diagonal of C (the numerical rank).  Then
// the pseudo-inverse of Gam, (Gam^T Gam)^-1 Gam^T, by Gauss-Jordan on the
// rank x rank Gram matrix (positive definite: no pivoting).  w: 2 MAXN^2
// scratch, Gam: MAXN^2 (shared).
__device__ void wgam(const double* C, int n, double* w, double* Gam, SetupOut* out)
{
    const int l = threadIdx.x & 31;
    double* Rm = w;
    for (int e = l; e < n * n; e += 32) { Rm[e] = C[e]; Gam[e] = 0.0; }
    __syncwarp();
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) dmax = fmax(dmax, Rm[i * n + i]);
    int rk = 0;
    for (; rk < n; ++rk) {
        int p = 0;                             // signed bit order: positive values in FP order
        long long best = __double_as_longlong(Rm[0]);
        for (int i = 1; i < n; ++i) {
            const long long v = __double_as_longlong(Rm[i * n + i]);
            if (v > best) { best = v; p = i; }
        }
        const double d = Rm[p * n + p];
        if (!(d > 1e-13 * dmax) || dmax <= 0.0) break;
        const double sd = sqrt(d);
        if (l < n) Gam[l * n + rk] = Rm[l * n + p] / sd;
        __syncwarp();
        for (int e = l; e < n * n; e += 32) {
            const int i = e / n, j = e - i * n;
            Rm[e] = fma(-Gam[i * n + rk], Gam[j * n + rk], Rm[e]);
        }
        __syncwarp();
    }
    for (int e = l; e < n * n; e += 32) out->Gam[e] = Gam[e];
    // Gram matrix beside the identity: [Gm | Gi], rk x 2 rk
    const int m = 2 * rk, E = rk * m;
    double* A = w;
    for (int e = l; e < E; e += 32) {
        const int a = e / m, c = e - a * m;
        double acc = 0.0;
        if (c < rk)
            for (int i = 0; i < n; ++i) acc = fma(Gam[i * n + a], Gam[i * n + c], acc);
        else
            acc = c - rk == a ? 1.0 : 0.0;
        A[e] = acc;
    }
    __syncwarp();
    constexpr int R = (2 * MAXN * MAXN + 31) / 32;
    for (int col = 0; col < rk; ++col) {
        const double ip = 1.0 / A[col * m + col];
        double nv[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int e = l + 32 * t;
            if (e < E) {
                const int r = e / m, c = e - r * m;
                const double pk = A[col * m + c] * ip;
                nv[t] = r == col ? pk : fma(-A[r * m + col], pk, A[e]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int e = l + 32 * t;
            if (e < E) A[e] = nv[t];
        }
        __syncwarp();
    }
    for (int e = l; e < n * n; e += 32) {
        const int a = e / n, i = e - a * n;
        double acc = 0.0;
        if (a < rk)
            for (int c = 0; c < rk; ++c) acc = fma(A[a * m + rk + c], Gam[i * n + c], acc);
        out->Gpinv[e] = acc;
    }
    if (l == 0) out->rank = rk;
    __syncwarp();
}

// 1/k for the Taylor terms, each rounded once at compile time
__constant__ double kRecip[25] = {0.0, 1.0 / 1, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8,
                                  1.0 / 9, 1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16,
                                  1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24};

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
    // Horner-free accumulation: term_k = term_{k-1} Z (1/k)
#pragma unroll 1
    for (int k = 1; k <= 24; ++k) {
        bmm(s.T1, s.Z, s.T2, d, d, d);
        for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
            s.T1[e] = s.T2[e] * kRecip[k];
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

// y = a x (n x k matrix, k-vector), all threads; ends with a barrier
__device__ void bmv(const double* a, const double* x, double* y, int n, int k)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int l = 0; l < k; ++l) s = fma(a[i * k + l], x[l], s);
        y[i] = s;
    }
    __syncthreads();
}

// Block element (mode 3; Section 5.1): `substeps` explicit Euler steps of all
// five rows of Eq. 37, each over h = dt / substeps from the boundary values,
//   A_s = I - h F, b_s = -h c, C_s = h Q, J_s = h H^T R^-1 H,
//   eta_s = h H^T R^-1 (y - r)   (the interval's sample y held),
// combined in time order by Eq. 36 (the later substep i on the left of the
// accumulated block j):
//   Mi = (I + C_i J_j)^-1,  T1 = A_j Mi,  T2 = (Mi A_i)^T = A_i^T (I + J_j C_i)^-1,
//   A = T1 A_i,  b = T1 (b_i + C_i eta_j) + b_j,  C = T1 C_i A_j^T + C_j,
//   eta = T2 (eta_j - J_j b_i) + eta_i,  J = T2 J_j A_i + J_i.
// b and eta stay affine in y: b = Bb y + b0, eta = Gy y - g0 (the substep
// has Bb = 0, Gy = h H^T R^-1, g0 = Gy r).  Outputs A, b (= b0), C, J,
// G (= Gy), Gr (= g0), Bb, and the substep element (sA, sb, sC, sJ, sG, sGr).
__device__ void setup_block(const SetupIn& in, SetupShared& s, SetupOut* out)
{
    const int n = in.nx, m = in.ny, ns = in.substeps < 1 ? 1 : in.substeps;
    const int nn = n * n, nm = n * m, tid = threadIdx.x, nth = blockDim.x;
    const double h = in.dt / ns;
    BlockWork& w = s.bw;
    for (int e = tid; e < nn; e += nth) {
        const int i = e / n, j = e % n;
        out->sA[e] = w.A[e] = (i == j ? 1.0 : 0.0) - h * in.F[e];
        out->sC[e] = w.C[e] = h * out->Q[e];
        out->sJ[e] = w.J[e] = h * s.Wm[e];
    }
    for (int e = tid; e < nm; e += nth) {
        out->sG[e] = w.Gy[e] = h * s.HR[e];
        w.Bb[e] = 0.0;
    }
    for (int i = tid; i < n; i += nth) {
        out->sb[i] = w.b0[i] = -h * in.c[i];
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc = fma(h * s.HR[i * m + l], in.r[l], acc);
        out->sGr[i] = w.g0[i] = acc;
    }
    __syncthreads();
    const double *Ai = out->sA, *Ci = out->sC, *Ji = out->sJ, *bi = out->sb, *Gi = out->sG, *gi = out->sGr;
#pragma unroll 1
    for (int step = 1; step < ns; ++step) {
        bmm(Ci, w.J, w.M, n, n, n);                            // I + C_i J_j
        for (int i = tid; i < n; i += nth) w.M[i * n + i] += 1.0;
        __syncthreads();
        if ((tid >> 5) == 0 && !winv(w.M, w.Mi, n, s.inw[0]) && (tid & 31) == 0) atomicOr(&s.flag, SETUP_SINGULAR_A);
        __syncthreads();
        bmm(w.A, w.Mi, w.T1, n, n, n);                         // T1 = A_j Mi
        bmm(w.T1, Ai, w.An, n, n, n);                          // A = T1 A_i
        bmm(w.T1, Ci, w.T2, n, n, n);                          // T1 C_i
        for (int e = tid; e < nn; e += nth) {                  // C = T1 C_i A_j^T + C_j
            const int i = e / n, j = e % n;
            double acc = w.C[e];
            for (int l = 0; l < n; ++l) acc = fma(w.T2[i * n + l], w.A[j * n + l], acc);
            w.Cn[e] = acc;
        }
        bmm(Ci, w.Gy, w.U, n, n, m);                           // C_i Gy_j
        bmm(w.T1, w.U, w.Bbn, n, n, m);
        for (int e = tid; e < nm; e += nth) w.Bbn[e] += w.Bb[e];       // Bb = T1 C_i Gy_j + Bb_j
        bmv(Ci, w.g0, w.u, n, n);                              // C_i g0_j
        for (int i = tid; i < n; i += nth) w.u[i] = bi[i] - w.u[i];
        __syncthreads();
        bmv(w.T1, w.u, w.b0n, n, n);
        for (int i = tid; i < n; i += nth) w.b0n[i] += w.b0[i];        // b0 = T1 (b_i - C_i g0_j) + b0_j
        bmm(w.Mi, Ai, w.T3, n, n, n);                          // Mi A_i
        for (int e = tid; e < nn; e += nth) w.T2[e] = w.T3[(e % n) * n + e / n];   // T2 = (Mi A_i)^T
        __syncthreads();
        bmm(w.T2, w.Gy, w.Gyn, n, n, m);
        for (int e = tid; e < nm; e += nth) w.Gyn[e] += Gi[e];         // Gy = T2 Gy_j + Gy_i
        bmv(w.J, bi, w.u, n, n);                               // J_j b_i
        for (int i = tid; i < n; i += nth) w.u[i] += w.g0[i];
        __syncthreads();
        bmv(w.T2, w.u, w.g0n, n, n);
        for (int i = tid; i < n; i += nth) w.g0n[i] += gi[i];          // g0 = T2 (g0_j + J_j b_i) + g0_i
        bmm(w.T2, w.J, w.T3, n, n, n);
        bmm(w.T3, Ai, w.Jn, n, n, n);
        for (int e = tid; e < nn; e += nth) w.Jn[e] += Ji[e];          // J = T2 J_j A_i + J_i
        __syncthreads();
        for (int e = tid; e < nn; e += nth) {
            w.A[e] = w.An[e];
            w.C[e] = w.Cn[e];
            w.J[e] = w.Jn[e];
        }
        for (int e = tid; e < nm; e += nth) {
            w.Bb[e] = w.Bbn[e];
            w.Gy[e] = w.Gyn[e];
        }
        for (int i = tid; i < n; i += nth) {
            w.b0[i] = w.b0n[i];
            w.g0[i] = w.g0n[i];
        }
        __syncthreads();
    }
    for (int e = tid; e < nn; e += nth) {
        const int i = e / n, j = e % n;
        out->A[e] = w.A[e];
        out->C[e] = 0.5 * (w.C[i * n + j] + w.C[j * n + i]);
        out->J[e] = 0.5 * (w.J[i * n + j] + w.J[j * n + i]);
    }
    for (int e = tid; e < nm; e += nth) {
        out->Bb[e] = w.Bb[e];
        out->G[e] = w.Gy[e];
    }
    for (int i = tid; i < n; i += nth) {
        out->b[i] = w.b0[i];
        out->Gr[i] = w.g0[i];
    }
    __syncthreads();
}

// Exact element (mode 4): all five rows of Eq. 37 with constant coefficients
// over dt, the interval's sample y held.  The element is the conditional
// minimum of the interval's cost; the reversed-time state x and costate p of
// that minimisation obey d/ds [x; p] = K0 [x; p] + k with
//   K0 = [[Ft, -Q], [-H^T R^-1 H, -Ft^T]],  k = [ct; H^T R^-1 (y - r)],
// Ft = -F, ct = -c, and the element's gradients are dV/dz = -p(dt),
// dV/dphi = p(0).  One exponential of [[K0 dt, I dt], [0, 0]] (order 4n)
// gives Psi = e^{K0 dt} and L = int_0^dt e^{K0 u} du, the affine part being
// psi = L k.  In blocks (x, p):
//   C = -Psi12 Psi22^-1,  A = Psi11 + C Psi21,  J = -Psi22^-1 Psi21,
//   b = psi1 + C psi2,    eta = Psi22^-1 psi2,
// so, with HR = H^T R^-1,
//   Bb = (L12 + C L22) HR,  b0 = -(L11 + C L21) c - Bb r,
//   Gy = Psi22^-1 L22 HR,   g0 = Psi22^-1 L21 c + Gy r.
// Scratch in the output arrays that the set-up overwrites afterwards (Phi,
// Cinv, Qinv) and in X, Y.
__device__ void setup_exact(const SetupIn& in, SetupShared& s, SetupOut* out)
{
    const int n = in.nx, m = in.ny, n2 = 2 * n, d = 4 * n, nn = n * n, tid = threadIdx.x, nth = blockDim.x;
    const double h = in.dt;
    for (int e = tid; e < d * d; e += nth) {
        const int i = e / d, j = e % d;
        double z = 0.0;
        if (i < n && j < n) z = -in.F[i * n + j] * h;
        else if (i < n && j < n2) z = -out->Q[i * n + (j - n)] * h;
        else if (i >= n && i < n2 && j < n) z = -s.Wm[(i - n) * n + j] * h;
        else if (i >= n && i < n2 && j >= n && j < n2) z = in.F[(j - n) * n + (i - n)] * h;
        else if (i < n2 && j >= n2 && j - n2 == i) z = h;
        s.Z[e] = z;
    }
    __syncthreads();
    bexpm(s, d);
    auto E = [&](int i, int j) { return s.E[i * d + j]; };
    for (int e = tid; e < nn; e += nth) s.X[e] = E(n + e / n, n + e % n);      // Psi22
    __syncthreads();
    if ((tid >> 5) == 0 && !winv(s.X, s.Y, n, s.inw[0]) && (tid & 31) == 0) atomicOr(&s.flag, SETUP_SINGULAR_A);
    __syncthreads();
    double* Pi = s.Y;                                                          // Psi22^-1
    for (int e = tid; e < nn; e += nth) {
        const int i = e / n, j = e % n;
        double c = 0.0, jj = 0.0;
        for (int l = 0; l < n; ++l) {
            c = fma(E(i, n + l), Pi[l * n + j], c);          // Psi12 Psi22^-1
            jj = fma(Pi[i * n + l], E(n + l, j), jj);        // Psi22^-1 Psi21
        }
        out->C[e] = -c;
        out->J[e] = -jj;
    }
    __syncthreads();
    double* LC1 = out->Cinv;
    double* LC2 = out->Qinv;
    double* PL = out->Phi;
    for (int e = tid; e < nn; e += nth) {
        const int i = e / n, j = e % n;
        double a = E(i, j), l1 = E(i, n2 + j), l2 = E(i, n2 + n + j), pl = 0.0;
        for (int l = 0; l < n; ++l) {
            a = fma(out->C[i * n + l], E(n + l, j), a);              // Psi11 + C Psi21
            l1 = fma(out->C[i * n + l], E(n + l, n2 + j), l1);       // L11 + C L21
            l2 = fma(out->C[i * n + l], E(n + l, n2 + n + j), l2);   // L12 + C L22
            pl = fma(Pi[i * n + l], E(n + l, n2 + n + j), pl);       // Psi22^-1 L22
        }
        out->A[e] = a;
        LC1[e] = l1;
        LC2[e] = l2;
        PL[e] = pl;
    }
    __syncthreads();
    bmm(LC2, s.HR, out->Bb, n, n, m);
    bmm(PL, s.HR, out->G, n, n, m);
    for (int i = tid; i < n; i += nth) {
        double lc = 0.0, l21c = 0.0;
        for (int l = 0; l < n; ++l) {
            lc = fma(LC1[i * n + l], in.c[l], lc);
            l21c = fma(E(n + i, n2 + l), in.c[l], l21c);     // L21 c
        }
        s.X[i] = l21c;
        double br = 0.0;
        for (int l = 0; l < m; ++l) br = fma(out->Bb[i * m + l], in.r[l], br);
        out->b[i] = -lc - br;
    }
    __syncthreads();
    for (int i = tid; i < n; i += nth) {
        double g = 0.0;
        for (int l = 0; l < n; ++l) g = fma(Pi[i * n + l], s.X[l], g);
        for (int l = 0; l < m; ++l) g = fma(out->G[i * m + l], in.r[l], g);
        out->Gr[i] = g;
    }
    __syncthreads();
    for (int e = tid; e < nn; e += nth) {
        const int i = e / n, j = e % n;
        s.X[e] = 0.5 * (out->C[i * n + j] + out->C[j * n + i]);
        s.T1[e] = 0.5 * (out->J[i * n + j] + out->J[j * n + i]);
    }
    __syncthreads();
    for (int e = tid; e < nn; e += nth) {
        out->C[e] = s.X[e];
        out->J[e] = s.T1[e];
    }
    __syncthreads();
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
    for (int e = threadIdx.x; e < n * m; e += blockDim.x) out->Bb[e] = 0.0;
    if (in.mode == 0) {
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e / n, j = e % n;
            out->A[e] = (i == j ? 1.0 : 0.0) - dt * in.F[e];
            out->C[e] = dt * out->Q[e];
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) out->b[i] = -dt * in.c[i];
        __syncthreads();
    } else if (in.mode >= 3) {
        // R^-1, H^T R^-1 and H^T R^-1 H first: the measurement rows of Eq. 37
        // enter the element itself
        if ((threadIdx.x >> 5) == 0 && !winv(in.R, out->Rinv, m, s.inw[0]) && (threadIdx.x & 31) == 0)
            atomicOr(&s.flag, SETUP_SINGULAR_R);
        __syncthreads();
        for (int e = threadIdx.x; e < n * m; e += blockDim.x) {
            const int i = e / m, j = e % m;
            double acc = 0.0;
            for (int l = 0; l < m; ++l) acc = fma(in.H[l * n + i], out->Rinv[l * m + j], acc);
            s.HR[e] = acc;
        }
        __syncthreads();
        bmm(s.HR, in.H, s.Wm, n, m, n);
        if (in.mode == 3)
            setup_block(in, s, out);
        else
            setup_exact(in, s, out);
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
    // inverses and the factor of C, one warp each, side by side
    {
        const int wid = threadIdx.x >> 5;
        int bad = 0;
        if (wid == 0) bad = winv(in.R, out->Rinv, m, s.inw[0]) ? 0 : SETUP_SINGULAR_R;
        else if (wid == 1) bad = winv(in.P0, out->S0, n, s.inw[1]) ? 0 : SETUP_SINGULAR_P0;
        else if (wid == 2) bad = winv(out->A, out->Phi, n, s.inw[2]) ? 0 : SETUP_SINGULAR_A;
        else if (wid == 3) bad = winv(out->Q, out->Qinv, n, s.inw[3]) ? 0 : SETUP_SINGULAR_Q;
        else if (wid == 4) bad = winv(out->C, out->Cinv, n, s.inw[4]) ? 0 : SETUP_SINGULAR_C;
        else if (wid == 5) wgam(out->C, n, s.inw[5], s.Gam, out);
        if (bad && (threadIdx.x & 31) == 0) atomicOr(&s.flag, bad);
    }
    __syncthreads();
    // measurement: G = dt H^T R^-1, J = G H (symmetrised), Gr = G r (modes 3
    // and 4 have set them with the element)
    if (in.mode < 3)
        for (int e = threadIdx.x; e < n * m; e += blockDim.x) {
            const int i = e / m, j = e % m;
            double acc = 0.0;
            for (int l = 0; l < m; ++l) acc = fma(in.H[l * n + i], out->Rinv[l * m + j], acc);
            out->G[e] = dt * acc;
        }
    __syncthreads();
    // prior: v0 = S0 m0
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < n; ++l) acc = fma(out->S0[i * n + l], in.m0[l], acc);
        out->v0[i] = acc;
    }
    // forward transition: beta = -Phi b, Sigma = Phi C Phi^T
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < n; ++l) acc = fma(out->Phi[i * n + l], out->b[l], acc);
        out->beta[i] = -acc;
    }
    bmm(out->Phi, out->C, s.T1, n, n, n);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc = fma(out->G[i * m + l], in.H[l * n + j], acc);
        s.Y[e] = acc;
        acc = 0.0;
        for (int l = 0; l < n; ++l) acc = fma(s.T1[i * n + l], out->Phi[j * n + l], acc);
        out->Sigma[e] = acc;
    }
    if (in.mode < 3)
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double acc = 0.0;
            for (int l = 0; l < m; ++l) acc = fma(out->G[i * m + l], in.r[l], acc);
            out->Gr[i] = acc;
        }
    __syncthreads();
    if (in.mode < 3)
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e / n, j = e % n;
            out->J[e] = 0.5 * (s.Y[i * n + j] + s.Y[j * n + i]);
        }
    if (threadIdx.x == 0) out->flags = s.flag;
}

cudaError_t launch_setup(const SetupIn& in, SetupOut* d_out, cudaStream_t st)
{
    k_setup<<<1, 256, 0, st>>>(in, d_out);
    return cudaGetLastError();
}

}  // namespace mapk
