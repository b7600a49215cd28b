// Element producers: build the interval element (A, b, C, eta, J) of step k in
// registers from per-step inputs, so elements are never stored.
//
// Orientation (time reversal, Section 2.2): element k spans [t_k, t_{k+1}];
// its start state phi is x_{k+1} and its end state z is x_k.  One explicit
// Euler step of Eq. (37) from the boundary values A = I, b = C = eta = J = 0
// gives, with the reversed drift F~ = -F, c~ = -c,
//   A = I - dt F,  b = -dt c,  C = dt Q,
//   J = dt H^T R^-1 H,  eta = dt H^T R^-1 (y_{k+1} - r),
// the measurement term being that of the start state x_{k+1}.  Steps k >= T
// (padding of the last tile) produce the identity element (I, 0, 0, 0, 0),
// which is neutral on both sides of the combine.
#pragma once
#include "elements.cuh"

namespace mapk {

// Load `CNT` consecutive scalars starting at src into dst; entries at or past
// `avail` are zero.  Uses 16-byte vector loads when the run is complete and
// aligned.
template <int CNT, typename S>
__device__ __forceinline__ void load_run(const S* __restrict__ src, long avail, S* dst)
{
    constexpr int V = 16 / sizeof(S);
    if (CNT % V == 0 && avail >= CNT && (reinterpret_cast<size_t>(src) & 15) == 0) {
#pragma unroll
        for (int i = 0; i < CNT; i += V) {
            if (sizeof(S) == 4) {
                float4 q = __ldg(reinterpret_cast<const float4*>(src + i));
                dst[i] = S(q.x); dst[i + 1] = S(q.y); dst[i + 2] = S(q.z); dst[i + 3] = S(q.w);
            } else {
                double2 q = __ldg(reinterpret_cast<const double2*>(src + i));
                dst[i] = S(q.x); dst[i + 1] = S(q.y);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < CNT; ++i) dst[i] = i < avail ? __ldg(src + i) : S(0);
    }
}

// ---------------------------------------------------------------------------
// linear time-invariant model: everything but eta is the same for every step
// ---------------------------------------------------------------------------
template <int N, int M, typename S>
struct LtiParams {
    static constexpr int NS = Sym<N>::SZ;
    static constexpr int R = (N + 1) / 2;   // column count of the low-rank factor of C
    S A[N * N];
    S b[N];
    S C[NS];
    S J[NS];
    S G[N * M];      // dt H^T R^-1
    S Gr[N];         // dt H^T R^-1 r
    S Gam[N * R];    // C = Gam Gam^T when lowrank (zero columns beyond the rank)
    S Gpinv[R * N];  // pseudo-inverse of Gam (zero rows beyond the rank)
    int lowrank;     // rank(C) <= R: the per-step value-function update uses Gam
};

template <int N, int M, typename S>
struct LtiProducer {
    static constexpr int W = M;      // scalars read per step
    static constexpr bool RESETS = false;
    static constexpr bool LINEAR_FOLD = true;   // see lti_fold.cuh
    static constexpr bool LOWRANK = true;
    __device__ __forceinline__ bool is_reset(long) const { return false; }
    const S* y;                      // (T, M), row k holds y_{k+1}
    long T;
    LtiParams<N, M, S> p;

    template <int K>
    __device__ __forceinline__ void load(long k0, S (&buf)[K * W]) const
    {
        const long avail = (T - k0) * W;
        load_run<K * W, S>(y + k0 * W, avail, buf);
    }

    // inputs of one step (zeros past T)
    __device__ __forceinline__ void load1(long k, S* row) const
    {
#pragma unroll
        for (int j = 0; j < W; ++j) row[j] = k < T ? __ldg(y + k * W + j) : S(0);
    }

    // terminal value function of a reversed scan (not used for forward scans)
    __device__ __forceinline__ void terminal(Red<N, S>& r) const
    {
#pragma unroll
        for (int i = 0; i < Red<N, S>::NCOMP; ++i) comp(r, i) = S(0);
    }

    __device__ __forceinline__ void make(long k, const S* row, Elem<N, S>& e) const
    {
        if (k >= T) { set_identity(e); return; }
#pragma unroll
        for (int i = 0; i < N * N; ++i) e.A[i] = p.A[i];
#pragma unroll
        for (int i = 0; i < N; ++i) e.b[i] = p.b[i];
#pragma unroll
        for (int i = 0; i < Sym<N>::SZ; ++i) { e.C[i] = p.C[i]; e.J[i] = p.J[i]; }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S s = -p.Gr[i];
#pragma unroll
            for (int j = 0; j < M; ++j) s = fma(p.G[i * M + j], row[j], s);
            e.eta[i] = s;
        }
    }
};

// ---------------------------------------------------------------------------
// Block and exact elements of a linear time-invariant model (Section 5.1
// blocks of Euler substeps, or Eq. 37 solved exactly): the interval's sample
// is held across the interval, so both offsets depend on it,
//   b_k = Bb y_{k+1} + b0,   eta_k = G y_{k+1} - Gr,
// while A, C, J are the same for every interval.  Elements are combined on
// the general path (no linear fold).
// ---------------------------------------------------------------------------
template <int N, int M, typename S>
struct BlockParams {
    static constexpr int NS = Sym<N>::SZ;
    S A[N * N];
    S C[NS];
    S J[NS];
    S Bb[N * M];
    S b0[N];
    S G[N * M];
    S Gr[N];
};

template <int N, int M, typename S>
struct BlockProducer {
    static constexpr int W = M;
    static constexpr bool RESETS = false;
    static constexpr bool LINEAR_FOLD = false;
    static constexpr bool LOWRANK = false;
    __device__ __forceinline__ bool is_reset(long) const { return false; }
    const S* y;                      // (T, M), row k holds y_{k+1}
    long T;
    BlockParams<N, M, S> p;

    __device__ __forceinline__ void load1(long k, S* row) const
    {
#pragma unroll
        for (int j = 0; j < W; ++j) row[j] = k < T ? __ldg(y + k * W + j) : S(0);
    }

    __device__ __forceinline__ void terminal(Red<N, S>& r) const
    {
#pragma unroll
        for (int i = 0; i < Red<N, S>::NCOMP; ++i) comp(r, i) = S(0);
    }

    __device__ __forceinline__ void make(long k, const S* row, Elem<N, S>& e) const
    {
        if (k >= T) { set_identity(e); return; }
#pragma unroll
        for (int i = 0; i < N * N; ++i) e.A[i] = p.A[i];
#pragma unroll
        for (int i = 0; i < Sym<N>::SZ; ++i) { e.C[i] = p.C[i]; e.J[i] = p.J[i]; }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S sb = p.b0[i], se = -p.Gr[i];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                sb = fma(p.Bb[i * M + j], row[j], sb);
                se = fma(p.G[i * M + j], row[j], se);
            }
            e.b[i] = sb;
            e.eta[i] = se;
        }
    }
};

// ---------------------------------------------------------------------------
// Many independent trajectories of one linear model in one scan.  Trajectory
// j > 0 is preceded by the model's prior element a_T = (0, 0, 0, P0^-1 m0,
// P0^-1) (Eq. 31): on the left of the combine (Eq. 36) an element with
// A = C = 0 keeps only its own (J, eta), so every prefix that contains it
// restarts at the prior, and its closed-loop map is the constant map to the
// argmin of the previous trajectory's last value function (Eq. 18).  Element k
// reads row k of y; rows at the inserted positions are unused.
// ---------------------------------------------------------------------------
template <int N, int M, typename S>
struct SegLtiProducer {
    static constexpr int W = M;
    static constexpr bool RESETS = true;
    static constexpr bool LINEAR_FOLD = false;
    static constexpr bool LOWRANK = true;
    const S* y;                      // (T, M) with an unused row at every reset
    const unsigned char* reset;      // (T): 1 where a trajectory starts (except the first)
    long T;
    LtiParams<N, M, S> p;
    S S0[Sym<N>::SZ];                // P0^-1
    S v0[N];                         // P0^-1 m0

    __device__ __forceinline__ bool is_reset(long k) const { return k < T && __ldg(reset + k) != 0; }

    __device__ __forceinline__ void load1(long k, S* row) const
    {
#pragma unroll
        for (int j = 0; j < W; ++j) row[j] = k < T ? __ldg(y + k * W + j) : S(0);
    }

    __device__ __forceinline__ void terminal(Red<N, S>& r) const
    {
#pragma unroll
        for (int i = 0; i < Red<N, S>::NCOMP; ++i) comp(r, i) = S(0);
    }

    __device__ __forceinline__ void make(long k, const S* row, Elem<N, S>& e) const
    {
        if (k >= T) { set_identity(e); return; }
        if (is_reset(k)) {
#pragma unroll
            for (int i = 0; i < N * N; ++i) e.A[i] = S(0);
#pragma unroll
            for (int i = 0; i < N; ++i) { e.b[i] = S(0); e.eta[i] = v0[i]; }
#pragma unroll
            for (int i = 0; i < Sym<N>::SZ; ++i) { e.C[i] = S(0); e.J[i] = S0[i]; }
            return;
        }
#pragma unroll
        for (int i = 0; i < N * N; ++i) e.A[i] = p.A[i];
#pragma unroll
        for (int i = 0; i < N; ++i) e.b[i] = p.b[i];
#pragma unroll
        for (int i = 0; i < Sym<N>::SZ; ++i) { e.C[i] = p.C[i]; e.J[i] = p.J[i]; }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S s = -p.Gr[i];
#pragma unroll
            for (int j = 0; j < M; ++j) s = fma(p.G[i * M + j], row[j], s);
            e.eta[i] = s;
        }
    }
};

// ---------------------------------------------------------------------------
// Adjoint of the MAP solve.  x* solves K x = g with K the (symmetric)
// Hessian of the discrete cost, so lambda = K^-1 d (d = dL/dx*) is the MAP
// trajectory of the same problem with b = 0, the measurement information
// vectors replaced by d_{k+1} (element k) and the prior term by d_0:
// same A, C, J; eta_k = d_{k+1}; terminal value function (d_0, P0^-1).
// ---------------------------------------------------------------------------
template <int N, typename S>
struct AdjParams {
    static constexpr int NS = Sym<N>::SZ;
    S A[N * N];
    S C[NS];
    S J[NS];
    S S0[NS];
};

template <int N, typename S>
struct AdjProducer {
    static constexpr int W = N;
    static constexpr bool RESETS = false;
    static constexpr bool LINEAR_FOLD = false;
    static constexpr bool LOWRANK = false;
    __device__ __forceinline__ bool is_reset(long) const { return false; }
    const S* d;                      // (T+1, N): dL/dx*
    long T;
    AdjParams<N, S> p;

    __device__ __forceinline__ void load1(long k, S* row) const
    {
#pragma unroll
        for (int j = 0; j < W; ++j) row[j] = k < T ? __ldg(d + (k + 1) * N + j) : S(0);
    }

    __device__ __forceinline__ void terminal(Red<N, S>& r) const
    {
#pragma unroll
        for (int i = 0; i < N; ++i) r.v[i] = __ldg(d + i);
#pragma unroll
        for (int i = 0; i < Sym<N>::SZ; ++i) r.P[i] = p.S0[i];
    }

    __device__ __forceinline__ void make(long k, const S* row, Elem<N, S>& e) const
    {
        if (k >= T) { set_identity(e); return; }
#pragma unroll
        for (int i = 0; i < N * N; ++i) e.A[i] = p.A[i];
#pragma unroll
        for (int i = 0; i < N; ++i) { e.b[i] = S(0); e.eta[i] = row[i]; }
#pragma unroll
        for (int i = 0; i < Sym<N>::SZ; ++i) { e.C[i] = p.C[i]; e.J[i] = p.J[i]; }
    }
};

// ---------------------------------------------------------------------------
// Backward information filter of the two-filter smoother (Section 3.5 second
// method, Section 4.3 Eq. 43): the same combine applied to the interval
// elements written the other way round.  The flipped element of interval k
// has start x_k and end x_{k+1}: the forward transition
//   A' = Phi = A^-1,  b' = beta = -A^-1 b,  C' = Sigma = A^-1 C A^-T,
// with x_k's own measurement (y_k, none for k = 0) as its (J', eta').  They are
// scanned in reversed order j = Tpad - 1 - k (Tpad = padded horizon, so that
// thread chunks coincide with those of the forward scan), starting from the
// terminal value function of x_T, which carries y_T.  The prefix before
// element j is then the information on x_{k+1} from y_{k+1}..y_T.
// ---------------------------------------------------------------------------
template <int N, int M, typename S>
struct FlipParams {
    static constexpr int NS = Sym<N>::SZ;
    S A[N * N];      // Phi
    S b[N];          // beta
    S C[NS];         // Sigma
    S J[NS];         // dt H^T R^-1 H
    S G[N * M];      // dt H^T R^-1
    S Gr[N];         // dt H^T R^-1 r
};

template <int N, int M, typename S>
struct RevFlipProducer {
    static constexpr int W = M;
    static constexpr bool RESETS = false;
    static constexpr bool LINEAR_FOLD = false;
    static constexpr bool LOWRANK = false;
    __device__ __forceinline__ bool is_reset(long) const { return false; }
    const S* y;                      // (T, M), row k-1 holds y_k
    long T;
    long Tpad;
    FlipParams<N, M, S> p;

    __device__ __forceinline__ void load1(long j, S* row) const
    {
        const long k = Tpad - 1 - j;
        const bool in = k >= 1 && k < T;
#pragma unroll
        for (int q = 0; q < W; ++q) row[q] = in ? __ldg(y + (k - 1) * W + q) : S(0);
    }

    // information of y_T on x_T
    __device__ __forceinline__ void terminal(Red<N, S>& r) const
    {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S s = -p.Gr[i];
#pragma unroll
            for (int q = 0; q < M; ++q) s = fma(p.G[i * M + q], __ldg(y + (T - 1) * M + q), s);
            r.v[i] = s;
        }
#pragma unroll
        for (int i = 0; i < Sym<N>::SZ; ++i) r.P[i] = p.J[i];
    }

    // the flipped element of interval k = Tpad - 1 - j (identity past the horizon)
    __device__ __forceinline__ void make(long j, const S* row, Elem<N, S>& e) const
    {
        const long k = Tpad - 1 - j;
        if (k >= T) { set_identity(e); return; }
#pragma unroll
        for (int i = 0; i < N * N; ++i) e.A[i] = p.A[i];
#pragma unroll
        for (int i = 0; i < N; ++i) e.b[i] = p.b[i];
#pragma unroll
        for (int i = 0; i < Sym<N>::SZ; ++i) e.C[i] = p.C[i];
        const bool meas = k >= 1;
#pragma unroll
        for (int i = 0; i < Sym<N>::SZ; ++i) e.J[i] = meas ? p.J[i] : S(0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S s = -p.Gr[i];
#pragma unroll
            for (int q = 0; q < M; ++q) s = fma(p.G[i * M + q], row[q], s);
            e.eta[i] = meas ? s : S(0);
        }
    }
};

// ---------------------------------------------------------------------------
// nonlinear models, linearised at a trajectory xbar (Section 4.4):
//   A = I - dt F(xbar_{k+1}),  b = -dt (f(xbar_{k+1}) - F xbar_{k+1}),  C = dt Q,
//   J = dt Hb^T R^-1 Hb,  eta = dt Hb^T R^-1 (y - h(xbar) + Hb xbar) - dt/2 grad div f(xbar)
// with Hb = dh/dx(xbar_{k+1}).  R is diagonal (Rinv holds its inverse).
// ---------------------------------------------------------------------------
template <int N, int M, typename S>
struct NlParams {
    static constexpr int NS = Sym<N>::SZ;
    S dt;
    int expm;         // per-step exact discretisation of the local linear drift
    S Q[NS];          // L W L^T
    S C[NS];          // dt Q
    S Rinv[M];        // diagonal of R^-1
    S F[N * N];       // linear part of the cubic drift
    S c[N];
    S H[M * N];       // linear measurement of the cubic model
    S r[M];
    S gamma;
};

template <typename S>
__device__ __forceinline__ S wrap_angle(S a)
{
    const S pi = S(3.14159265358979323846);
    const S twopi = S(6.28318530717958647692);
    a = a - twopi * floor((a + pi) / twopi);
    return a;
}

// coordinated turn (Section 5.2, Eq. 46), N = 5, M = 2
template <typename S>
struct CtModel {
    static constexpr int N = 5, M = 2;
    __device__ __forceinline__ static void drift(const NlParams<5, 2, S>&, const S* x, S* f, S* Fj, S* gdiv)
    {
#pragma unroll
        for (int i = 0; i < 25; ++i) Fj[i] = S(0);
        f[0] = x[2]; f[1] = x[3]; f[2] = -x[4] * x[3]; f[3] = x[4] * x[2]; f[4] = S(0);
        Fj[0 * 5 + 2] = S(1);
        Fj[1 * 5 + 3] = S(1);
        Fj[2 * 5 + 3] = -x[4]; Fj[2 * 5 + 4] = -x[3];
        Fj[3 * 5 + 2] = x[4];  Fj[3 * 5 + 4] = x[2];
#pragma unroll
        for (int i = 0; i < 5; ++i) gdiv[i] = S(0);   // div f = 0 for this drift
    }
    // residual y - h(x) (bearing wrapped to (-pi, pi]) and Jacobian of h
    __device__ __forceinline__ static void measure(const NlParams<5, 2, S>&, const S* x, const S* y, S* res, S* Hj)
    {
        const S r2 = x[0] * x[0] + x[1] * x[1];
        const S rho = sqrt(r2);
        res[0] = y[0] - rho;
        res[1] = wrap_angle<S>(y[1] - atan2(x[1], x[0]));
#pragma unroll
        for (int i = 0; i < 10; ++i) Hj[i] = S(0);
        Hj[0] = x[0] / rho; Hj[1] = x[1] / rho;
        Hj[5] = -x[1] / r2; Hj[6] = x[0] / r2;
    }
};

// cubic drift f = F x + c - gamma x^3 with linear measurement (state-dependent divergence)
template <int NN, int MM, typename S>
struct CubicModel {
    static constexpr int N = NN, M = MM;
    __device__ __forceinline__ static void drift(const NlParams<NN, MM, S>& p, const S* x, S* f, S* Fj, S* gdiv)
    {
#pragma unroll
        for (int i = 0; i < NN; ++i) {
            S s = p.c[i];
#pragma unroll
            for (int j = 0; j < NN; ++j) { s = fma(p.F[i * NN + j], x[j], s); Fj[i * NN + j] = p.F[i * NN + j]; }
            f[i] = s - p.gamma * x[i] * x[i] * x[i];
            Fj[i * NN + i] -= S(3) * p.gamma * x[i] * x[i];
            gdiv[i] = S(-6) * p.gamma * x[i];
        }
    }
    __device__ __forceinline__ static void measure(const NlParams<NN, MM, S>& p, const S* x, const S* y, S* res, S* Hj)
    {
#pragma unroll
        for (int i = 0; i < MM; ++i) {
            S s = p.r[i];
#pragma unroll
            for (int j = 0; j < NN; ++j) { s = fma(p.H[i * NN + j], x[j], s); Hj[i * NN + j] = p.H[i * NN + j]; }
            res[i] = y[i] - s;
        }
    }
};

// Exact interval element (A, b, C) of the local linear drift f ~ F x + c over
// dt (the A, b, C rows of Eq. 37 with constant coefficients, reversed drift
// -F): A = e^{-F dt}, b = -int_0^dt e^{-F u} du c,
// C = int_0^dt e^{-F u} Q e^{-F^T u} du.  Scaling and squaring: with
// h = dt / 2^s and |F| h <= 1/4, truncated series
//   A_h = sum_j X^j / j!,  b_h = -h sum_j X^j / (j+1)! c   (X = -F h),
//   C_h = sum_k h^(k+1) / (k+1)! L_k,  L_0 = Q,  L_{k+1} = -F L_k - L_k F^T
// (the Taylor coefficients of the integrand), then s doublings of the
// data-free element, (A, b, C) -> (A A, A b + b, A C A^T + C) (Eq. 36 with
// J = 0).  Terms up to order 6 in FP32, 12 in FP64.
template <int N, typename S>
__device__ __forceinline__ void local_exact_element(const S* F, const S* c, const S* Qp, S dt, S* A, S* b, S* Cp)
{
    constexpr int NN = N * N, P = sizeof(S) == 4 ? 6 : 12;
    S nrm = S(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        S r = S(0);
#pragma unroll
        for (int j = 0; j < N; ++j) r += fabs(F[i * N + j]);
        nrm = fmax(nrm, r);
    }
    int sq = 0;
    S h = dt;
    while (nrm * h > S(0.25) && sq < 30) { h *= S(0.5); ++sq; }
    S X[NN], Pw[NN], Ph[N], L[NN], Cf[NN];
#pragma unroll
    for (int q = 0; q < NN; ++q) {
        X[q] = -F[q] * h;
        Pw[q] = q % (N + 1) == 0 ? S(1) : S(0);          // X^0
        A[q] = Pw[q];
        L[q] = Qp[Sym<N>::at(q / N, q % N)];
        Cf[q] = h * L[q];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) Ph[i] = c[i];            // sum_j X^j / (j+1)! c, term j = 0
    S fj = S(1);                                         // j!
    S hk = h;                                            // h^(k+1) / (k+1)!
#pragma unroll 1
    for (int j = 1; j <= P; ++j) {
        S T1[NN];
        ms::mm<N, S>(Pw, X, T1);                         // X^j (j! folded in below)
        fj *= S(j);
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            Pw[q] = T1[q];
            A[q] += T1[q] / fj;
        }
        S v[N];
        ms::mv<N, S>(T1, c, v);
#pragma unroll
        for (int i = 0; i < N; ++i) Ph[i] += v[i] / (fj * S(j + 1));
        // L_j = -F L_{j-1} - L_{j-1} F^T
        S FL[NN];
        ms::mm<N, S>(F, L, FL);
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int d = 0; d < N; ++d) T1[a * N + d] = -(FL[a * N + d] + FL[d * N + a]);
        hk *= h / S(j + 1);
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            L[q] = T1[q];
            Cf[q] += hk * L[q];
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) b[i] = -h * Ph[i];
#pragma unroll 1
    for (int s2 = 0; s2 < sq; ++s2) {
        S A2[NN], AC[NN], C2[NN], Ab[N];
        ms::mm<N, S>(A, A, A2);
        ms::mv<N, S>(A, b, Ab);
        ms::mm<N, S>(A, Cf, AC);
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int d = 0; d < N; ++d) {
                S acc = Cf[a * N + d];
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(AC[a * N + q], A[d * N + q], acc);
                C2[a * N + d] = acc;
            }
#pragma unroll
        for (int q = 0; q < NN; ++q) { A[q] = A2[q]; Cf[q] = C2[q]; }
#pragma unroll
        for (int i = 0; i < N; ++i) b[i] += Ab[i];
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int d = a; d < N; ++d) Cp[Sym<N>::at(a, d)] = S(0.5) * (Cf[a * N + d] + Cf[d * N + a]);
}

// Row layout of the per-step exact elements (A, b, C packed) of an iteration,
// rows of whole 16-byte words
template <int N, typename S>
struct ExactRow {
    static constexpr int oA = 0, ob = N * N, oC = N * N + N;
    static constexpr int RS = ((N * N + N + Sym<N>::SZ) * (int)sizeof(S) + 15) / 16 * 16 / (int)sizeof(S);
};

template <class Model, typename S>
struct NlProducer {
    static constexpr int N = Model::N, M = Model::M;
    static constexpr int W = M + N;   // y_{k+1} then xbar_{k+1}
    static constexpr bool RESETS = false;
    static constexpr bool LINEAR_FOLD = false;
    static constexpr bool LOWRANK = false;
    __device__ __forceinline__ bool is_reset(long) const { return false; }
    const S* y;                       // (T, M)
    const S* xbar;                    // (T+1, N)
    long T;
    NlParams<N, M, S> p;
    const S* etab = nullptr;          // exact elements of this iteration (ExactRow), or formed per use

    template <int K>
    __device__ __forceinline__ void load(long k0, S (&buf)[K * W]) const
    {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const long k = k0 + i;
            const bool in = k < T;
#pragma unroll
            for (int j = 0; j < M; ++j) buf[i * W + j] = in ? __ldg(y + k * M + j) : S(0);
#pragma unroll
            for (int j = 0; j < N; ++j) buf[i * W + M + j] = in ? __ldg(xbar + (k + 1) * N + j) : S(0);
        }
    }

    __device__ __forceinline__ void load1(long k, S* row) const
    {
        const bool in = k < T;
#pragma unroll
        for (int j = 0; j < M; ++j) row[j] = in ? __ldg(y + k * M + j) : S(0);
#pragma unroll
        for (int j = 0; j < N; ++j) row[M + j] = in ? __ldg(xbar + (k + 1) * N + j) : S(0);
    }

    __device__ __forceinline__ void terminal(Red<N, S>& r) const
    {
#pragma unroll
        for (int i = 0; i < Red<N, S>::NCOMP; ++i) comp(r, i) = S(0);
    }

    __device__ __forceinline__ void make(long k, const S* row, Elem<N, S>& e) const
    {
        if (k >= T) { set_identity(e); return; }
        const S* yk = row;
        const S* x1 = row + M;
        S f[N], Fj[N * N], gd[N], res[M], Hj[M * N];
        Model::drift(p, x1, f, Fj, gd);
        Model::measure(p, x1, yk, res, Hj);
        const S dt = p.dt;
        if (p.expm) {
            // local linear drift F x + c, c = f(xbar) - F xbar, discretised exactly
            S cl[N];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                S s = f[i];
#pragma unroll
                for (int j = 0; j < N; ++j) s = fma(-Fj[i * N + j], x1[j], s);
                cl[i] = s;
            }
            if (etab) {
                using ER = ExactRow<N, S>;
                const S* r = etab + k * ER::RS;
#pragma unroll
                for (int q = 0; q < N * N; ++q) e.A[q] = __ldg(r + ER::oA + q);
#pragma unroll
                for (int q = 0; q < N; ++q) e.b[q] = __ldg(r + ER::ob + q);
#pragma unroll
                for (int q = 0; q < Sym<N>::SZ; ++q) e.C[q] = __ldg(r + ER::oC + q);
            } else {
                local_exact_element<N, S>(Fj, cl, p.Q, dt, e.A, e.b, e.C);
            }
        } else {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                S s = f[i];
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    e.A[i * N + j] = (i == j ? S(1) : S(0)) - dt * Fj[i * N + j];
                    s = fma(-Fj[i * N + j], x1[j], s);
                }
                e.b[i] = -dt * s;
            }
#pragma unroll
            for (int i = 0; i < Sym<N>::SZ; ++i) e.C[i] = p.C[i];
        }
        // measurement information and the linearised divergence term
        S u[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            S s = res[i];
#pragma unroll
            for (int j = 0; j < N; ++j) s = fma(Hj[i * N + j], x1[j], s);
            u[i] = s * p.Rinv[i] * dt;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            S s = S(-0.5) * dt * gd[i];
#pragma unroll
            for (int j = 0; j < M; ++j) s = fma(Hj[j * N + i], u[j], s);
            e.eta[i] = s;
        }
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = i; j < N; ++j) {
                S s = S(0);
#pragma unroll
                for (int l = 0; l < M; ++l) s = fma(Hj[l * N + i] * p.Rinv[l], Hj[l * N + j], s);
                e.J[Sym<N>::at(i, j)] = dt * s;
            }
    }
};

// The exact elements (A, b, C) of every step of one Gauss-Newton iteration,
// linearised at xbar_{k+1}: one thread per step, so that the scan kernels read
// them instead of forming them in each of their passes.
template <class Model, typename S>
__global__ void __launch_bounds__(128) k_exact_rows(const NlProducer<Model, S> prod, S* __restrict__ tab)
{
    constexpr int N = Model::N;
    using ER = ExactRow<N, S>;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= prod.T) return;
    S x1[N], f[N], Fj[N * N], gd[N], cl[N], A[N * N], b[N], Cp[Sym<N>::SZ];
#pragma unroll
    for (int j = 0; j < N; ++j) x1[j] = __ldg(prod.xbar + (k + 1) * N + j);
    Model::drift(prod.p, x1, f, Fj, gd);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        S s = f[i];
#pragma unroll
        for (int j = 0; j < N; ++j) s = fma(-Fj[i * N + j], x1[j], s);
        cl[i] = s;
    }
    local_exact_element<N, S>(Fj, cl, prod.p.Q, prod.p.dt, A, b, Cp);
    S* r = tab + k * ER::RS;
#pragma unroll
    for (int q = 0; q < N * N; ++q) r[ER::oA + q] = A[q];
#pragma unroll
    for (int q = 0; q < N; ++q) r[ER::ob + q] = b[q];
#pragma unroll
    for (int q = 0; q < Sym<N>::SZ; ++q) r[ER::oC + q] = Cp[q];
}

}  // namespace mapk
