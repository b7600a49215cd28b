/*
 * FP64 CPU oracle for continuous-time MAP trajectory estimation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or run this code.  The
 * CUDA library shares no code, header, table or helper with it.
 *
 * What it computes: the argmin of the discrete Onsager-Machlup cost (Eq. 2
 * on the time grid t_k = t0 + k dt, k = 0..T)
 *
 *   M(x) = 1/2 |x_0 - m0|^2_{P0^-1}
 *        + sum_{k=0}^{T-1} 1/2 |x_k - A_k x_{k+1} - b_k|^2_{C_k^-1}
 *        + sum_{k=1}^{T}   1/2 dt |y_k - h(x_k)|^2_{R^-1}
 *        + sum_{k=1}^{T}   1/2 dt div f(x_k)
 *
 * where (A_k, b_k, C_k) is the interval's conditional value function of
 * Eq. (37) integrated over [t_k, t_{k+1}] without the measurement term
 * (one explicit Euler step from the boundary values A=I, b=C=eta=J=0, or the
 * exact exponential solution).  The measurement on x_{k+1} enters as the
 * interval's (J_k, eta_k) on its start state (Eq. 37, eta and J rows).
 *
 * The linear argmin is computed by a different algorithm than the method: a
 * covariance-form Kalman filter on the equivalent forward model
 * x_{k+1} = Phi_k x_k + beta_k + N(0, Sigma_k),  Phi = A^-1, beta = -A^-1 b,
 * Sigma = A^-1 C A^-T, followed by the Rauch-Tung-Striebel smoother
 * (Section 2.5: the backward pass is the Kalman-Bucy filter, the forward
 * pass the RTS smoother).  Nonlinear models are handled by iterated
 * linearisation (Section 4.4, Gauss-Newton).  The paper's own combine rule
 * (Eq. 36) is restated here separately for the pins that test it.
 *
 * Matrices are row-major, FP64, plain loops, no BLAS.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_SINGULAR -4
#define ORC_ERR_ARG -1

/* ------------------------------------------------------------------ */
/* small dense helpers                                                 */
/* ------------------------------------------------------------------ */

static void mm(int n, int k, int m, const double *A, const double *B, double *C)
{ /* C (n x m) = A (n x k) B (k x m) */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * m + j];
            C[i * m + j] = s;
        }
}

static void mmT(int n, int k, int m, const double *A, const double *B, double *C)
{ /* C (n x m) = A (n x k) B^T, B is (m x k) */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += A[i * k + l] * B[j * k + l];
            C[i * m + j] = s;
        }
}

static void mTm(int n, int k, int m, const double *A, const double *B, double *C)
{ /* C (n x m) = A^T B, A is (k x n), B is (k x m) */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += A[l * n + i] * B[l * m + j];
            C[i * m + j] = s;
        }
}

static void mv(int n, int k, const double *A, const double *x, double *y)
{
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int l = 0; l < k; ++l) s += A[i * k + l] * x[l];
        y[i] = s;
    }
}

static void mTv(int n, int k, const double *A, const double *x, double *y)
{ /* y (n) = A^T x, A is (k x n) */
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int l = 0; l < k; ++l) s += A[l * n + i] * x[l];
        y[i] = s;
    }
}

static void eye(int n, double *I)
{
    memset(I, 0, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
}

static void symmetrise(int n, double *S)
{
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double a = 0.5 * (S[i * n + j] + S[j * n + i]);
            S[i * n + j] = a;
            S[j * n + i] = a;
        }
}

/* Gauss-Jordan inverse with partial pivoting.  Returns 0 or ORC_ERR_SINGULAR. */
static int inv(int n, const double *A, double *X)
{
    double *W = (double *)malloc(sizeof(double) * n * 2 * n);
    if (!W) return ORC_ERR_ARG;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j)
            W[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(W[r * 2 * n + c]) > fabs(W[p * 2 * n + c])) p = r;
        if (W[p * 2 * n + c] == 0.0) { free(W); return ORC_ERR_SINGULAR; }
        if (p != c)
            for (int j = 0; j < 2 * n; ++j) {
                double t = W[c * 2 * n + j];
                W[c * 2 * n + j] = W[p * 2 * n + j];
                W[p * 2 * n + j] = t;
            }
        double d = W[c * 2 * n + c];
        for (int j = 0; j < 2 * n; ++j) W[c * 2 * n + j] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = W[r * 2 * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * n; ++j) W[r * 2 * n + j] -= f * W[c * 2 * n + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) X[i * n + j] = W[i * 2 * n + n + j];
    free(W);
    return ORC_OK;
}

/* Matrix exponential by scaling and squaring of a truncated Taylor series
 * (Moler and Van Loan, "Nineteen dubious ways", methods 1 and 3): scale so the
 * 1-norm is below 1/2, sum 30 Taylor terms, square back. */
static void expm(int n, const double *A, double *E)
{
    double nrm = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fabs(A[i * n + j]);
        if (s > nrm) nrm = s;
    }
    int sq = 0;
    while (nrm > 0.5) { nrm *= 0.5; ++sq; }
    double scale = ldexp(1.0, -sq);
    double *X = (double *)malloc(sizeof(double) * n * n);
    double *term = (double *)malloc(sizeof(double) * n * n);
    double *tmp = (double *)malloc(sizeof(double) * n * n);
    for (int i = 0; i < n * n; ++i) X[i] = A[i] * scale;
    eye(n, E);
    eye(n, term);
    for (int k = 1; k <= 30; ++k) {
        mm(n, n, n, term, X, tmp);
        for (int i = 0; i < n * n; ++i) { term[i] = tmp[i] / k; E[i] += term[i]; }
    }
    for (int s = 0; s < sq; ++s) {
        mm(n, n, n, E, E, tmp);
        memcpy(E, tmp, sizeof(double) * n * n);
    }
    free(X); free(term); free(tmp);
}

/* ------------------------------------------------------------------ */
/* discretisation of one interval                                      */
/* ------------------------------------------------------------------ */

/*
 * Interval element (A, b, C) of Eq. (37) for a linear-affine drift F x + c
 * with Q = L W L^T over one step dt, measurement terms excluded.
 *   mode 0 (Euler, Section 5.1): one explicit Euler step of the A, b, C rows
 *          of Eq. (37) from the boundary values A=I, b=0, C=0 (Eq. 37 text):
 *          A = I - dt F, b = -dt c, C = dt Q   (reversed drift F~ = -F, c~ = -c).
 *   mode 1 (exact): the same rows solved exactly with constant coefficients:
 *          A = e^{-F dt}, C = int_0^dt e^{-F u} Q e^{-F^T u} du,
 *          b = -int_0^dt e^{-F u} du c, via Van Loan block exponentials.
 */
int orc_discretise(int n, double dt, const double *F, const double *c,
                   const double *Q, int mode, double *A, double *b, double *C)
{
    if (mode == 0) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                A[i * n + j] = (i == j ? 1.0 : 0.0) - dt * F[i * n + j];
                C[i * n + j] = dt * Q[i * n + j];
            }
        for (int i = 0; i < n; ++i) b[i] = -dt * c[i];
        return ORC_OK;
    }
    if (mode != 1) return ORC_ERR_ARG;
    int N2 = 2 * n;
    double *Z = (double *)calloc((size_t)N2 * N2, sizeof(double));
    double *EZ = (double *)malloc(sizeof(double) * N2 * N2);
    /* Z = [[-F, Q], [0, F^T]] dt:  e^Z = [[e^{-F dt}, G], [0, e^{F^T dt}]],
     * G = int_0^dt e^{-F(dt-s)} Q e^{F^T s} ds = C e^{F^T dt}  =>  C = G A^T. */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            Z[i * N2 + j] = -F[i * n + j] * dt;
            Z[i * N2 + n + j] = Q[i * n + j] * dt;
            Z[(n + i) * N2 + n + j] = F[j * n + i] * dt;
        }
    expm(N2, Z, EZ);
    double *G = (double *)calloc((size_t)n * n, sizeof(double));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            A[i * n + j] = EZ[i * N2 + j];
            G[i * n + j] = EZ[i * N2 + n + j];
        }
    mmT(n, n, n, G, A, C);
    symmetrise(n, C);
    free(Z); free(EZ); free(G);
    /* b: Z' = [[-F, c], [0, 0]] dt, top-right of e^{Z'} = int_0^dt e^{-F u} du c */
    int N1 = n + 1;
    double *Z1 = (double *)calloc((size_t)N1 * N1, sizeof(double));
    double *E1 = (double *)malloc(sizeof(double) * N1 * N1);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) Z1[i * N1 + j] = -F[i * n + j] * dt;
        Z1[i * N1 + n] = c[i] * dt;
    }
    expm(N1, Z1, E1);
    for (int i = 0; i < n; ++i) b[i] = -E1[i * N1 + n];
    free(Z1); free(E1);
    return ORC_OK;
}

/* Forward transition of an interval element: x_{k+1} = Phi x_k + beta + N(0, Sigma)
 * with Phi = A^-1, beta = -A^-1 b, Sigma = A^-1 C A^-T (the quadratic
 * |x_k - A x_{k+1} - b|^2_{C^-1} rewritten in x_{k+1}). */
int orc_forward_model(int n, const double *A, const double *b, const double *C,
                      double *Phi, double *beta, double *Sigma)
{
    if (inv(n, A, Phi)) return ORC_ERR_SINGULAR;
    double *t = (double *)malloc(sizeof(double) * n * n);
    mv(n, n, Phi, b, beta);
    for (int i = 0; i < n; ++i) beta[i] = -beta[i];
    mm(n, n, n, Phi, C, t);
    mmT(n, n, n, t, Phi, Sigma);
    symmetrise(n, Sigma);
    free(t);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Kalman filter + RTS smoother (covariance form)                      */
/* ------------------------------------------------------------------ */

/*
 * Sequential filter and smoother for
 *   x_0 ~ N(m0, P0),  x_{k+1} = Phi_k x_k + beta_k + N(0, Sigma_k),
 * with a Gaussian information term (J_k, eta_k) on x_{k+1}:
 *   exp(-1/2 x^T J_k x + eta_k^T x)   (k = 0..T-1).
 * For a measurement y = H x + r + N(0, R/dt) this is J = dt H^T R^-1 H,
 * eta = dt H^T R^-1 (y - r).  Per-step arrays use the given strides in
 * doubles (0 = the same matrix for every step).
 *
 * Update in information variables: P+ = (P-^-1 + J)^-1 = (I + P- J)^-1 P-,
 * m+ = m- + P+ (eta - J m-).  RTS: G = P_k Phi^T (P-_{k+1})^-1,
 * x_k = m_k + G (x_{k+1} - m-_{k+1}), x_T = m_T  (Section 2.5).
 * Outputs: x (T+1, n); optional mf (T+1, n), Pf (T+1, n, n) filtered moments.
 */
int orc_kf_rts(int n, int T,
               const double *Phi, long sPhi, const double *beta, long sbeta,
               const double *Sig, long sSig, const double *J, long sJ,
               const double *eta, long seta, const double *m0, const double *P0,
               double *x, double *mf_out, double *Pf_out)
{
    size_t nn = (size_t)n * n;
    double *mf = mf_out ? mf_out : (double *)malloc(sizeof(double) * (size_t)(T + 1) * n);
    double *Pf = Pf_out ? Pf_out : (double *)malloc(sizeof(double) * (size_t)(T + 1) * nn);
    double *mp = (double *)malloc(sizeof(double) * (size_t)(T + 1) * n);
    double *Pp = (double *)malloc(sizeof(double) * (size_t)(T + 1) * nn);
    double *t1 = (double *)malloc(sizeof(double) * nn);
    double *t2 = (double *)malloc(sizeof(double) * nn);
    double *t3 = (double *)malloc(sizeof(double) * nn);
    double *u = (double *)malloc(sizeof(double) * n);
    double *w = (double *)malloc(sizeof(double) * n);
    int rc = ORC_OK;
    memcpy(mf, m0, sizeof(double) * n);
    memcpy(Pf, P0, sizeof(double) * nn);
    for (int k = 0; k < T; ++k) {
        const double *Ph = Phi + (size_t)k * sPhi, *be = beta + (size_t)k * sbeta;
        const double *Sg = Sig + (size_t)k * sSig, *Jk = J + (size_t)k * sJ;
        const double *ek = eta + (size_t)k * seta;
        const double *m = mf + (size_t)k * n, *P = Pf + (size_t)k * nn;
        double *mpk = mp + (size_t)(k + 1) * n, *Ppk = Pp + (size_t)(k + 1) * nn;
        /* predict */
        mv(n, n, Ph, m, mpk);
        for (int i = 0; i < n; ++i) mpk[i] += be[i];
        mm(n, n, n, Ph, P, t1);
        mmT(n, n, n, t1, Ph, Ppk);
        for (size_t i = 0; i < nn; ++i) Ppk[i] += Sg[i];
        symmetrise(n, Ppk);
        /* update with the information term */
        mm(n, n, n, Ppk, Jk, t1);                /* P- J */
        for (int i = 0; i < n; ++i) t1[i * n + i] += 1.0;
        if (inv(n, t1, t2)) { rc = ORC_ERR_SINGULAR; goto done; }
        double *Pn = Pf + (size_t)(k + 1) * nn, *mn = mf + (size_t)(k + 1) * n;
        mm(n, n, n, t2, Ppk, Pn);
        symmetrise(n, Pn);
        mv(n, n, Jk, mpk, u);
        for (int i = 0; i < n; ++i) u[i] = ek[i] - u[i];
        mv(n, n, Pn, u, w);
        for (int i = 0; i < n; ++i) mn[i] = mpk[i] + w[i];
    }
    /* RTS smoother */
    memcpy(x + (size_t)T * n, mf + (size_t)T * n, sizeof(double) * n);
    for (int k = T - 1; k >= 0; --k) {
        const double *Ph = Phi + (size_t)k * sPhi;
        if (inv(n, Pp + (size_t)(k + 1) * nn, t1)) { rc = ORC_ERR_SINGULAR; goto done; }
        mmT(n, n, n, Pf + (size_t)k * nn, Ph, t2);    /* P_k Phi^T */
        mm(n, n, n, t2, t1, t3);                        /* G */
        for (int i = 0; i < n; ++i) u[i] = x[(size_t)(k + 1) * n + i] - mp[(size_t)(k + 1) * n + i];
        mv(n, n, t3, u, w);
        for (int i = 0; i < n; ++i) x[(size_t)k * n + i] = mf[(size_t)k * n + i] + w[i];
    }
done:
    if (!mf_out) free(mf);
    if (!Pf_out) free(Pf);
    free(mp); free(Pp); free(t1); free(t2); free(t3); free(u); free(w);
    return rc;
}

/*
 * Two-filter smoother (Section 4.3, Eq. 42 and the max-product form of
 * Section 3.4) in information form: a backward information filter gives the
 * information (Lam_k, zeta_k) on x_k from the information terms on
 * x_{k+1}..x_T, and the smoothed state is
 *   x_k = (P_k^-1 + Lam_k)^-1 (P_k^-1 m_k + zeta_k)
 * with the forward filter moments (m_k, P_k).  Backward prediction through
 * x_{k+1} = Phi x_k + beta + N(0, Sigma):  Om = L'(I + Sigma L')^-1,
 * om = (I + L' Sigma)^-1 z',  Lam_k = Phi^T Om Phi,
 * zeta_k = Phi^T (om - Om beta), where (L', z') already holds x_{k+1}'s term.
 */
int orc_two_filter(int n, int T,
                   const double *Phi, long sPhi, const double *beta, long sbeta,
                   const double *Sig, long sSig, const double *J, long sJ,
                   const double *eta, long seta, const double *m0, const double *P0,
                   double *x)
{
    size_t nn = (size_t)n * n;
    double *mf = (double *)malloc(sizeof(double) * (size_t)(T + 1) * n);
    double *Pf = (double *)malloc(sizeof(double) * (size_t)(T + 1) * nn);
    double *xs = (double *)malloc(sizeof(double) * (size_t)(T + 1) * n);
    int rc = orc_kf_rts(n, T, Phi, sPhi, beta, sbeta, Sig, sSig, J, sJ, eta, seta,
                        m0, P0, xs, mf, Pf);
    free(xs);
    if (rc) { free(mf); free(Pf); return rc; }
    double *Lam = (double *)calloc(nn, sizeof(double));
    double *zeta = (double *)calloc(n, sizeof(double));
    double *Lp = (double *)malloc(sizeof(double) * nn);
    double *zp = (double *)malloc(sizeof(double) * n);
    double *t1 = (double *)malloc(sizeof(double) * nn);
    double *t2 = (double *)malloc(sizeof(double) * nn);
    double *Om = (double *)malloc(sizeof(double) * nn);
    double *u = (double *)malloc(sizeof(double) * n);
    double *w = (double *)malloc(sizeof(double) * n);
    /* x_T: no information from later terms */
    memcpy(x + (size_t)T * n, mf + (size_t)T * n, sizeof(double) * n);
    for (int k = T - 1; k >= 0 && rc == ORC_OK; --k) {
        const double *Ph = Phi + (size_t)k * sPhi, *be = beta + (size_t)k * sbeta;
        const double *Sg = Sig + (size_t)k * sSig, *Jk = J + (size_t)k * sJ;
        const double *ek = eta + (size_t)k * seta;
        /* add x_{k+1}'s own information term */
        for (size_t i = 0; i < nn; ++i) Lp[i] = Lam[i] + Jk[i];
        for (int i = 0; i < n; ++i) zp[i] = zeta[i] + ek[i];
        /* backward prediction to x_k */
        mm(n, n, n, Sg, Lp, t1);                      /* Sigma L' */
        for (int i = 0; i < n; ++i) t1[i * n + i] += 1.0;
        if (inv(n, t1, t2)) { rc = ORC_ERR_SINGULAR; break; }   /* (I + Sigma L')^-1 */
        mm(n, n, n, Lp, t2, Om);                      /* L' (I + Sigma L')^-1 */
        symmetrise(n, Om);
        mTv(n, n, t2, zp, u);                          /* (I + L' Sigma)^-1 z' */
        mv(n, n, Om, be, w);
        for (int i = 0; i < n; ++i) u[i] -= w[i];
        mTm(n, n, n, Ph, Om, t1);                      /* Phi^T Om */
        mm(n, n, n, t1, Ph, Lam);
        symmetrise(n, Lam);
        mTv(n, n, Ph, u, zeta);
        /* combine with the forward filter at k */
        const double *m = mf + (size_t)k * n, *P = Pf + (size_t)k * nn;
        if (inv(n, P, t1)) { rc = ORC_ERR_SINGULAR; break; }   /* P^-1 */
        mv(n, n, t1, m, u);
        for (int i = 0; i < n; ++i) u[i] += zeta[i];
        for (size_t i = 0; i < nn; ++i) t1[i] += Lam[i];
        if (inv(n, t1, t2)) { rc = ORC_ERR_SINGULAR; break; }
        mv(n, n, t2, u, x + (size_t)k * n);
    }
    free(mf); free(Pf); free(Lam); free(zeta); free(Lp); free(zp);
    free(t1); free(t2); free(Om); free(u); free(w);
    return rc;
}

/* ------------------------------------------------------------------ */
/* the paper's combine rule and its sequential use                     */
/* ------------------------------------------------------------------ */
/* Element layout (full matrices): [A n*n | b n | C n*n | eta n | J n*n]. */
#define E_A(e, n) (e)
#define E_B(e, n) ((e) + (n) * (n))
#define E_C(e, n) ((e) + (n) * (n) + (n))
#define E_ETA(e, n) ((e) + 2 * (n) * (n) + (n))
#define E_J(e, n) ((e) + 2 * (n) * (n) + 2 * (n))

/*
 * (A,b,C,eta,J)_ij = e_i (x) e_j, the linear-affine combination rule of
 * Section 4.1 (Eq. 36) with i on [s, gamma] and j on [gamma, t]:
 *   A_ij = A_j (I + C_i J_j)^-1 A_i
 *   b_ij = A_j (I + C_i J_j)^-1 (b_i + C_i eta_j) + b_j
 *   C_ij = A_j (I + C_i J_j)^-1 C_i A_j^T + C_j
 *   eta_ij = A_i^T (I + J_j C_i)^-1 (eta_j - J_j b_i) + eta_i
 *   J_ij = A_i^T (I + J_j C_i)^-1 J_j A_i + J_i
 */
int orc_combine(int n, const double *ei, const double *ej, double *out)
{
    size_t nn = (size_t)n * n;
    const double *Ai = E_A(ei, n), *bi = E_B(ei, n), *Ci = E_C(ei, n), *hi = E_ETA(ei, n), *Ji = E_J(ei, n);
    const double *Aj = E_A(ej, n), *bj = E_B(ej, n), *Cj = E_C(ej, n), *hj = E_ETA(ej, n), *Jj = E_J(ej, n);
    double *M = (double *)malloc(sizeof(double) * nn), *Mi = (double *)malloc(sizeof(double) * nn);
    double *N = (double *)malloc(sizeof(double) * nn), *Ni = (double *)malloc(sizeof(double) * nn);
    double *t1 = (double *)malloc(sizeof(double) * nn), *t2 = (double *)malloc(sizeof(double) * nn);
    double *u = (double *)malloc(sizeof(double) * n), *w = (double *)malloc(sizeof(double) * n);
    double *o = (double *)malloc(sizeof(double) * (3 * nn + 2 * n));
    int rc = ORC_OK;
    mm(n, n, n, Ci, Jj, M);
    for (int i = 0; i < n; ++i) M[i * n + i] += 1.0;
    mm(n, n, n, Jj, Ci, N);
    for (int i = 0; i < n; ++i) N[i * n + i] += 1.0;
    if (inv(n, M, Mi) || inv(n, N, Ni)) { rc = ORC_ERR_SINGULAR; goto done; }
    /* A */
    mm(n, n, n, Aj, Mi, t1);
    mm(n, n, n, t1, Ai, E_A(o, n));
    /* b */
    mv(n, n, Ci, hj, u);
    for (int i = 0; i < n; ++i) u[i] += bi[i];
    mv(n, n, t1, u, w);
    for (int i = 0; i < n; ++i) E_B(o, n)[i] = w[i] + bj[i];
    /* C */
    mm(n, n, n, t1, Ci, t2);
    mmT(n, n, n, t2, Aj, E_C(o, n));
    for (size_t i = 0; i < nn; ++i) E_C(o, n)[i] += Cj[i];
    symmetrise(n, E_C(o, n));
    /* eta */
    mTm(n, n, n, Ai, Ni, t1);                     /* A_i^T (I + J_j C_i)^-1 */
    mv(n, n, Jj, bi, u);
    for (int i = 0; i < n; ++i) u[i] = hj[i] - u[i];
    mv(n, n, t1, u, w);
    for (int i = 0; i < n; ++i) E_ETA(o, n)[i] = w[i] + hi[i];
    /* J */
    mm(n, n, n, t1, Jj, t2);
    mm(n, n, n, t2, Ai, E_J(o, n));
    for (size_t i = 0; i < nn; ++i) E_J(o, n)[i] += Ji[i];
    symmetrise(n, E_J(o, n));
    memcpy(out, o, sizeof(double) * (3 * nn + 2 * n));
done:
    free(M); free(Mi); free(N); free(Ni); free(t1); free(t2); free(u); free(w); free(o);
    return rc;
}

/*
 * Interval elements of a linear model in original-time order: element k spans
 * [t_k, t_{k+1}]; its start state (phi) is x_{k+1} and its end state (z) is
 * x_k (time reversal, Section 2.2).  (A_k, b_k, C_k) as in orc_discretise and
 * the measurement y_{k+1} = H x_{k+1} + r + noise on the start state:
 * J_k = dt H^T R^-1 H, eta_k = dt H^T R^-1 (y_{k+1} - r)  (Eq. 37 eta, J rows
 * after one Euler step from the zero boundary values).
 * elems: (T, 3n^2 + 2n).
 */
int orc_elements_lti(int n, int m, int T, double dt, const double *A, const double *b,
                     const double *C, const double *H, const double *r,
                     const double *R, const double *y, double *elems)
{
    size_t nn = (size_t)n * n, es = 3 * nn + 2 * (size_t)n;
    double *Ri = (double *)malloc(sizeof(double) * m * m);
    double *HtRi = (double *)malloc(sizeof(double) * n * m);
    double *J = (double *)malloc(sizeof(double) * nn);
    double *d = (double *)malloc(sizeof(double) * m);
    if (inv(m, R, Ri)) { free(Ri); free(HtRi); free(J); free(d); return ORC_ERR_SINGULAR; }
    mTm(n, m, m, H, Ri, HtRi);
    mm(n, m, n, HtRi, H, J);
    for (int k = 0; k < T; ++k) {
        double *e = elems + (size_t)k * es;
        memcpy(E_A(e, n), A, sizeof(double) * nn);
        memcpy(E_B(e, n), b, sizeof(double) * n);
        memcpy(E_C(e, n), C, sizeof(double) * nn);
        for (int i = 0; i < m; ++i) d[i] = y[(size_t)k * m + i] - r[i];
        mv(n, m, HtRi, d, E_ETA(e, n));
        for (int i = 0; i < n; ++i) E_ETA(e, n)[i] *= dt;
        for (size_t i = 0; i < nn; ++i) E_J(e, n)[i] = dt * J[i];
    }
    free(Ri); free(HtRi); free(J); free(d);
    return ORC_OK;
}

/*
 * Value functions by a sequential fold of the combine (Eq. 32, second line):
 * V(., tau_i) = a_i (x) a_{i+1} (x) ... (x) a_T with the terminal element
 * a_T = -log p(x(t0)) = (0, 0, 0, P0^-1 m0, P0^-1) (Eq. 31).  In original time
 * this is S_{k+1}, v_{k+1} = (J, eta) of e_k (x) [S_k, v_k], S_0 = P0^-1.
 * Outputs S (T+1, n, n), v (T+1, n).
 */
int orc_filter_by_combine(int n, int T, const double *elems, const double *m0,
                          const double *P0, double *S, double *v)
{
    size_t nn = (size_t)n * n, es = 3 * nn + 2 * (size_t)n;
    double *acc = (double *)calloc(es, sizeof(double));
    double *tmp = (double *)malloc(sizeof(double) * es);
    if (inv(n, P0, E_J(acc, n))) { free(acc); free(tmp); return ORC_ERR_SINGULAR; }
    mv(n, n, E_J(acc, n), m0, E_ETA(acc, n));
    memcpy(S, E_J(acc, n), sizeof(double) * nn);
    memcpy(v, E_ETA(acc, n), sizeof(double) * n);
    for (int k = 0; k < T; ++k) {
        if (orc_combine(n, elems + (size_t)k * es, acc, tmp)) { free(acc); free(tmp); return ORC_ERR_SINGULAR; }
        memcpy(acc, tmp, sizeof(double) * es);
        memcpy(S + (size_t)(k + 1) * nn, E_J(acc, n), sizeof(double) * nn);
        memcpy(v + (size_t)(k + 1) * n, E_ETA(acc, n), sizeof(double) * n);
    }
    free(acc); free(tmp);
    return ORC_OK;
}

/*
 * The paper's two-filter smoother, literally (Section 4.3, Eq. 42-43): the
 * prefix e (x) a_0 (x) ... (x) a_{i-1} in reversed time, with the first
 * element replaced by abar_0 = e (x) a_0 (C_e = kappa I, kappa -> inf):
 *   Abar_0 = 0, bbar_0 = A_0 J_0^-1 eta_0 + b_0, Cbar_0 = A_0 J_0^-1 A_0^T + C_0,
 * then phi*(tau_i) = (I + Cbar S)^-1 (bbar + Cbar v).  (The printed bbar_0 lacks
 * the + b_0 that the combine with e yields.)  Needs J_0 invertible, i.e.
 * full-state measurements.  Reversed-time element a_i is original element
 * T-1-i.  Output x (T+1, n).
 */
int orc_two_filter_paper(int n, int T, const double *elems, const double *m0,
                         const double *P0, double *x)
{
    size_t nn = (size_t)n * n, es = 3 * nn + 2 * (size_t)n;
    double *S = (double *)malloc(sizeof(double) * (size_t)(T + 1) * nn);
    double *v = (double *)malloc(sizeof(double) * (size_t)(T + 1) * n);
    double *acc = (double *)calloc(es, sizeof(double));
    double *tmp = (double *)malloc(sizeof(double) * es);
    double *Ji = (double *)malloc(sizeof(double) * nn);
    double *t1 = (double *)malloc(sizeof(double) * nn), *t2 = (double *)malloc(sizeof(double) * nn);
    double *u = (double *)malloc(sizeof(double) * n), *w = (double *)malloc(sizeof(double) * n);
    int rc = orc_filter_by_combine(n, T, elems, m0, P0, S, v);
    if (rc) goto done;
    /* tau_0 <-> x_T: the prefix is e alone, Cbar -> inf: phi = S^-1 v */
    if (inv(n, S + (size_t)T * nn, t1)) { rc = ORC_ERR_SINGULAR; goto done; }
    mv(n, n, t1, v + (size_t)T * n, x + (size_t)T * n);
    for (int i = 1; i <= T; ++i) {
        const double *a = elems + (size_t)(T - i) * es;   /* a_{i-1} */
        if (i == 1) {
            if (inv(n, E_J(a, n), Ji)) { rc = ORC_ERR_SINGULAR; goto done; }
            memset(acc, 0, sizeof(double) * es);
            mm(n, n, n, E_A(a, n), Ji, t1);
            mv(n, n, t1, E_ETA(a, n), E_B(acc, n));
            for (int j = 0; j < n; ++j) E_B(acc, n)[j] += E_B(a, n)[j];
            mmT(n, n, n, t1, E_A(a, n), E_C(acc, n));
            for (size_t j = 0; j < nn; ++j) E_C(acc, n)[j] += E_C(a, n)[j];
            symmetrise(n, E_C(acc, n));
            memcpy(E_ETA(acc, n), E_ETA(a, n), sizeof(double) * n);
            memcpy(E_J(acc, n), E_J(a, n), sizeof(double) * nn);
        } else {
            if (orc_combine(n, acc, a, tmp)) { rc = ORC_ERR_SINGULAR; goto done; }
            memcpy(acc, tmp, sizeof(double) * es);
        }
        /* phi*(tau_i) with V(., tau_i) = filter at x_{T-i} */
        const double *Sk = S + (size_t)(T - i) * nn, *vk = v + (size_t)(T - i) * n;
        mm(n, n, n, E_C(acc, n), Sk, t1);
        for (int j = 0; j < n; ++j) t1[j * n + j] += 1.0;
        if (inv(n, t1, t2)) { rc = ORC_ERR_SINGULAR; goto done; }
        mv(n, n, E_C(acc, n), vk, u);
        for (int j = 0; j < n; ++j) u[j] += E_B(acc, n)[j];
        mv(n, n, t2, u, x + (size_t)(T - i) * n);
    }
done:
    free(S); free(v); free(acc); free(tmp); free(Ji); free(t1); free(t2); free(u); free(w);
    return rc;
}

/* ------------------------------------------------------------------ */
/* linear-model driver and cost                                        */
/* ------------------------------------------------------------------ */

/* MAP trajectory of a linear-affine model (Eq. 14) by the sequential
 * filter + smoother: discretise (orc_discretise), turn into the forward model
 * and run orc_kf_rts (smoother 0) or orc_two_filter (smoother 1).
 * y (T, m) holds y_1..y_T.  Optional filter outputs mf (T+1, n), Pf (T+1, n, n). */
int orc_smooth_lti(int n, int m, int T, double dt, int mode, int smoother,
                   const double *F, const double *c, const double *Q,
                   const double *H, const double *r, const double *R,
                   const double *m0, const double *P0, const double *y,
                   double *x, double *mf, double *Pf)
{
    size_t nn = (size_t)n * n;
    double *A = (double *)malloc(sizeof(double) * nn), *b = (double *)malloc(sizeof(double) * n);
    double *C = (double *)malloc(sizeof(double) * nn);
    double *Phi = (double *)malloc(sizeof(double) * nn), *beta = (double *)malloc(sizeof(double) * n);
    double *Sig = (double *)malloc(sizeof(double) * nn);
    double *Ri = (double *)malloc(sizeof(double) * m * m), *HtRi = (double *)malloc(sizeof(double) * n * m);
    double *J = (double *)malloc(sizeof(double) * nn);
    double *eta = (double *)malloc(sizeof(double) * (size_t)T * n);
    double *d = (double *)malloc(sizeof(double) * m);
    int rc = orc_discretise(n, dt, F, c, Q, mode, A, b, C);
    if (!rc) rc = orc_forward_model(n, A, b, C, Phi, beta, Sig);
    if (!rc && inv(m, R, Ri)) rc = ORC_ERR_SINGULAR;
    if (!rc) {
        mTm(n, m, m, H, Ri, HtRi);
        mm(n, m, n, HtRi, H, J);
        for (size_t i = 0; i < nn; ++i) J[i] *= dt;
        for (int k = 0; k < T; ++k) {
            for (int i = 0; i < m; ++i) d[i] = y[(size_t)k * m + i] - r[i];
            mv(n, m, HtRi, d, eta + (size_t)k * n);
            for (int i = 0; i < n; ++i) eta[(size_t)k * n + i] *= dt;
        }
        if (smoother == 0)
            rc = orc_kf_rts(n, T, Phi, 0, beta, 0, Sig, 0, J, 0, eta, n, m0, P0, x, mf, Pf);
        else
            rc = orc_two_filter(n, T, Phi, 0, beta, 0, Sig, 0, J, 0, eta, n, m0, P0, x);
    }
    free(A); free(b); free(C); free(Phi); free(beta); free(Sig); free(Ri); free(HtRi);
    free(J); free(eta); free(d);
    return rc;
}

/* ------------------------------------------------------------------ */
/* nonlinear models: drift, Jacobians, measurement, divergence          */
/* ------------------------------------------------------------------ */
/* kind 1: coordinated turn (Section 5.2, Eq. 46), n = 5, m = 2
 *   f = (x2, x3, -x4 x3, x4 x2, 0), h = (sqrt(x0^2+x1^2), atan2(x1, x0)).
 * kind 2: cubic drift f = F x + c - gamma x^3 (elementwise), h = H x + r.
 * kind 0: linear model, i.e. kind 2 with gamma = 0. */

static void drift_jac(int kind, int n, const double *x, const double *F, const double *c,
                      double gamma, double *f, double *Fj)
{
    if (kind == 1) {
        memset(Fj, 0, sizeof(double) * 25);
        f[0] = x[2]; f[1] = x[3]; f[2] = -x[4] * x[3]; f[3] = x[4] * x[2]; f[4] = 0.0;
        Fj[0 * 5 + 2] = 1.0;
        Fj[1 * 5 + 3] = 1.0;
        Fj[2 * 5 + 3] = -x[4]; Fj[2 * 5 + 4] = -x[3];
        Fj[3 * 5 + 2] = x[4];  Fj[3 * 5 + 4] = x[2];
    } else {
        for (int i = 0; i < n; ++i) {
            double s = c[i];
            for (int j = 0; j < n; ++j) { s += F[i * n + j] * x[j]; Fj[i * n + j] = F[i * n + j]; }
            f[i] = s - gamma * x[i] * x[i] * x[i];
            Fj[i * n + i] -= 3.0 * gamma * x[i] * x[i];
        }
    }
}

/* divergence of f and its gradient */
static double divergence(int kind, int n, const double *x, const double *F, double gamma, double *grad)
{
    if (kind == 1) { for (int i = 0; i < n; ++i) grad[i] = 0.0; return 0.0; }
    double d = 0.0;
    for (int i = 0; i < n; ++i) { d += F[i * n + i] - 3.0 * gamma * x[i] * x[i]; grad[i] = -6.0 * gamma * x[i]; }
    return d;
}

static double wrap_pi(double a)
{
    const double twopi = 6.283185307179586476925286766559;
    a = fmod(a + 3.14159265358979323846, twopi);
    if (a < 0) a += twopi;
    return a - 3.14159265358979323846;
}

/* residual y - h(x) (bearing wrapped) and Jacobian of h */
static void meas_res_jac(int kind, int n, int m, const double *x, const double *y,
                         const double *H, const double *r, double *res, double *Hj)
{
    if (kind == 1) {
        double rho2 = x[0] * x[0] + x[1] * x[1], rho = sqrt(rho2);
        res[0] = y[0] - rho;
        res[1] = wrap_pi(y[1] - atan2(x[1], x[0]));
        memset(Hj, 0, sizeof(double) * 10);
        Hj[0] = x[0] / rho; Hj[1] = x[1] / rho;
        Hj[5] = -x[1] / rho2; Hj[6] = x[0] / rho2;
    } else {
        for (int i = 0; i < m; ++i) {
            double s = r[i];
            for (int j = 0; j < n; ++j) { s += H[i * n + j] * x[j]; Hj[i * n + j] = H[i * n + j]; }
            res[i] = y[i] - s;
        }
    }
}

/*
 * Discrete Onsager-Machlup cost (Eq. 2) of trajectory x (T+1, n), Euler
 * intervals: dynamics residual x_k - x_{k+1} + dt f(x_{k+1}) with weight
 * (dt Q)^-1, measurement residuals with weight dt R^-1 at k = 1..T, divergence
 * 1/2 dt div f(x_k) at k = 1..T, prior at x_0.  kind 0: linear model
 * (F, c, H, r).  Requires Q invertible.  Constant terms are omitted.
 */
int orc_cost(int kind, int n, int m, int T, double dt, const double *F, const double *c,
             double gamma, const double *Q, const double *H, const double *r,
             const double *R, const double *m0, const double *P0, const double *y,
             const double *x, double *cost)
{
    size_t nn = (size_t)n * n;
    double *Qi = (double *)malloc(sizeof(double) * nn), *Ri = (double *)malloc(sizeof(double) * m * m);
    double *P0i = (double *)malloc(sizeof(double) * nn);
    double *f = (double *)malloc(sizeof(double) * n), *Fj = (double *)malloc(sizeof(double) * nn);
    double *e = (double *)malloc(sizeof(double) * n), *u = (double *)malloc(sizeof(double) * n);
    double *res = (double *)malloc(sizeof(double) * m), *Hj = (double *)malloc(sizeof(double) * m * n);
    double *g = (double *)malloc(sizeof(double) * n), *w = (double *)malloc(sizeof(double) * m);
    int rc = ORC_OK;
    if (inv(n, Q, Qi) || inv(m, R, Ri) || inv(n, P0, P0i)) { rc = ORC_ERR_SINGULAR; goto done; }
    double acc = 0.0;
    for (int i = 0; i < n; ++i) e[i] = x[i] - m0[i];
    mv(n, n, P0i, e, u);
    for (int i = 0; i < n; ++i) acc += 0.5 * e[i] * u[i];
    /* the linear model is the cubic drift with gamma = 0 */
    int dk = kind == 1 ? 1 : 2;
    double gm = kind == 0 ? 0.0 : gamma;
    for (int k = 0; k < T; ++k) {
        const double *xk = x + (size_t)k * n, *x1 = x + (size_t)(k + 1) * n;
        drift_jac(dk, n, x1, F, c, gm, f, Fj);
        for (int i = 0; i < n; ++i) e[i] = xk[i] - x1[i] + dt * f[i];
        mv(n, n, Qi, e, u);
        for (int i = 0; i < n; ++i) acc += 0.5 * e[i] * u[i] / dt;
        meas_res_jac(dk, n, m, x1, y + (size_t)k * m, H, r, res, Hj);
        mv(m, m, Ri, res, w);
        for (int i = 0; i < m; ++i) acc += 0.5 * dt * res[i] * w[i];
        acc += 0.5 * dt * divergence(dk, n, x1, F, gm, g);
    }
    *cost = acc;
done:
    free(Qi); free(Ri); free(P0i); free(f); free(Fj); free(e); free(u); free(res); free(Hj); free(g); free(w);
    return rc;
}

/*
 * Iterated linearisation (Section 4.4; continuous-time IEKS = Gauss-Newton):
 * starting from xbar (T+1, n), repeat `iters` times: linearise the drift at
 * x_{k+1}, f(x) ~ F_k x + c_k with F_k = F(xbar_{k+1}) and
 * c_k = f(xbar_{k+1}) - F_k xbar_{k+1}, and discretise that local linear
 * model over the interval (orc_discretise: mode 0 the Euler interval
 * A_k = I - dt F_k, b_k = -dt c_k, C_k = dt Q; mode 1 the exact solution of
 * the A, b, C rows of Eq. 37 with the local coefficients, A_k = e^{-F_k dt}
 * and so on); linearise the measurement at x_{k+1} (J_k = dt Hb^T R^-1 Hb,
 * eta_k = dt Hb^T R^-1 (y - h(xbar) + Hb xbar) - 1/2 dt grad div f(xbar));
 * solve the linear problem by filter + smoother, and set xbar to the result.
 * Output x (T+1, n).
 */
int orc_gauss_newton(int kind, int n, int m, int T, double dt, const double *F,
                     const double *c, double gamma, const double *Q, const double *H,
                     const double *r, const double *R, const double *m0,
                     const double *P0, const double *y, const double *xinit,
                     int iters, int mode, double *x)
{
    size_t nn = (size_t)n * n;
    double *Phi = (double *)malloc(sizeof(double) * (size_t)T * nn);
    double *beta = (double *)malloc(sizeof(double) * (size_t)T * n);
    double *Sig = (double *)malloc(sizeof(double) * (size_t)T * nn);
    double *J = (double *)malloc(sizeof(double) * (size_t)T * nn);
    double *eta = (double *)malloc(sizeof(double) * (size_t)T * n);
    double *xb = (double *)malloc(sizeof(double) * (size_t)(T + 1) * n);
    double *A = (double *)malloc(sizeof(double) * nn), *b = (double *)malloc(sizeof(double) * n);
    double *C = (double *)malloc(sizeof(double) * nn);
    double *f = (double *)malloc(sizeof(double) * n), *Fj = (double *)malloc(sizeof(double) * nn);
    double *Ri = (double *)malloc(sizeof(double) * m * m);
    double *res = (double *)malloc(sizeof(double) * m), *Hj = (double *)malloc(sizeof(double) * m * n);
    double *HtRi = (double *)malloc(sizeof(double) * n * m), *g = (double *)malloc(sizeof(double) * n);
    double *u = (double *)malloc(sizeof(double) * m);
    int rc = ORC_OK;
    if (inv(m, R, Ri)) { rc = ORC_ERR_SINGULAR; goto done; }
    if (kind == 0) { kind = 2; gamma = 0.0; }   /* linear = cubic drift with gamma = 0 */
    memcpy(xb, xinit, sizeof(double) * (size_t)(T + 1) * n);
    for (int it = 0; it < iters; ++it) {
        for (int k = 0; k < T; ++k) {
            const double *x1 = xb + (size_t)(k + 1) * n;
            drift_jac(kind, n, x1, F, c, gamma, f, Fj);
            for (int i = 0; i < n; ++i) {
                double s = f[i];
                for (int j = 0; j < n; ++j) s -= Fj[i * n + j] * x1[j];
                g[i] = s;                                   /* c_k of the local linear drift */
            }
            if (orc_discretise(n, dt, Fj, g, Q, mode, A, b, C)) { rc = ORC_ERR_ARG; goto done; }
            if (orc_forward_model(n, A, b, C, Phi + (size_t)k * nn, beta + (size_t)k * n,
                                  Sig + (size_t)k * nn)) { rc = ORC_ERR_SINGULAR; goto done; }
            meas_res_jac(kind, n, m, x1, y + (size_t)k * m, H, r, res, Hj);
            mTm(n, m, m, Hj, Ri, HtRi);
            mm(n, m, n, HtRi, Hj, J + (size_t)k * nn);
            for (size_t i = 0; i < nn; ++i) J[(size_t)k * nn + i] *= dt;
            for (int i = 0; i < m; ++i) {
                double s = res[i];
                for (int j = 0; j < n; ++j) s += Hj[i * n + j] * x1[j];
                u[i] = s;
            }
            mv(n, m, HtRi, u, eta + (size_t)k * n);
            divergence(kind, n, x1, F, gamma, g);
            for (int i = 0; i < n; ++i) eta[(size_t)k * n + i] = dt * eta[(size_t)k * n + i] - 0.5 * dt * g[i];
        }
        rc = orc_kf_rts(n, T, Phi, nn, beta, n, Sig, nn, J, nn, eta, n, m0, P0, x, NULL, NULL);
        if (rc) goto done;
        memcpy(xb, x, sizeof(double) * (size_t)(T + 1) * n);
    }
    if (iters <= 0) memcpy(x, xb, sizeof(double) * (size_t)(T + 1) * n);
done:
    free(Phi); free(beta); free(Sig); free(J); free(eta); free(xb); free(A); free(b); free(C);
    free(f); free(Fj); free(Ri); free(res); free(Hj); free(HtRi); free(g); free(u);
    return rc;
}

/* ------------------------------------------------------------------ */
/* gradient of a loss of the MAP trajectory (linear model, Euler)       */
/* ------------------------------------------------------------------ */

/*
 * Parameters theta = (F (n x n), log q, log r) with Q = q Q0, R = r R0.
 * x* = argmin M(x; theta) satisfies K(theta) x* = g(theta), K symmetric.
 *  - dLdx == NULL: L = M(x*(theta), theta) (the MAP cost, constants omitted
 *    unless logdet != 0, which adds 1/2 sum log det(2 pi C) + 1/2 sum
 *    log det(2 pi R/dt)); dL/dtheta = d_theta M at x* (envelope theorem).
 *  - otherwise: lambda = K^-1 dL/dx by the same filter + smoother with b = 0,
 *    information terms eta_k = dLdx_{k+1}, prior term P0^-1 lambda_0 - dLdx_0,
 *    and dL/dtheta = -d_theta [lambda^T grad_x M(x*, theta)] at fixed x*, lambda.
 * Requires Q0 invertible.  Output grad (n*n + 2), optional x (T+1, n).
 */
int orc_grad_lti(int n, int m, int T, double dt, const double *F, const double *c,
                 const double *Q0, double logq, const double *H, const double *r,
                 const double *R0, double logr, const double *m0, const double *P0,
                 const double *y, const double *dLdx, int logdet, double *grad,
                 double *x_out)
{
    size_t nn = (size_t)n * n;
    double q = exp(logq), rr = exp(logr);
    double *Q = (double *)malloc(sizeof(double) * nn), *R = (double *)malloc(sizeof(double) * m * m);
    double *x = (double *)malloc(sizeof(double) * (size_t)(T + 1) * n);
    double *lam = (double *)malloc(sizeof(double) * (size_t)(T + 1) * n);
    double *A = (double *)malloc(sizeof(double) * nn), *b = (double *)malloc(sizeof(double) * n);
    double *C = (double *)malloc(sizeof(double) * nn), *Ci = (double *)malloc(sizeof(double) * nn);
    double *Ri = (double *)malloc(sizeof(double) * m * m);
    double *rk = (double *)malloc(sizeof(double) * n), *sk = (double *)malloc(sizeof(double) * n);
    double *Cr = (double *)malloc(sizeof(double) * n), *Cs = (double *)malloc(sizeof(double) * n);
    double *e = (double *)malloc(sizeof(double) * m), *w = (double *)malloc(sizeof(double) * m);
    double *hl = (double *)malloc(sizeof(double) * m);
    int rc;
    for (size_t i = 0; i < nn; ++i) Q[i] = q * Q0[i];
    for (int i = 0; i < m * m; ++i) R[i] = rr * R0[i];
    rc = orc_smooth_lti(n, m, T, dt, 0, 0, F, c, Q, H, r, R, m0, P0, y, x, NULL, NULL);
    if (rc) goto done;
    if (x_out) memcpy(x_out, x, sizeof(double) * (size_t)(T + 1) * n);
    orc_discretise(n, dt, F, c, Q, 0, A, b, C);
    if (inv(n, C, Ci) || inv(m, R, Ri)) { rc = ORC_ERR_SINGULAR; goto done; }
    memset(grad, 0, sizeof(double) * (nn + 2));
    if (!dLdx) {
        /* envelope: partial derivatives of M at x* */
        for (int k = 0; k < T; ++k) {
            const double *xk = x + (size_t)k * n, *x1 = x + (size_t)(k + 1) * n;
            for (int i = 0; i < n; ++i) {
                double s = xk[i] - b[i];
                for (int j = 0; j < n; ++j) s -= A[i * n + j] * x1[j];
                rk[i] = s;
            }
            mv(n, n, Ci, rk, Cr);
            double quad = 0.0;
            for (int i = 0; i < n; ++i) quad += rk[i] * Cr[i];
            for (int a = 0; a < n; ++a)
                for (int bb = 0; bb < n; ++bb) grad[a * n + bb] += dt * Cr[a] * x1[bb];
            grad[nn] += -0.5 * quad;
            for (int i = 0; i < m; ++i) {
                double s = y[(size_t)k * m + i] - r[i];
                for (int j = 0; j < n; ++j) s -= H[i * n + j] * x1[j];
                e[i] = s;
            }
            mv(m, m, Ri, e, w);
            double mq = 0.0;
            for (int i = 0; i < m; ++i) mq += e[i] * w[i];
            grad[nn + 1] += -0.5 * dt * mq;
        }
        for (int a = 0; a < n; ++a) grad[a * n + a] += 0.5 * dt * T;   /* divergence tr F */
        if (logdet) { grad[nn] += 0.5 * n * T; grad[nn + 1] += 0.5 * m * T; }
        goto done;
    }
    {
        /* adjoint solve: same Hessian, linear term dL/dx */
        double *Phi = (double *)malloc(sizeof(double) * nn), *beta = (double *)calloc(n, sizeof(double));
        double *Sig = (double *)malloc(sizeof(double) * nn), *bz = (double *)calloc(n, sizeof(double));
        double *J = (double *)malloc(sizeof(double) * nn), *HtRi = (double *)malloc(sizeof(double) * n * m);
        double *lm0 = (double *)malloc(sizeof(double) * n);
        orc_forward_model(n, A, bz, C, Phi, beta, Sig);
        mTm(n, m, m, H, Ri, HtRi);
        mm(n, m, n, HtRi, H, J);
        for (size_t i = 0; i < nn; ++i) J[i] *= dt;
        mv(n, n, P0, dLdx, lm0);                       /* prior mean P0 d_0 */
        rc = orc_kf_rts(n, T, Phi, 0, beta, 0, Sig, 0, J, 0, dLdx + n, n, lm0, P0, lam, NULL, NULL);
        free(Phi); free(beta); free(Sig); free(bz); free(J); free(HtRi); free(lm0);
        if (rc) goto done;
    }
    for (int k = 0; k < T; ++k) {
        const double *xk = x + (size_t)k * n, *x1 = x + (size_t)(k + 1) * n;
        const double *lk = lam + (size_t)k * n, *l1 = lam + (size_t)(k + 1) * n;
        for (int i = 0; i < n; ++i) {
            double s = xk[i] - b[i], t = lk[i];
            for (int j = 0; j < n; ++j) { s -= A[i * n + j] * x1[j]; t -= A[i * n + j] * l1[j]; }
            rk[i] = s; sk[i] = t;
        }
        mv(n, n, Ci, rk, Cr);
        mv(n, n, Ci, sk, Cs);
        double sq = 0.0;
        for (int i = 0; i < n; ++i) sq += sk[i] * Cr[i];
        /* d/dF of s^T C^-1 r: dt [(C^-1 r) lambda_{k+1}^T + (C^-1 s) x_{k+1}^T] */
        for (int a = 0; a < n; ++a)
            for (int bb = 0; bb < n; ++bb)
                grad[a * n + bb] -= dt * (Cr[a] * l1[bb] + Cs[a] * x1[bb]);
        grad[nn] += sq;                                  /* -d/dlogq (-s^T C^-1 r) */
        for (int i = 0; i < m; ++i) {
            double s = r[i] - y[(size_t)k * m + i], t = 0.0;
            for (int j = 0; j < n; ++j) { s += H[i * n + j] * x1[j]; t += H[i * n + j] * l1[j]; }
            e[i] = s; hl[i] = t;
        }
        mv(m, m, Ri, e, w);
        double mq = 0.0;
        for (int i = 0; i < m; ++i) mq += hl[i] * w[i];
        grad[nn + 1] += dt * mq;
    }
done:
    free(Q); free(R); free(x); free(lam); free(A); free(b); free(C); free(Ci); free(Ri);
    free(rk); free(sk); free(Cr); free(Cs); free(e); free(w); free(hl);
    return rc;
}

/* ------------------------------------------------------------------ */
/* block elements, exact elements, dense output (Section 5.1, Eq. 37)  */
/* ------------------------------------------------------------------ */

/*
 * Block elements (Section 5.1: T blocks of nsub substeps each, the backward
 * conditional ODEs of Eq. 37 integrated by explicit Euler inside a block).
 * Substep j of block k spans [t_k + j h, t_k + (j+1) h], h = dt / nsub; its
 * element is one Euler step of Eq. 37 from the boundary values:
 *   A = I - h F, b = -h c, C = h Q, J = h H^T R^-1 H, eta = h H^T R^-1 (y - r),
 * with the block's sample y = y_{k+1} held over the block (Eq. 37 has a
 * continuous measurement; the data are one sample per block).  The block
 * element is the combination (Eq. 36) of its substeps, the later substep on
 * the left.  elems: (T, 3n^2 + 2n).
 */
int orc_block_elements(int n, int m, int T, int nsub, double dt, const double *F, const double *c,
                       const double *Q, const double *H, const double *r, const double *R,
                       const double *y, double *elems)
{
    if (nsub < 1) return ORC_ERR_ARG;
    size_t nn = (size_t)n * n, es = 3 * nn + 2 * (size_t)n;
    const double h = dt / nsub;
    double *A = (double *)malloc(sizeof(double) * nn), *b = (double *)malloc(sizeof(double) * n);
    double *C = (double *)malloc(sizeof(double) * nn);
    double *e = (double *)malloc(sizeof(double) * es), *acc = (double *)malloc(sizeof(double) * es);
    double *tmp = (double *)malloc(sizeof(double) * es);
    int rc = orc_discretise(n, h, F, c, Q, 0, A, b, C);
    for (int k = 0; k < T && !rc; ++k) {
        rc = orc_elements_lti(n, m, 1, h, A, b, C, H, r, R, y + (size_t)k * m, e);
        memcpy(acc, e, sizeof(double) * es);
        for (int j = 1; j < nsub && !rc; ++j) {
            rc = orc_combine(n, e, acc, tmp);
            memcpy(acc, tmp, sizeof(double) * es);
        }
        memcpy(elems + (size_t)k * es, acc, sizeof(double) * es);
    }
    free(A); free(b); free(C); free(e); free(acc); free(tmp);
    return rc;
}

/*
 * Exact elements: all five rows of Eq. 37 solved over [t_k, t_{k+1}] with
 * constant coefficients and y = y_{k+1} held.  The element is the conditional
 * minimum of the interval's cost; with the costate p of that minimisation the
 * reversed-time state and costate obey the linear Hamiltonian system
 *   d/ds [x; p; 1] = Z [x; p; 1],
 *   Z = [[Ft, -Q, ct], [-H^T R^-1 H, -Ft^T, H^T R^-1 (y - r)], [0, 0, 0]],
 * Ft = -F, ct = -c (time reversal, Section 2.2), and the element's gradients
 * are dV/dz = -p(dt) = C^-1 (z - A phi - b) and dV/dphi = p(0) = J phi - eta
 * - A^T C^-1 (z - A phi - b).  With Psi = e^{Z dt} in blocks (x, p, 1) this
 * gives
 *   C = -Psi12 Psi22^-1,  A = Psi11 + C Psi21,  J = -Psi22^-1 Psi21,
 *   b = psi1 + C psi2,    eta = Psi22^-1 psi2.
 * elems: (T, 3n^2 + 2n).
 */
int orc_exact_elements(int n, int m, int T, double dt, const double *F, const double *c,
                       const double *Q, const double *H, const double *r, const double *R,
                       const double *y, double *elems)
{
    size_t nn = (size_t)n * n, es = 3 * nn + 2 * (size_t)n;
    const int d = 2 * n + 1;
    double *Z = (double *)calloc((size_t)d * d, sizeof(double)), *E = (double *)malloc(sizeof(double) * d * d);
    double *Ri = (double *)malloc(sizeof(double) * m * m), *HtRi = (double *)malloc(sizeof(double) * n * m);
    double *W = (double *)malloc(sizeof(double) * nn), *u = (double *)malloc(sizeof(double) * m);
    double *q = (double *)malloc(sizeof(double) * n);
    double *P11 = (double *)malloc(sizeof(double) * nn), *P12 = (double *)malloc(sizeof(double) * nn);
    double *P21 = (double *)malloc(sizeof(double) * nn), *P22 = (double *)malloc(sizeof(double) * nn);
    double *P22i = (double *)malloc(sizeof(double) * nn), *t1 = (double *)malloc(sizeof(double) * nn);
    double *p1 = (double *)malloc(sizeof(double) * n), *p2 = (double *)malloc(sizeof(double) * n);
    int rc = ORC_OK;
    if (inv(m, R, Ri)) { rc = ORC_ERR_SINGULAR; goto done; }
    mTm(n, m, m, H, Ri, HtRi);
    mm(n, m, n, HtRi, H, W);
    for (int k = 0; k < T; ++k) {
        for (int i = 0; i < m; ++i) u[i] = y[(size_t)k * m + i] - r[i];
        mv(n, m, HtRi, u, q);
        for (int i = 0; i < d * d; ++i) Z[i] = 0.0;
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) {
                Z[i * d + j] = -F[i * n + j] * dt;                 /* Ft */
                Z[i * d + n + j] = -Q[i * n + j] * dt;             /* -Q */
                Z[(n + i) * d + j] = -W[i * n + j] * dt;           /* -H^T R^-1 H */
                Z[(n + i) * d + n + j] = F[j * n + i] * dt;        /* -Ft^T */
            }
            Z[i * d + 2 * n] = -c[i] * dt;                         /* ct */
            Z[(n + i) * d + 2 * n] = q[i] * dt;                    /* H^T R^-1 (y - r) */
        }
        expm(d, Z, E);
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) {
                P11[i * n + j] = E[i * d + j];
                P12[i * n + j] = E[i * d + n + j];
                P21[i * n + j] = E[(n + i) * d + j];
                P22[i * n + j] = E[(n + i) * d + n + j];
            }
            p1[i] = E[i * d + 2 * n];
            p2[i] = E[(n + i) * d + 2 * n];
        }
        if (inv(n, P22, P22i)) { rc = ORC_ERR_SINGULAR; goto done; }
        double *e = elems + (size_t)k * es;
        mm(n, n, n, P12, P22i, t1);
        for (size_t i = 0; i < nn; ++i) E_C(e, n)[i] = -t1[i];             /* C */
        symmetrise(n, E_C(e, n));
        mm(n, n, n, E_C(e, n), P21, t1);
        for (size_t i = 0; i < nn; ++i) E_A(e, n)[i] = P11[i] + t1[i];      /* A */
        mm(n, n, n, P22i, P21, t1);
        for (size_t i = 0; i < nn; ++i) E_J(e, n)[i] = -t1[i];              /* J */
        symmetrise(n, E_J(e, n));
        mv(n, n, E_C(e, n), p2, E_B(e, n));
        for (int i = 0; i < n; ++i) E_B(e, n)[i] += p1[i];                   /* b */
        mv(n, n, P22i, p2, E_ETA(e, n));                                     /* eta */
    }
done:
    free(Z); free(E); free(Ri); free(HtRi); free(W); free(u); free(q);
    free(P11); free(P12); free(P21); free(P22); free(P22i); free(t1); free(p1); free(p2);
    return rc;
}

/*
 * MAP trajectory for arbitrary per-step elements (original-time order,
 * element k on [t_k, t_{k+1}]): the forward model of every element
 * (orc_forward_model) and the Kalman filter + RTS smoother (orc_kf_rts) with
 * the element's (J_k, eta_k) as the information term on x_{k+1}.
 */
int orc_smooth_elements(int n, int T, const double *elems, const double *m0, const double *P0,
                        double *x, double *mf, double *Pf)
{
    size_t nn = (size_t)n * n, es = 3 * nn + 2 * (size_t)n;
    double *Phi = (double *)malloc(sizeof(double) * (size_t)T * nn);
    double *beta = (double *)malloc(sizeof(double) * (size_t)T * n);
    double *Sig = (double *)malloc(sizeof(double) * (size_t)T * nn);
    double *J = (double *)malloc(sizeof(double) * (size_t)T * nn);
    double *eta = (double *)malloc(sizeof(double) * (size_t)T * n);
    int rc = ORC_OK;
    for (int k = 0; k < T && !rc; ++k) {
        const double *e = elems + (size_t)k * es;
        rc = orc_forward_model(n, E_A(e, n), E_B(e, n), E_C(e, n), Phi + (size_t)k * nn, beta + (size_t)k * n,
                               Sig + (size_t)k * nn);
        memcpy(J + (size_t)k * nn, E_J(e, n), sizeof(double) * nn);
        memcpy(eta + (size_t)k * n, E_ETA(e, n), sizeof(double) * n);
    }
    if (!rc) rc = orc_kf_rts(n, T, Phi, nn, beta, n, Sig, nn, J, nn, eta, n, m0, P0, x, mf, Pf);
    free(Phi); free(beta); free(Sig); free(J); free(eta);
    return rc;
}

/*
 * Dense output of a block solve (Section 4.3, recovery of x*(tau) between
 * grid points): inside block k the filter value function at x_k (S = Pf_k^-1,
 * v = S mf_k) is carried across the substeps by the one-variable combine
 * (Eq. 36) with the substep elements, each substep's closed-loop map
 * E = (I + C S)^-1 A, g = (I + C S)^-1 (b + C v) (Eq. 40-41) is kept, and the
 * block's smoothed end state x_{k+1} is taken back through the maps.
 * xd: (nsub T + 1, n), row k nsub + j the state at t_k + j h.
 */
int orc_dense_block(int n, int m, int T, int nsub, double dt, const double *F, const double *c,
                    const double *Q, const double *H, const double *r, const double *R,
                    const double *y, const double *x, const double *mf, const double *Pf, double *xd)
{
    size_t nn = (size_t)n * n, es = 3 * nn + 2 * (size_t)n;
    const double h = dt / nsub;
    double *A = (double *)malloc(sizeof(double) * nn), *b = (double *)malloc(sizeof(double) * n);
    double *C = (double *)malloc(sizeof(double) * nn), *e = (double *)malloc(sizeof(double) * es);
    double *S = (double *)malloc(sizeof(double) * nn), *v = (double *)malloc(sizeof(double) * n);
    double *M = (double *)malloc(sizeof(double) * nn), *Mi = (double *)malloc(sizeof(double) * nn);
    double *Em = (double *)malloc(sizeof(double) * (size_t)nsub * nn), *gm = (double *)malloc(sizeof(double) * (size_t)nsub * n);
    double *t1 = (double *)malloc(sizeof(double) * nn), *t2 = (double *)malloc(sizeof(double) * nn);
    double *u = (double *)malloc(sizeof(double) * n), *w = (double *)malloc(sizeof(double) * n);
    int rc = orc_discretise(n, h, F, c, Q, 0, A, b, C);
    for (int k = 0; k < T && !rc; ++k) {
        rc = orc_elements_lti(n, m, 1, h, A, b, C, H, r, R, y + (size_t)k * m, e);
        if (rc || inv(n, Pf + (size_t)k * nn, S)) { rc = rc ? rc : ORC_ERR_SINGULAR; break; }
        mv(n, n, S, mf + (size_t)k * n, v);
        for (int j = 0; j < nsub && !rc; ++j) {
            mm(n, n, n, C, S, M);                                /* I + C S */
            for (int i = 0; i < n; ++i) M[i * n + i] += 1.0;
            if (inv(n, M, Mi)) { rc = ORC_ERR_SINGULAR; break; }
            mm(n, n, n, Mi, A, Em + (size_t)j * nn);             /* E */
            mv(n, n, C, v, u);
            for (int i = 0; i < n; ++i) u[i] += b[i];
            mv(n, n, Mi, u, gm + (size_t)j * n);                 /* g */
            /* S <- A^T S E + J,  v <- E^T (v - S b) + eta */
            mv(n, n, S, b, u);
            for (int i = 0; i < n; ++i) u[i] = v[i] - u[i];
            mTv(n, n, Em + (size_t)j * nn, u, w);
            for (int i = 0; i < n; ++i) v[i] = w[i] + E_ETA(e, n)[i];
            mm(n, n, n, S, Em + (size_t)j * nn, t1);
            mTm(n, n, n, A, t1, t2);
            for (size_t i = 0; i < nn; ++i) S[i] = t2[i] + E_J(e, n)[i];
            symmetrise(n, S);
        }
        memcpy(u, x + (size_t)(k + 1) * n, sizeof(double) * n);
        for (int j = nsub - 1; j >= 0; --j) {
            mv(n, n, Em + (size_t)j * nn, u, w);
            for (int i = 0; i < n; ++i) u[i] = w[i] + gm[(size_t)j * n + i];
            memcpy(xd + ((size_t)k * nsub + j) * n, u, sizeof(double) * n);
        }
    }
    if (!rc) memcpy(xd + (size_t)T * nsub * n, x + (size_t)T * n, sizeof(double) * n);
    free(A); free(b); free(C); free(e); free(S); free(v); free(M); free(Mi); free(Em); free(gm);
    free(t1); free(t2); free(u); free(w);
    return rc;
}
