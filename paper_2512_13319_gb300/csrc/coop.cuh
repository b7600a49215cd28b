// Sub-warp cooperative versions of the combine (Eq. 36), of its one-variable
// form and of the affine composition (Eq. 40-41), for the tree levels of the
// scans, where few operations are in flight and latency decides.
//
// A group of NL lanes (NL = smallest power of two >= N, at least 2) works on
// one operation; lane r of the group owns row r of every matrix (lanes r >= N
// duplicate row N-1 and never write).  Operands and results are tree nodes in
// shared memory, stored with full matrices row by row, rows padded to P
// scalars so that they can be read with 16-byte loads:
//   element node:  A[N][P] | C[N][P] | J[N][P] | b[P] | eta[P]
//   value node:    S[N][P] | v[P]          (V(x) = 1/2 x^T S x - v^T x)
//   affine node:   F[N][P] | c[P]          (x -> F x + c)
// The (I + C J) inverse is a row-per-lane Gauss-Jordan elimination with the
// pivot rows broadcast by shuffles; the same pivot test and condition
// estimate as the per-thread path decide whether the group recomputes the
// inverse in FP64.  All other cross-row data go through a per-group scratch
// area in shared memory with one __syncwarp.
//
// Every function must be called by all 32 lanes of a warp (groups that have
// no work pass `active = false` and a valid dummy node).
#pragma once
#include "elements.cuh"

namespace mapk {

template <int N, typename S>
struct CoopLayout {
    static constexpr int V = 16 / (int)sizeof(S);
    static constexpr int P = (N + V - 1) / V * V;
    static constexpr int NL = N <= 2 ? 2 : N <= 4 ? 4 : 8;
    // element node
    static constexpr int oA = 0, oC = N * P, oJ = 2 * N * P, ob = 3 * N * P, oeta = 3 * N * P + P;
    static constexpr int NE = 3 * N * P + 2 * P;
    // value node
    static constexpr int oS = 0, ov = N * P;
    static constexpr int NR = N * P + P;
    // affine node
    static constexpr int oF = 0, oc = N * P;
    static constexpr int NA = N * P + P;
    // group scratch: T3, D, T4 (N x P each) and z (P)
    static constexpr int sT3 = 0, sD = N * P, sT4 = 2 * N * P, sz = 3 * N * P;
    static constexpr int NSCR = 3 * N * P + P;
};

// One padded row (P scalars, 16-byte aligned: every node, scratch and level
// block keeps rows at multiples of P from a 16-byte aligned base) with 16-byte
// shared-memory loads; the first N scalars go to out.
template <int N, typename S>
__device__ __forceinline__ void padded_row_load(const S* __restrict__ row, S* out)
{
    constexpr int P = CoopLayout<N, S>::P;
    if constexpr (sizeof(S) == 4) {
#pragma unroll
        for (int j = 0; j < P; j += 4) {
            const float4 v = *reinterpret_cast<const float4*>(row + j);
            if (j < N) out[j] = v.x;
            if (j + 1 < N) out[j + 1] = v.y;
            if (j + 2 < N) out[j + 2] = v.z;
            if (j + 3 < N) out[j + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < P; j += 2) {
            const double2 v = *reinterpret_cast<const double2*>(row + j);
            if (j < N) out[j] = v.x;
            if (j + 1 < N) out[j + 1] = v.y;
        }
    }
}

template <int N, typename S>
__device__ __forceinline__ void row_load(const S* __restrict__ m, int r, S* out)
{
    constexpr int P = CoopLayout<N, S>::P;
    padded_row_load<N, S>(m + r * P, out);
}

template <int N, typename S>
__device__ __forceinline__ void mat_load(const S* __restrict__ m, S (*out)[N])
{
    constexpr int P = CoopLayout<N, S>::P;
#pragma unroll
    for (int k = 0; k < N; ++k) padded_row_load<N, S>(m + k * P, out[k]);
}

template <int N, typename S>
__device__ __forceinline__ void vec_load(const S* __restrict__ m, S* out)
{
#pragma unroll
    for (int q = 0; q < N; ++q) out[q] = m[q];
}

template <int NL, typename S>
__device__ __forceinline__ S group_max(S v)
{
#pragma unroll
    for (int o = NL / 2; o > 0; o >>= 1) {
        S w = __shfl_xor_sync(0xffffffffu, v, o, NL);
        v = w > v ? w : v;
    }
    return v;
}

// ---------------------------------------------------------------------------
// thread struct <-> node
// ---------------------------------------------------------------------------
template <int N, typename S>
__device__ __forceinline__ void node_store(const Elem<N, S>& e, S* __restrict__ nd)
{
    using L = CoopLayout<N, S>;
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            nd[L::oA + i * L::P + j] = e.A[i * N + j];
            nd[L::oC + i * L::P + j] = e.C[Sym<N>::at(i, j)];
            nd[L::oJ + i * L::P + j] = e.J[Sym<N>::at(i, j)];
        }
        nd[L::ob + i] = e.b[i];
        nd[L::oeta + i] = e.eta[i];
    }
}

template <int N, typename S>
__device__ __forceinline__ void node_load(const S* __restrict__ nd, Elem<N, S>& e)
{
    using L = CoopLayout<N, S>;
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) e.A[i * N + j] = nd[L::oA + i * L::P + j];
#pragma unroll
        for (int j = i; j < N; ++j) {
            e.C[Sym<N>::at(i, j)] = nd[L::oC + i * L::P + j];
            e.J[Sym<N>::at(i, j)] = nd[L::oJ + i * L::P + j];
        }
        e.b[i] = nd[L::ob + i];
        e.eta[i] = nd[L::oeta + i];
    }
}

template <int N, typename S>
__device__ __forceinline__ void node_store(const Red<N, S>& r, S* __restrict__ nd)
{
    using L = CoopLayout<N, S>;
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) nd[L::oS + i * L::P + j] = r.P[Sym<N>::at(i, j)];
        nd[L::ov + i] = r.v[i];
    }
}

template <int N, typename S>
__device__ __forceinline__ void node_load(const S* __restrict__ nd, Red<N, S>& r)
{
    using L = CoopLayout<N, S>;
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = i; j < N; ++j) r.P[Sym<N>::at(i, j)] = nd[L::oS + i * L::P + j];
        r.v[i] = nd[L::ov + i];
    }
}

template <int N, typename S>
__device__ __forceinline__ void node_store(const Aff<N, S>& a, S* __restrict__ nd)
{
    using L = CoopLayout<N, S>;
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) nd[L::oF + i * L::P + j] = a.F[i * N + j];
        nd[L::oc + i] = a.c[i];
    }
}

template <int N, typename S>
__device__ __forceinline__ void node_load(const S* __restrict__ nd, Aff<N, S>& a)
{
    using L = CoopLayout<N, S>;
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) a.F[i * N + j] = nd[L::oF + i * L::P + j];
        a.c[i] = nd[L::oc + i];
    }
}

// ---------------------------------------------------------------------------
// row-per-lane inverse of M = I + C X (C from node Cn, X from node Xn, both
// N x P full matrices in shared memory); returns this lane's row of M^-1
// ---------------------------------------------------------------------------
template <int N, typename S>
__device__ __forceinline__ void coop_inverse(const S* __restrict__ Cm, const S* __restrict__ Xm,
                                             int rr, int r, bool active, S* scr, S* mi,
                                             const CombineCtx& ctx)
{
    using L = CoopLayout<N, S>;
    constexpr int NL = L::NL;
    S c[N], X[N][N], x[N], y[N];
    row_load<N, S>(Cm, rr, c);
    mat_load<N, S>(Xm, X);
#pragma unroll
    for (int q = 0; q < N; ++q) {
        S s = (rr == q) ? S(1) : S(0);
#pragma unroll
        for (int k = 0; k < N; ++k) s = fma(c[k], X[k][q], s);
        x[q] = s;
        y[q] = (rr == q) ? S(1) : S(0);
    }
    S ra = S(0);
#pragma unroll
    for (int q = 0; q < N; ++q) ra += ms::sabs(x[q]);
    const S nM = group_max<NL, S>(ra);
    bool ok = true;
#pragma unroll
    for (int cc = 0; cc < N; ++cc) {
        S px[N], py[N];
#pragma unroll
        for (int q = 0; q < N; ++q) {
            px[q] = __shfl_sync(0xffffffffu, x[q], cc, NL);
            py[q] = __shfl_sync(0xffffffffu, y[q], cc, NL);
        }
        const S below = group_max<NL, S>(rr > cc ? ms::sabs(x[cc]) : S(0));
        const S p = px[cc];
        ok = ok && (ms::sabs(p) > S(0.5) * below) && (p != S(0));
        const S ip = ms::pivot_rcp(p);
        if (rr == cc) {
#pragma unroll
            for (int q = 0; q < N; ++q) { x[q] = px[q] * ip; y[q] = py[q] * ip; }
        } else {
            const S f = x[cc] * ip;
#pragma unroll
            for (int q = 0; q < N; ++q) { x[q] = fma(-f, px[q], x[q]); y[q] = fma(-f, py[q], y[q]); }
        }
    }
    S rb = S(0);
#pragma unroll
    for (int q = 0; q < N; ++q) rb += ms::sabs(y[q]);
    const S nMi = group_max<NL, S>(rb);
    ok = (ok && (float(nM) * float(nMi) <= ctx.cond_max)) || !active;
#pragma unroll
    for (int q = 0; q < N; ++q) mi[q] = y[q];
    if (__any_sync(0xffffffffu, !ok)) {
        constexpr int NS = Sym<N>::SZ;
        if (!ok && r == 0) {
            S buf[2 * NS], out[N * N];
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
                for (int j = i; j < N; ++j) {
                    buf[Sym<N>::at(i, j)] = Cm[i * L::P + j];
                    buf[NS + Sym<N>::at(i, j)] = Xm[i * L::P + j];
                }
            inverse_I_plus_fp64<N, S>(buf, out, ctx.stats, ctx.cond_max);
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
                for (int j = 0; j < N; ++j) scr[i * L::P + j] = out[i * N + j];
        }
        __syncwarp();
        if (!ok) row_load<N, S>(scr, rr, mi);
        __syncwarp();
    }
}

// On = Ln (x) Rn  (Ln: later interval, the left operand of Eq. 36)
template <int N, typename S>
__device__ __forceinline__ void coop_combine(const S* __restrict__ Ln, const S* __restrict__ Rn,
                                             S* __restrict__ On, S* __restrict__ scr, bool active,
                                             const CombineCtx& ctx)
{
    using L = CoopLayout<N, S>;
    constexpr int NL = L::NL, P = L::P;
    const int r = threadIdx.x & (NL - 1);
    const int rr = r < N ? r : N - 1;
    const bool wr = active && r < N;
    S mi[N];
    coop_inverse<N, S>(Ln + L::oC, Rn + L::oJ, rr, r, active, scr + L::sT3, mi, ctx);
    S AL[N][N], CL[N][N], JR[N][N], aR[N], bL[N], etaR[N];
    mat_load<N, S>(Ln + L::oA, AL);
    mat_load<N, S>(Ln + L::oC, CL);
    mat_load<N, S>(Rn + L::oJ, JR);
    row_load<N, S>(Rn + L::oA, rr, aR);
    vec_load<N, S>(Ln + L::ob, bL);
    vec_load<N, S>(Rn + L::oeta, etaR);
    // own rows of T3 = M^-1 A_L, D = M^-1 C_L, T4 = J_R A_L and z_rr of z = M^-1 b_L + D eta_R
    S t3[N], d[N], t4[N];
    S zr = S(0);
#pragma unroll
    for (int q = 0; q < N; ++q) {
        S s3 = S(0), sd = S(0), s4 = S(0);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            s3 = fma(mi[k], AL[k][q], s3);
            sd = fma(mi[k], CL[k][q], sd);
            s4 = fma(JR[rr][k], AL[k][q], s4);
        }
        t3[q] = s3; d[q] = sd; t4[q] = s4;
        zr = fma(mi[q], bL[q], zr);
    }
#pragma unroll
    for (int q = 0; q < N; ++q) zr = fma(d[q], etaR[q], zr);
    __syncwarp();
    if (r < N) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            scr[L::sT3 + rr * P + q] = t3[q];
            scr[L::sD + rr * P + q] = d[q];
            scr[L::sT4 + rr * P + q] = t4[q];
        }
        scr[L::sz + rr] = zr;
    }
    __syncwarp();
    S T3[N][N], D[N][N], T4[N][N], z[N], AR[N][N];
    mat_load<N, S>(scr + L::sT3, T3);
    mat_load<N, S>(scr + L::sD, D);
    mat_load<N, S>(scr + L::sT4, T4);
    vec_load<N, S>(scr + L::sz, z);
    mat_load<N, S>(Rn + L::oA, AR);
    S oa[N], oc[N], oj[N], u[N];
    S ob = Rn[L::ob + rr], oe = Ln[L::oeta + rr];
    // w = eta_R - J_R b_L (whole vector, every lane)
    S w[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        S s = etaR[k];
#pragma unroll
        for (int q = 0; q < N; ++q) s = fma(-JR[k][q], bL[q], s);
        w[k] = s;
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
        S sa = S(0), su = S(0), sj = Ln[L::oJ + rr * P + q];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            sa = fma(aR[k], T3[k][q], sa);          // A_out = A_R T3
            su = fma(aR[k], D[k][q], su);           // U = A_R D
            sj = fma(T3[k][rr], T4[k][q], sj);      // J_out = T3^T T4 + J_L
        }
        oa[q] = sa; u[q] = su; oj[q] = sj;
        ob = fma(aR[q], z[q], ob);                  // b_out = A_R z + b_R
        oe = fma(T3[q][rr], w[q], oe);              // eta_out = T3^T w + eta_L
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
        S s = Rn[L::oC + rr * P + q];
#pragma unroll
        for (int k = 0; k < N; ++k) s = fma(u[k], AR[q][k], s);   // C_out = U A_R^T + C_R
        oc[q] = s;
    }
    __syncwarp();
    if (wr) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            On[L::oA + rr * P + q] = oa[q];
            On[L::oC + rr * P + q] = oc[q];
            On[L::oJ + rr * P + q] = oj[q];
        }
        On[L::ob + rr] = ob;
        On[L::oeta + rr] = oe;
    }
}

// On (value node) = E (x) Pn for the element E whose A, C, J are those of
// node En and whose b, eta are the vectors eb, eeta; On may be Pn
template <int N, typename S>
__device__ __forceinline__ void coop_apply_parts(const S* __restrict__ En, const S* __restrict__ eb,
                                                 const S* __restrict__ eeta, const S* Pn, S* On,
                                                 S* __restrict__ scr, bool active, const CombineCtx& ctx)
{
    using L = CoopLayout<N, S>;
    constexpr int NL = L::NL, P = L::P;
    const int r = threadIdx.x & (NL - 1);
    const int rr = r < N ? r : N - 1;
    const bool wr = active && r < N;
    S mi[N];
    coop_inverse<N, S>(En + L::oC, Pn + L::oS, rr, r, active, scr + L::sT3, mi, ctx);
    S AE[N][N], SP[N][N], bE[N], v[N];
    mat_load<N, S>(En + L::oA, AE);
    mat_load<N, S>(Pn + L::oS, SP);
    vec_load<N, S>(eb, bE);
    vec_load<N, S>(Pn + L::ov, v);
    S e[N], t4[N], w[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
        S se = S(0), s4 = S(0);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            se = fma(mi[k], AE[k][q], se);          // E = M^-1 A
            s4 = fma(SP[rr][k], AE[k][q], s4);      // T4 = S A
        }
        e[q] = se; t4[q] = s4;
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {                   // w = v - S b
        S s = v[k];
#pragma unroll
        for (int q = 0; q < N; ++q) s = fma(-SP[k][q], bE[q], s);
        w[k] = s;
    }
    __syncwarp();
    if (r < N) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            scr[L::sT3 + rr * P + q] = e[q];
            scr[L::sT4 + rr * P + q] = t4[q];
        }
    }
    __syncwarp();
    S Ef[N][N], T4[N][N];
    mat_load<N, S>(scr + L::sT3, Ef);
    mat_load<N, S>(scr + L::sT4, T4);
    S os[N];
    S ov = eeta[rr];
#pragma unroll
    for (int q = 0; q < N; ++q) {
        S s = En[L::oJ + rr * P + q];
#pragma unroll
        for (int k = 0; k < N; ++k) s = fma(Ef[k][rr], T4[k][q], s);   // E^T S A + J
        os[q] = s;
        ov = fma(Ef[q][rr], w[q], ov);                                   // E^T w + eta
    }
    __syncwarp();
    if (wr) {
#pragma unroll
        for (int q = 0; q < N; ++q) On[L::oS + rr * P + q] = os[q];
        On[L::ov + rr] = ov;
    }
}

// On (value node) = En (x) Pn  (En: element node, Pn: value node); On may be Pn
template <int N, typename S>
__device__ __forceinline__ void coop_apply(const S* __restrict__ En, const S* Pn, S* On,
                                           S* __restrict__ scr, bool active, const CombineCtx& ctx)
{
    using L = CoopLayout<N, S>;
    coop_apply_parts<N, S>(En, En + L::ob, En + L::oeta, Pn, On, scr, active, ctx);
}

}  // namespace mapk
