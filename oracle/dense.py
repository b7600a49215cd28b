"""Brute-force dense MAP solve: the discrete cost minimised as one least-squares problem.

Test infrastructure (see the oracle package docstring).  For small T this
stacks, term by term, the whitened residuals of

  M(x) = 1/2 |x_0 - m0|^2_{P0^-1}
       + sum_k 1/2 |x_k - A_k x_{k+1} - b_k|^2_{C_k^-1}
       + sum_k 1/2 dt |y_{k+1} - H x_{k+1} - r|^2_{R^-1}

over the whole trajectory (x_0, ..., x_T) and minimises their sum of squares
with numpy.linalg.lstsq.  Singular C_k (a process noise of lower rank than the
state, as in every model of Section 5) is handled exactly: the directions in
C_k's null space become equality constraints N_k^T (x_k - A_k x_{k+1} - b_k) = 0,
eliminated by the null-space method; the range directions are weighted by the
pseudo-inverse.  This is the definition of the argmin written out, with no
recursion, filter or combine.
"""
from __future__ import annotations

import numpy as np


def _inv_sqrt_psd(S, tol):
    w, V = np.linalg.eigh(0.5 * (S + S.T))
    big = w > tol * max(1.0, np.max(np.abs(w)))
    return V, w, big


def dense_map(elems_A, elems_b, elems_C, meas_G, meas_g, m0, P0, rank_tol=1e-12):
    """Minimise the stacked least-squares form of the MAP cost.

    elems_A, elems_b, elems_C: (T, n, n), (T, n), (T, n, n) interval elements.
    meas_G, meas_g: (T, p, n), (T, p): whitened measurement residual
    G_k x_{k+1} - g_k on x_{k+1}.
    Returns x (T+1, n).
    """
    A = np.asarray(elems_A, float)
    T, n, _ = A.shape
    N = (T + 1) * n
    rows, rhs, crow, crhs = [], [], [], []
    w, V = np.linalg.eigh(np.asarray(P0, float))
    Pm = V @ np.diag(w ** -0.5) @ V.T
    r0 = np.zeros((n, N)); r0[:, :n] = Pm
    rows.append(r0); rhs.append(Pm @ np.asarray(m0, float))
    for k in range(T):
        D = np.zeros((n, N))
        D[:, k * n:(k + 1) * n] = np.eye(n)
        D[:, (k + 1) * n:(k + 2) * n] = -A[k]
        V, w, big = _inv_sqrt_psd(np.asarray(elems_C[k], float), rank_tol)
        if np.any(big):
            Wh = np.diag(w[big] ** -0.5) @ V[:, big].T
            rows.append(Wh @ D); rhs.append(Wh @ elems_b[k])
        if np.any(~big):
            Vn = V[:, ~big]
            crow.append(Vn.T @ D); crhs.append(Vn.T @ elems_b[k])
        G = np.zeros((meas_G[k].shape[0], N))
        G[:, (k + 1) * n:(k + 2) * n] = meas_G[k]
        rows.append(G); rhs.append(meas_g[k])
    Rm = np.concatenate(rows, axis=0)
    rv = np.concatenate(rhs)
    if crow:
        Gc = np.concatenate(crow, axis=0)
        hc = np.concatenate(crhs)
        xp = np.linalg.lstsq(Gc, hc, rcond=None)[0]
        _, s, Vt = np.linalg.svd(Gc)
        rank = int(np.sum(s > 1e-12 * s[0]))
        Z = Vt[rank:].T
        z = np.linalg.lstsq(Rm @ Z, rv - Rm @ xp, rcond=None)[0]
        x = xp + Z @ z
    else:
        x = np.linalg.lstsq(Rm, rv, rcond=None)[0]
    return x.reshape(T + 1, n)


def dense_map_lti(model, y, dt, A, b, C):
    """Dense solve for a linear model with constant element (A, b, C)."""
    y = np.asarray(y, float)
    T = y.shape[0]
    n = model.nx
    w, V = np.linalg.eigh(model.R / dt)
    Rm = V @ np.diag(w ** -0.5) @ V.T
    G = np.broadcast_to(Rm @ model.H, (T, model.ny, n))
    g = (y - model.r) @ Rm.T
    return dense_map(np.broadcast_to(A, (T, n, n)), np.broadcast_to(b, (T, n)),
                     np.broadcast_to(C, (T, n, n)), G, g, model.m0, model.P0)
