"""The identities behind the linear time-invariant fast path, checked in FP64
against the oracle's combine (Eq. 36), on the CPU.

The CUDA path for LTI models never runs these formulas on the host; the tests
pin the derivations its plan-time and per-solve kernels evaluate:

* the K-step fold as a linear function of the observations (its (A, C, J)
  recursion with the per-step maps Tb_i, Te_i, and the observation weights
  Gamma_i formed backward from those maps);
* the composition of the per-step closed-loop maps (Section 3.5, Eq. 40-41)
  of a run of elements equals the closed-loop map of their combined element,
  which lets the tile-end states be sums over a table of tile-map products;
* the coefficient form of a combine's (b, eta) part (tree levels and thread
  prefixes) and the tile Riccati recursion evaluated by doubling.
"""
import numpy as np
import pytest

import oracle
from paper_2512_13319_gb300 import synth


def lti_elements(n, m, T, seed):
    model = synth.ou_model(n, m, seed=seed)
    _, y = synth.simulate(model, T, 1e-3, seed=seed + 1, substeps=1)
    return oracle.elements_lti(model, y, 1e-3), model


def closed_loop(A, b, C, P, v):
    """z*(phi) = E phi + g for the element (A, b, C) against V(z) = 1/2 z'Pz - v'z."""
    M = np.eye(A.shape[0]) + C @ P
    return np.linalg.solve(M, A), np.linalg.solve(M, b + C @ v)


@pytest.mark.parametrize("n,m,K", [(4, 2, 7), (3, 1, 16), (6, 3, 5)])
def test_fold_is_linear_in_the_observations(n, m, K):
    """Item (1): with the accumulated fold (A, C, J) of steps 0..i-1 and
    Mi = (I + C J_acc)^-1, the step maps Tb_i = A_acc Mi C and
    Te_i = (Mi A)^T give the fold's (b, eta) as offsets + sum_i Gamma_i eta_i,
    Gamma_i = (Rb_i, Re_i) from R_{K-1} = (0, I), R_{i-1} = (Tb_i + Rb_i Te_i,
    Re_i Te_i).  Compared with the fold by the oracle's combine."""
    elems, _ = lti_elements(n, m, K, seed=11 * n + K)
    A, b, C, _, J = oracle.unpack_element(elems[0], n)
    etas = [oracle.unpack_element(e, n)[3] for e in elems]
    # the fold by the combine, later element on the left
    acc = elems[0]
    for i in range(1, K):
        acc = oracle.combine(elems[i], acc, n)
    Af, bf, Cf, ef, Jf = oracle.unpack_element(acc, n)
    # the recursion of the constants, with the eta_i as the data
    Aa, Ca, Ja = A.copy(), C.copy(), J.copy()
    ob, oe = b.copy(), np.zeros(n)
    Tb, Te = [None] * K, [None] * K
    for i in range(1, K):
        Mi = np.linalg.inv(np.eye(n) + C @ Ja)
        T1 = Aa @ Mi
        Tb[i], Te[i] = T1 @ C, (Mi @ A).T
        ob, oe = ob + Tb[i] @ oe + T1 @ b, Te[i] @ (oe - Ja @ b)
        Aa, Ca, Ja = T1 @ A, Tb[i] @ Aa.T + Ca, Te[i] @ Ja @ A + J
    Rb, Re = np.zeros((n, n)), np.eye(n)
    bl, el = ob.copy(), oe.copy()
    for j in range(K - 1, -1, -1):
        bl += Rb @ etas[j]
        el += Re @ etas[j]
        if j:
            Rb, Re = Tb[j] + Rb @ Te[j], Re @ Te[j]
    scale = max(1.0, np.abs(Af).max())
    assert np.abs(Aa - Af).max() <= 1e-12 * scale
    assert np.abs(Ca - Cf).max() <= 1e-12 * max(1.0, np.abs(Cf).max())
    assert np.abs(Ja - Jf).max() <= 1e-12 * max(1.0, np.abs(Jf).max())
    assert np.abs(bl - bf).max() <= 1e-12 * max(1.0, np.abs(bf).max())
    assert np.abs(el - ef).max() <= 1e-11 * max(1.0, np.abs(ef).max())


@pytest.mark.parametrize("n,m,K", [(4, 2, 18), (2, 1, 40), (5, 2, 9)])
def test_composed_closed_loop_maps_are_the_combined_elements_map(n, m, K):
    """Item (5): from the filter value function (P, v) before step k0, the
    per-step closed-loop maps x_k = E_k x_{k+1} + g_k of steps k0..k0+K-1
    compose to x_{k0} = Phi x_{k0+K} + beta, and (Phi, beta) is the
    closed-loop map of the combined element of those steps."""
    k0 = 23
    elems, model = lti_elements(n, m, k0 + K, seed=5 * n + K)
    S, v = oracle.filter_by_combine(elems, model.m0, model.P0)
    P, w = S[k0], v[k0]
    Phi, beta = np.eye(n), np.zeros(n)
    for k in range(k0, k0 + K):
        A, b, C, _, _ = oracle.unpack_element(elems[k], n)
        E, g = closed_loop(A, b, C, P, w)
        beta = beta + Phi @ g
        Phi = Phi @ E
        P, w = S[k + 1], v[k + 1]
    acc = elems[k0]
    for k in range(k0 + 1, k0 + K):
        acc = oracle.combine(elems[k], acc, n)
    Af, bf, Cf, _, _ = oracle.unpack_element(acc, n)
    Phi2, beta2 = closed_loop(Af, bf, Cf, S[k0], v[k0])
    assert np.abs(Phi - Phi2).max() <= 1e-10 * max(1.0, np.abs(Phi).max())
    assert np.abs(beta - beta2).max() <= 1e-10 * max(1.0, np.abs(beta).max())


def pair(U, D, n):
    """U (x) D (U the later operand) by the coefficient form of items (2)-(3):
    Mi = (I + C_U J_D)^-1, X = A_D Mi, Y = X C_U, Z = (Mi A_U)^T, W = Z J_D;
    b = X b_U + Y eta_D + b_D, eta = eta_U + Z eta_D - W b_U,
    A = X A_U, C = Y A_D^T + C_D, J = W A_U + J_U."""
    AU, bU, CU, eU, JU = oracle.unpack_element(U, n)
    AD, bD, CD, eD, JD = oracle.unpack_element(D, n)
    Mi = np.linalg.inv(np.eye(n) + CU @ JD)
    X = AD @ Mi
    Y = X @ CU
    Z = (Mi @ AU).T
    W = Z @ JD
    return (X @ AU, X @ bU + Y @ eD + bD, Y @ AD.T + CD, eU + Z @ eD - W @ bU, W @ AU + JU)


@pytest.mark.parametrize("n,m", [(4, 2), (2, 1), (6, 3)])
def test_pair_coefficients_reproduce_the_combine(n, m):
    """Items (2)-(3): the (b, eta) of a combine is a fixed linear map of the
    operands' (b, eta), with coefficients from their (A, C, J) alone; checked
    on folds of different lengths (different constants on each side)."""
    elems, _ = lti_elements(n, m, 12, seed=3 * n)
    U = elems[5]
    for k in range(6, 9):
        U = oracle.combine(elems[k], U, n)          # a fold of 4 steps
    D = elems[0]
    for k in range(1, 5):
        D = oracle.combine(elems[k], D, n)          # a fold of 5 steps
    ref = oracle.unpack_element(oracle.combine(U, D, n), n)
    got = pair(U, D, n)
    for r, g in zip(ref, got):
        assert np.abs(g - r).max() <= 1e-11 * max(1.0, np.abs(r).max())


@pytest.mark.parametrize("n,m", [(4, 2), (3, 1)])
def test_tile_riccati_by_doubling(n, m):
    """Item (4): the P part of the value function before full tile j follows
    P_{j+1} = A_T^T P_j (I + C_T P_j)^-1 A_T + J_T from the prior's P_0; the
    plan computes it for every j at once by applying the doubled tile
    elements (2^e tiles) of the set bits of j, highest first."""
    elems, model = lti_elements(n, m, 6 * 50, seed=7 * n)
    S, _ = oracle.filter_by_combine(elems, model.m0, model.P0)
    tile = elems[0]
    for k in range(1, 6):
        tile = oracle.combine(elems[k], tile, n)    # a tile of 6 steps

    def ric(el, P):
        A, _, C, _, J = oracle.unpack_element(el, n)
        return A.T @ P @ np.linalg.solve(np.eye(n) + C @ P, A) + J

    levels = [tile]
    for _ in range(6):
        levels.append(oracle.combine(levels[-1], levels[-1], n))
    P0 = np.linalg.inv(model.P0)
    P = P0.copy()
    for j in range(1, 50):
        P = ric(tile, P)                            # sequential, j tiles
        assert np.abs(P - S[6 * j]).max() <= 1e-10 * max(1.0, np.abs(P).max())   # the filter's S
        Q = P0.copy()
        for e in range(len(levels) - 1, -1, -1):
            if (j >> e) & 1:
                Q = ric(levels[e], Q)
        assert np.abs(Q - P).max() <= 1e-10 * max(1.0, np.abs(P).max()), j
