"""The identities behind the linear time-invariant fast path, checked in FP64
against the oracle's combine (Eq. 36), on the CPU.

The CUDA path for LTI models never runs these formulas on the host; the tests
pin the derivations its plan-time and per-solve kernels evaluate:

* the K-step fold as a linear function of the observations (its (A, C, J)
  recursion with the per-step maps Tb_i, Te_i, and the observation weights
  Gamma_i formed backward from those maps);
* the composition of the per-step closed-loop maps (Section 3.5, Eq. 40-41)
  of a run of elements equals the closed-loop map of their combined element,
  which lets the tile-end states be sums over a table of tile-map products.
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
