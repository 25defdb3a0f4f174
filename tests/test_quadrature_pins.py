"""Pins of the optimal-quadrature oracle (oracle/quadrature_oracle.py) to facts other than itself.

- The paper's error formula at the optimal weights equals the general quadratic error
  <I^2> - 2 w.c + w^T P w, and the Monte Carlo mean of (I^ - I)^2 over sampled Phi ~ N(0, P).
- All fine nodes: the error vanishes and the optimal weights are the fine weights q.
- The optimum is stationary: moving weight i by d raises the error by exactly d^2 P_ii.
- The greedy objective never rises; its first node is the closed-form best single node.
- A covariance of rank one is integrated exactly by one node.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def problem(L=4, ntot=12, jitter=1e-10):
    cp = W.COV
    return O.fine_problem(L, ntot, jitter, (cp.A, cp.ns, cp.kmin, cp.kmax, cp.nk), W.transfer_kernels)


def test_error_formula_matches_general_form_and_monte_carlo():
    pr = problem(jitter=1e-6)
    P, q = pr["P"][3], pr["q"][0, 3]
    S = [1, 4, 7, 10]
    w = O.optimal_weights(P, q, S)
    e_paper = O.expected_error(P, q, S)
    e_general = O.expected_error(P, q, S, w)
    assert abs(e_paper - e_general) < 1e-10 * O.los_moments(P, q)[0]
    rng = np.random.default_rng(3)
    M = 40000
    Lc = np.linalg.cholesky(P)
    phi = Lc @ rng.standard_normal((P.shape[0], M))
    err2 = (w @ phi[S] - q @ phi) ** 2
    assert abs(err2.mean() - e_paper) < 5 * math.sqrt(2.0 / M) * e_paper


def test_all_fine_nodes_are_exact():
    pr = problem(jitter=1e-6)
    for l in (0, 2, 4):
        P, q = pr["P"][l], pr["q"][0, l]
        S = list(range(P.shape[0]))
        I2 = O.los_moments(P, q)[0]
        assert abs(O.expected_error(P, q, S)) < 1e-10 * I2
        assert np.allclose(O.optimal_weights(P, q, S), q, rtol=1e-8, atol=1e-8 * np.max(np.abs(q)))


def test_optimum_is_stationary():
    pr = problem(jitter=1e-6)
    P, q = pr["P"][2], pr["q"][1, 2]
    S = [0, 5, 9]
    w = O.optimal_weights(P, q, S)
    e0 = O.expected_error(P, q, S, w)
    d = 1e-3 * np.max(np.abs(w))
    for i in range(len(S)):
        wp = w.copy()
        wp[i] += d
        rise = O.expected_error(P, q, S, wp) - e0
        assert abs(rise - d * d * P[S[i], S[i]]) < 1e-6 * d * d * P[S[i], S[i]]


def test_greedy_objective_never_rises_and_first_node_is_closed_form():
    pr = problem(L=3, ntot=16)
    P, q = pr["P"], pr["q"]
    res = O.greedy_nodes(P, q, 5)
    assert np.all(np.diff(res["objective"]) <= 1e-12 * res["objective"][0])
    score = np.zeros(P.shape[1])
    for l in range(P.shape[0]):
        for x in range(2):
            I2, c = O.los_moments(P[l], q[x, l])
            if I2 > 0:
                score += c * c / (np.diag(P[l]) * I2)
    assert res["nodes"][0] == int(np.argmax(score))
    assert len(set(res["nodes"])) == 5


def test_rank_one_covariance_needs_one_node():
    rng = np.random.default_rng(5)
    v = rng.uniform(0.5, 1.5, 10)
    P = np.outer(v, v)[None]
    q = rng.standard_normal((2, 1, 10))
    res = O.greedy_nodes(P, q, 1)
    assert res["objective"][0] < 1e-12
    j = res["nodes"][0]
    assert np.allclose(res["weights"][:, 0, 0], (q[:, 0] @ v) / v[j], rtol=1e-12)
