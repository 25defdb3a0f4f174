"""Plain FP64 CPU oracle of the optimal radial quadrature of Sect. 3 (Elsner & Wandelt).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  It shares no code with the CUDA library.

For one multipole l and field X the line-of-sight integral I = int dr r^2 alpha(r) Phi(r) is
first taken on a fine grid of N_tot shells (I = sum_k q_k Phi(r_k), q_k = u_k alpha(r_k) with the
fine rule's weights u_k r_k^2), then approximated by I^ = sum_{i in S} w_i Phi(r_i) on a subset S
of N nodes.  With the eigenpairs (lambda_k, phi_k) of the fine covariance P_Phi of Phi:

  <(I^ - I)^2> = sum_k lambda_k (int r^2 alpha phi_k)^2 - w^T P_SS w          (at the optimum)
  optimal w:   sum_j P_Phi(r_i, r_j) w_j = sum_k lambda_k phi_k(r_i) int r^2 alpha phi_k,  i in S
  greedy:      grow S one node at a time, each time adding the fine node that leaves the
               smallest summed error.

Readings (the paper keeps (l, m) fixed and sums the T and E errors with equal weights):
  - the greedy objective is sum over l = 0..l_max and X in {T, E} of the error relative to
    <I^2> of that (l, X) (fields with <I^2> = 0 left out), so that every degree counts alike;
    ties go to the smallest fine index;
  - P_Phi is the covariance the generator realises on the fine nodes, C_l + eps_l I with the
    filters' relative jitter (so every conditional variance stays >= eps_l > 0);
  - int dr r^2 alpha phi_k is the fine rule's sum_k u_k alpha(r_k) phi_k(r_k).

Pins (tests/test_quadrature_pins.py, CPU): the error formula against the general quadratic
error and a Monte Carlo mean; S = every fine node gives zero error and w = q; the optimum is
stationary; the objective never rises; a covariance of rank one needs one node; the first
greedy node against its closed form (largest sum c_j^2 / (P_jj <I^2>)).
"""
from __future__ import annotations

import numpy as np



def los_moments(P: np.ndarray, q: np.ndarray) -> tuple[float, np.ndarray]:
    """<I^2> = sum_k lambda_k (q . phi_k)^2 and the right-hand side c_i = sum_k lambda_k phi_k(r_i)
    (q . phi_k) of the normal equations, from the eigen-decomposition of P (one l)."""
    lam, phi = np.linalg.eigh(P)
    a = phi.T @ q                       # int r^2 alpha phi_k on the fine rule
    return float(np.sum(lam * a * a)), phi @ (lam * a)


def optimal_weights(P: np.ndarray, q: np.ndarray, S) -> np.ndarray:
    """w on the nodes S (in the order given): P_SS w = c_S."""
    S = np.asarray(S, dtype=int)
    _, c = los_moments(P, q)
    return np.linalg.solve(P[np.ix_(S, S)], c[S])


def expected_error(P: np.ndarray, q: np.ndarray, S, w=None) -> float:
    """<(I^ - I)^2> at the optimal weights of S (the paper's formula), or for given weights w the
    general quadratic form <I^2> - 2 w . c_S + w^T P_SS w."""
    S = np.asarray(S, dtype=int)
    I2, c = los_moments(P, q)
    if len(S) == 0:
        return I2
    if w is None:
        w = np.linalg.solve(P[np.ix_(S, S)], c[S])
        return I2 - float(w @ P[np.ix_(S, S)] @ w)
    return I2 - 2.0 * float(w @ c[S]) + float(w @ P[np.ix_(S, S)] @ w)


def greedy_nodes(P: np.ndarray, q: np.ndarray, n: int) -> dict:
    """Greedy node selection over all degrees and both fields, following the paper's steps:
    for every candidate j the optimal weights of S + {j} (a fresh solve) and the error formula,
    then the j with the smallest summed relative error.

    P: [L+1, N_tot, N_tot] fine covariances; q: [2, L+1, N_tot] fine line-of-sight weights.
    Returns nodes (selection order), objective after each step, rel_err [2, L+1] at the end,
    weights [2, L+1, n] in selection order and <I^2> [2, L+1]."""
    L1, Nt = P.shape[0], P.shape[1]
    mom = [[los_moments(P[l], q[x, l]) for l in range(L1)] for x in range(2)]
    I2 = np.array([[mom[x][l][0] for l in range(L1)] for x in range(2)])
    S: list[int] = []
    trace = []

    def objective(T):
        tot = 0.0
        for l in range(L1):
            Ptt = P[l][np.ix_(T, T)]
            for x in range(2):
                if I2[x, l] > 0:
                    c = mom[x][l][1][T]
                    w = np.linalg.solve(Ptt, c)
                    tot += (I2[x, l] - float(w @ Ptt @ w)) / I2[x, l]
        return tot

    for _ in range(min(n, Nt)):
        scores = [(objective(S + [j]), j) for j in range(Nt) if j not in S]
        best, best_j = min(scores)
        S.append(best_j)
        trace.append(best)
    rel = np.zeros((2, L1))
    W = np.zeros((2, L1, len(S)))
    for l in range(L1):
        for x in range(2):
            if I2[x, l] > 0:
                rel[x, l] = expected_error(P[l], q[x, l], S) / I2[x, l]
                W[x, l] = optimal_weights(P[l], q[x, l], S)
    return {"nodes": S, "objective": np.array(trace), "rel_err": rel, "weights": W, "I2": I2}


def fine_problem(lmax: int, ntot: int, jitter_rel: float, cov_params, transfer) -> dict:
    """The design problem on the fine midpoint grid of N_tot shells: P_l = C_l + eps_l I (Eq. 7
    covariance on the fine nodes, eps_l = jitter_rel * mean(diag C_l)) and q^X_l = u alpha^X_l
    with u_k = w_k r_k^2.  ``cov_params`` = (A, ns, kmin, kmax, nk); ``transfer(lmax, r)`` gives
    (alpha^T, alpha^E) [L+1, N_tot]."""
    from .fnl_oracle import covariance
    from workloads import radial_grid
    r, w = radial_grid(ntot)
    A, ns, kmin, kmax, nk = cov_params
    C = covariance(lmax, r, A, ns, kmin, kmax, nk)
    eps = jitter_rel * np.einsum("lii->l", C) / ntot
    P = C + eps[:, None, None] * np.eye(ntot)[None]
    aT, aE = transfer(lmax, r)
    u = w * r * r
    q = np.stack([aT * u[None, :], aE * u[None, :]])
    return {"r": r, "w": w, "P": P, "q": q}


__all__ = ["los_moments", "optimal_weights", "expected_error", "greedy_nodes", "fine_problem"]
