"""FP64 NumPy oracle for learning the projections -- TEST INFRASTRUCTURE ONLY.

Plain restatements of Sec. 2.1-2.4 of LeanVec (arXiv 2312.16335):

* second moments K = sum x x^T (uncentred; Sec. 2.2 "Efficiency"),
* LeanVec-ID: the d leading left singular vectors of X, i.e. the d leading
  eigenvectors of K_X, used as A = B (Sec. 2.1, problem "pca"),
* the LeanVec-OOD loss in Frobenius form (problem "leanvec_orthonormal") and in
  trace form over K_Q, K_X (problem "leanvec_efficient"),
* its partial derivatives (Eq. "leanvec_gradients"),
* the linear minimisation oracle over the spectral-norm ball: S = U V^T from the
  SVD of C (Sec. 2.3),
* Frank-Wolfe block coordinate descent (Algorithm 1) with step 1/(t+1)^alpha and
  the relative-change stop rule of Sec. 2.3, optionally the exact quadratic
  line search,
* eigenvector search (Algorithm 2): P(beta) = d leading eigenvectors of
  K_beta = (1-beta)/m K_Q + beta/n K_X, beta chosen by bounded Brent search,
* the pair form of the loss and its gradients over explicit (query, database)
  pairs, r_ij = q_j^T x_i - (A q_j)^T (B x_i), for the differentiation form.

Readings where the paper is silent (each listed in the design notes):
  alpha = 0.5; A0 = B0 = 0 makes the first A-gradient vanish, so an all-zero
  linear-minimisation input returns the LeanVec-ID solution; at most 500
  iterations; eigenvector signs: the largest-magnitude entry of each row is
  positive (first index on ties); Brent tolerance xatol = 1e-5.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use this.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize_scalar


def second_moment(X: np.ndarray) -> np.ndarray:
    """K = X^T X for X stored as rows (n x D): the paper's X X^T with X = D x n."""
    X64 = np.asarray(X, dtype=np.float64)
    return X64.T @ X64


def sign_fix(P: np.ndarray) -> np.ndarray:
    """Make the largest-|.| entry of every row positive (first index on ties)."""
    P = np.array(P, dtype=np.float64, copy=True)
    for i in range(P.shape[0]):
        j = int(np.argmax(np.abs(P[i])))
        if P[i, j] < 0:
            P[i] = -P[i]
    return P


def top_eigvecs(K: np.ndarray, d: int) -> tuple[np.ndarray, np.ndarray]:
    """Rows = the d eigenvectors of symmetric K with the largest eigenvalues
    (descending), plus all eigenvalues in descending order."""
    w, V = np.linalg.eigh(np.asarray(K, dtype=np.float64))
    order = np.argsort(-w, kind="stable")
    return sign_fix(V[:, order[:d]].T), w[order]


def fit_id(K_X: np.ndarray, d: int) -> np.ndarray:
    """LeanVec-ID (Sec. 2.1): M = d leading eigenvectors of K_X, A = B = M."""
    return top_eigvecs(K_X, d)[0]


def ood_loss_frobenius(A, B, Q, X) -> float:
    """|| Q^T A^T B X - Q^T X ||_F^2 with Q (m x D) and X (n x D) stored as rows."""
    Q = np.asarray(Q, np.float64)
    X = np.asarray(X, np.float64)
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    E = (Q @ A.T) @ (B @ X.T) - Q @ X.T
    return float(np.sum(E * E))


def ood_loss(A, B, K_Q, K_X) -> float:
    """tr(A K_Q A^T B K_X B^T) + tr(K_Q K_X) - 2 tr(K_Q A^T B K_X)."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    t1 = np.trace(A @ K_Q @ A.T @ B @ K_X @ B.T)
    t2 = np.trace(K_Q @ K_X)
    t3 = np.trace(K_Q @ A.T @ B @ K_X)
    return float(t1 + t2 - 2.0 * t3)


def ood_grads(A, B, K_Q, K_X) -> tuple[np.ndarray, np.ndarray]:
    """Eq. leanvec_gradients:
       dA = 2 B K_X B^T A K_Q - 2 B K_X K_Q,  dB = 2 A K_Q A^T B K_X - 2 A K_Q K_X."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    gA = 2.0 * B @ K_X @ B.T @ A @ K_Q - 2.0 * B @ K_X @ K_Q
    gB = 2.0 * A @ K_Q @ A.T @ B @ K_X - 2.0 * A @ K_Q @ K_X
    return gA, gB


def lmo(C: np.ndarray) -> np.ndarray:
    """argmax over ||S||_op <= 1 of <S, C>: S = U V^T from the thin SVD of C."""
    U, _, Vt = np.linalg.svd(np.asarray(C, np.float64), full_matrices=False)
    return U @ Vt


def op_norm(A: np.ndarray) -> float:
    return float(np.linalg.norm(np.asarray(A, np.float64), 2))


def _line_search(grad, S, Y, other, K_first, K_second, which: str) -> float:
    """Exact minimiser over gamma in [0, 1] of f(Y + gamma (S - Y)) for the block
    `which`; f is quadratic in one block with the other held fixed."""
    Dl = S - Y
    slope = float(np.sum(grad * Dl))
    if which == "A":
        # f(A) = tr(A K_Q A^T M) + ..., M = B K_X B^T
        M = other @ K_second @ other.T
        curv = float(np.trace(Dl @ K_first @ Dl.T @ M))
    else:
        M = other @ K_first @ other.T
        curv = float(np.trace(M @ Dl @ K_second @ Dl.T))
    if curv <= 0.0:
        return 1.0 if slope < 0 else 0.0
    return float(np.clip(-slope / (2.0 * curv), 0.0, 1.0))


def frank_wolfe(K_Q, K_X, d: int, alpha: float = 0.5, tol: float = 1e-3, max_iter: int = 500,
                A0=None, B0=None, line_search: bool = False) -> dict:
    """Algorithm 1 (Frank-Wolfe BCD): per iteration t, gamma = 1/(t+1)^alpha (or the
    exact line search), one FW step on A with B fixed, then one on B with the new A.
    Stops when |f(t+1) - f(t)| / f(t) <= tol.  Returns A, B, the loss trace and the
    FW gaps g_A, g_B (App. C)."""
    K_Q = np.asarray(K_Q, np.float64)
    K_X = np.asarray(K_X, np.float64)
    D = K_Q.shape[0]
    A = np.zeros((d, D)) if A0 is None else np.array(A0, np.float64)
    B = np.zeros((d, D)) if B0 is None else np.array(B0, np.float64)
    P_id = None
    f_prev = ood_loss(A, B, K_Q, K_X)
    trace = [f_prev]
    gaps = []
    it = 0
    for t in range(max_iter):
        it = t + 1
        gamma = 1.0 / (t + 1) ** alpha
        gA, _ = ood_grads(A, B, K_Q, K_X)
        C = -gA
        if not np.any(C):
            if P_id is None:
                P_id = fit_id(K_X, d)
            S_A = P_id
        else:
            S_A = lmo(C)
        g_a = float(np.sum(C * (S_A - A)))
        ga = _line_search(gA, S_A, A, B, K_Q, K_X, "A") if line_search else gamma
        A = (1.0 - ga) * A + ga * S_A
        _, gB = ood_grads(A, B, K_Q, K_X)
        C = -gB
        if not np.any(C):
            if P_id is None:
                P_id = fit_id(K_X, d)
            S_B = P_id
        else:
            S_B = lmo(C)
        g_b = float(np.sum(C * (S_B - B)))
        gb = _line_search(gB, S_B, B, A, K_Q, K_X, "B") if line_search else gamma
        B = (1.0 - gb) * B + gb * S_B
        f = ood_loss(A, B, K_Q, K_X)
        trace.append(f)
        gaps.append((g_a, g_b))
        stop = abs(f - f_prev) / f_prev <= tol if f_prev > 0 else True
        f_prev = f
        if stop:
            break
    return {"A": A, "B": B, "loss": np.array(trace), "gaps": np.array(gaps), "iterations": it}


def es_projection(K_Q, K_X, m: int, n: int, d: int, beta: float) -> np.ndarray:
    """Algorithm 2's projection(beta): d leading eigenvectors of
    K_beta = (1 - beta)/m K_Q + beta/n K_X."""
    Kb = (1.0 - beta) / m * np.asarray(K_Q, np.float64) + beta / n * np.asarray(K_X, np.float64)
    return top_eigvecs(Kb, d)[0]


def eigsearch(K_Q, K_X, m: int, n: int, d: int, xatol: float = 1e-5) -> dict:
    """Algorithm 2: beta in [0, 1] minimising the loss with A = B = projection(beta),
    found by a bounded derivative-free (Brent) scalar minimisation."""
    def obj(b):
        P = es_projection(K_Q, K_X, m, n, d, b)
        return ood_loss(P, P, K_Q, K_X)
    res = minimize_scalar(obj, bounds=(0.0, 1.0), method="bounded", options={"xatol": xatol})
    beta = float(res.x)
    P = es_projection(K_Q, K_X, m, n, d, beta)
    return {"P": P, "beta": beta, "loss": float(res.fun), "evaluations": int(res.nfev)}


def pair_loss_and_grads(A, B, Q, X) -> tuple[float, np.ndarray, np.ndarray]:
    """Differentiation form: over all pairs (query j, database i)
       r_ij = q_j^T x_i - (A q_j)^T (B x_i),  L = sum r^2 / (n m),
       dL/dA = -2/(nm) sum r_ij (B x_i) q_j^T,  dL/dB = -2/(nm) sum r_ij (A q_j) x_i^T."""
    Q = np.asarray(Q, np.float64)
    X = np.asarray(X, np.float64)
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    m, n = Q.shape[0], X.shape[0]
    Qp = Q @ A.T            # m x d
    Xp = X @ B.T            # n x d
    Rm = Q @ X.T - Qp @ Xp.T  # m x n, entry (j, i) = r_ij
    L = float(np.sum(Rm * Rm)) / (n * m)
    gA = -2.0 / (n * m) * (Rm @ Xp).T @ Q
    gB = -2.0 / (n * m) * (Rm.T @ Qp).T @ X
    return L, gA, gB


def reconstruction_error(P, X) -> float:
    """|| X - P^T P X ||_F^2 (problem pca) with X stored as rows."""
    X = np.asarray(X, np.float64)
    P = np.asarray(P, np.float64)
    E = X - (X @ P.T) @ P
    return float(np.sum(E * E))
