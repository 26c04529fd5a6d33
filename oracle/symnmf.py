"""FP64 oracle for the randomized SymNMF hot path (TEST INFRASTRUCTURE ONLY).

Each function restates one step of the paper in plain numpy/scipy, in the
paper's order and notation.  Sections cited are those of Hayashi, Aksoy,
Ballard, Park, "Randomized Algorithms for Symmetric Nonnegative Matrix
Factorization" (arXiv 2402.08134).

Conventions shared with the CUDA path (the readings of the paper):

* X is m x m symmetric (called n in the code), W and H are n x k, row-major.
* A "sweep" is one W-update followed by one H-update (Alg. LAI-SymNMF and
  Alg. LvS-SymNMF, loop body).  W0 := H0 (the algorithms initialise H only).
* HALS updates all columns of W in order 1..k, each using the columns already
  updated (Eq. symhals_update2), then all columns of H.
* Update(G, Y) receives the Gram G = F^T F *without* alpha I and the product
  Y = X F (n x k, i.e. the transpose of the paper's k x n Y) *without* alpha
  F; the rules add the alpha terms themselves.
"""

from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.linalg as sla
import scipy.optimize as sopt

from . import philox

# ------------------------------------------------------------------ objectives


def surrogate_objective(X, W, H, alpha):
    """||X - W H^T||_F^2 + alpha ||W - H||_F^2 computed directly (Eq. surrogate_symnmf_obj)."""
    R = X - W @ H.T
    return float((R * R).sum() + alpha * ((W - H) ** 2).sum())


def normalized_residual(X, W, H):
    """||X - W H^T||_F / ||X||_F computed directly (Appendix 'Stopping Criteria')."""
    return float(np.linalg.norm(X - W @ H.T) / np.linalg.norm(X))


def symnmf_residual(X, H):
    """||X - H H^T||_F / ||X||_F, the SymNMF objective of Eq. symnmf_obj, normalised."""
    return float(np.linalg.norm(X - H @ H.T) / np.linalg.norm(X))


def trace_trick_residual_sq(normX2, WtW, HtH, WtXH):
    """||X - W H^T||_F^2 = ||X||^2 + tr(W^T W H^T H) - 2 tr(W^T X H) (Appendix 'Fast Residual Evaluation')."""
    return float(normX2 + np.trace(WtW @ HtH) - 2.0 * np.trace(WtXH))


def projected_gradient_norm(X, W, H, alpha):
    """sqrt(||grad^P_W||^2 + ||grad^P_H||^2) of the surrogate (Appendix 'Projected Gradients').

    grad_W = 2 (W H^T H - X H) + 2 alpha (W - H), grad_H = 2 (H W^T W - X W) + 2 alpha (H - W);
    an entry counts when the gradient is negative or the variable is positive.
    """
    gW = 2.0 * (W @ (H.T @ H) - X @ H) + 2.0 * alpha * (W - H)
    gH = 2.0 * (H @ (W.T @ W) - X.T @ W) + 2.0 * alpha * (H - W)
    pW = np.where((gW < 0) | (W > 0), gW, 0.0)
    pH = np.where((gH < 0) | (H > 0), gH, 0.0)
    return float(math.sqrt((pW * pW).sum() + (pH * pH).sum()))


# ------------------------------------------------------------------- HALS rules


def hals_update_efficient(Wold, H, G, Y, alpha):
    """All columns of W by the efficient regularised rule (Eq. symhals_update2).

    w_i <- [ ((X - W H^T + alpha I) h_i) / (||h_i||^2 + alpha)
             + ||h_i||^2 / (||h_i||^2 + alpha) w_i ]_+ ,  i = 1..k in order,
    with (X - W H^T + alpha I) h_i = Y_i - W G_i + alpha h_i, G = H^T H, Y = X H,
    and W holding the columns already updated.
    """
    W = np.array(Wold, dtype=np.float64, copy=True)
    k = W.shape[1]
    for i in range(k):
        hh = G[i, i]
        resid_h = Y[:, i] - W @ G[:, i] + alpha * H[:, i]
        W[:, i] = np.maximum(resid_h / (hh + alpha) + hh / (hh + alpha) * W[:, i], 0.0)
    return W


def hals_update_explicit(X, Wold, H, alpha):
    """All columns of W by the explicit-residual rule (Eq. symhals_update1), O(m^2) per column.

    w_i = max( (R_i + alpha I) h_i / (||h_i||^2 + alpha), 0 ),
    R_i = X - sum_{j != i} w_j h_j^T with the current W.
    """
    W = np.array(Wold, dtype=np.float64, copy=True)
    k = W.shape[1]
    for i in range(k):
        others = [j for j in range(k) if j != i]
        R = X - W[:, others] @ H[:, others].T
        h = H[:, i]
        W[:, i] = np.maximum((R @ h + alpha * h) / (h @ h + alpha), 0.0)
    return W


def hals_update_standard(Wold, Gp, Yp, eps=0.0):
    """Standard HALS (Appendix 'Update() Function'): w_i <- [w_i + (Y_i - (W G)_i) / G_ii]_+.

    Called with Gp = H^T H + alpha I and Yp = X H + alpha H it must reproduce the
    regularised rule; with alpha = 0 it is plain HALS.
    """
    W = np.array(Wold, dtype=np.float64, copy=True)
    k = W.shape[1]
    for i in range(k):
        W[:, i] = np.maximum(W[:, i] + (Yp[:, i] - W @ Gp[:, i]) / (Gp[i, i] + eps), 0.0)
    return W


# -------------------------------------------------------------------- BPP rows


def nls_rows(Gp, Yp):
    """Exact row NLS: x_r = argmin_{x >= 0} 1/2 x^T Gp x - Yp_r^T x for every row r.

    This is the ANLS update of Eq. ANLS4symNMF written per row (the QPs of the
    Update() appendix, with the usual 1/2).  Gp must be SPD (alpha > 0).
    Solved with scipy's Lawson-Hanson NNLS on min ||L^T x - L^{-1} y||, Gp = L L^T.
    """
    L = np.linalg.cholesky(Gp)
    A = L.T
    out = np.empty_like(Yp, dtype=np.float64)
    for r in range(Yp.shape[0]):
        b = sla.solve_triangular(L, Yp[r], lower=True)
        out[r], _ = sopt.nnls(A, b, maxiter=50 * Gp.shape[0])
    return out


def nls_row_bruteforce(Gp, y):
    """Brute force over all 2^k supports; returns the unique KKT point (k <= 12)."""
    k = Gp.shape[0]
    best = None
    for mask in range(1 << k):
        F = [i for i in range(k) if (mask >> i) & 1]
        x = np.zeros(k)
        if F:
            x[F] = np.linalg.solve(Gp[np.ix_(F, F)], y[F])
            if (x[F] < -1e-12).any():
                continue
        g = Gp @ x - y
        nF = [i for i in range(k) if not (mask >> i) & 1]
        if nF and (g[nF] < -1e-10 * max(1.0, np.abs(y).max())).any():
            continue
        obj = 0.5 * x @ Gp @ x - y @ x
        if best is None or obj < best[0]:
            best = (obj, x)
    return best[1]


def bpp_update(H, G, Y, alpha):
    """W := Update(G + alpha I, Y + alpha H) with the exact NLS solve (BPP variant)."""
    k = G.shape[0]
    return nls_rows(G + alpha * np.eye(k), Y + alpha * H)


# ------------------------------------------------------------------ RRF / EVD


def rrf(X, Omega, q):
    """Randomised range finder (Alg. RRF) with re-orthonormalisation (Alg. Ada-RRF loop).

    Y = X Omega, Q = qr(Y); then q times: Q = qr(X^T Q), Q = qr(X Q).
    Householder thin QR (LAPACK) stands for the paper's thin-QR.
    """
    Q, _ = np.linalg.qr(X @ Omega)
    for _ in range(q):
        Q, _ = np.linalg.qr(X.T @ Q)
        Q, _ = np.linalg.qr(X @ Q)
    return Q


def apx_evd(X, Omega, q):
    """Alg. Apx-EVD: Q = RRF(X), T = Q^T X Q, T = Q_T Lambda Q_T^T, U = Q Q_T.

    All l eigenpairs are kept, negative ones included.  Returns (U, lam).
    """
    Q = rrf(X, Omega, q)
    T = Q.T @ (X @ Q)
    T = 0.5 * (T + T.T)
    lam, QT = np.linalg.eigh(T)
    return Q @ QT, lam


def ada_rrf(X, Omega, q_max, tol=1e-3):
    """Adaptive randomised range finder (appendix, Alg. Ada-RRF), X symmetric so X^T = X.

    Q = qr(X Omega); then at most q_max times: B^T = X^T Q, the QB residual
    ||Q B - X||_F^2 = ||X||_F^2 - ||B||_F^2 (the appendix's identity) gives the
    normalized residual r_j = sqrt(||X||^2 - ||B||^2) / ||X||, Q = qr(B^T);
    stop when the residual fell by less than `tol` since the previous check
    (the experiments' rule: 1e-3 per power iteration); otherwise Y = X Q,
    Q = qr(Y).  Householder thin QR stands for qr().

    Returns (Q, hist, passes): the residuals r_1, r_2, ... of the checks made,
    and the number of products with X.
    """
    normX2 = float((X * X).sum())
    Q, _ = np.linalg.qr(X @ Omega)
    passes, hist = 1, []
    for _ in range(q_max):
        Bt = X.T @ Q
        passes += 1
        hist.append(math.sqrt(max(normX2 - float((Bt * Bt).sum()), 0.0) / normX2))
        Q, _ = np.linalg.qr(Bt)
        if len(hist) >= 2 and hist[-2] - hist[-1] < tol:
            break
        Q, _ = np.linalg.qr(X @ Q)
        passes += 1
    return Q, hist, passes


def apx_evd_ada(X, Omega, q_max, tol=1e-3):
    """Alg. Apx-EVD with the basis from Alg. Ada-RRF: T = Q^T X Q = V Lambda V^T, U = Q V.

    Returns (U, lam, hist, passes); passes counts the product for T as well.
    """
    Q, hist, passes = ada_rrf(X, Omega, q_max, tol)
    T = Q.T @ (X @ Q)
    T = 0.5 * (T + T.T)
    lam, V = np.linalg.eigh(T)
    return Q @ V, lam, hist, passes + 1


def lai_product(U, lam, F):
    """X F replaced by U (Lambda (U^T F)) (Alg. LAI-SymNMF, Y_H and Y_W lines)."""
    return U @ (lam[:, None] * (U.T @ F))


# ---------------------------------------------------------------- solvers


def default_alpha(X):
    """alpha = max(X) (Section 'Experimental Results', WoS setup)."""
    return float(np.max(X))


def hals_symnmf(X, H0, alpha, sweeps, W0=None, rule="hals", record=True):
    """Regularised alternating SymNMF on the full X (W-update then H-update per sweep).

    Returns (W, H, objs) where objs[t] is the surrogate objective after sweep t.
    """
    H = np.array(H0, dtype=np.float64, copy=True)
    W = H.copy() if W0 is None else np.array(W0, dtype=np.float64, copy=True)
    objs = []
    for _ in range(sweeps):
        G, Y = H.T @ H, X @ H
        W = hals_update_efficient(W, H, G, Y, alpha) if rule == "hals" else bpp_update(H, G, Y, alpha)
        G, Y = W.T @ W, X @ W
        H = hals_update_efficient(H, W, G, Y, alpha) if rule == "hals" else bpp_update(W, G, Y, alpha)
        if record:
            objs.append(surrogate_objective(X, W, H, alpha))
    return W, H, objs


def lai_symnmf(U, lam, H0, alpha, sweeps, W0=None, rule="hals", record=True):
    """Alg. LAI-SymNMF sweeps on X ~ U Lambda U^T.

    objs[t] is the LAI surrogate objective ||U Lambda U^T - W H^T||^2 + alpha ||W - H||^2,
    evaluated with the trace trick (||U Lambda U^T||^2 = sum lambda^2 since U is orthonormal).
    """
    H = np.array(H0, dtype=np.float64, copy=True)
    W = H.copy() if W0 is None else np.array(W0, dtype=np.float64, copy=True)
    normX2 = float((lam ** 2).sum())
    objs = []
    for _ in range(sweeps):
        G, Y = H.T @ H, lai_product(U, lam, H)
        W = hals_update_efficient(W, H, G, Y, alpha) if rule == "hals" else bpp_update(H, G, Y, alpha)
        G, Y = W.T @ W, lai_product(U, lam, W)
        H = hals_update_efficient(H, W, G, Y, alpha) if rule == "hals" else bpp_update(W, G, Y, alpha)
        if record:
            # Y = U Lambda U^T W, so tr(H^T Y) = tr(W^T (U Lambda U^T) H)
            r2 = trace_trick_residual_sq(normX2, W.T @ W, H.T @ H, H.T @ Y)
            objs.append(r2 + alpha * float(((W - H) ** 2).sum()))
    return W, H, objs


# ------------------------------------------------------------- Compressed-NMF


def compressed_half(Xt_Q, Q, Fold, Ffix, alpha, rule="hals"):
    """One half of Compressed-SymNMF (appendix "Comparison between LAI-NMF and Compressed-NMF"):
    min_{F >= 0} ||Q^T (Ffix F^T - X)||_F^2 + alpha ||F - Ffix||_F^2, Q = RRF(X) (one basis, X symmetric).

    Its normal equations give Update(G_c + alpha I, Y_c + alpha Ffix) with M = Q^T Ffix (l x k),
    G_c = M^T M = Ffix^T Q Q^T Ffix and Y_c = X^T Q M (Xt_Q = X^T Q, computed once).
    """
    M = Q.T @ Ffix
    G = M.T @ M
    Y = Xt_Q @ M
    if rule == "hals":
        return hals_update_efficient(Fold, Ffix, G, Y, alpha), G, Y
    return bpp_update(Ffix, G, Y, alpha), G, Y


def compressed_symnmf(X, Q, H0, alpha, sweeps, W0=None, rule="hals"):
    """Compressed-SymNMF sweeps (W half then H half).  Returns (W, H, objs): objs[t] is the H half's
    compressed objective ||Q^T (W H^T - X)||_F^2 + alpha ||W - H||_F^2 after sweep t."""
    H = np.array(H0, dtype=np.float64, copy=True)
    W = H.copy() if W0 is None else np.array(W0, dtype=np.float64, copy=True)
    Xt_Q = X.T @ Q
    B = Q.T @ X
    objs = []
    for _ in range(sweeps):
        W, _, _ = compressed_half(Xt_Q, Q, W, H, alpha, rule)
        H, _, _ = compressed_half(Xt_Q, Q, H, W, alpha, rule)
        R = (Q.T @ W) @ H.T - B
        objs.append(float((R * R).sum() + alpha * ((W - H) ** 2).sum()))
    return W, H, objs


# ------------------------------------------------------------- PGNCG (all-at-once)


def gn_jacobian_apply(H, P):
    """J p for the residual r(H) = vec(H H^T - X): d/dt (H + t P)(H + t P)^T at t = 0 = P H^T + H P^T."""
    return P @ H.T + H @ P.T


def gn_normal_apply(H, G, P):
    """J^T J p = 2 (P H^T H + H P^T H) (section "Projected Gauss-Newton with Conjugate Gradients"),
    with G = H^T H; J^T applied to a symmetric n x n residual S is 2 S H."""
    return 2.0 * (P @ G + H @ (P.T @ H))


def pgncg_iteration(Y, H, s_max):
    """One PGNCG iteration (section "Projected Gauss-Newton with Conjugate Gradients", appendix
    Alg. LAI-PGNCG-SymNMF) given Y = X H (or U Lambda U^T H for LAI-PGNCG).

    R = J^T r = 2 (H (H^T H) - X H), the Gauss-Newton normal equations J^T J Z = R solved from
    Z = 0 by s_max steps of conjugate gradients, then H <- max(H - Z, 0).  The printed loop never
    updates the search direction and reuses alpha; this restatement takes standard CG (step
    alpha = e_old / <P, J^T J P>, beta = e_new / e_old, P <- R + beta P), stopped early once CG
    has converged (||R|| <= 1e-12 ||R_0||): past that point the recurrence divides rounding noise.
    """
    G = H.T @ H
    R = 2.0 * (H @ G - Y)
    P = R.copy()
    Z = np.zeros_like(H)
    e_old = float((R * R).sum())
    e_stop = 1e-24 * e_old
    for _ in range(s_max):
        if e_old <= e_stop or e_old == 0.0:
            break
        Yc = gn_normal_apply(H, G, P)
        a = e_old / float((P * Yc).sum())
        Z += a * P
        R -= a * Yc
        e_new = float((R * R).sum())
        P = R + (e_new / e_old) * P
        e_old = e_new
    return np.maximum(H - Z, 0.0)


def symnmf_objective(normX2, HtH, HtXH):
    """||X - H H^T||_F^2 = ||X||^2 - 2 tr(H^T X H) + ||H^T H||_F^2 (trace trick, Eq. symnmf_obj)."""
    return float(normX2 - 2.0 * np.trace(HtXH) + (HtH * HtH).sum())


def pgncg_symnmf(apply_x, normX2, H0, iters, s_max=5):
    """PGNCG-SymNMF (apply_x = X @) or LAI-PGNCG-SymNMF (apply_x = U Lambda U^T @).

    Returns (H, objs): objs[t] = ||X - H H^T||_F^2 after iteration t, with ||X||^2 = normX2.
    """
    H = np.array(H0, dtype=np.float64, copy=True)
    objs = []
    for _ in range(iters):
        H = pgncg_iteration(apply_x(H), H, s_max)
        objs.append(symnmf_objective(normX2, H.T @ H, H.T @ apply_x(H)))
    return H, objs


# ------------------------------------------------------------ leverage scores


def leverage_scores(F, rel_tol=1e-12):
    """Exact leverage scores of F via CholeskyQR (Alg. LvS-SymNMF, first three lines).

    R = chol(F^T F) (upper), Q = F R^{-1}, l_i = ||Q[i,:]||^2.  If F^T F is not
    positive definite, the pseudo-inverse form l_i = f_i V diag(1/s) V^T f_i^T
    over the eigenpairs with s > rel_tol * max(s) is used.
    Returns (lev, full_rank).
    """
    G = F.T @ F
    try:
        R = np.linalg.cholesky(G).T
        Q = sla.solve_triangular(R, F.T, trans="T", lower=False).T  # F R^{-1}
        return (Q * Q).sum(axis=1), True
    except np.linalg.LinAlgError:
        s, V = np.linalg.eigh(G)
        keep = s > rel_tol * s.max()
        Z = (F @ V[:, keep]) / np.sqrt(s[keep])
        return (Z * Z).sum(axis=1), False


QSHIFT = 40  # fixed-point bits of the integer sampling weights


def hybrid_sample(lev, k, s, tau, seed, it, side, ubits=64, words=None):
    """Hybrid leverage-score sampling (Section 'Practical Considerations for LvS-SymNMF').

    I_D = {i : l_i / k >= tau} (kept with weight 1, ascending index order),
    theta = sum_{I_D} l_i, s_D = |I_D|, s_R = max(s - s_D, 0) draws with
    replacement from I_R with p~_i proportional to l_i (the paper's l_i / (k - theta);
    the normaliser used is sum_{I_R} l_i, equal to k - theta for full-rank F).
    Draw weights on S^T S are 1 / (s_R p~_i) (Eq. lev_score_S).

    Integer draw map (the paper is silent on the sampler): q_i = floor(l_i 2^40)
    for i in I_R, C = inclusive prefix sum of q (exact integers), T = C[-1];
    draw j takes u_j (an `ubits`-bit uniform, Philox by default) and
    r = floor(u_j T / 2^ubits); the row is the first i with C_i > r.

    Returns dict(idx, wt, s_D, s_R, theta).
    """
    lev = np.asarray(lev, dtype=np.float64)
    n = lev.shape[0]
    thr = tau * k
    det = lev >= thr
    D = np.nonzero(det)[0]
    s_D = int(D.shape[0])
    theta = float(lev[D].sum())
    q = np.where(det, 0.0, np.floor(lev * float(1 << QSHIFT))).astype(np.uint64)
    C = np.cumsum(q, dtype=np.uint64)
    T = int(C[-1]) if n else 0
    s_R = max(s - s_D, 0) if T > 0 else 0
    if words is None:
        words = philox.philox_sample_words(s_R, it, side, seed)
    idx_R = np.empty(s_R, dtype=np.int64)
    for j in range(s_R):
        r = (words[j] * T) >> ubits
        idx_R[j] = np.searchsorted(C, np.uint64(r), side="right")
    mass_R = float(lev[~det].sum())
    pt = lev[idx_R] / mass_R if s_R else np.zeros(0)
    wt_R = 1.0 / (s_R * pt) if s_R else np.zeros(0)
    idx = np.concatenate([D.astype(np.int64), idx_R])
    wt = np.concatenate([np.ones(s_D), wt_R])
    return dict(idx=idx, wt=wt, s_D=s_D, s_R=s_R, theta=theta, T=T, C=C, q=q)


def sampled_products(X, F, idx, wt):
    """Y = X S^T S F (n x k) and G = F^T S^T S F (Alg. LvS-SymNMF, Y_H / G_H lines).

    Duplicate draws accumulate.  X may be dense (ndarray) or scipy sparse.
    """
    Fs = F[idx] * wt[:, None]
    Xs = X[:, idx]
    Y = np.asarray(Xs @ Fs)
    G = F[idx].T @ Fs
    return Y, G


def lvs_symnmf(X, H0, alpha, iters, s, tau, seed, W0=None, rule="hals", trace=None):
    """Alg. LvS-SymNMF: per half, leverage scores -> hybrid sample -> sampled Y, G -> Update."""
    H = np.array(H0, dtype=np.float64, copy=True)
    W = H.copy() if W0 is None else np.array(W0, dtype=np.float64, copy=True)
    k = H.shape[1]
    for it in range(iters):
        lev, _ = leverage_scores(H)
        smp = hybrid_sample(lev, k, s, tau, seed, it, 0)
        Y, G = sampled_products(X, H, smp["idx"], smp["wt"])
        W = hals_update_efficient(W, H, G, Y, alpha) if rule == "hals" else bpp_update(H, G, Y, alpha)
        if trace is not None:
            trace.append(("W", smp))
        lev, _ = leverage_scores(W)
        smp = hybrid_sample(lev, k, s, tau, seed, it, 1)
        Y, G = sampled_products(X, W, smp["idx"], smp["wt"])
        H = hals_update_efficient(H, W, G, Y, alpha) if rule == "hals" else bpp_update(W, G, Y, alpha)
        if trace is not None:
            trace.append(("H", smp))
    return W, H


# ------------------------------------------------------- the experiments' schedule


def stop_rule_phase(step, max_iters, tol=1e-4, count=4):
    """Iterate `step()` (returning the normalized residual after the iteration) until the residual
    has fallen by less than `tol` in `count` consecutive iterations (section "Experimental
    Results": 1e-4 for four consecutive iterations), or max_iters.  Returns (iterations, last NR)."""
    prev, nr, small, t = 0.0, 0.0, 0, 0
    while t < max_iters:
        nr = step()
        t += 1
        if t > 1:
            small = small + 1 if prev - nr < tol else 0
        prev = nr
        if small >= count:
            break
    return t, nr


def lai_schedule(X, Omega, H0, alpha, q_max=10, ada_tol=1e-3, tol=1e-4, count=4, max_iters=500,
                 refine=True, max_refine=200, rule="hals"):
    """LAI-HALS / LAI-BPP with the experiments' schedule: Ada-RRF + Apx-EVD, LAI sweeps to the
    stopping rule (NR of the surrogate against U Lambda U^T), then Iterative Refinement sweeps on X
    with the same rule.  Returns dict(W, H, passes, iters, refine_iters, nr_final)."""
    U, lam, hist, passes = apx_evd_ada(X, Omega, q_max, ada_tol)
    state = {"W": np.array(H0, dtype=np.float64, copy=True), "H": np.array(H0, dtype=np.float64, copy=True)}
    lai_nx2 = float((lam ** 2).sum())
    nx2 = float((X * X).sum())

    def lai_step():
        W, H, objs = lai_symnmf(U, lam, state["H"], alpha, 1, W0=state["W"], rule=rule)
        state["W"], state["H"] = W, H
        return math.sqrt(max(objs[-1], 0.0) / lai_nx2)

    def full_step():
        W, H, objs = hals_symnmf(X, state["H"], alpha, 1, W0=state["W"], rule=rule)
        state["W"], state["H"] = W, H
        return math.sqrt(max(objs[-1], 0.0) / nx2)

    iters, _ = stop_rule_phase(lai_step, max_iters, tol, count)
    riters = stop_rule_phase(full_step, max_refine, tol, count)[0] if refine else 0
    return dict(W=state["W"], H=state["H"], passes=passes, checks=len(hist), iters=iters, refine_iters=riters,
                nr_final=normalized_residual(X, state["W"], state["H"]))


# ----------------------------------------------------------------- helpers


def init_scale(X, k):
    """2 sqrt(zeta / k), zeta = mean(X): the initial-factor scale of the experiments section."""
    return 2.0 * math.sqrt(float(np.mean(X)) / k)


def cluster_labels(H):
    """Cluster of vertex i = argmax over row i of H (experiments section)."""
    return np.argmax(H, axis=1)


def adjusted_rand_index(a, b):
    """Adjusted Rand index of two labelings (Hubert & Arabie), for the planted-recovery pin."""
    a = np.asarray(a)
    b = np.asarray(b)
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    M = np.zeros((ai.max() + 1, bi.max() + 1))
    np.add.at(M, (ai, bi), 1)
    comb = lambda x: x * (x - 1) / 2.0  # noqa: E731
    sij = comb(M).sum()
    sa = comb(M.sum(1)).sum()
    sb = comb(M.sum(0)).sum()
    tot = comb(float(len(a)))
    exp = sa * sb / tot
    mx = 0.5 * (sa + sb)
    return float((sij - exp) / (mx - exp)) if mx != exp else 1.0


def all_supports(k):
    """Every subset of range(k) (for brute-force pins)."""
    for r in range(k + 1):
        yield from itertools.combinations(range(k), r)
