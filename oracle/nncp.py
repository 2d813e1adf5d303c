"""Plain FP64 statement of alternating-update NNCP (test infrastructure only).

Notation follows the paper (PLANC, arXiv 1909.01149):
  X            dense I_1 x ... x I_N tensor, stored mode-1 fastest (Sec. 4.1.2,
               "natural mode-descending" = generalised column-major).  Here it
               is a NumPy array of shape (I_1, ..., I_N); its Fortran-order
               ravel is the flat buffer the GPU library receives.
  H[n]         factor matrix H^(n), I_n x R.
  G[n]         Gram matrix H^(n)^T H^(n), R x R (Alg. 1).
  S            Hadamard product of the other modes' Grams (Alg. 1, S^(n)).
  M            MTTKRP result M^(n) = X_(n) (H^N kr ... kr H^(n+1) kr H^(n-1)
               kr ... kr H^1) (Eq. nls and Sec. 4.2).
  lam          column weights lambda (Sec. A.1, factor normalisation).

Nothing here uses a dimension tree: the MTTKRP is the explicit mode-n
matricization times the explicit Khatri-Rao product.  The dimension tree of
Sec. 4.2 reaches exactly this result (up to rounding order), so this is the
definition the GPU path must reproduce.

Readings of the paper where it is silent or inconsistent are marked
"reading:" in the docstrings; the same readings are implemented by the GPU
library.
"""

from __future__ import annotations

import itertools
import math

import numpy as np

# ----------------------------------------------------------------------------
# Tensor algebra (Sec. 2 and 4.2; Kolda-Bader conventions cited in Sec. 3)
# ----------------------------------------------------------------------------


def unfold(X: np.ndarray, n: int) -> np.ndarray:
    """Mode-n matricization X_(n) (0-based n), I_n x prod_{k != n} I_k.

    Column index j = sum_{k != n} i_k J_k with J_k = prod_{m < k, m != n} I_m,
    i.e. the lowest remaining mode varies fastest (Kolda-Bader, Sec. 3).
    """
    return np.reshape(np.moveaxis(X, n, 0), (X.shape[n], -1), order="F")


def khatri_rao(mats) -> np.ndarray:
    """Khatri-Rao product A_1 kr A_2 kr ... kr A_k (column-wise Kronecker).

    Column r is kron(A_1[:, r], ..., A_k[:, r]); the LAST matrix's row index
    varies fastest, as in the reverse-order products K^{i:j} = H^j kr ... kr
    H^i of Alg. 3.
    """
    mats = list(mats)
    R = mats[0].shape[1]
    out = np.ones((1, R))
    for A in mats:
        assert A.shape[1] == R
        out = (out[:, None, :] * A[None, :, :]).reshape(-1, R)
    return out


def krp_except(H, n: int) -> np.ndarray:
    """H^N kr ... kr H^(n+1) kr H^(n-1) kr ... kr H^1 (Eq. nls, Sec. 4.3)."""
    N = len(H)
    order = [H[k] for k in range(N - 1, -1, -1) if k != n]
    return khatri_rao(order)


def mttkrp(X: np.ndarray, H, n: int) -> np.ndarray:
    """M^(n) = X_(n) . krp_except(H, n)  (Alg. 1 MTTKRP; Eq. nls)."""
    return unfold(X, n) @ krp_except(H, n)


def mttkrp_rows(X: np.ndarray, H, n: int, rows) -> np.ndarray:
    """Selected rows of M^(n): the definition applied to the sub-tensor
    X[..., rows, ...] (mode n restricted to `rows`).  Lets a full-size result
    be sampled without forming the whole matricization."""
    idx = [slice(None)] * X.ndim
    idx[n] = np.asarray(rows)
    Xs = np.asarray(X[tuple(idx)], dtype=np.float64)
    return mttkrp(Xs, [h if k != n else h[np.asarray(rows)] for k, h in enumerate(H)], n)


def mttkrp_bruteforce(X: np.ndarray, H, n: int) -> np.ndarray:
    """Element-wise MTTKRP sum with Python loops; for tiny tensors only.

    M^(n)[i, r] = sum over all multi-indices with i_n = i of
    X[i_1, ..., i_N] * prod_{k != n} H^(k)[i_k, r]   (Sec. 4.2.1).
    """
    N = X.ndim
    R = H[0].shape[1]
    out = np.zeros((X.shape[n], R))
    for idx in itertools.product(*[range(s) for s in X.shape]):
        x = X[idx]
        for r in range(R):
            p = x
            for k in range(N):
                if k != n:
                    p *= H[k][idx[k], r]
            out[idx[n], r] += p
    return out


def gram(Hn: np.ndarray) -> np.ndarray:
    """G^(n) = H^(n)^T H^(n)  (Alg. 1, local SYRK of Alg. 2)."""
    return Hn.T @ Hn


def gram_hadamard(G, n: int) -> np.ndarray:
    """S^(n) = G^(1) * ... * G^(n-1) * G^(n+1) * ... * G^(N)  (Alg. 1)."""
    R = G[0].shape[0]
    S = np.ones((R, R))
    for k, Gk in enumerate(G):
        if k != n:
            S = S * Gk
    return S


def sqnorm(X: np.ndarray) -> float:
    """alpha = ||X||^2 (Alg. 4, Norm-Squared)."""
    x = np.asarray(X, dtype=np.float64).ravel()
    return float(x @ x)


def cp_full(H, lam=None) -> np.ndarray:
    """Dense [[lam; H^(1), ..., H^(N)]] as an (I_1, ..., I_N) array."""
    R = H[0].shape[1]
    w = np.ones(R) if lam is None else np.asarray(lam, dtype=np.float64)
    shape = tuple(h.shape[0] for h in H)
    # X_(1) = H^1 diag(w) (H^N kr ... kr H^2)^T, reshaped in Fortran order.
    X1 = (H[0] * w) @ krp_except(H, 0).T
    return np.reshape(X1, shape, order="F")


def choose_split(dims) -> int:
    """Root split S of the dimension tree (Sec. 4.2.2), 1-based, 1 <= S < N.

    reading: the text asks for the two products to be "nearly equal" and also
    states the literal rule "smallest S with prod(first S) > prod(rest)".  The
    library minimises |log(prod_{k<=S} I_k / prod_{k>S} I_k)| and breaks ties
    towards the larger S (this agrees with the literal rule on 3-way cubes).
    The MTTKRP results do not depend on S.
    """
    N = len(dims)
    assert N >= 2
    best, best_s = None, 1
    for s in range(1, N):
        left = sum(math.log(d) for d in dims[:s])
        right = sum(math.log(d) for d in dims[s:])
        score = abs(left - right)
        if best is None or score <= best + 1e-12:
            best, best_s = score, s
    return best_s


# ----------------------------------------------------------------------------
# NNLS updates (Sec. 4.3): solve min_{Hhat >= 0} ||K Hhat^T - X_(n)^T||_F
# given only S = K^T K and M = X_(n) K.  Rows of Hhat are independent.
# ----------------------------------------------------------------------------


def nls_objective(S: np.ndarray, M: np.ndarray, H: np.ndarray) -> float:
    """0.5 ||A X - B||^2 up to the constant 0.5 ||B||^2, with X = H^T:
    0.5 tr(H S H^T) - tr(H^T M)  (Eq. nls written with S and M only)."""
    return float(0.5 * np.sum((H @ S) * H) - np.sum(H * M))


MU_EPS = 1e-16


def nls_mu(S, M, H, eps: float = MU_EPS):
    """One multiplicative update (Eq. muupd) in row form:
    H <- H * M / (H S + eps).

    reading: the paper adds "a small value" to the denominator; it is 1e-16.
    """
    return H * M / (H @ S + eps)


HALS_TINY = 1e-300


def nls_hals(S, M, H, tiny: float = HALS_TINY):
    """One HALS sweep (Eq. halsupd) in row form, columns r = 1..R in order,
    each using the columns already updated in this sweep (Gauss-Seidel):
        H(:, r) <- [ H(:, r) + (M(:, r) - H S(:, r)) / S(r, r) ]_+ .

    reading: the division by S(r, r) of Eq. halsupd is kept (the shorter rule
    in Sec. 2 omits it); a column with S(r, r) <= tiny is left unchanged.  No
    normalisation inside the sweep; the factor is normalised after the update
    as in Alg. 4.
    """
    H = np.array(H, dtype=np.float64, copy=True)
    R = S.shape[0]
    for r in range(R):
        srr = S[r, r]
        if srr <= tiny:
            continue
        H[:, r] = np.maximum(0.0, H[:, r] + (M[:, r] - H @ S[:, r]) / srr)
    return H


ADMM_MAX_INNER = 5
ADMM_TOL = 1e-2


def nls_admm(S, M, H, U=None, max_inner: int = ADMM_MAX_INNER,
             tol: float = ADMM_TOL, return_state: bool = False):
    """AO-ADMM update (Eq. admmnls / admmupd) in row form (H = X^T):
        rho     = ||A||_F^2 / R = trace(S) / R
        L L^T   = S + rho I        (Cholesky, cached for all inner steps)
        Htil    <- (M + rho (H + U)) (S + rho I)^{-1}
        H       <- [Htil - U]_+
        U       <- U + H - Htil
    for at most 5 inner steps.

    reading: the printed update mixes transposes; this is its consistent row
    form.  U starts at zero on every call ("U is initialized as a matrix of
    all zeros").  Stop after the step where both
        ||H - Htil||_F^2 < tol ||H||_F^2   and
        ||H - H_prev||_F^2 < tol ||U||_F^2
    hold (tol = 1e-2); the paper defers the exact rule to its reference.
    """
    R = S.shape[0]
    tr = float(np.trace(S))
    rho = tr / R if tr > 0 else 1.0  # reading: an all-zero S uses rho = 1
    L = np.linalg.cholesky(S + rho * np.eye(R))
    H = np.array(H, dtype=np.float64, copy=True)
    U = np.zeros_like(H) if U is None else np.array(U, dtype=np.float64)
    steps = 0
    for _ in range(max_inner):
        H_prev = H
        rhs = M + rho * (H + U)
        # (S + rho I) is symmetric: Htil^T = (S + rho I)^{-1} rhs^T.
        Z = np.linalg.solve(L, rhs.T)
        Htil = np.linalg.solve(L.T, Z).T
        H = np.maximum(0.0, Htil - U)
        U = U + H - Htil
        steps += 1
        r_primal = np.sum((H - Htil) ** 2)
        r_dual = np.sum((H - H_prev) ** 2)
        if r_primal < tol * np.sum(H ** 2) and r_dual < tol * np.sum(U ** 2):
            break
    if return_state:
        return H, U, steps
    return H


BPP_BACKUP = 3


def nls_bpp_row(S, m, F0=None, max_iter=None):
    """Block principal pivoting for one row (Eq. snls; Kim and Park 2011).

    Solves min_{x >= 0} ||A x - b|| given S = A^T A and m = A^T b.  KKT:
    x >= 0, y = S x - m >= 0, x * y = 0.  F is the passive set.  Infeasible
    indices V = {i in F: x_i < 0} u {i not in F: y_i < 0} are exchanged in
    full while their count keeps falling; after 3 non-improving rounds the
    backup rule exchanges only the largest infeasible index.  The passive-set
    system S_FF x_F = m_F is solved by Cholesky (normal equations).

    reading: the paper defers the details to Kim-Park; the passive set starts
    from the warm start's support (F0) and the number of exchanges is capped
    at 10 R (then the current x, clipped at zero, is returned).  Returns
    (x, iterations, converged).
    """
    R = S.shape[0]
    if max_iter is None:
        max_iter = 10 * R
    F = np.zeros(R, dtype=bool) if F0 is None else np.array(F0, dtype=bool)

    def solve(F):
        x = np.zeros(R)
        if F.any():
            idx = np.flatnonzero(F)
            SFF = S[np.ix_(idx, idx)]
            Lc = np.linalg.cholesky(SFF)
            x[idx] = np.linalg.solve(Lc.T, np.linalg.solve(Lc, m[idx]))
        y = S @ x - m
        y[F] = 0.0
        return x, y

    x, y = solve(F)
    p = BPP_BACKUP
    ninf = R + 1
    it = 0
    converged = False
    while True:
        V = (F & (x < 0)) | (~F & (y < 0))
        nv = int(V.sum())
        if nv == 0:
            converged = True
            break
        if it >= max_iter:
            break
        if nv < ninf:
            ninf = nv
            p = BPP_BACKUP
            Vhat = V
        elif p >= 1:
            p -= 1
            Vhat = V
        else:
            Vhat = np.zeros(R, dtype=bool)
            Vhat[np.flatnonzero(V).max()] = True
        F = F ^ Vhat
        x, y = solve(F)
        it += 1
    return np.maximum(x, 0.0), it, converged


def nls_bpp(S, M, H=None):
    """BPP applied to every row of Hhat (rows decouple, Sec. 4.3).

    Returns (Hhat, max_iterations, all_converged)."""
    rows, R = M.shape
    out = np.zeros((rows, R))
    iters, conv = 0, True
    for i in range(rows):
        F0 = None if H is None else (np.asarray(H[i]) > 0)
        out[i], it, ok = nls_bpp_row(S, M[i], F0)
        iters = max(iters, it)
        conv = conv and ok
    return out, iters, conv


def nls_pgd(S, M, H, steps: int = 1):
    """Projected gradient steps on 0.5 tr(H S H^T) - tr(H^T M):
        H <- [H - eta (H S - M)]_+,  eta = 1 / ||S||_F.

    reading: the step 1/||S||_F is a safe bound on 1/lambda_max(S) that needs
    no eigen-solver; this is the project's gradient-driven NLS option.
    """
    eta = 1.0 / max(float(np.linalg.norm(S)), 1e-300)
    H = np.array(H, dtype=np.float64, copy=True)
    for _ in range(steps):
        H = np.maximum(0.0, H - eta * (H @ S - M))
    return H


def nls_ucp(S, M):
    """Unconstrained update (the UCP solver of Sec. 6, CP-ALS): the exact
    minimiser of the mode-n least-squares problem ||X_(n) - H K^T||^2 with no
    non-negativity, i.e. the solution of H S = M with S = K^T K (Alg. 1's S)
    symmetric positive definite."""
    S = np.asarray(S, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    return np.linalg.solve(S, M.T).T


NES_KAPPA = 100.0     # reading: largest condition number of the proximal problem
NES_MAX_INNER = 20    # Sec. 4.3.5: at most 20 inner iterations
NES_TOL = 1e-3        # reading: inner stop when max|X_{k+1} - Y_k| <= tol max|X_{k+1}|


def nes_params(S, kappa: float = NES_KAPPA):
    """Parameters of the Nesterov-type update (Sec. 4.3.5), from the extreme
    eigenvalues of S = A^T A (the paper defers their choice to the cited
    method; these are this project's readings):
      mu0, L0 = smallest / largest eigenvalue of S, clamped at 0;
      lam_p   = the smallest proximal weight that makes the condition number
                (L0 + lam_p) / (mu0 + lam_p) at most kappa, i.e.
                max(0, (L0 - kappa mu0) / (kappa - 1));
      L = L0 + lam_p, mu = mu0 + lam_p (Lipschitz and strong-convexity
      constants of f_p); beta = (1 - sqrt(mu/L)) / (1 + sqrt(mu/L)), the
      constant momentum of Nesterov's scheme for strongly convex f_p.
    Returns (lam_p, L, beta); L = 0 when S = 0."""
    ev = np.linalg.eigvalsh(np.asarray(S, dtype=np.float64))
    mu0, L0 = max(float(ev[0]), 0.0), max(float(ev[-1]), 0.0)
    lam_p = max(0.0, (L0 - kappa * mu0) / (kappa - 1.0))
    L, mu = L0 + lam_p, mu0 + lam_p
    if L <= 0.0:
        return lam_p, 0.0, 0.0
    sq = math.sqrt(mu / L)
    return lam_p, L, (1.0 - sq) / (1.0 + sq)


def nls_nes(S, M, Hstar, max_inner: int = NES_MAX_INNER, tol: float = NES_TOL,
            return_state: bool = False):
    """Nesterov-type update (Sec. 4.3.5, Eq. nesnls and Eq. nesinnerupd) in
    row form (X = H, A^T A = S, A^T B = M^T):
        f_p(H) = 1/2 tr(H S H^T) - tr(M^T H) + lam_p/2 ||H - H*||_F^2,  H >= 0,
    with H* the warm start (the factor of the previous outer iteration).
    Starting from X_0 = Y_0 = H*, each inner step takes
        grad = Y_k S - M + lam_p (Y_k - H*)       (reading: the true gradient
                                                  of f_p; the printed signs
                                                  disagree with each other)
        X_{k+1} = [Y_k - grad / L]_+
        Y_{k+1} = X_{k+1} + beta (X_{k+1} - X_k)
    and stops after the step where max|X_{k+1} - Y_k| <= tol max|X_{k+1}|
    (reading of the paper's bounds checks: the largest projected-gradient
    step, relative to the largest entry; one global check over all rows), or
    after max_inner steps.  S = 0 leaves H* unchanged.
    Returns Hhat, or (Hhat, steps) with return_state."""
    S = np.asarray(S, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    Hs = np.array(Hstar, dtype=np.float64, copy=True)
    lam_p, L, beta = nes_params(S)
    if L <= 0.0:
        return (Hs, 0) if return_state else Hs
    X, Y, k = Hs, Hs, 0
    while k < max_inner:
        grad = Y @ S - M + lam_p * (Y - Hs)
        Xn = np.maximum(0.0, Y - grad / L)
        step = float(np.max(np.abs(Xn - Y))) if Xn.size else 0.0
        big = float(np.max(np.abs(Xn))) if Xn.size else 0.0
        Y = Xn + beta * (Xn - X)
        X = Xn
        k += 1
        if step <= tol * big:
            break
    return (X, k) if return_state else X


def nes_extrapolate(H, lam, H_prev, lam_prev, s):
    """Outer acceleration candidate (Sec. 4.3.5, Eq. nesouterupd):
        F_new^(n) = F_i^(n) + s (F_i^(n) - F_{i-1}^(n))   for every mode n,
    on the model's factors with the weights absorbed into the last mode
    (F^(n) = H^(n) for n < N, F^(N) = H^(N) diag(lam)), which is the factor the
    last mode's update produced.  Readings: the candidate is projected onto
    the non-negative orthant (the NNCP constraint), then every factor's
    columns are normalised and the column norms multiplied into lam, so that
    [[lam_new; H_new]] = [[F_new]] (zero columns stay zero).
    Returns (H_new, lam_new)."""
    N = len(H)
    lam_new = None
    H_new = []
    for n in range(N):
        F = H[n] * lam if n == N - 1 else H[n]
        Fp = H_prev[n] * lam_prev if n == N - 1 else H_prev[n]
        Fn = np.maximum(0.0, F + s * (F - Fp))
        Hn, nu = normalize_columns(Fn)
        H_new.append(Hn)
        lam_new = nu if lam_new is None else lam_new * nu
    return H_new, lam_new


def model_error(X, H, lam, alpha):
    """Relative error of [[lam; H]] by the identity of Sec. A.2 at the last
    mode: one MTTKRP (the extra MTTKRP of Sec. 6's table) and the Grams."""
    N = len(H)
    G = [gram(h) for h in H]
    M = mttkrp(X, H, N - 1)
    S = gram_hadamard(G, N - 1)
    return fit_identity(alpha, M, H[N - 1] * lam, S, G[N - 1], lam)[0]


# ----------------------------------------------------------------------------
# Normalisation and error (Appendix, Alg. 4)
# ----------------------------------------------------------------------------


def normalize_columns(Hhat):
    """lam_r = ||Hhat(:, r)||_2; H = Hhat diag(lam)^{-1} (Alg. 4).

    reading: a zero column keeps lam_r = 0 and stays zero (no division)."""
    lam = np.sqrt(np.sum(Hhat * Hhat, axis=0))
    H = np.zeros_like(Hhat)
    nz = lam > 0
    H[:, nz] = Hhat[:, nz] / lam[nz]
    return H, lam


def fit_identity(alpha, M_N, Hhat_N, S_N, G_N, lam):
    """Relative error by the identity of Sec. A.2 / Alg. 4:
        beta  = <M^(N), Hhat^(N)>,  gamma = lam^T (S^(N) * G^(N)) lam,
        eps   = sqrt(max(0, alpha - 2 beta + gamma) / alpha).
    reading: the radicand is clamped at zero; fit = 1 - eps.
    Returns (eps, fit)."""
    beta = float(np.sum(M_N * Hhat_N))
    gamma = float(lam @ (S_N * G_N) @ lam)
    # reading: an all-zero tensor (alpha = 0) reports eps = 0
    eps = math.sqrt(max(0.0, alpha - 2.0 * beta + gamma) / alpha) if alpha > 0 else 0.0
    return eps, 1.0 - eps


def fit_explicit(X, H, lam):
    """Relative error ||X - [[lam; H]]|| / ||X|| by explicit reconstruction."""
    D = np.asarray(X, dtype=np.float64) - cp_full(H, lam)
    eps = math.sqrt(float(np.sum(D * D)) / sqnorm(X))
    return eps, 1.0 - eps


# ----------------------------------------------------------------------------
# The outer loop (Alg. 1 with the normalisation and error of Alg. 4)
# ----------------------------------------------------------------------------


def nncp(X, H_init, alg: str = "hals", iters: int = 10, tol=None,
         record_objective: bool = False, nes_accel: bool = True):
    """Alternating-update NNCP, Alg. 1 with Alg. 4's normalisation and error.

    reading: all N factors are initialised (the warm start needs H^(1) too);
    initial factors are not normalised; lam starts at 1; the NNLS warm start
    for mode n is H^(n) diag(lam) (the solve is for H^(n) Lambda); a fixed
    number of outer iterations is run unless tol is given.

    alg "nes": the Nesterov-type update per mode and, with nes_accel, the
    outer acceleration after every outer iteration but the first.

    Returns dict(H=list, lam=array, rel_err=list per outer iteration,
    inner=list of per-call inner counts, accepted=list of the acceleration
    decisions).
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.ndim
    H = [np.array(h, dtype=np.float64, copy=True) for h in H_init]
    R = H[0].shape[1]
    alpha = sqnorm(X)
    lam = np.ones(R)
    G = [gram(h) for h in H]
    rel_err, inner, objective, accepted = [], [], [], []
    H_prev, lam_prev = None, None
    for it in range(iters):
        for n in range(N):
            M = mttkrp(X, H, n)
            S = gram_hadamard(G, n)
            Hhat0 = H[n] * lam
            if alg == "mu":
                Hhat = nls_mu(S, M, Hhat0)
                inner.append(1)
            elif alg == "hals":
                Hhat = nls_hals(S, M, Hhat0)
                inner.append(1)
            elif alg == "admm":
                Hhat, _, k = nls_admm(S, M, Hhat0, return_state=True)
                inner.append(k)
            elif alg == "bpp":
                Hhat, k, _ = nls_bpp(S, M, Hhat0)
                inner.append(k)
            elif alg == "pgd":
                Hhat = nls_pgd(S, M, Hhat0)
                inner.append(1)
            elif alg == "ucp":
                Hhat = nls_ucp(S, M)
                inner.append(1)
            elif alg == "nes":
                Hhat, k = nls_nes(S, M, Hhat0, return_state=True)
                inner.append(k)
            else:
                raise ValueError(alg)
            H[n], lam = normalize_columns(Hhat)
            G[n] = gram(H[n])
            if record_objective:
                objective.append(fit_explicit(X, H, lam)[0])
        eps, _ = fit_identity(alpha, M, Hhat, S, G[N - 1], lam)
        if alg == "nes" and nes_accel:
            # outer acceleration (Eq. nesouterupd) from the second iteration
            # on, with s_i = i^(1/N) (i = 1-based outer iteration); accepted
            # only if the candidate's error is strictly lower
            if H_prev is not None:
                s_i = (it + 1) ** (1.0 / N)
                Hc, lamc = nes_extrapolate(H, lam, H_prev, lam_prev, s_i)
                eps_c = model_error(X, Hc, lamc, alpha)
                ok = eps_c < eps
                accepted.append(bool(ok))
                if ok:
                    H, lam, eps = Hc, lamc, eps_c
                    G = [gram(h) for h in H]
            H_prev = [h.copy() for h in H]
            lam_prev = lam.copy()
        rel_err.append(eps)
        if tol is not None and eps <= tol:
            break
    out = dict(H=H, lam=lam, rel_err=rel_err, inner=inner, alpha=alpha,
               accepted=accepted)
    if record_objective:
        out["objective"] = objective
    return out


# ----------------------------------------------------------------------------
# CP reconstruction loss and its gradient (the adjoint of the CP model)
# ----------------------------------------------------------------------------


def cp_loss(X, H) -> float:
    """f(H) = ||X - [[H^(1), ..., H^(N)]]||^2  (Eq. nncp objective)."""
    D = np.asarray(X, dtype=np.float64) - cp_full(H)
    return float(np.sum(D * D))


def cp_loss_grad(X, H):
    """Gradient of f: df/dH^(n) = 2 (H^(n) S^(n) - M^(n)), the MTTKRP and
    Hadamard-of-Grams matrices of Alg. 1 (Sec. 4.3, Eq. nls)."""
    G = [gram(h) for h in H]
    return [2.0 * (H[n] @ gram_hadamard(G, n) - mttkrp(X, H, n))
            for n in range(len(H))]
