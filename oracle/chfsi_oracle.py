"""Oracle for Chebyshev-filtered subspace iteration with locking (Algorithm 1).

TEST INFRASTRUCTURE ONLY.  This module is a plain, slow, FP64 CPU restatement of the
method of Di Napoli & Berljafa, "Block iterative eigensolvers for sequences of correlated
eigenvalue problems" (arXiv:1206.3768).  Only the tests, the package smoke check and the
CPU-baseline leg of the benchmark may import it; the GPU library never does, and it
shares no code with the GPU library.

Two parts:

* The *definition* (``definition_eigenpairs``): the nev lowest eigenpairs of the pencil
  A x = lam B x with B-orthonormal eigenvectors (Eq. 1, Section 1), via LAPACK.
* The *algorithm* (``chfsi_solve``): reduction to standard form (Section 3.2), a
  Lanczos upper bound, the Chebyshev filter, re-orthonormalisation, Rayleigh-Ritz and
  contiguous-prefix locking, in the order of Algorithm 1.  Where the paper leaves a step
  unspecified, each function names the reading it implements (readings R1-R14 below).

Readings of points the paper leaves open (same numbering in the design notes):
  R1  The loop repeats while fewer than nev pairs are locked (Algorithm 1 prints the
      stopping test inverted).
  R2  "converged" counts locked columns; the active block keeps the unlocked columns,
      so its width is blk - converged (nkeep = blk - nconv, Table 3).
  R3  Locked pairs are frozen; the active block is deflated against them (two passes of
      classical Gram-Schmidt) before re-orthonormalisation and Rayleigh-Ritz runs on the
      active block only.
  R4  The filter is the scaled three-term Chebyshev recurrence on [a, b] normalised at
      a0 (Zhou & Saad 2007), with a the largest Ritz value of the block (standing in for
      lambda_{blk+1}), a0 the smallest, and b the Lanczos upper bound.
  R5  lanczos-iter "10 : 3 x blk" (Table 3) is a range; k steps with full
      re-orthogonalisation, bound b = max eig(T_k) + |beta_k|.
  R6  Warm start: a0 = lambda_1 and a = theta_blk of the previous problem.  Cold start:
      one Rayleigh-Ritz on the start block, then a0 = theta_1 and
      a = theta_1 + (b - theta_1) * blk / n.
  R7  Locking test: standard residual ||Hs y - theta y|| / ||y|| < tau with
      tau = tol * max(|a0|, |b|) / 4 (absolute residuals scaled by the norm estimate, as the
      footnote of Section 3.3 allows).  Acceptance: the generalized residual
      ||A x - lam B x|| / (||A||_est ||x||) <= tol for every output pair; otherwise tau is
      divided by 10, all pairs are unlocked, and iteration continues (at most 3 times).
  R8  Adaptive degree (not in the paper): d_i = clamp(ceil(ln(r_i / tau) / ln rho_i),
      dmin, dmax), rho_i = |t_i| + sqrt(t_i^2 - 1), t_i = (theta_i - c) / e; columns
      past the nev-th use the largest degree of the wanted active columns.  The first
      adaptive loop needs residuals: after a cold start one Rayleigh-Ritz on the start
      block gives them; after a warm start they are the residuals of the carried vectors
      at their Rayleigh quotients, with the bounds from the carried Ritz values.
  R9  Conjugate transposes everywhere the paper writes transposes (complex data).
  R10 Only the lower triangles of A and B are referenced.
  R11 Warm vectors travel in x-coordinates and are mapped by the new L^H (identical to
      the paper's use of y when B is fixed).
  R12 Start vector of Lanczos and the cold-start block come from the counter-based
      SplitMix64 generator (Steele, Lea & Flood 2014) so that independent
      implementations draw identical numbers.

Parity status: every function below is pinned by tests against closed forms,
invariants or LAPACK definitions; none is marked "parity unpinned".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

# --------------------------------------------------------------------------------------
# Counter-based generator (reading R12).  SplitMix64: Steele, Lea & Flood, "Fast
# splittable pseudorandom number generators", OOPSLA 2014.
# --------------------------------------------------------------------------------------
_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """Output number index+1 of SplitMix64 started from state ``seed`` (uint64 array)."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + (idx + np.uint64(1)) * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, index: np.ndarray) -> np.ndarray:
    """53-bit uniform doubles in [0, 1) from SplitMix64 outputs."""
    z = splitmix64(seed, index)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def lanczos_start_vector(n: int, seed: int) -> np.ndarray:
    """v_j = (u_{2j} - 1/2) + i (u_{2j+1} - 1/2) (reading R12)."""
    j = np.arange(n, dtype=np.uint64)
    re = uniform01(seed, 2 * j) - 0.5
    im = uniform01(seed, 2 * j + 1) - 0.5
    return re + 1j * im


def cold_start_block(n: int, m: int, seed: int) -> np.ndarray:
    """Complex Gaussian n x m block by Box-Muller over SplitMix64 (column-major index)."""
    t = np.arange(n * m, dtype=np.uint64)
    u1 = uniform01(seed, 2 * t)
    u2 = uniform01(seed, 2 * t + 1)
    r = np.sqrt(-2.0 * np.log1p(-u1))
    z = (r * np.cos(2.0 * math.pi * u2) + 1j * r * np.sin(2.0 * math.pi * u2)) / math.sqrt(2.0)
    return z.reshape(m, n).T.copy()


# --------------------------------------------------------------------------------------
# Definition (Eq. 1): lowest nev eigenpairs of A x = lam B x, B-orthonormal x.
# --------------------------------------------------------------------------------------
def hermitian_from_lower(M: np.ndarray) -> np.ndarray:
    """Full Hermitian matrix from the lower triangle of M (reading R10)."""
    low = np.tril(M, -1)
    return low + low.conj().T + np.diag(np.real(np.diag(M)))


def definition_eigenpairs(A: np.ndarray, B: np.ndarray, nev: int):
    """LAPACK (zhegvx/zhegvr class) solution of the pencil: ascending values, X^H B X = I."""
    w, X = sla.eigh(hermitian_from_lower(A), hermitian_from_lower(B), lower=True,
                    subset_by_index=[0, nev - 1])
    return w, X


# --------------------------------------------------------------------------------------
# Reduction to standard form (Section 3.2): B = L L^H, Hs = L^{-1} A L^{-H}, y = L^H x.
# --------------------------------------------------------------------------------------
def cholesky_lower(B: np.ndarray) -> np.ndarray:
    return np.linalg.cholesky(hermitian_from_lower(B))


def reduce_standard(A: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Hs = L^{-1} A L^{-H}, made exactly Hermitian."""
    Af = hermitian_from_lower(A)
    M = sla.solve_triangular(L, Af, lower=True)            # L^{-1} A
    Hs = sla.solve_triangular(L, M.conj().T, lower=True)   # L^{-1} (L^{-1} A)^H
    return 0.5 * (Hs + Hs.conj().T)


def to_standard_vectors(L: np.ndarray, X: np.ndarray) -> np.ndarray:
    """y = L^H x."""
    return L.conj().T @ X


def to_generalized_vectors(L: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """x = L^{-H} y."""
    return sla.solve_triangular(L.conj().T, Y, lower=False)


# --------------------------------------------------------------------------------------
# Lanczos upper bound (Algorithm 1, first step; reading R5).
# --------------------------------------------------------------------------------------
def lanczos(H: np.ndarray, v0: np.ndarray, k: int):
    """k-step Lanczos with full re-orthogonalisation.

    Returns (upper, theta_min, alpha, beta): upper = max eig(T_k) + |beta_k| is the safe
    upper bound of the spectrum used by the filter; theta_min = min eig(T_k).
    """
    n = H.shape[0]
    k = min(k, n)
    V = np.zeros((n, k), dtype=np.complex128)
    alpha = np.zeros(k)
    beta = np.zeros(k)
    v = v0 / np.linalg.norm(v0)
    v_prev = np.zeros(n, dtype=np.complex128)
    b_prev = 0.0
    steps = k
    for j in range(k):
        V[:, j] = v
        w = H @ v
        alpha[j] = np.real(np.vdot(v, w))
        w = w - alpha[j] * v - b_prev * v_prev
        w = w - V[:, : j + 1] @ (V[:, : j + 1].conj().T @ w)
        beta[j] = np.linalg.norm(w)
        if beta[j] == 0.0:
            steps = j + 1
            break
        v_prev, v, b_prev = v, w / beta[j], beta[j]
    a = alpha[:steps]
    off = beta[: steps - 1]
    theta = sla.eigvalsh_tridiagonal(a, off) if steps > 1 else a.copy()
    return float(theta[-1] + abs(beta[steps - 1])), float(theta[0]), a, beta[:steps]


# --------------------------------------------------------------------------------------
# Chebyshev filter (Algorithm 1, filtering step; reading R4).
# --------------------------------------------------------------------------------------
def filter_coefficients(a0: float, a: float, b: float, dmax: int):
    """Per-step (alpha_k, beta_k, gamma_k) of Y_k = alpha_k H Y_{k-1} + beta_k Y_{k-1} + gamma_k Y_{k-2}.

    e = (b - a)/2, c = (b + a)/2, sigma_1 = e / (a0 - c),
    k = 1:  Y_1 = (sigma_1 / e)(H - c I) Y_0
    k >= 2: sigma_k = 1 / (2/sigma_1 - sigma_{k-1}),
            Y_k = (2 sigma_k / e)(H - c I) Y_{k-1} - sigma_{k-1} sigma_k Y_{k-2}
    """
    e = 0.5 * (b - a)
    c = 0.5 * (b + a)
    s1 = e / (a0 - c)
    coef = []
    s = s1
    for k in range(1, dmax + 1):
        if k == 1:
            al = s1 / e
            coef.append((al, -al * c, 0.0))
        else:
            s_new = 1.0 / (2.0 / s1 - s)
            al = 2.0 * s_new / e
            coef.append((al, -al * c, -s * s_new))
            s = s_new
    return coef


def chebyshev_filter(H: np.ndarray, X: np.ndarray, degrees, a0: float, a: float, b: float):
    """Column i of the result is p_{d_i}(H) X[:, i] with p_d(t) = T_d((t-c)/e) / T_d((a0-c)/e)."""
    degrees = np.asarray(degrees, dtype=np.int64)
    out = X.copy()
    dmax = int(degrees.max(initial=0))
    if dmax == 0:
        return out
    coef = filter_coefficients(a0, a, b, dmax)
    Yprev = X.copy()
    Ycur = X.copy()
    for k in range(1, dmax + 1):
        act = degrees >= k
        al, be, ga = coef[k - 1]
        Yn = al * (H @ Ycur[:, act]) + be * Ycur[:, act] + ga * Yprev[:, act]
        Yprev[:, act] = Ycur[:, act]
        Ycur[:, act] = Yn
        done = degrees == k
        out[:, done] = Ycur[:, done]
    return out


def chebyshev_T(d: int, t: np.ndarray) -> np.ndarray:
    """Closed form of the Chebyshev polynomial: cos(d acos t) on [-1,1], cosh outside."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1.0
    out[inside] = np.cos(d * np.arccos(t[inside]))
    hi = t > 1.0
    out[hi] = np.cosh(d * np.arccosh(t[hi]))
    lo = t < -1.0
    out[lo] = (-1.0) ** d * np.cosh(d * np.arccosh(-t[lo]))
    return out


# --------------------------------------------------------------------------------------
# Re-orthonormalisation (Algorithm 1; reading R3): CGS2 against the locked block, then
# Householder QR (the GPU path uses Cholesky QR; the spans agree).
# --------------------------------------------------------------------------------------
def orthonormalize(Y: np.ndarray, YL: np.ndarray | None = None) -> np.ndarray:
    Z = Y.copy()
    if YL is not None and YL.shape[1] > 0:
        for _ in range(2):
            Z = Z - YL @ (YL.conj().T @ Z)
    Q, _ = np.linalg.qr(Z)
    return Q


# --------------------------------------------------------------------------------------
# Rayleigh-Ritz (Algorithm 1) and residuals (deflation & locking test).
# --------------------------------------------------------------------------------------
def rayleigh_ritz(H: np.ndarray, Q: np.ndarray):
    """G = Q^H H Q; G w = theta w (ascending); returns (theta, Q W, (H Q) W)."""
    W = H @ Q
    G = Q.conj().T @ W
    G = 0.5 * (G + G.conj().T)
    theta, S = np.linalg.eigh(G)
    return theta, Q @ S, W @ S


def residual_norms(HY: np.ndarray, Y: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """r_i = ||H y_i - theta_i y_i|| / ||y_i||."""
    R = HY - Y * theta[None, :]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(Y, axis=0)


def lock_count(r: np.ndarray, tau: float, converged: int, nev: int) -> int:
    """Length of the leading run of r_i < tau among the first nev - converged columns."""
    cnt = 0
    for i in range(min(r.size, nev - converged)):
        if r[i] < tau:
            cnt += 1
        else:
            break
    return cnt


def adaptive_degrees(theta, r, a: float, b: float, tau: float, dmin: int, dmax: int,
                     n_wanted: int) -> np.ndarray:
    """Closed-form per-vector degree (reading R8)."""
    theta = np.asarray(theta, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    e = 0.5 * (b - a)
    c = 0.5 * (b + a)
    d = np.full(theta.size, dmax, dtype=np.int64)
    for i in range(theta.size):
        if r[i] <= tau:
            d[i] = dmin
            continue
        t = abs((theta[i] - c) / e)
        if t <= 1.0:
            d[i] = dmax
            continue
        rho = t + math.sqrt(t * t - 1.0)
        need = math.log(r[i] / tau) / math.log(rho)
        if not math.isfinite(need) or need >= dmax:
            d[i] = dmax
        else:
            d[i] = min(dmax, max(dmin, int(math.ceil(need))))
    if n_wanted < theta.size:
        top = int(d[:n_wanted].max()) if n_wanted > 0 else dmin
        d[n_wanted:] = top
    return d


# --------------------------------------------------------------------------------------
# Full solve of one problem, and of a sequence with warm starts.
# --------------------------------------------------------------------------------------
@dataclass
class SolveStats:
    loops: int = 0
    filtered_vectors: int = 0
    matvecs: int = 0
    locked_per_loop: list = field(default_factory=list)
    max_resid: float = float("nan")
    accept_rounds: int = 0
    lanczos_upper: float = float("nan")


@dataclass
class WarmState:
    X: np.ndarray          # n x blk Ritz vectors in x-coordinates (reading R11)
    lam: np.ndarray        # blk Ritz values ascending


def matrix_norm_estimate(M: np.ndarray, seed: int, k: int = 20) -> float:
    """max |Ritz value| of a k-step Lanczos run on M (a lower estimate of ||M||_2)."""
    v0 = lanczos_start_vector(M.shape[0], seed ^ 0x5A5A5A5A)
    up, tmin, a, bta = lanczos(M, v0, k)
    n = a.size
    theta = sla.eigvalsh_tridiagonal(a, bta[: n - 1]) if n > 1 else a
    return float(max(abs(theta[0]), abs(theta[-1])))


def generalized_residuals(A: np.ndarray, B: np.ndarray, X: np.ndarray, lam: np.ndarray,
                          a_norm: float) -> np.ndarray:
    """||A x_i - lam_i B x_i|| / (a_norm ||x_i||)."""
    R = A @ X - (B @ X) * lam[None, :]
    return np.linalg.norm(R, axis=0) / (a_norm * np.linalg.norm(X, axis=0))


def chfsi_solve(A, B, nev: int, blk: int, tol: float = 1e-10, deg: int = 25,
                deg_min: int = 8, deg_max: int = 25, warm: WarmState | None = None,
                V0: np.ndarray | None = None, seed: int = 12063768,
                lanczos_k_warm: int = 10, lanczos_k_cold: int = 40, max_loops: int = 50):
    """Algorithm 1 for the pencil (A, B): returns (lam[nev], X[n, nev], WarmState, SolveStats).

    deg > 0 fixes the filter degree; deg == 0 selects the adaptive rule of reading R8.
    """
    steps = chfsi_solve_loops(A, B, nev, blk, tol, deg, deg_min, deg_max, warm, V0, seed,
                              lanczos_k_warm, lanczos_k_cold, max_loops)
    while True:
        try:
            next(steps)
        except StopIteration as done:
            return done.value


def chfsi_solve_loops(A, B, nev: int, blk: int, tol: float = 1e-10, deg: int = 25,
                      deg_min: int = 8, deg_max: int = 25, warm: WarmState | None = None,
                      V0: np.ndarray | None = None, seed: int = 12063768,
                      lanczos_k_warm: int = 10, lanczos_k_cold: int = 40, max_loops: int = 50):
    """The same computation as chfsi_solve, as a generator that pauses after every filter loop
    (yielding the number of pairs that loop locked) and returns chfsi_solve's result when it
    finishes (the value of StopIteration), so that a caller can time the work loop by loop."""
    n = A.shape[0]
    if not (0 < nev <= blk <= n):
        raise ValueError("need 0 < nev <= blk <= n")
    st = SolveStats()
    Af = hermitian_from_lower(A)
    Bf = hermitian_from_lower(B)
    L = np.linalg.cholesky(Bf)
    H = reduce_standard(A, L)

    is_warm = warm is not None
    k = lanczos_k_warm if is_warm else lanczos_k_cold
    b_up, _, _, _ = lanczos(H, lanczos_start_vector(n, seed), k)
    st.lanczos_upper = b_up
    st.matvecs += min(k, n)

    if is_warm:
        Y = to_standard_vectors(L, warm.X)
    elif V0 is not None:
        Y = np.array(V0, dtype=np.complex128)
    else:
        Y = cold_start_block(n, blk, seed + 1)

    adaptive = deg == 0
    r = None
    if is_warm and adaptive:
        # Reading R8: the residuals the first adaptive loop needs are those of the carried
        # vectors at their Rayleigh quotients; the bounds come from the carried Ritz values.
        W = H @ Y
        theta = np.real(np.sum(Y.conj() * W, axis=0)) / np.real(np.sum(Y.conj() * Y, axis=0))
        r = residual_norms(W, Y, theta)
        st.matvecs += blk
        a0 = float(warm.lam[0])
        a = float(warm.lam[-1])
    elif not is_warm:
        Q = orthonormalize(Y)
        theta, Y, W = rayleigh_ritz(H, Q)
        r = residual_norms(W, Y, theta)
        st.matvecs += blk
        a0 = float(theta[0])
        a = a0 + (b_up - a0) * blk / n
    else:
        theta = np.array(warm.lam, dtype=np.float64)
        a0 = float(theta[0])
        a = float(theta[-1])
    tau = 0.25 * tol * max(abs(a0), abs(b_up))

    a_norm = matrix_norm_estimate(Af, seed)
    YL = np.zeros((n, 0), dtype=np.complex128)
    lamL = np.zeros(0)
    rL = np.zeros(0)
    converged = 0
    for _accept in range(4):
        while converged < nev and st.loops < max_loops:
            m = blk - converged
            if adaptive:
                d = adaptive_degrees(theta, r, a, b_up, tau, deg_min, deg_max, nev - converged)
            else:
                d = np.full(m, deg, dtype=np.int64)
            Y = chebyshev_filter(H, Y, d, a0, a, b_up)
            st.matvecs += int(d.sum())
            st.filtered_vectors += m
            Q = orthonormalize(Y, YL)
            theta, Y, W = rayleigh_ritz(H, Q)
            st.matvecs += m
            r = residual_norms(W, Y, theta)
            nl = lock_count(r, tau, converged, nev)
            st.loops += 1
            st.locked_per_loop.append(nl)
            yield nl
            if nl:
                YL = np.concatenate([YL, Y[:, :nl]], axis=1)
                lamL = np.concatenate([lamL, theta[:nl]])
                rL = np.concatenate([rL, r[:nl]])
                Y, theta, r = Y[:, nl:], theta[nl:], r[nl:]
                converged += nl
            a0 = float(theta[0])
            a = float(theta[-1])
        if converged < nev:
            break
        X = to_generalized_vectors(L, YL)
        gres = generalized_residuals(Af, Bf, X, lamL, a_norm)
        st.max_resid = float(gres.max())
        if st.max_resid <= tol or _accept == 3:
            break
        # Reading R7: tighten the locking threshold and iterate on all blk columns.
        st.accept_rounds += 1
        tau /= 10.0
        Y = np.concatenate([YL, Y], axis=1)
        theta = np.concatenate([lamL, theta])
        r = np.concatenate([rL, r])
        YL = np.zeros((n, 0), dtype=np.complex128)
        lamL, rL = np.zeros(0), np.zeros(0)
        converged = 0
        a0, a = float(theta[0]), float(theta[-1])

    Yall = np.concatenate([YL, Y], axis=1)
    lam_all = np.concatenate([lamL, theta])
    Xall = to_generalized_vectors(L, Yall)
    state = WarmState(X=Xall, lam=lam_all)
    lam = np.full(nev, np.nan)
    lam[:converged] = lamL[:nev]
    X = Xall[:, :nev]
    if converged >= nev and not math.isfinite(st.max_resid):
        st.max_resid = float(generalized_residuals(Af, Bf, X, lam, a_norm).max())
    return lam, X, state, st


def chfsi_solve_sequence(As, Bs, nev: int, blk: int, tol: float = 1e-10, deg: int = 25,
                         deg_min: int = 8, deg_max: int = 25, V0=None, seed: int = 12063768,
                         **kw):
    """Solve problems in order, each warm-started from the previous one's Ritz vectors."""
    warm = None
    out = []
    for ell, (A, B) in enumerate(zip(As, Bs)):
        lam, X, warm, st = chfsi_solve(A, B, nev, blk, tol, deg, deg_min, deg_max,
                                       warm=warm, V0=V0 if ell == 0 else None,
                                       seed=seed, **kw)
        out.append((lam, X, st))
    return out


# --------------------------------------------------------------------------------------
# Deviation angles between eigenvectors of adjacent problems (Section 2.2, the relation
# for the scalar products <x_i^(l) x_j^(l+1)> and the angles theta_i^(l) of Fig. 1).
# --------------------------------------------------------------------------------------
def scalar_products(X_prev: np.ndarray, X_cur: np.ndarray, B: np.ndarray) -> np.ndarray:
    """M_ij = <x_i^(l) x_j^(l+1)>.  With the Cholesky factor L of a fixed B the paper's
    product c^(l)H L L^H c^(l+1) is the B-inner product x_i^H B x_j."""
    return X_prev.conj().T @ (B @ X_cur)


def associate(M: np.ndarray) -> np.ndarray:
    """One-to-one association of previous to current eigenvectors from the dominant
    entries of |M| (Section 2.2): repeatedly take the largest |M_ij| among unassigned
    rows and columns (ties: smallest row, then smallest column).  Returns assoc with
    assoc[i] = j, the current vector matched to previous vector i."""
    A = np.abs(M).astype(np.float64)
    k = A.shape[0]
    assoc = np.full(k, -1, dtype=np.int64)
    free_r = np.ones(k, dtype=bool)
    free_c = np.ones(k, dtype=bool)
    for _ in range(k):
        best, bi, bj = -1.0, -1, -1
        for i in range(k):
            if not free_r[i]:
                continue
            for j in range(k):
                if free_c[j] and A[i, j] > best:
                    best, bi, bj = A[i, j], i, j
        assoc[bi] = bj
        free_r[bi] = False
        free_c[bj] = False
    return assoc


def deviation_angles(X_prev: np.ndarray, X_cur: np.ndarray, B: np.ndarray):
    """theta_i = angle between x_i^(l) and its associated x_assoc(i)^(l+1) in the B-inner
    product (B-normalised columns), computed as asin of the B-norm of the component of
    x_assoc(i) orthogonal to x_i, so that small angles keep full relative accuracy.
    Returns (theta, assoc)."""
    M = scalar_products(X_prev, X_cur, B)
    assoc = associate(M)
    k = M.shape[0]
    theta = np.empty(k)
    for i in range(k):
        xp = X_prev[:, i]
        xc = X_cur[:, assoc[i]]
        npv = math.sqrt(max(np.real(np.vdot(xp, B @ xp)), 0.0))
        ncv = math.sqrt(max(np.real(np.vdot(xc, B @ xc)), 0.0))
        up, uc = xp / npv, xc / ncv
        r = uc - up * np.vdot(up, B @ uc)
        s = math.sqrt(max(np.real(np.vdot(r, B @ r)), 0.0))
        theta[i] = math.asin(min(1.0, s))
    return theta, assoc
