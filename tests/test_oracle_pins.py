"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than itself: a closed
form, an invariant, a LAPACK definition, a planted answer or a published test vector.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import torch

import oracle.chfsi_oracle as O
from paper_1206_3768_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_problem(n=96, nev=8, blk=14, name="c1", N=1, spectrum=None, seed_offset=0):
    seq = inputs.planted_sequence(name, n=n, N=N, nev=nev, blk=blk, spectrum=spectrum,
                                  seed_offset=seed_offset)
    return seq


def _np(t):
    return t.numpy() if isinstance(t, torch.Tensor) else t


# ---------------------------------------------------------------- generator (R12)
def test_splitmix64_published_outputs():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    got = O.splitmix64(0, np.arange(4, dtype=np.uint64))
    assert [int(x) for x in got] == want


def test_uniform_and_gaussian_moments():
    u = O.uniform01(123, np.arange(200000, dtype=np.uint64))
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1.0 / 12.0) < 2e-3
    z = O.cold_start_block(400, 50, 7)
    assert z.shape == (400, 50)
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.02
    assert abs(np.mean(z)) < 0.02


# ---------------------------------------------------------------- definition (Eq. 1)
def test_definition_matches_planted_spectrum():
    seq = _small_problem()
    p = seq.problems[0]
    A, B = _np(p.A), _np(p.B)
    w, X = O.definition_eigenpairs(np.tril(A), np.tril(B), 8)
    scale = np.max(np.abs(p.lam))
    assert np.max(np.abs(w - p.lam[:8])) <= 1e-12 * scale
    assert np.allclose(X.conj().T @ B @ X, np.eye(8), atol=1e-12)
    # Planted vectors agree up to phase (isolated eigenvalues of the draw).
    Xp = _np(p.X)[:, :8]
    ov = np.abs(np.sum(X.conj() * (B @ Xp), axis=0))
    assert np.all(np.abs(ov - 1.0) < 1e-8)


def test_hermitian_from_lower_uses_lower_triangle_only():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    H = O.hermitian_from_lower(M)
    assert np.allclose(H, H.conj().T)
    assert np.allclose(np.tril(H, -1), np.tril(M, -1))
    M2 = M.copy()
    M2[np.triu_indices(5, 1)] = 99.0
    assert np.allclose(O.hermitian_from_lower(M2), H)


# ---------------------------------------------------------------- reduction (Section 3.2)
def test_reduction_invariants_and_planted_spectrum():
    seq = _small_problem(n=80)
    p = seq.problems[0]
    A, B = _np(p.A), _np(p.B)
    L = O.cholesky_lower(np.tril(B))
    assert np.allclose(np.triu(L, 1), 0.0)
    assert np.linalg.norm(L @ L.conj().T - B) <= 1e-14 * np.linalg.norm(B)
    Hs = O.reduce_standard(np.tril(A), L)
    assert np.linalg.norm(L @ Hs @ L.conj().T - A) <= 1e-13 * np.linalg.norm(A)
    assert np.max(np.abs(np.linalg.eigvalsh(Hs) - p.lam)) <= 1e-12 * np.max(np.abs(p.lam))
    # y = L^H x maps B-orthonormal x to orthonormal y and back.
    X = _np(p.X)[:, :5]
    Y = O.to_standard_vectors(L, X)
    assert np.allclose(Y.conj().T @ Y, np.eye(5), atol=1e-12)
    assert np.allclose(O.to_generalized_vectors(L, Y), X, atol=1e-12)


# ---------------------------------------------------------------- Chebyshev filter
def _diag_case(n=60, seed=3):
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.uniform(-2.0, 2.0, n))
    Z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Q, _ = np.linalg.qr(Z)
    H = (Q * lam) @ Q.conj().T
    return lam, Q, 0.5 * (H + H.conj().T)


@pytest.mark.parametrize("d", [1, 2, 3, 7, 10, 25, 40])
def test_filter_on_eigenvectors_matches_closed_form(d):
    lam, Q, H = _diag_case()
    a0, a, b = lam[0], lam[12], lam[-1] + 0.05
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    X = Q[:, :20]
    Y = O.chebyshev_filter(H, X, np.full(20, d), a0, a, b)
    p = O.chebyshev_T(d, (lam[:20] - c) / e) / O.chebyshev_T(d, np.array([(a0 - c) / e]))[0]
    ref = X * p[None, :]
    assert np.max(np.abs(Y - ref)) <= 1e-12 * max(1.0, np.max(np.abs(p)))
    # normalisation point: p(a0) = 1
    assert abs(p[0] - 1.0) < 1e-12


def test_filter_per_column_degrees():
    lam, Q, H = _diag_case()
    a0, a, b = lam[0], lam[15], lam[-1] + 0.1
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    degs = np.array([0, 1, 5, 9, 9, 3, 12, 2])
    X = Q[:, :8] * (1.0 + 0.5j)
    Y = O.chebyshev_filter(H, X, degs, a0, a, b)
    t0 = (a0 - c) / e
    for i, d in enumerate(degs):
        p = 1.0 if d == 0 else (O.chebyshev_T(d, np.array([(lam[i] - c) / e]))[0]
                                / O.chebyshev_T(d, np.array([t0]))[0])
        assert np.max(np.abs(Y[:, i] - p * X[:, i])) <= 1e-12 * max(1, abs(p))


def test_chebyshev_closed_form_trig_identity():
    th = np.linspace(0.0, math.pi, 41)
    for k in (0, 1, 2, 5, 13):
        assert np.allclose(O.chebyshev_T(k, np.cos(th)), np.cos(k * th), atol=1e-13)
    # three-term recurrence outside [-1, 1]
    x = np.array([-3.0, -1.5, 1.2, 4.0])
    T0, T1 = np.ones_like(x), x.copy()
    for k in range(2, 12):
        T0, T1 = T1, 2 * x * T1 - T0
        assert np.allclose(O.chebyshev_T(k, x), T1, rtol=1e-12)


def test_filter_mutation_is_caught(monkeypatch):
    """A sign slip in the recurrence must fail the closed-form pin."""
    lam, Q, H = _diag_case()
    a0, a, b = lam[0], lam[12], lam[-1] + 0.05
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    real = O.filter_coefficients

    def broken(*args):
        return [(al, be, -ga) for (al, be, ga) in real(*args)]

    monkeypatch.setattr(O, "filter_coefficients", broken)
    Y = O.chebyshev_filter(H, Q[:, :5], np.full(5, 6), a0, a, b)
    p = O.chebyshev_T(6, (lam[:5] - c) / e) / O.chebyshev_T(6, np.array([(a0 - c) / e]))[0]
    assert np.max(np.abs(Y - Q[:, :5] * p)) > 1e-3


# ---------------------------------------------------------------- Lanczos (R5)
def test_lanczos_bound_is_safe_and_exact_at_full_dimension():
    lam, Q, H = _diag_case(n=50)
    v0 = O.lanczos_start_vector(50, 99)
    up, tmin, a, bta = O.lanczos(H, v0, 10)
    assert up >= lam[-1] - 1e-12
    assert tmin >= lam[0] - 1e-12
    up_full, tmin_full, a, bta = O.lanczos(H, v0, 50)
    T = np.diag(a) + np.diag(bta[:-1], 1) + np.diag(bta[:-1], -1)
    th = np.linalg.eigvalsh(T)
    assert np.max(np.abs(th - lam)) < 1e-10
    assert abs(tmin_full - lam[0]) < 1e-10


# ---------------------------------------------------------------- re-orthonormalisation
def test_orthonormalize_span_and_deflation():
    rng = np.random.default_rng(5)
    n, m, k = 70, 9, 4
    YL, _ = np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))
    Y = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    Q = O.orthonormalize(Y, YL)
    assert np.allclose(Q.conj().T @ Q, np.eye(m), atol=1e-13)
    assert np.max(np.abs(YL.conj().T @ Q)) < 1e-13
    # span(Q) = span((I - P_L) Y)
    Z = Y - YL @ (YL.conj().T @ Y)
    Pz = Z @ np.linalg.pinv(Z)
    assert np.linalg.norm(Pz - Q @ Q.conj().T) < 1e-11


# ---------------------------------------------------------------- Rayleigh-Ritz, residuals
def test_rayleigh_ritz_on_invariant_subspace_is_exact():
    lam, Q, H = _diag_case(n=40)
    rng = np.random.default_rng(1)
    U, _ = np.linalg.qr(rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6)))
    S = Q[:, 3:9] @ U
    theta, Y, W = O.rayleigh_ritz(H, S)
    assert np.max(np.abs(theta - lam[3:9])) < 1e-13
    r = O.residual_norms(W, Y, theta)
    assert np.max(r) < 1e-13


def test_rayleigh_ritz_interlacing():
    lam, Q, H = _diag_case(n=40)
    rng = np.random.default_rng(2)
    S, _ = np.linalg.qr(rng.standard_normal((40, 7)) + 1j * rng.standard_normal((40, 7)))
    theta, Y, W = O.rayleigh_ritz(H, S)
    # Cauchy interlacing: lam_i <= theta_i <= lam_{n-m+i}
    assert np.all(theta >= lam[:7] - 1e-13)
    assert np.all(theta <= lam[-7:] + 1e-13)


def test_residual_closed_form_two_level():
    lam, Q, H = _diag_case(n=30)
    d = 1e-3
    y = (Q[:, 0] + d * Q[:, 5])[:, None]
    theta = np.array([lam[0]])
    r = O.residual_norms(H @ y, y, theta)
    assert abs(r[0] - d * abs(lam[5] - lam[0]) / math.sqrt(1 + d * d)) < 1e-14


# ---------------------------------------------------------------- locking (Algorithm 1)
def test_lock_count_contiguous_prefix():
    r = np.array([1e-12, 1e-13, 5e-9, 1e-14, 1e-14])
    assert O.lock_count(r, 1e-10, 0, 10) == 2
    assert O.lock_count(r, 1e-10, 9, 10) == 1          # only nev - converged allowed
    assert O.lock_count(r, 1e-8, 0, 10) == 5
    assert O.lock_count(np.array([1.0]), 1e-10, 0, 5) == 0


# ---------------------------------------------------------------- degree rule (R8)
def test_adaptive_degree_bounds_from_closed_form():
    a, b = -0.5, 10.0
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    theta = np.array([-1.0, -0.9, -0.7, -0.55, 3.0, -0.95])
    r = np.array([1e-3, 1e-5, 1e-2, 1e-4, 1e-1, 1e-12])
    tau = 1e-10
    d = O.adaptive_degrees(theta, r, a, b, tau, 4, 60, 5)
    assert d[5] == 60  # past the wanted columns: largest wanted degree
    assert d[4] == 60  # inside [a, b]: no damping, maximum degree
    for i in range(4):
        t = abs((theta[i] - c) / e)
        if 4 < d[i] < 60:
            # T_d(t) >= rho^d / 2 >= r/(2 tau) and T_{d-1}(t) <= rho^{d-1} < r/tau
            assert O.chebyshev_T(int(d[i]), np.array([t]))[0] >= r[i] / (2 * tau)
            assert O.chebyshev_T(int(d[i]) - 1, np.array([t]))[0] < r[i] / tau
    d2 = O.adaptive_degrees(np.array([-1.0]), np.array([1e-12]), a, b, 1e-10, 8, 25, 1)
    assert d2[0] == 8


def test_filter_reduces_residual_as_the_degree_rule_predicts():
    """Brute force on a planted spectrum: measured reduction vs 1/|T_d(t)| within 10x."""
    lam, Q, H = _diag_case(n=80, seed=11)
    a, b = lam[20], lam[-1] + 0.01
    a0 = lam[0]
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    i = 2
    rng = np.random.default_rng(4)
    coef = np.zeros(80, dtype=np.complex128)
    coef[i] = 1.0
    coef[21:] = 1e-4 * (rng.standard_normal(59) + 1j * rng.standard_normal(59))
    y = Q @ coef
    d = 12
    y2 = O.chebyshev_filter(H, y[:, None], [d], a0, a, b)[:, 0]

    def res(v):
        th = np.real(np.vdot(v, H @ v) / np.vdot(v, v))
        return np.linalg.norm(H @ v - th * v) / np.linalg.norm(v)

    measured = res(y2) / res(y)
    predicted = 1.0 / abs(O.chebyshev_T(d, np.array([(lam[i] - c) / e]))[0])
    assert predicted / 10 <= measured <= predicted * 10


# ---------------------------------------------------------------- full method
def _check_solution(p, lam, X, nev, tol=1e-10):
    A, B = _np(p.A), _np(p.B)
    a2 = np.linalg.norm(A, 2)
    scale = max(np.max(np.abs(p.lam)), 1.0)
    assert np.all(np.isfinite(lam))
    assert np.max(np.abs(lam - p.lam[:nev]) / np.maximum(np.abs(p.lam[:nev]), scale)) <= tol
    R = A @ X - (B @ X) * lam[None, :]
    res = np.linalg.norm(R, axis=0) / (a2 * np.linalg.norm(X, axis=0))
    assert res.max() <= tol
    assert np.allclose(X.conj().T @ B @ X, np.eye(nev), atol=1e-10)


def test_full_solve_small_c1_shape_fixed_degree():
    seq = _small_problem(n=192, nev=10, blk=16, N=3)
    As = [np.tril(_np(p.A)) for p in seq.problems]
    Bs = [np.tril(_np(p.B)) for p in seq.problems]
    out = O.chfsi_solve_sequence(As, Bs, 10, 16, 1e-10, deg=10)
    for p, (lam, X, st) in zip(seq.problems, out):
        _check_solution(p, lam, X, 10)
        assert st.loops < 50
        assert st.filtered_vectors >= 16


def test_full_solve_adaptive_ill_conditioned_overlap():
    seq = inputs.planted_sequence("c2", n=260, N=2, nev=10, blk=14)
    As = [np.tril(_np(p.A)) for p in seq.problems]
    Bs = [np.tril(_np(p.B)) for p in seq.problems]
    assert np.linalg.cond(_np(seq.problems[0].B)) > 5e3
    out = O.chfsi_solve_sequence(As, Bs, 10, 14, 1e-10, deg=0, deg_min=8, deg_max=25)
    for p, (lam, X, st) in zip(seq.problems, out):
        _check_solution(p, lam, X, 10)


def test_clustered_wanted_eigenvalues_projector():
    seq = _small_problem(n=160, nev=12, blk=20, spectrum="cluster_low")
    p = seq.problems[0]
    lam, X, state, st = O.chfsi_solve(np.tril(_np(p.A)), np.tril(_np(p.B)), 12, 20, deg=12)
    _check_solution(p, lam, X, 12)
    # The cluster of 8 values near -2 is resolved as a subspace (Davis-Kahan).
    B = _np(p.B)
    Xp = _np(p.X)[:, :12]
    P1 = X @ X.conj().T @ B
    P2 = Xp @ Xp.conj().T @ B
    assert np.linalg.norm(P1 - P2) < 1e-6


def test_warm_start_needs_fewer_matvecs_than_cold():
    seq = _small_problem(n=256, nev=12, blk=20, N=4)
    As = [np.tril(_np(p.A)) for p in seq.problems]
    Bs = [np.tril(_np(p.B)) for p in seq.problems]
    _, _, warm, _ = O.chfsi_solve(As[2], Bs[2], 12, 20, deg=10)
    _, _, _, st_w = O.chfsi_solve(As[3], Bs[3], 12, 20, deg=10, warm=warm)
    _, _, _, st_c = O.chfsi_solve(As[3], Bs[3], 12, 20, deg=10)
    assert st_w.matvecs < st_c.matvecs
    assert st_w.loops <= st_c.loops


def test_table3_defaults_golden():
    vals = {}
    for l in open(os.path.join(GOLDEN, "table3_parameters.txt")):
        if l.strip() and not l.startswith("#"):
            k, v = l.split()
            vals[k] = float(v)
    import inspect
    sig = inspect.signature(O.chfsi_solve)
    assert sig.parameters["deg"].default == vals["degree"]
    assert sig.parameters["tol"].default == vals["tol"]
    assert sig.parameters["lanczos_k_warm"].default == vals["lanczos_iter_min"]


# ---------------------------------------------------------------------------- deviation angles
def _bo_basis(rng, n, k, B):
    """k B-orthonormal columns (B-Gram-Schmidt via Cholesky of the Gram matrix)."""
    Z = (rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))) / np.sqrt(2)
    G = Z.conj().T @ B @ Z
    R = np.linalg.cholesky(G).conj().T
    return Z @ np.linalg.inv(R)


def test_deviation_angles_planted_rotations():
    """Columns rotated pairwise by known angles inside a B-orthonormal basis: the angles
    come back exactly and each vector is associated with its rotated self."""
    rng = np.random.default_rng(31)
    n, k = 60, 8
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    B = np.eye(n) + 0.05 * (G.conj().T @ G) / n
    X = _bo_basis(rng, n, k, B)
    phis = np.array([1e-1, 3e-3, 1e-5, 2e-8])
    Y = X.copy()
    for p, phi in enumerate(phis):
        a, b = 2 * p, 2 * p + 1
        c, s = math.cos(phi), math.sin(phi)
        Y[:, a] = c * X[:, a] + s * np.exp(0.3j) * X[:, b]
        Y[:, b] = -s * np.exp(-0.3j) * X[:, a] + c * X[:, b]
    theta, assoc = O.deviation_angles(X, Y, B)
    assert list(assoc) == list(range(k))
    expect = np.repeat(phis, 2)
    assert np.allclose(theta, expect, rtol=1e-9, atol=1e-15)


def test_deviation_angles_permutation_and_phases():
    """Reordered eigenvectors with arbitrary phases: zero angles, association = the
    permutation (the one-to-one matching of Section 2.2)."""
    rng = np.random.default_rng(32)
    n, k = 40, 6
    B = np.eye(n)
    X = _bo_basis(rng, n, k, B)
    perm = np.array([2, 0, 1, 5, 3, 4])
    Y = X[:, perm] * np.exp(1j * rng.uniform(0, 6, k))[None, :]
    theta, assoc = O.deviation_angles(X, Y, B)
    # previous vector i sits at position j of Y where perm[j] == i
    inv = np.argsort(perm)
    assert list(assoc) == list(inv)
    assert np.max(theta) < 1e-7


def test_deviation_angles_match_scipy_subspace_angles():
    """For single vectors the angle is scipy's principal angle between the spans."""
    rng = np.random.default_rng(33)
    n = 30
    B = np.eye(n)
    x = (rng.standard_normal((n, 1)) + 1j * rng.standard_normal((n, 1)))
    y = x + 0.2 * (rng.standard_normal((n, 1)) + 1j * rng.standard_normal((n, 1)))
    x /= np.linalg.norm(x)
    y /= np.linalg.norm(y)
    theta, _ = O.deviation_angles(x, y, B)
    assert abs(theta[0] - sla.subspace_angles(x, y)[0]) < 1e-12


def test_deviation_angles_decrease_along_planted_sequence():
    """On the planted sequences the angles shrink with the rotation scale eps_l (the
    trend of Fig. 1)."""
    seq = inputs.planted_sequence("c1", n=96, N=4, nev=6, blk=8, device="cpu")
    means = []
    for l in range(1, 4):
        P0, P1 = seq.problems[l - 1], seq.problems[l]
        th, _ = O.deviation_angles(P0.X.numpy()[:, :6], P1.X.numpy()[:, :6], P1.B.numpy())
        means.append(float(np.mean(th)))
    assert means[0] > means[1] > means[2]


def test_associate_is_greedy_not_optimal_assignment():
    """The association takes the largest remaining |M_ij| first (the reading of the
    one-to-one association of Section 2.2), which differs from the assignment of largest
    total weight: here greedy takes (0,0) and then (1,1), the optimum (0,1) and (1,0).
    Ties go to the smallest row, then the smallest column."""
    M = np.array([[0.9, 0.8], [0.85, 0.1]])
    assert list(O.associate(M)) == [0, 1]
    from scipy.optimize import linear_sum_assignment

    r, c = linear_sum_assignment(-M)
    assert list(c) == [1, 0]  # the optimum differs
    # complex entries are compared by modulus; ties broken by position
    T = np.array([[1.0, 1j], [-1.0, 0.5]])
    assert list(O.associate(T)) == [0, 1]
    E = np.ones((3, 3))
    assert list(O.associate(E)) == [0, 1, 2]


def test_scalar_products_of_b_orthonormal_vectors():
    """M = X_prev^H B X_cur is the identity for a B-orthonormal basis against itself and
    the B-inner products of planted eigenvectors of two neighbouring problems are close to
    a permutation of phases (Section 2.2, Eq. 9 with a fixed B)."""
    rng = np.random.default_rng(34)
    n, k = 50, 7
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    B = np.eye(n) + 0.1 * (G.conj().T @ G) / n
    X = _bo_basis(rng, n, k, B)
    assert np.allclose(O.scalar_products(X, X, B), np.eye(k), atol=1e-12)
    # the order of the arguments matters: M(Y, X) = M(X, Y)^H
    Y = _bo_basis(rng, n, k, B)
    assert np.allclose(O.scalar_products(Y, X, B), O.scalar_products(X, Y, B).conj().T, atol=1e-13)
    seq = inputs.planted_sequence("c1", n=96, N=2, nev=6, blk=8, device="cpu")
    X0, X1, B1 = seq.problems[0].X.numpy()[:, :6], seq.problems[1].X.numpy()[:, :6], seq.problems[1].B.numpy()
    M = O.scalar_products(X0, X1, B1)
    assert np.all(np.abs(np.diag(M)) > 0.9)  # diagonally dominant (eps_1 = 5e-3 rotations)


def test_generalized_residuals_closed_form():
    """Diagonal pencil: exact eigenpairs give zero; a shifted eigenvalue lam_i + d gives
    |d| ||B e_i|| / (a_norm ||e_i||) = |d| b_i / a_norm; the columns' scale cancels."""
    n = 6
    lam = np.array([-3.0, -1.0, 0.5, 2.0, 4.0, 7.0])
    bdiag = np.array([1.0, 2.0, 0.5, 3.0, 1.5, 1.0])
    A = np.diag(lam * bdiag).astype(np.complex128)
    B = np.diag(bdiag).astype(np.complex128)
    X = np.eye(n, dtype=np.complex128)[:, :4] * np.array([1.0, 2.0, 1j, -3.0])[None, :]
    r = O.generalized_residuals(A, B, X, lam[:4], a_norm=10.0)
    assert np.max(r) < 1e-15
    d = np.array([1e-3, -2e-4, 0.0, 5e-6])
    r = O.generalized_residuals(A, B, X, lam[:4] + d, a_norm=10.0)
    # (lam_i + d) is rounded: an absolute error of a few ulps of lam_i b_i / a_norm
    assert np.allclose(r, np.abs(d) * bdiag[:4] / 10.0, rtol=1e-9, atol=1e-15)


def test_matrix_norm_estimate_is_a_lower_bound_exact_at_full_dimension():
    """max |Ritz value| of Lanczos: never above ||M||_2; equal to it (up to rounding) when
    the run spans the whole space; the largest modulus may sit at either end."""
    rng = np.random.default_rng(35)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    for lam in (np.linspace(-9.0, 2.0, n), np.linspace(-1.0, 5.0, n)):
        M = (Q * lam) @ Q.conj().T
        M = 0.5 * (M + M.conj().T)
        true = np.max(np.abs(lam))
        est = O.matrix_norm_estimate(M, seed=7, k=5)
        assert est <= true * (1 + 1e-12)
        assert est > 0.5 * true
        assert abs(O.matrix_norm_estimate(M, seed=7, k=n) - true) < 1e-10 * true


# ---------------------------------------------------------------------------- degenerate cases
def test_repeated_problem_warm_start_converges_in_one_loop():
    """Problem 2 identical to problem 1: the carried Ritz vectors are its eigenvectors, so one
    filter loop locks every wanted pair (fixed and adaptive degree)."""
    p = _small_problem(n=96, nev=6, blk=10).problems[0]
    A, B = np.tril(p.A.numpy()), np.tril(p.B.numpy())
    for deg in (10, 0):
        out = O.chfsi_solve_sequence([A, A], [B, B], 6, 10, 1e-10, deg=deg)
        assert out[1][2].loops == 1
        for lam, _, _ in out:
            assert np.max(np.abs(lam - p.lam[:6])) < 1e-12


def test_block_spanning_the_whole_space_is_exact_in_one_loop():
    """blk = n: the subspace is the whole space, Rayleigh-Ritz is the full eigensolver."""
    n = 12
    rng = np.random.default_rng(36)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = 0.5 * (G + G.conj().T)
    lam, X, _, st = O.chfsi_solve(np.tril(H), np.eye(n, dtype=np.complex128), 5, n, 1e-10, deg=6)
    assert st.loops == 1
    assert np.max(np.abs(lam - np.linalg.eigvalsh(H)[:5])) < 1e-12


def test_identity_overlap_reduces_to_the_standard_problem():
    p = _small_problem(n=96, nev=6, blk=10).problems[0]
    A = np.tril(p.A.numpy())
    lam, X, _, st = O.chfsi_solve(A, np.eye(96, dtype=np.complex128), 6, 10, 1e-10, deg=10)
    w, V = sla.eigh(O.hermitian_from_lower(A), subset_by_index=[0, 5])
    assert np.max(np.abs(lam - w)) < 1e-12 * max(1.0, np.max(np.abs(w)))
    # eigenvectors up to phase: |<v_i, x_i>| = 1
    assert np.allclose(np.abs(np.sum(V.conj() * X, axis=0)), 1.0, atol=1e-9)


def test_unconverged_run_reports_only_the_locked_prefix():
    """blk = nev leaves the nev-th wanted value at the edge of the damped interval (a = the
    largest Ritz value), where the filter does not separate it: within the loop limit the
    run locks a prefix, reports those values exactly and NaN for the rest."""
    p = _small_problem(n=96, nev=6, blk=10).problems[0]
    A, B = np.tril(p.A.numpy()), np.tril(p.B.numpy())
    lam, X, _, st = O.chfsi_solve(A, B, 8, 8, 1e-10, deg=10, max_loops=20)
    done = np.isfinite(lam)
    assert st.loops == 20 and 0 < done.sum() < 8
    assert np.all(done[: done.sum()])  # a contiguous prefix
    assert np.max(np.abs(lam[done] - p.lam[: done.sum()])) < 1e-12
