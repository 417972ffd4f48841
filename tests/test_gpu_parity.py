"""Parity of the sm_103a library (called through its C ABI) with the CPU oracle.

Each test feeds the same seeded inputs to one entry point of libchfsi.so and to the
oracle function that restates the same step, and compares element by element within
an FP64 tolerance derived from the arithmetic (a few hundred ulps of the operands'
scale for one product; 1e-10 relative for eigenvalues and residuals of a whole solve,
the target of Table 3).
"""
import math

import numpy as np
import pytest
import torch

import oracle.chfsi_oracle as O
from paper_1206_3768_gb300 import binding as cb
from paper_1206_3768_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    s = cb.Solver(700, 160)
    yield s.ctx
    s.close()


def _rng(seed):
    return np.random.default_rng(seed)


def _cgauss(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def _herm(rng, n, spread=1.0):
    M = _cgauss(rng, n, n)
    return spread * 0.5 * (M + M.conj().T)


def _hpd(rng, n):
    G = _cgauss(rng, n, n)
    return np.eye(n) + 0.3 * (G.conj().T @ G) / n


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ---------------------------------------------------------------------------- GEMM
@pytest.mark.parametrize("opa,opb", [("N", "N"), ("N", "C"), ("C", "N"), ("C", "C")])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (70, 33, 45), (129, 130, 700), (64, 32, 16),
                                   (200, 5, 3000 // 5)])
def test_zgemm_matches_exact_product(ctx, opa, opb, M, N, K):
    rng = _rng(M * 7 + N * 3 + K)
    A = _cgauss(rng, M, K) if opa == "N" else _cgauss(rng, K, M)
    B = _cgauss(rng, K, N) if opb == "N" else _cgauss(rng, N, K)
    C0 = _cgauss(rng, M, N)
    opA = A if opa == "N" else A.conj().T
    opB = B if opb == "N" else B.conj().T
    ref = 0.75 * (opA @ opB) - 0.5 * C0
    got = _np(cb.chfsi_zgemm(ctx, opa, opb, 0.75, _t(A), _t(B), beta=-0.5, C=_t(C0)))
    scale = np.abs(opA) @ np.abs(opB) + np.abs(C0)
    assert np.max(np.abs(got - ref) / scale) < 64 * K * 2.2e-16


# ---------------------------------------------------------------------------- reduction
@pytest.mark.parametrize("n", [1, 37, 128, 300, 513])
def test_cholesky_matches_oracle(ctx, n):
    rng = _rng(n)
    B = _hpd(rng, n)
    Bl = np.tril(B) + np.triu(_cgauss(rng, n, n), 1) * 1e3  # upper triangle must be ignored
    L = _np(cb.chfsi_cholesky(ctx, _t(Bl)))
    Lo = O.cholesky_lower(np.tril(B))
    assert np.allclose(np.triu(L, 1), 0.0)
    assert _rel(L, Lo) < 1e-12


def test_cholesky_reports_not_positive_definite(ctx):
    rng = _rng(3)
    n = 200
    B = _hpd(rng, n)
    B[150, 150] = -5.0
    with pytest.raises(cb.ChfsiError) as ei:
        cb.chfsi_cholesky(ctx, _t(B))
    assert ei.value.code == cb.CHFSI_ENOTPD
    # the context stays usable
    L = _np(cb.chfsi_cholesky(ctx, _t(_hpd(rng, 50))))
    assert np.all(np.isfinite(L))


@pytest.fixture(scope="module")
def ctx64():
    s = cb.Solver(700, 160, precision=0)
    yield s.ctx
    s.close()


@pytest.mark.parametrize("n", [64, 257, 640])
@pytest.mark.parametrize("mode", ["split", "fp64"])
def test_reduce_matches_oracle(ctx, ctx64, n, mode):
    rng = _rng(n + 1)
    A = _herm(rng, n, 3.0)
    B = _hpd(rng, n)
    Lo = O.cholesky_lower(np.tril(B))
    c = ctx if mode == "split" else ctx64
    H = _np(cb.chfsi_reduce(c, _t(np.tril(A)), _t(Lo)))
    Ho = O.reduce_standard(np.tril(A), Lo)
    assert np.allclose(H, H.conj().T, atol=0)
    assert _rel(H, Ho) < 1e-12


# ---------------------------------------------------------------------------- Lanczos
@pytest.mark.parametrize("n,k", [(300, 10), (300, 40), (513, 20)])
@pytest.mark.parametrize("mode", ["split", "fp64"])
def test_lanczos_matches_oracle(ctx, ctx64, n, k, mode):
    """FP64 products: the oracle's bound to 1e-10.  Mixed precision runs the products with
    FP32 multiply-adds (a spectral bound needs no more): 1e-5, and still an upper bound."""
    rng = _rng(k)
    lam = np.sort(rng.uniform(-1, 5, n))
    Q, _ = np.linalg.qr(_cgauss(rng, n, n))
    H = (Q * lam) @ Q.conj().T
    H = 0.5 * (H + H.conj().T)
    v0 = _cgauss(rng, n)
    tol = 1e-10 if mode == "fp64" else 1e-5
    up, tmin, tmax = cb.chfsi_lanczos(ctx if mode == "split" else ctx64, _t(H), k, _t(v0))
    up_o, tmin_o, a, bta = O.lanczos(H, v0, k)
    assert abs(up - up_o) < tol * abs(up_o)
    assert abs(tmin - tmin_o) < tol * max(1, abs(tmin_o))
    assert up >= lam[-1] - 1e-12


@pytest.mark.parametrize("mode", ["split", "fp64"])
def test_lanczos_default_start_vector_is_splitmix(ctx, ctx64, mode):
    n = 200
    rng = _rng(9)
    H = _herm(rng, n)
    up, tmin, _ = cb.chfsi_lanczos(ctx if mode == "split" else ctx64, _t(H), 12, None)
    up_o, tmin_o, _, _ = O.lanczos(H, O.lanczos_start_vector(n, 12063768), 12)
    assert abs(up - up_o) < (1e-11 if mode == "fp64" else 1e-5) * abs(up_o)


# ---------------------------------------------------------------------------- filter
@pytest.mark.parametrize("n,m", [(300, 30), (513, 17), (640, 130)])
def test_filter_matches_oracle_per_column_degrees(ctx, n, m):
    rng = _rng(n + m)
    lam = np.sort(rng.uniform(-2, 2, n))
    Q, _ = np.linalg.qr(_cgauss(rng, n, n))
    H = (Q * lam) @ Q.conj().T
    H = 0.5 * (H + H.conj().T)
    Y = _cgauss(rng, n, m)
    degs = rng.integers(0, 26, m)
    degs[0] = 25
    a0, a, b = lam[0], lam[m + 5], lam[-1] + 0.01
    got = _np(cb.chfsi_filter(ctx, _t(H), _t(Y), degs, a0, a, b))
    ref = O.chebyshev_filter(H, Y, degs, a0, a, b)
    for j in range(m):
        assert np.max(np.abs(got[:, j] - ref[:, j])) <= 1e-11 * np.max(np.abs(ref[:, j])), j


def test_filter_fixed_degree_closed_form(ctx):
    n, m, d = 400, 24, 11
    rng = _rng(77)
    lam = np.sort(rng.uniform(-1, 3, n))
    Q, _ = np.linalg.qr(_cgauss(rng, n, n))
    H = (Q * lam) @ Q.conj().T
    H = 0.5 * (H + H.conj().T)
    a0, a, b = lam[0], lam[40], lam[-1] + 0.05
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    X = Q[:, :m]
    got = _np(cb.chfsi_filter(ctx, _t(H), _t(X), [d] * m, a0, a, b))
    p = O.chebyshev_T(d, (lam[:m] - c) / e) / O.chebyshev_T(d, np.array([(a0 - c) / e]))[0]
    assert np.max(np.abs(got - X * p[None, :])) < 1e-11


# ---------------------------------------------------------------------------- QR, RR
@pytest.mark.parametrize("n,m,k", [(300, 20, 0), (513, 40, 12), (640, 130, 30), (700, 160, 0)])
@pytest.mark.parametrize("mode", ["split", "fp64"])
def test_orthonormalize_matches_oracle_span(ctx, ctx64, n, m, k, mode):
    """Mixed precision (FP32 Cholesky QR steps, then FP64 Loewdin steps; m = 160 keeps the
    FP32 factor in global memory) and plain FP64 Cholesky QR."""
    rng = _rng(n + m + k)
    YL = np.linalg.qr(_cgauss(rng, n, k))[0] if k else None
    # an ill-conditioned block (column scales spread over 1e6, as after filtering)
    Y = _cgauss(rng, n, m) * np.logspace(0, -6, m)[None, :]
    got = _np(cb.chfsi_orthonormalize(ctx if mode == "split" else ctx64, _t(Y), _t(YL) if k else None))
    ref = O.orthonormalize(Y, YL)
    assert np.max(np.abs(got.conj().T @ got - np.eye(m))) < 1e-13
    if k:
        assert np.max(np.abs(YL.conj().T @ got)) < 1e-13
    assert np.linalg.norm(got @ got.conj().T - ref @ ref.conj().T) < 1e-9


@pytest.mark.parametrize("n,m,k", [(1400, 400, 30), (2600, 1200, 0), (1300, 161, 7)])
def test_orthonormalize_wide_blocks_match_oracle_span(n, m, k):
    """Blocks wider than one CTA's shared memory: the FP32 Cholesky QR steps run as one
    cooperative grid (blocked factorisation, 32-column panels; a ragged last panel at
    m = 161, 400 and 1200 = 37.5 panels).  The orthogonality bound of the narrow test
    (1e-13 up to 160 columns) grows with the width like the rounding of the last step's
    7-slice product Y T: each entry of Y T carries a relative error of about 2^-49 of its
    scales, and an entry of (Y T)^H (Y T) sums m such products, so the bound is scaled by
    sqrt(m / 160)."""
    rng = _rng(7 * n + m + k)
    YL = np.linalg.qr(_cgauss(rng, n, k))[0] if k else None
    Y = _cgauss(rng, n, m) * np.logspace(0, -6, m)[None, :]
    with cb.Solver(n, m) as s:
        got = _np(cb.chfsi_orthonormalize(s.ctx, _t(Y), _t(YL) if k else None))
    ref = O.orthonormalize(Y, YL)
    bound = 1e-13 * max(1.0, math.sqrt(m / 160))
    assert np.max(np.abs(got.conj().T @ got - np.eye(m))) < bound
    if k:
        assert np.max(np.abs(YL.conj().T @ got)) < bound
    assert np.linalg.norm(got @ got.conj().T - ref @ ref.conj().T) < 1e-9


def test_orthonormalize_wide_block_near_rank_deficiency():
    """A wide block whose Gram matrix breaks plain FP32 Cholesky takes the shifted retry
    inside the cooperative pass."""
    n, m = 900, 200
    rng = _rng(15)
    base = _cgauss(rng, n, m)
    Y = base.copy()
    Y[:, 150] = base[:, 149] + 1e-9 * _cgauss(rng, n)
    with cb.Solver(n, m) as s:
        got = _np(cb.chfsi_orthonormalize(s.ctx, _t(Y)))
    assert np.max(np.abs(got.conj().T @ got - np.eye(m))) < 1e-12
    keep = [j for j in range(m) if j != 150]
    P = got @ got.conj().T
    assert np.linalg.norm(P @ base[:, keep] - base[:, keep]) < 1e-6 * np.linalg.norm(base)


@pytest.mark.parametrize("mode", ["split", "fp64"])
def test_orthonormalize_survives_near_rank_deficiency(ctx, ctx64, mode):
    """A Gram matrix beyond plain Cholesky QR takes the shifted path."""
    n, m = 400, 16
    rng = _rng(5)
    base = _cgauss(rng, n, m)
    Y = base.copy()
    Y[:, 5] = base[:, 4] + 1e-9 * _cgauss(rng, n)
    got = _np(cb.chfsi_orthonormalize(ctx if mode == "split" else ctx64, _t(Y)))
    assert np.max(np.abs(got.conj().T @ got - np.eye(m))) < 1e-12
    # the span still holds the well-determined directions of Y
    keep = [j for j in range(m) if j != 5]
    P = got @ got.conj().T
    assert np.linalg.norm(P @ base[:, keep] - base[:, keep]) < 1e-6 * np.linalg.norm(base)


@pytest.mark.parametrize("n,m", [(300, 25), (640, 130), (513, 131)])
@pytest.mark.parametrize("mode", ["split", "fp64"])
def test_rayleigh_ritz_matches_oracle(ctx, ctx64, n, m, mode):
    rng = _rng(n * m)
    lam = np.sort(rng.uniform(-1, 4, n))
    Q, _ = np.linalg.qr(_cgauss(rng, n, n))
    H = (Q * lam) @ Q.conj().T
    H = 0.5 * (H + H.conj().T)
    S = np.linalg.qr(Q[:, :m] + 1e-3 * _cgauss(rng, n, m))[0]
    theta, Y, HY = cb.chfsi_rayleigh_ritz(ctx if mode == "split" else ctx64, _t(H), _t(S))
    th_o, Y_o, W_o = O.rayleigh_ritz(H, S)
    theta, Y, HY = _np(theta), _np(Y), _np(HY)
    assert np.max(np.abs(theta - th_o)) < 1e-12 * np.max(np.abs(lam))
    assert np.max(np.abs(HY - H @ Y)) < 1e-12 * np.max(np.abs(lam))
    assert np.max(np.abs(Y.conj().T @ Y - np.eye(m))) < 1e-12
    # Ritz vectors agree up to phase where the Ritz values are separated
    gaps = np.minimum(np.diff(np.r_[-np.inf, th_o]), np.diff(np.r_[th_o, np.inf]))
    ov = np.abs(np.sum(Y.conj() * Y_o, axis=0))
    assert np.all(np.abs(ov[gaps > 1e-6] - 1) < 1e-8)
    r = _np(cb.chfsi_residuals(ctx, _t(HY), _t(Y), _t(theta)))
    r_o = O.residual_norms(H @ Y, Y, theta)
    assert np.max(np.abs(r - r_o)) < 1e-12 * np.max(np.abs(lam))


@pytest.mark.parametrize("m", [1, 2, 7, 64, 130, 131, 160])
def test_heev_matches_lapack(ctx, m):
    rng = _rng(m + 100)
    G = _herm(rng, m, 2.0)
    w, V = cb.chfsi_heev(ctx, _t(G))
    w, V = _np(w), _np(V)
    w_ref = np.linalg.eigvalsh(G)
    nrm = np.linalg.norm(G, 2)
    assert np.max(np.abs(w - w_ref)) < 1e-13 * nrm * max(1, math.sqrt(m))
    assert np.max(np.abs(V.conj().T @ V - np.eye(m))) < 1e-13 * max(1, math.sqrt(m))
    assert np.max(np.abs(G @ V - V * w[None, :])) < 1e-13 * nrm * max(1, math.sqrt(m))


def test_heev_clustered_spectrum(ctx):
    m = 48
    rng = _rng(4)
    lam = np.r_[np.full(10, -1.0) + 1e-12 * rng.standard_normal(10), np.linspace(0, 3, 38)]
    U = np.linalg.qr(_cgauss(rng, m, m))[0]
    G = (U * lam) @ U.conj().T
    G = 0.5 * (G + G.conj().T)
    w, V = cb.chfsi_heev(ctx, _t(G))
    w, V = _np(w), _np(V)
    assert np.max(np.abs(w - np.sort(lam))) < 1e-13
    assert np.max(np.abs(G @ V - V * w[None, :])) < 1e-13


@pytest.mark.parametrize("m", [64, 97, 320, 601, 1200])
def test_heev_double_float_matches_lapack(m):
    """The double-float Jacobi (the mixed-precision Rayleigh-Ritz solver of wide blocks)
    against LAPACK: a random Hermitian matrix and a nearly diagonal one.  Its arithmetic
    carries about 48 significand bits (unit roundoff 2^-47 ~ 7e-15 per operation), so the
    bounds are those of the FP64 test with u = 2^-47 for 2^-53: 1e-13 -> 5e-12 relative to
    ||G||_2 sqrt(m), orthogonality 5e-12 sqrt(m)."""
    rng = _rng(3 * m + 1)
    G = _herm(rng, m, 2.0)
    D = np.diag(np.sort(rng.uniform(-2, 2, m))) + 1e-6 * _herm(rng, m)
    with cb.Solver(m, m) as s:
        for M in (G, D):
            w, V = cb.chfsi_heev_df(s.ctx, _t(M))
            w, V = _np(w), _np(V)
            w_ref = np.linalg.eigvalsh(M)
            nrm = np.linalg.norm(M, 2)
            assert np.max(np.abs(w - w_ref)) < 5e-12 * nrm * math.sqrt(m)
            assert np.max(np.abs(V.conj().T @ V - np.eye(m))) < 5e-12 * math.sqrt(m)
            assert np.max(np.abs(M @ V - V * w[None, :])) < 5e-12 * nrm * math.sqrt(m)
            assert np.all(np.diff(w) >= 0)


@pytest.mark.parametrize("m", [601, 700, 1200])
def test_heev_large_blocks_share_cooperative_ctas(m):
    """Blocks above ~600 columns (the n = 13,400 workload's blk = 1200) run with several
    rotation pairs per CTA of the cooperative grid: eigenpairs against LAPACK, a random
    Hermitian matrix and a nearly diagonal one (the Gram matrix of a warm loop)."""
    rng = _rng(m)
    G = _herm(rng, m, 2.0)
    D = np.diag(np.sort(rng.uniform(-2, 2, m))) + 1e-6 * _herm(rng, m)
    with cb.Solver(m, m) as s:
        for M in (G, D):
            w, V = cb.chfsi_heev(s.ctx, _t(M))
            w, V = _np(w), _np(V)
            w_ref = np.linalg.eigvalsh(M)
            nrm = np.linalg.norm(M, 2)
            assert np.max(np.abs(w - w_ref)) < 1e-13 * nrm * math.sqrt(m)
            assert np.max(np.abs(V.conj().T @ V - np.eye(m))) < 1e-13 * math.sqrt(m)
            assert np.max(np.abs(M @ V - V * w[None, :])) < 1e-13 * nrm * math.sqrt(m)


# ---------------------------------------------------------------------------- degrees
def test_degrees_bit_exact_with_oracle(ctx):
    rng = _rng(11)
    m = 130
    a, b = -0.5, 30.0
    theta = np.sort(np.r_[rng.uniform(-1.0, -0.55, 100), rng.uniform(-0.55, 2.0, 30)])
    r = 10.0 ** rng.uniform(-12, -1, m)
    tau = 1e-10
    for nw in (0, 37, 100, 130):
        got = _np(cb.chfsi_degrees(ctx, _t(theta), _t(r), a, b, tau, 8, 25, nw))
        ref = O.adaptive_degrees(theta, r, a, b, tau, 8, 25, nw)
        assert np.array_equal(got, ref)


# ---------------------------------------------------------------------------- whole solve
def _check_solution(p, lam, X, nev, tol=1e-10):
    A, B = p.A.numpy(), p.B.numpy()
    a2 = np.linalg.norm(A, 2)
    scale = max(np.max(np.abs(p.lam)), 1.0)
    err = np.max(np.abs(lam - p.lam[:nev]) / np.maximum(np.abs(p.lam[:nev]), scale))
    assert err <= tol, err
    R = A @ X - (B @ X) * lam[None, :]
    res = np.linalg.norm(R, axis=0) / (a2 * np.linalg.norm(X, axis=0))
    assert res.max() <= tol, res.max()
    assert np.max(np.abs(X.conj().T @ B @ X - np.eye(nev))) < 1e-10


def test_solve_sequence_c1_matches_oracle_and_planted_spectrum(ctx):
    seq = inputs.planted_sequence("c1")
    As = [torch.tril(p.A).to(DEV) for p in seq.problems]
    Bs = [torch.tril(p.B).to(DEV) for p in seq.problems]
    cb.chfsi_reset_warm_state(ctx)
    evals, evecs, stats = cb.chfsi_solve_sequence(ctx, As, Bs, seq.nev, seq.blk, seq.deg, 1e-10)
    ref = O.chfsi_solve_sequence([np.tril(p.A.numpy()) for p in seq.problems],
                                 [np.tril(p.B.numpy()) for p in seq.problems],
                                 seq.nev, seq.blk, 1e-10, deg=seq.deg)
    for ell, p in enumerate(seq.problems):
        lam = evals[ell].numpy()
        X = _np(evecs[ell])
        _check_solution(p, lam, X, seq.nev)
        w_def, _ = O.definition_eigenpairs(np.tril(p.A.numpy()), np.tril(p.B.numpy()), seq.nev)
        assert np.max(np.abs(lam - w_def)) < 1e-10 * max(1, np.max(np.abs(w_def)))
        lam_o, _, st_o = ref[ell]
        assert np.max(np.abs(lam - lam_o)) < 1e-10 * max(1, np.max(np.abs(lam_o)))
        assert abs(stats[ell]["loops"] - st_o.loops) <= 1
        assert stats[ell]["converged"] == seq.nev


def test_solve_adaptive_ill_conditioned_overlap(ctx):
    seq = inputs.planted_sequence("c2", n=520, N=3, nev=20, blk=26)
    cb.chfsi_reset_warm_state(ctx)
    for p in seq.problems:
        lam, X, st = cb.chfsi_solve_next(ctx, torch.tril(p.A).to(DEV), torch.tril(p.B).to(DEV),
                                         20, 26, 0, 1e-10)
        _check_solution(p, lam.cpu().numpy(), _np(X), 20)
        assert st["max_resid"] <= 1e-10


def test_host_pointers_give_the_device_result(ctx):
    seq = inputs.planted_sequence("c1", n=256, N=1, nev=10, blk=16)
    p = seq.problems[0]
    cb.chfsi_reset_warm_state(ctx)
    lam_d, X_d, _ = cb.chfsi_solve_next(ctx, p.A.to(DEV), p.B.to(DEV), 10, 16, 10)
    cb.chfsi_reset_warm_state(ctx)
    lam_h, X_h, _ = cb.chfsi_solve_next(ctx, p.A.clone(), p.B.clone(), 10, 16, 10, out_device="cpu")
    assert torch.equal(lam_d.cpu(), lam_h)
    assert torch.equal(X_d.cpu(), X_h)


def test_host_sequence_is_staged_ahead_and_gives_the_device_result(ctx):
    """chfsi_solve_sequence with host matrices copies problem l + 1 while problem l solves
    (two staging buffer pairs on a copy stream): the results equal the device-input solve."""
    seq = inputs.planted_sequence("c1", n=256, N=3, nev=10, blk=16)
    As = [torch.tril(p.A) for p in seq.problems]
    Bs = [torch.tril(p.B) for p in seq.problems]
    cb.chfsi_reset_warm_state(ctx)
    ev_d, X_d, _ = cb.chfsi_solve_sequence(ctx, [a.to(DEV) for a in As], [b.to(DEV) for b in Bs], 10, 16, 10)
    cb.chfsi_reset_warm_state(ctx)
    pinned = [a.mT.contiguous().pin_memory().mT for a in As]
    ev_h, X_h, _ = cb.chfsi_solve_sequence(ctx, pinned, Bs, 10, 16, 10)
    assert torch.equal(ev_d, ev_h)
    for xd, xh in zip(X_d, X_h):
        assert torch.equal(xd.cpu(), xh)


def test_cold_start_with_caller_block(ctx):
    seq = inputs.planted_sequence("c1", n=300, N=1, nev=12, blk=20)
    p = seq.problems[0]
    V0 = inputs.gaussian_block(300, 20, 5)
    cb.chfsi_reset_warm_state(ctx)
    lam, X, st = cb.chfsi_solve_next(ctx, p.A.to(DEV), p.B.to(DEV), 12, 20, 10, V0=V0.to(DEV))
    _check_solution(p, lam.cpu().numpy(), _np(X), 12)
    lam_o, _, _, st_o = O.chfsi_solve(np.tril(p.A.numpy()), np.tril(p.B.numpy()), 12, 20, deg=10,
                                      V0=V0.numpy())
    assert np.max(np.abs(lam.cpu().numpy() - lam_o)) < 1e-10
    assert abs(st["loops"] - st_o.loops) <= 1


def test_invalid_arguments_are_reported(ctx):
    seq = inputs.planted_sequence("c1", n=64, N=1, nev=4, blk=8)
    p = seq.problems[0]
    A, B = p.A.to(DEV), p.B.to(DEV)
    with pytest.raises(cb.ChfsiError) as ei:
        cb.chfsi_solve_next(ctx, A, B, 8, 4, 10)  # blk < nev
    assert ei.value.code == cb.CHFSI_EINVAL
    An = A.clone()
    An[10, 3] = float("nan")
    cb.chfsi_reset_warm_state(ctx)
    with pytest.raises(cb.ChfsiError) as ei:
        cb.chfsi_solve_next(ctx, An, B, 4, 8, 10)
    assert ei.value.code == cb.CHFSI_EINVAL
    Bn = -torch.eye(64, dtype=torch.complex128, device=DEV)
    cb.chfsi_reset_warm_state(ctx)
    with pytest.raises(cb.ChfsiError) as ei:
        cb.chfsi_solve_next(ctx, A, Bn, 4, 8, 10)
    assert ei.value.code == cb.CHFSI_ENOTPD
    # still usable afterwards
    cb.chfsi_reset_warm_state(ctx)
    lam, X, st = cb.chfsi_solve_next(ctx, A, B, 4, 8, 10)
    _check_solution(p, lam.cpu().numpy(), _np(X), 4)


# ---------------------------------------------------------------------------- split-BF16 filter
@pytest.mark.parametrize("n,m,slices,tol", [(300, 30, 7, 1e-12), (513, 17, 7, 1e-12),
                                            (640, 130, 7, 1e-12), (513, 40, 4, 1e-7),
                                            (300, 9, 3, 1e-5), (300, 12, 2, 2e-3),
                                            (64, 1, 8, 1e-13)])
def test_filter_split_matches_oracle(ctx, n, m, slices, tol):
    """Split-BF16 digit products reproduce the FP64 filter to about 2^(-7 slices), down to the
    two slices the adaptive slice count of the mixed-precision filter may choose.  The
    tensor-core path takes the product in the Gauss form, whose imaginary part is the
    difference of three real products (P2 - P0 - P1), each truncated at its own scales: its
    worst-case bound is up to six times the embedding's (the exact model in
    test_digit_arithmetic.py), the errors measured here stay within three times: 3 tol."""
    tol = 3.0 * tol
    rng = _rng(n + m + slices)
    lam = np.sort(rng.uniform(-2, 2, n))
    Q, _ = np.linalg.qr(_cgauss(rng, n, n))
    H = (Q * lam) @ Q.conj().T
    H = 0.5 * (H + H.conj().T)
    Y = _cgauss(rng, n, m)
    degs = rng.integers(0, 16, m)
    degs[0] = 15
    a0, a, b = lam[0], lam[min(n - 2, m + 5)], lam[-1] + 0.01
    got = _np(cb.chfsi_filter_split(ctx, _t(H), _t(Y), degs, a0, a, b, slices))
    ref = O.chebyshev_filter(H, Y, degs, a0, a, b)
    for j in range(m):
        scale = np.max(np.abs(ref[:, j]))
        assert np.max(np.abs(got[:, j] - ref[:, j])) <= tol * max(scale, 1e-300), (j, degs[j])


@pytest.mark.parametrize("m", [1, 16, 40, 64, 96, 112])
def test_filter_split_single_product_is_exact_to_fp64_level(m):
    """One degree-1 step with 8 slices against the FP64 product on random (not Hermitian-
    structured beyond symmetry) data: error at the level of FP64 rounding of the result.
    The widths cover every slice-group size of the tensor-core kernel (7, 3, 3, 2, 1 pairs
    per A tile, and the ragged last group of each A slice)."""
    n = 1100   # K = 2n = 2200 spans three exact 960-term chunks
    rng = _rng(99)
    H = _herm(rng, n, 1.0) * np.exp(rng.uniform(-3, 3, (n, 1)))  # rows on different scales
    H = 0.5 * (H + H.conj().T)
    Y = _cgauss(rng, n, m) * np.exp(rng.uniform(-5, 5, (1, m)))
    a0, a, b = -5.0, -1.0, 3.0   # degree 1: Y1 = (sigma1/e) (H - c) Y
    with cb.Solver(n, m) as s:
        got = _np(cb.chfsi_filter_split(s.ctx, _t(H), _t(Y), [1] * m, a0, a, b, 8))
    ref = O.chebyshev_filter(H, Y, [1] * m, a0, a, b)
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    s1 = e / (a0 - c)
    bound = abs(s1 / e) * (np.abs(H) @ np.abs(Y) + abs(c) * np.abs(Y))
    assert np.max(np.abs(got - ref) / bound) < 2 * n * 1.1e-16  # the FP64 GEMM error bound


def test_solve_plain_fp64_mode_matches_mixed_mode():
    seq = inputs.planted_sequence("c1", n=400, N=2, nev=12, blk=20)
    res = {}
    for prec in (0, 1):
        with cb.Solver(400, 20, precision=prec) as s:
            As = [torch.tril(p.A).to(DEV) for p in seq.problems]
            Bs = [torch.tril(p.B).to(DEV) for p in seq.problems]
            ev, X, st = cb.chfsi_solve_sequence(s.ctx, As, Bs, 12, 20, 10, 1e-10)
            res[prec] = (ev.numpy(), st)
            for ell, p in enumerate(seq.problems):
                _check_solution(p, ev[ell].numpy(), _np(X[ell]), 12)
    assert np.max(np.abs(res[0][0] - res[1][0])) < 1e-10
    assert all(s["filter_matvecs_fp64"] == s["filter_matvecs"] for s in res[0][1])
    assert all(s["tensor_flops"] > 0 for s in res[1][1])


# ---------------------------------------------------------------------------- deviation angles
def _b_orthonormal(rng, n, k, B):
    Z = _cgauss(rng, n, k)
    R = np.linalg.cholesky(Z.conj().T @ B @ Z).conj().T
    return Z @ np.linalg.inv(R)


@pytest.mark.parametrize("n,k", [(300, 8), (700, 160)])
def test_deviation_angles_planted(ctx, n, k):
    """Pairwise rotations by known angles from 0.3 down to 1e-9 inside a B-orthonormal
    basis, with the current vectors shuffled: angles and association match the oracle."""
    rng = _rng(n + k)
    B = _hpd(rng, n)
    X = _b_orthonormal(rng, n, k, B)
    phis = np.logspace(math.log10(0.3), -9, k // 2)
    Y = X.copy()
    for p, phi in enumerate(phis):
        a, b = 2 * p, 2 * p + 1
        c, s = math.cos(phi), math.sin(phi)
        Y[:, a] = c * X[:, a] + s * np.exp(0.7j) * X[:, b]
        Y[:, b] = -s * np.exp(-0.7j) * X[:, a] + c * X[:, b]
    perm = rng.permutation(k)
    Y = Y[:, perm] * np.exp(1j * rng.uniform(0, 6, k))[None, :]
    th_o, as_o = O.deviation_angles(X, Y, B)
    th, assoc = cb.chfsi_deviation_angles(ctx, _t(X), _t(Y), _t(B))
    th, assoc = _np(th), _np(assoc)
    assert list(assoc) == list(as_o)
    assert np.all(np.abs(th - th_o) <= 1e-9 * th_o + 1e-14)
    assert np.allclose(np.sort(th), np.sort(np.repeat(phis, 2)), rtol=1e-8, atol=1e-14)


def test_deviation_angles_along_planted_sequence(ctx):
    """Eigenvectors solved by the library along a planted sequence: the angles between
    adjacent problems match the oracle's on the same vectors and shrink along the sequence
    (the trend of Fig. 1)."""
    seq = inputs.planted_sequence("c1", n=256, N=4, nev=10, blk=16, device="cuda")
    As = [p.A for p in seq.problems]
    Bs = [p.B for p in seq.problems]
    cb.chfsi_reset_warm_state(ctx)
    _, evecs, _ = cb.chfsi_solve_sequence(ctx, As, Bs, 10, 16, 10, 1e-10)
    means = []
    for l in range(1, 4):
        th, assoc = cb.chfsi_deviation_angles(ctx, evecs[l - 1], evecs[l], Bs[l])
        th_o, as_o = O.deviation_angles(_np(evecs[l - 1]), _np(evecs[l]), _np(Bs[l]))
        assert list(_np(assoc)) == list(as_o)
        assert np.max(np.abs(_np(th) - th_o)) <= 1e-8 * np.max(th_o) + 1e-13
        means.append(float(np.mean(th_o)))
    assert means[0] > means[1] > means[2]


def test_solve_n9300_mixed_precision_workload():
    """The n = 9300 mixed-precision workload (nev 256, blk 320, degree 20) at full size, two
    problems (cold + warm): eigenvalues against the planted spectrum, generalized residuals
    against a lower bound of ||A||_2 (power iteration), and B-orthonormality, all on the GPU."""
    seq = inputs.planted_sequence("c3", N=2, device="cuda", keep_vectors=False)
    n, nev, blk = seq.n, seq.nev, seq.blk
    As = [cb.fortran(torch.tril(p.A)) for p in seq.problems]
    Bs = [cb.fortran(torch.tril(p.B)) for p in seq.problems]
    with cb.Solver(n, blk) as s:
        evals, evecs, stats = cb.chfsi_solve_sequence(s.ctx, As, Bs, nev, blk, seq.deg, seq.tol)
    scale = max(float(np.max(np.abs(p.lam))) for p in seq.problems)
    for ell, p in enumerate(seq.problems):
        lam = evals[ell]
        assert stats[ell]["converged"] == nev
        assert np.max(np.abs(lam.numpy() - p.lam[:nev])) <= 1e-10 * scale
        A, B, X = p.A, p.B, evecs[ell]
        assert stats[ell]["max_resid"] <= seq.tol
        v = torch.ones(n, 1, dtype=torch.complex128, device=A.device)
        for _ in range(30):
            v = A @ v
            v = v / torch.linalg.vector_norm(v)
        a_low = float(torch.linalg.vector_norm(A @ v))  # ||A v|| with ||v|| = 1: <= ||A||_2
        lam_d = lam.to(A.device).to(torch.complex128)
        R = A @ X - (B @ X) * lam_d[None, :]
        res = torch.linalg.vector_norm(R, dim=0) / (a_low * torch.linalg.vector_norm(X, dim=0))
        assert float(res.max()) <= 1e-10, float(res.max())
        E = X.mH @ (B @ X) - torch.eye(nev, dtype=torch.complex128, device=A.device)
        assert float(E.abs().max()) < 1e-10


def test_solve_wide_blocks_with_double_float_rayleigh_ritz():
    """The n = 13,400 workload's spectrum and adaptive degrees at n = 3000 with blocks of 400
    columns (two problems, cold + warm): the Rayleigh-Ritz eigensolver runs in double-float
    arithmetic from 384 columns; eigenvalues against the planted spectrum, generalized
    residuals and B-orthonormality at the solver's FP64 bar."""
    seq = inputs.planted_sequence("c5", n=3000, N=2, nev=300, blk=400, device="cuda", keep_vectors=False)
    n, nev, blk = seq.n, seq.nev, seq.blk
    As = [cb.fortran(torch.tril(p.A)) for p in seq.problems]
    Bs = [cb.fortran(torch.tril(p.B)) for p in seq.problems]
    with cb.Solver(n, blk, deg_min=seq.deg_min, deg_max=seq.deg_max) as s:
        evals, evecs, stats = cb.chfsi_solve_sequence(s.ctx, As, Bs, nev, blk, seq.deg, seq.tol)
    scale = max(float(np.max(np.abs(p.lam))) for p in seq.problems)
    for ell, p in enumerate(seq.problems):
        lam = evals[ell]
        assert stats[ell]["converged"] == nev
        assert np.max(np.abs(lam.numpy() - p.lam[:nev])) <= 1e-10 * scale
        A, B, X = p.A, p.B, evecs[ell]
        lam_d = lam.to(A.device).to(torch.complex128)
        R = A @ X - (B @ X) * lam_d[None, :]
        res = torch.linalg.vector_norm(R, dim=0) / (scale * torch.linalg.vector_norm(X, dim=0))
        assert float(res.max()) <= 1e-10, float(res.max())
        E = X.mH @ (B @ X) - torch.eye(nev, dtype=torch.complex128, device=A.device)
        assert float(E.abs().max()) < 1e-10


def test_solve_n2600_benchmark_workload_full_size():
    """The benchmark's n = 2600 workload (nev 100, blk 130, adaptive degree 8-25, cond(B) =
    1e4) at full size in the benchmark's launch configuration, three problems (cold + two
    warm): eigenvalues against the planted spectrum and, for the first and last problem,
    against LAPACK on the host; generalized residuals against a lower bound of ||A||_2
    (power iteration) and B-orthonormality, computed on the GPU."""
    seq = inputs.planted_sequence("c2", N=3, device="cuda", keep_vectors=False)
    n, nev, blk = seq.n, seq.nev, seq.blk
    As = [cb.fortran(torch.tril(p.A)) for p in seq.problems]
    Bs = [cb.fortran(torch.tril(p.B)) for p in seq.problems]
    with cb.Solver(n, blk, deg_min=seq.deg_min, deg_max=seq.deg_max) as s:
        evals, evecs, stats = cb.chfsi_solve_sequence(s.ctx, As, Bs, nev, blk, seq.deg, seq.tol)
    scale = max(float(np.max(np.abs(p.lam))) for p in seq.problems)
    for ell, p in enumerate(seq.problems):
        lam = evals[ell]
        assert stats[ell]["converged"] == nev
        assert np.max(np.abs(lam.numpy() - p.lam[:nev])) <= 1e-10 * scale
        if ell in (0, len(seq.problems) - 1):
            w_def, _ = O.definition_eigenpairs(np.tril(p.A.cpu().numpy()), np.tril(p.B.cpu().numpy()), nev)
            assert np.max(np.abs(lam.numpy() - w_def)) <= 1e-10 * scale
        A, B, X = p.A, p.B, evecs[ell]
        assert stats[ell]["max_resid"] <= seq.tol
        v = torch.ones(n, 1, dtype=torch.complex128, device=A.device)
        for _ in range(30):
            v = A @ v
            v = v / torch.linalg.vector_norm(v)
        a_low = float(torch.linalg.vector_norm(A @ v))  # ||A v|| with ||v|| = 1: <= ||A||_2
        lam_d = lam.to(A.device).to(torch.complex128)
        R = A @ X - (B @ X) * lam_d[None, :]
        res = torch.linalg.vector_norm(R, dim=0) / (a_low * torch.linalg.vector_norm(X, dim=0))
        assert float(res.max()) <= 1e-10, float(res.max())
        E = X.mH @ (B @ X) - torch.eye(nev, dtype=torch.complex128, device=A.device)
        assert float(E.abs().max()) < 1e-10


def test_batch_uneven_sequences_match_sequential():
    """Five k-point sequences of uneven size solved by a batch of three workers: every
    eigenvalue equals the one-context sequential solve's and the planted spectrum."""
    seqs = inputs.kpoint_sequences(K=5, N=2, n_range=(200, 460), device="cuda")
    data = [([torch.tril(p.A) for p in q.problems], [torch.tril(p.B) for p in q.problems]) for q in seqs]
    nev = [q.nev for q in seqs]
    blk = [q.blk for q in seqs]
    n_max = max(q.n for q in seqs)
    with cb.Batch(3, n_max, max(blk)) as batch:
        res = batch.solve(data, nev, blk, 20, 1e-10)
    with cb.Solver(n_max, max(blk)) as s:
        for q, (As, Bs), (ev_b, X_b, st_b) in zip(seqs, data, res):
            cb.chfsi_reset_warm_state(s.ctx)
            ev_s, _, _ = cb.chfsi_solve_sequence(s.ctx, As, Bs, q.nev, q.blk, 20, 1e-10)
            scale = max(float(np.max(np.abs(p.lam))) for p in q.problems)
            assert np.max(np.abs(ev_b.numpy() - ev_s.numpy())) <= 1e-12 * scale
            for ell, p in enumerate(q.problems):
                assert np.max(np.abs(ev_b[ell].numpy() - p.lam[:q.nev])) <= 1e-10 * scale
                assert st_b[ell]["converged"] == q.nev
                assert st_b[ell]["max_resid"] <= 1e-10


def test_warm_state_checkpoint_resumes_the_sequence_in_another_context():
    """The warm state (Section 3.2, stage 3) taken from one context after two problems and
    installed in a fresh context continues the sequence as the first context does: problem 2
    with the same loop count and eigenvalues to rounding; no state after a reset."""
    seq = inputs.planted_sequence("c1", N=3, keep_vectors=False)
    nev, blk = seq.nev, seq.blk
    As = [torch.tril(p.A).to(DEV) for p in seq.problems]
    Bs = [torch.tril(p.B).to(DEV) for p in seq.problems]
    with cb.Solver(seq.n, blk) as s1, cb.Solver(seq.n, blk) as s2:
        assert cb.chfsi_get_state(s2.ctx) is None
        for ell in (0, 1):
            cb.chfsi_solve_next(s1.ctx, As[ell], Bs[ell], nev, blk, seq.deg)
        state = cb.chfsi_get_state(s1.ctx)
        assert state is not None and tuple(state[0].shape) == (seq.n, blk) and state[1].shape[0] == blk
        # B-orthonormal x-vectors and ascending Ritz values of problem 1
        Bf = (Bs[1] + Bs[1].mH - torch.diag(torch.diagonal(Bs[1])))
        E = state[0].mH @ (Bf @ state[0]) - torch.eye(blk, dtype=torch.complex128, device=DEV)
        assert float(E.abs().max()) < 1e-10
        assert np.all(np.diff(state[1].numpy()) >= 0)
        cb.chfsi_set_state(s2.ctx, state)
        lam1, _, st1 = cb.chfsi_solve_next(s1.ctx, As[2], Bs[2], nev, blk, seq.deg)
        lam2, _, st2 = cb.chfsi_solve_next(s2.ctx, As[2], Bs[2], nev, blk, seq.deg)
        assert st1["loops"] == st2["loops"]
        p2 = seq.problems[2]
        scale = np.max(np.abs(p2.lam))
        assert np.max(np.abs(lam1.cpu().numpy() - lam2.cpu().numpy())) <= 1e-12 * scale
        assert np.max(np.abs(lam2.cpu().numpy() - p2.lam[:nev])) <= 1e-10 * scale
        cb.chfsi_reset_warm_state(s1.ctx)
        assert cb.chfsi_get_state(s1.ctx) is None
        cb.chfsi_set_state(s2.ctx, None)
        assert cb.chfsi_get_state(s2.ctx) is None
