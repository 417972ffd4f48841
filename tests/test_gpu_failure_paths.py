"""Failure paths of the library that can be exercised without faulting or hanging a GPU.

Every device-side wait of the library is bounded: a grid barrier of the Rayleigh-Ritz
eigensolver or an mbarrier wait of the split-BF16 product kernel that runs out sets a
status flag, the kernel unwinds (its own copies and tensor-core operations finish first)
and the call reports CHFSI_ETIMEOUT.  chfsi_set_wait_limit shortens the bound so that the
waits run out on a normal input; the same context must then work again with the default
bound.  A solve that reaches its loop limit reports CHFSI_ENOCONV with the locked prefix of
eigenvalues (Algorithm 1 locks a contiguous prefix) and NaN for the rest, like the oracle.
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


def _herm(seed, n):
    rng = np.random.default_rng(seed)
    M = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2)
    return 0.5 * (M + M.conj().T)


def test_eigensolver_barrier_timeout_is_reported_and_the_context_recovers():
    m = 96
    G = torch.from_numpy(_herm(11, m)).to(DEV)
    with cb.Solver(256, m) as s:
        cb.chfsi_set_wait_limit(s.ctx, 1)   # a waiting CTA gives up after two polls
        with pytest.raises(cb.ChfsiError) as ei:
            cb.chfsi_heev(s.ctx, G)
        assert ei.value.code == cb.CHFSI_ETIMEOUT
        cb.chfsi_set_wait_limit(s.ctx, 0)
        w, V = cb.chfsi_heev(s.ctx, G)
    w_ref = np.linalg.eigvalsh(G.cpu().numpy())
    assert np.max(np.abs(w.cpu().numpy() - w_ref)) <= 1e-12 * np.max(np.abs(w_ref))


def test_product_kernel_wait_timeout_is_reported_and_the_context_recovers():
    n, m = 2048, 64
    rng = np.random.default_rng(12)
    H = torch.from_numpy(_herm(13, n) / math.sqrt(n)).to(DEV)
    Y = torch.from_numpy((rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))) / math.sqrt(2)).to(DEV)
    degs = [2] * m
    with cb.Solver(n, m) as s:
        cb.chfsi_set_wait_limit(s.ctx, 1)
        codes = []
        for _ in range(4):   # each call streams many chunks: one of its first waits runs out
            try:
                cb.chfsi_filter_split(s.ctx, H, Y, degs, -2.0, -1.0, 2.5, 4)
                codes.append(cb.CHFSI_OK)
            except cb.ChfsiError as e:
                codes.append(e.code)
            if codes[-1] == cb.CHFSI_ETIMEOUT:
                break
        assert cb.CHFSI_ETIMEOUT in codes, codes
        assert all(c in (cb.CHFSI_OK, cb.CHFSI_ETIMEOUT) for c in codes), codes
        cb.chfsi_set_wait_limit(s.ctx, 0)
        got = cb.chfsi_filter_split(s.ctx, H, Y, degs, -2.0, -1.0, 2.5, 7).cpu().numpy()
    ref = O.chebyshev_filter(H.cpu().numpy(), Y.cpu().numpy(), degs, -2.0, -1.0, 2.5)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_loop_limit_reports_the_locked_prefix_like_the_oracle():
    """blk = nev leaves the nev-th wanted value at the edge of the damped interval, so within
    20 loops only a prefix locks (the oracle's pin of the same case)."""
    seq = inputs.planted_sequence("c1", n=96, N=1, nev=6, blk=10)
    p = seq.problems[0]
    A, B = torch.tril(p.A), torch.tril(p.B)
    ref, _, _, st_ref = O.chfsi_solve(A.numpy(), B.numpy(), 8, 8, 1e-10, deg=10, max_loops=20)
    with cb.Solver(96, 10, max_loops=20) as s:
        with pytest.raises(cb.ChfsiError) as ei:
            cb.chfsi_solve_next(s.ctx, A.to(DEV), B.to(DEV), 8, 8, 10)
        assert ei.value.code == cb.CHFSI_ENOCONV
        lam, _, st = ei.value.partial
        lam = lam.cpu().numpy()
        done = np.isfinite(lam)
        k = int(done.sum())
        assert st["loops"] == 20 and 0 < k < 8
        assert np.all(done[:k]) and not np.any(done[k:])   # a contiguous prefix, the rest NaN
        assert abs(k - int(np.isfinite(ref).sum())) <= 1
        assert np.max(np.abs(lam[:k] - p.lam[:k])) <= 1e-10 * np.max(np.abs(p.lam))
        # the context stays usable: a well-posed solve on it converges
        cb.chfsi_reset_warm_state(s.ctx)
        lam2, X2, st2 = cb.chfsi_solve_next(s.ctx, A.to(DEV), B.to(DEV), 6, 10, 10)
    assert np.max(np.abs(lam2.cpu().numpy() - p.lam[:6])) <= 1e-10 * np.max(np.abs(p.lam))
    assert st2["max_resid"] <= 1e-10


def test_unreachable_tolerance_reports_no_convergence():
    """A tolerance below what FP64 arithmetic can reach (1e-18 on the n = 512 workload) is
    reported as CHFSI_ENOCONV — never as success — with the pairs that did lock finite and
    the rest NaN, and the context solves a well-posed problem afterwards."""
    seq = inputs.planted_sequence("c1", N=1, keep_vectors=False)
    p = seq.problems[0]
    A, B = torch.tril(p.A).to(DEV), torch.tril(p.B).to(DEV)
    with cb.Solver(seq.n, seq.blk, max_loops=25) as s:
        with pytest.raises(cb.ChfsiError) as ei:
            cb.chfsi_solve_next(s.ctx, A, B, seq.nev, seq.blk, seq.deg, tol=1e-18)
        assert ei.value.code == cb.CHFSI_ENOCONV
        lam, _, st = ei.value.partial
        lam = lam.cpu().numpy()
        done = np.isfinite(lam)
        k = int(done.sum())
        assert np.all(done[:k]) and not np.any(done[k:])
        assert k < seq.nev
        cb.chfsi_reset_warm_state(s.ctx)
        lam2, _, st2 = cb.chfsi_solve_next(s.ctx, A, B, seq.nev, seq.blk, seq.deg, tol=seq.tol)
    assert np.max(np.abs(lam2.cpu().numpy() - p.lam[:seq.nev])) <= 1e-10 * np.max(np.abs(p.lam))
    assert st2["max_resid"] <= seq.tol
