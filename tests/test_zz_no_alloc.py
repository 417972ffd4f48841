"""The allocation-free eigensolver entry point agrees with the context-based one.

chfsi_heev_noalloc is for callers that cannot call cudaMalloc (for example an application
whose pool allocator owns all device memory) and so cannot create a context; it keeps its
scratch in a fixed device array shared by all calls.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import math

import numpy as np
import pytest
import torch

from paper_1206_3768_gb300 import binding as cb

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _herm(seed, m):
    rng = np.random.default_rng(seed)
    M = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / math.sqrt(2)
    return torch.from_numpy(0.5 * (M + M.conj().T)).to(DEV)


def _compare(w, V, w_ref, V_ref, G):
    w, V, w_ref, V_ref, G = (t.cpu().numpy() for t in (w, V, w_ref, V_ref, G))
    m = G.shape[0]
    nrm = np.linalg.norm(G, 2)
    tol = 1e-13 * nrm * max(1.0, math.sqrt(m))
    assert np.max(np.abs(w - w_ref)) <= tol
    assert np.max(np.abs(G @ V - V * w[None, :])) <= tol
    assert np.max(np.abs(V.conj().T @ V - np.eye(m))) <= 1e-13 * max(1.0, math.sqrt(m))
    # eigenvectors agree with the context path up to phase where eigenvalues are separated
    gaps = np.minimum(np.diff(np.r_[-np.inf, w_ref]), np.diff(np.r_[w_ref, np.inf]))
    ov = np.abs(np.sum(V.conj() * V_ref, axis=0))
    assert np.all(np.abs(ov[gaps > 1e-8 * nrm] - 1.0) < 1e-9)


def test_noalloc_matches_context_heev_on_two_calls_in_a_row():
    with cb.Solver(256, cb.HEEV_NOALLOC_MAX) as s:
        for seed, m in ((1, 100), (2, cb.HEEV_NOALLOC_MAX)):
            G = _herm(seed, m)
            w_ref, V_ref = cb.chfsi_heev(s.ctx, G)
            w, V = cb.chfsi_heev_noalloc(G)
            _compare(w, V, w_ref, V_ref, G)


def test_noalloc_small_and_odd_sizes_after_a_full_size_call():
    # the array keeps the previous call's contents: a full-size call first, then sizes whose
    # padded work copies (odd m adds a row and a column) cover only part of it
    with cb.Solver(256, cb.HEEV_NOALLOC_MAX) as s:
        for seed, m in ((4, cb.HEEV_NOALLOC_MAX), (5, 1), (6, cb.HEEV_NOALLOC_MAX - 1), (7, 3)):
            G = _herm(seed, m)
            w_ref, V_ref = cb.chfsi_heev(s.ctx, G)
            w, V = cb.chfsi_heev_noalloc(G)
            _compare(w, V, w_ref, V_ref, G)


def test_noalloc_strided_input_and_side_stream():
    # G as a column-major view with leading dimension above m, on a non-default stream
    m = 77
    G = _herm(8, m)
    big = cb.fortran_empty(m + 9, m, DEV)
    big.zero_()
    view = big[:m, :]
    view.copy_(G)
    assert view.stride(0) == 1 and view.stride(1) == m + 9
    side = torch.cuda.Stream(device=DEV)
    side.wait_stream(torch.cuda.current_stream())
    with cb.Solver(256, cb.HEEV_NOALLOC_MAX) as s:
        w_ref, V_ref = cb.chfsi_heev(s.ctx, G)
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            w, V = cb.chfsi_heev_noalloc(view)
        torch.cuda.current_stream().wait_stream(side)
        _compare(w, V, w_ref, V_ref, G)


def test_noalloc_rejects_sizes_beyond_its_array():
    G = _herm(3, cb.HEEV_NOALLOC_MAX + 1)
    with pytest.raises(cb.ChfsiError) as ei:
        cb.chfsi_heev_noalloc(G)
    assert ei.value.code == cb.CHFSI_EINVAL
