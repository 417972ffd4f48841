"""The seeded input recipe (CPU): the generator produces what the stated recipe says —
planted eigenpairs of the pencil, the overlap's condition number, the spectrum shapes, the
gap after the wanted set, the k-point size rules — and the same seeds give the same data."""
import math

import numpy as np
import torch

from paper_1206_3768_gb300 import inputs


def test_planted_pencil_and_overlap_condition_number():
    """c2 shape at a small size: A X = B X diag(lam), X^H B X = I, cond(B) = 1e4 exactly
    (alpha from the extreme eigenvalues of G^H G), B fixed along the sequence."""
    seq = inputs.planted_sequence("c2", n=240, N=2, nev=10, blk=13, device="cpu", keep_vectors=True)
    for p in seq.problems:
        A, B, X = p.A.numpy(), p.B.numpy(), p.X.numpy()
        assert np.allclose(A, A.conj().T, atol=0) and np.allclose(B, B.conj().T, atol=0)
        R = A @ X - (B @ X) * p.lam[None, :]
        assert np.max(np.abs(R)) < 1e-9 * np.max(np.abs(p.lam)) * np.linalg.norm(B, 2)
        assert np.allclose(X.conj().T @ B @ X, np.eye(240), atol=1e-9)
        mu = np.linalg.eigvalsh(B)
        assert abs(mu[-1] / mu[0] - 1e4) < 1e-6 * 1e4
    assert torch.equal(seq.problems[0].B, seq.problems[1].B)


def test_spectrum_shapes_and_gap():
    rng = inputs._rng(99)
    lam = inputs.planted_spectrum(rng, 1000, "dense_low", 40)
    assert np.all(np.diff(lam) >= 0)
    assert np.sum(lam < -0.6) == 100 and lam[0] >= -1.0 and lam[-1] <= 30.0
    lam = inputs.planted_spectrum(inputs._rng(98), 400, "uniform_cluster", 20)
    assert np.sum(np.abs(lam + 1.0) <= 1e-3) >= 20  # the 5% cluster near -1
    assert lam[0] >= -2.0 and lam[-1] <= 2.0
    # the gap after the nev-th value is at least 1e-6 max|lam|, even when the draw had none
    tight = np.sort(np.concatenate([np.linspace(-1, 0, 50), [0.0, 0.0], np.linspace(0.1, 1, 48)]))
    g = inputs._enforce_gap(tight, 51)
    assert g[51] - g[50] >= 1e-6 * np.max(np.abs(g)) * (1 - 1e-12)
    assert np.array_equal(inputs._enforce_gap(g, 51), g)


def test_sequences_are_seeded_and_correlated():
    """Same name and seed: identical data; another seed offset: another sequence; the
    eigenvectors of neighbouring problems differ by rotations of the scale eps_l."""
    s1 = inputs.planted_sequence("c1", n=80, N=3, nev=5, blk=8, device="cpu", keep_vectors=True)
    s2 = inputs.planted_sequence("c1", n=80, N=3, nev=5, blk=8, device="cpu", keep_vectors=True)
    s3 = inputs.planted_sequence("c1", n=80, N=3, nev=5, blk=8, device="cpu", keep_vectors=True,
                                 seed_offset=1)
    for a, b in zip(s1.problems, s2.problems):
        assert torch.equal(a.A, b.A) and torch.equal(a.B, b.B)
    assert not torch.equal(s1.problems[0].A, s3.problems[0].A)
    B = s1.problems[0].B.numpy()
    for l in (1, 2):
        eps = 1e-2 * 0.5 ** l
        X0, X1 = s1.problems[l - 1].X.numpy(), s1.problems[l].X.numpy()
        M = np.abs(X0.conj().T @ B @ X1)
        # the eigenvalue drift re-sorts the pairs: each previous vector has one partner
        # (a permutation), overlapping to 1 - O(eps^2), and every other overlap is O(eps)
        assert np.array_equal(np.sort(np.argmax(M, axis=1)), np.arange(80))
        srt = np.sort(M, axis=1)
        assert np.all(srt[:, -1] > 1 - eps ** 2) and np.all(srt[:, -2] < eps)


def test_kpoint_sizes_follow_the_rules():
    seqs = inputs.kpoint_sequences(K=4, N=2, n_range=(60, 120), device="cpu")
    again = inputs.kpoint_sequences(K=4, N=2, n_range=(60, 120), device="cpu")
    ns = [s.n for s in seqs]
    assert ns == [s.n for s in again]
    assert all(60 <= n <= 120 for n in ns)
    for s in seqs:
        assert s.nev == math.ceil(0.04 * s.n) and s.blk == math.ceil(1.3 * s.nev)
        assert len(s.problems) == 2 and s.problems[0].A.shape == (s.n, s.n)
    assert len({float(s.problems[0].A[0, 0].real) for s in seqs}) == 4  # independent k-points


def test_layered_rotations_keep_the_pencil_planted_and_the_deviation_scale():
    """The layered pairwise rotations used for large n: exactly unitary (planted eigenpairs and
    B-orthonormality at rounding level), Hermitian A from the lower block triangle, and a
    median deviation angle between neighbouring eigenvectors of eps_l / sqrt(2), as with the
    dense rotation expm(i eps K)."""
    for rot in ("layers", "dense"):
        s = inputs.planted_sequence("c1", n=300, N=4, nev=10, blk=16, keep_vectors=True, rotation=rot)
        B = s.problems[0].B.numpy()
        for ell, p in enumerate(s.problems):
            A, X = p.A.numpy(), p.X.numpy()
            assert np.array_equal(A, A.conj().T)
            assert np.max(np.abs(A @ X - (B @ X) * p.lam[None, :])) < 1e-11 * np.max(np.abs(p.lam))
            assert np.allclose(X.conj().T @ B @ X, np.eye(300), atol=1e-10)
            if ell:
                M = np.abs(s.problems[ell - 1].X.numpy().conj().T @ B @ X)
                top = np.sort(M, axis=1)[:, -1]
                ang = np.median(np.sqrt(np.maximum(0.0, 1.0 - top ** 2)))
                eps = 1e-2 * 0.5 ** ell
                assert 0.8 < ang / (eps / math.sqrt(2)) < 1.2, (rot, ell, ang)
    big = inputs.planted_sequence("c1", n=inputs.DENSE_ROTATION_MAX_N + 1, N=1, nev=4, blk=6,
                                  keep_vectors=False)
    assert big.problems[0].A.shape[0] == inputs.DENSE_ROTATION_MAX_N + 1  # the layered path runs
