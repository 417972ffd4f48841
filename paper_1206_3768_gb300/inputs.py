"""Seeded synthetic inputs: sequences of correlated generalized Hermitian pencils.

The paper's experiments run on FLEUR-generated sequences (Table 1: CaFe2As2, Au98Ag10,
Na15Cl14Li) that are not available here.  This module builds stand-ins with the same
structure and a *planted* spectrum, so that every problem has a known exact answer:

    B = I + alpha * G^H G            (HPD overlap, fixed along the sequence)
    B = L L^H                        (Cholesky factor of the generator, not of the method)
    A^(l) = L Q_l diag(lam_l) Q_l^H L^H

so the pencil A^(l) x = lam B x (Eq. 1, Section 1) has eigenvalues lam_l and
B-orthonormal eigenvectors X_l = L^{-H} Q_l.  Correlation between neighbouring problems
(the property of Section 2.2, Eq. 9) is emulated by a small unitary rotation of the
eigenvectors and a small drift of the eigenvalues:

    Q_l = Q_{l-1} expm(i eps_l K_l),  K_l = (G + G^H) / (2 sqrt(n)),  eps_l = 1e-2 * 0.5**l
    lam_l = sort(lam_{l-1} + 1e-3 * N(0, 1))  (pairs re-sorted together)

For the large workloads (n above DENSE_ROTATION_MAX_N) the dense rotation would cost an
n x n Hermitian eigendecomposition and three n^3 products per problem in FP64 (about 35 s
per problem at n = 9300 on one GB300), so there Q_l = Q_{l-1} U_l with U_l a product of
ROTATION_LAYERS layers of 2 x 2 unitary rotations between randomly paired columns, angles
N(0, 1) eps_l / sqrt(2 ROTATION_LAYERS) and random phases: exactly unitary, applied in
O(n^2) per layer, and giving each eigenvector the same first-order deviation angle as the
dense rotation (about eps_l / sqrt(2)).  A^(l) = M_l diag(lam_l) M_l^H with M_l = L Q_l kept
up to date by the same rotations, so one n^3 product (lower block triangle only) remains.

All random draws come from numpy's PCG64 seeded by SeedSequence(12063768 + config_id);
the dense linear algebra of the construction runs in torch on any device, so the CPU
and GPU builds of one sequence see the same random numbers.  Nothing here is part of
the eigensolver: it only builds inputs and their planted answers.

Matrices are returned as torch complex128 tensors in natural (row, column) indexing.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

SEED_BASE = 12063768

# Workloads: sizes and spectra of the five synthetic configurations.
CONFIGS = {
    # n=512 plain method, three problems, fixed degree 10.
    "c1": dict(config_id=1, n=512, nev=20, blk=30, deg=10, deg_min=10, deg_max=10, N=3,
               spectrum="uniform_cluster", overlap="mild", tol=1e-10),
    # n=2600 FLAPW-shaped, 20 problems, adaptive degree in [8, 25], cond(B) = 1e4.
    "c2": dict(config_id=2, n=2600, nev=100, blk=130, deg=0, deg_min=8, deg_max=25, N=20,
               spectrum="dense_low", overlap="kappa", kappa=1e4, tol=1e-10),
    # n=9300 mixed-precision workload, generated like c1.
    "c3": dict(config_id=3, n=9300, nev=256, blk=320, deg=20, deg_min=20, deg_max=20, N=20,
               spectrum="uniform_cluster", overlap="mild", tol=1e-10),
    # one k-point of the batched workload (kpoint_sequences draws n per k-point), like c1.
    "c4": dict(config_id=4, n=4500, nev=180, blk=234, deg=20, deg_min=20, deg_max=20, N=10,
               spectrum="uniform_cluster", overlap="mild", tol=1e-10),
    # n=13400 learned-degree workload: degrees in [4, 40], generated like c1.
    "c5": dict(config_id=5, n=13400, nev=1000, blk=1200, deg=0, deg_min=4, deg_max=40, N=20,
               spectrum="uniform_cluster", overlap="mild", tol=1e-10),
}

# Largest n built with the dense correlation rotation expm(i eps K); larger problems use the
# layered pairwise rotations described in the module docstring.
DENSE_ROTATION_MAX_N = 3000
ROTATION_LAYERS = 8


def _preload_cuda_linalg():
    """Load torch's CUDA linear-algebra library by absolute path once, so that the lazy
    load inside torch.linalg also works under tools that change the library search path
    (a profiler launching the benchmark)."""
    import ctypes
    import os

    lib = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(lib):
        try:
            ctypes.CDLL(lib, mode=ctypes.RTLD_GLOBAL)
        except OSError:
            pass


def _rng(config_id: int, stream: int = 0) -> np.random.Generator:
    ss = np.random.SeedSequence([SEED_BASE + config_id, stream])
    return np.random.Generator(np.random.PCG64(ss))


def complex_gaussian(rng: np.random.Generator, shape) -> np.ndarray:
    """(N(0,1) + i N(0,1)) / sqrt(2): unit expected squared modulus."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) / math.sqrt(2.0)


def planted_spectrum(rng, n: int, kind: str, nev: int) -> np.ndarray:
    """Sorted planted eigenvalues with a guaranteed gap after the nev-th value."""
    if kind == "uniform_cluster":
        # 95% uniform in [-2, 2], 5% clustered within 1e-3 of -1.
        nc = max(1, int(round(0.05 * n)))
        lam = np.concatenate([2.0 * rng.uniform(-1.0, 1.0, n - nc),
                              -1.0 + 1e-3 * rng.uniform(-1.0, 1.0, nc)])
    elif kind == "cluster_low":
        # Variant: the 5% cluster sits at the bottom of the spectrum, among the wanted values.
        nc = max(1, int(round(0.05 * n)))
        lam = np.concatenate([2.0 * rng.uniform(-1.0, 1.0, n - nc),
                              -2.0 + 1e-3 * rng.uniform(-1.0, 1.0, nc)])
    elif kind == "dense_low":
        # 10% dense in [-1, -0.6], the rest uniform in [-0.6, 30].
        nl = int(round(0.10 * n))
        lam = np.concatenate([rng.uniform(-1.0, -0.6, nl), rng.uniform(-0.6, 30.0, n - nl)])
    else:
        raise ValueError(f"unknown spectrum kind {kind!r}")
    return _enforce_gap(np.sort(lam), nev)


def _enforce_gap(lam: np.ndarray, nev: int) -> np.ndarray:
    """Keep lam[nev] - lam[nev-1] >= 1e-6 * max|lam| so the wanted set is well defined."""
    if nev >= lam.size:
        return lam
    thr = 1e-6 * float(np.max(np.abs(lam)))
    lam = lam.copy()
    if lam[nev] - lam[nev - 1] < thr:
        lam[nev:] = np.maximum(lam[nev:], lam[nev - 1] + thr)
        lam = np.sort(lam)
    return lam


@dataclass
class Problem:
    A: torch.Tensor          # n x n Hermitian (full storage), complex128
    B: torch.Tensor          # n x n HPD (full storage), complex128
    lam: np.ndarray          # planted eigenvalues, ascending (all n)
    X: torch.Tensor | None   # planted B-orthonormal eigenvectors L^{-H} Q (n x n) or None


@dataclass
class Sequence:
    n: int
    nev: int
    blk: int
    deg: int
    deg_min: int
    deg_max: int
    tol: float
    problems: list = field(default_factory=list)
    name: str = ""


def _haar_unitary(rng, n: int, device) -> torch.Tensor:
    Z = torch.from_numpy(complex_gaussian(rng, (n, n))).to(device)
    Q, R = torch.linalg.qr(Z)
    d = torch.diagonal(R)
    ph = d / d.abs()
    return Q * ph.unsqueeze(0)


def _overlap(rng, n: int, kind: str, kappa: float, device) -> torch.Tensor:
    G = torch.from_numpy(complex_gaussian(rng, (n, n))).to(device)
    GhG = G.conj().T @ G
    GhG = 0.5 * (GhG + GhG.conj().T)
    eye = torch.eye(n, dtype=torch.complex128, device=device)
    if kind == "mild":
        return eye + (0.1 / n) * GhG
    if kind == "kappa":
        mu = torch.linalg.eigvalsh(GhG)
        mu_min, mu_max = float(mu[0]), float(mu[-1])
        alpha = (kappa - 1.0) / (mu_max - kappa * mu_min)
        if alpha <= 0:
            raise ValueError("cannot reach the requested condition number")
        return eye + alpha * GhG
    raise ValueError(f"unknown overlap kind {kind!r}")


def _rotation_layers(rng, n: int, eps: float):
    """Random pairings and 2 x 2 unitary rotations [[c, -conj(w) s], [w s, c]] (c = cos phi,
    s = sin phi, w = exp(i psi)) of ROTATION_LAYERS layers, drawn from rng."""
    layers = []
    sig = eps / math.sqrt(2.0 * ROTATION_LAYERS)
    for _ in range(ROTATION_LAYERS):
        perm = rng.permutation(n)
        half = n // 2
        ia, ib = perm[:half], perm[half:2 * half]
        phi = sig * rng.standard_normal(half)
        psi = rng.uniform(0.0, 2.0 * math.pi, half)
        layers.append((ia, ib, np.cos(phi), np.sin(phi) * np.exp(1j * psi)))
    return layers


def _apply_layers(M: torch.Tensor, layers) -> torch.Tensor:
    """M <- M U for the rotation layers (columns a, b of each pair mixed: new a = c a + ws b,
    new b = -conj(ws) a + c b), applied in place."""
    dev = M.device
    for ia, ib, c, ws in layers:
        ta = torch.from_numpy(ia).to(dev)
        tb = torch.from_numpy(ib).to(dev)
        tc = torch.from_numpy(c).to(dev).to(M.dtype)
        tw = torch.from_numpy(ws).to(dev)
        Ma, Mb = M[:, ta], M[:, tb]
        M[:, ta] = Ma * tc + Mb * tw
        M[:, tb] = Mb * tc - Ma * tw.conj()
    return M


def _herm_product(M: torch.Tensor, lam: np.ndarray, blocks: int = 8) -> torch.Tensor:
    """M diag(lam) M^H from the products of its lower block triangle (about half the flops
    of the full product), completed to full Hermitian storage."""
    n = M.shape[0]
    lam_t = torch.from_numpy(lam).to(M.device).to(M.dtype)
    ML = M * lam_t.unsqueeze(0)
    A = torch.zeros((n, n), dtype=M.dtype, device=M.device)
    edges = [round(n * k / blocks) for k in range(blocks + 1)]
    for k in range(blocks):
        r0, r1 = edges[k], edges[k + 1]
        A[r0:r1, :r1] = ML[r0:r1] @ M[:r1].conj().T
    A = torch.tril(A) + torch.tril(A, -1).conj().T
    A.diagonal().imag.zero_()
    return A


def planted_sequence(name: str = "c1", *, n: int | None = None, N: int | None = None,
                     nev: int | None = None, blk: int | None = None,
                     spectrum: str | None = None, device="cpu",
                     keep_vectors: bool = True, seed_offset: int = 0,
                     rotation: str | None = None) -> Sequence:
    """Build a seeded correlated sequence for one of the configurations in CONFIGS.

    ``n``, ``N``, ``nev``, ``blk`` and ``spectrum`` override the configuration's values
    (used for small test cases with the same structure).  ``rotation`` ("dense" or "layers")
    overrides the choice by size (dense up to DENSE_ROTATION_MAX_N).  ``keep_vectors``: True
    (planted eigenvectors of every problem), False, or a collection of problem indices.
    """
    want_x = (lambda ell: True) if keep_vectors is True else (
        (lambda ell: False) if not keep_vectors else (lambda ell, s=frozenset(keep_vectors): ell in s))
    cfg = dict(CONFIGS[name])
    n = int(n or cfg["n"])
    N = int(N or cfg["N"])
    nev = int(nev or cfg["nev"])
    blk = int(blk or cfg["blk"])
    spectrum = spectrum or cfg["spectrum"]
    rotation = rotation or ("dense" if n <= DENSE_ROTATION_MAX_N else "layers")
    cid = cfg["config_id"] + 1000 * seed_offset
    rng = _rng(cid)
    dev = torch.device(device)
    if dev.type == "cuda":
        _preload_cuda_linalg()

    B = _overlap(rng, n, cfg["overlap"], cfg.get("kappa", 1e4), dev)
    Lg = torch.linalg.cholesky(B)
    Q = _haar_unitary(rng, n, dev)
    lam = planted_spectrum(rng, n, spectrum, nev)
    seq = Sequence(n=n, nev=nev, blk=blk, deg=cfg["deg"], deg_min=cfg["deg_min"],
                   deg_max=cfg["deg_max"], tol=cfg["tol"], name=name)
    M = Lg @ Q if rotation == "layers" else None
    if M is not None and not keep_vectors:
        del Q
        Q = None
    for ell in range(N):
        if ell > 0:
            eps = 1e-2 * 0.5 ** ell
            if rotation == "layers":
                layers = _rotation_layers(rng, n, eps)
                M = _apply_layers(M, layers)
                if Q is not None:
                    Q = _apply_layers(Q, layers)
            else:
                Gk = torch.from_numpy(complex_gaussian(rng, (n, n))).to(dev)
                K = (Gk + Gk.conj().T) / (2.0 * math.sqrt(n))
                kap, V = torch.linalg.eigh(K)
                U = (V * torch.exp(1j * eps * kap).unsqueeze(0)) @ V.conj().T
                Q = Q @ U
            lam = lam + 1e-3 * rng.standard_normal(n)
            order = np.argsort(lam, kind="stable")
            lam = _enforce_gap(lam[order], nev)
            idx = torch.from_numpy(order).to(dev)
            if M is not None:
                M = M[:, idx]
            if Q is not None:
                Q = Q[:, idx]
        if rotation == "layers":
            A = _herm_product(M, lam)
        else:
            LQ = Lg @ Q
            lam_t = torch.from_numpy(lam).to(dev).to(torch.complex128)
            A = (LQ * lam_t.unsqueeze(0)) @ LQ.conj().T
            A = 0.5 * (A + A.conj().T)
        X = None
        if want_x(ell):
            X = torch.linalg.solve_triangular(Lg.conj().T, Q, upper=True)
        seq.problems.append(Problem(A=A, B=B, lam=lam.copy(), X=X))
    return seq


def gaussian_block(n: int, m: int, seed: int) -> torch.Tensor:
    """Seeded complex Gaussian n x m start block (the caller-supplied V0 of a cold start)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_BASE, 7, seed])))
    return torch.from_numpy(complex_gaussian(rng, (n, m)))


def kpoint_sequences(K: int = 32, N: int = 10, n_range=(3000, 6000), device="cpu",
                     keep_vectors: bool = False, seed: int = 0) -> list:
    """K independent k-point sequences of uneven size (the batched workload): n_k drawn
    uniformly from n_range (seeded), nev_k = ceil(0.04 n_k), blk_k = ceil(1.3 nev_k),
    each generated like "c4" with its own seed offset."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_BASE, 4, seed])))
    ns = rng.integers(int(n_range[0]), int(n_range[1]) + 1, size=K)
    out = []
    for k, n in enumerate(ns):
        nev = int(math.ceil(0.04 * int(n)))
        blk = int(math.ceil(1.3 * nev))
        out.append(planted_sequence("c4", n=int(n), N=N, nev=nev, blk=blk, device=device,
                                    keep_vectors=keep_vectors, seed_offset=k + 1))
    return out
