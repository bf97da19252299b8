"""Seeded synthetic Hamiltonians and perturbations for the SP2 density-matrix path.

The paper measures on SCC-DFTB Hamiltonians of periodic liquid-water boxes
(6 orbitals per H2O; sizes N = 6 * n_water up to 19 020, section "GPU and tensor
core performance").  Those matrices are not available, so every workload here is
a seeded synthetic stand-in with the same shape: a dense, symmetric,
orthogonalised N x N Hamiltonian with a spectral gap at the Fermi level.

This module only builds inputs.  It holds none of the density-matrix method's
arithmetic (no spectral projection, no purification, no response); it is shared
by the tests, the oracle checks and the benchmark so that both sides of every
comparison see bit-identical inputs.  Random numbers come from NumPy's PCG64
(``numpy.random.default_rng``) with seed ``1000 * config + instance``.

Recipes
-------
* ``gapped_random``   -- H = Q diag(lam) Q^T, Q from the QR factorisation of a
  seeded Gaussian matrix, n_occ eigenvalues uniform in [-1, -0.05] and the rest
  uniform in [0.05, 1] (gap 0.1).  The eigensystem is known by construction.
* ``banded_tight_binding`` -- onsite energies N(0, 0.5^2) and off-diagonal
  hoppings N(0, 0.1^2) * exp(-|i-j|/16) within |i-j| <= 64, symmetric; the gap at
  the Fermi level is then opened to at least ``min_gap`` by shifting every
  unoccupied eigenvalue up by the same amount and rebuilding H from its
  eigenvectors (the band structure becomes approximate, the matrix dense).
* ``banded_perturbation`` -- symmetric perturbation with the same band pattern,
  entries N(0, sigma^2).
* ``symmetric_gaussian`` -- symmetric weight matrix G = (A + A^T)/2.
* ``sparse_perturbation`` -- symmetric matrix with a Bernoulli(p) pattern on the
  upper triangle (diagonal included), entries N(0, sigma^2), mirrored.
* ``md_sequence`` -- H_k = H_0 + sin(omega k) V.
* ``batch_sizes`` -- instance sizes drawn uniformly from {128, 256, ..., 2048}.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


def rng_for(config: int, instance: int = 0) -> np.random.Generator:
    """PCG64 generator for workload ``config`` and instance ``instance``."""
    return np.random.default_rng(1000 * config + instance)


@dataclasses.dataclass
class Hamiltonian:
    """A synthetic orthogonalised Hamiltonian.

    ``H`` is float64, symmetric, row-major.  ``eigvals`` (ascending) and
    ``eigvecs`` (columns) are the eigensystem used to build ``H`` when the recipe
    constructs it from one, else ``None``.
    """

    H: np.ndarray
    n_occ: int
    eigvals: Optional[np.ndarray] = None
    eigvecs: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return self.H.shape[0]


def _rebuild(q: np.ndarray, lam: np.ndarray) -> np.ndarray:
    h = (q * lam) @ q.T
    return 0.5 * (h + h.T)


def gapped_random(n: int, n_occ: int, rng: np.random.Generator,
                  occ_range=(-1.0, -0.05), virt_range=(0.05, 1.0)) -> Hamiltonian:
    """Dense H with a prescribed spectrum and a random orthogonal eigenbasis."""
    if not 0 <= n_occ <= n:
        raise ValueError("n_occ must lie in [0, n]")
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(occ_range[0], occ_range[1], n_occ),
                          rng.uniform(virt_range[0], virt_range[1], n - n_occ)])
    order = np.argsort(lam, kind="stable")
    lam = lam[order]
    q = q[:, order]
    return Hamiltonian(_rebuild(q, lam), n_occ, lam, q)


def banded_matrix(n: int, rng: np.random.Generator, bandwidth: int = 64,
                  offdiag_sigma: float = 0.1, decay: float = 16.0,
                  onsite_sigma: float = 0.5) -> np.ndarray:
    """Symmetric banded tight-binding-like matrix (no gap enforcement)."""
    h = np.zeros((n, n))
    idx = np.arange(n)
    h[idx, idx] = rng.normal(0.0, onsite_sigma, n)
    for d in range(1, min(bandwidth, n - 1) + 1):
        v = rng.normal(0.0, offdiag_sigma, n - d) * np.exp(-d / decay)
        h[idx[:-d], idx[d:]] = v
        h[idx[d:], idx[:-d]] = v
    return h


def banded_tight_binding(n: int, rng: np.random.Generator, n_occ: Optional[int] = None,
                         min_gap: float = 0.05, **band_kw) -> Hamiltonian:
    """Banded H with the Fermi-level gap opened to at least ``min_gap``."""
    n_occ = n // 2 if n_occ is None else n_occ
    if not 0 < n_occ < n:
        raise ValueError("n_occ must lie in (0, n) for a gapped banded Hamiltonian")
    h = banded_matrix(n, rng, **band_kw)
    lam, q = np.linalg.eigh(h)
    shift = max(0.0, min_gap - (lam[n_occ] - lam[n_occ - 1]))
    lam = lam.copy()
    lam[n_occ:] += shift
    return Hamiltonian(_rebuild(q, lam), n_occ, lam, q)


def banded_perturbation(n: int, rng: np.random.Generator, bandwidth: int = 64,
                        sigma: float = 0.01) -> np.ndarray:
    """Symmetric perturbation H1 with entries N(0, sigma^2) inside the band."""
    h = np.zeros((n, n))
    idx = np.arange(n)
    h[idx, idx] = rng.normal(0.0, sigma, n)
    for d in range(1, min(bandwidth, n - 1) + 1):
        v = rng.normal(0.0, sigma, n - d)
        h[idx[:-d], idx[d:]] = v
        h[idx[d:], idx[:-d]] = v
    return h


def overlap_matrix(n: int, rng: np.random.Generator, bandwidth: int = 16, sigma: float = 0.05,
                   decay: float = 4.0) -> np.ndarray:
    """Symmetric positive-definite overlap S = I + banded off-diagonal terms.

    Off-diagonal entries N(0, sigma^2) exp(-|i-j|/decay) within the band; the
    band is scaled down if needed so that its row sums stay below 1/2, which
    keeps the eigenvalues of S inside [1/2, 3/2] (Gershgorin).
    """
    b = banded_matrix(n, rng, bandwidth=bandwidth, offdiag_sigma=sigma, decay=decay, onsite_sigma=0.0)
    np.fill_diagonal(b, 0.0)
    rmax = np.abs(b).sum(axis=1).max()
    if rmax > 0.5:
        b *= 0.5 / rmax
    return np.eye(n) + b


def symmetric_gaussian(n: int, rng: np.random.Generator) -> np.ndarray:
    a = rng.standard_normal((n, n))
    return 0.5 * (a + a.T)


def sparse_perturbation(n: int, rng: np.random.Generator, density: float = 0.01,
                        sigma: float = 0.02) -> np.ndarray:
    mask = np.triu(rng.random((n, n)) < density)
    v = np.where(mask, rng.normal(0.0, sigma, (n, n)), 0.0)
    return v + np.triu(v, 1).T


def md_sequence(h0: np.ndarray, v: np.ndarray, k: int, omega: float = 0.05) -> np.ndarray:
    return h0 + np.sin(omega * k) * v


def batch_sizes(count: int, rng: np.random.Generator, lo: int = 128, hi: int = 2048,
                step: int = 128) -> list:
    choices = np.arange(lo, hi + 1, step)
    return [int(x) for x in rng.choice(choices, size=count)]


# Named workloads -------------------------------------------------------------

def plain_sp2_workload(n: int = 256) -> Hamiltonian:
    """Dense gapped H, N = 256, n_occ = N/2, eigenvalues in [-1,-0.05] and [0.05,1]."""
    return gapped_random(n, n // 2, rng_for(0))


def water_like_workload(n: int = 4096) -> Hamiltonian:
    """Banded tight-binding stand-in for the water Hamiltonians, n_occ = N/2, gap >= 0.05."""
    return banded_tight_binding(n, rng_for(1), n // 2)


def batched_workload(count: int = 64) -> list:
    """``count`` gapped random Hamiltonians of sizes in {128, ..., 2048}, n_occ = N/2."""
    sizes = batch_sizes(count, rng_for(2, 10_000))
    return [gapped_random(n, n // 2, rng_for(2, i)) for i, n in enumerate(sizes)]


def differentiation_workload(n: int = 4096):
    """(H, H1, G) for the response and adjoint checks."""
    ham = water_like_workload(n)
    rng = rng_for(3)
    return ham, banded_perturbation(n, rng), symmetric_gaussian(n, rng)
