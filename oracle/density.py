"""Definition of the zero-temperature density matrix and its first-order response.

Test infrastructure only (see the package docstring): nothing in the product path
imports this module.

All arithmetic is float64 NumPy/LAPACK.  The density matrix is the one the SP2
chain converges to, written out from its definition:

* Eq. DM-outer-product (section "The density matrix"):
  D_ij = sum_k f_k c_i^(k) c_j^(k), with f_k = 1 for the n_occ lowest
  eigenstates of the orthogonalised Hamiltonian and 0 for the others.
* Eq. theta: D = theta(mu I - H), the step placed at the chemical potential mu
  between the occupied and unoccupied eigenvalues.  mu is reported mid-gap; D
  does not depend on where in the gap it sits.

The response D1 = dD/dH [H1] and the adjoint dTr[D G]/dH are not given in the
paper; they follow from first-order perturbation theory of a spectral projector:
D1 = C (C^T H1 C  o  F) C^T with F_ij = (f_i - f_j)/(eps_i - eps_j) for
f_i != f_j and 0 otherwise ("o" is the element-wise product).  This map is
self-adjoint in the Frobenius inner product, so the adjoint of a symmetric weight
G is the same formula applied to sym(G).
"""
from __future__ import annotations

import numpy as np


def eigensystem(H: np.ndarray):
    """Ascending eigenvalues and orthonormal eigenvectors (columns) of symmetric H."""
    H = np.asarray(H, dtype=np.float64)
    lam, C = np.linalg.eigh(H)
    return lam, C


def occupations(n: int, n_occ: int) -> np.ndarray:
    """f_k of Eq. DM-outer-product at zero temperature: 1 for the n_occ lowest states."""
    if not 0 <= n_occ <= n:
        raise ValueError("n_occ must lie in [0, n]")
    f = np.zeros(n)
    f[:n_occ] = 1.0
    return f


def density_from_eigensystem(C: np.ndarray, n_occ: int) -> np.ndarray:
    """D_ij = sum_k f_k C_ik C_jk (Eq. DM-outer-product) for ascending columns C."""
    c_occ = np.asarray(C, dtype=np.float64)[:, :n_occ]
    return c_occ @ c_occ.T


def density_matrix(H: np.ndarray, n_occ: int) -> np.ndarray:
    """D = theta(mu I - H) (Eq. theta) by dense symmetric eigendecomposition."""
    lam, C = eigensystem(H)
    return density_from_eigensystem(C, n_occ)


def density_rows(C: np.ndarray, n_occ: int, rows) -> np.ndarray:
    """Selected rows of D from an eigensystem, one by one (for very large N)."""
    c_occ = np.asarray(C, dtype=np.float64)[:, :n_occ]
    rows = np.asarray(rows)
    return c_occ[rows] @ c_occ.T


def chemical_potential(lam: np.ndarray, n_occ: int) -> float:
    """mu placed mid-gap between the highest occupied and lowest unoccupied eigenvalue."""
    n = len(lam)
    if n_occ == 0:
        return -np.inf
    if n_occ == n:
        return np.inf
    return 0.5 * (lam[n_occ - 1] + lam[n_occ])


def homo_lumo_gap(lam: np.ndarray, n_occ: int) -> float:
    if n_occ in (0, len(lam)):
        return np.inf
    return float(lam[n_occ] - lam[n_occ - 1])


def band_energy(D: np.ndarray, H: np.ndarray) -> float:
    """Tr[D H] in float64 for symmetric D and H (sum of element-wise products)."""
    return float(np.sum(np.asarray(D, np.float64) * np.asarray(H, np.float64)))


def response_weights(lam: np.ndarray, n_occ: int) -> np.ndarray:
    """F_ij = (f_i - f_j)/(eps_i - eps_j) where f_i != f_j, else 0."""
    n = len(lam)
    f = occupations(n, n_occ)
    df = f[:, None] - f[None, :]
    de = lam[:, None] - lam[None, :]
    cross = df != 0
    if np.any(de[cross] == 0):
        raise ValueError("no gap between occupied and unoccupied eigenvalues")
    F = np.zeros((n, n))
    F[cross] = df[cross] / de[cross]
    return F


def symmetrise(A: np.ndarray) -> np.ndarray:
    A = np.asarray(A, dtype=np.float64)
    return 0.5 * (A + A.T)


def response(H: np.ndarray, H1: np.ndarray, n_occ: int) -> np.ndarray:
    """First-order response D1 = dD/dH [H1] for a symmetric perturbation H1."""
    lam, C = eigensystem(H)
    return response_from_eigensystem(lam, C, H1, n_occ)


def response_from_eigensystem(lam, C, H1, n_occ) -> np.ndarray:
    F = response_weights(lam, n_occ)
    h1 = C.T @ symmetrise(H1) @ C
    return C @ (h1 * F) @ C.T


def response_rows(lam, C, H1, n_occ: int, rows) -> np.ndarray:
    """Selected rows of D1 = C (C^T H1 C  o  F) C^T, for very large N.

    F is nonzero only between an occupied state o and an unoccupied state v, where
    F_ov = F_vo = 1/(eps_o - eps_v).  With C = [C_o  C_v] and W = (C_o^T H1 C_v) o F_ov
    the formula reads D1 = C_o W C_v^T + C_v W^T C_o^T, of which only the requested
    rows are formed.
    """
    lam = np.asarray(lam, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    rows = np.asarray(rows)
    f = occupations(len(lam), n_occ)
    occ, virt = f == 1.0, f == 0.0
    Co, Cv = C[:, occ], C[:, virt]
    gap = lam[occ][:, None] - lam[virt][None, :]
    if np.any(gap == 0):
        raise ValueError("no gap between occupied and unoccupied eigenvalues")
    W = (Co.T @ (symmetrise(H1) @ Cv)) / gap
    return Co[rows] @ W @ Cv.T + Cv[rows] @ W.T @ Co.T


def adjoint(H: np.ndarray, G: np.ndarray, n_occ: int) -> np.ndarray:
    """Gradient of Tr[D(H) G] with respect to symmetric H (self-adjoint response)."""
    return response(H, symmetrise(G), n_occ)


# -- non-orthogonal basis (section "The density matrix": H_orth = Z^T H Z, D = Z D_orth Z^T) --

def density_matrix_generalized(H: np.ndarray, S: np.ndarray, n_occ: int) -> np.ndarray:
    """D = sum_k f_k c_k c_k^T for H c = eps S c with C^T S C = I (Eq. KS-matrix, Eq. DM-outer-product)."""
    import scipy.linalg

    lam, C = scipy.linalg.eigh(np.asarray(H, np.float64), np.asarray(S, np.float64))
    return density_from_eigensystem(C, n_occ)


def inverse_factor_lowdin(S: np.ndarray) -> np.ndarray:
    """Z = S^(-1/2), one inverse factor with Z^T S Z = I."""
    lam, U = np.linalg.eigh(np.asarray(S, np.float64))
    return (U / np.sqrt(lam)) @ U.T


def inverse_factor_cholesky(S: np.ndarray) -> np.ndarray:
    """Z = L^(-T) from S = L L^T, another inverse factor with Z^T S Z = I."""
    L = np.linalg.cholesky(np.asarray(S, np.float64))
    return np.linalg.inv(L).T


def density_matrix_via_factor(H: np.ndarray, Z: np.ndarray, n_occ: int) -> np.ndarray:
    """D = Z theta(mu I - Z^T H Z) Z^T (the orthogonalised route of section "The density matrix")."""
    Z = np.asarray(Z, np.float64)
    Hp = Z.T @ np.asarray(H, np.float64) @ Z
    return Z @ density_matrix(symmetrise(Hp), n_occ) @ Z.T
