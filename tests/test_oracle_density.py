"""Pins for oracle/density.py: closed forms, hand-derived fixtures and invariants.

These tie the eigendecomposition definition of D = theta(mu I - H)
(Eq. DM-outer-product, Eq. theta) and its perturbation-theory response to facts
that do not come from the oracle itself.
"""
import numpy as np
import pytest

from oracle import density
from paper_2107_02737_gb300 import inputs
from tests._golden import load


def test_golden_2x2():
    g = load("density_2x2.txt")
    H = g["H"].reshape(2, 2)
    D = density.density_matrix(H, int(g["n_occ"]))
    np.testing.assert_allclose(D, g["D"].reshape(2, 2), atol=1e-15)
    lam, _ = density.eigensystem(H)
    assert density.chemical_potential(lam, 1) == pytest.approx(g["mu"], abs=1e-15)
    assert density.band_energy(D, H) == pytest.approx(g["band_energy"], abs=1e-14)


def test_golden_3x3_rational_basis():
    g = load("density_3x3.txt")
    H = g["H9"].reshape(3, 3) / 9.0
    lam, _ = density.eigensystem(H)
    for k in (1, 2):
        D = density.density_matrix(H, k)
        np.testing.assert_allclose(D, g[f"D9_occ{k}"].reshape(3, 3) / 9.0, atol=1e-14)
        assert density.chemical_potential(lam, k) == pytest.approx(g[f"mu_occ{k}"], abs=1e-14)
        assert density.band_energy(D, H) == pytest.approx(g[f"band_energy_occ{k}"], abs=1e-14)


def test_golden_3x3_rows_and_gap():
    """density_rows and homo_lumo_gap, which the full-size GPU checks use, against the
    hand-derived basis: any selection of rows, in any order, of D9 / 9, and the gaps 3, 2."""
    g = load("density_3x3.txt")
    C = g["Q3"].reshape(3, 3) / 3.0
    for k in (1, 2):
        ref = g[f"D9_occ{k}"].reshape(3, 3) / 9.0
        for rows in ([0], [2, 0], [1, 2, 0], [1, 1]):
            np.testing.assert_allclose(density.density_rows(C, k, rows), ref[rows], atol=1e-15)
        assert density.homo_lumo_gap(g["lam"], k) == g[f"gap_occ{k}"]
    assert density.homo_lumo_gap(g["lam"], 0) == np.inf
    assert density.homo_lumo_gap(g["lam"], 3) == np.inf
    np.testing.assert_array_equal(density.density_rows(C, 0, [1]), np.zeros((1, 3)))


def test_rows_and_gap_of_a_generated_spectrum():
    """On a generated Hamiltonian with a known spectrum: the rows equal those of the full
    outer product, and the gap is the one the generator opened (0.1 in this recipe)."""
    ham = inputs.gapped_random(40, 17, inputs.rng_for(9, 40))
    full = density.density_from_eigensystem(ham.eigvecs, 17)
    rows = [39, 0, 17, 16]
    np.testing.assert_allclose(density.density_rows(ham.eigvecs, 17, rows), full[rows], atol=1e-14)
    lam, _ = density.eigensystem(ham.H)
    gap = density.homo_lumo_gap(lam, 17)
    assert gap == pytest.approx(ham.eigvals[17] - ham.eigvals[16], abs=1e-12)
    assert gap >= 0.1 - 1e-12


def _closed_form_2x2(a, b, c):
    # Lower eigenvector projector of [[a, b], [b, c]]: D = I/2 - (H - (a+c)/2 I)/(2r).
    r = np.sqrt(((a - c) / 2) ** 2 + b * b)
    H = np.array([[a, b], [b, c]])
    return 0.5 * np.eye(2) - (H - 0.5 * (a + c) * np.eye(2)) / (2 * r)


@pytest.mark.parametrize("seed", range(5))
def test_two_by_two_closed_form(seed):
    a, b, c = np.random.default_rng(seed).normal(size=3)
    H = np.array([[a, b], [b, c]])
    np.testing.assert_allclose(density.density_matrix(H, 1), _closed_form_2x2(a, b, c), atol=1e-13)


def test_two_by_two_response_is_derivative_of_closed_form():
    a, b, c = 0.3, -0.7, 1.1
    da, db, dc = 0.2, 0.5, -0.4
    h = 1e-6
    fd = (_closed_form_2x2(a + h * da, b + h * db, c + h * dc)
          - _closed_form_2x2(a - h * da, b - h * db, c - h * dc)) / (2 * h)
    H = np.array([[a, b], [b, c]])
    H1 = np.array([[da, db], [db, dc]])
    np.testing.assert_allclose(density.response(H, H1, 1), fd, atol=1e-8)


def test_diagonal_hamiltonian():
    rng = np.random.default_rng(3)
    eps = rng.permutation(np.linspace(-2, 3, 9))
    H = np.diag(eps)
    n_occ = 4
    D = density.density_matrix(H, n_occ)
    expect = np.diag((eps <= np.sort(eps)[n_occ - 1]).astype(float))
    np.testing.assert_allclose(D, expect, atol=1e-14)
    assert density.band_energy(D, H) == pytest.approx(np.sort(eps)[:n_occ].sum(), abs=1e-13)


def test_diagonal_response_closed_form():
    rng = np.random.default_rng(4)
    eps = np.array([-1.5, 0.7, -0.2, 2.0, 0.1, -0.9])
    H = np.diag(eps)
    H1 = inputs.symmetric_gaussian(6, rng)
    n_occ = 3
    f = (eps <= np.sort(eps)[n_occ - 1]).astype(float)
    expect = np.zeros((6, 6))
    for i in range(6):
        for j in range(6):
            if f[i] != f[j]:
                expect[i, j] = H1[i, j] * (f[i] - f[j]) / (eps[i] - eps[j])
    np.testing.assert_allclose(density.response(H, H1, n_occ), expect, atol=1e-14)


@pytest.fixture(scope="module")
def gapped():
    return inputs.gapped_random(48, 20, np.random.default_rng(11))


def test_invariants(gapped):
    H, n_occ = gapped.H, gapped.n_occ
    D = density.density_matrix(H, n_occ)
    np.testing.assert_allclose(D @ D, D, atol=1e-13)
    assert np.trace(D) == pytest.approx(n_occ, abs=1e-12)
    np.testing.assert_allclose(H @ D - D @ H, 0, atol=1e-13)
    np.testing.assert_allclose(D, D.T, atol=1e-15)


def test_agrees_with_generator_eigensystem(gapped):
    # The generator builds H from a known spectrum; D and Tr[DH] follow from it directly.
    D = density.density_matrix(gapped.H, gapped.n_occ)
    np.testing.assert_allclose(D, density.density_from_eigensystem(gapped.eigvecs, gapped.n_occ), atol=1e-12)
    assert density.band_energy(D, gapped.H) == pytest.approx(gapped.eigvals[:gapped.n_occ].sum(), abs=1e-11)


def test_scale_and_shift_invariance(gapped):
    D = density.density_matrix(gapped.H, gapped.n_occ)
    D2 = density.density_matrix(2.5 * gapped.H - 0.7 * np.eye(gapped.n), gapped.n_occ)
    np.testing.assert_allclose(D2, D, atol=1e-12)


def test_particle_hole(gapped):
    n = gapped.n
    D = density.density_matrix(gapped.H, gapped.n_occ)
    Dm = density.density_matrix(-gapped.H, n - gapped.n_occ)
    np.testing.assert_allclose(Dm, np.eye(n) - D, atol=1e-12)


def test_permutation_covariance(gapped):
    perm = np.random.default_rng(5).permutation(gapped.n)
    P = np.eye(gapped.n)[perm]
    D = density.density_matrix(gapped.H, gapped.n_occ)
    np.testing.assert_allclose(density.density_matrix(P @ gapped.H @ P.T, gapped.n_occ), P @ D @ P.T, atol=1e-12)


def test_response_matches_central_differences(gapped):
    rng = np.random.default_rng(6)
    H1 = inputs.symmetric_gaussian(gapped.n, rng) * 0.1
    h = 1e-5
    fd = (density.density_matrix(gapped.H + h * H1, gapped.n_occ)
          - density.density_matrix(gapped.H - h * H1, gapped.n_occ)) / (2 * h)
    D1 = density.response(gapped.H, H1, gapped.n_occ)
    np.testing.assert_allclose(D1, fd, atol=1e-8)
    # D1 is symmetric and keeps the trace (the occupation is fixed).
    np.testing.assert_allclose(D1, D1.T, atol=1e-14)
    assert abs(np.trace(D1)) < 1e-12


def test_response_rows_match_central_differences_and_closed_form(gapped):
    """Sampled rows of D1 from the occupied-unoccupied block only: against central
    differences of the eigendecomposition D, and on a diagonal H against
    D1_ij = H1_ij (f_i - f_j)/(eps_i - eps_j)."""
    rng = np.random.default_rng(16)
    H1 = inputs.symmetric_gaussian(gapped.n, rng) * 0.1
    rows = [0, 7, 19, 20, 47]
    h = 1e-5
    fd = (density.density_matrix(gapped.H + h * H1, gapped.n_occ)
          - density.density_matrix(gapped.H - h * H1, gapped.n_occ)) / (2 * h)
    got = density.response_rows(gapped.eigvals, gapped.eigvecs, H1, gapped.n_occ, rows)
    np.testing.assert_allclose(got, fd[rows], atol=1e-8)
    eps = np.array([-0.9, -0.4, -0.1, 0.2, 0.5, 0.8])
    H1d = inputs.symmetric_gaussian(6, rng)
    f = density.occupations(6, 2)
    got = density.response_rows(eps, np.eye(6), H1d, 2, [1, 4])
    for a, i in enumerate([1, 4]):
        for j in range(6):
            expect = H1d[i, j] * (f[i] - f[j]) / (eps[i] - eps[j]) if f[i] != f[j] else 0.0
            assert got[a, j] == pytest.approx(expect, abs=1e-14)


def test_adjoint_duality_and_differences(gapped):
    rng = np.random.default_rng(7)
    G = rng.standard_normal((gapped.n, gapped.n))  # not symmetric on purpose
    E = inputs.symmetric_gaussian(gapped.n, rng)
    grad = density.adjoint(gapped.H, G, gapped.n_occ)
    lhs = np.sum(E * grad)
    rhs = np.sum(G * density.response(gapped.H, E, gapped.n_occ))
    assert lhs == pytest.approx(rhs, rel=1e-11)
    h = 1e-5
    f = lambda s: np.sum(density.density_matrix(gapped.H + s * E, gapped.n_occ) * G)
    assert lhs == pytest.approx((f(h) - f(-h)) / (2 * h), rel=1e-6)


def test_no_gap_is_rejected():
    H = np.diag([0.0, 1.0, 1.0, 2.0])
    with pytest.raises(ValueError):
        density.response(H, np.eye(4), 2)


# -- non-orthogonal basis ------------------------------------------------------

@pytest.fixture(scope="module")
def nonorth():
    rng = np.random.default_rng(31)
    n = 60
    H = inputs.symmetric_gaussian(n, rng) * 0.3
    S = inputs.overlap_matrix(n, rng)
    return H, S, 23


def test_overlap_is_positive_definite(nonorth):
    _, S, _ = nonorth
    lam = np.linalg.eigvalsh(S)
    assert 0.5 <= lam[0] and lam[-1] <= 1.5


def test_inverse_factors(nonorth):
    _, S, _ = nonorth
    for Z in (density.inverse_factor_lowdin(S), density.inverse_factor_cholesky(S)):
        np.testing.assert_allclose(Z.T @ S @ Z, np.eye(S.shape[0]), atol=1e-12)


def test_orthogonalised_route_matches_generalised_eigenproblem(nonorth):
    H, S, n_occ = nonorth
    ref = density.density_matrix_generalized(H, S, n_occ)
    for Z in (density.inverse_factor_lowdin(S), density.inverse_factor_cholesky(S)):
        # D does not depend on which inverse factor is used
        np.testing.assert_allclose(density.density_matrix_via_factor(H, Z, n_occ), ref, atol=1e-11)
    # idempotency in the S metric, occupation, and [H, D] in the S metric
    np.testing.assert_allclose(ref @ S @ ref, ref, atol=1e-11)
    assert np.trace(ref @ S) == pytest.approx(n_occ, abs=1e-10)
    np.testing.assert_allclose(H @ ref @ S, S @ ref @ H, atol=1e-11)


def test_identity_overlap_reduces_to_orthogonal(nonorth):
    H, _, n_occ = nonorth
    n = H.shape[0]
    np.testing.assert_allclose(density.density_matrix_generalized(H, np.eye(n), n_occ),
                               density.density_matrix(H, n_occ), atol=1e-12)
