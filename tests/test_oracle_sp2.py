"""Pins for oracle/sp2.py, the float64 DNN-SP2 chain (Eq. Deep_NN and its layer rule).

The chain is tied to: hand-computed layer sequences on diagonal H (fixtures in
tests/golden/), hand-computed Gershgorin discs, the same chain run on scalar
eigenvalues, the eigendecomposition definition of D, and, for the response and
adjoint, divided differences of the chain polynomial and central differences.
"""
import numpy as np
import pytest

from oracle import density, sp2
from paper_2107_02737_gb300 import inputs
from tests._golden import load


def test_gershgorin_golden():
    g = load("gershgorin_3x3.txt")
    lo, hi = sp2.gershgorin_bounds(g["H"].reshape(3, 3))
    assert (lo, hi) == (g["eps_min"], g["eps_max"])


def test_gershgorin_brackets_spectrum():
    ham = inputs.banded_tight_binding(200, np.random.default_rng(1), bandwidth=16)
    lo, hi = sp2.gershgorin_bounds(ham.H)
    lam = np.linalg.eigvalsh(ham.H)
    assert lo <= lam[0] and lam[-1] <= hi


def test_input_layer_maps_spectrum_reversed():
    H = np.diag([-1.0, 0.0, 3.0])
    X0 = sp2.input_layer(H, -1.0, 3.0)
    np.testing.assert_allclose(np.diag(X0), [1.0, 0.75, 0.0])


def test_golden_all_square_chain():
    g = load("sp2_diag_square.txt")
    r = sp2.sp2(np.diag(g["H_diag"]), int(g["n_occ"]))
    assert r.layers == int(g["layers"])
    assert r.choices == [int(c) for c in g["choices"]]
    np.testing.assert_allclose([s.trace for s in r.stats], g["trace"], rtol=0, atol=1e-15)
    np.testing.assert_allclose([s.trace_sq for s in r.stats], g["trace_sq"], rtol=0, atol=1e-15)
    assert r.stop_reason == int(g["stop_reason"])
    np.testing.assert_allclose(r.D, np.diag([1.0, 0.0, 0.0]), atol=1e-9)


def test_all_flip_chain_closed_form():
    # n_occ = 2 on diag(-1, 0, 1): every layer is 2X - X^2, middle eigenvalue 1 - 2^(-2^n).
    r = sp2.sp2(np.diag([-1.0, 0.0, 1.0]), 2)
    assert set(r.choices) == {sp2.FLIP}
    for n, s in enumerate(r.stats):
        assert s.trace == pytest.approx(2.0 - 2.0 ** (-(2 ** n)), abs=1e-15)


def test_golden_tie_and_flip():
    g = load("sp2_diag_tie_flip.txt")
    r = sp2.sp2(np.diag(g["H_diag"]), int(g["n_occ"]))
    k = len(g["choices_prefix"])
    assert r.choices[:k] == [int(c) for c in g["choices_prefix"]]
    np.testing.assert_allclose([s.trace for s in r.stats[:k]], g["trace_prefix"], atol=1e-15)
    np.testing.assert_allclose([s.trace_sq for s in r.stats[:k]], g["trace_sq_prefix"], atol=1e-15)


def test_layer_choice_rule():
    assert sp2.layer_choice(2.0, 1.625, 2) == sp2.SQUARE          # tie
    assert sp2.layer_choice(1.625, 1.3203125, 2) == sp2.FLIP
    assert sp2.layer_choice(3.0, 2.5, 2) == sp2.SQUARE


def test_stop_rule():
    assert sp2.stop_check([0.5, 1e-7], 1e-6, 100) == sp2.STOP_TOL
    assert sp2.stop_check([5.0, 2.0, 3.0], 1e-6, 100) == 0           # early rise is not a stall
    assert sp2.stop_check([1e-3, 5e-4, 2e-3], 1e-6, 100) == sp2.STOP_STALL
    assert sp2.stop_check([1e-3, 5e-4, 9e-4], 1e-6, 100) == 0
    assert sp2.stop_check([1e-3, -5e-4, -1.2e-3], 1e-6, 100) == sp2.STOP_STALL  # magnitudes
    assert sp2.stop_check([1.0, 0.9, 0.8], 1e-6, 2) == sp2.STOP_MAX


def test_trivial_occupations():
    H = np.diag([-1.0, 0.0, 1.0])
    assert np.array_equal(sp2.sp2(H, 0).D, np.zeros((3, 3)))
    assert np.array_equal(sp2.sp2(H, 3).D, np.eye(3))


@pytest.fixture(scope="module")
def c0_small():
    return inputs.gapped_random(128, 64, inputs.rng_for(0, 3))


def test_matrix_chain_matches_scalar_chain(c0_small):
    r = sp2.sp2(c0_small.H, c0_small.n_occ)
    p, stats, reason, _ = sp2.scalar_sp2(c0_small.eigvals, c0_small.n_occ, r.eps_min, r.eps_max)
    assert [s.choice for s in stats[1:]] == r.choices
    assert reason == r.stop_reason
    for a, b in zip(r.stats, stats):
        assert a.trace == pytest.approx(b.trace, abs=1e-9)
        assert a.trace_sq == pytest.approx(b.trace_sq, abs=1e-9)
    np.testing.assert_allclose(r.D, (c0_small.eigvecs * p) @ c0_small.eigvecs.T, atol=1e-10)


def test_chain_reaches_eigendecomposition_density(c0_small):
    r = sp2.sp2(c0_small.H, c0_small.n_occ)
    assert r.converged and r.stop_reason == sp2.STOP_TOL
    D = density.density_matrix(c0_small.H, c0_small.n_occ)
    assert np.linalg.norm(r.D - D) / np.sqrt(c0_small.n) < 1e-9
    assert abs(np.trace(r.D) - c0_small.n_occ) < 1e-6


def test_chain_on_banded_workload():
    ham = inputs.banded_tight_binding(256, inputs.rng_for(1, 1))
    r = sp2.sp2(ham.H, ham.n_occ)
    D = density.density_from_eigensystem(ham.eigvecs, ham.n_occ)
    assert r.converged
    assert np.linalg.norm(r.D - D) / np.sqrt(ham.n) < 1e-8


def test_zero_padding_in_x_space_is_inert(c0_small):
    # Zero rows/columns of X are fixed by both X^2 and 2X - X^2, so padding X_0 leaves D unchanged;
    # padding H itself with zeros would insert eigenvalue 0 below mu = 0 in the wrong cases.
    r = sp2.sp2(c0_small.H, c0_small.n_occ)
    n, pad = c0_small.n, 16
    X = np.zeros((n + pad, n + pad))
    X[:n, :n] = sp2.input_layer(c0_small.H, r.eps_min, r.eps_max)
    for c in r.choices:
        X = sp2.apply_layer(X, c)
    np.testing.assert_allclose(X[:n, :n], r.D, atol=1e-12)
    assert np.all(X[n:, :] == 0) and np.all(X[:, n:] == 0)


@pytest.fixture(scope="module")
def diff_case():
    ham = inputs.gapped_random(40, 17, np.random.default_rng(21))
    r = sp2.sp2(ham.H, ham.n_occ)
    rng = np.random.default_rng(22)
    return ham, r, inputs.symmetric_gaussian(40, rng) * 0.05, inputs.symmetric_gaussian(40, rng)


def test_chain_response_matches_divided_differences(diff_case):
    ham, r, H1, _ = diff_case
    a = sp2.chain_response(ham.H, H1, r.choices, r.eps_min, r.eps_max)
    b = sp2.chain_derivative_eigenbasis(ham.H, H1, r.choices, r.eps_min, r.eps_max)
    np.testing.assert_allclose(a, b, atol=1e-9)


def test_chain_response_matches_central_differences(diff_case):
    ham, r, H1, _ = diff_case
    h = 1e-6
    run = lambda s: sp2.sp2(ham.H + s * H1, ham.n_occ, bounds=(r.eps_min, r.eps_max),
                            choices=r.choices).D
    fd = (run(h) - run(-h)) / (2 * h)
    np.testing.assert_allclose(sp2.chain_response(ham.H, H1, r.choices, r.eps_min, r.eps_max), fd, atol=1e-6)


def test_chain_response_converges_to_theta_response(diff_case):
    ham, r, H1, _ = diff_case
    a = sp2.chain_response(ham.H, H1, r.choices, r.eps_min, r.eps_max)
    np.testing.assert_allclose(a, density.response(ham.H, H1, ham.n_occ), atol=1e-6)


def test_chain_adjoint_duality_and_self_adjointness(diff_case):
    ham, r, H1, G = diff_case
    grad = sp2.chain_adjoint(ham.H, G, r.choices, r.eps_min, r.eps_max)
    lhs = np.sum(H1 * grad)
    rhs = np.sum(G * sp2.chain_response(ham.H, H1, r.choices, r.eps_min, r.eps_max))
    assert lhs == pytest.approx(rhs, rel=1e-10)
    np.testing.assert_allclose(grad, sp2.chain_derivative_eigenbasis(ham.H, G, r.choices, r.eps_min, r.eps_max),
                               atol=1e-9)
    # The chain is converged only to its stop tolerance, so it matches theta's adjoint to ~1e-6 relative.
    exact = density.adjoint(ham.H, G, ham.n_occ)
    assert np.linalg.norm(grad - exact) / np.linalg.norm(exact) < 1e-5


def test_chain_adjoint_asymmetric_weight(diff_case):
    ham, r, _, _ = diff_case
    G = np.random.default_rng(23).standard_normal((ham.n, ham.n))
    a = sp2.chain_adjoint(ham.H, G, r.choices, r.eps_min, r.eps_max)
    b = sp2.chain_adjoint(ham.H, 0.5 * (G + G.T), r.choices, r.eps_min, r.eps_max)
    np.testing.assert_allclose(a, b, atol=1e-14)


def test_refinement_purifies_quadratically():
    # A projector with eigenvalues nudged by delta: two refinement layers map
    # 1 + d -> 1 - O(d^2) and d -> O(d^2) (closed form on a diagonal matrix).
    d = np.array([1e-4, -2e-4, 3e-4, -1e-4])
    lam = np.array([1.0, 1.0, 0.0, 0.0]) + d
    X, stats = sp2.refine(np.diag(lam), 2, layers=2)
    # by hand: Tr X = 2 + 1e-4 > 2 and the rule picks X^2 first, then 2X - X^2,
    # so every eigenvalue becomes 2 lam^2 - lam^4
    assert [s.choice for s in stats[1:]] == [sp2.SQUARE, sp2.FLIP]
    np.testing.assert_allclose(np.diag(X), 2 * lam ** 2 - lam ** 4, rtol=0, atol=1e-15)
    dev = np.minimum(np.abs(np.diag(X)), np.abs(1 - np.diag(X)))
    assert np.max(dev) < 2.5 * np.max(np.abs(d)) ** 2
    assert abs(stats[-1].idem) < 2 * np.sum(np.abs(d)) ** 2
    # the chosen signs follow the trace rule layer by layer
    for k in range(1, len(stats)):
        assert stats[k].choice == sp2.layer_choice(stats[k - 1].trace, stats[k - 1].trace_sq, 2)


def test_refinement_of_perturbed_density(c0_small):
    # An FP32-rounded converged chain refined in float64 reaches float64 idempotency.
    r = sp2.sp2(c0_small.H, c0_small.n_occ)
    X32 = r.D.astype(np.float32).astype(np.float64)
    X, stats = sp2.refine(X32, c0_small.n_occ, layers=2)
    assert np.linalg.norm(X @ X - X) < 1e-9
    assert abs(np.trace(X) - c0_small.n_occ) < 1e-9
    D = density.density_matrix(c0_small.H, c0_small.n_occ)
    assert np.linalg.norm(X - D) / np.sqrt(c0_small.n) < 1e-6


# -- accelerated chain (estimated HOMO / LUMO interval) ------------------------------

def test_golden_accelerated_layers():
    g = load("sp2_accel_diag.txt")
    H = np.diag(g["H_diag"])
    gap = tuple(g["gap"])
    r = sp2.sp2(H, int(g["n_occ"]), bounds=(0.0, 1.0), gap=gap, keep_layers=True)
    assert r.choices[:2] == [int(c) for c in g["choices"]]
    np.testing.assert_allclose(r.alphas[:2], g["alpha"], rtol=1e-15)
    np.testing.assert_allclose(np.diag(r.layers_X[1]), g["X1_diag_times_256"] / 256, atol=1e-15)
    np.testing.assert_allclose(np.diag(r.layers_X[2]), g["X2_diag_times_142129"] / 142129, atol=1e-15)
    # the tracked ends of the interval are the images of the estimated eigenvalues
    assert r.gap_images[1] == pytest.approx((135 / 256, 15 / 16), abs=1e-15)
    assert r.gap_images[2] == pytest.approx(((135 / 377) ** 2, (345 / 377) ** 2), abs=1e-15)
    np.testing.assert_allclose(r.D, np.diag([0, 0, 1, 1]), atol=1e-6)


def test_accelerated_with_whole_range_is_the_plain_chain(c0_small):
    lo, hi = sp2.gershgorin_bounds(c0_small.H)
    plain = sp2.sp2(c0_small.H, c0_small.n_occ)
    acc = sp2.sp2(c0_small.H, c0_small.n_occ, gap=(lo, hi))
    assert acc.choices == plain.choices and set(acc.alphas) == {1.0}
    assert np.array_equal(acc.D, plain.D)


@pytest.fixture(scope="module")
def accel_case():
    ham = inputs.gapped_random(96, 40, np.random.default_rng(41), occ_range=(-1.0, -0.02),
                               virt_range=(0.02, 1.0))
    gap = (ham.eigvals[ham.n_occ - 1], ham.eigvals[ham.n_occ])
    return ham, gap


def test_accelerated_chain_converges_in_fewer_layers(accel_case):
    ham, gap = accel_case
    plain = sp2.sp2(ham.H, ham.n_occ)
    acc = sp2.sp2(ham.H, ham.n_occ, gap=gap)
    ref = density.density_matrix(ham.H, ham.n_occ)
    assert acc.converged and acc.stop_reason == sp2.STOP_TOL
    assert np.linalg.norm(acc.D - ref) < 1e-6
    assert acc.layers <= 0.7 * plain.layers
    assert all(1.0 <= a <= 2.0 for a in acc.alphas)


def test_accelerated_images_follow_the_eigenvectors(accel_case):
    # With the exact HOMO / LUMO as the estimate, the tracked interval ends are the
    # Rayleigh quotients of the HOMO and LUMO eigenvectors in every layer.
    ham, gap = accel_case
    r = sp2.sp2(ham.H, ham.n_occ, gap=gap, keep_layers=True)
    c_homo = ham.eigvecs[:, ham.n_occ - 1]
    c_lumo = ham.eigvecs[:, ham.n_occ]
    for X, (x_lumo, x_homo) in zip(r.layers_X, r.gap_images):
        assert c_lumo @ X @ c_lumo == pytest.approx(x_lumo, abs=1e-11)
        assert c_homo @ X @ c_homo == pytest.approx(x_homo, abs=1e-11)


def test_accelerated_matrix_chain_matches_scalar_chain(accel_case):
    ham, gap = accel_case
    r = sp2.sp2(ham.H, ham.n_occ, gap=gap)
    p, stats, reason, _ = sp2.scalar_sp2(ham.eigvals, ham.n_occ, r.eps_min, r.eps_max, gap=gap)
    assert [s.choice for s in stats[1:]] == r.choices and reason == r.stop_reason
    for a, b in zip(stats, r.stats):
        assert a.trace == pytest.approx(b.trace, abs=1e-10)
        assert a.trace_sq == pytest.approx(b.trace_sq, abs=1e-10)


@pytest.mark.parametrize("how", ["wider", "narrower", "shifted_up", "shifted_down"])
def test_accelerated_any_overlapping_interval_converges(accel_case, how):
    ham, (e_homo, e_lumo) = accel_case
    w = e_lumo - e_homo
    est = {"wider": (e_homo - 3 * w, e_lumo + 3 * w), "narrower": (e_homo + 0.3 * w, e_lumo - 0.3 * w),
           "shifted_up": (e_homo + 0.6 * w, e_lumo + 0.6 * w),
           "shifted_down": (e_homo - 0.6 * w, e_lumo - 0.6 * w)}[how]
    r = sp2.sp2(ham.H, ham.n_occ, gap=est)
    assert r.converged
    assert np.linalg.norm(r.D - density.density_matrix(ham.H, ham.n_occ)) < 1e-6


def test_accelerated_interval_outside_the_gap_fails(accel_case):
    # An interval that misses the gap (between the two highest occupied levels)
    # breaks the ordering of the images: the chain no longer reaches theta(mu I - H).
    ham, _ = accel_case
    k = ham.n_occ
    r = sp2.sp2(ham.H, k, gap=(ham.eigvals[k - 3], ham.eigvals[k - 2]))
    ref = density.density_matrix(ham.H, k)
    assert not r.converged or np.linalg.norm(r.D - ref) > 1e-3


def test_accelerated_response_and_adjoint(accel_case):
    ham, gap = accel_case
    r = sp2.sp2(ham.H, ham.n_occ, gap=gap)
    rng = np.random.default_rng(42)
    H1 = inputs.symmetric_gaussian(ham.n, rng) * 0.05
    G = inputs.symmetric_gaussian(ham.n, rng)
    a = sp2.chain_response(ham.H, H1, r.choices, r.eps_min, r.eps_max, alphas=r.alphas)
    b = sp2.chain_derivative_eigenbasis(ham.H, H1, r.choices, r.eps_min, r.eps_max, gap=gap)
    np.testing.assert_allclose(a, b, atol=1e-8)
    np.testing.assert_allclose(a, density.response(ham.H, H1, ham.n_occ), atol=1e-5)
    h = 1e-6
    run = lambda s: sp2.sp2(ham.H + s * H1, ham.n_occ, bounds=(r.eps_min, r.eps_max), choices=r.choices,
                            gap=gap).D
    np.testing.assert_allclose(a, (run(h) - run(-h)) / (2 * h), atol=1e-5)
    grad = sp2.chain_adjoint(ham.H, G, r.choices, r.eps_min, r.eps_max, alphas=r.alphas)
    assert np.sum(H1 * grad) == pytest.approx(np.sum(G * a), rel=1e-10)
