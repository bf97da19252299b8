"""The seeded input recipe: every generator is deterministic for its seed, symmetric bit
for bit, and has the spectrum, gap, band structure and sizes its workload states."""
import numpy as np
import pytest

from paper_2107_02737_gb300 import inputs


def test_seeds_are_per_config_and_instance_and_deterministic():
    a = inputs.rng_for(2, 7).standard_normal(5)
    assert np.array_equal(a, inputs.rng_for(2, 7).standard_normal(5))
    assert np.array_equal(a, np.random.default_rng(2007).standard_normal(5))
    assert not np.array_equal(a, inputs.rng_for(2, 8).standard_normal(5))
    h1 = inputs.gapped_random(50, 20, inputs.rng_for(0, 1)).H
    assert np.array_equal(h1, inputs.gapped_random(50, 20, inputs.rng_for(0, 1)).H)


def test_gapped_random_spectrum_and_eigenbasis():
    ham = inputs.gapped_random(120, 45, inputs.rng_for(0, 2))
    H, lam, q = ham.H, ham.eigvals, ham.eigvecs
    assert np.array_equal(H, H.T)
    assert np.all(np.diff(lam) >= 0)
    assert np.all((lam[:45] >= -1.0) & (lam[:45] <= -0.05)) and np.all((lam[45:] >= 0.05) & (lam[45:] <= 1.0))
    np.testing.assert_allclose(q.T @ q, np.eye(120), atol=1e-12)
    np.testing.assert_allclose(H, (q * lam) @ q.T, atol=1e-13)
    np.testing.assert_allclose(np.linalg.eigvalsh(H), lam, atol=1e-12)


def test_banded_matrix_band_and_scales():
    n, bw = 400, 64
    h = inputs.banded_matrix(n, inputs.rng_for(1, 3), bandwidth=bw)
    assert np.array_equal(h, h.T)
    i, j = np.nonzero(h)
    assert np.abs(i - j).max() == bw
    # off-diagonal scale N(0, 0.1^2) exp(-d / 16): the first and a far diagonal
    d1 = np.diag(h, 1)
    d48 = np.diag(h, 48) / np.exp(-48 / 16)
    assert 0.07 < d1.std() / np.exp(-1 / 16) < 0.13 and 0.07 < d48.std() < 0.13
    assert 0.4 < np.diag(h).std() < 0.6


def test_water_like_recipe_opens_the_gap():
    ham = inputs.banded_tight_binding(300, inputs.rng_for(1, 4))
    lam = ham.eigvals
    assert ham.n_occ == 150 and np.array_equal(ham.H, ham.H.T)
    assert lam[150] - lam[149] >= 0.05 - 1e-15
    np.testing.assert_allclose(np.linalg.eigvalsh(ham.H), lam, atol=1e-12)
    with pytest.raises(ValueError):
        inputs.banded_tight_binding(10, inputs.rng_for(1, 5), n_occ=0)


def test_perturbations_overlap_and_md_sequence():
    rng = inputs.rng_for(3, 6)
    h1 = inputs.banded_perturbation(200, rng, bandwidth=8)
    assert np.array_equal(h1, h1.T)
    i, j = np.nonzero(h1)
    assert np.abs(i - j).max() == 8
    s = inputs.overlap_matrix(300, rng)
    ev = np.linalg.eigvalsh(s)
    assert np.array_equal(s, s.T) and ev.min() >= 0.5 and ev.max() <= 1.5
    v = inputs.sparse_perturbation(400, rng)
    assert np.array_equal(v, v.T)
    frac = np.count_nonzero(np.triu(v)) / (400 * 401 / 2)
    assert 0.005 < frac < 0.015
    h0 = inputs.symmetric_gaussian(30, rng)
    assert np.array_equal(h0, h0.T)
    vv = inputs.sparse_perturbation(30, rng, density=0.2)
    np.testing.assert_array_equal(inputs.md_sequence(h0, vv, 7), h0 + np.sin(0.05 * 7) * vv)


def test_batch_sizes_recipe():
    sizes = inputs.batch_sizes(64, inputs.rng_for(2, 10_000))
    assert len(sizes) == 64 and all(128 <= s <= 2048 and s % 128 == 0 for s in sizes)
    assert sizes == inputs.batch_sizes(64, inputs.rng_for(2, 10_000))
    assert len(set(sizes)) > 8
