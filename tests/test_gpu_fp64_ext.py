"""FP64 refinement layers and the non-orthogonal route (through the C ABI) against the
oracle: the refined output matches the oracle's refinement of the same chain output
and reaches FP64 idempotency and trace; the non-orthogonal D matches the generalised
eigenproblem and does not depend on the inverse factor."""
import numpy as np
import pytest
import torch

from oracle import density as odens
from oracle import sp2 as osp2
from paper_2107_02737_gb300 import inputs
import paper_2107_02737_gb300.sp2 as sp2
from tests._gpu import TOL_D, dev, fro_err, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [300, 640])
def test_refined_density(n):
    ham = inputs.gapped_random(n, n // 2, inputs.rng_for(5, n))
    H = dev(ham.H)
    D64, res = sp2.density_refined(H, ham.n_occ, refine_layers=2)
    D32, r32 = sp2.density(H, ham.n_occ)
    assert D64.dtype == torch.float64
    d = host(D64)
    ref = odens.density_from_eigensystem(ham.eigvecs, ham.n_occ)
    # eigenvectors are those of the chain; eigenvalues are purified to FP64 level
    assert fro_err(d, ref) <= 10 * max(fro_err(host(D32), ref), 1e-7)
    assert abs(res.trace_D - ham.n_occ) <= 1e-9
    assert np.linalg.norm(d @ d - d) <= 1e-9
    assert res.layers == r32.layers + 2
    # the oracle's refinement of the same chain output (same signs)
    X, stats = osp2.refine(host(D32), ham.n_occ, layers=2)
    assert [s.choice for s in stats[1:]] == res.choices[-2:]
    assert np.max(np.abs(d - X)) <= 1e-9
    assert res.band_energy == pytest.approx(np.sum(X * ham.H), abs=1e-8)


def test_refinement_zero_layers_is_the_chain():
    ham = inputs.gapped_random(256, 128, inputs.rng_for(5, 1))
    D64, res = sp2.density_refined(dev(ham.H), ham.n_occ, refine_layers=0)
    D32, _ = sp2.density(dev(ham.H), ham.n_occ)
    assert torch.equal(D64, D32.double())


@pytest.fixture(scope="module")
def nonorth_case():
    n = 320
    rng = inputs.rng_for(6, 1)
    ham = inputs.gapped_random(n, 130, rng)
    S = inputs.overlap_matrix(n, rng)
    # a Hamiltonian in the non-orthogonal basis with a gap: H = S^(1/2) H_orth S^(1/2)
    lam, U = np.linalg.eigh(S)
    Sh = (U * np.sqrt(lam)) @ U.T
    H = Sh @ ham.H @ Sh
    return 0.5 * (H + H.T), S, ham.n_occ


def test_nonorthogonal_density(nonorth_case):
    H, S, n_occ = nonorth_case
    ref = odens.density_matrix_generalized(H, S, n_occ)
    Ds = []
    for Z in (odens.inverse_factor_lowdin(S), odens.inverse_factor_cholesky(S)):
        D, res = sp2.density_nonorth(dev(H), dev(Z), n_occ, refine_layers=2)
        d = host(D)
        Ds.append(d)
        assert fro_err(d, ref) <= TOL_D["fp16"] * 1e-2
        assert np.trace(d @ S) == pytest.approx(n_occ, abs=1e-8)
        np.testing.assert_allclose(d @ S @ d, d, atol=1e-8)
        assert res.band_energy == pytest.approx(np.sum(ref * H), abs=1e-6)
    assert fro_err(Ds[0], Ds[1]) <= 1e-5
