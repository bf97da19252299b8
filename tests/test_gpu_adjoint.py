"""Parity of sp2_adjoint (reverse accumulation through the stored layers) and of the
autograd function: against the FP64 chain adjoint replaying the GPU's signs, the
eigenbasis formula, central differences of the FP64 oracle, and the GPU response
by duality <E, dTr[DG]/dH> = Tr[G D1(E)]."""
import numpy as np
import pytest
import torch

from oracle import density as odens
from oracle import sp2 as osp2
from paper_2107_02737_gb300 import inputs
import paper_2107_02737_gb300.sp2 as sp2
from tests._gpu import dev, host, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    n = 320
    ham = inputs.gapped_random(n, 120, inputs.rng_for(3, 77))
    rng = inputs.rng_for(3, 78)
    G = rng.standard_normal((n, n))          # asymmetric weight on purpose
    E = inputs.symmetric_gaussian(n, rng)
    return ham, G, E


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_adjoint_matches_chain_and_theta(case, precision):
    ham, G, _ = case
    D, dH, res = sp2.adjoint(dev(ham.H), dev(G), ham.n_occ, precision=precision)
    assert res.converged
    g = host(dH)
    chain = osp2.chain_adjoint(ham.H, G, res.choices, res.eps_min, res.eps_max)
    theta = odens.adjoint(ham.H, G, ham.n_occ)
    tol = 2e-3 if precision == "fp16" else 2e-2
    print(f"\n{precision}: rel err vs chain {rel_err(g, chain):.2e}, vs theta {rel_err(g, theta):.2e}")
    assert rel_err(g, chain) <= tol
    assert rel_err(g, theta) <= tol + 1e-3
    assert np.array_equal(g, g.T)


def test_adjoint_directional_differences(case):
    ham, G, E = case
    _, dH, _ = sp2.adjoint(dev(ham.H), dev(G), ham.n_occ, precision="fp16")
    h = 1e-4
    f = lambda s: np.sum(odens.density_matrix(ham.H + s * E, ham.n_occ) * G)
    fd = (f(h) - f(-h)) / (2 * h)
    assert np.sum(E * host(dH)) == pytest.approx(fd, rel=3e-3)


def test_adjoint_response_duality_on_gpu(case):
    ham, G, E = case
    _, res = sp2.density(dev(ham.H), ham.n_occ, precision="fp16")
    _, dH, _ = sp2.adjoint(dev(ham.H), dev(G), ham.n_occ, precision="fp16", fwd=res)
    _, D1, _ = sp2.response(dev(ham.H), dev(E), ham.n_occ, precision="fp16", fwd=res)
    lhs = np.sum(E * host(dH))
    rhs = np.sum(G * host(D1))
    assert lhs == pytest.approx(rhs, rel=2e-3)


def test_autograd_function(case):
    ham, G, _ = case
    H = dev(ham.H).requires_grad_(True)
    D = sp2.DensityMatrix.apply(H, ham.n_occ)
    loss = (D.double() * dev(G)).sum()
    loss.backward()
    ref = odens.adjoint(ham.H, G, ham.n_occ)
    assert H.grad.dtype == torch.float64
    assert rel_err(host(H.grad), ref) <= 3e-3


def test_adjoint_zero_layers_and_trivial():
    H = np.diag([-1.0, 1.0])   # X_0 is already idempotent: no layers
    G = np.array([[1.0, 2.0], [0.0, 3.0]])
    D, dH, res = sp2.adjoint(dev(H), dev(G), 1, precision="fp16")
    assert res.layers == 0
    lo, hi = res.eps_min, res.eps_max
    assert np.allclose(host(dH), -0.5 * (G + G.T) / (hi - lo), atol=1e-6)
    _, dH0, r0 = sp2.adjoint(dev(H), dev(G), 0, precision="fp16")
    assert torch.count_nonzero(dH0) == 0 and r0.stop_reason == sp2.STOP_TRIVIAL
