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
    tol = 1e-4 if precision == "fp16" else 3e-4   # about ten times the measured 1.1e-5 / 2.8e-5
    print(f"\n{precision}: rel err vs chain {rel_err(g, chain):.2e}, vs theta {rel_err(g, theta):.2e}")
    assert rel_err(g, chain) <= tol
    assert rel_err(g, theta) <= 2 * tol
    assert np.array_equal(g, g.T)


def test_adjoint_directional_differences(case):
    ham, G, E = case
    _, dH, _ = sp2.adjoint(dev(ham.H), dev(G), ham.n_occ, precision="fp16")
    h = 1e-4
    f = lambda s: np.sum(odens.density_matrix(ham.H + s * E, ham.n_occ) * G)
    fd = (f(h) - f(-h)) / (2 * h)
    print(f"\nadjoint vs central difference: rel err {abs(np.sum(E * host(dH)) - fd) / abs(fd):.2e}")
    assert np.sum(E * host(dH)) == pytest.approx(fd, rel=1e-4)   # measured 9.5e-6


def test_adjoint_response_duality_on_gpu(case):
    ham, G, E = case
    _, res = sp2.density(dev(ham.H), ham.n_occ, precision="fp16")
    _, dH, _ = sp2.adjoint(dev(ham.H), dev(G), ham.n_occ, precision="fp16", fwd=res)
    _, D1, _ = sp2.response(dev(ham.H), dev(E), ham.n_occ, precision="fp16", fwd=res)
    lhs = np.sum(E * host(dH))
    rhs = np.sum(G * host(D1))
    print(f"\nduality: rel gap {abs(lhs - rhs) / abs(rhs):.2e}")
    assert lhs == pytest.approx(rhs, rel=3e-5)   # measured 2.2e-6


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


# -- checkpointed recomputation: every s-th layer kept, the rest recomputed in the
# reverse sweep from the forward's recorded signs, offsets and expansions --

@pytest.fixture(scope="module")
def stored_adjoints(case):
    ham, G, _ = case
    out = {}
    for precision in ("fp16", "bf16"):
        _, res = sp2.density(dev(ham.H), ham.n_occ, precision=precision)
        out[precision] = (res,) + sp2.adjoint(dev(ham.H), dev(G), ham.n_occ, precision=precision)
    return out


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
@pytest.mark.parametrize("stride", [3, 4, 5, 7, -1])
@pytest.mark.parametrize("replay", [False, True])
def test_checkpointed_adjoint_is_bit_identical(case, stored_adjoints, precision, stride, replay):
    ham, G, _ = case
    fwd, D0, dH0, r0 = stored_adjoints[precision]
    D, dH, res = sp2.adjoint(dev(ham.H), dev(G), ham.n_occ, precision=precision,
                             fwd=fwd if replay else None, checkpoint_stride=stride)
    assert res.layers == r0.layers and res.choices == r0.choices
    assert torch.equal(D, D0)
    assert torch.equal(dH, dH0)


def test_checkpointing_saves_workspace():
    n, L = 4096, 33
    full = sp2.workspace_bytes(n, "adjoint", layers=L)
    auto = sp2.workspace_bytes(n, "adjoint", layers=L, checkpoint_stride=-1)
    s6 = sp2.workspace_bytes(n, "adjoint", layers=L, checkpoint_stride=6)
    assert auto <= s6 < full
    assert auto < 0.7 * full  # operands shrink 2x; FP32 masters and the second stream do not


def test_checkpointed_adjoint_accelerated(case):
    ham, G, _ = case
    gap = (float(ham.eigvals[ham.n_occ - 1]), float(ham.eigvals[ham.n_occ]))
    D0, g0, r0 = sp2.adjoint(dev(ham.H), dev(G), ham.n_occ, precision="fp16", gap=gap)
    assert any(a != 1.0 for a in r0.alphas)
    D1, g1, r1 = sp2.adjoint(dev(ham.H), dev(G), ham.n_occ, precision="fp16", gap=gap, checkpoint_stride=3)
    assert r1.alphas == r0.alphas
    assert torch.equal(D1, D0) and torch.equal(g1, g0)
    assert rel_err(host(g1), odens.adjoint(ham.H, G, ham.n_occ)) <= 3e-3


def test_adjoint_differentiation_workload_4096_checkpointed():
    """The differentiation workload (water-like H, N = 4096, symmetric Gaussian G) with the
    stride of least memory: bit-identical to keeping every layer, and sampled rows of the
    eigenbasis formula dTr[DG]/dH = C (C^T sym(G) C o F) C^T."""
    ham, _, G = inputs.differentiation_workload(4096)
    Ht, Gt = dev(ham.H), dev(G)
    _, res = sp2.density(Ht, ham.n_occ, precision="fp16")
    _, g0, _ = sp2.adjoint(Ht, Gt, ham.n_occ, precision="fp16", fwd=res)
    D, g1, r1 = sp2.adjoint(Ht, Gt, ham.n_occ, precision="fp16", fwd=res, checkpoint_stride=-1)
    assert r1.layers == res.layers
    assert torch.equal(g1, g0)
    C, lam = ham.eigvecs, ham.eigvals
    F = odens.response_weights(lam, ham.n_occ)
    M = (C.T @ odens.symmetrise(G) @ C) * F
    pick = np.random.default_rng(2).choice(ham.n, size=6, replace=False)
    ref = C[pick] @ M @ C.T
    got = host(g1[torch.tensor(pick, device="cuda")])
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"\nN=4096 adjoint (checkpointed): layers={r1.layers} sampled-row rel err {err:.2e}")
    assert err <= 3e-4  # measured 3.1e-5
