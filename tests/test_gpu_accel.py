"""Parity of the accelerated chain (sp2_opts.accelerate) with the oracle: the FP64
chain replaying the GPU's layer signs and expansions, the definition theta(mu I - H),
the oracle's own expansions from the same interval, and, for the response and the
adjoint, the FP64 chain derivatives and theta's perturbation formula."""
import numpy as np
import pytest
import torch

from oracle import density as odens
from oracle import sp2 as osp2
from paper_2107_02737_gb300 import inputs
import paper_2107_02737_gb300.sp2 as sp2
from tests._gpu import TOL_D, dev, fro_err, host, rel_err

pytestmark = pytest.mark.gpu

PATHS = [("fp32", 0), ("fp16", 1), ("fp16", 2), ("bf16", 2)]


def exact_gap(ham):
    return float(ham.eigvals[ham.n_occ - 1]), float(ham.eigvals[ham.n_occ])


@pytest.fixture(scope="module", params=[256, 520])
def case(request):
    n = request.param
    ham = inputs.gapped_random(n, n // 2, inputs.rng_for(5, n), occ_range=(-1.0, -0.02), virt_range=(0.02, 1.0))
    return ham


@pytest.mark.parametrize("precision,cg", PATHS)
def test_accelerated_density(case, precision, cg):
    ham = case
    gap = exact_gap(ham)
    D, res = sp2.density(dev(ham.H), ham.n_occ, precision=precision, cta_group=cg, gap=gap)
    _, plain = sp2.density(dev(ham.H), ham.n_occ, precision=precision, cta_group=cg)
    assert res.converged
    ref = odens.density_from_eigensystem(ham.eigvecs, ham.n_occ)
    err = fro_err(host(D), ref)
    print(f"\n{precision}/cg{cg} N={ham.n}: layers {res.layers} (plain {plain.layers}), err {err:.2e}, "
          f"trace err {res.trace_D - ham.n_occ:+.2e}")
    assert err <= TOL_D[precision]
    assert res.layers <= 0.7 * plain.layers
    assert all(1.0 <= a <= 2.0 for a in res.alphas) and res.alphas[0] > 1.0
    # The device tracks the interval ends in FP32: its expansions follow the oracle's
    # for the same signs to FP32 rounding.
    ora = osp2.sp2(ham.H, ham.n_occ, bounds=(res.eps_min, res.eps_max), choices=res.choices, gap=gap)
    np.testing.assert_allclose(res.alphas, ora.alphas, rtol=1e-5)
    # Every sign follows the trace rule from the device's own FP64 statistics.
    for n, c in enumerate(res.choices):
        assert c == osp2.layer_choice(res.trace[n], res.trace_sq[n], ham.n_occ)
    # The FP64 chain with the device's signs and expansions tracks the device's traces.
    rep = osp2.sp2(ham.H, ham.n_occ, bounds=(res.eps_min, res.eps_max), choices=res.choices, alphas=res.alphas)
    tol = 4e-6 * ham.n if precision != "fp32" else 5e-7 * ham.n  # measured: <= 1.6e-6 n, 1.5e-7 n
    print(f"max trace deviation from the FP64 replay: {np.max(np.abs(np.array(res.trace) - [s.trace for s in rep.stats])):.2e}")
    assert np.max(np.abs(np.array(res.trace) - [s.trace for s in rep.stats])) <= tol
    assert fro_err(host(D), rep.D) <= TOL_D[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_accelerated_plain_interval_is_the_plain_chain(case, precision):
    # The interval [eps_min, eps_max] keeps every a_n = 1.
    ham = case
    D0, r0 = sp2.density(dev(ham.H), ham.n_occ, precision=precision)
    D1, r1 = sp2.density(dev(ham.H), ham.n_occ, precision=precision, gap=(r0.eps_min, r0.eps_max))
    assert set(r1.alphas) == {1.0}
    assert r1.choices == r0.choices and torch.equal(D0, D1)


@pytest.mark.parametrize("how", ["wider", "narrower", "shifted"])
def test_accelerated_overlapping_estimates(case, how):
    ham = case
    e_h, e_l = exact_gap(ham)
    w = e_l - e_h
    est = {"wider": (e_h - 4 * w, e_l + 4 * w), "narrower": (e_h + 0.25 * w, e_l - 0.25 * w),
           "shifted": (e_h + 0.5 * w, e_l + 0.5 * w)}[how]
    D, res = sp2.density(dev(ham.H), ham.n_occ, precision="fp16", gap=est)
    assert res.converged
    assert fro_err(host(D), odens.density_from_eigensystem(ham.eigvecs, ham.n_occ)) <= TOL_D["fp16"]


def test_accelerated_interval_missing_the_gap_is_reported():
    # An interval between two occupied levels breaks the separation of the images:
    # the chain does not settle and the call reports it (status, not an exception).
    ham = inputs.gapped_random(256, 128, inputs.rng_for(5, 9))
    k = ham.n_occ
    D, res = sp2.density(dev(ham.H), k, precision="fp16", max_layers=60,
                         gap=(float(ham.eigvals[k - 3]), float(ham.eigvals[k - 2])))
    ref = odens.density_from_eigensystem(ham.eigvecs, k)
    assert not res.converged or fro_err(host(D), ref) > 1e-2


def test_accelerated_water_like_n4096():
    ham = inputs.water_like_workload(4096)
    gap = exact_gap(ham)
    D, res = sp2.density(dev(ham.H), ham.n_occ, precision="fp16", gap=gap)
    _, plain = sp2.density(dev(ham.H), ham.n_occ, precision="fp16")
    rows = np.arange(0, 4096, 97)
    ref = odens.density_rows(ham.eigvecs, ham.n_occ, rows)
    err = float(np.linalg.norm(host(D)[rows] - ref) / np.sqrt(len(rows)))
    print(f"\nwater-like 4096: layers {res.layers} vs plain {plain.layers}, sampled-row err {err:.2e}, "
          f"trace err {res.trace_D - ham.n_occ:+.2e}")
    assert res.converged and err <= TOL_D["fp16"]
    assert res.layers <= 0.65 * plain.layers
    assert abs(res.trace_D - ham.n_occ) <= 1e-3


@pytest.mark.parametrize("precision", ["fp16", "bf16"])  # the response runs on the tensor-core path
def test_accelerated_response(precision):
    n = 300
    ham = inputs.gapped_random(n, 150, inputs.rng_for(5, 31))
    H1 = inputs.symmetric_gaussian(n, inputs.rng_for(5, 32)) * 0.01
    gap = exact_gap(ham)
    D, res = sp2.density(dev(ham.H), ham.n_occ, precision=precision, gap=gap)
    D2, D1, r2 = sp2.response(dev(ham.H), dev(H1), ham.n_occ, precision=precision, fwd=res)
    assert r2.choices == res.choices and r2.alphas == res.alphas and torch.equal(D, D2)
    D3, D1b, r3 = sp2.response(dev(ham.H), dev(H1), ham.n_occ, precision=precision, gap=gap)
    assert torch.equal(D1, D1b)  # deciding on the device reproduces the replayed chain
    chain = osp2.chain_response(ham.H, H1, res.choices, res.eps_min, res.eps_max, alphas=res.alphas)
    theta = odens.response_from_eigensystem(ham.eigvals, ham.eigvecs, H1, ham.n_occ)
    g = host(D1)
    tol = 2e-3 if precision == "fp16" else 2e-2
    print(f"\n{precision}: D1 rel err vs chain {rel_err(g, chain):.2e}, vs theta {rel_err(g, theta):.2e}")
    assert rel_err(g, chain) <= tol
    assert rel_err(g, theta) <= tol + 1e-3


def test_accelerated_adjoint_and_duality():
    n = 320
    ham = inputs.gapped_random(n, 120, inputs.rng_for(5, 41))
    rng = inputs.rng_for(5, 42)
    G = rng.standard_normal((n, n))
    E = inputs.symmetric_gaussian(n, rng)
    gap = exact_gap(ham)
    D, dH, res = sp2.adjoint(dev(ham.H), dev(G), ham.n_occ, precision="fp16", gap=gap)
    assert res.converged and res.alphas[0] > 1.0
    g = host(dH)
    chain = osp2.chain_adjoint(ham.H, G, res.choices, res.eps_min, res.eps_max, alphas=res.alphas)
    theta = odens.adjoint(ham.H, G, ham.n_occ)
    print(f"\nadjoint: rel err vs chain {rel_err(g, chain):.2e}, vs theta {rel_err(g, theta):.2e}")
    assert rel_err(g, chain) <= 2e-3
    assert rel_err(g, theta) <= 3e-3
    _, D1, _ = sp2.response(dev(ham.H), dev(E), ham.n_occ, precision="fp16", fwd=res)
    lhs = float(np.sum(E * g))
    rhs = float(np.sum(0.5 * (G + G.T) * host(D1)))
    assert lhs == pytest.approx(rhs, rel=5e-3)
