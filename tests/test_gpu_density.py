"""End-to-end parity of sp2_density (C ABI) with the FP64 oracle.

Small and ragged sizes are compared element by element with D = theta(mu I - H)
from the eigendecomposition; the per-layer statistics are compared with the
FP64 chain replaying the GPU's own layer signs, and the signs and the stop are
checked against the rules applied to the GPU's own FP64 statistics.  At the full
sizes (N = 4096, 8192) sampled rows of D are compared with rows built from the
generator's eigensystem, and idempotency, trace and commutation are checked.
"""
import numpy as np
import pytest
import torch

from oracle import density as odens
from oracle import sp2 as osp2
from paper_2107_02737_gb300 import inputs
import paper_2107_02737_gb300.sp2 as sp2
from tests._gpu import TOL_D, dev, fro_err, host

pytestmark = pytest.mark.gpu

PRECISIONS = ["fp32", "fp16", "bf16"]


def check_rules(res, n_occ, tol=1e-6, max_layers=100):
    """The signs and the stop the device took follow the rules on its own statistics."""
    for k, c in enumerate(res.choices):
        assert c == osp2.layer_choice(res.trace[k], res.trace_sq[k], n_occ), f"layer {k + 1}"
    for k in range(len(res.idem)):
        assert res.idem[k] == res.trace[k] - res.trace_sq[k]
    reason = osp2.stop_check(res.idem, tol, max_layers)
    assert reason == res.stop_reason
    for k in range(len(res.idem) - 1):
        assert osp2.stop_check(res.idem[:k + 1], tol, max_layers) == 0


@pytest.fixture(scope="module")
def c0():
    return inputs.plain_sp2_workload(256)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_plain_workload_n256(c0, precision):
    D, res = sp2.density(dev(c0.H), c0.n_occ, tol=1e-6, precision=precision)
    Dh = host(D)
    ref = odens.density_matrix(c0.H, c0.n_occ)
    err = fro_err(Dh, ref)
    print(f"\n{precision}: layers={res.layers} reason={res.stop_reason} err={err:.2e} "
          f"trace_err={res.trace_D - c0.n_occ:+.2e} idem={np.linalg.norm(Dh @ Dh - Dh):.2e}")
    assert res.converged
    assert err <= TOL_D[precision]
    assert np.array_equal(Dh, Dh.T)
    check_rules(res, c0.n_occ)
    assert res.trace_D == pytest.approx(np.trace(Dh), abs=1e-9)
    assert res.band_energy == pytest.approx(np.sum(Dh * c0.H), rel=1e-12)
    assert res.band_energy == pytest.approx(c0.eigvals[:c0.n_occ].sum(), rel=1e-4)
    lo, hi = osp2.gershgorin_bounds(c0.H)
    # the device sums |H_ij| as float pairs and widens each disc by 2^-36 relative (plus
    # 2^-50 |H_ii| and N 2^-120) so that it still contains the exact FP64 disc
    assert res.eps_min <= lo and res.eps_max >= hi
    assert (res.eps_min, res.eps_max) == pytest.approx((lo, hi), rel=1e-10)
    # FP32 trace error bound at this size (the stated |Tr D - n_occ| <= 1e-6 target)
    if precision == "fp32":
        assert abs(res.trace_D - c0.n_occ) <= 1e-6


@pytest.mark.parametrize("precision", PRECISIONS)
def test_layer_statistics_match_oracle_replay(c0, precision):
    _, res = sp2.density(dev(c0.H), c0.n_occ, precision=precision)
    rep = osp2.sp2(c0.H, c0.n_occ, choices=res.choices)
    assert len(rep.stats) == len(res.trace)
    n = c0.n
    for k, s in enumerate(rep.stats):
        # The tensor cores' FP32 accumulator truncates once per K=16 instruction (a
        # relative bias of at most (3N/16) 2^-24 per square); FP32 FMAs round to nearest.
        drift = 0.0 if precision == "fp32" else k * (3 * n / 16) * 2.0 ** -23 * c0.n_occ
        assert res.trace[k] == pytest.approx(s.trace, abs=2e-4 + drift), k
        assert res.trace_sq[k] == pytest.approx(s.trace_sq, abs=2e-4 + drift), k
    # Until the chain reaches the rounding floor the signs agree with the FP64 chain's own.
    own = osp2.sp2(c0.H, c0.n_occ)
    k = 0
    while k < min(len(own.choices), len(res.choices)) and abs(own.stats[k].idem) > 1e-3:
        assert own.choices[k] == res.choices[k]
        k += 1
    assert k >= 10


@pytest.mark.parametrize("precision,cg", [("fp32", 0), ("fp16", 1), ("fp16", 2), ("bf16", 1), ("bf16", 2)])
@pytest.mark.parametrize("n", [300, 1000])
def test_ragged_sizes(precision, cg, n):
    ham = inputs.gapped_random(n, n // 3, inputs.rng_for(0, n))
    D, res = sp2.density(dev(ham.H), ham.n_occ, precision=precision, cta_group=cg)
    Dh = host(D)
    ref = odens.density_from_eigensystem(ham.eigvecs, ham.n_occ)
    assert res.converged
    assert fro_err(Dh, ref) <= TOL_D[precision]
    check_rules(res, ham.n_occ)


@pytest.mark.parametrize("precision,cg", [("fp32", 0), ("fp16", 2), ("bf16", 1)])
@pytest.mark.parametrize("n", [301, 1001])
def test_odd_sizes_and_unaligned_buffers(precision, cg, n):
    """Odd N and H, D that start off their vector alignment take the scalar paths of the
    lower-triangle passes (bounds, input layer, output); D is the same bit for bit."""
    ham = inputs.gapped_random(n, n // 3, inputs.rng_for(3, n))
    D, res = sp2.density(dev(ham.H), ham.n_occ, precision=precision, cta_group=cg)
    Dh = host(D)
    assert res.converged
    assert fro_err(Dh, odens.density_from_eigensystem(ham.eigvecs, ham.n_occ)) <= TOL_D[precision]
    lo, hi = osp2.gershgorin_bounds(ham.H)
    assert res.eps_min <= lo and res.eps_max >= hi
    assert (res.eps_min, res.eps_max) == pytest.approx((lo, hi), rel=1e-10)
    hbuf = torch.empty(n * n + 1, dtype=torch.float64, device="cuda")
    hbuf[1:] = dev(ham.H).reshape(-1)
    dbuf = torch.empty(n * n + 1, dtype=torch.float32, device="cuda")
    D2, res2 = sp2.density(hbuf[1:].view(n, n), ham.n_occ, precision=precision, cta_group=cg,
                           out=dbuf[1:].view(n, n))
    assert np.array_equal(host(D2), Dh)
    assert (res2.eps_min, res2.eps_max, res2.layers) == (res.eps_min, res.eps_max, res.layers)
    assert res2.band_energy == res.band_energy and res2.trace_D == res.trace_D


@pytest.mark.parametrize("precision,n", [("fp16", 300), ("bf16", 1001)])
def test_asymmetric_h_reads_the_lower_triangle(precision, n):
    """On the tensor-core path the bounds, the input layer and the output read H's lower
    triangle only: an H whose upper triangle is changed gives the bits of the symmetric
    matrix built from its lower triangle."""
    ham = inputs.gapped_random(n, n // 2, inputs.rng_for(5, n))
    Ha = ham.H.copy()
    iu = np.triu_indices(n, 1)
    Ha[iu] += np.random.default_rng(6).standard_normal(iu[0].size)
    D1, r1 = sp2.density(dev(Ha), ham.n_occ, precision=precision)
    D2, r2 = sp2.density(dev(ham.H), ham.n_occ, precision=precision)
    assert np.array_equal(host(D1), host(D2))
    assert (r1.eps_min, r1.eps_max, r1.layers, r1.band_energy, r1.trace_D) == \
        (r2.eps_min, r2.eps_max, r2.layers, r2.band_energy, r2.trace_D)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_banded_water_like_small(precision):
    ham = inputs.banded_tight_binding(768, inputs.rng_for(1, 768))
    D, res = sp2.density(dev(ham.H), ham.n_occ, precision=precision)
    ref = odens.density_from_eigensystem(ham.eigvecs, ham.n_occ)
    assert res.converged
    assert fro_err(host(D), ref) <= TOL_D[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_deterministic_and_host_pointers(c0, precision):
    H = dev(c0.H)
    a, ra = sp2.density(H, c0.n_occ, precision=precision)
    b, rb = sp2.density(H, c0.n_occ, precision=precision)
    assert torch.equal(a, b)
    assert ra.choices == rb.choices and ra.trace == rb.trace
    # Host-resident H and D go through the library's own staging.
    Hc = torch.tensor(c0.H, dtype=torch.float64).pin_memory()
    c, rc = sp2.density(Hc, c0.n_occ, precision=precision)
    assert c.device.type == "cpu"
    assert torch.equal(c, a.cpu())
    assert rc.choices == ra.choices


def test_workspace_argument(c0):
    n = c0.n
    ws = torch.empty(sp2.workspace_bytes(n, "density", "fp16"), dtype=torch.uint8, device="cuda")
    a, _ = sp2.density(dev(c0.H), c0.n_occ, workspace=ws)
    b, _ = sp2.density(dev(c0.H), c0.n_occ)
    assert torch.equal(a, b)
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(sp2.SP2Error):
        sp2.density(dev(c0.H), c0.n_occ, workspace=small)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_trivial_and_tiny(precision):
    H = inputs.gapped_random(5, 2, np.random.default_rng(1)).H
    D0, r0 = sp2.density(dev(H), 0, precision=precision)
    D5, r5 = sp2.density(dev(H), 5, precision=precision)
    assert torch.count_nonzero(D0) == 0 and r0.stop_reason == sp2.STOP_TRIVIAL
    assert torch.equal(D5, torch.eye(5, device="cuda")) and r5.stop_reason == sp2.STOP_TRIVIAL
    assert r5.band_energy == pytest.approx(np.trace(H))
    D2, r2 = sp2.density(dev(H), 2, precision=precision)
    assert fro_err(host(D2), odens.density_matrix(H, 2)) <= TOL_D[precision]
    h2 = np.array([[0.3, -0.7], [-0.7, 1.1]])
    D, r = sp2.density(dev(h2), 1, precision=precision)
    assert fro_err(host(D), odens.density_matrix(h2, 1)) <= TOL_D[precision]


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_user_bounds(c0, precision):
    lam = c0.eigvals
    bounds = (lam[0] - 0.01, lam[-1] + 0.01)
    D, res = sp2.density(dev(c0.H), c0.n_occ, precision=precision, bounds=bounds)
    assert (res.eps_min, res.eps_max) == bounds
    assert fro_err(host(D), odens.density_matrix(c0.H, c0.n_occ)) <= TOL_D[precision]
    _, rg = sp2.density(dev(c0.H), c0.n_occ, precision=precision)
    assert res.layers < rg.layers  # tight bounds need fewer layers


def _full_size_checks(ham, precision, rows=8, cta_group=0):
    H = dev(ham.H)
    D, res = sp2.density(H, ham.n_occ, precision=precision, cta_group=cta_group)
    torch.cuda.synchronize()
    n = ham.n
    assert res.converged
    check_rules(res, ham.n_occ)
    pick = np.random.default_rng(5).choice(n, size=rows, replace=False)
    ref_rows = odens.density_rows(ham.eigvecs, ham.n_occ, pick)
    got_rows = host(D[torch.tensor(pick, device="cuda")])
    row_err = float(np.sqrt(np.mean(np.sum((got_rows - ref_rows) ** 2, axis=1))))
    Dd = D.double()
    idem = float(torch.linalg.norm(Dd @ Dd - Dd)) / np.sqrt(n)
    comm = float(torch.linalg.norm(H @ Dd - Dd @ H)) / np.sqrt(n)
    print(f"\nN={n} {precision}: layers={res.layers} reason={res.stop_reason} row_err={row_err:.2e} "
          f"idem={idem:.2e} comm={comm:.2e} trace_err={res.trace_D - ham.n_occ:+.2e}")
    # per-row RMS error estimates ||D - D_oracle||_F / sqrt(N) on sampled rows
    assert row_err <= TOL_D[precision]
    assert idem <= TOL_D[precision]
    assert comm <= 10 * TOL_D[precision]
    return res


@pytest.fixture(scope="module")
def c1_4096():
    return inputs.water_like_workload(4096)


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_full_size_4096(c1_4096, precision):
    _full_size_checks(c1_4096, precision)


def test_full_size_4096_single_cta_tiles(c1_4096):
    _full_size_checks(c1_4096, "fp16", cta_group=1)


def test_full_size_8192_fp16():
    _full_size_checks(inputs.water_like_workload(8192), "fp16")
