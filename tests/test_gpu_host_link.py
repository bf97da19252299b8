"""Host-resident calls: page-locked matrices are used in place across the host
link (H and a response's H1 read from their lower triangle, D / D1 / dH written
directly), pageable ones copied whole.  Every combination must give the
device-resident call's result bit for bit."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2107_02737_gb300 import inputs, sp2
from tests._gpu import dev

pytestmark = pytest.mark.gpu


def _pinned(a, dtype=torch.float64):
    t = torch.tensor(np.ascontiguousarray(a), dtype=dtype).pin_memory()
    assert t.is_pinned()
    return t


def _pageable(a, dtype=torch.float64):
    t = torch.tensor(np.ascontiguousarray(a), dtype=dtype)
    assert not t.is_pinned()
    return t


MAKE = {"pinned": _pinned, "pageable": _pageable}


@pytest.fixture(scope="module", params=[300, 1000])
def ham(request):
    n = request.param  # ragged against the 32 x 32 staging tiles and the 128-row operand tiles
    return inputs.gapped_random(n, n // 2, inputs.rng_for(7, n))


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
@pytest.mark.parametrize("h_kind,d_kind", [("pinned", "pinned"), ("pageable", "pageable"),
                                           ("pinned", "pageable"), ("pageable", "pinned")])
def test_density_host_buffers_equal_device(ham, precision, h_kind, d_kind):
    n = ham.n
    ref, rr = sp2.density(dev(ham.H), ham.n_occ, precision=precision)
    out = MAKE[d_kind](np.full((n, n), np.nan), torch.float32)
    D, r = sp2.density(MAKE[h_kind](ham.H), ham.n_occ, precision=precision, out=out)
    assert D.data_ptr() == out.data_ptr()
    assert torch.equal(D, ref.cpu())
    assert r.choices == rr.choices
    assert r.band_energy == rr.band_energy and r.trace_D == rr.trace_D


def test_binding_returns_pinned_result_for_pinned_input(ham):
    D, _ = sp2.density(_pinned(ham.H), ham.n_occ)
    assert D.device.type == "cpu" and D.is_pinned()
    D, _ = sp2.density(_pageable(ham.H), ham.n_occ)
    assert D.device.type == "cpu" and not D.is_pinned()


def test_pinned_h_crosses_as_its_lower_triangle(ham):
    """Only the lower triangle of a page-locked H crosses the link: garbage above the
    diagonal changes nothing, and the result is that of the mirrored lower half.  A
    pageable H is copied whole, but the split-precision chain reads only its lower
    triangle on the device, so the result is the same there too."""
    n = ham.n
    assert np.array_equal(ham.H, ham.H.T)
    scrambled = ham.H + np.triu(1e-3 * np.random.default_rng(3).standard_normal((n, n)), 1)
    ref, _ = sp2.density(dev(ham.H), ham.n_occ)
    D, _ = sp2.density(_pinned(scrambled), ham.n_occ)
    assert torch.equal(D, ref.cpu())
    D2, _ = sp2.density(_pageable(scrambled), ham.n_occ)
    assert torch.equal(D2, ref.cpu())


@pytest.mark.parametrize("kind", ["pinned", "pageable"])
def test_response_host_buffers_equal_device(ham, kind):
    H1 = inputs.symmetric_gaussian(ham.n, inputs.rng_for(7, 20 + ham.n)) * 0.01
    Dr, D1r, rr = sp2.response(dev(ham.H), dev(H1), ham.n_occ)
    D, D1, r = sp2.response(MAKE[kind](ham.H), MAKE[kind](H1), ham.n_occ)
    assert D.device.type == "cpu" and D1.device.type == "cpu"
    assert torch.equal(D, Dr.cpu()) and torch.equal(D1, D1r.cpu())
    assert r.choices == rr.choices


@pytest.mark.parametrize("kind", ["pinned", "pageable"])
def test_adjoint_host_buffers_equal_device_with_asymmetric_weight(ham, kind):
    """The adjoint's weight G need not be symmetric, so it is never read from one triangle."""
    G = np.random.default_rng(11).standard_normal((ham.n, ham.n))
    assert not np.array_equal(G, G.T)
    Dr, gr, rr = sp2.adjoint(dev(ham.H), dev(G), ham.n_occ)
    D, g, r = sp2.adjoint(MAKE[kind](ham.H), MAKE[kind](G), ham.n_occ)
    assert torch.equal(D, Dr.cpu()) and torch.equal(g, gr.cpu())
    assert r.choices == rr.choices


def test_batched_pinned_members_equal_device():
    hams = [inputs.gapped_random(n, n // 2, inputs.rng_for(8, n)) for n in (200, 333, 640)]
    n_occ = [h.n_occ for h in hams]
    ref, _, s0 = sp2.density_batched([dev(h.H) for h in hams], n_occ, precision="bf16")
    Ds, _, s1 = sp2.density_batched([_pinned(hams[0].H), dev(hams[1].H), _pinned(hams[2].H)], n_occ,
                                    precision="bf16")
    assert s0 == sp2.OK and s1 == sp2.OK
    assert Ds[0].is_pinned() and Ds[1].device.type == "cuda" and Ds[2].is_pinned()
    for a, b in zip(Ds, ref):
        assert torch.equal(a.cpu(), b.cpu())


def test_pinned_output_needs_no_staging():
    """With every device allocation failing (test_hook = 2) and a workspace with room
    for H's staging only, a page-locked D succeeds (written in place) while a
    pageable D, which needs a staging buffer too, reports NOMEM."""
    n = 256
    ham = inputs.gapped_random(n, 128, inputs.rng_for(9, n))
    o = sp2.make_opts("fp16")
    o.test_hook = 2
    ws = torch.empty(sp2.workspace_bytes(n, precision="fp16") + n * n * 8 + 512, dtype=torch.uint8, device="cuda")
    Hh = _pinned(ham.H)
    ref, _ = sp2.density(dev(ham.H), ham.n_occ)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(D):
        st = sp2._new_stats()
        return sp2.load().sp2_density(ctypes.c_void_p(Hh.data_ptr()), n, float(ham.n_occ), 1e-6,
                                      ctypes.c_void_p(D.data_ptr()), ctypes.byref(st), ctypes.byref(o),
                                      ctypes.c_void_p(ws.data_ptr()), ws.numel(), stream)

    Dp = _pinned(np.zeros((n, n)), torch.float32)
    assert call(Dp) == sp2.OK
    assert torch.equal(Dp, ref.cpu())
    assert call(_pageable(np.zeros((n, n)), torch.float32)) == sp2.ERR_NOMEM


def test_fp64_entry_points_read_pinned_h_from_its_lower_triangle():
    """sp2_density_refined and sp2_density_nonorth follow the same convention: a
    page-locked H is read from its lower triangle, a non-symmetric Z is copied whole."""
    from oracle import density as odens

    n = 300
    ham = inputs.gapped_random(n, 150, inputs.rng_for(10, n))
    scrambled = ham.H + np.triu(1e-3 * np.random.default_rng(4).standard_normal((n, n)), 1)
    ref, _ = sp2.density_refined(dev(ham.H), ham.n_occ, refine_layers=1)
    D, _ = sp2.density_refined(_pinned(scrambled), ham.n_occ, refine_layers=1)
    assert D.device.type == "cpu"
    assert float((D - ref.cpu()).abs().max()) <= 1e-12
    S = inputs.overlap_matrix(n, inputs.rng_for(10, n + 1))
    Z = odens.inverse_factor_cholesky(S)
    assert not np.array_equal(Z, Z.T)
    ref, _ = sp2.density_nonorth(dev(ham.H), dev(Z), ham.n_occ)
    D, _ = sp2.density_nonorth(_pinned(scrambled), _pinned(Z), ham.n_occ)
    assert float((D - ref.cpu()).abs().max()) <= 1e-12
