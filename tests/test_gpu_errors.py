"""Error paths on the GPU: non-finite input, degenerate and gapless spectra, and a
device wait that runs out (a barrier arrival that is withheld on purpose) --
each returns a status and leaves the context usable."""
import numpy as np
import pytest
import torch

from oracle import density as odens
from paper_2107_02737_gb300 import inputs
import paper_2107_02737_gb300.sp2 as sp2
from tests._gpu import TOL_D, dev, fro_err, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_input(precision, bad):
    H = inputs.gapped_random(64, 32, np.random.default_rng(2)).H
    H[3, 7] = H[7, 3] = bad
    with pytest.raises(sp2.SP2Error) as e:
        sp2.density(dev(H), 32, precision=precision)
    assert e.value.status == sp2.ERR_NONFINITE


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_scalar_hamiltonian_is_not_converged(precision):
    D, res = sp2.density(dev(np.eye(40) * 0.3), 10, precision=precision)
    assert res.status == sp2.ERR_NOT_CONVERGED


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_gapless_spectrum_hits_layer_limit(precision):
    H = np.diag([-1.0, 0.0, 0.0, 1.0])
    D, res = sp2.density(dev(H), 2, precision=precision, max_layers=30)
    assert res.status == sp2.ERR_NOT_CONVERGED and res.stop_reason == sp2.STOP_MAX
    assert res.layers == 30


@pytest.mark.parametrize("precision,n", [("fp16", 256), ("fp32", 256), ("fp16", 4096)])
def test_barrier_timeout_returns_status(precision, n):
    """CTA 0 withholds its first barrier arrival (or, in the dataflow schedule of a lone
    tensor-core solve, its first tile completion); every other wait must run out after
    timeout_ms and the call return SP2_ERR_TIMEOUT.  N = 4096 takes the dataflow
    schedule over several waves with its rotated tile assignment."""
    ham = inputs.gapped_random(n, n // 2, np.random.default_rng(4))
    o = sp2.make_opts(precision, timeout_ms=100.0)
    o.test_hook = 1
    D = torch.empty((n, n), dtype=torch.float32, device="cuda")
    st = sp2._new_stats()
    H = dev(ham.H)
    import ctypes
    s = sp2.load().sp2_density(ctypes.c_void_p(H.data_ptr()), n, float(n // 2), 1e-6, ctypes.c_void_p(D.data_ptr()),
                               ctypes.byref(st), ctypes.byref(o), None, 0,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert s == sp2.ERR_TIMEOUT
    # the context is still usable
    D2, res = sp2.density(H, n // 2, precision=precision)
    if n <= 512:
        assert fro_err(host(D2), odens.density_matrix(ham.H, n // 2)) <= TOL_D[precision]
    else:
        rows = np.arange(0, n, 257)
        ref = odens.density_rows(ham.eigvecs, n // 2, rows)
        assert np.max(np.abs(host(D2)[rows].astype(np.float64) - ref)) <= 1e-3


def test_unsupported_combinations():
    H = dev(inputs.gapped_random(32, 16, np.random.default_rng(3)).H)
    with pytest.raises(sp2.SP2Error) as e:
        sp2.response(H, H, 16, precision="fp32")
    assert e.value.status == sp2.ERR_UNSUPPORTED
    with pytest.raises(sp2.SP2Error) as e:
        sp2.density(H, 16.5)
    assert e.value.status == sp2.ERR_ARG


def _raw_density(H_ptr, n, n_occ, D, o, ws=None):
    import ctypes
    wsp, wsb = (ctypes.c_void_p(ws.data_ptr()), ws.numel()) if ws is not None else (None, 0)
    st = sp2._new_stats()
    return sp2.load().sp2_density(ctypes.c_void_p(H_ptr), n, float(n_occ), 1e-6, ctypes.c_void_p(D.data_ptr()),
                                  ctypes.byref(st), ctypes.byref(o), wsp, wsb,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_allocation_failure_returns_nomem(precision):
    """Host-side injection (test_hook = 2): every device allocation of the call fails."""
    n = 256
    ham = inputs.gapped_random(n, 128, np.random.default_rng(5))
    H = dev(ham.H)
    D = torch.empty((n, n), dtype=torch.float32, device="cuda")
    o = sp2.make_opts(precision)
    o.test_hook = 2
    # no workspace given: the workspace allocation fails
    assert _raw_density(H.data_ptr(), n, 128, D, o) == sp2.ERR_NOMEM
    # an exact workspace but a host-resident H: its staging allocation fails
    ws = torch.empty(sp2.workspace_bytes(n, precision=precision), dtype=torch.uint8, device="cuda")
    Hh = np.ascontiguousarray(ham.H)
    assert _raw_density(Hh.ctypes.data, n, 128, D, o, ws) == sp2.ERR_NOMEM
    # device-resident inputs in a caller workspace need no allocation at all
    assert _raw_density(H.data_ptr(), n, 128, D, o, ws) == sp2.OK
    assert fro_err(host(D), odens.density_matrix(ham.H, 128)) <= TOL_D[precision]
    # and nothing is left behind: a normal call still works
    D2, _ = sp2.density(H, 128, precision=precision)
    assert torch.equal(D2, D)


def test_pair_residency_timeout_falls_back_to_single_cta():
    """A CTA pair that never becomes resident (test_hook = 3 withholds a barrier arrival in
    pair launches only): with the tile shape left to the library the call retries with
    single-CTA tiles and succeeds; forced to pairs it reports the timeout."""
    import ctypes
    n = 256
    ham = inputs.gapped_random(n, 128, np.random.default_rng(6))
    H = dev(ham.H)
    D = torch.empty((n, n), dtype=torch.float32, device="cuda")
    o = sp2.make_opts("fp16", timeout_ms=100.0)
    o.test_hook = 3
    st = sp2._new_stats()
    s = sp2.load().sp2_density(ctypes.c_void_p(H.data_ptr()), n, 128.0, 1e-6, ctypes.c_void_p(D.data_ptr()),
                               ctypes.byref(st), ctypes.byref(o), None, 0,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert s == sp2.OK and st.cta_group == 1
    assert fro_err(host(D), odens.density_matrix(ham.H, 128)) <= TOL_D["fp16"]
    o.cta_group = 2
    assert _raw_density(H.data_ptr(), n, 128, D, o) == sp2.ERR_TIMEOUT
