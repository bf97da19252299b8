"""sp2_density_noalloc: the allocation-free entry point for callers that must not
allocate device memory while running.  Called through the C ABI, its output must
match sp2_density's on the same input, on two calls in a row (the second call
reuses the static workspace the first one left behind).  This file is collected
last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2107_02737_gb300 import inputs
import paper_2107_02737_gb300.sp2 as sp2
from tests._gpu import TOL_D, dev, fro_err, host

pytestmark = pytest.mark.gpu


def _call(lib, H, n, n_occ, D, precision="fp16"):
    st = sp2._new_stats()
    o = sp2.make_opts(precision)
    s = lib.sp2_density_noalloc(ctypes.c_void_p(H.data_ptr()), n, float(n_occ), 1e-6, ctypes.c_void_p(D.data_ptr()),
                                ctypes.byref(st), ctypes.byref(o),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return s, st


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_noalloc_matches_density_on_consecutive_calls(precision):
    lib = sp2.load()
    for k, n in enumerate((300, 512)):
        ham = inputs.gapped_random(n, n // 2, inputs.rng_for(0, 7000 + k))
        H = dev(ham.H)
        D_ref, r_ref = sp2.density(H, ham.n_occ, precision=precision)
        D = torch.full((n, n), float("nan"), dtype=torch.float32, device="cuda")
        s, st = _call(lib, H, n, ham.n_occ, D, precision)
        torch.cuda.synchronize()
        assert s == sp2.OK
        assert st.layers == r_ref.layers
        assert fro_err(host(D), host(D_ref)) <= TOL_D[precision] * 1e-3
        assert np.max(np.abs(host(D) - host(D_ref))) <= 1e-6


def test_noalloc_rejects_what_it_cannot_serve():
    lib = sp2.load()
    n = sp2.NOALLOC_MAX_N + 1
    H = dev(np.eye(n))
    D = torch.empty((n, n), dtype=torch.float32, device="cuda")
    assert _call(lib, H, n, n // 2, D)[0] == sp2.ERR_ARG
    Hh = torch.eye(8, dtype=torch.float64)  # host memory would need staging
    Dd = torch.empty((8, 8), dtype=torch.float32, device="cuda")
    assert _call(lib, Hh, 8, 4, Dd)[0] == sp2.ERR_ARG
