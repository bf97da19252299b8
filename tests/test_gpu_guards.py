"""Stray-write checks without a sanitizer: every output matrix and the caller's
workspace sit between guard regions filled with a known pattern, at sizes with
ragged tiles; after the call the guards must be intact and the results correct."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import density as odens
from paper_2107_02737_gb300 import inputs
import paper_2107_02737_gb300.sp2 as sp2
from tests._gpu import TOL_D, dev, fro_err, host

pytestmark = pytest.mark.gpu

GUARD = 1 << 15          # elements (FP32 outputs) / bytes (workspace) on each side
SENTINEL = -7.25


def guarded_matrix(n):
    buf = torch.full((GUARD + n * n + GUARD,), SENTINEL, dtype=torch.float32, device="cuda")
    return buf, buf[GUARD:GUARD + n * n].view(n, n)


def guarded_workspace(nbytes):
    nbytes = (nbytes + 255) // 256 * 256
    buf = torch.full((GUARD + nbytes + GUARD,), 0xA5, dtype=torch.uint8, device="cuda")
    return buf, buf[GUARD:GUARD + nbytes]


def intact(buf, sentinel):
    return bool(torch.all(buf[:GUARD] == sentinel)) and bool(torch.all(buf[-GUARD:] == sentinel))


def stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("precision,cg", [("fp16", 2), ("fp16", 1), ("bf16", 2), ("fp32", 0)])
@pytest.mark.parametrize("n", [200, 300, 640])
def test_density_writes_stay_inside(precision, cg, n):
    ham = inputs.gapped_random(n, n // 2, inputs.rng_for(9, n))
    dbuf, D = guarded_matrix(n)
    o = sp2.make_opts(precision, cta_group=cg)
    wbuf, ws = guarded_workspace(sp2.load().sp2_density_workspace_bytes(n, ctypes.byref(o)))
    H = dev(ham.H)
    st = sp2._new_stats()
    s = sp2.load().sp2_density(ctypes.c_void_p(H.data_ptr()), n, float(n // 2), 1e-6, ctypes.c_void_p(D.data_ptr()),
                               ctypes.byref(st), ctypes.byref(o), ctypes.c_void_p(ws.data_ptr()), ws.numel(), stream())
    torch.cuda.synchronize()
    assert s == sp2.OK
    assert intact(dbuf, SENTINEL) and intact(wbuf, 0xA5)
    assert fro_err(host(D), odens.density_from_eigensystem(ham.eigvecs, n // 2)) <= TOL_D[precision]


@pytest.mark.parametrize("kind", ["response", "adjoint"])
def test_derivative_writes_stay_inside(kind):
    n = 300
    ham = inputs.gapped_random(n, 150, inputs.rng_for(9, 1))
    E = inputs.symmetric_gaussian(n, inputs.rng_for(9, 2)) * 0.01
    dbuf, D = guarded_matrix(n)
    gbuf, D1 = guarded_matrix(n)
    o = sp2.make_opts("fp16", checkpoint_stride=3 if kind == "adjoint" else 0)
    lib = sp2.load()
    _, fwd = sp2.density(dev(ham.H), 150)
    nb = (lib.sp2_response_workspace_bytes(n, ctypes.byref(o)) if kind == "response"
          else lib.sp2_adjoint_workspace_bytes(n, fwd.layers, ctypes.byref(o)))
    wbuf, ws = guarded_workspace(nb)
    H, Ed = dev(ham.H), dev(E)
    st = sp2._new_stats()
    fn = lib.sp2_response if kind == "response" else lib.sp2_adjoint
    s = fn(ctypes.c_void_p(H.data_ptr()), ctypes.c_void_p(Ed.data_ptr()), n, 150.0, 1e-6, ctypes.byref(fwd.raw),
           ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(D1.data_ptr()), ctypes.byref(st), ctypes.byref(o),
           ctypes.c_void_p(ws.data_ptr()), ws.numel(), stream())
    torch.cuda.synchronize()
    assert s == sp2.OK
    assert intact(dbuf, SENTINEL) and intact(gbuf, SENTINEL) and intact(wbuf, 0xA5)
    ref = odens.response_from_eigensystem(ham.eigvals, ham.eigvecs, E, 150)
    assert np.linalg.norm(host(D1) - ref) / np.linalg.norm(ref) <= 3e-3


def test_batched_writes_stay_inside():
    ns = [130, 257, 384, 75]
    hams = [inputs.gapped_random(n, n // 2, inputs.rng_for(9, 100 + n)) for n in ns]
    bufs, Ds = zip(*[guarded_matrix(n) for n in ns])
    Hs = [dev(h.H) for h in hams]
    o = sp2.make_opts("bf16")
    lib = sp2.load()
    nn = (ctypes.c_int * 4)(*ns)
    wbuf, ws = guarded_workspace(lib.sp2_density_batched_workspace_bytes(4, nn, ctypes.byref(o)))
    hp = (ctypes.c_void_p * 4)(*[h.data_ptr() for h in Hs])
    dp = (ctypes.c_void_p * 4)(*[d.data_ptr() for d in Ds])
    occ = (ctypes.c_double * 4)(*[float(n // 2) for n in ns])
    s = lib.sp2_density_batched(4, hp, nn, occ, 1e-6, dp, None, ctypes.byref(o), ctypes.c_void_p(ws.data_ptr()),
                                ws.numel(), stream())
    torch.cuda.synchronize()
    assert s == sp2.OK
    assert intact(wbuf, 0xA5) and all(intact(b, SENTINEL) for b in bufs)
    for h, D in zip(hams, Ds):
        assert fro_err(host(D), odens.density_from_eigensystem(h.eigvecs, h.n_occ)) <= TOL_D["bf16"]


def test_noalloc_writes_stay_inside():
    n = 300
    ham = inputs.gapped_random(n, 150, inputs.rng_for(9, 3))
    dbuf, D = guarded_matrix(n)
    sp2.density_noalloc(dev(ham.H), 150, D)
    torch.cuda.synchronize()
    assert intact(dbuf, SENTINEL)
    assert fro_err(host(D), odens.density_from_eigensystem(ham.eigvecs, 150)) <= TOL_D["fp16"]
