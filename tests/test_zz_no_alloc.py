"""sp2_density_noalloc: the allocation-free entry point, for callers that must not
allocate device memory while running (an MD engine whose device memory is held by
its own pool or another framework's caching allocator, or a step loop that cannot
wait for an allocation).

Called through the C ABI with the allocation-failure hook set (test_hook = 2 makes
every device allocation the library attempts report failure), it must still
succeed, and its D must equal sp2_density's bit for bit, on two calls in a row of
different sizes and precisions in both orders (the second call runs on whatever the
first left in the shared static array).  This file is collected last on purpose:
a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2107_02737_gb300 import inputs
import paper_2107_02737_gb300.sp2 as sp2
from tests._gpu import dev

pytestmark = pytest.mark.gpu

ALLOCATIONS_FAIL = 2  # sp2_opts.test_hook value: every device allocation reports failure


def _call(lib, H, n, n_occ, D, precision="fp16", hook=0):
    st = sp2._new_stats()
    o = sp2.make_opts(precision)
    o.test_hook = hook
    s = lib.sp2_density_noalloc(ctypes.c_void_p(H.data_ptr()), n, float(n_occ), 1e-6, ctypes.c_void_p(D.data_ptr()),
                                ctypes.byref(st), ctypes.byref(o),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return s, st


@pytest.mark.parametrize("first,second", [((512, "fp16"), (300, "bf16")), ((300, "fp16"), (512, "bf16")),
                                          ((512, "bf16"), (300, "fp32"))])
def test_noalloc_equals_density_on_consecutive_calls(first, second):
    lib = sp2.load()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    for k, (n, precision) in enumerate((first, second)):
        ham = inputs.gapped_random(n, n // 2, inputs.rng_for(0, 7000 + n + k))
        H = dev(ham.H)
        D_ref, r_ref = sp2.density(H, ham.n_occ, precision=precision)
        D = torch.full((n, n), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        mark = torch.cuda.memory_allocated()
        s, st = _call(lib, H, n, ham.n_occ, D, precision, hook=ALLOCATIONS_FAIL)
        torch.cuda.synchronize()
        assert s == sp2.OK, sp2.SP2Error(s, "sp2_density_noalloc").args
        assert torch.cuda.memory_allocated() == mark
        assert st.layers == r_ref.layers
        assert torch.equal(D, D_ref)
    assert torch.cuda.memory_allocated() >= before


def test_allocation_hook_is_live():
    """The hook the test above relies on does make an allocating call fail."""
    n = 256
    ham = inputs.gapped_random(n, n // 2, inputs.rng_for(0, 7100))
    H = dev(ham.H)
    D = torch.empty((n, n), dtype=torch.float32, device="cuda")
    st = sp2._new_stats()
    o = sp2.make_opts("fp16")
    o.test_hook = ALLOCATIONS_FAIL
    s = sp2.load().sp2_density(ctypes.c_void_p(H.data_ptr()), n, float(ham.n_occ), 1e-6, ctypes.c_void_p(D.data_ptr()),
                               ctypes.byref(st), ctypes.byref(o), None, 0,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert s == sp2.ERR_NOMEM


def test_noalloc_rejects_what_it_cannot_serve():
    lib = sp2.load()
    n = sp2.NOALLOC_MAX_N + 1
    H = dev(np.eye(n))
    D = torch.empty((n, n), dtype=torch.float32, device="cuda")
    assert _call(lib, H, n, n // 2, D)[0] == sp2.ERR_ARG
    Hh = torch.eye(8, dtype=torch.float64)  # host memory would need staging
    Dd = torch.empty((8, 8), dtype=torch.float32, device="cuda")
    assert _call(lib, Hh, 8, 4, Dd)[0] == sp2.ERR_ARG
