"""The C ABI on the CPU: the library loads without a GPU, exports every symbol that
include/sp2.h declares, and rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2107_02737_gb300 import build
import paper_2107_02737_gb300.sp2 as sp2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sp2.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sp2.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sp2_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), f"libsp2.so does not export {name}"
    assert sorted(names) == sorted(sp2.EXPORTS)


def test_default_opts_and_strings(lib):
    o = sp2.make_opts()
    assert (o.precision, o.max_layers, o.user_bounds, o.test_hook) == (1, 100, 0, 0)
    assert o.timeout_ms == 2000.0
    for code in range(8):
        assert lib.sp2_status_string(code)
    assert lib.sp2_status_string(0) == b"ok"


def test_workspace_sizes_grow_with_n(lib):
    a = sp2.workspace_bytes(256)
    b = sp2.workspace_bytes(4096)
    assert 0 < a < b
    # FP16 split at N = 4096: two FP32 masters + two slots of two 16-bit operands (hi, lo).
    assert b >= 2 * 4096 * 4096 * 4 + 2 * 2 * 4096 * 4096 * 2
    assert sp2.workspace_bytes(512, "adjoint", layers=10) > sp2.workspace_bytes(512, "response")


def _call_density(lib, n, n_occ, tol=1e-6, opts=None):
    H = np.eye(max(n, 1))
    D = np.zeros((max(n, 1), max(n, 1)), np.float32)
    return lib.sp2_density(H.ctypes.data_as(ctypes.c_void_p), n, float(n_occ), tol,
                           D.ctypes.data_as(ctypes.c_void_p), None, opts, None, 0, None)


def test_invalid_arguments_rejected_on_host(lib):
    assert _call_density(lib, 0, 0) == sp2.ERR_ARG
    assert _call_density(lib, 8, 2.5) == sp2.ERR_ARG
    assert _call_density(lib, 8, 9) == sp2.ERR_ARG
    assert _call_density(lib, 8, -1) == sp2.ERR_ARG
    assert _call_density(lib, 8, 4, tol=-1.0) == sp2.ERR_ARG
    o = sp2.make_opts(max_layers=0)
    assert _call_density(lib, 8, 4, opts=ctypes.byref(o)) == sp2.ERR_ARG
    o = sp2.make_opts(bounds=(1.0, 0.0))
    assert _call_density(lib, 8, 4, opts=ctypes.byref(o)) == sp2.ERR_ARG
    o = sp2.make_opts()
    o.test_hook = 4
    assert _call_density(lib, 8, 4, opts=ctypes.byref(o)) == sp2.ERR_ARG
    for stride in (-2, 201):
        o = sp2.make_opts(checkpoint_stride=stride)
        assert _call_density(lib, 8, 4, opts=ctypes.byref(o)) == sp2.ERR_ARG
    # the accelerated chain needs an ordered, finite interval
    for gap in [(0.5, 0.5), (0.6, 0.1), (float("nan"), 0.1), (0.0, float("inf"))]:
        o = sp2.make_opts(gap=gap)
        assert _call_density(lib, 8, 4, opts=ctypes.byref(o)) == sp2.ERR_ARG


def test_acceleration_rejected_where_unsupported(lib):
    o = sp2.make_opts(gap=(-0.1, 0.1))
    H = np.eye(8)
    D = np.zeros((8, 8), np.float32)
    hp = (ctypes.c_void_p * 1)(H.ctypes.data)
    dp = (ctypes.c_void_p * 1)(D.ctypes.data)
    nn = (ctypes.c_int * 1)(8)
    occ = (ctypes.c_double * 1)(4.0)
    assert lib.sp2_density_batched(1, hp, nn, occ, 1e-6, dp, None, ctypes.byref(o), None, 0, None) == sp2.ERR_ARG
    ch = (ctypes.c_int * 1)(0)
    X = np.zeros((8, 8), np.float32)
    assert lib.sp2_apply_layers(X.ctypes.data_as(ctypes.c_void_p), 8, ch, 1, X.ctypes.data_as(ctypes.c_void_p),
                                None, ctypes.byref(o), None) == sp2.ERR_ARG


def test_layer_stat_record_layout():
    # sp2_layer_stat: three doubles, two ints, the expansion a_n
    assert ctypes.sizeof(sp2.LayerStat) == 40 and sp2.LayerStat.alpha.offset == 32
    # sp2_opts ends with eps_lumo and checkpoint_stride (padded to 8 bytes)
    assert sp2.Opts.checkpoint_stride.offset == sp2.Opts.eps_lumo.offset + 8
    assert ctypes.sizeof(sp2.Opts) == sp2.Opts.checkpoint_stride.offset + 8


def test_result_reads_the_layer_records():
    st = sp2._new_stats()
    st.layers, st.stop_reason, st.eps_min, st.cta_group = 3, 1, -2.5, 2
    for k in range(4):
        st.layer[k].trace, st.layer[k].trace_sq, st.layer[k].idem = 1.5 * k, 0.25 * k, 0.125 * k
        st.layer[k].choice, st.layer[k].alpha = k % 2, 1.0 + k
    st.layer[4].trace = 99.0   # beyond the chain: not reported
    r = sp2._result(sp2.OK, st)
    assert (r.layers, r.stop_reason, r.eps_min, r.cta_group) == (3, 1, -2.5, 2)
    assert r.trace == [0.0, 1.5, 3.0, 4.5] and r.trace_sq == [0.0, 0.25, 0.5, 0.75]
    assert r.idem == [0.0, 0.125, 0.25, 0.375]
    assert r.choices == [1, 0, 1] and r.alphas == [2.0, 3.0, 4.0]
    assert all(type(c) is int for c in r.choices) and all(type(t) is float for t in r.trace)
    st.layers = 0
    assert sp2._result(sp2.OK, st).choices == []


def test_apply_layers_rejects_bad_choices(lib):
    X = np.zeros((4, 4), np.float32)
    ch = (ctypes.c_int * 2)(0, 2)
    r = lib.sp2_apply_layers(X.ctypes.data_as(ctypes.c_void_p), 4, ch, 2, X.ctypes.data_as(ctypes.c_void_p),
                             None, None, None)
    assert r == sp2.ERR_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(sp2, "_lib", None)
    monkeypatch.setattr(sp2, "_LIB_PATH", str(tmp_path / "libsp2.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        sp2.load()


def test_batch_plan_rejects_bad_arguments_on_host(lib):
    handle = ctypes.c_void_p()
    H = np.eye(8)
    D = np.zeros((8, 8), np.float32)
    hp = (ctypes.c_void_p * 1)(H.ctypes.data)
    dp = (ctypes.c_void_p * 1)(D.ctypes.data)
    nn = (ctypes.c_int * 1)(8)
    occ = (ctypes.c_double * 1)(4.0)
    bad_occ = (ctypes.c_double * 1)(4.5)
    assert lib.sp2_batch_plan_create(0, hp, nn, occ, 1e-6, dp, None, 0, None, ctypes.byref(handle)) == sp2.ERR_ARG
    assert lib.sp2_batch_plan_create(1, hp, nn, occ, 1e-6, dp, None, 0, None, None) == sp2.ERR_ARG
    assert lib.sp2_batch_plan_create(1, hp, nn, bad_occ, 1e-6, dp, None, 0, None, ctypes.byref(handle)) == sp2.ERR_ARG
    assert lib.sp2_batch_plan_create(1, hp, nn, occ, 1e-6, dp, None, 2, None, ctypes.byref(handle)) == sp2.ERR_ARG
    o = sp2.make_opts(gap=(-0.1, 0.1))
    assert lib.sp2_batch_plan_create(1, hp, nn, occ, 1e-6, dp, ctypes.byref(o), 0, None,
                                     ctypes.byref(handle)) == sp2.ERR_ARG
    # host matrices are not accepted by a plan (its launches make no host copies)
    assert lib.sp2_batch_plan_create(1, hp, nn, occ, 1e-6, dp, None, 0, None, ctypes.byref(handle)) == sp2.ERR_ARG
    assert not handle.value
    assert lib.sp2_batch_plan_launch(None, None) == sp2.ERR_ARG
    assert lib.sp2_batch_plan_cta_group(None) == 0
    lib.sp2_batch_plan_destroy(None)


def test_adjoint_checkpoint_workspace(lib):
    """Keeping every s-th layer (8 bytes per element each: hi, lo and the FP32 master) plus a
    ring of s - 1 (4 bytes) and two FP32 matrices instead of every layer (4 bytes each)."""
    n, L = 1024, 35
    mat = 1024 * 1024
    full = sp2.workspace_bytes(n, "adjoint", layers=L)
    for s in (3, 4, 6, 9):
        k = L // s + 1
        got = sp2.workspace_bytes(n, "adjoint", layers=L, checkpoint_stride=s)
        assert full - got == pytest.approx(mat * (4 * (L + 1) - 4 * (k + s - 1) - 4 * k - 8), abs=1 << 20)
    # stride 2 keeps 18 layers at 8 bytes: no saving over 36 at 4, so every layer is kept
    assert sp2.workspace_bytes(n, "adjoint", layers=L, checkpoint_stride=2) == full
    auto = sp2.workspace_bytes(n, "adjoint", layers=L, checkpoint_stride=-1)
    assert auto == min(sp2.workspace_bytes(n, "adjoint", layers=L, checkpoint_stride=s) for s in range(2, L + 1))
    # a stride that saves nothing keeps every layer
    assert sp2.workspace_bytes(n, "adjoint", layers=3, checkpoint_stride=2) == sp2.workspace_bytes(n, "adjoint", layers=3)


def test_build_compiles_every_cuda_source():
    """The in-tree build (the one the GPU machine runs) lists every translation unit under
    csrc/, so no kernel or entry point can be left out of libsp2.so there."""
    import os

    from paper_2107_02737_gb300 import build

    on_disk = {f for f in os.listdir(build.CSRC) if f.endswith(".cu")}
    assert on_disk == set(build.SOURCES)
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
