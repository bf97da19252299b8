"""Kernel-level parity: one or two SP2 layers applied to a given X_0, through the C ABI
(``sp2_apply_layers``), against float64 products of the same FP32 input."""
import numpy as np
import pytest
import torch

from oracle import sp2 as osp2
from paper_2107_02737_gb300 import inputs
import paper_2107_02737_gb300.sp2 as sp2
from tests._gpu import dev, host

pytestmark = pytest.mark.gpu

# Max-abs error of one square for entries of X with ||X||_2 <= 1 (derived from the
# representation error of each split and FP32 accumulation over K = 3N terms).
TOL_SQ = {"fp32": 2e-6, "fp16": 5e-6, "bf16": 6e-5}


def start_matrix(n, seed):
    ham = inputs.gapped_random(n, n // 2, np.random.default_rng(seed))
    lo, hi = osp2.gershgorin_bounds(ham.H)
    return osp2.input_layer(ham.H, lo, hi).astype(np.float32)


# (precision, CTAs per tensor-core tile): the FP32 path ignores the tile shape.
PATHS = [("fp32", 0), ("fp16", 1), ("fp16", 2), ("bf16", 1), ("bf16", 2)]


@pytest.mark.parametrize("precision,cg", PATHS)
@pytest.mark.parametrize("n", [256, 300, 640])
@pytest.mark.parametrize("choice", [0, 1])
def test_one_layer_matches_fp64_product(precision, cg, n, choice):
    X0 = start_matrix(n, 100 + n)
    X, res = sp2.apply_layers(dev(X0, torch.float32), [choice], precision=precision, cta_group=cg)
    got = host(X)
    x = X0.astype(np.float64)
    ref = osp2.apply_layer(x, choice)
    assert np.max(np.abs(got - ref)) < TOL_SQ[precision]
    # mirror stores make the result exactly symmetric
    assert np.array_equal(got, got.T)
    # FP64 traces of the result.  On the tensor-core path the statistics describe
    # stored X + c I exactly while the returned matrix rounds the diagonal sum to
    # FP32, so they agree to N FP32 half-ulps of the diagonal there.
    assert res.layers == 1
    rt = 1e-12 if precision == "fp32" else 0.0
    at = 1e-12 if precision == "fp32" else n * 2.0 ** -24
    assert res.trace[1] == pytest.approx(np.trace(got), rel=rt, abs=at)
    assert res.trace_sq[1] == pytest.approx(np.sum(got * got), rel=rt, abs=2 * at)
    assert res.trace[0] == pytest.approx(np.trace(x), rel=1e-12)
    assert res.trace_sq[0] == pytest.approx(np.sum(x * x), rel=1e-12)


@pytest.mark.parametrize("precision,cg", PATHS)
def test_layer_sequence_matches_replay(precision, cg):
    n = 384
    X0 = start_matrix(n, 7)
    choices = [0, 1, 1, 0, 1]
    X, res = sp2.apply_layers(dev(X0, torch.float32), choices, precision=precision, cta_group=cg)
    x = X0.astype(np.float64)
    for c in choices:
        x = osp2.apply_layer(x, c)
    assert res.choices == choices
    assert np.max(np.abs(host(X) - x)) < 5 * TOL_SQ[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_deterministic(precision):
    X0 = dev(start_matrix(512, 9), torch.float32)
    a, ra = sp2.apply_layers(X0, [0, 1, 0], precision=precision)
    b, rb = sp2.apply_layers(X0, [0, 1, 0], precision=precision)
    assert torch.equal(a, b)
    assert ra.trace == rb.trace and ra.trace_sq == rb.trace_sq


def test_tile_shapes_agree():
    # 128 x 256 single-CTA tiles and 256 x 256 CTA-pair tiles: same products,
    # different accumulation splits, so agreement within the split tolerance.
    X0 = dev(start_matrix(640, 11), torch.float32)
    a, _ = sp2.apply_layers(X0, [0, 1], precision="fp16", cta_group=1)
    b, _ = sp2.apply_layers(X0, [0, 1], precision="fp16", cta_group=2)
    assert float((a - b).abs().max()) < 2 * TOL_SQ["fp16"]


def test_zero_layers_returns_input():
    X0 = start_matrix(200, 3)
    X, res = sp2.apply_layers(dev(X0, torch.float32), [], precision="fp16")
    assert np.array_equal(host(X), X0.astype(np.float64))
    assert res.layers == 0
