"""sp2_density_batched: one grouped persistent launch over instances of uneven size.
Each instance must equal its own sp2_density run bit for bit (same tiles, same
arithmetic, same decisions) and match the oracle."""
import numpy as np
import pytest
import torch

from oracle import density as odens
from paper_2107_02737_gb300 import inputs
import paper_2107_02737_gb300.sp2 as sp2
from tests._gpu import TOL_D, dev, fro_err, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp32"])
def test_batched_equals_unbatched(precision):
    sizes = [128, 640, 256, 384, 130, 512]
    hams = [inputs.gapped_random(n, n // 2, inputs.rng_for(2, 500 + i)) for i, n in enumerate(sizes)]
    Ds, res, status = sp2.density_batched([dev(h.H) for h in hams], [h.n_occ for h in hams], precision=precision)
    assert status == sp2.OK
    for h, D, r in zip(hams, Ds, res):
        D1, r1 = sp2.density(dev(h.H), h.n_occ, precision=precision)
        assert torch.equal(D, D1), h.n
        assert r.choices == r1.choices and r.trace == r1.trace
        assert fro_err(host(D), odens.density_from_eigensystem(h.eigvecs, h.n_occ)) <= TOL_D[precision]


def test_batched_with_trivial_and_host_members():
    hams = [inputs.gapped_random(n, n // 2, inputs.rng_for(2, 900 + n)) for n in (200, 300)]
    Hs = [dev(hams[0].H), torch.tensor(hams[1].H, dtype=torch.float64), dev(np.eye(4))]
    Ds, res, status = sp2.density_batched(Hs, [hams[0].n_occ, hams[1].n_occ, 0], precision="bf16")
    assert status == sp2.OK
    assert Ds[1].device.type == "cpu"
    assert fro_err(host(Ds[1]), odens.density_from_eigensystem(hams[1].eigvecs, hams[1].n_occ)) <= 1e-3
    assert torch.count_nonzero(Ds[2]) == 0 and res[2].stop_reason == sp2.STOP_TRIVIAL


def test_batched_workload_64_instances():
    hams = inputs.batched_workload(64)
    Ds, res, status = sp2.density_batched([dev(h.H) for h in hams], [h.n_occ for h in hams], precision="bf16")
    assert status == sp2.OK
    errs = [fro_err(host(D), odens.density_from_eigensystem(h.eigvecs, h.n_occ)) for h, D in zip(hams, Ds)]
    print(f"\nbatched 64: max err {max(errs):.2e}, layers {min(r.layers for r in res)}..{max(r.layers for r in res)}")
    assert max(errs) <= TOL_D["bf16"]


@pytest.mark.parametrize("n,precision,cta_group", [(4096, "fp16", 1), (4096, "fp16", 2), (1000, "fp16", 2),
                                                   (2500, "bf16", 2), (1000, "bf16", 1)])
def test_dataflow_schedule_equals_barrier_schedule(n, precision, cta_group):
    """A lone density solve runs its layers without a grid barrier between them (each
    K block waits for the tiles that wrote it, the decision waits for the whole layer);
    the same instance in a batch runs with the barrier.  Every tile's arithmetic is the
    same, so D and every layer's statistics agree bit for bit: over several waves of
    tiles (N = 4096: 136 pair tiles, 272 single-CTA tiles) and at ragged sizes whose
    last pair tiles overhang the padded matrix (N = 1000, 2500: N_p = 1024, 2560)."""
    ham = inputs.water_like_workload(n) if n == 4096 else inputs.gapped_random(n, n // 2, inputs.rng_for(2, n))
    H = dev(ham.H)
    D1, r1 = sp2.density(H, ham.n_occ, precision=precision, cta_group=cta_group)
    small = inputs.gapped_random(128, 64, inputs.rng_for(2, 1))
    Ds, res, status = sp2.density_batched([H, dev(small.H)], [ham.n_occ, 64], precision=precision,
                                          cta_group=cta_group)
    assert status == sp2.OK and r1.converged
    assert r1.cta_group == cta_group
    assert torch.equal(Ds[0], D1)
    assert res[0].choices == r1.choices and res[0].trace == r1.trace and res[0].trace_sq == r1.trace_sq
