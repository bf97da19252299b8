"""Host-side HOMO / LUMO estimates from chain statistics (paper_2107_02737_gb300.gap),
checked against the spectra the generators build and the oracle's chains."""
import numpy as np
import pytest

from oracle import sp2 as osp2
from paper_2107_02737_gb300 import gap, inputs


def _check(est, eigvals, n_occ, frac=0.5):
    assert est is not None
    e_homo, e_lumo = est
    homo, lumo = eigvals[n_occ - 1], eigvals[n_occ]
    w = lumo - homo
    # overlapping the gap is what the accelerated chain needs
    assert e_lumo > homo and e_homo < lumo and e_homo < e_lumo
    # and the estimates land near the true levels
    assert abs(e_homo - homo) <= frac * w and abs(e_lumo - lumo) <= frac * w


@pytest.mark.parametrize("maker", ["water2048", "gapped512", "gapped_third"])
def test_estimate_from_plain_chain(maker):
    if maker == "water2048":
        ham = inputs.water_like_workload(2048)
    elif maker == "gapped512":
        ham = inputs.gapped_random(512, 256, np.random.default_rng(3))
    else:
        ham = inputs.gapped_random(600, 200, np.random.default_rng(4), occ_range=(-1, -0.01), virt_range=(0.01, 1))
    lo, hi = osp2.gershgorin_bounds(ham.H)
    _, stats, _, _ = osp2.scalar_sp2(ham.eigvals, ham.n_occ, lo, hi)
    est = gap.estimate_gap([s.trace for s in stats], [s.trace_sq for s in stats], [s.choice for s in stats[1:]],
                           None, ham.n_occ, lo, hi)
    _check(est, ham.eigvals, ham.n_occ)


def test_estimate_from_accelerated_chain():
    ham = inputs.gapped_random(300, 120, np.random.default_rng(5), occ_range=(-1, -0.02), virt_range=(0.02, 1))
    homo, lumo = ham.eigvals[119], ham.eigvals[120]
    w = lumo - homo
    r = osp2.sp2(ham.H, ham.n_occ, gap=(homo - 2 * w, lumo + 3 * w))
    assert r.converged and max(r.alphas) > 1.0
    est = gap.estimate_gap([s.trace for s in r.stats], [s.trace_sq for s in r.stats], r.choices, r.alphas,
                           ham.n_occ, r.eps_min, r.eps_max)
    _check(est, ham.eigvals, ham.n_occ)


def test_estimate_with_noisy_statistics():
    # Rounding noise on the statistics (of the size the split-precision chain shows)
    # only moves the estimates deeper into the gap or leaves them out.
    ham = inputs.water_like_workload(2048)
    lo, hi = osp2.gershgorin_bounds(ham.H)
    _, stats, _, _ = osp2.scalar_sp2(ham.eigvals, ham.n_occ, lo, hi)
    rng = np.random.default_rng(6)
    t = np.array([s.trace for s in stats]) + 1e-5 * rng.standard_normal(len(stats))
    q = np.array([s.trace_sq for s in stats]) + 1e-5 * rng.standard_normal(len(stats))
    est = gap.estimate_gap(t, q, [s.choice for s in stats[1:]], None, ham.n_occ, lo, hi, floor=1e-3)
    _check(est, ham.eigvals, ham.n_occ, frac=0.6)


def test_estimate_drives_an_accelerated_chain_to_the_same_density():
    ham = inputs.gapped_random(256, 128, np.random.default_rng(7))
    plain = osp2.sp2(ham.H, ham.n_occ)
    est = gap.estimate_gap([s.trace for s in plain.stats], [s.trace_sq for s in plain.stats], plain.choices,
                           None, ham.n_occ, plain.eps_min, plain.eps_max)
    acc = osp2.sp2(ham.H, ham.n_occ, gap=est)
    assert acc.converged and acc.layers < plain.layers
    np.testing.assert_allclose(acc.D, plain.D, atol=1e-6)


def test_no_estimate_from_an_empty_chain():
    assert gap.estimate_gap([1.0], [1.0], [], None, 1, 0.0, 1.0) is None
