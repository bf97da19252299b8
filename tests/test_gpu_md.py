"""The MD-sequence driver: every step's D and D1 against the oracle, the band energy
and its k-derivative against the eigendecomposition, and the energy drift along the
trajectory against the oracle's own trapezoid drift (same quadrature, exact inputs)."""
import math

import numpy as np
import pytest
import torch

from oracle import density as odens
from paper_2107_02737_gb300 import inputs, md
import paper_2107_02737_gb300.sp2 as sp2
from tests._gpu import TOL_D, dev, fro_err, host, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trajectory():
    n = 512
    ham = inputs.banded_tight_binding(n, inputs.rng_for(4, 1), n // 2)
    V = inputs.sparse_perturbation(n, inputs.rng_for(4, 2), density=0.05, sigma=0.002)
    return ham, V


@pytest.mark.parametrize("fixed,accelerate", [(False, False), (True, False), (False, True)])
def test_md_steps_match_oracle(trajectory, fixed, accelerate):
    ham, V = trajectory
    run = md.MDSequence(dev(ham.H), dev(V), ham.n_occ, omega=0.3, fixed_bounds=fixed, accelerate=accelerate)
    E_ref, F_ref = [], []
    for k in range(10):
        rec = run.step(k, check_gap=(k % 3 == 0))
        Hk = ham.H + math.sin(0.3 * k) * V
        H1k = 0.3 * math.cos(0.3 * k) * V
        lam, C = odens.eigensystem(Hk)
        true_gap = odens.homo_lumo_gap(lam, ham.n_occ)
        assert true_gap > 0.02  # the trajectory keeps a gap
        # the chain's own estimate overlaps the gap, each end within half a gap of the true
        # level; the eigenvalue check matches the oracle
        assert rec.gap_est is not None and 0.0 < rec.gap_est <= 2.0 * true_gap
        if rec.gap_check is not None:
            assert rec.gap_check == pytest.approx(true_gap, abs=1e-4)
        D_ref = odens.density_from_eigensystem(C, ham.n_occ)
        D1_ref = odens.response_from_eigensystem(lam, C, H1k, ham.n_occ)
        assert rec.stop_reason in (sp2.STOP_TOL, sp2.STOP_STALL)
        assert fro_err(host(run.D), D_ref) <= TOL_D["fp16"]
        assert rel_err(host(run.D1), D1_ref) <= 3e-3
        E_ref.append(lam[:ham.n_occ].sum())
        F_ref.append(np.sum(D_ref * H1k))
        assert rec.band_energy == pytest.approx(E_ref[-1], abs=1e-4 * abs(E_ref[-1]))
        assert rec.dE_dk == pytest.approx(F_ref[-1], abs=1e-3 * max(1e-3, abs(F_ref[-1])))
    if fixed:
        assert len({r.layers for r in run.records}) <= 2   # one interval: near-constant chain length
    if accelerate:
        # steps after the first reuse the previous step's HOMO / LUMO estimate
        assert all(r.accelerated for r in run.records[1:]) and not any(r.fallback for r in run.records)
        assert max(r.layers for r in run.records[1:]) < run.records[0].layers
    dr = run.drift()
    E_ref, F_ref = np.array(E_ref), np.array(F_ref)
    integ = np.concatenate([[0.0], np.cumsum(0.5 * (F_ref[1:] + F_ref[:-1]))])
    ref_dev = (E_ref - E_ref[0]) - integ
    assert dr["max_abs"] == pytest.approx(float(np.max(np.abs(ref_dev))), abs=2e-4)


def test_md_workload_full_size_12288():
    """The MD workload at its full size (N = 12288): the sequence's first Hamiltonian H_0
    and its sparse perturbation V through one sp2_response call, as each MD step makes
    it; sampled rows of D against the generator's eigensystem and of D1 = dD/dH[V]
    against the perturbation formula."""
    ham, V = md.trajectory_inputs(12288)
    n = ham.n
    D, D1, res = sp2.response(dev(ham.H), dev(V), ham.n_occ, precision="fp16")
    assert res.converged
    rows = np.random.default_rng(12).choice(n, size=6, replace=False)
    idx = torch.tensor(rows, device="cuda")
    ref = odens.density_rows(ham.eigvecs, ham.n_occ, rows)
    row_err = float(np.sqrt(np.mean(np.sum((host(D[idx]) - ref) ** 2, axis=1))))
    ref1 = odens.response_rows(ham.eigvals, ham.eigvecs, V, ham.n_occ, rows)
    err1 = float(np.linalg.norm(host(D1[idx]) - ref1) / np.linalg.norm(ref1))
    print(f"\nN=12288 MD start: layers={res.layers} D row err {row_err:.2e}, D1 sampled-row rel err {err1:.2e}, "
          f"Tr D - n_occ {res.trace_D - ham.n_occ:+.2e}")
    assert row_err <= TOL_D["fp16"]
    assert err1 <= 1e-2
