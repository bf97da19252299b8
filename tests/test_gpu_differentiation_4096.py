"""The differentiation workload at its own size (water-like H, N = 4096, FP16 split):
the forward response D1 and the adjoint dTr[D G]/dH of the chain against central
differences of the FP64 eigendecomposition oracle, h = 1e-4, along the workload's
own perturbation H1.  The scalar checked is the directional derivative
d/ds Tr[G D(H + s H1)] at s = 0, which is Tr[G D1(H1)] for the response and
<H1, dTr[DG]/dH> for the adjoint (D depends on H only through its eigenvectors'
occupied subspace, which is smooth while the gap stays open)."""
import numpy as np
import pytest
import torch

from oracle import density as odens
from paper_2107_02737_gb300 import inputs
import paper_2107_02737_gb300.sp2 as sp2
from tests._gpu import dev, host

pytestmark = pytest.mark.gpu

H_STEP = 1e-4


@pytest.fixture(scope="module")
def workload():
    ham, H1, G = inputs.differentiation_workload(4096)
    Gs = 0.5 * (G + G.T)
    f = lambda s: float(np.sum(Gs * odens.density_matrix(ham.H + s * H1, ham.n_occ)))
    fd = (f(H_STEP) - f(-H_STEP)) / (2 * H_STEP)
    return ham, H1, G, fd


def test_response_central_differences_4096(workload):
    ham, H1, G, fd = workload
    _, D1, res = sp2.response(dev(ham.H), dev(H1), ham.n_occ, precision="fp16")
    assert res.converged
    got = float(np.sum(0.5 * (G + G.T) * host(D1)))
    err = abs(got - fd) / abs(fd)
    print(f"\nN=4096 response: Tr[G D1] = {got:.10e}, central difference {fd:.10e}, rel err {err:.2e}")
    assert err <= 1e-4   # measured 1.0e-5


def test_adjoint_central_differences_4096(workload):
    ham, H1, G, fd = workload
    _, dH, res = sp2.adjoint(dev(ham.H), dev(G), ham.n_occ, precision="fp16", checkpoint_stride=-1)
    assert res.converged
    got = float(np.sum(H1 * host(dH)))
    err = abs(got - fd) / abs(fd)
    print(f"\nN=4096 adjoint: <H1, dH> = {got:.10e}, central difference {fd:.10e}, rel err {err:.2e}")
    assert err <= 1e-4   # measured 1.3e-5
