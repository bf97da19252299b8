"""MD-like sequence of Hamiltonians through the SP2 path, with drift tracking.

In quantum-based MD the density matrix is rebuilt at every step from a slowly
changing Hamiltonian (section "Microcanonical MD": one density-matrix solve per
step).  This driver reproduces that access pattern with a synthetic trajectory

    H_k = H_0 + sin(omega k) V,        dH_k/dk = omega cos(omega k) V,

and per step runs ``sp2_response`` (D_k and the response D1_k = dD_k/dk, both
from the library's kernels).  It records the band energy E_k = Tr[D_k H_k]
(reduced in FP64 on the device) and checks it for drift along the trajectory:
because D_k is a spectral projector of H_k, dE/dk = Tr[D_k dH_k/dk]
(Hellmann-Feynman), so E_k - E_0 must match the trapezoid integral of that
derivative up to the quadrature error.

Spectral bounds: by default the library takes Gershgorin bounds at every step.
With ``fixed_bounds`` the driver uses one interval for the whole trajectory,
[g_min(H_0) - |V|_inf, g_max(H_0) + |V|_inf] (|V|_inf the largest absolute row
sum), which contains the spectrum of every H_k (Weyl); the layer sequence then
changes only where the trajectory forces it.

With ``accelerate`` every step after the first runs the accelerated chain from an
estimated HOMO / LUMO interval taken from the previous step's layer statistics
(``gap.estimate_gap``); the interval only has to overlap the new gap, which a
slowly moving trajectory keeps.  A step whose accelerated chain does not settle,
or ends more than 1/2 away from the occupation, is rerun with the plain chain.

Every converged step also records the width of the HOMO / LUMO interval estimated
from its own statistics (``gap.estimate_gap``; None when the chain gives none), and
every ``check_gap_every``-th step the gap of H_k from a library eigenvalue solve, to
flag a trajectory whose gap closes.

    python -m paper_2107_02737_gb300.md --n 12288 --steps 200 [--accelerate]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import time
from typing import List, Optional

import numpy as np
import torch

from . import gap as gap_mod
from . import inputs
from . import sp2


@dataclasses.dataclass
class StepRecord:
    k: int
    layers: int
    stop_reason: int
    band_energy: float        # Tr[D_k H_k], FP64 on the device
    dE_dk: float              # Tr[D_k dH_k/dk]
    trace_err: float          # Tr D_k - n_occ
    ms: float                 # device time of the response solve (both solves after a fallback)
    accelerated: bool = False # the step used an estimated HOMO / LUMO interval
    fallback: bool = False    # ... which failed, so the step was rerun with the plain chain
    gap_est: Optional[float] = None   # eps_lumo - eps_homo as estimated from the chain's statistics
    gap_check: Optional[float] = None # HOMO-LUMO gap of H_k by a library eigenvalue solve (report only)


class MDSequence:
    def __init__(self, H0: torch.Tensor, V: torch.Tensor, n_occ: int, omega: float = 0.05,
                 precision: str = "fp16", tol: float = 1e-6, fixed_bounds: bool = False,
                 accelerate: bool = False):
        if H0.dtype != torch.float64 or V.dtype != torch.float64 or not H0.is_cuda:
            raise TypeError("H0 and V must be float64 CUDA tensors")
        self.H0, self.V, self.n_occ = H0, V, int(n_occ)
        self.omega, self.precision, self.tol = float(omega), precision, float(tol)
        self.n = H0.shape[0]
        self.bounds = None
        if fixed_bounds:
            # Gershgorin interval of H_0 from the library's own bound kernel, widened by |V|_inf.
            _, r0 = sp2.density(H0, self.n_occ, precision=precision, tol=tol)
            vinf = float(V.abs().sum(dim=1).max())
            self.bounds = (r0.eps_min - vinf, r0.eps_max + vinf)
        self.accelerate = bool(accelerate)
        self.gap = None  # (eps_homo, eps_lumo) estimated from the previous step
        self.records: List[StepRecord] = []
        self.D: Optional[torch.Tensor] = None
        self.D1: Optional[torch.Tensor] = None

    def hamiltonian(self, k: int):
        s, c = math.sin(self.omega * k), math.cos(self.omega * k)
        return self.H0 + s * self.V, (self.omega * c) * self.V

    def step(self, k: int, check_gap: bool = False) -> StepRecord:
        Hk, H1k = self.hamiltonian(k)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        use_gap = self.gap if self.accelerate else None
        D, D1, res = sp2.response(Hk, H1k, self.n_occ, tol=self.tol, precision=self.precision, bounds=self.bounds,
                                  gap=use_gap)
        fallback = use_gap is not None and (not res.converged or abs(res.trace_D - self.n_occ) > 0.5)
        if fallback:
            D, D1, res = sp2.response(Hk, H1k, self.n_occ, tol=self.tol, precision=self.precision,
                                      bounds=self.bounds)
        e1.record(stream)
        torch.cuda.synchronize()
        dE = float((D.double() * H1k).sum())
        rec = StepRecord(k, res.layers, res.stop_reason, res.band_energy, dE, res.trace_D - self.n_occ,
                         e0.elapsed_time(e1), use_gap is not None, fallback)
        self.records.append(rec)
        self.D, self.D1 = D, D1
        if res.converged:
            est = gap_mod.estimate_gap(res.trace, res.trace_sq, res.choices, res.alphas, self.n_occ,
                                       res.eps_min, res.eps_max)
            if est is not None:
                rec.gap_est = est[1] - est[0]
                if self.accelerate:
                    self.gap = est
        if check_gap:
            # Independent monitor of the trajectory's gap (the SP2 chain needs one):
            # FP32 eigenvalues from cuSOLVER, far below the gap in error.  Not part of the path.
            lam = torch.linalg.eigvalsh(Hk.float())
            rec.gap_check = float(lam[self.n_occ] - lam[self.n_occ - 1])
        return rec

    def run(self, steps: int, start: int = 0, check_every: int = 0) -> List[StepRecord]:
        for k in range(start, start + steps):
            self.step(k, check_gap=check_every > 0 and (k - start) % check_every == 0)
        return self.records

    def drift(self) -> dict:
        """Energy change along the trajectory against the integral of its derivative."""
        ks = np.array([r.k for r in self.records], dtype=np.float64)
        E = np.array([r.band_energy for r in self.records])
        F = np.array([r.dE_dk for r in self.records])
        integ = np.concatenate([[0.0], np.cumsum(0.5 * (F[1:] + F[:-1]) * np.diff(ks))])
        dev = (E - E[0]) - integ
        return {"max_abs": float(np.max(np.abs(dev))), "final": float(dev[-1]),
                "energy_span": float(E.max() - E.min())}


def trajectory_inputs(n: int, seed_config: int = 4):
    """H_0 (water-like banded, gap >= 0.05, n_occ = N/2) and the sparse symmetric V."""
    ham = inputs.banded_tight_binding(n, inputs.rng_for(1), n // 2)
    V = inputs.sparse_perturbation(n, inputs.rng_for(seed_config))
    return ham, V


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--n", type=int, default=12288)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--precision", default="fp16")
    ap.add_argument("--fixed-bounds", action="store_true")
    ap.add_argument("--accelerate", action="store_true")
    ap.add_argument("--check-gap-every", type=int, default=20,
                    help="eigenvalue check of the HOMO-LUMO gap every K steps (0 = off)")
    a = ap.parse_args(argv)
    t0 = time.time()
    ham, V = trajectory_inputs(a.n)
    gen_s = time.time() - t0
    run = MDSequence(torch.tensor(ham.H, device="cuda"), torch.tensor(V, device="cuda"), ham.n_occ,
                     precision=a.precision, fixed_bounds=a.fixed_bounds, accelerate=a.accelerate)
    recs = run.run(a.steps, check_every=a.check_gap_every)
    ms = [r.ms for r in recs[1:]] or [recs[0].ms]
    layers = [r.layers for r in recs]
    mean_ms = float(np.mean(ms))
    # forward square (2N^3) plus the response product X X1 (2N^3) per layer
    eff = float(np.mean(layers)) * 4.0 * float(a.n) ** 3 / (mean_ms * 1e-3) / 1e12
    out = {"n": a.n, "steps": a.steps, "precision": a.precision, "fixed_bounds": a.fixed_bounds,
           "accelerate": a.accelerate, "fallbacks": sum(1 for r in recs if r.fallback),
           "ms_per_step": mean_ms, "effective_tflops": eff, "layers_min": min(layers), "layers_max": max(layers),
           "not_converged_steps": sum(1 for r in recs if r.stop_reason == sp2.STOP_MAX),
           "max_abs_trace_err": max(abs(r.trace_err) for r in recs), "drift": run.drift(),
           "min_gap_estimate": min((r.gap_est for r in recs if r.gap_est is not None), default=None),
           "min_gap_checked": min((r.gap_check for r in recs if r.gap_check is not None), default=None),
           "gap_checks": sum(1 for r in recs if r.gap_check is not None),
           "steps_without_gap_estimate": sum(1 for r in recs if r.gap_est is None),
           "generation_s": gen_s}
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
