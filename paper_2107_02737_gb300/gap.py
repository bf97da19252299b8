"""Estimates of the HOMO and LUMO eigenvalues from the statistics of a finished chain.

The accelerated chain needs an interval [eps_homo, eps_lumo] that overlaps the gap
(section "GPU and tensor core performance" names the need for such estimates).  A
converged chain already carries them: every layer is a known polynomial map of the
eigenvalue images (X^2 or 2X - X^2 after the expansion a_n), and its FP64 statistics
Tr X_n and ||X_n||_F^2 give, late in the chain,

    u_n = (e_n + Tr X_n - N_occ) / 2  ~  sum over unoccupied images x_i,
    v_n = (e_n - Tr X_n + N_occ) / 2  ~  sum over occupied (1 - x_i),

with e_n = Tr X_n - ||X_n||_F^2.  Once the images have separated, u_n is dominated by
the largest unoccupied image (the LUMO's) and v_n by the HOMO's distance from 1, and
both sums bound those single terms from above.  Mapping u_n and 1 - v_n back through
the inverse layers (the root on the side of the gap) gives an image at least as deep
into the gap as the true one, hence energies inside or at the edge of the gap.  The
latest layer whose sum is still well above the statistics' rounding floor is used.

This is host-side arithmetic on the returned statistics (no device work).
"""
from __future__ import annotations

import math
from typing import Optional, Sequence, Tuple

SQUARE, FLIP = 0, 1


def _inverse(y: float, choice: int, alpha: float) -> float:
    """Preimage of y under one layer, on the branch that points into the gap."""
    if choice == SQUARE:      # y = T^2, T = a x + (1 - a): the non-negative root
        t = math.sqrt(max(y, 0.0))
        return (t - (1.0 - alpha)) / alpha
    t = 1.0 - math.sqrt(max(1.0 - y, 0.0))   # y = 2T - T^2, T = a x: the root T <= 1
    return t / alpha


def estimate_gap(trace: Sequence[float], trace_sq: Sequence[float], choices: Sequence[int],
                 alphas: Optional[Sequence[float]], n_occ: float, eps_min: float, eps_max: float,
                 floor: Optional[float] = None) -> Optional[Tuple[float, float]]:
    """(eps_homo, eps_lumo) estimated from one chain's per-layer statistics, or None.

    ``trace[n]``, ``trace_sq[n]`` are Tr X_n and ||X_n||_F^2 for n = 0..L, ``choices`` and
    ``alphas`` the L layers (alphas None: the plain chain).  ``floor`` is the level
    below which the sums are taken as rounding noise (default: 30 times the final
    idempotency error, at least 1e-9 N_occ).  Returns None when no layer qualifies or
    the two estimates cross.
    """
    L = len(choices)
    if L == 0 or len(trace) < L + 1:
        return None
    a = [1.0] * L if alphas is None else [float(x) for x in alphas]
    e_last = abs(trace[L] - trace_sq[L])
    if floor is None:
        floor = max(30.0 * e_last, 1e-9 * max(n_occ, 1.0))
    span = eps_max - eps_min

    def back(y: float, m: int) -> float:
        for k in range(m - 1, -1, -1):
            y = _inverse(y, choices[k], a[k])
        return y

    x_lumo = x_homo = None
    for m in range(L, 0, -1):
        e = trace[m] - trace_sq[m]
        u = 0.5 * (e + trace[m] - n_occ)
        v = 0.5 * (e - trace[m] + n_occ)
        # Only once the images sit near 0 and 1 (sums below 1/4) and above the floor.
        if x_lumo is None and floor < u < 0.25:
            x_lumo = back(u, m)
        if x_homo is None and floor < v < 0.25:
            x_homo = back(1.0 - v, m)
        if x_lumo is not None and x_homo is not None:
            break
    if x_lumo is None or x_homo is None or not x_lumo < x_homo:
        return None
    return eps_max - x_homo * span, eps_max - x_lumo * span
