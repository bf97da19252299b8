"""The arithmetic of the device's Gershgorin bounds, replayed on the CPU.

The bounds kernels unpack each FP64 |H_ij| into two floats (|hi| + 2^-24 |lo24|, the
integer part made a float through the exponent-field identity), sum a row's entries of
each 64-column block as four compensated FP32 chains of sixteen combined pairwise (a
diagonal block: its row and its column), convert the partial to FP64 once, add a row's
partials in FP64 (eight strided groups, then the groups in order) and widen the radius
by 2^-36 relative plus 2^-50 |d| + N 2^-120.  Here the same steps in numpy float32 /
float64 arithmetic (round to nearest, as the device's __fadd_rn) are checked against
exactly rounded sums (math.fsum): every disc must contain the exact one, and exceed it
by little more than the widening.  No GPU is involved.
"""
import math

import numpy as np

F = np.float32
AT = 64


def split_abs(v):
    """|hi|, |lo24| of the device's FP64 unpacking, for finite |v| in FP32 range."""
    b = np.abs(v).astype(np.float64).view(np.uint64)
    h32 = (b >> np.uint64(32)).astype(np.uint32)
    l32 = (b & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    e = ((h32 >> 20) & 0x7FF).astype(np.int64)
    e32 = e - 1023 + 127
    ok = (e != 0) & (e32 > 0) & (e32 < 255)
    mhi = ((h32 & 0xFFFFF) << 3) | (l32 >> 29)
    hi = ((np.clip(e32, 0, 255).astype(np.uint32) << 23) | mhi).view(np.float32)
    rem = (l32 & 0x1FFFFFFF) >> 5
    m = (np.uint32(0x4B000000) | (rem & 0x7FFFFF)).view(np.float32) - F(2.0 ** 23)
    q = m + np.where((rem >> 23) != 0, F(2.0 ** 23), F(0))
    scale = (np.where(e32 > 28, e32 - 23, 1).astype(np.uint32) << 23).view(np.float32)
    lo = np.where(e32 > 28, q * scale, F(0)).astype(np.float32)
    return np.where(ok, hi, F(0)).astype(np.float32), np.where(ok, lo, F(0)).astype(np.float32)


def ff_add(s, c, v):
    t = (s + v).astype(F)
    bp = (t - s).astype(F)
    err = ((s - (t - bp)) + (v - bp)).astype(F)
    return t, (c + err).astype(F)


def ff_add_ff(a, b):
    s, c = ff_add(a[0], a[1], b[0])
    return s, (c + b[1]).astype(F)


def ff_sum64(x):
    """x: (rows, 64) float32 -> compensated pair, four chains of sixteen combined pairwise."""
    chains = []
    for k in range(4):
        s = np.zeros(x.shape[0], F)
        c = np.zeros(x.shape[0], F)
        for j in range(16 * k, 16 * k + 16):
            s, c = ff_add(s, c, x[:, j])
        chains.append((s, c))
    a = ff_add_ff(chains[0], chains[1])
    b = ff_add_ff(chains[2], chains[3])
    return ff_add_ff(a, b)


def f_sum64(x):
    a = np.zeros(x.shape[0], F)
    for j in range(x.shape[1]):
        a = (a + x[:, j]).astype(F)
    return a


def device_bounds(H):
    n = H.shape[0]
    nt = (n + AT - 1) // AT
    Np = nt * AT
    Hp = np.zeros((Np, Np))
    Hp[:n, :n] = H
    hi, lo = split_abs(Hp)
    P = np.zeros((nt, Np))
    for ti in range(nt):
        for tj in range(ti + 1):
            sh = hi[ti * AT:(ti + 1) * AT, tj * AT:(tj + 1) * AT].copy()
            sl = lo[ti * AT:(ti + 1) * AT, tj * AT:(tj + 1) * AT].copy()
            if ti == tj:   # strictly below the diagonal
                keep = np.tril(np.ones((AT, AT), bool), -1)
                sh[~keep] = 0
                sl[~keep] = 0
                a = ff_add_ff(ff_sum64(sh), ff_sum64(sh.T.copy()))
                l = (f_sum64(sl) + f_sum64(sl.T.copy())).astype(F)
                P[tj, ti * AT:(ti + 1) * AT] = (a[0].astype(np.float64) + a[1]) + l.astype(np.float64) * 2.0 ** -24
            else:
                a = ff_sum64(sh)
                l = f_sum64(sl)
                P[tj, ti * AT:(ti + 1) * AT] = (a[0].astype(np.float64) + a[1]) + l.astype(np.float64) * 2.0 ** -24
                a = ff_sum64(sh.T.copy())
                l = f_sum64(sl.T.copy())
                P[ti, tj * AT:(tj + 1) * AT] = (a[0].astype(np.float64) + a[1]) + l.astype(np.float64) * 2.0 ** -24
    groups = np.zeros((8, Np))
    for w in range(8):
        for b in range(w, nt, 8):
            groups[w] += P[b]
    rs = np.zeros(Np)
    for w in range(8):
        rs += groups[w]
    rs = rs[:n]
    d = np.diag(H)
    rs = rs * (1.0 + 2.0 ** -36) + np.abs(d) * 2.0 ** -50 + n * 2.0 ** -120
    return d - rs, d + rs


def exact_radius(H):
    n = H.shape[0]
    return np.array([math.fsum(abs(H[i, j]) for j in range(n) if j != i) for i in range(n)])


def _check(H):
    lo, hi = device_bounds(H)
    r = exact_radius(H)
    d = np.diag(H)
    # contains every exact disc (the reference ends d -/+ r are themselves rounded, by at
    # most 2^-53 of |d| + r)
    slack = (np.abs(d) + r) * 2.0 ** -52
    assert np.all(lo - (d - r) <= slack) and np.all((d + r) - hi <= slack)
    # ... and exceeds it by about the widening: no more than 2^-35 of the radius (plus the terms)
    over = np.maximum((d - r) - lo, hi - (d + r))
    assert np.all(over <= r * 2.0 ** -35 + np.abs(d) * 2.0 ** -49 + H.shape[0] * 2.0 ** -119 + slack)
    return over / np.maximum(r, 1e-300)


def test_bounds_contain_exact_discs_random_magnitudes():
    rng = np.random.default_rng(11)
    n = 200
    A = rng.standard_normal((n, n)) * 10.0 ** rng.uniform(-9, 3, (n, n))
    H = (A + A.T) / 2
    rel = _check(H)
    assert rel.max() < 2.0 ** -35


def test_bounds_contain_exact_discs_equal_entries_and_ragged_size():
    # equal entries maximise the compensated sums' accumulated error terms
    n = 131
    H = np.full((n, n), 1.0 / 3.0)
    H[np.diag_indices(n)] = 2.0
    _check(H)
    rng = np.random.default_rng(12)
    A = rng.uniform(0.5, 1.0, (n, n)) * (1.0 + 2.0 ** -30)
    _check((A + A.T) / 2)


def test_exponent_field_integer_to_float_is_exact():
    rem = np.arange(0, 1 << 24, 4099, dtype=np.uint32)
    m = (np.uint32(0x4B000000) | (rem & 0x7FFFFF)).view(np.float32) - F(2.0 ** 23)
    q = m + np.where((rem >> 23) != 0, F(2.0 ** 23), F(0))
    assert np.array_equal(q.astype(np.int64), rem.astype(np.int64))
