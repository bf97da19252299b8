"""The DNN-SP2 chain in float64 on the CPU.

Test infrastructure only (see the package docstring): nothing in the product path
imports this module.

The chain (section "Deep-neural network electronic structure solver", Eq. Deep_NN
and the text around Figure 1):

* Input layer: W_0, B_0 map the spectrum of H linearly onto [0, 1] in reverse
  order, X_0 = (eps_max I - H) / (eps_max - eps_min).  The bounds are Gershgorin
  estimates unless given.
* Every further layer applies W_n = +-I, B_n = (I - W_n) S_{n-1} and the
  activation f(X) = X^2, so that X_{n+1} = X_n^2 or X_{n+1} = 2 X_n - X_n^2.
* The sign of each layer is chosen so that the trace moves toward the
  occupation n_occ, and the layers repeat until the eigenvalues are close to 0
  and 1, with idempotency measured from traces.

The paper leaves the sign rule and the stop rule unspecified.  Readings used
here (and identically by the CUDA path):

* Layer choice: X^2 iff |Tr X^2 - n_occ| <= |2 Tr X - Tr X^2 - n_occ|, else
  2X - X^2, with Tr X^2 taken as ||X||_F^2 of the stored symmetric X; a tie
  picks X^2.
* Stop rule, evaluated on X_n for n = 0, 1, ...: e_n = |Tr X_n - ||X_n||_F^2|.
  Stop with reason TOL when e_n <= tol; with reason STALL when n >= 2,
  e_n <= STALL_MAX and e_n >= e_{n-2} (the rounding floor has been reached);
  with reason MAX when n = max_layers.  TOL and STALL return OK, MAX returns
  NOT_CONVERGED.  The last X computed is returned.
* n_occ = 0 returns D = 0 and n_occ = N returns D = I without layers (the
  chain cannot reach them when a Gershgorin bound is attained by an
  eigenvalue, e.g. for diagonal H).

Layer statistics follow the CUDA path's record: entry n holds Tr X_n,
||X_n||_F^2, Tr X_n - ||X_n||_F^2 and the choice that produced X_n (-1 for the
input layer, 0 for X^2, 1 for 2X - X^2).

Accelerated chain.  Section "GPU and tensor core performance" remarks that up
to half of the layers can be saved when estimates of the highest occupied and
lowest unoccupied eigenvalues are known, and leaves that scheme out.  The
reading used here (and by the CUDA path): with the images x_lumo < x_homo of
an estimated interval [eps_homo, eps_lumo] under the input layer, every layer
first expands X affinely and then applies its branch,

    X^2 branch:     T_n = a_n X_n + (1 - a_n) I,  a_n = 2 / (2 - x_lumo),  X_{n+1} = T_n^2
    2X - X^2 branch: T_n = a_n X_n,               a_n = 2 / (1 + x_homo),  X_{n+1} = 2 T_n - T_n^2

(a layer S_n = W_n X_n + B_n of the same network with scalar weights), and
x_lumo, x_homo follow the same scalar map.  The branch is still taken by the
trace rule.  a_n lies in [1, 2], so every image stays in [0, 1]; a_n = 1 (the
interval [eps_min, eps_max]) is the plain chain.  The occupied images stay
above the unoccupied ones after every layer, so the chain still converges to
theta(mu I - H), whenever the estimated interval overlaps the gap:
eps_lumo > eps_HOMO and eps_homo < eps_LUMO.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

SQUARE = 0          # X_{n+1} = X_n^2
FLIP = 1            # X_{n+1} = 2 X_n - X_n^2
INPUT = -1          # the input layer X_0

STOP_TOL = 1
STOP_STALL = 2
STOP_MAX = 3
STOP_TRIVIAL = 4    # n_occ = 0 or n_occ = N

STALL_MAX = 1e-2
DEFAULT_TOL = 1e-6
DEFAULT_MAX_LAYERS = 100


@dataclasses.dataclass
class LayerStat:
    trace: float
    trace_sq: float
    idem: float
    choice: int


@dataclasses.dataclass
class SP2Result:
    D: np.ndarray
    stats: List[LayerStat]
    stop_reason: int
    converged: bool
    eps_min: float
    eps_max: float
    alphas: List[float] = dataclasses.field(default_factory=list)  # a_n per layer (1 = plain)

    @property
    def layers(self) -> int:
        """Number of square layers applied (X_0 is layer 0)."""
        return len(self.stats) - 1

    @property
    def choices(self) -> List[int]:
        return [s.choice for s in self.stats[1:]]


# -- input layer ----------------------------------------------------------------

def gershgorin_bounds(H: np.ndarray):
    """eps_min = min_i (H_ii - sum_{j!=i} |H_ij|), eps_max = max_i (H_ii + sum_{j!=i} |H_ij|)."""
    H = np.asarray(H, dtype=np.float64)
    d = np.diag(H)
    r = np.abs(H).sum(axis=1) - np.abs(d)
    return float(np.min(d - r)), float(np.max(d + r))


def input_layer(H: np.ndarray, eps_min: float, eps_max: float) -> np.ndarray:
    """X_0 = (eps_max I - H)/(eps_max - eps_min): spectrum onto [0, 1], reversed."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    return (eps_max * np.eye(n) - H) / (eps_max - eps_min)


# -- layer rule and stop rule ----------------------------------------------------

def layer_choice(trace: float, trace_sq: float, n_occ: float) -> int:
    """Trace-correcting sign of the next layer (X^2 on a tie)."""
    if abs(trace_sq - n_occ) <= abs(2.0 * trace - trace_sq - n_occ):
        return SQUARE
    return FLIP


def stop_check(idem: Sequence[float], tol: float, max_layers: int) -> int:
    """Stop reason after the latest entry of ``idem`` (Tr X_n - ||X_n||^2 per layer), 0 = go on."""
    n = len(idem) - 1
    e = [abs(v) for v in idem]
    if e[n] <= tol:
        return STOP_TOL
    if n >= 2 and e[n] <= STALL_MAX and e[n] >= e[n - 2]:
        return STOP_STALL
    if n >= max_layers:
        return STOP_MAX
    return 0


def apply_layer(X: np.ndarray, choice: int, alpha: float = 1.0) -> np.ndarray:
    """X_{n+1} from X_n: T = a X + (1 - a) I then T^2, or T = a X then 2T - T^2."""
    if alpha == 1.0:  # the plain layer: X^2 or 2X - X^2
        S = X @ X
        return S if choice == SQUARE else 2.0 * X - S
    if choice == SQUARE:
        T = alpha * X + (1.0 - alpha) * np.eye(X.shape[0])
        return T @ T
    T = alpha * X
    return 2.0 * T - T @ T


def gap_images(gap, eps_min: float, eps_max: float):
    """(x_lumo, x_homo): images of an estimated interval (eps_homo, eps_lumo) under the
    input layer, clipped to [0, 1]; (0, 1), the plain chain, when there is no estimate."""
    if gap is None:
        return 0.0, 1.0
    eps_homo, eps_lumo = gap
    if not eps_homo < eps_lumo:
        raise ValueError("the estimated interval needs eps_homo < eps_lumo")
    span = eps_max - eps_min
    x_lumo = min(max((eps_max - eps_lumo) / span, 0.0), 1.0)
    x_homo = min(max((eps_max - eps_homo) / span, 0.0), 1.0)
    return x_lumo, x_homo


def expansion(choice: int, x_lumo: float, x_homo: float) -> float:
    """a_n of the accelerated layer: 2/(2 - x_lumo) before X^2, 2/(1 + x_homo) before 2X - X^2."""
    return 2.0 / (2.0 - x_lumo) if choice == SQUARE else 2.0 / (1.0 + x_homo)


def scalar_layer(x, choice: int, alpha: float = 1.0):
    """The same layer on scalars (eigenvalues or the tracked interval ends)."""
    if choice == SQUARE:
        t = alpha * x + (1.0 - alpha)
        return t * t
    t = alpha * x
    return 2.0 * t - t * t


def _stat(X: np.ndarray, choice: int) -> LayerStat:
    t = float(np.trace(X))
    q = float(np.sum(X * X))
    return LayerStat(t, q, t - q, choice)


# -- the matrix chain ------------------------------------------------------------

def sp2(H: np.ndarray, n_occ: int, tol: float = DEFAULT_TOL,
        max_layers: int = DEFAULT_MAX_LAYERS, bounds=None,
        choices: Optional[Sequence[int]] = None, keep_layers: bool = False,
        gap=None, alphas: Optional[Sequence[float]] = None) -> SP2Result:
    """Run the DNN-SP2 chain on H in float64.

    ``choices`` replays a given sign sequence exactly (used to follow a
    sequence taken by another implementation); the stop rule is then only
    evaluated for the report.  With ``keep_layers`` the result carries every X_n in
    ``result.layers_X``.  ``gap = (eps_homo, eps_lumo)`` runs the accelerated
    chain (module docstring); ``alphas`` replays given expansions a_n together with
    ``choices``.
    """
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    eps_min, eps_max = gershgorin_bounds(H) if bounds is None else bounds
    if n_occ == 0 or n_occ == n:
        D = np.zeros((n, n)) if n_occ == 0 else np.eye(n)
        res = SP2Result(D, [_stat(D, INPUT)], STOP_TRIVIAL, True, eps_min, eps_max)
        res.layers_X = [D]
        return res
    X = input_layer(H, eps_min, eps_max)
    x_lumo, x_homo = gap_images(gap, eps_min, eps_max)
    stats = [_stat(X, INPUT)]
    used = []  # a_n of every layer applied
    images = [(x_lumo, x_homo)]
    kept = [X] if keep_layers else None

    def step(c):
        nonlocal X, x_lumo, x_homo
        a = expansion(c, x_lumo, x_homo) if alphas is None else float(alphas[len(stats) - 1])
        X = apply_layer(X, c, a)
        x_lumo, x_homo = scalar_layer(x_lumo, c, a), scalar_layer(x_homo, c, a)
        used.append(a)
        images.append((x_lumo, x_homo))
        stats.append(_stat(X, c))
        if keep_layers:
            kept.append(X)

    if choices is not None:
        # Exact replay of a given sign sequence; the stop rule is only reported.
        for c in choices:
            step(c)
        reason = stop_check([s.idem for s in stats], tol, max_layers)
    else:
        reason = stop_check([stats[0].idem], tol, max_layers)
        while not reason:
            step(layer_choice(stats[-1].trace, stats[-1].trace_sq, n_occ))
            reason = stop_check([s.idem for s in stats], tol, max_layers)
    res = SP2Result(X, stats, reason, reason in (STOP_TOL, STOP_STALL), eps_min, eps_max, used)
    res.layers_X = kept
    res.gap_images = images  # (x_lumo, x_homo) after each layer, entry 0 for X_0
    return res


# -- the same chain on scalar eigenvalues -------------------------------------------

def scalar_sp2(eigvals: np.ndarray, n_occ: int, eps_min: float, eps_max: float,
               tol: float = DEFAULT_TOL, max_layers: int = DEFAULT_MAX_LAYERS,
               choices: Optional[Sequence[int]] = None, gap=None):
    """The chain acting on the eigenvalues of H: x_0 = (eps_max - eps)/(eps_max - eps_min).

    Since every layer is a polynomial of X, X_n = C diag(p_n(eps)) C^T and
    Tr X_n = sum p_n, ||X_n||_F^2 = sum p_n^2.  Returns (p_L, stats, stop_reason,
    dp_L/dx) where the derivative is propagated by the scalar chain rule.
    ``gap`` as for ``sp2``.
    """
    x = (eps_max - np.asarray(eigvals, np.float64)) / (eps_max - eps_min)
    dx = np.ones_like(x)
    x_lumo, x_homo = gap_images(gap, eps_min, eps_max)
    stats = [LayerStat(float(x.sum()), float((x * x).sum()), float(x.sum() - (x * x).sum()), INPUT)]
    def step(c):
        nonlocal x, dx, x_lumo, x_homo
        a = expansion(c, x_lumo, x_homo)
        if c == SQUARE:
            dx = 2.0 * a * (a * x + 1.0 - a) * dx
        else:
            dx = (2.0 * a - 2.0 * a * a * x) * dx
        x = scalar_layer(x, c, a)
        x_lumo, x_homo = scalar_layer(x_lumo, c, a), scalar_layer(x_homo, c, a)
        t, q = float(x.sum()), float((x * x).sum())
        stats.append(LayerStat(t, q, t - q, c))

    if choices is not None:
        for c in choices:
            step(c)
        reason = stop_check([s.idem for s in stats], tol, max_layers)
    else:
        reason = stop_check([stats[0].idem], tol, max_layers)
        while not reason:
            step(layer_choice(stats[-1].trace, stats[-1].trace_sq, n_occ))
            reason = stop_check([s.idem for s in stats], tol, max_layers)
    return x, stats, reason, dx


# -- response, adjoint and derivative of the chain ----------------------------------

def chain_response(H: np.ndarray, H1: np.ndarray, choices: Sequence[int],
                   eps_min: float, eps_max: float, alphas=None) -> np.ndarray:
    """Forward-mode derivative of the chain with the layer signs (and a_n) held fixed.

    X1_0 = -H1/(eps_max - eps_min); per layer T = a X + (1 - a) I or a X and
    T1 = a X1_n; with C = T T1, X1_{n+1} = C + C^T (for X^2) or 2 T1 - (C + C^T)
    (for 2X - X^2), alongside X_{n+1}.  Returns X1_L.
    """
    X = input_layer(H, eps_min, eps_max)
    X1 = -np.asarray(H1, np.float64) / (eps_max - eps_min)
    n = X.shape[0]
    for k, c in enumerate(choices):
        a = 1.0 if alphas is None else alphas[k]
        T = a * X + (1.0 - a) * np.eye(n) if c == SQUARE else a * X
        T1 = a * X1
        P = T @ T1
        P = P + P.T
        S = T @ T
        if c == SQUARE:
            X, X1 = S, P
        else:
            X, X1 = 2.0 * T - S, 2.0 * T1 - P
    return X1


def chain_adjoint(H: np.ndarray, G: np.ndarray, choices: Sequence[int],
                  eps_min: float, eps_max: float, alphas=None) -> np.ndarray:
    """Reverse-mode gradient of Tr[X_L G] with respect to symmetric H.

    G_L = sym(G); for the layer that made X_{n+1} from X_n through T_n (T_n = X_n
    in the plain chain), G_n = a_n (G_{n+1} T_n + T_n G_{n+1}) (X^2) or
    a_n (2 G_{n+1} - (G_{n+1} T_n + T_n G_{n+1})) (2X - X^2); finally
    dTr[X_L G]/dH = -G_0/(eps_max - eps_min).
    """
    a_of = (lambda k: 1.0) if alphas is None else (lambda k: alphas[k])
    X = input_layer(H, eps_min, eps_max)
    n = X.shape[0]
    xs = [X]
    for k, c in enumerate(choices[:-1] if len(choices) else []):
        X = apply_layer(X, c, a_of(k))
        xs.append(X)
    Gb = 0.5 * (np.asarray(G, np.float64) + np.asarray(G, np.float64).T)
    for k in range(len(choices) - 1, -1, -1):
        a = a_of(k)
        T = a * xs[k] + (1.0 - a) * np.eye(n) if choices[k] == SQUARE else a * xs[k]
        P = Gb @ T
        P = P + P.T
        Gb = a * P if choices[k] == SQUARE else a * (2.0 * Gb - P)
    return -Gb / (eps_max - eps_min)


def chain_derivative_eigenbasis(H: np.ndarray, H1: np.ndarray, choices: Sequence[int],
                                eps_min: float, eps_max: float, gap=None) -> np.ndarray:
    """Exact Frechet derivative of the fixed-sign chain via divided differences.

    With H = C diag(eps) C^T and the chain polynomial p acting on
    x = (eps_max - eps)/(eps_max - eps_min), the derivative in direction H1 is
    C (C^T H1 C  o  Phi) C^T, Phi_ij = (p(x_i) - p(x_j))/(eps_i - eps_j) and
    Phi_ii = -p'(x_i)/(eps_max - eps_min).
    """
    lam, C = np.linalg.eigh(np.asarray(H, np.float64))
    p, _, _, dp = scalar_sp2(lam, 0, eps_min, eps_max, choices=list(choices), gap=gap)
    de = lam[:, None] - lam[None, :]
    dpv = p[:, None] - p[None, :]
    close = np.abs(de) <= 1e-12 * max(1.0, np.max(np.abs(lam)))
    phi = np.where(close, 0.0, dpv / np.where(close, 1.0, de))
    diag_like = -0.5 * (dp[:, None] + dp[None, :]) / (eps_max - eps_min)
    phi = np.where(close, diag_like, phi)
    h1 = C.T @ (0.5 * (H1 + H1.T)) @ C
    return C @ (h1 * phi) @ C.T


def refine(X: np.ndarray, n_occ: float, layers: int = 2):
    """Refinement: `layers` further layers of the same network in float64.

    The paper adds a few final layers in which X is held in double precision so
    that the eigenvalues are purified closer to 0 and 1 (section "Deep-neural
    network electronic structure solver", the refinement step).  Each layer
    takes its sign by the same trace-correcting rule.  Returns (X, stats).
    """
    X = np.asarray(X, np.float64)
    stats = [_stat(X, INPUT)]
    for _ in range(layers):
        c = layer_choice(stats[-1].trace, stats[-1].trace_sq, n_occ)
        X = apply_layer(X, c)
        stats.append(_stat(X, c))
    return X, stats


def band_energy_of(D: np.ndarray, H: np.ndarray) -> float:
    return float(np.sum(np.asarray(D, np.float64) * np.asarray(H, np.float64)))
