"""Python binding of libsp2 (the C ABI in include/sp2.h), argument marshalling only.

Every step of the SP2 chain runs in the library's CUDA kernels; this module only
passes tensor pointers, the current CUDA stream and option structs through
ctypes, and turns the returned statistics into Python objects.  There is no
fallback: if ``libsp2.so`` has not been built, importing the functions below
raises.

Tensors may live on the GPU or on the host (the library stages host matrices
through device memory).  H, H1 and G are float64; D, D1 and dH come back as
float32, on the device of H.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import List, Optional, Sequence

import numpy as np
import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsp2.so")

OK, ERR_ARG, ERR_NONFINITE, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_CUDA, ERR_NOMEM, ERR_UNSUPPORTED = range(8)
PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2}
STOP_NONE, STOP_TOL, STOP_STALL, STOP_MAX, STOP_TRIVIAL = range(5)
CHOICE_INPUT, CHOICE_SQUARE, CHOICE_FLIP = -1, 0, 1
MAX_LAYERS_LIMIT = 200


class LayerStat(ctypes.Structure):
    _fields_ = [("trace", ctypes.c_double), ("trace_sq", ctypes.c_double), ("idem", ctypes.c_double),
                ("choice", ctypes.c_int), ("reserved", ctypes.c_int), ("alpha", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("layers", ctypes.c_int), ("stop_reason", ctypes.c_int), ("eps_min", ctypes.c_double),
                ("eps_max", ctypes.c_double), ("band_energy", ctypes.c_double), ("trace_D", ctypes.c_double),
                ("layer", ctypes.POINTER(LayerStat)), ("layer_cap", ctypes.c_int), ("cta_group", ctypes.c_int),
                ("phase_ms", ctypes.c_float * 4)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_layers", ctypes.c_int), ("timeout_ms", ctypes.c_double),
                ("user_bounds", ctypes.c_int), ("test_hook", ctypes.c_int), ("eps_min", ctypes.c_double),
                ("eps_max", ctypes.c_double), ("profile", ctypes.c_int), ("cta_group", ctypes.c_int),
                ("accelerate", ctypes.c_int), ("eps_homo", ctypes.c_double), ("eps_lumo", ctypes.c_double),
                ("checkpoint_stride", ctypes.c_int), ("exact_slices", ctypes.c_int)]


EXPORTS = ["sp2_default_opts", "sp2_status_string", "sp2_device_info", "sp2_density", "sp2_density_workspace_bytes",
           "sp2_response", "sp2_response_workspace_bytes", "sp2_adjoint", "sp2_adjoint_workspace_bytes",
           "sp2_density_batched", "sp2_density_batched_workspace_bytes", "sp2_apply_layers",
           "sp2_density_noalloc", "sp2_density_refined", "sp2_density_nonorth", "sp2_batch_plan_create",
           "sp2_batch_plan_launch", "sp2_batch_plan_stats", "sp2_batch_plan_cta_group", "sp2_batch_plan_destroy",
           "sp2_congruence"]
NOALLOC_MAX_N = 512

_lib = None


def library_path() -> str:
    return _LIB_PATH


def load() -> ctypes.CDLL:
    """Load libsp2.so (built by ``python -m paper_2107_02737_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with `python -m paper_2107_02737_gb300.build` "
                           "(the SP2 path has no CPU fallback)")
    lib = ctypes.CDLL(_LIB_PATH)
    c_d, c_i, c_sz, c_p = ctypes.c_double, ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p
    P = ctypes.POINTER
    lib.sp2_default_opts.argtypes = [P(Opts)]
    lib.sp2_default_opts.restype = None
    lib.sp2_status_string.argtypes = [c_i]
    lib.sp2_status_string.restype = ctypes.c_char_p
    lib.sp2_device_info.argtypes = [P(c_i), P(c_i), P(c_i)]
    lib.sp2_device_info.restype = c_i
    lib.sp2_density.argtypes = [c_p, c_i, c_d, c_d, c_p, P(Stats), P(Opts), c_p, c_sz, c_p]
    lib.sp2_density.restype = c_i
    lib.sp2_density_workspace_bytes.argtypes = [c_i, P(Opts)]
    lib.sp2_density_workspace_bytes.restype = c_sz
    lib.sp2_response.argtypes = [c_p, c_p, c_i, c_d, c_d, P(Stats), c_p, c_p, P(Stats), P(Opts), c_p, c_sz, c_p]
    lib.sp2_response.restype = c_i
    lib.sp2_response_workspace_bytes.argtypes = [c_i, P(Opts)]
    lib.sp2_response_workspace_bytes.restype = c_sz
    lib.sp2_adjoint.argtypes = [c_p, c_p, c_i, c_d, c_d, P(Stats), c_p, c_p, P(Stats), P(Opts), c_p, c_sz, c_p]
    lib.sp2_adjoint.restype = c_i
    lib.sp2_adjoint_workspace_bytes.argtypes = [c_i, c_i, P(Opts)]
    lib.sp2_adjoint_workspace_bytes.restype = c_sz
    lib.sp2_density_batched.argtypes = [c_i, P(c_p), P(c_i), P(c_d), c_d, P(c_p), P(Stats), P(Opts), c_p, c_sz, c_p]
    lib.sp2_density_batched.restype = c_i
    lib.sp2_density_batched_workspace_bytes.argtypes = [c_i, P(c_i), P(Opts)]
    lib.sp2_density_batched_workspace_bytes.restype = c_sz
    lib.sp2_apply_layers.argtypes = [c_p, c_i, P(c_i), c_i, c_p, P(Stats), P(Opts), c_p]
    lib.sp2_apply_layers.restype = c_i
    lib.sp2_density_noalloc.argtypes = [c_p, c_i, c_d, c_d, c_p, P(Stats), P(Opts), c_p]
    lib.sp2_density_noalloc.restype = c_i
    lib.sp2_density_refined.argtypes = [c_p, c_i, c_d, c_d, c_i, c_p, P(Stats), P(Opts), c_p]
    lib.sp2_density_refined.restype = c_i
    lib.sp2_density_nonorth.argtypes = [c_p, c_p, c_i, c_d, c_d, c_i, c_p, P(Stats), P(Opts), c_p]
    lib.sp2_density_nonorth.restype = c_i
    lib.sp2_batch_plan_create.argtypes = [c_i, P(c_p), P(c_i), P(c_d), c_d, P(c_p), P(Opts), c_i, c_p, P(c_p)]
    lib.sp2_batch_plan_create.restype = c_i
    lib.sp2_batch_plan_launch.argtypes = [c_p, c_p]
    lib.sp2_batch_plan_launch.restype = c_i
    lib.sp2_batch_plan_stats.argtypes = [c_p, P(Stats), c_p]
    lib.sp2_batch_plan_stats.restype = c_i
    lib.sp2_batch_plan_cta_group.argtypes = [c_p]
    lib.sp2_batch_plan_cta_group.restype = c_i
    lib.sp2_batch_plan_destroy.argtypes = [c_p]
    lib.sp2_batch_plan_destroy.restype = None
    lib.sp2_congruence.argtypes = [c_p, c_p, c_i, c_i, c_p, P(Opts), c_p]
    lib.sp2_congruence.restype = c_i
    _lib = lib
    return lib


class SP2Error(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {load().sp2_status_string(status).decode()} (status {status})")


@dataclasses.dataclass
class Result:
    status: int
    layers: int
    stop_reason: int
    eps_min: float
    eps_max: float
    band_energy: float
    trace_D: float
    trace: List[float]
    trace_sq: List[float]
    idem: List[float]
    choices: List[int]          # choice that produced X_n, n = 1..layers
    raw: Stats = dataclasses.field(repr=False, default=None)
    phase_ms: List[float] = dataclasses.field(default_factory=list)
    cta_group: int = 0
    alphas: List[float] = dataclasses.field(default_factory=list)  # expansion a_n, n = 1..layers

    @property
    def converged(self) -> bool:
        return self.status == OK


def make_opts(precision: str = "fp16", max_layers: int = 100, timeout_ms: float = 2000.0,
              bounds: Optional[Sequence[float]] = None, profile: bool = False, cta_group: int = 0,
              gap: Optional[Sequence[float]] = None, checkpoint_stride: int = 0) -> Opts:
    """Options record; ``gap = (eps_homo, eps_lumo)`` selects the accelerated chain;
    ``checkpoint_stride`` (adjoint only): 0 keeps every layer, s >= 2 every s-th, -1 picks s."""
    o = Opts()
    load().sp2_default_opts(ctypes.byref(o))
    if precision not in PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
    o.precision = PRECISIONS[precision]
    o.max_layers = int(max_layers)
    o.timeout_ms = float(timeout_ms)
    if bounds is not None:
        o.user_bounds = 1
        o.eps_min, o.eps_max = float(bounds[0]), float(bounds[1])
    o.profile = 1 if profile else 0
    o.cta_group = int(cta_group)
    if gap is not None:
        o.accelerate = 1
        o.eps_homo, o.eps_lumo = float(gap[0]), float(gap[1])
    o.checkpoint_stride = int(checkpoint_stride)
    return o


def _new_stats(cap: int = MAX_LAYERS_LIMIT + 1):
    arr = (LayerStat * cap)()
    st = Stats()
    st.layer = ctypes.cast(arr, ctypes.POINTER(LayerStat))
    st.layer_cap = cap
    st._keep = arr  # keep the array alive with the struct
    return st


# The layout of LayerStat as a numpy record, to read a call's layer records in one copy.
_LAYER_DTYPE = np.dtype([("trace", "<f8"), ("trace_sq", "<f8"), ("idem", "<f8"), ("choice", "<i4"),
                         ("reserved", "<i4"), ("alpha", "<f8")])
assert _LAYER_DTYPE.itemsize == ctypes.sizeof(LayerStat)


def _result(status: int, st: Stats) -> Result:
    n = max(0, min(st.layers + 1, st.layer_cap))
    lay = np.frombuffer(ctypes.string_at(st.layer, n * _LAYER_DTYPE.itemsize), dtype=_LAYER_DTYPE)
    return Result(status, st.layers, st.stop_reason, st.eps_min, st.eps_max, st.band_energy, st.trace_D,
                  lay["trace"].tolist(), lay["trace_sq"].tolist(), lay["idem"].tolist(), lay["choice"][1:].tolist(),
                  st, list(st.phase_ms), st.cta_group, lay["alpha"][1:].tolist())


def _check(status: int, where: str):
    if status not in (OK, ERR_NOT_CONVERGED):
        raise SP2Error(status, where)


def _stream_handle(t: torch.Tensor, stream) -> int:
    if stream is not None:
        return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
    dev = t.device if t.is_cuda else torch.device("cuda", torch.cuda.current_device())
    return int(torch.cuda.current_stream(dev).cuda_stream)


def _square(t: torch.Tensor, name: str) -> int:
    if t.dim() != 2 or t.shape[0] != t.shape[1]:
        raise ValueError(f"{name} must be a square matrix")
    return int(t.shape[0])


def _f64(t: torch.Tensor, name: str) -> torch.Tensor:
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    return t.contiguous()


def _empty_like_host(H: torch.Tensor, n: int) -> torch.Tensor:
    """An N x N FP32 result on H's device; page-locked when H is, so that the
    library writes it in place across the host link instead of copying it."""
    pinned = H.device.type == "cpu" and H.is_pinned()
    return torch.empty((n, n), dtype=torch.float32, device=H.device, pin_memory=pinned)


def _ws_args(workspace: Optional[torch.Tensor]):
    if workspace is None:
        return None, 0
    return ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()


def workspace_bytes(n: int, kind: str = "density", precision: str = "fp16", layers: int = 0,
                    checkpoint_stride: int = 0) -> int:
    o = make_opts(precision, checkpoint_stride=checkpoint_stride)
    lib = load()
    if kind == "density":
        return int(lib.sp2_density_workspace_bytes(n, ctypes.byref(o)))
    if kind == "response":
        return int(lib.sp2_response_workspace_bytes(n, ctypes.byref(o)))
    if kind == "adjoint":
        return int(lib.sp2_adjoint_workspace_bytes(n, layers, ctypes.byref(o)))
    raise ValueError(kind)


def density(H: torch.Tensor, n_occ: int, tol: float = 1e-6, precision: str = "fp16", max_layers: int = 100,
            timeout_ms: float = 2000.0, bounds=None, out: Optional[torch.Tensor] = None,
            workspace: Optional[torch.Tensor] = None, stream=None, profile: bool = False, cta_group: int = 0,
            gap: Optional[Sequence[float]] = None):
    """D = theta(mu I - H) by the DNN-SP2 chain; returns (D, Result).

    ``cta_group`` selects the tensor-core tile shape (0 = library's choice, 1 or 2).
    ``gap = (eps_homo, eps_lumo)``: accelerated chain from an estimated interval that
    overlaps the gap between the highest occupied and lowest unoccupied eigenvalue.
    """
    H = _f64(H, "H")
    n = _square(H, "H")
    D = out if out is not None else _empty_like_host(H, n)
    st = _new_stats()
    o = make_opts(precision, max_layers, timeout_ms, bounds, profile, cta_group, gap)
    ws, wsb = _ws_args(workspace)
    s = load().sp2_density(ctypes.c_void_p(H.data_ptr()), n, float(n_occ), float(tol), ctypes.c_void_p(D.data_ptr()),
                           ctypes.byref(st), ctypes.byref(o), ws, wsb, ctypes.c_void_p(_stream_handle(H, stream)))
    _check(s, "sp2_density")
    return D, _result(s, st)


def response(H: torch.Tensor, H1: torch.Tensor, n_occ: int, tol: float = 1e-6, precision: str = "fp16",
             max_layers: int = 100, timeout_ms: float = 2000.0, fwd: Optional[Result] = None,
             workspace: Optional[torch.Tensor] = None, stream=None, bounds=None, cta_group: int = 0,
             gap: Optional[Sequence[float]] = None):
    """First-order response of the chain; returns (D, D1, Result).  ``gap`` as for ``density``
    (with ``fwd`` the forward run's layer signs and expansions are replayed instead)."""
    H, H1 = _f64(H, "H"), _f64(H1, "H1")
    n = _square(H, "H")
    D = _empty_like_host(H, n)
    D1 = _empty_like_host(H, n)
    st = _new_stats()
    o = make_opts(precision, max_layers, timeout_ms, bounds, cta_group=cta_group, gap=gap)
    ws, wsb = _ws_args(workspace)
    fp = ctypes.byref(fwd.raw) if fwd is not None else None
    s = load().sp2_response(ctypes.c_void_p(H.data_ptr()), ctypes.c_void_p(H1.data_ptr()), n, float(n_occ),
                            float(tol), fp, ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(D1.data_ptr()),
                            ctypes.byref(st), ctypes.byref(o), ws, wsb, ctypes.c_void_p(_stream_handle(H, stream)))
    _check(s, "sp2_response")
    return D, D1, _result(s, st)


def adjoint(H: torch.Tensor, G: torch.Tensor, n_occ: int, tol: float = 1e-6, precision: str = "fp16",
            max_layers: int = 100, timeout_ms: float = 2000.0, fwd: Optional[Result] = None,
            workspace: Optional[torch.Tensor] = None, stream=None, gap: Optional[Sequence[float]] = None,
            checkpoint_stride: int = 0):
    """Gradient dTr[D G]/dH of the chain by reverse accumulation; returns (D, dH, Result).
    ``gap`` as for ``density`` (with ``fwd`` its signs and expansions are replayed).
    ``checkpoint_stride`` s >= 2 keeps every s-th layer and recomputes the rest in the
    reverse sweep (same result bit for bit, less memory); -1 picks s."""
    H, G = _f64(H, "H"), _f64(G, "G")
    n = _square(H, "H")
    D = _empty_like_host(H, n)
    dH = _empty_like_host(H, n)
    st = _new_stats()
    o = make_opts(precision, max_layers, timeout_ms, gap=gap, checkpoint_stride=checkpoint_stride)
    ws, wsb = _ws_args(workspace)
    fp = ctypes.byref(fwd.raw) if fwd is not None else None
    s = load().sp2_adjoint(ctypes.c_void_p(H.data_ptr()), ctypes.c_void_p(G.data_ptr()), n, float(n_occ),
                           float(tol), fp, ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(dH.data_ptr()),
                           ctypes.byref(st), ctypes.byref(o), ws, wsb, ctypes.c_void_p(_stream_handle(H, stream)))
    _check(s, "sp2_adjoint")
    return D, dH, _result(s, st)


def density_batched(Hs: Sequence[torch.Tensor], n_occs: Sequence[int], tol: float = 1e-6,
                    precision: str = "bf16", max_layers: int = 100, timeout_ms: float = 2000.0,
                    outs: Optional[Sequence[torch.Tensor]] = None, workspace: Optional[torch.Tensor] = None,
                    stream=None, cta_group: int = 0):
    """Independent chains in one grouped launch; returns (list of D, list of Result, worst status)."""
    B = len(Hs)
    Hs = [_f64(h, f"H[{i}]") for i, h in enumerate(Hs)]
    ns = [_square(h, f"H[{i}]") for i, h in enumerate(Hs)]
    Ds = list(outs) if outs is not None else [_empty_like_host(h, n) for n, h in zip(ns, Hs)]
    sts = (Stats * B)()
    keep = []
    for b in range(B):
        arr = (LayerStat * (MAX_LAYERS_LIMIT + 1))()
        keep.append(arr)
        sts[b].layer = ctypes.cast(arr, ctypes.POINTER(LayerStat))
        sts[b].layer_cap = MAX_LAYERS_LIMIT + 1
    hp = (ctypes.c_void_p * B)(*[h.data_ptr() for h in Hs])
    dp = (ctypes.c_void_p * B)(*[d.data_ptr() for d in Ds])
    nn = (ctypes.c_int * B)(*ns)
    occ = (ctypes.c_double * B)(*[float(x) for x in n_occs])
    o = make_opts(precision, max_layers, timeout_ms, cta_group=cta_group)
    ws, wsb = _ws_args(workspace)
    s = load().sp2_density_batched(B, hp, nn, occ, float(tol), dp, sts, ctypes.byref(o), ws, wsb,
                                   ctypes.c_void_p(_stream_handle(Hs[0], stream)))
    _check(s, "sp2_density_batched")
    res = [_result(OK, sts[b]) for b in range(B)]
    for r in res:
        r.status = ERR_NOT_CONVERGED if r.stop_reason == STOP_MAX else OK
        r._keep = keep  # the per-layer arrays behind r.raw
    return Ds, res, s


class BatchPlan:
    """A batched solve set up once (``sp2_batch_plan_create``) and launched many times.

    ``Hs`` and ``outs`` (float32, default: allocated here) are device tensors that the
    plan reads and writes on every launch; write new Hamiltonians into ``Hs`` in place
    between launches.  ``launch`` only enqueues device work, so it can be captured in
    a CUDA graph (``capture``).  ``autotune`` picks the tensor-core tile shape by
    timing both on these inputs (cached per sizes for the process).
    """

    def __init__(self, Hs: Sequence[torch.Tensor], n_occs: Sequence[int], tol: float = 1e-6,
                 precision: str = "bf16", max_layers: int = 100, timeout_ms: float = 2000.0,
                 outs: Optional[Sequence[torch.Tensor]] = None, autotune: bool = True, cta_group: int = 0,
                 stream=None):
        self.B = len(Hs)
        for i, h in enumerate(Hs):
            if h.dtype != torch.float64 or not h.is_cuda or not h.is_contiguous():
                raise TypeError(f"H[{i}] must be a contiguous float64 CUDA tensor")
        self.Hs = list(Hs)
        ns = [_square(h, f"H[{i}]") for i, h in enumerate(Hs)]
        self.Ds = list(outs) if outs is not None else [torch.empty((n, n), dtype=torch.float32, device=h.device)
                                                        for n, h in zip(ns, Hs)]
        self.n_occs = [int(x) for x in n_occs]
        hp = (ctypes.c_void_p * self.B)(*[h.data_ptr() for h in self.Hs])
        dp = (ctypes.c_void_p * self.B)(*[d.data_ptr() for d in self.Ds])
        nn = (ctypes.c_int * self.B)(*ns)
        occ = (ctypes.c_double * self.B)(*[float(x) for x in n_occs])
        o = make_opts(precision, max_layers, timeout_ms, cta_group=cta_group)
        handle = ctypes.c_void_p()
        self._lib = load()
        s = self._lib.sp2_batch_plan_create(self.B, hp, nn, occ, float(tol), dp, ctypes.byref(o), 1 if autotune else 0,
                                            ctypes.c_void_p(_stream_handle(self.Hs[0], stream)),
                                            ctypes.byref(handle))
        _check(s, "sp2_batch_plan_create")
        self._h = handle

    @property
    def cta_group(self) -> int:
        return int(self._lib.sp2_batch_plan_cta_group(self._h))

    def launch(self, stream=None):
        s = self._lib.sp2_batch_plan_launch(self._h, ctypes.c_void_p(_stream_handle(self.Hs[0], stream)))
        _check(s, "sp2_batch_plan_launch")

    def stats(self, stream=None):
        """Wait for the stream; per-instance Results of the last launch and the worst status."""
        sts = (Stats * self.B)()
        keep = []
        for b in range(self.B):
            arr = (LayerStat * (MAX_LAYERS_LIMIT + 1))()
            keep.append(arr)
            sts[b].layer = ctypes.cast(arr, ctypes.POINTER(LayerStat))
            sts[b].layer_cap = MAX_LAYERS_LIMIT + 1
        s = self._lib.sp2_batch_plan_stats(self._h, sts, ctypes.c_void_p(_stream_handle(self.Hs[0], stream)))
        _check(s, "sp2_batch_plan_stats")
        res = [_result(OK, sts[b]) for b in range(self.B)]
        for r in res:
            r.status = ERR_NOT_CONVERGED if r.stop_reason == STOP_MAX else OK
            r._keep = keep
        return res, s

    def capture(self):
        """A torch CUDA graph holding one launch; ``graph.replay()`` re-runs the batch."""
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(device=self.Hs[0].device)
        side.wait_stream(torch.cuda.current_stream(self.Hs[0].device))
        with torch.cuda.graph(g, stream=side):
            self.launch(stream=side)
        torch.cuda.current_stream(self.Hs[0].device).wait_stream(side)
        return g

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sp2_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apply_layers(X0: torch.Tensor, choices: Sequence[int], precision: str = "fp16", timeout_ms: float = 2000.0,
                 stream=None, cta_group: int = 0):
    """Apply the given layer signs to X0 (float32, symmetric); returns (X, Result)."""
    if X0.dtype != torch.float32:
        raise TypeError("X0 must be float32")
    X0 = X0.contiguous()
    n = _square(X0, "X0")
    X = torch.empty_like(X0)
    st = _new_stats()
    o = make_opts(precision, MAX_LAYERS_LIMIT, timeout_ms, cta_group=cta_group)
    ch = (ctypes.c_int * max(1, len(choices)))(*[int(c) for c in choices])
    s = load().sp2_apply_layers(ctypes.c_void_p(X0.data_ptr()), n, ch, len(choices), ctypes.c_void_p(X.data_ptr()),
                                ctypes.byref(st), ctypes.byref(o), ctypes.c_void_p(_stream_handle(X0, stream)))
    _check(s, "sp2_apply_layers")
    return X, _result(s, st)


def density_noalloc(H: torch.Tensor, n_occ: int, out: torch.Tensor, tol: float = 1e-6, precision: str = "fp16",
                    max_layers: int = 100, timeout_ms: float = 2000.0, stream=None):
    """sp2_density on the library's static device workspace (N <= 512, device tensors only).

    For callers that must not allocate device memory while running: nothing is
    allocated here either, so ``out`` (float32, N x N, on the device of H) is
    required.  Calls that overlap on the GPU share the workspace and race.
    """
    H = _f64(H, "H")
    n = _square(H, "H")
    st = _new_stats()
    o = make_opts(precision, max_layers, timeout_ms)
    s = load().sp2_density_noalloc(ctypes.c_void_p(H.data_ptr()), n, float(n_occ), float(tol),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.byref(st), ctypes.byref(o),
                                   ctypes.c_void_p(_stream_handle(H, stream)))
    _check(s, "sp2_density_noalloc")
    return out, _result(s, st)


def density_refined(H: torch.Tensor, n_occ: int, refine_layers: int = 2, tol: float = 1e-6,
                    precision: str = "fp16", max_layers: int = 100, timeout_ms: float = 2000.0, stream=None,
                    gap: Optional[Sequence[float]] = None, exact_slices: int = 0, profile: bool = False):
    """The chain plus ``refine_layers`` FP64 layers; returns (D float64, Result).  ``gap`` as for
    ``density`` (the FP64 layers are plain); ``exact_slices`` (4..6, 0 = 6) sets the accuracy of
    the refinement squares; ``profile`` fills Result.phase_ms with device times."""
    H = _f64(H, "H")
    n = _square(H, "H")
    D = torch.empty((n, n), dtype=torch.float64, device=H.device)
    st = _new_stats()
    o = make_opts(precision, max_layers, timeout_ms, gap=gap, profile=profile)
    o.exact_slices = int(exact_slices)
    s = load().sp2_density_refined(ctypes.c_void_p(H.data_ptr()), n, float(n_occ), float(tol), int(refine_layers),
                                   ctypes.c_void_p(D.data_ptr()), ctypes.byref(st), ctypes.byref(o),
                                   ctypes.c_void_p(_stream_handle(H, stream)))
    _check(s, "sp2_density_refined")
    return D, _result(s, st)


def density_nonorth(H: torch.Tensor, Z: torch.Tensor, n_occ: int, refine_layers: int = 0, tol: float = 1e-6,
                    precision: str = "fp16", max_layers: int = 100, timeout_ms: float = 2000.0, stream=None,
                    exact_slices: int = 0):
    """D = Z theta(mu I - Z^T H Z) Z^T (float64) for an inverse overlap factor Z; returns (D, Result)."""
    H, Z = _f64(H, "H"), _f64(Z, "Z")
    n = _square(H, "H")
    D = torch.empty((n, n), dtype=torch.float64, device=H.device)
    st = _new_stats()
    o = make_opts(precision, max_layers, timeout_ms)
    o.exact_slices = int(exact_slices)
    s = load().sp2_density_nonorth(ctypes.c_void_p(H.data_ptr()), ctypes.c_void_p(Z.data_ptr()), n, float(n_occ),
                                   float(tol), int(refine_layers), ctypes.c_void_p(D.data_ptr()), ctypes.byref(st),
                                   ctypes.byref(o), ctypes.c_void_p(_stream_handle(H, stream)))
    _check(s, "sp2_density_nonorth")
    return D, _result(s, st)


def congruence(Z: torch.Tensor, M: torch.Tensor, side: int = 0, timeout_ms: float = 2000.0, stream=None,
               exact_slices: int = 0):
    """Z^T M Z (side 0) or Z M Z^T (side 1) for symmetric M, float64 device tensors; returns the result."""
    Z, M = _f64(Z, "Z"), _f64(M, "M")
    n = _square(Z, "Z")
    if _square(M, "M") != n:
        raise ValueError("Z and M must have the same size")
    out = torch.empty((n, n), dtype=torch.float64, device=M.device)
    o = make_opts("fp16", timeout_ms=timeout_ms)
    o.exact_slices = int(exact_slices)
    s = load().sp2_congruence(ctypes.c_void_p(Z.data_ptr()), ctypes.c_void_p(M.data_ptr()), n, int(side),
                              ctypes.c_void_p(out.data_ptr()), ctypes.byref(o),
                              ctypes.c_void_p(_stream_handle(M, stream)))
    _check(s, "sp2_congruence")
    return out


def device_info():
    sm, ma, mi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    s = load().sp2_device_info(ctypes.byref(sm), ctypes.byref(ma), ctypes.byref(mi))
    return s, sm.value, (ma.value, mi.value)


class DensityMatrix(torch.autograd.Function):
    """D(H) by the SP2 chain with a reverse-mode gradient through the chain.

    backward(G) returns dTr[D G]/dH from ``sp2_adjoint`` replaying the forward's
    layer signs and spectral bounds (both held constant); ``checkpoint_stride`` is
    passed to it (recomputation of the layers between kept ones at large N).
    """

    @staticmethod
    def forward(ctx, H, n_occ, tol=1e-6, precision="fp16", max_layers=100, checkpoint_stride=0):
        D, res = density(H, n_occ, tol=tol, precision=precision, max_layers=max_layers)
        ctx.save_for_backward(H)
        ctx.res, ctx.n_occ, ctx.tol, ctx.precision = res, n_occ, tol, precision
        ctx.checkpoint_stride = checkpoint_stride
        return D

    @staticmethod
    def backward(ctx, grad_D):
        (H,) = ctx.saved_tensors
        _, dH, _ = adjoint(H, grad_D.to(torch.float64).contiguous(), ctx.n_occ, tol=ctx.tol,
                           precision=ctx.precision, fwd=ctx.res, checkpoint_stride=ctx.checkpoint_stride)
        return dH.to(H.dtype), None, None, None, None, None
