"""Timing of the secondary workloads (one JSON line each).

    python -m paper_2107_02737_gb300.measure --workload batched|response|adjoint|md|refined|accel|host

* ``batched``  — 64 gapped Hamiltonians of N in {128, ..., 2048}, BF16 split, one
  grouped persistent launch per step; effective TFLOP/s = sum_i L_i 2 N_i^3 / t.  Under
  torchrun (WORLD_SIZE > 1) the instances are split across the ranks by LPT on N^3,
  each rank solves its share in one grouped launch, and rank 0 prints the whole-job
  rate (all ranks' work over the slowest rank's time).
* ``response`` — D and D1 at N = 4096 (water-like H, banded H1); counts 4 N^3 per
  layer (the square and the product X X1).
* ``adjoint``  — dTr[DG]/dH at N = 4096, forward replayed from a density run, with
  every layer kept and with checkpointed recomputation; counts 2 N^3 (forward) +
  2 N^3 (reverse) per layer.
* ``md``       — H_k = H_0 + sin(0.05 k) V through sp2_response (see md.py).
* ``refined``  — the N = 8192 chain plus two FP64 refinement layers (exact-slice
  products on the FP16 tensor cores) for 4, 5 and 6 slices; device time of the chain,
  the refinement and the whole call (profile events), trace and idempotency.
* ``nonorth``  — the congruences Z^T H Z and Z D Z^T at N = 4096 (sp2_congruence),
  and the whole non-orthogonal route; effective TFLOP/s count 4 N^3 per congruence.
* ``accel``    — the N = 8192 chain, plain and accelerated from the generator's exact
  HOMO / LUMO (and from an interval four gaps wide around it); ms to D and layers.
* ``host``     — the N = 8192 chain called with host-resident H and D: page-locked
  (H read in place as its lower triangle, D written in place) and pageable (both
  copied whole), host wall time per call against the device-resident call.

Device time with CUDA events around each call, after warm-up, inputs resident on
the device (``host``: host wall time of each synchronous call).  These are
reports, not the headline benchmark (bench.py).
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import inputs, md
from . import sp2


def _time(fn, steps, warmup):
    for _ in range(warmup):
        out = fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, out


def batched_sharded(steps, warmup, precision="bf16"):
    """The 64-instance batch over the ranks of a torchrun launch (one GPU each): every
    rank solves its longest-processing-time share in one grouped launch; only timing
    scalars and per-instance records cross ranks."""
    import os

    import torch.distributed as dist

    from . import shard

    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    hams = inputs.batched_workload(64)
    sizes = [h.n for h in hams]

    def solve(idx):
        Hs = [torch.tensor(hams[i].H, device="cuda") for i in idx]
        occ = [hams[i].n_occ for i in idx]
        if not idx:
            return {}, 0.0, 0.0
        ms, (Ds, res, status) = _time(lambda: sp2.density_batched(Hs, occ, precision=precision), steps, warmup)
        recs = {i: {"n": hams[i].n, "layers": r.layers, "trace_err": r.trace_D - hams[i].n_occ, "status": r.status}
                for i, r in zip(idx, res)}
        return recs, ms, sum(r.layers * 2.0 * hams[i].n ** 3 for i, r in zip(idx, res))

    recs, mine, ms, work = shard.run_sharded_batch(sizes, solve, rank, world, device=torch.device("cuda", local))
    out = None
    if rank == 0:
        out = {"workload": f"batched 64 x N in {{128..2048}} over {world} ranks (LPT on N^3)",
               "precision": precision, "n_gpus": world, "ms_per_step": ms,
               "effective_tflops": work / (ms * 1e-3) / 1e12, "instances": len(recs),
               "max_trace_err": max(abs(r["trace_err"]) for r in recs.values()),
               "all_ok": all(r["status"] == 0 for r in recs.values())}
    dist.destroy_process_group()
    return out


def batched(steps, warmup, precision="bf16"):
    import os

    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        return batched_sharded(steps, warmup, precision)
    hams = inputs.batched_workload(64)
    Hs = [torch.tensor(h.H, device="cuda") for h in hams]
    occ = [h.n_occ for h in hams]
    ms, (Ds, res, status) = _time(lambda: sp2.density_batched(Hs, occ, precision=precision), steps, warmup)
    work = sum(r.layers * 2.0 * h.n ** 3 for r, h in zip(res, hams))
    # Accuracy by properties that hold for the exact D: idempotency and trace.
    idem = max(float(torch.linalg.norm(D.double() @ D.double() - D.double())) / np.sqrt(h.n)
               for h, D in zip(hams, Ds))
    tr = max(abs(r.trace_D - h.n_occ) for h, r in zip(hams, res))
    seq_ms = 0.0
    for h, H in zip(hams, Hs):
        t, _ = _time(lambda: sp2.density(H, h.n_occ, precision=precision), 1, 1)
        seq_ms += t
    # The same batch as a reusable plan (tile shape by the autotuner), launched
    # directly and as a replayed CUDA graph.
    plan = sp2.BatchPlan(Hs, occ, precision=precision, autotune=True)
    plan_ms, _ = _time(plan.launch, steps, warmup)
    graph = plan.capture()
    graph_ms, _ = _time(graph.replay, steps, warmup)
    pres, pstatus = plan.stats()
    plan_cg = plan.cta_group
    same = all(torch.equal(a, b) for a, b in zip(Ds, plan.Ds)) if plan_cg == res[0].cta_group else None
    plan.close()
    return {"workload": "batched 64 x N in {128..2048}", "precision": precision, "ms_per_step": ms,
            "effective_tflops": work / (ms * 1e-3) / 1e12, "sum_layers": sum(r.layers for r in res),
            "one_by_one_ms": seq_ms, "max_idempotency_per_sqrtN": idem, "max_trace_err": tr, "status": status,
            "plan": {"cta_group": plan_cg, "launch_ms": plan_ms, "graph_replay_ms": graph_ms,
                     "effective_tflops_graph": work / (graph_ms * 1e-3) / 1e12, "status": pstatus,
                     "equal_to_batched_call": same}}


def response(steps, warmup, n=4096):
    ham, H1, _ = inputs.differentiation_workload(n)
    H, H1d = torch.tensor(ham.H, device="cuda"), torch.tensor(H1, device="cuda")
    ms, (D, D1, res) = _time(lambda: sp2.response(H, H1d, ham.n_occ), steps, warmup)
    return {"workload": f"response N={n}", "ms_per_step": ms, "layers": res.layers, "d1_norm": float(D1.norm()),
            "effective_tflops": res.layers * 4.0 * n ** 3 / (ms * 1e-3) / 1e12}


def adjoint(steps, warmup, n=4096):
    ham, _, G = inputs.differentiation_workload(n)
    H, Gd = torch.tensor(ham.H, device="cuda"), torch.tensor(G, device="cuda")
    _, fwd = sp2.density(H, ham.n_occ)
    out = {"workload": f"adjoint N={n}"}
    ref = None
    # every layer kept, then the checkpoint stride of least memory (layers between kept
    # ones recomputed in the reverse sweep; the gradient is the same bits)
    for name, stride in [("stored", 0), ("checkpointed", -1)]:
        ms, (D, dH, res) = _time(lambda: sp2.adjoint(H, Gd, ham.n_occ, fwd=fwd, checkpoint_stride=stride),
                                 steps, warmup)
        ref = dH if ref is None else ref
        out[name] = {"ms_per_step": ms, "layers": res.layers,
                     "effective_tflops": res.layers * 4.0 * n ** 3 / (ms * 1e-3) / 1e12,
                     "workspace_gb": sp2.workspace_bytes(n, "adjoint", layers=res.layers,
                                                         checkpoint_stride=stride) / 1e9,
                     "equal_to_stored": bool(torch.equal(dH, ref))}
    return out


def refined(steps, warmup, n=8192, layers=2, slice_counts=(4, 5, 6)):
    ham = inputs.water_like_workload(n)
    H = torch.tensor(ham.H, device="cuda")
    ws = torch.empty(sp2.workspace_bytes(n, "density"), dtype=torch.uint8, device="cuda")
    ms_chain, (_, r0) = _time(lambda: sp2.density(H, ham.n_occ, workspace=ws), steps, warmup)
    out = {"workload": f"refined N={n}", "refine_layers": layers, "chain_ms": ms_chain,
           "chain_trace_err": r0.trace_D - ham.n_occ}
    for slices in slice_counts:
        runs = []
        for k in range(warmup + steps):
            D, res = sp2.density_refined(H, ham.n_occ, refine_layers=layers, exact_slices=slices, profile=True)
            if k >= warmup:
                runs.append(res.phase_ms)
        torch.cuda.synchronize()
        mean = [float(np.mean([r[i] for r in runs])) for i in range(4)]
        out[f"slices_{slices}"] = {"device_ms_to_D": mean[3], "chain_device_ms": mean[0],
                                   "refinement_device_ms": mean[1], "output_device_ms": mean[2],
                                   "trace_err": res.trace_D - ham.n_occ,
                                   "idem_fro": float(torch.linalg.norm(D @ D - D))}
    return out


def nonorth(steps, warmup, n=4096):
    rng = inputs.rng_for(6, n)
    ham = inputs.water_like_workload(n)
    S = inputs.overlap_matrix(n, rng)
    lam, U = np.linalg.eigh(S)
    Z = torch.tensor((U / np.sqrt(lam)) @ U.T, device="cuda")     # Lowdin factor S^(-1/2)
    Sh = (U * np.sqrt(lam)) @ U.T
    Hn = Sh @ ham.H @ Sh
    H = torch.tensor(0.5 * (Hn + Hn.T), device="cuda")
    out = {"workload": f"non-orthogonal route N={n}"}
    for side in (0, 1):
        ms, C = _time(lambda: sp2.congruence(Z, H, side), steps, warmup)
        out[f"congruence_side{side}_ms"] = ms
        out[f"congruence_side{side}_tflops"] = 4.0 * n ** 3 / (ms * 1e-3) / 1e12
    ms, (D, res) = _time(lambda: sp2.density_nonorth(H, Z, ham.n_occ, refine_layers=2), steps, warmup)
    Sd = torch.tensor(S, device="cuda")
    out.update({"nonorth_ms": ms, "layers": res.layers,
                "trace_DS_err": float(torch.trace(D @ Sd)) - ham.n_occ,
                "DSD_minus_D_fro": float(torch.linalg.norm(D @ Sd @ D - D))})
    return out


def accel(steps, warmup, n=8192, precision="fp16"):
    ham = inputs.water_like_workload(n)
    H = torch.tensor(ham.H, device="cuda")
    homo, lumo = float(ham.eigvals[ham.n_occ - 1]), float(ham.eigvals[ham.n_occ])
    w = lumo - homo
    out = {"workload": f"accelerated N={n}", "precision": precision, "gap": w}
    for name, gap in [("plain", None), ("exact", (homo, lumo)), ("wide", (homo - 1.5 * w, lumo + 1.5 * w))]:
        ms, (D, res) = _time(lambda: sp2.density(H, ham.n_occ, precision=precision, gap=gap), steps, warmup)
        Dd = D.double()
        idem = float(torch.linalg.norm(Dd @ Dd - Dd))
        out[name] = {"ms_to_D": ms, "layers": res.layers, "trace_err": res.trace_D - ham.n_occ,
                     "idem_fro": idem, "effective_tflops": res.layers * 2.0 * n ** 3 / (ms * 1e-3) / 1e12}
    return out


def host(steps, warmup, n=8192, precision="fp16"):
    import time

    ham = inputs.water_like_workload(n)
    Hd = torch.tensor(ham.H, device="cuda")
    # Caller workspaces, as a repeated caller passes them: the solve's own, and with
    # room after it for staging host matrices (8 bytes per H and 4 per D element).
    wsb = sp2.workspace_bytes(n, "density", precision)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    ws_host = torch.empty(wsb + n * n * 12 + 4096, dtype=torch.uint8, device="cuda")
    dev_ms, (Dd, r0) = _time(lambda: sp2.density(Hd, ham.n_occ, precision=precision, workspace=ws), steps, warmup)
    ref = Dd.cpu()
    out = {"workload": f"host round trip N={n}", "precision": precision, "layers": r0.layers,
           "device_resident_ms": dev_ms}
    for name, pin in [("page_locked", True), ("pageable", False)]:
        H = torch.from_numpy(ham.H)
        D = torch.empty((n, n), dtype=torch.float32)
        if pin:
            H, D = H.pin_memory(), D.pin_memory()
        for _ in range(warmup):
            sp2.density(H, ham.n_occ, precision=precision, out=D, workspace=ws_host)
        t0 = time.perf_counter()
        for _ in range(steps):
            _, r = sp2.density(H, ham.n_occ, precision=precision, out=D, workspace=ws_host)
        ms = (time.perf_counter() - t0) * 1e3 / steps
        h2d = (n * (n + 1) // 2 if pin else n * n) * 8
        out[name] = {"ms_per_call": ms, "added_ms": ms - dev_ms, "h2d_bytes": h2d, "d2h_bytes": n * n * 4,
                     "effective_tflops": r.layers * 2.0 * n ** 3 / (ms * 1e-3) / 1e12,
                     "equal_to_device_result": bool(torch.equal(D, ref))}
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", choices=["batched", "response", "adjoint", "md", "refined", "nonorth", "accel",
                                           "host"], required=True)
    ap.add_argument("--accelerate", action="store_true", help="md: reuse HOMO / LUMO estimates step to step")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--layers", type=int, default=2, help="refined: FP64 refinement layers")
    ap.add_argument("--slices", type=int, default=0, help="refined: one slice count (4..6) instead of all three")
    a = ap.parse_args(argv)
    if a.workload == "batched":
        out = batched(a.steps, a.warmup)
        if out is None:   # a rank other than 0 of a sharded run
            return 0
    elif a.workload == "response":
        out = response(a.steps, a.warmup, a.n or 4096)
    elif a.workload == "adjoint":
        out = adjoint(a.steps, a.warmup, a.n or 4096)
    elif a.workload == "refined":
        out = refined(a.steps, a.warmup, a.n or 8192, a.layers, (a.slices,) if a.slices else (4, 5, 6))
    elif a.workload == "nonorth":
        out = nonorth(a.steps, a.warmup, a.n or 4096)
    elif a.workload == "accel":
        out = accel(a.steps, a.warmup, a.n or 8192)
    elif a.workload == "host":
        out = host(a.steps, a.warmup, a.n or 8192)
    else:
        return md.main(["--n", str(a.n or 12288), "--steps", str(a.steps)] + (["--accelerate"] if a.accelerate else []))
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
