"""Helpers shared by the GPU parity tests (device transfer and error norms)."""
import numpy as np
import torch


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().cpu().double().numpy()


def fro_err(D, ref):
    """||D - ref||_F / sqrt(N), the per-result error measure used throughout."""
    return float(np.linalg.norm(np.asarray(D, np.float64) - ref) / np.sqrt(ref.shape[0]))


def rel_err(a, ref):
    return float(np.linalg.norm(np.asarray(a, np.float64) - ref) / np.linalg.norm(ref))


# ||D - D_oracle||_F / sqrt(N) bounds: 1e-3 for the split 16-bit precisions and
# 1e-5 for FP32 (the stated agreement targets for this method).
TOL_D = {"fp16": 1e-3, "bf16": 1e-3, "fp32": 1e-5}
