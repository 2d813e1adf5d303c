"""Helpers shared by the GPU tests: build/load the library, move seeded
NumPy inputs to the device in the library's layouts, and compare."""

import os

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

TORCH_DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16,
            "f16": torch.float16}


def planc():
    lib = os.path.join(ROOT, "paper_1909_01149_gb300", "lib", "libplanc.so")
    if not os.path.exists(lib):
        from paper_1909_01149_gb300 import build
        build.build()
    from paper_1909_01149_gb300 import planc as p
    return p


def x_to_device(X: np.ndarray, dt: str):
    """Flat mode-1-fastest device tensor of X in storage dtype dt, and the
    float64 NumPy array of the values actually stored (for the oracle)."""
    flat = np.ravel(np.asarray(X, dtype=np.float64), order="F")
    t = torch.from_numpy(flat).to(TORCH_DT[dt]).cuda()
    stored = t.double().cpu().numpy().reshape(X.shape, order="F")
    return t, stored


def factors_to_device(H, fdt: str):
    """Device factors (row-major I_n x R) and their stored float64 values."""
    ts = [torch.from_numpy(np.ascontiguousarray(h, dtype=np.float64)).to(TORCH_DT[fdt]).cuda()
          for h in H]
    return ts, [t.double().cpu().numpy() for t in ts]


def max_rel(got, ref, floor=0.0):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.maximum(np.abs(ref), floor)
    return float(np.max(np.abs(got - ref) / den)) if ref.size else 0.0
