"""Write tests/golden/fullsize_oracle.json: the FP64 oracle's error history on
the full-size workloads, for the GPU parity tests that cannot run the oracle
in their own time budget.

Every value comes from ``oracle.nncp`` (Alg. 1 with Alg. 4's normalisation
and error identity) on inputs drawn by ``paper_1909_01149_gb300.synth``; the
BF16 case runs the oracle on the tensor rounded to BF16 (round to nearest
even, synth.to_bf16_bits, the rounding the library's storage uses), as the
mixed-precision reading prescribes.  Nothing here touches the CUDA library.

    python tests/golden/make_fullsize_golden.py          (about 10 minutes)
"""

from __future__ import annotations

import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as o  # noqa: E402
from paper_1909_01149_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "fullsize_oracle.json")


def _run(X, H0, alg, iters):
    t = time.time()
    r = o.nncp(np.asarray(X, dtype=np.float64), [np.asarray(h, dtype=np.float64) for h in H0],
               alg, iters=iters)
    print(f"  {alg} {iters} iterations: final {r['rel_err'][-1]:.12g} ({time.time() - t:.0f} s)",
          flush=True)
    return r


def dense512():
    """512^3 FP32 R=32, planted + 5% noise (the benchmark workload)."""
    dims, R = (512, 512, 512), 32
    X, _ = synth.planted(dims, R, 1, noise=0.05, dtype=np.float32)
    H0 = synth.init_factors(dims, R, 2, dtype=np.float32)
    out = {"dims": list(dims), "R": R, "data_seed": 1, "init_seed": 2, "noise": 0.05,
           "storage": "f32", "iters": 50}
    for alg in ("hals", "mu", "admm"):
        r = _run(X, H0, alg, 50)
        out[alg] = {"rel_err": r["rel_err"], "inner": r["inner"]}
    return out


def mouse_bf16():
    """128x128x200x100 R=16 mouse-like, stored in BF16; BPP, 30 iterations."""
    dims, R = (128, 128, 200, 100), 16
    X, _ = synth.mouse_like(dims, R, data_seed=1, dtype=np.float32)
    flat = synth.from_bf16_bits(synth.to_bf16_bits(synth.flat(X))).astype(np.float64)
    Xr = np.reshape(flat, dims, order="F")
    H0 = synth.init_factors(dims, R, 2, dtype=np.float32)
    r = _run(Xr, H0, "bpp", 30)
    return {"dims": list(dims), "R": R, "data_seed": 1, "init_seed": 2, "storage": "bf16",
            "iters": 30, "bpp": {"rel_err": r["rel_err"], "inner": r["inner"],
                                 "lam": [float(v) for v in r["lam"]],
                                 "colsum": [[float(v) for v in h.sum(axis=0)] for h in r["H"]]}}


def lownoise():
    """Planted 256^3 R=16 with 0.1% noise: from the usual random start (50
    HALS iterations) and from the planted factors perturbed by up to 10%
    (30 HALS iterations, close to the noise floor)."""
    dims, R = (256, 256, 256), 16
    X, A = synth.planted(dims, R, 1, noise=0.001, dtype=np.float32)
    out = {"dims": list(dims), "R": R, "data_seed": 1, "noise": 0.001, "storage": "f32"}
    H0 = synth.init_factors(dims, R, 2, dtype=np.float32)
    out["random_start"] = {"init_seed": 2, "iters": 50,
                           "rel_err": _run(X, H0, "hals", 50)["rel_err"]}
    Hp = synth.perturbed_factors(A, 0.1, 3, dtype=np.float32)
    out["near_start"] = {"perturb": 0.1, "perturb_seed": 3, "iters": 30,
                         "rel_err": _run(X, Hp, "hals", 30)["rel_err"]}
    return out


def main():
    doc = {"what": "FP64 oracle error histories (oracle.nncp) on seeded synthetic inputs",
           "generator": "tests/golden/make_fullsize_golden.py",
           "numpy": np.__version__, "machine": platform.machine()}
    for name, fn in (("lownoise256", lownoise), ("dense512", dense512), ("mouse4d_bf16", mouse_bf16)):
        print(name, flush=True)
        doc[name] = fn()
        with open(OUT, "w") as f:
            json.dump(doc, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
