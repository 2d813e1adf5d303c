"""Programmatic dependent launch changes only when kernels start, not what
they compute: solves with PLANC_PDL=0 and with it on (the default) give
bit-identical error histories and factors.  The switch is read once per
process, so each runs in a subprocess."""

import json
import os
import subprocess
import sys

import pytest

from helpers import ROOT, planc

pytestmark = pytest.mark.gpu

CODE = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
from helpers import planc
from paper_1909_01149_gb300 import synth
p = planc()
out = {}
for alg, dims, R in (("hals", (96, 128, 80), 16), ("nes", (64, 96, 72), 8), ("bpp", (40, 64, 30, 20), 6)):
    X, _ = synth.planted(dims, R, 5, noise=0.05, dtype=np.float32)
    Xd = torch.from_numpy(synth.flat(X)).cuda()
    H = [torch.from_numpy(h).cuda() for h in synth.init_factors(dims, R, 6, dtype=np.float32)]
    with p.Context(Xd, dims, R) as ctx:
        res = ctx.solve(H, alg, 6)
    out[alg] = {"rel_err": res["rel_err"], "H": [float(h.double().sum()) for h in H],
                "tc": res["tc_mask"]}
print(json.dumps(out))
"""


def _run(pdl):
    planc()  # library built
    env = dict(os.environ, PLANC_PDL=pdl)
    r = subprocess.run([sys.executable, "-c", CODE.replace("ROOT", repr(ROOT))], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_pdl_on_and_off_agree_bit_for_bit():
    on, off = _run("1"), _run("0")
    for alg in on:
        assert on[alg]["rel_err"] == off[alg]["rel_err"], alg
        assert on[alg]["H"] == off[alg]["H"], alg
    assert on["hals"]["tc"] == 3
