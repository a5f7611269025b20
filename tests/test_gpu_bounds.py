"""Bounds-checked build (QA_CHECK_BOUNDS; builder.build_checked -> libqa_checked.so).

The index-map gathers of the fused bubble + FFT (the -R map and the bubble's
term lists) and of the double-float self-energy (its target-grouped term
lists) check every index in that build and report QA_EBOUNDS instead of
reading out of range.  A step through the checked library must report no
violation and reproduce the product library's results exactly (the checks
change no arithmetic).  Each library runs in a subprocess of its own
(QA_LIB selects the build at the first load).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (workload, precision): the double-float line FFT with the fused bubble and the
# double-float self-energy (16x16x8), the generic reduced bubble (ragged grid), the
# register FFT with the fused bubble in FP64 (4x4x2)
CASES = [("peierls-16x16x8", "mixed"), ("five-orbital-4x3x2", "mixed"), ("peierls-4x4x2", "fp64")]

SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
import workloads as wl
from paper_2604_22223_gb300 import qa
out = {{}}
for i, (name, prec) in enumerate({cases!r}):
    ctx = qa.Context(wl.config(name), prec)
    G1, mu1, n1, st = ctx.step()
    G2, mu2, n2, st = ctx.step(G1)
    out["G%d" % i] = G2.cpu().numpy()
    out["S%d" % i] = np.asarray(ctx.get(qa.QA_SIGC_KTAU).cpu().numpy())
    out["mu%d" % i] = np.array([mu1, mu2])
np.savez({path!r}, **out)
"""


def _run(tmp_path, lib):
    path = str(tmp_path / ("out_%s.npz" % ("checked" if lib else "plain")))
    env = dict(os.environ)
    env.pop("QA_LIB", None)
    if lib:
        env["QA_LIB"] = lib
    code = SCRIPT.format(root=ROOT, cases=CASES, path=path)
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stdout + p.stderr
    return dict(np.load(path))


def test_checked_build_matches_product_library(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_22223_gb300 import builder
    builder.build()
    lib = builder.build_checked()
    assert os.path.exists(lib)
    plain = _run(tmp_path, None)
    checked = _run(tmp_path, lib)           # a QA_EBOUNDS status would raise in the subprocess
    assert plain.keys() == checked.keys()
    for k in plain:
        a, b = plain[k], checked[k]
        err = np.abs(a - b).max() / max(np.abs(a).max(), 1e-300)
        assert err <= 1e-13, (k, err)
