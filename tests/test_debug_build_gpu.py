"""The debug build (GPU): libbsm_debug.so, compiled with -DBSM_DEBUG, checks
every numeric item's output block and every product's operand blocks against
the arrays' sizes before computing it (a violation sets an error bit and the
multiply returns BSM_ERR_CUDA; nothing is read outside the arrays).  On valid
inputs no check may fire and the results must be bit for bit those of the
release build: both builds run the same script in fresh processes here
(the binding loads the debug build when BSM_DEBUG=1)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, ".")
from paper_1708_03604_gb300 import bsm, inputs as I
from tests.helpers import random_bcsr
torch.cuda.set_device(0)
out = {}
bs = np.random.default_rng(8).integers(1, 41, size=40).astype(np.int32)
A, B = random_bcsr(bs, bs, 0.2, seed=61), random_bcsr(bs, bs, 0.2, seed=62)
C0 = random_bcsr(bs, bs, 0.1, seed=63)
gA, gB = bsm.Matrix.from_host(A), bsm.Matrix.from_host(B)
for prec, fl in (("fp64", 0), ("fp64_dmma", 0), ("tf32x3", 0), ("tf32x3", 4), ("bf16x6", 0), ("bf16x3", 0),
                 ("ozaki", 0)):
    Cm = bsm.multiply(1.0, gA, gB, eps=0.5, prec=prec, flush_every=fl)
    out[f"{prec}_{fl}"] = Cm.data_host()
    G = torch.tensor(np.random.default_rng(3).standard_normal(Cm.info().data_len), device="cuda")
    dA = torch.zeros(len(A.data), dtype=torch.float64, device="cuda")
    dB = torch.zeros(len(B.data), dtype=torch.float64, device="cuda")
    bsm.multiply_backward(1.0, Cm, G, gA, gB, dA, dB, prec=prec)
    out[f"{prec}_{fl}_dA"] = dA.cpu().numpy()
    out[f"{prec}_{fl}_dB"] = dB.cpu().numpy()
Cb = bsm.multiply(2.0, gA, gB, beta=-0.5, Cm=bsm.Matrix.from_host(C0), eps=0.5)
out["beta"] = Cb.data_host()
tiny = I.mixed_sizes(60, (1, 2, 4, 5), (0.3, 0.2, 0.3, 0.2), seed=4)
T1, T2 = random_bcsr(tiny, tiny, 0.2, seed=71), random_bcsr(tiny, tiny, 0.2, seed=72)
for prec in ("fp64", "tf32x3", "ozaki"):
    out[f"tiny_{prec}"] = bsm.multiply(1.0, bsm.Matrix.from_host(T1), bsm.Matrix.from_host(T2), prec=prec).data_host()
np.savez(sys.argv[1], **out)
print("LIB", bsm.LIB_PATH)
'''


def _run(tmp_path, debug):
    env = dict(os.environ)
    env.pop("BSM_DEBUG", None)
    if debug:
        env["BSM_DEBUG"] = "1"
    path = str(tmp_path / ("dbg.npz" if debug else "rel.npz"))
    r = subprocess.run([sys.executable, "-c", SCRIPT, path], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return np.load(path), r.stdout


@pytest.fixture(scope="module")
def debug_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_03604_gb300 import build
    return build.build(debug=True)


def test_debug_build_runs_clean_and_matches_release(debug_lib, tmp_path):
    assert debug_lib.endswith("libbsm_debug.so")
    dbg, out_dbg = _run(tmp_path, True)
    rel, out_rel = _run(tmp_path, False)
    assert "libbsm_debug.so" in out_dbg and "libbsm.so" in out_rel
    assert sorted(dbg.files) == sorted(rel.files)
    for k in rel.files:
        np.testing.assert_array_equal(dbg[k], rel[k], err_msg=k)
