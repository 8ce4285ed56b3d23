"""The bounds-checked library (-DMS_DEBUG_BOUNDS) on every workload: no env
reports MS_ENV_BOUNDS, and its states equal the release library's bit for
bit (the checks read, never change, what the stages compute).  The debug
library runs in a child process: a process loads one libmsim."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import scenegen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = [("small", 64), ("arm", 64), ("clutter", 48), ("hand", 32), ("mixed", 48), ("hulls", 48), ("pick", 32)]
STEPS = 40

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2410_00425_b300 import _ffi
_ffi.load(sys.argv[2])
import torch, scenegen
from paper_2410_00425_b300 import Batch
out = {}
for name, E in json.loads(sys.argv[3]):
    sc = scenegen.make_scene(name, n_envs=E)
    b = Batch(sc)
    if sc.task is not None:
        b.set_task(sc.task)
    acts = sc.actions(0, int(sys.argv[4]))
    s = torch.cuda.Stream()
    for k in range(int(sys.argv[4])):
        a = None if acts is None else torch.from_numpy(acts[k:k + 1]).cuda()
        b.step(a, 1, stream=s)
    torch.cuda.synchronize()
    code, st = b.sync()
    out[name] = {"state": b.state().cpu().numpy().tolist(), "status": st.tolist()}
    b.close()
json.dump(out, open(sys.argv[5], "w"))
"""


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(lib, tmp_path, tag):
    dst = str(tmp_path / f"{tag}.json")
    subprocess.check_call([sys.executable, "-c", CHILD, ROOT, lib, json.dumps(CASES), str(STEPS), dst],
                          cwd=ROOT, timeout=900)
    return json.load(open(dst))


def test_debug_library_reports_nothing_and_matches_release(tmp_path):
    from paper_2410_00425_b300 import build
    dbg = _run(build.build(debug=True), tmp_path, "debug")
    rel = _run(build.build(), tmp_path, "release")
    bounds = 32                                     # MS_ENV_BOUNDS
    for name, _ in CASES:
        st = np.array(dbg[name]["status"], np.uint32)
        assert not (st & bounds).any(), (name, np.nonzero(st & bounds)[0].tolist())
        assert np.array_equal(np.array(dbg[name]["state"], np.float32), np.array(rel[name]["state"], np.float32)), name
