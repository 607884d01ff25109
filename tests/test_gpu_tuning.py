"""The tuning file: the library reads it once per process (EMST_TUNING_FILE),
applies the entry matching the GPU, dimension, form and size to the
parameters a call leaves open, ignores it on request, and the trees stay the
oracle's whatever it chooses."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, os.environ["EMST_ROOT"])
import numpy as np, torch, synth, oracle
import paper_2207_00514_gb300 as pkg
pkg.load_library()
out = []
for n, kw in [(50_000, {}), (200_000, {}), (200_000, {"ignore_tuning": True}),
              (200_000, {"block_size": 256})]:
    pts = synth.halos(n, 5)
    e, st = pkg.emst_compute_ex(torch.from_numpy(pts).cuda(), **kw)
    same = bool(np.array_equal(pkg.edges_numpy(e).view(np.uint8),
                               oracle.kd_boruvka(pts, threads=os.cpu_count() or 4).view(np.uint8)))
    out.append({"n": n, "kw": kw, "traversal": st["traversal_used"], "block": st["block_used"],
                "leaf": st["leaf_used"], "tuned": st["tuned"], "same": same})
print(json.dumps(out))
"""


def test_tuning_file_is_read_and_applied(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    name = torch.cuda.get_device_name().replace(" ", "_")
    f = tmp_path / "tuning.txt"
    f.write_text("# a test file\n"
                 f"gpu=Another_GPU dim=3 form=single nmin=0 nmax=1000000000 traversal=1 block=256\n"
                 f"gpu={name} dim=3 form=single nmin=0 nmax=100000 traversal=2 block=0 leaf=0 refill=4 chunk=32\n"
                 f"gpu={name} dim=3 form=single nmin=100000 nmax=1000000000 traversal=1 block=64 leaf=2 "
                 "refill=0 chunk=0  # trailing comment\n")
    env = dict(os.environ, EMST_TUNING_FILE=str(f), EMST_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, env=env,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert all(x["same"] for x in res)
    a, b, c, d = res
    assert a["tuned"] and a["traversal"] == 2
    assert b["tuned"] and b["traversal"] == 1 and b["block"] == 64 and b["leaf"] == 2
    assert not c["tuned"] and c["traversal"] == 1 and c["block"] == 128 and c["leaf"] == 1
    assert d["tuned"] and d["block"] == 256 and d["leaf"] == 2  # the caller's choice wins
