"""The committed tuning file (written by paper_2207_00514_gb300/tune.py on the
GPU) is well formed: every entry names a GPU, a dimension, a form and a size
range, and its choices are values the library accepts."""
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PATH = os.path.join(ROOT, "paper_2207_00514_gb300", "emst_tuning.txt")


def test_committed_tuning_file_is_well_formed():
    if not os.path.exists(PATH):
        return  # no tuned entries: the library uses its defaults
    entries = 0
    for line in open(PATH):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        kv = dict(tok.split("=", 1) for tok in line.split())
        for k in ("gpu", "dim", "form", "nmin", "nmax", "traversal"):
            assert k in kv, (k, line)
        assert kv["dim"] in ("2", "3") and kv["form"] in ("single", "batched")
        assert 0 <= int(kv["nmin"]) < int(kv["nmax"])
        assert kv["traversal"] in ("1", "2")
        b, leaf = int(kv.get("block", 0)), int(kv.get("leaf", 0))
        assert b == 0 or (64 <= b <= 256 and b % 32 == 0)
        assert leaf == 0 or leaf in (1, 2, 4, 8, 16)
        r, c = int(kv.get("refill", 0)), int(kv.get("chunk", 0))
        assert 0 <= r <= 32 and (c == 0 or c >= 32)
        entries += 1
    assert entries > 0
