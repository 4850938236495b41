"""The autotuner's JSON cache (host logic, no GPU): processes that record
tuned shapes at the same time, as the ranks of a multi-GPU run do, leave a
readable file whose entries each come whole from one of them."""
import json
import multiprocessing as mp

import pytest


def _writer(path, rank, count):
    import os
    os.environ["GPUTB_TUNE_CACHE"] = path
    from paper_2509_06525_gb300 import gputb as g
    g._gpu_name = lambda: "test-gpu"
    g.kpm_shape_info = lambda R, prec, shape: {"shape": int(shape)}
    for k in range(count):
        g._record_tuned(1 << (10 + k % 8), 8, 0, 1, rank)


def test_concurrent_records_leave_a_whole_file(tmp_path):
    pytest.importorskip("torch")
    path = str(tmp_path / "tuned.json")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_writer, args=(path, r, 40)) for r in range(4)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    data = json.load(open(path))
    entries = data["test-gpu"]
    assert 1 <= len(entries) <= 8
    for key, e in entries.items():
        assert e["R"] == 8 and e["mode"] == 1 and e["shape"] in range(4) and e["desc"] == {"shape": e["shape"]}
    assert not list(tmp_path.glob("*.tmp"))
