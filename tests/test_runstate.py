"""Run state: checkpoint/resume, corrupted checkpoints, and merging the
per-graph sums of several ranks (gloo, two processes, CPU)."""
import json
import os

import pytest
import torch.multiprocessing as mp

from paper_1909_08015_b300.runstate import RunState, rank_seed


def _fake(n, sy, sy2):
    return {"n": n, "sum_y": sy, "sum_y2": sy2, "mean_abs": abs(sy) / n, "n_dd": 1, "n_nonfinite": 0}


def test_checkpoint_roundtrip_and_resume(tmp_path):
    st = RunState([0, 1], [2, 1], seed=5)
    st.add(0, _fake(1000, 3.0, 20.0), 1000)
    st.add(1, _fake(1000, -1.0, 5.0), 1000)
    p = tmp_path / "ck.json"
    st.save(p)
    st2 = RunState.load(p)
    assert st2.next == [1000, 1000] and st2.sums == st.sums and st2.seed == 5
    st2.add(0, _fake(500, 1.0, 8.0), 500)     # resume continues from the stored counter
    assert st2.next[0] == 1500
    v, s = st2.estimate()
    assert v == pytest.approx(2 * 4.0 / 1500 + (-1.0 / 1000))


def test_corrupt_and_truncated_checkpoints_refused(tmp_path):
    st = RunState([0], [1], seed=1)
    st.add(0, _fake(10, 1.0, 1.0), 10)
    text = st.to_json()
    obj = json.loads(text)
    obj["payload"]["sums"][0]["sum_y"] = 2.0          # flipped value
    with pytest.raises(ValueError, match="checksum"):
        RunState.from_json(json.dumps(obj))
    with pytest.raises(ValueError, match="unreadable"):
        RunState.from_json(text[: len(text) // 2])   # truncated file


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    st = RunState([0, 1], [1, 2], seed=rank_seed(7, rank))
    st.add(0, _fake(100 * (rank + 1), 1.0 + rank, 2.0), 100)
    st.add(1, _fake(50, -0.5 * (rank + 1), 1.0), 50)
    st.merge_ranks()
    if rank == 0:
        out.put([s["n"] for s in st.sums] + [s["sum_y"] for s in st.sums])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=60)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [300.0, 100.0, 3.0, -1.5]
    assert rank_seed(7, 0) != rank_seed(7, 1)
