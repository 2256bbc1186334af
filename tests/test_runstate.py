"""Run state in libae (ae_run_*, ae_checkpoint, ae_resume) on a host-only
context: checkpoint/resume, refusal of corrupt, truncated or foreign
checkpoints, the set estimate (Eqs. eq_sigma_down, eq_sigma_sum) and the
merge of two ranks' runs (gloo, two processes, CPU)."""
import math
import os

import pytest
import torch.multiprocessing as mp

import paper_1909_08015_b300 as ae
from paper_1909_08015_b300.runstate import RunState, rank_seed


def _fake(n, sy, sy2, my2=1.0):
    return {"n": n, "sum_y": sy, "sum_y2": sy2, "mean_abs": abs(sy) / n, "n_dd": 1, "n_nonfinite": 0,
            "max_y2": my2}


def _host(loops=2):
    c = ae.Context(-1)
    c.load_graphs(loops)
    return c


def test_estimate_by_hand():
    """value = sum mult_j mean_j, sigma^2 = sum (mult_j sigma_down_j)^2 with
    sigma_down^2 = sum y^2/N^2 - (sum y)^2/N^3; sigma_up^2 = sigma_down^2 +
    max y^2/N^2 (library heuristic).  2-loop multiplicities: 2, 2, 1, 1."""
    c = _host()
    st = RunState(c, seed=5)
    st.add(0, _fake(4, 10.0, 30.0, 16.0), 4)        # y = 1, 2, 3, 4
    st.add(3, _fake(2, 2.0, 10.0, 9.0), 2)          # y = -1, 3
    v, s, su, per = st.estimate()
    assert v == pytest.approx(2 * 2.5 + 1.0)
    assert s == pytest.approx(math.sqrt(4 * 5 / 16 + 2.0))
    assert su == pytest.approx(math.sqrt(4 * (5 / 16 + 16 / 16) + (2.0 + 9 / 4)))
    assert per[1]["n"] == 0 and per[1]["value"] == 0 and per[1]["sigma"] == 0
    assert per[0]["mean_abs"] == pytest.approx(2.5)


def test_checkpoint_roundtrip_and_resume(tmp_path):
    c = _host()
    st = RunState(c, seed=5)
    st.add(0, _fake(1000, 3.0, 20.0), 1000)
    st.add(1, _fake(1000, -1.0, 5.0), 1000)
    p = str(tmp_path / "run.ckpt")
    st.save(p)
    c2 = _host()
    st2 = RunState(c2, seed=0)
    st2.load(p)
    a, seed_a = st.state()
    b, seed_b = st2.state()
    assert a == b and seed_b == 5
    assert [g["next"] for g in b] == [1000, 1000, 0, 0]
    st2.add(0, _fake(500, 1.0, 8.0), 500)     # resume continues from the stored counter
    assert st2.state()[0][0]["next"] == 1500
    v, s, su, per = st2.estimate()
    assert v == pytest.approx(2 * 4.0 / 1500 + 2 * (-1.0 / 1000))
    assert not os.path.exists(p + ".tmp")


def test_corrupt_truncated_and_foreign_checkpoints_refused(tmp_path):
    c = _host()
    st = RunState(c, seed=1)
    st.add(0, _fake(10, 1.0, 1.0), 10)
    p = str(tmp_path / "run.ckpt")
    st.save(p)
    raw = open(p, "rb").read()
    before = st.state()
    bad = bytearray(raw)
    bad[len(raw) // 2] ^= 0x01                        # one flipped bit
    q = str(tmp_path / "bad.ckpt")
    open(q, "wb").write(bytes(bad))
    with pytest.raises(ae.AeError, match="AE_ERR_STATE.*checksum"):
        st.load(q)
    open(q, "wb").write(raw[: len(raw) // 2])          # truncated file
    with pytest.raises(ae.AeError, match="AE_ERR_STATE"):
        st.load(q)
    open(q, "wb").write(b"not a checkpoint at all, not at all")
    with pytest.raises(ae.AeError, match="AE_ERR_STATE"):
        st.load(q)
    assert st.state() == before                        # nothing changed
    c1 = _host(1)                                      # another graph set
    with pytest.raises(ae.AeError, match="AE_ERR_STATE.*graph set"):
        RunState(c1, 0).load(p)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = ae.Context(-1)
    c.load_graphs(2)
    st = RunState(c, seed=rank_seed(7, rank))
    st.add(0, _fake(100 * (rank + 1), 1.0 + rank, 2.0), 100)
    st.add(1, _fake(50, -0.5 * (rank + 1), 1.0), 50)
    st.merge_ranks()
    s, _ = st.state()
    out.put((rank, [g["n"] for g in s] + [g["sum_y"][0] + g["sum_y"][1] for g in s] + [g["next"] for g in s]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert res[r][:8] == [300, 100, 0, 0, 3.0, -1.5, 0.0, 0.0]
        assert res[r][8:] == [100, 50, 0, 0]           # each rank keeps its own stream position
    assert rank_seed(7, 0) != rank_seed(7, 1)
