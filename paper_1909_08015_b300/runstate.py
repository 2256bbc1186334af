"""Run state of an integration campaign: a thin wrapper over libae's run
calls (ae_run_*, ae_checkpoint, ae_resume).

libae keeps, per loaded graph, the next sample index of its counter-based
stream and the running sums; it computes the estimate, writes and reads
checksummed checkpoints and merges runs.  This module only moves bytes:
under torch.distributed every rank integrates its own stream (seed offset by
rank, no collective on the data path) and merge_ranks() gathers the ranks'
raw run states once, each rank then adding the others' sums in rank order
through ae_run_merge.
"""
import ctypes

from . import AeRunGraph


def rank_seed(seed, rank):
    """Seed of a rank's disjoint Philox stream."""
    return int(seed) + 1000003 * int(rank)


class RunState:
    """A run over all graphs loaded in `ctx` (a paper_1909_08015_b300.Context)."""

    def __init__(self, ctx, seed):
        self.ctx = ctx
        ctx.run_reset(seed)

    @classmethod
    def attach(cls, ctx):
        """Wrap the run the context already holds (no reset)."""
        st = cls.__new__(cls)
        st.ctx = ctx
        return st

    def step(self, ids, n_samples):
        """One batched block: graph ids[i] continues its stream by n_samples[i]
        (returns the block's per-graph results)."""
        return self.ctx.run_step(ids, n_samples)

    def add(self, gid, result, count):
        """Fold an integration result of `count` samples of graph gid."""
        self.ctx.run_add(gid, result, count)

    def state(self):
        """(list of per-graph dicts, seed)."""
        arr, seed = self.ctx.run_get()
        out = []
        for g in arr:
            out.append({"next": g.next, "n": g.n, "n_dd": g.n_dd, "n_zero": g.n_zero,
                        "sum_y": tuple(g.sum_y), "sum_y2": tuple(g.sum_y2), "sum_abs": tuple(g.sum_abs),
                        "max_y2": g.max_y2})
        return out, seed

    def estimate(self):
        """(value, sigma_down, sigma_up, per-graph results)."""
        return self.ctx.run_estimate()

    def save(self, path):
        self.ctx.checkpoint(path)

    def load(self, path):
        self.ctx.resume(path)

    def merge_ranks(self, group=None):
        """Every rank ends with the sums of all ranks (its own next indices)."""
        import torch
        import torch.distributed as dist
        arr, _ = self.ctx.run_get()
        raw = bytes(arr)
        t = torch.frombuffer(bytearray(raw), dtype=torch.uint8)
        if dist.get_backend(group) == "nccl":   # NCCL moves device tensors only
            t = t.to(torch.device("cuda", torch.cuda.current_device()))
        world = dist.get_world_size(group)
        me = dist.get_rank(group)
        parts = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(parts, t, group=group)
        for r in range(world):
            if r == me:
                continue
            other = (AeRunGraph * len(arr)).from_buffer_copy(parts[r].cpu().numpy().tobytes())
            self.ctx.run_merge(other)
        return self
