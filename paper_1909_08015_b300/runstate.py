"""Run state of an integration: checkpoint/resume and multi-rank merging.

The per-graph state is (N, sum y, sum y^2, sum |y|, re-evaluated, zeroed) plus
the next Philox sample index.  Because the generator is counter-based,
continuing from the stored index draws exactly the samples an uninterrupted
run would have drawn.  Checkpoints are JSON with a SHA-256 of their payload,
so a corrupt or truncated file is refused rather than silently merged.

Under torch.distributed each rank integrates its own stream (seed offset by
rank) and the per-graph sums are added once at the end: no collective on the
data path.  Host logic only; the integration itself runs in libae.
"""
import hashlib
import json
import math

FIELDS = ("n", "sum_y", "sum_y2", "mean_abs_sum", "n_dd", "n_nonfinite")


def rank_seed(seed, rank):
    """Seed of a rank's disjoint Philox stream."""
    return int(seed) + 1000003 * int(rank)


class RunState:
    def __init__(self, graph_ids, mults, seed):
        self.graph_ids = list(graph_ids)
        self.mults = list(mults)
        self.seed = int(seed)
        self.next = [0] * len(self.graph_ids)
        self.sums = [{f: 0.0 for f in FIELDS} for _ in self.graph_ids]

    def add(self, k, res, count):
        """Fold one integration result of graph slot k covering `count` samples."""
        s = self.sums[k]
        s["n"] += res["n"]
        s["sum_y"] += res["sum_y"]
        s["sum_y2"] += res["sum_y2"]
        s["mean_abs_sum"] += res["mean_abs"] * res["n"]
        s["n_dd"] += res["n_dd"]
        s["n_nonfinite"] += res["n_nonfinite"]
        self.next[k] += int(count)

    def estimate(self):
        val = var = 0.0
        for m, s in zip(self.mults, self.sums):
            N = s["n"]
            if N == 0:
                continue
            v1 = s["sum_y2"] / N ** 2 - s["sum_y"] ** 2 / N ** 3
            val += m * s["sum_y"] / N
            var += m * m * max(v1, 0.0)
        return val, math.sqrt(var)

    # -------------------------------------------------------- checkpoints --
    def to_json(self):
        payload = {"graph_ids": self.graph_ids, "mults": self.mults, "seed": self.seed,
                   "next": self.next, "sums": self.sums}
        body = json.dumps(payload, sort_keys=True)
        return json.dumps({"sha256": hashlib.sha256(body.encode()).hexdigest(), "payload": payload},
                          sort_keys=True)

    def save(self, path):
        with open(path, "w") as f:
            f.write(self.to_json())

    @classmethod
    def from_json(cls, text):
        try:
            obj = json.loads(text)
            payload = obj["payload"]
            want = obj["sha256"]
        except (ValueError, KeyError, TypeError) as e:
            raise ValueError("checkpoint unreadable: %s" % e)
        body = json.dumps(payload, sort_keys=True)
        if hashlib.sha256(body.encode()).hexdigest() != want:
            raise ValueError("checkpoint checksum mismatch")
        st = cls(payload["graph_ids"], payload["mults"], payload["seed"])
        st.next = [int(x) for x in payload["next"]]
        st.sums = payload["sums"]
        if len(st.next) != len(st.graph_ids) or len(st.sums) != len(st.graph_ids):
            raise ValueError("checkpoint inconsistent")
        return st

    @classmethod
    def load(cls, path):
        with open(path) as f:
            return cls.from_json(f.read())

    # ------------------------------------------------------------ ranks ----
    def merge_ranks(self, group=None):
        """Add the per-graph sums of all ranks (torch.distributed, any
        backend); every rank gets the merged state."""
        import torch
        import torch.distributed as dist
        t = torch.tensor([[s[f] for f in FIELDS] for s in self.sums], dtype=torch.float64)
        dist.all_reduce(t, group=group)
        for s, row in zip(self.sums, t.tolist()):
            for f, v in zip(FIELDS, row):
                s[f] = v
        return self
