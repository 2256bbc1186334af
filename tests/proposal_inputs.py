"""Seeded synthetic inputs for the learned-proposal tests: network
parameters and training records (line orders, ln t values, weights).  Pure
random-number generation; none of the method's arithmetic lives here."""
import numpy as np

NPARAM = 11472
LAYOUT = [(64, 32), (64,), (64, 64), (64,), (64, 64), (64,), (16, 64), (16,)]


def params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for shp in LAYOUT:
        fan = shp[1] if len(shp) == 2 else 64
        out.append(rng.normal(0, scale / np.sqrt(fan), size=shp).ravel())
    return np.concatenate(out).astype(np.float32)


def records(seed, n, M):
    rng = np.random.default_rng(seed + 1)
    order = np.zeros((n, 16), dtype=np.uint8)
    for i in range(n):
        order[i, :M] = rng.permutation(M)
    lt = np.zeros((n, 16), dtype=np.float32)
    lt[:, 1:M] = -rng.exponential(2.0, size=(n, M - 1))
    w = rng.lognormal(0, 1.5, size=n)
    return order, lt, w
