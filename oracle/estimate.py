"""Oracle: Monte Carlo estimator (Sec. III.B) on the Philox sample stream.

TEST INFRASTRUCTURE ONLY (see the package header).

For sample index i of graph j under seed s:
    u    = Philox uniforms (philox.uniforms),
    z, g = sampler.sample(density, u),
    y_i  = I(z)/g(z)   (Eq. eq_integral_approx), computed range-safely as
           y = (I * 2^(kf - log2 g)) * 2^-kf with kf = floor(log2 g).
value = (1/N) sum y, sigma_down^2 = sum y^2/N^2 - (sum y)^2/N^3
(Eq. eq_sigma_down); set sums add mult_j value_j with sigma^2 = sum
(mult_j sigma_j)^2 (Eq. eq_sigma_sum).  Sums are compensated (math.fsum).

Pins: summarize() on hand-computed sigma_down; weight_many() against
weight() element by element; samples_batched() through the 2-loop set sum
against the closed form (a statistical pin) and its integrand against the
exact one point by point.
"""
import math
import numpy as np

from .graphs import enumerate_graphs
from .integrand import Integrand
from .philox import uniforms
from . import mrg32k3a
from .sampler import CALC1, CALC2, Density, sample, exp2_tab


def weight(I, lg):
    kf = math.floor(lg)
    s = float(exp2_tab(kf - lg))
    kc = min(max(kf, -100000.0), 100000.0)
    return math.ldexp(I * s, -int(kc))


def weight_many(I, lg):
    """weight() over arrays: y = (I 2^(kf - log2 g)) 2^-kf, kf = floor(log2 g)."""
    I = np.asarray(I, dtype=np.float64)
    lg = np.asarray(lg, dtype=np.float64)
    kf = np.floor(lg)
    s = exp2_tab(kf - lg)
    kc = np.clip(kf, -100000.0, 100000.0).astype(np.int64)
    return np.ldexp(I * s, -kc)


class GraphOracle:
    """calc=2: Philox4x32-10 and the Calc 2 constants; calc=1: MRG32k3a and
    the Calc 1 constants (Sec. V)."""

    def __init__(self, g, graph_id, calc=2, integrand=True, tables=None):
        self.g = g
        self.gid = graph_id
        self.calc = calc
        self.dens = Density(g, **(CALC1 if calc == 1 else CALC2))
        self.integrand = Integrand(g, tables=tables) if integrand else None

    def uniforms(self, idx, seed):
        if self.calc == 1:
            return mrg32k3a.uniforms(idx, self.gid, seed, self.dens.M)
        return uniforms(idx, self.gid, seed, self.dens.M)

    def points(self, first, count, seed=0):
        """Sample points and densities only (no integrand)."""
        idx = np.arange(first, first + count, dtype=np.uint64)
        z, lg, comp = sample(self.dens, self.uniforms(idx, seed))
        return dict(z=z, log2g=lg, comp=comp)

    def samples(self, first, count, seed=0):
        """Per-sample (z, log2g, I, K, y) for samples first..first+count-1."""
        idx = np.arange(first, first + count, dtype=np.uint64)
        u = self.uniforms(idx, seed)
        z, lg, comp = sample(self.dens, u)
        I = np.empty(count)
        K = np.empty(count)
        y = np.empty(count)
        for k in range(count):
            I[k], K[k] = self.integrand.evaluate(z[k])
            y[k] = weight(I[k], lg[k])
        return dict(z=z, log2g=lg, I=I, K=K, y=y, comp=comp)


    def samples_batched(self, first, count, seed=0, chunk=1 << 17):
        """Per-sample y for a large range, for statistical pins only: the
        integrand in the batched floating-point form (Integrand.evaluate_many)
        in long double and in double; points where the two disagree by more
        than 1e-3 relative, or are not finite, are evaluated exactly (the
        long-double value is then accurate to about 1e-3/2^11 relative).
        Returns (y, number of exactly re-evaluated points)."""
        ys = []
        n_exact = 0
        for lo in range(first, first + count, chunk):
            cnt = min(chunk, first + count - lo)
            p = self.points(lo, cnt, seed)
            I64, _ = self.integrand.evaluate_many(p["z"])
            IL, _ = self.integrand.evaluate_many(p["z"], np.longdouble)
            I = IL.astype(np.float64)
            bad = ~np.isfinite(I64) | ~np.isfinite(I) | (np.abs(I64 - I) > 1e-3 * np.abs(I))
            for k in np.nonzero(bad)[0]:
                I[k] = self.integrand.evaluate(p["z"][k])[0]
            n_exact += int(bad.sum())
            ys.append(weight_many(I, p["log2g"]))
        return np.concatenate(ys), n_exact


def summarize(y, mult=1):
    y = np.asarray(y, dtype=np.float64)
    N = len(y)
    sy = math.fsum(y)
    sy2 = math.fsum(y * y)
    mean = sy / N
    var = sy2 / (N * N) - sy * sy / (N * N * N)
    sig = math.sqrt(max(var, 0.0))
    return dict(mean=mean, sigma1=sig, value=mult * mean, sigma=mult * sig, n=N,
                sum_y=sy, sum_y2=sy2, mean_abs=math.fsum(np.abs(y)) / N)


def integrate(n_loops, n_samples, seed=0, graph_ids=None):
    gs = enumerate_graphs(n_loops)
    ids = range(len(gs)) if graph_ids is None else graph_ids
    total = 0.0
    var = 0.0
    per = []
    for gi in ids:
        o = GraphOracle(gs[gi], gi)
        r = summarize(o.samples(0, n_samples, seed)["y"], gs[gi].mult)
        per.append(r)
        total += r["value"]
        var += r["sigma"] ** 2
    return total, math.sqrt(var), per
