"""CPU oracle values for large per-sample comparisons, one graph per worker
process (run in a 'spawn' pool; imports only oracle/).

The oracle's integrand (Eq. eq_integrand_final and the forest terms of
Sec. II) is evaluated in its batched floating-point form twice, in long
double and in double.  The long-double value is the comparison value; the
difference between the two, delta, is the oracle's own error scale (the
long-double error is usually a small fraction of it), and 2^-40 times the oracle's
magnitude sum K covers samples where the two agree by accident.  That
estimate is a heuristic: where the graph functions (U, V, the flows) lose
digits in the unpivoted elimination, one precision can be accurate and the
other not, so a comparison that fails against it is decided by the exact
rational value (exact_values).  The samples with the largest error scale
relative to |I| are also evaluated exactly (Integrand.evaluate)."""
import numpy as np


def _oracle(loops, gi, tables_path=None):
    """The oracle of graph gi; its coefficient tables rebuilt, or read from a
    file written by tests/golden/make_oracle_tables.py."""
    from oracle.estimate import GraphOracle
    from oracle.graphs import enumerate_graphs
    tables = None
    if tables_path:
        import gzip
        import json
        from oracle.integrand import Integrand
        with gzip.open(tables_path, "rt") as f:
            rec = json.load(f)
        assert rec["loops"] == loops and rec["graph"] == gi
        tables = Integrand.tables_from_records(rec["tables"])
    return GraphOracle(enumerate_graphs(loops)[gi], gi, tables=tables)


def graph_values(args):
    """args = (loops, graph id, first, count, seed, n_exact[, tables path]).
    Returns a dict: first, z, log2g (the oracle sampler's), I (long double,
    rounded to double), scale (1e-10 |I| + delta + 2^-40 K: the oracle's
    uncertainty on I), exact_idx / exact_I (the n_exact samples of largest
    scale / |I|, indices from `first`)."""
    loops, gi, first, count, seed, n_exact = args[:6]
    o = _oracle(loops, gi, args[6] if len(args) > 6 else None)
    p = o.points(first, count, seed)
    z = p["z"]
    I = np.empty(count)
    scale = np.empty(count)
    step = 1 << 16
    for lo in range(0, count, step):
        hi = min(count, lo + step)
        IL, KL = o.integrand.evaluate_many(z[lo:hi], np.longdouble)
        ID, _ = o.integrand.evaluate_many(z[lo:hi])
        with np.errstate(invalid="ignore", over="ignore"):
            delta = np.abs(ID - IL).astype(np.float64)
            I[lo:hi] = IL.astype(np.float64)
            scale[lo:hi] = 1e-10 * np.abs(I[lo:hi]) + delta + 2.0 ** -40 * KL.astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        rel = np.where(np.isfinite(scale) & np.isfinite(I), scale / np.abs(I), np.inf)
    idx = np.argsort(-rel, kind="stable")[:n_exact]
    exact = np.array([float(o.integrand.evaluate(z[k])[0]) for k in idx])
    return dict(graph=gi, first=first, z=z, log2g=p["log2g"], I=I, scale=scale, exact_idx=idx, exact_I=exact)


def exact_values(args):
    """args = (loops, graph id, z rows[, tables path]).  The oracle's exact
    rational I at each row, rounded once to double: the referee where the
    batched form's uncertainty estimate does not cover a sample."""
    loops, gi, zs = args[:3]
    o = _oracle(loops, gi, args[3] if len(args) > 3 else None)
    return np.array([float(o.integrand.evaluate(z)[0]) for z in zs])
