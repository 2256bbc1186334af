"""Python binding of libae (argument marshalling only).

Every computation runs in libae.so: graph enumeration, forests and the
integrand compiler in its host C++ code, sampling, integrand evaluation and
reductions in its sm_103a kernels.  This module loads the library, converts
arguments and raises on error codes; it holds no arithmetic of the method.
Importing fails loudly if the library cannot be built or loaded.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

AE_ERRORS = {-1: "AE_ERR_ARG", -2: "AE_ERR_CUDA", -3: "AE_ERR_OOM", -4: "AE_ERR_TIMEOUT",
             -5: "AE_ERR_NONFINITE", -6: "AE_ERR_STATE", -7: "AE_ERR_NODEV"}


class AeOpts(ctypes.Structure):
    _fields_ = [("C2", ctypes.c_double), ("C3", ctypes.c_double), ("C4", ctypes.c_double),
                ("D", ctypes.c_double), ("C_subI", ctypes.c_double), ("C_subSE", ctypes.c_double),
                ("C_subO", ctypes.c_double), ("C_bigZ", ctypes.c_double), ("C_bigF", ctypes.c_double),
                ("C_add", ctypes.c_double), ("deg_max", ctypes.c_double), ("dd_tol", ctypes.c_double),
                ("block_size", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("rng", ctypes.c_int), ("grid_ctas", ctypes.c_int)]


class AeGraphMeta(ctypes.Structure):
    _fields_ = [("loops", ctypes.c_int), ("M", ctypes.c_int), ("mult", ctypes.c_int),
                ("klass", ctypes.c_int * 3), ("word", ctypes.c_int * 11),
                ("n_subgraphs", ctypes.c_int), ("n_terms", ctypes.c_int),
                ("tape_len", ctypes.c_int), ("nslots", ctypes.c_int),
                ("n_monomials", ctypes.c_int), ("flops", ctypes.c_double), ("canonical_id", ctypes.c_int),
                ("bound_depth", ctypes.c_int), ("flops_bound", ctypes.c_double), ("flops_dd", ctypes.c_double)]


class AeRunGraph(ctypes.Structure):
    _fields_ = [("next", ctypes.c_uint64), ("n", ctypes.c_uint64), ("n_dd", ctypes.c_uint64),
                ("n_zero", ctypes.c_uint64), ("sum_y", ctypes.c_double * 2), ("sum_y2", ctypes.c_double * 2),
                ("sum_abs", ctypes.c_double * 2), ("max_y2", ctypes.c_double)]


class AeTrainReport(ctypes.Structure):
    _fields_ = [("loss_initial", ctypes.c_double), ("loss_final", ctypes.c_double), ("steps", ctypes.c_int),
                ("n_train", ctypes.c_uint64), ("seconds", ctypes.c_double)]


class AeGraphResult(ctypes.Structure):
    _fields_ = [("value", ctypes.c_double), ("sigma", ctypes.c_double), ("mean", ctypes.c_double),
                ("sigma1", ctypes.c_double), ("mean_abs", ctypes.c_double),
                ("sum_y", ctypes.c_double), ("sum_y2", ctypes.c_double), ("max_y2", ctypes.c_double),
                ("n", ctypes.c_uint64), ("n_dd", ctypes.c_uint64), ("n_nonfinite", ctypes.c_uint64),
                ("seconds", ctypes.c_double), ("launches", ctypes.c_uint64),
                ("kernel_seconds", ctypes.c_double), ("d2h_bytes", ctypes.c_uint64),
                ("h2d_bytes", ctypes.c_uint64), ("sigma_up", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load (building first if needed) libae.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        dp = P(ctypes.c_double)
        L.ae_default_opts.argtypes = [P(AeOpts)]
        L.ae_calc1_opts.argtypes = [P(AeOpts)]
        L.ae_create.argtypes = [P(vp), ctypes.c_int, P(AeOpts)]
        L.ae_destroy.argtypes = [vp]
        L.ae_last_error.argtypes = [vp]
        L.ae_last_error.restype = ctypes.c_char_p
        L.ae_load_graphs.argtypes = [vp, ctypes.c_int, P(ctypes.c_int)]
        L.ae_seeded_subset.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64, P(ctypes.c_int)]
        L.ae_load_graph_subset.argtypes = [vp, ctypes.c_int, P(ctypes.c_int), ctypes.c_int, P(ctypes.c_int)]
        L.ae_graph_info.argtypes = [vp, ctypes.c_int, P(AeGraphMeta)]
        L.ae_integrate.argtypes = [vp, P(ctypes.c_int), ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                   dp, dp, P(AeGraphResult)]
        L.ae_integrate_batched.argtypes = [vp, P(ctypes.c_int), ctypes.c_int, P(ctypes.c_uint64),
                                           ctypes.c_uint64, dp, dp, P(AeGraphResult)]
        L.ae_integrate_range.argtypes = [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                         P(AeGraphResult)]
        L.ae_integrate_adaptive.argtypes = [vp, P(ctypes.c_int), ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_uint64, dp, dp,
                                            P(AeGraphResult)]
        L.ae_schedule_probabilities.argtypes = [dp, P(ctypes.c_uint64), dp, ctypes.c_int, ctypes.c_double, dp]
        L.ae_combine_runs.argtypes = [dp, dp, dp, dp, ctypes.c_int, dp, dp, dp, dp]
        L.ae_allocate.argtypes = [vp, P(ctypes.c_int), ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                  ctypes.c_uint64, ctypes.c_int, P(ctypes.c_uint64), dp]
        L.ae_train_proposal.argtypes = [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, P(AeTrainReport)]
        L.ae_set_proposal.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.ae_refine_proposal.argtypes = [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                         ctypes.c_double, P(AeTrainReport)]
        L.ae_set_accept_floor.argtypes = [vp, ctypes.c_int, ctypes.c_double]
        L.ae_set_train_cost_ratio.argtypes = [vp, ctypes.c_double]
        L.ae_proposal_eval.argtypes = [vp, ctypes.c_int, P(ctypes.c_float), dp, dp, P(ctypes.c_uint8),
                                       P(ctypes.c_float), dp, ctypes.c_uint64, dp, P(ctypes.c_float), dp, dp]
        L.ae_proposal_nparams.restype = ctypes.c_int
        L.ae_accept_widths.argtypes = [dp, ctypes.c_int, dp]
        L.ae_graph_classes.argtypes = [ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int), ctypes.c_int,
                                       P(ctypes.c_int)]
        L.ae_set_accept_width.argtypes = [vp, ctypes.c_int, ctypes.c_double]
        L.ae_proposal_export.argtypes = [vp, ctypes.c_int, P(ctypes.c_float), P(ctypes.c_float), dp]
        L.ae_run_reset.argtypes = [vp, ctypes.c_uint64]
        L.ae_run_step.argtypes = [vp, P(ctypes.c_int), ctypes.c_int, P(ctypes.c_uint64), P(AeGraphResult)]
        L.ae_run_add.argtypes = [vp, ctypes.c_int, P(AeGraphResult), ctypes.c_uint64]
        L.ae_run_get.argtypes = [vp, P(AeRunGraph), ctypes.c_int, P(ctypes.c_uint64)]
        L.ae_run_merge.argtypes = [vp, P(AeRunGraph), ctypes.c_int]
        L.ae_run_estimate.argtypes = [vp, dp, dp, dp, P(AeGraphResult)]
        L.ae_checkpoint.argtypes = [vp, ctypes.c_char_p]
        L.ae_resume.argtypes = [vp, ctypes.c_char_p]
        L.aetest_stage_timeout.argtypes = [vp, ctypes.c_int, ctypes.c_longlong]
        L.ae_integrate_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, P(AeGraphResult)]
        L.ae_eval_samples.argtypes = [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                      dp, dp, dp, dp, dp, dp]
        L.ae_eval_samples_dd.argtypes = [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                         dp, dp, dp, dp]
        L.ae_philox.argtypes = [vp, P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32), ctypes.c_size_t]
        L.ae_density_tables.argtypes = [vp, ctypes.c_int, dp, dp]
        L.ae_fp64_peak.argtypes = [vp, dp]
        L.ae_subgraphs.argtypes = [vp, ctypes.c_int, P(ctypes.c_int), ctypes.c_int, P(ctypes.c_int)]
        L.ae_terms.argtypes = [vp, ctypes.c_int, P(ctypes.c_int), ctypes.c_int, P(ctypes.c_int)]
        L.aetest_tape_replay.argtypes = [vp, ctypes.c_int, dp, ctypes.c_size_t, dp, dp, dp]
        L.aetest_fast_elem.argtypes = [vp, dp, dp, ctypes.c_size_t, dp]
        _lib = L
    return _lib


def _ptr(a, ct=ctypes.c_double):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def schedule_probabilities(sigma, N, t, p_floor=0.0):
    """Host: the paper's optimal sampling probabilities (ae_schedule_probabilities)."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    N = np.ascontiguousarray(N, dtype=np.uint64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    p = np.empty(len(sigma))
    rc = lib().ae_schedule_probabilities(_ptr(sigma), _ptr(N, ctypes.c_uint64), _ptr(t), len(sigma),
                                         ctypes.c_double(p_floor), _ptr(p))
    if rc != 0:
        raise AeError("ae_schedule_probabilities: AE_ERR_ARG")
    return p


def combine_runs(v1, s1, v2, s2):
    """Host: two calculations combined graph by graph, then summed
    (ae_combine_runs).  Returns (v, s, total, total_sigma)."""
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (v1, s1, v2, s2)]
    n = len(a[0])
    v = np.empty(n); s = np.empty(n)
    tot = ctypes.c_double(); ts = ctypes.c_double()
    rc = lib().ae_combine_runs(_ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(a[3]), n, _ptr(v), _ptr(s),
                               ctypes.byref(tot), ctypes.byref(ts))
    if rc != 0:
        raise AeError("ae_combine_runs: AE_ERR_ARG")
    return v, s, tot.value, ts.value


def accept_widths(sigma_down):
    """Host: widths of the paper's acceptance test (ae_accept_widths)."""
    sig = np.ascontiguousarray(sigma_down, dtype=np.float64)
    w = np.empty(len(sig))
    if lib().ae_accept_widths(_ptr(sig), len(sig), _ptr(w)) != 0:
        raise AeError("ae_accept_widths: AE_ERR_ARG")
    return w


def graph_classes(loops):
    """(klass [n, 3], mult [n]) of the canonical list of `loops` loops."""
    n = ctypes.c_int()
    if lib().ae_graph_classes(int(loops), None, None, 0, ctypes.byref(n)) != 0:
        raise AeError("ae_graph_classes: AE_ERR_ARG")
    k = np.empty((n.value, 3), dtype=np.int32)
    m = np.empty(n.value, dtype=np.int32)
    if lib().ae_graph_classes(int(loops), _ptr(k, ctypes.c_int), _ptr(m, ctypes.c_int), n.value,
                              ctypes.byref(n)) != 0:
        raise AeError("ae_graph_classes: AE_ERR_ARG")
    return k, m


def seeded_subset(n_total, k, seed=0):
    """k of n_total indices chosen by the library's Philox-driven shuffle."""
    out = np.empty(k, dtype=np.int32)
    if lib().ae_seeded_subset(int(n_total), int(k), int(seed), _ptr(out, ctypes.c_int)) != 0:
        raise AeError("AE_ERR_ARG: bad subset arguments")
    return out.tolist()


def default_opts():
    o = AeOpts()
    lib().ae_default_opts(ctypes.byref(o))
    return o


def calc1_opts():
    """The paper's Calc 1 settings: MRG32k3a, C3 = C4 = 0.035."""
    o = AeOpts()
    lib().ae_calc1_opts(ctypes.byref(o))
    return o


class AeError(RuntimeError):
    pass


class Context:
    """One libae context.  device=-1 gives a host-only context."""

    def __init__(self, device=0, opts=None):
        self._h = ctypes.c_void_p()
        o = opts if opts is not None else default_opts()
        self._check(lib().ae_create(ctypes.byref(self._h), device, ctypes.byref(o)))
        self.device = device
        self.n_graphs = 0

    def _check(self, rc):
        if rc != 0:
            msg = lib().ae_last_error(self._h).decode() if self._h else ""
            raise AeError("%s: %s" % (AE_ERRORS.get(rc, rc), msg))

    def close(self):
        if self._h:
            lib().ae_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_graphs(self, loops):
        n = ctypes.c_int()
        self._check(lib().ae_load_graphs(self._h, loops, ctypes.byref(n)))
        self.n_graphs = n.value
        return n.value

    def load_graph_subset(self, loops, canonical_ids):
        ids = np.ascontiguousarray(canonical_ids, dtype=np.int32)
        n = ctypes.c_int()
        self._check(lib().ae_load_graph_subset(self._h, loops, _ptr(ids, ctypes.c_int), len(ids), ctypes.byref(n)))
        self.n_graphs = n.value
        return n.value

    def graph_info(self, gid):
        m = AeGraphMeta()
        self._check(lib().ae_graph_info(self._h, gid, ctypes.byref(m)))
        d = {k: getattr(m, k) for k, _ in m._fields_}
        d["klass"] = tuple(m.klass)
        d["word"] = tuple(m.word[:2 * m.loops + 1])
        return d

    def integrate(self, ids, n_samples, seed=0):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        v = ctypes.c_double()
        s = ctypes.c_double()
        res = (AeGraphResult * len(ids))()
        self._check(lib().ae_integrate(self._h, _ptr(ids, ctypes.c_int), len(ids), int(n_samples), int(seed),
                                       ctypes.byref(v), ctypes.byref(s), res))
        return v.value, s.value, [r.as_dict() for r in res]

    def integrate_batched(self, ids, n_samples, seed=0):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        ns = np.ascontiguousarray(n_samples, dtype=np.uint64)
        v = ctypes.c_double()
        s = ctypes.c_double()
        res = (AeGraphResult * len(ids))()
        self._check(lib().ae_integrate_batched(self._h, _ptr(ids, ctypes.c_int), len(ids),
                                               _ptr(ns, ctypes.c_uint64), int(seed),
                                               ctypes.byref(v), ctypes.byref(s), res))
        return v.value, s.value, [r.as_dict() for r in res]

    def integrate_adaptive(self, ids, block_size, n_rounds, blocks_per_round, p_floor=0.1, seed=0):
        """The paper's controller: blocks drawn with the optimal probabilities."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        v = ctypes.c_double()
        s = ctypes.c_double()
        res = (AeGraphResult * len(ids))()
        self._check(lib().ae_integrate_adaptive(self._h, _ptr(ids, ctypes.c_int), len(ids), int(block_size),
                                                int(n_rounds), int(blocks_per_round), float(p_floor), int(seed),
                                                ctypes.byref(v), ctypes.byref(s), res))
        return v.value, s.value, [r.as_dict() for r in res]

    def integrate_range(self, gid, first, count, seed=0):
        r = AeGraphResult()
        self._check(lib().ae_integrate_range(self._h, gid, int(first), int(count), int(seed), ctypes.byref(r)))
        return r.as_dict()

    def allocate(self, ids, n_pilot, n_total, seed=0, mode=0):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        out = np.empty(len(ids), dtype=np.uint64)
        sig = np.empty(len(ids))
        self._check(lib().ae_allocate(self._h, _ptr(ids, ctypes.c_int), len(ids), int(n_pilot), int(n_total),
                                      int(seed), int(mode), _ptr(out, ctypes.c_uint64), _ptr(sig)))
        return out, sig

    def train_proposal(self, gid, n_train, seed=0, steps=200, lr=3e-3, beta=0.1):
        r = AeTrainReport()
        self._check(lib().ae_train_proposal(self._h, gid, int(n_train), int(seed), int(steps), float(lr),
                                            float(beta), ctypes.byref(r)))
        return {k: getattr(r, k) for k, _ in r._fields_}

    def refine_proposal(self, gid, n_train, seed=0, steps=100, lr=1e-3):
        """Continue training the graph's proposal on samples of its current mixture."""
        r = AeTrainReport()
        self._check(lib().ae_refine_proposal(self._h, gid, int(n_train), int(seed), int(steps), float(lr),
                                             ctypes.byref(r)))
        return {k: getattr(r, k) for k, _ in r._fields_}

    def set_proposal(self, gid, mode, beta=0.1):
        self._check(lib().ae_set_proposal(self._h, gid, int(mode), float(beta)))

    def set_train_cost_ratio(self, ratio):
        """Cost-aware training weights: |y| / sqrt(1 + ratio) for samples that
        need double-double (0: plain |y|)."""
        self._check(lib().ae_set_train_cost_ratio(self._h, float(ratio)))

    def set_accept_floor(self, gid, yfloor):
        """Absolute floor on |y| in the acceptance test of the graph's FP64
        values (kept when bound <= dd_tol * max(|y|, yfloor))."""
        self._check(lib().ae_set_accept_floor(self._h, gid, float(yfloor)))

    def set_accept_width(self, gid, width):
        """The paper's acceptance test for the graph: keep a value when its
        certified interval on y is at most `width` wide (0: relative test)."""
        self._check(lib().ae_set_accept_width(self._h, gid, float(width)))

    def proposal_export(self, gid):
        """(FP32 master weights, network outputs o(T) [2^M, 16], beta) of the
        graph's trained proposal."""
        M = self.graph_info(gid)["M"]
        p = np.empty(lib().ae_proposal_nparams(), dtype=np.float32)
        o = np.empty((1 << M) * 16, dtype=np.float32)
        b = ctypes.c_double()
        self._check(lib().ae_proposal_export(self._h, gid, _ptr(p, ctypes.c_float), _ptr(o, ctypes.c_float),
                                             ctypes.byref(b)))
        return p, o.reshape(1 << M, 16), b.value

    # ------------------------------------------------------- run state --
    def run_reset(self, seed):
        self._check(lib().ae_run_reset(self._h, int(seed)))

    def run_step(self, ids, n_samples):
        """One batched block of the run; returns this block's per-graph results."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        ns = np.ascontiguousarray(n_samples, dtype=np.uint64)
        res = (AeGraphResult * len(ids))()
        self._check(lib().ae_run_step(self._h, _ptr(ids, ctypes.c_int), len(ids), _ptr(ns, ctypes.c_uint64), res))
        return [r.as_dict() for r in res]

    def run_add(self, gid, result, count):
        r = AeGraphResult()
        for k, _ in AeGraphResult._fields_:
            if k in result:
                setattr(r, k, result[k])
        self._check(lib().ae_run_add(self._h, gid, ctypes.byref(r), int(count)))

    def run_get(self):
        """(array of AeRunGraph, one per loaded graph; seed)."""
        arr = (AeRunGraph * self.n_graphs)()
        seed = ctypes.c_uint64()
        self._check(lib().ae_run_get(self._h, arr, self.n_graphs, ctypes.byref(seed)))
        return arr, seed.value

    def run_merge(self, other):
        self._check(lib().ae_run_merge(self._h, other, len(other)))

    def run_estimate(self):
        """(value, sigma_down, sigma_up, per-graph results) of the run."""
        v = ctypes.c_double(); s = ctypes.c_double(); u = ctypes.c_double()
        res = (AeGraphResult * self.n_graphs)()
        self._check(lib().ae_run_estimate(self._h, ctypes.byref(v), ctypes.byref(s), ctypes.byref(u), res))
        return v.value, s.value, u.value, [r.as_dict() for r in res]

    def checkpoint(self, path):
        self._check(lib().ae_checkpoint(self._h, os.fsencode(path)))

    def resume(self, path):
        self._check(lib().ae_resume(self._h, os.fsencode(path)))

    def test_stage_timeout(self, gid, wait_cycles):
        """Test hook: make the bounded tape-staging wait run out (returns the
        error the integration would raise)."""
        self._check(lib().aetest_stage_timeout(self._h, gid, int(wait_cycles)))

    def proposal_eval(self, M, params, deg, wplain, order, lt, w):
        params = np.ascontiguousarray(params, dtype=np.float32)
        deg = np.ascontiguousarray(deg, dtype=np.float64)
        wplain = np.ascontiguousarray(wplain, dtype=np.float64)
        order = np.ascontiguousarray(order, dtype=np.uint8)
        lt = np.ascontiguousarray(lt, dtype=np.float32)
        w = np.ascontiguousarray(w, dtype=np.float64)
        n = w.shape[0]
        loss = ctypes.c_double()
        grad = np.empty(lib().ae_proposal_nparams(), dtype=np.float32)
        lp2 = np.empty((1 << M) * 16)
        dt = np.empty(1 << M)
        self._check(lib().ae_proposal_eval(self._h, M, _ptr(params, ctypes.c_float), _ptr(deg), _ptr(wplain),
                                           _ptr(order, ctypes.c_uint8), _ptr(lt, ctypes.c_float), _ptr(w), n,
                                           ctypes.byref(loss), _ptr(grad, ctypes.c_float), _ptr(lp2), _ptr(dt)))
        return loss.value, grad, lp2.reshape(1 << M, 16), dt

    def integrate_noalloc(self, gid, n_samples, seed=0):
        """One graph through the entry point that allocates no device memory
        (fixed static scratch; n_samples <= 524288)."""
        r = AeGraphResult()
        self._check(lib().ae_integrate_noalloc(self._h, gid, int(n_samples), int(seed), ctypes.byref(r)))
        return r.as_dict()

    def eval_samples(self, gid, first, count, seed=0):
        M = self.graph_info(gid)["M"]
        z = np.empty((count, M))
        lg = np.empty(count); I = np.empty(count); K = np.empty(count); y = np.empty(count)
        E = np.empty(count)
        self._check(lib().ae_eval_samples(self._h, gid, first, count, seed, _ptr(z), _ptr(lg),
                                          _ptr(I), _ptr(K), _ptr(y), _ptr(E)))
        return dict(z=z, log2g=lg, I=I, K=K, y=y, E=E)

    def eval_samples_dd(self, gid, first, count, seed=0):
        I = np.empty(count); K = np.empty(count); y = np.empty(count); E = np.empty(count)
        self._check(lib().ae_eval_samples_dd(self._h, gid, first, count, seed, _ptr(I), _ptr(K), _ptr(y),
                                             _ptr(E)))
        return dict(I=I, K=K, y=y, E=E)

    def philox(self, ctr, key):
        ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
        key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
        out = np.empty_like(ctr)
        self._check(lib().ae_philox(self._h, _ptr(ctr, ctypes.c_uint32), _ptr(key, ctypes.c_uint32),
                                    _ptr(out, ctypes.c_uint32), ctr.shape[0]))
        return out

    def fp64_peak(self):
        t = ctypes.c_double()
        self._check(lib().ae_fp64_peak(self._h, ctypes.byref(t)))
        return t.value

    def density_tables(self, gid):
        M = self.graph_info(gid)["M"]
        deg = np.empty(3 << M)
        phi = np.empty(3 << M)
        self._check(lib().ae_density_tables(self._h, gid, _ptr(deg), _ptr(phi)))
        return deg.reshape(3, 1 << M), phi.reshape(3, 1 << M)

    def _intlist(self, fn, gid):
        n = ctypes.c_int()
        self._check(fn(self._h, gid, None, 0, ctypes.byref(n)))
        buf = np.empty(max(n.value, 1), dtype=np.int32)
        self._check(fn(self._h, gid, _ptr(buf, ctypes.c_int), n.value, ctypes.byref(n)))
        return buf[:n.value].tolist()

    def subgraphs(self, gid):
        v = self._intlist(lib().ae_subgraphs, gid)
        return [tuple(v[i:i + 3]) for i in range(0, len(v), 3)]

    def terms(self, gid):
        v = self._intlist(lib().ae_terms, gid)
        out, i = [], 0
        while i < len(v):
            sign, cnt = v[i], v[i + 1]
            els = [tuple(v[i + 2 + 3 * k:i + 5 + 3 * k]) for k in range(cnt)]
            out.append((sign, els))
            i += 2 + 3 * cnt
        return out

    def fast_elem(self, x, y):
        """Test hook: (fexp2 x, exp2 x, flog2 y, log2 y) computed on the device."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        out = np.empty((len(x), 4))
        self._check(lib().aetest_fast_elem(self._h, _ptr(x), _ptr(y), len(x), _ptr(out)))
        return out

    def tape_replay(self, gid, z, bound=False):
        """Test hook: host replay of the compiled tape at points z: (I, K),
        and the rounding-error bound E of I with bound=True."""
        z = np.ascontiguousarray(z, dtype=np.float64)
        I = np.empty(z.shape[0]); K = np.empty(z.shape[0]); E = np.empty(z.shape[0])
        self._check(lib().aetest_tape_replay(self._h, gid, _ptr(z), z.shape[0], _ptr(I), _ptr(K), _ptr(E)))
        return (I, K, E) if bound else (I, K)
