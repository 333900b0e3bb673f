"""Shared helpers of the GPU tests: run a workload through the C ABI and
compare endpoint sets keyed by electron id."""
import numpy as np

from paper_2509_15377_gb300 import avalanche as A

# FP64 parity tolerance (relative to the larger of |reference| and a scale
# that is natural for the quantity: the transport is FP64 on both sides and
# differs only by rounding order, FMA contraction and 1-2 ulp differences of
# log/sqrt/sin/cos between CUDA's and the C library's implementations).
RTOL_FP64 = 1e-9


def run_gpu(av: "A.Avalanche", w, seed, t_max=None, coll_limit=None, precision=A.GT_FP64,
            mode=A.GT_BATCHED, capacity=None, prim=None, allow=(A.GT_OK,), **kw):
    prim = prim if prim is not None else w.primaries
    p = av.primaries_device(prim)
    opt = A.RunOptions(seed=seed, t_max=w.t_max if t_max is None else t_max,
                       coll_limit=w.coll_limit if coll_limit is None else coll_limit,
                       precision=precision, mode=mode, **kw)
    cap = capacity or max(64, 8 * prim.n)
    st = av.run(p, opt, capacity=cap, allow=allow)
    out = av.fetch(st["n_endpoints"])
    return st, out


def by_uid(o):
    idx = np.argsort(o["uid"], kind="stable")
    return {k: (v[idx] if (hasattr(v, "__len__") and len(v) == len(o["uid"]) and k not in
                           ("electrons", "tallies")) else v) for k, v in o.items()}


def assert_same_electrons(gpu, ref, scale_pos, scale_t, scale_e=1.0, rtol=RTOL_FP64):
    """Every electron (by id) has the same start and end within rtol, the
    same status and the same flight count."""
    g, r = by_uid(gpu), by_uid(ref)
    assert len(g["uid"]) == len(r["uid"]), (len(g["uid"]), len(r["uid"]))
    assert np.array_equal(g["uid"], r["uid"])
    assert np.array_equal(g["status"], r["status"])
    assert np.array_equal(g["aval"], r["aval"])
    assert np.array_equal(g["n_flight"].astype(np.int64), r["n_flight"].astype(np.int64))
    for keys, sc in ((("x0", "y0", "z0", "x1", "y1", "z1"), scale_pos), (("t0", "t1"), scale_t),
                     (("e0", "e1"), scale_e)):
        for k in keys:
            err = np.abs(g[k] - r[k])
            lim = rtol * np.maximum(np.abs(r[k]), sc)
            bad = np.nonzero(err > lim)[0]
            assert len(bad) == 0, (k, bad[:5], g[k][bad[:5]], r[k][bad[:5]])


def two_sample_ks(a, b):
    """Two-sample Kolmogorov-Smirnov statistic and asymptotic p-value."""
    from scipy import stats
    return stats.ks_2samp(a, b)


def ks_statistic(a, b):
    """Two-sample Kolmogorov-Smirnov statistic sup |F_a - F_b|."""
    a, b = np.sort(a), np.sort(b)
    x = np.concatenate([a, b])
    fa = np.searchsorted(a, x, side="right") / len(a)
    fb = np.searchsorted(b, x, side="right") / len(b)
    return float(np.abs(fa - fb).max())


def paired_avalanche_ks(va, ga, vb, gb, n_avalanches, n_perm=2000, seed=0):
    """p-value of the KS statistic between two electron-level samples of the
    same avalanches (values va with avalanche numbers ga, and vb, gb), from
    a permutation of whole avalanches: under the hypothesis that both runs
    draw each avalanche from one law, swapping avalanche i's electrons
    between the runs leaves the joint law unchanged.  The electrons of an
    avalanche are correlated, so the asymptotic p-value of a plain KS test
    on electrons is too small; swapping avalanches keeps that correlation."""
    rng = np.random.default_rng(seed)
    A = [va[ga == i] for i in range(n_avalanches)]
    B = [vb[gb == i] for i in range(n_avalanches)]
    d0 = ks_statistic(va, vb)
    hits = 0
    for _ in range(n_perm):
        sw = rng.random(n_avalanches) < 0.5
        pa = np.concatenate([B[i] if sw[i] else A[i] for i in range(n_avalanches)])
        pb = np.concatenate([A[i] if sw[i] else B[i] for i in range(n_avalanches)])
        hits += ks_statistic(pa, pb) >= d0
    return (1 + hits) / (1 + n_perm)


def ratio_se(num, den, n_boot=2000, seed=0):
    """Bootstrap standard error over avalanches of sum(num) / sum(den), with
    num, den per avalanche (a fraction of the electrons of a run, whose
    electrons are correlated within an avalanche)."""
    rng = np.random.default_rng(seed)
    num, den = np.asarray(num, dtype=float), np.asarray(den, dtype=float)
    idx = rng.integers(0, len(num), size=(n_boot, len(num)))
    r = num[idx].sum(axis=1) / np.maximum(den[idx].sum(axis=1), 1e-300)
    return float(r.std(ddof=1))
