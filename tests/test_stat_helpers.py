"""The avalanche-level statistics of the GPU tests, checked on synthetic
clustered samples whose law is known (no GPU, no oracle).

Electrons of one avalanche share its history, so an electron-level sample
is clustered.  The helpers must give calibrated p-values and standard
errors for such samples, and still see a real difference."""
import math

import numpy as np

from tests.gpu_helpers import ks_statistic, paired_avalanche_ks, ratio_se


def _clustered(rng, n_aval, shift=0.0):
    """Values clustered by avalanche: each avalanche draws a random offset
    and a random size (geometric), its electrons scatter around it."""
    sizes = rng.geometric(0.2, size=n_aval)
    groups = np.repeat(np.arange(n_aval), sizes)
    centre = rng.normal(0.0, 1.0, n_aval)
    vals = centre[groups] + 0.2 * rng.normal(size=len(groups)) + shift
    return vals, groups


def test_ks_statistic_matches_scipy():
    from scipy import stats
    rng = np.random.default_rng(1)
    a, b = rng.normal(size=300), rng.normal(0.3, 1.0, size=200)
    assert abs(ks_statistic(a, b) - stats.ks_2samp(a, b).statistic) < 1e-12


def test_paired_avalanche_ks_is_calibrated_on_clustered_samples():
    """Same law on both sides: the permutation p-value is roughly uniform
    (few below 0.05), while the plain electron-level KS p-value of scipy,
    which assumes independent electrons, is far too often tiny."""
    from scipy import stats
    rng = np.random.default_rng(2)
    n = 48
    p_perm, p_plain = [], []
    for _ in range(40):
        va, ga = _clustered(rng, n)
        vb, gb = _clustered(rng, n)
        p_perm.append(paired_avalanche_ks(va, ga, vb, gb, n, n_perm=200,
                                          seed=int(rng.integers(1 << 30))))
        p_plain.append(stats.ks_2samp(va, vb).pvalue)
    p_perm, p_plain = np.array(p_perm), np.array(p_plain)
    assert (p_perm < 0.05).mean() <= 0.15
    assert (p_plain < 0.05).mean() >= 0.5


def test_paired_avalanche_ks_sees_a_shift():
    rng = np.random.default_rng(3)
    n = 64
    va, ga = _clustered(rng, n)
    vb, gb = _clustered(rng, n, shift=1.5)
    assert paired_avalanche_ks(va, ga, vb, gb, n, n_perm=500) < 0.01


def test_ratio_se_matches_the_spread_over_repeats():
    """The bootstrap error of a pooled fraction over clustered avalanches
    agrees with the spread of that fraction over independent repeats."""
    rng = np.random.default_rng(4)
    n = 96
    fr, ses = [], []
    for _ in range(200):
        size = rng.geometric(0.1, size=n)
        p = rng.beta(2.0, 5.0, size=n)  # each avalanche its own fraction
        hit = rng.binomial(size, p)
        fr.append(hit.sum() / size.sum())
        if len(ses) < 20:
            ses.append(ratio_se(hit, size, n_boot=500, seed=len(ses)))
    spread = float(np.std(fr, ddof=1))
    se = float(np.mean(ses))
    assert 0.75 < se / spread < 1.33, (se, spread)
    # a binomial error that ignores the clustering is much too small
    naive = math.sqrt(np.mean(fr) * (1 - np.mean(fr)) / (n / 0.1))
    assert naive < 0.7 * spread
