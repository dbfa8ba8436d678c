"""Pins of the oracle's critical-percolation masks, activation rule and flip.

* Bond percolation at p = 1/2 (the labeling workload): the number of open
  bonds is Binomial(2N, 1/2), and the number of clusters per site approaches
  (3 sqrt3 - 5)/2 (Ziff, Finch & Adamchik 1997) up to O(1/N).
* Activation (Sec. II.A, Eq. 7): bonds between unequal spins are never
  open; among equal-spin bonds the open fraction is T / 2^32 (binomial).
* Flip (Sec. II.D): all sites of a cluster take one state; over clusters the
  new states are uniform on {0..q-1} (chi-square) and independent between
  distinct clusters.
"""
import math

import numpy as np
import pytest
from scipy.stats import chi2

import oracle
import oracle.exact as ex


def test_perc_open_bond_count_binomial():
    H = W = 512
    N = H * W
    for k in (0, 1):
        e, n = oracle.unpack_mask(oracle.perc_mask(H, W, k), N)
        b = int(e.sum()) + int(n.sum())
        assert abs(b - N) < 5 * math.sqrt(2 * N * 0.25)


def test_perc_cluster_density_matches_ziff():
    H = W = 1024
    dens = []
    for k in range(4):
        _, n = oracle.label(oracle.perc_mask(H, W, k), H, W, True)
        dens.append(n / (H * W))
    # finite-size correction on the torus is O(1/N) ~ 1e-6 here; statistical sd ~2e-4
    assert abs(np.mean(dens) - ex.PERC_CLUSTER_DENSITY) < 1e-3


@pytest.mark.parametrize("q,K", [(2, 0.8813735870195429), (4, math.log(3.0)), (3, 0.3)])
def test_activation_rule(q, K):
    L = 128
    T = oracle.threshold(K)
    s = oracle.init_spins(L, q, 77, True)
    m = oracle.activate(L, s, 77, 5, T)
    e, n = oracle.unpack_mask(m, L * L)
    i = np.arange(L * L)
    y, x = i // L, i % L
    eq_e = s == s[y * L + (x + 1) % L]
    eq_n = s == s[((y + 1) % L) * L + x]
    assert not np.any(e[~eq_e]) and not np.any(n[~eq_n])
    n_eq = int(eq_e.sum() + eq_n.sum())
    n_open = int(e.sum() + n.sum())
    p = T / 2 ** 32
    assert abs(n_open - p * n_eq) < 5 * math.sqrt(n_eq * p * (1 - p))


def test_activation_depends_on_sweep_and_seed():
    L = 64
    s = np.zeros(L * L, dtype=np.int8)
    T = oracle.threshold(0.7)
    a = oracle.activate(L, s, 1, 0, T)
    assert not np.array_equal(a, oracle.activate(L, s, 1, 1, T))
    assert not np.array_equal(a, oracle.activate(L, s, 2, 0, T))
    assert np.array_equal(a, oracle.activate(L, s, 1, 0, T))


@pytest.mark.parametrize("q", [2, 3, 5])
def test_flip_uniform_per_cluster_and_constant_on_clusters(q):
    H = W = 256
    mask = oracle.perc_mask(H, W, 4)
    lab, n = oracle.label(mask, H, W, True)
    roots = np.unique(lab)
    counts = np.zeros(q, dtype=np.int64)
    prev = None
    corr = []
    for sweep in range(6):
        s = oracle.flip(lab, q, 31, sweep)
        assert np.array_equal(s, s[lab])                    # one state per cluster
        st = s[roots].astype(np.int64)
        counts += np.bincount(st, minlength=q)
        corr.append(np.corrcoef(st[:-1], st[1:])[0, 1])
        if prev is not None:
            assert not np.array_equal(prev, st)             # fresh draw every sweep
        prev = st
    tot = counts.sum()
    stat = ((counts - tot / q) ** 2 / (tot / q)).sum()
    assert chi2.sf(stat, q - 1) > 1e-4
    assert abs(np.mean(corr)) < 5 / math.sqrt(6 * roots.size)


@pytest.mark.parametrize("q", [2, 3, 7])
def test_hot_start_uniform_and_uncorrelated(q):
    """Hot start (INIT draw per site): every state equally likely, no
    correlation between neighbouring sites, different seeds differ."""
    L = 256
    s = oracle.init_spins(L, q, 123, True).astype(np.int64)
    counts = np.bincount(s, minlength=q)
    stat = ((counts - s.size / q) ** 2 / (s.size / q)).sum()
    assert chi2.sf(stat, q - 1) > 1e-4
    r = np.corrcoef(s[:-1], s[1:])[0, 1]
    assert abs(r) < 5 / math.sqrt(s.size)
    assert not np.array_equal(s, oracle.init_spins(L, q, 124, True))
    assert not np.any(oracle.init_spins(L, q, 123, False))
