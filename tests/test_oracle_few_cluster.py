"""Pins of the oracle's few-cluster update (Sec. III, variant (c)).

The update keeps the SW decomposition (same bonds and clusters as the SW
sweep) and flips only the clusters that hold one of the ell^2 seed sites (one
per block of side L / ell), each with probability p_flip.  Pins, none of
which reuses the oracle's own flip code:

* closed forms: p_flip = 0 leaves every spin alone; with a seed on every site
  (ell = L) and p_flip = 1 every q = 2 spin flips (s -> 1 - s); with no bond
  open (T = 0) every site is its own cluster and its new state follows from
  the (separately pinned) Philox words of its own FLIP draw;
* the seed of block b lies in block b, from the SEED draw's two words, and is
  uniform over the block (chi-square over many sweeps);
* selection: on random chains, components of the bond graph computed by
  scipy either hold a seed and move as one (one common nonzero shift, or none
  at p_flip < 1), or hold none and keep their spins; at p_flip = 1 a
  component changes iff it holds a seed;
* the accepted fraction of selected clusters is p_flip (binomial);
* detailed balance: the chain samples the Potts Boltzmann distribution, so
  4 x 4 averages match exact enumeration (q = 2) and the exact density of
  states (q = 3) within binned error bars.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components
from scipy.stats import chi2

import oracle
import oracle.exact as ex

GOLD = os.path.join(os.path.dirname(__file__), "golden")
KC_ISING = 0.5 * math.log(1.0 + math.sqrt(2.0))
FULL = 1 << 32


def _components(mask, L):
    """Component id of every site of the periodic bond graph (scipy)."""
    N = L * L
    e, n = oracle.unpack_mask(mask, N)
    i = np.arange(N)
    x, y = i % L, i // L
    east = y * L + (x + 1) % L
    north = ((y + 1) % L) * L + x
    src = np.concatenate([i[e == 1], i[n == 1]])
    dst = np.concatenate([east[e == 1], north[n == 1]])
    g = coo_matrix((np.ones(src.size), (src, dst)), shape=(N, N))
    return connected_components(g, directed=False)[1]


def test_no_flip_probability_leaves_spins():
    L, q = 16, 3
    s = oracle.init_spins(L, q, 5, True)
    for ell in (1, 4, 16):
        s2, _, _, _ = oracle.few_sweep(L, q, oracle.threshold(0.9), 0, ell, 5, 3, s)
        assert np.array_equal(s2, s)


def test_seed_everywhere_flips_every_ising_spin():
    L = 32
    s = oracle.init_spins(L, 2, 9, True)
    for T in (0, 1 << 31, FULL):
        s2, _, _, _ = oracle.few_sweep(L, 2, T, FULL, L, 9, 4, s)
        assert np.array_equal(s2, 1 - s)


def test_no_bonds_single_site_clusters_closed_form():
    L, seed, sweep = 12, 77, 6
    for q in (2, 3, 5):
        s = oracle.init_spins(L, q, seed, True)
        s2, _, _, _ = oracle.few_sweep(L, q, 0, FULL, L, seed, sweep, s)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for i in range(L * L):
            w = oracle.philox4x32_10((i, sweep, 0, oracle.TAG_FLIP), key)
            shift = 1 + (w[0] * (q - 1) >> 32)
            assert s2[i] == (s[i] + shift) % q, (q, i)


def test_seed_lies_in_its_block_from_the_seed_draw():
    L, seed = 48, 123
    for ell in (1, 2, 3, 6, 48):
        B = L // ell
        for sweep in (0, 7, 1 << 33):
            for b in range(min(ell * ell, 40)):
                w = oracle.philox4x32_10((b, sweep & 0xFFFFFFFF, sweep >> 32, oracle.TAG_SEED), (seed, 0))
                x = (b % ell) * B + (w[0] * B >> 32)
                y = (b // ell) * B + (w[1] * B >> 32)
                assert oracle.few_seed(L, ell, seed, sweep, b) == y * L + x


def test_seed_uniform_over_block():
    L, ell = 8, 2
    B = L // ell
    counts = np.zeros((ell * ell, B * B))
    for sweep in range(4000):
        for b in range(ell * ell):
            site = oracle.few_seed(L, ell, 1, sweep, b)
            y, x = divmod(site, L)
            assert (y // B, x // B) == divmod(b, ell)
            counts[b, (y % B) * B + x % B] += 1
    for b in range(ell * ell):
        stat = ((counts[b] - 4000 / (B * B)) ** 2 / (4000 / (B * B))).sum()
        assert chi2.sf(stat, B * B - 1) > 1e-4


@pytest.mark.parametrize("q,P", [(2, FULL), (3, FULL), (2, int(0.3 * FULL)), (4, int(0.6 * FULL))])
def test_only_seeded_clusters_move_as_one(q, P):
    L, ell, seed = 24, 3, 31
    T = oracle.threshold(oracle.coupling_K(q, math.log(1 + math.sqrt(q)), 1.0, oracle.CONV_POTTS))
    s = oracle.init_spins(L, q, seed, True)
    n_sel = n_acc = 0
    for sweep in range(30):
        s2, mask, _, obs = oracle.few_sweep(L, q, T, P, ell, seed, sweep, s)
        comp = _components(mask, L)
        seeded = set(comp[oracle.few_seed(L, ell, seed, sweep, b)] for b in range(ell * ell))
        shift = (s2.astype(np.int64) - s) % q
        for c in np.unique(comp):
            sh = np.unique(shift[comp == c])
            assert sh.size == 1, "a cluster split"
            assert np.unique(s[comp == c]).size == 1, "bonds joined unequal spins"
            if c in seeded:
                n_sel += 1
                n_acc += int(sh[0] != 0)
                if P == FULL:
                    assert sh[0] != 0
            else:
                assert sh[0] == 0
        assert np.array_equal(obs, oracle.observables(L, q, s2))
        s = s2
    p = P / FULL
    assert abs(n_acc - p * n_sel) <= 5 * math.sqrt(n_sel * p * (1 - p)) + 1e-9


@pytest.mark.parametrize("ell,p_flip", [(2, 0.5), (1, 0.8)])
def test_ising_4x4_stationary_distribution(ell, p_flip):
    K = oracle.coupling_K(2, KC_ISING, 1.0, oracle.CONV_ISING)
    T = oracle.threshold(K)
    s0 = oracle.init_spins(4, 2, 3, True)
    _, obs = oracle.few_chain(4, 2, T, int(p_flip * FULL), ell, 3, 0, 300_000, s0)
    obs = obs[1000:]
    n_eq, counts = ex.enumerate_potts(4, 4, 2)
    exact = ex.moments_from_states(n_eq, counts, K, 2)
    n = obs[:, 0]
    absM = np.abs(obs[:, 1] - obs[:, 2])
    for series, key in ((n, "n_eq"), (n.astype(np.float64) ** 2, "n_eq2"), (absM, "absM")):
        x = np.asarray(series, dtype=np.float64)
        b = x[: len(x) // 50 * 50].reshape(50, -1).mean(axis=1)
        m, e = b.mean(), b.std(ddof=1) / math.sqrt(50)
        assert abs(m - exact[key]) < 4.5 * e, (key, m, exact[key], e)


def test_potts_q3_4x4_stationary_distribution():
    beta = math.log(1 + math.sqrt(3))
    K = oracle.coupling_K(3, beta, 1.0, oracle.CONV_POTTS)
    s0 = oracle.init_spins(4, 3, 8, True)
    _, obs = oracle.few_chain(4, 3, oracle.threshold(K), int(0.7 * FULL), 2, 8, 0, 300_000, s0)
    obs = obs[1000:]
    g = np.array(json.load(open(os.path.join(GOLD, "potts_dos_4x4.json")))["g"]["3"])
    exact = ex.dos_moments(g, K)
    n = obs[:, 0].astype(np.float64)
    for series, key in ((n, "n_eq"), (n * n, "n_eq2")):
        b = series[: len(series) // 50 * 50].reshape(50, -1).mean(axis=1)
        m, e = b.mean(), b.std(ddof=1) / math.sqrt(50)
        assert abs(m - exact[key]) < 4.5 * e, (key, m, exact[key], e)
    frac = obs[:, 1:].mean(axis=0) / 16.0
    assert np.all(np.abs(frac - 1.0 / 3) < 0.02)


def test_bad_block_grid_is_refused():
    with pytest.raises(ValueError):
        oracle.few_sweep(12, 2, 0, FULL, 5, 1, 0, np.zeros(144, np.int8))
