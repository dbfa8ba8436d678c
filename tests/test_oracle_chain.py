"""Pins of the oracle's whole Swendsen-Wang chain against exact equilibrium results.

The SW dynamics (Sec. II, three steps) must sample the Potts Boltzmann
distribution of Eq. 1.  The oracle's chain is run for many sweeps and its
time averages are compared with exact values, with error bars from binning
(bins much longer than the autocorrelation time):

* 4 x 4 torus, q = 2 at the Ising beta_c: <n_eq>, <n_eq^2>, <|M|> from brute
  force over all 2^16 states, and a chi-square of the n_eq histogram.
* 4 x 4 torus, q = 3 and 4 at their critical couplings: <n_eq>, <n_eq^2> from
  the exact transfer-matrix density of states (tests/golden/potts_dos_4x4.json).
* 16 x 16 and 64 x 64 tori, q = 2 at beta_c: energy and specific heat from the
  exact finite-torus Ising solution (tests/golden/ising_exact_beta_c.json), the
  comparison the paper itself makes (Sec. II.A).

A wrong coupling convention, a flip that is not uniform over q states, a
missing periodic bond or a labeling that merges or splits clusters shifts
these averages by many standard errors.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import oracle.exact as ex

GOLD = os.path.join(os.path.dirname(__file__), "golden")
KC_ISING = 0.5 * math.log(1.0 + math.sqrt(2.0))
Z_TOL = 4.5


def _binned(x, nbins=50):
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nbins * nbins
    b = x[:n].reshape(nbins, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nbins), b


def _jackknife_var(x, nbins=50):
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nbins * nbins
    xb = x[:n].reshape(nbins, -1)
    s1 = xb.sum(axis=1); s2 = (xb * xb).sum(axis=1)
    m = xb.shape[1]
    tot1, tot2, M = s1.sum(), s2.sum(), n
    full = tot2 / M - (tot1 / M) ** 2
    jk = np.array([((tot2 - s2[k]) / (M - m)) - ((tot1 - s1[k]) / (M - m)) ** 2 for k in range(nbins)])
    err = math.sqrt((nbins - 1) / nbins * ((jk - jk.mean()) ** 2).sum())
    return full, err


def _run(L, q, beta, conv, seed, n_sweeps, hot=True, burn=500):
    K = oracle.coupling_K(q, beta, 1.0, conv)
    T = oracle.threshold(K)
    s0 = oracle.init_spins(L, q, seed, hot)
    _, obs = oracle.chain(L, q, T, seed, 0, n_sweeps, s0)
    return K, obs[burn:]


def test_ising_4x4_against_enumeration():
    K, obs = _run(4, 2, KC_ISING, oracle.CONV_ISING, seed=5, n_sweeps=200_000)
    n_eq, counts = ex.enumerate_potts(4, 4, 2)
    exact = ex.moments_from_states(n_eq, counts, K, 2)
    n = obs[:, 0]
    absM = np.abs(obs[:, 1] - obs[:, 2])
    for series, key in ((n, "n_eq"), (n.astype(np.float64) ** 2, "n_eq2"), (absM, "absM")):
        m, e, _ = _binned(series)
        assert abs(m - exact[key]) < Z_TOL * e, (key, m, exact[key], e)


def test_ising_4x4_energy_histogram_chi2():
    K, obs = _run(4, 2, KC_ISING, oracle.CONV_ISING, seed=9, n_sweeps=200_000)
    g = np.array(json.load(open(os.path.join(GOLD, "potts_dos_4x4.json")))["g"]["2"])
    P = ex.dos_moments(g, K)["P"]
    thin = obs[::8, 0]                                  # thinning: SW tau_int << 8 here
    counts = np.bincount(thin, minlength=P.size)
    expect = P * thin.size
    sel = expect > 5
    stat = ((counts[sel] - expect[sel]) ** 2 / expect[sel]).sum()
    from scipy.stats import chi2
    assert chi2.sf(stat, sel.sum() - 1) > 1e-4
    assert counts[~sel].sum() < 5 * max(expect[~sel].sum(), 1.0) + 10


@pytest.mark.parametrize("q,beta", [(3, math.log(1 + math.sqrt(3))), (4, math.log(3.0))])
def test_potts_4x4_against_transfer_matrix(q, beta):
    K, obs = _run(4, q, beta, oracle.CONV_POTTS, seed=21 + q, n_sweeps=200_000)
    g = np.array(json.load(open(os.path.join(GOLD, "potts_dos_4x4.json")))["g"][str(q)])
    exact = ex.dos_moments(g, K)
    n = obs[:, 0].astype(np.float64)
    for series, key in ((n, "n_eq"), (n * n, "n_eq2")):
        m, e, _ = _binned(series)
        assert abs(m - exact[key]) < Z_TOL * e, (key, m, exact[key], e)
    # the state counts must be symmetric under permutations of the q states
    frac = obs[:, 1:].mean(axis=0) / 16.0
    assert np.all(np.abs(frac - 1.0 / q) < 0.02)


@pytest.mark.parametrize("L,n_sweeps,hot,seed", [(16, 100_000, True, 3), (64, 16_000, False, 1)])
def test_ising_energy_and_specific_heat_against_exact_torus(L, n_sweeps, hot, seed):
    """The paper's own check (Sec. II.A): q = 2 at criticality vs the exact
    finite-lattice solution.  L = 64, cold start, seed 1 is the small chain
    configuration the GPU parity tests also run."""
    ref = json.load(open(os.path.join(GOLD, "ising_exact_beta_c.json")))["sizes"][str(L)]
    K, obs = _run(L, 2, KC_ISING, oracle.CONV_ISING, seed=seed, n_sweeps=n_sweeps, hot=hot, burn=200)
    n = obs[:, 0]
    m, e, _ = _binned(n)
    assert abs(m - ref["mean_n_eq"]) < Z_TOL * e, (m, ref["mean_n_eq"], e)
    var, verr = _jackknife_var(n)
    assert abs(var - ref["var_n_eq"]) < Z_TOL * verr, (var, ref["var_n_eq"], verr)


# ---------------------------------------------------------------------------
# Off criticality: the beta / beta_c ratios of the paper's benchmark table
# (Table I: 0.6 and 1.4 for q = 2; q = 3 at the same ratios here).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ratio", [0.6, 1.4])
def test_ising_4x4_off_critical_against_enumeration(ratio):
    K, obs = _run(4, 2, ratio * KC_ISING, oracle.CONV_ISING, seed=31, n_sweeps=200_000)
    n_eq, counts = ex.enumerate_potts(4, 4, 2)
    exact = ex.moments_from_states(n_eq, counts, K, 2)
    n = obs[:, 0]
    absM = np.abs(obs[:, 1] - obs[:, 2])
    for series, key in ((n, "n_eq"), (n.astype(np.float64) ** 2, "n_eq2"), (absM, "absM")):
        m, e, _ = _binned(series)
        assert abs(m - exact[key]) < Z_TOL * e, (key, m, exact[key], e)


@pytest.mark.parametrize("ratio", [0.6, 1.4])
def test_potts_q3_4x4_off_critical_against_transfer_matrix(ratio):
    K, obs = _run(4, 3, ratio * math.log(1 + math.sqrt(3)), oracle.CONV_POTTS, seed=41, n_sweeps=200_000)
    g = np.array(json.load(open(os.path.join(GOLD, "potts_dos_4x4.json")))["g"]["3"])
    exact = ex.dos_moments(g, K)
    n = obs[:, 0].astype(np.float64)
    for series, key in ((n, "n_eq"), (n * n, "n_eq2")):
        m, e, _ = _binned(series)
        assert abs(m - exact[key]) < Z_TOL * e, (key, m, exact[key], e)


@pytest.mark.parametrize("ratio", [0.6, 1.4])
def test_ising_16x16_off_critical_against_exact_torus(ratio):
    ref = json.load(open(os.path.join(GOLD, "ising_exact_off_critical.json")))["ratios"][str(ratio)]
    K, obs = _run(16, 2, ratio * KC_ISING, oracle.CONV_ISING, seed=17, n_sweeps=60_000, burn=200)
    assert abs(K - 2 * ref["K"]) < 1e-15                # FK coupling = 2 x Ising coupling
    n = obs[:, 0]
    m, e, _ = _binned(n)
    assert abs(m - ref["mean_n_eq"]) < Z_TOL * e, (m, ref["mean_n_eq"], e)
    var, verr = _jackknife_var(n)
    assert abs(var - ref["var_n_eq"]) < Z_TOL * verr, (var, ref["var_n_eq"], verr)
