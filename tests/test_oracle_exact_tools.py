"""Pins of the exact tools that the chain pins rest on.

``oracle.exact`` supplies the exact equilibrium values that the whole-chain
pins compare the oracle's Swendsen-Wang averages against: the row transfer
matrix density of states (``potts_dos``) and Kaufman's finite-torus Ising
partition function (``ising_torus_logZ``, the exact solution the paper uses
as its check in Sec. II.A).  A slip in either would move the stored goldens
and every chain pin with them, so both are checked here against brute-force
enumeration of every spin state, which shares no arithmetic with them:

* ``potts_dos`` equals the histogram of n_eq over all q^N states of the
  4 x 4 torus (q = 2) and of the 3 x 4 and 4 x 3 tori (q = 3).
* ``ising_torus_logZ`` equals ln sum_states exp(K sum sigma_i sigma_j) on the
  4 x 4, 3 x 4 and 4 x 3 tori at couplings below, at and above K_c.
* The energy moments taken from Kaufman's ln Z by differentiation equal the
  enumerated <S> and Var(S) of S = sum sigma_i sigma_j on the 4 x 4 torus.
* On the 6 x 6 torus (2^36 states, beyond enumeration) the transfer matrix
  and Kaufman's formula, two independent exact methods, agree on ln Z.
"""
import math

import numpy as np
import pytest

import oracle.exact as ex

mpmath = pytest.importorskip("mpmath")

KC = 0.5 * math.log(1.0 + math.sqrt(2.0))


def _ising_S(Lx, Ly):
    """S = sum over the 2N bonds of sigma_i sigma_j = 2 n_eq - 2N, per state."""
    n_eq, _ = ex.enumerate_potts(Lx, Ly, 2)
    return 2 * n_eq - 2 * Lx * Ly


def _logsumexp(a):
    m = a.max()
    return float(m + np.log(np.exp(a - m).sum()))


@pytest.mark.parametrize("Lx,Ly,q", [(4, 4, 2), (3, 4, 3), (4, 3, 3), (2, 5, 3)])
def test_transfer_matrix_dos_equals_enumeration(Lx, Ly, q):
    n_eq, _ = ex.enumerate_potts(Lx, Ly, q)
    want = np.bincount(n_eq, minlength=2 * Lx * Ly + 1)
    got = ex.potts_dos(Lx, Ly, q)
    assert got.shape == want.shape
    assert np.array_equal(got, want)
    assert got.sum() == q ** (Lx * Ly)


@pytest.mark.parametrize("m,n", [(4, 4), (3, 4), (4, 3)])
@pytest.mark.parametrize("K", [0.2, KC, 0.7])
def test_kaufman_logZ_equals_enumeration(m, n, K):
    # Kaufman's (m, n) and the enumeration's (Lx, Ly) name the two sides; the
    # torus is symmetric in them, so both orders must give the same ln Z
    S = _ising_S(m, n).astype(np.float64)
    want = _logsumexp(K * S)
    got = float(ex.ising_torus_logZ(m, n, K))
    assert abs(got - want) < 1e-12 * max(1.0, abs(want))


def test_kaufman_energy_moments_equal_enumeration():
    S = _ising_S(4, 4).astype(np.float64)
    for K in (0.3, KC, 0.6):
        w = np.exp(K * S - (K * S).max())
        Z = w.sum()
        mean = float((w * S).sum() / Z)
        var = float((w * S * S).sum() / Z) - mean ** 2
        d1, d2 = ex.ising_torus_energy_moments(4, K)
        assert abs(d1 - mean) < 1e-10 * max(1.0, abs(mean))
        assert abs(d2 - var) < 1e-10 * max(1.0, abs(var))


def test_transfer_matrix_and_kaufman_agree_on_6x6():
    g = ex.potts_dos(6, 6, 2)
    assert g.sum() == 2 ** 36
    N = 36
    n = np.arange(g.size, dtype=np.float64)
    for K in (0.25, KC, 0.55):
        # Potts weights exp(2K n_eq) on the delta scale = Ising exp(K S) * exp(2K N)
        logw = np.where(g > 0, np.log(np.maximum(g, 1).astype(np.float64)) + K * (2 * n - 2 * N), -np.inf)
        want = _logsumexp(logw[np.isfinite(logw)])
        got = float(ex.ising_torus_logZ(6, 6, K))
        assert abs(got - want) < 1e-11 * abs(want)
