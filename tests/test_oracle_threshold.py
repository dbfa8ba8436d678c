"""Pins of the oracle's coupling convention, threshold and state map.

* The self-dual point of the FK / random-cluster model is
  p_c = sqrt(q) / (1 + sqrt(q)); at the critical couplings the paper quotes
  (beta_c = ln(1+sqrt2) for q = 2 in the delta convention, Sec. II.B.3) and
  the Ising convention beta_c = ln(1+sqrt2)/2, and q = 4 at beta = ln 3, the
  oracle's threshold must equal floor(p_c 2^32) computed in exact integer
  arithmetic.  A K = beta vs K = 2 beta mix-up fails this.
* F_q(w) = floor(w q / 2^32) must split [0, 2^32) into q intervals whose
  boundaries are ceil(k 2^32 / q).
"""
import json
import math
import os
from fractions import Fraction

import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _floor_pc_times_2_32(q):
    # p_c 2^32 = sqrt(q) 2^32 / (1 + sqrt(q)); sqrt(q) is rational only for square q,
    # so bracket it with integer square roots at 2^-96 precision.
    S = 1 << 96
    r = math.isqrt(q * S * S)            # floor(sqrt(q) * S)
    lo = Fraction(r, S)
    hi = Fraction(r + 1, S)
    f_lo = math.floor(lo * 2 ** 32 / (1 + lo))
    f_hi = math.floor(hi * 2 ** 32 / (1 + hi))
    assert f_lo == f_hi
    return f_lo


def test_paper_beta_c_q2_delta_convention():
    consts = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    beta_c = consts["beta_c_potts_q2"]["value"]
    K = oracle.coupling_K(2, beta_c, 1.0, oracle.CONV_POTTS)
    assert oracle.threshold(K) == _floor_pc_times_2_32(2)


@pytest.mark.parametrize("q,beta,conv", [
    (2, 0.5 * math.log(1 + math.sqrt(2)), oracle.CONV_ISING),
    (2, 0.5 * math.log(1 + math.sqrt(2)), oracle.CONV_AUTO),
    (3, math.log(1 + math.sqrt(3)), oracle.CONV_POTTS),
    (4, math.log(3.0), oracle.CONV_AUTO),
])
def test_threshold_at_self_dual_point(q, beta, conv):
    K = oracle.coupling_K(q, beta, 1.0, conv)
    assert oracle.threshold(K) == _floor_pc_times_2_32(q)


def test_threshold_limits():
    assert oracle.threshold(0.0) == 0
    assert oracle.threshold(-1.0) == 0
    assert oracle.threshold(800.0) == 1 << 32          # p = 1: every equal bond opens
    # ln 2: p = 1/2 exactly representable -> 2^31 (the percolation threshold)
    assert oracle.threshold(math.log(2.0)) == 1 << 31


@pytest.mark.parametrize("q", [2, 3, 4, 5, 7, 127])
def test_flip_state_interval_boundaries(q):
    for k in range(1, q):
        b = -((-k * 2 ** 32) // q)          # ceil(k 2^32 / q)
        assert oracle.flip_state(b, q) == k
        assert oracle.flip_state(b - 1, q) == k - 1
    assert oracle.flip_state(0, q) == 0
    assert oracle.flip_state(2 ** 32 - 1, q) == q - 1
