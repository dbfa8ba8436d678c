"""GPU parity of the few-cluster update (Sec. III, variant (c)) against the
oracle, through the C ABI.

The handle runs fused sweeps with SW_UPDATE_FEW: SW bonds and clusters, one
seed per block of an ell x ell grid, and only the seeded clusters move, each
with probability p_flip.  Spins and observables are compared bit for bit
after every call with the oracle's few-cluster chain.  Cases: ragged tiles
(L = 36 ... 292), ell from 1 (one seed) to L (a seed on every site), p_flip
0.5 and 1, q = 2, 3, 5 and 127, the degenerate thresholds, switches between
the SW and the few-cluster update within one chain, timed mode, argument
errors, and one-step equivalence at L = 8192 with 16^2 and 256^2 seeds.
"""
import math

import numpy as np
import pytest

import oracle
import paper_1105_5804_gb300 as sw

pytestmark = pytest.mark.gpu

FULL = 1 << 32
HALF = 1 << 31


def _T(q):
    return oracle.threshold(oracle.coupling_K(q, math.log(1 + math.sqrt(q)), 1.0, oracle.CONV_POTTS))


def _run_few(L, q, T, P, ell, seed, n_sweeps, per_call=3, timing=False):
    h = sw.sw_create_threshold(L, q, T, seed, True)
    try:
        sw.sw_set_update(h, sw.SW_UPDATE_FEW, ell, P)
        if timing:
            sw.sw_set_timing(h, True)
        s = oracle.init_spins(L, q, seed, True)
        done = 0
        while done < n_sweeps:
            k = min(per_call, n_sweeps - done)
            sw.sw_sweep(h, k)
            s, obs = oracle.few_chain(L, q, T, P, ell, seed, done, k, s)
            assert np.array_equal(sw.sw_get_spins(h), s), ("spins", L, q, ell, P, done)
            assert np.array_equal(sw.sw_observables(h, 4096), obs), ("obs", L, q, ell, P, done)
            done += k
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("P", [HALF, FULL])
@pytest.mark.parametrize("q", [2, 3])
@pytest.mark.parametrize("L,ells", [(36, (1, 3, 36)), (100, (2, 25, 100)), (256, (1, 16, 256)), (260, (1, 13, 65)),
                                    (292, (4, 73, 292))])
def test_few_cluster_chains(L, ells, q, P):
    for ell in ells:
        _run_few(L, q, _T(q), P, ell, seed=500 + L + q + ell, n_sweeps=8)


@pytest.mark.parametrize("q", [5, 127])
def test_few_cluster_many_states(q):
    _run_few(132, q, _T(q), int(0.7 * FULL), 4, seed=9, n_sweeps=6)


@pytest.mark.parametrize("T", [0, 1, HALF, FULL])
def test_few_cluster_degenerate_thresholds(T):
    _run_few(68, 2, T, FULL, 68, seed=3, n_sweeps=4)
    _run_few(68, 3, T, HALF, 2, seed=4, n_sweeps=4)


def test_few_cluster_timed_mode():
    _run_few(260, 2, _T(2), HALF, 5, seed=12, n_sweeps=6, per_call=1, timing=True)


# L = 256: the SW sweeps go through the site codes, the few-cluster sweeps
# through the 16-bit tile roots
@pytest.mark.parametrize("L,e1,e2", [(260, 5, 13), (256, 4, 16)])
def test_switching_between_sw_and_few_cluster(L, e1, e2):
    q, seed = 3, 71
    T = _T(q)
    h = sw.sw_create_threshold(L, q, T, seed, True)
    try:
        s = oracle.init_spins(L, q, seed, True)
        done = 0
        for upd, ell, P, n in [(sw.SW_UPDATE_SW, 0, 0, 3), (sw.SW_UPDATE_FEW, e1, HALF, 4),
                               (sw.SW_UPDATE_FEW, e2, FULL, 2), (sw.SW_UPDATE_SW, 0, 0, 2),
                               (sw.SW_UPDATE_FEW, e1, HALF, 3)]:
            sw.sw_set_update(h, upd, ell, P)
            sw.sw_sweep(h, n)
            if upd == sw.SW_UPDATE_SW:
                s, obs = oracle.chain(L, q, T, seed, done, n, s)
            else:
                s, obs = oracle.few_chain(L, q, T, P, ell, seed, done, n, s)
            done += n
            assert np.array_equal(sw.sw_get_spins(h), s), (upd, done)
            assert np.array_equal(sw.sw_observables(h, 4096), obs), (upd, done)
    finally:
        sw.sw_destroy(h)


def test_few_cluster_arguments_and_mode():
    h = sw.sw_create_threshold(64, 2, _T(2), 1, True)
    try:
        for ell, P in [(0, HALF), (3, HALF), (65, HALF), (4, FULL + 1)]:
            with pytest.raises(sw.SwcclError) as e:
                sw.sw_set_update(h, sw.SW_UPDATE_FEW, ell, P)
            assert e.value.code == sw.SW_ERR_ARG
        with pytest.raises(sw.SwcclError):
            sw.sw_set_update(h, 7, 4, HALF)
        sw.sw_set_update(h, sw.SW_UPDATE_FEW, 4, HALF)
        with pytest.raises(sw.SwcclError) as e:
            sw.sw_set_mode(h, sw.SW_MODE_STAGED)
        assert e.value.code == sw.SW_ERR_STATE
        sw.sw_set_update(h, sw.SW_UPDATE_SW)
        sw.sw_set_mode(h, sw.SW_MODE_STAGED)
        with pytest.raises(sw.SwcclError) as e:
            sw.sw_set_update(h, sw.SW_UPDATE_FEW, 4, HALF)
        assert e.value.code == sw.SW_ERR_STATE
    finally:
        sw.sw_destroy(h)
    assert sw.sw_prob_threshold(0.0) == 0 and sw.sw_prob_threshold(1.0) == FULL
    assert sw.sw_prob_threshold(0.5) == HALF and sw.sw_prob_threshold(-0.1) == (1 << 64) - 1


@pytest.mark.parametrize("ell", [16, 256])
def test_L8192_one_step_equivalence(ell):
    """L = 8192, q = 2 at beta_c, hot start seed 7, p_flip = 1/2: sweeps 0
    and 20 stepped by the oracle from the GPU's pre-sweep spins."""
    L, q, seed = 8192, 2, 7
    T = oracle.threshold(oracle.coupling_K(2, 0.5 * math.log(1 + math.sqrt(2)), 1.0, oracle.CONV_ISING))
    h = sw.sw_create_threshold(L, q, T, seed, True)
    try:
        sw.sw_set_update(h, sw.SW_UPDATE_FEW, ell, HALF)
        s = sw.sw_get_spins(h)
        done = 0
        for k in (0, 20):
            if k > done:
                sw.sw_sweep(h, k - done)
                sw.sw_observables(h, 4096)
                s = sw.sw_get_spins(h)
            sw.sw_sweep(h, 1)
            done = k + 1
            gs = sw.sw_get_spins(h)
            gobs = sw.sw_observables(h, 4)
            s_new, _, _, obs = oracle.few_sweep(L, q, T, HALF, ell, seed, k, s)
            assert np.array_equal(gs, s_new), (ell, k)
            assert np.array_equal(gobs[-1], obs), (ell, k)
            assert not np.array_equal(s_new, s)      # some seeded cluster moved
    finally:
        sw.sw_destroy(h)
