"""GPU parity off criticality and for q = 3: the workload variants of the
paper's benchmark table (Table I: q = 2 at beta/beta_c = 0.6, 1 and 1.4,
q = 3 and 4 at beta_c, L = 8192).

Below beta_c the clusters are small and many; above it one cluster spans the
lattice and nearly every seam bond joins it, the hardest case for the global
merge (long hook chains on one root).  Small lattices run whole chains
against the oracle in both modes; L = 8192 (the table's size) is checked by
one-step equivalence at sweep 0 and after 40 sweeps, when the ordered phase
has formed at 1.4 beta_c.  All comparisons are bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
import paper_1105_5804_gb300 as sw

pytestmark = pytest.mark.gpu


def _beta(q, ratio):
    return ratio * math.log(1.0 + math.sqrt(q))      # delta convention, beta_c = ln(1 + sqrt q)


def _chain(L, q, ratio, seed, n_sweeps, mode, per_call):
    T = oracle.threshold(oracle.coupling_K(q, _beta(q, ratio), 1.0, oracle.CONV_POTTS))
    h = sw.sw_create_threshold(L, q, T, seed, True)
    try:
        sw.sw_set_mode(h, mode)
        s = oracle.init_spins(L, q, seed, True)
        done = 0
        while done < n_sweeps:
            k = min(per_call, n_sweeps - done)
            sw.sw_sweep(h, k)
            s, obs = oracle.chain(L, q, T, seed, done, k, s)
            assert np.array_equal(sw.sw_get_spins(h), s), (L, q, ratio, done)
            assert np.array_equal(sw.sw_observables(h, 4096), obs), (L, q, ratio, done)
            done += k
        return s
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("ratio", [0.6, 1.4])
@pytest.mark.parametrize("q", [2, 3])
@pytest.mark.parametrize("L", [36, 256, 260])
def test_fused_chain_off_critical(L, q, ratio):
    s = _chain(L, q, ratio, seed=300 + L + q, n_sweeps=40, mode=sw.SW_MODE_FUSED, per_call=10)
    if ratio == 1.4 and q == 2:
        m = abs(2.0 * np.count_nonzero(s) - s.size) / s.size
        assert m > 0.5                                # ordered: one spin state dominates


@pytest.mark.parametrize("ratio", [0.6, 1.4])
@pytest.mark.parametrize("q", [2, 3])
def test_staged_chain_off_critical(q, ratio):
    _chain(100, q, ratio, seed=400 + q, n_sweeps=12, mode=sw.SW_MODE_STAGED, per_call=1)


@pytest.mark.parametrize("q,ratio", [(2, 0.6), (2, 1.4), (3, 1.0)])
def test_L8192_one_step_equivalence(q, ratio):
    """Fused sweeps at the table's lattice size, hot start seed 7: sweeps 0
    and 40 stepped by the oracle from the GPU's pre-sweep spins."""
    L, seed = 8192, 7
    beta = _beta(q, ratio)
    T = oracle.threshold(oracle.coupling_K(q, beta, 1.0, oracle.CONV_POTTS))
    h = sw.sw_create_ex(L, q, beta, 1.0, sw.SW_CONV_POTTS, seed, True)
    try:
        s = sw.sw_get_spins(h)
        done = 0
        for k in (0, 40):
            if k > done:
                sw.sw_sweep(h, k - done)
                sw.sw_observables(h, 4096)
                s = sw.sw_get_spins(h)
            sw.sw_sweep(h, 1)
            done = k + 1
            gs = sw.sw_get_spins(h)
            gobs = sw.sw_observables(h, 4)
            s_new, _, _, obs = oracle.sweep(L, q, T, seed, k, s)
            assert np.array_equal(gs, s_new), (q, ratio, k)
            assert np.array_equal(gobs[-1], obs), (q, ratio, k)
        if ratio == 1.4:
            assert obs[0] > 1.9 * L * L               # nearly every bond joins equal spins
    finally:
        sw.sw_destroy(h)
