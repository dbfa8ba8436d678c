"""GPU parity of the simple-cubic Swendsen-Wang chain against the oracle,
through the C ABI (sw3_*).

Every call compares the spins and the per-sweep observables bit for bit with
the oracle's 3D chain; single steps also compare the canonical labels of the
sweep's clusters.  Boxes: one brick exactly (32 x 8 x 16), ragged bricks,
sides of 1 and 2 (self bonds and doubled bonds), several bricks per axis;
q = 2, 3, 5, 127; the degenerate thresholds; timed mode; spin round trips and
errors; and, at 256^3 and 512^3 (the benchmark's box), one-step equivalence
from the GPU's pre-sweep spins.
"""
import math

import numpy as np
import pytest

import oracle
import paper_1105_5804_gb300 as sw

pytestmark = pytest.mark.gpu

KC3_ISING = 0.2216546   # simple-cubic Ising critical coupling (literature value), a test point only


def _T(q):
    if q == 2:
        return oracle.threshold(2 * KC3_ISING)
    return oracle.threshold(0.55 * math.log(1 + math.sqrt(q)))


def _chain(dims, q, T, seed, n_sweeps, per_call=2, hot=True, timing=False):
    X, Y, Z = dims
    h = sw.sw3_create(X, Y, Z, q, T, seed, hot)
    try:
        if timing:
            sw.sw3_set_timing(h, True)
        s = oracle.init_spins3(X, Y, Z, q, seed, hot)
        assert np.array_equal(sw.sw3_get_spins(h), s)
        done = 0
        while done < n_sweeps:
            k = min(per_call, n_sweeps - done)
            if k == 1:
                pre = s
            sw.sw3_sweep(h, k)
            s, obs = oracle.chain3(X, Y, Z, q, T, seed, done, k, s)
            assert np.array_equal(sw.sw3_get_spins(h), s), (dims, q, done)
            assert np.array_equal(sw.sw3_observables(h, 4096), obs), (dims, q, done)
            if k == 1:
                _, _, lab, _ = oracle.sweep3(X, Y, Z, q, T, seed, done, pre)
                assert np.array_equal(sw.sw3_labels(h), lab), (dims, q, done)
            done += k
        if timing:
            ms, n = sw.sw3_phase_times(h)
            assert n == n_sweeps and all(v >= 0 for v in ms.values())
    finally:
        sw.sw3_destroy(h)


BOXES = [(32, 8, 16), (4, 4, 4), (33, 9, 17), (64, 16, 32), (2, 2, 2), (1, 12, 20), (40, 1, 3), (96, 24, 48),
         (7, 31, 33)]


@pytest.mark.parametrize("dims", BOXES)
@pytest.mark.parametrize("q", [2, 3])
def test_chains(dims, q):
    _chain(dims, q, _T(q), seed=600 + sum(dims) + q, n_sweeps=6)


@pytest.mark.parametrize("dims", [(32, 8, 16), (33, 9, 17), (64, 16, 32)])
def test_single_steps_with_labels(dims):
    _chain(dims, 2, _T(2), seed=41, n_sweeps=5, per_call=1)


@pytest.mark.parametrize("q", [5, 127])
def test_many_states(q):
    _chain((40, 20, 24), q, _T(q), seed=8, n_sweeps=4)


@pytest.mark.parametrize("T", [0, 1, 1 << 31, (1 << 32) - 1, 1 << 32])
def test_degenerate_thresholds(T):
    _chain((36, 12, 20), 2, T, seed=3, n_sweeps=3, per_call=1)


def test_cold_start_and_timed_mode():
    _chain((64, 16, 32), 2, _T(2), seed=1, n_sweeps=20, per_call=5, hot=False)
    _chain((33, 9, 17), 3, _T(3), seed=2, n_sweeps=4, per_call=1, timing=True)


def test_spins_round_trip_and_errors():
    import torch
    X, Y, Z, q = 24, 16, 20, 3
    h = sw.sw3_create(X, Y, Z, q, _T(q), 5, True)
    try:
        with pytest.raises(sw.SwcclError):
            sw.sw3_labels(h)                          # no sweep yet
        rng = np.random.default_rng(0)
        s = rng.integers(0, q, X * Y * Z).astype(np.int8)
        sw.sw3_set_spins(h, s)
        assert np.array_equal(sw.sw3_get_spins(h), s)
        bad = s.copy()
        bad[17] = q
        with pytest.raises(sw.SwcclError) as e:
            sw.sw3_set_spins(h, bad)
        assert e.value.code == sw.SW_ERR_ARG
        assert np.array_equal(sw.sw3_get_spins(h), s)
        d = torch.from_numpy(s).cuda()
        sw.sw3_set_spins(h, d)
        sw.sw3_sweep(h, 1)
        s1, m, lab, obs = oracle.sweep3(X, Y, Z, q, _T(q), 5, 0, s)
        out = torch.empty(X * Y * Z, dtype=torch.int8, device="cuda")
        sw.sw3_get_spins(h, out)
        assert np.array_equal(out.cpu().numpy(), s1)
        lab_d = torch.empty(X * Y * Z, dtype=torch.int32, device="cuda")
        sw.sw3_labels(h, lab_d)
        assert np.array_equal(lab_d.cpu().numpy(), lab)
        assert np.array_equal(sw.sw3_observables(h)[-1], obs)
    finally:
        sw.sw3_destroy(h)
    for args in [(0, 4, 4, 2, 0, 1), (1024, 1024, 1025, 2, 0, 1), (8, 8, 8, 1, 0, 1), (8, 8, 8, 128, 0, 1),
                 (8, 8, 8, 2, (1 << 32) + 1, 1)]:
        with pytest.raises(sw.SwcclError):
            sw.sw3_create(*args)


@pytest.mark.parametrize("L,samples", [(256, (0, 12)), (512, (0, 5))])
def test_large_box_one_step_equivalence(L, samples):
    """q = 2 at the simple-cubic critical coupling, hot start seed 7; sampled
    sweeps are stepped by the oracle from the GPU's pre-sweep spins."""
    q, seed = 2, 7
    T = _T(q)
    h = sw.sw3_create(L, L, L, q, T, seed, True)
    try:
        done = 0
        s = sw.sw3_get_spins(h)
        for k in samples:
            if k > done:
                sw.sw3_sweep(h, k - done)
                sw.sw3_observables(h)
                s = sw.sw3_get_spins(h)
            sw.sw3_sweep(h, 1)
            done = k + 1
            s_new, _, lab, obs = oracle.sweep3(L, L, L, q, T, seed, k, s)
            assert np.array_equal(sw.sw3_get_spins(h), s_new), (L, k)
            assert np.array_equal(sw.sw3_observables(h)[-1], obs), (L, k)
            assert np.array_equal(sw.sw3_labels(h), lab), (L, k)
    finally:
        sw.sw3_destroy(h)
