"""GPU parity of batched chains (sw_batch_*) through the C ABI.

Every chain of a batch must follow exactly the chain a single handle (and the
oracle) computes from the same (L, q, beta, seed): spins and observables are
compared with the oracle bit for bit, under both schedules (one launch per
step; one persistent cooperative launch per sweep).  The 512-replica workload
(L log-uniform in [64, 2048], beta in [0.9, 1.1] beta_c, seed = replica id)
is checked on a sample of chains against the oracle, and on every chain for
agreement between the two schedules.
"""
import math

import numpy as np
import pytest

import oracle
import paper_1105_5804_gb300 as sw
from paper_1105_5804_gb300 import inputs

pytestmark = pytest.mark.gpu

KC = 0.5 * math.log(1.0 + math.sqrt(2.0))


def _oracle_T(q, beta, conv):
    return oracle.threshold(oracle.coupling_K(q, beta, 1.0, conv))


MIX = [  # (L, q, beta)
    (4, 2, KC), (36, 3, math.log(1 + math.sqrt(3))), (64, 2, 0.9 * KC), (100, 4, math.log(3.0)),
    (256, 2, 1.1 * KC), (260, 2, KC), (292, 3, 0.8), (8, 5, 1.2), (520, 2, KC),
]


@pytest.mark.parametrize("tile_w", [256, 128, 64])
@pytest.mark.parametrize("schedule", [sw.SW_BATCH_PHASES, sw.SW_BATCH_PERSISTENT])
def test_mixed_batch_matches_oracle(schedule, tile_w):
    """Every chain of a mixed batch (sizes from one ragged tile to several,
    q = 2..5) equals the oracle's chain, for each labeling tile width the
    autotuner can pick and both schedules."""
    conv = sw.SW_CONV_AUTO
    L = [m[0] for m in MIX]
    q = [m[1] for m in MIX]
    beta = [m[2] for m in MIX]
    seed = [1000 + 7 * r for r in range(len(MIX))]
    b = sw.sw_batch_create(L, q, beta, seed, conv, True, tile_w=tile_w)
    try:
        sw.sw_batch_set_schedule(b, schedule)
        spins = [oracle.init_spins(L[r], q[r], seed[r], True) for r in range(len(MIX))]
        done = 0
        for n in (1, 3, 2):
            sw.sw_batch_sweep(b, n)
            sw.sw_batch_sync(b)
            for r in range(len(MIX)):
                T = _oracle_T(q[r], beta[r], oracle.CONV_AUTO)
                spins[r], obs = oracle.chain(L[r], q[r], T, seed[r], done, n, spins[r])
                assert np.array_equal(sw.sw_batch_get_spins(b, r, L[r]), spins[r]), (schedule, r, done)
                assert np.array_equal(sw.sw_batch_observables(b, r, q[r]), obs), (schedule, r, done)
            done += n
        info = sw.sw_batch_info(b)
        assert info["chains"] == len(MIX) and info["sweeps"] == done and info["schedule"] == schedule
        assert info["tile_w"] == tile_w
    finally:
        sw.sw_batch_destroy(b)


def test_chain_is_the_same_alone_and_in_a_batch():
    """A chain's spins do not depend on the other chains of its batch."""
    L, q, beta, seed = 132, 3, 1.0, 77
    h = sw.sw_create_ex(L, q, beta, 1.0, sw.SW_CONV_AUTO, seed, True)
    b = sw.sw_batch_create([64, L, 260], [2, q, 4], [KC, beta, 1.1], [5, seed, 6], sw.SW_CONV_AUTO, True)
    try:
        sw.sw_sweep(h, 9)
        sw.sw_batch_sweep(b, 9)
        assert np.array_equal(sw.sw_batch_get_spins(b, 1, L), sw.sw_get_spins(h))
        assert np.array_equal(sw.sw_batch_observables(b, 1, q), sw.sw_observables(h))
    finally:
        sw.sw_destroy(h)
        sw.sw_batch_destroy(b)


def test_512_replica_workload_sample_and_schedules_agree():
    reps = inputs.batched_replicas()
    assert len(reps) == 512
    L = [r["L"] for r in reps]
    beta = [r["beta"] for r in reps]
    seed = [r["seed"] for r in reps]
    assert all(l % 32 == 0 and 64 <= l <= 2048 for l in L)
    q = [2] * 512
    b1 = sw.sw_batch_create(L, q, beta, seed, sw.SW_CONV_ISING, False)
    b2 = sw.sw_batch_create(L, q, beta, seed, sw.SW_CONV_ISING, False)
    b3 = sw.sw_batch_create(L, q, beta, seed, sw.SW_CONV_ISING, False, tile_w=128)
    b4 = sw.sw_batch_create(L, q, beta, seed, sw.SW_CONV_ISING, False, tile_w=64)
    try:
        sw.sw_batch_set_schedule(b2, sw.SW_BATCH_PERSISTENT)
        for b in (b1, b2, b3, b4):
            sw.sw_batch_sweep(b, 3)
        sample = sorted(range(512), key=lambda r: L[r])[:6] + [0, 255, 511]
        for r in range(512):
            s1 = sw.sw_batch_get_spins(b1, r, L[r])
            o1 = sw.sw_batch_observables(b1, r, 2)
            for b in (b2, b3, b4):                # other schedule, other tile widths
                assert np.array_equal(s1, sw.sw_batch_get_spins(b, r, L[r])), r
                assert np.array_equal(o1, sw.sw_batch_observables(b, r, 2)), r
            assert np.all(o1[:, 1] + o1[:, 2] == L[r] * L[r])
            if r in sample:
                T = _oracle_T(2, beta[r], oracle.CONV_ISING)
                s, obs = oracle.chain(L[r], 2, T, seed[r], 0, 3, oracle.init_spins(L[r], 2, seed[r], False))
                assert np.array_equal(s1, s), r
                assert np.array_equal(o1, obs), r
    finally:
        for b in (b1, b2, b3, b4):
            sw.sw_batch_destroy(b)


def test_autotuner_picks_a_tile_width_and_schedule_and_the_batch_matches_the_oracle(tmp_path, monkeypatch):
    from paper_1105_5804_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    L, q, beta, seed = [96, 160, 288, 64], [2, 2, 3, 2], [KC, 0.9 * KC, 0.8, 1.1 * KC], [21, 22, 23, 24]
    b, choice = autotune.create_tuned(L, q, beta, seed, sw.SW_CONV_AUTO, True, sweeps=2, max_blocks_per_sm=2)
    try:
        assert choice["tile_w"] in (64, 128, 256) and len(choice["timings"]) == 3 * 3
        assert sw.sw_batch_info(b)["tile_w"] == choice["tile_w"]
        sw.sw_batch_sweep(b, 2)
        sw.sw_batch_sync(b)
        for r in range(len(L)):
            T = _oracle_T(q[r], beta[r], oracle.CONV_AUTO)
            s, obs = oracle.chain(L[r], q[r], T, seed[r], 0, 2, oracle.init_spins(L[r], q[r], seed[r], True))
            assert np.array_equal(sw.sw_batch_get_spins(b, r, L[r]), s), r
            assert np.array_equal(sw.sw_batch_observables(b, r, q[r]), obs), r
    finally:
        sw.sw_batch_destroy(b)


def test_batch_rejects_bad_chains():
    with pytest.raises(sw.SwcclError):
        sw.sw_batch_create([64, 30], [2, 2], [0.4, 0.4], [1, 2])
    with pytest.raises(sw.SwcclError):
        sw.sw_batch_create([64], [200], [0.4], [1])


def test_persistent_barrier_timeout_is_reported_and_device_stays_usable():
    """The failure path of the persistent schedule's bounded grid barrier.
    With a limit of 0 cycles every CTA but the last to arrive gives up at its
    first barrier and returns (no wait at all, nothing hangs): the next
    synchronising call reports SW_ERR_TIMEOUT, the batch then refuses further
    sweeps with SW_ERR_STATE, and the device keeps working: a new batch with
    the default limit computes the oracle's chain."""
    import torch
    L, q, beta, seed = [64, 128, 256, 260], [2, 2, 3, 2], [KC, KC, 0.9, 1.1 * KC], [1, 2, 3, 4]
    b = sw.sw_batch_create(L, q, beta, seed, sw.SW_CONV_AUTO, True)
    try:
        sw.sw_batch_set_schedule(b, sw.SW_BATCH_PERSISTENT)
        assert sw.sw_batch_info(b)["persistent_blocks"] > 1
        sw.sw_batch_set_barrier_limit(b, 0)
        sw.sw_batch_sweep(b, 1)
        with pytest.raises(sw.SwcclError) as e:
            sw.sw_batch_sync(b)
        assert e.value.code == sw.SW_ERR_TIMEOUT
        with pytest.raises(sw.SwcclError) as e:
            sw.sw_batch_sweep(b, 1)
        assert e.value.code == sw.SW_ERR_STATE
        with pytest.raises(sw.SwcclError) as e:
            sw.sw_batch_set_barrier_limit(b, -1)
        assert e.value.code == sw.SW_ERR_ARG
    finally:
        sw.sw_batch_destroy(b)
    # the context is intact
    x = torch.arange(1 << 20, device="cuda", dtype=torch.int64)
    assert int(x.sum().item()) == (1 << 20) * ((1 << 20) - 1) // 2
    b = sw.sw_batch_create(L, q, beta, seed, sw.SW_CONV_AUTO, True)
    try:
        sw.sw_batch_set_schedule(b, sw.SW_BATCH_PERSISTENT)
        sw.sw_batch_sweep(b, 2)
        sw.sw_batch_sync(b)
        for r in range(len(L)):
            T = _oracle_T(q[r], beta[r], oracle.CONV_AUTO)
            s, obs = oracle.chain(L[r], q[r], T, seed[r], 0, 2, oracle.init_spins(L[r], q[r], seed[r], True))
            assert np.array_equal(sw.sw_batch_get_spins(b, r, L[r]), s), r
            assert np.array_equal(sw.sw_batch_observables(b, r, q[r]), obs), r
    finally:
        sw.sw_batch_destroy(b)


def test_batch_in_caller_workspace_without_graph_matches_oracle():
    """sw_batch_create_ws carves the batch from a caller's device buffer (no
    allocation by the library) and sweeps launched without a captured graph:
    the same chains, bit for bit, as the oracle; the size query equals what
    the call requires."""
    import torch
    L, q, beta, seed = [64, 100, 256, 36], [2, 3, 2, 4], [KC, 0.8, 1.1 * KC, math.log(3.0)], [5, 6, 7, 8]
    need = sw.sw_batch_device_bytes(L, q)
    assert need > sum(l * l for l in L)
    with pytest.raises(sw.SwcclError):
        sw.sw_batch_create_ws(L, q, beta, seed, torch.empty(need - 256, dtype=torch.uint8, device="cuda"),
                              sw.SW_CONV_AUTO, True)
    ws = torch.full((need,), 0x5A, dtype=torch.uint8, device="cuda")
    b = sw.sw_batch_create_ws(L, q, beta, seed, ws, sw.SW_CONV_AUTO, True)
    try:
        sw.sw_batch_set_graph(b, False)
        sw.sw_batch_sweep(b, 3)
        sw.sw_batch_sync(b)
        assert sw.sw_batch_info(b)["graph"] == 0
        for r in range(len(L)):
            T = _oracle_T(q[r], beta[r], oracle.CONV_AUTO)
            s, obs = oracle.chain(L[r], q[r], T, seed[r], 0, 3, oracle.init_spins(L[r], q[r], seed[r], True))
            assert np.array_equal(sw.sw_batch_get_spins(b, r, L[r]), s), r
            assert np.array_equal(sw.sw_batch_observables(b, r, q[r]), obs), r
    finally:
        sw.sw_batch_destroy(b)
    assert ws.numel() == need            # the caller still owns the workspace
