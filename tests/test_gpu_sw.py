"""GPU parity of the Swendsen-Wang chain against the oracle, through the C ABI.

Every sweep compares the bond mask, the canonical labels, the new spins and
the observables bit for bit (integer work).  Cases: the L = 64 Ising chain
at beta_c from a cold start with seed 1 for 1000 sweeps; odd lattice sizes
that leave ragged tiles (L = 4, 8, 36, 100, 132, 196); q = 2, 3, 4, 5, 9
and 127 (register and shared-memory state counters); the degenerate
thresholds T = 0 (no bond opens) and T = 2^32 (every equal bond opens); hot
starts.  At L = 16384, the size the benchmark times, sampled sweeps are
checked by one-step equivalence: the oracle steps the GPU's pre-sweep spins
once and must reproduce the GPU's mask, labels, spins and observables.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1105_5804_gb300 as sw

pytestmark = pytest.mark.gpu

KC = 0.5 * math.log(1.0 + math.sqrt(2.0))


def _run_parity(L, q, T, seed, hot, n_sweeps, sweep_graph=True):
    """Staged mode: every sweep's mask, labels, spins and observables."""
    h = sw.sw_create_threshold(L, q, T, seed, hot)
    try:
        sw.sw_set_mode(h, sw.SW_MODE_STAGED)
        if not sweep_graph:
            sw.sw_set_timing(h, True)
        s = oracle.init_spins(L, q, seed, hot)
        assert np.array_equal(sw.sw_get_spins(h), s)
        for k in range(n_sweeps):
            sw.sw_sweep(h, 1)
            s, m, lab, obs = oracle.sweep(L, q, T, seed, k, s)
            gm, glab = sw.sw_debug_dump(h)
            assert np.array_equal(gm, m), ("mask", L, q, k)
            assert np.array_equal(glab, lab), ("labels", L, q, k)
            assert np.array_equal(sw.sw_get_spins(h), s), ("spins", L, q, k)
            gobs = sw.sw_observables(h, 4)
            assert gobs.shape[0] == 1 and np.array_equal(gobs[0], obs), ("obs", L, q, k)
    finally:
        sw.sw_destroy(h)


def test_ising_L64_cold_start_1000_sweeps_bit_exact():
    """The small chain configuration: L = 64, q = 2, beta_c (Ising), cold
    start, seed 1, 1000 sweeps, every sweep compared; then <E>, <|M|> of the
    chain equal the oracle's (identical sequences)."""
    L, q, seed = 64, 2, 1
    T = oracle.threshold(oracle.coupling_K(q, KC, 1.0, oracle.CONV_ISING))
    h = sw.sw_create_ex(L, q, KC, 1.0, sw.SW_CONV_ISING, seed, False)
    try:
        sw.sw_set_mode(h, sw.SW_MODE_STAGED)
        s = oracle.init_spins(L, q, seed, False)
        gobs_all = []
        for k in range(1000):
            sw.sw_sweep(h, 1)
            s, m, lab, obs = oracle.sweep(L, q, T, seed, k, s)
            gm, glab = sw.sw_debug_dump(h)
            assert np.array_equal(gm, m), k
            assert np.array_equal(glab, lab), k
            assert np.array_equal(sw.sw_get_spins(h), s), k
            g = sw.sw_observables(h, 4)
            assert np.array_equal(g[0], obs), k
            gobs_all.append(g[0])
        gobs_all = np.array(gobs_all)
        _, oobs = oracle.chain(L, q, T, seed, 0, 1000, oracle.init_spins(L, q, seed, False))
        assert np.array_equal(gobs_all, oobs)
        N = L * L
        E = -(2 * gobs_all[:, 0] - 2 * N) / N
        M = np.abs(gobs_all[:, 1] - gobs_all[:, 2]) / N
        assert abs(E[100:].mean() - (-(2 * oobs[100:, 0] - 2 * N) / N).mean()) == 0.0
        assert 1.30 < -E[100:].mean() < 1.55 and 0.3 < M[100:].mean() < 0.95
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("L", [4, 8, 36, 100, 132, 196])
@pytest.mark.parametrize("q", [2, 3, 4])
def test_small_lattices_hot_start(L, q):
    beta = math.log(1 + math.sqrt(q))                 # Potts beta_c
    T = oracle.threshold(oracle.coupling_K(q, beta, 1.0, oracle.CONV_POTTS))
    _run_parity(L, q, T, seed=1000 + L + q, hot=True, n_sweeps=12)


@pytest.mark.parametrize("q", [5, 9, 127])
def test_many_states(q):
    T = oracle.threshold(oracle.coupling_K(q, math.log(1 + math.sqrt(q)), 1.0, oracle.CONV_POTTS))
    _run_parity(132, q, T, seed=7, hot=True, n_sweeps=6)


@pytest.mark.parametrize("T", [0, 1, 1 << 31, (1 << 32) - 1, 1 << 32])
def test_degenerate_thresholds(T):
    _run_parity(68, 2, T, seed=3, hot=True, n_sweeps=4)


def test_timed_mode_is_the_same_chain():
    T = oracle.threshold(oracle.coupling_K(2, KC, 1.0, oracle.CONV_ISING))
    _run_parity(100, 2, T, seed=11, hot=True, n_sweeps=5, sweep_graph=False)


def test_many_sweeps_per_call_and_observable_ring():
    L, q, seed = 36, 3, 5
    T = oracle.threshold(oracle.coupling_K(q, math.log(1 + math.sqrt(3)), 1.0, oracle.CONV_POTTS))
    h = sw.sw_create_threshold(L, q, T, seed, True)
    try:
        sw.sw_sweep(h, 300)
        s, obs = oracle.chain(L, q, T, seed, 0, 300, oracle.init_spins(L, q, seed, True))
        assert np.array_equal(sw.sw_observables(h, 1000), obs)
        assert np.array_equal(sw.sw_get_spins(h), s)
        # ring of 4096: after 5000 more sweeps only the last 4096 remain
        sw.sw_sweep(h, 5000)
        s2, obs2 = oracle.chain(L, q, T, seed, 300, 5000, s)
        got = sw.sw_observables(h, 8000)
        assert got.shape[0] == 4096 and np.array_equal(got, obs2[-4096:])
        assert sw.sw_get_info(h)["sweeps"] == 5300
    finally:
        sw.sw_destroy(h)


def test_set_spins_and_errors():
    L, q = 64, 3
    h = sw.sw_create_threshold(L, q, 1 << 31, 9, False)
    try:
        rng = np.random.default_rng(0)
        s = rng.integers(0, q, L * L).astype(np.int8)
        sw.sw_set_spins(h, s)
        assert np.array_equal(sw.sw_get_spins(h), s)
        sd = torch.from_numpy(np.roll(s, 5)).cuda()
        sw.sw_set_spins(h, sd)
        assert np.array_equal(sw.sw_get_spins(h), np.roll(s, 5))
        bad = s.copy()
        bad[17] = q
        with pytest.raises(sw.SwcclError):
            sw.sw_set_spins(h, bad)
        with pytest.raises(sw.SwcclError):
            sw.sw_set_spins(h, torch.from_numpy(bad).cuda())
        assert np.array_equal(sw.sw_get_spins(h), np.roll(s, 5))    # unchanged
        sw.sw_sweep(h, 2)
        s1, _, _, _ = oracle.sweep(L, q, 1 << 31, 9, 0, np.roll(s, 5))
        s2, _, _, _ = oracle.sweep(L, q, 1 << 31, 9, 1, s1)
        assert np.array_equal(sw.sw_get_spins(h), s2)
        out = torch.empty(L * L, dtype=torch.int8, device="cuda")
        sw.sw_get_spins(h, out)
        assert np.array_equal(out.cpu().numpy(), s2)
    finally:
        sw.sw_destroy(h)


def test_user_stream_and_two_handles_are_independent():
    st = torch.cuda.Stream()
    T = oracle.threshold(0.9)
    a = sw.sw_create_threshold(64, 2, T, 42, True, st)
    b = sw.sw_create_threshold(64, 2, T, 42, True)
    try:
        assert sw.sw_stream(a) == st.cuda_stream
        sw.sw_sweep(a, 7)
        sw.sw_sweep(b, 7)
        assert np.array_equal(sw.sw_get_spins(a), sw.sw_get_spins(b))
    finally:
        sw.sw_destroy(a)
        sw.sw_destroy(b)


@pytest.mark.parametrize("q,beta,conv", [(2, KC, sw.SW_CONV_ISING), (4, math.log(3.0), sw.SW_CONV_POTTS)])
def test_L16384_one_step_equivalence(q, beta, conv):
    """The benchmark's lattice: L = 16384, hot start seed 7.  Sampled sweeps 0
    and 2 (q = 2) / 0 (q = 4): the oracle steps the GPU's pre-sweep spins once
    and must reproduce the GPU's mask, labels, spins and observables."""
    L, seed = 16384, 7
    T = oracle.threshold(oracle.coupling_K(q, beta, 1.0, conv))
    h = sw.sw_create_ex(L, q, beta, 1.0, conv, seed, True)
    try:
        sw.sw_set_mode(h, sw.SW_MODE_STAGED)
        s = sw.sw_get_spins(h)
        assert np.array_equal(s[:1 << 16], oracle.init_spins(L, q, seed, True)[:1 << 16])
        samples = (0, 2) if q == 2 else (0,)
        done = 0
        for k in samples:
            if k > done:
                sw.sw_sweep(h, k - done)
                sw.sw_observables(h, 4096)
                s = sw.sw_get_spins(h)
            sw.sw_sweep(h, 1)
            done = k + 1
            gm, glab = sw.sw_debug_dump(h)
            gs = sw.sw_get_spins(h)
            gobs = sw.sw_observables(h, 4)
            s_new, m, lab, obs = oracle.sweep(L, q, T, seed, k, s)
            assert np.array_equal(gm, m)
            assert np.array_equal(glab, lab)
            assert np.array_equal(gs, s_new)
            assert np.array_equal(gobs[-1], obs)
            s = gs
    finally:
        sw.sw_destroy(h)


# ---------------------------------------------------------------------------
# Fused mode (default): bonds drawn inside the labeling kernel.  No mask or
# labels exist to dump; spins and observables are compared every sweep.
# ---------------------------------------------------------------------------
def _run_fused(L, q, T, seed, hot, n_sweeps, per_call=1, timing=False):
    h = sw.sw_create_threshold(L, q, T, seed, hot)
    try:
        if timing:
            sw.sw_set_timing(h, True)
        s = oracle.init_spins(L, q, seed, hot)
        done = 0
        while done < n_sweeps:
            k = min(per_call, n_sweeps - done)
            sw.sw_sweep(h, k)
            s, obs = oracle.chain(L, q, T, seed, done, k, s)
            assert np.array_equal(sw.sw_get_spins(h), s), ("spins", L, q, done)
            assert np.array_equal(sw.sw_observables(h, 4096), obs), ("obs", L, q, done)
            done += k
        with pytest.raises(sw.SwcclError):
            sw.sw_debug_dump(h)          # nothing to dump after a fused sweep
    finally:
        sw.sw_destroy(h)


def test_fused_ising_L64_cold_start_1000_sweeps():
    L, q, seed = 64, 2, 1
    T = oracle.threshold(oracle.coupling_K(q, KC, 1.0, oracle.CONV_ISING))
    _run_fused(L, q, T, seed, False, 1000, per_call=50)


# 256 and 512: every tile whole (the kernels without bounds checks)
@pytest.mark.parametrize("L", [4, 8, 36, 100, 132, 196, 256, 260, 292, 512])
@pytest.mark.parametrize("q", [2, 3, 4])
def test_fused_small_lattices(L, q):
    beta = math.log(1 + math.sqrt(q))
    T = oracle.threshold(oracle.coupling_K(q, beta, 1.0, oracle.CONV_POTTS))
    _run_fused(L, q, T, seed=2000 + L + q, hot=True, n_sweeps=8, per_call=3)


@pytest.mark.parametrize("L", [256, 260])
@pytest.mark.parametrize("q", [5, 9, 127])
def test_fused_many_states(L, q):
    T = oracle.threshold(oracle.coupling_K(q, math.log(1 + math.sqrt(q)), 1.0, oracle.CONV_POTTS))
    _run_fused(L, q, T, seed=8, hot=True, n_sweeps=5)


# L = 256 with T = 0: every site its own cluster, so every tile has more
# edge roots than code slots
@pytest.mark.parametrize("T", [0, 1, 1 << 31, (1 << 32) - 1, 1 << 32])
@pytest.mark.parametrize("per_call", [1, 4])
@pytest.mark.parametrize("L", [68, 256])
def test_fused_degenerate_thresholds(L, T, per_call):
    _run_fused(L, 2, T, seed=3, hot=True, n_sweeps=8, per_call=per_call)


@pytest.mark.parametrize("L", [292, 512])
def test_fused_timed_mode_and_one_sweep_per_call(L):
    T = oracle.threshold(oracle.coupling_K(2, KC, 1.0, oracle.CONV_ISING))
    _run_fused(L, 2, T, seed=12, hot=True, n_sweeps=6, timing=True)


def test_fused_timed_mode_several_sweeps_per_call():
    T = oracle.threshold(oracle.coupling_K(3, math.log(1 + math.sqrt(3)), 1.0, oracle.CONV_POTTS))
    h = sw.sw_create_threshold(292, 3, T, 21, True)
    try:
        sw.sw_set_timing(h, True)
        s = oracle.init_spins(292, 3, 21, True)
        done = 0
        for k in (3, 2, 5):
            sw.sw_sweep(h, k)
            s, obs = oracle.chain(292, 3, T, 21, done, k, s)
            assert np.array_equal(sw.sw_get_spins(h), s), done
            assert np.array_equal(sw.sw_observables(h, 4096), obs), done
            done += k
        ms, n = sw.sw_phase_times(h)
        assert n == done and all(v >= 0 for v in ms.values())
    finally:
        sw.sw_destroy(h)


# Calls of 1 to 6 fused sweeps on lattices of one tile that is its own east
# and north neighbour (L = 4, 8), ragged tiles (36, 260, 292), several
# ragged tiles each way (516) and whole tiles only (512); q = 127 counts the
# states one by one.
@pytest.mark.parametrize("L", [4, 8, 36, 260, 292, 512, 516])
@pytest.mark.parametrize("q", [2, 3, 127])
def test_fused_calls_of_several_sweeps(L, q):
    beta = math.log(1 + math.sqrt(q))
    T = oracle.threshold(oracle.coupling_K(q, beta, 1.0, oracle.CONV_POTTS))
    seed = 3000 + L + q
    h = sw.sw_create_threshold(L, q, T, seed, True)
    try:
        s = oracle.init_spins(L, q, seed, True)
        done = 0
        for k in (2, 3, 6, 1, 4, 5):
            sw.sw_sweep(h, k)
            s, obs = oracle.chain(L, q, T, seed, done, k, s)
            assert np.array_equal(sw.sw_get_spins(h), s), (L, q, done, k)
            assert np.array_equal(sw.sw_observables(h, 4096), obs), (L, q, done, k)
            done += k
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("L", [256, 260])
def test_mode_switches_keep_the_chain(L):
    """staged -> fused -> staged -> fused within one chain, with reads of the
    observables at every switch and in between (L = 256: the fused sweeps
    go through the site codes)."""
    q, seed = 3, 44
    T = oracle.threshold(oracle.coupling_K(q, math.log(1 + math.sqrt(3)), 1.0, oracle.CONV_POTTS))
    h = sw.sw_create_threshold(L, q, T, seed, True)
    try:
        s = oracle.init_spins(L, q, seed, True)
        done = 0
        all_obs = []
        for mode, n in [(sw.SW_MODE_STAGED, 3), (sw.SW_MODE_FUSED, 4), (sw.SW_MODE_STAGED, 2),
                        (sw.SW_MODE_FUSED, 5), (sw.SW_MODE_FUSED, 1)]:
            sw.sw_set_mode(h, mode)
            sw.sw_sweep(h, n)
            s, obs = oracle.chain(L, q, T, seed, done, n, s)
            done += n
            all_obs.append(obs)
            assert np.array_equal(sw.sw_get_spins(h), s)
        got = sw.sw_observables(h, 4096)
        assert np.array_equal(got, np.concatenate(all_obs))
        # set_spins after fused sweeps: the pending observables belong to the old spins
        sw.sw_sweep(h, 2)
        s, obs = oracle.chain(L, q, T, seed, done, 2, s)
        done += 2
        rng = np.random.default_rng(1)
        new = rng.integers(0, q, L * L).astype(np.int8)
        sw.sw_set_spins(h, new)
        sw.sw_sweep(h, 1)
        s2, obs2 = oracle.chain(L, q, T, seed, done, 1, new)
        assert np.array_equal(sw.sw_observables(h, 4096), np.concatenate([obs, obs2]))
        assert np.array_equal(sw.sw_get_spins(h), s2)
    finally:
        sw.sw_destroy(h)


# Sweeps of the L = 16384 benchmark chain checked by one-step equivalence:
# the first two, the end of the 100-sweep warm-up and the start of the timed
# sweeps, the middle and the last of 200 timed sweeps, plus three drawn at
# random (seeded) in between.  From sweep ~100 on the lattice carries the
# critical, lattice-spanning clusters whose merges cross every seam and the
# periodic wrap.
def _sampled_sweeps():
    rng = np.random.default_rng(16384)
    extra = sorted(int(v) for v in rng.choice(np.arange(2, 299), size=3, replace=False))
    return sorted(set([0, 1, 99, 100, 150, 299] + extra))


@pytest.mark.parametrize("q,beta,conv", [(2, KC, sw.SW_CONV_ISING), (4, math.log(3.0), sw.SW_CONV_POTTS)])
def test_fused_L16384_one_step_equivalence(q, beta, conv):
    """The benchmark's lattice: L = 16384, hot start seed 7.  A fused chain
    (the benchmark's mode, many sweeps per call) and a staged chain advance
    side by side to sweep 299.  At every sampled sweep s both chains' spins
    before the sweep must be equal; the oracle then steps those spins once
    (sweep index s), and the fused chain's spins and observables and the
    staged chain's bond mask, canonical labels, spins and observables after
    the sweep must equal the oracle's.  The oracle's sweeps run in worker
    threads while the GPU advances."""
    import concurrent.futures as cf
    import os
    L, seed = 16384, 7
    T = oracle.threshold(oracle.coupling_K(q, beta, 1.0, conv))
    samples = _sampled_sweeps()
    hf = sw.sw_create_ex(L, q, beta, 1.0, conv, seed, True)
    hs = sw.sw_create_ex(L, q, beta, 1.0, conv, seed, True)
    workers = max(2, min(len(samples), (os.cpu_count() or 2) // 2))
    pending = []

    def check(item):
        k, fut, fs, fobs, gm, glab, gs, gobs = item
        s_new, m, lab, obs = fut.result()
        assert np.array_equal(gm, m), ("mask", q, k)
        assert np.array_equal(glab, lab), ("labels", q, k)
        assert np.array_equal(gs, s_new), ("staged spins", q, k)
        assert np.array_equal(gobs, obs), ("staged observables", q, k)
        assert np.array_equal(fs, s_new), ("fused spins", q, k)
        assert np.array_equal(fobs, obs), ("fused observables", q, k)

    try:
        sw.sw_set_mode(hs, sw.SW_MODE_STAGED)
        with cf.ThreadPoolExecutor(workers) as pool:
            done = 0
            for k in samples:
                if k > done:
                    sw.sw_sweep(hf, k - done)
                    sw.sw_sweep(hs, k - done)
                    sw.sw_observables(hf, 4096)
                    sw.sw_observables(hs, 4096)
                pre = sw.sw_get_spins(hf)
                assert np.array_equal(sw.sw_get_spins(hs), pre), ("fused and staged chains differ", q, k)
                fut = pool.submit(oracle.sweep, L, q, T, seed, k, pre)
                sw.sw_sweep(hf, 1)
                sw.sw_sweep(hs, 1)
                done = k + 1
                fs = sw.sw_get_spins(hf)
                fobs = sw.sw_observables(hf, 4096)[-1]
                gm, glab = sw.sw_debug_dump(hs)
                gs = sw.sw_get_spins(hs)
                gobs = sw.sw_observables(hs, 4096)[-1]
                pending.append((k, fut, fs, fobs, gm, glab, gs, gobs))
                del pre
                while len(pending) >= workers:
                    check(pending.pop(0))
            while pending:
                check(pending.pop(0))
        assert sw.sw_get_info(hf)["sweeps"] == samples[-1] + 1
    finally:
        sw.sw_destroy(hf)
        sw.sw_destroy(hs)


# sw_sweep_io: the asynchronous pipeline step (input spins, sweeps, their
# observables and the output spins, no host wait) against the oracle chain
@pytest.mark.parametrize("L,q", [(36, 3), (256, 2), (260, 4)])
def test_sweep_io_matches_the_chain(L, q):
    T = oracle.threshold(oracle.coupling_K(q, math.log(1 + math.sqrt(q)), 1.0, oracle.CONV_POTTS))
    seed = 77 + L
    h = sw.sw_create_threshold(L, q, T, seed, True)
    try:
        s = oracle.init_spins(L, q, seed, True)
        done = 0
        rng = np.random.default_rng(L)
        out = torch.empty(L * L, dtype=torch.int8, device="cuda")
        for n, new_input in [(3, False), (1, True), (0, True), (4, False), (2, True)]:
            inp = None
            if new_input:
                s = rng.integers(0, q, L * L).astype(np.int8)
                inp = torch.from_numpy(s).cuda()
            obs = torch.zeros((max(n, 1), 1 + q), dtype=torch.int64).pin_memory()
            sw.sw_sweep_io(h, n, inp=inp, obs_out=obs if n else None, out=out)
            sw.sw_sync(h)
            s, ref = oracle.chain(L, q, T, seed, done, n, s)
            done += n
            assert np.array_equal(out.cpu().numpy(), s), (L, q, done)
            if n:
                assert np.array_equal(obs.numpy()[:n], ref), (L, q, done)
        # the rows count as read: nothing is left for sw_observables
        assert sw.sw_observables(h, 4096).shape[0] == 0
        assert np.array_equal(sw.sw_get_spins(h), s)
    finally:
        sw.sw_destroy(h)


def test_sweep_io_rejects_bad_input_on_the_device():
    L, q = 64, 3
    T = oracle.threshold(oracle.coupling_K(q, math.log(1 + math.sqrt(q)), 1.0, oracle.CONV_POTTS))
    h = sw.sw_create_threshold(L, q, T, 5, True)
    try:
        sw.sw_sweep(h, 2)
        before = sw.sw_get_spins(h)
        bad = torch.zeros(L * L, dtype=torch.int8, device="cuda")
        bad[L * L // 2] = q                       # one value outside [0, q)
        sw.sw_sweep_io(h, 0, inp=bad)             # enqueued: no error yet
        with pytest.raises(sw.SwcclError) as e:
            sw.sw_sync(h)
        assert e.value.code == sw.SW_ERR_ARG
        sw.sw_sync(h)                             # reported once
        assert np.array_equal(sw.sw_get_spins(h), before)
        # the chain goes on from the spins it kept
        s, _ = oracle.chain(L, q, T, 5, 2, 1, before)
        sw.sw_sweep(h, 1)
        assert np.array_equal(sw.sw_get_spins(h), s)
    finally:
        sw.sw_destroy(h)
