"""The serving loop (continuous batching) on the GPU.

A burst of mixed requests (segmentation jobs and Swendsen-Wang jobs of
different sizes) goes through the server with a small HBM budget and few
slots, so that admission waits for memory and slots and groups run
concurrently on different streams.  Every result must be the same as the job
computed alone: labels element by element against ccl_label of the same
image (and the oracle for a sample), SW observables and spins against a
single chain handle with the same arguments -- integer results, bit-exact.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1105_5804_gb300 as sw
from paper_1105_5804_gb300 import inputs, serve

pytestmark = pytest.mark.gpu

BETA_C = 0.5 * math.log(1 + math.sqrt(2.0))


def test_results_are_the_same_alone_and_in_the_mix():
    pool = inputs.blurred_noise_image(700, 700, seed=3)
    jobs = serve.make_jobs(rate=5000.0, n_jobs=48, seed=11, label_fraction=0.7, hw=(40, 600), sw_L=(32, 200),
                           image_pool=pool, sweeps=6)
    pixels = {j.id: np.ascontiguousarray(j.pixels) for j in jobs if j.kind == "label"}
    budget = 24 << 20
    server = serve.Server(budget, slots=3, max_group=6, keep_results=True)
    done = serve.run(jobs, server)
    assert len(done) == len(jobs)
    assert server.peak_in_use <= budget
    assert server.max_running >= 2                     # groups overlapped on the device
    s = serve.summary(done)
    assert s["p99_ms"] >= s["p50_ms"] > 0
    n_oracle = 0
    for j in done:
        if j.kind == "label":
            px = pixels[j.id]
            m = torch.empty(sw.mask_bytes(j.H * j.W), dtype=torch.uint8, device="cuda")
            sw.ccl_bonds_from_pixels(torch.from_numpy(px.reshape(-1)).cuda(), m, j.H, j.W, False)
            alone = torch.empty(j.H * j.W, dtype=torch.int32, device="cuda")
            sw.ccl_label(m, alone, j.H, j.W, False)
            got = j.labels.cpu().numpy()
            assert np.array_equal(got, alone.cpu().numpy()), j.id
            if n_oracle < 4:
                ref, _ = oracle.label(oracle.bonds_from_pixels(px, False), j.H, j.W, False)
                assert np.array_equal(got, ref), j.id
                n_oracle += 1
        else:
            h = sw.sw_create_ex(j.L, 2, BETA_C, 1.0, sw.SW_CONV_ISING, j.seed, True)
            try:
                sw.sw_sweep(h, j.sweeps)
                assert np.array_equal(j.observables, sw.sw_observables(h)), j.id
            finally:
                sw.sw_destroy(h)
    sw.ccl_status()


def test_admission_respects_budget_and_fifo():
    pool = inputs.blurred_noise_image(300, 300, seed=4)
    jobs = serve.make_jobs(rate=1e6, n_jobs=12, seed=5, label_fraction=1.0, hw=(64, 256), image_pool=pool)
    one = max(j.bytes for j in jobs)
    server = serve.Server(one + 1, slots=4, max_group=8)   # room for about one job at a time
    done = serve.run(jobs, server)
    assert len(done) == 12 and server.peak_in_use <= one + 1
    admits = [j.t_admit for j in sorted(done, key=lambda j: j.id)]
    assert admits == sorted(admits)                         # first in, first out
    with pytest.raises(ValueError):
        serve.run(serve.make_jobs(rate=1e6, n_jobs=1, seed=6, label_fraction=1.0, hw=(64, 64), image_pool=pool),
                  serve.Server(10, slots=1))
