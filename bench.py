"""Benchmark: Swendsen-Wang sweeps of the periodic L = 16384 Ising lattice at
beta_c (hot start, seed 7) on one GB300, through the library's C ABI.

One step = one full sweep (activation, tile labeling, seam merge, root
compression with root draws, flip with observables).  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the serial CPU oracle (the only reference this
method has) on a bounded sample of the same workload.  With N > 1 (torchrun)
every rank runs an independent replica (seed 7 + rank): the method does not
shard, so scaling is weak and there is no collective on the data path.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KC_ISING = 0.5 * math.log(1.0 + math.sqrt(2.0))
L_BENCH, Q_BENCH, SEED_BENCH = 16384, 2, 7
# the paper's number for this metric and workload: q = 2 at beta_c, L = 16384,
# self-labeling + sewing on a Tesla M2070, 3.573 ns per site and sweep (Table I)
PAPER_SITE_UPDATES_PER_NS = 1.0 / 3.573
WORKLOAD = "sw_ising_q2_L%d_beta_c_hot_start_seed7"
# Counters of the fused sweep's kernels from one ncu capture each (--set
# full, one launch, L = 8192, the third sweep from the hot start; the
# full-size launch is too large to capture under ncu's replay, and DRAM
# bytes and instructions grow with the sites processed), per site:
# DRAM bytes = dram__bytes_read.sum + dram__bytes_write.sum, warp
# instructions = smsp__inst_executed.sum.  Valid only for the code they were
# taken with (a hash of the sources without comments); otherwise the line
# reports null.
SWEEP_COUNTER_SOURCES = ("fused_tile.cuh", "tile_engine.cuh", "k_fused.cu", "k_label.cu", "swccl_device.cuh",
                         "swccl_shared.h")
SWEEP_COUNTER_HASH = "a64f8956685ba9d7"
SWEEP_COUNTERS = {      # kernel: (DRAM bytes per site, warp instructions per site)
    "k_sw_label": ((94.285824 + 141.310976) * 1e6 / 67108864, 187239060 / 67108864),
    "k_merge": ((78.399488 + 2.301952) * 1e6 / 67108864, 16679698 / 67108864),
    "k_sw_flip": ((216.701440 + 50.096128) * 1e6 / 67108864, 93623845 / 67108864),
}
# The stand-alone labeling call (k_ccl_tile, k_merge, k_ccl_final), one ncu
# capture per kernel of a 4096^2 critical percolation mask: DRAM bytes per site,
# for the build with CCL_COUNTER_TILE_W-wide tiles, to which the binding routes
# labeling.
CCL_COUNTER_SOURCES = ("label_tile.cuh", "tile_engine.cuh", "k_label.cu", "swccl_device.cuh", "swccl_shared.h")
CCL_COUNTER_HASH = "2c55f8edeccf7c13"
CCL_COUNTER_TILE_W = 128
CCL_TRAFFIC_BYTES_PER_SITE = ((7.725056 + 5.867776) + (19.986176 + 0.001280) + (59.200256 + 10.390016)) * 1e6 / 16777216
# Algorithmic HBM bytes per site: the fused sweep reads and writes the int8
# spins once (2 B, the minimum of any sweep); the kernel split adds the
# 16-bit tile roots written by k_sw_label and read by k_sw_flip (6 B).
SWEEP_MIN_BYTES_PER_SITE = 2.0
FUSED_SWEEP_BYTES_PER_SITE = 6.0
LABEL_BYTES_PER_SITE = 3.0      # k_sw_label: spins read 1 B, tile roots written 2 B
# Philox4x32-10 calls per site made by k_sw_label: one call per pair of
# x-adjacent sites (its four words are the pair's east and north bonds)
LABEL_PHILOX_CALLS_PER_SITE = 0.5
# sweeps of the separate pass that splits the sweep time by kernel
PHASE_SWEEPS = 10


def sources_hash(files):
    """Hash of kernel sources, code only: `//` comments, trailing blanks and
    empty lines are dropped, so that an edit of the comments keeps a recorded
    capture valid."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1105_5804_gb300", "csrc", f), encoding="utf-8") as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def sweep_counters():
    """Per-site (DRAM bytes, warp instructions) of the sweep's kernels, or
    None if their code changed since the capture."""
    return SWEEP_COUNTERS if sources_hash(SWEEP_COUNTER_SOURCES) == SWEEP_COUNTER_HASH else None


def _ccl_traffic(N):
    from paper_1105_5804_gb300 import _lib
    ok = sources_hash(CCL_COUNTER_SOURCES) == CCL_COUNTER_HASH and _lib.CCL_TILE_W == CCL_COUNTER_TILE_W
    return CCL_TRAFFIC_BYTES_PER_SITE * N if ok else None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0, t1):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [l for (t, l) in self.lines if t0 - 0.1 <= t <= t1 + 0.1] or [l for (_, l) in self.lines[-3:]]
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            p = [x.strip() for x in r.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, device=None):
    """Largest value of x over all ranks (plain x without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    if device is None:
        device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Seed of the independent replica run by a rank."""
    return SEED_BENCH + rank


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_sample(seconds=15.0, L=4096):
    """The serial oracle on this host: SW sweeps of an L x L sample of the
    workload (same q, beta, seed) for about `seconds`.  Returns the dict for
    the cpu_baseline key."""
    import oracle
    T = oracle.threshold(oracle.coupling_K(Q_BENCH, KC_ISING, 1.0, oracle.CONV_ISING))
    s = oracle.init_spins(L, Q_BENCH, SEED_BENCH, True)
    t0 = time.perf_counter()
    n = 0
    while True:
        s, _ = oracle.chain(L, Q_BENCH, T, SEED_BENCH, n, 1, s)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": L * L * n / (dt * 1e9), "unit": "site-updates/ns", "cores": 1, "kind": "oracle",
            "sample": "serial C oracle, %d SW sweeps of the L=%d q=2 Ising lattice at beta_c (hot start, "
                      "seed 7) on one host core, %.1f s" % (n, L, dt),
            "cpu": _cpu_model(), "host_cores": os.cpu_count()}


def _oracle_replica(args):
    """One process of the all-cores baseline: serial oracle sweeps of an
    independent L x L replica (seed 7 + r) for about `seconds`."""
    r, L, seconds = args
    sys.path.insert(0, ROOT)
    import oracle
    T = oracle.threshold(oracle.coupling_K(Q_BENCH, KC_ISING, 1.0, oracle.CONV_ISING))
    s = oracle.init_spins(L, Q_BENCH, SEED_BENCH + r, True)
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds:
        s, _ = oracle.chain(L, Q_BENCH, T, SEED_BENCH + r, n, 1, s)
        n += 1
    return L * L * n, time.perf_counter() - t0


def oracle_all_cores(seconds=8.0, L=1024):
    """The oracle on every host core at once: one independent replica per
    process (processes started with spawn: CUDA is already initialised)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_replica, [(r, L, seconds) for r in range(cores)])
    sites = sum(a for a, _ in res)
    dt = max(b for _, b in res)
    return {"value": sites / (dt * 1e9), "unit": "site-updates/ns", "cores": cores,
            "sample": "%d independent oracle replicas of the L=%d q=2 Ising lattice at beta_c, one per core, "
                      "%.1f s" % (cores, L, dt)}


def oracle_ccl_sample(seconds=10.0, H=4096):
    """The oracle's labeling (breadth-first search) of 4096^2 critical
    percolation masks (seeds 0, 1, ...) on one host core for about
    `seconds` of labeling time (mask generation not counted)."""
    import oracle
    n, dt = 0, 0.0
    while dt < seconds:
        m = oracle.perc_mask(H, H, n)
        t0 = time.perf_counter()
        oracle.label(m, H, H, True)
        dt += time.perf_counter() - t0
        n += 1
    return {"value": H * H * n / (dt * 1e9), "unit": "Gsites/s", "cores": 1, "kind": "oracle",
            "sample": "serial oracle labeling (breadth-first search) of %d periodic %dx%d p=1/2 masks "
                      "(seeds 0..%d) on one host core, %.1f s" % (n, H, H, n - 1, dt),
            "cpu": _cpu_model()}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args):
    """--impl reference: the oracle on the host cores, each step one sweep of
    an L = 1024 sample of the workload (same q, beta_c, hot start, seed)."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    L = 1024
    T = oracle.threshold(oracle.coupling_K(Q_BENCH, KC_ISING, 1.0, oracle.CONV_ISING))
    s = oracle.init_spins(L, Q_BENCH, SEED_BENCH, True)
    for k in range(args.warmup):
        s, _ = oracle.chain(L, Q_BENCH, T, SEED_BENCH, k, 1, s)
    t0 = time.perf_counter()
    for k in range(args.steps):
        s, _ = oracle.chain(L, Q_BENCH, T, SEED_BENCH, args.warmup + k, 1, s)
    dt = time.perf_counter() - t0
    value = L * L * args.steps / (dt * 1e9)
    line = {
        "impl": "reference", "metric": "SW site-updates/ns", "value": value, "unit": "site-updates/ns",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD % L_BENCH, "L": L_BENCH, "q": Q_BENCH, "beta": KC_ISING,
                   "sample_L": L, "note": "each step is one oracle sweep of an L=1024 sample"},
        "cpu_baseline": {"value": value, "unit": "site-updates/ns", "cores": 1, "kind": "oracle",
                         "sample": "one serial oracle sweep of the L=1024 q=2 Ising lattice at beta_c per step",
                         "cpu": _cpu_model()},
        "e2e": {"value": value, "unit": "site-updates/ns", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


CCL_H = 4096
# Algorithmic HBM bytes per site of stand-alone labeling: the packed 2-bit
# mask read (0.25 B) and the int32 label written (4 B).
CCL_BYTES_PER_SITE = 4.25


def ccl_line(torch, sw, n_seeds=20, e2e_seeds=20):
    """The labeling workload (periodic 4096^2 critical percolation masks, p =
    1/2, seeds 0..n_seeds-1): each label call timed alone with events on the
    launching stream, L2 flushed in between (`value`); and end to end through
    the C ABI (`e2e`): every mask goes up from pinned host memory, is
    labeled, and its labels come down to pinned host memory, on two copy
    streams, double-buffered."""
    H = W = CCL_H
    N = H * W
    mb = sw.mask_bytes(N)
    masks = torch.empty((n_seeds, mb), dtype=torch.uint8, device="cuda")
    for k in range(n_seeds):
        sw.ccl_perc_mask(k, masks[k], H, W)
    lab = torch.empty(N, dtype=torch.int32, device="cuda")
    ws = torch.empty(sw.ccl_workspace_bytes(H, W), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    for k in range(3):
        sw.ccl_label_ws(masks[k], lab, H, W, True, ws)
    times = []
    for k in range(n_seeds):
        flush.fill_(k & 0xFF)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        sw.ccl_label_ws(masks[k], lab, H, W, True, ws)
        b.record(st)
        times.append((a, b))
    torch.cuda.synchronize()
    sw.ccl_status()
    ms = sum(a.elapsed_time(b) for a, b in times) / n_seeds
    value = N / (ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    achieved = CCL_BYTES_PER_SITE * N / (ms * 1e-3) / 1e9

    # end to end: pinned host masks up, labels down, overlapped on two copy streams
    host_m = [masks[k % n_seeds].cpu().pin_memory() for k in range(2)]
    host_l = [torch.empty(N, dtype=torch.int32).pin_memory() for _ in range(2)]
    dev_m = [torch.empty(mb, dtype=torch.uint8, device="cuda") for _ in range(2)]
    dev_l = [torch.empty(N, dtype=torch.int32, device="cuda") for _ in range(2)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ev_up = [torch.cuda.Event() for _ in range(2)]
    ev_lab = [torch.cuda.Event() for _ in range(2)]
    ev_down = [torch.cuda.Event() for _ in range(2)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(up):
        dev_m[0].copy_(host_m[0], non_blocking=True)
        ev_up[0].record(up)
    for k in range(e2e_seeds):
        b = k % 2
        if k + 1 < e2e_seeds:
            with torch.cuda.stream(up):
                dev_m[1 - b].copy_(host_m[(k + 1) % 2], non_blocking=True)
                ev_up[1 - b].record(up)
        st.wait_event(ev_up[b])
        if k >= 2:
            st.wait_event(ev_down[b])           # dev_l[b]'s previous download done
        sw.ccl_label_ws(dev_m[b], dev_l[b], H, W, True, ws)
        ev_lab[b].record(st)
        with torch.cuda.stream(down):
            down.wait_event(ev_lab[b])
            host_l[b].copy_(dev_l[b], non_blocking=True)
            ev_down[b].record(down)
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    sw.ccl_status()
    return {
        "metric": "CCL Gsites/s", "value": value, "unit": "Gsites/s", "higher_is_better": True,
        "workload": "ccl_perc_p0.5_periodic_%dx%d_seeds0-%d" % (H, W, n_seeds - 1), "ms_per_label": ms,
        "l2": "flushed (256 MiB write) between labels",
        "gpu_launches_per_label": 3,
        "roofline": {"bound": "hbm", "kernel": "ccl_label (k_ccl_tile + k_merge + k_ccl_final)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind,
                     "work_model": "%.2f B/site algorithmic (2-bit mask read, int32 label written) x %d sites per "
                                   "label call" % (CCL_BYTES_PER_SITE, N),
                     "traffic": _ccl_traffic(N)},
        "e2e": {"value": N * e2e_seeds / (te * 1e9), "unit": "Gsites/s", "labels": e2e_seeds,
                "h2d_bytes_per_step": mb, "d2h_bytes_per_step": 4 * N,
                "path": "per label: mask up from pinned host memory, ccl_label_ws, int32 labels down to pinned "
                        "host memory; copies on two streams, double-buffered"},
    }


# The rows of the paper's benchmark table (Table I) at L = 8192: q, beta/beta_c
# (delta convention, beta_c = ln(1 + sqrt q)), and the paper's GPU time per
# site and sweep on a GTX 480 with self-labeling and sewing (context only).
TABLE_ROWS = ((2, 1.0, 3.179), (2, 0.6, 1.863), (2, 1.4, 4.164), (3, 1.0, 3.059), (4, 1.0, 2.887))


def table_secondary(torch, sw, L=8192, warm=100, sweeps=100):
    """The paper's table variants: fused sweeps of an L = 8192 lattice, hot
    start seed 7, after `warm` sweeps (the ordered phase has formed at 1.4
    beta_c), timed with events on the handle's stream."""
    out = {}
    for q, ratio, paper_ns in TABLE_ROWS:
        beta = ratio * math.log(1.0 + math.sqrt(q))
        h = sw.sw_create_ex(L, q, beta, 1.0, sw.SW_CONV_POTTS, SEED_BENCH, True)
        try:
            sw.sw_sweep(h, warm)
            st = torch.cuda.ExternalStream(sw.sw_stream(h))
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            sw.sw_sweep(h, sweeps)
            b.record(st)
            torch.cuda.synchronize()
            obs = sw.sw_observables(h, 4096)
            ms = a.elapsed_time(b)
            out["q%d_beta%.1f" % (q, ratio)] = {
                "value": L * L * sweeps / (ms * 1e6), "unit": "site-updates/ns", "ms_per_sweep": ms / sweeps,
                "beta": beta, "mean_n_eq_per_site": float(obs[-sweeps:, 0].mean()) / (L * L),
                "paper_gtx480_ns_per_site": paper_ns}
        finally:
            sw.sw_destroy(h)
    return {"workload": "sw_potts_L8192_hot_start_seed7_table_rows", "warmup_sweeps": warm, "sweeps": sweeps,
            "rows": out}


def few_cluster_secondary(torch, sw, L=L_BENCH, ells=(16, 256), p_flip=0.5, warm=20, sweeps=50):
    """Few-cluster update (Sec. III, variant (c)) on the benchmark lattice:
    q = 2 at beta_c, hot start seed 7, one seed per block of an ell x ell
    grid, seeded clusters flip with probability p_flip."""
    out = {}
    for ell in ells:
        h = sw.sw_create_ex(L, Q_BENCH, KC_ISING, 1.0, sw.SW_CONV_ISING, SEED_BENCH, True)
        try:
            sw.sw_set_update(h, sw.SW_UPDATE_FEW, ell, sw.sw_prob_threshold(p_flip))
            sw.sw_sweep(h, warm)
            st = torch.cuda.ExternalStream(sw.sw_stream(h))
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            sw.sw_sweep(h, sweeps)
            b.record(st)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            out["ell%d" % ell] = {"value": L * L * sweeps / (ms * 1e6), "unit": "site-updates/ns",
                                  "ms_per_sweep": ms / sweeps, "seeds": ell * ell}
        finally:
            sw.sw_destroy(h)
    return {"workload": "sw_few_cluster_ising_q2_L%d_beta_c_hot_start_seed7_pflip%.1f" % (L, p_flip),
            "warmup_sweeps": warm, "sweeps": sweeps, "rows": out}


KC3_ISING = 0.2216546   # simple-cubic Ising critical coupling (literature value)


def cubic_secondary(torch, sw, L=512, warm=20, sweeps=50):
    """Simple-cubic lattice (the paper's 3D generalisation): q = 2 at the
    critical coupling, L^3 sites, hot start seed 7; whole sweeps timed with
    events on the handle's stream, then one timed-mode pass for the split."""
    h = sw.sw3_create_ex(L, L, L, 2, KC3_ISING, 1.0, sw.SW_CONV_ISING, SEED_BENCH, True)
    try:
        sw.sw3_sweep(h, warm)
        st = torch.cuda.ExternalStream(sw.sw3_stream(h))
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        sw.sw3_sweep(h, sweeps)
        b.record(st)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        obs = sw.sw3_observables(h, 4096)
        sw.sw3_set_timing(h, True)
        sw.sw3_sweep(h, 10)
        phases, n = sw.sw3_phase_times(h)
    finally:
        sw.sw3_destroy(h)
    N = L ** 3
    return {"workload": "sw3_ising_q2_L%d_cubed_Kc_hot_start_seed7" % L, "value": N * sweeps / (ms * 1e6),
            "unit": "site-updates/ns", "ms_per_sweep": ms / sweeps, "sweeps": sweeps, "warmup_sweeps": warm,
            "mean_n_eq_per_site": float(obs[-sweeps:, 0].mean()) / N,
            "phase_ms_per_sweep": {k: v / n for k, v in phases.items()}}


def philox_ceiling(torch, sw, reps=3):
    """Measured integer-ALU ceiling: Philox4x32-10 calls per second of a
    kernel that does nothing else, 8 CTAs x 256 threads per SM on every SM."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * 8
    calls = 4096
    sink = torch.empty(blocks * 256, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    sw.sw_probe_philox(calls, blocks, sink)
    best = None
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        sw.sw_probe_philox(calls, blocks, sink)
        b.record(st)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    return blocks * 256 * calls / (best * 1e-3)


def batch_secondary(torch, sw, sweeps=50, single_sweeps=5):
    """The batched workload: 512 independent Ising chains, L log-uniform in
    [64, 2048] (multiples of 32), beta spread over [0.9, 1.1] beta_c, seed =
    chain id, cold start.  Site-updates/ns of the autotuned batch, of each
    schedule, and of the same chains launched one at a time on one stream."""
    from paper_1105_5804_gb300 import autotune, inputs
    reps = inputs.batched_replicas()
    L = [r["L"] for r in reps]
    beta = [r["beta"] for r in reps]
    seed = [r["seed"] for r in reps]
    q = [2] * len(L)
    total = sum(l * l for l in L)
    choice = autotune.tune(L, q, beta, sw.SW_CONV_ISING, use_cache=False)
    res = {"workload": "sw_batch_512_ising_L64-2048_beta0.9-1.1betac", "chains": len(L), "sites": total,
           "unit": "site-updates/ns", "sweeps": sweeps, "autotune": choice}
    for tw in sw.TILE_WIDTHS:
        b = sw.sw_batch_create(L, q, beta, seed, sw.SW_CONV_ISING, False, tile_w=tw)
        try:
            runs = [("phases", sw.SW_BATCH_PHASES, 0), ("persistent", sw.SW_BATCH_PERSISTENT, 0)]
            if tw == choice["tile_w"]:
                runs.append(("autotuned", choice["schedule"], choice["blocks_per_sm"]))
            for name, sched, bps in runs:
                sw.sw_batch_set_schedule(b, sched, bps)
                sw.sw_batch_sweep(b, 3)
                ms = autotune.time_batch(b, sweeps)
                key = name if name == "autotuned" else "%s_tile%d" % (name, tw)
                res[key] = total * sweeps / (ms * 1e6)
            res["graph"] = bool(sw.sw_batch_info(b)["graph"])
        finally:
            sw.sw_batch_destroy(b)
    res["value"] = res["autotuned"]
    # the same chains, one handle each, launched one after another on one stream
    st = torch.cuda.Stream()
    hs = [sw.sw_create_ex(L[r], 2, beta[r], 1.0, sw.SW_CONV_ISING, seed[r], False, st) for r in range(len(L))]
    try:
        for h in hs:
            sw.sw_sweep(h, 1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(single_sweeps):
            for h in hs:
                sw.sw_sweep(h, 1)
        e1.record(st)
        torch.cuda.synchronize()
        res["one_at_a_time"] = total * single_sweeps / (e0.elapsed_time(e1) * 1e6)
    finally:
        for h in hs:
            sw.sw_destroy(h)
    res["batched_over_one_at_a_time"] = res["value"] / res["one_at_a_time"]
    return res


def serving_jobs(rate, seconds=6.0, min_jobs=200, max_jobs=2000):
    """Jobs of one rate of the serving measurement: about `seconds` of the
    stream, at least min_jobs and at most max_jobs."""
    return int(min(max_jobs, max(min_jobs, rate * seconds)))


def serving_secondary(torch, rates=(10, 30, 100, 300, 1000, 2000)):
    """The serving workload: a Poisson stream of segmentation jobs (H, W
    uniform in [256, 8192], windows of a blurred-noise 8-level image) and SW
    jobs (L uniform in [128, 4096], 10 sweeps at the Ising beta_c), 80:20.
    Two arms on the same job stream: the continuous-batching server (32 GiB
    budget, 4 slots) and one job at a time through the single-job calls.
    Latency = result in host memory (labels in pinned memory, observables
    read) - arrival.  The image pool is in pinned host memory."""
    from paper_1105_5804_gb300 import inputs, serve
    # request payloads arrive in pinned host memory (a server's receive buffers)
    pool_pinned = torch.empty((8192, 8192), dtype=torch.uint8, pin_memory=True)
    pool = pool_pinned.numpy()
    pool[:] = inputs.blurred_noise_image(8192, 8192, seed=0)
    budget = 32 << 30
    out = {"workload": "serve_label_HW256-8192_sw_L128-4096_poisson", "budget_gib": budget >> 30, "slots": 4,
           "payload": "pinned host image pool, windows uploaded by ccl_copy_pixels_2d",
           "latency": "arrival to result in host memory (labels copied to pinned memory, observables read)",
           "one_at_a_time": "the same stream, each job through ccl_label or sw_create_ex + sw_sweep + "
                            "sw_observables + sw_destroy on one stream, finished before the next starts",
           "rates": {}}
    # the same streams for every run, as a long-running server has (torch
    # caches freed device memory per stream)
    slots = [torch.cuda.Stream() for _ in range(4)]
    single = torch.cuda.Stream()
    # warm-up: allocators (device and pinned host), libraries
    serve.run(serve.make_jobs(2000.0, 500, seed=99, image_pool=pool), serve.Server(budget, streams=slots))
    serve.run_serial(serve.make_jobs(2000.0, 20, seed=98, image_pool=pool), stream=single)
    for rate in rates:
        n = serving_jobs(rate)
        srv = serve.Server(budget, streams=slots)
        res = serve.summary(serve.run(serve.make_jobs(float(rate), n, seed=0, image_pool=pool), srv))
        res["max_concurrent_groups"] = srv.max_running
        res["peak_hbm_gib"] = srv.peak_in_use / 2 ** 30
        one = serve.summary(serve.run_serial(serve.make_jobs(float(rate), n, seed=0, image_pool=pool),
                                             stream=single))
        res["one_at_a_time"] = one
        res["served_over_one_at_a_time_jobs_per_s"] = res["jobs_per_s"] / one["jobs_per_s"]
        out["rates"][str(rate)] = res
    return out


def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_1105_5804_gb300 as sw
    sw.lib()    # fails loudly when the extension is missing

    L, q = args.L, Q_BENCH
    N = L * L
    seed = replica_seed(rank)
    h = sw.sw_create_ex(L, q, KC_ISING, 1.0, sw.SW_CONV_ISING, seed, True)
    stream = torch.cuda.ExternalStream(sw.sw_stream(h))

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # warm-up (graph capture happens in the first call of graph mode)
    sw.sw_sweep(h, max(args.warmup, 3))
    sw.sw_sync(h)
    sw.sw_observables(h, 4096)

    # timed region: the sweeps as a user runs them (one captured CUDA graph per
    # sweep, replayed), events on the handle's stream
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = local
    clocks = ClockSampler(uuid)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    ev0.record(stream)
    sw.sw_sweep(h, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    barrier()
    clk = clocks.stop(t0, t1)
    ms = max_over_ranks(ev0.elapsed_time(ev1))
    obs = sw.sw_observables(h, 4096)
    # phase split, in a separate untimed pass: the same sweeps launched
    # eagerly with events between the kernels
    sw.sw_set_timing(h, True)
    sw.sw_phase_times(h)
    sw.sw_sweep(h, PHASE_SWEEPS)
    sw.sw_sync(h)
    phases, n_timed = sw.sw_phase_times(h)
    sw.sw_set_timing(h, False)
    sw.sw_observables(h, 4096)
    value = world * N * args.steps / (ms * 1e6)

    # end to end through the C ABI with host buffers: every step uploads its
    # input spins from pinned host memory, sweeps once, and reads its
    # observables and spins back to pinned host memory.  Two variants:
    #  - synchronous: sw_set_spins, sw_sweep, sw_observables, sw_get_spins one
    #    after another, host buffers passed directly;
    #  - pipelined (the line's e2e): one sw_sweep_io per step on device
    #    staging buffers (input checked on the device, observables written to
    #    pinned host memory, nothing waits for the device), the host<->device
    #    copies on their own streams, double-buffered, so the upload of step
    #    k+1 and the download of step k-1 overlap step k.
    # Every step's bytes cross the host link inside the timed region.
    e2e_steps = 0 if args.no_e2e else max(3, min(args.steps, 20))
    host_in = [torch.empty(N, dtype=torch.int8).pin_memory() for _ in range(2)]
    host_out = [torch.empty(N, dtype=torch.int8).pin_memory() for _ in range(2)]
    sw.sw_get_spins(h, host_in[0].numpy())
    host_in[1].copy_(host_in[0])
    barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for _ in range(e2e_steps):
        sw.sw_set_spins(h, host_in[0].numpy())
        sw.sw_sweep(h, 1)
        o = sw.sw_observables(h, 1)
        sw.sw_get_spins(h, host_out[0].numpy())
    te_sync = max_over_ranks(time.perf_counter() - te0)
    dev_in = [torch.empty(N, dtype=torch.int8, device="cuda") for _ in range(2)]
    dev_out = [torch.empty(N, dtype=torch.int8, device="cuda") for _ in range(2)]
    obs_host = torch.zeros((max(e2e_steps, 1), q + 1), dtype=torch.int64).pin_memory()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    cs = torch.cuda.ExternalStream(sw.sw_stream(h))
    ev_up = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_down = [torch.cuda.Event() for _ in range(2)]
    barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    if e2e_steps:
        with torch.cuda.stream(up):
            dev_in[0].copy_(host_in[0], non_blocking=True)
            ev_up[0].record(up)
    for k in range(e2e_steps):
        b = k % 2
        if k + 1 < e2e_steps:                       # next step's input goes up meanwhile
            with torch.cuda.stream(up):
                if k >= 1:
                    up.wait_event(ev_comp[1 - b])   # step k-1 has read dev_in[1 - b]
                dev_in[1 - b].copy_(host_in[1 - b], non_blocking=True)
                ev_up[1 - b].record(up)
        cs.wait_event(ev_up[b])
        if k >= 2:
            cs.wait_event(ev_down[b])               # dev_out[b]'s previous download done
        sw.sw_sweep_io(h, 1, inp=dev_in[b], obs_out=obs_host[k], out=dev_out[b])
        ev_comp[b].record(cs)
        with torch.cuda.stream(down):               # this step's result comes down meanwhile
            down.wait_event(ev_comp[b])
            host_out[b].copy_(dev_out[b], non_blocking=True)
            ev_down[b].record(down)
    torch.cuda.synchronize()
    te = max_over_ranks(time.perf_counter() - te0)
    sw.sw_sync(h)                                   # device status of the pipelined steps
    e2e_value = world * N * e2e_steps / (te * 1e9) if e2e_steps else None

    secondary = {}
    ccl = ccl_line(torch, sw) if rank == 0 and not args.no_ccl else None
    if rank == 0 and not args.no_secondary:
        h4 = sw.sw_create_ex(L, 4, math.log(3.0), 1.0, sw.SW_CONV_POTTS, SEED_BENCH, True)
        sw.sw_sweep(h4, 10)
        s4 = torch.cuda.ExternalStream(sw.sw_stream(h4))
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s4)
        sw.sw_sweep(h4, 50)
        b.record(s4)
        torch.cuda.synchronize()
        secondary["sw_potts_q4_L16384"] = {"value": N * 50 / (a.elapsed_time(b) * 1e6),
                                           "unit": "site-updates/ns", "beta": math.log(3.0), "sweeps": 50}
        sw.sw_destroy(h4)
        secondary["table_L8192"] = table_secondary(torch, sw)
        secondary["few_cluster"] = few_cluster_secondary(torch, sw)
        secondary["cubic"] = cubic_secondary(torch, sw)
        secondary["batch_512"] = batch_secondary(torch, sw)
        secondary["serving"] = serving_secondary(torch)
    sw.sw_destroy(h)

    if rank != 0:
        return
    peak_hbm, peak_kind = _peaks()
    ms_sweep = ms / args.steps
    per = {k: v / max(n_timed, 1) for k, v in phases.items()}
    label_ms = per["local"]
    philox_peak = philox_ceiling(torch, sw)
    philox_achieved = LABEL_PHILOX_CALLS_PER_SITE * N / (label_ms * 1e-3)
    mean_n_eq = float(obs[:, 0].mean()) if len(obs) else None
    # issue-slot ceiling: every SM's four schedulers issue one warp
    # instruction per cycle, at the SM clock sampled during the timed region
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    issue_peak = props.multi_processor_count * 4 * sm_mhz * 1e6
    counters = sweep_counters()
    kernel_ms = {"k_sw_label": per["local"], "k_merge": per["merge"], "k_sw_flip": per["flip"]}

    def hbm_gbs(bytes_per_site, t_ms):
        return bytes_per_site * N / (t_ms * 1e-3) / 1e9

    kernels = {}
    for k, t in kernel_ms.items():
        d = {"ms_per_launch": t}
        if counters:
            b, wi = counters[k]
            d.update({"dram_bytes_per_site": b, "hbm_frac_measured": hbm_gbs(b, t) / peak_hbm,
                      "warp_instructions_per_site": wi, "issue_frac": wi * N / (t * 1e-3) / issue_peak})
        kernels[k] = d
    roofline = {
        "bound": "alu", "kernel": "k_sw_label", "unit": "G warp-instructions/s",
        "achieved": counters["k_sw_label"][1] * N / (label_ms * 1e-3) / 1e9 if counters else None,
        "peak": issue_peak / 1e9,
        "frac": counters["k_sw_label"][1] * N / (label_ms * 1e-3) / issue_peak if counters else None,
        "peak_kind": "derived: %d SMs x 4 schedulers x 1 warp instruction per cycle x %.0f MHz (median SM clock "
                     "sampled in the timed region)" % (props.multi_processor_count, sm_mhz),
        "work_model": "warp instructions per site (ncu smsp__inst_executed.sum of one launch at L=8192, per site) "
                      "x %d sites per launch: the kernel is bound by instruction issue (Philox, bond logic, "
                      "tile labeling), not by DRAM" % N,
        "traffic": counters["k_sw_label"][0] * N if counters else None,
        "traffic_note": "bytes per launch: ncu dram__bytes_read.sum + dram__bytes_write.sum per site at L=8192 "
                        "x sites",
        "ms_per_launch": label_ms,
        "hbm_frac_algorithmic": hbm_gbs(LABEL_BYTES_PER_SITE, label_ms) / peak_hbm,
        "hbm_frac_measured": hbm_gbs(counters["k_sw_label"][0], label_ms) / peak_hbm if counters else None,
        "hbm_peak": peak_hbm, "hbm_peak_kind": peak_kind,
        "philox": {"achieved_gcall_s": philox_achieved / 1e9, "ceiling_gcall_s": philox_peak / 1e9,
                   "frac": philox_achieved / philox_peak,
                   "ceiling_kind": "measured in this run: Philox-only kernel, 8 CTAs x 256 threads per SM"},
    }
    sweep_bytes = sum(v[0] for v in counters.values()) if counters else None
    hbm_view = {
        "unit": "GB/s", "peak": peak_hbm, "peak_kind": peak_kind, "ms_per_sweep": ms_sweep,
        "measured_bytes_per_site": sweep_bytes,
        "frac_measured": hbm_gbs(sweep_bytes, ms_sweep) / peak_hbm if counters else None,
        "frac_at_2B_per_site": hbm_gbs(SWEEP_MIN_BYTES_PER_SITE, ms_sweep) / peak_hbm,
        "frac_at_6B_per_site": hbm_gbs(FUSED_SWEEP_BYTES_PER_SITE, ms_sweep) / peak_hbm,
        "models": "2 B/site: spins read and written once (any sweep's minimum); 6 B/site: plus the 16-bit tile "
                  "roots k_sw_label writes and k_sw_flip reads; measured: the three kernels' ncu DRAM bytes",
    }
    line = {
        "metric": "SW site-updates/ns", "value": value, "unit": "site-updates/ns", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_SITE_UPDATES_PER_NS,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD % L, "L": L, "q": q, "beta": KC_ISING, "convention": "ising (K=2 beta J)",
                   "start": "hot", "seed": SEED_BENCH, "replicas": world, "parallelism": "replicas",
                   "l2": "inputs larger than L2 (spins %d MiB, 16-bit tile roots %d MiB per replica)"
                         % (N >> 20, (2 * N) >> 20),
                   "timed_path": "sw_sweep replaying one captured CUDA graph per sweep; the per-kernel split comes "
                                 "from a separate pass of %d eagerly launched sweeps with events" % PHASE_SWEEPS},
        "clocks": clk,
        "gpu_launches": 4 * args.steps,
        "e2e": {"value": e2e_value, "unit": "site-updates/ns", "h2d_bytes_per_step": N,
                "d2h_bytes_per_step": N + 8 * (q + 1), "steps": e2e_steps,
                "synchronous_value": world * N * e2e_steps / (te_sync * 1e9) if e2e_steps else None,
                "path": "per step: one sw_sweep_io (input spins from a device staging buffer, checked on the "
                        "device; one sweep; its observables to pinned host memory; the spins to a device staging "
                        "buffer; no host wait); spins up from and down to pinned host memory on two copy streams, "
                        "double-buffered (upload of step k+1 and download of step k-1 overlap step k); "
                        "synchronous_value: sw_set_spins + sw_sweep(1) + sw_observables + sw_get_spins on the host "
                        "buffers directly, one after another"},
        "roofline": roofline,
        "hbm_view": hbm_view,
        "kernels": kernels,
        "phase_ms_per_sweep": per,
        "kernels_per_phase": {"local": "k_sw_label (bond draws + tile labeling)", "merge": "k_merge",
                              "flip": "k_sw_flip", "activate": "(fused into local)", "roots": "(fused into flip)"},
        "mean_n_eq_per_site": mean_n_eq / N if mean_n_eq else None,
        "secondary": secondary,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(args.cpu_seconds)
        line["cpu_baseline"]["all_cores"] = oracle_all_cores()
    if ccl is not None:
        if not args.no_cpu_baseline:
            ccl["cpu_baseline"] = oracle_ccl_sample()
        line["ccl"] = ccl
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ccl", action="store_true")
    ap.add_argument("--L", type=int, default=L_BENCH,
                    help="lattice size (profiling of smaller cases only; the benchmark is L=16384)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
