"""Serving loop: continuous batching of labeling and Swendsen-Wang jobs.

Requests arrive over time (a Poisson stream in the benchmark).  Two kinds:

* label: an H x W image of grey levels -> the canonical labels of its
  4-neighbour equal-level clusters (open boundaries): the segmentation task the
  paper names as an application of cluster identification (Sec. I);
* sw:    an L x L Ising chain at a given beta -> n sweeps, their observables.

The server keeps a FIFO queue and a fixed number of slots, each with its own
CUDA stream.  On every step it admits queued jobs in arrival order while a
slot is free and the job's device memory fits the HBM budget; the label jobs
admitted in one step run as one ccl_label_batch call, the sw jobs as one
sw_batch, each group on a free slot's stream, so newly admitted work overlaps
on the GPU with work already running.  Completed groups (CUDA event queried,
never waited on) release their slot and memory.  Results do not depend on
what else ran: every job's computation reads only its own inputs and seed.

All computation runs in the library's kernels; torch provides device memory
(its caching allocator) and streams.  A label job's pixels (a window of a
host image, rows contiguous) are uploaded by one asynchronous 2-D copy on the
group's stream; when the host image is in pinned memory the copy is a DMA
that overlaps the server's work.  A job is done when its result is in host
memory: a label job's labels and an sw job's observables are copied to
pinned host memory on the group's stream before the group's completion
event, so the server loop never waits on a copy.  Admission allocates no device memory
through the driver: label buffers come from torch's caching allocator and an
sw group's chains are carved from one workspace of that allocator
(sw_batch_create_ws), so no cudaMalloc or cudaFree stalls the device while
other groups run.

run_serial() is the one-at-a-time counterpart: the same job stream, every
job through the plain single-job calls (ccl_label; sw_create_ex, sw_sweep,
sw_observables, sw_destroy) on one stream, each finished before the next
starts.
"""
import collections
import contextlib
import gc
import time

import numpy as np

from . import _lib as sw

LABEL_BYTES_PER_PX = 1 + 0.25 + 4          # pixels, packed mask, labels (+ workspace, counted exactly)


class PinnedPool:
    """Pinned host buffers for results, carved from one pinned arena.
    Pinning memory (cudaHostAlloc) takes milliseconds per hundred megabytes,
    far longer than a labeling job, so a server pins once, when the pool is
    made, and never while it serves.  The arena is managed as a buddy system
    of power-of-two blocks (from 64 KiB): a request takes the smallest free
    block that holds it, splitting larger ones; a freed block merges with its
    free buddy.  acquire() returns None when no block is free (the caller
    waits, like for device memory)."""

    MIN_ORDER = 16                          # 64 KiB

    def __init__(self, arena_bytes, arena=None):
        import torch
        top = max(self.MIN_ORDER, int(arena_bytes).bit_length() - 1)
        self.top = min(top, 28)                # blocks of at most 256 MiB
        n_top = max(1, int(arena_bytes) >> self.top)
        self.size = n_top << self.top
        self.arena = arena if arena is not None else torch.empty(self.size, dtype=torch.uint8, pin_memory=True)
        self.free = {k: set() for k in range(self.MIN_ORDER, self.top + 1)}
        self.free[self.top] = set(range(0, self.size, 1 << self.top))
        self.taken = {}                        # offset -> order

    def _order(self, nbytes):
        return max(self.MIN_ORDER, (max(int(nbytes), 1) - 1).bit_length())

    def acquire(self, nbytes):
        k = self._order(nbytes)
        if k > self.top:
            raise ValueError("a result of %d bytes is larger than the pool's largest block" % nbytes)
        j = k
        while j <= self.top and not self.free[j]:
            j += 1
        if j > self.top:
            return None
        off = min(self.free[j])                # lowest address first: keeps the top of the arena whole
        self.free[j].discard(off)
        while j > k:                           # split: keep the lower half, free the upper
            j -= 1
            self.free[j].add(off + (1 << j))
        self.taken[off] = k
        return self.arena[off: off + (1 << k)]

    def release(self, buf):
        off = buf.data_ptr() - self.arena.data_ptr()
        k = self.taken.pop(off)
        while k < self.top:
            buddy = off ^ (1 << k)
            if buddy not in self.free[k]:
                break
            self.free[k].discard(buddy)
            off = min(off, buddy)
            k += 1
        self.free[k].add(off)


_POOLS = {}


def pinned_pool(arena_bytes=12 << 30):
    """The process's pool of pinned result buffers (one per arena size)."""
    if arena_bytes not in _POOLS:
        _POOLS[arena_bytes] = PinnedPool(arena_bytes)
    return _POOLS[arena_bytes]


MAX_GROUP_WORK = 8 << 20          # pixels or site updates of one group (one job may exceed it)


class Job:
    __slots__ = ("id", "kind", "arrival", "H", "W", "pixels", "L", "beta", "sweeps", "seed", "bytes", "work",
                 "t_admit", "t_done", "labels", "observables", "spins", "host_buf")

    def __init__(self, jid, kind, arrival, **kw):
        self.id, self.kind, self.arrival = jid, kind, arrival
        self.H = kw.get("H")
        self.W = kw.get("W")
        self.pixels = kw.get("pixels")
        self.L = kw.get("L")
        self.beta = kw.get("beta")
        self.sweeps = kw.get("sweeps", 10)
        self.seed = kw.get("seed", jid)
        if kind == "label":
            self.bytes = int(self.H * self.W * LABEL_BYTES_PER_PX) + sw.ccl_batch_workspace_bytes([self.H], [self.W])
            self.work = self.H * self.W
        else:
            self.work = self.L * self.L * self.sweeps
            # what a batch of this one chain allocates (a group's batch takes the
            # sum of its chains' shares and one set of small tables)
            self.bytes = sw.sw_batch_device_bytes([self.L], [2])
        self.t_admit = self.t_done = None
        self.labels = self.observables = self.spins = self.host_buf = None


class _Group:
    """Jobs launched together on one slot."""

    def __init__(self, slot, jobs, kind):
        self.slot, self.jobs, self.kind = slot, jobs, kind
        self.event = None
        self.keep = []          # device buffers alive until completion
        self.batch = None       # sw_batch handle


class Server:
    def __init__(self, hbm_budget_bytes, slots=4, max_group=32, keep_results=False, pool=None, streams=None,
                 max_group_work=MAX_GROUP_WORK):
        """streams: the slots' CUDA streams (default: new ones).  A process
        that runs several servers should hand them the same streams: torch's
        caching allocator keeps freed device memory per stream, so memory
        cached for streams that are no longer used is not reused.
        max_group_work: a group takes further jobs only while its work (pixels
        of label jobs, site updates of sw jobs) stays within this bound, since
        every job of a group is done when the whole group is; a job larger
        than the bound runs as a group of its own."""
        import torch
        self.torch = torch
        self.clock = lambda: 0.0    # time since the start of run(), set by run()
        self.pool = pool or pinned_pool()
        self.budget = int(hbm_budget_bytes)
        self.in_use = 0
        self.streams = list(streams) if streams is not None else [torch.cuda.Stream() for _ in range(slots)]
        slots = len(self.streams)
        self.free_slots = list(range(slots))
        self.max_group = max_group
        self.max_group_work = max_group_work
        self.keep_results = keep_results
        self.queue = collections.deque()
        self.running = []
        self.done = []
        self.peak_in_use = 0
        self.max_running = 0

    def submit(self, job):
        self.queue.append(job)

    def idle(self):
        return not self.queue and not self.running

    # -- admission -----------------------------------------------------------
    def _admit(self, now):
        """Admit queued jobs in arrival order: the label jobs of this step form
        one group and the sw jobs another; a group needs a free slot; a job
        needs its bytes within the budget.  The first job that does not fit
        stops admission (first in, first out)."""
        groups = {"label": [], "sw": []}
        work = {"label": 0, "sw": 0}
        while self.queue:
            job = self.queue[0]
            if job.bytes > self.budget:
                raise ValueError("job %d needs %d bytes, more than the whole budget" % (job.id, job.bytes))
            grp = groups[job.kind]
            opened = sum(1 for g in groups.values() if g)
            if not grp and opened + 1 > len(self.free_slots):
                break
            if len(grp) >= self.max_group or self.in_use + job.bytes > self.budget:
                break
            if grp and work[job.kind] + job.work > self.max_group_work:
                break
            if job.kind == "label":            # its labels' pinned host buffer
                job.host_buf = self.pool.acquire(4 * job.H * job.W)
                if job.host_buf is None:
                    break
            self.queue.popleft()
            self.in_use += job.bytes
            work[job.kind] += job.work
            job.t_admit = now
            grp.append(job)
        self.peak_in_use = max(self.peak_in_use, self.in_use)
        for kind, jobs in groups.items():
            if jobs:
                self._launch(kind, jobs)

    def _launch(self, kind, jobs):
        torch = self.torch
        slot = self.free_slots.pop()
        st = self.streams[slot]
        g = _Group(slot, jobs, kind)
        with torch.cuda.stream(st):
            if kind == "label":
                masks, labels = [], []
                for j in jobs:
                    # the window goes up as it is (rows of the source image), no host repacking;
                    # the job keeps its host pixels until the group completes
                    src = j.pixels
                    if not (isinstance(src, np.ndarray) and src.ndim == 2 and src.strides[1] == 1):
                        src = j.pixels = np.ascontiguousarray(src).reshape(j.H, j.W)
                    px = torch.empty(j.H * j.W, dtype=torch.uint8, device="cuda")
                    sw.ccl_copy_pixels_2d(src, px, st)
                    m = torch.empty(sw.mask_bytes(j.H * j.W), dtype=torch.uint8, device="cuda")
                    sw.ccl_bonds_from_pixels(px, m, j.H, j.W, False, st)
                    lab = torch.empty(j.H * j.W, dtype=torch.int32, device="cuda")
                    masks.append(m)
                    labels.append(lab)
                    g.keep += [px, m]
                ws = torch.empty(sw.ccl_batch_workspace_bytes([j.H for j in jobs], [j.W for j in jobs]),
                                 dtype=torch.uint8, device="cuda")
                g.keep.append(ws)
                sw.ccl_label_batch(masks, labels, [j.H for j in jobs], [j.W for j in jobs], [False] * len(jobs),
                                   ws, st)
                for j, lab in zip(jobs, labels):
                    # the result goes to pinned host memory on the group's stream
                    host = j.host_buf[: 4 * j.H * j.W].view(torch.int32)
                    host.copy_(lab, non_blocking=True)
                    j.labels = host
                    g.keep.append(lab)
            else:
                Ls, qs = [j.L for j in jobs], [2] * len(jobs)
                ws = torch.empty(sw.sw_batch_device_bytes(Ls, qs), dtype=torch.uint8, device="cuda")
                g.keep.append(ws)
                b = sw.sw_batch_create_ws(Ls, qs, [j.beta for j in jobs], [j.seed for j in jobs], ws,
                                          sw.SW_CONV_ISING, True, st)
                sw.sw_batch_set_graph(b, False)     # a few sweeps: direct launches beat a capture
                g.batch = b
                n = max(j.sweeps for j in jobs)
                sw.sw_batch_sweep(b, n)
                for r, j in enumerate(jobs):
                    # observables to pinned host memory on the group's stream
                    host = torch.empty((n, 3), dtype=torch.int64, pin_memory=True)
                    sw.sw_batch_observables_async(b, r, 2, host)
                    j.observables = host
            g.event = torch.cuda.Event()
            g.event.record(st)
        self.running.append(g)
        self.max_running = max(self.max_running, len(self.running))

    # -- completion ----------------------------------------------------------
    def _collect(self, now):
        still = []
        for g in self.running:
            if not g.event.query():
                still.append(g)
                continue
            if g.kind == "sw":
                if self.keep_results:
                    for r, j in enumerate(g.jobs):
                        j.spins = sw.sw_batch_get_spins(g.batch, r, j.L)
                for j in g.jobs:
                    j.observables = j.observables.numpy()[: j.sweeps]
                sw.sw_batch_destroy(g.batch)
            else:
                for j in g.jobs:
                    if self.keep_results:
                        j.labels = j.labels.clone()
                    else:
                        j.labels = None
                    self.pool.release(j.host_buf)
                    j.host_buf = None
            for j in g.jobs:
                j.t_done = now
                j.pixels = None
                self.in_use -= j.bytes
                self.done.append(j)
            self.free_slots.append(g.slot)
        self.running = still

    def step(self, now):
        self._collect(now)
        self._admit(now)


def make_jobs(rate, n_jobs, seed=0, label_fraction=0.8, hw=(256, 8192), sw_L=(128, 4096), image_pool=None,
              sweeps=10, beta=0.5 * np.log(1 + np.sqrt(2.0))):
    """A Poisson stream of n_jobs requests at `rate` per second.  Label jobs
    take H, W uniform in hw and their pixels are windows of `image_pool` (a
    large blurred-noise image of grey levels); sw jobs take L uniform in sw_L
    (multiple of 4), the given beta, seed = job id."""
    from .inputs import poisson_arrivals
    rng = np.random.default_rng(seed)
    t = poisson_arrivals(rate, n_jobs, seed)
    jobs = []
    for k in range(n_jobs):
        if rng.random() < label_fraction:
            H = int(rng.integers(hw[0], hw[1] + 1))
            W = int(rng.integers(hw[0], hw[1] + 1))
            y = int(rng.integers(0, image_pool.shape[0] - H + 1))
            x = int(rng.integers(0, image_pool.shape[1] - W + 1))
            jobs.append(Job(k, "label", float(t[k]), H=H, W=W, pixels=image_pool[y:y + H, x:x + W]))
        else:
            L = 4 * int(rng.integers(sw_L[0] // 4, sw_L[1] // 4 + 1))
            jobs.append(Job(k, "sw", float(t[k]), L=L, beta=beta, sweeps=sweeps, seed=k))
    return jobs


@contextlib.contextmanager
def _no_collector_pauses():
    """Python's cyclic garbage collector stops the loop for tens of
    milliseconds when it scans a large heap; a serving loop keeps it off
    (reference counting still frees every result) and runs it afterwards."""
    was = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


def run(jobs, server, time_scale=1.0):
    """Feed jobs at their arrival times (seconds from now x time_scale) and
    step the server until all are done.  Returns the completed jobs."""
    with _no_collector_pauses():
        return _run(jobs, server, time_scale)


def _run(jobs, server, time_scale):
    torch = server.torch
    t0 = time.perf_counter()
    server.clock = lambda: time.perf_counter() - t0
    pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
    while pending or not server.idle():
        now = time.perf_counter() - t0
        while pending and pending[0].arrival * time_scale <= now:
            server.submit(pending.popleft())
        server.step(now)
        if not server.running and not server.queue and pending:
            wait = pending[0].arrival * time_scale - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.002))
    torch.cuda.synchronize()
    sw.ccl_status()             # device-side failures of any labeling group
    return server.done


def run_serial(jobs, stream=None, keep_results=False, pool=None):
    """The one-at-a-time arm: the same jobs in arrival order, each through the
    single-job calls on one stream and finished (result in host memory)
    before the next starts; a job that arrives while another runs waits.
    Returns the jobs with t_admit / t_done set (seconds from the start)."""
    with _no_collector_pauses():
        return _run_serial(jobs, stream, keep_results, pool)


def _run_serial(jobs, stream, keep_results, pool):
    import torch
    st = stream or torch.cuda.Stream()
    pool = pool or pinned_pool()
    order = sorted(jobs, key=lambda j: j.arrival)
    t0 = time.perf_counter()
    for j in order:
        wait = j.arrival - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        j.t_admit = time.perf_counter() - t0
        with torch.cuda.stream(st):
            if j.kind == "label":
                src = j.pixels
                if not (isinstance(src, np.ndarray) and src.ndim == 2 and src.strides[1] == 1):
                    src = np.ascontiguousarray(src).reshape(j.H, j.W)
                px = torch.empty(j.H * j.W, dtype=torch.uint8, device="cuda")
                sw.ccl_copy_pixels_2d(src, px, st)
                m = torch.empty(sw.mask_bytes(j.H * j.W), dtype=torch.uint8, device="cuda")
                sw.ccl_bonds_from_pixels(px, m, j.H, j.W, False, st)
                lab = torch.empty(j.H * j.W, dtype=torch.int32, device="cuda")
                sw.ccl_label(m, lab, j.H, j.W, False, st)
                buf = pool.acquire(4 * j.H * j.W)
                if buf is None:
                    raise RuntimeError("the pinned pool cannot hold one job's labels")
                host = buf[: 4 * j.H * j.W].view(torch.int32)
                host.copy_(lab, non_blocking=True)
                st.synchronize()
                j.labels = host.clone() if keep_results else None
                pool.release(buf)
            else:
                h = sw.sw_create_ex(j.L, 2, j.beta, 1.0, sw.SW_CONV_ISING, j.seed, True, st)
                try:
                    sw.sw_sweep(h, j.sweeps)
                    j.observables = sw.sw_observables(h, j.sweeps)
                    if keep_results:
                        j.spins = sw.sw_get_spins(h)
                finally:
                    sw.sw_destroy(h)
        j.t_done = time.perf_counter() - t0
        j.pixels = None
    sw.ccl_status()
    return order


def summary(done, time_scale=1.0):
    lat = np.array([j.t_done - j.arrival * time_scale for j in done])
    span = max(j.t_done for j in done) - min(j.arrival * time_scale for j in done)
    sites = sum((j.H * j.W) if j.kind == "label" else (j.L * j.L * j.sweeps) for j in done)
    return {"jobs": len(done), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "jobs_per_s": len(done) / span,
            "gsite_updates_per_s": sites / span / 1e9}
