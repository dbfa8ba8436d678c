/*
 * swccl.h -- C ABI of libswccl.so: Swendsen-Wang cluster updates of the
 * q-state Potts model and connected-component labeling of bond graphs on
 * periodic or open 2D square grids, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Weigel, "Connected component identification and cluster update on
 * GPU", arXiv:1105.5804.  The Swendsen-Wang sweep (Sec. II, the three-step
 * list after Eq. 5) is
 *   1. activation: a bond joining equal spins opens with probability
 *      p = 1 - exp(-K) (Sec. II below Eq. 4; rule of Eq. 7, Sec. II.A);
 *   2. identification of the connected components of the open-bond graph
 *      (Sec. II.B, II.C);
 *   3. a new uniformly random state for every component (Sec. II.D).
 *
 * Conventions (the paper leaves them open; every one is fixed here):
 *   - site index i = y*W + x (row-major); east of (x,y) is (x+1,y), north is
 *     (x,y+1); with periodic boundaries both wrap.
 *   - packed bond mask: byte i>>2 holds site i in bit 2*(i&3) (its east bond)
 *     and bit 2*(i&3)+1 (its north bond); ceil(N/4) bytes for N sites.
 *   - canonical labels: every site receives the smallest site index of its
 *     cluster (the label BFS gives when it seeds clusters in site order,
 *     Sec. II.B.1), so exactly one labeling is correct.
 *   - spins: int8 values 0..q-1; the Ising sigma = 1 - 2s for q = 2.
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), counter based,
 *     key = (seed_lo32, seed_hi32), counter = (c0, sweep_lo32, sweep_hi32, tag):
 *       BOND (tag 0): c0 = i>>1, word 2*(i&1) + dir (dir 0 east, 1 north);
 *       FLIP (tag 1): c0 = root (canonical label), word 0;
 *       INIT (tag 2): c0 = i, word 0, sweep 0;
 *       PERC (tag 3): key = (k, 0), sweep 0, words as BOND.
 *     A bond between equal spins opens iff r < T with the 32-bit threshold
 *     T = min(2^32, floor(p 2^32)) computed in IEEE double on the host;
 *     a cluster's new state is floor(r q / 2^32).
 *   - coupling: K = beta*J for the Potts delta convention (Eq. 1),
 *     K = 2*beta*J for +-1 Ising spins; SW_CONV_AUTO picks Ising for q = 2
 *     and Potts otherwise.  Both give p_c = sqrt(q)/(1+sqrt(q)) at the
 *     critical point.
 *
 * Threads: calls on different handles may run on different host threads.
 * One handle must not be used from two host threads at once.
 *
 * Errors: every int-returning call returns SW_OK (0) or one of the codes
 * below and sets a per-thread message readable with sw_last_error().
 * Kernels never trap: a device-side check that fails (an iteration bound
 * exceeded, which only corrupted buffers can cause) records SW_ERR_STATE in
 * a status word that the next synchronising call reports.
 */
#ifndef SWCCL_H
#define SWCCL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SW_OK 0
#define SW_ERR_ARG 1     /* invalid argument; nothing was launched           */
#define SW_ERR_OOM 2     /* device or host allocation failed                 */
#define SW_ERR_CUDA 3    /* a CUDA runtime call failed (message has details) */
#define SW_ERR_TIMEOUT 4 /* a bounded device wait ran out                    */
#define SW_ERR_STATE 5   /* a device-side consistency check failed           */

#define SW_CONV_AUTO 0   /* Ising (K = 2 beta J) for q = 2, Potts otherwise  */
#define SW_CONV_POTTS 1  /* delta coupling, Eq. 1: K = beta J                */
#define SW_CONV_ISING 2  /* +-1 spins: K = 2 beta J                          */

/* Phases timed by sw_phase_times(), in launch order. */
#define SW_PHASE_ACTIVATE 0  /* bond activation                 (Sec. II.A)   */
#define SW_PHASE_LOCAL 1     /* tile-local labeling             (Sec. II.B)   */
#define SW_PHASE_MERGE 2     /* union of roots across tile seams (Sec. II.C)  */
#define SW_PHASE_ROOTS 3     /* root compression + root draws   (Sec. II.C/D) */
#define SW_PHASE_FLIP 4      /* cluster flip + observables      (Sec. II.D)   */
#define SW_N_PHASES 5

/* How a handle runs a sweep (sw_set_mode).  Both compute the same chain,
 * bit for bit.
 *   SW_MODE_FUSED (default): the bonds are drawn inside the labeling kernel
 *     (the draws are counter-based, so they can be made where they are
 *     used); neither the bond mask nor per-site int32 labels go through
 *     device memory: three kernels per sweep.  Phase times: the drawing and
 *     local labeling kernel counts as SW_PHASE_LOCAL, the flip kernel (root
 *     lookup, draws, spins) as SW_PHASE_FLIP; ACTIVATE and ROOTS are zero.
 *   SW_MODE_STAGED: one kernel per step (activation writing the packed
 *     mask, local labeling writing int32 labels, merge, root compression,
 *     flip); required by sw_debug_dump. */
#define SW_MODE_STAGED 0
#define SW_MODE_FUSED 1

typedef struct sw_handle sw_handle;

/* Message of the last failed call on this host thread ("" if none).  The
 * string is owned by the library and stays valid until the next call. */
const char* sw_last_error(void);

/* The 32-bit activation threshold T for (q, beta, J, convention), as the
 * create calls compute it: T = min(2^32, floor((1 - exp(-K)) 2^32)).
 * Returns 0 for K <= 0. */
uint64_t sw_threshold_for(int q, double beta, double J, int convention);

/* ------------------------------------------------------------------------ */
/* Swendsen-Wang chain on one periodic L x L lattice                         */
/* ------------------------------------------------------------------------ */

/* Create a chain: L x L periodic lattice, q states, inverse temperature beta,
 * J = 1, SW_CONV_AUTO, cold start (every s = 0), its own CUDA stream.
 * Requirements: 4 <= L <= 46340, L % 4 == 0; 2 <= q <= 127; beta >= 0.
 * The library owns all device memory of the chain (spins, mask, labels,
 * 16-bit tile roots, root lists, seam records, a ring of per-sweep
 * observables); about 15.8 bytes per site.  Sweeps run in SW_MODE_FUSED.
 * Returns NULL on failure (see sw_last_error()). */
sw_handle* sw_create(int L, int q, double beta, uint64_t seed);

/* As sw_create with explicit coupling J, convention (SW_CONV_*), hot start
 * (hot_start != 0: s_i = floor(r q / 2^32) from the INIT draw) and stream
 * (a cudaStream_t; NULL makes the handle create its own non-blocking stream).
 * All work of the handle is ordered on that stream. */
sw_handle* sw_create_ex(int L, int q, double beta, double J, int convention, uint64_t seed,
                        int hot_start, void* stream);

/* As sw_create_ex with the threshold given directly, 0 <= T <= 2^32 (tests;
 * T = 2^32 opens every bond between equal spins). */
sw_handle* sw_create_threshold(int L, int q, uint64_t T, uint64_t seed, int hot_start, void* stream);

/* Free every device resource of the handle (waits for its stream first).
 * NULL is accepted. */
int sw_destroy(sw_handle* h);

/* Enqueue n >= 0 sweeps (Sec. II: activate, identify, flip) on the handle's
 * stream and return without waiting.  Sweep k of the chain (k = 0 for the
 * first sweep after create) draws its bonds and flips with sweep index k.
 * After each sweep the observables (n_eq, n_0..n_{q-1}) of the new spins
 * are stored in a device ring of the last 4096 sweeps. */
int sw_sweep(sw_handle* h, int n);

/* Wait for the handle's stream; report SW_ERR_STATE if a device check failed. */
int sw_sync(sw_handle* h);

/* Copy observables of sweeps not yet read, oldest first, to host memory:
 * out[k*(1+q) + 0] = n_eq = number of lattice bonds joining equal spins
 * (H = -J n_eq in the Potts convention of Eq. 1; E = -J (2 n_eq - 2N) for
 * Ising), out[k*(1+q) + 1 + s] = number of sites in state s.  At most
 * max_sweeps entries are written; *n_written receives the count.  Entries
 * older than the ring (4096 sweeps) are dropped.  Synchronises the stream. */
int sw_observables(sw_handle* h, int64_t* out, int max_sweeps, int* n_written);

/* Copy the current spins (int8[L*L], row-major) out, to host memory
 * (is_device == 0) or device memory (is_device != 0).  Synchronises. */
int sw_get_spins(sw_handle* h, int8_t* dst, int is_device);

/* Replace the current spins from host (is_device == 0) or device memory;
 * values must be in [0, q): otherwise SW_ERR_ARG and the spins are left
 * unchanged.  Host input is copied into the handle's label buffer and
 * checked on the device, so sw_debug_dump has nothing to report until the
 * next sweep.  Synchronises. */
int sw_set_spins(sw_handle* h, const int8_t* src, int is_device);

/* One step of a pipeline, fully asynchronous on the handle's stream (no call
 * in it waits for the device):
 *  - in != NULL: device memory, int8[L*L]; the spins are replaced by it if
 *    every value is in [0, q) (checked on the device, as sw_set_spins), else
 *    they stay unchanged and SW_ERR_ARG is noted in the handle's device
 *    status word, returned once by the next call that reads it (sw_sync,
 *    sw_observables, sw_get_spins).  The input must stay valid until the
 *    stream has passed this call.
 *  - n sweeps (0 <= n <= 4096), as sw_sweep.
 *  - obs_out != NULL (and n > 0): the observables of these n sweeps, n rows
 *    of 1 + q int64 as in sw_observables, written to obs_out (pinned host or
 *    device memory) in stream order; they count as read.
 *  - out != NULL: device memory, int8[L*L], receives the spins after the
 *    sweeps.
 * Results are ready when the stream reaches the end of the call (an event
 * recorded on sw_stream(h), or sw_sync).  Returns SW_OK, or SW_ERR_ARG /
 * SW_ERR_CUDA for what the host can see when enqueueing. */
int sw_sweep_io(sw_handle* h, const int8_t* in, int n, int64_t* obs_out, int8_t* out);

/* Copy the bond mask (ceil(L*L/4) bytes, packed as above) and the canonical
 * labels (int32[L*L]) of the last completed sweep, for bit-exact checks.
 * Either pointer may be NULL.  SW_ERR_STATE if the last sweep did not run in
 * SW_MODE_STAGED, or no sweep ran since creation or since the last host
 * sw_set_spins.  Synchronises. */
int sw_debug_dump(sw_handle* h, uint8_t* mask_out, int32_t* labels_out, int is_device);

/* info[0..7] = L, q, T, seed, sweeps enqueued so far, observable ring
 * capacity, tile height, tile width. */
int sw_get_info(sw_handle* h, int64_t* info);

/* Select SW_MODE_STAGED or SW_MODE_FUSED for the following sweeps (see
 * above); the chain continues unchanged.  Synchronises. */
int sw_set_mode(sw_handle* h, int mode);

/* The CUDA stream (cudaStream_t) all work of the handle is ordered on. */
void* sw_stream(sw_handle* h);

/* Per-phase timing.  With timing on, sw_sweep launches each phase directly
 * with CUDA events between phases (no graph); with it off (default) one
 * sweep is a captured CUDA graph.  Both compute the same chain. */
int sw_set_timing(sw_handle* h, int enable);

/* Milliseconds spent in each phase (ms[SW_N_PHASES]) summed over the sweeps
 * timed since the last call, and their number.  Synchronises and resets. */
int sw_phase_times(sw_handle* h, double* ms, int64_t* n_sweeps);

/* ------------------------------------------------------------------------ */
/* Few-cluster update (Sec. III, variant (c) of the single-cluster algorithm) */
/* ------------------------------------------------------------------------ */

/* The update a sweep applies after drawing the bonds and identifying the
 * clusters (sw_set_update):
 *   SW_UPDATE_SW (default): every cluster takes a new state (Sec. II.D);
 *   SW_UPDATE_FEW: the few-cluster update.  The lattice is cut into an
 *     ell x ell grid of blocks of side B = L / ell (the paper's tiles); each
 *     sweep draws one seed site per block: for block b = by*ell + bx the
 *     Philox draw w with counter (b, sweep_lo, sweep_hi, 4) gives
 *     x = bx*B + F_B(w0), y = by*B + F_B(w1), F_m(v) = floor(v m / 2^32).
 *     Every cluster holding at least one seed is selected; a selected
 *     cluster with root R (its minimum site index) and FLIP draw v (as in
 *     SW: counter (R, sweep_lo, sweep_hi, 1)) moves iff (uint64)v1 < P, from
 *     its state s to (s + 1 + F_{q-1}(v0)) mod q (for q = 2: s -> 1 - s);
 *     all other clusters keep their spins.  The bonds and clusters are those
 *     of the SW sweep with the same arguments.  P = p_flip 2^32 (see
 *     sw_prob_threshold); the paper asks p_flip < 1 for ergodicity, P = 2^32
 *     (always flip) is accepted too.
 * Cost: the SW sweep plus a memset of L*L/8 bytes and one thread per seed
 * (two tile-root reads and, for a cluster that leaves its tile, one root
 * lookup). */
#define SW_UPDATE_SW 0
#define SW_UPDATE_FEW 1

/* Select the update of the following sweeps.  For SW_UPDATE_FEW: ell >= 1
 * with L % ell == 0 and P <= 2^32 (ignored for SW_UPDATE_SW).  The few-
 * cluster update runs in SW_MODE_FUSED only: SW_ERR_STATE in staged mode
 * (and sw_set_mode(SW_MODE_STAGED) then fails likewise).  Allocates L*L/8
 * bytes of device memory on first use.  Synchronises. */
int sw_set_update(sw_handle* h, int update, int ell, uint64_t P);

/* min(2^32, floor(p 2^32)) for p in [0, 1]; UINT64_MAX for p outside. */
uint64_t sw_prob_threshold(double p);

/* ------------------------------------------------------------------------ */
/* Simple-cubic lattice (the paper's three-dimensional generalisation,      */
/* Secs. II and II.B: the same three steps with six neighbours)             */
/* ------------------------------------------------------------------------ */

/* A chain on the periodic X x Y x Z simple-cubic lattice: int8 spins, site
 * i = (z*Y + y)*X + x.  Each site owns its bonds to (x+1, y, z), (x, y+1, z)
 * and (x, y, z+1); bond d of site i is open iff the spins are equal and word
 * d of the Philox draw with counter (i, sweep_lo, sweep_hi, 5) is below T
 * (Eq. 7; no draw when T is 0 or 2^32).  Clusters, canonical labels (the
 * cluster's minimum site index), the flip (FLIP draw keyed by the root,
 * F_q of word 0) and the observables (n_eq over the 3N bonds, then n_k) are
 * as on the square lattice.  Hot start: INIT draw of site i as in 2D.
 * Requires X, Y, Z >= 1 with X*Y*Z <= 2^30, 2 <= q <= 127, T <= 2^32.  The
 * library owns the device memory: about 23 bytes per site (spins, brick
 * roots, parent array, labeling scratch) plus the observable ring.  NULL on failure (see sw_last_error).  Each sweep is
 * three kernels (brick-local union-find with the previous sweep's
 * observables, face merge, flip) and a counter advance, replayed as a
 * captured CUDA graph unless timing is on. */
typedef struct sw3_handle sw3_handle;
#define SW3_N_PHASES 4   /* local (+ observables), merge, flip, advance */

sw3_handle* sw3_create(int X, int Y, int Z, int q, uint64_t T, uint64_t seed, int hot_start, void* stream);
sw3_handle* sw3_create_ex(int X, int Y, int Z, int q, double beta, double J, int convention, uint64_t seed,
                          int hot_start, void* stream);
int sw3_destroy(sw3_handle* h);

/* n sweeps, asynchronously on the handle's stream. */
int sw3_sweep(sw3_handle* h, int n);

/* Waits for the stream; reports device-side failures (SW_ERR_STATE). */
int sw3_sync(sw3_handle* h);

/* Per-sweep (n_eq, n_0 .. n_{q-1}) not yet read, oldest first, at most
 * max_sweeps rows of 1 + q int64 (the ring keeps the last 4096).
 * Synchronises. */
int sw3_observables(sw3_handle* h, int64_t* out, int max_sweeps, int* n_written);

/* Copy the spins (int8[X*Y*Z]) out / in, host (is_device == 0) or device
 * memory; set_spins rejects values outside [0, q) with SW_ERR_ARG and keeps
 * the old spins.  Synchronise. */
int sw3_get_spins(sw3_handle* h, int8_t* dst, int is_device);
int sw3_set_spins(sw3_handle* h, const int8_t* src, int is_device);

/* Canonical labels (int32[X*Y*Z]) of the clusters of the last sweep, for
 * bit-exact checks.  SW_ERR_STATE before the first sweep and after a host
 * sw3_set_spins.  Synchronises. */
int sw3_labels(sw3_handle* h, int32_t* out, int is_device);

void* sw3_stream(sw3_handle* h);

/* info[0..7] = X, Y, Z, q, T, seed, sweeps enqueued, observable ring size. */
int sw3_get_info(sw3_handle* h, int64_t* info);

/* Per-phase timing as sw_set_timing / sw_phase_times, SW3_N_PHASES phases. */
int sw3_set_timing(sw3_handle* h, int enable);
int sw3_phase_times(sw3_handle* h, double* ms, int64_t* n_sweeps);

/* ------------------------------------------------------------------------ */
/* Batches of independent chains (no counterpart in the paper: many         */
/* replicas of uneven size and temperature advanced together)               */
/* ------------------------------------------------------------------------ */

/* How a batch runs one sweep of all its chains (the fused sweep of every
 * chain: draw + label, merge, flip):
 *   SW_BATCH_PHASES: one launch per step over the tiles of all chains;
 *   SW_BATCH_PERSISTENT: one cooperative launch per sweep; its CTAs walk the
 *     tiles of all chains step by step with grid barriers in between.  A
 *     barrier wait is bounded (SW_BATCH_BARRIER_LIMIT_DEFAULT clock64()
 *     cycles, about 2 s at 2 GHz, or the value of
 *     sw_batch_set_barrier_limit): on expiry the kernel records
 *     SW_ERR_TIMEOUT and returns; sw_batch_sync, sw_batch_observables and
 *     sw_batch_get_spins report it.  The chains are then invalid and the
 *     batch refuses further sweeps with SW_ERR_STATE: destroy it.
 * One sweep of either schedule is captured as a CUDA graph and replayed
 * (direct launches if capture is refused).  Both give, for every chain, the
 * same result bit for bit as a single handle with the same arguments. */
#define SW_BATCH_PHASES 0
#define SW_BATCH_PERSISTENT 1
#define SW_BATCH_BARRIER_LIMIT_DEFAULT 4000000000LL

typedef struct sw_batch sw_batch;

/* n chains; chain r: L[r] x L[r] periodic lattice (4 <= L <= 46340,
 * L % 4 == 0), q[r] states, inverse temperature beta[r], seed[r]; J = 1 and
 * the coupling convention are shared; hot_start as in sw_create_ex.  The
 * arrays are host memory, read during the call.  The batch owns all device
 * memory (about 15.8 bytes per site plus a 4096-sweep observable ring per
 * chain) and orders its work on `stream` (NULL: its own stream).  Default
 * schedule SW_BATCH_PHASES.  NULL on failure (sw_last_error()). */
sw_batch* sw_batch_create(int n, const int* L, const int* q, const double* beta, const uint64_t* seed,
                          int convention, int hot_start, void* stream);

/* Bytes of device memory a batch of these chains takes (what sw_batch_create
 * allocates; the workspace size sw_batch_create_ws needs); -1 if a size is
 * invalid.  L, q: host arrays of n entries. */
int64_t sw_batch_device_bytes(int n, const int* L, const int* q);

/* As sw_batch_create, with every device buffer of the batch carved from the
 * caller's `workspace` (device memory, 256-byte aligned, at least
 * sw_batch_device_bytes(n, L, q) bytes), so that creating the batch
 * allocates no device memory: a server that keeps a pool of device memory
 * admits jobs without cudaMalloc.  Returns without waiting: the
 * initialisation is ordered on `stream`.  The workspace must outlive the
 * batch; sw_batch_destroy does not free it.  NULL on failure. */
sw_batch* sw_batch_create_ws(int n, const int* L, const int* q, const double* beta, const uint64_t* seed,
                             int convention, int hot_start, void* workspace, int64_t ws_bytes, void* stream);

/* enable = 0: sweeps are launched directly instead of from a captured CUDA
 * graph (for a batch that runs only a few sweeps, the capture costs more
 * than it saves); enable = 1 (default): capture one sweep, replay it. */
int sw_batch_set_graph(sw_batch* b, int enable);

/* Free the batch (waits for its stream).  NULL is accepted. */
int sw_batch_destroy(sw_batch* b);

/* Select the schedule for the following sweeps; blocks_per_sm caps the
 * persistent kernel's CTAs per SM (0: as many as fit). */
int sw_batch_set_schedule(sw_batch* b, int schedule, int blocks_per_sm);

/* Bound of one grid-barrier wait of the persistent schedule, in clock64()
 * cycles (>= 0; default SW_BATCH_BARRIER_LIMIT_DEFAULT).  With 0 every CTA
 * but the last to arrive gives up at once, so the next persistent sweep
 * reports SW_ERR_TIMEOUT without waiting: a way to exercise the failure path
 * (the batch is invalid afterwards).  Takes effect at the next sweep. */
int sw_batch_set_barrier_limit(sw_batch* b, long long cycles);

/* Enqueue n sweeps of every chain; returns without waiting.  SW_ERR_STATE
 * (nothing enqueued) once a device-side failure of this batch was reported. */
int sw_batch_sweep(sw_batch* b, int n);

/* Wait; report SW_ERR_TIMEOUT / SW_ERR_STATE recorded by the device. */
int sw_batch_sync(sw_batch* b);

/* Observables of chain `replica` as sw_observables (own read position per
 * chain).  Synchronises. */
int sw_batch_observables(sw_batch* b, int replica, int64_t* out, int max_sweeps, int* n_written);

/* As sw_batch_observables, enqueued on the batch's stream without waiting:
 * the rows go to `dst` (pinned host or device memory: a pageable
 * destination makes the copy synchronous) once the work before them on the
 * stream is done; *n_written is the number of rows that will arrive.  No
 * device-status check: sw_batch_sync reports failures.  A server uses it to
 * have the results in host memory when the batch's work completes, without
 * a host wait per result. */
int sw_batch_observables_async(sw_batch* b, int replica, int64_t* dst, int max_sweeps, int* n_written);

/* Spins of chain `replica` (int8[L*L]) to host or device memory.  Synchronises. */
int sw_batch_get_spins(sw_batch* b, int replica, int8_t* dst, int is_device);

/* info[0..7] = chains, total sites, total tiles, sweeps enqueued, schedule,
 * persistent CTAs, 1 if the current schedule runs from a captured graph,
 * observable ring capacity. */
int sw_batch_info(sw_batch* b, int64_t* info);

/* The CUDA stream of the batch. */
void* sw_batch_stream(sw_batch* b);

/* ------------------------------------------------------------------------ */
/* Connected-component labeling of a bond mask (Sec. II.B, II.C)             */
/* ------------------------------------------------------------------------ */

/* Label the clusters of the open-bond graph of an H x W grid.
 * bond_mask: device pointer, ceil(H*W/4) bytes, packed layout above.
 * labels: device pointer, int32[H*W]; receives canonical labels.
 * periodic != 0: east/north bonds of the last column/row wrap around;
 * periodic == 0: those bonds are ignored (image segmentation).
 * Requires H, W >= 1 and H*W < 2^31.  Enqueued on `stream` (a
 * cudaStream_t, NULL = legacy default stream); returns without waiting.
 * Scratch memory (about 8.3 bytes per site) is taken with cudaMallocAsync
 * on the same stream and released in stream order. */
int ccl_label(const uint8_t* bond_mask, int32_t* labels, int H, int W, int periodic, void* stream);

/* Bytes of scratch ccl_label_ws needs for an H x W grid (-1 if invalid). */
int64_t ccl_workspace_bytes(int H, int W);

/* ccl_label with caller-owned scratch: `workspace` is a device pointer of
 * at least ccl_workspace_bytes(H, W) bytes, 256-byte aligned.  Calls that
 * share a workspace must be ordered (same stream or synchronised). */
int ccl_label_ws(const uint8_t* bond_mask, int32_t* labels, int H, int W, int periodic,
                 void* workspace, int64_t ws_bytes, void* stream);

/* Bond mask of an image (Potts mapping of segmentation, Sec. I): a bond is
 * open iff its two pixels have the same value.  px: device uint8[H*W];
 * mask: device, ceil(H*W/4) bytes.  With periodic == 0 bonds leaving the
 * grid are closed. */
int ccl_bonds_from_pixels(const uint8_t* px, uint8_t* mask, int H, int W, int periodic, void* stream);

/* Copy an H x W uint8 image whose rows are `src_pitch` bytes apart (a window
 * of a larger image) into the packed device array dst[H*W], asynchronously
 * on `stream`, without a host-side repacking (no counterpart in the paper:
 * the upload step of a labeling request).  src is host memory
 * (src_is_device == 0; pinned memory makes the copy a DMA that overlaps the
 * caller) or device memory.  The caller keeps src alive until the stream has
 * passed the copy.  SW_ERR_ARG for null pointers, H or W < 1, or
 * src_pitch < W. */
int ccl_copy_pixels_2d(const uint8_t* src, int64_t src_pitch, uint8_t* dst, int H, int W, int src_is_device,
                       void* stream);

/* Critical bond percolation mask (p = 1/2) of seed k: each of the 2*H*W
 * bond bits is open iff its PERC draw is below 2^31.  mask: device,
 * ceil(H*W/4) bytes. */
int ccl_perc_mask(uint64_t k, uint8_t* mask, int H, int W, void* stream);

/* Bytes of the fixed scratch array of ccl_label_noalloc (64 MiB).  Every GPU
 * that loads the library holds this much device memory until the process
 * exits.  A grid fits when ccl_workspace_bytes(H, W) is not larger, about
 * 8.3 bytes per site: up to about 7.9 million sites, e.g. 2816 x 2816. */
#define CCL_NOALLOC_SCRATCH_BYTES (64LL << 20)

/* ccl_label for callers that cannot allocate device memory when they label:
 * latency-bound loops (a labeling server) that must not call cudaMalloc or
 * cudaFree, because cudaFree synchronises the whole device and stalls every
 * other stream; and programs whose device memory belongs to another
 * framework's caching allocator, where an allocation behind its back can fail
 * (that allocator holds the free memory) or break its accounting.
 * The paper has no counterpart: it is a deployment variant of ccl_label.
 * Same arguments, layout and result as ccl_label; no cudaMalloc, cudaFree or
 * other allocating call is made.  Its scratch is one file-scope device array
 * of CCL_NOALLOC_SCRATCH_BYTES shared by all calls on a device, which keeps
 * the last call's contents (the kernels overwrite every part they read, so
 * nothing needs clearing).  Consequently two calls whose work overlaps on
 * the GPU (different streams, not ordered) race on that array and give
 * wrong labels: order them.  The first call on each device looks up the
 * array's device address and that of the labeling status word (the latter
 * also by the first call of any other ccl_* entry point), with that device
 * current (with lazy module loading the driver places the array in device
 * memory then); make that first call before any stream capture.  Grids whose
 * scratch exceeds CCL_NOALLOC_SCRATCH_BYTES are rejected with SW_ERR_ARG
 * before anything is launched.  Device-side failures are reported by
 * ccl_status(). */
int ccl_label_noalloc(const uint8_t* bond_mask, int32_t* labels, int H, int W, int periodic, void* stream);

/* Bytes of workspace ccl_label_batch needs for n grids of sizes H[j] x W[j]
 * (host arrays); -1 if a size is invalid. */
int64_t ccl_batch_workspace_bytes(int n, const int* H, const int* W);

/* Label n grids with one set of launches per 32 grids (one launch per step
 * over the tiles of those grids, which the kernels receive by value, so the
 * call copies nothing from host memory and never waits for the stream);
 * grid j: mask masks[j] -> labels labels[j] (device pointers, layouts as
 * ccl_label), H[j] x W[j], periodic[j].  The pointer and size arrays are
 * host memory, read during the call.  `workspace` is a
 * device pointer of at least ccl_batch_workspace_bytes(n, H, W) bytes,
 * 256-byte aligned; calls sharing a workspace must be ordered.  Each grid's
 * labels equal what ccl_label gives for it alone.  The paper labels one
 * lattice at a time; this batched form serves many small jobs (image
 * segmentation requests) with few launches.  Device-side failures are
 * reported by ccl_status(). */
int ccl_label_batch(int n, const uint8_t* const* masks, int32_t* const* labels, const int* H, const int* W,
                    const int* periodic, void* workspace, int64_t ws_bytes, void* stream);

/* Wait for the whole device and return the first device-side failure
 * recorded by ccl_* kernels since the last call (SW_OK if none); clears it. */
int ccl_status(void);

/* ------------------------------------------------------------------------ */
/* Measurement helper (not part of the method)                               */
/* ------------------------------------------------------------------------ */

/* Enqueue a kernel of `blocks` x 256 threads that only evaluates
 * Philox4x32-10: every thread makes calls_per_thread (a positive multiple of
 * 4) independent calls and stores one folded word to sink[thread]
 * (device, blocks*256 uint32).  Timing it gives the integer-ALU ceiling of
 * the bond draws (Philox4x32-10 calls per second), the bound of the
 * activation kernels. */
int sw_probe_philox(int64_t calls_per_thread, int blocks, uint32_t* sink, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SWCCL_H */
