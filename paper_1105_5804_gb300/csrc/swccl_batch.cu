// swccl_batch.cu -- C ABI of batched Swendsen-Wang chains (include/swccl.h).
//
// A batch owns R independent chains of different sizes, couplings and seeds
// and advances them together: every sw_batch_sweep call runs the fused sweep
// (draw + label, merge, flip) of all chains, either as one launch per step
// over the global tile list (SW_BATCH_PHASES) or as one persistent
// cooperative launch per sweep (SW_BATCH_PERSISTENT); one sweep of either
// schedule is captured once as a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "swccl_shared.h"

using namespace swccl;

namespace {
constexpr int BATCH_OBS_CAP = 4096;

inline int64_t al256(int64_t b) { return (b + 255) & ~(int64_t)255; }
}  // namespace

struct sw_batch {
  int n = 0;
  std::vector<int> L, q;
  std::vector<uint64_t> T, seed;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* arena = nullptr;          // control block, tables, and spins, roots, parents, scratch, rings of all chains
  bool own_arena = false;         // false: the caller's workspace (sw_batch_create_ws)
  bool use_graph = true;
  SwRep* d_reps = nullptr;
  int* d_tile_rep = nullptr;
  BatchCtl* ctl = nullptr;
  std::vector<SwRep> reps;
  BatchView view{};
  int schedule = SW_BATCH_PHASES;
  int blocks = 0;                 // persistent CTAs
  long long barrier_limit = SW_BATCH_BARRIER_LIMIT_DEFAULT;   // clock64() cycles per barrier wait
  int failed = 0;                 // device-side failure reported: the chains are invalid
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  bool graph_failed[2] = {false, false};
  uint64_t sweeps = 0;
  std::vector<uint64_t> obs_read;
  bool final_obs_pending = false;
  int64_t total_sites = 0;
};

namespace {

void free_batch(sw_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int k = 0; k < 2; ++k) {
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
    if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
  }
  if (b->own_arena) cudaFree(b->arena);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

cudaError_t enqueue_batch_sweep(sw_batch* b) {
  cudaError_t e;
  if (b->schedule == SW_BATCH_PERSISTENT)
    return launch_batch_persistent(b->view, b->ctl, b->blocks, b->barrier_limit, b->stream);
  if ((e = launch_batch_label(b->view, b->ctl, b->stream))) return e;
  if ((e = launch_batch_merge(b->view, b->stream))) return e;
  if ((e = launch_batch_flip(b->view, b->ctl, b->stream))) return e;
  return launch_batch_advance(b->view, b->ctl, b->stream);
}

// Forget the captured sweep of schedule k (its launch arguments changed).
void drop_graph(sw_batch* b, int k) {
  if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
  if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
  b->exec[k] = nullptr;
  b->graph[k] = nullptr;
  b->graph_failed[k] = false;
}

cudaError_t finish_batch_observables(sw_batch* b) {
  if (!b->final_obs_pending) return cudaSuccess;
  b->final_obs_pending = false;
  return launch_batch_observe(b->view, b->ctl, b->stream);
}

int batch_status(sw_batch* b) {
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return set_last_error(SW_ERR_CUDA, std::string("batch: ") + cudaGetErrorString(e));
  BatchCtl c;
  e = cudaMemcpyAsync(&c, b->ctl, sizeof(c), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return set_last_error(SW_ERR_CUDA, std::string("batch: ") + cudaGetErrorString(e));
  if (c.err) b->failed = c.err;
  if (c.err == SW_ERR_TIMEOUT)
    return set_last_error(SW_ERR_TIMEOUT, "batch: a grid barrier of the persistent sweep timed out; "
                                          "the chains are invalid, destroy the batch");
  if (c.err) return set_last_error(c.err, "batch: a device-side consistency check failed; "
                                          "the chains are invalid, destroy the batch");
  return SW_OK;
}

}  // namespace

namespace {

bool valid_chains(int n, const int* L, const int* q, const double* beta, const char* who) {
  if (n < 1 || !L || !q) {
    set_last_error(SW_ERR_ARG, std::string(who) + ": need n >= 1 and non-null arrays");
    return false;
  }
  for (int r = 0; r < n; ++r) {
    if (L[r] < 4 || L[r] > 46340 || L[r] % 4 != 0 || q[r] < 2 || q[r] > 127 ||
        (beta && (!(beta[r] >= 0.0) || !std::isfinite(beta[r])))) {
      set_last_error(SW_ERR_ARG, std::string(who) + ": chain " + std::to_string(r) +
                                     ": need 4 <= L <= 46340, L % 4 == 0, 2 <= q <= 127, finite beta >= 0");
      return false;
    }
  }
  return true;
}

// Layout of a batch's device memory: control block | chain table | tile map
// | per chain: spins | tile roots | parents | label scratch | observable ring.
struct BatchLayout {
  int64_t ctl = 0, reps = 0, tile_rep = 0, total = 0;
  std::vector<int64_t> chain;
  std::vector<Grid> grids;
  int n_tiles = 0;
  int64_t max_sites = 0, total_sites = 0;
};

int64_t chain_bytes(const Grid& g, int q) {
  const int64_t N = g.n_sites();
  return al256(N) + al256(2 * N) + al256(4 * N) + al256(label_scratch_bytes(g)) +
         al256((int64_t)BATCH_OBS_CAP * (q + 1) * 8);
}

BatchLayout batch_layout(int n, const int* L, const int* q) {
  BatchLayout lay;
  lay.grids.resize(n);
  for (int r = 0; r < n; ++r) {
    lay.grids[r] = make_grid(L[r], L[r], 1);
    lay.n_tiles += lay.grids[r].n_tiles();
    lay.max_sites = std::max(lay.max_sites, lay.grids[r].n_sites());
    lay.total_sites += lay.grids[r].n_sites();
  }
  int64_t off = 0;
  lay.ctl = off;
  off += al256(sizeof(BatchCtl));
  lay.reps = off;
  off += al256(sizeof(SwRep) * (int64_t)n);
  lay.tile_rep = off;
  off += al256(sizeof(int) * (int64_t)lay.n_tiles);
  lay.chain.resize(n);
  for (int r = 0; r < n; ++r) {
    lay.chain[r] = off;
    off += chain_bytes(lay.grids[r], q[r]);
  }
  lay.total = off;
  return lay;
}

sw_batch* create_batch(int n, const int* L, const int* q, const double* beta, const uint64_t* seed, int convention,
                       int hot_start, void* stream, void* workspace, int64_t ws_bytes, const char* who) {
  if (!valid_chains(n, L, q, beta, who)) return nullptr;
  if (!beta || !seed || convention < 0 || convention > 2) {
    set_last_error(SW_ERR_ARG, std::string(who) + ": need non-null beta and seed arrays and a valid convention");
    return nullptr;
  }
  const BatchLayout lay = batch_layout(n, L, q);
  if (workspace && (ws_bytes < lay.total || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)) {
    set_last_error(SW_ERR_ARG, std::string(who) + ": the workspace must be 256-byte aligned and hold " +
                                   std::to_string(lay.total) + " bytes (sw_batch_device_bytes)");
    return nullptr;
  }
  sw_batch* b = new sw_batch();
  b->n = n;
  b->L.assign(L, L + n);
  b->q.assign(q, q + n);
  b->seed.assign(seed, seed + n);
  b->obs_read.assign(n, 0);
  for (int r = 0; r < n; ++r) b->T.push_back(sw_threshold_for(q[r], beta[r], 1.0, convention));
  auto bad = [&](cudaError_t e, const char* what) -> sw_batch* {
    set_last_error(e == cudaErrorMemoryAllocation ? SW_ERR_OOM : SW_ERR_CUDA,
                   std::string(who) + ": " + what + ": " + cudaGetErrorString(e));
    free_batch(b);
    return nullptr;
  };
  cudaError_t e;
  if (stream) {
    b->stream = static_cast<cudaStream_t>(stream);
  } else {
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking))) return bad(e, "stream");
    b->own_stream = true;
  }
  if (workspace) {
    b->arena = workspace;
  } else {
    if ((e = cudaMalloc(&b->arena, lay.total))) return bad(e, "device memory for the chains");
    b->own_arena = true;
  }
  char* base = static_cast<char*>(b->arena);
  b->ctl = reinterpret_cast<BatchCtl*>(base + lay.ctl);
  b->d_reps = reinterpret_cast<SwRep*>(base + lay.reps);
  b->d_tile_rep = reinterpret_cast<int*>(base + lay.tile_rep);
  b->total_sites = lay.total_sites;
  int* err = reinterpret_cast<int*>(reinterpret_cast<char*>(b->ctl) + offsetof(BatchCtl, err));
  std::vector<int> tile_rep(lay.n_tiles);
  int t0 = 0;
  for (int r = 0; r < n; ++r) {
    const int64_t N = (int64_t)L[r] * L[r];
    char* p = base + lay.chain[r];
    SwRep R;
    R.spins = reinterpret_cast<int8_t*>(p);
    p += al256(N);
    R.lroot = reinterpret_cast<uint16_t*>(p);
    p += al256(2 * N);
    R.gpar = reinterpret_cast<int32_t*>(p);
    p += al256(4 * N);
    R.s = carve_label_scratch(lay.grids[r], p, err);
    p += al256(label_scratch_bytes(lay.grids[r]));
    R.obs = reinterpret_cast<int64_t*>(p);
    R.g = lay.grids[r];
    R.T = b->T[r];
    R.seed = seed[r];
    R.q = q[r];
    R.tile0 = t0;
    for (int k = 0; k < lay.grids[r].n_tiles(); ++k) tile_rep[t0 + k] = r;
    t0 += lay.grids[r].n_tiles();
    b->reps.push_back(R);
    if ((e = launch_init_spins(R.spins, L[r], q[r], seed[r], hot_start, b->stream))) return bad(e, "init spins");
    if ((e = cudaMemsetAsync(R.obs, 0, (int64_t)BATCH_OBS_CAP * (q[r] + 1) * 8, b->stream))) return bad(e, "memset");
  }
  if ((e = cudaMemcpyAsync(b->d_reps, b->reps.data(), sizeof(SwRep) * n, cudaMemcpyHostToDevice, b->stream)))
    return bad(e, "chain table");
  if ((e = cudaMemcpyAsync(b->d_tile_rep, tile_rep.data(), sizeof(int) * lay.n_tiles, cudaMemcpyHostToDevice,
                           b->stream)))
    return bad(e, "tile map");
  static const BatchCtl init_ctl = {0ull, -1ll, 0, 0u, 0u, 0};
  if ((e = cudaMemcpyAsync(b->ctl, &init_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, b->stream)))
    return bad(e, "control block");
  b->view.reps = b->d_reps;
  b->view.tile_rep = b->d_tile_rep;
  b->view.n_reps = n;
  b->view.n_tiles = lay.n_tiles;
  b->view.obs_cap = BATCH_OBS_CAP;
  b->view.limit = (int)std::min<int64_t>(lay.max_sites + 64, (int64_t)1 << 30);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->blocks = std::max(1, batch_persistent_blocks_per_sm()) * std::max(1, sms);
  // the host tables above are copied from pageable memory: the copies are
  // staged before cudaMemcpyAsync returns, so no wait is needed here
  return b;
}

}  // namespace

extern "C" {

sw_batch* sw_batch_create(int n, const int* L, const int* q, const double* beta, const uint64_t* seed,
                          int convention, int hot_start, void* stream) {
  sw_batch* b = create_batch(n, L, q, beta, seed, convention, hot_start, stream, nullptr, 0, "sw_batch_create");
  if (b) {
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
      set_last_error(SW_ERR_CUDA, std::string("sw_batch_create: sync: ") + cudaGetErrorString(e));
      free_batch(b);
      return nullptr;
    }
  }
  return b;
}

int64_t sw_batch_device_bytes(int n, const int* L, const int* q) {
  if (!valid_chains(n, L, q, nullptr, "sw_batch_device_bytes")) return -1;
  return batch_layout(n, L, q).total;
}

sw_batch* sw_batch_create_ws(int n, const int* L, const int* q, const double* beta, const uint64_t* seed,
                             int convention, int hot_start, void* workspace, int64_t ws_bytes, void* stream) {
  if (!workspace) {
    set_last_error(SW_ERR_ARG, "sw_batch_create_ws: null workspace");
    return nullptr;
  }
  return create_batch(n, L, q, beta, seed, convention, hot_start, stream, workspace, ws_bytes, "sw_batch_create_ws");
}

int sw_batch_set_graph(sw_batch* b, int enable) {
  if (!b) return set_last_error(SW_ERR_ARG, "sw_batch_set_graph: null batch");
  b->use_graph = enable != 0;
  return SW_OK;
}

int sw_batch_destroy(sw_batch* b) {
  free_batch(b);
  return SW_OK;
}

int sw_batch_set_schedule(sw_batch* b, int schedule, int blocks_per_sm) {
  if (!b || (schedule != SW_BATCH_PHASES && schedule != SW_BATCH_PERSISTENT) || blocks_per_sm < 0)
    return set_last_error(SW_ERR_ARG, "sw_batch_set_schedule: bad arguments");
  if (schedule == SW_BATCH_PERSISTENT) {
    const int max_per_sm = batch_persistent_blocks_per_sm();
    if (max_per_sm < 1) return set_last_error(SW_ERR_CUDA, "sw_batch_set_schedule: occupancy query failed");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = blocks_per_sm == 0 ? max_per_sm : std::min(blocks_per_sm, max_per_sm);
    const int blocks = per_sm * sms;
    if (blocks != b->blocks) drop_graph(b, SW_BATCH_PERSISTENT);
    b->blocks = blocks;
  }
  b->schedule = schedule;
  return SW_OK;
}

int sw_batch_set_barrier_limit(sw_batch* b, long long cycles) {
  if (!b || cycles < 0) return set_last_error(SW_ERR_ARG, "sw_batch_set_barrier_limit: need a batch and cycles >= 0");
  if (cycles != b->barrier_limit) drop_graph(b, SW_BATCH_PERSISTENT);
  b->barrier_limit = cycles;
  return SW_OK;
}

int sw_batch_sweep(sw_batch* b, int n) {
  if (!b || n < 0) return set_last_error(SW_ERR_ARG, "sw_batch_sweep: bad arguments");
  if (b->failed)
    return set_last_error(SW_ERR_STATE, "sw_batch_sweep: an earlier sweep failed on the device (code " +
                                            std::to_string(b->failed) + "); the chains are invalid, destroy the batch");
  if (n == 0) return SW_OK;
  const int k = b->schedule;
  cudaError_t e;
  if (b->use_graph && !b->exec[k] && !b->graph_failed[k]) {
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = enqueue_batch_sweep(b);
      cudaGraph_t gr = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &gr);
      if (e1 == cudaSuccess && e2 == cudaSuccess && gr &&
          cudaGraphInstantiate(&b->exec[k], gr, 0) == cudaSuccess) {
        b->graph[k] = gr;
      } else {
        if (gr) cudaGraphDestroy(gr);
        b->exec[k] = nullptr;
        b->graph_failed[k] = true;   // launch directly instead
        cudaGetLastError();
      }
    } else {
      b->graph_failed[k] = true;
      cudaGetLastError();
    }
  }
  for (int s = 0; s < n; ++s) {
    e = (b->use_graph && b->exec[k]) ? cudaGraphLaunch(b->exec[k], b->stream) : enqueue_batch_sweep(b);
    if (e != cudaSuccess) return set_last_error(SW_ERR_CUDA, std::string("sw_batch_sweep: ") + cudaGetErrorString(e));
    b->sweeps++;
  }
  b->final_obs_pending = true;
  return SW_OK;
}

int sw_batch_sync(sw_batch* b) {
  if (!b) return set_last_error(SW_ERR_ARG, "sw_batch_sync: null batch");
  return batch_status(b);
}

int sw_batch_observables(sw_batch* b, int replica, int64_t* out, int max_sweeps, int* n_written) {
  if (!b || replica < 0 || replica >= b->n || max_sweeps < 0 || (!out && max_sweeps > 0))
    return set_last_error(SW_ERR_ARG, "sw_batch_observables: bad arguments");
  if (n_written) *n_written = 0;
  cudaError_t e = finish_batch_observables(b);
  if (e != cudaSuccess) return set_last_error(SW_ERR_CUDA, std::string("sw_batch_observables: ") + cudaGetErrorString(e));
  int rc = batch_status(b);
  if (rc) return rc;
  uint64_t& rd = b->obs_read[replica];
  if (b->sweeps - rd > (uint64_t)BATCH_OBS_CAP) rd = b->sweeps - BATCH_OBS_CAP;
  const int64_t cnt = std::min<int64_t>((int64_t)(b->sweeps - rd), max_sweeps);
  const int row = b->q[replica] + 1;
  const int64_t* ring = b->reps[replica].obs;
  int64_t done = 0;
  while (done < cnt) {
    const int64_t slot = (int64_t)((rd + done) % BATCH_OBS_CAP);
    const int64_t run = std::min<int64_t>(cnt - done, BATCH_OBS_CAP - slot);
    e = cudaMemcpyAsync(out + done * row, ring + slot * row, run * row * 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return set_last_error(SW_ERR_CUDA, std::string("sw_batch_observables: ") + cudaGetErrorString(e));
    done += run;
  }
  rd += cnt;
  if (n_written) *n_written = (int)cnt;
  return SW_OK;
}

int sw_batch_observables_async(sw_batch* b, int replica, int64_t* dst, int max_sweeps, int* n_written) {
  if (!b || replica < 0 || replica >= b->n || max_sweeps < 0 || (!dst && max_sweeps > 0))
    return set_last_error(SW_ERR_ARG, "sw_batch_observables_async: bad arguments");
  if (n_written) *n_written = 0;
  cudaError_t e = finish_batch_observables(b);
  if (e != cudaSuccess)
    return set_last_error(SW_ERR_CUDA, std::string("sw_batch_observables_async: ") + cudaGetErrorString(e));
  uint64_t& rd = b->obs_read[replica];
  if (b->sweeps - rd > (uint64_t)BATCH_OBS_CAP) rd = b->sweeps - BATCH_OBS_CAP;
  const int64_t cnt = std::min<int64_t>((int64_t)(b->sweeps - rd), max_sweeps);
  const int row = b->q[replica] + 1;
  const int64_t* ring = b->reps[replica].obs;
  int64_t done = 0;
  while (done < cnt) {
    const int64_t slot = (int64_t)((rd + done) % BATCH_OBS_CAP);
    const int64_t run = std::min<int64_t>(cnt - done, BATCH_OBS_CAP - slot);
    e = cudaMemcpyAsync(dst + done * row, ring + slot * row, run * row * 8, cudaMemcpyDefault, b->stream);
    if (e != cudaSuccess)
      return set_last_error(SW_ERR_CUDA, std::string("sw_batch_observables_async: ") + cudaGetErrorString(e));
    done += run;
  }
  rd += cnt;
  if (n_written) *n_written = (int)cnt;
  return SW_OK;
}

int sw_batch_get_spins(sw_batch* b, int replica, int8_t* dst, int is_device) {
  if (!b || replica < 0 || replica >= b->n || !dst) return set_last_error(SW_ERR_ARG, "sw_batch_get_spins: bad arguments");
  int rc = batch_status(b);
  if (rc) return rc;
  const int64_t n = (int64_t)b->L[replica] * b->L[replica];
  cudaError_t e = is_device ? launch_copy_if(dst, b->reps[replica].spins, n, nullptr, b->stream)
                            : cudaMemcpyAsync(dst, b->reps[replica].spins, n, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return set_last_error(SW_ERR_CUDA, std::string("sw_batch_get_spins: ") + cudaGetErrorString(e));
  return SW_OK;
}

int sw_batch_info(sw_batch* b, int64_t* info) {
  if (!b || !info) return set_last_error(SW_ERR_ARG, "sw_batch_info: bad arguments");
  info[0] = b->n;
  info[1] = b->total_sites;
  info[2] = b->view.n_tiles;
  info[3] = (int64_t)b->sweeps;
  info[4] = b->schedule;
  info[5] = b->blocks;
  info[6] = (b->exec[b->schedule] != nullptr) ? 1 : 0;
  info[7] = BATCH_OBS_CAP;
  return SW_OK;
}

void* sw_batch_stream(sw_batch* b) { return b ? (void*)b->stream : nullptr; }

}  // extern "C"
