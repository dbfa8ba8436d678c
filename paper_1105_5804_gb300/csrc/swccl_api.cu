// swccl_api.cu -- host driver and C ABI of libswccl (declared in include/swccl.h).
//
// A Swendsen-Wang sweep (Sec. II, three steps) is five kernels on the
// handle's stream: activation, tile labeling, seam merge, root compression
// with root draws, flip with observables; a one-thread kernel then advances
// the sweep counter held in device memory, so one captured CUDA graph serves
// every sweep.  Nothing crosses to the host inside a sweep (the paper's
// relaxation checked its stopping rule on the CPU between launches,
// Sec. II.C.1; the atomic merge needs no such loop).
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "swccl_shared.h"

namespace swccl {
// k_bonds.cu: a nonzero *flag is recorded in *err (the first code stays)
cudaError_t launch_note_error(const int* flag, int* err, cudaStream_t st);
}  // namespace swccl

using namespace swccl;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr int OBS_CAP = 4096;
constexpr size_t READBACK_BYTES = 64 << 10;

}  // namespace

// Device status word of the stand-alone labeling calls.
__device__ int g_ccl_status;

namespace {
int* ccl_status_ptr() {
  static int* ptrs[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_ccl_status) != cudaSuccess) return nullptr;
    ptrs[dev] = static_cast<int*>(p);
  }
  return ptrs[dev];
}
}  // namespace

struct sw_handle {
  int L = 0, q = 0;
  uint64_t T = 0, seed = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  Grid grid{};
  int8_t* spins = nullptr;
  uint8_t* mask = nullptr;
  int32_t* labels = nullptr;
  void* scratch = nullptr;
  LabelScratch ls{};
  SwCtl* ctl = nullptr;
  int* chk = nullptr;
  int64_t* obs = nullptr;
  uint16_t* lroot = nullptr;   // fused mode: tile root of every site (local index)
  int mode = SW_MODE_FUSED;
  bool final_obs_pending = false;   // fused mode: observables of the last sweep not yet counted
  uint64_t sweeps = 0;     // sweeps enqueued
  uint64_t obs_read = 0;   // next sweep whose observables are unread
  cudaGraph_t graph = nullptr;        // one staged sweep
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph_fused = nullptr;  // one fused sweep
  cudaGraphExec_t exec_fused = nullptr;
  int update = SW_UPDATE_SW;         // SW_UPDATE_SW or SW_UPDATE_FEW (fused mode only)
  int ell = 0;                       // few-cluster: ell x ell seed blocks
  uint64_t P_flip = 0;               // few-cluster: flip threshold
  uint32_t* sel = nullptr;           // few-cluster: seeded-cluster roots, one bit per site
  void* readback = nullptr;          // mapped pinned host buffer for small reads (READBACK_BYTES)
  bool timing = false;
  bool dump_valid = false;  // mask/labels hold the last sweep's result
  std::vector<cudaEvent_t> ev_pending;   // SW_N_PHASES + 1 events per timed sweep
  std::vector<cudaEvent_t> ev_free;
};

namespace {

void free_handle(sw_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->exec_fused) cudaGraphExecDestroy(h->exec_fused);
  if (h->graph_fused) cudaGraphDestroy(h->graph_fused);
  for (auto e : h->ev_pending) cudaEventDestroy(e);
  for (auto e : h->ev_free) cudaEventDestroy(e);
  cudaFree(h->spins);
  cudaFree(h->sel);
  cudaFree(h->mask);
  cudaFree(h->labels);
  cudaFree(h->scratch);
  cudaFree(h->ctl);
  cudaFree(h->chk);
  if (h->readback) cudaFreeHost(h->readback);
  cudaFree(h->obs);
  cudaFree(h->lroot);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// Enqueue one sweep.
cudaError_t enqueue_sweep(sw_handle* h, cudaEvent_t* ev) {
  cudaError_t e;
  const cudaStream_t st = h->stream;
  if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
  if ((e = launch_activate(h->spins, h->mask, h->L, h->T, h->seed, h->ctl, h->obs, OBS_CAP, h->q, st)))
    return e;
  if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
  if ((e = launch_tile_label(h->mask, h->labels, h->grid, h->ls, st))) return e;
  if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
  if ((e = launch_merge(h->labels, h->grid, h->ls, st))) return e;
  if (ev && (e = cudaEventRecord(ev[3], st)) != cudaSuccess) return e;
  if ((e = launch_root_compress(h->labels, h->grid, h->ls, h->spins, h->q, h->seed, h->ctl, st))) return e;
  if (ev && (e = cudaEventRecord(ev[4], st)) != cudaSuccess) return e;
  if ((e = launch_flip(h->spins, h->labels, h->L, h->q, h->ctl, h->obs, OBS_CAP, st))) return e;
  if (ev && (e = cudaEventRecord(ev[5], st)) != cudaSuccess) return e;
  return launch_advance(h->ctl, st);
}

// Enqueue one fused sweep: draw + label, merge, flip, advance.  With timing
// events the activation and root phases are recorded as empty.
cudaError_t enqueue_sweep_fused(sw_handle* h, cudaEvent_t* ev) {
  cudaError_t e;
  const cudaStream_t st = h->stream;
  if (ev && ((e = cudaEventRecord(ev[0], st)) != cudaSuccess || (e = cudaEventRecord(ev[1], st)) != cudaSuccess))
    return e;
  if ((e = launch_sw_label(h->spins, h->lroot, h->labels, h->grid, h->ls, h->q, h->T, h->seed, h->ctl, h->obs,
                           OBS_CAP, st)))
    return e;
  if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
  if ((e = launch_merge(h->labels, h->grid, h->ls, st))) return e;
  if (ev && (e = cudaEventRecord(ev[3], st)) != cudaSuccess) return e;
  if (h->update == SW_UPDATE_FEW &&
      (e = launch_few_select(h->lroot, h->labels, h->grid, h->ls, h->seed, h->ell, h->sel, h->ctl, st)))
    return e;
  if (ev && (e = cudaEventRecord(ev[4], st)) != cudaSuccess) return e;
  if (h->update == SW_UPDATE_FEW) {
    if ((e = launch_sw_flip_few(h->spins, h->lroot, h->labels, h->grid, h->ls, h->q, h->seed, h->sel, h->P_flip,
                                h->ctl, st)))
      return e;
  } else if ((e = launch_sw_flip(h->spins, h->lroot, h->labels, h->grid, h->ls, h->q, h->seed, h->ctl, st))) {
    return e;
  }
  if (ev && (e = cudaEventRecord(ev[5], st)) != cudaSuccess) return e;
  return launch_advance_fused(h->ctl, h->obs, OBS_CAP, h->q, st);
}

// Fused mode counts a sweep's observables in the next sweep's first kernel;
// before the chain is read or changed, count the last sweep's here.
cudaError_t finish_observables(sw_handle* h) {
  if (!h->final_obs_pending) return cudaSuccess;
  h->final_obs_pending = false;
  return launch_observe(h->spins, h->L, h->q, h->ctl, h->obs, OBS_CAP, h->stream);
}

// Synchronous copy ordered on the handle's stream (never on the legacy
// default stream, which would also wait for every other blocking stream).
cudaError_t copy_on(cudaStream_t st, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, st);
  return e != cudaSuccess ? e : cudaStreamSynchronize(st);
}

// Small device-to-host reads go through the handle's mapped pinned buffer:
// a kernel stores the bytes there, the stream is synchronised, and the host
// reads them.  A copy engine would queue them behind large host transfers
// that other streams have in flight.
cudaError_t read_small(sw_handle* h, void* dst, const void* src, size_t bytes) {
  if (bytes > READBACK_BYTES) return copy_on(h->stream, dst, src, bytes, cudaMemcpyDeviceToHost);
  void* dev_view = nullptr;
  cudaError_t e = cudaHostGetDevicePointer(&dev_view, h->readback, 0);
  if (e == cudaSuccess) e = launch_copy_if(static_cast<int8_t*>(dev_view), static_cast<const int8_t*>(src),
                                           (int64_t)bytes, nullptr, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) std::memcpy(dst, h->readback, bytes);
  return e;
}

int check_device_status(sw_handle* h) {
  SwCtl c;
  CK(read_small(h, &c, h->ctl, sizeof(c)));
  if (c.err == SW_ERR_ARG) {
    // only sw_sweep_io records this code: an input it rejected, leaving the
    // spins unchanged; reported once
    CK(cudaMemsetAsync(reinterpret_cast<char*>(h->ctl) + offsetof(SwCtl, err), 0, sizeof(int), h->stream));
    return fail(SW_ERR_ARG, "sw_sweep_io: an input spin value was outside [0, q); the spins were left unchanged");
  }
  if (c.err) return fail(c.err, "a device-side consistency check failed in a sweep");
  return SW_OK;
}

double coupling_K(int q, double beta, double J, int conv) {
  if (conv == SW_CONV_AUTO) conv = (q == 2) ? SW_CONV_ISING : SW_CONV_POTTS;
  return conv == SW_CONV_ISING ? 2.0 * beta * J : beta * J;
}

uint64_t threshold_of(double K) {
  if (!(K > 0.0)) return 0;
  const double p = -std::expm1(-K);
  const double t = std::floor(p * 4294967296.0);
  if (t >= 4294967296.0) return 1ull << 32;
  if (t < 0.0) return 0;
  return (uint64_t)t;
}

}  // namespace

namespace swccl {
int set_last_error(int code, const std::string& msg) { return fail(code, msg); }
int* ccl_status_word() { return ccl_status_ptr(); }
}  // namespace swccl

extern "C" {

const char* sw_last_error(void) { return g_err.c_str(); }

uint64_t sw_threshold_for(int q, double beta, double J, int convention) {
  return threshold_of(coupling_K(q, beta, J, convention));
}

uint64_t sw_prob_threshold(double p) {
  if (!(p >= 0.0 && p <= 1.0)) return UINT64_MAX;
  const double t = std::floor(p * 4294967296.0);
  return t >= 4294967296.0 ? (uint64_t)1 << 32 : (uint64_t)t;
}

int sw_set_update(sw_handle* h, int update, int ell, uint64_t P) {
  if (!h || (update != SW_UPDATE_SW && update != SW_UPDATE_FEW)) return fail(SW_ERR_ARG, "sw_set_update: bad arguments");
  if (update == SW_UPDATE_FEW) {
    if (ell < 1 || h->L % ell != 0 || P > ((uint64_t)1 << 32))
      return fail(SW_ERR_ARG, "sw_set_update: need ell >= 1 dividing L and P <= 2^32");
    if (h->mode != SW_MODE_FUSED)
      return fail(SW_ERR_STATE, "sw_set_update: the few-cluster update runs in SW_MODE_FUSED only");
  } else {
    ell = 0;
    P = 0;
  }
  if (update == h->update && ell == h->ell && P == h->P_flip) return SW_OK;
  CK(cudaStreamSynchronize(h->stream));
  if (update == SW_UPDATE_FEW && !h->sel) {
    if (cudaMalloc(&h->sel, (size_t)few_sel_bytes(h->grid.n_sites())) != cudaSuccess) {
      cudaGetLastError();
      h->sel = nullptr;
      return fail(SW_ERR_OOM, "sw_set_update: cudaMalloc of the selection bits failed");
    }
  }
  // ell and P are launch arguments of the captured sweep: capture it again
  if (h->exec_fused) cudaGraphExecDestroy(h->exec_fused);
  if (h->graph_fused) cudaGraphDestroy(h->graph_fused);
  h->exec_fused = nullptr;
  h->graph_fused = nullptr;
  h->update = update;
  h->ell = ell;
  h->P_flip = P;
  return SW_OK;
}

sw_handle* sw_create_threshold(int L, int q, uint64_t T, uint64_t seed, int hot_start, void* stream) {
  if (L < 4 || L > 46340 || L % 4 != 0) {
    fail(SW_ERR_ARG, "sw_create: L must satisfy 4 <= L <= 46340 and L % 4 == 0");
    return nullptr;
  }
  if (q < 2 || q > 127) {
    fail(SW_ERR_ARG, "sw_create: q must be in [2, 127]");
    return nullptr;
  }
  if (T > (1ull << 32)) {
    fail(SW_ERR_ARG, "sw_create: threshold T must be <= 2^32");
    return nullptr;
  }
  sw_handle* h = new sw_handle();
  h->L = L;
  h->q = q;
  h->T = T;
  h->seed = seed;
  h->grid = make_grid(L, L, 1);
  const int64_t N = (int64_t)L * L;
  auto bad = [&](cudaError_t e, const char* what) -> sw_handle* {
    cuda_fail(e, what);
    if (e == cudaErrorMemoryAllocation) g_err = std::string("out of device memory: ") + what;
    free_handle(h);
    return nullptr;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&h->device))) return bad(e, "cudaGetDevice");
  if (stream) {
    h->stream = static_cast<cudaStream_t>(stream);
  } else {
    if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking))) return bad(e, "cudaStreamCreate");
    h->own_stream = true;
  }
  const int64_t sbytes = label_scratch_bytes(h->grid);
  if ((e = cudaMalloc(&h->spins, (N + 15) & ~15LL))) return bad(e, "spins");
  if ((e = cudaMalloc(&h->mask, ((N + 3) / 4 + 15) & ~15LL))) return bad(e, "mask");
  if ((e = cudaMalloc(&h->labels, N * 4))) return bad(e, "labels");
  if ((e = cudaMalloc(&h->scratch, sbytes))) return bad(e, "label scratch");
  if ((e = cudaMalloc(&h->ctl, sizeof(SwCtl)))) return bad(e, "control block");
  if ((e = cudaMalloc(&h->chk, sizeof(int)))) return bad(e, "check word");
  if ((e = cudaHostAlloc(&h->readback, READBACK_BYTES, cudaHostAllocMapped))) return bad(e, "read-back buffer");
  if ((e = cudaMalloc(&h->obs, (int64_t)OBS_CAP * (q + 1) * 8))) return bad(e, "observable ring");
  if ((e = cudaMalloc(&h->lroot, (N * 2 + 15) & ~15LL))) return bad(e, "tile roots");
  h->ls = carve_label_scratch(h->grid, h->scratch,
                              reinterpret_cast<int*>(reinterpret_cast<char*>(h->ctl) + offsetof(SwCtl, err)));
  {
    static const SwCtl init_ctl = {0ull, -1ll, 0, 0};
    if ((e = cudaMemcpyAsync(h->ctl, &init_ctl, sizeof(SwCtl), cudaMemcpyHostToDevice, h->stream)))
      return bad(e, "control block");
  }
  if ((e = cudaMemsetAsync(h->obs, 0, (int64_t)OBS_CAP * (q + 1) * 8, h->stream))) return bad(e, "memset");
  if ((e = launch_init_spins(h->spins, L, q, seed, hot_start, h->stream))) return bad(e, "init spins");
  if ((e = cudaStreamSynchronize(h->stream))) return bad(e, "sync");
  g_err.clear();
  return h;
}

sw_handle* sw_create_ex(int L, int q, double beta, double J, int convention, uint64_t seed,
                        int hot_start, void* stream) {
  if (!(beta >= 0.0) || !std::isfinite(beta) || !std::isfinite(J) || convention < 0 || convention > 2) {
    fail(SW_ERR_ARG, "sw_create_ex: beta must be finite and >= 0, J finite, convention in {0,1,2}");
    return nullptr;
  }
  return sw_create_threshold(L, q, threshold_of(coupling_K(q, beta, J, convention)), seed, hot_start, stream);
}

sw_handle* sw_create(int L, int q, double beta, uint64_t seed) {
  return sw_create_ex(L, q, beta, 1.0, SW_CONV_AUTO, seed, 0, nullptr);
}

int sw_destroy(sw_handle* h) {
  free_handle(h);
  return SW_OK;
}

int sw_sweep(sw_handle* h, int n) {
  if (!h) return fail(SW_ERR_ARG, "sw_sweep: null handle");
  if (n < 0) return fail(SW_ERR_ARG, "sw_sweep: n must be >= 0");
  if (n == 0) return SW_OK;
  const bool fused = h->mode == SW_MODE_FUSED;
  auto enqueue = fused ? enqueue_sweep_fused : enqueue_sweep;
  if (h->timing) {
    for (int k = 0; k < n; ++k) {
      cudaEvent_t ev[SW_N_PHASES + 1];
      for (auto& e : ev) {
        if (!h->ev_free.empty()) {
          e = h->ev_free.back();
          h->ev_free.pop_back();
        } else {
          CK(cudaEventCreate(&e));
        }
        h->ev_pending.push_back(e);
      }
      CK(enqueue(h, ev));
      h->sweeps++;
    }
  } else {
    cudaGraph_t& graph = fused ? h->graph_fused : h->graph;
    cudaGraphExec_t& exec = fused ? h->exec_fused : h->exec;
    if (!exec) {
      CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = enqueue(h, nullptr);
      cudaGraph_t gr = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(h->stream, &gr);
      if (e != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return cuda_fail(e, "capture of one sweep"); }
      if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
      graph = gr;
      CK(cudaGraphInstantiate(&exec, graph, 0));
    }
    for (int k = 0; k < n; ++k) {
      CK(cudaGraphLaunch(exec, h->stream));
      h->sweeps++;
    }
  }
  h->dump_valid = !fused;
  h->final_obs_pending = fused;
  return SW_OK;
}

int sw_set_mode(sw_handle* h, int mode) {
  if (!h || (mode != SW_MODE_STAGED && mode != SW_MODE_FUSED)) return fail(SW_ERR_ARG, "sw_set_mode: bad arguments");
  if (mode == h->mode) return SW_OK;
  if (mode == SW_MODE_STAGED && h->update == SW_UPDATE_FEW)
    return fail(SW_ERR_STATE, "sw_set_mode: the few-cluster update runs in SW_MODE_FUSED only");
  if (mode == SW_MODE_STAGED) {
    CK(finish_observables(h));
  } else {
    // the staged flip already counted the last sweep's observables
    const long long done = (long long)h->sweeps - 1;
    CK(cudaMemcpyAsync(reinterpret_cast<char*>(h->ctl) + offsetof(SwCtl, obs_done), &done, sizeof(done),
                       cudaMemcpyHostToDevice, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  h->mode = mode;
  return SW_OK;
}

int sw_sync(sw_handle* h) {
  if (!h) return fail(SW_ERR_ARG, "sw_sync: null handle");
  return check_device_status(h);
}

int sw_observables(sw_handle* h, int64_t* out, int max_sweeps, int* n_written) {
  if (!h || (!out && max_sweeps > 0) || max_sweeps < 0) return fail(SW_ERR_ARG, "sw_observables: bad arguments");
  if (n_written) *n_written = 0;
  CK(finish_observables(h));
  int rc = check_device_status(h);
  if (rc) return rc;
  if (h->sweeps - h->obs_read > (uint64_t)OBS_CAP) h->obs_read = h->sweeps - OBS_CAP;
  const int64_t avail = (int64_t)(h->sweeps - h->obs_read);
  const int64_t cnt = std::min<int64_t>(avail, max_sweeps);
  const int row = h->q + 1;
  int64_t done = 0;
  while (done < cnt) {
    const int64_t slot = (int64_t)((h->obs_read + done) % OBS_CAP);
    const int64_t run = std::min<int64_t>(cnt - done, OBS_CAP - slot);
    CK(read_small(h, out + done * row, h->obs + slot * row, run * row * 8));
    done += run;
  }
  h->obs_read += cnt;
  if (n_written) *n_written = (int)cnt;
  return SW_OK;
}

int sw_get_spins(sw_handle* h, int8_t* dst, int is_device) {
  if (!h || !dst) return fail(SW_ERR_ARG, "sw_get_spins: bad arguments");
  int rc = check_device_status(h);
  if (rc) return rc;
  if (is_device) {
    CK(launch_copy_if(dst, h->spins, (int64_t)h->L * h->L, nullptr, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  } else {
    CK(copy_on(h->stream, dst, h->spins, (size_t)h->L * h->L, cudaMemcpyDeviceToHost));
  }
  return SW_OK;
}

int sw_set_spins(sw_handle* h, const int8_t* src, int is_device) {
  if (!h || !src) return fail(SW_ERR_ARG, "sw_set_spins: bad arguments");
  const int64_t N = (int64_t)h->L * h->L;
  // Host input is staged in the label buffer (4N bytes, rewritten by the
  // next sweep) and validated there by a kernel; device input is validated
  // in place.  The spins change only if every value is in [0, q).
  CK(finish_observables(h));
  const int8_t* dsrc = src;
  if (!is_device) {
    int8_t* staging = reinterpret_cast<int8_t*>(h->labels);
    CK(cudaMemcpyAsync(staging, src, N, cudaMemcpyHostToDevice, h->stream));
    dsrc = staging;
    h->dump_valid = false;
  }
  CK(cudaMemsetAsync(h->chk, 0, sizeof(int), h->stream));
  CK(launch_check_spins(dsrc, N, h->q, h->chk, h->stream));
  CK(launch_copy_if(h->spins, dsrc, N, h->chk, h->stream));   // only if every value is valid
  int bad = 0;
  CK(read_small(h, &bad, h->chk, sizeof(int)));
  if (bad) return fail(SW_ERR_ARG, "sw_set_spins: spin value outside [0, q)");
  return SW_OK;
}

int sw_sweep_io(sw_handle* h, const int8_t* in, int n, int64_t* obs_out, int8_t* out) {
  if (!h || n < 0 || n > OBS_CAP) return fail(SW_ERR_ARG, "sw_sweep_io: bad arguments");
  const int64_t N = (int64_t)h->L * h->L;
  const cudaStream_t st = h->stream;
  if (in) {
    // the observables still pending belong to the spins being replaced; the
    // input goes in only if every value is valid, else the code is noted in
    // the status word (read by the next synchronising call)
    CK(finish_observables(h));
    CK(cudaMemsetAsync(h->chk, 0, sizeof(int), st));
    CK(launch_check_spins(in, N, h->q, h->chk, st));
    CK(launch_copy_if(h->spins, in, N, h->chk, st));
    CK(launch_note_error(h->chk, h->ls.err, st));
    h->dump_valid = false;
  }
  if (n > 0) {
    const int rc = sw_sweep(h, n);
    if (rc) return rc;
  }
  if (obs_out && n > 0) {
    CK(finish_observables(h));
    const int row = h->q + 1;
    int64_t done = 0;
    const uint64_t first = h->sweeps - (uint64_t)n;
    while (done < n) {
      const int64_t slot = (int64_t)((first + done) % OBS_CAP);
      const int64_t run = std::min<int64_t>(n - done, OBS_CAP - slot);
      CK(cudaMemcpyAsync(obs_out + done * row, h->obs + slot * row, run * row * 8, cudaMemcpyDefault, st));
      done += run;
    }
    h->obs_read = h->sweeps;
  }
  if (out) CK(launch_copy_if(out, h->spins, N, nullptr, st));
  return SW_OK;
}

int sw_debug_dump(sw_handle* h, uint8_t* mask_out, int32_t* labels_out, int is_device) {
  if (!h) return fail(SW_ERR_ARG, "sw_debug_dump: null handle");
  if (!h->dump_valid)
    return fail(SW_ERR_STATE,
                "sw_debug_dump: the last sweep did not run in SW_MODE_STAGED, or no sweep has run since "
                "creation or the last sw_set_spins");
  const int64_t N = (int64_t)h->L * h->L;
  const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (labels_out) {
    // after a sweep every label points at its tile root and the tile root at
    // the final root; one pointer jump makes every label canonical
    CK(launch_site_compress(h->labels, N, h->stream));
  }
  int rc = check_device_status(h);
  if (rc) return rc;
  if (mask_out) CK(copy_on(h->stream, mask_out, h->mask, (N + 3) / 4, kind));
  if (labels_out) CK(copy_on(h->stream, labels_out, h->labels, N * 4, kind));
  return SW_OK;
}

int sw_get_info(sw_handle* h, int64_t* info) {
  if (!h || !info) return fail(SW_ERR_ARG, "sw_get_info: bad arguments");
  info[0] = h->L;
  info[1] = h->q;
  info[2] = (int64_t)h->T;
  info[3] = (int64_t)h->seed;
  info[4] = (int64_t)h->sweeps;
  info[5] = OBS_CAP;
  info[6] = TILE_H;
  info[7] = TILE_W;
  return SW_OK;
}

void* sw_stream(sw_handle* h) { return h ? (void*)h->stream : nullptr; }

int sw_set_timing(sw_handle* h, int enable) {
  if (!h) return fail(SW_ERR_ARG, "sw_set_timing: null handle");
  h->timing = enable != 0;
  return SW_OK;
}

int sw_phase_times(sw_handle* h, double* ms, int64_t* n_sweeps) {
  if (!h || !ms) return fail(SW_ERR_ARG, "sw_phase_times: bad arguments");
  CK(cudaStreamSynchronize(h->stream));
  for (int p = 0; p < SW_N_PHASES; ++p) ms[p] = 0.0;
  const size_t per = SW_N_PHASES + 1;
  const int64_t n = (int64_t)(h->ev_pending.size() / per);
  for (int64_t k = 0; k < n; ++k) {
    for (int p = 0; p < SW_N_PHASES; ++p) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, h->ev_pending[k * per + p], h->ev_pending[k * per + p + 1]));
      ms[p] += t;
    }
  }
  for (auto e : h->ev_pending) h->ev_free.push_back(e);
  h->ev_pending.clear();
  if (n_sweeps) *n_sweeps = n;
  return SW_OK;
}

// ---------------------------------------------------------------------------
// Stand-alone labeling
// ---------------------------------------------------------------------------
namespace {
int ccl_validate(const void* mask, const void* labels, int H, int W) {
  if (!mask || !labels) return fail(SW_ERR_ARG, "ccl: null device pointer");
  if (H < 1 || W < 1 || (int64_t)H * W >= ((int64_t)1 << 31))
    return fail(SW_ERR_ARG, "ccl: need H, W >= 1 and H*W < 2^31");
  return SW_OK;
}

}  // namespace

int64_t ccl_workspace_bytes(int H, int W) {
  if (H < 1 || W < 1 || (int64_t)H * W >= ((int64_t)1 << 31)) return -1;
  return label_scratch_bytes(make_grid(H, W, 0));
}

int ccl_label_ws(const uint8_t* bond_mask, int32_t* labels, int H, int W, int periodic,
                 void* workspace, int64_t ws_bytes, void* stream) {
  int rc = ccl_validate(bond_mask, labels, H, W);
  if (rc) return rc;
  const Grid g = make_grid(H, W, periodic);
  if (!workspace || ws_bytes < label_scratch_bytes(g) || ((uintptr_t)workspace & 255))
    return fail(SW_ERR_ARG, "ccl_label_ws: workspace missing, too small or not 256-byte aligned");
  int* status = ccl_status_ptr();
  if (!status) return fail(SW_ERR_CUDA, "ccl: cannot resolve the device status word");
  const LabelScratch s = carve_label_scratch(g, workspace, status);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(launch_ccl(bond_mask, labels, g, s, st));
  return SW_OK;
}

int ccl_label(const uint8_t* bond_mask, int32_t* labels, int H, int W, int periodic, void* stream) {
  int rc = ccl_validate(bond_mask, labels, H, W);
  if (rc) return rc;
  const int64_t bytes = ccl_workspace_bytes(H, W);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* ws = nullptr;
  cudaError_t e = cudaMallocAsync(&ws, bytes, st);
  if (e == cudaErrorMemoryAllocation) return fail(SW_ERR_OOM, "ccl_label: out of device memory for scratch");
  if (e) return cuda_fail(e, "cudaMallocAsync");
  rc = ccl_label_ws(bond_mask, labels, H, W, periodic, ws, bytes, stream);
  cudaError_t e2 = cudaFreeAsync(ws, st);
  if (rc) return rc;
  if (e2) return cuda_fail(e2, "cudaFreeAsync");
  return SW_OK;
}

int ccl_bonds_from_pixels(const uint8_t* px, uint8_t* mask, int H, int W, int periodic, void* stream) {
  int rc = ccl_validate(px, mask, H, W);
  if (rc) return rc;
  CK(launch_pixel_bonds(px, mask, H, W, periodic, static_cast<cudaStream_t>(stream)));
  return SW_OK;
}

int ccl_copy_pixels_2d(const uint8_t* src, int64_t src_pitch, uint8_t* dst, int H, int W, int src_is_device,
                       void* stream) {
  if (!src || !dst || H < 1 || W < 1 || src_pitch < W) return fail(SW_ERR_ARG, "ccl_copy_pixels_2d: bad arguments");
  CK(cudaMemcpy2DAsync(dst, (size_t)W, src, (size_t)src_pitch, (size_t)W, (size_t)H,
                       src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       static_cast<cudaStream_t>(stream)));
  return SW_OK;
}

int ccl_perc_mask(uint64_t k, uint8_t* mask, int H, int W, void* stream) {
  int rc = ccl_validate(mask, mask, H, W);
  if (rc) return rc;
  CK(launch_perc_mask(mask, H, W, k, static_cast<cudaStream_t>(stream)));
  return SW_OK;
}

// ---------------------------------------------------------------------------
// Batched labeling
// ---------------------------------------------------------------------------
namespace {
inline int64_t al256b(int64_t b) { return (b + 255) & ~(int64_t)255; }

int64_t ccl_batch_bytes(int n, const int* H, const int* W, int64_t* n_tiles_out) {
  int64_t tiles = 0, scratch = 0;
  for (int j = 0; j < n; ++j) {
    if (H[j] < 1 || W[j] < 1 || (int64_t)H[j] * W[j] >= ((int64_t)1 << 31)) return -1;
    const Grid g = make_grid(H[j], W[j], 0);
    tiles += g.n_tiles();
    scratch += al256b(label_scratch_bytes(g));
  }
  if (n_tiles_out) *n_tiles_out = tiles;
  return al256b((int64_t)sizeof(CclJob) * n) + al256b(4 * tiles) + scratch;
}
}  // namespace

int64_t ccl_batch_workspace_bytes(int n, const int* H, const int* W) {
  if (n < 0 || (n > 0 && (!H || !W))) return -1;
  return ccl_batch_bytes(n, H, W, nullptr);
}

int ccl_label_batch(int n, const uint8_t* const* masks, int32_t* const* labels, const int* H, const int* W,
                    const int* periodic, void* workspace, int64_t ws_bytes, void* stream) {
  if (n < 0 || (n > 0 && (!masks || !labels || !H || !W || !periodic)))
    return fail(SW_ERR_ARG, "ccl_label_batch: bad arguments");
  if (n == 0) return SW_OK;
  int64_t n_tiles = 0;
  const int64_t need = ccl_batch_bytes(n, H, W, &n_tiles);
  if (need < 0) return fail(SW_ERR_ARG, "ccl_label_batch: need H, W >= 1 and H*W < 2^31 for every grid");
  if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255))
    return fail(SW_ERR_ARG, "ccl_label_batch: workspace missing, smaller than ccl_batch_workspace_bytes or not "
                            "256-byte aligned");
  if (n_tiles >= ((int64_t)1 << 31)) return fail(SW_ERR_ARG, "ccl_label_batch: too many tiles");
  for (int j = 0; j < n; ++j)
    if (!masks[j] || !labels[j]) return fail(SW_ERR_ARG, "ccl_label_batch: null mask or label pointer");
  int* status = ccl_status_ptr();
  if (!status) return fail(SW_ERR_CUDA, "ccl_label_batch: cannot resolve the device status word");
  // The grids go to the kernels by value, CCL_PARAM_JOBS at a time (one set
  // of launches each): no copy from host memory, so the call never waits
  // for the stream.  The workspace keeps room for a device-side table too.
  char* p = static_cast<char*>(workspace) + al256b((int64_t)sizeof(CclJob) * n) + al256b(4 * n_tiles);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int j0 = 0; j0 < n; j0 += CCL_PARAM_JOBS) {
    CclBatchView v;
    v.n_jobs = std::min(CCL_PARAM_JOBS, n - j0);
    int t0 = 0;
    int64_t max_sites = 0;
    for (int u = 0; u < v.n_jobs; ++u) {
      const int j = j0 + u;
      const Grid g = make_grid(H[j], W[j], periodic[j]);
      CclJob& J = v.jobs[u];
      J.mask = masks[j];
      J.labels = labels[j];
      J.s = carve_label_scratch(g, p, status);
      J.g = g;
      J.tile0 = t0;
      J.pad = 0;
      p += al256b(label_scratch_bytes(g));
      t0 += g.n_tiles();
      v.tile_end[u] = t0;
      max_sites = std::max<int64_t>(max_sites, g.n_sites());
    }
    v.n_tiles = t0;
    v.limit = (int)std::min<int64_t>(max_sites + 64, (int64_t)1 << 30);
    v.pad = 0;
    CK(launch_ccl_batch(v, st));
  }
  return SW_OK;
}

int sw_probe_philox(int64_t calls_per_thread, int blocks, uint32_t* sink, void* stream) {
  if (calls_per_thread < 4 || calls_per_thread % 4 != 0 || blocks < 1 || !sink)
    return fail(SW_ERR_ARG, "sw_probe_philox: calls_per_thread must be a positive multiple of 4, blocks >= 1");
  CK(launch_philox_probe(calls_per_thread, blocks, sink, static_cast<cudaStream_t>(stream)));
  return SW_OK;
}

int ccl_status(void) {
  CK(cudaDeviceSynchronize());
  int* p = ccl_status_ptr();
  if (!p) return fail(SW_ERR_CUDA, "ccl_status: cannot resolve the device status word");
  int v = 0;
  CK(cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemset(p, 0, sizeof(int)));
  if (v) return fail(v, "ccl: a device-side consistency check failed");
  return SW_OK;
}

}  // extern "C"
