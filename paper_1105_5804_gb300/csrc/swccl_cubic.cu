// swccl_cubic.cu -- host side of the simple-cubic Swendsen-Wang chain
// (sw3_* in include/swccl.h; kernels in k_cubic.cu).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "swccl_shared.h"

using namespace swccl;

namespace {

constexpr int OBS3_CAP = 4096;

int fail3(int code, const std::string& msg) { return set_last_error(code, msg); }

int cuda_fail3(cudaError_t e, const char* what) {
  return set_last_error(SW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK3(call)                                    \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail3(e_, #call); \
  } while (0)

}  // namespace

struct sw3_handle {
  Box3 box{};
  int q = 0;
  uint64_t T = 0, seed = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int8_t* spins = nullptr;
  uint16_t* lroot = nullptr;      // brick root of every site (16-bit local index)
  int32_t* gpar = nullptr;        // parents of edge roots; also staging for host spins
  uint32_t* edge_words = nullptr; // edge-root bits of every brick
  int32_t* scratch = nullptr;     // labeling scratch of every brick
  SwCtl* ctl = nullptr;
  int* chk = nullptr;             // spin-check flag of sw3_set_spins
  int64_t* obs = nullptr;
  uint64_t sweeps = 0, obs_read = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool timing = false;
  bool labels_valid = false;
  bool final_obs_pending = false;   // the last sweep's observables are counted when read
  std::vector<cudaEvent_t> ev_pending;   // SW3_N_PHASES + 1 per timed sweep
  std::vector<cudaEvent_t> ev_free;
};

namespace {

void free3(sw3_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  for (auto e : h->ev_pending) cudaEventDestroy(e);
  for (auto e : h->ev_free) cudaEventDestroy(e);
  cudaFree(h->spins);
  cudaFree(h->lroot);
  cudaFree(h->gpar);
  cudaFree(h->edge_words);
  cudaFree(h->scratch);
  cudaFree(h->ctl);
  cudaFree(h->chk);
  cudaFree(h->obs);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// The next sweep's local step counts a sweep's observables; before they are
// read or the spins replaced, count the last sweep's here.
cudaError_t finish3(sw3_handle* h) {
  if (!h->final_obs_pending) return cudaSuccess;
  h->final_obs_pending = false;
  return launch_observe3(h->spins, h->box, h->q, h->ctl, h->obs, OBS3_CAP, h->stream);
}

// Synchronous copy ordered on the handle's stream (not the legacy default stream).
cudaError_t copy3(cudaStream_t st, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, st);
  return e != cudaSuccess ? e : cudaStreamSynchronize(st);
}

int status3(sw3_handle* h) {
  CK3(cudaStreamSynchronize(h->stream));
  SwCtl c;
  CK3(copy3(h->stream, &c, h->ctl, sizeof(c), cudaMemcpyDeviceToHost));
  if (c.err) return fail3(c.err, "a device-side consistency check failed in a 3D sweep");
  return SW_OK;
}

}  // namespace

extern "C" {

sw3_handle* sw3_create(int X, int Y, int Z, int q, uint64_t T, uint64_t seed, int hot_start, void* stream) {
  const int64_t n = (int64_t)X * Y * Z;
  if (X < 1 || Y < 1 || Z < 1 || n > ((int64_t)1 << 30)) {
    fail3(SW_ERR_ARG, "sw3_create: need X, Y, Z >= 1 and X*Y*Z <= 2^30");
    return nullptr;
  }
  if (q < 2 || q > 127 || T > (1ull << 32)) {
    fail3(SW_ERR_ARG, "sw3_create: need 2 <= q <= 127 and T <= 2^32");
    return nullptr;
  }
  sw3_handle* h = new sw3_handle();
  h->box = make_box3(X, Y, Z);
  h->q = q;
  h->T = T;
  h->seed = seed;
  auto bail = [&](int code, const std::string& m) -> sw3_handle* {
    fail3(code, m);
    free3(h);
    return nullptr;
  };
  if (stream) {
    h->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(SW_ERR_CUDA, "sw3_create: cudaStreamCreate failed");
    h->own_stream = true;
  }
  if (cudaMalloc(&h->spins, (size_t)n) != cudaSuccess || cudaMalloc(&h->gpar, (size_t)n * 4) != cudaSuccess ||
      cudaMalloc(&h->lroot, (size_t)n * 2) != cudaSuccess ||
      cudaMalloc(&h->edge_words, (size_t)edge_words3(h->box) * 4) != cudaSuccess ||
      cudaMalloc(&h->scratch, (size_t)scratch_ints3(h->box) * 4) != cudaSuccess ||
      cudaMalloc(&h->ctl, sizeof(SwCtl)) != cudaSuccess || cudaMalloc(&h->chk, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->obs, (size_t)OBS3_CAP * (q + 1) * 8) != cudaSuccess) {
    cudaGetLastError();
    return bail(SW_ERR_OOM, "sw3_create: cudaMalloc failed");
  }
  SwCtl c{};
  c.obs_done = -1;
  if (cudaMemcpyAsync(h->ctl, &c, sizeof(c), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->obs, 0, (size_t)OBS3_CAP * (q + 1) * 8, h->stream) != cudaSuccess ||
      launch_init_spins_n(h->spins, n, q, seed, hot_start ? 1 : 0, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return bail(SW_ERR_CUDA, "sw3_create: initialisation failed");
  return h;
}

sw3_handle* sw3_create_ex(int X, int Y, int Z, int q, double beta, double J, int convention, uint64_t seed,
                          int hot_start, void* stream) {
  if (!(beta >= 0.0) || convention < 0 || convention > 2) {
    fail3(SW_ERR_ARG, "sw3_create_ex: beta must be >= 0 and convention in {0,1,2}");
    return nullptr;
  }
  return sw3_create(X, Y, Z, q, sw_threshold_for(q, beta, J, convention), seed, hot_start, stream);
}

int sw3_destroy(sw3_handle* h) {
  free3(h);
  return SW_OK;
}

int sw3_sweep(sw3_handle* h, int n) {
  if (!h || n < 0) return fail3(SW_ERR_ARG, "sw3_sweep: bad arguments");
  if (n == 0) return SW_OK;
  if (h->timing) {
    for (int k = 0; k < n; ++k) {
      cudaEvent_t ev[SW3_N_PHASES + 1];
      for (auto& e : ev) {
        if (!h->ev_free.empty()) {
          e = h->ev_free.back();
          h->ev_free.pop_back();
        } else {
          CK3(cudaEventCreate(&e));
        }
        h->ev_pending.push_back(e);
      }
      CK3(launch_sweep3(h->spins, h->lroot, h->gpar, h->edge_words, h->scratch, h->box, h->q, h->T, h->seed, h->ctl,
                        h->obs, OBS3_CAP, h->stream, ev));
      h->sweeps++;
    }
  } else {
    if (!h->exec) {
      CK3(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = launch_sweep3(h->spins, h->lroot, h->gpar, h->edge_words, h->scratch, h->box, h->q, h->T,
                                    h->seed, h->ctl, h->obs, OBS3_CAP, h->stream, nullptr);
      cudaGraph_t gr = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(h->stream, &gr);
      if (e != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return cuda_fail3(e, "capture of one 3D sweep");
      }
      if (e2 != cudaSuccess) return cuda_fail3(e2, "cudaStreamEndCapture");
      h->graph = gr;
      CK3(cudaGraphInstantiate(&h->exec, h->graph, 0));
    }
    for (int k = 0; k < n; ++k) {
      CK3(cudaGraphLaunch(h->exec, h->stream));
      h->sweeps++;
    }
  }
  h->labels_valid = true;
  h->final_obs_pending = true;
  return SW_OK;
}

int sw3_sync(sw3_handle* h) {
  if (!h) return fail3(SW_ERR_ARG, "sw3_sync: null handle");
  return status3(h);
}

int sw3_observables(sw3_handle* h, int64_t* out, int max_sweeps, int* n_written) {
  if (!h || (!out && max_sweeps > 0) || max_sweeps < 0) return fail3(SW_ERR_ARG, "sw3_observables: bad arguments");
  if (n_written) *n_written = 0;
  CK3(finish3(h));
  int rc = status3(h);
  if (rc) return rc;
  if (h->sweeps - h->obs_read > (uint64_t)OBS3_CAP) h->obs_read = h->sweeps - OBS3_CAP;
  const int64_t cnt = std::min<int64_t>((int64_t)(h->sweeps - h->obs_read), max_sweeps);
  const int row = h->q + 1;
  int64_t done = 0;
  while (done < cnt) {
    const int64_t slot = (int64_t)((h->obs_read + done) % OBS3_CAP);
    const int64_t run = std::min<int64_t>(cnt - done, OBS3_CAP - slot);
    CK3(copy3(h->stream, out + done * row, h->obs + slot * row, run * row * 8, cudaMemcpyDeviceToHost));
    done += run;
  }
  h->obs_read += cnt;
  if (n_written) *n_written = (int)cnt;
  return SW_OK;
}

int sw3_get_spins(sw3_handle* h, int8_t* dst, int is_device) {
  if (!h || !dst) return fail3(SW_ERR_ARG, "sw3_get_spins: bad arguments");
  int rc = status3(h);
  if (rc) return rc;
  if (is_device) {
    CK3(launch_copy_if(dst, h->spins, h->box.n(), nullptr, h->stream));
    CK3(cudaStreamSynchronize(h->stream));
  } else {
    CK3(copy3(h->stream, dst, h->spins, (size_t)h->box.n(), cudaMemcpyDeviceToHost));
  }
  return SW_OK;
}

int sw3_set_spins(sw3_handle* h, const int8_t* src, int is_device) {
  if (!h || !src) return fail3(SW_ERR_ARG, "sw3_set_spins: bad arguments");
  const int64_t n = h->box.n();
  CK3(finish3(h));   // the pending observables belong to the old spins
  int rc = status3(h);
  if (rc) return rc;
  // host input is staged in the parent array (4n bytes, rewritten by the
  // next sweep) and checked there; the spins change only if all are in [0, q)
  const int8_t* dsrc = src;
  if (!is_device) {
    int8_t* staging = reinterpret_cast<int8_t*>(h->gpar);
    CK3(cudaMemcpyAsync(staging, src, (size_t)n, cudaMemcpyHostToDevice, h->stream));
    dsrc = staging;
    h->labels_valid = false;
  }
  CK3(cudaMemsetAsync(h->chk, 0, sizeof(int), h->stream));
  CK3(launch_check_spins(dsrc, n, h->q, h->chk, h->stream));
  CK3(launch_copy_if(h->spins, dsrc, n, h->chk, h->stream));   // only if every value is valid
  int bad = 0;
  CK3(copy3(h->stream, &bad, h->chk, sizeof(int), cudaMemcpyDeviceToHost));
  if (bad) return fail3(SW_ERR_ARG, "sw3_set_spins: a spin is outside [0, q)");
  return SW_OK;
}

int sw3_labels(sw3_handle* h, int32_t* out, int is_device) {
  if (!h || !out) return fail3(SW_ERR_ARG, "sw3_labels: bad arguments");
  if (!h->labels_valid) return fail3(SW_ERR_STATE, "sw3_labels: no sweep since creation or the last host sw3_set_spins");
  const int64_t n = h->box.n();
  int32_t* dst = out;
  if (!is_device) CK3(cudaMalloc(&dst, (size_t)n * 4));
  cudaError_t e = launch_labels3(h->lroot, h->gpar, h->edge_words, h->box, dst, &h->ctl->err, h->stream);
  if (e == cudaSuccess && !is_device) e = cudaMemcpyAsync(out, dst, (size_t)n * 4, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (!is_device) cudaFree(dst);
  if (e != cudaSuccess) return cuda_fail3(e, "sw3_labels");
  return status3(h);
}

void* sw3_stream(sw3_handle* h) { return h ? static_cast<void*>(h->stream) : nullptr; }

int sw3_get_info(sw3_handle* h, int64_t* info) {
  if (!h || !info) return fail3(SW_ERR_ARG, "sw3_get_info: bad arguments");
  const int64_t v[8] = {h->box.X, h->box.Y, h->box.Z, h->q, (int64_t)h->T, (int64_t)h->seed, (int64_t)h->sweeps,
                        OBS3_CAP};
  std::memcpy(info, v, sizeof(v));
  return SW_OK;
}

int sw3_set_timing(sw3_handle* h, int enable) {
  if (!h) return fail3(SW_ERR_ARG, "sw3_set_timing: null handle");
  h->timing = enable != 0;
  return SW_OK;
}

int sw3_phase_times(sw3_handle* h, double* ms, int64_t* n_sweeps) {
  if (!h || !ms) return fail3(SW_ERR_ARG, "sw3_phase_times: bad arguments");
  CK3(cudaStreamSynchronize(h->stream));
  for (int k = 0; k < SW3_N_PHASES; ++k) ms[k] = 0.0;
  const size_t per = SW3_N_PHASES + 1;
  const size_t n = h->ev_pending.size() / per;
  for (size_t s = 0; s < n; ++s) {
    for (int k = 0; k < SW3_N_PHASES; ++k) {
      float t = 0.f;
      CK3(cudaEventElapsedTime(&t, h->ev_pending[s * per + k], h->ev_pending[s * per + k + 1]));
      ms[k] += t;
    }
  }
  for (auto e : h->ev_pending) h->ev_free.push_back(e);
  h->ev_pending.clear();
  if (n_sweeps) *n_sweeps = (int64_t)n;
  return SW_OK;
}

}  // extern "C"
