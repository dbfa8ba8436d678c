// swccl_noalloc.cu -- connected-component labeling that allocates nothing.
//
// ccl_label takes its scratch (tile-root lists, root counts, seam records)
// with cudaMallocAsync, and ccl_label_ws needs the caller to allocate it.
// Some callers can do neither when they label:
//   * latency-bound loops (serving) that must not call cudaMalloc/cudaFree,
//     since cudaFree synchronises the whole device and stalls other streams;
//   * programs whose device memory is owned by another framework's caching
//     allocator (an allocation behind its back can fail, because that
//     allocator holds the free memory, or break its accounting) and that
//     only pass inputs and outputs across this ABI.
// ccl_label_noalloc serves them: its scratch is a file-scope __device__
// array of CCL_NOALLOC_SCRATCH_BYTES.  The array exists on every GPU that
// loads the library, for the life of the process.
//
// In host code the array's name is only a host-side stand-in, not a device
// address; its device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and handed to the kernels.
// The first call on a device does this look-up (and that of the labeling
// status word), so it should come before any stream capture.
#include <mutex>
#include <string>

#include "swccl_shared.h"

using namespace swccl;

// Scratch of ccl_label_noalloc, shared by every call on this device.  Every
// part the kernels read is written by the same call first (root counts,
// root lists, seam records), so nothing needs clearing between calls.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CCL_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device; looked up on
// the first call per device.  Returns nullptr and fills `msg` on failure.
void* scratch_address(std::string& msg) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    msg = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return nullptr;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    msg = "device ordinal out of range";
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      msg = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
      return nullptr;
    }
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" int ccl_label_noalloc(const uint8_t* bond_mask, int32_t* labels, int H, int W, int periodic,
                                 void* stream) {
  if (!bond_mask || !labels) return set_last_error(SW_ERR_ARG, "ccl_label_noalloc: null device pointer");
  if (H < 1 || W < 1 || (int64_t)H * W >= ((int64_t)1 << 31))
    return set_last_error(SW_ERR_ARG, "ccl_label_noalloc: need H, W >= 1 and H*W < 2^31");
  const Grid g = make_grid(H, W, periodic);
  const int64_t need = label_scratch_bytes(g);
  if (need > (int64_t)CCL_NOALLOC_SCRATCH_BYTES)
    return set_last_error(SW_ERR_ARG, "ccl_label_noalloc: an " + std::to_string(H) + " x " + std::to_string(W) +
                                          " grid needs " + std::to_string(need) +
                                          " bytes of scratch, more than the fixed " +
                                          std::to_string((long long)CCL_NOALLOC_SCRATCH_BYTES) +
                                          "; use ccl_label or ccl_label_ws");
  std::string msg;
  void* ws = scratch_address(msg);
  if (!ws) return set_last_error(SW_ERR_CUDA, "ccl_label_noalloc: " + msg);
  int* status = ccl_status_word();
  if (!status) return set_last_error(SW_ERR_CUDA, "ccl_label_noalloc: cannot resolve the device status word");
  const LabelScratch s = carve_label_scratch(g, ws, status);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = launch_ccl(bond_mask, labels, g, s, st)) != cudaSuccess)
    return set_last_error(SW_ERR_CUDA, std::string("ccl_label_noalloc: launch: ") + cudaGetErrorString(e));
  return SW_OK;
}
