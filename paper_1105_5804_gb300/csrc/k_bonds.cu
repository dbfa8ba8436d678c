// k_bonds.cu -- kernels that produce packed bond masks and initial spins.
//
//  * k_activate: Swendsen-Wang step 1 (Sec. II, list after Eq. 5; rule of
//    Eq. 7, Sec. II.A): the bond (i, j) is open iff s_i == s_j and the BOND
//    draw r_ij < T.  One Philox call serves the two x-adjacent sites 2m, 2m+1
//    (four words = their east and north bonds), so activation costs half a
//    call per site.  A thread owns four sites (one mask byte) of a column
//    strip and walks ACT_ROWS rows, reusing the north row it loaded as the
//    next row's own spins.
//  * k_perc_mask: critical bond percolation, every bond open with p = 1/2.
//  * k_pixel_bonds: image segmentation bonds (equal pixel value, Sec. I).
//  * k_init_spins: hot start from the INIT draw.
#include "swccl_device.cuh"

namespace swccl {

constexpr int ACT_THREADS = 256;
constexpr int ACT_ROWS = 8;

__global__ void __launch_bounds__(ACT_THREADS)
k_activate(const int8_t* __restrict__ spins, uint8_t* __restrict__ mask, int L, uint64_t T,
           uint64_t seed, const SwCtl* __restrict__ ctl, int64_t* __restrict__ obs_ring,
           int obs_cap, int q) {
  const uint64_t sweep = ctl->sweep;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x <= q) {
    // open this sweep's observable slot; the flip kernel accumulates into it
    obs_ring[(int64_t)(sweep % (uint64_t)obs_cap) * (q + 1) + threadIdx.x] = 0;
  }
  const int quads = L >> 2;
  const int xq = blockIdx.x * ACT_THREADS + threadIdx.x;
  if (xq >= quads) return;
  const int x = xq << 2;
  const int y0 = blockIdx.y * ACT_ROWS;
  const int y1 = min(y0 + ACT_ROWS, L);
  const bool all_open = T >= (1ull << 32);
  const uint32_t thr = (uint32_t)T;
  const uint32_t klo = (uint32_t)seed, khi = (uint32_t)(seed >> 32);
  const uint32_t sw_lo = (uint32_t)sweep, sw_hi = (uint32_t)(sweep >> 32);
  const int xe = (x + 4 == L) ? 0 : x + 4;

  uint32_t cur = *reinterpret_cast<const uint32_t*>(spins + (int64_t)y0 * L + x);
  for (int y = y0; y < y1; ++y) {
    const int yn = (y + 1 == L) ? 0 : y + 1;
    const int64_t row = (int64_t)y * L;
    const uint32_t nor = *reinterpret_cast<const uint32_t*>(spins + (int64_t)yn * L + x);
    const uint32_t east4 = (uint32_t)(uint8_t)spins[row + xe];
    // east neighbours of the four sites: bytes 1..3 of cur, then east4
    const uint32_t eastv = (cur >> 8) | (east4 << 24);
    const uint32_t eq_e = ~(cur ^ eastv);   // byte k all ones iff site k equals its east neighbour
    const uint32_t eq_n = ~(cur ^ nor);
    uint32_t out = 0;
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
      const int k0 = 2 * pr, k1 = 2 * pr + 1;
      const bool e0 = ((eq_e >> (8 * k0)) & 0xFF) == 0xFF;
      const bool n0 = ((eq_n >> (8 * k0)) & 0xFF) == 0xFF;
      const bool e1 = ((eq_e >> (8 * k1)) & 0xFF) == 0xFF;
      const bool n1 = ((eq_n >> (8 * k1)) & 0xFF) == 0xFF;
      uint32_t bits = 0;
      if (all_open) {
        bits = (e0 ? 1u : 0u) | (n0 ? 2u : 0u) | (e1 ? 4u : 0u) | (n1 ? 8u : 0u);
      } else if (thr != 0 && (e0 | n0 | e1 | n1)) {
        const uint32_t c0 = (uint32_t)((row + x) >> 1) + (uint32_t)pr;
        const uint4 r = philox(make_uint4(c0, sw_lo, sw_hi, TAG_BOND), klo, khi);
        bits = ((e0 && r.x < thr) ? 1u : 0u) | ((n0 && r.y < thr) ? 2u : 0u) |
               ((e1 && r.z < thr) ? 4u : 0u) | ((n1 && r.w < thr) ? 8u : 0u);
      }
      out |= bits << (4 * pr);
    }
    mask[(row + x) >> 2] = (uint8_t)out;
    cur = nor;
  }
}

cudaError_t launch_activate(const int8_t* spins, uint8_t* mask, int L, uint64_t T, uint64_t seed,
                            const SwCtl* ctl, int64_t* obs_ring, int obs_cap, int q,
                            cudaStream_t st) {
  dim3 grid((unsigned)((L / 4 + ACT_THREADS - 1) / ACT_THREADS), (unsigned)((L + ACT_ROWS - 1) / ACT_ROWS));
  k_activate<<<grid, ACT_THREADS, 0, st>>>(spins, mask, L, T, seed, ctl, obs_ring, obs_cap, q);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void k_perc_mask(uint8_t* __restrict__ mask, int64_t n_sites, uint64_t k) {
  const int64_t nbytes = (n_sites + 3) >> 2;
  const uint32_t klo = (uint32_t)k, khi = (uint32_t)(k >> 32);
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbytes;
       b += (int64_t)gridDim.x * blockDim.x) {
    uint32_t out = 0;
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
      const int64_t i = 4 * b + 2 * pr;
      if (i >= n_sites) break;
      const uint4 r = philox(make_uint4((uint32_t)(i >> 1), 0u, 0u, TAG_PERC), klo, khi);
      uint32_t bits = ((r.x >> 31) ^ 1u) | (((r.y >> 31) ^ 1u) << 1);
      if (i + 1 < n_sites) bits |= (((r.z >> 31) ^ 1u) << 2) | (((r.w >> 31) ^ 1u) << 3);
      out |= bits << (4 * pr);
    }
    mask[b] = (uint8_t)out;
  }
}

cudaError_t launch_perc_mask(uint8_t* mask, int H, int W, uint64_t k, cudaStream_t st) {
  const int64_t n = (int64_t)H * W, nbytes = (n + 3) / 4;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((nbytes + threads - 1) / threads, 152 * 64);
  k_perc_mask<<<(unsigned)blocks, threads, 0, st>>>(mask, n, k);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void k_pixel_bonds(const uint8_t* __restrict__ px, uint8_t* __restrict__ mask, int H,
                              int W, int periodic) {
  const int64_t n = (int64_t)H * W, nbytes = (n + 3) >> 2;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbytes;
       b += (int64_t)gridDim.x * blockDim.x) {
    uint32_t out = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = 4 * b + k;
      if (i >= n) break;
      const int y = (int)(i / W), x = (int)(i - (int64_t)y * W);
      const uint8_t v = px[i];
      uint32_t bits = 0;
      if (periodic || x + 1 < W) bits |= (v == px[(int64_t)y * W + (x + 1 == W ? 0 : x + 1)]) ? 1u : 0u;
      if (periodic || y + 1 < H) bits |= (v == px[(int64_t)(y + 1 == H ? 0 : y + 1) * W + x]) ? 2u : 0u;
      out |= bits << (2 * k);
    }
    mask[b] = (uint8_t)out;
  }
}

cudaError_t launch_pixel_bonds(const uint8_t* px, uint8_t* mask, int H, int W, int periodic,
                               cudaStream_t st) {
  const int64_t nbytes = ((int64_t)H * W + 3) / 4;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((nbytes + threads - 1) / threads, 152 * 64);
  k_pixel_bonds<<<(unsigned)blocks, threads, 0, st>>>(px, mask, H, W, periodic);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void k_init_spins(int8_t* __restrict__ spins, int64_t n, int q, uint64_t seed, int hot) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    spins[i] = hot ? (int8_t)state_of(draw((uint32_t)i, 0, TAG_INIT, seed).x, q) : (int8_t)0;
  }
}

cudaError_t launch_init_spins(int8_t* spins, int L, int q, uint64_t seed, int hot, cudaStream_t st) {
  const int64_t n = (int64_t)L * L;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, 152 * 64);
  k_init_spins<<<(unsigned)blocks, threads, 0, st>>>(spins, n, q, seed, hot);
  return cudaGetLastError();
}

cudaError_t launch_init_spins_n(int8_t* spins, int64_t n, int q, uint64_t seed, int hot, cudaStream_t st) {
  const int threads = 256;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 64));
  k_init_spins<<<(unsigned)blocks, threads, 0, st>>>(spins, n, q, seed, hot);
  return cudaGetLastError();
}

// Spin checks and device copies run on the SMs, not on a copy engine: a
// device-to-device copy on a copy engine queues behind host transfers that
// other streams have in flight, while a kernel overlaps them.  Sixteen bytes
// per thread and step where both pointers are 16-byte aligned.
__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

__global__ void k_check_spins(const int8_t* __restrict__ spins, int64_t n, int q, int* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const uint32_t qq = 0x01010101u * (uint32_t)q;   // a byte is valid iff it is below q (negative int8 >= 128)
  int64_t head = 0;
  if (aligned16(spins)) {
    const uint4* v = reinterpret_cast<const uint4*>(spins);
    bool bad = false;
    for (int64_t i = t0; i < n / 16; i += stride) {
      const uint4 w = v[i];
      bad |= (__vcmpgeu4(w.x, qq) | __vcmpgeu4(w.y, qq) | __vcmpgeu4(w.z, qq) | __vcmpgeu4(w.w, qq)) != 0u;
    }
    if (bad) set_error(err, SW_ERR_ARG);
    head = n / 16 * 16;
  }
  for (int64_t i = head + t0; i < n; i += stride) {
    const int s = spins[i];
    if (s < 0 || s >= q) set_error(err, SW_ERR_ARG);
  }
}

// dst = src if *ok_flag == 0 (left unchanged otherwise).
__global__ void k_copy_if(int8_t* __restrict__ dst, const int8_t* __restrict__ src, int64_t n,
                          const int* __restrict__ ok_flag) {
  if (ok_flag && *ok_flag != 0) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t head = 0;
  if (aligned16(dst) && aligned16(src)) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (int64_t i = t0; i < n / 16; i += stride) d4[i] = s4[i];
    head = n / 16 * 16;
  }
  for (int64_t i = head + t0; i < n; i += stride) dst[i] = src[i];
}

static unsigned sm_copy_blocks(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n / 16 + 255) / 256, 152 * 16));
}

cudaError_t launch_check_spins(const int8_t* spins, int64_t n, int q, int* err, cudaStream_t st) {
  k_check_spins<<<sm_copy_blocks(n), 256, 0, st>>>(spins, n, q, err);
  return cudaGetLastError();
}

cudaError_t launch_copy_if(int8_t* dst, const int8_t* src, int64_t n, const int* ok_flag, cudaStream_t st) {
  k_copy_if<<<sm_copy_blocks(n), 256, 0, st>>>(dst, src, n, ok_flag);
  return cudaGetLastError();
}

// A check's failure code (flag != 0) is recorded in a status word; the
// first code there stays.
__global__ void k_note_error(const int* __restrict__ flag, int* err) {
  const int f = *flag;
  if (threadIdx.x == 0 && f != 0) atomicCAS(err, 0, f);
}

cudaError_t launch_note_error(const int* flag, int* err, cudaStream_t st) {
  k_note_error<<<1, 32, 0, st>>>(flag, err);
  return cudaGetLastError();
}

}  // namespace swccl

namespace swccl {

// ---------------------------------------------------------------------------
// Measurement helper: Philox4x32-10 throughput with no memory traffic.  Each
// thread makes `calls` independent calls (counter = thread id, call index)
// and folds the outputs into one word, stored once so that nothing is
// optimised away.  Times of this kernel give the integer-ALU ceiling of the
// bond draws.
__global__ void __launch_bounds__(256) k_philox_probe(long long calls, uint32_t* __restrict__ sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (long long i = 0; i < calls; i += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint4 r = philox(make_uint4(tid, (uint32_t)(i + u), 0u, TAG_BOND), 0x1234u, 0x5678u);
      acc ^= r.x ^ r.y ^ r.z ^ r.w;
    }
  }
  sink[tid] = acc;
}

cudaError_t launch_philox_probe(long long calls_per_thread, int blocks, uint32_t* sink, cudaStream_t st) {
  k_philox_probe<<<blocks, 256, 0, st>>>(calls_per_thread, sink);
  return cudaGetLastError();
}

}  // namespace swccl
