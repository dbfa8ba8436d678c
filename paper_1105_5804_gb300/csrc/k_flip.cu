// k_flip.cu -- Swendsen-Wang step 3 (Sec. II.D) and the observables of Eq. 1.
//
// After root compression every site's label points at its tile root and the
// tile root's entry holds the cluster's final root R (its minimum site
// index), whose new state was drawn into spins[R] (FLIP draw keyed by R).
// The flip therefore needs no per-site random number: s_i = spins[lab[lab[i]]].
// The paper drew a state at every site and read it at the root (Sec. II.D);
// drawing only at roots removes that work.
//
// Each thread owns four sites of a row (one int4 of labels) and walks
// FLIP_ROWS rows plus one halo row, so that it can count the bonds joining
// equal new spins (n_eq) and the sites per state (n_k) of the new
// configuration; one block reduction and one atomic per counter per block
// accumulate them into the sweep's slot of the observable ring.
#include "swccl_device.cuh"

namespace swccl {

constexpr int FLIP_THREADS = 256;
constexpr int FLIP_ROWS = 16;

template <int QMAX>
struct StateCounts {
  int c[QMAX];
  __device__ void zero() {
#pragma unroll
    for (int k = 0; k < QMAX; ++k) c[k] = 0;
  }
  __device__ void add(int s) {
#pragma unroll
    for (int k = 0; k < QMAX; ++k) c[k] += (s == k);
  }
};

__device__ __forceinline__ int new_state(const int8_t* spins, const int32_t* lab, int64_t i) {
  return spins[lab[lab[i]]];
}

// QMAX > 0: q <= QMAX, per-thread register counters.  QMAX == 0: any q,
// shared-memory histogram.
template <int QMAX>
__global__ void __launch_bounds__(FLIP_THREADS)
k_flip(int8_t* __restrict__ spins, const int32_t* __restrict__ lab, int L, int q,
       const SwCtl* __restrict__ ctl, int64_t* __restrict__ obs_ring, int obs_cap) {
  constexpr int NC = QMAX > 0 ? QMAX : 1;
  __shared__ unsigned long long red[FLIP_THREADS / 32][1 + (QMAX > 0 ? QMAX : 0)];
  __shared__ int hist[QMAX > 0 ? 1 : 128];
  if (QMAX == 0) {
    for (int k = threadIdx.x; k < 128; k += FLIP_THREADS) hist[k] = 0;
    __syncthreads();
  }
  StateCounts<NC> cnt;
  cnt.zero();
  int n_eq = 0;

  const int quads = L >> 2;
  const int xq = blockIdx.x * FLIP_THREADS + threadIdx.x;
  const int y0 = blockIdx.y * FLIP_ROWS;
  const int y1 = min(y0 + FLIP_ROWS, L);
  if (xq < quads) {
    const int x = xq << 2;
    const int xe = (x + 4 == L) ? 0 : x + 4;
    int prev[4] = {0, 0, 0, 0};
    for (int y = y0; y <= y1; ++y) {
      const int yy = (y == L) ? 0 : y;
      const int64_t row = (int64_t)yy * L;
      const int4 l4 = *reinterpret_cast<const int4*>(lab + row + x);
      int sv[4];
      sv[0] = spins[lab[l4.x]];
      sv[1] = spins[lab[l4.y]];
      sv[2] = spins[lab[l4.z]];
      sv[3] = spins[lab[l4.w]];
      if (y > y0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) n_eq += (prev[k] == sv[k]);
      }
      if (y < y1) {
        const int se = new_state(spins, lab, row + xe);
        n_eq += (sv[0] == sv[1]) + (sv[1] == sv[2]) + (sv[2] == sv[3]) + (sv[3] == se);
        const uint32_t packed = (uint32_t)(uint8_t)sv[0] | ((uint32_t)(uint8_t)sv[1] << 8) |
                                ((uint32_t)(uint8_t)sv[2] << 16) | ((uint32_t)(uint8_t)sv[3] << 24);
        *reinterpret_cast<uint32_t*>(spins + row + x) = packed;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (QMAX > 0) cnt.add(sv[k]);
          else atomicAdd(&hist[sv[k]], 1);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) prev[k] = sv[k];
    }
  }

  // block reduction: n_eq and (register) state counts
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long v = (unsigned long long)n_eq;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  if (lane == 0) red[warp][0] = v;
  if (QMAX > 0) {
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      unsigned long long c = (unsigned long long)cnt.c[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
      if (lane == 0 && QMAX > 0) red[warp][1 + (k < QMAX ? k : 0)] = c;
    }
  }
  __syncthreads();
  const uint64_t sweep = ctl->sweep;
  unsigned long long* slot =
      reinterpret_cast<unsigned long long*>(obs_ring + (int64_t)(sweep % (uint64_t)obs_cap) * (q + 1));
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (int w = 0; w < FLIP_THREADS / 32; ++w) tot += red[w][0];
    if (tot) atomicAdd(slot, tot);
  }
  if (QMAX > 0) {
    if (threadIdx.x >= 1 && threadIdx.x <= q) {
      const int k = threadIdx.x - 1;
      unsigned long long tot = 0;
      for (int w = 0; w < FLIP_THREADS / 32; ++w) tot += red[w][1 + (k < NC ? k : 0)];
      if (tot) atomicAdd(slot + 1 + k, tot);
    }
  } else {
    for (int k = threadIdx.x; k < q; k += FLIP_THREADS)
      if (hist[k]) atomicAdd(slot + 1 + k, (unsigned long long)hist[k]);
  }
}

cudaError_t launch_flip(int8_t* spins, const int32_t* labels, int L, int q, const SwCtl* ctl,
                        int64_t* obs_ring, int obs_cap, cudaStream_t st) {
  dim3 grid((unsigned)((L / 4 + FLIP_THREADS - 1) / FLIP_THREADS), (unsigned)((L + FLIP_ROWS - 1) / FLIP_ROWS));
  if (q == 2) k_flip<2><<<grid, FLIP_THREADS, 0, st>>>(spins, labels, L, q, ctl, obs_ring, obs_cap);
  else if (q <= 4) k_flip<4><<<grid, FLIP_THREADS, 0, st>>>(spins, labels, L, q, ctl, obs_ring, obs_cap);
  else if (q <= 8) k_flip<8><<<grid, FLIP_THREADS, 0, st>>>(spins, labels, L, q, ctl, obs_ring, obs_cap);
  else k_flip<0><<<grid, FLIP_THREADS, 0, st>>>(spins, labels, L, q, ctl, obs_ring, obs_cap);
  return cudaGetLastError();
}

__global__ void k_advance(SwCtl* ctl) { ctl->sweep += 1; }

cudaError_t launch_advance(SwCtl* ctl, cudaStream_t st) {
  k_advance<<<1, 1, 0, st>>>(ctl);
  return cudaGetLastError();
}

}  // namespace swccl
