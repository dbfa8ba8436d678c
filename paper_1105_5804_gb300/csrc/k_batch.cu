// k_batch.cu -- fused Swendsen-Wang sweeps of many independent lattices.
//
// A batch holds R chains of different sizes and temperatures (one SwRep
// each).  Their tiles are numbered consecutively; tile_rep[] maps a global
// tile to its chain.  Two schedules run the same three steps of the fused
// sweep (draw + label, seam merge, flip) over all tiles of all chains:
//
//  * phases: one launch per step over the global tile list (CUDA graph of
//    four kernels per sweep); kernel boundaries order the steps;
//  * persistent: one cooperative launch per sweep.  Each CTA walks the
//    global tile list step by step; a grid barrier separates the steps.  The
//    barrier's wait is bounded: if it does not complete within the time
//    limit, the kernel records SW_ERR_TIMEOUT and returns, so it can never
//    hang the device.
//
// Small lattices alone leave most SMs idle (L = 64 is two tiles); in one
// batch their tiles fill the machine.  Every chain draws from its own seed,
// so a chain's result is the same alone or in any batch.
#include "fused_tile.cuh"

namespace swccl {

namespace {

__device__ __forceinline__ bool batch_do_obs(const BatchCtl* ctl, uint64_t sweep) {
  return sweep > 0 && ctl->obs_done != (long long)(sweep - 1);
}

// Zero the observable slot of sweep s of every chain (the next sweep's draw
// step, or the observe kernel, fills it), then advance.  One CTA.
__device__ __forceinline__ void batch_advance_block(const BatchView& b, BatchCtl* ctl, uint64_t s) {
  for (int r = 0; r < b.n_reps; ++r) {
    const SwRep& R = b.reps[r];
    int64_t* slot = R.obs + (int64_t)(s % (uint64_t)b.obs_cap) * (R.q + 1);
    for (int k = threadIdx.x; k <= R.q; k += blockDim.x) slot[k] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) ctl->sweep = s + 1;
}

// Grid barrier for co-resident CTAs (cooperative launch).  Returns false if
// the wait ran out (limit_cycles of clock64()) or another CTA already
// failed; the error is recorded.  After a failure the barrier's counters are
// left as they are: the batch is not swept again (the host refuses).
__device__ __forceinline__ bool grid_barrier(BatchCtl* ctl, unsigned nblocks, long long limit_cycles) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = &ctl->bar_gen;
    const unsigned my_gen = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
    if (arrived == nblocks) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      // the limit is tested before the flag, so a limit of 0 makes every
      // CTA but the last give up at once
      const long long t0 = clock64();
      for (;;) {
        if (clock64() - t0 >= limit_cycles) {
          atomicCAS(&ctl->err, 0, SW_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        if (*gen != my_gen) break;
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*reinterpret_cast<volatile int*>(&ctl->err) != 0) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// Phase kernels: one CTA per global tile (merge: one thread per seam bond).
__global__ void __launch_bounds__(LABEL_THREADS, LABEL_CTAS_PER_SM) k_batch_label(BatchView b, const BatchCtl* __restrict__ ctl) {
  __shared__ LabelTileSmem ls;
  const uint64_t sweep = ctl->sweep;
  const bool do_obs = batch_do_obs(ctl, sweep);
  const int gt = blockIdx.x;
  const SwRep& R = b.reps[b.tile_rep[gt]];
  sw_label_tile(R, gt - R.tile0, sweep, do_obs, b.obs_cap, ls, SeedKey{(uint32_t)R.seed, (uint32_t)(R.seed >> 32)});
}

constexpr int BATCH_MERGE_THREADS = MERGE_PER_TILE;   // one CTA per tile

__global__ void __launch_bounds__(BATCH_MERGE_THREADS) k_batch_merge(BatchView b) {
  const int gt = blockIdx.x;
  const SwRep& R = b.reps[b.tile_rep[gt]];
  merge_seam_bond(R.gpar, R.g, R.s, gt - R.tile0, threadIdx.x, true, b.limit);
}

__global__ void __launch_bounds__(LABEL_THREADS, FLIP_CTAS_PER_SM) k_batch_flip(BatchView b, const BatchCtl* __restrict__ ctl) {
  __shared__ FlipTileSmem fs;
  const int gt = blockIdx.x;
  const SwRep& R = b.reps[b.tile_rep[gt]];
  sw_flip_tile(R, gt - R.tile0, ctl->sweep, b.limit, fs, SeedKey{(uint32_t)R.seed, (uint32_t)(R.seed >> 32)});
}

__global__ void k_batch_advance(BatchView b, BatchCtl* ctl) { batch_advance_block(b, ctl, ctl->sweep); }

__global__ void __launch_bounds__(LABEL_THREADS) k_batch_observe(BatchView b, BatchCtl* ctl) {
  __shared__ LabelTileSmem ls;
  const uint64_t done = ctl->sweep - 1;
  const int gt = blockIdx.x;
  const SwRep& R = b.reps[b.tile_rep[gt]];
  observe_tile(R, gt - R.tile0, done, b.obs_cap, ls);
  if (gt == 0 && threadIdx.x == 0) ctl->obs_done = (long long)done;
}

// ---------------------------------------------------------------------------
// Persistent kernel: the whole sweep in one cooperative launch.
union PersistentSmem {
  LabelTileSmem label;
  FlipTileSmem flip;
};

__global__ void __launch_bounds__(LABEL_THREADS, 4 * 256 / TILE_W) k_batch_persistent(BatchView b, BatchCtl* ctl, long long limit_cycles) {
  __shared__ PersistentSmem u;
  const uint64_t sweep = ctl->sweep;
  const bool do_obs = batch_do_obs(ctl, sweep);
  const unsigned nb = gridDim.x;
  // 1. draw bonds and label every tile
  for (int gt = blockIdx.x; gt < b.n_tiles; gt += nb) {
    const SwRep& R = b.reps[b.tile_rep[gt]];
    sw_label_tile(R, gt - R.tile0, sweep, do_obs, b.obs_cap, u.label,
                  SeedKey{(uint32_t)R.seed, (uint32_t)(R.seed >> 32)});
  }
  if (!grid_barrier(ctl, nb, limit_cycles)) return;
  // 2. seam merge: warp w of the CTA takes bonds 32w..32w+31 of a tile
  {
    constexpr int WARPS = LABEL_THREADS / 32, WPT = MERGE_PER_TILE / 32;
    const int64_t n_units = (int64_t)b.n_tiles * WPT;
    for (int64_t unit = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5); unit < n_units;
         unit += (int64_t)nb * WARPS) {
      const int gt = (int)(unit / WPT), part = (int)(unit - (int64_t)gt * WPT);
      const SwRep& R = b.reps[b.tile_rep[gt]];
      merge_seam_bond(R.gpar, R.g, R.s, gt - R.tile0, part * 32 + (threadIdx.x & 31), true, b.limit);
    }
  }
  if (!grid_barrier(ctl, nb, limit_cycles)) return;
  // 3. flip every tile
  for (int gt = blockIdx.x; gt < b.n_tiles; gt += nb) {
    const SwRep& R = b.reps[b.tile_rep[gt]];
    sw_flip_tile(R, gt - R.tile0, sweep, b.limit, u.flip, SeedKey{(uint32_t)R.seed, (uint32_t)(R.seed >> 32)});
  }
  if (!grid_barrier(ctl, nb, limit_cycles)) return;
  if (blockIdx.x == 0) batch_advance_block(b, ctl, sweep);
}

// ---------------------------------------------------------------------------
cudaError_t launch_batch_label(const BatchView& b, BatchCtl* ctl, cudaStream_t st) {
  k_batch_label<<<b.n_tiles, LABEL_THREADS, 0, st>>>(b, ctl);
  return cudaGetLastError();
}

cudaError_t launch_batch_merge(const BatchView& b, cudaStream_t st) {
  k_batch_merge<<<b.n_tiles, BATCH_MERGE_THREADS, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_batch_flip(const BatchView& b, BatchCtl* ctl, cudaStream_t st) {
  k_batch_flip<<<b.n_tiles, LABEL_THREADS, 0, st>>>(b, ctl);
  return cudaGetLastError();
}

cudaError_t launch_batch_advance(const BatchView& b, BatchCtl* ctl, cudaStream_t st) {
  k_batch_advance<<<1, 128, 0, st>>>(b, ctl);
  return cudaGetLastError();
}

cudaError_t launch_batch_observe(const BatchView& b, BatchCtl* ctl, cudaStream_t st) {
  k_batch_observe<<<b.n_tiles, LABEL_THREADS, 0, st>>>(b, ctl);
  return cudaGetLastError();
}

int batch_persistent_blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_persistent, LABEL_THREADS, 0) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_batch_persistent(const BatchView& b, BatchCtl* ctl, int blocks, long long limit_cycles,
                                    cudaStream_t st) {
  void* args[] = {(void*)&b, (void*)&ctl, (void*)&limit_cycles};
  return cudaLaunchCooperativeKernel((const void*)k_batch_persistent, dim3(blocks), dim3(LABEL_THREADS), args, 0, st);
}

}  // namespace swccl
