// k_ccl_batch.cu -- labeling many bond masks of different sizes at once.
//
// The tiles of all grids are numbered consecutively (a binary search of the
// grids' tile ranges, which the kernels get by value, maps a global tile to
// its grid), and each step of the stand-alone labeling path (local
// labeling, seam merge, final labels) runs as one launch over all tiles of
// all grids.  A grid's labels are the same as ccl_label gives for it
// alone: every grid has its own label array and scratch, and the steps only
// ever touch the grid of the tile at hand.
#include "label_tile.cuh"

namespace swccl {

__device__ __forceinline__ int job_of_tile(const CclBatchView& v, int gt) {
  int lo = 0, hi = v.n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (gt < v.tile_end[mid]) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__global__ void __launch_bounds__(LABEL_THREADS) k_cclb_tile(const __grid_constant__ CclBatchView v) {
  __shared__ TileSmem sm;
  const int gt = blockIdx.x;
  const CclJob& J = v.jobs[job_of_tile(v, gt)];
  ccl_label_tile<true>(J.mask, J.labels, J.g, J.s, gt - J.tile0, sm);
}

__global__ void __launch_bounds__(MERGE_PER_TILE) k_cclb_merge(const __grid_constant__ CclBatchView v) {
  const int gt = blockIdx.x;
  const CclJob& J = v.jobs[job_of_tile(v, gt)];
  merge_seam_bond(J.labels, J.g, J.s, gt - J.tile0, threadIdx.x, true, v.limit);
}

__global__ void __launch_bounds__(256) k_cclb_final(const __grid_constant__ CclBatchView v) {
  __shared__ int32_t table[TILE_SITES];
  const int gt = blockIdx.x;
  const CclJob& J = v.jobs[job_of_tile(v, gt)];
  final_labels_tile(J.labels, J.g, J.s, gt - J.tile0, table, v.limit);
}

cudaError_t launch_ccl_batch(const CclBatchView& v, cudaStream_t st) {
  if (v.n_tiles == 0) return cudaSuccess;
  k_cclb_tile<<<v.n_tiles, LABEL_THREADS, 0, st>>>(v);
  k_cclb_merge<<<v.n_tiles, MERGE_PER_TILE, 0, st>>>(v);
  k_cclb_final<<<v.n_tiles, 256, 0, st>>>(v);
  return cudaGetLastError();
}

}  // namespace swccl
