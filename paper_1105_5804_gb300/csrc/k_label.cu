// k_label.cu -- connected-component labeling of a packed bond mask.
//
// The paper's plan (Sec. II.B, II.C) is kept: label tiles independently,
// then consolidate labels across tile boundaries.  Its tile schemes
// (self-labeling, BFS, serial union-find) and its consolidation schemes
// (relaxation, hierarchical sewing) are replaced:
//
//  k_tile_label   one CTA per TILE_H x TILE_W tile.  Bond bits go to shared
//                 memory; each row is cut into runs of east-connected sites
//                 with one warp ballot per 32 sites (the run's leftmost site
//                 is its root); north bonds are joined with a lock-free
//                 shared-memory union-find that hooks larger roots under
//                 smaller ones, skipping a north bond whose left neighbour
//                 already joined the same two runs.  Each site's label is the
//                 global index of its tile-local root (the tile component's
//                 minimum site index); roots are appended to a per-tile list,
//                 and the labels and bond bits of the four tile edges go to a
//                 compact seam record.
//  k_merge        one thread per bond leaving a tile (the periodic wrap
//                 included, Sec. II.C): union of the two tile roots on the
//                 global label array with atomicMin hooking.  A lane whose
//                 root pair equals its left neighbour's skips the union, so
//                 consecutive seam bonds of one cluster cost one union.
//  k_root_compress  for every tile root: label = final root (pointer
//                 jumping).  Because hooks always go to the smaller index,
//                 the final root is the cluster's minimum site index.  In a
//                 Swendsen-Wang sweep the final roots also draw their
//                 cluster's new state here (Sec. II.D), keyed by the root.
//  k_site_compress  label[i] = label[label[i]] for every site (the staged
//                 sweep's dump of canonical labels).
// The stand-alone labeling (launch_ccl) uses k_ccl_tile, a k_tile_label that
// keeps every site's tile root as a 16-bit local index in the tile's scratch
// and writes label entries only for the tile roots on the tile edge (their
// parent entries), then k_merge, then k_ccl_final: per tile, each tile root
// finds its cluster root once and every site takes its tile root's from a
// shared-memory table -- every label written once, no gathers.
#include "label_tile.cuh"

namespace swccl {


__global__ void __launch_bounds__(LABEL_THREADS)
k_tile_label(const uint8_t* __restrict__ mask, int32_t* __restrict__ labels, Grid g, LabelScratch s) {
  __shared__ TileSmem sm;
  ccl_label_tile(mask, labels, g, s, blockIdx.x, sm);
}

cudaError_t launch_tile_label(const uint8_t* mask, int32_t* labels, const Grid& g,
                              const LabelScratch& s, cudaStream_t st) {
  k_tile_label<<<g.n_tiles(), LABEL_THREADS, 0, st>>>(mask, labels, g, s);
  return cudaGetLastError();
}

// Stand-alone labeling: local labeling with local-root labels, then (after
// the seam merge) the final labels of every tile in one pass.
__global__ void __launch_bounds__(LABEL_THREADS)
k_ccl_tile(const uint8_t* __restrict__ mask, int32_t* __restrict__ labels, Grid g, LabelScratch s) {
  __shared__ TileSmem sm;
  ccl_label_tile<true>(mask, labels, g, s, blockIdx.x, sm);
}

constexpr int FINAL_THREADS = 256;

__global__ void __launch_bounds__(FINAL_THREADS)
k_ccl_final(int32_t* labels, Grid g, LabelScratch s, int limit) {
  __shared__ int32_t table[TILE_SITES];
  final_labels_tile(labels, g, s, blockIdx.x, table, limit);
}

cudaError_t launch_ccl(const uint8_t* mask, int32_t* labels, const Grid& g, const LabelScratch& s, cudaStream_t st) {
  k_ccl_tile<<<g.n_tiles(), LABEL_THREADS, 0, st>>>(mask, labels, g, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = launch_merge(labels, g, s, st)) != cudaSuccess) return e;
  const int limit = (int)std::min<int64_t>(g.n_sites() + 64, (int64_t)1 << 30);
  k_ccl_final<<<g.n_tiles(), FINAL_THREADS, 0, st>>>(labels, g, s, limit);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Seam merge: thread k of tile t handles east seam bond k (k < TILE_H) or
// north seam bond k - TILE_H.
// ---------------------------------------------------------------------------
constexpr int MERGE_THREADS = 256;

__global__ void __launch_bounds__(MERGE_THREADS)
k_merge(int32_t* __restrict__ labels, Grid g, LabelScratch s, int limit) {
  const int64_t gid = blockIdx.x * (int64_t)MERGE_THREADS + threadIdx.x;
  const int64_t total = (int64_t)g.n_tiles() * MERGE_PER_TILE;
  if (gid - (threadIdx.x & 31) >= total) return;   // whole warp past the end
  const int t = (int)(gid / MERGE_PER_TILE);
  merge_seam_bond(labels, g, s, t, (int)(gid - (int64_t)t * MERGE_PER_TILE), gid < total, limit);
}

cudaError_t launch_merge(int32_t* labels, const Grid& g, const LabelScratch& s, cudaStream_t st) {
  const int64_t total = (int64_t)g.n_tiles() * MERGE_PER_TILE;
  const int64_t blocks = (total + MERGE_THREADS - 1) / MERGE_THREADS;
  const int limit = (int)std::min<int64_t>(g.n_sites() + 64, (int64_t)1 << 30);
  k_merge<<<(unsigned)blocks, MERGE_THREADS, 0, st>>>(labels, g, s, limit);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Root compression (+ root draws for a Swendsen-Wang sweep).
// ---------------------------------------------------------------------------
constexpr int ROOT_THREADS = 256;

__global__ void __launch_bounds__(ROOT_THREADS)
k_root_compress(int32_t* __restrict__ labels, Grid g, LabelScratch s, int8_t* __restrict__ spins,
                int q, uint64_t seed, const SwCtl* __restrict__ ctl, int limit) {
  root_compress_tile(labels, s, blockIdx.x, spins, q, seed, spins ? ctl->sweep : 0, limit);
}

cudaError_t launch_root_compress(int32_t* labels, const Grid& g, const LabelScratch& s,
                                 int8_t* spins, int q, uint64_t seed, const SwCtl* ctl,
                                 cudaStream_t st) {
  const int limit = (int)std::min<int64_t>(g.n_sites() + 64, (int64_t)1 << 30);
  k_root_compress<<<g.n_tiles(), ROOT_THREADS, 0, st>>>(labels, g, s, spins, q, seed, ctl, limit);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void k_site_compress(int32_t* __restrict__ labels, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = labels[i];
    const int R = labels[r];
    if (R != r) labels[i] = R;
  }
}

cudaError_t launch_site_compress(int32_t* labels, int64_t n_sites, cudaStream_t st) {
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((n_sites + threads - 1) / threads, 152 * 32);
  k_site_compress<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, st>>>(labels, n_sites);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
int64_t label_scratch_bytes(const Grid& g) {
  auto al = [](int64_t b) { return (b + 255) & ~(int64_t)255; };
  const int64_t nt = g.n_tiles();
  return 2 * al(nt * TILE_SITES * 4) + al(nt * 4) + al(nt * SeamLayout::INTS * 4) + al(4);
}

LabelScratch carve_label_scratch(const Grid& g, void* base, int* err) {
  auto al = [](int64_t b) { return (b + 255) & ~(int64_t)255; };
  const int64_t nt = g.n_tiles();
  char* p = static_cast<char*>(base);
  LabelScratch s;
  s.roots = reinterpret_cast<int32_t*>(p);
  p += al(nt * TILE_SITES * 4);
  s.work = reinterpret_cast<int32_t*>(p);
  p += al(nt * TILE_SITES * 4);
  s.root_counts = reinterpret_cast<int32_t*>(p);
  p += al(nt * 4);
  s.seams = reinterpret_cast<int32_t*>(p);
  p += al(nt * SeamLayout::INTS * 4);
  s.err = err ? err : reinterpret_cast<int*>(p);
  return s;
}

}  // namespace swccl
