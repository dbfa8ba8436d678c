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
//  k_site_compress  label[i] = label[label[i]] for every site (stand-alone
//                 labeling only: leaves every label canonical).
#include "tile_engine.cuh"

namespace swccl {


// Local labeling of one tile for the stand-alone labeling path: the tile's
// bond bits are copied from the packed mask into shared memory (bits of
// sites outside the grid and the east bond of the tile's last column
// cleared), the engine of tile_engine.cuh labels the tile, and the kernel
// writes every site's label (global index of its tile root, the minimum
// site index of its tile component), the tile's root list, and the seam
// record (labels and outgoing bond bits of the four tile edges).
__global__ void __launch_bounds__(LABEL_THREADS)
k_tile_label(const uint8_t* __restrict__ mask, int32_t* __restrict__ labels, Grid g,
             LabelScratch s) {
  __shared__ TileSmem sm;
  int* par = sm.par;
  unsigned long long* mb = sm.mb;
  int* warp_roots = sm.warp_roots;

  const int t = blockIdx.x;
  const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
  const int y0 = ty * TILE_H, x0 = tx * TILE_W;
  const int h = min(TILE_H, g.H - y0), w = min(TILE_W, g.W - x0);
  const int W = g.W;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t* slot = s.roots + (int64_t)t * TILE_SITES;     // pair lists, later the root list
  int32_t* hook_log = s.work + (int64_t)t * TILE_SITES;
  if (threadIdx.x == 0) sm.n_hooked = 0;

  // 1. bond bits
  for (int k = threadIdx.x; k < TILE_H * STRIPS; k += LABEL_THREADS) {
    const int ly = k / STRIPS, c = k - ly * STRIPS;
    const int nvalid = min(max(w - 32 * c, 0), 32);
    unsigned long long wd = 0ull;
    if (ly < h && nvalid > 0) {
      const int64_t site0 = (int64_t)(y0 + ly) * W + x0 + 32 * c;
      if ((W & 31) == 0 && (reinterpret_cast<uintptr_t>(mask) & 7) == 0) {
        wd = reinterpret_cast<const unsigned long long*>(mask)[site0 >> 5];
      } else {
        for (int i = 0; i < nvalid; ++i) wd |= (unsigned long long)site_bits(mask, site0 + i) << (2 * i);
      }
      if (nvalid < 32) wd &= (1ull << (2 * nvalid)) - 1ull;
      if (32 * c + nvalid == w) wd &= ~(1ull << (2 * (nvalid - 1)));   // east bond leaving the tile
    }
    mb[k] = wd;
  }
  __syncthreads();

  // 2-4a. label the tile
  tile_engine(sm, h, w, slot, hook_log, s.err);

  // 4b. every site's root; global labels; root list
  constexpr int PER_T = TILE_SITES / LABEL_THREADS;
  uint32_t mine = 0;      // bit j: site threadIdx.x + j*LABEL_THREADS is a root
#pragma unroll 4
  for (int j = 0; j < PER_T; ++j) {
    const int sidx = threadIdx.x + j * LABEL_THREADS;
    const int ly = sidx >> TILE_W_LOG2, lx = sidx & (TILE_W - 1);
    if (ly < h && lx < w) {
      const int p = par[sidx];
      const int r = par[p];
      labels[(int64_t)(y0 + ly) * W + x0 + lx] = (y0 + (r >> TILE_W_LOG2)) * W + x0 + (r & (TILE_W - 1));
      if (r == sidx) mine |= 1u << j;
    }
  }
  int cnt = __popc(mine), incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) warp_roots[warp] = incl;
  __syncthreads();
  int base = 0, total = 0;
#pragma unroll
  for (int k = 0; k < LABEL_THREADS / 32; ++k) {
    const int c = warp_roots[k];
    base += (k < warp) ? c : 0;
    total += c;
  }
  base += incl - cnt;
  while (mine) {
    const int j = __ffs(mine) - 1;
    mine &= mine - 1;
    const int sidx = threadIdx.x + j * LABEL_THREADS;
    slot[base++] =
        (y0 + (sidx >> TILE_W_LOG2)) * W + x0 + (sidx & (TILE_W - 1));
  }

  // 5. seam record
  int32_t* rec = s.seams + (int64_t)t * SeamLayout::INTS;
  auto glabel = [&](int ly, int lx) -> int32_t {
    const int r = par[par[ly * TILE_W + lx]];
    return (y0 + (r >> TILE_W_LOG2)) * W + x0 + (r & (TILE_W - 1));
  };
  for (int k = threadIdx.x; k < TILE_H; k += LABEL_THREADS) {
    const bool ok = k < h;
    rec[SeamLayout::COL_L + k] = ok ? glabel(k, 0) : -1;
    rec[SeamLayout::COL_R + k] = ok ? glabel(k, w - 1) : -1;
    const bool e = ok && (site_bits(mask, (int64_t)(y0 + k) * W + x0 + w - 1) & 1u);
    const uint32_t eb = __ballot_sync(FULL, e);
    if (lane == 0) rec[SeamLayout::E_BITS + (k >> 5)] = (int32_t)eb;
  }
  for (int k = threadIdx.x; k < TILE_W; k += LABEL_THREADS) {
    const bool ok = k < w;
    rec[SeamLayout::ROW_B + k] = ok ? glabel(0, k) : -1;
    rec[SeamLayout::ROW_T + k] = ok ? glabel(h - 1, k) : -1;
    const bool n = ok && ((mb[(h - 1) * STRIPS + (k >> 5)] >> (2 * (k & 31) + 1)) & 1ull);
    const uint32_t nb = __ballot_sync(FULL, n);
    if (lane == 0) rec[SeamLayout::N_BITS + (k >> 5)] = (int32_t)nb;
  }
  if (threadIdx.x == 0) s.root_counts[t] = total;
}

cudaError_t launch_tile_label(const uint8_t* mask, int32_t* labels, const Grid& g,
                              const LabelScratch& s, cudaStream_t st) {
  k_tile_label<<<g.n_tiles(), LABEL_THREADS, 0, st>>>(mask, labels, g, s);
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
  const int t = blockIdx.x;
  const int n = s.root_counts[t];
  const int32_t* list = s.roots + (int64_t)t * TILE_SITES;
  uint64_t sweep = 0;
  if (spins) sweep = ctl->sweep;
  for (int k = threadIdx.x; k < n; k += ROOT_THREADS) {
    const int r = list[k];
    const int R = g_find(labels, r, limit, s.err);
    if (R != r) atomicMin(labels + r, R);
    if (spins && R == r) spins[r] = (int8_t)state_of(draw((uint32_t)r, sweep, TAG_FLIP, seed).x, q);
  }
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
