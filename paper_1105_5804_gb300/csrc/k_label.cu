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
//                 global label array with atomicMin hooking.  Lanes that
//                 carry the same root pair are collapsed with a warp match,
//                 so consecutive seam bonds of one cluster cost one union.
//  k_root_compress  for every tile root: label = final root (pointer
//                 jumping).  Because hooks always go to the smaller index,
//                 the final root is the cluster's minimum site index.  In a
//                 Swendsen-Wang sweep the final roots also draw their
//                 cluster's new state here (Sec. II.D), keyed by the root.
//  k_site_compress  label[i] = label[label[i]] for every site (stand-alone
//                 labeling only: leaves every label canonical).
#include <climits>

#include "swccl_device.cuh"

namespace swccl {

namespace {
constexpr int TILE_SITES = TILE_H * TILE_W;
constexpr unsigned FULL = 0xFFFFFFFFu;
}  // namespace

// Shared-memory bond bits per tile site: bit 0 east bond inside the tile,
// bit 1 north bond inside the tile, bits 2..3 the raw mask bits.
__device__ __forceinline__ uint32_t tile_bits(uint32_t m, int lx, int ly, int w, int h) {
  uint32_t b = m << 2;
  if ((m & 1u) && lx + 1 < w) b |= 1u;
  if ((m & 2u) && ly + 1 < h) b |= 2u;
  return b;
}

// Local labeling of one tile.
//  1. the tile's bond bits go to shared memory;
//  2. warp c sweeps its 32-column strip from row 0 upwards.  The labels of
//     the row below stay in registers.  A row is cut into runs of
//     east-joined sites with one ballot; each run takes the smallest label
//     among the sites below it that reach it by a north bond (a segmented
//     minimum over the run's lanes, five shuffle steps), or, if none does, a
//     fresh label: the index of its first site.  Only a run reached from
//     below by two different labels joins them, with the shared-memory
//     union-find; every other site is labeled without an atomic.
//  3. east bonds between strips are joined with the union-find, skipping a
//     bond whose two ends were already joined through the row below;
//  4. every site resolves its root; the root is the smallest index of the
//     tile component (a fresh label is always a run's first site, the
//     component's smallest site starts a run nothing reaches from below, and
//     unions hook the larger root under the smaller), so its global index is
//     the minimum site index of the tile component.
__global__ void __launch_bounds__(LABEL_THREADS)
k_tile_label(const uint8_t* __restrict__ mask, int32_t* __restrict__ labels, Grid g,
             LabelScratch s) {
  __shared__ int par[TILE_SITES];
  __shared__ __align__(16) uint8_t bits[TILE_SITES];
  __shared__ int n_roots;

  const int t = blockIdx.x;
  const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
  const int y0 = ty * TILE_H, x0 = tx * TILE_W;
  const int h = min(TILE_H, g.H - y0), w = min(TILE_W, g.W - x0);
  const int W = g.W;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) n_roots = 0;

  // 1. bond bits of the tile
  if ((W & 3) == 0) {
    // rows start on mask-byte boundaries: one byte = four sites per thread
    constexpr int BPR = TILE_W / 4;
    for (int k = threadIdx.x; k < BPR * TILE_H; k += LABEL_THREADS) {
      const int ly = k / BPR, lx0 = (k - ly * BPR) * 4;
      uint32_t m4 = 0;
      if (ly < h && lx0 < w) m4 = mask[((int64_t)(y0 + ly) * W + x0 + lx0) >> 2];
      uint32_t out = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int lx = lx0 + j;
        if (ly < h && lx < w) out |= tile_bits((m4 >> (2 * j)) & 3u, lx, ly, w, h) << (8 * j);
      }
      *reinterpret_cast<uint32_t*>(bits + ly * TILE_W + lx0) = out;
    }
  } else {
    for (int sidx = threadIdx.x; sidx < TILE_SITES; sidx += LABEL_THREADS) {
      const int ly = sidx >> TILE_W_LOG2, lx = sidx & (TILE_W - 1);
      uint32_t b = 0;
      if (ly < h && lx < w) b = tile_bits(site_bits(mask, (int64_t)(y0 + ly) * W + x0 + lx), lx, ly, w, h);
      bits[sidx] = (uint8_t)b;
    }
  }
  __syncthreads();

  // 2. strip sweep
  {
    const int col = warp * 32 + lane;
    const unsigned below_lanes = (1u << lane) - 1u;
    int lab_below = 0;
    bool up_open = false;       // north bond from the site below into this lane's site
    for (int ly = 0; ly < h; ++ly) {
      const int sidx = ly * TILE_W + col;
      const uint32_t b = bits[sidx];
      const uint32_t east = __ballot_sync(FULL, b & 1u) & 0x7FFFFFFFu;   // runs stay inside the strip
      const uint32_t breaks = ~east & below_lanes;
      const int start = breaks ? 32 - __clz(breaks) : 0;
      const int end = lane + __ffs(~east >> lane) - 1;
      const int up = up_open ? lab_below : INT_MAX;
      int m = up;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(FULL, m, d);
        if (lane - d >= start) m = min(m, v);
      }
      const int mrun = __shfl_sync(FULL, m, end);
      const int label = (mrun == INT_MAX) ? ly * TILE_W + warp * 32 + start : mrun;
      par[sidx] = label;
      __syncwarp();
      const int up_left = __shfl_up_sync(FULL, up, 1);
      if (up != INT_MAX && up != label && !(lane > start && up_left == up))
        sm_union(par, up, label, TILE_SITES, s.err);
      __syncwarp();
      lab_below = label;
      up_open = (b & 2u) != 0;
    }
  }
  __syncthreads();

  // 3. east bonds between strips
  constexpr int STRIPS = TILE_W / 32;
  for (int k = threadIdx.x; k < TILE_H * (STRIPS - 1); k += LABEL_THREADS) {
    const int ly = k / (STRIPS - 1), c = k - ly * (STRIPS - 1);
    if (ly >= h) continue;
    const int a = ly * TILE_W + c * 32 + 31;
    if (!(bits[a] & 1u)) continue;
    if (ly > 0) {
      const int a0 = a - TILE_W;
      if ((bits[a0] & 1u) && (bits[a0] & 2u) && (bits[a0 + 1] & 2u)) continue;   // joined below
    }
    sm_union(par, a, a + 1, TILE_SITES, s.err);
  }
  __syncthreads();

  // 4. final tile roots -> global labels; collect roots
  const int64_t tile_base = (int64_t)t * TILE_SITES;
  for (int sidx = threadIdx.x; sidx < TILE_SITES; sidx += LABEL_THREADS) {
    const int ly = sidx >> TILE_W_LOG2, lx = sidx & (TILE_W - 1);
    const bool inside = ly < h && lx < w;
    int r = sidx, gr = 0;
    if (inside) {
      r = sm_find(par, sidx, TILE_SITES, s.err);
      atomicMin(&par[sidx], r);
      gr = (y0 + (r >> TILE_W_LOG2)) * W + x0 + (r & (TILE_W - 1));
      labels[(int64_t)(y0 + ly) * W + x0 + lx] = gr;
    }
    const bool is_root = inside && r == sidx;
    const uint32_t rb = __ballot_sync(FULL, is_root);
    int base = 0;
    if (lane == 0 && rb) base = atomicAdd(&n_roots, __popc(rb));
    base = __shfl_sync(FULL, base, 0);
    if (is_root) s.roots[tile_base + base + __popc(rb & ((1u << lane) - 1u))] = gr;
  }
  __syncthreads();

  // 5. seam record
  int32_t* rec = s.seams + (int64_t)t * SeamLayout::INTS;
  auto glabel = [&](int ly, int lx) -> int32_t {
    const int r = par[ly * TILE_W + lx];
    return (y0 + (r >> TILE_W_LOG2)) * W + x0 + (r & (TILE_W - 1));
  };
  for (int k = threadIdx.x; k < TILE_H; k += LABEL_THREADS) {
    const bool ok = k < h;
    rec[SeamLayout::COL_L + k] = ok ? glabel(k, 0) : -1;
    rec[SeamLayout::COL_R + k] = ok ? glabel(k, w - 1) : -1;
    const uint32_t eb = __ballot_sync(FULL, ok && (bits[k * TILE_W + w - 1] & 4u));
    if (lane == 0) rec[SeamLayout::E_BITS + (k >> 5)] = (int32_t)eb;
  }
  for (int k = threadIdx.x; k < TILE_W; k += LABEL_THREADS) {
    const bool ok = k < w;
    rec[SeamLayout::ROW_B + k] = ok ? glabel(0, k) : -1;
    rec[SeamLayout::ROW_T + k] = ok ? glabel(h - 1, k) : -1;
    const uint32_t nb = __ballot_sync(FULL, ok && (bits[(h - 1) * TILE_W + k] & 8u));
    if (lane == 0) rec[SeamLayout::N_BITS + (k >> 5)] = (int32_t)nb;
  }
  if (threadIdx.x == 0) s.root_counts[t] = n_roots;
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
constexpr int MERGE_PER_TILE = TILE_H + TILE_W;
constexpr int MERGE_THREADS = 256;

__global__ void __launch_bounds__(MERGE_THREADS)
k_merge(int32_t* __restrict__ labels, Grid g, LabelScratch s, int limit) {
  const int64_t gid = blockIdx.x * (int64_t)MERGE_THREADS + threadIdx.x;
  const int64_t total = (int64_t)g.n_tiles() * MERGE_PER_TILE;
  if (gid - (threadIdx.x & 31) >= total) return;   // whole warp past the end
  int a = -1, b = -1;
  bool valid = false;
  if (gid < total) {
    const int t = (int)(gid / MERGE_PER_TILE);
    const int k = (int)(gid - (int64_t)t * MERGE_PER_TILE);
    const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
    const int32_t* rec = s.seams + (int64_t)t * SeamLayout::INTS;
    if (k < TILE_H) {
      const bool has_east = g.periodic || tx + 1 < g.tiles_x;
      const uint32_t ebits = (uint32_t)rec[SeamLayout::E_BITS + (k >> 5)];
      if (has_east && ((ebits >> (k & 31)) & 1u)) {
        const int te = ty * g.tiles_x + (tx + 1 == g.tiles_x ? 0 : tx + 1);
        a = rec[SeamLayout::COL_R + k];
        b = s.seams[(int64_t)te * SeamLayout::INTS + SeamLayout::COL_L + k];
        valid = true;
      }
    } else {
      const int lx = k - TILE_H;
      const bool has_north = g.periodic || ty + 1 < g.tiles_y;
      const uint32_t nbits = (uint32_t)rec[SeamLayout::N_BITS + (lx >> 5)];
      if (has_north && ((nbits >> (lx & 31)) & 1u)) {
        const int tn = (ty + 1 == g.tiles_y ? 0 : ty + 1) * g.tiles_x + tx;
        a = rec[SeamLayout::ROW_T + lx];
        b = s.seams[(int64_t)tn * SeamLayout::INTS + SeamLayout::ROW_B + lx];
        valid = true;
      }
    }
  }
  valid = valid && a != b;
  const unsigned long long key =
      valid ? ((unsigned long long)(unsigned)min(a, b) << 32) | (unsigned)max(a, b) : ~0ull;
  const unsigned same = __match_any_sync(FULL, key);
  const bool leader = (__ffs(same) - 1) == (int)(threadIdx.x & 31);
  if (valid && leader) g_union(labels, a, b, limit, s.err);
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
  return al(nt * TILE_SITES * 4) + al(nt * 4) + al(nt * SeamLayout::INTS * 4) + al(4);
}

LabelScratch carve_label_scratch(const Grid& g, void* base, int* err) {
  auto al = [](int64_t b) { return (b + 255) & ~(int64_t)255; };
  const int64_t nt = g.n_tiles();
  char* p = static_cast<char*>(base);
  LabelScratch s;
  s.roots = reinterpret_cast<int32_t*>(p);
  p += al(nt * TILE_SITES * 4);
  s.root_counts = reinterpret_cast<int32_t*>(p);
  p += al(nt * 4);
  s.seams = reinterpret_cast<int32_t*>(p);
  p += al(nt * SeamLayout::INTS * 4);
  s.err = err ? err : reinterpret_cast<int*>(p);
  return s;
}

}  // namespace swccl
