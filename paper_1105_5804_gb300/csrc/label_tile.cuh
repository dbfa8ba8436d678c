// label_tile.cuh -- per-tile bodies of the stand-alone labeling path, shared
// by the single-grid kernels (k_label.cu) and the batched kernels over many
// grids (k_ccl_batch.cu): local labeling of a tile from the packed mask, root
// compression of a tile's root list, and the site pass that makes a tile's
// labels canonical.
#pragma once
#include "tile_engine.cuh"

namespace swccl {

// The even bits of a 64-bit word, packed into 32 bits (bit 2i -> bit i).
__device__ __forceinline__ uint32_t even_bits(unsigned long long x) {
  x &= 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
  x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
  x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
  return (uint32_t)x;
}

// Local labeling of one tile for the stand-alone labeling path: the tile's
// bond bits are copied from the packed mask into shared memory (bits of
// sites outside the grid and the east bond of the tile's last column
// cleared), the engine of tile_engine.cuh labels the tile, and the kernel
// writes every site's label (global index of its tile root, the minimum
// site index of its tile component), the tile's root list, and the seam
// record (labels and outgoing bond bits of the four tile edges).
// LOCAL (the stand-alone labeling path, finished by final_labels_tile): the
// label array receives only the parent entries of the tile roots whose
// component reaches the tile edge (label = own global index), which the
// seam merge and the final root walks use; every site's tile root goes, as
// a 16-bit local index, to the tile's hook-log slot (free once the engine
// has ended), in tile row-major order; the root list holds local indices,
// with CCL_EDGE_ROOT set on the edge roots.  final_labels_tile writes every
// site's label.
constexpr int CCL_EDGE_ROOT = 1 << 30;
template <bool LOCAL = false>
__device__ __forceinline__ void ccl_label_tile(const uint8_t* __restrict__ mask, int32_t* __restrict__ labels,
                                               const Grid& g, const LabelScratch& s, int t, TileSmem& sm) {
  int* par = sm.par;
  int* warp_roots = sm.warp_roots;

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
    sm.be[k] = even_bits(wd);        // the mask interleaves east (even) and north (odd) bits
    sm.bn[k] = even_bits(wd >> 1);
  }
  __syncthreads();

  // 2-4a. label the tile
  tile_engine(sm, h, slot, hook_log, s.err);

  // LOCAL: mark the tile roots whose component reaches the tile edge (only
  // they can belong to clusters that continue in other tiles); the marks go
  // to the shared words the engine no longer needs
  uint32_t* edge = reinterpret_cast<uint32_t*>(sm.pairs);
  if (LOCAL) {
    static_assert(TILE_SITES / 32 <= STRIPS * PAIR_FAST, "edge marks fit");
    for (int k = threadIdx.x; k < TILE_SITES / 32; k += LABEL_THREADS) edge[k] = 0u;
    __syncthreads();
    auto mark = [&](int ly, int lx) {
      const int r = par[par[ly * TILE_W + lx]];
      atomicOr(&edge[r >> 5], 1u << (r & 31));
    };
    for (int k = threadIdx.x; k < h; k += LABEL_THREADS) {
      mark(k, 0);
      mark(k, w - 1);
    }
    for (int k = threadIdx.x; k < w; k += LABEL_THREADS) {
      mark(0, k);
      mark(h - 1, k);
    }
    __syncthreads();
  }

  // 4b. every site's root; root list.  LOCAL: the roots as 16-bit local
  //     indices into the tile's hook-log slot (free since the engine ended),
  //     four consecutive sites per thread and step (lane-consecutive words of
  //     par); mine bit j: site 4 (threadIdx.x + (j / 4) LABEL_THREADS) + j % 4.
  //     Otherwise global labels; mine bit j: site threadIdx.x + j LABEL_THREADS.
  constexpr int PER_T = TILE_SITES / LABEL_THREADS;
  uint32_t mine = 0;
  if (LOCAL) {
    uint16_t* lr = reinterpret_cast<uint16_t*>(hook_log);
#pragma unroll 2
    for (int j = 0; j < PER_T / 4; ++j) {
      const int sidx = 4 * ((int)threadIdx.x + j * LABEL_THREADS);
      const int ly = sidx >> TILE_W_LOG2, lx = sidx & (TILE_W - 1);
      if (ly >= h) continue;   // rows past the grid: the engine wrote no entries there
      const int4 pv = *reinterpret_cast<const int4*>(&par[sidx]);
      const int r0 = par[pv.x], r1 = par[pv.y], r2 = par[pv.z], r3 = par[pv.w];
      *reinterpret_cast<uint2*>(lr + sidx) =
          make_uint2((uint32_t)r0 | ((uint32_t)r1 << 16), (uint32_t)r2 | ((uint32_t)r3 << 16));
      // columns past the grid (bondless, each its own root) are no roots of the tile
      const uint32_t in = lx + 4 <= w ? 0xFu : (lx < w ? (1u << (w - lx)) - 1u : 0u);
      const uint32_t is_root = (uint32_t)(r0 == sidx) | ((uint32_t)(r1 == sidx + 1) << 1) |
                               ((uint32_t)(r2 == sidx + 2) << 2) | ((uint32_t)(r3 == sidx + 3) << 3);
      mine |= (is_root & in) << (4 * j);
    }
  } else {
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
    if (LOCAL) {
      // an edge root's label entry is its parent entry for the seam merge
      const int sidx = 4 * ((int)threadIdx.x + (j >> 2) * LABEL_THREADS) + (j & 3);
      const bool on_edge = (edge[sidx >> 5] >> (sidx & 31)) & 1u;
      if (on_edge) {
        const int32_t gr = (y0 + (sidx >> TILE_W_LOG2)) * W + x0 + (sidx & (TILE_W - 1));
        labels[gr] = gr;
      }
      slot[base++] = sidx | (on_edge ? CCL_EDGE_ROOT : 0);
    } else {
      const int sidx = threadIdx.x + j * LABEL_THREADS;
      slot[base++] = (y0 + (sidx >> TILE_W_LOG2)) * W + x0 + (sidx & (TILE_W - 1));
    }
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
    const bool n = ok && ((sm.bn[(h - 1) * STRIPS + (k >> 5)] >> (k & 31)) & 1u);
    const uint32_t nb = __ballot_sync(FULL, n);
    if (lane == 0) rec[SeamLayout::N_BITS + (k >> 5)] = (int32_t)nb;
  }
  if (threadIdx.x == 0) s.root_counts[t] = total;
  __syncthreads();
}

// Tile t's roots: label = final root; in a Swendsen-Wang sweep (spins set)
// final roots also draw their cluster's new state.  All threads call it.
__device__ __forceinline__ void root_compress_tile(int32_t* __restrict__ labels, const LabelScratch& s, int t,
                                                   int8_t* __restrict__ spins, int q, uint64_t seed, uint64_t sweep,
                                                   int limit) {
  const int n = __ldcg(s.root_counts + t);
  const int32_t* list = s.roots + (int64_t)t * TILE_SITES;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int r = __ldcg(list + k);
    const int R = g_find(labels, r, limit, s.err);
    if (R != r) atomicMin(labels + r, R);
    if (spins && R == r) spins[r] = (int8_t)state_of(draw((uint32_t)r, sweep, TAG_FLIP, seed).x, q);
  }
}

// Site pass of tile t: every label of the tile points at a tile root whose
// entry holds the final root after root compression; one jump makes the
// label canonical.
__device__ __forceinline__ void site_compress_tile(int32_t* __restrict__ labels, const Grid& g, int t) {
  const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
  const int y0 = ty * TILE_H, x0 = tx * TILE_W;
  const int h = min(TILE_H, g.H - y0), w = min(TILE_W, g.W - x0);
  for (int k = threadIdx.x; k < TILE_SITES; k += blockDim.x) {
    const int ly = k >> TILE_W_LOG2, lx = k & (TILE_W - 1);
    if (ly < h && lx < w) {
      int32_t* p = labels + (int64_t)(y0 + ly) * g.W + x0 + lx;
      const int r = __ldcg(p);
      const int R = __ldcg(labels + r);
      if (R != r) *p = R;
    }
  }
}

// Final labels of tile t for the stand-alone path (after the seam merge, on
// what ccl_label_tile<true> wrote): each tile root (local root list) finds
// its cluster root R on the label array and stores it in `table` at its
// local index; then every site of the tile takes table[its tile root].
// A tile root's entry receives R (smaller than any value other walks may
// store there), so walks of other tiles through it stay valid.  All threads
// of the CTA call it; it synchronises the CTA.
__device__ __forceinline__ void final_labels_tile(int32_t* labels, const Grid& g, const LabelScratch& s, int t,
                                                  int32_t* table /* shared, TILE_SITES */, int limit) {
  const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
  const int y0 = ty * TILE_H, x0 = tx * TILE_W;
  const int h = min(TILE_H, g.H - y0), w = min(TILE_W, g.W - x0);
  const int n = __ldcg(s.root_counts + t);
  const int32_t* list = s.roots + (int64_t)t * TILE_SITES;
  // 1. cluster roots of the tile roots: a root whose component stays inside
  //    the tile is its cluster's root; the others walk the label array, four
  //    walks of a thread in flight together
  constexpr int U = 4;
  for (int k0 = threadIdx.x; k0 < n; k0 += U * (int)blockDim.x) {
    int r[U], x[U];
    bool act[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * (int)blockDim.x;
      const int raw = k < n ? __ldcg(list + k) : 0;
      r[u] = raw & ~CCL_EDGE_ROOT;   // local index
      act[u] = k < n && (raw & CCL_EDGE_ROOT);
      x[u] = tile_global(r[u], y0, x0, g.W);
    }
    g_find_multi<U>(labels, x, act, limit, s.err);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u * (int)blockDim.x < n) table[r[u]] = x[u];
  }
  __syncthreads();
  // 2. every site takes its tile root's cluster root; the tile roots are the
  //    16-bit local indices ccl_label_tile<true> left in the tile's hook-log
  //    slot, eight sites per 16-byte word, in tile row-major order; labels go
  //    out four sites per 16-byte store when rows start 16-byte aligned (a
  //    16-byte aligned array and W % 4 == 0; x0 is a multiple of TILE_W, so w
  //    is a multiple of 4 too)
  const uint16_t* lr = reinterpret_cast<const uint16_t*>(s.work + (int64_t)t * TILE_SITES);
  if ((g.W & 3) == 0 && (reinterpret_cast<uintptr_t>(labels) & 15) == 0) {
    for (int k = threadIdx.x; k < TILE_SITES / 8; k += blockDim.x) {
      const int sidx = 8 * k;
      const int ly = sidx >> TILE_W_LOG2, lx = sidx & (TILE_W - 1);
      if (ly >= h || lx >= w) continue;
      const uint4 v = __ldcg(reinterpret_cast<const uint4*>(lr + sidx));
      int32_t* p = labels + (int64_t)(y0 + ly) * g.W + x0 + lx;
      *reinterpret_cast<int4*>(p) =
          make_int4(table[v.x & 0xFFFFu], table[v.x >> 16], table[v.y & 0xFFFFu], table[v.y >> 16]);
      if (lx + 8 <= w)
        *reinterpret_cast<int4*>(p + 4) =
            make_int4(table[v.z & 0xFFFFu], table[v.z >> 16], table[v.w & 0xFFFFu], table[v.w >> 16]);
    }
  } else {
    for (int k = threadIdx.x; k < TILE_SITES; k += blockDim.x) {
      const int ly = k >> TILE_W_LOG2, lx = k & (TILE_W - 1);
      if (ly < h && lx < w) labels[(int64_t)(y0 + ly) * g.W + x0 + lx] = table[__ldcg(lr + k)];
    }
  }
  __syncthreads();
}

}  // namespace swccl
