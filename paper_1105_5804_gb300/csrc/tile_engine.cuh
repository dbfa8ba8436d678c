// tile_engine.cuh -- the tile-local labeling engine shared by the
// stand-alone labeling kernel (bond mask in memory) and the fused
// Swendsen-Wang kernel (bonds drawn on the fly).
//
// Input: the tile's bond bits in shared memory, two 32-bit words per row and
// 32-column strip (be: bit i = east bond of site i of the strip; bn: bit i =
// its north bond), with bits of sites outside the grid and the east bond of
// the tile's last column cleared.  A row's words are the lane masks the sweep
// needs, so it reads them with one broadcast load each.  Output: par[] such
// that every site's tile root is par[par[site]], the root being the smallest
// local index of the site's tile component.
//
//  1. warp c sweeps strip c from row 0 upwards with the labels of the row
//     below in registers.  A row is cut into runs of east-joined sites by bit
//     operations on its east word.  A run reached from below (the north word
//     of the row below) takes the
//     label of its leftmost such site (one shuffle); a run nothing reaches
//     gets a fresh label, the index of its first site (a union-find node).
//     A lane reached from below by a label other than its run's appends the
//     pair to its warp's list: no union-find work happens inside the sweep;
//  2. warp c joins the east bonds from strip c into strip c + 1 (one row per
//     lane) and the pairs it listed, with the shared-memory union-find
//     (larger root hooked under the smaller); hooked roots are logged;
//  3. logged roots resolve their final roots, so every node points at its
//     root and every site's label (a node) is one step from it.
// The root is the smallest index of the tile component: the component's
// smallest site starts a run nothing reaches from below, so it is a node,
// and a smaller root never hooks under a larger one.
#pragma once
#include <climits>

#include "swccl_device.cuh"

namespace swccl {

constexpr int TILE_SITES = TILE_H * TILE_W;
constexpr int STRIPS = TILE_W / 32;
constexpr int PAIR_CAP = TILE_SITES / STRIPS;   // per warp: (TILE_H - 1) * 32 pairs at most
static_assert((TILE_H - 1) * 32 <= PAIR_CAP, "pair list capacity");
static_assert(LABEL_THREADS == TILE_W, "one warp per 32-column strip");
constexpr unsigned FULL = 0xFFFFFFFFu;

struct TileSmem {
  alignas(16) int par[TILE_SITES];   // 16-byte aligned: read as int4 when the tile roots are written
  uint32_t be[TILE_H * STRIPS];   // east bonds, bit = lane of the strip
  uint32_t bn[TILE_H * STRIPS];   // north bonds
  int warp_roots[LABEL_THREADS / 32];
  int n_hooked;
};

// Global index of local index r of the tile at (y0, x0) of a W-wide grid.
__device__ __forceinline__ int tile_global(int r, int y0, int x0, int W) {
  return (y0 + (r >> TILE_W_LOG2)) * W + x0 + (r & (TILE_W - 1));
}

// Runs the engine; sm.be and sm.bn must be filled and sm.n_hooked zero, followed by a
// __syncthreads().  `slot` (TILE_SITES ints of global scratch) holds the
// pair lists; `hook_log` (TILE_SITES ints) the hooked roots.  Ends with a
// __syncthreads().
__device__ __forceinline__ void tile_engine(TileSmem& sm, int h, int w, int32_t* slot, int32_t* hook_log,
                                            int* err) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* par = sm.par;
  const uint32_t* be = sm.be;
  const uint32_t* bn = sm.bn;
  // 1. strip sweep
  int n_pairs = 0;
  {
    const int col = warp * 32 + lane;
    const unsigned below_lanes = (1u << lane) - 1u;
    int32_t* pairs = slot + warp * PAIR_CAP;
    int lab_below = 0;
    uint32_t upb = 0u;          // north bonds of the row below: the lanes reached from below
    for (int ly = 0; ly < h; ++ly) {
      // bit i of `ends`: lane i ends a run (no east bond to lane i + 1; bit 31
      // always, runs stay inside the strip)
      const uint32_t ends = ~be[ly * STRIPS + warp] | 0x80000000u;
      const uint32_t nrow = bn[ly * STRIPS + warp];
      const bool up_open = (upb >> lane) & 1u;   // north bond from the site below into this lane's site
      const int start = 32 - __clz(ends & below_lanes);   // first lane of my run (clz(0) = 32)
      // my run's lanes relative to start: up to the lowest set bit of tail
      const uint32_t tail = ends >> start;
      const uint32_t reach = (upb >> start) & (tail ^ (tail - 1u));   // its lanes reached from below
      const int first = reach ? start + __ffs(reach) - 1 : lane;
      const int from_below = __shfl_sync(FULL, lab_below, first);
      const int label = reach ? from_below : ly * TILE_W + warp * 32 + start;
      par[ly * TILE_W + col] = label;
      const int lab_left = __shfl_up_sync(FULL, lab_below, 1);
      const bool dup = lane > start && ((upb >> (lane - 1)) & 1u) && lab_left == lab_below;
      const bool pair = up_open && lab_below != label && !dup;
      const uint32_t pm = __ballot_sync(FULL, pair);
      if (pair) pairs[n_pairs + __popc(pm & below_lanes)] = (lab_below << 16) | label;
      n_pairs += __popc(pm);
      lab_below = label;
      upb = nrow;
    }
  }
  __syncthreads();

  // 2. joins: warp c joins the east bonds from strip c into strip c + 1 (one
  //    row per lane), then the pairs it listed
  {
    if (warp < STRIPS - 1 && lane < h) {
      const int ly = lane, c = warp;
      bool join = (be[ly * STRIPS + c] >> 31) & 1u;
      if (join && ly > 0) {
        const int k0 = (ly - 1) * STRIPS + c;
        if (((be[k0] >> 31) & 1u) && ((bn[k0] >> 31) & 1u) && (bn[k0 + 1] & 1u)) join = false;   // joined below
      }
      if (join) {
        const int a = ly * TILE_W + c * 32 + 31;
        sm_union_log(par, a, a + 1, TILE_SITES, err, hook_log, &sm.n_hooked, TILE_SITES);
      }
    }
    const int32_t* pairs = slot + warp * PAIR_CAP;
    for (int j = lane; j < n_pairs; j += 32) {
      const int v = pairs[j];
      sm_union_log(par, v >> 16, v & 0xFFFF, TILE_SITES, err, hook_log, &sm.n_hooked, TILE_SITES);
    }
  }
  __syncthreads();

  // 3. hooked roots resolve their final roots (every other node is a root)
  {
    const int nh = min(sm.n_hooked, TILE_SITES);
    for (int k = threadIdx.x; k < nh; k += LABEL_THREADS) {
      const int x = hook_log[k];
      const int r = sm_find(par, x, TILE_SITES, err);
      atomicMin(&par[x], r);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Seam merge (Sec. II.C): bond k of tile t leaves the tile east (k < TILE_H,
// row k) or north (k >= TILE_H, column k - TILE_H), the periodic wrap
// included.  If it is open, the two tile roots on its ends are joined on the
// global array `gpar` (atomicMin hooking, larger root under the smaller).  A
// lane whose root pair equals its left neighbour's skips the union, so runs
// of seam bonds of one cluster cost one union.  All 32 lanes of a warp must
// call together (active == false for lanes past the end); MERGE_PER_TILE is
// a multiple of 32, so a warp never spans two tiles.  Seam records are read
// through L2 (ld.cg): in a persistent kernel they were written by other SMs.
constexpr int MERGE_PER_TILE = TILE_H + TILE_W;
static_assert(MERGE_PER_TILE % 32 == 0, "warps must not straddle tiles");

__device__ __forceinline__ void merge_seam_bond(int32_t* gpar, const Grid& g, const LabelScratch& s, int t, int k,
                                                bool active, int limit) {
  int a = -1, b = -1;
  bool valid = false;
  if (active) {
    const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
    const int32_t* rec = s.seams + (int64_t)t * SeamLayout::INTS;
    if (k < TILE_H) {
      const bool has_east = g.periodic || tx + 1 < g.tiles_x;
      const uint32_t ebits = (uint32_t)__ldcg(rec + SeamLayout::E_BITS + (k >> 5));
      if (has_east && ((ebits >> (k & 31)) & 1u)) {
        const int te = ty * g.tiles_x + (tx + 1 == g.tiles_x ? 0 : tx + 1);
        a = __ldcg(rec + SeamLayout::COL_R + k);
        b = __ldcg(s.seams + (int64_t)te * SeamLayout::INTS + SeamLayout::COL_L + k);
        valid = true;
      }
    } else {
      const int lx = k - TILE_H;
      const bool has_north = g.periodic || ty + 1 < g.tiles_y;
      const uint32_t nbits = (uint32_t)__ldcg(rec + SeamLayout::N_BITS + (lx >> 5));
      if (has_north && ((nbits >> (lx & 31)) & 1u)) {
        const int tn = (ty + 1 == g.tiles_y ? 0 : ty + 1) * g.tiles_x + tx;
        a = __ldcg(rec + SeamLayout::ROW_T + lx);
        b = __ldcg(s.seams + (int64_t)tn * SeamLayout::INTS + SeamLayout::ROW_B + lx);
        valid = true;
      }
    }
  }
  valid = valid && a != b;
  const unsigned long long key =
      valid ? ((unsigned long long)(unsigned)min(a, b) << 32) | (unsigned)max(a, b) : ~0ull;
  const unsigned long long prev = __shfl_up_sync(FULL, key, 1);
  const bool leader = (threadIdx.x & 31) == 0 || prev != key;
  if (valid && leader) g_union(gpar, a, b, limit, s.err);
}

}  // namespace swccl
