// tile_engine.cuh -- the tile-local labeling engine shared by the
// stand-alone labeling kernel (bond mask in memory), the fused
// Swendsen-Wang kernel (bonds drawn on the fly) and the simple-cubic kernel.
//
// Input: the tile's bond bits as 32-bit words, one per row and 32-column
// strip (be: bit i = east bond of site i of the strip; bn: bit i = its north
// bond), with bits of sites outside the grid and the east bond of the tile's
// last column cleared.  Thread (lane, warp) holds the words of row `lane` of
// strip `warp`.  Output: par[] such that every site's tile root is
// par[par[site]], the root being the smallest local index of the site's tile
// component.
//
// A row word is cut into runs of east-joined sites.  Every run is labelled by
// a union-find node: a run that no north bond from the row below reaches
// starts a fresh node (the local index of its first site); a run that is
// reached takes the label of the site below its first contact.  Runs reached
// from several runs below are joined afterwards.
//  1. per row word (lane = row), bit-parallel: the run starts S, the first
//     contact F of every reached run (the lowest north bond from below inside
//     the run), the starts U of unreached runs, and the extra contacts X: for
//     each run of the row below that the run touches, the lowest contact in
//     their overlap, other than F.  Overlaps are the segments of sites joined
//     east in both rows, so one contact per overlap keeps exactly one per
//     pair of runs.
//  2. warp c sweeps strip c from row 0 upwards, one site per lane, with the
//     labels of the row below in registers.  A lane finds its run's start
//     (the highest bit of S at or below it) and its run's anchor (the lowest
//     bit of F | U from the start on: the first contact, or the start of an
//     unreached run); the anchor lane's candidate -- the label below it if it
//     is a first contact, else its own index -- is the run's label (one
//     shuffle).  No union-find work happens in the sweep.
//  3. the extra contacts whose two labels differ, and the east bonds from
//     strip c into strip c + 1, are listed per warp and joined with the
//     shared-memory union-find (larger root hooked under the smaller);
//     hooked roots are logged;
//  4. logged roots resolve their final roots, so every node points at its
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
static_assert(LABEL_THREADS == TILE_W, "one warp per 32-column strip");
static_assert(TILE_H == 32, "one lane per row of a strip");
constexpr unsigned FULL = 0xFFFFFFFFu;
// Per warp at most 32 pairs per row word: a run's first contact is no extra
// contact, so a row word of r runs has at most 32 - r <= 31, plus the
// strip join.
constexpr int PAIR_CAP = TILE_SITES / STRIPS;
// Lists kept in shared memory up to these lengths, the rest in global scratch.
constexpr int PAIR_FAST = 4 * TILE_H;           // per warp (the space of the sweep inputs)
constexpr int HOOK_FAST = 512;

struct TileSmem {
  alignas(16) int par[TILE_SITES];   // 16-byte aligned: read as int4 when the tile roots are written
  uint32_t be[TILE_H * STRIPS];   // east bonds, bit = lane of the strip
  uint32_t bn[TILE_H * STRIPS];   // north bonds
  union {
    alignas(16) uint4 rowinfo[STRIPS * TILE_H];   // per row word, strip-major: S, F | U, F (sweep inputs)
    int pairs[STRIPS * PAIR_FAST];                // then: the warps' first contacts to join
  };
  int hooks[HOOK_FAST];                           // the first hooked roots
  int warp_roots[LABEL_THREADS / 32];
  int n_hooked;
};

// Global index of local index r of the tile at (y0, x0) of a W-wide grid.
__device__ __forceinline__ int tile_global(int r, int y0, int x0, int W) {
  return (y0 + (r >> TILE_W_LOG2)) * W + x0 + (r & (TILE_W - 1));
}

// Inclusive OR of the bits of x towards higher bits inside segments: bit i
// and bit i + 1 are in one segment iff bit i of j is set.
__device__ __forceinline__ uint32_t seg_or_up(uint32_t x, uint32_t j) {
  uint32_t m = j << 1;           // bit i: i - 1 and i joined
  x |= (x << 1) & m;
  m &= m << 1;                   // bit i: i - 2 .. i joined
  x |= (x << 2) & m;
  m &= m << 2;
  x |= (x << 4) & m;
  m &= m << 4;
  x |= (x << 8) & m;
  m &= m << 8;
  x |= (x << 16) & m;
  return x;
}

// The same towards lower bits.
__device__ __forceinline__ uint32_t seg_or_down(uint32_t x, uint32_t j) {
  uint32_t m = j;                // bit i: i and i + 1 joined
  x |= (x >> 1) & m;
  m &= m >> 1;
  x |= (x >> 2) & m;
  m &= m >> 2;
  x |= (x >> 4) & m;
  m &= m >> 4;
  x |= (x >> 8) & m;
  m &= m >> 8;
  x |= (x >> 16) & m;
  return x;
}

// Runs the engine.  we, wn: the calling thread's row word (row = lane, strip =
// warp), zero for rows >= h.  sm.be and sm.bn must hold every row word and
// sm.n_hooked must be zero, followed by a __syncthreads().  `pairs` and
// `hook_log` (TILE_SITES ints of global scratch each) hold what does not fit
// in shared memory of the warps' lists of contacts to join and of the hooked
// roots.  Ends with a __syncthreads().
__device__ __forceinline__ void tile_engine_regs(TileSmem& sm, uint32_t we, uint32_t wn, int h, int32_t* pairs,
                                                 int32_t* hook_log, int* err) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* par = sm.par;
  const int colbase = warp * 32;
  // 1. run structure of my row word against the row below
  uint32_t X;
  {
    const uint32_t e_below = __shfl_up_sync(FULL, we, 1);
    uint32_t c = __shfl_up_sync(FULL, wn, 1);   // contacts: north bonds of the row below into my row
    if (lane == 0 || lane >= h) c = 0u;
    const uint32_t S = ~(we << 1);               // run starts (bit 0 always)
    const uint32_t before = (seg_or_up(c, we) << 1) & (we << 1);     // a contact earlier in my run
    const uint32_t F = c & ~before;
    const uint32_t U = S & ~seg_or_down(c, we);                     // starts of runs without contact
    const uint32_t j2 = we & e_below;                               // joined east in both rows
    const uint32_t before2 = (seg_or_up(c, j2) << 1) & (j2 << 1);
    X = c & ~before2 & ~F;
    sm.rowinfo[warp * TILE_H + lane] = make_uint4(S, F | U, F, 0u);
  }
  __syncwarp();
  // 2. strip sweep (lane = column)
  {
    const uint32_t upto = (2u << lane) - 1u;     // bits 0..lane
    const uint32_t me = 1u << lane;
    int lab_below = 0;
#pragma unroll
    for (int ly = 0; ly < TILE_H; ++ly) {
      if (ly < h) {
        const uint4 ri = sm.rowinfo[warp * TILE_H + ly];
        const int start = 31 - __clz(ri.x & upto);
        const int anchor = start + __ffs(ri.y >> start) - 1;
        const int site = ly * TILE_W + colbase + lane;
        const int cand = (ri.z & me) ? lab_below : site;
        const int label = __shfl_sync(FULL, cand, anchor);
        par[site] = label;
        lab_below = label;
      }
    }
  }
  __syncthreads();

  // 3. joins.  The extra contacts of my row (lane = row) whose two labels
  //    differ (a contact whose runs already carry one label joins nothing
  //    new), and the east bond of my row from strip c into strip c + 1, are
  //    listed in the warp's part of `pairs`; then the warp joins its list 32
  //    pairs at a time.
  {
    const uint32_t* be = sm.be;
    const uint32_t* bn = sm.bn;
    const int row = lane * TILE_W + colbase;
    uint32_t D = 0u;
    for (uint32_t x = X; x; x &= x - 1) {
      const int b = __ffs(x) - 1;
      if (par[row + b] != par[row - TILE_W + b]) D |= 1u << b;
    }
    bool join = false;   // east bond into the next strip, unless joined below
    if (warp < STRIPS - 1 && lane < h) {
      const int ly = lane, c = warp;
      join = (be[ly * STRIPS + c] >> 31) & 1u;
      if (join && ly > 0) {
        const int k0 = (ly - 1) * STRIPS + c;
        if (((be[k0] >> 31) & 1u) && ((bn[k0] >> 31) & 1u) && (bn[k0 + 1] & 1u)) join = false;
      }
    }
    const int cnt = __popc(D) + (join ? 1 : 0);
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += v;
    }
    const int total = __shfl_sync(FULL, incl, 31);   // at most PAIR_CAP
    int* fast = sm.pairs + warp * PAIR_FAST;
    int32_t* slow = pairs + warp * PAIR_CAP;
    __syncwarp();                                 // the warp's sweep inputs are read
    int k = incl - cnt;
    for (; D; D &= D - 1, ++k) {
      const int b = __ffs(D) - 1;
      const int v = (par[row + b] << 16) | par[row - TILE_W + b];
      if (k < PAIR_FAST) fast[k] = v;
      else slow[k - PAIR_FAST] = v;
    }
    if (join) {
      const int a = row + 31;   // last column of strip c, row `lane`
      const int v = (par[a] << 16) | par[a + 1];
      if (k < PAIR_FAST) fast[k] = v;
      else slow[k - PAIR_FAST] = v;
    }
    __syncwarp();
    for (int j = lane; j < total; j += 32) {
      const int v = j < PAIR_FAST ? fast[j] : slow[j - PAIR_FAST];
      sm_union_log(par, v >> 16, v & 0xFFFF, TILE_SITES, err, sm.hooks, HOOK_FAST, hook_log, &sm.n_hooked,
                   TILE_SITES);
    }
  }
  __syncthreads();

  // 4. hooked roots resolve their final roots (every other node is a root)
  {
    const int nh = min(sm.n_hooked, TILE_SITES + HOOK_FAST);
    for (int k = threadIdx.x; k < nh; k += LABEL_THREADS) {
      const int x = k < HOOK_FAST ? sm.hooks[k] : hook_log[k - HOOK_FAST];
      const int r = sm_find(par, x, TILE_SITES, err);
      atomicMin(&par[x], r);
    }
  }
  __syncthreads();
}

// The engine with the row words read from sm.be / sm.bn (rows < h filled,
// and sm.n_hooked zero, before a __syncthreads()).
__device__ __forceinline__ void tile_engine(TileSmem& sm, int h, int32_t* pairs, int32_t* hook_log, int* err) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool in = lane < h;
  tile_engine_regs(sm, in ? sm.be[lane * STRIPS + warp] : 0u, in ? sm.bn[lane * STRIPS + warp] : 0u, h, pairs,
                   hook_log, err);
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
    // the bond's bit and the roots at both ends are loaded together (the
    // neighbour index wraps, so the loads stay inside the records even
    // where the bond does not exist), then the bit decides
    const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
    const int32_t* rec = s.seams + (int64_t)t * SeamLayout::INTS;
    bool has;
    int tn, i_bits, i_a, i_b, bit;
    if (k < TILE_H) {
      has = g.periodic || tx + 1 < g.tiles_x;
      tn = ty * g.tiles_x + (tx + 1 == g.tiles_x ? 0 : tx + 1);
      i_bits = SeamLayout::E_BITS + (k >> 5);
      i_a = SeamLayout::COL_R + k;
      i_b = SeamLayout::COL_L + k;
      bit = k & 31;
    } else {
      const int lx = k - TILE_H;
      has = g.periodic || ty + 1 < g.tiles_y;
      tn = (ty + 1 == g.tiles_y ? 0 : ty + 1) * g.tiles_x + tx;
      i_bits = SeamLayout::N_BITS + (lx >> 5);
      i_a = SeamLayout::ROW_T + lx;
      i_b = SeamLayout::ROW_B + lx;
      bit = lx & 31;
    }
    const uint32_t bits = (uint32_t)__ldcg(rec + i_bits);
    const int ra = __ldcg(rec + i_a);
    const int rb = __ldcg(s.seams + (int64_t)tn * SeamLayout::INTS + i_b);
    if (has && ((bits >> bit) & 1u)) {
      a = ra;
      b = rb;
      valid = true;
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
