// fused_tile.cuh -- per-tile bodies of the fused Swendsen-Wang sweep, shared
// by the single-lattice kernels (k_fused.cu) and the batched / persistent
// kernels over many lattices (k_batch.cu).  Description of the steps in
// k_fused.cu.
#pragma once
#include "tile_engine.cuh"

namespace swccl {

namespace fused {

// Four byte lanes of a and b compared: bit k of the result is set iff byte k
// of a equals byte k of b.  Exact zero-byte test of a ^ b (no carry crosses a
// byte: each byte of (x & 0x7F..) + 0x7F.. is at most 0xFE), then the four
// flag bits are gathered by one multiply.
__device__ __forceinline__ uint32_t eq4(uint32_t a, uint32_t b) {
  const uint32_t x = a ^ b;
  const uint32_t y = ((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x;   // bit 7 of a byte set iff the byte is non-zero
  const uint32_t z = (~y & 0x80808080u) >> 7;                  // bit 0 of a byte set iff equal
  return (z * 0x00204081u) >> 21 & 0xFu;
}

// Bonds of 32 consecutive sites of one row, and the observables of the
// spins read (bonds joining equal spins; sites per state for q <= QREG).
struct RowBonds {
  uint32_t east, north;     // bit i: east / north bond of site i (rule of Eq. 7)
  int n_eq;                 // equal east and north neighbours among the sites
  int cnt[8];               // sites per state (q <= 8)
};

constexpr int QREG_MAX = 8;

template <class Keys>
__device__ __forceinline__ void row_bonds(const int8_t* __restrict__ spins, int L, int y, int x, int nvalid,
                                          uint64_t T, const Keys& keys, uint32_t sw_lo, uint32_t sw_hi,
                                          int q, RowBonds& rb) {
  const int yn = (y + 1 == L) ? 0 : y + 1;
  const int64_t row = (int64_t)y * L, rown = (int64_t)yn * L;
  uint32_t s[8], n[8];
  const int nw = nvalid >> 2;   // whole 4-site words (L % 4 == 0)
  if (nw == 8 && (L & 15) == 0) {
    const uint4 a0 = *reinterpret_cast<const uint4*>(spins + row + x);
    const uint4 a1 = *reinterpret_cast<const uint4*>(spins + row + x + 16);
    const uint4 b0 = *reinterpret_cast<const uint4*>(spins + rown + x);
    const uint4 b1 = *reinterpret_cast<const uint4*>(spins + rown + x + 16);
    s[0] = a0.x; s[1] = a0.y; s[2] = a0.z; s[3] = a0.w; s[4] = a1.x; s[5] = a1.y; s[6] = a1.z; s[7] = a1.w;
    n[0] = b0.x; n[1] = b0.y; n[2] = b0.z; n[3] = b0.w; n[4] = b1.x; n[5] = b1.y; n[6] = b1.z; n[7] = b1.w;
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      s[k] = (k < nw) ? *reinterpret_cast<const uint32_t*>(spins + row + x + 4 * k) : 0u;
      n[k] = (k < nw) ? *reinterpret_cast<const uint32_t*>(spins + rown + x + 4 * k) : 0u;
    }
  }
  const int xe = (x + nvalid == L) ? 0 : x + nvalid;
  const uint32_t east_byte = (uint32_t)(uint8_t)spins[row + xe];
  uint32_t eq_e = 0, eq_n = 0;
#pragma unroll
  for (int c = 0; c < QREG_MAX; ++c) rb.cnt[c] = 0;
  if (q == 2 && nw == 8) {
    // Ising spins (bytes 0 or 1) packed one bit per site: the product puts
    // byte k's bit 0 at bit 24 + k, nothing else reaches bits 24..27
    uint32_t sb = 0u, nb = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      sb |= ((s[k] * 0x01020408u) >> 24) << (4 * k);
      nb |= ((n[k] * 0x01020408u) >> 24) << (4 * k);
    }
    eq_e = ~(sb ^ ((sb >> 1) | ((east_byte & 1u) << 31)));
    eq_n = ~(sb ^ nb);
    rb.n_eq = __popc(eq_e) + __popc(eq_n);
    rb.cnt[1] = __popc(sb);
    rb.cnt[0] = 32 - rb.cnt[1];
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (k < nw) {
        const uint32_t next = (k + 1 < nw) ? s[k + 1] : east_byte;
        eq_e |= eq4(s[k], (s[k] >> 8) | (next << 24)) << (4 * k);
        eq_n |= eq4(s[k], n[k]) << (4 * k);
      }
    }
    // observables of the spins read
    const uint32_t valid = nvalid == 32 ? 0xFFFFFFFFu : ((1u << nvalid) - 1u);
    rb.n_eq = __popc(eq_e & valid) + __popc(eq_n & valid);
    if (q == 2) {
      int ones = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) ones += (k < nw) ? __popc(s[k] & 0x01010101u) : 0;
      rb.cnt[0] = nvalid - ones;
      rb.cnt[1] = ones;
    } else if (q <= QREG_MAX) {
#pragma unroll
      for (int c = 0; c < QREG_MAX; ++c) {
        if (c >= q) break;
        int m = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) m += (k < nw) ? __popc(eq4(s[k], 0x01010101u * (uint32_t)c)) : 0;
        rb.cnt[c] = m;
      }
    }
  }
  // bonds: one Philox call per pair of sites i, i+1 (words: east i, north i,
  // east i+1, north i+1)
  if (T >= (1ull << 32)) {
    rb.east = eq_e;                      // p = 1: every bond between equal spins opens
    rb.north = eq_n;
  } else if (T == 0) {
    rb.east = rb.north = 0u;
  } else {
    const uint32_t thr = (uint32_t)T;
    uint32_t e = 0u, n = 0u;
#pragma unroll
    for (int i = 0; i < 32; i += 2) {
      if (i >= nvalid) break;
      const uint4 r = philox_draw(make_uint4((uint32_t)((row + x + i) >> 1), sw_lo, sw_hi, TAG_BOND), keys);
      e |= ((uint32_t)(r.x < thr) | ((uint32_t)(r.z < thr) << 1)) << i;
      n |= ((uint32_t)(r.y < thr) | ((uint32_t)(r.w < thr) << 1)) << i;
    }
    rb.east = e & eq_e;
    rb.north = n & eq_n;
  }
}

// Block-wide sums of n_eq and the state counts, added to the observable slot.
template <int NTHREADS>
__device__ __forceinline__ void add_observables(long long n_eq, const int* cnt, int q, int qreg, unsigned long long* slot,
                                unsigned long long* red /* shared, (1 + qreg) * NTHREADS/32 */,
                                int* hist /* shared, 128, already holds counts when qreg == 0 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NTHREADS / 32;
  unsigned long long v = (unsigned long long)n_eq;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  if (lane == 0) red[warp] = v;
#pragma unroll
  for (int k = 0; k < QREG_MAX; ++k) {
    if (k >= qreg) break;
    unsigned long long c = (unsigned long long)cnt[k];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(FULL, c, o);
    if (lane == 0) red[(1 + k) * NW + warp] = c;
  }
  __syncthreads();
  if (threadIdx.x <= qreg) {
    unsigned long long tot = 0;
    for (int w = 0; w < NW; ++w) tot += red[threadIdx.x * NW + w];
    if (tot && (threadIdx.x == 0 || threadIdx.x - 1 < q)) atomicAdd(slot + threadIdx.x, tot);
  }
  if (qreg == 0) {
    for (int k = threadIdx.x; k < q; k += NTHREADS)
      if (hist[k]) atomicAdd(slot + 1 + k, (unsigned long long)hist[k]);
  }
}

// The two halves of add_observables, for a kernel that has a __syncthreads()
// between them anyway: every warp leaves its sums in `red` ...
template <int NTHREADS>
__device__ __forceinline__ void observables_warp_sums(long long n_eq, const int* cnt, int qreg,
                                                      unsigned long long* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NTHREADS / 32;
  unsigned long long v = (unsigned long long)n_eq;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  if (lane == 0) red[warp] = v;
#pragma unroll
  for (int k = 0; k < QREG_MAX; ++k) {
    if (k >= qreg) break;
    unsigned long long c = (unsigned long long)cnt[k];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(FULL, c, o);
    if (lane == 0) red[(1 + k) * NW + warp] = c;
  }
}

// ... and, after a barrier, the block's totals are added to the slot.
template <int NTHREADS>
__device__ __forceinline__ void observables_commit(int q, int qreg, unsigned long long* slot,
                                                   const unsigned long long* red, const int* hist) {
  constexpr int NW = NTHREADS / 32;
  if (threadIdx.x <= qreg) {
    unsigned long long tot = 0;
    for (int w = 0; w < NW; ++w) tot += red[threadIdx.x * NW + w];
    if (tot && (threadIdx.x == 0 || threadIdx.x - 1 < q)) atomicAdd(slot + threadIdx.x, tot);
  }
  if (qreg == 0) {
    for (int k = threadIdx.x; k < q; k += NTHREADS)
      if (hist[k]) atomicAdd(slot + 1 + k, (unsigned long long)hist[k]);
  }
}

constexpr int QREG = QREG_MAX;   // state counts kept in registers for q <= QREG

}  // namespace fused
using namespace fused;

// After the labeling kernel, the first TILE_SITES / 32 words of a tile's
// pair-list slot (no longer needed once the tile is labeled) hold its
// edge-root bits: bit r set iff local root r's component touches the tile
// edge, so that its cluster may continue in other tiles.  The flip and the
// few-cluster seed selection read them.
constexpr int EDGE_WORDS = TILE_SITES / 32;
static_assert(EDGE_WORDS == LABEL_THREADS, "one edge word per thread");
// Flag on a root-list entry (local indices are below TILE_SITES).
constexpr uint16_t EDGE_ROOT = 0x8000u;
constexpr uint16_t ROOT_MASK = 0x7FFFu;
static_assert(TILE_SITES <= ROOT_MASK + 1, "local index fits below the flag");

struct LabelTileSmem {
  TileSmem tile;
  uint32_t edge_bits[EDGE_WORDS];                   // local roots on the tile edge
  uint32_t e_last;                                  // raw east bit of column w-1, bit = row
  unsigned long long red[(1 + QREG) * (LABEL_THREADS / 32)];
  int hist[128];
};

struct FlipTileSmem {
  uint16_t rlist[TILE_SITES];   // the tile's roots (EDGE_ROOT flag on edge roots)
  uint8_t ns[TILE_SITES];       // new state, indexed by local root
  uint32_t edge_bits[EDGE_WORDS];
  int warp_cnt[LABEL_THREADS / 32];
};

// One tile of the fused draw-and-label step (see k_fused.cu).  All threads
// of the CTA call it; it synchronises the CTA internally and on return.
template <class Keys>
__device__ __forceinline__ void sw_label_tile(const SwRep& R, int t, uint64_t sweep, bool do_obs, int obs_cap,
                                              LabelTileSmem& ls, const Keys& keys) {
  TileSmem& sm = ls.tile;
  uint32_t& e_last = ls.e_last;
  unsigned long long* red = ls.red;
  int* hist = ls.hist;
  const int8_t* __restrict__ spins = R.spins;
  uint16_t* __restrict__ lroot = R.lroot;
  int32_t* __restrict__ gpar = R.gpar;
  const Grid& g = R.g;
  const LabelScratch& s = R.s;
  const int q = R.q;
  const uint64_t T = R.T;
  const int L = g.W;
  const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
  const int y0 = ty * TILE_H, x0 = tx * TILE_W;
  const int h = min(TILE_H, L - y0), w = min(TILE_W, L - x0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t* slot = s.roots + (int64_t)t * TILE_SITES;
  int32_t* hook_log = s.work + (int64_t)t * TILE_SITES;
  if (threadIdx.x == 0) {
    sm.n_hooked = 0;
    e_last = 0u;
  }
  for (int k = threadIdx.x; k < 128; k += LABEL_THREADS) hist[k] = 0;
  ls.edge_bits[threadIdx.x] = 0u;
  __syncthreads();

  // 1. bonds: warp c draws strip c, lane ly row ly
  long long n_eq = 0;
  int cnt[QREG];
#pragma unroll
  for (int k = 0; k < QREG; ++k) cnt[k] = 0;
  uint32_t we = 0u, wn = 0u;
  {
    const int ly = lane, c = warp;
    const int nvalid = min(max(w - 32 * c, 0), 32);
    if (ly < h && nvalid > 0) {
      const int y = y0 + ly, x = x0 + 32 * c;
      RowBonds rb;
      row_bonds(spins, L, y, x, nvalid, T, keys, (uint32_t)sweep, (uint32_t)(sweep >> 32), q, rb);
      we = rb.east;
      wn = rb.north;
      if (32 * c + nvalid == w) {                 // east bond leaving the tile
        const uint32_t bit = 1u << (nvalid - 1);
        if (we & bit) atomicOr(&e_last, 1u << ly);
        we &= ~bit;
      }
      if (do_obs) {
        n_eq = rb.n_eq;
        if (q <= QREG) {
#pragma unroll
          for (int k = 0; k < QREG; ++k) cnt[k] = rb.cnt[k];
        } else {
          const int8_t* p = spins + (int64_t)y * L + x;
          for (int j = 0; j < nvalid; ++j) atomicAdd(&hist[p[j]], 1);
        }
      }
    }
    sm.be[ly * STRIPS + c] = we;
    sm.bn[ly * STRIPS + c] = wn;
  }
  if (do_obs) observables_warp_sums<LABEL_THREADS>(n_eq, cnt, q <= QREG ? q : 0, red);
  __syncthreads();

  // 2. label the tile (the engine ends with a barrier)
  tile_engine_regs(sm, we, wn, h, slot, hook_log, s.err);
  if (do_obs) {   // observables of the spins read (the previous sweep's result)
    unsigned long long* oslot =
        reinterpret_cast<unsigned long long*>(R.obs + (int64_t)((sweep - 1) % (uint64_t)obs_cap) * (q + 1));
    observables_commit<LABEL_THREADS>(q, q <= QREG ? q : 0, oslot, red, hist);
  }

  // 3. tile roots as 16-bit local indices: per step a thread takes four
  //    consecutive sites (consecutive lanes, consecutive 16-byte words of
  //    par: no bank conflicts) and stores 8 bytes (L % 4 == 0; w is a
  //    multiple of 4, so four sites are all inside or all outside)
  auto entry = [&](int p) -> uint32_t { return (uint32_t)sm.par[p]; };   // p = par[site]
#pragma unroll 2
  for (int k = threadIdx.x; k < TILE_SITES / 4; k += LABEL_THREADS) {
    const int sidx = 4 * k;
    const int ly = sidx >> TILE_W_LOG2, lx = sidx & (TILE_W - 1);
    if (ly >= h || lx >= w) continue;
    const int4 pa = *reinterpret_cast<const int4*>(&sm.par[sidx]);
    uint16_t* dst = lroot + (int64_t)(y0 + ly) * L + x0 + lx;
    *reinterpret_cast<uint2*>(dst) = make_uint2(entry(pa.x) | (entry(pa.y) << 16), entry(pa.z) | (entry(pa.w) << 16));
  }

  // 4. seam record; parent entries of edge roots; edge roots marked
  int32_t* rec = s.seams + (int64_t)t * SeamLayout::INTS;
  uint32_t* edge_bits = ls.edge_bits;
  auto root_at = [&](int ly, int lx) -> int { return sm.par[sm.par[ly * TILE_W + lx]]; };
  auto edge_root = [&](bool ok, int r) -> int32_t {
    // global index of local root r; the first of a run of equal roots among
    // consecutive lanes writes its parent entry and its edge mark
    const int left = __shfl_up_sync(FULL, ok ? r : -1, 1);
    if (!ok) return -1;
    const int32_t gr = tile_global(r, y0, x0, L);
    if (lane == 0 || left != r) {
      gpar[gr] = gr;
      atomicOr(&edge_bits[r >> 5], 1u << (r & 31));
    }
    return gr;
  };
  for (int k = threadIdx.x; k < TILE_H; k += LABEL_THREADS) {
    const bool ok = k < h;
    rec[SeamLayout::COL_L + k] = edge_root(ok, ok ? root_at(k, 0) : 0);
    rec[SeamLayout::COL_R + k] = edge_root(ok, ok ? root_at(k, w - 1) : 0);
    if (lane == 0) rec[SeamLayout::E_BITS + (k >> 5)] = (int32_t)e_last;
  }
  for (int k = threadIdx.x; k < TILE_W; k += LABEL_THREADS) {
    const bool ok = k < w;
    rec[SeamLayout::ROW_B + k] = edge_root(ok, ok ? root_at(0, k) : 0);
    rec[SeamLayout::ROW_T + k] = edge_root(ok, ok ? root_at(h - 1, k) : 0);
    const bool n = ok && ((sm.bn[(h - 1) * STRIPS + (k >> 5)] >> (k & 31)) & 1u);
    const uint32_t nb = __ballot_sync(FULL, n);
    if (lane == 0) rec[SeamLayout::N_BITS + (k >> 5)] = (int32_t)nb;
  }

  __syncthreads();
  // 5. edge-root bits into the (now free) pair-list slot; each thread reads
  //    and next clears only its own word
  slot[threadIdx.x] = (int32_t)ls.edge_bits[threadIdx.x];
}

// One tile of the fused flip step (see k_fused.cu).  All threads of the CTA
// call it; it synchronises the CTA internally and on return.
// Site ownership of the flip: with G = TILE_W / 8 column groups, thread k
// owns, in each of four passes j, the eight sites (row 8j + k / G, columns
// 8 (k % G) .. 8 (k % G) + 7) of the tile; their tile roots are one 16-byte
// word per pass.
constexpr int FLIP_GROUPS = TILE_W / 8;
constexpr int FLIP_PASSES = TILE_SITES / (8 * LABEL_THREADS);
static_assert(FLIP_PASSES * 8 * LABEL_THREADS == TILE_SITES && LABEL_THREADS / FLIP_GROUPS == 8, "site ownership");

// Local root (16 bits) of site i (0..7) of a pass word.
__device__ __forceinline__ int root_in(const uint4& v, int i) {
  const uint32_t wv = (i < 2) ? v.x : (i < 4) ? v.y : (i < 6) ? v.z : v.w;
  return (int)((wv >> (16 * (i & 1))) & 0xFFFFu);
}

// The pass words of the calling thread.
struct RootsInRegs {
  uint4 r4[FLIP_PASSES];
  __device__ __forceinline__ uint4 get(int j) const { return r4[j]; }
};
// Steps 2-5 of the flip of tile t (see k_fused.cu) given the tile roots of
// the calling thread's sites.  All threads of the CTA call it; it ends with a
// barrier.
// FEW: the few-cluster update (Sec. III, variant (c)).  Only clusters whose
// global root has its bit set in `sel` (seeded clusters) move: with FLIP draw
// w of the root, iff (uint64)w.y < P, to state (s + 1 + F_{q-1}(w.x)) mod q,
// s being the cluster's current state (read at the tile root).
template <bool FEW, class Roots, class Keys>
__device__ __forceinline__ void flip_tile_core(const SwRep& R, int t, uint64_t sweep, int limit, FlipTileSmem& fs,
                                               const Roots& roots, const uint32_t* __restrict__ sel, uint64_t P,
                                               const Keys& keys) {
  constexpr int PASSES = FLIP_PASSES;
  uint16_t* rlist = fs.rlist;
  uint8_t* ns = fs.ns;
  int* warp_cnt = fs.warp_cnt;
  int8_t* __restrict__ spins = R.spins;
  int32_t* __restrict__ gpar = R.gpar;
  const Grid& g = R.g;
  const int q = R.q;
  int* err = R.s.err;
  const int L = g.W;
  const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
  const int y0 = ty * TILE_H, x0 = tx * TILE_W;
  const int h = min(TILE_H, L - y0), w = min(TILE_W, L - x0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int orow = threadIdx.x / FLIP_GROUPS, lx0 = 8 * (threadIdx.x % FLIP_GROUPS);   // my sites
  // the tile's edge-root bits, left by the labeling kernel
  fs.edge_bits[threadIdx.x] = (uint32_t)__ldcg(R.s.roots + (int64_t)t * TILE_SITES + threadIdx.x);

  // 2. my roots: a site is a tile root iff its entry is its own local index.
  //    Word k of pass j holds sites 2k and 2k + 1; both are compared at once
  //    (a half-word is zero iff its low 15 bits plus 0x7FFF stay below bit
  //    15 and its bit 15 is clear).  Sites outside the tile hold 0xFFFF and
  //    never match.  Bit 4j + k of `mine` flags site 2k of pass j, bit
  //    16 + 4j + k site 2k + 1.
  uint32_t mine = 0;
#pragma unroll
  for (int j = 0; j < PASSES; ++j) {
    const uint4 rv = roots.get(j);
    const uint32_t base = (uint32_t)((8 * j + orow) * TILE_W + lx0);
    const uint32_t own = base * 0x00010001u + 0x00010000u;   // (base, base + 1)
    const uint32_t wv[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t x = wv[k] ^ (own + (uint32_t)k * 0x00020002u);
      const uint32_t nz = ((x & 0x7FFF7FFFu) + 0x7FFF7FFFu) | x;
      mine |= (~nz & 0x80008000u) >> (15 - (4 * j + k));
    }
  }
  const int cnt = __popc(mine);
  int incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) warp_cnt[warp] = incl;
  __syncthreads();
  int base = 0, n_roots = 0;
#pragma unroll
  for (int k = 0; k < LABEL_THREADS / 32; ++k) {
    base += (k < warp) ? warp_cnt[k] : 0;
    n_roots += warp_cnt[k];
  }
  base += incl - cnt;
  while (mine) {   // the tile's root list, edge roots flagged
    const int b = __ffs(mine) - 1;
    mine &= mine - 1;
    const int jk = b & 15;
    const int r = (8 * (jk >> 2) + orow) * TILE_W + lx0 + 2 * (jk & 3) + (b >> 4);
    rlist[base++] = (uint16_t)r | (((fs.edge_bits[r >> 5] >> (r & 31)) & 1u) ? EDGE_ROOT : (uint16_t)0);
  }
  __syncthreads();

  // 4. one draw per tile root, keyed by its cluster's final root; a thread
  //    takes its roots two at a time, their parent walks in lock step
  constexpr int U = 2;
  for (int k0 = threadIdx.x; k0 < n_roots; k0 += U * LABEL_THREADS) {
    int r[U], Rg[U];
    bool act[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * LABEL_THREADS;
      const int raw = k < n_roots ? (int)rlist[k] : 0;
      r[u] = raw & ROOT_MASK;
      Rg[u] = tile_global(r[u], y0, x0, L);
      act[u] = k < n_roots && (raw & EDGE_ROOT);
    }
    g_find_multi<U>(gpar, Rg, act, limit, err);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u * LABEL_THREADS >= n_roots) break;
      if (FEW) {
        // the cluster's current state, read at the tile root (this tile's own
        // site: step 5 rewrites it only after a barrier)
        int v = spins[(int64_t)(y0 + (r[u] >> TILE_W_LOG2)) * L + x0 + (r[u] & (TILE_W - 1))];
        if ((__ldcg(sel + (Rg[u] >> 5)) >> (Rg[u] & 31)) & 1u) {
          const uint4 d =
              philox_draw(make_uint4((uint32_t)Rg[u], (uint32_t)sweep, (uint32_t)(sweep >> 32), TAG_FLIP), keys);
          if ((uint64_t)d.y < P) v = (v + 1 + state_of(d.x, q - 1)) % q;
        }
        ns[r[u]] = (uint8_t)v;
      } else {
        const uint4 d =
            philox_draw(make_uint4((uint32_t)Rg[u], (uint32_t)sweep, (uint32_t)(sweep >> 32), TAG_FLIP), keys);
        ns[r[u]] = (uint8_t)state_of(d.x, q);
      }
    }
  }
  __syncthreads();

  // 5. every site takes its tile root's state
#pragma unroll
  for (int j = 0; j < PASSES; ++j) {
    const int ly = 8 * j + orow;
    if (ly >= h || lx0 + 4 > w) continue;
    const uint4 rv = roots.get(j);
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) lo |= (uint32_t)ns[root_in(rv, i)] << (8 * i);
    int8_t* dst = spins + (int64_t)(y0 + ly) * L + x0 + lx0;
    *reinterpret_cast<uint32_t*>(dst) = lo;   // 4-byte aligned: L % 4 == 0
    if (lx0 + 8 <= w) {
#pragma unroll
      for (int i = 0; i < 4; ++i) hi |= (uint32_t)ns[root_in(rv, 4 + i)] << (8 * i);
      *reinterpret_cast<uint32_t*>(dst + 4) = hi;
    }
  }
  __syncthreads();
}

// Observables of the current spins of tile t (bonds joining equal spins, the
// tile's east and north bonds, and sites per state), added to the slot of
// sweep `done`.  All threads of the CTA call it.
__device__ __forceinline__ void observe_tile(const SwRep& R, int t, uint64_t done, int obs_cap, LabelTileSmem& ls) {
  const Grid& g = R.g;
  const int L = g.W, q = R.q;
  const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
  const int y0 = ty * TILE_H, x0 = tx * TILE_W;
  const int h = min(TILE_H, L - y0), w = min(TILE_W, L - x0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < 128; k += LABEL_THREADS) ls.hist[k] = 0;
  __syncthreads();
  long long n_eq = 0;
  int cnt[QREG];
#pragma unroll
  for (int k = 0; k < QREG; ++k) cnt[k] = 0;
  const int ly = lane, c = warp;
  const int nvalid = min(max(w - 32 * c, 0), 32);
  if (ly < h && nvalid > 0) {
    const int y = y0 + ly, x = x0 + 32 * c;
    const int yn = (y + 1 == L) ? 0 : y + 1;
    const int8_t* row = R.spins + (int64_t)y * L;
    const int8_t* rown = R.spins + (int64_t)yn * L;
    const int nw = nvalid >> 2;
    const int xe = (x + nvalid == L) ? 0 : x + nvalid;
    const uint32_t east_byte = (uint32_t)(uint8_t)row[xe];
    for (int k = 0; k < nw; ++k) {
      const uint32_t cur = *reinterpret_cast<const uint32_t*>(row + x + 4 * k);
      const uint32_t nor = *reinterpret_cast<const uint32_t*>(rown + x + 4 * k);
      const uint32_t next = (k + 1 < nw) ? *reinterpret_cast<const uint32_t*>(row + x + 4 * k + 4) : east_byte;
      n_eq += __popc(eq4(cur, (cur >> 8) | (next << 24))) + __popc(eq4(cur, nor));
      if (q <= QREG) {
#pragma unroll
        for (int s = 0; s < QREG; ++s)
          if (s < q) cnt[s] += __popc(eq4(cur, 0x01010101u * (uint32_t)s));
      } else {
        for (int j = 0; j < 4; ++j) atomicAdd(&ls.hist[(cur >> (8 * j)) & 0xFF], 1);
      }
    }
  }
  unsigned long long* oslot =
      reinterpret_cast<unsigned long long*>(R.obs + (int64_t)(done % (uint64_t)obs_cap) * (q + 1));
  add_observables<LABEL_THREADS>(n_eq, cnt, q, q <= QREG ? q : 0, oslot, ls.red, ls.hist);
  __syncthreads();
}


// The flip of tile t with the tile roots loaded into registers (one CTA per
// tile; also the batch kernels).
template <bool FEW = false, class Keys = SeedKey>
__device__ __forceinline__ void sw_flip_tile(const SwRep& R, int t, uint64_t sweep, int limit, FlipTileSmem& fs,
                                             const Keys& keys, const uint32_t* __restrict__ sel = nullptr,
                                             uint64_t P = 0) {
  const uint16_t* __restrict__ lroot = R.lroot;
  const int L = R.g.W;
  const int ty = t / R.g.tiles_x, tx = t - ty * R.g.tiles_x;
  const int y0 = ty * TILE_H, x0 = tx * TILE_W;
  const int h = min(TILE_H, L - y0), w = min(TILE_W, L - x0);
  const int orow = threadIdx.x / FLIP_GROUPS, lx0 = 8 * (threadIdx.x % FLIP_GROUPS);   // my sites
  // 1. tile roots of my sites (w is a multiple of 4: a group of eight sites is
  //    either wholly inside, or its first four are); read through L2 because a
  //    persistent kernel wrote them on other SMs
  RootsInRegs roots;
#pragma unroll
  for (int j = 0; j < FLIP_PASSES; ++j) {
    const int ly = 8 * j + orow;
    const uint16_t* src = lroot + (int64_t)(y0 + ly) * L + x0 + lx0;
    uint4 v = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
    // 16-byte loads need L % 8 == 0; L % 4 == 0 always allows 8-byte loads
    if (ly < h && lx0 + 8 <= w) {
      if ((L & 7) == 0) {
        v = __ldcg(reinterpret_cast<const uint4*>(src));
      } else {
        const uint2 a = __ldcg(reinterpret_cast<const uint2*>(src)), b = __ldcg(reinterpret_cast<const uint2*>(src + 4));
        v = make_uint4(a.x, a.y, b.x, b.y);
      }
    } else if (ly < h && lx0 + 4 <= w) {
      const uint2 a = __ldcg(reinterpret_cast<const uint2*>(src));
      v.x = a.x;
      v.y = a.y;
    }
    roots.r4[j] = v;
  }
  flip_tile_core<FEW>(R, t, sweep, limit, fs, roots, sel, P, keys);
}

// The flip of tile t when every tile of the lattice is whole (L a multiple
// of TILE_W, TILE_H and 8): the steps of flip_tile_core with no bounds
// checks, and the tile roots of the calling thread's sites read through L2
// twice (root discovery, site pass) instead of held in registers across
// the draws, which would not fit the register budget of six CTAs per SM.
template <class Keys>
__device__ __forceinline__ void sw_flip_whole_tile(const SwRep& R, int t, uint64_t sweep, int limit,
                                                   FlipTileSmem& fs, const Keys& keys) {
  constexpr int PASSES = FLIP_PASSES;
  const int L = R.g.W;
  const int ty = t / R.g.tiles_x, tx = t - ty * R.g.tiles_x;
  const int y0 = ty * TILE_H, x0 = tx * TILE_W;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int orow = threadIdx.x / FLIP_GROUPS, lx0 = 8 * (threadIdx.x % FLIP_GROUPS);   // my sites
  const uint16_t* src0 = R.lroot + (int64_t)(y0 + orow) * L + x0 + lx0;   // pass 0; 16-byte aligned
  const int64_t pass_stride = (int64_t)8 * L;
  uint16_t* rlist = fs.rlist;
  uint8_t* ns = fs.ns;
  int* warp_cnt = fs.warp_cnt;
  fs.edge_bits[threadIdx.x] = (uint32_t)__ldcg(R.s.roots + (int64_t)t * TILE_SITES + threadIdx.x);

  // 2. my roots (as in flip_tile_core)
  uint32_t mine = 0;
  {
    uint4 held[PASSES];
#pragma unroll
    for (int j = 0; j < PASSES; ++j) held[j] = __ldcg(reinterpret_cast<const uint4*>(src0 + j * pass_stride));
#pragma unroll
    for (int j = 0; j < PASSES; ++j) {
      const uint4 rv = held[j];
      const uint32_t base = (uint32_t)((8 * j + orow) * TILE_W + lx0);
      const uint32_t own = base * 0x00010001u + 0x00010000u;
      const uint32_t wv[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t x = wv[k] ^ (own + (uint32_t)k * 0x00020002u);
        const uint32_t nz = ((x & 0x7FFF7FFFu) + 0x7FFF7FFFu) | x;
        mine |= (~nz & 0x80008000u) >> (15 - (4 * j + k));
      }
    }
  }
  const int cnt = __popc(mine);
  int incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) warp_cnt[warp] = incl;
  __syncthreads();
  int base = 0, n_roots = 0;
#pragma unroll
  for (int k = 0; k < LABEL_THREADS / 32; ++k) {
    base += (k < warp) ? warp_cnt[k] : 0;
    n_roots += warp_cnt[k];
  }
  base += incl - cnt;
  while (mine) {   // 3. the tile's root list, edge roots flagged
    const int b = __ffs(mine) - 1;
    mine &= mine - 1;
    const int jk = b & 15;
    const int r = (8 * (jk >> 2) + orow) * TILE_W + lx0 + 2 * (jk & 3) + (b >> 4);
    rlist[base++] = (uint16_t)r | (((fs.edge_bits[r >> 5] >> (r & 31)) & 1u) ? EDGE_ROOT : (uint16_t)0);
  }
  __syncthreads();

  // 4. one draw per tile root, keyed by its cluster's final root
  constexpr int U = 4;   // four walks of a thread in flight (flip_tile_core, with the roots in registers, keeps two)
  for (int k0 = threadIdx.x; k0 < n_roots; k0 += U * LABEL_THREADS) {
    int r[U], Rg[U];
    bool act[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * LABEL_THREADS;
      const int raw = k < n_roots ? (int)rlist[k] : 0;
      r[u] = raw & ROOT_MASK;
      Rg[u] = tile_global(r[u], y0, x0, L);
      act[u] = k < n_roots && (raw & EDGE_ROOT);
    }
    g_find_multi<U>(R.gpar, Rg, act, limit, R.s.err);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u * LABEL_THREADS >= n_roots) break;
      const uint4 d =
          philox_draw(make_uint4((uint32_t)Rg[u], (uint32_t)sweep, (uint32_t)(sweep >> 32), TAG_FLIP), keys);
      ns[r[u]] = (uint8_t)state_of(d.x, R.q);
    }
  }
  __syncthreads();

  // 5. every site takes its tile root's state (tile roots read again)
#pragma unroll
  for (int j = 0; j < PASSES; ++j) {
    const int ly = 8 * j + orow;
    const uint4 rv = __ldcg(reinterpret_cast<const uint4*>(src0 + j * pass_stride));
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) lo |= (uint32_t)ns[root_in(rv, i)] << (8 * i);
#pragma unroll
    for (int i = 0; i < 4; ++i) hi |= (uint32_t)ns[root_in(rv, 4 + i)] << (8 * i);
    int8_t* dst = R.spins + (int64_t)(y0 + ly) * L + x0 + lx0;
    *reinterpret_cast<uint2*>(dst) = make_uint2(lo, hi);   // 8-byte aligned: L % 8 == 0
  }
}

// ---------------------------------------------------------------------------
// Few-cluster seed selection (Sec. III, variant (c)): the seed of block b of
// the ell x ell block grid (side B = L / ell) is (bx B + F_B(w.x),
// by B + F_B(w.y)) with w the SEED draw (b, sweep); the bit of its cluster's
// global root is set in `sel`.  Runs between the merge and the flip.  If the
// seed's tile root is an edge root (its cluster may leave the tile), its
// global root is found on gpar; otherwise the tile root is the cluster's root.
__device__ __forceinline__ void few_select_seed(const SwRep& R, int ell, int64_t b, uint64_t sweep, uint32_t* sel,
                                                int limit) {
  const Grid& g = R.g;
  const int L = g.W;
  const int B = L / ell;
  const int by = (int)(b / ell), bx = (int)(b - (int64_t)by * ell);
  const uint4 w = philox(make_uint4((uint32_t)b, (uint32_t)sweep, (uint32_t)(sweep >> 32), TAG_SEED),
                         (uint32_t)R.seed, (uint32_t)(R.seed >> 32));
  const int x = bx * B + state_of(w.x, B), y = by * B + state_of(w.y, B);
  const int ty = y / TILE_H, tx = x / TILE_W;
  const int r = R.lroot[(int64_t)y * L + x];
  const int G = tile_global(r, ty * TILE_H, tx * TILE_W, L);
  const int32_t* edge_bits = R.s.roots + (int64_t)(ty * g.tiles_x + tx) * TILE_SITES;
  const bool edge = (__ldcg(edge_bits + (r >> 5)) >> (r & 31)) & 1;
  const int root = edge ? g_find(R.gpar, G, limit, R.s.err) : G;
  atomicOr(sel + (root >> 5), 1u << (root & 31));
}

}  // namespace swccl
