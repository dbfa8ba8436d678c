// k_cubic.cu -- the Swendsen-Wang sweep on the periodic simple-cubic lattice.
//
// The paper develops the method on the square lattice and notes that the
// three-dimensional case follows the same steps with six neighbours
// (Secs. II and II.B).  Box X x Y x Z, site i = (z Y + y) X + x; each site
// owns its bonds to the +x, +y and +z neighbours (periodic), drawn from one
// Philox call per site (tag BOND3, counter (i, sweep), word = direction) and
// open iff the two spins are equal and the word is below T (Eq. 7).
//
// One sweep is three kernels and an advance, the structure of the fused
// square-lattice sweep (k_fused.cu) carried to bricks of 32 x 8 x 16 sites:
//  k3_local    one CTA per brick: draws the bonds of its sites, labels the
//              brick with the square-lattice tile engine (each warp sweeps an
//              (x, z) plane; +y bonds and wraps joined with shared-memory
//              unions; larger root hooked under the smaller, so a brick root
//              is the brick component's smallest index), writes each site's brick root as
//              a 16-bit local index, marks the roots whose component touches
//              the brick's faces (edge roots: bit words per brick, and a
//              parent entry gpar[G] = G at their global index G), and counts
//              the observables of the spins it read (the previous sweep's);
//  k3_merge    one thread per site on a brick face: redraws the face bond
//              (the draws are counter-based) and, if open, joins the brick
//              roots on its two ends on gpar with global atomics;
//  k3_flip     one CTA per brick: lists the brick's roots; an edge root looks
//              up its cluster root R on gpar, any other root is its own
//              cluster's root; one FLIP draw per root (keyed by R, Sec. II.D)
//              gives the state every site of the brick component takes.
//  k3_observe  counts the observables of the last sweep when they are read.
// HBM traffic per site: spins read 1 B and brick roots written 2 B (local),
// brick roots read 2 B and spins written 1 B (flip), plus the face sites,
// the edge-root bits (1/8 B) and the sparse parent entries.
#include "fused_tile.cuh"

namespace swccl {

constexpr int B3X = 32, B3Y = 8, B3Z = 16;
constexpr int B3_SITES = B3X * B3Y * B3Z;
constexpr int B3_THREADS = 256;
static_assert(B3_THREADS == B3X * B3Y, "thread (lx, ly) walks the brick along z");

__device__ __forceinline__ int64_t site3(const Box3& b, int x, int y, int z) {
  return ((int64_t)z * b.Y + y) * b.X + x;
}

// Bonds of site (x, y, z) in direction d (0 +x, 1 +y, 2 +z) given its spin
// s and Philox words w: open iff the neighbour's spin equals s and the word
// is below T.  Writes the neighbour's coordinates.
__device__ __forceinline__ bool bond3(const int8_t* __restrict__ spins, const Box3& b, int x, int y, int z, int d,
                                      int s, const uint4& w, uint64_t T, int& nx, int& ny, int& nz) {
  nx = x;
  ny = y;
  nz = z;
  uint32_t word;
  if (d == 0) {
    nx = (x + 1 == b.X) ? 0 : x + 1;
    word = w.x;
  } else if (d == 1) {
    ny = (y + 1 == b.Y) ? 0 : y + 1;
    word = w.y;
  } else {
    nz = (z + 1 == b.Z) ? 0 : z + 1;
    word = w.z;
  }
  return spins[site3(b, nx, ny, nz)] == s && (uint64_t)word < T;
}

__device__ __forceinline__ uint4 bond3_words(int64_t i, uint64_t sweep, uint64_t T, uint64_t seed) {
  if (T == 0 || T >= (1ull << 32)) return make_uint4(0u, 0u, 0u, 0u);   // p = 0 or 1: no draw needed
  return draw((uint32_t)i, sweep, TAG_BOND3, seed);
}

constexpr int B3_EDGE_WORDS = B3_SITES / 32;   // edge-root bits of one brick

struct Brick {
  int tbx, tby, tbz, x0, y0, z0, w, h, d;
};

__device__ __forceinline__ Brick brick_of(const Box3& b, int t) {
  Brick k;
  k.tbx = t % b.bx;
  k.tby = (t / b.bx) % b.by;
  k.tbz = t / (b.bx * b.by);
  k.x0 = k.tbx * B3X;
  k.y0 = k.tby * B3Y;
  k.z0 = k.tbz * B3Z;
  k.w = min(B3X, b.X - k.x0);
  k.h = min(B3Y, b.Y - k.y0);
  k.d = min(B3Z, b.Z - k.z0);
  return k;
}

// Global index of local index l of brick k (l = (lz B3Y + ly) B3X + lx).
__device__ __forceinline__ int64_t brick_global(const Box3& b, const Brick& k, int l) {
  return site3(b, k.x0 + l % B3X, k.y0 + (l / B3X) % B3Y, k.z0 + l / (B3X * B3Y));
}

// Spins of a brick and of its +x, +y, +z neighbour faces in shared memory:
// entry (lz, ly, lx) for lx <= w, ly <= h, lz <= d (one past the brick's end
// is the neighbouring brick's face, or the periodic wrap).
constexpr int SP_X = B3X + 1, SP_Y = B3Y + 1, SP_Z = B3Z + 1;
constexpr int SP_SIZE = SP_X * SP_Y * SP_Z;
__device__ __forceinline__ int sp_at(int lx, int ly, int lz) { return (lz * SP_Y + ly) * SP_X + lx; }

// A brick is labeled by the square-lattice tile engine (tile_engine.cuh):
// with row = lz and strip = ly its local index (lz B3Y + ly) B3X + lx is the
// engine's row * TILE_W + strip * 32 + lane, so each warp sweeps its (x, z)
// plane along z (the +x bonds are the engine's east bonds, the +z bonds its
// north bonds).  The +y bonds between the planes, and the periodic wraps of
// an axis one brick long, are joined afterwards with shared-memory unions.
static_assert(B3X == 32 && B3Y == STRIPS && B3Z <= TILE_H && B3X * B3Y == TILE_W, "brick = engine tile");

struct Local3Smem {
  TileSmem tile;
  uint32_t edge[B3_EDGE_WORDS];
  uint32_t ybits[B3Z * B3Y];     // open +y bond joined inside the brick, bit = lx
  uint32_t xwrap[B3Z * B3Y];     // open +x bond wrapping inside the brick (one brick along x)
  uint32_t zwrap[B3Y];           // open +z bond of the last plane wrapping inside the brick
  unsigned long long red[(1 + QREG) * (B3_THREADS / 32)];
  int hist[128];
  int8_t sp[SP_SIZE];
};

__global__ void __launch_bounds__(B3_THREADS, 4)
k3_local(const int8_t* __restrict__ spins, uint16_t* __restrict__ lroot, int32_t* __restrict__ gpar,
         uint32_t* __restrict__ edge_words, int32_t* __restrict__ scratch, Box3 b, int q, uint64_t T, uint64_t seed,
         const SwCtl* __restrict__ ctl, int64_t* obs, int obs_cap, int* err) {
  __shared__ Local3Smem ls;
  TileSmem& sm = ls.tile;
  int* par = sm.par;
  int8_t* sp = ls.sp;
  const Brick k = brick_of(b, blockIdx.x);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = lane, ly = warp;
  if (threadIdx.x == 0) sm.n_hooked = 0;
  for (int j = threadIdx.x; j < B3_EDGE_WORDS; j += B3_THREADS) ls.edge[j] = 0u;
  for (int j = threadIdx.x; j < 128; j += B3_THREADS) ls.hist[j] = 0;
  if (threadIdx.x < B3Y) ls.zwrap[threadIdx.x] = 0u;
  // 0. the brick's spins and the three neighbour faces (no edges or corners:
  //    bonds are along the axes).  Thread (lx, ly) loads its column, z face
  //    included; threads 0..127 the +x face, all threads two entries of the
  //    +y face; every load of a thread is issued before its stores.
  const int64_t XY = (int64_t)b.X * b.Y;
  const bool col = lx < k.w && ly < k.h;
  const int64_t i0 = col ? site3(b, k.x0 + lx, k.y0 + ly, k.z0) : 0;   // column base, z = z0
  const int zf = k.z0 + k.d == b.Z ? 0 : k.z0 + k.d;                      // z face (wrapped)
  int8_t cz[B3Z + 1];
#pragma unroll
  for (int lz = 0; lz <= B3Z; ++lz) {
    const bool in = col && lz < k.d;
    cz[lz] = in ? spins[i0 + lz * XY] : (col && lz == k.d ? spins[site3(b, k.x0 + lx, k.y0 + ly, zf)] : (int8_t)0);
  }
  const int xf = k.x0 + k.w == b.X ? 0 : k.x0 + k.w, yf = k.y0 + k.h == b.Y ? 0 : k.y0 + k.h;
  const int fx_ly = threadIdx.x & (B3Y - 1), fx_lz = threadIdx.x >> 3;             // +x face: 8 x 16
  const bool fx_in = threadIdx.x < B3Y * B3Z && fx_ly < k.h && fx_lz < k.d;
  const int8_t fx = fx_in ? spins[site3(b, xf, k.y0 + fx_ly, k.z0 + fx_lz)] : (int8_t)0;
  int8_t fy[2];                                                                       // +y face: 32 x 16
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = threadIdx.x + u * B3_THREADS, ex = e & (B3X - 1), ez = e >> 5;
    fy[u] = (ex < k.w && ez < k.d) ? spins[site3(b, k.x0 + ex, yf, k.z0 + ez)] : (int8_t)0;
  }
  if (col) {   // only the brick's own columns: the faces at lx = w and ly = h are written below
#pragma unroll
    for (int lz = 0; lz <= B3Z; ++lz)
      if (lz <= k.d) sp[sp_at(lx, ly, lz)] = cz[lz];
  }
  if (fx_in) sp[sp_at(k.w, fx_ly, fx_lz)] = fx;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = threadIdx.x + u * B3_THREADS, ex = e & (B3X - 1), ez = e >> 5;
    if (ex < k.w && ez < k.d) sp[sp_at(ex, k.h, ez)] = fy[u];
  }
  __syncthreads();
  const uint64_t sweep = ctl->sweep;
  const bool do_obs = sweep > 0 && ctl->obs_done != (long long)(sweep - 1);
  const uint32_t Tw = (uint32_t)T;
  const bool all_open = T >= (1ull << 32), none_open = T == 0;
  long long n_eq = 0;
  unsigned long long cpack = 0;   // sites per state, 8 bits per state (q <= 8; at most 16 sites)
  // 1. bonds of every site (plane ly = warp, lane lx, rows lz); observables
  //    of the spins read
  for (int lz = 0; lz < k.d; ++lz) {
    bool o0 = false, o1 = false, o2 = false;
    if (col) {
      const int s = sp[sp_at(lx, ly, lz)];
      const bool e0 = sp[sp_at(lx + 1, ly, lz)] == s, e1 = sp[sp_at(lx, ly + 1, lz)] == s,
                 e2 = sp[sp_at(lx, ly, lz + 1)] == s;
      if (do_obs) {
        n_eq += (int)e0 + (int)e1 + (int)e2;
        if (q <= QREG) cpack += 1ull << (8 * s);
        else atomicAdd(&ls.hist[s], 1);
      }
      if (!none_open && (e0 || e1 || e2)) {
        if (all_open) {
          o0 = e0;
          o1 = e1;
          o2 = e2;
        } else {
          const uint4 wd = draw((uint32_t)(i0 + lz * XY), sweep, TAG_BOND3, seed);
          o0 = e0 && wd.x < Tw;
          o1 = e1 && wd.y < Tw;
          o2 = e2 && wd.z < Tw;
        }
      }
    }
    // inside the brick: +x to lane lx+1, +z to row lz+1 (engine); +y to plane
    // ly+1 (union below); wraps of an axis one brick long (union below)
    const uint32_t east = __ballot_sync(FULL, o0 && lx + 1 < k.w);
    const uint32_t north = __ballot_sync(FULL, o2 && lz + 1 < k.d);
    const uint32_t ybit = __ballot_sync(FULL, o1 && (ly + 1 < k.h || b.by == 1));
    const uint32_t xw = __ballot_sync(FULL, o0 && lx + 1 == k.w && b.bx == 1);
    const uint32_t zw = __ballot_sync(FULL, o2 && lz + 1 == k.d && b.bz == 1);
    if (lane == 0) {
      sm.be[lz * STRIPS + ly] = east;
      sm.bn[lz * STRIPS + ly] = north;
      ls.ybits[lz * B3Y + ly] = ybit;
      ls.xwrap[lz * B3Y + ly] = xw;
      if (zw) ls.zwrap[ly] = zw;
    }
  }
  __syncthreads();
  // 2. the engine labels the brick's planes and joins them along z
  int32_t* slot = scratch + (int64_t)blockIdx.x * 2 * TILE_SITES;
  tile_engine(sm, k.d, slot, slot + TILE_SITES, err);
  // 3. +y bonds and wraps
  for (int lz = 0; lz < k.d; ++lz) {
    const int l = (lz * B3Y + ly) * B3X + lx;
    if ((ls.ybits[lz * B3Y + ly] >> lx) & 1u)
      sm_union(par, l, ly + 1 < k.h ? l + B3X : l - ly * B3X, B3_SITES, err);
    if ((ls.xwrap[lz * B3Y + ly] >> lx) & 1u) sm_union(par, l, l - lx, B3_SITES, err);
    if (lz + 1 == k.d && ((ls.zwrap[ly] >> lx) & 1u)) sm_union(par, l, l - lz * B3Y * B3X, B3_SITES, err);
  }
  __syncthreads();
  uint32_t* edge = ls.edge;
  int* hist = ls.hist;
  unsigned long long* red = ls.red;
  // 4. brick roots (16-bit local index) of every site; edge roots marked
  if (col) {
    for (int lz = 0; lz < k.d; ++lz) {
      const int l = (lz * B3Y + ly) * B3X + lx;
      const int r = sm_find(par, l, B3_SITES, err);
      lroot[i0 + lz * XY] = (uint16_t)r;
      if (lx == 0 || lx == k.w - 1 || ly == 0 || ly == k.h - 1 || lz == 0 || lz == k.d - 1)
        atomicOr(&edge[r >> 5], 1u << (r & 31));
    }
  }
  __syncthreads();
  // 5. parent entries of edge roots; the brick's edge bits for the flip
  if (col) {
    for (int lz = 0; lz < k.d; ++lz) {
      const int l = (lz * B3Y + ly) * B3X + lx;
      if (par[l] == l && ((edge[l >> 5] >> (l & 31)) & 1u)) gpar[i0 + lz * XY] = (int32_t)(i0 + lz * XY);
    }
  }
  for (int j = threadIdx.x; j < B3_EDGE_WORDS; j += B3_THREADS)
    edge_words[(int64_t)blockIdx.x * B3_EDGE_WORDS + j] = edge[j];
  if (do_obs) {
    int cnt[QREG];
#pragma unroll
    for (int j = 0; j < QREG; ++j) cnt[j] = (int)((cpack >> (8 * j)) & 0xFFu);
    unsigned long long* oslot =
        reinterpret_cast<unsigned long long*>(obs + (int64_t)((sweep - 1) % (uint64_t)obs_cap) * (q + 1));
    add_observables<B3_THREADS>(n_eq, cnt, q, q <= QREG ? q : 0, oslot, red, hist);
  }
}

// Face sites: for axis d, the coordinates whose +d neighbour lies in another
// brick (none when one brick spans the axis).
__device__ __forceinline__ int face_coord(int k, int extent, int brick) {
  return min((k + 1) * brick, extent) - 1;
}

__global__ void k3_merge(const int8_t* __restrict__ spins, const uint16_t* __restrict__ lroot, int32_t* gpar, Box3 b,
                         uint64_t T, uint64_t seed, const SwCtl* __restrict__ ctl, int limit, int* err) {
  const int64_t nfx = b.bx > 1 ? (int64_t)b.bx * b.Y * b.Z : 0;
  const int64_t nfy = b.by > 1 ? (int64_t)b.X * b.by * b.Z : 0;
  const int64_t nfz = b.bz > 1 ? (int64_t)b.X * b.Y * b.bz : 0;
  const int64_t total = nfx + nfy + nfz;
  const uint64_t sweep = ctl->sweep;
  const uint64_t Tp = T >= (1ull << 32) ? ~0ull : T;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z, d;
    if (k < nfx) {
      d = 0;
      const int64_t yz = k / b.bx;
      x = face_coord((int)(k - yz * b.bx), b.X, B3X);
      y = (int)(yz % b.Y);
      z = (int)(yz / b.Y);
    } else if (k < nfx + nfy) {
      d = 1;
      const int64_t m = k - nfx;
      x = (int)(m % b.X);
      const int64_t r = m / b.X;
      y = face_coord((int)(r % b.by), b.Y, B3Y);
      z = (int)(r / b.by);
    } else {
      d = 2;
      const int64_t m = k - nfx - nfy;
      x = (int)(m % b.X);
      const int64_t r = m / b.X;
      y = (int)(r % b.Y);
      z = face_coord((int)(r / b.Y), b.Z, B3Z);
    }
    const int64_t i = site3(b, x, y, z);
    const int s = spins[i];
    const uint4 wd = bond3_words(i, sweep, T, seed);
    int nx, ny, nz;
    if (bond3(spins, b, x, y, z, d, s, wd, Tp, nx, ny, nz)) {
      // the brick roots on the two ends (both edge roots)
      const Brick ka = brick_of(b, ((z / B3Z) * b.by + y / B3Y) * b.bx + x / B3X);
      const Brick kb = brick_of(b, ((nz / B3Z) * b.by + ny / B3Y) * b.bx + nx / B3X);
      const int ra = lroot[i], rb = lroot[site3(b, nx, ny, nz)];
      g_union(gpar, (int)brick_global(b, ka, ra), (int)brick_global(b, kb, rb), limit, err);
    }
  }
}

__global__ void __launch_bounds__(B3_THREADS, 6)
k3_flip(int8_t* __restrict__ spins, const uint16_t* __restrict__ lroot, int32_t* gpar,
        const uint32_t* __restrict__ edge_words, Box3 b, int q, uint64_t seed, const SwCtl* __restrict__ ctl,
        int limit, int* err) {
  __shared__ uint16_t rlist[B3_SITES];
  __shared__ uint8_t ns[B3_SITES];
  __shared__ uint32_t edge[B3_EDGE_WORDS];
  __shared__ int warp_cnt[B3_THREADS / 32];
  const Brick k = brick_of(b, blockIdx.x);
  const uint64_t sweep = ctl->sweep;
  for (int j = threadIdx.x; j < B3_EDGE_WORDS; j += B3_THREADS)
    edge[j] = edge_words[(int64_t)blockIdx.x * B3_EDGE_WORDS + j];
  const int lx = threadIdx.x & (B3X - 1), ly = threadIdx.x / B3X;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool col = lx < k.w && ly < k.h;
  // 1. brick roots of my sites (two per register), and which of them are roots
  uint32_t rr[B3Z / 2];
  uint32_t mine = 0;
#pragma unroll
  for (int lz = 0; lz < B3Z; ++lz) {
    uint32_t r = 0;
    if (col && lz < k.d) {
      r = lroot[site3(b, k.x0 + lx, k.y0 + ly, k.z0 + lz)];
      if ((int)r == (lz * B3Y + ly) * B3X + lx) mine |= 1u << lz;
    }
    if (lz & 1) rr[lz >> 1] |= r << 16;
    else rr[lz >> 1] = r;
  }
  // 2. the brick's root list
  const int cnt = __popc(mine);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_cnt[warp] = incl;
  __syncthreads();
  int base = 0, n_roots = 0;
#pragma unroll
  for (int j = 0; j < B3_THREADS / 32; ++j) {
    base += (j < warp) ? warp_cnt[j] : 0;
    n_roots += warp_cnt[j];
  }
  base += incl - cnt;
  while (mine) {
    const int lz = __ffs(mine) - 1;
    mine &= mine - 1;
    rlist[base++] = (uint16_t)((lz * B3Y + ly) * B3X + lx);
  }
  __syncthreads();
  // 3. one draw per brick root, keyed by its cluster's root; a thread takes
  //    its roots two at a time, their parent walks in lock step
  for (int j0 = threadIdx.x; j0 < n_roots; j0 += 2 * B3_THREADS) {
    int r[2], R[2];
    bool act[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int j = j0 + u * B3_THREADS;
      r[u] = j < n_roots ? (int)rlist[j] : 0;
      R[u] = (int)brick_global(b, k, r[u]);
      act[u] = j < n_roots && ((edge[r[u] >> 5] >> (r[u] & 31)) & 1u);
    }
    g_find_multi<2>(gpar, R, act, limit, err);
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (j0 + u * B3_THREADS < n_roots) ns[r[u]] = (uint8_t)state_of(draw((uint32_t)R[u], sweep, TAG_FLIP, seed).x, q);
  }
  __syncthreads();
  // 4. every site takes its brick root's state
  if (col) {
#pragma unroll
    for (int lz = 0; lz < B3Z; ++lz) {
      if (lz >= k.d) break;
      const int r = (rr[lz >> 1] >> (16 * (lz & 1))) & 0xFFFF;
      spins[site3(b, k.x0 + lx, k.y0 + ly, k.z0 + lz)] = (int8_t)ns[r];
    }
  }
}

constexpr int OBS3_THREADS = 256;

__global__ void __launch_bounds__(OBS3_THREADS)
k3_observe(const int8_t* __restrict__ spins, Box3 b, int q, SwCtl* __restrict__ ctl, int64_t* obs, int obs_cap) {
  __shared__ unsigned long long red[(1 + QREG) * (OBS3_THREADS / 32)];
  __shared__ int hist[128];
  for (int k = threadIdx.x; k < 128; k += OBS3_THREADS) hist[k] = 0;
  __syncthreads();
  long long n_eq = 0;
  int cnt[QREG];
#pragma unroll
  for (int k = 0; k < QREG; ++k) cnt[k] = 0;
  const int64_t n = (int64_t)b.X * b.Y * b.Z;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % b.X);
    const int64_t yz = i / b.X;
    const int y = (int)(yz % b.Y), z = (int)(yz / b.Y);
    const int s = spins[i];
    n_eq += spins[site3(b, x + 1 == b.X ? 0 : x + 1, y, z)] == s;
    n_eq += spins[site3(b, x, y + 1 == b.Y ? 0 : y + 1, z)] == s;
    n_eq += spins[site3(b, x, y, z + 1 == b.Z ? 0 : z + 1)] == s;
    if (q <= QREG) {
#pragma unroll
      for (int k = 0; k < QREG; ++k) cnt[k] += (s == k);
    } else {
      atomicAdd(&hist[s], 1);
    }
  }
  const uint64_t done = ctl->sweep - 1;
  unsigned long long* slot =
      reinterpret_cast<unsigned long long*>(obs + (int64_t)(done % (uint64_t)obs_cap) * (q + 1));
  add_observables<OBS3_THREADS>(n_eq, cnt, q, q <= QREG ? q : 0, slot, red, hist);
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->obs_done = (long long)done;
}

// End of a sweep: clear the observable slot of the sweep just done (the next
// sweep's k3_local, or k3_observe, fills it), then advance the counter.
__global__ void k3_advance(SwCtl* ctl, int64_t* obs, int obs_cap, int q) {
  const uint64_t s = ctl->sweep;
  if ((int)threadIdx.x <= q) obs[(int64_t)(s % (uint64_t)obs_cap) * (q + 1) + threadIdx.x] = 0;
  __syncthreads();
  if (threadIdx.x == 0) ctl->sweep = s + 1;
}

// Canonical labels of the last sweep: the cluster root of every site's brick root.
__global__ void k3_labels(const uint16_t* __restrict__ lroot, int32_t* gpar, const uint32_t* __restrict__ edge_words,
                          Box3 b, int32_t* out, int limit, int* err) {
  const int64_t n = b.n();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % b.X);
    const int64_t yz = i / b.X;
    const int y = (int)(yz % b.Y), z = (int)(yz / b.Y);
    const int t = ((z / B3Z) * b.by + y / B3Y) * b.bx + x / B3X;
    const Brick k = brick_of(b, t);
    const int r = lroot[i];
    int R = (int)brick_global(b, k, r);
    if ((edge_words[(int64_t)t * B3_EDGE_WORDS + (r >> 5)] >> (r & 31)) & 1u) R = g_find(gpar, R, limit, err);
    out[i] = R;
  }
}

// ---------------------------------------------------------------------------
Box3 make_box3(int X, int Y, int Z) {
  Box3 b;
  b.X = X;
  b.Y = Y;
  b.Z = Z;
  b.bx = (X + B3X - 1) / B3X;
  b.by = (Y + B3Y - 1) / B3Y;
  b.bz = (Z + B3Z - 1) / B3Z;
  return b;
}

static int limit3(const Box3& b) { return (int)std::min<int64_t>(b.n() + 64, (int64_t)1 << 30); }

static unsigned stride_blocks(int64_t n, int threads) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 16));
}

int64_t edge_words3(const Box3& b) { return b.n_bricks() * B3_EDGE_WORDS; }

int64_t scratch_ints3(const Box3& b) { return b.n_bricks() * 2 * TILE_SITES; }

cudaError_t launch_sweep3(int8_t* spins, uint16_t* lroot, int32_t* gpar, uint32_t* edge_words, int32_t* scratch,
                          const Box3& b, int q, uint64_t T, uint64_t seed, SwCtl* ctl, int64_t* obs, int obs_cap,
                          cudaStream_t st, cudaEvent_t* ev) {
  cudaError_t e;
  int* err = &ctl->err;
  if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
  k3_local<<<(unsigned)b.n_bricks(), B3_THREADS, 0, st>>>(spins, lroot, gpar, edge_words, scratch, b, q, T, seed,
                                                          ctl, obs, obs_cap, err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
  const int64_t faces = (b.bx > 1 ? (int64_t)b.bx * b.Y * b.Z : 0) + (b.by > 1 ? (int64_t)b.X * b.by * b.Z : 0) +
                        (b.bz > 1 ? (int64_t)b.X * b.Y * b.bz : 0);
  if (faces > 0) {
    k3_merge<<<stride_blocks(faces, 256), 256, 0, st>>>(spins, lroot, gpar, b, T, seed, ctl, limit3(b), err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
  k3_flip<<<(unsigned)b.n_bricks(), B3_THREADS, 0, st>>>(spins, lroot, gpar, edge_words, b, q, seed, ctl, limit3(b),
                                                         err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[3], st)) != cudaSuccess) return e;
  k3_advance<<<1, 128, 0, st>>>(ctl, obs, obs_cap, q);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[4], st)) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_observe3(const int8_t* spins, const Box3& b, int q, SwCtl* ctl, int64_t* obs, int obs_cap,
                            cudaStream_t st) {
  k3_observe<<<stride_blocks(b.n(), OBS3_THREADS), OBS3_THREADS, 0, st>>>(spins, b, q, ctl, obs, obs_cap);
  return cudaGetLastError();
}

cudaError_t launch_labels3(const uint16_t* lroot, int32_t* gpar, const uint32_t* edge_words, const Box3& b,
                           int32_t* out, int* err, cudaStream_t st) {
  k3_labels<<<stride_blocks(b.n(), 256), 256, 0, st>>>(lroot, gpar, edge_words, b, out, limit3(b), err);
  return cudaGetLastError();
}

}  // namespace swccl
