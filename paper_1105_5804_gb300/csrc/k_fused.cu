// k_fused.cu -- the Swendsen-Wang sweep with activation fused into labeling.
//
// The staged sweep writes the bond mask and an int32 label per site to HBM
// and reads them back.  Because the bond draws are counter-based (Philox
// keyed by seed, sweep and site), the bonds can be drawn where they are
// consumed instead.  A fused sweep is three kernels:
//
//  k_sw_label  one CTA per tile: reads the tile's spins (plus the north row
//              and east column beyond it), draws the tile's bonds (rule of
//              Eq. 7, Sec. II.A) into shared memory, labels the tile with
//              the engine of tile_engine.cuh, and writes each site's tile
//              root as a 16-bit local index (the root's own entry flagged
//              if its component touches the tile edge), the seam record of
//              the tile, and a parent entry gpar[r] = r for every tile root
//              r on the tile's edge.  It also counts, for the spins it read
//              (the result of the previous sweep), the bonds joining equal
//              spins and the sites per state, the observables of that sweep.
//  k_merge     (k_label.cu) joins tile roots across seams on gpar.
//  k_sw_flip   one CTA per tile: lists the tile's roots; a flagged root
//              (on the tile edge) looks up its final root R in gpar, any
//              other root is its own final root; each root draws its
//              cluster's new state once
//              (FLIP draw keyed by R, Sec. II.D) and every site copies the
//              state of its tile root.  When every tile is whole (L a
//              multiple of TILE_W), k_sw_flip_whole does the same without
//              bounds checks, reading a thread's tile roots twice through L2
//              instead of holding them in registers across the draws.
//
// HBM traffic per site: spins read 1 B, 16-bit roots written and read 4 B,
// spins written 1 B, plus seam records and edge-root entries.
//
// The few-cluster update (Sec. III, variant (c)) shares k_sw_label and
// k_merge; between the merge and the flip, k_few_select marks the global
// roots of the clusters holding the ell^2 seeds in a bit array, and
// k_sw_flip_few moves only those clusters (each with probability p_flip).
#include "fused_tile.cuh"

namespace swccl {

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(LABEL_THREADS, LABEL_CTAS_PER_SM)
k_sw_label(SwRep R, const SwCtl* __restrict__ ctl, int obs_cap, const __grid_constant__ PhiloxKeys keys) {
  __shared__ LabelTileSmem ls;
  const uint64_t sweep = ctl->sweep;
  const bool do_obs = sweep > 0 && ctl->obs_done != (long long)(sweep - 1);
  sw_label_tile(R, blockIdx.x, sweep, do_obs, obs_cap, ls, keys);
}

__global__ void __launch_bounds__(LABEL_THREADS, FLIP_CTAS_PER_SM)
k_sw_flip(SwRep R, const SwCtl* __restrict__ ctl, int limit, const __grid_constant__ PhiloxKeys keys) {
  __shared__ FlipTileSmem fs;
  sw_flip_tile(R, blockIdx.x, ctl->sweep, limit, fs, keys);
}

// k_sw_flip when every tile of the lattice is whole (selected on the host).
__global__ void __launch_bounds__(LABEL_THREADS, FLIP_CTAS_PER_SM)
k_sw_flip_whole(SwRep R, const SwCtl* __restrict__ ctl, int limit, const __grid_constant__ PhiloxKeys keys) {
  __shared__ FlipTileSmem fs;
  sw_flip_whole_tile(R, blockIdx.x, ctl->sweep, limit, fs, keys);
}

__global__ void __launch_bounds__(LABEL_THREADS, FLIP_CTAS_PER_SM)
k_sw_flip_few(SwRep R, const SwCtl* __restrict__ ctl, int limit, const uint32_t* __restrict__ sel, uint64_t P,
              const __grid_constant__ PhiloxKeys keys) {
  __shared__ FlipTileSmem fs;
  sw_flip_tile<true>(R, blockIdx.x, ctl->sweep, limit, fs, keys, sel, P);
}

constexpr int SELECT_THREADS = 256;

__global__ void __launch_bounds__(SELECT_THREADS)
k_few_select(SwRep R, const SwCtl* __restrict__ ctl, int ell, uint32_t* sel, int limit) {
  const int64_t b = blockIdx.x * (int64_t)SELECT_THREADS + threadIdx.x;   // one thread per seed
  if (b < (int64_t)ell * ell) few_select_seed(R, ell, b, ctl->sweep, sel, limit);
}

// ---------------------------------------------------------------------------
// Observables of the current spins (bonds joining equal spins, sites per
// state), added to the slot of sweep `ctl->sweep - 1`, which is then marked
// done so the next sweep's k_sw_label does not count it again.
constexpr int OBS_THREADS = 256;
constexpr int OBS_ROWS = 16;

__global__ void __launch_bounds__(OBS_THREADS)
k_observe(const int8_t* __restrict__ spins, int L, int q, SwCtl* __restrict__ ctl, int64_t* __restrict__ obs,
          int obs_cap) {
  __shared__ unsigned long long red[(1 + QREG) * (OBS_THREADS / 32)];
  __shared__ int hist[128];
  for (int k = threadIdx.x; k < 128; k += OBS_THREADS) hist[k] = 0;
  __syncthreads();
  const uint64_t done = ctl->sweep - 1;
  long long n_eq = 0;
  int cnt[QREG];
#pragma unroll
  for (int k = 0; k < QREG; ++k) cnt[k] = 0;
  const int xq = blockIdx.x * OBS_THREADS + threadIdx.x;
  if (xq < (L >> 2)) {
    const int x = xq << 2;
    const int xe = (x + 4 == L) ? 0 : x + 4;
    const int y1 = min((int)blockIdx.y * OBS_ROWS + OBS_ROWS, L);
    for (int y = blockIdx.y * OBS_ROWS; y < y1; ++y) {
      const int yn = (y + 1 == L) ? 0 : y + 1;
      const uint32_t cur = *reinterpret_cast<const uint32_t*>(spins + (int64_t)y * L + x);
      const uint32_t nor = *reinterpret_cast<const uint32_t*>(spins + (int64_t)yn * L + x);
      const uint32_t e = (cur >> 8) | ((uint32_t)(uint8_t)spins[(int64_t)y * L + xe] << 24);
      n_eq += __popc(eq4(cur, e)) + __popc(eq4(cur, nor));
      if (q <= QREG) {
#pragma unroll
        for (int k = 0; k < QREG; ++k)
          if (k < q) cnt[k] += __popc(eq4(cur, 0x01010101u * (uint32_t)k));
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) atomicAdd(&hist[(cur >> (8 * j)) & 0xFF], 1);
      }
    }
  }
  unsigned long long* oslot =
      reinterpret_cast<unsigned long long*>(obs + (int64_t)(done % (uint64_t)obs_cap) * (q + 1));
  add_observables<OBS_THREADS>(n_eq, cnt, q, q <= QREG ? q : 0, oslot, red, hist);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) ctl->obs_done = (long long)done;
}

// End of a fused sweep: clear the observable slot of the sweep just done
// (the next sweep's k_sw_label, or k_observe, fills it) and advance.
__global__ void k_advance_fused(SwCtl* ctl, int64_t* obs, int obs_cap, int q) {
  const uint64_t s = ctl->sweep;
  if ((int)threadIdx.x <= q) obs[(int64_t)(s % (uint64_t)obs_cap) * (q + 1) + threadIdx.x] = 0;
  __syncthreads();
  if (threadIdx.x == 0) ctl->sweep = s + 1;
}

// ---------------------------------------------------------------------------
SwRep make_rep(int8_t* spins, uint16_t* lroot, int32_t* gpar, int64_t* obs, const Grid& g,
               const LabelScratch& s, int q, uint64_t T, uint64_t seed) {
  SwRep R;
  R.spins = spins;
  R.lroot = lroot;
  R.gpar = gpar;
  R.obs = obs;
  R.s = s;
  R.g = g;
  R.T = T;
  R.seed = seed;
  R.q = q;
  R.tile0 = 0;
  return R;
}

cudaError_t launch_sw_label(const int8_t* spins, uint16_t* lroot, int32_t* gpar, const Grid& g,
                            const LabelScratch& s, int q, uint64_t T, uint64_t seed, const SwCtl* ctl,
                            int64_t* obs, int obs_cap, cudaStream_t st) {
  const SwRep R = make_rep(const_cast<int8_t*>(spins), lroot, gpar, obs, g, s, q, T, seed);
  k_sw_label<<<g.n_tiles(), LABEL_THREADS, 0, st>>>(R, ctl, obs_cap, philox_keys(seed));
  return cudaGetLastError();
}

cudaError_t launch_sw_flip(int8_t* spins, const uint16_t* lroot, int32_t* gpar, const Grid& g,
                           const LabelScratch& s, int q, uint64_t seed, const SwCtl* ctl, cudaStream_t st) {
  const int limit = (int)std::min<int64_t>(g.n_sites() + 64, (int64_t)1 << 30);
  const SwRep R = make_rep(spins, const_cast<uint16_t*>(lroot), gpar, nullptr, g, s, q, 0, seed);
  if (g.W % TILE_W == 0 && g.H % TILE_H == 0 && g.W % 8 == 0)   // every tile whole
    k_sw_flip_whole<<<g.n_tiles(), LABEL_THREADS, 0, st>>>(R, ctl, limit, philox_keys(seed));
  else
    k_sw_flip<<<g.n_tiles(), LABEL_THREADS, 0, st>>>(R, ctl, limit, philox_keys(seed));
  return cudaGetLastError();
}

// The same for L % 16 == 0 at HBM speed: a thread owns 16 columns (one
// 16-byte word per row) of a band of OBS16_ROWS rows and keeps the row it
// just read for the next row's north bonds, so every row is read once; the
// east neighbour of its last column is the next lane's first byte.
constexpr int OBS16_ROWS = 32;

__global__ void __launch_bounds__(OBS_THREADS)
k_observe16(const int8_t* __restrict__ spins, int L, int q, SwCtl* __restrict__ ctl, int64_t* __restrict__ obs,
            int obs_cap) {
  __shared__ unsigned long long red[(1 + QREG) * (OBS_THREADS / 32)];
  __shared__ int hist[128];
  for (int k = threadIdx.x; k < 128; k += OBS_THREADS) hist[k] = 0;
  __syncthreads();
  const uint64_t done = ctl->sweep - 1;
  long long n_eq = 0;
  int cnt[QREG];
#pragma unroll
  for (int k = 0; k < QREG; ++k) cnt[k] = 0;
  const int lane = threadIdx.x & 31;
  const int x = (blockIdx.x * OBS_THREADS + threadIdx.x) * 16;
  const bool active = x < L;
  const int xe = (x + 16 >= L) ? 0 : x + 16;        // east neighbour column of my last site
  const int y0 = blockIdx.y * OBS16_ROWS, y1 = min(y0 + OBS16_ROWS, L);
  auto row = [&](int y) -> uint4 {
    return active ? *reinterpret_cast<const uint4*>(spins + (int64_t)y * L + x) : make_uint4(0u, 0u, 0u, 0u);
  };
  uint4 cur = row(y0);
  for (int y = y0; y < y1; ++y) {
    const uint4 nor = row(y + 1 == L ? 0 : y + 1);
    // first byte east of my 16 columns: the next lane's, or (last lane / row end) a load
    const uint32_t from_next = __shfl_down_sync(FULL, cur.x, 1) & 0xFFu;
    const bool own_load = lane == 31 || xe == 0 || x + 16 >= L;
    const uint32_t east_b = own_load ? (active ? (uint32_t)(uint8_t)spins[(int64_t)y * L + xe] : 0u) : from_next;
    if (active) {
      const uint32_t w[4] = {cur.x, cur.y, cur.z, cur.w}, nw[4] = {nor.x, nor.y, nor.z, nor.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t next = k < 3 ? w[k + 1] : east_b;
        n_eq += __popc(eq4(w[k], (w[k] >> 8) | (next << 24))) + __popc(eq4(w[k], nw[k]));
        if (q == 2) {
          const int ones = __popc(w[k] & 0x01010101u);
          cnt[1] += ones;
          cnt[0] += 4 - ones;
        } else if (q <= QREG) {
#pragma unroll
          for (int c = 0; c < QREG; ++c)
            if (c < q) cnt[c] += __popc(eq4(w[k], 0x01010101u * (uint32_t)c));
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) atomicAdd(&hist[(w[k] >> (8 * j)) & 0xFF], 1);
        }
      }
    }
    cur = nor;
  }
  unsigned long long* oslot =
      reinterpret_cast<unsigned long long*>(obs + (int64_t)(done % (uint64_t)obs_cap) * (q + 1));
  add_observables<OBS_THREADS>(n_eq, cnt, q, q <= QREG ? q : 0, oslot, red, hist);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) ctl->obs_done = (long long)done;
}

cudaError_t launch_observe(const int8_t* spins, int L, int q, SwCtl* ctl, int64_t* obs, int obs_cap,
                           cudaStream_t st) {
  if (L % 16 == 0) {
    dim3 grid((unsigned)((L / 16 + OBS_THREADS - 1) / OBS_THREADS), (unsigned)((L + OBS16_ROWS - 1) / OBS16_ROWS));
    k_observe16<<<grid, OBS_THREADS, 0, st>>>(spins, L, q, ctl, obs, obs_cap);
  } else {
    dim3 grid((unsigned)((L / 4 + OBS_THREADS - 1) / OBS_THREADS), (unsigned)((L + OBS_ROWS - 1) / OBS_ROWS));
    k_observe<<<grid, OBS_THREADS, 0, st>>>(spins, L, q, ctl, obs, obs_cap);
  }
  return cudaGetLastError();
}

cudaError_t launch_few_select(const uint16_t* lroot, int32_t* gpar, const Grid& g, const LabelScratch& s,
                              uint64_t seed, int ell, uint32_t* sel, const SwCtl* ctl, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(sel, 0, few_sel_bytes(g.n_sites()), st);
  if (e != cudaSuccess) return e;
  const int limit = (int)std::min<int64_t>(g.n_sites() + 64, (int64_t)1 << 30);
  const SwRep R = make_rep(nullptr, const_cast<uint16_t*>(lroot), gpar, nullptr, g, s, 2, 0, seed);
  const int64_t seeds = (int64_t)ell * ell;
  const int64_t blocks = (seeds + SELECT_THREADS - 1) / SELECT_THREADS;
  k_few_select<<<(unsigned)blocks, SELECT_THREADS, 0, st>>>(R, ctl, ell, sel, limit);
  return cudaGetLastError();
}

cudaError_t launch_sw_flip_few(int8_t* spins, const uint16_t* lroot, int32_t* gpar, const Grid& g,
                               const LabelScratch& s, int q, uint64_t seed, const uint32_t* sel, uint64_t P,
                               const SwCtl* ctl, cudaStream_t st) {
  const int limit = (int)std::min<int64_t>(g.n_sites() + 64, (int64_t)1 << 30);
  const SwRep R = make_rep(spins, const_cast<uint16_t*>(lroot), gpar, nullptr, g, s, q, 0, seed);
  k_sw_flip_few<<<g.n_tiles(), LABEL_THREADS, 0, st>>>(R, ctl, limit, sel, P, philox_keys(seed));
  return cudaGetLastError();
}

cudaError_t launch_advance_fused(SwCtl* ctl, int64_t* obs, int obs_cap, int q, cudaStream_t st) {
  k_advance_fused<<<1, 128, 0, st>>>(ctl, obs, obs_cap, q);
  return cudaGetLastError();
}

}  // namespace swccl
