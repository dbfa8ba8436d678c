// k_cubic.cu -- the Swendsen-Wang sweep on the periodic simple-cubic lattice.
//
// The paper develops the method on the square lattice and notes that the
// three-dimensional case follows the same steps with six neighbours
// (Secs. II and II.B).  Box X x Y x Z, site i = (z Y + y) X + x; each site
// owns its bonds to the +x, +y and +z neighbours (periodic), drawn from one
// Philox call per site (tag BOND3, counter (i, sweep), word = direction) and
// open iff the two spins are equal and the word is below T (Eq. 7).
//
// One sweep is four kernels:
//  k3_local    one CTA per 32 x 8 x 16 brick: draws the bonds of its sites,
//              joins those inside the brick with union-find in shared memory
//              (larger root hooked under the smaller, so a brick root is the
//              brick component's smallest index), and writes for every site
//              gpar[i] = global index of its brick root;
//  k3_merge    one thread per site on a brick face: redraws the face bond
//              (the draws are counter-based) and, if open, joins the two
//              sides on gpar with global atomics;
//  k3_flip     every site finds its cluster root R on gpar and takes the
//              state F_q of the FLIP draw keyed by R (Sec. II.D);
//  k3_observe  bonds joining equal spins and sites per state of the new
//              spins, into the sweep's observable slot; then k3_advance.
// HBM traffic per site: spins read 1 B, gpar written 4 B (local), gpar read
// 4 B and spins written 1 B (flip), spins read 1 B (observe), plus the face
// sites' neighbours and the root chains.
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

__global__ void __launch_bounds__(B3_THREADS)
k3_local(const int8_t* __restrict__ spins, int32_t* __restrict__ gpar, Box3 b, uint64_t T, uint64_t seed,
         const SwCtl* __restrict__ ctl, int* err) {
  __shared__ int par[B3_SITES];
  const int t = blockIdx.x;
  const int tbx = t % b.bx, tby = (t / b.bx) % b.by, tbz = t / (b.bx * b.by);
  const int x0 = tbx * B3X, y0 = tby * B3Y, z0 = tbz * B3Z;
  const int w = min(B3X, b.X - x0), h = min(B3Y, b.Y - y0), dpt = min(B3Z, b.Z - z0);
  for (int l = threadIdx.x; l < B3_SITES; l += B3_THREADS) par[l] = l;
  __syncthreads();
  const uint64_t sweep = ctl->sweep;
  const uint64_t Tp = T >= (1ull << 32) ? ~0ull : T;   // p = 1: every equal bond opens
  const int lx = threadIdx.x & (B3X - 1), ly = threadIdx.x / B3X;
  if (lx < w && ly < h) {
    for (int lz = 0; lz < dpt; ++lz) {
      const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
      const int64_t i = site3(b, x, y, z);
      const int s = spins[i];
      const uint4 wd = bond3_words(i, sweep, T, seed);
      const int l = (lz * B3Y + ly) * B3X + lx;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        int nx, ny, nz;
        if (!bond3(spins, b, x, y, z, d, s, wd, Tp, nx, ny, nz)) continue;
        if (nx / B3X != tbx || ny / B3Y != tby || nz / B3Z != tbz) continue;   // face bond: k3_merge
        sm_union(par, l, ((nz - z0) * B3Y + (ny - y0)) * B3X + (nx - x0), B3_SITES, err);
      }
    }
  }
  __syncthreads();
  if (lx < w && ly < h) {
    for (int lz = 0; lz < dpt; ++lz) {
      const int l = (lz * B3Y + ly) * B3X + lx;
      const int r = sm_find(par, l, B3_SITES, err);
      const int rx = r % B3X, ry = (r / B3X) % B3Y, rz = r / (B3X * B3Y);
      gpar[site3(b, x0 + lx, y0 + ly, z0 + lz)] = (int32_t)site3(b, x0 + rx, y0 + ry, z0 + rz);
    }
  }
}

// Face sites: for axis d, the coordinates whose +d neighbour lies in another
// brick (none when one brick spans the axis).
__device__ __forceinline__ int face_coord(int k, int extent, int brick) {
  return min((k + 1) * brick, extent) - 1;
}

__global__ void k3_merge(const int8_t* __restrict__ spins, int32_t* gpar, Box3 b, uint64_t T, uint64_t seed,
                         const SwCtl* __restrict__ ctl, int limit, int* err) {
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
    if (bond3(spins, b, x, y, z, d, s, wd, Tp, nx, ny, nz))
      g_union(gpar, (int)i, (int)site3(b, nx, ny, nz), limit, err);
  }
}

__global__ void k3_flip(int8_t* __restrict__ spins, int32_t* gpar, int64_t n, int q, uint64_t seed,
                        const SwCtl* __restrict__ ctl, int limit, int* err) {
  const uint64_t sweep = ctl->sweep;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int R = g_find(gpar, (int)i, limit, err);
    spins[i] = (int8_t)state_of(draw((uint32_t)R, sweep, TAG_FLIP, seed).x, q);
  }
}

constexpr int OBS3_THREADS = 256;

__global__ void __launch_bounds__(OBS3_THREADS)
k3_observe(const int8_t* __restrict__ spins, Box3 b, int q, const SwCtl* __restrict__ ctl, int64_t* obs,
           int obs_cap) {
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
  unsigned long long* slot =
      reinterpret_cast<unsigned long long*>(obs + (int64_t)(ctl->sweep % (uint64_t)obs_cap) * (q + 1));
  add_observables<OBS3_THREADS>(n_eq, cnt, q, q <= QREG ? q : 0, slot, red, hist);
}

// Zero the next sweep's observable slot, then advance the sweep counter.
__global__ void k3_advance(SwCtl* ctl, int64_t* obs, int obs_cap, int q) {
  const uint64_t s = ctl->sweep + 1;
  if ((int)threadIdx.x <= q) obs[(int64_t)(s % (uint64_t)obs_cap) * (q + 1) + threadIdx.x] = 0;
  __syncthreads();
  if (threadIdx.x == 0) ctl->sweep = s;
}

__global__ void k3_labels(int32_t* gpar, int32_t* out, int64_t n, int limit, int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = g_find(gpar, (int)i, limit, err);
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

cudaError_t launch_sweep3(int8_t* spins, int32_t* gpar, const Box3& b, int q, uint64_t T, uint64_t seed, SwCtl* ctl,
                          int64_t* obs, int obs_cap, cudaStream_t st, cudaEvent_t* ev) {
  cudaError_t e;
  int* err = &ctl->err;
  const int64_t n = b.n();
  if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
  k3_local<<<(unsigned)b.n_bricks(), B3_THREADS, 0, st>>>(spins, gpar, b, T, seed, ctl, err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
  const int64_t faces = (b.bx > 1 ? (int64_t)b.bx * b.Y * b.Z : 0) + (b.by > 1 ? (int64_t)b.X * b.by * b.Z : 0) +
                        (b.bz > 1 ? (int64_t)b.X * b.Y * b.bz : 0);
  if (faces > 0) {
    k3_merge<<<stride_blocks(faces, 256), 256, 0, st>>>(spins, gpar, b, T, seed, ctl, limit3(b), err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
  k3_flip<<<stride_blocks(n, 256), 256, 0, st>>>(spins, gpar, n, q, seed, ctl, limit3(b), err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[3], st)) != cudaSuccess) return e;
  k3_observe<<<stride_blocks(n, OBS3_THREADS), OBS3_THREADS, 0, st>>>(spins, b, q, ctl, obs, obs_cap);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k3_advance<<<1, 128, 0, st>>>(ctl, obs, obs_cap, q);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[4], st)) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_labels3(int32_t* gpar, int32_t* out, const Box3& b, int* err, cudaStream_t st) {
  k3_labels<<<stride_blocks(b.n(), 256), 256, 0, st>>>(gpar, out, b.n(), limit3(b), err);
  return cudaGetLastError();
}

}  // namespace swccl
