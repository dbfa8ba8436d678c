// swccl_device.cuh -- device helpers shared by the sm_103a kernels of libswccl.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the packed 2-bit bond
// mask, and lock-free union-find on shared and global memory.  The union
// rule hooks the larger root under the smaller one, so every tree's root is
// the minimum index in it; with labels initialised to their own index this
// makes the final root of a cluster its minimum site index, the canonical
// label that breadth-first search seeded in site order produces (Sec. II.B.1).
#pragma once
#include <cstdint>

#include "swccl_shared.h"

namespace swccl {

// ---------------------------------------------------------------------------
// Philox4x32-10.  Each round takes the two 32x32->64 products of the even
// counter words with the published multipliers; the high halves are mixed
// with the odd words and the round key, the key advances by the Weyl
// constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 ctr, uint32_t key_lo, uint32_t key_hi) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const unsigned long long pa = (unsigned long long)ctr.x * 0xD2511F53ull;
    const unsigned long long pb = (unsigned long long)ctr.z * 0xCD9E8D57ull;
    uint4 nxt;
    nxt.x = (uint32_t)(pb >> 32) ^ ctr.y ^ key_lo;
    nxt.y = (uint32_t)pb;
    nxt.z = (uint32_t)(pa >> 32) ^ ctr.w ^ key_hi;
    nxt.w = (uint32_t)pa;
    ctr = nxt;
    key_lo += 0x9E3779B9u;
    key_hi += 0xBB67AE85u;
  }
  return ctr;
}

// The ten round keys of a seed, computed once on the host and passed to a
// kernel by value (in constant memory, read directly by the XORs of each
// round), so that a kernel that makes many draws with one seed does not
// recompute the key schedule per call.
struct PhiloxKeys {
  uint32_t lo[10], hi[10];
};

__host__ __device__ inline PhiloxKeys philox_keys(uint64_t seed) {
  PhiloxKeys k;
  uint32_t lo = (uint32_t)seed, hi = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    k.lo[r] = lo;
    k.hi[r] = hi;
    lo += 0x9E3779B9u;
    hi += 0xBB67AE85u;
  }
  return k;
}

// A seed whose key schedule is computed in every call (batches: one seed
// per lattice, read from device memory).
struct SeedKey {
  uint32_t lo, hi;
};

// Philox4x32-10 with the round keys given: the same rounds as philox().
__device__ __forceinline__ uint4 philox_draw(uint4 ctr, const PhiloxKeys& k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const unsigned long long pa = (unsigned long long)ctr.x * 0xD2511F53ull;
    const unsigned long long pb = (unsigned long long)ctr.z * 0xCD9E8D57ull;
    uint4 nxt;
    nxt.x = (uint32_t)(pb >> 32) ^ ctr.y ^ k.lo[round];
    nxt.y = (uint32_t)pb;
    nxt.z = (uint32_t)(pa >> 32) ^ ctr.w ^ k.hi[round];
    nxt.w = (uint32_t)pa;
    ctr = nxt;
  }
  return ctr;
}

__device__ __forceinline__ uint4 philox_draw(uint4 ctr, const SeedKey& k) { return philox(ctr, k.lo, k.hi); }

__device__ __forceinline__ uint4 draw(uint32_t c0, uint64_t sweep, uint32_t tag, uint64_t seed) {
  return philox(make_uint4(c0, (uint32_t)sweep, (uint32_t)(sweep >> 32), tag), (uint32_t)seed,
                (uint32_t)(seed >> 32));
}

// New state of a cluster from a 32-bit word: floor(w q / 2^32).
__device__ __forceinline__ int state_of(uint32_t w, int q) {
  return (int)(((unsigned long long)w * (unsigned)q) >> 32);
}

// Two bits of site i in the packed mask: bit 0 east bond, bit 1 north bond.
__device__ __forceinline__ uint32_t site_bits(const uint8_t* mask, int64_t i) {
  return (uint32_t)(mask[i >> 2] >> (2 * (i & 3))) & 3u;
}

// Record a device-side failure without trapping: the first code wins.
__device__ __forceinline__ void set_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------------------
// Union-find in shared memory.  par[x] <= x always; roots satisfy par[r] == r.
// ---------------------------------------------------------------------------
// Path halving writes with atomicMin, never with a plain store: a plain
// store of a grandparent read earlier could overwrite a smaller pointer that
// another thread has written since (for instance the final root), undoing
// its compression.  With atomicMin every entry only ever decreases, and a
// root, the minimum of its tree, once written stays.  Walks at most `limit`
// steps (a tile tree has fewer nodes); on overrun the error word is set.
__device__ __forceinline__ int sm_find(volatile int* par, int x, int limit, int* err) {
  int p = par[x];
  int steps = 0;
  while (p != x) {
    const int gp = par[p];
    if (gp != p) atomicMin((int*)&par[x], gp);   // path halving
    x = p;
    p = gp;
    if (++steps > limit) { set_error(err, SW_ERR_STATE); return x; }
  }
  return x;
}

// The roots of two nodes at once: the walks run in lock step, so that their
// shared-memory loads overlap.  No path compression: inside a tile the
// unions keep trees shallow, and the atomics that compression needs cost
// more than the steps they save; the hooked roots are resolved at the end.
// Same step limit as sm_find.
__device__ __forceinline__ void sm_find2(volatile int* par, int& a, int& b, int limit, int* err) {
  int pa = par[a], pb = par[b];
  for (int steps = 0; pa != a || pb != b; ++steps) {
    if (pa != a) { a = pa; pa = par[a]; }
    if (pb != b) { b = pb; pb = par[b]; }
    if (steps > limit) { set_error(err, SW_ERR_STATE); return; }
  }
}

// Join the sets of a and b.  atomicMin hooks the larger root under the
// smaller; when the target was hooked meanwhile, the returned old parent is
// joined in the next round, so no link is lost.  Every round strictly lowers
// the larger operand, so at most `limit` rounds run.
__device__ __forceinline__ void sm_union(int* par, int a, int b, int limit, int* err) {
  volatile int* vp = par;
  for (int rounds = 0; rounds <= limit; ++rounds) {
    a = sm_find(vp, a, limit, err);
    b = sm_find(vp, b, limit, err);
    if (a == b) return;
    if (a > b) { const int t = a; a = b; b = t; }
    const int old = atomicMin(&par[b], a);
    if (old == b) return;
    b = old;
  }
  set_error(err, SW_ERR_STATE);
}

// As sm_union; a root that gets hooked is appended to a log of the hooked
// roots (count in *n_hooked), so that only hooked nodes need resolving
// later.  Entry k goes to hooked_fast[k] (shared memory) for k < fast_cap,
// else to hooked[k - fast_cap] (capacity cap).
__device__ __forceinline__ void sm_union_log(int* par, int a, int b, int limit, int* err, int* hooked_fast,
                                             int fast_cap, int* hooked, int* n_hooked, int cap) {
  volatile int* vp = par;
  for (int rounds = 0; rounds <= limit; ++rounds) {
    sm_find2(vp, a, b, limit, err);
    if (a == b) return;
    if (a > b) { const int t = a; a = b; b = t; }
    const int old = atomicMin(&par[b], a);
    if (old == b) {
      const int k = atomicAdd(n_hooked, 1);
      if (k < fast_cap) hooked_fast[k] = b;
      else if (k - fast_cap < cap) hooked[k - fast_cap] = b;
      else set_error(err, SW_ERR_STATE);
      return;
    }
    b = old;
  }
  set_error(err, SW_ERR_STATE);
}

// ---------------------------------------------------------------------------
// Union-find on a global int32 array (the label array itself: the entry of a
// tile root is its parent pointer).  Loads bypass L1 (ld.cg) because other
// SMs update the array during the merge.  Bounded by `limit` steps: on
// overrun the error word is set and the walk stops.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int g_load(const int* p) { return __ldcg(p); }

__device__ __forceinline__ int g_find(int* lab, int x, int limit, int* err) {
  int p = g_load(lab + x);
  int steps = 0;
  while (p != x) {
    const int gp = g_load(lab + p);
    if (gp != p) atomicMin(lab + x, gp);   // path halving, decreasing only (see sm_find)
    x = p;
    p = gp;
    if (++steps > limit) { set_error(err, SW_ERR_STATE); return x; }
  }
  return x;
}

// g_find of up to U nodes at once (those with act[u] set): the walks run in
// lock step so that their loads are in flight together.  x[u] is replaced by
// its root; same path halving and step limit as g_find.
template <int U>
__device__ __forceinline__ void g_find_multi(int* lab, int (&x)[U], const bool (&act)[U], int limit, int* err) {
  int p[U];
#pragma unroll
  for (int u = 0; u < U; ++u) p[u] = act[u] ? g_load(lab + x[u]) : x[u];
  for (int steps = 0;; ++steps) {
    int gp[U];
    bool more = false;
#pragma unroll
    for (int u = 0; u < U; ++u) gp[u] = (p[u] != x[u]) ? g_load(lab + p[u]) : p[u];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (p[u] != x[u]) {
        if (gp[u] != p[u]) atomicMin(lab + x[u], gp[u]);
        x[u] = p[u];
        p[u] = gp[u];
        more = true;
      }
    }
    if (!more) return;
    if (steps > limit) {
      set_error(err, SW_ERR_STATE);
      return;
    }
  }
}

// Join the sets of a and b on the global array, as sm_union (atomicMin
// hooking of the larger root under the smaller, a lost race retried with the
// returned parent).  The two finds of a round walk in lock step, so that
// their loads are in flight together.
__device__ __forceinline__ void g_union(int* lab, int a, int b, int limit, int* err) {
  for (int rounds = 0; rounds <= limit; ++rounds) {
    int x[2] = {a, b};
    const bool act[2] = {true, true};
    g_find_multi<2>(lab, x, act, limit, err);
    a = x[0];
    b = x[1];
    if (a == b) return;
    if (a > b) { const int t = a; a = b; b = t; }
    const int old = atomicMin(lab + b, a);
    if (old == b) return;
    b = old;
  }
  set_error(err, SW_ERR_STATE);
}

}  // namespace swccl
