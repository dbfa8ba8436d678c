// swccl_shared.h -- declarations shared by the host driver and the kernel
// translation units of libswccl (not part of the public ABI).
#pragma once
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/swccl.h"

namespace swccl {

// Philox tags (counter word 3).
enum : uint32_t { TAG_BOND = 0, TAG_FLIP = 1, TAG_INIT = 2, TAG_PERC = 3, TAG_SEED = 4, TAG_BOND3 = 5 };

// Tile of the local labeling phase: TILE_H rows x TILE_W columns, one CTA
// per tile with one warp per 32-column strip (LABEL_THREADS = TILE_W).
// TILE_H = 32 (one lane per row of a strip); TILE_W is 64, 128 or 256.  The
// library is built with TILE_W = 256; the batch libraries the autotuner
// chooses from are built with SWCCL_TILE_W = 64 and 128 (narrower tiles
// waste fewer threads on lattices that are not a multiple of 256 wide).
#ifndef SWCCL_TILE_W
#define SWCCL_TILE_W 256
#endif
constexpr int TILE_H = 32;
constexpr int TILE_W = SWCCL_TILE_W;
static_assert(TILE_W == 64 || TILE_W == 128 || TILE_W == 256, "tile width");
constexpr int TILE_W_LOG2 = TILE_W == 64 ? 6 : TILE_W == 128 ? 7 : 8;
constexpr int LABEL_THREADS = TILE_W;
// Resident CTAs per SM the labeling and flip kernels are built for (the same
// threads per SM at every tile width).
constexpr int LABEL_CTAS_PER_SM = 5 * 256 / TILE_W;
constexpr int FLIP_CTAS_PER_SM = 6 * 256 / TILE_W;

// Per-tile seam record written by the local labeling phase and read by the
// merge: labels of the four tile edges and the raw bond bits leaving the
// tile.  Labels are global site indices of tile-local roots.
struct SeamLayout {
  static constexpr int COL_L = 0;                       // int32[TILE_H]: column 0
  static constexpr int COL_R = COL_L + TILE_H;          // int32[TILE_H]: column w-1
  static constexpr int ROW_B = COL_R + TILE_H;          // int32[TILE_W]: row 0
  static constexpr int ROW_T = ROW_B + TILE_W;          // int32[TILE_W]: row h-1
  static constexpr int E_BITS = ROW_T + TILE_W;         // uint32[TILE_H/32]: east bits of column w-1
  static constexpr int N_BITS = E_BITS + TILE_H / 32;   // uint32[TILE_W/32]: north bits of row h-1
  static constexpr int INTS = N_BITS + TILE_W / 32;
};

// Geometry of one labeling problem (an H x W grid cut into tiles).
struct Grid {
  int H, W;
  int tiles_x, tiles_y;
  int periodic;
  __host__ __device__ int64_t n_sites() const { return (int64_t)H * W; }
  __host__ __device__ int n_tiles() const { return tiles_x * tiles_y; }
};

// Periodic X x Y x Z simple-cubic box and its bricks (k_cubic.cu).
struct Box3 {
  int X, Y, Z;
  int bx, by, bz;   // bricks per axis
  __host__ __device__ int64_t n() const { return (int64_t)X * Y * Z; }
  __host__ __device__ int64_t n_bricks() const { return (int64_t)bx * by * bz; }
};

inline Grid make_grid(int H, int W, int periodic) {
  Grid g;
  g.H = H;
  g.W = W;
  g.tiles_x = (W + TILE_W - 1) / TILE_W;
  g.tiles_y = (H + TILE_H - 1) / TILE_H;
  g.periodic = periodic ? 1 : 0;
  return g;
}

// Scratch of one labeling problem.
struct LabelScratch {
  int32_t* roots;        // n_tiles * TILE_H * TILE_W: pair lists, then tile-root lists
  int32_t* work;         // n_tiles * TILE_H * TILE_W: per-tile log of hooked roots
  int32_t* root_counts;  // n_tiles
  int32_t* seams;        // n_tiles * SeamLayout::INTS
  int* err;              // device status word
};

// Control block of a Swendsen-Wang chain, in device memory.
struct SwCtl {
  unsigned long long sweep;  // index of the sweep being computed
  long long obs_done;        // fused mode: last sweep whose observables k_observe completed (-1: none)
  int err;                   // first device-side failure (SW_ERR_*)
  int pad;
};

// One lattice as the fused kernels see it (also one replica of a batch).
struct SwRep {
  int8_t* spins;      // L*L int8
  uint16_t* lroot;    // L*L tile roots (local index)
  int32_t* gpar;      // L*L parent entries (only edge roots are used)
  int64_t* obs;       // observable ring: obs_cap x (1 + q)
  LabelScratch s;     // per-tile pair lists, hook logs, seam records, status word
  Grid g;             // L x L, periodic
  uint64_t T, seed;
  int q;
  int tile0;          // first global tile of this lattice in a batch
};

// Control block of a batch of chains (all replicas advance together).
struct BatchCtl {
  unsigned long long sweep;
  long long obs_done;
  int err;
  unsigned int bar_count;    // grid barrier of the persistent kernel
  unsigned int bar_gen;
  int pad;
};

// What the batched kernels read: replica table and tile -> replica map, in
// device memory.
struct BatchView {
  const SwRep* reps;
  const int* tile_rep;
  int n_reps;
  int n_tiles;
  int obs_cap;
  int limit;          // union-find step bound: largest replica's sites + 64
};

// One grid of a batched labeling call.
struct CclJob {
  const uint8_t* mask;
  int32_t* labels;
  LabelScratch s;
  Grid g;
  int tile0;          // first global tile of this grid
  int pad;
};

// Up to CCL_PARAM_JOBS grids of a batched labeling call, passed to the
// kernels by value (no host-to-device copy, so the call never waits): the
// tile range of grid j ends at tile_end[j].
constexpr int CCL_PARAM_JOBS = 32;
struct CclBatchView {
  CclJob jobs[CCL_PARAM_JOBS];
  int tile_end[CCL_PARAM_JOBS];
  int n_jobs;
  int n_tiles;
  int limit;          // union-find step bound: largest grid's sites + 64
  int pad;
};

// Bytes of LabelScratch for a grid (each part 256-byte aligned).
int64_t label_scratch_bytes(const Grid& g);
LabelScratch carve_label_scratch(const Grid& g, void* base, int* err);

// ---------------------------------------------------------------------------
// Launchers (each enqueues on `st`, returns the launch error).
// ---------------------------------------------------------------------------
cudaError_t launch_init_spins(int8_t* spins, int L, int q, uint64_t seed, int hot, cudaStream_t st);
cudaError_t launch_activate(const int8_t* spins, uint8_t* mask, int L, uint64_t T, uint64_t seed,
                            const SwCtl* ctl, int64_t* obs_ring, int obs_cap, int q,
                            cudaStream_t st);
cudaError_t launch_perc_mask(uint8_t* mask, int H, int W, uint64_t k, cudaStream_t st);
cudaError_t launch_pixel_bonds(const uint8_t* px, uint8_t* mask, int H, int W, int periodic,
                               cudaStream_t st);
cudaError_t launch_philox_probe(long long calls_per_thread, int blocks, uint32_t* sink, cudaStream_t st);
cudaError_t launch_check_spins(const int8_t* spins, int64_t n, int q, int* err, cudaStream_t st);
// dst = src (device memory) if ok_flag is null or *ok_flag == 0; an SM copy.
cudaError_t launch_copy_if(int8_t* dst, const int8_t* src, int64_t n, const int* ok_flag, cudaStream_t st);
cudaError_t launch_init_spins_n(int8_t* spins, int64_t n, int q, uint64_t seed, int hot, cudaStream_t st);
// Simple-cubic sweep (k_cubic.cu).  ev, if not null, receives five events:
// before the local step, merge, flip, advance, and after the advance.  The
// observables of a sweep are counted by the next sweep's local step, or by
// launch_observe3 (the last sweep, when they are read).
Box3 make_box3(int X, int Y, int Z);
int64_t edge_words3(const Box3& b);     // uint32 words of edge-root bits
int64_t scratch_ints3(const Box3& b);   // int32 words of labeling scratch (pair lists, hook logs)
cudaError_t launch_sweep3(int8_t* spins, uint16_t* lroot, int32_t* gpar, uint32_t* edge_words, int32_t* scratch,
                          const Box3& b, int q, uint64_t T, uint64_t seed, SwCtl* ctl, int64_t* obs, int obs_cap,
                          cudaStream_t st, cudaEvent_t* ev);
cudaError_t launch_observe3(const int8_t* spins, const Box3& b, int q, SwCtl* ctl, int64_t* obs, int obs_cap,
                            cudaStream_t st);
cudaError_t launch_labels3(const uint16_t* lroot, int32_t* gpar, const uint32_t* edge_words, const Box3& b,
                           int32_t* out, int* err, cudaStream_t st);

cudaError_t launch_tile_label(const uint8_t* mask, int32_t* labels, const Grid& g,
                              const LabelScratch& s, cudaStream_t st);
cudaError_t launch_merge(int32_t* labels, const Grid& g, const LabelScratch& s, cudaStream_t st);
// Root compression; when `spins` is non-null also draws each final root's
// new state (FLIP tag, sweep from ctl) into spins[root].
cudaError_t launch_root_compress(int32_t* labels, const Grid& g, const LabelScratch& s,
                                 int8_t* spins, int q, uint64_t seed, const SwCtl* ctl,
                                 cudaStream_t st);
cudaError_t launch_site_compress(int32_t* labels, int64_t n_sites, cudaStream_t st);
// The stand-alone labeling of one grid: local labeling, seam merge, final labels.
cudaError_t launch_ccl(const uint8_t* mask, int32_t* labels, const Grid& g, const LabelScratch& s, cudaStream_t st);

cudaError_t launch_flip(int8_t* spins, const int32_t* labels, int L, int q, const SwCtl* ctl,
                        int64_t* obs_ring, int obs_cap, cudaStream_t st);
cudaError_t launch_advance(SwCtl* ctl, cudaStream_t st);

// Fused sweep (activation inside labeling; no mask or int32 labels in HBM).
cudaError_t launch_sw_label(const int8_t* spins, uint16_t* lroot, int32_t* gpar, const Grid& g,
                            const LabelScratch& s, int q, uint64_t T, uint64_t seed, const SwCtl* ctl,
                            int64_t* obs, int obs_cap, cudaStream_t st);
cudaError_t launch_sw_flip(int8_t* spins, const uint16_t* lroot, int32_t* gpar, const Grid& g,
                           const LabelScratch& s, int q, uint64_t seed, const SwCtl* ctl, cudaStream_t st);
cudaError_t launch_observe(const int8_t* spins, int L, int q, SwCtl* ctl, int64_t* obs, int obs_cap,
                           cudaStream_t st);
cudaError_t launch_advance_fused(SwCtl* ctl, int64_t* obs, int obs_cap, int q, cudaStream_t st);
// Few-cluster update: bytes of the seed-selection bit array of n sites, the
// selection (clears the array, then marks the seeded clusters' roots), and
// the flip of the selected clusters.
inline int64_t few_sel_bytes(int64_t n_sites) { return (n_sites + 31) / 32 * 4; }
cudaError_t launch_few_select(const uint16_t* lroot, int32_t* gpar, const Grid& g, const LabelScratch& s,
                              uint64_t seed, int ell, uint32_t* sel, const SwCtl* ctl, cudaStream_t st);
cudaError_t launch_sw_flip_few(int8_t* spins, const uint16_t* lroot, int32_t* gpar, const Grid& g,
                               const LabelScratch& s, int q, uint64_t seed, const uint32_t* sel, uint64_t P,
                               const SwCtl* ctl, cudaStream_t st);

// Batched chains (k_batch.cu).
cudaError_t launch_batch_label(const BatchView& b, BatchCtl* ctl, cudaStream_t st);
cudaError_t launch_batch_merge(const BatchView& b, cudaStream_t st);
cudaError_t launch_batch_flip(const BatchView& b, BatchCtl* ctl, cudaStream_t st);
cudaError_t launch_batch_advance(const BatchView& b, BatchCtl* ctl, cudaStream_t st);
cudaError_t launch_batch_observe(const BatchView& b, BatchCtl* ctl, cudaStream_t st);
// One persistent cooperative launch for the whole sweep; `blocks` CTAs; a
// grid-barrier wait gives up after limit_cycles of clock64().
cudaError_t launch_batch_persistent(const BatchView& b, BatchCtl* ctl, int blocks, long long limit_cycles,
                                    cudaStream_t st);
// Largest number of co-resident CTAs of the persistent kernel per SM.
int batch_persistent_blocks_per_sm();

// Batched labeling (k_ccl_batch.cu): the four steps over all tiles of all grids.
cudaError_t launch_ccl_batch(const CclBatchView& v, cudaStream_t st);

// Host helpers of the C ABI: set this thread's sw_last_error() message and
// return `code`; device address of the stand-alone labeling status word on
// the current device (nullptr on failure).
int set_last_error(int code, const std::string& msg);
int* ccl_status_word();

}  // namespace swccl
