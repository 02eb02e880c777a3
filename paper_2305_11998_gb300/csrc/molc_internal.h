// Internal declarations shared by the host planner (molc_host.cpp) and the CUDA kernels (molc_kernels.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "molc.h"

namespace molc {

constexpr int kMaxPolarFP32 = 8;     // FP32 sweep: polar cosines per azimuth handled by one half-warp
constexpr int kOutputs = 6;          // D, Fx, Fy, Nxx, Nxy, Nyy accumulators per (cell, group)
constexpr int kGatherPad = 4;        // FP32 moments: each cell's entry list is padded to a multiple of this
constexpr int kPartEntries = 256;    // FP32 moments: entries one thread sums (longer cell lists are split)
constexpr int kSweepBlock = 128;     // FP32 sweep: work items (threads) per block = width of a state bundle
constexpr size_t kMaxGatherSmem = 200 * 1024;  // FP32 moments: per-pair coefficient table in shared memory

// Device status bits (the first one set wins in molc_device_status).
constexpr int kStatusNonfinite = 1;
constexpr int kStatusRange = 2;
// FP32 states work in units scaled by 2^k with max B * 2^k in [2^99, 2^100); inputs above 2^124 are rejected.
constexpr int kScaleTargetExp = 100;
constexpr double kScaledMax = 21267647932558653966460912964485513216.0;  // 2^124

// One characteristic (track) of an azimuth pair; the + sense walks its segments forward, the - sense backward.
struct TrackDev {
  int64_t seg_off;      // first segment in the track-segment arrays
  int nseg;
  int pair;             // azimuth pair
  int entry_plus;       // edge the + sense enters through (0 L, 1 R, 2 B, 3 T)
  int entry_minus;      // edge the - sense enters through (= exit edge of the + sense)
  int64_t canon_plus;   // offset of this track's segments within the + sense direction's canonical block
  int64_t canon_minus;  // same for the - sense (tracks are in reverse order there)
  int pos[2];           // FP32 work items: position of the (track, + / - sense) in the item order
  double width;         // w_k
};

struct PairDev {
  double c, s;          // + sense in-plane direction (unit)
  float cf, sf;
};

struct PolarDev {       // per (pair, polar cosine)
  double w;             // omega of each of the two directions (+ and - sense)
  double sinz, inv_sinz;
  float wf, sinzf, inv_sinzf;
  int dir_plus, dir_minus;  // quadrature indices of the two directions
};

// Everything a kernel needs, by value.
struct PlanView {
  int nx, ny, ncell, G, n_pairs, n_polar;
  int64_t n_tracks, n_track_segments;
  const TrackDev *tracks;
  const int2 *seg32;            // FP32 sweep: {cell, len (f32 bits)} per track segment
  const int *seg_cell;          // FP64 path
  const double *seg_len;
  const double *seg_afrac;      // A / V (area fraction of the cell, after renormalisation)
  const PairDev *pairs;
  const PolarDev *polar;        // [pair][p]
  const double *geo;            // [4][cell]: sum_m omega sum_{C(i,m)} a times 1, Ox^2, OxOy, Oy^2
  const int64_t *dir_seg_off;   // canonical segment offset of each direction
  int *status;
  int gc32;                     // FP32 sweep: groups per chunk
  const int64_t *cell_off;      // FP32 moments: [ncell + 1] offsets into one chunk's gent entries
  const int4 *gent;             // FP32 moments: [chunk][entry] {state slot bits 0-31, slot bits 32-36 << 27 |
                                //   bundle length << 7 | lane, A/V f32 bits, 2 pair + sense} (gather_slot)
  int64_t gent_chunk;           // FP32 moments: entries per chunk (cell_off[ncell])
  const int2 *munit;            // FP32 moments: work units {cell, part}, cell-major; part k sums the cell's entries
                                //   [kPartEntries k, kPartEntries (k + 1))
  int64_t n_munits;
  const int4 *mmulti;           // FP32 moments: cells split in more than one part: {cell, first unit, parts, 0}
  int n_mmulti;
  double *mscratch;             // FP32 moments: [chunk][unit][6][gc] partial sums of split cells (or null)
  const int64_t *boff;          // FP32 state: [n_blocks + 1] first step slot of each bundle
  const int *block_order;       // FP32 sweep: bundle swept by each block of the launch (longest first)
  int sweep_depth;              // FP32 sweep: staging depth D (one of kSweepDepths; autotuned or 4)
  // face moments (Eq. 16), plans created with MOLC_FACES only (else null / 0)
  const int2 *seg_face;         // per track segment: upwind face of the + sense, of the - sense
  double *facc;                 // [chunk][face][6][gc] FP64 sums of omega w I (1, Omega, Omega Omega)
  unsigned long long *balance;  // MOLC_BALANCE: [0] bits of the largest per-ray relative balance residual, [1] bits
                                //   of max(B, boundary) of the sweep (else null)
  int n_faces;                  // x-faces (nx + 1) ny, then y-faces nx (ny + 1)
  double hx, hy;                // cell sizes (face lengths)
};

constexpr int kSweepDepths[] = {3, 4, 6};   // compiled staging depths of the FP32 sweep

// FP32 state, "bundle" layout: the work items (track, sense, group) of sweep block b, i.e. items
// [128 b, 128 b + 128), own the step slots [boff[b], boff[b+1]) (boff[b+1] - boff[b] = the longest track of the
// block); slot t holds the NP deviations of the block's 128 items side by side, so a block reads and writes
// 128 * NP contiguous values per step.  Items are numbered chunk-major:
// item = chunk * 2 T gc + pos[sense] * gcount + g_local, pos = TrackDev::pos (pair, then sense, then track).
__host__ __device__ inline int64_t bundle_index(const int64_t *boff, int64_t item, int s, int NP) {
  return ((boff[item / kSweepBlock] + s) * kSweepBlock + item % kSweepBlock) * NP;
}

// A moment-gather entry addresses the state slot of group 0 of its chunk directly: slot = (boff[b] + step) 128
// + lane for the item of group 0 at lane `lane` of bundle b.  Group gi of the same (track, sense) is item + gi:
// the same bundle while lane + gi < 128, else lane + gi - 128 of bundle b + 1, which starts blen(b) slots of
// 128 later.  Packing limits (checked by the planner): slot < 2^37, bundle length < 2^20.
constexpr int kGatherSlotHiShift = 27;
constexpr unsigned kGatherBlenMask = 0xFFFFFu;
__host__ __device__ inline int64_t gather_slot(int ex, int ey, int gi) {
  const unsigned y = (unsigned)ey;
  int64_t slot = (int64_t)(((uint64_t)(y >> kGatherSlotHiShift) << 32) | (unsigned)ex) + gi;
  if ((int)(y & (kSweepBlock - 1)) + gi >= kSweepBlock)
    slot += ((int64_t)((y >> 7) & kGatherBlenMask) - 1) * kSweepBlock;
  return slot;
}

// Group tiling of the opaque intensity state: groups are tiled in chunks of `gc` groups.  FP64 state: within a
// chunk, rows of width gcount*n_polar are ordered (track, sense, step); element (chunk, row, g_local, p).
// FP32 state: the bundle layout below.
struct Layout {
  int gc;                  // groups per chunk (FP64: G, FP32: PlanView::gc32)
  int n_chunks;
  int64_t rows;            // 2 * n_track_segments
};

inline Layout layout_for(const PlanView &v, molc_precision prec) {
  Layout L;
  L.gc = prec == MOLC_FP64 ? v.G : v.gc32;
  if (L.gc > v.G) L.gc = v.G;
  L.n_chunks = (v.G + L.gc - 1) / L.gc;
  L.rows = 2 * v.n_track_segments;
  return L;
}

// Byte offset of the reference Planck block inside an intensity state of `count` elements of `esize` bytes,
// and of the header after it: {scale, 1/scale, scratch (max bits), factor to this step's scale, block count}.
inline size_t bref_offset(int64_t count, int esize) { return ((size_t)count * esize + 255) / 256 * 256; }
inline size_t header_offset(int64_t count, int esize, int G, int ncell) {
  return bref_offset(count, esize) + ((size_t)G * ncell * 8 + 255) / 256 * 256;
}
constexpr size_t kHeaderBytes = 256;

struct SweepArgs {
  const double *kappa, *B, *bnd;
  double c, dt;
  double inv_c, inv_cdt;  // 1/c and 1/(c dt), formed on the host
  void *I;            // deviations delta = Ibar - B_ref, [chunk][row][g_local][p]
  double *Bref;       // [G][cell] Planck intensity the deviations refer to (inside the state)
  const double *scale;  // state header: [0] = scale of the stored deviations, [1] = 1/scale
  molc_moments out;
  float4 *cdat;       // FP32: [chunk][cell][gc] {kappa~, 1/(c dt kappa~), B_hi, B_lo}
  float *cdB;         // FP32: [chunk][cell][gc] (B_ref - B) / (c dt kappa~)
  double *acc;        // FP64 path: [cell][6][G] FP64 accumulators
  const int2 *items;  // FP32: one per thread, {track, sense | g_local << 1 | chunk << 16}; chunk-major,
                      // longest track first, then sense, then group
  int64_t n_items;
  double *fxx, *fxy, *fyy;   // Eddington factors [G][cell], written where the moments are assembled, or all null
};

struct TileInst;   // one instance of a tiled sweep launch (below)

// One instance of a batched FP32 sweep, as the batched kernels read it (device memory).
struct BatchInst {
  PlanView v;
  SweepArgs a;
  Layout L;
};

// Kernel launchers (molc_kernels.cu).  Return cudaSuccess or the launch error.
cudaError_t launch_prep(const PlanView &v, molc_precision prec, const SweepArgs &a, cudaStream_t st);
cudaError_t launch_sweep_fp64(const PlanView &v, const SweepArgs &a, cudaStream_t st);
cudaError_t launch_sweep_fp32(const PlanView &v, const SweepArgs &a, cudaStream_t st);
cudaError_t launch_finalize(const PlanView &v, molc_precision prec, const SweepArgs &a, cudaStream_t st);
cudaError_t launch_closure(const PlanView &v, const molc_moments &m, double c, double *fxx, double *fxy,
                           double *fyy, double *f_grey, cudaStream_t st);
cudaError_t launch_face_moments(const PlanView &v, molc_precision prec, const double *scale, double c,
                                const molc_moments &out, cudaStream_t st);
cudaError_t launch_grey(const PlanView &v, const molc_moments &m, const double *kappa, const double *B,
                        double *out, cudaStream_t st);
cudaError_t launch_intensity_copy(const PlanView &v, molc_precision prec, void *I, const double *Bref,
                                  const double *scale, int g_begin, int g_count, double *canon, bool to_canon,
                                  cudaStream_t st);
cudaError_t launch_balance_scale(const PlanView &v, const double *B, const double *bnd, cudaStream_t st);
cudaError_t launch_set_scale(const PlanView &v, molc_precision prec, const double *B, double *header,
                             cudaStream_t st);
// Batched FP32 kernels: one launch each over the blocks of all instances listed in a block map
// (prep: int4 {instance, chunk, tile, check boundary}; sweep: int2 {instance, bundle}, one launch per
// (polar count, staging depth) class; moments: int4 {instance, chunk, block, 0}, one launch per polar count;
// closure: int2 {instance, cell block}).
// Sweep-time scale update of an FP32 state from max(B, boundary) (see update_scale in molc_kernels.cu).
cudaError_t launch_update_scale(const PlanView &v, const double *B, const double *bnd, double *header,
                                cudaStream_t st);
// batched, several blocks per instance: map int4 {instance, block of the instance, blocks of the instance, 0}
// over `inst` (bundle batches) or `tinst` (tiled batches, when not null)
cudaError_t launch_update_scale_map(const BatchInst *inst, const TileInst *tinst, const int4 *map, int blocks,
                                    cudaStream_t st);
cudaError_t launch_prep_batch(const BatchInst *inst, const int4 *map, int blocks, cudaStream_t st);
cudaError_t launch_sweep_fp32_batch(const BatchInst *inst, const int2 *map, int blocks, int n_polar, int depth,
                                    cudaStream_t st);
cudaError_t launch_moments_fp32_batch(const BatchInst *inst, const int4 *map, int blocks, int n_polar,
                                      size_t smem, cudaStream_t st);
// combine step of split cells: map int4 {instance, chunk, block, 0} over the instance's split cells
cudaError_t launch_moments_combine_batch(const BatchInst *inst, const int4 *map, int blocks, cudaStream_t st);

// FP64 FMA rate of the current device in FLOP/s (2 per FMA), timed with CUDA events; synchronises.
cudaError_t fp64_fma_rate(double *flops_per_s);

// ---- Tiled FP32 sweep (plans without MOLC_FACES / MOLC_BALANCE, at most kMaxPolarFP32 polar cosines) ----------
// The material grid is cut into tiles of TS x TS cells.  Every characteristic is cut into pieces, one per tile it
// crosses; a work item is (tile, quadrant, group tile): the pieces of the directions that point into one quadrant
// (both senses of a pair lie in opposite quadrants) crossing the tile, for GT consecutive groups.  An item takes
// the intensity entering its pieces from the items upstream in its quadrant (the tiles before it in x and in y)
// and passes its outgoing intensity on, so the items of one (quadrant, group tile) form a wavefront over the
// tiles.  The item's previous-step state and cell table are staged in shared memory; its cell moments are summed
// there, per quadrant, and the four quadrant partials of a (tile, group tile) are combined by whichever item of
// the four finishes last.
constexpr int kTileThreadCandidates[] = {128, 256};   // threads of a tiled-sweep block (autotuned)
constexpr int kTileStateBytes = 88 * 1024;        // largest item state staged in shared memory
constexpr int kTileUnitEntries = 64;              // moment entries one thread sums (longer cell lists are split)
constexpr int kTileMaxUnits = 512;                // moment units of one item (shared-memory partials)
constexpr int kTileCandidates[] = {16, 8, 4, 2, 1};   // tile sizes tried, largest first
constexpr int kTileGroupCandidates[] = {4, 2, 1};      // groups per item tried, largest first
constexpr int kTileWaitLimit = 1 << 22;           // iterations of a bounded wait (with back-off, ~1-2 s)
constexpr int kStatusTimeout = 4;                 // device status: a bounded wait gave up

struct TileGeom {      // one (tile, quadrant) of a plan's tiled characteristic grid
  int tile, q;          // tile = ty * ntx + tx; q bit 0: the direction points towards -x, bit 1: towards -y
  int n_pieces, max_len, n_slots;
  int P_off;            // Ptab[P_off + t], t = 0..max_len: pieces still walking summed over the steps before t
  int64_t slot_base;    // first record of the geometry (records are indexed by geometry slot P[t] + rank)
  int64_t piece_off;    // global index of the geometry's rank-0 piece (pieces sorted longest first)
  int64_t ent_off;      // first moment entry of the geometry
  int unit_off, n_units;  // moment units of the geometry (cell-major)
  int cu_off;           // cell_units[cu_off + cell_local] = {first unit (relative), units}
  int up_x, up_y;       // upstream geometries of the same quadrant (previous tile in x, in y), or -1
  int delta;            // wavefront step of the tile in its quadrant
};

struct TileView {      // a plan's tiled FP32 layout and workspace, by value
  int TS, TS2p;        // tile side in cells; TS^2 rounded up to a multiple of 4 (per-group stride of tile tables)
  int ntx, nty, n_tiles, n_geoms;
  int GT, n_gt;        // groups per item, group tiles
  int n_items;         // n_gt * n_geoms (item id = gt * n_geoms + geom)
  int max_item_floats; // largest item state (floats, a multiple of 4)
  int max_len;
  const TileGeom *geoms;
  const int *Ptab;
  const int4 *pieces;  // {track, 2 len + sense, in (piece index >= 0, or -1 - entry edge), out (piece index or -1)}
  const int2 *recs;    // {cell_local, l (f32 bits)} per geometry slot, in the traversal order of the quadrant
  const int2 *ents;    // {geometry slot | pair << 24, A/V (f32 bits)} per (slot, cell), cell-major, by pair
  const int4 *units;   // {cell_local, first entry (relative), end entry, 0}
  const int2 *cell_units;
  const int64_t *item_off;   // state offset (floats) of each item
  // workspace (plan-owned, or carved from the static scratch)
  float4 *cdat;        // [tile][G][TS2p] {kappa~, 1/(c dt kappa~) x rescale, B_hi, B_lo}
  float *cdB;          // [tile][G][TS2p] (B_ref - B) / (c dt kappa~)
  float *bbuf;         // [piece][G][NP + 2]: intensity deviations entering the piece and B (hi, lo) before it
  double *part;        // [tile][gt][q][6][GT][TS2p]: per-quadrant moment partials
  int *cnt;            // [tile][gt]: quadrant items finished this step
  int *flags;          // [item]: the epoch of the last step the item finished
  int *ctrl;           // [0] ticket of the running launch, [1] epoch of this plan's steps
};

struct TileInst {      // one instance of a tiled sweep launch (device memory)
  PlanView v;
  TileView t;
  SweepArgs a;
};

// Shared-memory shape of a tiled-sweep launch: the largest item state (floats), cell-table entries (TS2p x GT),
// step count, azimuth pairs and split-cell moment units (units x GT) over its instances, and their common polar
// count (0 if they differ).
struct TileShape {
  int max_item_floats, cd_entries, max_len, n_pairs, split_units, np_exact;
};
// tiled sweep launchers: prep (cell tables, ticket reset, epoch; map {instance, first tile, group, check bnd}), the
// persistent sweep over the queue {instance, item} (ticket: the launch's counter, reset by the prep), intensity
// export/import
cudaError_t launch_tile_prep(const TileInst *inst, const int4 *map, int blocks, int *ticket, cudaStream_t st);
// one plan: `ov` (by value) is also stored at dst for the sweep launch that follows
cudaError_t launch_tile_prep_one(const TileInst &ov, TileInst *dst, const int4 *map, int blocks, int *ticket,
                                 cudaStream_t st);
cudaError_t launch_tile_sweep(const TileInst *inst, const int2 *queue, int n_queue, int *ticket, int np_max,
                              const TileShape &shape, int grid, int threads, cudaStream_t st);
size_t tile_sweep_smem(const TileShape &shape, int np_max);
// blocks of a persistent sweep launch: SMs x the blocks of `threads` threads and `smem` bytes one SM holds
int tile_sweep_grid(int np_max, size_t smem, int threads);
cudaError_t launch_tile_intensity_copy(const PlanView &v, const TileView &t, const int4 *tpiece,
                                       const int64_t *tpiece_off, float *I, const double *Bref,
                                       const double *scale, int g_begin, int g_count, double *canon, bool to_canon,
                                       cudaStream_t st);

// Fixed workspace of molc_sweep_static_scratch: a file-scope device array in molc_kernels.cu, 256-byte aligned.
constexpr size_t kStaticScratchBytes = (size_t)64 << 20;
// Device address of that array on the current device.  The first call per device looks the symbol up (which
// also loads the library's kernels on that device if nothing has yet); later calls return the cached address.
cudaError_t static_scratch_address(void **ptr);

}  // namespace molc
