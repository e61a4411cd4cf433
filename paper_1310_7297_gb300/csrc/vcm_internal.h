// vcm_internal.h -- structures shared by the host runtime (vcm_api.cpp) and
// the sm_103a kernels (vcm_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/vcm.h"

namespace vcm {

constexpr int kWarps = 4;                 // warps per block of the tile kernel
constexpr int kThreads = kWarps * 32;
constexpr int kPassCap = 2 * kThreads;       // cells listed per round of the grid walk
constexpr int kDistClasses = 128;            // distance classes of the candidate counting sort
// Launches whose requests all have this many patches use the whole-tile
// check (and the recorded-blocker pre-check): from 512, the 5,000-box step
// with 32 x 16 patches went 0.319 -> 0.305 ms (the bar was 1,024).
constexpr int kTileCheckMinPatches = 512;
constexpr int kMaxPlanes = 32;            // separating planes kept per tile hull
constexpr float kBand = 1e-6f;            // FP32 slab margin re-decided in FP64
constexpr int kMaxBoxCap = 5000;          // candidate boxes a tile stages in shared memory
// Candidate lists longer than this get the per-pass pyramid filter.  At 6-7
// blocks per SM the filter pays from short lists on (100,000-box step:
// 3.68 ms with 64, 3.55 with 16, 3.49 with 8, 3.52 with 0; the 256-request
// batch 102 ms with 0, 87-88 with 8 or more).
constexpr int kPyramidMinCount = 8;
constexpr int kMaxTileViewpoints = 1024;  // viewpoints in one tile (tile_x * tile_y)
constexpr int kClaimRounds = 4096;        // bounded retries of a spill-region claim (2 us pauses)

// Work sharing of the persistent tile kernel, in two passes.  In the first,
// a tile whose one-box check leaves at least its request's min_publish
// viewpoints open, and whose candidate list is staged whole and holds at
// most kPublishBoxes boxes, publishes them, chunk_vp at a time, as chunks;
// the second pass (a second launch of the same kernel) sweeps the chunks,
// each staging its owner's list again.
// The work buffer of a launch holds kWorkHeader counters (next tile,
// records, chunks published, chunks taken, id-pool ints used) and then the
// arena:
//   chunk[kChunkCap][2 + kChunkVp]   record index, count, viewpoints (tile-local)
//   record[kRecCap][kRecInts]        queue item, candidate count, offset of its ids in the pool
//   pool[kPoolInts]                  the records' candidate box ids, in the owner's order
//   blocker[kBlockerCap]             per tile position of each request (whole-tile-check
//                                    launches): a box id that blocked a tile there, or -1
// A tile whose publication would pass a cap keeps its viewpoints.
// 32 viewpoints per chunk: a block's 4 warps wait at the chunk's end for the
// slowest viewpoint, and more viewpoints per chunk spread that wait
// (100,000-box step 3.50 -> 3.38 ms against 16; 64: 3.44, and the 5,000-box
// step +7 %; 8: +5 %).
constexpr int kChunkVp = 32;
constexpr int kMinPublish = 8;
// Longer lists stay with their tile (the 100,000-box scene, lists of ~180
// boxes on average: 6.44 ms with this limit, 6.71 ms without it) unless the
// tile has at least kPublishHeavy open viewpoints (32: 3.84 -> 3.82 ms
// against 64; the tiles with 39-63 open viewpoints and lists just over 128
// had set the end of the tile pass).
constexpr int kPublishBoxes = 128;
constexpr int kPublishHeavy = 32;
constexpr int kChunkCap = 262144;
constexpr int kRecCap = 65536;
constexpr int kRecInts = 3;
constexpr int kPoolInts = 8 << 20;
constexpr int kBlockerCap = 1 << 20;
constexpr int kWorkHeader = 64;   // ints before the arena (256 bytes)
constexpr size_t kChunkOff = 0;
constexpr size_t kRecOff = kChunkOff + (size_t)kChunkCap * (2 + kChunkVp);
constexpr size_t kPoolOff = kRecOff + (size_t)kRecCap * kRecInts;
constexpr size_t kBlockerOff = kPoolOff + (size_t)kPoolInts;
constexpr size_t kArenaInts = kBlockerOff + (size_t)kBlockerCap;
constexpr size_t kWorkBytes = (kWorkHeader + kArenaInts) * sizeof(int);

inline size_t tiles_smem_bytes(int box_cap) { return (size_t)box_cap * (32 + 4); }

// Device view of the scene and its uniform-grid index.  Boxes are sorted by
// grid cell; `boxes[perm]` holds the same boxes with their coordinates
// permuted into one of the six (u, n, w) target frames, two float4 per box
// (lo.xyz, hi.xyz).  Permutation 0 is the world frame (x, y, z).
struct DevScene {
    const float4 *boxes[6];
    int n_boxes;
    int dims;
    const int *cell_start;     // [n_cells + 1] into the sorted box order
    const float4 *cell_lo;     // [n_cells] bounds of each cell's boxes (world)
    const float4 *cell_hi;
    float gx0, gy0;            // grid origin (world x, y)
    float cell, inv_cell;
    int gnx, gny;
    float overhang;            // how far a cell's bounds reach past the cell
};

// One canonicalised request (host-computed, lattice-exact coordinates).
// Target frame: axis 0 = u (patch columns), 1 = n (normal), 2 = w (rows).
struct DevRequest {
    int dims;
    int au, an, aw;            // world axis of u, n, w
    int perm;                  // index of the box copy in that frame
    float sn;                  // +1 / -1: side of the normal
    float p_n;                 // patch coordinate along the normal axis
    int nu, nw, P, words;
    float measure;             // patch area (3D) or length (2D), metres
    int nx, ny, nl;            // viewpoint grid
    int tile_x, tile_y, tiles_x, tiles_y, n_tiles;
    int nuc, groups, col_passes, row_passes, k_rows;   // lane mapping
    int chunk_vp, min_publish;   // work sharing: viewpoints per chunk, open viewpoints to publish
    int blk_base;                // offset of its tile positions in the blocker table, or -1
    const float *u_coord;      // [nu] patch centre coordinate along u
    const float *w_coord;      // [nw] along w (one 0 in 2D)
    const float *x_coord;      // [nx] viewpoint x
    const float *y_coord;      // [ny] viewpoint y
    const float *z_coord;      // [nl] layer heights (one 0 in 2D)
    float u_min, u_max, w_min, w_max;
    float *v_out;
    uint8_t *color_out;
    uint32_t *bits_out;
    vcm_stats *stats;
    float v_ref_given;
    int levels;
    unsigned flags;
    int box_cap;               // candidate boxes staged in shared memory
    int cone;                  // 1: a field-of-view cone masks the patches
    float cone_c;              // cosine of its half-angle
    float cone_a[3];           // its unit axis, world x, y, z
};

// Launch helpers implemented in vcm_kernels.cu.  All are asynchronous on
// `stream` and return the launch status.
cudaError_t launch_grid_build(const float *d_lo_world, const float *d_hi_world, int n, int dims,
                              float gx0, float gy0, float cell, int gnx, int gny,
                              int *d_cell_of, int *d_count, int *d_cursor, int *d_order,
                              int *d_cell_start, float4 *const *d_perm_boxes, float4 *d_cell_lo,
                              float4 *d_cell_hi, unsigned *d_overhang_bits, cudaStream_t stream);

// The tile kernel over `n_req` requests (their tiles concatenated,
// `d_tile_prefix` = exclusive prefix of tiles, n_req + 1 entries).  Persistent
// by default: grid_blocks blocks draw tiles from `d_work` (zeroed by the
// caller).  With one_tile, one block per tile, so concurrent launches
// interleave block by block; grid_blocks must then be at least the number of
// blocks that can be resident at once, and `d_spill_busy` (grid_blocks ints,
// all zero between launches) hands out the spill regions.  `d_spill` holds
// grid_blocks * n_boxes ints for candidate lists longer than box_cap.
// `extra` must be set when any request is two-sided or has a field-of-view
// cone: it selects the tile kernel's instantiation that handles them.
// `tile_check` selects the instantiation with the whole-tile check (any
// launch may use either; it pays when every request has many patches).
// `share` (persistent launches only): d_work is kWorkBytes long, and a second
// launch of the kernel works the open viewpoints that expensive tiles of the
// first published there.
// `claim_rounds` (1..kClaimRounds) bounds the retries of a one-tile block's
// spill-region claim; a block that gives up runs without a region and sets
// its request's vcm_stats.error to VCM_DEVERR_SPILL_WAIT if its candidate
// list needs one.
cudaError_t launch_tiles(const DevScene &sc, const DevRequest *d_reqs, const int *d_tile_prefix,
                         int n_req, int total_tiles, int *d_work, int *d_spill, int grid_blocks,
                         int box_cap, bool extra, bool tile_check, cudaStream_t stream, bool one_tile = false,
                         int *d_spill_busy = nullptr, bool share = false, int claim_rounds = kClaimRounds);
// Colors and edge counts for all viewpoints of n_req requests (grid over the
// concatenated viewpoints, `d_vp_prefix` = exclusive prefix, n_req + 1).
cudaError_t launch_quantise(const DevRequest *d_reqs, const long long *d_vp_prefix, int n_req,
                            long long total_vp, cudaStream_t stream);

// Values of one request (d_req[0]) recomputed from the occlusion bits its
// bits_out points at (read only); colors then come from launch_quantise.
// d_list: n_vp ints of scratch for the viewpoints that need a measure, and
// d_n_list their count (n_vp <= INT_MAX).
cudaError_t launch_recolor(const DevRequest *d_req, long long n_vp, int sm_count, int *d_list, int *d_n_list,
                           cudaStream_t stream);

// Zero the tile-queue counters (d_work[0..kWorkHeader)), every request's
// vcm_stats and, when
// any_bits, the occlusion-bit buffers of the requests with VCM_EMIT_BITS.
cudaError_t launch_prologue(const DevRequest *d_reqs, int n_req, int *d_work, bool any_bits, cudaStream_t stream);

// Blocks of the tile kernel that fit on one SM for this shared-memory size.
int tiles_blocks_per_sm(int box_cap);

// One-time per-device setup (constant tables, kernel attributes); must run
// before any launch is captured into a graph.
cudaError_t init_device();

// Device address and size of the file-scope scratch array used by
// vcm_compute_static on the current device (looked up once per device).
cudaError_t static_scratch(void **ptr, size_t *bytes);

}  // namespace vcm
