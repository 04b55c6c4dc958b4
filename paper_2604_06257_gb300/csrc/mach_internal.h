// mach_internal.h -- plan state shared between the host plan code and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mach.h"

namespace mach {

// Kernel variants.  "frame lanes" kernels put frames on the lanes of a warp (the
// paper's frame-contiguous layout, Sec. 4.4); "channel lanes" kernels put a voxel's
// elements on the lanes (for ensembles too short to fill a warp, Sec. 4.6 notes the
// loss of coalescing below 16 frames).
enum Variant : int32_t {
  V_CH_C64 = 0,      // channel lanes, F <= 4, complex64
  V_F16_C64,         // frame lanes, 16-frame tile, complex64 (F even)
  V_F32_C64,         // frame lanes, 32-frame tile, complex64 (F even)
  V_F64_C64,         // frame lanes, 64-frame tile, complex64 (F even)
  V_S32_C64,         // frame lanes, 32-frame tile, scalar loads (any F)
  V_CH_H16,          // channel lanes, F <= 4, float16 pairs
  V_F32_H16,         // frame lanes, 32-frame tile, float16 pairs (F % 4 == 0)
  V_F64_H16,         // frame lanes, 64-frame tile, float16 pairs (F % 4 == 0)
  V_S32_H16,         // frame lanes, 32-frame tile, scalar loads (any F)
  V_ST32_C64,        // staged (bulk copies into shared memory), 32-frame tile, complex64
  V_ST64_C64,        // staged, 64-frame tile, complex64
  V_ST32_H16,        // staged, 32-frame tile, float16 pairs
  V_ST64_H16,        // staged, 64-frame tile, float16 pairs
  V_ST32_C64_V4,     // staged, 32-frame tile, 4 voxels per lane group
  V_ST32_C64_V4W4,   // staged, 32-frame tile, 4 voxels per lane group, 4 consumer warps
  V_ST64_C64_V4,     // staged, 64-frame tile, 4 voxels per lane group
  V_ST64_H16_V4,     // staged, 64-frame tile, float16 pairs, 4 voxels per lane group
  V_CH_B16,          // channel lanes, F <= 4, bfloat16 pairs
  V_F32_B16,         // frame lanes, 32-frame tile, bfloat16 pairs (F % 4 == 0)
  V_F64_B16,         // frame lanes, 64-frame tile, bfloat16 pairs (F % 4 == 0)
  V_S32_B16,         // frame lanes, 32-frame tile, scalar loads, bfloat16 pairs
  V_ST32_B16,        // staged, 32-frame tile, bfloat16 pairs
  V_ST64_B16_V4,     // staged, 64-frame tile, bfloat16 pairs, 4 voxels per lane group
  V_ST32_C64_V4R56,  // staged_c64_ft32_v4 capped at 56 registers (4 blocks per SM)
  V_F32_C64P,        // frame lanes, 32-frame tile, split complex64 rows (F % 4 == 0)
  V_F64_C64P,        // frame lanes, 64-frame tile, split complex64 rows (F % 4 == 0)
  V_ST32_C64P_V4,    // staged, 32-frame tile, split complex64 rows, 4 voxels per lane group
  V_ST64_C64P_V4,    // staged, 64-frame tile, split complex64 rows, 4 voxels per lane group
  V_ST32_H16_V4,     // staged, 32-frame tile, float16 pairs, 4 voxels per lane group
  V_ST32_B16_V4,     // staged, 32-frame tile, bfloat16 pairs, 4 voxels per lane group
  V_ST32_C64P_V4W7,  // staged, split rows, 7 consumer warps, 64 registers: 4 blocks per SM
  V_ST32_C64_V4W7,   // staged, interleaved, 7 consumer warps, 64 registers: 4 blocks per SM
  V_SX32_C64P,       // staged, split rows, F = 32 exactly (compile-time frames), 7 consumer warps
  V_SX64_C64P,       // staged, split rows, F = 64 exactly (compile-time frames), 8 consumer warps
  V_SX32_F4V2W7,     // F = 32 exactly: 4 frames x 2 voxels per lane, 7 consumer warps
  V_SX32_F8V1W7,     // F = 32 exactly: 8 frames x 1 voxel per lane, 7 consumer warps
  V_SX32_F4V2W15,    // F = 32 exactly: 4 frames x 2 voxels per lane, 15 consumer warps
  V_SX32_F8V1W15,    // F = 32 exactly: 8 frames x 1 voxel per lane, 15 consumer warps
  V_SX64_F8V2,       // F = 64 exactly: 8 frames x 2 voxels per lane, 8 consumer warps
  V_SX32_F8V1W15T24, // as V_SX32_F8V1W15 with 24 x 5 voxel tiles (2D)
  V_SX32_F8V1W15T40, // as V_SX32_F8V1W15 with 40 x 3 voxel tiles (2D)
  V_SX32_F8V1W15T24S,// as V_SX32_F8V1W15T24, consumers suspended in hardware while waiting
  V_SX64_C64PS,      // as V_SX64_C64P, consumers suspended in hardware while waiting
  V_SX32_F8V1W7T14,  // F = 32: 8 frames x 1 voxel per lane, 7 consumer warps, 14 x 4 tiles
  V_SX32_F8V1W7T14E, // as V_SX32_F8V1W7T14, ring slots released per pair
  V_SX32_F4V2W7T14,  // F = 32: 4 frames x 2 voxels per lane, 7 consumer warps, 14 x 4 tiles
  V_SX32_F8V1W15T30R12,  // F = 32: 8 frames x 1 voxel, 15 consumer warps, 30 x 4 tiles, 12 slots
  V_SX32_F8V1W15T30R12E, // as V_SX32_F8V1W15T30R12, ring slots released per pair
  V_SX64_C64PE,      // as V_SX64_C64P, ring slots released per pair
  V_SX16_F4V2W7,     // F = 16 exactly: 4 frames x 2 voxels per lane, 7 consumer warps
  V_SX16_F4V1W7,     // F = 16 exactly: 4 frames x 1 voxel per lane, 7 consumer warps
  V_SX8_F4V1W7,      // F = 8 exactly: 4 frames x 1 voxel per lane, 7 consumer warps
  V_CH_C64_L16,      // channel lanes, F <= 4, complex64, 16 lanes per voxel
  V_CH_C64_L32,      // channel lanes, F <= 4, complex64, 32 lanes per voxel
  V_SX64_C64P_T16,   // as V_SX64_C64P with 16 x 4 voxel tiles (2D)
  V_SX64_C64P_T16E,  // as V_SX64_C64P_T16, ring slots released per pair
  V_SX32_C64P_T8X14,    // as V_SX32_C64P with one-plane 8 x 14 x 1 tiles on 3D grids
  V_SX32_F8V1W7_T8X7E,  // 8 frames x 1 voxel per lane, 7 consumer warps, 8 x 7 x 1 tiles on
                        // 3D grids (14 x 4 in 2D), ring slots released per pair
  V_SX64_C64P_T8X8,     // as V_SX64_C64P with one-plane 8 x 8 x 1 tiles on 3D grids
  V_SX16_F4V2W7_T8X14,  // as V_SX16_F4V2W7 with one-plane 8 x 14 x 1 tiles on 3D grids
  V_SX8_F4V1W7_T8X14,   // as V_SX8_F4V1W7 with one-plane 8 x 14 x 1 tiles on 3D grids
  V_COUNT
};

struct VariantShape {
  const char* name;
  int frames_per_lane;   // frames one thread accumulates
  int lanes_per_voxel;   // frame lanes per voxel, or channel slices per voxel
  int voxels_per_warp;
  int frame_tile;        // frames covered by one block
  int warps;             // warps per block (consumer warps for staged variants)
  bool channel_lanes;
  bool staged;           // + one producer warp and a shared-memory ring of sample windows
  int ring_slots;
  int iq_bytes;          // bytes per complex sample
  int iq_type;           // mach_iq_dtype the variant reads
  int tile2d_x;          // 2D tile width (0: squarest power-of-two split)
  bool exact_frames;     // serves only F == frame_tile (k_das_exact.cu)
  int tile3d_x;          // 3D tile width and height (the rest along z; 0: pick_tile's box)
  int tile3d_y;
};

const VariantShape& variant_shape(Variant v);

// Everything a DAS kernel reads, passed by value.
struct DasParams {
  const float4* vox;    // [V] voxel position in sample units (x, y, z, 0)
  const float4* elem;   // [C] element position in sample units
  const float* tx;      // [T][V] transmit delay in samples
  const void* iq;       // [T][C][S][F] complex (float2 or half2)
  float2* y;            // [V][F] or nullptr (row of voxel v at y + v * ystride)
  float* pd;            // [V] or nullptr
  float* pd_part;       // [frame_tiles][V] scratch when frame_tiles > 1
  int64_t V;
  int C, T, S, F;
  int64_t ystride;      // complex elements between consecutive voxels' output rows (F)
  int nx, ny, nz;       // voxel index space (a list is nx = V, ny = nz = 1)
  int tile_x, tile_y, tile_z;
  int tiles_x, tiles_y, tiles_z;
  int apod;
  float two_f;          // (float)(2 F#)
  float f_num;          // (float)F#
  float four_f2;        // RN_float(4 F#^2): aperture test rho^2 * 4F#^2 <= dz^2
  float f_num2;         // (float)(F#^2)
  float s_max;          // (float)(S - 1): a term needs 0 <= s < s_max
  float r_f;            // (float)(fc / fs)
  uint32_t phase_R;     // round(2^32 frac(fc / fs))
  uint32_t phase_Phi;   // round(2^32 frac(fc t0))
  int frame_tiles;
  // staged variants only
  const float4* tbox;   // [tiles][2] voxel bounding box of each tile (sample units)
  const float2* txr;    // [tiles][txr_stride] (min, max) transmit delay over each tile
  int txr_stride;       // transmits per tile row of txr (T; larger for a single-transmit run)
  int rows_cap;         // rows of one ring slot
  uint32_t wait_limit;  // polls before a wait gives up
  int* err;             // device error word (bit 0: a wait timed out)
  int debug_stall;      // test hook: the producer announces copies but never issues them
  int wb_x, wb_y, wb_z; // staged variants: voxel block of one warp inside the tile (0: row-major)
  // staged variants with a plan-time term table only
  const int64_t* tile_pairs;  // [tiles + 1] index of each tile's first pair (pairs in copy order)
  const int4* pair_desc;      // [pairs] (transmit, element, first row, rows) of each copied window
  const float4* term_rec;     // [pairs][voxel slots of a block] term records, in consumer order
};

// Tables built once per plan (kernel K1).
struct TableParams {
  const float* raw_vox;     // [V][3] metres (list) or nullptr (grid)
  const double* u;          // [T][3] direction cosines (plane waves) or nullptr
  const float* tx_seconds;  // [T][V] user arrival times or nullptr
  double k;                 // fs / c
  double t0fs;              // t0 * fs
  double fs;
  double origin[3], step[3];
  int nx, ny, nz;
  int64_t V;
  int T;
  float4* vox_out;
  float* tx_out;
};

cudaError_t launch_tables(const TableParams& tp, cudaStream_t s);
cudaError_t launch_iq_convert(const float2* src, int src_order, void* dst, int dst_dtype, int64_t T, int64_t C,
                              int64_t S, int64_t F, cudaStream_t s);
cudaError_t launch_das(const DasParams& p, Variant v, cudaStream_t s);
// Per-tile bounds for the staged variants; returns the largest window (rows) and the
// number of (tile, transmit, element) triples that need a copy.
cudaError_t launch_tile_bounds(const DasParams& p, float4* tbox, float2* txr, int* d_rows_pairs,
                               cudaStream_t s);
size_t staged_smem_bytes(Variant v, int rows_cap, int F, int T, bool table);
cudaError_t launch_das_staged(const DasParams& p, Variant v, cudaStream_t s);
// Staged variants whose frame count is a compile-time constant (k_das_exact.cu).
size_t exact_smem_bytes(Variant v, int rows_cap, int T);
cudaError_t launch_das_exact(const DasParams& p, Variant v, cudaStream_t s);
// Plan-time term table (k_das_table.cu): which staged variants have a table form, the
// per-(tile, element) windows of every transmit (rows 0 = pair not used) and their
// count, the pair list and records, and the table-mode launch.
bool table_supported(Variant v);
cudaError_t launch_pair_windows(const DasParams& p, int2* win, int* count, cudaStream_t s);
cudaError_t launch_term_records(const DasParams& p, Variant v, const int2* win, const int64_t* first, int4* desc,
                                float4* rec, cudaStream_t s);
cudaError_t launch_das_table(const DasParams& p, Variant v, cudaStream_t s);
cudaError_t launch_terms(const DasParams& p, const int64_t* vox_idx, int64_t n, int32_t* i0,
                         float* w, float* cw, cudaStream_t s);
size_t das_smem_bytes(Variant v);

// Ragged batches (k_batch.cu / batch.cpp).
constexpr int kBatchFrames = 0;     // frame lanes (frame_lanes = 4, 8 or 16 lanes per voxel)
constexpr int kBatchChannels = 1;   // channel lanes (F <= 4)
constexpr int kBatchStaged = 2;     // staged windows (frame_lanes = 8: F <= 32, 16: F <= 64)
struct alignas(16) BatchInstance {
  DasParams p;          // the instance's tables, tiling and bound buffers
  int mode;             // kBatchFrames, kBatchChannels or kBatchStaged
  int frame_lanes;
};
int batch_blocks_per_sm(int iq_dtype, size_t slot_bytes);
size_t batch_smem_bytes(size_t slot_bytes);
cudaError_t launch_batch(int iq_dtype, const BatchInstance* insts, const int2* items, int n_items, int* counter,
                         int grid, size_t slot_bytes, cudaStream_t s);
const DasParams* plan_params(mach_plan p);
int plan_iq_dtype(mach_plan p);
void pick_tile_shape(int n, int nx, int ny, int nz, bool list, int tile[3]);

// Host steps shared by mach_das_plan and the allocation-free entry point.
mach_status host_validate(const mach_das_desc* d);
Variant host_unstaged_variant(int iq_dtype, int F);
mach_status host_configure_tiles(DasParams& b, Variant v, bool list, int64_t V, int F);
uint32_t host_fixed_cycles(double cycles);

}  // namespace mach
