// plan.cpp -- the C ABI: argument validation, plan construction (Sec. 4.3 precompute),
// kernel-variant selection and the run entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "mach.h"
#include "mach_internal.h"

using namespace mach;

struct mach_plan_s {
  mach_das_desc d{};          // copy; pointer fields cleared
  int device = 0;
  Variant variant = V_COUNT;
  DasParams base{};           // everything but iq / y / pd
  float4* d_vox = nullptr;
  float4* d_elem = nullptr;
  float* d_tx = nullptr;
  float* d_pd_part = nullptr;
  float4* d_tbox = nullptr;     // staged variants: per-tile bounding boxes
  float2* d_txr = nullptr;      // staged variants: per-tile transmit-delay ranges
  int* d_err = nullptr;         // device error word
  int rows_cap = 0;
  int64_t copy_pairs = 0;
  int64_t device_bytes = 0;
  bool table = false;           // terms read from the plan-time term table
  int64_t* d_tile_pairs = nullptr;
  int4* d_pair_desc = nullptr;
  float4* d_term_rec = nullptr;
  int64_t table_bytes = 0;
};

namespace {

int g_fail_alloc_countdown = 0;   // test hook: > 0 -> the n-th allocation fails
int g_force_variant = -1;         // test hook: variant index, or -1 for automatic choice
uint32_t g_wait_limit = 0;        // test hook: polls per bounded wait (0 = default)
int g_stall = 0;                  // test hook: staged producer never issues its copies
constexpr uint32_t kDefaultWaitLimit = 1u << 24;   // ~ seconds of polling
constexpr size_t kStagedSmemCap = 110 * 1024;       // leaves room for two blocks per SM

mach_status dev_alloc(void** p, size_t bytes, int64_t* total) {
  *p = nullptr;
  if (g_fail_alloc_countdown > 0 && --g_fail_alloc_countdown == 0) return MACH_ERR_OOM;
  if (bytes == 0) bytes = 16;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return MACH_ERR_OOM;
  }
  if (e != cudaSuccess) return MACH_ERR_CUDA;
  *total += static_cast<int64_t>(bytes);
  return MACH_OK;
}

bool finite3(const float* p, int64_t n) {
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

mach_status validate(const mach_das_desc* d) {
  if (!d) return MACH_ERR_INVALID_ARG;
  if (d->ndim != 2 && d->ndim != 3) return MACH_ERR_INVALID_ARG;
  if (d->n_elem < 1 || !d->elem_pos) return MACH_ERR_INVALID_ARG;
  if (d->n_tx < 1 || (!d->tx_angles && !d->tx_table_dev)) return MACH_ERR_INVALID_ARG;
  if (!(d->fs > 0.0) || !std::isfinite(d->fs) || !(d->c > 0.0) || !std::isfinite(d->c))
    return MACH_ERR_INVALID_ARG;
  if (!(d->fc >= 0.0) || !std::isfinite(d->fc) || !std::isfinite(d->t0)) return MACH_ERR_INVALID_ARG;
  if (!(d->f_number >= 0.0) || !std::isfinite(d->f_number)) return MACH_ERR_INVALID_ARG;
  if (d->apod < MACH_APOD_NONE || d->apod > MACH_APOD_GAUSS) return MACH_ERR_INVALID_ARG;
  if (d->iq_dtype < MACH_IQ_C64 || d->iq_dtype > MACH_IQ_C64_SPLIT) return MACH_ERR_INVALID_ARG;
  if (d->term_table != 0 && d->term_table != 1) return MACH_ERR_INVALID_ARG;
  if (d->iq_dtype == MACH_IQ_C64_SPLIT && (d->n_frames % 4 != 0 || d->n_frames <= 4)) return MACH_ERR_UNSUPPORTED;
  if (d->n_samples < 2 || d->n_samples > (1 << 24)) return MACH_ERR_INVALID_ARG;
  if (d->n_frames < 1) return MACH_ERR_INVALID_ARG;
  // per-(t, c) slab offsets are computed in 64 bits, but one slab must stay indexable
  if (static_cast<int64_t>(d->n_samples) * d->n_frames > (int64_t{1} << 31) - 1) return MACH_ERR_UNSUPPORTED;
  if (!finite3(d->elem_pos, d->n_elem)) return MACH_ERR_INVALID_ARG;
  int64_t V;
  if (d->vox_pos) {
    if (d->n_vox < 1) return MACH_ERR_INVALID_ARG;
    V = d->n_vox;
    if (!finite3(d->vox_pos, V)) return MACH_ERR_INVALID_ARG;
  } else {
    for (int k = 0; k < 3; ++k) {
      if (d->grid_dims[k] < 1) return MACH_ERR_INVALID_ARG;
      if (!std::isfinite(d->grid_origin[k]) || !std::isfinite(d->grid_step[k])) return MACH_ERR_INVALID_ARG;
    }
    V = static_cast<int64_t>(d->grid_dims[0]) * d->grid_dims[1] * d->grid_dims[2];
    if (d->n_vox != 0 && d->n_vox != V) return MACH_ERR_INVALID_ARG;
  }
  if (V > (int64_t{1} << 40)) return MACH_ERR_UNSUPPORTED;
  if (d->tx_angles)
    for (int t = 0; t < 2 * d->n_tx; ++t)
      if (!std::isfinite(d->tx_angles[t])) return MACH_ERR_INVALID_ARG;
  if (d->ndim == 2) {   // a 2D acquisition lives in the plane y = 0
    for (int c = 0; c < d->n_elem; ++c)
      if (d->elem_pos[3 * c + 1] != 0.0f) return MACH_ERR_INVALID_ARG;
    if (d->tx_angles && !d->tx_table_dev)
      for (int t = 0; t < d->n_tx; ++t)
        if (d->tx_angles[2 * t + 1] != 0.0) return MACH_ERR_INVALID_ARG;
    if (d->vox_pos) {
      for (int64_t v = 0; v < V; ++v)
        if (d->vox_pos[3 * v + 1] != 0.0f) return MACH_ERR_INVALID_ARG;
    } else if (d->grid_dims[1] != 1 || d->grid_origin[1] != 0.0) {
      return MACH_ERR_INVALID_ARG;
    }
  }
  return MACH_OK;
}

Variant pick_variant(int iq_dtype, int F) {
  // staged 4-voxel-group kernels for 16 < F <= 64 (fastest measured shapes); L1-path
  // kernels for short, long (frame-tiled) or odd ensembles
  if (iq_dtype == MACH_IQ_C64) {
    if (F <= 4) return V_CH_C64;
    if (F % 2 == 0) {
      if (F <= 16) return V_F16_C64;
      if (F <= 32) return V_ST32_C64_V4W7;
      if (F <= 64) return V_ST64_C64_V4;
      return V_F64_C64;
    }
    return V_S32_C64;
  }
  if (iq_dtype == MACH_IQ_C64_SPLIT) {   // F % 4 == 0 and F > 4 (checked by validate)
    if (F == 8) return V_SX8_F4V1W7;
    if (F == 16) return V_SX16_F4V2W7;
    if (F == 32) return V_SX32_F8V1W7T14E;
    if (F == 64) return V_SX64_C64P;
    if (F <= 16) return V_F32_C64P;
    if (F <= 32) return V_ST32_C64P_V4W7;
    if (F <= 64) return V_ST64_C64P_V4;
    return V_F64_C64P;
  }
  if (iq_dtype == MACH_IQ_BF16X2) {
    if (F <= 4) return V_CH_B16;
    if (F % 4 == 0) {
      if (F <= 16) return V_F32_B16;
      if (F <= 32) return V_ST32_B16_V4;
      if (F <= 64) return V_ST64_B16_V4;
      return V_F64_B16;
    }
    return V_S32_B16;
  }
  if (F <= 4) return V_CH_H16;
  if (F % 4 == 0) {
    if (F <= 16) return V_F32_H16;
    if (F <= 32) return V_ST32_H16_V4;
    if (F <= 64) return V_ST64_H16_V4;
    return V_F64_H16;
  }
  return V_S32_H16;
}

// The non-staged variant with the same frame tile (used when the ring would not fit).
Variant unstaged(Variant v) {
  switch (v) {
    case V_ST32_C64: case V_ST32_C64_V4: case V_ST32_C64_V4W4: case V_ST32_C64_V4R56: case V_ST32_C64_V4W7:
      return V_F32_C64;
    case V_ST64_C64: case V_ST64_C64_V4: return V_F64_C64;
    case V_ST32_H16: case V_ST32_H16_V4: return V_F32_H16;
    case V_ST64_H16: case V_ST64_H16_V4: return V_F64_H16;
    case V_ST32_B16: case V_ST32_B16_V4: return V_F32_B16;
    case V_ST32_C64P_V4: case V_ST32_C64P_V4W7: case V_SX32_C64P: case V_SX32_F4V2W7: case V_SX32_F8V1W7:
    case V_SX32_F4V2W15: case V_SX32_F8V1W15: case V_SX32_F8V1W15T24: case V_SX32_F8V1W15T40:
    case V_SX32_F8V1W15T24S: case V_SX32_F8V1W7T14: case V_SX32_F8V1W7T14E: case V_SX32_F4V2W7T14:
    case V_SX32_F8V1W15T30R12: case V_SX32_F8V1W15T30R12E: case V_SX32_C64P_T8X14: case V_SX32_F8V1W7_T8X7E:
      return V_F32_C64P;
    case V_ST64_C64P_V4: case V_SX64_C64P: case V_SX64_F8V2: case V_SX64_C64PS: case V_SX64_C64PE:
    case V_SX64_C64P_T16: case V_SX64_C64P_T16E: case V_SX64_C64P_T8X8:
      return V_F64_C64P;
    case V_SX16_F4V2W7: case V_SX16_F4V1W7: case V_SX8_F4V1W7: case V_SX16_F4V2W7_T8X14: case V_SX8_F4V1W7_T8X14:
      return V_F32_C64P;
    case V_ST64_B16_V4: return V_F64_B16;
    default: return v;
  }
}

bool variant_accepts(Variant v, int iq_dtype, int F) {
  const VariantShape& s = variant_shape(v);
  if (s.iq_type != iq_dtype) return false;
  if (s.channel_lanes) return F <= s.frame_tile;
  const int vec = s.frames_per_lane == 1 ? 1 : (s.iq_type == MACH_IQ_C64 ? 2 : 4);
  if (F % vec != 0) return false;
  if (s.staged && F > s.frame_tile) return false;
  if (s.exact_frames && F != s.frame_tile) return false;
  return true;
}

// The variant to try when a staged variant's ring does not fit in shared memory: one with
// fewer ring slots (the variant itself when there is none).
Variant staged_fallback(Variant v) {
  switch (v) {
    case V_ST64_C64_V4: return V_ST64_C64;
    case V_ST64_H16_V4: return V_ST64_H16;
    case V_SX32_F8V1W15: case V_SX32_F4V2W15: case V_SX32_F8V1W7: case V_SX32_F4V2W7: case V_SX32_F8V1W15T24:
    case V_SX32_F8V1W15T40: case V_SX32_F8V1W15T24S: case V_SX32_F8V1W7T14: case V_SX32_F8V1W7T14E:
    case V_SX32_F4V2W7T14: case V_SX32_F8V1W15T30R12: case V_SX32_F8V1W15T30R12E: case V_SX32_F8V1W7_T8X7E:
      return V_SX32_C64P;
    default: return v;
  }
}

// The generic staged variant an exact-frame variant specialises (term tables are built
// for the generic kernels' record layout).
Variant generic_staged(Variant v) {
  switch (v) {
    case V_SX32_C64P: case V_SX32_F4V2W7: case V_SX32_F8V1W7: case V_SX32_F4V2W15: case V_SX32_F8V1W15:
    case V_SX32_F8V1W15T24: case V_SX32_F8V1W15T40: case V_SX32_F8V1W15T24S: case V_SX32_F8V1W7T14:
    case V_SX32_F8V1W7T14E: case V_SX32_F4V2W7T14: case V_SX32_F8V1W15T30R12: case V_SX32_F8V1W15T30R12E:
    case V_SX32_C64P_T8X14: case V_SX32_F8V1W7_T8X7E:
      return V_ST32_C64P_V4W7;
    case V_SX64_C64P: case V_SX64_F8V2: case V_SX64_C64PS: case V_SX64_C64PE: case V_SX64_C64P_T16:
    case V_SX64_C64P_T16E: case V_SX64_C64P_T8X8:
      return V_ST64_C64P_V4;
    case V_SX16_F4V2W7: case V_SX16_F4V1W7: case V_SX8_F4V1W7: case V_SX16_F4V2W7_T8X14: case V_SX8_F4V1W7_T8X14:
      return V_F32_C64P;
    default: return v;
  }
}

// Voxel tile of one block: compact boxes so that the voxels sharing a block (and the
// L1 cache) read overlapping sample windows of each element.
void pick_tile(int n, int nx, int ny, int nz, bool list, int tile[3]) {
  // the box always holds exactly n voxel slots
  if (list || (ny == 1 && nz == 1)) {
    tile[0] = n; tile[1] = 1; tile[2] = 1;
    return;
  }
  if (ny == 1) {   // 2D x-z grid: the squarest power-of-two width that divides n
    int tx = 1;
    while (tx * tx < n) tx *= 2;
    while (n % tx) tx /= 2;
    tile[0] = tx; tile[1] = 1; tile[2] = n / tx;
    return;
  }
  // 3D: up to 8 along x and 4 along y (powers of two dividing n), the rest along z
  int tx = 8;
  while (n % tx) tx /= 2;
  int ty = 4;
  while ((n / tx) % ty) ty /= 2;
  tile[0] = tx; tile[1] = ty; tile[2] = n / (tx * ty);
}

uint32_t fixed_cycles(double cycles) {   // round(2^32 frac(cycles))
  double f = cycles - std::floor(cycles);
  double r = std::nearbyint(f * 4294967296.0);
  if (r >= 4294967296.0) r -= 4294967296.0;
  return static_cast<uint32_t>(r);
}

void release(mach_plan_s* p) {
  if (!p) return;
  cudaFree(p->d_vox);
  cudaFree(p->d_elem);
  cudaFree(p->d_tx);
  cudaFree(p->d_pd_part);
  cudaFree(p->d_tbox);
  cudaFree(p->d_txr);
  cudaFree(p->d_err);
  cudaFree(p->d_tile_pairs);
  cudaFree(p->d_pair_desc);
  cudaFree(p->d_term_rec);
  delete p;
}

}  // namespace

extern "C" {

const char* mach_status_string(mach_status s) {
  switch (s) {
    case MACH_OK: return "ok";
    case MACH_ERR_INVALID_ARG: return "invalid argument";
    case MACH_ERR_CUDA: return "CUDA error";
    case MACH_ERR_OOM: return "out of device memory";
    case MACH_ERR_UNSUPPORTED: return "unsupported configuration";
    case MACH_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* mach_version(void) { return "mach-gb300 0.1.0 sm_103a"; }

void mach_debug_fail_alloc_after(int32_t n) { g_fail_alloc_countdown = n > 0 ? n : 0; }

// Tile geometry of a variant: voxel box per block and the number of blocks.
static mach_status configure_tiles(DasParams& b, Variant var, bool list, int64_t V, int F) {
  const VariantShape& shp = variant_shape(var);
  const int per_cta = shp.voxels_per_warp * shp.warps;
  int tile[3];
  pick_tile(per_cta, b.nx, b.ny, b.nz, list, tile);
  if (shp.tile2d_x && !list && b.ny == 1 && b.nz > 1 && per_cta % shp.tile2d_x == 0) {
    tile[0] = shp.tile2d_x;
    tile[1] = 1;
    tile[2] = per_cta / shp.tile2d_x;
  }
  if (shp.tile3d_x && !list && b.ny > 1 && per_cta % (shp.tile3d_x * shp.tile3d_y) == 0) {
    tile[0] = shp.tile3d_x;
    tile[1] = shp.tile3d_y;
    tile[2] = per_cta / (shp.tile3d_x * shp.tile3d_y);
  }
  if (tile[0] * tile[1] * tile[2] != per_cta) return MACH_ERR_UNSUPPORTED;   // slots must map 1:1
  b.tile_x = tile[0];
  b.tile_y = tile[1];
  b.tile_z = tile[2];
  b.tiles_x = (b.nx + tile[0] - 1) / tile[0];
  b.tiles_y = (b.ny + tile[1] - 1) / tile[1];
  b.tiles_z = (b.nz + tile[2] - 1) / tile[2];
  b.frame_tiles = (F + shp.frame_tile - 1) / shp.frame_tile;
  (void)V;
  // staged kernels: each warp owns a compact block of the tile, so that its voxels tend to
  // agree on which (element, transmit) pairs they use (the warp skips pairs none of them use)
  b.wb_x = b.wb_y = b.wb_z = 0;
  if (shp.staged && !list && !(b.ny == 1 && b.nz == 1)) {
    // candidate blocks, most compact first; the first one that divides the tile is used
    static const int c2d32[][3] = {{8, 1, 4}, {16, 1, 2}, {4, 1, 8}};
    static const int c2d16[][3] = {{4, 1, 4}, {8, 1, 2}, {16, 1, 1}};
    static const int c2d8[][3] = {{4, 1, 2}, {8, 1, 1}, {2, 1, 4}};
    static const int c3d32[][3] = {{4, 4, 2}, {8, 4, 1}};
    static const int c3d16[][3] = {{4, 4, 1}, {8, 2, 1}};
    static const int c3d8[][3] = {{4, 2, 1}, {8, 1, 1}};
    const int wv = shp.voxels_per_warp;
    const int(*cand)[3] = nullptr;
    int nc = 0;
    if (b.ny == 1) {
      if (wv == 32) { cand = c2d32; nc = 3; } else if (wv == 16) { cand = c2d16; nc = 3; } else if (wv == 8) { cand = c2d8; nc = 3; }
    } else {
      if (wv == 32) { cand = c3d32; nc = 2; } else if (wv == 16) { cand = c3d16; nc = 2; } else if (wv == 8) { cand = c3d8; nc = 2; }
    }
    for (int k = 0; k < nc; ++k) {
      if (tile[0] % cand[k][0] == 0 && tile[1] % cand[k][1] == 0 && tile[2] % cand[k][2] == 0) {
        b.wb_x = cand[k][0];
        b.wb_y = cand[k][1];
        b.wb_z = cand[k][2];
        break;
      }
    }
  }
  if (b.frame_tiles > 65535) return MACH_ERR_UNSUPPORTED;   // grid y limit
  if (static_cast<int64_t>(b.tiles_x) * b.tiles_y * b.tiles_z > INT32_MAX) return MACH_ERR_UNSUPPORTED;
  return MACH_OK;
}

// Plan-time term table (table mode): every usable (tile, element, transmit) pair's
// window and the records of all voxel slots of the block, in the order a run consumes
// them.  The windows come first; their counts, scanned on the host, give each pair its
// index, and one block per (tile, element) then writes the records.
static mach_status build_term_table(mach_plan_s* p, DasParams& b, cudaStream_t s) {
  const int64_t tiles = static_cast<int64_t>(b.tiles_x) * b.tiles_y * b.tiles_z;
  const int64_t n = tiles * b.C;
  if (n > INT32_MAX) return MACH_ERR_UNSUPPORTED;   // one record block per (tile, element)
  const VariantShape& sh = variant_shape(p->variant);
  const int64_t nrec = static_cast<int64_t>(sh.warps) * sh.voxels_per_warp;
  int2* d_win = nullptr;
  int* d_count = nullptr;
  int64_t* d_first = nullptr;
  int64_t scratch = 0;
  auto done = [&](mach_status e) {
    cudaFree(d_win);
    cudaFree(d_count);
    cudaFree(d_first);
    return e;
  };
  mach_status st;
  if ((st = dev_alloc(reinterpret_cast<void**>(&d_win), sizeof(int2) * n * b.T, &scratch)) != MACH_OK) return done(st);
  if ((st = dev_alloc(reinterpret_cast<void**>(&d_count), sizeof(int) * n, &scratch)) != MACH_OK) return done(st);
  if (launch_pair_windows(b, d_win, d_count, s) != cudaSuccess) return done(MACH_ERR_CUDA);
  std::vector<int> count(static_cast<size_t>(n));
  if (cudaMemcpyAsync(count.data(), d_count, sizeof(int) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return done(MACH_ERR_CUDA);
  std::vector<int64_t> first(static_cast<size_t>(n) + 1, 0);
  for (int64_t i = 0; i < n; ++i) first[i + 1] = first[i] + count[i];
  const int64_t pairs = first[n];
  std::vector<int64_t> tile_first(static_cast<size_t>(tiles) + 1);
  for (int64_t t = 0; t < tiles; ++t) tile_first[t] = first[t * b.C];
  tile_first[tiles] = pairs;
  const size_t bytes = sizeof(int64_t) * (tiles + 1) + sizeof(int4) * pairs + sizeof(float4) * pairs * nrec;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return done(MACH_ERR_CUDA);
  }
  if (bytes + sizeof(int64_t) * (n + 1) > free_b) return done(MACH_ERR_OOM);
  if ((st = dev_alloc(reinterpret_cast<void**>(&p->d_tile_pairs), sizeof(int64_t) * (tiles + 1), &p->device_bytes)) != MACH_OK)
    return done(st);
  if ((st = dev_alloc(reinterpret_cast<void**>(&p->d_pair_desc), sizeof(int4) * pairs, &p->device_bytes)) != MACH_OK)
    return done(st);
  if ((st = dev_alloc(reinterpret_cast<void**>(&p->d_term_rec), sizeof(float4) * pairs * nrec, &p->device_bytes)) != MACH_OK)
    return done(st);
  if ((st = dev_alloc(reinterpret_cast<void**>(&d_first), sizeof(int64_t) * (n + 1), &scratch)) != MACH_OK)
    return done(st);
  if (cudaMemcpyAsync(d_first, first.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p->d_tile_pairs, tile_first.data(), sizeof(int64_t) * (tiles + 1), cudaMemcpyHostToDevice, s) !=
          cudaSuccess)
    return done(MACH_ERR_CUDA);
  if (launch_term_records(b, p->variant, d_win, d_first, p->d_pair_desc, p->d_term_rec, s) != cudaSuccess)
    return done(MACH_ERR_CUDA);
  if (cudaStreamSynchronize(s) != cudaSuccess) return done(MACH_ERR_CUDA);
  b.tile_pairs = p->d_tile_pairs;
  b.pair_desc = p->d_pair_desc;
  b.term_rec = p->d_term_rec;
  p->table_bytes = static_cast<int64_t>(bytes);
  p->table = true;
  return done(MACH_OK);
}

mach_status mach_das_plan(const mach_das_desc* d, void* stream, mach_plan* out) {
  if (!out) return MACH_ERR_INVALID_ARG;
  *out = nullptr;
  mach_status st = validate(d);
  if (st != MACH_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  const int C = d->n_elem, T = d->n_tx, S = d->n_samples, F = d->n_frames;
  const bool list = d->vox_pos != nullptr;
  const int64_t V = list ? d->n_vox
                         : static_cast<int64_t>(d->grid_dims[0]) * d->grid_dims[1] * d->grid_dims[2];
  if (list && V > INT32_MAX) return MACH_ERR_UNSUPPORTED;
  Variant var = pick_variant(d->iq_dtype, F);
  // 3D grids with 32 frames: one-plane 8 x 7 x 1 tiles.  A step in depth moves the two-way
  // delay about twice as far as the step itself, a lateral step far less, so a tile one
  // plane deep needs the shortest sample windows; with 256-byte rows that shrinks the ring
  // (15 instead of 36 rows a slot) and more blocks stay resident (94 x 94 x 178 voxels,
  // 1024 elements: 2.82 T points/s, against 2.31 for 8 x 2 x 7 tiles at 4 frames per lane
  // and 2.10 for 8 x 1 x 7 tiles at 8)
  if (var == V_SX32_F8V1W7T14E && !list && d->grid_dims[1] > 1) var = V_SX32_F8V1W7_T8X7E;
  // 2D grids with 64 frames: shallow 16 x 4 tiles keep the windows short enough for the
  // 8-slot ring of 512-byte rows (the squarest 8 x 8 tiles do not fit; the L1 path then
  // ran 256 x 256 px at 1.47 against 2.11 T points/s)
  if (var == V_SX64_C64P && !list && d->grid_dims[1] == 1) var = V_SX64_C64P_T16;
  if (d->term_table) var = generic_staged(var);
  const bool forced = g_force_variant >= 0;
  if (forced) {
    if (g_force_variant >= V_COUNT || !variant_accepts(static_cast<Variant>(g_force_variant), d->iq_dtype, F))
      return MACH_ERR_UNSUPPORTED;
    var = static_cast<Variant>(g_force_variant);
  }

  DasParams b{};
  if (list) {
    b.nx = static_cast<int>(V);
    b.ny = b.nz = 1;
  } else {
    b.nx = d->grid_dims[0];
    b.ny = d->grid_dims[1];
    b.nz = d->grid_dims[2];
  }
  if ((st = configure_tiles(b, var, list, V, F)) != MACH_OK) return st;
  const int64_t tiles0 = static_cast<int64_t>(b.tiles_x) * b.tiles_y * b.tiles_z;

  // host-side size check before touching the device
  const size_t need = static_cast<size_t>(V) * (sizeof(float4) + sizeof(float) * T) + sizeof(float4) * C +
                      (b.frame_tiles > 1 ? sizeof(float) * V * b.frame_tiles : 0) +
                      (list ? sizeof(float) * 3 * V : 0) + sizeof(double) * 3 * T +
                      (variant_shape(var).staged ? static_cast<size_t>(tiles0) * (2 * sizeof(float4) + T * sizeof(float2)) : 0);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return MACH_ERR_CUDA;
  }
  if (need > free_b) return MACH_ERR_OOM;

  mach_plan_s* p = new (std::nothrow) mach_plan_s();
  if (!p) return MACH_ERR_OOM;
  p->d = *d;
  p->d.elem_pos = nullptr;
  p->d.vox_pos = nullptr;
  p->d.tx_angles = nullptr;
  p->d.tx_table_dev = nullptr;
  p->d.n_vox = V;
  p->variant = var;
  cudaGetDevice(&p->device);

  const double k = d->fs / d->c;
  const double t0fs = d->t0 * d->fs;
  std::vector<float4> elem(C);
  for (int c = 0; c < C; ++c)
    elem[c] = make_float4(static_cast<float>(static_cast<double>(d->elem_pos[3 * c]) * k),
                          static_cast<float>(static_cast<double>(d->elem_pos[3 * c + 1]) * k),
                          static_cast<float>(static_cast<double>(d->elem_pos[3 * c + 2]) * k), 0.0f);
  std::vector<double> u;
  if (!d->tx_table_dev) {
    u.resize(3 * static_cast<size_t>(T));
    for (int t = 0; t < T; ++t) {
      const double az = d->tx_angles[2 * t], el = d->tx_angles[2 * t + 1];
      u[3 * t] = std::sin(az) * std::cos(el);
      u[3 * t + 1] = std::sin(el);
      u[3 * t + 2] = std::cos(az) * std::cos(el);
    }
  }

  float* d_raw = nullptr;
  double* d_u = nullptr;
  int* d_stats = nullptr;
  int64_t scratch_bytes = 0;
  auto fail = [&](mach_status e) {
    cudaFree(d_raw);
    cudaFree(d_u);
    cudaFree(d_stats);
    release(p);
    return e;
  };
  if ((st = dev_alloc(reinterpret_cast<void**>(&p->d_vox), sizeof(float4) * V, &p->device_bytes)) != MACH_OK) return fail(st);
  if ((st = dev_alloc(reinterpret_cast<void**>(&p->d_elem), sizeof(float4) * C, &p->device_bytes)) != MACH_OK) return fail(st);
  if ((st = dev_alloc(reinterpret_cast<void**>(&p->d_tx), sizeof(float) * T * V, &p->device_bytes)) != MACH_OK) return fail(st);
  if ((st = dev_alloc(reinterpret_cast<void**>(&p->d_err), sizeof(int), &p->device_bytes)) != MACH_OK) return fail(st);
  if (list && (st = dev_alloc(reinterpret_cast<void**>(&d_raw), sizeof(float) * 3 * V, &scratch_bytes)) != MACH_OK)
    return fail(st);
  if (!u.empty() && (st = dev_alloc(reinterpret_cast<void**>(&d_u), sizeof(double) * u.size(), &scratch_bytes)) != MACH_OK)
    return fail(st);

  if (cudaMemsetAsync(p->d_err, 0, sizeof(int), s) != cudaSuccess) return fail(MACH_ERR_CUDA);
  if (cudaMemcpyAsync(p->d_elem, elem.data(), sizeof(float4) * C, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail(MACH_ERR_CUDA);
  if (list && cudaMemcpyAsync(d_raw, d->vox_pos, sizeof(float) * 3 * V, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail(MACH_ERR_CUDA);
  if (d_u && cudaMemcpyAsync(d_u, u.data(), sizeof(double) * u.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail(MACH_ERR_CUDA);

  TableParams tp{};
  tp.raw_vox = d_raw;
  tp.u = d_u;
  tp.tx_seconds = d->tx_table_dev;
  tp.k = k;
  tp.t0fs = t0fs;
  tp.fs = d->fs;
  for (int a = 0; a < 3; ++a) {
    tp.origin[a] = list ? 0.0 : d->grid_origin[a];
    tp.step[a] = list ? 0.0 : d->grid_step[a];
  }
  tp.nx = list ? 1 : d->grid_dims[0];
  tp.ny = list ? 1 : d->grid_dims[1];
  tp.nz = list ? 1 : d->grid_dims[2];
  tp.V = V;
  tp.T = T;
  tp.vox_out = p->d_vox;
  tp.tx_out = p->d_tx;
  if (launch_tables(tp, s) != cudaSuccess) return fail(MACH_ERR_CUDA);

  b.vox = p->d_vox;
  b.elem = p->d_elem;
  b.tx = p->d_tx;
  b.pd_part = p->d_pd_part;
  b.V = V;
  b.C = C;
  b.T = T;
  b.S = S;
  b.F = F;
  b.ystride = F;
  b.txr_stride = T;
  b.apod = d->apod;
  b.two_f = static_cast<float>(2.0 * d->f_number);
  b.f_num = static_cast<float>(d->f_number);
  b.four_f2 = static_cast<float>(4.0 * d->f_number * d->f_number);
  b.f_num2 = static_cast<float>(d->f_number * d->f_number);
  b.s_max = static_cast<float>(S - 1);
  b.r_f = static_cast<float>(d->fc / d->fs);
  b.phase_R = fixed_cycles(d->fc / d->fs);
  b.phase_Phi = fixed_cycles(d->fc * d->t0);
  b.err = p->d_err;
  b.wait_limit = g_wait_limit ? g_wait_limit : kDefaultWaitLimit;
  b.debug_stall = g_stall;

  if (variant_shape(var).staged) {
    // per-tile bounds, ring size, and the number of windows one run copies.  When the
    // chosen variant's ring does not fit, variants with fewer ring slots are tried in turn
    // (their tiles differ, so each gets its own bounds), and last the L1-path variant.
    const bool tab = d->term_table != 0;
    Variant chain[4];
    int nchain = 0;
    chain[nchain++] = var;
    if (!forced)
      for (Variant f = staged_fallback(var); f != chain[nchain - 1] && nchain < 4; f = staged_fallback(f))
        chain[nchain++] = f;
    int64_t tiles_max = tiles0;
    for (int k = 1; k < nchain; ++k) {
      DasParams tmp = b;
      if ((st = configure_tiles(tmp, chain[k], list, V, F)) != MACH_OK) return fail(st);
      tiles_max = std::max<int64_t>(tiles_max, static_cast<int64_t>(tmp.tiles_x) * tmp.tiles_y * tmp.tiles_z);
    }
    if ((st = dev_alloc(reinterpret_cast<void**>(&p->d_tbox), sizeof(float4) * 2 * tiles_max, &p->device_bytes)) != MACH_OK)
      return fail(st);
    if ((st = dev_alloc(reinterpret_cast<void**>(&p->d_txr), sizeof(float2) * T * tiles_max, &p->device_bytes)) != MACH_OK)
      return fail(st);
    if ((st = dev_alloc(reinterpret_cast<void**>(&d_stats), 2 * sizeof(int), &scratch_bytes)) != MACH_OK) return fail(st);
    b.tbox = p->d_tbox;
    b.txr = p->d_txr;
    bool fits = false;
    for (int k = 0; k < nchain && !fits; ++k) {
      if (k > 0) {
        var = chain[k];
        p->variant = var;
        if ((st = configure_tiles(b, var, list, V, F)) != MACH_OK) return fail(st);
      }
      if (launch_tile_bounds(b, p->d_tbox, p->d_txr, d_stats, s) != cudaSuccess) return fail(MACH_ERR_CUDA);
      int stats[2] = {0, 0};
      if (cudaMemcpyAsync(stats, d_stats, sizeof(stats), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return fail(MACH_ERR_CUDA);
      if (cudaStreamSynchronize(s) != cudaSuccess) return fail(MACH_ERR_CUDA);
      p->rows_cap = std::max(2, stats[0]);
      p->copy_pairs = stats[1];
      b.rows_cap = p->rows_cap;
      fits = staged_smem_bytes(var, p->rows_cap, F, T, tab) <= kStagedSmemCap;
    }
    if (!fits) {
      if (forced || tab) return fail(MACH_ERR_UNSUPPORTED);
      // the tiles' windows are too long for any ring: use the L1-cached variant
      cudaFree(p->d_tbox);
      cudaFree(p->d_txr);
      p->d_tbox = nullptr;
      p->d_txr = nullptr;
      b.tbox = nullptr;
      b.txr = nullptr;
      p->device_bytes -= static_cast<int64_t>(sizeof(float4) * 2 * tiles_max + sizeof(float2) * T * tiles_max);
      var = unstaged(var);
      p->variant = var;
      p->rows_cap = 0;
      p->copy_pairs = 0;
      if ((st = configure_tiles(b, var, list, V, F)) != MACH_OK) return fail(st);
    }
  }
  // partial Power Doppler sums when the frames span several frame tiles (known once the
  // variant is final)
  if (b.frame_tiles > 1 &&
      (st = dev_alloc(reinterpret_cast<void**>(&p->d_pd_part), sizeof(float) * b.frame_tiles * V, &p->device_bytes)) != MACH_OK)
    return fail(st);
  b.pd_part = p->d_pd_part;
  if (d->term_table) {
    // every term evaluated once here; runs read them instead of computing them
    if (!variant_shape(var).staged || !table_supported(var)) return fail(MACH_ERR_UNSUPPORTED);
    if ((st = build_term_table(p, b, s)) != MACH_OK) return fail(st);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(MACH_ERR_CUDA);
  cudaFree(d_raw);
  cudaFree(d_u);
  cudaFree(d_stats);
  d_raw = nullptr;
  d_u = nullptr;
  d_stats = nullptr;
  p->base = b;
  *out = p;
  return MACH_OK;
}

mach_status mach_plan_destroy(mach_plan p) {
  if (!p) return MACH_OK;
  release(p);
  return MACH_OK;
}

static mach_status run(mach_plan p, const void* iq, float* pd, void* y, void* stream) {
  if (!p || !iq || (!pd && !y)) return MACH_ERR_INVALID_ARG;
  // vector loads and bulk copies need 16-byte aligned IQ; outputs are float2 / float4
  if ((reinterpret_cast<uintptr_t>(iq) & 15u) || (reinterpret_cast<uintptr_t>(y) & 15u) ||
      (reinterpret_cast<uintptr_t>(pd) & 3u))
    return MACH_ERR_INVALID_ARG;
  DasParams q = p->base;
  q.iq = iq;
  q.y = static_cast<float2*>(y);
  q.pd = pd;
  const cudaError_t e = p->table ? launch_das_table(q, p->variant, static_cast<cudaStream_t>(stream))
                                 : launch_das(q, p->variant, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? MACH_OK : MACH_ERR_CUDA;
}

mach_status mach_das_run(mach_plan p, const void* iq_dev, void* y_dev, void* stream) {
  if (!y_dev) return MACH_ERR_INVALID_ARG;
  return run(p, iq_dev, nullptr, y_dev, stream);
}

mach_status mach_das_run_per_tx(mach_plan p, const void* iq_dev, void* y_dev, void* stream) {
  if (!p || !iq_dev || !y_dev) return MACH_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(iq_dev) & 15u) || (reinterpret_cast<uintptr_t>(y_dev) & 15u))
    return MACH_ERR_INVALID_ARG;
  const DasParams& b = p->base;
  const int T = b.T, F = b.F;
  // bytes of one transmit's IQ block [C][S][F] (split rows hold the same values)
  const size_t sample_bytes = (p->d.iq_dtype == MACH_IQ_F16X2 || p->d.iq_dtype == MACH_IQ_BF16X2) ? 4 : 8;
  const size_t tx_bytes = sample_bytes * static_cast<size_t>(b.C) * b.S * F;
  // vector stores need each transmit's slice of a row on the same alignment as the row
  const int vec = F % 4 == 0 ? 4 : (F % 2 == 0 ? 2 : 1);
  if ((static_cast<int64_t>(T) * F) % vec) return MACH_ERR_UNSUPPORTED;
  for (int t = 0; t < T; ++t) {
    DasParams q = b;
    q.T = 1;
    q.tx = b.tx + static_cast<size_t>(t) * b.V;
    q.txr = b.txr ? b.txr + t : nullptr;
    q.iq = static_cast<const char*>(iq_dev) + t * tx_bytes;
    q.y = static_cast<float2*>(y_dev) + static_cast<size_t>(t) * F;
    q.ystride = static_cast<int64_t>(T) * F;
    q.pd = nullptr;
    const cudaError_t e = launch_das(q, p->variant, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return MACH_ERR_CUDA;
  }
  return MACH_OK;
}

mach_status mach_power_doppler(mach_plan p, const void* iq_dev, float* pd_dev, void* y_dev_or_null,
                               void* stream) {
  if (!pd_dev) return MACH_ERR_INVALID_ARG;
  return run(p, iq_dev, pd_dev, y_dev_or_null, stream);
}

mach_status mach_plan_get_info(mach_plan p, mach_plan_info* info) {
  if (!p || !info) return MACH_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  const VariantShape& s = variant_shape(p->variant);
  std::strncpy(info->variant, s.name, sizeof(info->variant) - 1);
  info->frames_per_lane = s.frames_per_lane;
  info->lanes_per_voxel = s.lanes_per_voxel;
  info->voxels_per_cta = s.voxels_per_warp * s.warps;
  info->threads_per_cta = s.warps * 32;
  info->tile[0] = p->base.tile_x;
  info->tile[1] = p->base.tile_y;
  info->tile[2] = p->base.tile_z;
  info->frame_tiles = p->base.frame_tiles;
  info->ctas = static_cast<int64_t>(p->base.tiles_x) * p->base.tiles_y * p->base.tiles_z * p->base.frame_tiles;
  info->smem_bytes = static_cast<int64_t>(das_smem_bytes(p->variant));
  info->device_bytes = p->device_bytes;
  info->ring_rows = p->rows_cap;
  info->ring_slots = variant_shape(p->variant).ring_slots;
  info->copy_pairs = p->copy_pairs;
  info->term_table_bytes = p->table_bytes;
  if (variant_shape(p->variant).staged) {
    info->smem_bytes = static_cast<int64_t>(staged_smem_bytes(p->variant, p->rows_cap, p->base.F, p->base.T, p->table));
    info->threads_per_cta = (s.warps + 1) * 32;
  }
  return MACH_OK;
}

mach_status mach_plan_device_status(mach_plan p, void* stream) {
  if (!p) return MACH_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int err = 0;
  if (cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MACH_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MACH_ERR_CUDA;
  if (err == 0) return MACH_OK;
  if (cudaMemsetAsync(p->d_err, 0, sizeof(int), s) != cudaSuccess) return MACH_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MACH_ERR_CUDA;
  return MACH_ERR_TIMEOUT;
}

mach_status mach_debug_force_variant(const char* name) {
  if (!name || !*name) {
    g_force_variant = -1;
    return MACH_OK;
  }
  for (int v = 0; v < V_COUNT; ++v)
    if (std::strcmp(variant_shape(static_cast<Variant>(v)).name, name) == 0) {
      g_force_variant = v;
      return MACH_OK;
    }
  return MACH_ERR_INVALID_ARG;
}

void mach_debug_set_wait_limit(uint32_t polls) { g_wait_limit = polls; }

void mach_debug_stall_producer(int32_t on) { g_stall = on ? 1 : 0; }

mach_status mach_plan_tx_table(mach_plan p, float* out_dev, void* stream) {
  if (!p || !out_dev) return MACH_ERR_INVALID_ARG;
  const size_t bytes = sizeof(float) * static_cast<size_t>(p->base.T) * p->base.V;
  return cudaMemcpyAsync(out_dev, p->d_tx, bytes, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? MACH_OK
             : MACH_ERR_CUDA;
}

mach_status mach_das_terms(mach_plan p, const int64_t* vox_idx_dev, int64_t n, int32_t* i0_dev, float* w_dev,
                           float* cw_dev, void* stream) {
  if (!p || n < 0 || (n > 0 && !vox_idx_dev)) return MACH_ERR_INVALID_ARG;
  return launch_terms(p->base, vox_idx_dev, n, i0_dev, w_dev, cw_dev, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? MACH_OK
             : MACH_ERR_CUDA;
}

}  // extern "C"

namespace mach {
// Host steps shared with the allocation-free entry point (noalloc.cu): the same
// validation, choice among the non-staged kernels, voxel tiling and phase constants
// that a plan uses.
mach_status host_validate(const mach_das_desc* d) { return validate(d); }
Variant host_unstaged_variant(int iq_dtype, int F) { return unstaged(pick_variant(iq_dtype, F)); }
mach_status host_configure_tiles(DasParams& b, Variant v, bool list, int64_t V, int F) {
  return configure_tiles(b, v, list, V, F);
}
uint32_t host_fixed_cycles(double cycles) { return fixed_cycles(cycles); }
}  // namespace mach

namespace mach {
const DasParams* plan_params(mach_plan p) { return p ? &p->base : nullptr; }
int plan_iq_dtype(mach_plan p) { return p ? p->d.iq_dtype : -1; }
void pick_tile_shape(int n, int nx, int ny, int nz, bool list, int tile[3]) { pick_tile(n, nx, ny, nz, list, tile); }
}  // namespace mach
