// batch.cpp -- ragged batches of DAS instances in one persistent launch (host side).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "mach.h"
#include "mach_internal.h"

using namespace mach;

struct mach_batch_s {
  int n = 0;
  int iq_dtype = 0;
  std::vector<mach_plan> plans;          // tables of each instance
  std::vector<BatchInstance> host_insts;
  std::vector<mach_tile_shape> shapes;
  BatchInstance* d_insts = nullptr;
  int2* d_items = nullptr;
  int* d_counter = nullptr;
  int n_items = 0;
  int grid = 0;
  int per_sm = 0;
  size_t slot_bytes = 128;               // ring slot of the staged path (largest staged window)
  std::vector<void*> bounds;             // per staged instance: tile boxes and transmit-delay ranges
  int64_t points = 0;
  bool bound = false;
};

namespace {

void release(mach_batch_s* b) {
  if (!b) return;
  for (mach_plan p : b->plans) mach_plan_destroy(p);
  for (void* q : b->bounds) cudaFree(q);
  cudaFree(b->d_insts);
  cudaFree(b->d_items);
  cudaFree(b->d_counter);
  delete b;
}

// Largest ring slot the staged path uses: eight slots plus the per-warp scratch then leave
// room for two blocks per SM.
constexpr size_t kBatchSlotCap = 11 * 1024;

int voxels_per_block(const mach_tile_shape& s) {
  if (s.mode == kBatchChannels) return 32;
  if (s.mode == kBatchStaged) return 7 * 4 * (32 / s.frame_lanes);   // 7 consumer warps + a producer warp
  if (s.frame_lanes == 2) return 8 * 2 * 16;   // 8 warps x 16 lane pairs x 2 voxels
  return 8 * 4 * (32 / s.frame_lanes);         // 8 warps x (32 / FL) lane groups x 4 voxels
}

// Default lane mapping (measured on the 64-instance float16 batch): channel lanes for
// F <= 4; staged windows for F > 16 when F is not a multiple of 4 (rows off the 16-byte
// grid: the L1 path then reads one sample per frame from global memory, the staged path
// from shared memory); frame lanes through L1 otherwise, as few lanes per voxel as cover F.
mach_tile_shape default_shape(int F) {
  mach_tile_shape s{};
  if (F <= 4) {
    s.mode = kBatchChannels;
    s.frame_lanes = 0;
  } else if (F > 16 && F % 4 != 0) {
    s.mode = kBatchStaged;
    s.frame_lanes = F <= 32 ? 8 : 16;
  } else {
    s.mode = kBatchFrames;
    s.frame_lanes = F <= 8 ? 2 : F <= 16 ? 4 : (F <= 32 ? 8 : 16);
  }
  return s;
}

// The frame-lane mapping an instance falls back to when its staged windows do not fit.
mach_tile_shape frames_shape(int F) {
  mach_tile_shape s{};
  s.mode = kBatchFrames;
  s.frame_lanes = F <= 8 ? 2 : F <= 16 ? 4 : (F <= 32 ? 8 : 16);
  return s;
}

// Default voxel box of a staged block: shallow and wide (a window spans ~2 sample rows
// per voxel of depth but a fraction of a row per voxel of width).
void staged_tile(int n, int nx, int ny, int nz, bool list, int tile[3]) {
  if (list || (ny == 1 && nz == 1)) {
    tile[0] = n; tile[1] = 1; tile[2] = 1;
  } else if (ny == 1) {
    tile[0] = n / 4; tile[1] = 1; tile[2] = 4;
  } else {   // 112 = 4 x 4 x 7, 56 = 4 x 2 x 7
    tile[0] = 4; tile[1] = n / 28; tile[2] = 7;
  }
}

}  // namespace

extern "C" {

mach_status mach_batch_plan(const mach_das_desc* descs, int32_t n, const mach_tile_shape* shapes, void* stream,
                            mach_batch* out) {
  if (!out) return MACH_ERR_INVALID_ARG;
  *out = nullptr;
  if (!descs || n < 1) return MACH_ERR_INVALID_ARG;
  const int dt = descs[0].iq_dtype;
  for (int i = 0; i < n; ++i) {
    mach_status st = host_validate(&descs[i]);
    if (st != MACH_OK) return st;
    if (descs[i].term_table) return MACH_ERR_UNSUPPORTED;
    if (descs[i].iq_dtype != dt) return MACH_ERR_INVALID_ARG;
    if (descs[i].n_frames > 64) return MACH_ERR_UNSUPPORTED;
    if (shapes) {
      const mach_tile_shape& s = shapes[i];
      if (s.mode == kBatchChannels) {
        if (descs[i].n_frames > 4) return MACH_ERR_INVALID_ARG;
      } else if (s.mode == kBatchStaged) {
        if (s.frame_lanes != 8 && s.frame_lanes != 16) return MACH_ERR_INVALID_ARG;
        if (4 * s.frame_lanes < descs[i].n_frames) return MACH_ERR_INVALID_ARG;
      } else if (s.mode == kBatchFrames) {
        if (s.frame_lanes != 2 && s.frame_lanes != 4 && s.frame_lanes != 8 && s.frame_lanes != 16)
          return MACH_ERR_INVALID_ARG;
        if (4 * s.frame_lanes < descs[i].n_frames) return MACH_ERR_INVALID_ARG;
      } else {
        return MACH_ERR_INVALID_ARG;
      }
      const bool zero = s.tile[0] == 0 && s.tile[1] == 0 && s.tile[2] == 0;
      if (!zero && (s.tile[0] < 1 || s.tile[1] < 1 || s.tile[2] < 1 ||
                    s.tile[0] * s.tile[1] * s.tile[2] != voxels_per_block(s)))
        return MACH_ERR_INVALID_ARG;
    }
  }
  if (dt == MACH_IQ_C64_SPLIT) return MACH_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mach_batch_s* b = new (std::nothrow) mach_batch_s();
  if (!b) return MACH_ERR_OOM;
  b->n = n;
  b->iq_dtype = dt;
  b->plans.assign(n, nullptr);
  b->host_insts.resize(n);
  b->shapes.resize(n);
  struct Item { int inst; int64_t tile; double cost; };
  std::vector<Item> items;
  for (int i = 0; i < n; ++i) {
    mach_status st = mach_das_plan(&descs[i], stream, &b->plans[i]);
    if (st != MACH_OK) {
      release(b);
      return st;
    }
    mach_tile_shape sh = shapes ? shapes[i] : default_shape(descs[i].n_frames);
    const DasParams base = *plan_params(b->plans[i]);
    DasParams p = base;
    const bool list = descs[i].vox_pos != nullptr;
    auto set_tiles = [&](mach_tile_shape& t) -> bool {
      int tile[3] = {t.tile[0], t.tile[1], t.tile[2]};
      if (tile[0] == 0) {
        if (t.mode == kBatchStaged) staged_tile(voxels_per_block(t), p.nx, p.ny, p.nz, list, tile);
        else pick_tile_shape(voxels_per_block(t), p.nx, p.ny, p.nz, list, tile);
      }
      if (tile[0] * tile[1] * tile[2] != voxels_per_block(t)) return false;
      t.tile[0] = tile[0];
      t.tile[1] = tile[1];
      t.tile[2] = tile[2];
      p.tile_x = tile[0];
      p.tile_y = tile[1];
      p.tile_z = tile[2];
      p.tiles_x = (p.nx + tile[0] - 1) / tile[0];
      p.tiles_y = (p.ny + tile[1] - 1) / tile[1];
      p.tiles_z = (p.nz + tile[2] - 1) / tile[2];
      return true;
    };
    if (!set_tiles(sh)) {
      if (sh.mode != kBatchStaged || shapes) {
        release(b);
        return MACH_ERR_UNSUPPORTED;
      }
      sh = frames_shape(descs[i].n_frames);
      if (!set_tiles(sh)) {
        release(b);
        return MACH_ERR_UNSUPPORTED;
      }
    }
    p.frame_tiles = 1;
    p.wb_x = p.wb_y = p.wb_z = 0;
    p.ystride = p.F;
    p.iq = nullptr;
    p.y = nullptr;
    p.pd = nullptr;
    if (sh.mode == kBatchStaged) {
      // per-tile bounds for the batch tiling, and the largest window; instances whose
      // windows exceed the ring slot take the frame-lane path instead
      const int64_t tiles = static_cast<int64_t>(p.tiles_x) * p.tiles_y * p.tiles_z;
      void *tb = nullptr, *tr = nullptr, *st = nullptr;
      if (cudaMalloc(&tb, sizeof(float4) * 2 * tiles) != cudaSuccess ||
          cudaMalloc(&tr, sizeof(float2) * p.T * tiles) != cudaSuccess ||
          cudaMalloc(&st, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(tb);
        cudaFree(tr);
        cudaFree(st);
        release(b);
        return MACH_ERR_OOM;
      }
      b->bounds.push_back(tb);
      b->bounds.push_back(tr);
      b->bounds.push_back(st);
      p.tbox = static_cast<float4*>(tb);
      p.txr = static_cast<float2*>(tr);
      p.txr_stride = p.T;
      int stats[2] = {0, 0};
      if (launch_tile_bounds(p, static_cast<float4*>(tb), static_cast<float2*>(tr), static_cast<int*>(st), s) != cudaSuccess ||
          cudaMemcpyAsync(stats, st, sizeof(stats), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        release(b);
        return MACH_ERR_CUDA;
      }
      p.rows_cap = std::max(2, stats[0]);
      const size_t sample = (dt == MACH_IQ_F16X2 || dt == MACH_IQ_BF16X2) ? 4 : 8;
      const size_t need = (static_cast<size_t>(p.rows_cap) * p.F * sample + 32 + 127) / 128 * 128;
      if (need <= kBatchSlotCap) {
        b->slot_bytes = std::max(b->slot_bytes, need);
      } else if (shapes) {
        release(b);
        return MACH_ERR_UNSUPPORTED;
      } else {
        sh = frames_shape(descs[i].n_frames);
        sh.tile[0] = sh.tile[1] = sh.tile[2] = 0;
        if (!set_tiles(sh)) {
          release(b);
          return MACH_ERR_UNSUPPORTED;
        }
      }
    }
    b->host_insts[i].p = p;
    b->host_insts[i].mode = sh.mode;
    b->host_insts[i].frame_lanes = sh.frame_lanes;
    b->shapes[i] = sh;
    const int64_t tiles = static_cast<int64_t>(p.tiles_x) * p.tiles_y * p.tiles_z;
    // estimated cost of one tile: voxels x elements x transmits x frame slots it occupies
    const double frames_slots = sh.mode == kBatchChannels ? 4.0 : (sh.mode == kBatchStaged ? 2.0 * sh.frame_lanes
                                                                                          : 4.0 * sh.frame_lanes);
    const double cost = static_cast<double>(voxels_per_block(sh)) * p.C * p.T * frames_slots;
    // an instance's deepest tiles (widest apertures) first, its shallow ones last
    for (int64_t t = tiles - 1; t >= 0; --t) items.push_back({i, t, cost});
    b->points += static_cast<int64_t>(p.V) * p.C * p.T * p.F;
  }
  if (items.size() > static_cast<size_t>(INT32_MAX)) {
    release(b);
    return MACH_ERR_UNSUPPORTED;
  }
  std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& c) { return a.cost > c.cost; });
  std::vector<int2> hitems(items.size());
  for (size_t k = 0; k < items.size(); ++k) hitems[k] = make_int2(items[k].inst, static_cast<int>(items[k].tile));
  b->n_items = static_cast<int>(items.size());
  if (cudaMalloc(&b->d_insts, sizeof(BatchInstance) * n) != cudaSuccess ||
      cudaMalloc(&b->d_items, sizeof(int2) * hitems.size()) != cudaSuccess ||
      cudaMalloc(&b->d_counter, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    release(b);
    return MACH_ERR_OOM;
  }
  if (cudaMemcpyAsync(b->d_items, hitems.data(), sizeof(int2) * hitems.size(), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(b->d_counter, 0, 2 * sizeof(int), s) != cudaSuccess ||
      cudaMemcpyAsync(b->d_insts, b->host_insts.data(), sizeof(BatchInstance) * n, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    release(b);
    return MACH_ERR_CUDA;
  }
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->per_sm = batch_blocks_per_sm(dt, b->slot_bytes);
  b->grid = std::max(1, std::min(b->n_items, sms * b->per_sm));
  *out = b;
  return MACH_OK;
}

mach_status mach_batch_bind(mach_batch b, const void* const* iq_devs, void* const* y_devs, float* const* pd_devs,
                            void* stream) {
  if (!b || !iq_devs) return MACH_ERR_INVALID_ARG;
  for (int i = 0; i < b->n; ++i) {
    void* y = y_devs ? y_devs[i] : nullptr;
    float* pd = pd_devs ? pd_devs[i] : nullptr;
    if (!iq_devs[i] || (!y && !pd)) return MACH_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(iq_devs[i]) & 15u) || (reinterpret_cast<uintptr_t>(y) & 15u) ||
        (reinterpret_cast<uintptr_t>(pd) & 3u))
      return MACH_ERR_INVALID_ARG;
  }
  for (int i = 0; i < b->n; ++i) {
    b->host_insts[i].p.iq = iq_devs[i];
    b->host_insts[i].p.y = static_cast<float2*>(y_devs ? y_devs[i] : nullptr);
    b->host_insts[i].p.pd = pd_devs ? pd_devs[i] : nullptr;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(b->d_insts, b->host_insts.data(), sizeof(BatchInstance) * b->n, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MACH_ERR_CUDA;
  b->bound = true;
  return MACH_OK;
}

mach_status mach_batch_run(mach_batch b, void* stream) {
  if (!b || !b->bound) return MACH_ERR_INVALID_ARG;
  return launch_batch(b->iq_dtype, b->d_insts, b->d_items, b->n_items, b->d_counter, b->grid, b->slot_bytes,
                      static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? MACH_OK
             : MACH_ERR_CUDA;
}

mach_status mach_batch_get_info(mach_batch b, mach_batch_info* info, mach_tile_shape* shapes_or_null) {
  if (!b || !info) return MACH_ERR_INVALID_ARG;
  info->instances = b->n;
  info->items = b->n_items;
  info->blocks = b->grid;
  info->blocks_per_sm = b->per_sm;
  info->points = b->points;
  if (shapes_or_null) std::memcpy(shapes_or_null, b->shapes.data(), sizeof(mach_tile_shape) * b->n);
  return MACH_OK;
}

mach_status mach_batch_destroy(mach_batch b) {
  release(b);
  return MACH_OK;
}

}  // extern "C"
