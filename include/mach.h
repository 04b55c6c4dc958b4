/*
 * mach.h -- C ABI of the GB300 delay-and-sum (DAS) beamforming library.
 *
 * Method: delay-and-sum of baseband IQ channel data from plane-wave acquisitions
 * (arXiv 2604.06257, Sec. 2.1): for every voxel, compute the round-trip delay to each
 * receiving element, interpolate the received signal at that delay, and sum coherently
 * over elements and compounded transmits; Power Doppler sums |.|^2 over the frame
 * ensemble (Sec. 5).  Transmit arrival times are precomputed once per plan and receive
 * delays are computed on the fly (hybrid delays, Sec. 4.3).  Work is counted with Eq. 1:
 * voxels x channels x transmits x frames.
 *
 * Conventions (all entry points):
 *  - Units: metres, seconds, hertz, radians.  Axes x lateral, y elevation, z depth; the
 *    array lies in z = 0 for the aperture rule.
 *  - IQ layout in device memory: [n_tx][n_elem][n_samples][n_frames], frames contiguous
 *    (Sec. 4.4 stores [elements, samples, frames]; this ABI adds the transmit axis in
 *    front).  Element type: MACH_IQ_C64 = interleaved float32 (re, im) ("complex64",
 *    Sec. 4.1); MACH_IQ_F16X2 / MACH_IQ_BF16X2 = interleaved float16 / bfloat16 (re, im),
 *    widened to float32 before any arithmetic; MACH_IQ_C64_SPLIT = complex64 values with
 *    every [sample] row stored as F real parts followed by F imaginary parts.
 *  - Output layout: y complex64 [n_vox][n_frames] (frames contiguous); Power Doppler
 *    float32 [n_vox].  Voxel order = the order of vox_pos, or for a regular grid
 *    v = ix + nx*(iy + ny*iz).
 *  - Ownership: the caller owns every IQ and output buffer.  A plan copies every host
 *    array it is given at creation and owns its device tables; it never keeps a caller
 *    pointer.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Run calls
 *    are stream-ordered and asynchronous; they never synchronise the host.
 *  - Errors: arguments are checked before anything is launched; a call that returns an
 *    error before launching leaves the outputs untouched.  CUDA errors map to
 *    MACH_ERR_CUDA.  No C++ exception crosses this boundary.
 *  - Threads: a plan is read-only after creation.  Calls that share a plan may run on
 *    different streams concurrently, except when mach_plan_info.frame_tiles > 1 and
 *    Power Doppler is requested (those calls share the plan's partial-sum scratch and
 *    must be ordered on one stream).
 */
#ifndef MACH_H
#define MACH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MACH_OK = 0,
    MACH_ERR_INVALID_ARG = 1,   /* a NULL pointer, a size out of range, inconsistent geometry */
    MACH_ERR_CUDA = 2,          /* a CUDA runtime call or a launch failed                     */
    MACH_ERR_OOM = 3,           /* device allocation failed, or the plan would not fit        */
    MACH_ERR_UNSUPPORTED = 4,   /* valid request outside what this library implements        */
    MACH_ERR_TIMEOUT = 5        /* a bounded device-side wait gave up                         */
} mach_status;

/* F-number aperture windows (Sec. 4.1 "f-number").  With rho the lateral distance
 * voxel-element and dz the depth difference, an element contributes iff dz > 0 and
 * rho * 2 * f_number <= dz.  Window of t = rho * f_number / dz in [0, 1/2]:
 * BOXCAR 1, HANN cos^2(pi t), GAUSS exp(-8 t^2).  NONE: every element, weight 1. */
typedef enum {
    MACH_APOD_NONE = 0,
    MACH_APOD_BOXCAR = 1,
    MACH_APOD_HANN = 2,
    MACH_APOD_GAUSS = 3
} mach_apod;

typedef enum {
    MACH_IQ_C64 = 0,     /* float32 (re, im) per sample, 8 bytes */
    MACH_IQ_F16X2 = 1,   /* float16 (re, im) per sample, 4 bytes */
    MACH_IQ_BF16X2 = 2,  /* bfloat16 (re, im) per sample, 4 bytes */
    MACH_IQ_C64_SPLIT = 3 /* complex64 with each sample row split: the n_frames real parts,
                             then the n_frames imaginary parts (float32); n_frames a
                             multiple of 4 and > 4.  Lets the kernels accumulate two frames
                             per packed FP32x2 instruction */
} mach_iq_dtype;

/* Orders of channel data accepted by mach_iq_convert. */
typedef enum {
    MACH_ORDER_TCSF = 0,   /* [transmit][element][sample][frame]: the layout the kernels read */
    MACH_ORDER_FTCS = 1    /* [frame][transmit][element][sample]: acquisition order          */
} mach_iq_order;

typedef struct mach_plan_s *mach_plan;

/* Everything a plan needs (the inputs of Sec. 3.3's workflow and Table 3). */
typedef struct {
    int32_t ndim;                /* 2 (all y = 0, elevation angles 0) or 3               */
    int32_t n_elem;              /* receiving elements (channels), >= 1                  */
    const float *elem_pos;       /* host [n_elem][3] element positions, metres           */
    int64_t n_vox;               /* voxels: size of vox_pos, or 0 / nx*ny*nz for a grid  */
    const float *vox_pos;        /* host [n_vox][3] voxel positions, or NULL -> grid     */
    int32_t grid_dims[3];        /* regular grid (nx, ny, nz), x fastest                 */
    double grid_origin[3];       /* position of voxel (0, 0, 0), metres                  */
    double grid_step[3];         /* spacing per axis, metres                             */
    int32_t n_tx;                /* transmits compounded coherently, >= 1                */
    const double *tx_angles;     /* host [n_tx][2] plane-wave (azimuth, elevation), rad;
                                    direction u = (sin az cos el, sin el, cos az cos el),
                                    wavefront at the array origin at t = 0               */
    const float *tx_table_dev;   /* optional DEVICE [n_tx][n_vox] transmit arrival times
                                    in seconds (e.g. from a simulator, Sec. 3.3/4.3);
                                    when set it replaces the plane-wave model and
                                    tx_angles may be NULL.  Read during mach_das_plan only */
    double fs;                   /* IQ sampling rate, Hz, > 0                            */
    double fc;                   /* demodulation (centre) frequency, Hz, >= 0            */
    double c;                    /* speed of sound, m/s, > 0                             */
    double t0;                   /* time of sample 0, s                                  */
    double f_number;             /* >= 0                                                  */
    int32_t apod;                /* mach_apod                                            */
    int32_t n_samples;           /* samples per channel, 2 .. 2^24                       */
    int32_t n_frames;            /* frames (ensemble), >= 1                              */
    int32_t iq_dtype;            /* mach_iq_dtype                                        */
    int32_t term_table;          /* 0: receive delays, indices, weights and phases are
                                    computed in every run (Sec. 4.3's hybrid delays);
                                    1: the plan evaluates every term once and stores it
                                    (16 bytes per voxel slot and usable element-transmit
                                    pair of each voxel tile; mach_plan_info.
                                    term_table_bytes) and runs read the table instead.
                                    Same outputs bit for bit.  Plans only: the batch and
                                    allocation-free entry points need 0               */
} mach_das_desc;

/* Build a plan (Sec. 4.3 precompute): validates `d`, copies its host arrays, allocates
 * the device tables (voxel coordinates in sample units, element coordinates, the
 * transmit delay table [n_tx][n_vox] float32 built in FP64 on the device) and selects
 * the kernel variant.  Runs on `stream` and synchronises it before returning.
 * With term_table = 1 it also evaluates and stores every term (see mach_das_desc);
 * UNSUPPORTED when the selected kernel has no table form (ensembles of 16 frames or
 * fewer, or above 64, or sample windows too long for shared memory), OOM when the table
 * does not fit in free device memory.
 * Errors: INVALID_ARG (checked before any CUDA call), OOM, CUDA, UNSUPPORTED.
 * On error *out is set to NULL and nothing is leaked. */
mach_status mach_das_plan(const mach_das_desc *d, void *stream, mach_plan *out);

/* Delay-and-sum (Sec. 2.1 steps 1-3, compounding over all transmits):
 *   y[v][f] = sum_t sum_c a(v,c) e^{+j 2 pi fc (t0 + s/fs)} lerp(iq[t][c][.][f], s)
 * with s = s_tx(t,v) + |p_v - e_c| fs / c, linear interpolation between samples
 * floor(s) and floor(s)+1, and a term dropped unless 0 <= s < n_samples - 1.
 * iq_dev: device IQ as described above.  y_dev: device complex64 [n_vox][n_frames].
 * Errors: INVALID_ARG (NULL plan or pointer), CUDA. */
mach_status mach_das_run(mach_plan p, const void *iq_dev, void *y_dev, void *stream);

/* Ensemble Power Doppler (Sec. 5): pd[v] = sum_f |y[v][f]|^2, fused into the same
 * kernel as the DAS sums; y_dev_or_null additionally receives the complex frames
 * (B-mode data) when not NULL.  pd_dev: device float32 [n_vox].
 * Errors: INVALID_ARG, CUDA. */
mach_status mach_power_doppler(mach_plan p, const void *iq_dev, float *pd_dev,
                               void *y_dev_or_null, void *stream);

/* Power Doppler (Sec. 5) of `count` acquisitions held in HOST memory, pipelined: the
 * upload of acquisition k+1 overlaps the conversion and beamforming of k and the download
 * of k-1 (two device staging sets, separate upload / compute / download streams).
 *   iq_host[k]   host IQ of acquisition k: complex64 in `src_order` (MACH_ORDER_*), which
 *                K0 (mach_iq_convert) turns into the plan's layout on the device, or, with
 *                src_order = -1, already in the plan's layout and iq_dtype;
 *   pd_host[k]   host float32 [n_vox] receiving its Power Doppler;
 *   y_host       NULL, or y_host[k] = host complex64 [n_vox][n_frames] for its frames.
 * Host buffers should be pinned (page-locked) for the copies to overlap; the caller keeps
 * ownership.  Staging buffers and streams are allocated for the call and released before
 * it returns; the call returns when every result is in host memory.  Results are bitwise
 * those of mach_iq_convert + mach_power_doppler on each acquisition.
 * Errors: INVALID_ARG (NULL plan or pointer, count < 1, bad order), OOM, CUDA, and
 * TIMEOUT (the plan's device status, read and cleared after the last acquisition). */
mach_status mach_power_doppler_host_stream(mach_plan p, const void *const *iq_host, int32_t src_order,
                                           float *const *pd_host, void *const *y_host, int32_t count);

/* Channel-data preparation (K0): read complex64 IQ in `src_order` and write it in the
 * frame-contiguous layout [n_tx][n_elem][n_samples][n_frames] (Sec. 4.4's element,
 * sample, frame order with the transmit axis in front) as `dst_dtype` (float16 and
 * bfloat16 rounded to nearest even).  src_dev / dst_dev: distinct device buffers,
 * 8- and 4-byte aligned.  Stream-ordered; a bandwidth-bound transpose through shared
 * memory.  Errors: INVALID_ARG, UNSUPPORTED (grid limits), CUDA. */
mach_status mach_iq_convert(const void *src_dev, int32_t src_order, void *dst_dev, int32_t dst_dtype,
                            int32_t n_tx, int32_t n_elem, int32_t n_samples, int32_t n_frames,
                            void *stream);

/* RF input (Sec. 3: the method takes RF or IQ channel data): demodulate real RF samples
 * into the complex IQ that mach_das_run reads.
 *   rf_dev  float32 [n_tx][n_elem][n_rf][n_frames] (device), sample m at t0 + m / fs_rf;
 *   iq_dev  complex64 [n_tx][n_elem][n_iq][n_frames] (device), n_iq = (n_rf - 1) / decim + 1,
 *           sample n at t0 + n decim / fs_rf (so the plan's fs = fs_rf / decim, same t0);
 *   iq[n] = sum_{k<L} taps[k] rf[n decim + k - (L-1)/2] exp(-j 2 pi fc (t0 + (n decim + k - (L-1)/2) / fs_rf)),
 *           RF samples outside [0, n_rf) read as zero.
 * taps: host float [n_taps] low-pass filter (1 <= n_taps <= 128), copied.  For an echo
 * A g(t - tau) cos(2 pi fc (t - tau)) and a filter of unit DC gain that passes g's band and
 * stops 2 fc, iq approximates (A / 2) g(t - tau) exp(-j 2 pi fc tau), the IQ model of the
 * plan.  Arguments are checked before the launch; MACH_ERR_INVALID_ARG for bad sizes,
 * rates, taps or alignment; MACH_ERR_UNSUPPORTED above 4,194,240 IQ samples per channel
 * and frame, above 2^24 frames, or when 63 decim + n_taps exceeds 6144 (decimation above
 * about 95); CUDA.
 * Stream-ordered, asynchronous. */
mach_status mach_rf_to_iq(const float *rf_dev, void *iq_dev, int32_t n_tx, int32_t n_elem, int32_t n_rf,
                          int32_t n_frames, double fs_rf, double fc, double t0, const float *taps,
                          int32_t n_taps, int32_t decim, void *stream);

/* Uncompounded output (the output shape of the paper's memory table, Table 3: voxels x
 * compounded planes x frames): y_dev complex64 [n_vox][n_tx][n_frames], element
 * (v, t, f) = the delay-and-sum of transmit t alone, i.e. the terms of transmit t of
 * mach_das_run's sum (Sec. 2.1 before the coherent compounding over transmits).  One
 * launch per transmit on `stream`; same IQ layout, alignment and errors as mach_das_run
 * (MACH_ERR_UNSUPPORTED if a transmit's slice of an output row would break the vector
 * alignment the plan's kernel uses). */
mach_status mach_das_run_per_tx(mach_plan p, const void *iq_dev, void *y_dev, void *stream);

/* Release a plan and its device tables (synchronises the device).  NULL is a no-op. */
mach_status mach_plan_destroy(mach_plan p);

/* Static, NUL-terminated description of a status code. */
const char *mach_status_string(mach_status s);

/* ---- inspection (used by the parity tests; not needed for beamforming) --------- */

typedef struct {
    char variant[40];        /* kernel variant name                                    */
    int32_t frames_per_lane; /* frames accumulated by one thread                       */
    int32_t lanes_per_voxel; /* threads sharing one voxel (frames or channel slices)   */
    int32_t voxels_per_cta;  /* voxels of one thread block                             */
    int32_t threads_per_cta;
    int32_t tile[3];         /* voxel tile of one block (x, y, z)                      */
    int32_t frame_tiles;     /* blocks along the frame axis                            */
    int64_t ctas;            /* blocks of one run                                      */
    int64_t smem_bytes;      /* dynamic shared memory per block                        */
    int64_t device_bytes;    /* device memory held by the plan                         */
    int32_t ring_rows;       /* staged variants: sample rows per shared-memory slot     */
    int32_t ring_slots;      /* staged variants: slots in the ring (0 otherwise)        */
    int64_t copy_pairs;      /* staged variants: (tile, transmit, element) windows one
                                run copies; pairs no voxel can use are skipped          */
    int64_t term_table_bytes; /* device bytes of the term table (0 without one)         */
} mach_plan_info;

mach_status mach_plan_get_info(mach_plan p, mach_plan_info *info);

/* Copy the plan's transmit delay table, float32 [n_tx][n_vox] in samples
 * (s_tx = ((u.p)/c - t0) fs, or (arrival - t0) fs), into out_dev.  Stream-ordered. */
mach_status mach_plan_tx_table(mach_plan p, float *out_dev, void *stream);

/* Evaluate the per-term quantities exactly as the DAS kernels do, for n voxels:
 * outputs [n][n_elem][n_tx]: i0 (int32, -1 when the term is dropped by the range or
 * aperture rule), w = s - i0 (float32), complex weight a e^{j phi} (float32 pairs).
 * vox_idx_dev: device int64 [n].  Any output may be NULL.  Stream-ordered. */
mach_status mach_das_terms(mach_plan p, const int64_t *vox_idx_dev, int64_t n,
                           int32_t *i0_dev, float *w_dev, float *cw_dev, void *stream);

/* ---- ragged batches ---------------------------------------------------------- */

/* Lane mapping and voxel tile of one batch instance (chosen by an autotuner, or by
 * mach_batch_plan when not given).  mode 0: frame lanes, `frame_lanes` (2, 4, 8 or 16)
 * lanes share a voxel and each holds 4 frames, so 4 * frame_lanes >= n_frames; one
 * block covers 8 * 4 * (32 / frame_lanes) voxels (256 with 2 frame lanes, whose lanes
 * hold 2 voxels each); taps read through L1.  mode 1: channel
 * lanes (n_frames <= 4), 32 voxels per block.  mode 2: staged windows (the default for
 * n_frames > 16 that are not a multiple of 4; mode 0 for the other n_frames > 4):
 * `frame_lanes` 8 (n_frames <= 32) or 16 (n_frames <= 64), 4 frames per lane,
 * 7 * 4 * (32 / frame_lanes) voxels per block (a producer warp and 7 consumer warps); each usable (element, transmit) pair's sample
 * window is copied into a shared-memory ring and every term read from there (an instance
 * whose windows exceed the ring slot takes mode 0 when the shape was not given, else
 * mach_batch_plan returns UNSUPPORTED).  tile: the block's voxel box (x, y, z); its volume
 * must equal the block's voxel count (tile[1] = 1 in 2D), or all zero for the default box. */
typedef struct {
    int32_t mode;
    int32_t frame_lanes;
    int32_t tile[3];
} mach_tile_shape;

typedef struct mach_batch_s *mach_batch;

/* Plan a batch of n instances (each described as for mach_das_plan, all with the same
 * iq_dtype, not the split layout, n_frames <= 64): builds every instance's tables and one
 * work list of (instance, voxel tile) items, sorted by decreasing estimated cost, for
 * one persistent launch.  shapes: NULL or n entries.  Synchronises `stream`.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
mach_status mach_batch_plan(const mach_das_desc *descs, int32_t n, const mach_tile_shape *shapes,
                            void *stream, mach_batch *out);

/* Bind the device buffers of every instance (host arrays of n device pointers; per
 * instance y or pd may be NULL but not both).  Uploads the instance table on `stream`;
 * call again only when the buffers change. */
mach_status mach_batch_bind(mach_batch b, const void *const *iq_devs, void *const *y_devs,
                            float *const *pd_devs, void *stream);

/* Beamform every instance of the batch in one launch on `stream` (stream-ordered; no
 * host synchronisation, so it can be captured in a CUDA graph).  Runs on the same batch
 * must be ordered on one stream (they share the work counter). */
mach_status mach_batch_run(mach_batch b, void *stream);

typedef struct {
    int32_t instances;
    int32_t items;           /* (instance, tile) work items                    */
    int32_t blocks;          /* persistent blocks of one launch                */
    int32_t blocks_per_sm;
    int64_t points;          /* Eq. 1 points of one run (sum over instances)   */
} mach_batch_info;

mach_status mach_batch_get_info(mach_batch b, mach_batch_info *info, mach_tile_shape *shapes_or_null);
mach_status mach_batch_destroy(mach_batch b);

/* Synchronise `stream`, then report and clear the plan's device error word:
 * MACH_OK, or MACH_ERR_TIMEOUT when a bounded device-side wait of an earlier run on
 * this plan gave up (that run's outputs are then incomplete).  The staged kernels wait
 * on shared-memory barriers for their bulk copies; each wait polls a bounded number of
 * times (about a second) and then abandons the block instead of hanging the device. */
mach_status mach_plan_device_status(mach_plan p, void *stream);

/* Delay-and-sum (and Power Doppler) without allocating device memory.  The paper has
 * no counterpart: this is for callers that cannot call cudaMalloc -- code running where
 * the device allocator is off limits (a host callback, a real-time loop that must not
 * pay an allocation, a host framework that owns all device memory or enforces a memory
 * budget).  Instead of a plan's tables it uses one fixed device array inside the
 * library (8 MiB, held on every GPU that loads the library until the process exits).
 * Same arguments and results as mach_das_plan + mach_das_run / mach_power_doppler on
 * the non-staged kernels: `d` as for mach_das_plan (host arrays are copied on every
 * call), iq_dev as for mach_das_run, outputs y_dev_or_null (complex64 [n_vox][n_frames])
 * and/or pd_dev_or_null (float32 [n_vox]), at least one of them.
 * Errors: INVALID_ARG as for a plan or a NULL/misaligned buffer; UNSUPPORTED when the
 * tables exceed the 8 MiB array or when `stream` is being captured into a CUDA graph (the
 * call copies from host buffers that do not outlive it).  The tables are, each rounded up to a multiple of 256 B:
 * 16 B per voxel; 16 B per element; 4 B per voxel and transmit; 24 B per transmit for
 * plane waves (none with tx_table_dev); 12 B per voxel for a voxel list; 4 B per voxel
 * and frame tile for Power Doppler over more than one frame tile.  CUDA on a failed
 * copy or launch (the runtime's last error is cleared).  Nothing is enqueued on argument
 * errors, when the tables do not fit or during a capture.
 * The first call on a device looks up the array's device address (do it before any
 * stream capture) and keeps it for the life of the process: after cudaDeviceReset on that
 * device the kept address is stale, so do not call this again in that process.  Calls share the array, so calls that overlap on the GPU race;
 * order them on one stream.  Returns after the host arrays are copied; the
 * beamforming itself is stream-ordered. */
mach_status mach_das_run_noalloc(const mach_das_desc *d, const void *iq_dev, void *y_dev_or_null,
                                 float *pd_dev_or_null, void *stream);

/* Library version string, e.g. "mach-gb300 0.1.0 sm_103a". */
const char *mach_version(void);

/* Test hook: make the n-th device allocation from now fail (n >= 1); n <= 0 disarms.
 * Lets tests exercise the MACH_ERR_OOM clean-up path without exhausting memory. */
void mach_debug_fail_alloc_after(int32_t n);

/* Test hooks (process-wide, not thread-safe; read when a plan is created):
 *  - force the kernel variant named `name` (mach_plan_info.variant) for later plans, or
 *    restore the automatic choice with NULL / "".  INVALID_ARG for an unknown name;
 *    mach_das_plan returns UNSUPPORTED if the forced variant cannot serve the plan.
 *  - set the polls per bounded device wait (0 restores the default).
 *  - make the staged producer announce its copies without issuing them, so that the
 *    consumers' waits run out (exercises MACH_ERR_TIMEOUT without a fault). */
mach_status mach_debug_force_variant(const char *name);
void mach_debug_set_wait_limit(uint32_t polls);
void mach_debug_stall_producer(int32_t on);

#ifdef __cplusplus
}
#endif
#endif /* MACH_H */
