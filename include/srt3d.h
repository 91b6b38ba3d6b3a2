/*
 * srt3d.h - C ABI of the Sketched RT3D (SRT3D) hot path on one NVIDIA GB300
 * (sm_103a). Library: libsrt3d.so (built in-tree by
 * paper_2203_00952_gb300/build.py).
 *
 * Notation follows Tachella, Sheehan & Davies, "Sketched RT3D: How to
 * reconstruct billions of photons per second" (ICASSP 2022):
 *   x_p      photon time-of-arrival stamps, integers in [0, T-1]  (Sec. 2, Eq. 1)
 *   T        number of time bins of the stamp range               (Sec. 2, Eq. 1)
 *   y_b      per-pixel histogram, one bin per integer stamp       (Sec. 2, Eq. 2)
 *   m        number of sketch entries                             (Sec. 2, Eq. 3)
 *   z_l      sketch (1/n) sum_p exp(i w_l x_p), w_l = 2 pi l / T  (Sec. 2, Eq. 3)
 *   h        impulse response, hhat its transform                 (Sec. 2, Eqs. 1, 4)
 *   t_k, alpha_k, alpha_0   depths, signal and background probabilities
 *   N_r x N_c pixel array (rows x cols), pixel p = r * cols + c   (Sec. 3)
 *
 * Conventions for every entry point
 *   - Pointers marked "device" are CUDA device pointers on the context's
 *     device; "host" pointers are ordinary host memory. The caller owns every
 *     buffer it passes; the library owns only its internal scratch, its
 *     lookup tables and (for serving) the frame slots.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Compute
 *     entry points are asynchronous on that stream: they validate their
 *     arguments, launch, and return. Argument errors return synchronously
 *     and launch nothing.
 *   - Errors detected by a kernel (a stamp >= T, a malformed offset array, a
 *     histogram count above 65535) are latched in the context and returned by
 *     the next srt3d_sync() on that stream. Kernels never trap: the offending
 *     photon / pixel is skipped and the flag is set.
 *   - There is no CPU fallback. Without a usable CUDA device srt3d_create()
 *     returns SRT3D_ECUDA.
 *   - A context may be used from one thread at a time for the compute entry
 *     points; the serving entry points (srt3d_submit / srt3d_poll) are
 *     internally locked and may be called from any thread.
 *   - The first call with a new T (lookup tables) or a larger problem size
 *     (scratch) allocates and synchronises; later calls with the same or
 *     smaller sizes do not. Make such a first call before capturing a stream.
 */
#ifndef SRT3D_H
#define SRT3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int srt3d_status;

enum {
  SRT3D_OK = 0,
  SRT3D_EINVAL = -1,    /* invalid argument (synchronous)                      */
  SRT3D_ENOMEM = -2,    /* device or host allocation failed                    */
  SRT3D_ERANGE = -3,    /* a stamp >= T or a count > 65535 was seen (latched)  */
  SRT3D_ECUDA = -4,     /* CUDA runtime error; see srt3d_last_error()          */
  SRT3D_EAGAIN = -5,    /* serving: result not ready yet                       */
  SRT3D_ETIMEDOUT = -6, /* serving: poll timed out, or a device wait gave up   */
  SRT3D_EBUSY = -7,     /* serving: frame not admitted now (HBM budget/slots)  */
  SRT3D_ENOTFOUND = -8, /* serving: unknown frame id                           */
  SRT3D_EOFFSETS = -9   /* malformed CSR offsets seen by a kernel (latched)    */
};

/* Arithmetic of the histogram sketch (srt3d_sketch_hist). */
enum {
  SRT3D_FP32 = 0,       /* FP32 CUDA-core product with exact integer phases    */
  SRT3D_FP16_SPLIT = 1, /* tensor cores: FP16 counts x (F_hi + F_lo) FP16,
                           FP32 accumulation in TMEM                           */
  SRT3D_BF16 = 2        /* tensor cores: BF16 counts x BF16 F, FP32 accumulate */
};

/* Initialisation of srt3d_reconstruct. */
enum {
  SRT3D_INIT_MATCHED = 0, /* per-pixel sketched matched filter                 */
  SRT3D_INIT_GIVEN = 1    /* start from the depth/alpha/active passed in       */
};

typedef struct srt3d_ctx srt3d_ctx;

/* Reconstruction parameters (Sec. 3; the RT3D iteration the paper cites).
 * Field order and types are part of the ABI. */
typedef struct srt3d_params {
  uint32_t iters;      /* SRT3D iterations after initialisation              */
  uint32_t k_max;      /* surfaces per pixel, 1..4                           */
  uint32_t radius;     /* APSS pixel window half-width, 1..3                 */
  int32_t init_mode;   /* SRT3D_INIT_MATCHED or SRT3D_INIT_GIVEN             */
  int32_t regularize;  /* 1: SRT3D (APSS + intensity smoothing);
                          0: pixelwise sketched estimate (no spatial prior)  */
  float apss_h;        /* APSS weight support, pixel pitches                 */
  float d_max;         /* neighbour depth gate and largest APSS move, bins,
                          in (0, 1e6]                                         */
  float depth_scale;   /* pixel pitches per time bin in point coordinates,
                          in (0, 1e3]                                         */
  float prune_alpha;   /* a point with alpha below this is removed           */
  float smooth_lambda; /* intensity smoothing weight in [0, 1]               */
  float min_sep;       /* init: least circular separation of 2 surfaces, bins */
  int32_t weighting;   /* data-term weight W of Eq. 6: 0 = identity (SRT3D);
                          1 = (Sigma_theta + 1e-3 I)^-1, Sigma_theta of Eq. 5 at
                          the current state, re-evaluated every iteration;
                          1 requires regularize = 0 (pixelwise estimate)      */
  uint32_t birth_every; /* RT3D birth move (cited by Sec. 3; this library's
                          reading: one step of orthogonal matching pursuit)
                          after every birth_every-th iteration but the last;
                          0 = none. Per pixel with a free slot: the residual of
                          the least-squares fit of z by the active points at
                          their depths, its matched filter over integer depths
                          at least min_sep (circularly) from the nearest
                          integer of every active depth, the argmax (smallest
                          on ties) with its coefficient in the joint
                          least-squares fit as intensity; born in the first
                          free slot if that reaches prune_alpha, then the
                          pixel's alphas are rescaled if they sum above 1.
                          Not available in batches.                           */
} srt3d_params;

/* Create a context on CUDA device `device`. hbm_budget_bytes bounds the device
 * memory the serving runtime may hold for admitted frames (0 = 3/4 of the
 * free memory at creation). *out receives the context. */
srt3d_status srt3d_create(int device, size_t hbm_budget_bytes, srt3d_ctx** out);

/* Destroy a context: waits for its work, frees its scratch, tables and slots. */
void srt3d_destroy(srt3d_ctx* ctx);

/* Static string naming a status code. */
const char* srt3d_status_string(srt3d_status status);

/* Message of the last error raised on this context (owned by the context,
 * valid until the next call on it). */
const char* srt3d_last_error(srt3d_ctx* ctx);

/* Synchronise `stream` and report errors latched by kernels since the last
 * srt3d_sync on this context: SRT3D_ERANGE (stamp >= T or count > 65535),
 * SRT3D_EOFFSETS (offsets not non-decreasing or beyond num_stamps), or
 * SRT3D_ECUDA. Clears the latched flags. */
srt3d_status srt3d_sync(srt3d_ctx* ctx, void* stream);

/* Per-pixel histogram of a pixel-sorted stamp stream (Sec. 2, Eq. 2 with
 * T' = T and unit bins: y_b = #{p : x_p = b}).
 *   stamps   device, uint16 [num_stamps], pixel-sorted (any 2-byte alignment)
 *   offsets  device, uint32 [num_pixels + 1], CSR: the photons of pixel p are
 *            stamps[offsets[p] .. offsets[p+1]); offsets[num_pixels] <= num_stamps
 *   T        1..65536
 *   hist     device, uint16 [num_pixels][T] row-major, overwritten
 * Counts above 65535 saturate and latch SRT3D_ERANGE. */
srt3d_status srt3d_hist_from_stream(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                    uint64_t num_stamps, uint32_t num_pixels, uint32_t T,
                                    uint16_t* hist, void* stream);

/* Photon sketch of a pixel-sorted stamp stream (Sec. 2, Eq. 3, unnormalised):
 *   S[p][l-1] = sum over the photons of pixel p of exp(i 2 pi k / T),
 *   k = (l * x_p) mod T, l = 1..m;  n[p] = count.
 *   How the phasors are formed (a reading of Eq. 3's exact phase; the error
 *   per term is bounded and tested): for T <= 8192 the phase of the first
 *   harmonic, x_p itself, indexes a cos/sin table exactly; harmonics 2..m
 *   follow the Chebyshev recurrence e_l = 2 cos(w_1 x_p) e_{l-1} - e_{l-2} in
 *   FP32, restarted from the table at the exact integer phase (l x_p) mod T
 *   every 8 harmonics when m > 10 (at most 3.5e-6 per term for m <= 10,
 *   2.3e-6 with restarts). For T > 8192 the table is two-level and harmonics
 *   come from complex rotation by e_1, resynchronised at the exact integer
 *   phase every 16 harmonics; for m <= 2, half of each 16-byte word's
 *   photons take e_1 from the special-function unit instead (phase reduced to
 *   [-pi, pi); same per-term bound). The sums are FP32.
 *   stamps, offsets, num_stamps, T as for srt3d_hist_from_stream
 *   m        1..32
 *   accumulate  0: overwrite S and n;  1: add into S and n (online update of
 *            Sec. 2: a frame's photons may arrive in chunks);  2: overwrite
 *            with the normalised sketch z = S / n (0 where n = 0) and n, the
 *            values srt3d_finalize would give bit for bit: a frame sketched
 *            in one call needs no separate finalize
 *   S        device, float [num_pixels][m][2] (re, im interleaved)
 *   n        device, uint32 [num_pixels]
 * Stamps >= T are skipped and latch SRT3D_ERANGE. */
srt3d_status srt3d_sketch_stream(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                 uint64_t num_stamps, uint32_t num_pixels, uint32_t T, uint32_t m,
                                 int accumulate, float* S, uint32_t* n, void* stream);

/* Sketch of histograms (Sec. 2, Eqs. 2-3): S[p][l-1] = sum_b y[p][b] exp(i 2 pi
 * ((l b) mod T) / T), n[p] = sum_b y[p][b], as the product Y[P x T] F[T x 2m].
 *   hist      device, uint16 [num_pixels][T] row-major; 16-byte aligned base
 *             for the tensor-core precisions
 *   T         1..65536 (tensor-core precisions: a multiple of 64, and
 *             num_pixels < 2^31)
 *   m         1..32
 *   precision SRT3D_FP32, SRT3D_FP16_SPLIT or SRT3D_BF16
 *   S, n      as for srt3d_sketch_stream (overwritten) */
srt3d_status srt3d_sketch_hist(srt3d_ctx* ctx, const uint16_t* hist, uint32_t num_pixels, uint32_t T,
                               uint32_t m, int precision, float* S, uint32_t* n, void* stream);

/* The stream sketch of srt3d_sketch_stream (Sec. 2, Eq. 3) computed through
 * the per-pixel histogram (Eq. 2, one bin per stamp value) and the tensor-core
 * histogram sketch: its cost follows num_pixels x T and hardly m or the
 * photons per pixel, so it is the faster route at large m or dense pixels.
 *   stamps, offsets, num_stamps, num_pixels, S, n  as for srt3d_sketch_stream
 *   (S and n are overwritten: no accumulate)
 *   T          a multiple of 64 in [64, 65536]; num_pixels < 2^31
 *   m          1..32
 *   precision  SRT3D_FP16_SPLIT or SRT3D_BF16 (as for srt3d_sketch_hist)
 * The histogram (num_pixels x T uint16) lives in a context-owned device
 * buffer: calls on one context must not overlap on different streams. A bin
 * above 65535 counts saturates and is reported by srt3d_sync. */
srt3d_status srt3d_sketch_stream_tc(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                    uint64_t num_stamps, uint32_t num_pixels, uint32_t T, uint32_t m,
                                    int precision, float* S, uint32_t* n, void* stream);

/* srt3d_sketch_stream_tc without the histogram in HBM (Sec. 2, Eqs. 2-3): the
 * stamps of every tile of 128 pixels are first counting-sorted by bin / 64
 * into 2-byte entries, then the tensor-core kernel builds each 128 x 64-bin
 * stage of the histogram in shared memory from its entries (shared-memory
 * atomics), converts it in place and multiplies it by the Fourier stage. HBM
 * traffic: the stamps read twice and their entries written and read once,
 * against the num_pixels x T histogram written and read by
 * srt3d_sketch_stream_tc. Same arguments, precisions and results: S and n are
 * bit-identical to srt3d_sketch_stream_tc's (the same integer counts enter
 * the same products), except that a pixel with more than 65535 stamps
 * counts only its first 65535 (reported by srt3d_sync as a count out of
 * range). Stamps >= T are skipped, offsets out of order or past num_stamps
 * leave the pixel empty; both are reported by srt3d_sync. The sorted entries
 * (2 bytes per stamp) and the bucket starts live in a context-owned device
 * buffer: calls on one context must not overlap on different streams. */
srt3d_status srt3d_sketch_stream_tc_fused(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                          uint64_t num_stamps, uint32_t num_pixels, uint32_t T, uint32_t m,
                                          int precision, float* S, uint32_t* n, void* stream);

/* Normalise sketch states (Sec. 2, Eq. 3): z = S / n, and z = 0 where n = 0.
 *   S  device float [P][m][2];  n device uint32 [P];  z device float [P][m][2]
 *   (z may alias S). */
srt3d_status srt3d_finalize(srt3d_ctx* ctx, const float* S, const uint32_t* n, uint32_t num_pixels,
                            uint32_t m, float* z, void* stream);

/* SRT3D reconstruction from sketches (Sec. 3, Eq. 8 with W = I): initialise
 * (matched filter or given), then params->iters iterations of: sketched
 * gradient step on every point, APSS depth projection and intensity
 * smoothing / pruning over pixel-grid neighbourhoods (the RT3D iteration that
 * Sec. 3 adopts). The matched-filter init takes k_max greedy passes: point k
 * maximises s(t) = Re sum_l conj(hhat_l e^{i w_l t}) r_l over integer t, r the
 * sketch minus the earlier points' fits, at least min_sep bins (circularly)
 * from every earlier point; the argmax is exact over all T candidates. With
 * regularize = 0 the iterations are the gradient step alone (pixelwise
 * sketched estimate), optionally with W = Sigma_theta^-1 (params->weighting,
 * Eq. 6). All iterations run in one cooperative launch when the frame's tiles
 * fit on the device at once, else one launch per iteration; results are the
 * same either way.
 *   z         device float [P][m][2], normalised sketches (srt3d_finalize)
 *   n         device uint32 [P] photon counts, P = rows * cols
 *   rows, cols  array size N_r x N_c, pixel p = r * cols + c
 *   T, m      time bins (2..65536) and sketch size (1..32)
 *   h         device float [T], impulse response by circular lag (peak at 0)
 *   params    host, see srt3d_params
 *   depth     device float [P][k_max], bins in [0, T)      (in/out)
 *   alpha     device float [P][k_max], probabilities        (in/out)
 *   active    device uint8 [P][k_max], 1 = point present    (in/out)
 *   alpha0    device float [P], background probability      (out)
 * With SRT3D_INIT_GIVEN depth/alpha/active are read as the initial state. */
srt3d_status srt3d_reconstruct(srt3d_ctx* ctx, const float* z, const uint32_t* n, uint32_t rows,
                               uint32_t cols, uint32_t T, uint32_t m, const float* h,
                               const srt3d_params* params, float* depth, float* alpha,
                               uint8_t* active, float* alpha0, void* stream);

/* One frame of a batch (srt3d_process_batch). All pointers are device
 * pointers owned by the caller; P = rows * cols. */
typedef struct srt3d_frame {
  const uint16_t* stamps;  /* uint16 [num_stamps], pixel-sorted (Sec. 2, Eq. 1)        */
  const uint32_t* offsets; /* uint32 [P + 1], CSR offsets                               */
  uint64_t num_stamps;
  uint32_t rows, cols;     /* N_r x N_c (Sec. 3)                                        */
  uint32_t T, m;           /* time bins, sketch size (Sec. 2, Eq. 3)                    */
  const float* h;          /* float [T], impulse response by circular lag              */
  float* z;                /* float [P][m][2]: out, normalised sketch (Eq. 3)           */
  uint32_t* n;             /* uint32 [P]: out, photon counts                            */
  float* depth;            /* float [P][k_max]: out                                     */
  float* alpha;            /* float [P][k_max]: out                                     */
  uint8_t* active;         /* uint8 [P][k_max]: out                                     */
  float* alpha0;           /* float [P]: out                                            */
} srt3d_frame;

/* Sketch, normalise and reconstruct a batch of frames of different sizes, T,
 * m and photon densities (Sec. 2, Eq. 3; Sec. 3, Eq. 8), each stage as one
 * launch over all frames, the whole batch as one CUDA graph. The first call
 * for a given set of frames (pointers and shapes) and params tunes the
 * sketch's lanes per pixel for any new photon-density class (a few timed
 * launches that write z and n), builds the work lists and captures the graph
 * (synchronising); later calls with the same frames only launch the graph on
 * `stream`. params->init_mode must be SRT3D_INIT_MATCHED and
 * params->regularize 1. Results equal those of srt3d_sketch_stream +
 * srt3d_finalize + srt3d_reconstruct per frame up to the FP32 summation
 * order of the sketch. Errors: those of srt3d_reconstruct per frame, a NULL
 * frame pointer, num_stamps >= 2^32 - 16 or rows * cols * m >= 2^32 in a
 * frame (SRT3D_EINVAL). */
srt3d_status srt3d_process_batch(srt3d_ctx* ctx, const srt3d_frame* frames, uint32_t num_frames,
                                 const srt3d_params* params, void* stream);

/* Allocation-free variant of srt3d_reconstruct (the paper has no
 * counterpart; same arguments and results). For callers that cannot allocate
 * device memory while they reconstruct: a real-time lidar loop in which
 * cudaMalloc/cudaFree (which may synchronise the device and take unbounded
 * time) is not allowed, or a process whose device memory is wholly reserved
 * by another allocator. It calls no cudaMalloc, cudaFree or other allocating
 * routine: its scratch and phase table live in one 16 MiB file-scope device
 * array that every GPU loading libsrt3d.so holds until the process exits.
 *   Limit: rows * cols * k_max <= 655360 points (e.g. 512x512 with k_max = 2);
 *   larger frames are rejected with SRT3D_EINVAL and a message.
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device made current); make that first call before any
 *   stream capture. A device reset (cudaDeviceReset) invalidates that address
 *   along with every context of the device: create a new context after a
 *   reset (srt3d_create drops the cached address, and the next call through
 *   any context looks it up again).
 *   Each call rewrites the phase table at the array's end from host values
 *   carried in kernel parameters (the same values srt3d_reconstruct uses, so
 *   the results are bit for bit those of srt3d_reconstruct).
 *   All calls share the array and it keeps the last call's contents (every
 *   word is rewritten before use, and the iterations' exchange words, which
 *   must start at zero, are cleared by each call itself): calls that overlap
 *   on the GPU (different streams or contexts of the same device) race and
 *   must be serialised by the caller. Frames of up to about 290 000 points
 *   (rows * cols * k_max) also fit the iterations' tagged exchange buffers;
 *   larger ones exchange state through progress flags (same results, slower).
 *   Profiling (srt3d_profile_enable) must be off: it creates CUDA events. */
srt3d_status srt3d_reconstruct_noalloc(srt3d_ctx* ctx, const float* z, const uint32_t* n, uint32_t rows,
                                       uint32_t cols, uint32_t T, uint32_t m, const float* h,
                                       const srt3d_params* params, float* depth, float* alpha,
                                       uint8_t* active, float* alpha0, void* stream);

/* Serving (continuous batching). A frame is opened by its first chunk,
 * receives photon chunks as host CSR arrays that are sketched online into a
 * device-resident per-pixel state, and is reconstructed after its last chunk.
 * Frames are admitted while their device state fits the context's HBM budget
 * and a slot is free; chunks of admitted frames and reconstructions of
 * different frames overlap on the device.
 *   frame_id   caller-chosen id, unique among frames in flight
 *   rows, cols, T, m, params  as for srt3d_reconstruct (read on the first chunk)
 *   h          host float [T] (read on the first chunk)
 *   chunk_stamps   host uint16 [chunk_offsets[rows*cols]], pixel-sorted
 *   chunk_offsets  host uint32 [rows*cols + 1]
 *   last_chunk flags: SRT3D_LAST_CHUNK on the frame's final chunk;
 *              SRT3D_CHUNK_KEEP: the caller keeps this chunk's arrays
 *              unchanged until the frame's srt3d_poll returns, so pinned
 *              (page-locked) chunk arrays are uploaded asynchronously and
 *              submit returns without waiting for the copy
 * Returns SRT3D_EBUSY (nothing consumed; retry later) when the frame cannot
 * be admitted yet. Without SRT3D_CHUNK_KEEP, and for pageable arrays always,
 * the host arrays are copied (or staged) before return. */
enum { SRT3D_LAST_CHUNK = 1, SRT3D_CHUNK_KEEP = 2 };
srt3d_status srt3d_submit(srt3d_ctx* ctx, uint64_t frame_id, uint32_t rows, uint32_t cols, uint32_t T,
                          uint32_t m, const float* h, const srt3d_params* params,
                          const uint16_t* chunk_stamps, const uint32_t* chunk_offsets, int last_chunk);

/* Wait up to timeout_us for frame_id's result and copy it to host buffers
 * depth/alpha [P][k_max] float, active [P][k_max] uint8, alpha0 [P] float and
 * (if not NULL) n [P] uint32. Returns SRT3D_OK and releases the frame;
 * SRT3D_ETIMEDOUT if it is not done within timeout_us (the frame stays
 * pending; poll again); SRT3D_ENOTFOUND for an unknown id; or the frame's own
 * device error, after which the frame is released and the outputs hold what
 * the device produced: SRT3D_EOFFSETS / SRT3D_ERANGE for a malformed chunk,
 * SRT3D_ETIMEDOUT when a bounded device wait of the frame's reconstruction
 * (the grid barrier of the one-launch iteration kernel) gave up, leaving a
 * partial result. A frame's errors are its own: other frames in flight are
 * not affected and do not see them. */
srt3d_status srt3d_poll(srt3d_ctx* ctx, uint64_t frame_id, uint32_t timeout_us, float* depth,
                        float* alpha, uint8_t* active, float* alpha0, uint32_t* n);

/* Failure-detection self-test (the paper has no counterpart). Launches one
 * CTA that runs the persistent iteration kernel's bounded wait for a
 * neighbour tile's progress flag on a flag that nothing raises, with a limit
 * of wait_cycles SM clock
 * cycles (1..4e9): the wait gives up, latches the device timeout flag, and
 * the next srt3d_sync returns SRT3D_ETIMEDOUT (clearing the flag). The
 * context stays usable. */
srt3d_status srt3d_selftest_wait_timeout(srt3d_ctx* ctx, uint64_t wait_cycles, void* stream);

/* Launch planning, host only: no device, no context, no CUDA call. Reports
 * the shapes srt3d_sketch_stream and srt3d_reconstruct choose for a frame of
 * rows x cols pixels with T bins, m harmonics, k_max points per pixel and
 * APSS radius `radius`, given the device's SM count and the co-resident CTAs
 * per SM that the persistent iteration kernel reaches (an occupancy figure the
 * caller supplies; 2 on a GB300 at radius 1).
 *   sketch_m, init_m     harmonic count the sketch / matched-filter kernels are
 *                        instantiated for (the smallest instantiation >= m)
 *   sketch_lanes         lanes per pixel of the stream sketch at the given mean
 *                        photons per pixel (4, 8 or 16; a batch's tuner may
 *                        also choose 32 for a density class)
 *   init_grid_spacing    D of the matched filter's branch and bound: the largest
 *                        power of two <= 64 with w_m^2 D^2 / 8 <= 0.08, w_m =
 *                        2 pi m / T (bounds how far the matched-filter score
 *                        can rise between two grid points)
 *   init_grid_points     ceil(T / D), points scored per pixel and pass
 *   tile_height, tiles   rows per 16-column tile of the one-launch iteration
 *                        kernel and its tile (= CTA) count; 0, 0 when the frame
 *                        runs one launch per iteration (tiles do not fit at
 *                        once, or k_max > 2 with radius > 1)
 *   serving_frame_bytes  device bytes such a frame holds while admitted by
 *                        srt3d_submit (sketch state, counts, impulse response,
 *                        results and reconstruction scratch): its charge
 *                        against the context's HBM budget
 * Errors: SRT3D_EINVAL for a NULL `out` or an argument outside the ranges of
 * srt3d_reconstruct (T 2..65536, m 1..32, k_max 1..4, radius 1..3), zero
 * rows, cols, num_sms or ctas_per_sm, or a negative or NaN photon mean. */
typedef struct srt3d_plan_info {
  uint32_t sketch_m;
  uint32_t sketch_lanes;
  uint32_t init_m;
  uint32_t init_grid_spacing;
  uint32_t init_grid_points;
  uint32_t tile_height;
  uint32_t tiles;
  uint32_t reserved;    /* 0 */
  uint64_t serving_frame_bytes;
} srt3d_plan_info;

srt3d_status srt3d_plan(uint32_t rows, uint32_t cols, uint32_t T, uint32_t m, uint32_t k_max, uint32_t radius,
                        double mean_photons_per_pixel, uint32_t num_sms, uint32_t ctas_per_sm,
                        srt3d_plan_info* out);

/* Measurement aid (the paper has no counterpart). With profiling enabled the
 * library brackets each of its kernel launches with CUDA events on the
 * launching stream and accumulates, per kernel, the device time and the
 * launch count. srt3d_profile_enable(ctx, 1) clears the totals and starts
 * recording, 0 stops. srt3d_profile_read() waits for the recorded events and
 * returns the totals of kernel `kernel` (an index < srt3d_kernel_count());
 * srt3d_kernel_name() names it. An entry can span consecutive launches of
 * one stage ("prep" of a single frame is two kernels, both counted). */
srt3d_status srt3d_profile_enable(srt3d_ctx* ctx, int enable);
srt3d_status srt3d_profile_read(srt3d_ctx* ctx, uint32_t kernel, double* total_ms, uint64_t* launches);
uint32_t srt3d_kernel_count(void);
const char* srt3d_kernel_name(uint32_t kernel);

#ifdef __cplusplus
}
#endif

#endif /* SRT3D_H */
