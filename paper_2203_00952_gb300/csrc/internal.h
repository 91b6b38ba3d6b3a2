// Internal declarations shared by the translation units of libsrt3d.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/srt3d.h"

namespace srt3d {

// Bits of the device error word latched by kernels.
enum : uint32_t {
  FLAG_STAMP_RANGE = 1u,   // a stamp >= T
  FLAG_OFFSETS = 2u,       // offsets decreasing or beyond num_stamps
  FLAG_COUNT_RANGE = 4u,   // a histogram count > 65535
  FLAG_DEVICE_TIMEOUT = 8u // a bounded device wait gave up
};

// Phase table for one T: cos/sin of 2 pi k / T, k in [0, T), computed on the
// host in double and rounded to float. For T <= kDirectTableMax the table is
// direct (T entries); above it is two-level: lo[256] = e^{i 2 pi k_lo / T},
// hi[ceil(T/256)] = e^{i 2 pi 256 k_hi / T}, k = 256 k_hi + k_lo.
constexpr uint32_t kDirectTableMax = 8192;
struct PhaseTable {
  float2* dev = nullptr;
  uint32_t entries = 0;
  bool two_level = false;
};

// Growable device buffer owned by the context.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct Serving;  // serving runtime (serve.cu)

// One frame of a batch (srt3d_process_batch), as the batched kernels see it.
struct BatchFrame {
  const uint16_t* stamps;
  const uint32_t* offsets;
  uint32_t num_stamps;
  uint32_t rows, cols, P, T, m;
  int glog2;  // sketch lanes per pixel (log2), from the autotuner
  const float2* table;
  uint32_t tab_entries;
  int two_level;
  const float* h;
  float2* S;  // sketch state, then z in place
  uint32_t* n;
  float* depth;
  float* alpha;
  uint8_t* active;
  float* alpha0;
  float2* hh;  // per-frame reconstruction scratch: hhat [32], misc [8]
  float* misc;
  // tagged exchange words of the post-gradient state, [2][P][K] x 16 B
  // (alternating by iteration; zeroed before each launch)
  unsigned long long* xtag;
  uint32_t D;        // matched-filter grid spacing
  uint32_t tile0;    // first iteration tile of this frame in the batch
  uint32_t tiles_x;  // iteration tiles per row (16 pixels wide)
  uint32_t tiles_y;  // iteration tile rows (th pixels high)
};

// Slots of the per-frame reconstruction scalars (misc[]): step sizes, E2 =
// sum |hhat|^2, n_max, and two spare words (zeroed by the prep kernels).
enum : uint32_t { MISC_ETA_T = 0, MISC_ETA_A = 1, MISC_E2 = 2, MISC_NMAX = 3, MISC_BAR = 4, MISC_COUNT = 8 };

// Kernel ids for the profiling counters.
enum KernelId : uint32_t {
  KID_SKETCH_STREAM = 0,
  KID_FINALIZE,
  KID_HIST_FROM_STREAM,
  KID_SKETCH_HIST_FP32,
  KID_SKETCH_HIST_TC,
  KID_PREP,
  KID_INIT,
  KID_GRAD,
  KID_ITER,
  KID_ITER_ALL,
  KID_ALPHA0,
  KID_BATCH,
  KID_BIRTH,
  KID_BUCKET_STREAM,
  KID_SKETCH_STREAM_TC,
  KID_COUNT
};

// Per-kernel CUDA-event timing (enabled by srt3d_profile_enable).
struct Profiler {
  bool enabled = false;
  std::vector<cudaEvent_t> pool;
  struct Pending {
    uint32_t kid;
    cudaEvent_t a, b;
    uint32_t kernels;  // kernel launches between the two events
  };
  std::vector<Pending> pending;
  double total_ms[KID_COUNT] = {};
  uint64_t launches[KID_COUNT] = {};
  std::mutex mu;
};

}  // namespace srt3d

struct srt3d_ctx {
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  size_t hbm_budget = 0;
  std::string last_error;
  uint32_t* d_flags = nullptr;  // device error word
  std::map<uint32_t, srt3d::PhaseTable> tables;
  // reconstruction scratch
  srt3d::DevBuf rc_scratch;
  // device histogram of srt3d_sketch_stream_tc
  srt3d::DevBuf hist_scratch;
  // histogram tensor-core operands keyed by (T, m, precision)
  std::map<std::tuple<uint32_t, uint32_t, int>, srt3d::DevBuf> fourier;
  std::mutex mu;  // guards tables/scratch growth for concurrent serving streams
  srt3d::Serving* serving = nullptr;
  // autotuned launch shapes: key -> value
  std::map<uint64_t, int> tuned;
  srt3d::Profiler prof;
};

namespace srt3d {

srt3d_status set_error(srt3d_ctx* ctx, srt3d_status st, const std::string& msg);
srt3d_status cuda_error(srt3d_ctx* ctx, cudaError_t err, const char* what);
srt3d_status get_phase_table(srt3d_ctx* ctx, uint32_t T, PhaseTable* out);
// The phase table of T in host memory (out holds kDirectTableMax entries):
// cos/sin(2 pi k / T) in double, rounded once to float. Returns the entry
// count; *two_level tells the layout.
uint32_t phase_table_host(uint32_t T, float2* out, bool* two_level);
// Drop the cached device address of the allocation-free entry point's array
// on `device` (srt3d_create calls it, so a context created after a device
// reset resolves the address again).
void noalloc_forget_device(int device);
srt3d_status grow(srt3d_ctx* ctx, DevBuf* buf, size_t bytes);

// Launchers (no argument validation; callers validate).
srt3d_status launch_sketch_stream(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                  uint64_t num_stamps, uint32_t P, uint32_t T, uint32_t m,
                                  int accumulate, float2* S, uint32_t* n, cudaStream_t stream,
                                  uint32_t* flags = nullptr);
srt3d_status launch_finalize(srt3d_ctx* ctx, const float2* S, const uint32_t* n, uint32_t P,
                             uint32_t m, float2* z, cudaStream_t stream);
int sketch_round_m(uint32_t m);
int sketch_default_glog2(double mean_photons_per_pixel);
// Lanes per pixel (log2) the stream sketch takes for num_stamps photons over
// P pixels: the context's tuned value for that density class, else the default.
int sketch_glog2(srt3d_ctx* ctx, uint64_t num_stamps, uint32_t P, uint32_t T, uint32_t m);
srt3d_status launch_sketch_stream_g(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                    uint64_t num_stamps, uint32_t P, uint32_t T, uint32_t m, int accumulate,
                                    float2* S, uint32_t* n, cudaStream_t stream, uint32_t* flags, int glog2);
srt3d_status launch_sketch_batch(srt3d_ctx* ctx, const BatchFrame* d_frames, const uint3* d_items,
                                 uint32_t num_items, int M, uint32_t max_tab_entries, cudaStream_t stream);
// Init work items of one instantiated harmonic count M (see init_round_m).
struct InitGroup {
  int M;
  const uint3* items;
  uint32_t count;
};
// Prep and init of every frame, then all iterations of every frame in one
// cooperative launch over the frames' tiles (th rows high; tile_flags holds
// total_tiles progress flags). With iters_override >= 0 that many iterations
// run instead of prm.iters (tile-height tuning).
srt3d_status launch_reconstruct_batch(srt3d_ctx* ctx, const BatchFrame* d_frames, uint32_t nframes,
                                      const InitGroup* init_groups, uint32_t num_groups, uint32_t total_tiles,
                                      uint32_t th, unsigned* tile_flags, uint32_t max_tab_entries, uint32_t max_G,
                                      const srt3d_params& prm, cudaStream_t stream);
// The iterations alone (the frames' state is the init's or a previous run's).
srt3d_status launch_iterations_batch(srt3d_ctx* ctx, const BatchFrame* d_frames, uint32_t nframes,
                                     uint32_t total_tiles, uint32_t th, unsigned* tile_flags, uint32_t iters,
                                     const srt3d_params& prm, cudaStream_t stream);
// Stride of the per-tile progress flags (words) and the largest tile height.
uint32_t tile_flag_stride();
uint32_t max_tile_height();
// Matched-filter initialisation (init.cu): hh = hhat[m], misc = frame scalars
// (misc[MISC_NMAX] receives the largest photon count, as an unsigned).
srt3d_status launch_init(srt3d_ctx* ctx, const float2* z, const uint32_t* n, uint32_t P, uint32_t T, uint32_t m,
                         uint32_t K, const PhaseTable& tab, const float2* hh, float* misc,
                         const srt3d_params& prm, float* depth, float* alpha, uint8_t* active, float* alpha0,
                         cudaStream_t stream);
// Birth move of every pixel with a free slot (init.cu), in place.
srt3d_status launch_birth(srt3d_ctx* ctx, const float2* z, const uint32_t* n, uint32_t P, uint32_t T, uint32_t m,
                          uint32_t K, const PhaseTable& tab, const float2* hh, const float* misc,
                          const srt3d_params& prm, float* depth, float* alpha, uint8_t* active, float* alpha0,
                          cudaStream_t stream);
// Batched: every frame of the items has m <= M, M an instantiated count.
srt3d_status launch_init_batch(srt3d_ctx* ctx, const BatchFrame* d_frames, const uint3* d_items,
                               uint32_t num_items, uint32_t K, int M, uint32_t max_entries, uint32_t max_G,
                               const srt3d_params& prm, cudaStream_t stream);
int init_round_m(uint32_t m);
uint32_t mf_grid_spacing_host(uint32_t T, uint32_t m);
// Device bytes a serving frame holds while admitted (its share of the HBM budget).
size_t serving_frame_bytes(uint32_t rows, uint32_t cols, uint32_t T, uint32_t m, uint32_t k_max);
// Rows per tile of the persistent iteration kernel (0: one launch per iteration).
uint32_t plan_tile_height(uint32_t k_max, uint32_t radius, uint32_t rows, uint32_t cols, int num_sms, int bps);
srt3d_status launch_hist_from_stream(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                     uint64_t num_stamps, uint32_t P, uint32_t T, uint16_t* hist,
                                     cudaStream_t stream);
srt3d_status reconstruct_impl(srt3d_ctx* ctx, const float2* z, const uint32_t* n, uint32_t rows,
                              uint32_t cols, uint32_t T, uint32_t m, const float* h,
                              const srt3d_params& prm, float* depth, float* alpha, uint8_t* active,
                              float* alpha0, void* scratch, size_t scratch_bytes, cudaStream_t stream,
                              uint32_t* flags = nullptr, bool inject_barrier_timeout = false);
size_t reconstruct_scratch_bytes(uint32_t P, uint32_t k_max, uint32_t m);
srt3d_status validate_params(srt3d_ctx* ctx, uint32_t rows, uint32_t cols, uint32_t T, uint32_t m,
                             const srt3d_params* prm);

// Cooperative launches of this library on one device run one after another:
// each waits on a per-device event that the previous one recorded (see
// launch_cooperative_chained in reconstruct.cu). coop_chain_init creates the
// device's event (called by srt3d_create, with the device current).
srt3d_status coop_chain_init(srt3d_ctx* ctx);
srt3d_status launch_cooperative_chained(srt3d_ctx* ctx, const void* fn, dim3 grid, dim3 block, void** args,
                                        size_t smem, cudaStream_t stream);

void serving_destroy(srt3d_ctx* ctx);
void batch_destroy(srt3d_ctx* ctx);

// Profiling: prof_begin returns an event pair (or {nullptr,nullptr} when off)
// recorded around one launch on `stream`.
struct ProfMark {
  cudaEvent_t a = nullptr, b = nullptr;
};
ProfMark prof_begin(srt3d_ctx* ctx, uint32_t kid, cudaStream_t stream);
void prof_end(srt3d_ctx* ctx, uint32_t kid, const ProfMark& mk, cudaStream_t stream, uint32_t kernels = 1);

}  // namespace srt3d

#define SRT3D_CUDA_TRY(ctx, expr)                                  \
  do {                                                             \
    cudaError_t _e = (expr);                                       \
    if (_e != cudaSuccess) return ::srt3d::cuda_error(ctx, _e, #expr); \
  } while (0)
