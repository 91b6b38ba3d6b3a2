// Batched processing of uneven frames (srt3d_process_batch): photon sketch
// (Sec. 2, Eq. 3), normalisation and SRT3D reconstruction (Sec. 3, Eq. 8) of
// many frames of different sizes, T, m and photon densities.
//
// Every stage is one launch over all frames of the batch: the sketch (one
// launch per harmonic class, writing z = S / n directly) and the
// initialisation (one per instantiated harmonic count) walk work lists of
// (frame, pixel range) items of about equal work; one block per frame computes
// hhat and the step sizes; and all iterations of all frames run in ONE
// cooperative launch over the frames' tiles (k_iter_batch_persistent). The
// sequence is captured once into a CUDA graph that later calls with the same
// frames replay. Two autotuners pick launch shapes on the first call: the
// sketch's lanes per pixel, timed per photon-density class on the first frame
// of the class (cached in the context), and the iteration tiles' height,
// timed on the whole batch (two iterations per candidate, after an untimed
// sketch and init) and kept in the batch's graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>

#include "internal.h"

namespace srt3d {
namespace {

constexpr uint32_t kInitItemPixels = 128;
constexpr size_t kMaxGraphs = 16;
// Tile heights the iteration tuner times (pixels; tiles are 16 wide).
constexpr uint32_t kTileHeights[] = {16, 12, 8};
// Sketch work items: per CTA slot, and the largest pixel range of one item.
constexpr uint32_t kItemsPerSlot = 4;
constexpr double kMaxItemPixels = 2048.0;
// Fixed sketch work of one pixel in photon equivalents (offsets, the lane
// group's reduce-scatter of 2m sums, the stores), whatever its photon count.
double pixel_cost(uint32_t m) { return 16.0 + 2.0 * double(m); }

struct GraphEntry {
  std::vector<uint8_t> key;
  cudaGraphExec_t exec = nullptr;
  void* dmem = nullptr;  // frame descriptors, work lists, per-frame scratch
};

struct BatchCache {
  std::vector<GraphEntry> graphs;  // most recent last
  cudaStream_t capture = nullptr;
};

std::mutex g_cache_mu;
std::map<const srt3d_ctx*, BatchCache*> g_cache;

BatchCache* cache_of(srt3d_ctx* ctx) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  BatchCache*& c = g_cache[ctx];
  if (!c) c = new BatchCache();
  return c;
}

uint64_t tuner_key(int M, bool two_level, double mean) {
  const int bucket = mean < 1.0 ? 0 : int(std::log2(mean));
  return (uint64_t(M) << 40) | (uint64_t(two_level) << 32) | uint64_t(bucket);
}

// Autotuner: time the sketch with 4, 8, 16 and 32 lanes per pixel on `f`
// (two launches each, CUDA events on `stream`) and keep the fastest.
srt3d_status tune_glog2(srt3d_ctx* ctx, const srt3d_frame& f, cudaStream_t stream, int* out) {
  cudaEvent_t a, b;
  SRT3D_CUDA_TRY(ctx, cudaEventCreate(&a));
  SRT3D_CUDA_TRY(ctx, cudaEventCreate(&b));
  const uint32_t P = f.rows * f.cols;
  float best = 1e30f;
  int best_g = sketch_default_glog2(double(f.num_stamps) / double(P));
  for (int g = 2; g <= 5; ++g) {
    float total = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      SRT3D_CUDA_TRY(ctx, cudaEventRecord(a, stream));
      srt3d_status st = launch_sketch_stream_g(ctx, f.stamps, f.offsets, f.num_stamps, P, f.T, f.m, 0,
                                               reinterpret_cast<float2*>(f.z), f.n, stream, nullptr, g);
      if (st != SRT3D_OK) return st;
      SRT3D_CUDA_TRY(ctx, cudaEventRecord(b, stream));
      SRT3D_CUDA_TRY(ctx, cudaEventSynchronize(b));
      float ms = 0.f;
      SRT3D_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, a, b));
      if (rep > 0) total += ms;  // the first launch warms the caches
    }
    if (total < best) {
      best = total;
      best_g = g;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *out = best_g;
  return SRT3D_OK;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

void batch_destroy(srt3d_ctx* ctx) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  auto it = g_cache.find(ctx);
  if (it == g_cache.end()) return;
  for (auto& g : it->second->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.dmem) cudaFree(g.dmem);
  }
  if (it->second->capture) cudaStreamDestroy(it->second->capture);
  delete it->second;
  g_cache.erase(it);
}

}  // namespace srt3d

using namespace srt3d;

extern "C" srt3d_status srt3d_process_batch(srt3d_ctx* ctx, const srt3d_frame* frames, uint32_t num_frames,
                                            const srt3d_params* params, void* stream_v) {
  if (!ctx) return SRT3D_EINVAL;
  if (!frames || !params || num_frames == 0) return set_error(ctx, SRT3D_EINVAL, "no frames or params");
  if (params->init_mode != SRT3D_INIT_MATCHED || !params->regularize || params->birth_every)
    return set_error(ctx, SRT3D_EINVAL, "batches use the matched-filter init and the spatial prior, no births");
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  // ---------------------------------------------------------------- validation, tables, tuning
  std::vector<PhaseTable> tabs(num_frames);
  std::vector<int> glog2(num_frames);
  uint32_t max_entries = 0, max_G = 1;
  for (uint32_t i = 0; i < num_frames; ++i) {
    const srt3d_frame& f = frames[i];
    srt3d_status st = validate_params(ctx, f.rows, f.cols, f.T, f.m, params);
    if (st != SRT3D_OK) return st;
    if (!f.offsets || !f.h || !f.z || !f.n || !f.depth || !f.alpha || !f.active || !f.alpha0 ||
        (f.num_stamps && !f.stamps))
      return set_error(ctx, SRT3D_EINVAL, "NULL pointer in a frame");
    if (f.num_stamps >= (1ull << 32) - 16) return set_error(ctx, SRT3D_EINVAL, "num_stamps must be < 2^32 - 16");
    if (reinterpret_cast<uintptr_t>(f.z) % 8) return set_error(ctx, SRT3D_EINVAL, "z must be 8-byte aligned");
    if (uint64_t(f.rows) * f.cols * f.m >= (1ull << 32))
      return set_error(ctx, SRT3D_EINVAL, "rows * cols * m must be < 2^32 in a batch");
    st = get_phase_table(ctx, f.T, &tabs[i]);
    if (st != SRT3D_OK) return st;
    max_entries = std::max(max_entries, tabs[i].entries);
    const uint32_t D = mf_grid_spacing_host(f.T, f.m);
    max_G = std::max(max_G, (f.T + D - 1) / D);
  }
  for (uint32_t i = 0; i < num_frames; ++i) {
    const srt3d_frame& f = frames[i];
    const uint32_t P = f.rows * f.cols;
    const double mean = double(f.num_stamps) / double(P);
    const uint64_t key = tuner_key(sketch_round_m(f.m), tabs[i].two_level, mean);
    int g = -1;
    {
      std::lock_guard<std::mutex> lock(ctx->mu);
      auto it = ctx->tuned.find(key);
      if (it != ctx->tuned.end()) g = it->second;
    }
    if (g < 0) {
      srt3d_status st = tune_glog2(ctx, f, stream, &g);
      if (st != SRT3D_OK) return st;
      std::lock_guard<std::mutex> lock(ctx->mu);
      ctx->tuned[key] = g;
    }
    glog2[i] = g;
  }
  // ---------------------------------------------------------------- graph cache lookup
  std::vector<uint8_t> key(sizeof(srt3d_frame) * num_frames + sizeof(srt3d_params) + sizeof(int) * num_frames);
  std::memcpy(key.data(), frames, sizeof(srt3d_frame) * num_frames);
  std::memcpy(key.data() + sizeof(srt3d_frame) * num_frames, params, sizeof(srt3d_params));
  std::memcpy(key.data() + sizeof(srt3d_frame) * num_frames + sizeof(srt3d_params), glog2.data(),
              sizeof(int) * num_frames);
  BatchCache* cache = cache_of(ctx);
  std::lock_guard<std::mutex> glock(g_cache_mu);
  for (size_t gi = 0; gi < cache->graphs.size(); ++gi) {
    if (cache->graphs[gi].key == key) {
      GraphEntry e = cache->graphs[gi];
      cache->graphs.erase(cache->graphs.begin() + gi);
      cache->graphs.push_back(e);
      const ProfMark mk = prof_begin(ctx, KID_BATCH, stream);
      SRT3D_CUDA_TRY(ctx, cudaGraphLaunch(e.exec, stream));
      prof_end(ctx, KID_BATCH, mk, stream);
      return SRT3D_OK;
    }
  }
  // ---------------------------------------------------------------- descriptors and work lists
  std::vector<BatchFrame> hf(num_frames);
  std::map<int, std::vector<uint3>> sketch_items;  // by instantiated M
  std::map<int, double> group_cost;  // sketch work per m class, in photon equivalents
  std::map<int, std::vector<uint3>> init_items;  // by instantiated init M
  for (uint32_t i = 0; i < num_frames; ++i)
    group_cost[sketch_round_m(frames[i].m)] +=
        double(frames[i].num_stamps) + double(frames[i].rows) * frames[i].cols * pixel_cost(frames[i].m);
  for (uint32_t i = 0; i < num_frames; ++i) {
    const srt3d_frame& f = frames[i];
    BatchFrame& b = hf[i];
    b.stamps = f.stamps;
    b.offsets = f.offsets;
    b.num_stamps = uint32_t(f.num_stamps);
    b.rows = f.rows;
    b.cols = f.cols;
    b.P = f.rows * f.cols;
    b.T = f.T;
    b.m = f.m;
    b.glog2 = glog2[i];
    b.table = tabs[i].dev;
    b.tab_entries = tabs[i].entries;
    b.two_level = tabs[i].two_level ? 1 : 0;
    b.h = f.h;
    b.S = reinterpret_cast<float2*>(f.z);
    b.n = f.n;
    b.depth = f.depth;
    b.alpha = f.alpha;
    b.active = f.active;
    b.alpha0 = f.alpha0;
    b.D = mf_grid_spacing_host(f.T, f.m);
    b.tiles_x = (f.cols + 15) / 16;
    // sketch items of about equal work: photons plus a fixed cost per pixel
    // (its offsets, the group's reduction and the stores), several items per
    // CTA slot so that the last wave is short, and at most kMaxItemPixels
    // pixels per item (a sparse frame must not become one CTA's work)
    const int M = sketch_round_m(f.m);
    const double target =
        std::max(1.0, group_cost[M] / double(uint64_t(ctx->num_sms) * 4u * kItemsPerSlot));
    const double per_pixel = double(f.num_stamps) / double(b.P) + pixel_cost(f.m);
    const uint32_t span =
        uint32_t(std::min<double>(std::min<double>(b.P, kMaxItemPixels), std::max(32.0, std::ceil(target / per_pixel))));
    for (uint32_t p0 = 0; p0 < b.P; p0 += span) sketch_items[M].push_back(make_uint3(i, p0, std::min(b.P, p0 + span)));
    for (uint32_t p0 = 0; p0 < b.P; p0 += kInitItemPixels)
      init_items[init_round_m(f.m)].push_back(make_uint3(i, p0, std::min(b.P, p0 + kInitItemPixels)));
  }
  size_t items_total = 0;
  for (auto& kv : sketch_items) items_total += kv.second.size();
  for (auto& kv : init_items) items_total += kv.second.size();
  const size_t frames_bytes = al256(num_frames * sizeof(BatchFrame));
  const size_t scratch_per_frame = 512;  // hhat[32] float2 + misc[8] float
  const uint32_t K = params->k_max;
  size_t alt_bytes = 0;  // two buffers of tagged exchange words per frame, 16 B per point each
  for (uint32_t i = 0; i < num_frames; ++i) alt_bytes += al256(size_t(hf[i].P) * K * 32);
  // the frames' iteration tiles for a tile height (the tuner tries several)
  const auto layout = [&](uint32_t th) {
    uint32_t tiles = 0;
    for (uint32_t i = 0; i < num_frames; ++i) {
      hf[i].tile0 = tiles;
      hf[i].tiles_y = (hf[i].rows + th - 1) / th;
      tiles += hf[i].tiles_x * hf[i].tiles_y;
    }
    return tiles;
  };
  uint32_t max_tiles = 0;
  for (uint32_t th : kTileHeights) max_tiles = std::max(max_tiles, layout(th));
  const size_t flags_bytes = al256(size_t(max_tiles) * tile_flag_stride() * sizeof(unsigned));
  const size_t bytes = frames_bytes + al256(items_total * sizeof(uint3)) + num_frames * scratch_per_frame +
                       alt_bytes + flags_bytes;
  GraphEntry e;
  e.key = key;
  SRT3D_CUDA_TRY(ctx, cudaMalloc(&e.dmem, bytes));
  char* base = static_cast<char*>(e.dmem);
  char* scratch = base + frames_bytes + al256(items_total * sizeof(uint3));
  char* alt = scratch + num_frames * scratch_per_frame;
  char* const alt0 = alt;  // the tagged words, zeroed before every iteration launch
  for (uint32_t i = 0; i < num_frames; ++i) {
    hf[i].hh = reinterpret_cast<float2*>(scratch + i * scratch_per_frame);
    hf[i].misc = reinterpret_cast<float*>(scratch + i * scratch_per_frame + 256);
    hf[i].xtag = reinterpret_cast<unsigned long long*>(alt);
    alt += al256(size_t(hf[i].P) * K * 32);
  }
  unsigned* tile_flags = reinterpret_cast<unsigned*>(alt);
  std::vector<uint3> all_items;
  std::vector<std::pair<int, std::pair<size_t, size_t>>> groups;  // M -> (offset, count)
  for (auto& kv : sketch_items) {
    groups.push_back({kv.first, {all_items.size(), kv.second.size()}});
    all_items.insert(all_items.end(), kv.second.begin(), kv.second.end());
  }
  std::vector<std::pair<int, std::pair<size_t, size_t>>> igroups;  // init M -> (offset, count)
  for (auto& kv : init_items) {
    igroups.push_back({kv.first, {all_items.size(), kv.second.size()}});
    all_items.insert(all_items.end(), kv.second.begin(), kv.second.end());
  }
  SRT3D_CUDA_TRY(ctx, cudaMemcpy(base + frames_bytes, all_items.data(), all_items.size() * sizeof(uint3),
                                 cudaMemcpyHostToDevice));
  const BatchFrame* d_frames = reinterpret_cast<const BatchFrame*>(base);
  const uint3* d_items = reinterpret_cast<const uint3*>(base + frames_bytes);
  std::vector<InitGroup> init_groups;
  for (auto& g : igroups)
    init_groups.push_back({g.first, d_items + g.second.first, uint32_t(g.second.second)});
  const auto upload = [&](uint32_t th) {
    const uint32_t tiles = layout(th);
    const cudaError_t e = cudaMemcpy(base, hf.data(), num_frames * sizeof(BatchFrame), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? tiles : 0u;
  };
  const auto sketch_all = [&](cudaStream_t s) {
    srt3d_status r = SRT3D_OK;
    for (auto& g : groups)
      if (r == SRT3D_OK)
        r = launch_sketch_batch(ctx, d_frames, d_items + g.second.first, uint32_t(g.second.second), g.first,
                                max_entries, s);
    return r;
  };
  const bool prof_on = ctx->prof.enabled;
  ctx->prof.enabled = false;  // neither tuning launches nor graph nodes are profiled
  srt3d_status st = SRT3D_OK;
  // ---------------------------------------------------------------- tile-height tuner
  uint32_t best_th = kTileHeights[0];
  if (params->iters > 0) {
    cudaEvent_t ea = nullptr, eb = nullptr;
    float best = 1e30f;
    st = upload(kTileHeights[0]) ? SRT3D_OK : set_error(ctx, SRT3D_ECUDA, "descriptor upload");
    if (st == SRT3D_OK) st = sketch_all(stream);
    srt3d_params p0 = *params;
    p0.iters = 0;
    if (st == SRT3D_OK)
      st = launch_reconstruct_batch(ctx, d_frames, num_frames, init_groups.data(), uint32_t(init_groups.size()),
                                    layout(kTileHeights[0]), kTileHeights[0], tile_flags, max_entries, max_G, p0,
                                    stream);
    if (st == SRT3D_OK && (cudaEventCreate(&ea) != cudaSuccess || cudaEventCreate(&eb) != cudaSuccess ||
                           cudaStreamSynchronize(stream) != cudaSuccess))
      st = set_error(ctx, SRT3D_ECUDA, "tuner set-up");
    for (uint32_t th : kTileHeights) {
      if (st != SRT3D_OK) break;
      const uint32_t tiles = upload(th);
      if (!tiles) {
        st = set_error(ctx, SRT3D_ECUDA, "descriptor upload");
        break;
      }
      float ms = 0.f;
      for (int rep = 0; rep < 2 && st == SRT3D_OK; ++rep) {  // the first run warms up
        if (cudaMemsetAsync(tile_flags, 0, flags_bytes, stream) != cudaSuccess ||
            cudaMemsetAsync(alt0, 0, alt_bytes, stream) != cudaSuccess ||
            cudaEventRecord(ea, stream) != cudaSuccess) {
          st = set_error(ctx, SRT3D_ECUDA, "tuner launch");
          break;
        }
        st = launch_iterations_batch(ctx, d_frames, num_frames, tiles, th, tile_flags, 2, *params, stream);
        if (st == SRT3D_OK &&
            (cudaEventRecord(eb, stream) != cudaSuccess || cudaEventSynchronize(eb) != cudaSuccess ||
             cudaEventElapsedTime(&ms, ea, eb) != cudaSuccess))
          st = set_error(ctx, SRT3D_ECUDA, "tuner timing");
      }
      if (st == SRT3D_OK && ms < best) {
        best = ms;
        best_th = th;
      }
    }
    if (ea) cudaEventDestroy(ea);
    if (eb) cudaEventDestroy(eb);
  }
  const uint32_t tiles = st == SRT3D_OK ? upload(best_th) : 0u;
  if (st == SRT3D_OK && !tiles) st = set_error(ctx, SRT3D_ECUDA, "descriptor upload");
  if (st != SRT3D_OK) {
    ctx->prof.enabled = prof_on;
    cudaFree(e.dmem);
    return st;
  }
  // ---------------------------------------------------------------- capture
  if (!cache->capture) SRT3D_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&cache->capture, cudaStreamNonBlocking));
  cudaStream_t cs = cache->capture;
  SRT3D_CUDA_TRY(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  st = sketch_all(cs);
  if (st == SRT3D_OK && cudaMemsetAsync(alt0, 0, alt_bytes, cs) != cudaSuccess)
    st = set_error(ctx, SRT3D_ECUDA, "exchange words reset");
  if (st == SRT3D_OK)
    st = launch_reconstruct_batch(ctx, d_frames, num_frames, init_groups.data(), uint32_t(init_groups.size()),
                                  tiles, best_th, tile_flags, max_entries, max_G, *params, cs);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  ctx->prof.enabled = prof_on;
  if (st != SRT3D_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaFree(e.dmem);
    return st != SRT3D_OK ? st : cuda_error(ctx, ce, "cudaStreamEndCapture");
  }
  const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    cudaFree(e.dmem);
    return cuda_error(ctx, ie, "cudaGraphInstantiate");
  }
  if (cache->graphs.size() >= kMaxGraphs) {
    GraphEntry old = cache->graphs.front();
    cache->graphs.erase(cache->graphs.begin());
    cudaGraphExecDestroy(old.exec);
    cudaFree(old.dmem);
  }
  cache->graphs.push_back(e);
  const ProfMark mk = prof_begin(ctx, KID_BATCH, stream);
  SRT3D_CUDA_TRY(ctx, cudaGraphLaunch(e.exec, stream));
  prof_end(ctx, KID_BATCH, mk, stream);
  return SRT3D_OK;
}
