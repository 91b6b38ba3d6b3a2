// Serving runtime: continuous batching of lidar frames (srt3d_submit / srt3d_poll).
//
// A frame is opened by its first chunk, receives photon chunks that are
// sketched online into a device-resident per-pixel state (the online update
// of the sketch, Sec. 2, after Eq. 3), and is reconstructed after its last
// chunk (Sec. 3). The runtime owns a pool of slots; each slot has its own CUDA
// stream, pinned staging buffers and events, so the chunks and
// reconstructions of different frames overlap on the device. A frame is
// admitted when a slot is free and its device state fits the context's HBM
// budget; otherwise srt3d_submit returns SRT3D_EBUSY and consumes nothing.
// Device memory of a frame is stream-ordered (cudaMallocAsync on its slot's
// stream, cudaFreeAsync at release), so admission never synchronises the
// device. No kernel uses floating-point atomics, so a frame's result does not
// depend on which other frames share the device.
//
// Host-side fault injection for tests: SRT3D_FAULT=alloc makes the next
// admission fail with SRT3D_ENOMEM as if the allocation had failed;
// SRT3D_FAULT=gridwait:<frame id> launches that frame's persistent iteration
// kernel with a grid-barrier target one arrival beyond what its grid delivers
// and a ~50 us wait limit, so its barrier waits give up (the kernel returns,
// latching FLAG_DEVICE_TIMEOUT in the frame's own error word) and its poll
// returns SRT3D_ETIMEDOUT; the other frames are untouched.
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <thread>

#include "internal.h"

namespace srt3d {

namespace {
constexpr int kDefaultSlots = 8;
size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
}  // namespace

struct Slot {
  cudaStream_t stream = nullptr;       // sketches, reconstruction, result copies
  cudaStream_t copy_stream = nullptr;  // chunk uploads
  // two chunk buffers alternate so that the upload of chunk i+1 overlaps the
  // sketch of chunk i
  void* pin_in[2] = {nullptr, nullptr};  // staging for pageable caller memory
  size_t pin_in_bytes[2] = {0, 0};
  void* d_chunk[2] = {nullptr, nullptr};
  size_t d_chunk_bytes[2] = {0, 0};
  cudaEvent_t copied[2] = {nullptr, nullptr};    // upload into d_chunk[b] done
  cudaEvent_t consumed[2] = {nullptr, nullptr};  // sketch reading d_chunk[b] done
  int next = 0;
  void* pin_h = nullptr;  // impulse response staging
  size_t pin_h_bytes = 0;
  void* pin_out = nullptr;  // results
  size_t pin_out_bytes = 0;
  cudaEvent_t done = nullptr;
  bool busy = false;
};

struct Frame {
  uint64_t id = 0;
  uint32_t rows = 0, cols = 0, T = 0, m = 0;
  srt3d_params prm{};
  int slot = -1;
  size_t bytes = 0;
  void* dmem = nullptr;
  float2* S = nullptr;
  uint32_t* n = nullptr;
  float* h = nullptr;
  float* depth = nullptr;
  float* alpha = nullptr;
  uint8_t* active = nullptr;
  float* alpha0 = nullptr;
  uint32_t* flags = nullptr;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  bool closed = false;  // last chunk submitted
};

struct Serving {
  std::mutex mu;
  std::vector<Slot> slots;
  std::map<uint64_t, Frame*> frames;
  size_t used = 0;
};

namespace {

// Device bytes one frame holds while in flight.
size_t frame_layout(Frame* f, char* base) {
  const size_t P = size_t(f->rows) * f->cols, K = f->prm.k_max;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += al256(bytes);
    return p;
  };
  f->S = reinterpret_cast<float2*>(take(P * f->m * sizeof(float2)));
  f->n = reinterpret_cast<uint32_t*>(take(P * sizeof(uint32_t)));
  f->h = reinterpret_cast<float*>(take(size_t(f->T) * sizeof(float)));
  f->depth = reinterpret_cast<float*>(take(P * K * sizeof(float)));
  f->alpha = reinterpret_cast<float*>(take(P * K * sizeof(float)));
  f->active = reinterpret_cast<uint8_t*>(take(P * K));
  f->alpha0 = reinterpret_cast<float*>(take(P * sizeof(float)));
  f->flags = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t)));
  f->scratch_bytes = reconstruct_scratch_bytes(uint32_t(P), uint32_t(K), f->m);
  f->scratch = take(f->scratch_bytes);
  return off;
}

size_t out_bytes(const Frame* f) {
  const size_t P = size_t(f->rows) * f->cols, K = f->prm.k_max;
  return al256(P * K * 4) * 2 + al256(P * K) + al256(P * 4) * 2 + 256;
}

Serving* serving(srt3d_ctx* ctx) {
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (!ctx->serving) {
    Serving* sv = new Serving();
    int nslots = kDefaultSlots;
    if (const char* e = std::getenv("SRT3D_SLOTS")) nslots = std::max(1, std::min(64, std::atoi(e)));
    sv->slots.resize(nslots);
    ctx->serving = sv;
  }
  return ctx->serving;
}

srt3d_status ensure_slot(srt3d_ctx* ctx, Slot& s) {
  if (!s.stream) SRT3D_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
  if (!s.copy_stream) SRT3D_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&s.copy_stream, cudaStreamNonBlocking));
  for (int b = 0; b < 2; ++b) {
    if (!s.copied[b]) SRT3D_CUDA_TRY(ctx, cudaEventCreateWithFlags(&s.copied[b], cudaEventDisableTiming));
    if (!s.consumed[b]) SRT3D_CUDA_TRY(ctx, cudaEventCreateWithFlags(&s.consumed[b], cudaEventDisableTiming));
  }
  if (!s.done) SRT3D_CUDA_TRY(ctx, cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
  return SRT3D_OK;
}

bool is_pinned(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

srt3d_status grow_pinned(srt3d_ctx* ctx, void** p, size_t* have, size_t want) {
  if (*have >= want) return SRT3D_OK;
  if (*p) SRT3D_CUDA_TRY(ctx, cudaFreeHost(*p));
  *p = nullptr;
  *have = 0;
  const size_t sz = al256(want + want / 4);
  SRT3D_CUDA_TRY(ctx, cudaHostAlloc(p, sz, cudaHostAllocDefault));
  *have = sz;
  return SRT3D_OK;
}

void release_frame(srt3d_ctx* ctx, Serving* sv, Frame* f) {
  Slot& s = sv->slots[f->slot];
  if (f->dmem) cudaFreeAsync(f->dmem, s.stream);
  sv->used -= f->bytes;
  s.busy = false;
  sv->frames.erase(f->id);
  delete f;
  (void)ctx;
}

}  // namespace

size_t serving_frame_bytes(uint32_t rows, uint32_t cols, uint32_t T, uint32_t m, uint32_t k_max) {
  Frame probe;
  probe.rows = rows;
  probe.cols = cols;
  probe.T = T;
  probe.m = m;
  probe.prm.k_max = k_max;
  return frame_layout(&probe, nullptr);
}

void serving_destroy(srt3d_ctx* ctx) {
  Serving* sv = ctx->serving;
  if (!sv) return;
  for (auto& kv : sv->frames) {
    Slot& s = sv->slots[kv.second->slot];
    if (kv.second->dmem) cudaFreeAsync(kv.second->dmem, s.stream);
    delete kv.second;
  }
  for (Slot& s : sv->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.copy_stream) cudaStreamSynchronize(s.copy_stream);
    for (int b = 0; b < 2; ++b) {
      if (s.d_chunk[b]) cudaFree(s.d_chunk[b]);
      if (s.pin_in[b]) cudaFreeHost(s.pin_in[b]);
      if (s.copied[b]) cudaEventDestroy(s.copied[b]);
      if (s.consumed[b]) cudaEventDestroy(s.consumed[b]);
    }
    if (s.pin_h) cudaFreeHost(s.pin_h);
    if (s.pin_out) cudaFreeHost(s.pin_out);
    if (s.done) cudaEventDestroy(s.done);
    if (s.copy_stream) cudaStreamDestroy(s.copy_stream);
    if (s.stream) cudaStreamDestroy(s.stream);
  }
  delete sv;
  ctx->serving = nullptr;
}

}  // namespace srt3d

using namespace srt3d;

extern "C" srt3d_status srt3d_submit(srt3d_ctx* ctx, uint64_t frame_id, uint32_t rows, uint32_t cols, uint32_t T,
                                     uint32_t m, const float* h, const srt3d_params* params,
                                     const uint16_t* chunk_stamps, const uint32_t* chunk_offsets, int last_chunk) {
  if (!ctx) return SRT3D_EINVAL;
  srt3d_status st = validate_params(ctx, rows, cols, T, m, params);
  if (st != SRT3D_OK) return st;
  if (!chunk_offsets || !h) return set_error(ctx, SRT3D_EINVAL, "NULL pointer");
  const uint32_t P = rows * cols;
  // host-side validation of the chunk's CSR offsets
  if (chunk_offsets[0] != 0) return set_error(ctx, SRT3D_EINVAL, "chunk_offsets[0] must be 0");
  for (uint32_t p = 0; p < P; ++p)
    if (chunk_offsets[p + 1] < chunk_offsets[p]) return set_error(ctx, SRT3D_EINVAL, "chunk_offsets decrease");
  const uint64_t N = chunk_offsets[P];
  if (N && !chunk_stamps) return set_error(ctx, SRT3D_EINVAL, "NULL chunk_stamps");
  Serving* sv = serving(ctx);
  std::lock_guard<std::mutex> lock(sv->mu);
  Frame* f = nullptr;
  auto it = sv->frames.find(frame_id);
  if (it == sv->frames.end()) {
    // admission
    Frame probe;
    probe.rows = rows;
    probe.cols = cols;
    probe.T = T;
    probe.m = m;
    probe.prm = *params;
    const size_t bytes = frame_layout(&probe, nullptr);
    int slot = -1;
    for (size_t i = 0; i < sv->slots.size(); ++i)
      if (!sv->slots[i].busy) {
        slot = int(i);
        break;
      }
    if (slot < 0 || sv->used + bytes > ctx->hbm_budget)
      return set_error(ctx, SRT3D_EBUSY, "frame not admitted now (slots or HBM budget)");
    if (const char* e = std::getenv("SRT3D_FAULT"))
      if (std::strcmp(e, "alloc") == 0) return set_error(ctx, SRT3D_ENOMEM, "injected allocation failure");
    Slot& s = sv->slots[slot];
    st = ensure_slot(ctx, s);
    if (st != SRT3D_OK) return st;
    f = new Frame(probe);
    f->id = frame_id;
    f->slot = slot;
    f->bytes = bytes;
    cudaError_t e = cudaMallocAsync(&f->dmem, bytes, s.stream);
    if (e != cudaSuccess) {
      delete f;
      return cuda_error(ctx, e, "cudaMallocAsync(frame)");
    }
    frame_layout(f, static_cast<char*>(f->dmem));
    s.busy = true;
    sv->used += bytes;
    sv->frames[frame_id] = f;
    SRT3D_CUDA_TRY(ctx, cudaMemsetAsync(f->S, 0, size_t(P) * m * sizeof(float2), s.stream));
    SRT3D_CUDA_TRY(ctx, cudaMemsetAsync(f->n, 0, size_t(P) * sizeof(uint32_t), s.stream));
    SRT3D_CUDA_TRY(ctx, cudaMemsetAsync(f->flags, 0, sizeof(uint32_t), s.stream));
    // h: the previous frame of this slot finished (it was polled), so its
    // staging buffer is free
    st = grow_pinned(ctx, &s.pin_h, &s.pin_h_bytes, size_t(T) * sizeof(float));
    if (st != SRT3D_OK) return st;
    std::memcpy(s.pin_h, h, size_t(T) * sizeof(float));
    SRT3D_CUDA_TRY(ctx, cudaMemcpyAsync(f->h, s.pin_h, size_t(T) * sizeof(float), cudaMemcpyHostToDevice, s.stream));
  } else {
    f = it->second;
    if (f->closed) return set_error(ctx, SRT3D_EINVAL, "frame already received its last chunk");
    if (f->rows != rows || f->cols != cols || f->T != T || f->m != m)
      return set_error(ctx, SRT3D_EINVAL, "chunk shape differs from the frame's first chunk");
  }
  Slot& s = sv->slots[f->slot];
  // upload the chunk into the buffer not used by the previous chunk; pinned
  // caller memory is copied directly, pageable memory through staging
  const int b = s.next;
  s.next ^= 1;
  const size_t sb = al256(N * sizeof(uint16_t)), ob = size_t(P + 1) * sizeof(uint32_t);
  if (s.d_chunk_bytes[b] < sb + ob) {
    SRT3D_CUDA_TRY(ctx, cudaEventSynchronize(s.consumed[b]));
    if (s.d_chunk[b]) SRT3D_CUDA_TRY(ctx, cudaFree(s.d_chunk[b]));
    s.d_chunk[b] = nullptr;
    s.d_chunk_bytes[b] = 0;
    const size_t want = al256((sb + ob) + (sb + ob) / 4);
    SRT3D_CUDA_TRY(ctx, cudaMalloc(&s.d_chunk[b], want));
    s.d_chunk_bytes[b] = want;
  }
  char* dc = static_cast<char*>(s.d_chunk[b]);
  SRT3D_CUDA_TRY(ctx, cudaStreamWaitEvent(s.copy_stream, s.consumed[b], 0));
  const bool direct = N && is_pinned(chunk_stamps) && is_pinned(chunk_offsets);
  if (direct) {
    SRT3D_CUDA_TRY(ctx, cudaMemcpyAsync(dc, chunk_stamps, N * sizeof(uint16_t), cudaMemcpyHostToDevice,
                                        s.copy_stream));
    SRT3D_CUDA_TRY(ctx, cudaMemcpyAsync(dc + sb, chunk_offsets, ob, cudaMemcpyHostToDevice, s.copy_stream));
  } else {
    SRT3D_CUDA_TRY(ctx, cudaEventSynchronize(s.copied[b]));  // staging buffer b free again
    st = grow_pinned(ctx, &s.pin_in[b], &s.pin_in_bytes[b], sb + ob);
    if (st != SRT3D_OK) return st;
    char* pin = static_cast<char*>(s.pin_in[b]);
    if (N) std::memcpy(pin, chunk_stamps, N * sizeof(uint16_t));
    std::memcpy(pin + sb, chunk_offsets, ob);
    SRT3D_CUDA_TRY(ctx, cudaMemcpyAsync(dc, pin, sb + ob, cudaMemcpyHostToDevice, s.copy_stream));
  }
  SRT3D_CUDA_TRY(ctx, cudaEventRecord(s.copied[b], s.copy_stream));
  SRT3D_CUDA_TRY(ctx, cudaStreamWaitEvent(s.stream, s.copied[b], 0));
  const uint16_t* d_st = reinterpret_cast<const uint16_t*>(dc);
  const uint32_t* d_off = reinterpret_cast<const uint32_t*>(dc + sb);
  st = launch_sketch_stream(ctx, d_st, d_off, N, P, T, m, 1, f->S, f->n, s.stream, f->flags);
  if (st != SRT3D_OK) return st;
  SRT3D_CUDA_TRY(ctx, cudaEventRecord(s.consumed[b], s.stream));
  // the caller's arrays must be free to reuse when submit returns, unless the
  // caller promised to keep them until the poll
  if (direct && !(last_chunk & SRT3D_CHUNK_KEEP)) SRT3D_CUDA_TRY(ctx, cudaEventSynchronize(s.copied[b]));
  if (last_chunk & SRT3D_LAST_CHUNK) {
    f->closed = true;
    st = launch_finalize(ctx, f->S, f->n, P, m, f->S, s.stream);
    if (st != SRT3D_OK) return st;
    srt3d_params prm = f->prm;
    prm.init_mode = SRT3D_INIT_MATCHED;
    bool inject = false;
    if (const char* e = std::getenv("SRT3D_FAULT"))
      if (std::strncmp(e, "gridwait:", 9) == 0) inject = std::strtoull(e + 9, nullptr, 10) == frame_id;
    st = reconstruct_impl(ctx, f->S, f->n, rows, cols, T, m, f->h, prm, f->depth, f->alpha, f->active, f->alpha0,
                          f->scratch, f->scratch_bytes, s.stream, f->flags, inject);
    if (st != SRT3D_OK) return st;
    const size_t K = prm.k_max;
    st = grow_pinned(ctx, &s.pin_out, &s.pin_out_bytes, out_bytes(f));
    if (st != SRT3D_OK) return st;
    char* po = static_cast<char*>(s.pin_out);
    size_t off = 0;
    auto d2h = [&](const void* src, size_t bytes) {
      cudaError_t e = cudaMemcpyAsync(po + off, src, bytes, cudaMemcpyDeviceToHost, s.stream);
      off += al256(bytes);
      return e;
    };
    SRT3D_CUDA_TRY(ctx, d2h(f->depth, size_t(P) * K * 4));
    SRT3D_CUDA_TRY(ctx, d2h(f->alpha, size_t(P) * K * 4));
    SRT3D_CUDA_TRY(ctx, d2h(f->active, size_t(P) * K));
    SRT3D_CUDA_TRY(ctx, d2h(f->alpha0, size_t(P) * 4));
    SRT3D_CUDA_TRY(ctx, d2h(f->n, size_t(P) * 4));
    SRT3D_CUDA_TRY(ctx, d2h(f->flags, 4));
    SRT3D_CUDA_TRY(ctx, cudaEventRecord(s.done, s.stream));
  }
  return SRT3D_OK;
}

extern "C" srt3d_status srt3d_poll(srt3d_ctx* ctx, uint64_t frame_id, uint32_t timeout_us, float* depth,
                                   float* alpha, uint8_t* active, float* alpha0, uint32_t* n) {
  if (!ctx) return SRT3D_EINVAL;
  Serving* sv = serving(ctx);
  cudaEvent_t done = nullptr;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->frames.find(frame_id);
    if (it == sv->frames.end()) return set_error(ctx, SRT3D_ENOTFOUND, "unknown frame id");
    if (!it->second->closed) return set_error(ctx, SRT3D_EAGAIN, "frame has not received its last chunk");
    done = sv->slots[it->second->slot].done;
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t q = cudaEventQuery(done);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return cuda_error(ctx, q, "cudaEventQuery(frame)");
    const auto us = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0);
    if (uint64_t(us.count()) >= timeout_us) return set_error(ctx, SRT3D_ETIMEDOUT, "frame not done in time");
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->frames.find(frame_id);
  if (it == sv->frames.end()) return set_error(ctx, SRT3D_ENOTFOUND, "frame released concurrently");
  Frame* f = it->second;
  Slot& s = sv->slots[f->slot];
  const size_t P = size_t(f->rows) * f->cols, K = f->prm.k_max;
  const char* po = static_cast<const char*>(s.pin_out);
  size_t off = 0;
  auto out = [&](void* dst, size_t bytes) {
    if (dst) std::memcpy(dst, po + off, bytes);
    off += al256(bytes);
  };
  out(depth, P * K * 4);
  out(alpha, P * K * 4);
  out(active, P * K);
  out(alpha0, P * 4);
  out(n, P * 4);
  uint32_t flags = 0;
  out(&flags, 4);
  release_frame(ctx, sv, f);
  if (flags & FLAG_OFFSETS) return set_error(ctx, SRT3D_EOFFSETS, "malformed offsets in a chunk");
  if (flags & FLAG_STAMP_RANGE) return set_error(ctx, SRT3D_ERANGE, "a stamp >= T in a chunk");
  if (flags & FLAG_DEVICE_TIMEOUT)
    return set_error(ctx, SRT3D_ETIMEDOUT, "a device wait of the frame's reconstruction gave up (partial result)");
  return SRT3D_OK;
}
