// Runtime support: per-device grow-only workspace, pointer classification,
// launch accounting and status strings.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "engine.h"

namespace mp {

namespace {

constexpr int kSlots = 8;
constexpr int kMaxDevices = 64;

struct Ws {
  void* ptr[kSlots] = {};
  size_t size[kSlots] = {};
};

Ws g_ws[kMaxDevices];
std::mutex g_ws_mu;
std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_fail_allocs{0};   // injected workspace failures still to deliver

}  // namespace

void* workspace(size_t bytes, int slot) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  if (slot < 0 || slot >= kSlots) return nullptr;
  for (int left = g_fail_allocs.load(); left > 0;)
    if (g_fail_allocs.compare_exchange_weak(left, left - 1)) return nullptr;
  std::lock_guard<std::mutex> lock(g_ws_mu);
  Ws& w = g_ws[dev];
  if (bytes == 0) bytes = 256;
  if (w.size[slot] >= bytes) return w.ptr[slot];
  if (w.ptr[slot]) {
    // work already queued may still read the old buffer
    cudaDeviceSynchronize();
    cudaFree(w.ptr[slot]);
    w.ptr[slot] = nullptr;
    w.size[slot] = 0;
  }
  size_t want = bytes + bytes / 4;   // head-room so that small growths do not reallocate
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    want = bytes;
  }
  w.ptr[slot] = p;
  w.size[slot] = want;
  return p;
}

bool is_device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void* pinned_alias(const void* p) {
  if (!p) return nullptr;
  static const bool enabled = [] {
    const char* e = std::getenv("MAPPLE_PINNED_DIRECT");
    return !(e && e[0] == '0');
  }();
  if (!enabled) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
thread_local char g_err[512] = "";
}  // namespace

void record_cuda_error(cudaError_t e, const char* file, int line) {
  const char* base = file;
  for (const char* c = file; *c; ++c)
    if (*c == '/') base = c + 1;
  std::snprintf(g_err, sizeof(g_err), "%s:%d: %s (%s)", base, line, cudaGetErrorName(e), cudaGetErrorString(e));
}

namespace {
cudaEvent_t g_t0 = nullptr, g_t1 = nullptr;
bool g_armed = false;
cudaEvent_t g_lt0 = nullptr, g_lt1 = nullptr;   // the learned scorer's layer kernel
bool g_larmed = false;
}  // namespace

void timer_begin(cudaStream_t st) {
  if (g_armed && g_t0) cudaEventRecord(g_t0, st);
}

void timer_end(cudaStream_t st) {
  if (g_armed && g_t1) cudaEventRecord(g_t1, st);
  g_armed = false;
}

void layer_timer_begin(cudaStream_t st) {
  if (g_larmed && g_lt0) cudaEventRecord(g_lt0, st);
}

void layer_timer_end(cudaStream_t st) {
  if (g_larmed && g_lt1) cudaEventRecord(g_lt1, st);
  g_larmed = false;
}

}  // namespace mp

extern "C" const char* mp_strerror(int status) {
  switch (status) {
    case MP_OK: return "ok";
    case MP_EINVAL: return "invalid argument (transform, rank, extent or distribution)";
    case MP_EOVERFLOW: return "point count or id range overflows";
    case MP_ENOMEM: return "device workspace allocation failed";
    case MP_ECUDA: return "CUDA runtime error";
    case MP_ETIMEOUT: return "device-side wait timed out";
    case MP_ENOTSUP: return "size beyond the engine's supported limits";
    default: return "unknown status";
  }
}

extern "C" uint64_t mp_kernel_launches(void) { return mp::g_launches.load(); }

extern "C" const char* mp_last_error_detail(void) { return mp::g_err; }

extern "C" int mp_set_kernel_timer(void* start_event, void* stop_event) {
  mp::g_t0 = (cudaEvent_t)start_event;
  mp::g_t1 = (cudaEvent_t)stop_event;
  mp::g_armed = start_event && stop_event;
  return MP_OK;
}

extern "C" int mp_set_layer_timer(void* start_event, void* stop_event) {
  mp::g_lt0 = (cudaEvent_t)start_event;
  mp::g_lt1 = (cudaEvent_t)stop_event;
  mp::g_larmed = start_event && stop_event;
  return MP_OK;
}

extern "C" uint64_t mp_descriptor_bytes(void) { return sizeof(mp::MapDesc); }

extern "C" uint64_t mp_workspace_bytes(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= mp::kMaxDevices) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lock(mp::g_ws_mu);
  uint64_t total = 0;
  for (int s = 0; s < mp::kSlots; ++s) total += mp::g_ws[dev].size[s];
  return total;
}

extern "C" int mp_debug_fail_allocations(int32_t n) {
  if (n < 0) return MP_EINVAL;
  mp::g_fail_allocs.store(n);
  return MP_OK;
}
