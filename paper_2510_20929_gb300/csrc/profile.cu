// Per-kernel CUDA-event profiler behind ptycho_profile_enable / ptycho_profile_read.
#include <mutex>
#include <string.h>
#include <vector>

#include "ptycho.h"
#include "profile.h"

namespace ptycho {
namespace {
struct Pending {
  int id;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
int g_only = -1;   // record only this kernel id (-1: all)
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
double g_ms[K_COUNT];
long g_launches[K_COUNT];

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void drain_locked() {
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_ms[p.id] += ms;
      g_launches[p.id] += 1;
    }
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
}
}  // namespace

const char* kernel_name(int id) {
  static const char* names[K_COUNT] = {"k_pass1",      "k_pass2",        "k_probe_reduce", "k_norm_probe",
                                       "k_probe_update", "k_init_epoch", "k_opr_reduce",   "k_opr_weights",
                                       "k_tile_illum_max", "k_tile_clear", "k_pass1_ms",
                                       "k_clear_plane", "k_pass1_exit", "k_far_tc", "k_pass1_overlap",
                                       "k_dft_planes"};
  return (id >= 0 && id < K_COUNT) ? names[id] : "?";
}

bool profiling_on() { return g_on; }

cudaEvent_t profile_begin(int id, cudaStream_t s) {
  if (!g_on || (g_only >= 0 && id != g_only)) return nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t a = take_event();
  if (a) cudaEventRecord(a, s);
  return a;
}

void profile_end(int id, cudaEvent_t a, cudaStream_t s) {
  if (!a) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  if (!b) return;
  cudaEventRecord(b, s);
  g_pending.push_back({id, a, b});
}
}  // namespace ptycho

using namespace ptycho;

extern "C" {

ptycho_status ptycho_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return PTYCHO_OK;
}

int32_t ptycho_profile_select(const char* name) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!name) {
    g_only = -1;
    return 1;
  }
  for (int id = 0; id < K_COUNT; ++id)
    if (strcmp(name, kernel_name(id)) == 0) {
      g_only = id;
      return 1;
    }
  return 0;
}

int32_t ptycho_profile_read(ptycho_kernel_time* out, int32_t cap) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  int32_t n = 0;
  for (int id = 0; id < K_COUNT; ++id) {
    if (g_launches[id] == 0) continue;
    if (out && n < cap) {
      memset(&out[n], 0, sizeof(out[n]));
      strncpy(out[n].name, kernel_name(id), sizeof(out[n].name) - 1);
      out[n].launches = (int32_t)g_launches[id];
      out[n].total_ms = g_ms[id];
    }
    ++n;
    g_launches[id] = 0;
    g_ms[id] = 0.0;
  }
  return n;
}

}  // extern "C"
