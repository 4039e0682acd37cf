// Tracing: per-phase GPU time from CUDA events, and a small arithmetic
// throughput probe used for the ALU roofline.
//
// When profiling is on, every phase of gca_build and of the products
// records an event pair on its stream (PhaseScope); gca_profile_read
// synchronises, sums the elapsed times per phase name and clears them.
// Profiling is process wide and meant for one thread.

#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.hpp"

namespace gca {

namespace {

struct Pending {
  std::string name;
  cudaEvent_t a, b;
  int launches;
};

std::mutex g_mu;
bool g_on = false;
bool g_detail = false;
std::vector<Pending> g_pending;
std::map<std::string, std::pair<int64_t, double>> g_acc;  // launches, ms

void drain_locked() {
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      auto& e = g_acc[p.name];
      e.first += p.launches;
      e.second += ms;
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_pending.clear();
}

}  // namespace

bool profile_detail() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on && g_detail;
}

PhaseScope::PhaseScope(const char* name, cudaStream_t s) : name_(name), s_(s) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  if (cudaEventCreate(reinterpret_cast<cudaEvent_t*>(&a_)) != cudaSuccess) return;
  if (cudaEventCreate(reinterpret_cast<cudaEvent_t*>(&b_)) != cudaSuccess) {
    cudaEventDestroy(static_cast<cudaEvent_t>(a_));
    a_ = nullptr;
    return;
  }
  cudaEventRecord(static_cast<cudaEvent_t>(a_), s_);
  active_ = true;
}

PhaseScope::~PhaseScope() {
  if (!active_) return;
  cudaEventRecord(static_cast<cudaEvent_t>(b_), s_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_pending.push_back({name_, static_cast<cudaEvent_t>(a_), static_cast<cudaEvent_t>(b_), launches_});
  if (g_pending.size() > 4096) drain_locked();
}

namespace {

// FMA chains: 8 independent accumulators per thread, `iters` rounds
template <typename T>
__global__ void k_fma_probe(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = x[j] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == (T)-1.2345) out[0] = s;  // keep the chain alive
}

// The float32 chains as packed pairs (fma.rn.f32x2, the instruction of the
// float product and entry kernels): 8 independent pair accumulators.
__global__ void k_fma2_probe(float* out, int iters, float a, float b) {
  float2 x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = make_float2((float)(threadIdx.x + j), (float)(threadIdx.x - j));
  const float2 aa = make_float2(a, a), bb = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = __ffma2_rn(x[j], aa, bb);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j].x + x[j].y;
  if (s == -1.2345f) out[0] = s;  // keep the chain alive
}

template <typename T>
double fma_probe_flops() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return 0.0;
  const int threads = 256, blocks = sms * 8, iters = 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // float: packed pairs, two FMAs per instruction
  auto run = [&](int it) {
    if constexpr (sizeof(T) == 4)
      k_fma2_probe<<<blocks, threads>>>(out, it, 0.999f, 0.001f);
    else
      k_fma_probe<T><<<blocks, threads>>>(out, it, (T)0.999, (T)0.001);
  };
  run(64);  // warm up
  cudaEventRecord(e0);
  run(iters);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  const double flops = 2.0 * 8.0 * (sizeof(T) == 4 ? 2.0 : 1.0) * iters * (double)threads * blocks;
  return ms > 0.f ? flops / (ms * 1e-3) : 0.0;
}

}  // namespace

}  // namespace gca

extern "C" {

int gca_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(gca::g_mu);
  gca::g_on = on != 0;
  gca::g_detail = on >= 2;
  return GCA_OK;
}

int gca_profile_read(gca_phase* out, int32_t cap, int32_t* count) {
  if (!count || (cap > 0 && !out)) {
    gca::set_error("gca_profile_read: NULL argument");
    return GCA_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(gca::g_mu);
  gca::drain_locked();
  int32_t i = 0;
  for (auto& kv : gca::g_acc) {
    if (i < cap) {
      std::memset(&out[i], 0, sizeof(gca_phase));
      std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
      out[i].launches = kv.second.first;
      out[i].ms = kv.second.second;
    }
    ++i;
  }
  *count = i;
  gca::g_acc.clear();
  return GCA_OK;
}

int gca_peak_probe(double* fp64_flops, double* fp32_flops) {
  if (!fp64_flops || !fp32_flops) {
    gca::set_error("gca_peak_probe: NULL argument");
    return GCA_ERR_INVALID_ARG;
  }
  *fp64_flops = gca::fma_probe_flops<double>();
  *fp32_flops = gca::fma_probe_flops<float>();
  if (cudaGetLastError() != cudaSuccess) {
    gca::set_error("gca_peak_probe: launch failed");
    return GCA_ERR_CUDA;
  }
  return GCA_OK;
}

}  // extern "C"
