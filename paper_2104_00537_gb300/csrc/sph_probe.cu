// sph_probe.cu -- throughput of this GPU's FP32 and FP64 fused multiply-add
// pipes, the denominators of the interaction kernel's roofline (the pair loop
// is bound by FP32 arithmetic issue, not by HBM).  Not an operation of the
// paper: a measurement helper behind sph_probe_peaks.
//
// Every thread runs kChains independent FMA chains x <- x a + b (|a| < 1, so
// the values stay bounded), enough independent work per warp to hide the
// pipe latency; the grid fills every SM with kBlocksPerSm blocks of 256
// threads.  The chains' sum is stored only if it is NaN (never), which keeps
// the compiler from dropping the loop.
#include <algorithm>
#include <string>

#include "../../include/sph.h"
#include "sph_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T a, T b, T *sink) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 1
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int r = 0; r < 16; r++) {
#pragma unroll
      for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += x[k];
  if (s != s) *sink = s;
}

int fail(int code, const std::string &msg) {
  sph::set_last_error(msg);
  return code;
}

// Best of `reps` timed launches after one untimed launch; TFLOP/s.
template <typename T>
int measure(int sms, int iters, int reps, cudaStream_t s, T *sink, double *tflops) {
  const int blocks = sms * kBlocksPerSm;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(SPH_ERR_CUDA, "sph_probe_peaks: cudaEventCreate");
  float best = 1e30f;
  k_fma_chains<T><<<blocks, kThreads, 0, s>>>(iters, (T)0.999999, (T)1e-7, sink);
  for (int r = 0; r < reps; r++) {
    cudaEventRecord(e0, s);
    k_fma_chains<T><<<blocks, kThreads, 0, s>>>(iters, (T)0.999999, (T)1e-7, sink);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return fail(SPH_ERR_CUDA, cudaGetErrorString(err));
  // 2 FLOP per FMA
  const double flop = 2.0 * blocks * (double)kThreads * iters * 16.0 * kChains;
  *tflops = flop / (best * 1e-3) / 1e12;
  return SPH_OK;
}

}  // namespace

extern "C" int sph_probe_peaks(double *fp32_tflops, double *fp64_tflops, int32_t *sm_count,
                               void *stream) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0)
    return fail(SPH_ERR_CUDA, "sph_probe_peaks: no device");
  if (sm_count) *sm_count = sms;
  cudaStream_t s = (cudaStream_t)stream;
  void *sink = nullptr;
  if (cudaMalloc(&sink, 16) != cudaSuccess) return fail(SPH_ERR_OOM, "sph_probe_peaks: sink");
  int rc = SPH_OK;
  // ~10 ms per FP32 launch near 75 TFLOP/s; FP64 runs at a small fraction
  if (fp32_tflops) rc = measure<float>(sms, 8192, 3, s, (float *)sink, fp32_tflops);
  if (rc == SPH_OK && fp64_tflops) rc = measure<double>(sms, 96, 3, s, (double *)sink, fp64_tflops);
  cudaFree(sink);
  return rc;
}
