// Throughput probes for the roofline denominators of the ALU-bound blend
// kernels: FP32 FMA and MUFU ex2 rates of this GPU at its current clocks.
// Every thread runs kChains independent chains (no dependence stalls) and the
// grid fills every SM at full occupancy, so the rate is the issue limit.
#include <algorithm>

#include "internal.cuh"

namespace hpxgs {
namespace {

constexpr int kProbeThreads = 512, kChains = 8, kUnroll = 16;

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, float a, float b, float* sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)threadIdx.x * 1e-6f + (float)c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.2345f) sink[0] = s;   // a value the chains never reach: keeps them live
}

__device__ __forceinline__ float ex2_neg(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));   // 2^-x stays in (0.5, 1] for x in [0, 1]
  return y;
}

__global__ void __launch_bounds__(kProbeThreads) k_ex2_probe(int iters, float* sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)threadIdx.x * 1e-4f + 0.1f * (float)c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = ex2_neg(x[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.2345f) sink[0] = s;
}

// One grid barrier waiting for gridDim.x + missing arrivals.
__global__ void __launch_bounds__(128) k_barrier_probe(uint32_t* counter, uint32_t missing, uint64_t limit_ns,
                                                      uint32_t* passed, int32_t* status) {
  const bool ok = grid_barrier(counter, gridDim.x + missing, limit_ns, status);
  if (threadIdx.x == 0) passed[blockIdx.x] = ok ? 1u : 0u;
}

}  // namespace
}  // namespace hpxgs

using namespace hpxgs;

extern "C" int hpxgs_probe_alu_peak(double* fma_tflops, double* ex2_tops, hpxgs_stream_t stream) {
  if (!fma_tflops || !ex2_tops) return HPXGS_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return HPXGS_E_CUDA;
  if (cs != cudaStreamCaptureStatusNone) return HPXGS_E_CAPTURE;
  int per_sm = 0;
  HPXGS_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe, kProbeThreads, 0));
  const int grid_fma = std::max(1, per_sm) * num_sms();
  HPXGS_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ex2_probe, kProbeThreads, 0));
  const int grid_ex2 = std::max(1, per_sm) * num_sms();
  cudaEvent_t e[4];
  for (auto& ev : e) HPXGS_CUDA_CHECK(cudaEventCreate(&ev));
  const int it_fma = 4096, it_ex2 = 512;
  int rc = HPXGS_OK;
  // warm-up launches, then one timed launch of each
  k_fma_probe<<<grid_fma, kProbeThreads, 0, s>>>(64, 0.999f, 1e-3f, nullptr);
  k_ex2_probe<<<grid_ex2, kProbeThreads, 0, s>>>(16, nullptr);
  cudaEventRecord(e[0], s);
  k_fma_probe<<<grid_fma, kProbeThreads, 0, s>>>(it_fma, 0.999f, 1e-3f, nullptr);
  cudaEventRecord(e[1], s);
  cudaEventRecord(e[2], s);
  k_ex2_probe<<<grid_ex2, kProbeThreads, 0, s>>>(it_ex2, nullptr);
  cudaEventRecord(e[3], s);
  note_launches(4);
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e[3]) != cudaSuccess) rc = HPXGS_E_CUDA;
  float ms_fma = 0.f, ms_ex2 = 0.f;
  if (rc == HPXGS_OK && (cudaEventElapsedTime(&ms_fma, e[0], e[1]) != cudaSuccess ||
                         cudaEventElapsedTime(&ms_ex2, e[2], e[3]) != cudaSuccess || ms_fma <= 0.f || ms_ex2 <= 0.f))
    rc = HPXGS_E_CUDA;
  for (auto& ev : e) cudaEventDestroy(ev);
  if (rc != HPXGS_OK) return rc;
  const double per_thread = (double)kChains * kUnroll;
  *fma_tflops = 2.0 * per_thread * it_fma * (double)grid_fma * kProbeThreads / (ms_fma * 1e-3) / 1e12;
  *ex2_tops = per_thread * it_ex2 * (double)grid_ex2 * kProbeThreads / (ms_ex2 * 1e-3) / 1e12;
  return HPXGS_OK;
}

extern "C" int hpxgs_probe_grid_barrier(int blocks, int missing, uint64_t limit_ns, uint32_t* counter,
                                        uint32_t* passed, int32_t* status, hpxgs_stream_t stream) {
  if (blocks < 1 || missing < 0 || limit_ns > 2000000000ull || !counter || !passed || !status)
    return HPXGS_E_INVALID_ARG;
  int dev = 0, coop = 0, per_sm = 0;
  HPXGS_CUDA_CHECK(cudaGetDevice(&dev));
  HPXGS_CUDA_CHECK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  HPXGS_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barrier_probe, 128, 0));
  if (!coop || blocks > per_sm * num_sms()) return HPXGS_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  HPXGS_CUDA_CHECK(cudaMemsetAsync(counter, 0, sizeof(uint32_t), s));
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)blocks);
  lc.blockDim = dim3(128);
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  HPXGS_CUDA_CHECK(cudaLaunchKernelEx(&lc, k_barrier_probe, counter, (uint32_t)missing, limit_ns, passed, status));
  note_launches(1);
  return HPXGS_OK;
}
