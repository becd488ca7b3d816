// FP64 throughput probe: the denominator of the native-FP64 roofline.  Two register-resident
// loops fill every SM: one of FP64 tensor-core MMAs (mma.sync m16n8k4 f64, the instruction the
// FP64 GEMM kernel is built on) and one of FP64 fused multiply-adds, each with eight independent
// accumulator chains per thread so that issue, not latency, bounds the loop.  Nothing is read or
// written in the timed loop; one conditional store keeps the results live.
#include <cuda_runtime.h>

#include "las_common.cuh"

namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;

__global__ void __launch_bounds__(PROBE_THREADS)
k_probe_dmma(int iters, double* sink) {
  // per thread: two A values, one B value, four accumulators of the 16 x 8 tile
  const double a0 = 1e-3 * (threadIdx.x & 31), a1 = 2e-3, b = 1.0 + 1e-6 * blockIdx.x;
  double c[PROBE_CHAINS][4];
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j)
      asm volatile(
          "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
          "{%0,%1,%2,%3};"
          : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3])
          : "d"(a0), "d"(a1), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
  if (s == -1.0) sink[0] = s;   // never true for these operands; keeps the chains live
}

__global__ void __launch_bounds__(PROBE_THREADS)
k_probe_dfma(int iters, double* sink) {
  const double a = 1.0 - 1e-9 * threadIdx.x, b = 1e-7;
  double c[PROBE_CHAINS];
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) c[j] = (double)j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) c[j] = fma(c[j], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) s += c[j];
  if (s == -1.0) sink[0] = s;
}

// Seconds of one launch of `k` (after one warm-up launch), timed with events on `st`.
template <class K>
las_status time_launch(K k, int blocks, int iters, double* sink, cudaStream_t st, double* sec) {
  cudaEvent_t e0, e1;
  LAS_CUDA_TRY(cudaEventCreate(&e0));
  LAS_CUDA_TRY(cudaEventCreate(&e1));
  k<<<blocks, PROBE_THREADS, 0, st>>>(iters / 10 + 1, sink);
  las_count_launch();
  cudaEventRecord(e0, st);
  k<<<blocks, PROBE_THREADS, 0, st>>>(iters, sink);
  las_count_launch();
  cudaEventRecord(e1, st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "FP64 probe", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  *sec = ms * 1e-3;
  return LAS_OK;
}

}  // namespace

extern "C" las_status las_probe_fp64(double* dmma_tflops, double* dfma_tflops, void* stream) {
  if (!dmma_tflops || !dfma_tflops) return LAS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  LAS_CUDA_TRY(cudaGetDevice(&dev));
  LAS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  double* sink = nullptr;
  LAS_CUDA_TRY(cudaMalloc(&sink, sizeof(double)));
  const int blocks = 4 * nsm;   // 32 warps per SM
  const int it_mma = 4000, it_fma = 20000;
  double t = 0.0;
  las_status rc = time_launch(k_probe_dmma, blocks, it_mma, sink, st, &t);
  if (rc == LAS_OK) {
    // 2 * 16 * 8 * 4 flop per warp-wide MMA
    const double flop = (double)blocks * (PROBE_THREADS / 32) * it_mma * PROBE_CHAINS * 1024.0;
    *dmma_tflops = flop / t * 1e-12;
    rc = time_launch(k_probe_dfma, blocks, it_fma, sink, st, &t);
  }
  if (rc == LAS_OK) {
    const double flop = (double)blocks * PROBE_THREADS * it_fma * PROBE_CHAINS * 2.0;
    *dfma_tflops = flop / t * 1e-12;
  }
  cudaFree(sink);
  return rc;
}
