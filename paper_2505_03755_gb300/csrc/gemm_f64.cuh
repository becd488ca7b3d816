// FP64 GEMM on the double-precision tensor path (mma.sync.m16n8k4.f64, "DMMA").
//
//   C[z](m, n) (=|+=) alpha * sum_{k in split} A[b](m, k) * B[b](k, n),   b = z / ksplit
//
// CTA tile 64 x 64, K step 16, four warps with 32 x 32 warp tiles (2 x 4 DMMA tiles each).
// Operands are staged through shared memory element by element via loader objects (see
// las_common.cuh); on GB300 the FP64 pipe delivers about 3.5 flop/clk/SM, so one 64x64x16 step
// (131k flops) takes ~37k cycles of DMMA issue and the 2048 staged loads are not the bound.
#pragma once
#include "las_common.cuh"

namespace lasdf {

__device__ __forceinline__ void dmma_16x8x4(double (&c)[4], double a0, double a1, double b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};\n"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a0), "d"(a1), "d"(b0));
}

template <class LA, class LB, class SC>
__global__ void __launch_bounds__(128)
k_gemm_f64(int M, int N, int K, int ksplit, int kchunk, LA la, LB lb, SC sc) {
  __shared__ double As[16][64 + 2];
  __shared__ double Bs[16][64 + 2];
  const int z = blockIdx.z;
  const int b = z / ksplit;
  const int ks = z - b * ksplit;
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  const int kbeg = ks * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  const int g = lane >> 2, t = lane & 3;
  double acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0;

  for (int k0 = kbeg; k0 < kend; k0 += 16) {
#pragma unroll 4
    for (int i = tid; i < 1024; i += 128) {
      const int mm = i & 63, kk = i >> 6;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < kend) ? la(b, m, k) : 0.0;
      const int n = n0 + mm;
      Bs[kk][mm] = (n < N && k < kend) ? lb(b, k, n) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; kk += 4) {
      double a[2][2], bb[4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        a[i][0] = As[kk + t][wm + i * 16 + g];
        a[i][1] = As[kk + t][wm + i * 16 + g + 8];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk + t][wn + j * 8 + g];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dmma_16x8x4(acc[i][j], a[i][0], a[i][1], bb[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r0 = m0 + wm + i * 16 + g;
      const int c0 = n0 + wn + j * 8 + 2 * t;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = r0 + ((r >> 1) << 3);
        const int col = c0 + (r & 1);
        if (row < M && col < N) sc(z, row, col, acc[i][j][r]);
      }
    }
}

}  // namespace lasdf

template <class LA, class LB, class SC>
void gemm_f64(int M, int N, int K, int batch, int ksplit, LA a, LB b, SC c, cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (ksplit < 1) ksplit = 1;
  int kchunk = (K + ksplit - 1) / ksplit;
  kchunk = (kchunk + 15) / 16 * 16;
  if (kchunk < 16) kchunk = 16;
  dim3 grid((M + 63) / 64, (N + 63) / 64, batch * ksplit);
  lasdf::k_gemm_f64<LA, LB, SC><<<grid, 128, 0, s>>>(M, N, K, ksplit, kchunk, a, b, c);
  las_count_launch();
}
