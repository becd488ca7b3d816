// Internal declarations shared by the translation units of liblasdf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/las.h"

#define LAS_MAX_FRAG 64
#define LAS_MAX_ACT 96  // total active orbitals handled by the per-L kernel (3a^2 doubles of smem)

// Device status word codes (first error wins; see las_status).
#define LAS_DEV_OK 0

#define LAS_CUDA_TRY(expr)                               \
  do {                                                   \
    cudaError_t e_ = (expr);                             \
    if (e_ != cudaSuccess) {                             \
      las_record_cuda_error(e_, #expr, __FILE__, __LINE__); \
      return LAS_ERR_CUDA;                               \
    }                                                    \
  } while (0)

void las_record_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Process-wide count of kernels this library has launched (diagnostics).
void las_count_launch(long k = 1);

// Fragment description in constant-size form (passed by value to kernels).
struct FragInfo {
  int nfrag;
  int ncore;
  int nact;                      // total active orbitals a
  int off[LAS_MAX_FRAG + 1];     // active offsets (relative to the first active orbital)
  long dm1_off[LAS_MAX_FRAG];    // offset of fragment K in dm1s (doubles)
  long dm2_off[LAS_MAX_FRAG];    // offset of fragment K in dm2 (doubles)
};

// ------------------------------------------------------------------------------------------
// Generic FP64 GEMM on DMMA (mma.sync.m16n8k4.f64):  C[b](m,n) (+)= alpha * sum_k A[b](m,k) B[b](k,n)
// Operands are read through small loader objects so that packed-symmetric B, transposed views
// and batched/strided layouts share one kernel.  FP64 arithmetic on this part is slow enough
// (about 3.5 flop/clk/SM) that element-wise staging through shared memory is never the bound.
// ------------------------------------------------------------------------------------------
struct StridedA {  // element (b, m, k) = p[b*sb + m*sm + k*sk]
  const double* p;
  long sb, sm, sk;
  __device__ __forceinline__ double operator()(int b, int m, int k) const {
    return p[(long)b * sb + (long)m * sm + (long)k * sk];
  }
};

// Element (b, mu, nu) of the symmetric matrix b^L (L = l0 + b) stored packed lower-triangular.
struct PackedSymA {
  const double* Bp;
  long npair;
  long l0;
  __device__ __forceinline__ double operator()(int b, int mu, int nu) const {
    long hi = mu > nu ? mu : nu, lo = mu > nu ? nu : mu;
    return Bp[(l0 + b) * npair + hi * (hi + 1) / 2 + lo];
  }
};

struct StridedC {  // C[b*sb + m*sm + n*sn] (=|+=) alpha * acc
  double* p;
  long sb, sm, sn;
  double alpha;
  int accumulate;
  __device__ __forceinline__ void operator()(int b, int m, int n, double v) const {
    double* q = p + (long)b * sb + (long)m * sm + (long)n * sn;
    *q = accumulate ? (*q + alpha * v) : alpha * v;
  }
};

template <class LA, class LB, class SC>
void gemm_f64(int M, int N, int K, int batch, int ksplit, LA a, LB b, SC c, cudaStream_t s);

// Small helpers implemented in las_kernels.cu
void launch_pack_cocc(const double* C, int n, int nmo, int o, int op, double* Cocc,
                      cudaStream_t s);
las_status per_aux_prepare(int nact);
// gexp == nullptr: W[L][p][q];  otherwise W is written as Wt[q][L*op + p] * 2^gexp[L*op + p]
// CT[k][mu] = Cocc[mu][k] for k < r (Cocc is n x op)
void launch_transpose_cols(const double* Cocc, int n, int op, int r, double* CT, cudaStream_t s);
// vc[b] = 2 sum_{k<r} sum_mu Ht[(b*r + k)*n + mu] * CT[k*n + mu], b < nL (fixed summation order)
void launch_trace_ht(const double* Ht, const double* CT, int nL, int r, int n, double* vc,
                     cudaStream_t s);
void launch_per_aux(const double* T, int nL, int op, const double* dm1s, const double* dm2,
                    const FragInfo& fi, double* W, double* eps, double* vc, double* va,
                    int with_grad, const int* gexp, int* status, cudaStream_t s);
void launch_scale(double* p, long count, double a, cudaStream_t s);
void launch_mirror_lower(double* K, int n, cudaStream_t s);
void launch_axpy(double* y, const double* x, double a, long count, cudaStream_t s);
// dT[L] = X[L] + X[L]^T for L < nL (op x op each)
void launch_sym_add(const double* X, int nL, int op, double* dT, cudaStream_t s);
// *out (atomic max, caller zeroes it) = max_i |a[i]| as the bit pattern of the double
void launch_absmax_bits(const double* a, long count, unsigned long long* out, cudaStream_t s);
// Columns of each sign of w (k_sign_split), then the packed factor of one sign
void launch_sign_split(const double* w, int r, int* idx_pos, int* idx_neg, int* counts,
                       cudaStream_t s);
void launch_pack_weighted(const double* Cx, const double* w, const int* idx, int cnt,
                          double sign, int n, int r, int op, double* Cocc, cudaStream_t s);
void launch_reduce_partials(const double* part, int nsplit, long count, double* out,
                            int accumulate, cudaStream_t s);
void launch_assemble_grad(const double* Out, const double* hC, const double* dm1s,
                          const FragInfo& fi, int n, int nmo, int op, double* G,
                          cudaStream_t s);
void launch_energy_final(const double* eps, int X, const double* hmo, int op,
                         const double* dm1s, const FragInfo& fi, double* E, cudaStream_t s);
void launch_antisym(const double* M, int nmo, int o, int op, double* g, cudaStream_t s);
void launch_coulomb_packed(const double* Bp, const double* vc, int X, long npair,
                           double* Jp, cudaStream_t s);
void launch_unpack_sym(const double* Jp, int n, double* J, cudaStream_t s);
void launch_copy_cols(const double* Ht, int X, int op, int n, int c0, int a, double* Lmu,
                      cudaStream_t s);
