// Small FP64 kernels of the LAS energy/gradient chain: per-auxiliary-index contractions with the
// block-product RDMs, energy reduction, gradient assembly and layout helpers.
#include <algorithm>

#include "las_common.cuh"

namespace lasdf {

// Deterministic block sums of K doubles per thread: warp butterflies (lane 0's order is fixed),
// then the warp partials in warp order; every thread returns the K totals.  red: NT/32*K doubles.
template <int NT, int K>
__device__ void block_sums(double (&v)[K], double* red) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[w * K + k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) t += red[i * K + k];
    v[k] = t;
  }
  __syncthreads();
}

// Deterministic block reduction of one double per thread (fixed tree order).
template <int NT>
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

__global__ void k_pack_cocc(const double* __restrict__ C, int n, int nmo, int o, int op,
                            double* __restrict__ Cocc) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long total = (long)n * op;
  if (i >= total) return;
  int mu = (int)(i / op), p = (int)(i % op);
  Cocc[i] = (p < o) ? C[(long)mu * nmo + p] : 0.0;
}

__device__ __forceinline__ int frag_of(const FragInfo& fi, int u) {
  int K = 0;
  while (K + 1 < fi.nfrag && fi.off[K + 1] <= u) ++K;
  return K;
}

// Per auxiliary index L (one CTA each), given T_L = C_occ^T b^L C_occ (op x op):
//   vc = 2 sum_i T(i,i)                     (Coulomb vector of Dc, Eq. J_1 in the MO basis)
//   va = sum_uv D_uv T(u,v)                 (Coulomb vector of the active density)
//   Y(u,v) = sum_wx Gamma_uvwx T(w,x)       (block-product 2-RDM of Eq. las_wfn, applied
//                                            fragment-block by fragment-block)
//   eps_L  = vc^2/2 - sum_ij T(i,j)^2 + vc va - sum_{i,u} Z(i,u) T(i,u) + 1/2 sum_uv T(u,v) Y(u,v)
//            with Z = T(core,act) D  (the L-th term of the two-electron energy)
//   W_L(p,q): the matrix with  dE/dC(two-electron part) = sum_L H_L W_L, H_L = b^L C_occ.
// x * 2^g for normal or zero x (exponent-field arithmetic; no FP64 multiply)
__device__ __forceinline__ double scale2(double x, int g) {
  long long b = __double_as_longlong(x);
  if ((b & 0x7FF0000000000000ll) == 0) return x == 0.0 ? x : ldexp(x, g);
  return __longlong_as_double(b + (((long long)g) << 52));
}

__global__ void __launch_bounds__(256)
k_per_aux(const double* __restrict__ T, int nL, int op, const double* __restrict__ dm1s,
          const double* __restrict__ dm2, FragInfo fi, double* __restrict__ W,
          double* __restrict__ eps, double* __restrict__ vcv, double* __restrict__ vav,
          int with_grad, const int* __restrict__ gexp, int* status, int use_p) {
  extern __shared__ double sm[];
  const int a = fi.nact, c = fi.ncore, o = c + a;
  double* Taa = sm;             // a*a
  double* Ds = Taa + a * a;     // a*a (block diagonal D)
  double* Y = Ds + a * a;       // a*a
  double* red = Y + a * a;      // 256
  double* cK = red + 256;       // nfrag
  double* P = cK + LAS_MAX_FRAG;  // a*a when the launch provides it (fast cross-fragment path)
  const long Lb = blockIdx.x;
  const double* TL = T + Lb * (long)op * op;
  const int tid = threadIdx.x;

  for (int i = tid; i < a * a; i += 256) {
    int u = i / a, v = i % a;
    Taa[i] = TL[(long)(c + u) * op + c + v];
    int K = frag_of(fi, u);
    double d = 0.0;
    if (v >= fi.off[K] && v < fi.off[K + 1]) {
      int m = fi.off[K + 1] - fi.off[K];
      int uu = u - fi.off[K], vv = v - fi.off[K];
      const double* g = dm1s + fi.dm1_off[K];
      d = g[uu * m + vv] + g[m * m + uu * m + vv];
    }
    Ds[i] = d;
  }
  __syncthreads();

  double pvc = 0.0, pcore = 0.0;
  for (int i = tid; i < c; i += 256) pvc += TL[(long)i * op + i];
  for (long i = tid; i < (long)c * c; i += 256) {
    double x = TL[(i / c) * op + (i % c)];
    pcore += x * x;
  }
  double pva = 0.0;
  for (int i = tid; i < a * a; i += 256) pva += Ds[i] * Taa[i];
  double r3[3] = {pvc, pcore, pva};
  block_sums<256, 3>(r3, red);
  const double vc = 2.0 * r3[0], fro = r3[1], va = r3[2];
  if (tid < fi.nfrag) {
    int K = tid, o0 = fi.off[K], m = fi.off[K + 1] - o0;
    double s = 0.0;
    for (int u = 0; u < m; ++u)
      for (int v = 0; v < m; ++v) s += Ds[(o0 + u) * a + o0 + v] * Taa[(o0 + u) * a + o0 + v];
    cK[K] = s;
  }
  __syncthreads();

  // Y = Gamma . T over the active block, fragment structure of Eq. las_wfn.
  for (int i = tid; i < a * a; i += 256) {
    const int u = i / a, v = i % a;
    const int K = frag_of(fi, u), Kp = frag_of(fi, v);
    const int oK = fi.off[K], mK = fi.off[K + 1] - oK;
    double y = 0.0;
    if (K != Kp && use_p) {
      // cross-fragment blocks come from the factored form below
    } else if (K == Kp) {
      const double* g2 = dm2 + fi.dm2_off[K];
      const int uu = u - oK, vv = v - oK;
      const double* gr = g2 + ((long)uu * mK + vv) * mK * mK;
      for (int w = 0; w < mK; ++w)
        for (int x = 0; x < mK; ++x) y += gr[w * mK + x] * Taa[(oK + w) * a + oK + x];
      y += Ds[i] * (va - cK[K]);
    } else {
      // -sum_sigma sum_{x in K, w in K'} gK_s[u,x] T(x,w) gK'_s[w,v]
      const int oP = fi.off[Kp], mP = fi.off[Kp + 1] - oP;
      const double* gK = dm1s + fi.dm1_off[K];
      const double* gP = dm1s + fi.dm1_off[Kp];
      const int uu = u - oK, vv = v - oP;
      for (int s = 0; s < 2; ++s) {
        const double* gKs = gK + s * mK * mK;
        const double* gPs = gP + s * mP * mP;
        for (int x = 0; x < mK; ++x) {
          double gux = gKs[uu * mK + x];
          if (gux == 0.0) continue;
          double t = 0.0;
          for (int w = 0; w < mP; ++w) t += Taa[(oK + x) * a + oP + w] * gPs[w * mP + vv];
          y -= gux * t;
        }
      }
    }
    Y[i] = y;
  }
  if (use_p) {
    // -sum_sigma gK_s (T_KK' gK'_s) for K != K': P_s = T_aa blockdiag(g_s) first (a*a*m work),
    // then the left factor, instead of the inner sum per (u, v)
    for (int sg = 0; sg < 2; ++sg) {
      __syncthreads();
      for (int i = tid; i < a * a; i += 256) {
        const int x = i / a, v = i % a;
        const int Kp = frag_of(fi, v), oP = fi.off[Kp], mP = fi.off[Kp + 1] - oP;
        const double* gPs = dm1s + fi.dm1_off[Kp] + sg * mP * mP;
        const int vv = v - oP;
        double t = 0.0;
        for (int w = 0; w < mP; ++w) t += Taa[x * a + oP + w] * gPs[w * mP + vv];
        P[i] = t;
      }
      __syncthreads();
      for (int i = tid; i < a * a; i += 256) {
        const int u = i / a, v = i % a;
        const int K = frag_of(fi, u), Kp = frag_of(fi, v);
        if (K == Kp) continue;
        const int oK = fi.off[K], mK = fi.off[K + 1] - oK;
        const double* gKs = dm1s + fi.dm1_off[K] + sg * mK * mK;
        const int uu = u - oK;
        double t = 0.0;
        for (int x = 0; x < mK; ++x) t += gKs[uu * mK + x] * P[(oK + x) * a + v];
        Y[i] -= t;
      }
    }
  }
  __syncthreads();

  // Z(i,u) = sum_v T(i, c+v) D(v,u) over core i and active u; its contraction with T(i,u).
  double pz = 0.0;
  double* WL = W + Lb * (long)op * op;
  const long wld = (long)nL * op;
  // W_L(p,q) -> its storage slot (plain, or transposed and scaled by 2^gexp for split mode)
  auto putW = [&](int p, int q, double w) {
    if (gexp) {
      const long k = Lb * (long)op + p;
      W[(long)q * wld + k] = scale2(w, gexp[k]);
    } else {
      WL[(long)p * op + q] = w;
    }
  };
  for (long idx = tid; idx < (long)c * a; idx += 256) {
    const int i = (int)(idx / a), u = (int)(idx % a);
    const int K = frag_of(fi, u), oK = fi.off[K], mK = fi.off[K + 1] - oK;
    const double* Ti = TL + (long)i * op + c;
    double z = 0.0;
    for (int v = oK; v < oK + mK; ++v) z += Ti[v] * Ds[v * a + u];
    pz += z * Ti[u];
    if (with_grad) {
      putW(i, c + u, -2.0 * z);
      putW(c + u, i, -2.0 * z);
    }
  }
  double pe = 0.0;
  for (int i = tid; i < a * a; i += 256) pe += Taa[i] * Y[i];
  double r2[2] = {pz, pe};
  block_sums<256, 2>(r2, red);
  const double zt = r2[0], ty = r2[1];
  if (tid == 0) {
    eps[Lb] = 0.5 * vc * vc - fro + vc * va - zt + 0.5 * ty;
    vcv[Lb] = vc;
    vav[Lb] = va;
  }
  if (!with_grad) return;
  // core-core block, active-active block and zero padding
  for (long idx = tid; idx < (long)op * op; idx += 256) {
    // q-major in split mode so that consecutive threads write consecutive p (coalesced)
    const int p = gexp ? (int)(idx % op) : (int)(idx / op);
    const int q = gexp ? (int)(idx / op) : (int)(idx % op);
    double w;
    if (p < c && q < c) {
      w = -4.0 * TL[(long)p * op + q] + (p == q ? 4.0 * (vc + va) : 0.0);
    } else if (p >= c && p < o && q >= c && q < o) {
      const int wv = p - c, u = q - c;
      w = 2.0 * vc * Ds[wv * a + u] + 2.0 * Y[u * a + wv];
    } else if (p >= o || q >= o) {
      w = 0.0;
    } else {
      continue;  // core/active blocks written above
    }
    putW(p, q, w);
  }
}

// Cocc[mu][k] = Cx[mu][k] * sqrt(max(sign * w[k], 0)) for k < r, zero for r <= k < op
// Columns of one sign of the weights, in order: idx[0..cnt) (sign = +1 or -1 picks w > 0 or w < 0).
__global__ void k_sign_split(const double* __restrict__ w, int r, int* __restrict__ idx_pos,
                             int* __restrict__ idx_neg, int* __restrict__ counts) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int np = 0, nn = 0;
  for (int k = 0; k < r; ++k) {
    if (w[k] > 0.0) idx_pos[np++] = k;
    else if (w[k] < 0.0) idx_neg[nn++] = k;
  }
  counts[0] = np;
  counts[1] = nn;
}

// Cocc[mu][j] = Cx[mu][idx[j]] * sqrt(sign * w[idx[j]]) for j < cnt, zero for cnt <= j < op
__global__ void k_pack_weighted(const double* __restrict__ Cx, const double* __restrict__ w,
                                const int* __restrict__ idx, int cnt, double sign, int n, int r,
                                int op, double* __restrict__ Cocc) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)n * op) return;
  const int mu = (int)(i / op), j = (int)(i % op);
  double v = 0.0;
  if (j < cnt) {
    const int k = idx[j];
    v = Cx[(long)mu * r + k] * sqrt(sign * w[k]);
  }
  Cocc[i] = v;
}

// K[i][j] = K[j][i] for i < j (copy the lower triangle to the upper)
__global__ void k_mirror_lower(double* __restrict__ K, int n) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  if (i < j) K[idx] = K[(long)j * n + i];
}

// dT[L][p][q] = X[L][p][q] + X[L][q][p]  (the symmetric tangent of T_L = C^T b^L C)
__global__ void k_sym_add(const double* __restrict__ X, long nL, int op, double* __restrict__ dT) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long per = (long)op * op;
  if (i >= nL * per) return;
  const long L = i / per, r = i - L * per;
  const int p = (int)(r / op), q = (int)(r - (long)p * op);
  dT[i] = X[i] + X[L * per + (long)q * op + p];
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, double a, long count) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < count) y[i] += a * x[i];
}

__global__ void k_scale(double* __restrict__ p, long count, double a) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < count) p[i] *= a;
}

__global__ void k_reduce_partials(const double* __restrict__ part, int nsplit, long count,
                                  double* __restrict__ out, int accumulate) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= count) return;
  double s = accumulate ? out[i] : 0.0;
  for (int k = 0; k < nsplit; ++k) s += part[(long)k * count + i];
  out[i] = s;
}

// dE/dC = [4 h C_core | 2 h C_act D | 0] + Out   (Out = sum_L H_L W_L, n x op)
__global__ void k_assemble_grad(const double* __restrict__ Out, const double* __restrict__ hC,
                                const double* __restrict__ dm1s, FragInfo fi, int n, int nmo,
                                int op, double* __restrict__ G) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)n * nmo) return;
  const int mu = (int)(i / nmo), q = (int)(i % nmo);
  const int c = fi.ncore, o = c + fi.nact;
  double g = 0.0;
  if (q < c) {
    g = 4.0 * hC[(long)mu * op + q] + Out[(long)mu * op + q];
  } else if (q < o) {
    const int u = q - c;
    const int K = frag_of(fi, u), oK = fi.off[K], m = fi.off[K + 1] - oK;
    const double* gK = dm1s + fi.dm1_off[K];
    double s = 0.0;
    for (int v = 0; v < m; ++v) {
      double d = gK[v * m + (u - oK)] + gK[m * m + v * m + (u - oK)];
      s += hC[(long)mu * op + c + oK + v] * d;
    }
    g = 2.0 * s + Out[(long)mu * op + q];
  }
  G[i] = g;
}

// E = 2 sum_i hmo(i,i) + sum_uv hmo(c+u,c+v) D_uv + sum_L eps_L  (one CTA, fixed order,
// compensated summation).
__global__ void __launch_bounds__(256)
k_energy_final(const double* __restrict__ eps, int X, const double* __restrict__ hmo, int op,
               const double* __restrict__ dm1s, FragInfo fi, double* __restrict__ E) {
  __shared__ double red[256];
  double s = 0.0, comp = 0.0;
  auto add = [&](double x) {  // Neumaier
    double t = s + x;
    if (fabs(s) >= fabs(x)) comp += (s - t) + x; else comp += (x - t) + s;
    s = t;
  };
  for (int L = threadIdx.x; L < X; L += 256) add(eps[L]);
  const int c = fi.ncore;
  for (int i = threadIdx.x; i < c; i += 256) add(2.0 * hmo[(long)i * op + i]);
  for (int K = 0; K < fi.nfrag; ++K) {
    const int oK = fi.off[K], m = fi.off[K + 1] - oK;
    const double* g = dm1s + fi.dm1_off[K];
    for (int i = threadIdx.x; i < m * m; i += 256) {
      const int u = i / m, v = i % m;
      add(hmo[(long)(c + oK + u) * op + c + oK + v] * (g[i] + g[m * m + i]));
    }
  }
  double tot = block_sum<256>(s + comp, red);
  if (threadIdx.x == 0) *E = tot;
}

// g[p][q] = M'[p][q] - M'[q][p],  M'[p][q] = M[p][q] for q < o else 0  (M is nmo x op)
__global__ void k_antisym(const double* __restrict__ M, int nmo, int o, int op,
                          double* __restrict__ g) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)nmo * nmo) return;
  const int p = (int)(i / nmo), q = (int)(i % nmo);
  double x = (q < o) ? M[(long)p * op + q] : 0.0;
  double y = (p < o) ? M[(long)q * op + p] : 0.0;
  g[i] = x - y;
}

// Jp[pair] = sum_L vc[L] Bp[L][pair]  (Eq. J_2 on the packed triangle; coalesced along pairs)
__global__ void k_coulomb_packed(const double* __restrict__ Bp, const double* __restrict__ vc,
                                 int X, long npair, double* __restrict__ Jp) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= npair) return;
  double s = 0.0;
  for (int L = 0; L < X; ++L) s += vc[L] * Bp[(long)L * npair + i];
  Jp[i] = s;
}

__global__ void k_unpack_sym(const double* __restrict__ Jp, int n, double* __restrict__ J) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)n * n) return;
  long mu = i / n, nu = i % n;
  long hi = mu > nu ? mu : nu, lo = mu > nu ? nu : mu;
  J[i] = Jp[hi * (hi + 1) / 2 + lo];
}

// Lmu[L][mu][u] = Ht[L][c0+u][mu]
__global__ void k_copy_cols(const double* __restrict__ Ht, int X, int op, int n, int c0, int a,
                            double* __restrict__ Lmu) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long total = (long)X * n * a;
  if (i >= total) return;
  const int u = (int)(i % a);
  const long r = i / a;
  const int mu = (int)(r % n);
  const long L = r / n;
  Lmu[i] = Ht[(L * op + c0 + u) * n + mu];
}

__global__ void k_transpose_cols(const double* __restrict__ C, int n, int op, int r,
                                 double* __restrict__ CT) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;   // over r*n, mu fastest
  if (i >= (long)r * n) return;
  const int k = (int)(i / n), mu = (int)(i - (long)k * n);
  CT[i] = C[(long)mu * op + k];
}

// Coulomb traces: one block per aux row, coalesced along mu, tree reduction in a fixed order.
__global__ void __launch_bounds__(256)
k_trace_ht(const double* __restrict__ Ht, const double* __restrict__ CT, int r, int n,
           double* __restrict__ vc) {
  __shared__ double red[256];
  const long b = blockIdx.x;
  const long cnt = (long)r * n;
  const double* h = Ht + b * cnt;
  double acc = 0.0;
  for (long i = threadIdx.x; i < cnt; i += 256) acc = fma(h[i], CT[i], acc);
  const double t = block_sum<256>(acc, red);
  if (threadIdx.x == 0) vc[b] = 2.0 * t;
}

// out (atomic max) = max |a[i]| as an ordered bit pattern (block tree, then one atomic per block)
__global__ void __launch_bounds__(256)
k_absmax_bits(const double* __restrict__ a, long count, unsigned long long* out) {
  __shared__ unsigned long long red[256];
  unsigned long long m = 0;
  for (long i = blockIdx.x * 256L + threadIdx.x; i < count; i += (long)gridDim.x * 256) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(a[i]) & 0x7FFFFFFFFFFFFFFFull;
    m = b > m ? b : m;
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w && red[threadIdx.x + w] > red[threadIdx.x])
      red[threadIdx.x] = red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && red[0]) atomicMax(out, red[0]);
}

}  // namespace lasdf

using namespace lasdf;

static inline unsigned nblk(long count, int nt) { return (unsigned)((count + nt - 1) / nt); }

void launch_pack_cocc(const double* C, int n, int nmo, int o, int op, double* Cocc,
                      cudaStream_t s) {
  k_pack_cocc<<<nblk((long)n * op, 256), 256, 0, s>>>(C, n, nmo, o, op, Cocc);
  las_count_launch();
}

#define LAS_PER_AUX_FAST_MAX_ACT 84
static size_t per_aux_fast_smem(int a) {
  return (4 * (size_t)a * a + 256 + LAS_MAX_FRAG) * sizeof(double);
}

las_status per_aux_prepare(int nact) {
  // always the largest supported size, so that contexts with different active spaces coexist
  (void)nact;
  size_t smem = (3 * (size_t)LAS_MAX_ACT * LAS_MAX_ACT + 256 + LAS_MAX_FRAG) * sizeof(double);
  smem = std::max(smem, per_aux_fast_smem(LAS_PER_AUX_FAST_MAX_ACT));
  cudaError_t e = cudaFuncSetAttribute(k_per_aux, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)std::max<size_t>(smem, 48 * 1024));
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "cudaFuncSetAttribute(k_per_aux)", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  return LAS_OK;
}

void launch_per_aux(const double* T, int nL, int op, const double* dm1s, const double* dm2,
                    const FragInfo& fi, double* W, double* eps, double* vc, double* va,
                    int with_grad, const int* gexp, int* status, cudaStream_t s) {
  if (nL <= 0) return;
  // the factored cross-fragment path needs one more a*a buffer; it fits for a <= 84
  const int use_p = fi.nfrag > 1 && fi.nact <= LAS_PER_AUX_FAST_MAX_ACT;
  size_t smem = use_p ? per_aux_fast_smem(fi.nact)
                      : (3 * (size_t)fi.nact * fi.nact + 256 + LAS_MAX_FRAG) * sizeof(double);
  k_per_aux<<<nL, 256, smem, s>>>(T, nL, op, dm1s, dm2, fi, W, eps, vc, va, with_grad, gexp,
                                  status, use_p);
  las_count_launch();
}

void launch_sign_split(const double* w, int r, int* idx_pos, int* idx_neg, int* counts,
                       cudaStream_t s) {
  k_sign_split<<<1, 32, 0, s>>>(w, r, idx_pos, idx_neg, counts);
  las_count_launch();
}

void launch_pack_weighted(const double* Cx, const double* w, const int* idx, int cnt,
                          double sign, int n, int r, int op, double* Cocc, cudaStream_t s) {
  k_pack_weighted<<<nblk((long)n * op, 256), 256, 0, s>>>(Cx, w, idx, cnt, sign, n, r, op,
                                                         Cocc);
  las_count_launch();
}

void launch_mirror_lower(double* K, int n, cudaStream_t s) {
  k_mirror_lower<<<nblk((long)n * n, 256), 256, 0, s>>>(K, n);
  las_count_launch();
}

void launch_sym_add(const double* X, int nL, int op, double* dT, cudaStream_t s) {
  const long count = (long)nL * op * op;
  if (count <= 0) return;
  k_sym_add<<<nblk(count, 256), 256, 0, s>>>(X, nL, op, dT);
  las_count_launch();
}

void launch_axpy(double* y, const double* x, double a, long count, cudaStream_t s) {
  if (count <= 0) return;
  k_axpy<<<nblk(count, 256), 256, 0, s>>>(y, x, a, count);
  las_count_launch();
}

void launch_transpose_cols(const double* Cocc, int n, int op, int r, double* CT,
                           cudaStream_t s) {
  const long cnt = (long)r * n;
  if (cnt <= 0) return;
  k_transpose_cols<<<nblk(cnt, 256), 256, 0, s>>>(Cocc, n, op, r, CT);
  las_count_launch();
}

void launch_trace_ht(const double* Ht, const double* CT, int nL, int r, int n, double* vc,
                     cudaStream_t s) {
  if (nL <= 0) return;
  k_trace_ht<<<nL, 256, 0, s>>>(Ht, CT, r, n, vc);
  las_count_launch();
}

void launch_scale(double* p, long count, double a, cudaStream_t s) {
  if (count <= 0) return;
  k_scale<<<nblk(count, 256), 256, 0, s>>>(p, count, a);
  las_count_launch();
}

void launch_reduce_partials(const double* part, int nsplit, long count, double* out,
                            int accumulate, cudaStream_t s) {
  k_reduce_partials<<<nblk(count, 256), 256, 0, s>>>(part, nsplit, count, out, accumulate);
  las_count_launch();
}

void launch_assemble_grad(const double* Out, const double* hC, const double* dm1s,
                          const FragInfo& fi, int n, int nmo, int op, double* G,
                          cudaStream_t s) {
  k_assemble_grad<<<nblk((long)n * nmo, 256), 256, 0, s>>>(Out, hC, dm1s, fi, n, nmo, op, G);
  las_count_launch();
}

void launch_energy_final(const double* eps, int X, const double* hmo, int op,
                         const double* dm1s, const FragInfo& fi, double* E, cudaStream_t s) {
  k_energy_final<<<1, 256, 0, s>>>(eps, X, hmo, op, dm1s, fi, E);
  las_count_launch();
}

void launch_absmax_bits(const double* a, long count, unsigned long long* out, cudaStream_t s) {
  if (count <= 0) return;
  k_absmax_bits<<<(unsigned)std::min<long>(nblk(count, 256), 1024), 256, 0, s>>>(a, count, out);
  las_count_launch();
}

void launch_antisym(const double* M, int nmo, int o, int op, double* g, cudaStream_t s) {
  k_antisym<<<nblk((long)nmo * nmo, 256), 256, 0, s>>>(M, nmo, o, op, g);
  las_count_launch();
}

void launch_coulomb_packed(const double* Bp, const double* vc, int X, long npair, double* Jp,
                           cudaStream_t s) {
  k_coulomb_packed<<<nblk(npair, 256), 256, 0, s>>>(Bp, vc, X, npair, Jp);
  las_count_launch();
}

void launch_unpack_sym(const double* Jp, int n, double* J, cudaStream_t s) {
  k_unpack_sym<<<nblk((long)n * n, 256), 256, 0, s>>>(Jp, n, J);
  las_count_launch();
}

void launch_copy_cols(const double* Ht, int X, int op, int n, int c0, int a, double* Lmu,
                      cudaStream_t s) {
  k_copy_cols<<<nblk((long)X * n * a, 256), 256, 0, s>>>(Ht, X, op, n, c0, a, Lmu);
  las_count_launch();
}
