// C ABI of liblasdf: context, validation, workspace plan and the evaluation chain.
//
// Evaluation chain for a chunk of auxiliary indices L (all FP64 in LAS_FP64 mode):
//   S1  H_L  = b^L C_occ              half transform, Eq. ao2mo_1 (and the first GEMM of K_1)
//   S2  T_L  = C_occ^T H_L            full transform over the occupied space, Eq. ao2mo_2
//   S3/S4 per L: Coulomb vectors (Eq. J_1), Y_L = Gamma . T_L (the ppaa-type contraction with
//       the block-product 2-RDM), the energy term eps_L and the projection matrix W_L
//   S5/S6 Out += sum_L H_L W_L        (J_2 and K_2 projected on C_occ, and the active
//                                      two-electron gradient)
// then E = sum_L eps_L + one-electron terms, dE/dC = [4 h C_c | 2 h C_a D | 0] + Out, and
// g = C^T dE/dC - transpose.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "gemm_f64.cuh"
#include "las_common.cuh"
#include "las_split.cuh"

#define LAS_TIMING_RING 64
#define LAS_MARKS 6

#include <atomic>

static thread_local char g_last_error[512];
static std::atomic<long> g_launches{0};

void las_count_launch(long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

extern "C" long las_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void las_record_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s failed: %s (%s:%d)", what,
           cudaGetErrorString(e), file, line);
}

struct las_ctx {
  int n, X, nmo, c, a, o, op;
  long npair;
  las_precision prec;
  FragInfo fi;
  FragInfo fi_c;  // core only (for the Coulomb vector of Dc)
  const double* Bp;
  cudaStream_t stream;
  size_t ws_cap;
  int Lc;       // auxiliary chunk length
  int ksplit;   // split of the projection GEMM
  // workspace (device)
  double* Cocc;   // [n][op]
  double* Ht;     // [Lc][op][n]
  double* T;      // [Lc][op][op]
  double* W;      // [Lc][op][op]
  double* part;   // [ksplit][n][op]
  double* Out;    // [n][op]
  double* hC;     // [n][op]
  double* hmo;    // [op][op]
  double* M;      // [nmo][op]
  double* eps;    // [X]
  double* vc;     // [X]
  double* va;     // [X]
  double* Jp;     // [npair] (JK)
  double* Jt;     // [n][n]  J of one sign part (general-density JK)
  double* Kt;     // [n][n]  K of one sign part
  int* status;    // device status word
  // staging for the host-buffer call
  double *dC, *dh, *ddm1, *ddm2, *dE, *dG;
  long ndm1, ndm2;
  size_t bytes;
  // split-precision state (owned)
  SplitState* split;
  // fragment AO2MO workspace (allocated by the first las_frag_ao2mo call)
  double *fH, *fT, *fpart;
  long fLc, fpart_elems;
  size_t fbytes;   // device bytes of the fragment AO2MO workspace (counted in `bytes`)
  int fnmo, fma;
  FragSplit* fsplit;
  double *vJ, *vK;   // scratch of las_veff (allocated by its first call)
  // scratch of las_orbital_hvp (allocated by its first call): dC = C X and G(C) [n][nmo]; the
  // tangent chain's dC_occ, h dC_occ and projection [n][op], dH [Lc][op][n], X = H^T dC, dT and
  // the two W matrices of the tangent [Lc][op][op]
  double *hdC, *hG, *tCocc, *thC, *tOut, *tHt, *tX, *tdT, *tdW, *tWd;
  int* widx;          // [2*o + 2] columns of each weight sign and their counts (JK density)
  int wcount[2];      // host copy of those counts
  // timing: a ring of LAS_TIMING_RING evaluations x 6 stage marks, read without per-call syncs
  int timing;
  cudaEvent_t* ev;       // [LAS_TIMING_RING][6]
  int slot, recorded;
  int nstage;
};

extern "C" const char* las_status_str(las_status s) {
  switch (s) {
    case LAS_OK: return "ok";
    case LAS_ERR_ARG: return "invalid argument";
    case LAS_ERR_CUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case LAS_ERR_WORKSPACE: return "workspace cap too small";
    case LAS_ERR_TIMEOUT: return "device-side wait timed out";
    case LAS_ERR_INTERNAL: return "device-side consistency check failed";
    case LAS_ERR_UNSUPPORTED: return "unsupported size or mode";
  }
  return "unknown status";
}

static las_status dalloc(las_ctx* x, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return LAS_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
    *p = nullptr;
    return LAS_ERR_CUDA;
  }
  x->bytes += bytes;
  return LAS_OK;
}

static void free_all(las_ctx* x) {
  void* ptrs[] = {x->Cocc, x->Ht, x->T, x->W, x->part, x->Out, x->hC, x->hmo, x->M, x->eps,
                  x->vc, x->va, x->Jp, x->Jt, x->Kt, x->widx, x->status, x->dC, x->dh, x->ddm1, x->ddm2,
                  x->dE, x->dG};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (x->split) split_destroy(x->split);
  if (x->fsplit) frag_split_destroy(x->fsplit);
  for (double* q : {x->fH, x->fT, x->fpart, x->vJ, x->vK, x->hdC, x->hG, x->tCocc, x->thC,
                    x->tOut, x->tHt, x->tX, x->tdT, x->tdW, x->tWd})
    if (q) cudaFree(q);
  if (x->ev) {
    for (int i = 0; i < LAS_TIMING_RING * LAS_MARKS; ++i)
      if (x->ev[i]) cudaEventDestroy(x->ev[i]);
    free(x->ev);
  }
}

static size_t chunk_bytes(const las_ctx* x, int Lc) {
  size_t op = x->op, n = x->n;
  size_t b = (size_t)Lc * op * (n + 2 * op) * sizeof(double);
  if (x->prec == LAS_SPLIT_BF16) b += (size_t)Lc * split_bytes_per_aux(x->n, x->op);
  return b;
}

extern "C" las_status las_create(las_ctx** out, const las_dims* d, const double* B_packed,
                                 las_precision prec, size_t max_ws, void* stream) {
  if (!out || !d || !B_packed) return LAS_ERR_ARG;
  *out = nullptr;
  if (d->nao <= 0 || d->naux <= 0 || d->nmo <= 0 || d->ncore < 0 || d->nfrag < 0) return LAS_ERR_ARG;
  if (d->nfrag > LAS_MAX_FRAG || (d->nfrag > 0 && !d->nact)) return LAS_ERR_ARG;
  if (prec != LAS_FP64 && prec != LAS_SPLIT_BF16 && prec != LAS_SPLIT_BF16_PACKED)
    return LAS_ERR_ARG;
  // the packed-triangle digit layout is a variant of the split mode: the context runs as
  // LAS_SPLIT_BF16 everywhere else
  const int packed = prec == LAS_SPLIT_BF16_PACKED;
  if (packed) prec = LAS_SPLIT_BF16;
  int a = 0;
  for (int k = 0; k < d->nfrag; ++k) {
    if (d->nact[k] < 1) return LAS_ERR_ARG;
    a += d->nact[k];
  }
  if (d->ncore + a > d->nmo || d->nmo > d->nao) return LAS_ERR_ARG;
  if (a > LAS_MAX_ACT) return LAS_ERR_UNSUPPORTED;
  if (d->ncore + a == 0) return LAS_ERR_ARG;

  las_ctx* x = (las_ctx*)calloc(1, sizeof(las_ctx));
  if (!x) return LAS_ERR_INTERNAL;
  x->n = d->nao;
  x->X = d->naux;
  x->nmo = d->nmo;
  x->c = d->ncore;
  x->a = a;
  x->o = d->ncore + a;
  x->op = (x->o + 15) / 16 * 16;
  x->npair = (long)x->n * (x->n + 1) / 2;
  x->prec = prec;
  x->Bp = B_packed;
  x->stream = (cudaStream_t)stream;
  x->fi.nfrag = d->nfrag;
  x->fi.ncore = d->ncore;
  x->fi.nact = a;
  long o1 = 0, o2 = 0;
  x->fi.off[0] = 0;
  for (int k = 0; k < d->nfrag; ++k) {
    int m = d->nact[k];
    x->fi.off[k + 1] = x->fi.off[k] + m;
    x->fi.dm1_off[k] = o1;
    x->fi.dm2_off[k] = o2;
    o1 += 2L * m * m;
    o2 += (long)m * m * m * m;
  }
  x->ndm1 = o1;
  x->ndm2 = o2;
  memset(&x->fi_c, 0, sizeof(x->fi_c));
  x->fi_c.ncore = d->ncore;

  // Workspace plan: the largest auxiliary chunk that fits the cap.
  const size_t fixed = sizeof(double) * ((size_t)x->n * x->op * 4 + (size_t)x->op * x->op +
                                         (size_t)x->nmo * x->op + 3 * (size_t)x->X + x->npair);
  size_t cap = max_ws ? max_ws : (size_t)64 << 30;
  int Lc = x->X;
  while (Lc > 1 && fixed + chunk_bytes(x, Lc) + (size_t)64 * x->n * x->op * 8 > cap) Lc = (Lc + 1) / 2;
  if (fixed + chunk_bytes(x, Lc) > cap) {
    free(x);
    return LAS_ERR_WORKSPACE;
  }
  x->Lc = Lc;
  x->ws_cap = cap;
  {
    int tiles = ((x->n + 63) / 64) * ((x->op + 63) / 64);
    int ks = (4 * 152 + tiles - 1) / tiles;
    int kmax = std::max(1, (Lc * x->op) / 256);
    x->ksplit = std::max(1, std::min(std::min(ks, 64), kmax));
  }
  las_status st = LAS_OK;
#define ALLOC(ptr, count) \
  if (st == LAS_OK) st = dalloc(x, (void**)&x->ptr, sizeof(*x->ptr) * (size_t)(count));
  ALLOC(Cocc, (size_t)x->n * x->op);
  ALLOC(Ht, (size_t)Lc * x->op * x->n);
  ALLOC(T, (size_t)Lc * x->op * x->op);
  ALLOC(W, (size_t)Lc * x->op * x->op);
  ALLOC(part, (size_t)x->ksplit * x->n * x->op);
  ALLOC(Out, (size_t)x->n * x->op);
  ALLOC(hC, (size_t)x->n * x->op);
  ALLOC(hmo, (size_t)x->op * x->op);
  ALLOC(M, (size_t)x->nmo * x->op);
  ALLOC(eps, x->X);
  ALLOC(vc, x->X);
  ALLOC(va, x->X);
  ALLOC(Jp, x->npair);
  ALLOC(Jt, (size_t)x->n * x->n);
  ALLOC(Kt, (size_t)x->n * x->n);
  ALLOC(widx, 2 * (size_t)x->o + 2);
  ALLOC(status, 4);
  ALLOC(dC, (size_t)x->n * x->nmo);
  ALLOC(dh, (size_t)x->n * x->n);
  ALLOC(ddm1, std::max(1L, x->ndm1));
  ALLOC(ddm2, std::max(1L, x->ndm2));
  ALLOC(dE, 1);
  ALLOC(dG, (size_t)x->n * x->nmo);
#undef ALLOC
  if (st == LAS_OK) {
    cudaError_t e = cudaMemsetAsync(x->status, 0, 4 * sizeof(int), x->stream);
    if (e != cudaSuccess) {
      las_record_cuda_error(e, "cudaMemsetAsync", __FILE__, __LINE__);
      st = LAS_ERR_CUDA;
    }
  }
  if (st == LAS_OK) {
    st = per_aux_prepare(a);
  }
  if (st == LAS_OK && prec == LAS_SPLIT_BF16) {
    st = split_create(&x->split, x->n, x->X, x->op, x->Lc, B_packed, packed, x->status,
                      x->stream, &x->bytes);
  }
  if (st == LAS_OK) {
    cudaError_t e = cudaStreamSynchronize(x->stream);
    if (e != cudaSuccess) {
      las_record_cuda_error(e, "cudaStreamSynchronize", __FILE__, __LINE__);
      st = LAS_ERR_CUDA;
    }
  }
  if (st != LAS_OK) {
    free_all(x);
    free(x);
    return st;
  }
  *out = x;
  return LAS_OK;
}

// Captured batched evaluations, keyed by (contexts, item pointers, stream).
struct GraphEntry {
  std::vector<las_ctx*> ctxs;
  std::vector<las_batch_item> items;
  cudaStream_t stream;
  cudaGraphExec_t exec;
  void* probs;   // device descriptions of the grouped products (grouped graphs only)
};
static std::mutex g_graph_mu;
static std::vector<GraphEntry> g_graphs;

static void drop_graphs_of(las_ctx* x) {
  std::lock_guard<std::mutex> lock(g_graph_mu);
  for (size_t i = 0; i < g_graphs.size();) {
    bool hit = false;
    for (las_ctx* c : g_graphs[i].ctxs) hit |= (c == x);
    if (hit) {
      cudaGraphExecDestroy(g_graphs[i].exec);
      if (g_graphs[i].probs) cudaFree(g_graphs[i].probs);
      g_graphs.erase(g_graphs.begin() + i);
    } else {
      ++i;
    }
  }
}

extern "C" las_status las_destroy(las_ctx* x) {
  if (!x) return LAS_ERR_ARG;
  cudaStreamSynchronize(x->stream);
  drop_graphs_of(x);
  free_all(x);
  free(x);
  return LAS_OK;
}

extern "C" las_status las_set_stream(las_ctx* x, void* stream) {
  if (!x) return LAS_ERR_ARG;
  x->stream = (cudaStream_t)stream;
  return LAS_OK;
}

extern "C" size_t las_device_bytes(const las_ctx* x) { return x ? x->bytes : 0; }

static las_status check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "kernel launch", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  return LAS_OK;
}

extern "C" las_status las_sync(las_ctx* x) {
  if (!x) return LAS_ERR_ARG;
  LAS_CUDA_TRY(cudaStreamSynchronize(x->stream));
  int h[4] = {0, 0, 0, 0};
  LAS_CUDA_TRY(cudaMemcpy(h, x->status, sizeof(h), cudaMemcpyDeviceToHost));
  if (h[0] != 0) return (las_status)h[0];
  return LAS_OK;
}

extern "C" las_status las_set_timing(las_ctx* x, int enable) {
  if (!x) return LAS_ERR_ARG;
  if (enable && !x->ev) {
    x->ev = (cudaEvent_t*)calloc(LAS_TIMING_RING * LAS_MARKS, sizeof(cudaEvent_t));
    if (!x->ev) return LAS_ERR_INTERNAL;
    for (int i = 0; i < LAS_TIMING_RING * LAS_MARKS; ++i)
      LAS_CUDA_TRY(cudaEventCreate(&x->ev[i]));
  }
  x->timing = enable;
  x->slot = 0;
  x->recorded = 0;
  return LAS_OK;
}

// Average per-stage time over the evaluations recorded since timing was enabled or last read
// (at most LAS_TIMING_RING of them); waits for the last one only.
extern "C" int las_stage_times(las_ctx* x, float* ms, int cap) {
  if (!x || !x->timing || x->recorded == 0 || x->nstage == 0) return 0;
  const int nrec = x->recorded < LAS_TIMING_RING ? x->recorded : LAS_TIMING_RING;
  const int last = (x->slot + LAS_TIMING_RING - 1) % LAS_TIMING_RING;
  if (cudaEventSynchronize(x->ev[last * LAS_MARKS + x->nstage]) != cudaSuccess) return 0;
  int k = 0;
  for (; k < x->nstage && k < cap; ++k) {
    double acc = 0.0;
    for (int r = 0; r < nrec; ++r) {
      const int sl = (x->slot + LAS_TIMING_RING - 1 - r) % LAS_TIMING_RING;
      float t = 0.f;
      cudaEventElapsedTime(&t, x->ev[sl * LAS_MARKS + k], x->ev[sl * LAS_MARKS + k + 1]);
      acc += t;
    }
    ms[k] = (float)(acc / nrec);
  }
  x->recorded = 0;
  return k;
}

static inline void stage_mark(las_ctx* x, int i) {
  if (x->timing && i < LAS_MARKS) {
    cudaEventRecord(x->ev[x->slot * LAS_MARKS + i], x->stream);
    if (i > 0) x->nstage = i;
    if (i == LAS_MARKS - 1) {
      x->slot = (x->slot + 1) % LAS_TIMING_RING;
      ++x->recorded;
    }
  }
}

// ------------------------------------------------------------------------------------------
// Chain pieces
// ------------------------------------------------------------------------------------------
// S1 + S2 on auxiliary rows [l0, l0+nL): Ht[b][p][mu] = (b^L C_occ)(mu,p), T[b] = C_occ^T H
// H_L = b^L C_occ for the chunk's aux rows, over the first oc columns of C_occ (Ht layout
// [nL][oc][n]); with want_T (only for oc = op) also T_L = C_occ^T H_L.
static las_status half_and_full(las_ctx* x, int l0, int nL, int want_T, int mark = -1,
                                int oc = -1) {
  const int n = x->n, op = x->op;
  if (oc < 0) oc = op;
  if (want_T && oc != op) return LAS_ERR_INTERNAL;
  if (x->prec == LAS_SPLIT_BF16) {
    las_status st = split_half(x->split, l0, nL, oc, x->Ht, x->stream);
    if (st != LAS_OK) return st;
    if (mark >= 0) stage_mark(x, mark);
    return want_T ? split_full(x->split, nL, x->Ht, x->T, x->stream) : LAS_OK;
  }
  PackedSymA A{x->Bp, x->npair, l0};
  StridedA Bm{x->Cocc, 0, op, 1};
  StridedC Ch{x->Ht, (long)oc * n, 1, n, 1.0, 0};
  gemm_f64(n, oc, n, nL, 1, A, Bm, Ch, x->stream);
  if (mark >= 0) stage_mark(x, mark);
  if (want_T) {
    StridedA Ah{x->Ht, (long)op * n, n, 1};
    StridedC Ct{x->T, (long)op * op, op, 1, 1.0, 0};
    gemm_f64(op, op, n, nL, 1, Ah, Bm, Ct, x->stream);
  }
  return check_launch();
}

// Out (+)= sum_{b < nL} Ht_b^T W_b   (n x op), split over K = nL*op, partials reduced in order
static las_status project(las_ctx* x, int nL, int accumulate) {
  const int n = x->n, op = x->op;
  if (x->prec == LAS_SPLIT_BF16) {
    return split_project(x->split, nL, x->W, x->Out, accumulate, x->stream);
  }
  int ks = std::max(1, std::min(x->ksplit, (nL * op) / 64));
  StridedA A{x->Ht, 0, 1, n};
  StridedA Bw{x->W, 0, op, 1};
  StridedC Cp{x->part, (long)n * op, op, 1, 1.0, 0};
  gemm_f64(n, op, nL * op, 1, ks, A, Bw, Cp, x->stream);
  launch_reduce_partials(x->part, ks, (long)n * op, x->Out, accumulate, x->stream);
  return check_launch();
}

static las_status evaluate(las_ctx* x, const double* C, const double* h, const double* dm1s,
                           const double* dm2, double* E, double* G, double* gorb) {
  if (!x || !C || !h || !E) return LAS_ERR_ARG;
  if (x->a > 0 && (!dm1s || !dm2)) return LAS_ERR_ARG;
  const int n = x->n, op = x->op, nmo = x->nmo;
  const int with_grad = (G != nullptr) || (gorb != nullptr);
  if (gorb && !G) G = x->dG;
  las_status st;
  stage_mark(x, 0);
  launch_pack_cocc(C, n, nmo, x->o, op, x->Cocc, x->stream);
  if (x->prec == LAS_SPLIT_BF16) {
    st = split_prepare_C(x->split, x->Cocc, x->stream);
    if (st != LAS_OK) return st;
  }
  for (int l0 = 0; l0 < x->X; l0 += x->Lc) {
    const int nL = std::min(x->Lc, x->X - l0);
    if ((st = half_and_full(x, l0, nL, 1, l0 == 0 ? 1 : -1)) != LAS_OK) return st;
    if (l0 == 0) stage_mark(x, 2);
    // split mode: W is written transposed and row-scaled for the split projection GEMM
    launch_per_aux(x->T, nL, op, dm1s, dm2, x->fi, x->W, x->eps + l0, x->vc + l0, x->va + l0,
                   with_grad, x->split ? split_hexp(x->split) : nullptr, x->status, x->stream);
    if ((st = check_launch()) != LAS_OK) return st;
    if (l0 == 0) stage_mark(x, 3);
    if (with_grad && (st = project(x, nL, l0 > 0)) != LAS_OK) return st;
    if (l0 == 0) stage_mark(x, 4);
  }
  if (x->prec == LAS_SPLIT_BF16) {  // one-electron pieces: hC = h C_occ, hmo = C_occ^T hC
    if ((st = split_one_electron(x->split, h, x->hC, x->hmo, x->stream)) != LAS_OK) return st;
  } else {
    StridedA Ah{h, 0, n, 1};
    StridedA Bc{x->Cocc, 0, op, 1};
    StridedC Ch{x->hC, 0, op, 1, 1.0, 0};
    gemm_f64(n, op, n, 1, 1, Ah, Bc, Ch, x->stream);
    StridedA Act{x->Cocc, 0, 1, op};
    StridedA Bh{x->hC, 0, op, 1};
    StridedC Cm{x->hmo, 0, op, 1, 1.0, 0};
    gemm_f64(op, op, n, 1, 1, Act, Bh, Cm, x->stream);
  }
  launch_energy_final(x->eps, x->X, x->hmo, op, dm1s, x->fi, E, x->stream);
  if (with_grad) {
    launch_assemble_grad(x->Out, x->hC, dm1s, x->fi, n, nmo, op, G, x->stream);
    if (gorb) {
      StridedA Act{C, 0, 1, nmo};
      StridedA Bg{G, 0, nmo, 1};
      StridedC Cm{x->M, 0, op, 1, 1.0, 0};
      gemm_f64(nmo, x->o, n, 1, 1, Act, Bg, Cm, x->stream);
      launch_antisym(x->M, nmo, x->o, op, gorb, x->stream);
    }
  }
  stage_mark(x, 5);
  return check_launch();
}

extern "C" las_status las_energy(las_ctx* x, const double* C, const double* h,
                                 const double* dm1s, const double* dm2, double* E) {
  return evaluate(x, C, h, dm1s, dm2, E, nullptr, nullptr);
}

extern "C" las_status las_energy_grad(las_ctx* x, const double* C, const double* h,
                                      const double* dm1s, const double* dm2, double* E,
                                      double* dEdC, double* gorb) {
  if (!dEdC && !gorb) return LAS_ERR_ARG;
  return evaluate(x, C, h, dm1s, dm2, E, dEdC, gorb);
}

extern "C" las_status las_energy_grad_host(las_ctx* x, const double* C_host,
                                           const double* h_host, const double* dm1s_host,
                                           const double* dm2_host, double* E_host,
                                           double* dEdC_host) {
  if (!x || !C_host || !h_host || !E_host) return LAS_ERR_ARG;
  if (x->a > 0 && (!dm1s_host || !dm2_host)) return LAS_ERR_ARG;
  cudaStream_t s = x->stream;
  const size_t nC = (size_t)x->n * x->nmo;
  LAS_CUDA_TRY(cudaMemcpyAsync(x->dC, C_host, nC * 8, cudaMemcpyHostToDevice, s));
  LAS_CUDA_TRY(cudaMemcpyAsync(x->dh, h_host, (size_t)x->n * x->n * 8, cudaMemcpyHostToDevice, s));
  if (x->a > 0) {
    LAS_CUDA_TRY(cudaMemcpyAsync(x->ddm1, dm1s_host, x->ndm1 * 8, cudaMemcpyHostToDevice, s));
    LAS_CUDA_TRY(cudaMemcpyAsync(x->ddm2, dm2_host, x->ndm2 * 8, cudaMemcpyHostToDevice, s));
  }
  las_status st = evaluate(x, x->dC, x->dh, x->ddm1, x->ddm2, x->dE,
                           dEdC_host ? x->dG : nullptr, nullptr);
  if (st != LAS_OK) return st;
  LAS_CUDA_TRY(cudaMemcpyAsync(E_host, x->dE, 8, cudaMemcpyDeviceToHost, s));
  if (dEdC_host) LAS_CUDA_TRY(cudaMemcpyAsync(dEdC_host, x->dG, nC * 8, cudaMemcpyDeviceToHost, s));
  return las_sync(x);
}

// J and K of the density D = sum_{k < r} c_k c_k^T whose columns c_k are in x->Cocc (columns >= r
// zero):  J[mu][nu] = sum_L b^L_{mu nu} Tr(b^L D)  (Eqs. J_1, J_2),
//         K[mu][nu] = sum_L (b^L D b^L)_{mu nu}   (Eqs. K_1, K_2, with b^L D = H_L C^T).
static las_status jk_raw(las_ctx* x, int r, double* J, double* K) {
  const int n = x->n, op = x->op;
  if (x->prec == LAS_SPLIT_BF16) {
    las_status st = split_prepare_C(x->split, x->Cocc, x->stream);
    if (st != LAS_OK) return st;
  }
  // the first r columns of C_occ carry the density; `Out` (n x op, idle here) holds them
  // transposed for the traces of the Coulomb term
  if (J) launch_transpose_cols(x->Cocc, n, op, r, x->Out, x->stream);
  las_status st;
  for (int l0 = 0; l0 < x->X; l0 += x->Lc) {
    const int nL = std::min(x->Lc, x->X - l0);
    // H_L over the r density columns only: Ht is [nL][r][n] here
    if ((st = half_and_full(x, l0, nL, 0, -1, r)) != LAS_OK) return st;
    // vc_L = 2 sum_k c_k^T H_L(k,:)^T = 2 Tr(b^L D)
    if (J) launch_trace_ht(x->Ht, x->Out, nL, r, n, x->vc + l0, x->stream);
    if (K && x->prec == LAS_SPLIT_BF16) {  // K = sum_{L,k} H_L(k,:)^T H_L(k,:)
      if ((st = split_exchange(x->split, nL, r, x->Ht, K, l0 > 0, x->stream)) != LAS_OK)
        return st;
    } else if (K) {
      StridedA A{x->Ht, 0, 1, n};
      StridedA B{x->Ht, 0, n, 1};
      int ks = std::max(1, std::min(x->ksplit, (nL * r) / 64));
      // reuse `part` as [ks][n][n] only when it is large enough; otherwise accumulate directly
      if ((size_t)ks * n * n <= (size_t)x->ksplit * n * op) {
        StridedC Pk{x->part, (long)n * n, n, 1, 1.0, 0};
        gemm_f64(n, n, nL * r, 1, ks, A, B, Pk, x->stream);
        launch_reduce_partials(x->part, ks, (long)n * n, K, l0 > 0, x->stream);
      } else {
        StridedC Kd{K, 0, n, 1, 1.0, l0 > 0};
        gemm_f64(n, n, nL * r, 1, 1, A, B, Kd, x->stream);
      }
    }
    if ((st = check_launch()) != LAS_OK) return st;
  }
  if (K && x->prec == LAS_SPLIT_BF16) launch_mirror_lower(K, n, x->stream);
  if (J) {
    launch_coulomb_packed(x->Bp, x->vc, x->X, x->npair, x->Jp, x->stream);
    launch_unpack_sym(x->Jp, n, J, x->stream);
    launch_scale(J, (long)n * n, 0.5, x->stream);   // vc carried the factor 2
  }
  return check_launch();
}

extern "C" las_status las_df_jk(las_ctx* x, const double* C, double* J, double* K) {
  if (!x || !C) return LAS_ERR_ARG;
  if (!J && !K) return LAS_OK;
  const int n = x->n, op = x->op, c = x->c;
  if (c == 0) {
    if (J) LAS_CUDA_TRY(cudaMemsetAsync(J, 0, (size_t)n * n * 8, x->stream));
    if (K) LAS_CUDA_TRY(cudaMemsetAsync(K, 0, (size_t)n * n * 8, x->stream));
    return LAS_OK;
  }
  // core-only C_occ (columns >= c zeroed): D = C_core C_core^T and Dc = 2 D
  launch_pack_cocc(C, n, x->nmo, c, op, x->Cocc, x->stream);
  las_status st = jk_raw(x, c, J, K);
  if (st != LAS_OK) return st;
  if (J) launch_scale(J, (long)n * n, 2.0, x->stream);
  if (K) launch_scale(K, (long)n * n, 2.0, x->stream);
  return check_launch();
}

extern "C" las_status las_df_jk_density(las_ctx* x, const double* Cx, const double* w, int r,
                                        double* J, double* K) {
  if (!x || r < 0 || (r > 0 && (!Cx || !w))) return LAS_ERR_ARG;   // r = 0: D = 0
  if (r > x->o) return LAS_ERR_ARG;
  if (!J && !K) return LAS_OK;
  const int n = x->n;
  if (r == 0) {
    if (J) LAS_CUDA_TRY(cudaMemsetAsync(J, 0, (size_t)n * n * 8, x->stream));
    if (K) LAS_CUDA_TRY(cudaMemsetAsync(K, 0, (size_t)n * n * 8, x->stream));
    return LAS_OK;
  }
  // D = D+ - D-,  D± = sum_k max(±w_k, 0) c_k c_k^T, each over the columns of its sign only
  // (their counts size the transforms, so they are read back once)
  int* idx_pos = x->widx;
  int* idx_neg = x->widx + x->o;
  int* counts = x->widx + 2 * x->o;
  launch_sign_split(w, r, idx_pos, idx_neg, counts, x->stream);
  LAS_CUDA_TRY(cudaMemcpyAsync(x->wcount, counts, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                               x->stream));
  LAS_CUDA_TRY(cudaStreamSynchronize(x->stream));
  const int rp = x->wcount[0], rn = x->wcount[1];
  las_status st = LAS_OK;
  if (rp > 0) {
    launch_pack_weighted(Cx, w, idx_pos, rp, +1.0, n, r, x->op, x->Cocc, x->stream);
    if ((st = jk_raw(x, rp, J, K)) != LAS_OK) return st;
  } else {
    if (J) LAS_CUDA_TRY(cudaMemsetAsync(J, 0, (size_t)n * n * 8, x->stream));
    if (K) LAS_CUDA_TRY(cudaMemsetAsync(K, 0, (size_t)n * n * 8, x->stream));
  }
  if (rn > 0) {
    launch_pack_weighted(Cx, w, idx_neg, rn, -1.0, n, r, x->op, x->Cocc, x->stream);
    if ((st = jk_raw(x, rn, J ? x->Jt : nullptr, K ? x->Kt : nullptr)) != LAS_OK) return st;
    if (J) launch_axpy(J, x->Jt, -1.0, (long)n * n, x->stream);
    if (K) launch_axpy(K, x->Kt, -1.0, (long)n * n, x->stream);
  }
  return check_launch();
}

extern "C" las_status las_df_transform(las_ctx* x, const double* C, int p0, int p1,
                                       double* Lmu_u, double* Lpu) {
  if (!x || !C) return LAS_ERR_ARG;
  if (p0 < 0 || p1 < p0 || p1 > x->nmo) return LAS_ERR_ARG;
  if (x->a == 0) return LAS_OK;
  const int n = x->n, op = x->op, c = x->c, a = x->a, np = p1 - p0;
  launch_pack_cocc(C, n, x->nmo, x->o, op, x->Cocc, x->stream);
  if (x->prec == LAS_SPLIT_BF16) {
    las_status st = split_prepare_C(x->split, x->Cocc, x->stream);
    if (st != LAS_OK) return st;
  }
  las_status st;
  for (int l0 = 0; l0 < x->X; l0 += x->Lc) {
    const int nL = std::min(x->Lc, x->X - l0);
    if ((st = half_and_full(x, l0, nL, 0)) != LAS_OK) return st;
    if (Lmu_u) launch_copy_cols(x->Ht, nL, op, n, c, a, Lmu_u + (size_t)l0 * n * a, x->stream);
    if (Lpu && np > 0 && x->prec == LAS_SPLIT_BF16) {
      if ((st = split_lpu(x->split, nL, x->Ht, c, a, C, x->nmo, p0, np,
                          Lpu + (size_t)l0 * np * a, x->stream, &x->bytes)) != LAS_OK)
        return st;
    } else if (Lpu && np > 0) {
      // Lpu[b][p][u] = sum_mu C[mu][p0+p] Ht[b][c+u][mu]
      StridedA A{C + p0, 0, 1, x->nmo};
      StridedA B{x->Ht + (size_t)c * n, (long)op * n, 1, n};
      StridedC Co{Lpu + (size_t)l0 * np * a, (long)np * a, a, 1, 1.0, 0};
      // batch over L: A is shared (sb = 0), B and C advance per L
      gemm_f64(np, a, n, nL, 1, A, B, Co, x->stream);
    }
    if ((st = check_launch()) != LAS_OK) return st;
  }
  return LAS_OK;
}

// ------------------------------------------------------------------------------------------
// Effective potentials (Eqs. v_emb, vself): v_sigma = J[gamma_a + gamma_b] - K[gamma_sigma]
// ------------------------------------------------------------------------------------------
extern "C" las_status las_veff(las_ctx* x, const double* Ca, const double* wa, int ra,
                               const double* Cb, const double* wb, int rb, double* va,
                               double* vb) {
  if (!x || !va || !vb || ra < 0 || rb < 0) return LAS_ERR_ARG;
  if ((ra > 0 && (!Ca || !wa)) || (rb > 0 && (!Cb || !wb))) return LAS_ERR_ARG;
  if (ra > x->o || rb > x->o) return LAS_ERR_ARG;
  const long nn = (long)x->n * x->n;
  if (!x->vJ) {
    las_status st = LAS_OK;
    if ((st = dalloc(x, (void**)&x->vJ, sizeof(double) * nn)) != LAS_OK ||
        (st = dalloc(x, (void**)&x->vK, sizeof(double) * nn)) != LAS_OK)
      return st;
  }
  // alpha: va = J_a, vK = K_a;  beta: vJ = J_b, vb = K_b
  las_status st = las_df_jk_density(x, Ca, wa, ra, va, x->vK);
  if (st == LAS_OK) st = las_df_jk_density(x, Cb, wb, rb, x->vJ, vb);
  if (st != LAS_OK) return st;
  launch_axpy(va, x->vJ, 1.0, nn, x->stream);      // va = J[D]
  launch_scale(vb, nn, -1.0, x->stream);
  launch_axpy(vb, va, 1.0, nn, x->stream);         // vb = J[D] - K_b
  launch_axpy(va, x->vK, -1.0, nn, x->stream);     // va = J[D] - K_a
  return check_launch();
}

// ------------------------------------------------------------------------------------------
// Orbital Hessian-vector product at fixed fragment RDMs
// ------------------------------------------------------------------------------------------
// dE/dC = [4 h C_c | 2 h C_a D | 0] + sum_L H_L W(T_L) with H_L = b^L C_occ, T_L = C_occ^T H_L
// and W linear in T (the matrix the per-aux kernel builds), so its directional derivative along
// dC is the tangent chain
//     dG = [4 h dC_c | 2 h dC_a D | 0] + sum_L ( dH_L W(T_L) + H_L W(dT_L) ),
//     dH_L = b^L dC_occ,   dT_L = X_L + X_L^T,   X_L = H_L^T dC_occ   (b^L symmetric):
// one more half transform (dH), one more full-transform product (X), two per-aux passes and two
// projections; in split precision W(T_L) is scaled by the row exponents of dH and W(dT_L) by those
// of H, the operand each is projected against.  G(C) itself (for Dg) is one plain evaluation.
static las_status tangent_grad(las_ctx* x, const double* h, const double* dm1s,
                               const double* dm2, double* dG) {
  const int n = x->n, op = x->op, nmo = x->nmo;
  const bool split = x->prec == LAS_SPLIT_BF16;
  las_status st;
  launch_pack_cocc(x->hdC, n, nmo, x->o, op, x->tCocc, x->stream);   // dC_occ
  if (split && (st = split_tangent_prepare(x->split, x->tCocc, x->stream, &x->bytes)) != LAS_OK)
    return st;
  if (split && (st = split_prepare_C(x->split, x->Cocc, x->stream)) != LAS_OK) return st;
  for (int l0 = 0; l0 < x->X; l0 += x->Lc) {
    const int nL = std::min(x->Lc, x->X - l0);
    if (split) {
      if ((st = split_half(x->split, l0, nL, op, x->Ht, x->stream)) != LAS_OK ||
          (st = split_tangent_half(x->split, l0, nL, x->tHt, x->stream)) != LAS_OK ||
          (st = split_full(x->split, nL, x->Ht, x->T, x->stream)) != LAS_OK ||
          (st = split_tangent_full(x->split, nL, x->tHt, x->tX, x->stream)) != LAS_OK)
        return st;
    } else {
      PackedSymA A{x->Bp, x->npair, l0};
      StridedA Bc{x->Cocc, 0, op, 1}, Bd{x->tCocc, 0, op, 1};
      gemm_f64(n, op, n, nL, 1, A, Bc, StridedC{x->Ht, (long)op * n, 1, n, 1.0, 0}, x->stream);
      gemm_f64(n, op, n, nL, 1, A, Bd, StridedC{x->tHt, (long)op * n, 1, n, 1.0, 0}, x->stream);
      StridedA Ah{x->Ht, (long)op * n, n, 1};
      gemm_f64(op, op, n, nL, 1, Ah, Bc, StridedC{x->T, (long)op * op, op, 1, 1.0, 0}, x->stream);
      gemm_f64(op, op, n, nL, 1, Ah, Bd, StridedC{x->tX, (long)op * op, op, 1, 1.0, 0},
               x->stream);
    }
    launch_sym_add(x->tX, nL, op, x->tdT, x->stream);
    // W(T) against dH and W(dT) against H (the per-aux outputs eps, vc, va are not needed)
    const int* hexp = split ? split_hexp(x->split) : nullptr;
    const int* dhexp = split ? split_tangent_dhexp(x->split) : nullptr;
    launch_per_aux(x->T, nL, op, dm1s, dm2, x->fi, x->tWd, x->eps + l0, x->vc + l0, x->va + l0, 1,
                   dhexp, x->status, x->stream);
    launch_per_aux(x->tdT, nL, op, dm1s, dm2, x->fi, x->tdW, x->eps + l0, x->vc + l0, x->va + l0,
                   1, hexp, x->status, x->stream);
    if ((st = check_launch()) != LAS_OK) return st;
    if (split) {
      if ((st = split_tangent_project(x->split, nL, 0, x->tdW, x->tOut, l0 > 0, x->stream)) !=
              LAS_OK ||
          (st = split_tangent_project(x->split, nL, 1, x->tWd, x->tOut, 1, x->stream)) != LAS_OK)
        return st;
    } else {
      const int ks = std::max(1, std::min(x->ksplit, (nL * op) / 64));
      const double* Hs[2] = {x->Ht, x->tHt};
      const double* Ws[2] = {x->tdW, x->tWd};
      for (int k = 0; k < 2; ++k) {
        StridedA A{Hs[k], 0, 1, n};
        StridedA Bw{Ws[k], 0, op, 1};
        StridedC Cp{x->part, (long)n * op, op, 1, 1.0, 0};
        gemm_f64(n, op, nL * op, 1, ks, A, Bw, Cp, x->stream);
        launch_reduce_partials(x->part, ks, (long)n * op, x->tOut, l0 > 0 || k > 0, x->stream);
      }
    }
    if ((st = check_launch()) != LAS_OK) return st;
  }
  // h dC_occ
  if (split) {
    if ((st = split_one_electron_hc(x->split, h, x->hC, x->stream)) != LAS_OK ||
        (st = split_tangent_one_electron(x->split, x->thC, x->stream)) != LAS_OK)
      return st;
  } else {
    gemm_f64(n, op, n, 1, 1, StridedA{h, 0, n, 1}, StridedA{x->tCocc, 0, op, 1},
             StridedC{x->thC, 0, op, 1, 1.0, 0}, x->stream);
  }
  launch_assemble_grad(x->tOut, x->thC, dm1s, x->fi, n, nmo, op, dG, x->stream);
  return check_launch();
}

extern "C" las_status las_orbital_hvp(las_ctx* x, const double* C, const double* h,
                                      const double* dm1s, const double* dm2, const double* X,
                                      double* dG, double* Dg) {
  if (!x || !C || !h || !X || !dG) return LAS_ERR_ARG;
  if (x->a > 0 && (!dm1s || !dm2)) return LAS_ERR_ARG;
  const int n = x->n, nmo = x->nmo, op = x->op;
  const long nC = (long)n * nmo;
  const size_t chunk = (size_t)x->Lc * op;
  las_status st = LAS_OK;
  if (!x->hdC) {
    const struct { double** p; size_t cnt; } bufs[] = {
        {&x->hdC, (size_t)nC}, {&x->hG, (size_t)nC}, {&x->tCocc, (size_t)n * op},
        {&x->thC, (size_t)n * op}, {&x->tOut, (size_t)n * op}, {&x->tHt, chunk * n},
        {&x->tX, chunk * op}, {&x->tdT, chunk * op}, {&x->tdW, chunk * op},
        {&x->tWd, chunk * op}};
    for (const auto& b : bufs)
      if ((st = dalloc(x, (void**)b.p, sizeof(double) * b.cnt)) != LAS_OK) return st;
  }
  // dC = C X
  gemm_f64(n, nmo, nmo, 1, 1, StridedA{C, 0, nmo, 1}, StridedA{X, 0, nmo, 1},
           StridedC{x->hdC, 0, nmo, 1, 1.0, 0}, x->stream);
  // G(C): C_occ, its digits and those of h stay in place for the tangent chain
  if ((st = evaluate(x, C, h, dm1s, dm2, x->dE, x->hG, nullptr)) != LAS_OK) return st;
  if ((st = tangent_grad(x, h, dm1s, dm2, dG)) != LAS_OK) return st;
  if (Dg) {
    // Dg = (C X)^T G + C^T dG - transpose  (virtual columns of G and dG are zero)
    StridedA Ad{x->hdC, 0, 1, nmo};
    StridedA Bg{x->hG, 0, nmo, 1};
    StridedC Cm{x->M, 0, x->op, 1, 1.0, 0};
    gemm_f64(nmo, x->o, n, 1, 1, Ad, Bg, Cm, x->stream);
    StridedA Acc{C, 0, 1, nmo};
    StridedA Bdg{dG, 0, nmo, 1};
    StridedC Cm2{x->M, 0, x->op, 1, 1.0, 1};
    gemm_f64(nmo, x->o, n, 1, 1, Acc, Bdg, Cm2, x->stream);
    launch_antisym(x->M, nmo, x->o, x->op, Dg, x->stream);
  }
  return check_launch();
}

// ------------------------------------------------------------------------------------------
// Fragment-embedding AO2MO (Eqs. ao2mo_1, ao2mo_2, ppaa, papa)
// ------------------------------------------------------------------------------------------
// Operand loaders of the two integral products over the chunk's T[L][p][q] (nmo x nmo per L)
struct ActBlockB {   // (b, k = L, c = (u, v)) -> T[L][a0+u][a0+v]
  const double* T;
  long n2;
  int nmo, a0, ma;
  __device__ __forceinline__ double operator()(int, int k, int c) const {
    const int u = c / ma, v = c - u * ma;
    return T[(long)k * n2 + (long)(a0 + u) * nmo + a0 + v];
  }
};
struct PActA {       // (b, r = (p, u), k = L) -> T[L][p][a0+u]
  const double* T;
  long n2;
  int nmo, a0, ma;
  __device__ __forceinline__ double operator()(int, int r, int k) const {
    const int p = r / ma, u = r - p * ma;
    return T[(long)k * n2 + (long)p * nmo + a0 + u];
  }
};
struct PActB {       // (b, k = L, c = (q, v)) -> T[L][q][a0+v]
  PActA a;
  __device__ __forceinline__ double operator()(int b, int k, int c) const { return a(b, c, k); }
};

// Workspace of the fragment AO2MO: H [Lc][nmo][n] and T [Lc][nmo][nmo] per chunk of Lc
// auxiliary rows, split-K partials of the two products, and (split mode) the digit planes.
static las_status frag_workspace(las_ctx* x, int ma) {
  const int n = x->n, nmo = x->nmo;
  const long n2 = (long)nmo * nmo, m = (long)nmo * ma;
  const long part = 8 * std::max(n2 * ma * ma, m * m);   // up to 8 K splits
  const size_t per_aux = (size_t)8 * ((size_t)nmo * n + n2) +
                         (x->prec == LAS_SPLIT_BF16 ? (size_t)12 * ((size_t)nmo * n + n2 + m) : 0);
  const size_t fixed = (size_t)8 * part + (size_t)12 * nmo * n;
  int Lc = x->X;
  while (Lc > 1 && fixed + per_aux * Lc > x->ws_cap) Lc = (Lc + 1) / 2;
  if (fixed + per_aux * Lc > x->ws_cap) return LAS_ERR_WORKSPACE;
  const bool fits = x->fH && x->fnmo == nmo && x->fma >= ma && x->fLc >= Lc &&
                    x->fpart_elems >= part &&
                    (x->prec != LAS_SPLIT_BF16 || frag_split_fits(x->fsplit, n, nmo, ma, Lc));
  if (fits) return LAS_OK;
  LAS_CUDA_TRY(cudaStreamSynchronize(x->stream));
  for (double** q : {&x->fH, &x->fT, &x->fpart}) {
    if (*q) cudaFree(*q);
    *q = nullptr;
  }
  if (x->fsplit) frag_split_destroy(x->fsplit);
  x->fsplit = nullptr;
  x->bytes -= x->fbytes;
  x->fbytes = 0;
  x->fLc = 0;
  const size_t bytes0 = x->bytes;
  las_status st = LAS_OK;
  if ((st = dalloc(x, (void**)&x->fH, sizeof(double) * (size_t)Lc * nmo * n)) == LAS_OK &&
      (st = dalloc(x, (void**)&x->fT, sizeof(double) * (size_t)Lc * n2)) == LAS_OK &&
      (st = dalloc(x, (void**)&x->fpart, sizeof(double) * (size_t)part)) == LAS_OK &&
      x->prec == LAS_SPLIT_BF16)
    st = frag_split_create(&x->fsplit, n, nmo, ma, Lc, x->stream, &x->bytes);
  x->fbytes = x->bytes - bytes0;   // also what a failed attempt left allocated
  if (st != LAS_OK) return st;
  x->fLc = Lc;
  x->fnmo = nmo;
  x->fma = ma;
  x->fpart_elems = part;
  return LAS_OK;
}

extern "C" las_status las_frag_ao2mo(las_ctx* x, const double* M, int a0, int ma, double* ppaa,
                                     double* papa) {
  if (!x || !M) return LAS_ERR_ARG;
  if (ma < 1 || a0 < 0 || a0 + ma > x->nmo) return LAS_ERR_ARG;
  if (!ppaa && !papa) return LAS_OK;
  las_status st = frag_workspace(x, ma);
  if (st != LAS_OK) return st;
  const int n = x->n, nmo = x->nmo;
  const long n2 = (long)nmo * nmo, m = (long)nmo * ma;
  const bool split = x->prec == LAS_SPLIT_BF16;
  if (split && (st = frag_split_prepare_M(x->fsplit, M, x->stream)) != LAS_OK) return st;
  for (int l0 = 0; l0 < x->X; l0 += (int)x->fLc) {
    const int nL = (int)std::min<long>(x->fLc, x->X - l0);
    if (split) {
      st = frag_split_chunk(x->split, x->fsplit, l0, nL, x->fH, x->fT, a0, ma, ppaa, papa,
                            x->fpart, x->fpart_elems, l0 > 0, x->stream);
      if (st != LAS_OK) return st;
    } else {
      // Eq. ao2mo_1: H[L][p][e2] = sum_e1 b^L(e2, e1) M[e1][p]
      PackedSymA A{x->Bp, x->npair, l0};
      StridedA Bm{M, 0, nmo, 1};
      StridedC Ch{x->fH, (long)nmo * n, 1, n, 1.0, 0};
      gemm_f64(n, nmo, n, nL, 1, A, Bm, Ch, x->stream);
      // Eq. ao2mo_2: T[L][p][q] = sum_e H[L][p][e] M[e][q]
      StridedA Ah{x->fH, (long)nmo * n, n, 1};
      StridedC Ct{x->fT, n2, nmo, 1, 1.0, 0};
      gemm_f64(nmo, nmo, n, nL, 1, Ah, Bm, Ct, x->stream);
      if (ppaa) {
        // Eq. ppaa: ppaa[(p,q)][(u,v)] (+)= sum_L T[L][(p,q)] T[L][a0+u][a0+v]
        const long out = n2 * ma * ma;
        const int tiles = (int)(((n2 + 63) / 64) * ((ma * ma + 63) / 64));
        const int ks = (int)std::max(1L, std::min({8L, (2L * 152 + tiles - 1) / tiles,
                                                   (long)nL / 64, x->fpart_elems / out}));
        StridedA At{x->fT, 0, 1, n2};
        ActBlockB Bt{x->fT, n2, nmo, a0, ma};
        StridedC Cp{x->fpart, out, (long)ma * ma, 1, 1.0, 0};
        gemm_f64((int)n2, ma * ma, nL, 1, ks, At, Bt, Cp, x->stream);
        launch_reduce_partials(x->fpart, ks, out, ppaa, l0 > 0, x->stream);
      }
      if (papa) {
        // Eq. papa: papa[(p,u)][(q,v)] (+)= sum_L T[L][p][a0+u] T[L][q][a0+v]
        const long out = m * m;
        const int tiles = (int)(((m + 63) / 64) * ((m + 63) / 64));
        const int ks = (int)std::max(1L, std::min({8L, (2L * 152 + tiles - 1) / tiles,
                                                   (long)nL / 64, x->fpart_elems / out}));
        PActA Ap{x->fT, n2, nmo, a0, ma};
        PActB Bp2{Ap};
        StridedC Cp{x->fpart, out, m, 1, 1.0, 0};
        gemm_f64((int)m, (int)m, nL, 1, ks, Ap, Bp2, Cp, x->stream);
        launch_reduce_partials(x->fpart, ks, out, papa, l0 > 0, x->stream);
      }
    }
    if ((st = check_launch()) != LAS_OK) return st;
  }
  if (split && papa) launch_mirror_lower(papa, (int)m, x->stream);
  return check_launch();
}

// ------------------------------------------------------------------------------------------
// Batched evaluation under one captured CUDA graph
// ------------------------------------------------------------------------------------------
static bool same_items(const las_batch_item& a, const las_batch_item& b) {
  return a.C == b.C && a.h == b.h && a.dm1s == b.dm1s && a.dm2 == b.dm2 && a.E == b.E &&
         a.dEdC == b.dEdC;
}

// The batch in split precision as phases: each phase runs every problem's small kernels (digit
// slicing, per-aux contractions, reductions) on the branch streams, and the split products those
// kernels feed are recorded instead of launched; after the phase's join, all of them run as ONE
// persistent grouped launch (tiles in the order the problems are visited: largest first), then
// the next phase forks again.  Per auxiliary chunk c of each problem:
//   A: [c = 0: C_occ and h digits]      products: S1 of chunk c (+ h C_occ at c = 0)
//   B: digits of H                      products: S2 of chunk c (+ C_occ^T h C_occ at c = 0)
//   C: per-aux contractions, W digits   products: projection of chunk c
//   D: ordered sum of the projection's partials (run with the next round's A)
// then the energy and gradient assembly.  Problems with fewer chunks drop out of later rounds.
struct BatchPlan {
  int nsys, nb;
  const std::vector<int>* order;    // problems, largest first
  const std::vector<int>* branch;   // branch stream of each problem
  cudaStream_t cs;                  // the capture stream
  cudaStream_t* br;                 // [nb] branch streams
  cudaEvent_t fork_ev;
  cudaEvent_t* join_ev;             // [nb]
};

static las_status plan_fork(const BatchPlan& P) {
  cudaError_t e = cudaEventRecord(P.fork_ev, P.cs);
  for (int b = 0; b < P.nb && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(P.br[b], P.fork_ev, 0);
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "graph fork", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  return LAS_OK;
}

static las_status plan_join(const BatchPlan& P) {
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < P.nb && e == cudaSuccess; ++b) {
    e = cudaEventRecord(P.join_ev[b], P.br[b]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.cs, P.join_ev[b], 0);
  }
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "graph join", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  return LAS_OK;
}

static int batch_rounds(int nsys, las_ctx* const* ctxs) {
  int rounds = 0;
  for (int i = 0; i < nsys; ++i)
    rounds = std::max(rounds, (ctxs[i]->X + ctxs[i]->Lc - 1) / ctxs[i]->Lc);
  return rounds;
}

// Device bytes reserved per grouped launch: at most three products per problem (the half
// transform's two -- full row blocks of the packed triangle and ragged rows -- and h C_occ).
constexpr int kMaxGroupedPerProblem = 3;
static size_t batch_slot_bytes(int nsys) {
  return (ozgroup_bytes(kMaxGroupedPerProblem * (size_t)nsys) + 255) / 256 * 256;
}

static las_status capture_grouped(const BatchPlan& P, las_ctx* const* ctxs,
                                  const las_batch_item* items, void* dev,
                                  std::vector<OzGroup*>* groups) {
  const int nsys = P.nsys;
  const int rounds = batch_rounds(nsys, ctxs);
  const size_t slot = batch_slot_bytes(nsys);
  std::vector<int> ks(nsys, 1);
  // run `fn(i, x)` for every problem on its branch (products recorded into a new group when
  // `record`), join, run the group as one launch, fork again
  auto phase = [&](auto fn, bool record) -> las_status {
    OzGroup* g = nullptr;
    if (record) {
      g = ozgroup_new();
      groups->push_back(g);
      ozgroup_record(g);
    }
    las_status r = LAS_OK;
    for (int k = 0; k < nsys && r == LAS_OK; ++k) {
      const int i = (*P.order)[k];
      las_ctx* x = ctxs[i];
      cudaStream_t saved = x->stream;
      x->stream = P.br[(*P.branch)[i]];
      r = fn(i, x);
      x->stream = saved;
    }
    if (record) ozgroup_record(nullptr);
    if (r != LAS_OK) return r;
    if ((r = plan_join(P)) != LAS_OK) return r;
    if (record && ozgroup_bytes(ozgroup_count(g)) > slot) return LAS_ERR_INTERNAL;
    if (record && (r = ozgroup_launch(g, (uint8_t*)dev + (groups->size() - 1) * slot, P.cs)) !=
                      LAS_OK)
      return r;
    return plan_fork(P);
  };
  auto nchunks = [](las_ctx* x) { return (x->X + x->Lc - 1) / x->Lc; };
  las_status rc = plan_fork(P);
  for (int c = 0; c < rounds && rc == LAS_OK; ++c) {
    // A: the previous chunk's partial sums; at c = 0 the C_occ and h digits and h C_occ;
    //    S1 of chunk c
    rc = phase([&](int i, las_ctx* x) -> las_status {
      if (c > 0 && c - 1 < nchunks(x))
        split_project_reduce(x->split, ks[i], x->Out, c - 1 > 0, x->stream);
      if (c >= nchunks(x)) return LAS_OK;
      las_status r = LAS_OK;
      if (c == 0) {
        launch_pack_cocc(items[i].C, x->n, x->nmo, x->o, x->op, x->Cocc, x->stream);
        if ((r = split_prepare_C(x->split, x->Cocc, x->stream)) != LAS_OK) return r;
        if ((r = split_one_electron_hc(x->split, items[i].h, x->hC, x->stream)) != LAS_OK)
          return r;
      }
      const int l0 = c * x->Lc, nL = std::min(x->Lc, x->X - l0);
      return split_half(x->split, l0, nL, x->op, x->Ht, x->stream);
    }, true);
    if (rc != LAS_OK) break;
    // B: digits of H; S2 of chunk c (and C_occ^T h C_occ at c = 0)
    rc = phase([&](int i, las_ctx* x) -> las_status {
      if (c >= nchunks(x)) return LAS_OK;
      const int nL = std::min(x->Lc, x->X - c * x->Lc);
      las_status r = split_full(x->split, nL, x->Ht, x->T, x->stream);
      if (r == LAS_OK && c == 0) r = split_one_electron_hmo(x->split, x->hC, x->hmo, x->stream);
      return r;
    }, true);
    if (rc != LAS_OK) break;
    // C: per-aux contractions and W digits; projection of chunk c
    rc = phase([&](int i, las_ctx* x) -> las_status {
      if (c >= nchunks(x)) return LAS_OK;
      const int l0 = c * x->Lc, nL = std::min(x->Lc, x->X - l0);
      launch_per_aux(x->T, nL, x->op, items[i].dm1s, items[i].dm2, x->fi, x->W, x->eps + l0,
                     x->vc + l0, x->va + l0, 1, split_hexp(x->split), x->status, x->stream);
      las_status r = check_launch();
      if (r == LAS_OK) r = split_project_gemm(x->split, nL, x->W, &ks[i], x->stream);
      return r;
    }, true);
  }
  // the last chunk's partial sums, then energy and gradient assembly
  if (rc == LAS_OK)
    rc = phase([&](int i, las_ctx* x) -> las_status {
      const int last = nchunks(x) - 1;
      split_project_reduce(x->split, ks[i], x->Out, last > 0, x->stream);
      launch_energy_final(x->eps, x->X, x->hmo, x->op, items[i].dm1s, x->fi, items[i].E,
                          x->stream);
      launch_assemble_grad(x->Out, x->hC, items[i].dm1s, x->fi, x->n, x->nmo, x->op,
                           items[i].dEdC, x->stream);
      return check_launch();
    }, false);
  return rc;
}

extern "C" las_status las_energy_grad_batched(int nsys, las_ctx* const* ctxs,
                                              const las_batch_item* items, void* stream) {
  if (nsys < 0 || (nsys > 0 && (!ctxs || !items))) return LAS_ERR_ARG;
  if (nsys == 0) return LAS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < nsys; ++i) {
    if (!ctxs[i] || !items[i].C || !items[i].h || !items[i].E || !items[i].dEdC) return LAS_ERR_ARG;
    if (ctxs[i]->a > 0 && (!items[i].dm1s || !items[i].dm2)) return LAS_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return LAS_ERR_ARG;   // a context's workspace serves one item
  }
  std::lock_guard<std::mutex> lock(g_graph_mu);
  for (GraphEntry& g : g_graphs) {
    if (g.stream != st || (int)g.ctxs.size() != nsys) continue;
    bool match = true;
    for (int i = 0; i < nsys && match; ++i)
      match = g.ctxs[i] == ctxs[i] && same_items(g.items[i], items[i]);
    if (match) {
      LAS_CUDA_TRY(cudaGraphLaunch(g.exec, st));
      return LAS_OK;
    }
  }
  // capture on private streams (the caller's stream may be the legacy default stream, which
  // cannot be captured): forks into LAS_BRANCHES branch streams and joins, so that the small
  // kernels of different systems overlap on the GPU; systems are shared out largest first to
  // the branch with the least work so far; the graph is then launched on `st`.
  // Split precision: the phases of capture_grouped, each product kind of all systems as one
  // persistent grouped launch.  Otherwise (native FP64): each system's whole chain on its branch.
  constexpr int LAS_BRANCHES = 8;
  static cudaStream_t cap_stream[64], br_stream[64][LAS_BRANCHES];
  static cudaEvent_t fork_ev[64], join_ev[64][LAS_BRANCHES];
  int dev = 0;
  LAS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return LAS_ERR_UNSUPPORTED;
  if (!cap_stream[dev]) {
    LAS_CUDA_TRY(cudaStreamCreateWithFlags(&cap_stream[dev], cudaStreamNonBlocking));
    LAS_CUDA_TRY(cudaEventCreateWithFlags(&fork_ev[dev], cudaEventDisableTiming));
    for (int b = 0; b < LAS_BRANCHES; ++b) {
      LAS_CUDA_TRY(cudaStreamCreateWithFlags(&br_stream[dev][b], cudaStreamNonBlocking));
      LAS_CUDA_TRY(cudaEventCreateWithFlags(&join_ev[dev][b], cudaEventDisableTiming));
    }
  }
  cudaStream_t cs = cap_stream[dev];
  std::vector<int> order(nsys), branch(nsys);
  for (int i = 0; i < nsys; ++i) order[i] = i;
  auto cost = [&](int i) {   // the half transform's work: X n^2 op
    return (double)ctxs[i]->X * ctxs[i]->n * ctxs[i]->n * ctxs[i]->op;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  const int nb = std::min(nsys, LAS_BRANCHES);
  {
    double load[LAS_BRANCHES] = {0};
    for (int i : order) {
      int b = 0;
      for (int k = 1; k < nb; ++k)
        if (load[k] < load[b]) b = k;
      branch[i] = b;
      load[b] += cost(i);
    }
  }
  bool grouped = true;
  for (int i = 0; i < nsys; ++i) grouped &= (ctxs[i]->prec == LAS_SPLIT_BF16);
  void* probs = nullptr;   // device descriptions of the grouped products
  if (grouped)
    LAS_CUDA_TRY(cudaMalloc(&probs, 3 * (size_t)batch_rounds(nsys, ctxs) * batch_slot_bytes(nsys)));
  BatchPlan P{nsys, nb, &order, &branch, cs, br_stream[dev], fork_ev[dev], join_ev[dev]};
  std::vector<OzGroup*> groups;
  cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) {
    if (probs) cudaFree(probs);
    las_record_cuda_error(ce, "cudaStreamBeginCapture", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  las_status rc = LAS_OK;
  if (grouped) {
    rc = capture_grouped(P, ctxs, items, probs, &groups);
  } else {
    rc = plan_fork(P);
    for (int k = 0; k < nsys && rc == LAS_OK; ++k) {
      const int i = order[k];
      las_ctx* x = ctxs[i];
      cudaStream_t saved = x->stream;
      const int timing = x->timing;
      x->stream = br_stream[dev][branch[i]];
      x->timing = 0;
      rc = evaluate(x, items[i].C, items[i].h, items[i].dm1s, items[i].dm2, items[i].E,
                    items[i].dEdC, nullptr);
      x->stream = saved;
      x->timing = timing;
    }
    if (rc == LAS_OK) rc = plan_join(P);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  // the grouped launches read their product descriptions from `probs`: write them now
  const size_t slot = batch_slot_bytes(nsys);
  for (size_t gi = 0; gi < groups.size() && rc == LAS_OK && e == cudaSuccess; ++gi)
    rc = ozgroup_upload(groups[gi], (uint8_t*)probs + gi * slot);
  for (OzGroup* g : groups) ozgroup_free(g);
  if (rc != LAS_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (probs) cudaFree(probs);
    if (rc != LAS_OK) return rc;
    las_record_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    if (probs) cudaFree(probs);
    las_record_cuda_error(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  GraphEntry g;
  g.ctxs.assign(ctxs, ctxs + nsys);
  g.items.assign(items, items + nsys);
  g.stream = st;
  g.exec = exec;
  g.probs = probs;
  g_graphs.push_back(g);
  LAS_CUDA_TRY(cudaGraphLaunch(exec, st));
  return LAS_OK;
}

// ------------------------------------------------------------------------------------------
// Autotuner: tile widths of the split products and the split-K factor of the projection, chosen
// by timing whole evaluations
// ------------------------------------------------------------------------------------------
extern "C" las_status las_autotune(las_ctx* x, const double* C, const double* h,
                                   const double* dm1s, const double* dm2, double* E,
                                   double* dEdC) {
  if (!x || !C || !h || !E || !dEdC) return LAS_ERR_ARG;
  if (x->prec != LAS_SPLIT_BF16) return LAS_OK;   // the FP64 path is bound by FP64 arithmetic
  las_status st = las_set_timing(x, 1);
  if (st != LAS_OK) return st;
  // stage times of one evaluation with the current settings (the second of two runs)
  auto timed = [&](float* ms) -> las_status {
    las_status r = LAS_OK;
    for (int k = 0; k < 2 && r == LAS_OK; ++k) {
      r = evaluate(x, C, h, dm1s, dm2, E, dEdC, nullptr);
      if (r == LAS_OK && k == 0) {
        float d[8];
        las_stage_times(x, d, 8);
      }
    }
    if (r == LAS_OK && las_stage_times(x, ms, 8) < 5) r = LAS_ERR_INTERNAL;
    return r;
  };
  // tile width of each product kind, judged by the stage that holds it: [0] S1, [1] S2 and the
  // H slicer, [3] the projection, [4] the one-electron products, energy and assembly
  const int stage_of[SPLIT_NKIND] = {0, 1, 3, 4};
  const int widths[] = {96, 64};
  for (int kind = 0; kind < SPLIT_NKIND && st == LAS_OK; ++kind) {
    int best = split_get_tile(x->split, kind);
    float best_ms = 1e30f;
    for (int bn : widths) {
      if ((st = split_set_tile(x->split, kind, bn)) != LAS_OK) break;
      float ms[8] = {0};
      if ((st = timed(ms)) != LAS_OK) break;
      if (ms[stage_of[kind]] < best_ms) {
        best_ms = ms[stage_of[kind]];
        best = bn;
      }
    }
    if (st == LAS_OK) st = split_set_tile(x->split, kind, best);
  }
  // split-K factor of the projection: powers-of-two-ish ladder plus the factor that balances its
  // tiles over the SMs
  if (st == LAS_OK) {
    const int cands[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64,
                         split_balanced_ksplit(x->split, x->Lc)};
    int best = split_get_ksplit(x->split);
    float best_ms = 1e30f;
    for (int ks : cands) {
      split_set_ksplit(x->split, ks);
      float ms[8] = {0};
      if ((st = timed(ms)) != LAS_OK) break;
      if (ms[3] < best_ms) {
        best_ms = ms[3];
        best = ks;
      }
    }
    split_set_ksplit(x->split, best);
  }
  las_set_timing(x, 0);
  if (st != LAS_OK) return st;
  return las_sync(x);
}

// Tile widths chosen for a split context (or set by hand): product kinds S1, S2, projection,
// one-electron.
extern "C" las_status las_get_tiles(const las_ctx* x, int* bn4) {
  if (!x || !bn4) return LAS_ERR_ARG;
  if (x->prec != LAS_SPLIT_BF16) return LAS_ERR_UNSUPPORTED;
  for (int k = 0; k < SPLIT_NKIND; ++k) bn4[k] = split_get_tile(x->split, k);
  return LAS_OK;
}

extern "C" las_status las_set_tiles(las_ctx* x, const int* bn4) {
  if (!x || !bn4) return LAS_ERR_ARG;
  if (x->prec != LAS_SPLIT_BF16) return LAS_ERR_UNSUPPORTED;
  for (int k = 0; k < SPLIT_NKIND; ++k)
    if (bn4[k] != 64 && bn4[k] != 96) return LAS_ERR_ARG;
  for (int k = 0; k < SPLIT_NKIND; ++k) {
    las_status st = split_set_tile(x->split, k, bn4[k]);
    if (st != LAS_OK) return st;
  }
  return LAS_OK;
}
