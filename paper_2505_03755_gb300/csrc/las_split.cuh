// Split-precision (BF16 digit) path: emulated-FP64 GEMMs on tcgen05 tensor cores.
#pragma once
#include "las_common.cuh"

struct SplitState;

// Builds the one-time digit planes of the packed Cholesky vectors: full rows (L, mu) with one
// exponent per row (packed = 0), or the packed-triangle tiles with one exponent per auxiliary
// index (packed = 1, about 0.55 of the bytes).  Device errors (timeouts of bounded waits) are
// recorded in *status.
las_status split_create(SplitState** s, int n, int X, int op, int Lc, const double* Bp,
                        int packed, int* status, cudaStream_t st, size_t* bytes);
// Device bytes per auxiliary index of the per-evaluation digit workspace.
size_t split_bytes_per_aux(int n, int op);
// Row exponents of the current chunk's half-transformed rows (L, p): the per-aux kernel scales
// the projection matrix by 2^exp so that the exponents can be moved out of the left operand.
const int* split_hexp(SplitState* s);
void split_destroy(SplitState* s);
las_status split_prepare_C(SplitState* s, const double* Cocc, cudaStream_t st);
// S1: Ht[b][p][mu] = sum_nu b^{l0+b}(mu,nu) C_occ(nu,p)   (b < nL)
// H for aux rows l0..l0+nL of the first oc columns of C_occ, Ht layout [nL][oc][n]
las_status split_half(SplitState* s, int l0, int nL, int oc, double* Ht, cudaStream_t st);
// S2: T[b] = Ht[b] C_occ   (op x op per b)
las_status split_full(SplitState* s, int nL, const double* Ht, double* T, cudaStream_t st);
// K (+)= sum_{(L,p)} H(mu,(L,p)) H(nu,(L,p)) over the chunk's half transform Ht[(L,p)][mu];
// only the lower triangle (mu >= nu) is valid: mirror it afterwards
las_status split_exchange(SplitState* s, int nL, int oc, const double* Ht, double* K, int accumulate,
                          cudaStream_t st);
// Product kinds of an evaluation, each with its own tile width (64 or 96 columns; default 96):
// S1, S2 (with its H slicer), the projection and the two one-electron products.
enum { SPLIT_HALF = 0, SPLIT_FULL = 1, SPLIT_PROJECT = 2, SPLIT_ONE_ELECTRON = 3, SPLIT_NKIND = 4 };
int split_get_tile(SplitState* s, int kind);
las_status split_set_tile(SplitState* s, int kind, int bn);
// split-K factor of the projection GEMM (1..64)
int split_get_ksplit(SplitState* s);
// split-K of the projection that shares its tiles out most evenly over the SMs for nL aux rows
int split_balanced_ksplit(SplitState* s, int nL);
void split_set_ksplit(SplitState* s, int ks);
// hC = h C_occ and hmo = C_occ^T hC (split_prepare_C must have run for this C)
las_status split_one_electron(SplitState* s, const double* h, double* hC, double* hmo,
                              cudaStream_t st);
// Out (+)= sum_{(L,p)} H(mu,(L,p)) W((L,p),q) with Wt[q][(L,p)] = W_L(p,q) * 2^exp(L,p)
las_status split_project(SplitState* s, int nL, const double* Wt, double* Out, int accumulate,
                         cudaStream_t st);
// The same in two steps: digits of W and the split-K product into the partial buffer (ks_used
// receives the K split), then the ordered sum of the partials into Out.
las_status split_project_gemm(SplitState* s, int nL, const double* Wt, int* ks_used,
                              cudaStream_t st);
void split_project_reduce(SplitState* s, int ks, double* Out, int accumulate, cudaStream_t st);
// hC = h C_occ, then hmo = C_occ^T hC (split_one_electron = both)
las_status split_one_electron_hc(SplitState* s, const double* h, double* hC, cudaStream_t st);
las_status split_one_electron_hmo(SplitState* s, const double* hC, double* hmo,
                                  cudaStream_t st);

// Grouped launches: while a group is being recorded on the calling host thread, every split
// product of the functions above is appended to it instead of being launched; ozgroup_launch then
// runs all of them as one persistent launch whose CTAs walk the products' tiles in recording
// order.  The product descriptions live in device memory `dev` (at least ozgroup_bytes(count)
// bytes, 128-byte aligned), written by ozgroup_upload before the launch executes (the launch
// itself may be captured into a CUDA graph first).
struct OzGroup;
OzGroup* ozgroup_new();
void ozgroup_free(OzGroup* g);
void ozgroup_record(OzGroup* g);   // nullptr: launch products again
size_t ozgroup_count(const OzGroup* g);
size_t ozgroup_bytes(size_t nprob);
las_status ozgroup_launch(const OzGroup* g, void* dev, cudaStream_t st);
las_status ozgroup_upload(const OzGroup* g, void* dev);

// Fragment-embedding AO2MO (Eqs. ao2mo_1, ao2mo_2, ppaa, papa) in split precision: digit planes
// of M, of the chunk's half transform and of the slices of T that feed the two integral products.
struct FragSplit;
las_status frag_split_create(FragSplit** f, int n, int nmo, int ma, int Lc, cudaStream_t st,
                             size_t* bytes);
void frag_split_destroy(FragSplit* f);
int frag_split_fits(const FragSplit* f, int n, int nmo, int ma, int Lc);
las_status frag_split_prepare_M(FragSplit* f, const double* M, cudaStream_t st);
// One chunk of auxiliary rows [l0, l0+nL): H [nL][nmo][n] and T [nL][nmo][nmo] are FP64
// scratch; ppaa and papa are written (accumulate = 0) or accumulated; papa holds only its lower
// triangle (as an (nmo*ma)^2 matrix) until the caller mirrors it.
las_status frag_split_chunk(SplitState* s, FragSplit* f, int l0, int nL, double* H, double* T,
                            int a0, int ma, double* ppaa, double* papa, double* part,
                            long part_elems, int accumulate, cudaStream_t st);

// (L|pu) of las_df_transform for a chunk: Lpu[L][p][u] = sum_mu C[mu][p0+p] Ht[L][c+u][mu]
// (C: [n][nmo]; Lpu points at the chunk's first row).  The digit planes of C^T are allocated on
// the first call and their size is added to *bytes.
las_status split_lpu(SplitState* s, int nL, const double* Ht, int c, int a, const double* C,
                     int nmo, int p0, int np, double* Lpu, cudaStream_t st, size_t* bytes);

// Tangent of the evaluation along dC (orbital Hessian-vector product), split precision.
// split_tangent_prepare slices dC_occ (and allocates the tangent scratch on its first call,
// adding its size to *bytes); per chunk: split_tangent_half (dH = b dC_occ), then, after
// split_full of H, split_tangent_full (X = H^T dC and the digits of dH), and
// split_tangent_project for each of the two projection terms; split_tangent_one_electron gives
// h dC_occ (after split_one_electron of the same h).
las_status split_tangent_prepare(SplitState* s, const double* dCocc, cudaStream_t st,
                                 size_t* bytes);
las_status split_tangent_half(SplitState* s, int l0, int nL, double* dHt, cudaStream_t st);
las_status split_tangent_full(SplitState* s, int nL, const double* dHt, double* X,
                              cudaStream_t st);
const int* split_tangent_dhexp(SplitState* s);
las_status split_tangent_project(SplitState* s, int nL, int which, const double* Wt, double* Out,
                                 int accumulate, cudaStream_t st);
las_status split_tangent_one_electron(SplitState* s, double* hdC, cudaStream_t st);
