/*
 * las.h -- C ABI of the GB300 (sm_103a) library for the density-fitted LAS energy and its
 * orbital gradient.
 *
 * Problem statement followed (arXiv 2505.03755):
 *   - Cholesky / density-fitting factorisation of the two-electron integrals, Eq. cholesky:
 *       g^{mu1 mu3}_{mu2 mu4} = b^P_{mu1 mu2} b^P_{mu3 mu4};
 *     the vectors b^P are stored as packed lower triangles, Naux * Nao(Nao+1)/2 values
 *     (section "Calculation of effective potentials").
 *   - JK call, Eqs. J_1, J_2, K_1, K_2 (Coulomb and exchange matrices of a density).
 *   - AO2MO, Eqs. ao2mo_1, ao2mo_2, ppaa, papa (half and full transforms of b^P and the
 *     (pp|aa)- and (pa|pa)-type integrals).
 *   - Effective embedding and self potentials, Eqs. v_emb and vself.
 *   - LAS wave function, Eq. las_wfn (fragment CAS states times a closed-shell core), its
 *     energy E_LAS = <LAS|H|LAS>, the orbital gradient whose vanishing is Eq. MO_conv, and
 *     the orbital part of the second-order step of Eq. flas (Hessian-vector products).
 *
 * Conventions for every call:
 *   - All arrays are FP64, row-major (C order), and all pointers are DEVICE pointers unless a
 *     parameter says "host".  The caller owns every input and output buffer.
 *   - MO columns of C are ordered: core [0, ncore), fragment 0, fragment 1, ..., virtuals.
 *   - B_packed[L * nao(nao+1)/2 + mu(mu+1)/2 + nu] = b^L_{mu nu} for mu >= nu.
 *   - Calls are asynchronous on the context's stream, except where stated.  A call returns
 *     LAS_OK once its work is queued; errors found on the device (a failed bounds or status
 *     check inside a kernel) are recorded in a status word and reported by the next
 *     las_sync() (and by every later call).  The library never aborts and never traps.
 *   - Device memory is allocated by las_create and freed by las_destroy; the energy, gradient
 *     and JK calls allocate nothing.  The first call of las_frag_ao2mo, las_veff and
 *     las_orbital_hvp, and in LAS_SPLIT_BF16 mode the first las_df_transform that asks for
 *     Lpu, allocates that call's own scratch, kept until las_destroy (las_frag_ao2mo grows
 *     its scratch when a later call needs more, after waiting for the context's stream).
 *   - A context is not thread-safe: use one context per host thread, or serialise calls.
 */
#ifndef LAS_H_
#define LAS_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct las_ctx las_ctx;

typedef enum {
  LAS_OK = 0,
  LAS_ERR_ARG = 1,        /* invalid argument (sizes, partition, null pointer) */
  LAS_ERR_CUDA = 2,       /* a CUDA runtime call failed */
  LAS_ERR_WORKSPACE = 3,  /* workspace cap too small for the smallest chunk */
  LAS_ERR_TIMEOUT = 4,    /* a bounded device-side wait ran out */
  LAS_ERR_INTERNAL = 5,   /* a device-side consistency check failed */
  LAS_ERR_UNSUPPORTED = 6 /* valid request the library does not support (e.g. sizes too large) */
} las_status;

typedef enum {
  LAS_FP64 = 0,       /* all contractions in native FP64 (DMMA) */
  LAS_SPLIT_BF16 = 1, /* bulk contractions as split-precision (BF16 digit) GEMMs on tcgen05
                         with exact FP32 partial sums recombined in integer arithmetic;
                         reductions, traces and gradient assembly stay in FP64.  The digit
                         planes of B hold the full rows of every b^L, each row scaled by its
                         own power of two */
  LAS_SPLIT_BF16_PACKED = 2
                      /* LAS_SPLIT_BF16 with the digit planes of B in packed-triangle form
                         (section "Calculation of effective potentials": only the lower
                         triangle of each b^L is stored): 128 x 128 tiles of the lower triangle,
                         the diagonal tiles whole, the rows past the last whole 128-row block
                         whole; the half transform reads a stored tile as it is for its own row
                         block and transposed for its column block.  One power of two per b^L
                         (a stored element serves two rows), so about one bit less precision in
                         the half transform; about 0.55 of the digit bytes (46 GB instead of
                         83 GB at Nao = 1200, Naux = 4800).  Every call behaves as in
                         LAS_SPLIT_BF16. */
} las_precision;

typedef struct {
  int nao;          /* number of AOs n */
  int naux;         /* number of auxiliary (Cholesky) vectors X */
  int nmo;          /* number of MO columns of C, ncore + sum(nact) <= nmo <= nao */
  int ncore;        /* doubly occupied core orbitals c */
  int nfrag;        /* number of fragments (0 allowed: closed-shell core only) */
  const int* nact;  /* host array [nfrag]: active orbitals per fragment, each >= 1 */
} las_dims;

/* Create a context over the packed Cholesky vectors B_packed (device, naux*nao(nao+1)/2
 * doubles), the factors b^P of Eq. cholesky in the packed lower-triangle storage of section
 * "Calculation of effective potentials".  In LAS_FP64 mode the context keeps a reference to B_packed, which must stay valid
 * and unchanged until las_destroy.  In LAS_SPLIT_BF16 mode it builds, once, the digit planes of
 * B (owned by the context); afterwards B_packed is read only by the JK calls (las_df_jk,
 * las_df_jk_density, las_veff: the Coulomb matrix is accumulated over the packed triangle), so
 * a caller that never makes a JK call may free it after las_create returns.
 * max_workspace_bytes caps the per-evaluation workspace (0 = choose); the auxiliary index is
 * processed in chunks that fit it.  stream: a cudaStream_t (NULL = the legacy default stream).
 * Synchronous with respect to the set-up work.
 * B_packed may hold any block of auxiliary rows (dims->naux of them): every two-electron term of
 * the energy and of its gradients is a sum over L, so the results of contexts over disjoint
 * blocks that together cover the auxiliary index add up to the whole system's, provided that
 * exactly one of them is passed the one-electron matrix h and the others a zero matrix. */
las_status las_create(las_ctx** ctx, const las_dims* dims, const double* B_packed,
                      las_precision precision, size_t max_workspace_bytes, void* stream);

las_status las_destroy(las_ctx* ctx);

/* Change the stream later calls are queued on. */
las_status las_set_stream(las_ctx* ctx, void* stream);

/* Wait for all queued work of this context; return the first recorded error, if any. */
las_status las_sync(las_ctx* ctx);

/* Bytes of device memory owned by the context (workspace + digit planes). */
size_t las_device_bytes(const las_ctx* ctx);

/* AO2MO half and full transforms (Eqs. ao2mo_1, ao2mo_2) over the active orbitals u:
 *   Lmu_u[L][mu][u] = sum_nu b^L_{mu nu} C[nu][ncore+u]            (naux x nao x nact_total)
 *   Lpu[L][p-p0][u] = sum_mu C[mu][p] Lmu_u[L][mu][u],  p in [p0,p1) (naux x (p1-p0) x nact_total)
 * C: device [nao][nmo].  Either output may be NULL.  0 <= p0 <= p1 <= nmo.
 * In LAS_SPLIT_BF16 mode both products are split-precision GEMMs: the second takes the rows
 * (L, u) of the half transform and the rows p of C^T as digit planes and writes Lpu in the
 * layout above directly from the GEMM epilogue. */
las_status las_df_transform(las_ctx* ctx, const double* C, int p0, int p1, double* Lmu_u,
                            double* Lpu);

/* Coulomb and exchange matrices (Eqs. J_1-K_2) of the core density Dc = 2 C_core C_core^T:
 *   J[mu][nu] = sum_L b^L_{mu nu} sum_{la,si} b^L_{la si} Dc[la][si]
 *   K[mu][nu] = sum_L sum_{la,si} b^L_{mu la} Dc[la][si] b^L_{si nu}
 * J, K: device [nao][nao]; either may be NULL. */
las_status las_df_jk(las_ctx* ctx, const double* C, double* J, double* K);

/* The JK call of Eqs. J_1-K_2 for a general symmetric density given in factored form,
 *   D = sum_{k < r} w[k] Cx[:,k] Cx[:,k]^T     (Cx: device [nao][r] row-major, w: device [r]),
 * e.g. D = C_x M C_x^T after diagonalising M, or one spin density gamma_sigma of Eq. v_emb:
 *   J[mu][nu] = sum_L b^L_{mu nu} Tr(b^L D),   K[mu][nu] = sum_L (b^L D b^L)_{mu nu}.
 * Weights of either sign are allowed (D = D+ - D- is evaluated as two factored parts, each over
 * the columns of its sign; zero weights are skipped).  The call reads the two column counts back
 * to the host once (one synchronisation of the context's stream), so it is not graph-capturable.
 * Requires r <= ncore + sum(nact) of the context (create a JK context with ncore >= r and no
 * fragments for densities of other ranks).  r = 0 (Cx, w may then be NULL) gives J = K = 0.
 * J, K: device [nao][nao]; either may be NULL. */
las_status las_df_jk_density(las_ctx* ctx, const double* Cx, const double* w, int r, double* J,
                             double* K);

/* Fragment-embedding AO2MO of a CASSCF subproblem (Eqs. ao2mo_1, ao2mo_2, ppaa, papa): the
 * context holds the Cholesky vectors b^P_{e e'} in the fragment's embedded basis e (create it
 * with nao = nmo = the number of embedded orbitals, any ncore/fragments), M holds the embedded
 * MO coefficients and the active orbitals are its columns [a0, a0 + ma):
 *   b^P_{e2 p1} = b^P_{e1 e2} M[e1][p1],   b^P_{p1 p2} = b^P_{e2 p1} M[e2][p2],
 *   ppaa[p1][p2][a1][a2] = sum_P b^P_{p1 p2} b^P_{a0+a1, a0+a2}            (nmo x nmo x ma x ma)
 *   papa[p1][a1][p2][a2] = sum_P b^P_{p1, a0+a1} b^P_{p2, a0+a2}          (nmo x ma x nmo x ma)
 * M: device [nao][nmo] row-major; ppaa, papa: device, row-major as shown; either may be NULL.
 * The first call allocates the call's own workspace (kept by the context until las_destroy);
 * the auxiliary index is processed in chunks that fit the context's workspace cap. */
las_status las_frag_ao2mo(las_ctx* ctx, const double* M, int a0, int ma, double* ppaa,
                          double* papa);

/* Effective potentials of Eq. v_emb (Eq. vself when the context holds a fragment's embedded-basis
 * Cholesky vectors and the densities are the fragment's own), for spin densities in factored
 * form gamma_sigma = C_sigma diag(w_sigma) C_sigma^T (C_sigma: device [nao][r_sigma], w_sigma:
 * device [r_sigma]; either rank may be 0):
 *   v_sigma = J[gamma_alpha + gamma_beta] - K[gamma_sigma]          (device [nao][nao] each)
 * Two general-density JK calls (las_df_jk_density) and their combination; the same rank limit
 * applies to r_alpha and r_beta. */
las_status las_veff(las_ctx* ctx, const double* C_alpha, const double* w_alpha, int r_alpha,
                    const double* C_beta, const double* w_beta, int r_beta, double* v_alpha,
                    double* v_beta);

/* Orbital Hessian-vector product at fixed fragment RDMs (the orbital part of the second-order
 * step of Eq. flas; the paper leaves the forms to its references): for an antisymmetric
 * X (device [nmo][nmo]) and dC = C X,
 *   dG = directional derivative of dE/dC along dC                      (device [nao][nmo])
 *   Dg = d/dt g(C exp(tX)) at t = 0 = (C X)^T G + C^T dG - transpose   (device [nmo][nmo],
 *        NULL to skip; g = C^T dE/dC - transpose is the orbital-rotation gradient)
 * dG is the tangent of the evaluation chain (dE/dC = one-electron terms + sum_L H_L W(T_L), W
 * linear in T): one more half transform b^L dC, one more full-transform product, two per-aux
 * passes and two projections, next to one plain evaluation for G.  Asynchronous.  The first
 * call allocates the tangent's scratch (about the evaluation's per-chunk workspace again). */
las_status las_orbital_hvp(las_ctx* ctx, const double* C, const double* h, const double* dm1s,
                           const double* dm2, const double* X, double* dG, double* Dg);

/* LAS energy E_LAS = <LAS|H|LAS> of the product state of Eq. las_wfn (section "LASSCF
 * algorithm"; no constant term, as with Eq. h_emb), from the core and active densities: the
 * Coulomb and exchange parts of Eqs. J_1-K_2 and the active integrals of Eq. ppaa, both formed
 * per auxiliary index from b^L C_occ and never stored whole.
 * h: device [nao][nao] one-electron Hamiltonian (symmetric).
 * dm1s: device, per fragment K the spin-separated 1-RDM [2][m_K][m_K] (alpha, beta),
 *       concatenated over fragments.
 * dm2:  device, per fragment K the spin-summed 2-RDM [m_K]^4 in chemists' order,
 *       Gamma[p][q][r][s] = sum_{s,t} <p+_s r+_t s_t q_s>, concatenated over fragments.
 * E:    device pointer to one double (written asynchronously). */
las_status las_energy(las_ctx* ctx, const double* C, const double* h, const double* dm1s,
                      const double* dm2, double* E);

/* LAS energy and its derivative with respect to the MO coefficients (the gradient whose
 * vanishing is Eq. MO_conv):
 *   dEdC: device [nao][nmo], dE/dC[mu][p] (zero in the virtual columns);
 *   gorb: device [nmo][nmo] or NULL, the antisymmetric orbital-rotation gradient
 *         g = C^T dEdC - (C^T dEdC)^T, so that d/de E(C exp(e X))|_0 = sum_pq g[p][q] X[p][q] / 2
 *         for antisymmetric X (equivalently sum_pq (C^T dEdC)[p][q] X[p][q]). */
las_status las_energy_grad(las_ctx* ctx, const double* C, const double* h, const double* dm1s,
                           const double* dm2, double* E, double* dEdC, double* gorb);

/* The same evaluation with HOST inputs and outputs: C_host [nao][nmo], h_host [nao][nao],
 * dm1s_host, dm2_host as above, E_host (1 double), dEdC_host [nao][nmo] (may be NULL).
 * Copies in through context-owned device buffers, evaluates, copies back and synchronises.
 * Host buffers may be pageable; page-locked buffers give overlapped, faster copies. */
las_status las_energy_grad_host(las_ctx* ctx, const double* C_host, const double* h_host,
                                const double* dm1s_host, const double* dm2_host,
                                double* E_host, double* dEdC_host);

/* One item of a batched evaluation: device pointers as for las_energy_grad (dEdC required). */
typedef struct {
  const double* C;
  const double* h;
  const double* dm1s;
  const double* dm2;
  double* E;
  double* dEdC;
} las_batch_item;

/* Evaluate nsys independent problems (item i on ctxs[i], all distinct contexts) as one CUDA
 * graph on `stream`: the first call with a given list of contexts, item pointers and stream
 * captures every problem's chain of kernels; later calls with the same arguments replay the
 * captured graph with a single launch.  Inputs may change between calls (the pointers may not).
 * A graph is dropped when any of its contexts is destroyed.  Asynchronous. */
las_status las_energy_grad_batched(int nsys, las_ctx* const* ctxs, const las_batch_item* items,
                                   void* stream);

/* Autotuner (split mode; no-op in FP64 mode): by timing whole evaluations with per-stage CUDA
 * events, chooses for this context the tile width (64 or 96 output columns) of each product kind
 * -- the half transform S1, the full transform S2, the projection S5/S6 and the one-electron
 * products -- and then the split-K factor of the projection, keeping the fastest of each.  The
 * choices apply to every later call of the context, batched evaluations included.  Writes E and
 * dEdC as a side effect.  Synchronous. */
las_status las_autotune(las_ctx* ctx, const double* C, const double* h, const double* dm1s,
                        const double* dm2, double* E, double* dEdC);

/* Tile widths of the split products of a context (bn4: host int[4], for S1, S2, projection and
 * one-electron products; each 64 or 96), as chosen by las_autotune or set by hand.  Split mode
 * only (LAS_ERR_UNSUPPORTED otherwise). */
las_status las_get_tiles(const las_ctx* ctx, int* bn4);
las_status las_set_tiles(las_ctx* ctx, const int* bn4);

/* Per-stage device times (milliseconds), averaged over the evaluations run since timing was
 * enabled with las_set_timing(ctx, 1) or since the last las_stage_times call (up to the last
 * 64), measured with CUDA events recorded on the context's stream inside each evaluation; only
 * the last evaluation's final event is waited for.  Stage order: [0] C packing and half
 * transform (S1), [1] occupied full transform (S2), [2] per-aux contractions, [3] projections
 * (S5/S6), [4] one-electron terms, energy and gradient assembly.  With more than one auxiliary
 * chunk, stages 0-3 cover the first chunk only.  Returns the number of stages written (<= cap). */
las_status las_set_timing(las_ctx* ctx, int enable);
int las_stage_times(las_ctx* ctx, float* ms, int cap);

/* Emulated-FP64 GEMM on the BF16 tensor cores, the building block of LAS_SPLIT_BF16:
 *   C[M][N] = A[M][K] * B[K][N]   (row-major, leading dimensions lda >= K, ldb >= N, ldc >= N)
 * A is scaled per row and B per column by powers of two, each cut into six BF16 digits, and the
 * 21 digit products of total weight <= 2^-40 are formed with exact FP32 partial sums for the
 * four leading weights 2^0 ... 2^-24 (flushed to integers and recombined in integer arithmetic)
 * and one FP32 sum for the weights 2^-32 and 2^-40.  The error is
 * that of truncating both operands to 47 bits below their row / column maximum.
 * The method has no counterpart in the paper (which runs FP64 GEMMs and names reduced precision
 * only as an outlook, section "Outlook"); it implements that outlook for this hardware.
 * workspace: device buffer of at least las_split_gemm_workspace(M, N, K) bytes, 256-byte
 * aligned, owned by the caller.  Synchronous: returns after C is written (or an error). */
size_t las_split_gemm_workspace(long M, long N, long K);
las_status las_split_gemm(long M, long N, long K, const double* A, long lda, const double* B,
                          long ldb, double* C, long ldc, void* workspace,
                          size_t workspace_bytes, void* stream);

/* Allocation-free emulated-FP64 GEMM: the same product as las_split_gemm for callers that
 * cannot allocate device memory where they need a product -- plugins whose host application
 * owns every device allocation through its own pool (a cudaMalloc behind its back would break
 * its accounting or fail), or loops where a cudaMalloc could synchronise the device.  The paper
 * has no counterpart; this is a service of this library.
 * Scratch: a fixed LAS_NOALLOC_SCRATCH_BYTES device array inside the library image (held by
 * every GPU that loads the library until the process exits); nothing is allocated or freed.
 * Sizes whose digit planes do not fit the array, i.e. las_split_gemm_workspace(M, N, K) >
 * LAS_NOALLOC_SCRATCH_BYTES, are rejected with LAS_ERR_WORKSPACE before any GPU work.
 * The first call on each device looks up the array's device address (with that device
 * current) and keeps it for later calls; make that first call before any stream capture
 * begins.  A reset of the device's primary context (cudaDeviceReset) invalidates the kept
 * address: do not call this entry point after such a reset.
 * All calls share the one array, which keeps the last call's contents: calls that may overlap
 * on the GPU (different streams or host threads without ordering) race and must be serialised
 * by the caller.
 * Synchronous, like las_split_gemm: it waits for its stream and reads a status word back. */
#define LAS_NOALLOC_SCRATCH_BYTES (64u << 20)
las_status las_split_gemm_noalloc(long M, long N, long K, const double* A, long lda,
                                  const double* B, long ldb, double* C, long ldc, void* stream);

/* Self-test of the device-side failure detection (no counterpart in the paper): one kernel waits
 * on a barrier that is never signalled, with a short poll limit.  Returns LAS_ERR_TIMEOUT when
 * the bounded wait gave up and the kernel returned as designed (the device stays usable),
 * LAS_ERR_CUDA on a CUDA error.  stream: cudaStream_t or NULL. */
las_status las_selftest_bounded_wait(void* stream);

/* FP64 throughput probe (no counterpart in the paper; the denominator of the native-FP64
 * roofline): two register-resident loops over all SMs of the current device, one of FP64
 * tensor-core MMAs (mma.sync m16n8k4 f64, the instruction of the FP64 GEMMs) and one of FP64
 * fused multiply-adds, each timed with CUDA events on `stream` after a warm-up launch.
 * dmma_tflops, dfma_tflops: host pointers, written with the measured rates in TFLOP/s.
 * Allocates and frees 8 bytes of device memory.  Synchronous (about a second). */
las_status las_probe_fp64(double* dmma_tflops, double* dfma_tflops, void* stream);

/* Number of kernels this library has launched in this process so far (all contexts). */
long las_kernel_launches(void);

const char* las_status_str(las_status status);

#ifdef __cplusplus
}
#endif

#endif /* LAS_H_ */
