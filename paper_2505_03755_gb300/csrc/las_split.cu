// Split-precision (emulated FP64) GEMMs on the tcgen05 tensor cores.
//
// An FP64 operand is scaled per row (A) or per column (B) by a power of two 2^e with
// max|x| < 2^e, rounded to 47 fractional bits and cut into NDIG = 6 balanced base-256 digits,
//     x = 2^e * 2^-7 * sum_s d_s 2^-8s ,   |d_s| <= 128,
// each stored exactly as a BF16 "digit plane" value d_s * 2^-8s.  The product keeps the digit pairs
// with s + t <= 5 (21 of 36):
//   * groups q = s + t = 0..3 are accumulated EXACTLY: every partial sum is an integer multiple
//     of 2^-8q of magnitude at most 2^24 * 2^-8q when a group is flushed every 256 values of k,
//     so the FP32 tensor-core accumulator loses nothing; each flush is added, as an integer, into
//     an int64 fixed-point accumulator;
//   * groups q = 4, 5 (weights 2^-32 and 2^-40) each have one FP32 accumulator over the whole
//     K range of a tile.  (The tensor core's FP32 accumulation of products of very different
//     weights is measurably less accurate than IEEE rounding, which is why weight 2^-24 is kept
//     in the exact part and every accumulator holds one weight only.)
// The recombination uses integer arithmetic only (FP64 arithmetic is slow on this part): the
// fixed-point sum and the two rounded FP32 tails are merged into one int64 and turned into an
// FP64 value by building its bit pattern.  The chosen digit count and pair set follow the split-product
// ("Ozaki") scheme for emulating a higher precision with low-precision products.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "las_split.cuh"
#include "sm100_ptx.cuh"

namespace lasdf_split {

constexpr int NDIG = 6;
constexpr int BM = 128;          // rows per CTA tile (tcgen05 M)
constexpr int BK = 16;           // K per pipeline stage (one 32-byte swizzle row of BF16)
constexpr int NEXACT = 4;        // exact weight groups q = 0..3
constexpr int NGROUP = 6;        // weight groups q = s + t = 0..5 kept (21 digit pairs)

constexpr int CHUNK = 16;        // stages per exact chunk (256 values of k)
constexpr int A_PLANE = BM * BK * 2;                 // 4096 B
constexpr int A_BYTES = NDIG * A_PLANE;              // 24576
constexpr int TMEM_COLS = 512;
constexpr int EPI_WARPS = 16;    // epilogue warps: 4 column groups x 4 TMEM lane quarters
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;   // warp 0 TMA, warp 1 MMA, warps 2.. epilogue

// Tile width bn (columns of the output per CTA tile, a product's parameter: 64 or 96) and the
// stage layout, sized for the widest tile BN.  The exact weight groups q = 0..3 each own one
// FP32 accumulator of bn TMEM columns, at column q*bn, and the tail groups 4 and 5 share one
// more, at the fixed column TAIL_COL = 4*BN whatever the tile width, so that consecutive tiles
// of different widths in one launch never put one tile's tail where the previous tile's exact
// accumulators are still being drained (every accumulator starts at a multiple of 32).  The
// six B digit planes of a stage lie back to back in shared memory (plane t at t*bn rows), so
// that one MMA of A_s against planes t0..t1 of B (N = (t1-t0+1)*bn <= 256) lands every product
// A_s B_t in the accumulator of its own exact group s + t (mma_slab): the ten exact products of a
// stage take six MMAs at bn = 96 (four of N = 192) and four at bn = 64 (N = 256, 192, 128, 64).
// (Tiles with a second tail accumulator, so that the tail products could be merged the same way,
// measured slower: a shorter stage carries the same waits for data and for the exact drains.)
template <int BN_>
struct OzTile {
  static constexpr int BN = BN_;   // the widest tile the stage layout holds
  static_assert(BN % 32 == 0 && (NEXACT + 1) * BN <= TMEM_COLS, "tile width");
  static constexpr int B_PLANE = BN * BK * 2;    // bytes per B plane at the widest tile
  static constexpr int TAIL_COL = NEXACT * BN;   // TMEM column of the tail accumulator
  static constexpr int B_BYTES = NDIG * B_PLANE;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int NSTAGE = (220 * 1024) / STAGE_BYTES < 6 ? (220 * 1024) / STAGE_BYTES : 6;
  static constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024 + 256;
  // epilogue: a tile's bn columns as 8-column blocks dealt round-robin to the 4 column groups
  // (every TMEM load is 8 columns at an 8-aligned column)
  static constexpr int MAXB = (BN / 8 + 3) / 4;  // blocks per epilogue thread, at most
  static_assert(STAGE_BYTES % 1024 == 0, "stages stay 1024-byte aligned");
};

// Digit planes are stored K-blocked: element (s, r, k) of an operand with R rows lives at
//   s*plane + (k / BK) * (Rpad * BK) + r * BK + (k % BK),   Rpad = R rounded up to ROWPAD,
// so that every pipeline stage of every tile is one contiguous block per plane.  A tile box that
// reaches past Rpad reads the next K block's rows (finite digits) or, at the end of a plane, the
// TMA's zero fill: those rows only feed output rows or columns beyond M or N, which are never
// stored.
constexpr long ROWPAD = 384;

struct Planes {
  __nv_bfloat16* p;
  long R, Rpad, K, nkb, plane;   // rows, padded rows, K, K blocks, elements per plane
  __host__ __device__ __forceinline__ long idx(int s, long r, long k) const {
    return s * plane + (k / BK) * (Rpad * BK) + r * BK + (k % BK);
  }
};

static inline long planes_rpad(long R) { return (R + ROWPAD - 1) / ROWPAD * ROWPAD; }
static inline long planes_nkb(long K) { return (K + BK - 1) / BK; }
static inline size_t planes_bytes(long R, long K) {
  return (size_t)NDIG * planes_rpad(R) * planes_nkb(K) * BK * 2;
}
static inline Planes make_planes(void* p, long R, long K) {
  Planes P;
  P.p = (__nv_bfloat16*)p;
  P.R = R;
  P.Rpad = planes_rpad(R);
  P.K = K;
  P.nkb = planes_nkb(K);
  P.plane = P.nkb * P.Rpad * BK;
  return P;
}

// The Cholesky vectors as digit planes in packed-triangle form.  The first n1 = 128 nb1 rows of
// every b^L lie in full 128-row blocks, of which only the lower tiles (I >= J) are stored (the
// diagonal tiles whole): T = nb1 (nb1 + 1) / 2 tiles per L, tile (I, J) of L at index
// L T + I (I + 1) / 2 + J, each as 8 K blocks of 128 rows x 16 (the Planes layout with 128 rows
// and 8 X T K blocks).  The half transform reads a tile as it is stored for the rows of block I
// and MN-major (transposed) for the rows of block J.  The r = n - n1 ragged rows mu >= n1 of each
// b^L are stored whole (rows (L, mu - n1), K = nu); they are read as they are for their own rows
// and MN-major for the columns nu >= n1 of the full blocks.  One exponent per L (max |b^L| <
// 2^e(L)), so that a stored element has the same scale for both rows that use it.
struct BPacked {
  int n, X, nb1, T, r, n1;
  Planes tiles;       // R = Rpad = 128, nkb = 8 X T
  Planes rag;         // rows (L, j), j < r, of all X r; K = n
  int* exp;           // [X]
  unsigned long long* mx;   // [X] max |b^L| as ordered bit patterns (set-up scratch)
};

static inline BPacked bpacked_geometry(int n, int X) {
  BPacked b;
  memset(&b, 0, sizeof(b));
  b.n = n;
  b.X = X;
  b.nb1 = n / 128;
  b.T = b.nb1 * (b.nb1 + 1) / 2;
  b.n1 = 128 * b.nb1;
  b.r = n - b.n1;
  return b;
}
static inline size_t bpacked_tile_bytes(const BPacked& b) {
  return (size_t)NDIG * 8 * (size_t)b.X * b.T * 128 * BK * 2;
}

struct OzParams {
  int M, N;                // output rows / columns
  int a_rpad, b_rpad;      // padded rows of the A / B plane layouts
  int a_row0, b_row0;      // first row of A / B used (row offset inside the layouts)
  int kb_total;            // K blocks of BK
  int kb_per_split;
  int ksplit;
  const int* ea;           // row exponents [M] (nullptr: 0)
  const int* eb;           // column exponents [N]
  double* out;
  int mode;                // 0: out[z*zstride + r*ldc + c]; 1: Ht layout (rows (L,mu))
  long ldc, zstride;
  int ht_n, ht_op;
  int lower;               // symmetric product: only tiles that touch the lower triangle
  long tiles_z;            // tiles per K split (the lower-triangle ones only when lower != 0)
  int sh;                  // fractional bits kept when merging the tail
  int bn;                  // tile width: 64 or 96 columns
  int a_mn;                // A read MN-major: rows of the stored planes are K, their K is M
  // A = the Cholesky vectors in packed-triangle digit form (a_pack != 0; see BPacked): the
  // product's row tiles are the full 128-row blocks R of each b^L (tile m = L * pk_nb1 + R of the
  // chunk), and each 16-wide K block is read from the stored lower tile (R, J) as is (J <= R),
  // from the stored tile (J, R) MN-major (R < J < pk_nb1), or from the ragged rows nu >= n1 of
  // b^L MN-major (tensor maps tmA, tmA2 and tmA3)
  int a_pack;
  int pk_nb1, pk_T, pk_r;  // full row blocks per L, stored tiles per L, ragged rows per L
  int pk_L0;               // first auxiliary index of the chunk
  int ht_rows, ht_mu0;     // mode 1: rows of the product per L, and mu of its first row
  int ea_perL;             // the row exponents are per auxiliary index: ea[L], not ea[row]
  int* status;
};

// W * 2^E rounded once to FP64 (round to nearest even): the hardware int64 -> FP64 conversion,
// then an exponent-field shift (exact for normal results; the rare others go through ldexp).
__device__ __forceinline__ double make_double(long long W, int E) {
  const double v = __ll2double_rn(W);
  const long long b = __double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0 || ex + E <= 0 || ex + E >= 2047) return ldexp(v, E);
  return __longlong_as_double(b + ((long long)E << 52));
}

// Column tiles of row tile i that touch the lower triangle (column tile j with j*bn < (i+1)*BM).
__host__ __device__ __forceinline__ int lower_tiles_in_row(int i, int ntn, int bn) {
  const int c = ((i + 1) * BM + bn - 1) / bn;
  return c < ntn ? c : ntn;
}

__device__ __forceinline__ void tile_coords(const OzParams& p, long t, int& m0, int& n0,
                                            int& kb0, int& nkb) {
  const int bn = p.bn;
  const int ntn = (p.N + bn - 1) / bn;
  const int z = (int)(t / p.tiles_z);
  long rem = t - (long)z * p.tiles_z;
  // the column tiles of one row tile are adjacent in tile order so that concurrently running
  // CTAs share that row tile's digit planes through L2
  if (!p.lower) {
    m0 = (int)(rem / ntn) * BM;
    n0 = (int)(rem % ntn) * bn;
  } else {
    // only the tiles that touch the lower triangle are enumerated, so that the persistent CTAs
    // share out the work evenly
    int i = 0;
    for (int c = lower_tiles_in_row(0, ntn, bn); rem >= c; c = lower_tiles_in_row(++i, ntn, bn))
      rem -= c;
    m0 = i * BM;
    n0 = (int)rem * bn;
  }
  kb0 = z * p.kb_per_split;
  nkb = min(p.kb_total, kb0 + p.kb_per_split) - kb0;
}

// One product of a grouped launch: its tensor maps, parameters and first tile in the launch's
// tile order (problems are concatenated; tile0 of problem g+1 = tile0 + tiles of problem g).
struct OzProblem {   // aligned as its tensor maps
  CUtensorMap tmA, tmB, tmA2, tmA3;   // tmA2, tmA3: packed-triangle A only
  OzParams p;
  long tile0;
};

// The tile a role works on: its product (parameters and maps) and coordinates.  A role's tiles
// only ever increase, so the product index moves forward only.
template <bool GROUPED>
struct OzCursor {
  int g = 0;
  const OzParams* P = nullptr;
  const CUtensorMap* ma = nullptr;
  const CUtensorMap* mb = nullptr;
  const CUtensorMap* ma2 = nullptr;
  const CUtensorMap* ma3 = nullptr;
  int m0 = 0, n0 = 0, kb0 = 0, nkb = 0;
  __device__ __forceinline__ bool seek(long t, const OzParams& p1, const CUtensorMap* a1,
                                       const CUtensorMap* b1, const CUtensorMap* a2,
                                       const CUtensorMap* a3, const OzProblem* probs,
                                       int nprob) {
    long tl = t;
    bool moved = P == nullptr;
    if constexpr (GROUPED) {
      while (g + 1 < nprob && probs[g + 1].tile0 <= t) {
        ++g;
        moved = true;
      }
      P = &probs[g].p;
      ma = &probs[g].tmA;
      mb = &probs[g].tmB;
      ma2 = &probs[g].tmA2;
      ma3 = &probs[g].tmA3;
      tl = t - probs[g].tile0;
    } else {
      P = &p1;
      ma = a1;
      mb = b1;
      ma2 = a2;
      ma3 = a3;
    }
    tile_coords(*P, tl, m0, n0, kb0, nkb);
    return moved;
  }
};

// D[groups s+t0 .. s+t0+nt-1] (+)= A_s * [B_t0 .. B_t0+nt-1]^T: nt consecutive B planes (tile
// width BNV, planes BNV*32 bytes apart) against one A plane, as ceil(nt / maxp) MMAs of balanced
// width (N = np * BNV <= 256).  Everything is a compile-time constant once inlined: the single
// issuing thread must not spend its time on address arithmetic.
// Descriptor of A plane s of a stage: K-major, or MN-major (amn) when the stage holds the
// transposed access of planes stored with rows along K.
__device__ __forceinline__ uint64_t a_desc(uint32_t sa, int s, bool amn) {
  return amn ? sm100::smem_desc_sw32_mn(sa + s * A_PLANE) : sm100::smem_desc_sw32(sa + s * A_PLANE);
}

template <int BNV>
__device__ __forceinline__ void mma_slab(uint32_t tmem, uint32_t sa, uint32_t sb, int s, int t0,
                                         int nt, bool accumulate, bool amn) {
  constexpr int maxp = 256 / BNV;
  const int nm = (nt + maxp - 1) / maxp;
  int t = t0;
#pragma unroll
  for (int j = 0; j < nm; ++j) {
    const int np = (t0 + nt - t) / (nm - j);
    sm100::mma_bf16(tmem + (uint32_t)((s + t) * BNV), a_desc(sa, s, amn),
                    sm100::smem_desc_sw32(sb + t * BNV * BK * 2),
                    sm100::idesc_bf16(BM, np * BNV) | (amn ? sm100::IDESC_A_MN : 0u),
                    accumulate ? 1u : 0u);
    t += np;
  }
}

// One stage's tail products (groups 4 and 5, eleven MMAs into the tail accumulator at tail_col),
// started at the first stage of a tile.
template <int BNV>
__device__ __forceinline__ void mma_tail(uint32_t tmem_tail, uint32_t sa, uint32_t sb,
                                         bool first_stage, bool amn) {
  bool acc = !first_stage;
  const uint32_t idesc = sm100::idesc_bf16(BM, BNV) | (amn ? sm100::IDESC_A_MN : 0u);
#pragma unroll
  for (int s = 0; s < NDIG; ++s)
#pragma unroll
    for (int t = (s >= NEXACT ? 0 : NEXACT - s); s + t < NGROUP; ++t) {
      sm100::mma_bf16(tmem_tail, a_desc(sa, s, amn), sm100::smem_desc_sw32(sb + t * BNV * BK * 2),
                      idesc, acc ? 1u : 0u);
      acc = true;
    }
}

// One stage's exact products (groups 0..3): A_s against planes 0 .. 3-s; s = 0 spans all four
// groups and starts them at a chunk's first stage.
template <int BNV>
__device__ __forceinline__ void mma_exact(uint32_t tmem, uint32_t sa, uint32_t sb,
                                          bool first_in_chunk, bool amn) {
#pragma unroll
  for (int s = 0; s < NEXACT; ++s)
    mma_slab<BNV>(tmem, sa, sb, s, 0, NEXACT - s, s > 0 || !first_in_chunk, amn);
}

// Persistent CTAs (one per SM) walk the tiles (row tile, column tile, K split).  Roles:
// warp 0 streams digit-plane stages with TMA, warp 1 issues tcgen05.mma, warps 2..17 drain the
// TMEM accumulators.  Stage, chunk and tile counters run on across tiles so that the loads of the
// next tile overlap the last MMAs of the current one, and its MMAs overlap the current tile's
// conversion and stores.
// GROUPED: the launch walks the concatenated tiles of nprob products described in global
// memory (probs); otherwise the one product of the kernel parameters.  FIXBN: the tile width of
// every product of the launch as a compile-time constant (64 or 96), or 0 when products of both
// widths share a grouped launch (each tile then reads its product's width).  PACK: the launch
// may hold products whose A is the packed-triangle form of the Cholesky vectors (a_pack); the
// other instantiations leave that logic out of the issuing and loading threads entirely.  AMN:
// the A orientation of the launch's products as a compile-time constant (0: K-major, 1:
// MN-major), or 2 when each tile reads its product's; the issuing thread runs measurably faster
// with a constant.
template <int BN, bool GROUPED, int FIXBN, bool PACK, int AMN = 2>
__global__ void __launch_bounds__(NTHREADS, 1)
k_ozaki(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
        const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmA3,
        const __grid_constant__ OzParams p1, const OzProblem* __restrict__ probs, int nprob,
        long ntiles) {
  using T = OzTile<BN>;
  constexpr int NSTAGE = T::NSTAGE;
  constexpr int MAXB = T::MAXB;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + NSTAGE * T::STAGE_BYTES);
  uint64_t* full = bars;              // [NSTAGE]
  uint64_t* empty = bars + NSTAGE;    // [NSTAGE]
  uint64_t* accf = bars + 2 * NSTAGE;
  uint64_t* acce = bars + 2 * NSTAGE + 1;
  uint64_t* drain = bars + 2 * NSTAGE + 2;
  uint64_t* accT = bars + 2 * NSTAGE + 3;   // tail accumulators read out (once per tile)
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * NSTAGE + 4);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // status word for waits outside any tile (the first product's)
  int* const status0 = GROUPED ? probs[0].p.status : p1.status;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      sm100::mbar_init(&full[s], 1);
      sm100::mbar_init(&empty[s], 1);
    }
    sm100::mbar_init(accf, 1);
    sm100::mbar_init(acce, EPI_WARPS);
    sm100::mbar_init(accT, EPI_WARPS);
    sm100::mbar_init(drain, 1);
    *abort_flag = 0;
    sm100::fence_mbar_init();
    if (!GROUPED) {
      sm100::tma_prefetch_desc(&tmA);
      sm100::tma_prefetch_desc(&tmB);
      if (PACK && p1.a_pack) {
        sm100::tma_prefetch_desc(&tmA2);
        sm100::tma_prefetch_desc(&tmA3);
      }
    }
  }
  if (warp == 1) {
    sm100::tmem_alloc(tmem_slot, TMEM_COLS);
    sm100::tmem_relinquish();
  }
  sm100::tc_fence_before();
  __syncthreads();
  sm100::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    long gs = 0;
    bool ok = true;
    OzCursor<GROUPED> cur;
    for (long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      if (cur.seek(t, p1, &tmA, &tmB, &tmA2, &tmA3, probs, nprob) && GROUPED) {
        sm100::tma_prefetch_desc(cur.ma);
        sm100::tma_prefetch_desc(cur.mb);
        if (PACK && cur.P->a_pack) {
          sm100::tma_prefetch_desc(cur.ma2);
          sm100::tma_prefetch_desc(cur.ma3);
        }
      }
      const OzParams& p = *cur.P;
      // packed-triangle A, per tile: its row block R of b^L (tile (L, R) of the chunk), the K
      // block of stored tile (R, 0), the index of stored tile (R, R) less R (R + 1) / 2, and the
      // ragged row of K block 0, so that each stage adds its K block kb = 8 J + kk only
      int pk_R = 0;
      long pk_row = 0, pk_col = 0, pk_rag = 0;
      if (PACK && p.a_pack) {
        const int mt = cur.m0 / BM, Lr = mt / p.pk_nb1;
        pk_R = mt - Lr * p.pk_nb1;
        const long Lg = (long)p.pk_L0 + Lr;
        pk_row = (Lg * p.pk_T + pk_R * (pk_R + 1) / 2) * 8;
        pk_col = Lg * p.pk_T + pk_R;
        pk_rag = Lg * p.pk_r - 8L * p.pk_nb1 * BK;
      }
      for (int i = 0; i < cur.nkb; ++i, ++gs) {
        const int st = (int)(gs % NSTAGE);
        if (gs >= NSTAGE && !sm100::mbar_wait(&empty[st], (uint32_t)((gs / NSTAGE) - 1) & 1,
                                              abort_flag, p.status, LAS_ERR_TIMEOUT)) {
          ok = false;
          break;
        }
        uint8_t* sa = smem + st * T::STAGE_BYTES;
        sm100::mbar_arrive_expect_tx(&full[st], A_BYTES + NDIG * (FIXBN ? FIXBN : p.bn) * BK * 2);
        const int kb = cur.kb0 + i;
        if (PACK && p.a_pack) {   // K block kb = 8 J + kk lies in column block J of b^L
          const int J = kb >> 3;
          if (J <= pk_R)           // stored lower tile (R, J): rows mu, K = nu
            sm100::tma_load_3d(sa, cur.ma, &full[st], 0, (int)((pk_row + kb) * BM), 0);
          else if (J < p.pk_nb1)   // stored tile (J, R) read MN-major: its rows are this K
            sm100::tma_load_4d(sa, cur.ma2, &full[st], 0, (kb & 7) * BK,
                               (int)((pk_col + J * (J + 1) / 2) * 8), 0);
          else                     // ragged rows nu >= n1 of b^L, MN-major
            sm100::tma_load_4d(sa, cur.ma3, &full[st], 0, (int)(pk_rag + (long)kb * BK),
                               pk_R * (BM / BK), 0);
        } else if (p.a_mn) {   // rows of the stored planes are this product's K, their K blocks its M
          sm100::tma_load_4d(sa, cur.ma, &full[st], 0, p.a_row0 + kb * BK, cur.m0 / BK, 0);
        } else {
          sm100::tma_load_3d(sa, cur.ma, &full[st], 0, kb * p.a_rpad + p.a_row0 + cur.m0, 0);
        }
        sm100::tma_load_3d(sa + A_BYTES, cur.mb, &full[st], 0,
                           kb * p.b_rpad + p.b_row0 + cur.n0, 0);
      }
    }
    // never leave the CTA with a bulk copy still writing its shared memory
    for (long g = (gs > NSTAGE ? gs - NSTAGE : 0); g < gs; ++g)
      sm100::mbar_wait(&full[g % NSTAGE], (uint32_t)(g / NSTAGE) & 1, abort_flag, status0,
                       LAS_ERR_TIMEOUT);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    // Per stage the tail MMAs (groups 4 and 5) are issued at once; the exact-group MMAs of the
    // first stages of a chunk may be deferred (their stages stay resident) until the epilogue
    // has drained the previous chunk, so that the drain overlaps tensor work.
    long gs = 0, gc = 0, tcount = 0;
    bool ok = true, need_acce = false;
    OzCursor<GROUPED> cur;
    for (long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      cur.seek(t, p1, &tmA, &tmB, &tmA2, &tmA3, probs, nprob);
      const OzParams& p = *cur.P;
      const int nkb = cur.nkb;
      const int bn = FIXBN ? FIXBN : p.bn;
      const bool amn_tile = p.a_mn != 0;
      // packed-triangle A: K blocks of column blocks J > R (above the diagonal) are read MN-major
      const bool pack = PACK && p.a_pack != 0;
      const int kb_mn = pack ? 8 * ((cur.m0 / BM) % p.pk_nb1 + 1) : 0;
      // the tail accumulators of the previous tile must have been read out
      if (tcount > 0) {
        if (!sm100::mbar_wait(accT, (uint32_t)(tcount - 1) & 1, abort_flag, p.status,
                              LAS_ERR_TIMEOUT)) {
          ok = false;
          break;
        }
        sm100::tc_fence_after();
      }
      long pend0 = 0;     // first deferred stage (global index) and count
      int npend = 0, pend_i0 = 0;
      // One stage: wait for its data, issue its tail MMAs, then the exact-group MMAs of the
      // deferred stages and its own unless they are deferred again (never at the end of a chunk
      // or of a phase: flush).  amn is the stage's A orientation.  False when a wait ran out.
      auto stage = [&](auto amn_c, int i, bool flush) -> bool {
        constexpr bool amn = decltype(amn_c)::value;   // the orientation as a constant
        const int st = (int)(gs % NSTAGE);
        if (!sm100::mbar_wait(&full[st], (uint32_t)(gs / NSTAGE) & 1, abort_flag, p.status,
                              LAS_ERR_TIMEOUT))
          return false;
        sm100::tc_fence_after();
        {
          const uint32_t sa = sm100::smem_u32(smem + st * T::STAGE_BYTES);
          const uint32_t sb = sa + A_BYTES;
          // tail: the 11 products of groups 4 and 5 into the one tail accumulator
          if (bn == 64) mma_tail<64>(tmem + T::TAIL_COL, sa, sb, i == 0, amn);
          else mma_tail<96>(tmem + T::TAIL_COL, sa, sb, i == 0, amn);
        }
        const bool last_in_chunk = (i % CHUNK) == CHUNK - 1 || i == nkb - 1;
        if (need_acce) {
          if (!last_in_chunk && !flush && npend < NSTAGE - 1 &&
              !sm100::mbar_test_wait(acce, (uint32_t)(gc - 1) & 1)) {
            if (npend == 0) {
              pend0 = gs;
              pend_i0 = i;
            }
            ++npend;
            return true;   // defer this stage's exact-group MMAs
          }
          if (!sm100::mbar_wait(acce, (uint32_t)(gc - 1) & 1, abort_flag, p.status,
                                LAS_ERR_TIMEOUT))
            return false;
          sm100::tc_fence_after();
          need_acce = false;
        }
        if (npend == 0) {
          pend0 = gs;
          pend_i0 = i;
        }
        // exact groups q = 0..3 for the deferred stages and this one, in stage order: A_s
        // against planes 0 .. 3-s; s = 0 spans all four groups and starts them at a chunk's
        // first stage
        for (int j = 0; j <= npend; ++j) {
          const long g2 = pend0 + j;
          const int i2 = pend_i0 + j;
          const int st2 = (int)(g2 % NSTAGE);
          const bool first_in_chunk = (i2 % CHUNK) == 0;
          const uint32_t sa = sm100::smem_u32(smem + st2 * T::STAGE_BYTES);
          const uint32_t sb = sa + A_BYTES;
          if (bn == 64) mma_exact<64>(tmem, sa, sb, first_in_chunk, amn);
          else mma_exact<96>(tmem, sa, sb, first_in_chunk, amn);
          sm100::mma_commit(&empty[st2]);
        }
        npend = 0;
        if (last_in_chunk) {
          sm100::mma_commit(accf);
          ++gc;
          need_acce = true;   // the next chunk's exact MMAs wait for this chunk's drain
        }
        return true;
      };
      if constexpr (PACK) {
        using K_MAJOR = std::integral_constant<bool, false>;
        using MN_MAJOR = std::integral_constant<bool, true>;
        if (pack) {
          // packed-triangle A: the K-major stages (up to the diagonal block) and the MN-major
          // ones as two loops, each of one orientation; the first leaves nothing deferred
          const int isplit = min(nkb, max(0, kb_mn - cur.kb0));
          for (int i = 0; i < isplit && ok; ++i, ++gs) ok = stage(K_MAJOR(), i, i == isplit - 1);
          for (int i = isplit; i < nkb && ok; ++i, ++gs) ok = stage(MN_MAJOR(), i, false);
        } else if (amn_tile) {
          for (int i = 0; i < nkb && ok; ++i, ++gs) ok = stage(MN_MAJOR(), i, false);
        } else {
          for (int i = 0; i < nkb && ok; ++i, ++gs) ok = stage(K_MAJOR(), i, false);
        }
      } else {
        // the same per stage as `stage`, written out: one orientation for the whole tile
        const bool amn = AMN == 2 ? amn_tile : AMN == 1;
        for (int i = 0; i < nkb; ++i, ++gs) {
          const int st = (int)(gs % NSTAGE);
          if (!sm100::mbar_wait(&full[st], (uint32_t)(gs / NSTAGE) & 1, abort_flag, p.status,
                                LAS_ERR_TIMEOUT)) {
            ok = false;
            break;
          }
          sm100::tc_fence_after();
          {
            const uint32_t sa = sm100::smem_u32(smem + st * T::STAGE_BYTES);
            const uint32_t sb = sa + A_BYTES;
            if (bn == 64) mma_tail<64>(tmem + T::TAIL_COL, sa, sb, i == 0, amn);
            else mma_tail<96>(tmem + T::TAIL_COL, sa, sb, i == 0, amn);
          }
          const bool last_in_chunk = (i % CHUNK) == CHUNK - 1 || i == nkb - 1;
          if (need_acce) {
            if (!last_in_chunk && npend < NSTAGE - 1 &&
                !sm100::mbar_test_wait(acce, (uint32_t)(gc - 1) & 1)) {
              if (npend == 0) {
                pend0 = gs;
                pend_i0 = i;
              }
              ++npend;
              continue;   // defer this stage's exact-group MMAs
            }
            if (!sm100::mbar_wait(acce, (uint32_t)(gc - 1) & 1, abort_flag, p.status,
                                  LAS_ERR_TIMEOUT)) {
              ok = false;
              break;
            }
            sm100::tc_fence_after();
            need_acce = false;
          }
          if (npend == 0) {
            pend0 = gs;
            pend_i0 = i;
          }
          for (int j = 0; j <= npend; ++j) {
            const long g2 = pend0 + j;
            const int i2 = pend_i0 + j;
            const int st2 = (int)(g2 % NSTAGE);
            const bool first_in_chunk = (i2 % CHUNK) == 0;
            const uint32_t sa = sm100::smem_u32(smem + st2 * T::STAGE_BYTES);
            const uint32_t sb = sa + A_BYTES;
            if (bn == 64) mma_exact<64>(tmem, sa, sb, first_in_chunk, amn);
            else mma_exact<96>(tmem, sa, sb, first_in_chunk, amn);
            sm100::mma_commit(&empty[st2]);
          }
          npend = 0;
          if (last_in_chunk) {
            sm100::mma_commit(accf);
            ++gc;
            need_acce = true;
          }
        }
      }
      if (!ok) break;
      ++tcount;
    }
    // make sure no MMA is still writing TMEM when the CTA tears down
    sm100::mma_commit(drain);
    sm100::mbar_wait(drain, 0, abort_flag, status0, LAS_ERR_TIMEOUT);
  } else if (warp >= 2) {
    // ---------------- epilogue (16 warps) ----------------
    const int lq = warp & 3;                 // TMEM lane quarter this warp may access
    const int cg = (warp - 2) >> 2;          // column blocks cg, cg + 4, cg + 8, ... of 8
    const uint32_t tl = tmem + ((uint32_t)(lq * 32) << 16);
    long gc = 0;
    bool ok = true;
    OzCursor<GROUPED> cur;
    for (long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      cur.seek(t, p1, &tmA, &tmB, &tmA2, &tmA3, probs, nprob);
      const OzParams& p = *cur.P;
      const int m0 = cur.m0, n0 = cur.n0, kb0 = cur.kb0, nkb = cur.nkb;
      const int bn = FIXBN ? FIXBN : p.bn;
      const int nb = (bn / 8 - cg + 3) / 4;   // this warp's column blocks (warp-uniform)
      const float tscale = __int_as_float((127 + 8 * (NEXACT - 1) + p.sh) << 23);  // 2^(24+sh)
      const int nchunks = (nkb + CHUNK - 1) / CHUNK;
      unsigned long long acc[MAXB * 8];
#pragma unroll
      for (int j = 0; j < MAXB * 8; ++j) acc[j] = 0;
      for (int c = 0; c < nchunks; ++c, ++gc) {
        if (!sm100::mbar_wait(accf, (uint32_t)gc & 1, abort_flag, p.status, LAS_ERR_TIMEOUT,
                              256)) {
          ok = false;
          break;
        }
        sm100::tc_fence_after();
        const bool fin = (c == nchunks - 1);
        int extra = 0;
        if (fin) {
          // tail first, so that the next tile's tail MMAs can start:
          // acc <- acc * 2^sh + rint(tail * 2^(24+sh))  (int64, modulo 2^64)
#pragma unroll
          for (int b = 0; b < MAXB; ++b) {
            if (b < nb) {
              const uint32_t col = (uint32_t)((cg + 4 * b) * 8);
              uint32_t r[8];
              sm100::tmem_ld8(tl + T::TAIL_COL + col, r);
              sm100::tmem_wait_ld();
#pragma unroll
              for (int e = 0; e < 8; ++e)
                acc[b * 8 + e] =
                    (acc[b * 8 + e] << p.sh) +
                    (unsigned long long)__float2ll_rn(__uint_as_float(r[e]) * tscale);
            }
          }
          sm100::tc_fence_before();
          __syncwarp();
          if (lane == 0) sm100::mbar_arrive(accT);
          extra = p.sh;
        }
        // exact groups: integers g_q (|g_q| <= 2^24) in units of 2^-8q, merged as
        // V = ((g_0 2^8 + g_1) 2^8 + g_2) 2^8 + g_3 (the first step fits 32 bits)
        static_assert(NEXACT == 4, "the merge below is written for four exact groups");
#pragma unroll
        for (int b = 0; b < MAXB; ++b) {
          if (b < nb) {
            const uint32_t col = (uint32_t)((cg + 4 * b) * 8);
            uint32_t r[NEXACT][8];
#pragma unroll
            for (int q = 0; q < NEXACT; ++q) sm100::tmem_ld8(tl + q * bn + col, r[q]);
            sm100::tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int g0 = __float2int_rn(__uint_as_float(r[0][e]));
              const int g1 = __float2int_rn(__uint_as_float(r[1][e]) * 256.0f);
              const int g2 = __float2int_rn(__uint_as_float(r[2][e]) * 65536.0f);
              const int g3 = __float2int_rn(__uint_as_float(r[3][e]) * 16777216.0f);
              const long long v = (long long)(g0 * 256 + g1) * 65536 + (long long)g2 * 256 + g3;
              acc[b * 8 + e] += (unsigned long long)v << extra;
            }
          }
        }
        sm100::tc_fence_before();
        __syncwarp();
        if (lane == 0) sm100::mbar_arrive(acce);   // exact accumulators free from here on
      }
      if (!ok) break;
      // FP64 results (overlaps the next tile's MMAs)
      const int row = m0 + lq * 32 + lane;
      long L = 0, mu = 0;
      int ea;
      if constexpr (PACK) {
        if (p.mode == 1) {   // row (L, mu) of the Ht layout
          L = row / p.ht_rows;
          mu = p.ht_mu0 + (row - L * p.ht_rows);
        }
        ea = (p.ea && row < p.M) ? p.ea[p.ea_perL ? L : row] : 0;
      } else {
        ea = (p.ea && row < p.M) ? p.ea[row] : 0;
        if (p.mode == 1) {
          L = row / p.ht_n;
          mu = row - L * p.ht_n;
        }
      }
      const int z = kb0 / p.kb_per_split;
#pragma unroll
      for (int b = 0; b < MAXB; ++b) {
        if (b < nb) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int col = n0 + (cg + 4 * b) * 8 + e;
            if (row < p.M && col < p.N) {
              const int E = ea + p.eb[col] - 14 - 8 * (NEXACT - 1) - p.sh;
              const double v = make_double((long long)acc[b * 8 + e], E);
              if (p.mode == 0)
                p.out[(long)z * p.zstride + (long)row * p.ldc + col] = v;
              else
                p.out[(L * p.ht_op + col) * (long)p.ht_n + mu] = v;
            }
          }
        }
      }
    }
    sm100::tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    sm100::tc_fence_after();
    sm100::tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ------------------------------------------------------------------------------------------
// Digit extraction (integer operations on the FP64 bit patterns)
// ------------------------------------------------------------------------------------------
struct RowsStrided {  // element (r, k) = base[r*sr + k*sk] * 2^(gexp ? gexp[k] : 0)
  const double* base;
  long sr, sk;
  const int* gk;
  __device__ __forceinline__ double operator()(long r, long k) const {
    double x = base[r * sr + k * sk];
    if (gk) {
      long long b = __double_as_longlong(x);
      if ((b & 0x7FF0000000000000ll) != 0) b += ((long long)gk[k]) << 52;
      else if (x != 0.0) return ldexp(x, gk[k]);
      x = __longlong_as_double(b);
    }
    return x;
  }
};

// Row (L, u) of the active columns of the half transform, K = mu: Ht[(L op + c + u) n + mu]
struct RowsHtAct {
  const double* Ht;
  int n, op, c, a;
  __device__ __forceinline__ double operator()(long r, long k) const {
    const long L = r / a, u = r - L * a;
    return Ht[(L * op + c + u) * n + k];
  }
};

struct RowsPacked {   // element (r = L*n + mu, k = nu) of the packed symmetric b^L
  const double* Bp;
  long npair;
  int n;
  __device__ __forceinline__ double operator()(long r, long k) const {
    long L = r / n, mu = r - L * n;
    long hi = mu > k ? mu : k, lo = mu > k ? k : mu;
    return Bp[L * npair + hi * (hi + 1) / 2 + lo];
  }
};

// Six balanced base-256 digits of x * 2^-e rounded at 2^-47 (|x| < 2^e), returned as the BF16
// plane values d_s * 2^-8s.  Integer operations on the bit pattern only.
__device__ __forceinline__ void digits_of(double xv, int e, __nv_bfloat16 (&out)[NDIG]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(xv);
  const int bex = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  int ee = bex;
  if (bex != 0) m |= (1ull << 52); else ee = 1;
  // |x| * 2^(47 - e) = m * 2^(ee - 1075 + 47 - e), rounded to an integer below 2^47
  const int shift = ee - 1028 - e;
  unsigned long long y;
  if (shift >= 0) y = m << shift;
  else if (shift > -63) y = (m + (1ull << (-shift - 1))) >> (-shift);
  else y = 0;
  // balanced base-256 digits from the bottom, in 32-bit arithmetic on two 24-bit halves
  int lo = (int)(y & 0xFFFFFF), hi = (int)(y >> 24);
  if (b >> 63) {
    lo = -lo;
    hi = -hi;
  }
  int d[NDIG];
#pragma unroll
  for (int s = NDIG - 1; s >= 3; --s) {
    const int t = ((lo + 128) & 255) - 128;
    d[s] = t;
    lo = (lo - t) >> 8;
  }
  hi += lo;   // carry out of the low half (-1, 0 or 1)
#pragma unroll
  for (int s = 2; s >= 1; --s) {
    const int t = ((hi + 128) & 255) - 128;
    d[s] = t;
    hi = (hi - t) >> 8;
  }
  d[0] = hi;
  // d_s * 2^-8s as BF16 without conversion instructions: the float of d_s from the bit pattern
  // of 1.5*2^23 + d_s (exact for |d_s| < 2^22), scaled by a power of two, and its upper half
  // (exact: at most 8 significant bits)
#pragma unroll
  for (int s = 0; s < NDIG; ++s) {
    const float f = (__int_as_float(0x4B400000 + d[s]) - 12582912.0f) *
                    __int_as_float((127 - 8 * s) << 23);
    out[s] = __ushort_as_bfloat16((unsigned short)(__float_as_uint(f) >> 16));
  }
}

__device__ __forceinline__ int exp_of_maxbits(unsigned long long mx) {
  return mx ? (int)((mx >> 52) & 0x7FF) - 1022 : 0;   // max|x| < 2^e
}

__device__ __forceinline__ unsigned long long absbits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// Short rows: one warp per row r < rows (rows >= R are written as zeros); exponent e_r with
// max|x| < 2^e_r for r < R, digit planes for every k < kb*BK (zero beyond K).
template <class Acc>
__global__ void __launch_bounds__(256)
k_slice_rows(Acc acc, Planes P, long rows, long kb, int* ex) {
  const long r = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const bool live = r < P.R;
  unsigned long long mx = 0;
  if (live)
    for (long k = lane; k < P.K; k += 32) {
      const unsigned long long b = absbits(acc(r, k));
      mx = b > mx ? b : mx;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = v > mx ? v : mx;
  }
  const int e = exp_of_maxbits(mx);
  if (lane == 0 && live) ex[r] = e;
  const long kend = kb * BK;
  for (long k = lane; k < kend; k += 32) {
    __nv_bfloat16 d[NDIG];
    digits_of((live && k < P.K) ? acc(r, k) : 0.0, e, d);
#pragma unroll
    for (int s = 0; s < NDIG; ++s) P.p[P.idx(s, r, k)] = d[s];
  }
}

// Long rows, pass 1: mx[r] = max_k |x(r,k)| as ordered bit patterns (grid: segments x rows).
template <class Acc>
__global__ void __launch_bounds__(256)
k_rowmax_long(Acc acc, long K, long seg, unsigned long long* mx) {
  __shared__ unsigned long long red[8];
  const long r = blockIdx.y;
  const long k0 = (long)blockIdx.x * seg, k1 = min(K, k0 + seg);
  unsigned long long m = 0;
  for (long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const unsigned long long b = absbits(acc(r, k));
    m = b > m ? b : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
    if (m) atomicMax(&mx[r], m);
  }
}

// Long rows, pass 2: element-parallel digits over rows x kb*BK (zeros outside R x K).
template <class Acc>
__global__ void __launch_bounds__(256)
k_digits_long(Acc acc, Planes P, long rows, long kbc, const unsigned long long* mx, int* ex) {
  const long kend = kbc * BK;
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= rows * kend) return;
  // thread order follows the K-blocked output: (k block, row, k within the block)
  const long kb = i / (rows * BK), rem = i - kb * (rows * BK);
  const long r = rem / BK, k = kb * BK + (rem - r * BK);
  const bool live = r < P.R;
  const int e = live ? exp_of_maxbits(mx[r]) : 0;
  if (k == 0 && live) ex[r] = e;
  __nv_bfloat16 d[NDIG];
  digits_of((live && k < P.K) ? acc(r, k) : 0.0, e, d);
#pragma unroll
  for (int s = 0; s < NDIG; ++s) P.p[P.idx(s, r, k)] = d[s];
}

// Packed-triangle digit planes of B (see BPacked).  Pass 1: max |b^L| over the packed triangle
// of each L (one block per L) and its exponent.
__global__ void __launch_bounds__(256)
k_bpacked_max(const double* __restrict__ Bp, long npair, unsigned long long* __restrict__ mx,
              int* __restrict__ ex) {
  __shared__ unsigned long long red[8];
  const long L = blockIdx.x;
  const double* b = Bp + L * npair;
  unsigned long long m = 0;
  for (long k = threadIdx.x; k < npair; k += blockDim.x) {
    const unsigned long long v = absbits(b[k]);
    m = v > m ? v : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
    mx[L] = m;
    ex[L] = exp_of_maxbits(m);
  }
}

// Pass 2: the stored tiles, one thread per element in storage order (plane by plane: tile, K
// block of 16, row, column), digits relative to 2^e(L).
__global__ void __launch_bounds__(256)
k_bpacked_tiles(const double* __restrict__ Bp, long npair, int T, const int* __restrict__ ex,
                Planes P, long total) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int c = (int)(i & 15), row = (int)((i >> 4) & 127), kk = (int)((i >> 11) & 7);
  const long tt = i >> 14;              // tile index L T + t
  const long L = tt / T;
  const int t = (int)(tt - L * T);
  int I = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);   // t = I (I + 1) / 2 + J, J <= I
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  while (I * (I + 1) / 2 > t) --I;
  const int J = t - I * (I + 1) / 2;
  const long mu = 128L * I + row, nu = 128L * J + 16 * kk + c;
  const long hi = mu > nu ? mu : nu, lo = mu > nu ? nu : mu;
  __nv_bfloat16 d[NDIG];
  digits_of(Bp[L * npair + hi * (hi + 1) / 2 + lo], ex[L], d);
  const long o = (tt * 8 + kk) * (128L * BK) + row * BK + c;
#pragma unroll
  for (int s = 0; s < NDIG; ++s) P.p[s * P.plane + o] = d[s];
}

// Pass 3: the ragged rows mu = n1 + j (rows (L, j) of all X r, then zero padding rows), every
// K block of the layout (zero digits for nu >= n), in the K-blocked storage order.
__global__ void __launch_bounds__(256)
k_bpacked_ragged(const double* __restrict__ Bp, long npair, int n, int n1, int r,
                 const int* __restrict__ ex, Planes P, long live_rows) {
  const long kend = P.nkb * BK;
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= P.Rpad * kend) return;
  const long kb = i / (P.Rpad * BK), rem = i - kb * (P.Rpad * BK);
  const long row = rem / BK, k = kb * BK + (rem - row * BK);
  double x = 0.0;
  int e = 0;
  if (row < live_rows) {
    const long L = row / r, mu = n1 + (row - L * r);
    e = ex[L];
    if (k < n) {
      const long hi = mu > k ? mu : k, lo = mu > k ? k : mu;
      x = Bp[L * npair + hi * (hi + 1) / 2 + lo];
    }
  }
  __nv_bfloat16 d[NDIG];
  digits_of(x, e, d);
#pragma unroll
  for (int s = 0; s < NDIG; ++s) P.p[P.idx(s, row, k)] = d[s];
}

// Half-transformed rows (L,p) of Ht [R][n]: exponents and digit planes Hd (rows (L,p),
// K = mu); the full transform reads them K-major and the projection MN-major (rows mu, K =
// (L,p)), so one layout serves both.  Block: 16 rows r, 256 threads.  The row maxima are read
// first (warp per row); the digit pass then re-reads the block's rows: thread (r, c) cuts 8
// consecutive columns of row r per 128-column step (a warp's 16-byte stores into Hd cover 512
// contiguous bytes).  Rows of Hd beyond R and columns k >= n are written as zero digits within the
// block's K range; rows beyond the blocks stay zero from set-up.
__global__ void __launch_bounds__(256)
k_slice_ht(const double* __restrict__ Ht, long R, int n, Planes Hd, int* __restrict__ ex) {
  __shared__ int es[16];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long r0 = (long)blockIdx.x * 16;
  for (int i = 0; i < 2; ++i) {
    const int row = warp * 2 + i;
    const long r = r0 + row;
    unsigned long long mx = 0;
    if (r < R)
      for (int k = lane; k < n; k += 32) {
        const unsigned long long b = absbits(Ht[r * n + k]);
        mx = b > mx ? b : mx;
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = v > mx ? v : mx;
    }
    if (lane == 0) {
      es[row] = exp_of_maxbits(mx);
      if (r < R) ex[r] = es[row];
    }
  }
  __syncthreads();
  const long kend = Hd.nkb * BK;            // a multiple of 16
  const int rr = threadIdx.x & 15, kc = threadIdx.x >> 4;   // digit pass: row, 8-column group
  const long r = r0 + rr;
  if (r >= Hd.Rpad) return;
  const bool live = r < R;
  const int e = es[rr];
  const double* hrow = Ht + r * n;
  for (long k0 = 0; k0 < kend; k0 += 128) {
    const long k = k0 + kc * 8;
    if (k >= kend) break;
    double x[8];
    if (live && (n & 1) == 0 && k + 8 <= n) {
      // 16-byte loads (rows start 16-byte aligned when n is even)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const double2 t = *(const double2*)(hrow + k + 2 * j);
        x[2 * j] = t.x;
        x[2 * j + 1] = t.y;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = (live && k + j < n) ? hrow[k + j] : 0.0;
    }
    __nv_bfloat16 d[8][NDIG];
#pragma unroll
    for (int j = 0; j < 8; ++j) digits_of(x[j], e, d[j]);
#pragma unroll
    for (int s = 0; s < NDIG; ++s) {
      uint4 v;
      __nv_bfloat16* pv = (__nv_bfloat16*)&v;
#pragma unroll
      for (int j = 0; j < 8; ++j) pv[j] = d[j][s];
      *(uint4*)(Hd.p + Hd.idx(s, r, k)) = v;
    }
  }
}

// Column maxima of Ht [R][n] over its rows (coalesced along the columns): mx[mu] (atomic max of
// |x| bit patterns).  Grid: (ceil(n/256), row segments).
__global__ void __launch_bounds__(256)
k_colmax(const double* __restrict__ Ht, long R, int n, long seg, unsigned long long* mx) {
  const int mu = blockIdx.x * 256 + threadIdx.x;
  if (mu >= n) return;
  const long r0 = (long)blockIdx.y * seg, r1 = min(R, r0 + seg);
  unsigned long long m = 0;
  for (long r = r0; r < r1; ++r) {
    const unsigned long long b = absbits(Ht[r * n + mu]);
    m = b > m ? b : m;
  }
  if (m) atomicMax(&mx[mu], m);
}

// Digits of H^T scaled per row mu (exponents from the column maxima): HdT[s](mu, k) for the
// rows k = (L,p) of Ht, transposed through shared memory.  Block: 32 rows k x the columns
// [blockIdx.y*COLS_PER_BLOCK, ...) of mu.
constexpr int COLS_PER_BLOCK = 2048;
__global__ void __launch_bounds__(256)
k_slice_ht_cols(const double* __restrict__ Ht, long R, int n, const unsigned long long* mx,
                Planes HdT, int* __restrict__ ex) {
  __shared__ __nv_bfloat16 tile[NDIG][32][34];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long r0 = (long)blockIdx.x * 32;
  const int c0 = blockIdx.y * COLS_PER_BLOCK, c1 = min(n, c0 + COLS_PER_BLOCK);
  if (blockIdx.x == 0)
    for (int mu = c0 + threadIdx.x; mu < c1; mu += 256) ex[mu] = exp_of_maxbits(mx[mu]);
  for (int k0 = c0; k0 < c1; k0 += 32) {
    const int mu = k0 + lane;
    const int e = mu < c1 ? exp_of_maxbits(mx[mu]) : 0;
    for (int i = 0; i < 4; ++i) {
      const int row = warp + 8 * i;
      const long r = r0 + row;
      __nv_bfloat16 d[NDIG];
      digits_of((r < R && mu < c1) ? Ht[r * n + mu] : 0.0, e, d);
#pragma unroll
      for (int s = 0; s < NDIG; ++s) tile[s][row][lane] = d[s];
    }
    __syncthreads();
    for (int i = 0; i < 4; ++i) {
      const int kk = warp * 4 + i;
      const int m2 = k0 + kk;
      const long r = r0 + lane;
      if (m2 < c1 && r < HdT.nkb * BK) {
#pragma unroll
        for (int s = 0; s < NDIG; ++s) HdT.p[HdT.idx(s, m2, r)] = tile[s][lane][kk];
      }
    }
    __syncthreads();
  }
}

}  // namespace lasdf_split

using namespace lasdf_split;

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 3D map over K-blocked digit planes: dims {BK, nkb*Rpad, NDIG}, box {BK, box_rows, NDIG},
// 32-byte swizzle.  Each box is box_rows * 32 contiguous bytes per plane.
static las_status make_plane_map(CUtensorMap* m, const Planes& P, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return LAS_ERR_CUDA;
  const long rows = P.nkb * P.Rpad;
  if (((uintptr_t)P.p & 15) || rows <= 0 || rows > 0x7FFFFFFFL) return LAS_ERR_INTERNAL;
  cuuint64_t dims[3] = {(cuuint64_t)BK, (cuuint64_t)rows, (cuuint64_t)NDIG};
  cuuint64_t strides[2] = {(cuuint64_t)BK * 2, (cuuint64_t)P.plane * 2};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, (cuuint32_t)NDIG};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)P.p, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? LAS_OK : LAS_ERR_INTERNAL;
}

// 4D map for reading planes MN-major (as the A operand of a product whose K runs along the
// stored rows): dims {BK, Rpad, nkb, NDIG}; a box is 16 stored rows (16 values of K) of BM / BK
// consecutive K blocks of the stored layout (BM values of M), every plane: BM * 32 bytes per
// plane, as in the K-major case.  Boxes past the last stored K block read the TMA's zero fill.
static las_status make_plane_map_mn(CUtensorMap* m, const Planes& P) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return LAS_ERR_CUDA;
  if (((uintptr_t)P.p & 15) || P.Rpad <= 0 || P.Rpad > 0x7FFFFFFFL || P.nkb <= 0)
    return LAS_ERR_INTERNAL;
  cuuint64_t dims[4] = {(cuuint64_t)BK, (cuuint64_t)P.Rpad, (cuuint64_t)P.nkb, (cuuint64_t)NDIG};
  cuuint64_t strides[3] = {(cuuint64_t)BK * 2, (cuuint64_t)P.Rpad * BK * 2,
                           (cuuint64_t)P.plane * 2};
  cuuint32_t box[4] = {(cuuint32_t)BK, (cuuint32_t)BK, (cuuint32_t)(BM / BK), (cuuint32_t)NDIG};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)P.p, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? LAS_OK : LAS_ERR_INTERNAL;
}

// Widest tile (the stage layout's B region) and the default tile width of a product: 96
// columns, so that the four exact accumulators and the tail take 480 of the 512 TMEM columns.
// A product may run with 64-column tiles instead (las_autotune chooses per product kind).
constexpr int OZ_BN = 96;
static bool valid_bn(int bn) { return bn == 64 || bn == 96; }

// The launch attribute is a per-device setting: set once for each device that uses the kernels
// (a repeated set from two threads is harmless).
template <bool GROUPED, int FIXBN>
static cudaError_t ozaki_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_ozaki<OZ_BN, GROUPED, FIXBN, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       OzTile<OZ_BN>::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  if constexpr (!GROUPED && FIXBN != 0) {
    e = cudaFuncSetAttribute(k_ozaki<OZ_BN, GROUPED, FIXBN, false, 0>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, OzTile<OZ_BN>::SMEM_BYTES);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_ozaki<OZ_BN, GROUPED, FIXBN, false, 1>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               OzTile<OZ_BN>::SMEM_BYTES);
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(k_ozaki<OZ_BN, GROUPED, FIXBN, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              OzTile<OZ_BN>::SMEM_BYTES);
}

// Does the product need the instantiation with the packed-triangle logic (its A is the packed
// form, or its rows are the ragged rows of that form, with one exponent per auxiliary index)?
static inline bool needs_pack(const OzParams& p) { return p.a_pack || p.ea_perL; }

static las_status ozaki_prepare() {
  static volatile int done[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LAS_ERR_CUDA;
  if (done[dev]) return LAS_OK;
  cudaError_t e = ozaki_attr<false, 96>();
  if (e == cudaSuccess) e = ozaki_attr<false, 64>();
  if (e == cudaSuccess) e = ozaki_attr<true, 96>();
  if (e == cudaSuccess) e = ozaki_attr<true, 64>();
  if (e == cudaSuccess) e = ozaki_attr<true, 0>();
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "cudaFuncSetAttribute(k_ozaki)", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  done[dev] = 1;
  return LAS_OK;
}

static inline long rup(long x, long m) { return (x + m - 1) / m * m; }

static int num_sms() {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
      nsm = 148;
  }
  return nsm;
}


// out = A * B^T over K: rows [a_row0, a_row0 + M) of A (row exponents ea, or 0 when null),
// rows [b_row0, b_row0 + N) of B (row exponents eb: the column exponents of the product).
// mode 0: out[z*zstride + r*ldc + c] (z = K split); mode 1: Ht layout (rows (L, mu)).
// Output tiles of an M x N product per K split (lower: only those touching the lower triangle).
static long ozaki_tiles(long M, long N, int lower, int bn = OZ_BN) {
  const long ntm = (M + BM - 1) / BM, ntn = (N + bn - 1) / bn;
  if (!lower) return ntm * ntn;
  long t = 0;
  for (long i = 0; i < ntm; ++i) t += lower_tiles_in_row((int)i, (int)ntn, bn);
  return t;
}

// K-split factor in [1, cap] that shares `tiles` output tiles of a product with kb K blocks out
// most evenly over the persistent CTAs: ceil(tiles*ks / SMs) rounds, each of ceil(kb/ks) blocks
// plus about two chunks of pipeline fill and drain.
static int balanced_ksplit(long tiles, long kb, long cap) {
  const long sms = num_sms();
  int best = 1;
  double best_t = 1e300;
  for (long ks = 1; ks <= cap; ++ks) {
    const double t = (double)((tiles * ks + sms - 1) / sms) * (double)((kb + ks - 1) / ks + 2 * CHUNK);
    if (t < best_t * (1.0 - 1e-9)) {
      best_t = t;
      best = (int)ks;
    }
  }
  return best;
}

// Products recorded instead of launched while a group is being recorded on this host thread.
struct OzGroup {
  std::vector<OzProblem> probs;
  long tiles = 0;
};
static thread_local OzGroup* g_record = nullptr;

OzGroup* ozgroup_new() { return new OzGroup(); }
void ozgroup_free(OzGroup* g) { delete g; }
void ozgroup_record(OzGroup* g) { g_record = g; }
size_t ozgroup_count(const OzGroup* g) { return g ? g->probs.size() : 0; }
size_t ozgroup_bytes(size_t nprob) { return nprob * sizeof(OzProblem); }

// One persistent launch over every recorded product (tiles concatenated in recording order);
// `dev` is device memory for the product descriptions, filled by ozgroup_upload before the
// launch runs (the launch may be captured into a graph first).
las_status ozgroup_launch(const OzGroup* g, void* dev, cudaStream_t st) {
  if (!g || g->probs.empty()) return LAS_OK;
  if (!dev || ((uintptr_t)dev % alignof(OzProblem))) return LAS_ERR_INTERNAL;
  OzParams dummy;
  memset(&dummy, 0, sizeof(dummy));
  CUtensorMap m0;
  memset(&m0, 0, sizeof(m0));
  dim3 grid((unsigned)std::min<long>(g->tiles, num_sms()), 1, 1);
  int bn = g->probs[0].p.bn;   // one width for the whole launch, or 0: read per product
  for (const OzProblem& pr : g->probs)
    if (pr.p.bn != bn) bn = 0;
  bool pack = false;
  for (const OzProblem& pr : g->probs) pack |= needs_pack(pr.p);
  const OzProblem* probs = (const OzProblem*)dev;
  const int np = (int)g->probs.size();
  constexpr int SM = OzTile<OZ_BN>::SMEM_BYTES;
  auto go = [&](auto kern) {
    kern<<<grid, NTHREADS, SM, st>>>(m0, m0, m0, m0, dummy, probs, np, g->tiles);
  };
  if (bn == 96) pack ? go(k_ozaki<OZ_BN, true, 96, true>) : go(k_ozaki<OZ_BN, true, 96, false>);
  else if (bn == 64) pack ? go(k_ozaki<OZ_BN, true, 64, true>) : go(k_ozaki<OZ_BN, true, 64, false>);
  else pack ? go(k_ozaki<OZ_BN, true, 0, true>) : go(k_ozaki<OZ_BN, true, 0, false>);
  las_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "k_ozaki grouped launch", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  return LAS_OK;
}

las_status ozgroup_upload(const OzGroup* g, void* dev) {
  if (!g || g->probs.empty()) return LAS_OK;
  LAS_CUDA_TRY(cudaMemcpy(dev, g->probs.data(), g->probs.size() * sizeof(OzProblem),
                          cudaMemcpyHostToDevice));
  return LAS_OK;
}

// Launch one product (persistent: one CTA per SM), or record it into the group being recorded.
static las_status ozaki_submit(OzProblem& pr, cudaStream_t st) {
  const OzParams& p = pr.p;
  const long tiles = p.tiles_z * p.ksplit;
  if (g_record) {   // part of a grouped launch
    pr.tile0 = g_record->tiles;
    g_record->tiles += tiles;
    g_record->probs.push_back(pr);
    return LAS_OK;
  }
  dim3 grid((unsigned)std::min<long>(tiles, num_sms()), 1, 1);
  constexpr int SM = OzTile<OZ_BN>::SMEM_BYTES;
  auto go = [&](auto kern) {
    kern<<<grid, NTHREADS, SM, st>>>(pr.tmA, pr.tmB, pr.tmA2, pr.tmA3, p, nullptr, 0, tiles);
  };
  const bool pack = needs_pack(p);
  // full-row products take an instantiation with their A orientation as a compile-time constant
  if (pack) {
    if (p.bn == 64) go(k_ozaki<OZ_BN, false, 64, true>);
    else go(k_ozaki<OZ_BN, false, 96, true>);
  } else if (p.a_mn) {
    if (p.bn == 64) go(k_ozaki<OZ_BN, false, 64, false, 1>);
    else go(k_ozaki<OZ_BN, false, 96, false, 1>);
  } else {
    if (p.bn == 64) go(k_ozaki<OZ_BN, false, 64, false, 0>);
    else go(k_ozaki<OZ_BN, false, 96, false, 0>);
  }
  las_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "k_ozaki launch", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  return LAS_OK;
}

// Fractional bits kept for the tail: |fixed-point sum| < 2^38 * (k per CTA) must fit 62 bits.
static int tail_shift(int kb_per_split) {
  int lgk = 0;
  while ((1L << lgk) < (long)kb_per_split * BK) ++lgk;
  return std::max(0, std::min(20, 61 - 14 - 8 * (NEXACT - 1) - lgk));
}

// The product's description (tensor maps and parameters), ready to be launched or recorded.
static las_status ozaki_setup(OzProblem& pr, const Planes& A, long a_row0, const int* ea, long M,
                              const Planes& B, long b_row0, const int* eb, long N, long K,
                              int ksplit, int mode, double* out, long ldc, long zstride, int ht_n,
                              int ht_op, int* status, int lower, int bn, int a_mn) {
  // a_mn: A's stored rows [a_row0, a_row0 + K) are the product's K, its stored K the rows M
  const bool a_ok = a_mn ? (a_row0 + K <= A.Rpad && M <= A.nkb * BK)
                         : (a_row0 + M <= A.Rpad && K <= A.nkb * BK);
  if (!a_ok || b_row0 + N > B.Rpad || K > B.nkb * BK || !valid_bn(bn) || (a_mn && lower))
    return LAS_ERR_INTERNAL;
  las_status s = ozaki_prepare();
  if (s != LAS_OK) return s;
  memset(&pr, 0, sizeof(pr));
  if ((s = a_mn ? make_plane_map_mn(&pr.tmA, A) : make_plane_map(&pr.tmA, A, BM)) != LAS_OK)
    return s;
  if ((s = make_plane_map(&pr.tmB, B, bn)) != LAS_OK) return s;
  OzParams& p = pr.p;
  p.M = (int)M;
  p.N = (int)N;
  p.a_rpad = (int)A.Rpad;
  p.b_rpad = (int)B.Rpad;
  p.a_row0 = (int)a_row0;
  p.b_row0 = (int)b_row0;
  p.kb_total = (int)((K + BK - 1) / BK);
  if (p.kb_total < 1) p.kb_total = 1;
  if (ksplit < 1) ksplit = 1;
  p.kb_per_split = (p.kb_total + ksplit - 1) / ksplit;
  ksplit = (p.kb_total + p.kb_per_split - 1) / p.kb_per_split;
  p.ksplit = ksplit;
  p.ea = ea;
  p.eb = eb;
  p.out = out;
  p.mode = mode;
  p.ldc = ldc;
  p.zstride = zstride;
  p.ht_n = ht_n;
  p.ht_op = ht_op;
  p.ht_rows = ht_n;
  p.ht_mu0 = 0;
  p.lower = lower;
  p.tiles_z = ozaki_tiles(M, N, lower, bn);
  p.sh = tail_shift(p.kb_per_split);
  p.bn = bn;
  p.a_mn = a_mn;
  p.status = status;
  return LAS_OK;
}

las_status ozaki_gemm(const Planes& A, long a_row0, const int* ea, long M, const Planes& B,
                      long b_row0, const int* eb, long N, long K, int ksplit, int mode,
                      double* out, long ldc, long zstride, int ht_n, int ht_op, int* status,
                      cudaStream_t st, int lower = 0, int bn = OZ_BN, int a_mn = 0) {
  if (M <= 0 || N <= 0) return LAS_OK;
  OzProblem pr;
  las_status s = ozaki_setup(pr, A, a_row0, ea, M, B, b_row0, eb, N, K, ksplit, mode, out, ldc,
                             zstride, ht_n, ht_op, status, lower, bn, a_mn);
  return s == LAS_OK ? ozaki_submit(pr, st) : s;
}

// out[L][p][mu] (the Ht layout, ht_op columns per L) = sum_nu b^L(mu, nu) X(nu, p) for the
// auxiliary rows [l0, l0 + nL) of packed-triangle B and the N columns p of X whose digit planes
// (rows p, K = nu) start at row x_row0 of Xd (column exponents xexp).  Two products: the full
// 128-row blocks of every b^L from the stored tiles, and the ragged rows mu >= n1.
static las_status bpacked_half(const BPacked& b, int l0, int nL, const Planes& Xd, long x_row0,
                               const int* xexp, long N, double* out, int ht_op, int* status,
                               cudaStream_t st, int bn) {
  if (nL <= 0 || N <= 0) return LAS_OK;
  if (l0 < 0 || l0 + nL > b.X || x_row0 + N > Xd.Rpad || b.n > Xd.nkb * BK || !valid_bn(bn))
    return LAS_ERR_INTERNAL;
  las_status rc = ozaki_prepare();
  if (rc != LAS_OK) return rc;
  if (b.nb1 > 0) {
    const long M = (long)nL * b.n1;
    if (M > 0x7FFFFFFFL) return LAS_ERR_UNSUPPORTED;
    OzProblem pr;
    memset(&pr, 0, sizeof(pr));
    if ((rc = make_plane_map(&pr.tmA, b.tiles, BM)) != LAS_OK) return rc;
    if ((rc = make_plane_map_mn(&pr.tmA2, b.tiles)) != LAS_OK) return rc;
    if (b.r > 0 && (rc = make_plane_map_mn(&pr.tmA3, b.rag)) != LAS_OK) return rc;
    if ((rc = make_plane_map(&pr.tmB, Xd, bn)) != LAS_OK) return rc;
    OzParams& p = pr.p;
    p.M = (int)M;
    p.N = (int)N;
    p.a_rpad = BM;
    p.b_rpad = (int)Xd.Rpad;
    p.b_row0 = (int)x_row0;
    p.kb_total = (b.n + BK - 1) / BK;
    p.kb_per_split = p.kb_total;
    p.ksplit = 1;
    p.ea = b.exp + l0;
    p.eb = xexp;
    p.out = out;
    p.mode = 1;
    p.ht_n = b.n;
    p.ht_op = ht_op;
    p.ht_rows = b.n1;
    p.ht_mu0 = 0;
    p.ea_perL = 1;
    p.tiles_z = ozaki_tiles(M, N, 0, bn);
    p.sh = tail_shift(p.kb_per_split);
    p.bn = bn;
    p.a_pack = 1;
    p.pk_nb1 = b.nb1;
    p.pk_T = b.T;
    p.pk_r = b.r;
    p.pk_L0 = l0;
    p.status = status;
    if ((rc = ozaki_submit(pr, st)) != LAS_OK) return rc;
  }
  if (b.r > 0) {
    OzProblem pr;
    rc = ozaki_setup(pr, b.rag, (long)l0 * b.r, b.exp + l0, (long)nL * b.r, Xd, x_row0, xexp, N,
                     b.n, 1, 1, out, 0, 0, b.n, ht_op, status, 0, bn, 0);
    if (rc != LAS_OK) return rc;
    pr.p.ht_rows = b.r;
    pr.p.ht_mu0 = b.n1;
    pr.p.ea_perL = 1;
    rc = ozaki_submit(pr, st);
  }
  return rc;
}

// live_only: only rows < R and the K blocks that hold K are written (planes whose padding rows
// were zeroed at set-up); otherwise every padded row and K block of the layout is written.
template <class Acc>
static las_status slice_rows(Acc acc, const Planes& P, int* ex, cudaStream_t st,
                             unsigned long long* mx_ws = nullptr, bool live_only = false) {
  if (P.R <= 0) return LAS_OK;
  const long rows = live_only ? P.R : P.Rpad;
  const long kbc = live_only ? std::min(P.nkb, planes_nkb(P.K)) : P.nkb;
  if (P.K > 8192 && mx_ws && P.R <= 65535) {
    // long rows: block-parallel maxima, then element-parallel digits
    cudaError_t e0 = cudaMemsetAsync(mx_ws, 0, P.R * sizeof(unsigned long long), st);
    if (e0 != cudaSuccess) {
      las_record_cuda_error(e0, "cudaMemsetAsync(rowmax)", __FILE__, __LINE__);
      return LAS_ERR_CUDA;
    }
    const long seg = 8192;
    dim3 g1((unsigned)((P.K + seg - 1) / seg), (unsigned)P.R);
    k_rowmax_long<Acc><<<g1, 256, 0, st>>>(acc, P.K, seg, mx_ws);
    las_count_launch();
    const long tot = rows * kbc * BK;
    k_digits_long<Acc><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(acc, P, rows, kbc, mx_ws,
                                                                       ex);
    las_count_launch();
  } else {
    const long threads = rows * 32;
    k_slice_rows<Acc><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(acc, P, rows, kbc, ex);
    las_count_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "k_slice_rows launch", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  return LAS_OK;
}

struct SplitState {
  int n, X, op, Lc;
  int packed;            // layout of the Cholesky vectors' digit planes:
  Planes Bdig;           //   0: full rows (L, mu) of all X*n, K = nu, exponent per row
  int* Bexp;             //      [X*n]
  BPacked Bpk;           //   1: packed-triangle tiles, exponent per L
  Planes Cdig;           // rows p of C_occ^T, K = nu
  int* Cexp;             // [op]
  Planes Hdig;           // rows (L, p) of a chunk, K = mu
  int* Hexp;             // [Lc*op]
  Planes HdigT;          // rows mu, K = (L, p)
  Planes Wdig;           // rows q, K = (L, p)
  int* Wexp;             // [op]
  double* part;          // [ksplit][n][op]
  unsigned long long* mx;  // [op + n] row maxima for long-row slicing
  Planes Mpd;            // rows p of C[:, p0:p1]^T (K = mu) for the (L|pu) transform (lazy)
  int* Mpexp;
  void* Mpblob;
  Planes hdig;           // rows mu of h, K = nu
  int* hexp;             // [n]
  Planes hcdig;          // rows q of (h C_occ)^T, K = mu
  int* hcexp;            // [op]
  int ksplit6;           // partial buffers allocated for this many K splits
  int ks;                // split-K factor of the projection GEMM (autotunable)
  int bn[SPLIT_NKIND];   // tile width of each product kind (autotunable): 64 or 96
  // tangent (Hessian-vector) scratch, allocated by the first split_tangent_prepare: digit planes
  // of dC_occ^T (rows p, K = nu) and of the chunk's dH (rows (L, p), K = mu)
  Planes dCdig;
  int* dCexp;
  Planes dHdig;
  int* dHexp;
  void* tblob;
  int* status;
};

static void split_free(SplitState* s) {
  if (s->Mpblob) cudaFree(s->Mpblob);
  if (s->tblob) cudaFree(s->tblob);
  void* ptrs[] = {s->Bdig.p, s->Bexp, s->Bpk.tiles.p, s->Bpk.rag.p, s->Bpk.exp, s->Bpk.mx,
                  s->Cdig.p, s->Cexp,
                  s->Hdig.p, s->Hexp, s->HdigT.p,
                  s->Wdig.p, s->Wexp, s->part, s->mx, s->hdig.p, s->hexp, s->hcdig.p, s->hcexp};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

size_t split_bytes_per_aux(int n, int op) {
  // Hdig + HdigT + Wdig per auxiliary index (K-blocked, padded), plus exponents
  return (size_t)NDIG * op * rup(n, BK) * 2 * 2 + (size_t)NDIG * ROWPAD * op * 2 + (size_t)op * 4;
}

las_status split_create(SplitState** out, int n, int X, int op, int Lc, const double* Bp,
                        int packed, int* status, cudaStream_t st, size_t* bytes) {
  *out = nullptr;
  if (!encode_fn()) return LAS_ERR_UNSUPPORTED;
  SplitState* s = (SplitState*)calloc(1, sizeof(SplitState));
  if (!s) return LAS_ERR_INTERNAL;
  s->n = n;
  s->X = X;
  s->op = op;
  s->Lc = Lc;
  s->status = status;
  s->ksplit6 = 64;
  for (int k = 0; k < SPLIT_NKIND; ++k) s->bn[k] = OZ_BN;
  // one-time launch attributes, so that later calls can be captured into CUDA graphs
  if (ozaki_prepare() != LAS_OK || num_sms() <= 0) {
    free(s);
    return LAS_ERR_CUDA;
  }
  // projection split-K (autotunable): output n x op, K = the (L, p) rows of one chunk
  s->ks = balanced_ksplit(ozaki_tiles(n, op, 0), ((long)Lc * op + BK - 1) / BK,
                          std::min<long>(s->ksplit6, std::max(1L, ((long)Lc * op) / 2048)));
  size_t total = 0;
  las_status rc = LAS_OK;
  auto A = [&](void** p, size_t b) {
    if (rc != LAS_OK) return;
    if (cudaMalloc(p, b) != cudaSuccess) {
      *p = nullptr;
      rc = LAS_ERR_CUDA;
      las_record_cuda_error(cudaErrorMemoryAllocation, "cudaMalloc(split)", __FILE__, __LINE__);
      return;
    }
    total += b;
  };
  const long R = (long)Lc * op;
  void* q = nullptr;
  s->packed = packed != 0;
  BPacked& bp = s->Bpk;
  bp = bpacked_geometry(n, X);
  if (!s->packed) {
    A(&q, planes_bytes((long)X * n, n));
    s->Bdig = make_planes(q, (long)X * n, n);
    q = nullptr;
    A((void**)&s->Bexp, (size_t)X * n * 4);
  } else {
  if (bp.nb1 > 0) {
    A(&q, bpacked_tile_bytes(bp));
    bp.tiles.p = (__nv_bfloat16*)q;
    bp.tiles.R = bp.tiles.Rpad = 128;
    bp.tiles.nkb = 8L * X * bp.T;
    bp.tiles.K = bp.tiles.nkb * BK;
    bp.tiles.plane = bp.tiles.nkb * 128 * BK;
    q = nullptr;
  }
  if (bp.r > 0) {
    A(&q, planes_bytes((long)X * bp.r, n));
    bp.rag = make_planes(q, (long)X * bp.r, n);
    q = nullptr;
  }
  A((void**)&bp.exp, (size_t)X * 4);
  A((void**)&bp.mx, (size_t)X * 8);
  }
  A(&q, planes_bytes(op, n));        s->Cdig = make_planes(q, op, n);   q = nullptr;
  A((void**)&s->Cexp, (size_t)op * 4);
  A(&q, planes_bytes(R, n));         s->Hdig = make_planes(q, R, n);    q = nullptr;
  A((void**)&s->Hexp, (size_t)R * 4);
  A(&q, planes_bytes(n, R));         s->HdigT = make_planes(q, n, R);   q = nullptr;
  A(&q, planes_bytes(op, R));        s->Wdig = make_planes(q, op, R);   q = nullptr;
  A((void**)&s->Wexp, (size_t)op * 4);
  A((void**)&s->part, (size_t)s->ksplit6 * n * op * 8);
  A((void**)&s->mx, (size_t)(op + n) * 8);
  A(&q, planes_bytes(n, n));         s->hdig = make_planes(q, n, n);    q = nullptr;
  A((void**)&s->hexp, (size_t)n * 4);
  A(&q, planes_bytes(op, n));        s->hcdig = make_planes(q, op, n);  q = nullptr;
  A((void**)&s->hcexp, (size_t)op * 4);
  // rows mu >= n of the transposed planes and the padding rows of C, W, h and (h C)^T are never
  // written by the per-evaluation slicers: make them zero once
  const struct { void* p; size_t b; } zero[] = {
      {s->HdigT.p, planes_bytes(n, R)}, {s->Wdig.p, planes_bytes(op, R)},
      {s->Cdig.p, planes_bytes(op, n)}, {s->hdig.p, planes_bytes(n, n)},
      {s->hcdig.p, planes_bytes(op, n)}};
  for (const auto& z : zero) {
    if (rc != LAS_OK) break;
    cudaError_t e = cudaMemsetAsync(z.p, 0, z.b, st);
    if (e != cudaSuccess) {
      las_record_cuda_error(e, "cudaMemsetAsync(split planes)", __FILE__, __LINE__);
      rc = LAS_ERR_CUDA;
    }
  }
  if (rc == LAS_OK && !s->packed) {
    // one-time digit planes of the Cholesky vectors: rows (L, mu), K = nu
    RowsPacked acc{Bp, (long)n * (n + 1) / 2, n};
    rc = slice_rows(acc, s->Bdig, s->Bexp, st);
  } else if (rc == LAS_OK) {
    // one-time packed-triangle digit planes of the Cholesky vectors, one exponent per L
    const long npair = (long)n * (n + 1) / 2;
    k_bpacked_max<<<(unsigned)X, 256, 0, st>>>(Bp, npair, bp.mx, bp.exp);
    las_count_launch();
    if (bp.nb1 > 0) {
      const long total = 8L * X * bp.T * 128 * BK;
      k_bpacked_tiles<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Bp, npair, bp.T, bp.exp,
                                                                        bp.tiles, total);
      las_count_launch();
    }
    if (bp.r > 0) {
      const long total = bp.rag.Rpad * bp.rag.nkb * BK;
      k_bpacked_ragged<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
          Bp, npair, n, bp.n1, bp.r, bp.exp, bp.rag, (long)X * bp.r);
      las_count_launch();
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      las_record_cuda_error(e, "packed digit planes of B", __FILE__, __LINE__);
      rc = LAS_ERR_CUDA;
    }
  }
  if (rc != LAS_OK) {
    split_free(s);
    free(s);
    return rc;
  }
  *bytes += total;
  *out = s;
  return LAS_OK;
}

void split_destroy(SplitState* s) {
  if (!s) return;
  split_free(s);
  free(s);
}

const int* split_hexp(SplitState* s) { return s->Hexp; }

int split_get_ksplit(SplitState* s) { return s->ks; }
int split_balanced_ksplit(SplitState* s, int nL) {
  return balanced_ksplit(ozaki_tiles(s->n, s->op, 0, s->bn[SPLIT_PROJECT]),
                         ((long)nL * s->op + BK - 1) / BK,
                         std::min<long>(s->ksplit6, std::max(1L, ((long)nL * s->op) / 2048)));
}
int split_get_tile(SplitState* s, int kind) { return s->bn[kind]; }
las_status split_set_tile(SplitState* s, int kind, int bn) {
  if (kind < 0 || kind >= SPLIT_NKIND || !valid_bn(bn)) return LAS_ERR_ARG;
  s->bn[kind] = bn;
  return LAS_OK;
}
void split_set_ksplit(SplitState* s, int ks) { s->ks = std::max(1, std::min(ks, s->ksplit6)); }

// The half-transform-shaped products of the Cholesky vectors, in either digit layout:
// out[L][p][mu] (ht_op columns per L) = sum_nu b^L(mu, nu) X(nu, p) for L in [l0, l0 + nL), X
// given by the digit planes of its transpose (rows p from x_row0, K = nu; exponents xexp).
static las_status b_half(const SplitState* s, int l0, int nL, const Planes& Xd, long x_row0,
                         const int* xexp, long N, double* out, int ht_op, cudaStream_t st,
                         int bn) {
  if (s->packed)
    return bpacked_half(s->Bpk, l0, nL, Xd, x_row0, xexp, N, out, ht_op, s->status, st, bn);
  return ozaki_gemm(s->Bdig, (long)l0 * s->n, s->Bexp + (long)l0 * s->n, (long)nL * s->n, Xd,
                    x_row0, xexp, N, s->n, 1, 1, out, 0, 0, s->n, ht_op, s->status, st, 0, bn);
}

las_status split_prepare_C(SplitState* s, const double* Cocc, cudaStream_t st) {
  // rows p of C_occ^T (K = nu): element (p, nu) = Cocc[nu*op + p]
  RowsStrided acc{Cocc, 1, s->op, nullptr};
  return slice_rows(acc, s->Cdig, s->Cexp, st, nullptr, true);
}

// ------------------------------------------------------------------------------------------
// Tangent of the evaluation along dC (the orbital Hessian-vector product): the same products
// with dC_occ in place of C_occ where the chain rule puts it
// ------------------------------------------------------------------------------------------
las_status split_tangent_prepare(SplitState* s, const double* dCocc, cudaStream_t st,
                                 size_t* bytes) {
  if (!s->tblob) {
    const long R = (long)s->Lc * s->op;
    const size_t b0 = rup(planes_bytes(s->op, s->n), 256), b1 = rup((size_t)s->op * 4, 256);
    const size_t b2 = rup(planes_bytes(R, s->n), 256), b3 = rup((size_t)R * 4, 256);
    if (cudaMalloc(&s->tblob, b0 + b1 + b2 + b3) != cudaSuccess) {
      s->tblob = nullptr;
      las_record_cuda_error(cudaErrorMemoryAllocation, "cudaMalloc(tangent)", __FILE__, __LINE__);
      return LAS_ERR_CUDA;
    }
    // padding rows are never written by the slicers: zero once
    cudaError_t e = cudaMemsetAsync(s->tblob, 0, b0 + b1 + b2 + b3, st);
    if (e != cudaSuccess) {
      las_record_cuda_error(e, "cudaMemsetAsync(tangent)", __FILE__, __LINE__);
      return LAS_ERR_CUDA;
    }
    uint8_t* w = (uint8_t*)s->tblob;
    s->dCdig = make_planes(w, s->op, s->n);
    s->dCexp = (int*)(w + b0);
    s->dHdig = make_planes(w + b0 + b1, R, s->n);
    s->dHexp = (int*)(w + b0 + b1 + b2);
    *bytes += b0 + b1 + b2 + b3;
  }
  RowsStrided acc{dCocc, 1, s->op, nullptr};
  return slice_rows(acc, s->dCdig, s->dCexp, st, nullptr, true);
}

// dH = b^L dC_occ for the chunk's aux rows (Ht layout [nL][op][n])
las_status split_tangent_half(SplitState* s, int l0, int nL, double* dHt, cudaStream_t st) {
  return b_half(s, l0, nL, s->dCdig, 0, s->dCexp, s->op, dHt, s->op, st, s->bn[SPLIT_HALF]);
}

// After split_full of the chunk: X[(L,p)][q] = sum_mu H_L(mu,p) dC(mu,q) (so that dT_L = X_L +
// X_L^T), and the digits of dH (rows (L,p), K = mu) with their row exponents.
las_status split_tangent_full(SplitState* s, int nL, const double* dHt, double* X,
                              cudaStream_t st) {
  const long R = (long)nL * s->op;
  las_status rc = ozaki_gemm(s->Hdig, 0, s->Hexp, R, s->dCdig, 0, s->dCexp, s->op, s->n, 1, 0, X,
                             s->op, 0, 0, 0, s->status, st, 0, s->bn[SPLIT_FULL]);
  if (rc != LAS_OK) return rc;
  k_slice_ht<<<(unsigned)((R + 15) / 16), 256, 0, st>>>(dHt, R, s->n, s->dHdig, s->dHexp);
  las_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "k_slice_ht launch", __FILE__, __LINE__);
    return LAS_ERR_CUDA;
  }
  return LAS_OK;
}

const int* split_tangent_dhexp(SplitState* s) { return s->dHexp; }

// Out (+)= sum_{(L,p)} A(mu,(L,p)) W((L,p),q): A = H (which = 0) or dH (which = 1), read
// MN-major from its digit planes; Wt[q][(L,p)] holds W scaled by that operand's row exponents.
las_status split_tangent_project(SplitState* s, int nL, int which, const double* Wt, double* Out,
                                 int accumulate, cudaStream_t st) {
  const long R = (long)nL * s->op;
  Planes W = s->Wdig;
  W.K = R;
  las_status rc = slice_rows(RowsStrided{Wt, R, 1, nullptr}, W, s->Wexp, st, s->mx, true);
  if (rc != LAS_OK) return rc;
  const int ks = (int)std::max(1L, std::min((long)s->ks, (R + 32 * 64 - 1) / (32 * 64)));
  rc = ozaki_gemm(which ? s->dHdig : s->Hdig, 0, nullptr, s->n, W, 0, s->Wexp, s->op, R, ks, 0,
                  s->part, s->op, (long)s->n * s->op, 0, 0, s->status, st, 0,
                  s->bn[SPLIT_PROJECT], 1);
  if (rc != LAS_OK) return rc;
  launch_reduce_partials(s->part, ks, (long)s->n * s->op, Out, accumulate, st);
  return LAS_OK;
}

// hdC = h dC_occ (the digits of h from split_one_electron_hc of the same h)
las_status split_tangent_one_electron(SplitState* s, double* hdC, cudaStream_t st) {
  return ozaki_gemm(s->hdig, 0, s->hexp, s->n, s->dCdig, 0, s->dCexp, s->op, s->n, 1, 0, hdC,
                    s->op, 0, 0, 0, s->status, st, 0, s->bn[SPLIT_ONE_ELECTRON]);
}

las_status split_lpu(SplitState* s, int nL, const double* Ht, int c, int a, const double* C,
                     int nmo, int p0, int np, double* Lpu, cudaStream_t st, size_t* bytes) {
  // Lpu[L][p][u] = sum_mu C[mu][p0+p] Ht[L][c+u][mu]: rows (L,u) of the half transform times the
  // rows p of C[:, p0:p1]^T, written in the (L, p, u) layout by the half-transform epilogue mode
  const int n = s->n;
  if (a < 1 || np < 1) return LAS_OK;
  if (np > nmo) return LAS_ERR_INTERNAL;
  if (!s->Mpblob) {   // planes for all nmo rows of C^T: allocated once per context
    const size_t pb = planes_bytes(nmo, n), eb = rup((size_t)nmo * 4, 256);
    if (cudaMalloc(&s->Mpblob, rup(pb, 256) + eb) != cudaSuccess) {
      s->Mpblob = nullptr;
      las_record_cuda_error(cudaErrorMemoryAllocation, "cudaMalloc(lpu)", __FILE__, __LINE__);
      return LAS_ERR_CUDA;
    }
    *bytes += rup(pb, 256) + eb;
    cudaError_t e = cudaMemsetAsync(s->Mpblob, 0, rup(pb, 256) + eb, st);
    if (e != cudaSuccess) {
      las_record_cuda_error(e, "cudaMemsetAsync(lpu)", __FILE__, __LINE__);
      return LAS_ERR_CUDA;
    }
    s->Mpd = make_planes(s->Mpblob, nmo, n);
    s->Mpexp = (int*)((uint8_t*)s->Mpblob + rup(pb, 256));
  }
  Planes Mp = s->Mpd;
  Mp.R = np;
  las_status rc = slice_rows(RowsStrided{C + p0, 1, nmo, nullptr}, Mp, s->Mpexp, st, nullptr,
                             true);
  // the active rows (L,u) of this chunk, sliced into the H digit planes (capacity Lc*op rows)
  Planes Hd = s->Hdig;
  Hd.R = (long)nL * a;
  if (rc == LAS_OK) rc = slice_rows(RowsHtAct{Ht, n, s->op, c, a}, Hd, s->Hexp, st, nullptr, true);
  if (rc == LAS_OK)
    rc = ozaki_gemm(Hd, 0, s->Hexp, (long)nL * a, Mp, 0, s->Mpexp, np, n, 1, 1, Lpu, 0, 0, a, np,
                    s->status, st);
  return rc;
}

// When the half transform runs in 96-column tiles and the columns beyond the last whole tile
// number at most 64 (the JK call's 150 core columns: 96 + 54), those columns form a second product
// of 64-column tiles: 160 columns computed instead of 192, and a 64-column stage costs about three
// quarters of a 96-column one.  Not while products are recorded for a grouped launch, which would
// then mix tile widths.
las_status split_half(SplitState* s, int l0, int nL, int oc, double* Ht, cudaStream_t st) {
  if (oc < 1 || oc > s->op) return LAS_ERR_INTERNAL;
  const int bn = s->bn[SPLIT_HALF];
  const int whole = oc / 96 * 96, rest = oc - whole;
  if (bn == 96 && whole > 0 && rest > 0 && rest <= 64 && !g_record) {
    las_status rc = b_half(s, l0, nL, s->Cdig, 0, s->Cexp, whole, Ht, oc, st, 96);
    if (rc != LAS_OK) return rc;
    return b_half(s, l0, nL, s->Cdig, whole, s->Cexp + whole, rest, Ht + (size_t)whole * s->n,
                  oc, st, 64);
  }
  return b_half(s, l0, nL, s->Cdig, 0, s->Cexp, oc, Ht, oc, st, bn);
}

las_status split_full(SplitState* s, int nL, const double* Ht, double* T, cudaStream_t st) {
  const long R = (long)nL * s->op;
  k_slice_ht<<<(unsigned)((R + 15) / 16), 256, 0, st>>>(Ht, R, s->n, s->Hdig, s->Hexp);
  las_count_launch();
  {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      las_record_cuda_error(e, "k_slice_ht launch", __FILE__, __LINE__);
      return LAS_ERR_CUDA;
    }
  }
  return ozaki_gemm(s->Hdig, 0, s->Hexp, R, s->Cdig, 0, s->Cexp, s->op, s->n, 1, 0, T, s->op, 0,
                    0, 0, s->status, st, 0, s->bn[SPLIT_FULL]);
}

las_status split_project_gemm(SplitState* s, int nL, const double* Wt, int* ks_used,
                              cudaStream_t st) {
  const long R = (long)nL * s->op;      // K of the projection: (L, p); a multiple of 16
  // A: the digit planes of H written by split_full (rows (L,p), K = mu), read MN-major: rows mu,
  // K = (L,p); their per-(L,p) exponents are folded into W.
  // W rows q (K = (L,p)), already scaled by 2^Hexp[(L,p)] and stored transposed: Wt[q][R]
  Planes W = s->Wdig;
  W.K = R;
  RowsStrided acc{Wt, R, 1, nullptr};
  las_status rc = slice_rows(acc, W, s->Wexp, st, s->mx, true);
  if (rc != LAS_OK) return rc;
  const int ks = (int)std::max(1L, std::min((long)s->ks, (R + 32 * 64 - 1) / (32 * 64)));
  *ks_used = ks;
  return ozaki_gemm(s->Hdig, 0, nullptr, s->n, W, 0, s->Wexp, s->op, R, ks, 0, s->part, s->op,
                    (long)s->n * s->op, 0, 0, s->status, st, 0, s->bn[SPLIT_PROJECT], 1);
}

void split_project_reduce(SplitState* s, int ks, double* Out, int accumulate, cudaStream_t st) {
  launch_reduce_partials(s->part, ks, (long)s->n * s->op, Out, accumulate, st);
}

las_status split_project(SplitState* s, int nL, const double* Wt, double* Out, int accumulate,
                         cudaStream_t st) {
  int ks = 1;
  las_status rc = split_project_gemm(s, nL, Wt, &ks, st);
  if (rc != LAS_OK) return rc;
  split_project_reduce(s, ks, Out, accumulate, st);
  return LAS_OK;
}

las_status split_exchange(SplitState* s, int nL, int oc, const double* Ht, double* K, int accumulate,
                          cudaStream_t st) {
  // K(mu,nu) (+)= sum_{(L,p)} Ht[(L,p)][mu] Ht[(L,p)][nu]: rows mu of H^T, scaled per row over
  // the long index (L,p), serve as both operands
  const long R = (long)nL * oc, n = s->n;
  if (oc < 1 || oc > s->op) return LAS_ERR_INTERNAL;
  Planes HT = s->HdigT;
  HT.K = R;
  las_status rc = LAS_OK;
  {
    cudaError_t e = cudaMemsetAsync(s->mx, 0, n * sizeof(unsigned long long), st);
    if (e != cudaSuccess) {
      las_record_cuda_error(e, "cudaMemsetAsync(colmax)", __FILE__, __LINE__);
      return LAS_ERR_CUDA;
    }
    const long seg = 512;
    dim3 g1((unsigned)((n + 255) / 256), (unsigned)((R + seg - 1) / seg));
    k_colmax<<<g1, 256, 0, st>>>(Ht, R, (int)n, seg, s->mx);
    las_count_launch();
    dim3 g2((unsigned)((R + 31) / 32), (unsigned)((n + COLS_PER_BLOCK - 1) / COLS_PER_BLOCK));
    k_slice_ht_cols<<<g2, 256, 0, st>>>(Ht, R, (int)n, s->mx, HT, s->hexp);
    las_count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      las_record_cuda_error(e, "k_slice_ht_cols launch", __FILE__, __LINE__);
      return LAS_ERR_CUDA;
    }
  }
  // partials [ks][n][n] live in the projection's partial buffer (64 * n * op doubles)
  const long cap = std::max(1L, std::min((64L * s->op) / n, (R + 32 * 64 - 1) / (32 * 64)));
  const int ks = balanced_ksplit(ozaki_tiles(n, n, 1), (R + BK - 1) / BK, cap);
  // symmetric product: only tiles touching the lower triangle; the caller mirrors the result
  rc = ozaki_gemm(HT, 0, s->hexp, n, HT, 0, s->hexp, n, R, ks, 0, s->part, n, n * n, 0, 0,
                  s->status, st, 1);
  if (rc != LAS_OK) return rc;
  launch_reduce_partials(s->part, ks, n * n, K, accumulate, st);
  return LAS_OK;
}

las_status split_one_electron_hc(SplitState* s, const double* h, double* hC, cudaStream_t st) {
  // hC = h C_occ  (rows mu of h, columns p of C_occ: the digits of C_occ are already sliced)
  las_status rc = slice_rows(RowsStrided{h, s->n, 1, nullptr}, s->hdig, s->hexp, st, nullptr,
                             true);
  if (rc == LAS_OK)
    rc = ozaki_gemm(s->hdig, 0, s->hexp, s->n, s->Cdig, 0, s->Cexp, s->op, s->n, 1, 0, hC, s->op,
                    0, 0, 0, s->status, st, 0, s->bn[SPLIT_ONE_ELECTRON]);
  return rc;
}

las_status split_one_electron_hmo(SplitState* s, const double* hC, double* hmo,
                                  cudaStream_t st) {
  // hmo = C_occ^T hC  (rows p of C_occ^T are the C_occ digit rows; columns q of hC)
  las_status rc =
      slice_rows(RowsStrided{hC, 1, s->op, nullptr}, s->hcdig, s->hcexp, st, nullptr, true);
  if (rc == LAS_OK)
    rc = ozaki_gemm(s->Cdig, 0, s->Cexp, s->op, s->hcdig, 0, s->hcexp, s->op, s->n, 1, 0, hmo,
                    s->op, 0, 0, 0, s->status, st, 0, s->bn[SPLIT_ONE_ELECTRON]);
  return rc;
}

las_status split_one_electron(SplitState* s, const double* h, double* hC, double* hmo,
                              cudaStream_t st) {
  las_status rc = split_one_electron_hc(s, h, hC, st);
  if (rc == LAS_OK) rc = split_one_electron_hmo(s, hC, hmo, st);
  return rc;
}

// ------------------------------------------------------------------------------------------
// Standalone emulated-FP64 GEMM through the same kernels (C ABI)
// ------------------------------------------------------------------------------------------
static size_t sgemm_ws(long M, long N, long K) {
  return rup(planes_bytes(M, K), 256) + rup(planes_bytes(N, K), 256) + rup(M * 4, 256) +
         rup(N * 4, 256) + 256;
}

extern "C" size_t las_split_gemm_workspace(long M, long N, long K) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  return sgemm_ws(M, N, K);
}

extern "C" las_status las_split_gemm(long M, long N, long K, const double* A, long lda,
                                     const double* B, long ldb, double* C, long ldc,
                                     void* workspace, size_t workspace_bytes, void* stream) {
  if (M < 0 || N < 0 || K < 0) return LAS_ERR_ARG;
  if (M == 0 || N == 0) return LAS_OK;
  if (!A || !B || !C) return LAS_ERR_ARG;
  if (lda < K || ldb < N || ldc < N) return LAS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (K == 0) {
    for (long r = 0; r < M; ++r)
      LAS_CUDA_TRY(cudaMemsetAsync(C + r * ldc, 0, N * 8, st));
    return LAS_OK;
  }
  if (!workspace) return LAS_ERR_ARG;
  if (workspace_bytes < sgemm_ws(M, N, K) || ((uintptr_t)workspace & 255)) return LAS_ERR_WORKSPACE;
  uint8_t* w = (uint8_t*)workspace;
  Planes Ad = make_planes(w, M, K);
  w += rup(planes_bytes(M, K), 256);
  Planes Bd = make_planes(w, N, K);
  w += rup(planes_bytes(N, K), 256);
  int* ea = (int*)w;
  w += rup(M * 4, 256);
  int* eb = (int*)w;
  w += rup(N * 4, 256);
  int* status = (int*)w;
  LAS_CUDA_TRY(cudaMemsetAsync(status, 0, 4, st));
  las_status rc = slice_rows(RowsStrided{A, lda, 1, nullptr}, Ad, ea, st);
  if (rc == LAS_OK) rc = slice_rows(RowsStrided{B, 1, ldb, nullptr}, Bd, eb, st);
  if (rc == LAS_OK)
    rc = ozaki_gemm(Ad, 0, ea, M, Bd, 0, eb, N, K, 1, 0, C, ldc, 0, 0, 0, status, st);
  if (rc != LAS_OK) return rc;
  int h = 0;
  LAS_CUDA_TRY(cudaMemcpyAsync(&h, status, 4, cudaMemcpyDeviceToHost, st));
  LAS_CUDA_TRY(cudaStreamSynchronize(st));
  return h ? (las_status)h : LAS_OK;
}

// ------------------------------------------------------------------------------------------
// Fragment-embedding AO2MO in split precision (Eqs. ao2mo_1, ao2mo_2, ppaa, papa)
// ------------------------------------------------------------------------------------------
namespace lasdf_split {
// Row (u, v) of the active block of T (rows (L, p), columns q), K = the auxiliary row L:
// T[L][a0+u][a0+v]
struct RowsAA {
  const double* T;
  long n2;
  int nmo, a0, ma;
  __device__ __forceinline__ double operator()(long r, long k) const {
    const int u = (int)(r / ma), v = (int)(r - (long)u * ma);
    return T[k * n2 + (long)(a0 + u) * nmo + a0 + v];
  }
};
// Row (p, u) of the MO-active columns of T, K = L: T[L][p][a0+u]
struct RowsPA {
  const double* T;
  long n2;
  int nmo, a0, ma;
  __device__ __forceinline__ double operator()(long r, long k) const {
    const long p = r / ma, u = r - p * ma;
    return T[k * n2 + p * nmo + a0 + u];
  }
};
}  // namespace lasdf_split

struct FragSplit {
  int n, nmo, ma, Lc;
  Planes Mdig;   int* Mexp;     // rows p of M^T, K = e
  Planes Hd;     int* Hexp;     // rows (L, p) of the half transform, K = e
  Planes Tpl;    int* Texp;     // rows (p, q) of T, K = L
  Planes Taa;    int* Taaexp;   // rows (u, v) of the active block, K = L
  Planes Tpa;    int* Tpaexp;   // rows (p, u), K = L
  unsigned long long* mx;       // [nmo^2] column maxima of T
  void* blob;
};

las_status frag_split_create(FragSplit** out, int n, int nmo, int ma, int Lc, cudaStream_t st,
                             size_t* bytes) {
  *out = nullptr;
  if (!encode_fn()) return LAS_ERR_UNSUPPORTED;
  if (ozaki_prepare() != LAS_OK) return LAS_ERR_CUDA;
  FragSplit* f = (FragSplit*)calloc(1, sizeof(FragSplit));
  if (!f) return LAS_ERR_INTERNAL;
  f->n = n;
  f->nmo = nmo;
  f->ma = ma;
  f->Lc = Lc;
  const long n2 = (long)nmo * nmo, R1 = (long)Lc * nmo;
  const size_t parts[] = {planes_bytes(nmo, n),             (size_t)nmo * 4,
                          planes_bytes(R1, n),              (size_t)R1 * 4,
                          planes_bytes(n2, Lc),             (size_t)n2 * 4,
                          planes_bytes((long)ma * ma, Lc),  (size_t)ma * ma * 4,
                          planes_bytes((long)nmo * ma, Lc), (size_t)nmo * ma * 4,
                          (size_t)n2 * 8};   // each part is rounded up to 256 bytes below
  size_t total = 0;
  for (size_t b : parts) total += rup(b, 256);
  if (cudaMalloc(&f->blob, total) != cudaSuccess) {
    las_record_cuda_error(cudaErrorMemoryAllocation, "cudaMalloc(frag ao2mo)", __FILE__, __LINE__);
    free(f);
    return LAS_ERR_CUDA;
  }
  // padding rows and K blocks are never written by the live-row slicers: zero them once
  cudaError_t e = cudaMemsetAsync(f->blob, 0, total, st);
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "cudaMemsetAsync(frag ao2mo)", __FILE__, __LINE__);
    cudaFree(f->blob);
    free(f);
    return LAS_ERR_CUDA;
  }
  uint8_t* w = (uint8_t*)f->blob;
  auto take = [&](size_t b) { void* q = w; w += rup(b, 256); return q; };
  f->Mdig = make_planes(take(parts[0]), nmo, n);
  f->Mexp = (int*)take(parts[1]);
  f->Hd = make_planes(take(parts[2]), R1, n);
  f->Hexp = (int*)take(parts[3]);
  f->Tpl = make_planes(take(parts[4]), n2, Lc);
  f->Texp = (int*)take(parts[5]);
  f->Taa = make_planes(take(parts[6]), (long)ma * ma, Lc);
  f->Taaexp = (int*)take(parts[7]);
  f->Tpa = make_planes(take(parts[8]), (long)nmo * ma, Lc);
  f->Tpaexp = (int*)take(parts[9]);
  f->mx = (unsigned long long*)take(parts[10]);
  *bytes += total;
  *out = f;
  return LAS_OK;
}

void frag_split_destroy(FragSplit* f) {
  if (!f) return;
  if (f->blob) cudaFree(f->blob);
  free(f);
}

int frag_split_fits(const FragSplit* f, int n, int nmo, int ma, int Lc) {
  return f && f->n == n && f->nmo == nmo && f->ma >= ma && f->Lc >= Lc;
}

las_status frag_split_prepare_M(FragSplit* f, const double* M, cudaStream_t st) {
  // rows p of M^T (K = e): element (p, e) = M[e][p]
  return slice_rows(RowsStrided{M, 1, f->nmo, nullptr}, f->Mdig, f->Mexp, st, nullptr, true);
}

las_status frag_split_chunk(SplitState* s, FragSplit* f, int l0, int nL, double* H, double* T,
                            int a0, int ma, double* ppaa, double* papa, double* part,
                            long part_elems, int accumulate, cudaStream_t st) {
  const int n = f->n, nmo = f->nmo;
  const long n2 = (long)nmo * nmo, R1 = (long)nL * nmo;
  if (nL < 1 || nL > f->Lc || ma > f->ma) return LAS_ERR_INTERNAL;
  // Eq. ao2mo_1: H[L][p][e2] = sum_e1 b^L(e2, e1) M[e1][p]
  las_status rc = b_half(s, l0, nL, f->Mdig, 0, f->Mexp, nmo, H, nmo, st, OZ_BN);
  // Eq. ao2mo_2: T[L][p][q] = sum_e H[L][p][e] M[e][q]
  Planes Hd = f->Hd;
  Hd.R = R1;
  if (rc == LAS_OK) rc = slice_rows(RowsStrided{H, n, 1, nullptr}, Hd, f->Hexp, st, nullptr, true);
  if (rc == LAS_OK)
    rc = ozaki_gemm(Hd, 0, f->Hexp, R1, f->Mdig, 0, f->Mexp, nmo, n, 1, 0, T, nmo, 0, 0, 0,
                    s->status, st);
  if (rc != LAS_OK) return rc;
  const long kb = (nL + BK - 1) / BK;
  if (ppaa) {
    // Eq. ppaa: ppaa[(p,q)][(u,v)] (+)= sum_L T[L][(p,q)] T[L][a0+u][a0+v]
    Planes A = f->Tpl, B = f->Taa;
    A.K = nL;
    B.R = (long)ma * ma;
    B.K = nL;
    // rows (p,q) of T^T with per-row exponents: column maxima of T [nL][n2], then a transposing
    // slicer (coalesced reads along (p,q))
    cudaError_t e = cudaMemsetAsync(f->mx, 0, (size_t)n2 * 8, st);
    if (e != cudaSuccess) {
      las_record_cuda_error(e, "cudaMemsetAsync(frag colmax)", __FILE__, __LINE__);
      return LAS_ERR_CUDA;
    }
    const long seg = 512;
    dim3 g1((unsigned)((n2 + 255) / 256), (unsigned)((nL + seg - 1) / seg));
    k_colmax<<<g1, 256, 0, st>>>(T, nL, (int)n2, seg, f->mx);
    las_count_launch();
    dim3 g2((unsigned)((nL + 31) / 32), (unsigned)((n2 + COLS_PER_BLOCK - 1) / COLS_PER_BLOCK));
    k_slice_ht_cols<<<g2, 256, 0, st>>>(T, nL, (int)n2, f->mx, A, f->Texp);
    las_count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      las_record_cuda_error(e, "frag slicer launch", __FILE__, __LINE__);
      return LAS_ERR_CUDA;
    }
    if (rc == LAS_OK)
      rc = slice_rows(RowsAA{T, n2, nmo, a0, ma}, B, f->Taaexp, st, nullptr, true);
    const long out = n2 * ma * ma;
    const int ks = balanced_ksplit(ozaki_tiles(n2, (long)ma * ma, 0), kb,
                                   std::max(1L, std::min(kb, part_elems / out)));
    if (rc == LAS_OK)
      rc = ozaki_gemm(A, 0, f->Texp, n2, B, 0, f->Taaexp, (long)ma * ma, nL, ks, 0, part,
                      (long)ma * ma, out, 0, 0, s->status, st);
    if (rc != LAS_OK) return rc;
    launch_reduce_partials(part, ks, out, ppaa, accumulate, st);
  }
  if (papa) {
    // Eq. papa: papa[(p,u)][(q,v)] (+)= sum_L T[L][p][a0+u] T[L][q][a0+v] (lower triangle; the
    // caller mirrors it once all chunks are in)
    Planes A = f->Tpa;
    A.R = (long)nmo * ma;
    A.K = nL;
    rc = slice_rows(RowsPA{T, n2, nmo, a0, ma}, A, f->Tpaexp, st, nullptr, true);
    const long m = (long)nmo * ma, out = m * m;
    const int ks = balanced_ksplit(ozaki_tiles(m, m, 1), kb,
                                   std::max(1L, std::min(kb, part_elems / out)));
    if (rc == LAS_OK)
      rc = ozaki_gemm(A, 0, f->Tpaexp, m, A, 0, f->Tpaexp, m, nL, ks, 0, part, m, out, 0, 0,
                      s->status, st, 1);
    if (rc != LAS_OK) return rc;
    launch_reduce_partials(part, ks, out, papa, accumulate, st);
  }
  return LAS_OK;
}

// ------------------------------------------------------------------------------------------
// Self-test of the bounded waits: one CTA waits on an mbarrier that nothing ever arrives on,
// with a short poll limit; the wait must give up, record LAS_ERR_TIMEOUT and let the kernel
// return, leaving the context usable.
// ------------------------------------------------------------------------------------------
namespace lasdf_split {
__global__ void k_selftest_wait(int* status, long limit) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    sm100::mbar_init(&bar, 1);
    abort_flag = 0;
    sm100::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    sm100::mbar_wait(&bar, 0, (volatile int*)&abort_flag, status, LAS_ERR_TIMEOUT, 0, limit);
  __syncthreads();
}
}  // namespace lasdf_split

extern "C" las_status las_selftest_bounded_wait(void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int* status = nullptr;
  LAS_CUDA_TRY(cudaMalloc(&status, sizeof(int)));
  las_status rc = LAS_OK;
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    k_selftest_wait<<<1, 32, 0, st>>>(status, 1L << 16);
    las_count_launch();
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    las_record_cuda_error(e, "bounded-wait self-test", __FILE__, __LINE__);
    rc = LAS_ERR_CUDA;
  } else {
    rc = (las_status)h;
  }
  cudaFree(status);
  return rc;
}

// ------------------------------------------------------------------------------------------
// Allocation-free variant of las_split_gemm
//
// Some callers cannot allocate device memory at the point where they need a product: plugins
// whose host application owns every device allocation through its own pool, and
// latency-critical loops where a cudaMalloc could synchronise the device. This entry point takes
// its scratch from a fixed array that is part of the library image instead of asking for a
// buffer: the digit planes and exponents of both operands live in `g_noalloc_scratch`, a
// LAS_NOALLOC_SCRATCH_BYTES (64 MiB) file-scope device array that every GPU which loads the
// library holds until the process exits.  Like las_split_gemm it waits for its stream and reads
// its status word back before returning.
// ------------------------------------------------------------------------------------------
#include <mutex>

static __device__ __align__(256) unsigned char g_noalloc_scratch[LAS_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device ordinal
}  // namespace

extern "C" las_status las_split_gemm_noalloc(long M, long N, long K, const double* A, long lda,
                                             const double* B, long ldb, double* C, long ldc,
                                             void* stream) {
  if (M < 0 || N < 0 || K < 0) return LAS_ERR_ARG;
  if (M == 0 || N == 0) return LAS_OK;
  if (!A || !B || !C) return LAS_ERR_ARG;
  if (lda < K || ldb < N || ldc < N) return LAS_ERR_ARG;
  if (K > 0 && sgemm_ws(M, N, K) > (size_t)LAS_NOALLOC_SCRATCH_BYTES) return LAS_ERR_WORKSPACE;
  int dev = 0;
  LAS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return LAS_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  {
    // Set-up, once per device with that device current: in host code the array's name is only
    // a host-side stand-in, so its device address must be looked up.
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      LAS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_addr[dev] = p;
    }
    scratch = g_noalloc_addr[dev];
  }
  // The shared array keeps whatever the previous call left; las_split_gemm clears the status
  // word it keeps there before use and overwrites every digit plane it reads.
  return las_split_gemm(M, N, K, A, lda, B, ldb, C, ldc, scratch, LAS_NOALLOC_SCRATCH_BYTES,
                        stream);
}
