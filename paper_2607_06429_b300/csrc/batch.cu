// Multi-right-hand-side far-field sums on the 5th-generation tensor cores (tcgen05).
//
// For R right-hand sides the far-field sum of one source class is a dense contraction
//     Y[i, r] = sum_j C(x_i, y_j) q_j^(r),
// where the kernel tile C (complex) depends on the geometry only.  Each tile of C is
// evaluated once in FP32 on the CUDA cores and contracted with a block of R = 64 charge
// columns on the tensor cores, so the sine/cosine/rsqrt work is amortised R-fold.
//
// Precision: the contraction runs as three TF32 products with FP32 accumulation
// (C_lo Q_hi + C_hi Q_lo + C_hi Q_hi, where x_hi = tf32(x), x_lo = tf32(x - x_hi)),
// about 21 significant bits per product.  The tensor accumulator's rounding error grows
// with the number of MMAs summed into it, so it holds one source tile only: after each
// tile the evaluating warps fold it into a running FP32 sum H in tensor memory with a
// compensated (Kahan) step and leave the step's rounding error in the accumulator, where
// the next tile's MMAs add onto it.  A target tile leaves the CTA as H plus the pending
// compensation, in FP64.  Complex arithmetic as two real products of width N = 128,
//     [Y_re | Y_im] += C_re [Q_re | Q_im] + C_im [-Q_im | Q_re],
// the second with the instruction descriptor's negate-B bit applied to [Q_im | -Q_re].
//
// Layout.  One CTA (16 evaluating warps, an MMA warp and a copy warp; one CTA per SM) owns
// a tile of 128 targets (the MMA M) and streams the sources in tiles of 32 (the MMA K is
// 8, four k-steps per tile).
//   * A operand (128 x 32 each): C_re and C_im, hi and lo, written straight into tensor
//     memory by the evaluating warps (tcgen05.st) once the previous tile's MMAs retired;
//   * B operands (64 x 32 per block, K-major, no swizzle, 8 x 16-byte core matrices):
//     Q_re, Q_im, hi and lo, prepared per apply in global memory as the shared-memory
//     image of each source tile, preceded by the tile's 32 source records, and fetched
//     with two bulk asynchronous copies (TMA engine) that complete on an mbarrier; the
//     evaluating warps add the negated -Q_re blocks, so that each product is one N = 128
//     MMA over [Y_re | Y_im];
//   * two accumulator buffers D0, D1 (128 lanes x 128 FP32 columns: Y_re | Y_im) used by
//     alternate tiles, so the fold of one overlaps the MMAs of the next, and the running
//     sum H: all 512 tensor-memory columns, allocated by warp 0.
// Pipeline: four stages of charge images in shared memory (the copy engine runs up to
// three tiles ahead of the tensor cores) while the CUDA cores evaluate the next tile.
// Keeping A out of shared memory leaves its bandwidth to the B operand reads (a variant
// with a double-buffered A in shared memory ran 1.6x slower: the tensor cores' operand
// reads doubled and only two image stages fitted).  Each tcgen05.mma of 128 x 128 x 8 TF32
// occupies the issuing thread for about as long as the tensor pipe takes to execute it,
// so the MMA thread has a warp of its own, and so have the bulk copies, whose issue can
// also block.  Work is
// split over the CTAs with the same balanced item ranges (target tile, 2048-source chunk)
// and deterministic fix-up as the single-RHS sums.  Every wait on an mbarrier is bounded
// (2 s of wall time); on expiry the kernel records an error code, stops issuing work,
// waits (bounded again) for its copies and MMAs in flight and still releases its tensor
// memory.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "vsie_internal.h"

namespace vsie {

constexpr int BT_M = 128;             // targets per CTA tile
constexpr int BT_S = 32;              // sources per tile (MMA K = 8: four k-steps)
constexpr int BT_R = 64;              // right-hand sides per launch
constexpr int BT_CHUNK_TILES = 64;    // source tiles per work item (2048 sources; default, autotuned)
constexpr int BT_B_MAT = BT_R * BT_S * 4;        // 8 KB per B block (64 x 32 tf32)
constexpr int BT_HDR = 6 * BT_S * 4;             // -x, -y, -z, nx, ny, nz of the 32 sources
constexpr int BT_IMG = BT_HDR + 4 * BT_B_MAT;    // per-tile image in global memory
constexpr int BT_NB = 4;                         // stages of charge images (prefetch distance 3)
// An image stage in shared memory holds [header][Q_re hi][Q_im hi][-Q_re hi][Q_re lo][Q_im lo]
// [-Q_re lo]; the copy engine fills all but the two negated blocks, which the evaluating
// warps write.  Stacking (Q_re; Q_im) and (Q_im; -Q_re) along N gives the two B operands
// of the N = 128 products [Y_re | Y_im] += C_re (Q_re | Q_im) + C_im (-Q_im | Q_re).
constexpr int BT_SIMG = BT_HDR + 6 * BT_B_MAT;   // 49,920 bytes
constexpr int BT_S_HI = BT_HDR;                  // Q_re hi (then Q_im hi, -Q_re hi)
constexpr int BT_S_LO = BT_HDR + 3 * BT_B_MAT;   // Q_re lo (then Q_im lo, -Q_re lo)
constexpr int BT_B_OFF = 0;
constexpr int BT_BAR_OFF = BT_B_OFF + BT_NB * BT_SIMG;
constexpr int BT_NBARS = 1 + 2 * BT_NB + 2;      // a_full, b_full[NB], mma_done[NB], d_ready[2]
constexpr int BT_SMEM = BT_BAR_OFF + 8 * BT_NBARS + 16;
// tensor memory columns: accumulator buffers D0, D1 (Y_re | Y_im, 128 each), the running sum
// H (same layout) and the A operand of the current tile (C_re hi, C_re lo, C_im hi, C_im lo)
constexpr int BT_TMEM_COLS = 512;
constexpr uint32_t BT_COL_D = 0, BT_COL_H = 256, BT_COL_A = 384;
static_assert(BT_IMG % 16 == 0 && BT_SIMG % 16 == 0 && BT_BAR_OFF % 8 == 0, "alignment");
static_assert(BT_SMEM <= 227 * 1024, "shared memory budget");

// byte offset of element (row, k) in a K-major, no-swizzle operand with K = 32:
// core matrices of 8 rows x 16 bytes; along K they are 128 bytes apart (leading byte
// offset), along rows 1024 bytes apart (stride byte offset).
__host__ __device__ __forceinline__ uint32_t bt_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;   // leading byte offset: next core matrix along K
  d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;             // descriptor version (sm_100 family)
  return d;                           // base offset 0, no swizzle
}

// instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 128
__host__ __device__ constexpr uint32_t bt_idesc(bool negate_b) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((negate_b ? 1u : 0u) << 14) |
         ((uint32_t)((2 * BT_R) >> 3) << 17) | ((uint32_t)(BT_M >> 4) << 24);
}

__device__ __forceinline__ float tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Bounded wait: polls the mbarrier phase and gives up after BT_WAIT_NS of wall time
// (read from the global nanosecond timer every 256 polls).
constexpr uint64_t BT_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  {
    // fast path: a phase that has already completed is seen by a non-blocking test (the
    // blocking try_wait costs about 150 cycles even then)
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255) == 0) {
      const uint64_t t = global_ns();
      if (it == 0) t0 = t;
      else if (t - t0 > BT_WAIT_NS) return false;
    }
  }
}

// A operand in tensor memory (row i of A in lane i, one 32-bit column per k)
__device__ __forceinline__ void mma_tf32_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// ----------------------------------------------------------------- tile evaluation

// Image header (structure of arrays over the tile's 32 sources): -x~, -y~, -z~ (kappa-
// scaled positions, negated) and the unit normal n (K class; zero for G).
// G class:  C~ = e^{2 pi i t} / |d~|
// K class:  C~ = e^{2 pi i t} (2 pi i t - 1)(d~ . n) / |d~|^3
// Two sources per packed FP32x2 instruction (the same target).
struct EvalG {
  static constexpr bool kNormal = false;
};
struct EvalK {
  static constexpr bool kNormal = true;
};

__device__ __forceinline__ float2 bf2(float a) { return make_float2(a, a); }

template <class Ev>
__device__ __forceinline__ void eval_pair2(float2 tx, float2 ty, float2 tz, float2 nsx, float2 nsy, float2 nsz,
                                          float2 nx, float2 ny, float2 nz, float2& cre, float2& cim) {
  const float2 dx = __fadd2_rn(tx, nsx), dy = __fadd2_rn(ty, nsy), dz = __fadd2_rn(tz, nsz);
  float2 r2 = __fmul2_rn(dx, dx);
  r2 = __ffma2_rn(dy, dy, r2);
  r2 = __ffma2_rn(dz, dz, r2);
  float2 rinv;
  rinv.x = (r2.x > 0.0f) ? rsqrtf(r2.x) : 0.0f;
  rinv.y = (r2.y > 0.0f) ? rsqrtf(r2.y) : 0.0f;
  const float2 t = __fmul2_rn(r2, rinv);
  const float2 u = __fadd2_rn(t, bf2(12582912.0f));
  const float2 w = __fadd2_rn(u, bf2(-12582912.0f));
  const float2 f = __ffma2_rn(w, bf2(-1.0f), t);
  const float2 ang = __fmul2_rn(f, bf2(6.28318530717958647692f));
  float2 cs, sn;
  __sincosf(ang.x, &sn.x, &cs.x);
  __sincosf(ang.y, &sn.y, &cs.y);
  if (!Ev::kNormal) {
    cre = __fmul2_rn(cs, rinv);
    cim = __fmul2_rn(sn, rinv);
    return;
  }
  float2 dn = __fmul2_rn(dx, nx);
  dn = __ffma2_rn(dy, ny, dn);
  dn = __ffma2_rn(dz, nz, dn);
  const float2 g3 = __fmul2_rn(__fmul2_rn(__fmul2_rn(rinv, rinv), rinv), dn);
  const float2 kr = __fmul2_rn(t, bf2(6.28318530717958647692f));
  // (cos + i sin)(i kr - 1) = -(cos + kr sin) + i (kr cos - sin)
  const float2 A = __ffma2_rn(kr, sn, cs);
  const float2 Q = __ffma2_rn(kr, cs, __fmul2_rn(sn, bf2(-1.0f)));
  cre = __fmul2_rn(__fmul2_rn(g3, bf2(-1.0f)), A);
  cim = __fmul2_rn(g3, Q);
}

constexpr int BT_MAXP = 16;  // operators per persistent launch

// One launch covers nprob operators with the same work shape (targets, source tiles): the
// items (operator, target tile, chunk) are numbered operator-major, so that a global target
// tile index G stands for tile G % ntile_t of operator G / ntile_t.
struct BatchArgs {
  const float4* tgt[BT_MAXP];        // kappa-scaled FP32 target positions (nt) per operator
  const unsigned char* img[BT_MAXP]; // per-source-tile images (ntiles_src * BT_IMG bytes)
  double2* out[BT_MAXP];             // nt x nrhs_out column-major per operator
  int nprob;
  int64_t nt;               // targets
  int64_t ntiles_src;       // source tiles
  int64_t ntile_t;          // target tiles
  int64_t chunk_tiles;      // source tiles per work item
  int64_t nchunk;           // chunks of chunk_tiles source tiles
  int64_t nitems;           // nprob * ntile_t * nchunk
  int64_t grid;
  int64_t ld_out;           // nt
  int nrhs_out;             // columns written (<= BT_R)
  int mode;                 // 0 store, 1 add
  double* slots;            // [2 grid][2][BT_R][BT_M] FP64 partial target tiles for the fix-up
  int* status;              // nonzero on a timed-out wait
  int withhold_copies;      // failure-path test: the copy warp never starts the copies
};

__device__ __forceinline__ int64_t bt_begin(const BatchArgs& a, int64_t b) { return (b * a.nitems) / a.grid; }

// Warp roles: warps 0-15 (512 threads) evaluate the kernel tile and fold the tensor
// accumulator; warp 16 issues the MMAs from one lane; warp 17 issues the bulk copies.
// They meet only through mbarriers (a_full for the A operand; b_full, mma_done per image
// stage; d_ready per accumulator buffer), so evaluation, copies and tensor-core work
// overlap.
constexpr int BT_EVAL_THREADS = 512;
constexpr int BT_ALL_THREADS = BT_EVAL_THREADS + 64;

#define BT_LD8(addr, v)                                                                               \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"                  \
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]) \
               : "r"(addr)                                                                            \
               : "memory")
#define BT_ST8(addr, v)                                                                               \
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(addr),       \
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])         \
               : "memory")

template <class Ev>
__global__ void __launch_bounds__(BT_ALL_THREADS, 1) batch_tc_kernel(BatchArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + BT_BAR_OFF);
  uint64_t* a_full = bars;                      // A operand of the current tile written (16 warp arrivals)
  uint64_t* b_full = bars + 1;                  // [NB] charge image landed (tx bytes)
  uint64_t* mma_done = bars + 1 + BT_NB;        // [NB] MMAs of tile g retired (index g % NB)
  uint64_t* d_ready = bars + 1 + 2 * BT_NB;     // [2] accumulator buffer of tile g folded (index g % 2)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + BT_NBARS);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(a_full)), "r"(16));
    for (int i = 0; i < BT_NB; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b_full + i)), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(mma_done + i)), "r"(1));
    }
    for (int i = 0; i < 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(d_ready + i)), "r"(16));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(BT_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  bool err = false;
  const int64_t b = blockIdx.x;
  const int64_t k0 = bt_begin(a, b), k1 = bt_begin(a, b + 1);

  // The CTA's items [k0, k1) form segments: runs of consecutive chunks of one target tile.
  // Both roles walk the same sequence of source tiles; g counts them over the whole range.
  if (warp == BT_EVAL_THREADS / 32 + 1) {
    // ------------------------------------------------------------ copy warp
    // Streams the tiles' charge images into the stages, NB - 1 tiles ahead of the MMAs at
    // most: stage gp % NB is refilled once the MMAs of tile gp - NB, its last reader, have
    // retired.  A bulk copy can block its issuing thread while the copy engine is busy, so
    // it has a warp of its own rather than sharing the MMA thread.
    if (lane == 0) {
      uint32_t gp = 0;
      for (int64_t k = k0; k < k1 && !err;) {
        const int64_t tile = k / a.nchunk;
        const int64_t c0 = k - tile * a.nchunk;
        const int64_t c1 = min(a.nchunk, c0 + (k1 - k));
        const int64_t s_begin = c0 * a.chunk_tiles, s_end = min(a.ntiles_src, c1 * a.chunk_tiles);
        const unsigned char* pimg = a.img[tile / a.ntile_t];
        for (int64_t s = s_begin; s < s_end && !err; ++s, ++gp) {
          const int st2 = gp % BT_NB;
          if (gp >= BT_NB) err = !mbar_wait(mma_done + st2, ((gp - BT_NB) / BT_NB) & 1);
          if (err || a.withhold_copies) continue;
          unsigned char* bimg = smem + BT_B_OFF + st2 * BT_SIMG;
          const unsigned char* gimg = pimg + s * (int64_t)BT_IMG;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b_full + st2)),
                       "r"(BT_IMG)
                       : "memory");
          // [header][Q_re hi][Q_im hi] and [Q_re lo][Q_im lo]
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  su32(bimg)),
              "l"(gimg), "r"(BT_HDR + 2 * BT_B_MAT), "r"(su32(b_full + st2))
              : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  su32(bimg + BT_S_LO)),
              "l"(gimg + BT_HDR + 2 * BT_B_MAT), "r"(2 * BT_B_MAT), "r"(su32(b_full + st2))
              : "memory");
        }
        k = tile * a.nchunk + c1;
      }
      // before the CTA exits (and its shared memory goes away) every issued copy must have
      // landed; the last NB tiles' copies are the ones possibly in flight
      const bool err_wait = err;
      if (!a.withhold_copies)
        for (uint32_t t = gp > BT_NB ? gp - BT_NB : 0; t < gp; ++t)
          if (!mbar_wait(b_full + t % BT_NB, (t / BT_NB) & 1)) err = true;
      if (err || err_wait) atomicExch(a.status, 1);
    }
  } else if (warp == BT_EVAL_THREADS / 32) {
    // ------------------------------------------------------------ MMA warp
    if (lane == 0) {
      uint32_t g = 0;
      for (int64_t k = k0; k < k1 && !err;) {
        const int64_t tile = k / a.nchunk;
        const int64_t c0 = k - tile * a.nchunk;
        const int64_t c1 = min(a.nchunk, c0 + (k1 - k));
        const int64_t s_begin = c0 * a.chunk_tiles, s_end = min(a.ntiles_src, c1 * a.chunk_tiles);
        for (int64_t s = s_begin; s < s_end && !err; ++s, ++g) {
          const int sb = g % BT_NB;
          err = !mbar_wait(b_full + sb, (g / BT_NB) & 1) || !mbar_wait(a_full, g & 1);
          // accumulator buffer g % 2 was last used by tile g - 2, whose fold must have read it
          if (!err && g >= 2) err = !mbar_wait(d_ready + (g & 1), ((g - 2) >> 1) & 1);
          if (err) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dcol = tmem + BT_COL_D + 128 * (g & 1);
          const uint32_t acol = tmem + BT_COL_A;  // C_re hi, C_re lo, C_im hi, C_im lo: 32 columns each
          const uint32_t bbase = su32(smem + BT_B_OFF + sb * BT_SIMG);
          constexpr uint32_t ip = bt_idesc(false), in = bt_idesc(true);
          // B windows: (Q_re; Q_im) and (Q_im; -Q_re) of the hi and lo parts, the second
          // negated by the descriptor.
          const uint32_t ar[2] = {acol + 0, acol + 32};
          const uint32_t ai[2] = {acol + 64, acol + 96};
          const uint32_t bre[2] = {bbase + BT_S_HI, bbase + BT_S_LO};
          const uint32_t bim[2] = {bbase + BT_S_HI + BT_B_MAT, bbase + BT_S_LO + BT_B_MAT};
          // the small cross terms first (lo hi, hi lo), while the accumulator is small, then hi hi
          const int pa[3] = {1, 0, 0}, pb[3] = {0, 1, 0};
          // the first two tiles of a segment start their buffer afresh; later tiles accumulate
          // onto the compensation term that the fold of tile g - 2 left in it
          uint32_t acc_flag = (s - s_begin < 2) ? 0u : 1u;
#pragma unroll
          for (int pp = 0; pp < 3; ++pp) {
#pragma unroll
            for (int ks = 0; ks < BT_S / 8; ++ks) {
              mma_tf32_ta(dcol, ar[pa[pp]] + 8 * ks, smem_desc(bre[pb[pp]] + ks * 256), ip, acc_flag);
              acc_flag = 1u;
              mma_tf32_ta(dcol, ai[pa[pp]] + 8 * ks, smem_desc(bim[pb[pp]] + ks * 256), in, 1u);
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           su32(mma_done + sb))
                       : "memory");
        }
        k = tile * a.nchunk + c1;
      }
      // before the CTA exits (and its tensor memory goes away) the last MMAs must have
      // retired
      const bool err_wait = err;
      if (g > 0 && !mbar_wait(mma_done + (g - 1) % BT_NB, ((g - 1) / BT_NB) & 1)) err = true;
      if (err || err_wait) atomicExch(a.status, 1);
    }
  } else {
    // ------------------------------------------------------------ evaluating warps
    const int m = tid & (BT_M - 1);   // evaluated target row
    const int oct = tid >> 7;         // evaluated sources 8 oct .. 8 oct + 7
    const int lq = warp & 3;          // TMEM lane quarter this warp may access
    const int cb = warp >> 2;         // accumulator column block of 32 folded by this warp
    const int row = lq * 32 + lane;   // accumulator row (target) of this thread
    const int part = cb >> 1;         // 0: real, 1: imaginary
    const int r0 = (cb & 1) * 32;     // first right-hand side of the column block
    const uint32_t tlane = tmem + ((uint32_t)(lq * 32) << 16);
    uint32_t g = 0;
    // Compensated fold of tile gg's accumulator (buffer gg % 2) into the running sum H:
    //   t = H + d,  e = d - (t - H),  H <- t,  buffer <- e
    // so that the next tile accumulating into the buffer carries the rounding error e of
    // this step (Kahan summation, the compensation kept in the tensor accumulator).  After
    // a segment's last fold its sum is H plus the compensations pending in both buffers.
    auto fold = [&](uint32_t gg, bool first) {
      const uint32_t dcol = tlane + BT_COL_D + 128 * (gg & 1) + 32 * cb;
      const uint32_t hcol = tlane + BT_COL_H + 32 * cb;
#pragma unroll
      for (int piece = 0; piece < 2; ++piece) {
        uint32_t d[16], h[16];
        BT_LD8(dcol + 16 * piece, d);
        BT_LD8(dcol + 16 * piece + 8, (d + 8));
        if (!first) {
          BT_LD8(hcol + 16 * piece, h);
          BT_LD8(hcol + 16 * piece + 8, (h + 8));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
          const float2 dv = make_float2(__uint_as_float(d[q]), __uint_as_float(d[q + 1]));
          float2 t, e;
          if (first) {
            t = dv;
            e = make_float2(0.0f, 0.0f);
          } else {
            const float2 hv = make_float2(__uint_as_float(h[q]), __uint_as_float(h[q + 1]));
            t = __fadd2_rn(hv, dv);
            const float2 z = __ffma2_rn(hv, bf2(-1.0f), t);
            e = __ffma2_rn(z, bf2(-1.0f), dv);
          }
          h[q] = __float_as_uint(t.x);
          h[q + 1] = __float_as_uint(t.y);
          d[q] = __float_as_uint(e.x);
          d[q + 1] = __float_as_uint(e.y);
        }
        BT_ST8(hcol + 16 * piece, h);
        BT_ST8(hcol + 16 * piece + 8, (h + 8));
        BT_ST8(dcol + 16 * piece, d);
        BT_ST8(dcol + 16 * piece + 8, (d + 8));
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(d_ready + (gg & 1))) : "memory");
    };
    for (int64_t k = k0; k < k1;) {
      const int64_t tile = k / a.nchunk;
      const int64_t c0 = k - tile * a.nchunk;
      const int64_t c1 = min(a.nchunk, c0 + (k1 - k));
      const int64_t s_begin = c0 * a.chunk_tiles, s_end = min(a.ntiles_src, c1 * a.chunk_tiles);
      const int prob = (int)(tile / a.ntile_t);         // operator of this segment
      const int64_t ltile = tile - (int64_t)prob * a.ntile_t;
      const int64_t ti = ltile * BT_M + m;
      const float4 tp = ti < a.nt ? a.tgt[prob][ti] : make_float4(0.f, 0.f, 0.f, 0.f);
      for (int64_t s = s_begin; s < s_end; ++s, ++g) {
        const int sb = g % BT_NB;
        unsigned char* simg = smem + BT_B_OFF + sb * BT_SIMG;
        const float* hdr = reinterpret_cast<const float*>(simg);
        if (!err) err = !mbar_wait(b_full + sb, (g / BT_NB) & 1);
        // C for (target m, sources 8 oct .. 8 oct + 7), two sources per packed instruction
        float cre[8], cim[8];
        {
          const int j0 = 8 * oct;
          const float4 xa = *reinterpret_cast<const float4*>(hdr + 0 * BT_S + j0);
          const float4 xb = *reinterpret_cast<const float4*>(hdr + 0 * BT_S + j0 + 4);
          const float4 ya = *reinterpret_cast<const float4*>(hdr + 1 * BT_S + j0);
          const float4 yb = *reinterpret_cast<const float4*>(hdr + 1 * BT_S + j0 + 4);
          const float4 za = *reinterpret_cast<const float4*>(hdr + 2 * BT_S + j0);
          const float4 zb = *reinterpret_cast<const float4*>(hdr + 2 * BT_S + j0 + 4);
          float4 nxa = make_float4(0, 0, 0, 0), nxb = nxa, nya = nxa, nyb = nxa, nza = nxa, nzb = nxa;
          if (Ev::kNormal) {
            nxa = *reinterpret_cast<const float4*>(hdr + 3 * BT_S + j0);
            nxb = *reinterpret_cast<const float4*>(hdr + 3 * BT_S + j0 + 4);
            nya = *reinterpret_cast<const float4*>(hdr + 4 * BT_S + j0);
            nyb = *reinterpret_cast<const float4*>(hdr + 4 * BT_S + j0 + 4);
            nza = *reinterpret_cast<const float4*>(hdr + 5 * BT_S + j0);
            nzb = *reinterpret_cast<const float4*>(hdr + 5 * BT_S + j0 + 4);
          }
          const float2 tx = bf2(tp.x), ty = bf2(tp.y), tz = bf2(tp.z);
          const float2 sx[4] = {{xa.x, xa.y}, {xa.z, xa.w}, {xb.x, xb.y}, {xb.z, xb.w}};
          const float2 sy[4] = {{ya.x, ya.y}, {ya.z, ya.w}, {yb.x, yb.y}, {yb.z, yb.w}};
          const float2 sz[4] = {{za.x, za.y}, {za.z, za.w}, {zb.x, zb.y}, {zb.z, zb.w}};
          const float2 qx[4] = {{nxa.x, nxa.y}, {nxa.z, nxa.w}, {nxb.x, nxb.y}, {nxb.z, nxb.w}};
          const float2 qy[4] = {{nya.x, nya.y}, {nya.z, nya.w}, {nyb.x, nyb.y}, {nyb.z, nyb.w}};
          const float2 qz[4] = {{nza.x, nza.y}, {nza.z, nza.w}, {nzb.x, nzb.y}, {nzb.z, nzb.w}};
#pragma unroll
          for (int pr = 0; pr < 4; ++pr) {
            float2 cr2, ci2;
            eval_pair2<Ev>(tx, ty, tz, sx[pr], sy[pr], sz[pr], qx[pr], qy[pr], qz[pr], cr2, ci2);
            cre[2 * pr] = cr2.x;
            cre[2 * pr + 1] = cr2.y;
            cim[2 * pr] = ci2.x;
            cim[2 * pr + 1] = ci2.y;
          }
        }
        uint32_t rh[8], rl[8], ih[8], il[8];
#pragma unroll
        // hi = the value rounded to TF32; lo = the exact FP32 remainder, passed as it is: the
        // MMA reads its leading TF32 bits, and since the remainder's sign does not follow the
        // value's, dropping its low bits adds an unbiased error below 2^-21 of the value
        for (int q = 0; q < 8; ++q) {
          const float h1 = tf32(cre[q]), h2 = tf32(cim[q]);
          rh[q] = __float_as_uint(h1);
          rl[q] = __float_as_uint(cre[q] - h1);
          ih[q] = __float_as_uint(h2);
          il[q] = __float_as_uint(cim[q] - h2);
        }
        {
          // -Q_re (hi for threads 0-255, lo for 256-511), two 16-byte vectors each
          const int part_lo = tid >> 8;
          const int v = (tid & 255) * 2;
          const float4* src = reinterpret_cast<const float4*>(simg + (part_lo ? BT_S_LO : BT_S_HI)) + v;
          float4* dst = reinterpret_cast<float4*>(simg + (part_lo ? BT_S_LO : BT_S_HI) + 2 * BT_B_MAT) + v;
          const float4 q0 = src[0], q1 = src[1];
          dst[0] = make_float4(-q0.x, -q0.y, -q0.z, -q0.w);
          dst[1] = make_float4(-q1.x, -q1.y, -q1.z, -q1.w);
        }
        // the A operand buffer is free once the MMAs of the previous tile have retired
        if (g > 0 && !err) err = !mbar_wait(mma_done + (g - 1) % BT_NB, ((g - 1) / BT_NB) & 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // A operand into tensor memory: this warp's 32 rows, columns 8 oct .. 8 oct + 7
        {
          const uint32_t ta = tlane + BT_COL_A + 8 * oct;
          BT_ST8(ta + 0, rh);
          BT_ST8(ta + 32, rl);
          BT_ST8(ta + 64, ih);
          BT_ST8(ta + 96, il);
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the -Q_re blocks
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(a_full)) : "memory");
        // folds: the previous tile's accumulator (its MMAs retired, waited above) and, on the
        // segment's last tile, this tile's
        const int f_end = (s == s_end - 1) ? 2 : 1;
#pragma unroll 1
        for (int f = (s > s_begin) ? 0 : 1; f < f_end; ++f) {
          const uint32_t gg = g - 1 + f;
          if (f == 1) {
            if (!err) err = !mbar_wait(mma_done + gg % BT_NB, (gg / BT_NB) & 1);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          }
          fold(gg, s - 1 + f == s_begin);
        }
      }
      {
        // the segment's sum in FP64, H + the compensation in the last tile's buffer (+ that
        // in the other buffer, used by the segment's previous tile): the target tile
        // (complete) or its part (partial: the CTA's first segment to slot 2b, a later one
        // to 2b + 1)
        const uint32_t gl = g - 1;
        const bool complete = (c0 == 0 && c1 == a.nchunk);
        const bool other = (s_end - s_begin >= 2);
        const int64_t slot = (k == k0) ? 2 * b : 2 * b + 1;
        const int64_t i = ltile * BT_M + row;
        double2* outp = a.out[prob];
        const uint32_t dcol = tlane + BT_COL_D + 128 * (gl & 1) + 32 * cb;
        const uint32_t ocol = tlane + BT_COL_D + 128 * ((gl & 1) ^ 1) + 32 * cb;
        const uint32_t hcol = tlane + BT_COL_H + 32 * cb;
#pragma unroll 1
        for (int piece = 0; piece < 4; ++piece) {
          uint32_t d[8], h[8], o[8];
          BT_LD8(dcol + 8 * piece, d);
          BT_LD8(hcol + 8 * piece, h);
          if (other) BT_LD8(ocol + 8 * piece, o);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float c = __uint_as_float(d[q]) + (other ? __uint_as_float(o[q]) : 0.0f);
            const double v = (double)__uint_as_float(h[q]) + (double)c;
            const int r = r0 + 8 * piece + q;
            if (complete) {
              if (i < a.nt && r < a.nrhs_out) {
                double* op = reinterpret_cast<double*>(outp + (int64_t)r * a.ld_out + i) + part;
                *op = a.mode ? *op + v : v;
              }
            } else {
              a.slots[slot * (2 * BT_M * BT_R) + ((int64_t)part * BT_R + r) * BT_M + row] = v;
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      }
      k = tile * a.nchunk + c1;
    }
    if (err && lane == 0) atomicExch(a.status, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BT_TMEM_COLS));
}
#undef BT_LD8
#undef BT_ST8

__device__ __forceinline__ int64_t bt_block_of(const BatchArgs& a, int64_t k) {
  int64_t b = (k * a.grid) / a.nitems;
  while (b + 1 < a.grid && bt_begin(a, b + 1) <= k) ++b;
  while (b > 0 && bt_begin(a, b) > k) --b;
  return b;
}

// adds the pieces of target tiles that span several CTAs, in CTA order
__global__ void batch_fixup_kernel(BatchArgs a) {
  const int64_t tile = blockIdx.x;  // global target tile (operator-major)
  const int prob = (int)(tile / a.ntile_t);
  const int64_t ltile = tile - (int64_t)prob * a.ntile_t;
  const int64_t kf = tile * a.nchunk, kl = kf + a.nchunk - 1;
  const int64_t bs = bt_block_of(a, kf), be = bt_block_of(a, kl);
  if (bs == be) return;
  for (int e = threadIdx.x; e < BT_M * a.nrhs_out; e += blockDim.x) {
    const int row = e % BT_M, r = e / BT_M;
    const int64_t i = ltile * BT_M + row;
    if (i >= a.nt) continue;
    double sr = 0.0, si = 0.0;
    for (int64_t bb = bs; bb <= be; ++bb) {
      if (bt_begin(a, bb) == bt_begin(a, bb + 1)) continue;
      const int64_t slot = (bb == bs && bt_begin(a, bb) != kf) ? 2 * bb + 1 : 2 * bb;
      const double* sp = a.slots + slot * (2 * BT_M * BT_R);
      sr += sp[(int64_t)r * BT_M + row];
      si += sp[(int64_t)(BT_R + r) * BT_M + row];
    }
    double2* o = a.out[prob] + (int64_t)r * a.ld_out + i;
    if (a.mode) {
      const double2 v = *o;
      *o = make_double2(v.x + sr, v.y + si);
    } else {
      *o = make_double2(sr, si);
    }
  }
}

// ----------------------------------------------------------------- per-apply images

// One thread per (source tile, source in tile, rhs column): writes the tf32 hi/lo of the
// charge's real and imaginary parts into the tile image; rhs 0 also writes the header.
// G: q~ = -kappa s p/(4 pi);  K: c~ = kappa^2 sigma p/(4 pi) (position header + normal).
__global__ void batch_images_kernel(const double4_32a* __restrict__ ps, const double4_32a* __restrict__ aux,
                                    const int32_t* __restrict__ own, int64_t ns, const double2* __restrict__ x,
                                    int64_t ld_x, int nrhs, int r_base, double kap, int is_k,
                                    unsigned char* __restrict__ img, int64_t ntiles) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ntiles * BT_S * BT_R) return;
  const int r = (int)(e % BT_R);
  const int64_t js = e / BT_R;       // source slot: tile * 16 + j
  const int64_t tile = js / BT_S;
  const int j = (int)(js % BT_S);
  unsigned char* base = img + tile * (int64_t)BT_IMG;
  const bool valid = js < ns;
  double qr = 0.0, qi = 0.0;
  double4_32a y = make_double4_32a(0, 0, 0, 0);
  if (valid) {
    y = ps[js];
    const int rr = r_base + r;
    if (rr < nrhs) {
      const double2 p = x[(int64_t)rr * ld_x + own[js]];
      const double sc = is_k ? kap * kap * aux[js].w / kFourPi : -kap * y.w / kFourPi;
      qr = sc * p.x;
      qi = sc * p.y;
    }
  }
  if (r == 0) {
    float* hd = reinterpret_cast<float*>(base);
    hd[0 * BT_S + j] = -(float)(kap * y.x);
    hd[1 * BT_S + j] = -(float)(kap * y.y);
    hd[2 * BT_S + j] = -(float)(kap * y.z);
    if (is_k && valid) {
      const double4_32a nn = aux[js];
      hd[3 * BT_S + j] = (float)nn.x;
      hd[4 * BT_S + j] = (float)nn.y;
      hd[5 * BT_S + j] = (float)nn.z;
    } else {
      hd[3 * BT_S + j] = 0.0f;
      hd[4 * BT_S + j] = 0.0f;
      hd[5 * BT_S + j] = 0.0f;
    }
  }
  const float fr = (float)qr, fi = (float)qi;
  uint32_t hr, lr, hi, li;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hr) : "f"(fr));
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lr) : "f"(fr - __uint_as_float(hr)));
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(fi));
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(li) : "f"(fi - __uint_as_float(hi)));
  unsigned char* bm = base + BT_HDR;
  const uint32_t o = bt_off(r, j);
  *reinterpret_cast<uint32_t*>(bm + 0 * BT_B_MAT + o) = hr;
  *reinterpret_cast<uint32_t*>(bm + 1 * BT_B_MAT + o) = hi;
  *reinterpret_cast<uint32_t*>(bm + 2 * BT_B_MAT + o) = lr;
  *reinterpret_cast<uint32_t*>(bm + 3 * BT_B_MAT + o) = li;
}

// ----------------------------------------------------------------- host side

// Sets the kernels' shared-memory limit once per device (not during stream capture).
static vsie_status tc_attributes(int device) {
  static unsigned done = 0;  // bit per device
  if (device < 32 && (done >> device) & 1u) return VSIE_OK;
  VSIE_CUDA(cudaFuncSetAttribute(batch_tc_kernel<EvalK>, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM));
  VSIE_CUDA(cudaFuncSetAttribute(batch_tc_kernel<EvalG>, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM));
  if (device < 32) done |= 1u << device;
  return VSIE_OK;
}

// The G (is_k false) or K class of nop operators with equal work shapes, right-hand sides
// r_base .. r_base + 63 of each operator's block x[p] -> y[p]: per-operator charge images,
// then one persistent tensor-core launch over all operators' items and one fix-up launch.
static vsie_status batch_class_multi(vsie_handle* const* hs, int nop, bool is_k, const double2* const* x,
                                     double2* const* y, int nrhs, int r_base, int mode, cudaStream_t st,
                                     int64_t nt_limit = 0, int chunk_tiles = 0) {
  vsie_handle* h0 = hs[0];
  const Sources& S0 = is_k ? h0->K : h0->G;
  if (!S0.n || !h0->n) return VSIE_OK;
  const int64_t ntiles = (S0.n + BT_S - 1) / BT_S;
  const size_t img_bytes = (size_t)ntiles * BT_IMG;
  const int64_t nthr = ntiles * BT_S * BT_R;
  BatchArgs a{};
  a.nprob = nop;
  for (int p = 0; p < nop; ++p) {
    vsie_handle* h = hs[p];
    const Sources& S = is_k ? h->K : h->G;
    if (h->batch.img_bytes < img_bytes) {
      unsigned char* q = nullptr;
      VSIE_TRY(dalloc_t(h, &q, img_bytes));
      h->batch.img = q;
      h->batch.img_bytes = img_bytes;
    }
    const double kap = h->k0 / (2.0 * kPi);
    batch_images_kernel<<<(unsigned)((nthr + 255) / 256), 256, 0, st>>>(S.pos_s, S.aux, S.owner, S.n, x[p], h->n,
                                                                        nrhs, r_base, kap, is_k ? 1 : 0,
                                                                        h->batch.img, ntiles);
    VSIE_CUDA(cudaGetLastError());
    a.tgt[p] = h->tgt32;
    a.img[p] = h->batch.img;
    a.out[p] = y[p] + (int64_t)r_base * h->n;
  }
  a.nt = nt_limit > 0 ? std::min<int64_t>(nt_limit, h0->n) : h0->n;
  a.ntiles_src = ntiles;
  a.ntile_t = (a.nt + BT_M - 1) / BT_M;
  if (chunk_tiles <= 0) chunk_tiles = h0->tune.bt_chunk_tiles > 0 ? h0->tune.bt_chunk_tiles : BT_CHUNK_TILES;
  a.chunk_tiles = chunk_tiles;
  a.nchunk = (ntiles + a.chunk_tiles - 1) / a.chunk_tiles;
  a.nitems = (int64_t)nop * a.ntile_t * a.nchunk;
  a.grid = std::max<int64_t>(1, std::min<int64_t>(h0->num_sms > 0 ? h0->num_sms : 148, a.nitems));
  a.ld_out = h0->n;
  a.nrhs_out = std::min(BT_R, nrhs - r_base);
  a.mode = mode;
  const size_t slot_elems = (size_t)(2 * a.grid) * 2 * BT_M * BT_R;
  if (h0->batch.slot_elems < slot_elems) {
    double* q = nullptr;
    VSIE_TRY(dalloc_t(h0, &q, slot_elems));
    h0->batch.slots = q;
    h0->batch.slot_elems = slot_elems;
  }
  a.slots = h0->batch.slots;
  if (!h0->batch.status) {
    VSIE_TRY(dalloc_t(h0, &h0->batch.status, 1));
    VSIE_CUDA(cudaMemsetAsync(h0->batch.status, 0, sizeof(int), st));
  }
  a.status = h0->batch.status;
  a.withhold_copies = (h0->debug_flags & 1) ? 1 : 0;
  VSIE_TRY(tc_attributes(h0->device));
  if (is_k)
    batch_tc_kernel<EvalK><<<(unsigned)a.grid, BT_ALL_THREADS, BT_SMEM, st>>>(a);
  else
    batch_tc_kernel<EvalG><<<(unsigned)a.grid, BT_ALL_THREADS, BT_SMEM, st>>>(a);
  VSIE_CUDA(cudaGetLastError());
  batch_fixup_kernel<<<(unsigned)(nop * a.ntile_t), 256, 0, st>>>(a);
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

// y[p][:, r] = (far-field sums over the G and K classes of operator p) for all columns r,
// 64 at a time, up to BT_MAXP operators per launch; the operators must have equal numbers
// of collocation points and of G and K sources.
vsie_status far_batched_gk_multi(vsie_handle* const* hs, int nop, const double2* const* x, double2* const* y,
                                 int nrhs, cudaStream_t st) {
  for (int p0 = 0; p0 < nop; p0 += BT_MAXP) {
    const int np = std::min(BT_MAXP, nop - p0);
    vsie_handle* h0 = hs[p0];
    for (int r0 = 0; r0 < nrhs; r0 += BT_R) {
      int mode = 0;
      if (h0->G.n) {
        VSIE_TRY(batch_class_multi(hs + p0, np, false, x + p0, y + p0, nrhs, r0, mode, st));
        mode = 1;
      }
      if (h0->K.n) {
        VSIE_TRY(batch_class_multi(hs + p0, np, true, x + p0, y + p0, nrhs, r0, mode, st));
        mode = 1;
      }
      if (!mode) {
        const int cols = std::min(BT_R, nrhs - r0);
        for (int p = 0; p < np; ++p)
          VSIE_CUDA(cudaMemsetAsync(y[p0 + p] + (int64_t)r0 * h0->n, 0, sizeof(double2) * h0->n * cols, st));
      }
    }
  }
  return VSIE_OK;
}

vsie_status far_batched_gk(vsie_handle* h, const double2* x, double2* y, int nrhs, cudaStream_t st) {
  return far_batched_gk_multi(&h, 1, &x, &y, nrhs, st);
}

// Picks the source tiles per work item of the tensor-core sums by timing 16, 32, 64 and 128
// on a sample of the target tiles (sized to about 3e10 pair evaluations per class and
// candidate) for one block of 64 columns x.
vsie_status batch_autotune(vsie_handle* h, const double2* x, double2* y, cudaStream_t st, int* chunk_tiles,
                           double ms_out[2], int* candidates) {
  static const int cands[] = {16, 32, 64, 128};
  const int64_t ns = h->G.n + h->K.n;
  *chunk_tiles = 0;
  ms_out[0] = ms_out[1] = 0.0;
  if (!ns || !h->n) return VSIE_OK;
  const int64_t nt = std::min<int64_t>(h->n, std::max<int64_t>((int64_t)BT_M * 2 * std::max(h->num_sms, 1),
                                                               (int64_t)(3e10 / (double)ns)));
  cudaEvent_t e0, e1;
  VSIE_CUDA(cudaEventCreate(&e0));
  VSIE_CUDA(cudaEventCreate(&e1));
  float best = 1e30f, dflt = 0.0f;
  int best_c = BT_CHUNK_TILES;
  vsie_status s = VSIE_OK;
  for (int c : cands) {
    float cbest = 1e30f;
    for (int r = 0; r <= 2 && s == VSIE_OK; ++r) {  // the first run warms up
      cudaEventRecord(e0, st);
      int mode = 0;
      if (h->G.n && s == VSIE_OK) {
        s = batch_class_multi(&h, 1, false, &x, &y, 64, 0, mode, st, nt, c);
        mode = 1;
      }
      if (h->K.n && s == VSIE_OK) s = batch_class_multi(&h, 1, true, &x, &y, 64, 0, mode, st, nt, c);
      cudaEventRecord(e1, st);
      if (s == VSIE_OK && cudaEventSynchronize(e1) == cudaSuccess && r > 0) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        cbest = std::min(cbest, ms);
      }
    }
    if (s != VSIE_OK) break;
    ++*candidates;
    if (c == BT_CHUNK_TILES) dflt = cbest;
    if (cbest < best) {
      best = cbest;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  VSIE_TRY(s);
  VSIE_TRY(batch_status(h, st));
  h->tune.bt_chunk_tiles = best_c;
  *chunk_tiles = best_c;
  ms_out[0] = best;
  ms_out[1] = dflt;
  return VSIE_OK;
}

vsie_status batch_status(vsie_handle* h, cudaStream_t st) {
  if (!h->batch.status) return VSIE_OK;
  int flag = 0;
  VSIE_CUDA(cudaMemcpyAsync(&flag, h->batch.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  VSIE_CUDA(cudaStreamSynchronize(st));
  if (flag) {
    cudaMemsetAsync(h->batch.status, 0, sizeof(int), st);
    set_error("batched tensor-core far-field sum: a bounded mbarrier wait expired");
    return VSIE_ERR_CUDA;
  }
  return VSIE_OK;
}

}  // namespace vsie
