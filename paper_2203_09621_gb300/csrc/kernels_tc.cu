// Dual-precision layer product on the sm_103a tensor cores (tcgen05 + TMEM
// + TMA), with the SP2 layer update fused into the epilogue.
//
// What one launch computes (one deep layer of Sec. III, Algorithm 1):
//   square   (job 0):   X  = S0 S0             ~ hi*hi + hi*lo + lo*hi
//                       (Sec. II C, Eq. (S0 tensor core): A + B + B^T)
//   response (job 1+k): X1 = S0 S1_k + S1_k S0 ~ sum of the 3-term dual
//                       products of both orders (Sec. III D,
//                       Eq. (FP32S0S1), Eq. (S0S1 tensor core))
// each accumulated in FP32 in tensor memory, and then
//   S_n = sigma X + (1 - sigma) S_{n-1}      (Eq. (eq:Sn); Alg. 2 and 3)
// written as an FP32 master plus its new hi/lo split (Eq. (DualMat2)).
//
// Symmetry (Sec. III D): every S is symmetric, so the B operand of a row
// block product can be read as a row panel (B[k][j] = B[j][k], "K-major"
// for both operands) and only tiles holding elements with row <= col are
// computed; the epilogue stores each such element at (r, c) and (c, r).
// The response needs both orders S0 S1 and S1 S0 for a tile, which are two
// K passes into the same accumulator.
//
// Kernel structure (persistent, one CTA per SM, 320 threads):
//   warp 0      TMA producer: 4-stage ring of {A_hi, A_lo, B_hi, B_lo}
//               tiles (128x32, 128x32, 256x32, 256x32 16-bit, 64B swizzle)
//   warp 1      TMEM owner and MMA issuer: tcgen05.mma.cta_group::1
//               kind::f16, M = 128, N = 256, K = 16, FP32 accumulate, two
//               256-column accumulators in TMEM (double buffered)
//   warps 2..9  epilogue: two warps per TMEM lane quadrant, one row and one
//               column half per thread; fused update, stores, deterministic
//               FP64 partial norms per tile
// Accumulation in chunks: the tensor core adds each MMA's products into the
// FP32 accumulator with a truncating alignment, so an error that grows with
// the number of MMAs folded into one accumulator (and is biased) would
// build up over K = 3n terms.  The K sequence of a tile is therefore cut into
// chunks of `chunk` stages (default 256 K-elements); each chunk starts a
// fresh TMEM accumulator and the epilogue warps add the chunk results in
// FP32 with round-to-nearest in registers.  The two TMEM accumulators are
// used alternately, so the MMA of the next chunk overlaps that summation.
// Every mbarrier wait is bounded in time; on expiry the CTA raises
// State::timeout_flag, drains its copies in flight (bounded), frees TMEM and
// returns, and the host reports DMPT_ETIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <mutex>
#include <type_traits>

#include "dmpt_internal.cuh"

namespace dmpt {
namespace tc {

constexpr int BM = 128;          // rows per tile (TMEM lanes)
constexpr int BN = 256;          // columns per tile
constexpr int BK = 32;           // K elements per stage (64 B rows)
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;   // 8 KB
constexpr int B_BYTES = BN * BK * 2;   // 16 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // 48 KB
constexpr int TMEM_COLS = 512;   // two accumulators of BN columns
constexpr int EPI_WARPS = 8;     // two per TMEM lane quadrant (column halves)
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int EPI_WARP0 = 2;     // epilogue = warps 2 .. 9
constexpr int NUM_THREADS = 64 + EPI_THREADS;
// Epilogue scratch: a 2560-byte transpose buffer per epilogue warp (32 rows
// of 20 words); it shares its space with the reduction array of the tile's
// partial sums (EPI_THREADS x 4 doubles), which is used only after every
// epilogue warp has left its tile epilogue.
constexpr int EPI_SCRATCH = EPI_WARPS * 32 * 20 * 4;
static_assert(EPI_SCRATCH >= EPI_THREADS * 4 * 8, "reduction array fits the scratch");
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /* align */ + 1024 /* barriers etc */ +
                           EPI_SCRATCH;
constexpr int DEFAULT_CHUNK_K = 256;  // K elements per tensor-memory accumulation chunk

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
      "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]),
      "f"(v[15])
      : "memory");
}

// ---------------------------------------------------------------------------
// PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false when `limit_ns` passes or another role of this CTA
// has aborted.  On expiry it raises both abort flags.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns,
                                          volatile int* abort_smem, int* timeout_global) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  uint32_t it = 0;
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((++it & 255) == 0) {
      if (*abort_smem) return false;
      if (gtimer() - t0 > limit_ns) {
        *abort_smem = 1;
        atomicExch(timeout_global, 1);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor, K-major operand with 64-byte swizzle:
// rows of 64 B, 8-row groups 512 B apart (SBO), version 1, layout 4.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // LBO (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;    // SBO
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)4 << 61;             // SWIZZLE_64B
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A/B = F16 (0) or BF16 (1),
// both K-major, N = 256, M = 128.
__host__ __device__ constexpr uint32_t make_idesc(int ab_type) {
  return (1u << 4) | ((uint32_t)ab_type << 7) | ((uint32_t)ab_type << 10) |
         ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// FP16 / BF16 rounding (round to nearest even) used by the dual split.
template <bool BF>
struct Cvt;
template <>
struct Cvt<false> {
  using T = __half;
  static __device__ __forceinline__ T to(float x) { return __float2half_rn(x); }
  static __device__ __forceinline__ float from(T h) { return __half2float(h); }
};
template <>
struct Cvt<true> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ T to(float x) { return __float2bfloat16_rn(x); }
  static __device__ __forceinline__ float from(T h) { return __bfloat162float(h); }
};

// AND of a predicate over the epilogue threads (named barrier 1).
__device__ __forceinline__ int epi_all(int pred) {
  int out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 q, %1, 0;\n\t"
      "bar.red.and.pred p, 1, %2, q;\n\t"
      "selp.s32 %0, 1, 0, p;\n\t}"
      : "=r"(out)
      : "r"(pred), "n"(EPI_THREADS)
      : "memory");
  return out;
}
__device__ __forceinline__ void epi_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
}

// ---------------------------------------------------------------------------
// Work items: (job, tile).  Tiles: 128-row block I and 256-column block J
// with I <= 2J + 1 (the tile holds some element with row <= col).  Tile t
// is J-major: tiles of column block J are t = J(J+1) ... J(J+1) + 2J + 1.

__host__ __device__ inline int64_t num_tiles(int64_t Np) {
  const int64_t tj = Np / BN;
  return tj * (tj + 1);
}
__device__ __forceinline__ void tile_coords(int64_t t, int* I, int* J) {
  int j = (int)((sqrt(4.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((int64_t)(j + 1) * (j + 2) <= t) ++j;
  while ((int64_t)j * (j + 1) > t) --j;
  *J = j;
  *I = (int)(t - (int64_t)j * (j + 1));
}

// Jobs of a layer as a bit mask: bit 0 = square, bit 1 + j = response j.
// Item order: responses (ascending j) first, then the square.
__device__ __forceinline__ int job_at(uint32_t mask, int idx) {
  const uint32_t resp = mask & ~1u;
  const int nresp = __popc(resp);
  if (idx >= nresp) return 0;
  uint32_t m = resp;
  for (int i = 0; i < idx; ++i) m &= m - 1;  // drop the lowest set bits
  return __ffs(m) - 1;
}

// Jobs of a layer: 0 = square of S0; 1 + (o - 1) k1 + d = the order-o term
// of direction d (o = 1 .. order, d = 0 .. k1 - 1; k1 = first-order
// directions), whose activation is (Sec. III A, Eq. (S_n detailed))
//   S0 S_o + S_o S0 + sum_{a=1}^{o-1} S_a S_{o-a}
// in o + 1 K passes: pass 0 = S0 S_o, pass 1 = S_o S0, pass p >= 2 =
// S_{p-1} S_{o-p+1} (order 1: S0 S1, S1 S0; order 2 adds S1 S1).
// The job id is also the matrix slot of the result.
__device__ __forceinline__ int job_order(int job, int k1) { return 1 + (job - 1) / k1; }
__device__ __forceinline__ int job_passes(int job, int k1) {
  return job == 0 ? 1 : (job <= k1 ? 2 : 1 + job_order(job, k1));
}
// slot of the order-a term (a >= 1) of the direction of job `job`
__device__ __forceinline__ int job_slot(int job, int a, int k1) {
  return 1 + (a - 1) * k1 + (job - 1) % k1;
}
// operand slots (A, B) of pass `pass` of job `job`
__device__ __forceinline__ void job_operands(int job, int pass, int k1, int* mA, int* mB) {
  if (job == 0) {
    *mA = 0;
    *mB = 0;
  } else if (pass == 0) {
    *mA = 0;
    *mB = job;
  } else if (pass == 1) {
    *mA = job;
    *mB = 0;
  } else {
    *mA = job_slot(job, pass - 1, k1);
    *mB = job_slot(job, job_order(job, k1) - pass + 1, k1);
  }
}
// exact power-of-two unscale of a pass p >= 2 product (operands scaled by
// 2^e of their slots)
__device__ __forceinline__ float cross_unscale(const State* st, int job, int pass, int k1) {
  int mA, mB;
  job_operands(job, pass, k1, &mA, &mB);
  return ldexpf(1.0f, -(st->s1_exp_cur[mA - 1] + st->s1_exp_cur[mB - 1]));
}
// K-pass of accumulation chunk c (chunks never straddle passes); the
// producer of the pair kernel runs the passes backwards in odd rounds
__device__ __forceinline__ int chunk_pass(int c, int cpp, int passes, bool rev) {
  const int p = c / cpp;
  return rev ? passes - 1 - p : p;
}

// Operand slice of matrix m: S0 comes from the slice the control block
// names (ping-pong slot, or a tape slice when the S0 states are kept for the
// adjoint); S1_j from its ping-pong slot.
__device__ __forceinline__ int zop(int m, int buf, int part, int k, int z0) {
  return m == 0 ? z0 + part : zslice(buf, m, part, k);
}

// Bit pattern of a 16-bit float (FP16 or BF16).
template <class H16>
__device__ __forceinline__ uint32_t h16_bits(H16 x) {
  return (uint32_t)(*reinterpret_cast<const uint16_t*>(&x));
}

// Rolled tile epilogue of one thread: its row r, columns c0 .. c0 + 127 of a
// pair tile, whose sums the caller has written to tensor memory at ta_sum.
// Forms S_new = sigma X + (1 - sigma) S_old (Eq. (eq:Sn) / Eq. (dB)), its
// FP16/BF16 hi/lo split (Sec. II C), the partial sums (||S_new||_F^2 with
// TwoSum compensation, ||S_old - X||_F^2, trace, non-finite count) and stores
// each owned element (column >= row).  OFF: the tile is off the diagonal
// (every column > every row).
//
// Memory access pattern.  A warp holds 32 consecutive rows (one per lane)
// and the same columns, so an access down a column (lane = row) is one
// contiguous segment while an access along its rows touches 32 lines.
//  * The FP32 master is kept in one orientation only: element (r, c),
//    c >= r, at (c, r) (the lower triangle with the diagonal), written and
//    read down the columns.  S_old[r][c] is read there, 16 columns per batch
//    of loads; the next batch is loaded while the current one is stored.
//    The readers of a whole master (outputs, checkpoint reloads) take
//    element (r, c) from (max(r, c), min(r, c)).
//  * The 16-bit operand copies, which the tensor maps read as row panels,
//    are stored in both orientations: the mirror (c, r) down the columns,
//    and (r, c) through this warp's transpose buffer `xp` in shared memory
//    (32 rows of XP_STRIDE words; 16 columns at a time): each lane writes
//    its row, then the warp stores 4 rows x 32 B (hi, lo) per instruction.
//    The row stride of 20 words keeps both the 16-byte row writes and the
//    column-pair reads free of bank conflicts.
// The sums run over the columns in ascending order, so every thread's
// partial sums do not depend on the memory access pattern.
constexpr int XP_STRIDE = 20;                       // words per buffer row
constexpr int XP_WARP_BYTES = 32 * XP_STRIDE * 4;   // 2560 B per epilogue warp
static_assert(EPI_WARPS * XP_WARP_BYTES == EPI_SCRATCH, "transpose buffers");
template <class CV, bool OFF, int NG = 8>   // NG groups of 16 columns per thread row
__device__ __forceinline__ void rolled_tile_epilogue(
    const uint32_t ta_sum, const float* __restrict__ Sold, float* Snew, typename CV::T* hi_new,
    typename CV::T* lo_new, uint32_t* xp, const int lane, const int64_t Np, const int r,
    const int c0, const float sg, const float om, const float scale_new, const bool write,
    float& fn_s, float& fn_c, float& fd, float& trf, int& bad) {
  const int r0 = r - lane;   // row of lane 0
  const int np = (int)Np;
  // element (c, r) of the tile's columns at col_base + (c - c0) * np; element
  // (r0 + i, c) at row_base + i * np + (c - c0)  (32-bit offsets)
  const size_t col_base = (size_t)c0 * Np + r;
  const size_t row_base = (size_t)r0 * Np + c0;
  const float* Sc = Sold + col_base;
  float* Snc = Snew + col_base;
  uint16_t* hic = reinterpret_cast<uint16_t*>(hi_new) + col_base;
  uint16_t* loc = reinterpret_cast<uint16_t*>(lo_new) + col_base;
  uint16_t* hir = reinterpret_cast<uint16_t*>(hi_new) + row_base;
  uint16_t* lor = reinterpret_cast<uint16_t*>(lo_new) + row_base;
  float olds[16];   // S_old of the current 16 columns; the next 16 are loaded
                    // while the current ones are stored
#pragma unroll
  for (int q = 0; q < 16; ++q) olds[q] = __ldg(Sc + q * np);
#pragma unroll 1
  for (int g16 = 0; g16 < NG; ++g16) {
    uint32_t xs[16];
    tmem_ld16(ta_sum + 16 * g16, xs);
    const int cb16 = c0 + 16 * g16;
    // the hi/lo bits stay in registers, packed in column pairs, until the
    // group's values are formed
    uint32_t hp[8], lp[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) hp[i] = lp[i] = 0u;
#pragma unroll
    for (int gg = 0; gg < 4; ++gg) {
      const int cb = cb16 + 4 * gg;
      if (!OFF && r > cb + 3) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int e = 4 * gg + i;
        const float xv = __uint_as_float(xs[e]);
        const int c = cb + i;
        const bool own = OFF || c >= r;
        const float w = (!OFF && c == r) ? 1.0f : 2.0f;
        bad += (own && !isfinite(xv)) ? 1 : 0;
        const float old = olds[e];
        const float dd = old - xv;
        fd = own ? fmaf(w * dd, dd, fd) : fd;
        const float n1 = sg * xv + om * old;
        if (own && write) {
          const float p = w * n1 * n1;
          const float ee = w * fmaf(n1, n1, -n1 * n1);
          const float tt = fn_s + p;
          const float bp = tt - fn_s;
          fn_c += (fn_s - (tt - bp)) + (p - bp) + ee;
          fn_s = tt;
          if (!OFF && c == r) trf += n1;
        }
        const float y = n1 * scale_new;
        const typename CV::T h = CV::to(y);
        const uint32_t hbits = h16_bits(h);
        const uint32_t lbits = h16_bits(CV::to(y - CV::from(h)));
        hp[e >> 1] |= hbits << (16 * (e & 1));
        lp[e >> 1] |= lbits << (16 * (e & 1));
        if (write && own) {   // (c, r), down the column
          const int m = (c - c0) * np;
          Snc[m] = n1;
          if (OFF || c > r) {   // the 16-bit mirror; the diagonal goes with the rows
            hic[m] = (uint16_t)hbits;
            loc[m] = (uint16_t)lbits;
          }
        }
      }
    }
    if (g16 < NG - 1) {
#pragma unroll
      for (int q = 0; q < 16; ++q) olds[q] = __ldg(Sc + (16 * (g16 + 1) + q) * np);
    }
    if (!write) continue;
    // ---- 16-bit copies in the row direction (r, c) through the transpose buffer
    uint4* xr4 = reinterpret_cast<uint4*>(xp + lane * XP_STRIDE);
    xr4[0] = make_uint4(hp[0], hp[1], hp[2], hp[3]);
    xr4[1] = make_uint4(hp[4], hp[5], hp[6], hp[7]);
    xr4[2] = make_uint4(lp[0], lp[1], lp[2], lp[3]);
    xr4[3] = make_uint4(lp[4], lp[5], lp[6], lp[7]);
    __syncwarp();
#pragma unroll
    for (int sidx = 0; sidx < 8; ++sidx) {
      const int i = 8 * (sidx >> 1) + (sidx & 1) + 2 * (lane >> 3);   // rows i, +2, +4, +6
      const int m = lane & 7;                                           // column pair
      const uint32_t vh = xp[i * XP_STRIDE + m];
      const uint32_t vl = xp[i * XP_STRIDE + 8 + m];
      const int rr = r0 + i, c = cb16 + 2 * m;
      const int o = i * np + (c - c0);
      if (OFF || c >= rr) {
        *reinterpret_cast<uint32_t*>(hir + o) = vh;
        *reinterpret_cast<uint32_t*>(lor + o) = vl;
      } else if (c + 1 >= rr) {
        hir[o + 1] = (uint16_t)(vh >> 16);
        lor[o + 1] = (uint16_t)(vl >> 16);
      }
    }
    __syncwarp();
  }
}

template <bool BF16>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    layer_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                    State* st, float* __restrict__ master, uint16_t* __restrict__ ops,
                    int64_t Np, int k, double* __restrict__ partials, int64_t ptiles,
                    uint64_t limit_ns, int chunk, int inject_stall) {
  using CV = Cvt<BF16>;
  using H16 = typename CV::T;
  extern __shared__ uint8_t smem_raw[];
  if (st->done) return;

  // ---- plan of this layer (identical in every CTA)
  uint32_t jmask = st->plan_square ? 1u : 0u;
  for (int j = 0; j < k; ++j)
    if (st->plan_resp[j]) jmask |= 1u << (1 + j);
  const int njobs = __popc(jmask);
  if (njobs == 0) return;
  const int cur0 = st->cur0;
  const int sigma = st->sigma_cur;
  const int write0 = st->plan_write0;
  const int s0e = st->s0_exp;
  const int z0c = st->z0_cur, z0n = st->z0_next;
  const int k1 = st->order >= 2 ? st->k1 : k;   // first-order directions

  const int64_t tiles = num_tiles(Np);
  const int64_t items = tiles * njobs;
  const int kblocks = (int)(Np / BK);

  // ---- shared memory carve-up (1024-aligned stage ring)
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t ring = base;
  uint8_t* misc = gbase + STAGES * STAGE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(misc);  // full, empty, tfull, tempty, drain
  const uint32_t bar_full = smem_u32(bars);
  const uint32_t bar_empty = bar_full + 8 * STAGES;
  const uint32_t bar_tfull = bar_empty + 8 * STAGES;
  const uint32_t bar_tempty = bar_tfull + 8 * 2;
  const uint32_t bar_drain = bar_tempty + 8 * 2;
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(misc + 128);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(misc + 136);
  double* red = reinterpret_cast<double*>(misc + 1024);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_tfull + 8 * b, 1);
      mbar_init(bar_tempty + 8 * b, EPI_WARPS);  // one arrive per epilogue warp
    }
    mbar_init(bar_drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem_base = *tmem_slot;
  int* timeout_global = &st->timeout_flag;

  if (warp == 0) {
    // ================= TMA producer =================
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int inflight = 0;  // stages issued whose completion this thread has not observed
      bool ok = true;
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int job = job_at(jmask, (int)(it / tiles));
        int I, J;
        tile_coords(it % tiles, &I, &J);
        const int passes = job_passes(job, k1);
        for (int pass = 0; pass < passes && ok; ++pass) {
          // A = rows I of slot mA, B = rows J of slot mB (B[k][j] = B[j][k])
          int mA, mB;
          job_operands(job, pass, k1, &mA, &mB);
          const int bufA = mA == 0 ? cur0 : st->cur1[mA - 1];
          const int bufB = mB == 0 ? cur0 : st->cur1[mB - 1];
          const int zAh = zop(mA, bufA, 0, k, z0c), zAl = zop(mA, bufA, 1, k, z0c);
          const int zBh = zop(mB, bufB, 0, k, z0c), zBl = zop(mB, bufB, 1, k, z0c);
          for (int kb = 0; kb < kblocks; ++kb) {
            if (!mbar_wait(bar_empty + 8 * stage, phase ^ 1, limit_ns, abort_flag,
                           timeout_global)) {
              ok = false;
              break;
            }
            const uint32_t sA = ring + stage * STAGE_BYTES;
            const uint32_t fb = bar_full + 8 * stage;
            mbar_expect_tx(fb, STAGE_BYTES);
            tma_load_3d(sA, &mapA, kb * BK, I * BM, zAh, fb);
            tma_load_3d(sA + A_BYTES, &mapA, kb * BK, I * BM, zAl, fb);
            tma_load_3d(sA + 2 * A_BYTES, &mapB, kb * BK, J * BN, zBh, fb);
            tma_load_3d(sA + 2 * A_BYTES + B_BYTES, &mapB, kb * BK, J * BN, zBl, fb);
            inflight = inflight < STAGES ? inflight + 1 : STAGES;
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1;
            }
          }
        }
      }
      if (!ok) {
        // drain: wait (bounded) until the copies already issued have landed
        int s = stage;
        uint32_t ph = phase;
        for (int i = 0; i < inflight; ++i) {
          if (--s < 0) {
            s = STAGES - 1;
            ph ^= 1;
          }
          const uint64_t t0 = gtimer();
          while (!mbar_try_wait(bar_full + 8 * s, ph) && gtimer() - t0 < limit_ns) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ================= MMA issuer =================
    // The K sequence of an item (all passes) is cut into chunks of `chunk`
    // stages; each chunk accumulates from zero into one of the two TMEM
    // accumulators and is summed by the epilogue in FP32 on the CUDA cores.
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc(BF16 ? 1 : 0);
      int stage = 0;
      uint32_t phase = 0;
      int ab = 0;
      uint32_t abphase = 0;
      // test hook: wait on a barrier nothing arrives on, so that the bounded
      // waits of every role run out and the timeout path is exercised
      bool ok = !(inject_stall &&
                  !mbar_wait(bar_drain, 0, limit_ns, abort_flag, timeout_global));
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int job = job_at(jmask, (int)(it / tiles));
        const int nst = job_passes(job, k1) * kblocks;
        uint32_t d = 0, acc = 0;
        int sp = 0;   // stage within its K pass
        int cp = 0;   // stage within its accumulation chunk
        for (int si = 0; si < nst; ++si) {
          if (cp == 0) {
            if (!mbar_wait(bar_tempty + 8 * ab, abphase ^ 1, limit_ns, abort_flag,
                           timeout_global)) {
              ok = false;
              break;
            }
            fence_after();
            d = tmem_base + (uint32_t)(ab * BN);
            acc = 0;
          }
          if (!mbar_wait(bar_full + 8 * stage, phase, limit_ns, abort_flag, timeout_global)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t sA = ring + stage * STAGE_BYTES;
          const uint64_t ah = sw64_desc(sA), al = sw64_desc(sA + A_BYTES);
          const uint64_t bh = sw64_desc(sA + 2 * A_BYTES);
          const uint64_t bl = sw64_desc(sA + 2 * A_BYTES + B_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t off = (uint64_t)((kk * 32) >> 4);  // 16 elements = 32 B
            mma_f16(d, ah + off, bh + off, idesc, acc);        // hi * hi
            acc = 1;
            mma_f16(d, ah + off, bl + off, idesc, 1);          // hi * lo
            mma_f16(d, al + off, bh + off, idesc, 1);          // lo * hi
          }
          mma_commit(bar_empty + 8 * stage);  // frees the stage when these MMAs finish
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
          const bool chunk_end = cp == chunk - 1 || sp == kblocks - 1;
          if (++cp == chunk || sp == kblocks - 1) cp = 0;
          if (++sp == kblocks) sp = 0;
          if (chunk_end) {
            mma_commit(bar_tfull + 8 * ab);  // chunk accumulator ready
            if (++ab == 2) {
              ab = 0;
              abphase ^= 1;
            }
          }
        }
      }
      // wait (bounded) until every MMA this thread issued has completed, so
      // TMEM is idle before it is freed
      mma_commit(bar_drain);
      const uint64_t t0 = gtimer();
      while (!mbar_try_wait(bar_drain, 0) && gtimer() - t0 < limit_ns) {
      }
    }
  } else if (warp >= EPI_WARP0) {
    // ================= epilogue (warps 4..11) =================
    // Thread = one row of the tile (TMEM lane) and one half of its columns.
    const int q = warp & 3;                 // TMEM lane quadrant of this warp
    const int half = (warp - EPI_WARP0) >> 2;  // column half: 0 -> 0..127, 1 -> 128..255
    const int rloc = 32 * q + lane;         // row within the tile
    const int et = threadIdx.x - 32 * EPI_WARP0;  // 0..255
    const size_t mat = (size_t)Np * Np;
    const uint32_t tlane = (uint32_t)(32 * q) << 16;
    int ab = 0;
    uint32_t abphase = 0;
    bool alive = true;
    const bool crev = false;   // this kernel always runs the passes forwards
    for (int64_t it = blockIdx.x; it < items && alive; it += gridDim.x) {
      const int job = job_at(jmask, (int)(it / tiles));
      const int passes = job_passes(job, k1);
      const int cpp = (kblocks + chunk - 1) / chunk;   // chunks per pass
      const int nchunks = passes * cpp;
      // exact power-of-two unscale of the products of passes 0 and 1
      // (passes >= 2 of higher-order terms: cross_unscale)
      const float u01 = ldexpf(1.0f, -(s0e + (job == 0 ? s0e : st->s1_exp_cur[job - 1])));

      // ---- sum the chunk accumulators in FP32 (round to nearest)
      float sum[128];
#pragma unroll
      for (int i = 0; i < 128; ++i) sum[i] = 0.0f;
      for (int ch = 0; ch < nchunks; ++ch) {
        const bool ok =
            mbar_wait(bar_tfull + 8 * ab, abphase, limit_ns, abort_flag, timeout_global);
        // all epilogue threads take the same branch (warp-collective
        // tcgen05.ld follows)
        if (!epi_all(ok && !*abort_flag)) {
          alive = false;
          break;
        }
        fence_after();
        const uint32_t ta = tmem_base + tlane + (uint32_t)(ab * BN + half * 128);
        const int pc = chunk_pass(ch, cpp, passes, crev);
        const float u = pc < 2 ? u01 : cross_unscale(st, job, pc, k1);
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          uint32_t x[16];
          tmem_ld16(ta + 16 * cc, x);
#pragma unroll
          for (int i = 0; i < 16; ++i) sum[16 * cc + i] = fmaf(__uint_as_float(x[i]), u, sum[16 * cc + i]);
        }
        if (ch + 1 == nchunks) break;   // keep the last chunk's buffer
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_tempty + 8 * ab);
        if (++ab == 2) {
          ab = 0;
          abphase ^= 1;
        }
      }
      if (!alive) break;
      // the tile's sums go back into its last chunk's buffer
      const uint32_t ta_sum = tmem_base + tlane + (uint32_t)(ab * BN + half * 128);
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) tmem_st16(ta_sum + 16 * cc, sum + 16 * cc);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");

      // ---- fused layer update, split and stores
      const int64_t t = it % tiles;
      int I, J;
      tile_coords(t, &I, &J);
      const int curj = job == 0 ? cur0 : st->cur1[job - 1];
      const int e_new = job == 0 ? s0e : st->s1_exp_next[job - 1];
      const float scale_new = ldexpf(1.0f, e_new);   // exact power of two
      const float sg = (float)sigma, om = 1.0f - (float)sigma;
      const bool write = job != 0 || write0;
      const int r = I * BM + rloc;
      const int c0 = J * BN + half * 128;
      const float* Sold = master + (size_t)(curj * (1 + k) + job) * mat;
      float* Snew = master + (size_t)((curj ^ 1) * (1 + k) + job) * mat;
      const int zh_new = job == 0 ? z0n : zslice(curj ^ 1, job, 0, k);
      H16* hi_new = reinterpret_cast<H16*>(ops) + (size_t)zh_new * mat;
      H16* lo_new = reinterpret_cast<H16*>(ops) + (size_t)(zh_new + 1) * mat;

      // Partial norms in FP32 with compensation (GB300's FP64 rate is a small
      // fraction of its FP32 rate): ||S_new||^2 feeds the Alg. 2 test, so its
      // products are split exactly (FMA) and summed with TwoSum; the
      // FroErr sums only enter ratio tests and use plain FP32.
      float fn_s = 0.0f, fn_c = 0.0f, fd = 0.0f, trf = 0.0f;
      int bad = 0;
      uint32_t* xp = reinterpret_cast<uint32_t*>(misc + 1024) +
                     (warp - EPI_WARP0) * (XP_WARP_BYTES / 4);
      if (I * BM + BM - 1 < J * BN)   // every column of the tile above every row
        rolled_tile_epilogue<CV, true>(ta_sum, Sold, Snew, hi_new, lo_new, xp, lane, Np, r, c0,
                                       sg, om, scale_new, write, fn_s, fn_c, fd, trf, bad);
      else
        rolled_tile_epilogue<CV, false>(ta_sum, Sold, Snew, hi_new, lo_new, xp, lane, Np, r, c0,
                                        sg, om, scale_new, write, fn_s, fn_c, fd, trf, bad);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_tempty + 8 * ab);
      if (++ab == 2) {
        ab = 0;
        abphase ^= 1;
      }
      epi_sync();   // the reduction array overlays the transpose buffers
      // deterministic tile reduction over the 256 epilogue threads (FP64)
      red[0 * EPI_THREADS + et] = (double)trf;
      red[1 * EPI_THREADS + et] = (double)fn_s + (double)fn_c;
      red[2 * EPI_THREADS + et] = (double)fd;
      red[3 * EPI_THREADS + et] = (double)bad;
      epi_sync();
      for (int s = EPI_THREADS / 2; s > 0; s >>= 1) {
        if (et < s) {
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) red[qq * EPI_THREADS + et] += red[qq * EPI_THREADS + et + s];
        }
        epi_sync();
      }
      if (et == 0) {
        double* p = partials + ((size_t)job * ptiles + t) * kNQ;
        p[kQTrace] = red[0];
        p[kQFroNew] = red[EPI_THREADS];
        p[kQFroDiff] = red[2 * EPI_THREADS];
        p[kQBad] = red[3 * EPI_THREADS];
      }
      epi_sync();
    }
  }

  // ---- teardown: everyone done (or aborted); free TMEM
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS));
  }
}

// ---------------------------------------------------------------------------
// CTA-pair variant (cta_group::2).  A cluster of two CTAs computes a
// 256 x 256 tile: CTA r holds rows 128 r .. 128 r + 127 of A and B rows
// (output columns) 128 r .. 128 r + 127; the leader (rank 0) issues
// M = 256, N = 256 MMAs that read A from each CTA's own shared memory and B
// from both, and each CTA's tensor memory receives its 128 rows of the
// accumulator.  Per SM this halves the operand bytes loaded per MMA
// (32 KB per 6 MMAs instead of 48 KB).
//   full[s]   leader only: leader producer's expect_tx(64 KB); both CTAs'
//             TMA loads complete their bytes on it
//   empty[s]  each CTA: the leader's MMA commit arrives on both (multicast)
//   tfull[b]  each CTA: leader's commit, multicast
//   tempty[b] leader only: 16 arrivals (8 epilogue warps per CTA)

constexpr int P_STAGES = 6;
constexpr int P_STAGE_BYTES = 2 * A_BYTES + 2 * A_BYTES;   // A hi/lo + B-half hi/lo: 32 KB
constexpr int P_SMEM_BYTES = P_STAGES * P_STAGE_BYTES + 1024 + 1024 + EPI_SCRATCH;

__host__ __device__ inline int64_t num_pair_tiles(int64_t Np) {
  const int64_t tj = Np / BN;
  return tj * (tj + 1) / 2;
}
// pair tile t -> (I2, J), I2 <= J, J-major
__device__ __forceinline__ void pair_tile_coords(int64_t t, int* I2, int* J) {
  int j = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((int64_t)(j + 1) * (j + 2) / 2 <= t) ++j;
  while ((int64_t)j * (j + 1) / 2 > t) --j;
  *J = j;
  *I2 = (int)(t - (int64_t)j * (j + 1) / 2);
}

// Banded order of the pair tiles (I2 <= J): column blocks are grouped into
// bands of `band` blocks; inside a band the tiles run I2-major, so the pairs
// working at the same time cover a compact block of rows and columns and
// share their operand panels in L2.  band <= 0 keeps the plain J-major order.
__device__ __forceinline__ void pair_tile_banded(int64_t t, int tj, int band, int* I2, int* J) {
  if (band <= 0) {
    pair_tile_coords(t, I2, J);
    return;
  }
  int J0 = 0;
  while (true) {
    const int w = tj - J0 < band ? tj - J0 : band;
    const int64_t cnt = (int64_t)J0 * w + (int64_t)w * (w + 1) / 2;   // tiles in this band
    if (t < cnt || J0 + w >= tj) {
      if (t < (int64_t)J0 * w) {          // rows above the band's diagonal block
        *I2 = (int)(t / w);
        *J = J0 + (int)(t % w);
        return;
      }
      int64_t u = t - (int64_t)J0 * w;    // upper triangle of the w x w diagonal block
      int r = 0;
      while (u >= w - r) {
        u -= w - r;
        ++r;
      }
      *I2 = J0 + r;
      *J = J0 + r + (int)u;
      return;
    }
    t -= cnt;
    J0 += w;
  }
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(addr), "r"(rank));
  return out;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
// Arrive on a barrier of another CTA of the cluster.  Release at CTA scope
// only: the arrival signals that this warp's tensor-memory reads are done
// (tcgen05.wait::ld has returned), not that its global stores are visible,
// so no cluster-scope fence (which would wait for the previous tile's
// stores) is needed.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* map, int x, int y,
                                                 int z, uint32_t leader_bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(leader_bar)
      : "memory");
}
__device__ __forceinline__ void mma_f16_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                             uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
  const uint16_t mask = 0x3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar), "h"(mask)
      : "memory");
}
__host__ __device__ constexpr uint32_t make_idesc_m256(int ab_type) {
  return (1u << 4) | ((uint32_t)ab_type << 7) | ((uint32_t)ab_type << 10) |
         ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}

// Position in the shared-memory stage ring (stage index and phase bit) or
// in the two tensor-memory accumulators (buffer and phase bit).
struct RingPos {
  int idx = 0;
  uint32_t phase = 0;
  __device__ __forceinline__ void next(int size) {
    if (++idx == size) {
      idx = 0;
      phase ^= 1;
    }
  }
};

// TMA producer of a pair kernel, one work item: the item's passes over its
// K blocks (backwards when `rev`), each stage the hi and lo halves of this
// CTA's A rows and B rows, signalled on the pair leader's full barrier.
// False when a bounded wait expired or the CTA aborted.
__device__ __forceinline__ bool produce_item(RingPos& rg, const CUtensorMap* map,
                                             const State* st, int job, int passes, int k,
                                             int k1, int cur0, int z0c, int rowA, int rowB,
                                             int kblocks, bool rev, bool leader, uint32_t ring,
                                             uint32_t bar_full, uint32_t bar_empty,
                                             uint32_t lead_full, uint64_t limit_ns,
                                             volatile int* abort_flag, int* timeout_global) {
  for (int pp = 0; pp < passes; ++pp) {
    const int pass = rev ? passes - 1 - pp : pp;
    int mA, mB;
    job_operands(job, pass, k1, &mA, &mB);
    const int bufA = mA == 0 ? cur0 : st->cur1[mA - 1];
    const int bufB = mB == 0 ? cur0 : st->cur1[mB - 1];
    const int zAh = zop(mA, bufA, 0, k, z0c), zAl = zop(mA, bufA, 1, k, z0c);
    const int zBh = zop(mB, bufB, 0, k, z0c), zBl = zop(mB, bufB, 1, k, z0c);
    for (int kq = 0; kq < kblocks; ++kq) {
      const int kb = rev ? kblocks - 1 - kq : kq;
      if (!mbar_wait(bar_empty + 8 * rg.idx, rg.phase ^ 1, limit_ns, abort_flag, timeout_global))
        return false;
      const uint32_t sA = ring + rg.idx * P_STAGE_BYTES;
      if (leader) mbar_expect_tx(bar_full + 8 * rg.idx, 2 * P_STAGE_BYTES);
      const uint32_t fb = lead_full + 8 * rg.idx;
      tma_load_3d_pair(sA, map, kb * BK, rowA, zAh, fb);
      tma_load_3d_pair(sA + A_BYTES, map, kb * BK, rowA, zAl, fb);
      tma_load_3d_pair(sA + 2 * A_BYTES, map, kb * BK, rowB, zBh, fb);
      tma_load_3d_pair(sA + 3 * A_BYTES, map, kb * BK, rowB, zBl, fb);
      rg.next(P_STAGES);
    }
  }
  return true;
}

// Before a CTA exits, wait (bounded) for the copies it issued to land: the
// last P_STAGES stages were released by MMA commits or are pending.
__device__ __forceinline__ void producer_drain(RingPos rg, uint32_t bar_empty, uint64_t limit_ns) {
  for (int i = 0; i < P_STAGES; ++i) {
    const uint64_t t0 = gtimer();
    while (!mbar_try_wait(bar_empty + 8 * rg.idx, rg.phase ^ 1) && gtimer() - t0 < limit_ns) {
    }
    rg.next(P_STAGES);
  }
}

// MMA issuer of a pair kernel (leader CTA, one thread), one work item of
// `nst` stages: per stage the three products hi*hi, hi*lo, lo*hi for two K16
// steps into the current accumulation chunk; a chunk ends every `chunk`
// stages and at the end of each K pass (so chunks never straddle a pass),
// and is then published to both CTAs.  False when a bounded wait expired.
template <bool BF16>
__device__ __forceinline__ bool mma_item(RingPos& rg, RingPos& tb, int nst, int kblocks,
                                         int chunk, uint32_t tmem_base, uint32_t ring,
                                         uint32_t bar_full, uint32_t bar_empty,
                                         uint32_t bar_tfull, uint32_t bar_tempty,
                                         uint64_t limit_ns, volatile int* abort_flag,
                                         int* timeout_global) {
  constexpr uint32_t idesc = make_idesc_m256(BF16 ? 1 : 0);
  uint32_t d = 0, acc = 0;
  int sp = 0;   // stage within its K pass
  int cp = 0;   // stage within its accumulation chunk
  for (int si = 0; si < nst; ++si) {
    if (cp == 0) {
      if (!mbar_wait(bar_tempty + 8 * tb.idx, tb.phase ^ 1, limit_ns, abort_flag, timeout_global))
        return false;
      fence_after();
      d = tmem_base + (uint32_t)(tb.idx * BN);
      acc = 0;
    }
    if (!mbar_wait(bar_full + 8 * rg.idx, rg.phase, limit_ns, abort_flag, timeout_global))
      return false;
    fence_after();
    const uint32_t sA = ring + rg.idx * P_STAGE_BYTES;
    const uint64_t ah = sw64_desc(sA), al = sw64_desc(sA + A_BYTES);
    const uint64_t bh = sw64_desc(sA + 2 * A_BYTES);
    const uint64_t bl = sw64_desc(sA + 3 * A_BYTES);
#pragma unroll
    for (int kk = 0; kk < BK / 16; ++kk) {
      const uint64_t off = (uint64_t)((kk * 32) >> 4);
      mma_f16_pair(d, ah + off, bh + off, idesc, acc);   // hi * hi
      acc = 1;
      mma_f16_pair(d, ah + off, bl + off, idesc, 1);     // hi * lo
      mma_f16_pair(d, al + off, bh + off, idesc, 1);     // lo * hi
    }
    mma_commit_pair(bar_empty + 8 * rg.idx);   // frees the stage in both CTAs
    rg.next(P_STAGES);
    const bool chunk_end = cp == chunk - 1 || sp == kblocks - 1;
    if (++cp == chunk || sp == kblocks - 1) cp = 0;
    if (++sp == kblocks) sp = 0;
    if (chunk_end) {
      mma_commit_pair(bar_tfull + 8 * tb.idx);    // chunk ready in both CTAs
      tb.next(2);
    }
  }
  return true;
}

// Soft round alignment of the pair kernel's producers.  Items go to the
// pairs round-robin, so the 76 tiles of a round share their operand panels
// in L2 only while the pairs stay in step; a pair that drifts a round ahead
// fetches those panels from HBM again (with the fast, coalesced tile
// epilogue the pairs do drift, and DRAM reads per layer double).  The count
// is a scheduling hint only: no data depends on it.  At the start of each
// round r >= 1 a producer counts itself in and waits until every CTA that
// has an item in round r has started it.  The wait is bounded
// (kRoundAlignNs) and is never an error: after an expiry that producer stops
// waiting for the rest of the launch (it still counts itself in), so a grid
// whose CTAs are not all resident at once costs at most one bound.
constexpr uint64_t kRoundAlignNs = 300000;
__device__ __forceinline__ void round_start(unsigned* ctr, int64_t round, int64_t items,
                                            int64_t npairs, bool& align) {
  atomicAdd(ctr, 1u);
  if (!align) return;
  // CTAs with an item in rounds 1 .. round (only the last round is partial)
  const int64_t upto = (round + 1) * npairs < items ? (round + 1) * npairs : items;
  const unsigned target = (unsigned)(2 * (upto - npairs));
  const uint64_t t0 = gtimer();
  while (*reinterpret_cast<volatile unsigned*>(ctr) < target) {
    if (gtimer() - t0 > kRoundAlignNs) {
      align = false;
      return;
    }
    __nanosleep(128);
  }
}

// Tile epilogue of the pair kernel: after a tile's last chunk the sums are
// written back into that chunk's tensor-memory buffer and read 16 columns at
// a time by rolled_tile_epilogue (no register spills, little code per tile);
// the buffer returns to the MMA after that loop, so the MMA runs one chunk
// ahead of the epilogue during it.
template <bool BF16>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NUM_THREADS, 1)
    layer_tc2_kernel(const __grid_constant__ CUtensorMap mapA, State* st, float* __restrict__ master,
                     uint16_t* __restrict__ ops, int64_t Np, int k, double* __restrict__ partials,
                     int64_t ptiles, uint64_t limit_ns, int chunk, int k_snake, int band,
                     int inject_stall, int round_align) {
  using CV = Cvt<BF16>;
  using H16 = typename CV::T;
  extern __shared__ uint8_t smem_raw[];
  // every CTA takes the same early exits (state is read before any cluster
  // barrier, and both CTAs of a pair see the same values)
  if (st->done) return;
  uint32_t jmask = st->plan_square ? 1u : 0u;
  for (int j = 0; j < k; ++j)
    if (st->plan_resp[j]) jmask |= 1u << (1 + j);
  const int njobs = __popc(jmask);
  if (njobs == 0) return;
  const int cur0 = st->cur0;
  const int sigma = st->sigma_cur;
  const int write0 = st->plan_write0;
  const int s0e = st->s0_exp;
  const int z0c = st->z0_cur, z0n = st->z0_next;
  const int k1 = st->order >= 2 ? st->k1 : k;   // first-order directions
  // virtual index of the first item (0, except when the backward recomputes
  // a square alone: it then numbers the square's items as the forward launch
  // did, after its response items, so each tile keeps its round and K-snake
  // direction and the recomputed states are bit-identical)
  const int64_t vbase = st->item_base;

  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int64_t pair = blockIdx.x >> 1;
  const int64_t npairs = gridDim.x >> 1;
  const int64_t tiles = num_pair_tiles(Np);
  const int64_t items = tiles * njobs;
  const int kblocks = (int)(Np / BK);

  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t ring = base;
  uint8_t* misc = gbase + P_STAGES * P_STAGE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(misc);
  const uint32_t bar_full = smem_u32(bars);
  const uint32_t bar_empty = bar_full + 8 * P_STAGES;
  const uint32_t bar_tfull = bar_empty + 8 * P_STAGES;
  const uint32_t bar_tempty = bar_tfull + 8 * 2;
  const uint32_t bar_drain = bar_tempty + 8 * 2;
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(misc + 256);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(misc + 264);
  double* red = reinterpret_cast<double*>(misc + 1024);
  const uint32_t lead_full = map_to_rank(bar_full, 0);
  const uint32_t lead_tempty = map_to_rank(bar_tempty, 0);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_tfull + 8 * b, 1);
      mbar_init(bar_tempty + 8 * b, 2 * EPI_WARPS);
    }
    mbar_init(bar_drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  fence_before();
  cluster_sync_all();   // barriers of both CTAs initialised, TMEM allocated
  fence_after();
  const uint32_t tmem_base = *tmem_slot;
  int* timeout_global = &st->timeout_flag;

  if (warp == 0) {
    // ================= TMA producer (both CTAs load their own halves) ======
    if (lane == 0) {
      RingPos rg;
      bool ok = true;
      int64_t round = 0;
      bool align = round_align != 0;
      for (int64_t v = pair; v < vbase + items && ok; v += npairs, ++round) {
        if (v < vbase) continue;
        const int64_t it = v - vbase;
        if (round > 0) round_start(&st->round_ctr, round, items, npairs, align);
        const int job = job_at(jmask, (int)(it / tiles));
        int I2, J;
        pair_tile_banded(it % tiles, (int)(Np / BN), band, &I2, &J);
        // all pairs move through their tiles' K ranges in near lockstep; in
        // odd rounds the sweep runs backwards (passes and K blocks), so a
        // round starts on the panel slices the previous round loaded last,
        // which are still in L2
        const bool rev = k_snake && (round & 1);
        ok = produce_item(rg, &mapA, st, job, job_passes(job, k1), k, k1, cur0, z0c,
                          I2 * 2 * BM + (int)rank * BM, J * BN + (int)rank * BM, kblocks, rev,
                          leader, ring, bar_full, bar_empty, lead_full, limit_ns, abort_flag,
                          timeout_global);
      }
      producer_drain(rg, bar_empty, limit_ns);
    }
  } else if (warp == 1) {
    // ================= MMA issuer (leader CTA only) =================
    if (leader && lane == 0) {
      RingPos rg, tb;
      // test hook (see the single-CTA kernel)
      bool ok = !(inject_stall &&
                  !mbar_wait(bar_drain, 0, limit_ns, abort_flag, timeout_global));
      for (int64_t v = pair; v < vbase + items && ok; v += npairs) {
        if (v < vbase) continue;
        const int64_t it = v - vbase;
        const int job = job_at(jmask, (int)(it / tiles));
        ok = mma_item<BF16>(rg, tb, job_passes(job, k1) * kblocks, kblocks, chunk, tmem_base, ring,
                            bar_full, bar_empty, bar_tfull, bar_tempty, limit_ns, abort_flag,
                            timeout_global);
      }
      asm volatile(
          "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              bar_drain)
          : "memory");
      const uint64_t t0 = gtimer();
      while (!mbar_try_wait(bar_drain, 0) && gtimer() - t0 < limit_ns) {
      }
    }
  } else if (warp >= EPI_WARP0) {
    // ================= epilogue (both CTAs, own 128 rows) =================
    const int q = warp & 3;
    const int half = (warp - EPI_WARP0) >> 2;
    const int rloc = 32 * q + lane;
    const int et = threadIdx.x - 32 * EPI_WARP0;
    const size_t mat = (size_t)Np * Np;
    const uint32_t tlane = (uint32_t)(32 * q) << 16;
    int ab = 0;
    uint32_t abphase = 0;
    bool alive = true;
    int64_t eround = 0;
    for (int64_t v = pair; v < vbase + items && alive; v += npairs, ++eround) {
      if (v < vbase) continue;
      const int64_t it = v - vbase;
      const bool crev = k_snake && (eround & 1);   // same order as the producer
      const int job = job_at(jmask, (int)(it / tiles));
      const int passes = job_passes(job, k1);
      const int cpp = (kblocks + chunk - 1) / chunk;   // chunks per pass
      const int nchunks = passes * cpp;
      // exact power-of-two unscale of the products of passes 0 and 1
      // (passes >= 2 of higher-order terms: cross_unscale)
      const float u01 = ldexpf(1.0f, -(s0e + (job == 0 ? s0e : st->s1_exp_cur[job - 1])));
      float sum[128];
#pragma unroll
      for (int i = 0; i < 128; ++i) sum[i] = 0.0f;
      for (int ch = 0; ch < nchunks; ++ch) {
        const bool ok =
            mbar_wait(bar_tfull + 8 * ab, abphase, limit_ns, abort_flag, timeout_global);
        if (!epi_all(ok && !*abort_flag)) {
          alive = false;
          break;
        }
        fence_after();
        const uint32_t ta = tmem_base + tlane + (uint32_t)(ab * BN + half * 128);
        const int pc = chunk_pass(ch, cpp, passes, crev);
        const float u = pc < 2 ? u01 : cross_unscale(st, job, pc, k1);
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          uint32_t x[16];
          tmem_ld16(ta + 16 * cc, x);
#pragma unroll
          for (int i = 0; i < 16; ++i) sum[16 * cc + i] = fmaf(__uint_as_float(x[i]), u, sum[16 * cc + i]);
        }
        if (ch + 1 == nchunks) break;   // keep the last chunk's buffer
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(lead_tempty + 8 * ab);
        if (++ab == 2) {
          ab = 0;
          abphase ^= 1;
        }
      }
      if (!alive) break;
      // the tile's sums go back into its last chunk's buffer
      const uint32_t ta_sum = tmem_base + tlane + (uint32_t)(ab * BN + half * 128);
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) tmem_st16(ta_sum + 16 * cc, sum + 16 * cc);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");

      const int64_t t = it % tiles;
      int I2, J;
      pair_tile_banded(t, (int)(Np / BN), band, &I2, &J);
      const int curj = job == 0 ? cur0 : st->cur1[job - 1];
      const int e_new = job == 0 ? s0e : st->s1_exp_next[job - 1];
      const float scale_new = ldexpf(1.0f, e_new);   // exact power of two
      const float sg = (float)sigma, om = 1.0f - (float)sigma;
      const bool write = job != 0 || write0;
      const int r = I2 * 2 * BM + (int)rank * BM + rloc;
      const int c0 = J * BN + half * 128;
      const float* Sold = master + (size_t)(curj * (1 + k) + job) * mat;
      float* Snew = master + (size_t)((curj ^ 1) * (1 + k) + job) * mat;
      const int zh_new = job == 0 ? z0n : zslice(curj ^ 1, job, 0, k);
      H16* hi_new = reinterpret_cast<H16*>(ops) + (size_t)zh_new * mat;
      H16* lo_new = reinterpret_cast<H16*>(ops) + (size_t)(zh_new + 1) * mat;

      float fn_s = 0.0f, fn_c = 0.0f, fd = 0.0f, trf = 0.0f;
      int bad = 0;
      uint32_t* xp = reinterpret_cast<uint32_t*>(misc + 1024) +
                     (warp - EPI_WARP0) * (XP_WARP_BYTES / 4);
      if (I2 < J)
        rolled_tile_epilogue<CV, true>(ta_sum, Sold, Snew, hi_new, lo_new, xp, lane, Np, r, c0,
                                       sg, om, scale_new, write, fn_s, fn_c, fd, trf, bad);
      else
        rolled_tile_epilogue<CV, false>(ta_sum, Sold, Snew, hi_new, lo_new, xp, lane, Np, r, c0,
                                        sg, om, scale_new, write, fn_s, fn_c, fd, trf, bad);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(lead_tempty + 8 * ab);
      if (++ab == 2) {
        ab = 0;
        abphase ^= 1;
      }
      epi_sync();   // the reduction array overlays the transpose buffers
      red[0 * EPI_THREADS + et] = (double)trf;
      red[1 * EPI_THREADS + et] = (double)fn_s + (double)fn_c;
      red[2 * EPI_THREADS + et] = (double)fd;
      red[3 * EPI_THREADS + et] = (double)bad;
      epi_sync();
      for (int s2 = EPI_THREADS / 2; s2 > 0; s2 >>= 1) {
        if (et < s2) {
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) red[qq * EPI_THREADS + et] += red[qq * EPI_THREADS + et + s2];
        }
        epi_sync();
      }
      if (et == 0) {
        double* pp = partials + ((size_t)job * ptiles + 2 * t + rank) * kNQ;
        pp[kQTrace] = red[0];
        pp[kQFroNew] = red[EPI_THREADS];
        pp[kQFroDiff] = red[2 * EPI_THREADS];
        pp[kQBad] = red[3 * EPI_THREADS];
      }
      epi_sync();
    }
  }

  // ---- teardown: both CTAs done (or aborted); free TMEM of the pair
  fence_before();
  __syncthreads();
  cluster_sync_all();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS));
  }
}

// ---------------------------------------------------------------------------
// Grouped pair kernel: one layer of many instances of a batch in one launch.
//
// Each instance keeps its own control block, workspace and tensor map (a
// GroupInst in device memory).  At entry every CTA reads each instance's
// plan for this layer (which jobs run) and forms the prefix sums of the
// instances' item counts (tiles x jobs) in shared memory; the items of all
// instances make one pool that the 76 CTA pairs walk round-robin, as the
// single-instance kernel walks its own items.  An item's instance is found
// by binary search over the prefix sums.  Everything an item computes --
// its tile, passes, accumulation chunks, K direction (the K-snake parity is
// taken from the round the single-instance launch would run it in) and its
// tile epilogue -- is what the single-instance kernel
// computes for it, so the results are the same bit for bit.

// largest i with first[i] <= g (first[0] = 0 <= g)
__device__ __forceinline__ int group_find(const int64_t* first, int count, int64_t g) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void tensormap_acquire(const void* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

// The decoded item of a grouped launch.
struct GroupItem {
  int inst;        // instance
  int job;
  int passes;
  int kblocks;
  int64_t t;       // pair tile
  bool rev;        // K-snake direction
};

__device__ __forceinline__ GroupItem group_item(const GroupInst* __restrict__ inst,
                                                const int64_t* first, const uint32_t* jmask,
                                                int count, int64_t g, int k_snake) {
  GroupItem r;
  r.inst = group_find(first, count, g);
  const GroupInst& gi = inst[r.inst];
  const int64_t loc = g - first[r.inst];
  const int64_t tiles = num_pair_tiles(gi.Np);
  r.job = job_at(jmask[r.inst], (int)(loc / tiles));
  r.t = loc % tiles;
  r.passes = job_passes(r.job, gi.k);
  r.kblocks = (int)(gi.Np / BK);
  r.rev = k_snake && ((loc / gi.npairs) & 1);
  return r;
}

// Dynamic item assignment of a grouped launch (GroupQueue): a pair takes
// its next item when its producer is ready for one, so pairs that drew short
// items take more of them.  Everything an item computes still depends on the
// item alone, so results stay bit-identical to single-instance launches.
constexpr uint32_t kNoItem = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned long long claim_code(unsigned epoch, int64_t j, uint32_t g) {
  return ((unsigned long long)((epoch + 1u) & 0xFFFFFFu) << 40) |
         ((unsigned long long)((j / kQueueRing) & 0xFF) << 32) | g;
}

// Leader producer: claim the pair's j-th item and publish it.
__device__ __forceinline__ uint32_t claim_next(GroupQueue* gq, int64_t pair, int64_t j,
                                               unsigned epoch, int64_t items) {
  uint32_t g = atomicAdd(&gq->counter, 1u);
  if ((int64_t)g >= items) g = kNoItem;
  volatile unsigned long long* slot = &gq->slot[pair][j % kQueueRing];
  __threadfence();
  *slot = claim_code(epoch, j, g);
  return g;
}

// The pair's j-th item as its leader published it; false when the bounded
// wait expires (it then raises both abort flags) or another role aborted.
__device__ __forceinline__ bool claim_wait(GroupQueue* gq, int64_t pair, int64_t j,
                                           unsigned epoch, uint64_t limit_ns,
                                           volatile int* abort_smem, int* timeout_global,
                                           uint32_t* g) {
  volatile unsigned long long* slot = &gq->slot[pair][j % kQueueRing];
  const unsigned long long want = claim_code(epoch, j, 0u) >> 32;
  unsigned long long v = *slot;
  if ((v >> 32) == want) {
    *g = (uint32_t)v;
    return true;
  }
  const uint64_t t0 = gtimer();
  uint32_t it = 0;
  while (true) {
    v = *slot;
    if ((v >> 32) == want) {
      *g = (uint32_t)v;
      return true;
    }
    if ((++it & 63) == 0) {
      if (*abort_smem) return false;
      if (gtimer() - t0 > limit_ns) {
        *abort_smem = 1;
        atomicExch(timeout_global, 1);
        return false;
      }
    }
  }
}

template <bool BF16>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NUM_THREADS, 1)
    layer_tc2_group_kernel(const GroupInst* __restrict__ inst, int count, int* group_timeout,
                           GroupQueue* gq, uint64_t limit_ns, int chunk, int k_snake, int band) {
  using CV = Cvt<BF16>;
  using H16 = typename CV::T;
  extern __shared__ uint8_t smem_raw[];

  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t ring = base;
  uint8_t* misc = gbase + P_STAGES * P_STAGE_BYTES;
  int64_t* first = reinterpret_cast<int64_t*>(misc + 1024 + EPI_SCRATCH);
  uint32_t* jmask = reinterpret_cast<uint32_t*>(first + count + 1);

  // ---- this layer's items of every instance (same values in every CTA:
  //      the control blocks do not change during the launch)
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const State* sti = inst[i].st;
    uint32_t jm = 0;
    if (!sti->done) {
      jm = sti->plan_square ? 1u : 0u;
      for (int j = 0; j < inst[i].k; ++j)
        if (sti->plan_resp[j]) jm |= 1u << (1 + j);
    }
    jmask[i] = jm;
    first[i + 1] = num_pair_tiles(inst[i].Np) * __popc(jm);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    first[0] = 0;
    for (int i = 0; i < count; ++i) first[i + 1] += first[i];
  }
  __syncthreads();
  const int64_t items = first[count];
  if (items == 0) return;   // every CTA takes this exit together
  const unsigned epoch = *(volatile unsigned*)&gq->epoch;   // fixed during the launch

  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int64_t pair = blockIdx.x >> 1;

  uint64_t* bars = reinterpret_cast<uint64_t*>(misc);
  const uint32_t bar_full = smem_u32(bars);
  const uint32_t bar_empty = bar_full + 8 * P_STAGES;
  const uint32_t bar_tfull = bar_empty + 8 * P_STAGES;
  const uint32_t bar_tempty = bar_tfull + 8 * 2;
  const uint32_t bar_drain = bar_tempty + 8 * 2;
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(misc + 256);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(misc + 264);
  double* red = reinterpret_cast<double*>(misc + 1024);
  const uint32_t lead_full = map_to_rank(bar_full, 0);
  const uint32_t lead_tempty = map_to_rank(bar_tempty, 0);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_tfull + 8 * b, 1);
      mbar_init(bar_tempty + 8 * b, 2 * EPI_WARPS);
    }
    mbar_init(bar_drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  fence_before();
  cluster_sync_all();   // barriers of both CTAs initialised, TMEM allocated
  fence_after();
  const uint32_t tmem_base = *tmem_slot;
  int* timeout_global = group_timeout;

  if (warp == 0) {
    // ================= TMA producer (both CTAs load their own halves) ======
    if (lane == 0) {
      RingPos rg;
      bool ok = true;
      int last_inst = -1;
      for (int64_t j = 0; ok; ++j) {
        uint32_t g;
        if (leader)
          g = claim_next(gq, pair, j, epoch, items);
        else if (!claim_wait(gq, pair, j, epoch, limit_ns, abort_flag, timeout_global, &g))
          break;
        if (g == kNoItem) break;
        const GroupItem itm = group_item(inst, first, jmask, count, g, k_snake);
        const GroupInst& gi = inst[itm.inst];
        if (itm.inst != last_inst) {
          tensormap_acquire(&gi.map);
          last_inst = itm.inst;
        }
        const State* sti = gi.st;
        int I2, J;
        pair_tile_banded(itm.t, (int)(gi.Np / BN), band, &I2, &J);
        ok = produce_item(rg, &gi.map, sti, itm.job, itm.passes, gi.k, gi.k, sti->cur0,
                          sti->z0_cur, I2 * 2 * BM + (int)rank * BM, J * BN + (int)rank * BM,
                          itm.kblocks, itm.rev, leader, ring, bar_full, bar_empty, lead_full,
                          limit_ns, abort_flag, timeout_global);
      }
      producer_drain(rg, bar_empty, limit_ns);
    }
  } else if (warp == 1) {
    // ================= MMA issuer (leader CTA only) =================
    if (leader && lane == 0) {
      RingPos rg, tb;
      bool ok = true;
      for (int64_t j = 0; ok; ++j) {
        uint32_t g;
        if (!claim_wait(gq, pair, j, epoch, limit_ns, abort_flag, timeout_global, &g)) break;
        if (g == kNoItem) break;
        const GroupItem itm = group_item(inst, first, jmask, count, g, k_snake);
        ok = mma_item<BF16>(rg, tb, itm.passes * itm.kblocks, itm.kblocks, chunk, tmem_base,
                            ring, bar_full, bar_empty, bar_tfull, bar_tempty, limit_ns,
                            abort_flag, timeout_global);
      }
      asm volatile(
          "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              bar_drain)
          : "memory");
      const uint64_t t0 = gtimer();
      while (!mbar_try_wait(bar_drain, 0) && gtimer() - t0 < limit_ns) {
      }
    }
  } else if (warp >= EPI_WARP0) {
    // ================= epilogue (both CTAs, own 128 rows) =================
    const int q = warp & 3;
    const int half = (warp - EPI_WARP0) >> 2;
    const int rloc = 32 * q + lane;
    const int et = threadIdx.x - 32 * EPI_WARP0;
    const uint32_t tlane = (uint32_t)(32 * q) << 16;
    int ab = 0;
    uint32_t abphase = 0;
    bool alive = true;
    for (int64_t j = 0; alive; ++j) {
      // lane 0 of each warp reads the claim; every epilogue warp agrees on it
      uint32_t g = kNoItem;
      bool got = true;
      if (lane == 0) got = claim_wait(gq, pair, j, epoch, limit_ns, abort_flag, timeout_global, &g);
      g = __shfl_sync(0xFFFFFFFFu, g, 0);
      got = __shfl_sync(0xFFFFFFFFu, got ? 1 : 0, 0) != 0;
      if (!epi_all(got && !*abort_flag)) {
        alive = false;
        break;
      }
      if (g == kNoItem) break;
      const GroupItem itm = group_item(inst, first, jmask, count, g, k_snake);
      const GroupInst& gi = inst[itm.inst];
      const State* sti = gi.st;
      const int job = itm.job;
      const int k = gi.k;
      const int passes = itm.passes;
      const int cpp = (itm.kblocks + chunk - 1) / chunk;   // chunks per pass
      const int nchunks = passes * cpp;
      const int s0e = sti->s0_exp;
      // exact power-of-two unscale of the products (first-order jobs and the
      // square: passes 0 and 1 only)
      const float u = ldexpf(1.0f, -(s0e + (job == 0 ? s0e : sti->s1_exp_cur[job - 1])));
      float sum[128];
#pragma unroll
      for (int i = 0; i < 128; ++i) sum[i] = 0.0f;
      for (int ch = 0; ch < nchunks; ++ch) {
        const bool ok =
            mbar_wait(bar_tfull + 8 * ab, abphase, limit_ns, abort_flag, timeout_global);
        if (!epi_all(ok && !*abort_flag)) {
          alive = false;
          break;
        }
        fence_after();
        const uint32_t ta = tmem_base + tlane + (uint32_t)(ab * BN + half * 128);
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          uint32_t x[16];
          tmem_ld16(ta + 16 * cc, x);
#pragma unroll
          for (int i = 0; i < 16; ++i) sum[16 * cc + i] = fmaf(__uint_as_float(x[i]), u, sum[16 * cc + i]);
        }
        if (ch + 1 == nchunks) break;   // keep the last chunk's buffer
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(lead_tempty + 8 * ab);
        if (++ab == 2) {
          ab = 0;
          abphase ^= 1;
        }
      }
      if (!alive) break;
      // the tile's sums go back into its last chunk's buffer (rolled epilogue)
      const uint32_t ta_sum = tmem_base + tlane + (uint32_t)(ab * BN + half * 128);
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) tmem_st16(ta_sum + 16 * cc, sum + 16 * cc);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");

      const int64_t Np = gi.Np;
      const size_t mat = (size_t)Np * Np;
      int I2, J;
      pair_tile_banded(itm.t, (int)(Np / BN), band, &I2, &J);
      const int cur0 = sti->cur0;
      const int curj = job == 0 ? cur0 : sti->cur1[job - 1];
      const int e_new = job == 0 ? s0e : sti->s1_exp_next[job - 1];
      const float scale_new = ldexpf(1.0f, e_new);   // exact power of two
      const float sigma = (float)sti->sigma_cur;
      const float sg = sigma, om = 1.0f - sigma;
      const bool write = job != 0 || sti->plan_write0;
      const int r = I2 * 2 * BM + (int)rank * BM + rloc;
      const int c0 = J * BN + half * 128;
      float* master = gi.master;
      const float* Sold = master + (size_t)(curj * (1 + k) + job) * mat;
      float* Snew = master + (size_t)((curj ^ 1) * (1 + k) + job) * mat;
      const int zh_new = job == 0 ? sti->z0_next : zslice(curj ^ 1, job, 0, k);
      H16* hi_new = reinterpret_cast<H16*>(gi.ops) + (size_t)zh_new * mat;
      H16* lo_new = reinterpret_cast<H16*>(gi.ops) + (size_t)(zh_new + 1) * mat;

      float fn_s = 0.0f, fn_c = 0.0f, fd = 0.0f, trf = 0.0f;
      int bad = 0;
      uint32_t* xp = reinterpret_cast<uint32_t*>(misc + 1024) +
                     (warp - EPI_WARP0) * (XP_WARP_BYTES / 4);
      if (I2 < J)
        rolled_tile_epilogue<CV, true>(ta_sum, Sold, Snew, hi_new, lo_new, xp, lane, Np, r, c0,
                                       sg, om, scale_new, write, fn_s, fn_c, fd, trf, bad);
      else
        rolled_tile_epilogue<CV, false>(ta_sum, Sold, Snew, hi_new, lo_new, xp, lane, Np, r, c0,
                                        sg, om, scale_new, write, fn_s, fn_c, fd, trf, bad);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(lead_tempty + 8 * ab);
      if (++ab == 2) {
        ab = 0;
        abphase ^= 1;
      }
      epi_sync();   // the reduction array overlays the transpose buffers
      red[0 * EPI_THREADS + et] = (double)trf;
      red[1 * EPI_THREADS + et] = (double)fn_s + (double)fn_c;
      red[2 * EPI_THREADS + et] = (double)fd;
      red[3 * EPI_THREADS + et] = (double)bad;
      epi_sync();
      for (int s2 = EPI_THREADS / 2; s2 > 0; s2 >>= 1) {
        if (et < s2) {
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) red[qq * EPI_THREADS + et] += red[qq * EPI_THREADS + et + s2];
        }
        epi_sync();
      }
      if (et == 0) {
        double* pp = gi.partials + ((size_t)job * gi.ptiles + 2 * itm.t + rank) * kNQ;
        pp[kQTrace] = red[0];
        pp[kQFroNew] = red[EPI_THREADS];
        pp[kQFroDiff] = red[2 * EPI_THREADS];
        pp[kQBad] = red[3 * EPI_THREADS];
      }
      epi_sync();
    }
  }

  // ---- teardown: both CTAs done (or aborted); free TMEM of the pair
  fence_before();
  __syncthreads();
  cluster_sync_all();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS));
  }
}

// ---------------------------------------------------------------------------
// Grouped pair kernel on 256 x 128 tiles (batches; option of the batch path).
//
// The same pool of items, dynamic queue and per-item work as the 256 x 256
// grouped kernel, with three changes that suit small instances:
//  - N = 128: each CTA of a pair loads 64 B rows per stage (a 64-row tensor
//    map), so a stage is 24 KB and the ring holds 8 of them;
//  - tensor memory holds four 128-column accumulators, so a tile epilogue,
//    which keeps its tile's sums in the last chunk's accumulator while it
//    stores, leaves the MMA issuer three accumulators to run ahead with;
//  - the instances are padded to a multiple of 128 instead of 256.  A row
//    block of 256 can then extend 128 rows past the matrix: its second CTA
//    multiplies zeros (the tensor map fills rows past Np with zeros) and skips
//    its epilogue.
// Items run their K passes forwards (no K-snake): the queue keeps the items
// in flight within a few instances, whose operand panels stay in L2.  The
// tile order differs from the 256 x 256 kernels, so results agree with them
// to rounding, not bit for bit.
constexpr int G_BN = 128;                                   // tile columns
constexpr int G_BROWS = G_BN / 2;                           // B rows per CTA
constexpr int G_B_BYTES = G_BROWS * BK * 2;                 // 4 KB
constexpr int G_STAGES = 8;
constexpr int G_STAGE_BYTES = 2 * A_BYTES + 2 * G_B_BYTES;  // 24 KB
constexpr int G_ACC = 4;                                    // accumulators of G_BN columns
static_assert(G_ACC * G_BN == TMEM_COLS, "accumulators fill the allocation");
constexpr int G_SMEM_BYTES = G_STAGES * G_STAGE_BYTES + 1024 + 1024 + EPI_SCRATCH;
static_assert(G_SMEM_BYTES == P_SMEM_BYTES, "same shared memory as the 256 x 256 kernel");

__host__ __device__ constexpr uint32_t make_idesc_m256_n128(int ab_type) {
  return (1u << 4) | ((uint32_t)ab_type << 7) | ((uint32_t)ab_type << 10) |
         ((uint32_t)(G_BN >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}

// 256 x 128 tiles holding some element with row <= col: 256-row block I2 and
// 128-column block J' with J' >= 2 I2; row-major (I2, then J').
__host__ __device__ inline int64_t num_tiles128(int64_t Np) {
  const int64_t tj = Np / G_BN, t2 = (Np + 255) / 256;
  return t2 * tj - t2 * (t2 - 1);   // sum over I2 < t2 of (tj - 2 I2)
}
__device__ __forceinline__ void tile128_coords(int64_t t, int64_t Np, int* I2, int* J) {
  const int tj = (int)(Np / G_BN);
  int i = 0;
  while (t >= tj - 2 * i) {
    t -= tj - 2 * i;
    ++i;
  }
  *I2 = i;
  *J = 2 * i + (int)t;
}

struct GroupItem128 {
  int inst, job, passes, kblocks;
  int64_t t;
};

__device__ __forceinline__ GroupItem128 group_item128(const GroupInst* __restrict__ inst,
                                                      const int64_t* first, const uint32_t* jmask,
                                                      int count, int64_t g) {
  GroupItem128 r;
  r.inst = group_find(first, count, g);
  const GroupInst& gi = inst[r.inst];
  const int64_t loc = g - first[r.inst];
  const int64_t tiles = num_tiles128(gi.Np);
  r.job = job_at(jmask[r.inst], (int)(loc / tiles));
  r.t = loc % tiles;
  r.passes = job_passes(r.job, gi.k);
  r.kblocks = (int)(gi.Np / BK);
  return r;
}

// Producer of one 256 x 128 item: this CTA's 128 A rows (128-row map) and its
// 64 B rows (64-row map) per stage, signalled on the leader's full barrier.
__device__ __forceinline__ bool produce_item128(RingPos& rg, const CUtensorMap* map,
                                                const CUtensorMap* map64, const State* st,
                                                int job, int passes, int k, int cur0, int z0c,
                                                int rowA, int rowB, int kblocks, bool leader,
                                                uint32_t ring, uint32_t bar_full,
                                                uint32_t bar_empty, uint32_t lead_full,
                                                uint64_t limit_ns, volatile int* abort_flag,
                                                int* timeout_global) {
  for (int pass = 0; pass < passes; ++pass) {
    int mA, mB;
    job_operands(job, pass, k, &mA, &mB);
    const int bufA = mA == 0 ? cur0 : st->cur1[mA - 1];
    const int bufB = mB == 0 ? cur0 : st->cur1[mB - 1];
    const int zAh = zop(mA, bufA, 0, k, z0c), zAl = zop(mA, bufA, 1, k, z0c);
    const int zBh = zop(mB, bufB, 0, k, z0c), zBl = zop(mB, bufB, 1, k, z0c);
    for (int kb = 0; kb < kblocks; ++kb) {
      if (!mbar_wait(bar_empty + 8 * rg.idx, rg.phase ^ 1, limit_ns, abort_flag, timeout_global))
        return false;
      const uint32_t sA = ring + rg.idx * G_STAGE_BYTES;
      if (leader) mbar_expect_tx(bar_full + 8 * rg.idx, 2 * G_STAGE_BYTES);
      const uint32_t fb = lead_full + 8 * rg.idx;
      tma_load_3d_pair(sA, map, kb * BK, rowA, zAh, fb);
      tma_load_3d_pair(sA + A_BYTES, map, kb * BK, rowA, zAl, fb);
      tma_load_3d_pair(sA + 2 * A_BYTES, map64, kb * BK, rowB, zBh, fb);
      tma_load_3d_pair(sA + 2 * A_BYTES + G_B_BYTES, map64, kb * BK, rowB, zBl, fb);
      rg.next(G_STAGES);
    }
  }
  return true;
}

__device__ __forceinline__ void producer_drain128(RingPos rg, uint32_t bar_empty,
                                                  uint64_t limit_ns) {
  for (int i = 0; i < G_STAGES; ++i) {
    const uint64_t t0 = gtimer();
    while (!mbar_try_wait(bar_empty + 8 * rg.idx, rg.phase ^ 1) && gtimer() - t0 < limit_ns) {
    }
    rg.next(G_STAGES);
  }
}

// MMA issuer of one 256 x 128 item (leader CTA, one thread): as mma_item,
// with N = 128 and four accumulators.
template <bool BF16>
__device__ __forceinline__ bool mma_item128(RingPos& rg, RingPos& tb, int nst, int kblocks,
                                            int chunk, uint32_t tmem_base, uint32_t ring,
                                            uint32_t bar_full, uint32_t bar_empty,
                                            uint32_t bar_tfull, uint32_t bar_tempty,
                                            uint64_t limit_ns, volatile int* abort_flag,
                                            int* timeout_global) {
  constexpr uint32_t idesc = make_idesc_m256_n128(BF16 ? 1 : 0);
  uint32_t d = 0, acc = 0;
  int sp = 0;   // stage within its K pass
  int cp = 0;   // stage within its accumulation chunk
  for (int si = 0; si < nst; ++si) {
    if (cp == 0) {
      if (!mbar_wait(bar_tempty + 8 * tb.idx, tb.phase ^ 1, limit_ns, abort_flag, timeout_global))
        return false;
      fence_after();
      d = tmem_base + (uint32_t)(tb.idx * G_BN);
      acc = 0;
    }
    if (!mbar_wait(bar_full + 8 * rg.idx, rg.phase, limit_ns, abort_flag, timeout_global))
      return false;
    fence_after();
    const uint32_t sA = ring + rg.idx * G_STAGE_BYTES;
    const uint64_t ah = sw64_desc(sA), al = sw64_desc(sA + A_BYTES);
    const uint64_t bh = sw64_desc(sA + 2 * A_BYTES);
    const uint64_t bl = sw64_desc(sA + 2 * A_BYTES + G_B_BYTES);
#pragma unroll
    for (int kk = 0; kk < BK / 16; ++kk) {
      const uint64_t off = (uint64_t)((kk * 32) >> 4);
      mma_f16_pair(d, ah + off, bh + off, idesc, acc);   // hi * hi
      acc = 1;
      mma_f16_pair(d, ah + off, bl + off, idesc, 1);     // hi * lo
      mma_f16_pair(d, al + off, bh + off, idesc, 1);     // lo * hi
    }
    mma_commit_pair(bar_empty + 8 * rg.idx);   // frees the stage in both CTAs
    rg.next(G_STAGES);
    const bool chunk_end = cp == chunk - 1 || sp == kblocks - 1;
    if (++cp == chunk || sp == kblocks - 1) cp = 0;
    if (++sp == kblocks) sp = 0;
    if (chunk_end) {
      mma_commit_pair(bar_tfull + 8 * tb.idx);    // chunk ready in both CTAs
      tb.next(G_ACC);
    }
  }
  return true;
}

template <bool BF16>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NUM_THREADS, 1)
    layer_tc2_group128_kernel(const GroupInst* __restrict__ inst, int count, int* group_timeout,
                              GroupQueue* gq, uint64_t limit_ns, int chunk) {
  using CV = Cvt<BF16>;
  using H16 = typename CV::T;
  extern __shared__ uint8_t smem_raw[];

  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t ring = base;
  uint8_t* misc = gbase + G_STAGES * G_STAGE_BYTES;
  int64_t* first = reinterpret_cast<int64_t*>(misc + 1024 + EPI_SCRATCH);
  uint32_t* jmask = reinterpret_cast<uint32_t*>(first + count + 1);

  // ---- this layer's items of every instance (as in the 256 x 256 kernel)
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const State* sti = inst[i].st;
    uint32_t jm = 0;
    if (!sti->done) {
      jm = sti->plan_square ? 1u : 0u;
      for (int j = 0; j < inst[i].k; ++j)
        if (sti->plan_resp[j]) jm |= 1u << (1 + j);
    }
    jmask[i] = jm;
    first[i + 1] = num_tiles128(inst[i].Np) * __popc(jm);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    first[0] = 0;
    for (int i = 0; i < count; ++i) first[i + 1] += first[i];
  }
  __syncthreads();
  const int64_t items = first[count];
  if (items == 0) return;   // every CTA takes this exit together
  const unsigned epoch = *(volatile unsigned*)&gq->epoch;   // fixed during the launch

  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int64_t pair = blockIdx.x >> 1;

  uint64_t* bars = reinterpret_cast<uint64_t*>(misc);
  const uint32_t bar_full = smem_u32(bars);
  const uint32_t bar_empty = bar_full + 8 * G_STAGES;
  const uint32_t bar_tfull = bar_empty + 8 * G_STAGES;
  const uint32_t bar_tempty = bar_tfull + 8 * G_ACC;
  const uint32_t bar_drain = bar_tempty + 8 * G_ACC;
  static_assert(8 * (2 * G_STAGES + 2 * G_ACC + 1) <= 256, "barriers below the TMEM slot");
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(misc + 256);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(misc + 264);
  double* red = reinterpret_cast<double*>(misc + 1024);
  const uint32_t lead_full = map_to_rank(bar_full, 0);
  const uint32_t lead_tempty = map_to_rank(bar_tempty, 0);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < G_STAGES; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    for (int b = 0; b < G_ACC; ++b) {
      mbar_init(bar_tfull + 8 * b, 1);
      mbar_init(bar_tempty + 8 * b, 2 * EPI_WARPS);
    }
    mbar_init(bar_drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  fence_before();
  cluster_sync_all();   // barriers of both CTAs initialised, TMEM allocated
  fence_after();
  const uint32_t tmem_base = *tmem_slot;
  int* timeout_global = group_timeout;

  if (warp == 0) {
    // ================= TMA producer (both CTAs load their own rows) ======
    if (lane == 0) {
      RingPos rg;
      bool ok = true;
      int last_inst = -1;
      for (int64_t j = 0; ok; ++j) {
        uint32_t g;
        if (leader)
          g = claim_next(gq, pair, j, epoch, items);
        else if (!claim_wait(gq, pair, j, epoch, limit_ns, abort_flag, timeout_global, &g))
          break;
        if (g == kNoItem) break;
        const GroupItem128 itm = group_item128(inst, first, jmask, count, g);
        const GroupInst& gi = inst[itm.inst];
        if (itm.inst != last_inst) {
          tensormap_acquire(&gi.map);
          tensormap_acquire(&gi.map64);
          last_inst = itm.inst;
        }
        const State* sti = gi.st;
        int I2, J;
        tile128_coords(itm.t, gi.Np, &I2, &J);
        ok = produce_item128(rg, &gi.map, &gi.map64, sti, itm.job, itm.passes, gi.k, sti->cur0,
                             sti->z0_cur, I2 * 2 * BM + (int)rank * BM,
                             J * G_BN + (int)rank * G_BROWS, itm.kblocks, leader, ring, bar_full,
                             bar_empty, lead_full, limit_ns, abort_flag, timeout_global);
      }
      producer_drain128(rg, bar_empty, limit_ns);
    }
  } else if (warp == 1) {
    // ================= MMA issuer (leader CTA only) =================
    if (leader && lane == 0) {
      RingPos rg, tb;
      bool ok = true;
      for (int64_t j = 0; ok; ++j) {
        uint32_t g;
        if (!claim_wait(gq, pair, j, epoch, limit_ns, abort_flag, timeout_global, &g)) break;
        if (g == kNoItem) break;
        const GroupItem128 itm = group_item128(inst, first, jmask, count, g);
        ok = mma_item128<BF16>(rg, tb, itm.passes * itm.kblocks, itm.kblocks, chunk, tmem_base,
                               ring, bar_full, bar_empty, bar_tfull, bar_tempty, limit_ns,
                               abort_flag, timeout_global);
      }
      asm volatile(
          "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              bar_drain)
          : "memory");
      const uint64_t t0 = gtimer();
      while (!mbar_try_wait(bar_drain, 0) && gtimer() - t0 < limit_ns) {
      }
    }
  } else if (warp >= EPI_WARP0) {
    // ========== epilogue (both CTAs, own 128 rows; warps split 64 + 64 columns) ==========
    const int q = warp & 3;
    const int half = (warp - EPI_WARP0) >> 2;
    const int rloc = 32 * q + lane;
    const int et = threadIdx.x - 32 * EPI_WARP0;
    const uint32_t tlane = (uint32_t)(32 * q) << 16;
    RingPos ab;
    bool alive = true;
    for (int64_t j = 0; alive; ++j) {
      uint32_t g = kNoItem;
      bool got = true;
      if (lane == 0) got = claim_wait(gq, pair, j, epoch, limit_ns, abort_flag, timeout_global, &g);
      g = __shfl_sync(0xFFFFFFFFu, g, 0);
      got = __shfl_sync(0xFFFFFFFFu, got ? 1 : 0, 0) != 0;
      if (!epi_all(got && !*abort_flag)) {
        alive = false;
        break;
      }
      if (g == kNoItem) break;
      const GroupItem128 itm = group_item128(inst, first, jmask, count, g);
      const GroupInst& gi = inst[itm.inst];
      const State* sti = gi.st;
      const int job = itm.job;
      const int k = gi.k;
      const int cpp = (itm.kblocks + chunk - 1) / chunk;   // chunks per pass
      const int nchunks = itm.passes * cpp;
      const int s0e = sti->s0_exp;
      // exact power-of-two unscale of the products (first-order jobs and the
      // square: passes 0 and 1 only)
      const float u = ldexpf(1.0f, -(s0e + (job == 0 ? s0e : sti->s1_exp_cur[job - 1])));
      float sum[64];
#pragma unroll
      for (int i = 0; i < 64; ++i) sum[i] = 0.0f;
      for (int ch = 0; ch < nchunks; ++ch) {
        const bool ok =
            mbar_wait(bar_tfull + 8 * ab.idx, ab.phase, limit_ns, abort_flag, timeout_global);
        if (!epi_all(ok && !*abort_flag)) {
          alive = false;
          break;
        }
        fence_after();
        const uint32_t ta = tmem_base + tlane + (uint32_t)(ab.idx * G_BN + half * 64);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          uint32_t x[16];
          tmem_ld16(ta + 16 * cc, x);
#pragma unroll
          for (int i = 0; i < 16; ++i) sum[16 * cc + i] = fmaf(__uint_as_float(x[i]), u, sum[16 * cc + i]);
        }
        if (ch + 1 == nchunks) break;   // keep the last chunk's accumulator
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(lead_tempty + 8 * ab.idx);
        ab.next(G_ACC);
      }
      if (!alive) break;
      // the tile's sums go back into its last chunk's accumulator (rolled epilogue)
      const uint32_t ta_sum = tmem_base + tlane + (uint32_t)(ab.idx * G_BN + half * 64);
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) tmem_st16(ta_sum + 16 * cc, sum + 16 * cc);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");

      const int64_t Np = gi.Np;
      const size_t mat = (size_t)Np * Np;
      int I2, J;
      tile128_coords(itm.t, Np, &I2, &J);
      const int cur0 = sti->cur0;
      const int curj = job == 0 ? cur0 : sti->cur1[job - 1];
      const int e_new = job == 0 ? s0e : sti->s1_exp_next[job - 1];
      const float scale_new = ldexpf(1.0f, e_new);   // exact power of two
      const float sigma = (float)sti->sigma_cur;
      const float sg = sigma, om = 1.0f - sigma;
      const bool write = job != 0 || sti->plan_write0;
      const int row0 = I2 * 2 * BM + (int)rank * BM;   // this CTA's first row
      const int r = row0 + rloc;
      const int c0 = J * G_BN + half * 64;
      float* master = gi.master;
      const float* Sold = master + (size_t)(curj * (1 + k) + job) * mat;
      float* Snew = master + (size_t)((curj ^ 1) * (1 + k) + job) * mat;
      const int zh_new = job == 0 ? sti->z0_next : zslice(curj ^ 1, job, 0, k);
      H16* hi_new = reinterpret_cast<H16*>(gi.ops) + (size_t)zh_new * mat;
      H16* lo_new = reinterpret_cast<H16*>(gi.ops) + (size_t)(zh_new + 1) * mat;

      float fn_s = 0.0f, fn_c = 0.0f, fd = 0.0f, trf = 0.0f;
      int bad = 0;
      uint32_t* xp = reinterpret_cast<uint32_t*>(misc + 1024) +
                     (warp - EPI_WARP0) * (XP_WARP_BYTES / 4);
      // rows past Np (a 256-row block over a matrix padded to 128): nothing to
      // store; the products there are zeros
      if ((int64_t)row0 < Np) {
        if (c0 >= row0 + BM)   // every column of this warp's block right of every row
          rolled_tile_epilogue<CV, true, 4>(ta_sum, Sold, Snew, hi_new, lo_new, xp, lane, Np, r,
                                            c0, sg, om, scale_new, write, fn_s, fn_c, fd, trf,
                                            bad);
        else
          rolled_tile_epilogue<CV, false, 4>(ta_sum, Sold, Snew, hi_new, lo_new, xp, lane, Np, r,
                                             c0, sg, om, scale_new, write, fn_s, fn_c, fd, trf,
                                             bad);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(lead_tempty + 8 * ab.idx);
      ab.next(G_ACC);
      epi_sync();   // the reduction array overlays the transpose buffers
      red[0 * EPI_THREADS + et] = (double)trf;
      red[1 * EPI_THREADS + et] = (double)fn_s + (double)fn_c;
      red[2 * EPI_THREADS + et] = (double)fd;
      red[3 * EPI_THREADS + et] = (double)bad;
      epi_sync();
      for (int s2 = EPI_THREADS / 2; s2 > 0; s2 >>= 1) {
        if (et < s2) {
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) red[qq * EPI_THREADS + et] += red[qq * EPI_THREADS + et + s2];
        }
        epi_sync();
      }
      if (et == 0) {
        double* pp = gi.partials + ((size_t)job * gi.ptiles + 2 * itm.t + rank) * kNQ;
        pp[kQTrace] = red[0];
        pp[kQFroNew] = red[EPI_THREADS];
        pp[kQFroDiff] = red[2 * EPI_THREADS];
        pp[kQBad] = red[3 * EPI_THREADS];
      }
      epi_sync();
    }
  }

  // ---- teardown: both CTAs done (or aborted); free TMEM of the pair
  fence_before();
  __syncthreads();
  cluster_sync_all();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS));
  }
}


// ---------------------------------------------------------------------------
// Host side

// Per-device one-time setup of the tensor-core kernels (their shared-memory
// attribute is set in each device's context) and the device's SM count;
// thread-safe.
constexpr int kMaxDevices = 64;
struct DeviceSetup {
  std::once_flag once;
  int sms = 0;
};
int device_setup() {
  static DeviceSetup tab[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
  DeviceSetup& d = tab[dev];
  std::call_once(d.once, [&] {
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(layer_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         SMEM_BYTES);
    cudaFuncSetAttribute(layer_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         SMEM_BYTES);
    cudaFuncSetAttribute(layer_tc2_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         P_SMEM_BYTES);
    cudaFuncSetAttribute(layer_tc2_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         P_SMEM_BYTES);
    constexpr int group_smem = P_SMEM_BYTES + (kGroupMax + 1) * (int)sizeof(int64_t) +
                               kGroupMax * (int)sizeof(uint32_t);
    static_assert(group_smem <= 227 * 1024, "grouped kernel shared memory");
    cudaFuncSetAttribute(layer_tc2_group_kernel<false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, group_smem);
    cudaFuncSetAttribute(layer_tc2_group_kernel<true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, group_smem);
    cudaFuncSetAttribute(layer_tc2_group128_kernel<false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, group_smem);
    cudaFuncSetAttribute(layer_tc2_group128_kernel<true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, group_smem);
  });
  return d.sms;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
  // looked up once per process (thread-safe static initialisation)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}

bool make_map(CUtensorMap* map, void* base, int64_t Np, int slices, int box_rows, bool bf16) {
  auto enc = get_encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Np, (cuuint64_t)Np, (cuuint64_t)slices};
  cuuint64_t strides[2] = {(cuuint64_t)Np * 2, (cuuint64_t)Np * Np * 2};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                   3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace tc

int tc_tile() { return tc::BN; }

void pair_tile_info(const Layout& L, int64_t* entries, double* pass_flops, bool n128) {
  const int64_t tiles = n128 ? tc::num_tiles128(L.Np) : tc::num_pair_tiles(L.Np);
  const double cols = n128 ? tc::G_BN : tc::BN;
  if (entries) *entries = 2 * tiles;
  if (pass_flops) *pass_flops = (double)tiles * 2 * tc::BM * cols * (double)L.Np * 2.0;
}

bool make_group_inst(const Layout& L, void* ws, int sm_count, GroupInst* gi, bool n128) {
  using namespace tc;
  char* base = (char*)ws;
  const bool bf16 = L.precision == DMPT_DUAL_BF16;
  const int slices = 2 * (1 + L.k) * 2 + 2 * L.tape_states;
  if (!make_map(&gi->map, base + L.off_ops16, L.Np, slices, BM, bf16)) return false;
  if (n128 && !make_map(&gi->map64, base + L.off_ops16, L.Np, slices, G_BROWS, bf16)) return false;
  gi->st = (State*)(base + L.off_state);
  gi->master = (float*)(base + L.off_master);
  gi->ops = (uint16_t*)(base + L.off_ops16);
  gi->partials = (double*)(base + L.off_partials);
  gi->Np = L.Np;
  gi->ptiles = L.partial_tiles;
  gi->k = L.k;
  const int64_t max_items = num_pair_tiles(L.Np) * (1 + L.k);
  int64_t pairs = sm_count / 2;
  if (pairs > max_items) pairs = max_items;
  gi->npairs = (int)pairs;
  return true;
}

cudaError_t launch_layer_tc_group(const GroupInst* inst, int count, bool bf16, int* group_timeout,
                                  GroupQueue* queue, double timeout_s, int accum_chunk_k,
                                  int k_snake, int band, int sm_count, cudaStream_t s,
                                  bool n128) {
  using namespace tc;
  if (count < 1 || count > kGroupMax || !queue || sm_count / 2 > kQueuePairs)
    return cudaErrorInvalidValue;
  const int smem =
      P_SMEM_BYTES + (count + 1) * (int)sizeof(int64_t) + count * (int)sizeof(uint32_t);
  if (device_setup() == 0) return cudaErrorInvalidDevice;
  const uint64_t limit_ns = (uint64_t)(timeout_s * 1e9);
  const int ck = accum_chunk_k > 0 ? accum_chunk_k : DEFAULT_CHUNK_K;
  const int chunk = ck / BK < 1 ? 1 : ck / BK;
  const int grid = 2 * (sm_count / 2);
  if (n128) {
    if (bf16)
      layer_tc2_group128_kernel<true><<<grid, NUM_THREADS, smem, s>>>(inst, count, group_timeout,
                                                                      queue, limit_ns, chunk);
    else
      layer_tc2_group128_kernel<false><<<grid, NUM_THREADS, smem, s>>>(
          inst, count, group_timeout, queue, limit_ns, chunk);
    return cudaGetLastError();
  }
  if (bf16)
    layer_tc2_group_kernel<true><<<grid, NUM_THREADS, smem, s>>>(
        inst, count, group_timeout, queue, limit_ns, chunk, k_snake, band);
  else
    layer_tc2_group_kernel<false><<<grid, NUM_THREADS, smem, s>>>(
        inst, count, group_timeout, queue, limit_ns, chunk, k_snake, band);
  return cudaGetLastError();
}

cudaError_t launch_layer_tc(const Layout& L, void* ws, cudaStream_t s, double timeout_s,
                            int accum_chunk_k, int cta_pair, int k_snake, int band,
                            int64_t* entries, double* pass_flops, int inject_stall,
                            int round_align) {
  using namespace tc;
  char* base = (char*)ws;
  const bool bf16 = L.precision == DMPT_DUAL_BF16;
  const int slices = 2 * (1 + L.k) * 2 + 2 * L.tape_states;
  CUtensorMap mA, mB;
  if (!make_map(&mA, base + L.off_ops16, L.Np, slices, BM, bf16) ||
      !make_map(&mB, base + L.off_ops16, L.Np, slices, BN, bf16))
    return cudaErrorInvalidValue;
  const int sms = device_setup();
  if (sms == 0) return cudaErrorInvalidDevice;
  const uint64_t limit_ns = (uint64_t)(timeout_s * 1e9);
  int ck = accum_chunk_k > 0 ? accum_chunk_k : DEFAULT_CHUNK_K;
  int chunk = ck / BK;
  if (chunk < 1) chunk = 1;
  State* st = (State*)(base + L.off_state);
  float* master = (float*)(base + L.off_master);
  uint16_t* ops = (uint16_t*)(base + L.off_ops16);
  double* partials = (double*)(base + L.off_partials);
  if (cta_pair) {
    const int64_t tiles = num_pair_tiles(L.Np);
    const int64_t max_items = tiles * (1 + L.k);
    int64_t pairs = sms / 2;
    if (pairs > max_items) pairs = max_items;
    const int grid = (int)(2 * pairs);
    auto kern = bf16 ? layer_tc2_kernel<true> : layer_tc2_kernel<false>;
    kern<<<grid, NUM_THREADS, P_SMEM_BYTES, s>>>(
        mA, st, master, ops, L.Np, L.k, partials, L.partial_tiles, limit_ns, chunk, k_snake, band,
        inject_stall, round_align);
    if (entries) *entries = 2 * tiles;
    if (pass_flops) *pass_flops = (double)tiles * 2 * BM * BN * (double)L.Np * 2.0;
    return cudaGetLastError();
  }
  const int64_t tiles = num_tiles(L.Np);
  // the number of jobs is only known on the device; size the grid for the
  // largest case and let surplus CTAs exit
  int64_t max_items = tiles * (1 + L.k);
  int grid = (int)(max_items < sms ? max_items : sms);
  if (bf16)
    layer_tc_kernel<true><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(mA, mB, st, master, ops, L.Np,
                                                                L.k, partials, L.partial_tiles,
                                                                limit_ns, chunk, inject_stall);
  else
    layer_tc_kernel<false><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(mA, mB, st, master, ops, L.Np,
                                                                 L.k, partials, L.partial_tiles,
                                                                 limit_ns, chunk, inject_stall);
  if (entries) *entries = tiles;
  if (pass_flops) *pass_flops = (double)tiles * BM * BN * (double)L.Np * 2.0;
  return cudaGetLastError();
}

}  // namespace dmpt
