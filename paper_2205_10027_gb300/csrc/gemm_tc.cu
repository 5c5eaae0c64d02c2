// Split-precision dense products on the 5th-generation tensor cores.
//
// Each FP64 operand is split into hi + lo parts of a narrow type (TF32 or BF16); the product
// op(A) op(B) is formed as hi*hi + hi*lo + lo*hi by tcgen05.mma with FP32 accumulation in
// TMEM, and the epilogue writes alpha * acc + beta * C (alpha * acc in FP32, the sum with the
// FP64 C in FP64).  One
// CTA computes a 128 x TN output tile: one thread issues TMA loads of the four operand tiles
// of a k-stage (A_hi, A_lo: 128 rows; B_hi, B_lo: TN rows; KB bytes of K per row) into a
// shared-memory ring, one thread issues the MMAs, and all warps drain the accumulator with
// tcgen05.ld.  Two shapes: 128 x 256 tiles with 4 stages of 64-byte-swizzled K-slices (the
// default: twice the MMA work per staged byte of A, and a deeper ring), and 128 x 128 tiles
// with 3 stages of 128-byte-swizzled slices.  Every wait on an mbarrier is bounded; on a
// timeout the CTA records an error and leaves without writing.
#include <cuda.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdlib>
#include "engine.h"
#include "gemm_tc.h"

namespace glasso {

namespace {
constexpr int TM = 128;
constexpr long long WAIT_CYCLES = 4000000000LL;  // about two seconds at 2 GHz
constexpr int GROUP_M = 12;

// Tile shape and shared-memory ring of one kernel configuration.
template <int TN_, int STAGES_, int KB_>
struct TcCfg {
  static constexpr int TN = TN_;
  static constexpr int STAGES = STAGES_;
  static constexpr int KB = KB_;                          // bytes of K per operand row and stage
  static constexpr int THREADS = TN == 256 ? 256 : 128;   // epilogue: one warp per 32 x 128 block
  static constexpr uint32_t TMEM_COLS = TN;               // FP32 accumulator columns
  static constexpr int A_BYTES = TM * KB;
  static constexpr int B_BYTES = TN * KB;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr uint64_t LAYOUT = KB == 128 ? 2 : 4;   // descriptor: 128- or 64-byte swizzle
  static_assert(KB == 128 || KB == 64, "swizzle width");
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
};
using CfgWide = TcCfg<256, 4, 64>;
using CfgSquare = TcCfg<128, 3, 128>;

struct TcArgs {
  double* C;
  int64_t ldc;
  int M, N, K;
  double alpha, beta;
  int lower, krule;
  int kstep;          // K elements per stage: KB / element size
  int group_m;        // tile rows per group of the tile order
  uint32_t idesc;     // tcgen05 instruction descriptor
  const int* flag;
  int* err;
  int no_loads;       // failure injection for the tests of the timeout path: the producer
                      // issues no load, so the MMA warp's bounded wait runs out
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Wait for the phase with the given parity to complete; false after WAIT_CYCLES.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile in a swizzled layout: rows of KB
// bytes, 8-row groups 8 * KB bytes apart (layout code 2 = 128-byte, 4 = 64-byte swizzle).
template <int KB, uint64_t LAYOUT>
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading-dimension offset (unused here)
  d |= (uint64_t)((8 * KB) >> 4) << 32;      // stride between 8-row groups
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= LAYOUT << 61;                         // swizzle mode
  return d;
}

__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                    uint32_t accumulate, bool tf32) {
  if (tf32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <class CF>
__global__ void __launch_bounds__(CF::THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
              const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
              const __grid_constant__ TcArgs p) {
  constexpr int TN = CF::TN, STAGES = CF::STAGES, STAGE_BYTES = CF::STAGE_BYTES;
  constexpr int A_BYTES = CF::A_BYTES, B_BYTES = CF::B_BYTES;
  constexpr uint32_t TMEM_COLS = CF::TMEM_COLS;
  dep_wait();
  dep_release();
  if (p.flag && *p.flag == 0) return;
  // grouped tile order: consecutive blocks walk down a column of GROUP_M tiles, so the
  // CTAs resident at one time cover a near-square patch and share operand panels in L2
  const int tiles_m = (p.M + TM - 1) / TM, tiles_n = (p.N + TN - 1) / TN;
  const int per_group = p.group_m * tiles_n;
  const int b = blockIdx.x;
  const int first_m = (b / per_group) * p.group_m;
  const int gm = min(p.group_m, tiles_m - first_m);
  const int tm = first_m + (b % per_group) % gm, tn = (b % per_group) / gm;
  const int row0 = tm * TM, col0 = tn * TN;
  if (p.lower && row0 + TM <= col0) return;  // tile entirely above the diagonal
  int k_lo = 0, k_hi = p.K;
  if (p.krule == KR_LO_COL) k_lo = col0;
  else if (p.krule == KR_LO_ROW) k_lo = row0;
  else if (p.krule == KR_HI_ROW) k_hi = min(p.K, row0 + TM);
  else if (p.krule == KR_HI_COL) k_hi = min(p.K, col0 + TN);
  k_lo = (k_lo / p.kstep) * p.kstep;
  const int nk = k_hi > k_lo ? (k_hi - k_lo + p.kstep - 1) / p.kstep : 0;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* s_abort = reinterpret_cast<int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const bool tf32 = p.kstep == 32;

  if (warp == 0 && lane == 0 && nk > 0) {
    // producer: TMA loads of the four operand tiles of each k-stage
    int issued = 0;
    for (int i = 0; i < (p.no_loads ? 0 : nk); ++i) {
      const int s = i % STAGES;
      const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
      if (i >= STAGES && !mbar_wait(&empty[s], ph ^ 1u)) { *s_abort = 1; break; }
      uint8_t* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      const int kx = k_lo + i * p.kstep;
      tma_load_2d(st, &mAh, &full[s], kx, row0);
      tma_load_2d(st + A_BYTES, &mAl, &full[s], kx, row0);
      tma_load_2d(st + 2 * A_BYTES, &mBh, &full[s], kx, col0);
      tma_load_2d(st + 2 * A_BYTES + B_BYTES, &mBl, &full[s], kx, col0);
      ++issued;
    }
    // do not leave while loads may still land in shared memory
    for (int i = (issued > STAGES ? issued - STAGES : 0); i < issued; ++i) {
      if (!*s_abort) break;
      mbar_wait(&full[i % STAGES], (uint32_t)(i / STAGES) & 1u);
    }
  } else if (warp == 1 && lane == 0 && nk > 0) {
    // MMA issuer: KB / 32 instructions of 32 bytes along K per stage, three products each
    for (int i = 0; i < nk; ++i) {
      const int s = i % STAGES;
      const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph)) { *s_abort = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
      for (int kk = 0; kk < CF::KB / 32; ++kk) {
        const uint64_t ah = sw_desc<CF::KB, CF::LAYOUT>(base + kk * 32);
        const uint64_t al = sw_desc<CF::KB, CF::LAYOUT>(base + A_BYTES + kk * 32);
        const uint64_t bh = sw_desc<CF::KB, CF::LAYOUT>(base + 2 * A_BYTES + kk * 32);
        const uint64_t bl = sw_desc<CF::KB, CF::LAYOUT>(base + 2 * A_BYTES + B_BYTES + kk * 32);
        mma(tmem, al, bh, p.idesc, (i | kk) != 0, tf32);
        mma(tmem, ah, bl, p.idesc, 1, tf32);
        mma(tmem, ah, bh, p.idesc, 1, tf32);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncthreads();

  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows of the tile) and the
  // columns of its 128-column half w / 4, 32 x 32 at a time; each block is transposed through
  // shared memory (the drained operand ring) so that a warp stores 32 consecutive doubles of
  // one row per instruction
  bool ok = !*s_abort;
  if (ok && nk > 0) ok = mbar_wait(done, 0);
  ok = __syncthreads_and(ok);  // uniform: tcgen05.ld below is warp-collective
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int wq = warp & 3;
  // warp w reads TMEM lanes 32 (w % 4) ..; with eight warps, w and w + 4 split the tile's
  // 32-column chunks between them
  constexpr int CH = TN / 32 / (CF::THREADS / 128);
  const int c_first = (warp >> 2) * CH, c_end = c_first + CH;
  float* stage = reinterpret_cast<float*>(smem) + warp * (32 * 33);  // [32][33] per warp
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(p.err, 1);
  } else {
    // alpha * acc in FP32 (alpha is 0 or +-1 in every product of the solver), converted to
    // FP64 by integer arithmetic; beta != 0 (the trailing updates A22 -= L21 L21^T of the
    // factorisation) adds it to the FP64 C with one FP64 FMA, so the Schur complement keeps
    // FP64 accuracy apart from the split product's own error.  That is one FP64 operation
    // per output element of a K-long product: ~40 us of FP64 pipe per n = 10^4
    // factorisation, spread over the whole GPU.  The 32 C entries a lane updates per chunk are
    // all loaded before the first is stored, so their latencies overlap instead of adding up
    // row by row.
    const float al = (float)p.alpha;
#pragma unroll 1
    for (int c = c_first; c < c_end; ++c) {
      float v[32];
      if (nk > 0) {
        tmem_ld32(tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(c * 32), v);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0.f;
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = v[j];  // row lane, column j
      __syncwarp();
      const int col = col0 + c * 32 + lane;
      const int rbase = row0 + wq * 32;
      double* const cbase = p.C + (int64_t)rbase * p.ldc + col;
      if (p.beta == 0.0) {
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
          const int r = rbase + rr;
          if (r >= p.M || col >= p.N || (p.lower && col > r)) continue;
          cbase[(int64_t)rr * p.ldc] = f32_to_f64(al * stage[rr * 33 + lane]);
        }
      } else {
        double cv[32];
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) {
          const int r = rbase + rr;
          const bool in = r < p.M && col < p.N && !(p.lower && col > r);
          cv[rr] = in ? cbase[(int64_t)rr * p.ldc] : 0.0;
        }
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) {
          const int r = rbase + rr;
          if (r >= p.M || col >= p.N || (p.lower && col > r)) continue;
          cbase[(int64_t)rr * p.ldc] = fma(p.beta, cv[rr], f32_to_f64(al * stage[rr * 33 + lane]));
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ---- operand splitting: out[r][c] = op[r][c], op = src or its transpose, into hi + lo parts
// hi = x rounded to SIG significant bits (nearest, ties away), lo = (x - hi) rounded the same
// way, returned as FP32 bit patterns (the low 24 - SIG mantissa bits zero).  Integer
// arithmetic only: the FP64 pipe of this part is too narrow to convert at memory speed.
// Magnitudes outside the FP32 normal range become 0 (hi) or are dropped (lo).
template <int SIG>
__device__ __forceinline__ void split_bits(double x, uint32_t& hi, uint32_t& lo) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FF);
  hi = 0;
  lo = 0;
  if (e == 0 || e == 0x7FF) return;
  const uint64_t M = (1ull << 52) | (b & ((1ull << 52) - 1));
  constexpr int SH = 53 - SIG;
  uint64_t Mh = (M + (1ull << (SH - 1))) >> SH;
  const int64_t rem = (int64_t)M - (int64_t)(Mh << SH);
  int fe = e - 1023 + 127;
  if (Mh >> SIG) {
    Mh >>= 1;
    fe += 1;
  }
  if (fe <= 0 || fe >= 255) return;
  hi = sign | ((uint32_t)fe << 23) | ((uint32_t)(Mh & ((1u << (SIG - 1)) - 1)) << (24 - SIG));
  if (rem == 0) return;
  uint64_t r = rem < 0 ? (uint64_t)(-rem) : (uint64_t)rem;
  const uint32_t slo = (((uint32_t)(b >> 63)) ^ (rem < 0 ? 1u : 0u)) << 31;
  int top = 63 - __clzll((long long)r);
  uint64_t rr;
  if (top >= SIG) {
    const int s2 = top - (SIG - 1);
    rr = (r + (1ull << (s2 - 1))) >> s2;
    if (rr >> SIG) {
      rr >>= 1;
      top += 1;
    }
  } else {
    rr = r << ((SIG - 1) - top);
  }
  const int fe_lo = top + e - 1075 + 127;
  if (fe_lo <= 0 || fe_lo >= 255) return;
  lo = slo | ((uint32_t)fe_lo << 23) | ((uint32_t)(rr & ((1u << (SIG - 1)) - 1)) << (24 - SIG));
}

// One split job: out[r][c] = op[r][c] for r < rows_out (zero rows at and beyond `rows`).
struct SplitJob {
  const double* src;
  int64_t lds;
  int rows, rows_out, cols, trans;
  void* hi;
  void* lo;
  int64_t ldo;
  int tiles_x;  // 64-column tiles of the output
  int vec;      // rows of src are 16-byte aligned (source read as double2)
};

// blockIdx.z selects the job: the A and B operands of a product are split in one launch.  A
// block covers 32 rows x 64 columns of the output (K, the column count, is a multiple of 64);
// lane tx owns columns 2 tx and 2 tx + 1 and reads them as one 16-byte load when the source
// allows it (op not transposed, 16-byte aligned rows), else through a shared-memory transpose;
// each hi / lo pair of columns leaves as one 4-byte (BF16) or 8-byte (TF32) store.
template <bool BF16>
__device__ __forceinline__ void split_store(const SplitJob& j, int64_t o, double x0, double x1) {
  uint32_t h0, l0, h1, l1;
  if (BF16) {
    split_bits<8>(x0, h0, l0);
    split_bits<8>(x1, h1, l1);
    reinterpret_cast<uint32_t*>(j.hi)[o >> 1] = (h0 >> 16) | (h1 & 0xFFFF0000u);
    reinterpret_cast<uint32_t*>(j.lo)[o >> 1] = (l0 >> 16) | (l1 & 0xFFFF0000u);
  } else {
    split_bits<11>(x0, h0, l0);
    split_bits<11>(x1, h1, l1);
    reinterpret_cast<uint2*>(j.hi)[o >> 1] = make_uint2(h0, h1);
    reinterpret_cast<uint2*>(j.lo)[o >> 1] = make_uint2(l0, l1);
  }
}

template <bool BF16>
__global__ void __launch_bounds__(256) k_split(const __grid_constant__ SplitJob ja, const __grid_constant__ SplitJob jb) {
  dep_wait();
  dep_release();
  const SplitJob& j = blockIdx.z == 0 ? ja : jb;
  const int tiles_y = (j.rows_out + 31) / 32;
  if ((int)blockIdx.x >= j.tiles_x || (int)blockIdx.y >= tiles_y) return;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 64;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int c = c0 + 2 * tx;                     // this lane's two columns c, c + 1
  const double* __restrict__ src = j.src;
  if (!j.trans && j.vec) {
    double2 v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + ty + 8 * i;
      v[i] = (r < j.rows) ? *reinterpret_cast<const double2*>(src + (int64_t)r * j.lds + c) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + ty + 8 * i;
      if (r < j.rows_out) split_store<BF16>(j, (int64_t)r * j.ldo + c, v[i].x, v[i].y);
    }
    return;
  }
  __shared__ double t[32][65];  // t[r][c - c0]
  if (!j.trans) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + ty + 8 * i;
      const bool in = r < j.rows;
      t[ty + 8 * i][2 * tx] = in ? src[(int64_t)r * j.lds + c] : 0.0;
      t[ty + 8 * i][2 * tx + 1] = in ? src[(int64_t)r * j.lds + c + 1] : 0.0;
    }
  } else {
    // op[r][c] = src[c][r]: src rows c0 .. c0 + 63, columns r0 + tx (coalesced)
    const int r = r0 + tx;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int sr = c0 + ty + 8 * i;
      t[tx][ty + 8 * i] = (r < j.rows) ? src[(int64_t)sr * j.lds + r] : 0.0;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty + 8 * i;
    if (r < j.rows_out) split_store<BF16>(j, (int64_t)r * j.ldo + c, t[ty + 8 * i][2 * tx], t[ty + 8 * i][2 * tx + 1]);
  }
}

// ---- host side --------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
    else
      cudaGetLastError();
  });
  return fn;
}

// 2-D map over a rows x cols array (row stride ld elements) with box_rows x (kb bytes) boxes,
// swizzled to match the kb-byte rows of the MMA descriptors
CUtensorMap make_map(void* base, bool bf16, int rows, int cols, int64_t ld, int box_rows, int kb) {
  CUtensorMap m;
  const int esz = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(kb / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_fn()(&m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                                 base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 kb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(GLASSO_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return m;
}

SplitJob split_job(const double* src, int64_t lds, int rows, int rows_out, int cols, bool trans, void* hi,
                   void* lo, int64_t ldo) {
  if (cols % 64 || ldo % 2) throw Error(GLASSO_ERR_ARG, "split: K must be a multiple of 64");
  const bool vec = (reinterpret_cast<uintptr_t>(src) % 16) == 0 && lds % 2 == 0;
  return SplitJob{src, lds, rows, rows_out, cols, trans ? 1 : 0, hi, lo, ldo, cols / 64, vec ? 1 : 0};
}

// Both jobs in one launch; jobs == 1 runs only the first.
void split2(const SplitJob& a, const SplitJob& b, bool bf16, cudaStream_t st, int jobs = 2) {
  dim3 grid(std::max(a.tiles_x, b.tiles_x), (std::max(a.rows_out, b.rows_out) + 31) / 32, jobs);
  if (bf16)
    launch_dependent(k_split<true>, grid, dim3(32, 8), 0, st, a, b);
  else
    launch_dependent(k_split<false>, grid, dim3(32, 8), 0, st, a, b);
}

int* g_err = nullptr;     // device error word of the tensor-core kernels
bool g_no_loads = false;  // GLASSO_TEST_TC_NO_LOADS=1 (read once): see TcArgs::no_loads
}  // namespace

bool tc_available() { return encode_fn() != nullptr; }

// A parts padded to 128 rows, B parts to the widest tile (256 rows); 4-byte elements at most
size_t tc_scratch_bytes_for(int np) {
  const size_t mp = (size_t)(np + 127) / 128 * 128, npb = (size_t)(np + 255) / 256 * 256;
  return (2 * mp + 2 * npb) * (size_t)np * sizeof(float) + 256;
}

bool tc_gemm_supported(const GemmArgs& a) {
  return a.M % 64 == 0 && a.N % 64 == 0 && a.K % 64 == 0 && a.M > 0 && a.N > 0 && a.K > 0;
}

const int* tc_error_word() { return g_err; }

void tc_clear_error(cudaStream_t st) {
  if (g_err) CUDA_CHECK(cudaMemsetAsync(g_err, 0, sizeof(int), st));
}

int tc_error_flag(cudaStream_t st) {
  if (!g_err) return 0;
  int h = 0;
  CUDA_CHECK(cudaMemcpyAsync(&h, g_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(cudaStreamSynchronize(st));
  return h;
}

namespace {
template <class CF>
void tc_gemm_cfg(const GemmArgs& a, bool bf16, void* scratch, size_t scratch_bytes, cudaStream_t st) {
  constexpr int TN = CF::TN;
  const size_t esz = bf16 ? 2 : 4;
  // split operands are stored with their row counts rounded up to the tile (zero rows beyond
  // M or N), so every TMA box lies inside its tensor
  const int Mp = (a.M + TM - 1) / TM * TM, Np = (a.N + TN - 1) / TN * TN;
  const size_t need = esz * ((size_t)2 * Mp * a.K + (size_t)2 * Np * a.K);
  if (need + 256 > scratch_bytes) throw Error(GLASSO_ERR_OOM, "tensor-core scratch too small");
  static std::once_flag once;
  std::call_once(once, [] {
    CUDA_CHECK(cudaFuncSetAttribute(k_gemm_tc<CF>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM_BYTES));
  });
  uint8_t* base = static_cast<uint8_t*>(scratch);
  void* Ah = base;
  void* Al = base + esz * (size_t)Mp * a.K;
  void* Bh = base + esz * (size_t)2 * Mp * a.K;
  void* Bl = base + esz * ((size_t)2 * Mp * a.K + (size_t)Np * a.K);
  // A part: [M][K] = op(A); B part: [N][K] = op(B)^T.  When they are the same matrix (the
  // symmetric products op(A) op(A)^T of the trailing updates and of W = X^T X) it is split
  // once, with the B part's row padding, and both maps read it.
  const bool same = a.A == a.B && a.lda == a.ldb && (a.transA != 0) == (a.transB == 0) && a.M == a.N;
  if (same) {
    split2(split_job(a.B, a.ldb, a.N, Np, a.K, a.transB == 0, Bh, Bl, a.K),
           split_job(a.B, a.ldb, a.N, Np, a.K, a.transB == 0, Bh, Bl, a.K), bf16, st, 1);
    Ah = Bh;
    Al = Bl;
  } else {
    split2(split_job(a.A, a.lda, a.M, Mp, a.K, a.transA != 0, Ah, Al, a.K),
           split_job(a.B, a.ldb, a.N, Np, a.K, a.transB == 0, Bh, Bl, a.K), bf16, st);
  }
  const CUtensorMap mAh = make_map(Ah, bf16, Mp, a.K, a.K, TM, CF::KB);
  const CUtensorMap mAl = make_map(Al, bf16, Mp, a.K, a.K, TM, CF::KB);
  const CUtensorMap mBh = make_map(Bh, bf16, Np, a.K, a.K, TN, CF::KB);
  const CUtensorMap mBl = make_map(Bl, bf16, Np, a.K, a.K, TN, CF::KB);
  TcArgs p;
  p.C = a.C;
  p.ldc = a.ldc;
  p.M = a.M;
  p.N = a.N;
  p.K = a.K;
  p.alpha = a.alpha;
  p.beta = a.beta;
  p.lower = a.lower;
  p.krule = a.krule;
  p.kstep = CF::KB / (int)esz;
  p.group_m = GROUP_M;
  const uint32_t ab = bf16 ? 1u : 2u;  // operand format: BF16 = 1 (kind::f16), TF32 = 2 (kind::tf32)
  p.idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
  p.flag = a.flag;
  p.err = g_err;
  p.no_loads = g_no_loads ? 1 : 0;
  dim3 grid(((a.N + TN - 1) / TN) * ((a.M + TM - 1) / TM));
  launch_dependent(k_gemm_tc<CF>, grid, CF::THREADS, CF::SMEM_BYTES, st, mAh, mAl, mBh, mBl, p);
}
}  // namespace

void tc_gemm(const GemmArgs& a, TcKind kind, void* scratch, size_t scratch_bytes, cudaStream_t st, TcTile tile) {
  static std::once_flag once;
  static bool square_default = false;
  std::call_once(once, [] {
    CUDA_CHECK(cudaMalloc(&g_err, sizeof(int)));
    CUDA_CHECK(cudaMemset(g_err, 0, sizeof(int)));
    // GLASSO_TC_TILE=128 makes the 128 x 128 tiles the default (for comparison); the
    // autotuner may pick either tile per product shape
    const char* t = std::getenv("GLASSO_TC_TILE");
    square_default = t && std::atoi(t) == 128;
    const char* nl = std::getenv("GLASSO_TEST_TC_NO_LOADS");
    g_no_loads = nl && nl[0] == '1';
  });
  const bool bf16 = kind == TcKind::BF16x3;
  const bool square = tile == TcTile::Square || (tile == TcTile::Default && square_default);
  if (square)
    tc_gemm_cfg<CfgSquare>(a, bf16, scratch, scratch_bytes, st);
  else
    tc_gemm_cfg<CfgWide>(a, bf16, scratch, scratch_bytes, st);
}

}  // namespace glasso
