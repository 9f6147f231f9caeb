// gemm_tc.cu -- X = Q W (eq. (10)) on the 5th-generation tensor cores with
// FP64-level accuracy from BF16 products (an Ozaki-type split).
//
// Splitting.  Row i of Q is scaled by 2^-e_i (|Q_ij| 2^-e_i < 1/2) and written
// as five signed 8-bit digits m_p = rint(256 t_{p-1}), t_p = 256 t_{p-1} - m_p,
// so Q_ij = 2^(e_i-8) sum_p m_p 2^(-8(p-1)) + O(2^(e_i-41)).  The stored BF16
// slice p holds m_p 2^(-8(p-1)) (|m_p| <= 128: exact in BF16).  Columns of W
// are split the same way with exponents f_r.  Then
//   X_ir = 2^(e_i + f_r - 16) sum_{p+q <= 6} sum_j Qs_p[i,j] Ws_q[r,j]
// drops only products below 2^-40 of the row/column scale (15 slice pairs).
//
// Exact accumulation.  Every product of slices p, q is an integer multiple of
// 2^(-8(p+q-2)) of magnitude <= 2^14.  Pairs with the same g = p+q share one
// FP32 accumulator in tensor memory; for g <= 4 (6 pairs) a chunk of 256
// K-steps sums at most 3*256*2^14 < 2^24 such multiples, so the FP32 sum is
// exact, and the chunk sums are drained into double-float (hi, lo) registers.
// Groups g = 5, 6 (9 pairs) lie below 2^-24 of the result and accumulate over
// the whole K in one FP32 accumulator.
//
// Pipeline (one 128 x 128 output tile per CTA, 10 warps):
//   warp 0      TMA producer: 5 Q-slice and 5 W-slice tiles of 128 x 32 BF16
//               per stage (64-byte swizzle), 2 stages, mbarrier handshakes.
//   warp 1      MMA issuer: tcgen05.mma kind::f16, M=128 N=128 K=16, into four
//               TMEM accumulators (g=2,3,4 exact, g>=5 tail: 512 columns).
//   warps 2-9   epilogue: drain the exact groups every 256 K-steps
//               (tcgen05.ld), final scaling and FP64 stores.
// Every mbarrier wait is bounded; on timeout the CTA records EIG status bit
// ST_TIMEOUT, waits (bounded) for its own copies and MMAs, frees TMEM, exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "eig_internal.cuh"

namespace eig {
namespace {

constexpr int kSlices = kTcSlices;
constexpr int BM = 128, BN = 128, BK = 32;
constexpr int kStages = 2;
constexpr int kChunk = 256;                     // exact-accumulation chunk (K)
constexpr int kStagesPerChunk = kChunk / BK;    // 8
constexpr int kTileBytes = BM * BK * 2;         // 8 KB (A and B tiles are the same size)
constexpr int kStageBytes = 2 * kSlices * kTileBytes;  // 80 KB
constexpr int kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr int kThreads = 320;
constexpr int kTmemCols = 512;
constexpr unsigned long long kWaitCycles = 4000000000ull;  // ~2 s at 2 GHz

// Instruction descriptor, kind::f16: D=F32, A=B=BF16, both K-major, N=128, M=128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
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
// Bounded wait: false after ~2 s (the caller then records a timeout).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

// ---- TMA --------------------------------------------------------------------
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// ---- tcgen05 ----------------------------------------------------------------
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
// Three 16-column loads (one per exact group, columns `col` of each) and one
// wait: the waits, not the loads, dominate the drain.  The outputs are
// early-clobber: a later load's address must not share a register with an
// earlier load's destination.
__device__ __forceinline__ void tc_ld16x3(uint32_t t0, uint32_t t1, uint32_t t2, float (&v)[3][16]) {
  uint32_t r[48];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%48];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, "
      "%27, %28, %29, %30, %31}, [%49];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, "
      "%43, %44, %45, %46, %47}, [%50];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=&r"(r[0]), "=&r"(r[1]), "=&r"(r[2]), "=&r"(r[3]), "=&r"(r[4]), "=&r"(r[5]), "=&r"(r[6]), "=&r"(r[7]),
        "=&r"(r[8]), "=&r"(r[9]), "=&r"(r[10]), "=&r"(r[11]), "=&r"(r[12]), "=&r"(r[13]), "=&r"(r[14]),
        "=&r"(r[15]), "=&r"(r[16]), "=&r"(r[17]), "=&r"(r[18]), "=&r"(r[19]), "=&r"(r[20]), "=&r"(r[21]),
        "=&r"(r[22]), "=&r"(r[23]), "=&r"(r[24]), "=&r"(r[25]), "=&r"(r[26]), "=&r"(r[27]), "=&r"(r[28]),
        "=&r"(r[29]), "=&r"(r[30]), "=&r"(r[31]), "=&r"(r[32]), "=&r"(r[33]), "=&r"(r[34]), "=&r"(r[35]),
        "=&r"(r[36]), "=&r"(r[37]), "=&r"(r[38]), "=&r"(r[39]), "=&r"(r[40]), "=&r"(r[41]), "=&r"(r[42]),
        "=&r"(r[43]), "=&r"(r[44]), "=&r"(r[45]), "=&r"(r[46]), "=&r"(r[47])
      : "r"(t0), "r"(t1), "r"(t2)
      : "memory");
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int i = 0; i < 16; ++i) v[g][i] = __uint_as_float(r[16 * g + i]);
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major operand tile of 64-byte rows (32
// BF16, two MMA K steps), 64-byte swizzle, 8-row core groups 512 bytes apart
// (SBO), version 1, layout SWIZZLE_64B (4).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused, swizzled)
  d |= (uint64_t)((8 * BK * 2 >> 4) & 0x3FFFu) << 32;  // stride byte offset: 8 rows
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)4 << 61;                          // SWIZZLE_64B
  return d;
}

// ---- double-float accumulation ------------------------------------------------
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

struct GemmArgs {
  int n;           // rows of X and Q; the contraction length
  int ncols;       // columns of X and W (n for the full update)
  int ldx;         // leading dimension of X (column-major)
  double* X;
  const int* erow;  // e_i
  const int* fcol;  // f_r
  const DevStatus* st;  // skip on invalid input (may be null)
  int* err;             // timeout flag (status flags word)
  int tiles_m, tiles_n;
  // Non-zero map of W's slices 0 and 1 per 128-column x 32-row tile (bits 0,
  // 1; word tn * nch + j / 32), or null: MMAs against an all-zero W tile are
  // skipped (their products are exactly zero).
  const unsigned* wnz = nullptr;
  int nch = 0;
};

// One 128 x 128 output tile (the whole CTA takes part).
__device__ __forceinline__ void gemm_tc_tile(const CUtensorMap* mapQp, const CUtensorMap* mapWp,
                                             const GemmArgs& a, int tile) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  if (a.st && (a.st->flags & (ST_UNSORTED | ST_NONFINITE))) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // 1024-aligned operand area, barriers after it.
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  const uint32_t bar_full0 = smem_u32(&bars[0]);       // kStages
  const uint32_t bar_empty0 = smem_u32(&bars[kStages]);  // kStages
  const uint32_t bar_accf = smem_u32(&bars[2 * kStages]);
  const uint32_t bar_acce = smem_u32(&bars[2 * kStages + 1]);
  const uint32_t bar_done = smem_u32(&bars[2 * kStages + 2]);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(&bars[2 * kStages + 3]);
  __shared__ int s_fail;

  // Tile raster: groups of 16 row tiles sweep the columns together (L2 reuse).
  const int group = 16;
  const int per_group = group * a.tiles_n;
  const int gi = tile / per_group;
  const int first_m = gi * group;
  const int gsz = min(group, a.tiles_m - first_m);
  const int tm = first_m + (tile % per_group) % gsz;
  const int tn = (tile % per_group) / gsz;
  const int m0 = tm * BM, n0 = tn * BN;
  const int nk = (a.n + BK - 1) / BK;
  const int nchunks = (nk + kStagesPerChunk - 1) / kStagesPerChunk;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bar_full0 + 8 * s, 1);
      mbar_init(bar_empty0 + 8 * s, 1);
    }
    mbar_init(bar_accf, 1);
    mbar_init(bar_acce, 8);  // one arrival per epilogue warp
    mbar_init(bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      for (int kb = 0; kb < nk && ok; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (kb / kStages) & 1;
        if (!mbar_wait(bar_empty0 + 8 * s, ph ^ 1)) {
          ok = false;
          break;
        }
        if (*(volatile int*)&s_fail) {
          ok = false;
          break;
        }
        mbar_expect_tx(bar_full0 + 8 * s, kStageBytes);
        const uint32_t st_base = sbase + s * kStageBytes;
        for (int p = 0; p < kSlices; ++p)
          tma_load_3d(st_base + p * kTileBytes, mapQp, kb * BK, m0, p, bar_full0 + 8 * s);
        for (int q = 0; q < kSlices; ++q)
          tma_load_3d(st_base + (kSlices + q) * kTileBytes, mapWp, kb * BK, n0, q,
                      bar_full0 + 8 * s);
        issued = kb + 1;
      }
      if (!ok) {
        atomicOr(&s_fail, 1);
        // Wait (bounded) for the copies this thread has in flight.
        for (int kb = max(0, issued - kStages); kb < issued; ++kb)
          mbar_wait(bar_full0 + 8 * (kb % kStages), (kb / kStages) & 1);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      // Exact groups: whether an MMA has reset the group's accumulator in the
      // current chunk (the first one of a chunk overwrites, the rest add).
      bool started[3] = {false, false, false};
      for (int kb = 0; kb < nk && ok; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (kb / kStages) & 1;
        const int chunk = kb / kStagesPerChunk;
        const bool first_in_chunk = (kb % kStagesPerChunk) == 0;
        const bool last_in_chunk = ((kb % kStagesPerChunk) == kStagesPerChunk - 1) || (kb == nk - 1);
        // which of W's slices 0 and 1 have non-zeros in this stage's tile
        const unsigned wbits = a.wnz ? __ldg(a.wnz + (size_t)tn * a.nch + (kb * BK) / 32) : 3u;
        if (first_in_chunk) started[0] = started[1] = started[2] = false;
        if (first_in_chunk && chunk > 0) {
          if (!mbar_wait(bar_acce, (chunk - 1) & 1)) {
            ok = false;
            break;
          }
        }
        if (!mbar_wait(bar_full0 + 8 * s, ph)) {
          ok = false;
          break;
        }
        if (*(volatile int*)&s_fail) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t st_base = sbase + s * kStageBytes;
        // exact groups: g = p + q (0-based) in {0, 1, 2} -> TMEM columns 0, 128, 256
#pragma unroll
        for (int g = 0; g < 3; ++g) {
#pragma unroll
          for (int p = 0; p <= g; ++p) {
            const int q = g - p;
            if (q <= 1 && !((wbits >> q) & 1u)) continue;  // all-zero W tile
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
              const uint64_t ad = smem_desc(st_base + p * kTileBytes + ks * 32);
              const uint64_t bd = smem_desc(st_base + (kSlices + q) * kTileBytes + ks * 32);
              tc_mma(tmem + g * BN, ad, bd, started[g] ? 1u : 0u);
              started[g] = true;
            }
          }
        }
        if (last_in_chunk) {
          // A group that saw no MMA in this chunk still holds the last chunk's
          // sum: overwrite it with a product against this stage's all-zero W
          // slice 0 (every pair of the group was skipped, (g, 0) included).
#pragma unroll
          for (int g = 0; g < 3; ++g) {
            if (started[g]) continue;
            const uint64_t ad = smem_desc(st_base + g * kTileBytes);
            const uint64_t bd = smem_desc(st_base + kSlices * kTileBytes);
            tc_mma(tmem + g * BN, ad, bd, 0u);
            started[g] = true;
          }
          tc_commit(bar_accf);
        }
        // tail groups: p + q in {3, 4} -> TMEM column 384, accumulated over all K
#pragma unroll
        for (int g = 3; g < kSlices; ++g) {
#pragma unroll
          for (int p = 0; p <= g; ++p) {
            const int q = g - p;
            if (p >= kSlices || q >= kSlices) continue;
            if (q <= 1 && !((wbits >> q) & 1u)) continue;  // all-zero W tile (never the first MMA: q = 3)
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
              const uint64_t ad = smem_desc(st_base + p * kTileBytes + ks * 32);
              const uint64_t bd = smem_desc(st_base + (kSlices + q) * kTileBytes + ks * 32);
              const bool acc = !(kb == 0 && g == 3 && p == 0 && ks == 0);
              tc_mma(tmem + 3 * BN, ad, bd, acc ? 1u : 0u);
            }
          }
        }
        tc_commit(bar_empty0 + 8 * s);
      }
      if (!ok) atomicOr(&s_fail, 1);
      // All MMAs issued so far complete -> bar_done; wait for it (bounded) so
      // that TMEM is never freed under an MMA in flight.
      tc_commit(bar_done);
      if (!mbar_wait(bar_done, 0)) atomicOr(&s_fail, 1);
    }
  } else {
    // ---------------- epilogue (8 warps) ----------------
    const int quad = warp & 3;             // TMEM lanes 32*quad .. +31
    const int half = (warp - 2) >> 2;      // columns 64*half .. +63
    const int row = m0 + quad * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
    float hi[64], lo[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) {
      hi[c] = 0.f;
      lo[c] = 0.f;
    }
    bool ok = true;
    for (int ch = 0; ch < nchunks && ok; ++ch) {
      if (!mbar_wait(bar_accf, ch & 1)) {
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int cb = 0; cb < 4; ++cb) {
        const uint32_t col = tmem + lane_addr + (uint32_t)(half * 64 + cb * 16);
        float v[3][16];
        tc_ld16x3(col, col + BN, col + 2 * BN, v);
#pragma unroll
        for (int g = 0; g < 3; ++g)
#pragma unroll
          for (int c = 0; c < 16; ++c) df_add(hi[cb * 16 + c], lo[cb * 16 + c], v[g][c]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_acce);
    }
    if (ok && mbar_wait(bar_done, 0)) {
      tc_fence_after();
#pragma unroll
      for (int cb = 0; cb < 4; ++cb) {
        float v[16];
        tc_ld16(tmem + lane_addr + 3 * BN + (uint32_t)(half * 64 + cb * 16), v);
#pragma unroll
        for (int c = 0; c < 16; ++c) df_add(hi[cb * 16 + c], lo[cb * 16 + c], v[c]);
      }
      if (row < a.n) {
        const int er = a.erow[row];
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          const int col = n0 + half * 64 + c;
          if (col < a.ncols) {
            const double x = (double)hi[c] + (double)lo[c];
            a.X[(size_t)col * a.ldx + row] = ldexp(x, er + a.fcol[col] - 16);
          }
        }
      }
    } else {
      ok = false;
    }
    if (!ok) atomicOr(&s_fail, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (s_fail && threadIdx.x == 0) atomicOr(a.err, ST_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap mapQ, const __grid_constant__ CUtensorMap mapW,
                   GemmArgs a) {
  gemm_tc_tile(&mapQ, &mapW, a, blockIdx.x);
}

// Tiles of every update of a table: CTA b handles tile (b - prefix[p]) of update
// p; the tensor maps (Q slices, W slices per update) live in global memory.
__global__ void __launch_bounds__(kThreads, 1)
    gemm_tc_grouped_kernel(const CUtensorMap* __restrict__ maps, const ProbDesc* __restrict__ P,
                           const int* __restrict__ tile_prefix, int count) {
  const int p = find_owner(tile_prefix, count, (int)blockIdx.x);
  const ProbDesc& d = P[p];
  const CUtensorMap* mq = maps + 2 * p;
  const CUtensorMap* mw = maps + 2 * p + 1;
  if (threadIdx.x == 0) {
    // The maps were written by a host copy: order them for the tensor-map proxy.
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mq) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mw) : "memory");
  }
  GemmArgs a;
  a.n = d.n;
  a.ncols = d.n;
  a.ldx = d.n;
  a.X = d.Xout;
  a.erow = d.erow;
  a.fcol = d.fcol;
  a.st = d.st;
  a.err = &d.st->flags;
  a.tiles_m = (d.n + BM - 1) / BM;
  a.tiles_n = a.tiles_m;
  a.wnz = d.wnz;
  a.nch = (d.n + 31) / 32;
  gemm_tc_tile(mq, mw, a, (int)blockIdx.x - tile_prefix[p]);
}

// Non-zero map of W's slices 0 and 1: CTA = one 128 x 128 GEMM tile of an
// update (128 columns r of W^T, 128 rows j = four 32-row chunks); thread t
// reads column r = r0 + t % 128 of slice t / 128, 64 bytes per chunk.
__global__ void __launch_bounds__(256) wnz_scan_grouped_kernel(const ProbDesc* __restrict__ P, int count,
                                                               const int* __restrict__ tile_prefix) {
  __shared__ unsigned flags[4];
  const int p = find_owner(tile_prefix, count, (int)blockIdx.x);
  const ProbDesc& d = P[p];
  if (!d.wnz || (d.st->flags & (ST_UNSORTED | ST_NONFINITE))) return;  // uniform across the CTA
  const int n = d.n;
  const int tiles = (n + BM - 1) / BM;
  const int local = (int)blockIdx.x - tile_prefix[p];
  const int jb = local / tiles, rt = local % tiles;
  const int nch = (n + 31) / 32;
  const int lds = (n + 63) / 64 * 64;
  const size_t plane = (size_t)lds * (size_t)n;
  if (threadIdx.x < 4) flags[threadIdx.x] = 0u;
  __syncthreads();
  const int q = threadIdx.x >> 7;
  const int r = rt * BN + (threadIdx.x & 127);
  if (r < n) {
    const __nv_bfloat16* row = d.Ws + (size_t)q * plane + (size_t)r * lds;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j0 = jb * BM + c * 32;
      if (j0 >= lds) break;
      const uint4* v = reinterpret_cast<const uint4*>(row + j0);  // 64 bytes, 16-byte aligned
      unsigned nz = 0u;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const uint4 x = __ldcg(v + w);
        nz |= (x.x | x.y | x.z | x.w) & 0x7fff7fffu;  // any non-zero BF16 (either sign of zero ignored)
      }
      if (nz) atomicOr(&flags[c], 1u << q);
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // Slice-pair products the GEMM issues for these K steps of tile column rt,
    // over every tile row: 15 per step, less the 5 pairs (p, 0) when slice 0
    // is all zero and the 4 pairs (p, 1) when slice 1 is.
    unsigned long long issued = 0ull;
    if (threadIdx.x < 4) {
      const int ch = jb * 4 + threadIdx.x;
      if (ch < nch) {
        const unsigned f = flags[threadIdx.x];
        d.wnz[(size_t)rt * nch + ch] = f;
        issued = (unsigned long long)(15 - ((f & 1u) ? 0 : 5) - ((f & 2u) ? 0 : 4)) * (unsigned long long)tiles;
      }
    }
#pragma unroll
    for (int o = 2; o > 0; o >>= 1) issued += __shfl_down_sync(0xffffffffu, issued, o);
    if (threadIdx.x == 0 && issued)
      atomicAdd(reinterpret_cast<unsigned long long*>(&d.st->tc_pair_tiles), issued);
  }
}

// ---- slicing ------------------------------------------------------------------
// Row maxima of |Q| (column-major), as ordered bit patterns of non-negative doubles.
__global__ void rowmax_kernel(int n, const double* __restrict__ Q,
                              unsigned long long* __restrict__ rmax, const DevStatus* st) {
  if (st && (st->flags & (ST_UNSORTED | ST_NONFINITE))) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cols_per = (n + gridDim.y - 1) / gridDim.y;
  const int j0 = blockIdx.y * cols_per, j1 = min(n, j0 + cols_per);
  double m = 0.0;
  for (int j = j0; j < j1; ++j) m = fmax(m, fabs(Q[(size_t)j * n + i]));
  atomicMax(&rmax[i], (unsigned long long)__double_as_longlong(m));
}

// Q (column-major) -> slices Qs[p][i][j] (row-major, j contiguous, leading dim lds).
__global__ void slice_q_kernel(int n, const double* __restrict__ Q,
                               const unsigned long long* __restrict__ rmax, int* __restrict__ erow,
                               __nv_bfloat16* __restrict__ Qs, size_t plane, int lds,
                               const DevStatus* st) {
  if (st && (st->flags & (ST_UNSORTED | ST_NONFINITE))) return;
  __shared__ __nv_bfloat16 tile[kSlices][32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int jj = ty; jj < 32; jj += 8) {
    const int i = i0 + tx, j = j0 + jj;
    __nv_bfloat16 d[kSlices];
    if (i < n && j < n) {
      const int e = tc_scale_exp(__longlong_as_double((long long)rmax[i]));
      tc_split_scaled(Q[(size_t)j * n + i], ldexp(1.0, -e), d);
      if (j == 0) erow[i] = e;
    } else {
#pragma unroll
      for (int p = 0; p < kSlices; ++p) d[p] = __double2bfloat16(0.0);
    }
#pragma unroll
    for (int p = 0; p < kSlices; ++p) tile[p][tx][jj] = d[p];
  }
  __syncthreads();
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii, j = j0 + tx;
    if (i < n && j < n) {
#pragma unroll
      for (int p = 0; p < kSlices; ++p) Qs[(size_t)p * plane + (size_t)i * lds + j] = tile[p][ii][tx];
    }
  }
}

// Grouped versions: block b of the row-max grid covers rows of update p,
// block b of the slice grid one 32 x 32 tile of update p.
__global__ void rowmax_grouped_kernel(const ProbDesc* __restrict__ P, int count,
                                      const int* __restrict__ rb_prefix) {
  const int p = find_owner(rb_prefix, count, (int)blockIdx.x);
  const ProbDesc& d = P[p];
  if (d.st->flags & (ST_UNSORTED | ST_NONFINITE)) return;
  const int n = d.n;
  const int i = ((int)blockIdx.x - rb_prefix[p]) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cols_per = (n + gridDim.y - 1) / gridDim.y;
  const int j0 = blockIdx.y * cols_per, j1 = min(n, j0 + cols_per);
  const double* Qsrc = d.st->n_runs ? d.Xout : d.Q;  // Xout holds Q~ = Q B when lam has runs
  double m = 0.0;
  for (int j = j0; j < j1; ++j) m = fmax(m, fabs(Qsrc[(size_t)j * n + i]));
  if (j1 > j0) atomicMax(&d.rmax[i], (unsigned long long)__double_as_longlong(m));
}

__global__ void slice_q_grouped_kernel(const ProbDesc* __restrict__ P, int count,
                                       const int* __restrict__ tile_prefix) {
  __shared__ __nv_bfloat16 tile[kSlices][32][33];
  const int p = find_owner(tile_prefix, count, (int)blockIdx.x);
  const ProbDesc& d = P[p];
  if (d.st->flags & (ST_UNSORTED | ST_NONFINITE)) return;  // uniform across the CTA
  const int n = d.n;
  const int nt = (n + 31) / 32;
  const int local = (int)blockIdx.x - tile_prefix[p];
  const int i0 = (local / nt) * 32, j0 = (local % nt) * 32;
  const int lds = (n + 63) / 64 * 64;
  const size_t plane = (size_t)lds * (size_t)n;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const double* Qsrc = d.st->n_runs ? d.Xout : d.Q;  // Xout holds Q~ = Q B when lam has runs
  // The thread's row is fixed: its scale is formed once (one FMA per entry left).
  const int irow = i0 + tx;
  int erow_i = 0;
  double s40 = 0.0;
  if (irow < n) {
    erow_i = tc_scale_exp(__longlong_as_double((long long)d.rmax[irow]));
    s40 = ldexp(1.0, 40 - erow_i);
  }
  for (int jj = ty; jj < 32; jj += 8) {
    const int i = irow, j = j0 + jj;
    __nv_bfloat16 dd[kSlices];
    if (i < n && j < n) {
      tc_split_prescaled(Qsrc[(size_t)j * n + i], s40, dd);
      if (j == 0) d.erow[i] = erow_i;
    } else {
#pragma unroll
      for (int q = 0; q < kSlices; ++q) dd[q] = __double2bfloat16(0.0);
    }
#pragma unroll
    for (int q = 0; q < kSlices; ++q) tile[q][tx][jj] = dd[q];
  }
  __syncthreads();
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii, j = j0 + tx;
    if (i < n && j < n) {
#pragma unroll
      for (int q = 0; q < kSlices; ++q) d.Qs[(size_t)q * plane + (size_t)i * lds + j] = tile[q][ii][tx];
    }
  }
}

// Columns of a column-major n x m matrix W -> slices Ws[q][r][j] of W^T (row r =
// column r of W, j contiguous, leading dim lds), each with its own exponent
// f_r (one CTA per column: max |W[:, r]|, then the split).
constexpr int kRowThreads = 256;
__global__ void __launch_bounds__(kRowThreads) slice_cols_kernel(int n, const double* __restrict__ W,
                                                                 int* __restrict__ fcol,
                                                                 __nv_bfloat16* __restrict__ Ws, size_t plane,
                                                                 int lds) {
  __shared__ double sh[kRowThreads / 32];
  const int r = blockIdx.x;
  const double* w = W + (size_t)r * n;
  double mx = 0.0;
  for (int j = threadIdx.x; j < n; j += kRowThreads) mx = fmax(mx, fabs(w[j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < kRowThreads / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) sh[0] = mx;
  }
  __syncthreads();
  const int f = tc_scale_exp(sh[0]);
  if (threadIdx.x == 0) fcol[r] = f;
  const double s40 = ldexp(1.0, 40 - f);
  for (int j = threadIdx.x; j < n; j += kRowThreads) {
    __nv_bfloat16 d[kSlices];
    tc_split_prescaled(w[j], s40, d);
#pragma unroll
    for (int q = 0; q < kSlices; ++q) Ws[(size_t)q * plane + (size_t)r * lds + j] = d[q];
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// Map of a slice stack: kSlices planes of `rows` rows of n BF16 (leading dim lds).
int make_map(CUtensorMap* map, const void* base, int n, int lds, int rows) {
  if (!g_encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return -1;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)rows, (cuuint64_t)kSlices};
  cuuint64_t strides[2] = {(cuuint64_t)lds * 2, (cuuint64_t)lds * 2 * (cuuint64_t)rows};
  cuuint32_t box[3] = {BK, 128, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -2;
}

}  // namespace

int tc_slice_ld(int n) { return (n + 63) / 64 * 64; }
size_t tc_slice_plane(int n) { return (size_t)tc_slice_ld(n) * (size_t)n; }
int tc_num_slices() { return kSlices; }

cudaError_t launch_slice_q(int n, const double* Q, unsigned long long* rmax, int* erow,
                           __nv_bfloat16* Qs, const DevStatus* st, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(rmax, 0, sizeof(unsigned long long) * n, s);
  if (e != cudaSuccess) return e;
  dim3 g1((n + 255) / 256, (unsigned)min(64, max(1, n / 64)));
  rowmax_kernel<<<g1, 256, 0, s>>>(n, Q, rmax, st);
  dim3 g2((n + 31) / 32, (n + 31) / 32);
  slice_q_kernel<<<g2, dim3(32, 8), 0, s>>>(n, Q, rmax, erow, Qs, tc_slice_plane(n), tc_slice_ld(n),
                                            st);
  return cudaGetLastError();
}

cudaError_t launch_slice_cols(int n, int m, const double* W, int* fcol, __nv_bfloat16* Ws, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  slice_cols_kernel<<<m, kRowThreads, 0, s>>>(n, W, fcol, Ws, (size_t)tc_slice_ld(n) * (size_t)m, tc_slice_ld(n));
  return cudaGetLastError();
}

int tc_encode_map(void* map64, const void* base, int n) {
  return make_map(reinterpret_cast<CUtensorMap*>(map64), base, n, tc_slice_ld(n), n);
}

cudaError_t launch_slice_q_grouped(const ProbDesc* P, int count, const int* rb_prefix, int total_rb,
                                   const int* tile_prefix, int total_tiles, cudaStream_t s) {
  rowmax_grouped_kernel<<<dim3(total_rb, 64), 256, 0, s>>>(P, count, rb_prefix);
  slice_q_grouped_kernel<<<total_tiles, dim3(32, 8), 0, s>>>(P, count, tile_prefix);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc_grouped(const ProbDesc* P, int count, const void* maps, const int* tile_prefix,
                                   int total_tiles, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemBytes);
  if (e != cudaSuccess) return e;
  gemm_tc_grouped_kernel<<<total_tiles, kThreads, kSmemBytes, s>>>(
      reinterpret_cast<const CUtensorMap*>(maps), P, tile_prefix, count);
  return cudaGetLastError();
}

cudaError_t launch_wnz_scan_grouped(const ProbDesc* P, int count, const int* tile_prefix, int total_tiles,
                                    cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  wnz_scan_grouped_kernel<<<total_tiles, 256, 0, s>>>(P, count, tile_prefix);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(int n, const __nv_bfloat16* Qs, const __nv_bfloat16* Ws, const int* erow,
                           const int* fcol, double* X, int ldx, const DevStatus* st, int* err,
                           cudaStream_t s, int ncols) {
  if (ncols < 0) ncols = n;
  if (ncols == 0) return cudaSuccess;
  CUtensorMap mq, mw;
  const int lds = tc_slice_ld(n);
  if (make_map(&mq, Qs, n, lds, n) != 0 || make_map(&mw, Ws, n, lds, ncols) != 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemBytes);
  if (e != cudaSuccess) return e;
  GemmArgs a;
  a.n = n;
  a.ncols = ncols;
  a.ldx = ldx;
  a.X = X;
  a.erow = erow;
  a.fcol = fcol;
  a.st = st;
  a.err = err;
  a.tiles_m = (n + BM - 1) / BM;
  a.tiles_n = (ncols + BN - 1) / BN;
  gemm_tc_kernel<<<a.tiles_m * a.tiles_n, kThreads, kSmemBytes, s>>>(mq, mw, a);
  return cudaGetLastError();
}

}  // namespace eig
