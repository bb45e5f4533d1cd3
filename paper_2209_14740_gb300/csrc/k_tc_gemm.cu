// Complex GEMM with a constant right factor on the 5th-generation tensor
// cores (tcgen05, TF32 inputs, FP32 accumulation in tensor memory), used by
// the transforms of the 2D preconditioner.
//
//   C = X Q,  X: M x K complex64 rows (the data), Q: K x N complex (constant)
//
// The complex product is the real product of X viewed as an M x 2K real
// matrix (re, im interleaved, as stored) with the real embedding
//   B[2k][2n] = Re Q[k][n],   B[2k][2n+1] = Im Q[k][n],
//   B[2k+1][2n] = -Im Q[k][n], B[2k+1][2n+1] = Re Q[k][n],
// so C viewed as M x 2N real comes out interleaved as well.
//
// FP32 accuracy from TF32 inputs (the 3xTF32 split): every operand is
// x = hi + lo with hi = tf32(x), lo = x - hi, and C = Xhi Bhi + Xhi Blo +
// Xlo Bhi; the dropped Xlo Blo term is below FP32 rounding.  B's split is
// precomputed on the host, X's is formed per tile in shared memory.
// Without the split (SPLIT = false) C = X Bhi in plain TF32 (X's low
// mantissa bits are ignored by the tensor core): one MMA per K step, X
// copied straight into the MMA layout, relative error ~1e-3.
//
// One CTA owns 128 rows and BN (64 or 128) real output columns; the
// accumulator (128 lanes x BN columns FP32) lives in tensor memory.  K is
// walked in stages of 32 real values.  Warp roles:
//   warps 0-7  copy raw X rows by cp.async (16-byte copies when the row
//              pitch allows) two or three stages ahead and split them into
//              hi/lo in the canonical K-major layout (8-row x 16-byte core
//              matrices, no swizzle), or, without the split, copy X straight
//              into that layout three stages ahead; then they run the
//              epilogue;
//   warp 8     one lane issues the MMAs of each stage (M=128, N=BN, K=8; 12
//              with the split, 4 without) and commits them to an mbarrier;
//   warp 9     one lane copies the pre-laid-out B tiles (hi and lo, or hi
//              only) of each stage with bulk asynchronous copies completing
//              on an mbarrier.
// Every wait is bounded: on a timeout the kernel records it, drains its
// copies, frees tensor memory and returns.
//
// In the plain-TF32 form the A operand (X) is kept in the 128-byte swizzle
// layout: each K stage of a row is one 128-byte row of the tile.  With a
// tensor map of X (X rows of even length), the copy warp also loads X: one 2D
// tensor copy of 32 values x 128 rows per stage, 128-byte requests, lands in
// that layout directly, and the loader warps only run the epilogue.  (A
// layout of 16-byte core matrices filled by 16-byte requests kept the
// L1-to-L2 request path ~80 % busy at a quarter of its bandwidth.)  The B
// operand and the 3xTF32 form's split X tiles use the no-swizzle
// core-matrix layout.
//
// Launched as a programmatic dependent of the previous kernel in the stream:
// tensor-memory allocation, barrier set-up and the first B copies (B is
// constant) overlap the previous kernel's tail; nothing it wrote is read,
// and nothing in global memory is written, before griddepcontrol.wait.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "sg_internal.h"

namespace sgi {
namespace tc {

constexpr int BM = 128;                 // rows per CTA = TMEM lanes
constexpr int BK = 32;                  // real K values per stage (128 bytes of FP32)
constexpr int NLOAD = 256;              // loader / splitter / epilogue threads (warps 0-7)
constexpr int MMA_WARP = NLOAD / 32;    // warp 8
constexpr int THREADS = NLOAD + 64;     // + the MMA warp and the B-copy warp
constexpr int NAS = 2;                  // split A (hi, lo) slots
constexpr int RAW_PITCH = 144;          // bytes per raw X row (128 + 16: conflict-free split reads)
constexpr int RAW_TILE = BM * RAW_PITCH;
constexpr int A_TILE = BM * BK * 4;     // 16 KB, core-matrix layout
constexpr int OFF_RAW = 0;

// Layout that depends on the tile width and on the split.
#ifndef SG_TC_PLAIN_STAGES
#define SG_TC_PLAIN_STAGES 4
#endif
template <int BN, bool SPLIT>
struct Cfg {
  // B slots: a slot is refilled once the MMAs of the stage that used it
  // have completed, so more slots let the copies run further ahead
  static constexpr int NBS = !SPLIT ? SG_TC_PLAIN_STAGES : BN == 64 ? 4 : 3;
  // raw X slots (split only): stages s .. s + NRAW - 1 in flight
  static constexpr int NRAW = !SPLIT ? 0 : BN == 64 ? 4 : 3;
  // A slots: split (hi, lo) pairs, or X tiles copied straight into the MMA
  // layout (stages s .. s + NA - 1 in flight)
  // (measured: eight slots make the first stage land later, so the last one
  // lands no sooner; the kernel is bound by the L2 -> SM traffic of the
  // re-read X and B tiles at small sizes)
  static constexpr int NA = SPLIT ? NAS : SG_TC_PLAIN_STAGES;
  // MMA-completion barriers, indexed by stage % NDONE: at least NBS, so no
  // wait on one of them can fall two phases behind
  static constexpr int NDONE = NBS > 4 ? NBS : 4;
  static constexpr int A_SLOT = SPLIT ? 2 * A_TILE : A_TILE;
  static constexpr int NBP = SPLIT ? 2 : 1;                      // B parts per slot (hi, lo)
  static constexpr int B_TILE = BN * BK * 4;                     // 8 or 16 KB
  static constexpr int OFF_B = OFF_RAW + NRAW * RAW_TILE;        // [slot][hi, lo]
  static constexpr int OFF_A = ((OFF_B + NBS * NBP * B_TILE + 1023) / 1024) * 1024;
  static constexpr int OFF_BAR = OFF_A + NA * A_SLOT;           // full[NA], bfull[NBS], done[NDONE], TMEM addr, abort, accf
  static constexpr int SMEM_BYTES = OFF_BAR + 256 + 1024;        // + slack for 1024-byte alignment
  static constexpr int OUT_PITCH = BN / 2 + 1;                   // float2 per staged output row
  static constexpr uint32_t TMEM_COLS = BN;
  // Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major,
  // N = BN, M = BM.
  static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(BM >> 4) << 24);
  static_assert(BN == 64 || BN == 128, "tile width");
  // the row-major output is staged over the data slots (free by then)
  static_assert(BM * OUT_PITCH * 8 <= OFF_BAR, "output staging must fit below the barriers");
  static_assert(8 * (NA + NBS + NDONE) + 24 <= 256, "barrier area");
  static_assert(NDONE >= NBS && NDONE >= 2, "completion barriers");
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory budget");
};

// Byte offset of element (row, k) of a tile with 32 K values per row in the
// no-swizzle K-major layout: core matrix (row / 8, k / 4) at 128-byte
// granularity, K-adjacent core matrices 128 bytes apart (leading byte
// offset), 8-row groups 1024 bytes apart (stride byte offset).
__host__ __device__ constexpr int core_off(int row, int k) {
  return ((row >> 3) * 8 + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared memory matrix descriptor: start address, leading byte offset 128,
// stride byte offset 1024, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46);
}

// Shared memory matrix descriptor of a K-major tile in the 128-byte swizzle
// layout: rows of 128 bytes (32 TF32 values, one K stage), 16-byte chunk c of
// row r stored at chunk c ^ (r % 8); 8-row groups 1024 bytes apart (stride
// byte offset); the leading byte offset is unused (one MMA's 8 K values, 32
// bytes, lie inside a row); swizzle mode 2 (128 B) in bits 61-63.  The tile
// starts on a 1024-byte boundary; the k-th MMA of a stage starts 32 k bytes
// into it (the swizzle is a function of the address bits, so the offset
// start selects the k-th 32-byte column of every row).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

// Byte offset of element (row, k), k < 32, in the 128-byte swizzle layout.
__host__ __device__ constexpr int sw128_off(int row, int k) {
  return row * 128 + ((((k >> 2) ^ (row & 7)) & 7) << 4) + (k & 3) * 4;
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase with the given parity of an mbarrier; false after
// about 0.5 s (the copies and MMAs of one stage take well under a
// microsecond).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = now_ns();
  for (uint32_t it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255u) == 255u && now_ns() - t0 > 500000000ull) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}

// Arrive once and announce `bytes` of asynchronous copies on the barrier.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
               "r"(bytes)
               : "memory");
}

// Bulk global -> shared copy (16-byte aligned addresses, size a multiple of
// 16) that completes its bytes on an mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// 2D tensor copy global -> shared completing its bytes on an mbarrier
__device__ __forceinline__ void tensor_g2s_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
// 16-byte copy; bytes < 16 fills the rest of the destination with zeros
__device__ __forceinline__ void cp_async16z(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace tc

// Output placement of C (complex, Nc columns):
//   mode 0: C[m * ldc + n]
//   mode 1: row m = p * MB + r goes to C[(p * Nc + n) * ldc + r] (the
//           per-batch transpose used to switch the transformed direction;
//           ldc >= MB is the pitch of the transposed rows)
// With E: C *= E[n * e_ld + m % e_mod]; then C *= (*escale if given) * oscale.
struct TcArgs {
  const float* X;      // M rows of 2K floats, row stride ldx floats
  long long ldx;
  int M, K2;           // rows, real K (2K)
  int nks;             // K stages (ceil(K2 / 32)); B is laid out for nks stages
  int vec16;           // X 16-byte aligned and ldx a multiple of 4 floats
  const float* Bhi;    // [n tile][stage][BN x 32 core-matrix tile]
  const float* Blo;
  int Nc;              // complex output columns
  int ntiles;          // column tiles; CTA b owns column tile b % ntiles of row tile b / ntiles
  float2* C;
  long long ldc;
  int mode, MB;
  const float2* E;
  int e_ld, e_mod;
  const double* escale;
  const int* skip;
  int* err;            // set to 1 on a wait timeout
  int out_half;        // C holds binary16 pairs (round to nearest even) instead of complex64
  float oscale;        // every output value is multiplied by oscale (and by *escale if given)
};

// Element idx of C (one complex value), as complex64 or as a binary16 pair.
__device__ __forceinline__ void put_c(const TcArgs& a, size_t idx, float2 c) {
  if (a.out_half) reinterpret_cast<__half2*>(a.C)[idx] = __floats2half2_rn(c.x, c.y);
  else a.C[idx] = c;
}

// Named barrier of the loader warps (the MMA and copy warps do not take part).
__device__ __forceinline__ void loader_sync() { asm volatile("bar.sync 1, %0;" ::"n"(tc::NLOAD) : "memory"); }

// Loader barrier that also ORs a flag over the loaders, so that every loader
// takes the same branch afterwards.
__device__ __forceinline__ bool loader_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(tc::NLOAD)
      : "memory");
  return r != 0;
}

// Pipeline (stage s = 32 real K values):
//   loaders (split):  wait raw X of s landed -> wait MMA(s-2) (frees A slot
//             s%2) -> split raw -> A slot, arrive full[s%2]
//             -> issue X copies of s+NRAW-1
//   loaders (no split): wait own X copies of s landed, arrive full[s%NA]
//             -> wait MMA(s-1) (frees slot (s-1)%NA) -> issue X copies of
//             s+NA-1 into it
//   B copier: wait MMA(s-NBS) (frees B slot s%NBS) -> bulk-copy B of s
//   MMA lane: wait full and bfull of s -> 12 (3xTF32) or 4 MMAs over the 4
//             K steps -> commit done[s%NDONE]; after the last stage one
//             more commit to the single-phase accumulator barrier, which
//             the loaders wait on before the epilogue
// so the loads of later stages overlap the MMAs of stage s.  No waiter can
// fall two phases behind on a barrier: where the loaders copy X, the MMA
// lane runs at most one or two stages ahead of them; the copier waits only
// for stages the MMA lane has issued, and NDONE >= NBS.  With X by tensor
// copies nothing holds the MMA lane back for the loaders, so they wait only
// on the accumulator barrier.
template <int BN, bool SPLIT, bool TMAX>
__global__ void __launch_bounds__(tc::THREADS, 1) k_tc_cgemm(TcArgs a, const __grid_constant__ CUtensorMap xmap) {
  using namespace tc;
  using L = Cfg<BN, SPLIT>;
  static_assert(!(SPLIT && TMAX), "X by tensor copy only in the plain-TF32 form");
  static_assert(!TMAX || L::NA == L::NBS, "X and B stages share their slot index");
  constexpr int NBS = L::NBS, B_TILE = L::B_TILE, NRAW = L::NRAW, OFF_B = L::OFF_B, NA = L::NA;
  constexpr int NDONE = L::NDONE;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t s_base = smem_u32(sm);
  const uint32_t full0 = s_base + L::OFF_BAR;    // NA barriers, count NLOAD
  const uint32_t bfull0 = full0 + 8 * NA;        // NBS barriers, count 1 + transaction bytes
  const uint32_t done0 = bfull0 + 8 * NBS;       // NDONE barriers, count 1 (MMA commit)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::OFF_BAR + 8 * (NA + NBS + NDONE));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + L::OFF_BAR + 8 * (NA + NBS + NDONE) + 8);
  // accumulator complete: one phase per launch (the MMA warp's final commit,
  // or a plain arrival if it issued no MMA), so a wait on it cannot alias
  const uint32_t accf = done0 + 8 * NDONE + 16;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(L::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < NA; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8 * i), "n"(TMAX ? 1 : NLOAD)
                   : "memory");
    for (int i = 0; i < NBS; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bfull0 + 8 * i) : "memory");
    for (int i = 0; i < NDONE; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done0 + 8 * i) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(accf) : "memory");
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  // the column tiles of one row tile are consecutive CTAs, so they run close
  // together and read that row tile of X from L2 rather than from HBM
  const int ctile = (int)(blockIdx.x % (unsigned)a.ntiles);
  const int m0 = (int)(blockIdx.x / (unsigned)a.ntiles) * BM;
  const float* Bh = a.Bhi + (size_t)ctile * a.nks * (BN * BK);
  const float* Bl = a.Blo + (size_t)ctile * a.nks * (BN * BK);
  auto copy_b = [&](int t) {
    const uint32_t bar = bfull0 + 8 * (t % NBS);
    const uint32_t dst = s_base + OFF_B + (t % NBS) * L::NBP * B_TILE;
    mbar_expect_tx(bar, (uint32_t)(L::NBP * B_TILE));
    bulk_g2s(dst, Bh + (size_t)t * (BN * BK), B_TILE, bar);
    if (SPLIT) bulk_g2s(dst + B_TILE, Bl + (size_t)t * (BN * BK), B_TILE, bar);
  };
  // X of stage t by one tensor copy into A slot t % NA (TMAX)
  auto copy_x = [&](int t) {
    const uint32_t bar = full0 + 8 * (t % NA);
    mbar_expect_tx(bar, (uint32_t)A_TILE);
    tensor_g2s_2d(s_base + L::OFF_A + (t % NA) * L::A_SLOT, &xmap, t * BK, m0, bar);
  };
  // B is constant: its first stages are copied before the wait below
  const int pre = a.nks < NBS ? a.nks : NBS;
  if (warp == MMA_WARP + 1 && lane == 0)
    for (int t = 0; t < pre; ++t) copy_b(t);
  // everything the previous kernel wrote is visible after this; then the
  // next kernel may start its own set-up
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const bool skipped = a.skip && *a.skip;
  const int nks = skipped ? 0 : a.nks;

  if (warp < MMA_WARP) {
    bool bad = false;
    // Epilogue geometry: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of
    // the tile) and real columns [w / 4 * BN / 2, + BN / 2).  Its factors E
    // (constant) are loaded now, so their latency overlaps the K loop.
    constexpr int HALF = BN / 2;       // real columns per warp
    const int lg = warp & 3, chalf = warp >> 2;
    const int row = lg * 32 + lane, m = m0 + row;
    const bool mok = m < a.M;
    const int nq0 = ctile * (BN / 2) + chalf * (HALF / 2);   // first complex column of this warp
    float2 ev[HALF / 2];
    if (a.E) {
      const int mr = (mok ? m : 0) % a.e_mod;
#pragma unroll
      for (int q = 0; q < HALF / 2; ++q)
        ev[q] = nq0 + q < a.Nc ? a.E[(size_t)(nq0 + q) * a.e_ld + mr] : make_float2(0.f, 0.f);
    }
    if constexpr (TMAX) {
      // X arrives by tensor copies: the loaders have nothing to do until the
      // accumulator is complete (below).  They must not follow the per-stage
      // completion barriers: nothing holds the MMA warp back for them, and a
      // parity wait on a barrier two or more phases ahead never ends.
    } else if constexpr (!SPLIT) {
      // ----------------------------------------- loaders (no split): X tiles
      // go straight into the MMA layout; each loader arrives on full[s % NA]
      // once its own copies of stage s have landed
      auto issue = [&](int t) {
        const uint32_t dst = s_base + L::OFF_A + (t % NA) * L::A_SLOT;
        const int k0 = t * BK;
        if (a.vec16) {
  #pragma unroll
          for (int q = 0; q < (BM * BK / 4) / NLOAD; ++q) {
            const int idx = tid + q * NLOAD;
            const int r = idx >> 3, c = idx & 7;
            const int m = m0 + r, k = k0 + 4 * c;
            const int rem = (a.K2 - k) * 4;
            const int bytes = (m < a.M && rem > 0) ? (rem < 16 ? rem : 16) : 0;
            const float* src = bytes ? a.X + (size_t)m * a.ldx + k : a.X;
            cp_async16z(dst + sw128_off(r, 4 * c), src, bytes);
          }
        } else {
  #pragma unroll
          for (int q = 0; q < (BM * BK / 2) / NLOAD; ++q) {
            const int idx = tid + q * NLOAD;
            const int r = idx >> 4, kp = idx & 15;
            const int m = m0 + r, k = k0 + 2 * kp;
            const bool ok = m < a.M && k < a.K2;
            const float* src = ok ? a.X + (size_t)m * a.ldx + k : a.X;
            cp_async8(dst + sw128_off(r, 2 * kp), src, ok ? 8 : 0);
          }
        }
      };
      for (int t = 0; t < NA - 1; ++t) {
        if (t < nks) issue(t);
        cp_commit();
      }
      for (int s = 0; s < nks; ++s) {
        cp_wait<NA - 2>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(full0 + 8 * (s % NA));
        // stage s+NA-1 goes to the slot of stage s-1 once its MMAs are done
        if (s + NA - 1 < nks) {
          if (s >= 1 && !mbar_wait(done0 + 8 * ((s - 1) % NDONE), ((s - 1) / NDONE) & 1)) {
            bad = true;
            break;
          }
          issue(s + NA - 1);
        }
        cp_commit();
      }
    } else {
      // ----------------------------------------- loaders (split)
      auto issue = [&](int t) {
        const uint32_t raw = s_base + OFF_RAW + (t % NRAW) * RAW_TILE;
        const int k0 = t * BK;
        if (a.vec16) {
  #pragma unroll
          for (int q = 0; q < (BM * BK / 4) / NLOAD; ++q) {
            const int idx = tid + q * NLOAD;
            const int r = idx >> 3, c = idx & 7;
            const int m = m0 + r, k = k0 + 4 * c;
            const int rem = (a.K2 - k) * 4;
            const int bytes = (m < a.M && rem > 0) ? (rem < 16 ? rem : 16) : 0;
            const float* src = bytes ? a.X + (size_t)m * a.ldx + k : a.X;
            cp_async16z(raw + r * RAW_PITCH + c * 16, src, bytes);
          }
        } else {
  #pragma unroll
          for (int q = 0; q < (BM * BK / 2) / NLOAD; ++q) {
            const int idx = tid + q * NLOAD;
            const int r = idx >> 4, kp = idx & 15;
            const int m = m0 + r, k = k0 + 2 * kp;
            const bool ok = m < a.M && k < a.K2;
            const float* src = ok ? a.X + (size_t)m * a.ldx + k : a.X;
            cp_async8(raw + r * RAW_PITCH + kp * 8, src, ok ? 8 : 0);
          }
        }
      };
      for (int t = 0; t < NRAW - 1; ++t) {
        if (t < nks) issue(t);
        cp_commit();
      }
      for (int s = 0; s < nks; ++s) {
        cp_wait<NRAW - 2>();
        bool to = false;
        if (s >= 2) to = !mbar_wait(done0 + 8 * ((s - 2) % NDONE), ((s - 2) / NDONE) & 1);
        if (loader_sync_or(to || *abort_flag != 0)) { bad = true; break; }
        // split X into hi / lo: two threads per row, four 16-byte chunks each
        {
          const int row = tid & (BM - 1), half = tid >> 7;
          const unsigned char* raw = sm + OFF_RAW + (s % NRAW) * RAW_TILE + row * RAW_PITCH;
          unsigned char* ahi = sm + L::OFF_A + (s % NAS) * 2 * A_TILE;
          unsigned char* alo = ahi + A_TILE;
  #pragma unroll
          for (int cc = 0; cc < BK / 8; ++cc) {
            const int c = half * (BK / 8) + cc;
            const float4 v = *reinterpret_cast<const float4*>(raw + 16 * c);
            float4 h, l;
            h.x = tf32_hi(v.x); l.x = v.x - h.x;
            h.y = tf32_hi(v.y); l.y = v.y - h.y;
            h.z = tf32_hi(v.z); l.z = v.z - h.z;
            h.w = tf32_hi(v.w); l.w = v.w - h.w;
            *reinterpret_cast<float4*>(ahi + core_off(row, 4 * c)) = h;
            *reinterpret_cast<float4*>(alo + core_off(row, 4 * c)) = l;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(full0 + 8 * (s % NAS));
        // the raw slot of stage s+NRAW-1 was split at s-1 by every loader
        // (all of them passed the barrier above since)
        if (s + NRAW - 1 < nks) issue(s + NRAW - 1);
        cp_commit();
      }
    }
    // all MMAs done before the accumulator is read
    if (!bad && !mbar_wait(accf, 0)) bad = true;
    cp_wait<0>();
    bad = loader_sync_or(bad || *abort_flag != 0);
    if (bad) {
      *abort_flag = 1;
    } else if (!skipped) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // Epilogue, 32 real columns at a time
      const float es = (a.escale ? (float)*a.escale : 1.0f) * a.oscale;
      float2* stage = reinterpret_cast<float2*>(sm + OFF_RAW);
      size_t cb = 0;          // mode 1: index in C of this row's element of column nq0
      bool pad1 = false;      // mode 1: also zero the pad entry after the last row r
      if (a.mode == 1 && mok) {
        const int p = m / a.MB, r = m - p * a.MB;
        cb = ((size_t)p * a.Nc + nq0) * a.ldc + r;
        pad1 = r == a.MB - 1 && a.ldc > a.MB;
      }
      const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(chalf * HALF);
#pragma unroll
      for (int j0 = 0; j0 < HALF; j0 += 32) {
        uint32_t v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
            "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
            "[%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr + (uint32_t)j0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int qq = j0 / 2 + q;        // complex column within this warp's half
          const int n = nq0 + qq;
          float2 c = make_float2(__uint_as_float(v[2 * q]), __uint_as_float(v[2 * q + 1]));
          if (a.E) {
            const float2 e = ev[qq];
            c = make_float2(es * (c.x * e.x - c.y * e.y), es * (c.x * e.y + c.y * e.x));
          } else {
            c = make_float2(es * c.x, es * c.y);
          }
          if (a.mode == 1) {
            // lanes hold consecutive rows r: each store writes consecutive addresses
            if (mok && n < a.Nc) {
              put_c(a, cb + (size_t)qq * a.ldc, c);
              // rows padded to even length are read whole by the next
              // transform's tensor copies: keep the pad at zero
              if (pad1) put_c(a, cb + (size_t)qq * a.ldc + 1, make_float2(0.f, 0.f));
            }
          } else {
            stage[row * L::OUT_PITCH + chalf * (HALF / 2) + qq] = c;
          }
        }
      }
      if (a.mode == 0) {
        // row-major: all loader warps write the staged rows, consecutive
        // lanes on consecutive columns
        loader_sync();
        const int n0 = ctile * (BN / 2);
        for (int idx = tid; idx < BM * (BN / 2); idx += NLOAD) {
          const int rr = idx / (BN / 2), q = idx % (BN / 2);
          const int mm = m0 + rr, n = n0 + q;
          if (mm < a.M && n < a.Nc) {
            put_c(a, (size_t)mm * a.ldc + n, stage[rr * L::OUT_PITCH + q]);
            if (n == a.Nc - 1 && a.ldc > a.Nc) put_c(a, (size_t)mm * a.ldc + a.Nc, make_float2(0.f, 0.f));
          }
        }
      }
    }
  } else if (warp == MMA_WARP) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      int last = -1;
      for (int s = 0; s < nks; ++s) {
        if (!mbar_wait(full0 + 8 * (s % NA), (s / NA) & 1)) { *abort_flag = 1; break; }
        if (!mbar_wait(bfull0 + 8 * (s % NBS), (s / NBS) & 1)) { *abort_flag = 1; break; }
        if (*abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ahi = s_base + L::OFF_A + (s % NA) * L::A_SLOT, alo = ahi + A_TILE;
        const uint32_t bhi = s_base + OFF_B + (s % NBS) * L::NBP * B_TILE, blo = bhi + B_TILE;
#pragma unroll
        for (int ks = 0; ks < BK / 8; ++ks) {
          const uint32_t o = 256u * ks;   // 8 TF32 = two core matrices along K (no-swizzle tiles)
          // A: the 128-byte swizzle layout in the plain form (8 TF32 = 32 bytes of each row)
          const uint64_t ad = SPLIT ? sdesc(ahi + o) : sdesc_sw128(ahi + 32u * ks);
          mma_tf32(tmem, ad, sdesc(bhi + o), L::IDESC, (s > 0 || ks > 0) ? 1u : 0u);
          if (SPLIT) {
            mma_tf32(tmem, sdesc(ahi + o), sdesc(blo + o), L::IDESC, 1u);
            mma_tf32(tmem, sdesc(alo + o), sdesc(bhi + o), L::IDESC, 1u);
          }
        }
        mma_commit(done0 + 8 * (s % NDONE));
        last = s;
      }
      // one arrival on the accumulator barrier when every MMA issued has
      // completed (also after an abort: the accumulator must not be freed
      // under running MMAs); a plain arrival if none was issued
      if (last >= 0) mma_commit(accf);
      else mbar_arrive(accf);
      if (!mbar_wait(accf, 0)) *abort_flag = 1;
    }
  } else if (lane == 0) {
    // ---------------------------------------------------------------- B copies
    int issued = pre;   // stages copied before the wait (also when skipped)
    int xissued = 0;    // X stages copied (TMAX), after the wait
    if (TMAX)
      for (; xissued < pre && xissued < nks; ++xissued) copy_x(xissued);
    for (int t = pre; t < nks; ++t) {
      if (!mbar_wait(done0 + 8 * ((t - NBS) % NDONE), ((t - NBS) / NDONE) & 1)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      copy_b(t);
      issued = t + 1;
      if (TMAX) {
        copy_x(t);
        xissued = t + 1;
      }
    }
    // no tensor copy may still be writing shared memory when the CTA exits
    if (TMAX)
      for (int t = xissued > NA ? xissued - NA : 0; t < xissued; ++t)
        if (!mbar_wait(full0 + 8 * (t % NA), (t / NA) & 1)) *abort_flag = 1;
    // no copy may still be writing shared memory when the CTA exits: wait
    // for the last copy into every slot
    for (int t = issued > NBS ? issued - NBS : 0; t < issued; ++t)
      if (!mbar_wait(bfull0 + 8 * (t % NBS), (t / NBS) & 1)) *abort_flag = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicExch(a.err, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::TMEM_COLS)
                 : "memory");
}

// ------------------------------------------------------------------ persistent plain-TF32 form
// The plain-TF32 transform with X by tensor copies, as a persistent kernel:
// one CTA per SM walks the tiles b, b + G, b + 2G, ... (column tiles of a
// row tile consecutive, as above) with two accumulators in tensor memory
// (2 BN columns), so that the epilogue of tile i (TMEM -> registers ->
// global) runs while the MMAs of tile i + 1 accumulate into the other
// buffer, and the copies of tile i + 1 start while tile i's last stages
// are still in the MMA pipe.  Barriers:
//   full[s % NS], bfull[s % NS]  X and B of stage s landed (transaction bytes)
//   done[s % NS]                 MMAs of stage s complete (slot free)
//   accf[i % 2]                  accumulator of tile i complete
//   acce[i % 2]                  accumulator of tile i read by all 8 epilogue warps
//   fin                          every MMA issued has completed (teardown)
// Stages are counted across tiles.  No waiter can fall two phases behind:
// the copier waits only for stages the MMA lane has issued; the MMA lane
// starts tile i + 2 in buffer i % 2 only after the epilogue released tile i,
// and the epilogue waits for tile i's accumulator before releasing it.
#ifndef SG_TC_PDL
#define SG_TC_PDL 1
#endif
#ifndef SG_TC_PERSIST
#define SG_TC_PERSIST 1
#endif
#ifndef SG_TC_PS_STAGES
#define SG_TC_PS_STAGES 4
#endif
template <int BN>
struct CfgP {
  static constexpr int NS = SG_TC_PS_STAGES;
  static constexpr int B_TILE = BN * tc::BK * 4;
  static constexpr int OUT_PITCH = BN / 2 + 1;
  static constexpr int STAGE_BYTES = ((tc::BM * OUT_PITCH * 8 + 1023) / 1024) * 1024;   // mode-0 output staging
  static constexpr int OFF_B = STAGE_BYTES;
  static constexpr int OFF_A = OFF_B + NS * B_TILE;
  static constexpr int OFF_BAR = OFF_A + NS * tc::A_TILE;
  static constexpr int NBAR = 3 * NS + 5;
  static constexpr int SMEM_BYTES = OFF_BAR + 8 * NBAR + 16 + 1024;   // + TMEM address, abort flag, alignment slack
  static constexpr uint32_t TMEM_COLS = 2 * BN;
  static_assert(OFF_B % 1024 == 0 && OFF_A % 1024 == 0 && OFF_BAR % 8 == 0, "alignment");
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory budget");
};

template <int BN, bool H>
__global__ void __launch_bounds__(tc::THREADS, 1) k_tc_cgemm_ps(TcArgs a, const __grid_constant__ CUtensorMap xmap) {
  using namespace tc;
  using L = CfgP<BN>;
  constexpr int NS = L::NS, B_TILE = L::B_TILE;
  // H: binary16 operands (kind::f16, K = 16 per MMA, 64 per 128-byte stage
  // row; the byte layout of the stages is that of the TF32 form)
  constexpr uint32_t IDESC = H ? ((1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24))
                               : Cfg<BN, false>::IDESC;
  constexpr int KE = H ? 2 * BK : BK;   // K values per stage
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t s_base = smem_u32(sm);
  const uint32_t full0 = s_base + L::OFF_BAR, bfull0 = full0 + 8 * NS, done0 = bfull0 + 8 * NS;
  const uint32_t accf0 = done0 + 8 * NS, acce0 = accf0 + 16, fin = acce0 + 16;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::OFF_BAR + 8 * L::NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + L::OFF_BAR + 8 * L::NBAR + 8);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(L::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 3 * NS + 2; ++i)   // full, bfull, done, accf: one arrival (+ bytes / commit)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * i) : "memory");
    for (int i = 0; i < 2; ++i)            // acce: one arrival per epilogue warp
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(acce0 + 8 * i), "n"(NLOAD / 32) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(fin) : "memory");
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const bool skipped = a.skip && *a.skip;
  const int nks = a.nks;
  const int total = skipped ? 0 : ((a.M + BM - 1) / BM) * a.ntiles;

  if (warp < MMA_WARP) {
    // ---------------------------------------------------------------- epilogue
    constexpr int HALF = BN / 2;   // real columns per warp
    const int lg = warp & 3, chalf = warp >> 2;
    const int row = lg * 32 + lane;
    float2* stage = reinterpret_cast<float2*>(sm);
    const float es = (a.escale ? (float)*a.escale : 1.0f) * a.oscale;
    int it = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++it) {
      const int b = it & 1;
      const int ctile = t % a.ntiles, m0 = (t / a.ntiles) * BM;
      const int m = m0 + row;
      const bool mok = m < a.M;
      const int nq0 = ctile * (BN / 2) + chalf * (HALF / 2);
      float2 ev[HALF / 2];
      if (a.E) {   // loaded before the wait: the latency overlaps the MMAs
        const int mr = (mok ? m : 0) % a.e_mod;
#pragma unroll
        for (int q = 0; q < HALF / 2; ++q)
          ev[q] = nq0 + q < a.Nc ? a.E[(size_t)(nq0 + q) * a.e_ld + mr] : make_float2(0.f, 0.f);
      }
      const bool to = !mbar_wait(accf0 + 8 * b, (uint32_t)(it >> 1) & 1u);
      if (loader_sync_or(to || *abort_flag != 0)) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      size_t cb = 0;
      bool pad1 = false;
      if (a.mode == 1 && mok) {
        const int p = m / a.MB, r = m - p * a.MB;
        cb = ((size_t)p * a.Nc + nq0) * a.ldc + r;
        pad1 = r == a.MB - 1 && a.ldc > a.MB;
      }
      const uint32_t taddr = tmem + (uint32_t)(b * BN) + ((uint32_t)(lg * 32) << 16) + (uint32_t)(chalf * HALF);
#pragma unroll
      for (int j0 = 0; j0 < HALF; j0 += 32) {
        uint32_t v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
            "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
            "[%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr + (uint32_t)j0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (j0 + 32 >= HALF) {
          // this warp's last read of the accumulator: release it to the MMA lane
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(acce0 + 8 * b);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int qq = j0 / 2 + q;
          const int n = nq0 + qq;
          float2 c = make_float2(__uint_as_float(v[2 * q]), __uint_as_float(v[2 * q + 1]));
          if (a.E) {
            const float2 e = ev[qq];
            c = make_float2(es * (c.x * e.x - c.y * e.y), es * (c.x * e.y + c.y * e.x));
          } else {
            c = make_float2(es * c.x, es * c.y);
          }
          if (a.mode == 1) {
            if (mok && n < a.Nc) {
              put_c(a, cb + (size_t)qq * a.ldc, c);
              if (pad1) put_c(a, cb + (size_t)qq * a.ldc + 1, make_float2(0.f, 0.f));
            }
          } else {
            stage[row * L::OUT_PITCH + chalf * (HALF / 2) + qq] = c;
          }
        }
      }
      if (a.mode == 0) {
        loader_sync();
        const int n0 = ctile * (BN / 2);
        for (int idx = tid; idx < BM * (BN / 2); idx += NLOAD) {
          const int rr = idx / (BN / 2), q = idx % (BN / 2);
          const int mm = m0 + rr, n = n0 + q;
          if (mm < a.M && n < a.Nc) {
            put_c(a, (size_t)mm * a.ldc + n, stage[rr * L::OUT_PITCH + q]);
            if (n == a.Nc - 1 && a.ldc > a.Nc) put_c(a, (size_t)mm * a.ldc + a.Nc, make_float2(0.f, 0.f));
          }
        }
      }
    }
  } else if (warp == MMA_WARP) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      bool any = false, stop = false;
      int g = 0, it = 0;
      for (int t = blockIdx.x; t < total && !stop; t += gridDim.x, ++it) {
        const int b = it & 1;
        if (it >= 2 && !mbar_wait(acce0 + 8 * b, (uint32_t)((it >> 1) - 1) & 1u)) {
          *abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(b * BN);
        for (int s = 0; s < nks; ++s, ++g) {
          const int slot = g % NS;
          const uint32_t par = (uint32_t)(g / NS) & 1u;
          if (!mbar_wait(full0 + 8 * slot, par) || !mbar_wait(bfull0 + 8 * slot, par) || *abort_flag) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t aa = s_base + L::OFF_A + slot * A_TILE, bb = s_base + L::OFF_B + slot * B_TILE;
#pragma unroll
          for (int ks = 0; ks < BK / 8; ++ks) {
            if constexpr (H)
              mma_f16(acc, sdesc_sw128(aa + 32u * ks), sdesc(bb + 256u * ks), IDESC, (s > 0 || ks > 0) ? 1u : 0u);
            else
              mma_tf32(acc, sdesc_sw128(aa + 32u * ks), sdesc(bb + 256u * ks), IDESC, (s > 0 || ks > 0) ? 1u : 0u);
          }
          mma_commit(done0 + 8 * slot);
          any = true;
        }
        if (!stop) mma_commit(accf0 + 8 * b);
      }
      // tensor memory is freed only after every MMA issued has completed
      if (any) mma_commit(fin);
      else mbar_arrive(fin);
      if (!mbar_wait(fin, 0)) *abort_flag = 1;
    }
  } else if (lane == 0) {
    // ---------------------------------------------------------------- X and B copies
    int g = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < total && !stop; t += gridDim.x) {
      const int ctile = t % a.ntiles, m0 = (t / a.ntiles) * BM;
      const float* Bh = a.Bhi + (size_t)ctile * nks * (BN * BK);
      for (int s = 0; s < nks; ++s, ++g) {
        if (g >= NS && !mbar_wait(done0 + 8 * ((g - NS) % NS), (uint32_t)((g - NS) / NS) & 1u)) {
          *abort_flag = 1;
          stop = true;
          break;
        }
        if (*abort_flag) {
          stop = true;
          break;
        }
        const int slot = g % NS;
        mbar_expect_tx(bfull0 + 8 * slot, (uint32_t)B_TILE);
        bulk_g2s(s_base + L::OFF_B + slot * B_TILE, Bh + (size_t)s * (BN * BK), B_TILE, bfull0 + 8 * slot);
        mbar_expect_tx(full0 + 8 * slot, (uint32_t)A_TILE);
        tensor_g2s_2d(s_base + L::OFF_A + slot * A_TILE, &xmap, s * KE, m0, full0 + 8 * slot);
      }
    }
    // no copy may still be writing shared memory when the CTA exits
    for (int q = g > NS ? g - NS : 0; q < g; ++q) {
      const uint32_t par = (uint32_t)(q / NS) & 1u;
      if (!mbar_wait(full0 + 8 * (q % NS), par) || !mbar_wait(bfull0 + 8 * (q % NS), par)) *abort_flag = 1;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicExch(a.err, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::TMEM_COLS)
                 : "memory");
}

// ------------------------------------------------------------------ paired 256-column binary16 form
// The binary16 transform of large GEMMs as a persistent kernel on clusters
// of two CTAs.  A CTA owns 128 rows and 256 real output columns (MMAs of
// M = 128, N = 256, K = 16); the two CTAs of a cluster take vertically
// adjacent row tiles of the same column tile, so they need the same B stage,
// and each copies one half of it (rows 0-127 or 128-255 of the 256 x 64
// tile, 16 KB) into the shared memory of both with one multicast bulk copy.
// Per CTA and stage, L2 then delivers 16 KB of X and 16 KB of B for a
// 128 x 256 x 64 product: half the bytes per MMA of the 128-column form,
// whose large transforms run at a fixed ~32 KB per stage and SM whatever the
// MMA cost of the stage (TF32 or binary16), i.e. bound by the L2 -> SM
// traffic of the re-read X and B tiles.
// Barriers, per CTA:
//   full[s % NS]  X (16 KB) and both B halves (2 x 16 KB) of stage s landed
//   done[s % NS]  the MMAs of stage s completed in both CTAs (count 2: each
//                 MMA lane commits to the barrier at this offset in both)
//   accf[i % 2], acce[i % 2], fin  as in the 128-column persistent form
// A producer refills slot s % NS for stage s only after done(s - NS), that is
// after both MMA lanes consumed stage s - NS: no copy lands in a slot still
// being read, and no barrier gets arrivals for a phase beyond the one its
// waiter is on (the peer's copies of stage s need this CTA's commit of
// stage s - NS, which follows this CTA's wait on full(s - NS)).  Both CTAs
// walk the same sequence of tile pairs, so they run the same stages.  A
// cluster barrier after the barrier set-up and another before exit keep
// either CTA from sending into the other's shared memory outside its
// lifetime; before the last one each producer waits for the copies into its
// own shared memory and for both commits of its last stages.  Mode-0 output
// is staged per warp, 32 rows x 8 complex values at a time, so that the
// global stores are row-contiguous.
#ifndef SG_TC_W_STAGES
#define SG_TC_W_STAGES 4
#endif
namespace tcw {
constexpr int BN = 256;
constexpr int NS = SG_TC_W_STAGES;
constexpr int A_TILE = tc::A_TILE;               // 128 rows x 128 bytes
constexpr int B_TILE = BN * 128;                 // 256 rows x 64 binary16 values
constexpr int B_HALF = B_TILE / 2;
constexpr int OFF_A = 0;
constexpr int OFF_B = NS * A_TILE;
constexpr int STG_PITCH = 9;                     // float2 per staged row (8 + 1)
constexpr int STG_WARP = 32 * STG_PITCH * 8;
constexpr int OFF_STG = OFF_B + NS * B_TILE;
constexpr int OFF_BAR = OFF_STG + (tc::NLOAD / 32) * STG_WARP;
constexpr int NBAR = 2 * NS + 5;                 // full, done, accf[2], acce[2], fin
constexpr int SMEM_BYTES = OFF_BAR + 8 * NBAR + 16 + 1024;   // + TMEM address, abort flag, alignment slack
constexpr uint32_t TMEM_COLS = 2 * BN;
// kind::f16: D = F32, A = B = F16, both K-major, N = 256, M = 128
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(tc::BM >> 4) << 24);
static_assert(OFF_B % 1024 == 0 && OFF_STG % 1024 == 0 && OFF_BAR % 8 == 0, "alignment");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory budget");

// Bulk copy global -> shared into the same offset of every CTA in mask, each
// completing its bytes on its own mbarrier at offset bar.
__device__ __forceinline__ void bulk_g2s_mc(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar,
                                            uint16_t mask) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1], %2, [%3], "
      "%4;" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar), "h"(mask)
      : "memory");
}
// Commit of this CTA's MMAs to the mbarrier at offset bar of every CTA in mask.
__device__ __forceinline__ void mma_commit_mc(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          bar),
      "h"(mask)
      : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
}  // namespace tcw

__global__ void __launch_bounds__(tc::THREADS, 1) k_tc_hgemm_w(TcArgs a, const __grid_constant__ CUtensorMap xmap) {
  using namespace tc;
  constexpr int NS = tcw::NS, BN = tcw::BN;
  constexpr uint16_t PAIR = 3;   // both CTAs of the cluster
  extern __shared__ unsigned char smem_dyn[];
  // (the same offsets in both CTAs: they run the same layout from the same base)
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t s_base = smem_u32(sm);
  const uint32_t full0 = s_base + tcw::OFF_BAR, done0 = full0 + 8 * NS;
  const uint32_t accf0 = done0 + 8 * NS, acce0 = accf0 + 16, fin = acce0 + 16;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + tcw::OFF_BAR + 8 * tcw::NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + tcw::OFF_BAR + 8 * tcw::NBAR + 8);
  const int q = (int)tcw::cluster_rank();
  uint32_t cid, ncl;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(ncl));

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tcw::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * i) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(done0 + 8 * i) : "memory");
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(accf0 + 8 * i) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(acce0 + 8 * i), "n"(NLOAD / 32) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(fin) : "memory");
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  tcw::cluster_sync_all();   // the peer's barriers exist before anything is sent to them
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const bool skipped = a.skip && *a.skip;
  const int nks = a.nks;
  const int rtiles = (a.M + BM - 1) / BM;
  const int total = skipped ? 0 : ((rtiles + 1) / 2) * a.ntiles;   // tile pairs

  if (warp < MMA_WARP) {
    // ---------------------------------------------------------------- epilogue
    constexpr int HALF = BN / 2;   // real columns per warp
    const int lg = warp & 3, chalf = warp >> 2;
    const int row = lg * 32 + lane;
    float2* stg = reinterpret_cast<float2*>(sm + tcw::OFF_STG + warp * tcw::STG_WARP);
    const float es = (a.escale ? (float)*a.escale : 1.0f) * a.oscale;
    int it = 0;
    for (int u = (int)cid; u < total; u += (int)ncl, ++it) {
      const int b = it & 1;
      const int ctile = u % a.ntiles, m0 = ((u / a.ntiles) * 2 + q) * BM;
      const int m = m0 + row;
      const bool mok = m < a.M;
      const int nq0 = ctile * (BN / 2) + chalf * (HALF / 2);   // first complex column of this warp
      const int mr = (mok ? m : 0) % a.e_mod;
      // E of 16 complex columns from column n0 (zeros past Nc)
      auto load_e = [&](float2 (&e)[16], int n0) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
          e[k] = n0 + k < a.Nc ? a.E[(size_t)(n0 + k) * a.e_ld + mr] : make_float2(0.f, 0.f);
      };
      float2 ecur[16];
      if (a.E) load_e(ecur, nq0);   // before the wait: the latency overlaps the MMAs
      const bool to = !mbar_wait(accf0 + 8 * b, (uint32_t)(it >> 1) & 1u);
      if (loader_sync_or(to || *abort_flag != 0)) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      size_t cb = 0;
      bool pad1 = false;
      if (a.mode == 1 && mok) {
        const int p = m / a.MB, r = m - p * a.MB;
        cb = ((size_t)p * a.Nc + nq0) * a.ldc + r;
        pad1 = r == a.MB - 1 && a.ldc > a.MB;
      }
      const uint32_t taddr = tmem + (uint32_t)(b * BN) + ((uint32_t)(lg * 32) << 16) + (uint32_t)(chalf * HALF);
#pragma unroll 1
      for (int j0 = 0; j0 < HALF; j0 += 32) {
        if (a.E && j0 > 0) load_e(ecur, nq0 + j0 / 2);   // (lands during the accumulator read)
        uint32_t v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
            "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
            "[%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr + (uint32_t)j0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (j0 + 32 >= HALF) {
          // this warp's last read of the accumulator: release it to the MMA lane
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(acce0 + 8 * b);
        }
        // complex value k of this chunk, scaled (and times E)
        auto val = [&](int k) {
          const float2 x = make_float2(__uint_as_float(v[2 * k]), __uint_as_float(v[2 * k + 1]));
          if (a.E) {
            const float2 e = ecur[k];
            return make_float2(es * (x.x * e.x - x.y * e.y), es * (x.x * e.y + x.y * e.x));
          }
          return make_float2(es * x.x, es * x.y);
        };
        const int nc0 = nq0 + j0 / 2;   // first complex column of this chunk
        if (a.mode == 1) {
          if (mok) {
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (nc0 + k < a.Nc) {
                put_c(a, cb + (size_t)(j0 / 2 + k) * a.ldc, val(k));
                if (pad1) put_c(a, cb + (size_t)(j0 / 2 + k) * a.ldc + 1, make_float2(0.f, 0.f));
              }
          }
        } else {
          // 32 rows x 8 values through the warp's staging area, then row-contiguous stores
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
#pragma unroll
            for (int k = 0; k < 8; ++k) stg[lane * tcw::STG_PITCH + k] = val(8 * h2 + k);
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int rr = 4 * i + (lane >> 3), cc = lane & 7;
              const int mm = m0 + lg * 32 + rr, n = nc0 + 8 * h2 + cc;
              if (mm < a.M && n < a.Nc) {
                put_c(a, (size_t)mm * a.ldc + n, stg[rr * tcw::STG_PITCH + cc]);
                if (n == a.Nc - 1 && a.ldc > a.Nc) put_c(a, (size_t)mm * a.ldc + a.Nc, make_float2(0.f, 0.f));
              }
            }
            __syncwarp();
          }
        }
      }
    }
  } else if (warp == MMA_WARP) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      bool any = false, stop = false;
      int g = 0, it = 0;
      for (int u = (int)cid; u < total && !stop; u += (int)ncl, ++it) {
        const int b = it & 1;
        if (it >= 2 && !mbar_wait(acce0 + 8 * b, (uint32_t)((it >> 1) - 1) & 1u)) {
          *abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(b * BN);
        for (int s = 0; s < nks; ++s, ++g) {
          const int slot = g % NS;
          const uint32_t par = (uint32_t)(g / NS) & 1u;
          if (!mbar_wait(full0 + 8 * slot, par) || *abort_flag) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t aa = s_base + tcw::OFF_A + slot * tcw::A_TILE;
          const uint32_t bb = s_base + tcw::OFF_B + slot * tcw::B_TILE;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            mma_f16(acc, sdesc_sw128(aa + 32u * ks), sdesc(bb + 256u * ks), tcw::IDESC, (s > 0 || ks > 0) ? 1u : 0u);
          tcw::mma_commit_mc(done0 + 8 * slot, PAIR);   // the slot is free in both CTAs once both commit
          any = true;
        }
        if (!stop) mma_commit(accf0 + 8 * b);
      }
      // tensor memory is freed only after every MMA issued has completed
      if (any) mma_commit(fin);
      else mbar_arrive(fin);
      if (!mbar_wait(fin, 0)) *abort_flag = 1;
    }
  } else if (lane == 0) {
    // ---------------------------------------------------------------- X and B copies
    int g = 0;
    bool stop = false;
    const unsigned char* Bt = reinterpret_cast<const unsigned char*>(a.Bhi);
    for (int u = (int)cid; u < total && !stop; u += (int)ncl) {
      const int ctile = u % a.ntiles, m0 = ((u / a.ntiles) * 2 + q) * BM;
      for (int s = 0; s < nks; ++s, ++g) {
        if (g >= NS && !mbar_wait(done0 + 8 * ((g - NS) % NS), (uint32_t)((g - NS) / NS) & 1u)) {
          *abort_flag = 1;
          stop = true;
          break;
        }
        if (*abort_flag) {
          stop = true;
          break;
        }
        const int slot = g % NS;
        const uint32_t fb = full0 + 8 * slot;
        // this CTA's X (16 KB) and both B halves (its own and the peer's, 16 KB each)
        mbar_expect_tx(fb, (uint32_t)(tcw::A_TILE + tcw::B_TILE));
        tensor_g2s_2d(s_base + tcw::OFF_A + slot * tcw::A_TILE, &xmap, s * 2 * BK, m0, fb);
        tcw::bulk_g2s_mc(s_base + tcw::OFF_B + slot * tcw::B_TILE + q * tcw::B_HALF,
                         Bt + ((size_t)ctile * nks + s) * tcw::B_TILE + (size_t)q * tcw::B_HALF,
                         (uint32_t)tcw::B_HALF, fb, PAIR);
      }
    }
    // before the exit barrier: every copy into this CTA's shared memory has
    // landed, and both MMA lanes' commits of the last stages have arrived here
    const int t0 = g > NS ? g - NS : 0;
    for (int t = t0; t < g; ++t)
      if (!mbar_wait(full0 + 8 * (t % NS), (uint32_t)(t / NS) & 1u)) *abort_flag = 1;
    if (!*abort_flag)
      for (int t = t0; t < g; ++t)
        if (!mbar_wait(done0 + 8 * (t % NS), (uint32_t)(t / NS) & 1u)) *abort_flag = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  tcw::cluster_sync_all();
  if (tid == 0 && *abort_flag) atomicExch(a.err, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcw::TMEM_COLS)
                 : "memory");
}

// Check of the bounded wait: one warp waits for phase 0 of a barrier that
// nothing arrives on (count 1, no arrival, no copy), through the same
// mbar_wait as the transform kernel.  The wait must give up after its limit
// and the kernel must then report it in the device flag, as the transform
// does, and return; *done = 1 records that the kernel ran to its end.
__global__ void __launch_bounds__(32) k_wait_selftest(int* err, int* done) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(1) : "memory");
  __syncwarp();
  const bool ok = tc::mbar_wait(b, 0);
  __syncwarp();
  if (threadIdx.x == 0) {
    if (!ok) atomicExch(err, 1);
    atomicExch(done, 1);
  }
}

// ------------------------------------------------------------------ host side
// B layout for C = X Q with Q (kdim x ndim complex, row-major, FP64 on the
// host) and tile width bn: nt = ceil(2 ndim / bn) column tiles, nks =
// ceil(2 kdim / 32) K stages, each (tile, stage) a bn x 32 block in
// core-matrix order.
static float tf32_round_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return x;   // inf / nan unchanged
  u = (u + 0x1000u) & 0xFFFFE000u;                   // nearest, ties away from zero
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

TcOperand tc_make_operand(const std::vector<std::complex<double>>& Q, int kdim, int ndim, int bn) {
  using namespace tc;
  TcOperand op;
  op.kdim = kdim;
  op.ndim = ndim;
  op.bn = bn;
  op.nks = (2 * kdim + BK - 1) / BK;
  op.ntiles = (2 * ndim + bn - 1) / bn;
  const size_t per = (size_t)bn * BK;
  op.hi.assign(per * op.nks * op.ntiles, 0.0f);
  op.lo.assign(per * op.nks * op.ntiles, 0.0f);
  for (int nt = 0; nt < op.ntiles; ++nt)
    for (int ks = 0; ks < op.nks; ++ks) {
      const size_t blk = ((size_t)nt * op.nks + ks) * per;
      for (int row = 0; row < bn; ++row)
        for (int k = 0; k < BK; ++k) {
          const int nr = nt * bn + row, kr = ks * BK + k;   // real column of C, real K index
          double v = 0.0;
          if (nr < 2 * ndim && kr < 2 * kdim) {
            const std::complex<double> q = Q[(size_t)(kr >> 1) * ndim + (nr >> 1)];
            const int a = kr & 1, b = nr & 1;                // B[2k+a][2n+b]
            v = (a == 0) ? (b == 0 ? q.real() : q.imag()) : (b == 0 ? -q.imag() : q.real());
          }
          const float f = (float)v;
          const float hi = tf32_round_host(f);
          const float lo = tf32_round_host(f - hi);
          op.hi[blk + core_off(row, k) / 4] = hi;
          op.lo[blk + core_off(row, k) / 4] = lo;
        }
    }
  tc_fill_h16(op, Q, bn);
  return op;
}

// Binary16 tiles of the same factor (round to nearest even) for tile width
// bn (64, 128 or 256): K stages of 64 values, 128-byte rows, core matrices of
// 8 rows x 8 values.
void tc_fill_h16(TcOperand& op, const std::vector<std::complex<double>>& Q, int bn) {
  using namespace tc;
  const int kdim = op.kdim, ndim = op.ndim;
  op.nks16 = (2 * kdim + 2 * BK - 1) / (2 * BK);
  const int ntiles = (2 * ndim + bn - 1) / bn;
  const size_t per16 = (size_t)bn * 2 * BK;
  op.h16.assign(per16 * op.nks16 * ntiles, 0);
  for (int nt = 0; nt < ntiles; ++nt)
    for (int ks = 0; ks < op.nks16; ++ks) {
      const size_t blk = ((size_t)nt * op.nks16 + ks) * per16;
      for (int row = 0; row < bn; ++row)
        for (int k = 0; k < 2 * BK; ++k) {
          const int nr = nt * bn + row, kr = ks * 2 * BK + k;
          double v = 0.0;
          if (nr < 2 * ndim && kr < 2 * kdim) {
            const std::complex<double> q = Q[(size_t)(kr >> 1) * ndim + (nr >> 1)];
            const int a = kr & 1, b = nr & 1;
            v = (a == 0) ? (b == 0 ? q.real() : q.imag()) : (b == 0 ? -q.imag() : q.real());
          }
          const __half hv = __float2half_rn((float)v);
          uint16_t bits;
          std::memcpy(&bits, &hv, 2);
          const int off = ((row >> 3) * 8 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;   // bytes
          op.h16[blk + off / 2] = bits;
        }
    }
}

TcOperand tc_make_operand16(const std::vector<std::complex<double>>& Q, int kdim, int ndim, int bn) {
  TcOperand op;
  op.kdim = kdim;
  op.ndim = ndim;
  op.bn = bn;
  op.nks = (2 * kdim + tc::BK - 1) / tc::BK;
  op.ntiles = (2 * ndim + bn - 1) / bn;
  tc_fill_h16(op, Q, bn);
  return op;
}

bool tc_make_xmap16(CUtensorMap* map, const void* X, long long ldx, int M, int kdim) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  // rows of ldx binary16 pairs: the pitch (4 ldx bytes) must be a multiple of 16
  if (!enc || ldx % 4 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0 || M <= 0 || kdim <= 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)(2 * kdim), (cuuint64_t)M};
  cuuint64_t strides[1] = {(cuuint64_t)ldx * 4};
  cuuint32_t box[2] = {(cuuint32_t)(2 * tc::BK), (cuuint32_t)tc::BM};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(X), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int tc_tile_width(long long rows, int ndim, int num_sms) {
  // 128 columns halve the re-reads of X but give half as many CTAs: use
  // them only while every SM still gets two tiles of the narrow form
  const long long tiles64 = ((rows + tc::BM - 1) / tc::BM) * ((2LL * ndim + 63) / 64);
  return tiles64 >= 2LL * num_sms ? 128 : 64;
}

bool tc_make_xmap(CUtensorMap* map, const float2* X, long long ldx, int M, int kdim) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!enc || ldx % 2 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0 || M <= 0 || kdim <= 0) return false;
  // view: (2 kdim real values, M rows), row pitch a multiple of 16 bytes; a
  // box of 32 values x 128 rows (one K stage of one row tile, 128-byte rows)
  // lands in the 128-byte swizzle layout the MMA descriptor expects; values
  // past 2 kdim and rows past M are read as zeros
  cuuint64_t dims[2] = {(cuuint64_t)(2 * kdim), (cuuint64_t)M};
  cuuint64_t strides[1] = {(cuuint64_t)ldx * 8};
  cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)tc::BM};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(X), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static void tc_attributes() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_tc_cgemm<64, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         tc::Cfg<64, true>::SMEM_BYTES);
    cudaFuncSetAttribute(k_tc_cgemm<128, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         tc::Cfg<128, true>::SMEM_BYTES);
    cudaFuncSetAttribute(k_tc_cgemm<64, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         tc::Cfg<64, false>::SMEM_BYTES);
    cudaFuncSetAttribute(k_tc_cgemm<128, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         tc::Cfg<128, false>::SMEM_BYTES);
    cudaFuncSetAttribute(k_tc_cgemm<64, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         tc::Cfg<64, false>::SMEM_BYTES);
    cudaFuncSetAttribute(k_tc_cgemm<128, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         tc::Cfg<128, false>::SMEM_BYTES);
    cudaFuncSetAttribute(k_tc_cgemm_ps<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, CfgP<64>::SMEM_BYTES);
    cudaFuncSetAttribute(k_tc_cgemm_ps<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, CfgP<128>::SMEM_BYTES);
    cudaFuncSetAttribute(k_tc_cgemm_ps<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, CfgP<64>::SMEM_BYTES);
    cudaFuncSetAttribute(k_tc_cgemm_ps<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, CfgP<128>::SMEM_BYTES);
    cudaFuncSetAttribute(k_tc_hgemm_w, cudaFuncAttributeMaxDynamicSharedMemorySize, tcw::SMEM_BYTES);
  });
}

cudaError_t tc_cgemm(const TcDevOperand& B, const float2* X, long long ldx, int M, float2* C, long long ldc,
                     int mode, int MB, const float2* E, int e_ld, int e_mod, const double* escale, const int* skip,
                     int* err, cudaStream_t st, bool split, const CUtensorMap* xmap, bool out_half, float oscale) {
  if (B.bn != 64 && B.bn != 128) return cudaErrorInvalidValue;
  if (mode == 1 && (MB <= 0 || ldc < MB)) return cudaErrorInvalidValue;
  tc_attributes();
  TcArgs a;
  a.X = reinterpret_cast<const float*>(X);
  a.ldx = 2 * ldx;
  a.M = M;
  a.K2 = 2 * B.kdim;
  a.nks = B.nks;
  a.vec16 = (ldx % 2 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) ? 1 : 0;
  a.Bhi = B.hi;
  a.Blo = B.lo;
  a.Nc = B.ndim;
  a.ntiles = B.ntiles;
  a.C = C;
  a.ldc = ldc;
  a.mode = mode;
  a.MB = MB;
  a.E = E;
  a.e_ld = e_ld;
  a.e_mod = e_mod > 0 ? e_mod : 1;
  a.escale = escale;
  a.skip = skip;
  a.err = err;
  a.out_half = out_half ? 1 : 0;
  a.oscale = oscale;
  // programmatic dependent launch: may start while the previous kernel in
  // the stream finishes (the kernel waits for it before touching its data)
  cudaLaunchConfig_t cfg = {};
  const long long ctas = (long long)((M + tc::BM - 1) / tc::BM) * B.ntiles;
  if (ctas <= 0 || ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(tc::THREADS);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = SG_TC_PDL;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CUtensorMap none;
  std::memset(&none, 0, sizeof(none));
  // X by tensor copies when the transform has at least one tile per SM
  // (measured: 255^2 and 319^2 applies 3-5 % faster; at 127^2, 80 tiles, the
  // loader warps' own copies are faster)
  static const int num_sms = [] {   // thread-safe once (batched solves call from many threads)
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      v = 0;
    return v;
  }();
  const bool tmax = !split && xmap != nullptr && num_sms > 0 &&
                    (long long)cfg.gridDim.x >= num_sms;
  const CUtensorMap& m = tmax ? *xmap : none;
  cudaError_t e;
  if (tmax && SG_TC_PERSIST) {
    // persistent: one CTA per SM walks the tiles
    cfg.gridDim = dim3((unsigned)std::min<long long>(ctas, num_sms));
    cfg.dynamicSmemBytes = B.bn == 128 ? CfgP<128>::SMEM_BYTES : CfgP<64>::SMEM_BYTES;
    e = B.bn == 128 ? cudaLaunchKernelEx(&cfg, k_tc_cgemm_ps<128, false>, a, m)
                    : cudaLaunchKernelEx(&cfg, k_tc_cgemm_ps<64, false>, a, m);
  } else if (B.bn == 128 && split) {
    cfg.dynamicSmemBytes = tc::Cfg<128, true>::SMEM_BYTES;
    e = cudaLaunchKernelEx(&cfg, k_tc_cgemm<128, true, false>, a, m);
  } else if (split) {
    cfg.dynamicSmemBytes = tc::Cfg<64, true>::SMEM_BYTES;
    e = cudaLaunchKernelEx(&cfg, k_tc_cgemm<64, true, false>, a, m);
  } else if (B.bn == 128) {
    cfg.dynamicSmemBytes = tc::Cfg<128, false>::SMEM_BYTES;
    e = tmax ? cudaLaunchKernelEx(&cfg, k_tc_cgemm<128, false, true>, a, m)
             : cudaLaunchKernelEx(&cfg, k_tc_cgemm<128, false, false>, a, m);
  } else {
    cfg.dynamicSmemBytes = tc::Cfg<64, false>::SMEM_BYTES;
    e = tmax ? cudaLaunchKernelEx(&cfg, k_tc_cgemm<64, false, true>, a, m)
             : cudaLaunchKernelEx(&cfg, k_tc_cgemm<64, false, false>, a, m);
  }
  note_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t tc_hgemm(const TcDevOperand& B, const void* X, int M, void* C, long long ldc, int mode, int MB,
                     const float2* E, int e_ld, int e_mod, const double* escale, float oscale, bool out_half,
                     const int* skip, int* err, cudaStream_t st, const CUtensorMap* xmap) {
  if ((B.bn != 64 && B.bn != 128) || !B.h16 || !xmap) return cudaErrorInvalidValue;
  if (mode == 1 && (MB <= 0 || ldc < MB)) return cudaErrorInvalidValue;
  tc_attributes();
  TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.X = reinterpret_cast<const float*>(X);
  a.M = M;
  a.K2 = 2 * B.kdim;
  a.nks = B.nks16;
  a.Bhi = reinterpret_cast<const float*>(B.h16);
  a.Nc = B.ndim;
  a.ntiles = B.ntiles;
  a.C = reinterpret_cast<float2*>(C);
  a.ldc = ldc;
  a.mode = mode;
  a.MB = MB;
  a.E = E;
  a.e_ld = e_ld;
  a.e_mod = e_mod > 0 ? e_mod : 1;
  a.escale = escale;
  a.skip = skip;
  a.err = err;
  a.out_half = out_half ? 1 : 0;
  a.oscale = oscale;
  static const int num_sms = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      v = 0;
    return v;
  }();
  const long long ctas = (long long)((M + tc::BM - 1) / tc::BM) * B.ntiles;
  if (ctas <= 0 || ctas > 0x7fffffffLL || num_sms <= 0) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)std::min<long long>(ctas, num_sms));
  cfg.blockDim = dim3(tc::THREADS);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = SG_TC_PDL;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.dynamicSmemBytes = B.bn == 128 ? CfgP<128>::SMEM_BYTES : CfgP<64>::SMEM_BYTES;
  const cudaError_t e = B.bn == 128 ? cudaLaunchKernelEx(&cfg, k_tc_cgemm_ps<128, true>, a, *xmap)
                                    : cudaLaunchKernelEx(&cfg, k_tc_cgemm_ps<64, true>, a, *xmap);
  note_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Clusters of two 320-thread CTAs with the paired kernel's shared memory
// that the GPU holds at once (0 if the query fails).
static int tc_wide_clusters() {
  static const int n = [] {
    tc_attributes();
    cudaLaunchConfig_t qc = {};
    qc.gridDim = dim3(2);
    qc.blockDim = dim3(tc::THREADS);
    qc.dynamicSmemBytes = tcw::SMEM_BYTES;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    qc.attrs = at;
    qc.numAttrs = 1;
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, k_tc_hgemm_w, &qc) != cudaSuccess) {
      cudaGetLastError();
      c = 0;
    }
    return c;
  }();
  return n;
}

bool tc_wide_available() { return tc_wide_clusters() > 0; }

cudaError_t tc_hgemm_w(const TcDevOperand& B, const void* X, int M, void* C, long long ldc, int mode, int MB,
                       const float2* E, int e_ld, int e_mod, const double* escale, float oscale, bool out_half,
                       const int* skip, int* err, cudaStream_t st, const CUtensorMap* xmap) {
  if (B.bn != tcw::BN || !B.h16 || !xmap) return cudaErrorInvalidValue;
  if (mode == 1 && (MB <= 0 || ldc < MB)) return cudaErrorInvalidValue;
  const int ncl = tc_wide_clusters();
  if (ncl <= 0) return cudaErrorNotSupported;
  TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.X = reinterpret_cast<const float*>(X);
  a.M = M;
  a.K2 = 2 * B.kdim;
  a.nks = B.nks16;
  a.Bhi = reinterpret_cast<const float*>(B.h16);
  a.Nc = B.ndim;
  a.ntiles = B.ntiles;
  a.C = reinterpret_cast<float2*>(C);
  a.ldc = ldc;
  a.mode = mode;
  a.MB = MB;
  a.E = E;
  a.e_ld = e_ld;
  a.e_mod = e_mod > 0 ? e_mod : 1;
  a.escale = escale;
  a.skip = skip;
  a.err = err;
  a.out_half = out_half ? 1 : 0;
  a.oscale = oscale;
  const long long pairs = (((long long)(M + tc::BM - 1) / tc::BM + 1) / 2) * B.ntiles;
  if (pairs <= 0 || pairs > 0x3fffffffLL) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * std::min<long long>(pairs, ncl)));
  cfg.blockDim = dim3(tc::THREADS);
  cfg.dynamicSmemBytes = tcw::SMEM_BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = SG_TC_PDL;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_tc_hgemm_w, a, *xmap);
  note_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t tc_wait_selftest(int* err, int* done, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(err, done);
  note_launch();
  return cudaGetLastError();
}


}  // namespace sgi
