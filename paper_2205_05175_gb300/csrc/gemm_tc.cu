// tcgen05 tensor-core GEMM for the residual contractions (sm_103a).
//
// Output plane rb of C (0 = real part, 1 = imaginary part) gets
//     C[b][m][n] += alpha * sum_s (-1)^neg_s * sum_k A[planeA_s][b][m][k] * B[planeB_s][b][n][k]
// with A and B packed K-major as planes (re/im x hi/lo split parts, 128-byte K blocks) and C a
// strided float64 tensor addressed through index maps (no intermediate output buffer).
//
// Persistent, warp-specialised: one CTA per SM walks work items (batch, output plane or both
// planes, split-K slice, 128 x BN tile in grouped order):
//   warp 0 lane 0 : TMA producer (cp.async.bulk.tensor, 128-byte swizzle, mbarrier tx count;
//                   one K block per stage, or two through 4-D tensor maps)
//   warp 1 lane 0 : MMA issuer (tcgen05.mma kind::tf32, or kind::f16 with bf16 inputs; the
//                   instruction descriptor's negate-A bit gives -Ai Bi), tcgen05.commit
//                   releases smem stages and hands a finished accumulator to the epilogue
//   warps 2..     : epilogue (tcgen05.ld 32x32b over the warp's TMEM lane quarter, batched
//                   read-modify-write of C, shared-memory transpose when C is unit-stride in n);
//                   four warps, or eight that split the tile's columns
// In the split precision modes the MMAs accumulate bounded chunks of the K loop in TMEM slots and
// the epilogue folds them into the tile's sum with round-to-nearest float32 adds (see chunk_of).
// Two TMEM accumulator sets overlap the epilogue of one tile with the main loop of the next.
// When the K loop is short the epilogue dominates, so one item then covers both planes of a
// complex output and writes whole 16-byte elements once.  Every mbarrier wait is bounded (2 s
// of %globaltimer): on expiry the thread records a code in the device error word and leaves its
// loop; the MMA thread still commits so that issued MMAs drain before TMEM is released.
#include "common.cuh"
#include <cudaTypedefs.h>
#include <algorithm>
#include <cstdio>
#include <cstdlib>

namespace rtcc {
namespace {

constexpr int BM = 128;
constexpr int kFuseMaxBlocks = 24;   // segment x K-block count per plane below which planes are fused
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t cnt) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return r != 0;
}
__device__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  if (mbar_test(b, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (true) {
    if (mbar_test(b, parity)) return true;
    if (gtimer() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int x,
                                          int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
// The same for a 4-D map whose box holds two consecutive K blocks: {x, row, K block, batch}.
__device__ __forceinline__ void tma_load4(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int y, int kb, int z) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(y), "r"(kb), "r"(z), "r"(bar)
      : "memory");
}
// L2 prefetch of one tile of a tensor map (no shared memory, no barrier): brings a K block that
// the producer will load a few stages later from DRAM into L2, so that its TMA load hits in L2.
__device__ __forceinline__ void tma_prefetch3(const CUtensorMap* tm, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(x), "r"(y), "r"(z)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
template <int KIND>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (KIND == 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}
// tcgen05.wait::ld that names the loaded registers as operands, so that no use of them can be
// scheduled before the wait; reg_after_wait orders further register arrays after the same wait.
#define RTCC_R32_OPERANDS \
  "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : RTCC_R32_OPERANDS::"memory");
}
__device__ __forceinline__ void reg_after_wait(uint32_t (&r)[32]) { asm volatile("" : RTCC_R32_OPERANDS::"memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  tmem_wait_ld(r);
}

// tcgen05.ld without the wait (the next tmem_ld32 waits for every load of the thread)
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
// 16-column forms (32 lanes x 16 columns per warp), load with its wait
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])::"memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row core groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                      // descriptor version (tcgen05)
  d |= (uint64_t)2 << 61;                      // layout: SWIZZLE_128B
  return d;
}

// Instruction descriptor: D f32, A/B tf32 (kind::tf32) or bf16 (kind::f16), both K-major.
template <int KIND, int BN>
__device__ __forceinline__ uint32_t idesc_make() {
  const uint32_t fmt = (KIND == 0) ? 2u : 1u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

constexpr int kGroupM = 8;   // M tiles per rasterisation group (a wave shares A and B panels in L2)

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

struct Item {
  int m0, n0, rb, np, bz, v0, nvl;   // output planes rb .. rb + np - 1
};

template <int BN>
__device__ __forceinline__ Item decode_item(const TcGemmParams& p, int w, int splits) {
  const int num_m = (p.M + BM - 1) / BM, num_n = (p.N + BN - 1) / BN;
  const int tiles = num_m * num_n;
  const int pitems = p.fused ? 1 : p.nrb;   // plane items per tile
  const int per_b = pitems * splits * tiles;
  Item it;
  it.bz = w / per_b;
  int rem = w - it.bz * per_b;
  // output plane fastest: both planes of a tile run on neighbouring CTAs and share A/B panels in L2
  it.rb = p.fused ? 0 : rem % pitems;
  it.np = p.fused ? p.nrb : 1;
  rem /= pitems;
  const int tile = rem % tiles;
  const int sp = rem / tiles;
  const int group = tile / (kGroupM * num_n);
  const int first_m = group * kGroupM;
  const int gsize = min(num_m - first_m, kGroupM);
  const int pig = tile - group * kGroupM * num_n;
  it.m0 = (first_m + pig % gsize) * BM;
  it.n0 = (pig / gsize) * BN;
  const int nv = p.nseg[it.rb] * p.nkb;
  it.v0 = sp * p.vper;
  it.nvl = max(0, min(nv, it.v0 + p.vper) - it.v0);
  return it;
}

// Output writes: a store into a fresh (zeroed) output, otherwise an atomic add without return
// (the read-modify-write happens in L2, so the epilogue never waits on the old value; each
// element is written once per launch unless K is split, so the result equals old + val).
// Outputs hold float64 (complex128) or float32 (complex64) elements; float64 values are widened
// exactly from the float32 accumulators with integer operations.
__device__ __forceinline__ void put_real(void* C, long long i, bool f32, float v, bool store) {
  if (f32) {
    float* p = static_cast<float*>(C) + i;
    if (store) *p = v;
    else atomicAdd(p, v);
  } else {
    double* p = static_cast<double*>(C) + i;
    if (store) *p = f32_to_f64_bits(v);
    else atomicAdd(p, f32_to_f64_bits(v));
  }
}
__device__ __forceinline__ void put_cplx(void* C, long long i, bool f32, float vr, float vi, bool store) {
  if (f32) {
    float2* p = static_cast<float2*>(C) + i;
    if (store) *p = make_float2(vr, vi);
    else atomicAdd(p, make_float2(vr, vi));
  } else {
    double2* p = static_cast<double2*>(C) + i;
    if (store) {
      *p = make_double2(f32_to_f64_bits(vr), f32_to_f64_bits(vi));
    } else {
      atomicAdd(&p->x, f32_to_f64_bits(vr));
      atomicAdd(&p->y, f32_to_f64_bits(vi));
    }
  }
}

// Persistent warp-specialised GEMM: each CTA walks work items (batch, output plane(s), split, tile);
// two TMEM accumulator sets let the epilogue of one tile overlap the main loop of the next.
// EPW epilogue warps: with 8, two warps share each TMEM lane quarter and split its columns.
// KPB K blocks per pipeline stage: with 2, one TMA box of A and one of B carry two consecutive K
// blocks (the TMA unit takes a roughly fixed time per stage for boxes up to 32 KB, so a stage that
// carries twice the K halves that cost per MMA).  A stage holds two blocks when both lie in the
// item's K range and in one segment; otherwise its second half (loaded, possibly zero-filled past
// the last K block) is not used.
// Accumulation chunk of virtual K block v (segment-major) of output plane rb.  The segments that
// hold a low-order split part (hi x lo, lo x hi) come first and are summed in chunks of 16 x chunk
// blocks: their products are 2^8 (BF16) or 2^11 (TF32) smaller than the hi x hi ones, so a long
// float32 accumulation of them drifts no more than a chunk of the leading products does.  The
// hi x hi segments follow in chunks of `chunk` blocks.
__device__ __forceinline__ int chunk_of(const TcGemmParams& p, int rb, int v) {
  const int mv = p.nminor[rb] * p.nkb, lm = 16 * p.chunk;
  return v < mv ? v / lm : (mv + lm - 1) / lm + (v - mv) / p.chunk;
}
// First virtual K block after v that starts a new chunk (the MMA loop tracks chunks with it, one
// division per chunk instead of several per K block).
__device__ __forceinline__ int next_chunk_start(const TcGemmParams& p, int rb, int v) {
  const int mv = p.nminor[rb] * p.nkb, lm = 16 * p.chunk;
  return v < mv ? min(mv, (v / lm + 1) * lm) : mv + ((v - mv) / p.chunk + 1) * p.chunk;
}

template <int BN, int KIND, int STAGES, int EPW, int KPB>
__global__ void __launch_bounds__(64 + 32 * EPW, 1)
    tc_gemm_kernel(const __grid_constant__ TcGemmParams p, int splits, int total_items) {
  static_assert(KPB == 1 || KPB == 2, "K blocks per stage");
  constexpr int A_BLK = BM * 128, B_BLK = BN * 128;   // bytes of one K block of A and of B
  constexpr int A_BYTES = A_BLK * KPB;
  constexpr int B_BYTES = B_BLK * KPB;
  constexpr int KBLK = (KIND == 0) ? 32 : 64;
  constexpr int WCOLS = BN * 4 / EPW;   // accumulator columns per epilogue warp
  static_assert(WCOLS % 32 == 0, "epilogue column split");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + STAGES * A_BYTES;
  float* etile = reinterpret_cast<float*>(sB + STAGES * B_BYTES);          // EPW x 32 x 33 floats
  long long* coloff_all = reinterpret_cast<long long*>(etile + EPW * 32 * 33);   // EPW x WCOLS entries
  long long* coloff2_all = coloff_all + EPW * WCOLS;                               // second targets
  uint64_t* full = reinterpret_cast<uint64_t*>(coloff2_all + EPW * WCOLS);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* cfull = tempty + 2;
  uint64_t* cempty = cfull + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(cempty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int np_all = p.fused ? p.nrb : 1;                 // planes per work item
  // TMEM: nreg item accumulators (the sums), and with chunked accumulation nreg chunk slots after them;
  // two of each when they fit in the 512 columns (the epilogue of one item then overlaps the next)
  const int chunk = p.chunk;
  const int nreg = (chunk > 0 && 4 * np_all * BN > 512) ? 1 : 2;
  const int nslot = nreg;
  const uint32_t tcols = (uint32_t)((chunk > 0 ? 2 : 1) * nreg * np_all * BN);
  const uint32_t slot0 = (uint32_t)(nreg * np_all * BN);   // first chunk slot column
  // with one sum and one slot every chunk (the first too) goes through the slot and the epilogue
  // starts the sum by a copy: the MMAs never wait for the previous item's write-out of the sum
  const bool all_slots = chunk > 0 && nreg == 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 32 * EPW);
      mbar_init(&cfull[a], 1);
      mbar_init(&cempty[a], 32 * EPW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_holder)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;
      bool alive = true;
      for (int w = blockIdx.x; w < total_items && alive; w += gridDim.x) {
        const Item it = decode_item<BN>(p, w, splits);
        for (int pl = 0; pl < it.np && alive; ++pl) {
          const int rb = it.rb + pl;
          for (int i = 0; i < it.nvl; ++g) {
            const int v = it.v0 + i;
            const int sg = v / p.nkb, kb = v - sg * p.nkb;
            const int nb = (KPB == 2 && i + 1 < it.nvl && kb + 1 < p.nkb) ? 2 : 1;   // K blocks used
            const uint32_t s = g % STAGES;
            if (g >= STAGES && !mbar_wait(&empty[s], ((g / STAGES) - 1) & 1)) {
              atomicExch(p.err, DEV_TIMEOUT_PRODUCER);
              alive = false;
              break;
            }
            mbar_arrive_tx(&full[s], A_BYTES + B_BYTES);
            if constexpr (KPB == 2) {
              tma_load4(su32(sA + s * A_BYTES), &p.tmA2, su32(&full[s]), p.seg[rb][sg].pa * p.M + it.m0, kb, it.bz);
              tma_load4(su32(sB + s * B_BYTES), &p.tmB2, su32(&full[s]), p.seg[rb][sg].pb * p.N + it.n0, kb, it.bz);
            } else {
              tma_load3(su32(sA + s * A_BYTES), &p.tmA, su32(&full[s]), kb * KBLK, p.seg[rb][sg].pa * p.M + it.m0,
                        it.bz);
              tma_load3(su32(sB + s * B_BYTES), &p.tmB, su32(&full[s]), kb * KBLK, p.seg[rb][sg].pb * p.N + it.n0,
                        it.bz);
            }
            i += nb;
            // the K block this loop loads `prefetch` iterations from now (same item and plane), into L2
            if (KPB == 1 && p.prefetch > 0 && i - 1 + p.prefetch < it.nvl) {
              const int vf = v + p.prefetch;
              const int sgf = vf / p.nkb, kbf = vf - sgf * p.nkb;
              tma_prefetch3(&p.tmA, kbf * KBLK, p.seg[rb][sgf].pa * p.M + it.m0, it.bz);
              tma_prefetch3(&p.tmB, kbf * KBLK, p.seg[rb][sgf].pb * p.N + it.n0, it.bz);
            }
          }
        }
      }
      if (!alive) {
        // after an expired wait: let the copies already issued land before the CTA exits (bounded)
        for (uint32_t q = (g > STAGES ? g - STAGES : 0); q < g; ++q) mbar_wait(&full[q % STAGES], (q / STAGES) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_make<KIND, BN>();
      uint32_t g = 0, gs = 0;   // K blocks consumed, chunk slots used
      int local = 0;
      bool alive = true;
      for (int w = blockIdx.x; w < total_items && alive; w += gridDim.x, ++local) {
        const Item it = decode_item<BN>(p, w, splits);
        const int a = local % nreg, u = local / nreg;
        if (!all_slots && u > 0 && !mbar_wait(&tempty[a], (u - 1) & 1)) {
          atomicExch(p.err, DEV_TIMEOUT_MMA);
          break;
        }
        tc_fence_after();
        for (int pl = 0; pl < it.np && alive; ++pl) {
          const int rb = it.rb + pl;
          const uint32_t acc_sum = tmem + (uint32_t)((a * it.np + pl) * BN);
          uint32_t acc = acc_sum;
          uint32_t slot = 0;
          const int vend = it.v0 + it.nvl;
          int cnext = chunk > 0 ? next_chunk_start(p, rb, it.v0) : vend;   // where the next chunk starts
          bool later = false;                                             // past the item's first chunk
          for (int i = 0; i < it.nvl && alive; ++g) {
            const int v = it.v0 + i;
            const int sg = v / p.nkb;
            const int nb = (KPB == 2 && i + 1 < it.nvl && v - sg * p.nkb + 1 < p.nkb) ? 2 : 1;   // as the producer
            const uint32_t s = g % STAGES;
            for (int j = 0; j < nb; ++j) {
              const int vb = v + j;   // virtual K block
              // chunk 0 of the plane accumulates into the item's sum, every later chunk into a slot
              // that the epilogue folds into the sum
              bool cstart = j == 0 && i == 0;
              if (vb == cnext) {
                cstart = true;
                later = true;
                cnext = next_chunk_start(p, rb, vb);
              }
              const bool cend = vb + 1 == vend || vb + 1 == cnext;
              if (chunk > 0 && cstart && (later || all_slots)) {
                slot = gs % nslot;
                const uint32_t sp = gs / nslot;
                if (sp > 0 && !mbar_wait(&cempty[slot], (sp - 1) & 1)) {
                  atomicExch(p.err, DEV_TIMEOUT_MMA);
                  alive = false;
                  break;
                }
                tc_fence_after();
                acc = tmem + slot0 + (uint32_t)((slot * it.np + pl) * BN);
              }
              if (j == 0) {
                if (!mbar_wait(&full[s], (g / STAGES) & 1)) {
                  atomicExch(p.err, DEV_TIMEOUT_MMA);
                  alive = false;
                  break;
                }
                tc_fence_after();
              }
              const uint64_t ad = sdesc_sw128(su32(sA + s * A_BYTES + j * A_BLK));
              const uint64_t bd = sdesc_sw128(su32(sB + s * B_BYTES + j * B_BLK));
              const uint32_t id = idesc | ((uint32_t)p.seg[rb][sg].neg << 13);   // negate A for -Ai Bi
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)   // 4 MMAs of 32 bytes of K per 128-byte block
                tc_mma<KIND>(acc, ad + 2ull * kk, bd + 2ull * kk, id, (cstart && kk == 0) ? 0u : 1u);
              if (chunk > 0 && (later || all_slots) && cend) {
                tc_commit(su32(&cfull[slot]));   // this chunk's slot is complete
                ++gs;
              }
            }
            if (!alive) break;
            tc_commit(su32(&empty[s]));   // the stage is free once its MMAs have read it
            i += nb;
          }
        }
        // With one sum the item's MMAs never wait for the previous write-out, so the commit below must:
        // an mbarrier phase completes only once its waiter has seen the previous one, and a short item
        // (a split remainder of a few K blocks, or none) could otherwise complete tfull twice before the
        // epilogue waits on the first completion, which it would then never see.
        if (all_slots && alive && local > 0 && !mbar_wait(&tempty[a], (local - 1) & 1)) {
          atomicExch(p.err, DEV_TIMEOUT_MMA);
          break;
        }
        tc_commit(su32(&tfull[a]));   // arrives when this tile's MMAs have completed
      }
    }
    __syncwarp();
  } else {
    // epilogue warps: TMEM lane quarter q = warp % 4, columns [hc, hc + WCOLS) of the tile
    const int q = warp & 3, ew = warp - 2;
    const int hc = (ew / 4) * WCOLS;
    const TcEpilogue& e = p.epi;
    // the scale is applied in float32 (its rounding, 2^-24 relative, is far below the operand
    // split's resolution) and the result widened exactly with integer operations
    const float alpha_f = (float)e.alpha;
    // a fresh output is stored, unless K is split (the slices then add into the zeroed output)
    const bool store = e.store && splits == 1;
    float* tile = etile + ew * (32 * 33);
    long long* coloff = coloff_all + ew * WCOLS;   // warp-private: no cross-warp barrier in the epilogue
    long long* coloff2 = coloff2_all + ew * WCOLS;
    const bool dual = e.ctab1 != nullptr;          // pair-symmetric scatter to a second column
    const float s2 = e.sign2;
    int local = 0;
    uint32_t gs = 0;   // chunk slots folded
    bool alive = true;
    for (int w = blockIdx.x; w < total_items && alive; w += gridDim.x, ++local) {
      const Item it = decode_item<BN>(p, w, splits);
      const int a = local % nreg, u = local / nreg;
      if (chunk > 0) {
        // fold every chunk after the first into the plane's sum, in the order the MMA warp issued
        // them: sum += slot with round-to-nearest float32 adds, then the slot is handed back
        const uint32_t lanes = ((uint32_t)(q * 32) << 16);
        for (int pl = 0; pl < it.np && alive; ++pl) {
          const int rbp = it.rb + pl;
          const int nch = it.nvl > 0 ? chunk_of(p, rbp, it.v0 + it.nvl - 1) - chunk_of(p, rbp, it.v0) + 1 : 0;
          for (int c = all_slots ? 0 : 1; c < nch; ++c, ++gs) {
            const uint32_t slot = gs % nslot, sp = gs / nslot;
            bool okc = mbar_wait(&cfull[slot], sp & 1);
            okc = __all_sync(0xffffffffu, okc);
            if (!okc) {
              if (lane == 0) atomicExch(p.err, DEV_TIMEOUT_EPI);
              alive = false;
              break;
            }
            tc_fence_after();
            const uint32_t sum_c = tmem + lanes + (uint32_t)((a * it.np + pl) * BN + hc);
            const uint32_t slot_c = tmem + lanes + slot0 + (uint32_t)((slot * it.np + pl) * BN + hc);
            if constexpr (WCOLS <= 128) {
              // the slot's columns are copied into registers and the slot is handed back at once, so
              // the MMAs wait only for these loads; the sum is updated afterwards
              constexpr int NP = WCOLS / 32;
              uint32_t xs[NP][32];
#pragma unroll
              for (int k = 0; k < NP; ++k) tmem_ld32_nowait(slot_c + (uint32_t)(32 * k), xs[k]);
              tmem_wait_ld(xs[0]);
#pragma unroll
              for (int k = 1; k < NP; ++k) reg_after_wait(xs[k]);
              tc_fence_before();
              mbar_arrive(&cempty[slot]);
#pragma unroll
              for (int k = 0; k < NP; ++k) {
                if (c == 0) {   // the item's first chunk starts the sum
                  tmem_st32(sum_c + (uint32_t)(32 * k), xs[k]);
                } else {   // 16 columns at a time: the copy of the slot already holds most registers
#pragma unroll
                  for (int hh = 0; hh < 2; ++hh) {
                    uint32_t y[16];
                    tmem_ld16(sum_c + (uint32_t)(32 * k + 16 * hh), y);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                      y[j] = __float_as_uint(__fadd_rn(__uint_as_float(y[j]), __uint_as_float(xs[k][16 * hh + j])));
                    tmem_st16(sum_c + (uint32_t)(32 * k + 16 * hh), y);
                  }
                }
              }
              tmem_wait_st();
              continue;
            }
            if (c == 0) {   // the item's first chunk starts the sum
#pragma unroll 1
              for (int cc = 0; cc < WCOLS; cc += 32) {
                uint32_t x[32];
                tmem_ld32(slot_c + (uint32_t)cc, x);
                tmem_st32(sum_c + (uint32_t)cc, x);
              }
            } else if constexpr (WCOLS % 64 != 0) {
              uint32_t x[32], y[32];
              tmem_ld32_nowait(slot_c, x);
              tmem_ld32(sum_c, y);   // waits for both loads
              reg_after_wait(x);
#pragma unroll
              for (int j = 0; j < 32; ++j)
                y[j] = __float_as_uint(__fadd_rn(__uint_as_float(y[j]), __uint_as_float(x[j])));
              tmem_st32(sum_c, y);
            } else {
              // 64 columns per round trip: four loads in flight, one wait
#pragma unroll 1
              for (int cc = 0; cc < WCOLS; cc += 64) {
                uint32_t x[32], y[32], x2[32], y2[32];
                tmem_ld32_nowait(slot_c + (uint32_t)cc, x);
                tmem_ld32_nowait(sum_c + (uint32_t)cc, y);
                tmem_ld32_nowait(slot_c + (uint32_t)(cc + 32), x2);
                tmem_ld32(sum_c + (uint32_t)(cc + 32), y2);   // waits for all four loads
                reg_after_wait(x);
                reg_after_wait(y);
                reg_after_wait(x2);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                  y[j] = __float_as_uint(__fadd_rn(__uint_as_float(y[j]), __uint_as_float(x[j])));
                  y2[j] = __float_as_uint(__fadd_rn(__uint_as_float(y2[j]), __uint_as_float(x2[j])));
                }
                tmem_st32(sum_c + (uint32_t)cc, y);
                tmem_st32(sum_c + (uint32_t)(cc + 32), y2);
              }
            }
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(&cempty[slot]);
          }
        }
        if (!alive) break;
      }
      // output offsets of this item (computed while the MMAs of the item are still running)
      __syncwarp();
      for (int c = lane; c < WCOLS; c += 32) {
        const int n = it.n0 + hc + c;
        if (dual) {
          coloff[c] = (n < p.N) ? e.ctab1[n] : -1;
          coloff2[c] = (n < p.N) ? e.ctab2[n] : -1;
        } else {
          coloff[c] = (n < p.N) ? (e.flat_n ? (long long)n * e.sn : imap32(e.cn, (unsigned)n)) : -1;
        }
      }
      __syncwarp();
      const int row = it.m0 + q * 32 + lane;
      long long rowoff = 0;
      if (row < p.M) rowoff = imap32(e.cb, (unsigned)it.bz) + imap32(e.cm, (unsigned)row);
      bool ok = mbar_wait(&tfull[a], u & 1);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) atomicExch(p.err, DEV_TIMEOUT_EPI);
        break;
      }
      tc_fence_after();
      const uint32_t acc = tmem + (uint32_t)(a * it.np * BN + hc) + ((uint32_t)(q * 32) << 16);
      const bool both = it.np == 2 && e.c_cplx;   // write complex elements whole
#pragma unroll 1
      for (int c = 0; c < WCOLS; c += 32) {
        if (it.nvl == 0) continue;   // uniform over the warp
        if (both) {
          if (e.unit_n) {
            // transpose both planes through the warp's tile: lane then owns column c + lane
            float tre[32], tim[32];
            {
              uint32_t r[32];
              tmem_ld32(acc + (uint32_t)c, r);
#pragma unroll
              for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(r[j]);
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 32; ++j) tre[j] = tile[j * 33 + lane];
            __syncwarp();
            {
              uint32_t r[32];
              tmem_ld32(acc + (uint32_t)(BN + c), r);
#pragma unroll
              for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(r[j]);
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 32; ++j) tim[j] = tile[j * 33 + lane];
            __syncwarp();
            const long long noff = coloff[c + lane];
            const long long noff2 = dual ? coloff2[c + lane] : -1;
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) {
              const long long ro = __shfl_sync(0xffffffffu, rowoff, rr);
              if (noff >= 0 && it.m0 + q * 32 + rr < p.M) {
                put_cplx(e.C, ro + noff, e.c_f32, alpha_f * tre[rr], alpha_f * tim[rr], store);
                if (noff2 >= 0)
                  put_cplx(e.C, ro + noff2, e.c_f32, s2 * alpha_f * tre[rr], s2 * alpha_f * tim[rr], store);
              }
            }
          } else {
            uint32_t rre[32], rim[32];
            tmem_ld32(acc + (uint32_t)c, rre);
            tmem_ld32(acc + (uint32_t)(BN + c), rim);
            if (row >= p.M) continue;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const long long no = coloff[c + j];
              if (no >= 0) {
                put_cplx(e.C, rowoff + no, e.c_f32, alpha_f * __uint_as_float(rre[j]),
                         alpha_f * __uint_as_float(rim[j]), store);
                const long long no2 = dual ? coloff2[c + j] : -1;
                if (no2 >= 0)
                  put_cplx(e.C, rowoff + no2, e.c_f32, s2 * alpha_f * __uint_as_float(rre[j]),
                           s2 * alpha_f * __uint_as_float(rim[j]), store);
              }
            }
          }
          continue;
        }
        // one plane per pass: plane it.rb + pl of the output, one component of C at a time
        for (int pl = 0; pl < it.np; ++pl) {
          const int comp = it.rb + pl;
          uint32_t r[32];
          tmem_ld32(acc + (uint32_t)(pl * BN + c), r);
          if (e.unit_n) {
#pragma unroll
            for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(r[j]);
            __syncwarp();
            const long long noff = coloff[c + lane];
            const long long noff2 = dual ? coloff2[c + lane] : -1;
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) {
              const long long ro = __shfl_sync(0xffffffffu, rowoff, rr);
              if (noff >= 0 && it.m0 + q * 32 + rr < p.M) {
                const float val = alpha_f * tile[rr * 33 + lane];
                const long long off = ro + noff;
                put_real(e.C, e.c_cplx ? 2 * off + comp : off, e.c_f32, val, store);
                if (noff2 >= 0) {
                  const long long off2 = ro + noff2;
                  put_real(e.C, e.c_cplx ? 2 * off2 + comp : off2, e.c_f32, s2 * val, store);
                }
              }
            }
            __syncwarp();
          } else if (row < p.M) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const long long no = coloff[c + j];
              if (no >= 0) {
                const float val = alpha_f * __uint_as_float(r[j]);
                const long long off = rowoff + no;
                put_real(e.C, e.c_cplx ? 2 * off + comp : off, e.c_f32, val, store);
                const long long no2 = dual ? coloff2[c + j] : -1;
                if (no2 >= 0) {
                  const long long off2 = rowoff + no2;
                  put_real(e.C, e.c_cplx ? 2 * off2 + comp : off2, e.c_f32, s2 * val, store);
                }
              }
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[a]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
  }
}

template <int BN, int KIND, int STAGES, int EPW, int KPB>
constexpr size_t smem_bytes() {
  return 1024 + (size_t)STAGES * KPB * (BM * 128 + BN * 128) + (size_t)EPW * 32 * 33 * 4 + (size_t)2 * 4 * BN * 8 +
         (2 * STAGES + 8) * 8 + 16;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    RTCC_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || p == nullptr)
      throw Error(3, "cuTensorMapEncodeTiled is not available from the driver");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

void make_map(CUtensorMap* tm, int kind, const void* ptr, long long rows, long long Kpad, long long NB,
              int box_rows) {
  const int esz = (kind == 0) ? 4 : 2;
  RTCC_REQUIRE((reinterpret_cast<uintptr_t>(ptr) & 15) == 0, "TMA base address must be 16-byte aligned");
  RTCC_REQUIRE((Kpad * esz) % 128 == 0, "packed K must be whole 128-byte blocks");
  cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows, (cuuint64_t)NB};
  cuuint64_t strides[2] = {(cuuint64_t)(Kpad * esz), (cuuint64_t)(rows * Kpad * esz)};
  cuuint32_t box[3] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(tm, kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                           const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(3, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
}

// The same operand as a 4-D view {K within a block, row, K block, batch} (strides: row, 128 bytes,
// batch) whose box holds two consecutive K blocks of box_rows rows: in shared memory the two
// blocks land one after the other, each laid out as a single-block box.  Returns false when the
// driver does not accept the view (the two-block variant is then not used).
bool make_map_pair(CUtensorMap* tm, int kind, const void* ptr, long long rows, long long Kpad, long long NB,
                   int box_rows) {
  const int esz = (kind == 0) ? 4 : 2;
  const long long nkb = Kpad * esz / 128;
  cuuint64_t dims[4] = {(cuuint64_t)(128 / esz), (cuuint64_t)rows, (cuuint64_t)nkb, (cuuint64_t)NB};
  cuuint64_t strides[3] = {(cuuint64_t)(Kpad * esz), 128, (cuuint64_t)(rows * Kpad * esz)};
  cuuint32_t box[4] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows, 2, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode_fn()(tm, kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                           const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, int KIND, int STAGES, int EPW, int KPB = 1>
void launch_inst(const TcGemmPlan& pl, cudaStream_t s) {
  auto kern = tc_gemm_kernel<BN, KIND, STAGES, EPW, KPB>;
  constexpr size_t sm = smem_bytes<BN, KIND, STAGES, EPW, KPB>();
  static_assert(sm <= 227 * 1024, "shared memory budget");
  static bool attr = false;
  if (!attr) {
    RTCC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = true;
  }
  const int nsm = device_sm_count();
  const long long tiles = (long long)((pl.p.M + BM - 1) / BM) * ((pl.p.N + BN - 1) / BN);
  const long long items = tiles * (pl.p.fused ? 1 : pl.p.nrb) * pl.splits * pl.NB;
  RTCC_REQUIRE(items < (1ll << 31), "too many GEMM tiles");
  const unsigned grid = (unsigned)std::min<long long>(items, nsm);
  kern<<<grid, 64 + 32 * EPW, sm, s>>>(pl.p, pl.splits, (int)items);
  RTCC_CUDA(cudaGetLastError());
}

}  // namespace

int tc_kblock_elems(int kind) { return kind == 0 ? 32 : 64; }

void tc_gemm_plan(TcGemmPlan& pl, int kind, const void* A, int planesA, const void* B, int planesB, long long M,
                  long long N, long long Kpad, long long NB, int* err, int bn, int chunk) {
  RTCC_REQUIRE(chunk >= 0, "negative accumulation chunk");
  pl.p.chunk = chunk;
  pl.variant = 0;
  pl.p.prefetch = 0;
  RTCC_REQUIRE(M > 0 && N > 0 && Kpad > 0 && NB > 0, "empty GEMM");
  RTCC_REQUIRE(M * planesA < (1ll << 31) && N * planesB < (1ll << 31) && NB < 65536, "GEMM extents too large");
  pl.kind = kind;
  pl.bn = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
  if (bn == 64 || bn == 128 || bn == 256) pl.bn = bn;
  // RTCC_GEMM_TILE=<n>[:<variant>] forces the tile (n = 64, 128 or 256) and its variant, for tests
  // of every kernel instantiation; a complex output fused into one item still takes n <= 128
  int forced_variant = -1;
  if (const char* e = std::getenv("RTCC_GEMM_TILE")) {
    int fb = 0, fv = 0;
    const int got = std::sscanf(e, "%d:%d", &fb, &fv);
    if (got >= 1 && (fb == 64 || fb == 128 || fb == 256)) {
      pl.bn = fb;
      forced_variant = got == 2 ? std::max(0, std::min(fv, 2)) : 0;
    }
  }
  // Short K loops leave the epilogue as the bottleneck: one item then covers both planes of a
  // complex output (whole 16-byte elements written once, by eight epilogue warps).  Two planes
  // of accumulators, double-buffered, fit TMEM's 512 columns up to a 128-column tile.
  const bool both = pl.p.nrb == 2 && pl.p.epi.c_cplx && pl.p.nseg[0] == pl.p.nseg[1];
  pl.p.fused = (both && (long long)pl.p.nseg[0] * (Kpad / tc_kblock_elems(kind)) <= kFuseMaxBlocks) ? 1 : 0;
  if (pl.p.fused) pl.bn = std::min(pl.bn, 128);
  pl.NB = NB;
  pl.p.M = (int)M;
  pl.p.N = (int)N;
  pl.p.nkb = (int)(Kpad / tc_kblock_elems(kind));
  pl.p.err = err;
  make_map(&pl.p.tmA, kind, A, M * planesA, Kpad, NB, BM);
  make_map(&pl.p.tmB, kind, B, N * planesB, Kpad, NB, pl.bn);
  pl.pair_maps = make_map_pair(&pl.p.tmA2, kind, A, M * planesA, Kpad, NB, BM) &&
                 make_map_pair(&pl.p.tmB2, kind, B, N * planesB, Kpad, NB, pl.bn);
  // split K when the output has less than one wave of tiles and the K loop is long
  const long long tiles = ((M + BM - 1) / BM) * ((N + pl.bn - 1) / pl.bn) * NB * (pl.p.fused ? 1 : pl.p.nrb);
  const int nv = pl.p.nseg[0] * pl.p.nkb;
  int splits = 1;
  const long long nsm = device_sm_count();
  if (tiles < nsm && nv >= 32) splits = (int)std::max(1ll, std::min<long long>((2 * nsm + tiles - 1) / tiles, nv / 16));
  splits = std::min(splits, 64);
  pl.p.vper = (nv + splits - 1) / splits;
  pl.splits = (nv + pl.p.vper - 1) / pl.p.vper;
  // an item whose K loop fits in one chunk accumulates once, in the double-buffered accumulators
  if (pl.p.chunk >= pl.p.vper) pl.p.chunk = 0;
  // with chunks, the split parts' segments (planes are component x 2 + part, part 0 the high
  // half) go first, in their given order, then the hi x hi ones (see chunk_of)
  for (int rb = 0; rb < 2; ++rb) {
    pl.p.nminor[rb] = 0;
    if (pl.p.chunk == 0 || rb >= pl.p.nrb) continue;
    RTCC_REQUIRE(planesA % 2 == 0 && planesB % 2 == 0, "chunked accumulation needs split operand planes");
    TcSeg ordered[kMaxSeg];
    int n = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (int q = 0; q < pl.p.nseg[rb]; ++q) {
        const TcSeg& sgm = pl.p.seg[rb][q];
        const bool major = sgm.pa % 2 == 0 && sgm.pb % 2 == 0;
        if (major == (pass == 1)) ordered[n++] = sgm;
      }
    for (int q = 0; q < n; ++q) {
      pl.p.seg[rb][q] = ordered[q];
      if (!(ordered[q].pa % 2 == 0 && ordered[q].pb % 2 == 0)) pl.p.nminor[rb] = q + 1;
    }
  }
  if (forced_variant >= 0) pl.variant = forced_variant;
  if (pl.variant == 2 && !pl.pair_maps) pl.variant = 0;
}

template <int KIND>
void launch_kind(const TcGemmPlan& p, cudaStream_t s) {
  if (p.bn == 64) launch_inst<64, KIND, 7, 8>(p, s);
  else if (p.bn == 128) {
    if (p.variant == 2) launch_inst<128, KIND, 3, 4, 2>(p, s);
    else if (p.variant == 1) launch_inst<128, KIND, 6, 4>(p, s);
    else launch_inst<128, KIND, 5, 8>(p, s);
  } else if (p.variant == 2) {
    launch_inst<256, KIND, 2, 4, 2>(p, s);
  } else if (p.variant == 1) {
    launch_inst<256, KIND, 3, 8>(p, s);
  } else {
    launch_inst<256, KIND, 4, 4>(p, s);
  }
}

void launch_tc_gemm(const TcGemmPlan& p, cudaStream_t s) {
  RTCC_REQUIRE(p.variant != 2 || p.pair_maps, "two-K-block GEMM variant without its tensor maps");
  if (p.kind == 0) launch_kind<0>(p, s);
  else launch_kind<1>(p, s);
}

}  // namespace rtcc
