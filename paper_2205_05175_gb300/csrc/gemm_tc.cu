// tcgen05 tensor-core GEMM for the residual contractions (sm_103a).
//
// C[b][m][n] = sum_k A[b][m][k] * B[b][n][k], both operands K-major in global memory
// (packed by the pack kernel, rows padded to whole 128-byte K blocks), C float32.
//
// One CTA computes a 128 x BN tile with 128 threads:
//   warp 0 lane 0 : TMA producer (cp.async.bulk.tensor, 128-byte swizzle, mbarrier tx)
//   warp 1 lane 0 : MMA issuer (tcgen05.mma kind::tf32 or kind::f16 with bf16 inputs,
//                   accumulator in TMEM, tcgen05.commit releases smem stages)
//   warps 0-3     : epilogue (tcgen05.ld 32x32b, lane quarter per warp) -> global
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the thread records a
// code in the device error word and leaves its loop, the MMA thread still commits so
// that in-flight MMAs drain before TMEM is released.
#include "common.cuh"
#include <cudaTypedefs.h>
#include <algorithm>

namespace rtcc {
namespace {

constexpr int BM = 128;
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
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

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

template <int BN, int KIND, int STAGES>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   float* __restrict__ C, int M, int N, int nkb_total, int kb_per_split, int* __restrict__ err) {
  constexpr int A_BYTES = BM * 128;
  constexpr int B_BYTES = BN * 128;
  constexpr int KBLK = (KIND == 0) ? 32 : 64;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(accf + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped rasterisation: GROUP_M consecutive M tiles sweep all N tiles before the next group
  const int num_m = (M + BM - 1) / BM, num_n = (N + BN - 1) / BN;
  const int pid = blockIdx.x;
  const int group = pid / (kGroupM * num_n);
  const int first_m = group * kGroupM;
  const int gsize = min(num_m - first_m, kGroupM);
  const int pig = pid - group * kGroupM * num_n;
  const int m0 = (first_m + pig % gsize) * BM, n0 = (pig / gsize) * BN, bz = blockIdx.z;
  // split-K range of this CTA
  const int kb0 = blockIdx.y * kb_per_split;
  const int nkb = min(nkb_total, kb0 + kb_per_split) - kb0;
  const bool split = gridDim.y > 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_holder)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1)) {
        atomicExch(err, DEV_TIMEOUT_PRODUCER);
        break;
      }
      mbar_arrive_tx(&full[s], A_BYTES + B_BYTES);
      tma_load3(su32(sA + s * A_BYTES), &tmA, su32(&full[s]), (kb0 + kb) * KBLK, m0, bz);
      tma_load3(su32(sB + s * B_BYTES), &tmB, su32(&full[s]), (kb0 + kb) * KBLK, n0, bz);
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_make<KIND, BN>();
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full[s], (kb / STAGES) & 1)) {
        atomicExch(err, DEV_TIMEOUT_MMA);
        break;
      }
      tc_fence_after();
      const uint64_t ad = sdesc_sw128(su32(sA + s * A_BYTES));
      const uint64_t bd = sdesc_sw128(su32(sB + s * B_BYTES));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)  // 4 MMAs of 32 bytes of K per 128-byte block
        tc_mma<KIND>(tmem, ad + 2ull * kk, bd + 2ull * kk, idesc, (kb | kk) ? 1u : 0u);
      tc_commit(su32(&empty[s]));
    }
    tc_commit(su32(accf));
  }
  __syncwarp();

  bool ok = mbar_wait(accf, 0);
  ok = __all_sync(0xffffffffu, ok);
  if (!ok && lane == 0) atomicExch(err, DEV_TIMEOUT_EPI);
  tc_fence_after();
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    float* crow = C + ((size_t)bz * (size_t)M + (size_t)row) * (size_t)N;
    const bool vec = (N % 4) == 0;
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
      const int col0 = n0 + c;
      if (row < M && col0 < N && split) {
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (col0 + q < N) atomicAdd(crow + col0 + q, __uint_as_float(r[q]));
      } else if (row < M && col0 < N) {
        if (vec && col0 + 32 <= N) {
          float4* dst = reinterpret_cast<float4*>(crow + col0);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                 __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (col0 + q < N) crow[col0 + q] = __uint_as_float(r[q]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN)
                 : "memory");
  }
}

template <int BN, int KIND, int STAGES>
constexpr size_t smem_bytes() {
  return 1024 + (size_t)STAGES * (BM * 128 + BN * 128) + (2 * STAGES + 1) * 8 + 16;
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

template <int BN, int KIND, int STAGES>
void launch_inst(const TcGemmPlan& p, cudaStream_t s) {
  auto kern = tc_gemm_kernel<BN, KIND, STAGES>;
  constexpr size_t sm = smem_bytes<BN, KIND, STAGES>();
  static bool attr = false;
  if (!attr) {
    RTCC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = true;
  }
  const int nkb = (int)(p.Kpad / (KIND == 0 ? 32 : 64));
  const long long tiles = ((p.M + BM - 1) / BM) * ((p.N + BN - 1) / BN);
  // split K when the output has less than one wave of tiles and K is long
  int splits = 1;
  if (tiles * p.NB < 152 && nkb >= 32) {
    splits = (int)std::min<long long>((2 * 152 + tiles * p.NB - 1) / (tiles * p.NB), nkb / 16);
    splits = std::max(1, std::min(splits, 64));
  }
  const int per = (nkb + splits - 1) / splits;
  splits = (nkb + per - 1) / per;
  if (splits > 1) RTCC_CUDA(cudaMemsetAsync(p.C, 0, sizeof(float) * p.M * p.N * p.NB, s));
  dim3 grid((unsigned)tiles, (unsigned)splits, (unsigned)p.NB);
  kern<<<grid, 128, sm, s>>>(p.tmA, p.tmB, p.C, (int)p.M, (int)p.N, nkb, per, p.err);
  RTCC_CUDA(cudaGetLastError());
}

}  // namespace

int tc_kblock_elems(int kind) { return kind == 0 ? 32 : 64; }

void tc_gemm_plan(TcGemmPlan& p, int kind, const void* A, const void* B, float* C, long long M, long long N,
                  long long Kpad, long long NB, int* err) {
  RTCC_REQUIRE(M > 0 && N > 0 && Kpad > 0 && NB > 0, "empty GEMM");
  RTCC_REQUIRE(M < (1ll << 31) && N < (1ll << 31) && NB < 65536, "GEMM extents too large");
  p.kind = kind;
  p.bn = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
  p.M = M;
  p.N = N;
  p.Kpad = Kpad;
  p.NB = NB;
  p.C = C;
  p.err = err;
  make_map(&p.tmA, kind, A, M, Kpad, NB, BM);
  make_map(&p.tmB, kind, B, N, Kpad, NB, p.bn);
}

void launch_tc_gemm(const TcGemmPlan& p, cudaStream_t s) {
  if (p.kind == 0) {
    if (p.bn == 64) launch_inst<64, 0, 8>(p, s);
    else if (p.bn == 128) launch_inst<128, 0, 6>(p, s);
    else launch_inst<256, 0, 4>(p, s);
  } else {
    if (p.bn == 64) launch_inst<64, 1, 8>(p, s);
    else if (p.bn == 128) launch_inst<128, 1, 6>(p, s);
    else launch_inst<256, 1, 4>(p, s);
  }
}

}  // namespace rtcc
