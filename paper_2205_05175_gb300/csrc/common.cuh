// Shared declarations of the RT-CCSD CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>
#include <stdexcept>

namespace rtcc {

// ---------------------------------------------------------------------------------------
// Errors: library code throws rtcc::Error; the C-ABI layer converts it to a status code.
struct Error : std::runtime_error {
  int status;
  Error(int s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define RTCC_CUDA(call)                                                                  \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      throw ::rtcc::Error(3, std::string(#call) + ": " + cudaGetErrorString(e_) + " at " + \
                                 __FILE__ + ":" + std::to_string(__LINE__));             \
  } while (0)

#define RTCC_REQUIRE(cond, msg)                                                          \
  do {                                                                                   \
    if (!(cond)) throw ::rtcc::Error(1, std::string(msg));                              \
  } while (0)

// Records the message rtcc_last_error() returns (thread-local).
void set_last_error(const std::string& msg);

// Device error word written by kernels whose bounded waits expire (never trapped).
enum DevErr : int { DEV_OK = 0, DEV_TIMEOUT_PRODUCER = 1, DEV_TIMEOUT_MMA = 2, DEV_TIMEOUT_EPI = 3 };

// ---------------------------------------------------------------------------------------
// Mixed-radix index map: a linear index over a group of labels -> element offset.
constexpr int kMaxLab = 6;
struct IndexMap {
  int n;                       // number of labels in the group (0 = scalar group)
  int dims[kMaxLab];           // extents, outermost first
  long long strides[kMaxLab];  // element strides, same order
};

__host__ __device__ inline long long imap_offset(const IndexMap& m, long long idx) {
  long long off = 0;
  for (int d = m.n - 1; d >= 0; --d) {
    long long q = idx / m.dims[d];
    off += (idx - q * m.dims[d]) * m.strides[d];
    idx = q;
  }
  return off;
}

inline long long imap_size(const IndexMap& m) {
  long long s = 1;
  for (int d = 0; d < m.n; ++d) s *= m.dims[d];
  return s;
}

// ---------------------------------------------------------------------------------------
// Packed-operand description for the GEMM path.
//  rows' = nrb * R, cols' = Kpad >= nss * ncs * K.  Column kk -> (ss, cs, k); row r -> (rb, m).
//  value = sign[rb][cs] * component(src(m,k), comp[rb][cs]) then split part[ss].
enum PackElem : int { PE_F32 = 0, PE_BF16 = 1, PE_F64 = 2 };
enum SplitPart : int { SP_FULL = 0, SP_HI = 1, SP_LO = 2 };
constexpr int kMaxRb = 4;
struct PackDesc {
  const void* src;
  int src_cplx;
  int src_f32;      // source elements are float32 (complex64) instead of float64
  IndexMap rows;    // R labels
  IndexMap cols;    // K labels
  IndexMap bat;     // batch labels
  long long R, K, NB;
  int nrb, ncs, nss;
  int comp[kMaxRb][2];   // 0 = re, 1 = im
  int sign[kMaxRb][2];
  int part[3];           // split part per column segment (when nss > 1)
  int rb_part[kMaxRb];   // split part per row block (when nss == 1): planes of a tensor-core operand
  long long Kpad;   // padded row length of the packed matrix
  int elem;         // PackElem
  int round_tf32;   // round float32 values to TF32 (round-to-nearest) when packing
  int transpose;    // 1: the source's unit-stride index is a row index (shared-memory tile transpose)
  // transpose mode: rows are enumerated in "read order" (the source's unit-stride label last);
  // rd_src gives the source offset and rd_dst the packed row index of a read-order row
  IndexMap rd_src, rd_dst;
  void* dst;
  // pair-symmetric gather (plane packs, direct mode only): when ktab is set, packed column k
  // holds kw[k] * (src[o1] + ksign * src[o2]) with (o1, o2) = ktab[2k], ktab[2k+1] added to the
  // row offset (kw may be null: weight 1); when rtab is set, row m starts at rtab[m]
  const long long* ktab;
  const float* kw;
  float ksign;
  const long long* rtab;
};

// Unpack: C[bt, m, n] += alpha * (value assembled from the GEMM output).
enum OutMode : int { OM_REAL = 0, OM_STACK_M = 1, OM_STACK_N = 2 };
struct UnpackDesc {
  const void* gout;      // float32 or float64 [NB][rows'][cols']
  int gout_f64;
  long long ldg;         // row length of gout (cols')
  long long rows_g;      // rows' (batch stride = rows_g * ldg)
  int mode;              // OutMode
  long long M, N, NB;
  IndexMap cm, cn, cb;   // output offsets
  double* C;
  int c_cplx;
  double ar, ai;
  int transpose;         // 1: the output's unit-stride index is an M index (shared-memory tile transpose)
};

// Direct (small) contraction C[bt,m,n] += alpha * sum_k A[bt,m,k] B[bt,n,k] in float64.
struct DirectDesc {
  const void* A; const void* B; void* C;
  int a_cplx, b_cplx, c_cplx;
  int a_f32, b_f32, c_f32;   // float32 (complex64) elements
  IndexMap am, ak, ab, bn, bk, bb, cm, cn, cb;
  long long M, N, K, NB;
  double ar, ai;
  int store;        // 1: C is known to be zero: store instead of read-modify-write
  int f32;          // 1: sum products in float32 (reduced-precision programs)
};

// C[lc] (+)= sum_s alpha_s * A_s[la_s] with labels(A_s) a subset of labels(C) (broadcast over the
// rest); several sources when consecutive adds into one output are merged.
constexpr int kMaxAddSrc = 4;
struct AddDesc {
  void* C;
  int c_cplx;
  int c_f32;
  int store;        // 1: C is known to be zero: store instead of read-modify-write
  int f32;          // 1: sum in float32 (reduced-precision programs)
  IndexMap c_all;   // all C labels
  long long n;
  int nsrc;
  const void* A[kMaxAddSrc];
  int a_cplx[kMaxAddSrc];
  int a_f32[kMaxAddSrc];
  IndexMap a_all[kMaxAddSrc];   // C's labels, source s's strides (0 where the source lacks the label)
  double ar[kMaxAddSrc], ai[kMaxAddSrc];
};

// ---------------------------------------------------------------------------------------
// Kernel launchers (kernels.cu, gemm_tc.cu)
void launch_pack(const PackDesc& d, cudaStream_t s);
void launch_unpack(const UnpackDesc& d, cudaStream_t s);
void launch_direct(const DirectDesc& d, cudaStream_t s);
void launch_add(const AddDesc& d, cudaStream_t s);
void launch_gemm_f64(const double* A, const double* B, double* C, long long M, long long N,
                     long long Kpad, long long NB, cudaStream_t s);

// tcgen05 GEMM over operand planes.  The packed A holds planes (re/im x hi/lo) of M rows each,
// B planes of N rows; every row is Kpad elements (whole 128-byte K blocks).  Output plane rb
// (0 = real part, 1 = imaginary part) is  sum_s (-1)^neg_s A[planeA_s] B[planeB_s]^T, accumulated
// in TMEM and added (times a real alpha) straight into the strided float64 output tensor.
constexpr int kMaxSeg = 8;
struct TcSeg {
  int pa, pb, neg;
};
struct TcEpilogue {
  void* C;
  int c_cplx;
  int c_f32;           // float32 (complex64) output elements
  double alpha;
  IndexMap cm, cn, cb;
  int flat_n;          // 1: C offset of column n is rowoff + n * sn
  long long sn;
  int unit_n;          // 1: the output's unit stride runs along n (write through a shared-memory transpose)
  int store;           // 1: the output region is known to be zero: store instead of read-modify-write
  // pair-symmetric scatter: when ctab1 is set, column n goes to offset ctab1[n] and, when
  // ctab2[n] >= 0, sign2 times it to ctab2[n] (instead of the cn map)
  const long long* ctab1;
  const long long* ctab2;
  float sign2;
};
struct TcGemmParams {
  CUtensorMap tmA, tmB;
  CUtensorMap tmA2, tmB2;   // the same operands as boxes of two consecutive K blocks (4-D maps)
  int M, N, nkb;       // rows of one A plane, rows of one B plane, K blocks per plane
  int nrb;             // output planes
  int fused;           // 1: one work item covers both planes of a complex output (nseg[0] == nseg[1])
  int nseg[2];
  TcSeg seg[2][kMaxSeg];
  int vper;            // virtual K blocks (segments x nkb) per split
  int chunk;           // K blocks per accumulation chunk (0: one accumulation over the item's K loop)
  int nminor[2];       // leading segments of each output plane that hold a low-order split part
  int prefetch;        // L2 prefetch distance of the producer in K blocks (0: none)
  TcEpilogue epi;
  int* err;            // device error word
};
struct TcGemmPlan {
  TcGemmParams p;
  int kind;            // 0 tf32, 1 bf16
  int bn;              // N tile (64, 128 or 256)
  int variant;         // 0: default stages and epilogue warps for bn; 1: bn 128 with 6 stages and 4
                       // epilogue warps, or bn 256 with 3 stages and 8 epilogue warps; 2: two K
                       // blocks per pipeline stage (one TMA box each for A and B), bn 128 with 3
                       // stages or bn 256 with 2 stages, 4 epilogue warps (bn 64: as variant 0)
  bool pair_maps;      // the two-K-block tensor maps could be encoded (variant 2 usable)
  int splits;
  long long NB;
};
// bn: N tile to use (64, 128 or 256; 0 picks one from N); a tile the plan cannot use (256 for a
// both-plane item) falls back to the default choice.
// chunk > 0: the tensor cores accumulate at most `chunk` K blocks (of 128 bytes) in one float32
// accumulator; the chunks of an item are then summed with round-to-nearest float32 adds in the
// epilogue warps.  The tensor cores' float32 accumulation over a long K loop drifts (its rounding
// errors add up in one direction, about K/16 units in the last place for K products); summing
// short chunks keeps that drift to the chunk length.
void tc_gemm_plan(TcGemmPlan& pl, int kind, const void* A, int planesA, const void* B, int planesB, long long M,
                  long long N, long long Kpad, long long NB, int* err, int bn = 0, int chunk = 0);
void launch_tc_gemm(const TcGemmPlan& p, cudaStream_t s);
int tc_kblock_elems(int kind);   // K elements per 128-byte block: 32 (tf32) or 64 (bf16)
// Streaming multiprocessors of the current device (queried once per device; 152 on GB300).
// Grid sizes, split-K decisions and wave counts are all taken from this number.
int device_sm_count();

// 32-bit mixed-radix decode of one index group (extents < 2^31 per group).
__device__ __forceinline__ long long imap32(const IndexMap& m, unsigned idx) {
  long long off = 0;
  for (int d = m.n - 1; d >= 0; --d) {
    const unsigned dim = (unsigned)m.dims[d];
    const unsigned q = idx / dim;
    off += (long long)(idx - q * dim) * m.strides[d];
    idx = q;
  }
  return off;
}

// Same decode without the innermost label (the caller walks that one itself).
__device__ __forceinline__ long long imap32_outer(const IndexMap& m, unsigned idx) {
  long long off = 0;
  for (int d = m.n - 2; d >= 0; --d) {
    const unsigned dim = (unsigned)m.dims[d];
    const unsigned q = idx / dim;
    off += (long long)(idx - q * dim) * m.strides[d];
    idx = q;
  }
  return off;
}

// IEEE binary64 <-> binary32 conversions written with integer operations on the bit fields.
// Bandwidth-bound kernels use them so that they issue no instruction to the float64 pipe,
// which on this part runs at a small fraction of the float32 rate.
//
// binary64 -> binary32: the 52-bit significand is cut to 23 bits, rounding to nearest with
// ties away from zero (add half a unit in the last kept place, then truncate; a carry out of
// the significand moves into the exponent, which is the correctly rounded result).  Results
// below the smallest normal binary32 (2^-126) flush to signed zero; overflow gives infinity;
// NaN stays NaN.
__device__ __forceinline__ float f64_to_f32_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ahi = hi & 0x7fffffffu;
  // bits 31..23 = the low 9 exponent bits, 22..0 = the top 23 significand bits
  unsigned t = __funnelshift_l(lo, hi, 3);
  // for biased exponents 897..1150 the binary32 exponent (E - 896) is E's low 8 bits with the
  // top one flipped; adding the first dropped bit rounds (a carry moves into the exponent)
  t = ((t & 0x7fffffffu) ^ 0x40000000u) + ((lo >> 28) & 1u);
  if (ahi < 0x38100000u) {
    t = 0u;   // below 2^-126
  } else if (ahi >= 0x47f00000u) {
    t = (ahi > 0x7ff00000u || (ahi == 0x7ff00000u && lo != 0u)) ? 0x7fc00000u : 0x7f800000u;
  }
  return __uint_as_float(t | (hi & 0x80000000u));
}

// binary32 -> binary64, exact (subnormal inputs are normalised).
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned long long bits;
  if (e == 0xffu) {
    bits = (0x7ffull << 52) | ((unsigned long long)m << 29);
  } else if (e != 0u) {
    bits = ((unsigned long long)(e + 1023 - 127) << 52) | ((unsigned long long)m << 29);
  } else if (m != 0u) {
    const int p = 31 - __clz((int)m);   // value = m * 2^-149 = 1.f * 2^(p - 149)
    bits = ((unsigned long long)(p - 149 + 1023) << 52) | (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
  } else {
    bits = 0;
  }
  return __longlong_as_double((long long)(bits | sign));
}

}  // namespace rtcc
