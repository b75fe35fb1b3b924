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
struct PackDesc {
  const double* src;
  int src_cplx;
  IndexMap rows;    // R labels
  IndexMap cols;    // K labels
  IndexMap bat;     // batch labels
  long long R, K, NB;
  int nrb, ncs, nss;
  int comp[2][2];   // 0 = re, 1 = im
  int sign[2][2];
  int part[3];
  long long Kpad;   // padded row length of the packed matrix
  int elem;         // PackElem
  int round_tf32;   // round float32 values to TF32 (round-to-nearest) when packing
  int transpose;    // 1: the source's unit-stride index is a row index (shared-memory tile transpose)
  void* dst;
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
  const double* A; const double* B; double* C;
  int a_cplx, b_cplx, c_cplx;
  IndexMap am, ak, ab, bn, bk, bb, cm, cn, cb;
  long long M, N, K, NB;
  double ar, ai;
};

// C[lc] += alpha * A[la] with labels(A) a subset of labels(C) (broadcast over the rest).
struct AddDesc {
  const double* A; double* C;
  int a_cplx, c_cplx;
  IndexMap c_all;   // all C labels
  IndexMap a_all;   // same labels, A's strides (0 where A lacks the label)
  long long n;
  double ar, ai;
};

// ---------------------------------------------------------------------------------------
// Kernel launchers (kernels.cu, gemm_tc.cu)
void launch_pack(const PackDesc& d, cudaStream_t s);
void launch_unpack(const UnpackDesc& d, cudaStream_t s);
void launch_direct(const DirectDesc& d, cudaStream_t s);
void launch_add(const AddDesc& d, cudaStream_t s);
void launch_gemm_f64(const double* A, const double* B, double* C, long long M, long long N,
                     long long Kpad, long long NB, cudaStream_t s);

// tcgen05 GEMM: C[b][m][n] = sum_k A[b][m][k] B[b][n][k], A/B packed (float32 as TF32 or bf16),
// rows padded to Kpad (multiple of the 128-byte K block).  C float32 row-major [NB][M][N].
struct TcGemmPlan {
  CUtensorMap tmA, tmB;
  int kind;        // 0 tf32, 1 bf16
  int bn;          // N tile (64, 128 or 256)
  long long M, N, Kpad, NB;
  float* C;
  int* err;        // device error word
};
void tc_gemm_plan(TcGemmPlan& p, int kind, const void* A, const void* B, float* C, long long M,
                  long long N, long long Kpad, long long NB, int* err);
void launch_tc_gemm(const TcGemmPlan& p, cudaStream_t s);
int tc_kblock_elems(int kind);   // K elements per 128-byte block: 32 (tf32) or 64 (bf16)

}  // namespace rtcc
