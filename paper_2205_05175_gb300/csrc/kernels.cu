// Layout and small-contraction kernels of the contraction engine:
//   pack    : strided float64 tensor (real or complex) -> K-major GEMM operand
//             (float32 rounded to TF32, bf16, or float64), with re/im stacking, the
//             [[Ar,-Ai],[Ai,Ar]] complex embedding and hi/lo precision splits
//   unpack  : GEMM output -> C[...] += alpha * (re + i im) at strided positions
//   direct  : C[...] += alpha * sum_k A B for small contractions, float64 throughout
//   add     : C[...] += alpha * A[...] (permute / broadcast)
//   dgemm   : float64 SIMT GEMM for the float64 precision mode
#include "common.cuh"
#include <cuda_bf16.h>

namespace rtcc {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n, int threads = kThreads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152ll * 64) b = 152ll * 64;   // grid-stride beyond 64 blocks per SM
  if (b < 1) b = 1;
  return (unsigned)b;
}

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void pack_kernel(PackDesc d) {
  const long long rows = (long long)d.nrb * d.R;
  const long long total = d.NB * rows * d.Kpad;
  const long long segK = (long long)d.ncs * d.K;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long kk = idx % d.Kpad;
    const long long t = idx / d.Kpad;
    const long long r = t % rows;
    const long long bt = t / rows;
    double x = 0.0;
    int part = SP_FULL;
    if (kk < d.nss * segK) {
      const int ss = (int)(kk / segK);
      const long long rem = kk - ss * segK;
      const int cs = (int)(rem / d.K);
      const long long k = rem - cs * d.K;
      const int rb = (int)(r / d.R);
      const long long m = r - rb * d.R;
      const long long off = imap_offset(d.bat, bt) + imap_offset(d.rows, m) + imap_offset(d.cols, k);
      const int comp = d.comp[rb][cs];
      if (d.src_cplx) x = d.src[2 * off + comp];
      else x = (comp == 0) ? d.src[off] : 0.0;
      x *= (double)d.sign[rb][cs];
      part = d.part[ss];
    }
    if (d.elem == PE_F64) {
      static_cast<double*>(d.dst)[idx] = x;
    } else if (d.elem == PE_F32) {
      float v;
      if (part == SP_FULL) v = d.round_tf32 ? tf32_rn((float)x) : (float)x;
      else {
        const float hi = tf32_rn((float)x);
        v = (part == SP_HI) ? hi : tf32_rn((float)(x - (double)hi));
      }
      static_cast<float*>(d.dst)[idx] = v;
    } else {
      __nv_bfloat16 v;
      if (part == SP_FULL) v = __float2bfloat16_rn((float)x);
      else {
        const __nv_bfloat16 hi = __float2bfloat16_rn((float)x);
        v = (part == SP_HI) ? hi : __float2bfloat16_rn((float)(x - (double)__bfloat162float(hi)));
      }
      static_cast<__nv_bfloat16*>(d.dst)[idx] = v;
    }
  }
}

__global__ void unpack_kernel(UnpackDesc d) {
  const long long total = d.NB * d.M * d.N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long n = idx % d.N;
    const long long t = idx / d.N;
    const long long m = t % d.M;
    const long long bt = t / d.M;
    const long long gb = bt * d.rows_g * d.ldg;
    long long ire = gb + m * d.ldg + n, iim = -1;
    if (d.mode == OM_STACK_M) iim = gb + (m + d.M) * d.ldg + n;
    else if (d.mode == OM_STACK_N) iim = gb + m * d.ldg + n + d.N;
    double re, im = 0.0;
    if (d.gout_f64) {
      const double* g = static_cast<const double*>(d.gout);
      re = g[ire];
      if (iim >= 0) im = g[iim];
    } else {
      const float* g = static_cast<const float*>(d.gout);
      re = (double)g[ire];
      if (iim >= 0) im = (double)g[iim];
    }
    const long long off = imap_offset(d.cb, bt) + imap_offset(d.cm, m) + imap_offset(d.cn, n);
    const double vr = d.ar * re - d.ai * im;
    const double vi = d.ar * im + d.ai * re;
    if (d.c_cplx) {
      d.C[2 * off] += vr;
      d.C[2 * off + 1] += vi;
    } else {
      d.C[off] += vr;
    }
  }
}

__global__ void direct_kernel(DirectDesc d) {
  const long long total = d.NB * d.M * d.N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long n = idx % d.N;
    const long long t = idx / d.N;
    const long long m = t % d.M;
    const long long bt = t / d.M;
    const long long a0 = imap_offset(d.ab, bt) + imap_offset(d.am, m);
    const long long b0 = imap_offset(d.bb, bt) + imap_offset(d.bn, n);
    int ctr[kMaxLab];
    for (int q = 0; q < kMaxLab; ++q) ctr[q] = 0;
    long long ao = 0, bo = 0;
    double sr = 0.0, si = 0.0;
    for (long long k = 0; k < d.K; ++k) {
      double ar_, ai_ = 0.0, br_, bi_ = 0.0;
      if (d.a_cplx) { ar_ = d.A[2 * (a0 + ao)]; ai_ = d.A[2 * (a0 + ao) + 1]; }
      else ar_ = d.A[a0 + ao];
      if (d.b_cplx) { br_ = d.B[2 * (b0 + bo)]; bi_ = d.B[2 * (b0 + bo) + 1]; }
      else br_ = d.B[b0 + bo];
      sr += ar_ * br_ - ai_ * bi_;
      si += ar_ * bi_ + ai_ * br_;
      for (int q = d.ak.n - 1; q >= 0; --q) {
        ++ctr[q];
        ao += d.ak.strides[q];
        bo += d.bk.strides[q];
        if (ctr[q] < d.ak.dims[q]) break;
        ao -= (long long)d.ak.dims[q] * d.ak.strides[q];
        bo -= (long long)d.bk.dims[q] * d.bk.strides[q];
        ctr[q] = 0;
      }
    }
    const long long off = imap_offset(d.cb, bt) + imap_offset(d.cm, m) + imap_offset(d.cn, n);
    const double vr = d.ar * sr - d.ai * si;
    const double vi = d.ar * si + d.ai * sr;
    if (d.c_cplx) {
      d.C[2 * off] += vr;
      d.C[2 * off + 1] += vi;
    } else {
      d.C[off] += vr;
    }
  }
}

__global__ void add_kernel(AddDesc d) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < d.n;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long co = imap_offset(d.c_all, idx);
    const long long ao = imap_offset(d.a_all, idx);
    double xr, xi = 0.0;
    if (d.a_cplx) { xr = d.A[2 * ao]; xi = d.A[2 * ao + 1]; }
    else xr = d.A[ao];
    const double vr = d.ar * xr - d.ai * xi;
    const double vi = d.ar * xi + d.ai * xr;
    if (d.c_cplx) {
      d.C[2 * co] += vr;
      d.C[2 * co + 1] += vi;
    } else {
      d.C[co] += vr;
    }
  }
}

// Split-K reduction for contractions with few outputs and a long K (dot products):
// block (output, split) sums its K range and adds alpha * sum atomically.
__global__ void reduce_kernel(DirectDesc d, long long chunk) {
  const long long o = blockIdx.x;
  const long long n = o % d.N;
  const long long t = o / d.N;
  const long long m = t % d.M;
  const long long bt = t / d.M;
  const long long a0 = imap_offset(d.ab, bt) + imap_offset(d.am, m);
  const long long b0 = imap_offset(d.bb, bt) + imap_offset(d.bn, n);
  const long long k0 = (long long)blockIdx.y * chunk;
  const long long k1 = min(d.K, k0 + chunk);
  double sr = 0.0, si = 0.0;
  for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const long long ao = a0 + imap_offset(d.ak, k), bo = b0 + imap_offset(d.bk, k);
    double ar_, ai_ = 0.0, br_, bi_ = 0.0;
    if (d.a_cplx) { ar_ = d.A[2 * ao]; ai_ = d.A[2 * ao + 1]; }
    else ar_ = d.A[ao];
    if (d.b_cplx) { br_ = d.B[2 * bo]; bi_ = d.B[2 * bo + 1]; }
    else br_ = d.B[bo];
    sr += ar_ * br_ - ai_ * bi_;
    si += ar_ * bi_ + ai_ * br_;
  }
  __shared__ double shr[32], shi[32];
  for (int off = 16; off > 0; off >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, off);
    si += __shfl_down_sync(0xffffffffu, si, off);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { shr[w] = sr; shi[w] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    sr = 0.0; si = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { sr += shr[q]; si += shi[q]; }
    const long long off = imap_offset(d.cb, bt) + imap_offset(d.cm, m) + imap_offset(d.cn, n);
    const double vr = d.ar * sr - d.ai * si, vi = d.ar * si + d.ai * sr;
    if (d.c_cplx) { atomicAdd(&d.C[2 * off], vr); atomicAdd(&d.C[2 * off + 1], vi); }
    else atomicAdd(&d.C[off], vr);
  }
}

// float64 SIMT GEMM: 64x64 tile, 16-deep K slices, 256 threads with 4x4 outputs each.
__global__ void __launch_bounds__(256) dgemm_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                                    double* __restrict__ C, int M, int N, int K) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const size_t bz = blockIdx.z;
  A += bz * (size_t)M * K;
  B += bz * (size_t)N * K;
  C += bz * (size_t)M * N;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + q * 256;
      const int r = e >> 4, c = e & 15;
      As[c][r] = (m0 + r < M && k0 + c < K) ? A[(size_t)(m0 + r) * K + k0 + c] : 0.0;
      Bs[c][r] = (n0 + r < N && k0 + c < K) ? B[(size_t)(n0 + r) * K + k0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n < N) C[(size_t)m * N + n] = acc[i][j];
    }
  }
}

}  // namespace

void launch_pack(const PackDesc& d, cudaStream_t s) {
  const long long total = d.NB * (long long)d.nrb * d.R * d.Kpad;
  if (total == 0) return;
  pack_kernel<<<grid_for(total), kThreads, 0, s>>>(d);
  RTCC_CUDA(cudaGetLastError());
}
void launch_unpack(const UnpackDesc& d, cudaStream_t s) {
  const long long total = d.NB * d.M * d.N;
  if (total == 0) return;
  unpack_kernel<<<grid_for(total), kThreads, 0, s>>>(d);
  RTCC_CUDA(cudaGetLastError());
}
void launch_direct(const DirectDesc& d, cudaStream_t s) {
  const long long total = d.NB * d.M * d.N;
  if (total == 0) return;
  direct_kernel<<<grid_for(total, 128), 128, 0, s>>>(d);
  RTCC_CUDA(cudaGetLastError());
}
void launch_reduce(const DirectDesc& d, long long splits, cudaStream_t s) {
  const long long nout = d.NB * d.M * d.N;
  if (nout == 0) return;
  const long long chunk = (d.K + splits - 1) / splits;
  dim3 grid((unsigned)nout, (unsigned)splits);
  reduce_kernel<<<grid, 256, 0, s>>>(d, chunk);
  RTCC_CUDA(cudaGetLastError());
}
void launch_add(const AddDesc& d, cudaStream_t s) {
  if (d.n == 0) return;
  add_kernel<<<grid_for(d.n), kThreads, 0, s>>>(d);
  RTCC_CUDA(cudaGetLastError());
}
void launch_gemm_f64(const double* A, const double* B, double* C, long long M, long long N, long long Kpad,
                     long long NB, cudaStream_t s) {
  RTCC_REQUIRE(M < (1ll << 31) && N < (1ll << 31) && Kpad < (1ll << 31) && NB < 65536, "GEMM extents too large");
  dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64), (unsigned)NB);
  dgemm_kernel<<<grid, 256, 0, s>>>(A, B, C, (int)M, (int)N, (int)Kpad);
  RTCC_CUDA(cudaGetLastError());
}

}  // namespace rtcc
