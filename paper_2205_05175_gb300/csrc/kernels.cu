// Layout and small-contraction kernels of the contraction engine.  Tensors hold float64
// (complex128) or, for the temporaries of reduced-precision engines, float32 (complex64)
// elements; reduced-precision programs compute in float32 with integer-rounded operands.
//   pack    : strided tensor (real or complex) -> K-major GEMM operand (float32 rounded to
//             TF32, bf16, or float64), with re/im planes, hi/lo precision splits, the
//             [[Ar,-Ai],[Ai,Ar]] complex embedding of the float64 path, and gather tables for
//             the pair-symmetric contraction
//   unpack  : float64 GEMM output -> C[...] += alpha * (re + i im) at strided positions
//   direct  : C[...] (+)= alpha * sum_k A B for small contractions and outer products
//   reduce  : few outputs, long K: split-K block reduction (float64) or the staged
//             shared-memory reduction (float32, 2 x 2 outputs per thread)
//   skinny  : short K and few columns over many rows: one thread per row
//   add     : C[...] (+)= sum_s alpha_s * A_s[...] (permute / broadcast, up to four sources)
//   dgemm   : float64 SIMT GEMM for the float64 precision mode
#include "common.cuh"
#include <cuda_bf16.h>
#include <algorithm>
#include <type_traits>

namespace rtcc {

int device_sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 152;
    }
    cache[dev] = n;
  }
  return cache[dev];
}

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n, int threads = kThreads) {
  long long b = (n + threads - 1) / threads;
  const long long cap = (long long)device_sm_count() * 64;   // grid-stride beyond 64 blocks per SM
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <typename R>
__device__ __forceinline__ R cvt_r(double x) {
  if constexpr (std::is_same<R, float>::value) return f64_to_f32_bits(x);
  else return x;
}
__device__ __forceinline__ double cvt_d(float x) { return f32_to_f64_bits(x); }
__device__ __forceinline__ double cvt_d(double x) { return x; }
__device__ __forceinline__ float cvt_f(float x) { return x; }
__device__ __forceinline__ float cvt_f(double x) { return f64_to_f32_bits(x); }
template <typename R>
__device__ __forceinline__ R from_f(float x) {
  if constexpr (std::is_same<R, float>::value) return x;
  else return f32_to_f64_bits(x);
}

// Element access to a tensor of float64 or float32 (complex128 / complex64) elements; values
// move between the two widths with the integer conversions above (no float64 instructions).
template <typename R>
__device__ __forceinline__ void ld_elem(const void* p, long long i, int cplx, int f32, R& re, R& im) {
  if (f32) {
    if (cplx) {
      const float2 x = reinterpret_cast<const float2*>(p)[i];
      re = from_f<R>(x.x);
      im = from_f<R>(x.y);
    } else {
      re = from_f<R>(reinterpret_cast<const float*>(p)[i]);
      im = 0;
    }
  } else {
    if (cplx) {
      const double2 x = reinterpret_cast<const double2*>(p)[i];
      re = cvt_r<R>(x.x);
      im = cvt_r<R>(x.y);
    } else {
      re = cvt_r<R>(reinterpret_cast<const double*>(p)[i]);
      im = 0;
    }
  }
}
template <typename R>
__device__ __forceinline__ void st_elem(void* p, long long i, int cplx, int f32, R re, R im) {
  if (f32) {
    if (cplx) reinterpret_cast<float2*>(p)[i] = make_float2(cvt_f(re), cvt_f(im));
    else reinterpret_cast<float*>(p)[i] = cvt_f(re);
  } else {
    if (cplx) reinterpret_cast<double2*>(p)[i] = make_double2(cvt_d(re), cvt_d(im));
    else reinterpret_cast<double*>(p)[i] = cvt_d(re);
  }
}

template <int ELEM>
__device__ __forceinline__ void put(void* dst, size_t i, double x, int part, int round_tf32) {
  if constexpr (ELEM == PE_F64) {
    static_cast<double*>(dst)[i] = x;
  } else if constexpr (ELEM == PE_F32) {
    float v;
    if (part == SP_FULL) v = round_tf32 ? tf32_rn((float)x) : (float)x;
    else {
      const float hi = tf32_rn((float)x);
      v = (part == SP_HI) ? hi : tf32_rn((float)(x - (double)hi));
    }
    static_cast<float*>(dst)[i] = v;
  } else {
    __nv_bfloat16 v;
    if (part == SP_FULL) v = __float2bfloat16_rn((float)x);
    else {
      const __nv_bfloat16 hi = __float2bfloat16_rn((float)x);
      v = (part == SP_HI) ? hi : __float2bfloat16_rn((float)(x - (double)__bfloat162float(hi)));
    }
    static_cast<__nv_bfloat16*>(dst)[i] = v;
  }
}

// Write one source element (xr, xi) to every destination it feeds: row blocks rb (re/im
// stacking or the [[Ar,-Ai],[Ai,Ar]] embedding), column segments cs, precision parts ss.
template <int ELEM>
__device__ __forceinline__ void pack_store(const PackDesc& d, unsigned bt, unsigned m, unsigned k, double xr,
                                           double xi) {
  const size_t GR = (size_t)d.nrb * d.R;
  const size_t K = (size_t)d.K;
#pragma unroll 1
  for (int rb = 0; rb < d.nrb; ++rb) {
    const size_t rowbase = ((size_t)bt * GR + (size_t)rb * d.R + m) * (size_t)d.Kpad;
#pragma unroll 1
    for (int cs = 0; cs < d.ncs; ++cs) {
      const double x = (d.comp[rb][cs] ? xi : xr) * (double)d.sign[rb][cs];
#pragma unroll 1
      for (int ss = 0; ss < d.nss; ++ss)
        put<ELEM>(d.dst, rowbase + ((size_t)ss * d.ncs + cs) * K + k, x, d.nss > 1 ? d.part[ss] : d.rb_part[rb],
                  d.round_tf32);
    }
  }
}

template <int ELEM>
__device__ __forceinline__ void pack_pad(const PackDesc& d, unsigned bt, unsigned m, unsigned p) {
  const size_t GR = (size_t)d.nrb * d.R;
  const size_t c0 = (size_t)d.nss * d.ncs * d.K;
  for (int rb = 0; rb < d.nrb; ++rb)
    put<ELEM>(d.dst, ((size_t)bt * GR + (size_t)rb * d.R + m) * (size_t)d.Kpad + c0 + p, 0.0, SP_FULL, 0);
}

// Source unit stride along K: a row per thread-row, consecutive k per thread.
template <int ELEM>
__global__ void pack_direct_kernel(PackDesc d, unsigned kext, unsigned padw) {
  const unsigned R = (unsigned)d.R, K = (unsigned)d.K;
  const unsigned NR = (unsigned)(d.NB * d.R);
  for (unsigned row = blockIdx.y * blockDim.y + threadIdx.y; row < NR; row += gridDim.y * blockDim.y) {
    const unsigned bt = row / R, m = row - bt * R;
    const long long base = imap32(d.bat, bt) + imap32(d.rows, m);
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < kext; k += gridDim.x * blockDim.x) {
      if (k < K) {
        const long long off = base + imap32(d.cols, k);
        double xr, xi = 0.0;
        if (d.src_cplx) {
          const double2 v = reinterpret_cast<const double2*>(d.src)[off];
          xr = v.x;
          xi = v.y;
        } else {
          xr = static_cast<const double*>(d.src)[off];
        }
        pack_store<ELEM>(d, bt, m, k, xr, xi);
      } else if (k - K < padw) {
        pack_pad<ELEM>(d, bt, m, k - K);
      }
    }
  }
}

// Source unit stride along a row index: 32 x 32 tiles through shared memory (coalesced both ways).
template <int ELEM>
__global__ void __launch_bounds__(256) pack_transpose_kernel(PackDesc d, unsigned padw) {
  __shared__ double tre[32][33], tim[32][33];
  const unsigned R = (unsigned)d.R, K = (unsigned)d.K;
  const unsigned NR = (unsigned)(d.NB * d.R);
  const unsigned nkt = (K + 31) / 32, nrt = (NR + 31) / 32;
  const unsigned tx = threadIdx.x, ty = threadIdx.y;
  for (unsigned rt = blockIdx.y; rt < nrt; rt += gridDim.y) {
    for (unsigned kt = blockIdx.x; kt < nkt + (padw ? 1u : 0u); kt += gridDim.x) {
      const unsigned r0 = rt * 32, k0 = kt * 32;
      if (kt == nkt) {
        for (int i = 0; i < 4; ++i) {
          const unsigned row = r0 + ty + 8 * i;
          if (row >= NR) continue;
          const unsigned bt = row / R, m = (unsigned)imap32(d.rd_dst, row - bt * R);
          for (unsigned p = tx; p < padw; p += 32) pack_pad<ELEM>(d, bt, m, p);
        }
        continue;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const unsigned k = k0 + ty + 8 * i, row = r0 + tx;
        double xr = 0.0, xi = 0.0;
        if (row < NR && k < K) {
          const unsigned bt = row / R, mr = row - bt * R;
          const long long off = imap32(d.bat, bt) + imap32(d.rd_src, mr) + imap32(d.cols, k);
          if (d.src_cplx) {
            const double2 v = reinterpret_cast<const double2*>(d.src)[off];
            xr = v.x;
            xi = v.y;
          } else {
            xr = static_cast<const double*>(d.src)[off];
          }
        }
        tre[ty + 8 * i][tx] = xr;
        tim[ty + 8 * i][tx] = xi;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const unsigned row = r0 + ty + 8 * i, k = k0 + tx;
        if (row < NR && k < K) {
          const unsigned bt = row / R, mr = row - bt * R;
          const unsigned m = (unsigned)imap32(d.rd_dst, mr);
          pack_store<ELEM>(d, bt, m, k, tre[tx][ty + 8 * i], tim[tx][ty + 8 * i]);
        }
      }
      __syncthreads();
    }
  }
}

// ---- plane packs (tensor-core operands): planes = components (re, im) x split parts (hi, lo) ----
template <int ELEM>
struct Vec4;
template <>
struct Vec4<PE_F32> {
  using T = float4;
};
template <>
struct Vec4<PE_BF16> {
  using T = uint2;
};

// One split part of a value already rounded to binary32: hi = x rounded to the plane type,
// lo = x - hi (exact in binary32; the bf16 store rounds it).  The residual of the binary64 ->
// binary32 rounding (2^-24 relative) is far below what the hi/lo pair resolves.
template <int ELEM>
__device__ __forceinline__ float part_value(float x, int part) {
  if constexpr (ELEM == PE_F32) {
    const float hi = tf32_rn(x);
    return part == SP_LO ? tf32_rn(x - hi) : hi;
  } else {
    const float hi = __bfloat162float(__float2bfloat16_rn(x));
    return part == SP_LO ? x - hi : hi;
  }
}

template <int ELEM>
__device__ __forceinline__ void store4(void* dst, size_t idx, float a, float b, float c, float d) {
  if constexpr (ELEM == PE_F32) {
    *reinterpret_cast<float4*>(static_cast<float*>(dst) + idx) = make_float4(a, b, c, d);
  } else {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    uint2 v;
    v.x = *reinterpret_cast<uint32_t*>(&lo);
    v.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(dst) + idx) = v;
  }
}

template <int ELEM>
__device__ __forceinline__ void store2(void* dst, size_t idx, float a, float b) {
  if constexpr (ELEM == PE_F32) {
    *reinterpret_cast<float2*>(static_cast<float*>(dst) + idx) = make_float2(a, b);
  } else {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(dst) + idx) = v;
  }
}

// Source unit stride along K: 4 consecutive k per thread (their source offsets decoded once),
// rows in tiles of 32 whose offsets are decoded once per tile into shared memory.
template <int ELEM>
__global__ void __launch_bounds__(256) pack_planes_direct_kernel(PackDesc d) {
  constexpr int RT = 32;
  __shared__ long long s_src[RT];
  __shared__ unsigned long long s_dst[RT];   // packed element index of (row, plane 0, k = 0)
  const unsigned R = (unsigned)d.R, K = (unsigned)d.K, Kp = (unsigned)d.Kpad;
  const unsigned NR = (unsigned)(d.NB * d.R);
  const unsigned nrt = (NR + RT - 1) / RT;
  const unsigned tid = threadIdx.y * blockDim.x + threadIdx.x;
  const unsigned k4 = 4u * (blockIdx.x * blockDim.x + threadIdx.x);
  const bool kok = k4 < Kp;
  long long coff[4], coff2[4];
  float kwt[4];
  bool kv[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    kv[j] = k4 + j < K;
    coff[j] = 0;
    coff2[j] = -1;
    kwt[j] = 1.f;
    if (kv[j]) {
      if (d.ktab) {
        coff[j] = d.ktab[2 * (k4 + j)];
        coff2[j] = d.ktab[2 * (k4 + j) + 1];
        if (d.kw) kwt[j] = d.kw[k4 + j];
      } else {
        coff[j] = imap32(d.cols, k4 + j);
      }
    }
  }
  const int np = d.nrb;
  const unsigned long long pstride = (unsigned long long)R * Kp;   // plane stride in elements
  for (unsigned rt = blockIdx.y; rt < nrt; rt += gridDim.y) {
    __syncthreads();
    if (tid < RT) {
      const unsigned row = rt * RT + tid;
      if (row < NR) {
        const unsigned bt = row / R, m = row - bt * R;
        s_src[tid] = imap32(d.bat, bt) + (d.rtab ? d.rtab[m] : imap32(d.rows, m));
        s_dst[tid] = ((unsigned long long)bt * np * R + m) * Kp;
      }
    }
    __syncthreads();
    if (!kok) continue;
    const unsigned nrows = min((unsigned)RT, NR - rt * RT);
    for (unsigned r = threadIdx.y; r < nrows; r += blockDim.y) {
      const long long base = s_src[r];
      float xr[4], xi[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        xr[j] = 0.f;
        xi[j] = 0.f;
        if (kv[j]) {
          ld_elem<float>(d.src, base + coff[j], d.src_cplx, d.src_f32, xr[j], xi[j]);
          if (coff2[j] >= 0) {
            float yr, yi;
            ld_elem<float>(d.src, base + coff2[j], d.src_cplx, d.src_f32, yr, yi);
            xr[j] = kwt[j] * (xr[j] + d.ksign * yr);
            xi[j] = kwt[j] * (xi[j] + d.ksign * yi);
          }
        }
      }
      const unsigned long long drow = s_dst[r] + k4;
      for (int pl = 0; pl < np; ++pl) {
        const int part = d.rb_part[pl];
        const bool im = d.comp[pl][0] != 0;
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = part_value<ELEM>(im ? xi[j] : xr[j], part);
        store4<ELEM>(d.dst, drow + pl * pstride, o[0], o[1], o[2], o[3]);
      }
    }
  }
}

// Source unit stride along a row label: 32 read-order rows x 64 k per tile through shared memory,
// with the tile's k offsets and row offsets decoded once into shared memory; the store phase
// writes 2 consecutive k per thread (a warp covers 64 k of one row).
template <int ELEM>
__global__ void __launch_bounds__(256) pack_planes_transpose_kernel(PackDesc d) {
  __shared__ float2 tl[64][33];
  __shared__ long long s_k[64];
  __shared__ long long s_src[32];
  __shared__ unsigned long long s_dst[32];
  const unsigned R = (unsigned)d.R, K = (unsigned)d.K, Kp = (unsigned)d.Kpad;
  const unsigned NR = (unsigned)(d.NB * d.R);
  const unsigned nkt = (Kp + 63) / 64, nrt = (NR + 31) / 32;
  const unsigned tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int np = d.nrb;
  const unsigned long long pstride = (unsigned long long)R * Kp;
  for (unsigned rt = blockIdx.y; rt < nrt; rt += gridDim.y) {
    const unsigned r0 = rt * 32;
    __syncthreads();
    if (tid < 32) {
      const unsigned row = r0 + tid;
      long long src = -1;
      unsigned long long dst = 0;
      if (row < NR) {
        const unsigned bt = row / R, mr = row - bt * R;
        src = imap32(d.bat, bt) + imap32(d.rd_src, mr);
        dst = ((unsigned long long)bt * np * R + (unsigned)imap32(d.rd_dst, mr)) * Kp;
      }
      s_src[tid] = src;
      s_dst[tid] = dst;
    }
    for (unsigned kt = blockIdx.x; kt < nkt; kt += gridDim.x) {
      const unsigned k0 = kt * 64;
      if (tid >= 64 && tid < 128) {
        const unsigned k = k0 + tid - 64;
        s_k[tid - 64] = (k < K) ? imap32(d.cols, k) : -1;
      }
      __syncthreads();
      {
        const long long rbase = s_src[tx];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const long long ko = s_k[ty + 8 * i];
          float2 v = make_float2(0.f, 0.f);
          if (rbase >= 0 && ko >= 0) ld_elem<float>(d.src, rbase + ko, d.src_cplx, d.src_f32, v.x, v.y);
          tl[ty + 8 * i][tx] = v;
        }
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const unsigned r = ty + 8 * i, kk = 2 * tx, k = k0 + kk;
        if (r0 + r < NR && k < Kp) {
          const unsigned long long drow = s_dst[r] + k;
          const float2 v0 = tl[kk][r], v1 = tl[kk + 1][r];
          for (int pl = 0; pl < np; ++pl) {
            const int part = d.rb_part[pl];
            const bool im = d.comp[pl][0] != 0;
            const float a = part_value<ELEM>(im ? v0.y : v0.x, part);
            const float b = part_value<ELEM>(im ? v1.y : v1.x, part);
            store2<ELEM>(d.dst, drow + pl * pstride, a, b);
          }
        }
      }
      __syncthreads();
    }
  }
}

template <typename G>
__device__ __forceinline__ void unpack_one(const UnpackDesc& d, const G* g, unsigned bt, unsigned m, unsigned n,
                                           long long off) {
  const size_t gb = (size_t)bt * (size_t)d.rows_g * (size_t)d.ldg;
  double re = (double)g[gb + (size_t)m * d.ldg + n], im = 0.0;
  if (d.mode == OM_STACK_M) im = (double)g[gb + ((size_t)m + d.M) * d.ldg + n];
  else if (d.mode == OM_STACK_N) im = (double)g[gb + (size_t)m * d.ldg + n + d.N];
  const double vr = d.ar * re - d.ai * im, vi = d.ar * im + d.ai * re;
  if (d.c_cplx) {
    double2* c = reinterpret_cast<double2*>(d.C) + off;
    double2 x = *c;
    x.x += vr;
    x.y += vi;
    *c = x;
  } else {
    d.C[off] += vr;
  }
}

template <typename G>
__global__ void unpack_direct_kernel(UnpackDesc d) {
  const G* g = static_cast<const G*>(d.gout);
  const unsigned M = (unsigned)d.M, N = (unsigned)d.N;
  const unsigned NR = (unsigned)(d.NB * d.M);
  for (unsigned row = blockIdx.y * blockDim.y + threadIdx.y; row < NR; row += gridDim.y * blockDim.y) {
    const unsigned bt = row / M, m = row - bt * M;
    const long long base = imap32(d.cb, bt) + imap32(d.cm, m);
    for (unsigned n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x)
      unpack_one<G>(d, g, bt, m, n, base + imap32(d.cn, n));
  }
}

// Output unit stride along an M index: read GEMM tiles along n, write along m.
template <typename G>
__global__ void __launch_bounds__(256) unpack_transpose_kernel(UnpackDesc d) {
  __shared__ double tre[32][33], tim[32][33];
  const G* g = static_cast<const G*>(d.gout);
  const unsigned M = (unsigned)d.M, N = (unsigned)d.N;
  const unsigned NR = (unsigned)(d.NB * d.M);
  const unsigned nnt = (N + 31) / 32, nrt = (NR + 31) / 32;
  const unsigned tx = threadIdx.x, ty = threadIdx.y;
  for (unsigned rt = blockIdx.y; rt < nrt; rt += gridDim.y) {
    for (unsigned nt = blockIdx.x; nt < nnt; nt += gridDim.x) {
      const unsigned r0 = rt * 32, n0 = nt * 32;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const unsigned row = r0 + ty + 8 * i, n = n0 + tx;
        double re = 0.0, im = 0.0;
        if (row < NR && n < N) {
          const unsigned bt = row / M, m = row - bt * M;
          const size_t gb = (size_t)bt * (size_t)d.rows_g * (size_t)d.ldg;
          re = (double)g[gb + (size_t)m * d.ldg + n];
          if (d.mode == OM_STACK_M) im = (double)g[gb + ((size_t)m + M) * d.ldg + n];
          else if (d.mode == OM_STACK_N) im = (double)g[gb + (size_t)m * d.ldg + n + N];
        }
        tre[ty + 8 * i][tx] = re;
        tim[ty + 8 * i][tx] = im;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const unsigned n = n0 + ty + 8 * i, row = r0 + tx;
        if (row < NR && n < N) {
          const unsigned bt = row / M, m = row - bt * M;
          const long long off = imap32(d.cb, bt) + imap32(d.cm, m) + imap32(d.cn, n);
          const double re = tre[tx][ty + 8 * i], im = tim[tx][ty + 8 * i];
          const double vr = d.ar * re - d.ai * im, vi = d.ar * im + d.ai * re;
          if (d.c_cplx) {
            double2* c = reinterpret_cast<double2*>(d.C) + off;
            double2 x = *c;
            x.x += vr;
            x.y += vi;
            *c = x;
          } else {
            d.C[off] += vr;
          }
        }
      }
      __syncthreads();
    }
  }
}

// rows (bt, m) over blockIdx.y/threadIdx.y, n over x; K walked with an odometer (no divisions)
// F32: operands rounded to binary32 with integer operations and products summed in float32
// (reduced-precision programs, whose contractions resolve far less than 2^-24); otherwise
// float64 throughout.
template <bool F32>
__global__ void __launch_bounds__(128) direct_kernel(DirectDesc d) {
  using R = typename std::conditional<F32, float, double>::type;
  constexpr int RB = 32;   // rows per tile: their offsets are decoded once into shared memory
  __shared__ long long s_a[RB], s_b[RB], s_c[RB];
  const unsigned M = (unsigned)d.M, N = (unsigned)d.N;
  const unsigned NR = (unsigned)(d.NB * d.M);
  const unsigned nrt = (NR + RB - 1) / RB;
  const unsigned tid = threadIdx.y * blockDim.x + threadIdx.x;
  const R ar = (R)d.ar, ai = (R)d.ai;
  const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
  const bool col_ok = n < N;
  const long long bn_off = col_ok ? imap32(d.bn, n) : 0, cn_off = col_ok ? imap32(d.cn, n) : 0;
  for (unsigned rt = blockIdx.y; rt < nrt; rt += gridDim.y) {
    const unsigned r0 = rt * RB;
    __syncthreads();
    if (tid < RB) {
      const unsigned row = r0 + tid;
      long long a = 0, b = 0, c = 0;
      if (row < NR) {
        const unsigned bt = row / M, m = row - bt * M;
        a = imap32(d.ab, bt) + imap32(d.am, m);
        b = imap32(d.bb, bt);
        c = imap32(d.cb, bt) + imap32(d.cm, m);
      }
      s_a[tid] = a;
      s_b[tid] = b;
      s_c[tid] = c;
    }
    __syncthreads();
    if (!col_ok) continue;
    const unsigned nrows = min((unsigned)RB, NR - r0);
    for (unsigned r = threadIdx.y; r < nrows; r += blockDim.y) {
      const long long a0 = s_a[r], b0 = s_b[r] + bn_off;
      int ctr[kMaxLab];
      for (int q = 0; q < kMaxLab; ++q) ctr[q] = 0;
      long long ao = 0, bo = 0;
      R sr = 0, si = 0;
      for (long long k = 0; k < d.K; ++k) {
        R ar_, ai_, br_, bi_;
        ld_elem<R>(d.A, a0 + ao, d.a_cplx, d.a_f32, ar_, ai_);
        ld_elem<R>(d.B, b0 + bo, d.b_cplx, d.b_f32, br_, bi_);
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
      const long long off = s_c[r] + cn_off;
      R vr = ar * sr - ai * si, vi = ar * si + ai * sr;
      if (!d.store) {
        R cr, ci;
        ld_elem<R>(d.C, off, d.c_cplx, d.c_f32, cr, ci);
        vr += cr;
        vi += ci;
      }
      st_elem<R>(d.C, off, d.c_cplx, d.c_f32, vr, vi);
    }
  }
}

__device__ __forceinline__ double flip_sign(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

// C[all labels] (+)= sum_s alpha_s * A_s: the innermost label over threadIdx.x, the rest over
// rows.  F32 (reduced-precision programs): values are rounded to binary32 with integer
// operations and summed in float32, which keeps the kernel off the float64 pipe (its rounding,
// 2^-24 relative, is far below what those programs' contractions resolve); otherwise float64
// with one fused multiply-add per component and real scale.  A fresh output fed by a single
// unit-scale source is a plain copy (a sign-bit flip for -1) in both modes.
template <int NS, bool F32>
__global__ void __launch_bounds__(256) add_kernel(AddDesc d, unsigned inner) {
  using R = typename std::conditional<F32, float, double>::type;
  constexpr int RT = 32;   // rows per tile: their offsets are decoded once into shared memory
  __shared__ long long s_c[RT], s_a[NS][RT];
  const unsigned rows = (unsigned)(d.n / inner);
  const unsigned nrt = (rows + RT - 1) / RT;
  const unsigned tid = threadIdx.y * blockDim.x + threadIdx.x;
  const long long cs = d.c_all.strides[d.c_all.n - 1];
  long long as[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) as[q] = d.a_all[q].strides[d.a_all[q].n - 1];
  const bool copy = NS == 1 && d.store && d.ai[0] == 0.0 && (d.ar[0] == 1.0 || d.ar[0] == -1.0);
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  for (unsigned rt = blockIdx.y; rt < nrt; rt += gridDim.y) {
    __syncthreads();
    if (tid < RT) {
      const unsigned row = rt * RT + tid;
      if (row < rows) {
        s_c[tid] = imap32_outer(d.c_all, row);
#pragma unroll
        for (int q = 0; q < NS; ++q) s_a[q][tid] = imap32_outer(d.a_all[q], row);
      }
    }
    __syncthreads();
    if (i >= inner) continue;
    const unsigned nrows = min((unsigned)RT, rows - rt * RT);
    for (unsigned r = threadIdx.y; r < nrows; r += blockDim.y) {
      const long long c_off = s_c[r] + (long long)i * cs;
      if (copy) {
        const long long a_off = s_a[0][r] + (long long)i * as[0];
        if (!d.a_f32[0] && !d.c_f32) {   // float64 to float64: a bit copy (sign flip for -1)
          const bool neg = d.ar[0] < 0.0;
          double xr, xi;
          ld_elem<double>(d.A[0], a_off, d.a_cplx[0], 0, xr, xi);
          if (neg) {
            xr = flip_sign(xr);
            xi = flip_sign(xi);
          }
          st_elem<double>(d.C, c_off, d.c_cplx, 0, xr, xi);
        } else {
          float xr, xi;
          ld_elem<float>(d.A[0], a_off, d.a_cplx[0], d.a_f32[0], xr, xi);
          if (d.ar[0] < 0.0) {
            xr = -xr;
            xi = -xi;
          }
          st_elem<float>(d.C, c_off, d.c_cplx, d.c_f32, xr, xi);
        }
        continue;
      }
      R accr = 0, acci = 0;
      if (!d.store) ld_elem<R>(d.C, c_off, d.c_cplx, d.c_f32, accr, acci);
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        const long long a_off = s_a[q][r] + (long long)i * as[q];
        R xr, xi;
        ld_elem<R>(d.A[q], a_off, d.a_cplx[q], d.a_f32[q], xr, xi);
        const R ar = (R)d.ar[q], ai = (R)d.ai[q];
        if (d.ai[q] == 0.0) {
          accr = fma(ar, xr, accr);
          acci = fma(ar, xi, acci);
        } else {
          accr += ar * xr - ai * xi;
          acci += ar * xi + ai * xr;
        }
      }
      st_elem<R>(d.C, c_off, d.c_cplx, d.c_f32, accr, acci);
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
    double ar_, ai_, br_, bi_;
    ld_elem<double>(d.A, ao, d.a_cplx, d.a_f32, ar_, ai_);
    ld_elem<double>(d.B, bo, d.b_cplx, d.b_f32, br_, bi_);
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
    if (d.c_f32) {
      float* C = static_cast<float*>(d.C);
      if (d.c_cplx) { atomicAdd(&C[2 * off], f64_to_f32_bits(vr)); atomicAdd(&C[2 * off + 1], f64_to_f32_bits(vi)); }
      else atomicAdd(&C[off], f64_to_f32_bits(vr));
    } else {
      double* C = static_cast<double*>(d.C);
      if (d.c_cplx) { atomicAdd(&C[2 * off], vr); atomicAdd(&C[2 * off + 1], vi); }
      else atomicAdd(&C[off], vr);
    }
  }
}

// Few outputs, long K (M, N <= 32 per batch entry; reduced-precision programs): a block owns one
// batch entry and one K range; per 64-wide K chunk it stages A[m][k] and B[n][k] (float32,
// complex) in shared memory with the chunk's k offsets decoded once, every thread accumulates a
// 2 x 2 block of the M x N outputs, and the block adds its partial sums atomically at the end.
constexpr int kSmallMN = 32, kSmallKC = 64;
__global__ void __launch_bounds__(256) smallmn_kernel(DirectDesc d, long long kper) {
  __shared__ float2 sA[kSmallMN][kSmallKC + 1], sB[kSmallMN][kSmallKC + 1];
  __shared__ long long s_ka[kSmallKC], s_kb[kSmallKC], s_am[kSmallMN], s_bn[kSmallMN];
  const unsigned M = (unsigned)d.M, N = (unsigned)d.N, tid = threadIdx.x;
  const unsigned bt = blockIdx.y;
  const long long k0 = (long long)blockIdx.x * kper, k1 = min(d.K, k0 + kper);
  if (tid < M) s_am[tid] = imap32(d.ab, bt) + imap32(d.am, tid);
  if (tid >= 64 && tid - 64 < N) s_bn[tid - 64] = imap32(d.bb, bt) + imap32(d.bn, tid - 64);
  // each thread owns a 2 x 2 block of outputs (rows 2*mb, 2*mb+1; columns 2*nb, 2*nb+1), so every
  // shared-memory operand it reads feeds two products
  const unsigned nbn = (N + 1) / 2, mb = tid / nbn, nb = tid - mb * nbn;
  const bool active = mb < (M + 1) / 2;
  const unsigned m0 = 2 * mb, n0 = 2 * nb;
  const unsigned m1 = min(m0 + 1, M - 1), n1 = min(n0 + 1, N - 1);   // clamped reads; writes masked
  float cr[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, ci[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (long long kc = k0; kc < k1; kc += kSmallKC) {
    __syncthreads();
    if (tid < kSmallKC) {
      const long long k = kc + tid;
      s_ka[tid] = k < k1 ? imap32(d.ak, (unsigned)k) : -1;
    } else if (tid < 2 * kSmallKC) {
      const long long k = kc + tid - kSmallKC;
      s_kb[tid - kSmallKC] = k < k1 ? imap32(d.bk, (unsigned)k) : -1;
    }
    __syncthreads();
    for (unsigned idx = tid; idx < M * kSmallKC; idx += blockDim.x) {
      const unsigned m = idx / kSmallKC, kk = idx % kSmallKC;
      float xr = 0.f, xi = 0.f;
      if (s_ka[kk] >= 0) ld_elem<float>(d.A, s_am[m] + s_ka[kk], d.a_cplx, d.a_f32, xr, xi);
      sA[m][kk] = make_float2(xr, xi);
    }
    for (unsigned idx = tid; idx < N * kSmallKC; idx += blockDim.x) {
      const unsigned n = idx / kSmallKC, kk = idx % kSmallKC;
      float xr = 0.f, xi = 0.f;
      if (s_kb[kk] >= 0) ld_elem<float>(d.B, s_bn[n] + s_kb[kk], d.b_cplx, d.b_f32, xr, xi);
      sB[n][kk] = make_float2(xr, xi);
    }
    __syncthreads();
    if (active) {
#pragma unroll 8
      for (int kk = 0; kk < kSmallKC; ++kk) {
        const float2 a[2] = {sA[m0][kk], sA[m1][kk]}, b[2] = {sB[n0][kk], sB[n1][kk]};
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            cr[i][j] = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, cr[i][j]));
            ci[i][j] = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, ci[i][j]));
          }
      }
    }
  }
  if (!active) return;
  const float ar = (float)d.ar, ai = (float)d.ai;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const unsigned m = m0 + i, n = n0 + j;
      if (m >= M || n >= N) continue;
      const long long off = imap32(d.cb, bt) + imap32(d.cm, m) + imap32(d.cn, n);
      const float vr = ar * cr[i][j] - ai * ci[i][j], vi = ar * ci[i][j] + ai * cr[i][j];
      if (d.c_f32) {
        float* C = static_cast<float*>(d.C);
        if (d.c_cplx) {
          atomicAdd(&C[2 * off], vr);
          atomicAdd(&C[2 * off + 1], vi);
        } else {
          atomicAdd(&C[off], vr);
        }
      } else {
        double* C = static_cast<double*>(d.C);
        if (d.c_cplx) {
          atomicAdd(&C[2 * off], f32_to_f64_bits(vr));
          atomicAdd(&C[2 * off + 1], f32_to_f64_bits(vi));
        } else {
          atomicAdd(&C[off], f32_to_f64_bits(vr));
        }
      }
    }
}

// Short K and few columns (K, N <= 32; reduced-precision programs), many rows: one thread per
// row m keeps A[m][0..K) in registers and forms its N outputs against B[n][k] staged in shared
// memory (read as broadcasts); consecutive threads hold consecutive rows, so loads and the
// atomic adds into C are coalesced along m.
constexpr int kSkinny = 32;
__global__ void __launch_bounds__(256) skinny_kernel(DirectDesc d) {
  __shared__ __align__(16) float2 sB[kSkinny][kSkinny];
  __shared__ long long s_ak[kSkinny], s_cn[kSkinny];
  const unsigned bt = blockIdx.y, tid = threadIdx.x;
  const int K = (int)d.K, N = (int)d.N;
  for (unsigned idx = tid; idx < (unsigned)(N * kSkinny); idx += blockDim.x) {
    const unsigned n = idx / kSkinny, k = idx - n * kSkinny;
    float xr = 0.f, xi = 0.f;
    if (k < (unsigned)K)
      ld_elem<float>(d.B, imap32(d.bb, bt) + imap32(d.bn, n) + imap32(d.bk, k), d.b_cplx, d.b_f32, xr, xi);
    sB[n][k] = make_float2(xr, xi);
  }
  if (tid < (unsigned)K) s_ak[tid] = imap32(d.ak, tid);
  if (tid >= 64 && tid - 64 < (unsigned)N) s_cn[tid - 64] = imap32(d.cn, tid - 64);
  __syncthreads();
  const unsigned long long m = (unsigned long long)blockIdx.x * blockDim.x + tid;
  if (m >= (unsigned long long)d.M) return;
  const long long a0 = imap32(d.ab, bt) + imap32(d.am, (unsigned)m);
  const long long c0 = imap32(d.cb, bt) + imap32(d.cm, (unsigned)m);
  float2 a[kSkinny];
#pragma unroll
  for (int k = 0; k < kSkinny; ++k) {
    a[k] = make_float2(0.f, 0.f);
    if (k < K) ld_elem<float>(d.A, a0 + s_ak[k], d.a_cplx, d.a_f32, a[k].x, a[k].y);
  }
  const float ar = (float)d.ar, ai = (float)d.ai;
  for (int n = 0; n < N; ++n) {
    float sr = 0.f, si = 0.f;
    // two complex B values per 16-byte shared-memory read (rows are zero-padded past K)
    const float4* brow = reinterpret_cast<const float4*>(&sB[n][0]);
#pragma unroll
    for (int k2 = 0; k2 < kSkinny / 2; ++k2) {
      if (2 * k2 < K) {
        const float4 b = brow[k2];
        sr = fmaf(a[2 * k2].x, b.x, fmaf(-a[2 * k2].y, b.y, sr));
        si = fmaf(a[2 * k2].x, b.y, fmaf(a[2 * k2].y, b.x, si));
        sr = fmaf(a[2 * k2 + 1].x, b.z, fmaf(-a[2 * k2 + 1].y, b.w, sr));
        si = fmaf(a[2 * k2 + 1].x, b.w, fmaf(a[2 * k2 + 1].y, b.z, si));
      }
    }
    const float vr = ar * sr - ai * si, vi = ar * si + ai * sr;
    const long long off = c0 + s_cn[n];
    if (d.c_f32) {
      if (d.c_cplx) {
        float2* c = static_cast<float2*>(d.C) + off;
        if (d.store) *c = make_float2(vr, vi);
        else atomicAdd(c, make_float2(vr, vi));
      } else {
        float* c = static_cast<float*>(d.C) + off;
        if (d.store) *c = vr;
        else atomicAdd(c, vr);
      }
    } else {
      if (d.c_cplx) {
        double2* c = static_cast<double2*>(d.C) + off;
        if (d.store) {
          *c = make_double2(f32_to_f64_bits(vr), f32_to_f64_bits(vi));
        } else {
          atomicAdd(&c->x, f32_to_f64_bits(vr));
          atomicAdd(&c->y, f32_to_f64_bits(vi));
        }
      } else {
        double* c = static_cast<double*>(d.C) + off;
        if (d.store) *c = f32_to_f64_bits(vr);
        else atomicAdd(c, f32_to_f64_bits(vr));
      }
    }
  }
}

// float64 SIMT GEMM: 64x64 tile, 16-deep K slices, 256 threads with 4x4 outputs each.
__global__ void __launch_bounds__(256) dgemm_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                                    double* __restrict__ C, int M, int N, int K, int splits,
                                                    int kper) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const size_t bz = blockIdx.z / splits;
  const int sp = blockIdx.z - (int)bz * splits;
  const int kbeg = sp * kper, kend = min(K, kbeg + kper);
  A += bz * (size_t)M * K;
  B += bz * (size_t)N * K;
  C += bz * (size_t)M * N;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + q * 256;
      const int r = e >> 4, c = e & 15;
      As[c][r] = (m0 + r < M && k0 + c < kend) ? A[(size_t)(m0 + r) * K + k0 + c] : 0.0;
      Bs[c][r] = (n0 + r < N && k0 + c < kend) ? B[(size_t)(n0 + r) * K + k0 + c] : 0.0;
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
      if (n < N) {
        if (splits > 1) atomicAdd(&C[(size_t)m * N + n], acc[i][j]);
        else C[(size_t)m * N + n] = acc[i][j];
      }
    }
  }
}

}  // namespace

void launch_pack(const PackDesc& d, cudaStream_t s) {
  const long long NR = d.NB * d.R;
  if (NR == 0) return;
  RTCC_REQUIRE(NR < (1ll << 31) && d.K < (1ll << 31), "pack extents exceed 32-bit indexing");
  RTCC_REQUIRE(!(d.ktab || d.rtab) || (d.ncs == 1 && d.nss == 1 && d.elem != PE_F64 && d.Kpad % 4 == 0 && !d.transpose),
               "pair-symmetric gathers are tensor-core plane packs in direct mode");
  if (d.ncs == 1 && d.nss == 1 && d.elem != PE_F64 && d.Kpad % 4 == 0) {
    // tensor-core operand planes
    if (d.transpose) {
      const long long nkt = (d.Kpad + 63) / 64, nrt = (NR + 31) / 32;
      // each block walks several k tiles of one row tile (the row offsets are decoded once)
      const long long gx = std::max(1ll, std::min(nkt, ((long long)device_sm_count() * 32 + nrt - 1) / nrt));
      dim3 grid((unsigned)gx, (unsigned)std::min(nrt, 65535ll));
      dim3 blk(32, 8);
      if (d.elem == PE_F32) pack_planes_transpose_kernel<PE_F32><<<grid, blk, 0, s>>>(d);
      else pack_planes_transpose_kernel<PE_BF16><<<grid, blk, 0, s>>>(d);
    } else {
      const unsigned nq = (unsigned)(d.Kpad / 4);
      const unsigned bx = nq >= 128 ? 128u : std::max(32u, (nq + 31) / 32 * 32);
      const unsigned by = 256 / bx;
      dim3 blk(bx, by);
      dim3 grid((nq + bx - 1) / bx, (unsigned)std::min((NR + 31) / 32, 65535ll));
      if (d.elem == PE_F32) pack_planes_direct_kernel<PE_F32><<<grid, blk, 0, s>>>(d);
      else pack_planes_direct_kernel<PE_BF16><<<grid, blk, 0, s>>>(d);
    }
    RTCC_CUDA(cudaGetLastError());
    return;
  }
  RTCC_REQUIRE(!d.src_f32, "the float64 GEMM path packs float64 tensors only");
  const unsigned padw = (unsigned)(d.Kpad - (long long)d.nss * d.ncs * d.K);
  if (d.transpose) {
    const unsigned nkt = (unsigned)((d.K + 31) / 32) + (padw ? 1 : 0);
    const unsigned nrt = (unsigned)((NR + 31) / 32);
    dim3 grid(std::min(nkt, 4096u), std::min(nrt, 65535u));
    dim3 blk(32, 8);
    if (d.elem == PE_F64) pack_transpose_kernel<PE_F64><<<grid, blk, 0, s>>>(d, padw);
    else if (d.elem == PE_F32) pack_transpose_kernel<PE_F32><<<grid, blk, 0, s>>>(d, padw);
    else pack_transpose_kernel<PE_BF16><<<grid, blk, 0, s>>>(d, padw);
  } else {
    const unsigned kext = (unsigned)d.K + padw;
    const unsigned bx = kext >= 256 ? 256u : std::max(32u, (kext + 31) / 32 * 32);
    const unsigned by = 256 / bx;
    dim3 blk(bx, by);
    dim3 grid(std::min((kext + bx - 1) / bx, 4096u), (unsigned)std::min((NR + by - 1) / by, 65535ll));
    if (d.elem == PE_F64) pack_direct_kernel<PE_F64><<<grid, blk, 0, s>>>(d, kext, padw);
    else if (d.elem == PE_F32) pack_direct_kernel<PE_F32><<<grid, blk, 0, s>>>(d, kext, padw);
    else pack_direct_kernel<PE_BF16><<<grid, blk, 0, s>>>(d, kext, padw);
  }
  RTCC_CUDA(cudaGetLastError());
}
void launch_unpack(const UnpackDesc& d, cudaStream_t s) {
  const long long NR = d.NB * d.M;
  if (NR == 0 || d.N == 0) return;
  RTCC_REQUIRE(NR < (1ll << 31) && d.N < (1ll << 31), "unpack extents exceed 32-bit indexing");
  if (d.transpose) {
    dim3 grid((unsigned)std::min((d.N + 31) / 32, 4096ll), (unsigned)std::min((NR + 31) / 32, 65535ll));
    dim3 blk(32, 8);
    if (d.gout_f64) unpack_transpose_kernel<double><<<grid, blk, 0, s>>>(d);
    else unpack_transpose_kernel<float><<<grid, blk, 0, s>>>(d);
  } else {
    const unsigned N = (unsigned)d.N;
    const unsigned bx = N >= 256 ? 256u : std::max(32u, (N + 31) / 32 * 32);
    const unsigned by = 256 / bx;
    dim3 blk(bx, by);
    dim3 grid(std::min((N + bx - 1) / bx, 4096u), (unsigned)std::min((NR + by - 1) / by, 65535ll));
    if (d.gout_f64) unpack_direct_kernel<double><<<grid, blk, 0, s>>>(d);
    else unpack_direct_kernel<float><<<grid, blk, 0, s>>>(d);
  }
  RTCC_CUDA(cudaGetLastError());
}
void launch_direct(const DirectDesc& d, cudaStream_t s) {
  const long long NR = d.NB * d.M;
  if (NR == 0 || d.N == 0) return;
  RTCC_REQUIRE(NR < (1ll << 31) && d.N < (1ll << 31), "direct extents exceed 32-bit indexing");
  const unsigned N = (unsigned)d.N;
  const unsigned bx = N >= 128 ? 128u : std::max(32u, (N + 31) / 32 * 32);
  const unsigned by = 128 / bx;
  dim3 blk(bx, by);
  dim3 grid((N + bx - 1) / bx, (unsigned)std::min((NR + 31) / 32, 65535ll));
  if (d.f32) direct_kernel<true><<<grid, blk, 0, s>>>(d);
  else direct_kernel<false><<<grid, blk, 0, s>>>(d);
  RTCC_CUDA(cudaGetLastError());
}
void launch_skinny(const DirectDesc& d, cudaStream_t s) {
  RTCC_REQUIRE(d.K >= 1 && d.K <= kSkinny && d.N >= 1 && d.N <= kSkinny && d.M < (1ll << 31) && d.NB < 65536,
               "short-K contraction extents");
  if (d.M == 0) return;
  dim3 grid((unsigned)((d.M + 255) / 256), (unsigned)d.NB);
  skinny_kernel<<<grid, 256, 0, s>>>(d);
  RTCC_CUDA(cudaGetLastError());
}
void launch_smallmn(const DirectDesc& d, cudaStream_t s) {
  RTCC_REQUIRE(d.M <= kSmallMN && d.N <= kSmallMN && d.M * d.N <= 1024 && d.NB < 65536 && d.K < (1ll << 31),
               "small-output reduction extents");
  if (d.NB * d.M * d.N == 0 || d.K == 0) return;
  // about four blocks per SM in total, whole 64-wide chunks per block
  long long splits = std::max(1ll, std::min(((long long)device_sm_count() * 4 + d.NB - 1) / d.NB, (d.K + kSmallKC - 1) / kSmallKC));
  long long kper = (d.K + splits - 1) / splits;
  kper = (kper + kSmallKC - 1) / kSmallKC * kSmallKC;
  splits = (d.K + kper - 1) / kper;
  dim3 grid((unsigned)splits, (unsigned)d.NB);
  smallmn_kernel<<<grid, 256, 0, s>>>(d, kper);
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
  RTCC_REQUIRE(d.n < (1ll << 32) && d.c_all.n >= 1, "add extents exceed 32-bit indexing");
  const unsigned inner = (unsigned)d.c_all.dims[d.c_all.n - 1];
  const unsigned rows = (unsigned)(d.n / inner);
  const unsigned bx = inner >= 128 ? 128u : std::max(32u, (inner + 31) / 32 * 32);
  const unsigned by = 256 / bx;
  dim3 blk(bx, by);
  dim3 grid((inner + bx - 1) / bx, std::min((rows + 31) / 32, 65535u));
  const int key = d.nsrc * 2 + (d.f32 ? 1 : 0);
  switch (key) {
    case 2: add_kernel<1, false><<<grid, blk, 0, s>>>(d, inner); break;
    case 3: add_kernel<1, true><<<grid, blk, 0, s>>>(d, inner); break;
    case 4: add_kernel<2, false><<<grid, blk, 0, s>>>(d, inner); break;
    case 5: add_kernel<2, true><<<grid, blk, 0, s>>>(d, inner); break;
    case 6: add_kernel<3, false><<<grid, blk, 0, s>>>(d, inner); break;
    case 7: add_kernel<3, true><<<grid, blk, 0, s>>>(d, inner); break;
    case 8: add_kernel<4, false><<<grid, blk, 0, s>>>(d, inner); break;
    case 9: add_kernel<4, true><<<grid, blk, 0, s>>>(d, inner); break;
    default: throw Error(3, "add with an unsupported number of sources");
  }
  RTCC_CUDA(cudaGetLastError());
}
void launch_gemm_f64(const double* A, const double* B, double* C, long long M, long long N, long long Kpad,
                     long long NB, cudaStream_t s) {
  RTCC_REQUIRE(M < (1ll << 31) && N < (1ll << 31) && Kpad < (1ll << 31) && NB < 65536, "GEMM extents too large");
  const long long tiles = ((N + 63) / 64) * ((M + 63) / 64) * NB;
  int splits = 1;
  const long long nsm = device_sm_count();
  if (tiles < 2 * nsm && Kpad >= 512)
    splits = (int)std::max(1ll, std::min<long long>((4 * nsm + tiles - 1) / tiles, Kpad / 256));
  splits = (int)std::min<long long>(splits, 65535 / NB);
  const int kper = (int)(((Kpad + splits - 1) / splits + 15) / 16 * 16);
  splits = (int)((Kpad + kper - 1) / kper);
  if (splits > 1) RTCC_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * M * N * NB, s));
  dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64), (unsigned)(NB * splits));
  dgemm_kernel<<<grid, 256, 0, s>>>(A, B, C, (int)M, (int)N, (int)Kpad, splits, kper);
  RTCC_CUDA(cudaGetLastError());
}

}  // namespace rtcc
