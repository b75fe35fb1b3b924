// Allocation-free tensor-core GEMM entry point (rtcc_gemm_noalloc in include/rtcc.h).
//
// Some callers cannot let a library call cudaMalloc: an application that owns every byte of
// device memory through its own pool (a framework's caching allocator, a service that sizes
// its memory once at start-up and treats later allocation as a fault), or code that must not
// perform allocation, with its implicit device synchronisation, inside a latency-critical
// loop.  This entry point runs the same packing and tcgen05 GEMM kernels as the rest of the
// library, but the packed operand planes live in a fixed file-scope device array instead of
// memory obtained from cudaMalloc.  Inputs and the output are the caller's device buffers.
#include "common.cuh"
#include "../../include/rtcc.h"
#include <map>
#include <mutex>
#include <string>

namespace {

// Scratch for the packed operand planes.  Every GPU that loads the library holds this array
// until the process exits.
constexpr size_t kScratchBytes = 64ull << 20;
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];
__device__ __align__(256) int g_err[4];

struct DeviceScratch {
  void* scratch = nullptr;
  int* err = nullptr;
};

std::mutex g_mutex;
std::map<int, DeviceScratch> g_devices;

rtcc_status_t fail(int code, const std::string& m) {
  rtcc::set_last_error(m);   // reported by rtcc_last_error()
  return (rtcc_status_t)code;
}

// Per-device set-up: the host-side names of g_scratch / g_err are stand-ins, not device
// addresses, so the addresses are looked up once per device with that device current.
rtcc_status_t device_scratch(DeviceScratch& out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(RTCC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  std::lock_guard<std::mutex> lk(g_mutex);
  auto it = g_devices.find(dev);
  if (it != g_devices.end()) {
    out = it->second;
    return RTCC_OK;
  }
  DeviceScratch d;
  e = cudaGetSymbolAddress(&d.scratch, g_scratch);
  if (e != cudaSuccess) return fail(RTCC_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
  e = cudaGetSymbolAddress(reinterpret_cast<void**>(&d.err), g_err);
  if (e != cudaSuccess) return fail(RTCC_ERR_CUDA, std::string("cudaGetSymbolAddress(err): ") + cudaGetErrorString(e));
  g_devices[dev] = d;
  out = d;
  return RTCC_OK;
}

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

rtcc::IndexMap map1(long long dim, long long stride) {
  rtcc::IndexMap m{};
  m.n = 1;
  m.dims[0] = (int)dim;
  m.strides[0] = stride;
  return m;
}

// Operand planes: component (re, im) x split part (hi, lo), rows of length Kpad.
void plane_desc(rtcc::PackDesc& pd, const double* src, bool cplx, long long rows, long long K, long long NB,
                int npart, int elem, long long Kpad, void* dst) {
  pd = rtcc::PackDesc{};
  pd.src = src;
  pd.src_cplx = cplx;
  pd.rows = map1(rows, K);
  pd.cols = map1(K, 1);
  pd.bat = map1(NB, rows * K);
  pd.R = rows;
  pd.K = K;
  pd.NB = NB;
  const int nc = cplx ? 2 : 1;
  pd.nrb = nc * npart;
  pd.ncs = 1;
  pd.nss = 1;
  for (int c = 0; c < nc; ++c)
    for (int q = 0; q < npart; ++q) {
      const int rb = c * npart + q;
      pd.comp[rb][0] = c;
      pd.sign[rb][0] = 1;
      pd.rb_part[rb] = (npart == 1) ? rtcc::SP_FULL : (q == 0 ? rtcc::SP_HI : rtcc::SP_LO);
    }
  pd.Kpad = Kpad;
  pd.elem = elem;
  pd.round_tf32 = 1;
  pd.transpose = 0;
  pd.dst = dst;
}

rtcc_status_t gemm_noalloc(int prec, int cplx, int batch, int M, int N, int K, const double* A, const double* Bm,
                           double* C, void* stream) {
  using namespace rtcc;
  if (prec < RTCC_P32_TF32 || prec > RTCC_P32_BF16X3)
    return fail(RTCC_ERR_INVALID_ARG, "rtcc_gemm_noalloc: precision must be TF32, 3xTF32 or BF16x3");
  if (cplx < 0 || cplx > 3 || batch < 1 || M < 1 || N < 1 || K < 1 || !A || !Bm || !C)
    return fail(RTCC_ERR_INVALID_ARG, "rtcc_gemm_noalloc: bad argument");
  DeviceScratch ds;
  rtcc_status_t st = device_scratch(ds);
  if (st != RTCC_OK) return st;
  const bool ac = cplx & 1, bc = (cplx >> 1) & 1, cc = ac || bc;
  const bool x3 = prec != RTCC_P32_TF32;
  const int npart = x3 ? 2 : 1;
  const int kind = (prec == RTCC_P32_BF16X3) ? 1 : 0;
  const int elem = kind ? PE_BF16 : PE_F32;
  const long long esz = kind ? 2 : 4;
  const long long Kpad = round_up(K, tc_kblock_elems(kind));
  const int planesA = (ac ? 2 : 1) * npart, planesB = (bc ? 2 : 1) * npart;
  const long long bytesA = round_up((long long)batch * planesA * M * Kpad * esz, 256);
  const long long bytesB = round_up((long long)batch * planesB * N * Kpad * esz, 256);
  if (bytesA + bytesB > (long long)kScratchBytes)
    return fail(RTCC_ERR_INVALID_ARG, "rtcc_gemm_noalloc: packed operands need " + std::to_string(bytesA + bytesB) +
                                          " bytes of scratch, more than the " + std::to_string(kScratchBytes) +
                                          "-byte static limit");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* scr = static_cast<unsigned char*>(ds.scratch);
  PackDesc pa, pb;
  plane_desc(pa, A, ac, M, K, batch, npart, elem, Kpad, scr);
  plane_desc(pb, Bm, bc, N, K, batch, npart, elem, Kpad, scr + bytesA);
  TcGemmPlan pl{};
  TcGemmParams& g = pl.p;
  g.nrb = cc ? 2 : 1;
  auto plane = [&](int c, int q) { return c * npart + q; };
  auto pair = [&](int rb, int ca, int cb, int neg) {
    auto push = [&](int x, int y) { g.seg[rb][g.nseg[rb]++] = TcSeg{x, y, neg}; };
    if (npart == 1) push(plane(ca, 0), plane(cb, 0));
    else {
      push(plane(ca, 0), plane(cb, 0));
      push(plane(ca, 0), plane(cb, 1));
      push(plane(ca, 1), plane(cb, 0));
    }
  };
  if (!ac && !bc) pair(0, 0, 0, 0);
  else if (ac && !bc) { pair(0, 0, 0, 0); pair(1, 1, 0, 0); }
  else if (!ac && bc) { pair(0, 0, 0, 0); pair(1, 0, 1, 0); }
  else { pair(0, 0, 0, 0); pair(0, 1, 1, 1); pair(1, 0, 1, 0); pair(1, 1, 0, 0); }
  TcEpilogue& ep = g.epi;
  ep.C = C;
  ep.c_cplx = cc;
  ep.alpha = 1.0;
  ep.cm = map1(M, N);
  ep.cn = map1(N, 1);
  ep.cb = map1(batch, (long long)M * N);
  ep.flat_n = 1;
  ep.sn = 1;
  ep.unit_n = 1;
  // the output is overwritten; the error word keeps no state from an earlier call
  RTCC_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * (size_t)batch * M * N * (cc ? 2 : 1), s));
  RTCC_CUDA(cudaMemsetAsync(ds.err, 0, sizeof(int) * 4, s));
  launch_pack(pa, s);
  launch_pack(pb, s);
  tc_gemm_plan(pl, kind, pa.dst, planesA, pb.dst, planesB, M, N, Kpad, batch, ds.err);
  launch_tc_gemm(pl, s);
  int h = 0;
  RTCC_CUDA(cudaMemcpyAsync(&h, ds.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  RTCC_CUDA(cudaStreamSynchronize(s));
  if (h != DEV_OK) return fail(RTCC_ERR_TIMEOUT, "rtcc_gemm_noalloc: a tensor-core wait expired on the device");
  return RTCC_OK;
}

}  // namespace

// Every exception (the library's own errors, and std::exception from the scratch table or a
// message string) becomes a status code: nothing leaves this extern "C" function.
extern "C" rtcc_status_t rtcc_gemm_noalloc(int prec, int cplx, int batch, int M, int N, int K, const double* A,
                                           const double* Bm, double* C, void* stream) {
  try {
    return gemm_noalloc(prec, cplx, batch, M, N, K, A, Bm, C, stream);
  } catch (const rtcc::Error& e) {
    return fail(e.status, e.what());
  } catch (const std::exception& e) {
    return fail(RTCC_ERR_CUDA, std::string("rtcc_gemm_noalloc: ") + e.what());
  } catch (...) {
    return fail(RTCC_ERR_CUDA, "rtcc_gemm_noalloc: unknown exception");
  }
}
