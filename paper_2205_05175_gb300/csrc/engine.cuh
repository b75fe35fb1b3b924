// Contraction engine: einsum-style programs over device tensors, compiled once into a
// fixed launch sequence (pack -> GEMM -> unpack, or a direct kernel for small terms),
// plus a reverse-mode generator that turns a program into its vector-Jacobian program.
#pragma once
#include "common.cuh"
#include <complex>
#include <map>
#include <memory>
#include <string>
#include <vector>
#include <algorithm>

namespace rtcc {

using cplx = std::complex<double>;

enum class Prec : int { P64 = 0, TF32 = 1, TF32X3 = 2, BF16X3 = 3 };

enum Storage : int { ST_EXTERNAL = 0, ST_ARENA = 1, ST_OWNED = 2 };

struct Tensor {
  std::string name;
  std::vector<int> dims;
  std::vector<long long> strides;   // element strides (complex elements for complex tensors)
  bool cplx = true;
  bool f32 = false;                 // float32 / complex64 elements (temporaries of reduced-precision engines)
  bool constant = false;            // never differentiated; packed once when used in a GEMM
  int storage = ST_EXTERNAL;
  int arena = -1;                   // arena index for ST_ARENA
  long long arena_off = 0;          // offset in doubles
  double* ptr = nullptr;
  size_t esz() const { return (f32 ? 4u : 8u) * (cplx ? 2u : 1u); }   // bytes per element
  long long numel() const {
    long long n = 1;
    for (int d : dims) n *= d;
    return n;
  }
};

enum OpKind : int { OP_EIN = 0, OP_ADD = 1 };
struct Op {
  int kind;
  int c, a, b;
  std::string lc, la, lb;
  cplx alpha;
  // EIN only: B is a real constant tensor with two label pairs (its labels 0,1 and 2,3; one pair
  // contracted, the other kept) and B is unchanged by swapping both pairs at once, e.g.
  // (ae|bf) = (bf|ae).  The planner may then contract over ordered pairs only (half the work).
  bool pairsym = false;
};

struct Compiled;   // defined in engine.cu

struct Program {
  std::string name;
  std::vector<Op> ops;
  std::vector<int> zero_arenas;     // arenas cleared before the first op
  std::vector<int> zero_tensors;    // contiguous tensors cleared before the first op
  struct Zero2D { void* ptr; size_t pitch, width, height; };
  std::vector<Zero2D> zero2d;       // strided regions cleared before the first op
  int prec_override = -1;           // >= 0: run this program's GEMM-path contractions in this Prec
  bool tuned = false;               // its tensor-core tiles were chosen by Engine::autotune
  std::vector<std::shared_ptr<Compiled>> comp;
};

// Kernel classes of the launch profile (rtcc_profile_t in include/rtcc.h uses the same order).
enum KClass : int { KC_TC_GEMM = 0, KC_F64_GEMM = 1, KC_PACK = 2, KC_UNPACK = 3, KC_DIRECT = 4, KC_REDUCE = 5,
                    KC_ADD = 6, KC_RK = 7, KC_N = 8 };

// Optional CUDA-event timing of every launch (eager execution only).
class Profiler {
 public:
  ~Profiler();
  void begin();
  bool on() const { return on_; }
  void start(cudaStream_t s);
  void stop(cudaStream_t s, int cls, double flops, double bytes, const char* tag = nullptr);
  // synchronises, accumulates per class and turns profiling off
  void end(long long launches[KC_N], double ms[KC_N], double flops[KC_N], double bytes[KC_N]);
  long long count[KC_N] = {0};   // launches per class, counted whether or not timing is on
 private:
  struct Rec { int cls; int a, b; double flops, bytes; std::string tag; };
  cudaEvent_t get();
  bool on_ = false;
  std::vector<cudaEvent_t> pool_;
  size_t used_ = 0;
  std::vector<Rec> recs_;
  int pending_ = -1;
};

struct EngineStats {
  long long gemm_flops = 0;   // real multiply-adds x2 issued on the GEMM path per run (all programs)
  long long direct_flops = 0;
  int launches = 0;
};

class Engine {
 public:
  Engine(Prec p, cudaStream_t s);
  ~Engine();
  Engine(const Engine&) = delete;
  Engine& operator=(const Engine&) = delete;

  Prec prec() const { return prec_; }
  // Route every contraction with a summed index through the packed GEMM path (self-test).
  void set_force_gemm(bool f) { force_gemm_ = f; }
  cudaStream_t stream() const { return stream_; }
  int* dev_err() const { return dev_err_; }

  // --- tensors ------------------------------------------------------------------------
  int external(const std::string& name, const std::vector<int>& dims, bool cplx, double* ptr,
               std::vector<long long> strides = {}, bool constant = false);
  int owned(const std::string& name, const std::vector<int>& dims, bool cplx, bool constant);
  int new_arena();
  int temp(int arena, const std::string& name, const std::vector<int>& dims, bool cplx = true);
  // Temporaries created after arena_reset(a, mark) reuse the space from `mark` on; only
  // for programs that never run interleaved with one another.
  long long arena_mark(int arena) const { return arena_size_[arena]; }
  void arena_reset(int arena, long long mark) { arena_hwm_[arena] = std::max(arena_hwm_[arena], arena_size_[arena]); arena_size_[arena] = mark; }
  Tensor& T(int id) { return tensors_[id]; }
  const Tensor& T(int id) const { return tensors_[id]; }

  // --- program building ------------------------------------------------------------------
  static void ein(Program& P, int c, const std::string& lc, int a, const std::string& la, int b,
                  const std::string& lb, cplx alpha = 1.0, bool pairsym = false);
  static void add(Program& P, int c, const std::string& lc, int a, const std::string& la, cplx alpha = 1.0);

  // Reverse mode: given the forward program and the ids of its active inputs, return the
  // program that accumulates adjoints; adj maps tensor id -> adjoint tensor id (created in
  // `arena`; adjoints of inputs included).
  Program reverse(const Program& fwd, const std::vector<int>& active_inputs, int arena,
                  std::map<int, int>& adj);

  // Allocate arenas and owned tensors, plan every op of the given programs, allocate the
  // shared workspaces, bind pointers (tensor maps, constant packing).  Call once.
  void finalize(std::vector<Program*> progs);

  void run(const Program& P);
  // Tile autotuner: times every tensor-core GEMM of P (after finalize) with each usable N tile
  // (64, 128, 256 columns; the 256 tile also with three stages and eight epilogue warps) on this
  // GPU and keeps the fastest; choices are cached per GEMM shape on the engine.  Runs kernels on the stream: outside stream capture, and only while no data in the
  // programs' outputs or temporaries is needed (they are recomputed by every program run).
  // Returns the number of GEMMs whose tile changed.
  int autotune(Program& P);
  int tuned_gemms() const { return (int)tile_cache_.size(); }
  void set_profiler(Profiler* p) { prof_ = p; }
  EngineStats stats_of(const Program& P) const;
  void check_error();   // throws on a device-side timeout recorded by a kernel
  size_t device_bytes() const { return bytes_; }

 private:
  void plan(Program& P);
  void bind(Program& P);
  bool add_source(Compiled& k, const std::vector<Op>& ops, int oi, const std::string& lc);
  bool plan_pairsym(Compiled& k, const Op& op, const std::string& Lm, const std::string& Ln, const std::string& Lk,
                    const std::string& Lb, const IndexMap& am, const IndexMap& cm, Prec prec, bool c_fresh);
  void bind_gemm(Compiled& k, const Tensor& A, const Tensor& B, const Tensor& C);
  void run_gemm(const Compiled& k, Profiler& pr, const char* tag);
  const long long* upload(const std::vector<long long>& v);
  const float* upload(const std::vector<float>& v);
  void merge_adds(Program& P);
  void share_packs(Program& P);

  Prec prec_;
  cudaStream_t stream_;
  std::vector<Tensor> tensors_;
  std::vector<long long> arena_size_;
  std::vector<long long> arena_hwm_;
  std::vector<double*> arena_ptr_;
  std::vector<void*> allocs_;
  int* dev_err_ = nullptr;
  std::map<std::string, void*> const_packs_;   // pack image of a constant operand -> its packed planes
  std::map<std::string, void*> tables_;        // content of an uploaded index table -> its device copy
  std::map<std::string, int> tile_cache_;      // GEMM shape -> N tile chosen by the autotuner
  void* wsA_ = nullptr;
  void* wsB_ = nullptr;
  void* wsC_ = nullptr;
  size_t wsA_bytes_ = 0, wsB_bytes_ = 0, wsC_bytes_ = 0;
  size_t bytes_ = 0;
  bool finalized_ = false;
  bool force_gemm_ = false;
  Profiler* prof_ = nullptr;
};

// Allocation helper that records ownership (freed with the engine).
void* dev_alloc(size_t bytes);

}  // namespace rtcc
