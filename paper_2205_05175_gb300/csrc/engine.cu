// Contraction engine: planning and execution of einsum programs (see engine.cuh).
#include "engine.cuh"
#include <array>
#include <algorithm>
#include <set>
#include <cstdlib>

namespace rtcc {

void launch_reduce(const DirectDesc& d, long long splits, cudaStream_t s);
void launch_smallmn(const DirectDesc& d, cudaStream_t s);
void launch_skinny(const DirectDesc& d, cudaStream_t s);

namespace {

enum CompKind : int { CK_ADD = 0, CK_DIRECT = 1, CK_REDUCE = 2, CK_GEMM = 3, CK_MERGED = 4, CK_SMALLMN = 5, CK_SKINNY = 6 };   // CK_MERGED: folded into an earlier add

constexpr long long kDirectMaxWork = 1ll << 21;   // real multiply-adds below which a term runs direct
constexpr long long kReduceMaxOut = 2048;         // outputs up to which a long-K term is split-K reduced

IndexMap map_for(const Tensor& t, const std::string& tl, const std::string& labs) {
  IndexMap m{};
  RTCC_REQUIRE((int)labs.size() <= kMaxLab, "too many labels in one index group of " + t.name);
  m.n = (int)labs.size();
  for (int i = 0; i < m.n; ++i) {
    const size_t p = tl.find(labs[i]);
    RTCC_REQUIRE(p != std::string::npos, "label missing in " + t.name);
    m.dims[i] = t.dims[p];
    m.strides[i] = t.strides[p];
  }
  return m;
}

long long prod_dims(const IndexMap& m) {
  long long s = 1;
  for (int i = 0; i < m.n; ++i) s *= m.dims[i];
  return s;
}

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// K blocks per tensor-core accumulation chunk.  The split modes (hi/lo products) resolve about
// 2^-17 (BF16x3) or 2^-22 (3xTF32) per product, but the tensor cores' float32 accumulator drifts by
// about one unit in the last place per 16 products (measured: at K ~ 10^4 the drift dominates the
// dipole error of a whole trajectory), so their products are accumulated in chunks of 16 K blocks
// (1024 BF16 or 512 TF32 elements) and the chunks summed with round-to-nearest adds (at the hexamer
// shape: max|dmu| over 24 RK4 steps through the pulse 2.7e-6 au with chunks of 16 blocks, 2.3e-6 with
// 8, 1.2e-5 after 8 steps without chunks).  A single TF32 pass resolves only 2^-11 and keeps one
// accumulation.  RTCC_GEMM_CHUNK=<blocks> overrides (0: off).
int accumulation_chunk(Prec prec) {
  if (prec != Prec::TF32X3 && prec != Prec::BF16X3) return 0;
  if (const char* e = std::getenv("RTCC_GEMM_CHUNK")) return std::max(0, std::atoi(e));
  return 16;
}

// Order labels by decreasing |stride| in tensor t (so the unit-stride label comes last).
std::string by_stride(const std::string& labs, const Tensor& t, const std::string& tl) {
  std::string out = labs;
  std::stable_sort(out.begin(), out.end(), [&](char a, char b) {
    return std::llabs(t.strides[tl.find(a)]) > std::llabs(t.strides[tl.find(b)]);
  });
  return out;
}

// Chooses how a pack reads its source: directly along K when the source's unit-stride label is the
// last K label, else through shared-memory tiles enumerated with the unit-stride row label last.
void choose_pack_mode(PackDesc& pd, const Tensor& t, const std::string& tl, const std::string& rows,
                      const std::string& cols) {
  pd.transpose = 0;
  char u = 0;
  long long bs = -1;
  for (char l : rows + cols) {
    const long long st = std::llabs(t.strides[tl.find(l)]);
    if (bs < 0 || st < bs) {
      bs = st;
      u = l;
    }
  }
  if (u == 0 || rows.find(u) == std::string::npos) return;
  std::string rd = rows;
  rd.erase(rd.find(u), 1);
  rd.push_back(u);
  std::map<char, long long> P;
  long long acc = 1;
  for (int i = (int)rows.size() - 1; i >= 0; --i) {
    P[rows[i]] = acc;
    acc *= t.dims[tl.find(rows[i])];
  }
  pd.rd_src = map_for(t, tl, rd);
  pd.rd_dst = pd.rd_src;
  for (int i = 0; i < pd.rd_dst.n; ++i) pd.rd_dst.strides[i] = P[rd[i]];
  pd.transpose = 1;
}

// True when the smallest-stride label of t among (rows + cols) is the last row label.
bool row_is_unit(const Tensor& t, const std::string& tl, const std::string& rows, const std::string& cols) {
  if (rows.empty()) return false;
  char best = 0;
  long long bs = -1;
  for (char l : rows + cols) {
    const long long st = std::llabs(t.strides[tl.find(l)]);
    if (bs < 0 || st < bs) {
      bs = st;
      best = l;
    }
  }
  return best == rows.back();
}

}  // namespace

struct Compiled {
  int kind = CK_ADD;
  AddDesc add{};
  std::vector<int> add_ops;   // CK_ADD: the program ops whose sources this kernel sums (first = own op)
  std::shared_ptr<Compiled> twin;   // pair-symmetric contraction: the antisymmetric-part GEMM
  // pack sharing within a program: an operand packed identically by an earlier GEMM (source
  // unchanged in between) reuses that GEMM's planes; the earlier one then packs into its own buffer
  bool pa_keep = false, pb_keep = false;
  const Compiled* pa_from = nullptr;
  const Compiled* pb_from = nullptr;
  bool pa_from_b = false, pb_from_b = false;   // the provider's B (true) or A (false) planes
  DirectDesc dir{};
  long long splits = 1;
  // GEMM path
  PackDesc pa{}, pb{};
  bool a_const = false, b_const = false;
  void* a_pre = nullptr;
  void* b_pre = nullptr;
  size_t a_bytes = 0, b_bytes = 0, c_bytes = 0;
  UnpackDesc up{};
  long long GM = 0, GN = 0, Kpad = 0, NB = 0;
  int tc_kind = -1;   // -1: float64 SIMT GEMM, 0: tf32, 1: bf16
  int chunk = 0;      // K blocks per tensor-core accumulation chunk (0: none)
  TcGemmPlan tcp{};
  long long alg_flops = 0;    // useful real flops (one pass)
  long long exec_flops = 0;   // flops issued by the GEMM kernel (passes and padding included)
};

Profiler::~Profiler() {
  for (cudaEvent_t e : pool_) cudaEventDestroy(e);
}
void Profiler::begin() {
  on_ = true;
  used_ = 0;
  recs_.clear();
}
cudaEvent_t Profiler::get() {
  if (used_ == pool_.size()) {
    cudaEvent_t e;
    RTCC_CUDA(cudaEventCreate(&e));
    pool_.push_back(e);
  }
  return pool_[used_++];
}
void Profiler::start(cudaStream_t s) {
  if (!on_) return;
  pending_ = (int)used_;
  RTCC_CUDA(cudaEventRecord(get(), s));
}
void Profiler::stop(cudaStream_t s, int cls, double flops, double bytes, const char* tag) {
  ++count[cls];
  if (!on_) return;
  const int b = (int)used_;
  RTCC_CUDA(cudaEventRecord(get(), s));
  recs_.push_back(Rec{cls, pending_, b, flops, bytes, tag ? std::string(tag) : std::string()});
}
void Profiler::end(long long launches[KC_N], double ms[KC_N], double flops[KC_N], double bytes[KC_N]) {
  for (int c = 0; c < KC_N; ++c) {
    launches[c] = 0;
    ms[c] = flops[c] = bytes[c] = 0.0;
  }
  if (!recs_.empty()) RTCC_CUDA(cudaEventSynchronize(pool_[recs_.back().b]));
  const char* dump = std::getenv("RTCC_PROFILE_OPS");
  std::map<std::string, std::vector<double>> per;   // tag -> {class, launches, ms, flops, bytes}
  for (const Rec& r : recs_) {
    float t = 0.f;
    RTCC_CUDA(cudaEventElapsedTime(&t, pool_[r.a], pool_[r.b]));
    launches[r.cls] += 1;
    ms[r.cls] += t;
    flops[r.cls] += r.flops;
    bytes[r.cls] += r.bytes;
    if (dump) {
      auto& v = per[r.tag + "|" + std::to_string(r.cls)];
      if (v.empty()) v = {(double)r.cls, 0, 0, 0, 0};
      v[1] += 1;
      v[2] += t;
      v[3] += r.flops;
      v[4] += r.bytes;
    }
  }
  if (dump) {
    FILE* fp = std::fopen(dump, "w");
    if (fp) {
      std::fprintf(fp, "tag,class,launches,ms,flops,bytes\n");
      for (const auto& kv : per)
        std::fprintf(fp, "%s,%d,%.0f,%.4f,%.6g,%.6g\n", kv.first.substr(0, kv.first.rfind('|')).c_str(),
                     (int)kv.second[0], kv.second[1], kv.second[2], kv.second[3], kv.second[4]);
      std::fclose(fp);
    }
  }
  on_ = false;
  recs_.clear();
  used_ = 0;
}

static bool C_cplx_of(const Compiled& k) { return k.tcp.p.epi.c_cplx != 0; }

void* dev_alloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(2, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  return p;
}

Engine::Engine(Prec p, cudaStream_t s) : prec_(p), stream_(s) {
  dev_err_ = static_cast<int*>(dev_alloc(sizeof(int) * 4));
  allocs_.push_back(dev_err_);
  RTCC_CUDA(cudaMemsetAsync(dev_err_, 0, sizeof(int) * 4, stream_));
}

Engine::~Engine() {
  for (void* p : allocs_) cudaFree(p);
}

static std::vector<long long> contiguous_strides(const std::vector<int>& dims) {
  std::vector<long long> s(dims.size());
  long long acc = 1;
  for (int i = (int)dims.size() - 1; i >= 0; --i) {
    s[i] = acc;
    acc *= dims[i];
  }
  return s;
}

int Engine::external(const std::string& name, const std::vector<int>& dims, bool cplx, double* ptr,
                     std::vector<long long> strides, bool constant) {
  Tensor t;
  t.name = name;
  t.dims = dims;
  t.strides = strides.empty() ? contiguous_strides(dims) : strides;
  RTCC_REQUIRE(t.strides.size() == dims.size(), "stride rank mismatch for " + name);
  t.cplx = cplx;
  t.constant = constant;
  t.storage = ST_EXTERNAL;
  t.ptr = ptr;
  tensors_.push_back(t);
  return (int)tensors_.size() - 1;
}

int Engine::owned(const std::string& name, const std::vector<int>& dims, bool cplx, bool constant) {
  Tensor t;
  t.name = name;
  t.dims = dims;
  t.strides = contiguous_strides(dims);
  t.cplx = cplx;
  t.constant = constant;
  t.storage = ST_OWNED;
  const size_t bytes = (size_t)t.numel() * (cplx ? 16 : 8);
  t.ptr = static_cast<double*>(dev_alloc(bytes));
  allocs_.push_back(t.ptr);
  bytes_ += bytes;
  RTCC_CUDA(cudaMemsetAsync(t.ptr, 0, bytes, stream_));
  tensors_.push_back(t);
  return (int)tensors_.size() - 1;
}

int Engine::new_arena() {
  arena_size_.push_back(0);
  arena_hwm_.push_back(0);
  arena_ptr_.push_back(nullptr);
  return (int)arena_size_.size() - 1;
}

int Engine::temp(int arena, const std::string& name, const std::vector<int>& dims, bool cplx) {
  RTCC_REQUIRE(!finalized_, "engine already finalized");
  Tensor t;
  t.name = name;
  t.dims = dims;
  t.strides = contiguous_strides(dims);
  t.cplx = cplx;
  t.storage = ST_ARENA;
  // temporaries of reduced-precision engines hold float32 (complex64) elements: their
  // contractions resolve far less than float32 does, and every pass over them moves half the bytes
  t.f32 = (prec_ != Prec::P64);
  t.arena = arena;
  t.arena_off = arena_size_[arena];
  const long long nd = ((long long)(t.numel() * t.esz()) + 7) / 8;   // in doubles
  arena_size_[arena] += round_up(nd, 32);   // 256-byte alignment of every temporary
  tensors_.push_back(t);
  return (int)tensors_.size() - 1;
}

void Engine::ein(Program& P, int c, const std::string& lc, int a, const std::string& la, int b,
                 const std::string& lb, cplx alpha, bool pairsym) {
  P.ops.push_back(Op{OP_EIN, c, a, b, lc, la, lb, alpha, pairsym});
}

void Engine::add(Program& P, int c, const std::string& lc, int a, const std::string& la, cplx alpha) {
  P.ops.push_back(Op{OP_ADD, c, a, -1, lc, la, "", alpha});
}

Program Engine::reverse(const Program& fwd, const std::vector<int>& active_inputs, int arena,
                        std::map<int, int>& adj) {
  std::set<int> active(active_inputs.begin(), active_inputs.end());
  for (const Op& op : fwd.ops) {
    const bool act = (op.kind == OP_EIN) ? (active.count(op.a) || active.count(op.b)) : active.count(op.a) > 0;
    if (act) active.insert(op.c);
  }
  auto adj_of = [&](int id) {
    auto it = adj.find(id);
    if (it != adj.end()) return it->second;
    const Tensor& t = tensors_[id];
    const int d = temp(arena, "d_" + t.name, t.dims, true);
    adj[id] = d;
    return d;
  };
  for (int id : active) adj_of(id);
  Program R;
  R.name = fwd.name + "_vjp";
  R.zero_arenas = {arena};
  for (auto it = fwd.ops.rbegin(); it != fwd.ops.rend(); ++it) {
    const Op& op = *it;
    if (!active.count(op.c)) continue;
    const int dc = adj.at(op.c);
    if (op.kind == OP_EIN) {
      // the reverse of a pair-symmetric contraction keeps B and its symmetry
      if (active.count(op.a)) ein(R, adj.at(op.a), op.la, dc, op.lc, op.b, op.lb, op.alpha, op.pairsym);
      if (active.count(op.b)) ein(R, adj.at(op.b), op.lb, op.a, op.la, dc, op.lc, op.alpha);
    } else if (active.count(op.a)) {
      RTCC_REQUIRE(op.la.size() == op.lc.size(), "reverse of a broadcasting add of an active tensor");
      add(R, adj.at(op.a), op.la, dc, op.lc, op.alpha);
    }
  }
  return R;
}

void Engine::plan(Program& P) {
  P.comp.clear();
  const Prec prec = P.prec_override >= 0 ? (Prec)P.prec_override : prec_;
  // an arena temporary of an arena this program zeroes, not yet written by an earlier op of the
  // program, is known to be zero: its first writer stores instead of read-modify-writing
  // (tracked by arena extent, so temporaries that share reused arena space are never fresh twice)
  std::vector<std::array<long long, 3>> written;   // arena, first double, one past the last
  const std::set<int> zeroed(P.zero_arenas.begin(), P.zero_arenas.end());
  auto extent = [&](const Tensor& t) {   // arena, first byte, one past the last byte
    long long hi = 1;
    for (size_t i = 0; i < t.dims.size(); ++i) hi += (long long)(t.dims[i] - 1) * t.strides[i];
    return std::array<long long, 3>{t.arena, t.arena_off * 8, t.arena_off * 8 + hi * (long long)t.esz()};
  };
  auto fresh = [&](int id) {
    const Tensor& t = tensors_[id];
    if (t.storage != ST_ARENA || !zeroed.count(t.arena)) return false;
    const auto x = extent(t);
    for (const auto& w : written)
      if (w[0] == x[0] && w[1] < x[2] && x[1] < w[2]) return false;
    return true;
  };
  auto mark_written = [&](int id) {
    const Tensor& t = tensors_[id];
    if (t.storage == ST_ARENA) written.push_back(extent(t));
  };
  for (const Op& op : P.ops) {
    auto cp = std::make_shared<Compiled>();
    Compiled& k = *cp;
    const Tensor& C = tensors_[op.c];
    const Tensor& A = tensors_[op.a];
    RTCC_REQUIRE(op.lc.size() == C.dims.size(), "label/rank mismatch for output " + C.name + " in " + P.name);
    RTCC_REQUIRE(op.la.size() == A.dims.size(), "label/rank mismatch for " + A.name + " in " + P.name);
    RTCC_REQUIRE(C.cplx || (!A.cplx && (op.kind == OP_ADD || !tensors_[op.b].cplx)),
                 "complex result into real tensor " + C.name);
    RTCC_REQUIRE(!C.constant || P.name == "setup", "write to constant tensor " + C.name);
    const bool c_fresh = fresh(op.c);
    mark_written(op.c);
    if (op.kind == OP_ADD) {
      k.kind = CK_ADD;
      AddDesc& d = k.add;
      d.store = c_fresh ? 1 : 0;
      d.f32 = (prec != Prec::P64) ? 1 : 0;
      d.C = C.ptr;
      d.c_cplx = C.cplx;
      d.c_f32 = C.f32;
      d.c_all = map_for(C, op.lc, op.lc);
      d.n = prod_dims(d.c_all);
      d.nsrc = 0;
      add_source(k, P.ops, (int)P.comp.size(), op.lc);
      P.comp.push_back(cp);
      continue;
    }
    const Tensor& B = tensors_[op.b];
    RTCC_REQUIRE(op.lb.size() == B.dims.size(), "label/rank mismatch for " + B.name + " in " + P.name);
    std::string Lb, Lm, Ln, Lk;
    for (char l : op.lc) {
      const bool ina = op.la.find(l) != std::string::npos, inb = op.lb.find(l) != std::string::npos;
      RTCC_REQUIRE(ina || inb, std::string("output label only in output: ") + l + " in " + P.name);
      if (ina && inb) Lb += l;
      else if (ina) Lm += l;
      else Ln += l;
    }
    for (char l : op.la)
      if (op.lc.find(l) == std::string::npos) {
        RTCC_REQUIRE(op.lb.find(l) != std::string::npos, std::string("dangling label ") + l + " in " + P.name);
        Lk += l;
      }
    for (char l : op.lb)
      if (op.lc.find(l) == std::string::npos)
        RTCC_REQUIRE(op.la.find(l) != std::string::npos, std::string("dangling label ") + l + " in " + P.name);
    // label orders: M and N follow the output (the GEMM epilogue writes it in place), K follows the
    // larger operand that is packed every run; packs transpose through shared memory as needed
    Lm = by_stride(Lm, C, op.lc);
    Ln = by_stride(Ln, C, op.lc);
    {
      const bool use_a = !A.constant && (B.constant || A.numel() >= tensors_[op.b].numel());
      if (use_a) Lk = by_stride(Lk, A, op.la);
      else if (!tensors_[op.b].constant) Lk = by_stride(Lk, tensors_[op.b], op.lb);
    }
    // extent consistency
    auto ext = [&](const Tensor& t, const std::string& tl, char l) { return t.dims[tl.find(l)]; };
    for (char l : op.lc) {
      if (op.la.find(l) != std::string::npos)
        RTCC_REQUIRE(ext(A, op.la, l) == ext(C, op.lc, l), "extent mismatch " + A.name + "/" + C.name);
      if (op.lb.find(l) != std::string::npos)
        RTCC_REQUIRE(ext(B, op.lb, l) == ext(C, op.lc, l), "extent mismatch " + B.name + "/" + C.name);
    }
    for (char l : Lk) RTCC_REQUIRE(ext(A, op.la, l) == ext(B, op.lb, l), "K extent mismatch " + A.name + "/" + B.name);

    const long long NB = prod_dims(map_for(C, op.lc, Lb));
    const long long M = prod_dims(map_for(C, op.lc, Lm));
    const long long N = prod_dims(map_for(C, op.lc, Ln));
    const long long K = prod_dims(map_for(A, op.la, Lk));
    const int cfac = (A.cplx && B.cplx) ? 4 : ((A.cplx || B.cplx) ? 2 : 1);
    const long long work = NB * M * N * K * cfac;
    k.alg_flops = 2 * work;

    DirectDesc& d = k.dir;
    d.A = A.ptr;
    d.B = B.ptr;
    d.C = C.ptr;
    d.a_f32 = A.f32;
    d.b_f32 = B.f32;
    d.c_f32 = C.f32;
    d.a_cplx = A.cplx;
    d.b_cplx = B.cplx;
    d.c_cplx = C.cplx;
    d.am = map_for(A, op.la, Lm);
    d.ak = map_for(A, op.la, Lk);
    d.ab = map_for(A, op.la, Lb);
    d.bn = map_for(B, op.lb, Ln);
    d.bk = map_for(B, op.lb, Lk);
    d.bb = map_for(B, op.lb, Lb);
    d.cm = map_for(C, op.lc, Lm);
    d.cn = map_for(C, op.lc, Ln);
    d.cb = map_for(C, op.lc, Lb);
    d.M = M;
    d.N = N;
    d.K = K;
    d.NB = NB;
    d.ar = op.alpha.real();
    d.ai = op.alpha.imag();
    d.store = 0;
    d.f32 = (prec != Prec::P64) ? 1 : 0;

    const long long nout = NB * M * N;
    if (Lk.empty()) {
      k.kind = CK_DIRECT;
      d.store = c_fresh ? 1 : 0;
    } else if (force_gemm_) {
      k.kind = CK_GEMM;
    } else if (prec != Prec::P64 && K <= 32 && N <= 32 && M >= 4096 && !Lm.empty() &&
               A.strides[op.la.find(Lm.back())] == 1 && C.strides[op.lc.find(Lm.back())] == 1) {
      k.kind = CK_SKINNY;   // short K, few columns, many unit-stride rows: one thread per row
      d.store = c_fresh ? 1 : 0;
    } else if (prec != Prec::P64 && M <= 32 && N <= 32 && M * N <= 1024 && K >= 2048) {
      k.kind = CK_SMALLMN;   // few outputs per batch entry, long K: staged SIMT reduction
    } else if (nout <= kReduceMaxOut && K >= 256) {
      k.kind = CK_REDUCE;
      long long want = std::max(1ll, ((long long)device_sm_count() * 8) / std::max(1ll, nout));
      k.splits = std::max(1ll, std::min(want, (K + 1023) / 1024));
    } else if (work < kDirectMaxWork) {
      k.kind = CK_DIRECT;
      d.store = c_fresh ? 1 : 0;
    } else {
      k.kind = CK_GEMM;
    }
    if (k.kind == CK_GEMM && prec != Prec::P64 && op.pairsym &&
        plan_pairsym(k, op, Lm, Ln, Lk, Lb, d.am, d.cm, prec, c_fresh)) {
      // planned as two GEMMs over ordered pairs
    } else if (k.kind == CK_GEMM && prec != Prec::P64) {
      // tensor-core path: operands packed as planes (re/im x hi/lo), segment table per output plane
      const bool x3 = (prec == Prec::TF32X3 || prec == Prec::BF16X3);
      const int npart = x3 ? 2 : 1;
      const int elem = (prec == Prec::BF16X3) ? PE_BF16 : PE_F32;
      const int esz = (elem == PE_F32) ? 4 : 2;
      k.tc_kind = (prec == Prec::BF16X3) ? 1 : 0;
      k.chunk = accumulation_chunk(prec);
      const long long Kp = round_up(K, tc_kblock_elems(k.tc_kind));
      auto planes = [&](PackDesc& pd, const Tensor& T, const IndexMap& rows, const IndexMap& cols,
                        const IndexMap& bat, long long R) {
        pd = PackDesc{};
        pd.src = T.ptr;
        pd.src_cplx = T.cplx;
        pd.src_f32 = T.f32;
        pd.rows = rows;
        pd.cols = cols;
        pd.bat = bat;
        pd.R = R;
        pd.K = K;
        pd.NB = NB;
        const int nc = T.cplx ? 2 : 1;
        pd.nrb = nc * npart;
        pd.ncs = 1;
        pd.nss = 1;
        for (int c = 0; c < nc; ++c)
          for (int q = 0; q < npart; ++q) {
            const int rb = c * npart + q;
            pd.comp[rb][0] = c;
            pd.sign[rb][0] = 1;
            pd.rb_part[rb] = (npart == 1) ? SP_FULL : (q == 0 ? SP_HI : SP_LO);
          }
        pd.Kpad = Kp;
        pd.elem = elem;
        pd.round_tf32 = 1;
      };
      planes(k.pa, A, d.am, d.ak, d.ab, M);
      planes(k.pb, B, d.bn, d.bk, d.bb, N);
      choose_pack_mode(k.pa, A, op.la, Lm, Lk);
      choose_pack_mode(k.pb, B, op.lb, Ln, Lk);
      TcGemmParams& g = k.tcp.p;
      g = TcGemmParams{};
      g.nrb = (A.cplx || B.cplx) ? 2 : 1;
      auto pl = [&](int c, int q) { return c * npart + q; };
      auto pair = [&](int rb, int ca, int cb, int neg) {
        auto push = [&](int pa_, int pb_) {
          RTCC_REQUIRE(g.nseg[rb] < kMaxSeg, "too many GEMM segments");
          g.seg[rb][g.nseg[rb]++] = TcSeg{pa_, pb_, neg};
        };
        if (npart == 1) push(pl(ca, 0), pl(cb, 0));
        else {
          push(pl(ca, 0), pl(cb, 0));   // hi hi
          push(pl(ca, 0), pl(cb, 1));   // hi lo
          push(pl(ca, 1), pl(cb, 0));   // lo hi
        }
      };
      if (!A.cplx && !B.cplx) {
        pair(0, 0, 0, 0);
      } else if (A.cplx && !B.cplx) {
        pair(0, 0, 0, 0);
        pair(1, 1, 0, 0);
      } else if (!A.cplx && B.cplx) {
        pair(0, 0, 0, 0);
        pair(1, 0, 1, 0);
      } else {   // (Ar + i Ai)(Br + i Bi): re = Ar Br - Ai Bi, im = Ar Bi + Ai Br
        pair(0, 0, 0, 0);
        pair(0, 1, 1, 1);
        pair(1, 0, 1, 0);
        pair(1, 1, 0, 0);
      }
      RTCC_REQUIRE(op.alpha.imag() == 0.0, "tensor-core contractions take a real scale factor");
      TcEpilogue& ep = g.epi;
      ep.c_cplx = C.cplx;
      ep.c_f32 = C.f32;
      ep.alpha = op.alpha.real();
      ep.cm = d.cm;
      ep.cn = d.cn;
      ep.cb = d.cb;
      ep.flat_n = 1;
      for (int i = 0; i + 1 < ep.cn.n; ++i)
        if (ep.cn.strides[i] != ep.cn.strides[i + 1] * ep.cn.dims[i + 1]) ep.flat_n = 0;
      ep.sn = ep.cn.n ? ep.cn.strides[ep.cn.n - 1] : 0;
      ep.unit_n = (Ln.size() > 0 && !row_is_unit(C, op.lc, Lm, Ln)) ? 1 : 0;
      ep.store = c_fresh ? 1 : 0;
      k.Kpad = Kp;
      k.NB = NB;
      k.GM = (long long)k.pa.nrb * M;
      k.GN = (long long)k.pb.nrb * N;
      k.a_const = A.constant;
      k.b_const = B.constant;
      k.a_bytes = (size_t)(NB * k.GM * Kp * esz);
      k.b_bytes = (size_t)(NB * k.GN * Kp * esz);
      k.c_bytes = 0;
      k.exec_flops = 2 * NB * M * N * K * (long long)(g.nseg[0] + g.nseg[1]);
      if (!k.a_const) wsA_bytes_ = std::max(wsA_bytes_, k.a_bytes);
      if (!k.b_const) wsB_bytes_ = std::max(wsB_bytes_, k.b_bytes);
    } else if (k.kind == CK_GEMM) {
      const int nss = (prec == Prec::TF32X3 || prec == Prec::BF16X3) ? 3 : 1;
      const int elem = (prec == Prec::P64) ? PE_F64 : (prec == Prec::BF16X3 ? PE_BF16 : PE_F32);
      const int esz = (elem == PE_F64) ? 8 : (elem == PE_F32 ? 4 : 2);
      k.tc_kind = (prec == Prec::P64) ? -1 : (prec == Prec::BF16X3 ? 1 : 0);
      const long long kblk = (k.tc_kind < 0) ? 16 : tc_kblock_elems(k.tc_kind);
      PackDesc& pa = k.pa;
      PackDesc& pb = k.pb;
      pa = PackDesc{};
      pb = PackDesc{};
      pa.src = A.ptr;
      pa.src_cplx = A.cplx;
      pa.rows = d.am;
      pa.cols = d.ak;
      pa.bat = d.ab;
      pa.R = M;
      pa.K = K;
      pa.NB = NB;
      pb.src = B.ptr;
      pb.src_cplx = B.cplx;
      pb.rows = d.bn;
      pb.cols = d.bk;
      pb.bat = d.bb;
      pb.R = N;
      pb.K = K;
      pb.NB = NB;
      int mode = OM_REAL;
      auto set1 = [](PackDesc& p, int nrb, int ncs) {
        p.nrb = nrb;
        p.ncs = ncs;
        for (int r = 0; r < 2; ++r)
          for (int c = 0; c < 2; ++c) {
            p.comp[r][c] = 0;
            p.sign[r][c] = 1;
          }
      };
      if (!A.cplx && !B.cplx) {
        set1(pa, 1, 1);
        set1(pb, 1, 1);
      } else if (A.cplx && !B.cplx) {
        set1(pa, 2, 1);
        pa.comp[1][0] = 1;
        set1(pb, 1, 1);
        mode = OM_STACK_M;
      } else if (!A.cplx && B.cplx) {
        set1(pa, 1, 1);
        set1(pb, 2, 1);
        pb.comp[1][0] = 1;
        mode = OM_STACK_N;
      } else {
        PackDesc& ex = (M <= N) ? pa : pb;   // 2x2 real embedding on the side with fewer rows
        PackDesc& pl = (M <= N) ? pb : pa;
        set1(ex, 2, 2);
        ex.comp[0][0] = 0; ex.sign[0][0] = 1;
        ex.comp[0][1] = 1; ex.sign[0][1] = -1;
        ex.comp[1][0] = 1; ex.sign[1][0] = 1;
        ex.comp[1][1] = 0; ex.sign[1][1] = 1;
        set1(pl, 1, 2);
        pl.comp[0][1] = 1;
        mode = (M <= N) ? OM_STACK_M : OM_STACK_N;
      }
      pa.nss = pb.nss = nss;
      if (nss == 1) {
        pa.part[0] = pb.part[0] = SP_FULL;
      } else {
        pa.part[0] = SP_HI; pa.part[1] = SP_HI; pa.part[2] = SP_LO;
        pb.part[0] = SP_HI; pb.part[1] = SP_LO; pb.part[2] = SP_HI;
      }
      const long long Kp = round_up((long long)nss * pa.ncs * K, kblk);
      pa.Kpad = pb.Kpad = Kp;
      pa.elem = pb.elem = elem;
      pa.round_tf32 = pb.round_tf32 = 1;
      choose_pack_mode(pa, A, op.la, Lm, Lk);
      choose_pack_mode(pb, B, op.lb, Ln, Lk);
      k.GM = (long long)pa.nrb * M;
      k.GN = (long long)pb.nrb * N;
      k.Kpad = Kp;
      k.NB = NB;
      k.a_const = A.constant;
      k.b_const = B.constant;
      k.a_bytes = (size_t)(NB * k.GM * Kp * esz);
      k.b_bytes = (size_t)(NB * k.GN * Kp * esz);
      k.c_bytes = (size_t)(NB * k.GM * k.GN * (k.tc_kind < 0 ? 8 : 4));
      k.exec_flops = 2 * NB * k.GM * k.GN * Kp;
      UnpackDesc& u = k.up;
      u.gout_f64 = (k.tc_kind < 0);
      u.ldg = k.GN;
      u.rows_g = k.GM;
      u.mode = mode;
      u.M = M;
      u.N = N;
      u.NB = NB;
      u.cm = d.cm;
      u.cn = d.cn;
      u.cb = d.cb;
      u.C = C.ptr;
      u.c_cplx = C.cplx;
      u.ar = d.ar;
      u.ai = d.ai;
      u.transpose = row_is_unit(C, op.lc, Lm, Ln) ? 1 : 0;
      if (!k.a_const) wsA_bytes_ = std::max(wsA_bytes_, k.a_bytes);
      if (!k.b_const) wsB_bytes_ = std::max(wsB_bytes_, k.b_bytes);
      wsC_bytes_ = std::max(wsC_bytes_, k.c_bytes);
    }
    P.comp.push_back(cp);
  }
  merge_adds(P);
  share_packs(P);
}

namespace {
// Byte image of every field of a pack that decides its output (not the destination).
std::string pack_key(const PackDesc& d) {
  std::string k;
  auto put = [&](const void* p, size_t n) { k.append(static_cast<const char*>(p), n); };
  auto put_map = [&](const IndexMap& m) {
    put(&m.n, sizeof m.n);
    put(m.dims, sizeof(int) * m.n);
    put(m.strides, sizeof(long long) * m.n);
  };
  put(&d.src, sizeof d.src);
  put(&d.src_cplx, sizeof d.src_cplx);
  put(&d.src_f32, sizeof d.src_f32);
  put_map(d.rows);
  put_map(d.cols);
  put_map(d.bat);
  put(&d.R, sizeof d.R);
  put(&d.K, sizeof d.K);
  put(&d.NB, sizeof d.NB);
  put(&d.nrb, sizeof d.nrb);
  put(&d.ncs, sizeof d.ncs);
  put(&d.nss, sizeof d.nss);
  put(d.comp, sizeof d.comp);
  put(d.sign, sizeof d.sign);
  put(d.part, sizeof d.part);
  put(d.rb_part, sizeof d.rb_part);
  put(&d.Kpad, sizeof d.Kpad);
  put(&d.elem, sizeof d.elem);
  put(&d.round_tf32, sizeof d.round_tf32);
  put(&d.transpose, sizeof d.transpose);
  if (d.transpose) {
    put_map(d.rd_src);
    put_map(d.rd_dst);
  }
  put(&d.ktab, sizeof d.ktab);
  put(&d.kw, sizeof d.kw);
  put(&d.ksign, sizeof d.ksign);
  put(&d.rtab, sizeof d.rtab);
  return k;
}
}  // namespace

// A non-constant tensor-core operand packed by an earlier GEMM of the same program with an
// identical pack, whose source no op in between (nor that GEMM itself) has written, is not
// packed again: the later GEMM reads the earlier one's planes.
void Engine::share_packs(Program& P) {
  const size_t n = P.ops.size();
  auto range = [&](int id) {
    const Tensor& t = tensors_[id];
    long long hi = 1;
    for (size_t q = 0; q < t.dims.size(); ++q) hi += (long long)(t.dims[q] - 1) * std::llabs(t.strides[q]);
    const char* b = reinterpret_cast<const char*>(t.ptr);
    return std::make_pair(b, b + hi * (long long)t.esz());
  };
  auto overlaps = [&](int x, int y) {
    const auto a = range(x), b = range(y);
    return a.first < b.second && b.first < a.second;
  };
  for (size_t i = 0; i < n; ++i) {
    Compiled& k = *P.comp[i];
    if (k.kind != CK_GEMM || k.tc_kind < 0 || k.twin) continue;
    for (int side = 0; side < 2; ++side) {
      const bool cst = side ? k.b_const : k.a_const;
      if (cst) continue;
      const PackDesc& pd = side ? k.pb : k.pa;
      const int src = side ? P.ops[i].b : P.ops[i].a;
      const std::string key = pack_key(pd);
      for (size_t j = i; j-- > 0;) {
        // the source must not change between the provider's pack and this one
        if (P.comp[j]->kind != CK_MERGED && overlaps(P.ops[j].c, src)) break;
        Compiled& g = *P.comp[j];
        if (g.kind != CK_GEMM || g.tc_kind < 0 || g.twin) continue;
        bool hit = false, from_b = false;
        if (!g.a_const && !g.pa_from && pack_key(g.pa) == key) hit = true;
        else if (!g.b_const && !g.pb_from && pack_key(g.pb) == key) hit = from_b = true;
        if (!hit) continue;
        if (from_b) g.pb_keep = true;
        else g.pa_keep = true;
        if (side) {
          k.pb_from = &g;
          k.pb_from_b = from_b;
        } else {
          k.pa_from = &g;
          k.pa_from_b = from_b;
        }
        break;
      }
    }
  }
}

// Source `oi` (an add into the output of kernel k) expressed in the labels `lc` that k uses for
// its output: the op's own output labels are renamed position by position onto lc.
bool Engine::add_source(Compiled& k, const std::vector<Op>& ops, int oi, const std::string& lc) {
  AddDesc& d = k.add;
  if (d.nsrc >= kMaxAddSrc) return false;
  const Op& op = ops[oi];
  const Tensor& C = tensors_[op.c];
  const Tensor& A = tensors_[op.a];
  std::string la = op.la;
  if (op.lc != lc) {
    for (size_t x = 0; x < op.lc.size(); ++x)
      for (size_t y = x + 1; y < op.lc.size(); ++y)
        if (op.lc[x] == op.lc[y]) return false;   // repeated output labels: no renaming
    for (char& l : la) {
      const size_t p = op.lc.find(l);
      if (p == std::string::npos) return false;
      l = lc[p];
    }
  }
  for (char l : la) RTCC_REQUIRE(lc.find(l) != std::string::npos, "add reduces a label: " + A.name);
  const int q = d.nsrc;
  d.a_cplx[q] = A.cplx;
  d.a_all[q] = d.c_all;
  for (int i = 0; i < d.c_all.n; ++i) {
    const size_t p = la.find(lc[i]);
    if (p == std::string::npos) d.a_all[q].strides[i] = 0;
    else {
      RTCC_REQUIRE(A.dims[p] == C.dims[i], "extent mismatch in add " + A.name + " -> " + C.name);
      d.a_all[q].strides[i] = A.strides[p];
    }
  }
  d.A[q] = A.ptr;
  d.a_f32[q] = A.f32;
  d.ar[q] = op.alpha.real();
  d.ai[q] = op.alpha.imag();
  d.nsrc = q + 1;
  k.add_ops.push_back(oi);
  return true;
}

// Within a run of consecutive adds that neither read what the run writes nor write what it reads,
// adds into the same output become one kernel that reads each source once and writes the output once.
void Engine::merge_adds(Program& P) {
  const size_t n = P.ops.size();
  for (size_t i = 0; i < n;) {
    if (P.ops[i].kind != OP_ADD) {
      ++i;
      continue;
    }
    size_t j = i;
    std::set<int> wr, rd;
    while (j < n && P.ops[j].kind == OP_ADD) {
      wr.insert(P.ops[j].c);
      rd.insert(P.ops[j].a);
      ++j;
    }
    // independence by address range, so that views of one buffer count as the same data
    auto range = [&](int id) {
      const Tensor& t = tensors_[id];
      long long hi = 1;
      for (size_t q = 0; q < t.dims.size(); ++q) hi += (long long)(t.dims[q] - 1) * std::llabs(t.strides[q]);
      const char* b = reinterpret_cast<const char*>(t.ptr);
      return std::make_pair(b, b + hi * (long long)t.esz());
    };
    bool indep = true;
    for (int w : wr)
      for (int r : rd) {
        const auto x = range(w), y = range(r);
        if (x.first < y.second && y.first < x.second) indep = false;
      }
    if (indep) {
      for (size_t h = i; h < j; ++h) {
        Compiled& head = *P.comp[h];
        if (head.kind != CK_ADD) continue;
        for (size_t r = h + 1; r < j; ++r) {
          if (P.comp[r]->kind != CK_ADD || P.ops[r].c != P.ops[h].c) continue;
          if (add_source(head, P.ops, (int)r, P.ops[h].lc)) P.comp[r]->kind = CK_MERGED;
        }
      }
    }
    i = j;
  }
}

void Engine::bind(Program& P) {
  for (size_t i = 0; i < P.ops.size(); ++i) {
    const Op& op = P.ops[i];
    Compiled& k = *P.comp[i];
    // pointers of arena tensors are known only now
    const Tensor& C = tensors_[op.c];
    const Tensor& A = tensors_[op.a];
    if (k.kind == CK_ADD) {
      k.add.C = C.ptr;
      for (size_t q = 0; q < k.add_ops.size(); ++q) k.add.A[q] = tensors_[P.ops[k.add_ops[q]].a].ptr;
      continue;
    }
    if (k.kind == CK_MERGED) continue;
    const Tensor& B = tensors_[op.b];
    k.dir.A = A.ptr;
    k.dir.B = B.ptr;
    k.dir.C = C.ptr;
    if (k.kind != CK_GEMM) continue;
    bind_gemm(k, A, B, C);
    if (k.twin) bind_gemm(*k.twin, A, B, C);
  }
}

void Engine::bind_gemm(Compiled& k, const Tensor& A, const Tensor& B, const Tensor& C) {
  k.pa.src = A.ptr;
  k.pb.src = B.ptr;
  k.up.C = C.ptr;
  auto own = [&](size_t bytes) {
    void* p = dev_alloc(bytes);
    allocs_.push_back(p);
    bytes_ += bytes;
    return p;
  };
  // constant operands are packed once per distinct pack (programs built for several batch sizes
  // share them: a constant's pack does not depend on the number of trajectories)
  auto const_pack = [&](PackDesc& pd, size_t bytes) {
    const std::string key = pack_key(pd);
    auto it = const_packs_.find(key);
    if (it != const_packs_.end()) return it->second;
    void* p = own(bytes);
    pd.dst = p;
    launch_pack(pd, stream_);
    const_packs_[key] = p;
    return p;
  };
  if (k.a_const) {
    k.a_pre = const_pack(k.pa, k.a_bytes);
    k.pa.dst = k.a_pre;
  } else if (k.pa_from) {
    k.pa.dst = k.pa_from_b ? k.pa_from->pb.dst : k.pa_from->pa.dst;
  } else {
    k.pa.dst = k.pa_keep ? own(k.a_bytes) : wsA_;
  }
  if (k.b_const) {
    k.b_pre = const_pack(k.pb, k.b_bytes);
    k.pb.dst = k.b_pre;
  } else if (k.pb_from) {
    k.pb.dst = k.pb_from_b ? k.pb_from->pb.dst : k.pb_from->pa.dst;
  } else {
    k.pb.dst = k.pb_keep ? own(k.b_bytes) : wsB_;
  }
  k.up.gout = wsC_;
  if (k.tc_kind >= 0) {
    k.tcp.p.epi.C = C.ptr;
    tc_gemm_plan(k.tcp, k.tc_kind, k.pa.dst, k.pa.nrb, k.pb.dst, k.pb.nrb, k.pa.R, k.pb.R, k.Kpad, k.NB, dev_err_, 0,
                 k.chunk);
  }
}

// Index tables are uploaded once per distinct content, so that identical plans (the same
// contraction planned for several batch sizes) refer to the same tables and share packs.
const long long* Engine::upload(const std::vector<long long>& v) {
  std::string key("L");
  key.append(reinterpret_cast<const char*>(v.data()), v.size() * sizeof(long long));
  auto it = tables_.find(key);
  if (it != tables_.end()) return static_cast<const long long*>(it->second);
  void* p = dev_alloc(std::max<size_t>(1, v.size()) * sizeof(long long));
  allocs_.push_back(p);
  bytes_ += v.size() * sizeof(long long);
  RTCC_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(long long), cudaMemcpyHostToDevice));
  tables_[key] = p;
  return static_cast<const long long*>(p);
}
const float* Engine::upload(const std::vector<float>& v) {
  std::string key("F");
  key.append(reinterpret_cast<const char*>(v.data()), v.size() * sizeof(float));
  auto it = tables_.find(key);
  if (it != tables_.end()) return static_cast<const float*>(it->second);
  void* p = dev_alloc(std::max<size_t>(1, v.size()) * sizeof(float));
  allocs_.push_back(p);
  bytes_ += v.size() * sizeof(float);
  RTCC_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice));
  tables_[key] = p;
  return static_cast<const float*>(p);
}

// Pair-symmetric contraction C[m, n1, n2] += alpha sum_{k1,k2} A[m, k1, k2] V[n1, n2, k1, k2] with
// V[n1,n2,k1,k2] = V[n2,n1,k2,k1] (the particle-particle ladder with V = (ae|bf) and its reverse).
// Over ordered pairs p <= q of the contracted labels and x <= y of the kept ones,
//   A^s[m, pq] = A[m,p,q] + s A[m,q,p],   V^s[xy, pq] = w_pq (V[x,y,p,q] + s V[x,y,q,p]) / 2,
//   w_pq = 1 - delta_pq / 2,   P^s = A^s V^s^T   (s = +1, -1),
// and C[m,x,y] += P^+ + P^-, C[m,y,x] += P^+ - P^- (x < y): the sum over all (p, q) regrouped by
// the symmetry, with half the multiply-adds.  Two GEMMs; the second target of each output column
// and its sign are applied in the epilogue.  Returns false (generic path) when the shape does not fit.
bool Engine::plan_pairsym(Compiled& k, const Op& op, const std::string& Lm, const std::string& Ln,
                          const std::string& Lk, const std::string& Lb, const IndexMap& am, const IndexMap& cm,
                          Prec prec, bool c_fresh) {
  const Tensor& A = tensors_[op.a];
  const Tensor& B = tensors_[op.b];
  const Tensor& C = tensors_[op.c];
  const std::string& lb = op.lb;
  if (!Lb.empty() || Ln.size() != 2 || Lk.size() != 2 || lb.size() != 4 || B.cplx || !B.constant ||
      op.alpha.imag() != 0.0)
    return false;
  auto same_set = [](const std::string& pr, const std::string& L) {
    return (pr[0] == L[0] && pr[1] == L[1]) || (pr[0] == L[1] && pr[1] == L[0]);
  };
  std::string pn, pk;   // the kept and the contracted pair, each in B's label order
  if (same_set(lb.substr(0, 2), Ln) && same_set(lb.substr(2, 2), Lk)) {
    pn = lb.substr(0, 2);
    pk = lb.substr(2, 2);
  } else if (same_set(lb.substr(0, 2), Lk) && same_set(lb.substr(2, 2), Ln)) {
    pk = lb.substr(0, 2);
    pn = lb.substr(2, 2);
  } else {
    return false;
  }
  auto dimB = [&](char l) { return B.dims[lb.find(l)]; };
  auto strB = [&](char l) { return B.strides[lb.find(l)]; };
  const int dn = dimB(pn[0]), dk = dimB(pk[0]);
  if (dimB(pn[1]) != dn || dimB(pk[1]) != dk) return false;
  const long long Np = (long long)dn * (dn + 1) / 2, Kt = (long long)dk * (dk + 1) / 2;
  const long long M = prod_dims(am);
  const long long sa1 = A.strides[op.la.find(pk[0])], sa2 = A.strides[op.la.find(pk[1])];
  const long long sc1 = C.strides[op.lc.find(pn[0])], sc2 = C.strides[op.lc.find(pn[1])];
  const long long sv1 = strB(pn[0]), sv2 = strB(pn[1]), sk1 = strB(pk[0]), sk2 = strB(pk[1]);
  std::vector<long long> ka(2 * Kt), kv(2 * Kt), rv(Np), c1(Np), c2(Np);
  std::vector<float> wv(Kt);
  long long t = 0;
  for (int x = 0; x < dk; ++x)
    for (int y = x; y < dk; ++y, ++t) {
      ka[2 * t] = x * sa1 + y * sa2;
      ka[2 * t + 1] = y * sa1 + x * sa2;
      kv[2 * t] = x * sk1 + y * sk2;
      kv[2 * t + 1] = y * sk1 + x * sk2;
      wv[t] = (x == y) ? 0.25f : 0.5f;
    }
  t = 0;
  for (int x = 0; x < dn; ++x)
    for (int y = x; y < dn; ++y, ++t) {
      rv[t] = x * sv1 + y * sv2;
      c1[t] = x * sc1 + y * sc2;
      c2[t] = (x == y) ? -1 : y * sc1 + x * sc2;
    }
  const long long* ka_d = upload(ka);
  const long long* kv_d = upload(kv);
  const long long* rv_d = upload(rv);
  const long long* c1_d = upload(c1);
  const long long* c2_d = upload(c2);
  const float* wv_d = upload(wv);

  const bool x3 = (prec == Prec::TF32X3 || prec == Prec::BF16X3);
  const int npart = x3 ? 2 : 1;
  const int elem = (prec == Prec::BF16X3) ? PE_BF16 : PE_F32;
  const int esz = (elem == PE_F32) ? 4 : 2;
  const int kind = (prec == Prec::BF16X3) ? 1 : 0;
  const long long Kpad = round_up(Kt, tc_kblock_elems(kind));
  auto planes = [&](PackDesc& pd, const Tensor& T, long long R, int sign) {
    pd = PackDesc{};
    pd.src = T.ptr;
    pd.src_cplx = T.cplx;
    pd.src_f32 = T.f32;
    pd.R = R;
    pd.K = Kt;
    pd.NB = 1;
    const int nc = T.cplx ? 2 : 1;
    pd.nrb = nc * npart;
    pd.ncs = 1;
    pd.nss = 1;
    for (int c = 0; c < nc; ++c)
      for (int q = 0; q < npart; ++q) {
        const int rb = c * npart + q;
        pd.comp[rb][0] = c;
        pd.sign[rb][0] = 1;
        pd.rb_part[rb] = (npart == 1) ? SP_FULL : (q == 0 ? SP_HI : SP_LO);
      }
    pd.Kpad = Kpad;
    pd.elem = elem;
    pd.round_tf32 = 1;
    pd.transpose = 0;
    pd.ksign = (float)sign;
  };
  auto build = [&](Compiled& g, int sign) {
    g.kind = CK_GEMM;
    g.tc_kind = kind;
    g.chunk = accumulation_chunk(prec);
    planes(g.pa, A, M, sign);
    g.pa.rows = am;
    g.pa.ktab = ka_d;
    planes(g.pb, B, Np, sign);
    g.pb.rtab = rv_d;
    g.pb.ktab = kv_d;
    g.pb.kw = wv_d;
    TcGemmParams& gp = g.tcp.p;
    gp = TcGemmParams{};
    gp.nrb = A.cplx ? 2 : 1;
    auto pl = [&](int c, int q) { return c * npart + q; };
    auto pair = [&](int rb, int ca) {
      auto push = [&](int pa_, int pb_) { gp.seg[rb][gp.nseg[rb]++] = TcSeg{pa_, pb_, 0}; };
      if (npart == 1) push(pl(ca, 0), pl(0, 0));
      else {
        push(pl(ca, 0), pl(0, 0));
        push(pl(ca, 0), pl(0, 1));
        push(pl(ca, 1), pl(0, 0));
      }
    };
    pair(0, 0);
    if (A.cplx) pair(1, 1);
    TcEpilogue& ep = gp.epi;
    ep.c_cplx = C.cplx;
    ep.c_f32 = C.f32;
    ep.alpha = op.alpha.real();
    ep.cm = cm;
    ep.cb = IndexMap{};
    ep.flat_n = 0;
    ep.unit_n = (sc1 == 1 || sc2 == 1) ? 1 : 0;
    ep.store = (sign > 0 && c_fresh) ? 1 : 0;   // the + part writes every element once
    ep.ctab1 = c1_d;
    ep.ctab2 = c2_d;
    ep.sign2 = (float)sign;
    g.Kpad = Kpad;
    g.NB = 1;
    g.GM = (long long)g.pa.nrb * M;
    g.GN = (long long)g.pb.nrb * Np;
    g.a_const = A.constant;
    g.b_const = true;
    g.a_bytes = (size_t)(g.GM * Kpad * esz);
    g.b_bytes = (size_t)(g.GN * Kpad * esz);
    g.exec_flops = 2 * M * Np * Kt * (long long)(gp.nseg[0] + gp.nseg[1]);
    if (!g.a_const) wsA_bytes_ = std::max(wsA_bytes_, g.a_bytes);
  };
  build(k, +1);
  k.twin = std::make_shared<Compiled>();
  build(*k.twin, -1);
  return true;
}

void Engine::finalize(std::vector<Program*> progs) {
  RTCC_REQUIRE(!finalized_, "engine finalized twice");
  for (size_t a = 0; a < arena_size_.size(); ++a) {
    arena_size_[a] = std::max(arena_size_[a], arena_hwm_[a]);
    const size_t bytes = (size_t)std::max(1ll, arena_size_[a]) * 8;
    arena_ptr_[a] = static_cast<double*>(dev_alloc(bytes));
    allocs_.push_back(arena_ptr_[a]);
    bytes_ += bytes;
    RTCC_CUDA(cudaMemsetAsync(arena_ptr_[a], 0, bytes, stream_));
  }
  for (Tensor& t : tensors_)
    if (t.storage == ST_ARENA) t.ptr = arena_ptr_[t.arena] + t.arena_off;
  for (Program* P : progs) plan(*P);
  auto alloc_ws = [&](void*& p, size_t bytes) {
    if (bytes == 0) return;
    p = dev_alloc(bytes);
    allocs_.push_back(p);
    bytes_ += bytes;
  };
  alloc_ws(wsA_, wsA_bytes_);
  alloc_ws(wsB_, wsB_bytes_);
  alloc_ws(wsC_, wsC_bytes_);
  for (Program* P : progs) bind(*P);
  RTCC_CUDA(cudaStreamSynchronize(stream_));
  finalized_ = true;
}

void Engine::run(const Program& P) {
  for (int a : P.zero_arenas)
    RTCC_CUDA(cudaMemsetAsync(arena_ptr_[a], 0, (size_t)std::max(1ll, arena_size_[a]) * 8, stream_));
  for (int t : P.zero_tensors) {
    const Tensor& x = tensors_[t];
    RTCC_CUDA(cudaMemsetAsync(x.ptr, 0, (size_t)x.numel() * x.esz(), stream_));
  }
  for (const auto& z : P.zero2d) RTCC_CUDA(cudaMemset2DAsync(z.ptr, z.pitch, 0, z.width, z.height, stream_));
  Profiler dummy;
  Profiler& pr = prof_ ? *prof_ : dummy;
  std::string tagbuf;
  for (size_t oi = 0; oi < P.comp.size(); ++oi) {
    const Compiled& k = *P.comp[oi];
    const char* tag = nullptr;
    if (pr.on()) {
      const Op& op = P.ops[oi];
      tagbuf = P.name + "#" + std::to_string(oi) + " " + tensors_[op.c].name + "[" + op.lc + "]<-" +
               tensors_[op.a].name + "[" + op.la + "]" + (op.kind == OP_EIN ? "*" + tensors_[op.b].name + "[" + op.lb + "]" : "");
      tag = tagbuf.c_str();
    }
    switch (k.kind) {
      case CK_MERGED:
        break;
      case CK_ADD: {
        double abytes = 0.0;
        for (int q = 0; q < k.add.nsrc; ++q) abytes += (k.add.a_cplx[q] ? 2 : 1) * (k.add.a_f32[q] ? 4 : 8);
        const double cbytes = (k.add.c_cplx ? 2 : 1) * (k.add.c_f32 ? 4 : 8);
        pr.start(stream_);
        launch_add(k.add, stream_);
        pr.stop(stream_, KC_ADD, 0.0, (double)k.add.n * (abytes + (k.add.store ? 1 : 2) * cbytes), tag);
        break;
      }
      case CK_DIRECT:
        pr.start(stream_);
        launch_direct(k.dir, stream_);
        pr.stop(stream_, KC_DIRECT, (double)k.alg_flops, 0.0, tag);
        break;
      case CK_REDUCE:
        pr.start(stream_);
        launch_reduce(k.dir, k.splits, stream_);
        pr.stop(stream_, KC_REDUCE, (double)k.alg_flops, 0.0, tag);
        break;
      case CK_SMALLMN:
        pr.start(stream_);
        launch_smallmn(k.dir, stream_);
        pr.stop(stream_, KC_REDUCE, (double)k.alg_flops, 0.0, tag);
        break;
      case CK_SKINNY:
        pr.start(stream_);
        launch_skinny(k.dir, stream_);
        pr.stop(stream_, KC_DIRECT, (double)k.alg_flops, 0.0, tag);
        break;
      default:
        run_gemm(k, pr, tag);
        if (k.twin) run_gemm(*k.twin, pr, tag);
    }
  }
}

void Engine::run_gemm(const Compiled& k, Profiler& pr, const char* tag) {
  const double esz = (k.pa.elem == PE_F64) ? 8 : (k.pa.elem == PE_F32 ? 4 : 2);
  if (!k.a_const && !k.pa_from) {
    pr.start(stream_);
    launch_pack(k.pa, stream_);
    pr.stop(stream_, KC_PACK, 0.0,
            (double)k.NB * k.pa.R * k.pa.K * (k.pa.src_cplx ? 2 : 1) * (k.pa.src_f32 ? 4 : 8) + (double)k.NB * k.GM * k.Kpad * esz, tag);
  }
  if (!k.b_const && !k.pb_from) {
    pr.start(stream_);
    launch_pack(k.pb, stream_);
    pr.stop(stream_, KC_PACK, 0.0,
            (double)k.NB * k.pb.R * k.pb.K * (k.pb.src_cplx ? 2 : 1) * (k.pb.src_f32 ? 4 : 8) + (double)k.NB * k.GN * k.Kpad * esz, tag);
  }
  if (k.tc_kind >= 0) {
    // kernel-level algorithmic flops: real multiply-adds of all segments, without padding
    pr.start(stream_);
    launch_tc_gemm(k.tcp, stream_);
    pr.stop(stream_, KC_TC_GEMM, (double)k.exec_flops,
            (double)k.NB * (k.GM + k.GN) * k.Kpad * esz + 2.0 * k.NB * k.pa.R * k.pb.R * (C_cplx_of(k) ? 2 : 1) * (k.tcp.p.epi.c_f32 ? 4 : 8), tag);
    return;
  }
  const double kflops = 2.0 * k.NB * k.GM * k.GN * (double)(k.pa.nss * k.pa.ncs * k.pa.K);
  pr.start(stream_);
  launch_gemm_f64(static_cast<const double*>(k.pa.dst), static_cast<const double*>(k.pb.dst),
                  static_cast<double*>(wsC_), k.GM, k.GN, k.Kpad, k.NB, stream_);
  pr.stop(stream_, KC_F64_GEMM, kflops,
          (double)k.NB * (k.GM + k.GN) * k.Kpad * esz + (double)k.NB * k.GM * k.GN * 8, tag);
  pr.start(stream_);
  launch_unpack(k.up, stream_);
  pr.stop(stream_, KC_UNPACK, 0.0,
          (double)k.NB * k.GM * k.GN * (k.tc_kind >= 0 ? 4 : 8) + 2.0 * k.NB * k.up.M * k.up.N * (k.up.c_cplx ? 16 : 8), tag);
}

int Engine::autotune(Program& P) {
  if (P.tuned) return 0;
  P.tuned = true;
  cudaEvent_t e0, e1;
  RTCC_CUDA(cudaEventCreate(&e0));
  RTCC_CUDA(cudaEventCreate(&e1));
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev{e0, e1};
  int changed = 0;
  for (auto& cp : P.comp)
    for (Compiled* g = cp.get(); g; g = g->twin.get()) {
      if (g->kind != CK_GEMM || g->tc_kind < 0) continue;
      const TcGemmParams& q = g->tcp.p;
      const long long M = g->pa.R, N = g->pb.R;
      const std::string key = std::to_string(g->tc_kind) + ":" + std::to_string(M) + ":" + std::to_string(N) + ":" +
                              std::to_string(g->Kpad) + ":" + std::to_string(g->NB) + ":" + std::to_string(q.nrb) +
                              ":" + std::to_string(q.nseg[0]) + ":" + std::to_string(q.nseg[1]) + ":" +
                              std::to_string(g->pa.nrb) + ":" + std::to_string(g->pb.nrb) + ":" +
                              std::to_string(q.epi.c_cplx) + ":" + std::to_string(q.epi.unit_n) + ":" +
                              std::to_string(q.epi.ctab1 != nullptr) + ":" + std::to_string(g->chunk);
      int best = 0;
      auto it = tile_cache_.find(key);
      if (it != tile_cache_.end()) {
        best = it->second;
      } else {
        float tbest = 0.f;
        // candidates (code 4 * bn + variant): N tiles of 64, 128 and 256 columns; the 256 tile with
        // three stages and eight epilogue warps (a faster chunk fold, a shallower pipeline); the 128
        // and 256 tiles with two K blocks per pipeline stage
        for (int cand : {256, 512, 514, 1024, 1025, 1026}) {
          const int bn = cand / 4, var = cand & 3;
          if (bn > 64 && N <= bn / 2) continue;   // a tile twice as wide as N or more
          TcGemmPlan trial = g->tcp;
          tc_gemm_plan(trial, g->tc_kind, g->pa.dst, g->pa.nrb, g->pb.dst, g->pb.nrb, M, N, g->Kpad, g->NB, dev_err_, bn,
                       g->chunk);
          if (trial.bn != bn) continue;           // not usable for this item kind
          if (var == 2 && !trial.pair_maps) continue;
          trial.variant = var;
          launch_tc_gemm(trial, stream_);
          float tmin = 0.f;
          for (int r = 0; r < 3; ++r) {
            RTCC_CUDA(cudaEventRecord(e0, stream_));
            launch_tc_gemm(trial, stream_);
            RTCC_CUDA(cudaEventRecord(e1, stream_));
            RTCC_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            RTCC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (r == 0 || ms < tmin) tmin = ms;
          }
          if (best == 0 || tmin < tbest) {
            tbest = tmin;
            best = cand;
          }
        }
        tile_cache_[key] = best;
      }
      if (best != 0 && best != 4 * g->tcp.bn + g->tcp.variant) {
        tc_gemm_plan(g->tcp, g->tc_kind, g->pa.dst, g->pa.nrb, g->pb.dst, g->pb.nrb, M, N, g->Kpad, g->NB, dev_err_,
                     best / 4, g->chunk);
        g->tcp.variant = best & 3;
        ++changed;
      }
    }
  check_error();
  return changed;
}

EngineStats Engine::stats_of(const Program& P) const {
  EngineStats s;
  for (const auto& cp : P.comp) {
    if (cp->kind == CK_MERGED) continue;
    if (cp->kind == CK_GEMM) {
      s.gemm_flops += cp->alg_flops;
      // packs of non-constant operands, the GEMM, and the unpack of the float64 SIMT path
      for (const Compiled* g = cp.get(); g; g = g->twin.get())
        s.launches += (g->tc_kind >= 0 ? 1 : 2) + (g->a_const || g->pa_from ? 0 : 1) + (g->b_const || g->pb_from ? 0 : 1);
    } else {
      s.direct_flops += cp->alg_flops;
      s.launches += 1;
    }
  }
  s.launches += (int)(P.zero_arenas.size() + P.zero_tensors.size() + P.zero2d.size());
  return s;
}

void Engine::check_error() {
  int h = 0;
  RTCC_CUDA(cudaMemcpyAsync(&h, dev_err_, sizeof(int), cudaMemcpyDeviceToHost, stream_));
  RTCC_CUDA(cudaStreamSynchronize(stream_));
  if (h != DEV_OK) {
    RTCC_CUDA(cudaMemsetAsync(dev_err_, 0, sizeof(int), stream_));
    throw Error(7, "a tensor-core GEMM wait expired on the device (code " + std::to_string(h) + ")");
  }
}

}  // namespace rtcc
