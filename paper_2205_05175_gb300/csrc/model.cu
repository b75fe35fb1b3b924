// RT-CCSD model programs: integral blocks, closed-shell ket residual (Eq. derivT),
// its reverse-mode vector-Jacobian program (Eq. derivL), the dipole (Eq. dipole) and
// the correlation energy.
//
// Closed-shell conventions: t1[i][a] is the (i alpha -> a alpha) amplitude and
// t2[i][j][a][b] the (i alpha j beta -> a alpha b beta) amplitude; the residual
// components are the same spin blocks of <mu|e^{-T} H e^{T}|0>, written with
// Stanton-Gauss intermediates spin-integrated for a general (field-dressed,
// non-diagonal) Fock matrix.  Integrals: v[p][q][r][s] = <pq|rs> = (pr|qs).
// Index letters: z trajectory, x dipole component, P auxiliary, i j m n occupied,
// a b e f virtual.
#include "model.cuh"
#include <set>

namespace rtcc {

IntegralStore::~IntegralStore() {
  for (void* p : owned) cudaFree(p);
}

void build_integrals(IntegralStore& S, const double* dB, int naux, int o, int v, cudaStream_t stream) {
  S.o = o;
  S.v = v;
  S.naux = naux;
  const int n = o + v;
  Engine E(Prec::P64, stream);
  auto alloc = [&](int b, std::vector<int> dims) {
    long long ne = 1;
    for (int d : dims) ne *= d;
    const size_t bytes = (size_t)ne * 8;
    S.blk[b] = static_cast<double*>(dev_alloc(bytes));
    S.owned.push_back(S.blk[b]);
    S.bytes += bytes;
    RTCC_CUDA(cudaMemsetAsync(S.blk[b], 0, bytes, stream));
    return E.external("int" + std::to_string(b), dims, false, S.blk[b]);
  };
  using B = IntegralStore;
  double* Bp = const_cast<double*>(dB);
  const long long sP = (long long)n * n;
  const int Boo = E.external("Boo", {naux, o, o}, false, Bp, {sP, n, 1}, true);
  const int Bov = E.external("Bov", {naux, o, v}, false, Bp + o, {sP, n, 1}, true);
  const int Bvo = E.external("Bvo", {naux, v, o}, false, Bp + (size_t)o * n, {sP, n, 1}, true);
  const int Bvv = E.external("Bvv", {naux, v, v}, false, Bp + (size_t)o * n + o, {sP, n, 1}, true);
  const int oooo = alloc(B::OOOO, {o, o, o, o});
  const int ooov = alloc(B::OOOV, {o, o, o, v});
  const int oovo = alloc(B::OOVO, {o, o, v, o});
  const int oovv = alloc(B::OOVV, {o, o, v, v});
  const int ovov = alloc(B::OVOV, {o, v, o, v});
  const int ovvo = alloc(B::OVVO, {o, v, v, o});
  const int ovoo = alloc(B::OVOO, {o, v, o, o});
  const int ovvv = alloc(B::OVVV, {o, v, v, v});
  const int vvvo = alloc(B::VVVO, {v, v, v, o});
  const int vvvv = alloc(B::VVVV, {v, v, v, v});
  const int Lovvv = alloc(B::LOVVV, {o, v, v, v});
  const int Loovv = alloc(B::LOOVV, {o, o, v, v});
  const int Looov = alloc(B::LOOOV, {o, o, o, v});
  const int Lovvo = alloc(B::LOVVO, {o, v, v, o});
  const int Loovo = alloc(B::LOOVO, {o, o, v, o});
  Program P;
  P.name = "setup";
  // <pq|rs> = sum_P B[P][p][r] B[P][q][s]
  Engine::ein(P, oooo, "mnij", Boo, "Pmi", Boo, "Pnj");
  Engine::ein(P, ooov, "mnie", Boo, "Pmi", Bov, "Pne");
  Engine::ein(P, oovo, "mnei", Bov, "Pme", Boo, "Pni");
  Engine::ein(P, oovv, "mnef", Bov, "Pme", Bov, "Pnf");
  Engine::ein(P, ovov, "mbie", Boo, "Pmi", Bvv, "Pbe");
  Engine::ein(P, ovvo, "mbej", Bov, "Pme", Bvo, "Pbj");
  Engine::ein(P, ovoo, "mbij", Boo, "Pmi", Bvo, "Pbj");
  Engine::ein(P, ovvv, "mbef", Bov, "Pme", Bvv, "Pbf");
  Engine::ein(P, vvvo, "abej", Bvv, "Pae", Bvo, "Pbj");
  Engine::ein(P, vvvv, "abef", Bvv, "Pae", Bvv, "Pbf");
  // exchange combinations
  Engine::add(P, Lovvv, "mafe", ovvv, "mafe", 2.0);
  Engine::add(P, Lovvv, "mafe", ovvv, "maef", -1.0);
  Engine::add(P, Loovv, "mnef", oovv, "mnef", 2.0);
  Engine::add(P, Loovv, "mnef", oovv, "mnfe", -1.0);
  Engine::add(P, Looov, "mnie", ooov, "mnie", 2.0);
  Engine::add(P, Looov, "mnie", oovo, "mnei", -1.0);
  Engine::add(P, Lovvo, "nafi", ovvo, "nafi", 2.0);
  Engine::add(P, Lovvo, "nafi", ovov, "naif", -1.0);
  Engine::add(P, Loovo, "nmei", oovo, "nmei", 2.0);
  Engine::add(P, Loovo, "nmei", ooov, "nmie", -1.0);
  E.finalize({&P});
  E.run(P);
  RTCC_CUDA(cudaStreamSynchronize(stream));
}

IntIds register_integrals(Engine& E, const IntegralStore& S) {
  using B = IntegralStore;
  const int o = S.o, v = S.v;
  IntIds I;
  auto reg = [&](int b, std::vector<int> dims) { I.b[b] = E.external("v" + std::to_string(b), dims, false, S.blk[b], {}, true); };
  reg(B::OOOO, {o, o, o, o});
  reg(B::OOOV, {o, o, o, v});
  reg(B::OOVO, {o, o, v, o});
  reg(B::OOVV, {o, o, v, v});
  reg(B::OVOV, {o, v, o, v});
  reg(B::OVVO, {o, v, v, o});
  reg(B::OVOO, {o, v, o, o});
  reg(B::OVVV, {o, v, v, v});
  reg(B::VVVO, {v, v, v, o});
  reg(B::VVVV, {v, v, v, v});
  reg(B::LOVVV, {o, v, v, v});
  reg(B::LOOVV, {o, o, v, v});
  reg(B::LOOOV, {o, o, o, v});
  reg(B::LOVVO, {o, v, v, o});
  reg(B::LOOVO, {o, o, v, o});
  return I;
}

namespace {

// Views of one state-layout buffer [nz][ns] complex: x1 = [o][v] at 0, x2 = [o][o][v][v] at o*v,
// y1 at o*v + o*o*v*v, y2 after it.
struct StateViews {
  int x1, x2, y1, y2;
};
StateViews state_views(Engine& E, const std::string& nm, double* buf, int nz, int o, int v) {
  const long long ns = 2ll * o * v + 2ll * o * o * v * v;
  const long long n1 = (long long)o * v, n2 = (long long)o * o * v * v;
  StateViews s;
  s.x1 = E.external(nm + ".x1", {nz, o, v}, true, buf, {ns, v, 1});
  s.x2 = E.external(nm + ".x2", {nz, o, o, v, v}, true, buf + 2 * n1, {ns, (long long)o * v * v, (long long)v * v, v, 1});
  s.y1 = E.external(nm + ".y1", {nz, o, v}, true, buf + 2 * (n1 + n2), {ns, v, 1});
  s.y2 = E.external(nm + ".y2", {nz, o, o, v, v}, true, buf + 2 * (2 * n1 + n2),
                    {ns, (long long)o * v * v, (long long)v * v, v, 1});
  return s;
}

// Fock-like one-body operator views: f[.. p q] with an optional leading label.
struct OneBody {
  int oo, ov, vv;
  std::string pre;   // "z" when the operator carries the trajectory label, "" otherwise
};

struct Builder {
  Engine& E;
  Program& P;
  int arena;
  int nz, o, v;
  int nx;   // extent of the operator label of Fock-dependent intermediates (0: none)
  // amplitude-only intermediates carry the trajectory label z
  int tmp(const std::string& nm, std::vector<int> dims) {
    dims.insert(dims.begin(), nz);
    return E.temp(arena, nm, dims, true);
  }
  // intermediates that depend on the one-body operator carry its label too ("xz" or "z")
  int tmpf(const std::string& nm, std::vector<int> dims) {
    dims.insert(dims.begin(), nz);
    if (nx) dims.insert(dims.begin(), nx);
    return E.temp(arena, nm, dims, true);
  }
  void ein(int c, const std::string& lc, int a, const std::string& la, int b, const std::string& lb,
           cplx alpha = 1.0) {
    Engine::ein(P, c, lc, a, la, b, lb, alpha);
  }
  void add(int c, const std::string& lc, int a, const std::string& la, cplx alpha = 1.0) {
    Engine::add(P, c, lc, a, la, alpha);
  }
  // b's label pairs (0,1) and (2,3) swap together without changing it
  void ein_pairsym(int c, const std::string& lc, int a, const std::string& la, int bb, const std::string& lb,
                   cplx alpha = 1.0) {
    Engine::ein(P, c, lc, a, la, bb, lb, alpha, true);
  }
};

// Closed-shell CCSD ket residual into views (r1 "zia", r2 "zijab").
// Returns the id of tau (t2 + t1 t1) for the energy.
int residual_ops(Builder& b, const IntIds* I, int t1, int t2, const OneBody& f, int r1, int r2) {
  const int o = b.o, v = b.v;
  const std::string F = f.pre;
  const std::string Q = b.nx ? "xz" : "z";   // labels of Fock-dependent intermediates
  using B = IntegralStore;
  auto V = [&](int k) { return I->b[k]; };
  const bool two = (I != nullptr);

  const int tt = b.tmp("tt", {o, o, v, v});
  b.ein(tt, "zijab", t1, "zia", t1, "zjb");
  const int tau = b.tmp("tau", {o, o, v, v});
  b.add(tau, "zijab", t2, "zijab");
  b.add(tau, "zijab", tt, "zijab");
  const int taut = b.tmp("taut", {o, o, v, v});
  b.add(taut, "zijab", t2, "zijab");
  b.add(taut, "zijab", tt, "zijab", 0.5);

  // one-body intermediates
  const int Fae = b.tmpf("Fae", {v, v});
  b.add(Fae, Q + "ae", f.vv, F + "ae");
  b.ein(Fae, Q + "ae", f.ov, F + "me", t1, "zma", -0.5);
  const int Fmi = b.tmpf("Fmi", {o, o});
  b.add(Fmi, Q + "mi", f.oo, F + "mi");
  b.ein(Fmi, Q + "mi", t1, "zie", f.ov, F + "me", 0.5);
  const int Fme = b.tmpf("Fme", {o, v});
  b.add(Fme, Q + "me", f.ov, F + "me");
  if (two) {
    b.ein(Fae, Q + "ae", t1, "zmf", V(B::LOVVV), "mafe");
    b.ein(Fae, Q + "ae", taut, "zmnaf", V(B::LOOVV), "mnef", -1.0);
    b.ein(Fmi, Q + "mi", t1, "zne", V(B::LOOOV), "mnie");
    b.ein(Fmi, Q + "mi", taut, "zinef", V(B::LOOVV), "mnef");
    b.ein(Fme, Q + "me", t1, "znf", V(B::LOOVV), "mnef");
  }

  // singles
  const int t2t = b.tmp("t2t", {o, o, v, v});   // 2 t_imae - t_imea
  b.add(t2t, "zimae", t2, "zimae", 2.0);
  b.add(t2t, "zimae", t2, "zimea", -1.0);
  b.add(r1, Q + "ia", f.ov, F + "ia");
  b.ein(r1, Q + "ia", t1, "zie", Fae, Q + "ae");
  b.ein(r1, Q + "ia", t1, "zma", Fmi, Q + "mi", -1.0);
  b.ein(r1, Q + "ia", t2t, "zimae", Fme, Q + "me");
  if (two) {
    b.ein(r1, Q + "ia", t1, "znf", V(B::LOVVO), "nafi");
    b.ein(r1, Q + "ia", t2, "zimef", V(B::LOVVV), "mafe");
    b.ein(r1, Q + "ia", t2, "zmnae", V(B::LOOVO), "nmei", -1.0);
  }

  // doubles: Omega2 = S + S^(i<->j, a<->b)
  const int Xbe = b.tmpf("Xbe", {v, v});
  b.add(Xbe, Q + "be", Fae, Q + "be");
  b.ein(Xbe, Q + "be", t1, "zmb", Fme, Q + "me", -0.5);
  const int Zmj = b.tmpf("Zmj", {o, o});
  b.add(Zmj, Q + "mj", Fmi, Q + "mj");
  b.ein(Zmj, Q + "mj", t1, "zje", Fme, Q + "me", 0.5);
  const int S = b.tmpf("S", {o, o, v, v});
  b.ein(S, Q + "ijab", t2, "zijae", Xbe, Q + "be");
  b.ein(S, Q + "ijab", t2, "zimab", Zmj, Q + "mj", -1.0);
  if (two) {
    b.add(S, Q + "ijab", V(B::OOVV), "ijab", 0.5);
    // particle-particle ladder (half: the symmetrisation doubles it)
    // (vvvv[a][b][e][f] = (ae|bf) is unchanged by a<->b together with e<->f)
    b.ein_pairsym(S, Q + "ijab", tau, "zijef", V(B::VVVV), "abef", 0.5);
    // hole-hole ladder with W_mnij = <mn|ij> + P t1 terms + tau <mn|ef>
    const int Wmnij = b.tmp("Wmnij", {o, o, o, o});
    b.add(Wmnij, "zmnij", V(B::OOOO), "mnij");
    b.ein(Wmnij, "zmnij", t1, "zje", V(B::OOOV), "mnie");
    b.ein(Wmnij, "zmnij", t1, "zie", V(B::OOVO), "mnej");
    b.ein(Wmnij, "zmnij", tau, "zijef", V(B::OOVV), "mnef");
    b.ein(S, Q + "ijab", tau, "zmnab", Wmnij, "zmnij", 0.5);
    // Every term of the form -t1[ma] Y[ijmb] is summed into one o^3 v intermediate before a single
    // product with t1 (one pass over the o^2 v^2 output instead of four, and the same in the adjoint):
    // the t1 pieces of the particle-particle ladder tau <mb|ef>, the t1 t1 <mb|ej> and t1 t1 <mb|ie>
    // ring pieces, and t1 <mb|ij>.
    const int Xijmb = b.tmp("Xijmb", {o, o, o, v});
    b.ein(Xijmb, "zijmb", tau, "zijef", V(B::OVVV), "mbef");
    // ring intermediates: (m a, b b, e a, j b) and (m a, b b, e b, j a) spin blocks of W_mbej
    const int t1t1 = b.tmp("t1t1", {o, o, v, v});
    b.ein(t1t1, "zjnfb", t1, "zjf", t1, "znb");
    // Uh = t2/2 + t1 t1 enters both ring blocks through <mn|ef>: one o^3 v^3 product each (the
    // t2 and t1 t1 parts of W_mbej contracted together, and their adjoints in one product too)
    const int Uh = b.tmp("Uh", {o, o, v, v});
    b.add(Uh, "zjnfb", t2, "zjnfb", 0.5);
    b.add(Uh, "zjnfb", t1t1, "zjnfb");
    const int Wa = b.tmp("Wa", {o, v, v, o});
    b.add(Wa, "zmbej", V(B::OVVO), "mbej");
    b.ein(Wa, "zmbej", t1, "zjf", V(B::OVVV), "mbef");
    b.ein(Wa, "zmbej", t1, "znb", V(B::OOVO), "mnej", -1.0);
    b.ein(Wa, "zmbej", Uh, "zjnfb", V(B::OOVV), "mnef", -1.0);
    b.ein(Wa, "zmbej", t2, "zjnbf", V(B::LOOVV), "mnef", 0.5);
    const int U = b.tmp("U", {o, v, v, o});
    b.add(U, "zmbej", V(B::OVOV), "mbje", -1.0);
    b.ein(U, "zmbej", t1, "zjf", V(B::OVVV), "mbfe", -1.0);
    b.ein(U, "zmbej", t1, "znb", V(B::OOOV), "mnje");
    b.ein(U, "zmbej", Uh, "zjnfb", V(B::OOVV), "mnfe");
    b.ein(S, Q + "ijab", t2t, "zimae", Wa, "zmbej");
    b.ein(S, Q + "ijab", t2, "zimae", U, "zmbej");
    b.ein(S, Q + "ijab", t2, "zmjae", U, "zmbei");
    // t1 t1 <mb|ej> and t1 t1 <mb|ie> rings and t1 <mb|ij> join the ladder's t1 pieces; t1 <ab|ej>
    b.ein(Xijmb, "zijmb", t1, "zie", V(B::OVVO), "mbej");
    b.ein(Xijmb, "zijmb", t1, "zje", V(B::OVOV), "mbie");
    b.add(Xijmb, "zijmb", V(B::OVOO), "mbij");
    b.ein(S, Q + "ijab", t1, "zma", Xijmb, "zijmb", -1.0);
    b.ein(S, Q + "ijab", t1, "zie", V(B::VVVO), "abej");
  }
  b.add(r2, Q + "ijab", S, Q + "ijab");
  b.add(r2, Q + "ijab", S, Q + "jiba");
  return tau;
}

}  // namespace

namespace {
// an arena given by the caller is reused from its start (programs built for different batch
// sizes share it; they never run interleaved); -1 asks for a new arena
int reuse_arena(Engine& E, int a) {
  if (a < 0) return E.new_arena();
  E.arena_reset(a, 0);
  return a;
}
}  // namespace

RhsPrograms build_rhs(Engine& E, const IntIds& I, int nz, int o, int v, double* state, double* fock,
                      double* out, bool with_lambda, int fwd_arena, int rev_arena) {
  RhsPrograms R;
  const int n = o + v;
  const StateViews in = state_views(E, "y", state, nz, o, v);
  const StateViews ou = state_views(E, "r", out, nz, o, v);
  const long long sf = (long long)n * n;
  OneBody f;
  f.pre = "z";
  f.oo = E.external("f.oo", {nz, o, o}, false, fock, {sf, n, 1});
  f.ov = E.external("f.ov", {nz, o, v}, false, fock + o, {sf, n, 1});
  f.vv = E.external("f.vv", {nz, v, v}, false, fock + (size_t)o * n + o, {sf, n, 1});
  const int fa = reuse_arena(E, fwd_arena);
  R.fwd_arena = fa;
  R.fwd.name = "rhs_fwd";
  R.fwd.zero_arenas = {fa};
  const long long ns = 2ll * o * v + 2ll * o * o * v * v, nT = (long long)o * v + (long long)o * o * v * v;
  R.fwd.zero2d = {{out, (size_t)ns * 16, (size_t)nT * 16, (size_t)nz}};
  Builder b{E, R.fwd, fa, nz, o, v, 0};
  R.t1 = in.x1;
  R.t2 = in.x2;
  R.l1 = in.y1;
  R.l2 = in.y2;
  R.foo = f.oo;
  R.fov = f.ov;
  R.fvv = f.vv;
  R.r1 = ou.x1;
  R.r2 = ou.x2;
  R.rl1 = ou.y1;
  R.rl2 = ou.y2;
  R.tau = residual_ops(b, &I, in.x1, in.x2, f, ou.x1, ou.x2);
  if (!with_lambda) return R;
  std::map<int, int> adj;
  const int ra = reuse_arena(E, rev_arena);
  R.rev_arena = ra;
  R.rev = E.reverse(R.fwd, {in.x1, in.x2}, ra, adj);
  R.rev.zero2d = {{out + 2 * nT, (size_t)ns * 16, (size_t)nT * 16, (size_t)nz}};
  // seeds: dL/dOmega = l, dE/dt1 = 2 f_ov, dE/dtau = L_ijab
  std::vector<Op> seeds;
  seeds.push_back(Op{OP_ADD, adj.at(ou.x1), in.y1, -1, "zia", "zia", "", 1.0});
  seeds.push_back(Op{OP_ADD, adj.at(ou.x2), in.y2, -1, "zijab", "zijab", "", 1.0});
  seeds.push_back(Op{OP_ADD, adj.at(in.x1), f.ov, -1, "zia", "zia", "", 2.0});
  seeds.push_back(Op{OP_ADD, adj.at(R.tau), I.b[IntegralStore::LOOVV], -1, "zijab", "ijab", "", 1.0});
  R.rev.ops.insert(R.rev.ops.begin(), seeds.begin(), seeds.end());
  // outputs: R1 = dL/dt1, R2 = symmetrised dL/dt2
  Engine::add(R.rev, ou.y1, "zia", adj.at(in.x1), "zia");
  Engine::add(R.rev, ou.y2, "zijab", adj.at(in.x2), "zijab", 0.5);
  Engine::add(R.rev, ou.y2, "zijab", adj.at(in.x2), "zjiba", 0.5);
  return R;
}

DipolePrograms build_dipole(Engine& E, int nz, int o, int v, double* state, const double* mu_dev,
                            double* dip_out, int fwd_arena, int rev_arena) {
  // The dipole is the one-body Lagrangian evaluated with f -> mu_x (Eq. dipole).  That Lagrangian is
  // linear in the one-body operator, L1(f) = sum_pq rho_pq f_pq, so rho = dL1/df is the one-particle
  // density: one reverse sweep of the one-body program with f as the active input gives rho for
  // every trajectory, and mu_x = 2 sum_i mu_x,ii + sum_pq rho_pq mu_x,pq.
  DipolePrograms D;
  const int n = o + v;
  const StateViews in = state_views(E, "yd", state, nz, o, v);
  const int fa = reuse_arena(E, fwd_arena);
  const int ra = reuse_arena(E, rev_arena);
  D.fwd_arena = fa;
  D.rev_arena = ra;
  Program fwd;
  fwd.name = "dens_fwd";
  // a placeholder operator buffer: the pruned forward never reads it and the reverse pass only needs
  // the amplitude-only intermediates
  const long long sf = (long long)n * n;
  D.fdummy = static_cast<double*>(dev_alloc(sizeof(double) * (size_t)nz * n * n));
  RTCC_CUDA(cudaMemset(D.fdummy, 0, sizeof(double) * (size_t)nz * n * n));
  OneBody f;
  f.pre = "z";
  f.oo = E.external("fd.oo", {nz, o, o}, false, D.fdummy, {sf, n, 1});
  f.ov = E.external("fd.ov", {nz, o, v}, false, D.fdummy + o, {sf, n, 1});
  f.vv = E.external("fd.vv", {nz, v, v}, false, D.fdummy + (size_t)o * n + o, {sf, n, 1});
  Builder b{E, fwd, fa, nz, o, v, 0};
  const int om1 = b.tmp("om1mu", {o, v});
  const int om2 = b.tmp("om2mu", {o, o, v, v});
  residual_ops(b, nullptr, in.x1, in.x2, f, om1, om2);
  std::map<int, int> adj;
  Program rev = E.reverse(fwd, {f.oo, f.ov, f.vv}, ra, adj);
  // keep only the forward ops that do not depend on the operator (amplitude-only intermediates)
  std::set<int> dep = {f.oo, f.ov, f.vv};
  Program& P = D.prog;
  P.name = "dipole";
  // the recorded observable: float64 in the float64 mode, split-TF32 (float32-level accuracy) otherwise
  P.prec_override = (E.prec() == Prec::P64) ? (int)Prec::P64 : (int)Prec::TF32X3;
  P.zero_arenas = {fa, ra};
  for (const Op& op : fwd.ops) {
    const bool d = dep.count(op.a) || (op.kind == OP_EIN && dep.count(op.b));
    if (d) dep.insert(op.c);
    else P.ops.push_back(op);
  }
  // seeds: dL1/dOmega1 = l1, dL1/dOmega2 = l2, dE1/df_ov = 2 t1
  P.ops.push_back(Op{OP_ADD, adj.at(om1), in.y1, -1, "zia", "zia", "", 1.0});
  P.ops.push_back(Op{OP_ADD, adj.at(om2), in.y2, -1, "zijab", "zijab", "", 1.0});
  P.ops.push_back(Op{OP_ADD, adj.at(f.ov), in.x1, -1, "zia", "zia", "", 2.0});
  for (const Op& op : rev.ops) P.ops.push_back(op);
  double* m = const_cast<double*>(mu_dev);
  const int moo = E.external("mu.oo", {3, o, o}, false, m, {sf, n, 1}, true);
  const int mov = E.external("mu.ov", {3, o, v}, false, m + o, {sf, n, 1}, true);
  const int mvv = E.external("mu.vv", {3, v, v}, false, m + (size_t)o * n + o, {sf, n, 1}, true);
  const int dx = E.external("dip", {3, nz}, true, dip_out);
  P.zero_tensors = {dx};
  D.y1 = in.x1;
  D.y2 = in.x2;
  D.y3 = in.y1;
  D.y4 = in.y2;
  D.dip = dx;
  Engine::ein(P, dx, "xz", moo, "xij", adj.at(f.oo), "zij");
  Engine::ein(P, dx, "xz", mov, "xia", adj.at(f.ov), "zia");
  Engine::ein(P, dx, "xz", mvv, "xab", adj.at(f.vv), "zab");
  return D;
}

Program build_rhs_vjp(Engine& E, const RhsPrograms& R, int nz, int o, int v, double* cot, double* ybar,
                      double* fbar) {
  // the right-hand side is the concatenation fwd ; rev (seeds, reverse sweep, outputs)
  Program both;
  both.name = "rhs";
  both.ops = R.fwd.ops;
  both.ops.insert(both.ops.end(), R.rev.ops.begin(), R.rev.ops.end());
  std::map<int, int> adj;
  const int arena = E.new_arena();
  Program V = E.reverse(both, {R.t1, R.t2, R.l1, R.l2, R.foo, R.fov, R.fvv}, arena, adj);
  V.name = "rhs_vjp";
  const StateViews c = state_views(E, "cot", cot, nz, o, v);
  const StateViews yb = state_views(E, "ybar", ybar, nz, o, v);
  const int n = o + v;
  const long long sf = (long long)n * n;
  const int fboo = E.external("fbar.oo", {nz, o, o}, true, fbar, {sf, n, 1});
  const int fbov = E.external("fbar.ov", {nz, o, v}, true, fbar + 2 * o, {sf, n, 1});
  const int fbvv = E.external("fbar.vv", {nz, v, v}, true, fbar + 2 * ((size_t)o * n + o), {sf, n, 1});
  const long long ns = 2ll * o * v + 2ll * o * o * v * v;
  V.zero2d = {{ybar, (size_t)ns * 16, (size_t)ns * 16, (size_t)nz}, {fbar, (size_t)sf * 16, (size_t)sf * 16, (size_t)nz}};
  std::vector<Op> seeds;
  auto seed = [&](int out, int cv, const char* l) {
    auto it = adj.find(out);
    if (it != adj.end()) seeds.push_back(Op{OP_ADD, it->second, cv, -1, l, l, "", 1.0});
  };
  seed(R.r1, c.x1, "zia");
  seed(R.r2, c.x2, "zijab");
  seed(R.rl1, c.y1, "zia");
  seed(R.rl2, c.y2, "zijab");
  V.ops.insert(V.ops.begin(), seeds.begin(), seeds.end());
  auto out = [&](int dst, const char* ld, int src) {
    auto it = adj.find(src);
    if (it != adj.end()) Engine::add(V, dst, ld, it->second, ld);
  };
  out(yb.x1, "zia", R.t1);
  out(yb.x2, "zijab", R.t2);
  out(yb.y1, "zia", R.l1);
  out(yb.y2, "zijab", R.l2);
  out(fboo, "zij", R.foo);
  out(fbov, "zia", R.fov);
  out(fbvv, "zab", R.fvv);
  return V;
}

Program build_dipole_vjp(Engine& E, const DipolePrograms& D, int nz, int o, int v, double* wdip, double* ybar) {
  std::map<int, int> adj;
  const int arena = E.new_arena();
  Program V = E.reverse(D.prog, {D.y1, D.y2, D.y3, D.y4}, arena, adj);
  V.name = "dipole_vjp";
  V.prec_override = D.prog.prec_override;
  const int w = E.external("wdip", {3, nz}, true, wdip);
  auto it = adj.find(D.dip);
  RTCC_REQUIRE(it != adj.end(), "dipole does not depend on the state");
  V.ops.insert(V.ops.begin(), Op{OP_ADD, it->second, w, -1, "xz", "xz", "", 1.0});
  const StateViews yb = state_views(E, "ybar_obs", ybar, nz, o, v);
  auto out = [&](int dst, const char* ld, int src) {
    auto jt = adj.find(src);
    if (jt != adj.end()) Engine::add(V, dst, ld, jt->second, ld);
  };
  out(yb.x1, "zia", D.y1);
  out(yb.x2, "zijab", D.y2);
  out(yb.y1, "zia", D.y3);
  out(yb.y2, "zijab", D.y4);
  return V;
}

Program build_energy(Engine& E, const IntIds& I, const RhsPrograms& R, int nz, int o, int v, double* fock,
                     double* e_out) {
  Program P;
  P.name = "energy";
  const int n = o + v;
  const int fov = E.external("fe.ov", {nz, o, v}, false, fock + o, {(long long)n * n, n, 1});
  const int e = E.external("ecorr", {nz}, true, e_out);
  P.zero_tensors = {e};
  Engine::ein(P, e, "z", fov, "zia", R.t1, "zia", 2.0);
  Engine::ein(P, e, "z", R.tau, "zijab", I.b[IntegralStore::LOOVV], "ijab");
  return P;
}

}  // namespace rtcc
