// libmdwf host side: contexts, the fifth-dimension coefficient tables, the
// operator applies of the C ABI, and the batched even-odd CG solver.
//
// Solver (Sec. VII of arXiv:1701.07559: CG on the normal equations of the
// asymmetric even-odd operator, in "double-half" mixed precision):
//   Mhat x_e = bhat_e,  bhat_e = b_e - D_eo A^-1 b_o,  x_o = A^-1 (b_o - D_oe x_e).
// The normal equations are iterated in the CGLS arrangement (the same iterates
// as CG on Mhat^+ Mhat, with rho = bhat - Mhat x carried explicitly), so the
// stopping rule acts on ||bhat - Mhat x_e||, which equals the full-lattice
// residual ||b - D x|| after reconstruction.  Inner vectors live in the chosen
// storage precision (FP32 arithmetic); the solution accumulator x_hi, the
// residual recomputed at each reliable update, and every global sum are FP64.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/mdwf.h"
#include "blas.h"
#include "mdwf_internal.h"

using namespace mdwf;

struct Action {
  double M5 = 0, b5 = 0, c5 = 0, mf = 0;
  int L5 = 0;
  bool set = false;
};

struct Cfg {
  bool has_gauge = false;
  int anti = 1;
  double* U64 = nullptr;
  float* U32 = nullptr;
  Action act;
};

struct mdwf_ctx {
  int device = 0;
  Geom g;
  std::map<int, Cfg> cfgs;
  std::string err;
  cudaStream_t stream = nullptr;
};

namespace {

int fail(mdwf_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? MDWF_ERR_NOMEM : MDWF_ERR_CUDA,           \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                             \
  } while (0)

// Owning device allocation.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { if (p) cudaFree(p); }
  cudaError_t alloc(size_t b) {
    if (p) { cudaFree(p); p = nullptr; }
    bytes = b;
    return cudaMalloc(&p, b ? b : 16);
  }
  template <typename X> X* as() const { return reinterpret_cast<X*>(p); }
};

bool all_finite(const double* v, size_t n) {
  for (size_t i = 0; i < n; i++)
    if (!std::isfinite(v[i])) return false;
  return true;
}

// ---------------------------------------------------------------------------
// Fifth-dimension coefficient tables
// ---------------------------------------------------------------------------
// Per chirality (0: spins 0,1 = P_+; 1: spins 2,3 = P_-) the operators of the
// fifth dimension are real L5 x L5 matrices:
//   P_+ block: (P x)_s = x_{s-1}, x_{-1} = -m x_{L5-1};  P_- block: x_{s+1}, x_{L5} = -m x_0
//   A = alpha + beta P (alpha = b5 d + 1, beta = c5 d - 1, d = 4 - M5), B = b5 + c5 P.
// Adjoints are transposes.  A^-1 in closed form: with kappa = beta / alpha,
//   (A^-1)_{s s'} = (-kappa)^k sigma / (alpha (1 + m (-kappa)^L5)),
// k = number of shift steps from s' to s (mod L5), sigma = -m if the path
// crosses the wall and 1 otherwise.
enum MatKind { MK_A, MK_Ad, MK_B, MK_Bd, MK_Ainv, MK_Ainvd, MK_BAinv, MK_AinvdBd, MK_negA, MK_COUNT };

using Mat = std::vector<double>;

Mat mat_zero(int n) { return Mat((size_t)n * n, 0.0); }
Mat mat_eye(int n) { Mat m = mat_zero(n); for (int i = 0; i < n; i++) m[(size_t)i * n + i] = 1.0; return m; }
Mat mat_T(const Mat& a, int n) {
  Mat t = mat_zero(n);
  for (int i = 0; i < n; i++) for (int j = 0; j < n; j++) t[(size_t)j * n + i] = a[(size_t)i * n + j];
  return t;
}
Mat mat_mul(const Mat& a, const Mat& b, int n) {
  Mat c = mat_zero(n);
  for (int i = 0; i < n; i++)
    for (int k = 0; k < n; k++) {
      double aik = a[(size_t)i * n + k];
      for (int j = 0; j < n; j++) c[(size_t)i * n + j] += aik * b[(size_t)k * n + j];
    }
  return c;
}
Mat mat_lin(double x, const Mat& a, double y, const Mat& b) {
  Mat c(a.size());
  for (size_t i = 0; i < a.size(); i++) c[i] = x * a[i] + y * b[i];
  return c;
}
Mat mat_shift(int L5, double m, int chi) {
  Mat p = mat_zero(L5);
  for (int s = 0; s < L5; s++) {
    if (chi == 0) {
      if (s >= 1) p[(size_t)s * L5 + s - 1] = 1.0; else p[(size_t)s * L5 + L5 - 1] = -m;
    } else {
      if (s <= L5 - 2) p[(size_t)s * L5 + s + 1] = 1.0; else p[(size_t)s * L5] = -m;
    }
  }
  return p;
}
Mat mat_ainv(int L5, double alpha, double beta, double m, int chi) {
  const double kappa = beta / alpha;
  const double norm = 1.0 / (alpha * (1.0 + m * std::pow(-kappa, L5)));
  Mat a = mat_zero(L5);
  for (int s = 0; s < L5; s++)
    for (int sp = 0; sp < L5; sp++) {
      // chirality 0 shifts downward (s' -> s' + 1), chirality 1 upward
      int k = chi == 0 ? ((s - sp) % L5 + L5) % L5 : ((sp - s) % L5 + L5) % L5;
      bool wrap = chi == 0 ? (s < sp) : (s > sp);
      a[(size_t)s * L5 + sp] = std::pow(-kappa, k) * (wrap ? -m : 1.0) * norm;
    }
  return a;
}

// Host tables for N slots, each [MK][r][chi][L5][L5].
struct Tables {
  int L5 = 0, N = 0;
  std::vector<double> h;  // MK_COUNT * N * 2 * L5 * L5
  size_t block() const { return (size_t)N * 2 * L5 * L5; }
  void build(const Action& act, const std::vector<double>& masses) {
    L5 = act.L5;
    N = (int)masses.size();
    h.assign(MK_COUNT * block(), 0.0);
    const double d = 4.0 - act.M5;
    const double alpha = act.b5 * d + 1.0, beta = act.c5 * d - 1.0;
    const Mat I = mat_eye(L5);
    for (int r = 0; r < N; r++)
      for (int chi = 0; chi < 2; chi++) {
        Mat P = mat_shift(L5, masses[r], chi);
        Mat A = mat_lin(alpha, I, beta, P);
        Mat B = mat_lin(act.b5, I, act.c5, P);
        Mat Ai = mat_ainv(L5, alpha, beta, masses[r], chi);
        Mat all[MK_COUNT] = {A, mat_T(A, L5), B, mat_T(B, L5), Ai, mat_T(Ai, L5),
                             mat_mul(B, Ai, L5), mat_mul(mat_T(Ai, L5), mat_T(B, L5), L5), mat_lin(-1.0, A, 0.0, A)};
        for (int k = 0; k < MK_COUNT; k++)
          std::memcpy(&h[k * block() + ((size_t)r * 2 + chi) * L5 * L5], all[k].data(), sizeof(double) * L5 * L5);
      }
  }
};

// Device copies of the tables in T precision.
template <typename T>
struct DevTables {
  DBuf buf;
  size_t blk = 0;
  cudaError_t upload(const Tables& t, cudaStream_t st) {
    blk = t.block();
    std::vector<T> v(t.h.size());
    for (size_t i = 0; i < v.size(); i++) v[i] = (T)t.h[i];
    cudaError_t e = buf.alloc(sizeof(T) * v.size());
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(buf.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
  }
  const T* operator[](int k) const { return buf.as<T>() + (size_t)k * blk; }
};

// ---------------------------------------------------------------------------
// Operator building blocks on device fields
// ---------------------------------------------------------------------------
template <typename S>
struct F {           // one parity field, N slots
  S* v = nullptr;
  float* n = nullptr;
};

template <typename S>
struct FieldBuf {    // owning
  DBuf v, n;
  cudaError_t alloc(long units) {
    cudaError_t e = v.alloc(sizeof(S) * 24 * (size_t)units);
    if (e != cudaSuccess) return e;
    if (StoreTraits<S>::kNorm) return n.alloc(sizeof(float) * (size_t)units);
    return cudaSuccess;
  }
  F<S> f() const { F<S> r; r.v = v.as<S>(); r.n = n.as<float>(); return r; }
};

template <typename S, typename T>
struct Op {
  Geom g;
  int L5 = 0, N = 0, anti = 1;
  const T* U = nullptr;
  Tiling tl;
  cudaStream_t st = nullptr;

  // out = add + G same + kappa C H(in)   (hop) ; out = add + G in (local)
  cudaError_t run(bool hop, int out_par, int dagger, F<S> in, F<S> same, const T* G, F<S> add, const T* C, T kappa,
                  F<S> out, const int* active, double* partials) const {
    HopArgs<S, T> a;
    a.g = g; a.L5 = L5; a.N = N; a.out_par = out_par; a.dagger = dagger; a.antiperiodic = anti;
    a.in = in.v; a.in_nrm = in.n; a.same = same.v; a.same_nrm = same.n; a.add = add.v; a.add_nrm = add.n;
    a.out = out.v; a.out_nrm = out.n; a.U = U; a.Gm = G; a.Cm = C; a.kappa = kappa; a.active = active;
    a.partials = partials;
    return launch_hop<S, T>(a, tl, hop, st);
  }
  // q = Mhat p (dagger 0) or Mhat^+ p (dagger 1) on even sites; u, t scratch (even, odd).
  cudaError_t schur(int dagger, F<S> p, F<S> u, F<S> t, F<S> q, const DevTables<T>& M, const int* active,
                    double* partials) const {
    F<S> none;
    cudaError_t e;
    if (!dagger) {
      e = run(false, 0, 0, p, none, M[MK_B], none, nullptr, T(0), u, active, nullptr);
      if (e != cudaSuccess) return e;
      e = run(true, 1, 0, u, none, nullptr, none, M[MK_BAinv], T(1), t, active, nullptr);
      if (e != cudaSuccess) return e;
      return run(true, 0, 0, t, p, M[MK_A], none, nullptr, T(-0.25), q, active, partials);
    }
    e = run(true, 1, 1, p, none, nullptr, none, M[MK_AinvdBd], T(1), t, active, nullptr);
    if (e != cudaSuccess) return e;
    return run(true, 0, 1, t, p, M[MK_Ad], none, M[MK_Bd], T(-0.25), q, active, partials);
  }
};

template <typename S>
Tiling tiling_for(const Geom& g, int L5, int N, int nsb, bool two_buffers) {
  using T = typename StoreTraits<S>::T;
  int maxthr = hop_max_threads<S, T>();
  int smem_thr = (int)(200 * 1024 / ((two_buffers ? 2 : 1) * 25 * sizeof(T)));
  if (smem_thr < maxthr) maxthr = smem_thr;
  if (maxthr > 1024) maxthr = 1024;
  if (nsb * L5 > maxthr) nsb = maxthr / L5 > 0 ? maxthr / L5 : 1;
  return make_tiling(g.Vh, L5, N, nsb, maxthr);
}

// ---------------------------------------------------------------------------
// Scalar kernels of the batched CG (one thread per RHS slot)
// ---------------------------------------------------------------------------
struct Scal {
  double *gamma, *gamma_prev, *alpha, *beta, *rho2, *rho2_max, *stop2, *qq, *rr, *tmp;
  int *active, *flags, *iters;
  double delta2;
};
enum { FLAG_INNER_DONE = 1, FLAG_UPDATE = 2, FLAG_DONE = 4 };

__global__ void k_alpha(Scal c, int N) {
  int r = threadIdx.x;
  if (r < N && c.active[r]) { double q = c.qq[r]; c.alpha[r] = q > 0.0 ? c.gamma[r] / q : 0.0; }
}
__global__ void k_after_rho(Scal c, int N) {
  int r = threadIdx.x;
  if (r < N && c.active[r]) {
    double v = c.tmp[r];
    c.rho2[r] = v;
    if (v > c.rho2_max[r]) c.rho2_max[r] = v;
    if (v <= c.stop2[r]) { c.active[r] = 0; c.flags[r] |= FLAG_INNER_DONE; }
    else if (v < c.delta2 * c.rho2_max[r]) c.flags[r] |= FLAG_UPDATE;
  }
}
__global__ void k_beta(Scal c, int N) {
  int r = threadIdx.x;
  if (r < N && c.active[r]) {
    double rr = c.rr[r], g = c.gamma[r];
    c.beta[r] = g > 0.0 ? rr / g : 0.0;
    c.gamma_prev[r] = g;
    c.gamma[r] = rr;
    c.iters[r] += 1;
  }
}
__global__ void k_after_update(Scal c, int N, const int* umask) {
  int r = threadIdx.x;
  if (r < N && umask[r]) {
    double v = c.tmp[r];
    c.rho2[r] = v;
    c.rho2_max[r] = v;
    c.gamma[r] = c.rr[r];
    c.beta[r] = c.gamma_prev[r] > 0.0 ? c.gamma[r] / c.gamma_prev[r] : 0.0;
    if (c.flags[r] & FLAG_INNER_DONE) {
      if (v <= c.stop2[r]) { c.flags[r] = FLAG_DONE; c.active[r] = 0; }
      else { c.flags[r] = 0; c.active[r] = 1; }
    } else {
      c.flags[r] &= ~FLAG_UPDATE;
    }
  }
}

// ---------------------------------------------------------------------------
// The batched solver
// ---------------------------------------------------------------------------
template <typename S>
struct BatchSolver {
  using T = typename StoreTraits<S>::T;
  using SX = typename std::conditional<std::is_same<S, double>::value, double, float>::type;

  mdwf_ctx* ctx;
  const Cfg* cfg;
  int N, L5;
  Op<double, double> op64;
  Op<S, T> opS;
  Tiling tl_blas64, tl_blasS;
  DevTables<double> M64;
  DevTables<T> MS;
  // FP64 fields: b (even, odd), x (even = x_hi, odd), bhat, rho64, u64 (even), t64 (odd)
  FieldBuf<double> b_e, b_o, x_e, x_o, bhat, rho64, u64, t64;
  // inner fields
  FieldBuf<S> p, u, t, q, rho, r;
  FieldBuf<SX> xlo;
  DBuf partials, scal_d, scal_i, umask_d;
  Scal sc;
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;

  ~BatchSolver() { if (graph) cudaGraphExecDestroy(graph); }

  int init(mdwf_ctx* c, const Cfg* cf, const std::vector<double>& masses, int nsb, cudaStream_t st) {
    mdwf_ctx* ctx = c;
    this->ctx = c;
    cfg = cf;
    N = (int)masses.size();
    L5 = cf->act.L5;
    const Geom& g = c->g;
    op64.g = g; op64.L5 = L5; op64.N = N; op64.anti = cf->anti; op64.U = cf->U64; op64.st = st;
    op64.tl = tiling_for<double>(g, L5, N, nsb, true);
    opS.g = g; opS.L5 = L5; opS.N = N; opS.anti = cf->anti; opS.st = st;
    opS.U = std::is_same<T, double>::value ? (const T*)cf->U64 : (const T*)cf->U32;
    opS.tl = tiling_for<S>(g, L5, N, op64.tl.nsb, true);
    tl_blas64 = make_tiling(g.Vh, L5, N, op64.tl.nsb, 1024);
    tl_blasS = tl_blas64;
    Tables tab;
    tab.build(cf->act, masses);
    CK(M64.upload(tab, st));
    CK(MS.upload(tab, st));
    long units = g.Vh * L5 * N;
    FieldBuf<double>* f64[] = {&b_e, &b_o, &x_e, &x_o, &bhat, &rho64, &u64, &t64};
    for (auto* f : f64) CK(f->alloc(units));
    FieldBuf<S>* fS[] = {&p, &u, &t, &q, &rho, &r};
    for (auto* f : fS) CK(f->alloc(units));
    CK(xlo.alloc(units));
    // one partial per site covers every tiling (nsb >= 1)
    CK(partials.alloc(sizeof(double) * g.Vh * N));
    CK(scal_d.alloc(sizeof(double) * 10 * N));
    CK(scal_i.alloc(sizeof(int) * 3 * N));
    CK(umask_d.alloc(sizeof(int) * N));
    double* d = scal_d.as<double>();
    sc.gamma = d; sc.gamma_prev = d + N; sc.alpha = d + 2 * N; sc.beta = d + 3 * N; sc.rho2 = d + 4 * N;
    sc.rho2_max = d + 5 * N; sc.stop2 = d + 6 * N; sc.qq = d + 7 * N; sc.rr = d + 8 * N; sc.tmp = d + 9 * N;
    int* ip = scal_i.as<int>();
    sc.active = ip; sc.flags = ip + N; sc.iters = ip + 2 * N;
    CK(cudaMemsetAsync(scal_d.p, 0, scal_d.bytes, st));
    CK(cudaMemsetAsync(scal_i.p, 0, scal_i.bytes, st));
    CK(cudaMemsetAsync(x_e.v.p, 0, x_e.v.bytes, st));
    CK(cudaMemsetAsync(xlo.v.p, 0, xlo.v.bytes, st));
    for (auto* f : fS) { CK(cudaMemsetAsync(f->v.p, 0, f->v.bytes, st)); if (f->n.p) CK(cudaMemsetAsync(f->n.p, 0, f->n.bytes, st)); }
    return MDWF_OK;
  }

  // |field|^2 per slot into dst[N] (device).
  template <typename SS>
  cudaError_t norms(F<SS> f, const Tiling& tl, const int* mask, double* dst) {
    cudaError_t e = norm2_partials<SS>(f.v, f.n, tl, ctx->g.Vh, L5, N, mask, partials.as<double>(), op64.st);
    if (e != cudaSuccess) return e;
    return finalize(partials.as<double>(), tl.ntiles, N, dst, op64.st);
  }

  // One CG iteration on all active slots (see file header).
  cudaError_t iteration() {
    const Geom& g = ctx->g;
    cudaStream_t st = op64.st;
    double* part = partials.as<double>();
    cudaError_t e;
    const int N_ = N;
    e = xpay<S>(r.f().v, r.f().n, p.f().v, p.f().n, sc.beta, tl_blasS, g.Vh, L5, N_, sc.active, st);
    if (e != cudaSuccess) return e;
    e = opS.schur(0, p.f(), u.f(), t.f(), q.f(), MS, sc.active, part);
    if (e != cudaSuccess) return e;
    e = finalize(part, opS.tl.ntiles, N_, sc.qq, st);
    if (e != cudaSuccess) return e;
    k_alpha<<<1, 1024, 0, st>>>(sc, N_);
    e = axpy_x_rho<SX, S>(xlo.f().v, p.f().v, p.f().n, rho.f().v, rho.f().n, q.f().v, q.f().n, sc.alpha, tl_blasS,
                          g.Vh, L5, N_, sc.active, part, st);
    if (e != cudaSuccess) return e;
    e = finalize(part, tl_blasS.ntiles, N_, sc.tmp, st);
    if (e != cudaSuccess) return e;
    k_after_rho<<<1, 1024, 0, st>>>(sc, N_);
    e = opS.schur(1, rho.f(), u.f(), t.f(), r.f(), MS, sc.active, part);
    if (e != cudaSuccess) return e;
    e = finalize(part, opS.tl.ntiles, N_, sc.rr, st);
    if (e != cudaSuccess) return e;
    k_beta<<<1, 1024, 0, st>>>(sc, N_);
    return cudaGetLastError();
  }

  // FP64 residual recomputation for the slots in umask (device).
  int* umask() { return umask_d.as<int>(); }

  cudaError_t reliable_update(const int* um) {
    const Geom& g = ctx->g;
    cudaStream_t st = op64.st;
    double* part = partials.as<double>();
    cudaError_t e = accum_xhi<SX>(x_e.f().v, xlo.f().v, tl_blas64, g.Vh, L5, N, um, st);
    if (e != cudaSuccess) return e;
    F<double> none;
    // rho64 = bhat - A x + 1/4 H_eo B A^-1 H_oe B x
    e = op64.run(false, 0, 0, x_e.f(), none, M64[MK_B], none, nullptr, 0.0, u64.f(), um, nullptr);
    if (e != cudaSuccess) return e;
    e = op64.run(true, 1, 0, u64.f(), none, nullptr, none, M64[MK_BAinv], 1.0, t64.f(), um, nullptr);
    if (e != cudaSuccess) return e;
    e = op64.run(true, 0, 0, t64.f(), x_e.f(), M64[MK_negA], bhat.f(), nullptr, 0.25, rho64.f(), um, part);
    if (e != cudaSuccess) return e;
    e = finalize(part, op64.tl.ntiles, N, sc.tmp, st);
    if (e != cudaSuccess) return e;
    e = convert<double, S>(rho64.f().v, nullptr, rho.f().v, rho.f().n, tl_blas64, g.Vh, L5, N,
                           um, st);
    if (e != cudaSuccess) return e;
    e = opS.schur(1, rho.f(), u.f(), t.f(), r.f(), MS, um, part);
    if (e != cudaSuccess) return e;
    e = finalize(part, opS.tl.ntiles, N, sc.rr, st);
    if (e != cudaSuccess) return e;
    k_after_update<<<1, 1024, 0, st>>>(sc, N, um);
    return cudaGetLastError();
  }

  int run_chunk(int k, bool use_graph) {
    mdwf_ctx* ctx = this->ctx;
    cudaStream_t st = op64.st;
    if (!use_graph) {
      for (int i = 0; i < k; i++) CK(iteration());
      return MDWF_OK;
    }
    if (graph == nullptr || graph_iters != k) {
      if (graph) { cudaGraphExecDestroy(graph); graph = nullptr; }
      cudaGraph_t gr;
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
      cudaError_t err = cudaSuccess;
      for (int i = 0; i < k && err == cudaSuccess; i++) err = iteration();
      cudaError_t e2 = cudaStreamEndCapture(st, &gr);
      CK(err);
      CK(e2);
      cudaError_t e3 = cudaGraphInstantiate(&graph, gr, 0);
      cudaGraphDestroy(gr);
      CK(e3);
      graph_iters = k;
    }
    CK(cudaGraphLaunch(graph, st));
    return MDWF_OK;
  }
};

int check_cfg(mdwf_ctx* ctx, int cfg_id, Cfg** out) {
  if (!ctx) return MDWF_ERR_ARG;
  auto it = ctx->cfgs.find(cfg_id);
  if (it == ctx->cfgs.end() || !it->second.has_gauge) return fail(ctx, MDWF_ERR_STATE, "no gauge field for cfg_id");
  if (!it->second.act.set) return fail(ctx, MDWF_ERR_STATE, "no action set for cfg_id");
  *out = &it->second;
  return MDWF_OK;
}

cudaStream_t pick_stream(mdwf_ctx* ctx, void* s) { return s ? (cudaStream_t)s : ctx->stream; }

// Solve on device API-layout buffers.
template <typename S>
int solve_batch_impl(mdwf_ctx* ctx, Cfg* cfg, int n, const double* const* srcs, const std::vector<double>& masses,
                     double* const* xs, double tol, const mdwf_solver_opts& o, mdwf_solve_stats* stats,
                     cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  BatchSolver<S> sv;
  int rc = sv.init(ctx, cfg, masses, o.nsb > 0 ? o.nsb : 2, st);
  if (rc != MDWF_OK) return rc;
  const Geom& g = ctx->g;
  const int N = n, L5 = cfg->act.L5;
  // pack sources
  for (int i = 0; i < N; i++) {
    CK(pack_rhs<double>(srcs[i], sv.b_e.f().v, nullptr, g, L5, N, 0, i, st));
    CK(pack_rhs<double>(srcs[i], sv.b_o.f().v, nullptr, g, L5, N, 1, i, st));
  }
  // |b|^2 = |b_e|^2 + |b_o|^2 per slot
  std::vector<double> bb(N), bo(N);
  double* tmp = sv.sc.tmp;
  CK(sv.norms(sv.b_e.f(), sv.tl_blas64, nullptr, tmp));
  CK(cudaMemcpyAsync(bb.data(), tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
  CK(sv.norms(sv.b_o.f(), sv.tl_blas64, nullptr, tmp));
  CK(cudaMemcpyAsync(bo.data(), tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<double> stop2(N);
  std::vector<int> act(N, 1);
  for (int i = 0; i < N; i++) {
    double b2 = bb[i] + bo[i];
    if (!std::isfinite(b2)) return fail(ctx, MDWF_ERR_NONFINITE, "source has NaN/Inf");
    stop2[i] = 0.25 * tol * tol * b2;
    if (b2 == 0.0) act[i] = 0;
  }
  CK(cudaMemcpyAsync(sv.sc.stop2, stop2.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st));
  sv.sc.delta2 = o.delta * o.delta;
  // bhat_e = b_e + 1/2 H_eo B A^-1 b_o
  F<double> none;
  CK(sv.op64.run(false, 1, 0, sv.b_o.f(), none, sv.M64[MK_BAinv], none, nullptr, 0.0, sv.t64.f(), nullptr, nullptr));
  CK(sv.op64.run(true, 0, 0, sv.t64.f(), none, nullptr, sv.b_e.f(), nullptr, 0.5, sv.bhat.f(), nullptr, nullptr));
  // initial residual (x = 0): a reliable update on every slot
  std::vector<int> um(N);
  for (int i = 0; i < N; i++) um[i] = act[i];
  CK(cudaMemcpyAsync(sv.sc.active, act.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(sv.umask_d.p, um.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  CK(sv.reliable_update(sv.umask()));
  std::vector<int> flags(N), iters(N), nupd(N, 1);
  std::vector<int> done(N, 0);
  for (int i = 0; i < N; i++) if (!act[i]) done[i] = 1;
  const int chunk = o.chunk > 0 ? o.chunk : 16;
  for (;;) {
    bool all = true;
    for (int i = 0; i < N; i++) all = all && done[i];
    if (all) break;
    rc = sv.run_chunk(chunk, o.use_graph != 0);
    if (rc != MDWF_OK) return rc;
    CK(cudaMemcpyAsync(flags.data(), sv.sc.flags, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(iters.data(), sv.sc.iters, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bool any = false;
    for (int i = 0; i < N; i++) {
      um[i] = (!done[i] && (flags[i] & (FLAG_INNER_DONE | FLAG_UPDATE))) ? 1 : 0;
      any = any || um[i];
    }
    if (any) {
      CK(cudaMemcpyAsync(sv.umask_d.p, um.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
      CK(sv.reliable_update(sv.umask()));
      CK(cudaMemcpyAsync(flags.data(), sv.sc.flags, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int i = 0; i < N; i++) if (um[i]) nupd[i]++;
    }
    bool stop_any = false;
    for (int i = 0; i < N; i++) {
      if (flags[i] & FLAG_DONE) done[i] = 1;
      if (!done[i] && iters[i] >= o.max_iter) { done[i] = 1; act[i] = 0; stop_any = true; }
    }
    if (stop_any) {
      // freeze slots that hit max_iter
      std::vector<int> a(N);
      CK(cudaMemcpyAsync(a.data(), sv.sc.active, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int i = 0; i < N; i++) if (done[i]) a[i] = 0;
      CK(cudaMemcpyAsync(sv.sc.active, a.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
    }
  }
  // x_hi += x_lo for everything not yet accumulated
  CK(accum_xhi<typename BatchSolver<S>::SX>(sv.x_e.f().v, sv.xlo.f().v, sv.tl_blas64, g.Vh, L5, N, nullptr, st));
  // x_o = A^-1 b_o + 1/2 A^-1 H_oe B x_e
  CK(sv.op64.run(false, 0, 0, sv.x_e.f(), none, sv.M64[MK_B], none, nullptr, 0.0, sv.u64.f(), nullptr, nullptr));
  CK(sv.op64.run(true, 1, 0, sv.u64.f(), sv.b_o.f(), sv.M64[MK_Ainv], none, sv.M64[MK_Ainv], 0.5, sv.x_o.f(),
                 nullptr, nullptr));
  // true residual r = b - D x on both parities: b - A x + 1/2 H B x
  CK(sv.op64.run(false, 1, 0, sv.x_o.f(), none, sv.M64[MK_B], none, nullptr, 0.0, sv.t64.f(), nullptr, nullptr));
  CK(sv.op64.run(true, 0, 0, sv.t64.f(), sv.x_e.f(), sv.M64[MK_negA], sv.b_e.f(), nullptr, 0.5, sv.rho64.f(),
                 nullptr, nullptr));
  std::vector<double> re(N), ro(N);
  CK(sv.norms(sv.rho64.f(), sv.tl_blas64, nullptr, tmp));
  CK(cudaMemcpyAsync(re.data(), tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
  // odd part, reusing u64 (B x_e) and rho64 as scratch
  CK(sv.op64.run(true, 1, 0, sv.u64.f(), sv.x_o.f(), sv.M64[MK_negA], sv.b_o.f(), nullptr, 0.5, sv.rho64.f(),
                 nullptr, nullptr));
  CK(sv.norms(sv.rho64.f(), sv.tl_blas64, nullptr, tmp));
  CK(cudaMemcpyAsync(ro.data(), tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(iters.data(), sv.sc.iters, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
  for (int i = 0; i < N; i++) {
    CK(unpack_rhs<double>(sv.x_e.f().v, nullptr, xs[i], g, L5, N, 0, i, st));
    CK(unpack_rhs<double>(sv.x_o.f().v, nullptr, xs[i], g, L5, N, 1, i, st));
  }
  CK(cudaStreamSynchronize(st));
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int status = MDWF_OK;
  for (int i = 0; i < N; i++) {
    double b2 = bb[i] + bo[i];
    double rel = b2 > 0 ? std::sqrt((re[i] + ro[i]) / b2) : 0.0;
    bool conv = rel <= tol;
    if (!conv) status = MDWF_ERR_NOT_CONVERGED;
    if (stats) {
      stats[i].iters = iters[i];
      stats[i].reliable_updates = nupd[i];
      stats[i].converged = conv ? 1 : 0;
      stats[i].rel_true_resid = rel;
      stats[i].time_s = secs;
    }
  }
  if (status != MDWF_OK) fail(ctx, status, "solve did not reach the tolerance within max_iter");
  return status;
}

int solve_dispatch(mdwf_ctx* ctx, int cfg_id, int n, const double* const* srcs, const double* masses,
                   double* const* xs, double tol, const mdwf_solver_opts* opts, mdwf_solve_stats* stats,
                   cudaStream_t st) {
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (n < 1 || n > 1024 || !srcs || !xs || !(tol > 0)) return fail(ctx, MDWF_ERR_ARG, "solve: bad n, pointers or tol");
  mdwf_solver_opts o;
  mdwf_default_opts(&o);
  if (opts) o = *opts;
  std::vector<double> m(n, cfg->act.mf);
  if (masses) for (int i = 0; i < n; i++) m[i] = masses[i];
  for (int i = 0; i < n; i++) if (!srcs[i] || !xs[i] || !std::isfinite(m[i])) return fail(ctx, MDWF_ERR_ARG, "solve: bad source/solution/mass");
  CK(cudaSetDevice(ctx->device));
  switch (o.precision) {
    case MDWF_PREC_DOUBLE: return solve_batch_impl<double>(ctx, cfg, n, srcs, m, xs, tol, o, stats, st);
    case MDWF_PREC_SINGLE: return solve_batch_impl<float>(ctx, cfg, n, srcs, m, xs, tol, o, stats, st);
    case MDWF_PREC_HALF: return solve_batch_impl<__half>(ctx, cfg, n, srcs, m, xs, tol, o, stats, st);
    case MDWF_PREC_BF16: return solve_batch_impl<__nv_bfloat16>(ctx, cfg, n, srcs, m, xs, tol, o, stats, st);
    default: return fail(ctx, MDWF_ERR_ARG, "solve: unknown precision");
  }
}

// Host 5D field -> device staging buffer (checks finiteness).
int upload5(mdwf_ctx* ctx, const double* h, size_t n, DBuf& d, cudaStream_t st) {
  if (!h) return fail(ctx, MDWF_ERR_ARG, "null input");
  if (!all_finite(h, n)) return fail(ctx, MDWF_ERR_NONFINITE, "input has NaN/Inf");
  CK(d.alloc(sizeof(double) * n));
  CK(cudaMemcpyAsync(d.p, h, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  return MDWF_OK;
}

// Generic FP64 operator on device API-layout 5D fields, single RHS.
//   kind 0: dslash (out_par, dagger)   1: mdwf D / D^+   2: 5D local op (op, dagger)
//   3: make_source walls -> source     4: Schur (dagger, precision)
template <typename S>
int schur_apply_impl(mdwf_ctx* ctx, Cfg* cfg, const double* in_dev, double* out_dev, int dagger, cudaStream_t st);

int apply_dev(mdwf_ctx* ctx, Cfg* cfg, int kind, int arg1, int arg2, const double* in_dev, double* out_dev,
              cudaStream_t st) {
  const Geom& g = ctx->g;
  const int L5 = cfg->act.L5;
  Op<double, double> op;
  op.g = g; op.L5 = L5; op.N = 1; op.anti = cfg->anti; op.U = cfg->U64; op.st = st;
  op.tl = tiling_for<double>(g, L5, 1, 2, true);
  Tables tab;
  tab.build(cfg->act, std::vector<double>(1, cfg->act.mf));
  DevTables<double> M;
  CK(M.upload(tab, st));
  long units = g.Vh * L5;
  FieldBuf<double> ie, io, oe, oo, te, to;
  for (auto* f : {&ie, &io, &oe, &oo, &te, &to}) CK(f->alloc(units));
  CK(pack_rhs<double>(in_dev, ie.v.as<double>(), nullptr, g, L5, 1, 0, 0, st));
  CK(pack_rhs<double>(in_dev, io.v.as<double>(), nullptr, g, L5, 1, 1, 0, st));
  CK(cudaMemsetAsync(oe.v.p, 0, oe.v.bytes, st));
  CK(cudaMemsetAsync(oo.v.p, 0, oo.v.bytes, st));
  F<double> none;
  if (kind == 0) {
    int par = arg1, dag = arg2;
    if (par == 0 || par == -1) CK(op.run(true, 0, dag, io.f(), none, nullptr, none, nullptr, 1.0, oe.f(), nullptr, nullptr));
    if (par == 1 || par == -1) CK(op.run(true, 1, dag, ie.f(), none, nullptr, none, nullptr, 1.0, oo.f(), nullptr, nullptr));
  } else if (kind == 1) {
    if (!arg1) {  // D x = A x - 1/2 H B x
      CK(op.run(false, 0, 0, ie.f(), none, M[MK_B], none, nullptr, 0.0, te.f(), nullptr, nullptr));
      CK(op.run(false, 1, 0, io.f(), none, M[MK_B], none, nullptr, 0.0, to.f(), nullptr, nullptr));
      CK(op.run(true, 0, 0, to.f(), ie.f(), M[MK_A], none, nullptr, -0.5, oe.f(), nullptr, nullptr));
      CK(op.run(true, 1, 0, te.f(), io.f(), M[MK_A], none, nullptr, -0.5, oo.f(), nullptr, nullptr));
    } else {      // D^+ x = A^+ x - 1/2 B^+ H^+ x
      CK(op.run(true, 0, 1, io.f(), ie.f(), M[MK_Ad], none, M[MK_Bd], -0.5, oe.f(), nullptr, nullptr));
      CK(op.run(true, 1, 1, ie.f(), io.f(), M[MK_Ad], none, M[MK_Bd], -0.5, oo.f(), nullptr, nullptr));
    }
  } else if (kind == 2) {
    static const int kinds[3][2] = {{MK_A, MK_Ad}, {MK_B, MK_Bd}, {MK_Ainv, MK_Ainvd}};
    const double* G = M[kinds[arg1][arg2 ? 1 : 0]];
    CK(op.run(false, 0, 0, ie.f(), none, G, none, nullptr, 0.0, oe.f(), nullptr, nullptr));
    CK(op.run(false, 1, 0, io.f(), none, G, none, nullptr, 0.0, oo.f(), nullptr, nullptr));
  } else if (kind == 3) {
    // src = (1 - c5 D_W) w = (1 - c5 d) w + c5/2 H w
    Tables sc;
    sc.L5 = L5; sc.N = 1;
    sc.h.assign(sc.block(), 0.0);
    const double f = 1.0 - cfg->act.c5 * (4.0 - cfg->act.M5);
    for (int chi = 0; chi < 2; chi++) for (int s = 0; s < L5; s++) sc.h[((size_t)chi * L5 + s) * L5 + s] = f;
    DevTables<double> G;
    CK(G.upload(sc, st));
    CK(op.run(true, 0, 0, io.f(), ie.f(), G[0], none, nullptr, 0.5 * cfg->act.c5, oe.f(), nullptr, nullptr));
    CK(op.run(true, 1, 0, ie.f(), io.f(), G[0], none, nullptr, 0.5 * cfg->act.c5, oo.f(), nullptr, nullptr));
  }
  CK(unpack_rhs<double>(oe.v.as<double>(), nullptr, out_dev, g, L5, 1, 0, 0, st));
  CK(unpack_rhs<double>(oo.v.as<double>(), nullptr, out_dev, g, L5, 1, 1, 0, st));
  CK(cudaStreamSynchronize(st));
  return MDWF_OK;
}

template <typename S>
int schur_apply_impl(mdwf_ctx* ctx, Cfg* cfg, const double* in_dev, double* out_dev, int dagger, cudaStream_t st) {
  using T = typename StoreTraits<S>::T;
  const Geom& g = ctx->g;
  const int L5 = cfg->act.L5;
  Op<S, T> op;
  op.g = g; op.L5 = L5; op.N = 1; op.anti = cfg->anti; op.st = st;
  op.U = std::is_same<T, double>::value ? (const T*)cfg->U64 : (const T*)cfg->U32;
  op.tl = tiling_for<S>(g, L5, 1, 2, true);
  Tables tab;
  tab.build(cfg->act, std::vector<double>(1, cfg->act.mf));
  DevTables<T> M;
  CK(M.upload(tab, st));
  long units = g.Vh * L5;
  FieldBuf<S> in, u, t, out;
  for (auto* f : {&in, &u, &t, &out}) CK(f->alloc(units));
  FieldBuf<double> o64;
  CK(o64.alloc(2 * units));
  CK(pack_rhs<S>(in_dev, in.f().v, in.f().n, g, L5, 1, 0, 0, st));
  CK(op.schur(dagger, in.f(), u.f(), t.f(), out.f(), M, nullptr, nullptr));
  CK(unpack_rhs<S>(out.f().v, out.f().n, out_dev, g, L5, 1, 0, 0, st));
  // zero odd sites of out: unpack a zero field into parity 1
  CK(cudaMemsetAsync(o64.v.p, 0, o64.v.bytes, st));
  CK(unpack_rhs<double>(o64.f().v, nullptr, out_dev, g, L5, 1, 1, 0, st));
  CK(cudaStreamSynchronize(st));
  return MDWF_OK;
}

// Host wrapper: upload, run, download.
int host_apply(mdwf_ctx* ctx, int cfg_id, int kind, int a1, int a2, const double* in, double* out, size_t n_in) {
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (!out) return fail(ctx, MDWF_ERR_ARG, "null output");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const size_t n5 = (size_t)cfg->act.L5 * ctx->g.V * 24;
  DBuf din, dout;
  rc = upload5(ctx, in, n_in, din, st);
  if (rc) return rc;
  CK(dout.alloc(sizeof(double) * n5));
  if (kind == 4) {
    switch (a2) {
      case MDWF_PREC_DOUBLE: rc = schur_apply_impl<double>(ctx, cfg, din.as<double>(), dout.as<double>(), a1, st); break;
      case MDWF_PREC_SINGLE: rc = schur_apply_impl<float>(ctx, cfg, din.as<double>(), dout.as<double>(), a1, st); break;
      case MDWF_PREC_HALF: rc = schur_apply_impl<__half>(ctx, cfg, din.as<double>(), dout.as<double>(), a1, st); break;
      case MDWF_PREC_BF16: rc = schur_apply_impl<__nv_bfloat16>(ctx, cfg, din.as<double>(), dout.as<double>(), a1, st); break;
      default: return fail(ctx, MDWF_ERR_ARG, "unknown precision");
    }
  } else {
    rc = apply_dev(ctx, cfg, kind, a1, a2, din.as<double>(), dout.as<double>(), st);
  }
  if (rc) return rc;
  CK(cudaMemcpyAsync(out, dout.p, sizeof(double) * n5, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return MDWF_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void mdwf_default_opts(mdwf_solver_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = MDWF_PREC_HALF;
  o->max_iter = 100000;
  o->delta = 0.1;
  o->chunk = 16;
  o->use_graph = 1;
  o->nsb = 2;
}

int mdwf_create(const int dims[4], int device, mdwf_ctx** out) {
  if (!dims || !out) return MDWF_ERR_ARG;
  for (int i = 0; i < 4; i++)
    if (dims[i] < 2 || (dims[i] & 1)) return MDWF_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MDWF_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return MDWF_ERR_CUDA;
  mdwf_ctx* c = new mdwf_ctx();
  c->device = device;
  c->g = make_geom(dims);
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return MDWF_ERR_CUDA; }
  *out = c;
  return MDWF_OK;
}

int mdwf_destroy(mdwf_ctx* ctx) {
  if (!ctx) return MDWF_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->cfgs) {
    if (kv.second.U64) cudaFree(kv.second.U64);
    if (kv.second.U32) cudaFree(kv.second.U32);
  }
  cudaStreamDestroy(ctx->stream);
  delete ctx;
  return MDWF_OK;
}

const char* mdwf_last_error(const mdwf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int mdwf_load_gauge(mdwf_ctx* ctx, int cfg_id, const double* U, int t_antiperiodic) {
  if (!ctx) return MDWF_ERR_ARG;
  if (!U || cfg_id < 0) return fail(ctx, MDWF_ERR_ARG, "load_gauge: null field or negative cfg_id");
  const Geom& g = ctx->g;
  const size_t n = (size_t)g.V * 4 * 18;
  if (!all_finite(U, n)) return fail(ctx, MDWF_ERR_NONFINITE, "gauge field has NaN/Inf");
  // reorder to [parity][h][mu][18]
  std::vector<double> h64(n);
  std::vector<float> h32(n);
  for (long lex = 0; lex < g.V; lex++) {
    long r = lex;
    int c[4];
    for (int i = 0; i < 4; i++) { c[i] = (int)(r % g.L[i]); r /= g.L[i]; }
    int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    long h = lex >> 1;
    for (int mu = 0; mu < 4; mu++)
      for (int k = 0; k < 18; k++) {
        double v = U[(lex * 4 + mu) * 18 + k];
        size_t dst = (((size_t)par * g.Vh + h) * 4 + mu) * 18 + k;
        h64[dst] = v;
        h32[dst] = (float)v;
      }
  }
  CK(cudaSetDevice(ctx->device));
  Cfg& cfg = ctx->cfgs[cfg_id];
  if (!cfg.U64) CK(cudaMalloc(&cfg.U64, sizeof(double) * n));
  if (!cfg.U32) CK(cudaMalloc(&cfg.U32, sizeof(float) * n));
  CK(cudaMemcpy(cfg.U64, h64.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(cfg.U32, h32.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
  cfg.has_gauge = true;
  cfg.anti = t_antiperiodic ? 1 : 0;
  return MDWF_OK;
}

int mdwf_set_action(mdwf_ctx* ctx, int cfg_id, double M5, double b5, double c5, double mf, int L5) {
  if (!ctx) return MDWF_ERR_ARG;
  if (cfg_id < 0 || L5 < 2 || L5 > 32 || !std::isfinite(M5) || !std::isfinite(b5) || !std::isfinite(c5) ||
      !std::isfinite(mf))
    return fail(ctx, MDWF_ERR_ARG, "set_action: bad parameters");
  double alpha = b5 * (4.0 - M5) + 1.0;
  if (alpha == 0.0) return fail(ctx, MDWF_ERR_ARG, "set_action: b5 (4 - M5) + 1 must be nonzero");
  Action& a = ctx->cfgs[cfg_id].act;
  a.M5 = M5; a.b5 = b5; a.c5 = c5; a.mf = mf; a.L5 = L5; a.set = true;
  return MDWF_OK;
}

int mdwf_apply_dslash(mdwf_ctx* ctx, int cfg_id, const double* in, double* out, int out_parity, int dagger) {
  if (!ctx) return MDWF_ERR_ARG;
  if (out_parity < -1 || out_parity > 1) return fail(ctx, MDWF_ERR_ARG, "apply_dslash: out_parity must be -1, 0 or 1");
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  return host_apply(ctx, cfg_id, 0, out_parity, dagger ? 1 : 0, in, out, (size_t)cfg->act.L5 * ctx->g.V * 24);
}

int mdwf_apply_mdwf(mdwf_ctx* ctx, int cfg_id, const double* in, double* out, int dagger) {
  if (!ctx) return MDWF_ERR_ARG;
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  return host_apply(ctx, cfg_id, 1, dagger ? 1 : 0, 0, in, out, (size_t)cfg->act.L5 * ctx->g.V * 24);
}

int mdwf_apply_schur(mdwf_ctx* ctx, int cfg_id, const double* in, double* out, int dagger, int precision) {
  if (!ctx) return MDWF_ERR_ARG;
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  return host_apply(ctx, cfg_id, 4, dagger ? 1 : 0, precision, in, out, (size_t)cfg->act.L5 * ctx->g.V * 24);
}

int mdwf_apply_5d(mdwf_ctx* ctx, int cfg_id, int op, const double* in, double* out, int dagger) {
  if (!ctx) return MDWF_ERR_ARG;
  if (op < 0 || op > 2) return fail(ctx, MDWF_ERR_ARG, "apply_5d: op must be 0 (A), 1 (B) or 2 (A^-1)");
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  return host_apply(ctx, cfg_id, 2, op, dagger ? 1 : 0, in, out, (size_t)cfg->act.L5 * ctx->g.V * 24);
}

int mdwf_make_source(mdwf_ctx* ctx, int cfg_id, const double* eta4d, double* src5d) {
  if (!ctx) return MDWF_ERR_ARG;
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (!eta4d || !src5d) return fail(ctx, MDWF_ERR_ARG, "make_source: null pointer");
  const long V = ctx->g.V;
  const int L5 = cfg->act.L5;
  if (!all_finite(eta4d, (size_t)V * 24)) return fail(ctx, MDWF_ERR_NONFINITE, "source has NaN/Inf");
  // walls: P_+ eta on s = 0 (spins 0,1), P_- eta on s = L5-1 (spins 2,3)
  std::vector<double> w((size_t)L5 * V * 24, 0.0);
  for (long x = 0; x < V; x++)
    for (int k = 0; k < 24; k++) {
      int spin = k / 6;
      if (spin < 2) w[(size_t)x * 24 + k] = eta4d[(size_t)x * 24 + k];
      else w[((size_t)(L5 - 1) * V + x) * 24 + k] = eta4d[(size_t)x * 24 + k];
    }
  return host_apply(ctx, cfg_id, 3, 0, 0, w.data(), src5d, w.size());
}

int mdwf_solve_batch(mdwf_ctx* ctx, int cfg_id, int n, const double* const* srcs, const double* masses,
                     double* const* xs, double tol, const mdwf_solver_opts* opts, mdwf_solve_stats* stats) {
  if (!ctx) return MDWF_ERR_ARG;
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (n < 1 || n > 1024 || !srcs || !xs) return fail(ctx, MDWF_ERR_ARG, "solve_batch: bad n or pointers");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const size_t n5 = (size_t)cfg->act.L5 * ctx->g.V * 24;
  DBuf dsrc, dx;
  CK(dsrc.alloc(sizeof(double) * n5 * n));
  CK(dx.alloc(sizeof(double) * n5 * n));
  std::vector<const double*> s(n);
  std::vector<double*> x(n);
  for (int i = 0; i < n; i++) {
    if (!srcs[i] || !xs[i]) return fail(ctx, MDWF_ERR_ARG, "solve_batch: null source or solution");
    if (!all_finite(srcs[i], n5)) return fail(ctx, MDWF_ERR_NONFINITE, "source has NaN/Inf");
    CK(cudaMemcpyAsync(dsrc.as<double>() + n5 * i, srcs[i], sizeof(double) * n5, cudaMemcpyHostToDevice, st));
    s[i] = dsrc.as<double>() + n5 * i;
    x[i] = dx.as<double>() + n5 * i;
  }
  rc = solve_dispatch(ctx, cfg_id, n, s.data(), masses, x.data(), tol, opts, stats, st);
  if (rc != MDWF_OK && rc != MDWF_ERR_NOT_CONVERGED) return rc;
  for (int i = 0; i < n; i++)
    CK(cudaMemcpyAsync(xs[i], x[i], sizeof(double) * n5, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return rc;
}

int mdwf_solve(mdwf_ctx* ctx, int cfg_id, const double* src5d, double* x5d, double tol, const mdwf_solver_opts* opts,
               mdwf_solve_stats* stats) {
  return mdwf_solve_batch(ctx, cfg_id, 1, &src5d, nullptr, &x5d, tol, opts, stats);
}

int mdwf_solve_batch_dev(mdwf_ctx* ctx, int cfg_id, int n, const double* const* srcs, const double* masses,
                         double* const* xs, double tol, const mdwf_solver_opts* opts, mdwf_solve_stats* stats,
                         void* stream) {
  if (!ctx) return MDWF_ERR_ARG;
  return solve_dispatch(ctx, cfg_id, n, srcs, masses, xs, tol, opts, stats, pick_stream(ctx, stream));
}

int mdwf_apply_dslash_dev(mdwf_ctx* ctx, int cfg_id, const double* in, double* out, int out_parity, int dagger,
                          void* stream) {
  if (!ctx) return MDWF_ERR_ARG;
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (!in || !out || out_parity < -1 || out_parity > 1) return fail(ctx, MDWF_ERR_ARG, "apply_dslash_dev: bad args");
  CK(cudaSetDevice(ctx->device));
  return apply_dev(ctx, cfg, 0, out_parity, dagger ? 1 : 0, in, out, pick_stream(ctx, stream));
}

int mdwf_apply_mdwf_dev(mdwf_ctx* ctx, int cfg_id, const double* in, double* out, int dagger, void* stream) {
  if (!ctx) return MDWF_ERR_ARG;
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (!in || !out) return fail(ctx, MDWF_ERR_ARG, "apply_mdwf_dev: null pointer");
  CK(cudaSetDevice(ctx->device));
  return apply_dev(ctx, cfg, 1, dagger ? 1 : 0, 0, in, out, pick_stream(ctx, stream));
}

int mdwf_extract_prop4d(const double* x5d, const int dims[4], int L5, double* q4d) {
  if (!x5d || !dims || !q4d || L5 < 1) return MDWF_ERR_ARG;
  long V = 1;
  for (int i = 0; i < 4; i++) { if (dims[i] < 1) return MDWF_ERR_ARG; V *= dims[i]; }
  for (long x = 0; x < V; x++)
    for (int k = 0; k < 24; k++) {
      int spin = k / 6;   // P_+ (spins 0,1) from s = L5-1, P_- (spins 2,3) from s = 0
      q4d[x * 24 + k] = spin < 2 ? x5d[((size_t)(L5 - 1) * V + x) * 24 + k] : x5d[(size_t)x * 24 + k];
    }
  return MDWF_OK;
}

}  // extern "C"
