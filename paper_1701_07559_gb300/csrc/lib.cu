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
// Options: the symmetric form A^-1 Mhat (opts.schur = 1, the alternative Sec. VII
// names), the hop form chosen by timing (the autotuner), and solver sessions that
// keep the CG state of a set of slots resident and admit requests between chunks
// (continuous batching).  Device workspace is cached per context and reused: no
// call on the request path allocates or frees device memory once it exists.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <array>
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
  uint32_t* F16 = nullptr;  // tensor-core hop: fp16 B fragments [parity][h][mu][fwd, bwd][32 lanes]
  float* U12 = nullptr;     // two-row FP32 links for 12-real reconstruction (built on first use)
  Action act;
};

struct mdwf_ctx {
  int device = 0;
  Geom g;
  std::map<int, Cfg> cfgs;
  std::string err;
  cudaStream_t stream = nullptr;
  std::map<std::string, std::pair<void*, size_t>> ws;  // reusable device workspace
  int next_session = 0;
  // autotuned hop form per (L5, N, storage precision, candidate set): {variant, nsb}, best ms
  std::map<std::array<int, 4>, std::pair<std::array<int, 2>, double>> tuned;
};

struct SessionBase {
  virtual ~SessionBase() {}
  virtual int submit(const double* src, double mass, double* x, long long tag, int* slot) = 0;
  virtual int launch(int iters) = 0;
  virtual int poll(int max_done, long long* tags, mdwf_solve_stats* stats, int* n_done) = 0;
  virtual int occupied() const = 0;
};

struct mdwf_session {
  mdwf_ctx* ctx = nullptr;
  SessionBase* impl = nullptr;
  std::string prefix;
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
  T* ext = nullptr;     // a buffer of the context's workspace instead of buf (no allocation per call)
  size_t blk = 0;
  cudaError_t upload(const Tables& t, cudaStream_t st, T* into = nullptr) {
    blk = t.block();
    std::vector<T> v(t.h.size());
    for (size_t i = 0; i < v.size(); i++) v[i] = (T)t.h[i];
    ext = into;
    if (!ext) {
      cudaError_t e = buf.alloc(sizeof(T) * v.size());
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemcpyAsync(base(), v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
  }
  T* base() const { return ext ? ext : buf.as<T>(); }
  const T* operator[](int k) const { return base() + (size_t)k * blk; }
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

// Event timing of hop launches: pairs of events around every launch, either
// recorded directly (collected after the next stream synchronisation) or
// captured into a CUDA graph (collected after each graph launch).
struct Prof {
  std::vector<cudaEvent_t> pool, gpool;
  size_t used = 0, gused = 0;
  bool capturing = false;
  double ms = 0.0;
  long long n = 0;
  ~Prof() {
    for (auto e : pool) cudaEventDestroy(e);
    for (auto e : gpool) cudaEventDestroy(e);
  }
  cudaError_t record(cudaStream_t st) {
    std::vector<cudaEvent_t>& v = capturing ? gpool : pool;
    size_t& u = capturing ? gused : used;
    if (u >= v.size()) {
      cudaEvent_t e;
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return err;
      v.push_back(e);
    }
    // inside a capture only an "external" record becomes an event node of the graph
    return capturing ? cudaEventRecordWithFlags(v[u++], st, cudaEventRecordExternal) : cudaEventRecord(v[u++], st);
  }
  cudaError_t sum(const std::vector<cudaEvent_t>& v, size_t u) {
    for (size_t i = 0; i + 1 < u; i += 2) {
      float t = 0.f;
      cudaError_t err = cudaEventElapsedTime(&t, v[i], v[i + 1]);
      if (err != cudaSuccess) return err;
      ms += t;
      n += 1;
    }
    return cudaSuccess;
  }
  cudaError_t collect() { cudaError_t e = sum(pool, used); used = 0; return e; }   // after a sync
  cudaError_t collect_graph() { return sum(gpool, gused); }                        // after a graph launch + sync
};

template <typename S, typename T>
struct Op {
  Geom g;
  int L5 = 0, N = 0, anti = 1;
  const T* U = nullptr;
  Tiling tl;
  cudaStream_t st = nullptr;
  Prof* prof = nullptr;          // time hop launches when set
  long long* launches = nullptr; // count launches when set

  // out = add + G same + kappa C H(in)   (hop) ; out = add + G in (local)
  cudaError_t run(bool hop, int out_par, int dagger, F<S> in, F<S> same, const T* G, F<S> add, const T* C, T kappa,
                  F<S> out, const int* active, double* partials) const {
    HopArgs<S, T> a;
    a.g = g; a.L5 = L5; a.N = N; a.out_par = out_par; a.dagger = dagger; a.antiperiodic = anti;
    a.in = in.v; a.in_nrm = in.n; a.same = same.v; a.same_nrm = same.n; a.add = add.v; a.add_nrm = add.n;
    a.out = out.v; a.out_nrm = out.n; a.U = U; a.Gm = G; a.Cm = C; a.kappa = kappa; a.active = active;
    a.partials = partials;
    if (launches) *launches += 1;
    if (prof && hop) {
      cudaError_t e = prof->record(st);
      if (e != cudaSuccess) return e;
      e = launch_hop<S, T>(a, tl, hop, st);
      if (e != cudaSuccess) return e;
      return prof->record(st);
    }
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
  double *gamma, *gamma_prev, *alpha, *beta, *rho2, *rho2_max, *stop2, *qq, *rr, *tmp, *bhat2, *upd2;
  int *active, *flags, *iters;
  int* since;     // CG iterations since the last reliable update of the slot
  int stag_max;   // that many without one: the inner recursion stagnates (see k_after_rho)
  double delta2;  // periodic reliable update when |rho|^2 < delta2 * max |rho|^2 since the last one
  double tau2;    // FP64 re-reference when |rho|^2 <= tau2 * |bhat|^2 (bhat = current reference residual)
};
enum { FLAG_INNER_DONE = 1, FLAG_UPDATE = 2, FLAG_DONE = 4, FLAG_REREF = 8, FLAG_STAG = 16 };

__global__ void k_alpha(Scal c, int N) {
  int r = threadIdx.x;
  if (r < N && c.active[r]) { double q = c.qq[r]; c.alpha[r] = q > 0.0 ? c.gamma[r] / q : 0.0; }
}
// The low-precision residual recursion can stagnate for a system whose
// residual is already tiny: it neither reaches the stopping norm nor drops by
// delta, so no update would ever come.  After stag_max iterations without an
// update one is forced; it is followed by an FP64 re-reference and a restart of
// the search direction (beta = 0).
__global__ void k_after_rho(Scal c, int N) {
  int r = threadIdx.x;
  if (r < N && c.active[r]) {
    double v = c.tmp[r];
    c.rho2[r] = v;
    if (v > c.rho2_max[r]) c.rho2_max[r] = v;
    if (v <= c.stop2[r]) { c.active[r] = 0; c.flags[r] |= FLAG_INNER_DONE; }
    else if (v < c.delta2 * c.rho2_max[r] || v <= c.tau2 * c.bhat2[r]) c.flags[r] |= FLAG_UPDATE;
    else if (c.since[r] >= c.stag_max) c.flags[r] |= FLAG_UPDATE | FLAG_STAG;
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
    c.since[r] += 1;
  }
}
// After a residual recomputed with FP32 arithmetic.  Its error grows like
// 1e-7 kappa(Mhat) |bhat| (x_hi, accumulated since the last re-reference, is
// about kappa times bhat), so for light quarks it can sit above any fixed
// re-reference threshold.  An FP64 re-reference is requested when the residual
// reached tau |bhat|, when it fell below the stopping norm (the FP64 residual
// decides), or when it did not halve since the previous FP32 update (its
// accuracy floor).  Convergence is accepted on the FP32 residual alone only
// when bhat itself is within 10^3 of the stopping norm.  (tau = 1e-5.)
__global__ void k_after_update(Scal c, int N, const int* um) {
  int r = threadIdx.x;
  if (r < N && um[r]) {
    double v = c.tmp[r];
    const double prev = c.upd2[r];
    c.rho2[r] = v;
    c.rho2_max[r] = v;
    c.upd2[r] = v;
    c.gamma[r] = c.rr[r];
    c.beta[r] = c.gamma_prev[r] > 0.0 ? c.gamma[r] / c.gamma_prev[r] : 0.0;
    const bool fine = c.bhat2[r] <= 1e6 * c.stop2[r];
    const bool stag = (c.flags[r] & FLAG_STAG) != 0;
    const bool stalled = stag || (prev > 0.0 && v > 0.25 * prev);
    c.since[r] = 0;
    if (v <= c.stop2[r] && fine) { c.flags[r] = FLAG_DONE; c.active[r] = 0; }
    else if (v <= c.stop2[r] || v <= c.tau2 * c.bhat2[r] || stalled) {
      c.flags[r] = FLAG_REREF | (stag ? FLAG_STAG : 0);
      c.active[r] = 1;
    } else { c.flags[r] = 0; c.active[r] = 1; }
  }
}
// After an FP64 re-reference (bhat <- rho, x_acc += x_hi).
__global__ void k_after_reref(Scal c, int N, const int* um) {
  int r = threadIdx.x;
  if (r < N && um[r]) {
    double v = c.tmp[r];
    c.rho2[r] = v;
    c.rho2_max[r] = v;
    c.bhat2[r] = v;
    c.upd2[r] = 0.0;
    c.gamma[r] = c.rr[r];
    // after a stagnation the search direction restarts from the new residual
    c.beta[r] = (c.gamma_prev[r] > 0.0 && !(c.flags[r] & FLAG_STAG)) ? c.gamma[r] / c.gamma_prev[r] : 0.0;
    c.since[r] = 0;
    if (v <= c.stop2[r]) { c.flags[r] = FLAG_DONE; c.active[r] = 0; }
    else { c.flags[r] = 0; c.active[r] = 1; }
  }
}

// ---------------------------------------------------------------------------
// Fast operator passes
// ---------------------------------------------------------------------------
template <typename S, typename T>
struct FastOp {
  Geom g;
  int L5 = 0, N = 0, anti = 1;
  const T* U = nullptr;
  Tiling tl;
  cudaStream_t st = nullptr;
  Fifth<T> f;
  Prof* prof = nullptr;
  long long* launches = nullptr;
  const StageInfo* stage = nullptr;   // neighbour staging through shared memory, when the tiling allows
  const uint32_t* F16 = nullptr;      // fp16 link fragments for the tensor-core hop
  const float* U12 = nullptr;         // two-row links: the paired hop reconstructs the third row
  const T* halo_fwd = nullptr;        // time-split domain decomposition: faces of the neighbours
  const T* halo_bwd = nullptr;
  T halo_sgn_fwd = T(1), halo_sgn_bwd = T(1);
  bool mma = false;                   // use the tensor-core hop (fp16 storage only)
  bool mma_pipelined = false;         // its bulk-copy pipelined form

  cudaError_t dispatch(const FastArgs<S, T>& a, int epi) const {
    if constexpr (std::is_same<S, __half>::value) {
      if (mma) return launch_fast_mma(a, tl, epi, st, stage, mma_pipelined);
    }
    return launch_fast<S, T>(a, tl, epi, st, stage);
  }

  cudaError_t run(int epi, int out_par, int dagger, F<S> in, F<S> same, F<S> add, T g_same, T kappa, F<S> out,
                  const int* active, double* partials) const {
    FastArgs<S, T> a;
    a.g = g; a.L5 = L5; a.N = N; a.out_par = out_par; a.dagger = dagger; a.antiperiodic = anti;
    a.in = in.v; a.in_nrm = in.n; a.same = same.v; a.same_nrm = same.n; a.add = add.v; a.add_nrm = add.n;
    a.out = out.v; a.out_nrm = out.n; a.U = U; a.F16 = F16; a.U12 = U12; a.f = f; a.g_same = g_same;
    a.kappa = kappa;
    a.halo_fwd = halo_fwd; a.halo_bwd = halo_bwd; a.halo_sgn_fwd = halo_sgn_fwd; a.halo_sgn_bwd = halo_sgn_bwd;
    a.active = active;
    a.partials = partials;
    if (launches) *launches += 1;
    if (prof) {
      cudaError_t e = prof->record(st);
      if (e != cudaSuccess) return e;
      e = dispatch(a, epi);
      if (e != cudaSuccess) return e;
      return prof->record(st);
    }
    return dispatch(a, epi);
  }
  // q = Mhat p (needs u = B p already formed) ; t scratch (odd)
  cudaError_t mhat(F<S> p, F<S> u, F<S> t, F<S> q, const int* active, double* partials) const {
    F<S> none;
    cudaError_t e = run(E_BAINV, 1, 0, u, none, none, T(0), T(1), t, active, nullptr);
    if (e != cudaSuccess) return e;
    return run(E_A_SAME, 0, 0, t, p, none, T(1), T(-0.25), q, active, partials);
  }
  // r = Mhat^+ v ; t scratch (odd)
  cudaError_t mhat_dag(F<S> v, F<S> t, F<S> r, const int* active, double* partials) const {
    F<S> none;
    cudaError_t e = run(E_AINVD_BD, 1, 1, v, none, none, T(0), T(1), t, active, nullptr);
    if (e != cudaSuccess) return e;
    return run(E_AD_SAME_BD, 0, 1, t, v, none, T(1), T(-0.25), r, active, partials);
  }
  // Symmetric form Mhat_s = A^-1 Mhat = 1 - 1/4 A^-1 H B A^-1 H B:  q = p + A^-1 (-1/4 H t)
  cudaError_t mhat_sym(F<S> p, F<S> u, F<S> t, F<S> q, const int* active, double* partials) const {
    F<S> none;
    cudaError_t e = run(E_BAINV, 1, 0, u, none, none, T(0), T(1), t, active, nullptr);
    if (e != cudaSuccess) return e;
    return run(E_SAME_AINV, 0, 0, t, p, none, T(1), T(-0.25), q, active, partials);
  }
  // Mhat_s^+ v = Mhat^+ A^-+ v = v - 1/4 B^+ H^+ A^-+ B^+ H^+ w,  w = A^-+ v ; w, t scratch
  cudaError_t mhat_sym_dag(F<S> v, F<S> w, F<S> t, F<S> r, const int* active, double* partials) const {
    F<S> none;
    cudaError_t e = run(E_AINVD_SAME, 0, 1, none, v, none, T(0), T(0), w, active, nullptr);
    if (e != cudaSuccess) return e;
    e = run(E_AINVD_BD, 1, 1, w, none, none, T(0), T(1), t, active, nullptr);
    if (e != cudaSuccess) return e;
    return run(E_SAME_BD, 0, 1, t, v, none, T(1), T(-0.25), r, active, partials);
  }
};

// Tiling of the fast hop kernels.  Storage types narrower than FP64 stage the
// neighbour sites in shared memory when a block can hold whole sites (all N
// slots of nsb sites, at most ~200 KB of staging); FP64 runs unstaged.
// Hop kernel variants: 0 automatic, 1 CUDA-core direct loads (two slices per thread for FP32
// arithmetic), 2 CUDA-core staged, 3 tensor-core (fp16), 6 CUDA-core direct, one unit per thread.
enum { HOP_AUTO = 0, HOP_DIRECT = 1, HOP_STAGED = 2, HOP_MMA = 3, HOP_TUNE_ALL = 4, HOP_MMA_PIPE = 5,
       HOP_UNIT = 6, HOP_PAIR_PF = 7 };

template <typename S>
Tiling fast_tiling(const Geom& g, int L5, int N, int nsb_req, bool* staged, bool allow_staging);

// Tiling and kernel choice of a FastOp.
template <typename S, typename T>
void choose_hop(FastOp<S, T>& op, const Cfg* cfg, int nsb_req, int variant, const StageInfo* stage) {
  const Geom& g = op.g;
  const int L5 = op.L5, N = op.N, upb = L5 * N;
  bool staged = false;
  op.mma = false;
  op.mma_pipelined = variant == HOP_MMA_PIPE;
  if (variant == HOP_MMA_PIPE) variant = HOP_MMA;
  op.stage = nullptr;
  op.F16 = cfg->F16;
  if (variant == HOP_MMA && std::is_same<S, __half>::value && cfg->F16) {
    // whole sites per block; prefer a whole number of warps and 128..512 threads
    int nsb = 0;
    for (int k = 1; k <= 64 && nsb == 0; k++)
      if ((k * upb) % 32 == 0 && k * upb >= 128 && k * upb <= 512) nsb = k;
    if (nsb == 0) nsb = upb >= 128 ? 1 : (128 + upb - 1) / upb;
    if (nsb_req > 0) nsb = nsb_req;
    if (nsb > 64) nsb = 64;
    const int maxthr = mma_max_threads();
    while (nsb > 1 && nsb * L5 > maxthr) nsb--;
    op.tl = make_tiling(g.Vh, L5, N, nsb, maxthr);
    if (mma_hop_usable(op.tl, L5, N)) { op.mma = true; op.stage = stage; return; }
  }
  op.tl = fast_tiling<S>(g, L5, N, nsb_req, &staged, variant == HOP_STAGED);
  op.tl.form = variant == HOP_UNIT ? 1 : variant == HOP_PAIR_PF ? 2 : 0;
  op.stage = staged ? stage : nullptr;
}

template <typename S>
Tiling fast_tiling(const Geom& g, int L5, int N, int nsb_req, bool* staged, bool allow_staging) {
  using T = typename StoreTraits<S>::T;
  int maxthr = fast_max_threads<S, T>();
  if (maxthr > 1024) maxthr = 1024;
  const int upb = L5 * N;
  *staged = false;
  if (allow_staging && !std::is_same<S, double>::value && upb <= maxthr) {
    int nsb = nsb_req > 0 ? nsb_req : (128 / upb > 1 ? 128 / upb : 1);
    if (nsb > 64) nsb = 64;
    for (; nsb >= 1; nsb--) {
      if (nsb * upb > maxthr) continue;
      Tiling t = make_tiling(g.Vh, L5, N, nsb, nsb * upb);
      if (t.rt == N && staged_smem_bytes<S, T>(t, L5, N) <= 110 * 1024) { *staged = true; return t; }
    }
  }
  int smem_thr = (int)(200 * 1024 / (25 * sizeof(T)));
  if (smem_thr < maxthr) maxthr = smem_thr;
  int nsb = nsb_req > 0 ? nsb_req : 2;
  if (nsb > 64) nsb = 64;
  // by default keep every RHS slot of a site in one block (no ragged slot groups,
  // whose idle lanes cost the FP64 hop 40 % of its time when 2 sites did not fit)
  if (nsb_req <= 0)
    while (nsb > 1 && nsb * L5 * N > maxthr) nsb--;
  return make_tiling(g.Vh, L5, N, nsb, maxthr);
}

// Bound of device-side waits in clock cycles.
long long wait_budget(int device, double seconds) {
  int khz = 0;
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device) != cudaSuccess || khz <= 0) khz = 2000000;
  return (long long)(seconds * 1e3 * (double)khz);
}

template <typename T>
Fifth<T> make_fifth(const Action& act, const T* mass_dev) {
  Fifth<T> f;
  const double d = 4.0 - act.M5;
  const double alpha = act.b5 * d + 1.0, beta = act.c5 * d - 1.0;
  f.alpha = (T)alpha; f.beta = (T)beta; f.b5 = (T)act.b5; f.c5 = (T)act.c5;
  f.inv_alpha = (T)(1.0 / alpha); f.kap = (T)(beta / alpha);
  f.powL = (T)std::pow(-beta / alpha, act.L5);
  f.mass = mass_dev;
  return f;
}

// Named device buffers of a context, reused across calls (grown on demand).
void* ws_get(mdwf_ctx* ctx, const std::string& name, size_t bytes, cudaError_t* err) {
  auto& e = ctx->ws[name];
  if (e.second < bytes) {
    if (e.first) cudaFree(e.first);
    e.first = nullptr;
    e.second = 0;
    *err = cudaMalloc(&e.first, bytes ? bytes : 16);
    if (*err != cudaSuccess) return nullptr;
    e.second = bytes;
  }
  return e.first;
}

// Tables uploaded into a named workspace buffer of the context (no allocation once it exists).
template <typename T>
cudaError_t upload_tables_ws(mdwf_ctx* ctx, const std::string& name, const Tables& t, DevTables<T>* M,
                             cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  T* p = (T*)ws_get(ctx, name, sizeof(T) * t.h.size(), &e);
  if (e != cudaSuccess) return e;
  return M->upload(t, st, p);
}

template <typename S>
cudaError_t ws_field(mdwf_ctx* ctx, const std::string& name, long units, F<S>* f) {
  cudaError_t e = cudaSuccess;
  f->v = (S*)ws_get(ctx, name + ".v", sizeof(S) * 24 * (size_t)units, &e);
  if (e != cudaSuccess) return e;
  f->n = nullptr;
  if (StoreTraits<S>::kNorm) f->n = (float*)ws_get(ctx, name + ".n", sizeof(float) * (size_t)units, &e);
  return e;
}

// ---------------------------------------------------------------------------
// The batched solver
// ---------------------------------------------------------------------------
template <typename S>
struct BatchSolver {
  using T = typename StoreTraits<S>::T;
  using SX = typename std::conditional<std::is_same<S, double>::value, double, float>::type;
  static constexpr bool kFP64 = std::is_same<S, double>::value;

  mdwf_ctx* ctx;
  const Cfg* cfg;
  int N, L5;
  FastOp<double, double> op64;
  FastOp<float, float> op32;
  FastOp<S, T> opS;
  Tiling tl_blas;
  // FP64: sources, solution (x_acc + x_hi on even sites, x_o), reference residual bhat.
  // The batch solve keeps no x_o of its own: its reconstruction writes the odd
  // sites into x_hi, which is free by then (solve_batch_impl, finish).
  F<double> b_e, b_o, x_acc, x_hi, x_o, bhat, rho64, u64, t64;
  F<float> xf, uf, tf, qf;       // FP32 reliable updates
  F<S> p, u, t, q, rho, r;       // inner vectors
  F<SX> xlo;
  long xlo_n = 0;                 // units x_lo holds (tile-major FP32: the whole BLAS grid)
  double* part = nullptr;
  double* mass64 = nullptr;
  float* mass32 = nullptr;
  Scal sc;
  int* umask_d = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;
  long long launches = 0, graph_launches = 0;
  Prof prof;
  bool profiling = false;
  StageInfo stage;
  int* errw = nullptr;            // device status word of the bounded waits
  std::string wsp;                // prefix of this solver's workspace names (sessions own theirs)
  int tune_request = -1;          // HOP_AUTO / HOP_TUNE_ALL: pick the inner hop form by timing (tune())
  // Sources b_e, b_o: own fields (sessions, whose sources arrive one at a time), or
  // views of fields that are free when they are needed (the batch solve: rho64 and
  // x_hi before the iterations, bhat and x_hi after them; repacked from the caller's
  // sources, which stay valid for the whole call)
  bool own_b = false;
  bool sym = false;               // symmetric Schur form (opts.schur == 1)

  ~BatchSolver() { if (graph) cudaGraphExecDestroy(graph); }

  int init(mdwf_ctx* c, const Cfg* cf, const std::vector<double>& masses, int nsb, bool profile,
           const mdwf_solver_opts& o, cudaStream_t st) {
    mdwf_ctx* ctx = c;
    this->ctx = c;
    cfg = cf;
    N = (int)masses.size();
    L5 = cf->act.L5;
    const Geom& g = c->g;
    long units = g.Vh * L5 * N;
    cudaError_t e = cudaSuccess;
    mass64 = (double*)ws_get(c, wsp + "mass64", sizeof(double) * N, &e); CK(e);
    mass32 = (float*)ws_get(c, wsp + "mass32", sizeof(float) * N, &e); CK(e);
    std::vector<float> m32(masses.begin(), masses.end());
    CK(cudaMemcpyAsync(mass64, masses.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(mass32, m32.data(), sizeof(float) * N, cudaMemcpyHostToDevice, st));
    op64.g = g; op64.L5 = L5; op64.N = N; op64.anti = cf->anti; op64.U = cf->U64; op64.st = st;
    op64.f = make_fifth<double>(cf->act, mass64);
    op32.g = g; op32.L5 = L5; op32.N = N; op32.anti = cf->anti; op32.U = cf->U32; op32.st = st;
    op32.f = make_fifth<float>(cf->act, mass32);
    opS.g = g; opS.L5 = L5; opS.N = N; opS.anti = cf->anti; opS.st = st;
    opS.U = kFP64 ? (const T*)cf->U64 : (const T*)cf->U32;
    opS.f = make_fifth<T>(cf->act, kFP64 ? (const T*)mass64 : (const T*)mass32);
    if (nsb * L5 > 1024) nsb = 1;
    tl_blas = make_tiling(g.Vh, L5, N, 2, kFP64 ? 512 : 1024);
    errw = (int*)ws_get(c, wsp + "errw", sizeof(int), &e); CK(e);
    CK(cudaMemsetAsync(errw, 0, sizeof(int), st));
    stage.spin_bytes = stage.nrm_bytes = 0;
    stage.budget = wait_budget(c->device, o.wait_timeout_s > 0 ? o.wait_timeout_s : 2.0);
    stage.extra_tx = o.timeout_test ? 16u : 0u;
    stage.err = errw;
    // the wait-timeout test needs a kernel with waits: the staged one, or the
    // pipelined tensor-core one when that variant is asked for
    sym = o.schur == 1;
    int variant = o.timeout_test ? (o.hop_variant == HOP_MMA_PIPE ? HOP_MMA_PIPE : HOP_STAGED) : o.hop_variant;
    // the symmetric form's epilogues exist in the CUDA-core hops only
    if (sym && (variant == HOP_MMA || variant == HOP_MMA_PIPE || variant == HOP_TUNE_ALL)) variant = HOP_AUTO;
    choose_hop(op64, cf, 0, HOP_DIRECT, &stage);
    choose_hop(op32, cf, nsb, (variant == HOP_AUTO || variant == HOP_TUNE_ALL) ? HOP_DIRECT : variant, &stage);
    choose_hop(opS, cf, nsb, (variant == HOP_AUTO || variant == HOP_TUNE_ALL) ? HOP_DIRECT : variant, &stage);
    tune_request = (variant == HOP_AUTO || variant == HOP_TUNE_ALL) && nsb == 0 ? variant : -1;
    // 12-real links (the third row reconstructed) for the inner hops; the FP32
    // reliable updates keep the full links
    opS.U12 = (!kFP64 && o.link_recon == 12) ? cf->U12 : nullptr;
    if (!kFP64 && o.link_recon == 12 && cf->U12 == nullptr)
      return fail(c, MDWF_ERR_STATE, "12-real links requested but not built");
    op64.launches = op32.launches = opS.launches = &launches;
    profiling = profile;
    F<double>* f64[] = {&x_acc, &x_hi, &bhat, &rho64, &u64, &t64};
    const char* n64[] = {"x_acc", "x_hi", "bhat", "rho64", "u64", "t64"};
    for (int i = 0; i < 6; i++) CK(ws_field<double>(c, wsp + n64[i], units, f64[i]));
    if (own_b) {
      // sessions finish slots while others iterate: their sources and odd-site
      // solutions need fields of their own
      CK(ws_field<double>(c, wsp + "b_e", units, &b_e));
      CK(ws_field<double>(c, wsp + "b_o", units, &b_o));
      CK(ws_field<double>(c, wsp + "x_o", units, &x_o));
    }
    if (!kFP64) {
      // the FP32 reliable-update fields live in the FP64 temporaries u64 and t64:
      // an update (update32) and a re-reference (reref) never overlap
      const size_t n = 24 * (size_t)units;
      xf.v = reinterpret_cast<float*>(u64.v);
      uf.v = reinterpret_cast<float*>(u64.v) + n;
      tf.v = reinterpret_cast<float*>(t64.v);
      qf.v = reinterpret_cast<float*>(t64.v) + n;
      xf.n = uf.n = tf.n = qf.n = nullptr;
    }
    F<S>* fS[] = {&p, &u, &t, &q, &rho, &r};
    const char* nS[] = {"p", "u", "t", "q", "rho", "r"};
    for (int i = 0; i < 6; i++) CK(ws_field<S>(c, wsp + "S." + nS[i], units, fS[i]));
    // x_lo: tile-major over the BLAS tiling when it is FP32 (axpy_x_rho, accum_xhi, zero_xlo)
    xlo_n = xlo_units(tl_blas, units, !kFP64);
    CK(ws_field<SX>(c, wsp + "xlo", xlo_n, &xlo));
    part = (double*)ws_get(c, wsp + "partials", sizeof(double) * g.Vh * N, &e); CK(e);
    double* d = (double*)ws_get(c, wsp + "scal_d", sizeof(double) * 12 * N, &e); CK(e);
    int* ip = (int*)ws_get(c, wsp + "scal_i", sizeof(int) * 4 * N, &e); CK(e);
    umask_d = (int*)ws_get(c, wsp + "umask", sizeof(int) * N, &e); CK(e);
    sc.gamma = d; sc.gamma_prev = d + N; sc.alpha = d + 2 * N; sc.beta = d + 3 * N; sc.rho2 = d + 4 * N;
    sc.rho2_max = d + 5 * N; sc.stop2 = d + 6 * N; sc.qq = d + 7 * N; sc.rr = d + 8 * N; sc.tmp = d + 9 * N;
    sc.bhat2 = d + 10 * N;
    sc.upd2 = d + 11 * N;
    sc.active = ip; sc.flags = ip + N; sc.iters = ip + 2 * N; sc.since = ip + 3 * N;
    sc.stag_max = 128;
    CK(cudaMemsetAsync(d, 0, sizeof(double) * 12 * N, st));
    CK(cudaMemsetAsync(ip, 0, sizeof(int) * 4 * N, st));
    const size_t b64 = sizeof(double) * 24 * (size_t)units;
    CK(cudaMemsetAsync(x_acc.v, 0, b64, st));
    CK(cudaMemsetAsync(x_hi.v, 0, b64, st));
    CK(cudaMemsetAsync(xlo.v, 0, sizeof(SX) * 24 * (size_t)xlo_n, st));
    CK(cudaMemsetAsync(p.v, 0, sizeof(S) * 24 * (size_t)units, st));
    if (p.n) CK(cudaMemsetAsync(p.n, 0, sizeof(float) * (size_t)units, st));
    if (tune_request >= 0) {
      // the timing runs write t, q, r and the partial sums only; p is zeroed again after it
      if (int rc = tune(tune_request)) return rc;
      CK(cudaMemsetAsync(p.v, 0, sizeof(S) * 24 * (size_t)units, st));
      if (p.n) CK(cudaMemsetAsync(p.n, 0, sizeof(float) * (size_t)units, st));
    }
    if (profile) opS.prof = &prof;
    return MDWF_OK;
  }

  // Autotuner: time Mhat + Mhat^+ of the inner precision over the candidate hop
  // forms and block shapes on this solver's own fields, keep the fastest, and
  // remember it in the context for (L5, N, precision, candidate set).  HOP_AUTO
  // tries only forms with the same arithmetic (the CUDA-core direct hop with
  // 1..8 sites per block and, for fp16 storage, its prefetching form with 1..4),
  // so the choice never changes a result; HOP_TUNE_ALL
  // adds the staged and tensor-core hops, whose roundings differ.
  int tune(int which, int* variant_out = nullptr, int* nsb_out = nullptr, double* ms_out = nullptr) {
    mdwf_ctx* ctx = this->ctx;
    const int prec = kFP64 ? MDWF_PREC_DOUBLE : std::is_same<S, float>::value ? MDWF_PREC_SINGLE
                   : std::is_same<S, __half>::value ? MDWF_PREC_HALF : MDWF_PREC_BF16;
    const std::array<int, 4> key = {L5, N, prec, which == HOP_TUNE_ALL ? 1 : 0};
    auto it = ctx->tuned.find(key);
    if (it == ctx->tuned.end()) {
      std::vector<std::array<int, 2>> cand;
      for (int nsbc : {1, 2, 4, 8})
        if (nsbc * L5 <= 1024) cand.push_back({HOP_DIRECT, nsbc});
      // fp16 storage: the prefetching form of the paired hop, the same bits
      if (std::is_same<S, __half>::value)
        for (int nsbc : {1, 2, 4})
          if (nsbc * L5 <= 1024) cand.push_back({HOP_PAIR_PF, nsbc});
      if (which == HOP_TUNE_ALL && !kFP64) cand.push_back({HOP_STAGED, 0});
      if (which == HOP_TUNE_ALL && std::is_same<S, __half>::value) cand.push_back({HOP_MMA, 0});
      cudaStream_t st = op64.st;
      cudaEvent_t e0, e1;
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      const long long keep = launches;
      Prof* keep_prof = opS.prof;
      opS.prof = nullptr;
      std::array<int, 2> best = {HOP_DIRECT, 0};
      double best_ms = 1e300;
      int rc = MDWF_OK;
      for (const auto& cnd : cand) {
        choose_hop(opS, cfg, cnd[1], cnd[0], &stage);
        if (cnd[0] == HOP_MMA && !opS.mma) continue;
        if (cnd[0] == HOP_STAGED && opS.stage == nullptr) continue;
        if ((cnd[0] == HOP_DIRECT || cnd[0] == HOP_PAIR_PF) && opS.tl.nsb != cnd[1]) continue;
        float ms = 0.f;
        cudaError_t e = cudaSuccess;
        for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {
          if (rep == 1) e = cudaEventRecord(e0, st);
          if (e == cudaSuccess) e = opS.mhat(p, u, t, q, nullptr, nullptr);
          if (e == cudaSuccess) e = opS.mhat_dag(q, t, r, nullptr, nullptr);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { rc = fail(ctx, MDWF_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e)); break; }
        if (ms / 2.0 < best_ms) { best_ms = ms / 2.0; best = cnd; }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      launches = keep;
      opS.prof = keep_prof;
      if (rc) return rc;
      int herr = 0;
      CK(cudaMemcpyAsync(&herr, errw, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (herr) return fail(ctx, MDWF_ERR_TIMEOUT, "autotune: a bounded device wait ran out");
      it = ctx->tuned.emplace(key, std::make_pair(best, best_ms)).first;
    }
    choose_hop(opS, cfg, it->second.first[1], it->second.first[0], &stage);
    if (variant_out) *variant_out = it->second.first[0];
    if (nsb_out) *nsb_out = opS.tl.nsb;
    if (ms_out) *ms_out = it->second.second;
    return MDWF_OK;
  }

  template <typename SS>
  cudaError_t norms(F<SS> f, const int* mask, double* dst) {
    launches += 2;
    cudaError_t e = norm2_partials<SS>(f.v, f.n, tl_blas, ctx->g.Vh, L5, N, mask, part, op64.st);
    if (e != cudaSuccess) return e;
    return finalize(part, ctx->g.Vh, N, dst, op64.st);
  }

  // One CG iteration on all active slots.
  cudaError_t iteration() {
    const Geom& g = ctx->g;
    cudaStream_t st = op64.st;
    cudaError_t e;
    launches += 8;  // xpay_b, axpy, 3 finalize, 3 scalar kernels (+ 4 hops counted in FastOp::run)
    e = xpay_b<S>(r.v, r.n, p.v, p.n, u.v, u.n, sc.beta, opS.f, tl_blas, g.Vh, L5, N, sc.active, st);
    if (e != cudaSuccess) return e;
    e = sym ? opS.mhat_sym(p, u, t, q, sc.active, part) : opS.mhat(p, u, t, q, sc.active, part);
    if (e != cudaSuccess) return e;
    e = finalize(part, g.Vh, N, sc.qq, st);
    if (e != cudaSuccess) return e;
    k_alpha<<<1, 1024, 0, st>>>(sc, N);
    e = axpy_x_rho<SX, S>(xlo.v, p.v, p.n, rho.v, rho.n, q.v, q.n, sc.alpha, tl_blas, g.Vh, L5, N, sc.active, part, st);
    if (e != cudaSuccess) return e;
    e = finalize(part, g.Vh, N, sc.tmp, st);
    if (e != cudaSuccess) return e;
    k_after_rho<<<1, 1024, 0, st>>>(sc, N);
    // (u = B p is dead here: the symmetric form's scratch)
    e = sym ? opS.mhat_sym_dag(rho, u, t, r, sc.active, part) : opS.mhat_dag(rho, t, r, sc.active, part);
    if (e != cudaSuccess) return e;
    e = finalize(part, g.Vh, N, sc.rr, st);
    if (e != cudaSuccess) return e;
    k_beta<<<1, 1024, 0, st>>>(sc, N);
    return cudaGetLastError();
  }

  // r = Mhat^+ rho and |r|^2 for the slots in um.
  cudaError_t normal_residual(const int* um) {
    launches += 1;
    cudaError_t e = sym ? opS.mhat_sym_dag(rho, u, t, r, um, part) : opS.mhat_dag(rho, t, r, um, part);
    if (e != cudaSuccess) return e;
    return finalize(part, ctx->g.Vh, N, sc.rr, op64.st);
  }

  // Reliable update with FP32 arithmetic: rho = bhat - Mhat x_hi (FP64 difference).
  cudaError_t update32(const int* um) {
    const Geom& g = ctx->g;
    cudaStream_t st = op64.st;
    cudaError_t e;
    launches += 6;  // accum, convert, bop, resid_update, finalize, scalar kernel
    e = accum_xhi<SX>(x_hi.v, xlo.v, tl_blas, g.Vh, L5, N, um, st);
    if (e != cudaSuccess) return e;
    e = convert<double, float>(x_hi.v, nullptr, xf.v, nullptr, tl_blas, g.Vh, L5, N, um, st);
    if (e != cudaSuccess) return e;
    e = bop<float>(xf.v, nullptr, uf.v, nullptr, op32.f, tl_blas, g.Vh, L5, N, um, st);
    if (e != cudaSuccess) return e;
    e = sym ? op32.mhat_sym(xf, uf, tf, qf, um, nullptr) : op32.mhat(xf, uf, tf, qf, um, nullptr);
    if (e != cudaSuccess) return e;
    e = resid_update<S>(bhat.v, qf.v, rho.v, rho.n, tl_blas, g.Vh, L5, N, um, part, st);
    if (e != cudaSuccess) return e;
    e = finalize(part, g.Vh, N, sc.tmp, st);
    if (e != cudaSuccess) return e;
    e = normal_residual(um);
    if (e != cudaSuccess) return e;
    k_after_update<<<1, 1024, 0, st>>>(sc, N, um);
    return cudaGetLastError();
  }

  // FP64 re-reference: rho = bhat - Mhat x_hi in FP64, then bhat <- rho and
  // x_acc += x_hi, x_hi = 0.  With zero_x the operator is skipped (x_hi = 0).
  cudaError_t reref(const int* um, bool zero_x) {
    const Geom& g = ctx->g;
    cudaStream_t st = op64.st;
    cudaError_t e;
    F<double> none;
    if (zero_x) {
      launches += 1;
      e = convert<double, double>(bhat.v, nullptr, rho64.v, nullptr, tl_blas, g.Vh, L5, N, um, st);
      if (e != cudaSuccess) return e;
    } else {
      launches += 2;
      e = accum_xhi<SX>(x_hi.v, xlo.v, tl_blas, g.Vh, L5, N, um, st);
      if (e != cudaSuccess) return e;
      e = bop<double>(x_hi.v, nullptr, u64.v, nullptr, op64.f, tl_blas, g.Vh, L5, N, um, st);
      if (e != cudaSuccess) return e;
      e = op64.run(E_BAINV, 1, 0, u64, none, none, 0.0, 1.0, t64, um, nullptr);
      if (e != cudaSuccess) return e;
      // rho = bhat - Mhat x_hi  (symmetric form: bhat - Mhat_s x_hi)
      e = op64.run(sym ? E_SAME_AINV : E_A_SAME, 0, 0, t64, x_hi, bhat, -1.0, 0.25, rho64, um, nullptr);
      if (e != cudaSuccess) return e;
    }
    e = norms<double>(rho64, um, sc.tmp);
    if (e != cudaSuccess) return e;
    launches += 4;  // copy, accum, convert, scalar kernel
    e = convert<double, double>(rho64.v, nullptr, bhat.v, nullptr, tl_blas, g.Vh, L5, N, um, st);
    if (e != cudaSuccess) return e;
    e = accum_xhi<double>(x_acc.v, x_hi.v, tl_blas, g.Vh, L5, N, um, st);
    if (e != cudaSuccess) return e;
    e = convert<double, S>(rho64.v, nullptr, rho.v, rho.n, tl_blas, g.Vh, L5, N, um, st);
    if (e != cudaSuccess) return e;
    e = normal_residual(um);
    if (e != cudaSuccess) return e;
    k_after_reref<<<1, 1024, 0, st>>>(sc, N, um);
    return cudaGetLastError();
  }

  cudaError_t collect(bool after_graph) {
    if (!profiling) return cudaSuccess;
    cudaError_t e = prof.collect();
    if (e != cudaSuccess || !after_graph) return e;
    return prof.collect_graph();
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
      const long long c0 = launches;
      prof.gused = 0;
      prof.capturing = profiling;
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
      cudaError_t err = cudaSuccess;
      for (int i = 0; i < k && err == cudaSuccess; i++) err = iteration();
      cudaError_t e2 = cudaStreamEndCapture(st, &gr);
      prof.capturing = false;
      graph_launches = launches - c0;
      launches = c0;
      CK(err);
      CK(e2);
      cudaError_t e3 = cudaGraphInstantiate(&graph, gr, 0);
      cudaGraphDestroy(gr);
      CK(e3);
      graph_iters = k;
    }
    CK(cudaGraphLaunch(graph, st));
    launches += graph_launches;
    return MDWF_OK;
  }
};

// The symmetric form stops on |A^-1 (bhat - Mhat x)|; since |A| <= alpha + |beta|
// (A = alpha + beta P with |P| <= 1), stopping at tol / (alpha + |beta|) in that
// norm keeps the Schur residual, and so the full residual, below tol.
double sym_stop_factor(const Action& act, const mdwf_solver_opts& o) {
  if (o.schur != 1) return 1.0;
  const double d = 4.0 - act.M5;
  const double na = std::fabs(act.b5 * d + 1.0) + std::fabs(act.c5 * d - 1.0);
  return 1.0 / (na * na);
}

int check_cfg(mdwf_ctx* ctx, int cfg_id, Cfg** out) {
  if (!ctx) return MDWF_ERR_ARG;
  auto it = ctx->cfgs.find(cfg_id);
  if (it == ctx->cfgs.end() || !it->second.has_gauge) return fail(ctx, MDWF_ERR_STATE, "no gauge field for cfg_id");
  if (!it->second.act.set) return fail(ctx, MDWF_ERR_STATE, "no action set for cfg_id");
  *out = &it->second;
  return MDWF_OK;
}

cudaStream_t pick_stream(mdwf_ctx* ctx, void* s) { return s ? (cudaStream_t)s : ctx->stream; }

// The two-row FP32 links of cfg for 12-real reconstruction, built on first use.
int ensure_u12(mdwf_ctx* ctx, Cfg* cfg) {
  if (cfg->U12) return MDWF_OK;
  const long nlinks = ctx->g.V * 4;
  CK(cudaMalloc(&cfg->U12, sizeof(float) * 12 * (size_t)nlinks));
  CK(build_link12(cfg->U32, cfg->U12, nlinks, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MDWF_OK;
}

// Device time of the phases of a solve (opts.profile): an event pair per phase
// interval, read after the synchronisation that ends it.
struct Phases {
  bool on = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double ms[5] = {0, 0, 0, 0, 0};
  cudaError_t begin(bool enable, cudaStream_t st) {
    on = enable;
    if (!on) return cudaSuccess;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    return e;
  }
  // close the current interval as phase k and open the next one
  cudaError_t mark(int k, cudaStream_t st) {
    if (!on) return cudaSuccess;
    cudaError_t e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    ms[k] += t;
    std::swap(e0, e1);
    return e;
  }
  ~Phases() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};
enum { PH_PREP = 0, PH_CG = 1, PH_UPD32 = 2, PH_REREF = 3, PH_FINAL = 4 };

// Solve on device API-layout buffers.  After the CG loop every system's x is
// reconstructed and certified by its FP64 full-lattice residual |b - D x| / |b|;
// a system whose certificate misses tol (while it has iterations left) resumes
// from its x with a 16 times tighter Schur stopping norm, up to opts.max_restarts
// times (the restart of reading 7).
template <typename S>
int solve_batch_impl(mdwf_ctx* ctx, Cfg* cfg, int n, const double* const* srcs, const std::vector<double>& masses,
                     double* const* xs, double tol, const mdwf_solver_opts& o, mdwf_solve_stats* stats,
                     cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  Phases ph;
  CK(ph.begin(o.profile != 0, st));
  if (o.link_recon == 12) { if (int r12 = ensure_u12(ctx, cfg)) return r12; }
  BatchSolver<S> sv;
  int rc = sv.init(ctx, cfg, masses, o.nsb, o.profile != 0, o, st);
  if (rc != MDWF_OK) return rc;
  const Geom& g = ctx->g;
  const int N = n, L5 = cfg->act.L5;
  const size_t field_bytes = sizeof(double) * 24 * (size_t)g.Vh * L5 * N;
  F<double> none;
  double* tmp = sv.sc.tmp;
  std::vector<double> bb(N), bo(N), stop2(N);
  std::vector<int> act(N, 1), um(N), flags(N), iters(N), nupd(N, 1), done(N, 0), n32(N, 0), n64(N, 1);
  std::vector<int> cap(N, o.max_iter);   // iteration limit of each system (a restart gets a budget)
  int restarts = 0;

  // Schur right-hand side bhat_e = b_e + 1/2 H_eo B A^-1 b_o in bhat (FP64); the
  // sources are packed into rho64 (b_e) and x_hi (b_o), which are free then.
  auto schur_source = [&](bool norms) -> int {
    sv.launches += 2 * N;
    sv.b_e = sv.rho64;
    sv.b_o = sv.x_hi;
    for (int i = 0; i < N; i++) {
      CK(pack_rhs<double>(srcs[i], sv.b_e.v, nullptr, g, L5, N, 0, i, st));
      CK(pack_rhs<double>(srcs[i], sv.b_o.v, nullptr, g, L5, N, 1, i, st));
    }
    if (norms) {
      CK(sv.norms(sv.b_e, nullptr, tmp));
      CK(cudaMemcpyAsync(bb.data(), tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
      CK(sv.norms(sv.b_o, nullptr, tmp));
      CK(cudaMemcpyAsync(bo.data(), tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    Op<double, double> loc;
    loc.g = g; loc.L5 = L5; loc.N = N; loc.anti = cfg->anti; loc.U = cfg->U64; loc.st = st;
    loc.tl = tiling_for<double>(g, L5, N, sv.op64.tl.nsb, true);
    loc.launches = &sv.launches;
    Tables tab;
    tab.build(cfg->act, masses);
    DevTables<double> M;
    CK(upload_tables_ws<double>(ctx, sv.wsp + "tables", tab, &M, st));
    CK(loc.run(false, 1, 0, sv.b_o, none, M[MK_BAinv], none, nullptr, 0.0, sv.t64, nullptr, nullptr));
    CK(sv.op64.run(E_RAW, 0, 0, sv.t64, none, sv.b_e, 0.0, 0.5, sv.bhat, nullptr, nullptr));
    if (sv.sym) {   // symmetric form: the right-hand side A^-1 bhat
      CK(sv.op64.run(E_AINV_SAME, 0, 0, none, sv.bhat, none, 0.0, 0.0, sv.t64, nullptr, nullptr));
      CK((convert<double, double>(sv.t64.v, nullptr, sv.bhat.v, nullptr, sv.tl_blas, g.Vh, L5, N, nullptr, st)));
    }
    // x_hi held b_o
    CK(cudaMemsetAsync(sv.x_hi.v, 0, field_bytes, st));
    return MDWF_OK;
  };

  if ((rc = schur_source(true))) return rc;
  for (int i = 0; i < N; i++) {
    double b2 = bb[i] + bo[i];
    if (!std::isfinite(b2)) return fail(ctx, MDWF_ERR_NONFINITE, "source has NaN/Inf");
    stop2[i] = 0.25 * tol * tol * b2 * sym_stop_factor(cfg->act, o) * o.stop_scale_test * o.stop_scale_test;
    if (b2 == 0.0) act[i] = 0;
  }
  CK(cudaMemcpyAsync(sv.sc.stop2, stop2.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st));
  sv.sc.delta2 = BatchSolver<S>::kFP64 ? 0.0 : o.delta * o.delta;
  sv.sc.tau2 = BatchSolver<S>::kFP64 ? 0.0 : 1e-10;
  // initial residual (x = 0)
  for (int i = 0; i < N; i++) um[i] = act[i];
  CK(cudaMemcpyAsync(sv.sc.active, act.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(sv.umask_d, um.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  CK(sv.reref(sv.umask_d, true));
  CK(ph.mark(PH_PREP, st));
  for (int i = 0; i < N; i++) if (!act[i]) done[i] = 1;
  const int chunk = o.chunk > 0 ? o.chunk : 16;
  auto read_flags = [&]() -> int {
    int herr = 0;
    CK(cudaMemcpyAsync(flags.data(), sv.sc.flags, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(iters.data(), sv.sc.iters, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&herr, sv.errw, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr) {
      cudaMemsetAsync(sv.errw, 0, sizeof(int), st);
      cudaStreamSynchronize(st);
      return fail(ctx, MDWF_ERR_TIMEOUT, "a bounded device wait ran out (staged neighbour copies did not arrive)");
    }
    return MDWF_OK;
  };

  // CG chunks with reliable updates until every system is done
  auto iterate = [&]() -> int {
    int rc2;
    for (;;) {
      bool all = true;
      for (int i = 0; i < N; i++) all = all && done[i];
      if (all) break;
      rc2 = sv.run_chunk(chunk, o.use_graph != 0);
      if (rc2 != MDWF_OK) return rc2;
      if ((rc2 = read_flags())) return rc2;
      CK(ph.mark(PH_CG, st));
      CK(sv.collect(o.use_graph != 0));
      // reliable updates: FP32 arithmetic (mixed) or FP64 (FP64 solver)
      bool any = false;
      for (int i = 0; i < N; i++) {
        um[i] = (!done[i] && (flags[i] & (FLAG_INNER_DONE | FLAG_UPDATE))) ? 1 : 0;
        any = any || um[i];
      }
      if (any) {
        CK(cudaMemcpyAsync(sv.umask_d, um.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
        if (BatchSolver<S>::kFP64) CK(sv.reref(sv.umask_d, false));
        else CK(sv.update32(sv.umask_d));
        if ((rc2 = read_flags())) return rc2;
        CK(ph.mark(BatchSolver<S>::kFP64 ? PH_REREF : PH_UPD32, st));
        CK(sv.collect(false));
        for (int i = 0; i < N; i++) if (um[i]) { nupd[i]++; (BatchSolver<S>::kFP64 ? n64 : n32)[i]++; }
      }
      // FP64 re-references requested by the FP32 updates
      any = false;
      for (int i = 0; i < N; i++) {
        um[i] = (!done[i] && (flags[i] & FLAG_REREF)) ? 1 : 0;
        any = any || um[i];
      }
      if (any) {
        CK(cudaMemcpyAsync(sv.umask_d, um.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
        CK(sv.reref(sv.umask_d, false));
        if ((rc2 = read_flags())) return rc2;
        CK(ph.mark(PH_REREF, st));
        CK(sv.collect(false));
        for (int i = 0; i < N; i++) if (um[i]) { nupd[i]++; n64[i]++; }
      }
      bool stop_any = false;
      for (int i = 0; i < N; i++) {
        if (flags[i] & FLAG_DONE) done[i] = 1;
        if (!done[i] && iters[i] >= cap[i]) { done[i] = 1; stop_any = true; }
      }
      if (stop_any) {
        std::vector<int> a(N);
        CK(cudaMemcpyAsync(a.data(), sv.sc.active, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i < N; i++) if (done[i]) a[i] = 0;
        CK(cudaMemcpyAsync(sv.sc.active, a.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
      }
      CK(ph.mark(PH_CG, st));   // (host bookkeeping between chunks)
    }
    return MDWF_OK;
  };

  // x_e = x_acc (+ x_hi + x_lo), reconstruction, FP64 certificate on both
  // parities, unpacking into xs.  Odd sites: y = b_o + 1/2 H_oe B x_e (one FP64
  // hop), x_o = A^-1 y, and the odd residual b_o - A x_o + 1/2 H_oe B x_e = y - A x_o
  // reuses y.  Even sites: b_e - A x_e + 1/2 H_eo B x_o (the second FP64 hop).
  std::vector<double> re(N), ro(N);
  auto finish = [&]() -> int {
    sv.launches += 2 + 2 * N;
    CK(accum_xhi<typename BatchSolver<S>::SX>(sv.x_hi.v, sv.xlo.v, sv.tl_blas, g.Vh, L5, N, nullptr, st));
    CK(accum_xhi<double>(sv.x_acc.v, sv.x_hi.v, sv.tl_blas, g.Vh, L5, N, nullptr, st));
    // sources again, in fields now free (bhat, x_hi)
    sv.b_e = sv.bhat;
    sv.b_o = sv.x_hi;
    for (int i = 0; i < N; i++) {
      CK(pack_rhs<double>(srcs[i], sv.b_e.v, nullptr, g, L5, N, 0, i, st));
      CK(pack_rhs<double>(srcs[i], sv.b_o.v, nullptr, g, L5, N, 1, i, st));
    }
    sv.launches += 2;
    CK(bop<double>(sv.x_acc.v, nullptr, sv.u64.v, nullptr, sv.op64.f, sv.tl_blas, g.Vh, L5, N, nullptr, st));
    CK(sv.op64.run(E_RAW, 1, 0, sv.u64, none, sv.b_o, 0.0, 0.5, sv.t64, nullptr, nullptr));
    // y = t64 now holds b_o: the odd-site solution goes into x_hi (b_o's field)
    F<double> x_o = sv.x_hi;
    CK(sv.op64.run(E_AINV_SAME, 1, 0, none, sv.t64, none, 0.0, 0.0, x_o, nullptr, nullptr));
    CK(sv.op64.run(E_A_SAME, 1, 0, none, x_o, sv.t64, -1.0, 0.0, sv.rho64, nullptr, nullptr));
    CK(sv.norms(sv.rho64, nullptr, tmp));
    CK(cudaMemcpyAsync(ro.data(), tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    CK(bop<double>(x_o.v, nullptr, sv.u64.v, nullptr, sv.op64.f, sv.tl_blas, g.Vh, L5, N, nullptr, st));
    CK(sv.op64.run(E_A_SAME, 0, 0, sv.u64, sv.x_acc, sv.b_e, -1.0, 0.5, sv.rho64, nullptr, nullptr));
    CK(sv.norms(sv.rho64, nullptr, tmp));
    CK(cudaMemcpyAsync(re.data(), tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(iters.data(), sv.sc.iters, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
    sv.launches += 2 * N;
    for (int i = 0; i < N; i++) {
      CK(unpack_rhs<double>(sv.x_acc.v, nullptr, xs[i], g, L5, N, 0, i, st));
      CK(unpack_rhs<double>(x_o.v, nullptr, xs[i], g, L5, N, 1, i, st));
    }
    CK(cudaStreamSynchronize(st));
    CK(ph.mark(PH_FINAL, st));
    return MDWF_OK;
  };
  auto rel_of = [&](int i) {
    const double b2 = bb[i] + bo[i];
    return b2 > 0 ? std::sqrt((re[i] + ro[i]) / b2) : 0.0;
  };

  for (;;) {
    if ((rc = iterate())) return rc;
    if ((rc = finish())) return rc;
    bool any = false;
    for (int i = 0; i < N; i++) {
      um[i] = (act[i] && rel_of(i) > tol && iters[i] < o.max_iter) ? 1 : 0;
      any = any || um[i];
    }
    if (!any || restarts >= o.max_restarts) break;
    // resume the systems that missed tol from their x: bhat is rebuilt from the
    // sources, x_acc moves into x_hi for those systems, and an FP64 re-reference
    // forms bhat - Mhat x_hi with a 16 times tighter stopping norm
    restarts++;
    if ((rc = schur_source(false))) return rc;
    CK(cudaMemcpyAsync(sv.umask_d, um.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
    sv.launches += 1;
    CK(accum_xhi<double>(sv.x_hi.v, sv.x_acc.v, sv.tl_blas, g.Vh, L5, N, sv.umask_d, st));
    // each resumed system gets a budget of a quarter of the iterations it has
    // used (at least 64): a tighter norm below what its FP64 residual can
    // resolve then ends in NOT_CONVERGED with its certificate, not at max_iter
    for (int i = 0; i < N; i++)
      if (um[i]) {
        stop2[i] /= 256.0;
        done[i] = 0;
        cap[i] = (int)std::min<long long>(o.max_iter, (long long)iters[i] + std::max(64, iters[i] / 4));
      }
    CK(cudaMemcpyAsync(sv.sc.stop2, stop2.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st));
    CK(sv.reref(sv.umask_d, false));
    for (int i = 0; i < N; i++) if (um[i]) { nupd[i]++; n64[i]++; }
    CK(ph.mark(PH_REREF, st));
  }
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int status = MDWF_OK;
  for (int i = 0; i < N; i++) {
    const double rel = rel_of(i);
    bool conv = rel <= tol;
    if (!conv) status = MDWF_ERR_NOT_CONVERGED;
    if (stats) {
      stats[i].iters = iters[i];
      stats[i].reliable_updates = nupd[i];
      stats[i].converged = conv ? 1 : 0;
      stats[i].rel_true_resid = rel;
      stats[i].time_s = secs;
      stats[i].hop_launches = (int)sv.prof.n;
      stats[i].hop_ms = sv.prof.ms;
      stats[i].kernel_launches = sv.launches;
      stats[i].hop_units = (long long)g.Vh * L5 * N;
      for (int k = 0; k < 5; k++) stats[i].phase_ms[k] = ph.ms[k];
      stats[i].fp32_updates = n32[i];
      stats[i].fp64_rerefs = n64[i];
      stats[i].restarts = restarts;
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

// ---------------------------------------------------------------------------
// Solver sessions: continuous batching
// ---------------------------------------------------------------------------
// A session owns the state of a batch of `slots` right-hand sides for one gauge
// configuration.  Requests enter free slots between CG chunks (submit), every
// chunk advances all occupied slots at once (launch), and poll() performs the
// reliable updates and hands back the solutions of converged slots, freeing
// them for new requests.  A slot always enters at a chunk boundary and every
// per-slot operation is independent of the other slots, so a request follows
// the same arithmetic alone as in any mix.

template <typename S>
struct SessionImpl : SessionBase {
  mdwf_ctx* ctx;
  Cfg* cfg;
  BatchSolver<S> sv;
  int N = 0;
  double tol = 1e-10;
  mdwf_solver_opts o;
  cudaStream_t st = nullptr;
  std::vector<double> masses;
  std::vector<int> used, nupd;
  std::vector<long long> tags;
  std::vector<double*> outs;
  std::vector<double> b2;
  std::vector<std::chrono::steady_clock::time_point> t0;
  int* fmask = nullptr;   // device mask of the slots being finalised

  int create(mdwf_ctx* c, Cfg* cf, int slots, const mdwf_solver_opts& opts, double tl, cudaStream_t s,
             const std::string& prefix) {
    mdwf_ctx* ctx = c;
    this->ctx = c;
    cfg = cf;
    N = slots;
    o = opts;
    tol = tl;
    st = s;
    masses.assign(N, cf->act.mf);
    used.assign(N, 0);
    nupd.assign(N, 0);
    tags.assign(N, 0);
    outs.assign(N, nullptr);
    b2.assign(N, 0.0);
    t0.resize(N);
    sv.wsp = prefix;
    sv.own_b = true;
    if (o.link_recon == 12) { if (int r12 = ensure_u12(ctx, cf)) return r12; }
    int rc = sv.init(c, cf, masses, o.nsb, o.profile != 0, o, s);
    if (rc) return rc;
    sv.sc.delta2 = BatchSolver<S>::kFP64 ? 0.0 : o.delta * o.delta;
    sv.sc.tau2 = BatchSolver<S>::kFP64 ? 0.0 : 1e-10;
    cudaError_t e = cudaSuccess;
    fmask = (int*)ws_get(c, prefix + "fmask", sizeof(int) * N, &e);
    CK(e);
    CK(cudaStreamSynchronize(s));
    return MDWF_OK;
  }

  int occupied() const override {
    int k = 0;
    for (int u : used) k += u;
    return k;
  }

  int set_mask(int* dev, const std::vector<int>& h) {
    CK(cudaMemcpyAsync(dev, h.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
    return MDWF_OK;
  }

  int submit(const double* src, double mass, double* x, long long tag, int* slot) override {
    int r = -1;
    for (int i = 0; i < N; i++)
      if (!used[i]) { r = i; break; }
    if (r < 0) return fail(ctx, MDWF_ERR_FULL, "session has no free slot");
    const Geom& g = ctx->g;
    const int L5 = cfg->act.L5;
    masses[r] = mass;
    const float m32 = (float)mass;
    CK(cudaMemcpyAsync(sv.mass64 + r, &mass, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(sv.mass32 + r, &m32, sizeof(float), cudaMemcpyHostToDevice, st));
    std::vector<int> um(N, 0);
    um[r] = 1;
    if (int rc = set_mask(sv.umask_d, um)) return rc;
    // fresh per-slot state
    const int zi = 0;
    const double zd = 0.0;
    int* ia[] = {sv.sc.active, sv.sc.flags, sv.sc.iters, sv.sc.since};
    for (int* a : ia) CK(cudaMemcpyAsync(a + r, &zi, sizeof(int), cudaMemcpyHostToDevice, st));
    double* da[] = {sv.sc.gamma, sv.sc.gamma_prev, sv.sc.alpha, sv.sc.beta, sv.sc.rho2, sv.sc.rho2_max, sv.sc.qq,
                    sv.sc.rr, sv.sc.tmp, sv.sc.bhat2, sv.sc.upd2};
    for (double* a : da)
      CK(cudaMemcpyAsync(a + r, &zd, sizeof(double), cudaMemcpyHostToDevice, st));
    const int* m = sv.umask_d;
    CK(zero_masked<double>(sv.x_acc.v, nullptr, sv.tl_blas, g.Vh, L5, N, m, st));
    CK(zero_masked<double>(sv.x_hi.v, nullptr, sv.tl_blas, g.Vh, L5, N, m, st));
    CK(zero_xlo<typename BatchSolver<S>::SX>(sv.xlo.v, sv.tl_blas, g.Vh, L5, N, m, st));
    CK(zero_masked<S>(sv.p.v, sv.p.n, sv.tl_blas, g.Vh, L5, N, m, st));
    CK(pack_rhs<double>(src, sv.b_e.v, nullptr, g, L5, N, 0, r, st));
    CK(pack_rhs<double>(src, sv.b_o.v, nullptr, g, L5, N, 1, r, st));
    std::vector<double> be(N), bo(N);
    CK(sv.norms(sv.b_e, m, sv.sc.tmp));
    CK(cudaMemcpyAsync(be.data(), sv.sc.tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    CK(sv.norms(sv.b_o, m, sv.sc.tmp));
    CK(cudaMemcpyAsync(bo.data(), sv.sc.tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    b2[r] = be[r] + bo[r];
    if (!std::isfinite(b2[r])) return fail(ctx, MDWF_ERR_NONFINITE, "source has NaN/Inf");
    const double stop2 = 0.25 * tol * tol * b2[r] * sym_stop_factor(cfg->act, o);
    CK(cudaMemcpyAsync(sv.sc.stop2 + r, &stop2, sizeof(double), cudaMemcpyHostToDevice, st));
    // bhat_e = b_e + 1/2 H_eo B A^-1 b_o on this slot
    {
      F<double> none;
      Op<double, double> loc;
      loc.g = g; loc.L5 = L5; loc.N = N; loc.anti = cfg->anti; loc.U = cfg->U64; loc.st = st;
      loc.tl = tiling_for<double>(g, L5, N, sv.op64.tl.nsb, true);
      Tables tab;
      tab.build(cfg->act, masses);
      DevTables<double> M;
      CK(upload_tables_ws<double>(ctx, sv.wsp + "tables", tab, &M, st));
      CK(loc.run(false, 1, 0, sv.b_o, none, M[MK_BAinv], none, nullptr, 0.0, sv.t64, m, nullptr));
      CK(sv.op64.run(E_RAW, 0, 0, sv.t64, none, sv.b_e, 0.0, 0.5, sv.bhat, m, nullptr));
      if (sv.sym) {
        CK(sv.op64.run(E_AINV_SAME, 0, 0, none, sv.bhat, none, 0.0, 0.0, sv.t64, m, nullptr));
        CK((convert<double, double>(sv.t64.v, nullptr, sv.bhat.v, nullptr, sv.tl_blas, g.Vh, L5, N, m, st)));
      }
    }
    const int one = 1;
    CK(cudaMemcpyAsync(sv.sc.active + r, &one, sizeof(int), cudaMemcpyHostToDevice, st));
    if (b2[r] > 0.0) {
      CK(sv.reref(m, true));
    } else {
      const int done = FLAG_DONE;
      CK(cudaMemcpyAsync(sv.sc.flags + r, &done, sizeof(int), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(sv.sc.active + r, &zi, sizeof(int), cudaMemcpyHostToDevice, st));
    }
    CK(cudaStreamSynchronize(st));
    used[r] = 1;
    nupd[r] = 1;
    tags[r] = tag;
    outs[r] = x;
    t0[r] = std::chrono::steady_clock::now();
    if (slot) *slot = r;
    return MDWF_OK;
  }

  int launch(int iters) override {
    if (occupied() == 0) return MDWF_OK;
    return sv.run_chunk(iters > 0 ? iters : (o.chunk > 0 ? o.chunk : 16), o.use_graph != 0);
  }

  int poll(int max_done, long long* out_tags, mdwf_solve_stats* stats, int* n_done) override {
    *n_done = 0;
    if (occupied() == 0) return MDWF_OK;
    const Geom& g = ctx->g;
    const int L5 = cfg->act.L5;
    std::vector<int> flags(N), iters(N), um(N);
    auto read = [&]() -> int {
      int herr = 0;
      CK(cudaMemcpyAsync(flags.data(), sv.sc.flags, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(iters.data(), sv.sc.iters, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(&herr, sv.errw, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (herr) return fail(ctx, MDWF_ERR_TIMEOUT, "a bounded device wait ran out");
      return MDWF_OK;
    };
    if (int rc = read()) return rc;
    CK(sv.collect(o.use_graph != 0));
    bool any = false;
    for (int i = 0; i < N; i++) {
      um[i] = (used[i] && !(flags[i] & FLAG_DONE) && (flags[i] & (FLAG_INNER_DONE | FLAG_UPDATE))) ? 1 : 0;
      any = any || um[i];
    }
    if (any) {
      if (int rc = set_mask(sv.umask_d, um)) return rc;
      if (BatchSolver<S>::kFP64) CK(sv.reref(sv.umask_d, false));
      else CK(sv.update32(sv.umask_d));
      if (int rc = read()) return rc;
      CK(sv.collect(false));
      for (int i = 0; i < N; i++) if (um[i]) nupd[i]++;
    }
    any = false;
    for (int i = 0; i < N; i++) {
      um[i] = (used[i] && !(flags[i] & FLAG_DONE) && (flags[i] & FLAG_REREF)) ? 1 : 0;
      any = any || um[i];
    }
    if (any) {
      if (int rc = set_mask(sv.umask_d, um)) return rc;
      CK(sv.reref(sv.umask_d, false));
      if (int rc = read()) return rc;
      CK(sv.collect(false));
      for (int i = 0; i < N; i++) if (um[i]) nupd[i]++;
    }
    // slots that finished (converged or out of iterations), up to max_done
    std::vector<int> fin(N, 0);
    int nf = 0;
    for (int i = 0; i < N && nf < max_done; i++)
      if (used[i] && ((flags[i] & FLAG_DONE) || iters[i] >= o.max_iter)) { fin[i] = 1; nf++; }
    if (nf == 0) return MDWF_OK;
    if (int rc = set_mask(fmask, fin)) return rc;
    const int zi = 0;
    for (int i = 0; i < N; i++)
      if (fin[i]) CK(cudaMemcpyAsync(sv.sc.active + i, &zi, sizeof(int), cudaMemcpyHostToDevice, st));
    F<double> none;
    CK(accum_xhi<typename BatchSolver<S>::SX>(sv.x_hi.v, sv.xlo.v, sv.tl_blas, g.Vh, L5, N, fmask, st));
    CK(accum_xhi<double>(sv.x_acc.v, sv.x_hi.v, sv.tl_blas, g.Vh, L5, N, fmask, st));
    CK(bop<double>(sv.x_acc.v, nullptr, sv.u64.v, nullptr, sv.op64.f, sv.tl_blas, g.Vh, L5, N, fmask, st));
    CK(sv.op64.run(E_AINV_SAME, 1, 0, sv.u64, sv.b_o, none, 0.0, 0.5, sv.x_o, fmask, nullptr));
    CK(bop<double>(sv.x_o.v, nullptr, sv.t64.v, nullptr, sv.op64.f, sv.tl_blas, g.Vh, L5, N, fmask, st));
    CK(sv.op64.run(E_A_SAME, 0, 0, sv.t64, sv.x_acc, sv.b_e, -1.0, 0.5, sv.rho64, fmask, nullptr));
    std::vector<double> re(N), ro(N);
    CK(sv.norms(sv.rho64, fmask, sv.sc.tmp));
    CK(cudaMemcpyAsync(re.data(), sv.sc.tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    CK(sv.op64.run(E_A_SAME, 1, 0, sv.u64, sv.x_o, sv.b_o, -1.0, 0.5, sv.rho64, fmask, nullptr));
    CK(sv.norms(sv.rho64, fmask, sv.sc.tmp));
    CK(cudaMemcpyAsync(ro.data(), sv.sc.tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    for (int i = 0; i < N; i++) {
      if (!fin[i]) continue;
      CK(unpack_rhs<double>(sv.x_acc.v, nullptr, outs[i], g, L5, N, 0, i, st));
      CK(unpack_rhs<double>(sv.x_o.v, nullptr, outs[i], g, L5, N, 1, i, st));
    }
    CK(cudaStreamSynchronize(st));
    auto now = std::chrono::steady_clock::now();
    int k = 0;
    for (int i = 0; i < N; i++) {
      if (!fin[i]) continue;
      const double rel = b2[i] > 0 ? std::sqrt((re[i] + ro[i]) / b2[i]) : 0.0;
      if (out_tags) out_tags[k] = tags[i];
      if (stats) {
        std::memset(&stats[k], 0, sizeof(stats[k]));
        stats[k].iters = iters[i];
        stats[k].reliable_updates = nupd[i];
        stats[k].converged = rel <= tol ? 1 : 0;
        stats[k].rel_true_resid = rel;
        stats[k].time_s = std::chrono::duration<double>(now - t0[i]).count();
        stats[k].hop_units = (long long)g.Vh * L5 * N;
      }
      used[i] = 0;
      const int zf = 0;
      CK(cudaMemcpyAsync(sv.sc.flags + i, &zf, sizeof(int), cudaMemcpyHostToDevice, st));
      k++;
    }
    CK(cudaStreamSynchronize(st));
    *n_done = k;
    return MDWF_OK;
  }
};

void ws_release_prefix(mdwf_ctx* ctx, const std::string& prefix) {
  for (auto it = ctx->ws.begin(); it != ctx->ws.end();) {
    if (it->first.compare(0, prefix.size(), prefix) == 0) {
      if (it->second.first) cudaFree(it->second.first);
      it = ctx->ws.erase(it);
    } else {
      ++it;
    }
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
  CK(upload_tables_ws<double>(ctx, "apply.tables", tab, &M, st));
  long units = g.Vh * L5;
  // fields of the context's workspace: no allocation (and no device-wide
  // synchronisation of a free) once they exist
  struct WF {
    F<double> w;
    F<double> f() const { return w; }
  } ie, io, oe, oo, te, to;
  const char* names[] = {"apply.ie", "apply.io", "apply.oe", "apply.oo", "apply.te", "apply.to"};
  WF* fs[] = {&ie, &io, &oe, &oo, &te, &to};
  for (int i = 0; i < 6; i++) CK(ws_field<double>(ctx, names[i], units, &fs[i]->w));
  CK(pack_rhs<double>(in_dev, ie.w.v, nullptr, g, L5, 1, 0, 0, st));
  CK(pack_rhs<double>(in_dev, io.w.v, nullptr, g, L5, 1, 1, 0, st));
  CK(cudaMemsetAsync(oe.w.v, 0, sizeof(double) * 24 * (size_t)units, st));
  CK(cudaMemsetAsync(oo.w.v, 0, sizeof(double) * 24 * (size_t)units, st));
  F<double> none;
  cudaError_t me = cudaSuccess;
  double* mass = (double*)ws_get(ctx, "apply.mass", sizeof(double), &me);
  CK(me);
  CK(cudaMemcpyAsync(mass, &cfg->act.mf, sizeof(double), cudaMemcpyHostToDevice, st));
  FastOp<double, double> fo;
  fo.g = g; fo.L5 = L5; fo.N = 1; fo.anti = cfg->anti; fo.U = cfg->U64; fo.st = st;
  fo.f = make_fifth<double>(cfg->act, mass);
  choose_hop(fo, cfg, 0, HOP_DIRECT, nullptr);
  Tiling tb = make_tiling(g.Vh, L5, 1, 2, 512);
  if (kind == 0) {
    int par = arg1, dag = arg2;
    if (par == 0 || par == -1) CK(fo.run(E_RAW, 0, dag, io.f(), none, none, 0.0, 1.0, oe.f(), nullptr, nullptr));
    if (par == 1 || par == -1) CK(fo.run(E_RAW, 1, dag, ie.f(), none, none, 0.0, 1.0, oo.f(), nullptr, nullptr));
  } else if (kind == 1) {
    if (!arg1) {  // D x = A x - 1/2 H B x
      CK(bop<double>(ie.f().v, nullptr, te.f().v, nullptr, fo.f, tb, g.Vh, L5, 1, nullptr, st));
      CK(bop<double>(io.f().v, nullptr, to.f().v, nullptr, fo.f, tb, g.Vh, L5, 1, nullptr, st));
      CK(fo.run(E_A_SAME, 0, 0, to.f(), ie.f(), none, 1.0, -0.5, oe.f(), nullptr, nullptr));
      CK(fo.run(E_A_SAME, 1, 0, te.f(), io.f(), none, 1.0, -0.5, oo.f(), nullptr, nullptr));
    } else {      // D^+ x = A^+ x - 1/2 B^+ H^+ x
      CK(fo.run(E_AD_SAME_BD, 0, 1, io.f(), ie.f(), none, 1.0, -0.5, oe.f(), nullptr, nullptr));
      CK(fo.run(E_AD_SAME_BD, 1, 1, ie.f(), io.f(), none, 1.0, -0.5, oo.f(), nullptr, nullptr));
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
    CK(upload_tables_ws<double>(ctx, "apply.stables", sc, &G, st));
    CK(op.run(true, 0, 0, io.f(), ie.f(), G[0], none, nullptr, 0.5 * cfg->act.c5, oe.f(), nullptr, nullptr));
    CK(op.run(true, 1, 0, ie.f(), io.f(), G[0], none, nullptr, 0.5 * cfg->act.c5, oo.f(), nullptr, nullptr));
  }
  CK(unpack_rhs<double>(oe.w.v, nullptr, out_dev, g, L5, 1, 0, 0, st));
  CK(unpack_rhs<double>(oo.w.v, nullptr, out_dev, g, L5, 1, 1, 0, st));
  CK(cudaStreamSynchronize(st));
  return MDWF_OK;
}

// Time-split domain decomposition, FP64, one RHS: the operator of a local
// sub-domain whose time neighbours across both edges come from faces.
// kind 0: out = H in (dagger 0) or H^+ in; kind 1: out = D in or D^+ in.  With
// pack set, the faces of the field the hop reads (in; B in for D) are written to
// face_prev / face_next instead.  Faces: Lx Ly Lz * L5 * 12 doubles each.
int dd_impl(mdwf_ctx* ctx, Cfg* cfg, bool pack, int kind, int dagger, const double* in_dev, double* out_dev,
            double* face_prev, double* face_next, const double* halo_next, const double* halo_prev,
            double sign_next, double sign_prev, cudaStream_t st) {
  const Geom& g = ctx->g;
  const int L5 = cfg->act.L5;
  if (g.L[3] < 2 || (g.L[3] & 1)) return fail(ctx, MDWF_ERR_ARG, "dd: the local time extent must be even");
  const long units = g.Vh * L5;
  F<double> ie, io, te, to, oe, oo;
  CK(ws_field<double>(ctx, "dd.ie", units, &ie));
  CK(ws_field<double>(ctx, "dd.io", units, &io));
  CK(ws_field<double>(ctx, "dd.te", units, &te));
  CK(ws_field<double>(ctx, "dd.to", units, &to));
  CK(pack_rhs<double>(in_dev, ie.v, nullptr, g, L5, 1, 0, 0, st));
  CK(pack_rhs<double>(in_dev, io.v, nullptr, g, L5, 1, 1, 0, st));
  cudaError_t me = cudaSuccess;
  double* mass = (double*)ws_get(ctx, "dd.mass", sizeof(double), &me);
  CK(me);
  CK(cudaMemcpyAsync(mass, &cfg->act.mf, sizeof(double), cudaMemcpyHostToDevice, st));
  FastOp<double, double> fo;
  fo.g = g; fo.L5 = L5; fo.N = 1; fo.anti = cfg->anti; fo.U = cfg->U64; fo.st = st;
  fo.f = make_fifth<double>(cfg->act, mass);
  choose_hop(fo, cfg, 0, HOP_DIRECT, nullptr);
  Tiling tb = make_tiling(g.Vh, L5, 1, 2, 512);
  // the field the hop reads: B in for D, in otherwise
  const bool bfirst = kind == 1 && !dagger;
  if (bfirst) {
    CK(bop<double>(ie.v, nullptr, te.v, nullptr, fo.f, tb, g.Vh, L5, 1, nullptr, st));
    CK(bop<double>(io.v, nullptr, to.v, nullptr, fo.f, tb, g.Vh, L5, 1, nullptr, st));
  }
  const F<double> he = bfirst ? te : ie, ho = bfirst ? to : io;
  if (pack) {
    CK(dd_pack_faces(he.v, g, 0, L5, 1, dagger, cfg->U64, face_prev, face_next, st));
    CK(dd_pack_faces(ho.v, g, 1, L5, 1, dagger, cfg->U64, face_prev, face_next, st));
    CK(cudaStreamSynchronize(st));
    return MDWF_OK;
  }
  CK(ws_field<double>(ctx, "dd.oe", units, &oe));
  CK(ws_field<double>(ctx, "dd.oo", units, &oo));
  fo.halo_fwd = halo_next;
  fo.halo_bwd = halo_prev;
  fo.halo_sgn_fwd = sign_next;
  fo.halo_sgn_bwd = sign_prev;
  F<double> none;
  if (kind == 0) {
    CK(fo.run(E_RAW, 0, dagger, ho, none, none, 0.0, 1.0, oe, nullptr, nullptr));
    CK(fo.run(E_RAW, 1, dagger, he, none, none, 0.0, 1.0, oo, nullptr, nullptr));
  } else if (!dagger) {   // D x = A x - 1/2 H B x
    CK(fo.run(E_A_SAME, 0, 0, to, ie, none, 1.0, -0.5, oe, nullptr, nullptr));
    CK(fo.run(E_A_SAME, 1, 0, te, io, none, 1.0, -0.5, oo, nullptr, nullptr));
  } else {                // D^+ x = A^+ x - 1/2 B^+ H^+ x
    CK(fo.run(E_AD_SAME_BD, 0, 1, io, ie, none, 1.0, -0.5, oe, nullptr, nullptr));
    CK(fo.run(E_AD_SAME_BD, 1, 1, ie, io, none, 1.0, -0.5, oo, nullptr, nullptr));
  }
  CK(unpack_rhs<double>(oe.v, nullptr, out_dev, g, L5, 1, 0, 0, st));
  CK(unpack_rhs<double>(oo.v, nullptr, out_dev, g, L5, 1, 1, 0, st));
  CK(cudaStreamSynchronize(st));
  return MDWF_OK;
}

template <typename S>
int schur_apply_impl(mdwf_ctx* ctx, Cfg* cfg, const double* in_dev, double* out_dev, int dagger, cudaStream_t st) {
  using T = typename StoreTraits<S>::T;
  const Geom& g = ctx->g;
  const int L5 = cfg->act.L5;
  DBuf mass;
  CK(mass.alloc(sizeof(T)));
  const T m = (T)cfg->act.mf;
  CK(cudaMemcpyAsync(mass.p, &m, sizeof(T), cudaMemcpyHostToDevice, st));
  FastOp<S, T> op;
  op.g = g; op.L5 = L5; op.N = 1; op.anti = cfg->anti; op.st = st;
  op.U = std::is_same<T, double>::value ? (const T*)cfg->U64 : (const T*)cfg->U32;
  op.f = make_fifth<T>(cfg->act, mass.as<T>());
  DBuf errw;
  CK(errw.alloc(sizeof(int)));
  CK(cudaMemsetAsync(errw.p, 0, sizeof(int), st));
  StageInfo si;
  si.spin_bytes = si.nrm_bytes = 0;
  si.budget = wait_budget(ctx->device, 2.0);
  si.extra_tx = 0;
  si.err = errw.as<int>();
  choose_hop(op, cfg, 0, HOP_AUTO, &si);
  Tiling tb = make_tiling(g.Vh, L5, 1, 2, 512);
  long units = g.Vh * L5;
  FieldBuf<S> in, u, t, out;
  for (auto* f : {&in, &u, &t, &out}) CK(f->alloc(units));
  FieldBuf<double> o64;
  CK(o64.alloc(2 * units));
  CK(pack_rhs<S>(in_dev, in.f().v, in.f().n, g, L5, 1, 0, 0, st));
  if (!dagger) {
    CK(bop<S>(in.f().v, in.f().n, u.f().v, u.f().n, op.f, tb, g.Vh, L5, 1, nullptr, st));
    CK(op.mhat(in.f(), u.f(), t.f(), out.f(), nullptr, nullptr));
  } else {
    CK(op.mhat_dag(in.f(), t.f(), out.f(), nullptr, nullptr));
  }
  CK(unpack_rhs<S>(out.f().v, out.f().n, out_dev, g, L5, 1, 0, 0, st));
  CK(cudaMemsetAsync(o64.v.p, 0, o64.v.bytes, st));
  CK(unpack_rhs<double>(o64.f().v, nullptr, out_dev, g, L5, 1, 1, 0, st));
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, errw.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (herr) return fail(ctx, MDWF_ERR_TIMEOUT, "a bounded device wait ran out");
  return MDWF_OK;
}

// Batched Schur operator on device API-layout fields (the solver's hot kernels).
template <typename S>
int schur_batch_impl(mdwf_ctx* ctx, Cfg* cfg, int n, const double* const* in, double* const* out,
                     const std::vector<double>& masses, int dagger, int flags, cudaStream_t st) {
  using T = typename StoreTraits<S>::T;
  const Geom& g = ctx->g;
  const int L5 = cfg->act.L5, N = n;
  const long units = g.Vh * L5 * N;
  cudaError_t e = cudaSuccess;
  T* mass = (T*)ws_get(ctx, "sb.mass", sizeof(T) * N, &e); CK(e);
  std::vector<T> mh(masses.begin(), masses.end());
  CK(cudaMemcpyAsync(mass, mh.data(), sizeof(T) * N, cudaMemcpyHostToDevice, st));
  int* errw = (int*)ws_get(ctx, "sb.errw", sizeof(int), &e); CK(e);
  CK(cudaMemsetAsync(errw, 0, sizeof(int), st));
  FastOp<S, T> op;
  op.g = g; op.L5 = L5; op.N = N; op.anti = cfg->anti; op.st = st;
  op.U = std::is_same<T, double>::value ? (const T*)cfg->U64 : (const T*)cfg->U32;
  op.f = make_fifth<T>(cfg->act, mass);
  StageInfo si;
  si.spin_bytes = si.nrm_bytes = 0;
  si.budget = wait_budget(ctx->device, 2.0);
  si.extra_tx = 0;
  si.err = errw;
  choose_hop(op, cfg, (flags >> 8) & 0xff, flags & 0xff, &si);
  if ((flags >> 16) & 1) {   // 12-real links (the paired hop reconstructs the third row)
    if (int r12 = ensure_u12(ctx, cfg)) return r12;
    op.U12 = std::is_same<T, double>::value ? nullptr : cfg->U12;
  }
  Tiling tb = make_tiling(g.Vh, L5, N, 2, 1024);
  F<S> fin, fu, ft, fo;
  CK(ws_field<S>(ctx, "sb.in", units, &fin));
  CK(ws_field<S>(ctx, "sb.u", units, &fu));
  CK(ws_field<S>(ctx, "sb.t", units, &ft));
  CK(ws_field<S>(ctx, "sb.out", units, &fo));
  F<double> zero;
  CK(ws_field<double>(ctx, "sb.zero", g.Vh * L5, &zero));
  CK(cudaMemsetAsync(zero.v, 0, sizeof(double) * 24 * (size_t)g.Vh * L5, st));
  for (int i = 0; i < N; i++) CK(pack_rhs<S>(in[i], fin.v, fin.n, g, L5, N, 0, i, st));
  if (!dagger) {
    CK(bop<S>(fin.v, fin.n, fu.v, fu.n, op.f, tb, g.Vh, L5, N, nullptr, st));
    CK(op.mhat(fin, fu, ft, fo, nullptr, nullptr));
  } else {
    CK(op.mhat_dag(fin, ft, fo, nullptr, nullptr));
  }
  for (int i = 0; i < N; i++) {
    CK(unpack_rhs<S>(fo.v, fo.n, out[i], g, L5, N, 0, i, st));
    CK(unpack_rhs<double>(zero.v, nullptr, out[i], g, L5, 1, 1, 0, st));
  }
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, errw, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (herr) return fail(ctx, MDWF_ERR_TIMEOUT, "a bounded device wait ran out");
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
  o->nsb = 0;
  o->wait_timeout_s = 2.0;
  o->hop_variant = 0;
  o->max_restarts = 3;
  o->stop_scale_test = 1.0;
  o->link_recon = 18;
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
    if (kv.second.F16) cudaFree(kv.second.F16);
    if (kv.second.U12) cudaFree(kv.second.U12);
  }
  for (auto& kv : ctx->ws)
    if (kv.second.first) cudaFree(kv.second.first);
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
  {
    auto it = ctx->cfgs.find(cfg_id);    // a two-row copy of a previous field is stale now
    if (it != ctx->cfgs.end() && it->second.U12) { cudaFree(it->second.U12); it->second.U12 = nullptr; }
  }
  // reorder to [parity][h][mu][18] (FP64) and [parity][h][mu][20] (FP32, padded)
  const size_t n32 = (size_t)g.V * 4 * kLinkStride32;
  std::vector<double> h64(n);
  std::vector<float> h32(n32, 0.0f);
  for (long lex = 0; lex < g.V; lex++) {
    long r = lex;
    int c[4];
    for (int i = 0; i < 4; i++) { c[i] = (int)(r % g.L[i]); r /= g.L[i]; }
    int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    long h = lex >> 1;
    for (int mu = 0; mu < 4; mu++)
      for (int k = 0; k < 18; k++) {
        double v = U[(lex * 4 + mu) * 18 + k];
        size_t link = ((size_t)par * g.Vh + h) * 4 + mu;
        h64[link * 18 + k] = v;
        h32[link * kLinkStride32 + k] = (float)v;
      }
  }
  CK(cudaSetDevice(ctx->device));
  Cfg& cfg = ctx->cfgs[cfg_id];
  if (!cfg.U64) CK(cudaMalloc(&cfg.U64, sizeof(double) * n));
  if (!cfg.U32) CK(cudaMalloc(&cfg.U32, sizeof(float) * n32));
  if (!cfg.F16) CK(cudaMalloc(&cfg.F16, sizeof(uint32_t) * 64 * (size_t)g.V * 4));
  CK(cudaMemcpy(cfg.U64, h64.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
  CK(build_link_frags(cfg.U64, cfg.F16, (long)g.V * 4, nullptr));
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(cfg.U32, h32.data(), sizeof(float) * n32, cudaMemcpyHostToDevice));
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
  for (int i = 0; i < n; i++)
    if (!srcs[i] || !xs[i]) return fail(ctx, MDWF_ERR_ARG, "solve_batch: null source or solution");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const size_t n5 = (size_t)cfg->act.L5 * ctx->g.V * 24;
  // device copies of the sources and solutions live in the context's workspace
  // (allocated once, grown on demand); a non-finite source is caught by the
  // solve's own device norms (MDWF_ERR_NONFINITE), so the host does not scan it
  cudaError_t e = cudaSuccess;
  double* dsrc = (double*)ws_get(ctx, "e2e.src", sizeof(double) * n5 * n, &e);
  CK(e);
  double* dx = (double*)ws_get(ctx, "e2e.x", sizeof(double) * n5 * n, &e);
  CK(e);
  std::vector<const double*> s(n);
  std::vector<double*> x(n);
  for (int i = 0; i < n; i++) {
    CK(cudaMemcpyAsync(dsrc + n5 * i, srcs[i], sizeof(double) * n5, cudaMemcpyHostToDevice, st));
    s[i] = dsrc + n5 * i;
    x[i] = dx + n5 * i;
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

int mdwf_dd_pack_faces_dev(mdwf_ctx* ctx, int cfg_id, int kind, int dagger, const double* in, double* face_prev,
                           double* face_next, void* stream) {
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (!in || !face_prev || !face_next || (kind != 0 && kind != 1))
    return fail(ctx, MDWF_ERR_ARG, "dd_pack_faces: bad kind or null pointer");
  CK(cudaSetDevice(ctx->device));
  return dd_impl(ctx, cfg, true, kind, dagger ? 1 : 0, in, nullptr, face_prev, face_next, nullptr, nullptr, 1.0, 1.0,
                 pick_stream(ctx, stream));
}

int mdwf_dd_apply_dev(mdwf_ctx* ctx, int cfg_id, int kind, int dagger, const double* in, double* out,
                      const double* halo_next, const double* halo_prev, double sign_next, double sign_prev,
                      void* stream) {
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (!in || !out || !halo_next || !halo_prev || (kind != 0 && kind != 1))
    return fail(ctx, MDWF_ERR_ARG, "dd_apply: bad kind or null pointer");
  if (!std::isfinite(sign_next) || !std::isfinite(sign_prev)) return fail(ctx, MDWF_ERR_ARG, "dd_apply: bad sign");
  CK(cudaSetDevice(ctx->device));
  return dd_impl(ctx, cfg, false, kind, dagger ? 1 : 0, in, out, nullptr, nullptr, halo_next, halo_prev, sign_next,
                 sign_prev, pick_stream(ctx, stream));
}

int mdwf_apply_schur_batch_dev(mdwf_ctx* ctx, int cfg_id, int n, const double* const* in, double* const* out,
                               const double* masses, int dagger, int precision, int flags, void* stream) {
  if (!ctx) return MDWF_ERR_ARG;
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (n < 1 || n > 1024 || !in || !out) return fail(ctx, MDWF_ERR_ARG, "apply_schur_batch_dev: bad n or pointers");
  std::vector<double> m(n, cfg->act.mf);
  for (int i = 0; i < n; i++) {
    if (!in[i] || !out[i]) return fail(ctx, MDWF_ERR_ARG, "apply_schur_batch_dev: null field");
    if (masses) m[i] = masses[i];
  }
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = pick_stream(ctx, stream);
  switch (precision) {
    case MDWF_PREC_DOUBLE: return schur_batch_impl<double>(ctx, cfg, n, in, out, m, dagger, flags, st);
    case MDWF_PREC_SINGLE: return schur_batch_impl<float>(ctx, cfg, n, in, out, m, dagger, flags, st);
    case MDWF_PREC_HALF: return schur_batch_impl<__half>(ctx, cfg, n, in, out, m, dagger, flags, st);
    case MDWF_PREC_BF16: return schur_batch_impl<__nv_bfloat16>(ctx, cfg, n, in, out, m, dagger, flags, st);
    default: return fail(ctx, MDWF_ERR_ARG, "apply_schur_batch_dev: unknown precision");
  }
}

// --- sessions ---------------------------------------------------------------
long long mdwf_session_bytes(mdwf_ctx* ctx, int cfg_id, int slots, int precision) {
  if (!ctx) return -1;
  auto it = ctx->cfgs.find(cfg_id);
  if (it == ctx->cfgs.end() || !it->second.act.set || slots < 1) return -1;
  const double units = (double)ctx->g.Vh * it->second.act.L5 * slots;
  const double s = precision == MDWF_PREC_DOUBLE ? 192 : precision == MDWF_PREC_SINGLE ? 96
                 : precision == MDWF_PREC_HALF ? 52 : 48;
  const double x = precision == MDWF_PREC_DOUBLE ? 192 : 96;
  // nine FP64 fields (seven solver fields and the slots' own sources; the FP32
  // update fields share two of them), six inner fields, x_lo, partial sums
  return (long long)(units * (9 * 192 + 6 * s + x) + (double)ctx->g.Vh * slots * 8 + 4096.0 * slots);
}

int mdwf_session_create(mdwf_ctx* ctx, int cfg_id, int slots, const mdwf_solver_opts* opts, double tol, void* stream,
                        mdwf_session** out) {
  if (!ctx || !out) return MDWF_ERR_ARG;
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (slots < 1 || slots > 1024 || !(tol > 0)) return fail(ctx, MDWF_ERR_ARG, "session_create: bad slots or tol");
  mdwf_solver_opts o;
  mdwf_default_opts(&o);
  if (opts) o = *opts;
  CK(cudaSetDevice(ctx->device));
  mdwf_session* sess = new mdwf_session();
  sess->ctx = ctx;
  sess->prefix = "session" + std::to_string(ctx->next_session++) + ".";
  sess->stream = pick_stream(ctx, stream);
  switch (o.precision) {
    case MDWF_PREC_DOUBLE: { auto* p = new SessionImpl<double>(); sess->impl = p; rc = p->create(ctx, cfg, slots, o, tol, sess->stream, sess->prefix); break; }
    case MDWF_PREC_SINGLE: { auto* p = new SessionImpl<float>(); sess->impl = p; rc = p->create(ctx, cfg, slots, o, tol, sess->stream, sess->prefix); break; }
    case MDWF_PREC_HALF: { auto* p = new SessionImpl<__half>(); sess->impl = p; rc = p->create(ctx, cfg, slots, o, tol, sess->stream, sess->prefix); break; }
    case MDWF_PREC_BF16: { auto* p = new SessionImpl<__nv_bfloat16>(); sess->impl = p; rc = p->create(ctx, cfg, slots, o, tol, sess->stream, sess->prefix); break; }
    default: rc = fail(ctx, MDWF_ERR_ARG, "session_create: unknown precision");
  }
  if (rc) {
    delete sess->impl;
    ws_release_prefix(ctx, sess->prefix);
    delete sess;
    return rc;
  }
  *out = sess;
  return MDWF_OK;
}

int mdwf_session_destroy(mdwf_session* s) {
  if (!s) return MDWF_OK;
  cudaSetDevice(s->ctx->device);
  cudaStreamSynchronize(s->stream);
  delete s->impl;
  ws_release_prefix(s->ctx, s->prefix);
  delete s;
  return MDWF_OK;
}

int mdwf_session_submit(mdwf_session* s, const double* src5d, double mass, double* x5d, long long tag, int* slot) {
  if (!s) return MDWF_ERR_ARG;
  mdwf_ctx* ctx = s->ctx;
  if (!src5d || !x5d || !std::isfinite(mass)) return fail(ctx, MDWF_ERR_ARG, "session_submit: bad source, solution or mass");
  CK(cudaSetDevice(ctx->device));
  return s->impl->submit(src5d, mass, x5d, tag, slot);
}

int mdwf_session_launch(mdwf_session* s, int iters) {
  if (!s) return MDWF_ERR_ARG;
  mdwf_ctx* ctx = s->ctx;
  CK(cudaSetDevice(ctx->device));
  return s->impl->launch(iters);
}

int mdwf_session_poll(mdwf_session* s, int max_done, long long* tags, mdwf_solve_stats* stats, int* n_done) {
  if (!s || !n_done || max_done < 0) return MDWF_ERR_ARG;
  mdwf_ctx* ctx = s->ctx;
  CK(cudaSetDevice(ctx->device));
  return s->impl->poll(max_done, tags, stats, n_done);
}

int mdwf_session_occupied(const mdwf_session* s) { return s ? s->impl->occupied() : -1; }

int mdwf_make_source_dev(mdwf_ctx* ctx, int cfg_id, const double* eta4d, double* src5d, void* stream) {
  if (!ctx) return MDWF_ERR_ARG;
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (!eta4d || !src5d) return fail(ctx, MDWF_ERR_ARG, "make_source_dev: null pointer");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = pick_stream(ctx, stream);
  const size_t n5 = (size_t)cfg->act.L5 * ctx->g.V * 24;
  cudaError_t e = cudaSuccess;
  double* w = (double*)ws_get(ctx, "make_source.walls", sizeof(double) * n5, &e);
  CK(e);
  CK(cudaMemsetAsync(w, 0, sizeof(double) * n5, st));
  CK(walls(eta4d, w, ctx->g.V, cfg->act.L5, st));
  return apply_dev(ctx, cfg, 3, 0, 0, w, src5d, st);
}

int mdwf_z2_source_dev(mdwf_ctx* ctx, unsigned long long seed, double* eta4d, void* stream) {
  if (!ctx) return MDWF_ERR_ARG;
  if (!eta4d) return fail(ctx, MDWF_ERR_ARG, "z2_source_dev: null pointer");
  CK(cudaSetDevice(ctx->device));
  CK(z2_source(seed, eta4d, ctx->g.V, pick_stream(ctx, stream)));
  return MDWF_OK;
}

int mdwf_autotune(mdwf_ctx* ctx, int cfg_id, int n, int precision, int include_tensor_core, int* hop_variant,
                  int* nsb, double* ms_per_pair) {
  if (!ctx) return MDWF_ERR_ARG;
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (n < 1 || n > 1024) return fail(ctx, MDWF_ERR_ARG, "autotune: bad n");
  CK(cudaSetDevice(ctx->device));
  mdwf_solver_opts o;
  mdwf_default_opts(&o);
  o.precision = precision;
  o.hop_variant = include_tensor_core ? HOP_TUNE_ALL : HOP_AUTO;
  std::vector<double> m(n, cfg->act.mf);
  // the timing runs use the solver workspace of the context (the fields a solve of
  // n RHS uses and re-initialises), so they need no second set of fields
  auto run = [&](auto& sv) -> int {
    int r = sv.init(ctx, cfg, m, 0, false, o, ctx->stream);
    if (r) return r;
    return sv.tune(o.hop_variant, hop_variant, nsb, ms_per_pair);
  };
  switch (precision) {
    case MDWF_PREC_DOUBLE: { BatchSolver<double> sv; rc = run(sv); break; }
    case MDWF_PREC_SINGLE: { BatchSolver<float> sv; rc = run(sv); break; }
    case MDWF_PREC_HALF: { BatchSolver<__half> sv; rc = run(sv); break; }
    case MDWF_PREC_BF16: { BatchSolver<__nv_bfloat16> sv; rc = run(sv); break; }
    default: return fail(ctx, MDWF_ERR_ARG, "autotune: unknown precision");
  }
  return rc;
}

int mdwf_wilson_flow_dev(mdwf_ctx* ctx, double* U, double eps, int nsteps, void* stream) {
  if (!ctx) return MDWF_ERR_ARG;
  if (!U || nsteps < 0 || !std::isfinite(eps)) return fail(ctx, MDWF_ERR_ARG, "wilson_flow_dev: bad arguments");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = pick_stream(ctx, stream);
  const size_t nlink = (size_t)ctx->g.V * 4;
  cudaError_t e = cudaSuccess;
  double* Z = (double*)ws_get(ctx, "flow.Z", sizeof(double) * 54 * nlink, &e);
  CK(e);
  CK(wilson_flow(U, ctx->g.L, eps, nsteps, Z, st));
  CK(cudaStreamSynchronize(st));
  ws_release_prefix(ctx, "flow.");
  return MDWF_OK;
}

int mdwf_plaquette_dev(mdwf_ctx* ctx, const double* U, double* plaq) {
  if (!ctx) return MDWF_ERR_ARG;
  if (!U || !plaq) return fail(ctx, MDWF_ERR_ARG, "plaquette_dev: null pointer");
  CK(cudaSetDevice(ctx->device));
  cudaError_t e = cudaSuccess;
  double* part = (double*)ws_get(ctx, "plaq.part", sizeof(double) * (ctx->g.V + 1), &e);
  CK(e);
  CK(plaquette(U, ctx->g.L, part + 1, part, ctx->stream));
  double tot = 0.0;
  CK(cudaMemcpyAsync(&tot, part, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *plaq = tot / (18.0 * (double)ctx->g.V);
  return MDWF_OK;
}

int mdwf_mres_correlators_dev(mdwf_ctx* ctx, int cfg_id, int n, double* const* xs, double* c_pp, double* c_j5q,
                              void* stream) {
  if (!ctx) return MDWF_ERR_ARG;
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (n < 1 || !xs || !c_pp || !c_j5q) return fail(ctx, MDWF_ERR_ARG, "mres_correlators: bad arguments");
  for (int i = 0; i < n; i++)
    if (!xs[i]) return fail(ctx, MDWF_ERR_ARG, "mres_correlators: null solution");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = pick_stream(ctx, stream);
  const long V = ctx->g.V;
  const int Lt = ctx->g.L[3];
  cudaError_t e = cudaSuccess;
  double** dptr = (double**)ws_get(ctx, "mres.ptrs", sizeof(double*) * n, &e);
  CK(e);
  double* site = (double*)ws_get(ctx, "mres.site", sizeof(double) * (2 * V + 2 * Lt), &e);
  CK(e);
  CK(cudaMemcpyAsync(dptr, xs, sizeof(double*) * n, cudaMemcpyHostToDevice, st));
  CK(mres_correlators(dptr, n, V, Lt, cfg->act.L5, site, site + V, site + 2 * V, site + 2 * V + Lt, st));
  CK(cudaMemcpyAsync(c_pp, site + 2 * V, sizeof(double) * Lt, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(c_j5q, site + 2 * V + Lt, sizeof(double) * Lt, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return MDWF_OK;
}

int mdwf_smear_source_dev(mdwf_ctx* ctx, int cfg_id, double* eta4d, double sigma, int n_iter, void* stream) {
  if (!ctx) return MDWF_ERR_ARG;
  auto it = ctx->cfgs.find(cfg_id);
  if (it == ctx->cfgs.end() || !it->second.has_gauge) return fail(ctx, MDWF_ERR_STATE, "no gauge field for cfg_id");
  if (!eta4d || n_iter < 0 || !(sigma >= 0) || !std::isfinite(sigma))
    return fail(ctx, MDWF_ERR_ARG, "smear_source_dev: bad arguments");
  if (n_iter == 0 || sigma == 0.0) return MDWF_OK;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = pick_stream(ctx, stream);
  cudaError_t e = cudaSuccess;
  double* tmp = (double*)ws_get(ctx, "smear.tmp", sizeof(double) * 24 * (size_t)ctx->g.V, &e);
  CK(e);
  const double k = sigma * sigma / (4.0 * n_iter);
  double* a = eta4d;
  double* b = tmp;
  for (int i = 0; i < n_iter; i++) {
    CK(smear_step(it->second.U64, a, b, ctx->g, k, st));
    std::swap(a, b);
  }
  if (a != eta4d) CK(cudaMemcpyAsync(eta4d, a, sizeof(double) * 24 * (size_t)ctx->g.V, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  return MDWF_OK;
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

// ===========================================================================
// The batched Schur operator without device allocation
// ===========================================================================
// For callers that may not call cudaMalloc (the device memory belongs to another
// pool, or an allocation's implicit device synchronisation is not acceptable on
// their path).  All scratch comes from one fixed array that is part of this
// library's device image; see mdwf_apply_schur_batch_dev_noalloc in mdwf.h.
#include <mutex>

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MDWF_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on ctx's device (which must be current).
// In host code the array's name is only a stand-in; the address is looked up
// on every call (a host-side lookup that allocates nothing), so it is never
// stale after a context reset.
int noalloc_scratch(mdwf_ctx* ctx, unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr)
    return fail(ctx, MDWF_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array: ") +
                                        cudaGetErrorString(e));
  *out = static_cast<unsigned char*>(p);
  return MDWF_OK;
}

inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename S>
int schur_batch_noalloc_impl(mdwf_ctx* ctx, Cfg* cfg, int n, const double* const* in, double* const* out,
                             const std::vector<double>& masses, int dagger, cudaStream_t st) {
  using T = typename StoreTraits<S>::T;
  const Geom& g = ctx->g;
  const int L5 = cfg->act.L5, N = n;
  const size_t units = (size_t)g.Vh * L5 * N;
  const size_t fbytes = round256(sizeof(S) * 24 * units);
  const size_t nbytes = StoreTraits<S>::kNorm ? round256(sizeof(float) * units) : 0;
  const size_t mbytes = round256(sizeof(T) * N);
  const size_t need = mbytes + 4 * (fbytes + nbytes);
  if (need > (size_t)MDWF_NOALLOC_SCRATCH_BYTES)
    return fail(ctx, MDWF_ERR_ARG, "apply_schur_batch_dev_noalloc: this problem needs " + std::to_string(need) +
                                       " bytes of scratch, more than the fixed " +
                                       std::to_string((size_t)MDWF_NOALLOC_SCRATCH_BYTES) + " bytes");
  unsigned char* base = nullptr;
  int rc = noalloc_scratch(ctx, &base);
  if (rc) return rc;
  // carve: [masses][in][u][t][out], each field followed by its fp16 scales
  T* mass = reinterpret_cast<T*>(base);
  F<S> f[4];
  unsigned char* p = base + mbytes;
  for (int i = 0; i < 4; i++) {
    f[i].v = reinterpret_cast<S*>(p);
    p += fbytes;
    f[i].n = nbytes ? reinterpret_cast<float*>(p) : nullptr;
    p += nbytes;
  }
  F<S> fin = f[0], fu = f[1], ft = f[2], fo = f[3];
  std::vector<T> mh(masses.begin(), masses.end());
  CK(cudaMemcpyAsync(mass, mh.data(), sizeof(T) * N, cudaMemcpyHostToDevice, st));
  FastOp<S, T> op;
  op.g = g; op.L5 = L5; op.N = N; op.anti = cfg->anti; op.st = st;
  op.U = std::is_same<T, double>::value ? (const T*)cfg->U64 : (const T*)cfg->U32;
  op.f = make_fifth<T>(cfg->act, mass);
  choose_hop(op, cfg, 0, HOP_DIRECT, nullptr);
  Tiling tb = make_tiling(g.Vh, L5, N, 2, 1024);
  for (int i = 0; i < N; i++) CK(pack_rhs<S>(in[i], fin.v, fin.n, g, L5, N, 0, i, st));
  if (!dagger) {
    CK(bop<S>(fin.v, fin.n, fu.v, fu.n, op.f, tb, g.Vh, L5, N, nullptr, st));
    CK(op.mhat(fin, fu, ft, fo, nullptr, nullptr));
  } else {
    CK(op.mhat_dag(fin, ft, fo, nullptr, nullptr));
  }
  // the intermediate odd field is no longer needed: zero it and use it as the
  // source of the odd sites of every output (they must come out zero)
  CK(cudaMemsetAsync(ft.v, 0, fbytes, st));
  if (nbytes) CK(cudaMemsetAsync(ft.n, 0, nbytes, st));
  for (int i = 0; i < N; i++) {
    CK(unpack_rhs<S>(fo.v, fo.n, out[i], g, L5, N, 0, i, st));
    CK(unpack_rhs<S>(ft.v, ft.n, out[i], g, L5, N, 1, i, st));
  }
  CK(cudaStreamSynchronize(st));
  return MDWF_OK;
}

}  // namespace

extern "C" int mdwf_apply_schur_batch_dev_noalloc(mdwf_ctx* ctx, int cfg_id, int n, const double* const* in,
                                                  double* const* out, const double* masses, int dagger,
                                                  int precision, void* stream) {
  if (!ctx) return MDWF_ERR_ARG;
  Cfg* cfg;
  int rc = check_cfg(ctx, cfg_id, &cfg);
  if (rc) return rc;
  if (n < 1 || n > 1024 || !in || !out) return fail(ctx, MDWF_ERR_ARG, "apply_schur_batch_dev_noalloc: bad n or pointers");
  std::vector<double> m(n, cfg->act.mf);
  for (int i = 0; i < n; i++) {
    if (!in[i] || !out[i]) return fail(ctx, MDWF_ERR_ARG, "apply_schur_batch_dev_noalloc: null field");
    if (masses) m[i] = masses[i];
  }
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = pick_stream(ctx, stream);
  switch (precision) {
    case MDWF_PREC_DOUBLE: return schur_batch_noalloc_impl<double>(ctx, cfg, n, in, out, m, dagger, st);
    case MDWF_PREC_SINGLE: return schur_batch_noalloc_impl<float>(ctx, cfg, n, in, out, m, dagger, st);
    case MDWF_PREC_HALF: return schur_batch_noalloc_impl<__half>(ctx, cfg, n, in, out, m, dagger, st);
    case MDWF_PREC_BF16: return schur_batch_noalloc_impl<__nv_bfloat16>(ctx, cfg, n, in, out, m, dagger, st);
    default: return fail(ctx, MDWF_ERR_ARG, "apply_schur_batch_dev_noalloc: unknown precision");
  }
}
