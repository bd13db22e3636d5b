// Vector kernels of the solver: layout conversion, precision conversion,
// the CG updates with their fused norms, and the fixed-order reductions.
//
// All unit-wise kernels use the tile mapping of the hop kernel (tile of nsb
// sites x L5 slices x rt slots per block), so per-slot partial sums are formed
// per tile in a fixed order and the final sum over tiles is also fixed: a
// slot's result does not depend on how many other slots share the launch.
#include <cooperative_groups.h>

#include "blas.h"

namespace mdwf {

struct Unit {
  long h;
  int s, r, site_l, r_l;
  bool valid;
  long u;
};

__device__ __forceinline__ Unit unit_of(const Tiling& tl, long Vh, int L5, int N) {
  Unit x;
  const int tid = threadIdx.x;
  x.r_l = tid % tl.rt;
  x.s = (tid / tl.rt) % L5;
  x.site_l = tid / (tl.rt * L5);
  x.h = (long)blockIdx.x * tl.nsb + x.site_l;
  x.r = blockIdx.y * tl.rt + x.r_l;
  x.valid = (x.h < Vh) && (x.r < N);
  x.u = (x.h * L5 + x.s) * N + x.r;
  return x;
}

// The FP32 solution accumulator x_lo of the mixed-precision solver is stored
// tile-major: block b = blockIdx.y * gridDim.x + blockIdx.x of the BLAS tiling
// holds its T = tl.threads units as six planes of float4 (plane k: components
// 4k .. 4k+3 of the [spin][colour][re, im] order), thread t's plane k at float4
// index (6 b + k) T + t.  One plane of a warp is 512 contiguous bytes, where the
// unit-major layout would stride each thread's 16 bytes by 96.  Every kernel that
// touches x_lo uses the same tiling; the field holds xlo_units(tl) units.  An
// FP64 accumulator (the FP64 solver) keeps the unit-major layout.
template <typename SX>
struct XloLayout {
  static __device__ __forceinline__ void load(const SX* v, const Unit& x, const Tiling&, SX a[24]) {
    load24<SX, SX>(v, nullptr, x.u, a);
  }
  static __device__ __forceinline__ void store(SX* v, const Unit& x, const Tiling&, const SX a[24]) {
    store24<SX, SX>(v, nullptr, x.u, a);
  }
};
template <>
struct XloLayout<float> {
  static __device__ __forceinline__ long base(const Tiling& tl) {
    return ((long)blockIdx.y * gridDim.x + blockIdx.x) * 6 * tl.threads + threadIdx.x;
  }
  static __device__ __forceinline__ void load(const float* v, const Unit&, const Tiling& tl, float a[24]) {
    const float4* p = reinterpret_cast<const float4*>(v) + base(tl);
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const float4 t = __ldg(p + (long)k * tl.threads);
      a[4 * k] = t.x; a[4 * k + 1] = t.y; a[4 * k + 2] = t.z; a[4 * k + 3] = t.w;
    }
  }
  static __device__ __forceinline__ void store(float* v, const Unit&, const Tiling& tl, const float a[24]) {
    float4* p = reinterpret_cast<float4*>(v) + base(tl);
#pragma unroll
    for (int k = 0; k < 6; k++) p[(long)k * tl.threads] = make_float4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
  }
};

// Per-site, per-slot sum of `v` over the L5 slices (fixed order), written to
// partials[r][h]; the final sum over sites is then independent of the tiling.
__device__ __forceinline__ void block_partial(double v, const Unit& x, const Tiling& tl, int L5, long Vh,
                                              double* __restrict__ partials) {
  __shared__ double sred[1024];
  sred[threadIdx.x] = v;
  __syncthreads();
  if (x.s == 0 && x.valid) {
    double sum = 0.0;
    for (int k = 0; k < L5; k++) sum += sred[(x.site_l * L5 + k) * tl.rt + x.r_l];
    partials[(long)x.r * Vh + x.h] = sum;
  }
}

template <typename S>
__global__ void k_pack(const double* __restrict__ api, S* __restrict__ out, float* __restrict__ out_nrm, Geom g,
                       int L5, int N, int par, int r) {
  using T = typename StoreTraits<S>::T;
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.Vh * L5) return;
  long h = idx / L5;
  int s = (int)(idx - h * L5);
  int c[4];
  site_coords(g, par, h, c);
  long lex = lex_index(g, c);
  const double* src = api + ((long)s * g.V + lex) * 24;
  T a[24];
#pragma unroll
  for (int i = 0; i < 24; i++) a[i] = (T)src[i];
  store24<S, T>(out, out_nrm, (h * L5 + s) * N + r, a);
}

template <typename S>
__global__ void k_unpack(const S* __restrict__ in, const float* __restrict__ in_nrm, double* __restrict__ api, Geom g,
                         int L5, int N, int par, int r) {
  using T = typename StoreTraits<S>::T;
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.Vh * L5) return;
  long h = idx / L5;
  int s = (int)(idx - h * L5);
  int c[4];
  site_coords(g, par, h, c);
  long lex = lex_index(g, c);
  double* dst = api + ((long)s * g.V + lex) * 24;
  T a[24];
  load24<S, T>(in, in_nrm, (h * L5 + s) * N + r, a);
#pragma unroll
  for (int i = 0; i < 24; i++) dst[i] = (double)a[i];
}

template <typename Si, typename So>
__global__ void k_convert(const Si* __restrict__ in, const float* __restrict__ in_nrm, So* __restrict__ out,
                          float* __restrict__ out_nrm, Tiling tl, long Vh, int L5, int N, const int* __restrict__ mask) {
  Unit x = unit_of(tl, Vh, L5, N);
  if (!x.valid || (mask && !mask[x.r])) return;
  using Ti = typename StoreTraits<Si>::T;
  using To = typename StoreTraits<So>::T;
  Ti a[24];
  load24<Si, Ti>(in, in_nrm, x.u, a);
  To b[24];
#pragma unroll
  for (int i = 0; i < 24; i++) b[i] = (To)a[i];
  store24<So, To>(out, out_nrm, x.u, b);
}

// x += alpha_r p ; rho -= alpha_r q ; |rho|^2 of one unit, explicit roundings.
__device__ __forceinline__ float axpy_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double axpy_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename TX, typename T>
__device__ __forceinline__ T axpy_unit(T a, const T* pv, const T* qv, T* rv, TX* xv) {
  T n2t = 0;
#pragma unroll
  for (int i = 0; i < 24; i++) {
    xv[i] = axpy_fma((TX)a, (TX)pv[i], xv[i]);
    rv[i] = axpy_fma(-a, qv[i], rv[i]);
    n2t = axpy_fma(rv[i], rv[i], n2t);
  }
  return n2t;
}

template <typename SX, typename S>
__global__ void k_axpy_x_rho(SX* __restrict__ xv, const S* __restrict__ p, const float* __restrict__ p_nrm,
                             S* __restrict__ rho, float* __restrict__ rho_nrm, const S* __restrict__ q,
                             const float* __restrict__ q_nrm, const double* __restrict__ alpha, Tiling tl, long Vh,
                             int L5, int N, const int* __restrict__ active, double* __restrict__ partials) {
  using T = typename StoreTraits<S>::T;
  using TX = typename StoreTraits<SX>::T;
  Unit x = unit_of(tl, Vh, L5, N);
  double n2 = 0.0;
  if (x.valid && (!active || active[x.r])) {
    const T a = (T)alpha[x.r];
    T pv[24], qv[24], rv[24];
    TX xv_[24];
    load24<S, T>(p, p_nrm, x.u, pv);
    load24<S, T>(q, q_nrm, x.u, qv);
    load24<S, T>(rho, rho_nrm, x.u, rv);
    XloLayout<SX>::load(xv, x, tl, xv_);
    n2 = (double)axpy_unit<TX, T>(a, pv, qv, rv, xv_);
    XloLayout<SX>::store(xv, x, tl, xv_);
    store24<S, T>(rho, rho_nrm, x.u, rv);
  }
  block_partial(n2, x, tl, L5, Vh, partials);
}

// p = r + beta_r p
template <typename S>
__global__ void k_xpay(const S* __restrict__ r, const float* __restrict__ r_nrm, S* __restrict__ p,
                       float* __restrict__ p_nrm, const double* __restrict__ beta, Tiling tl, long Vh, int L5, int N,
                       const int* __restrict__ active) {
  using T = typename StoreTraits<S>::T;
  Unit x = unit_of(tl, Vh, L5, N);
  if (!x.valid || (active && !active[x.r])) return;
  const T b = (T)beta[x.r];
  T rv[24], pv[24];
  load24<S, T>(r, r_nrm, x.u, rv);
  load24<S, T>(p, p_nrm, x.u, pv);
#pragma unroll
  for (int i = 0; i < 24; i++) pv[i] = rv[i] + b * pv[i];
  store24<S, T>(p, p_nrm, x.u, pv);
}

// xhi += xlo ; xlo = 0
template <typename SX>
__global__ void k_accum_xhi(double* __restrict__ xhi, SX* __restrict__ xlo, Tiling tl, long Vh, int L5, int N,
                            const int* __restrict__ mask) {
  using TX = typename StoreTraits<SX>::T;
  Unit x = unit_of(tl, Vh, L5, N);
  if (!x.valid || (mask && !mask[x.r])) return;
  double h[24];
  TX l[24];
  load24<double, double>(xhi, nullptr, x.u, h);
  XloLayout<SX>::load(xlo, x, tl, l);
#pragma unroll
  for (int i = 0; i < 24; i++) { h[i] += (double)l[i]; l[i] = 0; }
  store24<double, double>(xhi, nullptr, x.u, h);
  XloLayout<SX>::store(xlo, x, tl, l);
}

// x_lo = 0 for the slots in mask (x_lo in the accumulator layout)
template <typename SX>
__global__ void k_zero_xlo(SX* __restrict__ xlo, Tiling tl, long Vh, int L5, int N, const int* __restrict__ mask) {
  Unit x = unit_of(tl, Vh, L5, N);
  if (!x.valid || !mask[x.r]) return;
  SX z[24];
#pragma unroll
  for (int i = 0; i < 24; i++) z[i] = 0;
  XloLayout<SX>::store(xlo, x, tl, z);
}

template <typename S>
__global__ void k_norm2(const S* __restrict__ v, const float* __restrict__ v_nrm, Tiling tl, long Vh, int L5, int N,
                        const int* __restrict__ mask, double* __restrict__ partials) {
  using T = typename StoreTraits<S>::T;
  Unit x = unit_of(tl, Vh, L5, N);
  double n2 = 0.0;
  if (x.valid && (!mask || mask[x.r])) {
    T a[24];
    load24<S, T>(v, v_nrm, x.u, a);
    T n2t = 0;
#pragma unroll
    for (int i = 0; i < 24; i++) n2t += a[i] * a[i];
    n2 = (double)n2t;
  }
  block_partial(n2, x, tl, L5, Vh, partials);
}

// out[r] = sum_h partials[r][h] in a fixed order that depends on nsites only: a
// cluster of kFinCluster blocks per slot, block c summing the c-th contiguous
// chunk (thread t takes sites t, t+256, ... of it, then a fixed tree), and block
// 0 adding the blocks' sums in rank order through distributed shared memory.
// Spreading a slot over several SMs matters on a part with few FP64 adders per SM.
constexpr int kFinCluster = 8;
__global__ void __cluster_dims__(kFinCluster, 1, 1) __launch_bounds__(256)
    k_finalize(const double* __restrict__ partials, long nsites, double* __restrict__ out) {
  namespace cg = cooperative_groups;
  __shared__ double sh[256];
  cg::cluster_group cluster = cg::this_cluster();
  const int r = blockIdx.y;
  const int c = (int)cluster.block_rank();
  const long len = (nsites + kFinCluster - 1) / kFinCluster;
  const long beg = (long)c * len;
  const long end = beg + len < nsites ? beg + len : nsites;
  const double* p = partials + (long)r * nsites;
  double s = 0.0;
  for (long k = beg + threadIdx.x; k < end; k += blockDim.x) s += p[k];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  cluster.sync();
  if (c == 0 && threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < kFinCluster; q++) tot += *cluster.map_shared_rank(&sh[0], q);
    out[r] = tot;
  }
  cluster.sync();   // every block's sum stays readable until block 0 has added it
}

// u = B x on one parity: P_+ half b5 x_s + c5 x_{s-1}, P_- half b5 x_s + c5 x_{s+1},
// with x_{-1} = -m x_{L5-1} and x_{L5} = -m x_0.
template <typename S>
__global__ void k_bop(const S* __restrict__ xv, const float* __restrict__ x_nrm, S* __restrict__ uv,
                      float* __restrict__ u_nrm, Fifth<typename StoreTraits<S>::T> f, Tiling tl, long Vh, int L5, int N,
                      const int* __restrict__ mask) {
  using T = typename StoreTraits<S>::T;
  Unit x = unit_of(tl, Vh, L5, N);
  if (!x.valid || (mask && !mask[x.r])) return;
  const T m = f.mass[x.r];
  const int s_dn = x.s == 0 ? L5 - 1 : x.s - 1, s_up = x.s == L5 - 1 ? 0 : x.s + 1;
  const T w_dn = x.s == 0 ? -m : T(1), w_up = x.s == L5 - 1 ? -m : T(1);
  T y[24], up[12], lo[12];
  load24<S, T>(xv, x_nrm, x.u, y);
  load_part<S, T>(xv, x_nrm, (x.h * L5 + s_dn) * N + x.r, 0, up);
  load_part<S, T>(xv, x_nrm, (x.h * L5 + s_up) * N + x.r, 1, lo);
#pragma unroll
  for (int i = 0; i < 12; i++) y[i] = f.b5 * y[i] + f.c5 * w_dn * up[i];
#pragma unroll
  for (int i = 0; i < 12; i++) y[12 + i] = f.b5 * y[12 + i] + f.c5 * w_up * lo[i];
  store24<S, T>(uv, u_nrm, x.u, y);
}

// p = r + beta_r p, then u = B p (the new p of the neighbouring slices comes from
// shared memory: a block holds every slice of its sites).
template <typename S>
__global__ void k_xpay_b(const S* __restrict__ r, const float* __restrict__ r_nrm, S* __restrict__ p,
                         float* __restrict__ p_nrm, S* __restrict__ uv, float* __restrict__ u_nrm,
                         const double* __restrict__ beta, Fifth<typename StoreTraits<S>::T> f, Tiling tl, long Vh,
                         int L5, int N, const int* __restrict__ active) {
  using T = typename StoreTraits<S>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sP = reinterpret_cast<T*>(smem_raw);
  Unit x = unit_of(tl, Vh, L5, N);
  const bool act = x.valid && (!active || active[x.r]);
  T pv[24];
#pragma unroll
  for (int i = 0; i < 24; i++) pv[i] = 0;
  if (act) {
    const T b = (T)beta[x.r];
    T rv[24];
    load24<S, T>(r, r_nrm, x.u, rv);
    load24<S, T>(p, p_nrm, x.u, pv);
#pragma unroll
    for (int i = 0; i < 24; i++) pv[i] = rv[i] + b * pv[i];
    store24<S, T>(p, p_nrm, x.u, pv);
  }
#pragma unroll
  for (int i = 0; i < 24; i++) sP[threadIdx.x * 25 + i] = pv[i];
  __syncthreads();
  if (!act) return;
  const T m = f.mass[x.r];
  const int s_dn = x.s == 0 ? L5 - 1 : x.s - 1, s_up = x.s == L5 - 1 ? 0 : x.s + 1;
  const T w_dn = x.s == 0 ? -m : T(1), w_up = x.s == L5 - 1 ? -m : T(1);
  const T* nd = sP + (size_t)((x.site_l * L5 + s_dn) * tl.rt + x.r_l) * 25;
  const T* nu = sP + (size_t)((x.site_l * L5 + s_up) * tl.rt + x.r_l) * 25;
  T y[24];
#pragma unroll
  for (int i = 0; i < 12; i++) y[i] = f.b5 * pv[i] + f.c5 * w_dn * nd[i];
#pragma unroll
  for (int i = 12; i < 24; i++) y[i] = f.b5 * pv[i] + f.c5 * w_up * nu[i];
  store24<S, T>(uv, u_nrm, x.u, y);
}

// Zero the units of the slots in mask.
template <typename S>
__global__ void k_zero_masked(S* __restrict__ v, float* __restrict__ nrm, Tiling tl, long Vh, int L5, int N,
                              const int* __restrict__ mask) {
  using T = typename StoreTraits<S>::T;
  Unit x = unit_of(tl, Vh, L5, N);
  if (!x.valid || !mask[x.r]) return;
  T z[24];
#pragma unroll
  for (int i = 0; i < 24; i++) z[i] = 0;
  store24<S, T>(v, nrm, x.u, z);
}

// Wall source of a 4D field (API layout): slice 0 gets the P_+ spins (0, 1),
// slice L5-1 the P_- spins (2, 3); the other slices must already be zero.
__global__ void k_walls(const double* __restrict__ eta, double* __restrict__ w, long V, int L5) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V * 24) return;
  const int k = (int)(i % 24);
  const int spin = k / 6;
  if (spin < 2) w[i] = eta[i];
  else w[(long)(L5 - 1) * V * 24 + i] = eta[i];
}

// Z2 noise source: complex element k of a 4D field ([t][z][y][x][spin][colour],
// k = 0 .. 12V-1) is (+1, 0) or (-1, 0) by the top bit of the k-th output of
// SplitMix64 from state `seed` (Steele, Lea and Flood, OOPSLA 2014): the state
// advances by the 64-bit golden-ratio increment and each output is the state
// passed through the 64-bit mixing finaliser of that generator.
__global__ void k_z2(unsigned long long seed, double* __restrict__ eta, long n) {
  long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  unsigned long long z = seed + (unsigned long long)(k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  eta[2 * k] = (z >> 63) ? -1.0 : 1.0;
  eta[2 * k + 1] = 0.0;
}

// One step of gauge-covariant Gaussian source smearing on a 4D field (the sources
// of the paper's propagators, Sec. VII):
//   out(x) = in(x) + k sum_{i = x,y,z} [U_i(x) in(x+i) + U_i(x-i)^+ in(x-i) - 2 in(x)],
// spin-diagonal, no hop in time.  in / out: C ABI layout [t][z][y][x][spin][colour];
// U: the context's FP64 links [parity][h][mu][18], h = lex / 2.
__global__ void k_smear_step(const double* __restrict__ U, const double* __restrict__ in, double* __restrict__ out,
                             Geom g, double k) {
  const long lex = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (lex >= g.V) return;
  int c[4];
  long r = lex;
  for (int i = 0; i < 4; i++) { c[i] = (int)(r % g.L[i]); r /= g.L[i]; }
  const double* me = in + lex * 24;
  double acc[24];
  for (int i = 0; i < 24; i++) acc[i] = (1.0 - 6.0 * k) * me[i];
  long stride = 1;
  for (int mu = 0; mu < 3; mu++) {
    const int Lm = g.L[mu];
    const long fw = c[mu] == Lm - 1 ? lex - (long)(Lm - 1) * stride : lex + stride;
    const long bw = c[mu] == 0 ? lex + (long)(Lm - 1) * stride : lex - stride;
    const int pf = (c[0] + c[1] + c[2] + c[3]) & 1;
    const double* uf = U + (((long)pf * g.Vh + (lex >> 1)) * 4 + mu) * 18;            // U_mu(x)
    const double* ub = U + (((long)(1 - pf) * g.Vh + (bw >> 1)) * 4 + mu) * 18;       // U_mu(x - mu)
    const double* pf_in = in + fw * 24;
    const double* pb_in = in + bw * 24;
    for (int sp = 0; sp < 4; sp++)
      for (int a = 0; a < 3; a++) {
        double re = 0.0, im = 0.0;
        for (int b = 0; b < 3; b++) {
          const double fr = uf[2 * (3 * a + b)], fi = uf[2 * (3 * a + b) + 1];      // U_ab
          const double vr = pf_in[6 * sp + 2 * b], vi = pf_in[6 * sp + 2 * b + 1];
          re += fr * vr - fi * vi;
          im += fr * vi + fi * vr;
          const double br = ub[2 * (3 * b + a)], bi = -ub[2 * (3 * b + a) + 1];     // (U^+)_ab = conj(U_ba)
          const double wr = pb_in[6 * sp + 2 * b], wi = pb_in[6 * sp + 2 * b + 1];
          re += br * wr - bi * wi;
          im += br * wi + bi * wr;
        }
        acc[6 * sp + 2 * a] += k * re;
        acc[6 * sp + 2 * a + 1] += k * im;
      }
    stride *= Lm;
  }
  for (int i = 0; i < 24; i++) out[lex * 24 + i] = acc[i];
}

// Residual-mass correlators (Eq. mres of arXiv:1701.07559): per 4D site, summed
// over the n solutions (spin-colour sources), the squared norms of the wall field
// q = P_- x_0 + P_+ x_{L5-1} and of the midpoint field Q = P_+ x_{L5/2-1} + P_- x_{L5/2};
// P_+ keeps spins 0, 1 and P_- spins 2, 3 (gamma_5 = diag(1, 1, -1, -1)).  FP64,
// solutions in the C ABI 5D layout.
__global__ void k_mres_sites(const double* const* __restrict__ xs, int n, long V, int L5, double* pp, double* j5) {
  const long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= V) return;
  const int sm = L5 / 2;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < n; k++) {
    const double* f = xs[k];
    const double* w0 = f + (x) * 24;                          // s = 0
    const double* wl = f + ((long)(L5 - 1) * V + x) * 24;     // s = L5 - 1
    const double* m0 = f + ((long)(sm - 1) * V + x) * 24;     // s = L5/2 - 1
    const double* m1 = f + ((long)sm * V + x) * 24;           // s = L5/2
    for (int i = 0; i < 12; i++) {                            // spins 0, 1: (re, im) x 3 colours x 2
      a += wl[i] * wl[i];
      b += m0[i] * m0[i];
    }
    for (int i = 12; i < 24; i++) {                           // spins 2, 3
      a += w0[i] * w0[i];
      b += m1[i] * m1[i];
    }
  }
  pp[x] = a;
  j5[x] = b;
}

// Per time slice, fixed-order sums of the site values (one block per slice).
__global__ void k_slice_sum(const double* __restrict__ v, long slice, double* out) {
  __shared__ double sh[256];
  const double* p = v + (long)blockIdx.x * slice;
  double s = 0.0;
  for (long i = threadIdx.x; i < slice; i += 256) s += p[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// rho = S(bhat - q) with bhat in FP64 and q in FP32 (the residual of a reliable
// update computed with FP32 arithmetic); partial |bhat - q|^2 in FP64.
template <typename S>
__global__ void k_resid_update(const double* __restrict__ bhat, const float* __restrict__ q, S* __restrict__ rho,
                               float* __restrict__ rho_nrm, Tiling tl, long Vh, int L5, int N,
                               const int* __restrict__ mask, double* __restrict__ partials) {
  using T = typename StoreTraits<S>::T;
  Unit x = unit_of(tl, Vh, L5, N);
  double n2 = 0.0;
  if (x.valid && (!mask || mask[x.r])) {
    double b[24];
    float qv[24];
    load24<double, double>(bhat, nullptr, x.u, b);
    load24<float, float>(q, nullptr, x.u, qv);
    T o[24];
#pragma unroll
    for (int i = 0; i < 24; i++) {
      double v = b[i] - (double)qv[i];
      n2 += v * v;
      o[i] = (T)v;
    }
    store24<S, T>(rho, rho_nrm, x.u, o);
  }
  block_partial(n2, x, tl, L5, Vh, partials);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline dim3 tile_grid(const Tiling& t) { return dim3((unsigned)t.ntiles, (unsigned)t.ngroups); }

template <typename S>
cudaError_t pack_rhs(const double* api, S* out, float* out_nrm, const Geom& g, int L5, int N, int par, int r,
                     cudaStream_t st) {
  long n = g.Vh * L5;
  k_pack<S><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(api, out, out_nrm, g, L5, N, par, r);
  return cudaGetLastError();
}

template <typename S>
cudaError_t unpack_rhs(const S* in, const float* in_nrm, double* api, const Geom& g, int L5, int N, int par, int r,
                       cudaStream_t st) {
  long n = g.Vh * L5;
  k_unpack<S><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, in_nrm, api, g, L5, N, par, r);
  return cudaGetLastError();
}

template <typename Si, typename So>
cudaError_t convert(const Si* in, const float* in_nrm, So* out, float* out_nrm, const Tiling& t, long Vh, int L5,
                    int N, const int* mask, cudaStream_t st) {
  k_convert<Si, So><<<tile_grid(t), t.threads, 0, st>>>(in, in_nrm, out, out_nrm, t, Vh, L5, N, mask);
  return cudaGetLastError();
}

template <typename SX, typename S>
cudaError_t axpy_x_rho(SX* x, const S* p, const float* p_nrm, S* rho, float* rho_nrm, const S* q, const float* q_nrm,
                       const double* alpha, const Tiling& t, long Vh, int L5, int N, const int* active,
                       double* partials, cudaStream_t st) {
  k_axpy_x_rho<SX, S><<<tile_grid(t), t.threads, 0, st>>>(x, p, p_nrm, rho, rho_nrm, q, q_nrm, alpha, t, Vh, L5, N,
                                                           active, partials);
  return cudaGetLastError();
}

template <typename S>
cudaError_t xpay(const S* r, const float* r_nrm, S* p, float* p_nrm, const double* beta, const Tiling& t, long Vh,
                 int L5, int N, const int* active, cudaStream_t st) {
  k_xpay<S><<<tile_grid(t), t.threads, 0, st>>>(r, r_nrm, p, p_nrm, beta, t, Vh, L5, N, active);
  return cudaGetLastError();
}

template <typename SX>
cudaError_t accum_xhi(double* xhi, SX* xlo, const Tiling& t, long Vh, int L5, int N, const int* mask,
                      cudaStream_t st) {
  k_accum_xhi<SX><<<tile_grid(t), t.threads, 0, st>>>(xhi, xlo, t, Vh, L5, N, mask);
  return cudaGetLastError();
}

template <typename SX>
cudaError_t zero_xlo(SX* xlo, const Tiling& t, long Vh, int L5, int N, const int* mask, cudaStream_t st) {
  k_zero_xlo<SX><<<tile_grid(t), t.threads, 0, st>>>(xlo, t, Vh, L5, N, mask);
  return cudaGetLastError();
}

long xlo_units(const Tiling& t, long units, bool tile_major) {
  return tile_major ? t.ntiles * (long)t.ngroups * t.threads : units;
}

template <typename S>
cudaError_t norm2_partials(const S* v, const float* v_nrm, const Tiling& t, long Vh, int L5, int N, const int* mask,
                           double* partials, cudaStream_t st) {
  k_norm2<S><<<tile_grid(t), t.threads, 0, st>>>(v, v_nrm, t, Vh, L5, N, mask, partials);
  return cudaGetLastError();
}

template <typename S>
cudaError_t bop(const S* x, const float* x_nrm, S* u, float* u_nrm, const Fifth<typename StoreTraits<S>::T>& f,
                const Tiling& t, long Vh, int L5, int N, const int* mask, cudaStream_t st) {
  k_bop<S><<<tile_grid(t), t.threads, 0, st>>>(x, x_nrm, u, u_nrm, f, t, Vh, L5, N, mask);
  return cudaGetLastError();
}

template <typename S>
cudaError_t xpay_b(const S* r, const float* r_nrm, S* p, float* p_nrm, S* u, float* u_nrm, const double* beta,
                   const Fifth<typename StoreTraits<S>::T>& f, const Tiling& t, long Vh, int L5, int N,
                   const int* active, cudaStream_t st) {
  using T = typename StoreTraits<S>::T;
  size_t smem = (size_t)t.threads * 25 * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_xpay_b<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_xpay_b<S><<<tile_grid(t), t.threads, smem, st>>>(r, r_nrm, p, p_nrm, u, u_nrm, beta, f, t, Vh, L5, N, active);
  return cudaGetLastError();
}

template <typename S>
cudaError_t resid_update(const double* bhat, const float* q, S* rho, float* rho_nrm, const Tiling& t, long Vh, int L5,
                         int N, const int* mask, double* partials, cudaStream_t st) {
  k_resid_update<S><<<tile_grid(t), t.threads, 0, st>>>(bhat, q, rho, rho_nrm, t, Vh, L5, N, mask, partials);
  return cudaGetLastError();
}

template <typename S>
cudaError_t zero_masked(S* v, float* nrm, const Tiling& t, long Vh, int L5, int N, const int* mask, cudaStream_t st) {
  k_zero_masked<S><<<tile_grid(t), t.threads, 0, st>>>(v, nrm, t, Vh, L5, N, mask);
  return cudaGetLastError();
}

cudaError_t walls(const double* eta, double* w, long V, int L5, cudaStream_t st) {
  long n = V * 24;
  k_walls<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(eta, w, V, L5);
  return cudaGetLastError();
}

cudaError_t z2_source(unsigned long long seed, double* eta, long V, cudaStream_t st) {
  const long n = V * 12;
  k_z2<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(seed, eta, n);
  return cudaGetLastError();
}

cudaError_t smear_step(const double* U, const double* in, double* out, const Geom& g, double k, cudaStream_t st) {
  k_smear_step<<<(unsigned)((g.V + 127) / 128), 128, 0, st>>>(U, in, out, g, k);
  return cudaGetLastError();
}

cudaError_t mres_correlators(const double* const* xs, int n, long V, int Lt, int L5, double* pp, double* j5,
                             double* c_pp, double* c_j5, cudaStream_t st) {
  k_mres_sites<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(xs, n, V, L5, pp, j5);
  k_slice_sum<<<Lt, 256, 0, st>>>(pp, V / Lt, c_pp);
  k_slice_sum<<<Lt, 256, 0, st>>>(j5, V / Lt, c_j5);
  return cudaGetLastError();
}

cudaError_t finalize(const double* partials, long ntiles, int N, double* out, cudaStream_t st) {
  k_finalize<<<dim3(kFinCluster, (unsigned)N), 256, 0, st>>>(partials, ntiles, out);
  return cudaGetLastError();
}

#define MDWF_INST_S(S)                                                                                          \
  template cudaError_t pack_rhs<S>(const double*, S*, float*, const Geom&, int, int, int, int, cudaStream_t);   \
  template cudaError_t unpack_rhs<S>(const S*, const float*, double*, const Geom&, int, int, int, int,          \
                                     cudaStream_t);                                                             \
  template cudaError_t xpay<S>(const S*, const float*, S*, float*, const double*, const Tiling&, long, int, int, \
                               const int*, cudaStream_t);                                                       \
  template cudaError_t norm2_partials<S>(const S*, const float*, const Tiling&, long, int, int, const int*,      \
                                         double*, cudaStream_t);

#define MDWF_INST_B(S)                                                                                           \
  template cudaError_t bop<S>(const S*, const float*, S*, float*, const Fifth<StoreTraits<S>::T>&, const Tiling&,  \
                              long, int, int, const int*, cudaStream_t);                                          \
  template cudaError_t xpay_b<S>(const S*, const float*, S*, float*, S*, float*, const double*,                    \
                                 const Fifth<StoreTraits<S>::T>&, const Tiling&, long, int, int, const int*,        \
                                 cudaStream_t);                                                                    \
  template cudaError_t resid_update<S>(const double*, const float*, S*, float*, const Tiling&, long, int, int,      \
                                       const int*, double*, cudaStream_t);
template cudaError_t zero_masked<double>(double*, float*, const Tiling&, long, int, int, const int*, cudaStream_t);
template cudaError_t zero_masked<float>(float*, float*, const Tiling&, long, int, int, const int*, cudaStream_t);
template cudaError_t zero_masked<__half>(__half*, float*, const Tiling&, long, int, int, const int*, cudaStream_t);
template cudaError_t zero_masked<__nv_bfloat16>(__nv_bfloat16*, float*, const Tiling&, long, int, int, const int*,
                                                cudaStream_t);

MDWF_INST_B(double)
MDWF_INST_B(float)
MDWF_INST_B(__half)
MDWF_INST_B(__nv_bfloat16)

MDWF_INST_S(double)
MDWF_INST_S(float)
MDWF_INST_S(__half)
MDWF_INST_S(__nv_bfloat16)

#define MDWF_INST_CONV(A, B)                                                                                  \
  template cudaError_t convert<A, B>(const A*, const float*, B*, float*, const Tiling&, long, int, int,       \
                                     const int*, cudaStream_t);
MDWF_INST_CONV(double, float)
MDWF_INST_CONV(double, __half)
MDWF_INST_CONV(double, __nv_bfloat16)
MDWF_INST_CONV(double, double)

#define MDWF_INST_AXPY(SX, S)                                                                                    \
  template cudaError_t axpy_x_rho<SX, S>(SX*, const S*, const float*, S*, float*, const S*, const float*,        \
                                         const double*, const Tiling&, long, int, int, const int*, double*,      \
                                         cudaStream_t);
MDWF_INST_AXPY(double, double)
MDWF_INST_AXPY(float, float)
MDWF_INST_AXPY(float, __half)
MDWF_INST_AXPY(float, __nv_bfloat16)

template cudaError_t accum_xhi<double>(double*, double*, const Tiling&, long, int, int, const int*, cudaStream_t);
template cudaError_t accum_xhi<float>(double*, float*, const Tiling&, long, int, int, const int*, cudaStream_t);
template cudaError_t zero_xlo<double>(double*, const Tiling&, long, int, int, const int*, cudaStream_t);
template cudaError_t zero_xlo<float>(float*, const Tiling&, long, int, int, const int*, cudaStream_t);

}  // namespace mdwf
