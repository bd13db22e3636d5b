// Wilson hop on all L5 slices x RHS slots with the structured fifth-dimension
// epilogues of the even-odd Moebius operator (the solver's hot path).
//
// With A = alpha + beta P and B = b5 + c5 P (Sec. II of arXiv:1701.07559 and
// the Brower-Neff-Orginos 5D form), P moves the P_+ half (spins 0,1) one slice
// down and the P_- half one slice up, with a -m_f factor across the wall.  On
// each chirality A and B are bidiagonal, and A^-1 follows from a first-order
// recursion along s plus one wall correction:
//   P_+ half:  z_s = x_s / alpha - kappa z_{s-1},  y_{L5-1} = z_{L5-1} / (1 + m (-kappa)^L5),
//              y_s = z_s - m (-kappa)^{s+1} y_{L5-1}                      (kappa = beta / alpha)
//   P_- half:  the same with s -> L5-1-s.
// Adjoints exchange the two shift directions.  The epilogues:
//   E_RAW        out = add + kappa H(in)
//   E_BAINV      out = B A^-1 (kappa H(in))                     Mhat, first hop
//   E_AINVD_BD   out = A^-+ B^+ (kappa H(in))                   Mhat^+, first hop
//   E_A_SAME     out = add + g A same + kappa H(in)             Mhat, second hop; D; residuals
//   E_AD_SAME_BD out = add + g A^+ same + kappa B^+ H(in)       Mhat^+, second hop; D^+
//   E_AINV_SAME  out = A^-1 (same + kappa H(in))                odd-site reconstruction
// The recursions run over columns (site, RHS, spin-colour component) of a
// shared-memory tile that holds every slice of the block's sites.
//
// Thread block: (rt RHS slots) x (L5 slices) x (nsb sites); a site's units
// (s, r) are contiguous in memory, so the block's loads of one neighbour site
// are one contiguous run.  Two variants of the hop: direct loads, or the eight
// neighbour sites of every site staged into shared memory by bulk asynchronous
// copies (cp.async.bulk + one mbarrier per direction) issued at block start.
#include "mdwf_internal.h"

namespace mdwf {

namespace {

template <typename T, bool DAG>
__device__ __forceinline__ void su3_mul(const T* __restrict__ l, const T* v, T* o) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    T re = 0, im = 0;
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const int k = DAG ? (3 * b + a) : (3 * a + b);
      const T ur = l[2 * k];
      const T ui = DAG ? -l[2 * k + 1] : l[2 * k + 1];
      re += ur * v[2 * b] - ui * v[2 * b + 1];
      im += ur * v[2 * b + 1] + ui * v[2 * b];
    }
    o[2 * a] = re;
    o[2 * a + 1] = im;
  }
}

// Spin projection (1 + sg g_mu) psi -> h (two colour vectors), DeGrand-Rossi
// basis: h = psi_up + sg e_mu psi_lo with e_x = i sigma_x, e_y = -i sigma_y,
// e_z = i sigma_z, e_t = 1.  The lower half of the projected spinor is
// sg e_mu^+ h, restored after the colour multiply.
template <int MU, typename T>
__device__ __forceinline__ void project(const T* p, T sg, T* h) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const T* p0 = p + 2 * c;
    const T* p1 = p + 6 + 2 * c;
    const T* p2 = p + 12 + 2 * c;
    const T* p3 = p + 18 + 2 * c;
    T* h0 = h + 2 * c;
    T* h1 = h + 6 + 2 * c;
    if (MU == 0) {
      h0[0] = p0[0] - sg * p3[1]; h0[1] = p0[1] + sg * p3[0];
      h1[0] = p1[0] - sg * p2[1]; h1[1] = p1[1] + sg * p2[0];
    } else if (MU == 1) {
      h0[0] = p0[0] - sg * p3[0]; h0[1] = p0[1] - sg * p3[1];
      h1[0] = p1[0] + sg * p2[0]; h1[1] = p1[1] + sg * p2[1];
    } else if (MU == 2) {
      h0[0] = p0[0] - sg * p2[1]; h0[1] = p0[1] + sg * p2[0];
      h1[0] = p1[0] + sg * p3[1]; h1[1] = p1[1] - sg * p3[0];
    } else {
      h0[0] = p0[0] + sg * p2[0]; h0[1] = p0[1] + sg * p2[1];
      h1[0] = p1[0] + sg * p3[0]; h1[1] = p1[1] + sg * p3[1];
    }
  }
}

// fp16: project the packed (scaled) values with half2 arithmetic, then unpack and scale.
template <int MU>
__device__ __forceinline__ void project_half(const uint4 q[3], float s, float sg, float* h) {
  const __half2* w = reinterpret_cast<const __half2*>(q);   // w[4 * colour + spin] (colour-major storage)
  const __half2 pp = __floats2half2_rn(sg, sg);
  const __half2 mp = __floats2half2_rn(-sg, sg);             // times swapped z: sg * i * z
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const __half2 p0 = w[4 * c], p1 = w[4 * c + 1], p2 = w[4 * c + 2], p3 = w[4 * c + 3];
    __half2 h0, h1;
    if (MU == 0) {
      h0 = __hfma2(__lowhigh2highlow(p3), mp, p0);
      h1 = __hfma2(__lowhigh2highlow(p2), mp, p1);
    } else if (MU == 1) {
      h0 = __hfma2(p3, __hneg2(pp), p0);
      h1 = __hfma2(p2, pp, p1);
    } else if (MU == 2) {
      h0 = __hfma2(__lowhigh2highlow(p2), mp, p0);
      h1 = __hfma2(__lowhigh2highlow(p3), __hneg2(mp), p1);
    } else {
      h0 = __hfma2(p2, pp, p0);
      h1 = __hfma2(p3, pp, p1);
    }
    const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
    h[2 * c] = f0.x * s; h[2 * c + 1] = f0.y * s;
    h[6 + 2 * c] = f1.x * s; h[6 + 2 * c + 1] = f1.y * s;
  }
}

// Load (global memory or shared memory) and project one neighbour spinor.
template <int MU, typename S, typename T>
struct Proj {
  static __device__ __forceinline__ void global(const S* __restrict__ v, const float* __restrict__ nrm, long u, T sg,
                                                T* h) {
    T psi[24];
    load24<S, T>(v, nrm, u, psi);
    project<MU, T>(psi, sg, h);
  }
  static __device__ __forceinline__ void shared(const S* sp, float nrm, T sg, T* h) {
    T psi[24];
    load24_smem<S, T>(sp, psi);
    if (StoreTraits<S>::kNorm) {
#pragma unroll
      for (int i = 0; i < 24; i++) psi[i] *= (T)nrm;
    }
    project<MU, T>(psi, sg, h);
  }
};
template <int MU>
struct Proj<MU, __half, float> {
  static __device__ __forceinline__ void global(const __half* __restrict__ v, const float* __restrict__ nrm, long u,
                                                float sg, float* h) {
    const uint4* p = reinterpret_cast<const uint4*>(v + 24 * u);
    uint4 q[3];
    q[0] = __ldg(p);
    q[1] = __ldg(p + 1);
    q[2] = __ldg(p + 2);
    project_half<MU>(q, __ldg(nrm + u), sg, h);
  }
  static __device__ __forceinline__ void shared(const __half* sp, float nrm, float sg, float* h) {
    const uint4* p = reinterpret_cast<const uint4*>(sp);
    uint4 q[3];
    q[0] = p[0];
    q[1] = p[1];
    q[2] = p[2];
    project_half<MU>(q, nrm, sg, h);
  }
};

template <int MU, typename T>
__device__ __forceinline__ void reconstruct(const T* chi, T sg, T* acc) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const T* x0 = chi + 2 * c;
    const T* x1 = chi + 6 + 2 * c;
    T* a0 = acc + 2 * c;
    T* a1 = acc + 6 + 2 * c;
    T* a2 = acc + 12 + 2 * c;
    T* a3 = acc + 18 + 2 * c;
    a0[0] += x0[0]; a0[1] += x0[1];
    a1[0] += x1[0]; a1[1] += x1[1];
    if (MU == 0) {
      a2[0] += sg * x1[1]; a2[1] -= sg * x1[0];
      a3[0] += sg * x0[1]; a3[1] -= sg * x0[0];
    } else if (MU == 1) {
      a2[0] += sg * x1[0]; a2[1] += sg * x1[1];
      a3[0] -= sg * x0[0]; a3[1] -= sg * x0[1];
    } else if (MU == 2) {
      a2[0] += sg * x0[1]; a2[1] -= sg * x0[0];
      a3[0] -= sg * x1[1]; a3[1] += sg * x1[0];
    } else {
      a2[0] += sg * x0[0]; a2[1] += sg * x0[1];
      a3[0] += sg * x1[0]; a3[1] += sg * x1[1];
    }
  }
}

// Site of the thread: coordinates, lexicographic index, strides of the four directions.
struct Site {
  int c[4];
  int lex;
  int stride[4];
};

__device__ __forceinline__ Site make_site(const Geom& g, int par, long h) {
  Site x;
  site_coords(g, par, h, x.c);
  x.stride[0] = 1;
  x.stride[1] = g.L[0];
  x.stride[2] = g.L[0] * g.L[1];
  x.stride[3] = g.L[0] * g.L[1] * g.L[2];
  x.lex = x.c[0] + x.stride[1] * x.c[1] + x.stride[2] * x.c[2] + x.stride[3] * x.c[3];
  return x;
}

// Half-lattice index of the neighbour in direction MU, forward or backward.
template <int MU, bool FWD>
__device__ __forceinline__ int nbr_half(const Geom& g, const Site& x) {
  const int st = x.stride[MU];
  const int wrap = (g.L[MU] - 1) * st;
  int n;
  if (FWD) n = (x.c[MU] == g.L[MU] - 1) ? x.lex - wrap : x.lex + st;
  else n = (x.c[MU] == 0) ? x.lex + wrap : x.lex - st;
  return n >> 1;
}

// One of the eight hopping terms; the neighbour spinor comes either from global
// memory (sp == nullptr) or from the shared staging buffer sp.
template <int MU, bool FWD, typename S, typename T>
__device__ __forceinline__ void hop_term(const FastArgs<S, T>& a, const Site& x, long h, int s, int r, const S* sp,
                                         float snrm, T* acc) {
  const int hn = nbr_half<MU, FWD>(a.g, x);
  const T sg = (a.dagger ? T(1) : T(-1)) * (FWD ? T(1) : T(-1));
  T hh[12], chi[12], l[18];
  if (sp == nullptr) Proj<MU, S, T>::global(a.in, a.in_nrm, ((long)hn * a.L5 + s) * a.N + r, sg, hh);
  else Proj<MU, S, T>::shared(sp, snrm, sg, hh);
  if (MU == 3 && a.antiperiodic && (FWD ? x.c[3] == a.g.L[3] - 1 : x.c[3] == 0)) {
#pragma unroll
    for (int i = 0; i < 12; i++) hh[i] = -hh[i];
  }
  if (FWD) {
    load_link<T>(a.U, ((long)a.out_par * a.g.Vh + h) * 4 + MU, l);
    su3_mul<T, false>(l, hh, chi);
    su3_mul<T, false>(l, hh + 6, chi + 6);
  } else {
    load_link<T>(a.U, ((long)(1 - a.out_par) * a.g.Vh + hn) * 4 + MU, l);
    su3_mul<T, true>(l, hh, chi);
    su3_mul<T, true>(l, hh + 6, chi + 6);
  }
  reconstruct<MU, T>(chi, sg, acc);
}

// A (dag = false) or A^+ (dag = true) of the stored field `same` at (h, s, r):
//   P_+ half: alpha y_s + beta y_{s-1} (A) or alpha y_s + beta y_{s+1} (A^+)
//   P_- half: alpha y_s + beta y_{s+1} (A) or alpha y_s + beta y_{s-1} (A^+)
// with y_{-1} = -m y_{L5-1}, y_{L5} = -m y_0.
template <typename S, typename T>
__device__ __forceinline__ void apply_A(const FastArgs<S, T>& a, long h, int s, int r, bool dag, T m, T* o) {
  const int L5 = a.L5;
  T y[24], up[12], lo[12];
  load24<S, T>(a.same, a.same_nrm, (h * L5 + s) * a.N + r, y);
  const int s_dn = s == 0 ? L5 - 1 : s - 1;
  const int s_up = s == L5 - 1 ? 0 : s + 1;
  const T w_dn = s == 0 ? -m : T(1);
  const T w_up = s == L5 - 1 ? -m : T(1);
  const int su = dag ? s_up : s_dn, sl = dag ? s_dn : s_up;
  const T wu = dag ? w_up : w_dn, wl = dag ? w_dn : w_up;
  load_part<S, T>(a.same, a.same_nrm, (h * L5 + su) * a.N + r, 0, up);
  load_part<S, T>(a.same, a.same_nrm, (h * L5 + sl) * a.N + r, 1, lo);
  const T al = a.f.alpha, bu = a.f.beta * wu, bl = a.f.beta * wl;
#pragma unroll
  for (int i = 0; i < 12; i++) o[i] = al * y[i] + bu * up[i];
#pragma unroll
  for (int i = 0; i < 12; i++) o[12 + i] = al * y[12 + i] + bl * lo[i];
}

// A strided shared-memory column, indexed along the recursion direction.
template <typename T>
struct Col {
  T* base;
  int step;
  __device__ __forceinline__ T& operator[](int k) const { return base[k * step]; }
};
template <typename T>
__device__ __forceinline__ Col<T> make_col(T* c, int st, int L5, bool down) {
  Col<T> r;
  r.base = down ? c : c + (L5 - 1) * st;
  r.step = down ? st : -st;
  return r;
}

// y = A^-1 x in place (A = alpha + beta S along the column, wall factor -m).
// Loads are issued four at a time ahead of the dependent recursion.
template <typename T>
__device__ __forceinline__ void col_ainv(Col<T> c, int L5, T inv_alpha, T kap, T m, T powL) {
  T z = 0;
  int k = 0;
  for (; k + 4 <= L5; k += 4) {
    T v0 = c[k], v1 = c[k + 1], v2 = c[k + 2], v3 = c[k + 3];
    z = v0 * inv_alpha - kap * z; v0 = z;
    z = v1 * inv_alpha - kap * z; v1 = z;
    z = v2 * inv_alpha - kap * z; v2 = z;
    z = v3 * inv_alpha - kap * z; v3 = z;
    c[k] = v0; c[k + 1] = v1; c[k + 2] = v2; c[k + 3] = v3;
  }
  for (; k < L5; k++) { z = c[k] * inv_alpha - kap * z; c[k] = z; }
  const T yl = z / (T(1) + m * powL);
  c[L5 - 1] = yl;
  // y_k = z_k - m (-kappa)^{k+1} y_{L5-1}
  const T mk = -kap;
  T w = m * yl * mk;
  k = 0;
  for (; k + 4 <= L5 - 1; k += 4) {
    T v0 = c[k], v1 = c[k + 1], v2 = c[k + 2], v3 = c[k + 3];
    v0 -= w; w *= mk;
    v1 -= w; w *= mk;
    v2 -= w; w *= mk;
    v3 -= w; w *= mk;
    c[k] = v0; c[k + 1] = v1; c[k + 2] = v2; c[k + 3] = v3;
  }
  for (; k < L5 - 1; k++) { c[k] -= w; w *= mk; }
}

// y = B x in place (B = b5 + c5 S along the column: y_k = b5 x_k + c5 x_{k-1}, x_{-1} = -m x_{L5-1}).
template <typename T>
__device__ __forceinline__ void col_bop(Col<T> c, int L5, T b5, T c5, T m) {
  T prev = -m * c[L5 - 1];
  int k = 0;
  for (; k + 4 <= L5; k += 4) {
    T v0 = c[k], v1 = c[k + 1], v2 = c[k + 2], v3 = c[k + 3];
    c[k] = b5 * v0 + c5 * prev;
    c[k + 1] = b5 * v1 + c5 * v0;
    c[k + 2] = b5 * v2 + c5 * v1;
    c[k + 3] = b5 * v3 + c5 * v2;
    prev = v3;
  }
  for (; k < L5; k++) { T v = c[k]; c[k] = b5 * v + c5 * prev; prev = v; }
}

constexpr int kPadF = 25;

// Thread coordinates of the (rt, L5, nsb) block.
struct Thr {
  int r_l, s, site_l, tid;
  long h;
  int r;
  bool valid, act;
  long u;
};

template <typename S, typename T>
__device__ __forceinline__ Thr thread_of(const FastArgs<S, T>& a, const Tiling& tl) {
  Thr t;
  t.r_l = threadIdx.x;
  t.s = threadIdx.y;
  t.site_l = threadIdx.z;
  t.tid = (t.site_l * a.L5 + t.s) * tl.rt + t.r_l;
  t.h = (long)blockIdx.x * tl.nsb + t.site_l;
  t.r = blockIdx.y * tl.rt + t.r_l;
  t.valid = (t.h < a.g.Vh) && (t.r < a.N);
  t.act = t.valid && (a.active == nullptr || a.active[t.r] != 0);
  t.u = (t.h * a.L5 + t.s) * a.N + t.r;
  return t;
}

// Epilogue shared by both hop variants: turns the hop sums acc into the output
// of the selected fifth-dimension form, stores it and forms the norm partials.
// sA: shared tile of (threads x kPadF) reals, also used for the partial sums.
template <typename S, typename T, int EPI>
__device__ __forceinline__ void epilogue(const FastArgs<S, T>& a, const Tiling& tl, const Thr& t, const T* acc,
                                         T* sA) {
  const int L5 = a.L5;
  const T m = t.valid ? a.f.mass[t.r] : T(0);
  T o[24];
  constexpr bool kCols = (EPI == E_BAINV || EPI == E_AINVD_BD || EPI == E_AINV_SAME);
  if (kCols || EPI == E_AD_SAME_BD) {
    T v[24];
#pragma unroll
    for (int i = 0; i < 24; i++) v[i] = a.kappa * acc[i];
    if (EPI == E_AINV_SAME && t.act) {
      T y[24];
      load24<S, T>(a.same, a.same_nrm, t.u, y);
#pragma unroll
      for (int i = 0; i < 24; i++) v[i] += y[i];
    }
#pragma unroll
    for (int i = 0; i < 24; i++) sA[t.tid * kPadF + i] = v[i];
    __syncthreads();
    if (kCols) {
      // thread (r_l, s, site_l) runs the columns comp = s, s + L5, ... of (site_l, r_l)
      if (t.act) {
        const int st = tl.rt * kPadF;
        T* base = sA + (size_t)(t.site_l * L5 * tl.rt + t.r_l) * kPadF;
        for (int comp = t.s; comp < 24; comp += L5) {
          const bool upper = comp < 12;
          if (EPI == E_BAINV) {
            Col<T> c = make_col<T>(base + comp, st, L5, upper);
            col_ainv<T>(c, L5, a.f.inv_alpha, a.f.kap, m, a.f.powL);
            col_bop<T>(c, L5, a.f.b5, a.f.c5, m);
          } else if (EPI == E_AINVD_BD) {
            Col<T> c = make_col<T>(base + comp, st, L5, !upper);
            col_bop<T>(c, L5, a.f.b5, a.f.c5, m);
            col_ainv<T>(c, L5, a.f.inv_alpha, a.f.kap, m, a.f.powL);
          } else {
            Col<T> c = make_col<T>(base + comp, st, L5, upper);
            col_ainv<T>(c, L5, a.f.inv_alpha, a.f.kap, m, a.f.powL);
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 24; i++) o[i] = sA[t.tid * kPadF + i];
    } else {
      // E_AD_SAME_BD: B^+ (kappa H) from this slice and its neighbour slice
      const int s_dn = t.s == 0 ? L5 - 1 : t.s - 1;
      const int s_up = t.s == L5 - 1 ? 0 : t.s + 1;
      const T w_dn = t.s == 0 ? -m : T(1);
      const T w_up = t.s == L5 - 1 ? -m : T(1);
      const T* me = sA + (size_t)t.tid * kPadF;
      const T* nu = sA + (size_t)((t.site_l * L5 + s_up) * tl.rt + t.r_l) * kPadF;   // P_+ half of B^+: s+1
      const T* nd = sA + (size_t)((t.site_l * L5 + s_dn) * tl.rt + t.r_l) * kPadF;   // P_- half of B^+: s-1
      const T cu = a.f.c5 * w_up, cl = a.f.c5 * w_dn;
#pragma unroll
      for (int i = 0; i < 12; i++) o[i] = a.f.b5 * me[i] + cu * nu[i];
#pragma unroll
      for (int i = 12; i < 24; i++) o[i] = a.f.b5 * me[i] + cl * nd[i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 24; i++) o[i] = a.kappa * acc[i];
  }

  T n2 = 0;
  if (t.act) {
    if (EPI == E_A_SAME || EPI == E_AD_SAME_BD) {
      if (a.g_same != T(0)) {
        T y[24];
        apply_A<S, T>(a, t.h, t.s, t.r, EPI == E_AD_SAME_BD, m, y);
#pragma unroll
        for (int i = 0; i < 24; i++) o[i] += a.g_same * y[i];
      }
    }
    if ((EPI == E_RAW || EPI == E_A_SAME || EPI == E_AD_SAME_BD) && a.add != nullptr) {
      T y[24];
      load24<S, T>(a.add, a.add_nrm, t.u, y);
#pragma unroll
      for (int i = 0; i < 24; i++) o[i] += y[i];
    }
    store24<S, T>(a.out, a.out_nrm, t.u, o);
    if (a.partials != nullptr) {
#pragma unroll
      for (int i = 0; i < 24; i++) n2 += o[i] * o[i];
    }
  }
  if (a.partials != nullptr) {
    // per-site, per-slot sums over the L5 slices (fixed order, FP64), stored as partials[r][h]
    __syncthreads();
    double* sred = reinterpret_cast<double*>(sA);
    sred[t.tid] = (double)n2;
    __syncthreads();
    if (t.s == 0 && t.valid) {
      double sum = 0.0;
      for (int k = 0; k < L5; k++) sum += sred[(t.site_l * L5 + k) * tl.rt + t.r_l];
      a.partials[(long)t.r * a.g.Vh + t.h] = sum;
    }
  }
}

template <typename S, typename T, int EPI>
__global__ void hop_fast_kernel(FastArgs<S, T> a, Tiling tl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Thr t = thread_of(a, tl);
  T acc[24];
#pragma unroll
  for (int i = 0; i < 24; i++) acc[i] = 0;
  if (t.act) {
    const Site x = make_site(a.g, a.out_par, t.h);
    hop_term<0, true, S, T>(a, x, t.h, t.s, t.r, nullptr, 1.f, acc);
    hop_term<0, false, S, T>(a, x, t.h, t.s, t.r, nullptr, 1.f, acc);
    hop_term<1, true, S, T>(a, x, t.h, t.s, t.r, nullptr, 1.f, acc);
    hop_term<1, false, S, T>(a, x, t.h, t.s, t.r, nullptr, 1.f, acc);
    hop_term<2, true, S, T>(a, x, t.h, t.s, t.r, nullptr, 1.f, acc);
    hop_term<2, false, S, T>(a, x, t.h, t.s, t.r, nullptr, 1.f, acc);
    hop_term<3, true, S, T>(a, x, t.h, t.s, t.r, nullptr, 1.f, acc);
    hop_term<3, false, S, T>(a, x, t.h, t.s, t.r, nullptr, 1.f, acc);
  }
  epilogue<S, T, EPI>(a, tl, t, acc, reinterpret_cast<T*>(smem_raw));
}

// ---------------------------------------------------------------------------
// Staged variant.  Every wait is bounded; on a timeout the block records an
// error code and returns (after a bounded wait for its own copies).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of bar for at most `budget` clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long budget) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

__device__ __forceinline__ int nbr_half_any(const Geom& g, const Site& x, int d) {
  switch (d) {
    case 0: return nbr_half<0, true>(g, x);
    case 1: return nbr_half<0, false>(g, x);
    case 2: return nbr_half<1, true>(g, x);
    case 3: return nbr_half<1, false>(g, x);
    case 4: return nbr_half<2, true>(g, x);
    case 5: return nbr_half<2, false>(g, x);
    case 6: return nbr_half<3, true>(g, x);
    default: return nbr_half<3, false>(g, x);
  }
}

template <int D, typename S, typename T>
__device__ __forceinline__ bool staged_term(const FastArgs<S, T>& a, const Tiling& tl, const StageInfo& si,
                                            const Thr& t, const Site& x, uint64_t* bars, const S* buf,
                                            const float* nbuf, bool ok, T* acc) {
  if (ok) ok = mbar_wait_bounded(&bars[D], 0, si.budget);
  if (ok && t.act) {
    const int upb = a.L5 * a.N;
    const int lu = t.s * a.N + t.r;
    const S* sp = buf + ((size_t)(D * tl.nsb + t.site_l) * upb + lu) * 24;
    float nrm = 1.0f;
    if (StoreTraits<S>::kNorm) {
      if (si.nrm_bytes) nrm = nbuf[(size_t)(D * tl.nsb + t.site_l) * upb + lu];
      else nrm = __ldg(a.in_nrm + (long)nbr_half<D / 2, (D % 2) == 0>(a.g, x) * upb + lu);
    }
    hop_term<D / 2, (D % 2) == 0, S, T>(a, x, t.h, t.s, t.r, sp, nrm, acc);
  }
  return ok;
}

template <typename S, typename T, int EPI>
__global__ void hop_staged_kernel(FastArgs<S, T> a, Tiling tl, StageInfo si) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  S* buf = reinterpret_cast<S*>(smem_raw + 128);
  float* nbuf = reinterpret_cast<float*>(smem_raw + 128 + si.spin_bytes);
  T* sA = reinterpret_cast<T*>(smem_raw + 128 + si.spin_bytes + si.nrm_bytes);
  const Thr t = thread_of(a, tl);
  const int upb = a.L5 * a.N;                      // units per site (rt == N)
  const long h0 = (long)blockIdx.x * tl.nsb;
  const int nsites = (int)((a.g.Vh - h0) < tl.nsb ? (a.g.Vh - h0) : tl.nsb);
  const bool skip = si.err != nullptr && *(volatile int*)si.err != 0;
  const unsigned chunk = (unsigned)(upb * 24 * sizeof(S));
  const unsigned nchunk = si.nrm_bytes ? (unsigned)(upb * sizeof(float)) : 0u;
  if (t.tid == 0) {
    for (int d = 0; d < 8; d++) {
      mbar_init(&bars[d], 1);
      if (!skip) mbar_expect_tx(&bars[d], (unsigned)nsites * (chunk + nchunk) + si.extra_tx);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // the (direction, site) pairs are spread over the threads; each issues that neighbour's copies
  if (!skip) {
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    for (int k = t.tid; k < 8 * nsites; k += nthr) {
      const int d = k / nsites, j = k - d * nsites;
      const Site xj = make_site(a.g, a.out_par, h0 + j);
      const long hn = nbr_half_any(a.g, xj, d);
      bulk_g2s(buf + ((size_t)(d * tl.nsb + j) * upb) * 24, a.in + (size_t)hn * upb * 24, chunk, &bars[d]);
      if (nchunk) bulk_g2s(nbuf + (size_t)(d * tl.nsb + j) * upb, a.in_nrm + (size_t)hn * upb, nchunk, &bars[d]);
    }
  }
  T acc[24];
#pragma unroll
  for (int i = 0; i < 24; i++) acc[i] = 0;
  const Site x = make_site(a.g, a.out_par, t.valid ? t.h : h0);
  bool ok = !skip;
  ok = staged_term<0, S, T>(a, tl, si, t, x, bars, buf, nbuf, ok, acc);
  ok = staged_term<1, S, T>(a, tl, si, t, x, bars, buf, nbuf, ok, acc);
  ok = staged_term<2, S, T>(a, tl, si, t, x, bars, buf, nbuf, ok, acc);
  ok = staged_term<3, S, T>(a, tl, si, t, x, bars, buf, nbuf, ok, acc);
  ok = staged_term<4, S, T>(a, tl, si, t, x, bars, buf, nbuf, ok, acc);
  ok = staged_term<5, S, T>(a, tl, si, t, x, bars, buf, nbuf, ok, acc);
  ok = staged_term<6, S, T>(a, tl, si, t, x, bars, buf, nbuf, ok, acc);
  ok = staged_term<7, S, T>(a, tl, si, t, x, bars, buf, nbuf, ok, acc);
  // a block that timed out (or skipped) records it and leaves, after making sure
  // no copy of its own is still writing into the shared memory
  if (__syncthreads_or(ok ? 0 : 1)) {
    if (t.tid == 0) {
      if (!skip)
        for (int d = 0; d < 8; d++) mbar_wait_bounded(&bars[d], 0, si.budget / 8);
      if (si.err) atomicExch(si.err, MDWF_TIMEOUT_CODE);
    }
    return;
  }
  epilogue<S, T, EPI>(a, tl, t, acc, sA);
}

template <typename S, typename T>
size_t staged_bytes(const Tiling& t, int L5, int N, unsigned* spin, unsigned* nrm) {
  const size_t upb = (size_t)L5 * N;
  const size_t sp = 8 * (size_t)t.nsb * upb * 24 * sizeof(S);
  const size_t nr = (StoreTraits<S>::kNorm && upb % 4 == 0) ? 8 * (size_t)t.nsb * upb * sizeof(float) : 0;
  size_t tail = (size_t)t.threads * kPadF * sizeof(T);
  if (tail < (size_t)t.threads * sizeof(double)) tail = (size_t)t.threads * sizeof(double);
  if (spin) *spin = (unsigned)sp;
  if (nrm) *nrm = (unsigned)nr;
  return 128 + sp + nr + tail;
}

template <typename S, typename T, int EPI>
cudaError_t launch_one(const FastArgs<S, T>& a, const Tiling& t, cudaStream_t st, const StageInfo* stage) {
  const dim3 grid((unsigned)t.ntiles, (unsigned)t.ngroups);
  const dim3 block((unsigned)t.rt, (unsigned)a.L5, (unsigned)t.nsb);
  if (stage != nullptr) {
    StageInfo si = *stage;
    size_t smem = staged_bytes<S, T>(t, a.L5, a.N, &si.spin_bytes, &si.nrm_bytes);
    cudaError_t e = cudaFuncSetAttribute(hop_staged_kernel<S, T, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    hop_staged_kernel<S, T, EPI><<<grid, block, smem, st>>>(a, t, si);
    return cudaGetLastError();
  }
  size_t smem = (size_t)t.threads * kPadF * sizeof(T);
  if (smem < (size_t)t.threads * sizeof(double)) smem = (size_t)t.threads * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(hop_fast_kernel<S, T, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  hop_fast_kernel<S, T, EPI><<<grid, block, smem, st>>>(a, t);
  return cudaGetLastError();
}

template <typename S, typename T, int EPI>
int max_threads_one() {
  cudaFuncAttributes fa, fb;
  if (cudaFuncGetAttributes(&fa, hop_fast_kernel<S, T, EPI>) != cudaSuccess) return 128;
  if (cudaFuncGetAttributes(&fb, hop_staged_kernel<S, T, EPI>) != cudaSuccess) return 128;
  return fa.maxThreadsPerBlock < fb.maxThreadsPerBlock ? fa.maxThreadsPerBlock : fb.maxThreadsPerBlock;
}

// ---------------------------------------------------------------------------
// Tensor-core variant for fp16 storage.  For one direction mu, the colour
// multiply of all (slice, RHS) units of a site by the same link is a small
// dense product.  A warp takes a tile of 16 units of one site and, per mu,
// four mma.sync.m16n8k16 (fp16 operands, FP32 accumulation):
//   A (16 x 16): row i = unit i of the tile; columns 0..7 = (re, im) of the
//                three colours (+ padding) of the forward term's projected
//                spin component, columns 8..15 the backward term's;
//   B (16 x 8):  rows 0..7 the real form of U_mu(x) (forward), rows 8..15 of
//                U_mu(x - mu)^+ (backward): B[2b][2a] = Re W_ab, B[2b+1][2a] = -Im W_ab,
//                B[2b][2a+1] = Im W_ab, B[2b+1][2a+1] = Re W_ab;
//   C (16 x 8):  (re, im) of colour a of sum_d W_d h_d, accumulated over mu.
// The two spin components k of the projected spinor h and of the rotated
// spinor g = sg e_mu^+ h (which feeds the lower spins) use one mma each:
// up_k += h_k B, lo_k += g_k B.  Every unit has its own fp16 scale per
// neighbour; they are divided by the unit's largest neighbour scale and folded
// into A (so A stays within fp16 range), and the FP32 result is multiplied by
// that largest scale at the end.  Lane (g, c), c = lane % 4, loads colour c of
// units g and g + 8 (one 16-byte word each); lanes with c = 3 carry zeros.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_m16n8k16(const uint32_t a[4], uint32_t b0, uint32_t b1, float d[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
__device__ __forceinline__ __half2 u2h(uint32_t u) { return *reinterpret_cast<__half2*>(&u); }
__device__ __forceinline__ uint32_t swap_hl(uint32_t x) { return __byte_perm(x, 0, 0x1032); }
constexpr uint32_t kNegHi = 0x80000000u, kNegLo = 0x00008000u;

// Projected (h0, h1) and rotated (g0, g1) half spinors of colour c of one unit,
// scaled by r (fp16 pair), from the 16-byte word q = spins 0..3 of that colour.
template <int MU>
__device__ __forceinline__ void mma_project(uint4 q, __half2 r, bool neg_sg, uint32_t& h0, uint32_t& h1, uint32_t& g0,
                                            uint32_t& g1) {
  const uint32_t sgn = neg_sg ? (kNegHi | kNegLo) : 0u;   // multiply by sg = -1
  const __half2 p0 = u2h(q.x), p1 = u2h(q.y), p2 = u2h(q.z), p3 = u2h(q.w);
  __half2 a0, a1;
  // h = psi_up + sg e_mu psi_lo ; e_x = i sigma_x, e_y = -i sigma_y, e_z = i sigma_z, e_t = 1
  if (MU == 0) {        // (i p3, i p2)
    a0 = __hadd2(p0, u2h(swap_hl(h2u(p3)) ^ kNegLo ^ sgn));
    a1 = __hadd2(p1, u2h(swap_hl(h2u(p2)) ^ kNegLo ^ sgn));
  } else if (MU == 1) { // (-p3, p2)
    a0 = __hadd2(p0, u2h(h2u(p3) ^ (kNegHi | kNegLo) ^ sgn));
    a1 = __hadd2(p1, u2h(h2u(p2) ^ sgn));
  } else if (MU == 2) { // (i p2, -i p3)
    a0 = __hadd2(p0, u2h(swap_hl(h2u(p2)) ^ kNegLo ^ sgn));
    a1 = __hadd2(p1, u2h(swap_hl(h2u(p3)) ^ kNegHi ^ sgn));
  } else {              // (p2, p3)
    a0 = __hadd2(p0, u2h(h2u(p2) ^ sgn));
    a1 = __hadd2(p1, u2h(h2u(p3) ^ sgn));
  }
  h0 = h2u(__hmul2(a0, r));
  h1 = h2u(__hmul2(a1, r));
  // g = sg e_mu^+ h ;  -i z = swap(z) with the high half negated, i z = swap(z) with the low half negated
  if (MU == 0) {        // (-i h1, -i h0)
    g0 = swap_hl(h1) ^ kNegHi ^ sgn;
    g1 = swap_hl(h0) ^ kNegHi ^ sgn;
  } else if (MU == 1) { // (h1, -h0)
    g0 = h1 ^ sgn;
    g1 = h0 ^ (kNegHi | kNegLo) ^ sgn;
  } else if (MU == 2) { // (-i h0, i h1)
    g0 = swap_hl(h0) ^ kNegHi ^ sgn;
    g1 = swap_hl(h1) ^ kNegLo ^ sgn;
  } else {              // (h0, h1)
    g0 = h0 ^ sgn;
    g1 = h1 ^ sgn;
  }
}

// B fragment of lane (g, c): rows 2c, 2c+1, column g (colour a = g / 2, part g % 2)
// of the real form of W = U (forward) or U^+ (backward).
__device__ __forceinline__ uint32_t mma_link(const __half2* __restrict__ U16, long link, int g, int c, bool fwd) {
  const int ca = g >> 1;
  if (c == 3 || ca == 3) return 0u;
  // W_ab = U_ab (forward) or conj(U_ba) (backward), a = ca, b = c
  const uint32_t e = h2u(__ldg(U16 + link * 9 + (fwd ? ca * 3 + c : c * 3 + ca)));
  if (g & 1) return fwd ? swap_hl(e) : (swap_hl(e) ^ kNegLo);    // (Im W, Re W)
  return fwd ? (e ^ kNegHi) : e;                                   // (Re W, -Im W)
}

template <int EPI>
__global__ void hop_mma_kernel(FastArgs<__half, float> a, Tiling tl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sA = reinterpret_cast<float*>(smem_raw);
  const Thr t = thread_of(a, tl);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  Site* sSite = reinterpret_cast<Site*>(smem_raw + (size_t)nthr * kPadF * sizeof(float));
  const int upb = a.L5 * a.N;                      // units per site (rt == N)
  const int lane = t.tid & 31, warp = t.tid >> 5, nwarp = nthr >> 5;
  const int g = lane >> 2, c = lane & 3;
  const long h0 = (long)blockIdx.x * tl.nsb;
  if (t.tid < tl.nsb && h0 + t.tid < a.g.Vh) sSite[t.tid] = make_site(a.g, a.out_par, h0 + t.tid);
  __syncthreads();
  const uint4* in4 = reinterpret_cast<const uint4*>(a.in);
  const int ntile = (tl.nsb * upb) >> 4;
  const bool dag = a.dagger != 0;
  for (int tile = warp; tile < ntile; tile += nwarp) {
    const int j = (tile << 4) / upb;
    const long h = h0 + j;
    if (h >= a.g.Vh) continue;                     // the whole warp skips together
    const Site x = sSite[j];
    const int lu0 = (tile << 4) - j * upb + g, lu1 = lu0 + 8;
    int hn[8];
    hn[0] = nbr_half<0, true>(a.g, x); hn[1] = nbr_half<0, false>(a.g, x);
    hn[2] = nbr_half<1, true>(a.g, x); hn[3] = nbr_half<1, false>(a.g, x);
    hn[4] = nbr_half<2, true>(a.g, x); hn[5] = nbr_half<2, false>(a.g, x);
    hn[6] = nbr_half<3, true>(a.g, x); hn[7] = nbr_half<3, false>(a.g, x);
    // neighbour scales (with the time boundary phase) and their largest magnitude per unit
    float s0[8], s1[8];
    float m0 = 0.f, m1 = 0.f;
#pragma unroll
    for (int d = 0; d < 8; d++) {
      s0[d] = __ldg(a.in_nrm + (long)hn[d] * upb + lu0);
      s1[d] = __ldg(a.in_nrm + (long)hn[d] * upb + lu1);
      m0 = fmaxf(m0, s0[d]);
      m1 = fmaxf(m1, s1[d]);
    }
    const bool tf = a.antiperiodic && x.c[3] == a.g.L[3] - 1, tb = a.antiperiodic && x.c[3] == 0;
    const float i0 = m0 > 0.f ? 1.f / m0 : 0.f, i1 = m1 > 0.f ? 1.f / m1 : 0.f;
    float up0[4] = {0.f, 0.f, 0.f, 0.f}, up1[4] = {0.f, 0.f, 0.f, 0.f};
    float lo0[4] = {0.f, 0.f, 0.f, 0.f}, lo1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      uint32_t ah0[4] = {0u, 0u, 0u, 0u}, ah1[4] = {0u, 0u, 0u, 0u};   // A for up_k0, up_k1
      uint32_t ag0[4] = {0u, 0u, 0u, 0u}, ag1[4] = {0u, 0u, 0u, 0u};   // A for lo_k0, lo_k1
#pragma unroll
      for (int fb = 0; fb < 2; fb++) {
        const int d = 2 * mu + fb;
        const bool fwd = fb == 0;
        // forward term uses sg = -1 (dagger: +1), backward the opposite
        const bool neg_sg = fwd ? !dag : dag;
        float r0 = s0[d] * i0, r1 = s1[d] * i1;
        if (mu == 3 && (fwd ? tf : tb)) { r0 = -r0; r1 = -r1; }
        if (c < 3) {
          const uint4 q0 = __ldg(in4 + ((long)hn[d] * upb + lu0) * 3 + c);
          const uint4 q1 = __ldg(in4 + ((long)hn[d] * upb + lu1) * 3 + c);
          const __half2 rr0 = __float2half2_rn(r0), rr1 = __float2half2_rn(r1);
          uint32_t x0, x1, y0, y1, z0, z1, w0, w1;
          if (mu == 0) { mma_project<0>(q0, rr0, neg_sg, x0, x1, y0, y1); mma_project<0>(q1, rr1, neg_sg, z0, z1, w0, w1); }
          else if (mu == 1) { mma_project<1>(q0, rr0, neg_sg, x0, x1, y0, y1); mma_project<1>(q1, rr1, neg_sg, z0, z1, w0, w1); }
          else if (mu == 2) { mma_project<2>(q0, rr0, neg_sg, x0, x1, y0, y1); mma_project<2>(q1, rr1, neg_sg, z0, z1, w0, w1); }
          else { mma_project<3>(q0, rr0, neg_sg, x0, x1, y0, y1); mma_project<3>(q1, rr1, neg_sg, z0, z1, w0, w1); }
          // rows g (unit lu0) and g + 8 (unit lu1); columns of this direction half: 2 fb
          ah0[2 * fb] = x0; ah0[2 * fb + 1] = z0;
          ah1[2 * fb] = x1; ah1[2 * fb + 1] = z1;
          ag0[2 * fb] = y0; ag0[2 * fb + 1] = w0;
          ag1[2 * fb] = y1; ag1[2 * fb + 1] = w1;
        }
      }
      const long lf = ((long)a.out_par * a.g.Vh + h) * 4 + mu;
      const long lb = ((long)(1 - a.out_par) * a.g.Vh + hn[2 * mu + 1]) * 4 + mu;
      const uint32_t bf = mma_link(a.U16, lf, g, c, true);
      const uint32_t bb = mma_link(a.U16, lb, g, c, false);
      mma_m16n8k16(ah0, bf, bb, up0);
      mma_m16n8k16(ah1, bf, bb, up1);
      mma_m16n8k16(ag0, bf, bb, lo0);
      mma_m16n8k16(ag1, bf, bb, lo1);
    }
    if (c < 3) {
      // C row g = unit lu0 (entries 0, 1), row g + 8 = unit lu1 (entries 2, 3); columns 2c, 2c+1 = colour c
      const int ub0 = (tile << 4) + g, ub1 = ub0 + 8;
      const int rr0 = lu0 % a.N, rr1 = lu1 % a.N;
      const bool live0 = a.active == nullptr || a.active[rr0] != 0;
      const bool live1 = a.active == nullptr || a.active[rr1] != 0;
      const float f0 = live0 ? m0 : 0.f, f1 = live1 ? m1 : 0.f;
      float* r0p = sA + (size_t)ub0 * kPadF + 2 * c;
      float* r1p = sA + (size_t)ub1 * kPadF + 2 * c;
      r0p[0] = f0 * up0[0]; r0p[1] = f0 * up0[1]; r0p[6] = f0 * up1[0]; r0p[7] = f0 * up1[1];
      r0p[12] = f0 * lo0[0]; r0p[13] = f0 * lo0[1]; r0p[18] = f0 * lo1[0]; r0p[19] = f0 * lo1[1];
      r1p[0] = f1 * up0[2]; r1p[1] = f1 * up0[3]; r1p[6] = f1 * up1[2]; r1p[7] = f1 * up1[3];
      r1p[12] = f1 * lo0[2]; r1p[13] = f1 * lo0[3]; r1p[18] = f1 * lo1[2]; r1p[19] = f1 * lo1[3];
    }
  }
  __syncthreads();
  float acc[24];
#pragma unroll
  for (int i = 0; i < 24; i++) acc[i] = sA[(size_t)t.tid * kPadF + i];
  __syncthreads();
  epilogue<__half, float, EPI>(a, tl, t, acc, sA);
}

template <int EPI>
cudaError_t launch_mma_one(const FastArgs<__half, float>& a, const Tiling& t, cudaStream_t st) {
  const dim3 grid((unsigned)t.ntiles, (unsigned)t.ngroups);
  const dim3 block((unsigned)t.rt, (unsigned)a.L5, (unsigned)t.nsb);
  size_t smem = (size_t)t.threads * kPadF * sizeof(float) + (size_t)t.nsb * sizeof(Site);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(hop_mma_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  hop_mma_kernel<EPI><<<grid, block, smem, st>>>(a, t);
  return cudaGetLastError();
}

}  // namespace

template <typename S, typename T>
size_t staged_smem_bytes(const Tiling& t, int L5, int N) {
  if (t.rt != N || t.ngroups != 1) return 0;
  return staged_bytes<S, T>(t, L5, N, nullptr, nullptr);
}

template <typename S, typename T>
cudaError_t launch_fast(const FastArgs<S, T>& a, const Tiling& t, int epi, cudaStream_t st, const StageInfo* stage) {
  if (stage && (t.rt != a.N || t.ngroups != 1)) stage = nullptr;
  switch (epi) {
    case E_RAW: return launch_one<S, T, E_RAW>(a, t, st, stage);
    case E_BAINV: return launch_one<S, T, E_BAINV>(a, t, st, stage);
    case E_AINVD_BD: return launch_one<S, T, E_AINVD_BD>(a, t, st, stage);
    case E_A_SAME: return launch_one<S, T, E_A_SAME>(a, t, st, stage);
    case E_AD_SAME_BD: return launch_one<S, T, E_AD_SAME_BD>(a, t, st, stage);
    case E_AINV_SAME: return launch_one<S, T, E_AINV_SAME>(a, t, st, stage);
    default: return cudaErrorInvalidValue;
  }
}

template <typename S, typename T>
int fast_max_threads() {
  int m = max_threads_one<S, T, E_RAW>();
  int v[] = {max_threads_one<S, T, E_BAINV>(), max_threads_one<S, T, E_AINVD_BD>(),
             max_threads_one<S, T, E_A_SAME>(), max_threads_one<S, T, E_AD_SAME_BD>(),
             max_threads_one<S, T, E_AINV_SAME>()};
  for (int x : v) m = x < m ? x : m;
  return m;
}

bool mma_hop_usable(const Tiling& t, int L5, int N) {
  const int upb = L5 * N;
  // whole sites per block, 16-unit tiles inside one site, whole warps
  return t.rt == N && t.ngroups == 1 && upb % 16 == 0 && t.threads % 32 == 0;
}

int mma_max_threads() {
  int m = 1024;
  const void* ks[] = {(const void*)hop_mma_kernel<E_RAW>, (const void*)hop_mma_kernel<E_BAINV>,
                      (const void*)hop_mma_kernel<E_AINVD_BD>, (const void*)hop_mma_kernel<E_A_SAME>,
                      (const void*)hop_mma_kernel<E_AD_SAME_BD>, (const void*)hop_mma_kernel<E_AINV_SAME>};
  for (const void* k : ks) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return 128;
    if (fa.maxThreadsPerBlock < m) m = fa.maxThreadsPerBlock;
  }
  return m;
}

cudaError_t launch_fast_mma(const FastArgs<__half, float>& a, const Tiling& t, int epi, cudaStream_t st) {
  if (!mma_hop_usable(t, a.L5, a.N) || a.U16 == nullptr) return cudaErrorInvalidValue;
  switch (epi) {
    case E_RAW: return launch_mma_one<E_RAW>(a, t, st);
    case E_BAINV: return launch_mma_one<E_BAINV>(a, t, st);
    case E_AINVD_BD: return launch_mma_one<E_AINVD_BD>(a, t, st);
    case E_A_SAME: return launch_mma_one<E_A_SAME>(a, t, st);
    case E_AD_SAME_BD: return launch_mma_one<E_AD_SAME_BD>(a, t, st);
    case E_AINV_SAME: return launch_mma_one<E_AINV_SAME>(a, t, st);
    default: return cudaErrorInvalidValue;
  }
}

#define MDWF_INST_FAST(S, T)                                                                          \
  template cudaError_t launch_fast<S, T>(const FastArgs<S, T>&, const Tiling&, int, cudaStream_t,     \
                                         const StageInfo*);                                           \
  template int fast_max_threads<S, T>();                                                             \
  template size_t staged_smem_bytes<S, T>(const Tiling&, int, int);

MDWF_INST_FAST(double, double)
MDWF_INST_FAST(float, float)
MDWF_INST_FAST(__half, float)
MDWF_INST_FAST(__nv_bfloat16, float)

}  // namespace mdwf
