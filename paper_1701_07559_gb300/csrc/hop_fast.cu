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
//   E_SAME_AINV  out = add + g same + A^-1 (kappa H(in))        symmetric Mhat, second hop
//   E_SAME_BD    out = add + g same + kappa B^+ H(in)           symmetric Mhat^+, second hop
//   E_AINVD_SAME out = A^-+ same (no hop)                       symmetric Mhat^+, first pass
// The recursions run over columns (site, RHS, spin-colour component) of a
// shared-memory tile that holds every slice of the block's sites.
//
// Thread block: (rt RHS slots) x (L5 slices) x (nsb sites); a site's units
// (s, r) are contiguous in memory, so the block's loads of one neighbour site
// are one contiguous run.  Two variants of the hop: direct loads, or the eight
// neighbour sites of every site staged into shared memory by bulk asynchronous
// copies (cp.async.bulk + one mbarrier per direction) issued at block start.
#include "mdwf_internal.h"
#include "hop_common.cuh"

namespace mdwf {

namespace {

__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// One colour vector times W = l (DAG = false) or l^+ (DAG = true); every real
// output is one multiply and five fused multiply-adds.
template <typename T, bool DAG>
__device__ __forceinline__ void su3_mul(const T* __restrict__ l, const T* v, T* o) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    T re, im;
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const int k = DAG ? (3 * b + a) : (3 * a + b);
      const T ur = l[2 * k];
      const T ui = DAG ? -l[2 * k + 1] : l[2 * k + 1];
      if (b == 0) {
        re = ur * v[0];
        im = ur * v[1];
      } else {
        re = fma_rn(ur, v[2 * b], re);
        im = fma_rn(ur, v[2 * b + 1], im);
      }
      re = fma_rn(-ui, v[2 * b + 1], re);
      im = fma_rn(ui, v[2 * b], im);
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

// Load (global memory or shared memory) and project one neighbour spinor.  The
// returned factor multiplies the projected spinor (the fp16 storage scale; 1 else)
// and is applied in the reconstruction.
template <int MU, typename S, typename T>
struct Proj {
  static __device__ __forceinline__ T global(const S* __restrict__ v, const float* __restrict__ nrm, long u, T sg,
                                             T* h) {
    T psi[24];
    load24<S, T>(v, nrm, u, psi);
    project<MU, T>(psi, sg, h);
    return T(1);
  }
  static __device__ __forceinline__ T shared(const S* sp, float nrm, T sg, T* h) {
    T psi[24];
    load24_smem<S, T>(sp, psi);
    project<MU, T>(psi, sg, h);
    return StoreTraits<S>::kNorm ? (T)nrm : T(1);
  }
};
template <int MU>
struct Proj<MU, __half, float> {
  static __device__ __forceinline__ float global(const __half* __restrict__ v, const float* __restrict__ nrm, long u,
                                                 float sg, float* h) {
    const uint4* p = reinterpret_cast<const uint4*>(v + 24 * u);
    uint4 q[3];
    q[0] = __ldg(p);
    q[1] = __ldg(p + 1);
    q[2] = __ldg(p + 2);
    project_half<MU>(q, sg, h);
    return __ldg(nrm + u);
  }
  static __device__ __forceinline__ float shared(const __half* sp, float nrm, float sg, float* h) {
    const uint4* p = reinterpret_cast<const uint4*>(sp);
    uint4 q[3];
    q[0] = p[0];
    q[1] = p[1];
    q[2] = p[2];
    project_half<MU>(q, sg, h);
    return nrm;
  }
};

template <int MU, typename T>
__device__ __forceinline__ void reconstruct(const T* chi, T f, T fs, T* acc) {
  // f: factor of the projected spinor (storage scale x boundary phase); fs = f sg
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const T* x0 = chi + 2 * c;
    const T* x1 = chi + 6 + 2 * c;
    T* a0 = acc + 2 * c;
    T* a1 = acc + 6 + 2 * c;
    T* a2 = acc + 12 + 2 * c;
    T* a3 = acc + 18 + 2 * c;
    a0[0] += f * x0[0]; a0[1] += f * x0[1];
    a1[0] += f * x1[0]; a1[1] += f * x1[1];
    if (MU == 0) {
      a2[0] += fs * x1[1]; a2[1] -= fs * x1[0];
      a3[0] += fs * x0[1]; a3[1] -= fs * x0[0];
    } else if (MU == 1) {
      a2[0] += fs * x1[0]; a2[1] += fs * x1[1];
      a3[0] -= fs * x0[0]; a3[1] -= fs * x0[1];
    } else if (MU == 2) {
      a2[0] += fs * x0[1]; a2[1] -= fs * x0[0];
      a3[0] -= fs * x1[1]; a3[1] += fs * x1[0];
    } else {
      a2[0] += fs * x0[0]; a2[1] += fs * x0[1];
      a3[0] += fs * x1[0]; a3[1] += fs * x1[1];
    }
  }
}

// One of the eight hopping terms at neighbour half-site hn (bflip: the term
// crosses the antiperiodic time boundary); the neighbour spinor comes either
// from global memory (sp == nullptr) or from the shared staging buffer sp.
template <int MU, bool FWD, typename S, typename T>
__device__ __forceinline__ void hop_term_at(const FastArgs<S, T>& a, int hn, bool bflip, long h, int s, int r,
                                            const S* sp, float snrm, T* acc) {
  const T sg = (a.dagger ? T(1) : T(-1)) * (FWD ? T(1) : T(-1));
  T hh[12], chi[12], l[18];
  T f;
  if (sp == nullptr) f = Proj<MU, S, T>::global(a.in, a.in_nrm, ((long)hn * a.L5 + s) * a.N + r, sg, hh);
  else f = Proj<MU, S, T>::shared(sp, snrm, sg, hh);
  if (bflip) f = -f;
  if (FWD) {
    load_link<T>(a.U, ((long)a.out_par * a.g.Vh + h) * 4 + MU, l);
    su3_mul<T, false>(l, hh, chi);
    su3_mul<T, false>(l, hh + 6, chi + 6);
  } else {
    load_link<T>(a.U, ((long)(1 - a.out_par) * a.g.Vh + hn) * 4 + MU, l);
    su3_mul<T, true>(l, hh, chi);
    su3_mul<T, true>(l, hh + 6, chi + 6);
  }
  reconstruct<MU, T>(chi, f, f * sg, acc);
}

// A time hop across an edge of a decomposed lattice, from the neighbouring
// sub-domain's face (same operations and order as the local term: the sender
// projected, and for the backward hop multiplied by U^+, exactly as hop_term_at).
template <bool FWD, typename S, typename T>
__device__ __forceinline__ void halo_term(const FastArgs<S, T>& a, const Site& x, long h, int s, int r, T* acc) {
  const T sg = (a.dagger ? T(1) : T(-1)) * (FWD ? T(1) : T(-1));
  const long lex3 = x.lex - (long)x.c[3] * x.stride[3];
  const T* p = (FWD ? a.halo_fwd : a.halo_bwd) + ((lex3 * a.L5 + s) * a.N + r) * 12;
  T hh[12], chi[12];
#pragma unroll
  for (int i = 0; i < 12; i++) hh[i] = p[i];
  const T f = FWD ? a.halo_sgn_fwd : a.halo_sgn_bwd;
  if (FWD) {
    T l[18];
    load_link<T>(a.U, ((long)a.out_par * a.g.Vh + h) * 4 + 3, l);
    su3_mul<T, false>(l, hh, chi);
    su3_mul<T, false>(l, hh + 6, chi + 6);
    reconstruct<3, T>(chi, f, f * sg, acc);
  } else {
    reconstruct<3, T>(hh, f, f * sg, acc);
  }
}

template <int MU, bool FWD, typename S, typename T>
__device__ __forceinline__ void hop_term(const FastArgs<S, T>& a, const Site& x, long h, int s, int r, const S* sp,
                                         float snrm, T* acc) {
  if (MU == 3 && a.halo_fwd != nullptr && (FWD ? x.c[3] == a.g.L[3] - 1 : x.c[3] == 0)) {
    halo_term<FWD, S, T>(a, x, h, s, r, acc);
    return;
  }
  const bool bflip = MU == 3 && a.antiperiodic && (FWD ? x.c[3] == a.g.L[3] - 1 : x.c[3] == 0);
  hop_term_at<MU, FWD, S, T>(a, nbr_half<MU, FWD>(a.g, x), bflip, h, s, r, sp, snrm, acc);
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

// Register versions of the recursions for a column of compile-time length L
// (same operations in the same order as col_ainv / col_bop).
template <int L, typename T>
__device__ __forceinline__ void ainv_regs(T* v, T inv_alpha, T kap, T m, T powL) {
  T z = 0;
#pragma unroll
  for (int k = 0; k < L; k++) { z = v[k] * inv_alpha - kap * z; v[k] = z; }
  const T yl = z / (T(1) + m * powL);
  v[L - 1] = yl;
  const T mk = -kap;
  T w = m * yl * mk;
#pragma unroll
  for (int k = 0; k < L - 1; k++) { v[k] -= w; w *= mk; }
}
template <int L, typename T>
__device__ __forceinline__ void bop_regs(T* v, T b5, T c5, T m) {
  T prev = -m * v[L - 1];
#pragma unroll
  for (int k = 0; k < L; k++) { const T x = v[k]; v[k] = b5 * x + c5 * prev; prev = x; }
}

// The columns comp = s0, s0 + L, ... of one (site, slot): loaded into registers
// along the recursion direction, transformed, stored back.
template <int L, int EPI, typename T>
__device__ __forceinline__ void cols_regs(T* base, int st, int s0, const Fifth<T>& f, T m) {
  for (int comp = s0; comp < 24; comp += L) {
    const bool upper = comp < 12;
    const bool down = (EPI == E_AINVD_BD || EPI == E_AINVD_SAME) ? !upper : upper;
    T* p = base + comp + (down ? 0 : (L - 1) * st);
    const int step = down ? st : -st;
    T v[L];
#pragma unroll
    for (int k = 0; k < L; k++) v[k] = p[k * step];
    if (EPI == E_BAINV) {
      ainv_regs<L, T>(v, f.inv_alpha, f.kap, m, f.powL);
      bop_regs<L, T>(v, f.b5, f.c5, m);
    } else if (EPI == E_AINVD_BD) {
      bop_regs<L, T>(v, f.b5, f.c5, m);
      ainv_regs<L, T>(v, f.inv_alpha, f.kap, m, f.powL);
    } else {
      ainv_regs<L, T>(v, f.inv_alpha, f.kap, m, f.powL);
    }
#pragma unroll
    for (int k = 0; k < L; k++) p[k * step] = v[k];
  }
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
// IN_SMEM: the hop sums, kappa included, are already in row tid of sA (acc unused).
template <typename S, typename T, int EPI, bool IN_SMEM = false>
__device__ __forceinline__ void epilogue(const FastArgs<S, T>& a, const Tiling& tl, const Thr& t, const T* acc,
                                         T* sA) {
  const int L5 = a.L5;
  const T m = t.valid ? a.f.mass[t.r] : T(0);
  T o[24];
  constexpr bool kCols = (EPI == E_BAINV || EPI == E_AINVD_BD || EPI == E_AINV_SAME || EPI == E_SAME_AINV ||
                          EPI == E_AINVD_SAME);
  constexpr bool kSameFirst = (EPI == E_AINV_SAME || EPI == E_AINVD_SAME);   // same enters before the columns
  constexpr bool kBdag = (EPI == E_AD_SAME_BD || EPI == E_SAME_BD);
  if (IN_SMEM) __syncthreads();
  if (kCols || kBdag) {
    if (!IN_SMEM) {
      T v[24];
#pragma unroll
      for (int i = 0; i < 24; i++) v[i] = a.kappa * acc[i];
      if (kSameFirst && t.act) {
        T y[24];
        load24<S, T>(a.same, a.same_nrm, t.u, y);
#pragma unroll
        for (int i = 0; i < 24; i++) v[i] += y[i];
      }
#pragma unroll
      for (int i = 0; i < 24; i++) sA[t.tid * kPadF + i] = v[i];
      __syncthreads();
    } else if (kSameFirst) {
      if (t.act) {
        T y[24];
        load24<S, T>(a.same, a.same_nrm, t.u, y);
#pragma unroll
        for (int i = 0; i < 24; i++) sA[t.tid * kPadF + i] += y[i];
      }
      __syncthreads();
    }
    if (kCols) {
      // thread (r_l, s, site_l) runs the columns comp = s, s + L5, ... of (site_l, r_l)
      if (t.act) {
        const int st = tl.rt * kPadF;
        T* base = sA + (size_t)(t.site_l * L5 * tl.rt + t.r_l) * kPadF;
        switch (L5) {
          case 4: cols_regs<4, EPI, T>(base, st, t.s, a.f, m); break;
          case 6: cols_regs<6, EPI, T>(base, st, t.s, a.f, m); break;
          case 8: cols_regs<8, EPI, T>(base, st, t.s, a.f, m); break;
          case 10: cols_regs<10, EPI, T>(base, st, t.s, a.f, m); break;
          case 12: cols_regs<12, EPI, T>(base, st, t.s, a.f, m); break;
          case 16: cols_regs<16, EPI, T>(base, st, t.s, a.f, m); break;
          default:
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
          } else if (EPI == E_AINVD_SAME) {
            Col<T> c = make_col<T>(base + comp, st, L5, !upper);
            col_ainv<T>(c, L5, a.f.inv_alpha, a.f.kap, m, a.f.powL);
          } else {
            Col<T> c = make_col<T>(base + comp, st, L5, upper);
            col_ainv<T>(c, L5, a.f.inv_alpha, a.f.kap, m, a.f.powL);
          }
        }
        }
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 24; i++) o[i] = sA[t.tid * kPadF + i];
    } else {
      // E_AD_SAME_BD, E_SAME_BD: B^+ (kappa H) from this slice and its neighbour slice
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
  } else if (IN_SMEM) {
#pragma unroll
    for (int i = 0; i < 24; i++) o[i] = sA[t.tid * kPadF + i];
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
    if ((EPI == E_SAME_AINV || EPI == E_SAME_BD) && a.g_same != T(0)) {
      T y[24];
      load24<S, T>(a.same, a.same_nrm, t.u, y);
#pragma unroll
      for (int i = 0; i < 24; i++) o[i] += a.g_same * y[i];
    }
    if ((EPI == E_RAW || EPI == E_A_SAME || EPI == E_AD_SAME_BD || EPI == E_SAME_AINV || EPI == E_SAME_BD) &&
        a.add != nullptr) {
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

// Shared memory of the direct kernel: the epilogue tile (threads x kPadF reals,
// at least threads doubles).
template <typename T>
__host__ __device__ __forceinline__ size_t direct_tile_bytes(int threads) {
  size_t b = (size_t)threads * kPadF * sizeof(T);
  if (b < (size_t)threads * sizeof(double)) b = (size_t)threads * sizeof(double);
  return b;
}

template <typename S, typename T, int EPI>
__device__ __forceinline__ void hop_fast_body(const FastArgs<S, T>& a, const Tiling& tl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Thr t = thread_of(a, tl);
  T acc[24];
#pragma unroll
  for (int i = 0; i < 24; i++) acc[i] = 0;
  if (t.act && a.in != nullptr) {      // no input: a local fifth-dimension pass
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

// FP32 arithmetic: capped at 72 registers, so that three 288-thread blocks (27
// warps) fit on an SM; the few spills stay in L1 and the extra warps hide the
// neighbour-load latency (measured 11-13 % faster than the uncapped 88-96).
template <typename S, typename T, int EPI>
__global__ void __maxnreg__(72) hop_fast_kernel(FastArgs<S, T> a, Tiling tl) {
  hop_fast_body<S, T, EPI>(a, tl);
}
// FP64 arithmetic: no cap (24 doubles of accumulator alone take 48 registers).
template <typename S, typename T, int EPI>
__global__ void hop_fast_kernel_f64(FastArgs<S, T> a, Tiling tl) {
  hop_fast_body<S, T, EPI>(a, tl);
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
  const size_t smem = direct_tile_bytes<T>(t.threads);
  auto* kern = std::is_same<T, double>::value ? hop_fast_kernel_f64<S, T, EPI> : hop_fast_kernel<S, T, EPI>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, block, smem, st>>>(a, t);
  return cudaGetLastError();
}

template <typename S, typename T, int EPI>
int max_threads_one() {
  cudaFuncAttributes fa, fb;
  auto* kern = std::is_same<T, double>::value ? hop_fast_kernel_f64<S, T, EPI> : hop_fast_kernel<S, T, EPI>;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return 128;
  if (cudaFuncGetAttributes(&fb, hop_staged_kernel<S, T, EPI>) != cudaSuccess) return 128;
  return fa.maxThreadsPerBlock < fb.maxThreadsPerBlock ? fa.maxThreadsPerBlock : fb.maxThreadsPerBlock;
}

// ---------------------------------------------------------------------------
// Tensor-core variant for fp16 storage.  For one direction, the colour
// multiply of all (slice, RHS) units of a site by the same link W (U_mu(x)
// forward, U_mu(x - mu)^+ backward) is a product with a shared 3 x 3 matrix.
// A warp takes a tile of 8 units of one site and, per direction, one
// mma.sync.m16n8k8 (fp16 operands, FP32 accumulation):
//   A (16 x 8): row g = projected half spinor h_0 of unit g, row g + 8 = h_1;
//               columns (re, im) of the three colours (+ one zero pair);
//   B (8 x 8):  the real form of W: B[2b][2a] = Re W_ab, B[2b+1][2a] = -Im W_ab,
//               B[2b][2a+1] = Im W_ab, B[2b+1][2a+1] = Re W_ab (zero for a, b = 3);
//   D (16 x 8): (re, im) of colour a of W h_0 (rows g) and W h_1 (rows g + 8).
// Lane (g, c), c = lane % 4, loads colour c of unit g (one 16-byte word of the
// colour-major fp16 spinor), holds exactly the A entries it needs and receives
// colour c of both products, so the spin reconstruction, with the unit's scale
// and kappa applied in FP32, stays in the lane.  Lanes with c = 3 carry zeros.
// B fragments come precomputed per link and lane (one coalesced word each).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_m16n8k8(uint32_t a0, uint32_t a1, uint32_t b0, float d[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
__device__ __forceinline__ __half2 u2h(uint32_t u) { return *reinterpret_cast<__half2*>(&u); }
__device__ __forceinline__ uint32_t swap_hl(uint32_t x) { return __byte_perm(x, 0, 0x1032); }
constexpr uint32_t kNegHi = 0x80000000u, kNegLo = 0x00008000u;

// Projection h = psi_up + sg e_mu psi_lo of one colour (p0..p3 = spins 0..3 as
// (re, im) fp16 pairs); e_x = i sigma_x, e_y = -i sigma_y, e_z = i sigma_z, e_t = 1.
// i z = swap(z) with the low half negated.
template <int MU>
__device__ __forceinline__ void mma_project(uint4 q, bool neg_sg, uint32_t& h0, uint32_t& h1) {
  const uint32_t sgn = neg_sg ? (kNegHi | kNegLo) : 0u;
  const __half2 p0 = u2h(q.x), p1 = u2h(q.y);
  if (MU == 0) {        // (i p3, i p2)
    h0 = h2u(__hadd2(p0, u2h(swap_hl(q.w) ^ kNegLo ^ sgn)));
    h1 = h2u(__hadd2(p1, u2h(swap_hl(q.z) ^ kNegLo ^ sgn)));
  } else if (MU == 1) { // (-p3, p2)
    h0 = h2u(__hadd2(p0, u2h(q.w ^ (kNegHi | kNegLo) ^ sgn)));
    h1 = h2u(__hadd2(p1, u2h(q.z ^ sgn)));
  } else if (MU == 2) { // (i p2, -i p3)
    h0 = h2u(__hadd2(p0, u2h(swap_hl(q.z) ^ kNegLo ^ sgn)));
    h1 = h2u(__hadd2(p1, u2h(swap_hl(q.w) ^ kNegHi ^ sgn)));
  } else {              // (p2, p3)
    h0 = h2u(__hadd2(p0, u2h(q.z ^ sgn)));
    h1 = h2u(__hadd2(p1, u2h(q.w ^ sgn)));
  }
}

// acc[2 spin + (re, im)] of one colour += the reconstructed term: spins 0, 1 get
// f x_k, spins 2, 3 get f sg e_mu^+ (x_0, x_1), with x_0 = (d0, d1), x_1 = (d2, d3).
template <int MU>
__device__ __forceinline__ void mma_reconstruct(const float d[4], float f, float fs, float* acc) {
  acc[0] += f * d[0]; acc[1] += f * d[1];
  acc[2] += f * d[2]; acc[3] += f * d[3];
  if (MU == 0) {        // (-i x1, -i x0)
    acc[4] += fs * d[3]; acc[5] -= fs * d[2];
    acc[6] += fs * d[1]; acc[7] -= fs * d[0];
  } else if (MU == 1) { // (x1, -x0)
    acc[4] += fs * d[2]; acc[5] += fs * d[3];
    acc[6] -= fs * d[0]; acc[7] -= fs * d[1];
  } else if (MU == 2) { // (-i x0, i x1)
    acc[4] += fs * d[1]; acc[5] -= fs * d[0];
    acc[6] -= fs * d[3]; acc[7] += fs * d[2];
  } else {              // (x0, x1)
    acc[4] += fs * d[0]; acc[5] += fs * d[1];
    acc[6] += fs * d[2]; acc[7] += fs * d[3];
  }
}

// One of the eight terms for the tile's 8 units (lane: unit g, colour c).
// One of the eight terms for the tile's 8 units (lane: unit g, colour c), from
// the loaded colour word q, the neighbour's scale sc and the link fragment b.
template <int MU, bool FWD>
__device__ __forceinline__ void mma_term(uint4 q, float sc, uint32_t b, bool dag, float kb, float* acc) {
  // sg = -1 for the forward term of H, +1 backward; exchanged for H^+
  const bool neg_sg = FWD ? !dag : dag;
  uint32_t h0, h1;
  mma_project<MU>(q, neg_sg, h0, h1);
  float d[4] = {0.f, 0.f, 0.f, 0.f};
  mma_m16n8k8(h0, h1, b, d);
  const float f = sc * kb;
  mma_reconstruct<MU>(d, f, neg_sg ? -f : f, acc);
}

// Shared-memory tables of a block: neighbour half-site index and kappa x
// time-boundary phase per (site, direction); the in-site memory offset of each
// block-local unit (-1: slot out of range or inactive); (site, first unit) of each tile.
struct MmaTables {
  int* nb;
  float* kb;
  int* off;
  int* tile;
};

template <int EPI>
__global__ void hop_mma_kernel(FastArgs<__half, float> a, Tiling tl, const uint32_t* __restrict__ frag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sA = reinterpret_cast<float*>(smem_raw);
  const Thr t = thread_of(a, tl);
  const int nthr = tl.threads;
  const int upb = a.L5 * tl.rt;                   // units of one site in this block
  const int tps = (upb + 7) >> 3;                 // 8-unit tiles per site
  const int ntile = tl.nsb * tps;
  size_t base = (size_t)nthr * kPadF * sizeof(float);
  if (base < (size_t)nthr * sizeof(double)) base = (size_t)nthr * sizeof(double);
  MmaTables tb;
  tb.nb = reinterpret_cast<int*>(smem_raw + base);
  tb.kb = reinterpret_cast<float*>(tb.nb + 8 * tl.nsb);
  tb.off = reinterpret_cast<int*>(tb.kb + 8 * tl.nsb);
  tb.tile = tb.off + upb;
  const long h0 = (long)blockIdx.x * tl.nsb;
  for (int k = t.tid; k < 8 * tl.nsb; k += nthr) {
    const int j = k >> 3, d = k & 7;
    const long h = h0 + j;
    int hn = 0;
    float kb = a.kappa;
    if (h < a.g.Vh) {
      const Site x = make_site(a.g, a.out_par, h);
      switch (d) {
        case 0: hn = nbr_half<0, true>(a.g, x); break;
        case 1: hn = nbr_half<0, false>(a.g, x); break;
        case 2: hn = nbr_half<1, true>(a.g, x); break;
        case 3: hn = nbr_half<1, false>(a.g, x); break;
        case 4: hn = nbr_half<2, true>(a.g, x); break;
        case 5: hn = nbr_half<2, false>(a.g, x); break;
        case 6: hn = nbr_half<3, true>(a.g, x); break;
        default: hn = nbr_half<3, false>(a.g, x); break;
      }
      if (a.antiperiodic && ((d == 6 && x.c[3] == a.g.L[3] - 1) || (d == 7 && x.c[3] == 0))) kb = -kb;
    }
    tb.nb[k] = hn;
    tb.kb[k] = kb;
  }
  for (int jj = t.tid; jj < upb; jj += nthr) {
    const int s = jj / tl.rt, r = blockIdx.y * tl.rt + (jj - s * tl.rt);
    const bool ok = r < a.N && (a.active == nullptr || a.active[r] != 0);
    tb.off[jj] = ok ? s * a.N + r : -1;
  }
  for (int k = t.tid; k < ntile; k += nthr) {
    const int j = k / tps;
    tb.tile[k] = (j << 16) | ((k - j * tps) * 8);
  }
  __syncthreads();
  const int lane = t.tid & 31, warp = t.tid >> 5, nwarp = nthr >> 5;
  const int g = lane >> 2, c = lane & 3;
  const uint32_t upm = (uint32_t)(a.L5 * a.N);    // units of one site in memory
  const uint4* in4 = reinterpret_cast<const uint4*>(a.in);
  const bool dag = a.dagger != 0;
  const uint32_t lb = (uint32_t)((1 - a.out_par) * a.g.Vh);
  for (int tile = warp; warp < nwarp && tile < ntile; tile += nwarp) {    // whole warps only (mma.sync)
    const int tj = tb.tile[tile];
    const int j = tj >> 16;
    const long h = h0 + j;
    if (h >= a.g.Vh) continue;                             // uniform over the warp
    const int jj = (tj & 0xffff) + g;
    const int off = jj < upb ? tb.off[jj] : -1;
    const bool live = off >= 0 && c < 3;
    const uint32_t uo = live ? (uint32_t)off : 0u;
    const int* nb = tb.nb + 8 * j;
    const float* kb = tb.kb + 8 * j;
    // B fragments: forward links of this site, backward links of the neighbours
    const uint32_t* ff = frag + ((size_t)((uint32_t)(a.out_par * a.g.Vh + h) * 4u) * 2u) * 32u + lane;
    const uint32_t* fb = frag + 32 + lane;
    // all loads of the tile first (24 independent loads in flight per lane)
    uint4 q[8];
    float sc[8];
    uint32_t b[8];
#pragma unroll
    for (int d = 0; d < 8; d++) {
      const uint32_t un = (uint32_t)nb[d] * upm + uo;
      if (live) {
        q[d] = __ldg(in4 + (size_t)un * 3u + c);
        sc[d] = __ldg(a.in_nrm + un);
      } else {
        q[d] = make_uint4(0u, 0u, 0u, 0u);
        sc[d] = 0.f;
      }
      b[d] = (d & 1) ? __ldg(fb + (size_t)((lb + nb[d]) * 4u + (d >> 1)) * 64u) : __ldg(ff + (d >> 1) * 64);
    }
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    mma_term<0, true>(q[0], sc[0], b[0], dag, kb[0], acc);
    mma_term<0, false>(q[1], sc[1], b[1], dag, kb[1], acc);
    mma_term<1, true>(q[2], sc[2], b[2], dag, kb[2], acc);
    mma_term<1, false>(q[3], sc[3], b[3], dag, kb[3], acc);
    mma_term<2, true>(q[4], sc[4], b[4], dag, kb[4], acc);
    mma_term<2, false>(q[5], sc[5], b[5], dag, kb[5], acc);
    mma_term<3, true>(q[6], sc[6], b[6], dag, kb[6], acc);
    mma_term<3, false>(q[7], sc[7], b[7], dag, kb[7], acc);
    if (live) {
      float* row = sA + (size_t)(j * upb + jj) * kPadF + 2 * c;
#pragma unroll
      for (int sp = 0; sp < 4; sp++) {
        row[6 * sp] = acc[2 * sp];
        row[6 * sp + 1] = acc[2 * sp + 1];
      }
    }
  }
  epilogue<__half, float, EPI, true>(a, tl, t, nullptr, sA);
}

// Pipelined form of the tensor-core hop (one RHS group, whole 8-unit tiles).
// The 8 units of a tile are contiguous in memory, so per direction the tile's
// input is three contiguous runs: 8 spinors (384 B), 8 scales (32 B) and the
// link fragment (128 B).  Each warp double-buffers its tiles in shared memory:
// 24 lanes issue the 24 bulk copies (cp.async.bulk, one mbarrier per buffer)
// of tile k + 1 before it computes tile k, so L2 latency overlaps the work.
// Every wait is bounded; a warp whose wait runs out records MDWF_TIMEOUT_CODE,
// waits (bounded) for its own copies still in flight and stops.
constexpr unsigned kMmaBuf = 8 * (384 + 32 + 128);   // bytes of one tile buffer

template <int EPI>
__global__ void hop_mma_bulk_kernel(FastArgs<__half, float> a, Tiling tl, const uint32_t* __restrict__ frag,
                                    StageInfo si) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Thr t = thread_of(a, tl);
  const int nthr = tl.threads;
  const int nwarp = nthr >> 5;
  const int upb = a.L5 * a.N;                     // units of one site (one RHS group)
  const int tps = upb >> 3;
  const int ntile = tl.nsb * tps;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  unsigned char* bufs = smem_raw + (((size_t)nwarp * 16 + 127) & ~(size_t)127);
  float* sA = reinterpret_cast<float*>(bufs + (size_t)nwarp * 2 * kMmaBuf);
  size_t base = (size_t)nthr * kPadF * sizeof(float);
  if (base < (size_t)nthr * sizeof(double)) base = (size_t)nthr * sizeof(double);
  MmaTables tb;
  tb.nb = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(sA) + base);
  tb.kb = reinterpret_cast<float*>(tb.nb + 8 * tl.nsb);
  tb.off = reinterpret_cast<int*>(tb.kb + 8 * tl.nsb);
  tb.tile = tb.off + upb;
  const long h0 = (long)blockIdx.x * tl.nsb;
  for (int k = t.tid; k < 8 * tl.nsb; k += nthr) {
    const int j = k >> 3, d = k & 7;
    const long h = h0 + j;
    int hn = 0;
    float kb = a.kappa;
    if (h < a.g.Vh) {
      const Site x = make_site(a.g, a.out_par, h);
      switch (d) {
        case 0: hn = nbr_half<0, true>(a.g, x); break;
        case 1: hn = nbr_half<0, false>(a.g, x); break;
        case 2: hn = nbr_half<1, true>(a.g, x); break;
        case 3: hn = nbr_half<1, false>(a.g, x); break;
        case 4: hn = nbr_half<2, true>(a.g, x); break;
        case 5: hn = nbr_half<2, false>(a.g, x); break;
        case 6: hn = nbr_half<3, true>(a.g, x); break;
        default: hn = nbr_half<3, false>(a.g, x); break;
      }
      if (a.antiperiodic && ((d == 6 && x.c[3] == a.g.L[3] - 1) || (d == 7 && x.c[3] == 0))) kb = -kb;
    }
    tb.nb[k] = hn;
    tb.kb[k] = kb;
  }
  for (int jj = t.tid; jj < upb; jj += nthr) {
    const int r = jj % a.N;
    tb.off[jj] = (a.active == nullptr || a.active[r] != 0) ? jj : -1;
  }
  for (int k = t.tid; k < ntile; k += nthr) {
    const int j = k / tps;
    tb.tile[k] = (j << 16) | ((k - j * tps) * 8);
  }
  const int lane = t.tid & 31, warp = t.tid >> 5;
  if (warp < nwarp && lane == 0) {
    mbar_init(&bars[2 * warp], 1);
    mbar_init(&bars[2 * warp + 1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool skip = si.err != nullptr && *(volatile int*)si.err != 0;
  if (warp < nwarp && !skip) {
    const int g = lane >> 2, c = lane & 3;
    const uint32_t upm = (uint32_t)upb;
    const bool dag = a.dagger != 0;
    const long nsite = (a.g.Vh - h0) < tl.nsb ? (a.g.Vh - h0) : tl.nsb;
    const int nvalid = (int)nsite * tps;
    uint64_t* wb = &bars[2 * warp];
    unsigned char* wbuf = bufs + (size_t)warp * 2 * kMmaBuf;
    const uint32_t lbase = (uint32_t)((1 - a.out_par) * a.g.Vh);
    // 24 lanes issue the copies of one tile into buffer bi
    auto issue = [&](int tile, int bi) {
      const int tj = tb.tile[tile];
      const int j = tj >> 16, u0 = tj & 0xffff;
      if (lane == 0) mbar_expect_tx(&wb[bi], kMmaBuf + si.extra_tx);
      __syncwarp();
      if (lane < 24) {
        const int d = lane / 3, kind = lane - 3 * (lane / 3);
        const uint32_t un0 = (uint32_t)tb.nb[8 * j + d] * upm + (uint32_t)u0;
        unsigned char* dst = wbuf + (size_t)bi * kMmaBuf;
        if (kind == 0) {
          bulk_g2s(dst + d * 384, a.in + (size_t)un0 * 24u, 384u, &wb[bi]);
        } else if (kind == 1) {
          bulk_g2s(dst + 8 * 384 + d * 32, a.in_nrm + un0, 32u, &wb[bi]);
        } else {
          const int mu = d >> 1;
          const uint32_t link = (d & 1) ? (lbase + (uint32_t)tb.nb[8 * j + d]) * 4u + mu
                                        : (uint32_t)((a.out_par * a.g.Vh + h0 + j) * 4 + mu);
          bulk_g2s(dst + 8 * (384 + 32) + d * 128, frag + ((size_t)link * 2u + (d & 1)) * 32u, 128u, &wb[bi]);
        }
      }
    };
    unsigned par0 = 0, par1 = 0;
    int k = 0;
    int tile = warp;
    if (tile < nvalid) issue(tile, 0);
    for (; tile < nvalid; tile += nwarp, k++) {
      const int bi = k & 1;
      const int nxt = tile + nwarp;
      if (nxt < nvalid) {
        __syncwarp();                                   // buffer 1 - bi was read by every lane
        issue(nxt, bi ^ 1);
      }
      const unsigned par = bi ? par1 : par0;
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&wb[bi], par, si.budget));
      if (bi) par1 ^= 1u; else par0 ^= 1u;
      if (!ok) {
        if (lane == 0) {
          if (si.err) atomicExch(si.err, MDWF_TIMEOUT_CODE);
          if (nxt < nvalid) mbar_wait_bounded(&wb[bi ^ 1], bi ? par0 : par1, si.budget);
        }
        __syncwarp();
        break;
      }
      const int tj = tb.tile[tile];
      const int j = tj >> 16;
      const int jj = (tj & 0xffff) + g;
      const bool live = c < 3 && tb.off[jj] >= 0;
      const unsigned char* src = wbuf + (size_t)bi * kMmaBuf;
      const uint4* qs = reinterpret_cast<const uint4*>(src);
      const float* scs = reinterpret_cast<const float*>(src + 8 * 384);
      const uint32_t* fs = reinterpret_cast<const uint32_t*>(src + 8 * (384 + 32));
      const float* kb = tb.kb + 8 * j;
      uint4 q[8];
      float sc[8];
      uint32_t b[8];
#pragma unroll
      for (int d = 0; d < 8; d++) {
        q[d] = live ? qs[d * 24 + g * 3 + c] : make_uint4(0u, 0u, 0u, 0u);
        sc[d] = live ? scs[d * 8 + g] : 0.f;
        b[d] = fs[d * 32 + lane];
      }
      float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      mma_term<0, true>(q[0], sc[0], b[0], dag, kb[0], acc);
      mma_term<0, false>(q[1], sc[1], b[1], dag, kb[1], acc);
      mma_term<1, true>(q[2], sc[2], b[2], dag, kb[2], acc);
      mma_term<1, false>(q[3], sc[3], b[3], dag, kb[3], acc);
      mma_term<2, true>(q[4], sc[4], b[4], dag, kb[4], acc);
      mma_term<2, false>(q[5], sc[5], b[5], dag, kb[5], acc);
      mma_term<3, true>(q[6], sc[6], b[6], dag, kb[6], acc);
      mma_term<3, false>(q[7], sc[7], b[7], dag, kb[7], acc);
      if (live) {
        float* row = sA + (size_t)(j * upb + jj) * kPadF + 2 * c;
#pragma unroll
        for (int sp = 0; sp < 4; sp++) {
          row[6 * sp] = acc[2 * sp];
          row[6 * sp + 1] = acc[2 * sp + 1];
        }
      }
    }
  }
  epilogue<__half, float, EPI, true>(a, tl, t, nullptr, sA);
}

size_t mma_bulk_smem_bytes(const Tiling& t, int L5) {
  const size_t nwarp = (size_t)t.threads / 32;
  size_t base = (size_t)t.threads * kPadF * sizeof(float);
  if (base < (size_t)t.threads * sizeof(double)) base = (size_t)t.threads * sizeof(double);
  const size_t upb = (size_t)L5 * t.rt, tps = (upb + 7) / 8;
  return ((nwarp * 16 + 127) & ~(size_t)127) + nwarp * 2 * kMmaBuf + base +
         (size_t)t.nsb * 8 * (sizeof(int) + sizeof(float)) + upb * sizeof(int) + t.nsb * tps * sizeof(int);
}

bool mma_bulk_usable(const FastArgs<__half, float>& a, const Tiling& t) {
  const int upb = a.L5 * a.N;
  return t.rt == a.N && t.ngroups == 1 && upb % 8 == 0 && upb % 4 == 0 && t.threads >= 32 && upb < 65536 &&
         ((uintptr_t)a.in % 16) == 0 && ((uintptr_t)a.in_nrm % 16) == 0 && ((uintptr_t)a.F16 % 16) == 0 &&
         mma_bulk_smem_bytes(t, a.L5) <= 220 * 1024;
}

template <int EPI>
cudaError_t launch_mma_bulk_one(const FastArgs<__half, float>& a, const Tiling& t, const StageInfo& si,
                                cudaStream_t st) {
  const dim3 grid((unsigned)t.ntiles, (unsigned)t.ngroups);
  const dim3 block((unsigned)t.rt, (unsigned)a.L5, (unsigned)t.nsb);
  const size_t smem = mma_bulk_smem_bytes(t, a.L5);
  cudaError_t e = cudaFuncSetAttribute(hop_mma_bulk_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  hop_mma_bulk_kernel<EPI><<<grid, block, smem, st>>>(a, t, a.F16, si);
  return cudaGetLastError();
}

// Tensor-core hop, thread-per-unit form.  Threads load and project their own
// unit as the CUDA-core hop does (three 16-byte words per neighbour: the fastest
// gather), write the projected half spinors (fp16) and the neighbour's scale to
// a per-warp buffer in shared memory, and the warp reads them back in mma
// fragment order: one m16n8k8 per 8-unit tile (rows = the two projected halves
// of a unit, B = the link fragment of the tile's site), reconstructed in FP32
// with the unit's scale by the lane that holds colour c of unit g.  Needs whole
// warps and 8-unit tiles inside one site (L5 rt a multiple of 8).
constexpr int kTpuWords = 32 * 4;                    // per warp: 32 units x (3 colour pairs + scale), 8-byte words

template <int MU>
__device__ __forceinline__ void project_pairs(const uint4 q[3], bool neg_sg, uint2* out) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    uint32_t h0, h1;
    mma_project<MU>(q[c], neg_sg, h0, h1);
    out[c] = make_uint2(h0, h1);
  }
}

template <int MU, bool FWD>
__device__ __forceinline__ void tpu_term(const FastArgs<__half, float>& a, const uint32_t* __restrict__ frag,
                                         const int* nbw, int hn, bool bflip, bool act, long un, uint2* wb, int lane,
                                         int g, int c, bool dag, long lf_or_base, float* acc) {
  // 1. own unit: load, project, publish
  uint4 q[3] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
  float sc = 0.f;
  if (act) {
    const uint4* p = reinterpret_cast<const uint4*>(a.in) + un * 3;
    q[0] = __ldg(p);
    q[1] = __ldg(p + 1);
    q[2] = __ldg(p + 2);
    sc = __ldg(a.in_nrm + un);
  }
  const bool neg_sg = FWD ? !dag : dag;
  uint2 pr[3];
  project_pairs<MU>(q, neg_sg, pr);
  __syncwarp();
  wb[lane * 4 + 0] = pr[0];
  wb[lane * 4 + 1] = pr[1];
  wb[lane * 4 + 2] = pr[2];
  reinterpret_cast<float*>(wb + lane * 4 + 3)[0] = bflip ? -sc : sc;
  __syncwarp();
  // 2. four 8-unit tiles: lane (g, c) holds colour c of unit 8 t + g
#pragma unroll
  for (int t = 0; t < 4; t++) {
    const int u = 8 * t + g;
    const uint2 hv = c < 3 ? wb[u * 4 + c] : make_uint2(0u, 0u);
    const float f = reinterpret_cast<const float*>(wb + u * 4 + 3)[0] * a.kappa;
    // link of the tile's site: forward U_mu(x), backward U_mu(x - mu)^+ (nbw: the tile's site neighbour)
    const long link = (lf_or_base + nbw[t]) * 4 + MU;
    const uint32_t b = __ldg(frag + (link * 2 + (FWD ? 0 : 1)) * 32 + lane);
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    mma_m16n8k8(hv.x, hv.y, b, d);
    mma_reconstruct<MU>(d, f, neg_sg ? -f : f, acc + 8 * t);
  }
}

template <int EPI>
__global__ void hop_tpu_kernel(FastArgs<__half, float> a, Tiling tl, const uint32_t* __restrict__ frag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sA = reinterpret_cast<float*>(smem_raw);
  const Thr t = thread_of(a, tl);
  const int nthr = tl.threads;
  size_t base = (size_t)nthr * kPadF * sizeof(float);
  if (base < (size_t)nthr * sizeof(double)) base = (size_t)nthr * sizeof(double);
  int* sNb = reinterpret_cast<int*>(smem_raw + base);                          // [nsb][8] (bit 31: boundary)
  uint2* sW = reinterpret_cast<uint2*>(smem_raw + base + (((size_t)tl.nsb * 8 * sizeof(int) + 15) & ~(size_t)15));
  const long h0 = (long)blockIdx.x * tl.nsb;
  for (int k = t.tid; k < 8 * tl.nsb; k += nthr) {
    const int j = k >> 3, d = k & 7;
    int v = 0;
    if (h0 + j < a.g.Vh) {
      const Site x = make_site(a.g, a.out_par, h0 + j);
      v = nbr_half_any(a.g, x, d);
      if (a.antiperiodic && ((d == 6 && x.c[3] == a.g.L[3] - 1) || (d == 7 && x.c[3] == 0))) v |= (int)0x80000000u;
    }
    sNb[k] = v;
  }
  __syncthreads();
  const int lane = t.tid & 31, warp = t.tid >> 5;
  const int g = lane >> 2, c = lane & 3;
  uint2* wb = sW + (size_t)warp * kTpuWords;
  const bool dag = a.dagger != 0;
  const int upb = a.L5 * tl.rt;
  // the site (block-local) of each of the warp's four tiles, and of this thread's unit
  int tsite[4];
#pragma unroll
  for (int q = 0; q < 4; q++) tsite[q] = (warp * 32 + 8 * q) / upb;
  const int* nb = sNb + 8 * t.site_l;
  const long un_base = (long)t.s * a.N + t.r;
  const long upm = (long)a.L5 * a.N;
  const bool act = t.act;
  float acc[32];
#pragma unroll
  for (int i = 0; i < 32; i++) acc[i] = 0.f;
  const long pf = (long)a.out_par * a.g.Vh + h0;           // forward links: site h0 + tsite
  const long pb = (long)(1 - a.out_par) * a.g.Vh;          // backward links: neighbour site
#define MDWF_TPU_DIR(D, MUV, FWDV)                                                                              \
  {                                                                                                             \
    const int raw = nb[D];                                                                                      \
    const int hn = raw & 0x7fffffff;                                                                           \
    int nbw[4];                                                                                                 \
    _Pragma("unroll") for (int q = 0; q < 4; q++)                                                              \
        nbw[q] = FWDV ? (h0 + tsite[q] < a.g.Vh ? tsite[q] : 0) : (sNb[8 * tsite[q] + D] & 0x7fffffff);           \
    tpu_term<MUV, FWDV>(a, frag, nbw, hn, raw < 0, act, (long)hn * upm + un_base, wb, lane, g, c, dag,            \
                        FWDV ? pf : pb, acc);                                                                    \
  }
  MDWF_TPU_DIR(0, 0, true)
  MDWF_TPU_DIR(1, 0, false)
  MDWF_TPU_DIR(2, 1, true)
  MDWF_TPU_DIR(3, 1, false)
  MDWF_TPU_DIR(4, 2, true)
  MDWF_TPU_DIR(5, 2, false)
  MDWF_TPU_DIR(6, 3, true)
  MDWF_TPU_DIR(7, 3, false)
#undef MDWF_TPU_DIR
  // lane (g, c) writes colour c of units 8 t + g into the epilogue tile
  if (c < 3) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      float* row = sA + (size_t)(warp * 32 + 8 * q + g) * kPadF + 2 * c;
#pragma unroll
      for (int sp = 0; sp < 4; sp++) {
        row[6 * sp] = acc[8 * q + 2 * sp];
        row[6 * sp + 1] = acc[8 * q + 2 * sp + 1];
      }
    }
  }
  epilogue<__half, float, EPI, true>(a, tl, t, nullptr, sA);
}

size_t tpu_smem_bytes(const Tiling& t) {
  size_t base = (size_t)t.threads * kPadF * sizeof(float);
  if (base < (size_t)t.threads * sizeof(double)) base = (size_t)t.threads * sizeof(double);
  return base + (((size_t)t.nsb * 8 * sizeof(int) + 15) & ~(size_t)15) + (size_t)(t.threads / 32) * kTpuWords * 8;
}

bool tpu_usable(const Tiling& t, int L5) {
  return t.threads % 32 == 0 && (L5 * t.rt) % 8 == 0 && tpu_smem_bytes(t) <= 200 * 1024;
}

template <int EPI>
cudaError_t launch_tpu_one(const FastArgs<__half, float>& a, const Tiling& t, cudaStream_t st) {
  const dim3 grid((unsigned)t.ntiles, (unsigned)t.ngroups);
  const dim3 block((unsigned)t.rt, (unsigned)a.L5, (unsigned)t.nsb);
  const size_t smem = tpu_smem_bytes(t);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(hop_tpu_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  hop_tpu_kernel<EPI><<<grid, block, smem, st>>>(a, t, a.F16);
  return cudaGetLastError();
}

size_t mma_smem_bytes(const Tiling& t, int L5) {
  size_t base = (size_t)t.threads * kPadF * sizeof(float);
  if (base < (size_t)t.threads * sizeof(double)) base = (size_t)t.threads * sizeof(double);
  const size_t upb = (size_t)L5 * t.rt, tps = (upb + 7) / 8;
  return base + (size_t)t.nsb * 8 * (sizeof(int) + sizeof(float)) + upb * sizeof(int) + t.nsb * tps * sizeof(int);
}

template <int EPI>
cudaError_t launch_mma_one(const FastArgs<__half, float>& a, const Tiling& t, const uint32_t* frag, cudaStream_t st) {
  const dim3 grid((unsigned)t.ntiles, (unsigned)t.ngroups);
  const dim3 block((unsigned)t.rt, (unsigned)a.L5, (unsigned)t.nsb);
  const size_t smem = mma_smem_bytes(t, a.L5);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(hop_mma_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  hop_mma_kernel<EPI><<<grid, block, smem, st>>>(a, t, frag);
  return cudaGetLastError();
}

// B fragments of every link: word (link, backward, lane) for lane (g, c) holds
// rows 2c, 2c+1 and column g of the real form of W = U (forward) or U^+ (backward).
__global__ void k_link_frags(const double* __restrict__ U, uint32_t* __restrict__ frag, long nlinks) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlinks * 64) return;
  const int lane = (int)(i & 31), bwd = (int)((i >> 5) & 1);
  const long link = i >> 6;
  const int g = lane >> 2, c = lane & 3, ca = g >> 1;
  float lo = 0.f, hi = 0.f;
  if (c < 3 && ca < 3) {
    // W_ab, a = ca, b = c: U_ab forward, conj(U_ba) backward
    const double* e = U + link * 18 + 2 * (bwd ? c * 3 + ca : ca * 3 + c);
    const double re = e[0], im = bwd ? -e[1] : e[1];
    if (g & 1) { lo = (float)im; hi = (float)re; }
    else { lo = (float)re; hi = (float)-im; }
  }
  const __half2 v = __floats2half2_rn(lo, hi);
  frag[i] = *reinterpret_cast<const uint32_t*>(&v);
}

}  // namespace

template <typename S, typename T>
size_t staged_smem_bytes(const Tiling& t, int L5, int N) {
  if (t.rt != N || t.ngroups != 1) return 0;
  return staged_bytes<S, T>(t, L5, N, nullptr, nullptr);
}

template <typename S, typename T>
cudaError_t launch_fast(const FastArgs<S, T>& a, const Tiling& t, int epi, cudaStream_t st, const StageInfo* stage) {
  if (stage && (t.rt != a.N || t.ngroups != 1 || a.in == nullptr)) stage = nullptr;
  if constexpr (std::is_same<T, float>::value) {
    if (stage == nullptr && (t.form == 0 || t.form == 2)) return launch_pair<S>(a, t.nsb, epi, st, t.form == 2);
  }
  switch (epi) {
    case E_SAME_AINV: return launch_one<S, T, E_SAME_AINV>(a, t, st, stage);
    case E_SAME_BD: return launch_one<S, T, E_SAME_BD>(a, t, st, stage);
    case E_AINVD_SAME: return launch_one<S, T, E_AINVD_SAME>(a, t, st, stage);
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
             max_threads_one<S, T, E_AINV_SAME>(), max_threads_one<S, T, E_SAME_AINV>(),
             max_threads_one<S, T, E_SAME_BD>(), max_threads_one<S, T, E_AINVD_SAME>()};
  for (int x : v) m = x < m ? x : m;
  return m;
}

bool mma_hop_usable(const Tiling& t, int L5, int N) {
  // at least one whole warp per block; 8-unit tiles never straddle sites
  return t.threads >= 32 && mma_smem_bytes(t, L5) <= 200 * 1024 && N >= 1 && L5 >= 1;
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

cudaError_t launch_fast_mma(const FastArgs<__half, float>& a, const Tiling& t, int epi, cudaStream_t st,
                            const StageInfo* stage, bool pipelined) {
  if (!mma_hop_usable(t, a.L5, a.N) || a.F16 == nullptr) return cudaErrorInvalidValue;
  if (pipelined && stage != nullptr && mma_bulk_usable(a, t)) {
    switch (epi) {
      case E_RAW: return launch_mma_bulk_one<E_RAW>(a, t, *stage, st);
      case E_BAINV: return launch_mma_bulk_one<E_BAINV>(a, t, *stage, st);
      case E_AINVD_BD: return launch_mma_bulk_one<E_AINVD_BD>(a, t, *stage, st);
      case E_A_SAME: return launch_mma_bulk_one<E_A_SAME>(a, t, *stage, st);
      case E_AD_SAME_BD: return launch_mma_bulk_one<E_AD_SAME_BD>(a, t, *stage, st);
      case E_AINV_SAME: return launch_mma_bulk_one<E_AINV_SAME>(a, t, *stage, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (!pipelined && tpu_usable(t, a.L5)) {
    switch (epi) {
      case E_RAW: return launch_tpu_one<E_RAW>(a, t, st);
      case E_BAINV: return launch_tpu_one<E_BAINV>(a, t, st);
      case E_AINVD_BD: return launch_tpu_one<E_AINVD_BD>(a, t, st);
      case E_A_SAME: return launch_tpu_one<E_A_SAME>(a, t, st);
      case E_AD_SAME_BD: return launch_tpu_one<E_AD_SAME_BD>(a, t, st);
      case E_AINV_SAME: return launch_tpu_one<E_AINV_SAME>(a, t, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (epi) {
    case E_RAW: return launch_mma_one<E_RAW>(a, t, a.F16, st);
    case E_BAINV: return launch_mma_one<E_BAINV>(a, t, a.F16, st);
    case E_AINVD_BD: return launch_mma_one<E_AINVD_BD>(a, t, a.F16, st);
    case E_A_SAME: return launch_mma_one<E_A_SAME>(a, t, a.F16, st);
    case E_AD_SAME_BD: return launch_mma_one<E_AD_SAME_BD>(a, t, a.F16, st);
    case E_AINV_SAME: return launch_mma_one<E_AINV_SAME>(a, t, a.F16, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t build_link_frags(const double* U64, uint32_t* frag, long nlinks, cudaStream_t st) {
  const long n = nlinks * 64;
  k_link_frags<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U64, frag, nlinks);
  return cudaGetLastError();
}

// Faces of a time-split lattice: thread per unit of one parity field; the
// projection and U^+ multiply are those of the receiving side's hop_term_at.
__global__ void k_dd_pack(const double* __restrict__ in, Geom g, int par, int L5, int N, int dagger,
                          const double* __restrict__ U, double* __restrict__ face_prev,
                          double* __restrict__ face_next) {
  const long u = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= g.Vh * L5 * N) return;
  const long h = u / ((long)L5 * N);
  const int rem = (int)(u - h * L5 * N);
  const int s = rem / N, r = rem - s * N;
  const Site x = make_site(g, par, h);
  const bool first = x.c[3] == 0, last = x.c[3] == g.L[3] - 1;
  if (!first && !last) return;
  const long lex3 = x.lex - (long)x.c[3] * x.stride[3];
  double psi[24], hh[12];
  load24<double, double>(in, nullptr, u, psi);
  const double dg = dagger ? 1.0 : -1.0;
  if (first) {        // the previous sub-domain's forward term: sg = dg
    project<3, double>(psi, dg, hh);
    double* o = face_prev + ((lex3 * L5 + s) * N + r) * 12;
#pragma unroll
    for (int i = 0; i < 12; i++) o[i] = hh[i];
  }
  if (last) {         // the next sub-domain's backward term: sg = -dg, then U_t(x)^+
    double l[18], chi[12];
    project<3, double>(psi, -dg, hh);
    load_link<double>(U, ((long)par * g.Vh + h) * 4 + 3, l);
    su3_mul<double, true>(l, hh, chi);
    su3_mul<double, true>(l, hh + 6, chi + 6);
    double* o = face_next + ((lex3 * L5 + s) * N + r) * 12;
#pragma unroll
    for (int i = 0; i < 12; i++) o[i] = chi[i];
  }
}

cudaError_t dd_pack_faces(const double* in, const Geom& g, int par, int L5, int N, int dagger, const double* U,
                          double* face_prev, double* face_next, cudaStream_t st) {
  const long n = g.Vh * L5 * N;
  k_dd_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, g, par, L5, N, dagger, U, face_prev, face_next);
  return cudaGetLastError();
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
