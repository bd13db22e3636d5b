// Wilson hop on all L5 slices x RHS slots with the fifth-dimension epilogues,
// two slices per thread (the default CUDA-core form for FP32 arithmetic).
//
// Thread (r, j, site) computes the units (site, s0 = 2j, r) and (site, s0 + 1, r)
// as the two lanes of packed FP32 values (float2, one FFMA2 per pair of FMAs):
// both units share the site, so the neighbour indices, the time-boundary phase
// and each of the eight links are computed or loaded once for the two.  The
// colour multiply W h (W = U_mu(x) forward, U_mu(x - mu)^+ backward) and the
// spin reconstruction are done row by row so that only one colour of the
// product is live.  The epilogues are those of hop_fast.cu (E_RAW ... E_AINVD_SAME,
// see there); their fifth-dimension recursions run on pairs of columns of a
// shared-memory tile, again as packed FP32.
//
// Every operation has an explicit rounding (fma.rn / mul.rn / add.rn, packed or
// scalar), so a unit's result does not depend on the block shape or on which
// lane of a pair it occupies: every tiling of this kernel gives the same bits.
//
// Prefetching form (fp16 storage, 18-real links): the block's eight links per
// site are copied to shared memory once, and each thread streams its neighbour
// pairs through a two-stage buffer of its own in shared memory with
// asynchronous copies (cp.async), issuing the loads of direction k + 2 while it
// computes direction k.  The arithmetic is the same, in the same order, so it
// gives the same bits as the plain form.
#include <type_traits>

#include "mdwf_internal.h"
#include "hop_common.cuh"

namespace mdwf {

namespace {

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Spin projection h = psi_up + sg e_mu psi_lo of a packed spinor p[24]
// ([spin][colour][re, im]); e_x = i sigma_x, e_y = -i sigma_y, e_z = i sigma_z,
// e_t = 1 (DeGrand-Rossi basis).  sg = +-1, so every product is exact.
template <int MU>
__device__ __forceinline__ void project2(const float2* p, float sg, float2* h) {
  const float2 ps = f2(sg), ms = f2(-sg);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const float2* p0 = p + 2 * c;
    const float2* p1 = p + 6 + 2 * c;
    const float2* p2 = p + 12 + 2 * c;
    const float2* p3 = p + 18 + 2 * c;
    float2* h0 = h + 2 * c;
    float2* h1 = h + 6 + 2 * c;
    if (MU == 0) {
      h0[0] = fma2(ms, p3[1], p0[0]); h0[1] = fma2(ps, p3[0], p0[1]);
      h1[0] = fma2(ms, p2[1], p1[0]); h1[1] = fma2(ps, p2[0], p1[1]);
    } else if (MU == 1) {
      h0[0] = fma2(ms, p3[0], p0[0]); h0[1] = fma2(ms, p3[1], p0[1]);
      h1[0] = fma2(ps, p2[0], p1[0]); h1[1] = fma2(ps, p2[1], p1[1]);
    } else if (MU == 2) {
      h0[0] = fma2(ms, p2[1], p0[0]); h0[1] = fma2(ps, p2[0], p0[1]);
      h1[0] = fma2(ps, p3[1], p1[0]); h1[1] = fma2(ms, p3[0], p1[1]);
    } else {
      h0[0] = fma2(ps, p2[0], p0[0]); h0[1] = fma2(ps, p2[1], p0[1]);
      h1[0] = fma2(ps, p3[0], p1[0]); h1[1] = fma2(ps, p3[1], p1[1]);
    }
  }
}

// Load and project the neighbour spinors of both units (uA, uB); f receives the
// factor of each projected spinor (the fp16 storage scale; 1 otherwise).
template <int MU, typename S>
struct PairProj {
  static __device__ __forceinline__ void run(const S* __restrict__ v, const float* __restrict__ nrm, long uA, long uB,
                                             float sg, float2* h, float2& f) {
    float pa[24], pb[24];
    load24<S, float>(v, nrm, uA, pa);
    load24<S, float>(v, nrm, uB, pb);
    float2 p[24];
#pragma unroll
    for (int i = 0; i < 24; i++) p[i] = make_float2(pa[i], pb[i]);
    project2<MU>(p, sg, h);
    f = f2(1.f);
  }
};
template <int MU>
struct PairProj<MU, __half> {
  static __device__ __forceinline__ void run(const __half* __restrict__ v, const float* __restrict__ nrm, long uA,
                                             long uB, float sg, float2* h, float2& f) {
    const uint4* pa = reinterpret_cast<const uint4*>(v + 24 * uA);
    const uint4* pb = reinterpret_cast<const uint4*>(v + 24 * uB);
    uint4 qa[3], qb[3];
    qa[0] = __ldg(pa); qa[1] = __ldg(pa + 1); qa[2] = __ldg(pa + 2);
    qb[0] = __ldg(pb); qb[1] = __ldg(pb + 1); qb[2] = __ldg(pb + 2);
    float ha[12], hb[12];
    project_half<MU>(qa, sg, ha);
    project_half<MU>(qb, sg, hb);
#pragma unroll
    for (int i = 0; i < 12; i++) h[i] = make_float2(ha[i], hb[i]);
    f = make_float2(__ldg(nrm + uA), __ldg(nrm + uB));
  }
};

// acc += reconstruction of W h, colour row by colour row.  h[12]: the projected
// half spinor (spins 0, 1 of [spin][colour][re, im]); f: factor of h, fs = f sg.
template <int MU, bool DAG>
__device__ __forceinline__ void mul_recon(const float* l, const float2* h, float2 f, float2 fs, float2* acc) {
  const float2 nfs = neg2(fs);
#pragma unroll
  for (int a = 0; a < 3; a++) {
    float2 x0r, x0i, x1r, x1i;
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const int k = DAG ? (3 * b + a) : (3 * a + b);
      const float2 ur = f2(l[2 * k]);
      const float2 ui = f2(DAG ? -l[2 * k + 1] : l[2 * k + 1]);
      const float2 nui = f2(DAG ? l[2 * k + 1] : -l[2 * k + 1]);
      if (b == 0) {
        x0r = mul2(ur, h[0]); x0i = mul2(ur, h[1]);
        x1r = mul2(ur, h[6]); x1i = mul2(ur, h[7]);
      } else {
        x0r = fma2(ur, h[2 * b], x0r); x0i = fma2(ur, h[2 * b + 1], x0i);
        x1r = fma2(ur, h[6 + 2 * b], x1r); x1i = fma2(ur, h[6 + 2 * b + 1], x1i);
      }
      x0r = fma2(nui, h[2 * b + 1], x0r); x0i = fma2(ui, h[2 * b], x0i);
      x1r = fma2(nui, h[6 + 2 * b + 1], x1r); x1i = fma2(ui, h[6 + 2 * b], x1i);
    }
    float2* a0 = acc + 2 * a;
    float2* a1 = acc + 6 + 2 * a;
    float2* a2 = acc + 12 + 2 * a;
    float2* a3 = acc + 18 + 2 * a;
    a0[0] = fma2(f, x0r, a0[0]); a0[1] = fma2(f, x0i, a0[1]);
    a1[0] = fma2(f, x1r, a1[0]); a1[1] = fma2(f, x1i, a1[1]);
    if (MU == 0) {
      a2[0] = fma2(fs, x1i, a2[0]); a2[1] = fma2(nfs, x1r, a2[1]);
      a3[0] = fma2(fs, x0i, a3[0]); a3[1] = fma2(nfs, x0r, a3[1]);
    } else if (MU == 1) {
      a2[0] = fma2(fs, x1r, a2[0]); a2[1] = fma2(fs, x1i, a2[1]);
      a3[0] = fma2(nfs, x0r, a3[0]); a3[1] = fma2(nfs, x0i, a3[1]);
    } else if (MU == 2) {
      a2[0] = fma2(fs, x0i, a2[0]); a2[1] = fma2(nfs, x0r, a2[1]);
      a3[0] = fma2(nfs, x1i, a3[0]); a3[1] = fma2(fs, x1r, a3[1]);
    } else {
      a2[0] = fma2(fs, x0r, a2[0]); a2[1] = fma2(fs, x0i, a2[1]);
      a3[0] = fma2(fs, x1r, a3[0]); a3[1] = fma2(fs, x1i, a3[1]);
    }
  }
}

// Two-row (12-real) link: rows 0 and 1 are loaded (three 16-byte words), row 2
// of an SU(3) matrix is the complex conjugate of their cross product,
// W_2j = conj(W_0k W_1l - W_0l W_1k) for (j, k, l) cyclic; the time-boundary
// phase is a separate sign, so every stored link has determinant 1.
__device__ __forceinline__ void load_link12(const float* __restrict__ U12, long idx, float l[18]) {
  const float4* p = reinterpret_cast<const float4*>(U12 + 12 * idx);
  const float4 t0 = __ldg(p), t1 = __ldg(p + 1), t2 = __ldg(p + 2);
  l[0] = t0.x; l[1] = t0.y; l[2] = t0.z; l[3] = t0.w;
  l[4] = t1.x; l[5] = t1.y; l[6] = t1.z; l[7] = t1.w;
  l[8] = t2.x; l[9] = t2.y; l[10] = t2.z; l[11] = t2.w;
#pragma unroll
  for (int j = 0; j < 3; j++) {
    const int k = (j + 1) % 3, m = (j + 2) % 3;
    const float akr = l[2 * k], aki = l[2 * k + 1], amr = l[2 * m], ami = l[2 * m + 1];
    const float bkr = l[6 + 2 * k], bki = l[6 + 2 * k + 1], bmr = l[6 + 2 * m], bmi = l[6 + 2 * m + 1];
    // c = a_k b_m - a_m b_k
    const float cr = __fmaf_rn(akr, bmr, __fmaf_rn(-aki, bmi, __fmaf_rn(-amr, bkr, __fmul_rn(ami, bki))));
    const float ci = __fmaf_rn(akr, bmi, __fmaf_rn(aki, bmr, __fmaf_rn(-amr, bki, -__fmul_rn(ami, bkr))));
    l[12 + 2 * j] = cr;
    l[12 + 2 * j + 1] = -ci;
  }
}

// Thread coordinates of the (rt, J, nsb) block, J = ceil(L5 / 2).
struct PThr {
  int r_l, j, site_l, row;   // row: the thread's row of the epilogue tile
  long h;
  int r, s0;
  bool two;                  // slice s0 + 1 exists
  bool valid, act;
  long u0;                   // unit of slice s0; slice s0 + 1 is u0 + N
};

template <typename S>
__device__ __forceinline__ PThr pair_thread(const FastArgs<S, float>& a) {
  PThr t;
  t.r_l = threadIdx.x;
  t.j = threadIdx.y;
  t.site_l = threadIdx.z;
  t.row = (t.site_l * blockDim.y + t.j) * blockDim.x + t.r_l;
  t.h = (long)blockIdx.x * blockDim.z + t.site_l;
  t.r = blockIdx.y * blockDim.x + t.r_l;
  t.s0 = 2 * t.j;
  t.two = t.s0 + 1 < a.L5;
  t.valid = (t.h < a.g.Vh) && (t.r < a.N);
  t.act = t.valid && (a.active == nullptr || a.active[t.r] != 0);
  t.u0 = t.valid ? (t.h * a.L5 + t.s0) * a.N + t.r : 0;
  return t;
}

template <int MU, bool FWD, typename S, bool R12>
__device__ __forceinline__ void pair_term(const FastArgs<S, float>& a, const Site& x, const PThr& t, float2* acc) {
  const float sg = (a.dagger ? 1.f : -1.f) * (FWD ? 1.f : -1.f);
  const int hn = nbr_half<MU, FWD>(a.g, x);
  const bool bflip = MU == 3 && a.antiperiodic && (FWD ? x.c[3] == a.g.L[3] - 1 : x.c[3] == 0);
  const long uA = ((long)hn * a.L5 + t.s0) * a.N + t.r;
  const long uB = t.two ? uA + a.N : uA;
  float2 hh[12], f;
  PairProj<MU, S>::run(a.in, a.in_nrm, uA, uB, sg, hh, f);
  if (bflip) f = neg2(f);
  const float2 fs = mul2(f, f2(sg));
  float l[18];
  const long li = FWD ? ((long)a.out_par * a.g.Vh + t.h) * 4 + MU : ((long)(1 - a.out_par) * a.g.Vh + hn) * 4 + MU;
  if (R12) load_link12(a.U12, li, l);
  else load_link<float>(a.U, li, l);
  if (FWD) mul_recon<MU, false>(l, hh, f, fs, acc);
  else mul_recon<MU, true>(l, hh, f, fs, acc);
}

// ---------------------------------------------------------------------------
// Epilogue tile: row (site, j, r) holds the 24 components of the thread's two
// slices interleaved, [component][slice parity], in kRS floats (16-byte rows).
// ---------------------------------------------------------------------------
constexpr int kRS = 52;

__device__ __forceinline__ int tile_row(int site_l, int j, int r_l) {
  return (site_l * (int)blockDim.y + j) * (int)blockDim.x + r_l;
}
// Component c of slice s of (site_l, r_l).
__device__ __forceinline__ float& tile_at(float* tile, int site_l, int r_l, int s, int c) {
  return tile[(size_t)tile_row(site_l, s >> 1, r_l) * kRS + 2 * c + (s & 1)];
}

// A^-1 along a pair of columns held as v[k], k along the recursion direction
// (A = alpha + beta S, wall factor -m):  z_k = x_k / alpha - kappa z_{k-1},
// y_{L-1} = z_{L-1} / (1 + m (-kappa)^L), y_k = z_k - m (-kappa)^{k+1} y_{L-1}.
struct Rec {
  float2 ia, nkap, mk, b5, c5, m, nm;
  float den;
};
template <int L>
__device__ __forceinline__ void ainv_v(float2* v, const Rec& c) {
  float2 z = f2(0.f);
#pragma unroll
  for (int k = 0; k < L; k++) { z = fma2(c.nkap, z, mul2(v[k], c.ia)); v[k] = z; }
  const float2 yl = make_float2(__fdiv_rn(z.x, c.den), __fdiv_rn(z.y, c.den));
  v[L - 1] = yl;
  float2 w = mul2(mul2(c.m, yl), c.mk);
#pragma unroll
  for (int k = 0; k < L - 1; k++) { v[k] = add2(v[k], neg2(w)); w = mul2(w, c.mk); }
}
// B = b5 + c5 S along the column: y_k = b5 x_k + c5 x_{k-1}, x_{-1} = -m x_{L-1}.
template <int L>
__device__ __forceinline__ void bop_v(float2* v, const Rec& c) {
  float2 prev = mul2(c.nm, v[L - 1]);
#pragma unroll
  for (int k = 0; k < L; k++) { const float2 x = v[k]; v[k] = fma2(c.c5, prev, mul2(c.b5, x)); prev = x; }
}
template <int EPI, int L>
__device__ __forceinline__ void transform_v(float2* v, const Rec& c) {
  if (EPI == E_BAINV) { ainv_v<L>(v, c); bop_v<L>(v, c); }
  else if (EPI == E_AINVD_BD) { bop_v<L>(v, c); ainv_v<L>(v, c); }
  else ainv_v<L>(v, c);
}

// Column pair p (components 2p, 2p + 1; UPPER: p < 6, the P_+ half) of
// (site_l, r_l), compile-time L5.
template <int EPI, int L, bool UPPER>
__device__ __forceinline__ void col_pair(float* tile, int site_l, int r_l, int p, const Rec& c) {
  constexpr int NQ = (L + 1) / 2;
  constexpr bool down = (EPI == E_AINVD_BD || EPI == E_AINVD_SAME) ? !UPPER : UPPER;
  float4 q[NQ];
#pragma unroll
  for (int i = 0; i < NQ; i++)
    q[i] = *reinterpret_cast<const float4*>(tile + (size_t)tile_row(site_l, i, r_l) * kRS + 4 * p);
  float2 v[L];
  if (down) {
#pragma unroll
    for (int s = 0; s < L; s++) v[s] = (s & 1) ? make_float2(q[s >> 1].y, q[s >> 1].w) : make_float2(q[s >> 1].x, q[s >> 1].z);
  } else {
#pragma unroll
    for (int s = 0; s < L; s++) v[L - 1 - s] = (s & 1) ? make_float2(q[s >> 1].y, q[s >> 1].w) : make_float2(q[s >> 1].x, q[s >> 1].z);
  }
  transform_v<EPI, L>(v, c);
#pragma unroll
  for (int s = 0; s < L; s++) {
    const float2 y = down ? v[s] : v[L - 1 - s];
    if (s & 1) { q[s >> 1].y = y.x; q[s >> 1].w = y.y; }
    else { q[s >> 1].x = y.x; q[s >> 1].z = y.y; }
  }
#pragma unroll
  for (int i = 0; i < NQ; i++)
    *reinterpret_cast<float4*>(tile + (size_t)tile_row(site_l, i, r_l) * kRS + 4 * p) = q[i];
}

// The same for a run-time L5, directly on the tile (same operations, same order).
template <int EPI, bool UPPER>
__device__ __forceinline__ void col_pair_any(float* tile, int site_l, int r_l, int p, int L, const Rec& c) {
  constexpr bool down = (EPI == E_AINVD_BD || EPI == E_AINVD_SAME) ? !UPPER : UPPER;
  auto get = [&](int k) {
    const int s = down ? k : L - 1 - k;
    return make_float2(tile_at(tile, site_l, r_l, s, 2 * p), tile_at(tile, site_l, r_l, s, 2 * p + 1));
  };
  auto put = [&](int k, float2 y) {
    const int s = down ? k : L - 1 - k;
    tile_at(tile, site_l, r_l, s, 2 * p) = y.x;
    tile_at(tile, site_l, r_l, s, 2 * p + 1) = y.y;
  };
  auto ainv = [&]() {
    float2 z = f2(0.f);
    for (int k = 0; k < L; k++) { z = fma2(c.nkap, z, mul2(get(k), c.ia)); put(k, z); }
    const float2 yl = make_float2(__fdiv_rn(z.x, c.den), __fdiv_rn(z.y, c.den));
    put(L - 1, yl);
    float2 w = mul2(mul2(c.m, yl), c.mk);
    for (int k = 0; k < L - 1; k++) { put(k, add2(get(k), neg2(w))); w = mul2(w, c.mk); }
  };
  auto bop = [&]() {
    float2 prev = mul2(c.nm, get(L - 1));
    for (int k = 0; k < L; k++) { const float2 x = get(k); put(k, fma2(c.c5, prev, mul2(c.b5, x))); prev = x; }
  };
  if (EPI == E_BAINV) { ainv(); bop(); }
  else if (EPI == E_AINVD_BD) { bop(); ainv(); }
  else ainv();
}

// The column pairs of the thread's (site, RHS) in one half: thread j takes
// p = j, j + J, ... among p = 0..5 (UPPER) or 6..11.
template <int EPI, bool UPPER>
__device__ __forceinline__ void col_pairs(float* tile, const PThr& t, int L5, const Rec& c) {
  const int J = blockDim.y;
  for (int q = t.j; q < 6; q += J) {
    const int p = UPPER ? q : 6 + q;
    switch (L5) {
      case 4: col_pair<EPI, 4, UPPER>(tile, t.site_l, t.r_l, p, c); break;
      case 6: col_pair<EPI, 6, UPPER>(tile, t.site_l, t.r_l, p, c); break;
      case 8: col_pair<EPI, 8, UPPER>(tile, t.site_l, t.r_l, p, c); break;
      case 10: col_pair<EPI, 10, UPPER>(tile, t.site_l, t.r_l, p, c); break;
      case 12: col_pair<EPI, 12, UPPER>(tile, t.site_l, t.r_l, p, c); break;
      case 16: col_pair<EPI, 16, UPPER>(tile, t.site_l, t.r_l, p, c); break;
      default: col_pair_any<EPI, UPPER>(tile, t.site_l, t.r_l, p, L5, c);
    }
  }
}

template <typename S>
__device__ __forceinline__ void load_pair24(const S* v, const float* nrm, const PThr& t, int N, float2* y) {
  float ya[24], yb[24];
  load24<S, float>(v, nrm, t.u0, ya);
  if (t.two) load24<S, float>(v, nrm, t.u0 + N, yb);
#pragma unroll
  for (int i = 0; i < 24; i++) y[i] = make_float2(ya[i], t.two ? yb[i] : 0.f);
}

// A y (dag = false) or A^+ y (dag = true) of the stored field `same` for both
// slices:  P_+ half alpha y_s + beta y_{s-1} (A) / y_{s+1} (A^+), P_- half the
// other neighbour; y_{-1} = -m y_{L5-1}, y_{L5} = -m y_0.
template <typename S>
__device__ __forceinline__ void apply_A_pair(const FastArgs<S, float>& a, const PThr& t, bool dag, float m,
                                             float2* o) {
  const int L5 = a.L5;
  const float al = a.f.alpha, g = a.g_same;
#pragma unroll
  for (int k = 0; k < 2; k++) {
    if (k == 1 && !t.two) break;
    const int s = t.s0 + k;
    const int s_dn = s == 0 ? L5 - 1 : s - 1;
    const int s_up = s == L5 - 1 ? 0 : s + 1;
    const float w_dn = s == 0 ? -m : 1.f;
    const float w_up = s == L5 - 1 ? -m : 1.f;
#pragma unroll
    for (int part = 0; part < 2; part++) {
      // part 0 (P_+): neighbour s - 1 (A) or s + 1 (A^+); part 1 (P_-): the other one
      const bool from_up = (part == 0) == dag;
      const int sn = from_up ? s_up : s_dn;
      const float bw = __fmul_rn(a.f.beta, from_up ? w_up : w_dn);
      float y[12], yn[12];
      load_part<S, float>(a.same, a.same_nrm, (t.h * L5 + s) * a.N + t.r, part, y);
      load_part<S, float>(a.same, a.same_nrm, (t.h * L5 + sn) * a.N + t.r, part, yn);
#pragma unroll
      for (int i = 0; i < 12; i++) {
        const float ay = __fmaf_rn(bw, yn[i], __fmul_rn(al, y[i]));
        float& oi = k == 0 ? o[12 * part + i].x : o[12 * part + i].y;
        oi = __fmaf_rn(g, ay, oi);
      }
    }
  }
}

// Store both units (the second only if it exists).
template <typename S>
__device__ __forceinline__ void store_pair24(S* v, float* nrm, const PThr& t, int N, const float2* o) {
  float oa[24], ob[24];
#pragma unroll
  for (int i = 0; i < 24; i++) { oa[i] = o[i].x; ob[i] = o[i].y; }
  store24<S, float>(v, nrm, t.u0, oa);
  if (t.two) store24<S, float>(v, nrm, t.u0 + N, ob);
}
// fp16: the same values as store24 (the scale is a power of two, so the scaling
// is exact whichever way it is multiplied), with packed multiplies.
template <>
__device__ __forceinline__ void store_pair24<__half>(__half* v, float* nrm, const PThr& t, int N, const float2* o) {
  float ma = 0.f, mb = 0.f;
#pragma unroll
  for (int i = 0; i < 24; i++) { ma = fmaxf(ma, fabsf(o[i].x)); mb = fmaxf(mb, fabsf(o[i].y)); }
  float sa, sb, ia, ib;
  half_scale(ma, &sa, &ia);
  half_scale(mb, &sb, &ib);
  const float2 inv = make_float2(ia, ib);
  float2 q[24];
#pragma unroll
  for (int i = 0; i < 24; i++) q[i] = mul2(o[i], inv);
  uint4 wa[3], wb[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    __half2* ha = reinterpret_cast<__half2*>(&wa[c]);
    __half2* hb = reinterpret_cast<__half2*>(&wb[c]);
#pragma unroll
    for (int k = 0; k < 4; k++) {     // colour-major: word c holds spins 0..3 of colour c
      ha[k] = __floats2half2_rn(q[6 * k + 2 * c].x, q[6 * k + 2 * c + 1].x);
      hb[k] = __floats2half2_rn(q[6 * k + 2 * c].y, q[6 * k + 2 * c + 1].y);
    }
  }
  uint4* pa = reinterpret_cast<uint4*>(v + 24 * t.u0);
  nrm[t.u0] = sa;
  pa[0] = wa[0]; pa[1] = wa[1]; pa[2] = wa[2];
  if (t.two) {
    uint4* pb = reinterpret_cast<uint4*>(v + 24 * (t.u0 + N));
    nrm[t.u0 + N] = sb;
    pb[0] = wb[0]; pb[1] = wb[1]; pb[2] = wb[2];
  }
}

template <typename S, int EPI>
__device__ __forceinline__ void pair_epilogue(const FastArgs<S, float>& a, const PThr& t, const float2* acc,
                                              float* tile) {
  const int L5 = a.L5;
  const float m = t.valid ? a.f.mass[t.r] : 0.f;
  constexpr bool kCols = (EPI == E_BAINV || EPI == E_AINVD_BD || EPI == E_AINV_SAME || EPI == E_SAME_AINV ||
                          EPI == E_AINVD_SAME);
  constexpr bool kSameFirst = (EPI == E_AINV_SAME || EPI == E_AINVD_SAME);
  constexpr bool kBdag = (EPI == E_AD_SAME_BD || EPI == E_SAME_BD);
  const float2 kap = f2(a.kappa);
  float2 o[24];
  if (kCols || kBdag) {
    float2 v[24];
    if (kSameFirst && t.act) {
      float2 y[24];
      load_pair24<S>(a.same, a.same_nrm, t, a.N, y);
#pragma unroll
      for (int i = 0; i < 24; i++) v[i] = fma2(kap, acc[i], y[i]);
    } else {
#pragma unroll
      for (int i = 0; i < 24; i++) v[i] = mul2(kap, acc[i]);
    }
    float2* row = reinterpret_cast<float2*>(tile + (size_t)t.row * kRS);
#pragma unroll
    for (int i = 0; i < 24; i++) row[i] = v[i];
    __syncthreads();
    if (kCols) {
      if (t.act) {
        Rec c;
        c.ia = f2(a.f.inv_alpha); c.nkap = f2(-a.f.kap); c.mk = f2(-a.f.kap);
        c.b5 = f2(a.f.b5); c.c5 = f2(a.f.c5); c.m = f2(m); c.nm = f2(-m);
        c.den = __fmaf_rn(m, a.f.powL, 1.f);
        col_pairs<EPI, true>(tile, t, L5, c);
        col_pairs<EPI, false>(tile, t, L5, c);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 24; i++) o[i] = row[i];
    } else {
      // B^+ (kappa H): P_+ half from slice s + 1, P_- half from slice s - 1
      float cu[2], cl[2];
      int su[2], sd[2];
#pragma unroll
      for (int k = 0; k < 2; k++) {
        const int s = t.two || k == 0 ? t.s0 + k : t.s0;
        su[k] = s == L5 - 1 ? 0 : s + 1;
        sd[k] = s == 0 ? L5 - 1 : s - 1;
        cu[k] = __fmul_rn(a.f.c5, s == L5 - 1 ? -m : 1.f);
        cl[k] = __fmul_rn(a.f.c5, s == 0 ? -m : 1.f);
      }
      const float2 b5 = f2(a.f.b5), cu2 = make_float2(cu[0], cu[1]), cl2 = make_float2(cl[0], cl[1]);
#pragma unroll
      for (int i = 0; i < 12; i++) {
        const float2 nu = make_float2(tile_at(tile, t.site_l, t.r_l, su[0], i), tile_at(tile, t.site_l, t.r_l, su[1], i));
        o[i] = fma2(cu2, nu, mul2(b5, v[i]));
      }
#pragma unroll
      for (int i = 12; i < 24; i++) {
        const float2 nd = make_float2(tile_at(tile, t.site_l, t.r_l, sd[0], i), tile_at(tile, t.site_l, t.r_l, sd[1], i));
        o[i] = fma2(cl2, nd, mul2(b5, v[i]));
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 24; i++) o[i] = mul2(kap, acc[i]);
  }

  float2 n2 = f2(0.f);
  if (t.act) {
    if ((EPI == E_A_SAME || EPI == E_AD_SAME_BD) && a.g_same != 0.f) apply_A_pair<S>(a, t, EPI == E_AD_SAME_BD, m, o);
    if ((EPI == E_SAME_AINV || EPI == E_SAME_BD) && a.g_same != 0.f) {
      float2 y[24];
      load_pair24<S>(a.same, a.same_nrm, t, a.N, y);
      const float2 g = f2(a.g_same);
#pragma unroll
      for (int i = 0; i < 24; i++) o[i] = fma2(g, y[i], o[i]);
    }
    if ((EPI == E_RAW || EPI == E_A_SAME || EPI == E_AD_SAME_BD || EPI == E_SAME_AINV || EPI == E_SAME_BD) &&
        a.add != nullptr) {
      float2 y[24];
      load_pair24<S>(a.add, a.add_nrm, t, a.N, y);
#pragma unroll
      for (int i = 0; i < 24; i++) o[i] = add2(o[i], y[i]);
    }
    store_pair24<S>(a.out, a.out_nrm, t, a.N, o);
    if (a.partials != nullptr) {
#pragma unroll
      for (int i = 0; i < 24; i++) n2 = fma2(o[i], o[i], n2);
    }
  }
  if (a.partials != nullptr) {
    // per-site, per-slot sums over the L5 slices (fixed order, FP64), stored as partials[r][h]
    __syncthreads();
    double* sred = reinterpret_cast<double*>(tile);
    const int rt = blockDim.x;
    sred[(t.site_l * L5 + t.s0) * rt + t.r_l] = (double)n2.x;
    if (t.two) sred[(t.site_l * L5 + t.s0 + 1) * rt + t.r_l] = (double)n2.y;
    __syncthreads();
    if (t.j == 0 && t.valid) {
      double sum = 0.0;
      for (int k = 0; k < L5; k++) sum += sred[(t.site_l * L5 + k) * rt + t.r_l];
      a.partials[(long)t.r * a.g.Vh + t.h] = sum;
    }
  }
}

// ---------------------------------------------------------------------------
// Prefetching form: asynchronous copies into per-thread stages.
// ---------------------------------------------------------------------------
constexpr int kStageBytes = 112;   // two fp16 units (2 x 48 B) + their two scales, padded to 16 B
constexpr int kLinkWords = 5;      // an FP32 link: five 16-byte words

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Term k of the hop: direction mu = k / 2, forward for even k.
template <int K>
__device__ __forceinline__ long pf_link_index(const FastArgs<__half, float>& a, const Site& x, long h) {
  constexpr int MU = K / 2;
  constexpr bool FWD = (K % 2) == 0;
  if (FWD) return ((long)a.out_par * a.g.Vh + h) * 4 + MU;
  return ((long)(1 - a.out_par) * a.g.Vh + nbr_half<MU, false>(a.g, x)) * 4 + MU;
}

// The block's links, [site_l][k][20 floats], loaded once by the whole block.
__device__ __forceinline__ void pf_load_links(const FastArgs<__half, float>& a, float4* slink) {
  const int nsb = blockDim.z;
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  for (int w = tid; w < nsb * 8 * kLinkWords; w += nthr) {
    const int site_l = w / (8 * kLinkWords);
    const int k = (w / kLinkWords) % 8;
    const int word = w % kLinkWords;
    const long h = (long)blockIdx.x * nsb + site_l;
    if (h >= a.g.Vh) continue;
    const Site x = make_site(a.g, a.out_par, h);
    long li;
    switch (k) {
      case 0: li = pf_link_index<0>(a, x, h); break;
      case 1: li = pf_link_index<1>(a, x, h); break;
      case 2: li = pf_link_index<2>(a, x, h); break;
      case 3: li = pf_link_index<3>(a, x, h); break;
      case 4: li = pf_link_index<4>(a, x, h); break;
      case 5: li = pf_link_index<5>(a, x, h); break;
      case 6: li = pf_link_index<6>(a, x, h); break;
      default: li = pf_link_index<7>(a, x, h); break;
    }
    slink[w] = __ldg(reinterpret_cast<const float4*>(a.U + kLinkStride32 * li) + word);
  }
}

// Issue the copies of term K's two neighbour units and their scales into a stage.
template <int K>
__device__ __forceinline__ void pf_issue(const FastArgs<__half, float>& a, const Site& x, const PThr& t,
                                         unsigned char* stage) {
  constexpr int MU = K / 2;
  constexpr bool FWD = (K % 2) == 0;
  const int hn = nbr_half<MU, FWD>(a.g, x);
  const long uA = ((long)hn * a.L5 + t.s0) * a.N + t.r;
  const long uB = t.two ? uA + a.N : uA;
  const uint4* pa = reinterpret_cast<const uint4*>(a.in + 24 * uA);
  const uint4* pb = reinterpret_cast<const uint4*>(a.in + 24 * uB);
  uint4* d = reinterpret_cast<uint4*>(stage);
  cp_async16(d, pa);
  cp_async16(d + 1, pa + 1);
  cp_async16(d + 2, pa + 2);
  cp_async16(d + 3, pb);
  cp_async16(d + 4, pb + 1);
  cp_async16(d + 5, pb + 2);
  float* sc = reinterpret_cast<float*>(d + 6);
  cp_async4(sc, a.in_nrm + uA);
  cp_async4(sc + 1, a.in_nrm + uB);
}

// Term K from a filled stage and the block's links (the operations of pair_term).
template <int K>
__device__ __forceinline__ void pf_compute(const FastArgs<__half, float>& a, const Site& x, const PThr& t,
                                           const unsigned char* stage, const float4* slink, float2* acc) {
  constexpr int MU = K / 2;
  constexpr bool FWD = (K % 2) == 0;
  const float sg = (a.dagger ? 1.f : -1.f) * (FWD ? 1.f : -1.f);
  const bool bflip = MU == 3 && a.antiperiodic && (FWD ? x.c[3] == a.g.L[3] - 1 : x.c[3] == 0);
  const uint4* q = reinterpret_cast<const uint4*>(stage);
  uint4 qa[3], qb[3];
  qa[0] = q[0]; qa[1] = q[1]; qa[2] = q[2];
  qb[0] = q[3]; qb[1] = q[4]; qb[2] = q[5];
  const float2 sc = *reinterpret_cast<const float2*>(q + 6);
  float ha[12], hb[12];
  project_half<MU>(qa, sg, ha);
  project_half<MU>(qb, sg, hb);
  float2 hh[12];
#pragma unroll
  for (int i = 0; i < 12; i++) hh[i] = make_float2(ha[i], hb[i]);
  float2 f = sc;
  if (bflip) f = neg2(f);
  const float2 fs = mul2(f, f2(sg));
  const float4* lw = slink + (t.site_l * 8 + K) * kLinkWords;
  const float4 t0 = lw[0], t1 = lw[1], t2 = lw[2], t3 = lw[3], t4 = lw[4];
  const float l[18] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, t2.x,
                       t2.y, t2.z, t2.w, t3.x, t3.y, t3.z, t3.w, t4.x, t4.y};
  if (FWD) mul_recon<MU, false>(l, hh, f, fs, acc);
  else mul_recon<MU, true>(l, hh, f, fs, acc);
}

// Step K of the two-stage pipeline: wait for term K, compute it, refill its stage with term K + 2.
template <int K>
__device__ __forceinline__ void pf_step(const FastArgs<__half, float>& a, const Site& x, const PThr& t,
                                        unsigned char* stages, const float4* slink, float2* acc) {
  unsigned char* stage = stages + (K & 1) * kStageBytes;
  if (K < 7) cp_async_wait<1>();
  else cp_async_wait<0>();
  pf_compute<K>(a, x, t, stage, slink, acc);
  if (K + 2 < 8) {
    pf_issue<(K + 2) & 7>(a, x, t, stage);
    cp_async_commit();
  }
}

// Bytes of the epilogue tile (or the reduction buffer) at the start of shared memory.
__host__ __device__ __forceinline__ size_t pair_tile_bytes(int threads, int nsb, int L5, int rt) {
  const size_t tile = (size_t)threads * kRS * sizeof(float);
  const size_t red = (size_t)nsb * L5 * rt * sizeof(double);
  const size_t b = tile > red ? tile : red;
  return (b + 15) & ~(size_t)15;
}
// Shared memory of the prefetching form beyond the tile: links and two stages per thread.
__host__ __device__ __forceinline__ size_t pair_pf_bytes(int threads, int nsb) {
  return (size_t)nsb * 8 * kLinkWords * 16 + (size_t)threads * 2 * kStageBytes;
}

#ifndef MDWF_PAIR_MAXREG
#define MDWF_PAIR_MAXREG 128
#endif
// R12: 12-real links (a.U12), the third row rebuilt; else the padded 18-real links (a.U).
// PF: the prefetching form (fp16 storage and 18-real links only).
template <typename S, int EPI, bool R12, bool PF>
__global__ void __maxnreg__(MDWF_PAIR_MAXREG) hop_pair_kernel(FastArgs<S, float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PThr t = pair_thread<S>(a);
  float2 acc[24];
#pragma unroll
  for (int i = 0; i < 24; i++) acc[i] = f2(0.f);
  if constexpr (PF) {
    static_assert(std::is_same<S, __half>::value && !R12, "the prefetching form is for fp16 and 18-real links");
    const int threads = blockDim.x * blockDim.y * blockDim.z;
    float4* slink = reinterpret_cast<float4*>(smem_raw + pair_tile_bytes(threads, blockDim.z, a.L5, blockDim.x));
    unsigned char* stages = reinterpret_cast<unsigned char*>(slink + blockDim.z * 8 * kLinkWords) +
                            (size_t)t.row * 2 * kStageBytes;
    if (a.in != nullptr) pf_load_links(a, slink);
    __syncthreads();
    if (t.act && a.in != nullptr) {
      const Site x = make_site(a.g, a.out_par, t.h);
      pf_issue<0>(a, x, t, stages);
      cp_async_commit();
      pf_issue<1>(a, x, t, stages + kStageBytes);
      cp_async_commit();
      pf_step<0>(a, x, t, stages, slink, acc);
      pf_step<1>(a, x, t, stages, slink, acc);
      pf_step<2>(a, x, t, stages, slink, acc);
      pf_step<3>(a, x, t, stages, slink, acc);
      pf_step<4>(a, x, t, stages, slink, acc);
      pf_step<5>(a, x, t, stages, slink, acc);
      pf_step<6>(a, x, t, stages, slink, acc);
      pf_step<7>(a, x, t, stages, slink, acc);
    }
  } else if (t.act && a.in != nullptr) {      // no input: a local fifth-dimension pass
    const Site x = make_site(a.g, a.out_par, t.h);
    pair_term<0, true, S, R12>(a, x, t, acc);
    pair_term<0, false, S, R12>(a, x, t, acc);
    pair_term<1, true, S, R12>(a, x, t, acc);
    pair_term<1, false, S, R12>(a, x, t, acc);
    pair_term<2, true, S, R12>(a, x, t, acc);
    pair_term<2, false, S, R12>(a, x, t, acc);
    pair_term<3, true, S, R12>(a, x, t, acc);
    pair_term<3, false, S, R12>(a, x, t, acc);
  }
  pair_epilogue<S, EPI>(a, t, acc, reinterpret_cast<float*>(smem_raw));
}

constexpr int kPairMaxThreads = 512;

}  // namespace

PairShape pair_shape(int L5, int N, int nsb) {
  PairShape p;
  p.J = (L5 + 1) / 2;
  if (nsb < 1) nsb = 1;
  while (nsb > 1 && nsb * p.J > kPairMaxThreads) nsb--;
  p.nsb = nsb;
  int rt = kPairMaxThreads / (nsb * p.J);
  if (rt < 1) rt = 1;
  p.rt = N < rt ? N : rt;
  p.threads = p.rt * p.J * p.nsb;
  p.smem = pair_tile_bytes(p.threads, p.nsb, L5, p.rt);
  p.smem_pf = p.smem + pair_pf_bytes(p.threads, p.nsb);
  return p;
}

constexpr size_t kPairMaxSmem = 200 * 1024;

template <typename S, int EPI>
static cudaError_t launch_pair_one(const FastArgs<S, float>& a, const PairShape& p, bool pf, cudaStream_t st) {
  const dim3 grid((unsigned)((a.g.Vh + p.nsb - 1) / p.nsb), (unsigned)((a.N + p.rt - 1) / p.rt));
  const dim3 block((unsigned)p.rt, (unsigned)p.J, (unsigned)p.nsb);
  auto* kern = a.U12 != nullptr ? hop_pair_kernel<S, EPI, true, false> : hop_pair_kernel<S, EPI, false, false>;
  size_t smem = p.smem;
  if constexpr (std::is_same<S, __half>::value) {
    if (pf && a.U12 == nullptr && p.smem_pf <= kPairMaxSmem) {
      kern = hop_pair_kernel<S, EPI, false, true>;
      smem = p.smem_pf;
    }
  }
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_pair(const FastArgs<S, float>& a, int nsb, int epi, cudaStream_t st, bool prefetch) {
  if (a.N < 1 || a.L5 < 1 || a.g.Vh < 1) return cudaErrorInvalidValue;
  const PairShape p = pair_shape(a.L5, a.N, nsb);
  if (p.smem > kPairMaxSmem) return cudaErrorInvalidValue;
  switch (epi) {
    case E_RAW: return launch_pair_one<S, E_RAW>(a, p, prefetch, st);
    case E_BAINV: return launch_pair_one<S, E_BAINV>(a, p, prefetch, st);
    case E_AINVD_BD: return launch_pair_one<S, E_AINVD_BD>(a, p, prefetch, st);
    case E_A_SAME: return launch_pair_one<S, E_A_SAME>(a, p, prefetch, st);
    case E_AD_SAME_BD: return launch_pair_one<S, E_AD_SAME_BD>(a, p, prefetch, st);
    case E_AINV_SAME: return launch_pair_one<S, E_AINV_SAME>(a, p, prefetch, st);
    case E_SAME_AINV: return launch_pair_one<S, E_SAME_AINV>(a, p, prefetch, st);
    case E_SAME_BD: return launch_pair_one<S, E_SAME_BD>(a, p, prefetch, st);
    case E_AINVD_SAME: return launch_pair_one<S, E_AINVD_SAME>(a, p, prefetch, st);
    default: return cudaErrorInvalidValue;
  }
}

__global__ void k_link12(const float* __restrict__ U32, float* __restrict__ U12, long nlinks) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlinks * 3) return;
  const long link = i / 3;
  const int w = (int)(i - link * 3);
  reinterpret_cast<float4*>(U12)[link * 3 + w] = __ldg(reinterpret_cast<const float4*>(U32 + kLinkStride32 * link) + w);
}

cudaError_t build_link12(const float* U32, float* U12, long nlinks, cudaStream_t st) {
  const long n = nlinks * 3;
  k_link12<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U32, U12, nlinks);
  return cudaGetLastError();
}

template cudaError_t launch_pair<float>(const FastArgs<float, float>&, int, int, cudaStream_t, bool);
template cudaError_t launch_pair<__half>(const FastArgs<__half, float>&, int, int, cudaStream_t, bool);
template cudaError_t launch_pair<__nv_bfloat16>(const FastArgs<__nv_bfloat16, float>&, int, int, cudaStream_t, bool);

}  // namespace mdwf
