// Wilson hopping term on all L5 slices and all RHS slots, with the Moebius
// fifth-dimension operators fused into the epilogue.
//
// The 4D Wilson operator inside the Moebius kernel (Sec. II of
// arXiv:1701.07559) is D_W = (4 - M5) - H/2 with
//   (H psi)(x) = sum_mu (1 - g_mu) U_mu(x) psi(x + mu) + (1 + g_mu) U_mu(x - mu)^+ psi(x - mu),
// antiperiodic in time.  The 5D operator D = A - H B / 2 with A, B polynomials
// in the fifth-dimension hop P (Brower-Neff-Orginos form of the Moebius
// action) only mixes the s index of one 4D site, so one block holds every
// slice of its sites and applies the L5 x L5 matrices from shared memory:
//
//   out(x, s, r) = add + sum_s' G_r[chi](s, s') same(x, s', r)
//                      + kappa sum_s' C_r[chi](s, s') (H in)(x, s', r)
//
// chi is the chirality of the spin component (DeGrand-Rossi basis: spins 0,1
// are P_+, spins 2,3 are P_-).  Every link of a site is loaded by the threads
// of that site's tile only, which cover all L5 x rt (slice, RHS) pairs.
#include "mdwf_internal.h"

namespace mdwf {

// o = U v (DAG = false) or U^+ v (DAG = true); colour vectors of 3 complex.
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

// Spinor index helpers: component (spin k, colour c, part p) at 6k + 2c + p.
// (1 + sg g_mu) psi = [h ; sg e_mu^+ h] with h = psi_up + sg e_mu psi_lo, where
// g_mu = [[0, e_mu], [e_mu^+, 0]], e_x = i sigma_x, e_y = -i sigma_y,
// e_z = i sigma_z, e_t = 1.  After the colour multiply chi = U h the upper
// spins receive chi and the lower spins sg e_mu^+ chi.
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
    if (MU == 0) {        // e psi_lo = (i p3, i p2)
      h0[0] = p0[0] - sg * p3[1]; h0[1] = p0[1] + sg * p3[0];
      h1[0] = p1[0] - sg * p2[1]; h1[1] = p1[1] + sg * p2[0];
    } else if (MU == 1) { // (-p3, p2)
      h0[0] = p0[0] - sg * p3[0]; h0[1] = p0[1] - sg * p3[1];
      h1[0] = p1[0] + sg * p2[0]; h1[1] = p1[1] + sg * p2[1];
    } else if (MU == 2) { // (i p2, -i p3)
      h0[0] = p0[0] - sg * p2[1]; h0[1] = p0[1] + sg * p2[0];
      h1[0] = p1[0] + sg * p3[1]; h1[1] = p1[1] - sg * p3[0];
    } else {              // (p2, p3)
      h0[0] = p0[0] + sg * p2[0]; h0[1] = p0[1] + sg * p2[1];
      h1[0] = p1[0] + sg * p3[0]; h1[1] = p1[1] + sg * p3[1];
    }
  }
}

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
    if (MU == 0) {        // e^+ chi = (-i x1, -i x0)
      a2[0] += sg * x1[1]; a2[1] -= sg * x1[0];
      a3[0] += sg * x0[1]; a3[1] -= sg * x0[0];
    } else if (MU == 1) { // (x1, -x0)
      a2[0] += sg * x1[0]; a2[1] += sg * x1[1];
      a3[0] -= sg * x0[0]; a3[1] -= sg * x0[1];
    } else if (MU == 2) { // (-i x0, i x1)
      a2[0] += sg * x0[1]; a2[1] -= sg * x0[0];
      a3[0] -= sg * x1[1]; a3[1] += sg * x1[0];
    } else {              // (x0, x1)
      a2[0] += sg * x0[0]; a2[1] += sg * x0[1];
      a3[0] += sg * x1[0]; a3[1] += sg * x1[1];
    }
  }
}

template <int MU, typename S, typename T>
__device__ __forceinline__ void hop_dir(const HopArgs<S, T>& a, const int c[4], long h, int s, int r, T* acc) {
  const int par = a.out_par;
  // forward neighbour: (1 - g_mu) U_mu(x) psi(x + mu)   [dagger: (1 + g_mu)]
  {
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[MU] = (c[MU] + 1 == a.g.L[MU]) ? 0 : c[MU] + 1;
    T phase = (MU == 3 && a.antiperiodic && c[3] == a.g.L[3] - 1) ? T(-1) : T(1);
    long hn = lex_index(a.g, n) >> 1;
    T psi[24], hh[12], chi[12], l[18];
    load24<S, T>(a.in, a.in_nrm, (hn * a.L5 + s) * a.N + r, psi);
    load_link<T>(a.U, ((long)par * a.g.Vh + h) * 4 + MU, l);
    const T sg = a.dagger ? T(1) : T(-1);
    project<MU, T>(psi, sg, hh);
    su3_mul<T, false>(l, hh, chi);
    su3_mul<T, false>(l, hh + 6, chi + 6);
#pragma unroll
    for (int i = 0; i < 12; i++) chi[i] *= phase;
    reconstruct<MU, T>(chi, sg, acc);
  }
  // backward neighbour: (1 + g_mu) U_mu(x - mu)^+ psi(x - mu)   [dagger: (1 - g_mu)]
  {
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[MU] = (c[MU] == 0) ? a.g.L[MU] - 1 : c[MU] - 1;
    T phase = (MU == 3 && a.antiperiodic && c[3] == 0) ? T(-1) : T(1);
    long hn = lex_index(a.g, n) >> 1;
    T psi[24], hh[12], chi[12], l[18];
    load24<S, T>(a.in, a.in_nrm, (hn * a.L5 + s) * a.N + r, psi);
    load_link<T>(a.U, ((long)(1 - par) * a.g.Vh + hn) * 4 + MU, l);
    const T sg = a.dagger ? T(-1) : T(1);
    project<MU, T>(psi, sg, hh);
    su3_mul<T, true>(l, hh, chi);
    su3_mul<T, true>(l, hh + 6, chi + 6);
#pragma unroll
    for (int i = 0; i < 12; i++) chi[i] *= phase;
    reconstruct<MU, T>(chi, sg, acc);
  }
}

constexpr int kPad = 25;  // shared-memory row of one unit (24 reals + 1 pad)

template <typename S, typename T, bool HOP>
__global__ void hop_kernel(HopArgs<S, T> a, Tiling tl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);                 // H(in) (HOP) or in (local)
  T* sG = sA + (size_t)tl.threads * kPad;                  // same (HOP with G)
  const int L5 = a.L5;
  const int tid = threadIdx.x;
  const int r_l = tid % tl.rt;
  const int s = (tid / tl.rt) % L5;
  const int site_l = tid / (tl.rt * L5);
  const long h = (long)blockIdx.x * tl.nsb + site_l;
  const int r = blockIdx.y * tl.rt + r_l;
  const bool valid = (h < a.g.Vh) && (r < a.N);
  const bool act = valid && (a.active == nullptr || a.active[r] != 0);
  const long u = (h * L5 + s) * a.N + r;

  T acc[24];
#pragma unroll
  for (int i = 0; i < 24; i++) acc[i] = 0;
  if (act) {
    if (HOP) {
      int c[4];
      site_coords(a.g, a.out_par, h, c);
      hop_dir<0, S, T>(a, c, h, s, r, acc);
      hop_dir<1, S, T>(a, c, h, s, r, acc);
      hop_dir<2, S, T>(a, c, h, s, r, acc);
      hop_dir<3, S, T>(a, c, h, s, r, acc);
    } else {
      load24<S, T>(a.in, a.in_nrm, u, acc);
    }
  }
#pragma unroll
  for (int i = 0; i < 24; i++) sA[tid * kPad + i] = acc[i];
  const bool g_from_same = HOP && a.Gm != nullptr;
  if (g_from_same) {
    T tmp[24];
#pragma unroll
    for (int i = 0; i < 24; i++) tmp[i] = 0;
    if (act) load24<S, T>(a.same, a.same_nrm, u, tmp);
#pragma unroll
    for (int i = 0; i < 24; i++) sG[tid * kPad + i] = tmp[i];
  }
  __syncthreads();

  double n2 = 0.0;
  if (act) {
    T o[24];
    if (a.add != nullptr) {
      load24<S, T>(a.add, a.add_nrm, u, o);
    } else {
#pragma unroll
      for (int i = 0; i < 24; i++) o[i] = 0;
    }
    const int base = site_l * L5 * tl.rt + r_l;   // thread of (site_l, s' = 0, r_l)
    if (HOP) {
      if (a.Cm != nullptr) {
        const T* Cu = a.Cm + ((size_t)r * 2 + 0) * L5 * L5 + (size_t)s * L5;
        const T* Cl = a.Cm + ((size_t)r * 2 + 1) * L5 * L5 + (size_t)s * L5;
        for (int sp = 0; sp < L5; sp++) {
          const T cu = a.kappa * __ldg(Cu + sp), cl = a.kappa * __ldg(Cl + sp);
          const T* src = sA + (size_t)(base + sp * tl.rt) * kPad;
#pragma unroll
          for (int i = 0; i < 12; i++) o[i] += cu * src[i];
#pragma unroll
          for (int i = 12; i < 24; i++) o[i] += cl * src[i];
        }
      } else {
#pragma unroll
        for (int i = 0; i < 24; i++) o[i] += a.kappa * acc[i];
      }
    }
    if (a.Gm != nullptr) {
      const T* Gu = a.Gm + ((size_t)r * 2 + 0) * L5 * L5 + (size_t)s * L5;
      const T* Gl = a.Gm + ((size_t)r * 2 + 1) * L5 * L5 + (size_t)s * L5;
      const T* sx = HOP ? sG : sA;
      for (int sp = 0; sp < L5; sp++) {
        const T gu = __ldg(Gu + sp), gl = __ldg(Gl + sp);
        const T* src = sx + (size_t)(base + sp * tl.rt) * kPad;
#pragma unroll
        for (int i = 0; i < 12; i++) o[i] += gu * src[i];
#pragma unroll
        for (int i = 12; i < 24; i++) o[i] += gl * src[i];
      }
    }
    store24<S, T>(a.out, a.out_nrm, u, o);
    if (a.partials != nullptr) {
#pragma unroll
      for (int i = 0; i < 24; i++) n2 += (double)o[i] * (double)o[i];
    }
  }
  if (a.partials != nullptr) {
    __syncthreads();
    double* sred = reinterpret_cast<double*>(smem_raw);
    sred[tid] = n2;
    __syncthreads();
    if (s == 0 && valid) {
      double sum = 0.0;
      for (int k = 0; k < L5; k++) sum += sred[(site_l * L5 + k) * tl.rt + r_l];
      a.partials[(long)r * a.g.Vh + h] = sum;
    }
  }
}

template <typename S, typename T>
size_t hop_smem_bytes(const Tiling& t, bool two) {
  size_t b = (size_t)t.threads * kPad * sizeof(T) * (two ? 2 : 1);
  size_t r = (size_t)t.threads * sizeof(double);
  return b > r ? b : r;
}

template <typename S, typename T>
cudaError_t launch_hop(const HopArgs<S, T>& a, const Tiling& t, bool hop, cudaStream_t st) {
  dim3 grid((unsigned)t.ntiles, (unsigned)t.ngroups);
  const bool two = hop && a.Gm != nullptr;
  size_t smem = hop_smem_bytes<S, T>(t, two);
  if (hop) {
    cudaError_t e = cudaFuncSetAttribute(hop_kernel<S, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    hop_kernel<S, T, true><<<grid, t.threads, smem, st>>>(a, t);
  } else {
    cudaError_t e = cudaFuncSetAttribute(hop_kernel<S, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    hop_kernel<S, T, false><<<grid, t.threads, smem, st>>>(a, t);
  }
  return cudaGetLastError();
}

// Largest block the kernel can take (registers) for the given storage type.
template <typename S, typename T>
int hop_max_threads() {
  cudaFuncAttributes fa1, fa2;
  if (cudaFuncGetAttributes(&fa1, hop_kernel<S, T, true>) != cudaSuccess) return 128;
  if (cudaFuncGetAttributes(&fa2, hop_kernel<S, T, false>) != cudaSuccess) return 128;
  return fa1.maxThreadsPerBlock < fa2.maxThreadsPerBlock ? fa1.maxThreadsPerBlock : fa2.maxThreadsPerBlock;
}

#define MDWF_INSTANTIATE_HOP(S, T)                                                                 \
  template cudaError_t launch_hop<S, T>(const HopArgs<S, T>&, const Tiling&, bool, cudaStream_t); \
  template int hop_max_threads<S, T>();                                                            \
  template size_t hop_smem_bytes<S, T>(const Tiling&, bool);

MDWF_INSTANTIATE_HOP(double, double)
MDWF_INSTANTIATE_HOP(float, float)
MDWF_INSTANTIATE_HOP(__half, float)
MDWF_INSTANTIATE_HOP(__nv_bfloat16, float)

}  // namespace mdwf
