// Internal definitions shared by the libmdwf CUDA sources.
//
// Device layouts
//   spinor field, one parity:   [h][s][r][24]   h = half-lattice site, s = fifth
//                                                 dimension slice, r = RHS slot,
//                                                 24 = [spin 4][colour 3][re, im]
//   16-bit storage adds a scale per (h, s, r):   nrm[h][s][r] (float); the stored
//                                                 values are v / nrm, nrm = max |v|.
//   gauge field:                [parity][h][mu][18]   (3x3 complex, row major),
//                                mu = 0..3 for x, y, z, t; U_mu(x) of the site x.
//   fifth-dimension matrices:   [r][chirality][L5][L5] real; chirality 0 acts on
//                                spins 0,1 (P_+), chirality 1 on spins 2,3 (P_-).
// Half-lattice index: lex = x + Lx (y + Ly (z + Lz t)), h = lex >> 1 (Lx even).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace mdwf {

struct Geom {
  int L[4];    // Lx, Ly, Lz, Lt
  int Lxh;     // Lx / 2
  long V, Vh;  // sites, half-lattice sites
};

inline Geom make_geom(const int d[4]) {
  Geom g;
  for (int i = 0; i < 4; i++) g.L[i] = d[i];
  g.Lxh = d[0] / 2;
  g.V = (long)d[0] * d[1] * d[2] * d[3];
  g.Vh = g.V / 2;
  return g;
}

__host__ __device__ __forceinline__ void site_coords(const Geom& g, int par, long h, int c[4]) {
  long r = h / g.Lxh;
  int xh = (int)(h - r * g.Lxh);
  c[1] = (int)(r % g.L[1]);
  r /= g.L[1];
  c[2] = (int)(r % g.L[2]);
  c[3] = (int)(r / g.L[2]);
  c[0] = 2 * xh + ((c[1] + c[2] + c[3] + par) & 1);
}

__host__ __device__ __forceinline__ long lex_index(const Geom& g, const int c[4]) {
  return c[0] + (long)g.L[0] * (c[1] + (long)g.L[1] * (c[2] + (long)g.L[2] * c[3]));
}

// ---------------------------------------------------------------------------
// storage types
// ---------------------------------------------------------------------------
enum Prec { PREC_DOUBLE = 0, PREC_SINGLE = 1, PREC_HALF = 2, PREC_BF16 = 3 };

template <typename S> struct StoreTraits;
template <> struct StoreTraits<double> { using T = double; static constexpr bool kNorm = false; };
template <> struct StoreTraits<float> { using T = float; static constexpr bool kNorm = false; };
template <> struct StoreTraits<__half> { using T = float; static constexpr bool kNorm = true; };
template <> struct StoreTraits<__nv_bfloat16> { using T = float; static constexpr bool kNorm = false; };

// Load the 24 reals of unit u (unit = (h * L5 + s) * N + r).
template <typename S, typename T>
__device__ __forceinline__ void load24(const S* __restrict__ v, const float* __restrict__ nrm, long u, T a[24]);

template <>
__device__ __forceinline__ void load24<double, double>(const double* __restrict__ v, const float*, long u, double a[24]) {
  const double2* p = reinterpret_cast<const double2*>(v + 24 * u);
#pragma unroll
  for (int i = 0; i < 12; i++) { double2 t = __ldg(p + i); a[2 * i] = t.x; a[2 * i + 1] = t.y; }
}
template <>
__device__ __forceinline__ void load24<float, float>(const float* __restrict__ v, const float*, long u, float a[24]) {
  const float4* p = reinterpret_cast<const float4*>(v + 24 * u);
#pragma unroll
  for (int i = 0; i < 6; i++) { float4 t = __ldg(p + i); a[4*i] = t.x; a[4*i+1] = t.y; a[4*i+2] = t.z; a[4*i+3] = t.w; }
}
template <>
__device__ __forceinline__ void load24<__half, float>(const __half* __restrict__ v, const float* __restrict__ nrm, long u, float a[24]) {
  const uint4* p = reinterpret_cast<const uint4*>(v + 24 * u);
  float s = __ldg(nrm + u);
#pragma unroll
  for (int i = 0; i < 3; i++) {
    uint4 t = __ldg(p + i);
    const __half2* hh = reinterpret_cast<const __half2*>(&t);
#pragma unroll
    for (int j = 0; j < 4; j++) { float2 f = __half22float2(hh[j]); a[8*i+2*j] = f.x * s; a[8*i+2*j+1] = f.y * s; }
  }
}
template <>
__device__ __forceinline__ void load24<__nv_bfloat16, float>(const __nv_bfloat16* __restrict__ v, const float*, long u, float a[24]) {
  const uint4* p = reinterpret_cast<const uint4*>(v + 24 * u);
#pragma unroll
  for (int i = 0; i < 3; i++) {
    uint4 t = __ldg(p + i);
    const __nv_bfloat162* hh = reinterpret_cast<const __nv_bfloat162*>(&t);
#pragma unroll
    for (int j = 0; j < 4; j++) { float2 f = __bfloat1622float2(hh[j]); a[8*i+2*j] = f.x; a[8*i+2*j+1] = f.y; }
  }
}

// Store the 24 reals of unit u.
template <typename S, typename T>
__device__ __forceinline__ void store24(S* __restrict__ v, float* __restrict__ nrm, long u, const T a[24]);

template <>
__device__ __forceinline__ void store24<double, double>(double* __restrict__ v, float*, long u, const double a[24]) {
  double2* p = reinterpret_cast<double2*>(v + 24 * u);
#pragma unroll
  for (int i = 0; i < 12; i++) p[i] = make_double2(a[2 * i], a[2 * i + 1]);
}
template <>
__device__ __forceinline__ void store24<float, float>(float* __restrict__ v, float*, long u, const float a[24]) {
  float4* p = reinterpret_cast<float4*>(v + 24 * u);
#pragma unroll
  for (int i = 0; i < 6; i++) p[i] = make_float4(a[4*i], a[4*i+1], a[4*i+2], a[4*i+3]);
}
template <>
__device__ __forceinline__ void store24<__half, float>(__half* __restrict__ v, float* __restrict__ nrm, long u, const float a[24]) {
  float m = 0.f;
#pragma unroll
  for (int i = 0; i < 24; i++) m = fmaxf(m, fabsf(a[i]));
  float inv = m > 0.f ? 1.0f / m : 0.f;
  nrm[u] = m;
  uint4* p = reinterpret_cast<uint4*>(v + 24 * u);
#pragma unroll
  for (int i = 0; i < 3; i++) {
    uint4 t;
    __half2* hh = reinterpret_cast<__half2*>(&t);
#pragma unroll
    for (int j = 0; j < 4; j++) hh[j] = __floats2half2_rn(a[8*i+2*j] * inv, a[8*i+2*j+1] * inv);
    p[i] = t;
  }
}
template <>
__device__ __forceinline__ void store24<__nv_bfloat16, float>(__nv_bfloat16* __restrict__ v, float*, long u, const float a[24]) {
  uint4* p = reinterpret_cast<uint4*>(v + 24 * u);
#pragma unroll
  for (int i = 0; i < 3; i++) {
    uint4 t;
    __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(&t);
#pragma unroll
    for (int j = 0; j < 4; j++) hh[j] = __floats2bfloat162_rn(a[8*i+2*j], a[8*i+2*j+1]);
    p[i] = t;
  }
}

// Link loads (T precision, 18 reals).
template <typename T>
__device__ __forceinline__ void load_link(const T* __restrict__ U, long idx, T l[18]);
template <>
__device__ __forceinline__ void load_link<double>(const double* __restrict__ U, long idx, double l[18]) {
  const double2* p = reinterpret_cast<const double2*>(U + 18 * idx);
#pragma unroll
  for (int i = 0; i < 9; i++) { double2 t = __ldg(p + i); l[2 * i] = t.x; l[2 * i + 1] = t.y; }
}
template <>
__device__ __forceinline__ void load_link<float>(const float* __restrict__ U, long idx, float l[18]) {
  const float2* p = reinterpret_cast<const float2*>(U + 18 * idx);
#pragma unroll
  for (int i = 0; i < 9; i++) { float2 t = __ldg(p + i); l[2 * i] = t.x; l[2 * i + 1] = t.y; }
}

// ---------------------------------------------------------------------------
// launch descriptors
// ---------------------------------------------------------------------------
// Work is organised in tiles of `nsb` half-lattice sites x all L5 slices x `rt`
// RHS slots (one thread per unit).  The per-slot partial sums of a reduction are
// formed per tile of sites, in a fixed order, so they do not depend on N or rt.
struct Tiling {
  int nsb;     // sites per tile
  int rt;      // slots per block
  long ntiles; // ceil(Vh / nsb)
  int ngroups; // ceil(N / rt)
  int threads; // nsb * L5 * rt
};

inline Tiling make_tiling(long Vh, int L5, int N, int nsb, int max_threads = 1024) {
  Tiling t;
  t.nsb = nsb;
  int maxrt = max_threads / (nsb * L5);
  if (maxrt < 1) maxrt = 1;
  t.rt = N < maxrt ? N : maxrt;
  t.ngroups = (N + t.rt - 1) / t.rt;
  t.ntiles = (Vh + nsb - 1) / nsb;
  t.threads = nsb * L5 * t.rt;
  return t;
}

// Operands of one Wilson-hop + fifth-dimension launch (see hop.cu):
//   out = add + G . same + kappa * C . H(in)      (HOP = true)
//   out = add + G . in                            (HOP = false)
// G, C: per-slot [2][L5][L5] matrices (null C = identity, null G = no term).
template <typename S, typename T>
struct HopArgs {
  Geom g;
  int L5, N;
  int out_par;          // parity of the output sites
  int dagger;           // 1: H^+ (projectors exchanged)
  int antiperiodic;     // time boundary phase -1
  const S* in; const float* in_nrm;        // opposite parity (HOP) or same parity (local)
  const S* same; const float* same_nrm;    // output parity, optional
  const S* add; const float* add_nrm;      // output parity, optional
  S* out; float* out_nrm;
  const T* U;           // gauge [2][Vh][4][18]
  const T* Gm;          // [N][2][L5][L5] or null
  const T* Cm;          // [N][2][L5][L5] or null (identity)
  T kappa;
  const int* active;    // [N] or null (all active)
  double* partials;     // [ntiles][N] |out|^2 per tile, or null
};

// Kernel launchers (hop.cu).
template <typename S, typename T>
cudaError_t launch_hop(const HopArgs<S, T>& a, const Tiling& t, bool hop, cudaStream_t st);
template <typename S, typename T>
int hop_max_threads();
template <typename S, typename T>
size_t hop_smem_bytes(const Tiling& t, bool two);

}  // namespace mdwf
