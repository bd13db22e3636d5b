// Internal definitions shared by the libmdwf CUDA sources.
//
// Device layouts
//   spinor field, one parity:   [h][s][r][24]   h = half-lattice site, s = fifth
//                                                 dimension slice, r = RHS slot,
//                                                 24 = [spin 4][colour 3][re, im]
//   16-bit storage adds a scale per (h, s, r):   nrm[h][s][r] (float); the stored
//                                                 values are v / nrm, nrm = the smallest power
//                                                 of two >= max |v| of the unit.
//   fp16 storage orders the 24 reals of a unit colour-major, [colour][spin][re,im],
//   so that the four spins of one colour are one 16-byte word (the tensor-core hop
//   loads them per lane); every other type, and every register copy, uses
//   [spin][colour][re,im].
//   gauge field:                [parity][h][mu][18]   (3x3 complex, row major),
//                                mu = 0..3 for x, y, z, t; U_mu(x) of the site x;
//                                the FP32 copy pads each link to 20 floats.
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

// 32-bit index arithmetic: lattices up to 2^31 sites.
__host__ __device__ __forceinline__ void site_coords(const Geom& g, int par, long h, int c[4]) {
  const int hi = (int)h;
  int r = hi / g.Lxh;
  const int xh = hi - r * g.Lxh;
  int q = r / g.L[1];
  c[1] = r - q * g.L[1];
  c[3] = q / g.L[2];
  c[2] = q - c[3] * g.L[2];
  c[0] = 2 * xh + ((c[1] + c[2] + c[3] + par) & 1);
}

__host__ __device__ __forceinline__ long lex_index(const Geom& g, const int c[4]) {
  return (long)(c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3])));
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
  const float s = __ldg(nrm + u);
#pragma unroll
  for (int c = 0; c < 3; c++) {           // word c: spins 0..3 of colour c
    uint4 t = __ldg(p + c);
    const __half2* hh = reinterpret_cast<const __half2*>(&t);
#pragma unroll
    for (int k = 0; k < 4; k++) { float2 f = __half22float2(hh[k]); a[6*k+2*c] = f.x * s; a[6*k+2*c+1] = f.y * s; }
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

// Scale of an fp16-stored unit whose largest |component| is m: the smallest
// power of two >= m.  Its reciprocal is exact, so each stored value is rounded
// once (to fp16), and the largest lies in [1/2, 1].  A unit whose largest entry
// is below the smallest normal float is stored as zero; above 2^126 the scale is
// m itself.
__device__ __forceinline__ void half_scale(float m, float* sc, float* inv) {
  *sc = 0.f;
  *inv = 0.f;
  if (m >= 1.17549435e-38f) {
    const unsigned mb = __float_as_uint(m);
    unsigned e = mb & 0x7f800000u;
    if (mb & 0x007fffffu) e += 0x00800000u;
    if (e <= (253u << 23)) {
      *sc = __uint_as_float(e);
      *inv = __uint_as_float(0x7f000000u - e);
    } else {
      *sc = m;
      *inv = 1.0f / m;
    }
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
  float sc, inv;
  half_scale(m, &sc, &inv);
  nrm[u] = sc;
  uint4* p = reinterpret_cast<uint4*>(v + 24 * u);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    uint4 t;
    __half2* hh = reinterpret_cast<__half2*>(&t);
#pragma unroll
    for (int k = 0; k < 4; k++) hh[k] = __floats2half2_rn(a[6*k+2*c] * inv, a[6*k+2*c+1] * inv);
    p[c] = t;
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

// Half of a stored spinor: part 0 = spins 0,1 (components 0..11), part 1 = spins 2,3.
template <typename S, typename T>
__device__ __forceinline__ void load_part(const S* __restrict__ v, const float* __restrict__ nrm, long u, int part,
                                          T* o);
template <>
__device__ __forceinline__ void load_part<double, double>(const double* __restrict__ v, const float*, long u, int part,
                                                          double* o) {
  const double2* p = reinterpret_cast<const double2*>(v + 24 * u + 12 * part);
#pragma unroll
  for (int i = 0; i < 6; i++) { double2 t = __ldg(p + i); o[2 * i] = t.x; o[2 * i + 1] = t.y; }
}
template <>
__device__ __forceinline__ void load_part<float, float>(const float* __restrict__ v, const float*, long u, int part,
                                                        float* o) {
  const float4* p = reinterpret_cast<const float4*>(v + 24 * u + 12 * part);
#pragma unroll
  for (int i = 0; i < 3; i++) { float4 t = __ldg(p + i); o[4*i] = t.x; o[4*i+1] = t.y; o[4*i+2] = t.z; o[4*i+3] = t.w; }
}
template <>
__device__ __forceinline__ void load_part<__half, float>(const __half* __restrict__ v, const float* __restrict__ nrm,
                                                         long u, int part, float* o) {
  // colour-major storage: spins 2 part, 2 part + 1 of colour c are the 8 bytes at 16 c + 8 part
  const float s = __ldg(nrm + u);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    uint2 t = __ldg(reinterpret_cast<const uint2*>(v + 24 * u + 8 * c + 4 * part));
    const __half2* hh = reinterpret_cast<const __half2*>(&t);
    float2 a = __half22float2(hh[0]), b = __half22float2(hh[1]);
    o[2*c] = a.x * s; o[2*c+1] = a.y * s; o[6+2*c] = b.x * s; o[6+2*c+1] = b.y * s;
  }
}
template <>
__device__ __forceinline__ void load_part<__nv_bfloat16, float>(const __nv_bfloat16* __restrict__ v, const float*,
                                                                long u, int part, float* o) {
  const uint2* p = reinterpret_cast<const uint2*>(v + 24 * u + 12 * part);
#pragma unroll
  for (int i = 0; i < 3; i++) {
    uint2 t = __ldg(p + i);
    const __nv_bfloat162* hh = reinterpret_cast<const __nv_bfloat162*>(&t);
    float2 a = __bfloat1622float2(hh[0]), b = __bfloat1622float2(hh[1]);
    o[4*i] = a.x; o[4*i+1] = a.y; o[4*i+2] = b.x; o[4*i+3] = b.y;
  }
}

// Plain (shared-memory) loads of a stored spinor, without the fp16 scale.
template <typename S, typename T>
__device__ __forceinline__ void load24_smem(const S* p, T a[24]);
template <>
__device__ __forceinline__ void load24_smem<double, double>(const double* p, double a[24]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int i = 0; i < 12; i++) { double2 t = q[i]; a[2 * i] = t.x; a[2 * i + 1] = t.y; }
}
template <>
__device__ __forceinline__ void load24_smem<float, float>(const float* p, float a[24]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < 6; i++) { float4 t = q[i]; a[4*i] = t.x; a[4*i+1] = t.y; a[4*i+2] = t.z; a[4*i+3] = t.w; }
}
template <>
__device__ __forceinline__ void load24_smem<__half, float>(const __half* p, float a[24]) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    uint4 t = q[c];
    const __half2* hh = reinterpret_cast<const __half2*>(&t);
#pragma unroll
    for (int k = 0; k < 4; k++) { float2 f = __half22float2(hh[k]); a[6*k+2*c] = f.x; a[6*k+2*c+1] = f.y; }
  }
}
template <>
__device__ __forceinline__ void load24_smem<__nv_bfloat16, float>(const __nv_bfloat16* p, float a[24]) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int i = 0; i < 3; i++) {
    uint4 t = q[i];
    const __nv_bfloat162* hh = reinterpret_cast<const __nv_bfloat162*>(&t);
#pragma unroll
    for (int j = 0; j < 4; j++) { float2 f = __bfloat1622float2(hh[j]); a[8*i+2*j] = f.x; a[8*i+2*j+1] = f.y; }
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
// FP32 links are padded to 20 floats (80 bytes) so that each is five aligned 16-byte loads.
constexpr int kLinkStride32 = 20;
template <>
__device__ __forceinline__ void load_link<float>(const float* __restrict__ U, long idx, float l[18]) {
  const float4* p = reinterpret_cast<const float4*>(U + kLinkStride32 * idx);
  float4 t0 = __ldg(p), t1 = __ldg(p + 1), t2 = __ldg(p + 2), t3 = __ldg(p + 3), t4 = __ldg(p + 4);
  l[0] = t0.x; l[1] = t0.y; l[2] = t0.z; l[3] = t0.w;
  l[4] = t1.x; l[5] = t1.y; l[6] = t1.z; l[7] = t1.w;
  l[8] = t2.x; l[9] = t2.y; l[10] = t2.z; l[11] = t2.w;
  l[12] = t3.x; l[13] = t3.y; l[14] = t3.z; l[15] = t3.w;
  l[16] = t4.x; l[17] = t4.y;
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
  int form = 0; // FP32-arithmetic direct hop: 0 two slices per thread (hop_pair.cu), 1 one unit per thread,
                // 2 two slices per thread with prefetching (hop_pair.cu)
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

// Structured fifth-dimension epilogues of the fast hop kernel (hop_fast.cu).
enum Epi { E_RAW = 0, E_BAINV = 1, E_AINVD_BD = 2, E_A_SAME = 3, E_AD_SAME_BD = 4, E_AINV_SAME = 5,
           // symmetric Schur form: add + g same + A^-1 (kappa H in); add + g same + kappa B^+ H in;
           // A^-+ same (no hop)
           E_SAME_AINV = 6, E_SAME_BD = 7, E_AINVD_SAME = 8 };

// A = alpha + beta P, B = b5 + c5 P; kap = beta / alpha; mass[r] = m_f of slot r.
template <typename T>
struct Fifth {
  T alpha, beta, b5, c5, inv_alpha, kap;
  T powL;          // (-kap)^L5
  const T* mass;
};

template <typename S, typename T>
struct FastArgs {
  Geom g;
  int L5, N;
  int out_par, dagger, antiperiodic;
  const S* in; const float* in_nrm;
  const S* same; const float* same_nrm;
  const S* add; const float* add_nrm;
  S* out; float* out_nrm;
  const T* U;
  const uint32_t* F16;  // tensor-core hop: fp16 B fragments [parity][h][mu][fwd, bwd][lane], or null
  const float* U12 = nullptr;  // two-row (12-real) FP32 links [parity][h][mu][12] (hop_pair.cu only)
  // Domain decomposition in time (hop_fast.cu kernels): when halo_fwd is set, the
  // t-neighbours across both edges of the local lattice come from the faces of
  // the neighbouring sub-domains instead of the local field: halo_fwd[(lex3 L5 + s) N + r]
  // holds the 12 reals of the projected half spinor of the next sub-domain's
  // first slice, halo_bwd those of U^+ times the projected half spinor of the
  // previous sub-domain's last slice (lex3 = x + Lx (y + Ly z)); each face carries
  // its boundary factor (-1 across the antiperiodic global time boundary).
  const T* halo_fwd = nullptr;
  const T* halo_bwd = nullptr;
  T halo_sgn_fwd = T(1), halo_sgn_bwd = T(1);
  Fifth<T> f;
  T g_same;             // coefficient of A same (E_A_SAME) / A^+ same (E_AD_SAME_BD)
  T kappa;              // coefficient of the hop term
  const int* active;
  double* partials;
};

// Shared-memory staging of the neighbour sites (hop_staged_kernel).
#define MDWF_TIMEOUT_CODE 1
struct StageInfo {
  unsigned spin_bytes;  // 8 * nsb * (L5 N) stored spinors
  unsigned nrm_bytes;   // 8 * nsb * (L5 N) fp16 scales (0: loaded directly)
  long long budget;     // bound of every barrier wait, in clock cycles
  unsigned extra_tx;    // bytes a barrier waits for beyond the copies (0; nonzero only to test the timeout)
  int* err;             // device status word: set to MDWF_TIMEOUT_CODE when a wait runs out
};

template <typename S, typename T>
cudaError_t launch_fast(const FastArgs<S, T>& a, const Tiling& t, int epi, cudaStream_t st,
                        const StageInfo* stage = nullptr);
// Two-slices-per-thread hop (hop_pair.cu): block (rt, J = ceil(L5 / 2), nsb).
struct PairShape {
  int J, nsb, rt, threads;
  size_t smem;      // plain form: the epilogue tile (or the reduction buffer)
  size_t smem_pf;   // prefetching form: + the block's links + two stages per thread
};
PairShape pair_shape(int L5, int N, int nsb);
// prefetch: the prefetching form where it applies (fp16 storage, 18-real links,
// shared memory within bounds), else the plain form; both give the same bits.
template <typename S>
cudaError_t launch_pair(const FastArgs<S, float>& a, int nsb, int epi, cudaStream_t st, bool prefetch);
// Tensor-core hop (fp16 storage): usable when a block holds whole sites and L5 N % 8 == 0.
bool mma_hop_usable(const Tiling& t, int L5, int N);
int mma_max_threads();
// stage: bound and status word of the waits of the pipelined form (null: unpipelined form)
// pipelined: the bulk-copy double-buffered form (needs stage), else the thread-per-unit
// form when the tiling allows it (whole warps, L5 rt a multiple of 8), else the tile form
cudaError_t launch_fast_mma(const FastArgs<__half, float>& a, const Tiling& t, int epi, cudaStream_t st,
                            const StageInfo* stage, bool pipelined);
cudaError_t build_link_frags(const double* U64, uint32_t* frag, long nlinks, cudaStream_t st);
// Two-row copy of the padded FP32 links (hop_pair.cu): U12[link][0..11] = U32[link][0..11].
cudaError_t build_link12(const float* U32, float* U12, long nlinks, cudaStream_t st);
// Faces of one parity field for the time-split domain decomposition (hop_fast.cu):
// sites at t = 0 give face_prev (the projected half spinor the previous
// sub-domain's forward hop needs), sites at t = Lt - 1 give face_next (U_t^+ times
// the projected half spinor its backward hop needs); layout as FastArgs::halo_*.
cudaError_t dd_pack_faces(const double* in, const Geom& g, int par, int L5, int N, int dagger, const double* U,
                          double* face_prev, double* face_next, cudaStream_t st);
// Wilson flow (flow.cu): U in the C ABI gauge layout, Z: workspace of 3 * 4V * 18 doubles.
cudaError_t wilson_flow(double* U, const int L[4], double eps, int nsteps, double* Z, cudaStream_t st);
// Sum over sites of Re tr of the six plaquettes into *out (device); part: V doubles of workspace.
cudaError_t plaquette(const double* U, const int L[4], double* part, double* out, cudaStream_t st);
// Shared-memory bytes of a staged launch (0 if the tiling cannot be staged).
template <typename S, typename T>
size_t staged_smem_bytes(const Tiling& t, int L5, int N);
template <typename S, typename T>
int fast_max_threads();

// Kernel launchers (hop.cu).
template <typename S, typename T>
cudaError_t launch_hop(const HopArgs<S, T>& a, const Tiling& t, bool hop, cudaStream_t st);
template <typename S, typename T>
int hop_max_threads();
template <typename S, typename T>
size_t hop_smem_bytes(const Tiling& t, bool two);

}  // namespace mdwf
