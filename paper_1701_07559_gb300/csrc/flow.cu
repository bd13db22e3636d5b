// Wilson (gradient) flow of a gauge field on the device, FP64.
//
// The paper smooths its ensembles' links by the gradient flow to t_gf = 1
// (Sec. III, citing Luscher, JHEP 08 (2010) 071) before the domain-wall
// solves.  Here: dV/dt = Z(V) V with Z = -P_TA(Omega), Omega_mu(x) the sum of
// the six plaquettes that start with V_mu(x) (Wilson plaquette action) and
// P_TA(M) = (M - M^+)/2 - tr(M - M^+)/6, integrated by Luscher's three-stage
// Runge-Kutta scheme:
//   W1 = exp(Z0 / 4) W0,  W2 = exp(8/9 Z1 - 17/36 Z0) W1,
//   W3 = exp(3/4 Z2 - 8/9 Z1 + 17/36 Z0) W2,   Z_i = eps Z(W_i).
// exp by scaling and squaring: scale X by 2^-k until |X|_F <= 1/8, sum the
// Taylor series to 12 terms (remainder below 1e-18 at that norm), square k times.
//
// Layout: the C ABI's gauge layout U[t][z][y][x][mu][a][b], complex (re, im),
// one thread per link.  Input preparation: the solver reads links only
// through mdwf_load_gauge.
#include "mdwf_internal.h"

namespace mdwf {

namespace {

struct C2 {
  double re, im;
};
struct M3 {
  C2 m[9];
};

__device__ __forceinline__ void mload(const double* __restrict__ p, M3& a) {
#pragma unroll
  for (int i = 0; i < 9; i++) { a.m[i].re = p[2 * i]; a.m[i].im = p[2 * i + 1]; }
}
__device__ __forceinline__ void mstore(double* p, const M3& a) {
#pragma unroll
  for (int i = 0; i < 9; i++) { p[2 * i] = a.m[i].re; p[2 * i + 1] = a.m[i].im; }
}
// c = a b (BD: c = a b^+)
template <bool BD>
__device__ __forceinline__ void mmul(const M3& a, const M3& b, M3& c) {
  M3 t;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const C2 x = a.m[3 * i + k];
        const C2 y = BD ? C2{b.m[3 * j + k].re, -b.m[3 * j + k].im} : b.m[3 * k + j];
        re += x.re * y.re - x.im * y.im;
        im += x.re * y.im + x.im * y.re;
      }
      t.m[3 * i + j] = C2{re, im};
    }
  c = t;
}

__device__ void mexp(const M3& X, M3& out) {
  double nrm = 0.0;
#pragma unroll
  for (int i = 0; i < 9; i++) nrm += X.m[i].re * X.m[i].re + X.m[i].im * X.m[i].im;
  nrm = sqrt(nrm);
  int sq = 0;
  while (nrm > 0.125 && sq < 64) { nrm *= 0.5; sq++; }
  const double sc = ldexp(1.0, -sq);
  M3 Y, term, sum;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    Y.m[i] = C2{X.m[i].re * sc, X.m[i].im * sc};
    term.m[i] = sum.m[i] = C2{(i % 4 == 0) ? 1.0 : 0.0, 0.0};
  }
  for (int k = 1; k <= 12; k++) {
    mmul<false>(term, Y, term);
    const double inv = 1.0 / k;
#pragma unroll
    for (int i = 0; i < 9; i++) {
      term.m[i].re *= inv;
      term.m[i].im *= inv;
      sum.m[i].re += term.m[i].re;
      sum.m[i].im += term.m[i].im;
    }
  }
  for (int i = 0; i < sq; i++) mmul<false>(sum, sum, sum);
  out = sum;
}

struct Lat {
  int L[4];
  long V;
};

__device__ __forceinline__ long lat_nbr(const Lat& g, const int c[4], int mu, int dir) {
  int d[4] = {c[0], c[1], c[2], c[3]};
  d[mu] = d[mu] + dir;
  if (d[mu] < 0) d[mu] += g.L[mu];
  if (d[mu] >= g.L[mu]) d[mu] -= g.L[mu];
  return d[0] + (long)g.L[0] * (d[1] + (long)g.L[1] * (d[2] + (long)g.L[2] * d[3]));
}

__device__ __forceinline__ const double* lnk(const double* U, long s, int mu) { return U + 18 * (4 * s + mu); }

// Z = eps * (-P_TA(Omega_mu(x))) for every link.
__global__ void k_flow_Z(const double* __restrict__ U, double* __restrict__ Z, Lat g, double eps) {
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 4 * g.V) return;
  const long s = k >> 2;
  const int mu = (int)(k & 3);
  int c[4];
  long r = s;
  for (int i = 0; i < 4; i++) { c[i] = (int)(r % g.L[i]); r /= g.L[i]; }
  M3 Umu, acc, a, b, w;
  mload(lnk(U, s, mu), Umu);
#pragma unroll
  for (int i = 0; i < 9; i++) acc.m[i] = C2{0.0, 0.0};
  const long xp = lat_nbr(g, c, mu, +1);
  int cp[4] = {c[0], c[1], c[2], c[3]};
  cp[mu] = cp[mu] + 1 == g.L[mu] ? 0 : cp[mu] + 1;
  for (int nu = 0; nu < 4; nu++) {
    if (nu == mu) continue;
    const long xn = lat_nbr(g, c, nu, +1), xm = lat_nbr(g, c, nu, -1), xpm = lat_nbr(g, cp, nu, -1);
    // U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
    mload(lnk(U, xp, nu), w);
    mmul<false>(Umu, w, a);
    mload(lnk(U, xn, mu), w);
    mmul<true>(a, w, b);
    mload(lnk(U, s, nu), w);
    mmul<true>(b, w, a);
#pragma unroll
    for (int i = 0; i < 9; i++) { acc.m[i].re += a.m[i].re; acc.m[i].im += a.m[i].im; }
    // U_mu(x) U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)
    mload(lnk(U, xpm, nu), w);
    mmul<true>(Umu, w, a);
    mload(lnk(U, xm, mu), w);
    mmul<true>(a, w, b);
    mload(lnk(U, xm, nu), w);
    mmul<false>(b, w, a);
#pragma unroll
    for (int i = 0; i < 9; i++) { acc.m[i].re += a.m[i].re; acc.m[i].im += a.m[i].im; }
  }
  // -P_TA, scaled by eps
  M3 t;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      const C2 x = acc.m[3 * i + j], y = acc.m[3 * j + i];
      t.m[3 * i + j] = C2{0.5 * (x.re - y.re), 0.5 * (x.im + y.im)};
    }
  const double tr = (t.m[0].im + t.m[4].im + t.m[8].im) / 3.0;
  t.m[0].im -= tr; t.m[4].im -= tr; t.m[8].im -= tr;
#pragma unroll
  for (int i = 0; i < 9; i++) t.m[i] = C2{-eps * t.m[i].re, -eps * t.m[i].im};
  mstore(Z + 18 * k, t);
}

// U <- exp(c0 Z0 + c1 Z1 + c2 Z2) U for every link.
__global__ void k_flow_update(double* __restrict__ U, const double* __restrict__ Z0, const double* __restrict__ Z1,
                              const double* __restrict__ Z2, long nlink, double c0, double c1, double c2) {
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nlink) return;
  M3 X, E, u;
#pragma unroll
  for (int i = 0; i < 18; i++) {
    double v = c0 * Z0[18 * k + i];
    if (Z1) v += c1 * Z1[18 * k + i];
    if (Z2) v += c2 * Z2[18 * k + i];
    if (i & 1) X.m[i >> 1].im = v; else X.m[i >> 1].re = v;
  }
  mexp(X, E);
  mload(U + 18 * k, u);
  mmul<false>(E, u, u);
  mstore(U + 18 * k, u);
}

// Per-site sum of Re tr of the six plaquettes.
__global__ void k_plaq(const double* __restrict__ U, double* __restrict__ part, Lat g) {
  const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  long r = s;
  for (int i = 0; i < 4; i++) { c[i] = (int)(r % g.L[i]); r /= g.L[i]; }
  double tot = 0.0;
  M3 a, b, w, u;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++) {
      mload(lnk(U, s, mu), u);
      mload(lnk(U, lat_nbr(g, c, mu, +1), nu), w);
      mmul<false>(u, w, a);
      mload(lnk(U, lat_nbr(g, c, nu, +1), mu), w);
      mmul<true>(a, w, b);
      mload(lnk(U, s, nu), w);
      mmul<true>(b, w, a);
      tot += a.m[0].re + a.m[4].re + a.m[8].re;
    }
  part[s] = tot;
}

// Fixed-order sum of n doubles by one block.
__global__ void k_sum(const double* __restrict__ v, long n, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (long i = threadIdx.x; i < n; i += 256) s += v[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

}  // namespace

cudaError_t wilson_flow(double* U, const int L[4], double eps, int nsteps, double* Z, cudaStream_t st) {
  Lat g;
  for (int i = 0; i < 4; i++) g.L[i] = L[i];
  g.V = (long)L[0] * L[1] * L[2] * L[3];
  const long nlink = 4 * g.V;
  double* Z0 = Z;
  double* Z1 = Z + 18 * nlink;
  double* Z2 = Z + 36 * nlink;
  const unsigned blk = 128, grid = (unsigned)((nlink + blk - 1) / blk);
  for (int n = 0; n < nsteps; n++) {
    k_flow_Z<<<grid, blk, 0, st>>>(U, Z0, g, eps);
    k_flow_update<<<grid, blk, 0, st>>>(U, Z0, nullptr, nullptr, nlink, 0.25, 0.0, 0.0);
    k_flow_Z<<<grid, blk, 0, st>>>(U, Z1, g, eps);
    k_flow_update<<<grid, blk, 0, st>>>(U, Z0, Z1, nullptr, nlink, -17.0 / 36.0, 8.0 / 9.0, 0.0);
    k_flow_Z<<<grid, blk, 0, st>>>(U, Z2, g, eps);
    k_flow_update<<<grid, blk, 0, st>>>(U, Z0, Z1, Z2, nlink, 17.0 / 36.0, -8.0 / 9.0, 0.75);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t plaquette(const double* U, const int L[4], double* part, double* out, cudaStream_t st) {
  Lat g;
  for (int i = 0; i < 4; i++) g.L[i] = L[i];
  g.V = (long)L[0] * L[1] * L[2] * L[3];
  k_plaq<<<(unsigned)((g.V + 127) / 128), 128, 0, st>>>(U, part, g);
  k_sum<<<1, 256, 0, st>>>(part, g.V, out);
  return cudaGetLastError();
}

}  // namespace mdwf
