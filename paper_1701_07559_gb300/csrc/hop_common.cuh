// Device helpers shared by the Wilson-hop kernels (hop_fast.cu, hop_pair.cu):
// the 4D site of a thread with its neighbour indices, and the spin projection
// of a colour-major fp16 spinor.
#pragma once
#include "mdwf_internal.h"

namespace mdwf {
namespace hopc {

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


// fp16: project the packed (scaled) values with half2 arithmetic, then unpack and scale.
template <int MU>
__device__ __forceinline__ void project_half(const uint4 q[3], float sg, float* h) {
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
    h[2 * c] = f0.x; h[2 * c + 1] = f0.y;
    h[6 + 2 * c] = f1.x; h[6 + 2 * c + 1] = f1.y;
  }
}

}  // namespace hopc
using hopc::Site;
using hopc::make_site;
using hopc::nbr_half;
using hopc::project_half;
}  // namespace mdwf
