// Declarations of the vector kernels in blas.cu.
#pragma once
#include "mdwf_internal.h"

namespace mdwf {

// API layout (one RHS, [s][t][z][y][x][spin][colour][re,im], FP64, device) <-> slot r of a parity field.
template <typename S>
cudaError_t pack_rhs(const double* api, S* out, float* out_nrm, const Geom& g, int L5, int N, int par, int r,
                     cudaStream_t st);
template <typename S>
cudaError_t unpack_rhs(const S* in, const float* in_nrm, double* api, const Geom& g, int L5, int N, int par, int r,
                       cudaStream_t st);

template <typename Si, typename So>
cudaError_t convert(const Si* in, const float* in_nrm, So* out, float* out_nrm, const Tiling& t, long Vh, int L5,
                    int N, const int* mask, cudaStream_t st);

template <typename SX, typename S>
cudaError_t axpy_x_rho(SX* x, const S* p, const float* p_nrm, S* rho, float* rho_nrm, const S* q, const float* q_nrm,
                       const double* alpha, const Tiling& t, long Vh, int L5, int N, const int* active,
                       double* partials, cudaStream_t st);

template <typename S>
cudaError_t xpay(const S* r, const float* r_nrm, S* p, float* p_nrm, const double* beta, const Tiling& t, long Vh,
                 int L5, int N, const int* active, cudaStream_t st);

template <typename SX>
cudaError_t accum_xhi(double* xhi, SX* xlo, const Tiling& t, long Vh, int L5, int N, const int* mask,
                      cudaStream_t st);
// x_lo = 0 for the slots in mask.
template <typename SX>
cudaError_t zero_xlo(SX* xlo, const Tiling& t, long Vh, int L5, int N, const int* mask, cudaStream_t st);
// Units a solution accumulator x_lo holds for the tiling t: an FP32 accumulator
// is stored tile-major (see blas.cu) and spans every thread of the grid; an
// FP64 one is unit-major, `units` long.  axpy_x_rho, accum_xhi and zero_xlo read
// and write x_lo in that layout, and must be given the same tiling.
long xlo_units(const Tiling& t, long units, bool tile_major);

template <typename S>
cudaError_t norm2_partials(const S* v, const float* v_nrm, const Tiling& t, long Vh, int L5, int N, const int* mask,
                           double* partials, cudaStream_t st);

template <typename S>
cudaError_t bop(const S* x, const float* x_nrm, S* u, float* u_nrm, const Fifth<typename StoreTraits<S>::T>& f,
                const Tiling& t, long Vh, int L5, int N, const int* mask, cudaStream_t st);

template <typename S>
cudaError_t xpay_b(const S* r, const float* r_nrm, S* p, float* p_nrm, S* u, float* u_nrm, const double* beta,
                   const Fifth<typename StoreTraits<S>::T>& f, const Tiling& t, long Vh, int L5, int N,
                   const int* active, cudaStream_t st);

template <typename S>
cudaError_t resid_update(const double* bhat, const float* q, S* rho, float* rho_nrm, const Tiling& t, long Vh, int L5,
                         int N, const int* mask, double* partials, cudaStream_t st);

template <typename S>
cudaError_t zero_masked(S* v, float* nrm, const Tiling& t, long Vh, int L5, int N, const int* mask, cudaStream_t st);

cudaError_t walls(const double* eta, double* w, long V, int L5, cudaStream_t st);
cudaError_t z2_source(unsigned long long seed, double* eta, long V, cudaStream_t st);
cudaError_t smear_step(const double* U, const double* in, double* out, const Geom& g, double k, cudaStream_t st);
cudaError_t mres_correlators(const double* const* xs, int n, long V, int Lt, int L5, double* pp, double* j5,
                             double* c_pp, double* c_j5, cudaStream_t st);

cudaError_t finalize(const double* partials, long ntiles, int N, double* out, cudaStream_t st);

}  // namespace mdwf
