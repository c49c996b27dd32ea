// Fixed-order block reductions of the residual partials of Eq. (2.19) and
// Eq. (5.1), shared by the step kernels and the stateless residual.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace ifd {

struct Partial {
  double du2, u2, dP2, P2, ek, du2max, u2max;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block reduction of the residual partials into slot `slot` (fixed order).
template <int NWARPS>
__device__ __forceinline__ void block_partial(Partial p, double *part, int slot) {
  __shared__ double sh[NWARPS][7];
  const int lane = threadIdx.x + threadIdx.y * blockDim.x;
  const int w = lane >> 5, l = lane & 31;
  double v[7] = {warp_sum(p.du2), warp_sum(p.u2), warp_sum(p.dP2), warp_sum(p.P2),
                 warp_sum(p.ek),  warp_max(p.du2max), warp_max(p.u2max)};
  if (l == 0)
#pragma unroll
    for (int k = 0; k < 7; ++k) sh[w][k] = v[k];
  __syncthreads();
  if (lane < 7) {
    double acc = sh[0][lane];
    for (int k = 1; k < NWARPS; ++k) acc = lane < 5 ? acc + sh[k][lane] : fmax(acc, sh[k][lane]);
    part[int64_t(slot) * NPART + lane] = acc;
  }
}

// Adds one node's terms of Eq. (2.19) (new vs old u, v, P) and of Eq. (5.1)
// (composite trapezoidal weights, Jacobian x_xi H) to p; flags a non-finite
// velocity in the status word.
__device__ __forceinline__ void accumulate_residual(Partial &p, double u1, double v1, double P1,
                                                    double u0, double v0, double P0, int i, int j,
                                                    const CavDev &cv, const Geo &geo,
                                                    unsigned *status) {
  if (!(isfinite(u1) && isfinite(v1))) atomicOr(status, 1u);
  const double du = u1 - u0, dv = v1 - v0, dP = P1 - P0;
  const double du2 = du * du + dv * dv, u2 = u1 * u1 + v1 * v1;
  p.du2 += du2;
  p.u2 += u2;
  p.dP2 += dP * dP;
  p.P2 += P1 * P1;
  p.du2max = fmax(p.du2max, du2);
  p.u2max = fmax(p.u2max, u2);
  const double wx = ((i == 0 || i == cv.nx - 1) ? 0.5 : 1.0) * cv.dxi;
  const double wy = ((j == 0 || j == cv.ny - 1) ? 0.5 : 1.0) * cv.deta;
  p.ek += 0.5 * wx * wy * (geo.xxi[cv.goff + j] * cv.H) * u2;
}

// One block of 256 threads: sums slots [0, nslots) of `part` in a fixed
// order and writes out[0] = E(u), out[1] = E(P) (Eq. 2.19), out[2] = the
// max-norm velocity residual, out[3] = the kinetic-energy sum (Eq. 5.1).
__device__ __forceinline__ void reduce_partials(const double *part, int nslots, double *out) {
  __shared__ double sh[256][7];
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int s = threadIdx.x; s < nslots; s += blockDim.x) {
    const double *pp = part + int64_t(s) * NPART;
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += pp[k];
    acc[5] = fmax(acc[5], pp[5]);
    acc[6] = fmax(acc[6], pp[6]);
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) sh[threadIdx.x][k] = acc[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int k = 0; k < 5; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + w][k];
      sh[threadIdx.x][5] = fmax(sh[threadIdx.x][5], sh[threadIdx.x + w][5]);
      sh[threadIdx.x][6] = fmax(sh[threadIdx.x][6], sh[threadIdx.x + w][6]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sqrt(sh[0][0]) / sqrt(sh[0][1]);  // E(u), Eq. (2.19)
    out[1] = sqrt(sh[0][2]) / sqrt(sh[0][3]);  // E(P), Eq. (2.19)
    out[2] = sqrt(sh[0][5]) / sqrt(sh[0][6]);  // max-norm velocity residual
    out[3] = sh[0][4];                          // kinetic energy, Eq. (5.1)
  }
}

// The same reduction by one block of NWARPS warps (any 32-multiple size):
// each thread sums a fixed stride of slots, then a fixed shuffle tree and a
// fixed pass over the warps, so that the result depends only on nslots and
// the block size.
template <int NWARPS>
__device__ __forceinline__ void reduce_partials_block(const double *part, int nslots, double *out) {
  __shared__ double sh[NWARPS][7];
  const int t = threadIdx.x, w = t >> 5, l = t & 31;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int s = t; s < nslots; s += NWARPS * 32) {
    const double *pp = part + int64_t(s) * NPART;
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += pp[k];
    acc[5] = fmax(acc[5], pp[5]);
    acc[6] = fmax(acc[6], pp[6]);
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) acc[k] = warp_sum(acc[k]);
  acc[5] = warp_max(acc[5]);
  acc[6] = warp_max(acc[6]);
  if (l == 0)
#pragma unroll
    for (int k = 0; k < 7; ++k) sh[w][k] = acc[k];
  __syncthreads();
  if (t == 0) {
    double r[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) r[k] = sh[0][k];
    for (int q = 1; q < NWARPS; ++q) {
#pragma unroll
      for (int k = 0; k < 5; ++k) r[k] += sh[q][k];
      r[5] = fmax(r[5], sh[q][5]);
      r[6] = fmax(r[6], sh[q][6]);
    }
    out[0] = sqrt(r[0]) / sqrt(r[1]);  // E(u), Eq. (2.19)
    out[1] = sqrt(r[2]) / sqrt(r[3]);  // E(P), Eq. (2.19)
    out[2] = sqrt(r[5]) / sqrt(r[6]);  // max-norm velocity residual
    out[3] = r[4];                     // kinetic energy, Eq. (5.1)
  }
}

}  // namespace ifd
