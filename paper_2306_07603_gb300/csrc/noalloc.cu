// ifdlbm_residual_fields_static: the Eq. (2.19) residuals of two sets of
// caller-owned device fields, with no device allocation of any kind.
//
// The per-block partial sums live in one file-scope __device__ array of fixed
// size that every GPU loading this library keeps until the process exits.
// Host code never uses the array's name as a pointer: its device address is
// taken once per device with cudaGetSymbolAddress (with that device current)
// and passed to the kernels.
#include <cstdio>
#include <mutex>

#include "ifdlbm.h"
#include "internal.h"
#include "reduce.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = IFDLBM_STATIC_MAX_NODES / kThreads;  // 8192 partial slots
constexpr int kMaxDevices = 64;

// 8192 slots x 8 doubles = 512 KiB per device.
static __device__ __align__(256) double g_static_partials[kMaxBlocks * ifd::NPART];

std::mutex g_mu;
double *g_addr[kMaxDevices] = {nullptr};

__global__ void __launch_bounds__(kThreads)
    k_field_partials(int64_t n, const double *u1, const double *v1, const double *p1,
                     const double *u0, const double *v0, const double *p0, double *part) {
  const int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x;
  ifd::Partial p = {0, 0, 0, 0, 0, 0, 0};
  if (k < n) {
    const double du = u1[k] - u0[k], dv = v1[k] - v0[k], dP = p1[k] - p0[k];
    p.du2 = du * du + dv * dv;
    p.u2 = u1[k] * u1[k] + v1[k] * v1[k];
    p.dP2 = dP * dP;
    p.P2 = p1[k] * p1[k];
    p.du2max = p.du2;
    p.u2max = p.u2;
  }
  ifd::block_partial<kThreads / 32>(p, part, blockIdx.x);
}

__global__ void __launch_bounds__(kThreads) k_field_reduce(const double *part, int nslots,
                                                           double *out) {
  __shared__ double res[4];
  ifd::reduce_partials(part, nslots, res);
  __syncthreads();
  if (threadIdx.x < 3) out[threadIdx.x] = res[threadIdx.x];
}

// Device address of the partials array on the current device (set-up on the
// first call per device).
int scratch_address(double **ptr) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ifd::set_global_error(IFDLBM_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return ifd::set_global_error(IFDLBM_ERR_INVALID_ARG, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_partials);
    if (e != cudaSuccess || !p)
      return ifd::set_global_error(IFDLBM_ERR_CUDA,
                                   std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    // With lazy module loading the module, and so the array, is set up on
    // first use; load both kernels here too, so that every device resource
    // this entry point needs is taken in this one set-up call.
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_field_partials);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_field_reduce);
    if (e != cudaSuccess)
      return ifd::set_global_error(IFDLBM_ERR_CUDA,
                                   std::string("cudaFuncGetAttributes: ") + cudaGetErrorString(e));
    g_addr[dev] = static_cast<double *>(p);
  }
  *ptr = g_addr[dev];
  return IFDLBM_OK;
}

}  // namespace

extern "C" int ifdlbm_residual_fields_static(int nx, int ny, const double *u1, const double *v1,
                                             const double *p1, const double *u0, const double *v0,
                                             const double *p0, double *out, void *stream) {
  if (nx < 1 || ny < 1 || !u1 || !v1 || !p1 || !u0 || !v0 || !p0 || !out)
    return ifd::set_global_error(IFDLBM_ERR_INVALID_ARG,
                                 "residual_fields_static: need nx, ny >= 1 and non-NULL arrays");
  const int64_t n = int64_t(nx) * ny;
  if (n > IFDLBM_STATIC_MAX_NODES) {
    char buf[200];
    std::snprintf(buf, sizeof buf,
                  "residual_fields_static: %lld nodes exceed the fixed limit of %d nodes of its "
                  "static scratch (use ifdlbm_residual on a handle instead)",
                  (long long)n, IFDLBM_STATIC_MAX_NODES);
    return ifd::set_global_error(IFDLBM_ERR_INVALID_ARG, buf);
  }
  double *part = nullptr;
  int rc = scratch_address(&part);
  if (rc) return rc;
  const int nblocks = int((n + kThreads - 1) / kThreads);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  (void)cudaGetLastError();  // a launch error left by earlier, unrelated work is not this call's
  k_field_partials<<<nblocks, kThreads, 0, s>>>(n, u1, v1, p1, u0, v0, p0, part);
  k_field_reduce<<<1, kThreads, 0, s>>>(part, nblocks, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return ifd::set_global_error(IFDLBM_ERR_CUDA,
                                 std::string("residual_fields_static launch: ") + cudaGetErrorString(e));
  ifd::count_launches(2);
  return IFDLBM_OK;
}
