// Host implementation of the C ABI declared in include/ifdlbm.h.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <cuda.h>  // CUtensorMap and its encoder's types (the encoder is found at run time)

#include "fastpow.cuh"
#include "ifdlbm.h"
#include "internal.h"
#include "tma.cuh"

using ifd::CavDev;

namespace {

std::atomic<int64_t> g_launches{0};
thread_local std::string g_create_error;

ifdlbm_alloc_fn g_alloc = nullptr;
ifdlbm_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;

struct Alloc {
  void *p;
  size_t bytes;
};

}  // namespace

struct ifdlbm_ctx {
  int ncav = 0;
  int precision = IFDLBM_FP64;
  int kernel = IFDLBM_KERNEL_STAGED;
  int device = 0;
  cudaStream_t stream = nullptr;
  ifdlbm_options opt{};
  std::vector<ifdlbm_cavity> spec;
  std::vector<ifdlbm_quad_cavity> quad;  // general quadrilaterals (empty for trapezoids)
  std::vector<CavDev> cav;
  std::vector<double> courant;
  ifd::Bufs b{};
  int ntiles = 0;
  int ntasks = 0;      // fused kernel tasks
  int fused_nt = 128;  // fused kernel threads per CTA
  int fused_rows = 0;  // rows per task (0: automatic)
  int schedule = IFDLBM_SCHED_GRID;
  int grid = 0;        // CTAs per fused launch
  int task_cap = 0;    // capacity of tasks / order / partial slots
  ifd::Task *tasks = nullptr;
  int *order = nullptr;
  int *counter = nullptr;
  unsigned char *tmaps = nullptr;  // [2][ncav] TMA tensor maps of g[0], g[1] (fused kernel)
  int tma_skip = 0;                // test hook (ifdlbm_inject_tma_timeout)
  // adjoint scratch (allocated on the first adjoint call)
  double *adj_g1 = nullptr, *adj_l1 = nullptr, *adj_fhb = nullptr, *adj_fbarb = nullptr,
         *adj_fbb = nullptr, *adj_lamb2 = nullptr, *adj_ppart = nullptr;
  int *adj_nodes = nullptr;  // [ncav][2] nodes of the psi objective
  int64_t total_plane = 0;
  int64_t geo_len = 0;
  int64_t max_n2 = 0;
  double *stage = nullptr;  // staging for host transfers: 10 * max_n2 doubles
  int cur = 0;
  int64_t steps = 0;
  int64_t rebased_at = 0;  // step count of the last re-basing (FP32DEV)
  int64_t bytes = 0;
  int64_t h2d_bytes = 0;
  std::vector<Alloc> allocs;
  std::string err;
  // graph_chunk steps captured per parity (graph_chunk is even)
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  ifdlbm_alloc_fn alloc = nullptr;
  ifdlbm_free_fn free_fn = nullptr;
  void *alloc_ctx = nullptr;
  // kernel timing (ifdlbm_profile)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, std::pair<size_t, size_t>>> ev_marks;  // kernel, (start, stop)
};

namespace {

int fail(ifdlbm_ctx *h, int code, const std::string &msg) {
  if (h)
    h->err = msg;
  else
    g_create_error = msg;
  return code;
}

int cuda_fail(ifdlbm_ctx *h, cudaError_t e, const char *what) {
  return fail(h, IFDLBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void *dalloc(ifdlbm_ctx *h, size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (h->alloc) {
    p = h->alloc(bytes, (void *)h->stream, h->alloc_ctx);
  } else {
    if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
  }
  if (p) {
    h->allocs.push_back({p, bytes});
    h->bytes += int64_t(bytes);
  }
  return p;
}

void release_all(ifdlbm_ctx *h) {
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear();
  for (int p = 0; p < 2; ++p)
    if (h->gexec[p]) {
      cudaGraphExecDestroy(h->gexec[p]);
      h->gexec[p] = nullptr;
    }
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  for (auto &a : h->allocs) {
    if (h->free_fn)
      h->free_fn(a.p, a.bytes, (void *)h->stream, h->alloc_ctx);
    else
      cudaFree(a.p);
  }
  h->allocs.clear();
}

double cot_deg(double theta_deg) {
  if (theta_deg == 90.0) return 0.0;
  const double t = theta_deg * (M_PI / 180.0);
  return std::cos(t) / std::sin(t);
}

int validate(ifdlbm_ctx *h, int idx, const ifdlbm_cavity &c) {
  char buf[256];
  auto bad = [&](const char *what) {
    std::snprintf(buf, sizeof buf, "cavity %d: %s", idx, what);
    return fail(h, IFDLBM_ERR_INVALID_ARG, buf);
  };
  if (c.nx < 5 || c.ny < 5) return bad("nx and ny must be >= 5");
  if ((int64_t)c.nx * c.ny > (int64_t)1 << 28) return bad("grid larger than 2^28 nodes");
  if (!(c.geom.L > 0) || !(c.geom.H > 0)) return bad("L and H must be > 0");
  if (!(c.geom.theta_deg > 0 && c.geom.theta_deg <= 90)) return bad("theta_deg must be in (0, 90]");
  if (!(c.Re > 0) || !(c.n > 0) || !(c.U_lid > 0)) return bad("Re, n and U_lid must be > 0");
  if (!std::isfinite(c.Re) || !std::isfinite(c.n) || !std::isfinite(c.U_lid))
    return bad("Re, n and U_lid must be finite");
  return IFDLBM_OK;
}

cudaEvent_t next_event(ifdlbm_ctx *h, size_t *idx) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->ev_pool.push_back(e);
  }
  *idx = h->ev_used;
  return h->ev_pool[h->ev_used++];
}

// Runs `launch` bracketed by events when profiling is on.
template <class F>
void timed(ifdlbm_ctx *h, int kernel, F &&launch) {
  if (!h->profiling) {
    launch();
    return;
  }
  size_t a, b;
  cudaEventRecord(next_event(h, &a), h->stream);
  launch();
  cudaEventRecord(next_event(h, &b), h->stream);
  h->ev_marks.push_back({kernel, {a, b}});
}

template <class T>
void enqueue_step(ifdlbm_ctx *h, int parity, bool want_residual) {
  if (h->kernel == IFDLBM_KERNEL_FUSED) {
    ifd::FusedArgs f{};
    f.cav = h->b.cav;
    f.geo = h->b.geo;
    f.tasks = h->tasks;
    f.order = h->order;
    f.counter = h->counter;
    f.ntasks = h->ntasks;
    f.schedule = h->schedule;
    f.g_in = h->b.g[parity];
    f.g_out = h->b.g[parity ^ 1];
    f.tmap_in = h->tmaps + size_t(parity) * h->ncav * ifd::TMAP_BYTES;
    f.lam_in = h->b.lam[parity];
    f.lam_out = h->b.lam[parity ^ 1];
    f.part = h->b.part;
    f.status = h->b.status;
    f.powtab = h->b.powtab;
    f.powt = h->b.powt;
    f.pref = h->b.pref;
    f.cav_done = h->b.cav_done;
    f.implicit = h->opt.lambda_mode == IFDLBM_LAMBDA_IMPLICIT ? 1 : 0;
    f.general = h->quad.empty() ? 0 : 1;
    f.pow32 = h->opt.power_fp32 ? 1 : 0;
    f.tma_skip = h->tma_skip;
    f.resid = h->b.resid;
    f.want_residual = want_residual ? 1 : 0;
    if (h->schedule == IFDLBM_SCHED_DYNAMIC) cudaMemsetAsync(h->counter, 0, sizeof(int), h->stream);
    // the residual of Eq. (2.19) is reduced inside the launch by each cavity's last task
    timed(h, IFDLBM_KPROF_FUSED, [&] { ifd::launch_fused<T>(f, h->fused_nt, h->grid, h->stream); });
    return;
  }
  ifd::StepArgs a{};
  a.cav = h->b.cav;
  a.geo = h->b.geo;
  a.tile_cav = h->b.tile_cav;
  a.g_in = h->b.g[parity];
  a.g_out = h->b.g[parity ^ 1];
  a.lam_in = h->b.lam[parity];
  a.lam_out = h->b.lam[parity ^ 1];
  a.fb = h->b.fb;
  a.fp = h->b.fp;
  a.fh = h->b.fh;
  a.m0 = h->b.m0;
  a.part = h->b.part;
  a.status = h->b.status;
  a.powtab = h->b.powtab;
  a.powt = h->b.powt;
  a.pref = h->b.pref;
  a.want_residual = want_residual ? 1 : 0;
  timed(h, IFDLBM_KPROF_COLLIDE, [&] { ifd::launch_collide<T>(a, h->ntiles, h->stream); });
  timed(h, IFDLBM_KPROF_HALF, [&] { ifd::launch_half<T>(a, h->ntiles, h->stream); });
  timed(h, IFDLBM_KPROF_FULL, [&] { ifd::launch_full<T>(a, h->ntiles, h->stream); });
  if (want_residual)
    timed(h, IFDLBM_KPROF_REDUCE, [&] {
      ifd::launch_residual_reduce(h->b.cav, h->b.part, h->b.resid, h->ncav, h->stream);
    });
}

void enqueue_step_any(ifdlbm_ctx *h, int parity, bool want_residual) {
  if (h->precision == IFDLBM_FP64)
    enqueue_step<double>(h, parity, want_residual);
  else
    enqueue_step<float>(h, parity, want_residual);
}

int launches_per_step(const ifdlbm_ctx *h, bool residual) {
  if (h->kernel == IFDLBM_KERNEL_FUSED) return 1;  // residual reduced inside the launch
  return residual ? 4 : 3;
}

int ensure_graph(ifdlbm_ctx *h, int parity) {
  if (h->gexec[parity]) return IFDLBM_OK;
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamBeginCapture");
  int p = parity;
  for (int s = 0; s < h->opt.graph_chunk; ++s) {
    enqueue_step_any(h, p, false);
    p ^= 1;
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(h->stream, &graph);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->gexec[parity], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
  return IFDLBM_OK;
}

int check_status(ifdlbm_ctx *h) {
  unsigned st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, h->b.status, sizeof st, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "status read");
  if (st & ifd::STATUS_TMA_TIMEOUT)
    return fail(h, IFDLBM_ERR_TIMEOUT, "a TMA row load of the fused kernel did not complete");
  if (st & ifd::STATUS_NONFINITE)
    return fail(h, IFDLBM_ERR_DIVERGED, "a step produced a non-finite velocity");
  return IFDLBM_OK;
}

// cuTensorMapEncodeTiled, looked up in the driver at run time (the library
// links the static runtime, not the driver library).
using TmapEncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
TmapEncodeFn tmap_encoder() {
  static const TmapEncodeFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return TmapEncodeFn(nullptr);
    return reinterpret_cast<TmapEncodeFn>(p);
  }();
  return fn;
}

// Tensor maps of the fused kernel's TMA row loads: per buffer g[p] and cavity,
// the 9 planes of nx x ny elements (row pitch and plane stride of the arena)
// as a 3-D tensor (x = xi, y = eta, z = population), box 32 x 1 x 9, columns
// outside the tensor read as zeros. Only this GPU's own memory is mapped.
int build_tmaps(ifdlbm_ctx *h, size_t tsize) {
  static_assert(sizeof(CUtensorMap) == ifd::TMAP_BYTES, "tensor map size");
  const TmapEncodeFn enc = tmap_encoder();
  if (!enc) return fail(h, IFDLBM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  std::vector<CUtensorMap> maps(size_t(2) * h->ncav);
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k < h->ncav; ++k) {
      const CavDev &cv = h->cav[k];
      void *base = static_cast<char *>(h->b.g[p]) + size_t(9 * cv.off) * tsize;
      const cuuint64_t dims[3] = {cuuint64_t(cv.nx), cuuint64_t(cv.ny), 9};
      const cuuint64_t strides[2] = {cuuint64_t(cv.pitch) * tsize, cuuint64_t(cv.plane) * tsize};
      const cuuint32_t box[3] = {32, 1, 9};
      const cuuint32_t estr[3] = {1, 1, 1};
      const CUresult r =
          enc(&maps[size_t(p) * h->ncav + k],
              tsize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
              base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return fail(h, IFDLBM_ERR_CUDA,
                    "cuTensorMapEncodeTiled failed (error " + std::to_string(int(r)) + ")");
    }
  cudaError_t e = cudaMemcpyAsync(h->tmaps, maps.data(), maps.size() * sizeof(CUtensorMap),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // the host vector goes out of scope
  if (e != cudaSuccess) return cuda_fail(h, e, "tensor map upload");
  h->h2d_bytes += int64_t(maps.size() * sizeof(CUtensorMap));
  return IFDLBM_OK;
}

bool cavity_ok(ifdlbm_ctx *h, int cavity) { return h && cavity >= 0 && cavity < h->ncav; }

// (Re)builds the fused kernel's tasks: per cavity, balanced strips of at most
// nt/2 - 8 columns times balanced segments of about `rows` rows (0: automatic),
// partial slots per cavity contiguous, and the scheduling order (largest
// tasks first). Uploads the tasks, the order and the cavity table; drops
// captured graphs. Asynchronous on the handle's stream.
int build_fused_tasks(ifdlbm_ctx *h, int nt, int rows, int sched) {
  const int W = ifd::fused_strip_width(nt);
  std::vector<ifd::Task> tasks;
  for (int k = 0; k < h->ncav; ++k) {
    CavDev &cv = h->cav[k];
    const int hs = rows ? rows : (h->total_plane < (int64_t(8) << 20) ? 32 : 64);
    // strips of a common width, a multiple of 4 columns (W is one too), so
    // that every strip starts on a 16-byte boundary: the fused kernel's TMA
    // row loads start at column i0 - 4 (+ 32 per warp)
    const int sx0 = (cv.nx + W - 1) / W;
    const int w4 = (((cv.nx + sx0 - 1) / sx0) + 3) / 4 * 4;
    const int sx = (cv.nx + w4 - 1) / w4;
    // a last strip of one column (the right wall alone) would not form column
    // nx - 2, from which the wall column extrapolates: its start moves 4 left
    const int shift = (sx >= 2 && cv.nx - (sx - 1) * w4 < 2) ? 4 : 0;
    const int sy = std::max(1, std::min((cv.ny + hs - 1) / hs, cv.ny / 2));
    cv.part0 = int(tasks.size());
    for (int b = 0; b < sy; ++b)
      for (int a = 0; a < sx; ++a) {
        ifd::Task t{};
        t.cav = k;
        t.i0 = a * w4 - (a == sx - 1 ? shift : 0);
        t.i1 = a == sx - 1 ? cv.nx : (a + 1) * w4 - (a == sx - 2 ? shift : 0);
        t.j0 = int(int64_t(b) * cv.ny / sy);
        t.j1 = int(int64_t(b + 1) * cv.ny / sy);
        tasks.push_back(t);
      }
    cv.nparts = int(tasks.size()) - cv.part0;
  }
  if (int(tasks.size()) > h->task_cap)
    return fail(h, IFDLBM_ERR_INVALID_ARG, "fused layout needs more tasks than allocated");
  std::vector<int> order(tasks.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = int(i);
  auto cost = [&](int i) {
    const ifd::Task &t = tasks[i];
    return int64_t(t.i1 - t.i0 + 8) * (t.j1 - t.j0 + 8);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  const bool fp64 = h->precision == IFDLBM_FP64;
  const int per_sm = fp64 ? ifd::fused_blocks_per_sm<double>(nt) : ifd::fused_blocks_per_sm<float>(nt);
  if (per_sm < 1) return fail(h, IFDLBM_ERR_INVALID_ARG, "fused layout does not fit on an SM");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  h->ntasks = int(tasks.size());
  h->fused_nt = nt;
  h->fused_rows = rows;
  h->schedule = sched;
  h->grid = sched == IFDLBM_SCHED_GRID ? h->ntasks : std::min(h->ntasks, sms * per_sm);
  for (int p = 0; p < 2; ++p)
    if (h->gexec[p]) {
      cudaGraphExecDestroy(h->gexec[p]);
      h->gexec[p] = nullptr;
    }
  cudaError_t e = cudaMemcpyAsync(h->tasks, tasks.data(), tasks.size() * sizeof(ifd::Task),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->b.cav, h->cav.data(), h->cav.size() * sizeof(CavDev),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // host vectors go out of scope
  if (e != cudaSuccess) return cuda_fail(h, e, "fused tasks upload");
  h->h2d_bytes += int64_t(tasks.size() * (sizeof(ifd::Task) + sizeof(int)) +
                          h->cav.size() * sizeof(CavDev));
  return IFDLBM_OK;
}

}  // namespace

int ifd::set_global_error(int code, const std::string &msg) { return fail(nullptr, code, msg); }

// Tables of pow_fast, in extended precision on the host: r_j = 1/(1 + (j + 1/2)/256)
// rounded to double, L_j = -log2(r_j) of that double, T_j = 2^(j/256).
void ifd::fill_pow_tables(double *tab) {
  for (int j = 0; j < 256; ++j) {
    const long double c = 1.0L + (j + 0.5L) / 256.0L;
    const double r = double(1.0L / c);
    tab[j] = r;
    tab[256 + j] = double(-log2l((long double)r));
    tab[512 + j] = double(exp2l((long double)j / 256.0L));
  }
}
// Table of pow_tab for exponent m and factor C, in extended precision:
// [2j] = c_j^m, [2j + 1] = 1/c_j with c_j = 1 + (j + 1/2)/256 (exact), and
// [512 + e] = C 2^(m (e - 127)), each rounded once to double.
void ifd::fill_cavity_pow_table(double *tab, double m, double C) {
  const long double ml = m, Cl = C;
  for (int j = 0; j < 256; ++j) {
    const long double c = 1.0L + (j + 0.5L) / 256.0L;
    tab[2 * j] = double(powl(c, ml));
    tab[2 * j + 1] = double(1.0L / c);
  }
  for (int e = 0; e < 256; ++e) tab[512 + e] = double(Cl * exp2l(ml * (e - 127)));
}
void ifd::count_launches(int64_t n) { g_launches += n; }

extern "C" {

int ifdlbm_set_allocator(ifdlbm_alloc_fn alloc, ifdlbm_free_fn free_fn, void *ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "allocator and free must be set together");
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return IFDLBM_OK;
}

int ifdlbm_default_options(ifdlbm_options *opt) {
  if (!opt) return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "opt is NULL");
  std::memset(opt, 0, sizeof *opt);
  opt->cfl = 0.5;
  opt->c = 1.0;
  opt->eta_b = 0.5;
  opt->gamma_min = 0.0;
  opt->dt = 0.0;
  opt->rho0 = 1.0;
  opt->precision = IFDLBM_FP64;
  opt->kernel = IFDLBM_KERNEL_AUTO;
  opt->graph_chunk = 32;
  opt->fused_threads = 0;
  opt->fused_rows = 0;
  opt->schedule = IFDLBM_SCHED_GRID;
  opt->dt_mode = IFDLBM_DT_CONTRAVARIANT;
  opt->lambda_mode = IFDLBM_LAMBDA_LAGGED;
  opt->power_fp32 = 0;
  return IFDLBM_OK;
}

}  // extern "C"

namespace {

int validate_quad(ifdlbm_ctx *h, int idx, const ifdlbm_quad_cavity &q) {
  char buf[256];
  auto bad = [&](const char *what) {
    std::snprintf(buf, sizeof buf, "quad cavity %d: %s", idx, what);
    return fail(h, IFDLBM_ERR_INVALID_ARG, buf);
  };
  for (double v : q.corners)
    if (!std::isfinite(v)) return bad("corners must be finite");
  if (!(q.H > 0) || !std::isfinite(q.H)) return bad("H must be > 0");
  // J is bilinear in (xi, eta): positive at the four corners means positive everywhere
  for (double xi : {0.0, 1.0})
    for (double eta : {0.0, 1.0}) {
      double m[7];
      ifd::quad_node_metrics(q.corners, xi, eta, m);
      if (!(m[6] > 0)) return bad("corners must make a convex, counter-clockwise quadrilateral");
    }
  const double tl = std::hypot(q.corners[6] - q.corners[4], q.corners[7] - q.corners[5]);
  if (!(tl > 0)) return bad("the top edge has zero length");
  return IFDLBM_OK;
}

// Shared by ifdlbm_create_batch (trapezoids) and ifdlbm_create_quad_batch
// (general quadrilaterals: `quads` non-NULL; `cavs` then holds their sizes
// and flow parameters).
int create_impl(int ncav, const ifdlbm_cavity *cavs, const ifdlbm_quad_cavity *quads,
                const ifdlbm_options *opt_in, void *stream, ifdlbm_handle *out) {
  ifdlbm_options opt;
  if (opt_in)
    opt = *opt_in;
  else
    ifdlbm_default_options(&opt);
  if (!(opt.cfl > 0) || !(opt.c > 0) || !(opt.eta_b >= 0 && opt.eta_b <= 1) || !(opt.rho0 > 0))
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: need cfl > 0, c > 0, eta_b in [0,1], rho0 > 0");
  if (opt.gamma_min > 0 && opt.gamma_min < 1e-100)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: gamma_min must be 0 (default) or >= 1e-100");
  if (opt.precision != IFDLBM_FP64 && opt.precision != IFDLBM_FP32DEV)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: unknown precision");
  if (opt.kernel < IFDLBM_KERNEL_AUTO || opt.kernel > IFDLBM_KERNEL_FUSED)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: unknown kernel");
  if (!(opt.fused_threads == 0 || opt.fused_threads == 64 || opt.fused_threads == 128 ||
        opt.fused_threads == 256))
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: fused_threads must be 0, 64, 128 or 256");
  if (opt.dt_mode != IFDLBM_DT_GRID && opt.dt_mode != IFDLBM_DT_CONTRAVARIANT)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: unknown dt_mode");
  if (opt.lambda_mode != IFDLBM_LAMBDA_LAGGED && opt.lambda_mode != IFDLBM_LAMBDA_IMPLICIT)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: unknown lambda_mode");
  if (opt.wall_pressure != IFDLBM_WALLP_ZEROTH && opt.wall_pressure != IFDLBM_WALLP_FIRST)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: unknown wall_pressure");
  if (opt.wall_pressure == IFDLBM_WALLP_FIRST && opt.kernel == IFDLBM_KERNEL_FUSED)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG,
                "options: the first-order wall pressure runs on the staged kernels");
  if (opt.power_fp32 != 0 && opt.power_fp32 != 1)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: power_fp32 must be 0 or 1");
  if (opt.power_fp32 && opt.precision != IFDLBM_FP32DEV)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: power_fp32 needs precision FP32DEV");
  if (opt.schedule < IFDLBM_SCHED_GRID || opt.schedule > IFDLBM_SCHED_DYNAMIC)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: unknown schedule");
  if (opt.fused_rows < 0 || opt.fused_rows == 1)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: fused_rows must be 0 or >= 2");
  if (opt.graph_chunk < 0 || (opt.graph_chunk % 2) != 0)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "options: graph_chunk must be 0 or even and > 0");
  // general quadrilaterals: the fused kernel has an FP32, lagged-lambda variant
  const bool quad_fused_ok = opt.precision == IFDLBM_FP32DEV && opt.lambda_mode == IFDLBM_LAMBDA_LAGGED;
  if (quads && opt.kernel == IFDLBM_KERNEL_FUSED && !quad_fused_ok)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG,
                "general quadrilaterals: the fused kernel needs FP32DEV and the lagged lambda "
                "(kernel AUTO or STAGED otherwise)");
  if (quads && opt.dt <= 0 && opt.dt_mode == IFDLBM_DT_GRID)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG,
                "dt_mode GRID is defined for trapezoids; give dt or use CONTRAVARIANT");

  auto *h = new ifdlbm_ctx();
  h->alloc = g_alloc;
  h->free_fn = g_free;
  h->alloc_ctx = g_alloc_ctx;
  for (int k = 0; k < ncav; ++k) {
    int rc = validate(h, k, cavs[k]);
    if (!rc && quads) rc = validate_quad(h, k, quads[k]);
    if (rc) {
      g_create_error = h->err;
      delete h;
      return rc;
    }
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev < 1) {
    delete h;
    return fail(nullptr, IFDLBM_ERR_CUDA, "no CUDA device is available");
  }
  cudaGetDevice(&h->device);
  h->ncav = ncav;
  h->opt = opt;
  h->precision = opt.precision;
  h->kernel = opt.kernel != IFDLBM_KERNEL_AUTO
                  ? opt.kernel
                  : (opt.precision == IFDLBM_FP32DEV && (!quads || quad_fused_ok) &&
                             opt.wall_pressure == IFDLBM_WALLP_ZEROTH
                         ? IFDLBM_KERNEL_FUSED
                         : IFDLBM_KERNEL_STAGED);
  h->fused_nt = opt.fused_threads ? opt.fused_threads : 128;
  const bool fused = h->kernel == IFDLBM_KERNEL_FUSED;
  h->stream = (cudaStream_t)stream;
  if (h->stream == nullptr) h->opt.graph_chunk = 0;  // the legacy stream cannot be captured
  h->spec.assign(cavs, cavs + ncav);
  if (quads) h->quad.assign(quads, quads + ncav);

  const size_t tsize = opt.precision == IFDLBM_FP64 ? sizeof(double) : sizeof(float);
  int64_t off = 0, goff = 0;
  int tile0 = 0;
  h->cav.resize(ncav);
  h->courant.resize(ncav);
  std::vector<double> xix, xeH, xxi, xeta;
  for (int k = 0; k < ncav; ++k) {
    const ifdlbm_cavity &s = cavs[k];
    CavDev &cv = h->cav[k];
    cv.nx = s.nx;
    cv.ny = s.ny;
    cv.pitch = (s.nx + 31) / 32 * 32;
    cv.plane = int64_t(s.ny) * cv.pitch;
    cv.off = off;
    off += cv.plane;
    cv.tiles_x = (s.nx + ifd::TILE_X - 1) / ifd::TILE_X;
    cv.tiles_y = (s.ny + ifd::TILE_Y - 1) / ifd::TILE_Y;
    cv.tile0 = tile0;
    tile0 += cv.tiles_x * cv.tiles_y;
    cv.part0 = cv.tile0;
    cv.nparts = cv.tiles_x * cv.tiles_y;
    cv.goff = goff;
    const int glen = std::max(s.nx, s.ny);
    goff += glen;
    const double L = s.geom.L, H = s.geom.H, ct = cot_deg(s.geom.theta_deg);
    cv.c = opt.c;
    cv.cs2 = opt.c * opt.c / 3.0;
    cv.inv_cs2 = 1.0 / cv.cs2;
    cv.K = std::pow(s.U_lid, 2.0 - s.n) * std::pow(H, s.n) / s.Re;  // Eq. (2.15.1)
    cv.nm1 = s.n - 1.0;
    cv.implicit = opt.lambda_mode == IFDLBM_LAMBDA_IMPLICIT ? 1 : 0;
    cv.wallp = opt.wall_pressure == IFDLBM_WALLP_FIRST ? 1 : 0;
    cv.pow32 = opt.power_fp32 ? 1 : 0;
    cv.gmin = opt.gamma_min > 0 ? opt.gamma_min : 1e-3 * s.U_lid / H;
    cv.dt = opt.dt > 0 ? opt.dt : opt.cfl * std::min(L / (s.nx - 1), H / (s.ny - 1)) / opt.c;
    cv.general = quads ? 1 : 0;
    cv.lid_ux = s.U_lid;
    cv.lid_uy = 0.0;
    if (quads) {
      // the lid moves along the top edge (corner 2 to 3); the per-node metric
      // planes are formed on the device (launch_quad_metrics)
      const double *cr = quads[k].corners;
      const double tl = std::hypot(cr[6] - cr[4], cr[7] - cr[5]);
      cv.lid_ux = s.U_lid * (cr[6] - cr[4]) / tl;
      cv.lid_uy = s.U_lid * (cr[7] - cr[5]) / tl;
    }
    if (quads && opt.dt <= 0) {
      // CFL on the contravariant speeds of Eq. (3.4), maxima over all nodes.
      // For the bilinear map c_xi = c (e_x y_eta - e_y x_eta) / J and
      // c_eta = c (e_y x_xi - e_x y_xi) / J, with x_xi, y_xi functions of eta
      // only, x_eta, y_eta of xi only and J > 0 linear in each coordinate: along
      // every grid line each is a ratio of linear functions, monotonic, so the
      // maxima of |c_xi| and |c_eta| sit at the four corner nodes.
      double mxi = 0.0, meta = 0.0;
      for (double xi : {0.0, 1.0})
        for (double eta : {0.0, 1.0}) {
          double m[7];
          ifd::quad_node_metrics(quads[k].corners, xi, eta, m);
          for (int q = 1; q < 9; ++q) {
            static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
            static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
            mxi = std::max(mxi, std::fabs(opt.c * (EX[q] * m[0] + EY[q] * m[1])));
            meta = std::max(meta, std::fabs(opt.c * (EX[q] * m[2] + EY[q] * m[3])));
          }
        }
      cv.dt = opt.cfl * std::min((1.0 / (s.nx - 1)) / mxi, (1.0 / (s.ny - 1)) / meta);
    } else if (opt.dt <= 0 && opt.dt_mode == IFDLBM_DT_CONTRAVARIANT) {
      // CFL applied to the contravariant speeds of Eq. (3.4): their largest
      // magnitudes sit at the ends of the xi range and at eta = 0 (x_xi smallest)
      double mxi = 0.0;
      for (int jj : {0, s.ny - 1})
        for (int ii : {0, s.nx - 1})
          for (int q = 1; q < 9; ++q) {
            static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
            static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
            const double eta = double(jj) / (s.ny - 1), xi = double(ii) / (s.nx - 1);
            const double x_xi = L + 2.0 * H * ct * eta, x_eta = H * ct * (2.0 * xi - 1.0);
            mxi = std::max(mxi, std::fabs(opt.c * (EX[q] - EY[q] * x_eta / H) / x_xi));
          }
      const double meta = opt.c / H;
      cv.dt = opt.cfl * std::min((1.0 / (s.nx - 1)) / mxi, (1.0 / (s.ny - 1)) / meta);
    }
    cv.eta_b = opt.eta_b;
    cv.dxi = 1.0 / (s.nx - 1);
    cv.deta = 1.0 / (s.ny - 1);
    cv.inv2dxi = 1.0 / (2.0 * cv.dxi);
    cv.inv2deta = 1.0 / (2.0 * cv.deta);
    cv.U = s.U_lid;
    cv.H = H;
    cv.rho0 = opt.rho0;
    cv.lam0 = cv.K * std::pow(cv.gmin, cv.nm1) / cv.cs2;
    cv.gmin2 = cv.gmin * cv.gmin;
    {
      const double t = s.geom.theta_deg * (M_PI / 180.0), sn = std::sin(t);
      cv.dcot = -(M_PI / 180.0) / (sn * sn);
    }
    cv.lnHU = std::log(H) - std::log(s.U_lid);
    cv.Re = s.Re;
    cv.half_nm1 = 0.5 * cv.nm1;
    cv.Kics2 = cv.K / cv.cs2;
    {  // pow_tab: binomial coefficients of (1 + t)^m, m = (n - 1)/2, and the FP32 clamp
      const double m = cv.half_nm1;
      cv.pb2 = m * (m - 1.0) / 2.0;
      cv.pb3 = float(cv.pb2 * (m - 2.0) / 3.0);
      cv.pb4 = float(cv.pb2 * (m - 2.0) * (m - 3.0) / 12.0);
      cv.pb5 = float(cv.pb2 * (m - 2.0) * (m - 3.0) * (m - 4.0) / 60.0);
      float g = float(cv.gmin2);
      if (double(g) > cv.gmin2) g = std::nextafter(g, 0.0f);
      cv.gmin2_f = std::max(g, FLT_MIN);
    }
    h->max_n2 = std::max<int64_t>(h->max_n2, int64_t(s.nx) * s.ny);
    // 1-D metric arrays of Eq. (3.8.2)
    xix.resize(goff), xeH.resize(goff), xxi.resize(goff), xeta.resize(goff);
    double cmax = 0;
    for (int j = 0; j < glen; ++j) {
      const double eta = j < s.ny ? double(j) / (s.ny - 1) : 1.0;
      const double x_xi = L + 2.0 * H * ct * eta;
      xxi[cv.goff + j] = x_xi;
      xix[cv.goff + j] = 1.0 / x_xi;
    }
    for (int i = 0; i < glen; ++i) {
      const double xi = i < s.nx ? double(i) / (s.nx - 1) : 1.0;
      const double x_eta = H * ct * (2.0 * xi - 1.0);
      xeta[cv.goff + i] = x_eta;
      xeH[cv.goff + i] = x_eta / H;
    }
    // (general quadrilaterals: dt (|c_xi| / dxi + |c_eta| / deta) is, along
    // each grid line, a ratio of piecewise linear functions to a positive
    // linear one, largest at an end: the corner nodes suffice)
    for (int j = 0; j < s.ny; j += quads ? std::max(1, s.ny - 1) : 1)
      for (int i = 0; i < s.nx; i += std::max(1, s.nx - 1))
        for (int q = 1; q < 9; ++q) {
          static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
          static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
          double cxi, ceta;
          if (quads) {
            double m[7];
            ifd::quad_node_metrics(quads[k].corners, double(i) / (s.nx - 1), double(j) / (s.ny - 1),
                                   m);
            cxi = opt.c * (EX[q] * m[0] + EY[q] * m[1]);
            ceta = opt.c * (EX[q] * m[2] + EY[q] * m[3]);
          } else {
            const double A = opt.c * xix[cv.goff + j];
            cxi = A * (EX[q] - EY[q] * xeH[cv.goff + i]);
            ceta = opt.c * EY[q] / H;
          }
          cmax = std::max(cmax, cv.dt * (std::fabs(cxi) / cv.dxi + std::fabs(ceta) / cv.deta));
        }
    h->courant[k] = cmax;
  }
  h->ntiles = tile0;
  h->total_plane = off;
  h->geo_len = goff;
  if (fused) {  // task capacity: the finest layout the autotuner tries (64 threads, 16 rows)
    int cap = 0;
    const int rmin = opt.fused_rows ? std::min(opt.fused_rows, 16) : 16;
    const int wmin = ifd::fused_strip_width(64);  // the narrowest strips
    for (const CavDev &cv : h->cav)
      cap += ((cv.nx + wmin - 1) / wmin) *
             std::max(1, std::min((cv.ny + rmin - 1) / rmin, cv.ny / 2));
    h->task_cap = std::max(cap, 1);
  }
  auto A = [&](size_t bytes) { return dalloc(h, bytes); };
  bool ok = true;
  for (int p = 0; p < 2; ++p) {
    ok &= (h->b.g[p] = A(9 * off * tsize)) != nullptr;
    ok &= (h->b.lam[p] = A(off * tsize)) != nullptr;
  }
  if (!fused) {  // scratch planes of the staged kernels
    ok &= (h->b.fb = A(9 * off * tsize)) != nullptr;
    ok &= (h->b.fp = A(9 * off * tsize)) != nullptr;
    ok &= (h->b.fh = A(9 * off * tsize)) != nullptr;
    ok &= (h->b.m0 = (double *)A(3 * off * sizeof(double))) != nullptr;
  } else {
    ok &= (h->tasks = (ifd::Task *)A(size_t(h->task_cap) * sizeof(ifd::Task))) != nullptr;
    ok &= (h->order = (int *)A(size_t(h->task_cap) * sizeof(int))) != nullptr;
    ok &= (h->counter = (int *)A(sizeof(int))) != nullptr;
    ok &= (h->tmaps = (unsigned char *)A(size_t(2) * ncav * ifd::TMAP_BYTES)) != nullptr;
  }
  const int nslots = fused ? h->task_cap : h->ntiles;
  ok &= (h->b.part = (double *)A(size_t(nslots) * ifd::NPART * sizeof(double))) != nullptr;
  ok &= (h->b.resid = (double *)A(size_t(ncav) * 4 * sizeof(double))) != nullptr;
  ok &= (h->b.tile_cav = (int *)A(size_t(h->ntiles) * sizeof(int))) != nullptr;
  ok &= (h->b.status = (unsigned *)A(sizeof(unsigned))) != nullptr;
  ok &= (h->b.cav = (CavDev *)A(size_t(ncav) * sizeof(CavDev))) != nullptr;
  double *geo = (double *)A(size_t(4 * goff) * sizeof(double));
  ok &= geo != nullptr;
  float *geof = (float *)A(size_t(2 * goff) * sizeof(float));
  ok &= geof != nullptr;
  ok &= (h->stage = (double *)A(size_t(10 * h->max_n2) * sizeof(double))) != nullptr;
  ok &= (h->b.powtab = (double *)A(ifd::POW_TABLE_SIZE * sizeof(double))) != nullptr;
  ok &= (h->b.powt = (double *)A(size_t(ncav) * ifd::POWT_SIZE * sizeof(double))) != nullptr;
  ok &= (h->b.pref = (double *)A(size_t(ncav) * sizeof(double))) != nullptr;
  ok &= (h->b.cav_done = (int *)A(size_t(ncav) * sizeof(int))) != nullptr;
  ok &= (h->b.ptile = (double *)A(size_t(h->ntiles + ncav) * sizeof(double))) != nullptr;
  double *gmet = nullptr;
  float *qmet_f = nullptr;  // FP32 roundings of the FP64 metrics (fused FP32 kernel)
  double *qcorners = nullptr;
  if (quads) ok &= (gmet = (double *)A(size_t(7 * off) * sizeof(double))) != nullptr;
  if (quads) ok &= (qcorners = (double *)A(size_t(8 * ncav) * sizeof(double))) != nullptr;
  if (quads && fused) ok &= (qmet_f = (float *)A(size_t(5 * off) * sizeof(float))) != nullptr;
  if (!ok) {
    release_all(h);
    delete h;
    return fail(nullptr, IFDLBM_ERR_OOM, "device allocation failed");
  }
  h->b.geo.xix = geo;
  h->b.geo.xeH = geo + goff;
  h->b.geo.xxi = geo + 2 * goff;
  h->b.geo.xeta = geo + 3 * goff;
  h->b.geo.cxix_f = geof;
  h->b.geo.jac_f = geof + goff;
  h->b.geo.gmet = gmet;
  h->b.geo.qmet_f = qmet_f;
  std::vector<float> geof_h(2 * goff);
  for (int k = 0; k < ncav; ++k) {
    const CavDev &cv = h->cav[k];
    for (int j = 0; j < cv.ny; ++j) {
      geof_h[cv.goff + j] = float(cv.c * xix[cv.goff + j]);
      geof_h[goff + cv.goff + j] = float(xxi[cv.goff + j] * cv.H);
    }
  }

  std::vector<int> tile_cav(h->ntiles);
  for (int k = 0; k < ncav; ++k)
    for (int t = 0; t < h->cav[k].tiles_x * h->cav[k].tiles_y; ++t) tile_cav[h->cav[k].tile0 + t] = k;
  std::vector<double> geo_h(4 * goff);
  std::copy(xix.begin(), xix.end(), geo_h.begin());
  std::copy(xeH.begin(), xeH.end(), geo_h.begin() + goff);
  std::copy(xxi.begin(), xxi.end(), geo_h.begin() + 2 * goff);
  std::copy(xeta.begin(), xeta.end(), geo_h.begin() + 3 * goff);

  cudaStream_t s = h->stream;
  h->h2d_bytes = int64_t(tile_cav.size() * sizeof(int) + h->cav.size() * sizeof(CavDev) +
                         geo_h.size() * sizeof(double) + geof_h.size() * sizeof(float) +
                         ifd::POW_TABLE_SIZE * sizeof(double) +
                         size_t(ncav) * ifd::POWT_SIZE * sizeof(double) +
                         (quads ? size_t(8 * ncav) * sizeof(double) : 0));
  e = cudaMemcpyAsync(h->b.tile_cav, tile_cav.data(), tile_cav.size() * sizeof(int),
                      cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->b.cav, h->cav.data(), h->cav.size() * sizeof(CavDev),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(geo, geo_h.data(), geo_h.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(geof, geof_h.data(), geof_h.size() * sizeof(float), cudaMemcpyHostToDevice,
                        s);
  std::vector<double> qcorners_h;
  for (int k = 0; quads && k < ncav; ++k)
    qcorners_h.insert(qcorners_h.end(), quads[k].corners, quads[k].corners + 8);
  if (qcorners && e == cudaSuccess)
    e = cudaMemcpyAsync(qcorners, qcorners_h.data(), qcorners_h.size() * sizeof(double),
                        cudaMemcpyHostToDevice, s);
  if (gmet && e == cudaSuccess) {
    e = cudaMemsetAsync(gmet, 0, size_t(7 * off) * sizeof(double), s);  // row padding too
    if (e == cudaSuccess) {
      ifd::launch_quad_metrics(h->b.cav, ncav, h->max_n2, qcorners, gmet, s);
      g_launches += 1;
      e = cudaGetLastError();
    }
  }
  if (qmet_f && e == cudaSuccess) {
    e = cudaMemsetAsync(qmet_f, 0, size_t(5 * off) * sizeof(float), s);  // row padding too
    if (e == cudaSuccess) {
      ifd::launch_quad_metrics_f32(h->b.cav, ncav, h->max_n2, gmet, qmet_f, s);
      g_launches += 1;
      e = cudaGetLastError();
    }
  }
  static std::vector<double> powtab_h = [] {
    std::vector<double> t(ifd::POW_TABLE_SIZE);
    ifd::fill_pow_tables(t.data());
    return t;
  }();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->b.powtab, powtab_h.data(), powtab_h.size() * sizeof(double),
                        cudaMemcpyHostToDevice, s);
  // The per-cavity tables of pow_tab in extended precision: ~0.5 ms a cavity where
  // long double is software quad precision, so the cavities are spread over host threads.
  std::vector<double> powt_h(size_t(ncav) * ifd::POWT_SIZE);
  {
    auto fill = [&](int k0, int k1) {
      for (int k = k0; k < k1; ++k)
        ifd::fill_cavity_pow_table(powt_h.data() + size_t(k) * ifd::POWT_SIZE, h->cav[k].half_nm1,
                                   h->cav[k].Kics2);
    };
    const int nth = std::max(1, std::min({ncav, 16, int(std::thread::hardware_concurrency())}));
    if (nth == 1) {
      fill(0, ncav);
    } else {
      std::vector<std::thread> pool;
      for (int t = 0; t < nth; ++t) pool.emplace_back(fill, ncav * t / nth, ncav * (t + 1) / nth);
      for (auto &th : pool) th.join();
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->b.powt, powt_h.data(), powt_h.size() * sizeof(double),
                        cudaMemcpyHostToDevice, s);
  // every buffer starts zeroed so that no read can ever see uninitialised memory
  for (void *ptr : {h->b.fb, h->b.fp, h->b.fh, h->b.g[1]})
    if (ptr && e == cudaSuccess) e = cudaMemsetAsync(ptr, 0, 9 * off * tsize, s);
  if (h->b.m0 && e == cudaSuccess) e = cudaMemsetAsync(h->b.m0, 0, 3 * off * sizeof(double), s);
  if (fused && e == cudaSuccess) {
    int rc = build_tmaps(h, tsize);
    if (!rc) rc = build_fused_tasks(h, h->fused_nt, opt.fused_rows, opt.schedule);
    if (rc) {
      std::string msg = h->err;
      release_all(h);
      delete h;
      return fail(nullptr, rc, msg);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->b.lam[1], 0, off * tsize, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->b.resid, 0, size_t(ncav) * 4 * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->b.status, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->b.pref, 0, size_t(ncav) * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->b.cav_done, 0, size_t(ncav) * sizeof(int), s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->b.ptile, 0, size_t(h->ntiles + ncav) * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->b.g[0], 0, 9 * off * tsize, s);
  if (e == cudaSuccess) {
    if (h->precision == IFDLBM_FP64)
      ifd::launch_init<double>(h->b.cav, h->b.tile_cav, h->b.g[0], h->b.lam[0], h->ntiles, s);
    else
      ifd::launch_init<float>(h->b.cav, h->b.tile_cav, h->b.g[0], h->b.lam[0], h->ntiles, s);
    g_launches += 1;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    std::string msg = std::string("create: ") + cudaGetErrorString(e);
    release_all(h);
    delete h;
    return fail(nullptr, IFDLBM_ERR_CUDA, msg);
  }
  *out = h;
  return IFDLBM_OK;
}

}  // namespace

extern "C" {

int ifdlbm_create_batch(int ncav, const ifdlbm_cavity *cavs, const ifdlbm_options *opt,
                        void *stream, ifdlbm_handle *out) {
  if (!out) return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (ncav < 1 || ncav > 4096 || !cavs)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "ncav must be in [1, 4096] with a cavity array");
  return create_impl(ncav, cavs, nullptr, opt, stream, out);
}

int ifdlbm_create_quad_batch(int ncav, const ifdlbm_quad_cavity *quads,
                             const ifdlbm_options *opt, void *stream, ifdlbm_handle *out) {
  if (!out) return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (ncav < 1 || ncav > 4096 || !quads)
    return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "ncav must be in [1, 4096] with a cavity array");
  // sizes and flow parameters in the trapezoid record; its geometry (unit
  // square) serves only the shared checks, the metrics come from the corners
  std::vector<ifdlbm_cavity> cavs(ncav);
  for (int k = 0; k < ncav; ++k) {
    cavs[k].nx = quads[k].nx;
    cavs[k].ny = quads[k].ny;
    cavs[k].geom = ifdlbm_geometry{1.0, quads[k].H, 90.0};
    cavs[k].Re = quads[k].Re;
    cavs[k].n = quads[k].n;
    cavs[k].U_lid = quads[k].U_lid;
  }
  return create_impl(ncav, cavs.data(), quads, opt, stream, out);
}

int ifdlbm_create(int nx, int ny, ifdlbm_geometry g, double Re, double n, double U_lid,
                  const ifdlbm_options *opt, void *stream, ifdlbm_handle *out) {
  ifdlbm_cavity c;
  c.nx = nx;
  c.ny = ny;
  c.geom = g;
  c.Re = Re;
  c.n = n;
  c.U_lid = U_lid;
  return ifdlbm_create_batch(1, &c, opt, stream, out);
}

// FP32 storage: every REBASE_EVERY steps the stored deviations are re-based
// on the cavity's mean pressure (launch_rebase), so that the drift of that
// neutral mode does not enlarge |g| and with it the FP32 rounding. The
// state (f-hat) is unchanged, apart from one rounding of g.
constexpr int64_t REBASE_EVERY = 1024;

static void maybe_rebase(ifdlbm_ctx *h) {
  if (h->precision != IFDLBM_FP32DEV || h->steps - h->rebased_at < REBASE_EVERY) return;
  ifd::launch_rebase<float>(h->b.cav, h->b.tile_cav, h->b.g[h->cur], h->b.pref, h->b.ptile,
                            h->ntiles, h->ncav, h->stream);
  g_launches += 3;
  h->rebased_at = h->steps;
}

int ifdlbm_step(ifdlbm_handle h, int nsteps) {
  if (!h) return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "handle is NULL");
  if (nsteps < 0) return fail(h, IFDLBM_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return IFDLBM_OK;
  cudaSetDevice(h->device);
  int remaining = nsteps - 1;  // the last step also forms the residual
  const int chunk = h->profiling ? 0 : h->opt.graph_chunk;
  if (chunk > 0) {
    while (remaining >= chunk) {
      int rc = ensure_graph(h, h->cur);
      if (rc) return rc;
      cudaError_t e = cudaGraphLaunch(h->gexec[h->cur], h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
      g_launches += int64_t(chunk) * launches_per_step(h, false);
      remaining -= chunk;
      h->steps += chunk;
      maybe_rebase(h);
    }
  }
  for (; remaining > 0; --remaining) {
    enqueue_step_any(h, h->cur, false);
    g_launches += launches_per_step(h, false);
    h->cur ^= 1;
    h->steps += 1;
    maybe_rebase(h);
  }
  enqueue_step_any(h, h->cur, true);
  g_launches += launches_per_step(h, true);
  h->cur ^= 1;
  h->steps += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
  return IFDLBM_OK;
}

int ifdlbm_macros_dev(ifdlbm_handle h, int cavity, double *rho, double *u, double *v,
                      double *psi) {
  if (!cavity_ok(h, cavity)) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle or cavity index");
  cudaSetDevice(h->device);
  const ifdlbm_cavity &s = h->spec[cavity];
  if (h->precision == IFDLBM_FP64)
    ifd::launch_macros<double>(h->b.cav, h->b.geo, cavity, h->b.pref, h->b.g[h->cur], rho, u, v, psi, s.nx,
                               s.ny, h->stream);
  else
    ifd::launch_macros<float>(h->b.cav, h->b.geo, cavity, h->b.pref, h->b.g[h->cur], rho, u, v, psi, s.nx,
                              s.ny, h->stream);
  g_launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "macros launch");
  return IFDLBM_OK;
}

int ifdlbm_batch_macros(ifdlbm_handle h, int cavity, double *rho, double *u, double *v,
                        double *psi) {
  if (!cavity_ok(h, cavity)) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle or cavity index");
  const ifdlbm_cavity &s = h->spec[cavity];
  const int64_t n2 = int64_t(s.nx) * s.ny;
  double *d[4] = {h->stage, h->stage + n2, h->stage + 2 * n2, h->stage + 3 * n2};
  double *dst[4] = {rho, u, v, psi};
  int rc = ifdlbm_macros_dev(h, cavity, d[0], d[1], d[2], d[3]);
  if (rc) return rc;
  for (int k = 0; k < 4; ++k)
    if (dst[k]) {
      cudaError_t e = cudaMemcpyAsync(dst[k], d[k], n2 * sizeof(double), cudaMemcpyDeviceToHost,
                                      h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "macros copy");
    }
  return check_status(h);
}

int ifdlbm_macros(ifdlbm_handle h, double *rho, double *u, double *v, double *psi) {
  return ifdlbm_batch_macros(h, 0, rho, u, v, psi);
}

int ifdlbm_eddies(ifdlbm_handle h, int cavity, ifdlbm_eddy out[3]) {
  if (!cavity_ok(h, cavity) || !out) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle, cavity or out");
  const ifdlbm_cavity &s = h->spec[cavity];
  std::vector<double> psi(size_t(s.nx) * s.ny);
  int rc = ifdlbm_batch_macros(h, cavity, nullptr, nullptr, nullptr, psi.data());
  if (rc) return rc;
  if (h->quad.empty()) {
    rc = ifdlbm_find_eddies(s.nx, s.ny, s.geom, psi.data(), out);
  } else {
    // the finder works in (xi, eta) (unit-square geometry: x = xi, y = eta);
    // the centres are then mapped through the bilinear map of the corners
    rc = ifdlbm_find_eddies(s.nx, s.ny, ifdlbm_geometry{1.0, 1.0, 90.0}, psi.data(), out);
    const double *cr = h->quad[cavity].corners;
    for (int k = 0; k < 3 && !rc; ++k)
      if (out[k].found) {
        const double xi = out[k].xi, eta = out[k].eta;
        const double w0 = (1 - xi) * (1 - eta), w1 = xi * (1 - eta), w2 = (1 - xi) * eta,
                     w3 = xi * eta;
        out[k].x = w0 * cr[0] + w1 * cr[2] + w2 * cr[4] + w3 * cr[6];
        out[k].y = w0 * cr[1] + w1 * cr[3] + w2 * cr[5] + w3 * cr[7];
      }
  }
  if (rc) return fail(h, rc, "eddies: " + std::string(ifdlbm_last_error(nullptr)));
  return IFDLBM_OK;
}

int ifdlbm_batch_residual(ifdlbm_handle h, double *out) {
  if (!h || !out) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle or out");
  cudaSetDevice(h->device);
  cudaError_t e = cudaMemcpyAsync(out, h->b.resid, size_t(h->ncav) * 4 * sizeof(double),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "residual copy");
  return check_status(h);
}

int ifdlbm_batch_residual_async(ifdlbm_handle h, double *out, unsigned *status) {
  if (!h || !out) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle or out");
  cudaSetDevice(h->device);
  cudaError_t e = cudaMemcpyAsync(out, h->b.resid, size_t(h->ncav) * 4 * sizeof(double),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && status)
    e = cudaMemcpyAsync(status, h->b.status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "residual_async copy");
  return IFDLBM_OK;
}

int ifdlbm_residual_dev(ifdlbm_handle h, double *out) {
  if (!h || !out) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle or out");
  cudaSetDevice(h->device);
  cudaError_t e = cudaMemcpyAsync(out, h->b.resid, size_t(h->ncav) * 4 * sizeof(double),
                                  cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "residual_dev copy");
  return IFDLBM_OK;
}

int ifdlbm_probe_dev(ifdlbm_handle h, int n, const int *probes, double *out) {
  if (!h || n < 0 || (n > 0 && (!probes || !out)))
    return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle, count or arrays");
  if (n == 0) return IFDLBM_OK;
  cudaSetDevice(h->device);
  if (h->precision == IFDLBM_FP64)
    ifd::launch_probe<double>(h->b.cav, h->ncav, h->b.pref, h->b.g[h->cur], n, probes, out,
                              h->stream);
  else
    ifd::launch_probe<float>(h->b.cav, h->ncav, h->b.pref, h->b.g[h->cur], n, probes, out,
                             h->stream);
  g_launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "probe launch");
  return IFDLBM_OK;
}

int ifdlbm_residual(ifdlbm_handle h, double *out) {
  if (!h || !out) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle or out");
  if (h->ncav == 1) return ifdlbm_batch_residual(h, out);
  std::vector<double> all(4 * size_t(h->ncav));
  int rc = ifdlbm_batch_residual(h, all.data());
  std::copy(all.begin(), all.begin() + 4, out);
  return rc;
}

int ifdlbm_get_state(ifdlbm_handle h, int cavity, double *fhat, double *lambda_prev) {
  if (!cavity_ok(h, cavity)) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle or cavity index");
  cudaSetDevice(h->device);
  const ifdlbm_cavity &s = h->spec[cavity];
  const int64_t n2 = int64_t(s.nx) * s.ny;
  if (h->precision == IFDLBM_FP64)
    ifd::launch_export<double>(h->b.cav, cavity, h->b.pref, h->b.g[h->cur], h->b.lam[h->cur], h->stage,
                               h->stage + 9 * n2, s.nx, s.ny, h->stream);
  else
    ifd::launch_export<float>(h->b.cav, cavity, h->b.pref, h->b.g[h->cur], h->b.lam[h->cur], h->stage,
                              h->stage + 9 * n2, s.nx, s.ny, h->stream);
  g_launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && fhat)
    e = cudaMemcpyAsync(fhat, h->stage, 9 * n2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && lambda_prev)
    e = cudaMemcpyAsync(lambda_prev, h->stage + 9 * n2, n2 * sizeof(double),
                        cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_state");
  return check_status(h);
}

int ifdlbm_set_state(ifdlbm_handle h, int cavity, const double *fhat, const double *lambda_prev) {
  if (!cavity_ok(h, cavity) || !fhat || !lambda_prev)
    return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle, cavity index or NULL array");
  cudaSetDevice(h->device);
  const ifdlbm_cavity &s = h->spec[cavity];
  const int64_t n2 = int64_t(s.nx) * s.ny;
  cudaError_t e =
      cudaMemcpyAsync(h->stage, fhat, 9 * n2 * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->stage + 9 * n2, lambda_prev, n2 * sizeof(double),
                        cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_state copy");
  if (h->precision == IFDLBM_FP64)
    ifd::launch_import<double>(h->b.cav, cavity, h->b.pref, h->b.g[h->cur], h->b.lam[h->cur], h->stage,
                               h->stage + 9 * n2, s.nx, s.ny, h->stream);
  else
    ifd::launch_import<float>(h->b.cav, cavity, h->b.pref, h->b.g[h->cur], h->b.lam[h->cur], h->stage,
                              h->stage + 9 * n2, s.nx, s.ny, h->stream);
  g_launches += 1;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_state");
  return IFDLBM_OK;
}

int64_t ifdlbm_state_bytes(ifdlbm_handle h) {
  if (!h) return -1;
  const size_t tsize = h->precision == IFDLBM_FP64 ? sizeof(double) : sizeof(float);
  return int64_t(9 * h->total_plane * tsize + h->total_plane * tsize + h->ncav * sizeof(double));
}

int ifdlbm_save_state_dev(ifdlbm_handle h, void *dst) {
  if (!h || !dst) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle or dst");
  cudaSetDevice(h->device);
  const size_t tsize = h->precision == IFDLBM_FP64 ? sizeof(double) : sizeof(float);
  const size_t gb = 9 * h->total_plane * tsize;
  const size_t lb = h->total_plane * tsize;
  cudaError_t e = cudaMemcpyAsync(dst, h->b.g[h->cur], gb, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((char *)dst + gb, h->b.lam[h->cur], lb, cudaMemcpyDeviceToDevice,
                        h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((char *)dst + gb + lb, h->b.pref, h->ncav * sizeof(double),
                        cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "save_state_dev");
  return IFDLBM_OK;
}

int ifdlbm_load_state_dev(ifdlbm_handle h, const void *src) {
  if (!h || !src) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle or src");
  cudaSetDevice(h->device);
  const size_t tsize = h->precision == IFDLBM_FP64 ? sizeof(double) : sizeof(float);
  const size_t gb = 9 * h->total_plane * tsize;
  const size_t lb = h->total_plane * tsize;
  cudaError_t e = cudaMemcpyAsync(h->b.g[h->cur], src, gb, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->b.lam[h->cur], (const char *)src + gb, lb, cudaMemcpyDeviceToDevice,
                        h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->b.pref, (const char *)src + gb + lb, h->ncav * sizeof(double),
                        cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "load_state_dev");
  return IFDLBM_OK;
}

int ifdlbm_info(ifdlbm_handle h, int cavity, ifdlbm_info_t *info) {
  if (!cavity_ok(h, cavity) || !info) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad arguments");
  const CavDev &cv = h->cav[cavity];
  info->nx = cv.nx;
  info->ny = cv.ny;
  info->precision = h->precision;
  info->kernel = h->kernel;
  info->dt = cv.dt;
  info->K = cv.K;
  info->gamma_min = cv.gmin;
  info->eta_b = cv.eta_b;
  info->courant_max = h->courant[cavity];
  info->steps = h->steps;
  info->device_bytes = h->bytes;
  info->h2d_bytes = h->h2d_bytes;
  info->fused_threads = h->kernel == IFDLBM_KERNEL_FUSED ? h->fused_nt : 0;
  info->fused_rows = h->fused_rows;
  info->schedule = h->schedule;
  info->ntasks = h->ntasks;
  return IFDLBM_OK;
}

int ifdlbm_sync(ifdlbm_handle h) {
  if (!h) return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "handle is NULL");
  cudaSetDevice(h->device);
  return check_status(h);
}

int ifdlbm_destroy(ifdlbm_handle h) {
  if (!h) return IFDLBM_OK;
  cudaSetDevice(h->device);
  release_all(h);
  delete h;
  return IFDLBM_OK;
}

const char *ifdlbm_last_error(ifdlbm_handle h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

int64_t ifdlbm_launch_count(void) { return g_launches.load(); }

namespace {

int adjoint_ready(ifdlbm_ctx *h) {
  if (h->precision != IFDLBM_FP64 || h->kernel != IFDLBM_KERNEL_STAGED)
    return fail(h, IFDLBM_ERR_INVALID_ARG, "adjoint: needs a FP64 handle with the staged kernels");
  if (h->opt.lambda_mode != IFDLBM_LAMBDA_LAGGED)
    return fail(h, IFDLBM_ERR_INVALID_ARG, "adjoint: differentiates the lagged relaxation time");
  if (!h->quad.empty())
    return fail(h, IFDLBM_ERR_INVALID_ARG, "adjoint: differentiates the trapezoid map of Eq. (3.8.1)");
  if (h->opt.wall_pressure != IFDLBM_WALLP_ZEROTH)
    return fail(h, IFDLBM_ERR_INVALID_ARG, "adjoint: differentiates the zeroth-order wall pressure");
  if (h->adj_g1) return IFDLBM_OK;
  const size_t P = size_t(h->total_plane) * sizeof(double);
  bool ok = true;
  ok &= (h->adj_g1 = (double *)dalloc(h, 9 * P)) != nullptr;
  ok &= (h->adj_l1 = (double *)dalloc(h, P)) != nullptr;
  ok &= (h->adj_fhb = (double *)dalloc(h, 9 * P)) != nullptr;
  ok &= (h->adj_fbarb = (double *)dalloc(h, 9 * P)) != nullptr;
  ok &= (h->adj_fbb = (double *)dalloc(h, 9 * P)) != nullptr;
  ok &= (h->adj_lamb2 = (double *)dalloc(h, P)) != nullptr;
  ok &= (h->adj_ppart = (double *)dalloc(h, size_t(h->ntiles) * 12 * sizeof(double))) != nullptr;
  ok &= (h->adj_nodes = (int *)dalloc(h, size_t(h->ncav) * 2 * sizeof(int))) != nullptr;
  if (!ok) return fail(h, IFDLBM_ERR_OOM, "adjoint: device allocation failed");
  for (double *p : {h->adj_fhb, h->adj_fbarb, h->adj_fbb})
    cudaMemsetAsync(p, 0, 9 * P, h->stream);
  cudaMemsetAsync(h->adj_lamb2, 0, P, h->stream);
  return IFDLBM_OK;
}

ifd::AdjArgs adj_args(ifdlbm_ctx *h, const void *state, void *adj) {
  ifd::AdjArgs a{};
  const int64_t n9 = 9 * h->total_plane;
  a.cav = h->b.cav;
  a.geo = h->b.geo;
  a.tile_cav = h->b.tile_cav;
  a.g = (const double *)state;
  a.lam_p = (const double *)state + n9;
  a.lam = h->adj_l1;
  a.fb = (const double *)h->b.fb;
  a.fp = (const double *)h->b.fp;
  a.fh = (const double *)h->b.fh;
  a.gn = h->adj_g1;
  a.adj_g = (double *)adj;
  a.adj_lam = (double *)adj + n9;
  a.fhb = h->adj_fhb;
  a.fbarb = h->adj_fbarb;
  a.fbb = h->adj_fbb;
  a.lamb2 = h->adj_lamb2;
  a.ppart = h->adj_ppart;
  return a;
}

}  // namespace

int ifdlbm_adjoint_seed_energy(ifdlbm_handle h, const void *state, void *adj, double *dparams) {
  if (!h || !state || !adj || !dparams) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad arguments");
  cudaSetDevice(h->device);
  int rc = adjoint_ready(h);
  if (rc) return rc;
  ifd::launch_adjoint_seed(adj_args(h, state, adj), h->ntiles, h->ncav, dparams, h->stream);
  g_launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint seed");
  return IFDLBM_OK;
}

int ifdlbm_adjoint_seed_psi(ifdlbm_handle h, const void *state, const int *nodes, void *adj,
                            double *dparams) {
  if (!h || !state || !nodes || !adj || !dparams)
    return fail(h, IFDLBM_ERR_INVALID_ARG, "bad arguments");
  for (int k = 0; k < h->ncav; ++k) {
    const ifdlbm_cavity &c = h->spec[k];
    if (nodes[2 * k] < 0 || nodes[2 * k] >= c.nx || nodes[2 * k + 1] < 0 || nodes[2 * k + 1] >= c.ny)
      return fail(h, IFDLBM_ERR_INVALID_ARG, "adjoint_seed_psi: node outside its cavity");
  }
  cudaSetDevice(h->device);
  int rc = adjoint_ready(h);
  if (rc) return rc;
  // pageable source: the copy is staged before the call returns
  cudaError_t e = cudaMemcpyAsync(h->adj_nodes, nodes, size_t(h->ncav) * 2 * sizeof(int),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint_seed_psi nodes");
  ifd::AdjArgs a = adj_args(h, state, adj);
  a.psi_nodes = h->adj_nodes;
  ifd::launch_adjoint_seed_psi(a, h->ntiles, h->ncav, dparams, h->stream);
  g_launches += 2;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint seed psi");
  return IFDLBM_OK;
}

int ifdlbm_adjoint_step(ifdlbm_handle h, const void *state_n, void *adj, double *dparams) {
  if (!h || !state_n || !adj || !dparams) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad arguments");
  cudaSetDevice(h->device);
  int rc = adjoint_ready(h);
  if (rc) return rc;
  // forward intermediates of step n from state n (staged kernels)
  ifd::StepArgs f{};
  f.cav = h->b.cav;
  f.geo = h->b.geo;
  f.tile_cav = h->b.tile_cav;
  f.g_in = state_n;
  f.lam_in = (const double *)state_n + 9 * h->total_plane;
  f.g_out = h->adj_g1;
  f.lam_out = h->adj_l1;
  f.fb = h->b.fb;
  f.fp = h->b.fp;
  f.fh = h->b.fh;
  f.m0 = h->b.m0;
  f.part = h->b.part;
  f.status = h->b.status;
  f.powtab = h->b.powtab;
  f.pref = h->b.pref;
  f.want_residual = 0;
  ifd::launch_collide<double>(f, h->ntiles, h->stream);
  ifd::launch_half<double>(f, h->ntiles, h->stream);
  ifd::launch_full<double>(f, h->ntiles, h->stream);
  ifd::launch_adjoint_step(adj_args(h, state_n, adj), h->ntiles, h->ncav, dparams, h->stream);
  g_launches += 3 + 9;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint step");
  return IFDLBM_OK;
}

int64_t ifdlbm_intermediate_bytes(ifdlbm_handle h) {
  if (!h) return -1;
  const size_t tsize = h->precision == IFDLBM_FP64 ? sizeof(double) : sizeof(float);
  return int64_t(27 * h->total_plane * tsize);
}

int ifdlbm_save_intermediates_dev(ifdlbm_handle h, void *dst) {
  if (!h || !dst) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad handle or dst");
  cudaSetDevice(h->device);
  int rc = adjoint_ready(h);
  if (rc) return rc;
  // the staged kernels' scratch planes hold the last step's f-bar^+, f-hat^+
  // and f(t + dt/2), in the order the adjoint reads them
  const size_t P9 = 9 * size_t(h->total_plane) * sizeof(double);
  cudaError_t e = cudaSuccess;
  const void *src[3] = {h->b.fb, h->b.fp, h->b.fh};
  for (int k = 0; k < 3 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync((char *)dst + k * P9, src[k], P9, cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "save_intermediates_dev");
  return IFDLBM_OK;
}

int ifdlbm_adjoint_step_saved(ifdlbm_handle h, const void *state_n, const void *state_np1,
                              const void *inter, void *adj, double *dparams) {
  if (!h || !state_n || !state_np1 || !inter || !adj || !dparams)
    return fail(h, IFDLBM_ERR_INVALID_ARG, "bad arguments");
  cudaSetDevice(h->device);
  int rc = adjoint_ready(h);
  if (rc) return rc;
  // step n's outputs (state n + 1: its populations and lambda(t), which the
  // step stores as the next step's lagged value) and intermediates, as saved
  const int64_t n9 = 9 * h->total_plane;
  ifd::AdjArgs a = adj_args(h, state_n, adj);
  a.gn = (const double *)state_np1;
  a.lam = (const double *)state_np1 + n9;
  a.fb = (const double *)inter;
  a.fp = (const double *)inter + n9;
  a.fh = (const double *)inter + 2 * n9;
  ifd::launch_adjoint_step(a, h->ntiles, h->ncav, dparams, h->stream);
  g_launches += 9;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint step (saved)");
  return IFDLBM_OK;
}

int ifdlbm_autotune(ifdlbm_handle h, int trial_steps, ifdlbm_tuning *best) {
  if (!h || !best || trial_steps < 1) return fail(h, IFDLBM_ERR_INVALID_ARG, "bad arguments");
  if (h->kernel != IFDLBM_KERNEL_FUSED)
    return fail(h, IFDLBM_ERR_INVALID_ARG, "autotune: needs a handle using the fused kernel");
  cudaSetDevice(h->device);
  const int64_t nbytes = ifdlbm_state_bytes(h);
  void *saved = dalloc(h, size_t(nbytes));
  if (!saved) return fail(h, IFDLBM_ERR_OOM, "autotune: device allocation failed");
  int rc = ifdlbm_save_state_dev(h, saved);
  if (rc) return rc;
  const bool profiling = h->profiling;
  h->profiling = false;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ifdlbm_tuning b{};
  b.ms_per_step = 1e300;
  const int nts[3] = {64, 128, 256};
  const int rows[5] = {16, 32, 64, 128, 256};
  for (int nt : nts) {
    for (int r : rows)
      for (int sc = IFDLBM_SCHED_GRID; sc <= IFDLBM_SCHED_DYNAMIC; ++sc) {
        if ((rc = build_fused_tasks(h, nt, r, sc))) goto done;
        if ((rc = ifdlbm_load_state_dev(h, saved))) goto done;
        for (int w = 0; w < 2; ++w) enqueue_step_any(h, h->cur ^ (w & 1), false);
        cudaEventRecord(e0, h->stream);
        for (int st = 0; st < trial_steps; ++st) enqueue_step_any(h, h->cur ^ (st & 1), false);
        cudaEventRecord(e1, h->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
          rc = cuda_fail(h, e, "autotune trial");
          goto done;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        g_launches += int64_t(trial_steps + 2) * launches_per_step(h, false);
        ++b.candidates;
        if (ms / trial_steps < b.ms_per_step) {
          b.ms_per_step = ms / trial_steps;
          b.fused_threads = nt;
          b.fused_rows = r;
          b.schedule = sc;
        }
      }
  }
  rc = build_fused_tasks(h, b.fused_threads, b.fused_rows, b.schedule);
  if (!rc) rc = ifdlbm_load_state_dev(h, saved);
  if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = fail(h, IFDLBM_ERR_CUDA, "autotune");
  b.ntasks = h->ntasks;
  *best = b;
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->profiling = profiling;
  return rc;
}

int ifdlbm_selftest_pow(ifdlbm_handle h, int n, const double *x, double m, double *fast,
                        double *ref) {
  if (!h || n < 0 || (n > 0 && (!x || !fast || !ref)))
    return fail(h, IFDLBM_ERR_INVALID_ARG, "selftest_pow: bad arguments");
  if (n == 0) return IFDLBM_OK;
  cudaSetDevice(h->device);
  ifd::launch_pow_selftest(n, x, m, h->b.powtab, fast, ref, h->stream);
  g_launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "selftest_pow");
  return IFDLBM_OK;
}

int ifdlbm_inject_tma_timeout(ifdlbm_handle h, int enable) {
  if (!h) return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "handle is NULL");
  if (h->kernel != IFDLBM_KERNEL_FUSED)
    return fail(h, IFDLBM_ERR_INVALID_ARG, "inject_tma_timeout: the handle runs the staged kernels");
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  for (int p = 0; p < 2; ++p)  // captured graphs hold the launch arguments
    if (h->gexec[p]) {
      cudaGraphExecDestroy(h->gexec[p]);
      h->gexec[p] = nullptr;
    }
  h->tma_skip = enable ? 1 : 0;
  return IFDLBM_OK;
}

int ifdlbm_selftest_pow_tab(ifdlbm_handle h, int cavity, int n, const double *x, double *out) {
  if (!cavity_ok(h, cavity) || n < 0 || (n > 0 && (!x || !out)))
    return fail(h, IFDLBM_ERR_INVALID_ARG, "selftest_pow_tab: bad arguments");
  if (n == 0) return IFDLBM_OK;
  cudaSetDevice(h->device);
  const CavDev &cv = h->cav[cavity];
  ifd::launch_pow_tab_selftest(n, x, cv.half_nm1, cv.Kics2,
                               h->b.powt + size_t(cavity) * ifd::POWT_SIZE, cv.pb2, cv.pb3,
                               cv.pb4, cv.pb5, out, h->stream);
  g_launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "selftest_pow_tab");
  return IFDLBM_OK;
}

int ifdlbm_selftest_pow_f32(ifdlbm_handle h, int n, const double *x, double m, double *out) {
  if (!h || n < 0 || (n > 0 && (!x || !out)))
    return fail(h, IFDLBM_ERR_INVALID_ARG, "selftest_pow_f32: bad arguments");
  if (n == 0) return IFDLBM_OK;
  cudaSetDevice(h->device);
  ifd::launch_pow_f32_selftest(n, x, m, out, h->stream);
  g_launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "selftest_pow_f32");
  return IFDLBM_OK;
}

int ifdlbm_profile(ifdlbm_handle h, int enable) {
  if (!h) return fail(nullptr, IFDLBM_ERR_INVALID_ARG, "handle is NULL");
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  h->profiling = enable != 0;
  h->ev_used = 0;
  h->ev_marks.clear();
  return IFDLBM_OK;
}

int ifdlbm_profile_read(ifdlbm_handle h, int kernel, double *total_ms, int64_t *launches) {
  if (!h || kernel < 0 || kernel >= IFDLBM_KPROF_COUNT || !total_ms || !launches)
    return fail(h, IFDLBM_ERR_INVALID_ARG, "bad arguments");
  cudaSetDevice(h->device);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "profile sync");
  double tot = 0;
  int64_t n = 0;
  for (auto &m : h->ev_marks)
    if (m.first == kernel) {
      float ms = 0;
      e = cudaEventElapsedTime(&ms, h->ev_pool[m.second.first], h->ev_pool[m.second.second]);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventElapsedTime");
      tot += ms;
      ++n;
    }
  *total_ms = tot;
  *launches = n;
  return IFDLBM_OK;
}

}  // extern "C"
