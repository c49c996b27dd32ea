// Internal structures shared by the host API (capi.cu) and the kernels.
// Not part of the public ABI (include/ifdlbm.h).
#pragma once
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

namespace ifd {

// Per-cavity constants, resident in device global memory (one entry per
// cavity of a handle). Offsets are in elements of the arena they index.
struct CavDev {
  int nx, ny, pitch;        // nodes along xi / eta; row pitch in elements
  int tile0, tiles_x, tiles_y;  // staged-kernel tiles of this cavity
  int64_t plane;            // ny * pitch
  int64_t off;              // start of plane 0 of this cavity (per-plane units)
  int64_t goff;             // start of this cavity's 1-D metric arrays
  int part0;                // first residual-partial slot of this cavity
  int nparts;               // number of partial slots
  double dt, K, nm1, gmin;  // time step, consistency coeff., n - 1, shear clamp
  double eta_b;             // blend of Eq. (2.5)
  double c, cs2, inv_cs2;   // lattice speed, c_s^2, 1/c_s^2
  double dxi, deta;         // computational grid spacings
  double inv2dxi, inv2deta; // 1/(2 dxi), 1/(2 deta)
  double U, H, rho0;        // lid speed, height, reference density
  double lam0;              // Eq. (2.14) at zero shear (initial lambda_prev)
  double gmin2;             // gamma_min^2
  double half_nm1;          // (n - 1) / 2: mu = K max(q, gamma_min^2)^((n-1)/2), q = gamma-dot^2
  double Kics2;             // K / c_s^2
  double dcot;              // d cot(theta) / d theta_deg (adjoint)
  double lnHU;              // ln H - ln U: d ln K / d n (adjoint)
  double Re;                // Reynolds number (adjoint)
  int implicit;             // 1: lambda from the implicit form of Eq. (2.14), 0: lagged
  int general;              // 1: general quadrilateral, per-node metrics in Geo::gmet
  int pow32;                // FP32 storage only: 1 power law (and implicit solve) in FP32
  int wallp;                // wall rule's pressure: 0 zeroth-order, 1 first-order (staged)
  double lid_ux, lid_uy;    // lid velocity (U, 0) on the trapezoid, U along the top edge in general
  // pow_tab (FP32 argument, FP64 result) of Eq. (1.4): binomial coefficients
  // b2 = m (m-1)/2 and, as floats, b3..b5 of (1 + t)^m with m = half_nm1; and
  // the clamp of the FP32 strain rate, max(largest float <= gamma_min^2, FLT_MIN)
  double pb2;
  float pb3, pb4, pb5, gmin2_f;
};

// 1-D metric arrays of the trapezoid map (Eq. 3.8.2), per cavity at goff:
//   xix[j]  = xi_x(eta_j) = 1 / x_xi(eta_j)             (ny entries)
//   xeH[i]  = x_eta(xi_i) / H                           (nx entries)
//   xxi[j]  = x_xi(eta_j)    (Jacobian J = x_xi * H)    (ny entries)
//   xeta[i] = x_eta(xi_i)    (stream function)          (nx entries)
//   cxix_f[j] = float(c xi_x(eta_j)), jac_f[j] = float(x_xi(eta_j) H): rounded
//   copies used only where the arithmetic is FP32 (fused FP32 kernel)
struct Geo {
  const double *xix, *xeH, *xxi, *xeta;
  const float *cxix_f, *jac_f;
  // general quadrilaterals (staged kernels): per node, at 7 * off + k * plane,
  // k = 0..6: xi_x, xi_y, eta_x, eta_y, x_eta, y_eta, J (Eqs. 3.2-3.3)
  const double *gmet;
  // general quadrilaterals (fused FP32 kernel): per node, at 5 * off + k * plane,
  // k = 0..4: c xi_x, c xi_y, c eta_x, c eta_y, J, each the FP32 rounding of
  // the FP64 value of gmet (the metrics are formed in FP64; only the FP32
  // arithmetic that uses them sees them rounded)
  const float *qmet_f;
};

// Device buffers of a handle. T is double (FP64) or float (FP32DEV).
struct Bufs {
  void *g[2];        // 9 planes per cavity: f-hat deviation g_i, ping-pong
  void *lam[2];      // 1 plane per cavity: relaxation time (storage type T), ping-pong
  void *fb;          // 9 planes: f-bar^+ (staged kernels)
  void *fp;          // 9 planes: f-hat^+ (staged kernels)
  void *fh;          // 9 planes: f(t + dt/2) (staged kernels)
  double *m0;        // 3 planes: u, v, P at the start of the step
  double *part;      // residual partials [nparts_total][8]
  double *resid;     // [ncav][4] residual outputs
  int *tile_cav;     // staged tile -> cavity
  unsigned *status;  // bit 0: non-finite velocity seen
  CavDev *cav;       // [ncav]
  Geo geo;
  double *powtab;    // tables of pow_fast (fastpow.cuh)
  double *powt;      // [ncav][POWT_SIZE] per-cavity tables of pow_tab (fastpow.cuh)
  double *pref;      // [ncav] reference pressure: f-hat = w rho0 + wbar pref / c_s^2 + g
  int *cav_done;     // [ncav] fused kernel: tasks finished in the current step
  double *ptile;     // [ntiles + ncav] scratch of the re-basing reduction
};

struct StepArgs {
  const CavDev *cav;
  Geo geo;
  const int *tile_cav;
  const void *g_in;
  void *g_out;
  const void *lam_in;  // relaxation-time planes in the storage type T
  void *lam_out;
  void *fb, *fp, *fh;
  double *m0;
  double *part;
  unsigned *status;
  const double *powtab;
  const double *powt;  // [ncav][POWT_SIZE] tables of pow_tab
  const double *pref;  // [ncav] reference pressure of the stored deviations
  int want_residual;
};

// One CTA task of the fused kernel: owned columns [i0, i1) (at most NT - 8)
// and rows [j0, j1) of cavity `cav`.
struct Task {
  int cav, i0, i1, j0, j1, pad0, pad1, pad2;
};

// Bytes of one TMA tensor map (CUtensorMap) in device memory (64-byte aligned).
constexpr int TMAP_BYTES = 128;

struct FusedArgs {
  const CavDev *cav;
  Geo geo;
  const Task *tasks;
  const int *order;   // scheduled position -> task index (largest tasks first)
  int *counter;       // dynamic schedule: next position (zeroed before each launch)
  int ntasks;
  int schedule;       // 0 grid (one CTA per task), 1 persistent static, 2 persistent dynamic
  const void *g_in;
  void *g_out;
  const void *tmap_in;  // [ncav] tensor maps of g_in (TMAP_BYTES each): box 32 x 1 x 9
  const void *lam_in;  // relaxation-time planes in the storage type T
  void *lam_out;
  double *part;
  unsigned *status;
  const double *powtab;
  const double *powt;  // [ncav][POWT_SIZE] tables of pow_tab
  const double *pref;  // [ncav] reference pressure of the stored deviations
  int *cav_done;       // [ncav] tasks of the step finished (zero between steps)
  int implicit;        // 1: implicit form of Eq. (2.14) (kernel variant), 0: lagged
  int general;         // 1: general quadrilaterals (kernel variant; FP32, lagged)
  int pow32;           // 1: FP32 power law (opt-in of the FP32 form; kernel variant)
  int tma_skip;        // test hook: 1 issues no TMA row loads, so that every row wait runs out
  double *resid;       // [ncav][4] residual outputs (formed by each cavity's last task)
  int want_residual;
};

// Fused kernel (fused.cu); nt in {64, 128, 256} threads, two per column: a
// CTA's strip holds nt/2 - 8 output columns plus a 4-column halo on each side.
constexpr int fused_strip_width(int nt) { return nt / 2 - 8; }
template <class T> bool launch_fused(const FusedArgs &a, int nt, int ntasks, cudaStream_t s);
template <class T> int fused_smem_bytes(int nt);
template <class T> int fused_blocks_per_sm(int nt);

// Staged kernels (staged.cu)
template <class T> void launch_collide(const StepArgs &a, int ntiles, cudaStream_t s);
template <class T> void launch_half(const StepArgs &a, int ntiles, cudaStream_t s);
template <class T> void launch_full(const StepArgs &a, int ntiles, cudaStream_t s);
void launch_residual_reduce(const CavDev *cav, const double *part, double *resid, int ncav,
                            cudaStream_t s);

// Discrete adjoint of one staged FP64 step (adjoint.cu). Buffers use the
// state layout: 9 planes then 1 plane per cavity at the usual offsets.
struct AdjArgs {
  const CavDev *cav;
  Geo geo;
  const int *tile_cav;
  const double *g, *lam_p;   // state n
  const double *lam;         // lambda(t) of step n (forward output)
  const double *fb, *fp, *fh;  // forward intermediates of step n
  const double *gn;          // state n + 1 (forward output)
  double *adj_g, *adj_lam;   // in: adjoint of state n + 1; out: of state n
  double *fhb, *fbarb, *fbb, *lamb2;  // adjoint scratch
  double *ppart;             // [ntiles][4 slots][3] parameter partials
  const int *psi_nodes;      // [ncav][2] (i, j) of the psi objective (seed_psi only)
};
void launch_adjoint_seed(const AdjArgs &a, int ntiles, int ncav, double *dparams, cudaStream_t s);
void launch_adjoint_seed_psi(const AdjArgs &a, int ntiles, int ncav, double *dparams,
                             cudaStream_t s);
void launch_adjoint_step(const AdjArgs &a, int ntiles, int ncav, double *dparams, cudaStream_t s);

// Host-built tables of pow_fast and of pow_tab (capi.cu) and their self-tests (staged.cu)
void fill_pow_tables(double *tab);
void fill_cavity_pow_table(double *tab, double m, double C);
void launch_pow_tab_selftest(int n, const double *x, double m, double C, const double *tab,
                             double b2, float b3, float b4, float b5, double *out, cudaStream_t s);
void launch_pow_f32_selftest(int n, const double *x, double m, double *out, cudaStream_t s);

// Metrics of the bilinear map of a general quadrilateral at (xi, eta),
// Eqs. (3.2)-(3.3), from its corners cr = {x0, y0, x1, y1, x2, y2, x3, y3}
// (bottom-left, bottom-right, top-left, top-right):
// m = xi_x, xi_y, eta_x, eta_y, x_eta, y_eta, J.
__host__ __device__ inline void quad_node_metrics(const double *cr, double xi, double eta,
                                                  double m[7]) {
  const double x_xi = (1 - eta) * (cr[2] - cr[0]) + eta * (cr[6] - cr[4]);
  const double y_xi = (1 - eta) * (cr[3] - cr[1]) + eta * (cr[7] - cr[5]);
  const double x_eta = (1 - xi) * (cr[4] - cr[0]) + xi * (cr[6] - cr[2]);
  const double y_eta = (1 - xi) * (cr[5] - cr[1]) + xi * (cr[7] - cr[3]);
  const double J = x_xi * y_eta - x_eta * y_xi;
  m[0] = y_eta / J;
  m[1] = -x_eta / J;
  m[2] = -y_xi / J;
  m[3] = x_xi / J;
  m[4] = x_eta;
  m[5] = y_eta;
  m[6] = J;
}
// Per-node metric planes (Geo::gmet) of every cavity of a quadrilateral
// handle, from corners [ncav][8]; max_n2 = the largest nx * ny.
void launch_quad_metrics(const CavDev *cav, int ncav, int64_t max_n2, const double *corners,
                         double *gmet, cudaStream_t s);
// The float planes Geo::qmet_f of the fused FP32 kernel, from the FP64 planes gmet.
void launch_quad_metrics_f32(const CavDev *cav, int ncav, int64_t max_n2, const double *gmet,
                             float *qmet_f, cudaStream_t s);
void launch_pow_selftest(int n, const double *x, double m, const double *tab, double *fast,
                         double *ref, cudaStream_t s);

// Utility kernels (staged.cu)
template <class T> void launch_init(const CavDev *cav, const int *tile_cav, void *g, void *lam,
                                    int ntiles, cudaStream_t s);
template <class T> void launch_macros(const CavDev *cav, Geo geo, int cavity, const double *pref,
                                      const void *g,
                                      double *rho, double *u, double *v, double *psi,
                                      int nx, int ny, cudaStream_t s);
template <class T> void launch_export(const CavDev *cav, int cavity, const double *pref,
                                      const void *g,
                                      const void *lam, double *fhat, double *lamo, int nx,
                                      int ny, cudaStream_t s);
template <class T> void launch_import(const CavDev *cav, int cavity, const double *pref,
                                      void *g, void *lam,
                                      const double *fhat, const double *lami, int nx, int ny,
                                      cudaStream_t s);
// u, v, P at probe nodes [n][3] = (cavity, i, j) into out [n][3] (NaN for a
// probe outside its cavity).
template <class T> void launch_probe(const CavDev *cav, int ncav, const double *pref, const void *g,
                                     int n, const int *probes, double *out, cudaStream_t s);
// Re-bases the stored deviations of every cavity on its mean pressure:
// shift = mean over the cavity's nodes of P(g), g_i -= wbar_i shift / c_s^2,
// pref += shift (the state f-hat = w rho0 + wbar pref / c_s^2 + g is
// unchanged). ptile: scratch of ntiles + ncav doubles.
template <class T> void launch_rebase(const CavDev *cav, const int *tile_cav, void *g,
                                      double *pref, double *ptile, int ntiles, int ncav,
                                      cudaStream_t s);

// Records `msg` as the handle-less last error (ifdlbm_last_error(NULL)) and
// returns `code`; counts kernel launches for ifdlbm_launch_count (capi.cu).
int set_global_error(int code, const std::string &msg);
void count_launches(int64_t n);

constexpr int TILE_X = 32;
constexpr int TILE_Y = 8;
constexpr int NPART = 8;  // doubles per residual partial slot

}  // namespace ifd
