// Fused IFDLBM step: Steps (2)-(6) and the residual partials in one launch.
//
// A CTA of NT threads owns a strip [i0, i1) of at most W = NT/2 - 8 columns
// of one cavity and a segment [j0, j1) of rows. Two threads share each of its
// NT/2 columns (the strip plus 4 recomputed halo columns on each side): half
// h = 0 takes the even rows of the march, half h = 1 the odd ones. Iteration
// k (k = j0 - 4, j0 - 2, ...) runs, in half h,
//
//   stage A  row k + h     moments, f^eq, lagged power-law lambda (FP64 power),
//                          f-hat^+ (Eq. 2.15), f-bar^+ (Eq. 2.16)
//   stage 1  row k - 2 + h half step f-bar(t+dt/2) (Eq. 3.7), its moments,
//                          f(t+dt/2) (Eq. 2.17); wall values by extrapolation
//   stage 2  row k - 4 + h full step f-hat(t+dt) (Eq. 3.6); wall values by
//                          extrapolation (Step 6); residual partials
//
// so that each node's state is read from and written to HBM once per step.
// Shared memory per column pair: six-row rings of f-bar^+ and f(t+dt/2)
// (slot = row mod 6), read across columns (xi stencils) and across the two
// halves (eta stencils); and, per thread, five slots that hold the state of a
// row from its prefetch (two iterations ahead) until stage A, and then, in
// place, its f-hat^+ until the full step two iterations later. The prefetch is
// one TMA copy per warp (tma.cuh): a 3-D tiled bulk copy of the warp's 32
// columns x 9 planes of the row into the warp's slot, completed on that slot's
// mbarrier, so that no thread issues per-population loads. That is ~430 B per
// thread in FP32, so that 16 warps fit on an SM. Three barriers per iteration
// order the stages across the halves.
//
// Wall nodes follow the rule of the staged kernels: a side-wall node takes
// its inner neighbour on the same row, a bottom/lid node the node
// (clamp(i, 1, nx-2), 1 or ny-2). The wall nodes of f(t+dt/2) are written
// by the thread that forms their neighbour in the half step (row 0 with row
// 1, the side walls with columns 1 and nx-2, the lid row ny-1, which has a
// buffer of its own, with row ny-2). The full-step values of columns 1 and
// nx-2, which the wall columns of f-hat(t+dt) extrapolate from, are published
// through a small shared array. In FP32 the first-order near-wall
// differences of the stencils come from ghost values beyond the walls
// (write_ghosts), written by the node that reads them, instead of per-plane
// selects on the wall flags.
//
// FP64 work per node is kept to the power of Eq. (1.4) and the residual
// accumulation: GB300 issues FP64 at 1/64 of the FP32 rate. With the pow32
// opt-in of the FP32 form the power is FP32 too (pow_f32), and the FP64 work
// is the conversion of lambda, whose plane is FP64, and the residual.
#include <cstdint>

#include "d2q9.cuh"
#include "internal.h"
#include "reduce.cuh"
#include "tma.cuh"

namespace ifd {

namespace {

constexpr int PF = 5;     // per-thread row slots: prefetched state, then f-hat^+
constexpr int LEAF = 16;  // rows per leaf sum of the residual terms
constexpr int RING = 6;   // rows of the f-bar^+ and f(t+dt/2) rings

template <class T, int NT>
struct FusedSmem {
  static constexpr int NC = NT / 2, NW = NT / 32;
  // per warp and slot, the TMA box of its 32 columns x 9 planes: g(t) of the
  // warp's row, then f-hat^+ in place (each box a multiple of 128 bytes)
  T sf[PF][NW][9][32];
  T fb[RING][9][NC];      // f-bar^+
  T fh[RING][9][NC];      // f(t + dt/2)
  T edge[2][3][NC];       // u, v, P(t) of rows 0 and ny-1 (wall-row residuals)
  T gw[2][2][9];          // f-hat(t+dt) of columns 1 and nx-2, per half
  T lid[9][NC];           // f(t + dt/2) of the lid row ny-1 (written with row ny-2, which
                          // can come one iteration before the ring slot of row ny-1 is free)
  uint64_t bar[PF][NW];   // mbarriers of the TMA row loads
};
// dynamic shared memory: the struct plus the slack of aligning it to 128 bytes
template <class T, int NT>
constexpr int fused_smem_size() {
  return int(sizeof(FusedSmem<T, NT>)) + 128;
}

// Ring slot of row r (r >= -12) and prefetch slot of iteration it (it >= 0):
// unsigned remainders by constants, a multiply-high and a shift each.
__device__ __forceinline__ int slot6(int r) { return int(unsigned(r + 12) % unsigned(RING)); }
__device__ __forceinline__ int pf_slot(int it) { return int(unsigned(it) % unsigned(PF)); }

// a / b for the relaxation weights and the strain-rate factor, whose
// denominators (2 lam + dt, 4 lam + dt, (2 lam + dt) c_s^2) are positive and
// normal: with FAST in FP32 the hardware reciprocal approximation
// (__fdividef, within 2 ulp), else a division. The transforms of
// Eqs. (2.15)-(2.17) move F towards f^eq, so an error in their weights leaves
// u and P unchanged and reaches the populations at 2e-7 of |f^eq - F|.
template <bool FAST, class T>
__device__ __forceinline__ T quot(T a, T b) {
  if constexpr (FAST && sizeof(T) == 4)
    return __fdividef(a, b);
  else
    return a / b;
}

// Mixed difference of Eqs. (2.5)-(2.7) times 2 d with the upwind side chosen
// at run time (general quadrilaterals): the upwind operands are selected,
// then one stencil is evaluated; `edge_pos` / `edge_neg` select the
// first-order near-wall form on either side.
template <class T>
__device__ __forceinline__ T dmix2_sel(T fm2, T fm1, T f0, T fp1, T fp2, bool pos, bool edge_pos,
                                       bool edge_neg, T eta_b) {
  const T fa = pos ? fm1 : fp1, fb = pos ? fm2 : fp2;
  const bool edge = pos ? edge_pos : edge_neg;
  const T u = edge ? T(2) * (f0 - fa) : (T(3) * f0 - T(4) * fa + fb);
  return eta_b * (fp1 - fm1) + (T(1) - eta_b) * (pos ? u : -u);
}

// The mixed difference of Eqs. (2.5)-(2.7) times 2 d, for the side "from
// below" (c >= 0) with a = F[k+1], b = F[k-1], cf = F[k-2], and for the side
// from above with a = F[k-1], b = F[k+1], cf = F[k+2], is
//   sigma [eta_b (a - b) + (1 - eta_b) (3 (F[k] - b) + (cf - b))],
// sigma = +1 and -1: both branches of Eq. (2.7) in one expression of the
// selected operands. Next to a wall the far upwind node cf is replaced by the
// linear extrapolation 2 b - F[k], which is the first-order near-wall
// difference (then cf - b = -(F[k] - b)). Differences are formed before they
// are scaled, so that a constant field gives exactly zero in any precision.
template <class T>
__device__ __forceinline__ T mixed_sum(T a, T b, T cf, T f0, bool edge, T kb, T ku3, T ku) {
  const T d2 = f0 - b;
  const T d3 = edge ? -d2 : cf - b;
  return kb * (a - b) + (ku3 * d2 + ku * d3);
}

// base_q - scale (c_{q xi} D_xi F + c_{q eta} D_eta F) at an interior node of
// the trapezoid (Eq. 3.7 with scale = dt/2, Eq. 3.6 with scale = dt):
// `row` is the xi row of plane q at this thread's lane l, `col` the five eta
// neighbours. xs = scale c_{q xi} / (2 dxi) = e_x As - e_y Bs, whose sign is
// the upwind side along xi (it absorbs sigma: xs D = |xs| sum); along eta the
// side is the sign of e_y (c_{q eta} = c e_y / H) and the factor is
// Es = scale (c / H) / (2 deta). As = scale c xi_x / (2 dxi) is positive, so
// the planes with e_y = 0 have the side of e_x. With EDGE the near-wall
// first-order form is selected by the flags; without it the far upwind
// neighbour outside the cavity holds the linear extrapolation (a ghost value,
// written by the caller), which gives the same difference.
template <int Q, bool EDGE, class T>
__device__ __forceinline__ T advect_out(T base, const T *row, int l, const T col[5], T As, T Bs,
                                        T Es, bool clo, bool chi, bool lo, bool hi, T kb, T ku3,
                                        T ku) {
  const T xs = T(ex(Q)) * As - T(ey(Q)) * Bs;
  const T f0 = col[2];
  const T fm1 = row[l - 1], fp1 = row[l + 1];
  const bool pos = ey(Q) == 0 ? ex(Q) > 0 : xs >= T(0);
  const T sx = mixed_sum(pos ? fp1 : fm1, pos ? fm1 : fp1, pos ? row[l - 2] : row[l + 2], f0,
                         EDGE && (pos ? clo : chi), kb, ku3, ku);
  T out = base - fabs(xs) * sx;
  if constexpr (ey(Q) > 0)
    out -= Es * mixed_sum(col[3], col[1], col[0], f0, EDGE && lo, kb, ku3, ku);
  else if constexpr (ey(Q) < 0)
    out -= Es * mixed_sum(col[1], col[3], col[4], f0, EDGE && hi, kb, ku3, ku);
  return out;
}

// Writes the ghost values of a near-wall node's stencils (the EDGE = false
// form of advect_out) into its ring (planes RS apart): `row` is the node's
// ring row at lane l, `below` / `above` column l of the ring rows beyond the
// bottom / lid, `wall_lo` / `wall_hi` column l of the wall rows. For a node
// next to a side wall the row neighbour beyond the wall, for a node next to
// the bottom / lid the column neighbour beyond it, each the linear
// extrapolation 2 F[wall] - F[node] of the plane. Each ghost is read by this
// thread's own stencil only (no other node takes it within the radius-2
// stencils), so no barrier orders the write.
template <class T, int RS>
__device__ __forceinline__ void write_ghosts(T *row, int l, bool clo, bool chi, bool lo, bool hi,
                                             T *below, const T *wall_lo, T *above,
                                             const T *wall_hi) {
  if (clo) {
#pragma unroll
    for (int q = 1; q < 9; ++q)
      row[q * RS + l - 2] = T(2) * row[q * RS + l - 1] - row[q * RS + l];
  }
  if (chi) {
#pragma unroll
    for (int q = 1; q < 9; ++q)
      row[q * RS + l + 2] = T(2) * row[q * RS + l + 1] - row[q * RS + l];
  }
  if (lo) {
#pragma unroll
    for (int q = 1; q < 9; ++q)
      if (ey(q) > 0) below[q * RS] = T(2) * wall_lo[q * RS] - row[q * RS + l];
  }
  if (hi) {
#pragma unroll
    for (int q = 1; q < 9; ++q)
      if (ey(q) < 0) above[q * RS] = T(2) * wall_hi[q * RS] - row[q * RS + l];
  }
}

// out[q] for q = Q..8; ring planes are RS apart, base planes BS apart.
template <class T, int Q, int RS, int BS, bool EDGE>
struct AdvectAll {
  __device__ __forceinline__ static void run(const T *rows, const T *const cols[5], int l, T As,
                                             T Bs, T Es, bool clo, bool chi, bool lo, bool hi,
                                             T kb, T ku3, T ku, const T *base, T out[9]) {
    const T col[5] = {cols[0][Q * RS], cols[1][Q * RS], cols[2][Q * RS], cols[3][Q * RS],
                      cols[4][Q * RS]};
    out[Q] = advect_out<Q, EDGE>(base[Q * BS], rows + Q * RS, l, col, As, Bs, Es, clo, chi, lo,
                                 hi, kb, ku3, ku);
    if constexpr (Q < 8)
      AdvectAll<T, Q + 1, RS, BS, EDGE>::run(rows, cols, l, As, Bs, Es, clo, chi, lo, hi, kb, ku3,
                                             ku, base, out);
  }
};

// General quadrilateral (per-node metrics, Eq. 3.4 in full): c_{q xi} =
// e_qx k_xx + e_qy k_xy and c_{q eta} = e_qx k_ex + e_qy k_ey with
// (k_xx, k_xy, k_ex, k_ey) = c (xi_x, xi_y, eta_x, eta_y) of the node; both
// upwind sides are chosen by sign at run time.
template <int Q, class T>
__device__ __forceinline__ T advect_q_gen(const T *row, int l, const T col[5], T kxx, T kxy, T kex,
                                          T key, bool clo, bool chi, bool lo, bool hi, T eta_b,
                                          T i2dxi, T i2deta) {
  const T cxi = T(ex(Q)) * kxx + T(ey(Q)) * kxy;
  const T ceta = T(ex(Q)) * kex + T(ey(Q)) * key;
  const T f0 = col[2];
  T adv = cxi * dmix2_sel(row[l - 2], row[l - 1], f0, row[l + 1], row[l + 2], cxi >= T(0), clo,
                          chi, eta_b) * i2dxi;
  adv += ceta * dmix2_sel(col[0], col[1], f0, col[3], col[4], ceta >= T(0), lo, hi, eta_b) * i2deta;
  return adv;
}

template <class T, int Q, int RS, int BS>
struct AdvectAllGen {
  __device__ __forceinline__ static void run(const T *rows, const T *const cols[5], int l, T kxx,
                                             T kxy, T kex, T key, bool clo, bool chi, bool lo,
                                             bool hi, T eta_b, T i2dxi, T i2deta, T scale,
                                             const T *base, T out[9]) {
    const T col[5] = {cols[0][Q * RS], cols[1][Q * RS], cols[2][Q * RS], cols[3][Q * RS],
                      cols[4][Q * RS]};
    out[Q] = base[Q * BS] - scale * advect_q_gen<Q>(rows + Q * RS, l, col, kxx, kxy, kex, key,
                                                    clo, chi, lo, hi, eta_b, i2dxi, i2deta);
    if constexpr (Q < 8)
      AdvectAllGen<T, Q + 1, RS, BS>::run(rows, cols, l, kxx, kxy, kex, key, clo, chi, lo, hi,
                                          eta_b, i2dxi, i2deta, scale, base, out);
  }
};

// Residual terms of one node, summed over up to LEAF rows in T before they
// are added to the FP64 partials (a leaf sum; every sum beyond it is FP64).
template <class T>
struct Leaf {
  T du2 = 0, u2 = 0, dP2 = 0, P2 = 0, ek = 0;
  T du2max = 0, u2max = 0;  // maxima are exact in any precision
  int n = 0;
};

template <class T>
__device__ __forceinline__ void leaf_flush(Leaf<T> &l, Partial &p) {
  p.du2 += double(l.du2);
  p.u2 += double(l.u2);
  p.dP2 += double(l.dP2);
  p.P2 += double(l.P2);
  p.ek += double(l.ek);
  l.du2 = l.u2 = l.dP2 = l.P2 = l.ek = T(0);
  l.n = 0;
}

// P1, P0 are pressures of the stored deviations; Pr their reference (the
// pressure of Eq. 2.11 is Pr + P), which cancels in the difference.
template <class T>
__device__ __forceinline__ void leaf_add(Leaf<T> &l, Partial &p, T u1, T v1, T P1, T u0, T v0,
                                         T P0, T Pr, T wJ, unsigned *status) {
  if (!(isfinite(u1) && isfinite(v1))) atomicOr(status, 1u);
  const T du = u1 - u0, dv = v1 - v0, dP = P1 - P0;
  const T du2 = du * du + dv * dv, u2 = u1 * u1 + v1 * v1;
  const T Pf = P1 + Pr;
  l.du2 += du2;
  l.u2 += u2;
  l.dP2 += dP * dP;
  l.P2 += Pf * Pf;
  l.ek += T(0.5) * wJ * u2;
  l.du2max = max(l.du2max, du2);
  l.u2max = max(l.u2max, u2);
  if (++l.n == LEAF) leaf_flush(l, p);
}

}  // namespace

template <class T, int NT, bool IMPL, bool GEN, bool P32>
__device__ __forceinline__ void fused_task(const FusedArgs &a, FusedSmem<T, NT> &S, int ti,
                                           unsigned &phase) {
  constexpr int NC = NT / 2;
  constexpr int SLOT = FusedSmem<T, NT>::NW * 9 * 32;  // elements of one slot (all warps)
  const Task task = a.tasks[ti];
  const CavDev &cv = a.cav[task.cav];
  const int i0 = task.i0, i1 = task.i1, j0 = task.j0, j1 = task.j1;
  // Everything the march needs from the cavity descriptor, read once: the
  // descriptor is in global memory, and the march's stores could alias it
  // as far as the compiler knows.
  const int nx = cv.nx, ny = cv.ny, pitch = cv.pitch;
  const int64_t plane = cv.plane, goff = cv.goff;
  const double cvc = cv.c, cvH = cv.H;
  const T Uw = GEN ? T(cv.lid_ux) : T(cv.U);        // lid velocity
  const T Uwy = GEN ? T(cv.lid_uy) : T(0);
  const int part0 = cv.part0, nparts = cv.nparts;
  // c xi_x of row j and the Jacobian x_xi H: FP64 metrics for FP64
  // arithmetic, their rounded float copies for FP32 arithmetic.
  auto row_cxix = [&](int j) -> T {
    if constexpr (sizeof(T) == 8)
      return cvc * a.geo.xix[goff + j];
    else
      return a.geo.cxix_f[goff + j];
  };
  auto row_jac = [&](int j) -> T {
    if constexpr (sizeof(T) == 8)
      return a.geo.xxi[goff + j] * cvH;
    else
      return a.geo.jac_f[goff + j];
  };
  const int t = threadIdx.x;
  const int h = t / NC;                              // row parity of this thread (warp-uniform)
  const int l = t - h * NC;                          // column lane
  const int c = i0 - 4 + l;                          // this thread's column
  const int cc = min(max(c, 0), nx - 1);             // clamped column for loads
  const bool colv = c >= 0 && c < nx;
  const bool own = colv && c >= i0 && c < i1;        // output column (i1 - i0 <= NC - 8)
  const bool inner_c = c >= 1 && c <= nx - 2;
  const bool wall_c = c == 0 || c == nx - 1;
  const bool clo = c == 1, chi = c == nx - 2;

  const int64_t b9 = 9 * cv.off;
  T *gout = (T *)a.g_out + b9;
  const T *lam_in = (const T *)a.lam_in + cv.off;   // relaxation time, storage type T
  T *lam_out = (T *)a.lam_out + cv.off;

  const T c_ = T(cv.c), cs2 = T(cv.cs2), ics2 = T(cv.inv_cs2);
  const T dt = T(cv.dt), hdt = T(0.5 * cv.dt);
  const T eta_b = T(cv.eta_b);
  const T i2dxi = T(cv.inv2dxi), i2deta = T(cv.inv2deta);
  const T ceta_unit = T(cv.c / cv.H);
  // factors of the trapezoid's advection (advect_out): scale / (2 dxi) and
  // scale (c / H) / (2 deta) with scale = dt/2 (half step) and dt (full step);
  // the blend weights of Eq. (2.5)
  const T hxs = T(0.5 * cv.dt * cv.inv2dxi), fxs = T(cv.dt * cv.inv2dxi);
  const T Es1 = T(0.5 * cv.dt * cv.inv2deta * cv.c / cv.H), Es2 = T(cv.dt * cv.inv2deta * cv.c / cv.H);
  const T ku = T(1.0 - cv.eta_b), ku3 = T(3.0 * (1.0 - cv.eta_b));
  const T xeH = GEN ? T(0) : T(a.geo.xeH[goff + cc]);  // x_eta / H of this column
  // general quadrilateral: the node's c xi_x, c xi_y, c eta_x, c eta_y and J of
  // Eqs. (3.2)-(3.3), formed in FP64 at creation and rounded to FP32 planes
  const float *qm = GEN ? a.geo.qmet_f + 5 * cv.off : nullptr;
  auto qmet = [&](int k, int j) -> T { return qm[k * plane + int64_t(j) * pitch + cc]; };
  const T wx = T(((c == 0 || c == nx - 1) ? 0.5 : 1.0) * cv.dxi);
  // The FP32 trapezoid stencils take their near-wall form from ghost values
  // (write_ghosts) instead of per-plane selects on the wall flags.
  constexpr bool GHOST = sizeof(T) == 4;
  // approximate FP32 quotients (quot); the general-quadrilateral variant, whose
  // registers are at the cap, keeps the division (the approximation's extra
  // live values spill there)
  constexpr bool FASTQ = !GEN;
  const T Pr = T(a.pref[task.cav]);                  // reference pressure of the deviations

  Partial p = {0, 0, 0, 0, 0, 0, 0};
  Leaf<T> leaf;

  const int kb = j0 - 4;
  const int rlo = max(kb, 0), rhi = min(j1 + 3, ny - 1);   // rows of stage A
  const int mlo = max(1, j0 - 2), mhi = min(ny - 2, j1 + 1);  // rows of the half step
  const int olo = max(1, j0), ohi = min(ny - 2, j1 - 1);      // rows of the full step
  const int nit = (j1 + 3 - kb) / 2 + 1;                      // k = kb + 2 it, it < nit
  auto row_of = [&](int it) { return kb + 2 * it + h; };      // this thread's stage-A row
  // Row prefetch: lane 0 of each warp copies the warp's 32 columns (from
  // column i0 - 4 + 32 (l / 32), a multiple of 4 since strips start at
  // multiples of 4) x 9 planes of row r into the warp's box of slot it % PF,
  // by TMA; columns outside the cavity arrive as zeros. The warp waits on the
  // slot's mbarrier before it reads the box (wait_row).
  const int wid = t >> 5, lane = t & 31;
  T *const sfme = &S.sf[0][wid][0][lane];               // this thread's column of slot 0
  const int tx = i0 - 4 + (l & ~31);
  const void *tmap = static_cast<const char *>(a.tmap_in) + size_t(task.cav) * TMAP_BYTES;
  const bool aligned = (tx & 3) == 0;
  const bool issue = aligned && !a.tma_skip;
  auto prefetch = [&](int it) {
    const int r = row_of(it);
    if (lane == 0 && r >= rlo && r <= rhi && issue)
      tma_load_box3(&S.sf[pf_slot(it)][wid][0][0], tmap, tx, r, &S.bar[pf_slot(it)][wid],
                    uint32_t(9 * 32 * sizeof(T)));
  };
  // A wait that runs out is reported in the status word; the warp then waits
  // no more for rows in this task (their data are lost anyway), so that a
  // failing task ends after one bounded wait per warp, and the end of the task
  // waits, bounded too, for the last copy it issued into each slot. The phase
  // bits follow the issued copies only.
  bool gave_up = false;
  auto wait_row = [&](int it) {
    const int r = row_of(it);
    if (r >= rlo && r <= rhi) {
      const int s = pf_slot(it);
      const bool ok = aligned && !gave_up && mbar_wait(&S.bar[s][wid], (phase >> s) & 1u);
      if (!ok && !gave_up && lane == 0) atomicOr(a.status, STATUS_TMA_TIMEOUT);
      gave_up = gave_up || !ok;
      if (issue) phase ^= 1u << s;
    }
  };
  // lambda_prev of a row Step (2) works on, loaded one iteration ahead
  auto lam_load = [&](int r) {
    return (r >= rlo && r <= rhi) ? lam_in[int64_t(r) * pitch + cc] : T(0);
  };
  // per-cavity constants of the relaxation time
  const double gmin2 = cv.gmin2, half_nm1 = cv.half_nm1, Kics2 = cv.Kics2;
  // the FP32 strain rate's clamp: the largest float not above gamma_min^2 (so
  // that every clamped q is >= it), and not below FLT_MIN
  const float gmin2_f = cv.gmin2_f;
  const float half_nm1_f = float(half_nm1), Kics2_f = float(Kics2);
  // pow_tab of the FP32 form: the cavity's table and binomial coefficients
  const double *powt = a.powt + int64_t(task.cav) * POWT_SIZE;
  const double pb2 = cv.pb2;
  const float pb3 = cv.pb3, pb4 = cv.pb4, pb5 = cv.pb5;
  const T wy_in = T(cv.deta), wy_edge = T(0.5 * cv.deta);
  // Step (2) for this thread's row of iteration `it`: moments, f^eq and
  // lambda(t). The row of iteration it + 1 is formed during the full step of
  // iteration it, so that the power overlaps the stencil work.
  T nux = 0, nuy = 0, nP = 0, ngeq[9];
  T nlam = T(0);
  struct Collided {
    T ux, uy, P, geq[9];
    T lam;
  };
  auto collide = [&](int it, T lam_prev) {
    Collided o;
    const int s = pf_slot(it);
    T g[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) g[q] = sfme[s * SLOT + q * 32];
    moments(g, c_, cs2, o.ux, o.uy, o.P);                 // Eqs. (2.10)-(2.11)
    equilibrium(o.P, o.ux, o.uy, c_, ics2, o.geq);        // Eq. (2.8)
    T d[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) d[q] = g[q] - o.geq[q];
    T pxx, pxy, pyy;
    second_moments(d, c_, pxx, pxy, pyy);
    if constexpr (IMPL) {                                  // implicit form of Eq. (2.14)
      const T G2 = T(0.5) * (pxx * pxx + T(2) * pxy * pxy + pyy * pyy);
      if constexpr (P32)
        o.lam = T(lambda_implicit_f32(float(T(2) * sqrt(G2) * ics2), float(lam_prev), cv));
      else
        o.lam = T(lambda_implicit(2.0 * sqrt(double(G2)) * cv.inv_cs2, double(lam_prev), cv,
                                  a.powtab));
      return o;
    }
    // Eqs. (2.12)-(2.14), (1.4): strain rate in T, power in FP64 (as
    // relaxation_time), or in FP32 with the pow32 opt-in
    const T k = quot<FASTQ>(T(-2), (T(2) * lam_prev + dt) * cs2);
    const T Sxx = k * pxx, Sxy = k * pxy, Syy = k * pyy;
    if constexpr (sizeof(T) == 4) {
      // the strain rate is FP32 here: clamped in FP32, then C q^m in FP64 by
      // pow_tab (7 FP64 instructions) and rounded to the FP32 plane
      const float qf = fmaxf(T(0.5) * (Sxx * Sxx + T(2) * Sxy * Sxy + Syy * Syy), gmin2_f);
      if constexpr (P32)
        o.lam = Kics2_f * pow_f32(qf, half_nm1_f);
      else
        o.lam = float(pow_tab(qf, powt, half_nm1, pb2, pb3, pb4, pb5));
    } else {
      double q = double(T(0.5) * (Sxx * Sxx + T(2) * Sxy * Sxy + Syy * Syy));
      q = q > gmin2 ? q : gmin2;
      o.lam = Kics2 * pow_fast(q, half_nm1, a.powtab);
    }
    return o;
  };
  auto take = [&](const Collided &o) {
    nux = o.ux;
    nuy = o.uy;
    nP = o.P;
#pragma unroll
    for (int q = 0; q < 9; ++q) ngeq[q] = o.geq[q];
    nlam = o.lam;
  };
  auto in_a = [&](int r) { return r >= rlo && r <= rhi; };

  if (lane == 0) tmap_acquire(tmap);
  prefetch(0);
  prefetch(1);
  wait_row(0);
  if (in_a(row_of(0))) take(collide(0, lam_load(row_of(0))));
  T lp_next = lam_load(row_of(1));       // lambda_prev of the next row
  T Lprev = T(0);                        // lambda(t) of this thread's previous row
  // metrics of this iteration's half-step and full-step rows, loaded one
  // iteration ahead (rows clamped into the cavity; unused outside it)
  auto crow = [&](int r) { return min(max(r, 0), ny - 1); };
  // (general quadrilaterals load their row values where they are used: one
  // broadcast load per warp, which keeps the register budget of the march)
  T A1 = 0, A2 = 0, J2 = 0;
  if constexpr (!GEN) {
    A1 = row_cxix(crow(kb - 2 + h)), A2 = row_cxix(crow(kb - 4 + h)), J2 = row_jac(crow(kb - 4 + h));
  }

  for (int it = 0; it < nit; ++it) {
    const int k = kb + 2 * it;

    // ---------------- stage A: row k + h (lambda formed in the previous iteration) ----------------
    const int ar = k + h;
    T Lcur = T(0);
    if (in_a(ar)) {
      const int s = pf_slot(it), sb = slot6(ar);
      if (own && ar >= j0 && ar < j1) lam_out[int64_t(ar) * pitch + c] = nlam;
      const T L = nlam;
      Lcur = L;
      const T i2 = quot<FASTQ>(T(1), T(2) * L + dt);
      const T bp = T(2) * dt * i2;     // Eq. (2.15): (2 lam - dt)/(2 lam + dt) = 1 - bp
      const T bb = T(1.5) * dt * i2;   // Eq. (2.16): 3 dt/(4 lam + 2 dt) = bb
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const T gq = sfme[s * SLOT + q * 32];
        S.fb[sb][q][l] = toward(gq, ngeq[q], bb);
        sfme[s * SLOT + q * 32] = toward(gq, ngeq[q], bp);  // f-hat^+ in place of g
      }
      if (ar == 0 || ar == ny - 1) {
        const int e = ar == 0 ? 0 : 1;
        S.edge[e][0][l] = nux;
        S.edge[e][1][l] = nuy;
        S.edge[e][2][l] = nP;
      }
    }
    __syncthreads();  // f-bar^+ of rows k, k + 1
    // the slot this prefetch fills was last read before the barrier above
    prefetch(it + 2);

    // ---------------- stage 1: row m = k - 2 + h ----------------
    const int m = k - 2 + h;
    const bool do1 = m >= mlo && m <= mhi;
    if (do1 && inner_c && l >= 2 && l < NC - 2) {
      const int sm = slot6(m);
      const bool lo = m == 1, hi = m == ny - 2;
      T fbar[9];
      fbar[0] = S.fb[sm][0][l];
      {
        const T *cols[5] = {&S.fb[slot6(m - 2)][0][l], &S.fb[slot6(m - 1)][0][l], &S.fb[sm][0][l],
                            &S.fb[slot6(m + 1)][0][l], &S.fb[slot6(m + 2)][0][l]};
        if constexpr (GEN) {
          AdvectAllGen<T, 1, NC, NC>::run(&S.fb[sm][0][0], cols, l, qmet(0, m), qmet(1, m),
                                          qmet(2, m), qmet(3, m), clo, chi, lo, hi, eta_b, i2dxi,
                                          i2deta, hdt,
                                          &S.fb[sm][0][l], fbar);  // Eq. (3.7)
        } else {
          const T As = A1 * hxs;                         // dt/2 c xi_x / (2 dxi) of row m
          const T Bs = As * xeH;                         // ... times x_eta / H
          if constexpr (GHOST)
            write_ghosts<T, NC>(&S.fb[sm][0][0], l, clo, chi, lo, hi, &S.fb[slot6(-1)][0][l],
                                &S.fb[slot6(0)][0][l], &S.fb[slot6(ny)][0][l],
                                &S.fb[slot6(ny - 1)][0][l]);
          AdvectAll<T, 1, NC, NC, !GHOST>::run(&S.fb[sm][0][0], cols, l, As, Bs, Es1, clo, chi, lo,
                                               hi, eta_b, ku3, ku, &S.fb[sm][0][l],
                                               fbar);  // Eq. (3.7)
        }
      }
      T ux, uy, P;
      moments(fbar, c_, cs2, ux, uy, P);
      T geq[9];
      equilibrium(P, ux, uy, c_, ics2, geq);
      const T L = Lprev;                                 // lambda(t) of row m
      const T bh = quot<FASTQ>(dt, T(4) * L + dt);       // Eq. (2.17): 1 - bh = 4 lam/(4 lam + dt)
      T fh[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) S.fh[sm][q][l] = fh[q] = toward(fbar[q], geq[q], bh);
      // Wall nodes of f(t + dt/2) that take this node as their neighbour, written
      // by this thread: the side wall of its row (column 1 -> 0, nx-2 -> nx-1),
      // the bottom (row 1 -> 0) and the lid (row ny-2 -> ny-1), and at the
      // corners the diagonal wall node. Every one of them but the lid's moving
      // nodes takes nee(F, 0); the lid's interior nodes take nee(F, u_lid).
      if (clo || chi || lo || hi) {
        T W[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) W[q] = fh[q];
        nee(W, T(0), T(0), c_, cs2, ics2);
        const int lw = clo ? l - 1 : l + 1;               // lane of the side wall column
        const bool side = (clo || chi) && lw >= 2 && lw < NC - 2;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          if (side) S.fh[sm][q][lw] = W[q];                           // (m, 0) / (m, nx-1)
          if (lo) S.fh[slot6(0)][q][l] = W[q];                        // (0, c)
          if (side && lo) S.fh[slot6(0)][q][lw] = W[q];               // corner (0, 0) / (0, nx-1)
          if (side && hi) S.lid[q][lw] = W[q];                        // corner (ny-1, 0) / (ny-1, nx-1)
        }
        if (hi) {                                                     // (ny-1, c): the lid
#pragma unroll
          for (int q = 0; q < 9; ++q) W[q] = fh[q];
          nee(W, Uw, Uwy, c_, cs2, ics2);
#pragma unroll
          for (int q = 0; q < 9; ++q) S.lid[q][l] = W[q];
        }
      }
    }
    Lprev = Lcur;
    __syncthreads();  // f(t + dt/2) of rows m, wall nodes included

    // ---------------- stage 2: row o = k - 4 + h ----------------
    const int o = k - 4 + h;
    const bool do2 = o >= olo && o <= ohi;
    const int sp = pf_slot(it + PF - 2);             // f-hat^+ of row o (iteration it - 2)
    wait_row(it + 1);                                // this warp's row of iteration it + 1
    T gnv[9];
    if (do2 && inner_c && l >= 4 && l < NC - 4) {
      const int so = slot6(o);
      const bool lo = o == 1, hi = o == ny - 2;
      gnv[0] = sfme[sp * SLOT];
      {
        // rows o-2..o+2 of f(t + dt/2); the lid row ny-1 has a buffer of its own
        auto fhrow = [&](int r) -> const T * {
          return r == ny - 1 ? &S.lid[0][l] : &S.fh[slot6(r)][0][l];
        };
        const T *cols[5] = {fhrow(o - 2), fhrow(o - 1), &S.fh[so][0][l], fhrow(o + 1),
                            fhrow(o + 2)};
        if constexpr (GEN) {
          AdvectAllGen<T, 1, NC, 32>::run(&S.fh[so][0][0], cols, l, qmet(0, o), qmet(1, o),
                                          qmet(2, o), qmet(3, o), clo, chi, lo, hi, eta_b, i2dxi,
                                          i2deta, dt,
                                          sfme + sp * SLOT, gnv);  // Eq. (3.6)
        } else {
          const T As = A2 * fxs;                         // dt c xi_x / (2 dxi) of row o
          const T Bs = As * xeH;
          if constexpr (GHOST)
            write_ghosts<T, NC>(&S.fh[so][0][0], l, clo, chi, lo, hi, &S.fh[slot6(-1)][0][l],
                                &S.fh[slot6(0)][0][l], &S.fh[slot6(ny)][0][l], &S.lid[0][l]);
          AdvectAll<T, 1, NC, 32, !GHOST>::run(&S.fh[so][0][0], cols, l, As, Bs, Es2, clo, chi, lo,
                                               hi, eta_b, ku3, ku, sfme + sp * SLOT,
                                               gnv);  // Eq. (3.6)
        }
      }
      if (clo || chi) {                                // values the wall columns extrapolate
#pragma unroll
        for (int q = 0; q < 9; ++q) S.gw[h][chi ? 1 : 0][q] = gnv[q];
      }
    }
    if (in_a(row_of(it + 1))) take(collide(it + 1, lp_next));  // lambda of the next row
    lp_next = lam_load(row_of(it + 2));
    [[maybe_unused]] const T J2o = J2;               // Jacobian of row o (trapezoid)
    if constexpr (!GEN) {
      A1 = row_cxix(crow(m + 2));
      A2 = row_cxix(crow(o + 2));
      J2 = row_jac(crow(o + 2));
    }
    __syncthreads();  // f-hat(t + dt) of columns 1 and nx-2

    if (do2 && own) {
      if (wall_c) {
        const int side = c == 0 ? 0 : 1;
#pragma unroll
        for (int q = 0; q < 9; ++q) gnv[q] = S.gw[h][side][q];
        nee(gnv, T(0), T(0), c_, cs2, ics2);
      }
      const int64_t node = int64_t(o) * pitch + c;
#pragma unroll
      for (int q = 0; q < 9; ++q) gout[q * plane + node] = gnv[q];
      if (a.want_residual) {
        T ux, uy, P, u0, v0, P0;
        moments(gnv, c_, cs2, ux, uy, P);
        T fpo[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) fpo[q] = sfme[sp * SLOT + q * 32];
        moments(fpo, c_, cs2, u0, v0, P0);  // u, P at t (moments of f-hat^+ equal those of f-hat)
        T Jo;
        if constexpr (GEN)
          Jo = qmet(4, o);                             // Jacobian of node (c, o)
        else
          Jo = J2o;
        const T wJ = wx * wy_in * Jo;
        leaf_add(leaf, p, ux, uy, P, u0, v0, P0, Pr, wJ, a.status);
      }
      // wall rows produced with their neighbour rows
      const bool bottom = o == 1 && j0 == 0;
      const bool top = o == ny - 2 && j1 == ny;
      if (bottom || top) {
        T F[9];
        if (wall_c) {
          const int side = c == 0 ? 0 : 1;
#pragma unroll
          for (int q = 0; q < 9; ++q) F[q] = S.gw[h][side][q];
        } else {
#pragma unroll
          for (int q = 0; q < 9; ++q) F[q] = gnv[q];
        }
        nee(F, (top && inner_c) ? Uw : T(0), (top && inner_c) ? Uwy : T(0), c_, cs2, ics2);
        const int r = bottom ? 0 : ny - 1;
        const int64_t nd = int64_t(r) * pitch + c;
#pragma unroll
        for (int q = 0; q < 9; ++q) gout[q * plane + nd] = F[q];
        if (a.want_residual) {
          T wx2, wy2, wP2;
          moments(F, c_, cs2, wx2, wy2, wP2);
          const int e = bottom ? 0 : 1;
          T Jr;
          if constexpr (GEN)
            Jr = qmet(4, r);
          else
            Jr = row_jac(r);
          const T wJ = wx * wy_edge * Jr;
          leaf_add(leaf, p, wx2, wy2, wP2, S.edge[e][0][l], S.edge[e][1][l], S.edge[e][2][l], Pr,
                   wJ, a.status);
        }
      }
    }
    // this iteration's reads and writes of the warp's boxes are ordered before
    // the TMA copies that refill them after the next barrier
    fence_proxy_async_smem();
  }
  // After a wait ran out, wait (bounded) for the last copy issued into each
  // slot, so that none is left writing into shared memory the next task uses
  // (a slot's previous phase counts as complete when none was issued).
  if (gave_up && issue)
    for (int s = 0; s < PF; ++s) mbar_wait(&S.bar[s][wid], ((phase >> s) & 1u) ^ 1u);
  if (a.want_residual) {
    leaf_flush(leaf, p);
    p.du2max = double(leaf.du2max);
    p.u2max = double(leaf.u2max);
    block_partial<NT / 32>(p, a.part, ti);
    // The last task of the cavity to finish reduces the cavity's partials
    // (a counter, no waiting: every other CTA just moves on).
    __shared__ int last;
    __syncthreads();                       // this task's partial is written
    if (threadIdx.x == 0) {
      __threadfence();                     // ... and visible device-wide
      last = atomicAdd(&a.cav_done[task.cav], 1) == nparts - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();                     // see the other tasks' partials
      reduce_partials_block<NT / 32>(a.part + int64_t(part0) * NPART, nparts,
                                     a.resid + 4 * task.cav);
      if (threadIdx.x == 0) a.cav_done[task.cav] = 0;   // re-armed for the next step
    }
  }
  __syncthreads();  // the next task reuses the shared rings
}

// Launch bounds: 16 resident warps per SM in FP32 (registers capped at 128),
// 8 in FP64 (its shared rings are twice as large).
template <class T, int NT>
struct Occ {
  static constexpr int blocks = (sizeof(T) == 4 ? 512 : 256) / NT > 0 ? (sizeof(T) == 4 ? 512 : 256) / NT : 1;
};

// Schedules: 0 one CTA per task; 1 persistent CTAs taking positions
// blockIdx.x, blockIdx.x + gridDim.x, ... of the largest-first order;
// 2 persistent CTAs taking positions from an atomic counter (no waiting on
// other CTAs: a CTA that finds the list exhausted returns).
template <class T, int NT, bool IMPL, bool GEN, bool P32>
__global__ void __launch_bounds__(NT, Occ<T, NT>::blocks) k_fused(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the TMA boxes want 128-byte aligned shared memory: align the struct
  const uint32_t s0 = smem_addr(smem_raw);
  FusedSmem<T, NT> &S =
      *reinterpret_cast<FusedSmem<T, NT> *>(smem_raw + (((s0 + 127u) & ~127u) - s0));
  __shared__ int next;
  constexpr int NW = FusedSmem<T, NT>::NW;
  if (threadIdx.x < PF * NW) mbar_init(&S.bar[0][0] + threadIdx.x, 1);
  mbar_init_fence();
  __syncthreads();
  unsigned phase = 0;  // bit s: parity of the next completion of slot s's barrier (this warp)
  if (a.schedule == 0) {
    fused_task<T, NT, IMPL, GEN, P32>(a, S, blockIdx.x, phase);
    return;
  }
  for (int it = 0;; ++it) {
    int pos;
    if (a.schedule == 1) {
      pos = blockIdx.x + it * gridDim.x;
    } else {
      if (threadIdx.x == 0) next = atomicAdd(a.counter, 1);
      __syncthreads();
      pos = next;
      __syncthreads();
    }
    if (pos >= a.ntasks) return;
    fused_task<T, NT, IMPL, GEN, P32>(a, S, a.order[pos], phase);
  }
}

template <class T, int NT, bool IMPL, bool GEN = false, bool P32 = false>
static void configure_nt() {
  static bool configured = false;  // the attribute is per function
  if (!configured) {
    cudaFuncSetAttribute(k_fused<T, NT, IMPL, GEN, P32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         fused_smem_size<T, NT>());
    configured = true;
  }
}

template <class T, int NT, bool IMPL, bool GEN, bool P32>
static void launch_variant(const FusedArgs &a, int grid, cudaStream_t s) {
  configure_nt<T, NT, IMPL, GEN, P32>();
  k_fused<T, NT, IMPL, GEN, P32><<<grid, NT, fused_smem_size<T, NT>(), s>>>(a);
}

template <class T, int NT>
static void launch_fused_nt(const FusedArgs &a, int grid, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    // FP32 storage: general quadrilaterals (lagged relaxation time only; the
    // host admits no other combination) and the FP32-power opt-in
    if (a.general) {
      if (a.pow32)
        launch_variant<T, NT, false, true, true>(a, grid, s);
      else
        launch_variant<T, NT, false, true, false>(a, grid, s);
      return;
    }
    if (a.pow32) {
      if (a.implicit)
        launch_variant<T, NT, true, false, true>(a, grid, s);
      else
        launch_variant<T, NT, false, false, true>(a, grid, s);
      return;
    }
  }
  if (a.implicit)
    launch_variant<T, NT, true, false, false>(a, grid, s);
  else
    launch_variant<T, NT, false, false, false>(a, grid, s);
}

template <class T, int NT>
static int blocks_per_sm_nt() {
  configure_nt<T, NT, false>();
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<T, NT, false, false, false>, NT,
                                                fused_smem_size<T, NT>());
  return n;
}

template <class T> int fused_blocks_per_sm(int nt) {
  switch (nt) {
    case 64: return blocks_per_sm_nt<T, 64>();
    case 128: return blocks_per_sm_nt<T, 128>();
    case 256: return blocks_per_sm_nt<T, 256>();
  }
  return 0;
}

template <class T> int fused_smem_bytes(int nt) {
  switch (nt) {
    case 64: return fused_smem_size<T, 64>();
    case 128: return fused_smem_size<T, 128>();
    case 256: return fused_smem_size<T, 256>();
  }
  return -1;
}

template <class T> bool launch_fused(const FusedArgs &a, int nt, int ntasks, cudaStream_t s) {
  switch (nt) {
    case 64: launch_fused_nt<T, 64>(a, ntasks, s); return true;
    case 128: launch_fused_nt<T, 128>(a, ntasks, s); return true;
    case 256: launch_fused_nt<T, 256>(a, ntasks, s); return true;
  }
  return false;
}

template bool launch_fused<float>(const FusedArgs &, int, int, cudaStream_t);
template bool launch_fused<double>(const FusedArgs &, int, int, cudaStream_t);
template int fused_smem_bytes<float>(int);
template int fused_smem_bytes<double>(int);
template int fused_blocks_per_sm<float>(int);
template int fused_blocks_per_sm<double>(int);

}  // namespace ifd
