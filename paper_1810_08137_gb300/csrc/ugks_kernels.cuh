// Device kernels of one explicit 2D UGKS step (Liu, Hu & Li, arXiv:1810.08137, Sec. 2).
//
// Per step, on one stream:
//   k_ghost_x, k_ghost_y  boundary ghost ring (periodic image, wall zero-gradient copy,
//                         pressure Maxwellian)
//   k_sums                per cell and side, the velocity sums of steps S1 and S7 (W0,
//                         tangential slope of W, free-transport sums) over one read of f
//   k_faces               per interface, steps S2-S5 (Maxwellian moments, Mt time weights,
//                         micro slopes a_L a_R b A, equilibrium flux) in FP64, the total
//                         macroscopic flux, and the coefficients of the micro flux (S6, S8);
//                         the FP32-f form runs the terms that carry slopes in FP32
//   k_cells               conservative W update (Eq. 4), g^n, g^{n+1}, tau^n, tau^{n+1}
//   k_face_flux           micro flux of every face and velocity (S6, S8), once, from its
//                         upwind cell, into face-flux buffers (second read of f)
//   k_cell_update         the implicit f update (Eq. 3) from the four fluxes of each
//                         velocity-cell, one write of f^{n+1}
//   (k_update, the same update in one pass that forms each interior flux twice, serves the
//   allocation-free entry point)
// These are the FP64 form's kernels; the FP32-f form (FP32 f in a paired-row layout) has
// its own ghost fill, sums and update in ugks_f32.cuh and shares the interface and cell
// bodies (faces_body, cells_body).
//
// Layout: f[(ny+4)(nx+4)][nq] of T2 = (h, b), velocity innermost (q = m*nu + k), a ghost
// ring two cells wide; W[4][(ny+2)(nx+2)] FP64 with a ghost ring one cell wide.
#pragma once
#include <math.h>

#include <type_traits>

#include "ugks_internal.h"
#include "ugks_dfcore.cuh"

namespace ugks {

constexpr unsigned kFull = 0xffffffffu;
constexpr double kPi = 3.14159265358979323846;

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

__host__ __device__ __forceinline__ size_t fcell(const Params& P, int i, int j) {
  return (size_t)(j + 2) * P.ex + (i + 2);
}
__host__ __device__ __forceinline__ int wcell(const Params& P, int i, int j) {
  return (j + 1) * P.wx + (i + 1);
}

// 1/s from the hardware FP64 reciprocal estimate and two Newton steps (each doubles the
// number of correct bits), within a few ulp of 1/s for normal s; an IEEE divide costs more
// FP64 instructions, and FP64 issues at 1/64 of the FP32 rate on this part.
__device__ __forceinline__ double rcp_nr(double s) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(s));
  double e = fma(-s, r, 1.0);
  r = fma(r, e, r);
  e = fma(-s, r, 1.0);
  return fma(r, e, r);
}
// van Leer limited slope of the stencil (a, c, b) times half the cell width:
// r = sigma dx / 2 = d1 d2 / (d1 + d2) if d1 d2 > 0, else 0, with d1 = c - a, d2 = b - c.
// (d1 d2 > 0 implies d1 + d2 != 0; a product small enough to make d1 + d2 subnormal
// underflows to 0 and takes the zero branch.)
__device__ __forceinline__ double vl_half(double a, double c, double b) {
  double d1 = c - a, d2 = b - c, p = d1 * d2;
  return p > 0.0 ? p * rcp_nr(d1 + d2) : 0.0;
}
// 2^x and 1/x with subnormal results flushed to zero (PTX approximate forms).
__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_ftz(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// 16-byte asynchronous global -> shared copies (per thread), in commit groups.
__device__ __forceinline__ void cp_async16(void* sm, const void* gm) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(sm);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gm) : "memory");
}
// The same, cached in L2 only (data read once by this warp).
__device__ __forceinline__ void cp_async16_cg(void* sm, const void* gm) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(sm);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gm) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async8(void* sm, const void* gm) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(sm);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(a), "l"(gm) : "memory");
}
// one f value (float2: 8 bytes, double2: 16 bytes)
__device__ __forceinline__ void cp_async_f(float2* sm, const float2* gm) { cp_async8(sm, gm); }
__device__ __forceinline__ void cp_async_f(double2* sm, const double2* gm) { cp_async16(sm, gm); }


// Collision time tau = mu / p with mu = mu_ref T^omega, T = 1/lam, p = rho / (2 lam).
__device__ __forceinline__ double collision_time(const Params& P, double rho, double lam) {
  const double lw = P.omega_half ? rsqrt(lam) : pow(lam, -P.omega);  // lam^-omega = T^omega
  return P.mu_ref * lw * 2.0 * lam / rho;
}

// Sum over the warp of v[lane % N] returned to each lane (N = 16 or 32): transpose
// reduce-scatter, N-1 shuffles instead of N*5.
template <int N, typename T>
__device__ __forceinline__ T warp_reduce_scatter(T (&v)[N], int lane) {
#pragma unroll
  for (int o = N / 2; o >= 1; o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; i++) {
      T send = upper ? v[i] : v[i + o];
      T keep = upper ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  T r = v[0];
#pragma unroll
  for (int o = N; o < 32; o <<= 1) r += __shfl_xor_sync(kFull, r, o);
  return r;
}

// Reference Maxwellian (h, b) of the FP32 form at velocity (u, v); zero when unused.
__host__ __device__ __forceinline__ void ref_maxwellian(const Params& P, double u, double v,
                                                        double& h, double& b) {
  if (!P.use_ref) { h = b = 0.0; return; }
  const double du = u - P.ref_U, dv = v - P.ref_V;
  h = P.ref_G * exp(-P.ref_lam * (du * du + dv * dv));
  b = P.ref_bf * h;
}

// -------------------------------------------------------------------------------------
// Boundary ghost ring
// -------------------------------------------------------------------------------------
// tab: shared memory of the block for 4 kMaxAxis doubles (per-axis Maxwellian factors)
constexpr int kGhostTab = 4 * kMaxAxis;
template <typename T2>
__device__ void fill_ghost_cell(const Params& P, T2* f, double* W, int nwe, int gi, int gj,
                                int si, int sj, int side, bool write_W, int wi, int wj,
                                double* tab) {
  const int kind = P.bc_kind[side];
  T2* dst = f + fcell(P, gi, gj) * P.nq;
  const T2* src = f + fcell(P, si, sj) * P.nq;
  const int sw = wcell(P, wi, wj);
  if (kind == 2) {  // pressure: Maxwellian(rho_bc, U and V of the adjacent cell, T_bc)
    // both Maxwellians factor into a u part and a v part: per-axis tables in shared memory
    double* fu = tab;
    double* fv = tab + kMaxAxis;
    double* ru = tab + 2 * kMaxAxis;
    double* rv = tab + 3 * kMaxAxis;
    const double rho_a = W[sw], U = W[nwe + sw] / rho_a, V = W[2 * nwe + sw] / rho_a;
    const double lam = 1.0 / P.bc_T[side], rho = P.bc_rho[side];
    const double G = rho * lam / kPi, bf = P.K / (2.0 * lam);
    __syncthreads();  // the tables of the previous cell are no longer read
    for (int k = threadIdx.x; k < P.nu; k += blockDim.x) {
      const double du = P.u[k] - U, dr = P.u[k] - P.ref_U;
      fu[k] = G * exp(-lam * du * du);
      ru[k] = P.use_ref ? P.ref_G * exp(-P.ref_lam * dr * dr) : 0.0;
    }
    for (int m = threadIdx.x; m < P.nv; m += blockDim.x) {
      const double dv = P.v[m] - V, dr = P.v[m] - P.ref_V;
      fv[m] = exp(-lam * dv * dv);
      rv[m] = exp(-P.ref_lam * dr * dr);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < P.nq; q += blockDim.x) {
      const int k = q % P.nu, m = q / P.nu;
      const double gh = fu[k] * fv[m], rh = ru[k] * rv[m];
      T2 o;
      o.x = gh - rh;
      o.y = bf * gh - P.ref_bf * rh;
      dst[q] = o;
    }
    if (write_W && threadIdx.x == 0) {
      const int g = wcell(P, gi, gj);
      W[g] = rho;
      W[nwe + g] = rho * U;
      W[2 * nwe + g] = rho * V;
      W[3 * nwe + g] = rho * (0.5 * (U * U + V * V) + (P.K + 2) / (4.0 * lam));
    }
  } else {  // periodic image or zero-gradient copy next to a wall
    for (int q = threadIdx.x; q < P.nq; q += blockDim.x) dst[q] = src[q];
    if (write_W && threadIdx.x == 0) {
      const int g = wcell(P, gi, gj), s = wcell(P, si, sj);
      for (int c = 0; c < 4; c++) W[c * nwe + g] = W[c * nwe + s];
    }
  }
}

// FP32 paired-row layout (ugks_f32.cuh)
__device__ void fill_ghost_cell(const Params& P, float4* f, double* W, int nwe, int gi, int gj,
                                int si, int sj, int side, bool write_W, int wi, int wj,
                                double* tab);

// x-sides, rows 0..ny-1; grid (ny, 4): blockIdx.y = side*2 + layer-1.
template <typename T2>
__device__ __forceinline__ void ghost_x_body(const Params& P, T2* f, double* W, int nwe, int bx, int by,
                                             double* tab) {
  const int j = bx, side = by >> 1, l = (by & 1) + 1;
  const int kind = P.bc_kind[side];
  const int gi = side == 0 ? -l : P.nx - 1 + l;
  int si;
  if (kind == 0) si = side == 0 ? P.nx - l : l - 1;
  else si = side == 0 ? 0 : P.nx - 1;
  const int ai = side == 0 ? 0 : P.nx - 1;  // adjacent interior cell (pressure velocity source)
  fill_ghost_cell(P, f, W, nwe, gi, j, si, j, side, l == 1, kind == 2 ? ai : si, j, tab);
}
template <typename T2>
__global__ void k_ghost_x(Params P, T2* f, double* W, int nwe) {
  __shared__ double tab[kGhostTab];
  ghost_x_body(P, f, W, nwe, blockIdx.x, blockIdx.y, tab);
}

// y-sides over all columns -2..nx+1 (corners included, after the x-sides);
// grid (nx+4, 4): blockIdx.y = side*2 + layer-1, side 0: S, 1: N.
template <typename T2>
__device__ __forceinline__ void ghost_y_body(const Params& P, T2* f, double* W, int nwe, int bx, int by,
                                             double* tab) {
  const int i = bx - 2, side = 2 + (by >> 1), l = (by & 1) + 1;
  const int kind = P.bc_kind[side];
  const int gj = side == 2 ? -l : P.ny - 1 + l;
  int sj;
  if (kind == 0) sj = side == 2 ? P.ny - l : l - 1;
  else sj = side == 2 ? 0 : P.ny - 1;
  const int aj = side == 2 ? 0 : P.ny - 1;
  const bool wcol = i >= -1 && i <= P.nx;
  const int wi = i < -1 ? -1 : (i > P.nx ? P.nx : i);
  fill_ghost_cell(P, f, W, nwe, i, gj, i, sj, side, l == 1 && wcol, wi, kind == 2 ? aj : sj, tab);
}
template <typename T2>
__global__ void k_ghost_y(Params P, T2* f, double* W, int nwe) {
  __shared__ double tab[kGhostTab];
  ghost_y_body(P, f, W, nwe, blockIdx.x, blockIdx.y, tab);
}

// -------------------------------------------------------------------------------------
// Steps S1 + S7: per-cell half-range velocity sums.  One warp per cell, lane = u index
// (chunks of 32), loop over v.  Cells: interior plus the first ghost layer of every
// side that is not a wall.
// -------------------------------------------------------------------------------------
template <typename T, typename T2>
__device__ __forceinline__ void finalize_y(T u, T wu, T tdx, T P0, T P1, T P2, T P3, T Pb0, T Pb1,
                                           T Q0, T Q1, T Q2, T Qb, T Z1, T Z2, T Z3, T Zb1,
                                           int lane, T* ws_side) {
  T v[16];
  const T uu = u * u;
  v[0] = wu * P0;
  v[1] = wu * u * P0;
  v[2] = wu * P1;
  v[3] = wu * (T(0.5) * (uu * P0 + P2) + T(0.5) * Pb0);
  const T ws = wu * tdx;
  v[4] = ws * Q0;
  v[5] = ws * u * Q0;
  v[6] = ws * Q1;
  v[7] = ws * (T(0.5) * (uu * Q0 + Q2) + T(0.5) * Qb);
  v[8] = wu * P1;
  v[9] = wu * u * P1;
  v[10] = wu * P2;
  v[11] = wu * (T(0.5) * (uu * P1 + P3) + T(0.5) * Pb1);
  v[12] = wu * Z1;
  v[13] = wu * u * Z1;
  v[14] = wu * Z2;
  v[15] = wu * (T(0.5) * (uu * Z1 + Z3) + T(0.5) * Zb1);
  const T r = warp_reduce_scatter<16>(v, lane);
  if (lane < 16) ws_side[lane] += r;
}

// wv v^n, n = 0..4, of row m (global tables, L1 resident)
__device__ __forceinline__ void wtab(const Params& P, int m, double* o) {
#pragma unroll
  for (int n = 0; n < 5; n++) o[n] = __ldg(P.mvd + n * P.nv + m);
}
__device__ __forceinline__ void utab(const Params& P, int k, double& u, double& wu) {
  u = P.u[k]; wu = P.wu[k];
}

// slopes: null, or [(nx+2)(ny+2) cells (W indexing)][nq][2] of (r_x,h r_x,b), (r_y,h r_y,b),
// written for every cell whose sums are formed (the update kernel then reads them)
// Sum over the warp (every lane gets it), FP64.
__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}
// Shakhov heat-flux moments of one side's face values, from the lane's (u = ud) v-weighted
// sums F_b = sum_v w_v v^b (h face values), b = 0..3, and Fb_b (b face values), b = 0, 1,
// with the lane weight wgt (w_u, times H(u_n) on the x sides): adds the warp's
// M20 M11 M02 M30 M21 M12 M03 B00 B10 B01 to o[0..9] (lane 0 writes).
__device__ __forceinline__ void heat_side(double wgt, double ud, double F0, double F1, double F2,
                                          double F3, double Fb0, double Fb1, double* o) {
  const double u2 = ud * ud;
  const double v[10] = {wgt * u2 * F0, wgt * ud * F1, wgt * F2, wgt * u2 * ud * F0, wgt * u2 * F1,
                        wgt * ud * F2, wgt * F3, wgt * Fb0, wgt * ud * Fb0, wgt * Fb1};
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < 10; t++) {
    const double r = warp_sum_d(v[t]);
    if (lane == 0) o[t] += r;
  }
  __syncwarp();
}
// The same for the cell values over every velocity: M00 M10 M01 M20 M11 M02 M30 M21 M12 M03
// B00 B10 B01 into o[0..12].
__device__ __forceinline__ void heat_cell(double wgt, double ud, double C0, double C1, double C2,
                                          double C3, double Cb0, double Cb1, double* o) {
  const double u2 = ud * ud;
  const double v[13] = {wgt * C0,      wgt * ud * C0, wgt * C1,      wgt * u2 * C0, wgt * ud * C1,
                        wgt * C2,      wgt * u2 * ud * C0, wgt * u2 * C1, wgt * ud * C2, wgt * C3,
                        wgt * Cb0,     wgt * ud * Cb0, wgt * Cb1};
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < 13; t++) {
    const double r = warp_sum_d(v[t]);
    if (lane == 0) o[t] += r;
  }
  __syncwarp();
}

template <typename T, typename T2>
__device__ __forceinline__ void sums_body(const Params& P, const T2* __restrict__ f,
                                          T* __restrict__ sums, unsigned char* smraw, int bx,
                                          T2* __restrict__ slopes = nullptr) {
  const int nv = P.nv, nu = P.nu, nq = P.nq;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* wsum = reinterpret_cast<T*>(smraw) + warp * kNSum;
  // per-thread totals over both halves, [14 + 4][128] (touched twice per u chunk)
  T* tot = reinterpret_cast<T*>(smraw + kWarpsPerBlock * kNSum * sizeof(T)) + tid;
  // Shakhov model: this warp's heat-flux moment sums (kNHeat, FP64)
  double* hsum = reinterpret_cast<double*>(smraw + (kWarpsPerBlock * kNSum + (kSumsTotals + kHeatTotals) * 128) *
                                                       sizeof(T)) + warp * kNHeat;
  const bool heat = P.hs != nullptr;
  for (int t = lane; t < kNSum; t += 32) wsum[t] = T(0);
  for (int t = lane; t < kNHeat; t += 32) hsum[t] = 0.0;
  __syncwarp();

  const int ncx = P.nx + 2;
  const int cell = bx * kWarpsPerBlock + warp;
  if (cell >= ncx * (P.ny + 2)) return;
  const int i = cell % ncx - 1, j = cell / ncx - 1;
  const bool xg = i < 0 || i >= P.nx, yg = j < 0 || j >= P.ny;
  if (xg && yg) return;
  if ((i < 0 && P.bc_kind[0] == 1) || (i >= P.nx && P.bc_kind[1] == 1) ||
      (j < 0 && P.bc_kind[2] == 1) || (j >= P.ny && P.bc_kind[3] == 1))
    return;
  const bool zs = (i < 0 && P.bc_kind[0] == 2) || (i >= P.nx && P.bc_kind[1] == 2) ||
                  (j < 0 && P.bc_kind[2] == 2) || (j >= P.ny && P.bc_kind[3] == 2);

  const T2* fc = f + fcell(P, i, j) * nq;
  const size_t rs = (size_t)P.ex * nq;
  T2* slc = slopes ? slopes + (size_t)wcell(P, i, j) * nq * 2 : nullptr;
  T tdx, tdy;
  if (sizeof(T) == 4) { tdx = (T)P.f_tdx; tdy = (T)P.f_tdy; }
  else { tdx = T(2.0 / P.dx); tdy = T(2.0 / P.dy); }

  const int mneg = P.m_neg, mpos = P.m_pos;
  const bool v0 = mpos > mneg;
  // Per lane (u_k) and per half of the v axis, weighted sums over the half's rows of the
  // cell value c, the x half slope r_x and the y half slope r_y (w_n = wv v^n):
  //   a_n = sum w_n c_h (n < 4), ab_n = sum w_n c_b (n < 2), x_n = sum w_n r_x,h (n < 4),
  //   xb_n = sum w_n r_x,b (n < 2), y_n = sum w_n r_y,h (n < 5), yb_n = sum w_n r_y,b (n < 3).
  // Every sum the faces need follows: the face values f -/+ r_y of the half give a_n -/+ y_n,
  // and u sigma_x + v sigma_y = cu r_x + (2/dy) v r_y gives sum w_n (.) = cu x_n + (2/dy) y_{n+1}.
  // The v = 0 row (H(0) = 1/2) enters both halves with half weight.
  for (int k0 = 0; k0 < nu; k0 += 32) {
    const int k = k0 + lane;
    const bool act = k < nu;
    const int kk = act ? k : nu - 1;
    T u, wu;
    utab(P, kk, u, wu);
    if (!act) wu = T(0);
    const T cu = u * tdx;
    // totals: tA0 tA1 tA2 tAb tR0 tR1 tR2 tRb tC0 tC1 tC2 tC3 tCb0 tCb1, then tA3 tAb1 tR3 tRb1
#pragma unroll
    for (int t = 0; t < kSumsTotals + kHeatTotals; t++) tot[t * 128] = T(0);
    T a0, a1, a2, a3, ab0, ab1, x0, x1, x2, x3, xb0, xb1, y0, y1, y2, y3, y4, yb0, yb1, yb2;
    auto zero = [&]() {
      a0 = a1 = a2 = a3 = ab0 = ab1 = x0 = x1 = x2 = x3 = xb0 = xb1 = T(0);
      y0 = y1 = y2 = y3 = y4 = yb0 = yb1 = yb2 = T(0);
    };
    // the five stencil values of row m (centre, x-, x+, y-, y+)
    auto load5 = [&](int m, T2 (&v)[5]) {
      const T2* src = fc + (size_t)m * nu + kk;
      v[0] = src[0];
      v[1] = src[-nq];
      v[2] = src[nq];
      v[3] = src[-(long)rs];
      v[4] = src[rs];
    };
    auto slopes5 = [&](const T2 (&v)[5], T& rxh, T& rxb, T& ryh, T& ryb) {
      rxh = rxb = ryh = ryb = T(0);
      if (!zs) {
        rxh = vl_half(v[1].x, v[0].x, v[2].x);
        rxb = vl_half(v[1].y, v[0].y, v[2].y);
        ryh = vl_half(v[3].x, v[0].x, v[4].x);
        ryb = vl_half(v[3].y, v[0].y, v[4].y);
      }
    };
    // keep the slopes of row m for the update kernel
    auto store = [&](int m, T rxh, T rxb, T ryh, T ryb) {
      if (slc && act) {
        T2* q = slc + 2 * ((size_t)m * nu + k);
        T2 a, b;
        a.x = rxh; a.y = rxb;
        b.x = ryh; b.y = ryb;
        q[0] = a;
        q[1] = b;
      }
    };
    auto slopes_of = [&](int m, T& rxh, T& rxb, T& ryh, T& ryb, T2& c) {
      T2 v[5];
      load5(m, v);
      slopes5(v, rxh, rxb, ryh, ryb);
      c = v[0];
    };
    auto acc = [&](int m, const T2 (&v)[5]) {
      T rxh, rxb, ryh, ryb;
      slopes5(v, rxh, rxb, ryh, ryb);
      store(m, rxh, rxb, ryh, ryb);
      const T2 c = v[0];
      T wn[5];
      wtab(P, m, wn);
      const T w0 = wn[0], w1 = wn[1], w2 = wn[2], w3 = wn[3], w4 = wn[4];
      a0 += w0 * c.x; a1 += w1 * c.x; a2 += w2 * c.x; a3 += w3 * c.x;
      ab0 += w0 * c.y; ab1 += w1 * c.y;
      x0 += w0 * rxh; x1 += w1 * rxh; x2 += w2 * rxh; x3 += w3 * rxh;
      xb0 += w0 * rxb; xb1 += w1 * rxb;
      y0 += w0 * ryh; y1 += w1 * ryh; y2 += w2 * ryh; y3 += w3 * ryh; y4 += w4 * ryh;
      yb0 += w0 * ryb; yb1 += w1 * ryb; yb2 += w2 * ryb;
    };
    // rows m0 .. m1-1 (loading the next row ahead of the arithmetic needs more registers
    // than the occupancy this latency-bound loop depends on: measured slower)
    auto rows = [&](int m0, int m1) {
#pragma unroll 1
      for (int m = m0; m < m1; m++) {
        T2 v[5];
        load5(m, v);
        acc(m, v);
      }
    };
    auto row_v0 = [&](int m) {  // v = 0: only the w_0 sums, half weight
      T rxh, rxb, ryh, ryb;
      T2 c;
      slopes_of(m, rxh, rxb, ryh, ryb, c);
      store(m, rxh, rxb, ryh, ryb);
      T wn[5];
      wtab(P, m, wn);
      const T hw = T(0.5) * wn[0];
      a0 += hw * c.x; ab0 += hw * c.y; x0 += hw * rxh; xb0 += hw * rxb; y0 += hw * ryh; yb0 += hw * ryb;
    };
    // close a half: its face sums (sy = -1: S side, +1: N side), then add it to the totals
    auto close = [&](T sy, T* side) {
      const T P0 = a0 + sy * y0, P1 = a1 + sy * y1, P2 = a2 + sy * y2, P3 = a3 + sy * y3;
      const T Pb0 = ab0 + sy * yb0, Pb1 = ab1 + sy * yb1;
      const T Z1 = cu * x1 + tdy * y2, Z2 = cu * x2 + tdy * y3, Z3 = cu * x3 + tdy * y4;
      const T Zb1 = cu * xb1 + tdy * yb2;
      finalize_y<T, T2>(u, wu, tdx, P0, P1, P2, P3, Pb0, Pb1, x0, x1, x2, xb0, Z1, Z2, Z3, Zb1, lane,
                        side);
      const T h[kSumsTotals + kHeatTotals] = {a0, a1, a2, ab0, x0, x1, x2, xb0, y0, y1, y2, y3, yb0, yb1,
                                              a3, ab1, x3, xb1};
#pragma unroll
      for (int t = 0; t < kSumsTotals + kHeatTotals; t++) tot[t * 128] += h[t];
      if (heat) {  // Shakhov: raw moments of the half's y-side face values (kHeatN / kHeatS)
        heat_side((double)wu, (double)u, (double)P0, (double)P1, (double)P2, (double)P3, (double)Pb0,
                  (double)Pb1, hsum + (sy > T(0) ? kHeatN : kHeatS));
      }
    };
    zero();
    rows(0, mneg);
    if (v0) row_v0(mneg);
    close(T(-1), wsum + kSumS);
    zero();
    if (v0) row_v0(mneg);
    rows(mpos, nv);
    close(T(1), wsum + kSumN);
    // x sides: E gets u > 0 (f + r_x), W gets u < 0 (f - r_x), u = 0 half to each.
    const T tA0 = tot[0], tA1 = tot[128], tA2 = tot[256], tAb = tot[384], tR0 = tot[512];
    const T tR1 = tot[640], tR2 = tot[768], tRb = tot[896], tC0 = tot[1024], tC1 = tot[1152];
    const T tC2 = tot[1280], tC3 = tot[1408], tCb0 = tot[1536], tCb1 = tot[1664];
    const T D0 = cu * tR0 + tdy * tC1, D1 = cu * tR1 + tdy * tC2, D2 = cu * tR2 + tdy * tC3;
    const T Db = cu * tRb + tdy * tCb1;
    const T hE = u > T(0) ? T(1) : (u < T(0) ? T(0) : T(0.5));
    const T hW = u < T(0) ? T(1) : (u > T(0) ? T(0) : T(0.5));
    T xv[32];
    const T uu = u * u;
#pragma unroll
    for (int sd = 0; sd < 2; sd++) {
      const T sg = sd == 0 ? T(1) : T(-1);
      const T wgt = wu * (sd == 0 ? hE : hW);
      const T F0 = tA0 + sg * tR0, F1 = tA1 + sg * tR1, F2 = tA2 + sg * tR2, Fb = tAb + sg * tRb;
      T* o = xv + 16 * sd;
      o[0] = wgt * F0;
      o[1] = wgt * u * F0;
      o[2] = wgt * F1;
      o[3] = wgt * (T(0.5) * (uu * F0 + F2) + T(0.5) * Fb);
      const T ws = wgt * tdy;
      o[4] = ws * tC0;
      o[5] = ws * u * tC0;
      o[6] = ws * tC1;
      o[7] = ws * (T(0.5) * (uu * tC0 + tC2) + T(0.5) * tCb0);
      const T wuu = wgt * u;
      o[8] = wuu * F0;
      o[9] = wuu * u * F0;
      o[10] = wuu * F1;
      o[11] = wuu * (T(0.5) * (uu * F0 + F2) + T(0.5) * Fb);
      o[12] = wuu * D0;
      o[13] = wuu * u * D0;
      o[14] = wuu * D1;
      o[15] = wuu * (T(0.5) * (uu * D0 + D2) + T(0.5) * Db);
    }
    const T r = warp_reduce_scatter<32>(xv, lane);
    wsum[kSumE + lane] += r;  // lanes 0..15: E side, 16..31: W side
    if (heat) {  // Shakhov: x-side face values and cell values (kHeatE, kHeatW, kHeatC)
      const double tA3 = (double)tot[1792], tAb1 = (double)tot[1920], tR3 = (double)tot[2048];
      const double tRb1 = (double)tot[2176];
      const double hE_ = (double)(wu * hE), hW_ = (double)(wu * hW), ud = (double)u;
      heat_side(hE_, ud, (double)(tA0 + tR0), (double)(tA1 + tR1), (double)(tA2 + tR2), tA3 + tR3,
                (double)(tAb + tRb), tAb1 + tRb1, hsum + kHeatE);
      heat_side(hW_, ud, (double)(tA0 - tR0), (double)(tA1 - tR1), (double)(tA2 - tR2), tA3 - tR3,
                (double)(tAb - tRb), tAb1 - tRb1, hsum + kHeatW);
      heat_cell((double)wu, ud, (double)tA0, (double)tA1, (double)tA2, tA3, (double)tAb, tAb1,
                hsum + kHeatC);
    }
  }
  __syncwarp();
  T* out = sums + (size_t)cell * kNSum;
  out[lane] = wsum[lane];
  out[lane + 32] = wsum[lane + 32];
  if (heat) {
    double* ho = P.hs + (size_t)cell * kNHeat;
    for (int t = lane; t < kNHeat; t += 32) ho[t] = hsum[t];
  }
}
template <typename T, typename T2>
__global__ void __launch_bounds__(128) k_sums(Params P, const T2* __restrict__ f,
                                              T* __restrict__ sums, T2* __restrict__ slopes) {
  extern __shared__ __align__(16) unsigned char smraw[];
  sums_body<T, T2>(P, f, sums, smraw, blockIdx.x, slopes);
}

// -------------------------------------------------------------------------------------
// Steps S2-S5 per interface, plus the coefficients of S6/S8 for the update kernel: all FP64
// in the FP64 form; first-order terms FP64 and slope-carrying terms FP32 in the FP32-f form.
// -------------------------------------------------------------------------------------

// Moments <x^n>, n = 0..6, of the normalised 1D Gaussian sqrt(lam/pi) exp(-lam (x-U)^2):
// full range, x > 0 and x < 0.  Integration by parts gives
// <x^{n+2}> = U <x^{n+1}> + (n+1)/(2 lam) <x^n> on every range.
// h = 1/(2 lam); the starting values come from gauss_half_start (FP64): the half-range
// masses mp0, mn0 and e = <x>_{x>0} - U mp0 = sqrt(lam/pi) exp(-lam U^2) / (2 lam).
template <typename T>
__device__ void gauss_moments7(T U, T h, T mp0, T mn0, T e, T* M, T* Mp, T* Mn) {
  M[0] = T(1);
  M[1] = U;
  Mp[0] = mp0;
  Mn[0] = mn0;
  Mp[1] = U * Mp[0] + e;
  Mn[1] = U * Mn[0] - e;
#pragma unroll
  for (int n = 0; n < 5; n++) {
    const T nh = T(n + 1) * h;
    M[n + 2] = U * M[n + 1] + nh * M[n];
    Mp[n + 2] = U * Mp[n + 1] + nh * Mp[n];
    Mn[n + 2] = U * Mn[n + 1] + nh * Mn[n];
  }
}
// One erfc: the half-range mass on the far side of U is erfc(sqrt(lam)|U|)/2, the near side
// 1 minus that; rl = 1/sqrt(lam).
__device__ __forceinline__ void gauss_half_start(double U, double lam, double rl, double& mp0, double& mn0,
                                                 double& e) {
  constexpr double kHalfRsqrtPi = 0.28209479177387814347;  // 1 / (2 sqrt(pi))
  const double sl = lam * rl;
  e = exp(-lam * U * U) * (kHalfRsqrtPi * rl);
  const double far = 0.5 * erfc(sl * fabs(U));
  mp0 = U >= 0.0 ? 1.0 - far : far;
  mn0 = U >= 0.0 ? far : 1.0 - far;
}

// Full-range moments only (tangential axis).
template <typename T>
__device__ void gauss_moments7_full(T U, T h, T* M) {
  M[0] = T(1);
  M[1] = U;
#pragma unroll
  for (int n = 0; n < 5; n++) M[n + 2] = U * M[n + 1] + T(n + 1) * h * M[n];
}

// <u^a v^b psi> for the normalised Maxwellian, u-moments Mu (one range), v-moments Mv,
// <xi^2> = X2.
template <typename T>
__device__ __forceinline__ void psi_mom(const T* Mu, const T* Mv, T X2, int a, int b, T* o) {
  o[0] = Mu[a] * Mv[b];
  o[1] = Mu[a + 1] * Mv[b];
  o[2] = Mu[a] * Mv[b + 1];
  o[3] = T(0.5) * (Mu[a + 2] * Mv[b] + Mu[a] * Mv[b + 2] + Mu[a] * Mv[b] * X2);
}
// <u^a v^b psi (c . psi)>, c . psi = c1 + c2 u + c3 v + c4 (u^2 + v^2 + xi^2)/2, from the
// factorised moments: with M(p, q) = Mu[p] Mv[q] and h = c4/2,
//   T(p, q) = <u^p v^q (c . psi)> = Mu[p] A(q) + Mu[p+1] c2 Mv[q] + Mu[p+2] h Mv[q],
//   A(q) = (c1 + h X2) Mv[q] + c3 Mv[q+1] + h Mv[q+2];
// the components are T(a, b), T(a+1, b), T(a, b+1), and for the energy
// (T(a+2, b) + T(a, b+2) + X2 T(a, b) + h (X4 - X2^2) M(a, b)) / 2, since
// <xi^2 (c . psi)> = X2 (c . psi with xi^2 -> X2) + h (X4 - X2^2).
// The tables A, B, C depend on (c, Mv, b) only and are shared by evaluations at several
// (Mu, a); X4m = X4 - X2^2.
template <typename T>
struct APsi {
  T A[3], B[3], C[3], h, mvb;
};
template <typename T>
__device__ __forceinline__ void apsi_prep(const T* Mv, T X2, int b, const T* c, APsi<T>& t) {
  t.h = T(0.5) * c[3];
  const T c0x = c[0] + t.h * X2;
#pragma unroll
  for (int q = 0; q < 3; q++) {
    t.A[q] = c0x * Mv[b + q] + c[2] * Mv[b + q + 1] + t.h * Mv[b + q + 2];
    t.B[q] = c[1] * Mv[b + q];
    t.C[q] = t.h * Mv[b + q];
  }
  t.mvb = Mv[b];
}
template <typename T>
__device__ __forceinline__ void apsi_eval(const APsi<T>& t, const T* Mu, T X2, T X4m, int a, T* o) {
  auto Tm = [&](int p, int q) { return Mu[a + p] * t.A[q] + Mu[a + p + 1] * t.B[q] + Mu[a + p + 2] * t.C[q]; };
  const T t00 = Tm(0, 0);
  o[0] = t00;
  o[1] = Tm(1, 0);
  o[2] = Tm(0, 1);
  o[3] = T(0.5) * (Tm(2, 0) + Tm(0, 2) + X2 * t00 + t.h * X4m * (Mu[a] * t.mvb));
}

// q = (K+2)/(4 lam) is the mean internal plus thermal energy per unit mass, c4 = lam/q.
template <typename T>
__device__ void micro_slope(T U, T V, T lam, T q, T c4, const T* s, T* a) {
  const T a4 = c4 * (T(2) * s[3] - T(2) * (U * s[1] + V * s[2]) + s[0] * (U * U + V * V - T(2) * q));
  const T a3 = T(2) * lam * (s[2] - V * s[0]) - V * a4;
  const T a2 = T(2) * lam * (s[1] - U * s[0]) - U * a4;
  const T a1 = s[0] - U * a2 - V * a3 - a4 * (T(0.5) * (U * U + V * V) + q);
  a[0] = a1;
  a[1] = a2;
  a[2] = a3;
  a[3] = a4;
}

// 1/n! as a constant expression (the loops that use it are unrolled).
__host__ __device__ constexpr double inv_factorial(int n) {
  double f = 1.0;
  for (int k = 2; k <= n; k++) f *= k;
  return 1.0 / f;
}

// Time integrals over one step of the Eq. 2 weights, x = dt/tau:
//   Mt1 = dt c1, Mt2 = dt^2 c2, Mt3 = dt^2 c3, Mt4 = dt c4, Mt5 = dt^2 c5
//   c4 = (1-e^{-x})/x, c1 = 1-c4, c5 = (c4-e^{-x})/x, c3 = 1/2 - c1/x, c2 = c5 - c1/x.
// Below x = 0.1 they come from the functions phi_k(y) = sum_n y^n/(n+k)! at y = -x (the
// exponential-integrator phi functions, phi_k = 1/k! + y phi_{k+1}): phi_3 by its power series
// (Horner, NT terms), then phi_2 = 1/2 - x phi_3 and phi_1 = 1 - x phi_2, none of which
// cancels for x < 0.1; in terms of them c4 = phi_1, c1 = x phi_2, c3 = x phi_3,
// c5 = sum (n+1) y^n/(n+2)! = phi_1 - phi_2 and c2 = -x sum (n+1) y^n/(n+3)! =
// -x (phi_2 - 2 phi_3), since (n+1)/(n+2)! = 1/(n+1)! - 1/(n+2)! and
// (n+1)/(n+3)! = 1/(n+2)! - 2/(n+3)!.
template <int NT>
__device__ __forceinline__ double phi3_series(double y) {
  double h = 0.0;
#pragma unroll
  for (int n = NT - 1; n >= 0; n--) h = h * y + inv_factorial(n + 3);
  return h;
}
__device__ void time_weights(double dt, double x, double* Mt) {
  double c1, c2, c3, c4, c5;
  if (x < 0.1) {
    // 8 terms below x = 0.01, 12 below 0.1: the first term left out is below 1e-23 of phi_3
    const double p3 = x < 0.01 ? phi3_series<8>(-x) : phi3_series<12>(-x);
    const double p2 = 0.5 - x * p3, p1 = 1.0 - x * p2;
    c4 = p1; c5 = p1 - p2; c1 = x * p2; c3 = x * p3; c2 = -x * (p2 - 2.0 * p3);
  } else {
    const double e = exp(-x), em = -expm1(-x), ix = 1.0 / x;
    c4 = em * ix;
    c1 = 1.0 - c4;
    c5 = (c4 - e) * ix;
    c3 = 0.5 - c1 * ix;
    c2 = c5 - c1 * ix;
  }
  Mt[0] = dt * c1;
  Mt[1] = dt * dt * c2;
  Mt[2] = dt * dt * c3;
  Mt[3] = dt * c4;
  Mt[4] = dt * dt * c5;
}
// Polynomial of (a . psi) g / g_h reduced over the internal variable, in the face frame:
// P(un, ut) = p0 + p1 un + p2 ut + p3 (un^2 + ut^2); component h or b.
__device__ __forceinline__ void shape_h(const double* a, double X2, double* p) {
  p[0] = a[0] + 0.5 * a[3] * X2;
  p[1] = a[1];
  p[2] = a[2];
  p[3] = 0.5 * a[3];
}
__device__ __forceinline__ void shape_b(const double* a, double X2, double X4, double* p) {
  p[0] = a[0] * X2 + 0.5 * a[3] * X4;
  p[1] = a[1] * X2;
  p[2] = a[2] * X2;
  p[3] = 0.5 * a[3] * X2;
}
__device__ __forceinline__ void qcoef(double M1, double Mt2, double Mt3, const double* pa,
                                      const double* pb, const double* pA, double* c) {
  c[0] = M1 + Mt3 * pA[0];
  c[1] = Mt3 * pA[1] + Mt2 * pa[0];
  c[2] = Mt3 * pA[2] + Mt2 * pb[0];
  c[3] = Mt3 * pA[3] + Mt2 * pa[1];
  c[4] = Mt2 * (pa[2] + pb[1]);
  c[5] = Mt3 * pA[3] + Mt2 * pb[2];
  c[6] = Mt2 * pa[3];
  c[7] = Mt2 * pb[3];
}

// FP32 record of a diffuse-wall face (see FaceRecF): no polynomial terms; the wall
// Maxwellian g_w = G_w exp(-lam |c - U_w|^2) enters as its exponent relative to g_ref's
// (log2 units, formed in FP64), so that the walk forms g_w - g_ref without cancellation;
// global velocity frame (y faces: un = v).
__device__ __forceinline__ void wall_face_f32(const Params& P, bool isx, double X2, double lam, double Ut, double G,
                              int wall, FaceRecF& RF) {
  constexpr double kLog2e = 1.4426950408889634;
#pragma unroll
  for (int sd = 0; sd < 2; sd++) {
#pragma unroll
    for (int c = 0; c < 8; c++) RF.Q[sd][c] = 0.f;
    RF.K[sd][0] = RF.K[sd][1] = RF.K[sd][2] = 0.f;
    RF.K[sd][3] = (float)X2;
  }
  const double Ux = isx ? 0.0 : Ut, Vy = isx ? Ut : 0.0;
  // (a wall density rho_w <= 0 only arises from a state that is already unphysical; it is
  // clamped so that the record stays finite, and the FP64 W update reports the failure)
  RF.E[0] = (float)((log2(fmax(G, 1e-300)) - lam * (Ux * Ux + Vy * Vy) * kLog2e) - P.ref_E[0]);
  RF.E[1] = (float)(2.0 * lam * Ux * kLog2e - P.ref_E[1]);
  RF.E[2] = (float)(2.0 * lam * Vy * kLog2e - P.ref_E[2]);
  RF.E[3] = (float)(-lam * kLog2e - P.ref_E[3]);
  RF.Mt4 = (float)P.dt;
  RF.nMt5 = 0.f;
  RF.wall = (float)wall;
  RF.gdt = (float)P.dt;
  RF.pad[0] = RF.pad[1] = RF.pad[2] = RF.pad[3] = 0.f;
}

// S2-S5 of one UGKS interface in the face frame (un, ut): interface primitive variables,
// Maxwellian moments (full and half range), collision time and Mt1..Mt5, the micro slopes
// a_L, a_R, b and the time slope A (compatibility condition), and the time-integrated
// macroscopic flux F (equilibrium part from analytic moments, free-transport part from the
// sums).  Inputs: the interface sums (S1, S7) and the cell W on both sides.
// Arithmetic: the primitive variables, exp and erfc of the half-range moments, tau and
// Mt1..Mt5, the slope targets and the free-transport part of F in FP64; the moment
// recurrences, the micro-slope solves, the compatibility moments and the equilibrium part of
// F in T: double (FP64 form) or dd, double-FP32 on the FP32 pipe (FP32-f and DF64 forms,
// about 2^-48 relative per operation, where FP64 would spend ~420 of its ~610 operations per
// face on the 1/64-rate FP64 pipe).
template <typename T>
struct FaceCoreT {
  double rho, U, V, lam, X2, X4;
  double Mt[5];
  T aL[4], aR[4], b[4], A[4];
  // Shakhov model: S_h and S_b on the face-frame monomials un^a ut^b (a + b <= 3), and the
  // coefficients of alpha L = alpha (c.q) (for the FP32 record's b terms)
  bool shk;
  double sh[4][4], sb[4][4], aLq[3];
};

// Heat flux (qn, qt) about (U, V) from the raw moments of a distribution (face frame):
// M[a][b] = sum w un^a ut^b h for a + b <= 3, B00 B10 B01 = sum w (1, un, ut) b;
// q = 1/2 sum w c (|c|^2 h + b), c = (un - U, ut - V).
__device__ __forceinline__ void heat_flux_of(const double (&M)[4][4], double B00, double B10, double B01,
                                             double U, double V, double* q) {
  const double cn3 = M[3][0] - 3.0 * U * M[2][0] + 3.0 * U * U * M[1][0] - U * U * U * M[0][0];
  const double cnt2 = M[1][2] - 2.0 * V * M[1][1] + V * V * M[1][0] - U * M[0][2] + 2.0 * U * V * M[0][1] -
                      U * V * V * M[0][0];
  const double ct3 = M[0][3] - 3.0 * V * M[0][2] + 3.0 * V * V * M[0][1] - V * V * V * M[0][0];
  const double ctn2 = M[2][1] - 2.0 * U * M[1][1] + U * U * M[0][1] - V * M[2][0] + 2.0 * U * V * M[1][0] -
                      U * U * V * M[0][0];
  q[0] = 0.5 * (cn3 + cnt2 + (B10 - U * B00));
  q[1] = 0.5 * (ct3 + ctn2 + (B01 - V * B00));
}

// Shakhov factors on monomials of the face frame: alpha L R with L = qn cn + qt ct and
// R = 2 lam (cn^2 + ct^2) + r0 (r0 = -4 for S_h, -2 for S_b / X2), cn = un - U, ct = ut - V.
__device__ __forceinline__ void shakhov_poly(double alpha, double U, double V, double lam, const double* q,
                                             double r0, double (&p)[4][4]) {
  const double l[3] = {-(q[0] * U + q[1] * V), q[0], q[1]};  // 1, un, ut
  double r[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};        // r[a][b]: un^a ut^b
  r[0][0] = 2.0 * lam * (U * U + V * V) + r0;
  r[1][0] = -4.0 * lam * U;
  r[0][1] = -4.0 * lam * V;
  r[2][0] = 2.0 * lam;
  r[0][2] = 2.0 * lam;
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) p[a][b] = 0.0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; a + b < 3; b++) {
      p[a][b] += alpha * l[0] * r[a][b];
      p[a + 1][b] += alpha * l[1] * r[a][b];
      p[a][b + 1] += alpha * l[2] * r[a][b];
    }
}
using FaceCore = FaceCoreT<double>;
template <typename T>
__device__ __forceinline__ void face_core(const Params& P, const double* W0, const double* St,
                                          const double* Sf, const double* Ss, const double* WL,
                                          const double* WR, double tdelta, double* F, FaceCoreT<T>& c,
                                          const double* qsh = nullptr) {
  const int K = P.K;
  // S2: interface primitive variables and Maxwellian moments
  const double rho = W0[0], irho = rcp_nr(rho), U = W0[1] * irho, V = W0[2] * irho;
  const double ilam4 = (W0[3] - 0.5 * rho * (U * U + V * V)) * irho * P.inv_kp2;  // 1/(4 lam)
  const double lam = 0.25 * rcp_nr(ilam4);
  const double h = 2.0 * ilam4;  // 1/(2 lam)
  const double rl = rsqrt(lam);
  double mp0, mn0, e;
  gauss_half_start(U, lam, rl, mp0, mn0, e);
  const T Ut = T(U), Vt = T(V), ht = T(h);
  T Mu[7], Mup[7], Mun[7], Mv[7];
  gauss_moments7<T>(Ut, ht, T(mp0), T(mn0), T(e), Mu, Mup, Mun);
  gauss_moments7_full<T>(Vt, ht, Mv);
  const double X2 = 2.0 * K * ilam4, X4 = (K * K + 2.0 * K) * 4.0 * ilam4 * ilam4;
  const T X2t = T(X2), X4m = T(X4 - X2 * X2);
  // S3: collision time tau = mu/p, mu = mu_ref T^omega, p = rho/(2 lam), and Mt1..Mt5 of
  // x = dt/tau (omega = 1/2: x = dt rho / (2 mu_ref sqrt(lam)))
  const double x = P.omega_half ? P.half_dt_mu * rho * rl : P.dt / collision_time(P, rho, lam);
  time_weights(P.dt, x, c.Mt);
  const double* Mt = c.Mt;
  // S4: micro slopes
  const double inv = irho * tdelta;
  const T lamt = T(lam), q = T((K + 2) * ilam4), c4 = T(4.0 * lam * lam * P.inv_kp2);
  T sL[4], sR[4], sT[4], sA[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    sL[k] = T((W0[k] - WL[k]) * inv);
    sR[k] = T((WR[k] - W0[k]) * inv);
    sT[k] = T(St[k] * irho);
  }
  micro_slope<T>(Ut, Vt, lamt, q, c4, sL, c.aL);
  micro_slope<T>(Ut, Vt, lamt, q, c4, sR, c.aR);
  micro_slope<T>(Ut, Vt, lamt, q, c4, sT, c.b);
  // moments of (u_n a_L, u_n a_R, u_t b) . psi g at the orders the compatibility condition
  // (t) and the flux (n: one more u_n) need; each table is dropped once evaluated
  T t1[4], t2[4], t3[4], n1[4], n2[4], n3[4], t4[4], p1[4];
  {
    APsi<T> tL;
    apsi_prep<T>(Mv, X2t, 0, c.aL, tL);
    apsi_eval<T>(tL, Mup, X2t, X4m, 1, t1);
    apsi_eval<T>(tL, Mup, X2t, X4m, 2, n1);
  }
  {
    APsi<T> tR;
    apsi_prep<T>(Mv, X2t, 0, c.aR, tR);
    apsi_eval<T>(tR, Mun, X2t, X4m, 1, t2);
    apsi_eval<T>(tR, Mun, X2t, X4m, 2, n2);
  }
  {
    APsi<T> tb;
    apsi_prep<T>(Mv, X2t, 1, c.b, tb);
    apsi_eval<T>(tb, Mu, X2t, X4m, 0, t3);
    apsi_eval<T>(tb, Mu, X2t, X4m, 1, n3);
  }
#pragma unroll
  for (int k = 0; k < 4; k++) sA[k] = -(t1[k] + t2[k] + t3[k]);
  micro_slope<T>(Ut, Vt, lamt, q, c4, sA, c.A);
  {
    APsi<T> tA;
    apsi_prep<T>(Mv, X2t, 0, c.A, tA);
    apsi_eval<T>(tA, Mu, X2t, X4m, 1, t4);
  }
  // S5: equilibrium part of the macroscopic flux; S7 free transport part from the sums
  psi_mom<T>(Mu, Mv, X2t, 1, 0, p1);
  const T M1 = T(Mt[0]), M2 = T(Mt[1]), M3 = T(Mt[2]), rhot = T(rho);
#pragma unroll
  for (int k = 0; k < 4; k++)
    F[k] = to_double(rhot * (M1 * p1[k] + M2 * (n1[k] + n2[k] + n3[k]) + M3 * t4[k])) + Mt[3] * Sf[k] -
           Mt[4] * Ss[k];
  c.rho = rho;
  c.U = U;
  c.V = V;
  c.lam = lam;
  c.X2 = X2;
  c.X4 = X4;
  // Shakhov model: the zeroth-order equilibrium term g0 (1 + S) of the integral solution
  // (weight Mt1): its part of the macroscopic flux from analytic full-range moments (FP64)
  c.shk = qsh != nullptr;
  if (c.shk) {
    const double alpha = P.shk_c * lam * lam * irho;
    shakhov_poly(alpha, U, V, lam, qsh, -4.0, c.sh);
    shakhov_poly(alpha * X2, U, V, lam, qsh, -2.0, c.sb);
    c.aLq[0] = -alpha * (qsh[0] * U + qsh[1] * V);
    c.aLq[1] = alpha * qsh[0];
    c.aLq[2] = alpha * qsh[1];
    double Mu[7], Mv[7];
    gauss_moments7_full<double>(U, h, Mu);
    gauss_moments7_full<double>(V, h, Mv);
    double e[4] = {0.0, 0.0, 0.0, 0.0};
    for (int a = 0; a < 4; a++)
      for (int b = 0; a + b < 4; b++) {
        const double ph = c.sh[a][b], pb = c.sb[a][b];
        e[0] += ph * Mu[a + 1] * Mv[b];
        e[1] += ph * Mu[a + 2] * Mv[b];
        e[2] += ph * Mu[a + 1] * Mv[b + 1];
        e[3] += 0.5 * (ph * (Mu[a + 3] * Mv[b] + Mu[a + 1] * Mv[b + 2]) + pb * Mu[a + 1] * Mv[b]);
      }
    for (int k = 0; k < 4; k++) F[k] += rho * Mt[0] * e[k];
  }
}

// FP64 form (T = double) and DF64 form (T = dd: the interface's polynomial work in
// double-FP32, as in the FP32-f form, then the record's coefficients in FP64): the interface
// (face_core) and its FP64 micro-flux record (the DF64 form splits it into pairs).
template <typename T>
__device__ void face_math(const Params& P, const double* W0, const double* St, const double* Sf,
                          const double* Ss, const double* WL, const double* WR, double tdelta,
                          bool isx, double* F, FaceRec& R, const double* qsh = nullptr) {
  FaceCoreT<T> c;
  face_core<T>(P, W0, St, Sf, Ss, WL, WR, tdelta, F, c, qsh);
  double aL[4], aR[4], bs[4], As[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    aL[k] = to_double(c.aL[k]);
    aR[k] = to_double(c.aR[k]);
    bs[k] = to_double(c.b[k]);
    As[k] = to_double(c.A[k]);
  }
  const double* Mt = c.Mt;
  const double X2 = c.X2, X4 = c.X4;
  R.G = c.rho * c.lam / kPi;
  R.Un = c.U;
  R.Ut = c.V;
  R.lam = c.lam;
  R.Mt4 = Mt[3];
  R.Mt5 = Mt[4];
  R.bfac = X2;
  R.wall = 0;
  // S6/S8 coefficients (FP64 record)
  double pa[4], pb[4], pA[4];
  for (int sd = 0; sd < 2; sd++) {
    const double* as = sd == 0 ? aL : aR;
    shape_h(as, X2, pa);
    shape_h(bs, X2, pb);
    shape_h(As, X2, pA);
    qcoef(Mt[0], Mt[1], Mt[2], pa, pb, pA, R.Q[sd][0]);
    shape_b(as, X2, X4, pa);
    shape_b(bs, X2, X4, pb);
    shape_b(As, X2, X4, pA);
    qcoef(Mt[0] * X2, Mt[1], Mt[2], pa, pb, pA, R.Q[sd][1]);
    if (c.shk) {  // Shakhov: Mt1 g0 S on (1, un, ut, un^2, un ut, ut^2, un r2, ut r2)
      for (int comp = 0; comp < 2; comp++) {
        const double(&p)[4][4] = comp == 0 ? c.sh : c.sb;
        double* q = R.Q[sd][comp];
        q[0] += Mt[0] * p[0][0];
        q[1] += Mt[0] * p[1][0];
        q[2] += Mt[0] * p[0][1];
        q[3] += Mt[0] * p[2][0];
        q[4] += Mt[0] * p[1][1];
        q[5] += Mt[0] * p[0][2];
        q[6] += Mt[0] * p[3][0];  // = p[1][2]: the cubic part is (qn un + qt ut) 2 lam r2
        q[7] += Mt[0] * p[0][3];  // = p[2][1]
      }
    }
  }
}

// FP32-f form: the interface (face_core with its polynomial work in double-FP32: primitive
// variables, half-range moments, Mt1..Mt5, micro-slope solves, compatibility condition,
// macroscopic flux), then the FP32 record its update walk reads.  The record is rounded to
// FP32 from the double-FP32 slopes and FP64 weights (f32_rn: on the integer pipe, not the
// 1/64-rate FP64 pipe the conversion instruction runs on): the walk applies it to FP32 f.
__device__ __forceinline__ void face_math_f32(const Params& P, const double* W0, const double* St,
                                              const double* Sf, const double* Ss, const double* WL,
                                              const double* WR, double tdelta, bool isx, double* F,
                                              double& Mt4, FaceRecF& RF, const double* qsh = nullptr) {
  FaceCoreT<dd> c;
  face_core<dd>(P, W0, St, Sf, Ss, WL, WR, tdelta, F, c, qsh);
  const double* Mt = c.Mt;
  Mt4 = Mt[3];
  const float fM1 = f32_rn(Mt[0]), fM2 = f32_rn(Mt[1]), fM3 = f32_rn(Mt[2]);
  const float fX2 = f32_rn(c.X2);
  const float fG = f32_rn(c.rho * c.lam / kPi);
  const float kap = f32_rn(0.5 * (c.X4 - c.X2 * c.X2));  // (X4 - X2^2)/2 = K/(4 lam^2)
  float aL[4], aR[4], b[4], A[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    aL[k] = to_float(c.aL[k]);
    aR[k] = to_float(c.aR[k]);
    b[k] = to_float(c.b[k]);
    A[k] = to_float(c.A[k]);
  }
  // shape polynomial of (a . psi) g / g_h reduced over the internal variable, face frame:
  // P(un, ut) = p0 + p1 un + p2 ut + p3 (un^2 + ut^2)
  auto shape = [&](const float* a4, float* o) {
    o[0] = fmaf(0.5f * a4[3], fX2, a4[0]);
    o[1] = a4[1];
    o[2] = a4[2];
    o[3] = 0.5f * a4[3];
  };
  float pb[4], pA[4];
  shape(b, pb);
  shape(A, pA);
  constexpr int py[8] = {0, 2, 1, 5, 4, 3, 7, 6};
#pragma unroll
  for (int sd = 0; sd < 2; sd++) {
    const float* as = sd == 0 ? aL : aR;
    float pa[4], Qf[8];
    shape(as, pa);
    // Q_h on (1, un, ut, un^2, un ut, ut^2, un r2, ut r2)
    Qf[0] = fmaf(fM3, pA[0], fM1);
    Qf[1] = fmaf(fM3, pA[1], fM2 * pa[0]);
    Qf[2] = fmaf(fM3, pA[2], fM2 * pb[0]);
    Qf[3] = fmaf(fM3, pA[3], fM2 * pa[1]);
    Qf[4] = fM2 * (pa[2] + pb[1]);
    Qf[5] = fmaf(fM3, pA[3], fM2 * pb[2]);
    Qf[6] = fM2 * pa[3];
    Qf[7] = fM2 * pb[3];
    if (c.shk) {  // Shakhov: Mt1 g0 S_h on the face-frame monomials (FP64 sums, then FP32)
      const double* M = Mt;
      Qf[0] += (float)(M[0] * c.sh[0][0]);
      Qf[1] += (float)(M[0] * c.sh[1][0]);
      Qf[2] += (float)(M[0] * c.sh[0][1]);
      Qf[3] += (float)(M[0] * c.sh[2][0]);
      Qf[4] += (float)(M[0] * c.sh[1][1]);
      Qf[5] += (float)(M[0] * c.sh[0][2]);
      Qf[6] += (float)(M[0] * c.sh[3][0]);
      Qf[7] += (float)(M[0] * c.sh[0][3]);
    }
#pragma unroll
    for (int k = 0; k < 8; k++) RF.Q[sd][k] = fG * (isx ? Qf[k] : Qf[py[k]]);
    // b polynomial: P_b(a) = X2 P_h(a) + a4 (X4 - X2^2)/2, so Q_b = X2 Q_h + kap (Mt3 A4 +
    // Mt2 un a4 + Mt2 ut b4)
    const float k0 = fG * kap * fM3 * A[3], kn = fG * kap * fM2 * as[3], kt = fG * kap * fM2 * b[3];
    RF.K[sd][0] = k0;
    RF.K[sd][1] = isx ? kn : kt;
    RF.K[sd][2] = isx ? kt : kn;
    RF.K[sd][3] = fX2;
    if (c.shk) {  // Shakhov: S_b = X2 S_h + 2 X2 alpha L, the second part linear in (un, ut)
      const double m = 2.0 * Mt[0] * c.X2 * (c.rho * c.lam / kPi);
      RF.K[sd][0] += (float)(m * c.aLq[0]);
      RF.K[sd][1] += (float)(m * (isx ? c.aLq[1] : c.aLq[2]));
      RF.K[sd][2] += (float)(m * (isx ? c.aLq[2] : c.aLq[1]));
    }
  }
  constexpr double kLog2e = 1.4426950408889634;
  const double lam = c.lam, Ux = isx ? c.U : c.V, Vy = isx ? c.V : c.U;
  RF.E[0] = f32_rn(-lam * (Ux * Ux + Vy * Vy) * kLog2e);
  RF.E[1] = f32_rn(2.0 * lam * Ux * kLog2e);
  RF.E[2] = f32_rn(2.0 * lam * Vy * kLog2e);
  RF.E[3] = f32_rn(-lam * kLog2e);
  RF.Mt4 = f32_rn(Mt[3]);
  RF.nMt5 = f32_rn(-Mt[4]);
  RF.wall = 0.f;
  RF.gdt = 0.f;
  RF.pad[0] = RF.pad[1] = RF.pad[2] = RF.pad[3] = 0.f;
}

// Record kind written for the update kernels: FP64 FaceRec (FP64 form), FP32 FaceRecF
// (FP32-f form), double-FP32 FaceRecD (DF64 form).  Every form's sums are FP64.
enum { kRecF64 = 0, kRecF32 = 1, kRecDF = 2 };

__device__ __forceinline__ float2 split_df(double a) {
  float2 r;
  split_f64(a, r.x, r.y);
  return r;
}
__device__ __forceinline__ void face_rec_df(const FaceRec& R, FaceRecD& D) {
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++)
#pragma unroll
      for (int c = 0; c < 8; c++) D.Q[a][b][c] = split_df(R.Q[a][b][c]);
  D.G = split_df(R.G);
  D.Un = split_df(R.Un);
  D.Ut = split_df(R.Ut);
  D.lam = split_df(R.lam);
  D.Mt4 = split_df(R.Mt4);
  D.Mt5 = split_df(R.Mt5);
  D.bfac = split_df(R.bfac);
  D.wall = R.wall;
  D.pad = 0;
}

// rx, ry: the x- and y-face records of kind REC (FaceRec, FaceRecF or FaceRecD).
// SHK: the Shakhov model's interface heat flux and terms (a separate instance, so that the
// BGK interface carries none of their code).
template <int REC, bool SHK = false>
__device__ __forceinline__ void faces_body(const Params& P, const double* __restrict__ sums,
                                           const double* __restrict__ W, int nwe,
                                           void* __restrict__ rx, void* __restrict__ ry,
                                           double* __restrict__ Fx, double* __restrict__ Fy,
                                           double* __restrict__ mt4, int t) {
  const int nx = P.nx, ny = P.ny;
  const int nfx = (nx + 1) * ny, nfy = nx * (ny + 1);
  if (t >= nfx + nfy) return;
  const bool isx = t < nfx;
  int i, j, cL, cR, oL, oR, wall = 0, side = 0;
  double tdelta;
  if (isx) {
    j = t / (nx + 1);
    i = t % (nx + 1) - 1;
    cL = wcell(P, i, j);
    cR = wcell(P, i + 1, j);
    oL = kSumE;
    oR = kSumW;
    tdelta = P.d_tdx;
    if (i == -1 && P.bc_kind[0] == 1) { wall = 1; side = 0; }
    if (i == nx - 1 && P.bc_kind[1] == 1) { wall = 2; side = 1; }
  } else {
    const int t2 = t - nfx;
    j = t2 / nx - 1;
    i = t2 % nx;
    cL = wcell(P, i, j);
    cR = wcell(P, i, j + 1);
    oL = kSumN;
    oR = kSumS;
    tdelta = P.d_tdy;
    if (j == -1 && P.bc_kind[2] == 1) { wall = 1; side = 2; }
    if (j == ny - 1 && P.bc_kind[3] == 1) { wall = 2; side = 3; }
  }
  FaceRec R;
  FaceRecF RF;
  constexpr bool f32 = REC == kRecF32;
  double F[4];
  if (wall) {
    // diffuse wall: incoming half range from the gas cell's sums, outgoing wall Maxwellian
    // with the density that cancels the mass flux; first order in time
    const int oin = wall == 1 ? oR : oL;
    const double* Se = wall == 1 ? sums + (size_t)cR * kNSum + oR + kOffSf
                                 : sums + (size_t)cL * kNSum + oL + kOffSf;
    double Sin[4];
#pragma unroll
    for (int c = 0; c < 4; c++) Sin[c] = Se[c] + P.refsum[oin / 16][kOffSf + c];
    const double rhow = -Sin[0] / P.wall_mom[side][0];
#pragma unroll
    for (int c = 0; c < 4; c++) F[c] = P.dt * (Sin[c] + rhow * P.wall_mom[side][c]);
    const double lam = 1.0 / P.bc_T[side];
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++)
        for (int c = 0; c < 8; c++) R.Q[a][b][c] = 0.0;
    R.G = rhow * lam / kPi;
    R.Un = 0.0;
    R.Ut = P.bc_U[side];
    R.lam = lam;
    R.Mt4 = P.dt;
    R.Mt5 = 0.0;
    R.bfac = P.K / (2.0 * lam);
    R.wall = wall;
    if (f32) wall_face_f32(P, isx, R.bfac, lam, R.Ut, R.G, wall, RF);
  } else {
    const int pm[4] = {0, isx ? 1 : 2, isx ? 2 : 1, 3};  // natural -> face frame
    const double* sL = sums + (size_t)cL * kNSum + oL;
    const double* sR = sums + (size_t)cR * kNSum + oR;
    double W0[4], St[4], Sf[4], Ss[4], WL[4], WR[4], Fr[4];
    const double* rp = P.refpair[isx ? 0 : 1];  // g_ref sums of both sides (FP32-f form)
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const int s = pm[c];
      W0[c] = (sL[kOffW0 + s] + sR[kOffW0 + s]) + rp[s];
      Sf[c] = (sL[kOffSf + s] + sR[kOffSf + s]) + rp[4 + s];
      St[c] = sL[kOffSt + s] + sR[kOffSt + s];
      Ss[c] = sL[kOffSs + s] + sR[kOffSs + s];
      WL[c] = W[s * nwe + cL];
      WR[c] = W[s * nwe + cR];
    }
    // Shakhov model: heat flux of the interface values about the interface velocity, from
    // the raw moments of both sides' face values (face frame), plus those of g_ref (FP32-f)
    double qsh[2];
    const double* qp = nullptr;
    if constexpr (SHK) {
      const int hL = isx ? kHeatE : kHeatN, hR = isx ? kHeatW : kHeatS;
      const double* a = P.hs + (size_t)cL * kNHeat + hL;
      const double* b = P.hs + (size_t)cR * kNHeat + hR;
      const double* ra = P.refheat[hL / 10];
      const double* rb = P.refheat[hR / 10];
      double n[10];  // natural frame: M20 M11 M02 M30 M21 M12 M03 B00 B10 B01
      for (int t = 0; t < 10; t++) n[t] = (a[t] + b[t]) + (ra[t] + rb[t]);
      double M[4][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
      M[0][0] = W0[0];
      M[1][0] = W0[1];
      M[0][1] = W0[2];
      // face frame: (un, ut) = (u, v) on x faces, (v, u) on y faces
      M[2][0] = isx ? n[0] : n[2];
      M[1][1] = n[1];
      M[0][2] = isx ? n[2] : n[0];
      M[3][0] = isx ? n[3] : n[6];
      M[2][1] = isx ? n[4] : n[5];
      M[1][2] = isx ? n[5] : n[4];
      M[0][3] = isx ? n[6] : n[3];
      const double B00 = n[7], B10 = isx ? n[8] : n[9], B01 = isx ? n[9] : n[8];
      heat_flux_of(M, B00, B10, B01, W0[1] / W0[0], W0[2] / W0[0], qsh);
      qp = qsh;
    }
    if constexpr (f32)
      face_math_f32(P, W0, St, Sf, Ss, WL, WR, tdelta, isx, Fr, R.Mt4, RF, qp);
    else if constexpr (REC == kRecDF)
      face_math<dd>(P, W0, St, Sf, Ss, WL, WR, tdelta, isx, Fr, R, qp);
    else
      face_math<double>(P, W0, St, Sf, Ss, WL, WR, tdelta, isx, Fr, R, qp);
#pragma unroll
    for (int c = 0; c < 4; c++) F[c] = (c == 1 || c == 2) && !isx ? Fr[3 - c] : Fr[c];
  }
  mt4[t] = R.Mt4;
  const int r = isx ? t : t - nfx;
  void* dst = isx ? rx : ry;
  if constexpr (REC == kRecF32) {
    static_cast<FaceRecF*>(dst)[r] = RF;
  } else if constexpr (REC == kRecDF) {
    FaceRecD D;
    face_rec_df(R, D);
    static_cast<FaceRecD*>(dst)[r] = D;
  } else {
    static_cast<FaceRec*>(dst)[r] = R;
  }
  if (isx) {
    for (int c = 0; c < 4; c++) Fx[4 * (size_t)t + c] = F[c];
  } else {
    for (int c = 0; c < 4; c++) Fy[4 * (size_t)(t - nfx) + c] = F[c];
  }
}
// FP64 form (REC = kRecF64) and DF64 form (REC = kRecDF)
template <int REC>
__global__ void __launch_bounds__(128, REC == kRecDF ? 4 : 3) k_faces(Params P, const double* __restrict__ sums, const double* __restrict__ W,
                        int nwe, void* __restrict__ rx, void* __restrict__ ry,
                        double* __restrict__ Fx, double* __restrict__ Fy, double* __restrict__ mt4) {
  if (P.shk)
    faces_body<REC, true>(P, sums, W, nwe, rx, ry, Fx, Fy, mt4, blockIdx.x * blockDim.x + threadIdx.x);
  else
    faces_body<REC, false>(P, sums, W, nwe, rx, ry, Fx, Fy, mt4, blockIdx.x * blockDim.x + threadIdx.x);
}


// -------------------------------------------------------------------------------------
// Eq. 4 per cell, plus g^n, g^{n+1}, tau^n, tau^{n+1} for Eq. 3, residual partials and
// the numerical-failure flag.
// -------------------------------------------------------------------------------------
// Records written: crf (FP32-f form) if set, else crd (DF64 form) if set, else cr (FP64).
__device__ __forceinline__ void cells_body(const Params& P, const double* __restrict__ Win,
                                           double* __restrict__ Wout, int nwe,
                                           const double* __restrict__ Fx,
                                           const double* __restrict__ Fy, CellRec* __restrict__ cr,
                                           double* __restrict__ rpart, int* __restrict__ err,
                                           CellRecF* __restrict__ crf,
                                           const double* __restrict__ mt4, double (*red)[128],
                                           int bx, CellRecD* __restrict__ crd = nullptr) {
  const int c = bx * blockDim.x + threadIdx.x;
  const int nx = P.nx, nc = P.nx * P.ny;
  double d2[4] = {0, 0, 0, 0}, am[4] = {0, 0, 0, 0};
  if (c < nc) {
    const int i = c % nx, j = c / nx;
    const size_t xw = (size_t)j * (nx + 1) + i, xe = xw + 1;
    const size_t ys = (size_t)j * nx + i, yn = (size_t)(j + 1) * nx + i;
    const int w = wcell(P, i, j);
    double Wn[4], W1[4];
    for (int k = 0; k < 4; k++) {
      Wn[k] = Win[k * nwe + w];
      W1[k] = Wn[k] + (Fx[4 * xw + k] - Fx[4 * xe + k]) * P.d_idx + (Fy[4 * ys + k] - Fy[4 * yn + k]) * P.d_idy;
      Wout[k * nwe + w] = W1[k];
      d2[k] = (W1[k] - Wn[k]) * (W1[k] - Wn[k]);
      am[k] = fabs(W1[k]);
    }
    const int K = P.K;
    // 1/lam = 4 (rho E - rho |U|^2 / 2) / ((K + 2) rho); dt / (2 tau) = dt rho / (4 mu_ref
    // lam^(1 - omega)), for omega = 1/2: dt rho / (4 mu_ref sqrt(lam)).  Reciprocals from
    // the refined estimate (a few ulp; a zero or non-finite input gives a non-finite
    // result, which the failure check below reports as an IEEE divide's would).
    const double rn = Wn[0], irn = rcp_nr(rn), Un = Wn[1] * irn, Vn = Wn[2] * irn;
    const double iln = 4.0 * (Wn[3] - 0.5 * rn * (Un * Un + Vn * Vn)) * irn * P.inv_kp2;
    const double ln = rcp_nr(iln);
    const double r1 = W1[0], ir1 = rcp_nr(r1), U1 = W1[1] * ir1, V1 = W1[2] * ir1;
    const double il1 = 4.0 * (W1[3] - 0.5 * r1 * (U1 * U1 + V1 * V1)) * ir1 * P.inv_kp2;
    const double l1 = rcp_nr(il1);
    if (!(r1 > 0.0) || !(l1 > 0.0) || !isfinite(l1) || !isfinite(U1) || !isfinite(V1))
      atomicOr(err, 1);
    CellRec R;
    R.Gn = rn * ln / kPi; R.Un = Un; R.Vn = Vn; R.lamn = ln; R.bn = 0.5 * K * iln;
    R.G1 = r1 * l1 / kPi; R.U1 = U1; R.V1 = V1; R.lam1 = l1; R.b1 = 0.5 * K * il1;
    if (P.omega_half) {
      R.cgn = P.quarter_dt_mu * rn * rsqrt(ln);
      R.cg1 = P.quarter_dt_mu * r1 * rsqrt(l1);
    } else {
      R.cgn = P.dt / (2.0 * collision_time(P, rn, ln));
      R.cg1 = P.dt / (2.0 * collision_time(P, r1, l1));
    }
    R.cf = 1.0 - R.cgn;
    R.inv = rcp_nr(1.0 + R.cg1);
    // Shakhov model: heat flux of f^n about (Un, Vn) from the cell's raw moments (plus those
    // of g_ref in the FP32-f form), and alpha of W^n and W^{n+1}
    R.qx = R.qy = R.an = R.a1 = 0.0;
    if (P.shk) {
      const double* hc = P.hs + (size_t)w * kNHeat + kHeatC;
      const double* rc = P.refheat[4];
      double M[4][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
      M[0][0] = hc[0] + rc[0]; M[1][0] = hc[1] + rc[1]; M[0][1] = hc[2] + rc[2];
      M[2][0] = hc[3] + rc[3]; M[1][1] = hc[4] + rc[4]; M[0][2] = hc[5] + rc[5];
      M[3][0] = hc[6] + rc[6]; M[2][1] = hc[7] + rc[7]; M[1][2] = hc[8] + rc[8];
      M[0][3] = hc[9] + rc[9];
      double q[2];
      heat_flux_of(M, hc[10] + P.refheatC[0], hc[11] + P.refheatC[1], hc[12] + P.refheatC[2], Un, Vn, q);
      R.qx = q[0];
      R.qy = q[1];
      R.an = P.shk_c * ln * ln * irn;
      R.a1 = P.shk_c * l1 * l1 * ir1;
    }
    if (crf) {
      const int nfx = (nx + 1) * P.ny;
      constexpr double kLog2e = 1.4426950408889634;
      const double refx = (mt4[xw] - mt4[xe]) * P.d_idx, refy = (mt4[nfx + ys] - mt4[nfx + yn]) * P.d_idy;
      CellRecF F;
      // exponents of g^n, g^{n+1} relative to those of g_ref (log2 units), in FP64 but for
      // the amplitude's log2(G / G_ref) = log2(1 + d), d = G / G_ref - 1 formed in FP64 and
      // log1p in FP32: its error is an ulp of a result that is small where G is near
      // G_ref (an FP32 log2 of G itself put ~1e-7 relative noise on g per cell, visible in
      // rho V at Kn 0.01); the record's FP32 fields rounded by f32_rn (integer pipe)
      constexpr float kLog2ef = 1.44269504f;
      const double r0 = P.ref_E0u, r1 = P.ref_E[1], r2 = P.ref_E[2], r3 = P.ref_E[3];
      const double ldn = f64_of(log1pf(f32_rn(fma(R.Gn, P.ref_iG, -1.0))) * kLog2ef);
      const double ld1 = f64_of(log1pf(f32_rn(fma(R.G1, P.ref_iG, -1.0))) * kLog2ef);
      F.dEn[0] = f32_rn((ldn - ln * (Un * Un + Vn * Vn) * kLog2e) - r0);
      F.dEn[1] = f32_rn(2.0 * ln * Un * kLog2e - r1);
      F.dEn[2] = f32_rn(2.0 * ln * Vn * kLog2e - r2);
      F.dEn[3] = f32_rn(-ln * kLog2e - r3);
      F.dE1[0] = f32_rn((ld1 - l1 * (U1 * U1 + V1 * V1) * kLog2e) - r0);
      F.dE1[1] = f32_rn(2.0 * l1 * U1 * kLog2e - r1);
      F.dE1[2] = f32_rn(2.0 * l1 * V1 * kLog2e - r2);
      F.dE1[3] = f32_rn(-l1 * kLog2e - r3);
      F.A1 = f32_rn(R.inv * R.cg1);
      F.An = f32_rn(R.inv * R.cgn);
      F.db1 = f32_rn(R.b1 - P.ref_bf);
      F.dbn = f32_rn(R.bn - P.ref_bf);
      F.nBs = f32_rn(-(R.inv * (R.cg1 + R.cgn)));
      F.irx = f32_rn(R.inv * refx);
      F.iry = f32_rn(R.inv * refy);
      F.inv = f32_rn(R.inv);
      crf[c] = F;
      if (P.shk) {  // Shakhov factors of g^n and g^{n+1}, global frame
        CellShkF S;
        double p[4][4];
        const double q[2] = {R.qx, R.qy};
        for (int g = 0; g < 2; g++) {
          const double al = g == 0 ? R.an : R.a1, Ug = g == 0 ? Un : U1, Vg = g == 0 ? Vn : V1;
          const double lg = g == 0 ? ln : l1, bg = g == 0 ? R.bn : R.b1;
          shakhov_poly(al, Ug, Vg, lg, q, -4.0, p);
          float* sg = g == 0 ? S.sn : S.s1;
          float* lb = g == 0 ? S.ln : S.l1;
          sg[0] = f32_rn(p[0][0]); sg[1] = f32_rn(p[1][0]); sg[2] = f32_rn(p[0][1]); sg[3] = f32_rn(p[2][0]);
          sg[4] = f32_rn(p[1][1]); sg[5] = f32_rn(p[0][2]); sg[6] = f32_rn(p[3][0]); sg[7] = f32_rn(p[0][3]);
          const double m = 2.0 * bg * al;
          lb[0] = f32_rn(-m * (q[0] * Ug + q[1] * Vg));
          lb[1] = f32_rn(m * q[0]);
          lb[2] = f32_rn(m * q[1]);
          lb[3] = 0.f;
        }
        P.cshk[c] = S;
      }
    } else if (crd) {
      CellRecD D;
      D.Gn = split_df(R.Gn); D.Un = split_df(R.Un); D.Vn = split_df(R.Vn);
      D.lamn = split_df(R.lamn); D.bn = split_df(R.bn);
      D.G1 = split_df(R.G1); D.U1 = split_df(R.U1); D.V1 = split_df(R.V1);
      D.lam1 = split_df(R.lam1); D.b1 = split_df(R.b1);
      D.inv = split_df(R.inv); D.cgn = split_df(R.cgn); D.cg1 = split_df(R.cg1);
      D.pad = make_float2(0.f, 0.f);
      crd[c] = D;
    } else {
      cr[c] = R;
    }
  }
  for (int k = 0; k < 4; k++) {
    red[k][threadIdx.x] = d2[k];
    red[4 + k][threadIdx.x] = am[k];
  }
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 4; k++) {
        red[k][threadIdx.x] += red[k][threadIdx.x + s];
        red[4 + k][threadIdx.x] = fmax(red[4 + k][threadIdx.x], red[4 + k][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 8) rpart[(size_t)bx * 8 + threadIdx.x] = red[threadIdx.x][0];
}
__global__ void __launch_bounds__(128) k_cells(Params P, const double* __restrict__ Win,
                                               double* __restrict__ Wout, int nwe,
                                               const double* __restrict__ Fx,
                                               const double* __restrict__ Fy,
                                               CellRec* __restrict__ cr, double* __restrict__ rpart,
                                               int* __restrict__ err, CellRecF* __restrict__ crf,
                                               const double* __restrict__ mt4,
                                               CellRecD* __restrict__ crd = nullptr) {
  __shared__ double red[8][128];
  cells_body(P, Win, Wout, nwe, Fx, Fy, cr, rpart, err, crf, mt4, red, blockIdx.x, crd);
}

// -------------------------------------------------------------------------------------
// S6 + S8 and Eq. 3: micro flux of the four faces from the upwind reconstruction and the
// face records, implicit collision update written as an increment, f^{n+1} = f^n + df,
//   df = inv [ flux + cg1 (g^{n+1} - f^n) + cgn (g^n - f^n) ],
// so that rounding acts on df rather than on f.  One warp per interior cell, lane = u
// index (chunks of 32); the v loop is split into v <= 0 and v > 0 so that the y-upwind
// side is fixed in each half.  FP64 form.
// -------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void poly_in_v_xface(const double* c, double u, T* q) {
  // face frame un = u (fixed), ut = v: Q = q0 + q1 v + q2 v^2 + q3 v^3
  q[0] = (T)(c[0] + u * (c[1] + u * (c[3] + u * c[6])));
  q[1] = (T)(c[2] + u * (c[4] + u * c[7]));
  q[2] = (T)(c[5] + u * c[6]);
  q[3] = (T)c[7];
}
template <typename T>
__device__ __forceinline__ void poly_in_v_yface(const double* c, double u, T* q) {
  // face frame un = v, ut = u (fixed): Q = q0 + q1 v + q2 v^2 + q3 v^3
  q[0] = (T)(c[0] + u * (c[2] + u * (c[5] + u * c[7])));
  q[1] = (T)(c[1] + u * (c[4] + u * c[6]));
  q[2] = (T)(c[3] + u * c[7]);
  q[3] = (T)c[6];
}

template <typename T>
__device__ __forceinline__ T horner3(const T* q, T v) {
  return ((q[3] * v + q[2]) * v + q[1]) * v + q[0];
}

// Per-cell constants of the update kernel, converted to T once per warp.
template <typename T>
struct UpdCell {
  T Mt4[4], Mt5[4], bf[4];
  T inv, cg1, cgn, cg1b, cgnb;
  int wall[4];
};

// The van Leer slopes of the cell and of its upwind neighbours are formed here (12 per
// velocity-cell), so the kernel needs no slope buffer.
template <typename T, typename T2>
__global__ void __launch_bounds__(128) k_update(Params P, const T2* __restrict__ f,
                                                T2* __restrict__ fo,
                                                const FaceRec* __restrict__ fxr,
                                                const FaceRec* __restrict__ fyr,
                                                const CellRec* __restrict__ cr) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nv = P.nv, nu = P.nu, nq = P.nq, nx = P.nx, ny = P.ny;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* sv = reinterpret_cast<T*>(smraw);
  T* ev = sv + nv + warp * 6 * nv;  // [6][nv]: x W, x E, y S, y N, g^n, g^{n+1} factors in v
  for (int m = tid; m < nv; m += blockDim.x) sv[m] = (T)P.v[m];
  __syncthreads();
  const int cell = blockIdx.x * kWarpsPerBlock + warp;
  if (cell >= nx * ny) return;
  const int i = cell % nx, j = cell / nx;
  const FaceRec& RW = fxr[(size_t)j * (nx + 1) + i];
  const FaceRec& RE = fxr[(size_t)j * (nx + 1) + i + 1];
  const FaceRec& RS = fyr[(size_t)j * nx + i];
  const FaceRec& RN = fyr[(size_t)(j + 1) * nx + i];
  const CellRec& C = cr[cell];
  for (int m = lane; m < nv; m += 32) {
    const double vv = P.v[m];
    double d;
    d = vv - RW.Ut; ev[0 * nv + m] = (T)exp(-RW.lam * d * d);  // x faces: ut = v
    d = vv - RE.Ut; ev[1 * nv + m] = (T)exp(-RE.lam * d * d);
    d = vv - RS.Un; ev[2 * nv + m] = (T)exp(-RS.lam * d * d);  // y faces: un = v
    d = vv - RN.Un; ev[3 * nv + m] = (T)exp(-RN.lam * d * d);
    d = vv - C.Vn;  ev[4 * nv + m] = (T)exp(-C.lamn * d * d);
    d = vv - C.V1;  ev[5 * nv + m] = (T)exp(-C.lam1 * d * d);
  }
  __syncwarp();
  UpdCell<T> K;
  {
    const FaceRec* R[4] = {&RW, &RE, &RS, &RN};
#pragma unroll
    for (int s = 0; s < 4; s++) {
      K.Mt4[s] = (T)R[s]->Mt4;
      K.Mt5[s] = (T)R[s]->Mt5;
      K.bf[s] = (T)R[s]->bfac;
      K.wall[s] = R[s]->wall;
    }
    K.inv = (T)C.inv;
    K.cg1 = (T)C.cg1;
    K.cgn = (T)C.cgn;
    K.cg1b = (T)(C.cg1 * C.b1);
    K.cgnb = (T)(C.cgn * C.bn);
  }
  const T tdx = T(2.0 / P.dx), tdy = T(2.0 / P.dy), idx = T(1.0 / P.dx), idy = T(1.0 / P.dy);
  const T dtT = (T)P.dt;
  const long rs = (long)P.ex * nq;
  const T2* fc0 = f + fcell(P, i, j) * nq;
  T2* fo0 = fo + fcell(P, i, j) * nq;
  const bool pW = P.bc_kind[0] == 2, pE = P.bc_kind[1] == 2, pS = P.bc_kind[2] == 2, pN = P.bc_kind[3] == 2;

  for (int k0 = 0; k0 < nu; k0 += 32) {
    const int k = k0 + lane;
    const bool act = k < nu;
    const int kk = act ? k : nu - 1;
    const double ud = P.u[kk];
    const T u = (T)ud;
    T gu[4], gun, gu1;
    {
      double d;
      d = ud - RW.Un; gu[0] = (T)(RW.G * exp(-RW.lam * d * d));
      d = ud - RE.Un; gu[1] = (T)(RE.G * exp(-RE.lam * d * d));
      d = ud - RS.Ut; gu[2] = (T)(RS.G * exp(-RS.lam * d * d));
      d = ud - RN.Ut; gu[3] = (T)(RN.G * exp(-RN.lam * d * d));
      d = ud - C.Un;  gun = (T)(C.Gn * exp(-C.lamn * d * d));
      d = ud - C.U1;  gu1 = (T)(C.G1 * exp(-C.lam1 * d * d));
    }
    const int xs = ud > 0.0 ? 0 : 1;
    T qW[2][4], qE[2][4];
#pragma unroll
    for (int c = 0; c < 2; c++) {
      poly_in_v_xface(RW.Q[xs][c], ud, qW[c]);
      poly_in_v_xface(RE.Q[xs][c], ud, qE[c]);
    }
    const bool up = ud > 0.0;  // x upwind neighbour: W for u > 0, E for u < 0
    const long xo = up ? -(long)nq : (long)nq;
    const bool xz = (up && i == 0 && pW) || (!up && i == nx - 1 && pE);
    const T cu = u * tdx, fxu = u * idx;

    // one half of the v range: VUP = (v > 0); y-upwind neighbour S for v > 0, N otherwise
    auto half = [&](auto vup_tag, int m0, int m1) {
      constexpr bool VUP = decltype(vup_tag)::value;
      T qS[2][4], qN[2][4];
#pragma unroll
      for (int c = 0; c < 2; c++) {
        poly_in_v_yface(RS.Q[VUP ? 0 : 1][c], ud, qS[c]);
        poly_in_v_yface(RN.Q[VUP ? 0 : 1][c], ud, qN[c]);
      }
      const long yo = VUP ? -rs : rs;
      const bool yz = (VUP && j == 0 && pS) || (!VUP && j == ny - 1 && pN);
      for (int m = m0; m < m1; m++) {
        const T vv = sv[m];
        const T2* p = fc0 + (size_t)m * nu + kk;
        const T2 c = p[0];
        const T2 xu = p[xo], yu = p[yo];
        // half slopes r = sigma h / 2 of the cell, its x-upwind and its y-upwind neighbour
        T rxch, rxcb, rych, rycb, rxuh, rxub, ryuh, ryub, rxvh, rxvb, ryvh, ryvb;
        {
          const T2 w = p[-(long)nq], e = p[nq], s = p[-rs], n = p[rs];
          const T2 xf = p[2 * xo], xs_ = p[xo - rs], xn = p[xo + rs];
          const T2 yf = p[2 * yo], yw = p[yo - (long)nq], ye = p[yo + (long)nq];
          rxch = vl_half(w.x, c.x, e.x); rxcb = vl_half(w.y, c.y, e.y);
          rych = vl_half(s.x, c.x, n.x); rycb = vl_half(s.y, c.y, n.y);
          if (up) { rxuh = vl_half(xf.x, w.x, c.x); rxub = vl_half(xf.y, w.y, c.y); }
          else    { rxuh = vl_half(c.x, e.x, xf.x); rxub = vl_half(c.y, e.y, xf.y); }
          ryuh = vl_half(xs_.x, xu.x, xn.x); ryub = vl_half(xs_.y, xu.y, xn.y);
          rxvh = vl_half(yw.x, yu.x, ye.x); rxvb = vl_half(yw.y, yu.y, ye.y);
          if (VUP) { ryvh = vl_half(yf.x, s.x, c.x); ryvb = vl_half(yf.y, s.y, c.y); }
          else     { ryvh = vl_half(c.x, n.x, yf.x); ryvb = vl_half(c.y, n.y, yf.y); }
        }
        if (xz) rxuh = rxub = ryuh = ryub = T(0);
        if (yz) rxvh = rxvb = ryvh = ryvb = T(0);
        const T cv = vv * tdy, fyv = vv * idy;
        // (u sigma_x + v sigma_y) of the three cells
        const T dch = cu * rxch + cv * rych, dcb = cu * rxcb + cv * rycb;
        const T duh = cu * rxuh + cv * ryuh, dub = cu * rxub + cv * ryub;
        const T dvh = cu * rxvh + cv * ryvh, dvb = cu * rxvb + cv * ryvb;
        // upwind interface values and slope terms
        T fWh, fWb, dWh, dWb, fEh, fEb, dEh, dEb;
        if (up) {
          fEh = c.x + rxch; fEb = c.y + rxcb; dEh = dch; dEb = dcb;
          fWh = xu.x + rxuh; fWb = xu.y + rxub; dWh = duh; dWb = dub;
        } else {
          fWh = c.x - rxch; fWb = c.y - rxcb; dWh = dch; dWb = dcb;
          fEh = xu.x - rxuh; fEb = xu.y - rxub; dEh = duh; dEb = dub;
        }
        T fSh, fSb, dSh, dSb, fNh, fNb, dNh, dNb;
        if (VUP) {
          fNh = c.x + rych; fNb = c.y + rycb; dNh = dch; dNb = dcb;
          fSh = yu.x + ryvh; fSb = yu.y + ryvb; dSh = dvh; dSb = dvb;
        } else {
          fSh = c.x - rych; fSb = c.y - rycb; dSh = dch; dSb = dcb;
          fNh = yu.x - ryvh; fNb = yu.y - ryvb; dNh = dvh; dNb = dvb;
        }
        // X = Q g + Mt4 f_up - Mt5 d (UGKS face), X = dt f_w (wall); F~ = u_n X
        T XWh, XWb, XEh, XEb, XSh, XSb, XNh, XNb;
        {
          const T g = gu[0] * ev[m];
          if (K.wall[0]) {
            const bool inc = !up;  // gas on the high side: incoming u < 0
            XWh = inc ? dtT * fWh : dtT * g;
            XWb = inc ? dtT * fWb : dtT * (K.bf[0] * g);
          } else {
            XWh = horner3(qW[0], vv) * g + K.Mt4[0] * fWh - K.Mt5[0] * dWh;
            XWb = horner3(qW[1], vv) * g + K.Mt4[0] * fWb - K.Mt5[0] * dWb;
          }
        }
        {
          const T g = gu[1] * ev[nv + m];
          if (K.wall[1]) {
            const bool inc = up;  // gas on the low side: incoming u > 0
            XEh = inc ? dtT * fEh : dtT * g;
            XEb = inc ? dtT * fEb : dtT * (K.bf[1] * g);
          } else {
            XEh = horner3(qE[0], vv) * g + K.Mt4[1] * fEh - K.Mt5[1] * dEh;
            XEb = horner3(qE[1], vv) * g + K.Mt4[1] * fEb - K.Mt5[1] * dEb;
          }
        }
        {
          const T g = gu[2] * ev[2 * nv + m];
          if (K.wall[2]) {
            XSh = !VUP ? dtT * fSh : dtT * g;
            XSb = !VUP ? dtT * fSb : dtT * (K.bf[2] * g);
          } else {
            XSh = horner3(qS[0], vv) * g + K.Mt4[2] * fSh - K.Mt5[2] * dSh;
            XSb = horner3(qS[1], vv) * g + K.Mt4[2] * fSb - K.Mt5[2] * dSb;
          }
        }
        {
          const T g = gu[3] * ev[3 * nv + m];
          if (K.wall[3]) {
            XNh = VUP ? dtT * fNh : dtT * g;
            XNb = VUP ? dtT * fNb : dtT * (K.bf[3] * g);
          } else {
            XNh = horner3(qN[0], vv) * g + K.Mt4[3] * fNh - K.Mt5[3] * dNh;
            XNb = horner3(qN[1], vv) * g + K.Mt4[3] * fNb - K.Mt5[3] * dNb;
          }
        }
        T flh = fxu * (XWh - XEh) + fyv * (XSh - XNh);
        T flb = fxu * (XWb - XEb) + fyv * (XSb - XNb);
        const T gnh = gun * ev[4 * nv + m], g1h = gu1 * ev[5 * nv + m];
        const T dh = K.inv * (flh + K.cg1 * (g1h - c.x) + K.cgn * (gnh - c.x));
        const T db = K.inv * (flb + (K.cg1b * g1h - K.cg1 * c.y) + (K.cgnb * gnh - K.cgn * c.y));
        T2 o;
        o.x = c.x + dh;
        o.y = c.y + db;
        if (act) fo0[(size_t)m * nu + kk] = o;
      }
    };
    half(std::integral_constant<bool, false>{}, 0, P.m_pos);
    half(std::integral_constant<bool, true>{}, P.m_pos, nv);
  }
}


// -------------------------------------------------------------------------------------
// The same update in two passes, FP64 form: every (face, velocity) micro flux once.
// k_face_flux: one warp per interior cell, lane = u index; for each velocity the cell forms
// the flux X = Q g + Mt4 f_up - Mt5 d_up (or the wall flux) through its downwind x-face and
// y-face from its own reconstruction, and a cell next to the boundary also forms the flux
// whose upwind side is the ghost cell or the wall.  Every face and velocity is written by
// exactly one warp, into Xx [(nx+1) ny][nq] and Xy [nx (ny+1)][nq] (face-major, velocity
// innermost).  k_cell_update then reads the four fluxes of each velocity-cell and applies
// Eq. 3.  The arithmetic of each flux and of the update is that of k_update, which forms
// the four face fluxes of every velocity-cell (each interior flux twice).
// -------------------------------------------------------------------------------------
template <typename T>
struct FaceK {
  T Mt4, Mt5, bf;
  int wall;
};
template <typename T, typename T2>
__global__ void __launch_bounds__(128) k_face_flux(Params P, const T2* __restrict__ f,
                                                   const FaceRec* __restrict__ fxr,
                                                   const FaceRec* __restrict__ fyr,
                                                   const T2* __restrict__ sl, T2* __restrict__ Xx,
                                                   T2* __restrict__ Xy) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nv = P.nv, nu = P.nu, nq = P.nq, nx = P.nx, ny = P.ny;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* sv = reinterpret_cast<T*>(smraw);
  T* ev = sv + nv + warp * 4 * nv;  // [4][nv]: x W, x E, y S, y N factors in v
  for (int m = tid; m < nv; m += blockDim.x) sv[m] = (T)P.v[m];
  __syncthreads();
  const int cell = blockIdx.x * kWarpsPerBlock + warp;
  if (cell >= nx * ny) return;
  const int i = cell % nx, j = cell / nx;
  const FaceRec& RW = fxr[(size_t)j * (nx + 1) + i];
  const FaceRec& RE = fxr[(size_t)j * (nx + 1) + i + 1];
  const FaceRec& RS = fyr[(size_t)j * nx + i];
  const FaceRec& RN = fyr[(size_t)(j + 1) * nx + i];
  for (int m = lane; m < nv; m += 32) {
    const double vv = P.v[m];
    double d;
    d = vv - RW.Ut; ev[0 * nv + m] = (T)exp(-RW.lam * d * d);  // x faces: ut = v
    d = vv - RE.Ut; ev[1 * nv + m] = (T)exp(-RE.lam * d * d);
    d = vv - RS.Un; ev[2 * nv + m] = (T)exp(-RS.lam * d * d);  // y faces: un = v
    d = vv - RN.Un; ev[3 * nv + m] = (T)exp(-RN.lam * d * d);
  }
  __syncwarp();
  auto faceK = [](const FaceRec& R) { return FaceK<T>{(T)R.Mt4, (T)R.Mt5, (T)R.bfac, R.wall}; };
  const FaceK<T> KW = faceK(RW), KE = faceK(RE), KS = faceK(RS), KN = faceK(RN);
  const T tdx = T(2.0 / P.dx), tdy = T(2.0 / P.dy);
  const T dtT = (T)P.dt;
  const long rs = (long)P.ex * nq;
  const T2* fc0 = f + fcell(P, i, j) * nq;
  const T2* sl0 = sl + (size_t)wcell(P, i, j) * nq * 2;  // this cell's slopes
  T2* xw0 = Xx + ((size_t)j * (nx + 1) + i) * nq;        // W face of the cell; E face: + nq
  T2* ys0 = Xy + ((size_t)j * nx + i) * nq;              // S face; N face: + nx nq
  const bool pW = P.bc_kind[0] == 2, pE = P.bc_kind[1] == 2, pS = P.bc_kind[2] == 2, pN = P.bc_kind[3] == 2;

  // X of a face from the face value fh, fb and slope term dh, db of its upwind side; inc:
  // the gas side is upwind (a wall face then passes dt f_up, else dt g_wall)
  auto flux = [&](const FaceK<T>& F, const T (&qh)[4], const T (&qb)[4], T vv, T g, T fh, T fb,
                  T dh, T db, bool inc) {
    T2 X;
    if (F.wall) {
      X.x = inc ? dtT * fh : dtT * g;
      X.y = inc ? dtT * fb : dtT * (F.bf * g);
    } else {
      X.x = horner3(qh, vv) * g + F.Mt4 * fh - F.Mt5 * dh;
      X.y = horner3(qb, vv) * g + F.Mt4 * fb - F.Mt5 * db;
    }
    return X;
  };

  for (int k0 = 0; k0 < nu; k0 += 32) {
    const int k = k0 + lane;
    const bool act = k < nu;
    const int kk = act ? k : nu - 1;
    const double ud = P.u[kk];
    const T u = (T)ud;
    T gu[4];
    {
      double d;
      d = ud - RW.Un; gu[0] = (T)(RW.G * exp(-RW.lam * d * d));
      d = ud - RE.Un; gu[1] = (T)(RE.G * exp(-RE.lam * d * d));
      d = ud - RS.Ut; gu[2] = (T)(RS.G * exp(-RS.lam * d * d));
      d = ud - RN.Ut; gu[3] = (T)(RN.G * exp(-RN.lam * d * d));
    }
    const int xs = ud > 0.0 ? 0 : 1;  // upwind side of the x-face records
    const bool up = ud > 0.0;         // downwind x-face: E for u > 0, W otherwise
    const T sgx = up ? T(1) : T(-1);  // f_up = f + sgx r_x on the downwind face
    // the downwind x-face (formed by this cell for every velocity) and the upwind one
    // (formed here only when its upwind side is a ghost cell or a wall)
    const FaceRec& RXd = up ? RE : RW;
    const FaceRec& RXg = up ? RW : RE;
    const FaceK<T> KXd = up ? KE : KW, KXg = up ? KW : KE;
    const T gXd = up ? gu[1] : gu[0], gXg = up ? gu[0] : gu[1];
    const T* evXd = ev + (up ? nv : 0);
    const T* evXg = ev + (up ? 0 : nv);
    T2* xd0 = up ? xw0 + nq : xw0;
    T2* xg0 = up ? xw0 : xw0 + nq;
    T qX[2][4];
#pragma unroll
    for (int c = 0; c < 2; c++) poly_in_v_xface(RXd.Q[xs][c], ud, qX[c]);
    const long xo = up ? -(long)nq : (long)nq;  // x-upwind neighbour in f, in q
    const bool xg = up ? i == 0 : i == nx - 1;  // it is a ghost cell (or a wall)
    const bool xz = (up && i == 0 && pW) || (!up && i == nx - 1 && pE);
    const T cu = u * tdx;

    auto half = [&](auto vup_tag, int m0, int m1) {
      constexpr bool VUP = decltype(vup_tag)::value;  // downwind y-face: N for v > 0, S otherwise
      constexpr int ys = VUP ? 0 : 1;
      const FaceRec& RYd = VUP ? RN : RS;
      const FaceRec& RYg = VUP ? RS : RN;
      const FaceK<T>& KYd = VUP ? KN : KS;
      const FaceK<T>& KYg = VUP ? KS : KN;
      const T gYd = VUP ? gu[3] : gu[2], gYg = VUP ? gu[2] : gu[3];
      const T* evYd = ev + (VUP ? 3 : 2) * nv;
      const T* evYg = ev + (VUP ? 2 : 3) * nv;
      T2* yd0 = VUP ? ys0 + (size_t)nx * nq : ys0;
      T2* yg0 = VUP ? ys0 : ys0 + (size_t)nx * nq;
      constexpr T sgy = VUP ? T(1) : T(-1);
      T qY[2][4];
#pragma unroll
      for (int c = 0; c < 2; c++) poly_in_v_yface(RYd.Q[ys][c], ud, qY[c]);
      const long yo = VUP ? -rs : rs;                             // y-upwind neighbour in f
      const long yso = VUP ? -(long)P.wx * nq : (long)P.wx * nq;  // ... in the slope buffer
      const bool yg = VUP ? j == 0 : j == ny - 1;
      const bool yz = (VUP && j == 0 && pS) || (!VUP && j == ny - 1 && pN);
      for (int m = m0; m < m1; m++) {
        const T vv = sv[m];
        const size_t q = (size_t)m * nu + kk;
        const T2* p = fc0 + q;
        const T2 c = p[0];
        const T2* sq = sl0 + 2 * q;
        const T2 a = sq[0], b = sq[1];  // half slopes r_x, r_y of the cell (h, b)
        const T cv = vv * tdy;
        const T dch = cu * a.x + cv * b.x, dcb = cu * a.y + cv * b.y;
        T2 X = flux(KXd, qX[0], qX[1], vv, gXd * evXd[m], c.x + sgx * a.x, c.y + sgx * a.y, dch,
                    dcb, true);
        if (act) xd0[q] = X;
        if (xg) {
          const T2 xu = p[xo];
          const T2* su = sq + 2 * xo;
          T2 au = su[0], bu = su[1];
          if (xz) au.x = au.y = bu.x = bu.y = T(0);
          const T duh = cu * au.x + cv * bu.x, dub = cu * au.y + cv * bu.y;
          T qg[2][4];
#pragma unroll
          for (int cc = 0; cc < 2; cc++) poly_in_v_xface(RXg.Q[xs][cc], ud, qg[cc]);
          X = flux(KXg, qg[0], qg[1], vv, gXg * evXg[m], xu.x + sgx * au.x, xu.y + sgx * au.y, duh,
                   dub, false);
          if (act) xg0[q] = X;
        }
        X = flux(KYd, qY[0], qY[1], vv, gYd * evYd[m], c.x + sgy * b.x, c.y + sgy * b.y, dch, dcb,
                 true);
        if (act) yd0[q] = X;
        if (yg) {
          const T2 yu = p[yo];
          const T2* sw = sq + 2 * yso;
          T2 av = sw[0], bv = sw[1];
          if (yz) av.x = av.y = bv.x = bv.y = T(0);
          const T dvh = cu * av.x + cv * bv.x, dvb = cu * av.y + cv * bv.y;
          T qg[2][4];
#pragma unroll
          for (int cc = 0; cc < 2; cc++) poly_in_v_yface(RYg.Q[ys][cc], ud, qg[cc]);
          X = flux(KYg, qg[0], qg[1], vv, gYg * evYg[m], yu.x + sgy * bv.x, yu.y + sgy * bv.y, dvh,
                   dvb, false);
          if (act) yg0[q] = X;
        }
      }
    };
    half(std::integral_constant<bool, false>{}, 0, P.m_pos);
    half(std::integral_constant<bool, true>{}, P.m_pos, nv);
  }
}

// Eq. 3 from the four face fluxes of each velocity-cell (k_face_flux), FP64 form.
template <typename T, typename T2>
__global__ void __launch_bounds__(128) k_cell_update(Params P, const T2* __restrict__ f,
                                                     T2* __restrict__ fo,
                                                     const CellRec* __restrict__ cr,
                                                     const T2* __restrict__ Xx,
                                                     const T2* __restrict__ Xy) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nv = P.nv, nu = P.nu, nq = P.nq, nx = P.nx, ny = P.ny;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* sv = reinterpret_cast<T*>(smraw);
  T* ev = sv + nv + warp * 2 * nv;  // [2][nv]: g^n, g^{n+1} factors in v
  for (int m = tid; m < nv; m += blockDim.x) sv[m] = (T)P.v[m];
  __syncthreads();
  const int cell = blockIdx.x * kWarpsPerBlock + warp;
  if (cell >= nx * ny) return;
  const int i = cell % nx, j = cell / nx;
  const CellRec& C = cr[cell];
  for (int m = lane; m < nv; m += 32) {
    const double vv = P.v[m];
    double d;
    d = vv - C.Vn; ev[m] = (T)exp(-C.lamn * d * d);
    d = vv - C.V1; ev[nv + m] = (T)exp(-C.lam1 * d * d);
  }
  __syncwarp();
  const T inv = (T)C.inv, cg1 = (T)C.cg1, cgn = (T)C.cgn;
  const T cg1b = (T)(C.cg1 * C.b1), cgnb = (T)(C.cgn * C.bn);
  const T idx = T(1.0 / P.dx), idy = T(1.0 / P.dy);
  const T2* fc0 = f + fcell(P, i, j) * nq;
  T2* fo0 = fo + fcell(P, i, j) * nq;
  const T2* xw0 = Xx + ((size_t)j * (nx + 1) + i) * nq;
  const T2* ys0 = Xy + ((size_t)j * nx + i) * nq;
  for (int k0 = 0; k0 < nu; k0 += 32) {
    const int k = k0 + lane;
    const bool act = k < nu;
    const int kk = act ? k : nu - 1;
    const double ud = P.u[kk];
    const T u = (T)ud;
    T gun, gu1;
    {
      double d;
      d = ud - C.Un; gun = (T)(C.Gn * exp(-C.lamn * d * d));
      d = ud - C.U1; gu1 = (T)(C.G1 * exp(-C.lam1 * d * d));
    }
    const T fxu = u * idx;
    for (int m = 0; m < nv; m++) {
      const T vv = sv[m];
      const T fyv = vv * idy;
      const size_t q = (size_t)m * nu + kk;
      const T2 c = fc0[q];
      const T2 XW = xw0[q], XE = xw0[nq + q], XS = ys0[q], XN = ys0[(size_t)nx * nq + q];
      T flh = fxu * (XW.x - XE.x) + fyv * (XS.x - XN.x);
      T flb = fxu * (XW.y - XE.y) + fyv * (XS.y - XN.y);
      const T gnh = gun * ev[m], g1h = gu1 * ev[nv + m];
      T dh, db;
      if (!P.shk) {
        dh = inv * (flh + cg1 * (g1h - c.x) + cgn * (gnh - c.x));
        db = inv * (flb + (cg1b * g1h - cg1 * c.y) + (cgnb * gnh - cgn * c.y));
      } else {  // Shakhov: g+_h = g_h (1 + S_h), g+_b = g_h (b + S_b), heat flux of f^n
        const double vd = P.v[m];
        double cu = ud - C.Un, cv = vd - C.Vn;
        double cq = cu * C.qx + cv * C.qy, c2 = 2.0 * C.lamn * (cu * cu + cv * cv);
        const T shn = (T)(C.an * cq * (c2 - 4.0)), sbn = (T)(C.an * cq * C.bn * (c2 - 2.0));
        cu = ud - C.U1; cv = vd - C.V1;
        cq = cu * C.qx + cv * C.qy; c2 = 2.0 * C.lam1 * (cu * cu + cv * cv);
        const T sh1 = (T)(C.a1 * cq * (c2 - 4.0)), sb1 = (T)(C.a1 * cq * C.b1 * (c2 - 2.0));
        const T gpnh = gnh + gnh * shn, gp1h = g1h + g1h * sh1;
        const T gpnb = gnh * ((T)C.bn + sbn), gp1b = g1h * ((T)C.b1 + sb1);
        dh = inv * (flh + cg1 * (gp1h - c.x) + cgn * (gpnh - c.x));
        db = inv * (flb + cg1 * (gp1b - c.y) + cgn * (gpnb - c.y));
      }
      T2 o;
      o.x = c.x + dh;
      o.y = c.y + db;
      if (act) fo0[q] = o;
    }
  }
}

}  // namespace ugks
