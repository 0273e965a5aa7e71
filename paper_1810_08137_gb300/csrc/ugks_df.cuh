// Double-FP32 arithmetic of the DF64 form beyond the scalar core of ugks_dfcore.cuh
// (error-free transformations, sums, products): division, lazily normalised running sums,
// e^x, and the same operations on packed FP32 pairs (two velocities per lane); then the DF64
// form's kernels.
#pragma once

#include "ugks_dfcore.cuh"

namespace ugks {

// a / b: quotient of the high parts, one correction from the double-FP32 remainder
__device__ __forceinline__ df df_div(df a, df b) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b.hi));
  r = __fmaf_rn(r, __fmaf_rn(-b.hi, r, 1.f), r);  // one Newton step: r to ~2^-24
  const float q1 = __fmul_rn(a.hi, r);
  const df rem = df_sub(a, df_mul(b, q1));
  return fast_two_sum(q1, __fmul_rn(rem.hi, r));
}
// Running sum acc + a b without renormalising: the rounding error of the high-part sum and
// the product's low parts go to acc.lo, which is left to grow (by at most an ulp of acc.hi
// per term); df_norm restores |lo| <= ulp(hi)/2 once the sum is complete.
__device__ __forceinline__ df df_acc(df acc, df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float pl = __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.hi, b.hi, -p)));
  const df s = two_sum(acc.hi, p);
  return {s.hi, __fadd_rn(acc.lo, __fadd_rn(s.lo, pl))};
}
__device__ __forceinline__ df df_norm(df a) { return two_sum(a.hi, a.lo); }

// e^x for x <= 0 (Maxwellian factors), about 2^-44 relative: x = k ln2 + r with
// |r| <= ln2 / 2, e^r = (e^(r/8))^8, e^(r/8) by its Taylor series to the 8th power in Horner
// form with double-FP32 coefficients 1/n (the first term left out is below 2^-50 for
// |r/8| <= 0.0434; each squaring doubles the relative error).  0 below x = -87.
__device__ __forceinline__ df df_exp(df x) {
  // ln 2 = kLn2Hi + kLn2Mid + kLn2Lo to about 2^-62; kLn2Hi has 15 significant bits, so
  // k kLn2Hi is exact for |k| < 2^9
  constexpr float kLn2Hi = 6.9314575e-01f, kLn2Mid = 1.4286068e-06f, kLn2Lo = 5.497923e-14f;
  // 1/n = kInvHi[n] + kInvLo[n]
  constexpr float kInvHi[9] = {0.f, 1.f, 5.e-01f, 3.3333334e-01f, 2.5e-01f, 2.e-01f, 1.6666667e-01f,
                               1.4285715e-01f, 1.25e-01f};
  constexpr float kInvLo[9] = {0.f, 0.f, 0.f, -9.934108e-09f, 0.f, -2.9802323e-09f, -4.967054e-09f,
                               -6.386212e-09f, 0.f};
  if (x.hi < -87.f) return {0.f, 0.f};
  const float k = rintf(__fmul_rn(x.hi, 1.442695e+00f));
  df r = df_add(x, df_of(-__fmul_rn(k, kLn2Hi)));
  r = df_sub(r, two_prod(k, kLn2Mid));
  r = df_add(r, df_of(-__fmul_rn(k, kLn2Lo)));
  const df t = {__fmul_rn(r.hi, 0.125f), __fmul_rn(r.lo, 0.125f)};
  // Horner: 1 + t (1 + t/2 (1 + t/3 (... (1 + t/8))))
  df p = df_of(1.f);
#pragma unroll
  for (int n = 8; n >= 1; n--) p = df_fma(df_mul(p, t), df{kInvHi[n], kInvLo[n]}, df_of(1.f));
  p = df_mul(p, p);
  p = df_mul(p, p);
  p = df_mul(p, p);
  const float s = __int_as_float(((int)k + 127) << 23);  // 2^k, k >= -126
  return {__fmul_rn(p.hi, s), __fmul_rn(p.lo, s)};
}

// ---- two double-FP32 numbers at once (two velocities of a lane), on packed FP32 pairs ----
// The operations of the scalar double-FP32 type, lane by lane: each packed instruction does
// the same operation on the .x and .y parts, so the results equal the scalar ones bitwise.
struct df2 {
  float2 hi, lo;
};
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  const float2 bb = sub2(s, a);
  return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
__device__ __forceinline__ df2 fast_two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  return {s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ df2 df2_add(df2 a, df2 b) {
  const df2 s = two_sum2(a.hi, b.hi);
  return fast_two_sum2(s.hi, add2(s.lo, add2(a.lo, b.lo)));
}
__device__ __forceinline__ df2 df2_neg(df2 a) { return {neg2(a.hi), neg2(a.lo)}; }
__device__ __forceinline__ df2 df2_sub(df2 a, df2 b) { return df2_add(a, df2_neg(b)); }
__device__ __forceinline__ df2 df2_mul(df2 a, df2 b) {
  const float2 p = mul2(a.hi, b.hi);
  const float2 e = fma2(a.lo, b.hi, fma2(a.hi, b.lo, fma2(a.hi, b.hi, neg2(p))));
  return fast_two_sum2(p, e);
}
// a b + c
__device__ __forceinline__ df2 df2_fma(df2 a, df2 b, df2 c) {
  const float2 p = mul2(a.hi, b.hi);
  const float2 pl = fma2(a.lo, b.hi, fma2(a.hi, b.lo, fma2(a.hi, b.hi, neg2(p))));
  const df2 s = two_sum2(c.hi, p);
  return fast_two_sum2(s.hi, add2(s.lo, add2(c.lo, pl)));
}
__device__ __forceinline__ df2 df2_bcast(df a) { return {make_float2(a.hi, a.hi), make_float2(a.lo, a.lo)}; }
__device__ __forceinline__ df2 df2_of(df a, df b) { return {make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}; }
__device__ __forceinline__ df df2_x(df2 a) { return {a.hi.x, a.lo.x}; }
__device__ __forceinline__ df df2_y(df2 a) { return {a.hi.y, a.lo.y}; }
__device__ __forceinline__ df2 df2_zero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

// =====================================================================================
// DF64 form of the step: f stored as double-FP32 pairs (DF4), the per-velocity arithmetic of
// the sums (S1, S7), the micro flux (S6, S8) and the implicit update (Eq. 3) in double-FP32
// on the FP32 pipe; the interface (S2-S5) and cell (Eq. 4) scalars in FP64 (the shared
// kernels, which write double-FP32 copies of their records).  The kernels follow the FP64
// form's kernels step for step: warp per cell, lane = u index, loop over the v rows.
// =====================================================================================
__device__ __forceinline__ df dfv(float2 a) { return {a.x, a.y}; }
__device__ __forceinline__ df dh(const DF4& v) { return {v.hh, v.hl}; }
__device__ __forceinline__ df db(const DF4& v) { return {v.bh, v.bl}; }
__device__ __forceinline__ DF4 mk4(df h, df b) {
  DF4 o;
  o.hh = h.hi; o.hl = h.lo; o.bh = b.hi; o.bl = b.lo;
  return o;
}
__device__ __forceinline__ DF4 split4(double h, double b) { return mk4(df_of(h), df_of(b)); }
__device__ __forceinline__ df df_half(df a) { return {0.5f * a.hi, 0.5f * a.lo}; }  // exact
__device__ __forceinline__ df df_zero() { return {0.f, 0.f}; }

// van Leer half slope d1 d2 / (d1 + d2) if d1 d2 > 0 else 0, d1 = c - a, d2 = b - c
__device__ __forceinline__ df vl_df(df a, df c, df b) {
  const df d1 = df_sub(c, a), d2 = df_sub(b, c);
  const df p = df_mul(d1, d2);
  const df r = df_div(p, df_add(d1, d2));
  return p.hi > 0.f ? r : df_zero();
}

// Warp sum of v[lane % N] returned to each lane (transpose reduce-scatter, as for FP64).
template <int N>
__device__ __forceinline__ df warp_reduce_scatter_df(df (&v)[N], int lane) {
#pragma unroll
  for (int o = N / 2; o >= 1; o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; i++) {
      const df send = upper ? v[i] : v[i + o];
      const df keep = upper ? v[i + o] : v[i];
      const df got = {__shfl_xor_sync(kFull, send.hi, o), __shfl_xor_sync(kFull, send.lo, o)};
      v[i] = df_add(keep, got);
    }
  }
  df r = v[0];
#pragma unroll
  for (int o = N; o < 32; o <<= 1)
    r = df_add(r, df{__shfl_xor_sync(kFull, r.hi, o), __shfl_xor_sync(kFull, r.lo, o)});
  return r;
}

// Ghost ring: the FP64 form's rules (pressure Maxwellian in FP64, periodic image,
// zero-gradient copy next to a wall), stored as double-FP32 pairs.
__device__ void fill_ghost_cell(const Params& P, DF4* f, double* W, int nwe, int gi, int gj,
                                int si, int sj, int side, bool write_W, int wi, int wj,
                                double* tab) {
  const int kind = P.bc_kind[side];
  DF4* dst = f + fcell(P, gi, gj) * P.nq;
  const DF4* src = f + fcell(P, si, sj) * P.nq;
  const int sw = wcell(P, wi, wj);
  if (kind == 2) {
    double* fu = tab;
    double* fv = tab + kMaxAxis;
    const double rho_a = W[sw], U = W[nwe + sw] / rho_a, V = W[2 * nwe + sw] / rho_a;
    const double lam = 1.0 / P.bc_T[side], rho = P.bc_rho[side];
    const double G = rho * lam / kPi, bf = P.K / (2.0 * lam);
    __syncthreads();  // the tables of the previous cell are no longer read
    for (int k = threadIdx.x; k < P.nu; k += blockDim.x) {
      const double du = P.u[k] - U;
      fu[k] = G * exp(-lam * du * du);
    }
    for (int m = threadIdx.x; m < P.nv; m += blockDim.x) {
      const double dv = P.v[m] - V;
      fv[m] = exp(-lam * dv * dv);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < P.nq; q += blockDim.x) {
      const int k = q % P.nu, m = q / P.nu;
      const double gh = fu[k] * fv[m];
      dst[q] = split4(gh, bf * gh);
    }
    if (write_W && threadIdx.x == 0) {
      const int g = wcell(P, gi, gj);
      W[g] = rho;
      W[nwe + g] = rho * U;
      W[2 * nwe + g] = rho * V;
      W[3 * nwe + g] = rho * (0.5 * (U * U + V * V) + (P.K + 2) / (4.0 * lam));
    }
  } else {
    for (int q = threadIdx.x; q < P.nq; q += blockDim.x) dst[q] = src[q];
    if (write_W && threadIdx.x == 0) {
      const int g = wcell(P, gi, gj), s = wcell(P, si, sj);
      for (int c = 0; c < 4; c++) W[c * nwe + g] = W[c * nwe + s];
    }
  }
}

// State conversion (set-up and checkpoint paths): FP64 rows [cell][q][(h, b)] of rows
// j0 .. j0+nrows-1 <-> double-FP32 f with its ghost ring; grid-stride over velocity-cells.
__global__ void k_rows_to_df(const double* __restrict__ src, DF4* __restrict__ dst, Params P, int j0,
                             int nrows) {
  const long n = (long)P.nx * nrows * P.nq;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const long c = t / P.nq;
    const int q = (int)(t - c * P.nq);
    const int r = (int)(c / P.nx), i = (int)(c - (long)r * P.nx);
    dst[((size_t)(j0 + r + 2) * P.ex + i + 2) * P.nq + q] = split4(src[2 * t], src[2 * t + 1]);
  }
}
__global__ void k_df_to_rows(const DF4* __restrict__ src, double* __restrict__ dst, Params P, int j0,
                             int nrows) {
  const long n = (long)P.nx * nrows * P.nq;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const long c = t / P.nq;
    const int q = (int)(t - c * P.nq);
    const int r = (int)(c / P.nx), i = (int)(c - (long)r * P.nx);
    const DF4 v = src[((size_t)(j0 + r + 2) * P.ex + i + 2) * P.nq + q];
    dst[2 * t] = (double)v.hh + (double)v.hl;
    dst[2 * t + 1] = (double)v.bh + (double)v.bl;
  }
}
// Pointwise Maxwellian of (rho, U, V, T) per cell (FP64, stored as double-FP32) and W.
__global__ void k_init_maxwellian_df(Params P, const double* __restrict__ prim, DF4* __restrict__ f,
                                     double* __restrict__ W, int nwe) {
  const int nc = P.nx * P.ny;
  const int cell = blockIdx.x;
  if (cell >= nc) return;
  const int i = cell % P.nx, j = cell / P.nx;
  const double rho = prim[cell], U = prim[nc + cell], V = prim[2 * nc + cell], T = prim[3 * nc + cell];
  const double lam = 1.0 / T, G = rho * lam / kPi, bf = P.K / (2.0 * lam);
  DF4* dst = f + fcell(P, i, j) * P.nq;
  for (int q = threadIdx.x; q < P.nq; q += blockDim.x) {
    const int k = q % P.nu, m = q / P.nu;
    const double du = P.u[k] - U, dv = P.v[m] - V;
    const double gh = G * exp(-lam * (du * du + dv * dv));
    dst[q] = split4(gh, bf * gh);
  }
  if (threadIdx.x == 0) {
    const int w = wcell(P, i, j);
    W[w] = rho;
    W[nwe + w] = rho * U;
    W[2 * nwe + w] = rho * V;
    W[3 * nwe + w] = rho * (0.5 * (U * U + V * V) + (P.K + 2) / (4.0 * lam));
  }
}

// -------------------------------------------------------------------------------------
// S1 + S7 in double-FP32: the FP64 form's sums kernel (sums_body) with every velocity-cell
// operation in double-FP32; the face sums each lane owns are accumulated in double-FP32
// registers over velocity chunks and converted to FP64 once per cell.  The slopes of every
// cell whose sums are formed go to the slope buffer (two DF4 per velocity-cell: r_x and r_y
// of h and b) for the face-flux kernel.
// -------------------------------------------------------------------------------------
// The per-lane sums of one half of the v axis (a_n, ab_n, x_n, xb_n, y_n, yb_n as in sums_body).
struct SumsHalfDF {
  df a0, a1, a2, a3, ab0, ab1, x0, x1, x2, x3, xb0, xb1, y0, y1, y2, y3, y4, yb0, yb1, yb2;
};
// Close a half (north: the N side, else S): its 16 face sums reduced over the warp into
// `side` (lanes < 16), and its sums added to the totals of the x sides.  Not inlined: one copy
// of this long reduction serves both halves (the kernel's code otherwise misses the
// instruction cache).
__device__ __noinline__ void close_half_df(const SumsHalfDF& h, df u, df wu, df cu, df tdx, df tdy, bool north,
                                           int lane, df& side, df* tot) {
  auto pm = [&](df a, df y) { return north ? df_add(a, y) : df_sub(a, y); };
  const df P0 = pm(h.a0, h.y0), P1 = pm(h.a1, h.y1), P2 = pm(h.a2, h.y2), P3 = pm(h.a3, h.y3);
  const df Pb0 = pm(h.ab0, h.yb0), Pb1 = pm(h.ab1, h.yb1);
  const df Z1 = df_fma(cu, h.x1, df_mul(tdy, h.y2)), Z2 = df_fma(cu, h.x2, df_mul(tdy, h.y3));
  const df Z3 = df_fma(cu, h.x3, df_mul(tdy, h.y4)), Zb1 = df_fma(cu, h.xb1, df_mul(tdy, h.yb2));
  const df uu = df_mul(u, u);
  // (uu A + B)/2 + C/2
  auto e4 = [&](df A, df B, df C) { return df_half(df_add(df_fma(uu, A, B), C)); };
  df v[16];
  v[0] = df_mul(wu, P0);
  v[1] = df_mul(df_mul(wu, u), P0);
  v[2] = df_mul(wu, P1);
  v[3] = df_mul(wu, e4(P0, P2, Pb0));
  const df ws = df_mul(wu, tdx);
  v[4] = df_mul(ws, h.x0);
  v[5] = df_mul(df_mul(ws, u), h.x0);
  v[6] = df_mul(ws, h.x1);
  v[7] = df_mul(ws, e4(h.x0, h.x2, h.xb0));
  v[8] = df_mul(wu, P1);
  v[9] = df_mul(df_mul(wu, u), P1);
  v[10] = df_mul(wu, P2);
  v[11] = df_mul(wu, e4(P1, P3, Pb1));
  v[12] = df_mul(wu, Z1);
  v[13] = df_mul(df_mul(wu, u), Z1);
  v[14] = df_mul(wu, Z2);
  v[15] = df_mul(wu, e4(Z1, Z3, Zb1));
  const df r = warp_reduce_scatter_df<16>(v, lane);
  if (lane < 16) side = df_add(side, r);
  const df add[kSumsTotals] = {h.a0, h.a1, h.a2, h.ab0, h.x0, h.x1, h.x2, h.xb0, h.y0, h.y1, h.y2, h.y3, h.yb0, h.yb1};
#pragma unroll
  for (int t = 0; t < kSumsTotals; t++) tot[t] = df_add(tot[t], add[t]);
}

// The face sums of the x sides from the totals over both halves (E: u > 0 with f + r_x,
// W: u < 0 with f - r_x, u = 0 half to each), reduced over the warp: entry `lane`.
__device__ __noinline__ df x_sums_df(const df* tot, df u, df wu, df cu, df tdy, int lane) {
  const df tA0 = tot[0], tA1 = tot[1], tA2 = tot[2], tAb = tot[3], tR0 = tot[4], tR1 = tot[5];
  const df tR2 = tot[6], tRb = tot[7], tC0 = tot[8], tC1 = tot[9], tC2 = tot[10], tC3 = tot[11];
  const df tCb0 = tot[12], tCb1 = tot[13];
  const df D0 = df_fma(cu, tR0, df_mul(tdy, tC1)), D1 = df_fma(cu, tR1, df_mul(tdy, tC2));
  const df D2 = df_fma(cu, tR2, df_mul(tdy, tC3)), Db = df_fma(cu, tRb, df_mul(tdy, tCb1));
  const bool upos = u.hi > 0.f, uneg = u.hi < 0.f;
  const df uu = df_mul(u, u);
  auto e4 = [&](df A, df B, df C) { return df_half(df_add(df_fma(uu, A, B), C)); };
  df xv[32];
#pragma unroll
  for (int sd = 0; sd < 2; sd++) {
    // weight: wu on the upwind side, wu/2 on both sides for u = 0, 0 otherwise
    const bool full = sd == 0 ? upos : uneg, none = sd == 0 ? uneg : upos;
    const df wgt = none ? df_zero() : (full ? wu : df_half(wu));
    auto pmx = [&](df a, df x) { return sd == 0 ? df_add(a, x) : df_sub(a, x); };
    const df F0 = pmx(tA0, tR0), F1 = pmx(tA1, tR1), F2 = pmx(tA2, tR2), Fb = pmx(tAb, tRb);
    df* o = xv + 16 * sd;
    const df wgu = df_mul(wgt, u);
    o[0] = df_mul(wgt, F0);
    o[1] = df_mul(wgu, F0);
    o[2] = df_mul(wgt, F1);
    o[3] = df_mul(wgt, e4(F0, F2, Fb));
    const df ws = df_mul(wgt, tdy);
    o[4] = df_mul(ws, tC0);
    o[5] = df_mul(df_mul(ws, u), tC0);
    o[6] = df_mul(ws, tC1);
    o[7] = df_mul(ws, e4(tC0, tC2, tCb0));
    o[8] = df_mul(wgu, F0);
    o[9] = df_mul(df_mul(wgu, u), F0);
    o[10] = df_mul(wgu, F1);
    o[11] = df_mul(wgu, e4(F0, F2, Fb));
    o[12] = df_mul(wgu, D0);
    o[13] = df_mul(df_mul(wgu, u), D0);
    o[14] = df_mul(wgu, D1);
    o[15] = df_mul(wgu, e4(D0, D2, Db));
  }
  return warp_reduce_scatter_df<32>(xv, lane);
}

__global__ void __launch_bounds__(128) k_sums_df(Params P, const DF4* __restrict__ f,
                                                 double* __restrict__ sums, DF4* __restrict__ slopes) {
  const int nv = P.nv, nu = P.nu, nq = P.nq;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncx = P.nx + 2;
  const int cell = blockIdx.x * kWarpsPerBlock + warp;
  if (cell >= ncx * (P.ny + 2)) return;
  const int i = cell % ncx - 1, j = cell / ncx - 1;
  const bool xg = i < 0 || i >= P.nx, yg = j < 0 || j >= P.ny;
  if (xg && yg) return;
  if ((i < 0 && P.bc_kind[0] == 1) || (i >= P.nx && P.bc_kind[1] == 1) ||
      (j < 0 && P.bc_kind[2] == 1) || (j >= P.ny && P.bc_kind[3] == 1))
    return;
  const bool zs = (i < 0 && P.bc_kind[0] == 2) || (i >= P.nx && P.bc_kind[1] == 2) ||
                  (j < 0 && P.bc_kind[2] == 2) || (j >= P.ny && P.bc_kind[3] == 2);
  const DF4* fc = f + fcell(P, i, j) * nq;
  const long rs = (long)P.ex * nq;
  DF4* slc = slopes + (size_t)wcell(P, i, j) * nq * 2;
  const df tdx = dfv(P.df_tdx), tdy = dfv(P.df_tdy);
  const float2* tu = P.gdf;                 // u[nu]
  const float2* twu = P.gdf + nu;           // wu[nu]
  const float2* twn = P.gdf + 2 * nu + nv;  // [5][nv] wv v^n
  const int mneg = P.m_neg, mpos = P.m_pos;
  const bool v0 = mpos > mneg;
  df ox = df_zero(), on = df_zero(), os = df_zero();  // owned face sums: E/W `lane`, N, S

  for (int k0 = 0; k0 < nu; k0 += 32) {
    const int k = k0 + lane;
    const bool act = k < nu;
    const int kk = act ? k : nu - 1;
    const df u = dfv(tu[kk]);
    const df wu = act ? dfv(twu[kk]) : df_zero();
    const df cu = df_mul(u, tdx);
    df a0, a1, a2, a3, ab0, ab1, x0, x1, x2, x3, xb0, xb1, y0, y1, y2, y3, y4, yb0, yb1, yb2;
    // totals over both halves for the x sides: A0 A1 A2 Ab R0 R1 R2 Rb C0 C1 C2 C3 Cb0 Cb1
    df tot[kSumsTotals];
#pragma unroll
    for (int t = 0; t < kSumsTotals; t++) tot[t] = df_zero();
    auto zero = [&]() {
      a0 = a1 = a2 = a3 = ab0 = ab1 = x0 = x1 = x2 = x3 = xb0 = xb1 = df_zero();
      y0 = y1 = y2 = y3 = y4 = yb0 = yb1 = yb2 = df_zero();
    };
    // slopes of row m and the cell value
    auto slopes_of = [&](int m, df& rxh, df& rxb, df& ryh, df& ryb, DF4& c) {
      const DF4* src = fc + (size_t)m * nu + kk;
      c = src[0];
      if (zs) {
        rxh = rxb = ryh = ryb = df_zero();
      } else {
        const DF4 w = src[-(long)nq], e = src[nq], s = src[-rs], n = src[rs];
        rxh = vl_df(dh(w), dh(c), dh(e));
        rxb = vl_df(db(w), db(c), db(e));
        ryh = vl_df(dh(s), dh(c), dh(n));
        ryb = vl_df(db(s), db(c), db(n));
      }
      if (act) {
        DF4* q = slc + 2 * ((size_t)m * nu + k);
        q[0] = mk4(rxh, rxb);
        q[1] = mk4(ryh, ryb);
      }
    };
    auto rows = [&](int m0, int m1) {
#pragma unroll 1
      for (int m = m0; m < m1; m++) {
        df rxh, rxb, ryh, ryb;
        DF4 c;
        slopes_of(m, rxh, rxb, ryh, ryb, c);
        const df w0 = dfv(twn[m]), w1 = dfv(twn[nv + m]), w2 = dfv(twn[2 * nv + m]);
        const df w3 = dfv(twn[3 * nv + m]), w4 = dfv(twn[4 * nv + m]);
        const df ch = dh(c), cb = db(c);
        a0 = df_acc(a0, w0, ch); a1 = df_acc(a1, w1, ch); a2 = df_acc(a2, w2, ch); a3 = df_acc(a3, w3, ch);
        ab0 = df_acc(ab0, w0, cb); ab1 = df_acc(ab1, w1, cb);
        x0 = df_acc(x0, w0, rxh); x1 = df_acc(x1, w1, rxh); x2 = df_acc(x2, w2, rxh); x3 = df_acc(x3, w3, rxh);
        xb0 = df_acc(xb0, w0, rxb); xb1 = df_acc(xb1, w1, rxb);
        y0 = df_acc(y0, w0, ryh); y1 = df_acc(y1, w1, ryh); y2 = df_acc(y2, w2, ryh);
        y3 = df_acc(y3, w3, ryh); y4 = df_acc(y4, w4, ryh);
        yb0 = df_acc(yb0, w0, ryb); yb1 = df_acc(yb1, w1, ryb); yb2 = df_acc(yb2, w2, ryb);
      }
    };
    auto row_v0 = [&](int m) {  // v = 0: only the w_0 sums, half weight
      df rxh, rxb, ryh, ryb;
      DF4 c;
      slopes_of(m, rxh, rxb, ryh, ryb, c);
      const df hw = df_half(dfv(twn[m]));
      a0 = df_acc(a0, hw, dh(c)); ab0 = df_acc(ab0, hw, db(c));
      x0 = df_acc(x0, hw, rxh); xb0 = df_acc(xb0, hw, rxb);
      y0 = df_acc(y0, hw, ryh); yb0 = df_acc(yb0, hw, ryb);
    };
    // close a half: its face sums, then add it to the totals
    auto close = [&](bool north, df& side) {
      const SumsHalfDF h = {df_norm(a0), df_norm(a1), df_norm(a2), df_norm(a3), df_norm(ab0),
                            df_norm(ab1), df_norm(x0), df_norm(x1), df_norm(x2), df_norm(x3),
                            df_norm(xb0), df_norm(xb1), df_norm(y0), df_norm(y1), df_norm(y2),
                            df_norm(y3), df_norm(y4), df_norm(yb0), df_norm(yb1), df_norm(yb2)};
      close_half_df(h, u, wu, cu, tdx, tdy, north, lane, side, tot);
    };
    zero();
    rows(0, mneg);
    if (v0) row_v0(mneg);
    close(false, os);
    zero();
    if (v0) row_v0(mneg);
    rows(mpos, nv);
    close(true, on);
    ox = df_add(ox, x_sums_df(tot, u, wu, cu, tdy, lane));
  }
  double* out = sums + (size_t)cell * kNSum;
  out[kSumE + lane] = to_double(ox);  // lanes 0..15: E side, 16..31: W side
  if (lane < 16) {
    out[kSumN + lane] = to_double(on);
    out[kSumS + lane] = to_double(os);
  }
}

// -------------------------------------------------------------------------------------
// S6 + S8 in double-FP32: the FP64 form's face-flux kernel (k_face_flux) -- one warp per
// interior cell, lane = u index, the v loop split at v = 0; the cell forms the micro flux
// X = Q g + Mt4 f_up - Mt5 d of its downwind x- and y-face for every velocity (and of the
// ghost- or wall-side faces of a boundary cell) into the face-flux buffers, from its slopes in
// the slope buffer and the double-FP32 face records.  The Maxwellian factors come from
// df_exp; nothing here runs on the FP64 pipe.
// -------------------------------------------------------------------------------------
__device__ __forceinline__ df neg_lam_sq(df lam, df d) { return df_neg(df_mul(lam, df_mul(d, d))); }

// Q in v for fixed u on an x face (un = u, ut = v) or a y face (un = v, ut = u), double-FP32
__device__ __forceinline__ void poly_v_df(const float2* c, df u, bool xface, df* q) {
  if (xface) {
    q[0] = df_fma(u, df_fma(u, df_fma(u, dfv(c[6]), dfv(c[3])), dfv(c[1])), dfv(c[0]));
    q[1] = df_fma(u, df_fma(u, dfv(c[7]), dfv(c[4])), dfv(c[2]));
    q[2] = df_fma(u, dfv(c[6]), dfv(c[5]));
    q[3] = dfv(c[7]);
  } else {
    q[0] = df_fma(u, df_fma(u, df_fma(u, dfv(c[7]), dfv(c[5])), dfv(c[2])), dfv(c[0]));
    q[1] = df_fma(u, df_fma(u, dfv(c[6]), dfv(c[4])), dfv(c[1]));
    q[2] = df_fma(u, dfv(c[7]), dfv(c[3]));
    q[3] = dfv(c[6]);
  }
}
__device__ __forceinline__ df horner3_df(const df* q, df v) {
  return df_fma(df_fma(df_fma(q[3], v, q[2]), v, q[1]), v, q[0]);
}

struct FaceKD {
  df Mt4, Mt5, bf;
  int wall;
};

__global__ void __launch_bounds__(128) k_face_flux_df(Params P, const DF4* __restrict__ f,
                                                      const FaceRecD* __restrict__ fxr,
                                                      const FaceRecD* __restrict__ fyr,
                                                      const DF4* __restrict__ sl, DF4* __restrict__ Xx,
                                                      DF4* __restrict__ Xy) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nv = P.nv, nu = P.nu, nq = P.nq, nx = P.nx, ny = P.ny;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float2* tu = P.gdf;
  const float2* tv = P.gdf + 2 * nu;
  df* ev = reinterpret_cast<df*>(smraw) + warp * 4 * nv;  // [4][nv]: x W, x E, y S, y N factors in v
  const int cell = blockIdx.x * kWarpsPerBlock + warp;
  if (cell >= nx * ny) return;
  const int i = cell % nx, j = cell / nx;
  const FaceRecD& RW = fxr[(size_t)j * (nx + 1) + i];
  const FaceRecD& RE = fxr[(size_t)j * (nx + 1) + i + 1];
  const FaceRecD& RS = fyr[(size_t)j * nx + i];
  const FaceRecD& RN = fyr[(size_t)(j + 1) * nx + i];
  for (int m = lane; m < nv; m += 32) {
    const df vv = dfv(tv[m]);
    ev[0 * nv + m] = df_exp(neg_lam_sq(dfv(RW.lam), df_sub(vv, dfv(RW.Ut))));  // x faces: ut = v
    ev[1 * nv + m] = df_exp(neg_lam_sq(dfv(RE.lam), df_sub(vv, dfv(RE.Ut))));
    ev[2 * nv + m] = df_exp(neg_lam_sq(dfv(RS.lam), df_sub(vv, dfv(RS.Un))));  // y faces: un = v
    ev[3 * nv + m] = df_exp(neg_lam_sq(dfv(RN.lam), df_sub(vv, dfv(RN.Un))));
  }
  __syncwarp();
  auto faceK = [](const FaceRecD& R) { return FaceKD{dfv(R.Mt4), dfv(R.Mt5), dfv(R.bfac), R.wall}; };
  const FaceKD KW = faceK(RW), KE = faceK(RE), KS = faceK(RS), KN = faceK(RN);
  const df tdx = dfv(P.df_tdx), tdy = dfv(P.df_tdy), dtT = dfv(P.df_dt);
  const long rs = (long)P.ex * nq;
  const DF4* fc0 = f + fcell(P, i, j) * nq;
  const DF4* sl0 = sl + (size_t)wcell(P, i, j) * nq * 2;  // this cell's slopes
  DF4* xw0 = Xx + ((size_t)j * (nx + 1) + i) * nq;        // W face of the cell; E face: + nq
  DF4* ys0 = Xy + ((size_t)j * nx + i) * nq;              // S face; N face: + nx nq
  const bool pW = P.bc_kind[0] == 2, pE = P.bc_kind[1] == 2, pS = P.bc_kind[2] == 2, pN = P.bc_kind[3] == 2;

  // X of a face for the two velocities of a lane (packed): face value (fh, fb) and slope term
  // (dh_, db_) of its upwind side; inc: the gas side is upwind (a wall face then passes
  // dt f_up, else dt g_wall)
  const df2 dt2 = df2_bcast(dtT);
  bool act_ = false;  // this lane's u index is a real one (set per chunk of 32 u)
  auto flux = [&](const FaceKD& F, const df (&qh)[4], const df (&qb)[4], df2 vv, df2 g, df2 fh, df2 fb,
                  df2 dh_, df2 db_, bool inc, df2& xh, df2& xb) {
    if (F.wall) {
      xh = inc ? df2_mul(dt2, fh) : df2_mul(dt2, g);
      xb = inc ? df2_mul(dt2, fb) : df2_mul(dt2, df2_mul(df2_bcast(F.bf), g));
      return;
    }
    auto horner = [&](const df (&q)[4]) {
      return df2_fma(df2_fma(df2_fma(df2_bcast(q[3]), vv, df2_bcast(q[2])), vv, df2_bcast(q[1])), vv,
                     df2_bcast(q[0]));
    };
    const df2 m4 = df2_bcast(F.Mt4), m5 = df2_bcast(F.Mt5);
    xh = df2_sub(df2_fma(horner(qh), g, df2_mul(m4, fh)), df2_mul(m5, dh_));
    xb = df2_sub(df2_fma(horner(qb), g, df2_mul(m4, fb)), df2_mul(m5, db_));
  };
  // store the pair of a face's fluxes: row A always, row B when it is a real row
  auto put = [&](DF4* base, size_t qA, size_t qB, bool hasB, df2 xh, df2 xb) {
    if (!act_) return;
    base[qA] = mk4(df2_x(xh), df2_x(xb));
    if (hasB) base[qB] = mk4(df2_y(xh), df2_y(xb));
  };
  auto gfac = [](const FaceRecD& R, df u, float2 U) {
    return df_mul(dfv(R.G), df_exp(neg_lam_sq(dfv(R.lam), df_sub(u, dfv(U)))));
  };

  for (int k0 = 0; k0 < nu; k0 += 32) {
    const int k = k0 + lane;
    const bool act = k < nu;
    const int kk = act ? k : nu - 1;
    act_ = act;
    const df u = dfv(tu[kk]);
    df gu[4];
    gu[0] = gfac(RW, u, RW.Un);
    gu[1] = gfac(RE, u, RE.Un);
    gu[2] = gfac(RS, u, RS.Ut);
    gu[3] = gfac(RN, u, RN.Ut);
    const bool up = u.hi > 0.f;     // downwind x-face: E for u > 0, W otherwise
    const int xs = up ? 0 : 1;      // upwind side of the x-face records
    const FaceRecD& RXd = up ? RE : RW;
    const FaceRecD& RXg = up ? RW : RE;
    const FaceKD KXd = up ? KE : KW, KXg = up ? KW : KE;
    const df gXd = up ? gu[1] : gu[0], gXg = up ? gu[0] : gu[1];
    const df* evXd = ev + (up ? nv : 0);
    const df* evXg = ev + (up ? 0 : nv);
    DF4* xd0 = up ? xw0 + nq : xw0;
    DF4* xg0 = up ? xw0 : xw0 + nq;
    df qX[2][4];
#pragma unroll
    for (int c = 0; c < 2; c++) poly_v_df(RXd.Q[xs][c], u, true, qX[c]);
    const long xo = up ? -(long)nq : (long)nq;  // x-upwind neighbour in f, in q
    const bool xg = up ? i == 0 : i == nx - 1;  // it is a ghost cell (or a wall)
    const bool xz = (up && i == 0 && pW) || (!up && i == nx - 1 && pE);
    const df cu = df_mul(u, tdx);

    auto half = [&](auto vup_tag, int m0, int m1) {
      constexpr bool VUP = decltype(vup_tag)::value;  // downwind y-face: N for v > 0, S otherwise
      constexpr int ys = VUP ? 0 : 1;
      const FaceRecD& RYd = VUP ? RN : RS;
      const FaceRecD& RYg = VUP ? RS : RN;
      const FaceKD& KYd = VUP ? KN : KS;
      const FaceKD& KYg = VUP ? KS : KN;
      const df gYd = VUP ? gu[3] : gu[2], gYg = VUP ? gu[2] : gu[3];
      const df* evYd = ev + (VUP ? 3 : 2) * nv;
      const df* evYg = ev + (VUP ? 2 : 3) * nv;
      DF4* yd0 = VUP ? ys0 + (size_t)nx * nq : ys0;
      DF4* yg0 = VUP ? ys0 : ys0 + (size_t)nx * nq;
      df qY[2][4];
#pragma unroll
      for (int c = 0; c < 2; c++) poly_v_df(RYd.Q[ys][c], u, false, qY[c]);
      const long yo = VUP ? -rs : rs;                             // y-upwind neighbour in f
      const long yso = VUP ? -(long)P.wx * nq : (long)P.wx * nq;  // ... in the slope buffer
      const bool yg = VUP ? j == 0 : j == ny - 1;
      const bool yz = (VUP && j == 0 && pS) || (!VUP && j == ny - 1 && pN);
      // two rows at a time (packed pairs; an odd last row is paired with itself)
      for (int m = m0; m < m1; m += 2) {
        const bool hasB = m + 1 < m1;
        const int mB = hasB ? m + 1 : m;
        const df2 vv = df2_of(dfv(tv[m]), dfv(tv[mB]));
        const size_t qA = (size_t)m * nu + kk, qB = (size_t)mB * nu + kk;
        const DF4* pA = fc0 + qA;
        const DF4* pB = fc0 + qB;
        const DF4 cA = pA[0], cB = pB[0];
        const DF4* sA = sl0 + 2 * qA;
        const DF4* sB = sl0 + 2 * qB;
        const DF4 aA = sA[0], bA = sA[1], aB = sB[0], bB = sB[1];  // half slopes r_x, r_y
        const df2 ch = df2_of(dh(cA), dh(cB)), cb = df2_of(db(cA), db(cB));
        const df2 axh = df2_of(dh(aA), dh(aB)), axb = df2_of(db(aA), db(aB));
        const df2 ayh = df2_of(dh(bA), dh(bB)), ayb = df2_of(db(bA), db(bB));
        const df2 cv = df2_mul(vv, df2_bcast(tdy));
        const df2 cu2 = df2_bcast(cu);
        const df2 dch = df2_fma(cu2, axh, df2_mul(cv, ayh)), dcb = df2_fma(cu2, axb, df2_mul(cv, ayb));
        df2 xh, xb;
        // downwind x face: f_up = f + r_x (u > 0) or f - r_x (u < 0)
        flux(KXd, qX[0], qX[1], vv, df2_mul(df2_bcast(gXd), df2_of(evXd[m], evXd[mB])),
             up ? df2_add(ch, axh) : df2_sub(ch, axh), up ? df2_add(cb, axb) : df2_sub(cb, axb), dch, dcb,
             true, xh, xb);
        put(xd0, qA, qB, hasB, xh, xb);
        if (xg) {
          const DF4 xuA = pA[xo], xuB = pB[xo];
          DF4 auA = sA[2 * xo], buA = sA[2 * xo + 1], auB = sB[2 * xo], buB = sB[2 * xo + 1];
          if (xz) auA = buA = auB = buB = mk4(df_zero(), df_zero());
          const df2 uxh = df2_of(dh(auA), dh(auB)), uxb = df2_of(db(auA), db(auB));
          const df2 uyh = df2_of(dh(buA), dh(buB)), uyb = df2_of(db(buA), db(buB));
          const df2 duh = df2_fma(cu2, uxh, df2_mul(cv, uyh)), dub = df2_fma(cu2, uxb, df2_mul(cv, uyb));
          const df2 gh_ = df2_of(dh(xuA), dh(xuB)), gb_ = df2_of(db(xuA), db(xuB));
          df qg[2][4];
#pragma unroll
          for (int cc = 0; cc < 2; cc++) poly_v_df(RXg.Q[xs][cc], u, true, qg[cc]);
          flux(KXg, qg[0], qg[1], vv, df2_mul(df2_bcast(gXg), df2_of(evXg[m], evXg[mB])),
               up ? df2_add(gh_, uxh) : df2_sub(gh_, uxh), up ? df2_add(gb_, uxb) : df2_sub(gb_, uxb), duh,
               dub, false, xh, xb);
          put(xg0, qA, qB, hasB, xh, xb);
        }
        // downwind y face: f_up = f + r_y (v > 0) or f - r_y (v < 0)
        flux(KYd, qY[0], qY[1], vv, df2_mul(df2_bcast(gYd), df2_of(evYd[m], evYd[mB])),
             VUP ? df2_add(ch, ayh) : df2_sub(ch, ayh), VUP ? df2_add(cb, ayb) : df2_sub(cb, ayb), dch, dcb,
             true, xh, xb);
        put(yd0, qA, qB, hasB, xh, xb);
        if (yg) {
          const DF4 yuA = pA[yo], yuB = pB[yo];
          DF4 avA = sA[2 * yso], bvA = sA[2 * yso + 1], avB = sB[2 * yso], bvB = sB[2 * yso + 1];
          if (yz) avA = bvA = avB = bvB = mk4(df_zero(), df_zero());
          const df2 vxh = df2_of(dh(avA), dh(avB)), vxb = df2_of(db(avA), db(avB));
          const df2 vyh = df2_of(dh(bvA), dh(bvB)), vyb = df2_of(db(bvA), db(bvB));
          const df2 dvh = df2_fma(cu2, vxh, df2_mul(cv, vyh)), dvb = df2_fma(cu2, vxb, df2_mul(cv, vyb));
          const df2 gh_ = df2_of(dh(yuA), dh(yuB)), gb_ = df2_of(db(yuA), db(yuB));
          df qg[2][4];
#pragma unroll
          for (int cc = 0; cc < 2; cc++) poly_v_df(RYg.Q[ys][cc], u, false, qg[cc]);
          flux(KYg, qg[0], qg[1], vv, df2_mul(df2_bcast(gYg), df2_of(evYg[m], evYg[mB])),
               VUP ? df2_add(gh_, vyh) : df2_sub(gh_, vyh), VUP ? df2_add(gb_, vyb) : df2_sub(gb_, vyb),
               dvh, dvb, false, xh, xb);
          put(yg0, qA, qB, hasB, xh, xb);
        }
      }
    };
    half(std::integral_constant<bool, false>{}, 0, P.m_pos);
    half(std::integral_constant<bool, true>{}, P.m_pos, nv);
  }
}

// Eq. 3 in double-FP32 from the four face fluxes of each velocity-cell (the FP64 form's
// k_cell_update): f^{n+1} = f^n + inv [flux + cg1 (g^{n+1} - f^n) + cgn (g^n - f^n)].
__global__ void __launch_bounds__(128) k_cell_update_df(Params P, const DF4* __restrict__ f,
                                                        DF4* __restrict__ fo,
                                                        const CellRecD* __restrict__ cr,
                                                        const DF4* __restrict__ Xx,
                                                        const DF4* __restrict__ Xy) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nv = P.nv, nu = P.nu, nq = P.nq, nx = P.nx, ny = P.ny;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float2* tu = P.gdf;
  const float2* tv = P.gdf + 2 * nu;
  df* ev = reinterpret_cast<df*>(smraw) + warp * 2 * nv;  // [2][nv]: g^n, g^{n+1} factors in v
  const int cell = blockIdx.x * kWarpsPerBlock + warp;
  if (cell >= nx * ny) return;
  const int i = cell % nx, j = cell / nx;
  const CellRecD& C = cr[cell];
  for (int m = lane; m < nv; m += 32) {
    const df vv = dfv(tv[m]);
    ev[m] = df_exp(neg_lam_sq(dfv(C.lamn), df_sub(vv, dfv(C.Vn))));
    ev[nv + m] = df_exp(neg_lam_sq(dfv(C.lam1), df_sub(vv, dfv(C.V1))));
  }
  __syncwarp();
  const df inv = dfv(C.inv), cg1 = dfv(C.cg1), cgn = dfv(C.cgn);
  const df cg1b = df_mul(cg1, dfv(C.b1)), cgnb = df_mul(cgn, dfv(C.bn));
  const df idx = dfv(P.df_idx), idy = dfv(P.df_idy);
  const DF4* fc0 = f + fcell(P, i, j) * nq;
  DF4* fo0 = fo + fcell(P, i, j) * nq;
  const DF4* xw0 = Xx + ((size_t)j * (nx + 1) + i) * nq;
  const DF4* ys0 = Xy + ((size_t)j * nx + i) * nq;
  for (int k0 = 0; k0 < nu; k0 += 32) {
    const int k = k0 + lane;
    const bool act = k < nu;
    const int kk = act ? k : nu - 1;
    const df u = dfv(tu[kk]);
    const df gun = df_mul(dfv(C.Gn), df_exp(neg_lam_sq(dfv(C.lamn), df_sub(u, dfv(C.Un)))));
    const df gu1 = df_mul(dfv(C.G1), df_exp(neg_lam_sq(dfv(C.lam1), df_sub(u, dfv(C.U1)))));
    const df2 fxu = df2_bcast(df_mul(u, idx));
    const df2 gun2 = df2_bcast(gun), gu12 = df2_bcast(gu1);
    const df2 inv2 = df2_bcast(inv), cg12 = df2_bcast(cg1), cgn2 = df2_bcast(cgn);
    const df2 cg1b2 = df2_bcast(cg1b), cgnb2 = df2_bcast(cgnb);
    // two rows at a time (packed pairs; an odd last row is paired with itself)
    for (int m = 0; m < nv; m += 2) {
      const bool hasB = m + 1 < nv;
      const int mB = hasB ? m + 1 : m;
      const df2 fyv = df2_mul(df2_of(dfv(tv[m]), dfv(tv[mB])), df2_bcast(idy));
      const size_t qA = (size_t)m * nu + kk, qB = (size_t)mB * nu + kk;
      const DF4 cA = fc0[qA], cB = fc0[qB];
      const DF4 WA = xw0[qA], EA = xw0[nq + qA], SA = ys0[qA], NA = ys0[(size_t)nx * nq + qA];
      const DF4 WB = xw0[qB], EB = xw0[nq + qB], SB = ys0[qB], NB = ys0[(size_t)nx * nq + qB];
      const df2 flh = df2_fma(fxu, df2_sub(df2_of(dh(WA), dh(WB)), df2_of(dh(EA), dh(EB))),
                              df2_mul(fyv, df2_sub(df2_of(dh(SA), dh(SB)), df2_of(dh(NA), dh(NB)))));
      const df2 flb = df2_fma(fxu, df2_sub(df2_of(db(WA), db(WB)), df2_of(db(EA), db(EB))),
                              df2_mul(fyv, df2_sub(df2_of(db(SA), db(SB)), df2_of(db(NA), db(NB)))));
      const df2 gnh = df2_mul(gun2, df2_of(ev[m], ev[mB])), g1h = df2_mul(gu12, df2_of(ev[nv + m], ev[nv + mB]));
      const df2 ch = df2_of(dh(cA), dh(cB)), cb = df2_of(db(cA), db(cB));
      const df2 dhh = df2_mul(inv2, df2_add(flh, df2_add(df2_mul(cg12, df2_sub(g1h, ch)),
                                                         df2_mul(cgn2, df2_sub(gnh, ch)))));
      const df2 dbb = df2_mul(inv2, df2_add(flb, df2_add(df2_sub(df2_mul(cg1b2, g1h), df2_mul(cg12, cb)),
                                                         df2_sub(df2_mul(cgnb2, gnh), df2_mul(cgn2, cb)))));
      const df2 nh = df2_add(ch, dhh), nb = df2_add(cb, dbb);
      if (act) {
        fo0[qA] = mk4(df2_x(nh), df2_x(nb));
        if (hasB) fo0[qB] = mk4(df2_y(nh), df2_y(nb));
      }
    }
  }
}

}  // namespace ugks
