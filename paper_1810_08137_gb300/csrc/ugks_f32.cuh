// FP32-f form of the step (FP32 f; FP64 W, cell scalars and first-order interface terms) in
// the paired-row layout: ghost fill, the per-cell velocity sums of S1 + S7, and the upwind
// strip walk of S6, S8 and Eq. 3 (Liu, Hu & Li, arXiv:1810.08137, Sec. 2), plus state
// conversion and initialisation.  The interface (S2-S5) and cell (Eq. 4) kernels are shared with the FP64
// form and write the FP32 records read here.
//
// Layout.  The v axis is split into its v < 0 rows and its v >= 0 rows; each half is padded
// to an even number of rows by repeating its last row, and the padded rows are taken in
// pairs (pr_neg pairs with v < 0, then the v >= 0 pairs, pr_all in total).  A cell holds
// fs = pr_all * nu float4 slots; slot s = pr * nu + k holds (h, h', b, b') of padded rows
// 2 pr and 2 pr + 1 at u_k, stored as e = f - g_ref.  The thread that owns a slot owns two
// velocities with the same u and the same sign of v, so they walk the mesh in the same
// order, and its arithmetic on them runs as packed FP32 pairs (one instruction for both).
// Padded rows have zero quadrature weight: the walk updates them like any velocity and the
// sums never see them.
#pragma once

namespace ugks {

// ---- packed FP32 pairs (sm_100 family: one instruction for both lanes of a pair) ----
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, exactly as a single subtraction (b * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// (h, b) of the two velocities of a slot
struct P4 {
  float2 h, b;
};
__device__ __forceinline__ P4 ldp(const float4* p) {
  const float4 v = __ldg(p);
  return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ P4 ldp_s(const float4* p) {
  const float4 v = *p;
  return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void stp(float4* p, const P4& v) { *p = make_float4(v.h.x, v.h.y, v.b.x, v.b.y); }
__device__ __forceinline__ P4 add4(const P4& a, const P4& b) { return {add2(a.h, b.h), add2(a.b, b.b)}; }
__device__ __forceinline__ P4 zero4() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

// van Leer half slope r = d1 d2 / (d1 + d2) if d1 d2 > 0 else 0 (d1 = c - a, d2 = b - c),
// both velocities of a pair
__device__ __forceinline__ float2 vl_p(float2 a, float2 c, float2 b) {
  const float2 d1 = sub2(c, a), d2 = sub2(b, c);
  const float2 p = mul2(d1, d2);
  const float2 s = add2(d1, d2);
  const float2 q = mul2(p, make_float2(rcp_ftz(s.x), rcp_ftz(s.y)));
  return make_float2(p.x > 0.f ? q.x : 0.f, p.y > 0.f ? q.y : 0.f);
}
__device__ __forceinline__ P4 vl4(const P4& a, const P4& c, const P4& b) {
  return {vl_p(a.h, c.h, b.h), vl_p(a.b, c.b, b.b)};
}

// Real velocity row of padded row r (the pad of each half repeats the half's last row).
__host__ __device__ __forceinline__ int prow(const Params& P, int r) {
  const int rn = 2 * P.pr_neg;
  return r < rn ? (r < P.m_neg - 1 ? r : P.m_neg - 1)
                : P.m_neg + (r - rn < P.nv - P.m_neg - 1 ? r - rn : P.nv - P.m_neg - 1);
}
// Padded row of real row m.
__host__ __device__ __forceinline__ int padrow(const Params& P, int m) {
  return m < P.m_neg ? m : 2 * P.pr_neg + (m - P.m_neg);
}

// -------------------------------------------------------------------------------------
// Ghost ring (same rules as the FP64 form's fill_ghost_cell: pressure Maxwellian, periodic
// image, zero-gradient copy next to a wall), over the slots of the paired layout.
// -------------------------------------------------------------------------------------
__device__ void fill_ghost_cell(const Params& P, float4* f, double* W, int nwe, int gi, int gj,
                                int si, int sj, int side, bool write_W, int wi, int wj,
                                double* tab) {
  const int kind = P.bc_kind[side];
  float4* dst = f + fcell(P, gi, gj) * P.fs;
  const float4* src = f + fcell(P, si, sj) * P.fs;
  const int sw = wcell(P, wi, wj);
  if (kind == 2) {
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
      ru[k] = P.ref_G * exp(-P.ref_lam * dr * dr);
    }
    for (int m = threadIdx.x; m < P.nv; m += blockDim.x) {
      const double dv = P.v[m] - V, dr = P.v[m] - P.ref_V;
      fv[m] = exp(-lam * dv * dv);
      rv[m] = exp(-P.ref_lam * dr * dr);
    }
    __syncthreads();
    for (int s = threadIdx.x; s < P.fs; s += blockDim.x) {
      const int pr = s / P.nu, k = s - pr * P.nu;
      const int m0 = prow(P, 2 * pr), m1 = prow(P, 2 * pr + 1);
      const double g0 = fu[k] * fv[m0], r0 = ru[k] * rv[m0];
      const double g1 = fu[k] * fv[m1], r1 = ru[k] * rv[m1];
      dst[s] = make_float4((float)(g0 - r0), (float)(g1 - r1), (float)(bf * g0 - P.ref_bf * r0),
                           (float)(bf * g1 - P.ref_bf * r1));
    }
    if (write_W && threadIdx.x == 0) {
      const int g = wcell(P, gi, gj);
      W[g] = rho;
      W[nwe + g] = rho * U;
      W[2 * nwe + g] = rho * V;
      W[3 * nwe + g] = rho * (0.5 * (U * U + V * V) + (P.K + 2) / (4.0 * lam));
    }
  } else {
    for (int s = threadIdx.x; s < P.fs; s += blockDim.x) dst[s] = src[s];
    if (write_W && threadIdx.x == 0) {
      const int g = wcell(P, gi, gj), s = wcell(P, si, sj);
      for (int c = 0; c < 4; c++) W[c * nwe + g] = W[c * nwe + s];
    }
  }
}

// -------------------------------------------------------------------------------------
// S1 + S7: per-cell half-range velocity sums (the sums of the FP64 form's sums_body, same
// output layout, FP64), one warp per cell, lane = u index (chunks of 32), loop over row
// pairs.  Per lane and half of the v axis, with w_n = wv v^n, the weighted sums of the cell
// value c, the x half slope r_x and the y half slope r_y:
//   a_n = sum w_n c_h (n < 4), ab_n = sum w_n c_b (n < 2), x_n = sum w_n r_x,h (n < 4),
//   xb_n = sum w_n r_x,b (n < 2), y_n = sum w_n r_y,h (n < 5), yb_n = sum w_n r_y,b (n < 3),
// accumulated over both rows of each pair.
// Precision: these FP32 sums run over a chunk of at most kSumChunkPairs row pairs
// (2 kSumChunkPairs rows); at the end of each chunk the warp weights them by the lane's u
// terms and reduces them across its lanes in FP32, and each lane adds the face sums it owns
// (one E/W value, and for lanes < 16 one N and one S value) to FP64 accumulators.  So FP32
// rounding acts within a chunk of one warp (at most 2 kSumChunkPairs rows x 32 lanes of the
// deviation e = f - g_ref), and every sum across chunks, velocity chunks and halves is FP64.
// The v = 0 row (H(0) = 1/2) enters both halves with half weight: the weight table carries
// its half weight in the v >= 0 half and its part of the v < 0 half is added separately.
// -------------------------------------------------------------------------------------
constexpr int kSumChunkPairs = 4;  // row pairs (2 rows each) per FP32 chunk

// The chunk's contribution to the 16 face sums of the y side of its half (sy = +1: N side,
// -1: S side), from the per-lane FP32 chunk sums; summed over the warp, entry lane % 16.
__device__ __forceinline__ float chunk_y_sums(float u, float wu, float cu, float tdx, float tdy, float sy,
                                              float a0, float a1, float a2, float a3, float ab0, float ab1,
                                              float x0, float x1, float x2, float x3, float xb0, float xb1,
                                              float y0, float y1, float y2, float y3, float y4, float yb0,
                                              float yb1, float yb2, int lane) {
  // face values of the half: c -/+ r_y; free-transport slope sums: cu x_n + (2/dy) y_{n+1}
  const float P0 = a0 + sy * y0, P1 = a1 + sy * y1, P2 = a2 + sy * y2, P3 = a3 + sy * y3;
  const float Pb0 = ab0 + sy * yb0, Pb1 = ab1 + sy * yb1;
  const float Z1 = cu * x1 + tdy * y2, Z2 = cu * x2 + tdy * y3, Z3 = cu * x3 + tdy * y4;
  const float Zb1 = cu * xb1 + tdy * yb2;
  float v[16];
  const float uu = u * u;
  v[0] = wu * P0;
  v[1] = wu * u * P0;
  v[2] = wu * P1;
  v[3] = wu * (0.5f * (uu * P0 + P2) + 0.5f * Pb0);
  const float ws = wu * tdx;
  v[4] = ws * x0;
  v[5] = ws * u * x0;
  v[6] = ws * x1;
  v[7] = ws * (0.5f * (uu * x0 + x2) + 0.5f * xb0);
  v[8] = wu * P1;
  v[9] = wu * u * P1;
  v[10] = wu * P2;
  v[11] = wu * (0.5f * (uu * P1 + P3) + 0.5f * Pb1);
  v[12] = wu * Z1;
  v[13] = wu * u * Z1;
  v[14] = wu * Z2;
  v[15] = wu * (0.5f * (uu * Z1 + Z3) + 0.5f * Zb1);
  return warp_reduce_scatter<16>(v, lane);
}

// The chunk's contribution to the 32 face sums of the x sides (E: entries 0..15 from u > 0
// with f + r_x, W: 16..31 from u < 0 with f - r_x, u = 0 half to each); entry lane.
// A transpose reduce-scatter in which a lane's own values are laid out by its lane bits 4
// and 3, so that those two exchange levels need no selects: every lane forms the 16 entries
// of the side it keeps (W on lanes 16..31, E on lanes 0..15) and the 16 of the side it sends
// to lane ^ 16; and since entries 8..11 of a side are u times entries 0..3, a lane with bit 3
// set holds u times its entries 0..3 in slots 0..3 and the unscaled ones in slots 8..11.
__device__ __forceinline__ float chunk_x_sums(float u, float wu, float cu, float tdy,
                                              float a0, float a1, float a2, float ab0,
                                              float x0, float x1, float x2, float xb0,
                                              float y0, float y1, float y2, float y3, float yb0,
                                              float yb1, int lane) {
  const float D0 = cu * x0 + tdy * y1, D1 = cu * x1 + tdy * y2, D2 = cu * x2 + tdy * y3;
  const float Db = cu * xb0 + tdy * yb1;
  const float hE = u > 0.f ? 1.f : (u < 0.f ? 0.f : 0.5f);
  const float hW = u < 0.f ? 1.f : (u > 0.f ? 0.f : 0.5f);
  const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
  const float mk = up8 ? u : 1.f, ms = up8 ? 1.f : u;  // scales of slots 0..3 and 8..11
  const float uu = u * u;
  // the 16 entries of one side (sign sg of r_x, weight wgt), slots 0..3 / 8..11 as above
  auto side = [&](float sg, float wgt, float* o) {
    const float F0 = a0 + sg * x0, F1 = a1 + sg * x1, F2 = a2 + sg * x2, Fb = ab0 + sg * xb0;
    const float b0 = wgt * F0, b1 = wgt * u * F0, b2 = wgt * F1;
    const float b3 = wgt * (0.5f * (uu * F0 + F2) + 0.5f * Fb);
    o[0] = mk * b0; o[1] = mk * b1; o[2] = mk * b2; o[3] = mk * b3;
    o[8] = ms * b0; o[9] = ms * b1; o[10] = ms * b2; o[11] = ms * b3;
    const float ws = wgt * tdy;
    o[4] = ws * y0;
    o[5] = ws * u * y0;
    o[6] = ws * y1;
    o[7] = ws * (0.5f * (uu * y0 + y2) + 0.5f * yb0);
    const float wuu = wgt * u;
    o[12] = wuu * D0;
    o[13] = wuu * u * D0;
    o[14] = wuu * D1;
    o[15] = wuu * (0.5f * (uu * D0 + D2) + 0.5f * Db);
  };
  float kv[16], sv[16];
  side(up16 ? -1.f : 1.f, wu * (up16 ? hW : hE), kv);
  side(up16 ? 1.f : -1.f, wu * (up16 ? hE : hW), sv);
#pragma unroll
  for (int i = 0; i < 16; i++) kv[i] += __shfl_xor_sync(kFull, sv[i], 16);
#pragma unroll
  for (int i = 0; i < 4; i++) kv[i] += __shfl_xor_sync(kFull, kv[i + 8], 8);
#pragma unroll
  for (int i = 4; i < 8; i++) {
    const float send = up8 ? kv[i] : kv[i + 8];
    const float keep = up8 ? kv[i + 8] : kv[i];
    kv[i] = keep + __shfl_xor_sync(kFull, send, 8);
  }
#pragma unroll
  for (int o = 4; o >= 1; o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; i++) {
      const float send = upper ? kv[i] : kv[i + o];
      const float keep = upper ? kv[i + o] : kv[i];
      kv[i] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return kv[0];
}

// Shakhov model: the chunk's contribution to the raw heat-flux moments (the kNHeat layout:
// E and W face values, the y face values of the current half, the cell values), from the
// lane's FP32 chunk sums, reduced across the warp in FP32 like the other chunk sums: 43
// entries in two transpose reduce-scatters of 32; r1 = entry lane, r2 = entry 32 + lane.
// Entries: [0..9] E, [10..19] W (M20 M11 M02 M30 M21 M12 M03 B00 B10 B01 each), [20..29] the
// half's y side, [30..42] the cell (M00 M10 M01 M20 M11 M02 M30 M21 M12 M03 B00 B10 B01).
__device__ __forceinline__ void chunk_heat_sums(float u, float wu, float sy, float a0, float a1, float a2,
                                                float a3, float ab0, float ab1, float x0, float x1,
                                                float x2, float x3, float xb0, float xb1, float y0,
                                                float y1, float y2, float y3, float yb0, float yb1,
                                                int lane, float& r1, float& r2) {
  const float hE = u > 0.f ? 1.f : (u < 0.f ? 0.f : 0.5f);
  const float hW = u < 0.f ? 1.f : (u > 0.f ? 0.f : 0.5f);
  const float uu = u * u, u3 = uu * u;
  float e1[32], e2[32];
  auto side = [&](float w, float F0, float F1, float F2, float F3, float Fb0, float Fb1, float* o) {
    o[0] = w * uu * F0; o[1] = w * u * F1; o[2] = w * F2; o[3] = w * u3 * F0; o[4] = w * uu * F1;
    o[5] = w * u * F2; o[6] = w * F3; o[7] = w * Fb0; o[8] = w * u * Fb0; o[9] = w * Fb1;
  };
  const float wE = wu * hE, wW = wu * hW;
  side(wE, a0 + x0, a1 + x1, a2 + x2, a3 + x3, ab0 + xb0, ab1 + xb1, e1);
  side(wW, a0 - x0, a1 - x1, a2 - x2, a3 - x3, ab0 - xb0, ab1 - xb1, e1 + 10);
  side(wu, a0 + sy * y0, a1 + sy * y1, a2 + sy * y2, a3 + sy * y3, ab0 + sy * yb0, ab1 + sy * yb1, e1 + 20);
  e1[30] = wu * a0;
  e1[31] = wu * u * a0;
  e2[0] = wu * a1; e2[1] = wu * uu * a0; e2[2] = wu * u * a1; e2[3] = wu * a2; e2[4] = wu * u3 * a0;
  e2[5] = wu * uu * a1; e2[6] = wu * u * a2; e2[7] = wu * a3; e2[8] = wu * ab0; e2[9] = wu * u * ab0;
  e2[10] = wu * ab1;
#pragma unroll
  for (int t = 11; t < 32; t++) e2[t] = 0.f;
  r1 = warp_reduce_scatter<32>(e1, lane);
  r2 = warp_reduce_scatter<32>(e2, lane);
}

// Velocity-space split (split = 1, 2 or 4 warps per cell, the warps of one cell in one
// block): warp g of a cell's group takes the g-th of `split` contiguous ranges of row pairs in
// each half of the v axis, and the group's FP64 face sums are added in shared memory (`red`,
// kWarpsPerBlock x kNSum doubles) in the order g = 0, 1, ... by the group's first warp.  With
// split > 1 every warp of the block reaches the two block barriers, so the caller's block
// must be uniform in `split` (it is: a block's cells belong to one instance).
// SPLIT = false: one warp per cell (split 1), without the range and reduction code; the
// caller inlines it and calls the split instance as a function of its own (sums_body_split),
// so that the split path's registers do not weigh on the one-warp path.  SHK: the Shakhov
// model's heat-flux moments too (P.hs; one warp per cell, in sums_phase_shk).
template <bool SPLIT, bool SHK = false>
__device__ __forceinline__ void sums_body_p(const Params& P, const float4* __restrict__ f,
                                            double* __restrict__ sums, int bx, int split_,
                                            double (*red)[kNSum]) {
  const int nu = P.nu, fs = P.fs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncx = P.nx + 2;
  const int split = SPLIT ? split_ : 1;
  const int gw = bx * kWarpsPerBlock + warp;
  const int cell = SPLIT ? gw / split : gw, g = SPLIT ? gw - cell * split : 0;
  const int i = cell % ncx - 1, j = cell / ncx - 1;
  const bool xg = i < 0 || i >= P.nx, yg = j < 0 || j >= P.ny;
  // a cell whose sums are never read: corner ghosts, ghosts behind a wall, past the end
  const bool skip = cell >= ncx * (P.ny + 2) || (xg && yg) || (i < 0 && P.bc_kind[0] == 1) ||
                    (i >= P.nx && P.bc_kind[1] == 1) || (j < 0 && P.bc_kind[2] == 1) ||
                    (j >= P.ny && P.bc_kind[3] == 1);
  if (!SPLIT && skip) return;
  const bool zs = (i < 0 && P.bc_kind[0] == 2) || (i >= P.nx && P.bc_kind[1] == 2) ||
                  (j < 0 && P.bc_kind[2] == 2) || (j >= P.ny && P.bc_kind[3] == 2);

  const float4* fc = f + fcell(P, i, j) * fs;
  // neighbour offsets; a cell next to a pressure ghost (zero slopes) reads itself, which
  // makes every van Leer slope exactly zero
  const long ox = zs ? 0 : fs, oy = zs ? 0 : (long)P.ex * fs;
  const float tdx = P.f_tdx, tdy = P.f_tdy;
  const int pn = P.pr_neg, pa = P.pr_all;
  const bool v0 = P.m_pos > P.m_neg;
  const float4* wt = P.pwt;
  // FP64 face sums owned by this lane: E/W entry `lane`; N and S entries `lane` (lane < 16)
  double sx = 0.0, sn = 0.0, ss = 0.0;
  double hx1 = 0.0, hyn = 0.0, hys = 0.0, hx2 = 0.0;  // Shakhov moments owned by this lane

  // this warp's row pairs: [p0, p1) of the v >= 0 half (pairs pn .. pa - 1) and [q0, q1) of
  // the v < 0 half (pairs 0 .. pn - 1); the v = 0 row's share of the v < 0 half goes with the
  // first v >= 0 pair
  const int p0 = SPLIT ? pn + (int)((long)(pa - pn) * g / split) : pn;
  const int p1 = SPLIT ? pn + (int)((long)(pa - pn) * (g + 1) / split) : pa;
  const int q0 = SPLIT ? (int)((long)pn * g / split) : 0;
  const int q1 = SPLIT ? (int)((long)pn * (g + 1) / split) : pn;

  for (int k0 = (SPLIT && skip) ? nu : 0; k0 < nu; k0 += 32) {
    const int k = k0 + lane;
    const bool act = k < nu;
    const int kk = act ? k : nu - 1;
    const float u = P.uwf[kk];
    const float wu = act ? P.uwf[nu + kk] : 0.f;
    const float cu = u * tdx;
    float a0, a1, a2, a3, ab0, ab1, x0, x1, x2, x3, xb0, xb1, y0, y1, y2, y3, y4, yb0, yb1, yb2;
    auto zero = [&]() {
      a0 = a1 = a2 = a3 = ab0 = ab1 = x0 = x1 = x2 = x3 = xb0 = xb1 = 0.f;
      y0 = y1 = y2 = y3 = y4 = yb0 = yb1 = yb2 = 0.f;
    };
    // stencil of one row pair (centre and its four neighbours), loaded one pair ahead of its
    // use so that each warp has two pairs' loads in flight
    struct Sten {
      P4 c, w, e, s, n;
    };
    auto load = [&](int pr) {
      const float4* src = fc + (long)pr * nu + kk;
      return Sten{ldp(src), ldp(src - ox), ldp(src + ox), ldp(src - oy), ldp(src + oy)};
    };
    // one row pair: slopes and accumulation; returns the slopes
    auto use = [&](int pr, const Sten& q, P4& rx, P4& ry) {
      rx = vl4(q.w, q.c, q.e);
      ry = vl4(q.s, q.c, q.n);
      const P4 c = q.c;
      const float4 t0 = __ldg(wt + 3 * pr), t1 = __ldg(wt + 3 * pr + 1), t2 = __ldg(wt + 3 * pr + 2);
      const float2 w0 = make_float2(t0.x, t0.y), w1 = make_float2(t0.z, t0.w);
      const float2 w2 = make_float2(t1.x, t1.y), w3 = make_float2(t1.z, t1.w);
      const float2 w4 = make_float2(t2.x, t2.y);
      // one scalar accumulator per sum over both rows of the pair (fewer registers than a
      // packed pair of accumulators, which buys the occupancy this latency-bound loop needs)
      auto acc = [](float& a, float2 w, float2 v) { a = fmaf(w.y, v.y, fmaf(w.x, v.x, a)); };
      acc(a0, w0, c.h); acc(a1, w1, c.h); acc(a2, w2, c.h); acc(a3, w3, c.h);
      acc(ab0, w0, c.b); acc(ab1, w1, c.b);
      acc(x0, w0, rx.h); acc(x1, w1, rx.h); acc(x2, w2, rx.h); acc(x3, w3, rx.h);
      acc(xb0, w0, rx.b); acc(xb1, w1, rx.b);
      acc(y0, w0, ry.h); acc(y1, w1, ry.h); acc(y2, w2, ry.h); acc(y3, w3, ry.h); acc(y4, w4, ry.h);
      acc(yb0, w0, ry.b); acc(yb1, w1, ry.b); acc(yb2, w2, ry.b);
    };
    // end of a chunk of the half whose y side is sy: warp sums in FP32, then FP64
    auto flush = [&](float sy, double& sside) {
      const float ry = chunk_y_sums(u, wu, cu, tdx, tdy, sy, a0, a1, a2, a3, ab0, ab1, x0, x1, x2, x3,
                                    xb0, xb1, y0, y1, y2, y3, y4, yb0, yb1, yb2, lane);
      const float rx = chunk_x_sums(u, wu, cu, tdy, a0, a1, a2, ab0, x0, x1, x2, xb0, y0, y1, y2, y3,
                                    yb0, yb1, lane);
      sside += (double)ry;
      sx += (double)rx;
      if constexpr (SHK) {
        float r1, r2;
        chunk_heat_sums(u, wu, sy, a0, a1, a2, a3, ab0, ab1, x0, x1, x2, x3, xb0, xb1, y0, y1, y2, y3,
                        yb0, yb1, lane, r1, r2);
        if (lane >= 20 && lane < 30) (sy > 0.f ? hyn : hys) += (double)r1;
        else hx1 += (double)r1;
        hx2 += (double)r2;
      }
    };
    // the v >= 0 half (pairs pn .. pa - 1), then the v < 0 half (pairs 0 .. pn - 1); the first
    // v >= 0 pair holds the v = 0 row (if any) as its first row
    zero();
    float s0h = 0.f, s0b = 0.f, s0xh = 0.f, s0xb = 0.f, s0yh = 0.f, s0yb = 0.f;
    if (p1 > p0) {
      Sten q = load(p0);
      Sten nq = load(p0 + 1 < p1 ? p0 + 1 : p0);
      P4 rx, ry;
      use(p0, q, rx, ry);
      if (v0 && (!SPLIT || p0 == pn)) {  // the v = 0 row's half weight for the v < 0 half
        const float hw = __ldg(&wt[3 * pn].x);
        s0h = hw * q.c.h.x; s0b = hw * q.c.b.x; s0xh = hw * rx.h.x; s0xb = hw * rx.b.x;
        s0yh = hw * ry.h.x; s0yb = hw * ry.b.x;
      }
      int n = 1;
#pragma unroll 1
      for (int pr = p0 + 1; pr < p1; pr++) {
        if (n == kSumChunkPairs) {
          flush(1.f, sn);
          zero();
          n = 0;
        }
        q = nq;
        nq = load(pr + 1 < p1 ? pr + 1 : pr);  // the last pair reloads itself (in bounds)
        use(pr, q, rx, ry);
        n++;
      }
    }
    flush(1.f, sn);
    zero();
    a0 = s0h; ab0 = s0b; x0 = s0xh; xb0 = s0xb; y0 = s0yh; yb0 = s0yb;
    if (q1 > q0) {
      Sten nq = load(q0);
      int n = 0;
#pragma unroll 1
      for (int pr = q0; pr < q1; pr++) {
        if (n == kSumChunkPairs) {
          flush(-1.f, ss);
          zero();
          n = 0;
        }
        const Sten q = nq;
        nq = load(pr + 1 < q1 ? pr + 1 : pr);
        P4 rx, ry;
        use(pr, q, rx, ry);
        n++;
      }
    }
    flush(-1.f, ss);
  }
  if (!SPLIT) {
    double* out = sums + (size_t)cell * kNSum;
    out[kSumE + lane] = sx;  // lanes 0..15: E side, 16..31: W side
    if (lane < 16) {
      out[kSumN + lane] = sn;
      out[kSumS + lane] = ss;
    }
    if constexpr (SHK) {
      double* ho = P.hs + (size_t)cell * kNHeat;
      if (lane < 20) ho[kHeatE + lane] = hx1;  // E then W
      else if (lane < 30) {
        ho[kHeatN + lane - 20] = hyn;
        ho[kHeatS + lane - 20] = hys;
      } else {
        ho[kHeatC + lane - 30] = hx1;
      }
      if (lane < 11) ho[kHeatC + 2 + lane] = hx2;
    }
    return;
  }
  __syncthreads();  // red[] of the previous virtual block has been read
  red[warp][kSumE + lane] = sx;
  if (lane < 16) {
    red[warp][kSumN + lane] = sn;
    red[warp][kSumS + lane] = ss;
  }
  __syncthreads();
  if (g == 0 && !skip) {
    double* out = sums + (size_t)cell * kNSum;
    for (int e = lane; e < kNSum; e += 32) {
      double t = red[warp][e];
      for (int w = 1; w < split; w++) t += red[warp + w][e];
      out[e] = t;
    }
  }
}

__device__ __noinline__ void sums_body_split(const Params& P, const float4* __restrict__ f,
                                            double* __restrict__ sums, int bx, int split,
                                            double (*red)[kNSum]) {
  sums_body_p<true>(P, f, sums, bx, split, red);
}


// -------------------------------------------------------------------------------------
// S6 + S8 and Eq. 3 as an upwind strip walk.  For one velocity the micro flux through a face
// depends only on its upwind cell, so each cell evaluates the flux through its downwind
// x-face and downwind y-face and receives the flux through its upwind faces from its upwind
// neighbours.  A warp (lane = slot: two velocities with the same u and the same sign of v)
// owns a strip of W adjacent columns and walks it row by row in the direction of v; within
// a row it visits the columns in the direction of u.  The x-upwind flux of a column is the
// previous column's downwind flux, the y-upwind flux is the previous row's, both carried in
// registers; only the strip's first column needs the flux out of the cell before the strip
// (U), evaluated from U's own reconstruction.  Slopes are taken along the walk (upwind,
// centre, downwind), so the upwind face value is f + slope and u sigma_x = |u| (2/dx) slope.
// Work item: (slot chunk of 32, v < 0 chunks first; tile of `rows` rows; strip).
// -------------------------------------------------------------------------------------
constexpr int kWalkRows = 64;  // default rows per walk tile
constexpr int kStripW = 4;     // columns per strip
constexpr int kRing = 2;       // rows of face and cell records staged in shared memory
constexpr int kFRing = 4;      // rows of f staged in shared memory: P, C, N and the next one
constexpr int kFPos = kStripW + 3;  // walk positions of a staged f row: UU, U, strip, D
// 16-byte chunks of one row's records of a strip: W + 1 x-faces, W y-faces, W cells
constexpr int kFaceF4 = sizeof(FaceRecF) / 16, kCellF4 = sizeof(CellRecF) / 16;
constexpr int kStripChunks = (kStripW + 1) * kFaceF4 + kStripW * kFaceF4 + kStripW * kCellF4;
// shared memory of one warp of the walk (float4): f ring, then record ring
// ... and one 16-byte slot for the two mbarriers of the record ring
constexpr int kStripWarpF4 = kFRing * kFPos * 32 + kRing * kStripChunks + 1;
constexpr size_t kStripSmem = (size_t)kWarpsPerBlock * kStripWarpF4 * sizeof(float4);

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// ---- bulk asynchronous copies (the tensor-memory-access unit) with mbarrier completion ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// one try of the wait for phase `parity`; true once that phase has completed
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// Polls of a bounded mbarrier wait in the walk (each try suspends the thread for a
// hardware-chosen time): about a second at the least before the walk gives up.
constexpr int kWalkWaitPolls = 1 << 22;

// Per-lane velocity constants of the walk (u shared by the pair, v per velocity).
struct PairLane {
  float u, uu, cu, au, dt;   // u, u^2, |u| 2/dx, |u|/dx, dt
  float bref;                // b_ref = K / (2 lam_ref): g_ref,b = b_ref g_ref,h
  float2 v, uv, vv, r2, ur2, vr2;
  float2 cv, av;             // |v| 2/dy, |v|/dy
  float2 grh, grb;           // g_ref (h, b)
};

// E0 + E1 u + E2 v + E3 r2 for both velocities
__device__ __forceinline__ float2 epoly_p(const float4 e, const PairLane& L) {
  return fma2(f2(e.w), L.r2, fma2(f2(e.z), L.v, f2(fmaf(e.y, L.u, e.x))));
}
// 2^(E0 + E1 u + E2 v + E3 r2) for both velocities
__device__ __forceinline__ float2 exp_p(const float4 e, const PairLane& L) {
  const float2 a = epoly_p(e, L);
  return make_float2(ex2_ftz(a.x), ex2_ftz(a.y));
}
// 2^x - 1 for both lanes, to FP32 precision relative to the result: the Taylor series of
// 2^x - 1 = sum_{n>=1} (x ln 2)^n / n! (7 terms; the first one left out is below 2e-8
// relative for |x| <= 1/2), else 2^x - 1 from the exp2 estimate (no cancellation there).
__device__ __forceinline__ float2 ex2m1_p(float2 x) {
  constexpr float c1 = 0.69314718055994531f, c2 = 0.24022650695910071f, c3 = 0.055504108664821580f;
  constexpr float c4 = 0.0096181291076284772f, c5 = 0.0013333558146428443f;
  constexpr float c6 = 1.5403530393381609e-4f, c7 = 1.5252733804059841e-5f;
  float2 p = fma2(f2(c7), x, f2(c6));
  p = fma2(p, x, f2(c5));
  p = fma2(p, x, f2(c4));
  p = fma2(p, x, f2(c3));
  p = fma2(p, x, f2(c2));
  p = fma2(p, x, f2(c1));
  p = mul2(p, x);
  return make_float2(fabsf(x.x) <= 0.5f ? p.x : ex2_ftz(x.x) - 1.f,
                     fabsf(x.y) <= 0.5f ? p.y : ex2_ftz(x.y) - 1.f);
}

// Micro flux through a face (FaceRecF), e-form f_up and d = u sigma_x + v sigma_y.
__device__ __forceinline__ P4 face_p(const FaceRecF* R, int side, const PairLane& L, const P4& fup,
                                     const P4& d) {
  const float4 a = ld4(&R->Q[side][0]);
  const float4 b = ld4(&R->Q[side][4]);
  const float4 k = ld4(&R->K[side][0]);
  const float4 e = ld4(&R->E[0]);
  const float2 t = *reinterpret_cast<const float2*>(&R->Mt4);  // Mt4, -Mt5
  float2 qh = fma2(f2(a.z), L.v, f2(fmaf(a.y, L.u, a.x)));
  qh = fma2(f2(a.w), f2(L.uu), qh);
  qh = fma2(f2(b.x), L.uv, qh);
  qh = fma2(f2(b.y), L.vv, qh);
  qh = fma2(f2(b.z), L.ur2, qh);
  qh = fma2(f2(b.w), L.vr2, qh);
  const float2 qb = fma2(f2(k.w), qh, fma2(f2(k.z), L.v, f2(fmaf(k.y, L.u, k.x))));
  const float2 g = exp_p(e, L);
  P4 X;
  X.h = fma2(qh, g, fma2(f2(t.x), fup.h, mul2(f2(t.y), d.h)));
  X.b = fma2(qb, g, fma2(f2(t.x), fup.b, mul2(f2(t.y), d.b)));
  return X;
}

// Flux leaving a diffuse wall into the gas, e-form: dt (g_w - g_ref) for h and
// dt (b_w g_w - b_ref g_ref) = dt (b_w D + (b_w - b_ref) g_ref,h) for b, D = g_w - g_ref formed
// from the wall exponent relative to g_ref's (FaceRecF).
__device__ __forceinline__ P4 wall_p(const FaceRecF* R, const PairLane& L) {
  const float4 e = ld4(&R->E[0]);
  const float dt = R->gdt, bw = R->K[0][3];
  const float2 D = mul2(L.grh, ex2m1_p(epoly_p(e, L)));
  P4 X;
  X.h = mul2(f2(dt), D);
  X.b = mul2(f2(dt), fma2(f2(bw), D, mul2(f2(bw - L.bref), L.grh)));
  return X;
}

// Shakhov factor S_h of one g for both velocities (s: 8 coefficients on the monomials
// 1, u, v, u^2, uv, v^2, u r2, v r2) and its linear b term Lb (l: on 1, u, v).
__device__ __forceinline__ float2 shk_sh(const float4 a, const float4 b, const PairLane& L) {
  float2 r = f2(fmaf(a.w, L.uu, fmaf(a.y, L.u, a.x)));
  r = fma2(f2(a.z), L.v, r);
  r = fma2(f2(b.x), L.uv, r);
  r = fma2(f2(b.y), L.vv, r);
  r = fma2(f2(b.z), L.ur2, r);
  return fma2(f2(b.w), L.vr2, r);
}

// Eq. 3 increment of one cell (CellRecF); Xi / Xo: inflow / outflow flux in x and y.
// SHK: the Shakhov model (CS: the cell's Shakhov factors, global memory): g+ in place of g.
template <bool SHK = false>
__device__ __forceinline__ P4 collide_p(const CellRecF* C, const PairLane& L, const P4& e,
                                        const P4& Xix, const P4& Xox, const P4& Xiy, const P4& Xoy,
                                        const CellShkF* CS = nullptr) {
  const float4 en = ld4(&C->dEn[0]);
  const float4 e1 = ld4(&C->dE1[0]);
  const float4 A = ld4(&C->A1);    // A1 An db1 dbn
  const float4 B = ld4(&C->nBs);   // -Bs irx iry inv
  // g - g_ref for g^n and g^{n+1}, from the exponents relative to g_ref's
  float2 Dn = mul2(L.grh, ex2m1_p(epoly_p(en, L))), D1 = mul2(L.grh, ex2m1_p(epoly_p(e1, L)));
  // Shakhov: D -> D + g_h S_h, and the b terms gain g_h Lb
  float2 Xbn = f2(0.f), Xb1 = f2(0.f);
  if constexpr (SHK) {
    const float4* cs = reinterpret_cast<const float4*>(CS);
    const float4 sn0 = __ldg(cs), sn1 = __ldg(cs + 1), s10 = __ldg(cs + 2), s11 = __ldg(cs + 3);
    const float4 lbn = __ldg(cs + 4), lb1 = __ldg(cs + 5);
    const float2 Gn = add2(Dn, L.grh), G1 = add2(D1, L.grh);
    Dn = fma2(Gn, shk_sh(sn0, sn1, L), Dn);
    D1 = fma2(G1, shk_sh(s10, s11, L), D1);
    Xbn = mul2(Gn, fma2(f2(lbn.z), L.v, f2(fmaf(lbn.y, L.u, lbn.x))));
    Xb1 = mul2(G1, fma2(f2(lb1.z), L.v, f2(fmaf(lb1.y, L.u, lb1.x))));
  }
  const float2 r = fma2(L.v, f2(B.z), f2(L.u * B.y));
  const float aui = L.au * B.w;
  const float2 avi = mul2(L.av, f2(B.w));
  float2 dh = fma2(f2(aui), sub2(Xix.h, Xox.h), mul2(avi, sub2(Xiy.h, Xoy.h)));
  float2 db = fma2(f2(aui), sub2(Xix.b, Xox.b), mul2(avi, sub2(Xiy.b, Xoy.b)));
  // b g - g_ref,b = b D + (b - b_ref) g_ref,h
  dh = fma2(f2(A.x), D1, fma2(f2(A.y), Dn, fma2(r, L.grh, fma2(f2(B.x), e.h, dh))));
  if constexpr (!SHK) {
    db = fma2(f2(A.x), fma2(f2(A.z + L.bref), D1, mul2(f2(A.z), L.grh)),
              fma2(f2(A.y), fma2(f2(A.w + L.bref), Dn, mul2(f2(A.w), L.grh)),
                   fma2(r, L.grb, fma2(f2(B.x), e.b, db))));
  } else {
    db = fma2(f2(A.x), fma2(f2(A.z + L.bref), D1, fma2(f2(A.z), L.grh, Xb1)),
              fma2(f2(A.y), fma2(f2(A.w + L.bref), Dn, fma2(f2(A.w), L.grh, Xbn)),
                   fma2(r, L.grb, fma2(f2(B.x), e.b, db))));
  }
  return {add2(e.h, dh), add2(e.b, db)};
}

__device__ __forceinline__ P4 slope_d(const PairLane& L, const P4& rx, const P4& ry) {
  return {fma2(f2(L.cu), rx.h, mul2(L.cv, ry.h)), fma2(f2(L.cu), rx.b, mul2(L.cv, ry.b))};
}

// sm: this warp's shared memory (kStripWarpF4 float4: f ring, record ring, two mbarriers,
// initialised by the caller); nrec: record stages this warp has issued on them so far (the
// phases of the mbarriers follow from it).  Returns false if a wait for records gave up
// (err then has bit 1 set).
template <int W, bool FULL, bool SHK = false>
__device__ __forceinline__ bool strip_body_p(const Params& P, const float4* __restrict__ f,
                                             float4* __restrict__ fo, const FaceRecF* __restrict__ fxr,
                                             const FaceRecF* __restrict__ fyr,
                                             const CellRecF* __restrict__ cr, int nchunk_neg,
                                             int rows, int bx, int by, int chunk,
                                             float4* __restrict__ sm, unsigned& nrec,
                                             int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int nx = P.nx, ny = P.ny, nu = P.nu, fs = P.fs;
  const int i0 = bx * W;
  const int wc = FULL ? W : min(W, nx - i0);         // columns of this strip (FULL: W)
  const bool vpos = chunk >= nchunk_neg;
  const int sn = P.pr_neg * nu;                        // slots of the v < 0 half
  const int s = vpos ? sn + (chunk - nchunk_neg) * 32 + lane : chunk * 32 + lane;
  const int send = vpos ? fs : sn;
  const bool act = s < send;
  const int ss = act ? s : send - 1;
  const int pr = ss / nu, k = ss - pr * nu;
  PairLane L;
  L.u = P.uwf[k];
  {
    const float4 t2 = __ldg(P.pwt + 3 * pr + 2);
    L.v = make_float2(t2.z, t2.w);
  }
  L.uu = L.u * L.u;
  L.uv = mul2(f2(L.u), L.v);
  L.vv = mul2(L.v, L.v);
  L.r2 = add2(f2(L.uu), L.vv);
  L.ur2 = mul2(f2(L.u), L.r2);
  L.vr2 = mul2(L.v, L.r2);
  L.cu = fabsf(L.u) * P.f_tdx;
  L.au = fabsf(L.u) * P.f_idx;
  L.cv = make_float2(fabsf(L.v.x) * P.f_tdy, fabsf(L.v.y) * P.f_tdy);
  L.av = make_float2(fabsf(L.v.x) * P.f_idy, fabsf(L.v.y) * P.f_idy);
  {
    const float4 g = __ldg(P.gref4 + ss);
    L.grh = make_float2(g.x, g.y);
    L.grb = make_float2(g.z, g.w);
  }
  L.dt = P.f_dt;
  L.bref = (float)P.ref_bf;
  const int su = L.u > 0.f ? 1 : -1;
  const int sv = vpos ? 1 : -1;
  const int xside = su > 0 ? 0 : 1, yside = vpos ? 0 : 1;
  const int ib = su > 0 ? i0 : i0 + wc - 1;            // strip position 0 (walk order)
  const int iU = ib - su;                              // upwind neighbour column U
  const bool pW = P.bc_kind[0] == 2, pE = P.bc_kind[1] == 2, pS = P.bc_kind[2] == 2, pN = P.bc_kind[3] == 2;
  const bool zu = (iU < 0 && pW) || (iU >= nx && pE);  // U is a pressure ghost: zero slopes
  const int xo = su * fs;                              // one column in walk order, in slots
  // walk position p (-2 = UU, -1 = U, 0..W-1 strip, W = D) -> column offset; strip positions
  // past the strip's end read column D (they are not updated)
  auto col = [&](int p) { return (p < wc ? p : wc) * xo; };

  const int j0 = by * rows;
  const int j1 = min(j0 + rows, ny);
  const int jfirst = sv > 0 ? j0 : j1 - 1;
  const int nsteps = j1 - j0;
  const long rs = (long)sv * P.ex * fs;                // one row in walk order, in slots
  const long base = ((long)(jfirst + 2) * P.ex + ib + 2) * fs + ss;
  const float4* pr_ = f + base;                        // (position 0, row jfirst)
  float4* pw = fo + base;

  // prologue: flux through the y-face between the halo row jp = jfirst - sv and jfirst
  // (read from global memory: once per walk)
  P4 Xiy[W];
  {
    const int jp = jfirst - sv;
    const FaceRecF* RY = fyr + (long)(sv > 0 ? jfirst : jfirst + 1) * nx + ib;
    const bool zp = (jp < 0 && pS) || (jp >= ny && pN);
    if (RY->wall != 0.f) {
#pragma unroll
      for (int t = 0; t < W; t++)
        if (t < wc) Xiy[t] = wall_p(RY + su * t, L);
    } else {
      const float4* rp = pr_ - rs;                     // row jp
      P4 a = ldp(rp + col(-1)), c = ldp(rp + col(0));
#pragma unroll
      for (int t = 0; t < W; t++) {
        if (t < wc) {
          const P4 b = ldp(rp + col(t + 1));
          P4 rx = vl4(a, c, b);
          P4 ry = vl4(ldp(rp - rs + col(t)), c, ldp(pr_ + col(t)));
          if (zp) rx = ry = zero4();
          Xiy[t] = face_p(RY + su * t, yside, L, add4(c, ry), slope_d(L, rx, ry));
          a = c;
          c = b;
        }
      }
    }
  }

  // f rows q = 0 .. nsteps + 1 (row jfirst + (q - 1) sv) pass through a ring of kFRing rows
  // in shared memory, each at the walk positions -2 .. W (UU, U, strip, D); a lane copies
  // (cp.async) and reads only its own slot's column.  The face and cell records of a row
  // pass through a ring of kRing rows: [x-faces i0..i0+wc][y-faces i0..i0+wc-1 on the
  // downwind side][cells i0..i0+wc-1], read by every lane: three contiguous segments, each
  // one bulk copy issued by lane 0 and completed on the ring slot's mbarrier.  Row st's
  // records and f row st + 2 are issued one row ahead.
  float4* fring = sm;
  float4* ring = sm + kFRing * kFPos * 32;
  const uint32_t bars = smem_addr(ring + kRing * kStripChunks);  // mbarrier of ring slot b at bars + 8 b
  constexpr int oY = (W + 1) * kFaceF4, oC = oY + W * kFaceF4;
  auto stage_f = [&](int q) {
    if (q <= nsteps + 1) {
      const float4* src = pr_ + (long)(q - 1) * rs;
      float4* dst = fring + (q % kFRing) * (kFPos * 32) + lane;
#pragma unroll
      for (int p = -2; p <= W; p++) cp_async16_cg(dst + (p + 2) * 32, src + col(p));
    }
  };
  auto stage = [&](int st) {
    if (st < nsteps && lane == 0) {
      const int j = jfirst + sv * st;
      const FaceRecF* gx = fxr + (long)j * (nx + 1) + i0;
      const FaceRecF* gy = fyr + (long)(sv > 0 ? j + 1 : j) * nx + i0;
      const CellRecF* gc = cr + (long)j * nx + i0;
      float4* dst = ring + (st % kRing) * kStripChunks;
      const uint32_t bar = bars + 8 * ((nrec + st) % kRing);
      const uint32_t bx_ = (wc + 1) * sizeof(FaceRecF), by_ = wc * sizeof(FaceRecF), bc_ = wc * sizeof(CellRecF);
      // the generic-proxy reads of this ring slot (two rows ago) are ordered before the
      // copies that overwrite it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar, bx_ + by_ + bc_);
      bulk_g2s(smem_addr(dst), gx, bx_, bar);
      bulk_g2s(smem_addr(dst + oY), gy, by_, bar);
      bulk_g2s(smem_addr(dst + oC), gc, bc_, bar);
    }
    stage_f(st + 2);
    cp_async_commit();
  };
  // wait (bounded by `polls`) for the records of row st; the same verdict on every lane
  auto wait_rec = [&](int st, int polls) {
    const unsigned k = nrec + st;
    const uint32_t bar = bars + 8 * (k % kRing), parity = (k / kRing) & 1;
    bool ok = false;
    for (int it = 0; it < polls && !ok; it++) ok = mbar_try_wait(bar, parity);
    return __all_sync(kFull, ok);
  };
  __syncwarp();                      // the rings' previous contents are no longer read
  stage_f(0);
  stage_f(1);
  stage(0);
  // local record index of walk position t (-1 = U's face for x) within the staged row
  const int xl0 = su > 0 ? 0 : wc;   // x-face between U and position 0
  auto cl = [&](int t) { return su > 0 ? t : wc - 1 - t; };
  for (int st = 0; st < nsteps; st++) {
    __syncwarp();                    // every lane is done with the slots refilled next
    stage(st + 1);
    cp_async_wait<1>();
    if (!wait_rec(st, P.walk_wait_polls)) {
      // give up: wait (bounded) for the copies already issued, so that none lands after the
      // walk has returned, record the failure, return
      cp_async_wait<0>();
      wait_rec(st, kWalkWaitPolls);
      if (st + 1 < nsteps) wait_rec(st + 1, kWalkWaitPolls);
      if (lane == 0) atomicOr(err, 2);
      nrec += nsteps;
      return false;
    }
    __syncwarp();
    const float4* row = ring + (st % kRing) * kStripChunks;
    const FaceRecF* RX = reinterpret_cast<const FaceRecF*>(row);
    const FaceRecF* RY = reinterpret_cast<const FaceRecF*>(row + oY);
    const CellRecF* CC = reinterpret_cast<const CellRecF*>(row + oC);
    // rows P (st), C (st + 1), N (st + 2) of the f ring, at walk position 0
    const float4* fP = fring + (st % kFRing) * (kFPos * 32) + 64 + lane;
    const float4* fC = fring + ((st + 1) % kFRing) * (kFPos * 32) + 64 + lane;
    const float4* fN = fring + ((st + 2) % kFRing) * (kFPos * 32) + 64 + lane;
    auto at = [](const float4* r, int p) { return ldp_s(r + p * 32); };

    // flux into position 0 out of U (or off the wall)
    P4 cm = at(fC, -1), c0 = at(fC, 0);
    P4 Xix;
    const FaceRecF* RXi = RX + xl0;
    if (RXi->wall != 0.f) {
      Xix = wall_p(RXi, L);
    } else {
      P4 rx = vl4(at(fC, -2), cm, c0);
      P4 ry = vl4(at(fP, -1), cm, at(fN, -1));
      if (zu) rx = ry = zero4();
      Xix = face_p(RXi, xside, L, add4(cm, rx), slope_d(L, rx, ry));
    }
#pragma unroll
    for (int t = 0; t < W; t++) {
      if (t < wc) {
        const P4 cn = at(fC, t + 1);
        const P4 rx = vl4(cm, c0, cn);
        const P4 ry = vl4(at(fP, t), c0, at(fN, t));
        const P4 d = slope_d(L, rx, ry);
        const P4 Xox = face_p(RXi + su * (t + 1), xside, L, add4(c0, rx), d);
        const P4 Xoy = face_p(RY + cl(t), yside, L, add4(c0, ry), d);
        const P4 o = collide_p<SHK>(CC + cl(t), L, c0, Xix, Xox, Xiy[t], Xoy,
                                    SHK ? P.cshk + (long)(jfirst + sv * st) * nx + i0 + cl(t) : nullptr);
        if (act) stp(pw + col(t), o);
        Xix = Xox;
        Xiy[t] = Xoy;
        cm = c0;
        c0 = cn;
      }
    }
    pw += rs;
  }
  cp_async_wait<0>();
  nrec += nsteps;
  return true;
}

// -------------------------------------------------------------------------------------
// State conversion and initialisation (set-up and checkpoint paths, not the step)
// -------------------------------------------------------------------------------------
// FP64 rows [cell][q][(h, b)] (rows j0 .. j0+nrows-1) -> paired slots, e = f - g_ref.  One
// thread per slot (grid-stride over all slots of the rows): it reads (h, b) of its two rows
// at u_k (a padding row repeats the half's last row, so it reads that row twice) and writes
// the slot with one 16-byte store.  Adjacent threads read adjacent (h, b) pairs of a row,
// coalesced also when the rows are host memory read over the C2C link; A16: the rows are
// 16-byte aligned and each pair is one 16-byte load, else two 8-byte loads (the rows need
// only 8-byte alignment).
template <bool A16>
__global__ void k_rows_to_f32(const double* __restrict__ src, float4* __restrict__ dst, Params P,
                              const double2* __restrict__ grefd, int j0, int nrows) {
  const long nslot = (long)P.nx * nrows * P.fs;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < nslot; t += (long)gridDim.x * blockDim.x) {
    const long c = t / P.fs;
    const int s = (int)(t - c * P.fs);
    const int r = (int)(c / P.nx), i = (int)(c - (long)r * P.nx);
    const int pr = s / P.nu, k = s - pr * P.nu;
    const int q0 = prow(P, 2 * pr) * P.nu + k, q1 = prow(P, 2 * pr + 1) * P.nu + k;
    const double* row = src + (size_t)c * P.nq * 2;
    double2 a, b;
    if constexpr (A16) {
      a = reinterpret_cast<const double2*>(row)[q0];
      b = reinterpret_cast<const double2*>(row)[q1];
    } else {
      a = make_double2(row[2 * q0], row[2 * q0 + 1]);
      b = make_double2(row[2 * q1], row[2 * q1 + 1]);
    }
    const double2 g0 = grefd[q0], g1 = grefd[q1];
    dst[((size_t)(j0 + r + 2) * P.ex + i + 2) * P.fs + s] =
        make_float4((float)(a.x - g0.x), (float)(b.x - g1.x), (float)(a.y - g0.y), (float)(b.y - g1.y));
  }
}
// paired slots -> FP64 rows, f = e + g_ref; one thread per velocity in the order of the rows
// (adjacent (h, b) pairs; A16: one 16-byte store per pair, else two 8-byte stores)
template <bool A16>
__global__ void k_f32_to_rows(const float4* __restrict__ src, double* __restrict__ dst, Params P,
                              const double2* __restrict__ grefd, int j0, int nrows) {
  const int ncell = P.nx * nrows;
  for (int c = blockIdx.x; c < ncell; c += gridDim.x) {
    const int r = c / P.nx, i = c - r * P.nx;
    const float* s = reinterpret_cast<const float*>(src + ((size_t)(j0 + r + 2) * P.ex + i + 2) * P.fs);
    double* d = dst + (size_t)c * P.nq * 2;
    for (int q = threadIdx.x; q < P.nq; q += blockDim.x) {
      const int m = q / P.nu, k = q - m * P.nu, pr = padrow(P, m);
      const float* e = s + 4 * ((size_t)(pr >> 1) * P.nu + k) + (pr & 1);
      const double2 g = grefd[q];
      const double h = (double)e[0] + g.x, b = (double)e[2] + g.y;
      if constexpr (A16) {
        reinterpret_cast<double2*>(d)[q] = make_double2(h, b);
      } else {
        d[2 * q] = h;
        d[2 * q + 1] = b;
      }
    }
  }
}

// Pointwise Maxwellian of (rho, U, V, T) per cell, paired slots, and W.
__global__ void k_init_maxwellian_p(Params P, const double* __restrict__ prim, float4* __restrict__ f,
                                    double* __restrict__ W, int nwe) {
  const int nc = P.nx * P.ny;
  const int cell = blockIdx.x;
  if (cell >= nc) return;
  const int i = cell % P.nx, j = cell / P.nx;
  const double rho = prim[cell], U = prim[nc + cell], V = prim[2 * nc + cell], T = prim[3 * nc + cell];
  const double lam = 1.0 / T, G = rho * lam / kPi, bf = P.K / (2.0 * lam);
  float4* dst = f + fcell(P, i, j) * P.fs;
  for (int t = threadIdx.x; t < P.fs; t += blockDim.x) {
    const int pr = t / P.nu, k = t - pr * P.nu;
    double o[4];
    for (int h = 0; h < 2; h++) {
      const int m = prow(P, 2 * pr + h);
      const double du = P.u[k] - U, dv = P.v[m] - V;
      const double gh = G * exp(-lam * (du * du + dv * dv));
      double rh, rb;
      ref_maxwellian(P, P.u[k], P.v[m], rh, rb);
      o[h] = gh - rh;
      o[2 + h] = bf * gh - rb;
    }
    dst[t] = make_float4((float)o[0], (float)o[1], (float)o[2], (float)o[3]);
  }
  if (threadIdx.x == 0) {
    const int w = wcell(P, i, j);
    W[w] = rho;
    W[nwe + w] = rho * U;
    W[2 * nwe + w] = rho * V;
    W[3 * nwe + w] = rho * (0.5 * (U * U + V * V) + (P.K + 2) / (4.0 * lam));
  }
}

}  // namespace ugks
