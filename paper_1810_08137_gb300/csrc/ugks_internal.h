// Internal device-side data structures of the UGKS library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace ugks {

constexpr int kMaxAxis = 512;        // nu, nv limit (shared-memory tables per axis)
constexpr int kMaxNq = 65536;        // nu * nv limit
constexpr int kWarpsPerBlock = 4;    // warp-per-cell kernels: 4 cells per 128-thread block

// Per-cell half-range velocity sums written by the sums kernel (step S1 + S7 of the flux
// table, split by the side of the cell the sums feed).  64 doubles per cell:
//   [side][quantity][component], side: E (u>0), W (u<0), N (v>0), S (v<0);
//   quantity: W0 = sum w psi f_face, St = sum w psi sigma_t, Sf = sum w u_n psi f_face,
//             Ss = sum w u_n psi (u sigma_x + v sigma_y); component: psi = 1, u, v, E.
// A face's sums are the E (N) side of its low cell plus the W (S) side of its high cell.
enum { kSumE = 0, kSumW = 16, kSumN = 32, kSumS = 48, kNSum = 64 };
enum { kOffW0 = 0, kOffSt = 4, kOffSf = 8, kOffSs = 12 };
constexpr int kSumsTotals = 14;    // per-thread totals of the sums kernel (shared memory)
constexpr int kHeatTotals = 4;     // and the four more the Shakhov heat-flux sums need
// dynamic shared memory of the sums kernel: per-warp sums, per-thread totals
template <typename T>
__host__ __device__ constexpr size_t sums_smem_bytes() {
  return (kWarpsPerBlock * kNSum + (kSumsTotals + kHeatTotals) * 128) * sizeof(T) +
         kWarpsPerBlock * 56 * sizeof(double);  // per-warp Shakhov heat-flux sums (kNHeat)
}

// Shakhov model: per-cell raw velocity moments the heat fluxes need (FP64, kNHeat per cell),
// in the natural frame (u, v).  Per side E (u > 0), W (u < 0), N (v > 0), S (v < 0), of the
// side's face values (f +/- the half slope), weighted by H(u_n) like the other face sums:
//   M20 M11 M02 M30 M21 M12 M03 (h, M_ab = sum w u^a v^b h) and B00 B10 B01 (b);
// then of the cell values over every velocity: M00 M10 M01 M20 M11 M02 M30 M21 M12 M03 B00
// B10 B01.  (M00, M10, M01 and M20 + M02 + B00 of the faces are in the kNSum sums.)
enum { kHeatE = 0, kHeatW = 10, kHeatN = 20, kHeatS = 30, kHeatC = 40, kNHeat = 56 };

// What the update kernel needs about one face (written by the face kernel).
// Micro flux in the face frame (u_n normal, u_t tangential), per component c (h, b):
//   F~_c = u_n [ Q_c(u_n, u_t) g_h + Mt4 f_up,c - Mt5 (u sigma_x + v sigma_y)_up,c ]
//   g_h  = G exp(-lam (u_n - Un)^2) exp(-lam (u_t - Ut)^2)
//   Q_c  = c00 + c10 un + c01 ut + c20 un^2 + c11 un ut + c02 ut^2
//          + cn3 un (un^2 + ut^2) + ct3 ut (un^2 + ut^2)
// with one coefficient set for u_n > 0 (a_L side) and one for u_n < 0 (a_R side).
// Wall faces: F~_c = u_n dt f_w,c, f_w = incoming interior value or the wall Maxwellian.
struct FaceRec {
  double Q[2][2][8];   // [side 0: un>0, 1: un<0][comp h, b][c00 c10 c01 c20 c11 c02 cn3 ct3]
  double G, Un, Ut, lam;
  double Mt4, Mt5;
  double bfac;         // K / (2 lam): g_b = bfac g_h
  int wall;            // 0: UGKS interface; 1: wall, gas on the high side; 2: gas on the low side
  int pad;
};

// Per-cell coefficients of the implicit f update (Eq. 3):
//   f^{n+1} = inv [ cf f^n + flux + cg1 g^{n+1} + cgn g^n ]
struct CellRec {
  double Gn, Un, Vn, lamn, bn;   // g^n_h = Gn exp(-lamn (u-Un)^2) exp(-lamn (v-Vn)^2), g_b = bn g_h
  double G1, U1, V1, lam1, b1;   // same for g^{n+1}
  double cf, cgn, cg1, inv;
  // Shakhov model: the heat flux of f^n (qx, qy) and alpha = (1 - Pr) 4 lam^2 / ((K+4) rho)
  // of W^n and W^{n+1}; the Shakhov factors are S_h = alpha (c.q) (2 lam |c|^2 - 4) and
  // S_b = alpha (c.q) (K/(2 lam)) (2 lam |c|^2 - 2): g+_h = g_h (1 + S_h), g+_b = g_h (b + S_b)
  double qx, qy, an, a1;
};

// FP32 records of the FP32 form's update kernel (written by the FP64 face and cell
// kernels, so the update kernel does no FP64 arithmetic or conversion).  They are stated in
// the global velocity frame on the monomials m = (1, u, v, u^2, uv, v^2, u r2, v r2),
// r2 = u^2 + v^2, with the Maxwellian amplitude folded into the coefficients and each
// Maxwellian written as 2^(E0 + E1 u + E2 v + E3 r2), so that a lane evaluates a face or
// cell with fused multiply-adds and one exp2.
//   micro flux through a face, side s = 0 (un > 0) or 1 (un < 0), e-form f_up and d:
//     X_h = Q_h g + Mt4 f_up,h + nMt5 d_h,  Q_h = sum_k Q[s][k] m_k,  nMt5 = -Mt5,
//     X_b = Q_b g + Mt4 f_up,b + nMt5 d_b,  Q_b = K[s][3] Q_h + K[s][0] + K[s][1] u + K[s][2] v,
//     g = 2^(E . (1, u, v, r2))
//   inflow from a diffuse wall (wall != 0): X_h = gdt D, X_b = gdt (K[0][3] D + (K[0][3] - b_ref)
//     g_ref,h), D = g_w - g_ref,h = g_ref,h (2^(E . (1, u, v, r2)) - 1) with E the wall
//     Maxwellian's exponent relative to g_ref's and gdt = dt
// 144 bytes (pad): the update walk stages a row's records in shared memory, and lanes with
// u > 0 and u < 0 read different records of the row in the same instruction; at a 128-byte
// stride two records would fall in the same shared-memory banks, at 144 bytes they do not.
struct __align__(16) FaceRecF {
  float Q[2][8];
  float K[2][4];
  float E[4];
  float Mt4, nMt5, wall, gdt;
  float pad[4];
};
// Eq. 3 as an increment e^{n+1} = e^n + d, per component, with the Maxwellians taken
// relative to g_ref before they are weighted (the terms stay at the deviation's scale):
//   d_h = aui dX_h + avi dY_h + r g_ref,h + A1 D1 + An Dn + nBs e_h
//   d_b = aui dX_b + avi dY_b + r g_ref,b + A1 (b1 D1 + db1 g_ref,h) + An (bn Dn + dbn g_ref,h)
//         + nBs e_b
// with D = g - g_ref,h = g_ref,h (2^(dE . (1, u, v, r2)) - 1) for g^n and g^{n+1}, where dE are
// the exponent coefficients of g relative to those of g_ref (formed in FP64, so they are
// small and exact for a state near the reference, and D keeps FP32 precision relative to
// itself); b = db + b_ref, aui = inv |u|/dx, avi = inv |v|/dy, r = u irx + v iry, dX / dY the
// inflow minus outflow micro flux in x / y.
struct __align__(16) CellRecF {
  float dEn[4];
  float dE1[4];
  float A1, An, db1, dbn;   // inv cg1, inv cgn, K/(2 lam^{n+1}) - b_ref, K/(2 lam^n) - b_ref
  float nBs, irx, iry, inv; // -inv (cg1 + cgn), inv (Mt4_W - Mt4_E)/dx, inv (Mt4_S - Mt4_N)/dy
};

// FP32-f form, Shakhov model: per cell, the Shakhov factors of g^n and g^{n+1} in the
// global velocity frame (FP32, from FP64 coefficients): S_h on the monomials
// (1, u, v, u^2, uv, v^2, u r2, v r2) (sn, s1), and Lb = 2 b alpha (c.q) on (1, u, v) (ln, l1),
// so that g+_h - g_ref,h = D + g_h S_h and g+_b - g_ref,b = b D + (b - b_ref) g_ref,h +
// g_h (b S_h + Lb), D = g_h - g_ref,h.
struct __align__(16) CellShkF {
  float sn[8], s1[8];
  float ln[4], l1[4];
};

// DF64 form: f of one velocity, (h, b) as double-FP32 pairs (h = hh + hl, b = bh + bl)
struct __align__(16) DF4 {
  float hh, hl, bh, bl;
};
// DF64 form: the FP64 records (FaceRec, CellRec) as double-FP32 pairs, written by the FP64
// interface and cell kernels for the DF64 update kernels (which do no FP64 arithmetic)
struct __align__(16) FaceRecD {
  float2 Q[2][2][8];
  float2 G, Un, Ut, lam, Mt4, Mt5, bfac;
  int wall, pad;
};
struct __align__(16) CellRecD {
  float2 Gn, Un, Vn, lamn, bn, G1, U1, V1, lam1, b1, inv, cgn, cg1, pad;
};

struct Params {
  int nx, ny, nu, nv, nq, K;
  // Shakhov model (pr != 1): shk = 1, hs the heat-flux moment sums (kNHeat per cell, the
  // cells of the sums buffer), shk_c = (1 - Pr) 4 / (K + 4) (alpha = shk_c lam^2 / rho)
  int shk;
  double pr, shk_c;
  double* hs;
  CellShkF* cshk;         // FP32-f form: the Shakhov cell records (written by the cells kernel)
  double refheat[5][10];  // FP32-f form: the kNHeat moments of g_ref per side and of the cell
                          // (zero in the FP64 form): E, W, N, S (10 each), cell (first 10
                          // of its 13 in refheat[4], B-moments in refheatC)
  double refheatC[3];
  int ex;                 // f row length in cells: nx + 4 (two-cell ghost ring)
  int wx;                 // W row length in cells: nx + 2 (one-cell ghost ring)
  double dx, dy, dt;
  double mu_ref, omega;
  int bc_kind[4];
  double bc_rho[4], bc_T[4], bc_U[4];
  double wall_mom[4][4];  // per side: sum over outgoing velocities of w u_n psi g_wall(rho=1)
  int m_pos;              // first v index with v > 0 (v ascending); nv if none
  int m_neg;              // number of v indices with v < 0
  // Reference Maxwellian of the FP32 form: the FP32 buffers hold e = f - g_ref, and every
  // sum or flux of f is the FP32 sum of e plus the exact FP64 sum of g_ref.
  int use_ref;
  double ref_G, ref_U, ref_V, ref_lam, ref_bf;  // g_ref,h = G exp(-lam((u-U)^2+(v-V)^2)), b = bf h
  double ref_E[4];        // g_ref,h = 2^(ref_E . (1, u, v, u^2 + v^2))
  double ref_iG, ref_E0u;  // 1 / ref_G; ref_E[0] - log2(ref_G)
  double refsum[4][16];   // per side E, W, N, S (order of kSumE..kSumS / 16): half-range
                          // sums of g_ref in the W0 and Sf slots, zero in St and Ss
  double refpair[2][8];   // refsum of both sides of a face: x faces (E + W), y faces (N + S);
                          // W0 slots then Sf slots
  // FP32 form, paired-row layout (see ugks_f32.cuh): pr_neg row pairs with v < 0, pr_all
  // row pairs in total, fs = pr_all * nu float4 slots per cell
  int pr_neg, pr_all, fs;
  const float4* gref4;    // [fs] g_ref of each slot (h, h', b, b')
  const float4* pwt;      // [pr_all][3]: (w0 w0' w1 w1') (w2 w2' w3 w3') (w4 w4' v v'),
                          // w_n = wv v^n of the pair's two rows; zero on padded rows, half
                          // of wv on the v = 0 row
  int omega_half;         // omega == 1/2: lam^-omega = rsqrt(lam)
  // derived FP64 constants (set by set_derived): 1/(K+2), dt/(2 mu_ref), dt/(4 mu_ref),
  // 2/dx, 2/dy, 1/dx, 1/dy
  double inv_kp2, half_dt_mu, quarter_dt_mu, d_tdx, d_tdy, d_idx, d_idy;
  const float* uwf;       // FP32 tables: [2][nu] u, wu
  const double* mvd;      // [5][nv] wv v^n, n = 0..4
  float f_tdx, f_tdy, f_idx, f_idy, f_dt;  // FP32 2/dx, 2/dy, 1/dx, 1/dy, dt
  int walk_wait_polls;    // FP32-f walk: bound of its wait for record copies (polls)
  const double* u;        // [nu]
  const double* v;        // [nv]
  const double* wu;       // [nu]
  const double* wv;       // [nv]
  // DF64 form: the same grid tables as double-FP32 pairs (hi, lo): [nu] u, [nu] wu, [nv] v,
  // [5][nv] wv v^n; 2/dx, 2/dy, 1/dx, 1/dy, dt
  const float2* gdf;
  float2 df_tdx, df_tdy, df_idx, df_idy, df_dt;
};

}  // namespace ugks
