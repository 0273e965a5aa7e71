// Internal device-side data structures of the UGKS library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
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
};

// FP32 copies of the face and cell records for the FP32 form's update kernel (written by the
// FP64 face and cell kernels, so the update kernel does no FP64 arithmetic or conversion).
// b component of the micro flux: Q_b = X2 Q_h + kb0 + kb1 un + kb2 ut.
struct __align__(16) FaceRecF {
  float Q[2][8];     // Q_h per side (0: un > 0, 1: un < 0): c00 c10 c01 c20 c11 c02 cn3 ct3
  float kb[2][4];    // kb0 kb1 kb2 (pad) per side
  float lam, Un, Ut, G;
  float Mt4, Mt5, X2, wall;
};
struct __align__(16) CellRecF {
  float Gn, Un, Vn, lamn;
  float G1, U1, V1, lam1;
  float bn, b1, inv, cg1;
  float cgn, refx, refy, pad;   // refx = (Mt4_W - Mt4_E)/dx, refy = (Mt4_S - Mt4_N)/dy
};

struct Params {
  int nx, ny, nu, nv, nq, K;
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
  double refsum[4][16];   // per side E, W, N, S (order of kSumE..kSumS / 16): half-range
                          // sums of g_ref in the W0 and Sf slots, zero in St and Ss
  const void* gref;       // [nq] T2 table of g_ref (FP32 form), else null
  int omega_half;         // omega == 1/2: lam^-omega = rsqrt(lam)
  const float* mvf;       // FP32 tables: [5][nv] wv, wv v, wv v^2, wv v^3, v
  const float* uwf;       // FP32 tables: [2][nu] u, wu
  float f_tdx, f_tdy, f_idx, f_idy, f_dt;  // FP32 2/dx, 2/dy, 1/dx, 1/dy, dt
  const double* u;        // [nu]
  const double* v;        // [nv]
  const double* wu;       // [nu]
  const double* wv;       // [nv]
};

}  // namespace ugks
