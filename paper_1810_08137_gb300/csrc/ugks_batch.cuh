// Batched execution of many independent UGKS instances (FP32-f form): every kernel of the
// step runs once per step for all active instances, as a persistent grid that walks a
// device-resident work table of virtual blocks, and the whole step is one CUDA graph
// replay.  The table (and each instance's ping-pong parity) lives in device memory, so
// admitting or retiring an instance changes data, not the captured graph.
// Included by ugks.cu (same translation unit as the single-instance kernels).
#pragma once

namespace ugks {

constexpr int kMaxSlots = 256;
constexpr int kPhases = 6;  // ghost_x, ghost_y, sums, faces, cells, update (strip walk)

// What the phase kernels need about one instance.
struct SlotDev {
  Params P;
  float4* f[2];
  double* W[2];
  float* sums;
  FaceRecF* fxf;
  FaceRecF* fyf;
  CellRecF* cellf;
  double* Fx;
  double* Fy;
  double* mt4;
  double* rpart;
  int* err;
  int nwe, nrblocks, nchunk_neg, nchunk_pos;
  int walk_rows;   // tile rows of the walk kernel (autotuned per velocity-grid class)
  int cur;         // ping-pong parity, flipped on the device after every step
};

// Work table: virtual-block prefix sums per phase over the active instances.
struct BatchWork {
  int n;                            // active instances
  int slot[kMaxSlots];              // slot of active instance a
  int start[kPhases][kMaxSlots + 1];
};

// Virtual blocks of one instance per phase (must match the decoding in the kernels).
__host__ __device__ inline int phase_blocks(const SlotDev& S, int phase) {
  const Params& P = S.P;
  switch (phase) {
    case 0: return P.ny * 4;
    case 1: return (P.nx + 4) * 4;
    case 2: return ((P.nx + 2) * (P.ny + 2) + kWarpsPerBlock - 1) / kWarpsPerBlock;
    case 3: return ((P.nx + 1) * P.ny + P.nx * (P.ny + 1) + 127) / 128;
    case 4: return S.nrblocks;
    default: {
      const long items = (long)((P.nx + kStripW - 1) / kStripW) *
                         ((P.ny + S.walk_rows - 1) / S.walk_rows) * (S.nchunk_neg + S.nchunk_pos);
      return (int)((items + kWarpsPerBlock - 1) / kWarpsPerBlock);
    }
  }
}

// Active instance owning virtual block vb (binary search in the prefix sums).
__device__ __forceinline__ int find_instance(const int* start, int n, int vb) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= vb) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void kb_ghost_x(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk) {
  const int total = wk->start[0][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[0], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    const int loc = vb - wk->start[0][a], c = S.cur;
    ghost_x_body(S.P, S.f[c], S.W[c], S.nwe, loc % S.P.ny, loc / S.P.ny);
  }
}

__global__ void kb_ghost_y(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk) {
  const int total = wk->start[1][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[1], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    const int loc = vb - wk->start[1][a], c = S.cur, w = S.P.nx + 4;
    ghost_y_body(S.P, S.f[c], S.W[c], S.nwe, loc % w, loc / w);
  }
}

__global__ void __launch_bounds__(128, 5) kb_sums(const SlotDev* __restrict__ slots,
                                               const BatchWork* __restrict__ wk) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int total = wk->start[2][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[2], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    sums_body_p(S.P, S.f[S.cur], S.sums, smraw, vb - wk->start[2][a]);
  }
}

__global__ void __launch_bounds__(128) kb_faces(const SlotDev* __restrict__ slots,
                                                const BatchWork* __restrict__ wk) {
  const int total = wk->start[3][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[3], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    const int loc = vb - wk->start[3][a];
    faces_body<float>(S.P, S.sums, S.W[S.cur], S.nwe, nullptr, nullptr, S.Fx, S.Fy, S.fxf, S.fyf,
                      S.mt4, loc * 128 + threadIdx.x);
  }
}

__global__ void __launch_bounds__(128) kb_cells(const SlotDev* __restrict__ slots,
                                                const BatchWork* __restrict__ wk) {
  __shared__ double red[8][128];
  const int total = wk->start[4][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    __syncthreads();  // red[] of the previous virtual block has been read
    const int a = find_instance(wk->start[4], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    const int c = S.cur;
    cells_body(S.P, S.W[c], S.W[c ^ 1], S.nwe, S.Fx, S.Fy, nullptr, S.rpart, S.err, S.cellf, S.mt4,
               red, vb - wk->start[4][a]);
  }
}

// Update sweep: one warp per work item (strip, tile, velocity chunk).
__global__ void __launch_bounds__(128, 3) kb_strip(const SlotDev* __restrict__ slots,
                                                const BatchWork* __restrict__ wk) {
  extern __shared__ __align__(16) float4 strip_sm[];  // kStripSmem bytes
  const int warp = threadIdx.x >> 5;
  const int total = wk->start[5][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[5], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    const int ns = (S.P.nx + kStripW - 1) / kStripW, nt = (S.P.ny + S.walk_rows - 1) / S.walk_rows;
    const int it = (vb - wk->start[5][a]) * kWarpsPerBlock + warp;
    const int nch = S.nchunk_neg + S.nchunk_pos;
    if (it < ns * nt * nch) {
      const int c = S.cur;
      // velocity chunks fastest: the warps of a block share the strip's records and halo
      const int bx = (it / nch) % ns, by = it / (nch * ns), ck = it % nch;
      // full strips (all but the last of a row when kStripW does not divide nx) with the
      // strip width known at compile time
      if ((bx + 1) * kStripW <= S.P.nx)
        strip_body_p<kStripW, true>(S.P, S.f[c], S.f[c ^ 1], S.fxf, S.fyf, S.cellf, S.nchunk_neg,
                                    S.walk_rows, bx, by, ck, strip_sm + warp * kStripWarpF4);
      else
        strip_body_p<kStripW, false>(S.P, S.f[c], S.f[c ^ 1], S.fxf, S.fyf, S.cellf, S.nchunk_neg,
                                     S.walk_rows, bx, by, ck, strip_sm + warp * kStripWarpF4);
    }
  }
}

// After the step: every active instance swaps its buffers.
__global__ void kb_flip(SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk) {
  for (int a = threadIdx.x; a < wk->n; a += blockDim.x) slots[wk->slot[a]].cur ^= 1;
}

}  // namespace ugks
