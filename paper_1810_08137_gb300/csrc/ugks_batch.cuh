// Batched execution of many independent UGKS instances (FP32-f form): every phase of the
// step runs once per step for all active instances, as a persistent grid that walks a
// device-resident work table of virtual blocks.  The step is either one cooperative launch
// of kb_step (all phases, grid barriers with bounded waits between them) or seven phase
// launches; either way one CUDA graph replay.  The table (and each instance's ping-pong
// parity) lives in device memory, so admitting or retiring an instance changes data, not
// the captured graph.
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
  double* sums;
  FaceRecF* fxf;
  FaceRecF* fyf;
  CellRecF* cellf;
  double* Fx;
  double* Fy;
  double* mt4;
  double* rpart;
  int* err;
  int nwe, nrblocks, nchunk_neg, nchunk_pos;
  int walk_rows;   // cell tile of the walk: rows per tile (autotuned per velocity-grid class)
  int walk_vtile;  // velocity tile of the walk: 32-slot chunks per tile, 0 = all (autotuned)
  int sums_split;  // warps per cell in the sums phase (1, 2 or 4): velocity-space split
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
    case 2: return ((P.nx + 2) * (P.ny + 2) * S.sums_split + kWarpsPerBlock - 1) / kWarpsPerBlock;
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

// ---- phase bodies: one pass of a phase over the whole work table, grid-strided ----------
// Not inlined: the persistent step and the phase kernels call the same compiled body, so an
// instance's floating-point results do not depend on which of them runs it (inlined into
// different kernels, the compiler may fuse a multiply and an add differently).
__device__ __noinline__ void ghost_x_phase(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk,
                                              double* tab) {
  const int total = wk->start[0][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[0], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    const int loc = vb - wk->start[0][a], c = S.cur;
    ghost_x_body(S.P, S.f[c], S.W[c], S.nwe, loc % S.P.ny, loc / S.P.ny, tab);
  }
}

__device__ __noinline__ void ghost_y_phase(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk,
                                              double* tab) {
  const int total = wk->start[1][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[1], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    const int loc = vb - wk->start[1][a], c = S.cur, w = S.P.nx + 4;
    ghost_y_body(S.P, S.f[c], S.W[c], S.nwe, loc % w, loc / w, tab);
  }
}

__device__ __noinline__ void sums_phase(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk,
                                        double (*red)[kNSum]) {
  const int total = wk->start[2][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[2], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    if (S.P.shk) continue;  // Shakhov instances: sums_phase_shk
    if (S.sums_split > 1)
      sums_body_split(S.P, S.f[S.cur], S.sums, vb - wk->start[2][a], S.sums_split, red);
    else
      sums_body_p<false>(S.P, S.f[S.cur], S.sums, vb - wk->start[2][a], 1, red);
  }
}

// The phases of the Shakhov model's instances (heat-flux sums, Shakhov interface, walk with
// g+), over the same work table, skipping the BGK instances: functions and kernels of their
// own, so that the BGK phases carry none of their code or registers.
__device__ __noinline__ void sums_phase_shk(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk) {
  const int total = wk->start[2][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[2], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    if (S.P.shk) sums_body_p<false, true>(S.P, S.f[S.cur], S.sums, vb - wk->start[2][a], 1, nullptr);
  }
}

__device__ __noinline__ void faces_phase(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk) {
  const int total = wk->start[3][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[3], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    const int loc = vb - wk->start[3][a];
    if (S.P.shk) continue;  // Shakhov instances: faces_phase_shk
    faces_body<kRecF32>(S.P, S.sums, S.W[S.cur], S.nwe, S.fxf, S.fyf, S.Fx, S.Fy, S.mt4,
                        loc * 128 + threadIdx.x);
  }
}

__device__ __noinline__ void faces_phase_shk(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk) {
  const int total = wk->start[3][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[3], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    if (!S.P.shk) continue;
    const int loc = vb - wk->start[3][a];
    faces_body<kRecF32, true>(S.P, S.sums, S.W[S.cur], S.nwe, S.fxf, S.fyf, S.Fx, S.Fy, S.mt4,
                              loc * 128 + threadIdx.x);
  }
}

__device__ __noinline__ void cells_phase(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk,
                                            double (*red)[128]) {
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

// Work item `it` of an instance's walk -> (strip bx, row tile by, velocity chunk ck).  The
// chunks are grouped into velocity tiles of walk_vtile chunks (0: all chunks of the cell);
// items run velocity tile slowest, then row tile, then strip, chunk of the tile fastest, so
// that consecutive warps (the warps of a block) walk the same strip and rows for the chunks
// of one velocity tile (sharing its face and cell records in L1), and a tile of one chunk
// puts adjacent strips on consecutive warps (sharing f halo columns instead).
__device__ __forceinline__ void walk_item(const SlotDev& S, int ns, int nt, int it, int& bx, int& by, int& ck) {
  const int nch = S.nchunk_neg + S.nchunk_pos;
  const int vt = (S.walk_vtile > 0 && S.walk_vtile < nch) ? S.walk_vtile : nch;
  const int per = nt * ns * vt;  // items of a full velocity tile
  const int nvt = (nch + vt - 1) / vt;
  int t = it / per;
  if (t > nvt - 1) t = nvt - 1;
  int rem = it - t * per;
  const int vts = (t == nvt - 1) ? nch - t * vt : vt;  // chunks of this velocity tile
  const int c = rem % vts;
  rem /= vts;
  bx = rem % ns;
  by = rem / ns;
  ck = t * vt + c;
}

// Update sweep: one warp per work item (strip, row tile, velocity chunk).
// Returns the record stages this warp has issued on its mbarriers (the Shakhov walk of the
// persistent step continues on them).
__device__ __noinline__ unsigned strip_phase(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk,
                                             float4* strip_sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this warp's two mbarriers of the record ring (shared memory may have served another
  // phase before: initialise them here)
  float4* wsm = strip_sm + warp * kStripWarpF4;
  const uint32_t bars = smem_addr(wsm + kFRing * kFPos * 32 + kRing * kStripChunks);
  if (lane == 0) {
    mbar_init(bars, 1);
    mbar_init(bars + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  unsigned nrec = 0;
  bool ok = true;
  const int total = wk->start[5][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[5], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    const int ns = (S.P.nx + kStripW - 1) / kStripW, nt = (S.P.ny + S.walk_rows - 1) / S.walk_rows;
    const int it = (vb - wk->start[5][a]) * kWarpsPerBlock + warp;
    const int nch = S.nchunk_neg + S.nchunk_pos;
    if (it < ns * nt * nch) {
      const int c = S.cur;
      int bx, by, ck;
      walk_item(S, ns, nt, it, bx, by, ck);
      // full strips (all but the last of a row when kStripW does not divide nx) with the
      // strip width known at compile time
      if (!ok) continue;  // a wait of this warp gave up: its walks are skipped (err is set)
      if (S.P.shk) continue;  // Shakhov instances: strip_phase_shk
      if ((bx + 1) * kStripW <= S.P.nx)
        ok = strip_body_p<kStripW, true>(S.P, S.f[c], S.f[c ^ 1], S.fxf, S.fyf, S.cellf, S.nchunk_neg,
                                         S.walk_rows, bx, by, ck, wsm, nrec, S.err);
      else
        ok = strip_body_p<kStripW, false>(S.P, S.f[c], S.f[c ^ 1], S.fxf, S.fyf, S.cellf, S.nchunk_neg,
                                          S.walk_rows, bx, by, ck, wsm, nrec, S.err);
    }
  }
  return nrec;
}

// The walk of the Shakhov model's instances (g+ in the collision term; any strip width).
// init: initialise this warp's mbarriers (a launch of its own); otherwise continue on the
// ones strip_phase initialised in the same launch, after its nrec0 record stages.
__device__ __noinline__ void strip_phase_shk(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk,
                                             float4* strip_sm, bool init, unsigned nrec0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4* wsm = strip_sm + warp * kStripWarpF4;
  const uint32_t bars = smem_addr(wsm + kFRing * kFPos * 32 + kRing * kStripChunks);
  if (init && lane == 0) {
    mbar_init(bars, 1);
    mbar_init(bars + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  unsigned nrec = nrec0;
  bool ok = true;
  const int total = wk->start[5][wk->n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int a = find_instance(wk->start[5], wk->n, vb);
    const SlotDev& S = slots[wk->slot[a]];
    if (!S.P.shk) continue;
    const int ns = (S.P.nx + kStripW - 1) / kStripW, nt = (S.P.ny + S.walk_rows - 1) / S.walk_rows;
    const int it = (vb - wk->start[5][a]) * kWarpsPerBlock + warp;
    const int nch = S.nchunk_neg + S.nchunk_pos;
    if (it < ns * nt * nch && ok) {
      const int c = S.cur;
      int bx, by, ck;
      walk_item(S, ns, nt, it, bx, by, ck);
      ok = strip_body_p<kStripW, false, true>(S.P, S.f[c], S.f[c ^ 1], S.fxf, S.fyf, S.cellf, S.nchunk_neg,
                                              S.walk_rows, bx, by, ck, wsm, nrec, S.err);
    }
  }
}

// ---- one kernel per phase (the step as a graph of seven launches) ------------------------
__global__ void kb_ghost_x(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk) {
  __shared__ double tab[kGhostTab];
  ghost_x_phase(slots, wk, tab);
}

__global__ void kb_ghost_y(const SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk) {
  __shared__ double tab[kGhostTab];
  ghost_y_phase(slots, wk, tab);
}

__global__ void __launch_bounds__(128, 5) kb_sums(const SlotDev* __restrict__ slots,
                                               const BatchWork* __restrict__ wk) {
  __shared__ double red[kWarpsPerBlock][kNSum];  // face sums of split cells
  sums_phase(slots, wk, red);
}

// eight blocks per SM (64 registers, the rest on the stack): the interface is latency-bound
// on its FP64 and double-FP32 chains, and 32 resident warps hide more of it than 12 (0.59 ->
// 0.50 ms at 800x400x28^2; six blocks 0.52 ms)
__global__ void __launch_bounds__(128, 8) kb_faces(const SlotDev* __restrict__ slots,
                                                const BatchWork* __restrict__ wk) {
  faces_phase(slots, wk);
}

__global__ void __launch_bounds__(128) kb_cells(const SlotDev* __restrict__ slots,
                                                const BatchWork* __restrict__ wk) {
  __shared__ double red[8][128];
  cells_phase(slots, wk, red);
}

__global__ void __launch_bounds__(128, 3) kb_strip(const SlotDev* __restrict__ slots,
                                                const BatchWork* __restrict__ wk) {
  extern __shared__ __align__(16) float4 strip_sm[];  // kStripSmem bytes
  strip_phase(slots, wk, strip_sm);
}

// The Shakhov model's phases (instances with pr != 1; the others are skipped).
__global__ void __launch_bounds__(128, 4) kb_sums_shk(const SlotDev* __restrict__ slots,
                                                   const BatchWork* __restrict__ wk) {
  sums_phase_shk(slots, wk);
}
__global__ void __launch_bounds__(128, 4) kb_faces_shk(const SlotDev* __restrict__ slots,
                                                    const BatchWork* __restrict__ wk) {
  faces_phase_shk(slots, wk);
}
__global__ void __launch_bounds__(128, 3) kb_strip_shk(const SlotDev* __restrict__ slots,
                                                    const BatchWork* __restrict__ wk) {
  extern __shared__ __align__(16) float4 strip_sm[];  // kStripSmem bytes
  strip_phase_shk(slots, wk, strip_sm, true, 0u);
}

// After the step: every active instance swaps its buffers.
__global__ void kb_flip(SlotDev* __restrict__ slots, const BatchWork* __restrict__ wk) {
  for (int a = threadIdx.x; a < wk->n; a += blockDim.x) slots[wk->slot[a]].cur ^= 1;
}

// ---- the whole step as one persistent cooperative launch ---------------------------------
// Grid-wide barrier between the phases, with a bounded wait: a block that has waited
// `limit` polls (about 0.13 us each) without the generation advancing, or that sees another
// block's timeout, records kBarrierTimeout in `err` and the whole grid leaves the kernel at
// that barrier (the host reports UGKS_ETIMEOUT).  No phase has copies in flight at a
// barrier (the walk waits for its own cp.async groups before it returns).  count and gen
// are zeroed before every launch; limit and err persist.
struct BarrierDev {
  unsigned int count;       // blocks arrived at the current barrier
  unsigned int gen;         // barriers completed in this launch
  unsigned long long limit; // polls before a block gives up
  int err;                  // kBarrierTimeout once any block gave up (cleared by the host)
  int pad;
};
constexpr int kBarrierTimeout = 1;

__device__ __forceinline__ bool grid_sync(BarrierDev* g) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile BarrierDev* vg = g;
    const unsigned int gen = vg->gen;
    __threadfence();  // this block's results are visible before it arrives
    const unsigned int arrived = atomicAdd(&g->count, 1u);
    int good = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(&g->count, 0u);
      __threadfence();
      atomicAdd(&g->gen, 1u);
    } else {
      const unsigned long long limit = vg->limit;
      unsigned long long n = 0;
      while (vg->gen == gen) {
        if (vg->err != 0 || n >= limit) {
          atomicOr(&g->err, kBarrierTimeout);
          good = 0;
          break;
        }
        n++;
        __nanosleep(128);
      }
    }
    __threadfence();  // the other blocks' results are visible after it
    ok = good && vg->err == 0;
  }
  __syncthreads();
  return ok != 0;
}

// dynamic shared memory of the persistent step: the largest phase's (the walk's rings; the
// ghost tables and the cells reduction alias its start)
constexpr size_t kStepSmem = kStripSmem;
static_assert(kStepSmem >= sizeof(double) * kGhostTab && kStepSmem >= sizeof(double) * 8 * 128 &&
                  kStepSmem >= sizeof(double) * kWarpsPerBlock * kNSum,
              "persistent step: shared memory of every phase");

__global__ void __launch_bounds__(128, 3) kb_step(SlotDev* __restrict__ slots,
                                               const BatchWork* __restrict__ wk,
                                               BarrierDev* __restrict__ bar) {
  extern __shared__ __align__(16) float4 step_sm[];
  double* tab = reinterpret_cast<double*>(step_sm);
  ghost_x_phase(slots, wk, tab);
  if (!grid_sync(bar)) return;
  ghost_y_phase(slots, wk, tab);
  if (!grid_sync(bar)) return;
  sums_phase(slots, wk, reinterpret_cast<double(*)[kNSum]>(step_sm));
  sums_phase_shk(slots, wk);
  if (!grid_sync(bar)) return;
  faces_phase(slots, wk);
  faces_phase_shk(slots, wk);
  if (!grid_sync(bar)) return;
  cells_phase(slots, wk, reinterpret_cast<double(*)[128]>(step_sm));
  if (!grid_sync(bar)) return;
  const unsigned nrec = strip_phase(slots, wk, step_sm);
  strip_phase_shk(slots, wk, step_sm, false, nrec);
  if (!grid_sync(bar)) return;
  if (blockIdx.x == 0)
    for (int a = threadIdx.x; a < wk->n; a += blockDim.x) slots[wk->slot[a]].cur ^= 1;
}

}  // namespace ugks
