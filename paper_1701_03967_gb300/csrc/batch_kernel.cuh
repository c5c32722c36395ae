// The dependency-driven kernel of the batched solver (one instantiation per
// element order n) and the work-list records it reads.
//
// Work list.  Every problem's mixed-precision solve (algorithm (a) or (b) of
// Section 4 in float32, then float64 residual refinement) is a linear chain
// of steps: pencil passes along the axes, the three phases of the band solve
// of algorithm (b) and operator applies.  A step is cut
// into items (one pass tile, or a few apply blocks); every item of step s of
// a problem needs all items of step s-1 of the same problem.  The items are
// numbered in "level" order (step 0 of every problem, then step 1 of every
// problem, ...), so every item's dependencies carry smaller numbers.
//
// Execution.  One launch covers the whole work list: each CTA takes the next
// number from an atomic ticket counter when it starts, waits (thread 0)
// until the completion counter of its item's predecessor step is full, does
// the item and publishes its completion.  Tickets go only to CTAs that are
// running, so the unfinished item with the smallest number is always held by
// a running CTA whose dependencies are all finished: the schedule cannot
// deadlock, whatever the number of resident CTAs.  The waits are still
// bounded: after a time limit the waiting CTA records FEM_FFT_ERR_TIMEOUT and
// every later CTA returns at once.  Completion is published with a release
// pattern (block barrier, fence, atomic increment) and observed with an
// acquire load followed by a block barrier; fields written inside the launch
// are read with L2-coherent loads.  A CTA does one item and exits (a loop
// over items inside one CTA made the register allocator spill the pass
// bodies heavily).
#pragma once
#include <cuda_runtime.h>

#include "../../include/femfft.h"
#include "apply.cuh"
#include "band.cuh"
#include "pencil.cuh"

namespace femfft {

constexpr int kBatchThreads = 256;
constexpr int kBatchCtasPerSm = 4;   // resident CTAs overlap one another's prologue and barriers (measured: 4 > 3 > 2)
constexpr long long kItemDof = 1 << 16;  // target unknowns per item
constexpr unsigned kMaxSpin = 1u << 24;  // hard iteration bound of a dependency wait
static_assert(kBandThreads == kBatchThreads, "band blocks are laid out for the batch kernel's block size");

enum BatchKind { BATCH_PENCIL = 0, BATCH_APPLY = 1, BATCH_BAND = 2 };

struct BatchStage {
  int kind;           // BatchKind
  int mode;           // pencil: MODE_*; apply: number of outputs (1 or 2); band: phase (0 condense, 1 vertex, 2 back)
  int n;
  int TW;             // apply, band: positions of the contiguous axis per block
  int dep;            // index of the step this one waits for (-1: none)
  unsigned need;      // items of that step
  int units_per_item;
  int tile_smem;      // apply in double-float: bytes of its staged input tiles
  long long units;    // pass tiles or apply blocks
  long long first;    // first ticket
  long long items;
  PassParams pp;
  ApplyParams ap;
  BandParams bp;      // float32 field and tables
};

struct BatchArgs {
  const BatchStage* stages;
  const int* item_stage;      // ticket -> step
  long long total;            // number of tickets
  unsigned* done;             // per-step finished items
  unsigned long long* ticket;
  int* status;                // FEM_FFT_OK or FEM_FFT_ERR_TIMEOUT
  int* where;                 // step whose wait timed out
  unsigned long long wait_ns;
};

// Dynamic shared memory of an apply item: matrices and exchange buffers,
// then a copy of its parameters.
template <int NORD>
__host__ __device__ constexpr size_t batch_apply_scratch() {
  return sizeof(ApplySmem<NORD, 2, kBatchThreads>) > sizeof(ApplySmemDF<NORD, 2, kBatchThreads>)
             ? sizeof(ApplySmem<NORD, 2, kBatchThreads>)
             : sizeof(ApplySmemDF<NORD, 2, kBatchThreads>);
}
template <int NORD>
__host__ __device__ constexpr size_t batch_apply_smem() {
  return batch_apply_scratch<NORD>() + sizeof(ApplyParams);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 only.  Returns 0 once step d has `need` finished items, 1 when the
// batch is stopping (another CTA gave up, or this wait ran out of time).
static __device__ __noinline__ int batch_wait(const BatchArgs& A, int d, unsigned need, int st) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0; it < kMaxSpin; ++it) {
    if (ld_acquire_u32(&A.done[d]) >= need) return 0;
    if (ld_relaxed_s32(A.status) != FEM_FFT_OK) return 1;
    if (global_ns() - t0 > A.wait_ns) break;
    __nanosleep(it < 32 ? 64 : 512);
  }
  atomicCAS(A.status, FEM_FFT_OK, FEM_FFT_ERR_TIMEOUT);
  atomicExch(A.where, st);
  return 1;
}

template <int NORD, int NOUT>
__device__ __forceinline__ void batch_apply_item(const ApplyParams& P, int TW, long long b0, long long b1,
                                                 unsigned char* smem) {
  auto& S = *reinterpret_cast<ApplySmem<NORD, NOUT, kBatchThreads>*>(smem);
  apply_stage_mats<NORD, NOUT, kBatchThreads>(P, S);
  __syncthreads();
  for (long long b = b0; b < b1; ++b) {
    apply_block<NORD, NOUT, kBatchThreads, false>(P, TW, b, S);
    __syncthreads();
  }
}

template <int NORD, int NOUT>
__device__ __forceinline__ void batch_apply_item_df(const ApplyParams& P, int TW, long long b0, long long b1,
                                                    unsigned char* smem, float2* tiles) {
  auto& S = *reinterpret_cast<ApplySmemDF<NORD, NOUT, kBatchThreads>*>(smem);
  apply_stage_mats_df<NORD, NOUT, kBatchThreads>(P, S);
  for (long long b = b0; b < b1; ++b) {
    apply_block_df<NORD, NOUT, kBatchThreads, false>(P, TW, b, S, tiles);
    __syncthreads();
  }
}

// The kernel for the problems of element order NORD: one item per CTA.
template <int NORD>
__global__ void __launch_bounds__(kBatchThreads, kBatchCtasPerSm) batch_kernel(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_ticket;
  __shared__ int s_stage, s_abort;
  __shared__ __align__(16) PassParams s_pp;
  __shared__ float s_base[kMaxW];
  if (threadIdx.x == 0) {
    const long long t = (long long)atomicAdd(A.ticket, 1ULL);
    int abort = 0, st = -1;
    if (t >= A.total || ld_relaxed_s32(A.status) != FEM_FFT_OK) {
      abort = 1;
    } else {
      st = __ldg(&A.item_stage[t]);
      const int d = __ldg(&A.stages[st].dep);
      if (d >= 0) abort = batch_wait(A, d, __ldg(&A.stages[st].need), st);
    }
    s_ticket = t;
    s_stage = st;
    s_abort = abort;
  }
  __syncthreads();
  if (s_abort) return;
  const int st = s_stage;
  const BatchStage& S = A.stages[st];
  const long long item = s_ticket - S.first;
  const int kind = S.kind, mode = S.mode;
  const long long u0 = item * S.units_per_item;
  const long long u1 = min(u0 + (long long)S.units_per_item, S.units);
  if (kind == BATCH_PENCIL) {
    const int* src = reinterpret_cast<const int*>(&S.pp);
    int* dst = reinterpret_cast<int*>(&s_pp);
    for (int i = threadIdx.x; i < (int)(sizeof(PassParams) / sizeof(int)); i += blockDim.x) dst[i] = __ldg(&src[i]);
    __syncthreads();
    // one tile per item (units_per_item = 1)
    if (mode == MODE_FWD) pencil_tile<float, NORD, MODE_FWD, kMaxW, false>(s_pp, u0, smem, s_base, true);
    else if (mode == MODE_INV) pencil_tile<float, NORD, MODE_INV, kMaxW, false>(s_pp, u0, smem, s_base, true);
    else if (mode == MODE_FWD_DIV) pencil_tile<float, NORD, MODE_FWD_DIV, kMaxW, false>(s_pp, u0, smem, s_base, true);
    else pencil_tile<float, NORD, MODE_FUSED, kMaxW, false>(s_pp, u0, smem, s_base, true);
  } else if (kind == BATCH_BAND) {
    BandParams* bp = reinterpret_cast<BandParams*>(smem);
    const int* src = reinterpret_cast<const int*>(&S.bp);
    int* dst = reinterpret_cast<int*>(bp);
    for (int i = threadIdx.x; i < (int)(sizeof(BandParams) / sizeof(int)); i += blockDim.x) dst[i] = __ldg(&src[i]);
    __syncthreads();
    // blocks are independent: no barrier between them
    for (long long b = u0; b < u1; ++b) {
      if (mode == 0) band_condense_block<float, NORD, true>(*bp, S.TW, b);
      else if (mode == 1) band_vertex_block<float, NORD, true>(*bp, b);
      else band_back_block<float, NORD, true>(*bp, S.TW, b);
    }
  } else {
    ApplyParams* ap = reinterpret_cast<ApplyParams*>(smem + batch_apply_scratch<NORD>());
    const int* src = reinterpret_cast<const int*>(&S.ap);
    int* dst = reinterpret_cast<int*>(ap);
    for (int i = threadIdx.x; i < (int)(sizeof(ApplyParams) / sizeof(int)); i += blockDim.x) dst[i] = __ldg(&src[i]);
    __syncthreads();
    if (ap->df) {
      float2* tiles = reinterpret_cast<float2*>(smem + batch_apply_smem<NORD>());
      if (mode <= 1) batch_apply_item_df<NORD, 1>(*ap, S.TW, u0, u1, smem, tiles);
      else batch_apply_item_df<NORD, 2>(*ap, S.TW, u0, u1, smem, tiles);
    } else {
      if (mode <= 1) batch_apply_item<NORD, 1>(*ap, S.TW, u0, u1, smem);
      else batch_apply_item<NORD, 2>(*ap, S.TW, u0, u1, smem);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&A.done[st], 1u);
  }
}

// Kernel entry of order n (instantiated in batch_k*.cu), or nullptr.
const void* batch_kernel_fn_1(int n);   // orders 1..3
const void* batch_kernel_fn_2(int n);   // orders 4..6
const void* batch_kernel_fn_3(int n);   // orders 7..9

}  // namespace femfft
