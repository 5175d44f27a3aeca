// dmr_period.cuh -- the EM steps of a whole period (Sec. III.C sub-cycling,
// N_T coarse steps with r fine sub-steps each) in one persistent launch.
//
// The per-step launches (k_em2, k_em) each cover a mesh in blocks of
// EM_WARPS warp strips.  Here every such block of every step is a unit of
// work, and the units wait for exactly the units whose output they read
// instead of for the whole previous launch.  The units of one step are the
// blocks of fine sub-steps k = 1..r (phases 1..r, their coarse-fine side
// blocks first) and then the coarse step's blocks (phase 0), numbered in
// that order; block b of the grid takes units b, b + G, b + 2G, ... of
// every step in turn.  Each unit does what its block does in the per-step
// launch (em_segment), with loads through L2, with two changes that give
// the same values: every fine sub-step evaluates the coarse E^{n+1} on its
// boundary lines from the coarse level-n state (as the first one always
// does, Eq. 5b), and the coarse step leaves the edges under the rectangle
// that the last fine sub-step overwrites with the fine means (a8) to it.
// So a fine sub-step never waits for the coarse step of its own coarse
// step, and the results are the same bit for bit.
//
// Dependencies of a unit of step q (counts since the period started):
//  * coarse unit: its eight neighbouring coarse units have finished step
//    q - 1 (their E, H, v and CPML memory are its halo, and it overwrites
//    the buffers they read at step q - 1); a unit within `margin` coarse
//    cells of the rectangle also waits for every unit of the last fine
//    sub-step of step q - 1 (the fine means a8 are in its input, and the
//    fine sub-steps of step q - 1 read the coarse lines it overwrites);
//  * fine sub-step 1: every unit of the last fine sub-step of step q - 1,
//    and every coarse unit near the rectangle at step q - 1 (the coarse
//    level-n state around the boundary lines that sub-steps 1..r read);
//  * fine sub-step k >= 2: every unit of sub-step k - 1 of step q.
// A unit waits only for units that come before it in the order (step,
// phase 1..r, phase 0), and every block takes its units in that order, so
// with all blocks resident (a cooperative launch) the earliest unfinished
// unit can always run.  Coarse units publish a per-unit step count, the
// coarse units near the rectangle add to a count per step, fine units to a
// count per sub-step (each count on a cache line of its own); the
// period-end launch k_pe_rates clears them all.  Every wait is bounded:
// after `limit` polls the block sets bit 8 of the control block's error
// word and returns, and every other block, seeing that bit while it waits,
// returns too.
#pragma once
#include "dmr_kernels.cuh"

namespace dmr {

constexpr int kMaxR = 8;          // refinement factors of the persistent launch
constexpr int kSchedErr = 8;      // control-block error bit: a bounded wait gave up
constexpr int kCntStride = 32;    // words between the fine sub-step counts (one 128-byte line each)

struct PerSched {
  unsigned* flag;          // [nC] coarse units: steps of this period finished
  unsigned* cnt;           // [k * kCntStride]: units of fine sub-step k finished (k = 1..r)
  unsigned* rnq;           // [q]: coarse units near the rectangle that finished step q
  Ctl* ctl;
  long long m0;            // coarse level at the period's start
  long long limit;         // polls of a wait before it gives up
  int NT, r;               // coarse steps per period, refinement factor (1: no fine mesh)
  int nC, gxC, nyC;        // coarse units; strips across; unit rows
  int nFt;                 // fine units per step (all sub-steps)
  int rowsC, swC;          // node rows per warp and owned columns per strip of the coarse units
  int nF[kMaxR + 1];       // units of fine sub-step k (k = 1..r)
  int nU;                  // units per step
  int nRN;                 // coarse units near the rectangle
  int rn[4];               // coarse node box of "near": the rectangle grown by the margin
  int stall;               // test only: coarse unit 0 waits at step 1 for a count nothing reaches
};

// true if coarse unit u lies within the margin of the rectangle
__device__ __forceinline__ bool near_rect(const PerSched& S, int u) {
  if (S.r < 2) return false;
  const int bx = u % S.gxC, by = u / S.gxC;
  const int i0 = bx * S.swC - 1, i1 = bx * S.swC + S.swC;
  const int j0 = by * EM_WARPS * S.rowsC - 1, j1 = (by + 1) * EM_WARPS * S.rowsC;
  return i1 >= S.rn[0] && i0 <= S.rn[2] && j1 >= S.rn[1] && j0 <= S.rn[3];
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_i(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Warp 0 waits until every lane's word has reached its target (lanes with
// no word pass at once): each lane polls its own word, the warp leaves
// together, then every lane fences so that the block's later loads see what
// was published before the words.  False when the wait gave up or another
// block has.
__device__ __forceinline__ bool warp_wait(const unsigned* w, unsigned target, const PerSched& S) {
  long long it = 0;
  bool ok = w == nullptr;
  while (true) {
    if (!ok) ok = ld_relaxed(w) >= target;
    if (__all_sync(0xffffffffu, ok)) break;
    if (++it >= S.limit) {
      if ((threadIdx.x & 31) == 0) atomicOr(&S.ctl->err, kSchedErr);
      return false;
    }
    if ((it & 63) == 0) {
      const int e = (threadIdx.x & 31) == 0 ? ld_relaxed_i(&S.ctl->err) : 0;
      if (__shfl_sync(0xffffffffu, e, 0) & kSchedErr) return false;
    }
    if (it > 32) __nanosleep(64);
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  return true;
}

// the dependencies of unit (phase ph, index iu) of step q, waited on by warp 0
__device__ __forceinline__ bool unit_wait(const PerSched& S, int q, int ph, int iu) {
  const int lane = threadIdx.x & 31;
  const unsigned* w = nullptr;
  unsigned target = 0;
  if (ph == 0) {
    if (q > 0 && lane < 9 && lane != 4) {
      const int bx = iu % S.gxC + lane % 3 - 1, by = iu / S.gxC + lane / 3 - 1;
      if (bx >= 0 && bx < S.gxC && by >= 0 && by < S.nyC) {
        w = S.flag + by * S.gxC + bx;
        target = (unsigned)q;
      }
    }
    if (q > 0 && lane == 9 && near_rect(S, iu)) {
      w = S.cnt + S.r * kCntStride;
      target = (unsigned)q * (unsigned)S.nF[S.r];
    }
    if (S.stall && q == 1 && iu == 0 && lane == 10) {
      w = S.rnq;
      target = 0xffffffffu;
    }
  } else if (ph == 1) {
    if (q > 0 && lane == 0) {
      w = S.cnt + S.r * kCntStride;
      target = (unsigned)q * (unsigned)S.nF[S.r];
    }
    if (q > 0 && lane == 1) {
      w = S.rnq + (q - 1);
      target = (unsigned)S.nRN;
    }
  } else {
    if (lane == 0) {
      w = S.cnt + (ph - 1) * kCntStride;
      target = (unsigned)(q + 1) * (unsigned)S.nF[ph - 1];
    }
  }
  return warp_wait(w, target, S);
}

// publish unit (ph, iu) of step q as finished (thread 0, after the block's
// barrier: the release orders every thread's stores before the word)
__device__ __forceinline__ void unit_done(const PerSched& S, int q, int ph, int iu) {
  if (ph == 0) {
    st_release(S.flag + iu, (unsigned)(q + 1));
    if (near_rect(S, iu)) add_release(S.rnq + q, 1u);
  } else {
    add_release(S.cnt + ph * kCntStride, 1u);
  }
}

// The persistent period.  tab: the launch arguments of phase ph for steps of
// parity par at tab[par * nph + ph] (nph = r + 1 with a fine mesh, else 1),
// copied into dynamic shared memory; the level-dependent fields are filled
// per step as the batched launch does (em_set_level).
template <class T, bool PML>
__global__ void __launch_bounds__(32 * EM_WARPS, kEmMinBlocks<T>) k_period(const EmArgs<T>* __restrict__ tab,
                                                                         PerSched S) {
  extern __shared__ __align__(16) unsigned char per_smem[];
  EmArgs<T>* A = reinterpret_cast<EmArgs<T>*>(per_smem);
  __shared__ int give_up;
  const int nph = S.r > 1 ? S.r + 1 : 1;
  {
    const int* src = reinterpret_cast<const int*>(tab);
    int* dst = reinterpret_cast<int*>(A);
    const int n = 2 * nph * (int)(sizeof(EmArgs<T>) / sizeof(int));
    for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
  }
  if (threadIdx.x == 0) give_up = 0;
  __syncthreads();
  for (int q = 0; q < S.NT; ++q) {
    const long long m = S.m0 + q;
    const int par = q & 1;
    for (int u = blockIdx.x; u < S.nU; u += gridDim.x) {
      int ph = 0, iu = u;
      if (iu < S.nFt) {
        ph = 1;
        while (ph < S.r && iu >= S.nF[ph]) { iu -= S.nF[ph]; ++ph; }
      } else {
        iu -= S.nFt;
      }
      EmArgs<T>& a = A[par * nph + ph];
      if (threadIdx.x < 32) {
        if (!unit_wait(S, q, ph, iu) && threadIdx.x == 0) give_up = 1;
      } else if (threadIdx.x == 32) {
        em_set_level(a, m, ph == 0 ? 1 : ph);
        if (ph > 0) a.b.recompute = 1;   // coarse E^{n+1} on the lines from level n (Eq. 5b)
      }
      __syncthreads();
      if (give_up) return;
      if (ph == 0) em_segment<T, PML, false, true>(a, iu);
      else if (ph == S.r) em_segment<T, false, true, true>(a, iu);
      else em_segment<T, false, false, true>(a, iu);
      __syncthreads();
      if (threadIdx.x == 0) unit_done(S, q, ph, iu);
    }
  }
}

}  // namespace dmr
