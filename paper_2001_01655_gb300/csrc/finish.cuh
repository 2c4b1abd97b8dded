// Device-side completion of the outer Krylov reductions (Sec. 3.1 CG / flexible CG).
//
// A kernel that produces per-block FP64 partials of a dot product can finish the reduction
// itself: every block writes its partial, takes a ticket, and the block that arrives last adds
// all partials in block order (the same fixed order as a separate single-block pass, so the
// result does not depend on scheduling) and updates the scalar state.  This removes one kernel
// launch per reduction from the iteration.
#pragma once

#include "ops.h"

namespace tomg {

// True in exactly one of the nblk blocks that share `ticket`: the last one to arrive, after
// every one of them has made its partials visible (nblk = the whole grid, or the blocks of one
// right-hand side of a block solve, which each have their own ticket).  All threads of every
// block must call it (no early exit before it).  The ticket is left at zero for the next launch.
__device__ __forceinline__ bool last_block(unsigned* ticket, unsigned nblk) {
  __shared__ unsigned s_last;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == nblk - 1) ? 1u : 0u;
    if (s_last) *ticket = 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0u;
}

// Adds the partials pa[0..na) and pb[0..nb) in a fixed order with the whole (1D) block and
// applies step `kind` of the scalar recurrence.  The partials are read past L1 (they were
// written by other blocks of the same grid).
__device__ inline void finish_body(int kind, const double* pa, int na, const double* pb, int nb,
                                   Scalars* sc, double* sred) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < na; i += blockDim.x) a += __ldcg(pa + i);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) b += __ldcg(pb + i);
  a = block_sum(a, sred);
  b = block_sum(b, sred);
  if (threadIdx.x != 0) return;
  switch (kind) {
    case FIN_INIT:  // a = r.r, b = b.b
      sc->rr = a;
      sc->bb = b;
      sc->tol2 = sc->rtol2 * b;
      sc->it = 0;
      sc->status = TOMG_OK;
      sc->done = (b == 0.0 || a <= sc->tol2) ? 1 : 0;
      if (a != a) { sc->status = TOMG_E_BREAKDOWN; sc->done = 1; }
      break;
    case FIN_RZ0:
      sc->rz = a;
      // CG needs z.r > 0 (SPD preconditioner); flexible CG only needs a finite value
      if (sc->flexible ? (a != a) : !(a > 0.0)) { sc->status = TOMG_E_BREAKDOWN; sc->done = 1; sc->pad = 2; }
      break;
    case FIN_ALPHA:
      sc->pq = a;
      if (!(a > 0.0)) { sc->status = TOMG_E_BREAKDOWN; sc->done = 1; sc->pad = 3; break; }
      sc->alpha = sc->rz / a;
      break;
    case FIN_RR:
      sc->rr = a;
      sc->it += 1;
      if (a != a) { sc->status = TOMG_E_BREAKDOWN; sc->done = 1; sc->pad = 1; }
      else if (a <= sc->tol2) { sc->done = 1; }
      else if (sc->it >= sc->max_iter) { sc->status = TOMG_NOT_CONVERGED; sc->done = 1; }
      break;
    case FIN_BETA:  // a = z.r (new), b = z.q
      // CG: beta = z.r / z_old.r_old.  Flexible CG (Notay 2000): beta = z^T (r - r_old) /
      // z_old.r_old = -alpha z.q / z_old.r_old = -z.q / p.q, which needs no sign of z.r.
      if (sc->flexible ? (a != a || b != b) : !(a > 0.0)) {
        sc->status = TOMG_E_BREAKDOWN; sc->done = 1; sc->pad = 4; break;
      }
      sc->rz_new = a;
      sc->zq = b;
      sc->beta = sc->flexible ? (-b / sc->pq) : (a / sc->rz);
      sc->rz = a;
      break;
  }
  __threadfence();
}

}  // namespace tomg
