// Block-CSR (BSR) kernels for the algebraic levels (Sec. 3.2, Sec. 4): SpMV / residual /
// point-block Jacobi, rectangular transfers with P and R = P^T, block diagonal inverses,
// transpose, the two-phase SpGEMM used for A T, A P and P^T (A P) (Eq. 9), prefix sums.
//
// SpGEMM: symbolic phase with one warp per output row and an open-addressing hash table in
// shared memory (global memory for rows whose candidate count exceeds the shared table);
// columns of each output row are sorted by rank counting, so the result is canonical.
// Numeric phase: one lane per output block, A's row walked in order and B's row searched by
// bisection, so every block is accumulated in a fixed order (deterministic).
#include <algorithm>

#include "ops.h"

namespace tomg {

namespace {

// One stored block (NE values) into registers.  Neighbouring lanes read different blocks, so
// each load instruction touches one cache line per lane: where a block is a whole number of
// 16-byte words (6 x 6 in FP32 or FP64, 2 x 2) it is read in 16-byte words, four times fewer
// instructions and L1 lookups than scalar loads.  Blocks are contiguous from a 256-byte
// aligned base, so block p starts on a 16-byte boundary whenever its size is a multiple of 16.
template <int NE, class T>
__device__ __forceinline__ void load_block(const T* __restrict__ blk, T* v) {
  if constexpr ((NE * sizeof(T)) % 16 == 0) {
    constexpr int W = 16 / sizeof(T);
    const float4* q = reinterpret_cast<const float4*>(blk);
#pragma unroll
    for (int k = 0; k < NE / W; k++) {
      const float4 w = __ldg(q + k);
      memcpy(v + W * k, &w, 16);
    }
  } else {
#pragma unroll
    for (int t = 0; t < NE; t++) v[t] = blk[t];
  }
}

// G lanes cooperate on one block row (strided over its blocks), partial sums combined with a
// fixed butterfly, so the result does not depend on scheduling.
template <int G, class T, int B>
__device__ __forceinline__ void group_reduce(T* acc) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < B; r++) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
}

template <class T, int B, int MODE, int G>
__global__ void __launch_bounds__(256) k_bsr(int nbr, const int* __restrict__ rp,
                                             const int* __restrict__ ci, const T* __restrict__ V,
                                             const T* __restrict__ x, T* __restrict__ y,
                                             const T* __restrict__ b, const T* __restrict__ Dinv,
                                             T omega, const int* done, T* __restrict__ xo, T c1,
                                             int dmode, T w0) {
  // operator data is fixed during a solve: the row bounds, this lane's first block and (small
  // blocks) the diagonal inverse are fetched before waiting for the producer of x and b
  constexpr bool PRE = B <= 3;
  constexpr bool NEED_D = MODE == MODE_JACOBI || MODE == MODE_CHEB || MODE == MODE_CHEB0;
  pdl_launch();
  {  // right-hand side blockIdx.y of a block solve
    const int64_t vo = (int64_t)blockIdx.y * rhs_stride((int64_t)B * nbr);
    if (x) x += vo;
    y += vo;
    if (b) b += vo;
    if (xo) xo += vo;
  }
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gtid / G, sub = gtid % G;
  const bool live = i < nbr;
  int p = 0, pend = 0, j0 = 0;
  T blk0[PRE ? B * B : 1];
  T Dl[PRE && NEED_D ? B * B : 1];
  if (PRE && live) {
    p = rp[i] + sub;
    pend = rp[i + 1];
    if (p < pend) {
      j0 = ci[p];
      load_block<B * B>(V + (int64_t)p * B * B, blk0);
    }
    if (NEED_D && sub == 0) {
#pragma unroll
      for (int t = 0; t < B * B; t++) Dl[t] = Dinv[(int64_t)B * B * i + t];
    }
  }
  pdl_wait();
  if (solve_done(done)) return;
  T acc[B];
#pragma unroll
  for (int r = 0; r < B; r++) acc[r] = T(0);
  if (live) {
    if (!PRE) {
      p = rp[i] + sub;
      pend = rp[i + 1];
    } else if (p < pend) {
      T xv[B];
      if (MODE == MODE_RESID0) {
        jacobi_first<T, B>(Dinv, b, j0, omega, xv);
      } else if (MODE == MODE_CHEB0) {
        jacobi_first<T, B>(Dinv, b, j0, w0, xv);
      } else {
#pragma unroll
        for (int c = 0; c < B; c++) xv[c] = x[(int64_t)B * j0 + c];
      }
#pragma unroll
      for (int r = 0; r < B; r++)
#pragma unroll
        for (int c = 0; c < B; c++) acc[r] += blk0[r * B + c] * xv[c];
      p += G;
    }
    for (; p < pend; p += G) {
      const int j = ci[p];
      T blk[B * B];
      load_block<B * B>(V + (int64_t)p * B * B, blk);
      T xv[B];
      if (MODE == MODE_RESID0) {
        jacobi_first<T, B>(Dinv, b, j, omega, xv);
      } else if (MODE == MODE_CHEB0) {
        jacobi_first<T, B>(Dinv, b, j, w0, xv);
      } else {
#pragma unroll
        for (int c = 0; c < B; c++) xv[c] = x[(int64_t)B * j + c];
      }
#pragma unroll
      for (int r = 0; r < B; r++)
#pragma unroll
        for (int c = 0; c < B; c++) acc[r] += blk[r * B + c] * xv[c];
    }
  }
  group_reduce<G, T, B>(acc);
  if (!live || sub != 0) return;
  if (MODE == MODE_RESID0) {
    T xi[B];
    jacobi_first<T, B>(Dinv, b, i, omega, xi);
#pragma unroll
    for (int r = 0; r < B; r++) {
      xo[(int64_t)B * i + r] = xi[r];
      y[(int64_t)B * i + r] = b[(int64_t)B * i + r] - acc[r];
    }
  } else if (MODE == MODE_APPLY) {
#pragma unroll
    for (int r = 0; r < B; r++) y[(int64_t)B * i + r] = acc[r];
  } else if (MODE == MODE_RESID) {
#pragma unroll
    for (int r = 0; r < B; r++) y[(int64_t)B * i + r] = b[(int64_t)B * i + r] - acc[r];
  } else {
    T res[B], xi[B], D[B * B];
    if (MODE == MODE_CHEB0) jacobi_first<T, B>(Dinv, b, i, w0, xi);
#pragma unroll
    for (int r = 0; r < B; r++) {
      res[r] = b[(int64_t)B * i + r] - acc[r];
      if (MODE != MODE_CHEB0) xi[r] = x[(int64_t)B * i + r];
    }
#pragma unroll
    for (int t = 0; t < B * B; t++) D[t] = PRE ? Dl[PRE && NEED_D ? t : 0] : Dinv[(int64_t)B * B * i + t];
#pragma unroll
    for (int r = 0; r < B; r++) {
      T v = T(0);
#pragma unroll
      for (int c = 0; c < B; c++) v += D[r * B + c] * res[c];
      if (MODE == MODE_CHEB || MODE == MODE_CHEB0) {
        const int dmo = MODE == MODE_CHEB0 ? 2 : dmode;
        const T prev = dmo == 2 ? xi[r] : (dmo == 1 ? xo[(int64_t)B * i + r] : T(0));
        const T dn = c1 * prev + omega * v;
        y[(int64_t)B * i + r] = xi[r] + dn;
        xo[(int64_t)B * i + r] = dn;
      } else {
        y[(int64_t)B * i + r] = xi[r] + omega * v;
      }
    }
  }
}

template <class T, int BR, int BC, int G>
__global__ void __launch_bounds__(256) k_bsr_rect(int nbr, int nbc, const int* __restrict__ rp,
                                                  const int* __restrict__ ci,
                                                  const T* __restrict__ V, const T* __restrict__ x,
                                                  T* __restrict__ y, int accumulate,
                                                  const int* done) {
  // the transfer operator is fixed during a solve: row bounds and this lane's first block are
  // fetched before waiting for the producer of x
  pdl_launch();
  x += (int64_t)blockIdx.y * rhs_stride((int64_t)BC * nbc);  // right-hand side blockIdx.y
  y += (int64_t)blockIdx.y * rhs_stride((int64_t)BR * nbr);
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gtid / G, sub = gtid % G;
  const bool live = i < nbr;
  int p = 0, pend = 0, j0 = 0;
  T blk0[BR * BC];
  if (live) {
    p = rp[i] + sub;
    pend = rp[i + 1];
    if (p < pend) {
      j0 = ci[p];
      load_block<BR * BC>(V + (int64_t)p * BR * BC, blk0);
    }
  }
  pdl_wait();
  if (solve_done(done)) return;
  T acc[BR];
#pragma unroll
  for (int r = 0; r < BR; r++) acc[r] = T(0);
  if (live && p < pend) {
#pragma unroll
    for (int c = 0; c < BC; c++) {
      const T xv = x[(int64_t)BC * j0 + c];
#pragma unroll
      for (int r = 0; r < BR; r++) acc[r] += blk0[r * BC + c] * xv;
    }
    for (p += G; p < pend; p += G) {
      const int j = ci[p];
      T blk[BR * BC];
      load_block<BR * BC>(V + (int64_t)p * BR * BC, blk);
#pragma unroll
      for (int c = 0; c < BC; c++) {
        const T xv = x[(int64_t)BC * j + c];
#pragma unroll
        for (int r = 0; r < BR; r++) acc[r] += blk[r * BC + c] * xv;
      }
    }
  }
  group_reduce<G, T, BR>(acc);
  if (!live || sub != 0) return;
#pragma unroll
  for (int r = 0; r < BR; r++) y[(int64_t)BR * i + r] = (accumulate ? y[(int64_t)BR * i + r] : T(0)) + acc[r];
}

// lanes per block row from the mean row length
inline int lanes_for(const Bsr& A) {
  const double avg = A.nbr > 0 ? (double)A.nnzb / A.nbr : 1.0;
  return avg <= 6 ? 4 : (avg <= 20 ? 8 : (avg <= 48 ? 16 : 32));
}

template <int B>
__global__ void k_bsr_diag(int nbr, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ V, double* Dinv64, float* Dinv32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  double D[B * B], Di[B * B];
  for (int t = 0; t < B * B; t++) D[t] = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; p++)
    if (ci[p] == i)
      for (int t = 0; t < B * B; t++) D[t] = V[(int64_t)p * B * B + t];
  spd_inverse<B>(D, Di);
  for (int t = 0; t < B * B; t++) {
    Dinv64[(int64_t)B * B * i + t] = Di[t];
    Dinv32[(int64_t)B * B * i + t] = (float)Di[t];
  }
}

__global__ void k_bsr_dense(int nbr, int b, int64_t n, const int* __restrict__ rp,
                            const int* __restrict__ ci, const double* __restrict__ V, double* A) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= nbr) return;
  for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
    const int j = ci[p];
    for (int r = 0; r < b; r++)
      for (int c = 0; c < b; c++) A[((int64_t)b * i + r) * n + (int64_t)b * j + c] = V[((int64_t)p * b + r) * b + c];
  }
}

__global__ void k_col_counts(int nbr, const int* __restrict__ rp, const int* __restrict__ ci,
                             int* counts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  for (int p = rp[i]; p < rp[i + 1]; p++) atomicAdd(&counts[ci[p]], 1);
}

__global__ void k_transpose_scatter(int nbr, const int* __restrict__ rp, const int* __restrict__ ci,
                                    const int* __restrict__ rpT, int* cursor, int* rowT, int* srcT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  for (int p = rp[i]; p < rp[i + 1]; p++) {
    const int j = ci[p];
    const int pos = rpT[j] + atomicAdd(&cursor[j], 1);
    rowT[pos] = i;
    srcT[pos] = p;
  }
}

// one warp per row of the transpose: every entry goes to its rank by source row (the source
// rows of one column are distinct), and its block is copied transposed
__global__ void k_transpose_finish(int nbc, int br, int bc, const int* __restrict__ rpT,
                                   const int* __restrict__ rowU, const int* __restrict__ srcU,
                                   int* ciT, const double* __restrict__ V, double* VT) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (j >= nbc) return;
  const int a = rpT[j], e = rpT[j + 1];
  for (int p = a + lane; p < e; p += 32) {
    const int kr = rowU[p];
    int rank = 0;
    for (int q = a; q < e; q++) rank += rowU[q] < kr ? 1 : 0;
    const int dstp = a + rank;
    ciT[dstp] = kr;
    const double* src = V + (int64_t)srcU[p] * br * bc;
    double* dst = VT + (int64_t)dstp * br * bc;
    for (int r = 0; r < br; r++)
      for (int c = 0; c < bc; c++) dst[c * br + r] = src[r * bc + c];
  }
}

// ------------------------------- SpGEMM ------------------------------------------------
constexpr int SPG_WARPS = 2;
constexpr int SPG_SMEM_T = 2048;

__device__ __forceinline__ int next_pow2(int x) { return x <= 1 ? 1 : 1 << (32 - __clz(x - 1)); }
__device__ __forceinline__ int warp_sum_int(int v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned hash_col(int key) { return (unsigned)key * 2654435761u; }
// hash table size of a row of C: twice the bound on its distinct columns (products summed over
// A's row, at most B's column count), a power of two; a row whose distinct columns cannot
// exceed the shared-memory table uses that table even when the sum of products is larger
// (linear probing ends: there are never more keys than slots)
__device__ __forceinline__ int spg_table(int ub, int nbcB) {
  const int lim = min(ub, nbcB);
  int T = max(64, next_pow2(2 * lim));
  if (T > SPG_SMEM_T && lim <= SPG_SMEM_T) T = SPG_SMEM_T;
  return T;
}

// per-row hash table size when it does not fit in shared memory (0 otherwise)
__global__ void k_spgemm_big(int nrows, const int* __restrict__ Arp, const int* __restrict__ Aci,
                             const int* __restrict__ Brp, int nbcB, int* big) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrows) return;
  int ub = 0;
  for (int a = Arp[row]; a < Arp[row + 1]; a++) ub += Brp[Aci[a] + 1] - Brp[Aci[a]];
  const int T = spg_table(ub, nbcB);
  big[row] = (T > SPG_SMEM_T) ? 2 * T : 0;  // table + compaction area
}

__global__ void __launch_bounds__(32 * SPG_WARPS)
    k_spgemm_sym(int nrows, const int* __restrict__ Arp, const int* __restrict__ Aci,
                 const int* __restrict__ Brp, const int* __restrict__ Bci, int nbcB,
                 const int* __restrict__ goff, int* gtable, int* countsC,
                 const int* __restrict__ rpC, int* ciC) {
  __shared__ int tab[SPG_WARPS][SPG_SMEM_T];
  __shared__ int cmp[SPG_WARPS][SPG_SMEM_T];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * SPG_WARPS + w;
  if (row >= nrows) return;  // warp-uniform
  int ub = 0;
  for (int a = Arp[row] + lane; a < Arp[row + 1]; a += 32) ub += Brp[Aci[a] + 1] - Brp[Aci[a]];
  ub = warp_sum_int(ub);
  const int T = spg_table(ub, nbcB);
  int* table = (T <= SPG_SMEM_T) ? tab[w] : gtable + goff[row];
  for (int s = lane; s < T; s += 32) table[s] = -1;
  __syncwarp();
  int newc = 0;
  for (int a = Arp[row]; a < Arp[row + 1]; a++) {
    const int k = Aci[a];
    for (int q = Brp[k] + lane; q < Brp[k + 1]; q += 32) {
      const int key = Bci[q];
      unsigned h = hash_col(key) & (unsigned)(T - 1);
      while (true) {
        const int prev = atomicCAS(&table[h], -1, key);
        if (prev == -1) { newc++; break; }
        if (prev == key) break;
        h = (h + 1) & (unsigned)(T - 1);
      }
    }
  }
  newc = warp_sum_int(newc);
  __syncwarp();
  if (countsC) {
    if (lane == 0) countsC[row] = newc;
    return;
  }
  // compact the occupied slots (warp ballot prefix), then place every key at its rank
  int* ck = (T <= SPG_SMEM_T) ? cmp[w] : table + T;
  int cnt = 0;
  for (int s0 = 0; s0 < T; s0 += 32) {
    const int key = table[s0 + lane];
    const bool occ = key != -1;
    const unsigned bal = __ballot_sync(0xffffffffu, occ);
    if (occ) ck[cnt + __popc(bal & ((1u << lane) - 1u))] = key;
    cnt += __popc(bal);
  }
  __syncwarp();
  const int base = rpC[row];
  for (int q = lane; q < cnt; q += 32) {
    const int key = ck[q];
    int rank = 0;
    for (int t = 0; t < cnt; t++) rank += (ck[t] < key) ? 1 : 0;
    ciC[base + rank] = key;
  }
}

// position of column c in row r of a CSR pattern (sorted columns), or -1
__device__ __forceinline__ int64_t csr_find(const int* __restrict__ rp, const int* __restrict__ ci,
                                            int r, int c) {
  int l = rp[r], h = rp[r + 1];
  const int end = h;
  while (l < h) {
    const int mid = (l + h) >> 1;
    if (ci[mid] < c) l = mid + 1;
    else h = mid;
  }
  return (l < end && ci[l] == c) ? l : -1;
}

// Numeric phase for long rows of A (the coarse Galerkin products): one warp per output block,
// the lanes split A's row and their partial blocks are combined by a fixed butterfly, so the
// work of one output block is spread over 32 lanes instead of one (still deterministic).  With
// sym set (C = P^T A P, symmetric, square blocks) the warp of an upper block (j > row) also
// writes its transpose into the mirror block, and the warp of a lower block with a mirror does
// nothing: half the FP64 work, and C symmetric to the last bit.
template <int BR, int BK, int BC>
__global__ void __launch_bounds__(128) k_spgemm_num_w(int nrows, int64_t nnzC,
                                                      const int* __restrict__ Arp,
                                                      const int* __restrict__ Aci,
                                                      const double* __restrict__ VA,
                                                      const int* __restrict__ Brp,
                                                      const int* __restrict__ Bci,
                                                      const double* __restrict__ VB,
                                                      const int* __restrict__ Crp,
                                                      const int* __restrict__ Cci, double* VC,
                                                      int sym) {
  const int64_t pc = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (pc >= nnzC) return;  // warp-uniform
  int lo = 0, hi = nrows;  // the row: Crp[lo] <= pc < Crp[lo + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (Crp[mid] <= pc) lo = mid;
    else hi = mid;
  }
  const int row = lo, j = Cci[pc];
  int64_t mirror = -1;
  if (BR == BC && sym && j != row) {
    mirror = csr_find(Crp, Cci, j, row);  // warp-uniform
    if (j < row && mirror >= 0) return;   // written by the warp of block (j, row)
    if (j < row) mirror = -1;
  }
  double acc[BR * BC];
#pragma unroll
  for (int t = 0; t < BR * BC; t++) acc[t] = 0.0;
  for (int a = Arp[row] + lane; a < Arp[row + 1]; a += 32) {
    const int k = Aci[a];
    const int bh = Brp[k + 1];
    int l = Brp[k], h = bh;
    while (l < h) {
      const int mid = (l + h) >> 1;
      if (Bci[mid] < j) l = mid + 1;
      else h = mid;
    }
    if (l >= bh || Bci[l] != j) continue;
    const double* Ab = VA + (int64_t)a * BR * BK;
    const double* Bb = VB + (int64_t)l * BK * BC;
#pragma unroll
    for (int r = 0; r < BR; r++)
#pragma unroll
      for (int t = 0; t < BK; t++) {
        const double av = Ab[r * BK + t];
#pragma unroll
        for (int c = 0; c < BC; c++) acc[r * BC + c] += av * Bb[t * BC + c];
      }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int t = 0; t < BR * BC; t++) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
  double* Cb = VC + pc * BR * BC;
#pragma unroll
  for (int t = 0; t < BR * BC; t++)
    if (lane == (t & 31)) Cb[t] = acc[t];
  if (BR == BC && mirror >= 0) {
    double* Ct = VC + mirror * BR * BC;
#pragma unroll
    for (int t = 0; t < BR * BC; t++)
      if (lane == (t & 31)) Ct[(t % BC) * BR + t / BC] = acc[t];
  }
}

// Numeric phase, one warp per row of C: for each output block of the row the lanes first
// search B's rows for the block column j in parallel (lane q takes A block q of the row), then
// every hit, in ascending order of A's blocks, is applied by all lanes at once, lane q owning
// scalars q and q + 32 of the BR x BC output block.  Each scalar sums A[r][t] B[t][c] over the
// hits in A's order and t ascending (the order of a one-thread-per-block loop), and no FP64
// instruction runs for a block that only some lanes would use.
template <int BR, int BK, int BC>
__global__ void __launch_bounds__(128) k_spgemm_num_s(int nrows, const int* __restrict__ Arp,
                                                      const int* __restrict__ Aci,
                                                      const double* __restrict__ VA,
                                                      const int* __restrict__ Brp,
                                                      const int* __restrict__ Bci,
                                                      const double* __restrict__ VB,
                                                      const int* __restrict__ Crp,
                                                      const int* __restrict__ Cci, double* VC) {
  constexpr int NS = BR * BC;
  static_assert(NS <= 64, "two output scalars per lane at most");
  const int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= nrows) return;  // warp-uniform
  const int q0 = lane, q1 = lane + 32;
  const int r0 = q0 / BC, c0 = q0 % BC, r1 = q1 / BC, c1 = q1 % BC;
  const int a_lo = Arp[row], a_hi = Arp[row + 1];
  for (int pc = Crp[row]; pc < Crp[row + 1]; pc++) {
    const int j = Cci[pc];
    double acc0 = 0.0, acc1 = 0.0;
    for (int base = a_lo; base < a_hi; base += 32) {
      const int a = base + lane;
      int l = -1;
      if (a < a_hi) {
        const int k = Aci[a];
        const int bh = Brp[k + 1];
        int lo = Brp[k], hi = bh;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (Bci[mid] < j) lo = mid + 1;
          else hi = mid;
        }
        if (lo < bh && Bci[lo] == j) l = lo;
      }
      unsigned hits = __ballot_sync(0xffffffffu, l >= 0);
      while (hits) {
        const int src = __ffs(hits) - 1;
        hits &= hits - 1u;
        const int lh = __shfl_sync(0xffffffffu, l, src);
        const double* Ab = VA + (int64_t)(base + src) * BR * BK;
        const double* Bb = VB + (int64_t)lh * BK * BC;
        if (q0 < NS) {
#pragma unroll
          for (int t = 0; t < BK; t++) acc0 += Ab[r0 * BK + t] * Bb[t * BC + c0];
        }
        if (NS > 32 && q1 < NS) {
#pragma unroll
          for (int t = 0; t < BK; t++) acc1 += Ab[r1 * BK + t] * Bb[t * BC + c1];
        }
      }
    }
    double* Cb = VC + (int64_t)pc * NS;
    if (q0 < NS) Cb[q0] = acc0;
    if (NS > 32 && q1 < NS) Cb[q1] = acc1;
  }
}

template <class A, class B>
__global__ void k_cast(const A* __restrict__ a, B* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (B)a[i];
}

// ------------------------------- scan --------------------------------------------------
constexpr int SCAN_B = 1024;
__global__ void k_scan_block(const int* __restrict__ in, int* out, int64_t n, int* sums) {
  __shared__ int warp_tot[32];
  const int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  const int v = (i < n) ? in[i] : 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = warp_tot[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  const int incl = x + (w > 0 ? warp_tot[w - 1] : 0);
  if (i < n) out[i] = incl - v;
  if (threadIdx.x == SCAN_B - 1) sums[blockIdx.x] = incl;
}
__global__ void k_scan_add(int* out, int64_t n, const int* offs) {
  const int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  if (i < n) out[i] += offs[blockIdx.x];
}

void scan_rec(cudaStream_t s, const int* in, int* out, int64_t n, int* total_dev) {
  // writes exclusive scan of in[0..n) to out[0..n) and the total to *total_dev
  const int nb = ceil_div(n, SCAN_B);
  DBuf<int> sums, offs;
  sums.resize(nb);
  offs.resize(nb + 1);
  LAUNCH(k_scan_block, nb, SCAN_B, 0, s, in, out, n, sums.p);
  if (nb == 1) {
    CK(cudaMemcpyAsync(total_dev, sums.p, sizeof(int), cudaMemcpyDeviceToDevice, s));
  } else {
    scan_rec(s, sums.p, offs.p, nb, total_dev);
    LAUNCH(k_scan_add, nb, SCAN_B, 0, s, out, n, offs.p);
  }
  CK(cudaStreamSynchronize(s));  // temporaries are freed on return
}

}  // namespace

template <class T>
void bsr_op(cudaStream_t s, int mode, const Bsr& A, const T* V, const T* x, T* y, const T* b,
            const T* Dinv, double omega, const int* done, const ChebArg* ch) {
  if (reinterpret_cast<uintptr_t>(V) % 16) TOMG_THROW(TOMG_E_INVALID, "block values not 16-byte aligned");
  const int G = lanes_for(A);
  const dim3 grid(ceil_div((int64_t)A.nbr * G, 256), batch_rhs());
  const bool cheb = mode == MODE_CHEB || mode == MODE_CHEB0;
  if (cheb && !ch) TOMG_THROW(TOMG_E_INVALID, "Chebyshev step without its state");
  T* xo = mode == MODE_RESID0 ? const_cast<T*>(x) : (cheb ? (T*)ch->d : nullptr);
  const T c1 = cheb ? (T)ch->c1 : T(0);
  const int dm = cheb ? ch->dmode : 0;
  const T w0 = cheb ? (T)ch->w0 : T(0);
#define BOP(B, M, GG) LAUNCH((k_bsr<T, B, M, GG>), grid, 256, 0, s, A.nbr, A.rp, A.ci, V, x, y, b, Dinv, (T)omega, done, xo, c1, dm, w0)
#define BG(B, M)                         \
  if (G == 4) BOP(B, M, 4);              \
  else if (G == 8) BOP(B, M, 8);         \
  else if (G == 16) BOP(B, M, 16);       \
  else BOP(B, M, 32);
#define BMODES(B)                                   \
  if (mode == MODE_APPLY) { BG(B, MODE_APPLY) }     \
  else if (mode == MODE_RESID) { BG(B, MODE_RESID) } \
  else if (mode == MODE_RESID0) { BG(B, MODE_RESID0) } \
  else if (mode == MODE_CHEB) { BG(B, MODE_CHEB) } \
  else if (mode == MODE_CHEB0) { BG(B, MODE_CHEB0) } \
  else { BG(B, MODE_JACOBI) }
  if (A.br == 2) { BMODES(2) }
  else if (A.br == 3) { BMODES(3) }
  else if (A.br == 6) { BMODES(6) }
  else TOMG_THROW(TOMG_E_INVALID, "unsupported block size %d", A.br);
#undef BMODES
#undef BG
#undef BOP
}
template void bsr_op<float>(cudaStream_t, int, const Bsr&, const float*, const float*, float*,
                            const float*, const float*, double, const int*, const ChebArg*);
template void bsr_op<double>(cudaStream_t, int, const Bsr&, const double*, const double*, double*,
                             const double*, const double*, double, const int*, const ChebArg*);

template <class T>
void bsr_spmv_rect(cudaStream_t s, const Bsr& A, const T* V, const T* x, T* y, int accumulate,
                   const int* done) {
  if (reinterpret_cast<uintptr_t>(V) % 16) TOMG_THROW(TOMG_E_INVALID, "block values not 16-byte aligned");
  const int G = lanes_for(A);
  const dim3 grid(ceil_div((int64_t)A.nbr * G, 256), batch_rhs());
#define RL(R, C, GG) LAUNCH((k_bsr_rect<T, R, C, GG>), grid, 256, 0, s, A.nbr, A.nbc, A.rp, A.ci, V, x, y, accumulate, done)
#define RECT(R, C)                     \
  if (A.br == R && A.bc == C) {        \
    if (G == 4) RL(R, C, 4);           \
    else if (G == 8) RL(R, C, 8);      \
    else if (G == 16) RL(R, C, 16);    \
    else RL(R, C, 32);                 \
    return;                            \
  }
  RECT(2, 2) RECT(3, 3) RECT(6, 6) RECT(2, 3) RECT(3, 2) RECT(3, 6) RECT(6, 3)
#undef RECT
#undef RL
  TOMG_THROW(TOMG_E_INVALID, "unsupported transfer block %dx%d", A.br, A.bc);
}
template void bsr_spmv_rect<float>(cudaStream_t, const Bsr&, const float*, const float*, float*,
                                   int, const int*);
template void bsr_spmv_rect<double>(cudaStream_t, const Bsr&, const double*, const double*,
                                    double*, int, const int*);

void bsr_block_diag_inv(cudaStream_t s, const Bsr& A, const double* V, double* D64, float* D32) {
  const int grid = ceil_div(A.nbr, 128);
  if (A.br == 2) LAUNCH(k_bsr_diag<2>, grid, 128, 0, s, A.nbr, A.rp, A.ci, V, D64, D32);
  else if (A.br == 3) LAUNCH(k_bsr_diag<3>, grid, 128, 0, s, A.nbr, A.rp, A.ci, V, D64, D32);
  else if (A.br == 6) LAUNCH(k_bsr_diag<6>, grid, 128, 0, s, A.nbr, A.rp, A.ci, V, D64, D32);
  else TOMG_THROW(TOMG_E_INVALID, "unsupported block size %d", A.br);
}

void bsr_to_dense(cudaStream_t s, const Bsr& A, const double* V, double* Ad) {
  const int64_t n = (int64_t)A.nbr * A.br;
  CK(cudaMemsetAsync(Ad, 0, sizeof(double) * n * n, s));
  LAUNCH(k_bsr_dense, ceil_div((int64_t)A.nbr * 32, 128), 128, 0, s, A.nbr, A.br, n, A.rp, A.ci, V, Ad);
}

void bsr_col_counts(cudaStream_t s, const Bsr& A, int* counts) {
  CK(cudaMemsetAsync(counts, 0, sizeof(int) * A.nbc, s));
  LAUNCH(k_col_counts, ceil_div(A.nbr, 256), 256, 0, s, A.nbr, A.rp, A.ci, counts);
}

void bsr_transpose_fill(cudaStream_t s, const Bsr& A, const double* V, const int* rpT, int* ciT,
                        double* VT, int* cursor) {
  DBuf<int> src, rowu;
  src.resize(A.nnzb > 0 ? A.nnzb : 1);
  rowu.resize(A.nnzb > 0 ? A.nnzb : 1);
  CK(cudaMemsetAsync(cursor, 0, sizeof(int) * A.nbc, s));
  LAUNCH(k_transpose_scatter, ceil_div(A.nbr, 256), 256, 0, s, A.nbr, A.rp, A.ci, rpT, cursor,
         rowu.p, src.p);
  LAUNCH(k_transpose_finish, ceil_div((int64_t)A.nbc * 32, 128), 128, 0, s, A.nbc, A.br, A.bc,
         rpT, rowu.p, src.p, ciT, V, VT);
}

void spgemm_counts(cudaStream_t s, const Bsr& A, const Bsr& B, int* counts, SpgemmWork& w) {
  w.big.resize(A.nbr + 1);
  w.goff.resize(A.nbr + 1);
  LAUNCH(k_spgemm_big, ceil_div(A.nbr, 256), 256, 0, s, A.nbr, A.rp, A.ci, B.rp, B.nbc, w.big.p);
  const int64_t tot = exclusive_scan(s, w.big.p, w.goff.p, A.nbr);
  if (tot > 0x7fffffffLL) TOMG_THROW(TOMG_E_OOM, "SpGEMM hash tables too large (%lld)", (long long)tot);
  w.gtable.resize(tot > 0 ? tot : 1);
  LAUNCH(k_spgemm_sym, ceil_div(A.nbr, SPG_WARPS), 32 * SPG_WARPS, 0, s, A.nbr, A.rp, A.ci, B.rp,
         B.ci, B.nbc, w.goff.p, w.gtable.p, counts, (const int*)nullptr, (int*)nullptr);
}

void spgemm_fill(cudaStream_t s, const Bsr& A, const Bsr& B, const int* rpC, int* ciC,
                 SpgemmWork& w) {
  LAUNCH(k_spgemm_sym, ceil_div(A.nbr, SPG_WARPS), 32 * SPG_WARPS, 0, s, A.nbr, A.rp, A.ci, B.rp,
         B.ci, B.nbc, w.goff.p, w.gtable.p, (int*)nullptr, rpC, ciC);
}

void spgemm_numeric(cudaStream_t s, const Bsr& A, const double* VA, const Bsr& B, const double* VB,
                    const Bsr& C, double* VC, bool sym) {
  const int grid = ceil_div((int64_t)A.nbr * 32, 128);
  // few rows with many products per output block (the coarse Galerkin products: about 4 per
  // block for A P on the first AMG level, a hundred and more for R (A P)): one warp per output
  // block, the lanes over A's row.  Fewer products per block (A T: about one) keep the
  // row-per-warp kernel, whose lanes own the output scalars (no butterfly per output block)
  const double per_block = (double)A.nnzb * ((double)B.nnzb / std::max(1, B.nbr)) /
                           (double)std::max<int64_t>(1, C.nnzb);
  const bool long_rows = A.nbr > 0 && A.nbr < 4096 && per_block >= 3.0;
  const int gridw = (int)std::max<int64_t>(1, ceil_div(C.nnzb * 32, 128));
#define NUM(R, K, CC)                                                                          \
  if (A.br == R && A.bc == K && B.bc == CC) {                                                  \
    if (long_rows) {                                                                           \
      if (C.nnzb > 0)                                                                          \
        LAUNCH((k_spgemm_num_w<R, K, CC>), gridw, 128, 0, s, A.nbr, C.nnzb, A.rp, A.ci, VA,     \
               B.rp, B.ci, VB, C.rp, C.ci, VC, sym ? 1 : 0);                                   \
      return;                                                                                  \
    }                                                                                          \
    LAUNCH((k_spgemm_num_s<R, K, CC>), grid, 128, 0, s, A.nbr, A.rp, A.ci, VA, B.rp, B.ci, VB, \
           C.rp, C.ci, VC);                                                                    \
    return;                                                                                    \
  }
  NUM(2, 2, 3) NUM(3, 3, 3) NUM(3, 3, 6) NUM(6, 6, 6) NUM(3, 2, 3) NUM(6, 3, 6) NUM(2, 2, 2)
#undef NUM
  TOMG_THROW(TOMG_E_INVALID, "SpGEMM block shape %dx%d * %dx%d not instantiated", A.br, A.bc, B.br, B.bc);
}

void cast_f64_f32(cudaStream_t s, const double* a, float* b, int64_t n) {
  if (n > 0) LAUNCH((k_cast<double, float>), ceil_div(n, 256), 256, 0, s, a, b, n);
}
void cast_f32_f64(cudaStream_t s, const float* a, double* b, int64_t n) {
  if (n > 0) LAUNCH((k_cast<float, double>), ceil_div(n, 256), 256, 0, s, a, b, n);
}

void exclusive_scan_nosync(cudaStream_t s, const int* in, int* out, int64_t n) {
  if (n == 0) {
    CK(cudaMemsetAsync(out, 0, sizeof(int), s));
    return;
  }
  scan_rec(s, in, out, n, out + n);
}

int64_t exclusive_scan(cudaStream_t s, const int* in, int* out, int64_t n) {
  if (n == 0) {
    CK(cudaMemsetAsync(out, 0, sizeof(int), s));
    return 0;
  }
  scan_rec(s, in, out, n, out + n);
  int tot = 0;
  CK(cudaMemcpyAsync(&tot, out + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return tot;
}

}  // namespace tomg
