// Smoothed-aggregation setup on the device (Sec. 3.2 AMG; Sec. 4: strength measured per node block,
// rigid-body candidates, Jacobi-smoothed tentative prolongator):
//   strength   ||A_ij||_F^2 > beta ||A_ii||_F ||A_jj||_F, one value per node   (Eq. 10)
//   aggregates distance-2 maximal independent set in synchronous rounds with splitmix64
//              priorities (Bell, Dalton & Olson 2012), then two attachment phases
//   tentative  modified Gram-Schmidt QR of the candidates on every aggregate
//   smoothing  P = T - omega D^-1 A T, omega = 4 / (3 rho(D^-1 A)), rho by power iteration
// splitmix64 is written here from its published definition (Steele, Lea & Flood 2014).
#include "finish.cuh"

namespace tomg {

namespace {

constexpr uint64_t SALT_MIS = 0x4D495332ull;
constexpr uint64_t SALT_POWER = 0x504F5752ull;
constexpr uint64_t TOP = ~0ull;
enum { UND = 0, IN = 1, OUT = 2 };

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t mis_key(int64_t i, int level) {
  const uint64_t h = splitmix64((uint64_t)i + (SALT_MIS << 24) + ((uint64_t)level << 40));
  return ((h >> 33) << 32) + (uint64_t)i + 1ull;
}

__device__ __forceinline__ double block_fro(const double* blk, int bb) {
  double s = 0.0;
  for (int t = 0; t < bb; t++) s += blk[t] * blk[t];
  return sqrt(s);
}

__global__ void k_diag_fro(int nbr, int b, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ V, double* dnorm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  double d = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; p++)
    if (ci[p] == i) d = block_fro(V + (int64_t)p * b * b, b * b);
  dnorm[i] = d;
}

// one warp per node row; strong neighbours are compacted in column order (ballot prefix)
__global__ void k_strength(int nbr, int b, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ V, const double* __restrict__ dnorm,
                           double beta, int* counts, const int* __restrict__ srp, int* sci) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= nbr) return;
  const double di = dnorm[i];
  const int base = srp ? srp[i] : 0;
  int cnt = 0;
  for (int p0 = rp[i]; p0 < rp[i + 1]; p0 += 32) {
    const int p = p0 + lane;
    bool strong = false;
    int j = -1;
    if (p < rp[i + 1]) {
      j = ci[p];
      if (j != i) {
        const double F = block_fro(V + (int64_t)p * b * b, b * b);
        strong = F * F > beta * di * dnorm[j];
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, strong);
    if (strong && srp) sci[base + cnt + __popc(bal & ((1u << lane) - 1u))] = j;
    cnt += __popc(bal);
  }
  if (counts && lane == 0) counts[i] = cnt;
}

// All MIS-2 rounds in one cooperative launch (every block resident): the three phases of a
// round (values, neighbour maxima, update) are separated by a grid barrier, and the blocks stop
// together after the first round that leaves no node undecided.  Per round: v = TOP for a node
// in the set, its key for an undecided node, 0 otherwise; m1 = the largest v within distance 1;
// an undecided node whose largest m1 within distance 1 is TOP leaves, one whose own key is that
// maximum joins (distance-2 independence).  Values written by other blocks
// are read past L1 (ld.global.cg).  Barrier waits are bounded: a block that gives up sets
// sync[4] and leaves, and so do the others when their own waits run out.
//   sync[0] arrivals, sync[1] generation, sync[2..3] undecided counts of even / odd rounds,
//   sync[4] error, sync[5] rounds run
constexpr unsigned MIS_WAIT_LIMIT = 1u << 24;

int g_grid_wait_polls = 0;  // test hook: > 0 replaces the grid barriers' wait limits

__global__ void __launch_bounds__(256) k_mis2_loop(int n, int level, const int* __restrict__ srp,
                                                   const int* __restrict__ sci, int* state,
                                                   uint64_t* v, uint64_t* m1, unsigned* sync,
                                                   int max_rounds, unsigned wait_limit) {
  auto grid_barrier = [&](unsigned* sy, unsigned nblocks) {
    return grid_sync(sy, sy + 4, nblocks, wait_limit);
  };
  __shared__ unsigned red[8];
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nb = gridDim.x;
  for (int i = t0; i < n; i += stride) state[i] = (srp[i + 1] == srp[i]) ? OUT : UND;
  if (!grid_barrier(sync, nb)) return;
  for (int r = 0; r < max_rounds; r++) {
    for (int i = t0; i < n; i += stride) {
      const int st = state[i];
      v[i] = (st == IN) ? TOP : (st == UND ? mis_key(i, level) : 0ull);
    }
    if (!grid_barrier(sync, nb)) return;
    // the other round's count: every block has read it before the barrier above
    if (t0 == 0) sync[2 + ((r + 1) & 1)] = 0;
    for (int i = t0; i < n; i += stride) {
      uint64_t best = __ldcg(v + i);
      for (int p = srp[i]; p < srp[i + 1]; p++) best = max(best, __ldcg(v + sci[p]));
      m1[i] = best;
    }
    if (!grid_barrier(sync, nb)) return;
    unsigned und = 0;
    for (int i = t0; i < n; i += stride) {
      if (state[i] != UND) continue;
      uint64_t m2 = __ldcg(m1 + i);
      for (int p = srp[i]; p < srp[i + 1]; p++) m2 = max(m2, __ldcg(m1 + sci[p]));
      int st = UND;
      if (m2 == TOP) st = OUT;
      else if (m2 == mis_key(i, level)) st = IN;
      state[i] = st;
      und += st == UND ? 1u : 0u;
    }
    for (int o = 16; o > 0; o >>= 1) und += __shfl_xor_sync(0xffffffffu, und, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = und;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned tot = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += red[w];
      if (tot) atomicAdd(sync + 2 + (r & 1), tot);
    }
    if (!grid_barrier(sync, nb)) return;
    if (*(volatile unsigned*)(sync + 2 + (r & 1)) == 0) {
      if (t0 == 0) sync[5] = (unsigned)(r + 1);
      return;
    }
  }
  if (t0 == 0) sync[5] = (unsigned)max_rounds;
}

__global__ void k_root_flags(int n, const int* __restrict__ state, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flags[i] = (state[i] == IN) ? 1 : 0;
}
__global__ void k_agg_phase1(int n, const int* __restrict__ srp, const int* __restrict__ sci,
                             const int* __restrict__ state, const int* __restrict__ root_scan,
                             int* agg1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = -1;
  if (state[i] == IN) {
    a = root_scan[i];
  } else if (srp[i + 1] > srp[i]) {
    for (int p = srp[i]; p < srp[i + 1]; p++) {
      const int j = sci[p];
      if (state[j] == IN) { a = root_scan[j]; break; }
    }
  }
  agg1[i] = a;
}
__global__ void k_agg_phase2(int n, int level, const int* __restrict__ srp,
                             const int* __restrict__ sci, const int* __restrict__ agg1, int* agg2,
                             int* failures) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = agg1[i];
  if (a < 0 && srp[i + 1] > srp[i]) {
    uint64_t best = 0;
    for (int p = srp[i]; p < srp[i + 1]; p++) {
      const int j = sci[p];
      if (agg1[j] < 0) continue;
      const uint64_t kj = mis_key(j, level);
      if (kj > best) { best = kj; a = agg1[j]; }
    }
    if (a < 0) atomicAdd(failures, 1);
  }
  agg2[i] = a;
}

// members of each aggregate in ascending node order (counting sort + per-aggregate sort)
__global__ void k_agg_count(int n, const int* __restrict__ agg, int* cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) atomicAdd(&cnt[agg[i]], 1);
}
__global__ void k_agg_scatter(int n, const int* __restrict__ agg, const int* __restrict__ start,
                              int* cursor, int* members) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || agg[i] < 0) return;
  const int a = agg[i];
  members[start[a] + atomicAdd(&cursor[a], 1)] = i;
}
// the members of each aggregate in ascending node order: one warp per aggregate, each member
// placed at its rank (the count of smaller members; node ids are distinct)
__global__ void k_agg_sort(int n_agg, const int* __restrict__ start,
                           const int* __restrict__ unsorted, int* members) {
  const int a = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (a >= n_agg) return;
  const int s = start[a], e = start[a + 1];
  for (int p = s + lane; p < e; p += 32) {
    const int v = unsorted[p];
    int rank = 0;
    for (int q = s; q < e; q++) rank += unsorted[q] < v ? 1 : 0;
    members[s + rank] = v;
  }
}

__global__ void k_T_pattern(int n, const int* __restrict__ agg, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flags[i] = agg[i] >= 0 ? 1 : 0;
}
__global__ void k_T_cols(int n, const int* __restrict__ agg, int* Tci, const int* __restrict__ Trp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) Tci[Trp[i]] = agg[i];
}

// the aggregate's rows of B (m <= 32 RPL) held in registers, row t on lane t % 32: the same
// modified Gram-Schmidt as the general path below, operation for operation (padding rows are
// zero and add nothing)
constexpr int TENT_RPL = 8;
template <int K>
__device__ __forceinline__ void tentative_regs(int m, int b, const int* __restrict__ mem,
                                               const int* __restrict__ Trp,
                                               const double* __restrict__ B, double* TV,
                                               double* R, int lane) {
  double v[TENT_RPL][K];
#pragma unroll
  for (int j = 0; j < TENT_RPL; j++) {
    const int t = lane + 32 * j;
#pragma unroll
    for (int c = 0; c < K; c++) v[j][c] = 0.0;
    if (t < m) {
      const int node = mem[t / b];
#pragma unroll
      for (int c = 0; c < K; c++) v[j][c] = B[((int64_t)node * b + (t % b)) * K + c];
    }
  }
#pragma unroll
  for (int c = 0; c < K; c++) {
    double n0 = 0.0;
#pragma unroll
    for (int j = 0; j < TENT_RPL; j++) n0 += v[j][c] * v[j][c];
    for (int o = 16; o > 0; o >>= 1) n0 += __shfl_xor_sync(0xffffffffu, n0, o);
    n0 = sqrt(n0);
#pragma unroll
    for (int i = 0; i < c; i++) {
      double d = 0.0;
#pragma unroll
      for (int j = 0; j < TENT_RPL; j++) d += v[j][i] * v[j][c];
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (lane == 0) R[i * K + c] = d;
#pragma unroll
      for (int j = 0; j < TENT_RPL; j++) v[j][c] -= d * v[j][i];
    }
    double nr = 0.0;
#pragma unroll
    for (int j = 0; j < TENT_RPL; j++) nr += v[j][c] * v[j][c];
    for (int o = 16; o > 0; o >>= 1) nr += __shfl_xor_sync(0xffffffffu, nr, o);
    nr = sqrt(nr);
    const bool live = n0 > 0.0 && nr > 1e-8 * n0;
#pragma unroll
    for (int j = 0; j < TENT_RPL; j++) v[j][c] = live ? v[j][c] / nr : 0.0;
    if (lane == 0) R[c * K + c] = live ? nr : 0.0;
  }
#pragma unroll
  for (int j = 0; j < TENT_RPL; j++) {
    const int t = lane + 32 * j;
    if (t < m) {
      const int node = mem[t / b];
#pragma unroll
      for (int c = 0; c < K; c++) TV[((int64_t)Trp[node] * b + (t % b)) * K + c] = v[j][c];
    }
  }
}

// one warp per aggregate: modified Gram-Schmidt on the aggregate's rows of B (m x k), written
// in place into the T blocks (b x k per member node); R goes to Bc (k x k per aggregate)
__global__ void k_tentative(int n_agg, int b, int k, const int* __restrict__ start,
                            const int* __restrict__ members, const int* __restrict__ Trp,
                            const double* __restrict__ B, double* TV, double* Bc) {
  const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (a >= n_agg) return;
  const int s = start[a], e = start[a + 1];
  const int m = (e - s) * b;
  if (m <= 32 * TENT_RPL && (k == 3 || k == 6)) {  // warp-uniform
    double* Rr = Bc + (int64_t)a * k * k;
    for (int t = lane; t < k * k; t += 32) Rr[t] = 0.0;
    __syncwarp();
    if (k == 3) tentative_regs<3>(m, b, members + s, Trp, B, TV, Rr, lane);
    else tentative_regs<6>(m, b, members + s, Trp, B, TV, Rr, lane);
    return;
  }
  // row t of the aggregate = member (t / b), component (t % b)
  auto tv = [&](int t, int c) -> double& {
    const int node = members[s + t / b];
    return TV[((int64_t)Trp[node] * b + (t % b)) * k + c];
  };
  for (int t = lane; t < m; t += 32) {
    const int node = members[s + t / b];
    for (int c = 0; c < k; c++) tv(t, c) = B[((int64_t)node * b + (t % b)) * k + c];
  }
  __syncwarp();
  double* R = Bc + (int64_t)a * k * k;
  for (int t = lane; t < k * k; t += 32) R[t] = 0.0;
  __syncwarp();
  for (int c = 0; c < k; c++) {
    double n0 = 0.0;
    for (int t = lane; t < m; t += 32) n0 += tv(t, c) * tv(t, c);
    for (int o = 16; o > 0; o >>= 1) n0 += __shfl_xor_sync(0xffffffffu, n0, o);
    n0 = sqrt(n0);
    for (int j = 0; j < c; j++) {
      double d = 0.0;
      for (int t = lane; t < m; t += 32) d += tv(t, j) * tv(t, c);
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (lane == 0) R[j * k + c] = d;
      for (int t = lane; t < m; t += 32) tv(t, c) -= d * tv(t, j);
      __syncwarp();
    }
    double nr = 0.0;
    for (int t = lane; t < m; t += 32) nr += tv(t, c) * tv(t, c);
    for (int o = 16; o > 0; o >>= 1) nr += __shfl_xor_sync(0xffffffffu, nr, o);
    nr = sqrt(nr);
    const bool live = n0 > 0.0 && nr > 1e-8 * n0;
    for (int t = lane; t < m; t += 32) tv(t, c) = live ? tv(t, c) / nr : 0.0;
    if (lane == 0) R[c * k + c] = live ? nr : 0.0;
    __syncwarp();
  }
}

__global__ void k_power_init(int64_t n, int level, double* v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t h = splitmix64((uint64_t)i + SALT_POWER + (uint64_t)level);
  v[i] = (double)(h >> 11) * 0x1.0p-53 - 0.5;
}
// w = scale * Dinv (A v), with `scale` read from the device (1/||v|| of the previous step) so
// the iteration runs without host round trips; 8 lanes per block row; partial sums of w.w
template <int B>
__global__ void __launch_bounds__(256) k_power_step(int nbr, const int* __restrict__ rp,
                                                    const int* __restrict__ ci,
                                                    const double* __restrict__ V,
                                                    const double* __restrict__ Dinv,
                                                    const double* __restrict__ v,
                                                    const double* __restrict__ scale, double* w,
                                                    double* partials, double* out,
                                                    unsigned* ticket) {
  constexpr int G = 8;
  __shared__ double sred[32];
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gtid / G, sub = gtid % G;
  double acc[B];
#pragma unroll
  for (int r = 0; r < B; r++) acc[r] = 0.0;
  if (i < nbr) {
    for (int p = rp[i] + sub; p < rp[i + 1]; p += G) {
      const int j = ci[p];
      const double* blk = V + (int64_t)p * B * B;
#pragma unroll
      for (int r = 0; r < B; r++)
#pragma unroll
        for (int c = 0; c < B; c++) acc[r] += blk[r * B + c] * v[(int64_t)B * j + c];
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < B; r++) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  double ss = 0.0;
  if (i < nbr && sub == 0) {
    const double sc = *scale;
    const double* D = Dinv + (int64_t)B * B * i;
#pragma unroll
    for (int r = 0; r < B; r++) {
      double t = 0.0;
#pragma unroll
      for (int c = 0; c < B; c++) t += D[r * B + c] * acc[c];
      t *= sc;
      w[(int64_t)B * i + r] = t;
      ss += t * t;
    }
  }
  const double tot = block_sum(ss, sred);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  // the last block forms ||w|| and 1 / ||w|| for the next step (fixed summation order)
  if (last_block(ticket, gridDim.x * gridDim.y * gridDim.z)) {
    double a = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) a += __ldcg(partials + q);
    a = block_sum(a, sred);
    if (threadIdx.x == 0) {
      const double nrm = sqrt(a);
      out[0] = nrm;
      out[1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    }
  }
}
// out[0] = sqrt(sum of partials), out[1] = 1 / out[0] (fixed summation order)
__global__ void k_norm_finish(const double* __restrict__ partials, int np, double* out) {
  __shared__ double sred[32];
  double a = 0.0;
  for (int q = threadIdx.x; q < np; q += blockDim.x) a += partials[q];
  a = block_sum(a, sred);
  if (threadIdx.x == 0) {
    const double nrm = sqrt(a);
    out[0] = nrm;
    out[1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
  }
}
__global__ void k_sumsq_partials(int64_t n, const double* __restrict__ v, double* partials) {
  __shared__ double sred[32];
  double ss = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    ss += v[i] * v[i];
  const double tot = block_sum(ss, sred);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// P = T - omega D^-1 (A T), row block i of P by one warp: the lanes take the scalars of the
// row's blocks in turn (block p, row r, column c), each the same b-term sum as a serial loop
__global__ void k_smooth_P(int nbr, int b, int k, const int* __restrict__ rp,
                           const int* __restrict__ ci, const double* __restrict__ ATV,
                           const int* __restrict__ agg, const int* __restrict__ Trp,
                           const double* __restrict__ TV, const double* __restrict__ Dinv,
                           double omega, double* PV) {
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= nbr) return;
  const double* D = Dinv + (int64_t)b * b * i;
  const int p0 = rp[i], bk = b * k;
  const int items = (rp[i + 1] - p0) * bk;
  const int ai = agg[i];
  for (int it = lane; it < items; it += 32) {
    const int p = p0 + it / bk, rc = it % bk, r = rc / k, c = rc % k;
    const double* X = ATV + (int64_t)p * bk;
    double t = 0.0;
    for (int q = 0; q < b; q++) t += D[r * b + q] * X[q * k + c];
    const bool own = ai >= 0 && ci[p] == ai;
    PV[(int64_t)p * bk + rc] = (own ? TV[(int64_t)Trp[i] * bk + rc] : 0.0) - omega * t;
  }
}

__global__ void k_fix_zero_rows(int nbr, int b, const int* __restrict__ rp,
                                const int* __restrict__ ci, double* V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  for (int r = 0; r < b; r++) {
    bool zero = true;
    for (int p = rp[i]; p < rp[i + 1] && zero; p++)
      for (int c = 0; c < b; c++)
        if (V[((int64_t)p * b + r) * b + c] != 0.0) { zero = false; break; }
    if (!zero) continue;
    for (int p = rp[i]; p < rp[i + 1]; p++)
      if (ci[p] == i) V[((int64_t)p * b + r) * b + r] = 1.0;
  }
}

__global__ void k_rbm(int dim, int nx, int ny, int nz, const double* __restrict__ xs,
                      const double* __restrict__ ys, const double* __restrict__ zs, double* B) {
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (dim == 3 ? nz + 1 : 1);
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  int i, j, k;
  node_ijk(node, nx, ny, dim, i, j, k);
  const double x = xs[i], y = ys[j];
  if (dim == 2) {
    double* r0 = B + (2 * node) * 3;
    double* r1 = r0 + 3;
    r0[0] = 1.0; r0[1] = 0.0; r0[2] = -y;
    r1[0] = 0.0; r1[1] = 1.0; r1[2] = x;
  } else {
    const double z = zs[k];
    double* r0 = B + (3 * node) * 6;
    double* r1 = r0 + 6;
    double* r2 = r1 + 6;
    // [tx, ty, tz, rot_x (0,-z,y), rot_y (z,0,-x), rot_z (-y,x,0)]
    r0[0] = 1; r0[1] = 0; r0[2] = 0; r0[3] = 0.0; r0[4] = z;    r0[5] = -y;
    r1[0] = 0; r1[1] = 1; r1[2] = 0; r1[3] = -z;  r1[4] = 0.0;  r1[5] = x;
    r2[0] = 0; r2[1] = 0; r2[2] = 1; r2[3] = y;   r2[4] = -x;   r2[5] = 0.0;
  }
}

}  // namespace

void amg_strength_counts(cudaStream_t s, const Bsr& A, const double* V, double beta, int* counts) {
  DBuf<double> dn;
  dn.resize(A.nbr);
  LAUNCH(k_diag_fro, ceil_div(A.nbr, 256), 256, 0, s, A.nbr, A.br, A.rp, A.ci, V, dn.p);
  LAUNCH(k_strength, ceil_div((int64_t)A.nbr * 32, 256), 256, 0, s, A.nbr, A.br, A.rp, A.ci, V, dn.p, beta,
         counts, (const int*)nullptr, (int*)nullptr);
  CK(cudaStreamSynchronize(s));
}

void amg_strength_fill(cudaStream_t s, const Bsr& A, const double* V, double beta, const int* srp,
                       int* sci) {
  DBuf<double> dn;
  dn.resize(A.nbr);
  LAUNCH(k_diag_fro, ceil_div(A.nbr, 256), 256, 0, s, A.nbr, A.br, A.rp, A.ci, V, dn.p);
  LAUNCH(k_strength, ceil_div((int64_t)A.nbr * 32, 256), 256, 0, s, A.nbr, A.br, A.rp, A.ci, V, dn.p, beta,
         (int*)nullptr, srp, sci);
  CK(cudaStreamSynchronize(s));
}

void set_grid_wait_limit(int polls) { g_grid_wait_polls = polls; }
unsigned grid_wait_limit(unsigned dflt) {  // polls = 1: the kernels' limit 0, give up at once
  return g_grid_wait_polls > 0 ? (unsigned)(g_grid_wait_polls - 1) : dflt;
}

int amg_mis2(cudaStream_t s, int n, const int* srp, const int* sci, int level, int* state,
             uint64_t* v, uint64_t* m1, int* flag_host, int* flag_dev) {
  (void)flag_dev;
  if (n == 0) return 0;
  // one cooperative launch, every block resident (grid-stride loops over the nodes)
  static int per_sm = 0;
  if (per_sm == 0)
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mis2_loop, 256, 0));
  const int grid = std::max(1, std::min(ceil_div(n, 256), per_sm * num_sms()));
  constexpr int MAX_ROUNDS = 100000;
  DBuf<unsigned> sync;
  sync.resize(6);
  sync.zero(s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  CK(cudaLaunchKernelEx(&cfg, k_mis2_loop, n, level, srp, sci, state, v, m1, sync.p,
                        MAX_ROUNDS, grid_wait_limit(MIS_WAIT_LIMIT)));
  g_launches++;
  unsigned h[6];
  CK(cudaMemcpyAsync(h, sync.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  (void)flag_host;
  if (h[4]) TOMG_THROW(TOMG_E_TIMEOUT, "MIS-2 grid barrier wait ran out");
  if ((int)h[5] >= MAX_ROUNDS) TOMG_THROW(TOMG_E_BREAKDOWN, "MIS-2 did not terminate");
  return (int)h[5];
}

int amg_aggregate(cudaStream_t s, int n, const int* srp, const int* sci, int level,
                  const int* state, int* agg, int* root_scan) {
  DBuf<int> flags, agg1, fail;
  flags.resize(n);
  agg1.resize(n);
  fail.resize(1);
  fail.zero(s);
  const int g = ceil_div(n, 256);
  LAUNCH(k_root_flags, g, 256, 0, s, n, state, flags.p);
  const int n_agg = (int)exclusive_scan(s, flags.p, root_scan, n);
  LAUNCH(k_agg_phase1, g, 256, 0, s, n, srp, sci, state, root_scan, agg1.p);
  LAUNCH(k_agg_phase2, g, 256, 0, s, n, level, srp, sci, agg1.p, agg, fail.p);
  int nf = 0;
  CK(cudaMemcpyAsync(&nf, fail.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (nf) TOMG_THROW(TOMG_E_BREAKDOWN, "%d nodes left unaggregated", nf);
  return n_agg;
}

int64_t amg_tentative(cudaStream_t s, int n, int b, int k, int n_agg, const int* agg,
                      const double* B, int* Trp, int* Tci, double* TV, double* Bc) {
  const int g = ceil_div(n, 256);
  DBuf<int> flags, cnt, start, cursor, members;
  flags.resize(n);
  LAUNCH(k_T_pattern, g, 256, 0, s, n, agg, flags.p);
  const int64_t nT = exclusive_scan(s, flags.p, Trp, n);
  LAUNCH(k_T_cols, g, 256, 0, s, n, agg, Tci, Trp);
  cnt.resize(n_agg + 1);
  start.resize(n_agg + 1);
  cursor.resize(n_agg + 1);
  members.resize(nT > 0 ? nT : 1);
  cnt.zero(s);
  cursor.zero(s);
  LAUNCH(k_agg_count, g, 256, 0, s, n, agg, cnt.p);
  exclusive_scan_nosync(s, cnt.p, start.p, n_agg);
  DBuf<int> unsorted;
  unsorted.resize(nT > 0 ? nT : 1);
  LAUNCH(k_agg_scatter, g, 256, 0, s, n, agg, start.p, cursor.p, unsorted.p);
  LAUNCH(k_agg_sort, ceil_div((int64_t)n_agg * 32, 128), 128, 0, s, n_agg, start.p, unsorted.p,
         members.p);
  LAUNCH(k_tentative, ceil_div((int64_t)n_agg * 32, 128), 128, 0, s, n_agg, b, k, start.p,
         members.p, Trp, B, TV, Bc);
  return nT;
}

void amg_power_alloc(cudaStream_t s, AmgPower& ps, const Bsr& A, int iters) {
  const int64_t n = (int64_t)A.nbr * A.br;
  const int gb = ceil_div((int64_t)A.nbr * 8, 256);
  ps.iters = iters;
  ps.v.resize(n);
  ps.w.resize(n);
  ps.parts.resize(std::max(gb, 256));
  ps.nrm.resize(2 * (iters + 1));
  ps.ticket.resize(1);
  ps.ticket.zero(s);
}

void amg_power_enqueue(cudaStream_t s, AmgPower& ps, const Bsr& A, const double* V,
                       const double* Dinv, int level) {
  // u_0 = splitmix64 vector; step: w = (1/||u_it||) D^-1 A u_it, rho_it = ||w||, u_{it+1} = w.
  // Norms and their reciprocals stay on the device; the host reads the last rho only.
  const int64_t n = (int64_t)A.nbr * A.br;
  const int gb = ceil_div((int64_t)A.nbr * 8, 256);
  const int gp = 256;
  double* v = ps.v.p;
  double* w = ps.w.p;
  LAUNCH(k_power_init, ceil_div(n, 256), 256, 0, s, n, level, v);
  LAUNCH(k_sumsq_partials, gp, 256, 0, s, n, v, ps.parts.p);
  LAUNCH(k_norm_finish, 1, 256, 0, s, ps.parts.p, gp, ps.nrm.p);
  for (int it = 0; it < ps.iters; it++) {
    const double* sc = ps.nrm.p + 2 * it + 1;
    double* o = ps.nrm.p + 2 * (it + 1);
    if (A.br == 2) LAUNCH(k_power_step<2>, gb, 256, 0, s, A.nbr, A.rp, A.ci, V, Dinv, v, sc, w, ps.parts.p, o, ps.ticket.p);
    else if (A.br == 3) LAUNCH(k_power_step<3>, gb, 256, 0, s, A.nbr, A.rp, A.ci, V, Dinv, v, sc, w, ps.parts.p, o, ps.ticket.p);
    else if (A.br == 6) LAUNCH(k_power_step<6>, gb, 256, 0, s, A.nbr, A.rp, A.ci, V, Dinv, v, sc, w, ps.parts.p, o, ps.ticket.p);
    else TOMG_THROW(TOMG_E_INVALID, "unsupported block %d", A.br);
    std::swap(v, w);
  }
}

double amg_power_result(cudaStream_t s, const AmgPower& ps) {
  double rho = 0.0;
  CK(cudaMemcpyAsync(&rho, ps.nrm.p + 2 * ps.iters, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (!(rho > 0.0)) TOMG_THROW(TOMG_E_BREAKDOWN, "power iteration collapsed");
  return rho;
}

// w = scale * Dinv t (B x B blocks), scale read from the device
template <int B>
__global__ void k_dinv_scale(int64_t nodes, const double* __restrict__ Dinv,
                             const double* __restrict__ t, const double* __restrict__ scale,
                             double* __restrict__ w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nodes) return;
  const double sc = *scale;
  const double* D = Dinv + (int64_t)B * B * i;
#pragma unroll
  for (int q = 0; q < B; q++) {
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < B; c++) v += D[q * B + c] * t[B * i + c];
    w[B * i + q] = sc * v;
  }
}

// FP32 step of the power iteration on a geometric level: w = scale Dinv32 t (B x B blocks),
// scale = 1/||u|| of the previous step read from the device, and ||w|| with 1/||w|| formed by
// the last block (per-thread sums of squares in FP32, combined in FP64 in a fixed order)
template <int B>
__global__ void __launch_bounds__(256) k_dinv_scale32(int64_t nodes, const float* __restrict__ Dinv,
                                                      const float* __restrict__ t,
                                                      const double* __restrict__ scale,
                                                      float* __restrict__ w, double* partials,
                                                      double* out, unsigned* ticket) {
  __shared__ double sred[32];
  const float sc = (float)*scale;
  float ss = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nodes;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float* D = Dinv + (int64_t)B * B * i;
    float tv[B];
#pragma unroll
    for (int c = 0; c < B; c++) tv[c] = t[B * i + c];
#pragma unroll
    for (int q = 0; q < B; q++) {
      float v = 0.f;
#pragma unroll
      for (int c = 0; c < B; c++) v = fmaf(D[q * B + c], tv[c], v);
      const float wv = sc * v;
      w[B * i + q] = wv;
      ss = fmaf(wv, wv, ss);
    }
  }
  const double tot = block_sum((double)ss, sred);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  if (last_block(ticket, gridDim.x)) {
    double a = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) a += __ldcg(partials + q);
    a = block_sum(a, sred);
    if (threadIdx.x == 0) {
      const double nrm = sqrt(a);
      out[0] = nrm;
      out[1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    }
  }
}

void splitmix_uniform(cudaStream_t s, int64_t n, int level, double* v) {
  LAUNCH(k_power_init, ceil_div(n, 256), 256, 0, s, n, level, v);
}

constexpr int PW32_BLOCKS = 1216;  // one full wave of 256-thread blocks on the 152-SM GB300

void power_alloc(PowerState& ps, int64_t nodes, int bs, int iters, bool f32) {
  const int64_t n = nodes * bs;
  ps.nodes = nodes;
  ps.bs = bs;
  ps.iters = iters;
  ps.v.resize(n);
  if (f32) {
    ps.v32.resize(n);
    ps.w32.resize(n);
    ps.t32.resize(n);
    ps.ticket.resize(1);
    ps.ticket.zero(alloc_stream());
  } else {
    ps.w.resize(n);
    ps.t.resize(n);
  }
  ps.parts.resize(std::max(256, PW32_BLOCKS));
  ps.nrm.resize(2 * (iters + 1));
}

void power_enqueue_f32(cudaStream_t s, PowerState& ps, const float* Dinv32, int level,
                       const std::function<void(const float*, float*)>& apply) {
  // u_0 = the FP64 path's splitmix64 vector rounded to FP32; w = (1/||u_it||) D^-1 A u_it,
  // rho_it = ||w||, u_{it+1} = w, all vectors in FP32
  const int64_t nodes = ps.nodes, n = nodes * ps.bs;
  const int gp = 256;
  LAUNCH(k_power_init, ceil_div(n, 256), 256, 0, s, n, level, ps.v.p);
  LAUNCH(k_sumsq_partials, gp, 256, 0, s, n, ps.v.p, ps.parts.p);
  LAUNCH(k_norm_finish, 1, 256, 0, s, ps.parts.p, gp, ps.nrm.p);
  cast_f64_f32(s, ps.v.p, ps.v32.p, n);
  float* a = ps.v32.p;
  float* c = ps.w32.p;
  const int g = std::max(1, std::min(PW32_BLOCKS, ceil_div(nodes, 256)));
  for (int it = 0; it < ps.iters; it++) {
    apply(a, ps.t32.p);
    const double* sc = ps.nrm.p + 2 * it + 1;
    double* o = ps.nrm.p + 2 * (it + 1);
    if (ps.bs == 2) LAUNCH(k_dinv_scale32<2>, g, 256, 0, s, nodes, Dinv32, ps.t32.p, sc, c, ps.parts.p, o, ps.ticket.p);
    else if (ps.bs == 3) LAUNCH(k_dinv_scale32<3>, g, 256, 0, s, nodes, Dinv32, ps.t32.p, sc, c, ps.parts.p, o, ps.ticket.p);
    else if (ps.bs == 6) LAUNCH(k_dinv_scale32<6>, g, 256, 0, s, nodes, Dinv32, ps.t32.p, sc, c, ps.parts.p, o, ps.ticket.p);
    else TOMG_THROW(TOMG_E_INVALID, "unsupported block %d", ps.bs);
    std::swap(a, c);
  }
}

void power_enqueue(cudaStream_t s, PowerState& ps, const double* Dinv, int level,
                   const std::function<void(const double*, double*)>& apply) {
  // the same iteration as amg_spectral_radius, with the operator applied by the caller:
  // u_0 = splitmix64 vector; w = (1/||u_it||) D^-1 A u_it, rho_it = ||w||, u_{it+1} = w
  const int64_t nodes = ps.nodes, n = nodes * ps.bs;
  const int gp = 256;
  LAUNCH(k_power_init, ceil_div(n, 256), 256, 0, s, n, level, ps.v.p);
  LAUNCH(k_sumsq_partials, gp, 256, 0, s, n, ps.v.p, ps.parts.p);
  LAUNCH(k_norm_finish, 1, 256, 0, s, ps.parts.p, gp, ps.nrm.p);
  double* a = ps.v.p;
  double* c = ps.w.p;
  for (int it = 0; it < ps.iters; it++) {
    apply(a, ps.t.p);
    const double* sc = ps.nrm.p + 2 * it + 1;
    const int g = ceil_div(nodes, 256);
    if (ps.bs == 2) LAUNCH(k_dinv_scale<2>, g, 256, 0, s, nodes, Dinv, ps.t.p, sc, c);
    else if (ps.bs == 3) LAUNCH(k_dinv_scale<3>, g, 256, 0, s, nodes, Dinv, ps.t.p, sc, c);
    else if (ps.bs == 6) LAUNCH(k_dinv_scale<6>, g, 256, 0, s, nodes, Dinv, ps.t.p, sc, c);
    else TOMG_THROW(TOMG_E_INVALID, "unsupported block %d", ps.bs);
    LAUNCH(k_sumsq_partials, gp, 256, 0, s, n, c, ps.parts.p);
    LAUNCH(k_norm_finish, 1, 256, 0, s, ps.parts.p, gp, ps.nrm.p + 2 * (it + 1));
    std::swap(a, c);
  }
}

double power_result(cudaStream_t s, const PowerState& ps) {
  double rho = 0.0;
  CK(cudaMemcpyAsync(&rho, ps.nrm.p + 2 * ps.iters, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (!(rho > 0.0)) TOMG_THROW(TOMG_E_BREAKDOWN, "power iteration collapsed");
  return rho;
}

double spectral_radius_op(cudaStream_t s, int64_t nodes, int bs, const double* Dinv, int level,
                          int iters, const std::function<void(const double*, double*)>& apply) {
  PowerState ps;
  power_alloc(ps, nodes, bs, iters);
  power_enqueue(s, ps, Dinv, level, apply);
  return power_result(s, ps);
}

void amg_smooth_prolongator(cudaStream_t s, const Bsr& AT, const double* ATV, const int* agg,
                            const double* TV, const int* Trp, const double* Dinv, double omega,
                            int b, double* PV) {
  LAUNCH(k_smooth_P, ceil_div((int64_t)AT.nbr * 32, 128), 128, 0, s, AT.nbr, b, AT.bc, AT.rp,
         AT.ci, ATV, agg, Trp, TV, Dinv, omega, PV);
}

void amg_fix_zero_rows(cudaStream_t s, const Bsr& A, double* V) {
  LAUNCH(k_fix_zero_rows, ceil_div(A.nbr, 128), 128, 0, s, A.nbr, A.br, A.rp, A.ci, V);
}

void rigid_body_modes(cudaStream_t s, const Geo& g, const double* xs, const double* ys,
                      const double* zs, double* B) {
  LAUNCH(k_rbm, ceil_div(g.nodes(), 256), 256, 0, s, g.dim, g.nx, g.ny, g.nz, xs, ys, zs, B);
}

}  // namespace tomg
