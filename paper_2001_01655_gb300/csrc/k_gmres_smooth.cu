// GMRES smoother.  Sec. 4.1 studies SOR-preconditioned GMRES iterations as the multigrid
// smoother (under flexible GMRES); here the preconditioner is the point-block diagonal, as for
// the Chebyshev smoother.  m steps of right-preconditioned GMRES (Saad, Iterative Methods for
// Sparse Linear Systems, 2nd ed., Alg. 9.5) for A x = b from x_0:
//   r_0 = b - A x_0, beta = ||r_0||, v_0 = r_0 / beta;
//   step j: z_j = D^-1 v_j, w = A z_j, projections on v_0..v_j by classical Gram-Schmidt
//           applied twice, h_{j+1,j} = ||w''||, v_{j+1} = w'' / h_{j+1,j};
//   y = argmin ||beta e_1 - Hbar y|| by Givens rotations, x = x_0 + sum_j y_j z_j.
// Every scalar stays in device memory, so a smoothing is part of the captured solve graph.
// Vectors are in the level's precision T; every reduction is FP64 with a fixed summation
// order (per-block partials added in block order by the last block to finish).  The second
// Gram-Schmidt pass takes the norm from its own input, ||w''||^2 = ||w'||^2 - ||h''||^2 (h'' the
// second pass's projections, which are of the order of the first pass's rounding), and the
// subtraction of V h'' is folded into the next step's scaling kernel.  An exact breakdown
// (beta = 0 or h_{j+1,j} = 0) ends the steps: the least-squares problem keeps the columns
// before it, and the later vectors are zero.
#include "finish.cuh"
#include "ops.h"

namespace tomg {

namespace {

constexpr int GM_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(GM_THREADS) k_gm_start(int64_t n, const T* __restrict__ src,
                                                         double* parts, GmState* st, int m,
                                                         const int* done) {
  __shared__ double sred[32];
  pdl_launch();
  pdl_wait();
  if (solve_done(done)) return;
  double a = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)src[i];
    a += v * v;
  }
  a = block_sum(a, sred);
  if (threadIdx.x == 0) parts[blockIdx.x] = a;
  if (last_block(&st->tk, gridDim.x * gridDim.y * gridDim.z)) {
    double t = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) t += __ldcg(parts + q);
    t = block_sum(t, sred);
    if (threadIdx.x == 0) {
      const double beta = sqrt(t);
      st->beta = beta;
      st->inv = beta > 0.0 ? 1.0 / beta : 0.0;
      st->meff = beta > 0.0 ? m : 0;
    }
  }
}

// v_j = (src - sum_{k<j} h''_k v_k) * inv (in place when src is v_j's slot), z_j = D^-1 v_j
template <class T, int B>
__global__ void __launch_bounds__(GM_THREADS) k_gm_next(int64_t nodes, int j,
                                                        const T* __restrict__ src, T* V,
                                                        int64_t ldv, T* __restrict__ Z,
                                                        const T* __restrict__ Dinv,
                                                        const GmState* __restrict__ st,
                                                        const int* done) {
  pdl_launch();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T D[B * B];
  if (i < nodes) {
#pragma unroll
    for (int t = 0; t < B * B; t++) D[t] = Dinv[(int64_t)B * B * i + t];
  }
  pdl_wait();
  if (solve_done(done) || i >= nodes) return;
  const double inv = st->inv;
  T v[B];
#pragma unroll
  for (int c = 0; c < B; c++) {
    const int64_t idx = (int64_t)B * i + c;
    double a = (double)src[idx];
    for (int k = 0; k < j; k++) a -= st->h2[k] * (double)V[(int64_t)k * ldv + idx];
    v[c] = (T)(a * inv);
    V[(int64_t)j * ldv + idx] = v[c];
  }
#pragma unroll
  for (int r = 0; r < B; r++) {
    T a = T(0);
#pragma unroll
    for (int c = 0; c < B; c++) a += D[r * B + c] * v[c];
    Z[(int64_t)j * ldv + (int64_t)B * i + r] = a;
  }
}

// h'_k = v_k . w for k <= j (w in slot j + 1)
template <class T>
__global__ void __launch_bounds__(GM_THREADS) k_gm_dots(int64_t n, int j, const T* __restrict__ V,
                                                        int64_t ldv, double* parts, GmState* st,
                                                        const int* done) {
  __shared__ double sred[32];
  pdl_launch();
  pdl_wait();
  if (solve_done(done)) return;
  const T* w = V + (int64_t)(j + 1) * ldv;
  double acc[GM_MAX];
#pragma unroll
  for (int k = 0; k < GM_MAX; k++) acc[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double wv = (double)w[i];
#pragma unroll
    for (int k = 0; k < GM_MAX; k++)
      if (k <= j) acc[k] += (double)V[(int64_t)k * ldv + i] * wv;
  }
  const int nb = gridDim.x;
  for (int k = 0; k <= j; k++) {
    const double a = block_sum(acc[k], sred);
    if (threadIdx.x == 0) parts[(int64_t)k * nb + blockIdx.x] = a;
  }
  if (last_block(&st->tk, gridDim.x * gridDim.y * gridDim.z)) {
    for (int k = 0; k <= j; k++) {
      double t = 0.0;
      for (int q = threadIdx.x; q < nb; q += blockDim.x) t += __ldcg(parts + (int64_t)k * nb + q);
      t = block_sum(t, sred);
      if (threadIdx.x == 0) st->h1[k] = t;
    }
  }
}

// Hbar (m + 1 rows, meff columns) -> y by Givens rotations and back substitution (one thread)
__device__ void gm_least_squares(GmState* st, int m) {
  const int k = st->meff;
  double R[(GM_MAX + 1) * GM_MAX], g[GM_MAX + 1], cs[GM_MAX], sn[GM_MAX];
  for (int q = 0; q < (GM_MAX + 1) * GM_MAX; q++) R[q] = st->H[q];
  for (int q = 0; q <= GM_MAX; q++) g[q] = 0.0;
  g[0] = st->beta;
  constexpr int LD = GM_MAX + 1;
  for (int c = 0; c < k; c++) {
    for (int i = 0; i < c; i++) {
      const double a = R[i + LD * c], b = R[i + 1 + LD * c];
      R[i + LD * c] = cs[i] * a + sn[i] * b;
      R[i + 1 + LD * c] = -sn[i] * a + cs[i] * b;
    }
    const double a = R[c + LD * c], b = R[c + 1 + LD * c];
    const double r = sqrt(a * a + b * b);
    cs[c] = r > 0.0 ? a / r : 1.0;
    sn[c] = r > 0.0 ? b / r : 0.0;
    R[c + LD * c] = r;
    R[c + 1 + LD * c] = 0.0;
    g[c + 1] = -sn[c] * g[c];
    g[c] = cs[c] * g[c];
  }
  for (int c = GM_MAX - 1; c >= 0; c--) {
    if (c >= k) {
      if (c < m) st->y[c] = 0.0;
      continue;
    }
    double t = g[c];
    for (int i = c + 1; i < k; i++) t -= R[c + LD * i] * st->y[i];
    st->y[c] = R[c + LD * c] != 0.0 ? t / R[c + LD * c] : 0.0;
  }
}

// w' = w - sum_{k<=j} h'_k v_k (in place), h''_k = v_k . w', ||w'||^2; the last block completes
// column j of Hbar and, after the last step, solves the least-squares problem
template <class T>
__global__ void __launch_bounds__(GM_THREADS) k_gm_orth(int64_t n, int j, int m, T* V, int64_t ldv,
                                                        double* parts, GmState* st,
                                                        const int* done) {
  __shared__ double sred[32];
  __shared__ double sh[GM_MAX];
  pdl_launch();
  pdl_wait();
  if (solve_done(done)) return;
  if (threadIdx.x <= j) sh[threadIdx.x] = st->h1[threadIdx.x];
  __syncthreads();
  T* w = V + (int64_t)(j + 1) * ldv;
  double acc[GM_MAX + 1];
#pragma unroll
  for (int k = 0; k <= GM_MAX; k++) acc[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double vk[GM_MAX];
    double a = (double)w[i];
#pragma unroll
    for (int k = 0; k < GM_MAX; k++)
      if (k <= j) {
        vk[k] = (double)V[(int64_t)k * ldv + i];
        a -= sh[k] * vk[k];
      }
    const T wt = (T)a;
    w[i] = wt;
    const double wd = (double)wt;
#pragma unroll
    for (int k = 0; k < GM_MAX; k++)
      if (k <= j) acc[k] += vk[k] * wd;
    acc[GM_MAX] += wd * wd;
  }
  const int nb = gridDim.x;
  for (int k = 0; k <= j; k++) {
    const double a = block_sum(acc[k], sred);
    if (threadIdx.x == 0) parts[(int64_t)k * nb + blockIdx.x] = a;
  }
  {
    const double a = block_sum(acc[GM_MAX], sred);
    if (threadIdx.x == 0) parts[(int64_t)GM_MAX * nb + blockIdx.x] = a;
  }
  if (last_block(&st->tk, gridDim.x * gridDim.y * gridDim.z)) {
    __shared__ double tot[GM_MAX + 1];
    for (int k = 0; k <= GM_MAX; k++) {
      if (k > j && k < GM_MAX) continue;
      double t = 0.0;
      for (int q = threadIdx.x; q < nb; q += blockDim.x) t += __ldcg(parts + (int64_t)k * nb + q);
      t = block_sum(t, sred);
      if (threadIdx.x == 0) tot[k] = t;
    }
    if (threadIdx.x == 0) {
      double hn2 = tot[GM_MAX];
      for (int k = 0; k <= j; k++) {
        st->h2[k] = tot[k];
        st->H[k + (GM_MAX + 1) * j] = sh[k] + tot[k];
        hn2 -= tot[k] * tot[k];
      }
      const double hn = sqrt(fmax(hn2, 0.0));
      st->H[j + 1 + (GM_MAX + 1) * j] = hn;
      st->inv = hn > 0.0 ? 1.0 / hn : 0.0;
      if (!(hn > 0.0) && st->meff > j + 1) st->meff = j + 1;
      if (j == m - 1) gm_least_squares(st, m);
    }
  }
}

// out = x0 + sum_{k<m} y_k z_k (x0 = nullptr: zero)
template <class T>
__global__ void __launch_bounds__(GM_THREADS) k_gm_update(int64_t n, int m, const T* __restrict__ Z,
                                                          int64_t ldv,
                                                          const GmState* __restrict__ st,
                                                          const T* __restrict__ x0,
                                                          T* __restrict__ out, const int* done) {
  pdl_launch();
  pdl_wait();
  if (solve_done(done)) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = x0 ? (double)x0[i] : 0.0;
  for (int k = 0; k < m; k++) a += st->y[k] * (double)Z[(int64_t)k * ldv + i];
  out[i] = (T)a;
}

int gm_blocks(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(2 * 152, ceil_div(n, 4 * GM_THREADS)));
}

}  // namespace

int gmres_smooth_parts(int64_t n) { return (GM_MAX + 1) * gm_blocks(n); }

template <class T>
void gmres_smooth_begin(cudaStream_t s, int64_t n, const T* r0, double* parts, GmState* st, int m,
                        const int* done) {
  if (m < 1 || m > GM_MAX) TOMG_THROW(TOMG_E_INVALID, "GMRES smoother steps %d outside 1..%d", m, GM_MAX);
  LAUNCH((k_gm_start<T>), gm_blocks(n), GM_THREADS, 0, s, n, r0, parts, st, m, done);
}

template <class T>
void gmres_smooth_next(cudaStream_t s, int bs, int64_t nodes, int j, const T* src, T* V,
                       int64_t ldv, T* Z, const T* Dinv, const GmState* st, const int* done) {
  const int g = (int)ceil_div(nodes, GM_THREADS);
  if (bs == 2) LAUNCH((k_gm_next<T, 2>), g, GM_THREADS, 0, s, nodes, j, src, V, ldv, Z, Dinv, st, done);
  else if (bs == 3) LAUNCH((k_gm_next<T, 3>), g, GM_THREADS, 0, s, nodes, j, src, V, ldv, Z, Dinv, st, done);
  else if (bs == 6) LAUNCH((k_gm_next<T, 6>), g, GM_THREADS, 0, s, nodes, j, src, V, ldv, Z, Dinv, st, done);
  else TOMG_THROW(TOMG_E_INVALID, "unsupported block size %d", bs);
}

template <class T>
void gmres_smooth_orth(cudaStream_t s, int64_t n, int j, int m, T* V, int64_t ldv, double* parts,
                       GmState* st, const int* done) {
  const int nb = gm_blocks(n);
  LAUNCH((k_gm_dots<T>), nb, GM_THREADS, 0, s, n, j, V, ldv, parts, st, done);
  LAUNCH((k_gm_orth<T>), nb, GM_THREADS, 0, s, n, j, m, V, ldv, parts, st, done);
}

template <class T>
void gmres_smooth_finish(cudaStream_t s, int64_t n, int m, const T* Z, int64_t ldv,
                         const GmState* st, const T* x0, T* out, const int* done) {
  LAUNCH((k_gm_update<T>), ceil_div(n, GM_THREADS), GM_THREADS, 0, s, n, m, Z, ldv, st, x0, out,
         done);
}

#define GM_INST(T)                                                                              \
  template void gmres_smooth_begin<T>(cudaStream_t, int64_t, const T*, double*, GmState*, int,  \
                                      const int*);                                              \
  template void gmres_smooth_next<T>(cudaStream_t, int, int64_t, int, const T*, T*, int64_t, T*, \
                                     const T*, const GmState*, const int*);                     \
  template void gmres_smooth_orth<T>(cudaStream_t, int64_t, int, int, T*, int64_t, double*,     \
                                     GmState*, const int*);                                     \
  template void gmres_smooth_finish<T>(cudaStream_t, int64_t, int, const T*, int64_t,           \
                                       const GmState*, const T*, T*, const int*);
GM_INST(float)
GM_INST(double)

}  // namespace tomg
