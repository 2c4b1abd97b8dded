// Outer Krylov loop kernels (Sec. 3.1 CG; flexible CG after Notay 2000 for the FP32 V-cycle),
// deterministic FP64 reductions, precision casts, the first Jacobi sweep from x = 0 and the
// coarsest-level direct solve (Sec. 3.2: dense Cholesky factorisation at setup, explicit
// inverse applied as a GEMV in every V-cycle).
//
// Reductions: every kernel that produces a dot product writes one FP64 partial per block
// (fixed tree inside the block); a single-block "finish" kernel adds the partials in a fixed
// order and updates the device-resident scalar state, so no host round trip is needed per
// iteration and results do not depend on scheduling.
#include "finish.cuh"

namespace tomg {

namespace {

constexpr int RED_THREADS = 256;
// one full wave (8 resident blocks of 256 threads per SM on the 152-SM GB300): twice the
// elements per thread of two waves, so the block reductions take half the FP64 share
constexpr int RED_MAX_BLOCKS = 1216;

// Vector kernels walk the DOFs in pairs (16-byte loads of FP64 vectors), one pair per thread
// when the grid allows it, so every load of a thread is issued at once; an odd last DOF is
// handled by the thread of pair index n / 2.  Each thread's share of a dot product is one chain
// of FMAs in DOF order, written out so that the rounding does not depend on how the compiler
// contracts a sum of two products (and two FP64 instructions per pair instead of three).
template <class T> struct P2;
template <> struct P2<double> { using type = double2; };
template <> struct P2<float> { using type = float2; };
template <class T>
__device__ __forceinline__ typename P2<T>::type ld2(const T* a, int64_t k, int64_t n) {
  if (2 * k + 1 < n) return reinterpret_cast<const typename P2<T>::type*>(a)[k];
  typename P2<T>::type v;
  v.x = a[2 * k];
  v.y = T(0);
  return v;
}

__global__ void __launch_bounds__(RED_THREADS) k_dot(const double* __restrict__ x,
                                                     const double* __restrict__ y, int64_t n,
                                                     double* partials, const int* done) {
  __shared__ double sred[32];
  pdl_prologue();
  if (solve_done(done)) return;
  x += (int64_t)blockIdx.y * rhs_stride(n);  // right-hand side blockIdx.y of a block solve
  y += (int64_t)blockIdx.y * rhs_stride(n);
  partials += (int64_t)blockIdx.y * gridDim.x;
  double s = 0.0;
  const int64_t np = (n + 1) / 2;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = ld2(x, k, n), b = ld2(y, k, n);
    s = fma(a.y, b.y, fma(a.x, b.x, s));
  }
  s = block_sum(s, sred);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_finish(int kind, const double* __restrict__ pa, int na,
                                                 const double* __restrict__ pb, int nb,
                                                 Scalars* sc) {
  __shared__ double sred[32];
  pdl_prologue();
  sc += blockIdx.x;  // right-hand side blockIdx.x of a block solve
  pa += (int64_t)blockIdx.x * na;
  if (pb) pb += (int64_t)blockIdx.x * nb;
  if (kind != FIN_INIT && sc->done) return;
  finish_body(kind, pa, na, pb, nb, sc, sred);
}

__global__ void __launch_bounds__(RED_THREADS) k_xr(double* __restrict__ x, double* __restrict__ r,
                                                    const double* __restrict__ p,
                                                    const double* __restrict__ q, int64_t n,
                                                    Scalars* sc, double* partials,
                                                    float* __restrict__ r32) {
  __shared__ double sred[32];
  pdl_prologue();
  {  // right-hand side blockIdx.y of a block solve: its vectors, partials and scalar state
    const int64_t vo = (int64_t)blockIdx.y * rhs_stride(n);
    x += vo;
    r += vo;
    p += vo;
    q += vo;
    if (r32) r32 += vo;
    partials += (int64_t)blockIdx.y * gridDim.x;
    sc += blockIdx.y;
  }
  if (sc->done) return;
  const double alpha = sc->alpha;
  double s = 0.0;
  const int64_t np = (n + 1) / 2;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 xv = ld2(x, k, n), pv = ld2(p, k, n), rv = ld2(r, k, n), qv = ld2(q, k, n);
    const double x0 = xv.x + alpha * pv.x, x1 = xv.y + alpha * pv.y;
    const double r0 = rv.x - alpha * qv.x, r1 = rv.y - alpha * qv.y;
    if (2 * k + 1 < n) {
      reinterpret_cast<double2*>(x)[k] = make_double2(x0, x1);
      reinterpret_cast<double2*>(r)[k] = make_double2(r0, r1);
      if (r32) reinterpret_cast<float2*>(r32)[k] = make_float2(d2f_bits(r0), d2f_bits(r1));
      s = fma(r1, r1, fma(r0, r0, s));
    } else {
      x[2 * k] = x0;
      r[2 * k] = r0;
      if (r32) r32[2 * k] = d2f_bits(r0);
      s = fma(r0, r0, s);
    }
  }
  s = block_sum(s, sred);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
  if (last_block(&sc->tk[TK_RR], gridDim.x))
    finish_body(FIN_RR, partials, gridDim.x, nullptr, 0, sc, sred);
}

// p = z + beta p.  The last kernel of an iteration: with has_cond it also sets the while
// condition of the captured loop from the done flag (before any early exit, so the loop ends
// on every path that sets done).
__global__ void k_p(double* __restrict__ p, const double* __restrict__ z, int64_t n,
                    const Scalars* sc, cudaGraphConditionalHandle cond, int has_cond) {
  pdl_prologue();
  p += (int64_t)blockIdx.y * rhs_stride(n);  // right-hand side blockIdx.y of a block solve
  z += (int64_t)blockIdx.y * rhs_stride(n);
  sc += blockIdx.y;
  const int done = *(volatile const int*)&sc->done;
  if (has_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, done ? 0u : 1u);
  if (done) return;
  const double beta = sc->beta;
  const int64_t np = (n + 1) / 2;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 zv = ld2(z, k, n), pv = ld2(p, k, n);
    if (2 * k + 1 < n) reinterpret_cast<double2*>(p)[k] = make_double2(zv.x + beta * pv.x, zv.y + beta * pv.y);
    else p[2 * k] = zv.x + beta * pv.x;
  }
}

__device__ __forceinline__ double to_f64(float v) { return f2d_bits(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }

template <class T>
__global__ void __launch_bounds__(RED_THREADS) k_zdots(const T* __restrict__ z, double* z64,
                                                       const double* __restrict__ r,
                                                       const double* __restrict__ q, int64_t n,
                                                       double* pa, double* pb, Scalars* sc,
                                                       int kind) {
  __shared__ double sred[32];
  pdl_prologue();
  const bool copy = (const void*)z != (const void*)z64;
  {  // right-hand side blockIdx.y of a block solve
    const int64_t vo = (int64_t)blockIdx.y * rhs_stride(n);
    z += vo;
    z64 += vo;
    r += vo;
    if (q) q += vo;
    pa += (int64_t)blockIdx.y * gridDim.x;
    if (q) pb += (int64_t)blockIdx.y * gridDim.x;
    sc += blockIdx.y;
  }
  if (sc->done) return;
  double a = 0.0, b = 0.0;
  const int64_t np = (n + 1) / 2;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += (int64_t)gridDim.x * blockDim.x) {
    const auto zv = ld2(z, k, n);
    const double z0 = to_f64(zv.x), z1 = to_f64(zv.y);
    const double2 rv = ld2(r, k, n);
    if (copy) {
      if (2 * k + 1 < n) reinterpret_cast<double2*>(z64)[k] = make_double2(z0, z1);
      else z64[2 * k] = z0;
    }
    a = fma(z1, rv.y, fma(z0, rv.x, a));
    if (q) {
      const double2 qv = ld2(q, k, n);
      b = fma(z1, qv.y, fma(z0, qv.x, b));
    }
  }
  a = block_sum(a, sred);
  b = block_sum(b, sred);
  if (threadIdx.x == 0) {
    pa[blockIdx.x] = a;
    if (q) pb[blockIdx.x] = b;
  }
  if (last_block(&sc->tk[TK_DOTS], gridDim.x))
    finish_body(kind, pa, gridDim.x, pb, q ? gridDim.x : 0, sc, sred);
}

// while condition of a captured block solve: go on while some right-hand side is not done
__global__ void k_block_cond(const Scalars* sc, int nrhs, cudaGraphConditionalHandle cond) {
  pdl_prologue();
  if (threadIdx.x != 0) return;
  int any = 0;
  for (int r = 0; r < nrhs; r++) any |= (*(volatile const int*)&sc[r].done) ? 0 : 1;
  cudaGraphSetConditional(cond, any ? 1u : 0u);
}

template <class T>
__global__ void k_cast_in(const double* __restrict__ a, T* __restrict__ b, int64_t n,
                          const int* done) {
  pdl_prologue();
  if (solve_done(done)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (T)a[i];
}

__global__ void k_mask_vec(const double* __restrict__ f, double* __restrict__ b,
                           const uint8_t* __restrict__ mask, int dim, int64_t nn) {
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  const unsigned m = mask[node];
  for (int c = 0; c < dim; c++) b[dim * node + c] = ((m >> c) & 1u) ? 0.0 : f[dim * node + c];
}

template <class T, int B>
__global__ void k_jacobi0(int64_t nodes, const T* __restrict__ Dinv, const T* __restrict__ b,
                          T* __restrict__ x, T omega, const int* done) {
  pdl_launch();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nodes) return;
  b += (int64_t)blockIdx.y * rhs_stride(B * nodes);  // right-hand side blockIdx.y
  x += (int64_t)blockIdx.y * rhs_stride(B * nodes);
  T D[B * B];  // the smoother block is fixed during a solve: fetched before the wait
#pragma unroll
  for (int t = 0; t < B * B; t++) D[t] = Dinv[(int64_t)B * B * i + t];
  pdl_wait();
  if (solve_done(done)) return;
  T bv[B], xv[B];
#pragma unroll
  for (int c = 0; c < B; c++) bv[c] = b[B * i + c];
  jacobi_block<T, B>(D, bv, omega, xv);
#pragma unroll
  for (int r = 0; r < B; r++) x[B * i + r] = xv[r];
}

// Flexible GMRES building blocks.  parts[k * gridDim.x + block] = partial of V_k . w over the
// block's grid-stride share (V_k = V + k * ldv); grid.y = number of vectors.
__global__ void k_mdot(int64_t n, const double* __restrict__ V, int64_t ldv,
                       const double* __restrict__ w, double* parts) {
  __shared__ double sred[32];
  const double* v = V + (int64_t)blockIdx.y * ldv;
  double a = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a += v[i] * w[i];
  a = block_sum(a, sred);
  if (threadIdx.x == 0) parts[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = a;
}
// h[k] = sum over blocks of parts[k * nb + b], fixed order; one block per vector
__global__ void k_mdot_finish(const double* __restrict__ parts, int nb, double* h) {
  __shared__ double sred[32];
  double a = 0.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) a += parts[(int64_t)blockIdx.x * nb + q];
  a = block_sum(a, sred);
  if (threadIdx.x == 0) h[blockIdx.x] = a;
}
// w += sign * sum_k c[k] V_k (k < J, fixed order)
__global__ void k_mupdate(int64_t n, int J, const double* __restrict__ V, int64_t ldv,
                          const double* __restrict__ c, double sign, double* __restrict__ w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0;
  for (int k = 0; k < J; k++) a += c[k] * V[(int64_t)k * ldv + i];
  w[i] += sign * a;
}
__global__ void k_scale_into(int64_t n, const double* __restrict__ w, double s, double* v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = s * w[i];
}

template <class T>
__global__ void k_gemv(int n, const T* __restrict__ A, const T* __restrict__ b, T* __restrict__ x,
                       const int* done) {
  // the coarse inverse is fixed during a solve: each lane fetches its first PF entries of the
  // row before waiting for the producer of b
  constexpr int PF = 24;
  pdl_launch();
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= n) return;
  b += (int64_t)blockIdx.y * rhs_stride(n);  // right-hand side blockIdx.y of a block solve
  x += (int64_t)blockIdx.y * rhs_stride(n);
  const T* a = A + (int64_t)row * n;
  T ap[PF];
#pragma unroll
  for (int k = 0; k < PF; k++) {
    const int c = lane + 32 * k;
    ap[k] = c < n ? a[c] : T(0);
  }
  pdl_wait();
  if (solve_done(done)) return;
  T s = T(0);
#pragma unroll
  for (int k = 0; k < PF; k++) {
    const int c = lane + 32 * k;
    if (c < n) s += ap[k] * b[c];
  }
  for (int c = lane + 32 * PF; c < n; c += 32) s += a[c] * b[c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = s;
}

// Inverse of the SPD coarsest-level matrix (Sec. 3.2: dense Cholesky factorisation at setup)
// in one cooperative launch, FP64, blocks of NB = 32: the blocked right-looking Cholesky
// A = L L^T, the block forward substitution Y = L^-1 (L Y = I), and A^-1 = Y^T Y.  Step b of
// the factorisation has two phases, each closed by a grid barrier:
//   1. every CTA factors the diagonal block L_bb and inverts it in its own shared memory (the
//      same arithmetic on every CTA, so no barrier is spent on broadcasting it); then the rows
//      below, L_ib = A_ib L_bb^-T, and the forward-substitution update of the row blocks
//      i >= b with the previous step's solved block row, B_i -= L_i,b-1 X_b-1 (tiles j < b);
//   2. the trailing lower triangle, A_ij -= L_ib L_jb^T (32 x 32 tiles), and the solved block
//      row X_b = L_bb^-1 B_b (tiles j <= b).
// A final phase forms Y^T Y (lower triangle, mirrored, so exactly symmetric).  Every entry is
// summed in a fixed order (increasing inner index), independent of the grid.  Values written by
// other CTAs are read past L1 (ld.global.cg).
constexpr int NB = 32;
constexpr int INV_THREADS = 512;  // 16 warps: 16 rows of 32 columns per pass over a tile
constexpr unsigned INV_WAIT_LIMIT = 1u << 24;
constexpr int TRI = NB * (NB - 1) / 2;  // entries of the largest trailing triangle (k = 0)

struct InvSmem {
  double s[NB][NB + 1];   // the diagonal block, factored in place
  double li[NB][NB + 1];  // its inverse L_bb^-1
  double ta[NB][NB + 1], tb[NB][NB + 1];  // operand tiles
  double rdiag[NB];
  unsigned char tri_r[TRI], tri_c[TRI];  // (row, column) offsets of the packed triangle
};

// Factor the diagonal block at k0 in shared memory and invert it, right-looking: at pivot k,
// column k of L and row k of L_kk^-1 are scaled by 1 / sqrt(d_k), then the trailing lower
// triangle (s_ij -= l_ik l_jk) and the rows of L_kk^-1 below k (x_ic -= l_ik x_kc) are updated.
// The entries of each update are packed onto consecutive threads, so only as many warps issue
// FP64 work as the step has entries, and the next pivot's 1 / sqrt is taken by the thread that
// has just updated that diagonal entry: two block barriers per pivot.  Rows and columns past n
// are padded with the identity.
__device__ void potrf_tile(int n, int k0, const double* A, InvSmem& m, int* fail) {
  const int t = threadIdx.x;
  const int kb = min(NB, n - k0);
  for (int e = t; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    m.s[r][c] = (r < kb && c < kb) ? __ldcg(A + (int64_t)(k0 + r) * n + k0 + c)
                                   : (r == c ? 1.0 : 0.0);
    m.li[r][c] = r == c ? 1.0 : 0.0;
  }
  __syncthreads();
  auto pivot = [&](int k) {
    double d = m.s[k][k];
    if (!(d > 0.0)) {
      if (k < kb) atomicCAS(fail, 0, k0 + k + 1);
      d = 1.0;
    }
    const double y = rsqrt_newton(d);
    m.s[k][k] = d * y;  // sqrt(d)
    m.rdiag[k] = y;
  };
  if (t == 0) pivot(0);
  __syncthreads();
  for (int k = 0; k < NB; k++) {
    const double y = m.rdiag[k];
    if (t > k && t < NB) m.s[t][k] *= y;                          // column k of L
    if (t >= NB && t - NB <= k && t < 2 * NB) m.li[k][t - NB] *= y;  // row k of L^-1
    __syncthreads();
    const int cnt = (NB - 1 - k) * (NB - k) / 2;
    if (t < cnt) {
      const int i = k + 1 + m.tri_r[t], j = k + 1 + m.tri_c[t];
      m.s[i][j] -= m.s[i][k] * m.s[j][k];
    }
    const int lc = (NB - 1 - k) * (k + 1);
    for (int u = t; u < lc; u += blockDim.x) {
      const int i = k + 1 + u / (k + 1), c = u % (k + 1);
      m.li[i][c] -= m.s[i][k] * m.li[k][c];
    }
    // entry 0 of the trailing triangle is the next diagonal entry, just updated by thread 0
    if (t == 0 && k + 1 < NB) pivot(k + 1);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(INV_THREADS) k_spd_inverse(int n, double* A, double* Y,
                                                             int* fail, unsigned* sync,
                                                             unsigned wait_limit) {
  __shared__ InvSmem m;
  const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
  const int G = gridDim.x, bid = blockIdx.x;
  const int nblk = (n + NB - 1) / NB;
  for (int u = t; u < TRI; u += blockDim.x) {  // u = r (r + 1) / 2 + c, 0 <= c <= r
    int r = 0;
    while ((r + 1) * (r + 2) / 2 <= u) r++;
    m.tri_r[u] = (unsigned char)r;
    m.tri_c[u] = (unsigned char)(u - r * (r + 1) / 2);
  }
  for (int64_t e = (int64_t)bid * blockDim.x + t; e < (int64_t)n * n; e += (int64_t)G * blockDim.x)
    Y[e] = (e / n == e % n) ? 1.0 : 0.0;  // the right-hand side B = I
  __syncthreads();

  for (int b = 0; b < nblk; b++) {
    const int k0 = b * NB, kb = min(NB, n - k0);
    const int rest = n - k0 - kb;
    // ---- phase 1: L_bb and L_bb^-1 (every CTA), the panel, the update with X_b-1
    potrf_tile(n, k0, A, m, fail);
    const int n_panel = (rest + 15) / 16;
    const int n_upd = b * (nblk - b);  // tiles (i, j), i in [b, nblk), j in [0, b)
    for (int u = bid; u < n_panel + n_upd; u += G) {
      if (u < n_panel) {  // 16 rows, one per warp: L_ib = A_ib L_bb^-T
        const int i = k0 + kb + u * 16 + ty;
        const bool ok = i < n && tx < kb;
        m.ta[ty][tx] = ok ? __ldcg(A + (int64_t)i * n + k0 + tx) : 0.0;
        __syncwarp();
        if (ok) {
          double v = 0.0;
          for (int q = 0; q <= tx; q++) v += m.ta[ty][q] * m.li[tx][q];
          A[(int64_t)i * n + k0 + tx] = v;
        }
        __syncwarp();
      } else {  // B_i -= L_i,b-1 X_b-1 on tile (i, j)
        const int w = u - n_panel;
        const int K0 = (b - 1) * NB, kbp = min(NB, n - K0);
        const int r0 = (b + w / b) * NB, c0 = (w % b) * NB;
        __syncthreads();
        for (int r = ty; r < NB; r += 16) {
          const int gi = r0 + r, c = c0 + tx;
          m.ta[r][tx] = (gi < n && tx < kbp) ? __ldcg(A + (int64_t)gi * n + K0 + tx) : 0.0;
          m.tb[r][tx] = (r < kbp && c < n) ? __ldcg(Y + (int64_t)(K0 + r) * n + c) : 0.0;
        }
        __syncthreads();
        for (int r = ty; r < NB; r += 16) {
          const int gi = r0 + r, c = c0 + tx;
          if (gi >= n || c >= n) continue;
          double v = 0.0;
#pragma unroll 8
          for (int q = 0; q < NB; q++) v += m.ta[r][q] * m.tb[q][tx];
          const int64_t o = (int64_t)gi * n + c;
          Y[o] = __ldcg(Y + o) - v;
        }
      }
    }
    if (!grid_sync(sync, sync + 2, G, wait_limit)) return;
    // ---- phase 2: X_b = L_bb^-1 B_b, the trailing update
    const int n_x = b + 1;  // tiles j <= b of block row b
    const int nt = (rest + 31) / 32;
    const int n_syrk = nt * (nt + 1) / 2;
    for (int u = bid; u < n_x + n_syrk; u += G) {
      __syncthreads();
      if (u < n_x) {
        const int c0 = u * NB;
        for (int r = ty; r < NB; r += 16) {
          const int c = c0 + tx;
          m.ta[r][tx] = (r < kb && c < n) ? __ldcg(Y + (int64_t)(k0 + r) * n + c) : 0.0;
        }
        __syncthreads();
        for (int r = ty; r < kb; r += 16) {
          const int c = c0 + tx;
          double v = 0.0;
          for (int q = 0; q <= r; q++) v += m.li[r][q] * m.ta[q][tx];
          if (c < n) Y[(int64_t)(k0 + r) * n + c] = v;
        }
      } else {  // tile (ti, tj), tj <= ti, of the trailing lower triangle
        const int w = u - n_x;
        int ti = 0;
        while ((ti + 1) * (ti + 2) / 2 <= w) ti++;
        const int tj = w - ti * (ti + 1) / 2;
        const int i0 = k0 + kb + ti * 32, j0 = k0 + kb + tj * 32;
        for (int r = ty; r < 32; r += 16) {
          const int gi = i0 + r, gj = j0 + r;
          m.ta[r][tx] = (gi < n && tx < kb) ? __ldcg(A + (int64_t)gi * n + k0 + tx) : 0.0;
          m.tb[r][tx] = (gj < n && tx < kb) ? __ldcg(A + (int64_t)gj * n + k0 + tx) : 0.0;
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 16) {
          const int gi = i0 + r, gj = j0 + tx;
          if (gi >= n || gj >= n || gj > gi) continue;
          double v = 0.0;
          for (int q = 0; q < kb; q++) v += m.ta[r][q] * m.tb[tx][q];
          const int64_t o = (int64_t)gi * n + gj;
          A[o] = __ldcg(A + o) - v;
        }
      }
    }
    if (!grid_sync(sync, sync + 2, G, wait_limit)) return;
  }

  // ---- A^-1 = Y^T Y: entry (i, j), j <= i, sums Y_ti Y_tj over t = i .. n - 1 in order.
  // Tiles of 16 rows i x 32 columns j; Y is staged 32 rows t at a time.
  const int nti = (n + 15) / 16, ntj = (n + 31) / 32;
  for (int u = bid; u < nti * ntj; u += G) {
    const int i0 = (u / ntj) * 16, j0 = (u % ntj) * 32;
    if (j0 > i0 + 15) continue;  // above the diagonal (uniform over the CTA)
    const int i = i0 + ty, j = j0 + tx;
    double v = 0.0;
    for (int tc = i0; tc < n; tc += 32) {
      __syncthreads();
      {
        const int q = t >> 4, c = t & 15;  // 32 rows x 16 columns i
        m.ta[q][c] = (tc + q < n && i0 + c < n) ? __ldcg(Y + (int64_t)(tc + q) * n + i0 + c) : 0.0;
      }
      for (int e = t; e < 32 * 32; e += blockDim.x) {
        const int q = e >> 5, c = e & 31;
        m.tb[q][c] = (tc + q < n && j0 + c < n) ? __ldcg(Y + (int64_t)(tc + q) * n + j0 + c) : 0.0;
      }
      __syncthreads();
      if (i < n && j <= i) {
        const int q0 = max(0, i - tc), q1 = min(32, n - tc);
        for (int q = q0; q < q1; q++) v += m.ta[q][ty] * m.tb[q][tx];
      }
    }
    if (i < n && j <= i) {
      A[(int64_t)i * n + j] = v;
      A[(int64_t)j * n + i] = v;
    }
  }
}

inline int grid_for(int64_t n) {
  return std::max(1, std::min(RED_MAX_BLOCKS, ceil_div((n + 1) / 2, RED_THREADS)));
}

}  // namespace

int red_blocks(int64_t n) { return grid_for(n); }

constexpr int MDOT_BLOCKS = 120;  // partial sums per dot of the FGMRES kernels

void multi_dot(cudaStream_t s, int64_t n, int J, const double* V, int64_t ldv, const double* w,
               double* parts, double* h) {
  if (J < 1) return;
  LAUNCH(k_mdot, dim3(MDOT_BLOCKS, J), 256, 0, s, n, V, ldv, w, parts);
  LAUNCH(k_mdot_finish, J, 256, 0, s, parts, MDOT_BLOCKS, h);
}
int multi_dot_parts(int J) { return MDOT_BLOCKS * J; }

void multi_update(cudaStream_t s, int64_t n, int J, const double* V, int64_t ldv, const double* c,
                  double sign, double* w) {
  if (J < 1) return;
  LAUNCH(k_mupdate, ceil_div(n, 256), 256, 0, s, n, J, V, ldv, c, sign, w);
}

void scale_into(cudaStream_t s, int64_t n, const double* w, double sc, double* v) {
  LAUNCH(k_scale_into, ceil_div(n, 256), 256, 0, s, n, w, sc, v);
}

void dot_partials(cudaStream_t s, const double* x, const double* y, int64_t n, double* partials,
                  const int* done) {
  LAUNCH(k_dot, dim3(grid_for(n), batch_rhs()), RED_THREADS, 0, s, x, y, n, partials, done);
}

void finish(cudaStream_t s, int kind, const double* pa, int na, const double* pb, int nb,
            Scalars* sc) {
  LAUNCH(k_finish, batch_rhs(), 256, 0, s, kind, pa, na, pb, nb, sc);
}

void xr_update(cudaStream_t s, double* x, double* r, const double* p, const double* q, int64_t n,
               Scalars* sc, double* partials, float* r32) {
  LAUNCH(k_xr, dim3(grid_for(n), batch_rhs()), RED_THREADS, 0, s, x, r, p, q, n, sc, partials, r32);
}

void p_update(cudaStream_t s, double* p, const double* z, int64_t n, const Scalars* sc,
              cudaGraphConditionalHandle cond, int has_cond) {
  if (batch_rhs() > 1 && has_cond) TOMG_THROW(TOMG_E_INVALID, "block p update sets no condition");
  LAUNCH(k_p, dim3(grid_for(n), batch_rhs()), RED_THREADS, 0, s, p, z, n, sc, cond, has_cond);
}

void block_cond(cudaStream_t s, const Scalars* sc, int nrhs, cudaGraphConditionalHandle cond) {
  LAUNCH(k_block_cond, 1, 32, 0, s, sc, nrhs, cond);
}

template <class T>
void z_dots(cudaStream_t s, const T* z, double* z64, const double* r, const double* q, int64_t n,
            double* pa, double* pb, Scalars* sc, int kind) {
  LAUNCH((k_zdots<T>), dim3(grid_for(n), batch_rhs()), RED_THREADS, 0, s, z, z64, r, q, n, pa, pb,
         sc, kind);
}
template void z_dots<float>(cudaStream_t, const float*, double*, const double*, const double*,
                            int64_t, double*, double*, Scalars*, int);
template void z_dots<double>(cudaStream_t, const double*, double*, const double*, const double*,
                             int64_t, double*, double*, Scalars*, int);

template <class T>
void cast_in(cudaStream_t s, const double* a, T* b, int64_t n, const int* done) {
  // elementwise: the right-hand sides of a block solve are one contiguous vector
  if (batch_rhs() > 1 && done) TOMG_THROW(TOMG_E_INVALID, "block cast with a done flag");
  if (batch_rhs() > 1) n = batch_rhs() * rhs_stride(n);  // padding entries included
  LAUNCH((k_cast_in<T>), grid_for(n), RED_THREADS, 0, s, a, b, n, done);
}
template void cast_in<float>(cudaStream_t, const double*, float*, int64_t, const int*);
template void cast_in<double>(cudaStream_t, const double*, double*, int64_t, const int*);

void copy_f64(cudaStream_t s, const double* a, double* b, int64_t n, const int* done) {
  cast_in<double>(s, a, b, n, done);
}

void mask_vec(cudaStream_t s, const double* f, double* b, const uint8_t* mask, int dim, int64_t nn) {
  no_batch("mask_vec");
  LAUNCH(k_mask_vec, ceil_div(nn, 256), 256, 0, s, f, b, mask, dim, nn);
}

template <class T>
void jacobi0(cudaStream_t s, int bs, int64_t nodes, const T* Dinv, const T* b, T* x, double omega,
             const int* done) {
  const dim3 g(ceil_div(nodes, 256), batch_rhs());
  if (bs == 2) LAUNCH((k_jacobi0<T, 2>), g, 256, 0, s, nodes, Dinv, b, x, (T)omega, done);
  else if (bs == 3) LAUNCH((k_jacobi0<T, 3>), g, 256, 0, s, nodes, Dinv, b, x, (T)omega, done);
  else if (bs == 6) LAUNCH((k_jacobi0<T, 6>), g, 256, 0, s, nodes, Dinv, b, x, (T)omega, done);
  else TOMG_THROW(TOMG_E_INVALID, "unsupported block size %d", bs);
}
template void jacobi0<float>(cudaStream_t, int, int64_t, const float*, const float*, float*,
                             double, const int*);
template void jacobi0<double>(cudaStream_t, int, int64_t, const double*, const double*, double*,
                              double, const int*);

template <class T>
void dense_gemv(cudaStream_t s, int n, const T* Ainv, const T* b, T* x, const int* done) {
  LAUNCH((k_gemv<T>), dim3(ceil_div((int64_t)n * 32, 256), batch_rhs()), 256, 0, s, n, Ainv, b, x,
         done);
}
template void dense_gemv<float>(cudaStream_t, int, const float*, const float*, float*, const int*);
template void dense_gemv<double>(cudaStream_t, int, const double*, const double*, double*,
                                 const int*);

int dense_spd_inverse(cudaStream_t s, int n, double* A, double* work) {
  SetupTrace tr(s);
  if (n <= 0) return 0;
  // one cooperative launch, every CTA resident
  static int per_sm = 0;
  if (per_sm == 0)
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spd_inverse, INV_THREADS, 0));
  const int nblk = ceil_div(n, NB);
  const int work_items = std::max(nblk * (nblk + 1) / 2, ceil_div(n, 16) * ceil_div(n, 32) / 2);
  // one CTA per SM at most: every CTA factors the diagonal block itself, and two on one SM
  // would share its FP64 pipe on that critical path
  if (per_sm < 1) TOMG_THROW(TOMG_E_CUDA, "coarse inverse kernel cannot be resident");
  const int grid = std::max(1, std::min(num_sms(), work_items));
  DBuf<int> fail;
  DBuf<unsigned> sync;  // arrivals, generation, error
  fail.resize(1);
  sync.resize(3);
  fail.zero(s);
  sync.zero(s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(INV_THREADS);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  CK(cudaLaunchKernelEx(&cfg, k_spd_inverse, n, A, work, fail.p, sync.p,
                        grid_wait_limit(INV_WAIT_LIMIT)));
  g_launches++;
  int f = 0;
  unsigned err = 0;
  CK(cudaMemcpyAsync(&f, fail.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&err, sync.p + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  tr.mark("  cholesky + inverse");
  if (err) TOMG_THROW(TOMG_E_TIMEOUT, "coarse inverse: a grid barrier wait ran out");
  return f;
}


}  // namespace tomg
