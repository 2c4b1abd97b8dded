// Geometric levels (Sec. 3.2): operators stored as structured 3^d nodal stencils (no column
// indices), bilinear / trilinear transfers built from the coarse grid's shape functions, and
// the Galerkin product A_c = P^T A P (Eq. 9) computed directly on the stencils.
//
// Coarsening: ceil(n/2) coarse elements per axis, coarse node I at fine position min(2I, n);
// 1D weights are 1 at a coincident node and 1/2 at a fine node midway between two coarse
// nodes.  Stencil layout (SoA, coalesced over nodes):
//   S[((o * b + r) * b + c) * n_nodes + node],  o = (ox+1) + 3 (oy+1) + 9 (oz+1).
#include "finish.cuh"

namespace tomg {

namespace {

__device__ __forceinline__ double w1(int p, int I, int nf) {
  const int pI = min(2 * I, nf);
  if (p == pI) return 1.0;
  const int d = p - pI;
  if (d != 1 && d != -1) return 0.0;
  if ((p & 1) == 0 || p == nf) return 0.0;  // p is itself a coarse position
  return 0.5;
}

// the same weight in FP32 (1, 1/2 or 0: products of three are exact in FP32, so the transfer
// kernels form their weights without FP64 instructions, with the same values)
__device__ __forceinline__ float w1f(int p, int I, int nf) {
  const int pI = min(2 * I, nf);
  if (p == pI) return 1.f;
  const int d = p - pI;
  if (d != 1 && d != -1) return 0.f;
  if ((p & 1) == 0 || p == nf) return 0.f;
  return 0.5f;
}

// position of stored entry t (of he per node) of node i in an FP32 half stencil
__host__ __device__ __forceinline__ int64_t half_index(int64_t i, int t, int he) {
  return ((i >> 5) * he + t) * 32 + (i & 31);
}

// FP32 half stencil from the FP64 stencil: entries of the centre and the offsets after it
__global__ void k_stencil_half(int64_t nn, int he, int64_t first, const double* __restrict__ S64,
                               float* __restrict__ S32) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn * he) return;
  const int t = (int)(e / nn);
  const int64_t i = e % nn;
  S32[half_index(i, t, he)] = (float)S64[first + e];
}

template <int DIM>
__device__ __forceinline__ bool in_grid(int i, int j, int k, int nx, int ny, int nz) {
  return i >= 0 && i <= nx && j >= 0 && j <= ny && (DIM == 2 || (k >= 0 && k <= nz));
}

// PROL (MODE_CHEB, dmode 0): the step's iterate is x + P xc, the coarse correction xc (grid
// cnx x cny x cnz) prolonged at every node read, with the prolongation kernel's own arithmetic
template <class T, int DIM, int MODE, bool PROL = false>
__global__ void __launch_bounds__(256) k_stencil(int nx, int ny, int nz, const T* __restrict__ S,
                                                 const T* __restrict__ x, T* __restrict__ y,
                                                 const T* __restrict__ b,
                                                 const T* __restrict__ Dinv, T omega,
                                                 const int* done, T* __restrict__ xo, T c1,
                                                 int dmode, T w0, const T* __restrict__ xc,
                                                 int cnx, int cny, int cnz) {
  constexpr int NO = (DIM == 3) ? 27 : 9, BB = DIM * DIM, C0 = NO / 2;
  // 2D: the node's stencil row (fixed during a solve) is fetched before the wait for the
  // producer of x and b; 3D rows (243 values) are read as they are used
  constexpr bool PRE = DIM == 2;
  // FP32 stencils are stored as their upper half (the centre and the offsets after it): the
  // block of offset o < centre is the transpose of the neighbour's block of offset NO - 1 - o
  // (the Galerkin operators are symmetric), read at the neighbour.  Half the bytes per apply.
  // Layout: tiles of 32 nodes, entry-major inside a tile (half_index), so that the values of
  // the 32 nodes of a warp are one contiguous run per entry and per tile.
  constexpr bool HALF = sizeof(T) == 4;
  constexpr int HE = (NO - C0) * BB;  // stored entries per node
  pdl_launch();
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (DIM == 3 ? nz + 1 : 1);
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  {  // right-hand side blockIdx.y of a block solve
    const int64_t vo = (int64_t)blockIdx.y * rhs_stride(DIM * nn);
    if (x) x += vo;
    y += vo;
    if (b) b += vo;
    if (xo) xo += vo;
    if (PROL)
      xc += (int64_t)blockIdx.y *
            rhs_stride((int64_t)DIM * (cnx + 1) * (cny + 1) * (DIM == 3 ? cnz + 1 : 1));
  }
  int i, j, k;
  node_ijk(node, nx, ny, DIM, i, j, k);
  // entry (r, c) of the block of offset o (neighbour nb)
  auto sval = [&](int o, int r, int c, int64_t nb) -> T {
    if (!HALF) return S[((int64_t)o * BB + r * DIM + c) * nn + node];
    if (o >= C0) return S[half_index(node, (o - C0) * BB + r * DIM + c, HE)];
    return S[half_index(nb, (NO - 1 - o - C0) * BB + c * DIM + r, HE)];
  };
  T Sr[PRE ? NO * BB : 1];
  if (PRE) {
#pragma unroll
    for (int o = 0; o < NO; o++) {
      const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = (DIM == 3) ? o / 9 - 1 : 0;
      const bool in = in_grid<DIM>(i + ox, j + oy, k + oz, nx, ny, nz);
      const int64_t nb = in ? node_id(i + ox, j + oy, k + oz, nx, ny) : node;
#pragma unroll
      for (int t = 0; t < BB; t++) Sr[o * BB + t] = in ? sval(o, t / DIM, t % DIM, nb) : T(0);
    }
  }
  pdl_wait();
  if (solve_done(done)) return;
  AxisP pa[3][3];  // PROL: coarse partners of fine positions i-1..i+1 (and j, k) per axis
  if (PROL) {
#pragma unroll
    for (int d = 0; d < 3; d++) {
      pa[0][d] = axis_partners(i - 1 + d, nx);
      pa[1][d] = axis_partners(j - 1 + d, ny);
      pa[2][d] = DIM == 3 ? axis_partners(k - 1 + d, nz) : AxisP{1, {0, 0}, {1.f, 0.f}};
    }
  }
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; c++) acc[c] = T(0);
#pragma unroll
  for (int o = 0; o < NO; o++) {
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = (DIM == 3) ? o / 9 - 1 : 0;
    if (!in_grid<DIM>(i + ox, j + oy, k + oz, nx, ny, nz)) continue;
    const int64_t nb = node_id(i + ox, j + oy, k + oz, nx, ny);
    T xv[DIM];
    if (MODE == MODE_RESID0) {
      jacobi_first<T, DIM>(Dinv, b, nb, omega, xv);
    } else if (MODE == MODE_CHEB0) {
      jacobi_first<T, DIM>(Dinv, b, nb, w0, xv);
    } else {
#pragma unroll
      for (int c = 0; c < DIM; c++) xv[c] = x[DIM * nb + c];
      if (PROL)
        prolong_acc<T, DIM>(pa[0][ox + 1], pa[1][oy + 1], pa[2][oz + 1], cnx, cny, xc, xv);
    }
#pragma unroll
    for (int r = 0; r < DIM; r++)
#pragma unroll
      for (int c = 0; c < DIM; c++)
        acc[r] += (PRE ? Sr[PRE ? o * BB + r * DIM + c : 0] : sval(o, r, c, nb)) * xv[c];
  }
  if (MODE == MODE_RESID0) {
    T xi[DIM];
    jacobi_first<T, DIM>(Dinv, b, node, omega, xi);
#pragma unroll
    for (int c = 0; c < DIM; c++) {
      xo[DIM * node + c] = xi[c];
      y[DIM * node + c] = b[DIM * node + c] - acc[c];
    }
  } else if (MODE == MODE_APPLY) {
#pragma unroll
    for (int c = 0; c < DIM; c++) y[DIM * node + c] = acc[c];
  } else if (MODE == MODE_RESID) {
#pragma unroll
    for (int c = 0; c < DIM; c++) y[DIM * node + c] = b[DIM * node + c] - acc[c];
  } else if (MODE == MODE_CHEB || MODE == MODE_CHEB0) {
    T r[DIM], xi[DIM];
    if (MODE == MODE_CHEB0) jacobi_first<T, DIM>(Dinv, b, node, w0, xi);
#pragma unroll
    for (int c = 0; c < DIM; c++) {
      r[c] = b[DIM * node + c] - acc[c];
      if (MODE == MODE_CHEB) xi[c] = x[DIM * node + c];
    }
    if (MODE == MODE_CHEB && PROL) prolong_acc<T, DIM>(pa[0][1], pa[1][1], pa[2][1], cnx, cny, xc, xi);
    cheb_node<T, DIM>(node, r, xi, Dinv, c1, omega, MODE == MODE_CHEB0 ? 2 : dmode, xo, y);
  } else {
    T r[DIM];
#pragma unroll
    for (int c = 0; c < DIM; c++) r[c] = b[DIM * node + c] - acc[c];
    const T* D = Dinv + (int64_t)BB * node;
#pragma unroll
    for (int c = 0; c < DIM; c++) {
      T v = T(0);
#pragma unroll
      for (int c2 = 0; c2 < DIM; c2++) v += D[c * DIM + c2] * r[c2];
      y[DIM * node + c] = x[DIM * node + c] + omega * v;
    }
  }
}

// y = S x with one FP64 partial of x . y per block (the outer CG apply on the assembled
// fine-level stencil: 9 / 27 node blocks per row instead of 4 / 8 element products)
template <int DIM>
__global__ void __launch_bounds__(256) k_stencil_apply_dot(int nx, int ny, int nz,
                                                           const double* __restrict__ S,
                                                           const double* __restrict__ x,
                                                           double* __restrict__ y,
                                                           const int* done, double* partials,
                                                           Scalars* sc) {
  constexpr int NO = (DIM == 3) ? 27 : 9, BB = DIM * DIM;
  __shared__ double sred[32];
  pdl_prologue();
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (DIM == 3 ? nz + 1 : 1);
  {  // right-hand side blockIdx.y of a block solve: its vectors, partials and scalar state
    const int64_t vo = (int64_t)blockIdx.y * rhs_stride(DIM * nn);
    x += vo;
    y += vo;
    if (partials) partials += (int64_t)blockIdx.y * gridDim.x;
    if (sc) {
      sc += blockIdx.y;
      if (done) done = &sc->done;
    }
  }
  if (solve_done(done)) return;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double dotv = 0.0;
  if (node < nn) {
    int i, j, k;
    node_ijk(node, nx, ny, DIM, i, j, k);
    double acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; c++) acc[c] = 0.0;
#pragma unroll
    for (int o = 0; o < NO; o++) {
      const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = (DIM == 3) ? o / 9 - 1 : 0;
      if (!in_grid<DIM>(i + ox, j + oy, k + oz, nx, ny, nz)) continue;
      const int64_t nb = node_id(i + ox, j + oy, k + oz, nx, ny);
      double xv[DIM];
#pragma unroll
      for (int c = 0; c < DIM; c++) xv[c] = x[DIM * nb + c];
#pragma unroll
      for (int r = 0; r < DIM; r++)
#pragma unroll
        for (int c = 0; c < DIM; c++) acc[r] += S[((int64_t)o * BB + r * DIM + c) * nn + node] * xv[c];
    }
#pragma unroll
    for (int c = 0; c < DIM; c++) {
      y[DIM * node + c] = acc[c];
      dotv += x[DIM * node + c] * acc[c];
    }
  }
  if (!partials) return;  // plain y = S x (uniform over the grid)
  const double tot = block_sum(dotv, sred);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  if (sc && last_block(&sc->tk[TK_ALPHA], gridDim.x))
    finish_body(FIN_ALPHA, partials, gridDim.x, nullptr, 0, sc, sred);
}

template <int DIM>
__global__ void k_stencil_diag(int nx, int ny, int nz, const double* __restrict__ S, double* Dinv64,
                               float* Dinv32) {
  constexpr int BB = DIM * DIM, CENTER = (DIM == 3) ? 13 : 4;
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (DIM == 3 ? nz + 1 : 1);
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  double D[BB], Di[BB];
  for (int t = 0; t < BB; t++) D[t] = S[((int64_t)CENTER * BB + t) * nn + node];
  spd_inverse<DIM>(D, Di);
  for (int t = 0; t < BB; t++) {
    Dinv64[BB * node + t] = Di[t];
    Dinv32[BB * node + t] = (float)Di[t];
  }
}

// per-axis list of (fine offset from pI, stencil offset, weight) with nonzero weight product
struct AxisPairs {
  int n;
  int di[9], o[9];
  double w[9];
};
__device__ __forceinline__ void axis_pairs(int I, int J, int nf, AxisPairs& L) {
  L.n = 0;
  const int pI = min(2 * I, nf);
  for (int d = -1; d <= 1; d++) {
    const int p = pI + d;
    if (p < 0 || p > nf) continue;
    const double wi = w1(p, I, nf);
    if (wi == 0.0) continue;
    for (int o = -1; o <= 1; o++) {
      const int q = p + o;
      if (q < 0 || q > nf) continue;
      const double wj = w1(q, J, nf);
      if (wj == 0.0) continue;
      L.di[L.n] = p;
      L.o[L.n] = o;
      L.w[L.n] = wi * wj;
      L.n++;
    }
  }
}

// One axis of the Galerkin product.  P is a tensor product of 1D interpolations, so
// P^T A P = Px^T (Py^T (Pz^T A Pz) Py) Px can be formed one axis at a time: the stencil stays
// 3^d-point after each step, and every output block sums at most 7 weighted input blocks
// instead of up to 7^d for the direct product.  Input grid (nx, ny, nz) with `axis` fine,
// output grid with that axis coarsened to cn (the other axes unchanged).
template <int AXIS>
__global__ void k_rap_axis(int nx, int ny, int nz, int cn, const double* __restrict__ Sin,
                           double* __restrict__ Sout) {
  constexpr int BB = 9;
  const int onx = AXIS == 0 ? cn : nx, ony = AXIS == 1 ? cn : ny, onz = AXIS == 2 ? cn : nz;
  const int64_t nin = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  const int64_t nout = (int64_t)(onx + 1) * (ony + 1) * (onz + 1);
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int O = blockIdx.y;
  if (I >= nout) return;
  int c[3];
  node_ijk(I, onx, ony, 3, c[0], c[1], c[2]);
  const int oo[3] = {O % 3 - 1, (O / 3) % 3 - 1, O / 9 - 1};
  const int na = AXIS == 0 ? nx : (AXIS == 1 ? ny : nz);  // fine extent along the axis
  const int cnA = AXIS == 0 ? onx : (AXIS == 1 ? ony : onz);
  double acc[BB];
#pragma unroll
  for (int t = 0; t < BB; t++) acc[t] = 0.0;
  const int Ia = c[AXIS], Ja = Ia + oo[AXIS];
  if (Ja >= 0 && Ja <= cnA) {
    AxisPairs L;
    axis_pairs(Ia, Ja, na, L);
    for (int a = 0; a < L.n; a++) {
      int f[3] = {c[0], c[1], c[2]};
      f[AXIS] = L.di[a];
      int fo[3] = {oo[0], oo[1], oo[2]};
      fo[AXIS] = L.o[a];
      const int64_t fi = node_id(f[0], f[1], f[2], nx, ny);
      const int oi = (fo[0] + 1) + 3 * (fo[1] + 1) + 9 * (fo[2] + 1);
      const double wt = L.w[a];
#pragma unroll
      for (int t = 0; t < BB; t++) acc[t] += wt * Sin[((int64_t)oi * BB + t) * nin + fi];
    }
  }
#pragma unroll
  for (int t = 0; t < BB; t++) Sout[((int64_t)O * BB + t) * nout + I] = acc[t];
}

template <int DIM>
__global__ void k_rap(int fnx, int fny, int fnz, int cnx, int cny, int cnz,
                      const double* __restrict__ Sf, double* __restrict__ Sc) {
  constexpr int BB = DIM * DIM;
  const int64_t nnc = (int64_t)(cnx + 1) * (cny + 1) * (DIM == 3 ? cnz + 1 : 1);
  const int64_t nnf = (int64_t)(fnx + 1) * (fny + 1) * (DIM == 3 ? fnz + 1 : 1);
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int O = blockIdx.y;
  if (I >= nnc) return;
  int Ix, Iy, Iz;
  node_ijk(I, cnx, cny, DIM, Ix, Iy, Iz);
  const int Ox = O % 3 - 1, Oy = (O / 3) % 3 - 1, Oz = (DIM == 3) ? O / 9 - 1 : 0;
  const int Jx = Ix + Ox, Jy = Iy + Oy, Jz = Iz + Oz;
  double acc[BB];
#pragma unroll
  for (int t = 0; t < BB; t++) acc[t] = 0.0;
  if (in_grid<DIM>(Jx, Jy, Jz, cnx, cny, cnz)) {
    AxisPairs Lx, Ly, Lz;
    axis_pairs(Ix, Jx, fnx, Lx);
    axis_pairs(Iy, Jy, fny, Ly);
    if (DIM == 3) axis_pairs(Iz, Jz, fnz, Lz);
    else { Lz.n = 1; Lz.di[0] = 0; Lz.o[0] = 0; Lz.w[0] = 1.0; }
    for (int c = 0; c < Lz.n; c++)
      for (int bq = 0; bq < Ly.n; bq++)
        for (int a = 0; a < Lx.n; a++) {
          const double wt = Lx.w[a] * Ly.w[bq] * Lz.w[c];
          const int64_t fi = node_id(Lx.di[a], Ly.di[bq], Lz.di[c], fnx, fny);
          const int oi = (Lx.o[a] + 1) + 3 * (Ly.o[bq] + 1) + (DIM == 3 ? 9 * (Lz.o[c] + 1) : 0);
#pragma unroll
          for (int t = 0; t < BB; t++) acc[t] += wt * Sf[((int64_t)oi * BB + t) * nnf + fi];
        }
  }
#pragma unroll
  for (int t = 0; t < BB; t++) Sc[((int64_t)O * BB + t) * nnc + I] = acc[t];
}

template <class T, int DIM>
__global__ void k_restrict(int fnx, int fny, int fnz, int cnx, int cny, int cnz,
                           const T* __restrict__ rf, T* __restrict__ bc, const int* done) {
  pdl_prologue();
  if (solve_done(done)) return;
  const int64_t nnc = (int64_t)(cnx + 1) * (cny + 1) * (DIM == 3 ? cnz + 1 : 1);
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nnc) return;
  {  // right-hand side blockIdx.y of a block solve
    const int64_t nnf = (int64_t)(fnx + 1) * (fny + 1) * (DIM == 3 ? fnz + 1 : 1);
    rf += (int64_t)blockIdx.y * rhs_stride(DIM * nnf);
    bc += (int64_t)blockIdx.y * rhs_stride(DIM * nnc);
  }
  int Ix, Iy, Iz;
  node_ijk(I, cnx, cny, DIM, Ix, Iy, Iz);
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; c++) acc[c] = T(0);
  const int px = min(2 * Ix, fnx), py = min(2 * Iy, fny), pz = (DIM == 3) ? min(2 * Iz, fnz) : 0;
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); dz++) {
    const int z = pz + dz;
    if (DIM == 3 && (z < 0 || z > fnz)) continue;
    const float wz = (DIM == 3) ? w1f(z, Iz, fnz) : 1.f;
    if (wz == 0.f) continue;
    for (int dy = -1; dy <= 1; dy++) {
      const int yy = py + dy;
      if (yy < 0 || yy > fny) continue;
      const float wy = w1f(yy, Iy, fny);
      if (wy == 0.f) continue;
      for (int dx = -1; dx <= 1; dx++) {
        const int xx = px + dx;
        if (xx < 0 || xx > fnx) continue;
        const float wx = w1f(xx, Ix, fnx);
        if (wx == 0.f) continue;
        const T w = (T)(wx * wy * wz);
        const int64_t fi = node_id(xx, yy, z, fnx, fny);
#pragma unroll
        for (int c = 0; c < DIM; c++) acc[c] += w * rf[DIM * fi + c];
      }
    }
  }
#pragma unroll
  for (int c = 0; c < DIM; c++) bc[DIM * I + c] = acc[c];
}


template <class T, int DIM>
__global__ void k_prolong_add(int fnx, int fny, int fnz, int cnx, int cny, int cnz,
                              const T* __restrict__ xc, T* __restrict__ xf, const int* done) {
  pdl_prologue();
  if (solve_done(done)) return;
  const int64_t nnf = (int64_t)(fnx + 1) * (fny + 1) * (DIM == 3 ? fnz + 1 : 1);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnf) return;
  {  // right-hand side blockIdx.y of a block solve
    const int64_t nnc = (int64_t)(cnx + 1) * (cny + 1) * (DIM == 3 ? cnz + 1 : 1);
    xc += (int64_t)blockIdx.y * rhs_stride(DIM * nnc);
    xf += (int64_t)blockIdx.y * rhs_stride(DIM * nnf);
  }
  int x, y, z;
  node_ijk(i, fnx, fny, DIM, x, y, z);
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; c++) acc[c] = xf[DIM * i + c];
  prolong_node<T, DIM>(x, y, z, fnx, fny, fnz, cnx, cny, xc, acc);
#pragma unroll
  for (int c = 0; c < DIM; c++) xf[DIM * i + c] = acc[c];
}

template <int DIM>
__global__ void k_stencil_dense(int nx, int ny, int nz, const double* __restrict__ S, double* A) {
  constexpr int NO = (DIM == 3) ? 27 : 9, BB = DIM * DIM;
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (DIM == 3 ? nz + 1 : 1);
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  const int64_t n = DIM * nn;
  int i, j, k;
  node_ijk(node, nx, ny, DIM, i, j, k);
  for (int o = 0; o < NO; o++) {
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = (DIM == 3) ? o / 9 - 1 : 0;
    if (!in_grid<DIM>(i + ox, j + oy, k + oz, nx, ny, nz)) continue;
    const int64_t nb = node_id(i + ox, j + oy, k + oz, nx, ny);
    for (int r = 0; r < DIM; r++)
      for (int c = 0; c < DIM; c++)
        A[(DIM * node + r) * n + DIM * nb + c] = S[((int64_t)o * BB + r * DIM + c) * nn + node];
  }
}

template <int DIM>
__global__ void k_stencil_counts(int nx, int ny, int nz, int* counts) {
  constexpr int NO = (DIM == 3) ? 27 : 9;
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (DIM == 3 ? nz + 1 : 1);
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  int i, j, k;
  node_ijk(node, nx, ny, DIM, i, j, k);
  int cnt = 0;
  for (int o = 0; o < NO; o++) {
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = (DIM == 3) ? o / 9 - 1 : 0;
    cnt += in_grid<DIM>(i + ox, j + oy, k + oz, nx, ny, nz) ? 1 : 0;
  }
  counts[node] = cnt;
}

template <int DIM>
__global__ void k_stencil_bsr(int nx, int ny, int nz, const double* __restrict__ S,
                              const int* __restrict__ rp, int* ci, double* val) {
  constexpr int NO = (DIM == 3) ? 27 : 9, BB = DIM * DIM;
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (DIM == 3 ? nz + 1 : 1);
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  int i, j, k;
  node_ijk(node, nx, ny, DIM, i, j, k);
  int64_t pos = rp[node];
  for (int o = 0; o < NO; o++) {
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = (DIM == 3) ? o / 9 - 1 : 0;
    if (!in_grid<DIM>(i + ox, j + oy, k + oz, nx, ny, nz)) continue;
    ci[pos] = (int)node_id(i + ox, j + oy, k + oz, nx, ny);
    for (int t = 0; t < BB; t++) val[pos * BB + t] = S[((int64_t)o * BB + t) * nn + node];
    pos++;
  }
}

template <int DIM>
__global__ void k_geoP(int fnx, int fny, int fnz, int cnx, int cny, const int* rp, int* counts,
                       int* ci, double* val) {
  const int64_t nnf = (int64_t)(fnx + 1) * (fny + 1) * (DIM == 3 ? fnz + 1 : 1);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnf) return;
  int x, y, z;
  node_ijk(i, fnx, fny, DIM, x, y, z);
  int Ix[2], Iy[2], Iz[2] = {0, 0};
  double wx[2], wy[2], wz[2] = {1.0, 0.0};
  const int nxs = coarse_of(x, fnx, Ix, wx), nys = coarse_of(y, fny, Iy, wy);
  const int nzs = (DIM == 3) ? coarse_of(z, fnz, Iz, wz) : 1;
  if (counts) { counts[i] = nxs * nys * nzs; return; }
  int64_t pos = rp[i];
  for (int c3 = 0; c3 < nzs; c3++)
    for (int b = 0; b < nys; b++)
      for (int a = 0; a < nxs; a++) {
        ci[pos] = (int)node_id(Ix[a], Iy[b], Iz[c3], cnx, cny);
        const double w = wx[a] * wy[b] * wz[c3];
        for (int r = 0; r < DIM; r++)
          for (int c = 0; c < DIM; c++) val[pos * DIM * DIM + r * DIM + c] = (r == c) ? w : 0.0;
        pos++;
      }
}

}  // namespace

template <class T>
void stencil_op(cudaStream_t s, int mode, const Geo& g, const T* S, const T* x, T* y, const T* b,
                const T* Dinv, double omega, const int* done, const ChebArg* ch) {
  const int64_t nn = g.nodes();
  const dim3 grid(ceil_div(nn, 256), batch_rhs());
  const bool cheb = mode == MODE_CHEB || mode == MODE_CHEB0;
  if (cheb && !ch) TOMG_THROW(TOMG_E_INVALID, "Chebyshev step without its state");
  T* xo = mode == MODE_RESID0 ? const_cast<T*>(x) : (cheb ? (T*)ch->d : nullptr);
  const T c1 = cheb ? (T)ch->c1 : T(0);
  const int dm = cheb ? ch->dmode : 0;
  const T w0 = cheb ? (T)ch->w0 : T(0);
#define STN(D, M) LAUNCH((k_stencil<T, D, M>), grid, 256, 0, s, g.nx, g.ny, g.nz, S, x, y, b, Dinv, (T)omega, done, xo, c1, dm, w0, (const T*)nullptr, 0, 0, 0)
  if (mode == MODE_CHEB && ch->xc) {  // the prolongation fused into the first post-smoothing step
    if (ch->dmode != 0) TOMG_THROW(TOMG_E_INVALID, "fused prolongation on a later step");
    const T* xc = static_cast<const T*>(ch->xc);
    if (g.dim == 2)
      LAUNCH((k_stencil<T, 2, MODE_CHEB, true>), grid, 256, 0, s, g.nx, g.ny, g.nz, S, x, y, b, Dinv,
             (T)omega, done, xo, c1, dm, w0, xc, ch->cnx, ch->cny, ch->cnz);
    else
      LAUNCH((k_stencil<T, 3, MODE_CHEB, true>), grid, 256, 0, s, g.nx, g.ny, g.nz, S, x, y, b, Dinv,
             (T)omega, done, xo, c1, dm, w0, xc, ch->cnx, ch->cny, ch->cnz);
    return;
  }
  if (g.dim == 2) {
    if (mode == MODE_APPLY) STN(2, MODE_APPLY);
    else if (mode == MODE_RESID) STN(2, MODE_RESID);
    else if (mode == MODE_RESID0) STN(2, MODE_RESID0);
    else if (mode == MODE_CHEB) STN(2, MODE_CHEB);
    else if (mode == MODE_CHEB0) STN(2, MODE_CHEB0);
    else STN(2, MODE_JACOBI);
  } else {
    if (mode == MODE_APPLY) STN(3, MODE_APPLY);
    else if (mode == MODE_RESID) STN(3, MODE_RESID);
    else if (mode == MODE_RESID0) STN(3, MODE_RESID0);
    else if (mode == MODE_CHEB) STN(3, MODE_CHEB);
    else if (mode == MODE_CHEB0) STN(3, MODE_CHEB0);
    else STN(3, MODE_JACOBI);
  }
#undef STN
}
template void stencil_op<float>(cudaStream_t, int, const Geo&, const float*, const float*, float*,
                                const float*, const float*, double, const int*, const ChebArg*);
template void stencil_op<double>(cudaStream_t, int, const Geo&, const double*, const double*,
                                 double*, const double*, const double*, double, const int*,
                                 const ChebArg*);

int stencil_blocks(const Geo& g) { return ceil_div(g.nodes(), 256); }

int64_t stencil_half_size(const Geo& g) {
  const int no = g.dim == 3 ? 27 : 9, bb = g.dim * g.dim;
  return (g.nodes() + 31) / 32 * 32 * (int64_t)(no - no / 2) * bb;
}

void stencil_half_f32(cudaStream_t s, const Geo& g, const double* S64, float* S32) {
  const int no = g.dim == 3 ? 27 : 9, bb = g.dim * g.dim, he = (no - no / 2) * bb;
  const int64_t nn = g.nodes();
  CK(cudaMemsetAsync(S32, 0, sizeof(float) * stencil_half_size(g), s));  // tile padding
  LAUNCH(k_stencil_half, ceil_div(nn * he, 256), 256, 0, s, nn, he, (int64_t)(no / 2) * bb * nn,
         S64, S32);
}

void stencil_apply_dot(cudaStream_t s, const Geo& g, const double* S, const double* x, double* y,
                       const int* done, double* partials, Scalars* sc) {
  const dim3 grid(stencil_blocks(g), batch_rhs());
  if (g.dim == 2)
    LAUNCH(k_stencil_apply_dot<2>, grid, 256, 0, s, g.nx, g.ny, g.nz, S, x, y, done, partials, sc);
  else
    LAUNCH(k_stencil_apply_dot<3>, grid, 256, 0, s, g.nx, g.ny, g.nz, S, x, y, done, partials, sc);
}

void stencil_block_diag_inv(cudaStream_t s, const Geo& g, const double* S, double* Dinv64,
                            float* Dinv32) {
  const int grid = ceil_div(g.nodes(), 128);
  if (g.dim == 2) LAUNCH(k_stencil_diag<2>, grid, 128, 0, s, g.nx, g.ny, g.nz, S, Dinv64, Dinv32);
  else LAUNCH(k_stencil_diag<3>, grid, 128, 0, s, g.nx, g.ny, g.nz, S, Dinv64, Dinv32);
}

void stencil_rap(cudaStream_t s, const Geo& f, const Geo& c, const double* Sf, double* Sc) {
  if (f.dim == 2) {
    dim3 grid(ceil_div(c.nodes(), 128), 9);
    LAUNCH(k_rap<2>, grid, 128, 0, s, f.nx, f.ny, f.nz, c.nx, c.ny, c.nz, Sf, Sc);
    return;
  }
  // hex8: x, then y, then z (two intermediate stencils)
  const int64_t n1 = (int64_t)(c.nx + 1) * (f.ny + 1) * (f.nz + 1);
  const int64_t n2 = (int64_t)(c.nx + 1) * (c.ny + 1) * (f.nz + 1);
  DBuf<double> S1, S2;
  S1.resize(243 * n1);
  S2.resize(243 * n2);
  LAUNCH(k_rap_axis<0>, dim3(ceil_div(n1, 128), 27), 128, 0, s, f.nx, f.ny, f.nz, c.nx, Sf, S1.p);
  LAUNCH(k_rap_axis<1>, dim3(ceil_div(n2, 128), 27), 128, 0, s, c.nx, f.ny, f.nz, c.ny, S1.p, S2.p);
  LAUNCH(k_rap_axis<2>, dim3(ceil_div(c.nodes(), 128), 27), 128, 0, s, c.nx, c.ny, f.nz, c.nz, S2.p, Sc);
}

template <class T>
void geo_restrict(cudaStream_t s, const Geo& f, const Geo& c, const T* rf, T* bc, const int* done) {
  const dim3 grid(ceil_div(c.nodes(), 256), batch_rhs());
  if (f.dim == 2)
    LAUNCH((k_restrict<T, 2>), grid, 256, 0, s, f.nx, f.ny, f.nz, c.nx, c.ny, c.nz, rf, bc, done);
  else
    LAUNCH((k_restrict<T, 3>), grid, 256, 0, s, f.nx, f.ny, f.nz, c.nx, c.ny, c.nz, rf, bc, done);
}
template void geo_restrict<float>(cudaStream_t, const Geo&, const Geo&, const float*, float*,
                                  const int*);
template void geo_restrict<double>(cudaStream_t, const Geo&, const Geo&, const double*, double*,
                                   const int*);

template <class T>
void geo_prolong_add(cudaStream_t s, const Geo& f, const Geo& c, const T* xc, T* xf,
                     const int* done) {
  const dim3 grid(ceil_div(f.nodes(), 256), batch_rhs());
  if (f.dim == 2)
    LAUNCH((k_prolong_add<T, 2>), grid, 256, 0, s, f.nx, f.ny, f.nz, c.nx, c.ny, c.nz, xc, xf, done);
  else
    LAUNCH((k_prolong_add<T, 3>), grid, 256, 0, s, f.nx, f.ny, f.nz, c.nx, c.ny, c.nz, xc, xf, done);
}
template void geo_prolong_add<float>(cudaStream_t, const Geo&, const Geo&, const float*, float*,
                                     const int*);
template void geo_prolong_add<double>(cudaStream_t, const Geo&, const Geo&, const double*, double*,
                                      const int*);

void stencil_to_dense(cudaStream_t s, const Geo& g, const double* S, double* A) {
  const int64_t n = g.dim * g.nodes();
  CK(cudaMemsetAsync(A, 0, sizeof(double) * n * n, s));
  const int grid = ceil_div(g.nodes(), 128);
  if (g.dim == 2) LAUNCH(k_stencil_dense<2>, grid, 128, 0, s, g.nx, g.ny, g.nz, S, A);
  else LAUNCH(k_stencil_dense<3>, grid, 128, 0, s, g.nx, g.ny, g.nz, S, A);
}

void stencil_row_counts(cudaStream_t s, const Geo& g, int* counts) {
  const int grid = ceil_div(g.nodes(), 256);
  if (g.dim == 2) LAUNCH(k_stencil_counts<2>, grid, 256, 0, s, g.nx, g.ny, g.nz, counts);
  else LAUNCH(k_stencil_counts<3>, grid, 256, 0, s, g.nx, g.ny, g.nz, counts);
}

void stencil_to_bsr(cudaStream_t s, const Geo& g, const double* S, const int* rp, int* ci,
                    double* val) {
  const int grid = ceil_div(g.nodes(), 128);
  if (g.dim == 2) LAUNCH(k_stencil_bsr<2>, grid, 128, 0, s, g.nx, g.ny, g.nz, S, rp, ci, val);
  else LAUNCH(k_stencil_bsr<3>, grid, 128, 0, s, g.nx, g.ny, g.nz, S, rp, ci, val);
}

void geo_prolong_counts(cudaStream_t s, const Geo& f, const Geo& c, int* counts) {
  const int grid = ceil_div(f.nodes(), 256);
  if (f.dim == 2)
    LAUNCH(k_geoP<2>, grid, 256, 0, s, f.nx, f.ny, f.nz, c.nx, c.ny, (const int*)nullptr, counts,
           (int*)nullptr, (double*)nullptr);
  else
    LAUNCH(k_geoP<3>, grid, 256, 0, s, f.nx, f.ny, f.nz, c.nx, c.ny, (const int*)nullptr, counts,
           (int*)nullptr, (double*)nullptr);
}

void geo_prolong_fill(cudaStream_t s, const Geo& f, const Geo& c, const int* rp, int* ci,
                      double* val) {
  const int grid = ceil_div(f.nodes(), 256);
  if (f.dim == 2)
    LAUNCH(k_geoP<2>, grid, 256, 0, s, f.nx, f.ny, f.nz, c.nx, c.ny, rp, (int*)nullptr, ci, val);
  else
    LAUNCH(k_geoP<3>, grid, 256, 0, s, f.nx, f.ny, f.nz, c.nx, c.ny, rp, (int*)nullptr, ci, val);
}

}  // namespace tomg
