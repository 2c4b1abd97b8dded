// Galerkin product of the hex8 level-0 operator straight from the elements to the first
// coarse stencil (Sec. 3.2, Eq. 9: A_1 = P^T A_0 P), without assembling the fine stencil.
//
// A_0 = M (sum_e E_e L_e^T Ke L_e) M + (I - M) (M the free-DOF mask).  P is the trilinear
// interpolation of the coarse grid (coarse node I at fine position min(2I, n) per axis), so
// every fine element e lies inside one coarse element and P restricted to it is a fixed 8 x 8
// node weight matrix W_t (times I_3) that depends only on the child's type t: per axis A (first
// child: weights (1, 0) and (1/2, 1/2)), B (second child: (1/2, 1/2) and (0, 1)) or C (the
// single child of the last coarse element of an odd axis: the identity).  Hence
//   A_1 = sum_E L_E^T ( sum_{children e of E} W_t^T (local A_0 of e) W_t ) L_E,
// and for an element that touches no fixed DOF the inner term is E_e T_t with the 24 x 24 table
// T_t = W_t^T Ke W_t (27 types).  Elements that touch a fixed DOF get their own 24 x 24 matrix
// W_t^T (E_e M_e Ke M_e + J_e) W_t, where J_e holds the unit diagonal of the fixed DOFs whose
// owner e is (the element with the lowest index that contains the node), so that the (I - M)
// term is counted once.
//
// One thread per coarse node computes the 3 x 3 blocks of the 14 offsets o >= 13 (the centre
// and the lexicographically positive half: o = (ox+1) + 3 (oy+1) + 9 (oz+1)) as a fixed-order sum
// over the coarse elements containing both nodes and their children, and writes each block
// both at (I, o) and, transposed, at (I + o, 26 - o): the stencil is symmetric by construction.
// The stencil layout is the one of the geometric levels: S[((o * 3 + a) * 3 + b) * n + node].
#include "finish.cuh"

namespace tomg {

namespace {

constexpr int TB = 10;  // stride of one 3 x 3 block of the type table (padded for 16-byte loads)

// 1D weight of fine local node lp of a child of type t towards coarse local node l
__host__ __device__ __forceinline__ double wt1(int t, int lp, int l) {
  if (t == 2) return lp == l ? 1.0 : 0.0;           // C: identity
  if (t == 0) return lp == 0 ? (l == 0 ? 1.0 : 0.0) : 0.5;   // A
  return lp == 1 ? (l == 1 ? 1.0 : 0.0) : 0.5;      // B
}
__device__ __forceinline__ int child_type(int ce, int ch, int nf) {
  return ch ? 1 : (2 * ce + 1 < nf ? 0 : 2);
}
__device__ __forceinline__ double wt3(int t3, int p, int P) {
  return wt1(t3 % 3, p & 1, P & 1) * wt1((t3 / 3) % 3, (p >> 1) & 1, (P >> 1) & 1) *
         wt1(t3 / 9, (p >> 2) & 1, (P >> 2) & 1);
}

// T[(t * 64 + P * 8 + Q) * TB + 3 a + b] = sum_{p, q} W_t(p, P) W_t(q, Q) Ke[3p + a][3q + b]
__global__ void k_gal_table(const double* __restrict__ Ke, double* __restrict__ T) {
  const int t = blockIdx.x, P = threadIdx.x >> 3, Q = threadIdx.x & 7;
  double acc[9];
#pragma unroll
  for (int k = 0; k < 9; k++) acc[k] = 0.0;
  for (int p = 0; p < 8; p++) {
    const double wp = wt3(t, p, P);
    if (wp == 0.0) continue;
    for (int q = 0; q < 8; q++) {
      const double w = wp * wt3(t, q, Q);
      if (w == 0.0) continue;
#pragma unroll
      for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) acc[3 * a + b] += w * Ke[(3 * p + a) * 24 + 3 * q + b];
    }
  }
  double* o = T + (t * 64 + P * 8 + Q) * TB;
#pragma unroll
  for (int k = 0; k < 9; k++) o[k] = acc[k];
  o[9] = 0.0;
}

__global__ void k_gal_flag(int nx, int ny, int nz, const uint8_t* __restrict__ mask,
                           int* __restrict__ flag) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nel = (int64_t)nx * ny * nz;
  if (e >= nel) return;
  const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
  unsigned m = 0;
#pragma unroll
  for (int c = 0; c < 8; c++) m |= mask[node_id(i + (c & 1), j + ((c >> 1) & 1), k + (c >> 2), nx, ny)];
  flag[e] = m ? 1 : 0;
}

__global__ void k_gal_index(int64_t nel, const int* __restrict__ flag, const int* __restrict__ pos,
                            int* __restrict__ midx, int* __restrict__ elist) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  if (flag[e]) {
    midx[e] = pos[e];
    elist[pos[e]] = (int)e;
  } else {
    midx[e] = -1;
  }
}

// the coarse-local 24 x 24 matrix of one fine element that touches a fixed DOF
__global__ void __launch_bounds__(64) k_gal_masked(int nx, int ny, int nz,
                                                   const double* __restrict__ Ke,
                                                   const double* __restrict__ E,
                                                   const uint8_t* __restrict__ mask,
                                                   const int* __restrict__ elist,
                                                   double* __restrict__ Mc) {
  __shared__ double L[576], T1[576], W[64];
  __shared__ unsigned m[8], own[8];
  const int tid = threadIdx.x;
  const int e = elist[blockIdx.x];
  const int fx = e % nx, fy = (e / nx) % ny, fz = e / (nx * ny);
  const int t3 = child_type(fx >> 1, fx & 1, nx) + 3 * child_type(fy >> 1, fy & 1, ny) +
                 9 * child_type(fz >> 1, fz & 1, nz);
  W[tid] = wt3(t3, tid >> 3, tid & 7);  // W[p * 8 + P]
  if (tid < 8) {
    const int px = tid & 1, py = (tid >> 1) & 1, pz = tid >> 2;
    m[tid] = mask[node_id(fx + px, fy + py, fz + pz, nx, ny)];
    // owner of node (i, j, k): element (min(i, nx-1), min(j, ny-1), min(k, nz-1))
    own[tid] = (px == 0 || fx + 1 == nx) && (py == 0 || fy + 1 == ny) && (pz == 0 || fz + 1 == nz);
  }
  __syncthreads();
  const double Ee = E[e];
  for (int k = tid; k < 576; k += 64) {
    const int r = k / 24, c = k % 24;
    const bool fr = (m[r / 3] >> (r % 3)) & 1u, fc = (m[c / 3] >> (c % 3)) & 1u;
    double v = (fr || fc) ? 0.0 : Ee * Ke[k];
    if (r == c && fr && own[r / 3]) v = 1.0;
    L[k] = v;
  }
  __syncthreads();
  for (int k = tid; k < 576; k += 64) {  // T1[p a][Q b] = sum_q L[p a][q b] W(q, Q)
    const int r = k / 24, Q = (k % 24) / 3, b = k % 3;
    double s = 0.0;
    for (int q = 0; q < 8; q++) s += L[r * 24 + 3 * q + b] * W[q * 8 + Q];
    T1[k] = s;
  }
  __syncthreads();
  double* out = Mc + (int64_t)blockIdx.x * 576;
  for (int k = tid; k < 576; k += 64) {  // Mc[P a][Q b] = sum_p W(p, P) T1[p a][Q b]
    const int P = k / 72, a = (k / 24) % 3, c = k % 24;
    double s = 0.0;
    for (int p = 0; p < 8; p++) s += W[p * 8 + P] * T1[(3 * p + a) * 24 + c];
    out[k] = s;
  }
}

__device__ __forceinline__ void gal_range(int I, int J, int nc, int& lo, int& hi) {
  lo = max(max(I, J) - 1, 0);
  hi = min(min(I, J), nc - 1);
}

__global__ void __launch_bounds__(128) k_gal_stencil(int nfx, int nfy, int nfz, int ncx, int ncy,
                                                     int ncz, const double* __restrict__ T,
                                                     const double* __restrict__ E,
                                                     const int* __restrict__ midx,
                                                     const double* __restrict__ Mc,
                                                     double* __restrict__ S) {
  const int64_t ncn = (int64_t)(ncx + 1) * (ncy + 1) * (ncz + 1);
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= ncn) return;
  int Ix, Iy, Iz;
  node_ijk(I, ncx, ncy, 3, Ix, Iy, Iz);
  for (int o = 13; o < 27; o++) {
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
    const int Jx = Ix + ox, Jy = Iy + oy, Jz = Iz + oz;
    const bool inJ = Jx <= ncx && Jy <= ncy && Jz <= ncz && Jx >= 0 && Jy >= 0 && Jz >= 0;
    double blk[9];
#pragma unroll
    for (int k = 0; k < 9; k++) blk[k] = 0.0;
    if (inJ) {
      int x0, x1, y0, y1, z0, z1;
      gal_range(Ix, Jx, ncx, x0, x1);
      gal_range(Iy, Jy, ncy, y0, y1);
      gal_range(Iz, Jz, ncz, z0, z1);
      for (int ez = z0; ez <= z1; ez++)
        for (int ey = y0; ey <= y1; ey++)
          for (int ex = x0; ex <= x1; ex++) {
            const int P = (Ix - ex) + 2 * (Iy - ey) + 4 * (Iz - ez);
            const int Q = (Jx - ex) + 2 * (Jy - ey) + 4 * (Jz - ez);
#pragma unroll 1
            for (int ch = 0; ch < 8; ch++) {
              const int cx = ch & 1, cy = (ch >> 1) & 1, cz = ch >> 2;
              const int fx = 2 * ex + cx, fy = 2 * ey + cy, fz = 2 * ez + cz;
              if (fx >= nfx || fy >= nfy || fz >= nfz) continue;
              const int64_t f = fx + (int64_t)nfx * (fy + (int64_t)nfy * fz);
              const int idx = __ldg(midx + f);
              if (idx < 0) {
                const int t3 = child_type(ex, cx, nfx) + 3 * child_type(ey, cy, nfy) +
                               9 * child_type(ez, cz, nfz);
                const double w = __ldg(E + f);
                const double2* Tp = reinterpret_cast<const double2*>(T + (t3 * 64 + P * 8 + Q) * TB);
#pragma unroll
                for (int k = 0; k < 4; k++) {
                  const double2 v = __ldg(Tp + k);
                  blk[2 * k] += w * v.x;
                  blk[2 * k + 1] += w * v.y;
                }
                blk[8] += w * __ldg(T + (t3 * 64 + P * 8 + Q) * TB + 8);
              } else {
                const double* M = Mc + (int64_t)idx * 576 + (3 * P) * 24 + 3 * Q;
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                  for (int b = 0; b < 3; b++) blk[3 * a + b] += M[a * 24 + b];
              }
            }
          }
    }
#pragma unroll
    for (int k = 0; k < 9; k++) S[((int64_t)o * 9 + k) * ncn + I] = blk[k];
    if (o != 13) {
      const int on = 26 - o;
      if (inJ) {
        const int64_t J = node_id(Jx, Jy, Jz, ncx, ncy);
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
          for (int b = 0; b < 3; b++) S[((int64_t)on * 9 + 3 * b + a) * ncn + J] = blk[3 * a + b];
      }
      // the slot (I, 26 - o) is written by node I - o; with no such node it is zero
      const int Kx = Ix - ox, Ky = Iy - oy, Kz = Iz - oz;
      if (Kx < 0 || Ky < 0 || Kz < 0 || Kx > ncx || Ky > ncy || Kz > ncz) {
#pragma unroll
        for (int k = 0; k < 9; k++) S[((int64_t)on * 9 + k) * ncn + I] = 0.0;
      }
    }
  }
}

}  // namespace

bool ebe_galerkin_stencil(cudaStream_t s, const Ebe& op64, const Geo& c, double* Sc) {
  if (op64.dim != 3) return false;
  const int nx = op64.nx, ny = op64.ny, nz = op64.nz;
  if (c.nx != (nx + 1) / 2 || c.ny != (ny + 1) / 2 || c.nz != (nz + 1) / 2)
    TOMG_THROW(TOMG_E_INVALID, "coarse grid %dx%dx%d is not the coarsening of %dx%dx%d", c.nx,
               c.ny, c.nz, nx, ny, nz);
  const int64_t nel = (int64_t)nx * ny * nz;
  DBuf<int> flag, pos, midx, elist;
  flag.resize(nel);
  pos.resize(nel + 1);
  LAUNCH(k_gal_flag, ceil_div(nel, 256), 256, 0, s, nx, ny, nz, op64.mask, flag.p);
  const int64_t nm = exclusive_scan(s, flag.p, pos.p, nel);
  // elements that touch a fixed DOF keep a 24 x 24 matrix each; beyond one in eight elements
  // the assembled fine stencil and the product on stencils take less memory
  if (nm > nel / 8) return false;
  midx.resize(nel);
  elist.resize(nm > 0 ? nm : 1);
  LAUNCH(k_gal_index, ceil_div(nel, 256), 256, 0, s, nel, flag.p, pos.p, midx.p, elist.p);
  DBuf<double> T, Mc;
  T.resize(27 * 64 * TB);
  Mc.resize(nm > 0 ? nm * 576 : 1);
  const double* Ke = static_cast<const double*>(op64.Ke);
  const double* E = static_cast<const double*>(op64.E);
  LAUNCH(k_gal_table, 27, 64, 0, s, Ke, T.p);
  if (nm > 0)
    LAUNCH(k_gal_masked, (int)nm, 64, 0, s, nx, ny, nz, Ke, E, op64.mask, elist.p, Mc.p);
  LAUNCH(k_gal_stencil, ceil_div(c.nodes(), 128), 128, 0, s, nx, ny, nz, c.nx, c.ny, c.nz, T.p,
         E, midx.p, Mc.p, Sc);
  return true;
}

}  // namespace tomg
