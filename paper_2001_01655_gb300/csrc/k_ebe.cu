// Level-0 operator: matrix-free SIMP element-by-element stiffness apply (Sec. 2.1 Eq. 2,
// Sec. 3.1), its point-block diagonal (Sec. 4.1 block Jacobi) and its assembly into a
// structured 3^d stencil for the Galerkin products (Sec. 3.2 Eq. 9).
//
// Node-centric gather: one thread per node sums E_e * Ke[a, :] x_e over the 2^d elements
// around it (no atomics, deterministic).  Ke is staged in shared memory per block.
// Boundary conditions: A = M K M + (I - M) with M the free-DOF mask.
#include "ops.h"

namespace tomg {

namespace {

template <class T, int DIM, int MODE, bool DOT>
__global__ void __launch_bounds__(256) k_ebe(int nx, int ny, int nz, const T* __restrict__ Ke,
                                             const T* __restrict__ E,
                                             const uint8_t* __restrict__ mask,
                                             const T* __restrict__ x, T* __restrict__ y,
                                             const T* __restrict__ b, const T* __restrict__ Dinv,
                                             T omega, const int* done, double* partials,
                                             T* __restrict__ dch, T c1, int dmode) {
  constexpr int NN = 1 << DIM, ND = DIM * NN;
  __shared__ T sKe[ND * ND];
  __shared__ double sred[32];
  pdl_prologue();
  if (solve_done(done)) return;
  for (int t = threadIdx.x; t < ND * ND; t += blockDim.x) sKe[t] = Ke[t];
  __syncthreads();
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (DIM == 3 ? nz + 1 : 1);
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double dotv = 0.0;
  if (node < nn) {
    int i, j, k;
    node_ijk(node, nx, ny, DIM, i, j, k);
    T acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; c++) acc[c] = T(0);
#pragma unroll
    for (int e = 0; e < NN; e++) {
      const int ex = e & 1, ey = (e >> 1) & 1, ez = (e >> 2) & 1;
      const int ie = i - 1 + ex, je = j - 1 + ey, ke = (DIM == 3) ? k - 1 + ez : 0;
      if (ie < 0 || ie >= nx || je < 0 || je >= ny) continue;
      if (DIM == 3 && (ke < 0 || ke >= nz)) continue;
      const int a = (1 - ex) + 2 * (1 - ey) + (DIM == 3 ? 4 * (1 - ez) : 0);
      const T Ee = E[ie + (int64_t)nx * (je + (int64_t)ny * ke)];
      T part[DIM];
#pragma unroll
      for (int c = 0; c < DIM; c++) part[c] = T(0);
#pragma unroll
      for (int bn = 0; bn < NN; bn++) {
        const int64_t nb = node_id(ie + (bn & 1), je + ((bn >> 1) & 1),
                                   ke + (DIM == 3 ? ((bn >> 2) & 1) : 0), nx, ny);
        const unsigned mb = mask[nb];
#pragma unroll
        for (int c2 = 0; c2 < DIM; c2++) {
          const T xv = ((mb >> c2) & 1u) ? T(0) : x[DIM * nb + c2];
#pragma unroll
          for (int c = 0; c < DIM; c++) part[c] += sKe[(DIM * a + c) * ND + DIM * bn + c2] * xv;
        }
      }
#pragma unroll
      for (int c = 0; c < DIM; c++) acc[c] += Ee * part[c];
    }
    const unsigned mi = mask[node];
    T Ax[DIM], xi[DIM];
#pragma unroll
    for (int c = 0; c < DIM; c++) {
      xi[c] = x[DIM * node + c];
      Ax[c] = ((mi >> c) & 1u) ? xi[c] : acc[c];
    }
    if (MODE == MODE_APPLY) {
#pragma unroll
      for (int c = 0; c < DIM; c++) {
        y[DIM * node + c] = Ax[c];
        if (DOT) dotv += (double)xi[c] * (double)Ax[c];
      }
    } else if (MODE == MODE_RESID) {
#pragma unroll
      for (int c = 0; c < DIM; c++) y[DIM * node + c] = b[DIM * node + c] - Ax[c];
    } else if (MODE == MODE_CHEB) {
      T r[DIM];
#pragma unroll
      for (int c = 0; c < DIM; c++) r[c] = b[DIM * node + c] - Ax[c];
      cheb_node<T, DIM>(node, r, xi, Dinv, c1, omega, dmode, dch, y);
    } else {
      T r[DIM];
#pragma unroll
      for (int c = 0; c < DIM; c++) r[c] = b[DIM * node + c] - Ax[c];
      const T* D = Dinv + (int64_t)DIM * DIM * node;
#pragma unroll
      for (int c = 0; c < DIM; c++) {
        T v = T(0);
#pragma unroll
        for (int c2 = 0; c2 < DIM; c2++) v += D[c * DIM + c2] * r[c2];
        y[DIM * node + c] = xi[c] + omega * v;
      }
    }
  }
  if (DOT) {
    double s = block_sum(dotv, sred);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

template <int DIM>
__global__ void k_ebe_diag(int nx, int ny, int nz, const double* __restrict__ Ke,
                           const double* __restrict__ E, const uint8_t* __restrict__ mask,
                           double* Dinv64, float* Dinv32) {
  constexpr int NN = 1 << DIM, ND = DIM * NN;
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (DIM == 3 ? nz + 1 : 1);
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  int i, j, k;
  node_ijk(node, nx, ny, DIM, i, j, k);
  double D[DIM * DIM];
  for (int t = 0; t < DIM * DIM; t++) D[t] = 0.0;
  for (int e = 0; e < NN; e++) {
    const int ex = e & 1, ey = (e >> 1) & 1, ez = (e >> 2) & 1;
    const int ie = i - 1 + ex, je = j - 1 + ey, ke = (DIM == 3) ? k - 1 + ez : 0;
    if (ie < 0 || ie >= nx || je < 0 || je >= ny) continue;
    if (DIM == 3 && (ke < 0 || ke >= nz)) continue;
    const int a = (1 - ex) + 2 * (1 - ey) + (DIM == 3 ? 4 * (1 - ez) : 0);
    const double Ee = E[ie + (int64_t)nx * (je + (int64_t)ny * ke)];
    for (int r = 0; r < DIM; r++)
      for (int c = 0; c < DIM; c++) D[r * DIM + c] += Ee * Ke[(DIM * a + r) * ND + DIM * a + c];
  }
  const unsigned m = mask[node];
  for (int r = 0; r < DIM; r++)
    for (int c = 0; c < DIM; c++) {
      const bool fr = (m >> r) & 1u, fc = (m >> c) & 1u;
      if (fr || fc) D[r * DIM + c] = (r == c) ? 1.0 : 0.0;
    }
  double Di[DIM * DIM];
  spd_inverse<DIM>(D, Di);
  for (int t = 0; t < DIM * DIM; t++) {
    Dinv64[DIM * DIM * node + t] = Di[t];
    Dinv32[DIM * DIM * node + t] = (float)Di[t];
  }
}

template <int DIM>
__global__ void k_ebe_stencil(int nx, int ny, int nz, const double* __restrict__ Ke,
                              const double* __restrict__ E, const uint8_t* __restrict__ mask,
                              double* __restrict__ S) {
  constexpr int NN = 1 << DIM, ND = DIM * NN, NO = (DIM == 3) ? 27 : 9;
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (DIM == 3 ? nz + 1 : 1);
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  int i, j, k;
  node_ijk(node, nx, ny, DIM, i, j, k);
  const unsigned mi = mask[node];
  for (int o = 0; o < NO; o++) {
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = (DIM == 3) ? o / 9 - 1 : 0;
    const int jx = i + ox, jy = j + oy, jz = k + oz;
    double blk[DIM * DIM];
    for (int t = 0; t < DIM * DIM; t++) blk[t] = 0.0;
    const bool in = jx >= 0 && jx <= nx && jy >= 0 && jy <= ny && (DIM == 2 || (jz >= 0 && jz <= nz));
    if (in) {
      const unsigned mj = mask[node_id(jx, jy, jz, nx, ny)];
      // elements containing both nodes
      for (int e = 0; e < NN; e++) {
        const int ex = e & 1, ey = (e >> 1) & 1, ez = (e >> 2) & 1;
        const int ie = i - 1 + ex, je = j - 1 + ey, ke = (DIM == 3) ? k - 1 + ez : 0;
        if (ie < 0 || ie >= nx || je < 0 || je >= ny) continue;
        if (DIM == 3 && (ke < 0 || ke >= nz)) continue;
        const int bx = jx - ie, by = jy - je, bz = (DIM == 3) ? jz - ke : 0;
        if (bx < 0 || bx > 1 || by < 0 || by > 1 || bz < 0 || bz > 1) continue;
        const int a = (1 - ex) + 2 * (1 - ey) + (DIM == 3 ? 4 * (1 - ez) : 0);
        const int bl = bx + 2 * by + 4 * bz;
        const double Ee = E[ie + (int64_t)nx * (je + (int64_t)ny * ke)];
        for (int r = 0; r < DIM; r++)
          for (int c = 0; c < DIM; c++)
            blk[r * DIM + c] += Ee * Ke[(DIM * a + r) * ND + DIM * bl + c];
      }
      for (int r = 0; r < DIM; r++)
        for (int c = 0; c < DIM; c++) {
          const bool fr = (mi >> r) & 1u, fc = (mj >> c) & 1u;
          if (fr || fc) blk[r * DIM + c] = (o == NO / 2 && r == c && fr) ? 1.0 : 0.0;
        }
    }
    for (int t = 0; t < DIM * DIM; t++) S[((int64_t)o * DIM * DIM + t) * nn + node] = blk[t];
  }
}

__global__ void k_simp(int64_t nel, const double* __restrict__ rho, double E0, double Emin,
                       double penal, double* E64, float* E32, int* bad) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  const double r = rho[e];
  if (!(r >= 0.0)) atomicExch(bad, 1);
  const double Ev = Emin + (E0 - Emin) * pow(r, penal);
  E64[e] = Ev;
  E32[e] = (float)Ev;
}

inline int64_t nodes_of(const Ebe& op) {
  return (int64_t)(op.nx + 1) * (op.ny + 1) * (op.dim == 3 ? op.nz + 1 : 1);
}

// (the tiled 2D operator lives in k_ebe2d.cu)

template <class T, int DIM, int MODE, bool DOT>
void launch_ebe(cudaStream_t s, const Ebe& op, const T* x, T* y, const T* b, const T* Dinv,
                double omega, const int* done, double* parts, const ChebArg* ch = nullptr) {
  // FP32 quad4: tiled kernel (memory/latency bound).  FP64: the node-per-thread kernel, whose
  // low register count keeps enough warps in flight to hide the long FP64 pipe latency.
  if (DIM == 3 && sizeof(T) == 4 && !DOT && op.tc) {
    ebe3d_tc_launch(s, MODE, op, reinterpret_cast<const float*>(x), reinterpret_cast<float*>(y),
                    reinterpret_cast<const float*>(b), reinterpret_cast<const float*>(Dinv),
                    omega, done, ch);
    return;
  }
  no_batch("the element operator other than the tensor-core hex8 kernel");
  if (DIM == 3 && sizeof(T) == 4 && !DOT) {
    ebe3d_launch(s, MODE, op, reinterpret_cast<const float*>(x), reinterpret_cast<float*>(y),
                 reinterpret_cast<const float*>(b), reinterpret_cast<const float*>(Dinv), omega,
                 done, ch);
    return;
  }
  if (DIM == 2 && sizeof(T) == 4) {
    ebe2d_launch<T, MODE, DOT>(s, op, x, y, b, Dinv, omega, done, parts, ch);
    return;
  }
  if (MODE == MODE_CHEB && !ch) TOMG_THROW(TOMG_E_INVALID, "Chebyshev step without its state");
  T* dch = MODE == MODE_CHEB ? (T*)ch->d : nullptr;
  const T c1 = MODE == MODE_CHEB ? (T)ch->c1 : T(0);
  const int dm = MODE == MODE_CHEB ? ch->dmode : 0;
  const int64_t nn = nodes_of(op);
  LAUNCH((k_ebe<T, DIM, MODE, DOT>), ceil_div(nn, 256), 256, 0, s, op.nx, op.ny, op.nz,
         (const T*)op.Ke, (const T*)op.E, op.mask, x, y, b, Dinv, (T)omega, done, parts, dch, c1,
         dm);
}

}  // namespace

int ebe_blocks(const Ebe& op) {
  (void)0;  // partial counts: FP64 applies (the only ones with fused dots) use the generic grid
  return ceil_div(nodes_of(op), 256);
}

template <class T>
void ebe_op(cudaStream_t s, int mode, const Ebe& op, const T* x, T* y, const T* b, const T* Dinv,
            double omega, const int* done, double* parts, const ChebArg* ch) {
  if (mode == MODE_CHEB) {
    if (op.dim == 2) launch_ebe<T, 2, MODE_CHEB, false>(s, op, x, y, b, Dinv, omega, done, parts, ch);
    else launch_ebe<T, 3, MODE_CHEB, false>(s, op, x, y, b, Dinv, omega, done, parts, ch);
    return;
  }
  if (mode == MODE_CHEB0) {
    if (op.dim == 3 && ebe_fuses_transfers<T>(op)) {
      ebe3d_tc_launch(s, MODE_CHEB0, op, reinterpret_cast<const float*>(x),
                      reinterpret_cast<float*>(y), reinterpret_cast<const float*>(b),
                      reinterpret_cast<const float*>(Dinv), omega, done, ch);
      return;
    }
    if (op.dim != 2) TOMG_THROW(TOMG_E_INVALID, "fused first Chebyshev steps on quad4 only");
    ebe2d_launch<T, MODE_CHEB0, false>(s, op, x, y, b, Dinv, omega, done, parts, ch);
    return;
  }
  if (ch && ch->xc && !(op.dim == 3 && ebe_fuses_transfers<T>(op)))
    TOMG_THROW(TOMG_E_INVALID, "fused prolongation on the hex8 tensor-core operator only");
  if (op.dim == 2) {
    if (mode == MODE_APPLY) {
      if (parts) launch_ebe<T, 2, MODE_APPLY, true>(s, op, x, y, b, Dinv, omega, done, parts);
      else launch_ebe<T, 2, MODE_APPLY, false>(s, op, x, y, b, Dinv, omega, done, parts);
    } else if (mode == MODE_RESID) {
      launch_ebe<T, 2, MODE_RESID, false>(s, op, x, y, b, Dinv, omega, done, parts);
    } else if (mode == MODE_RESID0) {
      ebe2d_launch<T, MODE_RESID0, false>(s, op, x, y, b, Dinv, omega, done, parts);
    } else {
      launch_ebe<T, 2, MODE_JACOBI, false>(s, op, x, y, b, Dinv, omega, done, parts);
    }
  } else {
    if (mode == MODE_APPLY) {
      if (parts) launch_ebe<T, 3, MODE_APPLY, true>(s, op, x, y, b, Dinv, omega, done, parts);
      else launch_ebe<T, 3, MODE_APPLY, false>(s, op, x, y, b, Dinv, omega, done, parts);
    } else if (mode == MODE_RESID) {
      launch_ebe<T, 3, MODE_RESID, false>(s, op, x, y, b, Dinv, omega, done, parts);
    } else if (mode == MODE_RESID0) {
      // hex8: the first sweep as its own pass, then the residual
      jacobi0<T>(s, 3, nodes_of(op), Dinv, b, const_cast<T*>(x), omega, done);
      launch_ebe<T, 3, MODE_RESID, false>(s, op, x, y, b, Dinv, omega, done, parts);
    } else {
      launch_ebe<T, 3, MODE_JACOBI, false>(s, op, x, y, b, Dinv, omega, done, parts);
    }
  }
}
template void ebe_op<float>(cudaStream_t, int, const Ebe&, const float*, float*, const float*,
                            const float*, double, const int*, double*, const ChebArg*);
template void ebe_op<double>(cudaStream_t, int, const Ebe&, const double*, double*, const double*,
                             const double*, double, const int*, double*, const ChebArg*);

void ebe_block_diag_inv(cudaStream_t s, const Ebe& op, double* Dinv64, float* Dinv32) {
  const int64_t nn = nodes_of(op);
  if (op.dim == 2)
    LAUNCH(k_ebe_diag<2>, ceil_div(nn, 128), 128, 0, s, op.nx, op.ny, op.nz,
           (const double*)op.Ke, (const double*)op.E, op.mask, Dinv64, Dinv32);
  else
    LAUNCH(k_ebe_diag<3>, ceil_div(nn, 128), 128, 0, s, op.nx, op.ny, op.nz,
           (const double*)op.Ke, (const double*)op.E, op.mask, Dinv64, Dinv32);
}

void ebe_assemble_stencil(cudaStream_t s, const Ebe& op, double* S) {
  const int64_t nn = nodes_of(op);
  if (op.dim == 2)
    LAUNCH(k_ebe_stencil<2>, ceil_div(nn, 128), 128, 0, s, op.nx, op.ny, op.nz,
           (const double*)op.Ke, (const double*)op.E, op.mask, S);
  else
    LAUNCH(k_ebe_stencil<3>, ceil_div(nn, 128), 128, 0, s, op.nx, op.ny, op.nz,
           (const double*)op.Ke, (const double*)op.E, op.mask, S);
}

void simp_moduli(cudaStream_t s, int64_t nel, const double* rho, double E0, double Emin,
                 double penal, double* E64, float* E32, int* bad) {
  LAUNCH(k_simp, ceil_div(nel, 256), 256, 0, s, nel, rho, E0, Emin, penal, E64, E32, bad);
}

}  // namespace tomg
