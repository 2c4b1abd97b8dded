// Linear buckling (Sec. 2.2, Eq. 4-5): element stresses at the element centres and the
// matrix-free stress stiffness operator K_sigma, in FP64.
//
//   sigma_e = E_sigma(rho_e) (D_0 B(centre)) u_e,  E_sigma = E0 rho^p for rho >= 0.1, else 0
//   K_sigma = -sum_e H_e (x) I_d,   H_e[a, b] = sum_ij S_e,ij L_ij[a, b],
//   L_ij[a, b] = integral over the unit element of dN_a/dx_i dN_b/dx_j
// (S_e the d x d stress tensor; the sign makes compression give positive eigenvalues of
// K_sigma Phi = lambda K Phi).  Fixed DOFs: M K_sigma M.  The apply is node-centric like the
// level-0 stiffness kernel: every node sums the rows of the elements around it (no atomics).
#include "ops.h"

namespace tomg {

namespace {

template <int DIM>
struct StabConst {
  double DB[(DIM == 3 ? 6 : 3) * DIM * (1 << DIM)];  // D_0 B(centre), Voigt rows x element DOFs
  double L[DIM * DIM * (1 << DIM) * (1 << DIM)];     // L_ij[a][b] at ((i * DIM + j) * NN + a) * NN + b
};

template <int DIM>
__global__ void k_stress(int nx, int ny, int nz, const StabConst<DIM> C,
                         const double* __restrict__ rho, const double* __restrict__ u, double E0,
                         double penal, double* __restrict__ sig) {
  constexpr int NN = 1 << DIM, ND = DIM * NN, NV = DIM == 3 ? 6 : 3;
  const int64_t nel = (int64_t)nx * ny * (DIM == 3 ? nz : 1);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  const int i = (int)(e % nx);
  const int64_t r = e / nx;
  const int j = (int)(r % ny), k = (int)(r / ny);
  double ue[ND];
#pragma unroll
  for (int a = 0; a < NN; a++) {
    const int64_t node = node_id(i + (a & 1), j + ((a >> 1) & 1), DIM == 3 ? k + ((a >> 2) & 1) : 0,
                                 nx, ny);
#pragma unroll
    for (int c = 0; c < DIM; c++) ue[DIM * a + c] = u[DIM * node + c];
  }
  const double re = rho[e];
  const double Es = re >= 0.1 ? E0 * pow(re, penal) : 0.0;
#pragma unroll
  for (int v = 0; v < NV; v++) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < ND; q++) s += C.DB[v * ND + q] * ue[q];
    sig[(int64_t)NV * e + v] = Es * s;
  }
}

// stress tensor entry (i, j) from the Voigt vector: 2D [xx, yy, xy]; 3D [xx, yy, zz, yz, xz, xy]
template <int DIM>
__device__ __forceinline__ double s_ij(const double* sv, int i, int j) {
  if (DIM == 2) return i == j ? sv[i] : sv[2];
  if (i == j) return sv[i];
  const int m = i + j;  // (1,2) -> yz, (0,2) -> xz, (0,1) -> xy
  return m == 3 ? sv[3] : (m == 2 ? sv[4] : sv[5]);
}

template <int DIM>
__global__ void __launch_bounds__(128) k_ksigma_apply(int nx, int ny, int nz,
                                                      const StabConst<DIM> C,
                                                      const double* __restrict__ sig,
                                                      const uint8_t* __restrict__ mask,
                                                      const double* __restrict__ x,
                                                      double* __restrict__ y) {
  constexpr int NN = 1 << DIM, NV = DIM == 3 ? 6 : 3;
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (DIM == 3 ? nz + 1 : 1);
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  int i, j, k;
  node_ijk(node, nx, ny, DIM, i, j, k);
  const unsigned mi = mask[node];
  double acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; c++) acc[c] = 0.0;
#pragma unroll
  for (int e = 0; e < NN; e++) {
    const int ex = e & 1, ey = (e >> 1) & 1, ez = (e >> 2) & 1;
    const int ie = i - 1 + ex, je = j - 1 + ey, ke = DIM == 3 ? k - 1 + ez : 0;
    if (ie < 0 || ie >= nx || je < 0 || je >= ny) continue;
    if (DIM == 3 && (ke < 0 || ke >= nz)) continue;
    const int a = (1 - ex) + 2 * (1 - ey) + (DIM == 3 ? 4 * (1 - ez) : 0);
    const int64_t el = ie + (int64_t)nx * (je + (int64_t)ny * ke);
    double sv[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) sv[v] = sig[(int64_t)NV * el + v];
#pragma unroll
    for (int b = 0; b < NN; b++) {
      double h = 0.0;
#pragma unroll
      for (int p = 0; p < DIM; p++)
#pragma unroll
        for (int q = 0; q < DIM; q++) h += s_ij<DIM>(sv, p, q) * C.L[((p * DIM + q) * NN + a) * NN + b];
      const int64_t nb = node_id(ie + (b & 1), je + ((b >> 1) & 1), DIM == 3 ? ke + ((b >> 2) & 1) : 0,
                                 nx, ny);
      const unsigned mb = mask[nb];
#pragma unroll
      for (int c = 0; c < DIM; c++)
        if (!((mb >> c) & 1u)) acc[c] -= h * x[DIM * nb + c];
    }
  }
#pragma unroll
  for (int c = 0; c < DIM; c++) y[DIM * node + c] = ((mi >> c) & 1u) ? 0.0 : acc[c];
}

// shape-function gradients on [0,1]^DIM at xi (2^DIM x DIM)
template <int DIM>
void shape_grad_host(const double* xi, double* G) {
  for (int a = 0; a < (1 << DIM); a++)
    for (int kk = 0; kk < DIM; kk++) {
      double g = ((a >> kk) & 1) ? 1.0 : -1.0;
      for (int m = 0; m < DIM; m++)
        if (m != kk) g *= ((a >> m) & 1) ? xi[m] : 1.0 - xi[m];
      G[a * DIM + kk] = g;
    }
}

template <int DIM>
StabConst<DIM> make_const(double nu) {
  constexpr int NN = 1 << DIM, ND = DIM * NN, NV = DIM == 3 ? 6 : 3;
  StabConst<DIM> C{};
  // D_0 (unit modulus) and B at the centre
  double D[NV * NV] = {};
  if (DIM == 2) {
    const double c = 1.0 / (1.0 - nu * nu);
    D[0] = c; D[1] = c * nu; D[3] = c * nu; D[4] = c; D[8] = c * 0.5 * (1.0 - nu);
  } else {
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));
    for (int p = 0; p < 3; p++)
      for (int q = 0; q < 3; q++) D[p * NV + q] = lam + (p == q ? 2.0 * mu : 0.0);
    for (int p = 3; p < 6; p++) D[p * NV + p] = mu;
  }
  double xc[DIM], G[NN * DIM];
  for (int m = 0; m < DIM; m++) xc[m] = 0.5;
  shape_grad_host<DIM>(xc, G);
  double B[NV * ND] = {};
  for (int a = 0; a < NN; a++) {
    const double* g = G + a * DIM;
    if (DIM == 2) {
      B[0 * ND + 2 * a] = g[0];
      B[1 * ND + 2 * a + 1] = g[1];
      B[2 * ND + 2 * a] = g[1];
      B[2 * ND + 2 * a + 1] = g[0];
    } else {
      const int c = 3 * a;
      B[0 * ND + c] = g[0];
      B[1 * ND + c + 1] = g[1];
      B[2 * ND + c + 2] = g[2];
      B[3 * ND + c + 1] = g[2]; B[3 * ND + c + 2] = g[1];
      B[4 * ND + c] = g[2]; B[4 * ND + c + 2] = g[0];
      B[5 * ND + c] = g[1]; B[5 * ND + c + 1] = g[0];
    }
  }
  for (int v = 0; v < NV; v++)
    for (int q = 0; q < ND; q++) {
      double s = 0.0;
      for (int w = 0; w < NV; w++) s += D[v * NV + w] * B[w * ND + q];
      C.DB[v * ND + q] = s;
    }
  // L_ij by the 2x2(x2) Gauss rule (exact for these integrands)
  const double gp[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
  const double w = std::pow(0.5, DIM);
  for (int p = 0; p < (1 << DIM); p++) {
    double xi[DIM];
    for (int m = 0; m < DIM; m++) xi[m] = gp[(p >> m) & 1];
    shape_grad_host<DIM>(xi, G);
    for (int ii = 0; ii < DIM; ii++)
      for (int jj = 0; jj < DIM; jj++)
        for (int a = 0; a < NN; a++)
          for (int b = 0; b < NN; b++)
            C.L[((ii * DIM + jj) * NN + a) * NN + b] += w * G[a * DIM + ii] * G[b * DIM + jj];
  }
  return C;
}

}  // namespace

int stress_components(int dim) { return dim == 3 ? 6 : 3; }

void element_stresses(cudaStream_t s, int dim, int nx, int ny, int nz, double nu, double E0,
                      double penal, const double* rho, const double* u, double* sig) {
  const int64_t nel = (int64_t)nx * ny * (dim == 3 ? nz : 1);
  if (dim == 2)
    LAUNCH(k_stress<2>, ceil_div(nel, 128), 128, 0, s, nx, ny, nz, make_const<2>(nu), rho, u, E0,
           penal, sig);
  else
    LAUNCH(k_stress<3>, ceil_div(nel, 128), 128, 0, s, nx, ny, nz, make_const<3>(nu), rho, u, E0,
           penal, sig);
}

void stress_stiffness_apply(cudaStream_t s, int dim, int nx, int ny, int nz, double nu,
                            const double* sig, const uint8_t* mask, const double* x, double* y) {
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (dim == 3 ? nz + 1 : 1);
  if (dim == 2)
    LAUNCH(k_ksigma_apply<2>, ceil_div(nn, 128), 128, 0, s, nx, ny, nz, make_const<2>(nu), sig,
           mask, x, y);
  else
    LAUNCH(k_ksigma_apply<3>, ceil_div(nn, 128), 128, 0, s, nx, ny, nz, make_const<3>(nu), sig,
           mask, x, y);
}

}  // namespace tomg
