// Linear buckling (Sec. 2.2, Eq. 4-5): element stresses at the element centres and the
// matrix-free stress stiffness operator K_sigma, in FP64.
//
//   sigma_e = E_sigma(rho_e) (D_0 B(centre)) u_e,  E_sigma = E0 rho^p for rho >= 0.1, else 0
//   K_sigma = -sum_e H_e (x) I_d,   H_e[a, b] = sum_ij S_e,ij L_ij[a, b],
//   L_ij[a, b] = integral over the unit element of dN_a/dx_i dN_b/dx_j
// (S_e the d x d stress tensor; the sign makes compression give positive eigenvalues of
// K_sigma Phi = lambda K Phi).  Fixed DOFs: M K_sigma M.  The apply is node-centric like the
// level-0 stiffness kernel: every node sums the rows of the elements around it (no atomics).
//
// Sensitivities (Eq. 6-9).  With w_e,v(Phi) = sum over the index pairs (i, j) of Voigt component
// v of sum_ab L_ij[a, b] Phi_a . Phi_b, the mode's energy is Phi^T K_sigma Phi =
// -sum_e sum_v sigma_e,v w_e,v, so (K_sigma linear in u) the adjoint right-hand side is
//   g = d(Phi^T K_sigma Phi)/du = -sum_e E_sigma(rho_e) (D_0 B)^T w_e   (masked),
// gathered node by node from per-element Voigt weights.  For a K-normalised mode and the
// adjoint solution v of K v = g:
//   dlambda/drho_e = E_sigma'(rho_e) Phi_e^T K_sigma,e^1 Phi_e - lambda E'(rho_e) Phi_e^T Ke Phi_e
//                    - E'(rho_e) v_e^T Ke u_e,
// and the p-norm F = (sum lambda_i^p)^(1/p) has dF/drho = sum_i c_i dlambda_i/drho with
// c_i = F^(1-p) lambda_i^(p-1) (host scalars).
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

// w_v for one element: Phi_e (masked, node-major) against the gradient products
template <int DIM>
__device__ __forceinline__ void mode_weights(const StabConst<DIM>& C, const double* ph, double* w) {
  constexpr int NN = 1 << DIM, NV = DIM == 3 ? 6 : 3;
  double G[DIM * DIM];
#pragma unroll
  for (int t = 0; t < DIM * DIM; t++) G[t] = 0.0;
#pragma unroll
  for (int a = 0; a < NN; a++)
#pragma unroll
    for (int b = 0; b < NN; b++) {
      double pp = 0.0;
#pragma unroll
      for (int c = 0; c < DIM; c++) pp += ph[DIM * a + c] * ph[DIM * b + c];
#pragma unroll
      for (int t = 0; t < DIM * DIM; t++) G[t] += C.L[(t * NN + a) * NN + b] * pp;
    }
  if (DIM == 2) {
    w[0] = G[0]; w[1] = G[3]; w[2] = G[1] + G[2];
  } else {
    w[0] = G[0]; w[1] = G[4]; w[2] = G[8];
    w[3] = G[5] + G[7]; w[4] = G[2] + G[6]; w[5] = G[1] + G[3];
  }
  (void)NV;
}

// element DOF values of a nodal vector, zero at fixed DOFs
template <int DIM>
__device__ __forceinline__ void gather_masked(int i, int j, int k, int nx, int ny,
                                              const uint8_t* __restrict__ mask,
                                              const double* __restrict__ x, double* xe) {
#pragma unroll
  for (int a = 0; a < (1 << DIM); a++) {
    const int64_t node = node_id(i + (a & 1), j + ((a >> 1) & 1), DIM == 3 ? k + ((a >> 2) & 1) : 0,
                                 nx, ny);
    const unsigned m = mask[node];
#pragma unroll
    for (int c = 0; c < DIM; c++) xe[DIM * a + c] = ((m >> c) & 1u) ? 0.0 : x[DIM * node + c];
  }
}

// per mode (blockIdx.y) and element: the Voigt weights s_e,v = -E_sigma(rho_e) w_e,v(Phi_m)
template <int DIM>
__global__ void k_adjoint_weights(int nx, int ny, int nz, const StabConst<DIM> C,
                                  const double* __restrict__ rho, const uint8_t* __restrict__ mask,
                                  const double* __restrict__ Phi, int64_t ldp, double E0,
                                  double penal, double* __restrict__ sw) {
  constexpr int ND = DIM << DIM, NV = DIM == 3 ? 6 : 3;
  const int64_t nel = (int64_t)nx * ny * (DIM == 3 ? nz : 1);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  const int i = (int)(e % nx);
  const int64_t r = e / nx;
  const int j = (int)(r % ny), k = (int)(r / ny);
  const int m = blockIdx.y;
  double ph[ND], w[NV];
  gather_masked<DIM>(i, j, k, nx, ny, mask, Phi + m * ldp, ph);
  mode_weights<DIM>(C, ph, w);
  const double re = rho[e];
  const double Es = re >= 0.1 ? E0 * pow(re, penal) : 0.0;
  double* o = sw + ((int64_t)m * nel + e) * NV;
#pragma unroll
  for (int v = 0; v < NV; v++) o[v] = -Es * w[v];
}

// per mode (blockIdx.y) and node: g = sum over the adjacent elements of (D_0 B)^T s_e, masked
template <int DIM>
__global__ void __launch_bounds__(128) k_adjoint_gather(int nx, int ny, int nz,
                                                        const StabConst<DIM> C,
                                                        const double* __restrict__ sw,
                                                        const uint8_t* __restrict__ mask,
                                                        double* __restrict__ g, int64_t ldg) {
  constexpr int NN = 1 << DIM, ND = DIM * NN, NV = DIM == 3 ? 6 : 3;
  const int64_t nel = (int64_t)nx * ny * (DIM == 3 ? nz : 1);
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (DIM == 3 ? nz + 1 : 1);
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  const int m = blockIdx.y;
  int i, j, k;
  node_ijk(node, nx, ny, DIM, i, j, k);
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
    const double* sv = sw + ((int64_t)m * nel + el) * NV;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const double x = sv[v];
#pragma unroll
      for (int c = 0; c < DIM; c++) acc[c] += C.DB[v * ND + DIM * a + c] * x;
    }
  }
  const unsigned mi = mask[node];
#pragma unroll
  for (int c = 0; c < DIM; c++) g[m * ldg + DIM * node + c] = ((mi >> c) & 1u) ? 0.0 : acc[c];
}

constexpr int MAX_SENS_MODES = 16;
struct SensScalars {
  double lam[MAX_SENS_MODES], coef[MAX_SENS_MODES];
};

// per element: dlambda_m/drho_e for every mode (optional output) and sum_m coef_m dlambda_m
template <int DIM>
__global__ void __launch_bounds__(128) k_eig_sens(int nx, int ny, int nz, const StabConst<DIM> C,
                                                  const double* __restrict__ Ke,
                                                  const double* __restrict__ rho,
                                                  const uint8_t* __restrict__ mask,
                                                  const double* __restrict__ u,
                                                  const double* __restrict__ Phi,
                                                  const double* __restrict__ Vadj, int64_t ld,
                                                  int nm, const SensScalars S, double E0,
                                                  double Emin, double penal,
                                                  double* __restrict__ dlam,
                                                  double* __restrict__ dF) {
  constexpr int ND = DIM << DIM, NV = DIM == 3 ? 6 : 3;
  __shared__ double sKe[ND * ND];
  for (int t = threadIdx.x; t < ND * ND; t += blockDim.x) sKe[t] = Ke[t];
  __syncthreads();
  const int64_t nel = (int64_t)nx * ny * (DIM == 3 ? nz : 1);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  const int i = (int)(e % nx);
  const int64_t r = e / nx;
  const int j = (int)(r % ny), k = (int)(r / ny);
  double ue[ND], Ku[ND], s1[NV];
  gather_masked<DIM>(i, j, k, nx, ny, mask, u, ue);
#pragma unroll
  for (int v = 0; v < NV; v++) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < ND; q++) t += C.DB[v * ND + q] * ue[q];
    s1[v] = t;
  }
#pragma unroll 4
  for (int a = 0; a < ND; a++) {
    double t = 0.0;
#pragma unroll
    for (int b = 0; b < ND; b++) t += sKe[a * ND + b] * ue[b];
    Ku[a] = t;
  }
  const double re = rho[e];
  const double dE = penal * pow(re, penal - 1.0) * (E0 - Emin);
  const double dEs = re >= 0.1 ? penal * E0 * pow(re, penal - 1.0) : 0.0;
  double tot = 0.0;
  for (int m = 0; m < nm; m++) {
    double pe[ND], w[NV];
    gather_masked<DIM>(i, j, k, nx, ny, mask, Phi + m * ld, pe);
    mode_weights<DIM>(C, pe, w);
    double geo = 0.0;
#pragma unroll
    for (int v = 0; v < NV; v++) geo -= s1[v] * w[v];
    double pKp = 0.0;
#pragma unroll 4
    for (int a = 0; a < ND; a++) {
      double t = 0.0;
#pragma unroll
      for (int b = 0; b < ND; b++) t += sKe[a * ND + b] * pe[b];
      pKp += pe[a] * t;
    }
    double ve[ND];
    gather_masked<DIM>(i, j, k, nx, ny, mask, Vadj + m * ld, ve);
    double vKu = 0.0;
#pragma unroll
    for (int a = 0; a < ND; a++) vKu += ve[a] * Ku[a];
    const double d = dEs * geo - S.lam[m] * dE * pKp - dE * vKu;
    if (dlam) dlam[m * nel + e] = d;
    tot += S.coef[m] * d;
  }
  if (dF) dF[e] = tot;
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

void buckling_adjoint_rhs(cudaStream_t s, int dim, int nx, int ny, int nz, double nu, double E0,
                          double penal, const double* rho, const uint8_t* mask, int nm,
                          const double* Phi, int64_t ldp, double* sw, double* g, int64_t ldg) {
  const int64_t nel = (int64_t)nx * ny * (dim == 3 ? nz : 1);
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (dim == 3 ? nz + 1 : 1);
  const dim3 ge((unsigned)ceil_div(nel, 128), (unsigned)nm), gn((unsigned)ceil_div(nn, 128), (unsigned)nm);
  if (dim == 2) {
    const StabConst<2> C = make_const<2>(nu);
    LAUNCH(k_adjoint_weights<2>, ge, 128, 0, s, nx, ny, nz, C, rho, mask, Phi, ldp, E0, penal, sw);
    LAUNCH(k_adjoint_gather<2>, gn, 128, 0, s, nx, ny, nz, C, sw, mask, g, ldg);
  } else {
    const StabConst<3> C = make_const<3>(nu);
    LAUNCH(k_adjoint_weights<3>, ge, 128, 0, s, nx, ny, nz, C, rho, mask, Phi, ldp, E0, penal, sw);
    LAUNCH(k_adjoint_gather<3>, gn, 128, 0, s, nx, ny, nz, C, sw, mask, g, ldg);
  }
}

void buckling_sensitivity(cudaStream_t s, int dim, int nx, int ny, int nz, double nu, double E0,
                          double Emin, double penal, const double* Ke, const double* rho,
                          const uint8_t* mask, const double* u, int nm, const double* lam,
                          const double* coef, const double* Phi, const double* Vadj, int64_t ld,
                          double* dlam, double* dF) {
  if (nm < 1 || nm > MAX_SENS_MODES) TOMG_THROW(TOMG_E_INVALID, "1 <= n_modes <= 16");
  SensScalars S{};
  for (int m = 0; m < nm; m++) { S.lam[m] = lam[m]; S.coef[m] = coef[m]; }
  const int64_t nel = (int64_t)nx * ny * (dim == 3 ? nz : 1);
  if (dim == 2)
    LAUNCH(k_eig_sens<2>, ceil_div(nel, 128), 128, 0, s, nx, ny, nz, make_const<2>(nu), Ke, rho,
           mask, u, Phi, Vadj, ld, nm, S, E0, Emin, penal, dlam, dF);
  else
    LAUNCH(k_eig_sens<3>, ceil_div(nel, 128), 128, 0, s, nx, ny, nz, make_const<3>(nu), Ke, rho,
           mask, u, Phi, Vadj, ld, nm, S, E0, Emin, penal, dlam, dF);
}

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
