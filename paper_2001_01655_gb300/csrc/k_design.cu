// The steps on either side of the solve in a design iteration (Sec. 2.1): the linear density
// filter rho = S alpha (Eq. 1; radius 1.5 element sizes in Sec. 4), its transpose for the
// chain rule, and the compliance sensitivities of Eq. 3, all in FP64.
//
// Filter: w_ej = max(0, r - |c_e - c_j|) between element centroids; S_ej = w_ej / W_e with the
// row sum W_e over the in-grid neighbours.  w is symmetric, so both S and S^T are one gather
// over the integer offsets inside the radius:  out_i = post_i sum_k w_ik pre_k in_k  with
// (pre, post) = (1, 1/W) for S and (1/W, 1) for S^T.  The offsets and weights are computed on
// the host and passed by value.
#include <cmath>

#include "ops.h"

namespace tomg {

namespace {

constexpr int MAX_OFFS = 128;  // offsets with w > 0 for radius <= 3 in 3D: 123

struct FilterOffsets {
  int n;
  int ox[MAX_OFFS], oy[MAX_OFFS], oz[MAX_OFFS];
  double w[MAX_OFFS];
};

FilterOffsets make_offsets(int dim, double radius) {
  FilterOffsets f{};
  const int reach = (int)std::ceil(radius);
  for (int z = (dim == 3 ? -reach : 0); z <= (dim == 3 ? reach : 0); z++)
    for (int y = -reach; y <= reach; y++)
      for (int x = -reach; x <= reach; x++) {
        const double w = radius - std::sqrt((double)(x * x + y * y + z * z));
        if (w <= 0.0) continue;
        if (f.n >= MAX_OFFS) TOMG_THROW(TOMG_E_INVALID, "filter radius %g too large", radius);
        f.ox[f.n] = x; f.oy[f.n] = y; f.oz[f.n] = z; f.w[f.n] = w;
        f.n++;
      }
  return f;
}

__device__ __forceinline__ void elem_ijk(int64_t e, int nx, int ny, int& i, int& j, int& k) {
  i = (int)(e % nx);
  const int64_t r = e / nx;
  j = (int)(r % ny);
  k = (int)(r / ny);
}

// W_e: sum of the weights of the in-grid neighbours of every element
__global__ void k_filter_rowsum(int nx, int ny, int nz, const FilterOffsets F, double* W) {
  const int64_t nel = (int64_t)nx * ny * nz;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  int i, j, k;
  elem_ijk(e, nx, ny, i, j, k);
  double s = 0.0;
  for (int q = 0; q < F.n; q++) {
    const int a = i + F.ox[q], b = j + F.oy[q], c = k + F.oz[q];
    if (a >= 0 && a < nx && b >= 0 && b < ny && c >= 0 && c < nz) s += F.w[q];
  }
  W[e] = s;
}

// out_e = (transpose ? 1 : 1/W_e) sum_j w_ej (transpose ? in_j / W_j : in_j)
__global__ void k_filter_apply(int nx, int ny, int nz, const FilterOffsets F, int transpose,
                               const double* __restrict__ W, const double* __restrict__ in,
                               double* __restrict__ out) {
  const int64_t nel = (int64_t)nx * ny * nz;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  int i, j, k;
  elem_ijk(e, nx, ny, i, j, k);
  double s = 0.0;
  for (int q = 0; q < F.n; q++) {
    const int a = i + F.ox[q], b = j + F.oy[q], c = k + F.oz[q];
    if (a < 0 || a >= nx || b < 0 || b >= ny || c < 0 || c >= nz) continue;
    const int64_t nb = a + (int64_t)nx * (b + (int64_t)ny * c);
    s += F.w[q] * (transpose ? in[nb] / W[nb] : in[nb]);
  }
  out[e] = transpose ? s : s / W[e];
}

// dF/drho_e = -p rho_e^(p-1) (E0 - Emin) u_e^T Ke u_e (Ke for unit modulus, FP64)
template <int DIM>
__global__ void k_compliance_sens(int nx, int ny, int nz, const double* __restrict__ Ke,
                                  const double* __restrict__ rho, const double* __restrict__ u,
                                  double E0, double Emin, double penal, double* __restrict__ dc) {
  constexpr int NN = 1 << DIM, ND = DIM * NN;
  __shared__ double sKe[ND * ND];
  for (int t = threadIdx.x; t < ND * ND; t += blockDim.x) sKe[t] = Ke[t];
  __syncthreads();
  const int64_t nel = (int64_t)nx * ny * (DIM == 3 ? nz : 1);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  int i, j, k;
  elem_ijk(e, nx, ny, i, j, k);
  double ue[ND];
#pragma unroll
  for (int a = 0; a < NN; a++) {
    const int64_t node = node_id(i + (a & 1), j + ((a >> 1) & 1), DIM == 3 ? k + ((a >> 2) & 1) : 0,
                                 nx, ny);
#pragma unroll
    for (int c = 0; c < DIM; c++) ue[DIM * a + c] = u[DIM * node + c];
  }
  double en = 0.0;
#pragma unroll 4
  for (int r = 0; r < ND; r++) {
    double row = 0.0;
#pragma unroll
    for (int c = 0; c < ND; c++) row += sKe[r * ND + c] * ue[c];
    en += ue[r] * row;
  }
  const double re = rho[e];
  dc[e] = -penal * pow(re, penal - 1.0) * (E0 - Emin) * en;
}

}  // namespace

void density_filter(cudaStream_t s, int dim, int nx, int ny, int nz, double radius, int transpose,
                    const double* in, double* out, double* W) {
  if (!(radius > 0.0) || radius > 3.0)
    TOMG_THROW(TOMG_E_INVALID, "filter radius %g outside (0, 3]", radius);
  const FilterOffsets F = make_offsets(dim, radius);
  const int nzz = dim == 3 ? nz : 1;
  const int64_t nel = (int64_t)nx * ny * nzz;
  LAUNCH(k_filter_rowsum, ceil_div(nel, 256), 256, 0, s, nx, ny, nzz, F, W);
  LAUNCH(k_filter_apply, ceil_div(nel, 256), 256, 0, s, nx, ny, nzz, F, transpose, W, in, out);
}

void compliance_sensitivity(cudaStream_t s, int dim, int nx, int ny, int nz, const double* Ke,
                            const double* rho, const double* u, double E0, double Emin,
                            double penal, double* dc) {
  const int64_t nel = (int64_t)nx * ny * (dim == 3 ? nz : 1);
  if (dim == 2)
    LAUNCH(k_compliance_sens<2>, ceil_div(nel, 128), 128, 0, s, nx, ny, nz, Ke, rho, u, E0, Emin,
           penal, dc);
  else
    LAUNCH(k_compliance_sens<3>, ceil_div(nel, 128), 128, 0, s, nx, ny, nz, Ke, rho, u, E0, Emin,
           penal, dc);
}

}  // namespace tomg
