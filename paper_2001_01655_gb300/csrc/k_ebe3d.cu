// Level-0 SIMP element operator on hex8 grids in FP32 (Sec. 2.1 Eq. 2, Sec. 3.1), tiled.
//
// One block covers 32 x 4 x 4 nodes with 32 x 4 threads, each thread owning a column of four
// nodes along z.  The block stages the masked displacements of the tile plus a one-node halo
// and the moduli of the 33 x 5 x 5 surrounding elements in shared memory (out-of-grid elements
// read as E = 0), all loads issued before the first shared-memory store.  Each thread then
// walks the eight element roles: it loads the three Ke rows of that role (72 values) once into
// registers and applies them to its four nodes, so Ke traffic is amortised over the column.
#include "ops.h"

namespace tomg {

namespace {

constexpr int BX = 32, BY = 4, TZ = 4;
constexpr int SXX = BX + 2, SXY = BY + 2, SXZ = TZ + 2;  // node tile with halo
constexpr int SEX = BX + 1, SEY = BY + 1, SEZ = TZ + 1;  // element tile
constexpr int NTH = BX * BY;

template <int MODE>
__global__ void __launch_bounds__(NTH) k_ebe3(int nx, int ny, int nz, const float* __restrict__ Ke,
                                              const float* __restrict__ E,
                                              const uint8_t* __restrict__ mask,
                                              const float* __restrict__ x, float* __restrict__ y,
                                              const float* __restrict__ b,
                                              const float* __restrict__ Dinv, float omega,
                                              const int* done, float* __restrict__ dch, float c1,
                                              int dmode) {
  __shared__ __align__(16) float sKe[576];
  __shared__ float sx[SXZ][SXY][SXX][3];
  __shared__ float sE[SEZ][SEY][SEX];
  pdl_prologue();
  if (solve_done(done)) return;
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY, k0 = blockIdx.z * TZ;
  const int W = nx + 1, H = ny + 1;
  for (int t = tid; t < 576; t += NTH) sKe[t] = Ke[t];
  constexpr int NX = SXX * SXY * SXZ, NE = SEX * SEY * SEZ;
  constexpr int NXL = (NX + NTH - 1) / NTH, NEL = (NE + NTH - 1) / NTH;
  float xv[NXL][3];
  unsigned mv[NXL];
  float ev[NEL];
#pragma unroll
  for (int q = 0; q < NXL; q++) {
    const int t = tid + q * NTH;
    const int lx = t % SXX, ly = (t / SXX) % SXY, lz = t / (SXX * SXY);
    const int gi = i0 - 1 + lx, gj = j0 - 1 + ly, gk = k0 - 1 + lz;
    xv[q][0] = xv[q][1] = xv[q][2] = 0.f;
    mv[q] = 7u;
    if (t < NX && gi >= 0 && gi <= nx && gj >= 0 && gj <= ny && gk >= 0 && gk <= nz) {
      const int64_t node = gi + (int64_t)W * (gj + (int64_t)H * gk);
      mv[q] = __ldg(mask + node);
      xv[q][0] = __ldg(x + 3 * node);
      xv[q][1] = __ldg(x + 3 * node + 1);
      xv[q][2] = __ldg(x + 3 * node + 2);
    }
  }
#pragma unroll
  for (int q = 0; q < NEL; q++) {
    const int t = tid + q * NTH;
    const int lx = t % SEX, ly = (t / SEX) % SEY, lz = t / (SEX * SEY);
    const int ge = i0 - 1 + lx, gf = j0 - 1 + ly, gg = k0 - 1 + lz;
    ev[q] = (t < NE && ge >= 0 && ge < nx && gf >= 0 && gf < ny && gg >= 0 && gg < nz)
                ? __ldg(E + ge + (int64_t)nx * (gf + (int64_t)ny * gg)) : 0.f;
  }
#pragma unroll
  for (int q = 0; q < NXL; q++) {
    const int t = tid + q * NTH;
    if (t < NX) {
      const int lx = t % SXX, ly = (t / SXX) % SXY, lz = t / (SXX * SXY);
#pragma unroll
      for (int c = 0; c < 3; c++) sx[lz][ly][lx][c] = ((mv[q] >> c) & 1u) ? 0.f : xv[q][c];
    }
  }
#pragma unroll
  for (int q = 0; q < NEL; q++) {
    const int t = tid + q * NTH;
    if (t < NE) {
      const int lx = t % SEX, ly = (t / SEX) % SEY, lz = t / (SEX * SEY);
      sE[lz][ly][lx] = ev[q];
    }
  }
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y;
  float acc[TZ][3];
#pragma unroll
  for (int q = 0; q < TZ; q++) acc[q][0] = acc[q][1] = acc[q][2] = 0.f;
#pragma unroll 1
  for (int e = 0; e < 8; e++) {
    // element (i-1+ex, j-1+ey, k-1+ez) around the node; the node is its local node a
    const int ex = e & 1, ey = (e >> 1) & 1, ez = (e >> 2) & 1;
    const int a = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
    float kr[3][24];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int c = 0; c < 24; c += 4) {
        const float4 v = *reinterpret_cast<const float4*>(sKe + (3 * a + r) * 24 + c);
        kr[r][c] = v.x; kr[r][c + 1] = v.y; kr[r][c + 2] = v.z; kr[r][c + 3] = v.w;
      }
#pragma unroll
    for (int q = 0; q < TZ; q++) {
      float p0 = 0.f, p1 = 0.f, p2 = 0.f;
#pragma unroll
      for (int bn = 0; bn < 8; bn++) {
        const float* xn = sx[q + ez + ((bn >> 2) & 1)][ty + ey + ((bn >> 1) & 1)][tx + ex + (bn & 1)];
        const float u0 = xn[0], u1 = xn[1], u2 = xn[2];
        p0 += kr[0][3 * bn] * u0 + kr[0][3 * bn + 1] * u1 + kr[0][3 * bn + 2] * u2;
        p1 += kr[1][3 * bn] * u0 + kr[1][3 * bn + 1] * u1 + kr[1][3 * bn + 2] * u2;
        p2 += kr[2][3 * bn] * u0 + kr[2][3 * bn + 1] * u1 + kr[2][3 * bn + 2] * u2;
      }
      const float Ee = sE[q + ez][ty + ey][tx + ex];
      acc[q][0] += Ee * p0;
      acc[q][1] += Ee * p1;
      acc[q][2] += Ee * p2;
    }
  }
  const int i = i0 + tx, j = j0 + ty;
  if (i > nx || j > ny) return;
#pragma unroll
  for (int q = 0; q < TZ; q++) {
    const int k = k0 + q;
    if (k > nz) continue;
    const int64_t node = i + (int64_t)W * (j + (int64_t)H * k);
    const unsigned m = mask[node];
    float xi[3], Ax[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      xi[c] = x[3 * node + c];
      Ax[c] = ((m >> c) & 1u) ? xi[c] : acc[q][c];
    }
    if (MODE == MODE_APPLY) {
#pragma unroll
      for (int c = 0; c < 3; c++) y[3 * node + c] = Ax[c];
    } else {
      float r[3];
#pragma unroll
      for (int c = 0; c < 3; c++) r[c] = b[3 * node + c] - Ax[c];
      if (MODE == MODE_RESID) {
#pragma unroll
        for (int c = 0; c < 3; c++) y[3 * node + c] = r[c];
      } else if (MODE == MODE_CHEB) {
        cheb_node<float, 3>(node, r, xi, Dinv, c1, omega, dmode, dch, y);
      } else {
        const float* D = Dinv + 9 * node;
#pragma unroll
        for (int c = 0; c < 3; c++)
          y[3 * node + c] = xi[c] + omega * (D[3 * c] * r[0] + D[3 * c + 1] * r[1] + D[3 * c + 2] * r[2]);
      }
    }
  }
}

}  // namespace

void ebe3d_launch(cudaStream_t s, int mode, const Ebe& op, const float* x, float* y,
                  const float* b, const float* Dinv, double omega, const int* done,
                  const ChebArg* ch) {
  dim3 grid(ceil_div(op.nx + 1, BX), ceil_div(op.ny + 1, BY), ceil_div(op.nz + 1, TZ));
  dim3 block(BX, BY);
  const float* Ke = (const float*)op.Ke;
  const float* E = (const float*)op.E;
  if (mode == MODE_CHEB && !ch) TOMG_THROW(TOMG_E_INVALID, "Chebyshev step without its state");
  float* dch = mode == MODE_CHEB ? (float*)ch->d : nullptr;
  const float c1 = mode == MODE_CHEB ? (float)ch->c1 : 0.f;
  const int dm = mode == MODE_CHEB ? ch->dmode : 0;
#define E3(M) LAUNCH(k_ebe3<M>, grid, block, 0, s, op.nx, op.ny, op.nz, Ke, E, op.mask, x, y, b, \
                     Dinv, (float)omega, done, dch, c1, dm)
  if (mode == MODE_APPLY) E3(MODE_APPLY);
  else if (mode == MODE_RESID) E3(MODE_RESID);
  else if (mode == MODE_CHEB) E3(MODE_CHEB);
  else E3(MODE_JACOBI);
#undef E3
}

}  // namespace tomg
