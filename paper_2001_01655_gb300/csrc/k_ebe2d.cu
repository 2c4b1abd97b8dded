// Level-0 SIMP element operator on quad4 grids (Sec. 2.1 Eq. 2, Sec. 3.1), tiled for sm_103a.
//
// One block covers a 32 x 32 tile of nodes with 32 x 8 threads; each thread owns a column of
// four nodes.  The block stages the masked displacements of the tile plus a one-node halo
// (coalesced 8/16-byte vector loads) and the moduli of the 33 x 33 surrounding elements in
// shared memory (out-of-grid elements read as E = 0, so the gather has no branches).  Each
// thread then keeps a 6 x 3 node window and a 5 x 2 element window in registers, loads each of
// the four element-role row pairs of Ke once, and applies it to its four nodes:
// 64 FMAs per node, every input element read once from DRAM.
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "ops.h"

namespace tomg {

namespace {

constexpr int BX = 32, BY = 8;

// Ke by value: a kernel parameter lives in the constant bank, and with the element and node
// loops unrolled every Ke entry is a compile-time constant-bank operand of its FMA (no loads)
template <class T> struct KeP2 { T v[64]; };

template <class T> struct V2t;
template <> struct V2t<float> { using type = float2; };
template <> struct V2t<double> { using type = double2; };

// NPT nodes per thread along y (tile 32 x 8 NPT): more nodes per thread reuse more of the
// staged halo, fewer give more blocks per SM; the setup's autotuner picks per grid
template <class T, int MODE, bool DOT, int NPT>
__global__ void __launch_bounds__(BX * BY) k_ebe2(int nx, int ny, const KeP2<T> K,
                                                  const T* __restrict__ E,
                                                  const uint8_t* __restrict__ mask,
                                                  const T* __restrict__ x, T* __restrict__ y,
                                                  const T* __restrict__ b,
                                                  const T* __restrict__ Dinv, T omega,
                                                  const int* done, double* partials,
                                                  T* __restrict__ xo, T c1, int dmode, T w0) {
  using V2 = typename V2t<T>::type;
  constexpr int TH = BY * NPT;
  __shared__ V2 sx[TH + 2][BX + 2];
  __shared__ T sE[TH + 1][BX + 1];
  __shared__ double red[BX * BY / 32];
  pdl_launch();
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int i0 = blockIdx.x * BX, j0 = blockIdx.y * TH;
  const int W = nx + 1;
  // staging: issue every global load of this thread first (independent, all in flight at
  // once), then write shared memory, so the tile costs one memory latency, not several.  The
  // mask and the moduli are fixed during a solve and are fetched before the wait for the
  // producer of x (b and the smoother blocks for the fused first sweep).
  constexpr int NXL = ((TH + 2) * (BX + 2) + BX * BY - 1) / (BX * BY);
  constexpr int NEL = ((TH + 1) * (BX + 1) + BX * BY - 1) / (BX * BY);
  V2 xv[NXL];
  unsigned mv[NXL];
  T evv[NEL];
#pragma unroll
  for (int k = 0; k < NXL; k++) {
    const int t = tid + k * BX * BY;
    const int ly = t / (BX + 2), lx = t - ly * (BX + 2);
    const int gi = i0 - 1 + lx, gj = j0 - 1 + ly;
    mv[k] = 3u | 4u;  // bit 2: outside the tile or the grid
    if (t < (TH + 2) * (BX + 2) && gi >= 0 && gi <= nx && gj >= 0 && gj <= ny)
      mv[k] = __ldg(mask + gj * W + gi);
  }
#pragma unroll
  for (int k = 0; k < NEL; k++) {
    const int t = tid + k * BX * BY;
    const int ly = t / (BX + 1), lx = t - ly * (BX + 1);
    const int ge = i0 - 1 + lx, gf = j0 - 1 + ly;
    evv[k] = (t < (TH + 1) * (BX + 1) && ge >= 0 && ge < nx && gf >= 0 && gf < ny)
                 ? __ldg(E + gf * nx + ge) : T(0);
  }
  pdl_wait();
  if (solve_done(done)) return;
#pragma unroll
  for (int k = 0; k < NXL; k++) {
    const int t = tid + k * BX * BY;
    const int ly = t / (BX + 2), lx = t - ly * (BX + 2);
    const int node = (j0 - 1 + ly) * W + i0 - 1 + lx;
    xv[k].x = T(0);
    xv[k].y = T(0);
    if (!(mv[k] & 4u)) {
      if (MODE == MODE_RESID0 || MODE == MODE_CHEB0) {
        // x = w Dinv b of the first sweep, formed where it is needed
        const T wf = MODE == MODE_CHEB0 ? w0 : omega;
        const V2 bv = reinterpret_cast<const V2*>(b)[node];
        const V2 d01 = __ldg(reinterpret_cast<const V2*>(Dinv) + 2 * node);
        const V2 d23 = __ldg(reinterpret_cast<const V2*>(Dinv) + 2 * node + 1);
        xv[k].x = wf * (d01.x * bv.x + d01.y * bv.y);
        xv[k].y = wf * (d23.x * bv.x + d23.y * bv.y);
      } else {
        xv[k] = reinterpret_cast<const V2*>(x)[node];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NXL; k++) {
    const int t = tid + k * BX * BY;
    if (t < (TH + 2) * (BX + 2)) {
      const int ly = t / (BX + 2), lx = t - ly * (BX + 2);
      V2 v;
      v.x = (mv[k] & 1u) ? T(0) : xv[k].x;
      v.y = (mv[k] & 2u) ? T(0) : xv[k].y;
      sx[ly][lx] = v;
    }
  }
#pragma unroll
  for (int k = 0; k < NEL; k++) {
    const int t = tid + k * BX * BY;
    if (t < (TH + 1) * (BX + 1)) {
      const int ly = t / (BX + 1), lx = t - ly * (BX + 1);
      sE[ly][lx] = evv[k];
    }
  }
  __syncthreads();
  const int tx = threadIdx.x, r0 = threadIdx.y * NPT;
  V2 xw[NPT + 2][3];
  T ew[NPT + 1][2];
#pragma unroll
  for (int rr = 0; rr < NPT + 2; rr++)
#pragma unroll
    for (int cc = 0; cc < 3; cc++) xw[rr][cc] = sx[r0 + rr][tx + cc];
#pragma unroll
  for (int rr = 0; rr < NPT + 1; rr++)
#pragma unroll
    for (int cc = 0; cc < 2; cc++) ew[rr][cc] = sE[r0 + rr][tx + cc];
  T a0[NPT], a1[NPT];
#pragma unroll
  for (int q = 0; q < NPT; q++) a0[q] = a1[q] = T(0);
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const int ex = e & 1, ey = e >> 1;
    const int a = (1 - ex) + 2 * (1 - ey);
    T k0[8], k1[8];
#pragma unroll
    for (int t = 0; t < 8; t++) {
      k0[t] = K.v[(2 * a) * 8 + t];
      k1[t] = K.v[(2 * a + 1) * 8 + t];
    }
#pragma unroll
    for (int q = 0; q < NPT; q++) {
      T p0 = T(0), p1 = T(0);
#pragma unroll
      for (int bn = 0; bn < 4; bn++) {
        const V2 xv = xw[q + ey + (bn >> 1)][ex + (bn & 1)];
        p0 += k0[2 * bn] * xv.x + k0[2 * bn + 1] * xv.y;
        p1 += k1[2 * bn] * xv.x + k1[2 * bn + 1] * xv.y;
      }
      const T Ee = ew[q + ey][ex];
      a0[q] += Ee * p0;
      a1[q] += Ee * p1;
    }
  }
  double dotv = 0.0;
  const int i = i0 + tx;
#pragma unroll
  for (int q = 0; q < NPT; q++) {
    const int j = j0 + r0 + q;
    if (i > nx || j > ny) continue;
    const int node = j * W + i;
    const unsigned m = mask[node];
    V2 xi;
    if (MODE == MODE_RESID0 || MODE == MODE_CHEB0) {
      const T wf = MODE == MODE_CHEB0 ? w0 : omega;
      const V2 bv = reinterpret_cast<const V2*>(b)[node];
      const V2 d01 = reinterpret_cast<const V2*>(Dinv)[2 * node];
      const V2 d23 = reinterpret_cast<const V2*>(Dinv)[2 * node + 1];
      xi.x = wf * (d01.x * bv.x + d01.y * bv.y);
      xi.y = wf * (d23.x * bv.x + d23.y * bv.y);
      if (MODE == MODE_RESID0) reinterpret_cast<V2*>(xo)[node] = xi;
    } else {
      xi = reinterpret_cast<const V2*>(x)[node];
    }
    const T Ax0 = (m & 1u) ? xi.x : a0[q], Ax1 = (m & 2u) ? xi.y : a1[q];
    V2 out;
    if (MODE == MODE_APPLY) {
      out.x = Ax0;
      out.y = Ax1;
      if (DOT) dotv += (double)xi.x * (double)Ax0 + (double)xi.y * (double)Ax1;
    } else {
      const V2 bv = reinterpret_cast<const V2*>(b)[node];
      const T r0v = bv.x - Ax0, r1v = bv.y - Ax1;
      if (MODE == MODE_RESID || MODE == MODE_RESID0) {
        out.x = r0v;
        out.y = r1v;
      } else if (MODE == MODE_CHEB || MODE == MODE_CHEB0) {
        const T* D = Dinv + 4 * (int64_t)node;
        const T v0 = D[0] * r0v + D[1] * r1v, v1 = D[2] * r0v + D[3] * r1v;
        V2 dp = {T(0), T(0)};
        if (MODE == MODE_CHEB0 || dmode == 2) dp = xi;
        else if (dmode == 1) dp = reinterpret_cast<const V2*>(xo)[node];
        V2 dn;
        dn.x = c1 * dp.x + omega * v0;
        dn.y = c1 * dp.y + omega * v1;
        out.x = xi.x + dn.x;
        out.y = xi.y + dn.y;
        reinterpret_cast<V2*>(xo)[node] = dn;
      } else {
        const T* D = Dinv + 4 * (int64_t)node;
        out.x = xi.x + omega * (D[0] * r0v + D[1] * r1v);
        out.y = xi.y + omega * (D[2] * r0v + D[3] * r1v);
      }
    }
    reinterpret_cast<V2*>(y)[node] = out;
  }
  if (DOT) {
    double v = dotv;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < BX * BY / 32; w++) s += red[w];
      partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
  }
}

}  // namespace

int ebe2d_blocks(const Ebe& op) {
  const int npt = op.tile == 1 || op.tile == 2 ? op.tile : 4;
  return ceil_div(op.nx + 1, BX) * ceil_div(op.ny + 1, BY * npt);
}

template <class T, int MODE, bool DOT>
void ebe2d_launch(cudaStream_t s, const Ebe& op, const T* x, T* y, const T* b, const T* Dinv,
                  double omega, const int* done, double* parts, const ChebArg* ch) {
  constexpr bool CHEB = MODE == MODE_CHEB || MODE == MODE_CHEB0;
  if (CHEB && !ch) TOMG_THROW(TOMG_E_INVALID, "Chebyshev step without its state");
  T* xo = MODE == MODE_RESID0 ? const_cast<T*>(x) : (CHEB ? (T*)ch->d : nullptr);
  const T c1 = CHEB ? (T)ch->c1 : T(0);
  const int dm = CHEB ? ch->dmode : 0;
  const T w0 = CHEB ? (T)ch->w0 : T(0);
  const int npt = DOT ? 4 : (op.tile == 1 || op.tile == 2 ? op.tile : 4);  // dots: fixed tile
  dim3 grid(ceil_div(op.nx + 1, BX), ceil_div(op.ny + 1, BY * npt));
  if (!op.Kh) TOMG_THROW(TOMG_E_INVALID, "tiled element kernel without a host copy of Ke");
  KeP2<T> K;
  memcpy(K.v, op.Kh, sizeof(K.v));
#define EB(N) LAUNCH((k_ebe2<T, MODE, DOT, N>), grid, dim3(BX, BY), 0, s, op.nx, op.ny, K,     \
                     (const T*)op.E, op.mask, x, y, b, Dinv, (T)omega, done, parts, xo, c1, dm, w0)
  if (npt == 1) EB(1);
  else if (npt == 2) EB(2);
  else EB(4);
#undef EB
}

int ebe2d_autotune(cudaStream_t s, const Ebe& op, const float* Dinv) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;
  const std::pair<int, int> key(op.nx, op.ny);
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  const int64_t n = 2 * (int64_t)(op.nx + 1) * (op.ny + 1);
  DBuf<float> x, y, b;
  x.resize(n);
  y.resize(n);
  b.resize(n);
  x.zero(s);
  b.zero(s);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int best = 4;
  float best_ms = 1e30f;
  for (int npt : {4, 2, 1}) {
    Ebe o = op;
    o.tile = npt;
    ebe2d_launch<float, MODE_RESID, false>(s, o, x.p, y.p, b.p, Dinv, 0.5, nullptr, nullptr);
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < 5; r++)
      ebe2d_launch<float, MODE_RESID, false>(s, o, x.p, y.p, b.p, Dinv, 0.5, nullptr, nullptr);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < 0.97f * best_ms) {  // a smaller tile must win clearly
      best_ms = ms;
      best = npt;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> g(mu);
  cache[key] = best;
  return best;
}

#define INST(T, M, D)                                                                      \
  template void ebe2d_launch<T, M, D>(cudaStream_t, const Ebe&, const T*, T*, const T*,     \
                                      const T*, double, const int*, double*, const ChebArg*);
INST(float, MODE_APPLY, true) INST(float, MODE_APPLY, false) INST(float, MODE_RESID, false)
INST(float, MODE_JACOBI, false) INST(float, MODE_RESID0, false) INST(double, MODE_APPLY, true)
INST(double, MODE_APPLY, false) INST(double, MODE_RESID, false) INST(double, MODE_JACOBI, false)
INST(double, MODE_RESID0, false) INST(float, MODE_CHEB, false) INST(double, MODE_CHEB, false)
INST(float, MODE_CHEB0, false) INST(double, MODE_CHEB0, false)
#undef INST

}  // namespace tomg
