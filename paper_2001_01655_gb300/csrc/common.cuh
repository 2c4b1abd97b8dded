// Shared definitions of the tomg CUDA library: error handling, device buffers, launch
// accounting, kernel-side helpers.  Everything here is project code for sm_103a.
#pragma once

#include <chrono>
#include <cstdio>
#include <cstdlib>

#include <cuda_runtime.h>
#include <atomic>
#include <stdint.h>
#include <stdio.h>
#include <string>
#include <vector>

#include "../../include/tomg.h"

namespace tomg {

// ---------------------------------------------------------------------------------------
// errors
void set_error(const char* fmt, ...);
const char* get_error();

struct Error {
  tomg_status st;
};

#define TOMG_THROW(status, ...)          \
  do {                                   \
    ::tomg::set_error(__VA_ARGS__);      \
    throw ::tomg::Error{status};         \
  } while (0)

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      if (e_ == cudaErrorMemoryAllocation)                                              \
        TOMG_THROW(TOMG_E_OOM, "%s:%d %s: %s", __FILE__, __LINE__, #call,               \
                   cudaGetErrorString(e_));                                             \
      TOMG_THROW(TOMG_E_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,                \
                 cudaGetErrorString(e_));                                               \
    }                                                                                   \
  } while (0)

// count of kernels launched by this library (per process; contexts read deltas)
extern std::atomic<int64_t> g_launches;

// Programmatic dependent launch for the captured solve loop: while enabled (on this thread),
// kernels are launched with programmatic stream serialisation, so the next kernel of the
// chain is scheduled while the current one drains.  Every kernel of the loop starts with
// pdl_prologue(): it lets its dependants launch, then waits until its predecessor grid has
// completed and its writes are visible, before touching any data.
bool pdl_enabled();
void set_pdl(bool on);
// Right-hand sides of a block solve (Sec. 2.2, 4.2: several loads and adjoint right-hand sides
// on one hierarchy): while a BatchScope of R > 1 is active on this thread, the wrappers of the
// solve's kernels launch R copies of their grid (blockIdx.y, or a factor of blockIdx.z for the
// 3D-tiled element kernel) and the kernels offset every vector by the copy index times the
// vector's length; matrices, moduli, masks and smoother blocks are shared.  Wrappers without a
// block form throw while a scope is active.
int batch_rhs();
void set_batch_rhs(int r);
// distance between consecutive right-hand sides of a block vector whose vectors have n
// entries: n rounded up to a multiple of 4, so that every right-hand side starts on a 16-byte
// boundary (FP64 and FP32) and the paired 8 / 16-byte vector loads stay aligned
__host__ __device__ __forceinline__ int64_t rhs_stride(int64_t n) { return (n + 3) & ~(int64_t)3; }
struct BatchScope {
  int saved;
  explicit BatchScope(int r) : saved(batch_rhs()) { set_batch_rhs(r); }
  ~BatchScope() { set_batch_rhs(saved); }
};
void no_batch(const char* what);  // throws E_INVALID inside a BatchScope of R > 1

__device__ __forceinline__ void pdl_prologue() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
// The two halves of pdl_prologue, for kernels that first fetch data no kernel of the solve
// loop writes (operator values, structure, smoother blocks: fixed between setups), so those
// loads overlap the predecessor's tail; everything produced by the loop is read after
// pdl_wait().  Without programmatic serialisation the wait returns at once.
__device__ __forceinline__ void pdl_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

#define LAUNCH(kernel, grid, block, smem, strm_, ...)                                   \
  do {                                                                                 \
    if (::tomg::pdl_enabled()) {                                                       \
      cudaLaunchConfig_t cfg_ = {};                                                    \
      cfg_.gridDim = dim3(grid);                                                       \
      cfg_.blockDim = dim3(block);                                                     \
      cfg_.dynamicSmemBytes = (smem);                                                  \
      cfg_.stream = (strm_);                                                           \
      cudaLaunchAttribute at_[1];                                                      \
      at_[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                  \
      at_[0].val.programmaticStreamSerializationAllowed = 1;                           \
      cfg_.attrs = at_;                                                                \
      cfg_.numAttrs = 1;                                                               \
      CK(cudaLaunchKernelEx(&cfg_, kernel, __VA_ARGS__));                              \
    } else {                                                                           \
      kernel<<<(grid), (block), (smem), (strm_)>>>(__VA_ARGS__);                       \
    }                                                                                  \
    ::tomg::g_launches++;                                                              \
    CK(cudaGetLastError());                                                            \
  } while (0)

// ---------------------------------------------------------------------------------------
// device buffers (owning, move-only), stream-ordered: allocated and freed on the stream of the
// API call in progress through CUDA's stream-ordered pool, which keeps freed memory cached
// (no device-wide synchronisation on free, no driver round trip on reuse)
cudaStream_t alloc_stream();              // stream of the API call in progress
void set_alloc_stream(cudaStream_t s);    // set by every API entry point

template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, alloc_stream());
    p = nullptr;
    n = 0;
  }
  // (re)allocate to exactly `count` elements (keeps the buffer if already that size)
  void resize(size_t count) {
    if (count == n && p) return;
    release();
    if (count == 0) return;
    CK(cudaMallocAsync((void**)&p, count * sizeof(T), alloc_stream()));
    n = count;
  }
  void zero(cudaStream_t s) {
    if (n) CK(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
  size_t bytes() const { return n * sizeof(T); }
};

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// number of SMs of the current device (cached)
int num_sms();

// ---------------------------------------------------------------------------------------
// kernel-side helpers
template <class T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// deterministic block reduction of one double per thread (fixed tree order);
// result valid in thread 0.  blockDim.x must be a multiple of 32 and <= 1024.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;
}

// early-exit flag shared by the solve loop: kernels become no-ops once the solve is done
// Phase timing of the setup for diagnosis (TOMG_TRACE_SETUP=1): synchronises the stream at
// each mark and prints the host time since the previous mark to stderr.
struct SetupTrace {
  bool on;
  cudaStream_t s;
  std::chrono::steady_clock::time_point t0;
  explicit SetupTrace(cudaStream_t st) : on(getenv("TOMG_TRACE_SETUP") != nullptr), s(st),
                                         t0(std::chrono::steady_clock::now()) {}
  void mark(const char* what, int level = -1) {
    if (!on) return;
    cudaStreamSynchronize(s);
    const auto t = std::chrono::steady_clock::now();
    fprintf(stderr, "[setup] %-22s L%-2d %8.3f ms\n", what, level,
            std::chrono::duration<double, std::milli>(t - t0).count());
    t0 = t;
  }
};

__device__ __forceinline__ bool solve_done(const int* done) { return done && *(volatile const int*)done; }

// First point-block Jacobi sweep from x = 0 at one node: x = w Dinv_node b_node (B x B blocks).
// Every kernel that forms this value (the sweep itself and the smoothing steps that fuse it)
// goes through jacobi_block, so they agree bit for bit.
template <class T, int B>
__device__ __forceinline__ void jacobi_block(const T* D, const T* bv, T omega, T* xv) {
#pragma unroll
  for (int r = 0; r < B; r++) {
    T v = T(0);
#pragma unroll
    for (int c = 0; c < B; c++) v += D[r * B + c] * bv[c];
    xv[r] = omega * v;
  }
}
template <class T, int B>
__device__ __forceinline__ void jacobi_first(const T* __restrict__ Dinv, const T* __restrict__ b,
                                             int64_t node, T omega, T* xv) {
  T D[B * B], bv[B];
#pragma unroll
  for (int t = 0; t < B * B; t++) D[t] = Dinv[(int64_t)B * B * node + t];
#pragma unroll
  for (int c = 0; c < B; c++) bv[c] = b[(int64_t)B * node + c];
  jacobi_block<T, B>(D, bv, omega, xv);
}

// Chebyshev smoother step at one node (B components) from its residual r = b - A x:
// dn = c1 d_prev + c2 Dinv r, y = x + dn, d = dn; d_prev = 0 (dmode 0), d (1) or x (2)
template <class T, int B>
__device__ __forceinline__ void cheb_node(int64_t node, const T* r, const T* xi,
                                          const T* __restrict__ Dinv, T c1, T c2, int dmode,
                                          T* __restrict__ d, T* __restrict__ y) {
  const T* D = Dinv + (int64_t)B * B * node;
#pragma unroll
  for (int q = 0; q < B; q++) {
    T v = T(0);
#pragma unroll
    for (int c = 0; c < B; c++) v += D[q * B + c] * r[c];
    const T prev = dmode == 2 ? xi[q] : (dmode == 1 ? d[(int64_t)B * node + q] : T(0));
    const T dn = c1 * prev + c2 * v;
    y[(int64_t)B * node + q] = xi[q] + dn;
    d[(int64_t)B * node + q] = dn;
  }
}

}  // namespace tomg

namespace tomg {
// Barrier over every block of a cooperative launch (all blocks resident).  sync[0] counts the
// arrivals, sync[1] is the generation the last arrival advances.  A wait is bounded: past
// `limit` polls, or once *err is set by another block, the block sets *err and every thread
// of it gets false, so that no kernel waits forever on a block that has gone.  limit = 0 (a
// test hook) gives up at once, without looking at the barrier.
__device__ __forceinline__ bool grid_sync(unsigned* sync, unsigned* err, unsigned nblocks,
                                          unsigned limit) {
  __syncthreads();
  unsigned ok = 1;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = sync + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(sync, 1u) == nblocks - 1) {
      sync[0] = 0;
      __threadfence();
      atomicAdd(sync + 1, 1u);
    } else {
      unsigned it = 0;
      while (limit == 0 || *gen == g) {
        if (++it > limit || *(volatile unsigned*)err) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (!ok) atomicExch(err, 1u);
  }
  return __syncthreads_and(ok) != 0;
}

// FP32 <-> FP64 conversions by integer operations on the bit patterns, for the vector kernels
// of the outer loop: there the conversion instructions share GB300's narrow FP64 pipe with the
// dot products.  Both are exact restatements of IEEE 754 binary32 / binary64 conversion (round
// to nearest even on the way down) for zeros and normal numbers; subnormals, infinities and
// NaNs take the hardware conversion, in a function of its own, so that the compiler cannot
// replace the branch by computing both and selecting (which would put the conversion
// instruction back on every element).
static __device__ __noinline__ double f2d_hw(float f) { return (double)f; }
static __device__ __noinline__ float d2f_hw(double x) { return (float)x; }
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  if (e == 0u && (u & 0x7fffffu) == 0u) return __longlong_as_double((long long)sign);
  if (e == 0u || e == 0xffu) return f2d_hw(f);
  // exponent bias 127 -> 1023, the 23 fraction bits at the top of the 52
  return __longlong_as_double(
      (long long)(sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7fffffu) << 29)));
}
__device__ __forceinline__ float d2f_bits(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  if ((b << 1) == 0u) return __uint_as_float(sign);
  const int e = (int)((b >> 52) & 0x7ffu) - 896;  // binary32 biased exponent
  if (e < 1 || e > 254) return d2f_hw(x);          // subnormal or out of range, inf, NaN
  const uint64_t m = b & 0xfffffffffffffull;
  uint32_t u = sign | ((uint32_t)e << 23) | (uint32_t)(m >> 29);
  const uint32_t rest = (uint32_t)(m & 0x1fffffffu);  // the 29 dropped fraction bits
  // round to nearest, ties to even; a carry out of the fraction raises the exponent, which is
  // the correctly rounded result (up to infinity from the largest exponent)
  if (rest > 0x10000000u || (rest == 0x10000000u && (u & 1u))) u += 1u;
  return __uint_as_float(u);
}

// 1 / sqrt(d) in FP64 from the FP32 hardware estimate and two Newton steps for the reciprocal
// square root, y <- y (3 - d y^2) / 2, each of which doubles the number of correct bits
// (about 22 -> 44 -> 88).  A few FP64 FMAs instead of an FP64 square root and division, which
// are long sequences on GB300's narrow FP64 pipe.  Outside the FP32 range: the plain formula.
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double y = (double)rsqrtf((float)d);
  y = y * (1.5 - 0.5 * d * y * y);
  y = y * (1.5 - 0.5 * d * y * y);
  return y;
}

// Inverse of a small SPD block (row-major B x B, FP64) through its Cholesky factor; the B
// reciprocal square roots of the pivots replace every square root and division.
// Returns false if a pivot is not positive (the block is then left unchanged in Ainv = 0).
template <int B>
__device__ __forceinline__ bool spd_inverse(const double* A, double* Ainv) {
  double L[B][B], rL[B];
#pragma unroll
  for (int i = 0; i < B; i++)
#pragma unroll
    for (int j = 0; j < B; j++) L[i][j] = 0.0;
  bool ok = true;
#pragma unroll
  for (int j = 0; j < B; j++) {
    double d = A[j * B + j];
#pragma unroll
    for (int k = 0; k < j; k++) d -= L[j][k] * L[j][k];
    if (!(d > 0.0)) ok = false;
    const double rl = ok ? rsqrt_newton(d) : 1.0;  // 1 / L_jj
    rL[j] = rl;
    L[j][j] = ok ? d * rl : 1.0;
#pragma unroll
    for (int i = j + 1; i < B; i++) {
      double v = A[i * B + j];
#pragma unroll
      for (int k = 0; k < j; k++) v -= L[i][k] * L[j][k];
      L[i][j] = v * rl;
    }
  }
  // columns of L^-1, then Ainv = L^-T L^-1
  double Li[B][B];
#pragma unroll
  for (int c = 0; c < B; c++) {
#pragma unroll
    for (int i = 0; i < B; i++) {
      double v = (i == c) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < i; k++) v -= L[i][k] * Li[k][c];
      Li[i][c] = v * rL[i];
    }
  }
#pragma unroll
  for (int i = 0; i < B; i++)
#pragma unroll
    for (int j = 0; j < B; j++) {
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < B; k++) v += Li[k][i] * Li[k][j];
      Ainv[i * B + j] = ok ? v : 0.0;
    }
  return ok;
}

// linear node index <-> grid coordinates
__device__ __forceinline__ void node_ijk(int64_t node, int nx, int ny, int dim, int& i, int& j,
                                         int& k) {
  if (node >= 0 && node < 0x7fffffffLL) {  // 32-bit division (a 64-bit one is a long sequence)
    const unsigned n = (unsigned)node, a = (unsigned)(nx + 1);
    i = (int)(n % a);
    const unsigned r = n / a;
    if (dim == 3) {
      j = (int)(r % (unsigned)(ny + 1));
      k = (int)(r / (unsigned)(ny + 1));
    } else {
      j = (int)r;
      k = 0;
    }
    return;
  }
  i = (int)(node % (nx + 1));
  int64_t r = node / (nx + 1);
  if (dim == 3) {
    j = (int)(r % (ny + 1));
    k = (int)(r / (ny + 1));
  } else {
    j = (int)r;
    k = 0;
  }
}
__device__ __forceinline__ int64_t node_id(int i, int j, int k, int nx, int ny) {
  return (int64_t)i + (int64_t)(nx + 1) * ((int64_t)j + (int64_t)(ny + 1) * k);
}

// Geometric transfers (Sec. 3.2): coarse node I sits at fine position min(2I, nf) per axis; a
// fine node at a coarse position takes weight 1 from it, one midway between two coarse nodes
// 1/2 from each.  coarse_of lists the coarse partners of fine position p and their weights.
__host__ __device__ __forceinline__ int coarse_of(int p, int nf, int* I, double* w) {
  const int nc = (nf + 1) / 2;
  if (p == nf) { I[0] = nc; w[0] = 1.0; return 1; }
  if ((p & 1) == 0) { I[0] = p / 2; w[0] = 1.0; return 1; }
  I[0] = (p - 1) / 2; w[0] = 0.5;
  I[1] = (p + 1) / 2; w[1] = 0.5;
  return 2;
}
// the same partners along one axis with FP32 weights (1 or 1/2: products of three are exact
// in any precision, so no FP64 instruction is needed to form them)
struct AxisP {
  int n;
  int I[2];
  float w[2];
};
__device__ __forceinline__ AxisP axis_partners(int p, int nf) {
  AxisP a;
  const int nc = (nf + 1) / 2;
  if (p == nf) { a.n = 1; a.I[0] = nc; a.w[0] = 1.f; a.I[1] = nc; a.w[1] = 0.f; return a; }
  if ((p & 1) == 0) { a.n = 1; a.I[0] = p >> 1; a.w[0] = 1.f; a.I[1] = a.I[0]; a.w[1] = 0.f; return a; }
  a.n = 2; a.I[0] = (p - 1) >> 1; a.w[0] = 0.5f; a.I[1] = (p + 1) >> 1; a.w[1] = 0.5f;
  return a;
}
// acc += (P xc) at the fine node with axis partners (px, py, pz), coarse vector xc on the grid
// cnx x cny (x cnz), in a fixed order (z, y, x partners).  The prolongation kernel and the
// smoothing steps that fuse it all go through here, so they agree bit for bit.
template <class T, int DIM>
__device__ __forceinline__ void prolong_acc(const AxisP& px, const AxisP& py, const AxisP& pz,
                                            int cnx, int cny, const T* __restrict__ xc, T* acc) {
  const int nzs = DIM == 3 ? pz.n : 1;
  for (int c3 = 0; c3 < nzs; c3++)
    for (int b = 0; b < py.n; b++)
      for (int a = 0; a < px.n; a++) {
        const T w = (T)(px.w[a] * py.w[b] * (DIM == 3 ? pz.w[c3] : 1.f));
        const int64_t I = node_id(px.I[a], py.I[b], DIM == 3 ? pz.I[c3] : 0, cnx, cny);
#pragma unroll
        for (int c = 0; c < DIM; c++) acc[c] += w * xc[DIM * I + c];
      }
}
template <class T, int DIM>
__device__ __forceinline__ void prolong_node(int x, int y, int z, int fnx, int fny, int fnz,
                                             int cnx, int cny, const T* __restrict__ xc, T* acc) {
  const AxisP px = axis_partners(x, fnx), py = axis_partners(y, fny);
  const AxisP pz = DIM == 3 ? axis_partners(z, fnz) : AxisP{1, {0, 0}, {1.f, 0.f}};
  prolong_acc<T, DIM>(px, py, pz, cnx, cny, xc, acc);
}
}  // namespace tomg
