// FP64 level-0 SIMP element operator on hex8 grids (Sec. 2.1 Eq. 2, Sec. 3.1: the outer Krylov
// loop's K p and residuals) with the element contractions on the FP16 tensor cores, exact to
// the FP64 rounding of the result.
//
// GB300 issues FP64 at about 2 FMAs per clock and SM, so the assembled 243-entry stencil the
// FP64 apply used to run on is bound by that pipe.  Here every product of the element
// contraction is computed exactly in integers on the tensor cores (the splitting idea of Ozaki
// et al., 2012), and FP64 is left with the scaling and the node sums:
//   * for nu with a rational ratio lambda / mu = p / q (nu = 0.3: 3 / 2), Ke = c C with C =
//     p K_l + q K_m an integer matrix (K_l, K_m the 72-scaled parts; entries of C up to 88,
//     absolute row sums up to 472) and c = mu / (72 q);
//   * each element row x_e (24 values) is written in fixed point on its largest exponent:
//     X_j = round(x_j 2^(52 - e)) with |X_j| <= 2^53, and |X_j| is cut into five digits of 11
//     bits that carry the sign of X_j (sign-magnitude, in [-2047, 2047]); every digit is an
//     exact FP16 value;
//   * one MMA chain per digit (K = 24 padded to 32, N = 24 outputs padded to 32) accumulates
//     sum_j C_oj d_j in FP32 exactly (|sum| < 2^20);
//   * the digit sums are turned back into integers and combined in int64: Z_o = sum_j C_oj X_j
//     exactly; y_o = (E_e c 2^(e - 52)) Z_o, one FP64 conversion and one FP64 product per
//     output.
// The result differs from the exact element product only by the rounding of X (2^-53 of the
// row's largest entry) and the FP64 roundings of the conversion, the product and the node sums.
// The FP64 pipe is left with these, the node sums and the dot product.
//
// Tiling as in the FP32 tensor-core kernel (k_ebe3tc.cu), with one M = 128 tile per element
// layer (32 x 4 elements, 128 threads, 31 x 3 owned nodes): the block walks the element layers
// of its column of nodes; per layer it builds the 5 digit rows of its elements in tensor
// memory, issues 10 MMAs, waits, and folds the accumulators into node sums (x-neighbour by warp
// shuffle, y-neighbour through shared memory, z in registers), all in a fixed order.  Tensor
// memory: digit k of A at column 16 k, its accumulator at 80 + 32 k (256 columns, two blocks
// per SM).  Modes: y = A x with the partials of x . y and FIN_ALPHA in the last block (the
// outer apply), and r = b - A x.  All waits are bounded as in the FP32 kernel.
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "finish.cuh"

namespace tomg {

namespace {

constexpr int TEX = 32, TY = 4;              // elements of a layer tile in x and y
constexpr int TNX = TEX + 1, TNY = TY + 1;   // nodes of a layer tile
constexpr int ROWS = TEX * TY;               // 128 element rows: the tensor-memory lanes
constexpr int NT = 2 * ROWS;                 // two threads per element row (bottom, top half)
constexpr int LAYER_NODES = TNX * TNY;       // 165
constexpr int KD = 24;                       // element DOFs
constexpr int KH = KD / 2;                   // DOFs (inputs and outputs) of one half
constexpr int ND = 5;                        // digits of 11 bits
constexpr int NB = 32;                       // N: 24 outputs padded
constexpr int KP = 32;                       // K per digit: 24 padded
constexpr int LBO = 128;                     // core matrices adjacent in K
constexpr int SBO = (KP / 8) * LBO;          // 8-row groups: 512
constexpr int B_BYTES = (NB / 8) * SBO;      // 2048
constexpr int A_COL = 0, ACC_COL = 80, TMEM_COLS = 256;
constexpr int PS = 7;                        // staged y-pair partials: row stride (doubles)
constexpr int OFF_B = 0;
constexpr int OFF_X = OFF_B + B_BYTES;                         // x ring, FP64
constexpr int OFF_P = OFF_X + 2 * LAYER_NODES * 3 * 8;         // y pairs, FP64
constexpr int OFF_T = OFF_P + 2 * TY * TNX * PS * 8;           // top-half node sums, FP64
constexpr int OFF_R = OFF_T + 2 * LAYER_NODES * 3 * 8;         // reduction scratch
constexpr int OFF_BAR = OFF_R + 32 * 8;                        // mbarrier, TMEM address
constexpr int SMEM_ALLOC = OFF_BAR + 16 + 128;
static_assert(ACC_COL >= ND * KP / 2 && ACC_COL + ND * NB <= TMEM_COLS, "tensor memory map");
static_assert(OFF_X % 16 == 0 && OFF_P % 16 == 0 && OFF_T % 16 == 0 && OFF_BAR % 8 == 0,
              "alignment");
static_assert(LAYER_NODES <= NT, "one node per thread stages a layer");

// kind::f16, D FP32, A and B FP16, K-major, N = 32, M = 128
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(NB >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr uint32_t WAIT_LIMIT = 1u << 22;

__device__ int g_x64_error;  // set by a block whose MMA completion wait ran out

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(LBO >> 4) << 16) |
         ((uint64_t)(SBO >> 4) << 32) | (1ull << 46);
}
__host__ __device__ __forceinline__ int op_off(int row, int k) {
  return (row >> 3) * SBO + (k >> 3) * LBO + (row & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
      :: "r"(d), "r"(a), "l"(b), "r"(IDESC), "r"(acc) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < WAIT_LIMIT; i++)
    if (mbar_try(bar, parity)) return true;
  return false;
}
// n FP32 columns of this thread's lane from column taddr (n = 8 or 4; no wait)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 4; i++) v[i] = __uint_as_float(r[i]);
}
// 12 FP32 columns of one half of the 24 outputs: half 0 columns 0-11 (x8 at 0, x4 at 8),
// half 1 columns 12-23 (x4 at 12, x8 at 16); every access aligned to its width
__device__ __forceinline__ void tmem_ld12(uint32_t taddr, int h, float* v) {
  if (h == 0) {
    tmem_ld8(taddr, v);
    tmem_ld4(taddr + 8u, v + 8);
  } else {
    tmem_ld4(taddr + 12u, v);
    tmem_ld8(taddr + 16u, v + 4);
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_st2(uint32_t taddr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};\n"
               :: "r"(taddr), "r"(v[0]), "r"(v[1]) : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};\n"
               :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]) : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n"
      :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
         "r"(v[6]), "r"(v[7])
      : "memory");
}

// an integer |v| < 2^22 as an exact FP32 value (rounding-free: the magic constant 1.5 x 2^23
// puts v in the last place of the significand)
__device__ __forceinline__ float int_to_f32(int v) {
  return __int_as_float(0x4B400000 + v) - 12582912.0f;
}

// node layer kk of the tile (FP64): values and mask bits of one node per thread
struct XPre {
  double v[3];
  unsigned m;
};
__device__ __forceinline__ void x_fetch(XPre& p, int kk, int EX0, int EY0, int nx, int ny, int nz,
                                        const uint8_t* __restrict__ mask,
                                        const double* __restrict__ x) {
  const int q = threadIdx.x;
  p.v[0] = p.v[1] = p.v[2] = 0.0;
  p.m = 7u;
  if (q < LAYER_NODES) {
    const int gi = EX0 + q % TNX, gj = EY0 + q / TNX;
    if (gi >= 0 && gi <= nx && gj >= 0 && gj <= ny && kk >= 0 && kk <= nz) {
      const int64_t node = node_id(gi, gj, kk, nx, ny);
      p.m = __ldg(mask + node);
#pragma unroll
      for (int c = 0; c < 3; c++) p.v[c] = __ldg(x + 3 * node + c);
    }
  }
}
__device__ __forceinline__ void x_store(const XPre& p, double* sx) {
  const int q = threadIdx.x;
  if (q < LAYER_NODES) {
#pragma unroll
    for (int c = 0; c < 3; c++) sx[3 * q + c] = ((p.m >> c) & 1u) ? 0.0 : p.v[c];
  }
}
__device__ __forceinline__ double e_fetch(int ke, int ex, int ey, int EX0, int EY0, int nx, int ny,
                                          int nz, const double* __restrict__ E) {
  const int ge = EX0 + ex, gf = EY0 + ey;
  if (ge < 0 || ge >= nx || gf < 0 || gf >= ny || ke < 0 || ke >= nz) return 0.0;
  return __ldg(E + ge + (int64_t)nx * (gf + (int64_t)ny * ke));
}

// input k (0..23) of element (ex, ey): DOF k % 3 of local node k / 3, from the ring slots of
// node layers ke (s0: local nodes 0-3) and ke + 1 (s1: local nodes 4-7)
__device__ __forceinline__ double elem_in(const double* s0, const double* s1, int ex, int ey, int k) {
  const int bn = k / 3, c = k % 3;
  const double* sx = (bn & 4) ? s1 : s0;
  return sx[3 * ((ey + ((bn >> 1) & 1)) * TNX + ex + (bn & 1)) + c];
}

// Element (ex, ey) of layer ke, half h: the largest biased FP64 exponent e of the row's 24
// entries (both halves find the same), then this half's 12 entries in fixed point on it,
// X_j = round(x_j 2^(1075 - e)), |X_j| <= 2^53, cut into five FP16 digits of 11 bits and written
// to tensor memory: digit q at taddr + 16 q holds 12 words of digit pairs (lower K index in the
// low half) and 4 zero words of K padding; half 0 writes words 0-5, half 1 words 6-11 and the
// padding.  Returns e, or 0 for a row whose entries are all below 2^-970 (zero digits).
__device__ __forceinline__ int a_digits(uint32_t taddr, const double* s0, const double* s1,
                                        int ex, int ey, int h) {
  int emax = 0;
#pragma unroll
  for (int k = 0; k < KD; k++)
    emax = max(emax, (int)((__double_as_longlong(elem_in(s0, s1, ex, ey, k)) >> 52) & 0x7FF));
  if (emax < 53) emax = 0;
  // |X_j| and its sign: every digit of |X_j| carries the sign of X_j (sign-magnitude digits in
  // [-2047, 2047], each exact in FP16), so that sum_q 2^(11 q) d_q,j = X_j
  uint64_t A[KH];
  uint32_t sg[KH / 2];
#pragma unroll
  for (int t = 0; t < KH; t++) {
    const uint64_t bits = __double_as_longlong(elem_in(s0, s1, ex, ey, KH * h + t));
    const int e = (int)((bits >> 52) & 0x7FFu);
    const uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
    const int sh = emax - e;
    uint64_t a = 0;
    if (emax && sh <= 54) a = (m + ((1ull << sh) >> 1)) >> sh;  // round half up
    A[t] = a;
    const uint32_t neg = (uint32_t)(bits >> 63);
    if (t & 1) sg[t / 2] |= neg << 31;
    else sg[t / 2] = neg << 15;
  }
#pragma unroll
  for (int q = 0; q < ND; q++) {
    uint32_t w[8];
#pragma unroll
    for (int c = 0; c < KH / 2; c++) {
      const int d0 = (int)((A[2 * c] >> (11 * q)) & 2047);
      const int d1 = (int)((A[2 * c + 1] >> (11 * q)) & 2047);
      const __half2 hv = __floats2half2_rn(int_to_f32(d0), int_to_f32(d1));  // exact
      w[c] = *reinterpret_cast<const uint32_t*>(&hv) ^ sg[c];
    }
    const uint32_t col = taddr + (uint32_t)(16 * q);
    if (h == 0) {  // words 0-5
      tmem_st4(col, w);
      tmem_st2(col + 4u, w + 4);
    } else {  // words 6-11, then the padding words 12-15
      tmem_st2(col + 6u, w);
      w[0] = w[2]; w[1] = w[3]; w[2] = w[4]; w[3] = w[5];
      w[4] = w[5] = w[6] = w[7] = 0u;
      tmem_st8(col + 8u, w);
    }
  }
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  return emax;
}

// the digit MMAs of one layer: digit q's rows against B (K steps of 16) into accumulator q
__device__ __forceinline__ void issue_mmas(uint32_t tmem, uint32_t bbase, uint32_t bar) {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
  for (int q = 0; q < ND; q++)
#pragma unroll
    for (int s = 0; s < KP / 16; s++)
      mma_ts(tmem + (uint32_t)(ACC_COL + NB * q), tmem + (uint32_t)(A_COL + 16 * q + 8 * s),
             sdesc(bbase + 2 * LBO * s), s ? 1u : 0u);
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
               :: "r"(bar) : "memory");
}

// this thread's half of its element row of the previous layer: Z_o = sum_q D_q,o 2^(11 q)
// exactly, then v_o = scale Z_o in FP64, scale = E_e c 2^(p - 1075) (0 for a zero row or no
// element).  Each digit sum D (an integer, |D| < 2^20, exact in FP32) is read as the bit
// pattern of D + 1.5 x 2^23 (one FP32 add), and the five patterns are combined with 32 x 32-bit
// wide multiply-adds modulo 2^64; the offsets they carry, 0x4B400000 (1 + 2^11 + ... + 2^44), are
// removed by one subtraction.  The wrap-around cancels: Z itself fits in 64 bits.
// Measured against converting Z with integer operations instead of the FP64 conversion, and
// against forming ec Z 2^(p - 1075) entirely with integer operations: both slower.
__device__ __forceinline__ void fold_digits(uint32_t taddr, int h, double scale, double* v) {
  constexpr uint64_t MAGIC = 0x4B400000ull;
  constexpr uint64_t OFFSET = MAGIC * (1ull + (1ull << 11) + (1ull << 22) + (1ull << 33) +
                                       (1ull << 44));
  uint64_t lo[KH], hi[KH];  // digits 0-2 and 3-4
#pragma unroll
  for (int q = 0; q < ND; q++) {
    float d[KH];
    tmem_ld12(taddr + (uint32_t)(ACC_COL + NB * q), h, d);
#pragma unroll
    for (int o = 0; o < KH; o++) {
      const uint64_t bq = __float_as_uint(d[o] + 12582912.0f);
      if (q == 0) lo[o] = bq;
      else if (q < 3) lo[o] += bq * (1ull << (11 * q));
      else if (q == 3) hi[o] = bq;
      else hi[o] += bq * (1ull << 11);
    }
  }
#pragma unroll
  for (int o = 0; o < KH; o++) {
    const int64_t Z = (int64_t)(lo[o] + (hi[o] << 33) - OFFSET);
    v[o] = scale * __ll2double_rn(Z);
  }
}

struct Fin {
  double x[3], b[3];
  unsigned m;
};

// Kernel 1 of an apply: the element products of one tile of the grid's element partition (32 x 4
// elements x nz_tile layers; every element belongs to exactly one tile) summed into the nodes of
// the tile's node box (33 x 5 x (nz_tile + 1)), written as partial sums; nodes on the box faces
// also receive sums from the neighbouring tiles, which kernel 2 adds.  Two threads per element
// row (its tensor-memory lane): half 0 (warps 0-3) builds the digits of the row's bottom inputs
// and folds its bottom outputs, half 1 (warps 4-7) the top ones.  Node layer L of the box is
// the top sums of element layer L - 1 (half 1, staged in shared memory) plus the bottom sums of
// element layer L (half 0); within a layer, x-neighbour sums by warp shuffle (lane 31 also
// carries the box's last column), y-neighbour sums through shared memory.
__global__ void __launch_bounds__(NT, 2)
k_ebe3x64_tiles(int nx, int ny, int nz, int nz_tile, int nzc, const uint4* __restrict__ Bimg,
                const double* __restrict__ E, double c, const uint8_t* __restrict__ mask,
                const double* __restrict__ x, double* __restrict__ pbuf, const int* done,
                Scalars* sc) {
  extern __shared__ uint8_t smem_raw[];
  pdl_prologue();
  // blockIdx.z = chunk of element layers + nzc x right-hand side of a block solve
  const int zc = blockIdx.z % nzc, rhs = blockIdx.z / nzc;
  const int64_t tile = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * zc);
  const int64_t ntile = (int64_t)gridDim.x * gridDim.y * nzc;
  const int slots = LAYER_NODES * (nz_tile + 1);
  {
    const int64_t vo = (int64_t)rhs * rhs_stride((int64_t)3 * (nx + 1) * (ny + 1) * (nz + 1));
    x += vo;
    pbuf += ((int64_t)rhs * ntile + tile) * slots * 3;
    if (sc) {
      sc += rhs;
      if (done) done = &sc->done;
    }
  }
  if (solve_done(done)) return;
  uint8_t* sm = smem_raw + ((128 - (smem_u32(smem_raw) & 127u)) & 127u);
  double* sxr = reinterpret_cast<double*>(sm + OFF_X);  // [2][LAYER_NODES][3]
  double* sP = reinterpret_cast<double*>(sm + OFF_P);   // [2][TY][TNX][PS]
  double* sT = reinterpret_cast<double*>(sm + OFF_T);   // [2][LAYER_NODES][3]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + OFF_BAR + 8);
  const uint32_t sbase = smem_u32(sm), bar0 = smem_u32(bar);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int h = tid / ROWS;  // half
  const int ex = lane, ey = (warp & 3);
  const int EX0 = blockIdx.x * TEX, EY0 = blockIdx.y * TY;
  const int k0 = zc * nz_tile;
  const int k1 = min(k0 + nz_tile, nz);  // element layers [k0, k1), node layers [k0, k1]

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 :: "r"(smem_u32(tmem_slot)), "r"(TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(bar0), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  for (int t = tid; t < B_BYTES / 16; t += NT) reinterpret_cast<uint4*>(sm + OFF_B)[t] = Bimg[t];
  for (int t = tid; t < 2 * LAYER_NODES * 3; t += NT) sT[t] = 0.0;

  XPre pre, pre2;
  x_fetch(pre, k0, EX0, EY0, nx, ny, nz, mask, x);
  x_fetch(pre2, k0 + 1, EX0, EY0, nx, ny, nz, mask, x);
  x_store(pre, sxr + (k0 & 1) * LAYER_NODES * 3);
  x_store(pre2, sxr + ((k0 + 1) & 1) * LAYER_NODES * 3);
  x_fetch(pre, k0 + 2, EX0, EY0, nx, ny, nz, mask, x);
  double ec_cur = c * e_fetch(k0, ex, ey, EX0, EY0, nx, ny, nz, E);  // E c of layer ke
  double sc_prev = 0.0;  // E c 2^(p - 1075) of this thread's row of layer ke - 1
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;

  uint32_t parity = 0, pending = 0;
  bool failed = false;

  for (int ke = k0; ke <= k1; ke++) {
    const bool mma_now = ke < k1;
    const int j = ke & 1, jp = j ^ 1;
    bool ok = true;
    double v[KH];
    if (ke > k0) {
      // the MMAs of layer ke - 1; the phase advances only on success (see the drain below)
      ok = mbar_wait(bar0, parity);
      if (ok) {
        parity ^= 1u;
        pending = 0u;
      }
      // the tensor-memory loads and stores below are warp-collective: a warp takes part only
      // if every lane saw the MMAs complete (otherwise the whole block gives up below)
      ok = __all_sync(0xffffffffu, ok);
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      // the accumulators are single-buffered: read before this layer's MMAs are issued
      if (ok) fold_digits(tmem + lane_base, h, sc_prev, v);
    }
    double sc_now = 0.0;
    if (ok && mma_now) {
      const int p = a_digits(tmem + lane_base + A_COL, sxr + j * LAYER_NODES * 3,
                             sxr + jp * LAYER_NODES * 3, ex, ey, h);
      if (p) sc_now = ec_cur * __longlong_as_double((long long)(p - 52) << 52);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    if (__syncthreads_or(!ok)) {  // a wait that ran out anywhere stops the whole block
      failed = true;
      break;
    }
    if (mma_now) {
      if (tid == 0) issue_mmas(tmem, sbase + OFF_B, bar0);
      pending = 1u;
    }
    // refill the ring: node layer ke + 2 replaces layer ke (read by the digits above)
    if (mma_now && ke + 2 <= k1) {
      x_store(pre, sxr + j * LAYER_NODES * 3);
      if (ke + 3 <= k1) x_fetch(pre, ke + 3, EX0, EY0, nx, ny, nz, mask, x);
    }
    const double ec_next =
        (ke + 1 < k1) ? c * e_fetch(ke + 1, ex, ey, EX0, EY0, nx, ny, nz, E) : 0.0;
    // x-pair sums of this half's node layer of element layer ke - 1: node column ex gets the
    // dx = 0 corner of element ex and the dx = 1 corner of element ex - 1 (none for column 0);
    // lane 31 also holds column 32 (the dx = 1 corner of element 31 alone)
    double pr[2][3], p32[2][3];
    if (ke > k0) {
#pragma unroll
      for (int dy = 0; dy < 2; dy++)
#pragma unroll
        for (int q = 0; q < 3; q++) {
          const double r1 = v[3 * (1 + 2 * dy) + q];
          const double left = __shfl_up_sync(0xffffffffu, r1, 1);
          pr[dy][q] = v[3 * (2 * dy) + q] + (lane ? left : 0.0);
          p32[dy][q] = r1;
        }
      double* myP = sP + ((j * TY + ey) * TNX + ex) * PS;
#pragma unroll
      for (int q = 0; q < 3; q++) myP[3 * h + q] = pr[1][q];
      if (lane == 31) {
        double* myP32 = sP + ((j * TY + ey) * TNX + TEX) * PS;
#pragma unroll
        for (int q = 0; q < 3; q++) myP32[3 * h + q] = p32[1][q];
      }
    }
    __syncthreads();
    if (ke > k0) {
      // the box positions of this thread: (ex, ey), with lane 31 also column 32 and element
      // row 3 also node row 4; node (lx, ly) sums the dy = 0 pairs of element row ly and the
      // dy = 1 pairs of element row ly - 1
      const int L = h ? ke : ke - 1;  // the node layer of this half's corners
      for (int cx = 0; cx < (lane == 31 ? 2 : 1); cx++) {
        const int lx = ex + cx;
        for (int cy = 0; cy < (ey == TY - 1 ? 2 : 1); cy++) {
          const int ly = ey + cy;
          double sum[3];
#pragma unroll
          for (int q = 0; q < 3; q++) {
            const double own = (cy == 0) ? (cx ? p32[0][q] : pr[0][q]) : 0.0;
            double up = 0.0;
            if (ly >= 1) {
              const double* upP = sP + ((j * TY + (ly - 1)) * TNX + lx) * PS;
              up = upP[3 * h + q];
            }
            sum[q] = up + own;
          }
          const int pos = ly * TNX + lx;
          if (h == 1 && L < k1) {  // staged for node layer L, finished next step by half 0
#pragma unroll
            for (int q = 0; q < 3; q++) sT[(j * LAYER_NODES + pos) * 3 + q] = sum[q];
          } else {  // node layer L complete within the tile: top of L - 1 plus bottom of L
            double* out = pbuf + ((int64_t)(L - k0) * LAYER_NODES + pos) * 3;
#pragma unroll
            for (int q = 0; q < 3; q++)
              out[q] = (h == 0 ? sT[(jp * LAYER_NODES + pos) * 3 + q] : 0.0) + sum[q];
          }
        }
      }
    }
    sc_prev = sc_now;
    ec_cur = ec_next;
  }

  if (failed) {
    if (tid == 0) atomicExch(&g_x64_error, 1);
    // MMAs still in flight write the accumulators until they complete
    if (pending) mbar_wait(bar0, parity);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n"
                 :: "r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// Kernel 2: every node's sum of the partial sums of the (one to eight) tiles whose boxes hold it,
// in ascending tile order, then the outer operator's finishing: A x = x on fixed DOFs, y = A x
// with the partials of x . y and FIN_ALPHA in the last block (MODE_APPLY), or y = b - A x.
constexpr int FIN_THREADS = 256;
constexpr int FIN_NPT = 4;  // nodes per thread: one block reduction of the dot per 1024 nodes
constexpr int X64_NZ_TILE = 8;  // element layers per tile

__device__ __forceinline__ int tiles_of(int i, int n_t, int w, int* t0) {
  // tiles t (0 <= t < n_t) with t w <= i <= t w + w; returns their count (1 or 2), first in *t0
  const int hi = min(i / w, n_t - 1);
  const int lo = (i % w == 0 && i > 0) ? i / w - 1 : hi;
  *t0 = lo;
  return hi - lo + 1;
}

template <int MODE, int NZT>
__global__ void __launch_bounds__(FIN_THREADS)
k_ebe3x64_nodes(int nx, int ny, int nz, int gx, int gy, int nzc,
                const double* __restrict__ pbuf, const uint8_t* __restrict__ mask,
                const double* __restrict__ x, double* __restrict__ y,
                const double* __restrict__ b, const int* done, double* partials, Scalars* sc) {
  __shared__ double sred[32];
  pdl_prologue();
  constexpr int nz_tile = NZT;
  const int rhs = blockIdx.y;
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  const int slots = LAYER_NODES * (nz_tile + 1);
  const int64_t ntile = (int64_t)gx * gy * nzc;
  {
    const int64_t vo = (int64_t)rhs * rhs_stride(3 * nn);
    x += vo;
    y += vo;
    if (b) b += vo;
    pbuf += (int64_t)rhs * ntile * slots * 3;
    if (partials) partials += (int64_t)rhs * gridDim.x;
    if (sc) {
      sc += rhs;
      if (done) done = &sc->done;
    }
  }
  if (solve_done(done)) return;
  double dotv = 0.0;
  for (int r = 0; r < FIN_NPT; r++) {  // FIN_NPT nodes per thread, FIN_THREADS apart
    const int64_t node = ((int64_t)blockIdx.x * FIN_NPT + r) * FIN_THREADS + threadIdx.x;
    if (node >= nn) break;
    int i, j, k;
    node_ijk(node, nx, ny, 3, i, j, k);
    int tx, ty, tz;
    const int cx = tiles_of(i, gx, TEX, &tx), cy = tiles_of(j, gy, TY, &ty);
    const int cz = tiles_of(k, nzc, nz_tile, &tz);
    // the first tile's partial starts the sum; the others are added in a fixed order (fixed
    // trip counts, the absent second tiles of an axis skipped by predicate)
    double acc[3];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int bb = 0; bb < 2; bb++)
#pragma unroll
        for (int d = 0; d < 2; d++) {
          if (a >= cz || bb >= cy || d >= cx) continue;
          const int bx = tx + d, by = ty + bb, bz = tz + a;
          const int64_t t = bx + (int64_t)gx * (by + (int64_t)gy * bz);
          const int slot = ((k - bz * nz_tile) * TNY + (j - by * TY)) * TNX + (i - bx * TEX);
          const double* pp = pbuf + (t * slots + slot) * 3;
#pragma unroll
          for (int q = 0; q < 3; q++) {
            const double v = __ldg(pp + q);
            acc[q] = (a | bb | d) ? acc[q] + v : v;
          }
        }
    const unsigned m = mask[node];
    double xv[3], Ax[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
      xv[q] = x[3 * node + q];
      Ax[q] = ((m >> q) & 1u) ? xv[q] : acc[q];
    }
    if (MODE == MODE_APPLY) {
#pragma unroll
      for (int q = 0; q < 3; q++) {
        y[3 * node + q] = Ax[q];
        dotv = fma(xv[q], Ax[q], dotv);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 3; q++) y[3 * node + q] = b[3 * node + q] - Ax[q];
    }
  }
  if (MODE != MODE_APPLY || !partials) return;  // uniform over the grid
  const double tot = block_sum(dotv, sred);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  if (sc && last_block(&sc->tk[TK_ALPHA], gridDim.x))
    finish_body(FIN_ALPHA, partials, gridDim.x, nullptr, 0, sc, sred);
}

struct X64Grid {
  int gx, gy, nzc;
};
inline X64Grid x64_grid(const Ebe& op) {
  return X64Grid{ceil_div(op.nx, TEX), ceil_div(op.ny, TY), ceil_div(op.nz, X64_NZ_TILE)};
}

template <int MODE>
void launch(cudaStream_t s, const Ebe& op, const void* Bimg, double c, const double* x, double* y,
            const double* b, const int* done, double* partials, Scalars* sc, double* pbuf) {
  // two blocks per SM at most: their 256 tensor-memory columns each fill the SM's 512 (a third
  // block would wait in tcgen05.alloc), so the dynamic shared memory is raised until no more fit
  static int smem = 0;
  if (smem == 0) {
    int bytes = SMEM_ALLOC, per_sm = 0;
    CK(cudaFuncSetAttribute(k_ebe3x64_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            110 << 10));
    for (;;) {
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ebe3x64_tiles, NT, bytes));
      if (per_sm <= 2 || bytes >= (110 << 10)) break;
      bytes += 4 << 10;
    }
    smem = bytes;
  }
  if (!pbuf) TOMG_THROW(TOMG_E_INVALID, "FP64 tensor-core element operator without its buffer");
  const X64Grid g = x64_grid(op);
  const dim3 grid(g.gx, g.gy, g.nzc * batch_rhs());
  LAUNCH(k_ebe3x64_tiles, grid, NT, smem, s, op.nx, op.ny, op.nz, X64_NZ_TILE, g.nzc,
         reinterpret_cast<const uint4*>(Bimg), (const double*)op.E, c, op.mask, x, pbuf, done,
         sc);
  const int64_t nn = (int64_t)(op.nx + 1) * (op.ny + 1) * (op.nz + 1);
  LAUNCH((k_ebe3x64_nodes<MODE, X64_NZ_TILE>), dim3(ceil_div(nn, FIN_THREADS * FIN_NPT), batch_rhs()),
         FIN_THREADS, 0, s, op.nx, op.ny, op.nz, g.gx, g.gy, g.nzc, (const double*)pbuf, op.mask,
         x, y, b, done, partials, sc);
}

}  // namespace

bool ebe3x_operand(double nu, uint32_t* img, double* c) {
  // lambda / mu = 2 nu / (1 - 2 nu) = p / q with a small q, so that C = p K_l + q K_m (the
  // 72-scaled integer parts) is an integer matrix whose digit products stay exact in FP32
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));
  const double ratio = lam / mu;
  int q = 0;
  for (int t = 1; t <= 8 && !q; t++)
    if (std::fabs(ratio * t - std::nearbyint(ratio * t)) < 1e-12 * std::max(1.0, ratio * t)) q = t;
  if (!q) return false;
  const double p = std::nearbyint(ratio * q);
  std::vector<double> Kl, Km, Dl(36, 0.0), Dm(36, 0.0);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) Dl[i * 6 + j] = 1.0;
  for (int i = 0; i < 6; i++) Dm[i * 6 + i] = i < 3 ? 2.0 : 1.0;
  element_stiffness_D(3, Dl.data(), Kl);
  element_stiffness_D(3, Dm.data(), Km);
  uint16_t* h = reinterpret_cast<uint16_t*>(img);
  for (int i = 0; i < B_BYTES / 2; i++) h[i] = 0;
  double rowmax = 0.0;
  for (int n = 0; n < KD; n++) {
    double rs = 0.0;
    for (int k = 0; k < KD; k++) {
      const double v = p * 72.0 * Kl[n * KD + k] + q * 72.0 * Km[n * KD + k];
      const double r = std::nearbyint(v);
      if (std::fabs(v - r) > 1e-8 || std::fabs(r) > 2048.0) return false;
      rs += std::fabs(r);
      const __half hv = __double2half(r);
      uint16_t bits;
      std::memcpy(&bits, &hv, 2);
      h[op_off(n, k) / 2] = bits;
    }
    rowmax = std::max(rowmax, rs);
  }
  // digit sums: |sum_k C_nk d_k| <= rowmax x 2047 must stay below 2^22 (exact in FP32 and in
  // the integer conversion)
  if (rowmax * 2047.0 >= 4194304.0) return false;
  *c = mu / (72.0 * q);
  return true;
}

int ebe3x_operand_words() { return B_BYTES / 4; }

int ebe3x_blocks(const Ebe& op) {
  return ceil_div((int64_t)(op.nx + 1) * (op.ny + 1) * (op.nz + 1), FIN_THREADS * FIN_NPT);
}

int64_t ebe3x_buffer_doubles(const Ebe& op) {
  const X64Grid g = x64_grid(op);
  return (int64_t)g.gx * g.gy * g.nzc * LAYER_NODES * (X64_NZ_TILE + 1) * 3;
}

void ebe3x_apply(cudaStream_t s, int mode, const Ebe& op, const void* Bimg, double c,
                 const double* x, double* y, const double* b, const int* done, double* partials,
                 Scalars* sc, double* pbuf) {
  if (mode == MODE_APPLY) launch<MODE_APPLY>(s, op, Bimg, c, x, y, b, done, partials, sc, pbuf);
  else if (mode == MODE_RESID)
    launch<MODE_RESID>(s, op, Bimg, c, x, y, b, done, nullptr, nullptr, pbuf);
  else TOMG_THROW(TOMG_E_INVALID, "FP64 tensor-core element operator: apply and residual only");
}

bool ebe3x_error(cudaStream_t s) {
  int v = 0;
  CK(cudaMemcpyFromSymbolAsync(&v, g_x64_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (v) {
    const int zero = 0;
    CK(cudaMemcpyToSymbolAsync(g_x64_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  return v != 0;
}

}  // namespace tomg
