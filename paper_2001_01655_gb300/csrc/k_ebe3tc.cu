// Level-0 SIMP element operator on hex8 grids (Sec. 2.1 Eq. 2, Sec. 3.1) with the element
// contractions on the fifth-generation tensor cores: tcgen05.mma kind::f16, A operands and
// accumulators in tensor memory, B operand in shared memory.
//
// The element products y_e = Ke x_e of a tile of elements form one dense product
//   Y (elements x 24) = X (elements x 24) . Ke^T (24 x 24)
// whose rows are the gathered element displacement vectors.  Two facts make it cheap on FP16
// tensor cores:
//   * on the unit cube with the 2x2x2 Gauss rule, Ke = lambda K_l + mu K_m where 72 K_l and
//     72 K_m are integer matrices (entries up to 8 and 32): exact in FP16, so B needs no split;
//   * each element row is scaled by a power of two 2^-s (s from its largest |x|), t = x 2^-s,
//     and split into two FP16 parts, h0 = fp16(t) and h1 = fp16(2^11 (t - h0)); the second part
//     is scaled up so that it stays clear of the FP16 subnormal range, and its B half carries
//     the factor 2^-11 (still exact).  t - h0 - 2^-11 h1 is below 2^-22 |t| per entry, plus
//     2^-36 of the row's largest entry for entries under 2^-13 of it: the accuracy of the
//     3xTF32 split products this replaces, with one B operand instead of two.
// One MMA chain of K = 48 (h0 | h1 against K_int | 2^-11 K_int) and N = 48 (K_l rows | K_m
// rows) accumulates both parts in FP32; the epilogue forms
// y_e = E_e 2^s (lambda/72 Z_l + mu/72 Z_m).  That is 3 MMAs (K-steps of 16) per M = 128 tile.
//
// Tiling.  A block owns a column of output nodes: 31 x (TY-1) nodes in x and y and `nz_tile`
// node layers in z.  It walks the element layers under and inside that column.  One element
// layer of the tile is 32 x TY elements = TY / 4 tiles of M = 128; thread (lane ex, warp ey)
// owns element (ex, ey) and, for ex, ey >= 1, node (ex, ey) of the layer tile.  Per layer:
//   1. the masked displacements of the next node layer (33 x (TY+1) nodes) are staged in shared
//      memory, and each thread keeps its element's modulus (both fetched one layer ahead);
//   2. every thread scales and splits its element's 24 displacements and writes them as its row
//      of the A operand in tensor memory (tcgen05.st: lane = row);
//   3. one thread issues 3 MMAs per tile and commits them to an mbarrier;
//   4. while they run, the threads finish the previous element layer: each reads its element's
//      accumulator row (tcgen05.ld) and scales it; node sums over the four elements of the layer
//      around a node take the x-neighbour through a warp shuffle and the y-neighbour through
//      shared memory;
//   5. a node layer is complete after the element layers below and above it, and is then
//      finished (mask, residual or Jacobi / Chebyshev update) and written.
// The accumulators are double-buffered (layer ke's MMAs overlap the finishing of layer ke - 1);
// the A operands are single-buffered and rewritten once the previous layer's MMAs completed.
// The outer ring of nodes of each tile is computed but not written: the neighbouring tile owns
// it, so every node's sum comes from one block, in a fixed order, with no atomics.
// All waits are bounded: a block whose wait for its MMAs runs out sets an error word (read by
// the host after the solve), waits with the full limit for the MMAs it still has in flight,
// releases its tensor memory and returns.
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ops.h"

namespace tomg {

namespace {

constexpr int TEX = 32;                       // elements of one layer of the tile in x
constexpr int TNX = TEX + 1;                  // nodes of one layer of the tile in x (33)
constexpr int ONX = TEX - 1;                  // owned nodes per layer in x (31)
constexpr int KD = 24;                        // element DOFs
constexpr int KA = 2 * KD;                    // K of the product: two FP16 parts of x
constexpr int AW = KA / 2;                    // A row in 32-bit tensor-memory columns (24)
constexpr int NB = 2 * KD;                    // N: K_l rows, then K_m rows (48)
constexpr int KDEN = 72;                      // 72 K_l and 72 K_m are integer matrices
// B operand in shared memory, canonical K-major layout without swizzle: a core matrix is
// 8 rows x 16 bytes (8 FP16); core matrices adjacent in K are LBO bytes apart, adjacent 8-row
// groups SBO bytes apart
constexpr int LBO = 128;
constexpr int SBO = (KA / 8) * LBO;           // 768
constexpr int B_BYTES = (NB / 8) * SBO;       // 4608
constexpr int PS = 7;                         // staged y-pair partial sums: row stride (floats)

// Tile shapes: TY = 8 element rows (256 threads, two M = 128 tiles, 31 x 7 owned nodes per
// layer) or TY = 4 (128 threads, one tile, 31 x 3 owned nodes).  Tensor memory columns: the A
// operand of tile m (24 columns) at 32 m, accumulators of pipeline stage j, tile m at
// ACC + (j MT + m) 48 with ACC = 32 MT (every operand starts on a multiple of 16 columns).
template <int TY>
struct Cfg {
  static constexpr int TNY = TY + 1, ONY = TY - 1;
  static constexpr int NT = TEX * TY;                     // one element per thread
  static constexpr int MT = TY / 4;                       // M = 128 tiles per layer
  static constexpr int LAYER_NODES = TNX * TNY;
  static constexpr int ACC = 32 * MT;                     // after the A operands
  static constexpr int TMEM_COLS = TY == 8 ? 256 : 128;   // a power of 2
  static constexpr int MAX_BLOCKS = 512 / TMEM_COLS;      // blocks per SM the TMEM can hold
  // dynamic shared memory map (bytes from a 128-aligned base)
  static constexpr int OFF_B = 0;                                               // B operand
  static constexpr int OFF_X = OFF_B + B_BYTES;                                 // x ring
  static constexpr int OFF_P = (OFF_X + 2 * LAYER_NODES * 3 * 4 + 15) / 16 * 16;  // y pairs
  static constexpr int OFF_BAR = OFF_P + 2 * NT * PS * 4; // 3 mbarriers + TMEM address
  static constexpr int SMEM_ALLOC = OFF_BAR + 32 + 128;   // + room to align the base
  static_assert(AW * MT <= ACC && ACC + 2 * MT * NB <= TMEM_COLS, "tensor memory map");
  static_assert(OFF_X % 16 == 0 && OFF_P % 16 == 0 && OFF_BAR % 8 == 0, "alignment");
  static_assert(LAYER_NODES <= 2 * NT, "two nodes per thread stage a layer");
};

// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B FP16 (bits 7-9 and 10-12
// = 0), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(NB >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

constexpr uint32_t WAIT_LIMIT = 1u << 22;  // mbarrier polls before a block gives up

__device__ int g_tc_error;  // set to 1 by a block whose MMA completion wait ran out

// test hook (tomg_debug_tc_wait_limit): polls > 0 makes the in-loop MMA waits of later launches
// watch a third barrier that nothing arrives on and give up after that many polls, so that the
// error path runs exactly as after a real timeout (the MMAs complete on their own barrier,
// which the drain then waits for with the full limit)
int g_first_wait_limit = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), fixed 0b001 at
// bits 46-48, base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(LBO >> 4) << 16) |
         ((uint64_t)(SBO >> 4) << 32) | (1ull << 46);
}

// byte offset of element (row, k) in the B operand layout above
__host__ __device__ __forceinline__ int op_off(int row, int k) {
  return (row >> 3) * SBO + (k >> 3) * LBO + (row & 7) * 16 + (k & 7) * 2;
}

// D (tmem) (+)= A (tmem) . B (smem descriptor)^T
__device__ __forceinline__ void mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b,
                                           uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
      :: "r"(d_tmem), "r"(a_tmem), "l"(b), "r"(IDESC), "r"(acc) : "memory");
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

// bounded wait for the phase of the barrier with parity `parity`; true if it completed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; i++)
    if (mbar_try(bar, parity)) return true;
  return false;
}

// this thread's TMEM lane, 48 consecutive FP32 columns from taddr (16-column aligned); the wait
// for the loads is part of the same asm statement, so no use of the registers can be
// scheduled before it
__device__ __forceinline__ void tmem_ld48(uint32_t taddr, float* v) {
  uint32_t r[48];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%48];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,"
      "%28,%29,%30,%31}, [%49];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,"
      "%44,%45,%46,%47}, [%50];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]),
        "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]),
        "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
      : "r"(taddr), "r"(taddr + 16u), "r"(taddr + 32u)
      : "memory");
#pragma unroll
  for (int i = 0; i < 48; i++) v[i] = __uint_as_float(r[i]);
}

// this thread's TMEM lane, 24 consecutive 32-bit columns from taddr (8-column aligned); the
// wait for the stores is part of the same asm statement
__device__ __forceinline__ void tmem_st24(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17};\n\t"
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%18,%19,%20,%21,%22,%23,%24,%25};\n\t"
      "tcgen05.wait::st.sync.aligned;\n"
      :: "r"(taddr), "r"(taddr + 16u), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]),
         "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]),
         "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
         "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23])
      : "memory");
}

// Input transforms of a Chebyshev step that fuses the kernel before it: the iterate of the step
// is formed where it is read (in the layer ring and for the owned nodes), with the same device
// functions as the kernels it replaces, so the results are bit-identical to the unfused pair.
//   XF_NONE  x as stored
//   XF_JAC0  x = w0 Dinv b       (the first step from x = 0: the k_jacobi0 sweep)
//   XF_PROL  x = x + P xc        (the coarse correction: the k_prolong_add pass)
enum { XF_NONE = 0, XF_JAC0 = 1, XF_PROL = 2 };
struct XfArg {
  const float* Dinv;
  const float* xc;  // coarse correction (XF_PROL), grid cnx x cny x cnz
  int cnx, cny, cnz;
  float w0;         // weight of the first step (XF_JAC0)
};

// one node layer of the tile: displacements (XF_JAC0: right-hand sides) and mask bits of up to
// two nodes per thread.  The loads are independent (the mask and the transform are applied when
// the layer is stored), so a prefetch issued at the top of a layer step never stalls the thread
// before the values are needed.
struct XPre {
  float v[2][3];
  unsigned m[2];
};

template <int TY, int XF>
__device__ __forceinline__ void x_fetch(XPre& p, int kk, int EX0, int EY0, int nx, int ny, int nz,
                                        const uint8_t* __restrict__ mask,
                                        const float* __restrict__ x, const float* __restrict__ b) {
  const float* src = XF == XF_JAC0 ? b : x;
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int q = threadIdx.x + h * Cfg<TY>::NT;
    p.v[h][0] = p.v[h][1] = p.v[h][2] = 0.f;
    p.m[h] = 7u;
    if (q < Cfg<TY>::LAYER_NODES) {
      const int gi = EX0 + q % TNX, gj = EY0 + q / TNX;
      if (gi >= 0 && gi <= nx && gj >= 0 && gj <= ny && kk >= 0 && kk <= nz) {
        const int64_t node = node_id(gi, gj, kk, nx, ny);
        p.m[h] = __ldg(mask + node);
#pragma unroll
        for (int c = 0; c < 3; c++) p.v[h][c] = __ldg(src + 3 * node + c);
      }
    }
  }
}

// the fused input transform at one node (v: x, or b for XF_JAC0)
template <int XF>
__device__ __forceinline__ void x_transform(float* v, int gi, int gj, int kk, int64_t node,
                                            int nx, int ny, int nz, const XfArg& xa) {
  if (XF == XF_JAC0) {
    float D[9], bv[3];
#pragma unroll
    for (int t = 0; t < 9; t++) D[t] = __ldg(xa.Dinv + 9 * node + t);
#pragma unroll
    for (int c = 0; c < 3; c++) bv[c] = v[c];
    jacobi_block<float, 3>(D, bv, xa.w0, v);
  } else if (XF == XF_PROL) {
    prolong_node<float, 3>(gi, gj, kk, nx, ny, nz, xa.cnx, xa.cny, xa.xc, v);
  }
}

template <int TY, int XF>
__device__ __forceinline__ void x_store(XPre& p, float* sx, int kk, int EX0, int EY0, int nx,
                                        int ny, int nz, const XfArg& xa) {
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int q = threadIdx.x + h * Cfg<TY>::NT;
    if (q < Cfg<TY>::LAYER_NODES) {
      // a node outside the grid has all three bits set, as has one fixed in every direction:
      // neither needs the transform (its values are stored as zero)
      if (XF != XF_NONE && p.m[h] != 7u) {
        const int gi = EX0 + q % TNX, gj = EY0 + q / TNX;
        x_transform<XF>(p.v[h], gi, gj, kk, node_id(gi, gj, kk, nx, ny), nx, ny, nz, xa);
      }
#pragma unroll
      for (int c = 0; c < 3; c++) sx[3 * q + c] = ((p.m[h] >> c) & 1u) ? 0.f : p.v[h][c];
    }
  }
}

// what finishing an owned node needs besides its sum: x (unmasked), mask, b, block inverse
struct FinData {
  float x[3], b[3], D[9];
  unsigned m;
};

template <int MODE, int XF>
__device__ __forceinline__ void fin_fetch(FinData& f, bool valid, int gi, int gj, int kk, int nx,
                                          int ny, int nz, const uint8_t* __restrict__ mask,
                                          const float* __restrict__ x,
                                          const float* __restrict__ b,
                                          const float* __restrict__ Dinv, const XfArg& xa) {
  if (!valid) return;
  const int64_t node = node_id(gi, gj, kk, nx, ny);
  f.m = __ldg(mask + node);
  if (MODE != MODE_APPLY) {
#pragma unroll
    for (int c = 0; c < 3; c++) f.b[c] = __ldg(b + 3 * node + c);
  }
  if (MODE == MODE_JACOBI || MODE == MODE_CHEB) {
#pragma unroll
    for (int c = 0; c < 9; c++) f.D[c] = __ldg(Dinv + 9 * node + c);
  }
  if (XF == XF_JAC0) {
    jacobi_block<float, 3>(f.D, f.b, xa.w0, f.x);
  } else {
#pragma unroll
    for (int c = 0; c < 3; c++) f.x[c] = __ldg(x + 3 * node + c);
    if (XF == XF_PROL) x_transform<XF_PROL>(f.x, gi, gj, kk, node, nx, ny, nz, xa);
  }
}

__device__ __forceinline__ float e_fetch(int ke, int EX0, int EY0, int nx, int ny, int nz,
                                         const float* __restrict__ E) {
  const int ge = EX0 + (int)(threadIdx.x % TEX), gf = EY0 + (int)(threadIdx.x / TEX);
  if (ge < 0 || ge >= nx || gf < 0 || gf >= ny || ke < 0 || ke >= nz) return 0.f;
  return __ldg(E + ge + (int64_t)nx * (gf + (int64_t)ny * ke));
}

// element (ex, ey) of layer ke: its 24 displacements from the ring slots of node layers ke
// (bottom, local nodes 0-3) and ke + 1 (top, local nodes 4-7), scaled by 2^-s so that the
// largest magnitude lies in [1/2, 1), t = x 2^-s, and split into FP16 parts h0 = fp16(t) and
// h1 = fp16(2^11 (t - h0)): the thread's row of the A operand, K order (h0 of DOFs 0..23, h1
// of DOFs 0..23), two FP16 per 32-bit word (lower K index in the low half).  Returns 2^s.
__device__ __forceinline__ float a_row(uint32_t* w, const float* s0, const float* s1, int ex,
                                       int ey) {
  float xv[KD];
  float amax = 0.f;
#pragma unroll
  for (int k = 0; k < KD; k++) {
    const int bn = k / 3, c = k % 3;
    const float* sx = (bn & 4) ? s1 : s0;
    xv[k] = sx[3 * ((ey + ((bn >> 1) & 1)) * TNX + ex + (bn & 1)) + c];
    amax = fmaxf(amax, fabsf(xv[k]));
  }
  // 2^s with amax 2^-s in [1/2, 1): s = biased exponent of amax - 126 (a zero or subnormal
  // row keeps s = 0: its parts then flush below the FP16 range, far below the FP32 rounding of
  // any row that matters)
  const int be = (int)((__float_as_uint(amax) >> 23) & 0xffu);
  const int s = be > 0 ? min(be - 126, 127) : 0;                  // in [-125, 127]
  const float down = __uint_as_float((uint32_t)(127 - s) << 23);  // 2^-s
  const float up = __uint_as_float((uint32_t)(127 + s) << 23);    // 2^s
  // h0 pairs packed by one conversion each; h1 from the exact remainder t - h0
#pragma unroll
  for (int c = 0; c < KD / 2; c++) {
    const float ta = xv[2 * c] * down, tb = xv[2 * c + 1] * down;
    const __half2 p0 = __floats2half2_rn(ta, tb);
    const float2 h0 = __half22float2(p0);
    const __half2 p1 = __floats2half2_rn(2048.f * (ta - h0.x), 2048.f * (tb - h0.y));
    w[c] = *reinterpret_cast<const uint32_t*>(&p0);
    w[KD / 2 + c] = *reinterpret_cast<const uint32_t*>(&p1);
  }
  return up;
}

// MT M-tiles x 3 K-steps of M128 N48 K16 into the accumulators at column d, then a commit to the
// barrier (executed by one thread)
template <int MT>
__device__ __forceinline__ void issue_mmas(uint32_t d, uint32_t a, uint32_t bbase, uint32_t bar) {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
  for (int m = 0; m < MT; m++) {
#pragma unroll
    for (int s = 0; s < KA / 16; s++)
      mma_f16_ts(d + (uint32_t)(m * NB), a + (uint32_t)(32 * m + 8 * s),
                 sdesc(bbase + 2 * LBO * s), s ? 1u : 0u);
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
               :: "r"(bar) : "memory");
}

template <int MODE, int TY, int XF>
__global__ void __launch_bounds__(Cfg<TY>::NT, Cfg<TY>::MAX_BLOCKS)
k_ebe3tc(int nx, int ny, int nz, int nz_tile, const uint4* __restrict__ Bimg,
         const float* __restrict__ E, const uint8_t* __restrict__ mask,
         const float* __restrict__ x, float* __restrict__ y, const float* __restrict__ b,
         const float* __restrict__ Dinv, float omega, const int* done, float* __restrict__ dch,
         float c1, int dmode, float cl, float cm, uint32_t wait_limit, int nzc, XfArg xa) {
  using C = Cfg<TY>;
  constexpr int NT = C::NT, LAYER_NODES = C::LAYER_NODES, ONY = C::ONY, MT = C::MT;
  constexpr int OFF_B = C::OFF_B, OFF_X = C::OFF_X, OFF_P = C::OFF_P, OFF_BAR = C::OFF_BAR;
  constexpr int ACC = C::ACC, TMEM_COLS = C::TMEM_COLS;
  extern __shared__ uint8_t smem_raw[];
  pdl_prologue();
  if (solve_done(done)) return;
  uint8_t* sm = smem_raw + ((128 - (smem_u32(smem_raw) & 127u)) & 127u);
  float* sxr = reinterpret_cast<float*>(sm + OFF_X);          // [2][LAYER_NODES][3]
  float* sP = reinterpret_cast<float*>(sm + OFF_P);           // [2][TY][TEX][PS]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + OFF_BAR);  // [3]; [2] never arrives
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + OFF_BAR + 24);
  const uint32_t sbase = smem_u32(sm);
  const uint32_t bar0 = smem_u32(bar);  // barrier j at bar0 + 8 j
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ex = lane, ey = warp;  // element of this thread; node (ex, ey) if owned

  const int EX0 = blockIdx.x * ONX - 1, EY0 = blockIdx.y * ONY - 1;
  // blockIdx.z = chunk of node layers + nzc x right-hand side of a block solve
  const int zc = blockIdx.z % nzc, rhs = blockIdx.z / nzc;
  {
    const int64_t vo = (int64_t)rhs * rhs_stride((int64_t)3 * (nx + 1) * (ny + 1) * (nz + 1));
    if (x) x += vo;
    y += vo;
    if (b) b += vo;
    if (dch) dch += vo;
    if (XF == XF_PROL)
      xa.xc += (int64_t)rhs * rhs_stride((int64_t)3 * (xa.cnx + 1) * (xa.cny + 1) * (xa.cnz + 1));
  }
  const int k0 = zc * nz_tile;
  const int k1 = min(k0 + nz_tile, nz + 1);  // owned node layers [k0, k1)

  // tensor memory (one warp), the MMA barriers, the B operand
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 :: "r"(smem_u32(tmem_slot)), "r"(TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(bar0), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(bar0 + 8u), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(bar0 + 16u), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  for (int t = tid; t < B_BYTES / 16; t += NT)
    reinterpret_cast<uint4*>(sm + OFF_B)[t] = Bimg[t];

  const bool owner = ex >= 1 && ey >= 1;
  const int gi = EX0 + ex, gj = EY0 + ey;
  const bool in_plane = owner && gi <= nx && gj <= ny;

  XPre pre, pre2;
  x_fetch<TY, XF>(pre, k0 - 1, EX0, EY0, nx, ny, nz, mask, x, b);
  x_fetch<TY, XF>(pre2, k0, EX0, EY0, nx, ny, nz, mask, x, b);
  x_store<TY, XF>(pre, sxr + ((k0 - 1) & 1) * LAYER_NODES * 3, k0 - 1, EX0, EY0, nx, ny, nz, xa);
  x_store<TY, XF>(pre2, sxr + (k0 & 1) * LAYER_NODES * 3, k0, EX0, EY0, nx, ny, nz, xa);
  x_fetch<TY, XF>(pre, k0 + 1, EX0, EY0, nx, ny, nz, mask, x, b);  // stored after layer k0 - 1
  float e_cur = e_fetch(k0 - 1, EX0, EY0, nx, ny, nz, E);  // modulus of element layer ke
  float e_prev = 0.f;                                      // ... of layer ke - 1
  float sc_prev = 1.f;                                     // 2^s of the row of layer ke - 1
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const int mt = warp >> 2;  // M-tile of this thread's element row (TY = 8: two tiles)

  float acc[3] = {0.f, 0.f, 0.f};  // node layer ke - 1: contributions gathered so far
  FinData fd;                      // finishing data of node layer ke - 1
  uint32_t parity = 0;             // bit j: phase of barrier j to wait for next
  uint32_t pending = 0;            // bit j: MMAs committed to barrier j not yet seen complete
  bool failed = false;

  for (int ke = k0 - 1; ke <= k1; ke++) {
    const bool mma_now = ke < k1;  // the last step only finishes layer k1 - 1
    const int j = ke & 1, jp = j ^ 1;
    bool ok = true;
    if (ke >= k0) {
      // the MMAs of layer ke - 1 (every thread waits itself): their accumulators are read
      // below, their A operands are overwritten now.  The phase bit advances only on success,
      // so that a block that gives up still knows which phase its MMAs in flight complete.
      const bool probe = wait_limit < WAIT_LIMIT;  // test hook: a barrier nothing completes
      ok = mbar_wait(probe ? bar0 + 16u : bar0 + 8u * jp, probe ? 0u : (parity >> jp) & 1u,
                     wait_limit);
      if (ok) {
        parity ^= 1u << jp;
        pending &= ~(1u << jp);
      }
      // the tensor-memory stores and loads below are warp-collective: a warp takes part only
      // if every lane saw the MMAs complete (otherwise the whole block gives up below)
      ok = __all_sync(0xffffffffu, ok);
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    float sc_now = 1.f;
    if (ok && mma_now) {
      uint32_t w[AW];
      sc_now = a_row(w, sxr + j * LAYER_NODES * 3, sxr + jp * LAYER_NODES * 3, ex, ey);
      tmem_st24(tmem + lane_base + (uint32_t)(32 * mt), w);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    if (__syncthreads_or(!ok)) {  // a wait that ran out anywhere stops the whole block
      failed = true;
      break;
    }
    if (mma_now) {
      if (tid == 0)
        issue_mmas<MT>(tmem + (uint32_t)(ACC + j * MT * NB), tmem, sbase + OFF_B, bar0 + 8u * j);
      pending |= 1u << j;
    }
    // refill the ring: node layer ke + 2 replaces layer ke (read by the row build above)
    if (mma_now && ke + 2 <= k1) {
      x_store<TY, XF>(pre, sxr + j * LAYER_NODES * 3, ke + 2, EX0, EY0, nx, ny, nz, xa);
      if (ke + 3 <= k1) x_fetch<TY, XF>(pre, ke + 3, EX0, EY0, nx, ny, nz, mask, x, b);
    }
    const float e_next = (ke + 1 < k1) ? e_fetch(ke + 1, EX0, EY0, nx, ny, nz, E) : 0.f;
    // finishing data of node layer ke, used one step later
    FinData fd_next;
    const bool fin_next = in_plane && ke >= k0 && ke < k1;
    fin_fetch<MODE, XF>(fd_next, fin_next, gi, gj, ke, nx, ny, nz, mask, x, b, Dinv, xa);

    float pr[2][2][3];  // x-pair sums of element layer ke - 1 at node column ex: [dy][dz][c]
    if (ke >= k0) {
      // finish element layer ke - 1 and node layer ke - 1
      float v[NB];
      tmem_ld48(tmem + lane_base + (uint32_t)(ACC + (jp * MT + mt) * NB), v);
      const float sl = e_prev * sc_prev * cl, sm_ = e_prev * sc_prev * cm;
#pragma unroll
      for (int n = 0; n < KD; n++) v[n] = sl * v[n] + sm_ * v[KD + n];
      // x-pairs: node column ex gets the dx = 1 corners of element ex - 1 (previous lane) and
      // the dx = 0 corners of element ex; p[dy][dz][c]
#pragma unroll
      for (int dy = 0; dy < 2; dy++)
#pragma unroll
        for (int dz = 0; dz < 2; dz++)
#pragma unroll
          for (int c = 0; c < 3; c++) {
            const float left = __shfl_up_sync(0xffffffffu, v[3 * (1 + 2 * dy + 4 * dz) + c], 1);
            pr[dy][dz][c] = v[3 * (2 * dy + 4 * dz) + c] + left;  // lane 0: not an owned node
          }
      // y-pairs: node row ey gets the dy = 1 sums of element row ey - 1 through shared memory
      float* myP = sP + (j * NT + ey * TEX + ex) * PS;
#pragma unroll
      for (int dz = 0; dz < 2; dz++)
#pragma unroll
        for (int c = 0; c < 3; c++) myP[3 * dz + c] = pr[1][dz][c];
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    }
    // makes the y-pair partials and the ring layer stored above visible to the block
    __syncthreads();
    if (ke >= k0) {
      const int kn = ke - 1;
      const bool fin = in_plane && kn >= k0;
      const int64_t node = node_id(gi, gj, kn, nx, ny);
      if (owner) {
        const float* upP = sP + (j * NT + (ey - 1) * TEX + ex) * PS;
        float top[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
          acc[c] += upP[c] + pr[0][0][c];
          top[c] = upP[3 + c] + pr[0][1][c];
        }
        if (fin) {
          float Ax[3];
#pragma unroll
          for (int c = 0; c < 3; c++) Ax[c] = ((fd.m >> c) & 1u) ? fd.x[c] : acc[c];
          if (MODE == MODE_APPLY) {
#pragma unroll
            for (int c = 0; c < 3; c++) y[3 * node + c] = Ax[c];
          } else {
            float r[3];
#pragma unroll
            for (int c = 0; c < 3; c++) r[c] = fd.b[c] - Ax[c];
            if (MODE == MODE_RESID) {
#pragma unroll
              for (int c = 0; c < 3; c++) y[3 * node + c] = r[c];
            } else if (MODE == MODE_CHEB) {
#pragma unroll
              for (int c = 0; c < 3; c++) {
                const float v = fd.D[3 * c] * r[0] + fd.D[3 * c + 1] * r[1] + fd.D[3 * c + 2] * r[2];
                const float prev = dmode == 2 ? fd.x[c] : (dmode == 1 ? dch[3 * node + c] : 0.f);
                const float dn = c1 * prev + omega * v;
                y[3 * node + c] = fd.x[c] + dn;
                dch[3 * node + c] = dn;
              }
            } else {
#pragma unroll
              for (int c = 0; c < 3; c++)
                y[3 * node + c] = fd.x[c] + omega * (fd.D[3 * c] * r[0] + fd.D[3 * c + 1] * r[1] +
                                                     fd.D[3 * c + 2] * r[2]);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 3; c++) acc[c] = top[c];
      }
    }
    e_prev = e_cur;
    e_cur = e_next;
    sc_prev = sc_now;
    fd = fd_next;
  }

  if (failed) {
    if (tid == 0) atomicExch(&g_tc_error, 1);
    // MMAs still in flight write their accumulators until they complete: wait for them with
    // the full limit before the tensor memory is released
#pragma unroll
    for (int q = 0; q < 2; q++)
      if ((pending >> q) & 1u) mbar_wait(bar0 + 8u * q, (parity >> q) & 1u, WAIT_LIMIT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n"
                 :: "r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

template <int MODE, int TY, int XF>
void launch_tile(cudaStream_t s, const Ebe& op, const float* x, float* y, const float* b,
                 const float* Dinv, double omega, const int* done, const ChebArg* ch) {
  using C = Cfg<TY>;
  // dynamic shared memory per block, raised if needed so that the blocks sharing an SM never
  // ask for more than its 512 tensor-memory columns (a further block would wait in
  // tcgen05.alloc)
  static int smem = 0;  // per instantiation
  if (smem == 0) {
    int bytes = C::SMEM_ALLOC, per_sm = 0;
    CK(cudaFuncSetAttribute(k_ebe3tc<MODE, TY, XF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            100 << 10));
    for (;;) {
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ebe3tc<MODE, TY, XF>, C::NT,
                                                       bytes));
      if (per_sm <= C::MAX_BLOCKS || bytes >= (100 << 10)) break;
      bytes += 4 << 10;
    }
    smem = bytes;
  }
  const int nzt = op.tc_nz > 0 ? op.tc_nz : 8;
  const int nzc = ceil_div(op.nz + 1, nzt);
  dim3 grid(ceil_div(op.nx + 1, ONX), ceil_div(op.ny + 1, C::ONY), nzc * batch_rhs());
  if (MODE == MODE_CHEB && !ch) TOMG_THROW(TOMG_E_INVALID, "Chebyshev step without its state");
  float* dch = MODE == MODE_CHEB ? (float*)ch->d : nullptr;
  const float c1 = MODE == MODE_CHEB ? (float)ch->c1 : 0.f;
  const int dm = XF == XF_JAC0 ? 2 : (MODE == MODE_CHEB ? ch->dmode : 0);
  XfArg xa{Dinv, nullptr, 0, 0, 0, 0.f};
  if (XF == XF_JAC0) xa.w0 = (float)ch->w0;
  if (XF == XF_PROL) {
    if (ch->dmode != 0) TOMG_THROW(TOMG_E_INVALID, "fused prolongation on a later step");
    xa.xc = static_cast<const float*>(ch->xc);
    xa.cnx = ch->cnx;
    xa.cny = ch->cny;
    xa.cnz = ch->cnz;
  }
  const uint32_t wl = g_first_wait_limit > 0 ? (uint32_t)g_first_wait_limit : WAIT_LIMIT;
  LAUNCH((k_ebe3tc<MODE, TY, XF>), grid, C::NT, smem, s, op.nx, op.ny, op.nz, nzt,
         reinterpret_cast<const uint4*>(op.Ktc), (const float*)op.E, op.mask, x, y, b, Dinv,
         (float)omega, done, dch, c1, dm, op.tc_cl, op.tc_cm, wl, nzc, xa);
}

template <int MODE, int XF = XF_NONE>
void launch_mode(cudaStream_t s, const Ebe& op, const float* x, float* y, const float* b,
                 const float* Dinv, double omega, const int* done, const ChebArg* ch = nullptr) {
  if (op.tc_ty == 4) launch_tile<MODE, 4, XF>(s, op, x, y, b, Dinv, omega, done, ch);
  else launch_tile<MODE, 8, XF>(s, op, x, y, b, Dinv, omega, done, ch);
}

}  // namespace

void ebe3d_tc_operand(double nu, uint32_t* img, float* cl, float* cm) {
  // K_l, K_m: the hex8 element stiffness of D = m m^T and of D = diag(2, 2, 2, 1, 1, 1); Ke =
  // lambda K_l + mu K_m for E = 1.  Rows 0..23 of B are 72 K_l, rows 24..47 are 72 K_m (both
  // symmetric, so row n is also column n): K columns 0..23 (against h0) hold the integers,
  // K columns 24..47 (against h1 = 2^11 (t - h0)) hold them times 2^-11.
  std::vector<double> Kl, Km;
  std::vector<double> Dl(36, 0.0), Dm(36, 0.0);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) Dl[i * 6 + j] = 1.0;
  for (int i = 0; i < 6; i++) Dm[i * 6 + i] = i < 3 ? 2.0 : 1.0;
  element_stiffness_D(3, Dl.data(), Kl);
  element_stiffness_D(3, Dm.data(), Km);
  uint16_t* h = reinterpret_cast<uint16_t*>(img);
  for (int i = 0; i < B_BYTES / 2; i++) h[i] = 0;
  for (int n = 0; n < NB; n++)
    for (int k = 0; k < KD; k++) {
      const double v = KDEN * (n < KD ? Kl[n * KD + k] : Km[(n - KD) * KD + k]);
      const double r = std::nearbyint(v);
      if (std::fabs(v - r) > 1e-9 || std::fabs(r) > 2048.0)
        TOMG_THROW(TOMG_E_INVALID, "element stiffness part is not a small integer / 72");
      const __half hv = __double2half(r);             // exact: |r| <= 2048
      const __half hs = __double2half(r / 2048.0);    // exact: a power-of-two scaling, normal
      uint16_t bits, bits_s;
      std::memcpy(&bits, &hv, 2);
      std::memcpy(&bits_s, &hs, 2);
      h[op_off(n, k) / 2] = bits;
      h[op_off(n, KD + k) / 2] = bits_s;
    }
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));
  *cl = (float)(lam / KDEN);
  *cm = (float)(mu / KDEN);
}

int ebe3d_tc_operand_words() { return B_BYTES / 4; }

void ebe3d_tc_launch(cudaStream_t s, int mode, const Ebe& op, const float* x, float* y,
                     const float* b, const float* Dinv, double omega, const int* done,
                     const ChebArg* ch) {
  if (mode == MODE_APPLY) launch_mode<MODE_APPLY>(s, op, x, y, b, Dinv, omega, done);
  else if (mode == MODE_RESID) launch_mode<MODE_RESID>(s, op, x, y, b, Dinv, omega, done);
  else if (mode == MODE_CHEB0)  // the first sweep from x = 0 fused into the second step
    launch_mode<MODE_CHEB, XF_JAC0>(s, op, nullptr, y, b, Dinv, omega, done, ch);
  else if (mode == MODE_CHEB && ch && ch->xc)  // the prolongation fused into the first step
    launch_mode<MODE_CHEB, XF_PROL>(s, op, x, y, b, Dinv, omega, done, ch);
  else if (mode == MODE_CHEB) launch_mode<MODE_CHEB>(s, op, x, y, b, Dinv, omega, done, ch);
  else launch_mode<MODE_JACOBI>(s, op, x, y, b, Dinv, omega, done);
}

// fastest tile shape for this grid (element rows per block 8 or 4, node layers per block 4 to
// 32): each candidate timed on the stream with scratch vectors the first time a grid shape is
// seen, cached per shape afterwards.  Returns rows * 1000 + layers.
int ebe3d_tc_autotune(cudaStream_t s, const Ebe& op, const float* Dinv) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, int> cache;
  const auto key = std::make_tuple(op.nx, op.ny, op.nz);
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  const int64_t n = 3 * (int64_t)(op.nx + 1) * (op.ny + 1) * (op.nz + 1);
  DBuf<float> x, y, b;
  x.resize(n);
  y.resize(n);
  b.resize(n);
  x.zero(s);
  b.zero(s);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int best = 8, best_ty = 8;
  float best_ms = 1e30f;
  // node layers per block: powers of two, and the sizes that split the node layers into 2-12
  // near-equal chunks (each chunk computes one more element layer than it owns, so fewer,
  // even chunks waste less)
  std::vector<int> nzs = {8, 4, 16, 32};
  for (int k = 2; k <= 12; k++) {
    const int t = (op.nz + 1 + k - 1) / k;
    if (t >= 4 && t <= 64 && std::find(nzs.begin(), nzs.end(), t) == nzs.end()) nzs.push_back(t);
  }
  const int nc = (int)nzs.size();
  for (int cand = 0; cand < 2 * nc; cand++) {
    const int ty = cand < nc ? 8 : 4;
    const int nzt = nzs[cand % nc];
    if (nzt > 8 && nzt / 2 >= op.nz + 1) continue;  // no more blocks to split off
    Ebe o = op;
    o.tc_nz = nzt;
    o.tc_ty = ty;
    launch_mode<MODE_JACOBI>(s, o, x.p, y.p, b.p, Dinv, 0.5, nullptr);
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < 5; r++) launch_mode<MODE_JACOBI>(s, o, x.p, y.p, b.p, Dinv, 0.5, nullptr);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < 0.97f * best_ms) {
      best_ms = ms;
      best = nzt;
      best_ty = ty;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int code = best_ty * 1000 + best;
  std::lock_guard<std::mutex> g(mu);
  cache[key] = code;
  return code;
}

// reads and clears the error word of the tensor-core kernel (synchronises the stream)
bool ebe3d_tc_error(cudaStream_t s) {
  int v = 0;
  CK(cudaMemcpyFromSymbolAsync(&v, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (v) {
    const int zero = 0;
    CK(cudaMemcpyToSymbolAsync(g_tc_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  return v != 0;
}

// polls of the in-loop MMA completion waits of later launches (0 restores the default)
void ebe3d_tc_set_wait_limit(int polls) { g_first_wait_limit = polls > 0 ? polls : 0; }

}  // namespace tomg
