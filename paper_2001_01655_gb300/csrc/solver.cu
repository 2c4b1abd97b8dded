// Host runtime: problem state, preconditioner setup (Sec. 3.2 Eq. 9, Sec. 4), the V-cycle of
// Algorithm 1 with point-block Jacobi smoothing, and the outer CG / flexible-CG loop (Sec. 3.1)
// whose iteration is captured once into a CUDA graph with a device-side while loop, so a
// whole solve is one graph launch with no host round trip per iteration.  Several right-hand
// sides run on concurrent solve slots that share the hierarchy.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <chrono>
#include <cstdio>

#include "solver.h"

namespace tomg {



// ----------------------------------------------------------------------------------------
// element stiffness by 2x2(x2) Gauss quadrature on the unit element (bilinear quad4 plane
// stress, trilinear hex8 isotropic); local node a = (a&1, a>>1&1, a>>2&1), DOF = dim*a + c
void element_stiffness_host(int dim, double nu, std::vector<double>& Ke) {
  const int ns = dim == 2 ? 3 : 6;
  std::vector<double> D(ns * ns, 0.0);
  if (dim == 2) {
    const double c = 1.0 / (1.0 - nu * nu);
    D[0] = c; D[1] = c * nu; D[3] = c * nu; D[4] = c; D[8] = c * 0.5 * (1.0 - nu);
  } else {
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) D[i * 6 + j] = lam + (i == j ? 2.0 * mu : 0.0);
    for (int i = 3; i < 6; i++) D[i * 6 + i] = mu;
  }
  element_stiffness_D(dim, D.data(), Ke);
}

void element_stiffness_D(int dim, const double* D, std::vector<double>& Ke) {
  const int nn = 1 << dim, nd = dim * nn, ns = dim == 2 ? 3 : 6;
  Ke.assign(nd * nd, 0.0);
  const double g[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
  const double w = std::pow(0.5, dim);
  std::vector<double> B(ns * nd), DB(ns * nd);
  for (int p = 0; p < nn; p++) {
    double xi[3] = {g[p & 1], g[(p >> 1) & 1], g[(p >> 2) & 1]};
    std::fill(B.begin(), B.end(), 0.0);
    for (int a = 0; a < nn; a++) {
      double G[3];
      for (int k = 0; k < dim; k++) {
        double v = ((a >> k) & 1) ? 1.0 : -1.0;
        for (int m = 0; m < dim; m++)
          if (m != k) v *= ((a >> m) & 1) ? xi[m] : 1.0 - xi[m];
        G[k] = v;
      }
      if (dim == 2) {
        B[0 * nd + 2 * a] = G[0];
        B[1 * nd + 2 * a + 1] = G[1];
        B[2 * nd + 2 * a] = G[1];
        B[2 * nd + 2 * a + 1] = G[0];
      } else {
        const int c = 3 * a;
        B[0 * nd + c] = G[0];
        B[1 * nd + c + 1] = G[1];
        B[2 * nd + c + 2] = G[2];
        B[3 * nd + c + 1] = G[2]; B[3 * nd + c + 2] = G[1];
        B[4 * nd + c] = G[2];     B[4 * nd + c + 2] = G[0];
        B[5 * nd + c] = G[1];     B[5 * nd + c + 1] = G[0];
      }
    }
    for (int i = 0; i < ns; i++)
      for (int j = 0; j < nd; j++) {
        double v = 0.0;
        for (int k = 0; k < ns; k++) v += D[i * ns + k] * B[k * nd + j];
        DB[i * nd + j] = v;
      }
    for (int i = 0; i < nd; i++)
      for (int j = 0; j < nd; j++) {
        double v = 0.0;
        for (int k = 0; k < ns; k++) v += B[k * nd + i] * DB[k * nd + j];
        Ke[i * nd + j] += w * v;
      }
  }
  for (int i = 0; i < nd; i++)  // exact symmetry
    for (int j = i + 1; j < nd; j++) {
      const double v = 0.5 * (Ke[i * nd + j] + Ke[j * nd + i]);
      Ke[i * nd + j] = Ke[j * nd + i] = v;
    }
}

namespace {

// typed views of the per-precision buffers
template <class T> struct V;
template <> struct V<double> {
  static const double* S(const Level& l) { return l.S64.p; }
  static const double* Vv(const Level& l) { return l.V64.p; }
  static const double* D(const Level& l) { return l.D64.p; }
  static const double* Pv(const Level& l) { return l.Pv64.p; }
  static const double* Rv(const Level& l) { return l.Rv64.p; }
  static double* b(LevelWork& l) { return l.b64.p; }
  static double* x(LevelWork& l) { return l.x64.p; }
  static double* r(LevelWork& l) { return l.r64.p; }
  static double* y(LevelWork& l) { return l.y64.p; }
  static double* gV(LevelWork& l) { return l.gV64.p; }
  static double* gZ(LevelWork& l) { return l.gZ64.p; }
  static const double* Ainv(const tomg_problem* P) { return P->Ainv64.p; }
  static Ebe ebe(const tomg_problem* P) {
    return Ebe{P->dim, P->nx, P->ny, P->nz, P->Ke64.p, P->E64.p, P->mask.p, 0, P->Ke_host.data()};
  }
};
template <> struct V<float> {
  static const float* S(const Level& l) { return l.S32.p; }
  static const float* Vv(const Level& l) { return l.V32.p; }
  static const float* D(const Level& l) { return l.D32.p; }
  static const float* Pv(const Level& l) { return l.Pv32.p; }
  static const float* Rv(const Level& l) { return l.Rv32.p; }
  static float* b(LevelWork& l) { return l.b32.p; }
  static float* x(LevelWork& l) { return l.x32.p; }
  static float* r(LevelWork& l) { return l.r32.p; }
  static float* y(LevelWork& l) { return l.y32.p; }
  static float* gV(LevelWork& l) { return l.gV32.p; }
  static float* gZ(LevelWork& l) { return l.gZ32.p; }
  static const float* Ainv(const tomg_problem* P) { return P->Ainv32.p; }
  static Ebe ebe(const tomg_problem* P) {
    Ebe op{P->dim, P->nx, P->ny, P->nz, P->Ke32.p, P->E32.p, P->mask.p, P->ebe_tile,
           P->Ke32_host.data()};
    const bool tc = P->tc_mode >= 0 ? P->tc_mode != 0 : P->opt.prec == TOMG_PREC_TC_VCYCLE;
    op.tc = (P->dim == 3 && tc && P->Ketc.p) ? 1 : 0;
    op.tc_nz = P->tc_nz;
    op.tc_ty = P->tc_ty;
    op.Ktc = P->Ketc.p;
    op.tc_cl = P->tc_cl;
    op.tc_cm = P->tc_cm;
    return op;
  }
};

inline cudaStream_t st(const tomg_problem* P) { return P->stream; }

// single-step calls with an explicit precision choose the hex8 FP32 kernel by that precision
struct TcScope {
  tomg_problem* P;
  int saved;
  TcScope(tomg_problem* p, int prec) : P(p), saved(p->tc_mode) {
    P->tc_mode = prec == TOMG_PREC_TC_VCYCLE ? 1 : 0;
  }
  ~TcScope() { P->tc_mode = saved; }
};

// the setup's side streams and their events, created on first use
void ensure_side_streams(tomg_problem* P) {
  if (P->side) return;
  CK(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&P->side2, cudaStreamNonBlocking));
  for (cudaEvent_t* e : {&P->ev_fork, &P->ev_side, &P->ev_fork2, &P->ev_side2})
    CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
}

// Makes stream `s` wait for event `ev` (recorded on another stream) once: at join(), or when
// the guard goes out of scope, including on an exception.
struct StreamJoin {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  void arm(cudaStream_t s_, cudaEvent_t ev_) { s = s_; ev = ev_; }
  void join() {
    if (ev) CK(cudaStreamWaitEvent(s, ev, 0));
    ev = nullptr;
  }
  ~StreamJoin() {
    if (ev) cudaStreamWaitEvent(s, ev, 0);
  }
};

template <class T>
void level_op(tomg_problem* P, cudaStream_t s, int l, int mode, const T* x, T* y, const T* b,
              const int* done, const ChebArg* ch = nullptr) {
  Level& Lv = *P->L[l];
  const double w = ((mode == MODE_CHEB || mode == MODE_CHEB0) && ch) ? ch->c2 : P->opt.omega;
  switch (Lv.kind) {
    case KIND_EBE:
      // FP64: the assembled fine stencil kept by the setup halves the FP64 arithmetic
      if (sizeof(T) == 8 && Lv.S64.p)
        stencil_op<T>(s, mode, Lv.g, reinterpret_cast<const T*>(Lv.S64.p), x, y, b, V<T>::D(Lv), w,
                      done, ch);
      else
        ebe_op<T>(s, mode, V<T>::ebe(P), x, y, b, V<T>::D(Lv), w, done, nullptr, ch);
      break;
    case KIND_STENCIL:
      stencil_op<T>(s, mode, Lv.g, V<T>::S(Lv), x, y, b, V<T>::D(Lv), w, done, ch);
      break;
    default:
      bsr_op<T>(s, mode, Lv.bsr(), V<T>::Vv(Lv), x, y, b, V<T>::D(Lv), w, done, ch);
  }
}

template <class T>
void restrict_to(tomg_problem* P, cudaStream_t s, int l, const T* r, T* bc, const int* done) {
  Level& Lv = *P->L[l];
  Level& C = *P->L[l + 1];
  if (Lv.geo_next) geo_restrict<T>(s, Lv.g, C.g, r, bc, done);
  else bsr_spmv_rect<T>(s, Lv.Rmat(C.nn), V<T>::Rv(Lv), r, bc, 0, done);
}

template <class T>
void prolong_add(tomg_problem* P, cudaStream_t s, int l, const T* xc, T* x, const int* done) {
  Level& Lv = *P->L[l];
  Level& C = *P->L[l + 1];
  if (Lv.geo_next) geo_prolong_add<T>(s, Lv.g, C.g, xc, x, done);
  else bsr_spmv_rect<T>(s, Lv.Pmat(C.nn), V<T>::Pv(Lv), xc, x, 1, done);
}

// out = x0 + (m steps of point-block-Jacobi right-preconditioned GMRES on A_l from x0, whose
// initial residual r0 is given); x0 = nullptr means x0 = 0 (r0 = b)
template <class T>
void gmres_smooth(tomg_problem* P, Work& W, int l, const T* r0, const T* x0, T* out,
                  const int* done) {
  Level& Lv = *P->L[l];
  LevelWork& lw = W.lw[l];
  cudaStream_t s = W.stream;
  const int m = P->opt.gmres_steps;
  const int64_t n = Lv.n;
  T* Vb = V<T>::gV(lw);
  T* Zb = V<T>::gZ(lw);
  GmState* st = lw.gst.p;
  gmres_smooth_begin<T>(s, n, r0, lw.gparts.p, st, m, done);
  for (int j = 0; j < m; j++) {
    gmres_smooth_next<T>(s, Lv.b, Lv.nn, j, j == 0 ? r0 : Vb + (int64_t)j * n, Vb, n, Zb,
                         V<T>::D(Lv), st, done);
    level_op<T>(P, s, l, MODE_APPLY, Zb + (int64_t)j * n, Vb + (int64_t)(j + 1) * n, nullptr, done);
    gmres_smooth_orth<T>(s, n, j, m, Vb, n, lw.gparts.p, st, done);
  }
  gmres_smooth_finish<T>(s, n, m, Zb, n, st, x0, out, done);
}

// V-cycle of Algorithm 1: out = MG(b) on level l (x = 0 initial guess), work vectors of slot W
template <class T>
void vcycle(tomg_problem* P, Work& W, int l, const T* b, T* out, const int* done) {
  Level& Lv = *P->L[l];
  LevelWork& lw = W.lw[l];
  cudaStream_t s = W.stream;
  const int nl = (int)P->L.size();
  const double w = P->opt.omega;
  if (P->jacobi_only) {
    jacobi0<T>(s, Lv.b, Lv.nn, V<T>::D(Lv), b, out, w, done);
    return;
  }
  if (l == nl - 1) {
    dense_gemv<T>(s, P->nc, V<T>::Ainv(P), b, out, done);
    return;
  }
  T* x = V<T>::x(lw);
  T* r = V<T>::r(lw);
  if (P->opt.smoother == 2) {
    // GMRES smoothing: from x = 0 before the coarse correction (r_0 = b), from the corrected
    // iterate after it (r_0 = b - A x)
    gmres_smooth<T>(P, W, l, b, nullptr, x, done);
    level_op<T>(P, s, l, MODE_RESID, x, r, b, done);
    LevelWork& cw = W.lw[l + 1];
    restrict_to<T>(P, s, l, r, V<T>::b(cw), done);
    vcycle<T>(P, W, l + 1, V<T>::b(cw), V<T>::y(cw), done);
    prolong_add<T>(P, s, l, V<T>::y(cw), x, done);
    level_op<T>(P, s, l, MODE_RESID, x, r, b, done);
    gmres_smooth<T>(P, W, l, r, x, out, done);
    return;
  }
  if (P->opt.smoother == 1) {
    // Chebyshev smoothing (m steps of Chebyshev acceleration, the same polynomial before and
    // after the coarse correction), each step one fused residual + update launch writing the
    // new iterate to the other of two buffers.  Starting in x, the iterate ends in `out` for
    // every m; r holds the step vector d, except while it carries the restricted residual.
    const int m = P->opt.cheb_degree;
    T* cur = x;
    T* nxt = out;
    int k = 1;
    // x_1 = d_0 fused with the second step on quad4 level 0 (its tiled kernel forms w0 Dinv b
    // once per staged node), on 2D stencil levels (9 neighbours) and, with fuse_transfers, on
    // the FP32 tensor-core hex8 operator.  3D stencil and BSR kernels would form it at every
    // neighbour they read (27 and 30-60 per row): a separate sweep is cheaper there (measured
    // on the 3D cantilever 192x96x96 and the 2D cantilever 768x384)
    const bool ebe_fuses = Lv.kind == KIND_EBE && ebe_fuses_transfers<T>(V<T>::ebe(P));
    const bool fuse =
        m >= 2 && (Lv.kind == KIND_EBE ? (P->dim == 2 || (ebe_fuses && P->opt.fuse_transfers))
                                       : (Lv.kind == KIND_STENCIL && P->dim == 2));
    if (fuse) {
      ChebArg ch;
      ch.d = r; ch.c1 = Lv.cheb_c1[1]; ch.c2 = Lv.cheb_c2[1]; ch.dmode = 2; ch.w0 = Lv.cheb_c2[0];
      level_op<T>(P, s, l, MODE_CHEB0, cur, nxt, b, done, &ch);
      std::swap(cur, nxt);
      k = 2;
    } else {
      jacobi0<T>(s, Lv.b, Lv.nn, V<T>::D(Lv), b, cur, Lv.cheb_c2[0], done);  // x_1 = d_0
    }
    for (; k < m; k++) {
      ChebArg ch;
      ch.d = r; ch.c1 = Lv.cheb_c1[k]; ch.c2 = Lv.cheb_c2[k]; ch.dmode = k == 1 ? 2 : 1;
      level_op<T>(P, s, l, MODE_CHEB, cur, nxt, b, done, &ch);
      std::swap(cur, nxt);
    }
    level_op<T>(P, s, l, MODE_RESID, cur, r, b, done);
    LevelWork& cw = W.lw[l + 1];
    restrict_to<T>(P, s, l, r, V<T>::b(cw), done);
    vcycle<T>(P, W, l + 1, V<T>::b(cw), V<T>::y(cw), done);
    // the coarse correction: its own pass, or (geometric transfer into a 3^d stencil level or
    // the FP32 tensor-core hex8 operator) prolonged inside the first post-smoothing step
    const bool fuse_prol = P->opt.fuse_transfers && Lv.geo_next &&
                           (Lv.kind == KIND_STENCIL || ebe_fuses);
    if (!fuse_prol) prolong_add<T>(P, s, l, V<T>::y(cw), cur, done);
    for (int k = 0; k < m; k++) {
      ChebArg ch;
      ch.d = r; ch.c1 = Lv.cheb_c1[k]; ch.c2 = Lv.cheb_c2[k]; ch.dmode = k == 0 ? 0 : 1;
      if (k == 0 && fuse_prol) {
        const Level& C = *P->L[l + 1];
        ch.xc = V<T>::y(cw);
        ch.cnx = C.g.nx;
        ch.cny = C.g.ny;
        ch.cnz = C.g.nz;
      }
      level_op<T>(P, s, l, MODE_CHEB, cur, nxt, b, done, &ch);
      std::swap(cur, nxt);
    }
    return;  // cur == out
  }
  // pre-smoothing; the first sweep from x = 0 needs no operator apply, and with a single
  // pre-sweep in FP32 it is fused into the residual pass (x = w Dinv b, r = b - A x in one
  // kernel; forming w Dinv b at every neighbour is cheap on the FP32 pipes, not on FP64)
  if (P->opt.n_pre == 1 && sizeof(T) == 4) {
    level_op<T>(P, s, l, MODE_RESID0, x, r, b, done);
  } else {
    jacobi0<T>(s, Lv.b, Lv.nn, V<T>::D(Lv), b, x, w, done);
    for (int k = 1; k < P->opt.n_pre; k++) {
      level_op<T>(P, s, l, MODE_JACOBI, x, r, b, done);
      std::swap(x, r);
    }
    level_op<T>(P, s, l, MODE_RESID, x, r, b, done);  // r = b - A x
  }
  LevelWork& cw = W.lw[l + 1];
  restrict_to<T>(P, s, l, r, V<T>::b(cw), done);
  vcycle<T>(P, W, l + 1, V<T>::b(cw), V<T>::y(cw), done);
  prolong_add<T>(P, s, l, V<T>::y(cw), x, done);
  T* cur = x;
  for (int k = 0; k < P->opt.n_post; k++) {
    T* dst = (k == P->opt.n_post - 1) ? out : (cur == x ? r : x);
    level_op<T>(P, s, l, MODE_JACOBI, cur, dst, b, done);
    cur = dst;
  }
}

// z = M r (outer residual in FP64), then z.r (and z.q) reduced into the scalar state (FIN_RZ0
// without q, FIN_BETA with it).  r32_ready: the FP32 copy of r is already in the level-0 b32.
void apply_M_and_dots(tomg_problem* P, Work& W, const double* q, const int* done, bool r32_ready) {
  const int64_t n = P->n;
  LevelWork& l0 = W.lw[0];
  cudaStream_t s = W.stream;
  if (P->opt.prec == TOMG_PREC_FP64) {
    vcycle<double>(P, W, 0, W.r.p, W.z.p, done);
    z_dots<double>(s, W.z.p, W.z.p, W.r.p, q, n, W.partA.p, W.partB.p, W.sc.p, q ? FIN_BETA : FIN_RZ0);
  } else {
    if (!r32_ready) cast_in<float>(s, W.r.p, l0.b32.p, n, done);
    vcycle<float>(P, W, 0, l0.b32.p, l0.y32.p, done);
    z_dots<float>(s, l0.y32.p, W.z.p, W.r.p, q, n, W.partA.p, W.partB.p, W.sc.p, q ? FIN_BETA : FIN_RZ0);
  }
}

// FP64 outer operator K (masked): the assembled fine stencil when the setup kept it (36 / 243
// FMAs per node instead of 72 / 600 for the element products), else the matrix-free kernel
// whether the outer FP64 applies of hex8 run on the tensor cores (k_ebe3x64.cu)
bool x64_active(const tomg_problem* P) { return P->dim == 3 && P->Kx64.p && P->opt.fp64_tc; }

// the FP64 tensor-core operator's work buffer for launches on stream s (one per stream: solve
// slots apply concurrently), sized for the current block of right-hand sides.  Allocated
// outside graph captures (build_graph asks for it before capturing).
double* x64_buffer(tomg_problem* P, cudaStream_t s) {
  const int64_t need = ebe3x_buffer_doubles(V<double>::ebe(P)) * batch_rhs();
  DBuf<double>& b = P->x64buf[s];
  if ((int64_t)b.n < need) b.resize(need);
  return b.p;
}

// Outer-loop K in FP64: on hex8 the element products on the tensor cores (exact integer digit
// products, FP64 scaling and node sums) when nu allows them; else the assembled fine stencil
// when the setup kept it (36 / 243 FMAs per node instead of 64 / 576 for the element products),
// else the FP64 element kernel.  Partials of x . y (nullable); with sc set, FIN_ALPHA is
// applied to the scalar state on the device.
void fine64_apply_dot(tomg_problem* P, cudaStream_t s, const double* x, double* y, const int* done,
                      double* partials, Scalars* sc) {
  Level& L0 = *P->L[0];
  if (x64_active(P)) {
    ebe3x_apply(s, MODE_APPLY, V<double>::ebe(P), P->Kx64.p, P->x64_c, x, y, nullptr, done,
                partials, sc, x64_buffer(P, s));
  } else if (L0.S64.p) {
    stencil_apply_dot(s, L0.g, L0.S64.p, x, y, done, partials, sc);
  } else {
    ebe_op<double>(s, MODE_APPLY, V<double>::ebe(P), x, y, nullptr, nullptr, 0.0, done, partials);
    if (sc) finish(s, FIN_ALPHA, partials, ebe_blocks(V<double>::ebe(P)), nullptr, 0, sc);
  }
}
void fine64_resid(tomg_problem* P, cudaStream_t s, const double* x, double* y, const double* b) {
  if (x64_active(P))
    ebe3x_apply(s, MODE_RESID, V<double>::ebe(P), P->Kx64.p, P->x64_c, x, y, b, nullptr, nullptr,
                nullptr, x64_buffer(P, s));
  else
    level_op<double>(P, s, 0, MODE_RESID, x, y, b, nullptr);
}

void iteration_body(tomg_problem* P, Work& W) {
  const int64_t n = P->n;
  Scalars* sc = W.sc.p;
  const int* done = &sc->done;
  cudaStream_t s = W.stream;
  const bool mixed = P->opt.prec != TOMG_PREC_FP64;
  fine64_apply_dot(P, s, W.p.p, W.q.p, done, W.partA.p, sc);                // + FIN_ALPHA
  xr_update(s, W.x.p, W.r.p, W.p.p, W.q.p, n, sc, W.partA.p,
            mixed ? W.lw[0].b32.p : nullptr);                               // + FIN_RR
  apply_M_and_dots(P, W, W.q.p, done, mixed);                               // + FIN_BETA
  p_update(s, W.p.p, W.z.p, n, sc, W.cond, W.has_cond);
}

// One outer iteration of a block solve: the iteration_body sequence with every launch covering
// the W.block right-hand sides (BatchScope).  The Krylov kernels read each right-hand side's own
// scalar state and leave a converged one untouched; the V-cycle between them runs for all of
// them (its result is not used for a converged one).  The last kernel sets the captured loop's
// condition from all done flags.
void block_iteration_body(tomg_problem* P, Work& W) {
  const int64_t n = P->n;
  const int R = W.block;
  Scalars* sc = W.sc.p;
  cudaStream_t s = W.stream;
  BatchScope bs(R);
  fine64_apply_dot(P, s, W.p.p, W.q.p, &sc->done, W.partA.p, sc);  // + FIN_ALPHA per rhs
  xr_update(s, W.x.p, W.r.p, W.p.p, W.q.p, n, sc, W.partA.p, W.lw[0].b32.p);  // + FIN_RR
  vcycle<float>(P, W, 0, W.lw[0].b32.p, W.lw[0].y32.p, nullptr);
  z_dots<float>(s, W.lw[0].y32.p, W.z.p, W.r.p, W.q.p, n, W.partA.p, W.partB.p, sc, FIN_BETA);
  p_update(s, W.p.p, W.z.p, n, sc, 0, 0);
  if (W.has_cond) block_cond(s, sc, R, W.cond);
}

void destroy_graph(Work& W) {
  if (W.gexec) cudaGraphExecDestroy(W.gexec);
  if (W.graph) cudaGraphDestroy(W.graph);
  W.gexec = nullptr;
  W.graph = nullptr;
  W.graph_mode = 0;
}

void build_graph(tomg_problem* P, Work& W) {
  destroy_graph(W);
  const int mode = W.block > 1 ? 2 : P->opt.use_graph;
  if (mode > 0 && x64_active(P)) {  // the outer operator's buffer, before any capture
    BatchScope bs(W.block > 1 ? W.block : 1);
    x64_buffer(P, W.stream);
  }
  auto run_body = [&]() {
    if (W.block > 1) block_iteration_body(P, W);
    else iteration_body(P, W);
  };
  if (mode <= 0) return;
  cudaStream_t s = W.stream;
  const int64_t saved = g_launches;
  // programmatic dependent launch between the captured kernels (TOMG_NO_PDL=1 turns it off)
  struct PdlScope {
    PdlScope() { set_pdl(getenv("TOMG_NO_PDL") == nullptr); }
    ~PdlScope() { set_pdl(false); }
  } pdl_scope;
  if (mode >= 2) {
    CK(cudaGraphCreate(&W.graph, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, W.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, W.graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    W.cond = h;
    W.has_cond = 1;
    try {
      run_body();
    } catch (...) {
      W.has_cond = 0;
      cudaGraph_t dummy;
      cudaStreamEndCapture(s, &dummy);
      g_launches = saved;
      throw;
    }
    W.has_cond = 0;
    CK(cudaStreamEndCapture(s, &body));
  } else {
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
      run_body();
    } catch (...) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(s, &dummy);
      g_launches = saved;
      throw;
    }
    CK(cudaStreamEndCapture(s, &W.graph));
  }
  W.kernels_per_iter = g_launches - saved;
  g_launches = saved;
  CK(cudaGraphInstantiate(&W.gexec, W.graph, 0));
  W.graph_mode = mode >= 2 ? 2 : 1;
}

// level positions along one axis after `level` coarsenings (fine-grid coordinates)
std::vector<double> level_positions(int n, int level) {
  std::vector<int> pos(n + 1);
  for (int i = 0; i <= n; i++) pos[i] = i;
  int m = n;
  for (int l = 0; l < level; l++) {
    const int mc = (m + 1) / 2;
    std::vector<int> np(mc + 1);
    for (int I = 0; I <= mc; I++) np[I] = pos[std::min(2 * I, m)];
    pos.swap(np);
    m = mc;
  }
  return std::vector<double>(pos.begin(), pos.end());
}

Geo coarse_geo(const Geo& g) {
  return Geo{g.dim, (g.nx + 1) / 2, (g.ny + 1) / 2, g.dim == 3 ? (g.nz + 1) / 2 : 1};
}

struct OwnedBsr {
  DBuf<int> rp, ci;
  DBuf<double> V;
  Bsr m;
};

void spgemm_full(cudaStream_t s, const Bsr& A, const double* VA, const Bsr& B, const double* VB,
                 OwnedBsr& C, bool sym = false) {
  DBuf<int> counts;
  counts.resize(A.nbr > 0 ? A.nbr : 1);
  C.rp.resize(A.nbr + 1);
  SpgemmWork w;
  SetupTrace tr(s);
  spgemm_counts(s, A, B, counts.p, w);
  const int64_t nnz = exclusive_scan(s, counts.p, C.rp.p, A.nbr);
  tr.mark("  spgemm count+scan");
  C.ci.resize(nnz > 0 ? nnz : 1);
  spgemm_fill(s, A, B, C.rp.p, C.ci.p, w);
  tr.mark("  spgemm fill");
  C.m.nbr = A.nbr; C.m.nbc = B.nbc; C.m.br = A.br; C.m.bc = B.bc; C.m.nnzb = nnz;
  C.m.rp = C.rp.p; C.m.ci = C.ci.p;
  C.V.resize(std::max<int64_t>(1, nnz * A.br * B.bc));
  spgemm_numeric(s, A, VA, B, VB, C.m, C.V.p, sym);
  tr.mark("  spgemm numeric");
}

// level operator (stencil or matrix-free level 0 via its assembled stencil) -> BSR in Lv
void make_bsr_from_stencil(tomg_problem* P, Level& Lv) {
  cudaStream_t s = st(P);
  DBuf<int> counts;
  counts.resize(Lv.nn);
  stencil_row_counts(s, Lv.g, counts.p);
  Lv.rp.resize(Lv.nn + 1);
  Lv.nnzb = exclusive_scan(s, counts.p, Lv.rp.p, Lv.nn);
  Lv.ci.resize(Lv.nnzb);
  Lv.V64.resize(Lv.nnzb * Lv.b * Lv.b);
  stencil_to_bsr(s, Lv.g, Lv.S64.p, Lv.rp.p, Lv.ci.p, Lv.V64.p);
}

void amg_extend(tomg_problem* P, int start) {
  cudaStream_t s = st(P);
  SetupTrace tr(s);
  const tomg_options& o = P->opt;
  {
    Level& S0 = *P->L[start];
    make_bsr_from_stencil(P, S0);
  }
  const int k = P->dim == 2 ? 3 : 6;
  // candidates: rigid-body modes at the node coordinates of the start level
  DBuf<double> B;
  {
    Level& S0 = *P->L[start];
    auto xs = level_positions(P->nx, start), ys = level_positions(P->ny, start);
    auto zs = level_positions(P->dim == 3 ? P->nz : 0, P->dim == 3 ? start : 0);
    DBuf<double> dx, dy, dz;
    dx.resize(xs.size()); dy.resize(ys.size()); dz.resize(zs.size());
    CK(cudaMemcpyAsync(dx.p, xs.data(), xs.size() * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dy.p, ys.data(), ys.size() * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dz.p, zs.data(), zs.size() * 8, cudaMemcpyHostToDevice, s));
    B.resize(S0.n * k);
    rigid_body_modes(s, S0.g, dx.p, dy.p, dz.p, B.p);
    // (xs, ys, zs are pageable: each copy has read them before cudaMemcpyAsync returned)
  }
  tr.mark("bsr+rbm", start);
  int cur = start;
  while (P->L[cur]->n >= o.max_coarse_dofs && (int)P->L.size() < o.max_levels) {
    Level& A = *P->L[cur];
    const Bsr Ab = A.bsr();
    const int nn = (int)A.nn, b = A.b;
    // rho(D^-1 A) for the prolongator smoothing (and a Chebyshev smoother on this level) reads
    // only this level's operator: it runs on the second side stream during the strength,
    // aggregation, tentative prolongator and A T phases and is joined before the smoothing
    // (the guard joins on every exit from this step, before the buffers are released)
    AmgPower rho_pw;
    StreamJoin rho_join;
    ensure_side_streams(P);
    amg_power_alloc(s, rho_pw, Ab, 20);
    CK(cudaEventRecord(P->ev_fork2, s));
    CK(cudaStreamWaitEvent(P->side2, P->ev_fork2, 0));
    amg_power_enqueue(P->side2, rho_pw, Ab, A.V64.p, A.D64.p, cur);
    CK(cudaEventRecord(P->ev_side2, P->side2));
    rho_join.arm(s, P->ev_side2);
    // strength of connection (Eq. 10)
    DBuf<int> scnt, srp, sci;
    scnt.resize(nn);
    srp.resize(nn + 1);
    amg_strength_counts(s, Ab, A.V64.p, o.soc_beta, scnt.p);
    const int64_t nS = exclusive_scan(s, scnt.p, srp.p, nn);
    sci.resize(nS > 0 ? nS : 1);
    amg_strength_fill(s, Ab, A.V64.p, o.soc_beta, srp.p, sci.p);
    tr.mark("strength", cur);
    // aggregation
    DBuf<int> state, root_scan, agg;
    DBuf<uint64_t> vv, m1;
    state.resize(nn); root_scan.resize(nn + 1); agg.resize(nn); vv.resize(nn); m1.resize(nn);
    amg_mis2(s, nn, srp.p, sci.p, cur, state.p, vv.p, m1.p, P->flag_host, P->flag_dev.p);
    tr.mark("mis2", cur);
    const int n_agg = amg_aggregate(s, nn, srp.p, sci.p, cur, state.p, agg.p, root_scan.p);
    tr.mark("aggregate", cur);
    if (n_agg == 0 || (int64_t)n_agg * k >= A.n) break;
    // tentative prolongator
    DBuf<int> Trp, Tci;
    DBuf<double> TV, Bc;
    Trp.resize(nn + 1); Tci.resize(nn); TV.resize((int64_t)nn * b * k); Bc.resize((int64_t)n_agg * k * k);
    const int nT = (int)amg_tentative(s, nn, b, k, n_agg, agg.p, B.p, Trp.p, Tci.p, TV.p, Bc.p);
    Bsr Tm;
    Tm.nbr = nn; Tm.nbc = n_agg; Tm.br = b; Tm.bc = k; Tm.nnzb = nT; Tm.rp = Trp.p; Tm.ci = Tci.p;
    tr.mark("tentative", cur);
    // P = T - omega D^-1 A T
    OwnedBsr AT;
    spgemm_full(s, Ab, A.V64.p, Tm, TV.p, AT);
    tr.mark("A*T", cur);
    // prolongator smoothing weight from rho(D^-1 A)
    rho_join.join();
    const double rho = amg_power_result(s, rho_pw);
    A.lam = rho;  // the same estimate bounds a Chebyshev smoother on this level
    const double omegaP = 4.0 / (3.0 * rho);
    tr.mark("spectral_radius", cur);
    A.Pnnzb = AT.m.nnzb;
    A.Prp = std::move(AT.rp);
    A.Pci = std::move(AT.ci);
    A.Pv64.resize(std::max<int64_t>(1, A.Pnnzb * b * k));
    A.bc = k;
    Bsr Pm = A.Pmat(n_agg);
    amg_smooth_prolongator(s, Pm, AT.V.p, agg.p, TV.p, Trp.p, A.D64.p, omegaP, b, A.Pv64.p);
    // R = P^T
    {
      DBuf<int> cnt, cursor;
      cnt.resize(n_agg); cursor.resize(n_agg);
      bsr_col_counts(s, Pm, cnt.p);
      A.Rrp.resize(n_agg + 1);
      exclusive_scan_nosync(s, cnt.p, A.Rrp.p, n_agg);
      A.Rci.resize(std::max<int64_t>(1, A.Pnnzb));
      A.Rv64.resize(std::max<int64_t>(1, A.Pnnzb * b * k));
      bsr_transpose_fill(s, Pm, A.Pv64.p, A.Rrp.p, A.Rci.p, A.Rv64.p, cursor.p);
    }
    tr.mark("smoothP+transpose", cur);
    // A_c = R (A P)  (Eq. 9)
    OwnedBsr AP, Ac;
    spgemm_full(s, Ab, A.V64.p, Pm, A.Pv64.p, AP);
    tr.mark("A*P", cur);
    spgemm_full(s, A.Rmat(n_agg), A.Rv64.p, AP.m, AP.V.p, Ac, true);
    tr.mark("R*(AP)", cur);
    amg_fix_zero_rows(s, Ac.m, Ac.V.p);
    A.Pv32.resize(A.Pv64.n); cast_f64_f32(s, A.Pv64.p, A.Pv32.p, A.Pv64.n);
    A.Rv32.resize(A.Rv64.n); cast_f64_f32(s, A.Rv64.p, A.Rv32.p, A.Rv64.n);
    A.geo_next = false;
    A.agg = std::move(agg);
    auto C = std::make_unique<Level>();
    C->kind = KIND_BSR;
    C->b = k;
    C->nn = n_agg;
    C->n = (int64_t)n_agg * k;
    C->geometric = false;
    C->g = Geo{P->dim, 0, 0, 0};
    C->nnzb = Ac.m.nnzb;
    C->rp = std::move(Ac.rp);
    C->ci = std::move(Ac.ci);
    C->V64 = std::move(Ac.V);
    C->D64.resize(C->nn * k * k);
    C->D32.resize(C->nn * k * k);
    bsr_block_diag_inv(s, C->bsr(), C->V64.p, C->D64.p, C->D32.p);
    C->V32.resize(C->V64.n);
    cast_f64_f32(s, C->V64.p, C->V32.p, C->V64.n);
    P->L.push_back(std::move(C));
    B = std::move(Bc);
    cur++;
    tr.mark("coarse level", cur);
  }
}

}  // namespace

int levels_for_cap(int dim, int nx, int ny, int nz, int cap, int max_levels) {
  int L = 1;
  Geo g{dim, nx, ny, dim == 3 ? nz : 1};
  while ((int64_t)dim * g.nodes() >= cap && L < max_levels) {
    Geo c = coarse_geo(g);
    if (c.nx == g.nx && c.ny == g.ny && c.nz == g.nz) break;
    g = c;
    L++;
  }
  return L;
}

Work::~Work() {
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (sc_host) cudaFreeHost(sc_host);
  if (partE_host) cudaFreeHost(partE_host);
  if (partC_host) cudaFreeHost(partC_host);
  for (cudaEvent_t e : {ev0, ev1, evdone, evsync})
    if (e) cudaEventDestroy(e);
  if (stream) cudaStreamDestroy(stream);
}

StreamScope::StreamScope(tomg_problem* p) : P(p) {
  CK(cudaEventRecord(P->ev_in, P->ctx->stream));
  CK(cudaStreamWaitEvent(P->stream, P->ev_in, 0));
}
StreamScope::~StreamScope() {
  if (cudaEventRecord(P->ev_out, P->stream) == cudaSuccess)
    cudaStreamWaitEvent(P->ctx->stream, P->ev_out, 0);
}

void problem_init(tomg_problem* P) {
  CK(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming));
  CK(cudaEventCreate(&P->ev0));
  CK(cudaEventCreate(&P->ev1));
  StreamScope scope(P);
  cudaStream_t s = st(P);
  set_alloc_stream(s);
  element_stiffness_host(P->dim, P->nu, P->Ke_host);
  const size_t nk = P->Ke_host.size();
  P->Ke64.resize(nk);
  P->Ke32.resize(nk);
  P->Ke32_host.assign(P->Ke_host.begin(), P->Ke_host.end());
  CK(cudaMemcpyAsync(P->Ke64.p, P->Ke_host.data(), nk * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P->Ke32.p, P->Ke32_host.data(), nk * 4, cudaMemcpyHostToDevice, s));
  if (P->dim == 3) {
    std::vector<uint32_t> img(ebe3d_tc_operand_words());
    ebe3d_tc_operand(P->nu, img.data(), &P->tc_cl, &P->tc_cm);
    P->Ketc.resize(img.size());
    CK(cudaMemcpyAsync(P->Ketc.p, img.data(), img.size() * 4, cudaMemcpyHostToDevice, s));
    std::vector<uint32_t> imgx(ebe3x_operand_words());
    if (ebe3x_operand(P->nu, imgx.data(), &P->x64_c)) {
      P->Kx64.resize(imgx.size());
      CK(cudaMemcpyAsync(P->Kx64.p, imgx.data(), imgx.size() * 4, cudaMemcpyHostToDevice, s));
    }
    CK(cudaStreamSynchronize(s));  // img, imgx are host temporaries
  }
  P->mask.resize(P->nn);
  P->mask.zero(s);
  P->rho.resize(P->nel);
  P->E64.resize(P->nel);
  P->E32.resize(P->nel);
  P->flag_dev.resize(1);
  CK(cudaMallocHost((void**)&P->flag_host, sizeof(int)));
  CK(cudaStreamSynchronize(s));
}

void set_fixed(tomg_problem* P, const int64_t* dofs, int64_t count) {
  if (count < 0 || (count > 0 && !dofs)) TOMG_THROW(TOMG_E_INVALID, "bad fixed-DOF array");
  std::vector<uint8_t> m(P->nn, 0);
  for (int64_t i = 0; i < count; i++) {
    const int64_t d = dofs[i];
    if (d < 0 || d >= P->n) TOMG_THROW(TOMG_E_INVALID, "fixed DOF %lld out of range [0, %lld)", (long long)d, (long long)P->n);
    m[d / P->dim] |= (uint8_t)(1u << (d % P->dim));
  }
  CK(cudaMemcpyAsync(P->mask.p, m.data(), m.size(), cudaMemcpyHostToDevice, st(P)));
  CK(cudaStreamSynchronize(st(P)));
  P->setup_valid = false;
}

void set_density(tomg_problem* P, const double* rho, int on_device) {
  cudaStream_t s = st(P);
  if (!rho) TOMG_THROW(TOMG_E_INVALID, "null density");
  CK(cudaMemcpyAsync(P->rho.p, rho, P->nel * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  P->flag_dev.zero(s);
  simp_moduli(s, P->nel, P->rho.p, P->E0, P->Emin, P->penal, P->E64.p, P->E32.p, P->flag_dev.p);
  CK(cudaMemcpyAsync(P->flag_host, P->flag_dev.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  P->setup_valid = false;
  if (*P->flag_host) {
    P->have_density = false;
    TOMG_THROW(TOMG_E_INVALID, "density has negative or NaN entries");
  }
  P->have_density = true;
}

void setup(tomg_problem* P, const tomg_options& opt) {
  cudaStream_t s = st(P);
  if (!P->have_density) TOMG_THROW(TOMG_E_INVALID, "tomg_setup: no density set");
  if (opt.pc < 0 || opt.pc > 3 || opt.prec < 0 || opt.prec > 2)
    TOMG_THROW(TOMG_E_INVALID, "unknown preconditioner %d or precision %d", opt.pc, opt.prec);
  if (!(opt.rtol > 0.0) || opt.max_iter < 1 || opt.max_iter > 1000000 || !(opt.omega > 0.0) ||
      !(opt.omega < 2.0) || opt.n_pre < 1 || opt.n_pre > 8 || opt.n_post < 1 || opt.n_post > 8 ||
      opt.max_coarse_dofs < 1 || opt.max_levels < 1 || opt.max_levels > 64 || opt.smoother < 0 ||
      opt.smoother > 2 || opt.concurrency < 0 || opt.concurrency > 64 ||
      (opt.smoother == 2 && (opt.gmres_steps < 1 || opt.gmres_steps > GM_MAX)) ||
      (opt.smoother == 1 && (opt.cheb_degree < 1 || opt.cheb_degree > 8 ||
                             !(opt.cheb_lower > 0.0) || !(opt.cheb_upper > opt.cheb_lower))) ||
      (opt.adaptive_geo != 0 && (opt.adaptive_iters < 1 || opt.adaptive_min_geo < 1)) ||
      opt.krylov < 0 || opt.krylov > 1 || opt.block_rhs < 0 || opt.block_rhs > 64 ||
      (opt.block_rhs > 1 && (P->dim != 3 || opt.prec != TOMG_PREC_TC_VCYCLE || opt.smoother == 2 ||
                             opt.krylov != 0)) ||
      (opt.krylov == 1 && (opt.gmres_restart < 1 || opt.gmres_restart > 200)))
    TOMG_THROW(TOMG_E_INVALID, "invalid options");
  P->setup_valid = false;
  P->setup_gen++;
  P->opt = opt;
  CK(cudaEventRecord(P->ev0, s));
  SetupTrace tr(s);
  // side-stream power iterations (declared before the join guard, released after it)
  std::vector<PowerState> cheb_pw;
  StreamJoin side_join;
  P->L.clear();
  P->jacobi_only = (opt.pc == TOMG_PC_JACOBI);
  // level 0: matrix-free SIMP operator
  {
    auto L0 = std::make_unique<Level>();
    L0->kind = KIND_EBE;
    L0->b = P->dim;
    L0->nn = P->nn;
    L0->n = P->n;
    L0->g = Geo{P->dim, P->nx, P->ny, P->dim == 3 ? P->nz : 1};
    L0->geometric = true;
    L0->D64.resize(P->nn * P->dim * P->dim);
    L0->D32.resize(P->nn * P->dim * P->dim);
    ebe_block_diag_inv(s, V<double>::ebe(P), L0->D64.p, L0->D32.p);
    if (P->dim == 2 && opt.prec != TOMG_PREC_FP64 && P->ebe_tile == 0)
      P->ebe_tile = ebe2d_autotune(s, V<float>::ebe(P), L0->D32.p);
    if (P->dim == 3 && opt.prec == TOMG_PREC_TC_VCYCLE && P->tc_nz == 0 && P->Ketc.p) {
      TcScope tcs(P, TOMG_PREC_TC_VCYCLE);
      // TOMG_TC_TILE = rows * 1000 + layers fixes the tile instead of timing the candidates
      // (for profiler runs, under which the timed choice is not the one of a plain run)
      const char* forced = getenv("TOMG_TC_TILE");
      const int code = forced ? atoi(forced) : ebe3d_tc_autotune(s, V<float>::ebe(P), L0->D32.p);
      if (code / 1000 != 8 && code / 1000 != 4)
        TOMG_THROW(TOMG_E_INVALID, "TOMG_TC_TILE: rows 8 or 4 (rows * 1000 + layers)");
      P->tc_nz = std::max(1, code % 1000);
      P->tc_ty = code / 1000;
      if (getenv("TOMG_TRACE_SETUP"))
        fprintf(stderr, "[setup] tensor-core tile: %d element rows, %d node layers\n", P->tc_ty,
                P->tc_nz);
    }
    P->L.push_back(std::move(L0));
  }
  tr.mark("level0 diag", 0);
  if (!P->jacobi_only) {
    int n_geo = 1;
    if (opt.pc == TOMG_PC_GMG)
      n_geo = opt.n_levels > 0 ? opt.n_levels
                               : levels_for_cap(P->dim, P->nx, P->ny, P->nz, opt.max_coarse_dofs, opt.max_levels);
    else if (opt.pc == TOMG_PC_HYBRID && opt.adaptive_geo) {
      // adaptive hybrid (Sec. 4.4): the count carried over from the previous solves
      if (P->adapt_geo == 0) P->adapt_geo = std::max(opt.adaptive_min_geo, opt.n_geo_levels);
      n_geo = P->adapt_geo;
    } else if (opt.pc == TOMG_PC_HYBRID)
      n_geo = std::max(1, opt.n_geo_levels);
    n_geo = std::min(n_geo, opt.max_levels);
    Level& L0 = *P->L[0];
    // hex8: the first coarse stencil straight from the elements (k_galerkin.cu).  The assembled
    // FP64 level-0 stencil is built only where something reads it: the product on stencils
    // when the direct one declines, AMG or the dense solve on level 0, and the FP64
    // applications of K on level 0 unless the tensor-core FP64 operator carries them
    std::unique_ptr<Level> C1;
    if (P->dim == 3 && n_geo >= 2) {
      C1 = std::make_unique<Level>();
      C1->g = coarse_geo(L0.g);
      C1->S64.resize((int64_t)stencil_q(P->dim) * C1->g.nodes());
      if (!ebe_galerkin_stencil(s, V<double>::ebe(P), C1->g, C1->S64.p)) C1.reset();
      tr.mark("level1 from elements", 1);
    }
    const bool keep_S0 = !C1 || opt.prec == TOMG_PREC_FP64 || !x64_active(P);
    if (keep_S0) {
      L0.S64.resize((int64_t)stencil_q(P->dim) * P->nn);
      ebe_assemble_stencil(s, V<double>::ebe(P), L0.S64.p);
      tr.mark("level0 stencil", 0);
    }
    for (int l = 1; l < n_geo; l++) {
      Level& F = *P->L[l - 1];
      auto C = (l == 1 && C1) ? std::move(C1) : std::make_unique<Level>();
      C->kind = KIND_STENCIL;
      C->b = P->dim;
      C->g = coarse_geo(F.g);
      C->nn = C->g.nodes();
      C->n = C->nn * P->dim;
      C->geometric = true;
      if (!C->S64.p) {
        C->S64.resize((int64_t)stencil_q(P->dim) * C->nn);
        stencil_rap(s, F.g, C->g, F.S64.p, C->S64.p);
      }
      C->S32.resize(stencil_half_size(C->g));  // FP32 upper half for the V-cycle
      stencil_half_f32(s, C->g, C->S64.p, C->S32.p);
      C->D64.resize(C->nn * P->dim * P->dim);
      C->D32.resize(C->nn * P->dim * P->dim);
      stencil_block_diag_inv(s, C->g, C->S64.p, C->D64.p, C->D32.p);
      F.geo_next = true;
      P->L.push_back(std::move(C));
      tr.mark("geometric RAP", l);
    }
    // Chebyshev bounds of the geometric levels above the last one: they read only those
    // levels, so their power iterations run on the side stream while the algebraic levels and
    // the coarse inverse are built (phases with many host synchronisations and small kernels;
    // the last geometric level gets its estimate from the prolongator smoothing, or is the
    // coarsest).  The guard makes the problem stream wait for the side stream on every exit,
    // before any of the buffers involved is released.
    if (opt.smoother == 1 && n_geo >= 2) {
      ensure_side_streams(P);
      // with an FP32 V-cycle the estimate runs in FP32 on the cycle's own operator and block
      // inverses (norms in FP64): the bound only sets the Chebyshev interval, and FP64 vector
      // work here competes with the FP64-bound algebraic setup on GB300's narrow FP64 pipe
      const bool f32 = opt.prec != TOMG_PREC_FP64;
      cheb_pw.resize(n_geo - 1);
      for (int l = 0; l + 1 < n_geo; l++)
        power_alloc(cheb_pw[l], P->L[l]->nn, P->L[l]->b, 20, f32);
      CK(cudaEventRecord(P->ev_fork, s));
      CK(cudaStreamWaitEvent(P->side, P->ev_fork, 0));
      for (int l = 0; l + 1 < n_geo; l++) {
        Level& Lv = *P->L[l];
        if (f32) {
          power_enqueue_f32(P->side, cheb_pw[l], Lv.D32.p, l, [&](const float* xv, float* yv) {
            level_op<float>(P, P->side, l, MODE_APPLY, xv, yv, nullptr, nullptr);
          });
        } else {
          power_enqueue(P->side, cheb_pw[l], Lv.D64.p, l, [&](const double* xv, double* yv) {
            level_op<double>(P, P->side, l, MODE_APPLY, xv, yv, nullptr, nullptr);
          });
        }
      }
      CK(cudaEventRecord(P->ev_side, P->side));
      side_join.arm(s, P->ev_side);
    }
    if (opt.pc == TOMG_PC_AMG || opt.pc == TOMG_PC_HYBRID) amg_extend(P, (int)P->L.size() - 1);
    tr.mark("amg total");
    // coarsest level: dense FP64 Cholesky -> explicit inverse
    Level& Cl = *P->L.back();
    if (Cl.n > 16384)
      TOMG_THROW(TOMG_E_INVALID, "coarsest level has %lld DOFs (dense solve limit 16384); use more levels", (long long)Cl.n);
    P->nc = (int)Cl.n;
    P->Ainv64.resize((int64_t)P->nc * P->nc);
    if (Cl.kind == KIND_BSR) bsr_to_dense(s, Cl.bsr(), Cl.V64.p, P->Ainv64.p);
    else stencil_to_dense(s, Cl.g, Cl.S64.p, P->Ainv64.p);
    DBuf<double> work;
    work.resize((int64_t)P->nc * P->nc);
    const int fail = dense_spd_inverse(s, P->nc, P->Ainv64.p, work.p);
    if (fail) TOMG_THROW(TOMG_E_BREAKDOWN, "coarse operator not SPD (pivot %d)", fail - 1);
    P->Ainv32.resize(P->Ainv64.n);
    cast_f64_f32(s, P->Ainv64.p, P->Ainv32.p, P->Ainv64.n);
    tr.mark("coarse inverse", (int)P->L.size() - 1);
    if (opt.smoother == 1) {
      // Chebyshev smoother on every level above the coarsest: lambda_max(D^-1 A_l) by 20 power
      // iterations, interval [lower, upper] x lambda, three-term recurrence coefficients
      side_join.join();
      for (int l = 0; l + 1 < (int)P->L.size(); l++) {
        Level& Lv = *P->L[l];
        if (l < (int)cheb_pw.size())  // estimated on the side stream, now joined
          Lv.lam = power_result(s, cheb_pw[l]);
        else if (!(Lv.lam > 0.0))  // levels coarsened by aggregation have it already
          Lv.lam = spectral_radius_op(s, Lv.nn, Lv.b, Lv.D64.p, l, 20,
                                      [&](const double* xv, double* yv) {
                                        level_op<double>(P, s, l, MODE_APPLY, xv, yv, nullptr, nullptr);
                                      });
        const double a = opt.cheb_lower * Lv.lam, bnd = opt.cheb_upper * Lv.lam;
        const double theta = 0.5 * (bnd + a), delta = 0.5 * (bnd - a), sigma = theta / delta;
        double rho = 1.0 / sigma;
        Lv.cheb_c1[0] = 0.0;
        Lv.cheb_c2[0] = 1.0 / theta;
        for (int k = 1; k < opt.cheb_degree; k++) {
          const double rn = 1.0 / (2.0 * sigma - rho);
          Lv.cheb_c1[k] = rn * rho;
          Lv.cheb_c2[k] = 2.0 * rn / delta;
          rho = rn;
        }
      }
      tr.mark("chebyshev bounds");
    }
    // setup-only storage of the fine level.  Its FP64 stencil stays where it carries the FP64
    // applications of K (see fine64_apply_dot); with an FP32 V-cycle on hex8 with the FP64
    // tensor-core operator nothing reads it after the setup (3.5 GB at 5.4 M DOFs)
    L0.rp.release(); L0.ci.release(); L0.V64.release();
    if (P->dim == 3 && x64_active(P) && opt.prec != TOMG_PREC_FP64) L0.S64.release();
    for (auto& lv : P->L)
      if (lv->kind == KIND_STENCIL) { lv->rp.release(); lv->ci.release(); lv->V64.release(); }
  }
  CK(cudaEventRecord(P->ev1, s));
  CK(cudaEventSynchronize(P->ev1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, P->ev0, P->ev1));
  P->setup_ms = ms;
  P->setup_valid = true;
}

// ----------------------------------------------------------------------------------------
namespace {

// solve slot k, sized for the current hierarchy (vectors reused when sizes match)
Work& ensure_work(tomg_problem* P, int k) {
  while ((int)P->works.size() <= k) {
    auto W = std::make_unique<Work>();
    CK(cudaStreamCreateWithFlags(&W->stream, cudaStreamNonBlocking));
    CK(cudaEventCreate(&W->ev0));
    CK(cudaEventCreate(&W->ev1));
    CK(cudaEventCreateWithFlags(&W->evdone, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&W->evsync, cudaEventDisableTiming));
    const Ebe op{P->dim, P->nx, P->ny, P->nz, nullptr, nullptr, nullptr};
    W->np = std::max(std::max(ebe_blocks(op), red_blocks(P->n)), P->dim == 3 ? ebe3x_blocks(op) : 0);
    CK(cudaMallocHost((void**)&W->sc_host, sizeof(Scalars)));
    CK(cudaMallocHost((void**)&W->partE_host, sizeof(double) * W->np));
    CK(cudaMallocHost((void**)&W->partC_host, sizeof(double) * W->np));
    P->works.push_back(std::move(W));
  }
  Work& W = *P->works[k];
  if (W.built_for != P->setup_gen) {
    for (auto* v : {&W.f, &W.bvec, &W.x, &W.r, &W.p, &W.q, &W.z, &W.t}) v->resize(P->n);
    for (auto* v : {&W.partA, &W.partB, &W.partE, &W.partC}) v->resize(W.np);
    W.sc.resize(1);
    W.lw.resize(P->L.size());
    for (size_t l = 0; l < P->L.size(); l++) {
      LevelWork& lw = W.lw[l];
      const int64_t n = P->L[l]->n;
      for (auto* v : {&lw.b64, &lw.x64, &lw.r64, &lw.y64}) v->resize(n);
      for (auto* v : {&lw.b32, &lw.x32, &lw.r32, &lw.y32}) v->resize(n);
      if (P->opt.smoother == 2 && !P->jacobi_only && l + 1 < P->L.size()) {
        const int m = P->opt.gmres_steps;
        if (P->opt.prec == TOMG_PREC_FP64) {
          lw.gV64.resize((m + 1) * n);
          lw.gZ64.resize(m * n);
        } else {
          lw.gV32.resize((m + 1) * n);
          lw.gZ32.resize(m * n);
        }
        lw.gparts.resize(gmres_smooth_parts(n));
        lw.gst.resize(1);
        CK(cudaMemsetAsync(lw.gst.p, 0, sizeof(GmState), W.stream));
      }
    }
    destroy_graph(W);
    W.built_for = P->setup_gen;
  }
  return W;
}

// make W's stream wait for everything enqueued so far on the problem stream
void fork_to(tomg_problem* P, Work& W) {
  CK(cudaEventRecord(W.evsync, st(P)));
  CK(cudaStreamWaitEvent(W.stream, W.evsync, 0));
}
void join_from(tomg_problem* P, Work& W) {
  CK(cudaEventRecord(W.evsync, W.stream));
  CK(cudaStreamWaitEvent(st(P), W.evsync, 0));
}

// initial residual, first preconditioned direction (graph-free)
void init_solve(tomg_problem* P, Work& W, int max_iter) {
  cudaStream_t s = W.stream;
  const int64_t n = P->n;
  fine64_resid(P, s, W.x.p, W.r.p, W.bvec.p);
  dot_partials(s, W.r.p, W.r.p, n, W.partA.p, nullptr);
  dot_partials(s, W.bvec.p, W.bvec.p, n, W.partB.p, nullptr);
  Scalars h;
  memset(&h, 0, sizeof(h));
  h.rtol2 = P->opt.rtol * P->opt.rtol;
  h.max_iter = max_iter;
  // the FP64 V-cycle is a fixed symmetric operator (PCG) unless the GMRES smoother makes it
  // depend on its input
  h.flexible = (P->opt.prec == TOMG_PREC_FP64 && P->opt.smoother != 2) ? 0 : 1;
  *W.sc_host = h;
  CK(cudaMemcpyAsync(W.sc.p, W.sc_host, sizeof(Scalars), cudaMemcpyHostToDevice, s));
  finish(s, FIN_INIT, W.partA.p, red_blocks(n), W.partB.p, red_blocks(n), W.sc.p);
  apply_M_and_dots(P, W, nullptr, &W.sc.p->done, false);  // + FIN_RZ0
  copy_f64(s, W.z.p, W.p.p, n, &W.sc.p->done);
}

// one attempt of the outer loop on slot W, then the true residual and compliance partials
// and the scalar state copied to pinned host memory; W.evdone marks completion
void launch_attempt(tomg_problem* P, Work& W, int max_iter) {
  cudaStream_t s = W.stream;
  const int64_t n = P->n;
  init_solve(P, W, max_iter);
  if (W.graph_mode == 2) {
    CK(cudaGraphLaunch(W.gexec, s));
  } else {
    // bounded host-polled loop: every check_every iterations read the scalar state
    const int every = std::max(1, P->opt.check_every);
    while (true) {
      for (int k = 0; k < every; k++) {
        if (W.graph_mode == 1) {
          CK(cudaGraphLaunch(W.gexec, s));
          g_launches += W.kernels_per_iter;
        } else {
          iteration_body(P, W);
        }
      }
      CK(cudaMemcpyAsync(W.sc_host, W.sc.p, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (W.sc_host->done) break;
    }
  }
  fine64_resid(P, s, W.x.p, W.t.p, W.bvec.p);
  dot_partials(s, W.t.p, W.t.p, n, W.partE.p, nullptr);
  dot_partials(s, W.f.p, W.x.p, n, W.partC.p, nullptr);
  const int nr = red_blocks(n);
  CK(cudaMemcpyAsync(W.sc_host, W.sc.p, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(W.partE_host, W.partE.p, sizeof(double) * nr, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(W.partC_host, W.partC.p, sizeof(double) * nr, cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(W.evdone, s));
}

// stage right-hand side j on slot W and launch its first attempt
void start_rhs(tomg_problem* P, Work& W, int j, const double* f, const double* u, int on_device) {
  cudaStream_t s = W.stream;
  const int64_t n = P->n;
  const cudaMemcpyKind h2d = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  W.rhs = j;
  W.attempts = 0;
  W.total_it = 0;
  CK(cudaEventRecord(W.ev0, s));
  CK(cudaMemcpyAsync(W.f.p, f + (int64_t)j * n, n * 8, h2d, s));
  CK(cudaMemcpyAsync(W.t.p, u + (int64_t)j * n, n * 8, h2d, s));
  mask_vec(s, W.f.p, W.bvec.p, P->mask.p, P->dim, P->nn);
  mask_vec(s, W.t.p, W.x.p, P->mask.p, P->dim, P->nn);
  if (!W.gexec && P->opt.use_graph > 0) {
    SetupTrace tr(W.stream);
    build_graph(P, W);
    tr.mark("graph build");
  }
  launch_attempt(P, W, P->opt.max_iter);
}

// wait for slot W's attempt; returns true when its right-hand side is finished (result
// written, u copy enqueued), false when it relaunched from the current iterate
bool finish_rhs(tomg_problem* P, Work& W, double* u, int on_device, tomg_result* res) {
  CK(cudaEventSynchronize(W.evdone));
  const int nr = red_blocks(P->n);
  const Scalars sc = *W.sc_host;
  if (W.graph_mode == 2) g_launches += W.kernels_per_iter * std::max(1, sc.it);
  W.total_it += sc.it;
  W.attempts++;
  double rr_true = 0.0, comp = 0.0;
  for (int q = 0; q < nr; q++) rr_true += W.partE_host[q];
  for (int q = 0; q < nr; q++) comp += W.partC_host[q];
  const double bb = sc.bb;
  const double tol2 = P->opt.rtol * P->opt.rtol * bb;
  int status = sc.status;
  if (status == TOMG_OK && bb > 0.0 && !(rr_true <= tol2)) {
    // recursive residual converged but the true one did not: restart from x
    if (W.attempts < 4 && W.total_it < P->opt.max_iter) {
      launch_attempt(P, W, P->opt.max_iter - W.total_it);
      return false;
    }
    status = TOMG_NOT_CONVERGED;
  }
  const int j = W.rhs;
  const int64_t n = P->n;
  CK(cudaMemcpyAsync(u + (int64_t)j * n, W.x.p, n * 8,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, W.stream));
  CK(cudaEventRecord(W.ev1, W.stream));
  CK(cudaEventSynchronize(W.ev1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, W.ev0, W.ev1));
  res[j].iterations = W.total_it;
  res[j].rel_residual = bb > 0.0 ? std::sqrt(rr_true / bb) : 0.0;
  res[j].compliance = comp;
  res[j].setup_ms = P->setup_ms;
  res[j].solve_ms = ms;
  res[j].status = status;
  if (status == TOMG_E_BREAKDOWN) {
    static const char* what[] = {"?", "NaN residual", "z.r <= 0 with a CG preconditioner",
                                 "p^T K p <= 0", "z.r or z.q not finite / z.r <= 0"};
    const int code = sc.pad;
    set_error("solver breakdown at iteration %d: %s (rhs %d)", W.total_it,
              what[(code >= 0 && code <= 4) ? code : 0], j);
  } else if (status == TOMG_NOT_CONVERGED) {
    set_error("not converged after %d iterations (rel residual %.3e, rhs %d)", W.total_it,
              res[j].rel_residual, j);
  }
  W.rhs = -1;
  return true;
}

// z = M v: one V-cycle of the current setup in its precision (FP64 in and out)
void precondition(tomg_problem* P, Work& W, const double* v, double* z) {
  cudaStream_t s = W.stream;
  const int64_t n = P->n;
  if (P->opt.prec == TOMG_PREC_FP64) {
    vcycle<double>(P, W, 0, v, z, nullptr);
  } else {
    LevelWork& l0 = W.lw[0];
    cast_in<float>(s, v, l0.b32.p, n, nullptr);
    vcycle<float>(P, W, 0, l0.b32.p, l0.y32.p, nullptr);
    cast_f32_f64(s, l0.y32.p, z, n);
  }
}

// h[0..J) = V_k . w, read back to the host (synchronises the stream)
void host_dots(cudaStream_t s, int64_t n, int J, const double* V, int64_t ldv, const double* w,
               double* parts, double* hd, double* hh) {
  multi_dot(s, n, J, V, ldv, w, parts, hd);
  CK(cudaMemcpyAsync(hh, hd, sizeof(double) * J, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
}

// Flexible GMRES(m) (Saad, Alg. 9.6), right preconditioned by the V-cycle: Arnoldi with
// classical Gram-Schmidt applied twice (two multi-dot / multi-update launches each) on the
// device, Givens rotations and the small triangular solve on the host.  Every cycle starts
// from the true FP64 residual b - K x; the solve stops when it is within rtol ||b||.
void solve_fgmres(tomg_problem* P, int nrhs, const double* f, double* u, int on_device,
                  tomg_result* res) {
  Work& W = ensure_work(P, 0);
  fork_to(P, W);
  cudaStream_t s = W.stream;
  const int64_t n = P->n;
  const int m = P->opt.gmres_restart;
  const cudaMemcpyKind h2d = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  DBuf<double> V, Z, w, hd, parts, cd;
  V.resize((int64_t)(m + 1) * n);
  Z.resize((int64_t)m * n);
  w.resize(n);
  hd.resize(m + 2);
  parts.resize(multi_dot_parts(m + 1));
  cd.resize(m + 1);
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), h1(m + 2), h2(m + 2), y(m);
  auto Hc = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  const double rtol2 = P->opt.rtol * P->opt.rtol;
  for (int rj = 0; rj < nrhs; rj++) {
    CK(cudaEventRecord(W.ev0, s));
    CK(cudaMemcpyAsync(W.f.p, f + (int64_t)rj * n, n * 8, h2d, s));
    CK(cudaMemcpyAsync(W.t.p, u + (int64_t)rj * n, n * 8, h2d, s));
    mask_vec(s, W.f.p, W.bvec.p, P->mask.p, P->dim, P->nn);
    mask_vec(s, W.t.p, W.x.p, P->mask.p, P->dim, P->nn);
    double bb = 0.0;
    host_dots(s, n, 1, W.bvec.p, n, W.bvec.p, parts.p, hd.p, &bb);
    int it = 0, status = TOMG_NOT_CONVERGED;
    double rr = 0.0;
    if (bb == 0.0) {
      CK(cudaMemsetAsync(W.x.p, 0, n * 8, s));
      status = TOMG_OK;
    }
    while (status != TOMG_OK) {
      fine64_resid(P, s, W.x.p, W.r.p, W.bvec.p);
      host_dots(s, n, 1, W.r.p, n, W.r.p, parts.p, hd.p, &rr);
      if (!std::isfinite(rr)) { status = TOMG_E_BREAKDOWN; break; }
      if (rr <= rtol2 * bb) { status = TOMG_OK; break; }
      if (it >= P->opt.max_iter) break;
      const double beta = std::sqrt(rr);
      scale_into(s, n, W.r.p, 1.0 / beta, V.p);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int k = 0;
      for (int j = 0; j < m; j++) {
        double* vj = V.p + (int64_t)j * n;
        double* zj = Z.p + (int64_t)j * n;
        precondition(P, W, vj, zj);
        fine64_apply_dot(P, s, zj, w.p, nullptr, nullptr, nullptr);
        host_dots(s, n, j + 1, V.p, n, w.p, parts.p, hd.p, h1.data());
        multi_update(s, n, j + 1, V.p, n, hd.p, -1.0, w.p);
        host_dots(s, n, j + 1, V.p, n, w.p, parts.p, hd.p, h2.data());
        multi_update(s, n, j + 1, V.p, n, hd.p, -1.0, w.p);
        double hn2 = 0.0;
        host_dots(s, n, 1, w.p, n, w.p, parts.p, hd.p, &hn2);
        const double hn = std::sqrt(hn2);
        for (int i = 0; i <= j; i++) Hc(i, j) = h1[i] + h2[i];
        if (hn > 0.0) scale_into(s, n, w.p, 1.0 / hn, V.p + (int64_t)(j + 1) * n);
        double hj1 = hn;
        for (int i = 0; i < j; i++) {
          const double t = cs[i] * Hc(i, j) + sn[i] * Hc(i + 1, j);
          Hc(i + 1, j) = -sn[i] * Hc(i, j) + cs[i] * Hc(i + 1, j);
          Hc(i, j) = t;
        }
        const double den = std::hypot(Hc(j, j), hj1);
        if (!(den > 0.0) || !std::isfinite(den)) { status = TOMG_E_BREAKDOWN; break; }
        cs[j] = Hc(j, j) / den;
        sn[j] = hj1 / den;
        Hc(j, j) = den;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        it++;
        k = j + 1;
        if (g[j + 1] * g[j + 1] <= rtol2 * bb || it >= P->opt.max_iter || hn == 0.0) break;
      }
      if (status == TOMG_E_BREAKDOWN) break;
      for (int i = k - 1; i >= 0; i--) {
        double a = g[i];
        for (int q = i + 1; q < k; q++) a -= Hc(i, q) * y[q];
        y[i] = a / Hc(i, i);
      }
      CK(cudaMemcpyAsync(cd.p, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
      multi_update(s, n, k, Z.p, n, cd.p, 1.0, W.x.p);
      CK(cudaStreamSynchronize(s));  // y is a host vector reused by the next cycle
    }
    // fixed DOFs exactly zero, compliance f^T u
    mask_vec(s, W.x.p, W.t.p, P->mask.p, P->dim, P->nn);
    double comp = 0.0;
    host_dots(s, n, 1, W.f.p, n, W.t.p, parts.p, hd.p, &comp);
    CK(cudaMemcpyAsync(u + (int64_t)rj * n, W.t.p, n * 8,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(W.ev1, s));
    CK(cudaEventSynchronize(W.ev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, W.ev0, W.ev1));
    res[rj].iterations = it;
    res[rj].rel_residual = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    res[rj].compliance = comp;
    res[rj].setup_ms = P->setup_ms;
    res[rj].solve_ms = ms;
    res[rj].status = status;
    if (status == TOMG_NOT_CONVERGED)
      set_error("FGMRES not converged after %d iterations (rel residual %.3e, rhs %d)", it,
                res[rj].rel_residual, rj);
    else if (status == TOMG_E_BREAKDOWN)
      set_error("FGMRES breakdown at iteration %d (rhs %d)", it, rj);
  }
  join_from(P, W);
}

// Work of a block solve of R right-hand sides: every outer vector and the FP32 V-cycle vectors
// of every level hold R vectors back to back (right-hand side r at r x length), R scalar
// states, R x (blocks) reduction partials
Work& ensure_block_work(tomg_problem* P, int R) {
  if (P->bwork && P->bwork->block != R) P->bwork.reset();
  if (!P->bwork) {
    auto W = std::make_unique<Work>();
    CK(cudaStreamCreateWithFlags(&W->stream, cudaStreamNonBlocking));
    CK(cudaEventCreate(&W->ev0));
    CK(cudaEventCreate(&W->ev1));
    CK(cudaEventCreateWithFlags(&W->evdone, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&W->evsync, cudaEventDisableTiming));
    W->block = R;
    const Ebe op{P->dim, P->nx, P->ny, P->nz, nullptr, nullptr, nullptr};
    W->np = std::max(std::max(stencil_blocks(Geo{P->dim, P->nx, P->ny, P->dim == 3 ? P->nz : 1}),
                              red_blocks(P->n)),
                     P->dim == 3 ? ebe3x_blocks(op) : 0);
    CK(cudaMallocHost((void**)&W->sc_host, sizeof(Scalars) * R));
    CK(cudaMallocHost((void**)&W->partE_host, sizeof(double) * W->np * R));
    CK(cudaMallocHost((void**)&W->partC_host, sizeof(double) * W->np * R));
    P->bwork = std::move(W);
  }
  Work& W = *P->bwork;
  if (W.built_for != P->setup_gen) {
    for (auto* v : {&W.f, &W.bvec, &W.x, &W.r, &W.p, &W.q, &W.z, &W.t}) v->resize(rhs_stride(P->n) * R);
    for (auto* v : {&W.partA, &W.partB, &W.partE, &W.partC}) v->resize((size_t)W.np * R);
    W.sc.resize(R);
    W.lw.resize(P->L.size());
    for (size_t l = 0; l < P->L.size(); l++) {
      LevelWork& lw = W.lw[l];
      for (auto* v : {&lw.b32, &lw.x32, &lw.r32, &lw.y32}) v->resize(rhs_stride(P->L[l]->n) * R);
    }
    destroy_graph(W);
    W.built_for = P->setup_gen;
  }
  return W;
}

// Block solve of right-hand sides [j0, j0 + R): one flexible-CG loop over all of them in one
// captured graph (block_iteration_body), then the true residuals and compliances.  A right-hand
// side whose recursive residual converged while its true one did not is finished by the
// single-right-hand-side path from the block's iterate.
void solve_block(tomg_problem* P, int j0, int R, const double* f, double* u, int on_device,
                 tomg_result* res) {
  Work& W = ensure_block_work(P, R);
  cudaStream_t s = W.stream;
  const int64_t n = P->n, ld = rhs_stride(n);  // right-hand side r at r x ld
  const cudaMemcpyKind h2d = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  fork_to(P, W);
  CK(cudaEventRecord(W.ev0, s));
  for (int r = 0; r < R; r++) {
    CK(cudaMemcpyAsync(W.f.p + r * ld, f + (int64_t)(j0 + r) * n, n * 8, h2d, s));
    CK(cudaMemcpyAsync(W.t.p + r * ld, u + (int64_t)(j0 + r) * n, n * 8, h2d, s));
    mask_vec(s, W.f.p + r * ld, W.bvec.p + r * ld, P->mask.p, P->dim, P->nn);
    mask_vec(s, W.t.p + r * ld, W.x.p + r * ld, P->mask.p, P->dim, P->nn);
  }
  if (!W.gexec) {
    SetupTrace tr(s);
    build_graph(P, W);
    tr.mark("block graph build");
  }
  const int nr = red_blocks(n);
  {
    BatchScope bs(R);
    fine64_resid(P, s, W.x.p, W.r.p, W.bvec.p);
    dot_partials(s, W.r.p, W.r.p, n, W.partA.p, nullptr);
    dot_partials(s, W.bvec.p, W.bvec.p, n, W.partB.p, nullptr);
    for (int r = 0; r < R; r++) {
      Scalars h;
      memset(&h, 0, sizeof(h));
      h.rtol2 = P->opt.rtol * P->opt.rtol;
      h.max_iter = P->opt.max_iter;
      h.flexible = 1;  // FP32 V-cycle
      W.sc_host[r] = h;
    }
    CK(cudaMemcpyAsync(W.sc.p, W.sc_host, sizeof(Scalars) * R, cudaMemcpyHostToDevice, s));
    finish(s, FIN_INIT, W.partA.p, nr, W.partB.p, nr, W.sc.p);
    cast_in<float>(s, W.r.p, W.lw[0].b32.p, n, nullptr);
    vcycle<float>(P, W, 0, W.lw[0].b32.p, W.lw[0].y32.p, nullptr);
    z_dots<float>(s, W.lw[0].y32.p, W.z.p, W.r.p, nullptr, n, W.partA.p, W.partB.p, W.sc.p,
                  FIN_RZ0);
    copy_f64(s, W.z.p, W.p.p, n, nullptr);
  }
  CK(cudaGraphLaunch(W.gexec, s));
  {
    BatchScope bs(R);
    fine64_resid(P, s, W.x.p, W.t.p, W.bvec.p);
    dot_partials(s, W.t.p, W.t.p, n, W.partE.p, nullptr);
    dot_partials(s, W.f.p, W.x.p, n, W.partC.p, nullptr);
  }
  CK(cudaMemcpyAsync(W.sc_host, W.sc.p, sizeof(Scalars) * R, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(W.partE_host, W.partE.p, sizeof(double) * nr * R, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(W.partC_host, W.partC.p, sizeof(double) * nr * R, cudaMemcpyDeviceToHost, s));
  for (int r = 0; r < R; r++)
    CK(cudaMemcpyAsync(u + (int64_t)(j0 + r) * n, W.x.p + r * ld, n * 8,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(W.ev1, s));
  CK(cudaEventSynchronize(W.ev1));
  join_from(P, W);
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, W.ev0, W.ev1));
  int max_it = 0;
  for (int r = 0; r < R; r++) max_it = std::max(max_it, W.sc_host[r].it);
  g_launches += W.kernels_per_iter * std::max(1, max_it);
  std::vector<int> again;
  for (int r = 0; r < R; r++) {
    const Scalars& sc = W.sc_host[r];
    double rr_true = 0.0, comp = 0.0;
    for (int q = 0; q < nr; q++) rr_true += W.partE_host[(size_t)r * nr + q];
    for (int q = 0; q < nr; q++) comp += W.partC_host[(size_t)r * nr + q];
    tomg_result& o = res[j0 + r];
    o.iterations = sc.it;
    o.rel_residual = sc.bb > 0.0 ? std::sqrt(rr_true / sc.bb) : 0.0;
    o.compliance = comp;
    o.setup_ms = P->setup_ms;
    o.solve_ms = ms;
    o.status = sc.status;
    if (sc.status == TOMG_OK && sc.bb > 0.0 &&
        !(rr_true <= P->opt.rtol * P->opt.rtol * sc.bb) && sc.it < P->opt.max_iter)
      again.push_back(j0 + r);
  }
  // the single path restarts from the block's iterate (u now holds it)
  for (int j : again) {
    const int it0 = res[j].iterations;
    const float ms0 = (float)res[j].solve_ms;
    tomg_options o = P->opt;
    P->opt.block_rhs = 0;
    P->opt.max_iter = std::max(1, o.max_iter - it0);
    try {
      solve(P, 1, f + (int64_t)j * n, u + (int64_t)j * n, on_device, &res[j]);
    } catch (...) {
      P->opt = o;
      throw;
    }
    P->opt = o;
    res[j].iterations += it0;
    res[j].solve_ms += ms0;
  }
}

}  // namespace

tomg_status solve(tomg_problem* P, int nrhs, const double* f, double* u, int on_device,
                  tomg_result* res) {
  if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "tomg_solve: call tomg_setup after changing density or fixed DOFs");
  if (nrhs < 0 || (nrhs > 0 && (!f || !u || !res))) TOMG_THROW(TOMG_E_INVALID, "bad solve arguments");
  if (nrhs == 0) return TOMG_OK;
  if (P->opt.krylov == 1) {
    solve_fgmres(P, nrhs, f, u, on_device, res);
  } else if (P->opt.block_rhs > 1 && nrhs > 1) {
    const int64_t n = P->n;
    for (int j0 = 0; j0 < nrhs; j0 += P->opt.block_rhs) {
      const int R = std::min(P->opt.block_rhs, nrhs - j0);
      if (R > 1) {
        solve_block(P, j0, R, f, u, on_device, res);
        continue;
      }
      // a last single right-hand side: the slot path
      const tomg_options o = P->opt;
      P->opt.block_rhs = 0;
      try {
        solve(P, 1, f + j0 * n, u + j0 * n, on_device, res + j0);
      } catch (...) {
        P->opt = o;
        throw;
      }
      P->opt = o;
    }
  } else {
    const int slots = std::max(1, std::min(nrhs, P->opt.concurrency > 0 ? P->opt.concurrency : 1));
    for (int k = 0; k < slots; k++) ensure_work(P, k);
    for (int k = 0; k < slots; k++) fork_to(P, *P->works[k]);
    int next = 0;
    for (int k = 0; k < slots; k++) start_rhs(P, *P->works[k], next++, f, u, on_device);
    int active = slots;
    while (active > 0) {
      for (int k = 0; k < slots; k++) {
        Work& W = *P->works[k];
        if (W.rhs < 0) continue;
        if (!finish_rhs(P, W, u, on_device, res)) continue;
        if (next < nrhs) start_rhs(P, W, next++, f, u, on_device);
        else active--;
      }
    }
    for (int k = 0; k < slots; k++) join_from(P, *P->works[k]);
  }
  CK(cudaStreamSynchronize(st(P)));
  if (P->dim == 3 && ((P->opt.prec == TOMG_PREC_TC_VCYCLE && ebe3d_tc_error(st(P))) ||
                      (x64_active(P) && ebe3x_error(st(P)))))
    for (int j = 0; j < nrhs; j++) res[j].status = TOMG_E_TIMEOUT;
  if (P->opt.pc == TOMG_PC_HYBRID && P->opt.adaptive_geo && P->adapt_geo > 0) {
    // adaptive hybrid (Sec. 4.4): a solve over the iteration limit moves the next setup one
    // geometric level towards aggregation
    int worst_it = 0;
    for (int j = 0; j < nrhs; j++) worst_it = std::max(worst_it, res[j].iterations);
    if (worst_it > P->opt.adaptive_iters && P->adapt_geo > P->opt.adaptive_min_geo) P->adapt_geo--;
  }
  tomg_status worst = TOMG_OK;
  for (int j = 0; j < nrhs; j++) {
    const int s = res[j].status;
    if (s < 0 || (worst >= 0 && s > worst)) worst = (tomg_status)s;
  }
  return worst;
}

// ----------------------------------------------------------------------------------------
// Linear buckling: K_sigma from the centre stresses of u, generalized Davidson (Algorithm 2)
namespace {
// eigenvalues (descending) and orthonormal eigenvectors (columns of Q, n x n row-major) of the
// symmetric n x n matrix A (row-major, destroyed) by cyclic Jacobi rotations
void sym_eig(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& Q) {
  Q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; i++) Q[(size_t)i * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; i++)
      for (int j = 0; j < n; j++) {
        tot += a(i, j) * a(i, j);
        if (i != j) off += a(i, j) * a(i, j);
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; p++)
      for (int q = p + 1; q < n; q++) {
        if (a(p, q) == 0.0) continue;
        const double th = 0.5 * (a(q, q) - a(p, p)) / a(p, q);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; k++) {  // columns p, q
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - sn * akq;
          a(k, q) = sn * akp + c * akq;
        }
        for (int k = 0; k < n; k++) {  // rows p, q
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - sn * aqk;
          a(q, k) = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; k++) {
          const double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
          Q[(size_t)k * n + p] = c * qkp - sn * qkq;
          Q[(size_t)k * n + q] = sn * qkp + c * qkq;
        }
      }
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; i++) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int x, int y) { return a(x, x) > a(y, y); });
  w.resize(n);
  std::vector<double> Qs((size_t)n * n);
  for (int c = 0; c < n; c++) {
    w[c] = a(idx[c], idx[c]);
    for (int k = 0; k < n; k++) Qs[(size_t)k * n + c] = Q[(size_t)k * n + idx[c]];
  }
  Q.swap(Qs);
}
}  // namespace

void stress_stiffness_op(tomg_problem* P, const double* u, const double* x, double* y) {
  cudaStream_t s = st(P);
  DBuf<double> sig;
  sig.resize(P->nel * stress_components(P->dim));
  element_stresses(s, P->dim, P->nx, P->ny, P->nz, P->nu, P->E0, P->penal, P->rho.p, u, sig.p);
  stress_stiffness_apply(s, P->dim, P->nx, P->ny, P->nz, P->nu, sig.p, P->mask.p, x, y);
  CK(cudaStreamSynchronize(s));
}

tomg_status buckling(tomg_problem* P, const double* u, int n_eig, int jmin, int jmax, double tol,
                     int max_iter, double* lambdas, double* modes, int on_device, int* iterations) {
  if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "tomg_buckling: needs a setup");
  if (n_eig < 1 || n_eig > 16 || jmin <= n_eig || jmax <= jmin || jmax > 64 || !(tol > 0.0) ||
      max_iter < 0 || !lambdas)
    TOMG_THROW(TOMG_E_INVALID, "bad buckling arguments");
  Work& W = ensure_work(P, 0);
  fork_to(P, W);
  cudaStream_t s = W.stream;
  const int64_t n = P->n;
  DBuf<double> du, sig, V, KV, SV, z, Kz, r, q, tmp, parts, hd, cd, dm;
  const double* uu = u;
  if (!on_device) {
    du.resize(n);
    CK(cudaMemcpyAsync(du.p, u, n * 8, cudaMemcpyHostToDevice, s));
    uu = du.p;
  }
  sig.resize(P->nel * stress_components(P->dim));
  element_stresses(s, P->dim, P->nx, P->ny, P->nz, P->nu, P->E0, P->penal, P->rho.p, uu, sig.p);
  V.resize((int64_t)jmax * n); KV.resize((int64_t)jmax * n); SV.resize((int64_t)jmax * n);
  z.resize(n); Kz.resize(n); r.resize(n); q.resize(n); tmp.resize((int64_t)jmin * n);
  parts.resize(multi_dot_parts(jmax + 1)); hd.resize(jmax + 1); cd.resize(jmax + 1);
  auto Kapply = [&](const double* x, double* y) { fine64_apply_dot(P, s, x, y, nullptr, nullptr, nullptr); };
  auto Sapply = [&](const double* x, double* y) {
    stress_stiffness_apply(s, P->dim, P->nx, P->ny, P->nz, P->nu, sig.p, P->mask.p, x, y);
  };
  auto dot = [&](const double* a, const double* b) {
    double v = 0.0;
    host_dots(s, n, 1, a, n, b, parts.p, hd.p, &v);
    return v;
  };
  std::vector<double> Hp((size_t)jmax * jmax, 0.0), h(jmax + 1), c(jmax + 1);
  int j = 0;
  // K-orthonormalise z against V (classical Gram-Schmidt twice) and append it
  auto add_vector = [&]() -> bool {
    const double n0 = std::sqrt(dot(z.p, z.p));
    for (int pass = 0; pass < 2 && j > 0; pass++) {
      multi_dot(s, n, j, KV.p, n, z.p, parts.p, hd.p);
      multi_update(s, n, j, V.p, n, hd.p, -1.0, z.p);
    }
    if (!(std::sqrt(dot(z.p, z.p)) > 1e-10 * n0)) return false;
    Kapply(z.p, Kz.p);
    const double nz = std::sqrt(std::max(dot(z.p, Kz.p), 0.0));
    if (!(nz > 0.0)) return false;
    scale_into(s, n, z.p, 1.0 / nz, V.p + (int64_t)j * n);
    scale_into(s, n, Kz.p, 1.0 / nz, KV.p + (int64_t)j * n);
    Sapply(V.p + (int64_t)j * n, SV.p + (int64_t)j * n);
    host_dots(s, n, j + 1, V.p, n, SV.p + (int64_t)j * n, parts.p, hd.p, h.data());
    for (int i = 0; i <= j; i++) Hp[(size_t)i * jmax + j] = Hp[(size_t)j * jmax + i] = h[i];
    j++;
    return true;
  };
  // out = sum_k coef[k] M_k over the first j columns of M (device coefficients through cd)
  auto combine = [&](const double* M, const double* coef, double sign, double* out, bool zero) {
    CK(cudaMemcpyAsync(cd.p, coef, sizeof(double) * j, cudaMemcpyHostToDevice, s));
    if (zero) CK(cudaMemsetAsync(out, 0, n * 8, s));
    multi_update(s, n, j, M, n, cd.p, sign, out);
    CK(cudaStreamSynchronize(s));  // coef is a host vector the caller may reuse
  };
  for (int k = 0; k < jmin; k++) {
    splitmix_uniform(s, n, 1000 + k, z.p);
    add_vector();
  }
  int it = 0, status = TOMG_NOT_CONVERGED;
  std::vector<double> th, Q, Hw;
  int k = 0;
  while (true) {
    Hw.assign((size_t)j * j, 0.0);
    for (int a = 0; a < j; a++)
      for (int b = 0; b < j; b++) Hw[(size_t)a * j + b] = Hp[(size_t)a * jmax + b];
    sym_eig(j, Hw, th, Q);
    k = std::min(n_eig, j);
    int t = -1;
    for (int i = 0; i < k && t < 0; i++) {
      for (int a = 0; a < j; a++) c[a] = Q[(size_t)a * j + i];
      combine(SV.p, c.data(), 1.0, r.p, true);
      combine(KV.p, c.data(), -th[i], r.p, false);
      combine(KV.p, c.data(), 1.0, q.p, true);
      const double nr = std::sqrt(dot(r.p, r.p)), nq = std::sqrt(dot(q.p, q.p));
      if (!std::isfinite(nr)) { status = TOMG_E_BREAKDOWN; break; }
      if (!(nr <= tol * std::fabs(th[i]) * nq)) t = i;
    }
    if (status == TOMG_E_BREAKDOWN) break;
    if (t < 0) { status = TOMG_OK; break; }
    if (it >= max_iter) break;
    if (j >= jmax) {
      // restart from the j_min best Ritz vectors (V^T K_sigma V becomes diagonal)
      for (DBuf<double>* M : {&V, &KV, &SV}) {
        for (int cc = 0; cc < jmin; cc++) {
          for (int a = 0; a < j; a++) c[a] = Q[(size_t)a * j + cc];
          combine(M->p, c.data(), 1.0, tmp.p + (int64_t)cc * n, true);
        }
        CK(cudaMemcpyAsync(M->p, tmp.p, (size_t)jmin * n * 8, cudaMemcpyDeviceToDevice, s));
      }
      std::fill(Hp.begin(), Hp.end(), 0.0);
      for (int a = 0; a < jmin; a++) Hp[(size_t)a * jmax + a] = th[a];
      j = jmin;
    }
    precondition(P, W, r.p, z.p);
    it++;
    add_vector();
  }
  for (int i = 0; i < k; i++) lambdas[i] = th[i];
  if (modes) {
    for (int i = 0; i < k; i++) {
      for (int a = 0; a < j; a++) c[a] = Q[(size_t)a * j + i];
      combine(V.p, c.data(), 1.0, q.p, true);
      CK(cudaMemcpyAsync(modes + (int64_t)i * n, q.p, n * 8,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    }
  }
  CK(cudaStreamSynchronize(s));
  join_from(P, W);
  if (iterations) *iterations = it;
  if (status == TOMG_NOT_CONVERGED) set_error("Davidson not converged after %d iterations", it);
  if (status == TOMG_E_BREAKDOWN) set_error("Davidson breakdown (non-finite residual)");
  return (tomg_status)status;
}

// ----------------------------------------------------------------------------------------
void level_apply(tomg_problem* P, int level, int prec, const double* x, double* y) {
  if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "no valid setup");
  if (level < 0 || level >= (int)P->L.size()) TOMG_THROW(TOMG_E_INVALID, "bad level %d", level);
  Work& W = ensure_work(P, 0);
  LevelWork& lw = W.lw[level];
  const int64_t n = P->L[level]->n;
  cudaStream_t s = st(P);
  if (prec == TOMG_PREC_FP64) {
    CK(cudaMemcpyAsync(lw.b64.p, x, n * 8, cudaMemcpyDeviceToDevice, s));
    level_op<double>(P, s, level, MODE_APPLY, lw.b64.p, lw.y64.p, nullptr, nullptr);
    CK(cudaMemcpyAsync(y, lw.y64.p, n * 8, cudaMemcpyDeviceToDevice, s));
  } else {
    TcScope tcs(P, prec);
    cast_f64_f32(s, x, lw.b32.p, n);
    level_op<float>(P, s, level, MODE_APPLY, lw.b32.p, lw.y32.p, nullptr, nullptr);
    cast_f32_f64(s, lw.y32.p, y, n);
  }
  CK(cudaStreamSynchronize(s));
  if (P->dim == 3 && prec == TOMG_PREC_TC_VCYCLE && ebe3d_tc_error(s))
    TOMG_THROW(TOMG_E_TIMEOUT, "tensor-core element kernel: MMA completion wait expired");
}

void outer_operator_apply(tomg_problem* P, const double* x, double* y) {
  if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "no valid setup");
  cudaStream_t s = st(P);
  fine64_apply_dot(P, s, x, y, nullptr, nullptr, nullptr);
  CK(cudaStreamSynchronize(s));
}

void vcycle_apply(tomg_problem* P, const double* r, double* z) {
  if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "no valid setup");
  Work& W = ensure_work(P, 0);
  fork_to(P, W);
  CK(cudaMemcpyAsync(W.r.p, r, P->n * 8, cudaMemcpyDeviceToDevice, W.stream));
  // fresh scalar state: the z.r reduction then runs (and is discarded) like at a solve start
  CK(cudaMemsetAsync(W.sc.p, 0, sizeof(Scalars), W.stream));
  apply_M_and_dots(P, W, nullptr, nullptr, false);
  CK(cudaMemcpyAsync(z, W.z.p, P->n * 8, cudaMemcpyDeviceToDevice, W.stream));
  join_from(P, W);
  CK(cudaStreamSynchronize(st(P)));
}

void coarse_apply(tomg_problem* P, const double* b, double* x) {
  if (!P->setup_valid || P->jacobi_only) TOMG_THROW(TOMG_E_INVALID, "no coarse level");
  cudaStream_t s = st(P);
  dense_gemv<double>(s, P->nc, P->Ainv64.p, b, x, nullptr);
  CK(cudaStreamSynchronize(s));
}

namespace {
void bsr_to_host(cudaStream_t s, int nbr, int bb, const int* rp, const int* ci, const double* v,
                 int64_t nnzb, int64_t* hrp, int64_t* hci, double* hv) {
  std::vector<int> trp(nbr + 1), tci(nnzb);
  CK(cudaMemcpyAsync(trp.data(), rp, (nbr + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (nnzb) CK(cudaMemcpyAsync(tci.data(), ci, nnzb * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (nnzb) CK(cudaMemcpyAsync(hv, v, nnzb * bb * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i <= nbr; i++) hrp[i] = trp[i];
  for (int64_t i = 0; i < nnzb; i++) hci[i] = tci[i];
}
}  // namespace

void level_export(tomg_problem* P, int level, int64_t* nnzb, int64_t* hrp, int64_t* hci, double* hv) {
  if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "no valid setup");
  if (level < 0 || level >= (int)P->L.size()) TOMG_THROW(TOMG_E_INVALID, "bad level %d", level);
  Level& Lv = *P->L[level];
  cudaStream_t s = st(P);
  if (Lv.kind == KIND_BSR) {
    *nnzb = Lv.nnzb;
    if (hrp) bsr_to_host(s, (int)Lv.nn, Lv.b * Lv.b, Lv.rp.p, Lv.ci.p, Lv.V64.p, Lv.nnzb, hrp, hci, hv);
    return;
  }
  // stencil levels (level 0 assembled on the fly) -> block CSR
  Level tmp;
  tmp.kind = KIND_STENCIL;
  tmp.b = Lv.b; tmp.nn = Lv.nn; tmp.n = Lv.n; tmp.g = Lv.g;
  tmp.S64.resize((int64_t)stencil_q(P->dim) * Lv.nn);
  if (Lv.kind == KIND_EBE) ebe_assemble_stencil(s, V<double>::ebe(P), tmp.S64.p);
  else CK(cudaMemcpyAsync(tmp.S64.p, Lv.S64.p, Lv.S64.bytes(), cudaMemcpyDeviceToDevice, s));
  make_bsr_from_stencil(P, tmp);
  *nnzb = tmp.nnzb;
  if (hrp) bsr_to_host(s, (int)tmp.nn, tmp.b * tmp.b, tmp.rp.p, tmp.ci.p, tmp.V64.p, tmp.nnzb, hrp, hci, hv);
}

void prolong_export(tomg_problem* P, int level, int64_t* nnzb, int64_t* hrp, int64_t* hci, double* hv) {
  if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "no valid setup");
  if (level < 0 || level + 1 >= (int)P->L.size()) TOMG_THROW(TOMG_E_INVALID, "no prolongation below level %d", level);
  Level& Lv = *P->L[level];
  Level& C = *P->L[level + 1];
  cudaStream_t s = st(P);
  if (!Lv.geo_next) {
    *nnzb = Lv.Pnnzb;
    if (hrp) bsr_to_host(s, (int)Lv.nn, Lv.b * Lv.bc, Lv.Prp.p, Lv.Pci.p, Lv.Pv64.p, Lv.Pnnzb, hrp, hci, hv);
    return;
  }
  DBuf<int> counts, rp, ci;
  DBuf<double> v;
  counts.resize(Lv.nn);
  rp.resize(Lv.nn + 1);
  geo_prolong_counts(s, Lv.g, C.g, counts.p);
  const int64_t nz = exclusive_scan(s, counts.p, rp.p, Lv.nn);
  ci.resize(nz);
  v.resize(nz * Lv.b * Lv.b);
  geo_prolong_fill(s, Lv.g, C.g, rp.p, ci.p, v.p);
  *nnzb = nz;
  if (hrp) bsr_to_host(s, (int)Lv.nn, Lv.b * Lv.b, rp.p, ci.p, v.p, nz, hrp, hci, hv);
}


double time_fine_operator(tomg_problem* P, int op, int prec, int reps, int cold_l2) {
  if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "no valid setup");
  if (op < 0 || op > 3 || reps < 1 || reps > 10000) TOMG_THROW(TOMG_E_INVALID, "bad timing request");
  cudaStream_t s = st(P);
  Work& W = ensure_work(P, 0);
  LevelWork& l0 = W.lw[0];
  const int mode = op == 0 ? MODE_APPLY : (op == 1 ? MODE_RESID : MODE_JACOBI);
  DBuf<char> flush;
  if (cold_l2) flush.resize((size_t)256 << 20);
  std::vector<cudaEvent_t> ev(2 * reps);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  for (int k = 0; k < reps; k++) {
    if (cold_l2) CK(cudaMemsetAsync(flush.p, k & 0xff, flush.n, s));
    CK(cudaEventRecord(ev[2 * k], s));
    if (op == 3) fine64_apply_dot(P, s, W.p.p, W.q.p, nullptr, W.partA.p, nullptr);
    else if (prec == TOMG_PREC_FP64) level_op<double>(P, s, 0, mode, l0.x64.p, l0.y64.p, l0.b64.p, nullptr);
    else {
      TcScope tcs(P, prec);
      level_op<float>(P, s, 0, mode, l0.x32.p, l0.y32.p, l0.b32.p, nullptr);
    }
    CK(cudaEventRecord(ev[2 * k + 1], s));
  }
  CK(cudaStreamSynchronize(s));
  double tot = 0.0;
  for (int k = 0; k < reps; k++) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
    tot += ms;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return tot / reps;
}

}  // namespace tomg

// device bytes the problem holds: its inputs, the hierarchy and every solve slot
size_t tomg::problem_device_bytes(const tomg_problem* P) {
  using namespace tomg;
  size_t b = P->Ketc.bytes() + P->Kx64.bytes() + P->Ke64.bytes() + P->Ke32.bytes() + P->mask.bytes() +
             P->rho.bytes() + P->E64.bytes() + P->E32.bytes() + P->flag_dev.bytes() +
             P->Ainv64.bytes() + P->Ainv32.bytes();
  for (const auto& lp : P->L) {
    const Level& l = *lp;
    b += l.S64.bytes() + l.S32.bytes() + l.rp.bytes() + l.ci.bytes() + l.V64.bytes() +
         l.V32.bytes() + l.D64.bytes() + l.D32.bytes() + l.Prp.bytes() + l.Pci.bytes() +
         l.Rrp.bytes() + l.Rci.bytes() + l.Pv64.bytes() + l.Rv64.bytes() + l.Pv32.bytes() +
         l.Rv32.bytes() + l.agg.bytes();
  }
  std::vector<const Work*> all;
  for (const auto& wp : P->works) all.push_back(wp.get());
  if (P->bwork) all.push_back(P->bwork.get());
  for (const Work* wp : all) {
    const Work& w = *wp;
    b += w.f.bytes() + w.bvec.bytes() + w.x.bytes() + w.r.bytes() + w.p.bytes() + w.q.bytes() +
         w.z.bytes() + w.t.bytes() + w.partA.bytes() + w.partB.bytes() + w.partE.bytes() +
         w.partC.bytes() + w.sc.bytes();
    for (const auto& lw : w.lw)
      b += lw.b64.bytes() + lw.x64.bytes() + lw.r64.bytes() + lw.y64.bytes() + lw.b32.bytes() +
           lw.x32.bytes() + lw.r32.bytes() + lw.y32.bytes() + lw.gV64.bytes() + lw.gZ64.bytes() +
           lw.gparts.bytes() + lw.gV32.bytes() + lw.gZ32.bytes() + lw.gst.bytes();
  }
  return b;
}

tomg_problem::~tomg_problem() {
  if (stream) cudaStreamSynchronize(stream);
  works.clear();
  bwork.reset();
  L.clear();
  if (flag_host) cudaFreeHost(flag_host);
  for (cudaEvent_t e : {ev0, ev1, ev_in, ev_out, ev_fork, ev_side, ev_fork2, ev_side2})
    if (e) cudaEventDestroy(e);
  // device buffers are released by their destructors on this stream before it is destroyed
  Ke64.release(); Ke32.release(); Ketc.release(); Kx64.release(); mask.release(); rho.release(); E64.release(); E32.release();
  flag_dev.release(); Ainv64.release(); Ainv32.release();
  if (stream) {
    cudaStreamSynchronize(stream);
    cudaStreamDestroy(stream);
  }
  for (cudaStream_t q : {side, side2})
    if (q) {
      cudaStreamSynchronize(q);
      cudaStreamDestroy(q);
    }
}
