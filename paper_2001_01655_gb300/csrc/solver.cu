// Host runtime: problem state, preconditioner setup (Sec. 3.2 Eq. 9, Sec. 4), the V-cycle of
// Algorithm 1 with point-block Jacobi smoothing, and the outer CG / flexible-CG loop (Sec. 3.1)
// whose iteration is captured once into a CUDA graph with a device-side while loop, so a
// whole solve is one graph launch with no host round trip per iteration.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "solver.h"

namespace tomg {

// ----------------------------------------------------------------------------------------
// element stiffness by 2x2(x2) Gauss quadrature on the unit element (bilinear quad4 plane
// stress, trilinear hex8 isotropic); local node a = (a&1, a>>1&1, a>>2&1), DOF = dim*a + c
void element_stiffness_host(int dim, double nu, std::vector<double>& Ke) {
  const int nn = 1 << dim, nd = dim * nn, ns = dim == 2 ? 3 : 6;
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
  static double* b(Level& l) { return l.b64.p; }
  static double* x(Level& l) { return l.x64.p; }
  static double* r(Level& l) { return l.r64.p; }
  static double* y(Level& l) { return l.y64.p; }
  static const double* Ainv(const tomg_problem* P) { return P->Ainv64.p; }
  static Ebe ebe(const tomg_problem* P) {
    return Ebe{P->dim, P->nx, P->ny, P->nz, P->Ke64.p, P->E64.p, P->mask.p};
  }
};
template <> struct V<float> {
  static const float* S(const Level& l) { return l.S32.p; }
  static const float* Vv(const Level& l) { return l.V32.p; }
  static const float* D(const Level& l) { return l.D32.p; }
  static const float* Pv(const Level& l) { return l.Pv32.p; }
  static const float* Rv(const Level& l) { return l.Rv32.p; }
  static float* b(Level& l) { return l.b32.p; }
  static float* x(Level& l) { return l.x32.p; }
  static float* r(Level& l) { return l.r32.p; }
  static float* y(Level& l) { return l.y32.p; }
  static const float* Ainv(const tomg_problem* P) { return P->Ainv32.p; }
  static Ebe ebe(const tomg_problem* P) {
    return Ebe{P->dim, P->nx, P->ny, P->nz, P->Ke32.p, P->E32.p, P->mask.p};
  }
};

inline cudaStream_t st(const tomg_problem* P) { return P->ctx->stream; }

template <class T>
void level_op(tomg_problem* P, int l, int mode, const T* x, T* y, const T* b, const int* done) {
  Level& Lv = *P->L[l];
  const double w = P->opt.omega;
  switch (Lv.kind) {
    case KIND_EBE:
      ebe_op<T>(st(P), mode, V<T>::ebe(P), x, y, b, V<T>::D(Lv), w, done, nullptr);
      break;
    case KIND_STENCIL:
      stencil_op<T>(st(P), mode, Lv.g, V<T>::S(Lv), x, y, b, V<T>::D(Lv), w, done);
      break;
    default:
      bsr_op<T>(st(P), mode, Lv.bsr(), V<T>::Vv(Lv), x, y, b, V<T>::D(Lv), w, done);
  }
}

template <class T>
void restrict_to(tomg_problem* P, int l, const T* r, T* bc, const int* done) {
  Level& Lv = *P->L[l];
  Level& C = *P->L[l + 1];
  if (Lv.geo_next) geo_restrict<T>(st(P), Lv.g, C.g, r, bc, done);
  else bsr_spmv_rect<T>(st(P), Lv.Rmat(C.nn), V<T>::Rv(Lv), r, bc, 0, done);
}

template <class T>
void prolong_add(tomg_problem* P, int l, const T* xc, T* x, const int* done) {
  Level& Lv = *P->L[l];
  Level& C = *P->L[l + 1];
  if (Lv.geo_next) geo_prolong_add<T>(st(P), Lv.g, C.g, xc, x, done);
  else bsr_spmv_rect<T>(st(P), Lv.Pmat(C.nn), V<T>::Pv(Lv), xc, x, 1, done);
}

// V-cycle of Algorithm 1: out = MG(b) on level l (x = 0 initial guess)
template <class T>
void vcycle(tomg_problem* P, int l, const T* b, T* out, const int* done) {
  Level& Lv = *P->L[l];
  const int nl = (int)P->L.size();
  const double w = P->opt.omega;
  if (P->jacobi_only) {
    jacobi0<T>(st(P), Lv.b, Lv.nn, V<T>::D(Lv), b, out, w, done);
    return;
  }
  if (l == nl - 1) {
    dense_gemv<T>(st(P), P->nc, V<T>::Ainv(P), b, out, done);
    return;
  }
  T* x = V<T>::x(Lv);
  T* r = V<T>::r(Lv);
  // pre-smoothing, the first sweep from x = 0 needs no operator apply
  jacobi0<T>(st(P), Lv.b, Lv.nn, V<T>::D(Lv), b, x, w, done);
  for (int k = 1; k < P->opt.n_pre; k++) {
    level_op<T>(P, l, MODE_JACOBI, x, r, b, done);
    std::swap(x, r);
  }
  level_op<T>(P, l, MODE_RESID, x, r, b, done);  // r = b - A x
  Level& C = *P->L[l + 1];
  restrict_to<T>(P, l, r, V<T>::b(C), done);
  vcycle<T>(P, l + 1, V<T>::b(C), V<T>::y(C), done);
  prolong_add<T>(P, l, V<T>::y(C), x, done);
  T* cur = x;
  for (int k = 0; k < P->opt.n_post; k++) {
    T* dst = (k == P->opt.n_post - 1) ? out : (cur == x ? r : x);
    level_op<T>(P, l, MODE_JACOBI, cur, dst, b, done);
    cur = dst;
  }
}

// z = M r (outer residual in FP64), then partials of z.r (and z.q)
void apply_M_and_dots(tomg_problem* P, const double* q, const int* done) {
  const int64_t n = P->n;
  Level& L0 = *P->L[0];
  if (P->opt.prec == TOMG_PREC_FP64) {
    vcycle<double>(P, 0, P->r.p, P->z.p, done);
    z_dots<double>(st(P), P->z.p, P->z.p, P->r.p, q, n, P->partA.p, q ? P->partB.p : nullptr, done);
  } else {
    cast_in<float>(st(P), P->r.p, L0.b32.p, n, done);
    vcycle<float>(P, 0, L0.b32.p, L0.y32.p, done);
    z_dots<float>(st(P), L0.y32.p, P->z.p, P->r.p, q, n, P->partA.p, q ? P->partB.p : nullptr, done);
  }
}

void iteration_body(tomg_problem* P) {
  const int64_t n = P->n;
  Scalars* sc = P->sc.p;
  const int* done = &sc->done;
  const Ebe op = V<double>::ebe(P);
  ebe_op<double>(st(P), MODE_APPLY, op, P->p.p, P->q.p, nullptr, nullptr, 0.0, done, P->partA.p);
  finish(st(P), FIN_ALPHA, P->partA.p, ebe_blocks(op), nullptr, 0, sc);
  xr_update(st(P), P->x.p, P->r.p, P->p.p, P->q.p, n, sc, P->partA.p);
  finish(st(P), FIN_RR, P->partA.p, red_blocks(n), nullptr, 0, sc);
  apply_M_and_dots(P, P->q.p, done);
  finish(st(P), FIN_BETA, P->partA.p, red_blocks(n), P->partB.p, red_blocks(n), sc);
  p_update(st(P), P->p.p, P->z.p, n, sc);
}

void destroy_graph(tomg_problem* P) {
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->graph) cudaGraphDestroy(P->graph);
  P->gexec = nullptr;
  P->graph = nullptr;
  P->graph_mode = 0;
}

void build_graph(tomg_problem* P) {
  destroy_graph(P);
  const int mode = P->opt.use_graph;
  if (mode <= 0) return;
  cudaStream_t s = st(P);
  const int64_t saved = g_launches;
  if (mode >= 2) {
    CK(cudaGraphCreate(&P->graph, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, P->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, P->graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
      iteration_body(P);
      set_conditional(s, h, P->sc.p);
    } catch (...) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(s, &dummy);
      g_launches = saved;
      throw;
    }
    CK(cudaStreamEndCapture(s, &body));
  } else {
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
      iteration_body(P);
    } catch (...) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(s, &dummy);
      g_launches = saved;
      throw;
    }
    CK(cudaStreamEndCapture(s, &P->graph));
  }
  P->kernels_per_iter = g_launches - saved;
  g_launches = saved;
  CK(cudaGraphInstantiate(&P->gexec, P->graph, 0));
  P->graph_mode = mode >= 2 ? 2 : 1;
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
                 OwnedBsr& C) {
  DBuf<int> counts;
  counts.resize(A.nbr > 0 ? A.nbr : 1);
  C.rp.resize(A.nbr + 1);
  SpgemmWork w;
  spgemm_counts(s, A, B, counts.p, w);
  const int64_t nnz = exclusive_scan(s, counts.p, C.rp.p, A.nbr);
  C.ci.resize(nnz > 0 ? nnz : 1);
  spgemm_fill(s, A, B, C.rp.p, C.ci.p, w);
  C.m.nbr = A.nbr; C.m.nbc = B.nbc; C.m.br = A.br; C.m.bc = B.bc; C.m.nnzb = nnz;
  C.m.rp = C.rp.p; C.m.ci = C.ci.p;
  C.V.resize(std::max<int64_t>(1, nnz * A.br * B.bc));
  spgemm_numeric(s, A, VA, B, VB, C.m, C.V.p);
  CK(cudaStreamSynchronize(s));
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

void alloc_work(Level& Lv) {
  Lv.b64.resize(Lv.n); Lv.x64.resize(Lv.n); Lv.r64.resize(Lv.n); Lv.y64.resize(Lv.n);
  Lv.b32.resize(Lv.n); Lv.x32.resize(Lv.n); Lv.r32.resize(Lv.n); Lv.y32.resize(Lv.n);
}

void amg_extend(tomg_problem* P, int start) {
  cudaStream_t s = st(P);
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
    CK(cudaStreamSynchronize(s));
  }
  int cur = start;
  while (P->L[cur]->n >= o.max_coarse_dofs && (int)P->L.size() < o.max_levels) {
    Level& A = *P->L[cur];
    const Bsr Ab = A.bsr();
    const int nn = (int)A.nn, b = A.b;
    // strength of connection (Eq. 10)
    DBuf<int> scnt, srp, sci;
    scnt.resize(nn);
    srp.resize(nn + 1);
    amg_strength_counts(s, Ab, A.V64.p, o.soc_beta, scnt.p);
    const int64_t nS = exclusive_scan(s, scnt.p, srp.p, nn);
    sci.resize(nS > 0 ? nS : 1);
    amg_strength_fill(s, Ab, A.V64.p, o.soc_beta, srp.p, sci.p);
    // aggregation
    DBuf<int> state, root_scan, agg;
    DBuf<uint64_t> vv, m1;
    state.resize(nn); root_scan.resize(nn + 1); agg.resize(nn); vv.resize(nn); m1.resize(nn);
    amg_mis2(s, nn, srp.p, sci.p, cur, state.p, vv.p, m1.p, P->flag_host, P->flag_dev.p);
    const int n_agg = amg_aggregate(s, nn, srp.p, sci.p, cur, state.p, agg.p, root_scan.p);
    if (n_agg == 0 || (int64_t)n_agg * k >= A.n) break;
    // tentative prolongator
    DBuf<int> Trp, Tci;
    DBuf<double> TV, Bc;
    Trp.resize(nn + 1); Tci.resize(nn); TV.resize((int64_t)nn * b * k); Bc.resize((int64_t)n_agg * k * k);
    amg_tentative(s, nn, b, k, n_agg, agg.p, B.p, Trp.p, Tci.p, TV.p, Bc.p);
    int nT = 0;
    CK(cudaMemcpy(&nT, Trp.p + nn, sizeof(int), cudaMemcpyDeviceToHost));
    Bsr Tm;
    Tm.nbr = nn; Tm.nbc = n_agg; Tm.br = b; Tm.bc = k; Tm.nnzb = nT; Tm.rp = Trp.p; Tm.ci = Tci.p;
    // prolongator smoothing weight from rho(D^-1 A)
    DBuf<double> pv, pw, parts;
    pv.resize(A.n); pw.resize(A.n); parts.resize(std::max(ceil_div(nn, 256), 256));
    const double rho = amg_spectral_radius(s, Ab, A.V64.p, A.D64.p, cur, 20, pv.p, pw.p, parts.p);
    const double omegaP = 4.0 / (3.0 * rho);
    // P = T - omega D^-1 A T
    OwnedBsr AT;
    spgemm_full(s, Ab, A.V64.p, Tm, TV.p, AT);
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
      exclusive_scan(s, cnt.p, A.Rrp.p, n_agg);
      A.Rci.resize(std::max<int64_t>(1, A.Pnnzb));
      A.Rv64.resize(std::max<int64_t>(1, A.Pnnzb * b * k));
      bsr_transpose_fill(s, Pm, A.Pv64.p, A.Rrp.p, A.Rci.p, A.Rv64.p, cursor.p);
    }
    // A_c = R (A P)  (Eq. 9)
    OwnedBsr AP, Ac;
    spgemm_full(s, Ab, A.V64.p, Pm, A.Pv64.p, AP);
    spgemm_full(s, A.Rmat(n_agg), A.Rv64.p, AP.m, AP.V.p, Ac);
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
    CK(cudaStreamSynchronize(s));
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

void problem_init(tomg_problem* P) {
  cudaStream_t s = P->ctx->stream;
  element_stiffness_host(P->dim, P->nu, P->Ke_host);
  const size_t nk = P->Ke_host.size();
  P->Ke64.resize(nk);
  P->Ke32.resize(nk);
  std::vector<float> k32(P->Ke_host.begin(), P->Ke_host.end());
  CK(cudaMemcpyAsync(P->Ke64.p, P->Ke_host.data(), nk * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P->Ke32.p, k32.data(), nk * 4, cudaMemcpyHostToDevice, s));
  P->mask.resize(P->nn);
  P->mask.zero(s);
  P->rho.resize(P->nel);
  P->E64.resize(P->nel);
  P->E32.resize(P->nel);
  for (auto* v : {&P->f, &P->bvec, &P->x, &P->r, &P->p, &P->q, &P->z, &P->t}) v->resize(P->n);
  const Ebe op{P->dim, P->nx, P->ny, P->nz, nullptr, nullptr, nullptr};
  const int np = std::max(ebe_blocks(op), red_blocks(P->n));
  P->partA.resize(np);
  P->partB.resize(np);
  P->partE.resize(np);
  P->sc.resize(1);
  P->sc.zero(s);
  P->flag_dev.resize(1);
  CK(cudaMallocHost((void**)&P->sc_host, sizeof(Scalars)));
  CK(cudaMallocHost((void**)&P->flag_host, sizeof(int)));
  CK(cudaEventCreate(&P->ev0));
  CK(cudaEventCreate(&P->ev1));
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
  CK(cudaMemcpyAsync(P->mask.p, m.data(), m.size(), cudaMemcpyHostToDevice, P->ctx->stream));
  CK(cudaStreamSynchronize(P->ctx->stream));
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
  if (opt.pc < 0 || opt.pc > 3 || opt.prec < 0 || opt.prec > 1)
    TOMG_THROW(TOMG_E_INVALID, "unknown preconditioner %d or precision %d", opt.pc, opt.prec);
  if (!(opt.rtol > 0.0) || opt.max_iter < 1 || opt.max_iter > 1000000 || !(opt.omega > 0.0) ||
      !(opt.omega < 2.0) || opt.n_pre < 1 || opt.n_pre > 8 || opt.n_post < 1 || opt.n_post > 8 ||
      opt.max_coarse_dofs < 1 || opt.max_levels < 1 || opt.max_levels > 64 || opt.smoother != 0)
    TOMG_THROW(TOMG_E_INVALID, "invalid options");
  destroy_graph(P);
  P->setup_valid = false;
  P->opt = opt;
  CK(cudaEventRecord(P->ev0, s));
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
    P->L.push_back(std::move(L0));
  }
  if (!P->jacobi_only) {
    int n_geo = 1;
    if (opt.pc == TOMG_PC_GMG)
      n_geo = opt.n_levels > 0 ? opt.n_levels
                               : levels_for_cap(P->dim, P->nx, P->ny, P->nz, opt.max_coarse_dofs, opt.max_levels);
    else if (opt.pc == TOMG_PC_HYBRID)
      n_geo = std::max(1, opt.n_geo_levels);
    n_geo = std::min(n_geo, opt.max_levels);
    // assembled level-0 stencil (FP64) for the Galerkin products / AMG / dense coarse solve
    Level& L0 = *P->L[0];
    L0.S64.resize((int64_t)stencil_q(P->dim) * P->nn);
    ebe_assemble_stencil(s, V<double>::ebe(P), L0.S64.p);
    for (int l = 1; l < n_geo; l++) {
      Level& F = *P->L[l - 1];
      auto C = std::make_unique<Level>();
      C->kind = KIND_STENCIL;
      C->b = P->dim;
      C->g = coarse_geo(F.g);
      C->nn = C->g.nodes();
      C->n = C->nn * P->dim;
      C->geometric = true;
      C->S64.resize((int64_t)stencil_q(P->dim) * C->nn);
      stencil_rap(s, F.g, C->g, F.S64.p, C->S64.p);
      C->S32.resize(C->S64.n);
      cast_f64_f32(s, C->S64.p, C->S32.p, C->S64.n);
      C->D64.resize(C->nn * P->dim * P->dim);
      C->D32.resize(C->nn * P->dim * P->dim);
      stencil_block_diag_inv(s, C->g, C->S64.p, C->D64.p, C->D32.p);
      F.geo_next = true;
      P->L.push_back(std::move(C));
    }
    if (opt.pc == TOMG_PC_AMG || opt.pc == TOMG_PC_HYBRID) amg_extend(P, (int)P->L.size() - 1);
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
    // setup-only storage of the fine level
    L0.S64.release();
    L0.rp.release(); L0.ci.release(); L0.V64.release();
    for (auto& lv : P->L)
      if (lv->kind == KIND_STENCIL) { lv->rp.release(); lv->ci.release(); lv->V64.release(); }
  }
  for (auto& lv : P->L) alloc_work(*lv);
  CK(cudaEventRecord(P->ev1, s));
  CK(cudaEventSynchronize(P->ev1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, P->ev0, P->ev1));
  P->setup_ms = ms;
  P->setup_valid = true;
}

// ----------------------------------------------------------------------------------------
namespace {

void init_solve(tomg_problem* P, const double* u0, bool u_on_device, int max_iter) {
  cudaStream_t s = st(P);
  const int64_t n = P->n;
  const Ebe op = V<double>::ebe(P);
  mask_vec(s, P->f.p, P->bvec.p, P->mask.p, P->dim, P->nn);
  if (u0) {
    CK(cudaMemcpyAsync(P->t.p, u0, n * 8, u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    mask_vec(s, P->t.p, P->x.p, P->mask.p, P->dim, P->nn);
  }
  ebe_op<double>(s, MODE_RESID, op, P->x.p, P->r.p, P->bvec.p, nullptr, 0.0, nullptr, nullptr);
  dot_partials(s, P->r.p, P->r.p, n, P->partA.p, nullptr);
  dot_partials(s, P->bvec.p, P->bvec.p, n, P->partB.p, nullptr);
  Scalars h;
  memset(&h, 0, sizeof(h));
  h.rtol2 = P->opt.rtol * P->opt.rtol;
  h.max_iter = max_iter;
  h.flexible = P->opt.prec == TOMG_PREC_FP64 ? 0 : 1;
  *P->sc_host = h;
  CK(cudaMemcpyAsync(P->sc.p, P->sc_host, sizeof(Scalars), cudaMemcpyHostToDevice, s));
  finish(s, FIN_INIT, P->partA.p, red_blocks(n), P->partB.p, red_blocks(n), P->sc.p);
  apply_M_and_dots(P, nullptr, &P->sc.p->done);
  finish(s, FIN_RZ0, P->partA.p, red_blocks(n), nullptr, 0, P->sc.p);
  copy_f64(s, P->z.p, P->p.p, n, &P->sc.p->done);
}

void read_scalars(tomg_problem* P) {
  CK(cudaMemcpyAsync(P->sc_host, P->sc.p, sizeof(Scalars), cudaMemcpyDeviceToHost, st(P)));
  CK(cudaStreamSynchronize(st(P)));
}

void run_iterations(tomg_problem* P) {
  cudaStream_t s = st(P);
  if (P->graph_mode == 2) {
    CK(cudaGraphLaunch(P->gexec, s));
    read_scalars(P);
    g_launches += P->kernels_per_iter * std::max(1, P->sc_host->it);
    return;
  }
  const int every = std::max(1, P->opt.check_every);
  while (true) {
    for (int k = 0; k < every; k++) {
      if (P->graph_mode == 1) {
        CK(cudaGraphLaunch(P->gexec, s));
        g_launches += P->kernels_per_iter;
      } else {
        iteration_body(P);
      }
    }
    read_scalars(P);
    if (P->sc_host->done) return;
  }
}

double host_sum(tomg_problem* P, const double* partials, int np) {
  std::vector<double> h(np);
  CK(cudaMemcpyAsync(h.data(), partials, np * 8, cudaMemcpyDeviceToHost, st(P)));
  CK(cudaStreamSynchronize(st(P)));
  double t = 0.0;
  for (double v : h) t += v;
  return t;
}

}  // namespace

tomg_status solve(tomg_problem* P, int nrhs, const double* f, double* u, int on_device,
                  tomg_result* res) {
  if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "tomg_solve: call tomg_setup after changing density or fixed DOFs");
  if (nrhs < 0 || (nrhs > 0 && (!f || !u || !res))) TOMG_THROW(TOMG_E_INVALID, "bad solve arguments");
  cudaStream_t s = st(P);
  const int64_t n = P->n;
  if (!P->gexec && P->opt.use_graph > 0) build_graph(P);
  tomg_status worst = TOMG_OK;
  const cudaMemcpyKind h2d = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind d2h = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const Ebe op = V<double>::ebe(P);
  for (int j = 0; j < nrhs; j++) {
    CK(cudaEventRecord(P->ev0, s));
    CK(cudaMemcpyAsync(P->f.p, f + (int64_t)j * n, n * 8, h2d, s));
    int total_it = 0;
    int status = TOMG_OK;
    double rr_true = 0.0, bb = 0.0;
    const double* u0 = u + (int64_t)j * n;
    for (int attempt = 0; attempt < 4; attempt++) {
      init_solve(P, u0, on_device != 0, P->opt.max_iter - total_it);
      u0 = nullptr;  // restarts keep x
      run_iterations(P);
      read_scalars(P);
      total_it += P->sc_host->it;
      status = P->sc_host->status;
      bb = P->sc_host->bb;
      // true residual of the final iterate
      ebe_op<double>(s, MODE_RESID, op, P->x.p, P->t.p, P->bvec.p, nullptr, 0.0, nullptr, nullptr);
      dot_partials(s, P->t.p, P->t.p, n, P->partE.p, nullptr);
      rr_true = host_sum(P, P->partE.p, red_blocks(n));
      if (status != TOMG_OK || bb == 0.0) break;
      if (rr_true <= P->opt.rtol * P->opt.rtol * bb) break;
      if (total_it >= P->opt.max_iter) { status = TOMG_NOT_CONVERGED; break; }
      // recursive residual converged but the true one did not: restart from x
    }
    if (status == TOMG_OK && bb > 0.0 && !(rr_true <= P->opt.rtol * P->opt.rtol * bb)) status = TOMG_NOT_CONVERGED;
    if (status == TOMG_E_BREAKDOWN) {
      static const char* what[] = {"?", "NaN residual", "z.r <= 0 with a CG preconditioner",
                                   "p^T K p <= 0", "z.r or z.q not finite / z.r <= 0"};
      const int code = P->sc_host->pad;
      set_error("solver breakdown at iteration %d: %s (rhs %d)", total_it,
                what[(code >= 0 && code <= 4) ? code : 0], j);
    } else if (status == TOMG_NOT_CONVERGED) {
      set_error("not converged after %d iterations (rel residual %.3e, rhs %d)", total_it,
                bb > 0.0 ? std::sqrt(rr_true / bb) : 0.0, j);
    }
    dot_partials(s, P->f.p, P->x.p, n, P->partE.p, nullptr);
    const double comp = host_sum(P, P->partE.p, red_blocks(n));
    CK(cudaMemcpyAsync(u + (int64_t)j * n, P->x.p, n * 8, d2h, s));
    CK(cudaEventRecord(P->ev1, s));
    CK(cudaEventSynchronize(P->ev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, P->ev0, P->ev1));
    res[j].iterations = total_it;
    res[j].rel_residual = bb > 0.0 ? std::sqrt(rr_true / bb) : 0.0;
    res[j].compliance = comp;
    res[j].setup_ms = P->setup_ms;
    res[j].solve_ms = ms;
    res[j].status = status;
    if (status < 0 || (worst >= 0 && status > worst)) worst = (tomg_status)status;
  }
  return worst;
}

// ----------------------------------------------------------------------------------------
void level_apply(tomg_problem* P, int level, int prec, const double* x, double* y) {
  if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "no valid setup");
  if (level < 0 || level >= (int)P->L.size()) TOMG_THROW(TOMG_E_INVALID, "bad level %d", level);
  Level& Lv = *P->L[level];
  cudaStream_t s = st(P);
  if (prec == TOMG_PREC_FP64) {
    CK(cudaMemcpyAsync(Lv.b64.p, x, Lv.n * 8, cudaMemcpyDeviceToDevice, s));
    level_op<double>(P, level, MODE_APPLY, Lv.b64.p, Lv.y64.p, nullptr, nullptr);
    CK(cudaMemcpyAsync(y, Lv.y64.p, Lv.n * 8, cudaMemcpyDeviceToDevice, s));
  } else {
    cast_f64_f32(s, x, Lv.b32.p, Lv.n);
    level_op<float>(P, level, MODE_APPLY, Lv.b32.p, Lv.y32.p, nullptr, nullptr);
    cast_f32_f64(s, Lv.y32.p, y, Lv.n);
  }
  CK(cudaStreamSynchronize(s));
}

void vcycle_apply(tomg_problem* P, const double* r, double* z) {
  if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "no valid setup");
  cudaStream_t s = st(P);
  CK(cudaMemcpyAsync(P->r.p, r, P->n * 8, cudaMemcpyDeviceToDevice, s));
  apply_M_and_dots(P, nullptr, nullptr);
  CK(cudaMemcpyAsync(z, P->z.p, P->n * 8, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
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

}  // namespace tomg

tomg_problem::~tomg_problem() {
  tomg::destroy_graph(this);
  if (sc_host) cudaFreeHost(sc_host);
  if (flag_host) cudaFreeHost(flag_host);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
}

namespace tomg {
double time_fine_operator(tomg_problem* P, int op, int prec, int reps, int cold_l2) {
  if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "no valid setup");
  if (op < 0 || op > 2 || reps < 1 || reps > 10000) TOMG_THROW(TOMG_E_INVALID, "bad timing request");
  cudaStream_t s = st(P);
  Level& L0 = *P->L[0];
  const int mode = op == 0 ? MODE_APPLY : (op == 1 ? MODE_RESID : MODE_JACOBI);
  DBuf<char> flush;
  if (cold_l2) flush.resize((size_t)256 << 20);
  std::vector<cudaEvent_t> ev(2 * reps);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  for (int k = 0; k < reps; k++) {
    if (cold_l2) CK(cudaMemsetAsync(flush.p, k & 0xff, flush.n, s));
    CK(cudaEventRecord(ev[2 * k], s));
    if (prec == TOMG_PREC_FP64) level_op<double>(P, 0, mode, L0.x64.p, L0.y64.p, L0.b64.p, nullptr);
    else level_op<float>(P, 0, mode, L0.x32.p, L0.y32.p, L0.b32.p, nullptr);
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
