// C ABI of the tomg library (declared in include/tomg.h): argument checks, error capture and
// host/device marshalling around the runtime in solver.cu.  No exception crosses the ABI.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <vector>

#include "solver.h"

namespace tomg {

std::atomic<int64_t> g_launches{0};
static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
const char* get_error() { return g_err; }

static thread_local bool g_pdl = false;
bool pdl_enabled() { return g_pdl; }
void set_pdl(bool on) { g_pdl = on; }

static thread_local int g_batch = 1;
int batch_rhs() { return g_batch; }
void set_batch_rhs(int r) { g_batch = r > 1 ? r : 1; }
void no_batch(const char* what) {
  if (g_batch > 1) TOMG_THROW(TOMG_E_INVALID, "%s has no block (several right-hand sides) form", what);
}

static thread_local cudaStream_t g_alloc_stream = nullptr;
cudaStream_t alloc_stream() { return g_alloc_stream; }
void set_alloc_stream(cudaStream_t s) { g_alloc_stream = s; }

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

namespace {

template <class F>
tomg_status guarded(F&& fn) {
  // a non-sticky error left behind by another library's runtime call in this thread would
  // otherwise surface at our first post-launch check; every call of ours is checked itself
  (void)cudaGetLastError();
  try {
    return fn();
  } catch (const Error& e) {
    return e.st;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return TOMG_E_OOM;
  } catch (...) {
    set_error("unexpected internal error");
    return TOMG_E_CUDA;
  }
}

// device view of a caller array: the pointer itself (device) or a staged copy (host)
// Caller arrays as kernel operands.  Device arrays are used in place when 16-byte aligned (the
// kernels load DOF pairs as 16-byte vectors); host arrays and unaligned device arrays go
// through a library buffer.
inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
struct DevArray {
  DBuf<double> buf;
  const double* p = nullptr;
  DevArray(const double* src, int64_t n, int on_device, cudaStream_t s) {
    if (on_device && aligned16(src)) { p = src; return; }
    buf.resize(n > 0 ? n : 1);
    if (n)
      CK(cudaMemcpyAsync(buf.p, src, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    p = buf.p;
  }
};
struct DevOut {
  DBuf<double> buf;
  double* p = nullptr;
  double* dst;
  int64_t n;
  int on_device;
  bool direct = false;
  cudaStream_t s;
  DevOut(double* d, int64_t count, int on_dev, cudaStream_t st) : dst(d), n(count), on_device(on_dev), s(st) {
    if (on_device && aligned16(d)) { p = d; direct = true; return; }
    buf.resize(n > 0 ? n : 1);
    p = buf.p;
  }
  void commit() {
    if (!direct && n)
      CK(cudaMemcpyAsync(dst, p, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
};

void set_device(const tomg_ctx* c) {
  CK(cudaSetDevice(c->device));
  set_alloc_stream(c->stream);
}
void set_device(const tomg_problem* P) {
  CK(cudaSetDevice(P->ctx->device));
  set_alloc_stream(P->stream);
}

}  // namespace
}  // namespace tomg

using namespace tomg;

extern "C" {

const char* tomg_last_error(void) { return get_error(); }

void tomg_options_default(tomg_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->pc = TOMG_PC_GMG;
  o->prec = TOMG_PREC_FP64;
  o->rtol = 1e-8;
  o->max_iter = 1000;
  o->n_levels = 0;
  o->max_coarse_dofs = 2000;
  o->n_geo_levels = 3;
  o->smoother = 0;
  o->cheb_degree = 2;
  o->cheb_lower = 0.1;
  o->cheb_upper = 1.1;
  o->adaptive_geo = 0;
  o->adaptive_iters = 200;
  o->adaptive_min_geo = 2;
  o->krylov = 0;
  o->gmres_restart = 30;
  o->gmres_steps = 2;
  o->omega = 0.5;
  o->n_pre = 1;
  o->n_post = 1;
  o->soc_beta = 0.003;
  o->check_every = 4;
  o->use_graph = 2;
  o->max_levels = 25;
  o->concurrency = 4;
  o->fp64_tc = 1;
  o->fuse_transfers = 0;
}

tomg_status tomg_ctx_create(tomg_ctx** out, int device, void* cuda_stream) {
  return guarded([&]() -> tomg_status {
    if (!out) TOMG_THROW(TOMG_E_INVALID, "null output handle");
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) TOMG_THROW(TOMG_E_INVALID, "device %d not present (%d devices)", device, ndev);
    CK(cudaSetDevice(device));
    auto* c = new tomg_ctx();
    c->device = device;
    if (cuda_stream) {
      c->stream = (cudaStream_t)cuda_stream;
    } else {
      cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) { delete c; CK(e); }
      c->own_stream = true;
    }
    c->launches0 = g_launches;
    // keep freed blocks of the stream-ordered pool cached for reuse by later setups
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    *out = c;
    return TOMG_OK;
  });
}

tomg_status tomg_ctx_destroy(tomg_ctx* c) {
  return guarded([&]() -> tomg_status {
    if (!c) return TOMG_OK;
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return TOMG_OK;
  });
}

tomg_status tomg_kernel_launches(const tomg_ctx* c, int64_t* count) {
  if (!c || !count) { set_error("null argument"); return TOMG_E_INVALID; }
  *count = g_launches - c->launches0;
  return TOMG_OK;
}

tomg_status tomg_problem_create(tomg_ctx* c, int dim, int nx, int ny, int nz, double E0,
                                double Emin, double penal, double nu, tomg_problem** out) {
  return guarded([&]() -> tomg_status {
    if (!c || !out) TOMG_THROW(TOMG_E_INVALID, "null argument");
    if (dim != 2 && dim != 3) TOMG_THROW(TOMG_E_INVALID, "dim must be 2 or 3");
    if (nx < 1 || ny < 1 || (dim == 3 && nz < 1)) TOMG_THROW(TOMG_E_INVALID, "grid sizes must be >= 1");
    if (!(E0 > 0.0) || !(Emin >= 0.0) || !(penal >= 0.0) || !(nu > -1.0) || !(nu < 0.5))
      TOMG_THROW(TOMG_E_INVALID, "invalid material constants");
    const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (dim == 3 ? nz + 1 : 1);
    if (nn * dim >= 0x7fffffffLL) TOMG_THROW(TOMG_E_INVALID, "grid too large");
    set_device(c);
    auto* P = new tomg_problem();
    P->ctx = c;
    P->dim = dim; P->nx = nx; P->ny = ny; P->nz = dim == 3 ? nz : 1;
    P->E0 = E0; P->Emin = Emin; P->penal = penal; P->nu = nu;
    P->nn = nn;
    P->n = nn * dim;
    P->nel = (int64_t)nx * ny * (dim == 3 ? nz : 1);
    try {
      problem_init(P);
    } catch (...) {
      delete P;
      throw;
    }
    *out = P;
    return TOMG_OK;
  });
}

tomg_status tomg_problem_destroy(tomg_problem* P) {
  return guarded([&]() -> tomg_status {
    if (!P) return TOMG_OK;
    set_device(P->ctx);
    cudaStreamSynchronize(P->ctx->stream);
    delete P;
    return TOMG_OK;
  });
}

tomg_status tomg_problem_sizes(const tomg_problem* P, int64_t* n, int64_t* nn, int64_t* nel) {
  if (!P) { set_error("null problem"); return TOMG_E_INVALID; }
  if (n) *n = P->n;
  if (nn) *nn = P->nn;
  if (nel) *nel = P->nel;
  return TOMG_OK;
}

tomg_status tomg_set_fixed_dofs(tomg_problem* P, const int64_t* dofs, int64_t count) {
  return guarded([&]() -> tomg_status {
    if (!P) TOMG_THROW(TOMG_E_INVALID, "null problem");
    set_device(P);
    StreamScope sc(P);
    set_fixed(P, dofs, count);
    return TOMG_OK;
  });
}

tomg_status tomg_set_density(tomg_problem* P, const double* rho, int on_device) {
  return guarded([&]() -> tomg_status {
    if (!P) TOMG_THROW(TOMG_E_INVALID, "null problem");
    set_device(P);
    StreamScope sc(P);
    set_density(P, rho, on_device);
    return TOMG_OK;
  });
}

tomg_status tomg_setup(tomg_problem* P, const tomg_options* opt) {
  return guarded([&]() -> tomg_status {
    if (!P) TOMG_THROW(TOMG_E_INVALID, "null problem");
    set_device(P);
    StreamScope sc(P);
    tomg_options o;
    if (opt) o = *opt;
    else tomg_options_default(&o);
    setup(P, o);
    return TOMG_OK;
  });
}

tomg_status tomg_solve(tomg_problem* P, int nrhs, const double* f, double* u, int on_device,
                       tomg_result* results) {
  return guarded([&]() -> tomg_status {
    if (!P) TOMG_THROW(TOMG_E_INVALID, "null problem");
    set_device(P);
    StreamScope sc(P);
    return solve(P, nrhs, f, u, on_device, results);
  });
}

tomg_status tomg_adaptive_geo_levels(const tomg_problem* P, int* n) {
  if (!P || !n) { set_error("null argument"); return TOMG_E_INVALID; }
  *n = P->adapt_geo;
  return TOMG_OK;
}

tomg_status tomg_num_levels(const tomg_problem* P, int* n) {
  if (!P || !n) { set_error("null argument"); return TOMG_E_INVALID; }
  if (!P->setup_valid) { set_error("no valid setup"); return TOMG_E_INVALID; }
  *n = (int)P->L.size();
  return TOMG_OK;
}

tomg_status tomg_level_info_get(const tomg_problem* P, int level, tomg_level_info* info) {
  if (!P || !info) { set_error("null argument"); return TOMG_E_INVALID; }
  if (!P->setup_valid || level < 0 || level >= (int)P->L.size()) { set_error("bad level"); return TOMG_E_INVALID; }
  const Level& L = *P->L[level];
  info->kind = L.kind;
  info->block = L.b;
  info->n_nodes = L.nn;
  info->n_dofs = L.n;
  info->nnzb = L.kind == KIND_BSR ? L.nnzb : L.nn * (P->dim == 3 ? 27 : 9);
  info->nx = L.geometric ? L.g.nx : 0;
  info->ny = L.geometric ? L.g.ny : 0;
  info->nz = L.geometric ? L.g.nz : 0;
  info->geometric = L.geo_next ? 1 : 0;
  return TOMG_OK;
}

tomg_status tomg_level_export(tomg_problem* P, int level, int64_t* nnzb, int64_t* rp, int64_t* ci,
                              double* val) {
  return guarded([&]() -> tomg_status {
    if (!P || !nnzb) TOMG_THROW(TOMG_E_INVALID, "null argument");
    set_device(P);
    StreamScope sc(P);
    level_export(P, level, nnzb, rp, ci, val);
    return TOMG_OK;
  });
}

tomg_status tomg_prolongation_export(tomg_problem* P, int level, int64_t* nnzb, int64_t* rp,
                                     int64_t* ci, double* val) {
  return guarded([&]() -> tomg_status {
    if (!P || !nnzb) TOMG_THROW(TOMG_E_INVALID, "null argument");
    set_device(P);
    StreamScope sc(P);
    prolong_export(P, level, nnzb, rp, ci, val);
    return TOMG_OK;
  });
}

tomg_status tomg_aggregates_export(tomg_problem* P, int level, int64_t* agg) {
  return guarded([&]() -> tomg_status {
    if (!P || !agg) TOMG_THROW(TOMG_E_INVALID, "null argument");
    if (!P->setup_valid || level < 0 || level + 1 >= (int)P->L.size() || P->L[level]->geo_next)
      TOMG_THROW(TOMG_E_INVALID, "level %d has no aggregation", level);
    set_device(P);
    StreamScope sc(P);
    const Level& L = *P->L[level];
    std::vector<int> h(L.nn);
    CK(cudaMemcpyAsync(h.data(), L.agg.p, L.nn * sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    for (int64_t i = 0; i < L.nn; i++) agg[i] = h[i];
    return TOMG_OK;
  });
}

tomg_status tomg_block_diag_inv_export(tomg_problem* P, int level, double* dinv) {
  return guarded([&]() -> tomg_status {
    if (!P || !dinv) TOMG_THROW(TOMG_E_INVALID, "null argument");
    if (!P->setup_valid || level < 0 || level + 1 >= (int)P->L.size() || !P->L[level]->D64.p)
      TOMG_THROW(TOMG_E_INVALID, "level %d has no smoother blocks", level);
    set_device(P);
    StreamScope sc(P);
    const Level& L = *P->L[level];
    CK(cudaMemcpyAsync(dinv, L.D64.p, L.D64.bytes(), cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    return TOMG_OK;
  });
}

tomg_status tomg_level_apply(tomg_problem* P, int level, int prec, const double* x, double* y,
                             int on_device) {
  return guarded([&]() -> tomg_status {
    if (!P || !x || !y) TOMG_THROW(TOMG_E_INVALID, "null argument");
    if (!P->setup_valid || level < 0 || level >= (int)P->L.size()) TOMG_THROW(TOMG_E_INVALID, "bad level");
    set_device(P);
    StreamScope sc(P);
    const int64_t n = P->L[level]->n;
    DevArray xin(x, n, on_device, P->stream);
    DevOut yout(y, n, on_device, P->stream);
    level_apply(P, level, prec, xin.p, yout.p);
    yout.commit();
    return TOMG_OK;
  });
}

tomg_status tomg_outer_apply(tomg_problem* P, const double* x, double* y, int on_device) {
  return guarded([&]() -> tomg_status {
    if (!P || !x || !y) TOMG_THROW(TOMG_E_INVALID, "null argument");
    if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "no valid setup");
    set_device(P);
    StreamScope sc(P);
    DevArray xin(x, P->n, on_device, P->stream);
    DevOut yout(y, P->n, on_device, P->stream);
    outer_operator_apply(P, xin.p, yout.p);
    yout.commit();
    return TOMG_OK;
  });
}

tomg_status tomg_vcycle(tomg_problem* P, const double* r, double* z, int on_device) {
  return guarded([&]() -> tomg_status {
    if (!P || !r || !z) TOMG_THROW(TOMG_E_INVALID, "null argument");
    set_device(P);
    StreamScope sc(P);
    DevArray rin(r, P->n, on_device, P->stream);
    DevOut zout(z, P->n, on_device, P->stream);
    vcycle_apply(P, rin.p, zout.p);
    zout.commit();
    return TOMG_OK;
  });
}

tomg_status tomg_coarse_solve(tomg_problem* P, const double* b, double* x, int on_device) {
  return guarded([&]() -> tomg_status {
    if (!P || !b || !x) TOMG_THROW(TOMG_E_INVALID, "null argument");
    if (!P->setup_valid) TOMG_THROW(TOMG_E_INVALID, "no valid setup");
    set_device(P);
    StreamScope sc(P);
    DevArray bin(b, P->nc, on_device, P->stream);
    DevOut xout(x, P->nc, on_device, P->stream);
    coarse_apply(P, bin.p, xout.p);
    xout.commit();
    return TOMG_OK;
  });
}

tomg_status tomg_moduli(tomg_problem* P, double* E, int on_device) {
  return guarded([&]() -> tomg_status {
    if (!P || !E) TOMG_THROW(TOMG_E_INVALID, "null argument");
    if (!P->have_density) TOMG_THROW(TOMG_E_INVALID, "no density set");
    set_device(P);
    StreamScope sc(P);
    CK(cudaMemcpyAsync(E, P->E64.p, P->nel * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    return TOMG_OK;
  });
}

tomg_status tomg_density_filter(tomg_problem* P, double radius, int transpose, const double* in,
                                double* out, int on_device) {
  return guarded([&]() -> tomg_status {
    if (!P || !in || !out || in == out) TOMG_THROW(TOMG_E_INVALID, "null or aliased argument");
    set_device(P);
    StreamScope sc(P);
    cudaStream_t s = P->stream;
    const size_t bytes = (size_t)P->nel * 8;
    tomg::DBuf<double> W, din, dout;
    W.resize(P->nel);
    const double* a = in;
    double* o = out;
    if (!on_device) {
      din.resize(P->nel);
      dout.resize(P->nel);
      CK(cudaMemcpyAsync(din.p, in, bytes, cudaMemcpyHostToDevice, s));
      a = din.p;
      o = dout.p;
    }
    tomg::density_filter(s, P->dim, P->nx, P->ny, P->nz, radius, transpose, a, o, W.p);
    if (!on_device) CK(cudaMemcpyAsync(out, o, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return TOMG_OK;
  });
}

tomg_status tomg_compliance_sensitivity(tomg_problem* P, const double* u, double* out,
                                        int on_device) {
  return guarded([&]() -> tomg_status {
    if (!P || !u || !out) TOMG_THROW(TOMG_E_INVALID, "null argument");
    if (!P->have_density) TOMG_THROW(TOMG_E_INVALID, "no density set");
    set_device(P);
    StreamScope sc(P);
    cudaStream_t s = P->stream;
    tomg::DBuf<double> du, dout;
    const double* uu = u;
    double* o = out;
    if (!on_device) {
      du.resize(P->n);
      dout.resize(P->nel);
      CK(cudaMemcpyAsync(du.p, u, (size_t)P->n * 8, cudaMemcpyHostToDevice, s));
      uu = du.p;
      o = dout.p;
    }
    tomg::compliance_sensitivity(s, P->dim, P->nx, P->ny, P->nz, P->Ke64.p, P->rho.p, uu, P->E0,
                                 P->Emin, P->penal, o);
    if (!on_device) CK(cudaMemcpyAsync(out, o, (size_t)P->nel * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return TOMG_OK;
  });
}

tomg_status tomg_stress_stiffness_apply(tomg_problem* P, const double* u, const double* x,
                                        double* y, int on_device) {
  return guarded([&]() -> tomg_status {
    if (!P || !u || !x || !y) TOMG_THROW(TOMG_E_INVALID, "null argument");
    if (!P->have_density) TOMG_THROW(TOMG_E_INVALID, "no density set");
    set_device(P);
    StreamScope sc(P);
    cudaStream_t s = P->stream;
    const size_t bytes = (size_t)P->n * 8;
    if (on_device) {
      tomg::stress_stiffness_op(P, u, x, y);
      return TOMG_OK;
    }
    tomg::DBuf<double> du, dx, dy;
    du.resize(P->n); dx.resize(P->n); dy.resize(P->n);
    CK(cudaMemcpyAsync(du.p, u, bytes, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dx.p, x, bytes, cudaMemcpyHostToDevice, s));
    tomg::stress_stiffness_op(P, du.p, dx.p, dy.p);
    CK(cudaMemcpyAsync(y, dy.p, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return TOMG_OK;
  });
}

tomg_status tomg_buckling(tomg_problem* P, const double* u, int n_eig, int j_min, int j_max,
                          double tol, int max_iter, double* lambdas, double* modes, int on_device,
                          int* iterations) {
  return guarded([&]() -> tomg_status {
    if (!P || !u || !lambdas) TOMG_THROW(TOMG_E_INVALID, "null argument");
    set_device(P);
    StreamScope sc(P);
    return tomg::buckling(P, u, n_eig, j_min, j_max, tol, max_iter, lambdas, modes, on_device,
                          iterations);
  });
}

tomg_status tomg_buckling_adjoint_rhs(tomg_problem* P, int n_modes, const double* modes,
                                      double* g, int on_device) {
  return guarded([&]() -> tomg_status {
    if (!P || !modes || !g) TOMG_THROW(TOMG_E_INVALID, "null argument");
    if (!P->have_density) TOMG_THROW(TOMG_E_INVALID, "no density set");
    if (n_modes < 1 || n_modes > 16) TOMG_THROW(TOMG_E_INVALID, "1 <= n_modes <= 16");
    set_device(P);
    StreamScope sc(P);
    cudaStream_t s = P->stream;
    const size_t bytes = (size_t)P->n * n_modes * 8;
    tomg::DBuf<double> dphi, dg, sw;
    const double* ph = modes;
    double* gg = g;
    if (!on_device) {
      dphi.resize((int64_t)P->n * n_modes);
      dg.resize((int64_t)P->n * n_modes);
      CK(cudaMemcpyAsync(dphi.p, modes, bytes, cudaMemcpyHostToDevice, s));
      ph = dphi.p;
      gg = dg.p;
    }
    sw.resize(P->nel * n_modes * tomg::stress_components(P->dim));
    tomg::buckling_adjoint_rhs(s, P->dim, P->nx, P->ny, P->nz, P->nu, P->E0, P->penal, P->rho.p,
                               P->mask.p, n_modes, ph, P->n, sw.p, gg, P->n);
    if (!on_device) CK(cudaMemcpyAsync(g, gg, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return TOMG_OK;
  });
}

tomg_status tomg_buckling_sensitivity(tomg_problem* P, const double* u, int n_modes,
                                      const double* lambdas, const double* modes,
                                      const double* adjoints, double pnorm, double* dlambda,
                                      double* dF, double* F, int on_device) {
  return guarded([&]() -> tomg_status {
    if (!P || !u || !lambdas || !modes || !adjoints) TOMG_THROW(TOMG_E_INVALID, "null argument");
    if (!P->have_density) TOMG_THROW(TOMG_E_INVALID, "no density set");
    if (n_modes < 1 || n_modes > 16) TOMG_THROW(TOMG_E_INVALID, "1 <= n_modes <= 16");
    if (!(pnorm >= 1.0)) TOMG_THROW(TOMG_E_INVALID, "pnorm %g < 1", pnorm);
    double sum = 0.0;
    for (int k = 0; k < n_modes; k++) sum += std::pow(lambdas[k], pnorm);
    const double Fv = std::pow(sum, 1.0 / pnorm);
    if (!(sum > 0.0) || !std::isfinite(Fv))
      TOMG_THROW(TOMG_E_INVALID, "p-norm of the eigenvalues is not positive and finite");
    std::vector<double> coef(n_modes);
    for (int k = 0; k < n_modes; k++)
      coef[k] = std::pow(Fv, 1.0 - pnorm) * std::pow(lambdas[k], pnorm - 1.0);
    if (F) *F = Fv;
    if (!dlambda && !dF) return TOMG_OK;
    set_device(P);
    StreamScope sc(P);
    cudaStream_t s = P->stream;
    const int64_t n = P->n, nel = P->nel;
    tomg::DBuf<double> du, dphi, dv, ddl, ddf;
    const double *uu = u, *ph = modes, *vv = adjoints;
    double *dl = dlambda, *df = dF;
    if (!on_device) {
      du.resize(n); dphi.resize(n * n_modes); dv.resize(n * n_modes);
      CK(cudaMemcpyAsync(du.p, u, (size_t)n * 8, cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(dphi.p, modes, (size_t)n * n_modes * 8, cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(dv.p, adjoints, (size_t)n * n_modes * 8, cudaMemcpyHostToDevice, s));
      uu = du.p; ph = dphi.p; vv = dv.p;
      if (dlambda) { ddl.resize(nel * n_modes); dl = ddl.p; }
      if (dF) { ddf.resize(nel); df = ddf.p; }
    }
    tomg::buckling_sensitivity(s, P->dim, P->nx, P->ny, P->nz, P->nu, P->E0, P->Emin, P->penal,
                               P->Ke64.p, P->rho.p, P->mask.p, uu, n_modes, lambdas, coef.data(),
                               ph, vv, n, dl, df);
    if (!on_device) {
      if (dlambda)
        CK(cudaMemcpyAsync(dlambda, dl, (size_t)nel * n_modes * 8, cudaMemcpyDeviceToHost, s));
      if (dF) CK(cudaMemcpyAsync(dF, df, (size_t)nel * 8, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return TOMG_OK;
  });
}

tomg_status tomg_element_stiffness(const tomg_problem* P, double* Ke) {
  if (!P || !Ke) { set_error("null argument"); return TOMG_E_INVALID; }
  memcpy(Ke, P->Ke_host.data(), P->Ke_host.size() * sizeof(double));
  return TOMG_OK;
}

}  // extern "C"

namespace tomg {
double time_fine_operator(tomg_problem* P, int op, int prec, int reps, int cold_l2);
}

extern "C" tomg_status tomg_time_fine_operator(tomg_problem* P, int op, int prec, int reps,
                                               int cold_l2, double* ms) {
  return tomg::guarded([&]() -> tomg_status {
    if (!P || !ms) TOMG_THROW(TOMG_E_INVALID, "null argument");
    tomg::set_device(P);
    tomg::StreamScope sc(P);
    *ms = tomg::time_fine_operator(P, op, prec, reps, cold_l2);
    return TOMG_OK;
  });
}

extern "C" tomg_status tomg_debug_tc_wait_limit(int polls) {
  tomg::ebe3d_tc_set_wait_limit(polls);
  return TOMG_OK;
}

extern "C" tomg_status tomg_debug_grid_wait_limit(int polls) {
  tomg::set_grid_wait_limit(polls);
  return TOMG_OK;
}
