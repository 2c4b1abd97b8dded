// Host runtime of the tomg library: problem state, hierarchy setup, V-cycle, outer Krylov
// loop, its CUDA-graph capture, and concurrent solve slots.
//
// Streams: every problem owns a stream; API calls order themselves after the context stream
// on entry and make the context stream wait for them on exit.  A solve of several right-hand
// sides spreads them over solve slots (each with its own stream, vectors and captured graph)
// that share the read-only hierarchy, so their kernels overlap on the device.
#pragma once

#include <atomic>
#include <map>
#include <memory>

#include "ops.h"

struct tomg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t launches0 = 0;
};

namespace tomg {

enum LevelKind { KIND_EBE = 0, KIND_STENCIL = 1, KIND_BSR = 2 };

struct Level {
  int kind = KIND_EBE;
  int b = 2;          // DOFs per node
  int64_t nn = 0;     // nodes
  int64_t n = 0;      // DOFs
  Geo g{2, 0, 0, 1};  // geometric levels
  bool geometric = false;
  bool geo_next = false;  // transfer to the next level is geometric
  // structured stencil (geometric levels >= 1; level 0 during setup)
  DBuf<double> S64;
  DBuf<float> S32;  // the upper half of S64 (centre and later offsets), for the FP32 V-cycle
  // block CSR (AMG levels; the level an AMG part starts from, during setup)
  DBuf<int> rp, ci;
  DBuf<double> V64;
  DBuf<float> V32;
  int64_t nnzb = 0;
  // point-block diagonal inverse
  DBuf<double> D64;
  DBuf<float> D32;
  // algebraic transfer to the next level: P (n x nc) and R = P^T
  int bc = 0;
  DBuf<int> Prp, Pci, Rrp, Rci;
  DBuf<double> Pv64, Rv64;
  DBuf<float> Pv32, Rv32;
  int64_t Pnnzb = 0;
  DBuf<int> agg;
  // Chebyshev smoother: lambda_max(D^-1 A) estimate and the step coefficients
  double lam = 0.0;
  double cheb_c1[8] = {0}, cheb_c2[8] = {0};

  Bsr bsr() const {
    Bsr A;
    A.nbr = A.nbc = (int)nn;
    A.br = A.bc = b;
    A.nnzb = nnzb;
    A.rp = rp.p;
    A.ci = ci.p;
    return A;
  }
  Bsr Pmat(int64_t nn_next) const {
    Bsr A;
    A.nbr = (int)nn; A.nbc = (int)nn_next; A.br = b; A.bc = bc; A.nnzb = Pnnzb;
    A.rp = Prp.p; A.ci = Pci.p;
    return A;
  }
  Bsr Rmat(int64_t nn_next) const {
    Bsr A;
    A.nbr = (int)nn_next; A.nbc = (int)nn; A.br = bc; A.bc = b; A.nnzb = Pnnzb;
    A.rp = Rrp.p; A.ci = Rci.p;
    return A;
  }
};

// V-cycle work vectors of one level for one solve slot
struct LevelWork {
  DBuf<double> b64, x64, r64, y64;
  DBuf<float> b32, x32, r32, y32;
  // GMRES smoother: Arnoldi basis (m + 1 vectors), preconditioned basis (m), scratch, state
  DBuf<double> gV64, gZ64, gparts;
  DBuf<float> gV32, gZ32;
  DBuf<GmState> gst;
};

// One solve slot: stream, outer Krylov vectors, V-cycle work, scalars and captured iteration
struct Work {
  cudaStream_t stream = nullptr;
  DBuf<double> f, bvec, x, r, p, q, z, t;
  DBuf<double> partA, partB, partE, partC;
  DBuf<Scalars> sc;
  Scalars* sc_host = nullptr;  // pinned
  double* partE_host = nullptr;  // pinned, true-residual partials
  double* partC_host = nullptr;  // pinned, compliance partials
  int np = 0;
  std::vector<LevelWork> lw;
  int64_t built_for = -1;  // setup generation the vectors / graph belong to
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_mode = 0;  // 0 none, 1 one-iteration graph, 2 conditional while loop
  cudaGraphConditionalHandle cond = 0;  // while condition, set while capturing mode 2
  int has_cond = 0;
  int64_t kernels_per_iter = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evdone = nullptr, evsync = nullptr;
  int block = 0;  // right-hand sides of a block solve work (vectors and scalars x block); 0: slot
  // per right-hand side bookkeeping while a solve is in flight
  int rhs = -1;
  int attempts = 0;
  int total_it = 0;
  ~Work();
};


}  // namespace tomg

struct tomg_problem {
  tomg_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;  // the problem's own stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // setup work that overlaps the rest of the setup (created on first use): the Chebyshev
  // bounds of the geometric levels on `side`, the AMG levels' spectral radii on `side2`
  cudaStream_t side = nullptr, side2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_side = nullptr, ev_fork2 = nullptr, ev_side2 = nullptr;
  int dim = 2, nx = 0, ny = 0, nz = 1;
  double E0 = 1, Emin = 1e-9, penal = 3, nu = 0.3;
  int64_t nn = 0, n = 0, nel = 0;
  std::vector<double> Ke_host;
  std::vector<float> Ke32_host;
  int ebe_tile = 0;    // autotuned tile of the quad4 FP32 element kernel (0 = default)
  int tc_mode = -1;    // hex8 FP32 element kernel: -1 as opt.prec says, 0 CUDA cores, 1 tensor cores
  int tc_nz = 0;       // node layers per block of the tensor-core kernel (0 = default)
  int tc_ty = 0;       // element rows per block of the tensor-core kernel (0 = default)
  int adapt_geo = 0;   // adaptive hybrid: geometric levels of the next setup (0 = not started)
  tomg::DBuf<uint32_t> Ketc;  // FP16 integer B operand of the tensor-core kernel (hex8)
  float tc_cl = 0.f, tc_cm = 0.f;  // its scales lambda / 72 and mu / 72
  tomg::DBuf<uint32_t> Kx64;  // integer B operand of the FP64 tensor-core kernel (hex8; empty if
  double x64_c = 0.0;         // nu admits none) and its scale: Ke = x64_c C
  std::map<cudaStream_t, tomg::DBuf<double>> x64buf;  // its work buffers, one per stream
  tomg::DBuf<double> Ke64;
  tomg::DBuf<float> Ke32;
  tomg::DBuf<uint8_t> mask;
  bool have_density = false;
  tomg::DBuf<double> rho, E64;
  tomg::DBuf<float> E32;
  // hierarchy
  bool setup_valid = false;
  int64_t setup_gen = 0;
  tomg_options opt{};
  double setup_ms = 0.0;
  bool jacobi_only = false;
  std::vector<std::unique_ptr<tomg::Level>> L;
  int nc = 0;  // coarsest DOFs
  tomg::DBuf<double> Ainv64;
  tomg::DBuf<float> Ainv32;
  // solve slots, and the work of a block solve of several right-hand sides
  std::vector<std::unique_ptr<tomg::Work>> works;
  std::unique_ptr<tomg::Work> bwork;
  int* flag_host = nullptr;  // pinned
  tomg::DBuf<int> flag_dev;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  ~tomg_problem();
};

namespace tomg {
// order the problem's stream after the context stream (entry) / the context after it (exit)
struct StreamScope {
  tomg_problem* P;
  explicit StreamScope(tomg_problem* p);
  ~StreamScope();
};

void problem_init(tomg_problem* P);
void set_fixed(tomg_problem* P, const int64_t* dofs, int64_t count);
void set_density(tomg_problem* P, const double* rho, int on_device);
void setup(tomg_problem* P, const tomg_options& opt);
tomg_status solve(tomg_problem* P, int nrhs, const double* f, double* u, int on_device,
                  tomg_result* res);
// single steps for parity checks
void level_apply(tomg_problem* P, int level, int prec, const double* x, double* y);
void outer_operator_apply(tomg_problem* P, const double* x, double* y);
void vcycle_apply(tomg_problem* P, const double* r, double* z);
void coarse_apply(tomg_problem* P, const double* b, double* x);
void level_export(tomg_problem* P, int level, int64_t* nnzb, int64_t* rp, int64_t* ci, double* v);
void prolong_export(tomg_problem* P, int level, int64_t* nnzb, int64_t* rp, int64_t* ci, double* v);
void element_stiffness_host(int dim, double nu, std::vector<double>& Ke);
size_t problem_device_bytes(const tomg_problem* P);
double time_fine_operator(tomg_problem* P, int op, int prec, int reps, int cold_l2);
void stress_stiffness_op(tomg_problem* P, const double* u, const double* x, double* y);
tomg_status buckling(tomg_problem* P, const double* u, int n_eig, int jmin, int jmax, double tol,
                     int max_iter, double* lambdas, double* modes, int on_device, int* iterations);
}  // namespace tomg
