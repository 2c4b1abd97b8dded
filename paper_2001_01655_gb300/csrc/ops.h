// Host-side launchers of the tomg kernels (one translation unit per kernel family).
// All launches are asynchronous on the given stream; `done` (nullable) is the solve's
// device flag: once it is set the solve-loop kernels return immediately.
#pragma once

#include <vector>

#include <functional>

#include "common.cuh"

namespace tomg {

// MODE_RESID0 fuses the first smoothing sweep from a zero guess with the residual that follows
// it: x = w Dinv b is WRITTEN to the x argument, and y = b - A x.
// MODE_CHEB is one step of the Chebyshev smoother with its residual: r = b - A x,
// d = c1 d_prev + c2 Dinv r (c2 passed as the omega argument), y = x + d (y must not alias
// x), d written to ChebArg::d; d_prev = 0 (dmode 0), the stored d (1) or x itself (2).
// MODE_CHEB0 fuses the first Chebyshev step from a zero guess with the second: x_1 = w0 Dinv b
// is formed where it is needed (never stored), then as MODE_CHEB with d_prev = x_1.
enum OpMode { MODE_APPLY = 0, MODE_RESID = 1, MODE_JACOBI = 2, MODE_RESID0 = 3, MODE_CHEB = 4,
              MODE_CHEB0 = 5 };
struct ChebArg {
  void* d = nullptr;  // T[n]
  double c1 = 0.0;
  double c2 = 0.0;    // the launchers take it through their omega argument
  int dmode = 0;
  double w0 = 0.0;    // MODE_CHEB0: weight of the first step
  // MODE_CHEB, dmode 0, with xc set: the step's iterate is x + P xc, the coarse correction xc of
  // the level below (grid cnx x cny x cnz) prolonged on the fly (the prolongation fused into the
  // first post-smoothing step; x itself is not written back)
  const void* xc = nullptr;
  int cnx = 0, cny = 0, cnz = 0;
};
// operator families whose kernels implement MODE_CHEB0 (quad4 level 0, stencils, BSR levels)
struct Scalars;

// ---------------- level 0: matrix-free SIMP element-by-element operator ----------------
// A = M (sum_e E_e Ke) M + (I - M), M = free-DOF mask (mask byte per node, bit c = DOF c
// fixed).  MODE_APPLY y = A x; MODE_RESID y = b - A x; MODE_JACOBI y = x + w Dinv (b - A x).
// dot_partials (nullable, MODE_APPLY only): one FP64 partial of x . y per block.
struct Ebe {
  int dim, nx, ny, nz;
  const void* Ke;  // T[nd*nd], nd = dim * 2^dim
  const void* E;   // T[n_elems]
  const uint8_t* mask;
  int tile = 0;    // quad4 FP32: nodes per thread of the tiled kernel (1, 2, 4; 0 = 4)
  const void* Kh = nullptr;  // host copy of Ke (T); the tiled kernels take Ke by value
  // hex8 FP32: element contractions on the tensor cores when tc != 0; Ktc holds the integer
  // FP16 B operand (ebe3d_tc_operand), tc_cl / tc_cm its scales lambda / 72, mu / 72, tc_nz the
  // node layers per block (0 = 8)
  int tc = 0;
  int tc_nz = 0;
  int tc_ty = 0;   // element rows per block of the tensor-core kernel (8 or 4; 0 = 8)
  const void* Ktc = nullptr;
  float tc_cl = 0.f, tc_cm = 0.f;
};
template <class T>
void ebe_op(cudaStream_t s, int mode, const Ebe& op, const T* x, T* y, const T* b,
            const T* Dinv, double omega, const int* done, double* dot_partials,
            const ChebArg* ch = nullptr);
int ebe_blocks(const Ebe& op);  // number of blocks (= number of dot partials) of ebe_op
// whether ebe_op in precision T takes MODE_CHEB0 on hex8 and a fused prolongation (ChebArg::xc):
// the FP32 tensor-core hex8 operator does
template <class T>
inline bool ebe_fuses_transfers(const Ebe& op) {
  return op.dim == 3 && sizeof(T) == 4 && op.tc != 0;
}
// quad4 tiled implementation behind ebe_op (k_ebe2d.cu)
template <class T, int MODE, bool DOT>
void ebe2d_launch(cudaStream_t s, const Ebe& op, const T* x, T* y, const T* b, const T* Dinv,
                  double omega, const int* done, double* parts, const ChebArg* ch = nullptr);
int ebe2d_blocks(const Ebe& op);
// fastest quad4 FP32 tile (nodes per thread) for this grid, timed on the stream with scratch
// vectors the first time a grid shape is seen, cached per shape afterwards
int ebe2d_autotune(cudaStream_t s, const Ebe& op, const float* Dinv);
// hex8 FP32 tiled implementation behind ebe_op (k_ebe3d.cu; no fused dot)
void ebe3d_launch(cudaStream_t s, int mode, const Ebe& op, const float* x, float* y,
                  const float* b, const float* Dinv, double omega, const int* done,
                  const ChebArg* ch = nullptr);
// hex8 FP32 on the tensor cores (k_ebe3tc.cu): tcgen05 kind::f16, x split in two FP16 parts
// against the integer parts of Ke, same modes
void ebe3d_tc_launch(cudaStream_t s, int mode, const Ebe& op, const float* x, float* y,
                     const float* b, const float* Dinv, double omega, const int* done,
                     const ChebArg* ch = nullptr);
// B operand of the tensor-core kernel for Poisson ratio nu: 72 K_l and 72 K_m (Ke = lambda K_l
// + mu K_m) as FP16 in the kernel's shared-memory layout; cl = lambda / 72, cm = mu / 72
void ebe3d_tc_operand(double nu, uint32_t* img, float* cl, float* cm);
// FP64 hex8 operator on the tensor cores (k_ebe3x64.cu): exact integer digit products of the
// element contractions, FP64 scaling and node sums.  ebe3x_operand builds its B operand (the
// integer matrix C with Ke = c C) and returns false when nu gives no small integer C.
bool ebe3x_operand(double nu, uint32_t* img, double* c);
int ebe3x_operand_words();
int ebe3x_blocks(const Ebe& op);  // blocks (= dot partials) of one apply, per right-hand side
// doubles of the work buffer of one apply per right-hand side (the tiles' node partial sums)
int64_t ebe3x_buffer_doubles(const Ebe& op);
// MODE_APPLY: y = A x, partials of x . y (nullable), FIN_ALPHA with sc; MODE_RESID: y = b - A x.
// pbuf: ebe3x_buffer_doubles x batch_rhs() doubles, owned by the caller (one per stream)
void ebe3x_apply(cudaStream_t s, int mode, const Ebe& op, const void* Bimg, double c,
                 const double* x, double* y, const double* b, const int* done, double* partials,
                 Scalars* sc, double* pbuf);
bool ebe3x_error(cudaStream_t s);  // a wait of the FP64 tensor-core kernel ran out (syncs s)
// polls of the tensor-core kernel's in-loop MMA waits in later launches (0 = the default);
// a test shortens it to make the waits run out and exercise the error path
void ebe3d_tc_set_wait_limit(int polls);
// polls of the grid barriers of the cooperative kernels (MIS-2 rounds, coarse inverse) in later
// launches (0 = each kernel's default); a test shortens it to make the waits run out
void set_grid_wait_limit(int polls);
unsigned grid_wait_limit(unsigned dflt);
// element stiffness of the unit quad4 / hex8 element for a constitutive matrix D (3x3 / 6x6,
// row-major), 2x2(x2) Gauss rule
void element_stiffness_D(int dim, const double* D, std::vector<double>& Ke);
int ebe3d_tc_operand_words();
// fastest tile of the tensor-core kernel for this grid, rows * 1000 + node layers per block
// (tc_ty, tc_nz), timed once per grid shape and cached
int ebe3d_tc_autotune(cudaStream_t s, const Ebe& op, const float* Dinv);
// true if a tensor-core kernel gave up waiting for its MMAs since the last call (syncs s)
bool ebe3d_tc_error(cudaStream_t s);
// point-block diagonal inverse of the level-0 operator, FP64 and FP32 copies
void ebe_block_diag_inv(cudaStream_t s, const Ebe& op64, double* Dinv64, float* Dinv32);
// level-0 operator assembled as a structured 3^dim stencil, FP64, SoA layout
// S[((o * dim + r) * dim + c) * n_nodes + node], o = (ox+1) + 3 (oy+1) + 9 (oz+1)
void ebe_assemble_stencil(cudaStream_t s, const Ebe& op64, double* S);
// E = Emin + (E0 - Emin) rho^p in FP64 and FP32; *bad set to 1 if rho < 0 or NaN
void simp_moduli(cudaStream_t s, int64_t nel, const double* rho, double E0, double Emin,
                 double penal, double* E64, float* E32, int* bad);

// ---------------- design iteration: density filter and sensitivities (k_design.cu) ------
// rho = S alpha (transpose = 0) or S^T g (transpose = 1), linear filter of radius in (0, 3];
// W: n_elems scratch (row sums)
void density_filter(cudaStream_t s, int dim, int nx, int ny, int nz, double radius, int transpose,
                    const double* in, double* out, double* W);
// dF/drho_e = -p rho_e^(p-1) (E0 - Emin) u_e^T Ke u_e
void compliance_sensitivity(cudaStream_t s, int dim, int nx, int ny, int nz, const double* Ke,
                            const double* rho, const double* u, double E0, double Emin,
                            double penal, double* dc);

// ---------------- linear buckling (k_stability.cu) -----------------------------------
int stress_components(int dim);  // 3 (2D) or 6 (3D) Voigt components per element
// centre stresses sigma_e = E_sigma(rho_e) D_0 B(centre) u_e, n_elems x stress_components
void element_stresses(cudaStream_t s, int dim, int nx, int ny, int nz, double nu, double E0,
                      double penal, const double* rho, const double* u, double* sig);
// y = M K_sigma M x from the element stresses (FP64)
void stress_stiffness_apply(cudaStream_t s, int dim, int nx, int ny, int nz, double nu,
                            const double* sig, const uint8_t* mask, const double* x, double* y);
// adjoint right-hand sides g_m = d(Phi_m^T K_sigma Phi_m)/du for nm modes (columns of Phi,
// leading dimension ldp); sw: scratch, nm x n_elems x stress_components doubles
void buckling_adjoint_rhs(cudaStream_t s, int dim, int nx, int ny, int nz, double nu, double E0,
                          double penal, const double* rho, const uint8_t* mask, int nm,
                          const double* Phi, int64_t ldp, double* sw, double* g, int64_t ldg);
// dlambda_m/drho (n_elems x nm, nullable) and sum_m coef_m dlambda_m/drho (n_elems, nullable);
// lam, coef: host arrays of nm <= 16 values
void buckling_sensitivity(cudaStream_t s, int dim, int nx, int ny, int nz, double nu, double E0,
                          double Emin, double penal, const double* Ke, const double* rho,
                          const uint8_t* mask, const double* u, int nm, const double* lam,
                          const double* coef, const double* Phi, const double* Vadj, int64_t ld,
                          double* dlam, double* dF);

// ---------------- geometric levels: structured stencils and transfers -----------------
struct Geo {
  int dim, nx, ny, nz;  // element counts of this level (nz = 1 in 2D)
  int64_t nodes() const { return (int64_t)(nx + 1) * (ny + 1) * (dim == 3 ? nz + 1 : 1); }
};
inline int stencil_q(int dim) { return dim == 3 ? 27 * 9 : 9 * 4; }
template <class T>
void stencil_op(cudaStream_t s, int mode, const Geo& g, const T* S, const T* x, T* y, const T* b,
                const T* Dinv, double omega, const int* done, const ChebArg* ch = nullptr);
void stencil_block_diag_inv(cudaStream_t s, const Geo& g, const double* S, double* Dinv64,
                            float* Dinv32);
// FP64 y = S x with per-block partials of x . y (stencil_blocks(g) partials); with sc set, the
// last block applies FIN_ALPHA (sc->done is then the early-exit flag)
void stencil_apply_dot(cudaStream_t s, const Geo& g, const double* S, const double* x, double* y,
                       const int* done, double* partials, Scalars* sc);
int stencil_blocks(const Geo& g);
// Galerkin product with bilinear / trilinear P (coarse node I at fine position min(2I, n))
void stencil_rap(cudaStream_t s, const Geo& fine, const Geo& coarse, const double* Sf, double* Sc);
// the FP32 copy the V-cycle's stencil kernels read: the upper half of the FP64 stencil (the
// centre and the offsets after it), in tiles of 32 nodes with the entries of a tile contiguous
int64_t stencil_half_size(const Geo& g);
void stencil_half_f32(cudaStream_t s, const Geo& g, const double* S64, float* S32);
// hex8: the first coarse stencil P^T A_0 P straight from the level-0 elements (FP64 operator
// op64, coarse grid c = the coarsening of op64's grid).  Returns false, writing nothing, when
// more than one element in eight touches a fixed DOF (the caller then takes the product on the
// assembled fine stencil).  Synchronises s once (the count of those elements).
bool ebe_galerkin_stencil(cudaStream_t s, const Ebe& op64, const Geo& c, double* Sc);
template <class T>
void geo_restrict(cudaStream_t s, const Geo& fine, const Geo& coarse, const T* rf, T* bc,
                  const int* done);
template <class T>
void geo_prolong_add(cudaStream_t s, const Geo& fine, const Geo& coarse, const T* xc, T* xf,
                     const int* done);
// stencil -> dense (n x n, row-major) and stencil -> BSR (two calls: counts then fill)
void stencil_to_dense(cudaStream_t s, const Geo& g, const double* S, double* Adense);
void stencil_row_counts(cudaStream_t s, const Geo& g, int* counts);
void stencil_to_bsr(cudaStream_t s, const Geo& g, const double* S, const int* rowptr, int* col,
                    double* val);
// geometric prolongation as BSR (dim x dim blocks w I): counts then fill
void geo_prolong_counts(cudaStream_t s, const Geo& fine, const Geo& coarse, int* counts);
void geo_prolong_fill(cudaStream_t s, const Geo& fine, const Geo& coarse, const int* rowptr,
                      int* col, double* val);

// ---------------- block CSR (BSR) ------------------------------------------------------
struct Bsr {
  int nbr = 0, nbc = 0, br = 0, bc = 0;
  int64_t nnzb = 0;
  const int* rp = nullptr;
  const int* ci = nullptr;
};
template <class T>
void bsr_op(cudaStream_t s, int mode, const Bsr& A, const T* V, const T* x, T* y, const T* b,
            const T* Dinv, double omega, const int* done, const ChebArg* ch = nullptr);
// y (+)= A x for rectangular blocks (transfers): accumulate = 1 adds into y
template <class T>
void bsr_spmv_rect(cudaStream_t s, const Bsr& A, const T* V, const T* x, T* y, int accumulate,
                   const int* done);
void bsr_block_diag_inv(cudaStream_t s, const Bsr& A, const double* V, double* Dinv64,
                        float* Dinv32);
void bsr_to_dense(cudaStream_t s, const Bsr& A, const double* V, double* Adense);
// transpose: rowptr of A^T from column counts, then fill (rows of A^T sorted)
void bsr_col_counts(cudaStream_t s, const Bsr& A, int* counts /* nbc, zeroed inside */);
void bsr_transpose_fill(cudaStream_t s, const Bsr& A, const double* V, const int* rpT, int* ciT,
                        double* VT, int* cursor /* nbc scratch */);
// SpGEMM C = A B (FP64): symbolic counts, symbolic fill (sorted columns), numeric
struct SpgemmWork {
  DBuf<int> big, goff, gtable;  // per-row hash-table sizes / offsets for rows too long for smem
};
void spgemm_counts(cudaStream_t s, const Bsr& A, const Bsr& B, int* counts, SpgemmWork& w);
void spgemm_fill(cudaStream_t s, const Bsr& A, const Bsr& B, const int* rpC, int* ciC,
                 SpgemmWork& w);
// sym: C is known to be symmetric with square blocks (a Galerkin product P^T (A P)): the few
// long rows of the coarse products then compute each off-diagonal block pair once
void spgemm_numeric(cudaStream_t s, const Bsr& A, const double* VA, const Bsr& B,
                    const double* VB, const Bsr& C, double* VC, bool sym = false);
void cast_f64_f32(cudaStream_t s, const double* a, float* b, int64_t n);
void cast_f32_f64(cudaStream_t s, const float* a, double* b, int64_t n);

// ---------------- prefix sums --------------------------------------------------------
// exclusive scan of n ints into out (n+1 entries; out[n] = total); returns total (syncs)
int64_t exclusive_scan(cudaStream_t s, const int* in, int* out, int64_t n);
// the same scan without reading the total back (no host synchronisation)
void exclusive_scan_nosync(cudaStream_t s, const int* in, int* out, int64_t n);

// ---------------- smoothed aggregation ------------------------------------------------
void amg_strength_counts(cudaStream_t s, const Bsr& A, const double* V, double beta, int* counts);
void amg_strength_fill(cudaStream_t s, const Bsr& A, const double* V, double beta, const int* srp,
                       int* sci);
// distance-2 MIS rounds; returns number of rounds
int amg_mis2(cudaStream_t s, int n, const int* srp, const int* sci, int level, int* state,
             uint64_t* v, uint64_t* m1, int* flag_host_pinned, int* flag_dev);
// aggregates from MIS-2 states: agg (n), returns number of aggregates
int amg_aggregate(cudaStream_t s, int n, const int* srp, const int* sci, int level,
                  const int* state, int* agg, int* root_scan);
// tentative prolongator: T as BSR (one block per aggregated node), Bc (n_agg*k x k)
int64_t amg_tentative(cudaStream_t s, int n_nodes, int b, int k, int n_agg, const int* agg,
                   const double* B, int* Trp, int* Tci, double* TV, double* Bc);
// spectral radius of D^-1 A by power iteration (FP64) on an assembled BSR level, in three
// steps so that the launches can run on another stream than the allocation: amg_power_alloc
// (buffers and the zeroed ticket, in the order of stream s), amg_power_enqueue (launches on s),
// amg_power_result (copies rho back on s and synchronises s)
struct AmgPower {
  DBuf<double> v, w, parts, nrm;
  DBuf<unsigned> ticket;
  int iters = 0;
};
void amg_power_alloc(cudaStream_t s, AmgPower& ps, const Bsr& A, int iters);
void amg_power_enqueue(cudaStream_t s, AmgPower& ps, const Bsr& A, const double* V,
                       const double* Dinv, int level);
double amg_power_result(cudaStream_t s, const AmgPower& ps);
// v[i] = (splitmix64(i + SALT_POWER + level) >> 11) 2^-53 - 0.5 (the power-iteration start vector)
void splitmix_uniform(cudaStream_t s, int64_t n, int level, double* v);
// spectral radius of D^-1 A for an operator applied by `apply(x, y)` (y = A x, FP64, n = nodes *
// bs), same start vector and iteration as amg_spectral_radius; returns rho (syncs)
double spectral_radius_op(cudaStream_t s, int64_t nodes, int bs, const double* Dinv, int level,
                          int iters, const std::function<void(const double*, double*)>& apply);
// the same iteration in two halves, so that it can run on another stream than the one that
// allocates its buffers: power_alloc (allocation-stream order), power_enqueue (launches only, on
// s), power_result (copies rho back on s and synchronises s)
struct PowerState {
  DBuf<double> v, w, t, parts, nrm;
  DBuf<float> v32, w32, t32;  // iteration vectors of the FP32 variant
  DBuf<unsigned> ticket;
  int64_t nodes = 0;
  int bs = 0, iters = 0;
};
void power_alloc(PowerState& ps, int64_t nodes, int bs, int iters, bool f32 = false);
void power_enqueue(cudaStream_t s, PowerState& ps, const double* Dinv, int level,
                   const std::function<void(const double*, double*)>& apply);
// the same iteration with FP32 vectors, operator and block inverses (Dinv32), for the
// Chebyshev interval of a mixed-precision cycle; norms accumulated and kept in FP64
void power_enqueue_f32(cudaStream_t s, PowerState& ps, const float* Dinv32, int level,
                       const std::function<void(const float*, float*)>& apply);
double power_result(cudaStream_t s, const PowerState& ps);
// P = T - omega Dinv (A T) on the pattern of AT
void amg_smooth_prolongator(cudaStream_t s, const Bsr& AT, const double* ATV, const int* agg,
                            const double* TV, const int* Trp, const double* Dinv, double omega,
                            int b, double* PV);
// coarse DOFs with an all-zero row get a unit diagonal
void amg_fix_zero_rows(cudaStream_t s, const Bsr& A, double* V);
// rigid-body modes at node coordinates (dim 2: 3 modes, dim 3: 6 modes), n x k row-major
void rigid_body_modes(cudaStream_t s, const Geo& g, const double* xs, const double* ys,
                      const double* zs, double* B);

// ---------------- Krylov vectors, reductions, coarse solve -----------------------------
struct Scalars {     // device-resident state of one outer solve
  double bb, rr, rz, pq, zq, rz_new, alpha, beta, rtol2, tol2;
  int done, it, status, max_iter, flexible, pad;
  unsigned tk[4];    // arrival tickets of the kernels that finish their own reductions
};
enum Ticket { TK_ALPHA = 0, TK_RR = 1, TK_DOTS = 2 };
int red_blocks(int64_t n);
void dot_partials(cudaStream_t s, const double* x, const double* y, int64_t n, double* partials,
                  const int* done);
// finish kernels (single block): combine partials and update the scalar state
enum FinishKind { FIN_INIT = 0, FIN_RZ0 = 1, FIN_ALPHA = 2, FIN_RR = 3, FIN_BETA = 4 };
void finish(cudaStream_t s, int kind, const double* partA, int nA, const double* partB, int nB,
            Scalars* sc);
// x += alpha p, r -= alpha q, r32 = (float) r (nullable), then FIN_RR in the last block
void xr_update(cudaStream_t s, double* x, double* r, const double* p, const double* q, int64_t n,
               Scalars* sc, double* partials, float* r32);
// while condition of a captured block solve of nrhs right-hand sides: some one not done
void block_cond(cudaStream_t s, const Scalars* sc, int nrhs, cudaGraphConditionalHandle cond);
// p = z + beta p; with has_cond, also sets the graph's while condition to !done
void p_update(cudaStream_t s, double* p, const double* z, int64_t n, const Scalars* sc,
              cudaGraphConditionalHandle cond, int has_cond);
// z64 = (double) z (T = float) or z itself; partials of z.r and z.q (q nullable), then finish
// step `kind` (FIN_RZ0 or FIN_BETA) in the last block
template <class T>
void z_dots(cudaStream_t s, const T* z, double* z64, const double* r, const double* q, int64_t n,
            double* partA, double* partB, Scalars* sc, int kind);
template <class T>
void cast_in(cudaStream_t s, const double* a, T* b, int64_t n, const int* done);
void copy_f64(cudaStream_t s, const double* a, double* b, int64_t n, const int* done);
void mask_vec(cudaStream_t s, const double* f, double* b, const uint8_t* mask, int dim, int64_t nn);
// x = w Dinv b (first Jacobi sweep from x = 0), block size bs
template <class T>
void jacobi0(cudaStream_t s, int bs, int64_t nodes, const T* Dinv, const T* b, T* x, double omega,
             const int* done);
// GMRES smoother (k_gmres_smooth.cu): state of one smoothing in device memory; the ticket
// must be zero when the state is first used
constexpr int GM_MAX = 8;  // most Arnoldi steps per smoothing
struct GmState {
  double H[(GM_MAX + 1) * GM_MAX];  // Hbar, column-major, leading dimension GM_MAX + 1
  double h1[GM_MAX], h2[GM_MAX];    // the two Gram-Schmidt passes' projections of a step
  double beta, inv;                 // ||r_0||; 1 / norm of the vector being normalised
  double y[GM_MAX];                 // least-squares solution
  int meff;                         // steps before an exact breakdown
  unsigned tk;                      // last-block ticket
};
int gmres_smooth_parts(int64_t n);  // FP64 scratch partials for vectors of n entries
// beta = ||r0||, first scale
template <class T>
void gmres_smooth_begin(cudaStream_t s, int64_t n, const T* r0, double* parts, GmState* st, int m,
                        const int* done);
// v_j (from src: r0 for j = 0, slot j of V otherwise), z_j = D^-1 v_j (bs x bs blocks)
template <class T>
void gmres_smooth_next(cudaStream_t s, int bs, int64_t nodes, int j, const T* src, T* V,
                       int64_t ldv, T* Z, const T* Dinv, const GmState* st, const int* done);
// after w = A z_j is in slot j + 1 of V: both Gram-Schmidt passes, column j of Hbar, and the
// least-squares solve after the last step (j = m - 1)
template <class T>
void gmres_smooth_orth(cudaStream_t s, int64_t n, int j, int m, T* V, int64_t ldv, double* parts,
                       GmState* st, const int* done);
// out = x0 + Z y (x0 nullable: zero)
template <class T>
void gmres_smooth_finish(cudaStream_t s, int64_t n, int m, const T* Z, int64_t ldv,
                         const GmState* st, const T* x0, T* out, const int* done);
// flexible GMRES: h[k] = V_k . w for k < J (V_k = V + k ldv; parts: multi_dot_parts(J)
// scratch), w += sign sum_k c[k] V_k, v = s w
void multi_dot(cudaStream_t s, int64_t n, int J, const double* V, int64_t ldv, const double* w,
               double* parts, double* h);
int multi_dot_parts(int J);
void multi_update(cudaStream_t s, int64_t n, int J, const double* V, int64_t ldv, const double* c,
                  double sign, double* w);
void scale_into(cudaStream_t s, int64_t n, const double* w, double sc, double* v);
// coarse solve x = Ainv b (dense GEMV)
template <class T>
void dense_gemv(cudaStream_t s, int n, const T* Ainv, const T* b, T* x, const int* done);
// dense SPD inverse via Cholesky (FP64, in place: A -> A^-1); returns 0 or row of failure+1
int dense_spd_inverse(cudaStream_t s, int n, double* A, double* work);

}  // namespace tomg
