// Launchers of the CUDA kernels (host-callable, defined in the .cu files).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace fdfd {

// ---- assembly.cu: stencil coefficients (Eq. 1-2 with SC-PML) ---------------
// (sxc, syc: the stretch factors at cell centres, whose product is the symmetriser D)
void launch_coef(double2* cxm, double2* cxp, double2* cym, double2* cyp, double* k0dx2, double2* sxc,
                 double2* syc, const double* k0dx_dev, int n_omega, int nx, int ny, int npml_x, int npml_y,
                 double ln_R, double order, cudaStream_t s);
void launch_scatter_design(double* eps, const double* eps_design, int ny, int x0, int y0, int w,
                           int h, cudaStream_t s);

// ---- factor.cu: multifrontal numeric factorisation -----------------------
struct FactorLaunch {
  DevPlan P;
  DevCoef C;
  void* store;             // float2* or double2*, [n_omega][store_stride]
  long long store_stride;
  int* perm;               // [n_omega][perm_stride]
  int perm_stride;
  float* growth;           // [n_omega][n_fronts]: max |L| entry (inf when a pivot is zero)
  int n_fronts;
  int n_omega;             // wavelengths launched: [w0, w0 + n_omega)
  int w0;
  int* swp;                // panel row-swap scratch: [n_omega launched][swp_stride][130]
  int swp_stride;          // >= number of fronts in one large-front list
  void* istore;            // triangular inverses (same type as store), [n_omega][istore_stride]
  long long istore_stride;
  void* dblk;              // a panel step's diagonal-block factors, [n_omega launched][swp_stride][kDiagBlkElems]
  int sym;                 // 1: symmetric form, M = D A = L diag(d) L^T without pivoting (see factor.cu)
  const unsigned char* pivonly = nullptr;   // per front, or null: 1 = the panel steps factor the k x k pivot block
                                            // only; L21 and U12 then come from the tensor cores
                                            // (TcFront modes 1, 2)
};
constexpr int kDiagBlkElems = 32 * 32 + 32;   // L\U rows in pivot order, then 1 / U_pp
// L11^-1 (strictly lower part) and U11^-1 (upper part) of the listed large fronts,
// one CTA per (front, 32-column block, triangle); kmax = largest k listed.
template <typename T> void launch_lu_inv(const FactorLaunch& a, const int* flist, int nf, int kmax, cudaStream_t s);
// max over growth[0..count) (NaN wins) into *out
cudaError_t launch_growth_max(const float* growth, long long count, float* out, cudaStream_t s);
// build (assemble originals + extend-add children) rows listed in tasks (front, row0)
template <typename T> void launch_build(const FactorLaunch& a, const int2* tasks, int ntasks, cudaStream_t s);
// whole-front LU in shared memory, one CTA per front
template <typename T> void launch_lu_small(const FactorLaunch& a, const int* flist, int nf, int nmax,
                                           cudaStream_t s);
// blocked right-looking LU of large fronts: one panel step at column j0.
// panel: pivot-candidate rows [j0, k) of columns [j0, j0+nb) (kmax = largest k listed);
// l21: boundary rows [k, n) of the panel (mmax = largest m listed).
template <typename T> void launch_lu_panel(const FactorLaunch& a, const int* flist, int nf, int j0,
                                           int nb, int kmax, cudaStream_t s);
template <typename T> void launch_lu_l21(const FactorLaunch& a, const int* flist, int nf, int j0,
                                         int nb, int mmax, int nmax, int below, cudaStream_t s);
// Pivoting restricted to the 32 x 32 diagonal block J = [j0, j0 + 32): one launch
// does the block's LU, the L columns below it, the U rows right of it, the row
// permutation of earlier columns and perm, and writes L_JJ^-1 / U_JJ^-1 into the
// diagonal block of the inverse store; then launch_lu_gemm does the trailing
// update and launch_lu_inv_fold the rest of block row / column J of the inverses.
// nmax = largest n listed.
template <typename T> void launch_lu_step_local(const FactorLaunch& a, const int* flist, int nf, int j0,
                                                int nmax, cudaStream_t s);
constexpr int kSwapScratchInts = 130;   // ints of swap scratch per (wavelength, listed front)
template <typename T> void launch_lu_trsm(const FactorLaunch& a, const int* flist, int nf, int j0,
                                          int nb, int nmax, cudaStream_t s);
// Update matrix of the listed large fronts after their last panel: S = F22 - L21 U12
// (K = k), SIMT complex FMA; mmax = largest m listed.
template <typename T> void launch_schur_simt(const FactorLaunch& a, const int* flist, int nf, int mmax,
                                             cudaStream_t s);
// The same update matrix on the tensor cores (tc_schur.cu), complex64 fronts only:
// P = L21 U12 as one real GEMM of the interleaved L21 with the 2 x 2 real
// embedding of U12, FP32 accumulation in tensor memory, S = F22 - P in place.
// Output tiles are kTcRows x kTcCols complex; the contraction advances kTcPivots
// pivots per pipeline stage.  form: 1 = TF32, 2 = TF32 hi + lo (three products),
// 3 = BF16 three-way split (six products).
constexpr int kTcRows = 128, kTcCols = 128, kTcPivots = 8;
// The same pipeline also forms the off-diagonal blocks of a front whose panel
// steps factored only its pivot block (P F11 = L11 U11, inverses in the inverse
// store), as products with the triangular inverses:
//   mode 1: L21 = F21 U11^-1      (m x k, written over F21; its largest |entry| is growth)
//   mode 2: U12 = L11^-1 (P F12)  (k x m, written over F12; rows of F12 gathered by perm)
// A triangular operand's zero blocks are skipped: an output tile of columns
// (mode 1) or rows (mode 2) below 128 (t + 1) contracts over the first 128 (t + 1)
// pivots only.
struct TcFront {           // one front of a tensor-core launch
  long long aoff, boff;    // byte offsets of its packed A / B planes in one wavelength's workspace
  long long poff;          // float offset of its split partial sums in one wavelength's partial buffer
  int f;                   // front index
  int Mt, Nt, Kt;          // row tiles, column tiles, k-tiles (mode 0: ceil(m/128), ceil(m/128), ceil(k/8))
  int nsplit;              // contraction split over this many CTAs per output tile (1 = none; modes 1, 2: 1)
  int mode = 0;            // 0: S = F22 - L21 U12; 1: L21; 2: U12
};
constexpr int kTcPartFloats = kTcRows * 2 * kTcCols;   // one split partial: 128 x 256 FP32
struct TcLaunch {
  const TcFront* fronts;
  const int4* tasks;       // pack: (slot, 0 = L21 / 1 = U12, row or column tile, k-tile); product: (slot, mt, nt, 0)
  unsigned char* ws;       // packed planes, [n_omega launched][ws_stride] bytes
  long long ws_stride;
  int* err;                // set to 2 when a pipeline wait gives up
  int chunk;               // k-tiles summed in tensor memory before the FP32 register sum takes them
  float* part;             // split partial sums, [n_omega launched][part_stride] floats
  long long part_stride;
};
// K splits of a front's output tiles so that a launch of `tiles` tiles (over all
// wavelengths) fills min_ctas CTAs, each split keeping at least 4 k-tiles.
int tc_splits(long long tiles, int Kt, int min_ctas);
long long tc_tile_bytes_a(int form);   // bytes of one packed L21 tile (all planes)
long long tc_tile_bytes_b(int form);   // bytes of one packed U12 tile (all planes)
void launch_schur_tc_pack(const FactorLaunch& a, const TcLaunch& t, int ntasks, int form, cudaStream_t s);
void launch_schur_tc(const FactorLaunch& a, const TcLaunch& t, int ntiles, int form, cudaStream_t s);
// split tiles: S -= the sum of their partials; tasks (slot, mt, nt, first row of 16)
void launch_schur_split_sum(const FactorLaunch& a, const TcLaunch& t, int ntasks, cudaStream_t s);
cudaError_t tc_init_attributes();        // once per device, before the first factorisation
// one bounded mbarrier wait (the product kernel's) on a barrier nothing arrives at; sets *err = 2
cudaError_t launch_mbar_probe(int* err, cudaStream_t s);
// panel-step trailing update restricted to the pivot-block rows and columns
template <typename T> void launch_lu_gemm(const FactorLaunch& a, const int* flist, int nf, int j0,
                                          int nb, int nmax, cudaStream_t s);
// block row J of L11^-1 and block column J of U11^-1 (J = [j0, j0 + 32)) after
// launch_lu_step_local wrote the diagonal block J and the folds of
// the earlier blocks are done; reads only entries that no later step writes, so
// it may run beside the front's later steps.
template <typename T> void launch_lu_inv_fold(const FactorLaunch& a, const int* flist, int nf, int j0,
                                              cudaStream_t s);
int lu_small_max_n(int elem_bytes);
// largest n of small-front size class c (0..kSmallClasses-1); each class is one launch per level
constexpr int kSmallClasses = 4;
int lu_small_class_n(int c);
cudaError_t factor_init_attributes();   // once per device, before the first factorisation
int lu_panel_width(int elem_bytes);

// ---- solve.cu: level-scheduled triangular sweeps ---------------------------
// sweep task words: front index in the low 29 bits; bit 29 = a row task of
// 2 x sweep_row_block() rows (two per warp); bit 30 = off-diagonal block; bit 31
// = a whole small or medium front
constexpr int kSweepFrontMask = 0x1fffffff;
constexpr int kSweepTaskTall = 0x20000000;
struct SolveLaunch {
  DevPlan P;
  const void* store;       // factor storage (T), [n_omega][store_stride]
  long long store_stride;
  const int* perm;
  int perm_stride;
  const void* istore;      // triangular inverses (T), [n_omega][istore_stride]
  long long istore_stride;
  void* vb;                // front vectors (T), [n_sys][vec_stride]
  long long vec_stride;
  int n_omega, nrhs;       // wavelengths launched [w0, w0 + n_omega); nrhs = layout stride
  int w0, r0, nr;          // right-hand sides processed: [r0, r0 + nr)
  long long n;             // unknowns per system
  // symmetric-form factors (L diag(d) L^T of D A): the L sweep gathers D b
  // (sym_in), the L^T sweep takes w = y / d where it first reads a front's y
  // (sym_mid) and writes D x (sym_out); D from the stretch tables below
  int sym_in = 0, sym_mid = 0, sym_out = 0;
  const double2* sxc = nullptr;   // [n_omega][nx]
  const double2* syc = nullptr;   // [n_omega][ny]
};
// With sym_out the L^T sweep writes D x; the fronts below read their boundary values x_m
// back from the output, so they divide D out again.
// sweep: 0 = L (forward, non-transposed), 1 = U (backward, non-transposed),
//        2 = U^T (forward of the transpose solve), 3 = L^T (backward of the transpose solve).
// Large fronts are cut into row tasks of sweep_row_block() rows (sweeps 0, 1)
// or column tasks of sweep_col_block() columns (sweeps 2, 3).
int sweep_row_block();
int sweep_col_block();

// One direction of a sweep pair as a single persistent launch (dataflow over
// the elimination tree).  tasks: the direction's inverse-block, off-diagonal
// and whole-front tasks in dependency order (per level: whole small fronts,
// whole medium fronts, then the large fronts' phase-1 and phase-2 tasks),
// x = front | 1<<31 (whole front: y = 0 for one warp, y = 1 for one CTA) |
// 1<<30 (off-diagonal task), y = first row / column.
struct FlowQueue {
  const int2* tasks;
  const int2* units;       // what one CTA takes at a time: (first task, 1) for a large-front task or a
                           // whole medium front, or
                           // (first task, 0x80000000 | count) for up to 8 whole small fronts of one level
  int nunits;              // units; each runs for every launched wavelength
  int* ctr;                // [1 + 2 * n_omega * n_fronts] ints, zero before the launch
  const int* need_all;     // [n_fronts] tasks of each front in this queue
  const int* need_ph1;     // [n_fronts] its phase-1 tasks (inverse-block bottom-up, off-diagonal top-down)
  int* err;                // set to 1 by a wait that gives up (never cleared by the kernel)
  int n_fronts;
};
// in: right-hand sides, out: solutions, both complex128 [systems][n] whatever the
// factor precision T (converted where the sweeps gather them and store them).
// wide: the variant that keeps six CTAs resident per SM (large problems) instead of four
// pairs: allow the paired-RHS variant (complex64 factors, even count per wavelength)
template <typename T> void launch_sweep_flow(const SolveLaunch& a, int sweep, const FlowQueue& q, int vmax,
                                             int grid, const void* in, void* out, cudaStream_t s, bool wide,
                                             bool pairs);
// pair: the variant that takes right-hand sides in pairs (complex64 factors, even count per wavelength)
int flow_blocks_per_sm(int elem_bytes, int vmax, bool wide, bool pair = false);
int flow_whole_max_n();   // largest front the flow kernel runs as a one-warp whole-front task
int flow_cta_max_n();     // largest front it runs as one whole-front task of a CTA
// one bounded wait on a zero flag (gives up, sets *err); for the self-test entry point
cudaError_t launch_wait_probe(const int* flag, int* err, cudaStream_t s);

// ---- vec.cu: FP64 refinement, objective, gradient ---------------------------
// y = A x (op = 0) or r = b - A x (op = 1), FP64 matrix-free stencil, all systems.
void launch_stencil(const DevCoef& c, int n_omega, int nrhs, int transpose, const double2* x,
                    const double2* b, double2* y, int op, cudaStream_t s);
// batched dot products h[s][i] = sum conj(V_i[s]) w[s], i < nv (V_i at V + i*vstride)
void launch_multidot(const double2* V, long long vstride, int nv, const double2* w, long long n,
                     int nsys, double2* partial, int nblk, double2* out, int out_ld, cudaStream_t s);
// w[s] -= sum_i h[s][i] V_i[s]
void launch_multiaxpy(const double2* V, long long vstride, int nv, const double2* h, int h_ld,
                      double2* w, long long n, int nsys, const int* active, cudaStream_t s);
int multidot_blocks(long long n);
int multidot_max_vectors();
int arnoldi_blocks(long long n);   // chunks of an Arnoldi pass (partial sums per output)

// FGMRES bookkeeping (one thread per system); see vec.cu
void gm_start(const double2* rr, int rr_ld, const double2* bb, int bb_ld, int nsys, double tol, int m,
              double2* g, double* vscale, int* active, double* resid, double* bnorm, int first, cudaStream_t s);
void gm_solve(const double2* H, const double2* g, int nsys, int m, const int* njs, double2* ny_out,
              cudaStream_t s);
void gm_scale(double2* dst, const double2* src, const double* scale, long long n, int nsys, cudaStream_t s);
// One FGMRES Arnoldi step (classical Gram-Schmidt twice, then the Givens
// update) for every active system in three launches, pass = 0, 1, 2:
//   0: w = A z (A^T if transpose), h1 = V^H w;  1: w -= V h1, h2 = V^H w;
//   2: w -= V h2, hn = |w|^2, column nv - 1 of H from h1 + h2 and hn, nj += 1.
// h1, h2, hn: [nsys][multidot_max_vectors()]; partial: [nsys][multidot_max_vectors()]
// [arnoldi_blocks(n)];
// cnt: [nsys] zero, left zero.
struct ArnoldiStep {
  DevCoef C;
  int nrhs, transpose;
  const double2* z;
  const double2* V;
  long long vstride;
  int nv;                  // V_0 .. V_{nv-1}; the step is j = nv - 1
  double2* w;
  double2* partial;
  int* cnt;
  double2 *h1, *h2, *hn;
  int* nj;
  int* active;
  double* resid;
  const double* bnorm;
  double* vscale;
  double2 *H, *cs, *sn, *g;
  int m;
  double tol;
};
void launch_arnoldi(const ArnoldiStep& g, int nsys, int pass, cudaStream_t s);

// objective o = g^T x on a monitor column, F = sum weight |o|^2 with adjoint source weight conj(o) g,
// or with target != NULL F = sum weight (|o|^2 - target)^2 with adjoint source 2 weight (|o|^2 - target) conj(o) g
void launch_objective(const double2* x, long long N, int ny, const int* cols, const double2* gline,
                      const double* weight, const double* target, int nsys, double2* o, double* F, double2* badj,
                      cudaStream_t s);
// dF/deps over the design box: sum weight * 2 (k0dx)^2 Re(x_adj x_fwd)
void launch_grad(const double2* xf, const double2* xa, long long N, int ny, int x0, int y0, int w, int h,
                 int n_omega, int nrhs, const double* k0dx2, const double* weight, double* grad, int accumulate,
                 cudaStream_t s);
cudaError_t solve_init_attributes();

// ---- design.cu: smoothing filter and projection of the design density (Sec. III)
// off / wt: the filter taps (integer offsets inside the radius and their weights
// radius - distance), ntap of them; pixels x-major (i * h + j).
void launch_filter_project(const double* rho, int w, int h, const int2* off, const double* wt, int ntap,
                           double beta, double eta, double eps_lo, double deps, double* eps, double* slope,
                           double* norm, cudaStream_t s);
// eps = eps_lo + rho * deps over n pixels
void launch_density_eps(const double* rho, long long n, double eps_lo, double deps, double* eps, cudaStream_t s);
void launch_filter_adjoint(const double* g, const double* slope, const double* norm, int w, int h, const int2* off,
                           const double* wt, int ntap, double* out, cudaStream_t s);

}  // namespace fdfd
