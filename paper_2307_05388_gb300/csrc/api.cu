// C ABI of libfdfd (declared in include/fdfd.h): context, level scheduling of
// the multifrontal factorisation and of the triangular sweeps, the FGMRES
// refinement driver and the operation counters of the paper's Sec. III-IV.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fdfd.h"
#include "kernels.h"
#include "plan.h"

using namespace fdfd;

namespace fdfd {
cudaError_t launch_growth_max(const float* growth, long long count, float* out, cudaStream_t s);
}

namespace {

// k-tiles (of kTcPivots pivots) a tensor-core update matrix sums in tensor memory
// before its FP32 register sum takes them
constexpr int kTcChunk = 1;

struct LevelList {
  int task_off = 0, ntasks = 0;      // build tasks (int2) offset / count
  int small_off[kSmallClasses] = {}, nsmall[kSmallClasses] = {}, nmax_small[kSmallClasses] = {};   // small fronts by size class
  int large_off = 0, nlarge = 0, nmax_large = 0, kmax_large = 0, mmax_large = 0;
  int simt_off = 0, nsimt = 0, mmax_simt = 0;   // large fronts whose update matrix is formed by SIMT
  int tcf_off = 0, ntcf = 0;                    // ... on the tensor cores: TcFront records
  int tcp_off = 0, ntcp = 0;                    // their pack tasks (int4)
  int tct_off = 0, ntct = 0;                    // their output tiles and K splits (int4)
  int tcs_off = 0, ntcs = 0;                    // 16-row sums of their split tiles (int4)
  // c64 LU fronts on the tensor cores: their L21 and U12 too (TcFront modes 1, 2), after
  // panel steps over the pivot block only
  int tqf_off = 0, ntqf = 0;                    // TcFront records (two per front)
  int tqp_off = 0, ntqp = 0;                    // their pack tasks
  int tqt_off = 0, ntqt = 0;                    // their output tiles
};

struct TaskList {
  int off = 0, n = 0;      // int2 (front, first row or column) tasks at d_lists + off
};


// Sweep tasks of one level; index 0 = row tasks (sweeps L, U), 1 = column tasks (U^T, L^T).
struct SolveList {
  TaskList tri[2];         // inverse-block products, every front of the level
  TaskList rect_m[2];      // off-diagonal block split over the m boundary rows/columns
  TaskList rect_k[2];      // off-diagonal block split over the k pivot rows/columns
  int kmax = 0;            // shared-memory vector entries the tri launch needs
  int kbig = 0, mbig = 0;  // largest k and m among fronts with boundary rows
};

template <typename P>
cudaError_t dalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  return cudaMalloc((void**)p, bytes);
}

}  // namespace

struct fdfd_ctx {
  int nx = 0, ny = 0;
  double dx = 0;
  int n_omega = 0;
  std::vector<double> k0dx;
  fdfd_pml pml{};
  fdfd_box box{};
  fdfd_options opt{};
  cudaStream_t stream = nullptr;
  // CUDA graphs of fixed launch sequences (factorisations, sweep pairs on the
  // internal buffers), captured on a private stream joined to `stream` by events
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  // side stream of a factorisation: the inverse folds of the large fronts run
  // there, forked after each panel step and joined at the end
  cudaStream_t istream = nullptr;
  cudaEvent_t iev_fork = nullptr, iev_join = nullptr;
  struct GraphEntry { int key; cudaGraphExec_t exec; };
  std::vector<GraphEntry> graphs;
  std::string err;
  int device = -1;

  Plan plan;
  bool analyzed = false;
  bool uploaded = false;

  // device copy of the plan
  FrontDesc* d_fronts = nullptr;
  int* d_children = nullptr;
  int* d_idx = nullptr;
  int* d_inv = nullptr;
  int* d_orig_ptr = nullptr;
  int* d_orig_col = nullptr;
  int* d_orig_code = nullptr;
  int* d_lists = nullptr;          // all per-level lists (ints; build tasks as int pairs)
  std::vector<int> h_lists;
  // tensor-core update matrices: front records, pack and tile tasks, packed-operand workspace
  TcFront* d_tcf = nullptr;
  int4* d_tct = nullptr;
  unsigned char* d_tcws = nullptr;
  long long tc_ws_stride = 0;      // bytes per wavelength
  float* d_tcpart = nullptr;       // split partial sums
  long long tc_part_stride = 0;    // floats per wavelength
  std::vector<TcFront> h_tcf;
  std::vector<int4> h_tct;
  unsigned char* d_pivonly = nullptr;   // [full, design][front]: c64 LU panel steps over the pivot block only
  std::vector<unsigned char> h_pivonly;
  std::vector<LevelList> lv_full[3], lv_design[3];   // [0 = c64 LU, 1 = c128 LU, 2 = c64 symmetric form]
  std::vector<SolveList> lv_solve;
  // dataflow sweep queues [task type: 0 rows, 1 columns][direction: 0 bottom-up, 1 top-down]
  struct FlowList { int off = 0, n = 0, uoff = 0, nu = 0, need_all = 0, need_ph1 = 0; } flow[2][2];
  int flow_vmax = 0;               // shared-memory vector entries of the flow kernel
  int* d_flow_ctr = nullptr;       // queue head and per-front counters
  int* d_flow_err = nullptr;       // set by a wait that gave up
  // taps of the design-density filter (offsets and weights) for radius tap_radius
  int* d_probe = nullptr;          // counter of the deferred wait self-test (never incremented)
  // fdfd_design_iteration's buffers: fields, adjoint source, overlaps, F, gradient, design eps
  int it_nrhs = 0;
  double2 *d_itx = nullptr, *d_ita = nullptr, *d_itb = nullptr, *d_ito = nullptr;
  double *d_itF = nullptr, *d_itg = nullptr, *d_itepsd = nullptr;
  int2* d_taps = nullptr;
  double* d_tapw = nullptr;
  int ntap = 0;
  double tap_radius = 0;
  int* h_flow_err = nullptr;       // pinned copy
  int flow_grid[3] = {0, 0, 0};    // persistent CTAs [0 = c64, 1 = c128, 2 = c64 with right-hand sides in pairs]

  // coefficients and permittivity
  double2 *d_cxm = nullptr, *d_cxp = nullptr, *d_cym = nullptr, *d_cyp = nullptr;
  double2 *d_sxc = nullptr, *d_syc = nullptr;   // stretch factors at cell centres (the symmetriser)
  double* d_k0dx = nullptr;
  double* d_k0dx2 = nullptr;
  double* d_eps = nullptr;
  bool have_eps = false;

  // factor storage
  float2* d_store32 = nullptr;
  double2* d_store64 = nullptr;
  int* d_perm32 = nullptr;
  int* d_perm64 = nullptr;
  float2* d_inv32 = nullptr;       // triangular inverses of the pivot blocks
  double2* d_inv64 = nullptr;
  float* d_growth = nullptr;
  float* d_growth_max = nullptr;
  int* d_swp = nullptr;            // panel row-swap scratch
  void* d_dblk = nullptr;          // panel steps' diagonal-block factors
  int max_nlarge = 0;              // longest large-front list of any level
  float* h_growth_max = nullptr;   // pinned
  bool valid32 = false, valid64 = false;
  bool sym32 = false;              // the complex FP32 factors are in the symmetric form (L diag(d) L^T of D A)
  bool growth_pending = false;     // growth of the last FP32 factorisation not yet checked
  bool growth_ready = false;       // ... and its pinned copy has landed

  // solve workspace
  int ws_nrhs = 0;
  void* d_vb = nullptr;            // front vectors, sized for double2
  // FGMRES workspace
  int gm_nrhs = 0, gm_m = 0;
  double2 *d_V = nullptr, *d_Z = nullptr, *d_r = nullptr, *d_w = nullptr;
  double2 *d_h = nullptr, *d_h2 = nullptr, *d_hn = nullptr, *d_bd = nullptr;
  double2 *d_H = nullptr, *d_cs = nullptr, *d_sn = nullptr, *d_g = nullptr, *d_ycoef = nullptr;
  double2* d_partial = nullptr;
  double *d_vscale = nullptr, *d_resid = nullptr, *d_bnorm = nullptr;
  int *d_active = nullptr, *d_nj = nullptr;
  int* d_gcnt = nullptr;           // per-system counters of the Arnoldi passes (zero between launches)
  int* h_active = nullptr;          // pinned
  int* h_nj = nullptr;              // pinned: Krylov vectors each system used in the last cycle
  double* h_resid = nullptr;        // pinned

  // per-kernel profile (CUDA events around every launch when enabled)
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct ProfRec { int kind; size_t e0, e1; double flops, bytes; };
  std::vector<ProfRec> prof_recs;

  // counters
  long long sf = 0, nf = 0, bs = 0, sweeps = 0, fallbacks = 0, repivots = 0;
  long long last_iters = 0;
  long long gm_expect[2] = {1, 1};  // FGMRES iterations the previous solve needed [transpose]
  double last_resid = 0;
  double last_growth = 0;
};

namespace {

fdfd_status fail(fdfd_ctx* c, fdfd_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

#define CK(expr)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? FDFD_ERR_OOM : FDFD_ERR_CUDA,    \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

#define CKS(expr)                              \
  do {                                         \
    fdfd_status s_ = (expr);                   \
    if (s_ != FDFD_OK) return s_;              \
  } while (0)

void free_ptr(void* p) {
  if (p) cudaFree(p);
}

enum ProfKind { PK_BUILD = 0, PK_LU_SMALL, PK_LU_STEP, PK_LU_PANEL, PK_LU_TRSM, PK_LU_GEMM, PK_LU_SCHUR, PK_LU_INV,
                PK_TC_PACK, PK_LU_SCHUR_TC, PK_TC_SUM, PK_LU_TRSM_TC,
                PK_SWEEP_L, PK_SWEEP_U, PK_SWEEP_UT, PK_SWEEP_LT, PK_SWEEP_RECT, PK_STENCIL, PK_DOT, PK_AXPY,
                PK_ARNOLDI, PK_OTHER, PK_COUNT };
const char* const kProfNames[PK_COUNT] = {"front_build", "lu_small", "lu_step", "lu_panel", "lu_trsm", "lu_gemm",
                                          "lu_schur", "lu_inv", "lu_schur_pack", "lu_schur_tc", "lu_schur_sum",
                                          "lu_trsm_tc",
                                          "sweep_L", "sweep_U", "sweep_Ut", "sweep_Lt", "sweep_rect", "stencil_f64",
                                          "gmres_dot", "gmres_axpy", "gmres_arnoldi", "other"};

size_t prof_event(fdfd_ctx* c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return (size_t)-1;
    c->ev_pool.push_back(e);
  }
  cudaEventRecord(c->ev_pool[c->ev_used], c->stream);
  return c->ev_used++;
}

// Brackets one kernel launch with events when profiling is on; flops and bytes
// are the launch's algorithmic work (what the method must do, not what ran).
struct Prof {
  fdfd_ctx* c;
  int kind;
  double flops, bytes;
  size_t e0 = (size_t)-1;
  Prof(fdfd_ctx* ctx, int k, double f, double b) : c(ctx), kind(k), flops(f), bytes(b) {
    if (c->prof_on) e0 = prof_event(c);
  }
  ~Prof() {
    if (c->prof_on && e0 != (size_t)-1) {
      size_t e1 = prof_event(c);
      if (e1 != (size_t)-1) c->prof_recs.push_back({kind, e0, e1, flops, bytes});
    }
  }
};

void free_plan_device(fdfd_ctx* c) {
  free_ptr(c->d_fronts); free_ptr(c->d_children); free_ptr(c->d_idx); free_ptr(c->d_inv);
  free_ptr(c->d_orig_ptr); free_ptr(c->d_orig_col); free_ptr(c->d_orig_code); free_ptr(c->d_lists);
  c->d_fronts = nullptr; c->d_children = c->d_idx = c->d_inv = c->d_orig_ptr = c->d_orig_col = nullptr;
  c->d_orig_code = c->d_lists = nullptr;
  free_ptr(c->d_tcf); free_ptr(c->d_tct); free_ptr(c->d_tcws); free_ptr(c->d_tcpart); free_ptr(c->d_pivonly);
  c->d_tcf = nullptr; c->d_tct = nullptr; c->d_tcws = nullptr; c->d_tcpart = nullptr; c->d_pivonly = nullptr;
  c->tc_ws_stride = c->tc_part_stride = 0;
  c->uploaded = false;
}

void free_factor(fdfd_ctx* c) {
  free_ptr(c->d_store32); free_ptr(c->d_store64); free_ptr(c->d_perm32); free_ptr(c->d_perm64);
  free_ptr(c->d_inv32); free_ptr(c->d_inv64);
  c->d_inv32 = nullptr; c->d_inv64 = nullptr;
  free_ptr(c->d_growth);
  free_ptr(c->d_swp);
  c->d_swp = nullptr;
  free_ptr(c->d_dblk);
  c->d_dblk = nullptr;
  c->d_store32 = nullptr; c->d_store64 = nullptr; c->d_perm32 = c->d_perm64 = nullptr; c->d_growth = nullptr;
  c->valid32 = c->valid64 = false;
}

// Captured graphs bake in buffer addresses and plan lists: drop them whenever
// either changes.
void drop_graphs(fdfd_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

void free_ws(fdfd_ctx* c) {
  drop_graphs(c);
  free_ptr(c->d_vb); free_ptr(c->d_flow_ctr);
  c->d_vb = nullptr;
  c->d_flow_ctr = nullptr;
  c->ws_nrhs = 0;
}

void free_gm(fdfd_ctx* c) {
  void* ps[] = {c->d_V, c->d_Z, c->d_r, c->d_w, c->d_h, c->d_h2, c->d_hn, c->d_bd, c->d_H, c->d_cs,
                c->d_sn, c->d_g, c->d_ycoef, c->d_partial, c->d_vscale, c->d_resid, c->d_bnorm,
                c->d_active, c->d_nj, c->d_gcnt};
  for (void* p : ps) free_ptr(p);
  c->d_V = c->d_Z = c->d_r = c->d_w = c->d_h = c->d_h2 = c->d_hn = c->d_bd = nullptr;
  c->d_H = c->d_cs = c->d_sn = c->d_g = c->d_ycoef = c->d_partial = nullptr;
  c->d_vscale = c->d_resid = c->d_bnorm = nullptr;
  c->d_active = c->d_nj = c->d_gcnt = nullptr;
  c->gm_nrhs = c->gm_m = 0;
}

long long n_cells(const fdfd_ctx* c) { return (long long)c->nx * c->ny; }

// Host symbolic phase (no device work).
fdfd_status analyze_host(fdfd_ctx* ctx) {
  std::string e = build_plan(ctx->nx, ctx->ny, ctx->box.x0, ctx->box.y0, ctx->box.w, ctx->box.h,
                             ctx->opt.leaf_area, &ctx->plan);
  if (!e.empty()) return fail(ctx, FDFD_ERR_ARG, "symbolic phase: " + e);
  for (const auto& d : ctx->plan.fronts)
    if (d.nchild > 2) return fail(ctx, FDFD_ERR_ARG, "symbolic phase: front with more than two children");
  ctx->analyzed = true;
  ctx->sf += 1;
  return FDFD_OK;
}

template <typename P>
fdfd_status upload(fdfd_ctx* ctx, P** dst, const std::vector<P>& v) {
  CK(dalloc(dst, v.size() * sizeof(P)));
  if (!v.empty())
    CK(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(P), cudaMemcpyHostToDevice, ctx->stream));
  return FDFD_OK;
}

// Uploads the plan and builds the per-level launch lists.  The host vectors
// are kept alive by the context until the next upload, so the asynchronous
// copies may still be in flight when this returns.
fdfd_status upload_plan(fdfd_ctx* ctx) {
  drop_graphs(ctx);
  if (ctx->uploaded) CK(cudaStreamSynchronize(ctx->stream));   // old plan may still be in use
  free_plan_device(ctx);
  const Plan& p = ctx->plan;
  CKS(upload(ctx, &ctx->d_fronts, p.fronts));
  CKS(upload(ctx, &ctx->d_children, p.children));
  CKS(upload(ctx, &ctx->d_idx, p.idx));
  CKS(upload(ctx, &ctx->d_inv, p.inv));
  CKS(upload(ctx, &ctx->d_orig_ptr, p.orig_ptr));
  CKS(upload(ctx, &ctx->d_orig_col, p.orig_col));
  CKS(upload(ctx, &ctx->d_orig_code, p.orig_code));
  std::vector<int> lists;
  std::vector<TcFront> tcf;
  std::vector<int4> tct;
  std::vector<unsigned char> pivonly(2 * p.fronts.size(), 0);
  long long tc_ws = 0, tc_part = 0;
  const int planes = ctx->opt.tensor_form;   // form of the tensor-core operands (0 = off)
  int min_tiles = ctx->opt.tensor_min_tiles;
  if (min_tiles == 0) {   // one wave: one tile per SM
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&min_tiles, cudaDevAttrMultiProcessorCount, dev));
  }
  const int L = p.n_levels;
  for (int form = 0; form < 3; ++form) {
    // form 2 (the symmetric form) has the c64 front-size classes and, for now, SIMT update matrices
    const int prec = form == 1 ? 1 : 0;
    const int small_n = lu_small_max_n(prec == 0 ? 8 : 16);
    for (int design = 0; design < 2; ++design) {
      std::vector<LevelList>& out = design ? ctx->lv_design[form] : ctx->lv_full[form];
      out.assign(L, LevelList{});
      for (int l = 0; l < L; ++l) {
        LevelList& ll = out[l];
        std::vector<int> fl;
        for (int f : p.level_fronts[l])
          if (!design || p.fronts[f].design) fl.push_back(f);
        ll.task_off = (int)lists.size();   // build tasks: large fronts only (small ones assemble in their LU)
        for (int f : fl)
          if (p.fronts[f].n > small_n)
            for (int r0 = 0; r0 < p.fronts[f].n; r0 += 8) { lists.push_back(f); lists.push_back(r0); ll.ntasks++; }
        // small fronts in one launch per size class
        for (int c = 0, lo = 0; c < kSmallClasses; lo = lu_small_class_n(c), ++c) {
          const int hi = std::min(small_n, lu_small_class_n(c));
          ll.small_off[c] = (int)lists.size();
          for (int f : fl)
            if (p.fronts[f].n > lo && p.fronts[f].n <= hi) {
              lists.push_back(f); ll.nsmall[c]++; ll.nmax_small[c] = std::max(ll.nmax_small[c], p.fronts[f].n);
            }
        }
        ll.large_off = (int)lists.size();
        for (int f : fl)
          if (p.fronts[f].n > small_n) {
            lists.push_back(f); ll.nlarge++;
            ll.nmax_large = std::max(ll.nmax_large, p.fronts[f].n);
            ll.kmax_large = std::max(ll.kmax_large, p.fronts[f].k);
            ll.mmax_large = std::max(ll.mmax_large, p.fronts[f].m);
          }
        ctx->max_nlarge = std::max(ctx->max_nlarge, ll.nlarge);
        // update matrices: complex64 fronts with m >= tensor_min_m on the tensor cores, the rest SIMT
        auto eligible = [&](const FrontDesc& d) {
          return form != 1 && planes > 0 && d.n > small_n && d.m >= ctx->opt.tensor_min_m && d.k > 0;
        };
        // output tiles of a front: all of them, or for the symmetric form the lower ones
        auto tiles_of = [&](long long t) { return form == 2 ? t * (t + 1) / 2 : t * t; };
        // output tiles of the level over all wavelengths; when they fill less than a wave,
        // each tile's contraction is split over several CTAs; the level goes to the
        // tensor cores when the split tiles fill half a wave at least
        long long level_tiles = 0;
        for (int f : fl)
          if (eligible(p.fronts[f])) {
            const long long t = (p.fronts[f].m + kTcRows - 1) / kTcRows;
            level_tiles += tiles_of(t);
          }
        level_tiles *= ctx->n_omega;
        auto splits_of = [&](const FrontDesc& d) {
          return tc_splits(level_tiles, (d.k + kTcPivots - 1) / kTcPivots, min_tiles);
        };
        long long level_ctas = 0;
        for (int f : fl)
          if (eligible(p.fronts[f])) {
            const long long t = (p.fronts[f].m + kTcRows - 1) / kTcRows;
            level_ctas += tiles_of(t) * splits_of(p.fronts[f]) * ctx->n_omega;
          }
        const bool level_tc = level_tiles > 0 && 2 * level_ctas >= min_tiles;
        auto on_tc = [&](const FrontDesc& d) { return level_tc && eligible(d); };
        ll.simt_off = (int)lists.size();
        for (int f : fl)
          if (p.fronts[f].n > small_n && !on_tc(p.fronts[f]) && p.fronts[f].m > 0) {
            lists.push_back(f); ll.nsimt++; ll.mmax_simt = std::max(ll.mmax_simt, p.fronts[f].m);
          }
        ll.tcf_off = (int)tcf.size();
        long long wsb = 0, pfl = 0;
        for (int f : fl)
          if (on_tc(p.fronts[f])) {
            const FrontDesc& d = p.fronts[f];
            TcFront r;
            r.f = f;
            r.mode = 0;
            r.Mt = (d.m + kTcRows - 1) / kTcRows;
            r.Nt = (d.m + kTcCols - 1) / kTcCols;
            r.Kt = (d.k + kTcPivots - 1) / kTcPivots;
            r.nsplit = splits_of(d);
            r.aoff = wsb;
            wsb += (long long)r.Mt * r.Kt * tc_tile_bytes_a(planes);
            r.boff = wsb;
            wsb += (long long)r.Nt * r.Kt * tc_tile_bytes_b(planes);
            r.poff = pfl;
            if (r.nsplit > 1) pfl += (long long)r.Mt * r.Nt * r.nsplit * kTcPartFloats;
            tcf.push_back(r);
          }
        ll.ntcf = (int)tcf.size() - ll.tcf_off;
        tc_ws = std::max(tc_ws, wsb);
        tc_part = std::max(tc_part, pfl);
        ll.tcp_off = (int)tct.size();
        for (int sl = 0; sl < ll.ntcf; ++sl) {
          const TcFront& r = tcf[ll.tcf_off + sl];
          for (int mt = 0; mt < r.Mt; ++mt)
            for (int kt = 0; kt < r.Kt; ++kt) tct.push_back(make_int4(sl, 0, mt, kt));
          for (int nt = 0; nt < r.Nt; ++nt)
            for (int kt = 0; kt < r.Kt; ++kt) tct.push_back(make_int4(sl, 1, nt, kt));
        }
        ll.ntcp = (int)tct.size() - ll.tcp_off;
        ll.tct_off = (int)tct.size();
        for (int sl = 0; sl < ll.ntcf; ++sl) {
          const TcFront& r = tcf[ll.tcf_off + sl];
          for (int mt = 0; mt < r.Mt; ++mt)
            for (int nt = 0; nt < r.Nt; ++nt)
              if (form != 2 || nt <= mt)
                for (int sp = 0; sp < r.nsplit; ++sp) tct.push_back(make_int4(sl, mt, nt, sp));
        }
        ll.ntct = (int)tct.size() - ll.tct_off;
        ll.tcs_off = (int)tct.size();
        for (int sl = 0; sl < ll.ntcf; ++sl) {
          const TcFront& r = tcf[ll.tcf_off + sl];
          if (r.nsplit > 1)
            for (int mt = 0; mt < r.Mt; ++mt)
              for (int nt = 0; nt < r.Nt; ++nt)
                if (form != 2 || nt <= mt)
                  for (int r0 = 0; r0 < kTcRows; r0 += 16) tct.push_back(make_int4(sl, mt, nt, r0));
        }
        ll.ntcs = (int)tct.size() - ll.tcs_off;
        if (form == 0) {
          // L21 = F21 U11^-1 and U12 = L11^-1 (P F12) of the same fronts, before their
          // update matrices (the workspace is free then: its planes start at 0)
          ll.tqf_off = (int)tcf.size();
          long long wsq = 0;
          for (int f : fl)
            if (on_tc(p.fronts[f])) {
              const FrontDesc& d = p.fronts[f];
              pivonly[(size_t)design * p.fronts.size() + f] = 1;
              const int tk = (d.k + kTcRows - 1) / kTcRows, tm = (d.m + kTcRows - 1) / kTcRows;
              for (int mode = 1; mode <= 2; ++mode) {
                TcFront r;
                r.f = f;
                r.mode = mode;
                r.Mt = mode == 1 ? tm : tk;
                r.Nt = mode == 1 ? tk : tm;
                r.Kt = (d.k + kTcPivots - 1) / kTcPivots;
                r.nsplit = 1;
                r.aoff = wsq;
                wsq += (long long)r.Mt * r.Kt * tc_tile_bytes_a(planes);
                r.boff = wsq;
                wsq += (long long)r.Nt * r.Kt * tc_tile_bytes_b(planes);
                r.poff = 0;
                tcf.push_back(r);
              }
            }
          ll.ntqf = (int)tcf.size() - ll.tqf_off;
          tc_ws = std::max(tc_ws, wsq);
          // pack tasks: the triangular operand's tiles only up to its last nonzero k-tile
          constexpr int kTri = kTcRows / kTcPivots;   // k-tiles per 128 pivots
          ll.tqp_off = (int)tct.size();
          for (int sl = 0; sl < ll.ntqf; ++sl) {
            const TcFront& r = tcf[ll.tqf_off + sl];
            for (int mt = 0; mt < r.Mt; ++mt)
              for (int kt = 0; kt < (r.mode == 2 ? std::min(r.Kt, kTri * (mt + 1)) : r.Kt); ++kt)
                tct.push_back(make_int4(sl, 0, mt, kt));
            for (int nt = 0; nt < r.Nt; ++nt)
              for (int kt = 0; kt < (r.mode == 1 ? std::min(r.Kt, kTri * (nt + 1)) : r.Kt); ++kt)
                tct.push_back(make_int4(sl, 1, nt, kt));
          }
          ll.ntqp = (int)tct.size() - ll.tqp_off;
          ll.tqt_off = (int)tct.size();
          for (int sl = 0; sl < ll.ntqf; ++sl) {
            const TcFront& r = tcf[ll.tqf_off + sl];
            for (int mt = 0; mt < r.Mt; ++mt)
              for (int nt = 0; nt < r.Nt; ++nt) tct.push_back(make_int4(sl, mt, nt, 0));
          }
          ll.ntqt = (int)tct.size() - ll.tqt_off;
        }
        if (lists.size() % 2) lists.push_back(0);   // keep int2 task arrays 8-byte aligned
      }
    }
  }
  ctx->lv_solve.assign(L, SolveList{});
  // task lists (front, first row/column): [0] row tasks, [1] column tasks.
  // A small or medium front is one whole-front task (front | bit 31; y = 0 for
  // one warp, 1 for one CTA); a large front is split into row or column tasks
  // in both directions.
  const int whole_n = flow_whole_max_n();   // fronts swept whole by one warp
  const int cta_n = flow_cta_max_n();       // ... or by one CTA
  auto small = [cta_n](const FrontDesc& d) { return d.n <= cta_n; };
  // Row tasks of a level with many of them take two rows per warp (kSweepTaskTall,
  // flagged in the task word): fewer, longer tasks with more loads in flight.
  int sweep_nsm = 0;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sweep_nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sweep_nsm = 1;
  }
  auto tall_level = [&](int l) {
    long long cnt = 0;
    for (int f : p.level_fronts[l]) {
      const FrontDesc& d = p.fronts[f];
      if (small(d)) continue;
      cnt += (d.k + 7) / 8 + (d.m + 7) / 8;
    }
    return cnt * ctx->n_omega >= 16LL * sweep_nsm;
  };
  auto add_tasks = [&](TaskList& tl, int l, bool rect, bool over_m, int step) {
    if (lists.size() % 2) lists.push_back(0);   // int2 task arrays stay 8-byte aligned
    tl.off = (int)lists.size();
    const bool tall = step == sweep_row_block() && tall_level(l);
    const int st = tall ? 2 * step : step;
    const unsigned flag = tall ? (unsigned)kSweepTaskTall : 0u;
    for (int f : p.level_fronts[l]) {
      const FrontDesc& d = p.fronts[f];
      if (small(d)) {
        if (!rect) {
          lists.push_back((int)(0x80000000u | (unsigned)f));
          lists.push_back(d.n <= whole_n ? 0 : 1);
          tl.n++;
        }
        continue;
      }
      if (rect && d.m == 0) continue;
      const int len = over_m ? d.m : d.k;
      for (int s0 = 0; s0 < len; s0 += st) { lists.push_back((int)(flag | (unsigned)f)); lists.push_back(s0); tl.n++; }
    }
  };
  const int steps[2] = {sweep_row_block(), sweep_col_block()};
  for (int l = 0; l < L; ++l) {
    SolveList& sl = ctx->lv_solve[l];
    for (int t = 0; t < 2; ++t) {
      add_tasks(sl.tri[t], l, false, false, steps[t]);     // inverse blocks (whole small fronts)
      add_tasks(sl.rect_m[t], l, true, true, steps[t]);    // off-diagonal block, over boundary rows/cols
      add_tasks(sl.rect_k[t], l, true, false, steps[t]);   // off-diagonal block, over pivot rows/cols
    }
    for (int f : p.level_fronts[l]) {
      const FrontDesc& d = p.fronts[f];
      sl.kmax = std::max(sl.kmax, small(d) ? d.n + d.k : d.k);   // shared-memory vectors of the tri launch
      if (!small(d) && d.m > 0) {
        sl.mbig = std::max(sl.mbig, d.m);
        sl.kbig = std::max(sl.kbig, d.k);
      }
    }
    ctx->flow_vmax = std::max({ctx->flow_vmax, sl.kmax, sl.kbig, sl.mbig});
  }
  // Dataflow queues: the same tasks as the level lists, in dependency order,
  // off-diagonal tasks tagged with bit 30; per level the whole small fronts
  // first, in units of up to 8 (one warp each), then the whole medium fronts
  // (one CTA each), then the large fronts' tasks (one unit each) in phase
  // order; per-front task counts beside them.
  const int nf = (int)p.fronts.size();
  for (int t = 0; t < 2; ++t) {
    for (int dir = 0; dir < 2; ++dir) {
      auto& fl = ctx->flow[t][dir];
      fl = fdfd_ctx::FlowList{};                 // the plan may be uploaded again (plain mode)
      std::vector<int> all(nf, 0), ph1(nf, 0);
      std::vector<int> tasks, units;
      auto put_unit = [&](int first, int y) { units.push_back(first); units.push_back(y); };
      auto put_whole = [&](const SolveList& sl) {
        int first = -1, cnt = 0;
        for (int i = 0; i < sl.tri[t].n; ++i) {
          const int code = lists[sl.tri[t].off + 2 * i];
          if (code >= 0 || lists[sl.tri[t].off + 2 * i + 1] != 0) continue;   // not a small front
          const int f = code & kSweepFrontMask;
          if (cnt == 0) first = (int)tasks.size() / 2;
          tasks.push_back(code); tasks.push_back(0);
          all[f]++;
          if (++cnt == 8) { put_unit(first, (int)(0x80000000u | 8u)); cnt = 0; }
        }
        if (cnt) put_unit(first, (int)(0x80000000u | (unsigned)cnt));
        for (int i = 0; i < sl.tri[t].n; ++i) {               // whole medium fronts, one unit each
          const int code = lists[sl.tri[t].off + 2 * i];
          if (code >= 0 || lists[sl.tri[t].off + 2 * i + 1] != 1) continue;
          put_unit((int)tasks.size() / 2, 1);
          tasks.push_back(code); tasks.push_back(1);
          all[code & kSweepFrontMask]++;
        }
      };
      auto put_tri = [&](const SolveList& sl) {
        for (int i = 0; i < sl.tri[t].n; ++i) {
          const int code = lists[sl.tri[t].off + 2 * i], s0 = lists[sl.tri[t].off + 2 * i + 1];
          if (code < 0) continue;                            // whole small front
          put_unit((int)tasks.size() / 2, 1);
          tasks.push_back(code); tasks.push_back(s0);
          all[code & kSweepFrontMask]++;
          if (dir == 0) ph1[code & kSweepFrontMask]++;
        }
      };
      auto put_rect = [&](const TaskList& tl) {
        for (int i = 0; i < tl.n; ++i) {
          const int code = lists[tl.off + 2 * i], s0 = lists[tl.off + 2 * i + 1];
          const int f = code & kSweepFrontMask;
          put_unit((int)tasks.size() / 2, 1);
          tasks.push_back((int)(0x40000000u | (unsigned)code)); tasks.push_back(s0);
          all[f]++;
          if (dir == 1) ph1[f]++;
        }
      };
      if (dir == 0) {
        for (int l = 0; l < L; ++l) {
          put_whole(ctx->lv_solve[l]); put_tri(ctx->lv_solve[l]); put_rect(ctx->lv_solve[l].rect_m[t]);
        }
      } else {
        for (int l = L - 1; l >= 0; --l) {
          put_rect(ctx->lv_solve[l].rect_k[t]); put_whole(ctx->lv_solve[l]); put_tri(ctx->lv_solve[l]);
        }
      }
      if (lists.size() % 2) lists.push_back(0);
      fl.off = (int)lists.size();
      fl.n = (int)tasks.size() / 2;
      lists.insert(lists.end(), tasks.begin(), tasks.end());
      fl.uoff = (int)lists.size();
      fl.nu = (int)units.size() / 2;
      lists.insert(lists.end(), units.begin(), units.end());
      fl.need_all = (int)lists.size();
      lists.insert(lists.end(), all.begin(), all.end());
      fl.need_ph1 = (int)lists.size();
      lists.insert(lists.end(), ph1.begin(), ph1.end());
    }
  }
  ctx->h_lists.swap(lists);
  CKS(upload(ctx, &ctx->d_lists, ctx->h_lists));
  ctx->h_tcf.swap(tcf);
  ctx->h_tct.swap(tct);
  if (!ctx->h_tcf.empty()) {
    CKS(upload(ctx, &ctx->d_tcf, ctx->h_tcf));
    CKS(upload(ctx, &ctx->d_tct, ctx->h_tct));
    ctx->h_pivonly.swap(pivonly);
    CKS(upload(ctx, &ctx->d_pivonly, ctx->h_pivonly));
    ctx->tc_ws_stride = tc_ws;
    CK(dalloc(&ctx->d_tcws, (size_t)tc_ws * ctx->n_omega));
    ctx->tc_part_stride = std::max<long long>(tc_part, 4);
    CK(dalloc(&ctx->d_tcpart, sizeof(float) * (size_t)ctx->tc_part_stride * ctx->n_omega));
  }
  ctx->uploaded = true;
  return FDFD_OK;
}

// Device runtime: kernel attributes, stencil coefficient tables, eps buffer.
fdfd_status ensure_runtime(fdfd_ctx* ctx) {
  if (ctx->device < 0) {
    CK(cudaGetDevice(&ctx->device));
    CK(factor_init_attributes());
    CK(tc_init_attributes());
    CK(solve_init_attributes());
    CK(dalloc(&ctx->d_cxm, sizeof(double2) * ctx->n_omega * ctx->nx));
    CK(dalloc(&ctx->d_cxp, sizeof(double2) * ctx->n_omega * ctx->nx));
    CK(dalloc(&ctx->d_cym, sizeof(double2) * ctx->n_omega * ctx->ny));
    CK(dalloc(&ctx->d_cyp, sizeof(double2) * ctx->n_omega * ctx->ny));
    CK(dalloc(&ctx->d_sxc, sizeof(double2) * ctx->n_omega * ctx->nx));
    CK(dalloc(&ctx->d_syc, sizeof(double2) * ctx->n_omega * ctx->ny));
    CK(dalloc(&ctx->d_k0dx, sizeof(double) * ctx->n_omega));
    CK(dalloc(&ctx->d_k0dx2, sizeof(double) * ctx->n_omega));
    CK(dalloc(&ctx->d_eps, sizeof(double) * n_cells(ctx)));
    CK(dalloc(&ctx->d_growth_max, sizeof(float)));
    CK(cudaMallocHost((void**)&ctx->h_growth_max, sizeof(float)));
    CK(dalloc(&ctx->d_flow_err, sizeof(int)));
    CK(cudaMemsetAsync(ctx->d_flow_err, 0, sizeof(int), ctx->stream));
    CK(cudaMallocHost((void**)&ctx->h_flow_err, sizeof(int)));
    *ctx->h_flow_err = 0;
    CK(cudaMemcpyAsync(ctx->d_k0dx, ctx->k0dx.data(), sizeof(double) * ctx->n_omega, cudaMemcpyHostToDevice,
                       ctx->stream));
    launch_coef(ctx->d_cxm, ctx->d_cxp, ctx->d_cym, ctx->d_cyp, ctx->d_k0dx2, ctx->d_sxc, ctx->d_syc,
                ctx->d_k0dx, ctx->n_omega,
                ctx->nx, ctx->ny, ctx->pml.npml_x, ctx->pml.npml_y, ctx->pml.ln_R, ctx->pml.order, ctx->stream);
    CK(cudaGetLastError());
  }
  return FDFD_OK;
}

// Runtime plus the symbolic plan on the device (analysed on first use).
fdfd_status ensure_device(fdfd_ctx* ctx) {
  CKS(ensure_runtime(ctx));
  if (!ctx->analyzed) CKS(analyze_host(ctx));
  if (!ctx->uploaded) CKS(upload_plan(ctx));
  return FDFD_OK;
}

DevPlan dev_plan(const fdfd_ctx* c) {
  DevPlan P;
  P.fronts = c->d_fronts; P.children = c->d_children; P.idx = c->d_idx; P.inv = c->d_inv;
  P.orig_ptr = c->d_orig_ptr; P.orig_col = c->d_orig_col; P.orig_code = c->d_orig_code;
  P.nx = c->nx; P.ny = c->ny;
  return P;
}

DevCoef dev_coef(const fdfd_ctx* c) {
  DevCoef C;
  C.cxm = c->d_cxm; C.cxp = c->d_cxp; C.cym = c->d_cym; C.cyp = c->d_cyp;
  C.k0dx2 = c->d_k0dx2; C.eps = c->d_eps; C.nx = c->nx; C.ny = c->ny;
  C.sxc = c->d_sxc; C.syc = c->d_syc;
  return C;
}

fdfd_status ensure_store(fdfd_ctx* ctx, int prec) {
  const Plan& p = ctx->plan;
  const size_t nfr = p.fronts.size();
  if (!ctx->d_growth) CK(dalloc(&ctx->d_growth, sizeof(float) * nfr * ctx->n_omega));
  if (!ctx->d_swp)
    CK(dalloc(&ctx->d_swp, sizeof(int) * (size_t)kSwapScratchInts * std::max(1, ctx->max_nlarge) * ctx->n_omega));
  if (!ctx->d_dblk)
    CK(dalloc(reinterpret_cast<char**>(&ctx->d_dblk),
              sizeof(double2) * (size_t)kDiagBlkElems * std::max(1, ctx->max_nlarge) * ctx->n_omega));
  if (prec == 0 && !ctx->d_store32) {
    CK(dalloc(&ctx->d_store32, sizeof(float2) * (size_t)p.store_total * ctx->n_omega));
    CK(dalloc(&ctx->d_perm32, sizeof(int) * (size_t)std::max(1, p.perm_total) * ctx->n_omega));
    CK(dalloc(&ctx->d_inv32, sizeof(float2) * (size_t)p.inv_total * ctx->n_omega));
  }
  if (prec == 1 && !ctx->d_store64) {
    CK(dalloc(&ctx->d_store64, sizeof(double2) * (size_t)p.store_total * ctx->n_omega));
    CK(dalloc(&ctx->d_perm64, sizeof(int) * (size_t)std::max(1, p.perm_total) * ctx->n_omega));
    CK(dalloc(&ctx->d_inv64, sizeof(double2) * (size_t)p.inv_total * ctx->n_omega));
  }
  return FDFD_OK;
}

// Level-by-level numeric factorisation of the listed fronts, for wavelengths [w0, w0+nw).
template <typename T>
fdfd_status factor_levels(fdfd_ctx* ctx, bool design_only, int w0 = 0, int nw = -1, bool sym = false) {
  const int prec = sizeof(T) == 8 ? 0 : 1;
  sym = sym && prec == 0;
  CKS(ensure_store(ctx, prec));
  const Plan& p = ctx->plan;
  FactorLaunch fa;
  fa.P = dev_plan(ctx);
  fa.C = dev_coef(ctx);
  fa.store = prec == 0 ? (void*)ctx->d_store32 : (void*)ctx->d_store64;
  fa.store_stride = p.store_total;
  fa.perm = prec == 0 ? ctx->d_perm32 : ctx->d_perm64;
  fa.perm_stride = std::max(1, p.perm_total);
  fa.growth = ctx->d_growth;
  fa.n_fronts = (int)p.fronts.size();
  fa.n_omega = nw < 0 ? ctx->n_omega : nw;
  fa.w0 = w0;
  fa.swp = ctx->d_swp;
  fa.dblk = ctx->d_dblk;
  fa.swp_stride = std::max(1, ctx->max_nlarge);
  fa.istore = prec == 0 ? (void*)ctx->d_inv32 : (void*)ctx->d_inv64;
  fa.istore_stride = p.inv_total;
  fa.sym = sym ? 1 : 0;
  const int form = sym ? 2 : prec;
  // complex64 LU with block-local pivoting: the fronts whose update matrices go to the
  // tensor cores take their L21 and U12 from there too (panel steps over the pivot block)
  const bool trsm_tc = prec == 0 && !sym && ctx->opt.pivoting == 1 && ctx->opt.tensor_offdiag == 1 &&
                       ctx->d_pivonly != nullptr;
  fa.pivonly = trsm_tc ? ctx->d_pivonly + (design_only ? p.fronts.size() : 0) : nullptr;
  const std::vector<LevelList>& lv = design_only ? ctx->lv_design[form] : ctx->lv_full[form];
  const int nb = lu_panel_width(sizeof(T));
  cudaStream_t s = ctx->stream;
  // inverse folds beside the panel steps (on the main stream while profiling,
  // so that each launch is timed on its own)
  cudaStream_t si = (ctx->prof_on || !ctx->istream) ? s : ctx->istream;
  bool forked = false;
  const double es = sizeof(T), nwd = fa.n_omega;
  const int* hl = ctx->h_lists.data();
  for (int l = 0; l < p.n_levels; ++l) {
    const LevelList& ll = lv[l];
    {
      double by = 0;
      if (ctx->prof_on)
        for (int t = 0; t < ll.ntasks; ++t) {
          const FrontDesc& d = p.fronts[hl[ll.task_off + 2 * t]];
          const int rows = std::min(8, d.n - hl[ll.task_off + 2 * t + 1]);
          by += es * rows * d.n;                                   // front rows written
          for (int ci = 0; ci < d.nchild; ++ci) {                  // child update rows read
            const FrontDesc& c = p.fronts[p.children[d.child0 + ci]];
            by += es * (double)c.m * c.m * rows / std::max(1, d.n);
          }
        }
      Prof pr(ctx, PK_BUILD, 0, by * nwd);
      launch_build<T>(fa, reinterpret_cast<const int2*>(ctx->d_lists + ll.task_off), ll.ntasks, s);
    }
    {
      double fl = 0, by = 0;
      if (ctx->prof_on)
        for (int c = 0; c < kSmallClasses; ++c)
          for (int t = 0; t < ll.nsmall[c]; ++t) {
            const FrontDesc& d = p.fronts[hl[ll.small_off[c] + t]];
            for (int j = 0; j < d.k; ++j) fl += 8.0 * (double)(d.n - j - 1) * (d.n - j - 1);
            by += 2.0 * es * d.n * d.n;
          }
      if (sym) fl *= 0.5;   // lower triangles only: (n-j-1)(n-j)/2 per pivot, up to the diagonal terms
      Prof pr(ctx, PK_LU_SMALL, fl * nwd, by * nwd);
      for (int c = 0; c < kSmallClasses; ++c)
        launch_lu_small<T>(fa, ctx->d_lists + ll.small_off[c], ll.nsmall[c], ll.nmax_small[c], s);
    }
    const bool local_piv = ctx->opt.pivoting == 1 || sym;   // the symmetric form uses the one-launch panel step
    for (int j0 = 0; j0 < ll.kmax_large; j0 += nb) {
      const int* fl = ctx->d_lists + ll.large_off;
      double pf = 0, pb = 0, lf = 0, lb = 0, tf = 0, tb = 0, gf = 0, gb = 0;
      if (ctx->prof_on)
        for (int t = 0; t < ll.nlarge; ++t) {
          const FrontDesc& d = p.fronts[hl[ll.large_off + t]];
          if (j0 >= d.k) continue;
          const int b = std::min(nb, d.k - j0);
          for (int j = j0; j < j0 + b; ++j) pf += 8.0 * (double)(d.k - j - 1) * (j0 + b - j);
          pb += 2.0 * es * (double)(d.k - j0) * b;
          const double below = ctx->opt.pivoting == 1 ? d.n - j0 - b : d.m;   // rows eliminated against the block
          lf += 8.0 * 0.5 * b * (b + 1.0) * below;
          lb += 2.0 * es * b * below;
          const double rem = d.n - j0 - b;
          const double kr = d.k - j0 - b;                  // pivot columns still to factor
          tf += 8.0 * 0.5 * b * (b - 1) * rem;
          tb += 2.0 * es * b * rem;
          if (sym) {
            // lower triangle of the remaining pivot columns: rows c..n-1 of each column c
            const double cols = kr, lower = cols * (d.n - (j0 + b)) - cols * (cols - 1) / 2;
            gf += 8.0 * b * lower;
            gb += es * (2.0 * lower + 2.0 * rem * b);
          } else {
            gf += 8.0 * b * (rem * kr + kr * d.m);          // pivot-block rows and columns only
            gb += es * (2.0 * (rem * kr + kr * d.m) + 2.0 * rem * b);
          }
        }
      if (local_piv) {
        {
          // block LU and inverses, L columns, U rows and the row permutation of the step in one launch
          Prof pr(ctx, PK_LU_STEP, (pf + lf + tf) * nwd, (pb + lb + tb) * nwd);
          launch_lu_step_local<T>(fa, fl, ll.nlarge, j0, ll.nmax_large, s);
        }
        // block row J of L11^-1 and block column J of U11^-1: products with the
        // inverse so far, then with the block's own inverse
        double vf = 0, vb = 0;
        if (ctx->prof_on)
          for (int t = 0; t < ll.nlarge; ++t) {
            const FrontDesc& d = p.fronts[hl[ll.large_off + t]];
            if (j0 >= d.k) continue;
            const double b = std::min(nb, d.k - j0);
            vf += 8.0 * (sym ? 1.0 : 2.0) * (0.5 * b * (double)j0 * j0 + b * b * j0);
            vb += es * (sym ? 1.0 : 2.0) * (0.5 * (double)j0 * j0 + 2.0 * b * j0);
          }
        if (si != s && j0 > 0) {
          CK(cudaEventRecord(ctx->iev_fork, s));
          CK(cudaStreamWaitEvent(si, ctx->iev_fork, 0));
          forked = true;
        }
        if (j0 > 0) {
          Prof pr(ctx, PK_LU_INV, vf * nwd, vb * nwd);
          launch_lu_inv_fold<T>(fa, fl, ll.nlarge, j0, si);
        }
      } else {
        { Prof pr(ctx, PK_LU_PANEL, pf * nwd, pb * nwd);
          launch_lu_panel<T>(fa, fl, ll.nlarge, j0, nb, ll.kmax_large, s); }
        { Prof pr(ctx, PK_LU_TRSM, lf * nwd, lb * nwd);
          launch_lu_l21<T>(fa, fl, ll.nlarge, j0, nb, ll.mmax_large, ll.nmax_large, 0, s); }
        { Prof pr(ctx, PK_LU_TRSM, tf * nwd, tb * nwd);
          launch_lu_trsm<T>(fa, fl, ll.nlarge, j0, nb, ll.nmax_large, s); }
      }
      { Prof pr(ctx, PK_LU_GEMM, gf * nwd, gb * nwd); launch_lu_gemm<T>(fa, fl, ll.nlarge, j0, nb, ll.nmax_large, s); }
    }
    if (trsm_tc && ll.ntqf > 0) {
      // L21 = F21 U11^-1 and U12 = L11^-1 (P F12) on the tensor cores: the inverse folds of
      // the last panel steps (side stream) must have finished
      if (forked) {
        CK(cudaEventRecord(ctx->iev_join, si));
        CK(cudaStreamWaitEvent(s, ctx->iev_join, 0));
      }
      TcLaunch tq;
      tq.fronts = ctx->d_tcf + ll.tqf_off;
      tq.ws = ctx->d_tcws;
      tq.ws_stride = ctx->tc_ws_stride;
      tq.err = ctx->d_flow_err;
      tq.chunk = kTcChunk;
      tq.part = ctx->d_tcpart;
      tq.part_stride = ctx->tc_part_stride;
      const int planes = ctx->opt.tensor_form;
      double qf = 0, qb = 0, qp = 0;
      if (ctx->prof_on)
        for (int t = 0; t < ll.ntqf; ++t) {
          const TcFront& r = ctx->h_tcf[ll.tqf_off + t];
          const FrontDesc& d = p.fronts[r.f];
          qf += 8.0 * 0.5 * (double)d.k * d.k * d.m;              // a triangular solve's multiply-adds
          qb += es * (2.0 * (double)d.k * d.m + 0.5 * (double)d.k * d.k) +
                (double)r.Kt * r.Mt * r.Nt * 0.5 * (tc_tile_bytes_a(planes) + tc_tile_bytes_b(planes));
          qp += es * ((double)d.k * d.m + 0.5 * (double)d.k * d.k) +
                (double)r.Kt * (r.Mt * tc_tile_bytes_a(planes) + r.Nt * tc_tile_bytes_b(planes));
        }
      {
        Prof pr(ctx, PK_TC_PACK, 0, qp * nwd);
        tq.tasks = ctx->d_tct + ll.tqp_off;
        launch_schur_tc_pack(fa, tq, ll.ntqp, planes, s);
      }
      {
        Prof pr(ctx, PK_LU_TRSM_TC, qf * nwd, qb * nwd);
        tq.tasks = ctx->d_tct + ll.tqt_off;
        launch_schur_tc(fa, tq, ll.ntqt, planes, s);
      }
    }
    if (ll.nsimt > 0) {
      // update matrices of the level's large fronts: S = F22 - L21 U12 (k m^2 complex multiply-adds)
      double sf = 0, sb = 0;
      if (ctx->prof_on)
        for (int t = 0; t < ll.nsimt; ++t) {
          const FrontDesc& d = p.fronts[hl[ll.simt_off + t]];
          if (sym) {
            sf += 8.0 * (double)d.k * d.m * (d.m + 1) / 2;
            sb += es * ((double)d.m * (d.m + 1) + 2.0 * (double)d.k * d.m);
          } else {
            sf += 8.0 * (double)d.k * d.m * d.m;
            sb += es * (2.0 * (double)d.m * d.m + 2.0 * (double)d.k * d.m);
          }
        }
      Prof pr(ctx, PK_LU_SCHUR, sf * nwd, sb * nwd);
      launch_schur_simt<T>(fa, ctx->d_lists + ll.simt_off, ll.nsimt, ll.mmax_simt, s);
    }
    if (ll.ntct > 0) {
      // the same on the tensor cores: pack L21 / U12 into TF32 planes, then the tiled product
      TcLaunch tl;
      tl.fronts = ctx->d_tcf + ll.tcf_off;
      tl.ws = ctx->d_tcws;
      tl.ws_stride = ctx->tc_ws_stride;
      tl.err = ctx->d_flow_err;
      tl.chunk = kTcChunk;
      tl.part = ctx->d_tcpart;
      tl.part_stride = ctx->tc_part_stride;
      const int planes = ctx->opt.tensor_form;
      double sf = 0, sb = 0, pb = 0;
      if (ctx->prof_on)
        for (int t = 0; t < ll.ntcf; ++t) {
          const TcFront& r = ctx->h_tcf[ll.tcf_off + t];
          const FrontDesc& d = p.fronts[r.f];
          const double tiles = sym ? 0.5 * r.Mt * (r.Mt + 1.0) : (double)r.Mt * r.Nt;
          sf += sym ? 8.0 * (double)d.k * d.m * (d.m + 1) / 2 : 8.0 * (double)d.k * d.m * d.m;
          sb += es * (sym ? 1.0 : 2.0) * (double)d.m * d.m +
                (double)r.Kt * tiles * (tc_tile_bytes_a(planes) + tc_tile_bytes_b(planes));
          pb += es * 2.0 * (double)d.k * d.m +
                (double)r.Kt * (r.Mt * tc_tile_bytes_a(planes) + r.Nt * tc_tile_bytes_b(planes));
        }
      {
        Prof pr(ctx, PK_TC_PACK, 0, pb * nwd);
        tl.tasks = ctx->d_tct + ll.tcp_off;
        launch_schur_tc_pack(fa, tl, ll.ntcp, planes, s);
      }
      {
        Prof pr(ctx, PK_LU_SCHUR_TC, sf * nwd, sb * nwd);
        tl.tasks = ctx->d_tct + ll.tct_off;
        launch_schur_tc(fa, tl, ll.ntct, planes, s);
      }
      if (ll.ntcs > 0) {
        double qb = 0;
        if (ctx->prof_on)
          for (int t = 0; t < ll.ntcf; ++t) {
            const TcFront& r = ctx->h_tcf[ll.tcf_off + t];
            if (r.nsplit > 1) qb += (double)r.Mt * r.Nt * (4.0 * r.nsplit * kTcPartFloats + 2.0 * es * kTcRows * kTcCols);
          }
        Prof pr(ctx, PK_TC_SUM, 0, qb * nwd);
        tl.tasks = ctx->d_tct + ll.tcs_off;
        launch_schur_split_sum(fa, tl, ll.ntcs, s);
      }
    }
    if (ll.nlarge > 0 && !local_piv) {
      // triangular inverses of the level's large fronts (2/3 k^3 complex multiply-adds each);
      // block-local pivoting forms them inside the panel steps instead
      double vf = 0, vb = 0;
      if (ctx->prof_on)
        for (int t = 0; t < ll.nlarge; ++t) {
          const FrontDesc& d = p.fronts[hl[ll.large_off + t]];
          vf += 8.0 * (2.0 / 6.0) * (double)d.k * d.k * d.k;
          vb += es * 2.0 * (double)d.k * d.k;
        }
      Prof pr(ctx, PK_LU_INV, vf * nwd, vb * nwd);
      launch_lu_inv<T>(fa, ctx->d_lists + ll.large_off, ll.nlarge, ll.kmax_large, s);
    }
  }
  if (forked) {
    CK(cudaEventRecord(ctx->iev_join, si));
    CK(cudaStreamWaitEvent(s, ctx->iev_join, 0));
  }
  CK(cudaGetLastError());
  Prof pr_g(ctx, PK_OTHER, 0, 4.0 * p.fronts.size() * ctx->n_omega);
  CK(launch_growth_max(ctx->d_growth, (long long)p.fronts.size() * ctx->n_omega, ctx->d_growth_max, s));
  CK(cudaMemcpyAsync(ctx->h_growth_max, ctx->d_growth_max, sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(ctx->h_flow_err, ctx->d_flow_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  return FDFD_OK;
}

// Sweeps of problems with at least 2^20 unknowns over all wavelengths run the
// flow-kernel variant with six resident CTAs per SM (more loads in flight);
// smaller ones keep four, with more registers per thread for their
// latency-bound tasks.
bool flow_wide(const fdfd_ctx* ctx) { return (long long)ctx->nx * ctx->ny * ctx->n_omega >= (1LL << 20); }

fdfd_status ensure_ws(fdfd_ctx* ctx, int nrhs) {
  if (ctx->ws_nrhs >= nrhs) return FDFD_OK;
  free_ws(ctx);
  const size_t S = (size_t)ctx->n_omega * nrhs;
  CK(dalloc(&ctx->d_vb, sizeof(double2) * S * (size_t)ctx->plan.vec_total));
  CK(dalloc(&ctx->d_flow_ctr, sizeof(int) * (1 + 2 * (size_t)ctx->n_omega * ctx->plan.fronts.size())));
  int nsm = 0;
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  for (int v = 0; v < 3; ++v)
    ctx->flow_grid[v] = nsm * flow_blocks_per_sm(v == 1 ? 16 : 8, std::max(1, ctx->flow_vmax), flow_wide(ctx), v == 2);
  ctx->ws_nrhs = nrhs;
  return FDFD_OK;
}

// Launch description of the sweeps over the cached factors of precision T.
template <typename T>
SolveLaunch solve_launch(const fdfd_ctx* ctx, void* vb, int nrhs, int w0, int nw, int r0, int nr) {
  const int prec = sizeof(T) == 8 ? 0 : 1;
  const Plan& p = ctx->plan;
  SolveLaunch sa;
  sa.P = dev_plan(ctx);
  sa.store = prec == 0 ? (const void*)ctx->d_store32 : (const void*)ctx->d_store64;
  sa.store_stride = p.store_total;
  sa.perm = prec == 0 ? ctx->d_perm32 : ctx->d_perm64;
  sa.perm_stride = std::max(1, p.perm_total);
  sa.istore = prec == 0 ? (const void*)ctx->d_inv32 : (const void*)ctx->d_inv64;
  sa.istore_stride = p.inv_total;
  sa.vb = vb;
  sa.vec_stride = p.vec_total;
  sa.n_omega = nw < 0 ? ctx->n_omega : nw;
  sa.nrhs = nrhs;
  sa.w0 = w0;
  sa.r0 = r0;
  sa.nr = nr < 0 ? nrhs : nr;
  sa.n = n_cells(ctx);
  sa.sxc = ctx->d_sxc;
  sa.syc = ctx->d_syc;
  // the symmetric form's mid scaling marks it; sweep_pair sets the D scalings per direction
  sa.sym_mid = (prec == 0 && ctx->sym32) ? 1 : 0;
  return sa;
}

// Persistent CTAs of the dataflow sweep for precision prec (host queries only).
int flow_grid(fdfd_ctx* ctx, int prec) {
  if (ctx->flow_grid[prec] > 0) return ctx->flow_grid[prec];   // prec 2: the paired-RHS variant of c64
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || nsm <= 0) nsm = 1;
  ctx->flow_grid[prec] = nsm * flow_blocks_per_sm(prec == 1 ? 16 : 8, std::max(1, ctx->flow_vmax), flow_wide(ctx),
                                                  prec == 2);
  return ctx->flow_grid[prec];
}

// Sweep pair on factor precision T: out = A^-1 in (or A^-T in), one persistent
// dataflow launch per direction.  ctr: counter buffer of at least
// 1 + 2 * n_omega * n_fronts ints (cleared here before each launch).
template <typename T>
fdfd_status sweep_pair(fdfd_ctx* ctx, const SolveLaunch& sa, int transpose, const void* in, void* out, int* ctr) {
  const int prec = sizeof(T) == 8 ? 0 : 1;
  const Plan& p = ctx->plan;
  cudaStream_t s = ctx->stream;
  // symmetric form: both solves are the L sweep then the L^T sweep (A x = b with D b
  // gathered, A^T x = b with D x written), 1 / d taken between them
  const bool sym = sa.sym_mid != 0;
  const int fwd = sym ? 0 : (transpose ? 2 : 0), bwd = sym ? 3 : (transpose ? 3 : 1);
  const double es = sizeof(T), nsys = (double)sa.n_omega * sa.nr;
  int tt = transpose ? 1 : 0;                             // row tasks (L, U) or column tasks (U^T, L^T)
  int step = tt ? sweep_col_block() : sweep_row_block();
  // algorithmic work: every entry of the swept triangle (and of the off-diagonal
  // block) read once per right-hand side, 8 flops per entry, plus the vectors
  auto tri_work = [&](const TaskList& tl, bool lower, double* fl, double* by) {
    *fl = *by = 0;
    if (!ctx->prof_on) return;
    for (int t = 0; t < tl.n; ++t) {
      const int e = ctx->h_lists[tl.off + 2 * t];
      const FrontDesc& d = p.fronts[e & kSweepFrontMask];
      const bool whole = e < 0;
      const int b0 = whole ? 0 : ctx->h_lists[tl.off + 2 * t + 1];
      const int rows = (e & kSweepTaskTall) ? 2 * step : step;
      const int b1 = whole ? d.k : std::min(d.k, b0 + rows);
      double ent = 0;   // entries of this task's rows (or columns) inside the triangle
      for (int r = b0; r < b1; ++r) ent += lower ? r : (d.k - r);
      if (whole) ent += (double)d.k * d.m;   // whole-front tasks also do the off-diagonal block
      *fl += 8.0 * ent * nsys;
      *by += es * (ent + (b1 - b0)) * nsys;
    }
  };
  auto rect_work = [&](const TaskList& tl, bool over_m, double* fl, double* by) {
    *fl = *by = 0;
    if (!ctx->prof_on) return;
    for (int t = 0; t < tl.n; ++t) {
      const int e = ctx->h_lists[tl.off + 2 * t];
      const FrontDesc& d = p.fronts[e & kSweepFrontMask];
      const int s0 = ctx->h_lists[tl.off + 2 * t + 1];
      const double rows = std::min((e & kSweepTaskTall) ? 2 * step : step, (over_m ? d.m : d.k) - s0);
      const double other = over_m ? d.k : d.m;
      *fl += 8.0 * rows * other * nsys;
      *by += es * rows * (other + 1) * nsys;
    }
  };
  const int* dl = ctx->d_lists;
  const size_t ctr_bytes = sizeof(int) * (1 + 2 * (size_t)sa.n_omega * p.fronts.size());
  // complex64 factors with an even number of right-hand sides per wavelength: the paired variant
  const bool pairs = prec == 0 && ctx->opt.sweep_rhs_pairs && sa.nr >= 2 && sa.nr % 2 == 0;
  const int grid_max = flow_grid(ctx, pairs ? 2 : prec);
  for (int dir = 0; dir < 2; ++dir) {
    SolveLaunch sd = sa;
    if (sym) {
      tt = dir;                                            // L: row tasks; L^T: column tasks
      step = tt ? sweep_col_block() : sweep_row_block();
      sd.sym_in = (dir == 0 && !transpose) ? 1 : 0;
      sd.sym_out = (dir == 1 && transpose) ? 1 : 0;
      sd.sym_mid = dir == 1 ? 1 : 0;
    }
    const auto& fq = ctx->flow[tt][dir];
    double fl = 0, by = 0;
    for (int l = 0; l < p.n_levels; ++l) {
      const SolveList& sl = ctx->lv_solve[l];
      double f1, b1;
      tri_work(sl.tri[tt], sym ? true : (dir == 0 ? !transpose : transpose), &f1, &b1);
      fl += f1; by += b1;
      rect_work(dir == 0 ? sl.rect_m[tt] : sl.rect_k[tt], dir == 0, &f1, &b1);
      fl += f1; by += b1;
    }
    CK(cudaMemsetAsync(ctr, 0, ctr_bytes, s));
    FlowQueue q;
    q.tasks = reinterpret_cast<const int2*>(dl + fq.off);
    q.units = reinterpret_cast<const int2*>(dl + fq.uoff);
    q.nunits = fq.nu;
    q.ctr = ctr;
    q.need_all = dl + fq.need_all;
    q.need_ph1 = dl + fq.need_ph1;
    q.err = ctx->d_flow_err;
    q.n_fronts = (int)p.fronts.size();
    const int grid = std::max(1, std::min(grid_max, fq.nu * sa.n_omega));
    const int kind = sym ? (dir == 0 ? PK_SWEEP_L : PK_SWEEP_LT)
                         : (dir == 0 ? (transpose ? PK_SWEEP_UT : PK_SWEEP_L) : (transpose ? PK_SWEEP_LT : PK_SWEEP_U));
    Prof pr(ctx, kind, fl, by);
    launch_sweep_flow<T>(sd, dir == 0 ? fwd : bwd, q, std::max(1, ctx->flow_vmax), grid, in, out, s, flow_wide(ctx),
                         pairs);
  }
  CK(cudaGetLastError());
  return FDFD_OK;
}

// Triangular sweeps on factor precision T with the context's buffers.
template <typename T>
fdfd_status sweeps(fdfd_ctx* ctx, int nrhs, int transpose, const void* in, void* out, int w0 = 0,
                   int nw = -1, int r0 = 0, int nr = -1) {
  return sweep_pair<T>(ctx, solve_launch<T>(ctx, ctx->d_vb, nrhs, w0, nw, r0, nr), transpose, in, out,
                       ctx->d_flow_ctr);
}

// Runs `body`, which issues its work on ctx->stream, as a CUDA graph keyed by
// `key`: captured (on the private stream) the first time, replayed afterwards,
// joined to the caller's stream by events.  While profiling, runs it directly
// so that every launch keeps its own events.
template <typename Body>
fdfd_status run_graph(fdfd_ctx* ctx, int key, Body&& body) {
  if (ctx->prof_on) return body();
  if (!ctx->gstream) {
    CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->gev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->gev_out, cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&ctx->istream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->iev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->iev_join, cudaEventDisableTiming));
  }
  cudaGraphExec_t exec = nullptr;
  for (const auto& g : ctx->graphs)
    if (g.key == key) exec = g.exec;
  if (!exec) {
    cudaStream_t user = ctx->stream;
    ctx->stream = ctx->gstream;
    cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
    fdfd_status st = FDFD_OK;
    if (e == cudaSuccess) st = body();
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(ctx->gstream, &g) : e;
    ctx->stream = user;
    if (st != FDFD_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    CK(e);
    CK(e2);
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    ctx->graphs.push_back({key, exec});
  }
  CK(cudaEventRecord(ctx->gev_in, ctx->stream));
  CK(cudaStreamWaitEvent(ctx->gstream, ctx->gev_in, 0));
  CK(cudaGraphLaunch(exec, ctx->gstream));
  CK(cudaEventRecord(ctx->gev_out, ctx->gstream));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->gev_out, 0));
  return FDFD_OK;
}

// Full or design factorisation of every wavelength, replayed from a graph.
template <typename T>
fdfd_status factor_all(fdfd_ctx* ctx, bool design_only, bool sym = false) {
  CKS(ensure_store(ctx, sizeof(T) == 8 ? 0 : 1));      // allocations stay outside the capture
  const int key = (sizeof(T) == 8 ? (sym ? 4 : 0) : 2) + (design_only ? 1 : 0);
  return run_graph(ctx, key, [&]() { return factor_levels<T>(ctx, design_only, 0, -1, sym); });
}

// Applies the cached factors M^-1 to FP64 vectors: dst = M^-1 src (all systems).
fdfd_status precond(fdfd_ctx* ctx, int nrhs, int transpose, const double2* src, double2* dst) {
  ctx->sweeps += 1;
  if (ctx->valid64) return sweeps<double2>(ctx, nrhs, transpose, src, dst);
  // complex64 factors: the sweeps read src and write dst in complex128 themselves
  return sweeps<float2>(ctx, nrhs, transpose, src, dst);
}

fdfd_status ensure_gm(fdfd_ctx* ctx, int nrhs, int m) {
  if (ctx->gm_nrhs >= nrhs && ctx->gm_m >= m) return FDFD_OK;
  free_gm(ctx);
  const size_t S = (size_t)ctx->n_omega * nrhs;
  const size_t N = (size_t)n_cells(ctx);
  const int D = multidot_max_vectors();
  const int nblk = multidot_blocks((long long)N);
  CK(dalloc(&ctx->d_V, sizeof(double2) * (m + 1) * S * N));
  CK(dalloc(&ctx->d_Z, sizeof(double2) * m * S * N));
  CK(dalloc(&ctx->d_r, sizeof(double2) * S * N));
  CK(dalloc(&ctx->d_w, sizeof(double2) * S * N));
  CK(dalloc(&ctx->d_h, sizeof(double2) * S * D));
  CK(dalloc(&ctx->d_h2, sizeof(double2) * S * D));
  CK(dalloc(&ctx->d_hn, sizeof(double2) * S * D));
  CK(dalloc(&ctx->d_bd, sizeof(double2) * S * D));
  CK(dalloc(&ctx->d_H, sizeof(double2) * S * m * (m + 1)));
  CK(dalloc(&ctx->d_cs, sizeof(double2) * S * m));
  CK(dalloc(&ctx->d_sn, sizeof(double2) * S * m));
  CK(dalloc(&ctx->d_g, sizeof(double2) * S * (m + 1)));
  CK(dalloc(&ctx->d_ycoef, sizeof(double2) * S * D));
  CK(dalloc(&ctx->d_partial, sizeof(double2) * S * D * std::max(nblk, arnoldi_blocks((long long)N))));
  CK(dalloc(&ctx->d_vscale, sizeof(double) * S));
  CK(dalloc(&ctx->d_resid, sizeof(double) * S));
  CK(dalloc(&ctx->d_bnorm, sizeof(double) * S));
  CK(dalloc(&ctx->d_active, sizeof(int) * S));
  CK(dalloc(&ctx->d_nj, sizeof(int) * S));
  CK(dalloc(&ctx->d_gcnt, sizeof(int) * S));
  CK(cudaMemsetAsync(ctx->d_gcnt, 0, sizeof(int) * S, ctx->stream));
  if (!ctx->h_active) {
    CK(cudaMallocHost((void**)&ctx->h_active, sizeof(int) * 4096));
    CK(cudaMallocHost((void**)&ctx->h_nj, sizeof(int) * 4096));
    CK(cudaMallocHost((void**)&ctx->h_resid, sizeof(double) * 4096));
  }
  ctx->gm_nrhs = nrhs;
  ctx->gm_m = m;
  return FDFD_OK;
}

// A dataflow sweep whose wait gave up leaves its error word set; report it once
// (the pinned copy is refreshed at every synchronisation point) and clear it.
fdfd_status check_flow_err(fdfd_ctx* ctx) {
  if (!ctx->h_flow_err || *ctx->h_flow_err == 0) return FDFD_OK;
  const int code = *ctx->h_flow_err;
  *ctx->h_flow_err = 0;
  CK(cudaMemsetAsync(ctx->d_flow_err, 0, sizeof(int), ctx->stream));
  return fail(ctx, FDFD_ERR_TIMEOUT, code == 2 ? "a tensor-core update matrix gave up waiting on its copy/MMA pipeline"
                                                : "a sweep gave up waiting for a front it depends on");
}

fdfd_status any_active(fdfd_ctx* ctx, int S, bool* any, double* maxres) {
  CK(cudaMemcpyAsync(ctx->h_active, ctx->d_active, sizeof(int) * S, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(ctx->h_nj, ctx->d_nj, sizeof(int) * S, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(ctx->h_resid, ctx->d_resid, sizeof(double) * S, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(ctx->h_flow_err, ctx->d_flow_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->growth_pending) ctx->growth_ready = true;
  CKS(check_flow_err(ctx));
  *any = false;
  *maxres = 0;
  for (int i = 0; i < S; ++i) {
    if (ctx->h_active[i]) *any = true;
    const double r = ctx->h_resid[i];
    if (!(r <= *maxres)) *maxres = r;
  }
  return FDFD_OK;
}

// Flexible GMRES, right-preconditioned by the cached LU, FP64 residuals and updates.
fdfd_status fgmres(fdfd_ctx* ctx, const double2* b, double2* x, int nrhs, int transpose) {
  const int m = std::max(1, std::min(ctx->opt.gmres_restart, multidot_max_vectors() - 1));
  CKS(ensure_gm(ctx, nrhs, m));
  const int S = ctx->n_omega * nrhs;
  if (S > 4096) return fail(ctx, FDFD_ERR_ARG, "too many systems for one solve (max 4096)");
  const long long N = n_cells(ctx);
  const size_t vs = (size_t)S * N;   // stride between Krylov vectors
  const int D = multidot_max_vectors();
  const int nblk = multidot_blocks(N);
  const double tol = ctx->opt.ir_tol;
  const DevCoef C = dev_coef(ctx);
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(x, 0, sizeof(double2) * vs, s));
  CK(cudaMemcpyAsync(ctx->d_r, b, sizeof(double2) * vs, cudaMemcpyDeviceToDevice, s));
  { Prof pr(ctx, PK_DOT, 8.0 * N * S, 16.0 * N * S);
    launch_multidot(b, 0, 1, b, N, S, ctx->d_partial, nblk, ctx->d_bd, D, s); }
  long long total = 0;
  double res = 0;
  bool converged = false;
  int cycles = 0;
  for (int cycle = 0;; ++cycle) {
    cycles = cycle;
    if (cycle > 0) {
      Prof pr(ctx, PK_STENCIL, 48.0 * N * S, 56.0 * N * S);
      launch_stencil(C, ctx->n_omega, nrhs, transpose, x, b, ctx->d_r, 1, s);
    }
    { Prof pr(ctx, PK_DOT, 8.0 * N * S, 16.0 * N * S);
      launch_multidot(ctx->d_r, 0, 1, ctx->d_r, N, S, ctx->d_partial, nblk, ctx->d_hn, D, s); }
    { Prof pr(ctx, PK_OTHER, 0, 0);
    gm_start(ctx->d_hn, D, ctx->d_bd, D, S, tol, m, ctx->d_g, ctx->d_vscale, ctx->d_active, ctx->d_resid,
             ctx->d_bnorm, cycle == 0 ? 1 : 0, s); }
    CK(cudaGetLastError());
    bool any = true;
    // The first cycle starts from x = 0 (r = b), so nothing can have converged
    // yet; later cycles start from the true FP64 residual and decide.
    if (cycle > 0 || ctx->opt.ir_max_iter == 0) {
      CKS(any_active(ctx, S, &any, &res));
      if (!any) { converged = res <= tol; break; }   // a NaN residual is never converged
    }
    if (total >= ctx->opt.ir_max_iter) break;
    { Prof pr(ctx, PK_OTHER, 0, 32.0 * N * S); gm_scale(ctx->d_V, ctx->d_r, ctx->d_vscale, N, S, s); }
    CK(cudaMemsetAsync(ctx->d_nj, 0, sizeof(int) * S, s));
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      double2* Vj = ctx->d_V + (size_t)j * vs;
      double2* Zj = ctx->d_Z + (size_t)j * vs;
      CKS(precond(ctx, nrhs, transpose, Vj, Zj));
      // w = A z_j, classical Gram-Schmidt applied twice, |w|, Givens update: three passes
      ArnoldiStep as;
      as.C = C; as.nrhs = nrhs; as.transpose = transpose;
      as.z = Zj; as.V = ctx->d_V; as.vstride = (long long)vs; as.nv = j + 1; as.w = ctx->d_w;
      as.partial = ctx->d_partial; as.cnt = ctx->d_gcnt;
      as.h1 = ctx->d_h; as.h2 = ctx->d_h2; as.hn = ctx->d_hn;
      as.nj = ctx->d_nj; as.active = ctx->d_active; as.resid = ctx->d_resid; as.bnorm = ctx->d_bnorm;
      as.vscale = ctx->d_vscale; as.H = ctx->d_H; as.cs = ctx->d_cs; as.sn = ctx->d_sn; as.g = ctx->d_g;
      as.m = m; as.tol = tol;
      const double pf = 8.0 * (j + 1) * N * S, pb = 16.0 * (j + 3) * N * S;
      { Prof pr(ctx, PK_ARNOLDI, 48.0 * N * S + pf, 40.0 * N * S + 16.0 * (j + 1) * N * S);
        launch_arnoldi(as, S, 0, s); }
      { Prof pr(ctx, PK_ARNOLDI, 2.0 * pf, pb); launch_arnoldi(as, S, 1, s); }
      { Prof pr(ctx, PK_ARNOLDI, pf + 4.0 * N * S, pb); launch_arnoldi(as, S, 2, s); }
      CK(cudaGetLastError());
      ++total;
      jdone = j + 1;
      // The first cycle stops, without asking the host, once it has done as many
      // iterations as the previous solve needed: the update and the true residual
      // of the next cycle then decide (one host synchronisation per solve when
      // the expectation holds; a restart when it does not).  Later cycles look at
      // the convergence flags after every iteration; meanwhile the device-side
      // flags already freeze converged systems (zero search directions, no updates).
      if (cycle == 0 && total == ctx->gm_expect[transpose ? 1 : 0] && total < ctx->opt.ir_max_iter) break;
      if (total >= ctx->gm_expect[transpose ? 1 : 0] || j + 1 == m || total >= ctx->opt.ir_max_iter) {
        CKS(any_active(ctx, S, &any, &res));
        if (!any) break;
      }
      if (total >= ctx->opt.ir_max_iter) break;
      if (j + 1 < m) {
        Prof pr(ctx, PK_OTHER, 0, 32.0 * N * S);
        gm_scale(ctx->d_V + (size_t)(j + 1) * vs, ctx->d_w, ctx->d_vscale, N, S, s);
      }
    }
    { Prof pr(ctx, PK_OTHER, 0, 0); gm_solve(ctx->d_H, ctx->d_g, S, m, ctx->d_nj, ctx->d_ycoef, s); }
    { Prof pr(ctx, PK_AXPY, 8.0 * jdone * N * S, 16.0 * (jdone + 2) * N * S);
      launch_multiaxpy(ctx->d_Z, (long long)vs, jdone, ctx->d_ycoef, D, x, N, S, nullptr, s); }
    CK(cudaGetLastError());
  }
  ctx->last_iters = total;
  ctx->last_resid = res;
  // Next solve's first cycle: as many iterations as this one needed.  When one
  // cycle sufficed, that is the largest count of Krylov vectors a system used
  // before its Givens residual met the tolerance (the device stops counting
  // then), which may be fewer than the iterations run here.
  long long expect = total;
  if (converged && cycles == 1) {
    int mx = 0;
    for (int i = 0; i < S; ++i) mx = std::max(mx, ctx->h_nj[i]);
    if (mx > 0) expect = std::min<long long>(expect, mx);
  }
  ctx->gm_expect[transpose ? 1 : 0] = std::max<long long>(1, expect);
  if (!converged)
    return fail(ctx, FDFD_ERR_NOT_CONVERGED,
                "refinement stopped at relative residual " + std::to_string(res) + " after " +
                    std::to_string(total) + " iterations");
  return FDFD_OK;
}

// The whole factorisation in FP64, partial pivoting over every pivot row of each front.
fdfd_status refactor_f64(fdfd_ctx* ctx) {
  ctx->fallbacks += 1;
  const int piv_saved = ctx->opt.pivoting;
  ctx->opt.pivoting = 0;
  const fdfd_status fst = factor_levels<double2>(ctx, false);
  ctx->opt.pivoting = piv_saved;
  CKS(fst);
  CK(cudaStreamSynchronize(ctx->stream));
  const float g64 = *ctx->h_growth_max;
  ctx->last_growth = g64;
  if (!std::isfinite(g64))
    return fail(ctx, FDFD_ERR_PIVOT, "zero or non-finite pivot in the FP64 factorisation");
  ctx->valid64 = true;
  return FDFD_OK;
}

// Checks the pivot growth of the last FP32 factorisation.  Above the bound, a
// factorisation with block-local pivoting is first redone in FP32 with partial
// pivoting over every pivot row of each front; if the growth is still above the
// bound (or that was already the pivoting used), the factorisation is redone in
// FP64.  The growth figure is copied to pinned host memory at the end of the
// factorisation; any later stream synchronisation makes it readable.
// refined: the caller refines the solve on these factors (FGMRES with the FP64 residual), so
// factors with finite growth above the bound can be kept after the repivot; a raw solve
// (no refinement to check them) sends them to FP64 instead.
fdfd_status settle_growth(fdfd_ctx* ctx, bool* fell_back = nullptr, bool* repivoted = nullptr,
                          bool refined = false) {
  if (fell_back) *fell_back = false;
  if (repivoted) *repivoted = false;
  if (!ctx->growth_pending) return FDFD_OK;
  if (!ctx->growth_ready) CK(cudaStreamSynchronize(ctx->stream));
  ctx->growth_pending = false;
  ctx->growth_ready = false;
  CKS(check_flow_err(ctx));
  float g = *ctx->h_growth_max;
  ctx->last_growth = g;
  if (g <= ctx->opt.growth_bound) return FDFD_OK;
  const int piv_saved = ctx->opt.pivoting;
  if (ctx->sym32 || piv_saved == 1) {
    // the symmetric form (no pivoting) or block-local pivoting exceeded the bound:
    // complex FP32 LU with partial pivoting over all pivot rows of each front
    ctx->repivots += 1;
    if (repivoted) *repivoted = true;
    ctx->opt.pivoting = 0;
    ctx->sym32 = false;
    const fdfd_status fst = factor_levels<float2>(ctx, false);
    ctx->opt.pivoting = piv_saved;
    CKS(fst);
    CK(cudaStreamSynchronize(ctx->stream));
    CKS(check_flow_err(ctx));
    g = *ctx->h_growth_max;
    ctx->last_growth = g;
    if (g <= ctx->opt.growth_bound) return FDFD_OK;
  }
  // Finite growth above the bound with partial pivoting over all pivot rows: for a refined
  // solve the complex FP32 factors are kept, and refinement, which measures the FP64 residual,
  // decides (a solve that does not converge on them sends the factorisation to FP64).  A zero
  // or non-finite pivot (inf / NaN growth), or a raw solve, goes to FP64 at once.
  if (refined && g < INFINITY) return FDFD_OK;
  if (fell_back) *fell_back = true;
  return refactor_f64(ctx);
}

fdfd_status solve_direct(fdfd_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, int transpose,
                         bool* handled);
fdfd_status solve_refined(fdfd_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, int transpose);

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void fdfd_default_options(fdfd_options* o) {
  if (!o) return;
  o->mode = FDFD_MODE_MIXED;
  o->ir_tol = 1e-9;
  o->ir_max_iter = 40;
  o->gmres_restart = 8;
  o->growth_bound = 1e7;
  o->leaf_area = 32;
  o->pivoting = 1;
  o->tensor_form = 3;
  o->tensor_min_m = 128;
  o->tensor_min_tiles = 0;
  o->factor_form = 0;
  o->sweep_rhs_pairs = 0;
  o->tensor_offdiag = 0;
}

fdfd_status fdfd_create(fdfd_ctx** out, fdfd_grid grid, double dx, const double* k0_host, int n_omega,
                        fdfd_pml pml, fdfd_box design, const fdfd_options* opt, void* cuda_stream) {
  if (!out) return FDFD_ERR_ARG;
  *out = nullptr;
  if (grid.nx <= 0 || grid.ny <= 0 || n_omega <= 0 || !k0_host || !(dx > 0)) return FDFD_ERR_ARG;
  if (pml.npml_x < 0 || pml.npml_y < 0 || 2 * pml.npml_x > grid.nx || 2 * pml.npml_y > grid.ny)
    return FDFD_ERR_ARG;
  if (design.w < 0 || design.h < 0) return FDFD_ERR_ARG;
  if (design.w > 0 && design.h > 0 &&
      (design.x0 < 0 || design.y0 < 0 || design.x0 + design.w > grid.nx || design.y0 + design.h > grid.ny))
    return FDFD_ERR_ARG;
  if ((long long)grid.nx * grid.ny * 5 >= (1LL << 31)) return FDFD_ERR_ARG;
  if (opt && (opt->mode < FDFD_MODE_MIXED || opt->mode > FDFD_MODE_PLAIN)) return FDFD_ERR_ARG;
  for (int w = 0; w < n_omega; ++w)
    if (!(k0_host[w] > 0)) return FDFD_ERR_ARG;
  fdfd_ctx* c = new fdfd_ctx();
  c->nx = grid.nx;
  c->ny = grid.ny;
  c->dx = dx;
  c->n_omega = n_omega;
  for (int w = 0; w < n_omega; ++w) c->k0dx.push_back(k0_host[w] * dx);
  c->pml = pml;
  if (!(c->pml.order > 0)) c->pml.order = 3.0;
  if (!(c->pml.ln_R < 0)) c->pml.ln_R = std::log(1e-8);
  c->box = design;
  if (design.w == 0 || design.h == 0) c->box = fdfd_box{0, 0, 0, 0};
  fdfd_default_options(&c->opt);
  if (opt) c->opt = *opt;
  if (c->opt.gmres_restart < 1) c->opt.gmres_restart = 1;
  if (c->opt.gmres_restart > 16) c->opt.gmres_restart = 16;
  if (c->opt.leaf_area < 1) c->opt.leaf_area = 32;
  if (c->opt.pivoting != 0) c->opt.pivoting = 1;
  if (c->opt.tensor_form < 0 || c->opt.tensor_form > 3) c->opt.tensor_form = 3;
  if (c->opt.tensor_min_m < 1) c->opt.tensor_min_m = 1;
  if (c->opt.tensor_min_tiles < 0) c->opt.tensor_min_tiles = 0;
  if (c->opt.factor_form != 1) c->opt.factor_form = 0;
  if (c->opt.sweep_rhs_pairs != 0) c->opt.sweep_rhs_pairs = 1;
  if (c->opt.tensor_offdiag != 0) c->opt.tensor_offdiag = 1;
  if (c->opt.ir_max_iter < 0) c->opt.ir_max_iter = 0;
  {
    fdfd_options def;
    fdfd_default_options(&def);
    if (!(c->opt.ir_tol > 0)) c->opt.ir_tol = def.ir_tol;
    if (!(c->opt.growth_bound > 0)) c->opt.growth_bound = def.growth_bound;
  }
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  *out = c;
  return FDFD_OK;
}

fdfd_status fdfd_analyze(fdfd_ctx* ctx) {
  if (!ctx) return FDFD_ERR_ARG;
  ctx->err.clear();
  if (ctx->analyzed) return FDFD_OK;
  return analyze_host(ctx);
}

fdfd_status fdfd_factor(fdfd_ctx* ctx, const double* eps_dev) {
  if (!ctx || !eps_dev) return FDFD_ERR_ARG;
  ctx->err.clear();
  CKS(ensure_runtime(ctx));
  CK(cudaMemcpyAsync(ctx->d_eps, eps_dev, sizeof(double) * n_cells(ctx), cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->have_eps = true;
  ctx->valid32 = ctx->valid64 = false;
  if (ctx->opt.mode == FDFD_MODE_PLAIN) return FDFD_OK;   // factorised inside every solve
  CKS(ensure_device(ctx));
  if (ctx->opt.mode == FDFD_MODE_F64) {
    CKS(factor_all<double2>(ctx, false));
    ctx->valid64 = true;
    ctx->growth_pending = false;
  } else {
    const bool sym = ctx->opt.factor_form == 1;
    CKS(factor_all<float2>(ctx, false, sym));
    ctx->valid32 = true;
    ctx->sym32 = sym;
    ctx->growth_pending = true;
  }
  ctx->nf += ctx->n_omega;
  return FDFD_OK;
}

fdfd_status fdfd_refactor_design(fdfd_ctx* ctx, const double* eps_design_dev) {
  if (!ctx || !eps_design_dev) return FDFD_ERR_ARG;
  ctx->err.clear();
  if (!ctx->have_eps) return fail(ctx, FDFD_ERR_STATE, "fdfd_refactor_design before fdfd_factor");
  if (ctx->box.w == 0) return fail(ctx, FDFD_ERR_STATE, "context has no design box");
  CKS(ensure_runtime(ctx));
  {
    Prof pr_s(ctx, PK_OTHER, 0, 16.0 * ctx->box.w * ctx->box.h);
    launch_scatter_design(ctx->d_eps, eps_design_dev, ctx->ny, ctx->box.x0, ctx->box.y0, ctx->box.w,
                          ctx->box.h, ctx->stream);
  }
  CK(cudaGetLastError());
  if (ctx->opt.mode == FDFD_MODE_PLAIN) return FDFD_OK;
  CKS(ensure_device(ctx));
  if (ctx->opt.mode == FDFD_MODE_F64) {
    if (!ctx->valid64) return fail(ctx, FDFD_ERR_STATE, "no cached factorisation");
    CKS(factor_all<double2>(ctx, true));
  } else {
    if (!ctx->valid32) return fail(ctx, FDFD_ERR_STATE, "no cached factorisation");
    const bool sym = ctx->opt.factor_form == 1;
    // the untouched fronts' update matrices must be in the form being refactored: after a
    // fallback from the symmetric form to LU the whole factorisation is redone
    const bool design_only = sym == ctx->sym32;
    CKS(factor_all<float2>(ctx, design_only, sym));
    ctx->sym32 = sym;
    ctx->valid64 = false;
    ctx->growth_pending = true;
  }
  ctx->nf += ctx->n_omega;
  return FDFD_OK;
}

fdfd_status fdfd_solve(fdfd_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, int transpose) {
  if (!ctx || !b_dev || !x_dev || nrhs <= 0 || b_dev == x_dev) return FDFD_ERR_ARG;
  ctx->err.clear();
  if (!ctx->have_eps) return fail(ctx, FDFD_ERR_STATE, "fdfd_solve before fdfd_factor");
  bool handled = false;
  const fdfd_status st = solve_direct(ctx, b_dev, x_dev, nrhs, transpose, &handled);
  if (handled) {
    // direct paths do not synchronise: their sweep error word is copied back
    // now and reported by the next call
    if (ctx->h_flow_err) CK(cudaMemcpyAsync(ctx->h_flow_err, ctx->d_flow_err, sizeof(int), cudaMemcpyDeviceToHost,
                                            ctx->stream));
    return st;
  }
  return solve_refined(ctx, b_dev, x_dev, nrhs, transpose);
}

}  // extern "C"

namespace {

// Direct solves (plain, FP64 and raw modes); *handled = false when the
// refined path applies instead.
fdfd_status solve_direct(fdfd_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, int transpose,
                         bool* handled) {
  *handled = true;
  CKS(check_flow_err(ctx));
  const double2* b = reinterpret_cast<const double2*>(b_dev);
  double2* x = reinterpret_cast<double2*>(x_dev);
  const long long N = n_cells(ctx);
  const int S = ctx->n_omega * nrhs;
  if (ctx->opt.mode == FDFD_MODE_PLAIN) {
    // The paper's uncached arm: every system gets its own symbolic and numeric factorisation.
    CKS(ensure_runtime(ctx));
    for (int r = 0; r < nrhs; ++r) {
      for (int w = 0; w < ctx->n_omega; ++w) {
        CKS(analyze_host(ctx));
        CKS(upload_plan(ctx));
        CKS(ensure_ws(ctx, nrhs));
        CKS(factor_levels<double2>(ctx, false, w, 1));
        ctx->nf += 1;
        CKS(sweeps<double2>(ctx, nrhs, transpose, b, x, w, 1, r, 1));
        ctx->sweeps += 1;
        ctx->bs += 1;
      }
    }
    ctx->last_iters = 0;
    (void)S;
    return FDFD_OK;
  }
  CKS(ensure_device(ctx));
  CKS(ensure_ws(ctx, nrhs));
  ctx->bs += S;
  if (ctx->valid64 && (ctx->opt.mode == FDFD_MODE_F64)) {
    CKS(sweeps<double2>(ctx, nrhs, transpose, b, x));
    ctx->sweeps += 1;
    ctx->last_iters = 0;
    return FDFD_OK;
  }
  if (ctx->opt.ir_max_iter == 0) {
    // raw solve on the cached factors, no refinement
    CKS(settle_growth(ctx));
    return precond(ctx, nrhs, transpose, b, x);
  }
  (void)N;
  *handled = false;
  return FDFD_OK;
}

fdfd_status solve_refined(fdfd_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, int transpose) {
  const double2* b = reinterpret_cast<const double2*>(b_dev);
  double2* x = reinterpret_cast<double2*>(x_dev);
  // Refinement first: its synchronisations make the growth figure of a fresh
  // FP32 factorisation readable for free.  A front with too much growth sends
  // the whole factorisation to FP32 with full partial pivoting, then if need be
  // to FP64, and the solve is repeated on the new factors when needed.
  const fdfd_status st = fgmres(ctx, b, x, nrhs, transpose);
  if (st != FDFD_OK && st != FDFD_ERR_NOT_CONVERGED) return st;
  bool fell_back = false, repivoted = false;
  CKS(settle_growth(ctx, &fell_back, &repivoted, true));
  // a solve that converged on the first factors stands; otherwise it is repeated
  // on the refactored ones
  if (fell_back || (repivoted && st == FDFD_ERR_NOT_CONVERGED)) {
    const fdfd_status st2 = fgmres(ctx, b, x, nrhs, transpose);
    if (st2 != FDFD_ERR_NOT_CONVERGED || ctx->valid64) return st2;
  } else if (st != FDFD_ERR_NOT_CONVERGED || ctx->valid64) {
    return st;
  }
  // refinement on complex FP32 factors did not converge: the factorisation is
  // redone in FP64 and the solve repeated on it
  ctx->err.clear();
  CKS(refactor_f64(ctx));
  return fgmres(ctx, b, x, nrhs, transpose);
}

}  // namespace

extern "C" {

fdfd_status fdfd_objective_target(fdfd_ctx* ctx, const double* x_dev, int nrhs, const int* cols_dev,
                                  const double* g_dev, const double* weight_dev, const double* target_dev,
                                  double* o_dev, double* F_dev, double* b_adj_dev) {
  if (!ctx || !x_dev || nrhs <= 0 || !cols_dev || !g_dev || !o_dev || !F_dev) return FDFD_ERR_ARG;
  ctx->err.clear();
  Prof pr(ctx, PK_OTHER, 0, 0);
  launch_objective(reinterpret_cast<const double2*>(x_dev), n_cells(ctx), ctx->ny, cols_dev,
                   reinterpret_cast<const double2*>(g_dev), weight_dev, target_dev, ctx->n_omega * nrhs,
                   reinterpret_cast<double2*>(o_dev), F_dev, reinterpret_cast<double2*>(b_adj_dev), ctx->stream);
  CK(cudaGetLastError());
  return FDFD_OK;
}

fdfd_status fdfd_objective(fdfd_ctx* ctx, const double* x_dev, int nrhs, const int* cols_dev, const double* g_dev,
                           const double* weight_dev, double* o_dev, double* F_dev, double* b_adj_dev) {
  return fdfd_objective_target(ctx, x_dev, nrhs, cols_dev, g_dev, weight_dev, nullptr, o_dev, F_dev, b_adj_dev);
}

fdfd_status fdfd_design_iteration(fdfd_ctx* ctx, const double* eps_design, const double* b_dev, int nrhs,
                                  const int* cols_dev, const double* g_dev, const double* weight_dev,
                                  const double* target_dev, double* F_out, double* grad_out, double* x_dev,
                                  double* xadj_dev, int flags) {
  if (!ctx || !eps_design || !b_dev || nrhs <= 0 || !cols_dev || !g_dev || !F_out || !grad_out ||
      (flags & ~(FDFD_HOST_EPS | FDFD_HOST_OUT)) != 0)
    return FDFD_ERR_ARG;
  ctx->err.clear();
  if (!ctx->have_eps) return fail(ctx, FDFD_ERR_STATE, "fdfd_design_iteration before fdfd_factor");
  if (ctx->box.w == 0) return fail(ctx, FDFD_ERR_STATE, "context has no design box");
  if (x_dev && (x_dev == b_dev || x_dev == xadj_dev)) return FDFD_ERR_ARG;
  CKS(ensure_runtime(ctx));
  const size_t S = (size_t)ctx->n_omega * nrhs, N = (size_t)n_cells(ctx);
  const size_t nd = (size_t)ctx->box.w * ctx->box.h;
  if (ctx->it_nrhs < nrhs) {
    void* ps[] = {ctx->d_itx, ctx->d_ita, ctx->d_itb, ctx->d_ito};
    for (void* p : ps) free_ptr(p);
    ctx->d_itx = ctx->d_ita = ctx->d_itb = ctx->d_ito = nullptr;
    ctx->it_nrhs = 0;
    CK(dalloc(&ctx->d_itx, sizeof(double2) * S * N));
    CK(dalloc(&ctx->d_ita, sizeof(double2) * S * N));
    CK(dalloc(&ctx->d_itb, sizeof(double2) * S * N));
    CK(dalloc(&ctx->d_ito, sizeof(double2) * S));
    ctx->it_nrhs = nrhs;
  }
  if (!ctx->d_itF) {
    CK(dalloc(&ctx->d_itF, sizeof(double)));
    CK(dalloc(&ctx->d_itg, sizeof(double) * nd));
    CK(dalloc(&ctx->d_itepsd, sizeof(double) * nd));
  }
  const double* epsd = eps_design;
  if (flags & FDFD_HOST_EPS) {
    CK(cudaMemcpyAsync(ctx->d_itepsd, eps_design, sizeof(double) * nd, cudaMemcpyHostToDevice, ctx->stream));
    epsd = ctx->d_itepsd;
  }
  const bool host_out = (flags & FDFD_HOST_OUT) != 0;
  double* x = x_dev ? x_dev : reinterpret_cast<double*>(ctx->d_itx);
  double* xa = xadj_dev ? xadj_dev : reinterpret_cast<double*>(ctx->d_ita);
  double* badj = reinterpret_cast<double*>(ctx->d_itb);
  double* Fd = host_out ? ctx->d_itF : F_out;
  double* gd = host_out ? ctx->d_itg : grad_out;
  CKS(fdfd_refactor_design(ctx, epsd));
  CKS(fdfd_solve(ctx, b_dev, x, nrhs, 0));
  CKS(fdfd_objective_target(ctx, x, nrhs, cols_dev, g_dev, weight_dev, target_dev,
                            reinterpret_cast<double*>(ctx->d_ito), Fd, badj));
  CKS(fdfd_solve(ctx, badj, xa, nrhs, 1));
  // the adjoint source already carries the per-system weights (and target factors)
  CKS(fdfd_grad(ctx, x, xa, nrhs, nullptr, gd, 0));
  if (host_out) {
    CK(cudaMemcpyAsync(F_out, ctx->d_itF, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(grad_out, ctx->d_itg, sizeof(double) * nd, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return FDFD_OK;
}

fdfd_status fdfd_grad(fdfd_ctx* ctx, const double* x_fwd_dev, const double* x_adj_dev, int nrhs,
                      const double* weight_dev, double* grad_dev, int accumulate) {
  if (!ctx || !x_fwd_dev || !x_adj_dev || nrhs <= 0 || !grad_dev) return FDFD_ERR_ARG;
  ctx->err.clear();
  if (ctx->box.w == 0) return fail(ctx, FDFD_ERR_STATE, "context has no design box");
  CKS(ensure_runtime(ctx));
  Prof pr(ctx, PK_OTHER, 0, 0);
  launch_grad(reinterpret_cast<const double2*>(x_fwd_dev), reinterpret_cast<const double2*>(x_adj_dev),
              n_cells(ctx), ctx->ny, ctx->box.x0, ctx->box.y0, ctx->box.w, ctx->box.h, ctx->n_omega, nrhs,
              ctx->d_k0dx2, weight_dev, grad_dev, accumulate, ctx->stream);
  CK(cudaGetLastError());
  return FDFD_OK;
}

// The filter taps for this radius on the device: integer offsets with distance
// below the radius, row-major over [-r, r]^2, weight radius - distance.
static fdfd_status ensure_taps(fdfd_ctx* ctx, double radius) {
  if (ctx->d_taps && ctx->tap_radius == radius) return FDFD_OK;
  const int r = (int)std::ceil(radius);
  std::vector<int2> off;
  std::vector<double> wt;
  for (int di = -r; di <= r; ++di)
    for (int dj = -r; dj <= r; ++dj) {
      const double d = std::hypot((double)di, (double)dj);
      if (d < radius) {
        off.push_back(make_int2(di, dj));
        wt.push_back(radius - d);
      }
    }
  CK(cudaStreamSynchronize(ctx->stream));   // the old taps may still be in use
  free_ptr(ctx->d_taps);
  free_ptr(ctx->d_tapw);
  ctx->d_taps = nullptr;
  ctx->d_tapw = nullptr;
  CK(dalloc(&ctx->d_taps, sizeof(int2) * off.size()));
  CK(dalloc(&ctx->d_tapw, sizeof(double) * wt.size()));
  CK(cudaMemcpy(ctx->d_taps, off.data(), sizeof(int2) * off.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_tapw, wt.data(), sizeof(double) * wt.size(), cudaMemcpyHostToDevice));
  ctx->ntap = (int)off.size();
  ctx->tap_radius = radius;
  return FDFD_OK;
}

fdfd_status fdfd_filter_project(fdfd_ctx* ctx, const double* rho_dev, double radius, double beta, double eta,
                                double eps_lo, double eps_hi, double* eps_dev, double* work_dev) {
  if (!ctx || !rho_dev || !eps_dev || !work_dev || !(radius > 0 && radius <= 25) || !(beta > 0) ||
      !(eta > 0 && eta < 1))
    return FDFD_ERR_ARG;
  ctx->err.clear();
  if (ctx->box.w == 0 || ctx->box.h == 0) return fail(ctx, FDFD_ERR_ARG, "context has no design box");
  CKS(ensure_taps(ctx, radius));
  const int w = ctx->box.w, h = ctx->box.h;
  Prof pr(ctx, PK_OTHER, 0, 0);
  launch_filter_project(rho_dev, w, h, ctx->d_taps, ctx->d_tapw, ctx->ntap, beta, eta, eps_lo, eps_hi - eps_lo,
                        eps_dev, work_dev, work_dev + (size_t)w * h, ctx->stream);
  CK(cudaGetLastError());
  return FDFD_OK;
}

fdfd_status fdfd_density_eps(fdfd_ctx* ctx, const double* rho_dev, double eps_lo, double eps_hi, double* eps_dev) {
  if (!ctx || !rho_dev || !eps_dev) return FDFD_ERR_ARG;
  ctx->err.clear();
  if (ctx->box.w == 0 || ctx->box.h == 0) return fail(ctx, FDFD_ERR_ARG, "context has no design box");
  Prof pr(ctx, PK_OTHER, 0, 16.0 * ctx->box.w * ctx->box.h);
  launch_density_eps(rho_dev, (long long)ctx->box.w * ctx->box.h, eps_lo, eps_hi - eps_lo, eps_dev, ctx->stream);
  CK(cudaGetLastError());
  return FDFD_OK;
}

fdfd_status fdfd_filter_project_adjoint(fdfd_ctx* ctx, const double* g_eps_dev, const double* work_dev,
                                        double radius, double* g_rho_dev) {
  if (!ctx || !g_eps_dev || !work_dev || !g_rho_dev || g_rho_dev == g_eps_dev || !(radius > 0 && radius <= 25))
    return FDFD_ERR_ARG;
  ctx->err.clear();
  if (ctx->box.w == 0 || ctx->box.h == 0) return fail(ctx, FDFD_ERR_ARG, "context has no design box");
  CKS(ensure_taps(ctx, radius));
  const int w = ctx->box.w, h = ctx->box.h;
  Prof pr(ctx, PK_OTHER, 0, 0);
  launch_filter_adjoint(g_eps_dev, work_dev, work_dev + (size_t)w * h, w, h, ctx->d_taps, ctx->d_tapw, ctx->ntap,
                        g_rho_dev, ctx->stream);
  CK(cudaGetLastError());
  return FDFD_OK;
}

fdfd_status fdfd_apply(fdfd_ctx* ctx, const double* x_dev, double* y_dev, int nrhs, int transpose) {
  if (!ctx || !x_dev || !y_dev || nrhs <= 0 || x_dev == y_dev) return FDFD_ERR_ARG;
  ctx->err.clear();
  if (!ctx->have_eps) return fail(ctx, FDFD_ERR_STATE, "fdfd_apply before fdfd_factor");
  CKS(ensure_runtime(ctx));
  launch_stencil(dev_coef(ctx), ctx->n_omega, nrhs, transpose, reinterpret_cast<const double2*>(x_dev), nullptr,
                 reinterpret_cast<double2*>(y_dev), 0, ctx->stream);
  CK(cudaGetLastError());
  return FDFD_OK;
}

fdfd_status fdfd_set_options(fdfd_ctx* ctx, const fdfd_options* opt) {
  if (!ctx || !opt) return FDFD_ERR_ARG;
  ctx->opt.ir_tol = opt->ir_tol;
  ctx->opt.ir_max_iter = std::max(0, opt->ir_max_iter);
  ctx->opt.gmres_restart = std::max(1, std::min(16, opt->gmres_restart));
  return FDFD_OK;
}

fdfd_status fdfd_stats_get(fdfd_ctx* ctx, fdfd_stats* o) {
  if (!ctx || !o) return FDFD_ERR_ARG;
  if (ctx->device >= 0) CK(cudaStreamSynchronize(ctx->stream));
  std::memset(o, 0, sizeof(*o));
  o->sf = ctx->sf;
  o->nf = ctx->nf;
  o->bs = ctx->bs;
  o->sweeps = ctx->sweeps;
  o->ir_iters = ctx->last_iters;
  o->ir_resid = ctx->last_resid;
  o->fallbacks = ctx->fallbacks;
  o->repivots = ctx->repivots;
  o->growth = ctx->last_growth;
  o->factor_form = (ctx->valid32 && !ctx->valid64 && ctx->sym32) ? 1 : 0;
  if (ctx->analyzed) {
    const Plan& p = ctx->plan;
    o->n_fronts = (int)p.fronts.size();
    o->n_levels = p.n_levels;
    o->max_front = p.max_front;
    o->factor_entries = p.factor_entries;
    o->flops_factor = p.flops_factor;
    o->flops_design = p.flops_design;
    long long b = 0;
    if (ctx->d_store32) b += (long long)p.store_total * ctx->n_omega * 8;
    if (ctx->d_store64) b += (long long)p.store_total * ctx->n_omega * 16;
    o->store_bytes = b;
  }
  return FDFD_OK;
}

fdfd_status fdfd_plan_sizes(fdfd_ctx* ctx, int* n_host, int* ld_host, int* ldk_host) {
  if (!ctx) return FDFD_ERR_ARG;
  if (!ctx->analyzed) return fail(ctx, FDFD_ERR_STATE, "plan requested before fdfd_analyze");
  const Plan& p = ctx->plan;
  for (size_t f = 0; f < p.fronts.size(); ++f) {
    if (n_host) n_host[f] = p.fronts[f].n;
    if (ld_host) ld_host[f] = p.fronts[f].ld;
    if (ldk_host) ldk_host[f] = p.fronts[f].ldk;
  }
  return FDFD_OK;
}

fdfd_status fdfd_plan_fronts(fdfd_ctx* ctx, int* k, int* m, int* parent, int* level, int* design, int* idx) {
  if (!ctx) return FDFD_ERR_ARG;
  if (!ctx->analyzed) return fail(ctx, FDFD_ERR_STATE, "plan requested before fdfd_analyze");
  const Plan& p = ctx->plan;
  for (size_t f = 0; f < p.fronts.size(); ++f) {
    const FrontDesc& d = p.fronts[f];
    if (k) k[f] = d.k;
    if (m) m[f] = d.m;
    if (parent) parent[f] = d.parent;
    if (level) level[f] = d.level;
    if (design) design[f] = d.design;
  }
  if (idx) std::memcpy(idx, p.idx.data(), sizeof(int) * p.idx.size());
  return FDFD_OK;
}

fdfd_status fdfd_front_copy(fdfd_ctx* ctx, int w, int f, void* front_host, void* inv_host) {
  if (!ctx || w < 0 || w >= ctx->n_omega || f < 0) return FDFD_ERR_ARG;
  ctx->err.clear();
  if (!ctx->analyzed || f >= (int)ctx->plan.fronts.size()) return fail(ctx, FDFD_ERR_ARG, "no such front");
  if (!ctx->valid32 && !ctx->valid64) return fail(ctx, FDFD_ERR_STATE, "no factorisation");
  const FrontDesc& d = ctx->plan.fronts[f];
  const bool f64 = ctx->valid64;
  const size_t es = f64 ? sizeof(double2) : sizeof(float2);
  const char* st = f64 ? reinterpret_cast<const char*>(ctx->d_store64) : reinterpret_cast<const char*>(ctx->d_store32);
  const char* iv = f64 ? reinterpret_cast<const char*>(ctx->d_inv64) : reinterpret_cast<const char*>(ctx->d_inv32);
  CK(cudaStreamSynchronize(ctx->stream));
  if (front_host)
    CK(cudaMemcpy(front_host, st + es * ((size_t)w * ctx->plan.store_total + d.st_off), es * (size_t)d.n * d.ld,
                  cudaMemcpyDeviceToHost));
  if (inv_host)
    CK(cudaMemcpy(inv_host, iv + es * ((size_t)w * ctx->plan.inv_total + d.iv_off), es * (size_t)d.k * d.ldk,
                  cudaMemcpyDeviceToHost));
  return FDFD_OK;
}

fdfd_status fdfd_selftest_schur_tc(fdfd_ctx* ctx, void* front_dev, int k, int m, int ld, int planes) {
  if (!ctx || !front_dev || k < 1 || m < 1 || ld < k + m || planes < 1 || planes > 3 ||
      (reinterpret_cast<uintptr_t>(front_dev) & 7))
    return FDFD_ERR_ARG;
  ctx->err.clear();
  CKS(ensure_runtime(ctx));
  CKS(check_flow_err(ctx));
  FrontDesc d;
  std::memset(&d, 0, sizeof(d));
  d.k = k; d.m = m; d.n = k + m; d.ld = ld; d.parent = -1;
  TcFront r;
  r.f = 0;
  r.Mt = (m + kTcRows - 1) / kTcRows;
  r.Nt = (m + kTcCols - 1) / kTcCols;
  r.Kt = (k + kTcPivots - 1) / kTcPivots;
  int nsm = 0;
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  r.nsplit = tc_splits((long long)r.Mt * r.Nt, r.Kt, nsm);
  r.poff = 0;
  r.aoff = 0;
  r.boff = (long long)r.Mt * r.Kt * tc_tile_bytes_a(planes);
  const long long wsb = r.boff + (long long)r.Nt * r.Kt * tc_tile_bytes_b(planes);
  const long long pfl = r.nsplit > 1 ? (long long)r.Mt * r.Nt * r.nsplit * kTcPartFloats : 4;
  std::vector<int4> tasks;
  for (int mt = 0; mt < r.Mt; ++mt)
    for (int kt = 0; kt < r.Kt; ++kt) tasks.push_back(make_int4(0, 0, mt, kt));
  for (int nt = 0; nt < r.Nt; ++nt)
    for (int kt = 0; kt < r.Kt; ++kt) tasks.push_back(make_int4(0, 1, nt, kt));
  const int npack = (int)tasks.size();
  for (int mt = 0; mt < r.Mt; ++mt)
    for (int nt = 0; nt < r.Nt; ++nt)
      for (int sp = 0; sp < r.nsplit; ++sp) tasks.push_back(make_int4(0, mt, nt, sp));
  const int nprod = (int)tasks.size() - npack;
  if (r.nsplit > 1)
    for (int mt = 0; mt < r.Mt; ++mt)
      for (int nt = 0; nt < r.Nt; ++nt)
        for (int r0 = 0; r0 < kTcRows; r0 += 16) tasks.push_back(make_int4(0, mt, nt, r0));
  FrontDesc* dd = nullptr;
  TcFront* dr = nullptr;
  int4* dt = nullptr;
  unsigned char* dws = nullptr;
  float* dpart = nullptr;
  cudaError_t e = dalloc(&dd, sizeof(FrontDesc));
  if (e == cudaSuccess) e = dalloc(&dpart, sizeof(float) * (size_t)pfl);
  if (e == cudaSuccess) e = dalloc(&dr, sizeof(TcFront));
  if (e == cudaSuccess) e = dalloc(&dt, sizeof(int4) * tasks.size());
  if (e == cudaSuccess) e = dalloc(&dws, (size_t)wsb);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dd, &d, sizeof(d), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dr, &r, sizeof(r), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dt, tasks.data(), sizeof(int4) * tasks.size(), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) {
    FactorLaunch fa;
    std::memset(&fa, 0, sizeof(fa));
    fa.P.fronts = dd;
    fa.store = front_dev;
    fa.n_omega = 1;
    TcLaunch tl;
    tl.fronts = dr;
    tl.ws = dws;
    tl.ws_stride = wsb;
    tl.err = ctx->d_flow_err;
    tl.chunk = kTcChunk;
    tl.part = dpart;
    tl.part_stride = pfl;
    tl.tasks = dt;
    launch_schur_tc_pack(fa, tl, npack, planes, ctx->stream);
    tl.tasks = dt + npack;
    launch_schur_tc(fa, tl, nprod, planes, ctx->stream);
    tl.tasks = dt + npack + nprod;
    launch_schur_split_sum(fa, tl, (int)tasks.size() - npack - nprod, ctx->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_flow_err, ctx->d_flow_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  const cudaError_t es = cudaStreamSynchronize(ctx->stream);
  cudaFree(dd); cudaFree(dr); cudaFree(dt); cudaFree(dws); cudaFree(dpart);
  CK(e);
  CK(es);
  return check_flow_err(ctx);
}

fdfd_status fdfd_selftest_wait(fdfd_ctx* ctx) {
  if (!ctx) return FDFD_ERR_ARG;
  ctx->err.clear();
  CKS(ensure_runtime(ctx));
  CKS(check_flow_err(ctx));
  int* flag = nullptr;
  CK(dalloc(&flag, sizeof(int)));
  const cudaError_t e0 = cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream);
  const cudaError_t e1 = e0 == cudaSuccess ? launch_wait_probe(flag, ctx->d_flow_err, ctx->stream) : e0;
  const cudaError_t e2 = e1 == cudaSuccess ? cudaMemcpyAsync(ctx->h_flow_err, ctx->d_flow_err, sizeof(int),
                                                             cudaMemcpyDeviceToHost, ctx->stream)
                                           : e1;
  const cudaError_t e3 = cudaStreamSynchronize(ctx->stream);
  cudaFree(flag);
  CK(e2);
  CK(e3);
  return check_flow_err(ctx);
}

fdfd_status fdfd_selftest_mbar_wait(fdfd_ctx* ctx) {
  if (!ctx) return FDFD_ERR_ARG;
  ctx->err.clear();
  CKS(ensure_runtime(ctx));
  CKS(check_flow_err(ctx));
  const cudaError_t e1 = launch_mbar_probe(ctx->d_flow_err, ctx->stream);
  const cudaError_t e2 = e1 == cudaSuccess ? cudaMemcpyAsync(ctx->h_flow_err, ctx->d_flow_err, sizeof(int),
                                                             cudaMemcpyDeviceToHost, ctx->stream)
                                           : e1;
  const cudaError_t e3 = cudaStreamSynchronize(ctx->stream);
  CK(e2);
  CK(e3);
  return check_flow_err(ctx);
}

fdfd_status fdfd_selftest_wait_async(fdfd_ctx* ctx) {
  if (!ctx) return FDFD_ERR_ARG;
  ctx->err.clear();
  CKS(ensure_runtime(ctx));
  CKS(check_flow_err(ctx));
  if (!ctx->d_probe) CK(dalloc(&ctx->d_probe, sizeof(int)));
  CK(cudaMemsetAsync(ctx->d_probe, 0, sizeof(int), ctx->stream));
  CK(launch_wait_probe(ctx->d_probe, ctx->d_flow_err, ctx->stream));
  // the error word comes back with the stream, as after a sweep that gave up
  CK(cudaMemcpyAsync(ctx->h_flow_err, ctx->d_flow_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  return FDFD_OK;
}

fdfd_status fdfd_profile_enable(fdfd_ctx* ctx, int on) {
  if (!ctx) return FDFD_ERR_ARG;
  if (ctx->device >= 0) CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof_on = on != 0;
  ctx->prof_recs.clear();
  ctx->ev_used = 0;
  return FDFD_OK;
}

fdfd_status fdfd_profile_get(fdfd_ctx* ctx, fdfd_kernel_profile* out, int max_out, int* n_out) {
  if (!ctx || !n_out || (max_out > 0 && !out)) return FDFD_ERR_ARG;
  if (ctx->device >= 0) CK(cudaStreamSynchronize(ctx->stream));
  fdfd_kernel_profile acc[PK_COUNT];
  std::memset(acc, 0, sizeof(acc));
  for (int k = 0; k < PK_COUNT; ++k) std::snprintf(acc[k].name, sizeof(acc[k].name), "%s", kProfNames[k]);
  for (const auto& r : ctx->prof_recs) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, ctx->ev_pool[r.e0], ctx->ev_pool[r.e1]));
    acc[r.kind].launches += 1;
    acc[r.kind].ms += ms;
    acc[r.kind].flops += r.flops;
    acc[r.kind].bytes += r.bytes;
  }
  int n = 0;
  for (int k = 0; k < PK_COUNT && n < max_out; ++k) out[n++] = acc[k];
  *n_out = PK_COUNT;
  return FDFD_OK;
}

void fdfd_reset_counters(fdfd_ctx* ctx) {
  if (!ctx) return;
  ctx->sf = ctx->nf = ctx->bs = ctx->sweeps = ctx->fallbacks = ctx->repivots = 0;
}

const char* fdfd_last_error(const fdfd_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void fdfd_destroy(fdfd_ctx* ctx) {
  if (!ctx) return;
  if (ctx->device >= 0) cudaStreamSynchronize(ctx->stream);
  free_plan_device(ctx);
  free_factor(ctx);
  free_ws(ctx);
  free_gm(ctx);
  void* ps[] = {ctx->d_cxm, ctx->d_cxp, ctx->d_cym, ctx->d_cyp, ctx->d_sxc, ctx->d_syc, ctx->d_k0dx, ctx->d_k0dx2,
                ctx->d_eps,
                ctx->d_growth_max, ctx->d_flow_err, ctx->d_taps, ctx->d_tapw, ctx->d_probe,
                ctx->d_itx, ctx->d_ita, ctx->d_itb, ctx->d_ito, ctx->d_itF, ctx->d_itg, ctx->d_itepsd};
  for (void* p : ps) free_ptr(p);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  drop_graphs(ctx);
  if (ctx->gstream) {
    cudaStreamSynchronize(ctx->gstream);
    cudaStreamDestroy(ctx->gstream);
    cudaEventDestroy(ctx->gev_in);
    cudaEventDestroy(ctx->gev_out);
  }
  if (ctx->istream) {
    cudaStreamSynchronize(ctx->istream);
    cudaStreamDestroy(ctx->istream);
    cudaEventDestroy(ctx->iev_fork);
    cudaEventDestroy(ctx->iev_join);
  }
  if (ctx->h_growth_max) cudaFreeHost(ctx->h_growth_max);
  if (ctx->h_flow_err) cudaFreeHost(ctx->h_flow_err);
  if (ctx->h_active) cudaFreeHost(ctx->h_active);
  if (ctx->h_nj) cudaFreeHost(ctx->h_nj);
  if (ctx->h_resid) cudaFreeHost(ctx->h_resid);
  delete ctx;
}

}  // extern "C"

// ===========================================================================
// Solve on the cached factors without allocating device memory
// ===========================================================================
//
// Some callers cannot call cudaMalloc at solve time: a real-time design loop
// that must not synchronise the device (cudaMalloc and cudaFree can), a host
// process running under an allocator budget or a pool it does not own, or an
// embedding application that forbids allocation after its set-up phase.  For
// them this entry point applies the cached factorisation once (the raw
// forward and backward sweeps, no refinement) with all of its temporary
// storage in the fixed device array below instead of the context's buffers.
//
// The array is a static __device__ object: every GPU that loads this library
// holds its 32 MiB until the process exits.  Its device address is looked up
// once per device, on the first call made with that device current; make that
// first call before any stream capture.  All calls share the one array and
// nothing in it needs to start at zero (every entry is written before it is
// read); calls that overlap on the GPU (two streams, two host threads, two
// contexts) race on it and must be serialised by the caller.
namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
constexpr int kNoAllocMaxDevices = 64;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mu;

template <typename T>
fdfd_status sweeps_in(fdfd_ctx* ctx, int nrhs, int transpose, const void* in, void* out, void* vb, int* ctr) {
  return sweep_pair<T>(ctx, solve_launch<T>(ctx, vb, nrhs, 0, -1, 0, -1), transpose, in, out, ctr);
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" {

size_t fdfd_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }


fdfd_status fdfd_solve_raw_noalloc(fdfd_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, int transpose) {
  if (!ctx || !b_dev || !x_dev || nrhs <= 0 || b_dev == x_dev) return FDFD_ERR_ARG;
  ctx->err.clear();
  if (!ctx->uploaded || !(ctx->valid32 || ctx->valid64) || ctx->opt.mode == FDFD_MODE_PLAIN)
    return fail(ctx, FDFD_ERR_STATE, "fdfd_solve_raw_noalloc needs a cached factorisation (fdfd_factor first)");
  const bool use64 = ctx->valid64;
  const size_t S = (size_t)ctx->n_omega * nrhs;
  const size_t N = (size_t)n_cells(ctx);
  const size_t es = use64 ? sizeof(double2) : sizeof(float2);
  const size_t vb_bytes = align256(S * (size_t)ctx->plan.vec_total * es);
  const size_t ctr_bytes = align256(sizeof(int) * (1 + 2 * (size_t)ctx->n_omega * ctx->plan.fronts.size()));
  if (vb_bytes + ctr_bytes > kNoAllocScratchBytes)
    return fail(ctx, FDFD_ERR_ARG,
                "fdfd_solve_raw_noalloc: this solve needs " + std::to_string(vb_bytes + ctr_bytes) +
                    " bytes of scratch; the fixed device array holds " + std::to_string(kNoAllocScratchBytes));
  // the context's factors, counters and stream live on ctx->device; the array's
  // address is per device, so the call runs with that device current
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != ctx->device)
    return fail(ctx, FDFD_ERR_STATE, "fdfd_solve_raw_noalloc: the current device (" + std::to_string(dev) +
                                         ") is not the context's device (" + std::to_string(ctx->device) + ")");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(ctx, FDFD_ERR_ARG, "fdfd_solve_raw_noalloc: device index out of range");
  // a bounded wait that gave up in an earlier sweep or factorisation is reported here
  CKS(check_flow_err(ctx));
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      // one-time set-up on this device: the host-side symbol is not a device
      // address, so ask the runtime where the array lives on the current device
      void* p = nullptr;
      CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_addr[dev] = p;
    }
    scratch = reinterpret_cast<unsigned char*>(g_noalloc_addr[dev]);
  }
  if (ctx->growth_pending && !use64) {
    // the factorisation's growth figure decides whether FP32 factors may be used;
    // this call cannot redo the factorisation in FP64 (that allocates)
    if (!ctx->growth_ready) CK(cudaStreamSynchronize(ctx->stream));
    // the same synchronisation brought back the factorisation's error word
    CKS(check_flow_err(ctx));
    const float g = *ctx->h_growth_max;
    if (!(g <= ctx->opt.growth_bound))
      return fail(ctx, FDFD_ERR_PIVOT,
                  "fdfd_solve_raw_noalloc: FP32 factors exceed the growth bound; call fdfd_solve once first");
    // checked once per factorisation: later calls on the same factors do not synchronise
    ctx->growth_pending = false;
    ctx->growth_ready = false;
    ctx->last_growth = g;
  }
  int* ctr = reinterpret_cast<int*>(scratch + vb_bytes);
  if (use64) CKS(sweeps_in<double2>(ctx, nrhs, transpose, b_dev, x_dev, scratch, ctr));
  else CKS(sweeps_in<float2>(ctx, nrhs, transpose, b_dev, x_dev, scratch, ctr));
  if (ctx->h_flow_err) CK(cudaMemcpyAsync(ctx->h_flow_err, ctx->d_flow_err, sizeof(int), cudaMemcpyDeviceToHost,
                                          ctx->stream));
  CK(cudaGetLastError());
  return FDFD_OK;
}

}  // extern "C"
