// Operator assembly tables (Eq. 1-2 with stretched-coordinate PML), the FP64
// matrix-free stencil used by the refinement, FGMRES vector kernels, the
// mode-overlap objective with its adjoint source (Eq. 4) and the pixel
// gradient (Eq. 3).
//
// Operator (dimensionless: Eq. 1 multiplied by mu0 dx^2), row (i, j):
//   A[(i,j),(i-1,j)] = cxm[i] = -1 / (sx(i+1/2) sx(i)),   A[(i,j),(i+1,j)] = cxp[i] = -1 / (sx(i+1/2) sx(i+1))
//   A[(i,j),(i,j-1)] = cym[j],                            A[(i,j),(i,j+1)] = cyp[j]
//   A[(i,j),(i,j)]   = -(cxm + cxp + cym + cyp) - (k0 dx)^2 eps[i,j]
// with positions in cell units (cell i centred at i + 1/2) and the stretch
//   s(u) = 1 - i * [-(order+1) ln R / (2 k0dx npml)] * d(u)^order,
//   d(u) = max(npml - u, u - (n - npml), 0) / npml,
// i.e. e^{+i w t} convention: s = 1 - i sigma / (omega eps0).  Neighbours
// beyond the grid are zero (PEC behind the PML).
#include "kernels.h"

namespace fdfd {

namespace {

__device__ double2 stretch(double u, int n, int npml, double k0dx, double ln_R, double order) {
  if (npml <= 0) return make_double2(1.0, 0.0);
  double d = fmax(fmax((double)npml - u, u - (double)(n - npml)), 0.0) / (double)npml;
  double smax = -(order + 1.0) * ln_R / (2.0 * k0dx * (double)npml);
  double p = (order == 3.0) ? d * d * d : pow(d, order);
  return make_double2(1.0, -smax * p);
}

__device__ double2 neg_inv_prod(double2 a, double2 b) {
  double2 p = cmul(a, b);
  double2 r = crcp(p);
  return make_double2(-r.x, -r.y);
}

__global__ void coef_kernel(double2* cxm, double2* cxp, double2* cym, double2* cyp, double* k0dx2,
                            double2* sxc, double2* syc, const double* k0dx, int n_omega, int nx, int ny, int px,
                            int py, double ln_R, double order) {
  const int w = blockIdx.y;
  const double kd = k0dx[w];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) k0dx2[w] = kd * kd;
  if (t < nx) {
    const double2 sc = stretch(t + 0.5, nx, px, kd, ln_R, order);
    cxm[(size_t)w * nx + t] = neg_inv_prod(sc, stretch(t, nx, px, kd, ln_R, order));
    cxp[(size_t)w * nx + t] = neg_inv_prod(sc, stretch(t + 1.0, nx, px, kd, ln_R, order));
    sxc[(size_t)w * nx + t] = sc;
  }
  if (t < ny) {
    const double2 sc = stretch(t + 0.5, ny, py, kd, ln_R, order);
    cym[(size_t)w * ny + t] = neg_inv_prod(sc, stretch(t, ny, py, kd, ln_R, order));
    cyp[(size_t)w * ny + t] = neg_inv_prod(sc, stretch(t + 1.0, ny, py, kd, ln_R, order));
    syc[(size_t)w * ny + t] = sc;
  }
}

__global__ void scatter_design_kernel(double* eps, const double* ed, int ny, int x0, int y0, int w, int h) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)w * h) return;
  const int i = (int)(t / h), j = (int)(t - (long long)i * h);
  eps[(size_t)(x0 + i) * ny + y0 + j] = ed[t];
}

// (A X)[cell] (transpose: A^T) for wavelength w, X one system's vector
__device__ __forceinline__ double2 stencil_at(const DevCoef& c, int w, int transpose, const double2* __restrict__ X,
                                              long long cell) {
  const int ci = (int)cell;                    // grids stay below 2^31 cells
  const int i = ci / c.ny, j = ci - i * c.ny;
  const double2* cxm = c.cxm + (size_t)w * c.nx;
  const double2* cxp = c.cxp + (size_t)w * c.nx;
  const double2* cym = c.cym + (size_t)w * c.ny;
  const double2* cyp = c.cyp + (size_t)w * c.ny;
  double2 dg;
  dg.x = -(cxm[i].x + cxp[i].x + cym[j].x + cyp[j].x) - c.k0dx2[w] * c.eps[cell];
  dg.y = -(cxm[i].y + cxp[i].y + cym[j].y + cyp[j].y);
  double2 acc = cmul(dg, X[cell]);
  if (!transpose) {
    if (i > 0) acc = cfma(cxm[i], X[cell - c.ny], acc);
    if (i + 1 < c.nx) acc = cfma(cxp[i], X[cell + c.ny], acc);
    if (j > 0) acc = cfma(cym[j], X[cell - 1], acc);
    if (j + 1 < c.ny) acc = cfma(cyp[j], X[cell + 1], acc);
  } else {
    if (i > 0) acc = cfma(cxp[i - 1], X[cell - c.ny], acc);
    if (i + 1 < c.nx) acc = cfma(cxm[i + 1], X[cell + c.ny], acc);
    if (j > 0) acc = cfma(cyp[j - 1], X[cell - 1], acc);
    if (j + 1 < c.ny) acc = cfma(cym[j + 1], X[cell + 1], acc);
  }
  return acc;
}

// y = A x (op 0) or y = b - A x (op 1); transpose selects A^T.
__global__ void stencil_kernel(DevCoef c, int nrhs, int transpose, const double2* __restrict__ x,
                               const double2* __restrict__ b, double2* __restrict__ y, int op) {
  const int sys = blockIdx.y;
  const long long N = (long long)c.nx * c.ny;
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= N) return;
  double2 acc = stencil_at(c, sys / nrhs, transpose, x + (size_t)sys * N, cell);
  if (op == 1) {
    const double2 bb = b[(size_t)sys * N + cell];
    acc = make_double2(bb.x - acc.x, bb.y - acc.y);
  }
  y[(size_t)sys * N + cell] = acc;
}

constexpr int kDotThreads = 256;
constexpr int kMaxDot = 17;

// Partial sums of h[s][i] = sum_t conj(V_i[s][t]) w[s][t]: one CTA per
// (chunk of kDotPer * 256 entries, vector i, system), one accumulator per
// thread (low register use keeps the FP64 pipes fed by many warps), CTA
// reduction in a fixed order.
constexpr int kDotPer = 4;
constexpr int kArnPer = 2;   // entries per thread of an Arnoldi pass: FP64 FMA is 2 per SM per clock, so
                             // the CTAs cover every SM while the FP64 adds of the reductions stay few

__global__ void __launch_bounds__(kDotThreads)
multidot_partial_kernel(const double2* __restrict__ V, long long vstride, int nv,
                        const double2* __restrict__ w, long long n, double2* partial, int nblk) {
  __shared__ double2 red[kDotThreads / 32];
  const int i = blockIdx.y, sys = blockIdx.z;
  const double2* W = w + (size_t)sys * n;
  const double2* Vi = V + (size_t)i * vstride + (size_t)sys * n;
  const long long t0 = (long long)blockIdx.x * (kDotThreads * kDotPer) + threadIdx.x;
  double2 vv[kDotPer], ww[kDotPer];
#pragma unroll
  for (int u = 0; u < kDotPer; ++u) {
    const long long t = t0 + (long long)u * kDotThreads;
    vv[u] = t < n ? Vi[t] : make_double2(0, 0);
    ww[u] = t < n ? W[t] : make_double2(0, 0);
  }
  double2 acc = make_double2(0, 0);
#pragma unroll
  for (int u = 0; u < kDotPer; ++u) acc = cfma(cconj(vv[u]), ww[u], acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = red[0];
    for (int q = 1; q < kDotThreads / 32; ++q) s = cadd(s, red[q]);
    partial[((size_t)sys * kMaxDot + i) * nblk + blockIdx.x] = s;
  }
}

// One warp per (system, vector): lane-strided partial sums, then a shuffle tree
// (fixed order, so the result does not depend on timing).
__global__ void multidot_final_kernel(const double2* partial, int nblk, int nv, double2* out, int out_ld) {
  const int sys = blockIdx.x;
  const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (i >= nv) return;
  double2 s = make_double2(0, 0);
  const double2* p = partial + ((size_t)sys * kMaxDot + i) * nblk;
  for (int b = lane; b < nblk; b += 32) s = cadd(s, p[b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
  }
  if (lane == 0) out[(size_t)sys * out_ld + i] = s;
}

// w[s] -= sum_i h[s][i] V_i[s]; the coefficients sit in shared memory.
__global__ void multiaxpy_kernel(const double2* __restrict__ V, long long vstride, int nv,
                                 const double2* __restrict__ h, int h_ld, double2* w, long long n,
                                 const int* active) {
  __shared__ double2 hh[kMaxDot];
  const int sys = blockIdx.y;
  if (active && !active[sys]) return;
  if (threadIdx.x < nv) hh[threadIdx.x] = h[(size_t)sys * h_ld + threadIdx.x];
  __syncthreads();
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double2 acc = w[(size_t)sys * n + t];
    for (int i = 0; i < nv; ++i) acc = cfms(hh[i], V[(size_t)i * vstride + (size_t)sys * n + t], acc);
    w[(size_t)sys * n + t] = acc;
  }
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 4096 ? b : 4096);
}

}  // namespace

void launch_coef(double2* cxm, double2* cxp, double2* cym, double2* cyp, double* k0dx2, double2* sxc,
                 double2* syc, const double* k0dx_dev, int n_omega, int nx, int ny, int npml_x, int npml_y,
                 double ln_R, double order, cudaStream_t s) {
  const int nmax = nx > ny ? nx : ny;
  coef_kernel<<<dim3((nmax + 127) / 128, n_omega), 128, 0, s>>>(cxm, cxp, cym, cyp, k0dx2, sxc, syc, k0dx_dev,
                                                               n_omega, nx, ny, npml_x, npml_y, ln_R, order);
}

void launch_scatter_design(double* eps, const double* eps_design, int ny, int x0, int y0, int w, int h,
                           cudaStream_t s) {
  const long long n = (long long)w * h;
  if (n <= 0) return;
  scatter_design_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(eps, eps_design, ny, x0, y0, w, h);
}

void launch_stencil(const DevCoef& c, int n_omega, int nrhs, int transpose, const double2* x,
                    const double2* b, double2* y, int op, cudaStream_t s) {
  const long long N = (long long)c.nx * c.ny;
  stencil_kernel<<<dim3((unsigned)((N + 255) / 256), n_omega * nrhs), 256, 0, s>>>(c, nrhs, transpose, x, b, y, op);
}


// chunks of kDotPer entries per thread
int multidot_blocks(long long n) {
  long long b = (n + kDotThreads * kDotPer - 1) / (kDotThreads * kDotPer);
  if (b < 1) b = 1;
  return (int)b;
}
int multidot_max_vectors() { return kMaxDot; }
int arnoldi_blocks(long long n) { return (int)((n + kDotThreads * kArnPer - 1) / (kDotThreads * kArnPer)); }

void launch_multidot(const double2* V, long long vstride, int nv, const double2* w, long long n, int nsys,
                     double2* partial, int nblk, double2* out, int out_ld, cudaStream_t s) {
  multidot_partial_kernel<<<dim3(nblk, nv, nsys), kDotThreads, 0, s>>>(V, vstride, nv, w, n, partial, nblk);
  multidot_final_kernel<<<nsys, 32 * kMaxDot, 0, s>>>(partial, nblk, nv, out, out_ld);
}

void launch_multiaxpy(const double2* V, long long vstride, int nv, const double2* h, int h_ld, double2* w,
                      long long n, int nsys, const int* active, cudaStream_t s) {
  multiaxpy_kernel<<<dim3(grid_for(n), nsys), 256, 0, s>>>(V, vstride, nv, h, h_ld, w, n, active);
}

// ---------------------------------------------------------------------------
// FGMRES bookkeeping per system (one thread per system).
// ---------------------------------------------------------------------------
namespace {

__global__ void gm_start_kernel(const double2* rr, int rr_ld, const double2* bb, int bb_ld, int nsys,
                                double tol, int m, double2* g, double* vscale, int* active, double* resid,
                                double* bnorm, int first) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  // norms from sums of squares; a NaN stays NaN (fmax would turn it into 0, and a
  // poisoned solve would then look converged)
  const double rr2 = rr[(size_t)s * rr_ld].x, bb2 = bb[(size_t)s * bb_ld].x;
  const double beta = rr2 > 0.0 ? sqrt(rr2) : (rr2 == rr2 ? 0.0 : rr2);
  if (first) bnorm[s] = bb2 > 0.0 ? sqrt(bb2) : (bb2 == bb2 ? 0.0 : bb2);
  const double bn = bnorm[s];
  for (int i = 0; i <= m; ++i) g[(size_t)s * (m + 1) + i] = make_double2(0, 0);
  g[(size_t)s * (m + 1)] = make_double2(beta, 0);
  resid[s] = bn > 0 ? beta / bn : 0.0;
  const int act = (bn > 0) && (beta > tol * bn) && (beta == beta);
  active[s] = act;
  vscale[s] = act ? 1.0 / beta : 0.0;
}

// Column j of the Hessenberg matrix of system s from its projections h[0..j]
// and hn2 = |w|^2: earlier rotations applied, a new one formed, the residual
// estimate updated; a system whose estimate meets tol (or breaks down: exact
// solution) becomes inactive.
__device__ void givens_step(int s, const double2* hs, double hn2, int j, int m, double tol, double2* H, double2* cs,
                            double2* sn, double2* g, double* vscale, int* active, double* resid, const double* bnorm) {
  double2* Hc = H + ((size_t)s * m + j) * (m + 1);   // column j of H
  for (int i = 0; i <= j; ++i) Hc[i] = hs[i];
  const double hnorm = hn2 > 0.0 ? sqrt(hn2) : (hn2 == hn2 ? 0.0 : hn2);
  Hc[j + 1] = make_double2(hnorm, 0);
  double2* C = cs + (size_t)s * m;
  double2* S = sn + (size_t)s * m;
  for (int i = 0; i < j; ++i) {   // apply earlier rotations
    const double2 x = Hc[i], y = Hc[i + 1];
    const double c = C[i].x;
    Hc[i] = cadd(make_double2(c * x.x, c * x.y), cmul(S[i], y));
    Hc[i + 1] = csub(make_double2(c * y.x, c * y.y), cmul(cconj(S[i]), x));
  }
  const double2 a = Hc[j];
  const double b = hnorm;
  const double aa = sqrt(a.x * a.x + a.y * a.y);
  double c;
  double2 sv, r;
  if (aa == 0.0) {
    c = 0.0; sv = make_double2(1, 0); r = make_double2(b, 0);
  } else {
    const double t = sqrt(aa * aa + b * b);
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    c = aa / t;
    sv = make_double2(ph.x * b / t, ph.y * b / t);
    r = make_double2(ph.x * t, ph.y * t);
  }
  C[j] = make_double2(c, 0);
  S[j] = sv;
  Hc[j] = r;
  Hc[j + 1] = make_double2(0, 0);
  double2* G = g + (size_t)s * (m + 1);
  const double2 gj = G[j];
  G[j + 1] = make_double2(-(sv.x * gj.x + sv.y * gj.y), -(sv.x * gj.y - sv.y * gj.x));  // -conj(s) g_j
  G[j] = make_double2(c * gj.x, c * gj.y);
  const double rn = sqrt(G[j + 1].x * G[j + 1].x + G[j + 1].y * G[j + 1].y);
  const double bn = bnorm[s];
  resid[s] = rn / bn;
  vscale[s] = hnorm > 0 ? 1.0 / hnorm : 0.0;
  if (!(rn > tol * bn) || !(hnorm > 0)) active[s] = 0;   // converged (or breakdown: solution exact)
}

// y = R^-1 g over the first nj columns, then x += sum_i y_i Z_i is done by multiaxpy with -y.
__global__ void gm_solve_kernel(const double2* H, const double2* g, int nsys, int m, const int* njs,
                                double2* ny_out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  const int nj = njs[s];
  const double2* Hs = H + (size_t)s * m * (m + 1);
  const double2* G = g + (size_t)s * (m + 1);
  double2 y[kMaxDot];
  for (int i = nj - 1; i >= 0; --i) {
    double2 acc = G[i];
    for (int q = i + 1; q < nj; ++q) acc = cfms(Hs[(size_t)q * (m + 1) + i], y[q], acc);
    y[i] = cmul(acc, crcp(Hs[(size_t)i * (m + 1) + i]));
  }
  for (int i = 0; i < kMaxDot; ++i)
    ny_out[(size_t)s * kMaxDot + i] = i < nj ? make_double2(-y[i].x, -y[i].y) : make_double2(0, 0);
}

__global__ void scale_vec_kernel(double2* dst, const double2* src, const double* scale, long long n) {
  const int sys = blockIdx.y;
  const double sc = scale[sys];
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double2 v = src[(size_t)sys * n + t];
    dst[(size_t)sys * n + t] = make_double2(v.x * sc, v.y * sc);
  }
}


// One Arnoldi step of FGMRES with classical Gram-Schmidt applied twice, for
// every active system, in three passes over the vectors (pass p):
//   0: w = A z_j,             h1_i = V_i^H w
//   1: w -= sum_i h1_i V_i,   h2_i = V_i^H w
//   2: w -= sum_i h2_i V_i,   |w|^2, then h = h1 + h2 and the Givens update
// (the second projection is always needed here: with a preconditioner this
// close to A^-1, A z_j lies almost in the span of V and the first projection
// cancels most of w).
// CTA (chunk of kArnPer * 256 entries, system); each CTA writes its partial
// sums, and the last CTA of a system (a counter it resets afterwards) adds
// them in chunk order, so results do not depend on timing.
__global__ void __launch_bounds__(kDotThreads)
arnoldi_kernel(ArnoldiStep g, int pass) {
  __shared__ double2 red[kDotThreads / 32][kMaxDot];
  __shared__ double2 hc[kMaxDot];
  __shared__ int s_last;
  const int sys = blockIdx.y;
  if (!g.active[sys]) return;
  const int nv = g.nv, nblk = gridDim.x;
  const long long n = (long long)g.C.nx * g.C.ny;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (pass > 0 && tid < nv) hc[tid] = (pass == 1 ? g.h1 : g.h2)[(size_t)sys * kMaxDot + tid];
  __syncthreads();
  double2* W = g.w + (size_t)sys * n;
  const double2* Vs = g.V + (size_t)sys * n;
  const long long t0 = (long long)blockIdx.x * (kDotThreads * kArnPer) + tid;
  double2 wv[kArnPer];
#pragma unroll
  for (int u = 0; u < kArnPer; ++u) {
    const long long t = t0 + (long long)u * kDotThreads;
    double2 x = make_double2(0, 0);
    if (t < n) {
      if (pass == 0) {
        x = stencil_at(g.C, sys / g.nrhs, g.transpose, g.z + (size_t)sys * n, t);
      } else {
        x = W[t];
        for (int i = 0; i < nv; ++i) x = cfms(hc[i], Vs[(size_t)i * g.vstride + t], x);
      }
      W[t] = x;
    }
    wv[u] = x;
  }
  const int nout = pass < 2 ? nv : 1;
  for (int i = 0; i < nout; ++i) {
    double2 acc = make_double2(0, 0);
    if (pass < 2) {
#pragma unroll
      for (int u = 0; u < kArnPer; ++u) {
        const long long t = t0 + (long long)u * kDotThreads;
        if (t < n) acc = cfma(cconj(Vs[(size_t)i * g.vstride + t]), wv[u], acc);
      }
    } else {
#pragma unroll
      for (int u = 0; u < kArnPer; ++u) acc.x += wv[u].x * wv[u].x + wv[u].y * wv[u].y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) red[warp][i] = acc;
  }
  __syncthreads();
  if (tid < nout) {
    double2 sum = red[0][tid];
    for (int q = 1; q < kDotThreads / 32; ++q) sum = cadd(sum, red[q][tid]);
    g.partial[((size_t)sys * kMaxDot + tid) * nblk + blockIdx.x] = sum;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&g.cnt[sys], 1) == nblk - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double2* out = pass == 0 ? g.h1 : (pass == 1 ? g.h2 : g.hn);
  for (int o = warp; o < nout; o += kDotThreads / 32) {   // warp adds outputs o, o + 8, ...: lane-strided, then a shuffle tree
    const double2* p = g.partial + ((size_t)sys * kMaxDot + o) * nblk;
    double2 sum = make_double2(0, 0);
    for (int b = lane; b < nblk; b += 32) sum = cadd(sum, __ldcg(p + b));
#pragma unroll
    for (int q = 16; q > 0; q >>= 1) {
      sum.x += __shfl_xor_sync(0xffffffffu, sum.x, q);
      sum.y += __shfl_xor_sync(0xffffffffu, sum.y, q);
    }
    if (lane == 0) out[(size_t)sys * kMaxDot + o] = sum;
  }
  if (tid == 0) g.cnt[sys] = 0;
  if (pass == 2) {
    __syncthreads();
    if (tid == 0) {
      double2 hs[kMaxDot];
      for (int i = 0; i < nv; ++i) hs[i] = cadd(g.h1[(size_t)sys * kMaxDot + i], g.h2[(size_t)sys * kMaxDot + i]);
      g.nj[sys] += 1;
      givens_step(sys, hs, g.hn[(size_t)sys * kMaxDot].x, nv - 1, g.m, g.tol, g.H, g.cs, g.sn, g.g, g.vscale,
                  g.active, g.resid, g.bnorm);
    }
  }
}

}  // namespace

void gm_start(const double2* rr, int rr_ld, const double2* bb, int bb_ld, int nsys, double tol, int m,
              double2* g, double* vscale, int* active, double* resid, double* bnorm, int first, cudaStream_t s) {
  gm_start_kernel<<<(nsys + 63) / 64, 64, 0, s>>>(rr, rr_ld, bb, bb_ld, nsys, tol, m, g, vscale, active, resid,
                                                  bnorm, first);
}
void gm_solve(const double2* H, const double2* g, int nsys, int m, const int* njs, double2* ny_out,
              cudaStream_t s) {
  gm_solve_kernel<<<(nsys + 63) / 64, 64, 0, s>>>(H, g, nsys, m, njs, ny_out);
}
void gm_scale(double2* dst, const double2* src, const double* scale, long long n, int nsys, cudaStream_t s) {
  scale_vec_kernel<<<dim3(grid_for(n), nsys), 256, 0, s>>>(dst, src, scale, n);
}
void launch_arnoldi(const ArnoldiStep& g, int nsys, int pass, cudaStream_t s) {
  const long long n = (long long)g.C.nx * g.C.ny;
  arnoldi_kernel<<<dim3(arnoldi_blocks(n), nsys), kDotThreads, 0, s>>>(g, pass);
}

// ---------------------------------------------------------------------------
// Objective (mode overlap), adjoint source and pixel gradient.
// ---------------------------------------------------------------------------
namespace {

__global__ void overlap_kernel(const double2* __restrict__ x, long long N, int ny, const int* cols,
                               const double2* __restrict__ gline, double2* o) {
  __shared__ double2 red[8];
  const int sys = blockIdx.x;
  const int col = cols[sys];
  if (col < 0 || (long long)(col + 1) * ny > N) {   // monitor column outside the grid
    if (threadIdx.x == 0) o[sys] = make_double2(NAN, NAN);
    return;
  }
  const double2* X = x + (size_t)sys * N + (size_t)col * ny;
  const double2* G = gline + (size_t)sys * ny;
  double2 acc = make_double2(0, 0);
  for (int j = threadIdx.x; j < ny; j += blockDim.x) acc = cfma(G[j], X[j], acc);
  for (int off = 16; off > 0; off >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0, 0);
    for (int q = 0; q < 8; ++q) s = cadd(s, red[q]);
    o[sys] = s;
  }
}

// F = sum_q w_q |o_q|^2, or with targets t_q the squared transmission error
// F = sum_q w_q (|o_q|^2 - t_q)^2 (summed in system order by one thread)
__global__ void objective_kernel(const double2* o, const double* weight, const double* target, int nsys, double* F) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0;
  for (int q = 0; q < nsys; ++q) {
    const double p = o[q].x * o[q].x + o[q].y * o[q].y;
    const double wt = weight ? weight[q] : 1.0;
    if (target) {
      const double d = p - target[q];
      s += wt * d * d;
    } else {
      s += wt * p;
    }
  }
  *F = s;
}

// (dF/dE)^T on the monitor column (Wirtinger derivative, E* held fixed):
// w conj(o) g for F = w |o|^2, and 2 w (|o|^2 - t) conj(o) g for F = w (|o|^2 - t)^2
__global__ void adjoint_source_kernel(const double2* o, const double* weight, const double* target, long long N,
                                      int ny, const int* cols, const double2* __restrict__ gline, double2* badj) {
  const int sys = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ny || cols[sys] < 0 || (long long)(cols[sys] + 1) * ny > N) return;
  double wt = weight ? weight[sys] : 1.0;
  if (target) wt *= 2.0 * (o[sys].x * o[sys].x + o[sys].y * o[sys].y - target[sys]);
  const double2 oc = make_double2(wt * o[sys].x, -wt * o[sys].y);
  badj[(size_t)sys * N + (size_t)cols[sys] * ny + j] = cmul(oc, gline[(size_t)sys * ny + j]);
}

__global__ void grad_kernel(const double2* __restrict__ xf, const double2* __restrict__ xa, long long N, int ny,
                            int x0, int y0, int w, int h, int n_omega, int nrhs, const double* k0dx2,
                            const double* weight, double* grad, int accumulate) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)w * h) return;
  const int i = (int)(t / h), j = (int)(t - (long long)i * h);
  const size_t cell = (size_t)(x0 + i) * ny + y0 + j;
  double acc = 0;
  for (int om = 0; om < n_omega; ++om)
    for (int r = 0; r < nrhs; ++r) {
      const size_t sys = (size_t)om * nrhs + r;
      const double2 p = cmul(xa[sys * N + cell], xf[sys * N + cell]);
      acc += (weight ? weight[sys] : 1.0) * 2.0 * k0dx2[om] * p.x;
    }
  grad[t] = accumulate ? grad[t] + acc : acc;
}

}  // namespace

void launch_objective(const double2* x, long long N, int ny, const int* cols, const double2* gline,
                      const double* weight, const double* target, int nsys, double2* o, double* F, double2* badj,
                      cudaStream_t s) {
  overlap_kernel<<<nsys, 256, 0, s>>>(x, N, ny, cols, gline, o);
  objective_kernel<<<1, 32, 0, s>>>(o, weight, target, nsys, F);
  if (badj) {
    cudaMemsetAsync(badj, 0, sizeof(double2) * (size_t)nsys * N, s);
    adjoint_source_kernel<<<dim3((ny + 255) / 256, nsys), 256, 0, s>>>(o, weight, target, N, ny, cols, gline,
                                                                        badj);
  }
}

void launch_grad(const double2* xf, const double2* xa, long long N, int ny, int x0, int y0, int w, int h,
                 int n_omega, int nrhs, const double* k0dx2, const double* weight, double* grad, int accumulate,
                 cudaStream_t s) {
  const long long n = (long long)w * h;
  if (n <= 0) return;
  grad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xf, xa, N, ny, x0, y0, w, h, n_omega, nrhs, k0dx2,
                                                          weight, grad, accumulate);
}

}  // namespace fdfd
