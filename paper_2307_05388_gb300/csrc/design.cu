// Smoothing filter and projection of the design density (Sec. III: a smoothing
// filter of 200 nm radius and a sigmoid-like projection binarise the geometry
// before each solve; the forms here are a conic filter and a tanh projection):
//   rho~_i = sum_j w_ij rho_j / N_i,  w_ij = max(0, R - |p_i - p_j|),  N_i = sum_j w_ij
//   rho^_i = (tanh(b e) + tanh(b (rho~_i - e))) / (tanh(b e) + tanh(b (1 - e)))
//   eps_i  = eps_lo + rho^_i (eps_hi - eps_lo)
// with sums over the pixels of the design box, and the chain rule back to rho:
//   g_rho_j = sum_i w_ij g_eps_i s_i / N_i,  s_i = d eps_i / d rho~_i.
// One thread per pixel; the tap weights (one per integer offset inside the
// radius, in a fixed order) sit in shared memory, so each pixel's sums run in
// the same order every time.
#include "kernels.h"

namespace fdfd {
namespace {

constexpr int kFiltThreads = 256;

__global__ void __launch_bounds__(kFiltThreads)
filter_project_kernel(const double* __restrict__ rho, int w, int h, const int2* __restrict__ off,
                      const double* __restrict__ wt, int ntap, double beta, double eta, double eps_lo,
                      double deps, double* __restrict__ eps, double* __restrict__ slope, double* __restrict__ norm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_w = reinterpret_cast<double*>(smem_raw);
  int2* s_off = reinterpret_cast<int2*>(s_w + ntap);
  for (int t = threadIdx.x; t < ntap; t += blockDim.x) {
    s_w[t] = wt[t];
    s_off[t] = off[t];
  }
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= w * h) return;
  const int i = p / h, j = p - i * h;
  double s = 0.0, n = 0.0;
  for (int t = 0; t < ntap; ++t) {
    const int ii = i + s_off[t].x, jj = j + s_off[t].y;
    if (ii < 0 || ii >= w || jj < 0 || jj >= h) continue;
    s += s_w[t] * rho[ii * h + jj];
    n += s_w[t];
  }
  const double rt = s / n;
  const double a = tanh(beta * eta);
  const double den = a + tanh(beta * (1.0 - eta));
  const double th = tanh(beta * (rt - eta));
  eps[p] = eps_lo + (a + th) / den * deps;
  slope[p] = beta * (1.0 - th * th) / den * deps;
  norm[p] = n;
}

__global__ void __launch_bounds__(kFiltThreads)
filter_adjoint_kernel(const double* __restrict__ g, const double* __restrict__ slope,
                      const double* __restrict__ norm, int w, int h, const int2* __restrict__ off,
                      const double* __restrict__ wt, int ntap, double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_w = reinterpret_cast<double*>(smem_raw);
  int2* s_off = reinterpret_cast<int2*>(s_w + ntap);
  for (int t = threadIdx.x; t < ntap; t += blockDim.x) {
    s_w[t] = wt[t];
    s_off[t] = off[t];
  }
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= w * h) return;
  const int i = p / h, j = p - i * h;
  double s = 0.0;
  for (int t = 0; t < ntap; ++t) {
    const int ii = i + s_off[t].x, jj = j + s_off[t].y;
    if (ii < 0 || ii >= w || jj < 0 || jj >= h) continue;
    const int q = ii * h + jj;
    s += s_w[t] * g[q] * slope[q] / norm[q];
  }
  out[p] = s;
}

size_t filter_smem(int ntap) { return (size_t)ntap * (sizeof(double) + sizeof(int2)); }

// eps_i = eps_lo + rho_i (eps_hi - eps_lo): the design pixel's permittivity from its density
// without filtering or projection (the parametrisation of the benchmark workloads)
__global__ void density_eps_kernel(const double* __restrict__ rho, long long n, double eps_lo, double deps,
                                   double* __restrict__ eps) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) eps[p] = eps_lo + rho[p] * deps;
}

}  // namespace

void launch_density_eps(const double* rho, long long n, double eps_lo, double deps, double* eps, cudaStream_t s) {
  if (n <= 0) return;
  density_eps_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rho, n, eps_lo, deps, eps);
}

void launch_filter_project(const double* rho, int w, int h, const int2* off, const double* wt, int ntap,
                           double beta, double eta, double eps_lo, double deps, double* eps, double* slope,
                           double* norm, cudaStream_t s) {
  const int n = w * h;
  if (n <= 0) return;
  filter_project_kernel<<<(n + kFiltThreads - 1) / kFiltThreads, kFiltThreads, filter_smem(ntap), s>>>(
      rho, w, h, off, wt, ntap, beta, eta, eps_lo, deps, eps, slope, norm);
}

void launch_filter_adjoint(const double* g, const double* slope, const double* norm, int w, int h, const int2* off,
                           const double* wt, int ntap, double* out, cudaStream_t s) {
  const int n = w * h;
  if (n <= 0) return;
  filter_adjoint_kernel<<<(n + kFiltThreads - 1) / kFiltThreads, kFiltThreads, filter_smem(ntap), s>>>(
      g, slope, norm, w, h, off, wt, ntap, out);
}

}  // namespace fdfd
