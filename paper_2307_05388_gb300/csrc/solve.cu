// Triangular sweeps over the cached factors (paper Eq. 5 and Eq. 6; Sec. II,
// "back substitution").  Forward solve A x = b is L then U; the adjoint
// (transpose) solve A^T x = b reuses the same factors as U^T then L^T, so no
// second factorisation is needed (the first caching idea of Sec. II).
//
// Per front, with the factored front [L11\U11 U12; L21 S] and row permutation P:
//   L   : y = L11^-1 (P v)_k,          u = v_m - L21 y
//   U   : x_k = U11^-1 (y - U12 x_m)
//   U^T : w = U11^-T v_k,              u = v_m - U12^T w
//   L^T : x_k = P^T L11^-T (w - L21^T x_m)
// where v gathers the front's entries of the right-hand side plus the update
// vectors u of its children (through the same inverse extend-add maps as the
// factorisation), and x_m are the already final values of the boundary
// variables.  Levels run bottom-up for L / U^T and top-down for U / L^T.  Each
// CTA owns one front of one system; every read of the factor is coalesced
// along a row of the row-major front, and each factor entry is read once per
// right-hand side.
#include "kernels.h"

namespace fdfd {

namespace {

constexpr int kSolveThreads = 256;
constexpr int kWarps = kSolveThreads / 32;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
template <typename T>
__device__ __forceinline__ T shfl(T v, int src) {
  v.x = __shfl_sync(0xffffffffu, v.x, src);
  v.y = __shfl_sync(0xffffffffu, v.y, src);
  return v;
}

// v[a] for a < n: rhs entry (pivot rows only) plus the children's update vectors.
// src maps the front-local slot to the local row whose value it receives.
template <typename T>
__device__ __forceinline__ void gather_front(const SolveLaunch& a, const FrontDesc& d, const T* rhs,
                                             const T* vbs, const int* Pm, bool permute, T* vs) {
  const int* idx = a.P.idx + d.idx_off;
  for (int s = threadIdx.x; s < d.n; s += blockDim.x) {
    const int src = (permute && s < d.k) ? Pm[s] : s;
    T v = src < d.k ? rhs[idx[src]] : czero<T>();
    for (int ci = 0; ci < d.nchild; ++ci) {
      const FrontDesc c = a.P.fronts[a.P.children[d.child0 + ci]];
      const int t = a.P.inv[c.inv_off + src];
      if (t >= 0) v = cadd(v, vbs[c.v_off + c.k + t]);
    }
    vs[s] = v;
  }
}

template <typename T, int SWEEP>
__global__ void __launch_bounds__(kSolveThreads)
sweep_kernel(SolveLaunch a, const int* __restrict__ flist, const T* __restrict__ in, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* vs = reinterpret_cast<T*>(smem_raw);
  const int w = blockIdx.y + a.w0;
  const int f = flist[blockIdx.x];
  const FrontDesc d = a.P.fronts[f];
  const int n = d.n, k = d.k, m = d.m, ld = d.ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* F = reinterpret_cast<const T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const int* Pm = a.perm + (size_t)w * a.perm_stride + d.piv_off;
  const int* idx = a.P.idx + d.idx_off;
  for (int r = a.r0; r < a.r0 + a.nr; ++r) {
    const size_t sys = (size_t)w * a.nrhs + r;
    T* vbs = reinterpret_cast<T*>(a.vb) + sys * a.vec_stride;
    if (SWEEP == 0) {
      // ---- L: forward substitution on P v, then the L21 update ----------------
      gather_front(a, d, in + sys * a.n, vbs, Pm, true, vs);
      __syncthreads();
      for (int kb = 0; kb < k; kb += 32) {
        const int bs = min(32, k - kb);
        for (int rr = warp; rr < bs; rr += kWarps) {
          const int row = kb + rr;
          T acc = czero<T>();
          for (int c = lane; c < kb; c += 32) acc = cfma(F[(size_t)row * ld + c], vs[c], acc);
          acc = warp_sum(acc);
          if (lane == 0) vs[row] = csub(vs[row], acc);
        }
        __syncthreads();
        if (warp == 0) {
          T yi = lane < bs ? vs[kb + lane] : czero<T>();
          for (int jj = 0; jj < bs - 1; ++jj) {
            const T yj = shfl(yi, jj);
            if (lane > jj && lane < bs) yi = cfms(F[(size_t)(kb + lane) * ld + kb + jj], yj, yi);
          }
          if (lane < bs) vs[kb + lane] = yi;
        }
        __syncthreads();
      }
      for (int t = warp; t < m; t += kWarps) {
        const int row = k + t;
        T acc = czero<T>();
        for (int c = lane; c < k; c += 32) acc = cfma(F[(size_t)row * ld + c], vs[c], acc);
        acc = warp_sum(acc);
        if (lane == 0) vs[row] = csub(vs[row], acc);
      }
      __syncthreads();
      for (int s = tid; s < n; s += blockDim.x) vbs[d.v_off + s] = vs[s];
    } else if (SWEEP == 1) {
      // ---- U: x_k = U11^-1 (y - U12 x_m) ------------------------------------
      T* xo = out + sys * a.n;
      for (int s = tid; s < k; s += blockDim.x) vs[s] = vbs[d.v_off + s];
      for (int t = tid; t < m; t += blockDim.x) vs[k + t] = xo[idx[k + t]];
      __syncthreads();
      for (int row = warp; row < k; row += kWarps) {
        T acc = czero<T>();
        for (int t = lane; t < m; t += 32) acc = cfma(F[(size_t)row * ld + k + t], vs[k + t], acc);
        acc = warp_sum(acc);
        if (lane == 0) vs[row] = csub(vs[row], acc);
      }
      __syncthreads();
      for (int kb = ((k - 1) / 32) * 32; kb >= 0; kb -= 32) {
        const int bs = min(32, k - kb);
        for (int rr = warp; rr < bs; rr += kWarps) {
          const int row = kb + rr;
          T acc = czero<T>();
          for (int c = kb + bs + lane; c < k; c += 32) acc = cfma(F[(size_t)row * ld + c], vs[c], acc);
          acc = warp_sum(acc);
          if (lane == 0) vs[row] = csub(vs[row], acc);
        }
        __syncthreads();
        if (warp == 0) {
          T zi = lane < bs ? vs[kb + lane] : czero<T>();
          for (int jj = bs - 1; jj >= 0; --jj) {
            if (lane == jj) zi = cmul(zi, crcp(F[(size_t)(kb + jj) * ld + kb + jj]));
            const T xj = shfl(zi, jj);
            if (lane < jj) zi = cfms(F[(size_t)(kb + lane) * ld + kb + jj], xj, zi);
          }
          if (lane < bs) vs[kb + lane] = zi;
        }
        __syncthreads();
      }
      for (int s = tid; s < k; s += blockDim.x) xo[idx[s]] = vs[s];
    } else if (SWEEP == 2) {
      // ---- U^T: w = U11^-T v_k, u = v_m - U12^T w ----------------------------
      gather_front(a, d, in + sys * a.n, vbs, Pm, false, vs);
      __syncthreads();
      for (int kb = 0; kb < k; kb += 32) {
        const int bs = min(32, k - kb);
        if (warp == 0) {
          T wi = lane < bs ? vs[kb + lane] : czero<T>();
          for (int bb = 0; bb < bs; ++bb) {
            if (lane == bb) wi = cmul(wi, crcp(F[(size_t)(kb + bb) * ld + kb + bb]));
            const T wb = shfl(wi, bb);
            if (lane > bb && lane < bs) wi = cfms(F[(size_t)(kb + bb) * ld + kb + lane], wb, wi);
          }
          if (lane < bs) vs[kb + lane] = wi;
        }
        __syncthreads();
        for (int c = kb + bs + tid; c < n; c += blockDim.x) {
          T acc = vs[c];
          for (int bb = 0; bb < bs; ++bb) acc = cfms(F[(size_t)(kb + bb) * ld + c], vs[kb + bb], acc);
          vs[c] = acc;
        }
        __syncthreads();
      }
      for (int s = tid; s < n; s += blockDim.x) vbs[d.v_off + s] = vs[s];
    } else {
      // ---- L^T: x_k = P^T L11^-T (w - L21^T x_m) ------------------------------
      T* xo = out + sys * a.n;
      for (int s = tid; s < k; s += blockDim.x) vs[s] = vbs[d.v_off + s];
      for (int t = tid; t < m; t += blockDim.x) vs[k + t] = xo[idx[k + t]];
      __syncthreads();
      for (int c = tid; c < k; c += blockDim.x) {
        T acc = vs[c];
        for (int t = 0; t < m; ++t) acc = cfms(F[(size_t)(k + t) * ld + c], vs[k + t], acc);
        vs[c] = acc;
      }
      __syncthreads();
      for (int kb = ((k - 1) / 32) * 32; kb >= 0; kb -= 32) {
        const int bs = min(32, k - kb);
        if (warp == 0) {
          T qi = lane < bs ? vs[kb + lane] : czero<T>();
          for (int bb = bs - 1; bb > 0; --bb) {
            const T qb = shfl(qi, bb);
            if (lane < bb) qi = cfms(F[(size_t)(kb + bb) * ld + kb + lane], qb, qi);
          }
          if (lane < bs) vs[kb + lane] = qi;
        }
        __syncthreads();
        for (int c = tid; c < kb; c += blockDim.x) {
          T acc = vs[c];
          for (int bb = 0; bb < bs; ++bb) acc = cfms(F[(size_t)(kb + bb) * ld + c], vs[kb + bb], acc);
          vs[c] = acc;
        }
        __syncthreads();
      }
      for (int s = tid; s < k; s += blockDim.x) xo[idx[Pm[s]]] = vs[s];
    }
    __syncthreads();
  }
}

}  // namespace

template <typename T>
void launch_sweep(const SolveLaunch& a, int sweep, const int* flist, int nf, int nmax, int kmax,
                  const void* in, void* out, cudaStream_t s) {
  (void)kmax;
  if (nf <= 0) return;
  const size_t smem = (size_t)nmax * sizeof(T);
  const T* i = reinterpret_cast<const T*>(in);
  T* o = reinterpret_cast<T*>(out);
  dim3 grid(nf, a.n_omega);
  switch (sweep) {
    case 0: sweep_kernel<T, 0><<<grid, kSolveThreads, smem, s>>>(a, flist, i, o); break;
    case 1: sweep_kernel<T, 1><<<grid, kSolveThreads, smem, s>>>(a, flist, i, o); break;
    case 2: sweep_kernel<T, 2><<<grid, kSolveThreads, smem, s>>>(a, flist, i, o); break;
    default: sweep_kernel<T, 3><<<grid, kSolveThreads, smem, s>>>(a, flist, i, o); break;
  }
}

cudaError_t solve_init_attributes() {
  const int lim = 160 * 1024;
  cudaError_t e = cudaSuccess;
#define FDFD_ATTR(T, S)                                                                          \
  if (e == cudaSuccess)                                                                          \
    e = cudaFuncSetAttribute(sweep_kernel<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  FDFD_ATTR(float2, 0) FDFD_ATTR(float2, 1) FDFD_ATTR(float2, 2) FDFD_ATTR(float2, 3)
  FDFD_ATTR(double2, 0) FDFD_ATTR(double2, 1) FDFD_ATTR(double2, 2) FDFD_ATTR(double2, 3)
#undef FDFD_ATTR
  return e;
}

template void launch_sweep<float2>(const SolveLaunch&, int, const int*, int, int, int, const void*,
                                   void*, cudaStream_t);
template void launch_sweep<double2>(const SolveLaunch&, int, const int*, int, int, int, const void*,
                                    void*, cudaStream_t);

}  // namespace fdfd
