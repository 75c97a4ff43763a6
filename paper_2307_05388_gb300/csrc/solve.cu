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
// variables.  Levels run bottom-up for L / U^T and top-down for U / L^T.
//
// Work split per level: a triangular kernel (one CTA per front and system)
// does the gather and the dense triangular solve; for large fronts the
// rectangular products (L21 y, U12 x_m, U12^T w, L21^T x_m) are split over
// many CTAs of a second kernel, 32 rows or 32 columns each, so that the big
// fronts at the top of the tree stream their factor with the whole GPU.
// Every factor read is coalesced along a row of the row-major front and each
// factor entry is read once per right-hand side; reductions run in a fixed
// order (deterministic results).
#include "kernels.h"

namespace fdfd {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRect = 32;           // rows (or columns) per rectangular task

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

// sum_{c in [c0, c1)} row[c] * vec[c], lanes striding the row (coalesced), warp-reduced.
// Eight loads per lane are issued before they are used, so that a single
// front's row keeps enough bytes in flight to cover the memory latency.
template <typename T>
__device__ __forceinline__ T warp_dot(const T* __restrict__ row, const T* vec, int c0, int c1, int lane) {
  constexpr int UN = 8;
  T acc[2] = {czero<T>(), czero<T>()};
  int c = c0 + lane;
  for (; c + 32 * (UN - 1) < c1; c += 32 * UN) {
    T r[UN];
#pragma unroll
    for (int u = 0; u < UN; ++u) r[u] = row[c + 32 * u];
#pragma unroll
    for (int u = 0; u < UN; ++u) acc[u & 1] = cfma(r[u], vec[c + 32 * u], acc[u & 1]);
  }
  for (; c < c1; c += 32) acc[0] = cfma(row[c], vec[c], acc[0]);
  return warp_sum(cadd(acc[0], acc[1]));
}

// vs[c] -= sum_{bb < bs} F[(kb + bb) * ld + c] * vs[kb + bb]: one column per thread,
// loads issued eight at a time ahead of their multiply-adds.
template <typename T>
__device__ __forceinline__ void col_update(const T* __restrict__ F, int ld, int kb, int bs, int c, T* vs) {
  constexpr int UN = 8;
  T a0 = vs[c], a1 = czero<T>();
  int bb = 0;
  for (; bb + UN <= bs; bb += UN) {
    T f[UN];
#pragma unroll
    for (int u = 0; u < UN; ++u) f[u] = F[(size_t)(kb + bb + u) * ld + c];
#pragma unroll
    for (int u = 0; u < UN; u += 2) {
      a0 = cfms(f[u], vs[kb + bb + u], a0);
      a1 = cfms(f[u + 1], vs[kb + bb + u + 1], a1);
    }
  }
  for (; bb < bs; ++bb) a0 = cfms(F[(size_t)(kb + bb) * ld + c], vs[kb + bb], a0);
  vs[c] = cadd(a0, a1);
}

// v[s] for s < n: rhs entry (pivot rows only) plus the children's update vectors.
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

// ---------------------------------------------------------------------------
// Triangular part (and, for small fronts, the whole front).
// list entries: front id, with bit 31 set when a rectangular task list covers
// the front's off-diagonal block.
// ---------------------------------------------------------------------------
template <typename T, int SWEEP>
__global__ void __launch_bounds__(kThreads)
tri_kernel(SolveLaunch a, const int* __restrict__ flist, const T* __restrict__ in, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T Ds[32][33];
  T* vs = reinterpret_cast<T*>(smem_raw);
  const int w = blockIdx.y + a.w0;
  const int entry = flist[blockIdx.x];
  const bool big = entry < 0;
  const int f = entry & 0x7fffffff;
  const FrontDesc d = a.P.fronts[f];
  const int n = d.n, k = d.k, m = d.m, ld = d.ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* F = reinterpret_cast<const T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const int* Pm = a.perm + (size_t)w * a.perm_stride + d.piv_off;
  const int* idx = a.P.idx + d.idx_off;
  for (int r = a.r0; r < a.r0 + a.nr; ++r) {
    const size_t sys = (size_t)w * a.nrhs + r;
    T* vbs = reinterpret_cast<T*>(a.vb) + sys * a.vec_stride;
    T* vf = vbs + d.v_off;
    if (SWEEP == 0) {
      // ---- L: y = L11^-1 (P v)_k; small fronts also u = v_m - L21 y ---------------
      gather_front(a, d, in + sys * a.n, vbs, Pm, true, vs);
      __syncthreads();
      for (int kb = 0; kb < k; kb += 32) {
        const int bs = min(32, k - kb);
        for (int e = tid; e < bs * 32; e += kThreads) {
          const int i = e >> 5, j = e & 31;
          if (j < bs) Ds[i][j] = F[(size_t)(kb + i) * ld + kb + j];
        }
        for (int rr = warp; rr < bs; rr += kWarps) {
          const T acc = warp_dot(F + (size_t)(kb + rr) * ld, vs, 0, kb, lane);
          if (lane == 0) vs[kb + rr] = csub(vs[kb + rr], acc);
        }
        __syncthreads();
        if (warp == 0) {
          T yi = lane < bs ? vs[kb + lane] : czero<T>();
          for (int jj = 0; jj < bs - 1; ++jj) {
            const T yj = shfl(yi, jj);
            if (lane > jj && lane < bs) yi = cfms(Ds[lane][jj], yj, yi);
          }
          if (lane < bs) vs[kb + lane] = yi;
        }
        __syncthreads();
      }
      if (!big) {
        for (int t = warp; t < m; t += kWarps) {
          const T acc = warp_dot(F + (size_t)(k + t) * ld, vs, 0, k, lane);
          if (lane == 0) vs[k + t] = csub(vs[k + t], acc);
        }
        __syncthreads();
      }
      for (int s = tid; s < n; s += kThreads) vf[s] = vs[s];
    } else if (SWEEP == 1) {
      // ---- U: x_k = U11^-1 (y - U12 x_m); big fronts had U12 x_m subtracted --------
      T* xo = out + sys * a.n;
      for (int s = tid; s < k; s += kThreads) vs[s] = vf[s];
      if (!big)
        for (int t = tid; t < m; t += kThreads) vs[k + t] = xo[idx[k + t]];
      __syncthreads();
      if (!big) {
        for (int row = warp; row < k; row += kWarps) {
          const T acc = warp_dot(F + (size_t)row * ld, vs, k, n, lane);
          if (lane == 0) vs[row] = csub(vs[row], acc);
        }
        __syncthreads();
      }
      for (int kb = ((k - 1) / 32) * 32; kb >= 0; kb -= 32) {
        const int bs = min(32, k - kb);
        for (int e = tid; e < bs * 32; e += kThreads) {
          const int i = e >> 5, j = e & 31;
          if (j < bs) Ds[i][j] = F[(size_t)(kb + i) * ld + kb + j];
        }
        for (int rr = warp; rr < bs; rr += kWarps) {
          const T acc = warp_dot(F + (size_t)(kb + rr) * ld, vs, kb + bs, k, lane);
          if (lane == 0) vs[kb + rr] = csub(vs[kb + rr], acc);
        }
        __syncthreads();
        if (warp == 0) {
          T zi = lane < bs ? vs[kb + lane] : czero<T>();
          const T dj = lane < bs ? crcp(Ds[lane][lane]) : czero<T>();
          for (int jj = bs - 1; jj >= 0; --jj) {
            if (lane == jj) zi = cmul(zi, dj);
            const T xj = shfl(zi, jj);
            if (lane < jj) zi = cfms(Ds[lane][jj], xj, zi);
          }
          if (lane < bs) vs[kb + lane] = zi;
        }
        __syncthreads();
      }
      for (int s = tid; s < k; s += kThreads) xo[idx[s]] = vs[s];
    } else if (SWEEP == 2) {
      // ---- U^T: w = U11^-T v_k; small fronts also u = v_m - U12^T w ---------------
      gather_front(a, d, in + sys * a.n, vbs, Pm, false, vs);
      __syncthreads();
      const int cend = big ? k : n;
      for (int kb = 0; kb < k; kb += 32) {
        const int bs = min(32, k - kb);
        if (warp == 0) {
          // stage the diagonal block (row by row, coalesced) so the dependent chain
          // below touches only shared memory and registers
          for (int i = 0; i < bs; ++i)
            if (lane < bs) Ds[i][lane] = F[(size_t)(kb + i) * ld + kb + lane];
          __syncwarp();
          const T dj = lane < bs ? crcp(Ds[lane][lane]) : czero<T>();
          T wi = lane < bs ? vs[kb + lane] : czero<T>();
          for (int bb = 0; bb < bs; ++bb) {
            if (lane == bb) wi = cmul(wi, dj);
            const T wb = shfl(wi, bb);
            if (lane > bb && lane < bs) wi = cfms(Ds[bb][lane], wb, wi);
          }
          if (lane < bs) vs[kb + lane] = wi;
          __syncwarp();
        }
        __syncthreads();
        for (int c = kb + bs + tid; c < cend; c += kThreads) col_update(F, ld, kb, bs, c, vs);
        __syncthreads();
      }
      for (int s = tid; s < n; s += kThreads) vf[s] = vs[s];
    } else {
      // ---- L^T: x_k = P^T L11^-T (w - L21^T x_m); big fronts had L21^T x_m subtracted --
      T* xo = out + sys * a.n;
      for (int s = tid; s < k; s += kThreads) vs[s] = vf[s];
      if (!big)
        for (int t = tid; t < m; t += kThreads) vs[k + t] = xo[idx[k + t]];
      __syncthreads();
      if (!big) {
        for (int c = tid; c < k; c += kThreads) {
          T acc = vs[c];
          for (int t = 0; t < m; ++t) acc = cfms(F[(size_t)(k + t) * ld + c], vs[k + t], acc);
          vs[c] = acc;
        }
        __syncthreads();
      }
      for (int kb = ((k - 1) / 32) * 32; kb >= 0; kb -= 32) {
        const int bs = min(32, k - kb);
        if (warp == 0) {
          for (int i = 0; i < bs; ++i)
            if (lane < bs) Ds[i][lane] = F[(size_t)(kb + i) * ld + kb + lane];
          __syncwarp();
          T qi = lane < bs ? vs[kb + lane] : czero<T>();
          for (int bb = bs - 1; bb > 0; --bb) {
            const T qb = shfl(qi, bb);
            if (lane < bb) qi = cfms(Ds[bb][lane], qb, qi);
          }
          if (lane < bs) vs[kb + lane] = qi;
          __syncwarp();
        }
        __syncthreads();
        for (int c = tid; c < kb; c += kThreads) col_update(F, ld, kb, bs, c, vs);
        __syncthreads();
      }
      for (int s = tid; s < k; s += kThreads) xo[idx[Pm[s]]] = vs[s];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Rectangular part of large fronts; task = (front, first row or column).
//   SWEEP 0: rows t of L21:   u[t]  = v[k+t] - L21[t,:] y        (y = vf[0..k))
//   SWEEP 1: rows a of U12:   z[a]  = y[a]   - U12[a,:] x_m      (x_m gathered from out)
//   SWEEP 2: cols t of U12:   u[t]  = v[k+t] - U12[:,t]^T w      (w = vf[0..k))
//   SWEEP 3: cols a of L21:   q[a]  = w[a]   - L21[:,a]^T x_m
// ---------------------------------------------------------------------------
template <typename T, int SWEEP>
__global__ void __launch_bounds__(kThreads)
rect_kernel(SolveLaunch a, const int2* __restrict__ tasks, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red[kWarps][32];
  T* vs = reinterpret_cast<T*>(smem_raw);
  const int w = blockIdx.y + a.w0;
  const int2 task = tasks[blockIdx.x];
  const FrontDesc d = a.P.fronts[task.x];
  const int k = d.k, m = d.m, n = d.n, ld = d.ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* F = reinterpret_cast<const T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const int* idx = a.P.idx + d.idx_off;
  const int s0 = task.y;
  for (int r = a.r0; r < a.r0 + a.nr; ++r) {
    const size_t sys = (size_t)w * a.nrhs + r;
    T* vf = reinterpret_cast<T*>(a.vb) + sys * a.vec_stride + d.v_off;
    const T* xo = out + sys * a.n;
    // the vector the block multiplies: y / w (forward) or x_m (backward)
    if (SWEEP == 0 || SWEEP == 2) {
      for (int s = tid; s < k; s += kThreads) vs[s] = vf[s];
    } else {
      for (int t = tid; t < m; t += kThreads) vs[t] = xo[idx[k + t]];
    }
    __syncthreads();
    if (SWEEP == 0 || SWEEP == 1) {
      const int rows = SWEEP == 0 ? m : k;
      for (int rr = warp; rr < kRect; rr += kWarps) {
        const int row = s0 + rr;
        if (row >= rows) break;
        const T* Frow = SWEEP == 0 ? F + (size_t)(k + row) * ld : F + (size_t)row * ld + k;
        const T acc = warp_dot(Frow, vs, 0, SWEEP == 0 ? k : m, lane);
        if (lane == 0) {
          const int slot = SWEEP == 0 ? k + row : row;
          vf[slot] = csub(vf[slot], acc);
        }
      }
    } else {
      // column block: lane = column, warps split the rows, fixed-order reduction
      const int cols = SWEEP == 2 ? m : k;
      const int rows = SWEEP == 2 ? k : m;
      const int c = s0 + lane;
      T a0 = czero<T>(), a1 = czero<T>();
      if (c < cols) {
        constexpr int UN = 8;
        const T* base = SWEEP == 2 ? F + k + c : F + (size_t)k * ld + c;
        int i = warp;
        for (; i + (UN - 1) * kWarps < rows; i += UN * kWarps) {
          T fr[UN];
#pragma unroll
          for (int u = 0; u < UN; ++u) fr[u] = base[(size_t)(i + u * kWarps) * ld];
#pragma unroll
          for (int u = 0; u < UN; u += 2) {
            a0 = cfma(fr[u], vs[i + u * kWarps], a0);
            a1 = cfma(fr[u + 1], vs[i + (u + 1) * kWarps], a1);
          }
        }
        for (; i < rows; i += kWarps) a0 = cfma(base[(size_t)i * ld], vs[i], a0);
      }
      red[warp][lane] = cadd(a0, a1);
      __syncthreads();
      if (warp == 0 && c < cols) {
        T s = red[0][lane];
        for (int q = 1; q < kWarps; ++q) s = cadd(s, red[q][lane]);
        const int slot = SWEEP == 2 ? k + c : c;
        vf[slot] = csub(vf[slot], s);
      }
    }
    (void)n;
    __syncthreads();
  }
}

}  // namespace

template <typename T>
void launch_sweep_tri(const SolveLaunch& a, int sweep, const int* flist, int nf, int nmax, const void* in,
                      void* out, cudaStream_t s) {
  if (nf <= 0) return;
  const size_t smem = (size_t)nmax * sizeof(T);
  const T* i = reinterpret_cast<const T*>(in);
  T* o = reinterpret_cast<T*>(out);
  dim3 grid(nf, a.n_omega);
  switch (sweep) {
    case 0: tri_kernel<T, 0><<<grid, kThreads, smem, s>>>(a, flist, i, o); break;
    case 1: tri_kernel<T, 1><<<grid, kThreads, smem, s>>>(a, flist, i, o); break;
    case 2: tri_kernel<T, 2><<<grid, kThreads, smem, s>>>(a, flist, i, o); break;
    default: tri_kernel<T, 3><<<grid, kThreads, smem, s>>>(a, flist, i, o); break;
  }
}

template <typename T>
void launch_sweep_rect(const SolveLaunch& a, int sweep, const int2* tasks, int ntasks, int vmax, void* out,
                       cudaStream_t s) {
  if (ntasks <= 0) return;
  const size_t smem = (size_t)vmax * sizeof(T);
  T* o = reinterpret_cast<T*>(out);
  dim3 grid(ntasks, a.n_omega);
  switch (sweep) {
    case 0: rect_kernel<T, 0><<<grid, kThreads, smem, s>>>(a, tasks, o); break;
    case 1: rect_kernel<T, 1><<<grid, kThreads, smem, s>>>(a, tasks, o); break;
    case 2: rect_kernel<T, 2><<<grid, kThreads, smem, s>>>(a, tasks, o); break;
    default: rect_kernel<T, 3><<<grid, kThreads, smem, s>>>(a, tasks, o); break;
  }
}

int sweep_rect_block() { return kRect; }

cudaError_t solve_init_attributes() {
  const int lim = 160 * 1024;
  cudaError_t e = cudaSuccess;
#define FDFD_ATTR(K, T, S)                                                                       \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  FDFD_ATTR(tri_kernel, float2, 0) FDFD_ATTR(tri_kernel, float2, 1) FDFD_ATTR(tri_kernel, float2, 2)
  FDFD_ATTR(tri_kernel, float2, 3) FDFD_ATTR(tri_kernel, double2, 0) FDFD_ATTR(tri_kernel, double2, 1)
  FDFD_ATTR(tri_kernel, double2, 2) FDFD_ATTR(tri_kernel, double2, 3)
  FDFD_ATTR(rect_kernel, float2, 0) FDFD_ATTR(rect_kernel, float2, 1) FDFD_ATTR(rect_kernel, float2, 2)
  FDFD_ATTR(rect_kernel, float2, 3) FDFD_ATTR(rect_kernel, double2, 0) FDFD_ATTR(rect_kernel, double2, 1)
  FDFD_ATTR(rect_kernel, double2, 2) FDFD_ATTR(rect_kernel, double2, 3)
#undef FDFD_ATTR
  return e;
}

template void launch_sweep_tri<float2>(const SolveLaunch&, int, const int*, int, int, const void*, void*,
                                       cudaStream_t);
template void launch_sweep_tri<double2>(const SolveLaunch&, int, const int*, int, int, const void*, void*,
                                        cudaStream_t);
template void launch_sweep_rect<float2>(const SolveLaunch&, int, const int2*, int, int, void*, cudaStream_t);
template void launch_sweep_rect<double2>(const SolveLaunch&, int, const int2*, int, int, void*, cudaStream_t);

}  // namespace fdfd
