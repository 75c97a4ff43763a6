// Triangular sweeps over the cached factors (paper Eq. 5 and Eq. 6; Sec. II,
// "back substitution").  Forward solve A x = b is L then U; the adjoint
// (transpose) solve A^T x = b reuses the same factors as U^T then L^T, so no
// second factorisation is needed (the first caching idea of Sec. II).
//
// Per front, with the factored front [L11\U11 U12; L21 S], its row permutation
// P and the triangular inverses X_L = L11^-1, X_U = U11^-1 stored at
// factorisation time:
//   L   : y = X_L (P v)_k,                 u = v_m - L21 y
//   U   : x_k = X_U (y - U12 x_m)
//   U^T : w = X_U^T v_k,                   u = v_m - U12^T w
//   L^T : x_k = P^T X_L^T (w - L21^T x_m)
// where v gathers the front's entries of the right-hand side plus the update
// vectors u of its children (through the same inverse extend-add maps as the
// factorisation) and x_m are the already final values of the boundary
// variables.  Levels run bottom-up for L / U^T and top-down for U / L^T.
//
// With the inverses every step is a matrix-vector product.  A small front
// (n <= 64) is one task done by one warp; a large front is cut into tasks of
// 8 rows (one per warp) or 32 columns (one per lane) of its k x k inverse block
// (phase 1 bottom-up) and of its off-diagonal block (the other phase).  One
// persistent launch per direction runs every task in elimination-tree order
// (the dataflow sweep below), so the whole GPU streams the factor with no
// sequential substitution chain and no launch per level.  Every factor read
// is coalesced along a row or served from L1 by a lane's own row, each factor
// entry is read once per right-hand side, and reductions run in a fixed order
// (deterministic).
#include "kernels.h"

namespace fdfd {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRowBlk = kWarps;     // rows per row-type task (one per warp)
constexpr int kColBlk = 32;         // columns per column-type task (one per lane)

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Vector entries written by other CTAs of the same launch (the dataflow sweep)
// are read through L2 only: the per-SM L1 is not coherent.
__device__ __forceinline__ float2 ldv(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldv(const double2* p) { return __ldcg(p); }

// sum_{c in [c0, c1)} row[c] * vec[c], lanes striding the row (coalesced), warp-reduced.
// Eight loads per lane are issued before they are used.
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

// Column block product: lane = column, warps split the rows [r0, r1) of a
// row-major block with stride ld; column c = c0 + lane uses only rows r with
// lo(c) <= r < hi(c) (triangle masks).  Returns the per-lane column sum,
// reduced over warps in a fixed order (valid in warp 0).
template <typename T, typename Mask>
__device__ __forceinline__ T col_dot(const T* __restrict__ base, int ld, const T* vec, int r0, int r1,
                                     bool live, Mask inside, T (*red)[32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int UN = 4;
  T a0 = czero<T>(), a1 = czero<T>();
  if (live) {
    int r = r0 + warp;
    for (; r + (UN - 1) * kWarps < r1; r += UN * kWarps) {
      T f[UN];
#pragma unroll
      for (int u = 0; u < UN; ++u) f[u] = base[(size_t)(r + u * kWarps) * ld];
#pragma unroll
      for (int u = 0; u < UN; ++u)
        if (inside(r + u * kWarps)) {
          if (u & 1) a1 = cfma(f[u], vec[r + u * kWarps], a1);
          else a0 = cfma(f[u], vec[r + u * kWarps], a0);
        }
    }
    for (; r < r1; r += kWarps)
      if (inside(r)) a0 = cfma(base[(size_t)r * ld], vec[r], a0);
  }
  red[warp][lane] = cadd(a0, a1);
  __syncthreads();
  T s = red[0][lane];
  if (warp == 0)
    for (int q = 1; q < kWarps; ++q) s = cadd(s, red[q][lane]);
  return s;
}

// The two (at most) children of a front as the gathers need them: where their
// extend-add maps start and where their update vectors sit in a system's
// front-vector buffer.  Loaded once per task instead of once per slot.
struct Kids {
  int n;
  int inv_off[2];
  long long ubase[2];     // child's v_off + k
};

__device__ __forceinline__ Kids load_kids(const SolveLaunch& a, const FrontDesc& d) {
  Kids c;
  c.n = d.nchild;
#pragma unroll
  for (int ci = 0; ci < 2; ++ci) {
    c.inv_off[ci] = 0;
    c.ubase[ci] = 0;
    if (ci < d.nchild) {
      const FrontDesc& cd = a.P.fronts[a.P.children[d.child0 + ci]];
      c.inv_off[ci] = cd.inv_off;
      c.ubase[ci] = cd.v_off + cd.k;
    }
  }
  return c;
}

// Right-hand side entry of local slot src (pivot slots only, when rhs is given)
// plus the children's update vectors at that slot.
template <typename T>
__device__ __forceinline__ T gather_slot(const SolveLaunch& a, const FrontDesc& d, const Kids& kids, const T* rhs,
                                         const T* vbs, int src) {
  const int t0 = kids.n > 0 ? a.P.inv[kids.inv_off[0] + src] : -1;
  const int t1 = kids.n > 1 ? a.P.inv[kids.inv_off[1] + src] : -1;
  T v = (rhs && src < d.k) ? rhs[a.P.idx[d.idx_off + src]] : czero<T>();
  if (t0 >= 0) v = cadd(v, ldv(vbs + kids.ubase[0] + t0));
  if (t1 >= 0) v = cadd(v, ldv(vbs + kids.ubase[1] + t1));
  return v;
}

// ---------------------------------------------------------------------------
// Inverse-block products; task = (front, first row or column of the k range).
//   SWEEP 0: rows r:    y[r]  = (P v)_r + sum_{b<r} X_L[r][b] (P v)_b
//   SWEEP 1: rows a:    x[a]  = sum_{b>=a} X_U[a][b] z[b]          (z = vf[0..k))
//   SWEEP 2: cols a:    w[a]  = sum_{b<=a} X_U[b][a] v_b
//   SWEEP 3: cols a:    q[a]  = t[a] + sum_{b>a} X_L[b][a] t[b]    (t = vf[0..k)), x[P a] = q[a]
// ---------------------------------------------------------------------------
// A whole small front done by one warp (the dataflow sweep runs up to eight of
// them per CTA): lane = row (L, U) or column (U^T, L^T) of each product, each
// lane's dot product with eight loads in flight; vs is the warp's own slice
// of n + k entries.
template <typename T>
__device__ __forceinline__ T lane_dot(const T* __restrict__ row, const T* vec, int c0, int c1) {
  T acc[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
  int c = c0;
  for (; c + 7 < c1; c += 8) {
    T f[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) f[u] = row[c + u];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u & 3] = cfma(f[u], vec[c + u], acc[u & 3]);
  }
  for (; c < c1; ++c) acc[0] = cfma(row[c], vec[c], acc[0]);
  return cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
}
template <typename T>
__device__ __forceinline__ T lane_col_dot(const T* __restrict__ col, int ld, const T* vec, int r0, int r1) {
  T acc[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
  int r = r0;
  for (; r + 7 < r1; r += 8) {
    T f[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) f[u] = col[(size_t)(r + u) * ld];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u & 3] = cfma(f[u], vec[r + u], acc[u & 3]);
  }
  for (; r < r1; ++r) acc[0] = cfma(col[(size_t)r * ld], vec[r], acc[0]);
  return cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
}

template <typename T, int SWEEP>
__device__ __forceinline__ void whole_front_warp(const SolveLaunch& a, const FrontDesc& d, int w,
                                                 const T* __restrict__ in, T* __restrict__ out, T* vs) {
  const int k = d.k, m = d.m, n = d.n, ldk = d.ldk, ld = d.ld;
  const int lane = threadIdx.x & 31;
  const T* X = reinterpret_cast<const T*>(a.istore) + (size_t)w * a.istore_stride + d.iv_off;
  const T* F = reinterpret_cast<const T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const int* Pm = a.perm + (size_t)w * a.perm_stride + d.piv_off;
  const int* idx = a.P.idx + d.idx_off;
  const Kids kids = load_kids(a, d);
  T* ws = vs + n;
  for (int r = a.r0; r < a.r0 + a.nr; ++r) {
    const size_t sys = (size_t)w * a.nrhs + r;
    T* vbs = reinterpret_cast<T*>(a.vb) + sys * a.vec_stride;
    T* vf = vbs + d.v_off;
    T* xo = out + sys * a.n;
    if (SWEEP == 0 || SWEEP == 2) {
      const T* rhs = in + sys * a.n;
      for (int s = lane; s < n; s += 32) vs[s] = gather_slot(a, d, kids, rhs, vbs, (SWEEP == 0 && s < k) ? Pm[s] : s);
    } else {
      for (int s = lane; s < k; s += 32) vs[s] = ldv(vf + s);
      for (int t = lane; t < m; t += 32) {
        const T x = ldv(xo + idx[k + t]);
        vs[k + t] = SWEEP == 3 ? csub(czero<T>(), x) : x;
      }
    }
    __syncwarp();
    if (SWEEP == 0) {                              // y = X_L (P v)_k;  u = v_m - L21 y
      for (int row = lane; row < k; row += 32) ws[row] = cadd(vs[row], lane_dot(X + (size_t)row * ldk, vs, 0, row));
      __syncwarp();
      for (int t = lane; t < m; t += 32) vf[k + t] = csub(vs[k + t], lane_dot(F + (size_t)(k + t) * ld, ws, 0, k));
      for (int s = lane; s < k; s += 32) vf[s] = ws[s];
    } else if (SWEEP == 1) {                       // z = y - U12 x_m;  x_k = X_U z
      for (int row = lane; row < k; row += 32) ws[row] = csub(vs[row], lane_dot(F + (size_t)row * ld + k, vs + k, 0, m));
      __syncwarp();
      for (int row = lane; row < k; row += 32) xo[idx[row]] = lane_dot(X + (size_t)row * ldk, ws, row, k);
    } else if (SWEEP == 2) {                       // w = X_U^T v_k;  u = v_m - U12^T w
      for (int c = lane; c < k; c += 32) ws[c] = lane_col_dot(X + c, ldk, vs, 0, c + 1);
      __syncwarp();
      for (int t = lane; t < m; t += 32) vf[k + t] = csub(vs[k + t], lane_col_dot(F + k + t, ld, ws, 0, k));
      for (int s = lane; s < k; s += 32) vf[s] = ws[s];
    } else {                                       // t = w - L21^T x_m;  x_k = P^T X_L^T t   (vs[k..n) = -x_m)
      for (int c = lane; c < k; c += 32) ws[c] = cadd(vs[c], lane_col_dot(F + (size_t)k * ld + c, ld, vs + k, 0, m));
      __syncwarp();
      for (int c = lane; c < k; c += 32) xo[idx[Pm[c]]] = cadd(ws[c], lane_col_dot(X + c, ldk, ws, c + 1, k));
    }
    __syncwarp();
  }
}

// One inverse-block task of a large front (rows or columns from b0).
template <typename T, int SWEEP>
__device__ __forceinline__ void tri_task(const SolveLaunch& a, const FrontDesc& d, int b0, int w,
                                         const T* __restrict__ in, T* __restrict__ out, T* vs, T (*red)[32]) {
  const int k = d.k, ldk = d.ldk;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* X = reinterpret_cast<const T*>(a.istore) + (size_t)w * a.istore_stride + d.iv_off;
  const int* Pm = a.perm + (size_t)w * a.perm_stride + d.piv_off;
  const int* idx = a.P.idx + d.idx_off;
  const Kids kids = load_kids(a, d);
  for (int r = a.r0; r < a.r0 + a.nr; ++r) {
    const size_t sys = (size_t)w * a.nrhs + r;
    T* vbs = reinterpret_cast<T*>(a.vb) + sys * a.vec_stride;
    T* vf = vbs + d.v_off;
    if (SWEEP == 0 || SWEEP == 2) {
      const T* rhs = in + sys * a.n;
      for (int s = tid; s < k; s += 2 * kThreads) {
        const int s2 = s + kThreads;
        const T g1 = gather_slot(a, d, kids, rhs, vbs, SWEEP == 0 ? Pm[s] : s);
        const T g2 = s2 < k ? gather_slot(a, d, kids, rhs, vbs, SWEEP == 0 ? Pm[s2] : s2) : czero<T>();
        vs[s] = g1;
        if (s2 < k) vs[s2] = g2;
      }
    } else {
      for (int s = tid; s < k; s += kThreads) vs[s] = ldv(vf + s);
    }
    __syncthreads();
    if (SWEEP == 0) {
      for (int rr = warp; rr < kRowBlk; rr += kWarps) {
        const int row = b0 + rr;
        if (row >= k) break;
        const T acc = warp_dot(X + (size_t)row * ldk, vs, 0, row, lane);
        if (lane == 0) vf[row] = cadd(vs[row], acc);
      }
    } else if (SWEEP == 1) {
      T* xo = out + sys * a.n;
      for (int rr = warp; rr < kRowBlk; rr += kWarps) {
        const int row = b0 + rr;
        if (row >= k) break;
        const T acc = warp_dot(X + (size_t)row * ldk, vs, row, k, lane);
        if (lane == 0) xo[idx[row]] = acc;
      }
    } else if (SWEEP == 2) {
      const int c = b0 + lane;
      const T s = col_dot(X + c, ldk, vs, 0, min(b0 + kColBlk, k), c < k, [&](int b) { return b <= c; }, red);
      if (warp == 0 && c < k) vf[c] = s;
    } else {
      const int c = b0 + lane;
      T* xo = out + sys * a.n;
      const T s = col_dot(X + c, ldk, vs, b0 + 1, k, c < k, [&](int b) { return b > c; }, red);
      if (warp == 0 && c < k) xo[idx[Pm[c]]] = cadd(vs[c], s);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Off-diagonal blocks; task = (front, first row or column).
//   SWEEP 0: rows t of L21:   u[t] = g_t - L21[t,:] y          (g_t gathered, y = vf[0..k))
//   SWEEP 1: rows a of U12:   z[a] = y[a] - U12[a,:] x_m       (x_m gathered from out)
//   SWEEP 2: cols t of U12:   u[t] = g_t - U12[:,t]^T w        (w = vf[0..k))
//   SWEEP 3: cols a of L21:   t[a] = w[a] - L21[:,a]^T x_m
// ---------------------------------------------------------------------------
// One off-diagonal task of a large front (rows or columns from s0).
template <typename T, int SWEEP>
__device__ __forceinline__ void rect_task(const SolveLaunch& a, const FrontDesc& d, int s0, int w,
                                          T* __restrict__ out, T* vs, T (*red)[32]) {
  const int k = d.k, m = d.m, ld = d.ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* F = reinterpret_cast<const T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const int* idx = a.P.idx + d.idx_off;
  const Kids kids = load_kids(a, d);
  for (int r = a.r0; r < a.r0 + a.nr; ++r) {
    const size_t sys = (size_t)w * a.nrhs + r;
    T* vbs = reinterpret_cast<T*>(a.vb) + sys * a.vec_stride;
    T* vf = vbs + d.v_off;
    const T* xo = out + sys * a.n;
    if (SWEEP == 0 || SWEEP == 2) {
      for (int s = tid; s < k; s += kThreads) vs[s] = ldv(vf + s);
    } else {
      for (int t = tid; t < m; t += kThreads) vs[t] = ldv(xo + idx[k + t]);
    }
    __syncthreads();
    if (SWEEP == 0 || SWEEP == 1) {
      for (int rr = warp; rr < kRowBlk; rr += kWarps) {
        const int row = s0 + rr;
        if (row >= (SWEEP == 0 ? m : k)) break;
        const T* Frow = SWEEP == 0 ? F + (size_t)(k + row) * ld : F + (size_t)row * ld + k;
        // the value the product is subtracted from, fetched before the product
        const T g = SWEEP == 0 ? gather_slot(a, d, kids, (const T*)nullptr, vbs, k + row) : ldv(vf + row);
        const T acc = warp_dot(Frow, vs, 0, SWEEP == 0 ? k : m, lane);
        if (lane == 0) vf[SWEEP == 0 ? k + row : row] = csub(g, acc);
      }
    } else {
      const int cols = SWEEP == 2 ? m : k;
      const int rows = SWEEP == 2 ? k : m;
      const int c = s0 + lane;
      const T* base = SWEEP == 2 ? F + k + c : F + (size_t)k * ld + c;
      // the value the product is subtracted from, fetched before the product
      T g = czero<T>();
      if (warp == 0 && c < cols) g = SWEEP == 2 ? gather_slot(a, d, kids, (const T*)nullptr, vbs, k + c) : ldv(vf + c);
      const T s = col_dot(base, ld, vs, 0, rows, c < cols, [](int) { return true; }, red);
      if (warp == 0 && c < cols) vf[SWEEP == 2 ? k + c : c] = csub(g, s);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Dataflow sweep: one persistent launch runs every task of one direction.
// CTAs take tasks from a queue in dependency order (bottom-up levels for
// L / U^T, top-down for U / L^T; inside a level, the phase-1 tasks of a large
// front before its phase-2 tasks); a task first waits for the per-front
// completion counters it depends on, then runs, then bumps its front's
// counters.  A task only ever waits for tasks earlier in the queue, which are
// held by running CTAs, so the queue drains whatever the residency.
//   bottom-up: whole / inverse-block tasks wait for the children; the
//              off-diagonal tasks of a front wait for its inverse-block tasks;
//   top-down:  whole / off-diagonal tasks wait for the parent; the
//              inverse-block tasks of a front wait for its off-diagonal tasks
//              (and for the parent).
// Every wait gives up after kSpinLimit polls: it sets *err, and the CTA stops.
// ---------------------------------------------------------------------------
constexpr int kSpinLimit = 1 << 21;


__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool wait_ge(const int* p, int need, int* err) {
  for (int it = 0; it < kSpinLimit; ++it) {
    if (ld_acquire(p) >= need) return true;
    if (ld_acquire(err) != 0) return false;
    __nanosleep(64);
  }
  atomicExch(err, 1);
  return false;
}

constexpr int kWarpSlice = 128;   // vector entries per warp for a whole small front (n + k, n <= 64)

template <typename T, int SWEEP>
__global__ void __launch_bounds__(kThreads)
flow_kernel(SolveLaunch a, FlowQueue q, const T* __restrict__ in, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red[kWarps][32];
  __shared__ int s_unit, s_ok, s_fail;
  T* vs = reinterpret_cast<T*>(smem_raw);
  constexpr bool kUp = SWEEP == 0 || SWEEP == 2;
  const int nf = q.n_fronts;
  int* head = q.ctr;
  int* done = q.ctr + 1;                       // [n_omega launched][nf]
  int* ph1 = done + (size_t)a.n_omega * nf;    // [n_omega launched][nf]
  const int total = q.nunits * a.n_omega;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_fail = 0;
  for (;;) {
    if (tid == 0) s_unit = atomicAdd(head, 1);
    __syncthreads();
    const int u = s_unit;
    if (u >= total) break;
    const int ui = u / a.n_omega, wl = u - ui * a.n_omega;
    const int w = wl + a.w0;
    const int2 unit = q.units[ui];
    const int* dn = done + (size_t)wl * nf;
    if ((unsigned)unit.y & 0x80000000u) {
      // a batch of whole small fronts of one level: one per warp, each waits for its own dependencies
      const int cnt = unit.y & 0xff;
      if (warp < cnt) {
        const int2 task = q.tasks[unit.x + warp];
        const int f = (int)((unsigned)task.x & 0x3fffffffu);
        const FrontDesc d = a.P.fronts[f];
        bool ok = true;
        if (lane == 0) {
          if (kUp) {
            for (int ci = 0; ci < d.nchild && ok; ++ci) {
              const int c = a.P.children[d.child0 + ci];
              ok = wait_ge(dn + c, q.need_all[c], q.err);
            }
          } else if (d.parent >= 0) {
            ok = wait_ge(dn + d.parent, q.need_all[d.parent], q.err);
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok) {
          whole_front_warp<T, SWEEP>(a, d, w, in, out, vs + warp * kWarpSlice);
          if (lane == 0) {
            __threadfence();
            atomicAdd(done + (size_t)wl * nf + f, 1);
          }
        } else if (lane == 0) {
          s_fail = 1;
        }
      }
      __syncthreads();
      if (s_fail) break;
      continue;
    }
    // one task of a large front for the whole CTA
    const int2 task = q.tasks[unit.x];
    const unsigned code = (unsigned)task.x;
    const bool rect = ((code >> 30) & 1u) != 0;
    const int f = (int)(code & 0x3fffffffu);
    const FrontDesc d = a.P.fronts[f];
    if (tid == 0) {
      bool ok = true;
      if (kUp) {
        if (rect) {
          ok = wait_ge(ph1 + (size_t)wl * nf + f, q.need_ph1[f], q.err);
        } else {
          for (int ci = 0; ci < d.nchild && ok; ++ci) {
            const int c = a.P.children[d.child0 + ci];
            ok = wait_ge(dn + c, q.need_all[c], q.err);
          }
        }
      } else {
        if (d.parent >= 0) ok = wait_ge(dn + d.parent, q.need_all[d.parent], q.err);
        if (ok && !rect) ok = wait_ge(ph1 + (size_t)wl * nf + f, q.need_ph1[f], q.err);
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    if (rect) rect_task<T, SWEEP>(a, d, task.y, w, out, vs, red);
    else tri_task<T, SWEEP>(a, d, task.y, w, in, out, vs, red);
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      // phase 1: inverse-block tasks bottom-up, off-diagonal tasks top-down
      if (kUp ? !rect : rect) atomicAdd(ph1 + (size_t)wl * nf + f, 1);
      atomicAdd(done + (size_t)wl * nf + f, 1);
    }
  }
}

}  // namespace

// One wait on *flag >= 1 (nothing sets it) by one thread: exercises the
// bounded wait of the dataflow sweep, which must give up, set *err and return.
__global__ void wait_probe_kernel(const int* flag, int* err) {
  if (threadIdx.x == 0) (void)wait_ge(flag, 1, err);
}

cudaError_t launch_wait_probe(const int* flag, int* err, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(flag, err);
  return cudaGetLastError();
}

size_t flow_smem(int vmax, size_t es) {
  const int e = vmax > kWarps * kWarpSlice ? vmax : kWarps * kWarpSlice;
  return (size_t)e * es;
}

template <typename T>
void launch_sweep_flow(const SolveLaunch& a, int sweep, const FlowQueue& q, int vmax, int grid, const void* in,
                       void* out, cudaStream_t s) {
  if (q.nunits <= 0) return;
  const size_t smem = flow_smem(vmax, sizeof(T));
  const T* i = reinterpret_cast<const T*>(in);
  T* o = reinterpret_cast<T*>(out);
  switch (sweep) {
    case 0: flow_kernel<T, 0><<<grid, kThreads, smem, s>>>(a, q, i, o); break;
    case 1: flow_kernel<T, 1><<<grid, kThreads, smem, s>>>(a, q, i, o); break;
    case 2: flow_kernel<T, 2><<<grid, kThreads, smem, s>>>(a, q, i, o); break;
    default: flow_kernel<T, 3><<<grid, kThreads, smem, s>>>(a, q, i, o); break;
  }
}

int flow_blocks_per_sm(int elem_bytes, int vmax) {
  int nb = 0;
  const size_t smem = flow_smem(vmax, elem_bytes);
  const cudaError_t e = elem_bytes == 8
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, flow_kernel<float2, 1>, kThreads, smem)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, flow_kernel<double2, 1>, kThreads, smem);
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

int sweep_row_block() { return kRowBlk; }

int flow_whole_max_n() { return kWarpSlice / 2; }
int sweep_col_block() { return kColBlk; }

cudaError_t solve_init_attributes() {
  const int lim = 160 * 1024;
  cudaError_t e = cudaSuccess;
#define FDFD_ATTR(K, T, S)                                                                       \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  FDFD_ATTR(flow_kernel, float2, 0) FDFD_ATTR(flow_kernel, float2, 1) FDFD_ATTR(flow_kernel, float2, 2)
  FDFD_ATTR(flow_kernel, float2, 3) FDFD_ATTR(flow_kernel, double2, 0) FDFD_ATTR(flow_kernel, double2, 1)
  FDFD_ATTR(flow_kernel, double2, 2) FDFD_ATTR(flow_kernel, double2, 3)
#undef FDFD_ATTR
  return e;
}

template void launch_sweep_flow<float2>(const SolveLaunch&, int, const FlowQueue&, int, int, const void*, void*,
                                        cudaStream_t);
template void launch_sweep_flow<double2>(const SolveLaunch&, int, const FlowQueue&, int, int, const void*, void*,
                                         cudaStream_t);

}  // namespace fdfd
