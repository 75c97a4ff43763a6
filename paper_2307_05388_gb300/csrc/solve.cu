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
// where v gathers the front's entries of the right-hand side (complex128, cast
// to the factor precision as it is gathered) plus the update
// vectors u of its children (through the same inverse extend-add maps as the
// factorisation) and x_m are the already final values of the boundary
// variables (the solution is stored in complex128 as it is produced).  Levels
// run bottom-up for L / U^T and top-down for U / L^T.
//
// With the inverses every step is a matrix-vector product.  A small front
// (n <= 64) is one task done by one warp, a medium front (n <= 320) one task
// of a CTA; a large front is cut into tasks of 8 rows (one per warp) or 16
// columns (two lanes per column in each warp) of its k x k inverse block
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
constexpr int kRowBlk = kWarps;     // rows per row-type task (one per warp; tall tasks: two)
constexpr int kColBlk = 16;         // columns per column-type task (each column: two lanes per warp)

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

// Two rows over the same columns at once: sixteen loads per lane in flight.
template <typename T>
__device__ __forceinline__ void warp_dot2(const T* __restrict__ ra, const T* __restrict__ rb, const T* vec, int c0,
                                          int c1, int lane, T& sa, T& sb) {
  constexpr int UN = 8;
  T a0[2] = {czero<T>(), czero<T>()}, b0[2] = {czero<T>(), czero<T>()};
  int c = c0 + lane;
  for (; c + 32 * (UN - 1) < c1; c += 32 * UN) {
    T x[UN], y[UN];
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      x[u] = ra[c + 32 * u];
      y[u] = rb[c + 32 * u];
    }
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      const T v = vec[c + 32 * u];
      a0[u & 1] = cfma(x[u], v, a0[u & 1]);
      b0[u & 1] = cfma(y[u], v, b0[u & 1]);
    }
  }
  for (; c < c1; c += 32) {
    const T v = vec[c];
    a0[0] = cfma(ra[c], v, a0[0]);
    b0[0] = cfma(rb[c], v, b0[0]);
  }
  sa = warp_sum(cadd(a0[0], a0[1]));
  sb = warp_sum(cadd(b0[0], b0[1]));
}

// Column block product over kColBlk columns: lane = (column c = lane % kColBlk,
// row slice lane / kColBlk), the warps' slices split the rows [r0, r1) of a
// row-major block with stride ld (base points at the lane's column); column c
// uses only rows r with lo(c) <= r < hi(c) (triangle masks).  Returns the
// column sum, reduced over the slices and the warps in a fixed order (valid in
// warp 0, lanes < kColBlk).
template <typename T, typename Mask>
__device__ __forceinline__ T col_dot(const T* __restrict__ base, int ld, const T* vec, int r0, int r1,
                                     bool live, Mask inside, T (*red)[32]) {
  constexpr int SL = 32 / kColBlk;              // row slices per warp
  constexpr int RS = kWarps * SL;               // row stride of one thread
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int UN = sizeof(T) == 8 ? 16 : 8;
  T a0 = czero<T>(), a1 = czero<T>();
  if (live) {
    int r = r0 + warp * SL + lane / kColBlk;
    for (; r + (UN - 1) * RS < r1; r += UN * RS) {
      T f[UN];
#pragma unroll
      for (int u = 0; u < UN; ++u) f[u] = base[(size_t)(r + u * RS) * ld];
#pragma unroll
      for (int u = 0; u < UN; ++u)
        if (inside(r + u * RS)) {
          if (u & 1) a1 = cfma(f[u], vec[r + u * RS], a1);
          else a0 = cfma(f[u], vec[r + u * RS], a0);
        }
    }
    for (; r < r1; r += RS)
      if (inside(r)) a0 = cfma(base[(size_t)r * ld], vec[r], a0);
  }
  T s = cadd(a0, a1);
#pragma unroll
  for (int o = kColBlk; o < 32; o <<= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
  }
  red[warp][lane] = s;
  __syncthreads();
  s = red[0][lane];
  if (warp == 0)
    for (int q = 1; q < kWarps; ++q) s = cadd(s, red[q][lane]);
  return s;
}

// Two right-hand sides at once: each factor entry is loaded once and multiplied into
// both systems' vectors (v0, v1).  Row form of warp_dot.
template <typename T>
__device__ __forceinline__ void warp_dot_pair(const T* __restrict__ row, const T* v0, const T* v1, int c0, int c1,
                                              int lane, T& s0, T& s1) {
  constexpr int UN = 8;
  T a0 = czero<T>(), a1 = czero<T>();
  int c = c0 + lane;
  for (; c + 32 * (UN - 1) < c1; c += 32 * UN) {
    T r[UN];
#pragma unroll
    for (int u = 0; u < UN; ++u) r[u] = row[c + 32 * u];
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      a0 = cfma(r[u], v0[c + 32 * u], a0);
      a1 = cfma(r[u], v1[c + 32 * u], a1);
    }
  }
  for (; c < c1; c += 32) {
    const T rv = row[c];
    a0 = cfma(rv, v0[c], a0);
    a1 = cfma(rv, v1[c], a1);
  }
  s0 = warp_sum(a0);
  s1 = warp_sum(a1);
}

// Column form (col_dot) for two right-hand sides; red0 / red1 are separate reduction tiles.
template <typename T, typename Mask>
__device__ __forceinline__ void col_dot_pair(const T* __restrict__ base, int ld, const T* v0, const T* v1, int r0,
                                             int r1, bool live, Mask inside, T (*red0)[32], T (*red1)[32], T& s0,
                                             T& s1) {
  constexpr int SL = 32 / kColBlk;
  constexpr int RS = kWarps * SL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int UN = sizeof(T) == 8 ? 8 : 4;
  T a0 = czero<T>(), a1 = czero<T>();
  if (live) {
    int r = r0 + warp * SL + lane / kColBlk;
    for (; r + (UN - 1) * RS < r1; r += UN * RS) {
      T f[UN];
#pragma unroll
      for (int u = 0; u < UN; ++u) f[u] = base[(size_t)(r + u * RS) * ld];
#pragma unroll
      for (int u = 0; u < UN; ++u)
        if (inside(r + u * RS)) {
          a0 = cfma(f[u], v0[r + u * RS], a0);
          a1 = cfma(f[u], v1[r + u * RS], a1);
        }
    }
    for (; r < r1; r += RS)
      if (inside(r)) {
        const T fv = base[(size_t)r * ld];
        a0 = cfma(fv, v0[r], a0);
        a1 = cfma(fv, v1[r], a1);
      }
  }
#pragma unroll
  for (int o = kColBlk; o < 32; o <<= 1) {
    a0.x += __shfl_xor_sync(0xffffffffu, a0.x, o);
    a0.y += __shfl_xor_sync(0xffffffffu, a0.y, o);
    a1.x += __shfl_xor_sync(0xffffffffu, a1.x, o);
    a1.y += __shfl_xor_sync(0xffffffffu, a1.y, o);
  }
  red0[warp][lane] = a0;
  red1[warp][lane] = a1;
  __syncthreads();
  s0 = red0[0][lane];
  s1 = red1[0][lane];
  if (warp == 0)
    for (int q = 1; q < kWarps; ++q) {
      s0 = cadd(s0, red0[q][lane]);
      s1 = cadd(s1, red1[q][lane]);
    }
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

// D[cell] of the symmetric form (stretch factors at the cell centre)
__device__ __forceinline__ double2 sym_d(const SolveLaunch& a, int w, int cell) {
  const int i = cell / a.P.ny, j = cell - i * a.P.ny;
  return cmul(a.sxc[(size_t)w * a.P.nx + i], a.syc[(size_t)w * a.P.ny + j]);
}

// The solution value written for cell: x, or D x for the transposed symmetric-form solve.
template <typename T>
__device__ __forceinline__ double2 out_val(const SolveLaunch& a, int w, int cell, T v) {
  const double2 x = cto64(v);
  return a.sym_out ? cmul(sym_d(a, w, cell), x) : x;
}

// x_m of a front below, read back from the output: D x was written there for the
// transposed symmetric-form solve
__device__ __forceinline__ double2 xm_val(const SolveLaunch& a, int w, int cell, double2 x) {
  if (!a.sym_out) return x;
  const double2 d = sym_d(a, w, cell);
  const double q = 1.0 / (d.x * d.x + d.y * d.y);
  return cmul(x, make_double2(d.x * q, -d.y * q));
}

// w = y / d for the symmetric form (1 / d on the diagonal of the inverse store)
template <typename T>
__device__ __forceinline__ T mid_val(const SolveLaunch& a, const T* X, int ldk, int s, T v) {
  return a.sym_mid ? cmul(v, X[(size_t)s * ldk + s]) : v;
}

// Right-hand side entry of local slot src (pivot slots only, when rhs is given;
// times D for the symmetric form) plus the children's update vectors at that slot.
template <typename T>
__device__ __forceinline__ T gather_slot(const SolveLaunch& a, const FrontDesc& d, const Kids& kids,
                                         const double2* rhs, const T* vbs, int src, int w = 0) {
  const int t0 = kids.n > 0 ? a.P.inv[kids.inv_off[0] + src] : -1;
  const int t1 = kids.n > 1 ? a.P.inv[kids.inv_off[1] + src] : -1;
  T v = czero<T>();
  if (rhs && src < d.k) {
    const int cell = a.P.idx[d.idx_off + src];
    const double2 b = rhs[cell];
    v = cfrom<T>(a.sym_in ? cmul(sym_d(a, w, cell), b) : b);
  }
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
// them per CTA), every product spread over all 32 lanes: a row product gives
// each row 32/R lanes (R rows at a time), a column product gives each column
// 32/C lanes that split its rows (C columns at a time), partial sums combined
// by a fixed butterfly; vs is the warp's own slice of n + k entries.
template <typename T, typename Lo, typename Hi, typename Out>
__device__ __forceinline__ void warp_rows_dot(const T* __restrict__ A, int ld, int nrows, const T* vec, Lo lo, Hi hi,
                                              Out out) {
  constexpr int UN = sizeof(T) == 8 ? 16 : 8;
  const int lane = threadIdx.x & 31;
  int R = 32;
  while (R > 1 && R / 2 >= nrows) R >>= 1;      // rows at a time
  const int G = 32 / R;                          // lanes per row
  const int gl = lane & (G - 1), ri = lane / G;
  for (int i0 = 0; i0 < nrows; i0 += R) {
    const int i = i0 + ri;
    T a0 = czero<T>(), a1 = czero<T>();
    if (i < nrows) {
      const T* row = A + (size_t)i * ld;
      const int e = hi(i);
      int c = lo(i) + gl;
      for (; c + (UN - 1) * G < e; c += UN * G) {
        T f[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) f[u] = row[c + u * G];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
          if (u & 1) a1 = cfma(f[u], vec[c + u * G], a1);
          else a0 = cfma(f[u], vec[c + u * G], a0);
        }
      }
      for (; c < e; c += G) a0 = cfma(row[c], vec[c], a0);
    }
    T acc = cadd(a0, a1);
    for (int o = 1; o < G; o <<= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (gl == 0 && i < nrows) out(i, acc);
  }
}
template <typename T, typename Lo, typename Hi, typename Out>
__device__ __forceinline__ void warp_cols_dot(const T* __restrict__ A, int ld, int ncols, const T* vec, Lo lo, Hi hi,
                                              Out out) {
  constexpr int UN = sizeof(T) == 8 ? 16 : 8;
  const int lane = threadIdx.x & 31;
  int C = 32;
  while (C > 1 && C / 2 >= ncols) C >>= 1;      // columns at a time
  const int S = 32 / C;                          // row slices per column
  const int cl = lane & (C - 1), si = lane / C;
  for (int j0 = 0; j0 < ncols; j0 += C) {
    const int j = j0 + cl;
    T a0 = czero<T>(), a1 = czero<T>();
    if (j < ncols) {
      const int e = hi(j);
      int r = lo(j) + si;
      for (; r + (UN - 1) * S < e; r += UN * S) {
        T f[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) f[u] = A[(size_t)(r + u * S) * ld + j];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
          if (u & 1) a1 = cfma(f[u], vec[r + u * S], a1);
          else a0 = cfma(f[u], vec[r + u * S], a0);
        }
      }
      for (; r < e; r += S) a0 = cfma(A[(size_t)r * ld + j], vec[r], a0);
    }
    T acc = cadd(a0, a1);
    for (int o = C; o < 32; o <<= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (si == 0 && j < ncols) out(j, acc);
  }
}

template <typename T, int SWEEP>
__device__ __forceinline__ void whole_front_warp(const SolveLaunch& a, const FrontDesc& d, int w,
                                                 const double2* __restrict__ in, double2* __restrict__ out, T* vs) {
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
    double2* xo = out + sys * a.n;
    if (SWEEP == 0 || SWEEP == 2) {
      const double2* rhs = in + sys * a.n;
      for (int s = lane; s < n; s += 32)
        vs[s] = gather_slot(a, d, kids, rhs, vbs, (SWEEP == 0 && s < k) ? Pm[s] : s, w);
    } else {
      for (int s = lane; s < k; s += 32) vs[s] = SWEEP == 3 ? mid_val(a, X, ldk, s, ldv(vf + s)) : ldv(vf + s);
      for (int t = lane; t < m; t += 32) {
        const T x = cfrom<T>(SWEEP == 3 ? xm_val(a, w, idx[k + t], ldv(xo + idx[k + t])) : ldv(xo + idx[k + t]));
        vs[k + t] = SWEEP == 3 ? csub(czero<T>(), x) : x;
      }
    }
    __syncwarp();
    if (SWEEP == 0) {                              // y = X_L (P v)_k;  u = v_m - L21 y
      warp_rows_dot(X, ldk, k, vs, [](int) { return 0; }, [](int i) { return i; },
                    [&](int i, T acc) { ws[i] = cadd(vs[i], acc); });
      __syncwarp();
      warp_rows_dot(F + (size_t)k * ld, ld, m, ws, [](int) { return 0; }, [&](int) { return k; },
                    [&](int t, T acc) { vf[k + t] = csub(vs[k + t], acc); });
      for (int s = lane; s < k; s += 32) vf[s] = ws[s];
    } else if (SWEEP == 1) {                       // z = y - U12 x_m;  x_k = X_U z
      warp_rows_dot(F + k, ld, k, vs + k, [](int) { return 0; }, [&](int) { return m; },
                    [&](int i, T acc) { ws[i] = csub(vs[i], acc); });
      __syncwarp();
      warp_rows_dot(X, ldk, k, ws, [](int i) { return i; }, [&](int) { return k; },
                    [&](int i, T acc) { xo[idx[i]] = cto64(acc); });
    } else if (SWEEP == 2) {                       // w = X_U^T v_k;  u = v_m - U12^T w
      warp_cols_dot(X, ldk, k, vs, [](int) { return 0; }, [](int j) { return j + 1; },
                    [&](int j, T acc) { ws[j] = acc; });
      __syncwarp();
      warp_cols_dot(F + k, ld, m, ws, [](int) { return 0; }, [&](int) { return k; },
                    [&](int t, T acc) { vf[k + t] = csub(vs[k + t], acc); });
      for (int s = lane; s < k; s += 32) vf[s] = ws[s];
    } else {                                       // t = w - L21^T x_m;  x_k = P^T X_L^T t   (vs[k..n) = -x_m)
      warp_cols_dot(F + (size_t)k * ld, ld, k, vs + k, [](int) { return 0; }, [&](int) { return m; },
                    [&](int j, T acc) { ws[j] = cadd(vs[j], acc); });
      __syncwarp();
      warp_cols_dot(X, ldk, k, ws, [](int j) { return j + 1; }, [&](int) { return k; },
                    [&](int j, T acc) { xo[idx[Pm[j]]] = out_val(a, w, idx[Pm[j]], cadd(ws[j], acc)); });
    }
    __syncwarp();
  }
}

// One inverse-block task of a large front (rows or columns from b0).
template <typename T, int SWEEP>
__device__ __forceinline__ void tri_task(const SolveLaunch& a, const FrontDesc& d, int b0, int nrows, int w,
                                         const double2* __restrict__ in, double2* __restrict__ out, T* vs,
                                         T (*red)[32]) {
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
      const double2* rhs = in + sys * a.n;
      for (int s = tid; s < k; s += 2 * kThreads) {
        const int s2 = s + kThreads;
        const T g1 = gather_slot(a, d, kids, rhs, vbs, SWEEP == 0 ? Pm[s] : s, w);
        const T g2 = s2 < k ? gather_slot(a, d, kids, rhs, vbs, SWEEP == 0 ? Pm[s2] : s2, w) : czero<T>();
        vs[s] = g1;
        if (s2 < k) vs[s2] = g2;
      }
    } else {
      // without an off-diagonal block (m = 0) the L^T sweep reads y here first
      for (int s = tid; s < k; s += kThreads)
        vs[s] = (SWEEP == 3 && d.m == 0) ? mid_val(a, X, ldk, s, ldv(vf + s)) : ldv(vf + s);
    }
    __syncthreads();
    if (SWEEP == 0) {
      for (int rr = warp; rr < nrows; rr += kWarps) {
        const int row = b0 + rr;
        if (row >= k) break;
        const T acc = warp_dot(X + (size_t)row * ldk, vs, 0, row, lane);
        if (lane == 0) vf[row] = cadd(vs[row], acc);
      }
    } else if (SWEEP == 1) {
      double2* xo = out + sys * a.n;
      for (int rr = warp; rr < nrows; rr += kWarps) {
        const int row = b0 + rr;
        if (row >= k) break;
        const T acc = warp_dot(X + (size_t)row * ldk, vs, row, k, lane);
        if (lane == 0) xo[idx[row]] = cto64(acc);
      }
    } else if (SWEEP == 2) {
      const int c = b0 + (lane & (kColBlk - 1));
      const T s = col_dot(X + c, ldk, vs, 0, min(b0 + kColBlk, k), c < k, [&](int b) { return b <= c; }, red);
      if (warp == 0 && lane < kColBlk && c < k) vf[c] = s;
    } else {
      const int c = b0 + (lane & (kColBlk - 1));
      double2* xo = out + sys * a.n;
      const T s = col_dot(X + c, ldk, vs, b0 + 1, k, c < k, [&](int b) { return b > c; }, red);
      if (warp == 0 && lane < kColBlk && c < k) xo[idx[Pm[c]]] = out_val(a, w, idx[Pm[c]], cadd(vs[c], s));
    }
    __syncthreads();
  }
}

// tri_task for right-hand sides in pairs (r, r + 1): the same products, each inverse-block
// entry loaded once for both systems; v1 = vs + vstride holds the second system's vector.
template <typename T, int SWEEP>
__device__ __forceinline__ void tri_task_pair(const SolveLaunch& a, const FrontDesc& d, int b0, int nrows, int w,
                                              const double2* __restrict__ in, double2* __restrict__ out, T* vs,
                                              int vstride, T (*red0)[32], T (*red1)[32]) {
  const int k = d.k, ldk = d.ldk;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* X = reinterpret_cast<const T*>(a.istore) + (size_t)w * a.istore_stride + d.iv_off;
  const int* Pm = a.perm + (size_t)w * a.perm_stride + d.piv_off;
  const int* idx = a.P.idx + d.idx_off;
  const Kids kids = load_kids(a, d);
  T* v0 = vs;
  T* v1 = vs + vstride;
  for (int r = a.r0; r < a.r0 + a.nr; r += 2) {
    const size_t sys0 = (size_t)w * a.nrhs + r, sys1 = sys0 + 1;
    T* vbs0 = reinterpret_cast<T*>(a.vb) + sys0 * a.vec_stride;
    T* vbs1 = reinterpret_cast<T*>(a.vb) + sys1 * a.vec_stride;
    T* vf0 = vbs0 + d.v_off;
    T* vf1 = vbs1 + d.v_off;
    if (SWEEP == 0 || SWEEP == 2) {
      const double2* rhs0 = in + sys0 * a.n;
      const double2* rhs1 = in + sys1 * a.n;
      for (int s = tid; s < k; s += kThreads) {
        const int src = SWEEP == 0 ? Pm[s] : s;
        v0[s] = gather_slot(a, d, kids, rhs0, vbs0, src, w);
        v1[s] = gather_slot(a, d, kids, rhs1, vbs1, src, w);
      }
    } else {
      for (int s = tid; s < k; s += kThreads) {
        const bool mid = SWEEP == 3 && d.m == 0;
        v0[s] = mid ? mid_val(a, X, ldk, s, ldv(vf0 + s)) : ldv(vf0 + s);
        v1[s] = mid ? mid_val(a, X, ldk, s, ldv(vf1 + s)) : ldv(vf1 + s);
      }
    }
    __syncthreads();
    if (SWEEP == 0 || SWEEP == 1) {
      double2* xo0 = out + sys0 * a.n;
      double2* xo1 = out + sys1 * a.n;
      for (int rr = warp; rr < nrows; rr += kWarps) {
        const int row = b0 + rr;
        if (row >= k) break;
        T s0, s1;
        warp_dot_pair(X + (size_t)row * ldk, v0, v1, SWEEP == 0 ? 0 : row, SWEEP == 0 ? row : k, lane, s0, s1);
        if (lane == 0) {
          if (SWEEP == 0) {
            vf0[row] = cadd(v0[row], s0);
            vf1[row] = cadd(v1[row], s1);
          } else {
            xo0[idx[row]] = cto64(s0);
            xo1[idx[row]] = cto64(s1);
          }
        }
      }
    } else {
      const int c = b0 + (lane & (kColBlk - 1));
      T s0, s1;
      if (SWEEP == 2) {
        col_dot_pair(X + c, ldk, v0, v1, 0, min(b0 + kColBlk, k), c < k, [&](int b) { return b <= c; }, red0, red1,
                     s0, s1);
        if (warp == 0 && lane < kColBlk && c < k) {
          vf0[c] = s0;
          vf1[c] = s1;
        }
      } else {
        col_dot_pair(X + c, ldk, v0, v1, b0 + 1, k, c < k, [&](int b) { return b > c; }, red0, red1, s0, s1);
        if (warp == 0 && lane < kColBlk && c < k) {
          const int cell = idx[Pm[c]];
          out[sys0 * a.n + cell] = out_val(a, w, cell, cadd(v0[c], s0));
          out[sys1 * a.n + cell] = out_val(a, w, cell, cadd(v1[c], s1));
        }
      }
    }
    __syncthreads();
  }
}

// rect_task for right-hand sides in pairs (each off-diagonal entry loaded once for both).
template <typename T, int SWEEP>
__device__ __forceinline__ void rect_task_pair(const SolveLaunch& a, const FrontDesc& d, int s0, int nrows, int w,
                                               double2* __restrict__ out, T* vs, int vstride, T (*red0)[32],
                                               T (*red1)[32]) {
  const int k = d.k, m = d.m, ld = d.ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* F = reinterpret_cast<const T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const T* X = reinterpret_cast<const T*>(a.istore) + (size_t)w * a.istore_stride + d.iv_off;
  const int* idx = a.P.idx + d.idx_off;
  const Kids kids = load_kids(a, d);
  T* v0 = vs;
  T* v1 = vs + vstride;
  for (int r = a.r0; r < a.r0 + a.nr; r += 2) {
    const size_t sys0 = (size_t)w * a.nrhs + r, sys1 = sys0 + 1;
    T* vbs0 = reinterpret_cast<T*>(a.vb) + sys0 * a.vec_stride;
    T* vbs1 = reinterpret_cast<T*>(a.vb) + sys1 * a.vec_stride;
    T* vf0 = vbs0 + d.v_off;
    T* vf1 = vbs1 + d.v_off;
    const double2* xo0 = out + sys0 * a.n;
    const double2* xo1 = out + sys1 * a.n;
    if (SWEEP == 0 || SWEEP == 2) {
      for (int q = tid; q < k; q += kThreads) {
        v0[q] = ldv(vf0 + q);
        v1[q] = ldv(vf1 + q);
      }
    } else {
      for (int t = tid; t < m; t += kThreads) {
        const int cell = idx[k + t];
        v0[t] = cfrom<T>(SWEEP == 3 ? xm_val(a, w, cell, ldv(xo0 + cell)) : ldv(xo0 + cell));
        v1[t] = cfrom<T>(SWEEP == 3 ? xm_val(a, w, cell, ldv(xo1 + cell)) : ldv(xo1 + cell));
      }
    }
    __syncthreads();
    if (SWEEP == 0 || SWEEP == 1) {
      // rows s0 + warp (and s0 + warp + kWarps in a tall task), one at a time, both systems per load
      const int lim = SWEEP == 0 ? m : k, len = SWEEP == 0 ? k : m;
      for (int rr = warp; rr < nrows; rr += kWarps) {
        const int ro = s0 + rr;
        if (ro >= lim) break;
        const T* Fr = SWEEP == 0 ? F + (size_t)(k + ro) * ld : F + (size_t)ro * ld + k;
        const T g0 = SWEEP == 0 ? gather_slot(a, d, kids, (const double2*)nullptr, vbs0, k + ro) : ldv(vf0 + ro);
        const T g1 = SWEEP == 0 ? gather_slot(a, d, kids, (const double2*)nullptr, vbs1, k + ro) : ldv(vf1 + ro);
        T p0, p1;
        warp_dot_pair(Fr, v0, v1, 0, len, lane, p0, p1);
        if (lane == 0) {
          vf0[SWEEP == 0 ? k + ro : ro] = csub(g0, p0);
          vf1[SWEEP == 0 ? k + ro : ro] = csub(g1, p1);
        }
      }
    } else {
      const int cols = SWEEP == 2 ? m : k;
      const int rows = SWEEP == 2 ? k : m;
      const int c = s0 + (lane & (kColBlk - 1));
      const bool mine = warp == 0 && lane < kColBlk && c < cols;
      const T* base = SWEEP == 2 ? F + k + c : F + (size_t)k * ld + c;
      T g0 = czero<T>(), g1 = czero<T>();
      if (mine) {
        if (SWEEP == 2) {
          g0 = gather_slot(a, d, kids, (const double2*)nullptr, vbs0, k + c);
          g1 = gather_slot(a, d, kids, (const double2*)nullptr, vbs1, k + c);
        } else {
          g0 = mid_val(a, X, d.ldk, c, ldv(vf0 + c));
          g1 = mid_val(a, X, d.ldk, c, ldv(vf1 + c));
        }
      }
      T p0, p1;
      col_dot_pair(base, ld, v0, v1, 0, rows, c < cols, [](int) { return true; }, red0, red1, p0, p1);
      if (mine) {
        vf0[SWEEP == 2 ? k + c : c] = csub(g0, p0);
        vf1[SWEEP == 2 ? k + c : c] = csub(g1, p1);
      }
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
__device__ __forceinline__ void rect_task(const SolveLaunch& a, const FrontDesc& d, int s0, int nrows, int w,
                                          double2* __restrict__ out, T* vs, T (*red)[32]) {
  const int k = d.k, m = d.m, ld = d.ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* F = reinterpret_cast<const T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const int* idx = a.P.idx + d.idx_off;
  const Kids kids = load_kids(a, d);
  for (int r = a.r0; r < a.r0 + a.nr; ++r) {
    const size_t sys = (size_t)w * a.nrhs + r;
    T* vbs = reinterpret_cast<T*>(a.vb) + sys * a.vec_stride;
    T* vf = vbs + d.v_off;
    const double2* xo = out + sys * a.n;
    if (SWEEP == 0 || SWEEP == 2) {
      for (int s = tid; s < k; s += kThreads) vs[s] = ldv(vf + s);
    } else {
      for (int t = tid; t < m; t += kThreads)
        vs[t] = cfrom<T>(SWEEP == 3 ? xm_val(a, w, idx[k + t], ldv(xo + idx[k + t])) : ldv(xo + idx[k + t]));
    }
    __syncthreads();
    if (SWEEP == 0 || SWEEP == 1) {
      // rows s0 + warp and s0 + warp + kWarps, their loads interleaved
      const int lim = SWEEP == 0 ? m : k, len = SWEEP == 0 ? k : m;
      const int ra = s0 + warp, rb = nrows > kWarps ? ra + kWarps : lim;   // a tall task: two rows per warp
      if (ra < lim) {
        const T* Fa = SWEEP == 0 ? F + (size_t)(k + ra) * ld : F + (size_t)ra * ld + k;
        const T* Fb = SWEEP == 0 ? F + (size_t)(k + rb) * ld : F + (size_t)rb * ld + k;
        // the values the products are subtracted from, fetched before the products
        const T ga = SWEEP == 0 ? gather_slot(a, d, kids, (const double2*)nullptr, vbs, k + ra) : ldv(vf + ra);
        if (rb < lim) {
          const T gb = SWEEP == 0 ? gather_slot(a, d, kids, (const double2*)nullptr, vbs, k + rb) : ldv(vf + rb);
          T sa, sb;
          warp_dot2(Fa, Fb, vs, 0, len, lane, sa, sb);
          if (lane == 0) {
            vf[SWEEP == 0 ? k + ra : ra] = csub(ga, sa);
            vf[SWEEP == 0 ? k + rb : rb] = csub(gb, sb);
          }
        } else {
          const T sa = warp_dot(Fa, vs, 0, len, lane);
          if (lane == 0) vf[SWEEP == 0 ? k + ra : ra] = csub(ga, sa);
        }
      }
    } else {
      const int cols = SWEEP == 2 ? m : k;
      const int rows = SWEEP == 2 ? k : m;
      const int c = s0 + (lane & (kColBlk - 1));
      const bool mine = warp == 0 && lane < kColBlk && c < cols;
      const T* base = SWEEP == 2 ? F + k + c : F + (size_t)k * ld + c;
      // the value the product is subtracted from, fetched before the product
      T g = czero<T>();
      if (mine)
        g = SWEEP == 2 ? gather_slot(a, d, kids, (const double2*)nullptr, vbs, k + c)
                       : mid_val(a, reinterpret_cast<const T*>(a.istore) + (size_t)w * a.istore_stride + d.iv_off,
                                 d.ldk, c, ldv(vf + c));
      const T s = col_dot(base, ld, vs, 0, rows, c < cols, [](int) { return true; }, red);
      if (mine) vf[SWEEP == 2 ? k + c : c] = csub(g, s);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// A whole medium front (64 < n <= flow_cta_max_n()) done by one CTA: both
// products of the front in one task, separated by a CTA barrier instead of a
// completion counter.  Row products give each row a group of G lanes (G chosen
// so that a lane holds at most 8 entries of a row, two rows in flight per
// group); column products give each column a lane and split the rows over the
// warps when there are fewer than 8 column groups, reducing the partial sums in
// a fixed order.
// ---------------------------------------------------------------------------
template <typename T, int G, typename Lo, typename Hi, typename Out>
__device__ __forceinline__ void rows_dot_g(const T* __restrict__ A, int ld, int nrows, const T* vec, Lo lo, Hi hi,
                                           Out out) {
  constexpr int NG = kThreads / G;       // row groups in the CTA
  constexpr int UN = 8;
  const int sl = threadIdx.x & (G - 1), grp = threadIdx.x / G;
  for (int base = 0; base < nrows; base += 2 * NG) {   // same trip count for every lane of a warp
    const int i0 = base + grp, i1 = base + NG + grp;
    const bool v0 = i0 < nrows, v1 = i1 < nrows;
    const int h0 = v0 ? hi(i0) : 0, h1 = v1 ? hi(i1) : 0;
    int c0 = (v0 ? lo(i0) : 0) + sl, c1 = (v1 ? lo(i1) : 0) + sl;
    const T* r0 = A + (size_t)(v0 ? i0 : 0) * ld;
    const T* r1 = A + (size_t)(v1 ? i1 : 0) * ld;
    T a0 = czero<T>(), a1 = czero<T>();
    while (c0 < h0 || c1 < h1) {
      T f0[UN], f1[UN];
#pragma unroll
      for (int u = 0; u < UN; ++u) {
        f0[u] = c0 + u * G < h0 ? r0[c0 + u * G] : czero<T>();
        f1[u] = c1 + u * G < h1 ? r1[c1 + u * G] : czero<T>();
      }
#pragma unroll
      for (int u = 0; u < UN; ++u) {
        if (c0 + u * G < h0) a0 = cfma(f0[u], vec[c0 + u * G], a0);
        if (c1 + u * G < h1) a1 = cfma(f1[u], vec[c1 + u * G], a1);
      }
      c0 += UN * G;
      c1 += UN * G;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      a0.x += __shfl_xor_sync(0xffffffffu, a0.x, o);
      a0.y += __shfl_xor_sync(0xffffffffu, a0.y, o);
      a1.x += __shfl_xor_sync(0xffffffffu, a1.x, o);
      a1.y += __shfl_xor_sync(0xffffffffu, a1.y, o);
    }
    if (sl == 0) {
      if (v0) out(i0, a0);
      if (v1) out(i1, a1);
    }
  }
}

// out(i, sum_{c in [lo(i), hi(i))} A[i][c] vec[c]) for rows i < nrows; len = longest row
template <typename T, typename Lo, typename Hi, typename Out>
__device__ __forceinline__ void rows_dot(const T* __restrict__ A, int ld, int nrows, int len, const T* vec, Lo lo,
                                         Hi hi, Out out) {
  if (len <= 16) rows_dot_g<T, 2>(A, ld, nrows, vec, lo, hi, out);
  else if (len <= 32) rows_dot_g<T, 4>(A, ld, nrows, vec, lo, hi, out);
  else if (len <= 64) rows_dot_g<T, 8>(A, ld, nrows, vec, lo, hi, out);
  else if (len <= 128) rows_dot_g<T, 16>(A, ld, nrows, vec, lo, hi, out);
  else rows_dot_g<T, 32>(A, ld, nrows, vec, lo, hi, out);
}

// out(j, sum_{r in [lo(j), hi(j))} A[r][j] vec[r]) for columns j < ncols (rows < nrows)
template <typename T, typename Lo, typename Hi, typename Out>
__device__ __forceinline__ void cols_dot(const T* __restrict__ A, int ld, int ncols, int nrows, const T* vec, Lo lo,
                                         Hi hi, Out out, T (*red)[32]) {
  constexpr int UN = sizeof(T) == 8 ? 16 : 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncg = (ncols + 31) / 32;
  const int ns = ncg >= kWarps ? 1 : kWarps / ncg;     // row slices per column group
  const int gpr = kWarps / ns;                          // column groups per round
  const int slen = (nrows + ns - 1) / ns;
  for (int g0 = 0; g0 < ncg; g0 += gpr) {
    const int gi = g0 + warp / ns, si = warp - (warp / ns) * ns;
    const int j = gi * 32 + lane;
    T acc0 = czero<T>(), acc1 = czero<T>();
    if (warp / ns < gpr && gi < ncg && j < ncols) {
      const int rb = max(lo(j), si * slen), re = min(hi(j), min(nrows, (si + 1) * slen));
      int r = rb;
      for (; r + UN - 1 < re; r += UN) {
        T f[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) f[u] = A[(size_t)(r + u) * ld + j];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
          if (u & 1) acc1 = cfma(f[u], vec[r + u], acc1);
          else acc0 = cfma(f[u], vec[r + u], acc0);
        }
      }
      for (; r < re; ++r) acc0 = cfma(A[(size_t)r * ld + j], vec[r], acc0);
    }
    if (ns > 1) {
      red[warp][lane] = cadd(acc0, acc1);
      __syncthreads();
      const int gj = g0 + warp, jj = gj * 32 + lane;
      if (warp < gpr && gj < ncg && jj < ncols) {
        T sum = red[warp * ns][lane];
        for (int q = 1; q < ns; ++q) sum = cadd(sum, red[warp * ns + q][lane]);
        out(jj, sum);
      }
      __syncthreads();
    } else if (gi < ncg && j < ncols) {
      out(j, cadd(acc0, acc1));
    }
  }
}

template <typename T, int SWEEP>
__device__ __forceinline__ void medium_front(const SolveLaunch& a, const FrontDesc& d, int w,
                                             const double2* __restrict__ in, double2* __restrict__ out, T* vs,
                                             T (*red)[32]) {
  const int k = d.k, m = d.m, n = d.n, ldk = d.ldk, ld = d.ld;
  const int tid = threadIdx.x;
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
    double2* xo = out + sys * a.n;
    if (SWEEP == 0 || SWEEP == 2) {
      const double2* rhs = in + sys * a.n;
      for (int s = tid; s < n; s += 2 * kThreads) {
        const int s2 = s + kThreads;
        const T g1 = gather_slot(a, d, kids, rhs, vbs, (SWEEP == 0 && s < k) ? Pm[s] : s, w);
        const T g2 = s2 < n ? gather_slot(a, d, kids, rhs, vbs, (SWEEP == 0 && s2 < k) ? Pm[s2] : s2, w)
                            : czero<T>();
        vs[s] = g1;
        if (s2 < n) vs[s2] = g2;
      }
    } else {
      for (int s = tid; s < k; s += kThreads) vs[s] = SWEEP == 3 ? mid_val(a, X, ldk, s, ldv(vf + s)) : ldv(vf + s);
      for (int t = tid; t < m; t += kThreads) {
        const T x = cfrom<T>(SWEEP == 3 ? xm_val(a, w, idx[k + t], ldv(xo + idx[k + t])) : ldv(xo + idx[k + t]));
        vs[k + t] = SWEEP == 3 ? csub(czero<T>(), x) : x;
      }
    }
    __syncthreads();
    if (SWEEP == 0) {                              // y = X_L (P v)_k;  u = v_m - L21 y
      rows_dot(X, ldk, k, k, vs, [](int) { return 0; }, [](int i) { return i; },
               [&](int i, T acc) { ws[i] = cadd(vs[i], acc); });
      __syncthreads();
      rows_dot(F + (size_t)k * ld, ld, m, k, ws, [](int) { return 0; }, [&](int) { return k; },
               [&](int t, T acc) { vf[k + t] = csub(vs[k + t], acc); });
      for (int s = tid; s < k; s += kThreads) vf[s] = ws[s];
    } else if (SWEEP == 1) {                       // z = y - U12 x_m;  x_k = X_U z
      rows_dot(F + k, ld, k, m, vs + k, [](int) { return 0; }, [&](int) { return m; },
               [&](int i, T acc) { ws[i] = csub(vs[i], acc); });
      __syncthreads();
      rows_dot(X, ldk, k, k, ws, [](int i) { return i; }, [&](int) { return k; },
               [&](int i, T acc) { xo[idx[i]] = cto64(acc); });
    } else if (SWEEP == 2) {                       // w = X_U^T v_k;  u = v_m - U12^T w
      cols_dot(X, ldk, k, k, vs, [](int) { return 0; }, [](int j) { return j + 1; },
               [&](int j, T acc) { ws[j] = acc; }, red);
      __syncthreads();
      cols_dot(F + k, ld, m, k, ws, [](int) { return 0; }, [&](int) { return k; },
               [&](int t, T acc) { vf[k + t] = csub(vs[k + t], acc); }, red);
      for (int s = tid; s < k; s += kThreads) vf[s] = ws[s];
    } else {                                       // t = w - L21^T x_m;  x_k = P^T X_L^T t   (vs[k..n) = -x_m)
      cols_dot(F + (size_t)k * ld, ld, k, m, vs + k, [](int) { return 0; }, [&](int) { return m; },
               [&](int j, T acc) { ws[j] = cadd(vs[j], acc); }, red);
      __syncthreads();
      cols_dot(X, ldk, k, k, ws, [](int j) { return j + 1; }, [&](int) { return k; },
               [&](int j, T acc) { xo[idx[Pm[j]]] = out_val(a, w, idx[Pm[j]], cadd(ws[j], acc)); }, red);
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
constexpr int kCtaWholeMaxN = 320;   // largest front swept whole by one CTA

// resident CTAs per SM the register allocation aims for: small problems (few
// tasks, each latency-bound) keep more registers per thread, large ones (the
// sweeps bound by loads in flight) run more CTAs
constexpr int kFlowBlocksNarrow = 4, kFlowBlocksWide = 6;

// NRP = 2: large-front tasks take the right-hand sides in pairs (the launch's count of
// them per wavelength is even); the second vector of a pair sits vstride entries above
// the first in shared memory.
template <typename T, int SWEEP, int MINB, int NRP>
__global__ void __launch_bounds__(kThreads, MINB)
flow_kernel(SolveLaunch a, FlowQueue q, const double2* __restrict__ in, double2* __restrict__ out, int vstride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red[NRP][kWarps][32];
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
        const int f = (int)((unsigned)task.x & (unsigned)kSweepFrontMask);
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
    const bool med = (code >> 31) != 0;          // a whole medium front
    const bool rect = !med && ((code >> 30) & 1u) != 0;
    const int f = (int)(code & (unsigned)kSweepFrontMask);
    const int rows = (code & (unsigned)kSweepTaskTall) ? 2 * kRowBlk : kRowBlk;   // row tasks
    const FrontDesc d = a.P.fronts[f];
    if (tid == 0) {
      bool ok = true;
      if (med) {
        if (kUp) {
          for (int ci = 0; ci < d.nchild && ok; ++ci) {
            const int c = a.P.children[d.child0 + ci];
            ok = wait_ge(dn + c, q.need_all[c], q.err);
          }
        } else if (d.parent >= 0) {
          ok = wait_ge(dn + d.parent, q.need_all[d.parent], q.err);
        }
      } else if (kUp) {
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
    if (med) medium_front<T, SWEEP>(a, d, w, in, out, vs, red[0]);
    else if (NRP == 2 && rect) rect_task_pair<T, SWEEP>(a, d, task.y, rows, w, out, vs, vstride, red[0], red[NRP - 1]);
    else if (NRP == 2) tri_task_pair<T, SWEEP>(a, d, task.y, rows, w, in, out, vs, vstride, red[0], red[NRP - 1]);
    else if (rect) rect_task<T, SWEEP>(a, d, task.y, rows, w, out, vs, red[0]);
    else tri_task<T, SWEEP>(a, d, task.y, rows, w, in, out, vs, red[0]);
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      // phase 1: inverse-block tasks bottom-up, off-diagonal tasks top-down
      if (!med && (kUp ? !rect : rect)) atomicAdd(ph1 + (size_t)wl * nf + f, 1);
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

// vector entries of one shared-memory slot (a pair variant holds two slots)
int flow_slot(int vmax) { return vmax > kWarps * kWarpSlice ? vmax : kWarps * kWarpSlice; }
size_t flow_smem(int vmax, size_t es, bool pair) { return (size_t)flow_slot(vmax) * es * (pair ? 2 : 1); }

template <typename T>
void launch_sweep_flow(const SolveLaunch& a, int sweep, const FlowQueue& q, int vmax, int grid, const void* in,
                       void* out, cudaStream_t s, bool wide, bool pairs) {
  if (q.nunits <= 0) return;
  // right-hand sides in pairs for the complex64 factors when the count per wavelength is even
  const bool pair = pairs && sizeof(T) == 8 && a.nr >= 2 && a.nr % 2 == 0;
  const size_t smem = flow_smem(vmax, sizeof(T), pair);
  const int vst = flow_slot(vmax);
  const double2* i = reinterpret_cast<const double2*>(in);
  double2* o = reinterpret_cast<double2*>(out);
#define FDFD_FLOW_LAUNCH(B, P)                                                                 \
  switch (sweep) {                                                                             \
    case 0: flow_kernel<T, 0, B, P><<<grid, kThreads, smem, s>>>(a, q, i, o, vst); break;      \
    case 1: flow_kernel<T, 1, B, P><<<grid, kThreads, smem, s>>>(a, q, i, o, vst); break;      \
    case 2: flow_kernel<T, 2, B, P><<<grid, kThreads, smem, s>>>(a, q, i, o, vst); break;      \
    default: flow_kernel<T, 3, B, P><<<grid, kThreads, smem, s>>>(a, q, i, o, vst); break;     \
  }
  if constexpr (sizeof(T) == 8) {
    if (pair) {
      if (wide) { FDFD_FLOW_LAUNCH(kFlowBlocksWide, 2) } else { FDFD_FLOW_LAUNCH(kFlowBlocksNarrow, 2) }
      return;
    }
  }
  if (wide) { FDFD_FLOW_LAUNCH(kFlowBlocksWide, 1) } else { FDFD_FLOW_LAUNCH(kFlowBlocksNarrow, 1) }
#undef FDFD_FLOW_LAUNCH
}

int flow_blocks_per_sm(int elem_bytes, int vmax, bool wide, bool pair) {
  int nb = 0;
  pair = pair && elem_bytes == 8;
  const size_t smem = flow_smem(vmax, elem_bytes, pair);
  cudaError_t e;
  if (pair)
    e = wide ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, flow_kernel<float2, 1, kFlowBlocksWide, 2>, kThreads, smem)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, flow_kernel<float2, 1, kFlowBlocksNarrow, 2>, kThreads, smem);
  else if (wide)
    e = elem_bytes == 8
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, flow_kernel<float2, 1, kFlowBlocksWide, 1>, kThreads, smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, flow_kernel<double2, 1, kFlowBlocksWide, 1>, kThreads, smem);
  else
    e = elem_bytes == 8
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, flow_kernel<float2, 1, kFlowBlocksNarrow, 1>, kThreads, smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, flow_kernel<double2, 1, kFlowBlocksNarrow, 1>, kThreads, smem);
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

int sweep_row_block() { return kRowBlk; }

int flow_whole_max_n() { return kWarpSlice / 2; }
int flow_cta_max_n() { return kCtaWholeMaxN; }
int sweep_col_block() { return kColBlk; }

cudaError_t solve_init_attributes() {
  const int lim = 160 * 1024;
  cudaError_t e = cudaSuccess;
#define FDFD_ATTR(K, T, S, P)                                                                          \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K<T, S, kFlowBlocksNarrow, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K<T, S, kFlowBlocksWide, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  FDFD_ATTR(flow_kernel, float2, 0, 1) FDFD_ATTR(flow_kernel, float2, 1, 1) FDFD_ATTR(flow_kernel, float2, 2, 1)
  FDFD_ATTR(flow_kernel, float2, 3, 1) FDFD_ATTR(flow_kernel, double2, 0, 1) FDFD_ATTR(flow_kernel, double2, 1, 1)
  FDFD_ATTR(flow_kernel, double2, 2, 1) FDFD_ATTR(flow_kernel, double2, 3, 1)
  FDFD_ATTR(flow_kernel, float2, 0, 2) FDFD_ATTR(flow_kernel, float2, 1, 2) FDFD_ATTR(flow_kernel, float2, 2, 2)
  FDFD_ATTR(flow_kernel, float2, 3, 2)
#undef FDFD_ATTR
  return e;
}

template void launch_sweep_flow<float2>(const SolveLaunch&, int, const FlowQueue&, int, int, const void*, void*,
                                        cudaStream_t, bool, bool);
template void launch_sweep_flow<double2>(const SolveLaunch&, int, const FlowQueue&, int, int, const void*, void*,
                                         cudaStream_t, bool, bool);

}  // namespace fdfd
