// Numeric multifrontal factorisation (paper Sec. II, "numerical factorization").
//
// Every front f is a dense (k+m) x (k+m) matrix, row-major with row stride ld,
// ordered [k pivots | m boundary variables]:
//     [F11 F12]      P F11 = L11 U11,  U12 = L11^-1 P F12,
//     [F21 F22]      L21 = F21 U11^-1,  S = F22 - L21 U12.
// After factorisation the front holds L11\U11 (unit L), U12, L21 and, in its
// trailing m x m block, the update matrix S that the parent extend-adds.  S is
// never modified afterwards, so the fronts of an unchanged subtree remain valid
// update sources for a later design refactor.
//
// Pivoting is partial, restricted to the k fully-summed rows of the front.
// The largest |L| entry of each front is recorded as its pivot-growth figure.
// All reductions run in a fixed order: a factorisation is a deterministic
// function of its inputs, bit for bit.
#include <algorithm>
#include <cfloat>

#include "kernels.h"

namespace fdfd {

namespace {

constexpr int kBuildWarps = 8;
constexpr int kSwpInts = kSwapScratchInts;   // per panel: count + up to 64 (dst, src) row pairs

// entry (i, j) of a symmetric-form child's update matrix (its lower triangle is stored)
template <typename T>
__device__ __forceinline__ T child_sym(const T* st, const FrontDesc& c, int i, int j) {
  return i >= j ? st[c.st_off + (size_t)(c.k + i) * c.ld + c.k + j] : st[c.st_off + (size_t)(c.k + j) * c.ld + c.k + i];
}

// ---------------------------------------------------------------------------
// Front build: F = originals + sum over children of their update matrices,
// gathered through the children's inverse extend-add maps (no atomics).
// One warp per front row, 8 rows per CTA.  The first task of a front also
// clears its growth figure.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBuildWarps * 32)
build_kernel(FactorLaunch a, const int2* __restrict__ tasks) {
  const int w = blockIdx.y + a.w0;
  const int2 t = tasks[blockIdx.x];
  const int f = t.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const FrontDesc d = a.P.fronts[f];
  if (t.y == 0 && threadIdx.x == 0) a.growth[(size_t)w * a.n_fronts + f] = 0.f;   // accumulated by atomicMax later
  const int r = t.y + warp;
  if (r >= d.n) return;
  T* st = reinterpret_cast<T*>(a.store) + (size_t)w * a.store_stride;
  T* F = st + d.st_off + (size_t)r * d.ld;
  if (a.sym) {
    // symmetric form: columns <= r only; children's update matrices read from their
    // lower triangles, originals scaled by D of the row's cell
    FrontDesc c0, c1;
    int ia = -1, ib = -1;
    if (d.nchild > 0) { c0 = a.P.fronts[a.P.children[d.child0]]; ia = a.P.inv[c0.inv_off + r]; }
    if (d.nchild > 1) { c1 = a.P.fronts[a.P.children[d.child0 + 1]]; ib = a.P.inv[c1.inv_off + r]; }
    for (int b = lane; b <= r; b += 32) {
      T v = czero<T>();
      if (ia >= 0) { const int i0 = a.P.inv[c0.inv_off + b]; if (i0 >= 0) v = cadd(v, child_sym(st, c0, ia, i0)); }
      if (ib >= 0) { const int i1 = a.P.inv[c1.inv_off + b]; if (i1 >= 0) v = cadd(v, child_sym(st, c1, ib, i1)); }
      F[b] = v;
    }
    __syncwarp();
    const int e0 = a.P.orig_ptr[d.orig_off + r], e1 = a.P.orig_ptr[d.orig_off + r + 1];
    const double2 Dr = sym_scale(a.C, w, a.P.idx[d.idx_off + r]);
    for (int e = e0 + lane; e < e1; e += 32) {
      const int b = a.P.orig_col[e];
      if (b <= r) F[b] = cadd(F[b], cfrom<T>(cmul(Dr, stencil_entry(a.C, w, a.P.orig_code[e]))));
    }
    return;
  }
  // up to two children (nested dissection splits into at most two parts)
  const T* S0 = nullptr;
  const T* S1 = nullptr;
  const int* inv0 = nullptr;
  const int* inv1 = nullptr;
  int ld0 = 0, ld1 = 0;
  if (d.nchild > 0) {
    const FrontDesc c = a.P.fronts[a.P.children[d.child0]];
    const int ia = a.P.inv[c.inv_off + r];
    if (ia >= 0) {
      S0 = st + c.st_off + (size_t)(c.k + ia) * c.ld + c.k;
      inv0 = a.P.inv + c.inv_off;
      ld0 = c.ld;
    }
  }
  if (d.nchild > 1) {
    const FrontDesc c = a.P.fronts[a.P.children[d.child0 + 1]];
    const int ia = a.P.inv[c.inv_off + r];
    if (ia >= 0) {
      S1 = st + c.st_off + (size_t)(c.k + ia) * c.ld + c.k;
      inv1 = a.P.inv + c.inv_off;
      ld1 = c.ld;
    }
  }
  (void)ld0; (void)ld1;
  // children's rows, gathered through their maps: eight columns per lane in
  // flight (maps first, then the update-matrix entries they select)
  constexpr int UN = 8;
  for (int b0 = lane; b0 < d.n; b0 += 32 * UN) {
    int i0[UN], i1[UN];
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      const int b = b0 + 32 * u;
      i0[u] = (S0 && b < d.n) ? inv0[b] : -1;
      i1[u] = (S1 && b < d.n) ? inv1[b] : -1;
    }
    T v[UN];
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      v[u] = czero<T>();
      if (i0[u] >= 0) v[u] = cadd(v[u], S0[i0[u]]);
      if (i1[u] >= 0) v[u] = cadd(v[u], S1[i1[u]]);
    }
#pragma unroll
    for (int u = 0; u < UN; ++u)
      if (b0 + 32 * u < d.n) F[b0 + 32 * u] = v[u];
  }
  // the row's original entries (each column at most once), one lane each
  __syncwarp();
  const int e0 = a.P.orig_ptr[d.orig_off + r], e1 = a.P.orig_ptr[d.orig_off + r + 1];
  for (int e = e0 + lane; e < e1; e += 32) {
    const int b = a.P.orig_col[e];
    F[b] = cadd(F[b], cfrom<T>(stencil_entry(a.C, w, a.P.orig_code[e])));
  }
}

// max that lets a NaN win, so that a poisoned front is always flagged
template <typename R>
__device__ __forceinline__ R nanmax(R a, R b) {
  if (a != a) return a;
  if (b != b) return b;
  return a > b ? a : b;
}

// complex value of lane src, for every lane of the warp
template <typename T>
__device__ __forceinline__ T shfl_c(T v, int src) {
  v.x = __shfl_sync(0xffffffffu, v.x, src);
  v.y = __shfl_sync(0xffffffffu, v.y, src);
  return v;
}

// warp argmax of |v|^2 with ties going to the smaller index
template <typename R>
__device__ __forceinline__ void warp_argmax(R& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    R ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
  }
}

// ---------------------------------------------------------------------------
// Small fronts: one CTA per front, assembled in shared memory (the children's
// update matrices, then the original entries, one thread per row), factored in
// registers and written back once with its triangular inverses.
//
// The factorisation holds the front with lanes over rows and warps over
// columns: thread (lane, warp) owns the entries (lane + 32 i, warp + NWARP jj),
// i < RI, jj < RJ.  Partial pivoting over the k pivot rows moves no rows: step j
// takes the unused pivot row p_j with the largest |F[r][j]| (ties to the smaller
// row), every other unused row takes l_r = F[r][j] / F[p_j][j], updates
// F[r][c] -= l_r F[p_j][c] for c > j, and l_r goes to column j of the shared
// copy.  The warp owning column j + 1 publishes its entries and the argmax key
// of the unused candidates (|v|^2 as float with its 7 low bits replaced by
// 127 - row: the larger magnitude wins to 16 bits, ties to the smaller row, NaN
// wins) while it finishes step j; after one barrier every warp takes p_j, the
// lane holding row p_j hands the warp its pivot-row entries through shared
// memory, and every thread updates its tile.  At the end the tile goes back to
// the shared copy where the multipliers are not: row p_j is pivot row j of
// L11\U11 and U12, rows >= k are L21 and the update matrix S in place.
//
// Then the triangular inverses, one warp per row, lanes over the columns,
// from the factors in shared memory into the inverse store:
//   row i of L11^-1: X[i][i] = 1, X[i][l] = -sum_{l < m <= i} X[i][m] L[m][l], m descending;
//   row i of U11^-1: X[i][c] = (delta_ic - sum_{i <= l < c} X[i][l] U[l][c]) / U[c][c], l ascending.
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 256;
constexpr int kSmallNarrowN = 48;   // symmetric-form fronts up to this size run with kSmallThreads / 2 threads
constexpr int kSmallMaxK = 256;
constexpr int kSmallSlots = 3;      // columns per lane in the inverse rows (k <= 96)
constexpr int kSmallMaxN = 96;      // largest complex64 front of the small path (complex128: 64)

template <typename T>
__device__ __forceinline__ T pick_slot(const T (&v)[kSmallSlots], int q) {
  return q == 0 ? v[0] : (q == 1 ? v[1] : v[2]);
}
template <typename T, int KS>
__device__ __forceinline__ T pick_slot(const T (&v)[KS], int q) {
  T r = v[0];
#pragma unroll
  for (int t = 1; t < KS; ++t)
    if (q == t) r = v[t];
  return r;
}

// 1 / z as conj(z) / |z|^2 with a correctly rounded reciprocal (pivots here are
// far from the over/underflow range; a zero pivot gives inf/NaN, flagged as growth)
__device__ __forceinline__ double2 fast_crcp(double2 z) {
  const double s = __drcp_rn(z.x * z.x + z.y * z.y);
  return make_double2(z.x * s, -z.y * s);
}

// 1 / z for a pivot: conj(z) / |z|^2 with the hardware reciprocal estimate of
// |z|^2 refined by one Newton-Raphson step (double: the correctly rounded one)
__device__ __forceinline__ float2 pivot_rcp(float2 z) {
  const float dd = z.x * z.x + z.y * z.y;
  float s0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s0) : "f"(dd));
  const float sc = fmaf(s0, fmaf(-dd, s0, 1.0f), s0);
  return make_float2(z.x * sc, -z.y * sc);
}
__device__ __forceinline__ double2 pivot_rcp(double2 z) { return fast_crcp(z); }

// argmax key of a pivot candidate in row r < 128: |v|^2 (as float) with its 7
// low bits replaced by 127 - r; 0 means no candidate
template <typename R>
__device__ __forceinline__ unsigned small_key(R v2, int r) {
  return (__float_as_uint((float)v2) & ~127u) | (unsigned)(127 - r);
}

// x[jq] for a slot index known only at run time (uniform over the warp): one
// indexed branch instead of a chain of selects over the row's RJ registers
template <typename T, int RJ>
__device__ __forceinline__ T tile_slot(const T (&x)[RJ], int jq) {
  static_assert(RJ <= 16, "tile rows of at most 16 slots");
#define FDFD_SLOT(q) \
  case q:            \
    if constexpr (q < RJ) return x[q]; \
    break;
  switch (jq) {
    FDFD_SLOT(0) FDFD_SLOT(1) FDFD_SLOT(2) FDFD_SLOT(3) FDFD_SLOT(4) FDFD_SLOT(5) FDFD_SLOT(6) FDFD_SLOT(7)
    FDFD_SLOT(8) FDFD_SLOT(9) FDFD_SLOT(10) FDFD_SLOT(11) FDFD_SLOT(12) FDFD_SLOT(13) FDFD_SLOT(14) FDFD_SLOT(15)
    default: break;
  }
#undef FDFD_SLOT
  return x[0];
}

// The warp owning column jn posts the column's entries (its slot jq) to col and
// the argmax key of its unused pivot candidates (rows < k) to *key.
template <typename T, int RI, int RJ>
__device__ __forceinline__ void small_post_column(const T (&x)[RI][RJ], unsigned done, int jq, int n, int k, int lane,
                                                  T* col, unsigned* key) {
  using R = typename RealOf<T>::type;
  unsigned best = 0;
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    const int r = lane + 32 * i;
    const T v = tile_slot(x[i], jq);
    if (r < n) col[r] = v;
    if (r < k && !((done >> i) & 1u)) {
      const R a2 = cabs2(v);
      best = max(best, a2 == a2 ? small_key(a2, r) : (0xffffff80u | (unsigned)(127 - r)));
    }
  }
  best = __reduce_max_sync(0xffffffffu, best);
  if (lane == 0) *key = best;
}

template <typename T, int NWARP, int RI, int RJ, int MINB>
__global__ void __launch_bounds__(NWARP * 32, MINB)
lu_small_kernel(FactorLaunch a, const int* __restrict__ flist) {
  using R = typename RealOf<T>::type;
  constexpr int THREADS = NWARP * 32, NMAX = 32 * RI < NWARP * RJ ? 32 * RI : NWARP * RJ;
  static_assert(NMAX <= 128, "the argmax key holds the row in 7 bits");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);       // n x ls, ls = n | 1 (odd: rows by lane are conflict-free)
  __shared__ T s_col[2][NMAX];                 // column j of the step, double-buffered
  __shared__ __align__(16) T s_u[NWARP][RJ];   // each warp's columns of the pivot row
  __shared__ int s_i0[NMAX], s_i1[NMAX];       // the children's extend-add maps
  __shared__ int s_op[NMAX + 1];               // the rows' original-entry offsets
  __shared__ int s_pm[NMAX];                   // p_j: the row that became pivot row j
  __shared__ int s_pos[NMAX];                  // j for row p_j, k for the other rows
  __shared__ unsigned s_key[2];
  __shared__ R s_red[NWARP];
  const int w = blockIdx.y + a.w0;
  const int f = flist[blockIdx.x];
  const FrontDesc d = a.P.fronts[f];
  const int n = d.n, k = d.k, ls = n | 1;
  T* F = reinterpret_cast<T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // assemble the front in shared memory
  {
    const T* st = reinterpret_cast<const T*>(a.store) + (size_t)w * a.store_stride;
    FrontDesc c0, c1;
    const int nc = d.nchild;
    if (nc > 0) c0 = a.P.fronts[a.P.children[d.child0]];
    if (nc > 1) c1 = a.P.fronts[a.P.children[d.child0 + 1]];
    for (int c = tid; c <= n; c += THREADS) {
      if (c < n) {
        s_i0[c] = nc > 0 ? a.P.inv[c0.inv_off + c] : -1;
        s_i1[c] = nc > 1 ? a.P.inv[c1.inv_off + c] : -1;
        s_pos[c] = k;
      }
      s_op[c] = a.P.orig_ptr[d.orig_off + c];
    }
    __syncthreads();
    // the children's update-matrix rows through their inverse extend-add maps
#pragma unroll 2
    for (int r = warp; r < n; r += NWARP) {
      const int ia = s_i0[r], ib = s_i1[r];
      const T* S0 = ia >= 0 ? st + c0.st_off + (size_t)(c0.k + ia) * c0.ld + c0.k : nullptr;
      const T* S1 = ib >= 0 ? st + c1.st_off + (size_t)(c1.k + ib) * c1.ld + c1.k : nullptr;
      for (int c = lane; c < n; c += 32) {
        T v = czero<T>();
        if (S0) { const int i0 = s_i0[c]; if (i0 >= 0) v = cadd(v, S0[i0]); }
        if (S1) { const int i1 = s_i1[c]; if (i1 >= 0) v = cadd(v, S1[i1]); }
        S[r * ls + c] = v;
      }
    }
    __syncthreads();
    // the original entries, one thread per row (each column at most once per row)
    for (int r = tid; r < n; r += THREADS) {
      const int e0 = s_op[r], e1 = s_op[r + 1];
      for (int e = e0; e < e1; ++e) {
        const int b = a.P.orig_col[e];
        S[r * ls + b] = cadd(S[r * ls + b], cfrom<T>(stencil_entry(a.C, w, a.P.orig_code[e])));
      }
    }
  }
  __syncthreads();
  T x[RI][RJ];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int jj = 0; jj < RJ; ++jj) {
      const int r = lane + 32 * i, c = warp + NWARP * jj;
      x[i][jj] = (r < n && c < n) ? S[r * ls + c] : czero<T>();
    }
  unsigned done = 0;   // bit i: row lane + 32 i has been taken as a pivot row
  R gmax = 0;
  if (k > 0 && warp == 0) small_post_column<T, RI, RJ>(x, done, 0, n, k, lane, s_col[0], &s_key[0]);
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    const int par = j & 1, sw = j % NWARP;   // column j is slot j / NWARP of warp sw
    const int p = min(127 - (int)(s_key[par] & 127u), n - 1);   // (a candidate always exists)
    const T pv = s_col[par][p];
    const T inv = pivot_rcp(pv);
    if (tid == 0) {
      if (pv.x == 0 && pv.y == 0) gmax = INFINITY;
      s_pm[j] = p;
      s_pos[p] = j;
    }
    // the lane holding row p hands its warp the pivot row's entries in the warp's columns
    if (lane == (p & 31)) {
      const int pi = p >> 5;
#pragma unroll
      for (int i = 0; i < RI; ++i)
        if (i == pi) {
#pragma unroll
          for (int jj = 0; jj < RJ; ++jj) s_u[warp][jj] = x[i][jj];
        }
      done |= 1u << pi;
    }
    __syncwarp();
    T l[RI];
    bool act[RI];
#pragma unroll
    for (int i = 0; i < RI; ++i) {
      const int r = lane + 32 * i;
      act[i] = r < n && !((done >> i) & 1u);
      l[i] = act[i] ? cmul(s_col[par][r], inv) : czero<T>();
    }
    if (warp == sw) {
      // the multipliers take column j of the shared copy
#pragma unroll
      for (int i = 0; i < RI; ++i)
        if (act[i]) {
          S[(lane + 32 * i) * ls + j] = l[i];
          gmax = nanmax(gmax, cabs2(l[i]));
        }
    }
    // every column of the unused rows: the ones up to j are below the row's own
    // pivot step (or < k), so they are never written back
#pragma unroll
    for (int jj = 0; jj < RJ; ++jj) {
      const T u = s_u[warp][jj];
#pragma unroll
      for (int i = 0; i < RI; ++i)
        if (act[i]) x[i][jj] = cfms(l[i], u, x[i][jj]);
    }
    if (j + 1 < k && warp == (j + 1) % NWARP)
      small_post_column<T, RI, RJ>(x, done, (j + 1) / NWARP, n, k, lane, s_col[par ^ 1], &s_key[par ^ 1]);
    __syncthreads();
  }
  // the tile back to the shared copy, except where the multipliers are (columns
  // before the row's own pivot step; every column < k of the boundary rows)
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    const int r = lane + 32 * i;
    const int lim = r < n ? s_pos[r] : 0;
#pragma unroll
    for (int jj = 0; jj < RJ; ++jj) {
      const int c = warp + NWARP * jj;
      if (r < n && c < n && c >= lim) S[r * ls + c] = x[i][jj];
    }
  }
  __syncthreads();
  // triangular inverses, rows i = warp, warp + NWARP, ...; lane holds columns lane + 32 q (KS slots: k <= 32 KS)
  constexpr int KS = (NMAX + 31) / 32;
  T* Xg = reinterpret_cast<T*>(a.istore) + (size_t)w * a.istore_stride + d.iv_off;
  const T one = cmk(R(1), R(0));
  T dinv[KS];
#pragma unroll
  for (int q = 0; q < KS; ++q) {
    const int c = lane + 32 * q;
    dinv[q] = c < k ? pivot_rcp(S[s_pm[c] * ls + c]) : czero<T>();
  }
  for (int i = warp; i < k; i += NWARP) {
    T acc[KS];
    // row i of L11^-1, columns l < i
#pragma unroll
    for (int q = 0; q < KS; ++q) acc[q] = czero<T>();
    for (int m = i; m >= 1; --m) {
      const T ym = m == i ? one : shfl_c(pick_slot<T, KS>(acc, m >> 5), m & 31);
      const T* Lm = S + s_pm[m] * ls;
#pragma unroll
      for (int q = 0; q < KS; ++q) {
        const int l = lane + 32 * q;
        if (l < m) acc[q] = cfms(ym, Lm[l], acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < KS; ++q) {
      const int l = lane + 32 * q;
      if (l < i) Xg[(size_t)i * d.ldk + l] = acc[q];
    }
    // row i of U11^-1, columns c >= i
#pragma unroll
    for (int q = 0; q < KS; ++q) acc[q] = (lane + 32 * q == i) ? one : czero<T>();
    for (int l = i; l < k; ++l) {
      const int q = l >> 5;
      const T yl = shfl_c(cmul(pick_slot<T, KS>(acc, q), pick_slot<T, KS>(dinv, q)), l & 31);
      const T* Ul = S + s_pm[l] * ls;
#pragma unroll
      for (int qq = 0; qq < KS; ++qq) {
        const int c = lane + 32 * qq;
        if (c > l && c < k) acc[qq] = cfms(yl, Ul[c], acc[qq]);
      }
    }
#pragma unroll
    for (int q = 0; q < KS; ++q) {
      const int c = lane + 32 * q;
      if (c >= i && c < k) Xg[(size_t)i * d.ldk + c] = cmul(acc[q], dinv[q]);
    }
  }
  // the front but its pivot block (U12 in pivot order, L21, S), the permutation, the growth
  for (int r = warp; r < n; r += NWARP) {
    const T* Sr = S + (r < k ? s_pm[r] : r) * ls;
    T* Fr = F + (size_t)r * d.ld;
    for (int c = (r < k ? k : 0) + lane; c < n; c += 32) Fr[c] = Sr[c];
  }
  int* P = a.perm + (size_t)w * a.perm_stride + d.piv_off;
  for (int i = tid; i < k; i += THREADS) P[i] = s_pm[i];
  for (int o = 16; o > 0; o >>= 1) gmax = nanmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  if (lane == 0) s_red[warp] = gmax;
  __syncthreads();
  if (tid == 0) {
    R g = 0;
    for (int i = 0; i < NWARP; ++i) g = nanmax(g, s_red[i]);
    a.growth[(size_t)w * a.n_fronts + f] = (float)sqrt((double)g);
  }
}

// Warps and tile per size class (largest n of the class): NWARP warps, RI x RJ
// entries per thread, MINB CTAs per SM: complex64 classes up to n = 64 are held
// to 64 registers (twice the resident warps of an unbounded build, without
// spilling); complex128 keeps its registers.
template <typename T, int N> struct SmallCfg;
template <typename T> struct SmallCfg<T, 32> {
  static constexpr int kThreads = 64;
  static auto kernel() { return lu_small_kernel<T, 2, 1, 16, sizeof(T) == 8 ? 16 : 8>; }
};
template <typename T> struct SmallCfg<T, 48> {
  static constexpr int kThreads = 128;
  static auto kernel() { return lu_small_kernel<T, 4, 2, 12, sizeof(T) == 8 ? 8 : 4>; }
};
template <typename T> struct SmallCfg<T, 64> {
  static constexpr int kThreads = 256;
  static auto kernel() { return lu_small_kernel<T, 8, 2, 8, sizeof(T) == 8 ? 4 : 2>; }
};
template <typename T> struct SmallCfg<T, 96> {
  static constexpr int kThreads = 256;
  static auto kernel() { return lu_small_kernel<T, 8, 3, 12, 2>; }
};

// ---------------------------------------------------------------------------
// Symmetric form (complex-symmetric LDL^T).  M = D A with D = diag(s_x s_y) is
// complex symmetric (discrete reciprocity), so in the plan's elimination order
// every front of M factors as F = L diag(d) L^T with no pivoting: L11 unit
// lower, L21 = F21 L11^-T diag(d)^-1, update matrix S = F22 - L21 diag(d) L21^T.
// Only lower triangles are formed, updated and stored: the fronts hold L21 and
// the lower triangle of S (which the parent reads symmetrically), the inverse
// store holds L11^-1 strictly below the diagonal and 1 / d on it, and the
// permutation is the identity.  A solve of A x = b is then
//     x = L^-T diag(d)^-1 L^-1 D b   (transpose: A^T x = b gives x = D L^-T diag(d)^-1 L^-1 b),
// the L and L^T sweeps of the LU path with D and 1 / d applied in between.
// Small fronts: one CTA per front in shared memory, as lu_small_kernel.  Per
// pivot j, each row r > j takes l_r = F[r][j] / d_j and updates its entries
// j < c <= r by F[r][c] -= l_r F[c][j]; column j is read from a contiguous copy
// (written, double-buffered, by whoever updates column j of each row in the
// step before), and is scaled to l in place in the next step, when nothing
// reads it any more.  One barrier per pivot.
// ---------------------------------------------------------------------------

template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS)
ldl_small_kernel(FactorLaunch a, const int* __restrict__ flist) {
  using R = typename RealOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);
  __shared__ T colj[2][kSmallMaxK + 128];        // column j of the current step, contiguous
  __shared__ R s_red[THREADS / 32];
  const int w = blockIdx.y + a.w0;
  const int f = flist[blockIdx.x];
  const FrontDesc d = a.P.fronts[f];
  const int n = d.n, k = d.k;
  T* F = reinterpret_cast<T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = THREADS / 32;
  const int* idx = a.P.idx + d.idx_off;
  // assemble the lower triangle: children's update matrices (read symmetrically)
  // plus D times the original entries of column <= row (the mirrored ones are
  // the same numbers of M)
  {
    const T* st = reinterpret_cast<const T*>(a.store) + (size_t)w * a.store_stride;
    FrontDesc c0, c1;
    const int nc = d.nchild;
    if (nc > 0) c0 = a.P.fronts[a.P.children[d.child0]];
    if (nc > 1) c1 = a.P.fronts[a.P.children[d.child0 + 1]];
    for (int r = warp; r < n; r += NW) {
      const int ia = nc > 0 ? a.P.inv[c0.inv_off + r] : -1;
      const int ib = nc > 1 ? a.P.inv[c1.inv_off + r] : -1;
      for (int c = lane; c <= r; c += 32) {
        T v = czero<T>();
        if (ia >= 0) { const int i0 = a.P.inv[c0.inv_off + c]; if (i0 >= 0) v = cadd(v, child_sym(st, c0, ia, i0)); }
        if (ib >= 0) { const int i1 = a.P.inv[c1.inv_off + c]; if (i1 >= 0) v = cadd(v, child_sym(st, c1, ib, i1)); }
        S[r * n + c] = v;
      }
      __syncwarp();
      const int e0 = a.P.orig_ptr[d.orig_off + r], e1 = a.P.orig_ptr[d.orig_off + r + 1];
      const double2 Dr = sym_scale(a.C, w, idx[r]);
      for (int e = e0 + lane; e < e1; e += 32) {
        const int b = a.P.orig_col[e];
        if (b <= r) S[r * n + b] = cadd(S[r * n + b], cfrom<T>(cmul(Dr, stencil_entry(a.C, w, a.P.orig_code[e]))));
      }
    }
  }
  __syncthreads();
  for (int r = tid; r < n; r += THREADS) colj[0][r] = S[r * n];
  __syncthreads();
  R gmax = 0;
  T inv_prev = czero<T>();
  for (int j = 0; j < k; ++j) {
    const T* cj = colj[j & 1];
    T* cn = colj[(j + 1) & 1];
    const T p = cj[j];
    const T inv = crcp(p);
    if (tid == 0 && p.x == 0 && p.y == 0) gmax = INFINITY;
    for (int r = j + warp; r < n; r += NW) {
      // column j - 1 of this row is no longer read: scale it to the multiplier
      if (j > 0 && r > j - 1 && lane == 0) {
        const T l = cmul(S[r * n + j - 1], inv_prev);
        S[r * n + j - 1] = l;
        gmax = nanmax(gmax, cabs2(l));
      }
      if (r == j) continue;
      const T l = cmul(cj[r], inv);
      for (int c = j + 1 + lane; c <= r; c += 32) {
        const T v = cfms(l, cj[c], S[r * n + c]);
        S[r * n + c] = v;
        if (c == j + 1) cn[r] = v;
      }
    }
    inv_prev = inv;
    __syncthreads();
  }
  // the last pivot column
  if (k > 0)
    for (int r = k + tid; r < n; r += THREADS) {
      const T l = cmul(S[r * n + k - 1], inv_prev);
      S[r * n + k - 1] = l;
      gmax = nanmax(gmax, cabs2(l));
    }
  __syncthreads();
  // L11^-1 rows (as in lu_small_kernel) and 1 / d on the diagonal of the inverse store
  T* Xg = reinterpret_cast<T*>(a.istore) + (size_t)w * a.istore_stride + d.iv_off;
  const T one = cmk(R(1), R(0));
  for (int i = warp; i < k; i += NW) {
    T acc[kSmallSlots];
#pragma unroll
    for (int q = 0; q < kSmallSlots; ++q) acc[q] = czero<T>();
    for (int m = i; m >= 1; --m) {
      const T ym = m == i ? one : shfl_c(pick_slot(acc, m >> 5), m & 31);
#pragma unroll
      for (int q = 0; q < kSmallSlots; ++q) {
        const int l = lane + 32 * q;
        if (l < m) acc[q] = cfms(ym, S[m * n + l], acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < kSmallSlots; ++q) {
      const int l = lane + 32 * q;
      if (l < i) Xg[(size_t)i * d.ldk + l] = acc[q];
    }
    if (lane == 0) Xg[(size_t)i * d.ldk + i] = crcp(S[i * n + i]);
  }
  // rows below the pivots: L21 and the lower triangle of S
  for (int e = tid; e < (n - k) * n; e += THREADS) {
    const int r = k + e / n, c = e - (r - k) * n;
    if (c <= r) F[(size_t)r * d.ld + c] = S[r * n + c];
  }
  int* P = a.perm + (size_t)w * a.perm_stride + d.piv_off;
  for (int i = tid; i < k; i += THREADS) P[i] = i;
  for (int o = 16; o > 0; o >>= 1) gmax = nanmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  if (lane == 0) s_red[warp] = gmax;
  __syncthreads();
  if (tid == 0) {
    R g = 0;
    for (int i = 0; i < NW; ++i) g = nanmax(g, s_red[i]);
    a.growth[(size_t)w * a.n_fronts + f] = (float)sqrt((double)g);
  }
}

// ---------------------------------------------------------------------------
// Large fronts, blocked right-looking LU.  One panel step at column j0:
//   panel: factor columns [j0, j0+nb) over rows [j0, n) (one CTA per front),
//   trsm:  U rows [j0, j0+nb) of columns [j0+nb, n) (one CTA per 128 columns),
//   gemm:  trailing update of [j0+nb, n)^2 (one CTA per 64 x 64 tile).
// ---------------------------------------------------------------------------
constexpr int kPanelThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kPanelThreads)
lu_panel_kernel(FactorLaunch a, const int* __restrict__ flist, int j0, int nbmax) {
  using R = typename RealOf<T>::type;
  __shared__ R s_v[kPanelThreads / 32];
  __shared__ int s_i[kPanelThreads / 32];
  __shared__ int s_piv;
  const int w = blockIdx.y + a.w0;
  const int f = flist[blockIdx.x];
  const FrontDesc d = a.P.fronts[f];
  if (j0 >= d.k) return;
  const int nb = min(nbmax, d.k - j0);
  const int n = d.n, k = d.k, ld = d.ld;
  T* F = reinterpret_cast<T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  int* P = a.perm + (size_t)w * a.perm_stride + d.piv_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (j0 == 0) {
    for (int i = tid; i < k; i += blockDim.x) P[i] = i;
    __syncthreads();
  }
  R gmax = 0;
  for (int j = j0; j < j0 + nb; ++j) {
    R best = -1;
    int bi = j;
    for (int r = j + tid; r < k; r += blockDim.x) {
      const R v = cabs2(F[(size_t)r * ld + j]);
      if (v > best) { best = v; bi = r; }
    }
    warp_argmax(best, bi);
    if (lane == 0) { s_v[warp] = best; s_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      R bv = s_v[0];
      int bidx = s_i[0];
      for (int i = 1; i < kPanelThreads / 32; ++i)
        if (s_v[i] > bv || (s_v[i] == bv && s_i[i] < bidx)) { bv = s_v[i]; bidx = s_i[i]; }
      s_piv = bidx;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != j) {
      for (int c = tid; c < n; c += blockDim.x) {
        const T x = F[(size_t)j * ld + c];
        F[(size_t)j * ld + c] = F[(size_t)piv * ld + c];
        F[(size_t)piv * ld + c] = x;
      }
      if (tid == 0) { const int x = P[j]; P[j] = P[piv]; P[piv] = x; }
    }
    __syncthreads();
    const T pv = F[(size_t)j * ld + j];
    const T inv = crcp(pv);
    if (pv.x == 0 && pv.y == 0) gmax = INFINITY;
    for (int r = j + 1 + tid; r < k; r += blockDim.x) {
      const T l = cmul(F[(size_t)r * ld + j], inv);
      F[(size_t)r * ld + j] = l;
      gmax = nanmax(gmax, cabs2(l));
    }
    __syncthreads();
    const int cols = j0 + nb - (j + 1);
    if (cols > 0) {
      // rank-1 update of the panel columns (j, j0+nb), pivot rows only: thread -> (row, col)
      for (long long e = tid; e < (long long)(k - j - 1) * cols; e += blockDim.x) {
        const int r = j + 1 + (int)(e / cols), c = j + 1 + (int)(e % cols);
        F[(size_t)r * ld + c] = cfms(F[(size_t)r * ld + j], F[(size_t)j * ld + c], F[(size_t)r * ld + c]);
      }
    }
    __syncthreads();
  }
  if (tid == 0) a.swp[((size_t)blockIdx.y * a.swp_stride + blockIdx.x) * kSwpInts] = 0;  // swaps done here
  for (int o = 16; o > 0; o >>= 1) gmax = nanmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  if (lane == 0) s_v[warp] = gmax;
  __syncthreads();
  if (tid == 0) {
    R g = 0;
    for (int i = 0; i < kPanelThreads / 32; ++i) g = nanmax(g, s_v[i]);
    float* gp = a.growth + (size_t)w * a.n_fronts + f;
    const float gv = (float)sqrt((double)g);
    *gp = (j0 == 0) ? gv : nanmax(*gp, gv);
  }
}

constexpr int kTrsmCols = 128;
constexpr int kMaxNb = 32;

// Panel of the k - j0 pivot-candidate rows staged in shared memory (one CTA
// per front).  Per column: block argmax, swap of the two panel rows, then one
// warp per row scales and updates the row (lane = column).  The row swaps are
// applied to the columns outside the panel afterwards, in order.
constexpr int kPanelSmemThreads = 512;
constexpr int kPanelSmemBytes = 200 * 1024;

template <typename T>
__global__ void __launch_bounds__(kPanelSmemThreads)
lu_panel_smem_kernel(FactorLaunch a, const int* __restrict__ flist, int j0, int nbmax) {
  using R = typename RealOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ps = reinterpret_cast<T*>(smem_raw);
  constexpr int NW = kPanelSmemThreads / 32;
  __shared__ R s_v[NW];
  __shared__ int s_i[NW];
  __shared__ int s_swap[kMaxNb];
  const int w = blockIdx.y + a.w0;
  const int f = flist[blockIdx.x];
  const FrontDesc d = a.P.fronts[f];
  if (j0 >= d.k) return;
  const int nb = min(nbmax, d.k - j0);
  const int k = d.k, ld = d.ld;
  const int R_ = k - j0, ldp = nb + 1;
  T* F = reinterpret_cast<T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  int* P = a.perm + (size_t)w * a.perm_stride + d.piv_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (j0 == 0)
    for (int i = tid; i < k; i += kPanelSmemThreads) P[i] = i;
  for (int e = tid; e < R_ * nb; e += kPanelSmemThreads) {
    const int r = e / nb, c = e - r * nb;
    Ps[r * ldp + c] = F[(size_t)(j0 + r) * ld + j0 + c];
  }
  __syncthreads();
  R gmax = 0;
  {  // argmax of the first panel column
    R best = -1;
    int bi = 0;
    for (int r = tid; r < R_; r += kPanelSmemThreads) {
      const R v = cabs2(Ps[r * ldp]);
      if (v > best) { best = v; bi = r; }
    }
    warp_argmax(best, bi);
    if (lane == 0) { s_v[warp] = best; s_i[warp] = bi; }
    __syncthreads();
  }
  constexpr int U = 4;                    // rows in flight per warp
  for (int jj = 0; jj < nb; ++jj) {
    // pivot of column jj from the per-warp partial maxima (ties to the smaller row)
    R bv = s_v[0];
    int piv = s_i[0];
    for (int i = 1; i < NW; ++i)
      if (s_v[i] > bv || (s_v[i] == bv && s_i[i] < piv)) { bv = s_v[i]; piv = s_i[i]; }
    if (piv < jj) piv = jj;                // every candidate row was empty
    if (piv != jj && tid < nb) {
      const T x = Ps[jj * ldp + tid];
      Ps[jj * ldp + tid] = Ps[piv * ldp + tid];
      Ps[piv * ldp + tid] = x;
    }
    if (tid == 0) s_swap[jj] = piv;
    __syncthreads();
    const T pv = Ps[jj * ldp + jj];
    const T inv = crcp(pv);
    if (pv.x == 0 && pv.y == 0) gmax = INFINITY;
    const T urow = lane < nb ? Ps[jj * ldp + lane] : czero<T>();
    const int nx = jj + 1;                 // next column: its argmax is gathered on the way
    R best = -1;
    int bi = nx;
    for (int r = jj + 1 + warp; r < R_; r += U * NW) {
      T l[U], cur[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int ru = r + u * NW;
        const bool ok = ru < R_;
        l[u] = ok ? cmul(Ps[ru * ldp + jj], inv) : czero<T>();
        cur[u] = (ok && lane < nb) ? Ps[ru * ldp + lane] : czero<T>();
      }
      __syncwarp();                        // every lane has read its entries before any lane writes
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int ru = r + u * NW;
        if (ru < R_) {                     // warp-uniform
          const T nv = lane == jj ? l[u] : (lane > jj ? cfms(l[u], urow, cur[u]) : cur[u]);
          if (lane < nb) Ps[ru * ldp + lane] = nv;
          const R v = cabs2(nv);
          if (lane == nx && v > best) { best = v; bi = ru; }
          gmax = nanmax(gmax, cabs2(l[u]));
        }
      }
    }
    if (nx < nb) {
      // lane nx holds this warp's partial maximum of the next column (rows in
      // increasing order per warp, so ties keep the smaller row)
      const R wb = __shfl_sync(0xffffffffu, best, nx);
      const int wi = __shfl_sync(0xffffffffu, bi, nx);
      if (lane == 0) { s_v[warp] = wb; s_i[warp] = wi; }
    }
    __syncthreads();
  }
  for (int e = tid; e < R_ * nb; e += kPanelSmemThreads) {
    const int r = e / nb, c = e - r * nb;
    F[(size_t)(j0 + r) * ld + j0 + c] = Ps[r * ldp + c];
  }
  __syncthreads();
  // Net effect of the panel's row swaps on the columns outside the panel:
  // row j0 + dst receives the old row j0 + src, for at most 2 nb pairs.  The
  // shared panel buffer is reused as the position map; the swaps themselves are
  // applied by the column-block CTAs of the next launch (lu_l21_swap_kernel).
  int* map = reinterpret_cast<int*>(smem_raw);
  for (int r = tid; r < R_; r += kPanelSmemThreads) map[r] = r;
  __syncthreads();
  if (tid == 0) {
    for (int jj = 0; jj < nb; ++jj) {
      const int piv = s_swap[jj];
      if (piv != jj) {
        const int x = map[jj]; map[jj] = map[piv]; map[piv] = x;
        const int y = P[j0 + jj]; P[j0 + jj] = P[j0 + piv]; P[j0 + piv] = y;
      }
    }
    int* out = a.swp + ((size_t)blockIdx.y * a.swp_stride + blockIdx.x) * kSwpInts;
    int cnt = 0;
    for (int t = 0; t < 2 * nb; ++t) {
      const int p = t < nb ? t : s_swap[t - nb];
      if (t >= nb) {
        if (p < nb) continue;                           // already listed
        bool dup = false;
        for (int q = 0; q < t - nb; ++q) dup |= (s_swap[q] == p);
        if (dup) continue;
      }
      if (map[p] != p) { out[1 + 2 * cnt] = p; out[2 + 2 * cnt] = map[p]; ++cnt; }
    }
    out[0] = cnt;
  }
  for (int o = 16; o > 0; o >>= 1) gmax = nanmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  if (lane == 0) s_v[warp] = gmax;
  __syncthreads();
  if (tid == 0) {
    R g = 0;
    for (int i = 0; i < NW; ++i) g = nanmax(g, s_v[i]);
    float* gp = a.growth + (size_t)w * a.n_fronts + f;
    const float gv = (float)sqrt((double)g);
    *gp = (j0 == 0) ? gv : nanmax(*gp, gv);
  }
}

// Panel with the pivot-candidate rows held in registers: warp w owns rows
// w, w + 16, w + 32, ... (RPW of them), lane c holds column c.  Per column: the
// pivot row (and the row it displaces) go through shared memory once, every
// warp updates its rows in registers with the pivot row broadcast, and lane
// jj+1 collects the next column's argmax on the way (2 barriers per column).
constexpr int kRegWarps = 16;

template <typename T, int N>
__device__ __forceinline__ T pick(const T (&v)[N], int s) {
  T r = v[0];
#pragma unroll
  for (int i = 1; i < N; ++i)
    if (i == s) r = v[i];
  return r;
}
template <typename T, int N>
__device__ __forceinline__ void put(T (&v)[N], int s, T x) {
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i == s) v[i] = x;
}

template <typename T, int RPW>
__global__ void __launch_bounds__(kRegWarps * 32)
lu_panel_reg_kernel(FactorLaunch a, const int* __restrict__ flist, int j0, int nbmax) {
  using R = typename RealOf<T>::type;
  constexpr int NW = kRegWarps;
  __shared__ T prow[32];
  __shared__ T srow[32];
  __shared__ R s_v[NW];
  __shared__ int s_i[NW];
  __shared__ int s_swap[kMaxNb];
  __shared__ int map[NW * RPW];
  const int w = blockIdx.y + a.w0;
  const int f = flist[blockIdx.x];
  const FrontDesc d = a.P.fronts[f];
  if (j0 >= d.k) return;
  const int nb = min(nbmax, d.k - j0);
  const int k = d.k, ld = d.ld;
  const int R_ = k - j0;                       // <= NW * RPW (checked by the launcher)
  T* F = reinterpret_cast<T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  int* P = a.perm + (size_t)w * a.perm_stride + d.piv_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (j0 == 0)
    for (int i = tid; i < k; i += NW * 32) P[i] = i;
  T row[RPW];
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = warp + i * NW;
    row[i] = (r < R_ && lane < nb) ? F[(size_t)(j0 + r) * ld + j0 + lane] : czero<T>();
  }
  {  // argmax of column 0 (held by lane 0)
    R best = -1;
    int bi = 0;
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
      const int r = warp + i * NW;
      if (r < R_) {
        const R v = cabs2(row[i]);
        if (v > best) { best = v; bi = r; }
      }
    }
    best = __shfl_sync(0xffffffffu, best, 0);
    bi = __shfl_sync(0xffffffffu, bi, 0);
    if (lane == 0) { s_v[warp] = best; s_i[warp] = bi; }
  }
  __syncthreads();
  R gmax = 0;
  for (int jj = 0; jj < nb; ++jj) {
    R bv = s_v[0];
    int piv = s_i[0];
#pragma unroll
    for (int i = 1; i < NW; ++i)
      if (s_v[i] > bv || (s_v[i] == bv && s_i[i] < piv)) { bv = s_v[i]; piv = s_i[i]; }
    if (piv < jj) piv = jj;
    const int ow_j = jj % NW, sl_j = jj / NW, ow_p = piv % NW, sl_p = piv / NW;
    if (warp == ow_p) prow[lane] = pick(row, sl_p);
    if (piv != jj && warp == ow_j) srow[lane] = pick(row, sl_j);
    if (tid == 0) s_swap[jj] = piv;
    __syncthreads();
    if (piv != jj) {
      if (warp == ow_j) put(row, sl_j, prow[lane]);
      if (warp == ow_p) put(row, sl_p, srow[lane]);
    }
    const T ur = prow[lane];
    const T pv = prow[jj];
    const T inv = crcp(pv);
    if (pv.x == 0 && pv.y == 0) gmax = INFINITY;
    const int nx = jj + 1;
    R best = -1;
    int bi = nx;
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
      const int r = warp + i * NW;
      if (r > jj && r < R_) {                   // warp-uniform
        const T l = cmul(shfl_c(row[i], jj), inv);
        const T upd = cfms(l, ur, row[i]);
        row[i] = lane == jj ? l : (lane > jj ? upd : row[i]);
        gmax = nanmax(gmax, cabs2(l));
        const R v = cabs2(row[i]);
        if (lane == nx && v > best) { best = v; bi = r; }
      }
    }
    if (nx < nb) {
      best = __shfl_sync(0xffffffffu, best, nx);
      bi = __shfl_sync(0xffffffffu, bi, nx);
      if (lane == 0) { s_v[warp] = best; s_i[warp] = bi; }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = warp + i * NW;
    if (r < R_ && lane < nb) F[(size_t)(j0 + r) * ld + j0 + lane] = row[i];
  }
  // net row permutation of the panel for the columns outside it (see lu_panel_smem_kernel)
  for (int r = tid; r < R_; r += NW * 32) map[r] = r;
  __syncthreads();
  if (tid == 0) {
    for (int jj = 0; jj < nb; ++jj) {
      const int piv = s_swap[jj];
      if (piv != jj) {
        const int x = map[jj]; map[jj] = map[piv]; map[piv] = x;
        const int y = P[j0 + jj]; P[j0 + jj] = P[j0 + piv]; P[j0 + piv] = y;
      }
    }
    int* out = a.swp + ((size_t)blockIdx.y * a.swp_stride + blockIdx.x) * kSwpInts;
    int cnt = 0;
    for (int t = 0; t < 2 * nb; ++t) {
      const int p = t < nb ? t : s_swap[t - nb];
      if (t >= nb) {
        if (p < nb) continue;
        bool dup = false;
        for (int q = 0; q < t - nb; ++q) dup |= (s_swap[q] == p);
        if (dup) continue;
      }
      if (map[p] != p) { out[1 + 2 * cnt] = p; out[2 + 2 * cnt] = map[p]; ++cnt; }
    }
    out[0] = cnt;
  }
  for (int o = 16; o > 0; o >>= 1) gmax = nanmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  if (lane == 0) s_v[warp] = gmax;
  __syncthreads();
  if (tid == 0) {
    R g = 0;
    for (int i = 0; i < NW; ++i) g = nanmax(g, s_v[i]);
    float* gp = a.growth + (size_t)w * a.n_fronts + f;
    const float gv = (float)sqrt((double)g);
    *gp = (j0 == 0) ? gv : nanmax(*gp, gv);
  }
}

// ---------------------------------------------------------------------------
// Block-local pivoting: one launch per panel step does everything that depends
// only on the 32 x 32 diagonal block B = F[J, J], J = [j0, j0 + nb):
//   every CTA LU-factors B itself (warps 0-3, rows in registers, pivot rows
//   chosen inside B; deterministic, so every CTA gets the same bits) while
//   warps 4-7 stage the CTA's operand, then does one role:
//     role D (block 0): the row permutation of J into perm, L_JJ^-1 and U_JJ^-1
//                       into the diagonal block of the inverse store (L_JJ^-1
//                       strictly below the diagonal, U_JJ^-1 on and above it),
//                       growth of its multipliers;
//     role L: rows r >= j0 + nb, L[r, J] U_JJ = F[r, J]          (64 rows / CTA);
//     role U: columns c >= j0 + nb, L_JJ U[J, c] = (P F)[J, c]   (64 columns / CTA);
//     role P: columns c < j0, F[J, c] <- (P F)[J, c]             (64 columns / CTA);
//   L and U by one-thread-per-row/column substitution against the factored B.
// The factored diagonal block is not stored back into F (nothing reads it there:
// the sweeps and lu_inv_fold use the inverse store).  Roles touch disjoint
// entries of F and read B only, so the CTAs are independent.
// ---------------------------------------------------------------------------
constexpr int kStepRows = 256;   // roles L and U: rows / columns per CTA, one per thread
constexpr int kStepCols = 64;    // role P: columns per CTA
static_assert(kStepRows == 1 << 8 && kStepCols == 1 << 6, "the staging loops shift by 8 and 6");

// LU of the nb x nb block at (j0, j0) with row pivoting inside the block, by
// warps 0-3 (lane = row; warp w holds columns 8w..8w+7 in registers).  No rows
// are swapped: at step p the warp owning column p picks the unused lane r with
// the largest |a_p| (one redux over packed keys: |a_p|^2 in the high bits,
// 31 - lane in the low 5, so ties go to the lower lane) and publishes r and
// every lane's multiplier through shared memory (double-buffered, one 128-thread
// named barrier per step); each warp then updates its own columns.  On return
// (after the caller's __syncthreads) LU[p] holds row p of L\U in pivot order,
// src[p] the block row it came from, dinv[p] = 1 / U[p][p].  Returns this
// lane's largest |multiplier|^2 (NaN -> inf).
template <typename T>
__device__ __forceinline__ typename RealOf<T>::type diag_lu_4warps(const T* __restrict__ F, int ld, int j0, int nb,
                                                                   T (*LU)[kMaxNb + 1], int* src, T* dinv,
                                                                   T (*s_l)[32], int* s_r, bool sym = false) {
  using R = typename RealOf<T>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T one = cmk(R(1), R(0));
  T a[8];
  // symmetric form: only the block's lower triangle is current (read it mirrored),
  // and the pivots are the diagonal in order (no pivoting)
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int j = 8 * warp + c;
    const int ri = (sym && j > lane) ? j : lane, ci = (sym && j > lane) ? lane : j;
    a[c] = (lane < nb && j < nb) ? F[(size_t)(j0 + ri) * ld + j0 + ci] : (lane == j ? one : czero<T>());
  }
  bool used = false;
  int myp = lane;                 // padding lanes (>= nb) keep their own position
  R g = 0;
  for (int p = 0; p < nb; ++p) {
    const int buf = p & 1, cp = p & 7;
    if ((p >> 3) == warp) {
      T ap = a[0];
#pragma unroll
      for (int c = 1; c < 8; ++c)
        if (c == cp) ap = a[c];
      const float v = (float)cabs2(ap);
      const T myinv = pivot_rcp(ap);    // every lane's candidate, formed beside the redux
      unsigned key = used ? 0u : ((__float_as_uint(v) & ~31u) | (unsigned)(31 - lane));
      if (!used && !(v == v)) key = 0xffffffe0u | (unsigned)(31 - lane);   // NaN wins
      if (sym) key = lane == p ? (0xffffffe0u | (unsigned)(31 - lane)) : 0u;   // the diagonal, in order
      const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
      const int r = 31 - (int)(kmax & 31u);
      const T inv = shfl_c(myinv, r);
      const bool elim = !used && lane != r;
      const T l = elim ? cmul(ap, inv) : czero<T>();
      s_l[buf][lane] = l;
      if (lane == 0) { s_r[buf] = r; src[p] = r; dinv[p] = inv; }
      if (elim) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c == cp) a[c] = l;        // the multiplier is stored in column p
      }
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    const int r = s_r[buf];
    const T l = s_l[buf][lane];
    if (lane == r) { used = true; myp = p; }
    {
      const R a2 = cabs2(l);
      g = (a2 == a2) ? (a2 > g ? a2 : g) : R(INFINITY);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int j = 8 * warp + c;
      const T u = shfl_c(a[c], r);
      if (j > p) a[c] = cfms(l, u, a[c]);   // l = 0 on the pivot and on used lanes
    }
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) LU[myp][8 * warp + c] = a[c];
  if (lane >= nb && warp == 0) { src[lane] = lane; dinv[lane] = one; }   // padding rows stay in place
  return g;
}

// phase 0: every CTA factors the diagonal block itself (one wave or less);
// phase 1: only the role-0 CTA of each front, which also posts the block's
//          factors (rows of L\U in pivot order, 1 / U_pp, source rows) to the
//          front's scratch slot;
// phase 2: the other roles, which load those factors instead (many waves).
template <typename T>
__global__ void __launch_bounds__(256)
lu_step_local_kernel(FactorLaunch a, const int* __restrict__ flist, int j0, int nl, int nu, int phase) {
  using R = typename RealOf<T>::type;
  using Blk = T[kMaxNb + 1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Blk* LU = reinterpret_cast<Blk*>(smem_raw);                  // [32][33]
  T* dinv = reinterpret_cast<T*>(LU + kMaxNb);                 // [32]
  T (*s_l)[32] = reinterpret_cast<T (*)[32]>(dinv + kMaxNb);   // [2][32] multipliers of a step
  Blk* Ws = reinterpret_cast<Blk*>(s_l + 2);   // [kStepRows][33]: role L rows x J; roles U, P: [c][p];
                                               // role D its first 64 rows (a phase-1 launch has only those)
  __shared__ int src[kMaxNb];
  __shared__ int s_r[2];
  __shared__ R s_g[8];
  const int w = blockIdx.z + a.w0;
  const int f = flist[blockIdx.y];
  const FrontDesc d = a.P.fronts[f];
  if (j0 >= d.k) return;
  // L rows and U columns up to n; a front whose off-diagonal blocks come from the
  // tensor cores stops at its pivot block
  const int nb = min(kMaxNb, d.k - j0), n = (a.pivonly && a.pivonly[f]) ? d.k : d.n, ld = d.ld;
  const int bx = blockIdx.x + (phase == 2 ? 1 : 0);
  const size_t slot = (size_t)blockIdx.z * a.swp_stride + blockIdx.y;
  T* blk = reinterpret_cast<T*>(a.dblk) + slot * kDiagBlkElems;
  int* bsrc = a.swp + slot * kSwpInts;
  // role and range; CTAs whose range is empty for this front leave before any work
  int role, lo = 0;
  if (bx == 0) {
    role = 0;
  } else if (bx <= nl) {
    role = 1; lo = j0 + nb + (bx - 1) * kStepRows;
    if (lo >= n) return;
  } else if (bx <= nl + nu) {
    role = 2; lo = j0 + nb + (bx - 1 - nl) * kStepRows;
    if (lo >= n) return;
  } else {
    role = 3; lo = (bx - 1 - nl - nu) * kStepCols;
    if (lo >= j0) return;
  }
  T* F = reinterpret_cast<T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  R g = 0;
  if (warp < 4) {
    if (phase == 2) {
      for (int e = tid; e < kMaxNb * kMaxNb; e += 128) LU[e >> 5][e & 31] = blk[e];
      if (tid < kMaxNb) {
        dinv[tid] = blk[kMaxNb * kMaxNb + tid];
        src[tid] = bsrc[tid];
      }
    } else {
      g = diag_lu_4warps<T>(F, ld, j0, nb, LU, src, dinv, s_l, s_r, a.sym != 0);
    }
  } else if (role == 1) {
    // meanwhile warps 4-7 stage rows [lo, lo + kStepRows) of the block columns
    for (int e = tid - 128; e < kStepRows * kMaxNb; e += 128) {
      const int rr = e >> 5, l = e & 31, r = lo + rr;
      Ws[rr][l] = (r < n && l < nb) ? F[(size_t)r * ld + j0 + l] : czero<T>();
    }
  } else if (role >= 2) {
    // ... or the block rows (not yet permuted) over columns [lo, lo + width)
    const int hi = role == 2 ? n : j0;
    const int lw = role == 2 ? 8 : 6;   // log2 of the width: kStepRows (role U) or kStepCols (role P)
    for (int e = tid - 128; e < (kMaxNb << lw); e += 128) {
      const int p = e >> lw, cc = e & ((1 << lw) - 1), c = lo + cc;
      Ws[cc][p] = (c < hi && p < nb) ? F[(size_t)(j0 + p) * ld + c] : czero<T>();
    }
  }
  __syncthreads();
  if (phase == 1) {
    for (int e = tid; e < kMaxNb * kMaxNb; e += blockDim.x) blk[e] = LU[e >> 5][e & 31];
    if (tid < kMaxNb) {
      blk[kMaxNb * kMaxNb + tid] = dinv[tid];
      bsrc[tid] = src[tid];
    }
  }
  // Role D: warp 0 (lane = column c) solves L_JJ x = e_c, warp 1
  // (lane = row r) solves x U_JJ = e_r, with the same substitution code as roles
  // U and L; the columns of L_JJ^-1 and rows of U_JJ^-1 meet in the staging tile.
  const T one = cmk(R(1), R(0));
  const bool sub_up = (role == 1 && tid < kStepRows) || (role == 0 && warp == 1);
  const bool sub_lo = (role == 2 && tid < kStepRows) || (role == 0 && warp == 0);
  if (role == 0 && tid < nb) a.perm[(size_t)w * a.perm_stride + d.piv_off + j0 + tid] = j0 + src[tid];
  if (sub_up) {
    // x U_JJ = b: one thread per row, right-looking substitution
    T x[kMaxNb];
#pragma unroll
    for (int j = 0; j < kMaxNb; ++j) x[j] = role == 1 ? Ws[tid][j] : (j == lane ? one : czero<T>());
#pragma unroll
    for (int j = 0; j < kMaxNb; ++j) {
      x[j] = cmul(x[j], dinv[j]);
#pragma unroll
      for (int jj = j + 1; jj < kMaxNb; ++jj) x[jj] = cfms(x[j], LU[j][jj], x[jj]);
    }
    if (role == 1) {
      // L[r, J] = F[r, J] U_JJ^-1
      const int r = lo + tid;
      if (r < n) {
#pragma unroll
        for (int j = 0; j < kMaxNb; ++j)
          if (j < nb) {
            F[(size_t)r * ld + j0 + j] = x[j];
            const R a2 = cabs2(x[j]);
            g = (a2 == a2) ? (a2 > g ? a2 : g) : R(INFINITY);
          }
      }
    } else {
#pragma unroll
      for (int j = 0; j < kMaxNb; ++j) Ws[kMaxNb + lane][j] = x[j];   // row lane of U_JJ^-1
    }
  } else if (sub_lo) {
    // L_JJ x = b: one thread per column, unit-lower substitution
    T x[kMaxNb];
#pragma unroll
    for (int i = 0; i < kMaxNb; ++i) x[i] = role == 2 ? Ws[tid][src[i]] : (i == lane ? one : czero<T>());
#pragma unroll
    for (int i = 0; i < kMaxNb; ++i)
#pragma unroll
      for (int ii = i + 1; ii < kMaxNb; ++ii) x[ii] = cfms(LU[ii][i], x[i], x[ii]);
    if (role == 2) {
      // U[J, c] = L_JJ^-1 (P F)[J, c]
      const int c = lo + tid;
      if (c < n)
#pragma unroll
        for (int i = 0; i < kMaxNb; ++i)
          if (i < nb) F[(size_t)(j0 + i) * ld + c] = x[i];
    } else {
#pragma unroll
      for (int i = 0; i < kMaxNb; ++i) Ws[i][lane] = x[i];             // column lane of L_JJ^-1
    }
  } else if (role == 3) {
    // role P: (P F)[i][c] for the columns left of the block
    const int cc = tid & 63, ig = tid >> 6;
    const int c = lo + cc;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = ig + 4 * q;
      if (c < j0 && i < nb) F[(size_t)(j0 + i) * ld + c] = Ws[cc][src[i]];
    }
  }
  if (role == 0) {
    // the diagonal block of the inverse store: L_JJ^-1 strictly below the
    // diagonal, U_JJ^-1 on and above it
    T* X = reinterpret_cast<T*>(a.istore) + (size_t)w * a.istore_stride + d.iv_off;
    __syncthreads();
    for (int e = tid; e < nb * nb; e += blockDim.x) {
      const int i = e / nb, j = e - i * nb;
      X[(size_t)(j0 + i) * d.ldk + j0 + j] = i > j ? Ws[i][j] : Ws[kMaxNb + i][j];
    }
  }
  if (role <= 1) {
    for (int o = 16; o > 0; o >>= 1) g = nanmax(g, __shfl_xor_sync(0xffffffffu, g, o));
    if (lane == 0) s_g[warp] = g;
    __syncthreads();
    if (tid == 0) {
      R gg = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) gg = nanmax(gg, s_g[i]);
      float gv = (float)sqrt((double)gg);
      if (!(gv == gv)) gv = INFINITY;
      // max of non-negative floats is order independent as an int max
      atomicMax(reinterpret_cast<int*>(a.growth + (size_t)w * a.n_fronts + f), __float_as_int(gv));
    }
  }
}

// Triangular inverses of a factored large front, written to the inverse store
// (L11^-1 strictly below the diagonal, U11^-1 on and above it).  One CTA per
// 32-column block of one triangle; it walks its column block one 32-row block
// at a time: a product with the rows already inverted (read back from global
// memory), then a substitution inside the diagonal block by one warp (lane =
// column).  Different CTAs write disjoint entries.
template <typename T>
__global__ void __launch_bounds__(256)
lu_inv_kernel(FactorLaunch a, const int* __restrict__ flist, int nblk) {
  // two 32 x 33 tiles: (Ls, Xs) during the products, then (Acc, Dg) for the
  // diagonal block; every switch is separated by a barrier
  __shared__ T tile0[32][33];
  __shared__ T tile1[32][33];
  T (&Ls)[32][33] = tile0;
  T (&Acc)[32][33] = tile0;
  T (&Xs)[32][33] = tile1;
  T (&Dg)[32][33] = tile1;
  const int w = blockIdx.z + a.w0;
  const int f = flist[blockIdx.y];
  const FrontDesc d = a.P.fronts[f];
  const bool upper = (int)blockIdx.x >= nblk;
  const int cb = (upper ? (int)blockIdx.x - nblk : (int)blockIdx.x) * 32;
  const int k = d.k;
  if (cb >= k) return;
  const int ld = d.ld, ldk = d.ldk;
  const int cw = min(32, k - cb);
  const T* F = reinterpret_cast<const T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  T* X = reinterpret_cast<T*>(a.istore) + (size_t)w * a.istore_stride + d.iv_off;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c = cb + tx;
  const T one = cmk(typename RealOf<T>::type(1), typename RealOf<T>::type(0));
  if (!upper) {
    // X[r][c] = delta_rc - sum_{l in [c, r)} L[r][l] X[l][c], X[c][c] = 1, X[l][c] = 0 for l < c
    for (int rb = cb; rb < k; rb += 32) {
      const int rh = min(32, k - rb);
      T acc[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
      for (int l0 = cb; l0 < rb; l0 += 32) {      // rows already inverted, 32 at a time via shared memory
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
          const int i = e >> 5, j = e & 31;
          Ls[i][j] = (i < rh) ? F[(size_t)(rb + i) * ld + l0 + j] : czero<T>();
          const int l = l0 + i, cc = cb + j;
          Xs[i][j] = (j < cw) ? (l > cc ? X[(size_t)l * ldk + cc] : (l == cc ? one : czero<T>())) : czero<T>();
        }
        __syncthreads();
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
          const T xv = Xs[j][tx];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] = cfma(Ls[ty + 8 * q][j], xv, acc[q]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = ty + 8 * q;
        if (i < rh) Acc[i][tx] = csub(rb + i == c ? one : czero<T>(), acc[q]);
      }
      for (int e = threadIdx.x; e < rh * 32; e += 256) {
        const int i = e >> 5, j = e & 31;
        if (j < rh) Dg[i][j] = F[(size_t)(rb + i) * ld + rb + j];
      }
      __syncthreads();
      if (ty == 0 && tx < cw) {
        T xc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          if (i < rh) {
            T v = Acc[i][tx];
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < i) v = cfms(Dg[i][j], xc[j], v);
            xc[i] = v;
            if (rb + i > c) X[(size_t)(rb + i) * ldk + c] = v;
          }
        }
      }
      __syncthreads();
    }
  } else {
    // X[r][c] = (delta_rc - sum_{l in (r, c]} U[r][l] X[l][c]) / U[r][r] for r <= c
    for (int rb = cb; rb >= 0; rb -= 32) {
      const int rh = min(32, k - rb);
      T acc[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
      for (int l0 = rb + 32; l0 < cb + cw; l0 += 32) {   // rows below, already inverted (l <= c)
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
          const int i = e >> 5, j = e & 31;
          Ls[i][j] = (i < rh && l0 + j < k) ? F[(size_t)(rb + i) * ld + l0 + j] : czero<T>();
          const int l = l0 + i, cc = cb + j;
          Xs[i][j] = (j < cw && l < k && l <= cc) ? X[(size_t)l * ldk + cc] : czero<T>();
        }
        __syncthreads();
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
          const T xv = Xs[j][tx];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] = cfma(Ls[ty + 8 * q][j], xv, acc[q]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = ty + 8 * q;
        if (i < rh) Acc[i][tx] = csub(rb + i == c ? one : czero<T>(), acc[q]);
      }
      for (int e = threadIdx.x; e < rh * 32; e += 256) {
        const int i = e >> 5, j = e & 31;
        if (j < rh) Dg[i][j] = F[(size_t)(rb + i) * ld + rb + j];
      }
      __syncthreads();
      if (ty == 0 && tx < cw) {
        T xc[32];
#pragma unroll
        for (int i = 31; i >= 0; --i) {
          if (i < rh) {
            const int r = rb + i;
            T v = czero<T>();
            if (r <= c) {
              v = Acc[i][tx];
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j > i && j < rh && rb + j <= c) v = cfms(Dg[i][j], xc[j], v);
              v = cmul(v, crcp(Dg[i][i]));
              X[(size_t)r * ldk + c] = v;
            }
            xc[i] = v;
          }
        }
      }
      __syncthreads();
    }
  }
}

// dynamic shared memory of lu_step_local_kernel: LU, the 64 x 33 staging tile, 1/U[p][p],
// the multipliers of one step (double-buffered)
size_t step_local_smem(size_t es) {
  return ((size_t)(kMaxNb + kStepRows) * (kMaxNb + 1) + kMaxNb + 2 * 32) * es;
}
// a phase-1 launch (the diagonal block and role D only): the staging tile's first 64 rows
size_t step_diag_smem(size_t es) {
  return ((size_t)(kMaxNb + 2 * kMaxNb) * (kMaxNb + 1) + kMaxNb + 2 * 32) * es;
}

// Boundary rows of the panel: L21[:, j0:j0+nb] = A21[:, j0:j0+nb] U_jj^-1 (right
// triangular solve with the panel's upper block), 64 rows per CTA.
constexpr int kL21Rows = 64;

// CTAs with blockIdx.x >= nl21 instead apply the panel's net row permutation
// (pairs written by lu_panel_smem_kernel) to 32 columns outside the panel.
template <typename T>
__global__ void __launch_bounds__(256)
lu_l21_kernel(FactorLaunch a, const int* __restrict__ flist, int j0, int nbmax, int nl21, int below) {
  using R = typename RealOf<T>::type;
  __shared__ T Us[kMaxNb][kMaxNb + 1];
  __shared__ T Xs[kL21Rows][kMaxNb + 1];
  __shared__ R s_g[8];
  const int w = blockIdx.z + a.w0;
  const int f = flist[blockIdx.y];
  const FrontDesc d = a.P.fronts[f];
  if (j0 >= d.k) return;
  const int nb = min(nbmax, d.k - j0);
  if ((int)blockIdx.x >= nl21) {
    // ---- row swaps on columns [c0, c0 + 32) of the non-panel columns -------
    const int* pr = a.swp + ((size_t)blockIdx.z * a.swp_stride + blockIdx.y) * kSwpInts;
    const int cnt = pr[0];
    const int cb = (blockIdx.x - nl21) * 32;
    if (cnt == 0 || cb >= d.n - nb) return;
    T* F = reinterpret_cast<T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
    T* buf = &Xs[0][0];                    // 64 x 33 entries: one row of 32 columns per pair
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int ci = cb + lane;
    const int c = ci < j0 ? ci : ci + nb;  // skip the panel columns
    const bool ok = ci < d.n - nb;
    for (int t = wp; t < cnt; t += 8)
      if (ok) buf[t * (kMaxNb + 1) + lane] = F[(size_t)(j0 + pr[2 + 2 * t]) * d.ld + c];
    __syncthreads();
    for (int t = wp; t < cnt; t += 8)
      if (ok) F[(size_t)(j0 + pr[1 + 2 * t]) * d.ld + c] = buf[t * (kMaxNb + 1) + lane];
    return;
  }
  // rows eliminated against the panel's diagonal block: the boundary rows, or
  // (block-local pivoting) every row below the block
  const int r0 = (below ? j0 + nb : d.k) + blockIdx.x * kL21Rows;
  if (r0 >= d.n) return;
  const int rows = min(kL21Rows, d.n - r0);
  T* F = reinterpret_cast<T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += 256) {
    const int i = e / nb, c = e - i * nb;
    Us[i][c] = F[(size_t)(j0 + i) * d.ld + j0 + c];
  }
  for (int e = tid; e < rows * nb; e += 256) {
    const int i = e / nb, c = e - i * nb;
    Xs[i][c] = F[(size_t)(r0 + i) * d.ld + j0 + c];
  }
  __syncthreads();
  R gmax = 0;
  if (tid < rows) {
    for (int j = 0; j < nb; ++j) {
      T x = Xs[tid][j];
      for (int l = 0; l < j; ++l) x = cfms(Xs[tid][l], Us[l][j], x);
      x = cmul(x, crcp(Us[j][j]));
      Xs[tid][j] = x;
      gmax = nanmax(gmax, cabs2(x));
    }
  }
  __syncthreads();
  for (int e = tid; e < rows * nb; e += 256) {
    const int i = e / nb, c = e - i * nb;
    F[(size_t)(r0 + i) * d.ld + j0 + c] = Xs[i][c];
  }
  for (int o = 16; o > 0; o >>= 1) gmax = nanmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  if ((tid & 31) == 0) s_g[tid >> 5] = gmax;
  __syncthreads();
  if (tid == 0) {
    R g = 0;
    for (int i = 0; i < 8; ++i) g = nanmax(g, s_g[i]);
    // max of non-negative floats (NaN included) is order independent as an int max
    atomicMax(reinterpret_cast<int*>(a.growth + (size_t)w * a.n_fronts + f), __float_as_int((float)sqrt((double)g)));
  }
}

template <typename T>
__global__ void __launch_bounds__(kTrsmCols)
lu_trsm_kernel(FactorLaunch a, const int* __restrict__ flist, int j0, int nbmax) {
  __shared__ T Ls[kMaxNb][kMaxNb + 1];
  const int w = blockIdx.z + a.w0;
  const int f = flist[blockIdx.y];
  const FrontDesc d = a.P.fronts[f];
  if (j0 >= d.k) return;
  const int nb = min(nbmax, d.k - j0);
  const int c = j0 + nb + blockIdx.x * kTrsmCols + threadIdx.x;
  if (j0 + nb + blockIdx.x * kTrsmCols >= d.n) return;
  T* F = reinterpret_cast<T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, l = e - i * nb;
    Ls[i][l] = F[(size_t)(j0 + i) * d.ld + j0 + l];
  }
  __syncthreads();
  if (c >= d.n) return;
  T x[kMaxNb];
#pragma unroll
  for (int i = 0; i < kMaxNb; ++i)
    if (i < nb) x[i] = F[(size_t)(j0 + i) * d.ld + c];
#pragma unroll
  for (int i = 1; i < kMaxNb; ++i) {
    if (i < nb) {
      T v = x[i];
#pragma unroll
      for (int l = 0; l < kMaxNb; ++l)
        if (l < i) v = cfms(Ls[i][l], x[l], v);
      x[i] = v;
    }
  }
#pragma unroll
  for (int i = 1; i < kMaxNb; ++i)
    if (i < nb) F[(size_t)(j0 + i) * d.ld + c] = x[i];
}

constexpr int kGemmTile = 64;
template <typename T> struct GemmKc;
template <> struct GemmKc<float2> { static constexpr int v = 32; };
template <> struct GemmKc<double2> { static constexpr int v = 16; };

// Two uses (SIMT complex FMA, 64 x 64 tiles):
//   schur = 0: panel step at j0 -- trailing update restricted to the pivot-block
//              rows and columns; the m x m update matrix S is left untouched
//   schur = 1: once per front after its last panel -- S = F22 - L21 U12, K = k
// Block row J of L11^-1 and block column J of U11^-1 of the listed large fronts,
// once the diagonal block J of the inverse store holds L_JJ^-1 / U_JJ^-1 and
// every block before J is done (block-local pivoting: rows of J never move
// again, and nothing later writes the entries read here):
//   lower, columns c in [c0, c0 + 32):  X[J][c] = -L_JJ^-1  sum_{l in [c, j0)} L[J][l] X[l][c]   (from L X = I)
//   upper, rows r in [r0, r0 + 32):     X[r][J] = -(sum_{l in [r, j0)} X[r][l] U[l][J]) U_JJ^-1 (from X U = I)
// One CTA per (32-wide chunk, triangle, front): blockIdx.x < nq lower chunk
// q = blockIdx.x, else upper chunk q = blockIdx.x - nq.  The contraction runs
// over 32-wide slices of l with the next slice prefetched into registers.
template <typename T>
__global__ void __launch_bounds__(256)
lu_inv_fold_kernel(FactorLaunch a, const int* __restrict__ flist, int j0, int nq) {
  __shared__ T Am[32][33];   // left operand slice, then T (the sum)
  __shared__ T Bm[32][33];   // right operand slice, then the diagonal inverse block
  using R = typename RealOf<T>::type;
  const int w = blockIdx.z + a.w0;
  const FrontDesc d = a.P.fronts[flist[blockIdx.y]];
  if (j0 >= d.k) return;
  const bool upper = (int)blockIdx.x >= nq;
  const int c0 = (upper ? (int)blockIdx.x - nq : (int)blockIdx.x) * 32;
  if (c0 >= j0) return;
  const int nb = min(kMaxNb, d.k - j0);
  const int ld = d.ld, ldk = d.ldk;
  const T* F = reinterpret_cast<const T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  T* X = reinterpret_cast<T*>(a.istore) + (size_t)w * a.istore_stride + d.iv_off;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const T one = cmk(R(1), R(0));
  // element e = ty + 8 q' of this thread's four: row (ty + 8 q'), column tx of a slice
  auto fetch = [&](int l0, T* ra, T* rb) {
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      const int i = ty + 8 * qq;
      const int la = l0 + tx;            // A[i][tx]: column l of the left operand
      T va = czero<T>();
      if (la < j0) {
        if (!upper) va = i < nb ? F[(size_t)(j0 + i) * ld + la] : czero<T>();
        else {
          const int r = c0 + i;
          va = (la >= r) ? X[(size_t)r * ldk + la] : czero<T>();
        }
      }
      ra[qq] = va;
      const int lb = l0 + i;             // B[i][tx]: row l of the right operand
      T vb = czero<T>();
      if (lb < j0) {
        if (!upper) {
          const int c = c0 + tx;
          vb = lb > c ? X[(size_t)lb * ldk + c] : (lb == c ? one : czero<T>());
        } else {
          vb = tx < nb ? F[(size_t)lb * ld + j0 + tx] : czero<T>();
        }
      }
      rb[qq] = vb;
    }
  };
  T acc[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};   // T[ty + 8 q'][tx]
  T ra[4], rb[4];
  fetch(c0, ra, rb);
  for (int l0 = c0; l0 < j0; l0 += 32) {
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      Am[ty + 8 * qq][tx] = ra[qq];
      Bm[ty + 8 * qq][tx] = rb[qq];
    }
    __syncthreads();
    if (l0 + 32 < j0) fetch(l0 + 32, ra, rb);
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const T bv = Bm[kk][tx];
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) acc[qq] = cfma(Am[ty + 8 * qq][kk], bv, acc[qq]);
    }
    __syncthreads();
  }
  // Am <- T, Bm <- L_JJ^-1 (unit diagonal) or U_JJ^-1, zero outside the block
#pragma unroll
  for (int qq = 0; qq < 4; ++qq) {
    const int i = ty + 8 * qq, j = tx;
    Am[i][j] = acc[qq];
    T v = czero<T>();
    if (i < nb && j < nb) {
      if (!upper) v = (j < i) ? X[(size_t)(j0 + i) * ldk + j0 + j] : (i == j ? one : czero<T>());
      else v = (j >= i) ? X[(size_t)(j0 + i) * ldk + j0 + j] : czero<T>();
    }
    Bm[i][j] = v;
  }
  __syncthreads();
#pragma unroll
  for (int qq = 0; qq < 4; ++qq) {
    const int i = ty + 8 * qq;
    T o0 = czero<T>(), o1 = czero<T>();
    if (!upper) {
      // X[J + i][c0 + tx] = -sum_t Li[i][t] T[t][tx]
#pragma unroll 8
      for (int t = 0; t < 32; t += 2) {
        o0 = cfms(Bm[i][t], Am[t][tx], o0);
        o1 = cfms(Bm[i][t + 1], Am[t + 1][tx], o1);
      }
      if (i < nb && c0 + tx < j0) X[(size_t)(j0 + i) * ldk + c0 + tx] = cadd(o0, o1);
    } else {
      // X[c0 + i][J + tx] = -sum_t T[i][t] Ui[t][tx]
#pragma unroll 8
      for (int t = 0; t < 32; t += 2) {
        o0 = cfms(Am[i][t], Bm[t][tx], o0);
        o1 = cfms(Am[i][t + 1], Bm[t + 1][tx], o1);
      }
      if (c0 + i < j0 && tx < nb) X[(size_t)(c0 + i) * ldk + j0 + tx] = cadd(o0, o1);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
lu_gemm_kernel(FactorLaunch a, const int* __restrict__ flist, int j0, int nbmax, int schur) {
  constexpr int KC = GemmKc<T>::v;
  __shared__ T As[kGemmTile][KC + 1];
  __shared__ T Bs[KC][kGemmTile + 1];
  __shared__ T dks[KC];                                 // symmetric form: d of the contracted pivots
  const int w = blockIdx.z + a.w0;
  const int f = flist[blockIdx.y];
  const FrontDesc d = a.P.fronts[f];
  if (!schur && j0 >= d.k) return;
  const int nb = schur ? d.k : min(nbmax, d.k - j0);   // contraction length
  const int kbeg = schur ? 0 : j0;                      // first contracted column of L / row of U
  const int base = schur ? d.k : j0 + nb;
  const int rem = d.n - base;
  if (rem <= 0) return;
  const int nt = (rem + kGemmTile - 1) / kGemmTile;
  if ((int)blockIdx.x >= nt * nt) return;
  const int ti = blockIdx.x / nt, tj = blockIdx.x - ti * nt;
  const int r0 = base + ti * kGemmTile, c0 = base + tj * kGemmTile;
  if (!schur && r0 >= d.k && c0 >= d.k) return;        // tile inside S: deferred to the Schur product
  // a front whose off-diagonal blocks come from the tensor cores: the pivot block only
  const bool pivonly = !schur && a.pivonly && a.pivonly[f];
  if (pivonly && (r0 >= d.k || c0 >= d.k)) return;
  // symmetric form: the lower triangle only, and in a panel step only the pivot columns
  const bool sym = a.sym != 0;
  if (sym && (r0 + kGemmTile - 1 < c0 || (!schur && c0 >= d.k))) return;
  j0 = kbeg;
  T* F = reinterpret_cast<T*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const T* X = reinterpret_cast<const T*>(a.istore) + (size_t)w * a.istore_stride + d.iv_off;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = czero<T>();
  for (int kc = 0; kc < nb; kc += KC) {
    for (int e = tid; e < kGemmTile * KC; e += 256) {
      const int r = e / KC, kk = e - r * KC;
      const int gr = r0 + r, gk = kc + kk;
      As[r][kk] = (gr < d.n && gk < nb) ? F[(size_t)gr * d.ld + j0 + gk] : czero<T>();
    }
    if (sym) {
      // B = diag(d) L^T over the contracted pivots j0 + gk: row gc of L (final: the panel step
      // that wrote it has finished), d from 1 / d on the diagonal of the inverse store
      if (tid < KC) {
        const int gk = kc + tid;
        dks[tid] = gk < nb ? crcp(X[(size_t)(j0 + gk) * d.ldk + j0 + gk]) : czero<T>();
      }
      __syncthreads();
      for (int e = tid; e < kGemmTile * KC; e += 256) {
        const int c = e / KC, kk = e - c * KC;
        const int gc = c0 + c, gk = kc + kk;
        Bs[kk][c] = (gc < d.n && gk < nb) ? cmul(dks[kk], F[(size_t)gc * d.ld + j0 + gk]) : czero<T>();
      }
    } else {
      for (int e = tid; e < kGemmTile * KC; e += 256) {
        const int kk = e / kGemmTile, c = e - kk * kGemmTile;
        const int gc = c0 + c, gk = kc + kk;
        Bs[kk][c] = (gc < d.n && gk < nb) ? F[(size_t)(j0 + gk) * d.ld + gc] : czero<T>();
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[ty + 16 * i][kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cfma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = r0 + ty + 16 * i;
    if (gr >= d.n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = c0 + tx + 16 * j;
      const bool live = sym       ? (gr >= gc && (schur || gc < d.k))
                        : pivonly ? (gr < d.k && gc < d.k)
                                  : (schur || gr < d.k || gc < d.k);
      if (gc < d.n && live) {
        T* p = F + (size_t)gr * d.ld + gc;
        *p = csub(*p, acc[i][j]);
      }
    }
  }
}

}  // namespace

int lu_small_max_n(int elem_bytes) { return elem_bytes == 8 ? kSmallMaxN : 64; }
int lu_small_class_n(int c) { return c == 0 ? 32 : c == 1 ? 48 : c == 2 ? 64 : kSmallMaxN; }

namespace {
__global__ void growth_max_kernel(const float* g, long long count, float* out) {
  __shared__ float red[32];
  float v = 0.f;
  for (long long t = threadIdx.x; t < count; t += blockDim.x) v = nanmax(v, g[t]);
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = nanmax(r, red[i]);
    *out = r;
  }
}
}  // namespace

cudaError_t launch_growth_max(const float* growth, long long count, float* out, cudaStream_t s) {
  growth_max_kernel<<<1, 1024, 0, s>>>(growth, count, out);
  return cudaGetLastError();
}

cudaError_t factor_init_attributes() {
  // small fronts: the front in shared memory
  cudaError_t e = cudaFuncSetAttribute(SmallCfg<float2, 96>::kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       96 * 97 * 8);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(SmallCfg<double2, 64>::kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 65 * 16);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(ldl_small_kernel<float2, kSmallThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           96 * 96 * 8);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(lu_step_local_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)step_local_smem(8));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(lu_step_local_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)step_local_smem(16));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(lu_panel_smem_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kPanelSmemBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(lu_panel_smem_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kPanelSmemBytes);
}
int lu_panel_width(int elem_bytes) { (void)elem_bytes; return kMaxNb; }

template <typename T>
void launch_build(const FactorLaunch& a, const int2* tasks, int ntasks, cudaStream_t s) {
  if (ntasks <= 0) return;
  build_kernel<T><<<dim3(ntasks, a.n_omega), kBuildWarps * 32, 0, s>>>(a, tasks);
}

template <typename T>
void launch_lu_small(const FactorLaunch& a, const int* flist, int nf, int nmax, cudaStream_t s) {
  if (nf <= 0) return;
  // fronts up to kSmallNarrowN: half the threads, so that twice as many fit on an SM
  if (a.sym) {
    const size_t smem = (size_t)nmax * nmax * sizeof(T);
    if (nmax <= kSmallNarrowN) ldl_small_kernel<T, kSmallThreads / 2><<<dim3(nf, a.n_omega), kSmallThreads / 2, smem, s>>>(a, flist);
    else ldl_small_kernel<T, kSmallThreads><<<dim3(nf, a.n_omega), kSmallThreads, smem, s>>>(a, flist);
    return;
  }
  const dim3 grid(nf, a.n_omega);
  const size_t smem = (size_t)nmax * (nmax | 1) * sizeof(T);   // rows of odd stride
  if (nmax <= 32) SmallCfg<T, 32>::kernel()<<<grid, SmallCfg<T, 32>::kThreads, smem, s>>>(a, flist);
  else if (nmax <= 48) SmallCfg<T, 48>::kernel()<<<grid, SmallCfg<T, 48>::kThreads, smem, s>>>(a, flist);
  else if (nmax <= 64) SmallCfg<T, 64>::kernel()<<<grid, SmallCfg<T, 64>::kThreads, smem, s>>>(a, flist);
  else if constexpr (sizeof(T) == 8) SmallCfg<T, 96>::kernel()<<<grid, SmallCfg<T, 96>::kThreads, smem, s>>>(a, flist);
}

template <typename T>
void launch_lu_panel(const FactorLaunch& a, const int* flist, int nf, int j0, int nb, int kmax, cudaStream_t s) {
  if (nf <= 0 || j0 >= kmax) return;
  const int rows = kmax - j0;
  const dim3 grid(nf, a.n_omega), blk(kRegWarps * 32);
  if (rows <= kRegWarps * 8) { lu_panel_reg_kernel<T, 8><<<grid, blk, 0, s>>>(a, flist, j0, nb); return; }
  if (rows <= kRegWarps * 16) { lu_panel_reg_kernel<T, 16><<<grid, blk, 0, s>>>(a, flist, j0, nb); return; }
  const size_t smem = (size_t)(kmax - j0) * (nb + 1) * sizeof(T);
  if (smem <= (size_t)kPanelSmemBytes)
    lu_panel_smem_kernel<T><<<dim3(nf, a.n_omega), kPanelSmemThreads, smem, s>>>(a, flist, j0, nb);
  else
    lu_panel_kernel<T><<<dim3(nf, a.n_omega), kPanelThreads, 0, s>>>(a, flist, j0, nb);
}

template <typename T>
void launch_lu_inv(const FactorLaunch& a, const int* flist, int nf, int kmax, cudaStream_t s) {
  if (nf <= 0 || kmax <= 0) return;
  const int nblk = (kmax + 31) / 32;
  lu_inv_kernel<T><<<dim3(2 * nblk, nf, a.n_omega), 256, 0, s>>>(a, flist, nblk);
}

template <typename T>
void launch_lu_step_local(const FactorLaunch& a, const int* flist, int nf, int j0, int nmax, cudaStream_t s) {
  if (nf <= 0) return;
  const int span = std::max(0, nmax - j0 - 1);
  const int nl = (span + kStepRows - 1) / kStepRows;
  // symmetric form: no U rows (the trailing update takes diag(d) L^T instead) and no row permutation
  const int nu = a.sym ? 0 : nl;
  const int np = a.sym ? 0 : (j0 + kStepCols - 1) / kStepCols;
  // CTAs resident at once on the current device
  int dev = 0, nsm = 0, per_sm = 0;
  const long long wave =
      (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
       cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lu_step_local_kernel<T>, 256, step_local_smem(sizeof(T))) ==
           cudaSuccess)
          ? (long long)std::max(1, per_sm) * nsm
          : (1LL << 40);
  const long long ctas = (long long)(1 + nl + nu + np) * nf * a.n_omega;
  if (ctas > wave && a.dblk) {
    // more than one wave: the diagonal block once per front (four warps: the block LU, then
    // role D; a smaller footprint, so that more fronts share an SM), then the substitutions
    lu_step_local_kernel<T><<<dim3(1, nf, a.n_omega), 128, step_diag_smem(sizeof(T)), s>>>(a, flist, j0, nl, nu, 1);
    if (nl + nu + np > 0)
      lu_step_local_kernel<T><<<dim3(nl + nu + np, nf, a.n_omega), 256, step_local_smem(sizeof(T)), s>>>(
          a, flist, j0, nl, nu, 2);
  } else {
    lu_step_local_kernel<T><<<dim3(1 + nl + nu + np, nf, a.n_omega), 256, step_local_smem(sizeof(T)), s>>>(
        a, flist, j0, nl, nu, 0);
  }
}

template <typename T>
void launch_lu_l21(const FactorLaunch& a, const int* flist, int nf, int j0, int nb, int mmax, int nmax,
                   int below, cudaStream_t s) {
  if (nf <= 0) return;
  const int rows = below ? nmax - j0 : mmax;
  const int nl21 = (rows + kL21Rows - 1) / kL21Rows;
  const int nswap = (nmax + 31) / 32;
  lu_l21_kernel<T><<<dim3(nl21 + nswap, nf, a.n_omega), 256, 0, s>>>(a, flist, j0, nb, nl21, below);
}

template <typename T>
void launch_lu_trsm(const FactorLaunch& a, const int* flist, int nf, int j0, int nb, int nmax,
                    cudaStream_t s) {
  const int cols = nmax - j0 - 1;
  if (nf <= 0 || cols <= 0) return;
  const int gx = (cols + kTrsmCols - 1) / kTrsmCols;
  lu_trsm_kernel<T><<<dim3(gx, nf, a.n_omega), kTrsmCols, 0, s>>>(a, flist, j0, nb);
}

template <typename T>
void launch_lu_gemm(const FactorLaunch& a, const int* flist, int nf, int j0, int nb, int nmax,
                    cudaStream_t s) {
  const int rem = nmax - j0 - 1;
  if (nf <= 0 || rem <= 0) return;
  const int nt = (rem + kGemmTile - 1) / kGemmTile;
  lu_gemm_kernel<T><<<dim3(nt * nt, nf, a.n_omega), 256, 0, s>>>(a, flist, j0, nb, 0);
}

template <typename T>
void launch_lu_inv_fold(const FactorLaunch& a, const int* flist, int nf, int j0, cudaStream_t s) {
  const int nq = (j0 + 31) / 32;
  if (nf <= 0 || nq <= 0) return;
  // the symmetric form needs L11^-1 only (the first nq CTAs)
  lu_inv_fold_kernel<T><<<dim3(a.sym ? nq : 2 * nq, nf, a.n_omega), 256, 0, s>>>(a, flist, j0, nq);
}

template <typename T>
void launch_schur_simt(const FactorLaunch& a, const int* flist, int nf, int mmax, cudaStream_t s) {
  if (nf <= 0 || mmax <= 0) return;
  const int nt = (mmax + kGemmTile - 1) / kGemmTile;
  lu_gemm_kernel<T><<<dim3(nt * nt, nf, a.n_omega), 256, 0, s>>>(a, flist, 0, 0, 1);
}

#define FDFD_INST(T)                                                                              \
  template void launch_build<T>(const FactorLaunch&, const int2*, int, cudaStream_t);            \
  template void launch_lu_small<T>(const FactorLaunch&, const int*, int, int, cudaStream_t);      \
  template void launch_lu_panel<T>(const FactorLaunch&, const int*, int, int, int, int, cudaStream_t); \
  template void launch_lu_l21<T>(const FactorLaunch&, const int*, int, int, int, int, int, int, cudaStream_t); \
  template void launch_lu_step_local<T>(const FactorLaunch&, const int*, int, int, int, cudaStream_t); \
  template void launch_lu_inv<T>(const FactorLaunch&, const int*, int, int, cudaStream_t); \
  template void launch_lu_trsm<T>(const FactorLaunch&, const int*, int, int, int, int, cudaStream_t); \
  template void launch_lu_gemm<T>(const FactorLaunch&, const int*, int, int, int, int, cudaStream_t); \
  template void launch_lu_inv_fold<T>(const FactorLaunch&, const int*, int, int, cudaStream_t); \
  template void launch_schur_simt<T>(const FactorLaunch&, const int*, int, int, cudaStream_t);
FDFD_INST(float2)
FDFD_INST(double2)
#undef FDFD_INST

}  // namespace fdfd
