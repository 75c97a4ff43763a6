// Update matrix of a front on the fifth-generation tensor cores (Sec. II: the
// multifrontal elimination forms S = F22 - L21 U12 for the parent's extend-add).
//
// The complex product P = L21 U12 (m x k times k x m, complex FP32) runs as one real
// GEMM on tcgen05 with FP32 accumulation in tensor memory:
//   A' = L21 as m x 2k reals (re, im interleaved along k, as stored),
//   B' = the 2k x 2m real embedding of U12: for U = U12[l][j] the 2 x 2 block at
//        (2l.., 2j..) is [[Re U, Im U], [-Im U, Re U]],
// so that (A' B')[r][2j] = Re P[r][j] and (A' B')[r][2j+1] = Im P[r][j]: the
// accumulator holds P already interleaved like the front, and the epilogue
// subtracts it from F22 in place.  Three forms of the FP32 operands:
//   1  TF32 (x rounded to 11 significant bits), one product;
//   2  TF32 hi + lo (hi = x rounded to TF32, lo = the remainder rounded to TF32),
//      products hi*hi + hi*lo + lo*hi;
//   3  BF16 three-way split x = x0 + x1 + x2 (each part the remainder rounded to
//      BF16: 24 significant bits together, i.e. x exactly), the six products whose
//      plane indices sum to at most 2 (the dropped ones are below 2^-24 |x y|); on
//      kind::f16 these take as long as form 2's three TF32 products.
//
// A pack kernel writes the planes of each 128-row (A) or 256-real-column (B) by
// 16-real-K tile into a workspace in the tensor core's canonical K-major layout
// without swizzle: 8-row x 16-byte core matrices, 128 contiguous bytes each, the
// K-adjacent ones of an 8-row group next to each other (leading byte offset 128),
// 8-row groups one tile row of 16 reals apart (stride byte offset).  The product
// kernel, one CTA per 128 x 128 complex output tile, streams the planes of a stage
// into a shared-memory ring with bulk asynchronous copies completed on mbarriers;
// one thread issues the MMAs (M = 128, N = 256) and frees a stage with
// tcgen05.commit; eight more warps move finished chunks of the sum out of tensor
// memory into FP32 registers and finally subtract the tile from F22.
// Every wait is bounded: a wait that gives up sets the error word to 2, the CTA
// drains its copies (bounded), frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "kernels.h"

namespace fdfd {
namespace {

constexpr int kTcM = kTcRows;              // output rows per CTA = MMA M
constexpr int kTcN = 2 * kTcCols;          // real output columns per CTA = MMA N
constexpr int kTcK = 2 * kTcPivots;        // real K per stage
constexpr int kTcRingMax = 196608;         // shared-memory ring bytes at most
constexpr int kTcTmemCols = 512;           // two FP32 accumulators of MMA N = 256 columns
constexpr int kTcThreads = 320;            // copy warp, MMA warp, 8 accumulation warps
constexpr int kTcAccWarps = 8;
constexpr int kTileStride = 2 * kTcCols + 1;   // floats per staged output row (odd: rows in distinct banks)

template <int FORM> struct Form {
  static_assert(FORM >= 1 && FORM <= 3, "forms 1-3");
  static constexpr int es = FORM == 3 ? 2 : 4;                    // bytes per element
  static constexpr int planes = FORM;
  static constexpr int nprod = FORM == 1 ? 1 : (FORM == 2 ? 3 : 6);
  static constexpr int tileA = kTcM * kTcK * es;                  // one plane of an A tile
  static constexpr int tileB = kTcN * kTcK * es;                  // one plane of a B tile
  static constexpr int stage = planes * (tileA + tileB);
  static constexpr int S = kTcRingMax / stage < 8 ? kTcRingMax / stage : 8;   // ring stages
  static constexpr int ring = S * stage;
  static constexpr int smem = ring + 256;                         // ring + barriers and flags
  static constexpr int upr = kTcK * es / 16;                      // 16-byte units per tile row
  static constexpr int group = upr * 128;                         // stride between 8-row groups
  static constexpr int ksteps = kTcK * es / 32;                   // MMAs of 32 bytes of K per stage
  // instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B type (bits 7-9,
  // 10-12: TF32 = 2 of kind::tf32, BF16 = 1 of kind::f16), both K-major, N >> 3 at
  // bit 17, M >> 4 at bit 24
  static constexpr uint32_t idesc = (1u << 4) | ((FORM == 3 ? 1u : 2u) << 7) | ((FORM == 3 ? 1u : 2u) << 10) |
                                    ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
  static_assert(tileA % 1024 == 0 && tileB % 1024 == 0 && stage % 1024 == 0, "1 KB alignment");
  static_assert(S >= 2 && smem <= 227 * 1024, "ring fits");
};
// plane indices (of A, of B) of product i, smallest terms first
__device__ __forceinline__ constexpr int prod_a(int form, int i) {
  return form == 2 ? (i == 0 ? 1 : 0) : form == 3 ? (i == 0 ? 2 : i == 1 ? 0 : i == 2 ? 1 : i == 3 ? 1 : 0) : 0;
}
__device__ __forceinline__ constexpr int prod_b(int form, int i) {
  return form == 2 ? (i == 1 ? 1 : 0) : form == 3 ? (i == 0 ? 0 : i == 1 ? 2 : i == 2 ? 1 : i == 3 ? 0 : i == 4 ? 1 : 0) : 0;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity to complete; false after limit_ns of
// global time (or 2^26 polls, should the timer not advance).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (uint32_t it = 1; it < (1u << 26); ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63) == 0 && gtimer() - t0 > limit_ns) return false;
  }
  return false;
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Shared-memory matrix descriptor, canonical K-major layout without swizzle:
// start address >> 4 (bits 0-13), leading byte offset >> 4 (16-29), stride byte
// offset >> 4 (32-45), the constant 1 at bit 46, layout type 0 (bits 61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t group) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(group >> 4) << 32) |
         (1ull << 46);
}
template <int FORM>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t ad, uint64_t bd, uint32_t acc) {
  if (FORM == 3)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d), "l"(ad), "l"(bd), "r"(Form<FORM>::idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d), "l"(ad), "l"(bd), "r"(Form<FORM>::idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
// 32 consecutive accumulator columns of this warp's 32 lanes (one row per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  // the registers are read only after the load has completed
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                 "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]),
                 "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]),
                 "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
               :
               : "memory");
}
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t bf16_bits(float x) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// One CTA per pack task (slot, operand, tile row, k-tile).  Unit u of a plane tile
// (16 bytes: 4 TF32 or 8 BF16 reals of one row) is (8-row group g, unit c of the
// row, row rr) with u = (g * upr + c) * 8 + rr.
template <int FORM>
__global__ void __launch_bounds__(256)
schur_pack_kernel(FactorLaunch a, TcLaunch t) {
  using Fm = Form<FORM>;
  constexpr int RU = 16 / Fm::es;   // reals per unit
  constexpr int CU = RU / 2;        // complex pivots per unit
  const int4 task = t.tasks[blockIdx.x];
  const TcFront fr = t.fronts[task.x];
  const int w = blockIdx.y + a.w0;
  const FrontDesc d = a.P.fronts[fr.f];
  const float2* F = reinterpret_cast<const float2*>(a.store) + (size_t)w * a.store_stride + d.st_off;
  const bool isA = task.y == 0;
  const int tile = isA ? Fm::tileA : Fm::tileB;
  unsigned char* dst = t.ws + (size_t)blockIdx.y * t.ws_stride + (isA ? fr.aoff : fr.boff) +
                       ((size_t)task.z * fr.Kt + task.w) * Fm::planes * tile;
  for (int u = threadIdx.x; u < tile / 16; u += blockDim.x) {
    const int rr = u & 7, c = (u >> 3) % Fm::upr, g = (u >> 3) / Fm::upr;
    const int l0 = task.w * kTcPivots + c * CU;   // first complex pivot of the unit
    float x[RU];
    const float2* X = reinterpret_cast<const float2*>(a.istore) + (size_t)w * a.istore_stride + d.iv_off;
    if (isA) {
      // A' row r: (Re, Im) of L21[r][l0..] (mode 0), of F21[r][l0..] (mode 1), of L11^-1[r][l0..] (mode 2)
      const int r = task.z * kTcM + g * 8 + rr;
#pragma unroll
      for (int i = 0; i < CU; ++i) {
        const int l = l0 + i;
        float2 v = make_float2(0.f, 0.f);
        if (fr.mode == 2) {
          if (r < d.k && l <= r) v = l == r ? make_float2(1.f, 0.f) : X[(size_t)r * d.ldk + l];
        } else if (r < d.m && l < d.k) {
          v = F[(size_t)(d.k + r) * d.ld + l];
        }
        x[2 * i] = v.x;
        x[2 * i + 1] = v.y;
      }
    } else {
      // B' (K-major) row n = 2 j + tt: (Re U, -Im U) per pivot for tt = 0, (Im U, Re U) for tt = 1,
      // U = U12[l][j] (mode 0), U11^-1[l][j] (mode 1), F12[perm l][j] (mode 2); the symmetric
      // form's U12 is diag(d) L21^T: d_l L21[j][l], 1 / d_l on the inverse store diagonal
      const int nrow = g * 8 + rr;
      const int j = task.z * kTcCols + (nrow >> 1), tt = nrow & 1;
      const int* Pm = a.perm + (size_t)w * a.perm_stride + d.piv_off;
#pragma unroll
      for (int i = 0; i < CU; ++i) {
        const int l = l0 + i;
        float2 v = make_float2(0.f, 0.f);
        if (fr.mode == 1) {
          if (j < d.k && l <= j) v = X[(size_t)l * d.ldk + j];
        } else if (j < d.m && l < d.k) {
          v = fr.mode == 2 ? F[(size_t)Pm[l] * d.ld + d.k + j]
              : a.sym     ? cmul(crcp(X[(size_t)l * d.ldk + l]), F[(size_t)(d.k + j) * d.ld + l])
                          : F[(size_t)l * d.ld + d.k + j];
        }
        x[2 * i] = tt ? v.y : v.x;
        x[2 * i + 1] = tt ? v.x : -v.y;
      }
    }
    if constexpr (FORM == 3) {
      uint32_t p0[RU / 2], p1[RU / 2], p2[RU / 2];
#pragma unroll
      for (int i = 0; i < RU; i += 2) {
        uint32_t h0[2], h1[2], h2[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float v = x[i + e];
          const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
          const float r1 = v - __bfloat162float(b0);
          const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
          const float r2 = r1 - __bfloat162float(b1);
          h0[e] = __bfloat16_as_ushort(b0);
          h1[e] = __bfloat16_as_ushort(b1);
          h2[e] = bf16_bits(r2);
        }
        p0[i / 2] = h0[0] | (h0[1] << 16);
        p1[i / 2] = h1[0] | (h1[1] << 16);
        p2[i / 2] = h2[0] | (h2[1] << 16);
      }
      reinterpret_cast<uint4*>(dst)[u] = make_uint4(p0[0], p0[1], p0[2], p0[3]);
      reinterpret_cast<uint4*>(dst + tile)[u] = make_uint4(p1[0], p1[1], p1[2], p1[3]);
      reinterpret_cast<uint4*>(dst + 2 * tile)[u] = make_uint4(p2[0], p2[1], p2[2], p2[3]);
    } else {
      static_assert(RU == 4, "TF32 units hold four reals");
      float4 h;
      h.x = tf32_rna(x[0]); h.y = tf32_rna(x[1]); h.z = tf32_rna(x[2]); h.w = tf32_rna(x[3]);
      reinterpret_cast<float4*>(dst)[u] = h;
      if constexpr (FORM == 2)
        reinterpret_cast<float4*>(dst + tile)[u] =
            make_float4(tf32_rna(x[0] - h.x), tf32_rna(x[1] - h.y), tf32_rna(x[2] - h.z), tf32_rna(x[3] - h.w));
    }
  }
}

constexpr unsigned long long kRoleWaitNs = 2000000000ull;   // copy / MMA waits
constexpr unsigned long long kDoneWaitNs = 6000000000ull;   // accumulation waits: outlast both roles
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// One CTA per output tile (slot, mt, nt): F22[128 mt.., 128 nt..] -= (L21 U12) tile.
// Warp 0 (lane 0) streams the plane tiles, warp 1 (lane 0) issues the MMAs, warps
// 2-9 accumulate.  The tensor core sums each chunk of t.chunk stages in one of two
// tensor-memory accumulators, alternately; the accumulation warps add every
// finished chunk into FP32 registers (round to nearest) while the next chunk runs
// in the other accumulator, so the tensor core's own accumulation rounding acts
// over one chunk at most.
template <int FORM>
__global__ void __launch_bounds__(kTcThreads, 1)
schur_tc_kernel(FactorLaunch a, TcLaunch t) {
  using Fm = Form<FORM>;
  constexpr int S = Fm::S, kA = Fm::planes * Fm::tileA, kB = Fm::planes * Fm::tileB, kStage = Fm::stage;
  extern __shared__ __align__(1024) unsigned char smem[];
  // full[S], empty[S], accumulator full[2], accumulator empty[2], done
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Fm::ring);
  // [0] tensor-memory address, [1] error, [2] k-tiles issued, [3] k-tiles consumed
  volatile uint32_t* sh = reinterpret_cast<volatile uint32_t*>(bar + 2 * S + 5);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 task = t.tasks[blockIdx.x];
  const TcFront fr = t.fronts[task.x];
  const int w = blockIdx.y + a.w0;
  const FrontDesc d = a.P.fronts[fr.f];
  const int chunk = t.chunk;
  // this CTA's share of the contraction: k-tiles [kb, kb + nk); a triangular operand
  // (modes 1, 2) is zero beyond pivot 128 (t + 1) of output column / row tile t
  const int kt_hi = fr.mode == 1 ? min(fr.Kt, (kTcCols / kTcPivots) * (task.z + 1))
                    : fr.mode == 2 ? min(fr.Kt, (kTcRows / kTcPivots) * (task.y + 1)) : fr.Kt;
  const int kb = (int)((long long)task.w * kt_hi / fr.nsplit);
  const int nk = (int)((long long)(task.w + 1) * kt_hi / fr.nsplit) - kb, nch = (nk + chunk - 1) / chunk;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t full0 = smem_u32(bar), empty0 = full0 + 8 * S, tfull0 = full0 + 16 * S, tempty0 = tfull0 + 16,
                 done = tfull0 + 32;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, kTcAccWarps);
    }
    mbar_init(done, 1);
    sh[1] = 0; sh[2] = 0; sh[3] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32((const void*)&sh[0])), "r"(kTcTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh[0];
  const unsigned char* ws = t.ws + (size_t)blockIdx.y * t.ws_stride;
  if (warp == 0) {
    if (lane == 0) {   // copies: plane tiles of A' row block mt and B' column block nt
      const unsigned char* ga = ws + fr.aoff + ((size_t)task.y * fr.Kt + kb) * kA;
      const unsigned char* gb = ws + fr.boff + ((size_t)task.z * fr.Kt + kb) * kB;
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % S;
        if (kt >= S && !mbar_wait(empty0 + 8 * s, ((kt / S) - 1) & 1, kRoleWaitNs)) { sh[1] = 1; break; }
        const uint32_t dst = sbase + s * kStage;
        mbar_expect_tx(full0 + 8 * s, kStage);
        bulk_g2s(dst, ga + (size_t)kt * kA, kA, full0 + 8 * s);
        bulk_g2s(dst + kA, gb + (size_t)kt * kB, kB, full0 + 8 * s);
        sh[2] = kt + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issue: ksteps MMAs of 32 bytes of K per stage, nprod products each
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % S, c = kt / chunk, b = c & 1;
        const bool first = kt % chunk == 0;
        if (first && c >= 2 && !mbar_wait(tempty0 + 8 * b, ((c >> 1) - 1) & 1, kRoleWaitNs)) { sh[1] = 1; break; }
        if (!mbar_wait(full0 + 8 * s, (kt / S) & 1, kRoleWaitNs)) { sh[1] = 1; break; }
        tc_fence_after();
        const uint32_t sa = sbase + s * kStage, sb = sa + kA, dacc = tmem + (uint32_t)(b * kTcN);
#pragma unroll
        for (int ks = 0; ks < Fm::ksteps; ++ks) {
#pragma unroll
          for (int pr = 0; pr < Fm::nprod; ++pr) {
            const uint64_t ad = sdesc(sa + prod_a(FORM, pr) * Fm::tileA + ks * 256, Fm::group);
            const uint64_t bd = sdesc(sb + prod_b(FORM, pr) * Fm::tileB + ks * 256, Fm::group);
            tc_mma<FORM>(dacc, ad, bd, (!first || ks != 0 || pr != 0) ? 1u : 0u);
          }
        }
        tc_commit(empty0 + 8 * s);
        if (kt % chunk == chunk - 1 || kt == nk - 1) tc_commit(tfull0 + 8 * b);
        sh[3] = kt + 1;
      }
      tc_commit(done);   // arrives once every MMA issued above has completed
      mbar_wait(done, 0, kDoneWaitNs);
    }
    __syncwarp();
  } else {
    // accumulation warp: TMEM lanes 32 (warp % 4).. (rows), real columns 128 h.. of each chunk
    const int q = warp & 3, h = (warp - 2) >> 2;
    float acc[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) acc[i] = 0.f;
    bool ok = nk > 0;
    for (int c = 0; c < nch; ++c) {
      const int b = c & 1;
      ok = __all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * b, (c >> 1) & 1, kDoneWaitNs));
      if (!ok) break;
      tc_fence_after();
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kTcN + h * 128 + j * 32), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[32 * j + i] += __uint_as_float(v[i]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * b);
    }
    // every accumulation warp reaches this barrier (named, the 256 accumulation threads)
    if (!ok && lane == 0) sh[1] = 1;
    asm volatile("bar.sync 1, 256;" ::: "memory");
    const bool good = sh[1] == 0;
    const int r = task.y * kTcM + 32 * q + lane;   // row of the output block
    bool apply = good;
    if (good && fr.nsplit > 1) {
      // post this split's partial sum; schur_split_sum_kernel adds the splits in order
      const size_t tile = (size_t)task.y * fr.Nt + task.z;
      float* pt = t.part + (size_t)blockIdx.y * t.part_stride + fr.poff + tile * fr.nsplit * kTcPartFloats;
      float4* mine = reinterpret_cast<float4*>(pt + (size_t)task.w * kTcPartFloats + (32 * q + lane) * kTcN + h * 128);
#pragma unroll
      for (int i = 0; i < 32; ++i) mine[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
      apply = false;
    }
    float2* const F = reinterpret_cast<float2*>(a.store) + (size_t)w * a.store_stride + d.st_off;
    const int j0 = task.z * kTcCols + h * 64;
    if (fr.mode == 0 && fr.nsplit == 1) {
      // the tile through shared memory (the ring is idle once every k-tile has been
      // consumed), so that F22 is read and written a row at a time by whole warps:
      // thread (row 32 q + lane, half h) stores its 128 reals, then each warp takes rows
      static_assert(Fm::ring >= kTcM * kTileStride * 4, "the staged tile fits in the ring");
      float* tile = reinterpret_cast<float*>(smem);
      if (apply) {
        float* mine = tile + (size_t)(32 * q + lane) * kTileStride + h * 128;
#pragma unroll
        for (int i = 0; i < 128; ++i) mine[i] = acc[i];
      }
      asm volatile("bar.sync 2, 256;" ::: "memory");   // every accumulation thread, good or not
      if (apply) {
        // warp aw takes rows aw, aw + 8, ...: four rows' loads (16 per lane) issued together
        constexpr int RB = 4, CU = kTcCols / 32;
        const int aw = warp - 2;                         // accumulation warp 0..7
        const int c0 = task.z * kTcCols;
        for (int rb = aw; rb < kTcM; rb += kTcAccWarps * RB) {
          float2 v[RB][CU];
#pragma unroll
          for (int t = 0; t < RB; ++t) {
            const int rr = task.y * kTcM + rb + kTcAccWarps * t;
            const float2* row = F + (size_t)(d.k + rr) * d.ld + d.k + c0;
#pragma unroll
            for (int u = 0; u < CU; ++u) {
              const int jc = lane + 32 * u;
              v[t][u] = (rr < d.m && c0 + jc < d.m) ? row[jc] : make_float2(0.f, 0.f);
            }
          }
#pragma unroll
          for (int t = 0; t < RB; ++t) {
            const int rl = rb + kTcAccWarps * t, rr = task.y * kTcM + rl;
            float2* row = F + (size_t)(d.k + rr) * d.ld + d.k + c0;
            const float* src = tile + (size_t)rl * kTileStride;
#pragma unroll
            for (int u = 0; u < CU; ++u) {
              const int jc = lane + 32 * u;
              if (rr < d.m && c0 + jc < d.m)
                row[jc] = make_float2(v[t][u].x - src[2 * jc], v[t][u].y - src[2 * jc + 1]);
            }
          }
        }
      }
    } else if (fr.mode == 0) {
      if (apply && r < d.m) {
        float2* row = F + (size_t)(d.k + r) * d.ld + d.k;
#pragma unroll
        for (int jj = 0; jj < 64; ++jj) {
          const int j = j0 + jj;
          if (j < d.m) {
            float2 sv = row[j];
            sv.x -= acc[2 * jj];
            sv.y -= acc[2 * jj + 1];
            row[j] = sv;
          }
        }
      }
    } else {
      // modes 1, 2: the product is the block itself (rows of L21 / of U12)
      const int nr = fr.mode == 1 ? d.m : d.k, nc = fr.mode == 1 ? d.k : d.m;
      float g2 = 0.f;
      if (apply && r < nr) {
        float2* row = fr.mode == 1 ? F + (size_t)(d.k + r) * d.ld : F + (size_t)r * d.ld + d.k;
#pragma unroll
        for (int jj = 0; jj < 64; ++jj) {
          const int j = j0 + jj;
          if (j < nc) {
            const float2 v = make_float2(acc[2 * jj], acc[2 * jj + 1]);
            row[j] = v;
            const float a2 = v.x * v.x + v.y * v.y;
            g2 = (a2 == a2) ? fmaxf(g2, a2) : INFINITY;
          }
        }
      }
      if (fr.mode == 1) {
        // growth: the largest |L21| entry (NaN -> inf), as the panel steps record it
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float og = __shfl_xor_sync(0xffffffffu, g2, o);
          g2 = og > g2 ? og : g2;
        }
        if (lane == 0 && g2 > 0.f) {
          float gv = sqrtf(g2);
          if (!(gv == gv)) gv = INFINITY;
          atomicMax(reinterpret_cast<int*>(a.growth + (size_t)w * a.n_fronts + fr.f), __float_as_int(gv));
        }
      }
    }
    if (!good && warp == 2 && lane == 0) atomicExch(t.err, 2);
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && sh[1] != 0) {
    // a role gave up: let the copies still in flight land before the CTA exits
    for (int kt = (int)sh[3]; kt < (int)sh[2]; ++kt)
      if (!mbar_wait(full0 + 8 * (kt % S), (kt / S) & 1, kRoleWaitNs)) break;
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
  }
}

// Split update matrices: S = F22 - sum over splits (in split order) of the partial
// sums, 16 rows of one output tile per CTA, thread = (row, 8 complex columns).
__global__ void __launch_bounds__(256)
schur_split_sum_kernel(FactorLaunch a, TcLaunch t) {
  const int4 task = t.tasks[blockIdx.x];   // (slot, mt, nt, first row of 16)
  const TcFront fr = t.fronts[task.x];
  const int w = blockIdx.y + a.w0;
  const FrontDesc d = a.P.fronts[fr.f];
  const int rr = task.w + (threadIdx.x >> 4), cq = threadIdx.x & 15;
  const int r = task.y * kTcM + rr;
  const float* pt = t.part + (size_t)blockIdx.y * t.part_stride + fr.poff +
                    ((size_t)task.y * fr.Nt + task.z) * fr.nsplit * kTcPartFloats + (size_t)rr * kTcN + cq * 16;
  float v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = 0.f;
  for (int sp = 0; sp < fr.nsplit; ++sp) {
    const float4* src = reinterpret_cast<const float4*>(pt + (size_t)sp * kTcPartFloats);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 x = __ldcg(src + i);
      v[4 * i] += x.x; v[4 * i + 1] += x.y; v[4 * i + 2] += x.z; v[4 * i + 3] += x.w;
    }
  }
  if (r >= d.m) return;
  float2* row = reinterpret_cast<float2*>(a.store) + (size_t)w * a.store_stride + d.st_off + (size_t)(d.k + r) * d.ld +
                d.k;
  const int j0 = task.z * kTcCols + cq * 8;
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int j = j0 + jj;
    if (j < d.m) {
      float2 sv = row[j];
      sv.x -= v[2 * jj];
      sv.y -= v[2 * jj + 1];
      row[j] = sv;
    }
  }
}

}  // namespace

void launch_schur_split_sum(const FactorLaunch& a, const TcLaunch& t, int ntasks, cudaStream_t s) {
  if (ntasks <= 0) return;
  schur_split_sum_kernel<<<dim3(ntasks, a.n_omega), 256, 0, s>>>(a, t);
}

int tc_splits(long long tiles, int Kt, int min_ctas) {
  if (tiles <= 0 || tiles >= min_ctas) return 1;
  const long long want = (min_ctas + tiles - 1) / tiles;
  const int most = Kt / 4 < 16 ? Kt / 4 : 16;
  return most < 1 ? 1 : (int)(want < most ? want : most);
}

long long tc_tile_bytes_a(int form) {
  return form == 3 ? 3LL * Form<3>::tileA : form == 2 ? 2LL * Form<2>::tileA : (long long)Form<1>::tileA;
}
namespace {
// Self-test of the pipeline's bounded waits: one mbarrier that nothing arrives at,
// waited on by the product kernel's own mbar_wait with a 1 ms limit.  The wait gives
// up and the error word is set to 2, exactly as by a product CTA whose copy or MMA
// never completed; the CTA then returns.
__global__ void mbar_probe_kernel(int* err) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) mbar_init(b, 1);
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(b, 0, 1000000ull)) atomicExch(err, 2);
}
}  // namespace

cudaError_t launch_mbar_probe(int* err, cudaStream_t s) {
  mbar_probe_kernel<<<1, 32, 0, s>>>(err);
  return cudaGetLastError();
}

long long tc_tile_bytes_b(int form) {
  return form == 3 ? 3LL * Form<3>::tileB : form == 2 ? 2LL * Form<2>::tileB : (long long)Form<1>::tileB;
}

void launch_schur_tc_pack(const FactorLaunch& a, const TcLaunch& t, int ntasks, int form, cudaStream_t s) {
  if (ntasks <= 0) return;
  const dim3 grid(ntasks, a.n_omega);
  if (form == 3) schur_pack_kernel<3><<<grid, 256, 0, s>>>(a, t);
  else if (form == 2) schur_pack_kernel<2><<<grid, 256, 0, s>>>(a, t);
  else schur_pack_kernel<1><<<grid, 256, 0, s>>>(a, t);
}

cudaError_t tc_init_attributes() {
  cudaError_t e = cudaFuncSetAttribute(schur_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, Form<1>::smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(schur_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Form<2>::smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(schur_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, Form<3>::smem);
}

void launch_schur_tc(const FactorLaunch& a, const TcLaunch& t, int ntiles, int form, cudaStream_t s) {
  if (ntiles <= 0) return;
  const dim3 grid(ntiles, a.n_omega);
  if (form == 3) schur_tc_kernel<3><<<grid, kTcThreads, Form<3>::smem, s>>>(a, t);
  else if (form == 2) schur_tc_kernel<2><<<grid, kTcThreads, Form<2>::smem, s>>>(a, t);
  else schur_tc_kernel<1><<<grid, kTcThreads, Form<1>::smem, s>>>(a, t);
}

}  // namespace fdfd
