// Fused pull-scheme kernels of the primal and adjoint steps.
//
// State buffer B (storage type S, M rows of N, deviations for the fluid):
// B^n_j(x) = W_j(f^{n-1}(x)), so the pre-collision state of Eq.
// "normal:iteration" is f^n_j(x) = w_j + B^n_j(x - e_j) (periodic shifts).
// One primal step gathers f^n(x) from the 19 (or 9) neighbours, applies the
// node operator W^x and writes B^{n+1}(x) at x: the reads are the only
// misaligned accesses, the writes are fully coalesced.
//
// Adjoint (Eqs. "adjoint:iteration" and "adjoint:operator", unsteady form):
// lambda^n_k(x) = sum_j lambda^{n+1}_j(x + e_j) dW^x_j/df_k(f^n(x)) + c_n dF^x/df_k,
// so the kernel gathers lambda^{n+1} from x + e_j, gathers f^n from B^n at
// x - e_j, applies the transposed node operator in registers and writes
// lambda^n(x) at x; the theta terms (Eq. "adjoint:derivative") are added to
// the FP64 gradient of the node.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "albm_node.cuh"

namespace albm {

// ---- launch tunables (minimum resident blocks per SM of 256 threads) -----
// primal: 7 blocks of 128 threads per SM (73 registers, no spills) measured
// fastest among 4x256, 5x256, 8x128 (64 registers, small spills) and 7x128
#ifndef ALBM_PRIMAL_MINB
#define ALBM_PRIMAL_MINB 7
#endif
#ifndef ALBM_PRIMAL_BLOCK
#define ALBM_PRIMAL_BLOCK 128
#endif
// resident blocks of the primal kernel on steps that record no objective:
// 8 (64 registers, no spills) with at most one scalar lattice, measured 2 %
// faster on the exchanger; with two scalars 8 blocks spill and lose 6 %
#ifndef ALBM_PRIMAL_MINB_NOOBJ
#define ALBM_PRIMAL_MINB_NOOBJ 8
#endif
#ifndef ALBM_PRIMAL_MINB_NOOBJ_NS2
#define ALBM_PRIMAL_MINB_NOOBJ_NS2 7
#endif
#ifndef ALBM_ADJOINT_MINB
#define ALBM_ADJOINT_MINB 8
#endif
// threads per block of the single-instance adjoint kernel: at its ~119
// registers 16 warps fit an SM; 8 blocks of 64 measured 1 % faster than 4 of
// 128 and 5 % faster than 2 of 256 (tighter caps spill and lose)
#ifndef ALBM_ADJ_BLOCK
#define ALBM_ADJ_BLOCK 64
#endif
// resident blocks of the adjoint kernel without objective sources: 10 holds
// the mixer's (MRT, two scalars) at 96 registers, which the inlet branches
// would otherwise raise to 104 (9 blocks)
#ifndef ALBM_ADJOINT_MINB_NOSRC
#define ALBM_ADJOINT_MINB_NOSRC 10
#endif
// streaming (evict-first) stores for the state and adjoint outputs, which
// the same kernel never reads back
#ifndef ALBM_STREAM_STORES
#define ALBM_STREAM_STORES 0
#endif
// ---- storage conversions -------------------------------------------------
__device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void st(float* p, float v) {
#if ALBM_STREAM_STORES
  __stcs(p, v);
#else
  *p = v;
#endif
}
__device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }

// Fluid deviation of population i from its stored value and back.  16-bit
// storage holds d_i - dev_off[i] (the deviation from the equilibrium at the
// reference velocity, smaller than the deviation from rest in a channel
// flowing near that velocity, so rounded with a smaller absolute error);
// FP32 storage holds d_i itself.
template <class S>
__device__ __forceinline__ float dev_in(const KParams& P, int i, float raw) {
  if constexpr (sizeof(S) == 2) return raw + P.dev_off[i];
  else return raw;
}
template <class S>
__device__ __forceinline__ float dev_out(const KParams& P, int i, float d) {
  if constexpr (sizeof(S) == 2) return d - P.dev_off[i];
  else return d;
}

// Element offset of density m at node j + off: m N + j + off.
__device__ __forceinline__ long long elem(int m, long long N, long long j, long long off = 0) {
  return (long long)m * N + j + off;
}

// ---- periodic neighbourhood of one node ----------------------------------
struct Geo {
  long long idx;
  int x, y, z;
  long long oxm, oxp, oym, oyp, ozm, ozp;  // index offsets to x-1, x+1, ...
  __device__ __forceinline__ long long off(int sx, int sy, int sz) const {
    long long o = 0;
    if (sx > 0) o += oxp;
    if (sx < 0) o += oxm;
    if (sy > 0) o += oyp;
    if (sy < 0) o += oym;
    if (sz > 0) o += ozp;
    if (sz < 0) o += ozm;
    return o;
  }
};

__device__ __forceinline__ Geo make_geo(const KParams& P, long long idx) {
  Geo g;
  g.idx = idx;
  // 32-bit index arithmetic (N < 2^31 is checked at creation)
  const unsigned n = (unsigned)idx;
  const unsigned r = fdiv(n, P.fd_nx);
  g.x = (int)(n - r * (unsigned)P.nx);
  g.z = (int)fdiv(r, P.fd_ny);
  g.y = (int)(r - (unsigned)g.z * (unsigned)P.ny);
  const long long sxy = (long long)P.nx * P.ny;
  g.oxm = (g.x == 0) ? (P.nx - 1) : -1;
  g.oxp = (g.x == P.nx - 1) ? -(P.nx - 1) : 1;
  g.oym = ((g.y == 0) ? (P.ny - 1) : -1) * (long long)P.nx;
  g.oyp = ((g.y == P.ny - 1) ? -(P.ny - 1) : 1) * (long long)P.nx;
  g.ozm = ((g.z == 0) ? (P.nz - 1) : -1) * sxy;
  g.ozp = ((g.z == P.nz - 1) ? -(P.nz - 1) : 1) * sxy;
  return g;
}

// ---- deterministic objective reduction ------------------------------------
// Each block writes the sums of its nodes' objective terms to its own slot
// of a partials array (plain stores: every slot is rewritten on each use, so
// nothing needs clearing); fold_partials_kernel then adds the slots in a
// fixed order.  J is therefore bit-reproducible, alone or batched.
__device__ __forceinline__ void block_partial2(double a, double b, double* out) {
  __shared__ double sa[32], sb[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sa[wid] = a;
    sb[wid] = b;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      out[0] = a;
      out[1] = b;
    }
  }
}

// out[k] = sum over blocks of partials[2 b + k], one block, fixed order
__global__ void __launch_bounds__(1024) fold_partials_kernel(const double* __restrict__ partials,
                                                            long long nblocks,
                                                            double* __restrict__ out);

// 16-bit primal steps work on the stored values (see ALBM_FOLD_OFFSET)
template <class S>
__host__ __device__ constexpr bool fold_offsets() {
  return ALBM_FOLD_OFFSET && sizeof(S) == 2;
}

template <class L, int NS, class S>
struct Gather {
  using LS = typename ScalarOf<L>::type;
  static constexpr int Q = L::Q, QS = LS::Q;
  static constexpr int NSA = NS > 0 ? NS : 1;
  // f^n(x) from B^n: d_j = B_j(x - e_j), g_j = B_{Q+s QS+j}(x - e_j)
  // RAW: the fluid values as stored (no reference offsets added)
  template <bool RAW = false>
  __device__ static __forceinline__ void pre(const KParams& P, const Geo& geo, long long N,
                                             const S* __restrict__ B, float* d, float (*g)[QS]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float raw = ld(B + elem(i, N, geo.idx, geo.off(-L::ex(i), -L::ey(i), -L::ez(i))));
      d[i] = RAW ? raw : dev_in<S>(P, i, raw);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i)
        g[s][i] = ld(B + elem(Q + s * QS + i, N, geo.idx,
                              geo.off(-LS::ex(i), -LS::ey(i), -LS::ez(i))));
  }
};

// ---------------------------------------------------------------------------
// primal step: B^{n+1}(x) = W^x(f^n(x)); optional objective terms of f^n
// ---------------------------------------------------------------------------
// OBJ: objective form compiled in (obj_kind); 0 when the step records no
// objective (obj is null): the objective terms and the block reduction are
// compiled out.
template <class L, int NS, bool MRT, class S, int OBJ = 2>
__device__ __forceinline__ void primal_body(const KParams& P, const S* __restrict__ Bin,
                                            S* __restrict__ Bout, const float* __restrict__ theta,
                                            const uint8_t* __restrict__ flags,
                                            double* __restrict__ obj, long long idx, int block) {
  using Ops = NodeOps<L, NS, MRT>;
  constexpr int Q = Ops::Q, QS = Ops::QS, NSA = Ops::NSA;
  double o1 = 0.0, o2 = 0.0;
  if (idx < P.N) {
    constexpr bool FOLD = fold_offsets<S>();
    const Geo geo = make_geo(P, idx);
    float d[Q], g[NSA][QS];
    Gather<L, NS, S>::template pre<FOLD>(P, geo, P.N, Bin, d, g);
    const uint8_t type = flags[idx];
    const float th = theta[idx];
    Ops::template forward<OBJ, FOLD>(P, type, th, geo.y, d, g, OBJ != 0 && obj != nullptr, o1, o2);
#pragma unroll
    for (int i = 0; i < Q; ++i) st(Bout + elem(i, P.N, idx), FOLD ? d[i] : dev_out<S>(P, i, d[i]));
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i) st(Bout + elem(Q + s * QS + i, P.N, idx), g[s][i]);
  }
  if (OBJ != 0 && obj != nullptr) block_partial2(o1, o2, obj + 2 * (long long)block);
}

template <class L, int NS, bool MRT, class S, int OBJ>
__global__ void __launch_bounds__(ALBM_PRIMAL_BLOCK,
                                  OBJ != 0 ? ALBM_PRIMAL_MINB
                                      : (NS >= 2 ? ALBM_PRIMAL_MINB_NOOBJ_NS2 : ALBM_PRIMAL_MINB_NOOBJ))
    primal_kernel(KParams P, const S* __restrict__ Bin,
                                                     S* __restrict__ Bout,
                                                     const float* __restrict__ theta,
                                                     const uint8_t* __restrict__ flags,
                                                     double* __restrict__ obj) {
  primal_body<L, NS, MRT, S, OBJ>(P, Bin, Bout, theta, flags, obj,
                                  (long long)blockIdx.x * blockDim.x + threadIdx.x, blockIdx.x);
}

// ---------------------------------------------------------------------------
// primal step for 16-bit storage, two nodes (2k, 2k+1) of a row per thread:
// every gather and store moves a 4-byte pair.  For a density with e_x = 0
// the pair is one aligned word; with e_x = +1 (source x - 1) it is the high
// half of the word before and the low half of the word at 2k, with e_x = -1
// the high half of the word at 2k and the low half of the next word (the
// words wrap at the ends of the row: periodic x).  Needs nx even.
// ---------------------------------------------------------------------------
template <class S> struct Pair;
template <> struct Pair<__nv_bfloat16> {
  using W = __nv_bfloat162;
  __device__ static __forceinline__ float2 ld(const __nv_bfloat16* p) {
    return __bfloat1622float2(__ldg(reinterpret_cast<const W*>(p)));
  }
  __device__ static __forceinline__ void st(__nv_bfloat16* p, float a, float b) {
    *reinterpret_cast<W*>(p) = __floats2bfloat162_rn(a, b);
  }
};
template <> struct Pair<__half> {
  using W = __half2;
  __device__ static __forceinline__ float2 ld(const __half* p) {
    return __half22float2(__ldg(reinterpret_cast<const W*>(p)));
  }
  __device__ static __forceinline__ void st(__half* p, float a, float b) {
    *reinterpret_cast<W*>(p) = __floats2half2_rn(a, b);
  }
};

// p points at the word of the pair's own column in the source row; dxm and
// dxp are the element offsets of the words before and after it (-2 and +2,
// or across the row's periodic wrap)
template <class S>
__device__ __forceinline__ void gather_pair(const S* p, int ex, int dxm, int dxp, float& a, float& b) {
  if (ex == 0) {
    const float2 w = Pair<S>::ld(p);
    a = w.x;
    b = w.y;
  } else if (ex > 0) {  // sources x - 1, x
    const float2 w0 = Pair<S>::ld(p + dxm);
    const float2 w1 = Pair<S>::ld(p);
    a = w0.y;
    b = w1.x;
  } else {              // sources x + 1, x + 2
    const float2 w1 = Pair<S>::ld(p);
    const float2 w2 = Pair<S>::ld(p + dxp);
    a = w1.y;
    b = w2.x;
  }
}

template <class L, int NS, bool MRT, class S, int OBJ = 2>
__device__ __forceinline__ void primal_pair_body(const KParams& P, const S* __restrict__ Bin,
                                                 S* __restrict__ Bout, const float* __restrict__ theta,
                                                 const uint8_t* __restrict__ flags,
                                                 double* __restrict__ obj, long long pair, int block) {
  using Ops = NodeOps<L, NS, MRT>;
  using LS = typename Ops::LS;
  constexpr int Q = Ops::Q, QS = Ops::QS, NSA = Ops::NSA;
  double o1 = 0.0, o2 = 0.0;
  const int hx = P.nx >> 1;
  if (pair < P.N / 2) {
    const unsigned rw = fdiv((unsigned)pair, P.fd_hx);
    const long long row = rw;
    const int x = 2 * (int)((unsigned)pair - rw * (unsigned)hx);
    const int z = (int)fdiv(rw, P.fd_ny);
    const int y = (int)(rw - (unsigned)z * (unsigned)P.ny);
    const int ym = y == 0 ? P.ny - 1 : y - 1, yp = y == P.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? P.nz - 1 : z - 1, zp = z == P.nz - 1 ? 0 : z + 1;
    // One 64-bit base pointer at the pair's first node; every gather and
    // store is a 32-bit element offset from it (the state has fewer than
    // 2^31 elements: checked by the launcher), density m at m N plus the
    // source row's shift.
    const long long idx = row * P.nx + x;
    const int N32 = (int)P.N;
    auto rowrel = [&](int ey, int ez) -> int {  // source row of shift (ey, ez), relative
      const int ys = ey > 0 ? ym : (ey < 0 ? yp : y);
      const int zs = ez > 0 ? zm : (ez < 0 ? zp : z);
      return ((zs - z) * P.ny + (ys - y)) * P.nx;
    };
    const int dxm = (x == 0 ? P.nx - 2 : x - 2) - x;
    const int dxp = (x + 2 == P.nx ? 0 : x + 2) - x;
    const S* bin = Bin + idx;
    float da[Q], db[Q], ga[NSA][QS], gb[NSA][QS];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      gather_pair<S>(bin + (i * N32 + rowrel(L::ey(i), L::ez(i))), L::ex(i), dxm, dxp, da[i], db[i]);
      if constexpr (!fold_offsets<S>()) {
        da[i] = dev_in<S>(P, i, da[i]);
        db[i] = dev_in<S>(P, i, db[i]);
      }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i)
        gather_pair<S>(bin + ((Q + s * QS + i) * N32 + rowrel(LS::ey(i), LS::ez(i))), LS::ex(i), dxm,
                       dxp, ga[s][i], gb[s][i]);
    const float2 th = *reinterpret_cast<const float2*>(theta + idx);
    const uint8_t ta = flags[idx], tb = flags[idx + 1];
    constexpr bool FOLD = fold_offsets<S>();
    Ops::template forward<OBJ, FOLD>(P, ta, th.x, y, da, ga, OBJ != 0 && obj != nullptr, o1, o2);
    Ops::template forward<OBJ, FOLD>(P, tb, th.y, y, db, gb, OBJ != 0 && obj != nullptr, o1, o2);
    S* bout = Bout + idx;
#pragma unroll
    for (int i = 0; i < Q; ++i)
      Pair<S>::st(bout + i * N32, FOLD ? da[i] : dev_out<S>(P, i, da[i]),
                  FOLD ? db[i] : dev_out<S>(P, i, db[i]));
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i) Pair<S>::st(bout + (Q + s * QS + i) * N32, ga[s][i], gb[s][i]);
  }
  if (OBJ != 0 && obj != nullptr) block_partial2(o1, o2, obj + 2 * (long long)block);
}

// resident blocks of the paired 16-bit primal (128 threads): 6 (80
// registers, a few spilled bytes) measured 1.3 % faster than 5 (96
// registers) on the exchanger; two scalars keep 4 (they spill at 5)
#ifndef ALBM_PAIR_MINB
#define ALBM_PAIR_MINB 6
#endif
template <class L, int NS, bool MRT, class S, int OBJ>
__global__ void __launch_bounds__(ALBM_PRIMAL_BLOCK, NS >= 2 ? 4 : ALBM_PAIR_MINB) primal_pair_kernel(
    KParams P, const S* __restrict__ Bin, S* __restrict__ Bout, const float* __restrict__ theta,
    const uint8_t* __restrict__ flags, double* __restrict__ obj) {
  primal_pair_body<L, NS, MRT, S, OBJ>(P, Bin, Bout, theta, flags, obj,
                                       (long long)blockIdx.x * blockDim.x + threadIdx.x, blockIdx.x);
}

// objective terms of f^n only (no state write), used for F(f^N)
template <class L, int NS, bool MRT, class S>
__global__ void __launch_bounds__(256) objective_kernel(KParams P, const S* __restrict__ Bin,
                                                        const float* __restrict__ theta,
                                                        const uint8_t* __restrict__ flags,
                                                        double* __restrict__ obj) {
  using Ops = NodeOps<L, NS, MRT>;
  constexpr int Q = Ops::Q, QS = Ops::QS, NSA = Ops::NSA;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double o1 = 0.0, o2 = 0.0;
  if (idx < P.N) {
    const uint8_t type = flags[idx];
    const bool relevant = (P.objective == OBJ_DISSIPATION) ? (type == FLUID)
                                                           : (type == OUTLET || type == INLET);
    if (relevant) {
      const Geo geo = make_geo(P, idx);
      float d[Q], g[NSA][QS];
      Gather<L, NS, S>::pre(P, geo, P.N, Bin, d, g);
      Ops::forward(P, type, theta[idx], geo.y, d, g, true, o1, o2);
    }
  }
  block_partial2(o1, o2, obj + 2 * (long long)blockIdx.x);
}


// ---------------------------------------------------------------------------
// adjoint step: lambda^n(x) from lambda^{n+1}(x + e_j) and f^n(x)
// ---------------------------------------------------------------------------
// Gradient modes of the adjoint step.  Unsteady adjoint (default): the
// theta terms are added to grad.  Fixed-point ALBS at a held state (Sec.
// 2.2, Eq. adjoint:iteration; overwrite set): the node's gradient estimate
// g of Eq. adjoint:derivative from the iterate this step consumes
// overwrites grad.  One-shot design update fused into the step (Sec. 3.3,
// Eq. gradient:update with the penalty of Eq. P; theta_out set): g
// overwrites grad and, on design nodes, theta_out = clamp(theta + zeta
// (sign g - penalty (1 - 2 theta)), 0, 1) in FP32.  Each thread reads and
// writes only its own node's theta, after its last read of it.
struct OneShot {
  const uint8_t* design;
  float* theta_out;
  float zeta, penalty, sign;
  int overwrite;
};

// lambda^{n+1} prefetch of the single-instance adjoint (ALBM_ADJ_CPASYNC):
// each thread copies its own gathers into its column of a shared-memory
// block with 4-byte cp.async right after the node index is known, so they
// travel while the forward quantities are recomputed, and reads them back
// after waiting for its own copies (no barrier: no thread reads another's).
#ifndef ALBM_ADJ_CPASYNC
#define ALBM_ADJ_CPASYNC 0
#endif
__device__ __forceinline__ void lam_cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void lam_cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void lam_cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <class L, int NS, bool MRT, class S, int SRC = 2, bool PREF = false>
__device__ __forceinline__ void adjoint_body(const KParams& P, const float* __restrict__ lam_in,
                                             const S* __restrict__ Bn, float* __restrict__ lam_out,
                                             const float* __restrict__ theta,
                                             const uint8_t* __restrict__ flags,
                                             double* __restrict__ grad, float ws,
                                             const double* __restrict__ stat_n, int has_next,
                                             long long idx, const OneShot& os) {
  using Ops = NodeOps<L, NS, MRT>;
  using LS = typename Ops::LS;
  constexpr int Q = Ops::Q, QS = Ops::QS, NSA = Ops::NSA;
  if (idx >= P.N) return;
  const Geo geo = make_geo(P, idx);
  [[maybe_unused]] float* sl = nullptr;
  if constexpr (PREF) {
    extern __shared__ float adj_lam_smem[];
    sl = adj_lam_smem + threadIdx.x;
    if (has_next) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        lam_cp_async4(sl + i * blockDim.x,
                      lam_in + elem(i, P.N, idx, geo.off(L::ex(i), L::ey(i), L::ez(i))));
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int i = 0; i < QS; ++i)
          lam_cp_async4(sl + (Q + s * QS + i) * blockDim.x,
                        lam_in + elem(Q + s * QS + i, P.N, idx,
                                      geo.off(LS::ex(i), LS::ey(i), LS::ez(i))));
      lam_cp_async_commit();
    }
  }
  float d[Q], g[NSA][QS];
  Gather<L, NS, S>::pre(P, geo, P.N, Bn, d, g);
  const uint8_t type = flags[idx];
  // outlet mean of scalar 0 at this step (variance objective)
  const float cbar = stat_n != nullptr ? (float)(stat_n[0] * (double)P.inv_A_out) : 0.0f;
  // lambda^{n+1}_j(x + e_j), or zero for the first (source-only) step
  auto load = [&](float* a, float (*b)[QS]) {
    if (has_next && PREF) {
      lam_cp_async_wait_all();
#pragma unroll
      for (int i = 0; i < Q; ++i) a[i] = sl[i * blockDim.x];
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int i = 0; i < QS; ++i) b[s][i] = sl[(Q + s * QS + i) * blockDim.x];
    } else if (has_next) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        a[i] = __ldg(lam_in + elem(i, P.N, idx, geo.off(L::ex(i), L::ey(i), L::ez(i))));
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int i = 0; i < QS; ++i)
          b[s][i] = __ldg(lam_in + elem(Q + s * QS + i, P.N, idx,
                                        geo.off(LS::ex(i), LS::ey(i), LS::ez(i))));
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) a[i] = 0.0f;
#pragma unroll
      for (int s = 0; s < NSA; ++s)
#pragma unroll
        for (int i = 0; i < QS; ++i) b[s][i] = 0.0f;
    }
  };
  float lam[Q], lamg[NSA][QS], dth;
  const float th = theta[idx];
  Ops::template reverse<decltype(load), SRC>(P, type, th, geo.y, d, g, load, ws, cbar, lam, lamg,
                                             dth);
#pragma unroll
  for (int i = 0; i < Q; ++i) st(lam_out + elem(i, P.N, idx), lam[i]);
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int i = 0; i < QS; ++i) st(lam_out + elem(Q + s * QS + i, P.N, idx), lamg[s][i]);
  const bool has_theta = type == FLUID || type == INLET || type == OUTLET;
  if (os.theta_out != nullptr || os.overwrite) {
    const float gk = has_theta ? dth : 0.0f;
    grad[idx] = (double)gk;
    if (os.theta_out != nullptr && os.design[idx]) {
      const float tn = th + os.zeta * (os.sign * gk - os.penalty * (1.0f - 2.0f * th));
      os.theta_out[idx] = fminf(fmaxf(tn, 0.0f), 1.0f);
    }
  } else if (has_theta) {
    grad[idx] += (double)dth;
  }
}

// SRC: source form compiled in (obj_kind of ws != 0); most steps of a long
// horizon with a short objective window carry none, and the kernels with
// fewer source terms hold fewer registers across the lambda gathers
template <class L, int NS, bool MRT, class S, int SRC>
__global__ void __launch_bounds__(ALBM_ADJ_BLOCK, SRC == 2 ? ALBM_ADJOINT_MINB : ALBM_ADJOINT_MINB_NOSRC) adjoint_kernel(KParams P, const float* __restrict__ lam_in,
                                                      const S* __restrict__ Bn,
                                                      float* __restrict__ lam_out,
                                                      const float* __restrict__ theta,
                                                      const uint8_t* __restrict__ flags,
                                                      double* __restrict__ grad, float ws,
                                                      const double* __restrict__ stat_n,
                                                      int has_next, OneShot os) {
  adjoint_body<L, NS, MRT, S, SRC, ALBM_ADJ_CPASYNC != 0>(
      P, lam_in, Bn, lam_out, theta, flags, grad, ws, stat_n, has_next,
      (long long)blockIdx.x * blockDim.x + threadIdx.x, os);
}

// ---------------------------------------------------------------------------
// batched steps: one launch advances every instance of a batch by one step.
// The instance table travels in the kernel's parameter space (grid
// constant); block b belongs to the instance whose block range holds b, so
// every block is uniform in its instance and runs exactly the per-node code
// of the single-instance kernels (bit-identical results).
// ---------------------------------------------------------------------------
constexpr int kMaxBatch = 64;

struct InstanceDesc {
  KParams P;
  const void* Bin;      // primal: state n; adjoint: state n (f^n)
  void* Bout;           // primal: state n+1
  const float* theta;
  const uint8_t* flags;
  double* obj;          // primal: per-block objective partials, or null
  const float* lam_in;
  float* lam_out;
  double* grad;
  const double* stat_n;
  float ws;
  int has_next;
  long long block_begin;
};

struct BatchArgs {
  int n;
  InstanceDesc inst[kMaxBatch];
};
// kernel parameters may take up to 32764 bytes (sm_70 and newer)
static_assert(sizeof(BatchArgs) <= 32000, "instance table exceeds the kernel parameter space");

// the instance whose block range holds this block: binary search over the
// ascending block_begin of the table
__device__ __forceinline__ int batch_instance(const BatchArgs& a) {
  int lo = 0, hi = a.n - 1;
  const long long b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b >= a.inst[mid].block_begin) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <class L, int NS, bool MRT, class S>
__global__ void __launch_bounds__(ALBM_PRIMAL_BLOCK, 1024 / ALBM_PRIMAL_BLOCK) primal_batch_kernel(const __grid_constant__ BatchArgs args) {
  const InstanceDesc& D = args.inst[batch_instance(args)];
  const int block = (int)((long long)blockIdx.x - D.block_begin);
  const long long idx = (long long)block * blockDim.x + threadIdx.x;
  // the same specialisation as the single-instance launch of this step, so
  // that batched and lone results agree bit for bit
  switch (obj_kind(D.obj != nullptr, D.P.objective)) {
    case 0:
      primal_body<L, NS, MRT, S, 0>(D.P, (const S*)D.Bin, (S*)D.Bout, D.theta, D.flags, D.obj, idx,
                                    block);
      break;
    case 1:
      primal_body<L, NS, MRT, S, 1>(D.P, (const S*)D.Bin, (S*)D.Bout, D.theta, D.flags, D.obj, idx,
                                    block);
      break;
    default:
      primal_body<L, NS, MRT, S, 2>(D.P, (const S*)D.Bin, (S*)D.Bout, D.theta, D.flags, D.obj, idx,
                                    block);
  }
}

template <class L, int NS, bool MRT, class S>
__global__ void __launch_bounds__(256, 2) adjoint_batch_kernel(const __grid_constant__ BatchArgs args) {
  const InstanceDesc& D = args.inst[batch_instance(args)];
  const long long block = (long long)blockIdx.x - D.block_begin;
  const long long idx = block * blockDim.x + threadIdx.x;
  switch (obj_kind(D.ws != 0.0f, D.P.objective)) {
    case 0:
      adjoint_body<L, NS, MRT, S, 0>(D.P, D.lam_in, (const S*)D.Bin, D.lam_out, D.theta, D.flags,
                                     D.grad, D.ws, D.stat_n, D.has_next, idx, OneShot{});
      break;
    case 1:
      adjoint_body<L, NS, MRT, S, 1>(D.P, D.lam_in, (const S*)D.Bin, D.lam_out, D.theta, D.flags,
                                     D.grad, D.ws, D.stat_n, D.has_next, idx, OneShot{});
      break;
    default:
      adjoint_body<L, NS, MRT, S, 2>(D.P, D.lam_in, (const S*)D.Bin, D.lam_out, D.theta, D.flags,
                                     D.grad, D.ws, D.stat_n, D.has_next, idx, OneShot{});
  }
}

// ---------------------------------------------------------------------------
// state import / export (full values, FP32) and health check
// ---------------------------------------------------------------------------
template <class L, int NS, class S>
__global__ void export_kernel(KParams P, const S* __restrict__ B, float* __restrict__ out, int post) {
  using LS = typename ScalarOf<L>::type;
  constexpr int Q = L::Q, QS = LS::Q;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
  const Geo geo = make_geo(P, idx);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const long long src = post ? idx : idx + geo.off(-L::ex(i), -L::ey(i), -L::ez(i));
    out[(long long)i * P.N + idx] = L::w(i) + dev_in<S>(P, i, ld(B + (long long)i * P.N + src));
  }
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int i = 0; i < QS; ++i) {
      const long long m = Q + s * QS + i;
      const long long src = post ? idx : idx + geo.off(-LS::ex(i), -LS::ey(i), -LS::ez(i));
      out[m * P.N + idx] = ld(B + m * P.N + src);
    }
}

// B_j(x) = f_j(x + e_j) - w_j, so that the gather of the next step sees f
template <class L, int NS, class S>
__global__ void import_kernel(KParams P, const float* __restrict__ in, S* __restrict__ B) {
  using LS = typename ScalarOf<L>::type;
  constexpr int Q = L::Q, QS = LS::Q;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
  const Geo geo = make_geo(P, idx);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const long long src = idx + geo.off(L::ex(i), L::ey(i), L::ez(i));
    st(B + (long long)i * P.N + idx, dev_out<S>(P, i, __ldg(in + (long long)i * P.N + src) - L::w(i)));
  }
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int i = 0; i < QS; ++i) {
      const long long m = Q + s * QS + i;
      const long long src = idx + geo.off(LS::ex(i), LS::ey(i), LS::ez(i));
      st(B + m * P.N + idx, __ldg(in + m * P.N + src));
    }
}

// the rest state f^0 = w (deviation 0), fluid rows as stored, scalars 0
template <class L, int NS, class S>
__global__ void rest_kernel(KParams P, S* __restrict__ B) {
  using LS = typename ScalarOf<L>::type;
  constexpr int Q = L::Q, QS = LS::Q;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
#pragma unroll
  for (int i = 0; i < Q; ++i) st(B + (long long)i * P.N + idx, dev_out<S>(P, i, 0.0f));
#pragma unroll
  for (int m = Q; m < Q + NS * QS; ++m) st(B + (long long)m * P.N + idx, 0.0f);
}

template <class S>
__global__ void nonfinite_kernel(const S* __restrict__ B, long long n, unsigned long long* count) {
  unsigned long long c = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = ld(B + i);
    if (!isfinite(v)) ++c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// ---------------------------------------------------------------------------
// host-side launchers, one set per (lattice, collision, scalars, storage)
// ---------------------------------------------------------------------------
}  // namespace albm

#include "albm_tiles.cuh"

namespace albm {

struct StepArgs {
  const void* Bin;
  void* Bout;
  const float* theta;
  const uint8_t* flags;
  double* obj;
  const float* lam_in;
  float* lam_out;
  double* grad;
  float ws;
  const double* stat_n;
  int has_next;
  const float* fin;
  float* fout;
  int post;
  unsigned long long* count;
  int* err;             // set by a staged kernel whose bounded wait expired
  OneShot os;           // fused one-shot update of the adjoint step (theta_out null: off)
};

struct KernelSet {
  cudaError_t (*primal)(const KParams&, const StepArgs&, cudaStream_t);
  cudaError_t (*objective)(const KParams&, const StepArgs&, cudaStream_t);
  cudaError_t (*adjoint)(const KParams&, const StepArgs&, cudaStream_t);
  cudaError_t (*exportf)(const KParams&, const StepArgs&, cudaStream_t);
  cudaError_t (*importf)(const KParams&, const StepArgs&, cudaStream_t);
  cudaError_t (*nonfinite)(const KParams&, const StepArgs&, int M, cudaStream_t);
  cudaError_t (*rest)(const KParams&, const StepArgs&, cudaStream_t);
  cudaError_t (*preload)();  // load every kernel of the set on the current device
  cudaError_t (*primal_batch)(const BatchArgs&, long long blocks, cudaStream_t);
  cudaError_t (*adjoint_batch)(const BatchArgs&, long long blocks, cudaStream_t);
  cudaError_t (*primal_tiles)(const KParams&, const StepArgs&, cudaStream_t);
  cudaError_t (*adjoint_tiles)(const KParams&, const StepArgs&, cudaStream_t);
  cudaError_t (*primal_async)(const KParams&, const StepArgs&, cudaStream_t);
  cudaError_t (*adjoint_async)(const KParams&, const StepArgs&, cudaStream_t);
  long long (*primal_partials)(const KParams&);  // objective slots the primal kernel writes
  int storage_bytes;
};

// persistent grid of a staged kernel: resident blocks per SM x SMs, at most
// the number of tiles
template <class K>
inline cudaError_t tiles_grid(K kernel, size_t smem, long long ntiles, unsigned* grid) {
  int dev = 0, sms = 0, bps = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, kTile, smem);
  if (e != cudaSuccess) return e;
  long long g = (long long)sms * (bps > 0 ? bps : 1);
  *grid = (unsigned)(g < ntiles ? g : ntiles);
  return cudaSuccess;
}

constexpr int kBlock = 256;

template <class L, int NS, bool MRT, class S>
struct Launch {
  static unsigned blocks(const KParams& P) { return (unsigned)((P.N + kBlock - 1) / kBlock); }
  // 16-bit storage with an even nx runs two nodes per thread (element
  // offsets within one state in 32 bits: fewer than 2^31 elements)
  static bool paired(const KParams& P) {
    return sizeof(S) == 2 && (P.nx % 2) == 0 &&
           (long long)(L::Q + NS * ScalarOf<L>::type::Q) * P.N < (1LL << 31);
  }
  static cudaError_t primal(const KParams& P, const StepArgs& a, cudaStream_t st) {
    if constexpr (sizeof(S) == 2) {
      if (paired(P)) {
        const unsigned nb = (unsigned)((P.N / 2 + ALBM_PRIMAL_BLOCK - 1) / ALBM_PRIMAL_BLOCK);
        const int ok = obj_kind(a.obj != nullptr, P.objective);
        auto k = ok == 0 ? primal_pair_kernel<L, NS, MRT, S, 0>
                 : ok == 1 ? primal_pair_kernel<L, NS, MRT, S, 1>
                           : primal_pair_kernel<L, NS, MRT, S, 2>;
        k<<<nb, ALBM_PRIMAL_BLOCK, 0, st>>>(P, (const S*)a.Bin, (S*)a.Bout, a.theta, a.flags,
                                            a.obj);
        return cudaGetLastError();
      }
    }
    const unsigned nb = (unsigned)((P.N + ALBM_PRIMAL_BLOCK - 1) / ALBM_PRIMAL_BLOCK);
    const int ok = obj_kind(a.obj != nullptr, P.objective);
    auto k = ok == 0 ? primal_kernel<L, NS, MRT, S, 0>
             : ok == 1 ? primal_kernel<L, NS, MRT, S, 1>
                       : primal_kernel<L, NS, MRT, S, 2>;
    k<<<nb, ALBM_PRIMAL_BLOCK, 0, st>>>(P, (const S*)a.Bin, (S*)a.Bout, a.theta, a.flags, a.obj);
    return cudaGetLastError();
  }
  static cudaError_t objective(const KParams& P, const StepArgs& a, cudaStream_t st) {
    objective_kernel<L, NS, MRT, S><<<blocks(P), kBlock, 0, st>>>(P, (const S*)a.Bin, a.theta,
                                                                  a.flags, a.obj);
    return cudaGetLastError();
  }
  static cudaError_t adjoint(const KParams& P, const StepArgs& a, cudaStream_t st) {
    const unsigned nb = (unsigned)((P.N + ALBM_ADJ_BLOCK - 1) / ALBM_ADJ_BLOCK);
    const int sk = obj_kind(a.ws != 0.0f, P.objective);
    auto k = sk == 0 ? adjoint_kernel<L, NS, MRT, S, 0>
             : sk == 1 ? adjoint_kernel<L, NS, MRT, S, 1>
                       : adjoint_kernel<L, NS, MRT, S, 2>;
    const size_t smem = ALBM_ADJ_CPASYNC ? sizeof(float) * (size_t)(L::Q + NS * ScalarOf<L>::type::Q) *
                                               ALBM_ADJ_BLOCK
                                         : 0;
    k<<<nb, ALBM_ADJ_BLOCK, smem, st>>>(P, a.lam_in, (const S*)a.Bin, a.lam_out, a.theta, a.flags,
                                        a.grad, a.ws, a.stat_n, a.has_next, a.os);
    return cudaGetLastError();
  }
  static cudaError_t exportf(const KParams& P, const StepArgs& a, cudaStream_t st) {
    export_kernel<L, NS, S><<<blocks(P), kBlock, 0, st>>>(P, (const S*)a.Bin, a.fout, a.post);
    return cudaGetLastError();
  }
  static cudaError_t importf(const KParams& P, const StepArgs& a, cudaStream_t st) {
    import_kernel<L, NS, S><<<blocks(P), kBlock, 0, st>>>(P, a.fin, (S*)a.Bout);
    return cudaGetLastError();
  }
  static cudaError_t rest(const KParams& P, const StepArgs& a, cudaStream_t st) {
    rest_kernel<L, NS, S><<<blocks(P), kBlock, 0, st>>>(P, (S*)a.Bout);
    return cudaGetLastError();
  }
  static cudaError_t nonfinite(const KParams& P, const StepArgs& a, int M, cudaStream_t st) {
    nonfinite_kernel<S><<<152 * 8, kBlock, 0, st>>>((const S*)a.Bin, (long long)M * P.N, a.count);
    return cudaGetLastError();
  }
  static cudaError_t primal_batch(const BatchArgs& a, long long blocks, cudaStream_t st) {
    primal_batch_kernel<L, NS, MRT, S><<<(unsigned)blocks, ALBM_PRIMAL_BLOCK, 0, st>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t adjoint_batch(const BatchArgs& a, long long blocks, cudaStream_t st) {
    adjoint_batch_kernel<L, NS, MRT, S><<<(unsigned)blocks, kBlock, 0, st>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t primal_tiles(const KParams& P, const StepArgs& a, cudaStream_t st) {
    using Lay = TileLayout<L, NS, S, kTile>;
    const size_t smem = Lay::header + 2 * Lay::primal_stage;
    auto k = primal_tiles_kernel<L, NS, MRT, S, kTile>;
    static unsigned grid_cache = 0;
    static long long tiles_cache = -1;
    const long long ntiles = P.N / kTile;
    if (tiles_cache != ntiles) {
      cudaError_t e = tiles_grid(k, smem, ntiles, &grid_cache);
      if (e != cudaSuccess) return e;
      tiles_cache = ntiles;
    }
    k<<<grid_cache, kTile, smem, st>>>(P, (const S*)a.Bin, (S*)a.Bout, a.theta, a.flags, a.obj, a.err);
    return cudaGetLastError();
  }
  static cudaError_t adjoint_tiles(const KParams& P, const StepArgs& a, cudaStream_t st) {
    using Lay = TileLayout<L, NS, S, kTile>;
    const size_t smem = Lay::header + 2 * Lay::adjoint_stage;
    auto k = adjoint_tiles_kernel<L, NS, MRT, S, kTile>;
    static unsigned grid_cache = 0;
    static long long tiles_cache = -1;
    const long long ntiles = P.N / kTile;
    if (tiles_cache != ntiles) {
      cudaError_t e = tiles_grid(k, smem, ntiles, &grid_cache);
      if (e != cudaSuccess) return e;
      tiles_cache = ntiles;
    }
    k<<<grid_cache, kTile, smem, st>>>(P, a.lam_in, (const S*)a.Bin, a.lam_out, a.theta, a.flags,
                                       a.grad, a.ws, a.stat_n, a.has_next, a.err);
    return cudaGetLastError();
  }
  static cudaError_t primal_async(const KParams& P, const StepArgs& a, cudaStream_t st) {
    using Lay = TileLayout<L, NS, S, kTile>;
    const size_t smem = Lay::header_async + 2 * Lay::primal_stage;
    auto k = primal_async_kernel<L, NS, MRT, S, kTile>;
    static unsigned grid_cache = 0;
    static long long tiles_cache = -1;
    const long long ntiles = P.N / kTile;
    if (tiles_cache != ntiles) {
      cudaError_t e = tiles_grid(k, smem, ntiles, &grid_cache);
      if (e != cudaSuccess) return e;
      tiles_cache = ntiles;
    }
    k<<<grid_cache, kTile, smem, st>>>(P, (const S*)a.Bin, (S*)a.Bout, a.theta, a.flags, a.obj);
    return cudaGetLastError();
  }
  static cudaError_t adjoint_async(const KParams& P, const StepArgs& a, cudaStream_t st) {
    using Lay = TileLayout<L, NS, S, kTile>;
    const size_t smem = Lay::header_async + 2 * Lay::adjoint_stage;
    auto k = adjoint_async_kernel<L, NS, MRT, S, kTile>;
    static unsigned grid_cache = 0;
    static long long tiles_cache = -1;
    const long long ntiles = P.N / kTile;
    if (tiles_cache != ntiles) {
      cudaError_t e = tiles_grid(k, smem, ntiles, &grid_cache);
      if (e != cudaSuccess) return e;
      tiles_cache = ntiles;
    }
    k<<<grid_cache, kTile, smem, st>>>(P, a.lam_in, (const S*)a.Bin, a.lam_out, a.theta, a.flags,
                                       a.grad, a.ws, a.stat_n, a.has_next);
    return cudaGetLastError();
  }
  // With lazy module loading a kernel is loaded at its first launch, which
  // allocates device memory: a launch late in a run, when state pools have
  // taken the memory, could fail.  Querying every kernel's attributes loads
  // them all while the handle is created.
  static cudaError_t preload() {
    static std::atomic<unsigned long long> done{0};   // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return cudaSuccess;
    cudaFuncAttributes fa;
    const void* ks[] = {
        (const void*)primal_kernel<L, NS, MRT, S, 0>, (const void*)primal_kernel<L, NS, MRT, S, 1>,
        (const void*)primal_kernel<L, NS, MRT, S, 2>, (const void*)objective_kernel<L, NS, MRT, S>,
        (const void*)adjoint_kernel<L, NS, MRT, S, 0>, (const void*)adjoint_kernel<L, NS, MRT, S, 1>,
        (const void*)adjoint_kernel<L, NS, MRT, S, 2>, (const void*)export_kernel<L, NS, S>,
        (const void*)import_kernel<L, NS, S>, (const void*)rest_kernel<L, NS, S>,
        (const void*)nonfinite_kernel<S>, (const void*)primal_batch_kernel<L, NS, MRT, S>,
        (const void*)adjoint_batch_kernel<L, NS, MRT, S>,
        (const void*)primal_tiles_kernel<L, NS, MRT, S, kTile>,
        (const void*)adjoint_tiles_kernel<L, NS, MRT, S, kTile>,
        (const void*)primal_async_kernel<L, NS, MRT, S, kTile>,
        (const void*)adjoint_async_kernel<L, NS, MRT, S, kTile>};
    for (const void* k : ks) {
      e = cudaFuncGetAttributes(&fa, k);
      if (e != cudaSuccess) return e;
    }
    if constexpr (sizeof(S) == 2) {
      const void* kp[] = {(const void*)primal_pair_kernel<L, NS, MRT, S, 0>,
                          (const void*)primal_pair_kernel<L, NS, MRT, S, 1>,
                          (const void*)primal_pair_kernel<L, NS, MRT, S, 2>};
      for (const void* k : kp) {
        e = cudaFuncGetAttributes(&fa, k);
        if (e != cudaSuccess) return e;
      }
    }
    done.fetch_or(bit);
    return cudaSuccess;
  }
  static long long primal_partials(const KParams& P) {
    const long long threads = paired(P) ? P.N / 2 : P.N;
    return (threads + ALBM_PRIMAL_BLOCK - 1) / ALBM_PRIMAL_BLOCK;
  }
  static KernelSet set() {
    return KernelSet{&primal, &objective, &adjoint, &exportf, &importf, &nonfinite, &rest,
                     &preload, &primal_batch, &adjoint_batch, &primal_tiles, &adjoint_tiles,
                     &primal_async, &adjoint_async, &primal_partials, (int)sizeof(S)};
  }
};

// The kernel set of one (lattice, collision, storage) for 0..MAXNS scalars.
template <class L, bool MRT, class S, int MAXNS>
bool pick_scalars(int nscalars, KernelSet* out) {
  switch (nscalars) {
    case 0: *out = Launch<L, 0, MRT, S>::set(); return true;
    case 1: *out = Launch<L, 1, MRT, S>::set(); return true;
    case 2:
      if constexpr (MAXNS >= 2) {
        *out = Launch<L, 2, MRT, S>::set();
        return true;
      }
      return false;
    default: return false;
  }
}

// Lookup of the instantiated sets, defined in the per-lattice translation
// units (split by storage type so that they build in parallel).
bool kernels_d2q9_f32(bool mrt, int nscalars, KernelSet* out);
bool kernels_d2q9_bf16(bool mrt, int nscalars, KernelSet* out);
bool kernels_d2q9_f16(bool mrt, int nscalars, KernelSet* out);
bool kernels_d3q19_bgk_f32(int nscalars, KernelSet* out);
bool kernels_d3q19_bgk_bf16(int nscalars, KernelSet* out);
bool kernels_d3q19_bgk_f16(int nscalars, KernelSet* out);
bool kernels_d3q19_mrt_f32(int nscalars, KernelSet* out);
bool kernels_d3q19_mrt_bf16(int nscalars, KernelSet* out);
bool kernels_d3q19_mrt_f16(int nscalars, KernelSet* out);

inline bool kernels_d2q9(bool mrt, int nscalars, int precision, KernelSet* out) {
  switch (precision) {
    case 0: return kernels_d2q9_f32(mrt, nscalars, out);
    case 1: return kernels_d2q9_bf16(mrt, nscalars, out);
    case 2: return kernels_d2q9_f16(mrt, nscalars, out);
    default: return false;
  }
}

inline bool kernels_d3q19(bool mrt, int nscalars, int precision, KernelSet* out) {
  switch (precision) {
    case 0: return mrt ? kernels_d3q19_mrt_f32(nscalars, out) : kernels_d3q19_bgk_f32(nscalars, out);
    case 1: return mrt ? kernels_d3q19_mrt_bf16(nscalars, out) : kernels_d3q19_bgk_bf16(nscalars, out);
    case 2: return mrt ? kernels_d3q19_mrt_f16(nscalars, out) : kernels_d3q19_bgk_f16(nscalars, out);
    default: return false;
  }
}

}  // namespace albm
