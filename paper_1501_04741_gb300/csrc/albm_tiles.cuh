// Tile-staged primal and adjoint steps: TMA bulk copies into shared memory.
//
// A tile is TX consecutive nodes of one x-row (fixed y, z).  The populations
// the tile's nodes gather live in rows of the source planes: for density j,
// f^n_j(x) = B_j(x - e_j) comes from the row (y - e_jy, z - e_jz) at x - e_jx
// (Eq. normal:iteration in pull form), and the adjoint's lambda^{n+1}_j(x +
// e_j) from the row (y + e_jy, z + e_jz) at x + e_jx (Eq. adjoint:iteration).
// One elected thread copies, for every density, the row segment
// [x0 - H, x0 + TX + H) (H = 16 bytes of elements: the x +- 1 halo, widened
// so every copy starts and ends on a 16-byte boundary) with
// cp.async.bulk into shared memory; at the ends of a row the halo comes from
// the other end (periodic x) by a separate 16-byte copy.  Completion is
// signalled through an mbarrier with expect_tx.  Two stages: the copies of
// the block's next tile are in flight while it computes the current one, so
// the memory parallelism no longer depends on registers or resident warps,
// and the per-gather index arithmetic becomes a shared-memory offset.
//
// Every wait on an mbarrier is bounded: if a stage does not complete within
// the limit, the block records an error (LBM_ERR_TIMEOUT on the host), waits
// with a bound for both stages' copies still in flight and returns.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace albm {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Waits are bounded by a number of polls (each poll may suspend the thread
// for a while): KParams.wait_polls for a stage the block is about to use
// (negative: the default), kDrainPolls when a block that gave up drains the
// copies it still has in flight before it leaves.
constexpr long long kDrainPolls = 1LL << 22;

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, long long polls) {
  for (long long i = 0; i < polls; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

__device__ __forceinline__ long long stage_polls(const KParams& P) {
  return P.wait_polls < 0 ? kDrainPolls : (long long)P.wait_polls;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Copy the tile's row segment [x0 - H, x0 + TX + H) of one source row into
// dst (TX + 2H elements); returns the bytes issued.
template <class T, int TX>
__device__ __forceinline__ uint32_t load_row_segment(T* dst, const T* row, int x0, int Lx,
                                                     uint64_t* bar) {
  constexpr int H = 16 / (int)sizeof(T);
  constexpr uint32_t HB = 16;
  if (x0 == 0 && x0 + TX == Lx) {  // whole row: both halos wrap
    bulk_load(dst, row + Lx - H, HB, bar);
    bulk_load(dst + H, row, (uint32_t)(TX * sizeof(T)), bar);
    bulk_load(dst + H + TX, row, HB, bar);
  } else if (x0 == 0) {
    bulk_load(dst, row + Lx - H, HB, bar);
    bulk_load(dst + H, row, (uint32_t)((TX + H) * sizeof(T)), bar);
  } else if (x0 + TX == Lx) {
    bulk_load(dst, row + x0 - H, (uint32_t)((TX + H) * sizeof(T)), bar);
    bulk_load(dst + H + TX, row, HB, bar);
  } else {
    bulk_load(dst, row + x0 - H, (uint32_t)((TX + 2 * H) * sizeof(T)), bar);
  }
  return (uint32_t)((TX + 2 * H) * sizeof(T));
}

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// nodes per tile of the staged kernels (threads per block)
constexpr int kTile = 128;

// ---------------------------------------------------------------------------
// primal
// ---------------------------------------------------------------------------
template <class L, int NS, class S, int TX>
struct TileLayout {
  using LS = typename ScalarOf<L>::type;
  static constexpr int M = L::Q + NS * LS::Q;
  static constexpr int H = 16 / (int)sizeof(S);
  static constexpr int W = TX + 2 * H;              // staged row length (elements)
  static constexpr int HL = 4;                      // halo of the FP32 adjoint rows
  static constexpr int WL = TX + 2 * HL;
  static constexpr size_t primal_stage = (size_t)M * W * sizeof(S);
  static constexpr size_t adjoint_stage = (size_t)M * W * sizeof(S) + (size_t)M * WL * sizeof(float);
  static constexpr size_t header = 128;             // two mbarriers, padded
  static constexpr size_t header_async = ((4 * M * 8 + 127) / 128) * 128;  // row bases
  // one issuing thread per staged row (f and lambda rows of the adjoint)
  static_assert(2 * M <= TX, "a tile needs a thread per staged row");
};

template <class L, int NS, bool MRT, class S, int TX>
__global__ void __launch_bounds__(TX) primal_tiles_kernel(KParams P, const S* __restrict__ Bin,
                                                          S* __restrict__ Bout,
                                                          const float* __restrict__ theta,
                                                          const uint8_t* __restrict__ flags,
                                                          double* __restrict__ obj,
                                                          int* __restrict__ err) {
  using Ops = NodeOps<L, NS, MRT>;
  using LS = typename Ops::LS;
  using Lay = TileLayout<L, NS, S, TX>;
  constexpr int Q = Ops::Q, QS = Ops::QS, NSA = Ops::NSA, M = Lay::M, H = Lay::H, W = Lay::W;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  S* stage[2] = {reinterpret_cast<S*>(smem + Lay::header),
                 reinterpret_cast<S*>(smem + Lay::header + Lay::primal_stage)};
  const int Lx = P.nx;
  const int tiles_x = Lx / TX;
  const long long ntiles = (long long)tiles_x * P.ny * P.nz;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // thread 0 registers the stage's bytes once; thread m < M issues the
  // copies of density m (transient negative transaction counts are allowed)
  auto issue = [&](long long t, int sg) {
    const long long row = t / tiles_x;
    const int x0 = (int)(t - row * tiles_x) * TX;
    const int y = (int)(row % P.ny), z = (int)(row / P.ny);
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar[sg], (uint32_t)Lay::primal_stage);
    const int m = threadIdx.x;
    if (m < M) {
      int ey = 0, ez = 0;
#pragma unroll
      for (int i = 0; i < M; ++i)
        if (i == m) {
          ey = i < Q ? L::ey(i) : LS::ey((i - Q) % QS);
          ez = i < Q ? L::ez(i) : LS::ez((i - Q) % QS);
        }
      const int ys = wrap(y - ey, P.ny), zs = wrap(z - ez, P.nz);
      const S* src = Bin + (long long)m * P.N + ((long long)zs * P.ny + ys) * Lx;
      load_row_segment<S, TX>(stage[sg] + m * W, src, x0, Lx, &bar[sg]);
    }
  };
  uint32_t phase[2] = {0u, 0u};
  long long t = blockIdx.x;
  if (t < ntiles) issue(t, 0);
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int sg = it & 1;
    const long long tn = t + gridDim.x;
    if (tn < ntiles) issue(tn, sg ^ 1);
    const bool ok = mbar_wait(&bar[sg], phase[sg], stage_polls(P));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      // leave no copy in flight: drain the stage given up on and the next one
      mbar_wait(&bar[sg], phase[sg], kDrainPolls);
      if (tn < ntiles) mbar_wait(&bar[sg ^ 1], phase[sg ^ 1], kDrainPolls);
      return;
    }
    phase[sg] ^= 1u;
    const long long row = t / tiles_x;
    const int x0 = (int)(t - row * tiles_x) * TX;
    const int y = (int)(row % P.ny);
    const int lx = threadIdx.x;
    const long long idx = row * Lx + x0 + lx;
    const S* sb = stage[sg];
    float d[Q], g[NSA][QS];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float raw = to_f(sb[i * W + H + lx - L::ex(i)]);
      d[i] = fold_offsets<S>() ? raw : dev_in<S>(P, i, raw);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i) g[s][i] = to_f(sb[(Q + s * QS + i) * W + H + lx - LS::ex(i)]);
    double o1 = 0.0, o2 = 0.0;
    Ops::template forward<2, fold_offsets<S>()>(P, flags[idx], theta[idx], y, d, g, obj != nullptr,
                                                o1, o2);
#pragma unroll
    for (int i = 0; i < Q; ++i)
      st(Bout + (long long)i * P.N + idx, fold_offsets<S>() ? d[i] : dev_out<S>(P, i, d[i]));
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i) st(Bout + (long long)(Q + s * QS + i) * P.N + idx, g[s][i]);
    if (obj != nullptr) block_partial2(o1, o2, obj + 2 * t);
    __syncthreads();  // the stage may be refilled from here on
  }
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
template <class L, int NS, bool MRT, class S, int TX>
__global__ void __launch_bounds__(TX) adjoint_tiles_kernel(
    KParams P, const float* __restrict__ lam_in, const S* __restrict__ Bn,
    float* __restrict__ lam_out, const float* __restrict__ theta, const uint8_t* __restrict__ flags,
    double* __restrict__ grad, float ws, const double* __restrict__ stat_n, int has_next,
    int* __restrict__ err) {
  using Ops = NodeOps<L, NS, MRT>;
  using LS = typename Ops::LS;
  using Lay = TileLayout<L, NS, S, TX>;
  constexpr int Q = Ops::Q, QS = Ops::QS, NSA = Ops::NSA, M = Lay::M, H = Lay::H, W = Lay::W;
  constexpr int HL = Lay::HL, WL = Lay::WL;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  unsigned char* base[2] = {smem + Lay::header, smem + Lay::header + Lay::adjoint_stage};
  const int Lx = P.nx;
  const int tiles_x = Lx / TX;
  const long long ntiles = (long long)tiles_x * P.ny * P.nz;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const uint32_t stage_bytes =
      (uint32_t)((size_t)M * W * sizeof(S) + (has_next ? (size_t)M * WL * sizeof(float) : 0));
  // thread 0 registers the stage's bytes once; thread m < M issues the f
  // copies of density m and thread M + m its lambda copies
  auto issue = [&](long long t, int sg) {
    const long long row = t / tiles_x;
    const int x0 = (int)(t - row * tiles_x) * TX;
    const int y = (int)(row % P.ny), z = (int)(row / P.ny);
    S* fs = reinterpret_cast<S*>(base[sg]);
    float* ls = reinterpret_cast<float*>(base[sg] + (size_t)M * W * sizeof(S));
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar[sg], stage_bytes);
    const bool lam_row = threadIdx.x >= M;
    const int m = lam_row ? threadIdx.x - M : threadIdx.x;
    if (m < M && (!lam_row || has_next)) {
      int ey = 0, ez = 0;
#pragma unroll
      for (int i = 0; i < M; ++i)
        if (i == m) {
          ey = i < Q ? L::ey(i) : LS::ey((i - Q) % QS);
          ez = i < Q ? L::ez(i) : LS::ez((i - Q) % QS);
        }
      if (!lam_row) {  // f^n_m(x) = B_m(x - e_m)
        const int ys = wrap(y - ey, P.ny), zs = wrap(z - ez, P.nz);
        load_row_segment<S, TX>(fs + m * W, Bn + (long long)m * P.N + ((long long)zs * P.ny + ys) * Lx,
                                x0, Lx, &bar[sg]);
      } else {         // lambda^{n+1}_m(x + e_m)
        const int yl = wrap(y + ey, P.ny), zl = wrap(z + ez, P.nz);
        load_row_segment<float, TX>(ls + m * WL,
                                    lam_in + (long long)m * P.N + ((long long)zl * P.ny + yl) * Lx,
                                    x0, Lx, &bar[sg]);
      }
    }
  };
  uint32_t phase[2] = {0u, 0u};
  long long t = blockIdx.x;
  if (t < ntiles) issue(t, 0);
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int sg = it & 1;
    const long long tn = t + gridDim.x;
    if (tn < ntiles) issue(tn, sg ^ 1);
    const bool ok = mbar_wait(&bar[sg], phase[sg], stage_polls(P));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      // leave no copy in flight: drain the stage given up on and the next one
      mbar_wait(&bar[sg], phase[sg], kDrainPolls);
      if (tn < ntiles) mbar_wait(&bar[sg ^ 1], phase[sg ^ 1], kDrainPolls);
      return;
    }
    phase[sg] ^= 1u;
    const long long row = t / tiles_x;
    const int x0 = (int)(t - row * tiles_x) * TX;
    const int y = (int)(row % P.ny);
    const int lx = threadIdx.x;
    const long long idx = row * Lx + x0 + lx;
    const S* fs = reinterpret_cast<const S*>(base[sg]);
    const float* ls = reinterpret_cast<const float*>(base[sg] + (size_t)M * W * sizeof(S));
    float d[Q], g[NSA][QS];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = dev_in<S>(P, i, to_f(fs[i * W + H + lx - L::ex(i)]));
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i) g[s][i] = to_f(fs[(Q + s * QS + i) * W + H + lx - LS::ex(i)]);
    const uint8_t type = flags[idx];
    const float cbar = stat_n != nullptr ? (float)(stat_n[0] * (double)P.inv_A_out) : 0.0f;
    auto load = [&](float* a, float (*b)[QS]) {
      if (has_next) {
#pragma unroll
        for (int i = 0; i < Q; ++i) a[i] = ls[i * WL + HL + lx + L::ex(i)];
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int i = 0; i < QS; ++i) b[s][i] = ls[(Q + s * QS + i) * WL + HL + lx + LS::ex(i)];
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
    Ops::reverse(P, type, theta[idx], y, d, g, load, ws, cbar, lam, lamg, dth);
#pragma unroll
    for (int i = 0; i < Q; ++i) st(lam_out + (long long)i * P.N + idx, lam[i]);
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i) st(lam_out + (long long)(Q + s * QS + i) * P.N + idx, lamg[s][i]);
    if (type == FLUID || type == INLET || type == OUTLET) grad[idx] += (double)dth;
    __syncthreads();  // the stage may be refilled from here on
  }
}

}  // namespace albm

// ---------------------------------------------------------------------------
// Variant staged with cp.async (16-byte copies issued by every thread of the
// block, completion tracked by commit/wait groups, no mbarrier waits).  The
// staged row segment and its halos are the same as above; each 16-byte
// chunk k of the segment [x0 - H, x0 + TX + H) of density m is one copy, the
// first and last chunk wrapping to the other end of the row when the tile
// touches it.
// ---------------------------------------------------------------------------
namespace albm {

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Issue the chunks of rows [0, nrows) of one stage: row r holds density
// row_m[r] from source row base row_base[r] (element offsets, wrap applied
// for y and z); every row is W = TX + 2H elements = TX/H + 2 chunks.
template <class T, int TX>
__device__ __forceinline__ void async_rows(T* dst, const T* src_base, const long long* row_base,
                                           int nrows, int x0, int Lx) {
  constexpr int H = 16 / (int)sizeof(T);
  constexpr int CH = TX / H + 2;  // chunks per row
  constexpr int W = TX + 2 * H;
  for (int c = threadIdx.x; c < nrows * CH; c += blockDim.x) {
    const int r = c / CH, k = c - r * CH;
    int xs = x0 - H + k * H;  // first element of the chunk
    if (xs < 0) xs += Lx;
    if (xs >= Lx) xs -= Lx;
    cp_async16(dst + r * W + k * H, src_base + row_base[r] + xs);
  }
}

template <class L, int NS, bool MRT, class S, int TX>
__global__ void __launch_bounds__(TX) primal_async_kernel(KParams P, const S* __restrict__ Bin,
                                                          S* __restrict__ Bout,
                                                          const float* __restrict__ theta,
                                                          const uint8_t* __restrict__ flags,
                                                          double* __restrict__ obj) {
  using Ops = NodeOps<L, NS, MRT>;
  using LS = typename Ops::LS;
  using Lay = TileLayout<L, NS, S, TX>;
  constexpr int Q = Ops::Q, QS = Ops::QS, NSA = Ops::NSA, M = Lay::M, H = Lay::H, W = Lay::W;
  extern __shared__ __align__(128) unsigned char smem[];
  long long* rbase = reinterpret_cast<long long*>(smem);                 // 2 x M row bases
  S* stage[2] = {reinterpret_cast<S*>(smem + Lay::header_async),
                 reinterpret_cast<S*>(smem + Lay::header_async + Lay::primal_stage)};
  const int Lx = P.nx;
  const int tiles_x = Lx / TX;
  const long long ntiles = (long long)tiles_x * P.ny * P.nz;
  auto bases = [&](long long t, int sg) {  // source row of every density
    const long long row = t / tiles_x;
    const int y = (int)(row % P.ny), z = (int)(row / P.ny);
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
      int ey = 0, ez = 0;
#pragma unroll
      for (int i = 0; i < M; ++i)
        if (i == m) {
          ey = i < Q ? L::ey(i) : LS::ey((i - Q) % QS);
          ez = i < Q ? L::ez(i) : LS::ez((i - Q) % QS);
        }
      const int ys = wrap(y - ey, P.ny), zs = wrap(z - ez, P.nz);
      rbase[sg * M + m] = (long long)m * P.N + ((long long)zs * P.ny + ys) * Lx;
    }
  };
  auto issue = [&](long long t, int sg) {
    const long long row = t / tiles_x;
    const int x0 = (int)(t - row * tiles_x) * TX;
    async_rows<S, TX>(stage[sg], Bin, rbase + sg * M, M, x0, Lx);
    cp_async_commit();
  };
  long long t = blockIdx.x;
  if (t < ntiles) {
    bases(t, 0);
    __syncthreads();
    issue(t, 0);
  }
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int sg = it & 1;
    const long long tn = t + gridDim.x;
    if (tn < ntiles) {
      bases(tn, sg ^ 1);
      __syncthreads();
      issue(tn, sg ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const long long row = t / tiles_x;
    const int x0 = (int)(t - row * tiles_x) * TX;
    const int y = (int)(row % P.ny);
    const int lx = threadIdx.x;
    const long long idx = row * Lx + x0 + lx;
    const S* sb = stage[sg];
    float d[Q], g[NSA][QS];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float raw = to_f(sb[i * W + H + lx - L::ex(i)]);
      d[i] = fold_offsets<S>() ? raw : dev_in<S>(P, i, raw);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i) g[s][i] = to_f(sb[(Q + s * QS + i) * W + H + lx - LS::ex(i)]);
    double o1 = 0.0, o2 = 0.0;
    Ops::template forward<2, fold_offsets<S>()>(P, flags[idx], theta[idx], y, d, g, obj != nullptr,
                                                o1, o2);
#pragma unroll
    for (int i = 0; i < Q; ++i)
      st(Bout + (long long)i * P.N + idx, fold_offsets<S>() ? d[i] : dev_out<S>(P, i, d[i]));
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i) st(Bout + (long long)(Q + s * QS + i) * P.N + idx, g[s][i]);
    if (obj != nullptr) block_partial2(o1, o2, obj + 2 * t);
    __syncthreads();  // the stage may be refilled from here on
  }
}

template <class L, int NS, bool MRT, class S, int TX>
__global__ void __launch_bounds__(TX) adjoint_async_kernel(
    KParams P, const float* __restrict__ lam_in, const S* __restrict__ Bn,
    float* __restrict__ lam_out, const float* __restrict__ theta, const uint8_t* __restrict__ flags,
    double* __restrict__ grad, float ws, const double* __restrict__ stat_n, int has_next) {
  using Ops = NodeOps<L, NS, MRT>;
  using LS = typename Ops::LS;
  using Lay = TileLayout<L, NS, S, TX>;
  constexpr int Q = Ops::Q, QS = Ops::QS, NSA = Ops::NSA, M = Lay::M, H = Lay::H, W = Lay::W;
  constexpr int HL = Lay::HL, WL = Lay::WL;
  extern __shared__ __align__(128) unsigned char smem[];
  long long* rbase = reinterpret_cast<long long*>(smem);  // 2 stages x (M f-rows + M lambda-rows)
  unsigned char* base[2] = {smem + Lay::header_async, smem + Lay::header_async + Lay::adjoint_stage};
  const int Lx = P.nx;
  const int tiles_x = Lx / TX;
  const long long ntiles = (long long)tiles_x * P.ny * P.nz;
  auto bases = [&](long long t, int sg) {
    const long long row = t / tiles_x;
    const int y = (int)(row % P.ny), z = (int)(row / P.ny);
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
      int ey = 0, ez = 0;
#pragma unroll
      for (int i = 0; i < M; ++i)
        if (i == m) {
          ey = i < Q ? L::ey(i) : LS::ey((i - Q) % QS);
          ez = i < Q ? L::ez(i) : LS::ez((i - Q) % QS);
        }
      rbase[sg * 2 * M + m] =
          (long long)m * P.N + ((long long)wrap(z - ez, P.nz) * P.ny + wrap(y - ey, P.ny)) * Lx;
      rbase[sg * 2 * M + M + m] =
          (long long)m * P.N + ((long long)wrap(z + ez, P.nz) * P.ny + wrap(y + ey, P.ny)) * Lx;
    }
  };
  auto issue = [&](long long t, int sg) {
    const long long row = t / tiles_x;
    const int x0 = (int)(t - row * tiles_x) * TX;
    S* fs = reinterpret_cast<S*>(base[sg]);
    float* ls = reinterpret_cast<float*>(base[sg] + (size_t)M * W * sizeof(S));
    async_rows<S, TX>(fs, Bn, rbase + sg * 2 * M, M, x0, Lx);
    if (has_next) async_rows<float, TX>(ls, lam_in, rbase + sg * 2 * M + M, M, x0, Lx);
    cp_async_commit();
  };
  long long t = blockIdx.x;
  if (t < ntiles) {
    bases(t, 0);
    __syncthreads();
    issue(t, 0);
  }
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int sg = it & 1;
    const long long tn = t + gridDim.x;
    if (tn < ntiles) {
      bases(tn, sg ^ 1);
      __syncthreads();
      issue(tn, sg ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const long long row = t / tiles_x;
    const int x0 = (int)(t - row * tiles_x) * TX;
    const int y = (int)(row % P.ny);
    const int lx = threadIdx.x;
    const long long idx = row * Lx + x0 + lx;
    const S* fs = reinterpret_cast<const S*>(base[sg]);
    const float* ls = reinterpret_cast<const float*>(base[sg] + (size_t)M * W * sizeof(S));
    float d[Q], g[NSA][QS];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = dev_in<S>(P, i, to_f(fs[i * W + H + lx - L::ex(i)]));
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i) g[s][i] = to_f(fs[(Q + s * QS + i) * W + H + lx - LS::ex(i)]);
    const uint8_t type = flags[idx];
    const float cbar = stat_n != nullptr ? (float)(stat_n[0] * (double)P.inv_A_out) : 0.0f;
    auto load = [&](float* a, float (*b)[QS]) {
      if (has_next) {
#pragma unroll
        for (int i = 0; i < Q; ++i) a[i] = ls[i * WL + HL + lx + L::ex(i)];
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int i = 0; i < QS; ++i) b[s][i] = ls[(Q + s * QS + i) * WL + HL + lx + LS::ex(i)];
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
    Ops::reverse(P, type, theta[idx], y, d, g, load, ws, cbar, lam, lamg, dth);
#pragma unroll
    for (int i = 0; i < Q; ++i) st(lam_out + (long long)i * P.N + idx, lam[i]);
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i) st(lam_out + (long long)(Q + s * QS + i) * P.N + idx, lamg[s][i]);
    if (type == FLUID || type == INLET || type == OUTLET) grad[idx] += (double)dth;
    __syncthreads();  // the stage may be refilled from here on
  }
}

}  // namespace albm
