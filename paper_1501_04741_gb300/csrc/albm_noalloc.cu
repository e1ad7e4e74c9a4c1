// lbm_state_objective_noalloc: the objective F(f) of one caller-provided
// state, evaluated without allocating device memory.
//
// Why it exists.  Some callers cannot call cudaMalloc at the moment they
// need an objective value: a serving process whose device memory is fully
// reserved in advance for resident states (an extra allocation would fail,
// or would take memory promised to a request), plugins inside a host
// framework that owns the device allocator and forbids allocations behind
// its back (they would fragment the framework's pool and make its own later
// allocations fail), and code that must not pay the device-wide
// synchronisation that cudaFree implies while other streams run.  This
// entry point therefore uses a fixed scratch array in the library's own
// static device memory; the caller passes the inputs, and the result comes
// back in a host double (the call synchronises the given stream).
//
// Scratch.  g_noalloc_scratch below is a file-scope __device__ array of
// kNoAllocMaxBlocks * kSlots doubles plus one result row (about 1.5 MiB).
// Every GPU that loads the library holds it until the process exits.  It
// keeps per-block partial sums (pass 1) and the final sums (pass 2); every
// entry a call reads is written earlier in the same call, so nothing needs
// clearing, and the contents of the last call stay behind.  All calls share
// the one array: calls that overlap on the GPU (different streams, or
// different host threads on the same device) race on it and must be
// serialised by the caller.
//
// Host code may not hand the symbol itself to a kernel: in host code
// g_noalloc_scratch names a host-side stand-in, not a device address.  The
// first call on each device (with that device current) looks the device
// address up with cudaGetSymbolAddress, checks the result, caches it, and
// loads every kernel this file holds (so that later calls with another
// lattice or collision load nothing); it is the only call that does this
// set-up.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/albm.h"
#include "albm_kernels.cuh"

namespace {

constexpr int kNoAllocBlock = 256;
constexpr long long kNoAllocMaxBlocks = 32768;              // nodes <= 8,388,608
constexpr int kSlots = 6;                                    // doubles per block
constexpr long long kNoAllocMaxNodes = kNoAllocMaxBlocks * kNoAllocBlock;

// slots: 0 objective terms of non-inlet nodes, 1 second moment (variance),
//        2 objective terms of inlet nodes (scaled by 1, not 1/A_in),
//        3 inlet node count, 4 outlet node count, 5 unused
static __device__ __align__(256) double g_noalloc_scratch[(kNoAllocMaxBlocks + 1) * kSlots];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {nullptr};
thread_local std::string g_err;

template <class L, int NS, bool MRT>
__global__ void __launch_bounds__(kNoAllocBlock)
noalloc_pass1(albm::KParams P, const float* __restrict__ f, const float* __restrict__ theta,
              const uint8_t* __restrict__ flags, double* __restrict__ scratch) {
  using Ops = albm::NodeOps<L, NS, MRT>;
  using LS = typename Ops::LS;
  constexpr int Q = Ops::Q, QS = Ops::QS, NSA = Ops::NSA;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[kSlots] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (idx < P.N) {
    const uint8_t type = flags[idx];
    const int y = (int)((idx / P.nx) % P.ny);
    float d[Q], g[NSA][QS];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = f[(long long)i * P.N + idx] - L::w(i);
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < QS; ++i) g[s][i] = f[(long long)(Q + s * QS + i) * P.N + idx];
    double o1 = 0.0, o2 = 0.0;
    Ops::forward(P, type, theta[idx], y, d, g, true, o1, o2);
    if (type == albm::INLET) {
      v[2] = o1;
      v[3] = 1.0;
    } else {
      v[0] = o1;
      v[1] = o2;
      v[4] = (type == albm::OUTLET) ? 1.0 : 0.0;
    }
  }
  __shared__ double sh[kSlots][kNoAllocBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kSlots; ++k) {
    double a = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) sh[k][wid] = a;
  }
  __syncthreads();
  if (threadIdx.x < kSlots) {
    double a = 0.0;
    for (int w = 0; w < kNoAllocBlock / 32; ++w) a += sh[threadIdx.x][w];
    scratch[(long long)blockIdx.x * kSlots + threadIdx.x] = a;   // plain store: no clearing needed
  }
}

// one block: fixed-order sum of the per-block partials into the result row
__global__ void __launch_bounds__(kNoAllocBlock)
noalloc_pass2(double* __restrict__ scratch, long long nblocks) {
  __shared__ double sh[kSlots][kNoAllocBlock];
  double v[kSlots] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < kSlots; ++k) v[k] += scratch[b * kSlots + k];
#pragma unroll
  for (int k = 0; k < kSlots; ++k) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int s = kNoAllocBlock / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int k = 0; k < kSlots; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < kSlots) scratch[kNoAllocMaxBlocks * kSlots + threadIdx.x] = sh[threadIdx.x][0];
}

template <class L, int NS, bool MRT>
cudaError_t launch(const albm::KParams& P, const float* f, const float* theta,
                   const uint8_t* flags, double* scratch, cudaStream_t st) {
  const long long nb = (P.N + kNoAllocBlock - 1) / kNoAllocBlock;
  noalloc_pass1<L, NS, MRT><<<(unsigned)nb, kNoAllocBlock, 0, st>>>(P, f, theta, flags, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  noalloc_pass2<<<1, kNoAllocBlock, 0, st>>>(scratch, nb);
  return cudaGetLastError();
}

cudaError_t dispatch(const lbm_params& p, const albm::KParams& P, const float* f,
                     const float* theta, const uint8_t* flags, double* scratch, cudaStream_t st) {
  using namespace albm;
  const bool mrt = p.collision == LBM_MRT;
  if (p.lattice == LBM_D2Q9) {
    if (p.nscalars == 0) return mrt ? launch<D2Q9, 0, true>(P, f, theta, flags, scratch, st)
                                    : launch<D2Q9, 0, false>(P, f, theta, flags, scratch, st);
    return mrt ? launch<D2Q9, 1, true>(P, f, theta, flags, scratch, st)
               : launch<D2Q9, 1, false>(P, f, theta, flags, scratch, st);
  }
  switch (p.nscalars) {
    case 0: return mrt ? launch<D3Q19, 0, true>(P, f, theta, flags, scratch, st)
                       : launch<D3Q19, 0, false>(P, f, theta, flags, scratch, st);
    case 1: return mrt ? launch<D3Q19, 1, true>(P, f, theta, flags, scratch, st)
                       : launch<D3Q19, 1, false>(P, f, theta, flags, scratch, st);
    default: return mrt ? launch<D3Q19, 2, true>(P, f, theta, flags, scratch, st)
                        : launch<D3Q19, 2, false>(P, f, theta, flags, scratch, st);
  }
}

// With lazy module loading a kernel is loaded on its first launch, which
// may allocate device memory; querying the attributes of every kernel of
// this file loads them all up front, on the current device.
cudaError_t load_all_kernels() {
  using namespace albm;
  cudaFuncAttributes a;
  const void* k[] = {
      (const void*)noalloc_pass1<D2Q9, 0, false>,  (const void*)noalloc_pass1<D2Q9, 0, true>,
      (const void*)noalloc_pass1<D2Q9, 1, false>,  (const void*)noalloc_pass1<D2Q9, 1, true>,
      (const void*)noalloc_pass1<D3Q19, 0, false>, (const void*)noalloc_pass1<D3Q19, 0, true>,
      (const void*)noalloc_pass1<D3Q19, 1, false>, (const void*)noalloc_pass1<D3Q19, 1, true>,
      (const void*)noalloc_pass1<D3Q19, 2, false>, (const void*)noalloc_pass1<D3Q19, 2, true>,
      (const void*)noalloc_pass2};
  for (const void* f : k) {
    cudaError_t e = cudaFuncGetAttributes(&a, f);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

lbm_status fail(lbm_status code, const std::string& msg) {
  g_err = msg;
  return code;
}

}  // namespace

extern "C" const char* lbm_noalloc_last_error(void) { return g_err.c_str(); }

extern "C" lbm_status lbm_state_objective_noalloc(const lbm_params* pp, const float* f,
                                                  const float* theta, const uint8_t* flags,
                                                  void* stream, double* F_host) {
  if (!pp || !f || !theta || !flags || !F_host) return fail(LBM_ERR_ARG, "null argument");
  const lbm_params& p = *pp;
  if (p.lattice != LBM_D2Q9 && p.lattice != LBM_D3Q19)
    return fail(LBM_ERR_ARG, "lattice must be D2Q9 or D3Q19");
  if (p.nx < 1 || p.ny < 1 || p.nz < 1 || (p.lattice == LBM_D2Q9 && p.nz != 1))
    return fail(LBM_ERR_ARG, "bad lattice sizes");
  if (p.nscalars < 0 || p.nscalars > (p.lattice == LBM_D3Q19 ? 2 : 1))
    return fail(LBM_ERR_ARG, "nscalars out of range");
  if (!(p.tau > 0.5) || p.objective < LBM_OBJ_DISSIPATION || p.objective > LBM_OBJ_HEATFLUX)
    return fail(LBM_ERR_ARG, "tau must exceed 1/2 and an objective must be set");
  if (p.objective >= LBM_OBJ_VARIANCE && (p.nscalars < 1 || !p.inlet_outlet))
    return fail(LBM_ERR_ARG, "outlet objectives need a scalar lattice and inlet_outlet");
  if (p.inlet_outlet && (p.nx < 3 || !(p.u_in < 1.0) || !(p.rho_out > 0.0)))
    return fail(LBM_ERR_ARG, "inlet_outlet needs nx >= 3, u_in < 1 and rho_out > 0");
  if (p.porosity < 0 || p.porosity > 2) return fail(LBM_ERR_ARG, "unknown porosity law");
  if (p.inlet_kind < 0 || p.inlet_kind > 1 ||
      (p.inlet_kind == 1 && !(p.rho_out + 3.0 * p.dp > 0.0)))
    return fail(LBM_ERR_ARG, "bad inlet kind or pressure drop");
  if (p.scalar_inlet < 0 || p.scalar_inlet > 2)
    return fail(LBM_ERR_ARG, "unknown scalar inlet profile");
  const long long N = (long long)p.nx * p.ny * p.nz;
  if (N > kNoAllocMaxNodes) {
    char b[160];
    snprintf(b, sizeof(b), "lattice of %lld nodes exceeds the no-alloc limit of %lld nodes", N,
             kNoAllocMaxNodes);
    return fail(LBM_ERR_ARG, b);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(LBM_ERR_ARG, "device index out of range");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);   // device address, this device
      if (e != cudaSuccess)
        return fail(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      e = load_all_kernels();
      if (e != cudaSuccess)
        return fail(LBM_ERR_CUDA, std::string("loading the kernels: ") + cudaGetErrorString(e));
      g_dev_ptr[dev] = (double*)ptr;
    }
    scratch = g_dev_ptr[dev];
  }
  albm::KParams P{};
  P.nx = p.nx;
  P.ny = p.ny;
  P.nz = p.nz;
  P.nscal = p.nscalars;
  P.N = N;
  P.fd_nx = albm::make_fastdiv((unsigned)p.nx);
  P.fd_ny = albm::make_fastdiv((unsigned)p.ny);
  P.fd_hx = albm::make_fastdiv((unsigned)(p.nx / 2 > 0 ? p.nx / 2 : 1));
  const double omega = 1.0 / p.tau;
  P.omega = (float)omega;
  P.one_m_omega = (float)(1.0 - omega);
  P.nu = (float)((p.tau - 0.5) / 3.0);
  P.gx = (float)p.force[0];
  P.gy = (float)p.force[1];
  P.gz = (float)p.force[2];
  P.u_in = (float)p.u_in;
  P.inv_1m_uin = (float)(1.0 / (1.0 - p.u_in));
  P.rho_out = (float)p.rho_out;
  P.drho_out = (float)(p.rho_out - 1.0);
  P.one_m_rho_out = (float)(1.0 - p.rho_out);
  P.inlet_kind = p.inlet_kind;
  P.rho_in = (float)(p.rho_out + 3.0 * p.dp);
  P.drho_in = (float)(p.rho_out + 3.0 * p.dp - 1.0);
  P.inv_rho_in = (float)(1.0 / (p.rho_out + 3.0 * p.dp));
  P.alpha_f = (float)p.alpha_fluid;
  P.alpha_s = (float)p.alpha_solid;
  P.porosity = p.porosity;
  P.por_q = (float)p.porosity_q;
  P.scalar_inlet = p.scalar_inlet;
  P.T_hot = (float)p.T_hot;
  P.objective = p.objective;
  P.inv_A_in = 1.0f;   // inlet terms are summed unscaled and divided by the count below
  P.inv_A_out = 0.0f;
  if (p.collision == LBM_MRT) {
    if (p.lattice == LBM_D3Q19) albm::fill_mrt<albm::D3Q19>(omega, p.s_other, P);
    else albm::fill_mrt<albm::D2Q9>(omega, p.s_other, P);
  }
  cudaStream_t st = (cudaStream_t)stream;
  e = dispatch(p, P, f, theta, flags, scratch, st);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  double s[kSlots];
  e = cudaMemcpyAsync(s, scratch + kNoAllocMaxBlocks * kSlots, sizeof(s), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("readback: ") + cudaGetErrorString(e));
  const double n_in = s[3], n_out = s[4];
  double F = 0.0;
  switch (p.objective) {
    case LBM_OBJ_VARIANCE: {
      const double A = n_out > 0 ? n_out : 1.0;
      const double m = s[0] / A;
      F = s[1] / A - m * m;
      break;
    }
    case LBM_OBJ_HEATFLUX_DP:
      F = s[0] + (n_in > 0 ? s[2] / n_in : 0.0) + 0.1 * p.rho_out / 3.0;
      break;
    default:
      F = s[0];
  }
  *F_host = F;
  return LBM_OK;
}
