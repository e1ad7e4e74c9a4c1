// Host runtime of libalbm.so: the C ABI declared in include/albm.h.
//
// A handle owns the device state of one problem:
//   * flags (uint8, N), theta (FP32, N), the FP64 gradient (N) and the
//     per-step objective record (FP64, 2 per step),
//   * a pool of state buffers B^n (M x N in the storage precision), indexed
//     by the time n they hold.  The primal kernel writes each new state into
//     a pool buffer, so keeping a state for the adjoint costs no copy,
//   * two FP32 adjoint buffers (lambda^{n+1} -> lambda^n ping-pong).
//
// Checkpoint schedule of the unsteady adjoint.  The primal pass keeps f^n
// at every multiple of the level-1 stride K.  When the adjoint needs f^n
// and it is not kept, the runtime recomputes forward from the latest kept
// state c < n: if the n - c states fit in the free buffers it keeps them
// all, otherwise it keeps the densest tail ending at n that fits (and, when
// even that would leave a head longer than the tail, sub-checkpoints spread
// over the head); each later request then recomputes a shorter span.  Kept
// states newer than the adjoint time are released as the adjoint passes
// them, so the pool never needs more than its budget.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <set>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/albm.h"
#include "albm_kernels.cuh"

using albm::KernelSet;
using albm::KParams;
using albm::StepArgs;

struct lbm_ctx {
  lbm_params p{};
  KParams kp{};
  KernelSet ks{};
  int Q = 0, QS = 0, M = 0;
  long long N = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  uint8_t* flags = nullptr;
  float* theta = nullptr;
  double* grad = nullptr;
  double* stats = nullptr;          // 2 doubles per step 0..nsteps
  double* partials = nullptr;       // 2 doubles per block (or tile) of one launch
  long long nblocks = 0;            // blocks of the one-thread-per-node kernels
  long long ntiles = 0;             // tiles of the staged kernels
  int staged = 0;                   // 0: per-node kernels; 2: TMA-staged; 3: cp.async-staged
  int* d_err = nullptr;             // bounded-wait failure flag of staged kernels
  unsigned long long* counter = nullptr;
  float* lam[2] = {nullptr, nullptr};
  int lam_cur = 0;
  size_t state_bytes = 0;
  size_t state_stride = 0;          // state_bytes rounded up to 256
  int slab_states = 1;              // most states per allocation
  std::vector<void*> slabs;         // the allocations holding the states
  char* slab_next = nullptr;
  int slab_left = 0;
  std::vector<void*> bufs;
  std::vector<int> buf_time;        // per buffer: time held, -1 free, -2 reserved
  std::vector<int> time_buf;        // per time 0..nsteps: the buffer holding it, or -1
  std::vector<int> free_bufs;       // buffers that became free (stack)
  std::set<int> held;               // times held
  std::set<int> evictable;          // held times that are not level-1 checkpoints
  int max_bufs = 3;
  int ckpt = 1;                     // level-1 stride
  int t = 0;                        // primal time
  int t_adj = -1;                   // adjoint time (-1: not started)
  int n_in = 0, n_out = 0;
  std::vector<double> c;            // time weights c_n
  std::vector<uint8_t> flags_host;
  // profiling: events around launches, grouped by kind
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_used;   // (kind, first event index)
  size_t ev_next = 0;
  cudaEvent_t t0 = nullptr, t1 = nullptr, t2 = nullptr, t3 = nullptr;
  float last_primal_ms = 0.f, last_adjoint_ms = 0.f;
  bool primal_timed = false, adjoint_timed = false;
  long long recompute_steps = 0;
  long long launches_other = 0;     // objective / fold / import / export kernels
  // one-shot optimisation: the current state is the pool buffer labelled 0
  bool oneshot = false;
  uint8_t* design = nullptr;        // design mask (device, N); null until first use
  bool design_default = true;       // mask = FLUID nodes
  double* os_stats = nullptr;       // objective record of the current state (2 doubles)
  float* theta_saved = nullptr;     // continuous design during a threshold scan
  // MMA history: x^{k-1}, x^{k-2}, last asymptotes (FP32, N each)
  float* mma_hist = nullptr;
  int mma_k = -1;                   // -1: lbm_mma_reset not called
  // fixed-point ALBS at the held state (adjoint_mode 1): iterations done
  int frozen_k = 0;
  bool frozen_seeded = false;       // v^0 given by lbm_adjoint_seed (else 0)
  std::string err;
};

static const char* kNoHandle = "null handle";

#define FAIL(h, code, ...)                                   \
  do {                                                       \
    char _b[512];                                            \
    snprintf(_b, sizeof(_b), __VA_ARGS__);                   \
    (h)->err = _b;                                           \
    return code;                                             \
  } while (0)

#define CK(h, call)                                                               \
  do {                                                                            \
    cudaError_t _e = (call);                                                      \
    if (_e != cudaSuccess) {                                                      \
      FAIL(h, _e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,       \
           "%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__, __LINE__); \
    }                                                                             \
  } while (0)

namespace {

enum { K_PRIMAL = 0, K_RECOMPUTE = 1, K_ADJOINT = 2, K_OTHER = 3 };

int scalar_q(int lattice) { return lattice == LBM_D3Q19 ? 7 : 9; }
int fluid_q(int lattice) { return lattice == LBM_D3Q19 ? 19 : 9; }

// node types of the channel geometry: inlet/outlet faces, then wall planes
// (box edges are walls), then the hot patch on the y = 0 plane
void build_flags(const lbm_params& p, std::vector<uint8_t>& fl) {
  const long long nx = p.nx, ny = p.ny, nz = p.nz;
  fl.assign((size_t)(nx * ny * nz), (uint8_t)LBM_NODE_FLUID);
  for (long long z = 0; z < nz; ++z)
    for (long long y = 0; y < ny; ++y)
      for (long long x = 0; x < nx; ++x) {
        uint8_t t = LBM_NODE_FLUID;
        if (p.inlet_outlet) {
          if (x == 0) t = LBM_NODE_INLET;
          if (x == nx - 1) t = LBM_NODE_OUTLET;
        }
        if ((p.walls & 1) && (y == 0 || y == ny - 1)) t = LBM_NODE_WALL;
        if ((p.walls & 2) && (z == 0 || z == nz - 1)) t = LBM_NODE_WALL;
        if (p.hot[1] > p.hot[0] && y == 0 && x >= p.hot[0] && x < p.hot[1] && z >= p.hot[2] &&
            z < p.hot[3])
          t = LBM_NODE_HOT;
        fl[(size_t)(x + nx * (y + ny * z))] = t;
      }
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// ---------------------------------------------------------------------------
// buffer pool
// ---------------------------------------------------------------------------
// Every change of a buffer's label goes through set_time, which keeps the
// time -> buffer index, the sets of held and evictable times and the stack
// of free buffers in step, so that every lookup of a step is O(1) or
// O(log n) in the number of held states (a linear scan per step would make
// a long horizon quadratic on the host).
static void set_time(lbm_ctx* h, int b, int t) {
  const int old = h->buf_time[b];
  if (old == t) return;
  if (old >= 0) {
    h->time_buf[old] = -1;
    h->held.erase(old);
    h->evictable.erase(old);
  }
  h->buf_time[b] = t;
  if (t >= 0) {
    h->time_buf[t] = b;
    h->held.insert(t);
    if (t % h->ckpt != 0) h->evictable.insert(t);
  } else if (t == -1) {
    h->free_bufs.push_back(b);
  }
}

static void reset_pool(lbm_ctx* h) {
  for (size_t b = 0; b < h->bufs.size(); ++b) set_time(h, (int)b, -1);
}

static int find_buf(lbm_ctx* h, int t) {
  return (t >= 0 && t < (int)h->time_buf.size()) ? h->time_buf[t] : -1;
}

static int n_kept(lbm_ctx* h) { return (int)h->held.size(); }

// a free buffer, reserved (-2) for the caller, or -1
static int pop_free(lbm_ctx* h) {
  while (!h->free_bufs.empty()) {
    const int b = h->free_bufs.back();
    h->free_bufs.pop_back();
    if (h->buf_time[b] == -1) {
      set_time(h, b, -2);
      return b;
    }
  }
  return -1;
}

// A buffer reserved (-2) for the caller, who labels it with set_time.
static lbm_status acquire(lbm_ctx* h, int* out) {
  const int fb = pop_free(h);
  if (fb >= 0) {
    *out = fb;
    return LBM_OK;
  }
  if ((int)h->bufs.size() >= h->max_bufs)
    FAIL(h, LBM_ERR_OOM, "state pool exhausted (%d buffers of %zu bytes)", h->max_bufs,
         h->state_bytes);
  if (h->slab_left == 0) {
    // the pool grows by slabs of several states: as many as it holds
    // already (at least 4), at most about 1 GiB and never past the budget,
    // so that a long trajectory costs a few dozen allocations, and freeing
    // the pool (cudaFree synchronises the device) a few dozen frees
    const int held = (int)h->bufs.size();
    int n = std::max(4, held);
    n = std::min(n, h->slab_states);
    n = std::min(n, h->max_bufs - held);
    void* slab = nullptr;
    CK(h, cudaMalloc(&slab, (size_t)n * h->state_stride));
    h->slabs.push_back(slab);
    h->slab_next = (char*)slab;
    h->slab_left = n;
  }
  void* p = h->slab_next;
  h->slab_next += h->state_stride;
  h->slab_left--;
  h->bufs.push_back(p);
  h->buf_time.push_back(-2);
  *out = (int)h->bufs.size() - 1;
  return LBM_OK;
}

// Forward pass: a free buffer, a new one while the pool is below its
// budget, else the buffer of the oldest kept state that is neither a level-1
// checkpoint nor `keep`.  The forward pass thus leaves the most recent states
// in the pool, which the adjoint needs first, instead of recomputing them.
static lbm_status acquire_evict(lbm_ctx* h, int keep, int* out) {
  const int fb = pop_free(h);
  if (fb >= 0) {
    *out = fb;
    return LBM_OK;
  }
  if ((int)h->bufs.size() < h->max_bufs) return acquire(h, out);
  auto it = h->evictable.begin();
  if (it != h->evictable.end() && *it == keep) ++it;
  if (it == h->evictable.end())
    FAIL(h, LBM_ERR_OOM, "state pool exhausted by checkpoints (%d buffers of %zu bytes)",
         h->max_bufs, h->state_bytes);
  const int best = h->time_buf[*it];
  set_time(h, best, -2);
  *out = best;
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// profiling events
// ---------------------------------------------------------------------------
static void prof_begin(lbm_ctx* h, int kind, int* slot) {
  *slot = -1;
  if (!h->profile) return;
  if (h->ev_next + 2 > h->ev_pool.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      h->ev_pool.push_back(e);
    }
  }
  *slot = (int)h->ev_next;
  h->ev_next += 2;
  cudaEventRecord(h->ev_pool[*slot], h->stream);
  h->ev_used.push_back({kind, *slot});
}

static void prof_end(lbm_ctx* h, int slot) {
  if (slot >= 0) cudaEventRecord(h->ev_pool[slot + 1], h->stream);
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
static StepArgs blank_args(lbm_ctx* h) {
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.theta = h->theta;
  a.flags = h->flags;
  return a;
}

namespace albm {
__global__ void __launch_bounds__(1024) fold_partials_kernel(const double* __restrict__ partials,
                                                             long long nblocks,
                                                             double* __restrict__ out) {
  __shared__ double sh[2][1024];
  double a = 0.0, b = 0.0;
  for (long long i = threadIdx.x; i < nblocks; i += blockDim.x) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sh[0][0];
    out[1] = sh[1][0];
  }
}

// ---- one-shot optimisation (Sec. 3.3) --------------------------------------
// per-block sums of theta (1 - theta) over design nodes (P of Eq. P)
__global__ void __launch_bounds__(256) penalty_kernel(long long N, const float* __restrict__ theta,
                                                      const uint8_t* __restrict__ design,
                                                      double* __restrict__ partials) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < N && design[i]) {
    const double t = (double)theta[i];
    v = t * (1.0 - t);
  }
  block_partial2(v, 0.0, partials + 2 * (long long)blockIdx.x);
}

// threshold of Sec. 3.2: w = 1 - theta below eta -> solid (theta = 1), else
// fluid (theta = 0), in FP32, on design nodes; other nodes copied
__global__ void __launch_bounds__(256) threshold_kernel(long long N, const float* __restrict__ src,
                                                        float* __restrict__ dst,
                                                        const uint8_t* __restrict__ design,
                                                        float eta) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float t = src[i];
  dst[i] = design[i] ? ((1.0f - t < eta) ? 1.0f : 0.0f) : t;
}

// One MMA iteration per design node (Svanberg's method, box 0..1, no other
// constraints; the steps and constants of lbm_mma_update): asymptotes from
// the last two changes, move limits, and the minimiser of the convex
// separable approximation.  FP32; sign = -1 turns a maximised J into f = -J.
__global__ void __launch_bounds__(256) mma_update_kernel(long long N, float* __restrict__ theta,
                                                         float* __restrict__ x1,
                                                         float* __restrict__ x2,
                                                         float* __restrict__ Lh,
                                                         float* __restrict__ Uh,
                                                         const double* __restrict__ grad,
                                                         const uint8_t* __restrict__ design,
                                                         int k, float sign, float move) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || !design[i]) return;
  const float x = theta[i];
  const float g = sign * (float)grad[i];
  float l, u;
  if (k < 2) {
    l = x - 0.5f;
    u = x + 0.5f;
  } else {
    const float xa = x1[i], xb = x2[i];
    const float d1 = x - xa, d2 = xa - xb;   // exact signs (differences of FP32 values)
    float gamma = 1.0f;
    if ((d1 > 0.0f && d2 < 0.0f) || (d1 < 0.0f && d2 > 0.0f)) gamma = 0.7f;
    else if ((d1 > 0.0f && d2 > 0.0f) || (d1 < 0.0f && d2 < 0.0f)) gamma = 1.2f;
    const float dl = fminf(fmaxf(gamma * (xa - Lh[i]), 0.01f), 10.0f);
    const float du = fminf(fmaxf(gamma * (Uh[i] - xa), 0.01f), 10.0f);
    l = x - dl;
    u = x + du;
  }
  const float alpha = fmaxf(fmaxf(0.0f, l + 0.1f * (x - l)), x - move);
  const float beta = fminf(fminf(1.0f, u - 0.1f * (u - x)), x + move);
  const float gp = fmaxf(g, 0.0f), gm = fmaxf(-g, 0.0f);
  const float p = (u - x) * (u - x) * (1.001f * gp + 0.001f * gm + 1e-5f);
  const float q = (x - l) * (x - l) * (0.001f * gp + 1.001f * gm + 1e-5f);
  const float sp = sqrtf(p), sq = sqrtf(q);
  const float y = (sp * l + sq * u) / (sp + sq);
  x2[i] = x1[i];
  x1[i] = x;
  Lh[i] = l;
  Uh[i] = u;
  theta[i] = fminf(fmaxf(y, alpha), beta);
}

// default design mask: FLUID nodes
__global__ void __launch_bounds__(256) fluid_mask_kernel(long long N, const uint8_t* __restrict__ flags,
                                                         uint8_t* __restrict__ design) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) design[i] = flags[i] == FLUID ? 1 : 0;
}
}  // namespace albm

// the runtime's own kernels, loaded once per device (see Launch::preload)
static cudaError_t preload_runtime_kernels() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load() & bit) return cudaSuccess;
  cudaFuncAttributes fa;
  const void* ks[] = {(const void*)albm::fold_partials_kernel, (const void*)albm::penalty_kernel,
                      (const void*)albm::threshold_kernel, (const void*)albm::mma_update_kernel,
                      (const void*)albm::fluid_mask_kernel};
  for (const void* k : ks) {
    e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
  }
  done.fetch_or(bit);
  return cudaSuccess;
}

// after a synchronisation: report an expired bounded wait of a staged kernel
static lbm_status check_timeout(lbm_ctx* h) {
  if (!h->d_err) return LBM_OK;
  int v = 0;
  CK(h, cudaMemcpy(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) {
    cudaMemset(h->d_err, 0, sizeof(int));
    FAIL(h, LBM_ERR_TIMEOUT, "a staged kernel's bounded wait for its shared-memory copies expired");
  }
  return LBM_OK;
}

// fold the per-block partials of step t into the objective record
static lbm_status fold_objective(lbm_ctx* h, int t, long long count) {
  albm::fold_partials_kernel<<<1, 1024, 0, h->stream>>>(h->partials, count,
                                                         h->stats + 2 * (size_t)t);
  h->launches_other++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) FAIL(h, LBM_ERR_CUDA, "objective fold launch: %s", cudaGetErrorString(e));
  return LBM_OK;
}

// one primal step from the state kept at time t (buffer src) into buffer dst
static lbm_status launch_primal(lbm_ctx* h, int src, int dst, int t, bool record, int kind) {
  StepArgs a = blank_args(h);
  a.Bin = h->bufs[src];
  a.Bout = h->bufs[dst];
  a.obj = (record && t <= h->p.nsteps && h->c[t] != 0.0) ? h->partials : nullptr;
  a.err = h->d_err;
  int slot;
  prof_begin(h, kind, &slot);
  cudaError_t e = h->staged == 2   ? h->ks.primal_tiles(h->kp, a, h->stream)
                  : h->staged == 3 ? h->ks.primal_async(h->kp, a, h->stream)
                                   : h->ks.primal(h->kp, a, h->stream);
  prof_end(h, slot);
  if (e != cudaSuccess) FAIL(h, LBM_ERR_CUDA, "primal kernel launch: %s", cudaGetErrorString(e));
  if (a.obj) return fold_objective(h, t, h->staged ? h->ntiles : h->ks.primal_partials(h->kp));
  return LBM_OK;
}

static lbm_status record_final_objective(lbm_ctx* h) {
  const int t = h->t;
  if (t > h->p.nsteps || h->c[t] == 0.0 || h->p.objective == LBM_OBJ_NONE) return LBM_OK;
  StepArgs a = blank_args(h);
  a.Bin = h->bufs[find_buf(h, t)];
  a.obj = h->partials;
  cudaError_t e = h->ks.objective(h->kp, a, h->stream);
  h->launches_other++;
  if (e != cudaSuccess) FAIL(h, LBM_ERR_CUDA, "objective kernel launch: %s", cudaGetErrorString(e));
  return fold_objective(h, t, h->nblocks);
}

// make f^n available in the pool (recompute from the latest kept state < n)
static lbm_status ensure_state(lbm_ctx* h, int n) {
  if (find_buf(h, n) >= 0) return LBM_OK;
  auto it = h->held.lower_bound(n);
  if (it == h->held.begin()) FAIL(h, LBM_ERR_STATE, "no kept state before time %d", n);
  --it;
  const int c = *it, cb = h->time_buf[c];
  const int L = n - c;
  const int free_now = h->max_bufs - n_kept(h);
  // states to keep on this pass
  std::vector<char> keep((size_t)L + 1, 0);  // keep[k] for time c + k
  if (L <= free_now) {
    for (int k = 1; k <= L; ++k) keep[k] = 1;
  } else {
    const int slots = free_now - 2;  // two scratch buffers for states not kept
    if (slots < 1) FAIL(h, LBM_ERR_OOM, "state pool too small to recompute (free %d)", free_now);
    const int head = L - slots;
    if (head <= slots) {
      for (int k = L - slots + 1; k <= L; ++k) keep[k] = 1;  // dense tail
    } else {
      const int stride = (L + slots - 1) / slots;  // sub-checkpoints
      for (int k = stride; k < L; k += stride) keep[k] = 1;
      keep[L] = 1;
    }
  }
  int cur = cb;
  int scratch[2] = {-1, -1};
  // on failure the scratch buffers go back to the pool (kept states stay valid)
  auto release = [&](lbm_status s) {
    for (int j = 0; j < 2; ++j)
      if (scratch[j] >= 0 && h->buf_time[scratch[j]] == -2) set_time(h, scratch[j], -1);
    return s;
  };
  for (int k = 1; k <= L; ++k) {
    int dst;
    if (keep[k]) {
      lbm_status s = acquire(h, &dst);
      if (s) return release(s);
    } else {
      // a scratch buffer that is not the source
      int pick = -1;
      for (int j = 0; j < 2; ++j)
        if (scratch[j] >= 0 && scratch[j] != cur) pick = scratch[j];
      if (pick < 0) {
        lbm_status s = acquire(h, &pick);   // reserved (-2) as scratch
        if (s) return release(s);
        if (scratch[0] < 0) scratch[0] = pick; else scratch[1] = pick;
      }
      dst = pick;
    }
    lbm_status s = launch_primal(h, cur, dst, c + k - 1, false, K_RECOMPUTE);
    if (s) return release(s);
    h->recompute_steps++;
    set_time(h, dst, keep[k] ? c + k : -2);
    cur = dst;
  }
  for (int j = 0; j < 2; ++j)
    if (scratch[j] >= 0 && h->buf_time[scratch[j]] == -2) set_time(h, scratch[j], -1);
  return LBM_OK;
}

static lbm_status launch_adjoint(lbm_ctx* h, int n, int has_next) {
  StepArgs a = blank_args(h);
  a.Bin = h->bufs[find_buf(h, n)];
  a.lam_in = h->lam[h->lam_cur];
  a.lam_out = h->lam[1 - h->lam_cur];
  a.grad = h->grad;
  a.ws = (float)h->c[n];
  a.stat_n = (h->p.objective == LBM_OBJ_VARIANCE && h->c[n] != 0.0) ? h->stats + 2 * (size_t)n
                                                                     : nullptr;
  a.has_next = has_next;
  a.err = h->d_err;
  int slot;
  prof_begin(h, K_ADJOINT, &slot);
  cudaError_t e = h->staged == 2   ? h->ks.adjoint_tiles(h->kp, a, h->stream)
                  : h->staged == 3 ? h->ks.adjoint_async(h->kp, a, h->stream)
                                   : h->ks.adjoint(h->kp, a, h->stream);
  prof_end(h, slot);
  if (e != cudaSuccess) FAIL(h, LBM_ERR_CUDA, "adjoint kernel launch: %s", cudaGetErrorString(e));
  h->lam_cur = 1 - h->lam_cur;
  return LBM_OK;
}

static lbm_status do_reset(lbm_ctx* h) {
  h->oneshot = false;
  reset_pool(h);
  int b;
  lbm_status s = acquire(h, &b);
  if (s) return s;
  if (h->ks.storage_bytes == 4) {
    CK(h, cudaMemsetAsync(h->bufs[b], 0, h->state_bytes, h->stream));  // f^0 = rest state
  } else {
    StepArgs a = blank_args(h);   // rest state relative to the reference offsets
    a.Bout = h->bufs[b];
    CK(h, h->ks.rest(h->kp, a, h->stream));
    h->launches_other++;
  }
  set_time(h, b, 0);
  h->t = 0;
  h->t_adj = -1;
  h->recompute_steps = 0;
  CK(h, cudaMemsetAsync(h->stats, 0, sizeof(double) * 2 * (size_t)(h->p.nsteps + 1), h->stream));
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* lbm_last_error(lbm_handle h) { return h ? h->err.c_str() : kNoHandle; }

lbm_status lbm_create(lbm_handle* out, const lbm_params* pp, const float* theta,
                      const uint8_t* flags, void* stream) {
  if (!out || !pp) return LBM_ERR_ARG;
  *out = nullptr;
  lbm_ctx* h = new lbm_ctx();
  h->p = *pp;
  const lbm_params& p = h->p;
  auto bad = [&](const char* msg) {
    h->err = msg;
    return LBM_ERR_ARG;
  };
  lbm_status st = LBM_OK;
  if (p.lattice != LBM_D2Q9 && p.lattice != LBM_D3Q19) st = bad("lattice must be D2Q9 or D3Q19");
  else if (p.nx < 1 || p.ny < 1 || p.nz < 1) st = bad("lattice sizes must be positive");
  else if ((long long)p.nx * p.ny * p.nz >= (1LL << 31) - 1024)
    st = bad("lattices of 2^31 nodes or more are not supported (32-bit node indices)");
  else if (p.lattice == LBM_D2Q9 && p.nz != 1) st = bad("D2Q9 needs nz == 1");
  else if (p.lattice == LBM_D2Q9 && p.force[2] != 0.0) st = bad("D2Q9 needs force[2] == 0");
  else if (p.collision != LBM_BGK && p.collision != LBM_MRT) st = bad("collision must be BGK or MRT");
  else if (!(p.tau > 0.5)) st = bad("tau must exceed 1/2");
  else if (p.nscalars < 0 || p.nscalars > (p.lattice == LBM_D3Q19 ? 2 : 1))
    st = bad("nscalars out of range (D3Q19: 0..2, D2Q9: 0..1)");
  else if (p.precision < 0 || p.precision > 2) st = bad("precision must be FP32, BF16 or FP16");
  else if (p.nsteps < 0) st = bad("nsteps must be >= 0");
  else if (p.obj_window < 0 || p.obj_window > p.nsteps + 1) st = bad("obj_window out of range");
  else if (p.objective < 0 || p.objective > 5) st = bad("unknown objective");
  else if (p.objective >= LBM_OBJ_VARIANCE && (p.nscalars < 1 || !p.inlet_outlet))
    st = bad("outlet objectives need a scalar lattice and inlet_outlet");
  else if (p.porosity < 0 || p.porosity > 2) st = bad("unknown porosity law");
  else if (p.scalar_inlet < 0 || p.scalar_inlet > 2) st = bad("unknown scalar inlet profile");
  else if (p.porosity == LBM_POR_POWER && p.porosity_q < 1.0) st = bad("power porosity needs q >= 1");
  else if (p.inlet_outlet && (p.nx < 3 || !(p.u_in < 1.0) || !(p.rho_out > 0.0)))
    st = bad("inlet_outlet needs nx >= 3, u_in < 1 and rho_out > 0");
  else if (p.inlet_kind < 0 || p.inlet_kind > 1) st = bad("inlet_kind must be 0 or 1");
  else if (p.inlet_kind == 1 && !(p.rho_out + 3.0 * p.dp > 0.0))
    st = bad("a pressure inlet needs rho_out + 3 dp > 0");
  else if (p.adjoint_mode < 0 || p.adjoint_mode > 1) st = bad("adjoint_mode must be 0 or 1");
  else if (p.adjoint_mode == 1 && p.obj_window != 0)
    st = bad("the fixed-point adjoint (adjoint_mode 1) needs obj_window 0: J = F(f^N)");
  else if (!theta) st = bad("theta must not be NULL");
  if (st) {
    *out = h;  // so that lbm_last_error can report; caller destroys
    return st;
  }
  h->Q = fluid_q(p.lattice);
  h->QS = scalar_q(p.lattice);
  h->M = h->Q + p.nscalars * h->QS;
  h->N = (long long)p.nx * p.ny * p.nz;
  h->stream = (cudaStream_t)stream;
  bool ok = p.lattice == LBM_D2Q9
                ? albm::kernels_d2q9(p.collision == LBM_MRT, p.nscalars, p.precision, &h->ks)
                : albm::kernels_d3q19(p.collision == LBM_MRT, p.nscalars, p.precision, &h->ks);
  if (!ok) {
    *out = h;
    h->err = "no kernel for this lattice/collision/scalars/precision";
    return LBM_ERR_ARG;
  }
  // kernel constants
  KParams& k = h->kp;
  k.nx = p.nx;
  k.ny = p.ny;
  k.nz = p.nz;
  k.nscal = p.nscalars;
  k.N = h->N;
  k.wait_polls = -1;
  k.fd_nx = albm::make_fastdiv((unsigned)p.nx);
  k.fd_ny = albm::make_fastdiv((unsigned)p.ny);
  k.fd_hx = albm::make_fastdiv((unsigned)std::max(p.nx / 2, 1));
  const double omega = 1.0 / p.tau;
  k.omega = (float)omega;
  k.one_m_omega = (float)(1.0 - omega);
  k.nu = (float)((p.tau - 0.5) / 3.0);
  k.gx = (float)p.force[0];
  k.gy = (float)p.force[1];
  k.gz = (float)p.force[2];
  k.u_in = (float)p.u_in;
  k.inv_1m_uin = (float)(1.0 / (1.0 - p.u_in));
  k.rho_out = (float)p.rho_out;
  k.drho_out = (float)(p.rho_out - 1.0);
  k.one_m_rho_out = (float)(1.0 - p.rho_out);
  k.inlet_kind = p.inlet_kind;
  k.rho_in = (float)(p.rho_out + 3.0 * p.dp);
  k.drho_in = (float)(p.rho_out + 3.0 * p.dp - 1.0);
  k.inv_rho_in = (float)(1.0 / (p.rho_out + 3.0 * p.dp));
  k.alpha_f = (float)p.alpha_fluid;
  k.alpha_s = (float)p.alpha_solid;
  k.porosity = p.porosity;
  k.por_q = (float)p.porosity_q;
  k.scalar_inlet = p.scalar_inlet;
  k.T_hot = (float)p.T_hot;
  k.objective = p.objective;
  if (p.collision == LBM_MRT) {
    if (p.lattice == LBM_D3Q19) albm::fill_mrt<albm::D3Q19>(omega, p.s_other, k);
    else albm::fill_mrt<albm::D2Q9>(omega, p.s_other, k);
  }
  if (p.precision != LBM_FP32) {
    // 16-bit storage holds deviations from the equilibrium at the inlet
    // velocity (rest for periodic channels)
    const double u_ref[3] = {p.inlet_outlet ? p.u_in : 0.0, 0.0, 0.0};
    if (p.lattice == LBM_D3Q19) albm::fill_dev_off<albm::D3Q19>(u_ref, k);
    else albm::fill_dev_off<albm::D2Q9>(u_ref, k);
  }
  h->state_bytes = (size_t)h->M * (size_t)h->N * (size_t)h->ks.storage_bytes;
  h->state_stride = (h->state_bytes + 255) / 256 * 256;
  // states are carved out of slabs of up to about 1 GiB (at least one state)
  h->slab_states = (int)std::max<size_t>(1, std::min<size_t>(4096, (1ull << 30) / h->state_stride));
  // time weights c_n of J = sum_n c_n F(f^n)
  h->c.assign((size_t)p.nsteps + 1, 0.0);
  if (p.objective != LBM_OBJ_NONE) {
    if (p.obj_window <= 0) h->c[p.nsteps] = 1.0;
    else
      for (int n = std::max(p.nsteps - p.obj_window + 1, 0); n <= p.nsteps; ++n)
        h->c[n] = 1.0 / p.obj_window;
  }
  auto fail = [&](lbm_status s) {
    *out = h;
    return s;
  };
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    h->err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return fail(LBM_ERR_CUDA);
  }
  e = h->ks.preload();
  if (e == cudaSuccess) e = preload_runtime_kernels();
  if (e != cudaSuccess) {
    h->err = std::string("loading the kernels: ") + cudaGetErrorString(e);
    return fail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA);
  }
  // device arrays
#define CKC(call)                                                            \
  do {                                                                       \
    cudaError_t _e = (call);                                                 \
    if (_e != cudaSuccess) {                                                 \
      h->err = std::string(#call) + ": " + cudaGetErrorString(_e);           \
      return fail(_e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA); \
    }                                                                        \
  } while (0)
  CKC(cudaMalloc(&h->flags, (size_t)h->N));
  CKC(cudaMalloc(&h->theta, sizeof(float) * (size_t)h->N));
  CKC(cudaMalloc(&h->grad, sizeof(double) * (size_t)h->N));
  CKC(cudaMalloc(&h->stats, sizeof(double) * 2 * (size_t)(p.nsteps + 1)));
  h->nblocks = (h->N + albm::kBlock - 1) / albm::kBlock;
  h->ntiles = h->N / albm::kTile;
  {
    const bool eligible = p.nx % albm::kTile == 0;
    if (p.kernel < 0 || p.kernel > 3) {
      h->err = "kernel must be 0 (automatic), 1 (per node), 2 or 3 (tile-staged)";
      return fail(LBM_ERR_ARG);
    }
    if (p.kernel >= 2 && !eligible) {
      h->err = "tile-staged kernels need nx to be a multiple of 128";
      return fail(LBM_ERR_ARG);
    }
    h->staged = p.kernel >= 2 ? p.kernel : 0;
  }
  CKC(cudaMalloc(&h->partials, sizeof(double) * 2 *
                                  (size_t)std::max(std::max(h->nblocks, h->ntiles),
                                                   h->ks.primal_partials(h->kp))));
  CKC(cudaMalloc(&h->d_err, sizeof(int)));
  CKC(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  CKC(cudaMalloc(&h->counter, sizeof(unsigned long long)));
  CKC(cudaMalloc(&h->lam[0], sizeof(float) * (size_t)h->M * (size_t)h->N));
  CKC(cudaMalloc(&h->lam[1], sizeof(float) * (size_t)h->M * (size_t)h->N));
  CKC(cudaMemsetAsync(h->grad, 0, sizeof(double) * (size_t)h->N, h->stream));
  CKC(cudaMemcpyAsync(h->theta, theta, sizeof(float) * (size_t)h->N, cudaMemcpyDefault, h->stream));
  if (flags) {
    h->flags_host.resize((size_t)h->N);
    CKC(cudaMemcpyAsync(h->flags_host.data(), flags, (size_t)h->N, cudaMemcpyDefault, h->stream));
    CKC(cudaStreamSynchronize(h->stream));
    for (uint8_t v : h->flags_host)
      if (v > LBM_NODE_HOT) {
        h->err = "flags hold an unknown node type";
        return fail(LBM_ERR_ARG);
      }
  } else {
    build_flags(p, h->flags_host);
  }
  CKC(cudaMemcpyAsync(h->flags, h->flags_host.data(), (size_t)h->N, cudaMemcpyHostToDevice,
                      h->stream));
  for (uint8_t v : h->flags_host) {
    h->n_in += v == LBM_NODE_INLET;
    h->n_out += v == LBM_NODE_OUTLET;
  }
  k.inv_A_in = h->n_in ? 1.0f / (float)h->n_in : 0.f;
  k.inv_A_out = h->n_out ? 1.0f / (float)h->n_out : 0.f;
  // state pool budget
  double budget = p.mem_budget;
  if (budget <= 0) {
    size_t fr = 0, tot = 0;
    CKC(cudaMemGetInfo(&fr, &tot));
    budget = 0.90 * (double)fr;
  }
  h->max_bufs = (int)std::max(3.0, std::floor(budget / (double)h->state_stride));
  // level-1 checkpoint stride: given, or every state if all fit, else
  // spread over half of the pool
  if (p.ckpt_every > 0) h->ckpt = p.ckpt_every;
  else if (p.nsteps + 2 <= h->max_bufs) h->ckpt = 1;
  else h->ckpt = std::max(1, (p.nsteps + h->max_bufs / 2 - 1) / std::max(1, h->max_bufs / 2));
  h->time_buf.assign((size_t)p.nsteps + 2, -1);
  CKC(cudaEventCreate(&h->t0));
  CKC(cudaEventCreate(&h->t1));
  CKC(cudaEventCreate(&h->t2));
  CKC(cudaEventCreate(&h->t3));
#undef CKC
  lbm_status s = do_reset(h);
  if (s) return fail(s);
  *out = h;
  return LBM_OK;
}

void lbm_destroy(lbm_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (void* b : h->slabs) cudaFree(b);
  cudaFree(h->flags);
  cudaFree(h->theta);
  cudaFree(h->grad);
  cudaFree(h->stats);
  cudaFree(h->partials);
  cudaFree(h->d_err);
  cudaFree(h->counter);
  cudaFree(h->lam[0]);
  cudaFree(h->lam[1]);
  cudaFree(h->design);
  cudaFree(h->os_stats);
  cudaFree(h->theta_saved);
  cudaFree(h->mma_hist);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->t0) cudaEventDestroy(h->t0);
  if (h->t1) cudaEventDestroy(h->t1);
  if (h->t2) cudaEventDestroy(h->t2);
  if (h->t3) cudaEventDestroy(h->t3);
  delete h;
}

lbm_status lbm_reset(lbm_handle h) {
  if (!h) return LBM_ERR_ARG;
  return do_reset(h);
}

lbm_status lbm_set_theta(lbm_handle h, const float* theta) {
  if (!h || !theta) return LBM_ERR_ARG;
  CK(h, cudaMemcpyAsync(h->theta, theta, sizeof(float) * (size_t)h->N, cudaMemcpyDefault,
                        h->stream));
  return do_reset(h);
}

int lbm_time(lbm_handle h) { return h ? h->t : -1; }
int lbm_adjoint_time(lbm_handle h) { return h ? h->t_adj : -1; }

lbm_status lbm_primal_step(lbm_handle h, int k) {
  if (!h) return LBM_ERR_ARG;
  if (k < 0 || h->t + k > h->p.nsteps)
    FAIL(h, LBM_ERR_ARG, "primal steps %d from time %d exceed the horizon %d", k, h->t,
         h->p.nsteps);
  if (h->oneshot) FAIL(h, LBM_ERR_STATE, "a one-shot run is active; reset first");
  if (h->t_adj >= 0) FAIL(h, LBM_ERR_STATE, "the adjoint of this trajectory has started; reset first");
  CK(h, cudaEventRecord(h->t0, h->stream));
  for (int i = 0; i < k; ++i) {
    const int src = find_buf(h, h->t);
    int dst;
    lbm_status s = acquire_evict(h, h->t, &dst);
    if (s) return s;
    s = launch_primal(h, src, dst, h->t, true, K_PRIMAL);
    if (s) return s;
    set_time(h, dst, h->t + 1);  // f^t stays while the pool has room
    h->t += 1;
  }
  if (k > 0 && h->t == h->p.nsteps) {
    lbm_status s = record_final_objective(h);
    if (s) return s;
  }
  CK(h, cudaEventRecord(h->t1, h->stream));
  h->primal_timed = k > 0;
  return LBM_OK;
}

lbm_status lbm_objective(lbm_handle h, double* J) {
  if (!h || !J) return LBM_ERR_ARG;
  std::vector<double> st(2 * (size_t)(h->p.nsteps + 1));
  CK(h, cudaMemcpyAsync(st.data(), h->stats, sizeof(double) * st.size(), cudaMemcpyDeviceToHost,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  {
    lbm_status ts = check_timeout(h);
    if (ts) return ts;
  }
  double acc = 0.0;
  const double A = h->n_out > 0 ? (double)h->n_out : 1.0;
  for (int n = 0; n <= std::min(h->t, h->p.nsteps); ++n) {
    if (h->c[n] == 0.0) continue;
    double Fn;
    switch (h->p.objective) {
      case LBM_OBJ_VARIANCE: {
        const double m = st[2 * n] / A;
        Fn = st[2 * n + 1] / A - m * m;
        break;
      }
      case LBM_OBJ_HEATFLUX_DP:
        Fn = st[2 * n] + 0.1 * h->p.rho_out / 3.0;
        break;
      default:
        Fn = st[2 * n];
    }
    acc += h->c[n] * Fn;
  }
  *J = acc;
  return LBM_OK;
}

// ---- fixed-point ALBS at the held state (Sec. 2.2) -------------------------
// v^k = (d(SW)/df(f-hat))^T v^{k-1} + dF/df(f-hat) with f-hat the current
// primal state, v^0 = 0 (or the seed); each iteration also writes the
// gradient estimate of Eq. adjoint:derivative from the iterate it consumes.
static lbm_status state_objective(lbm_ctx* h, int b);

static lbm_status frozen_start(lbm_ctx* h) {
  const int b = find_buf(h, h->t);
  if (b < 0) FAIL(h, LBM_ERR_STATE, "the current primal state is not held");
  CK(h, cudaMemsetAsync(h->grad, 0, sizeof(double) * (size_t)h->N, h->stream));
  h->lam_cur = 0;
  h->t_adj = h->t;
  h->frozen_k = 0;
  h->frozen_seeded = false;
  if (h->p.objective == LBM_OBJ_VARIANCE) {
    // the variance source needs the outlet mean of f-hat
    if (!h->os_stats) CK(h, cudaMalloc(&h->os_stats, 2 * sizeof(double)));
    lbm_status s = state_objective(h, b);
    if (s) return s;
  }
  return LBM_OK;
}

static lbm_status frozen_iteration(lbm_ctx* h) {
  StepArgs a = blank_args(h);
  a.Bin = h->bufs[find_buf(h, h->t_adj)];
  a.lam_in = h->lam[h->lam_cur];
  a.lam_out = h->lam[1 - h->lam_cur];
  a.grad = h->grad;
  a.ws = 1.0f;
  a.stat_n = h->p.objective == LBM_OBJ_VARIANCE ? h->os_stats : nullptr;
  a.has_next = (h->frozen_k > 0 || h->frozen_seeded) ? 1 : 0;   // v^0 = 0 needs no gather
  a.os.overwrite = 1;
  int slot;
  prof_begin(h, K_ADJOINT, &slot);
  cudaError_t e = h->ks.adjoint(h->kp, a, h->stream);
  prof_end(h, slot);
  if (e != cudaSuccess) FAIL(h, LBM_ERR_CUDA, "adjoint kernel launch: %s", cudaGetErrorString(e));
  h->lam_cur = 1 - h->lam_cur;
  h->frozen_k++;
  return LBM_OK;
}

static lbm_status adjoint_start(lbm_handle h) {
  CK(h, cudaMemsetAsync(h->grad, 0, sizeof(double) * (size_t)h->N, h->stream));
  h->lam_cur = 0;
  h->t_adj = h->t;
  // lambda^T = c_T dF/df(f^T): the adjoint kernel without the next state
  return launch_adjoint(h, h->t, 0);
}

lbm_status lbm_adjoint_step(lbm_handle h, int k) {
  if (!h) return LBM_ERR_ARG;
  if (k < 0) FAIL(h, LBM_ERR_ARG, "negative step count");
  if (h->oneshot) FAIL(h, LBM_ERR_STATE, "a one-shot run is active; reset first");
  CK(h, cudaEventRecord(h->t2, h->stream));
  if (h->p.adjoint_mode == 1) {
    if (h->t_adj < 0) {
      lbm_status s = frozen_start(h);
      if (s) return s;
    }
    for (int i = 0; i < k; ++i) {
      lbm_status s = frozen_iteration(h);
      if (s) return s;
    }
    CK(h, cudaEventRecord(h->t3, h->stream));
    h->adjoint_timed = true;
    return LBM_OK;
  }
  if (h->t_adj < 0) {
    lbm_status s = adjoint_start(h);
    if (s) return s;
  }
  if (k > h->t_adj) FAIL(h, LBM_ERR_STATE, "%d adjoint steps requested, %d remain", k, h->t_adj);
  for (int i = 0; i < k; ++i) {
    const int n = h->t_adj - 1;
    // states newer than n are no longer needed
    while (!h->held.empty() && *h->held.rbegin() > n) set_time(h, h->time_buf[*h->held.rbegin()], -1);
    lbm_status s = ensure_state(h, n);
    if (s) return s;
    s = launch_adjoint(h, n, 1);
    if (s) return s;
    h->t_adj = n;
  }
  CK(h, cudaEventRecord(h->t3, h->stream));
  h->adjoint_timed = true;
  return LBM_OK;
}

lbm_status lbm_adjoint_seed(lbm_handle h, const float* lam) {
  if (!h || !lam) return LBM_ERR_ARG;
  if (find_buf(h, h->t) < 0) FAIL(h, LBM_ERR_STATE, "current state not held");
  if (h->p.adjoint_mode == 1 && !h->oneshot) {
    lbm_status s = frozen_start(h);
    if (s) return s;
    h->frozen_seeded = true;
  }
  CK(h, cudaMemsetAsync(h->grad, 0, sizeof(double) * (size_t)h->N, h->stream));
  h->lam_cur = 0;
  h->t_adj = h->t;
  CK(h, cudaMemcpyAsync(h->lam[0], lam, sizeof(float) * (size_t)h->M * (size_t)h->N,
                        cudaMemcpyDefault, h->stream));
  if (!is_device_ptr(lam)) CK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_profile(lbm_handle h, int enable) {
  if (!h) return LBM_ERR_ARG;
  CK(h, cudaStreamSynchronize(h->stream));
  h->profile = enable != 0;
  h->launches_other = 0;
  h->ev_used.clear();
  h->ev_next = 0;
  return LBM_OK;
}

lbm_status lbm_profile_read(lbm_handle h, double* out) {
  if (!h || !out) return LBM_ERR_ARG;
  CK(h, cudaStreamSynchronize(h->stream));
  for (int i = 0; i < 8; ++i) out[i] = 0.0;
  for (auto& u : h->ev_used) {
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, h->ev_pool[u.second], h->ev_pool[u.second + 1]));
    out[2 * u.first] += 1.0;
    out[2 * u.first + 1] += ms;
  }
  out[6] = (double)h->launches_other;
  out[7] = out[0] + out[2] + out[4] + out[6];
  h->launches_other = 0;
  h->ev_used.clear();
  h->ev_next = 0;
  return LBM_OK;
}

long long lbm_recompute_steps(lbm_handle h) { return h ? h->recompute_steps : -1; }

// ---------------------------------------------------------------------------
// batched steps over several handles of one kernel family
// ---------------------------------------------------------------------------
static lbm_status batch_check(const lbm_handle* hs, int n) {
  if (!hs || n < 1) return LBM_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return LBM_ERR_ARG;
    if (hs[i]->oneshot) {
      hs[0]->err = "a batched handle has an active one-shot run";
      return LBM_ERR_STATE;
    }
    if (hs[i]->ks.primal != hs[0]->ks.primal || hs[i]->stream != hs[0]->stream) {
      hs[0]->err = "batched handles need the same lattice, collision, scalars, precision and stream";
      return LBM_ERR_ARG;
    }
  }
  return LBM_OK;
}

// report a member's failure on the first handle, which the caller queries
static lbm_status batch_fail(lbm_ctx* h0, lbm_ctx* h, lbm_status code) {
  if (h != h0) h0->err = std::string("batched handle: ") + h->err;
  return code;
}

static lbm_status batch_launch(lbm_ctx* h0, albm::BatchArgs& args, long long blocks, bool adjoint) {
  cudaError_t e = adjoint ? h0->ks.adjoint_batch(args, blocks, h0->stream)
                          : h0->ks.primal_batch(args, blocks, h0->stream);
  if (e != cudaSuccess)
    FAIL(h0, LBM_ERR_CUDA, "batched %s launch: %s", adjoint ? "adjoint" : "primal",
         cudaGetErrorString(e));
  args.n = 0;
  return LBM_OK;
}

// Instances at least this large fill the GPU alone: inside a batched step
// they run their own single-instance launch (the same kernels as when they
// are driven alone), and only the smaller ones share the batched launch.
constexpr long long kBatchAloneNodes = 1LL << 20;

struct BatchMove {
  lbm_ctx* h;
  int src, dst;
  bool alone;
};

// Batched primal steps; handle i stops at time stop[i] (its horizon at most).
static lbm_status batch_primal(const lbm_handle* hs, int n, const int* ks, int kall) {
  lbm_status st = batch_check(hs, n);
  if (st) return st;
  std::vector<int> stop((size_t)n);
  int k = 0;
  for (int i = 0; i < n; ++i) {
    if (hs[i]->t_adj >= 0) FAIL(hs[i], LBM_ERR_STATE, "the adjoint of this trajectory has started");
    const int ki = ks ? ks[i] : kall;
    if (ki < 0) FAIL(hs[0], LBM_ERR_ARG, "negative step count");
    stop[(size_t)i] = (int)std::min<long long>((long long)hs[i]->t + ki, hs[i]->p.nsteps);
    k = std::max(k, ki);
  }
  static thread_local albm::BatchArgs args;
  for (int step = 0; step < k; ++step) {
    args.n = 0;
    long long blocks = 0;
    std::vector<BatchMove> moved;
    // on failure: instances that ran their own launch keep their new state,
    // the others give back the buffer reserved for the batched launch
    auto unwind = [&](lbm_ctx* hf, lbm_status s) {
      for (auto& m : moved) {
        if (m.alone) {
          set_time(m.h, m.dst, m.h->t + 1);
          m.h->t += 1;
        } else if (m.h->buf_time[m.dst] == -2) {
          set_time(m.h, m.dst, -1);
        }
      }
      return batch_fail(hs[0], hf, s);
    };
    for (int i = 0; i < n; ++i) {
      lbm_ctx* h = hs[i];
      if (h->t >= stop[(size_t)i]) continue;  // horizon or this call's steps reached
      const int src = find_buf(h, h->t);
      int dst;
      lbm_status s = acquire_evict(h, h->t, &dst);
      if (s) return unwind(h, s);
      if (h->N >= kBatchAloneNodes) {
        s = launch_primal(h, src, dst, h->t, true, K_PRIMAL);  // folds its own objective
        if (s) return unwind(h, s);
        moved.push_back({h, src, dst, true});
        continue;
      }
      // dst stays reserved (-2) until the launch is issued
      albm::InstanceDesc& D = args.inst[args.n++];
      memset(&D, 0, sizeof(D));
      D.P = h->kp;
      D.Bin = h->bufs[src];
      D.Bout = h->bufs[dst];
      D.theta = h->theta;
      D.flags = h->flags;
      D.obj = h->c[h->t] != 0.0 ? h->partials : nullptr;
      D.block_begin = blocks;
      // blocks of the single-instance primal's size, so that the objective
      // partials are grouped as when the instance runs alone
      blocks += (h->N + ALBM_PRIMAL_BLOCK - 1) / ALBM_PRIMAL_BLOCK;
      moved.push_back({h, src, dst, false});
      if (args.n == albm::kMaxBatch) {
        s = batch_launch(hs[0], args, blocks, false);
        if (s) return unwind(hs[0], s);
        blocks = 0;
      }
    }
    if (args.n > 0) {
      lbm_status s = batch_launch(hs[0], args, blocks, false);
      if (s) return unwind(hs[0], s);
    }
    for (auto& m : moved) {
      lbm_ctx* h = m.h;
      if (!m.alone && h->c[h->t] != 0.0) {
        lbm_status s = fold_objective(h, h->t, (h->N + ALBM_PRIMAL_BLOCK - 1) / ALBM_PRIMAL_BLOCK);
        if (s) return batch_fail(hs[0], h, s);
      }
      set_time(h, m.dst, h->t + 1);
      h->t += 1;
      if (h->t == h->p.nsteps) {
        lbm_status s = record_final_objective(h);
        if (s) return batch_fail(hs[0], h, s);
      }
    }
    if (moved.empty()) break;
  }
  return LBM_OK;
}

lbm_status lbm_batch_primal_step(const lbm_handle* hs, int n, int k) {
  return batch_primal(hs, n, nullptr, k);
}

lbm_status lbm_batch_primal_steps(const lbm_handle* hs, int n, const int* ks) {
  if (!ks) return LBM_ERR_ARG;
  return batch_primal(hs, n, ks, 0);
}

// Batched adjoint steps; handle i stops at adjoint time stop[i] (0 at least).
static lbm_status batch_adjoint(const lbm_handle* hs, int n, const int* ks, int kall) {
  lbm_status st = batch_check(hs, n);
  if (st) return st;
  for (int i = 0; i < n; ++i) {
    if (hs[i]->p.adjoint_mode != 0)
      FAIL(hs[0], LBM_ERR_ARG, "batched adjoint steps need the unsteady adjoint (adjoint_mode 0)");
    if ((ks ? ks[i] : kall) < 0) FAIL(hs[0], LBM_ERR_ARG, "negative step count");
  }
  for (int i = 0; i < n; ++i)
    if (hs[i]->t_adj < 0) {
      lbm_status s = adjoint_start(hs[i]);
      if (s) return batch_fail(hs[0], hs[i], s);
    }
  std::vector<int> stop((size_t)n);
  int k = 0;
  for (int i = 0; i < n; ++i) {
    const int ki = ks ? ks[i] : kall;
    stop[(size_t)i] = std::max(hs[i]->t_adj - ki, 0);
    k = std::max(k, ki);
  }
  static thread_local albm::BatchArgs args;
  for (int step = 0; step < k; ++step) {
    args.n = 0;
    long long blocks = 0;
    std::vector<lbm_ctx*> moved;
    bool any = false;
    for (int i = 0; i < n; ++i) {
      lbm_ctx* h = hs[i];
      if (h->t_adj <= stop[(size_t)i]) continue;  // adjoint finished or this call's steps done
      const int nn = h->t_adj - 1;
      while (!h->held.empty() && *h->held.rbegin() > nn)
        set_time(h, h->time_buf[*h->held.rbegin()], -1);
      lbm_status s = ensure_state(h, nn);
      if (s) return batch_fail(hs[0], h, s);
      any = true;
      if (h->N >= kBatchAloneNodes) {
        s = launch_adjoint(h, nn, 1);  // flips its own adjoint buffers
        if (s) return batch_fail(hs[0], h, s);
        h->t_adj = nn;
        continue;
      }
      albm::InstanceDesc& D = args.inst[args.n++];
      memset(&D, 0, sizeof(D));
      D.P = h->kp;
      D.Bin = h->bufs[find_buf(h, nn)];
      D.theta = h->theta;
      D.flags = h->flags;
      D.lam_in = h->lam[h->lam_cur];
      D.lam_out = h->lam[1 - h->lam_cur];
      D.grad = h->grad;
      D.ws = (float)h->c[nn];
      D.stat_n = (h->p.objective == LBM_OBJ_VARIANCE && h->c[nn] != 0.0) ? h->stats + 2 * (size_t)nn
                                                                         : nullptr;
      D.has_next = 1;
      D.block_begin = blocks;
      blocks += (h->N + albm::kBlock - 1) / albm::kBlock;
      moved.push_back(h);
      if (args.n == albm::kMaxBatch) {
        s = batch_launch(hs[0], args, blocks, true);
        if (s) return s;
        blocks = 0;
      }
    }
    if (args.n > 0) {
      lbm_status s = batch_launch(hs[0], args, blocks, true);
      if (s) return s;
    }
    for (lbm_ctx* h : moved) {
      h->lam_cur = 1 - h->lam_cur;
      h->t_adj -= 1;
    }
    if (!any) break;
  }
  return LBM_OK;
}

lbm_status lbm_batch_adjoint_step(const lbm_handle* hs, int n, int k) {
  return batch_adjoint(hs, n, nullptr, k);
}

lbm_status lbm_batch_adjoint_steps(const lbm_handle* hs, int n, const int* ks) {
  if (!ks) return LBM_ERR_ARG;
  return batch_adjoint(hs, n, ks, 0);
}

lbm_status lbm_run(lbm_handle h) {
  if (!h) return LBM_ERR_ARG;
  lbm_status s = do_reset(h);
  if (s) return s;
  s = lbm_primal_step(h, h->p.nsteps);
  if (s) return s;
  return lbm_adjoint_step(h, h->p.nsteps);
}

lbm_status lbm_gradient(lbm_handle h, double* dst) {
  if (!h || !dst) return LBM_ERR_ARG;
  if (h->t_adj < 0) FAIL(h, LBM_ERR_STATE, "no adjoint has run");
  CK(h, cudaMemcpyAsync(dst, h->grad, sizeof(double) * (size_t)h->N, cudaMemcpyDefault, h->stream));
  if (!is_device_ptr(dst)) {
    CK(h, cudaStreamSynchronize(h->stream));
    return check_timeout(h);
  }
  return LBM_OK;
}

static lbm_status export_state(lbm_handle h, int time, float* dst, int which) {
  const int b = find_buf(h, time);
  if (b < 0) FAIL(h, LBM_ERR_STATE, "state of time %d is not held", time);
  const bool dev = is_device_ptr(dst);
  float* out = dst;
  if (!dev) CK(h, cudaMalloc(&out, sizeof(float) * (size_t)h->M * (size_t)h->N));
  StepArgs a = blank_args(h);
  a.Bin = h->bufs[b];
  a.fout = out;
  a.post = which;
  cudaError_t e = h->ks.exportf(h->kp, a, h->stream);
  if (e == cudaSuccess && !dev)
    e = cudaMemcpyAsync(dst, out, sizeof(float) * (size_t)h->M * (size_t)h->N,
                        cudaMemcpyDeviceToHost, h->stream);
  if (!dev) {
    cudaStreamSynchronize(h->stream);
    cudaFree(out);
  }
  if (e != cudaSuccess) FAIL(h, LBM_ERR_CUDA, "export: %s", cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_get_populations(lbm_handle h, float* dst, int which) {
  if (!h || !dst) return LBM_ERR_ARG;
  return export_state(h, h->t, dst, which);
}

lbm_status lbm_get_populations_at(lbm_handle h, int time, float* dst, int which) {
  if (!h || !dst) return LBM_ERR_ARG;
  return export_state(h, time, dst, which);
}

lbm_status lbm_set_populations(lbm_handle h, const float* src) {
  if (!h || !src) return LBM_ERR_ARG;
  reset_pool(h);
  int b;
  lbm_status s = acquire(h, &b);
  if (s) return s;
  const bool dev = is_device_ptr(src);
  const float* in = src;
  float* tmp = nullptr;
  if (!dev) {
    CK(h, cudaMalloc(&tmp, sizeof(float) * (size_t)h->M * (size_t)h->N));
    CK(h, cudaMemcpyAsync(tmp, src, sizeof(float) * (size_t)h->M * (size_t)h->N,
                          cudaMemcpyHostToDevice, h->stream));
    in = tmp;
  }
  StepArgs a = blank_args(h);
  a.fin = in;
  a.Bout = h->bufs[b];
  cudaError_t e = h->ks.importf(h->kp, a, h->stream);
  if (tmp) {
    cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
  }
  if (e != cudaSuccess) FAIL(h, LBM_ERR_CUDA, "import: %s", cudaGetErrorString(e));
  set_time(h, b, 0);
  h->t = 0;
  h->t_adj = h->oneshot ? 0 : -1;
  CK(h, cudaMemsetAsync(h->stats, 0, sizeof(double) * 2 * (size_t)(h->p.nsteps + 1), h->stream));
  return LBM_OK;
}

lbm_status lbm_get_adjoint(lbm_handle h, float* dst) {
  if (!h || !dst) return LBM_ERR_ARG;
  if (h->t_adj < 0) FAIL(h, LBM_ERR_STATE, "no adjoint has run");
  CK(h, cudaMemcpyAsync(dst, h->lam[h->lam_cur], sizeof(float) * (size_t)h->M * (size_t)h->N,
                        cudaMemcpyDefault, h->stream));
  if (!is_device_ptr(dst)) CK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_get_flags(lbm_handle h, uint8_t* dst) {
  if (!h || !dst) return LBM_ERR_ARG;
  CK(h, cudaMemcpyAsync(dst, h->flags, (size_t)h->N, cudaMemcpyDefault, h->stream));
  if (!is_device_ptr(dst)) CK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_check_finite(lbm_handle h, long long* count) {
  if (!h || !count) return LBM_ERR_ARG;
  const int b = find_buf(h, h->t);
  if (b < 0) FAIL(h, LBM_ERR_STATE, "current state not held");
  CK(h, cudaMemsetAsync(h->counter, 0, sizeof(unsigned long long), h->stream));
  StepArgs a = blank_args(h);
  a.Bin = h->bufs[b];
  a.count = h->counter;
  cudaError_t e = h->ks.nonfinite(h->kp, a, h->M, h->stream);
  if (e != cudaSuccess) FAIL(h, LBM_ERR_CUDA, "nonfinite: %s", cudaGetErrorString(e));
  unsigned long long c = 0;
  CK(h, cudaMemcpyAsync(&c, h->counter, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  {
    lbm_status ts = check_timeout(h);
    if (ts) return ts;
  }
  *count = (long long)c;
  if (c) FAIL(h, LBM_ERR_NONFINITE, "%llu non-finite values in the state at time %d", c, h->t);
  return LBM_OK;
}

lbm_status lbm_set_wait_polls(lbm_handle h, long long polls) {
  if (!h) return LBM_ERR_ARG;
  h->kp.wait_polls = polls < 0 ? -1 : (int)std::min<long long>(polls, 1LL << 30);
  return LBM_OK;
}

lbm_status lbm_set_stream(lbm_handle h, void* stream) {
  if (!h) return LBM_ERR_ARG;
  cudaStream_t ns = (cudaStream_t)stream;
  if (ns == h->stream) return LBM_OK;
  // work already queued for this handle on its old stream comes first
  cudaEvent_t ev = nullptr;
  CK(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ns, ev, 0);
  cudaEventDestroy(ev);
  if (e != cudaSuccess) FAIL(h, LBM_ERR_CUDA, "lbm_set_stream: %s", cudaGetErrorString(e));
  h->stream = ns;
  return LBM_OK;
}

lbm_status lbm_sizes(lbm_handle h, int* M, long long* N) {
  if (!h) return LBM_ERR_ARG;
  if (M) *M = h->M;
  if (N) *N = h->N;
  return LBM_OK;
}

lbm_status lbm_last_timing(lbm_handle h, float* primal_ms, float* adjoint_ms) {
  if (!h) return LBM_ERR_ARG;
  CK(h, cudaStreamSynchronize(h->stream));
  if (primal_ms) {
    *primal_ms = 0.f;
    if (h->primal_timed) CK(h, cudaEventElapsedTime(primal_ms, h->t0, h->t1));
  }
  if (adjoint_ms) {
    *adjoint_ms = 0.f;
    if (h->adjoint_timed) CK(h, cudaEventElapsedTime(adjoint_ms, h->t2, h->t3));
  }
  return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// one-shot optimisation (Sec. 3.3) and the threshold scan (Sec. 3.2)
// ---------------------------------------------------------------------------
static unsigned node_blocks(const lbm_ctx* h) { return (unsigned)((h->N + 255) / 256); }

static lbm_status ensure_design(lbm_ctx* h) {
  if (!h->design) {
    CK(h, cudaMalloc(&h->design, (size_t)h->N));
    h->design_default = true;
  }
  if (h->design_default) {
    albm::fluid_mask_kernel<<<node_blocks(h), 256, 0, h->stream>>>(h->N, h->flags, h->design);
    h->launches_other++;
    CK(h, cudaGetLastError());
  }
  if (!h->os_stats) CK(h, cudaMalloc(&h->os_stats, 2 * sizeof(double)));
  return LBM_OK;
}

static int oneshot_buf(lbm_ctx* h) { return find_buf(h, 0); }

// F of the state in buffer b into h->os_stats (objective kernel + fold)
static lbm_status state_objective(lbm_ctx* h, int b) {
  StepArgs a = blank_args(h);
  a.Bin = h->bufs[b];
  a.obj = h->partials;
  cudaError_t e = h->ks.objective(h->kp, a, h->stream);
  h->launches_other++;
  if (e != cudaSuccess) FAIL(h, LBM_ERR_CUDA, "objective kernel launch: %s", cudaGetErrorString(e));
  albm::fold_partials_kernel<<<1, 1024, 0, h->stream>>>(h->partials, h->nblocks, h->os_stats);
  h->launches_other++;
  CK(h, cudaGetLastError());
  return LBM_OK;
}

// the objective from its two folded sums (the formulas of lbm_objective)
static double objective_value(const lbm_ctx* h, const double* st) {
  const double A = h->n_out > 0 ? (double)h->n_out : 1.0;
  switch (h->p.objective) {
    case LBM_OBJ_VARIANCE: {
      const double m = st[0] / A;
      return st[1] / A - m * m;
    }
    case LBM_OBJ_HEATFLUX_DP:
      return st[0] + 0.1 * h->p.rho_out / 3.0;
    default:
      return st[0];
  }
}

static lbm_status oneshot_iteration(lbm_ctx* h, double zeta, double penalty, double s) {
  const int src = oneshot_buf(h);
  if (src < 0) FAIL(h, LBM_ERR_STATE, "the one-shot state is not held");
  int dst;
  lbm_status st = acquire(h, &dst);
  if (st) return st;
  const bool variance = h->p.objective == LBM_OBJ_VARIANCE;
  // 1. primal step f^k -> f^{k+1}; the variance source needs the outlet mean of f^k
  StepArgs a = blank_args(h);
  a.Bin = h->bufs[src];
  a.Bout = h->bufs[dst];
  a.obj = variance ? h->partials : nullptr;
  a.err = h->d_err;
  int slot;
  prof_begin(h, K_PRIMAL, &slot);
  cudaError_t e = h->ks.primal(h->kp, a, h->stream);
  prof_end(h, slot);
  if (e != cudaSuccess) FAIL(h, LBM_ERR_CUDA, "primal kernel launch: %s", cudaGetErrorString(e));
  if (variance) {
    albm::fold_partials_kernel<<<1, 1024, 0, h->stream>>>(h->partials, h->ks.primal_partials(h->kp),
                                                          h->os_stats);
    h->launches_other++;
    CK(h, cudaGetLastError());
  }
  // 2.-4. ALBS step at f^k with the source every iteration; the adjoint
  // kernel writes the estimate g^k into grad and updates theta in place
  StepArgs b = blank_args(h);
  b.Bin = h->bufs[src];
  b.lam_in = h->lam[h->lam_cur];
  b.lam_out = h->lam[1 - h->lam_cur];
  b.grad = h->grad;
  b.ws = 1.0f;
  b.stat_n = variance ? h->os_stats : nullptr;
  b.has_next = 1;
  b.err = h->d_err;
  b.os.design = h->design;
  b.os.theta_out = h->theta;
  b.os.zeta = (float)zeta;
  b.os.penalty = (float)penalty;
  b.os.sign = (float)s;
  prof_begin(h, K_ADJOINT, &slot);
  e = h->ks.adjoint(h->kp, b, h->stream);
  prof_end(h, slot);
  if (e != cudaSuccess) FAIL(h, LBM_ERR_CUDA, "adjoint kernel launch: %s", cudaGetErrorString(e));
  h->lam_cur = 1 - h->lam_cur;
  set_time(h, src, -1);
  set_time(h, dst, 0);
  return LBM_OK;
}

extern "C" {

lbm_status lbm_set_design(lbm_handle h, const uint8_t* mask) {
  if (!h) return LBM_ERR_ARG;
  if (!h->design) CK(h, cudaMalloc(&h->design, (size_t)h->N));
  if (!mask) {
    h->design_default = true;
    return ensure_design(h);
  }
  h->design_default = false;
  CK(h, cudaMemcpyAsync(h->design, mask, (size_t)h->N, cudaMemcpyDefault, h->stream));
  if (!is_device_ptr(mask)) CK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_oneshot_reset(lbm_handle h) {
  if (!h) return LBM_ERR_ARG;
  lbm_status s = do_reset(h);   // f^0 = rest state in the buffer of time 0
  if (s) return s;
  s = ensure_design(h);
  if (s) return s;
  CK(h, cudaMemsetAsync(h->lam[0], 0, sizeof(float) * (size_t)h->M * (size_t)h->N, h->stream));
  CK(h, cudaMemsetAsync(h->grad, 0, sizeof(double) * (size_t)h->N, h->stream));
  CK(h, cudaMemsetAsync(h->os_stats, 0, 2 * sizeof(double), h->stream));
  h->lam_cur = 0;
  h->t_adj = 0;
  h->oneshot = true;
  return LBM_OK;
}

lbm_status lbm_oneshot_step(lbm_handle h, int iters, double zeta, double penalty, int maximize) {
  if (!h) return LBM_ERR_ARG;
  if (!h->oneshot) FAIL(h, LBM_ERR_STATE, "no one-shot run started (lbm_oneshot_reset)");
  if (iters < 0 || !(zeta >= 0.0) || !(penalty >= 0.0) || !std::isfinite(zeta) ||
      !std::isfinite(penalty))
    FAIL(h, LBM_ERR_ARG, "one-shot needs iters >= 0 and finite zeta, penalty >= 0");
  const double s = maximize ? 1.0 : -1.0;
  for (int i = 0; i < iters; ++i) {
    lbm_status st = oneshot_iteration(h, zeta, penalty, s);
    if (st) return st;
  }
  return LBM_OK;
}

lbm_status lbm_oneshot_eval(lbm_handle h, double* J, double* P) {
  if (!h) return LBM_ERR_ARG;
  if (!h->oneshot) FAIL(h, LBM_ERR_STATE, "no one-shot run started (lbm_oneshot_reset)");
  double st[2] = {0.0, 0.0}, pp[2] = {0.0, 0.0};
  if (J) {
    lbm_status s = state_objective(h, oneshot_buf(h));
    if (s) return s;
    CK(h, cudaMemcpyAsync(st, h->os_stats, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));   // os_stats is reused below
  }
  if (P) {
    albm::penalty_kernel<<<node_blocks(h), 256, 0, h->stream>>>(h->N, h->theta, h->design,
                                                               h->partials);
    albm::fold_partials_kernel<<<1, 1024, 0, h->stream>>>(h->partials, (long long)node_blocks(h),
                                                          h->os_stats);
    h->launches_other += 2;
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(pp, h->os_stats, sizeof(pp), cudaMemcpyDeviceToHost, h->stream));
  }
  CK(h, cudaStreamSynchronize(h->stream));
  {
    lbm_status ts = check_timeout(h);
    if (ts) return ts;
  }
  if (J) *J = objective_value(h, st);
  if (P) *P = pp[0];
  return LBM_OK;
}

lbm_status lbm_threshold_scan(lbm_handle h, const double* eta, int n, int nsteps, double* J_out) {
  if (!h || !eta || !J_out || n < 1 || nsteps < 1) return LBM_ERR_ARG;
  lbm_status s = ensure_design(h);
  if (s) return s;
  if (!h->theta_saved) CK(h, cudaMalloc(&h->theta_saved, sizeof(float) * (size_t)h->N));
  CK(h, cudaMemcpyAsync(h->theta_saved, h->theta, sizeof(float) * (size_t)h->N,
                        cudaMemcpyDeviceToDevice, h->stream));
  lbm_status result = LBM_OK;
  for (int i = 0; i < n && result == LBM_OK; ++i) {
    albm::threshold_kernel<<<node_blocks(h), 256, 0, h->stream>>>(h->N, h->theta_saved, h->theta,
                                                                 h->design, (float)eta[i]);
    h->launches_other++;
    if (cudaGetLastError() != cudaSuccess) {
      h->err = "threshold kernel launch failed";
      result = LBM_ERR_CUDA;
      break;
    }
    result = do_reset(h);
    int cur = find_buf(h, 0);
    for (int k = 0; k < nsteps && result == LBM_OK; ++k) {
      int dst;
      result = acquire(h, &dst);
      if (result) break;
      result = launch_primal(h, cur, dst, 0, false, K_PRIMAL);
      set_time(h, cur, -1);
      set_time(h, dst, 0);
      cur = dst;
    }
    if (result == LBM_OK) result = state_objective(h, cur);
    double st[2] = {0.0, 0.0};
    if (result == LBM_OK) {
      if (cudaMemcpyAsync(st, h->os_stats, sizeof(st), cudaMemcpyDeviceToHost, h->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(h->stream) != cudaSuccess) {
        h->err = "threshold scan: reading the objective failed";
        result = LBM_ERR_CUDA;
      } else {
        result = check_timeout(h);
      }
    }
    if (result == LBM_OK) J_out[i] = objective_value(h, st);
  }
  // restore the continuous design and a fresh state whatever happened
  cudaMemcpyAsync(h->theta, h->theta_saved, sizeof(float) * (size_t)h->N, cudaMemcpyDeviceToDevice,
                  h->stream);
  lbm_status r2 = do_reset(h);
  return result ? result : r2;
}

lbm_status lbm_threshold_apply(lbm_handle h, double eta) {
  if (!h || !std::isfinite(eta)) return LBM_ERR_ARG;
  lbm_status s = ensure_design(h);
  if (s) return s;
  if (!h->theta_saved) CK(h, cudaMalloc(&h->theta_saved, sizeof(float) * (size_t)h->N));
  CK(h, cudaMemcpyAsync(h->theta_saved, h->theta, sizeof(float) * (size_t)h->N,
                        cudaMemcpyDeviceToDevice, h->stream));
  albm::threshold_kernel<<<node_blocks(h), 256, 0, h->stream>>>(h->N, h->theta_saved, h->theta,
                                                               h->design, (float)eta);
  h->launches_other++;
  CK(h, cudaGetLastError());
  return do_reset(h);
}

lbm_status lbm_mma_reset(lbm_handle h) {
  if (!h) return LBM_ERR_ARG;
  lbm_status s = ensure_design(h);
  if (s) return s;
  if (!h->mma_hist) CK(h, cudaMalloc(&h->mma_hist, 4 * sizeof(float) * (size_t)h->N));
  h->mma_k = 0;
  return LBM_OK;
}

static lbm_status mma_launch(lbm_ctx* h, const double* grad, int maximize, double move) {
  if (h->mma_k < 0) FAIL(h, LBM_ERR_STATE, "MMA not started (lbm_mma_reset)");
  if (h->oneshot) FAIL(h, LBM_ERR_STATE, "a one-shot run is active");
  if (!(move > 0.0 && move <= 1.0)) FAIL(h, LBM_ERR_ARG, "MMA move limit must be in (0, 1]");
  float* hb = h->mma_hist;
  const size_t n = (size_t)h->N;
  albm::mma_update_kernel<<<node_blocks(h), 256, 0, h->stream>>>(
      h->N, h->theta, hb, hb + n, hb + 2 * n, hb + 3 * n, grad, h->design, h->mma_k,
      maximize ? -1.0f : 1.0f, (float)move);
  h->launches_other++;
  CK(h, cudaGetLastError());
  h->mma_k++;
  return LBM_OK;
}

lbm_status lbm_mma_update(lbm_handle h, int maximize, double move) {
  if (!h) return LBM_ERR_ARG;
  const bool done = h->p.adjoint_mode == 1 ? (h->t_adj >= 0 && h->frozen_k > 0) : h->t_adj == 0;
  if (h->oneshot || !done)
    FAIL(h, LBM_ERR_STATE, "MMA needs a completed adjoint (lbm_run) before the update");
  lbm_status s = mma_launch(h, h->grad, maximize, move);
  if (s) return s;
  return do_reset(h);
}

lbm_status lbm_mma_update_with(lbm_handle h, const double* grad, int maximize, double move) {
  if (!h || !grad) return LBM_ERR_ARG;
  const double* g = grad;
  double* tmp = nullptr;
  if (!is_device_ptr(grad)) {
    CK(h, cudaMalloc(&tmp, sizeof(double) * (size_t)h->N));
    CK(h, cudaMemcpyAsync(tmp, grad, sizeof(double) * (size_t)h->N, cudaMemcpyHostToDevice,
                          h->stream));
    g = tmp;
  }
  lbm_status s = mma_launch(h, g, maximize, move);
  if (tmp) {
    cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
  }
  return s;
}

lbm_status lbm_get_theta(lbm_handle h, float* dst) {
  if (!h || !dst) return LBM_ERR_ARG;
  CK(h, cudaMemcpyAsync(dst, h->theta, sizeof(float) * (size_t)h->N, cudaMemcpyDefault, h->stream));
  if (!is_device_ptr(dst)) CK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

}  // extern "C"
