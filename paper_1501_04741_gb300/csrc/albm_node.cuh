// Node operator W^x (Eq. "normal:iteration") and its transpose (Eq.
// "adjoint:operator") for every node type, as device functions.
//
// Fluid populations are carried as deviations d_i = f_i - w_i from the rest
// state (rho = 1, u = 0); this keeps the non-equilibrium part f - f_eq, a
// small difference of O(1) numbers, accurate in FP32 and lets BF16/FP16
// storage hold only the small part.  Scalars have a zero rest state and are
// carried as they are.
//
// Interior collision (Sec. 3.1 and 3.2), per node with rho = 1 + drho,
// u = j / rho and the post-collision velocity v = G(theta) u + g:
//   deq_i(rho, u) = w_i (drho + rho P_i(u)),  P_i(u) = 3 e.u + 4.5 (e.u)^2 - 1.5 u.u
//   BGK  (Eq. SRT + Exact-Difference term):  W_i - w_i = deq_i(rho,v) + (1-omega)(d_i - deq_i(rho,u))
//   FMRT (Sec. 3.1):                          W_i - w_i = deq_i(rho,v) + [U^-1 (I-T) U (d - deq(rho,u))]_i
// with U^-1 (I-T) U = sum_k r_k U_k U_k^T, r_k = (1 - s_k) / |U_k|^2 (U has
// orthogonal rows), a symmetric operator, so its transpose is itself.
//
// Reverse mode.  For adjoint weights a on the fluid outputs let
//   H_a(rho, u) = sum_i a_i deq_i(rho, u) = drho A0 + rho (3 A1.u + 4.5 u.A2.u - 1.5 A0 u.u)
// with A0 = sum a_i w_i, A1 = sum a_i w_i e_i, A2 = sum a_i w_i e_i e_i^T.  Then
//   sum_i a_i W_i = H_a(rho, v) + sum_i c_i d_i - H_c(rho, u),  c = (1-omega) a  or  (U^-1(I-T)U) a,
// whose partial derivatives give the adjoint of every population in a few
// dot products (the paper reverse-differentiates W with TAPENADE, Sec. 3.4;
// here the derivative is written out by hand and checked against the oracle).
#pragma once
#include <stdint.h>

#include <utility>

#include "albm_lattice.cuh"

namespace albm {

enum : uint8_t { FLUID = 0, WALL = 1, INLET = 2, OUTLET = 3, HOT = 4 };
enum {
  OBJ_NONE = 0,
  OBJ_DISSIPATION = 1,
  OBJ_VARIANCE = 2,
  OBJ_HEATFLUX_DP = 3,
  OBJ_MIXFLUX = 4,
  OBJ_HEATFLUX = 5
};
enum { POR_LINEAR = 0, POR_POWER = 1, POR_RAMP = 2 };

// Objective form a launch compiles in: 0 when the step records or sources no
// objective, 2 for the dissipation (a term at every fluid node), 1 for the
// outlet/inlet objectives (terms at boundary nodes only, so the kernel keeps
// no per-population source in registers).  Host and batched launches use
// the same rule, so a node gets the same code alone or batched.
__host__ __device__ inline int obj_kind(bool active, int objective) {
  return !active ? 0 : (objective == OBJ_DISSIPATION ? 2 : 1);
}

#ifndef ALBM_ADJ_TWO_PHASE
#define ALBM_ADJ_TWO_PHASE 1
#endif
// MRT through all 19 moments instead of the rank-one form (same operator)
#ifndef ALBM_MRT_FULL
#define ALBM_MRT_FULL 0
#endif
// adjoint: the weighted moments C of c summed over the populations instead
// of derived from A and the MRT moments (same values up to rounding)
#ifndef ALBM_C_LOOP
#define ALBM_C_LOOP 0
#endif
// scalar collision as g + om (geq - g) per population instead of the
// polynomial form of NodeOps::scalars_forward (same values up to rounding)
#ifndef ALBM_SCALAR_DIRECT
#define ALBM_SCALAR_DIRECT 0
#endif
// 16-bit storage: the interior-node primal works on the stored values and
// carries the reference offsets as constants of the moments and of the
// collision (instead of adding them to every population loaded and
// subtracting them from every population stored).  Measured slower (the
// paired kernel spills more with the boundary path beside the folded
// one: 0.682 -> 0.708 ms on the exchanger), so off by default.
#ifndef ALBM_FOLD_OFFSET
#define ALBM_FOLD_OFFSET 0
#endif
// fluid collision as two equilibria per population (the direct form of the
// operator) instead of the polynomial form of NodeOps::collide_fluid
#ifndef ALBM_COLLIDE_DIRECT
#define ALBM_COLLIDE_DIRECT 0
#endif
// MRT: keep the conserved moments in the rank-one operator.  They act on
// f - f_eq(rho, u), whose density and momentum vanish, and in the adjoint on
// a vector that (I - d f_eq / d f)^T annihilates along them, so by default
// only the stress moments are applied (results equal up to rounding).
#ifndef ALBM_MRT_CONSERVED
#define ALBM_MRT_CONSERVED 0
#endif

// Division of a 32-bit unsigned n by a divisor d that is fixed for the
// problem, by a multiply-high and two shifts (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, Fig.
// 4.1: l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n -
// t) >> min(l, 1))) >> max(l - 1, 0) with t = mulhi(m, n); exact for every
// 32-bit n and d >= 1).  Replaces the 64-bit division of a node index by
// the row length, which costs tens of instructions per node.
struct FastDiv {
  unsigned m, s1, s2;
};

inline FastDiv make_fastdiv(unsigned d) {
  unsigned l = 0;
  while (l < 32 && (1ull << l) < (unsigned long long)d) ++l;
  FastDiv f;
  f.m = (unsigned)((((1ull << 32) * ((1ull << l) - (unsigned long long)d)) / d) + 1ull);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

__host__ __device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
  const unsigned t = __umulhi(f.m, n);
#else
  const unsigned t = (unsigned)(((unsigned long long)f.m * n) >> 32);
#endif
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

// Reciprocals of the density and of the scalar relaxation time: the fast
// approximate division (at most 2 ulp off; measured 1.4 % on the 16-bit
// primal and 0.8 % on the mixer adjoint), or IEEE division with
// ALBM_FAST_RCP=0.
#ifndef ALBM_FAST_RCP
#define ALBM_FAST_RCP 1
#endif
__device__ __forceinline__ float rcp(float x) {
#if ALBM_FAST_RCP
  return __fdividef(1.0f, x);
#else
  return 1.0f / x;
#endif
}

// Constants of one problem, passed by value to every kernel.
struct KParams {
  int nx, ny, nz, nscal;
  long long N;
  float omega, one_m_omega, nu;
  float gx, gy, gz;
  float u_in, inv_1m_uin, rho_out, drho_out, one_m_rho_out;
  int inlet_kind;        // 0 velocity inlet at u_in; 1 pressure inlet at rho_in, capped at u_in
  float rho_in, drho_in, inv_rho_in;
  float alpha_f, alpha_s;
  int porosity;
  float por_q;
  int scalar_inlet;
  float T_hot;
  int objective;
  float inv_A_in, inv_A_out;
  float mrt_diag;
  float mrt_r[19];
  // 16-bit storage: stored value = d_i - dev_off[i], with dev_off[i] =
  // f_eq,i(1, u_ref) - w_i the equilibrium deviation at the reference
  // velocity (zero for FP32 storage)
  float dev_off[19];
  // 16-bit storage: sums over the populations of dev_off and of e_i dev_off
  // (the density and momentum of the reference offsets: 0 and u_ref)
  float drho_off, j_off[3];
  // n / nx, n / ny and n / (nx / 2) for node, row and pair indices (N < 2^31)
  FastDiv fd_nx, fd_ny, fd_hx;
  // polls a tile-staged kernel waits for a stage's copies (< 0: default)
  int wait_polls;
};

// MRT coefficients of NodeOps::mrt_op for rates omega (stress moments),
// s_other (other non-conserved moments) and 0 (conserved moments)
template <class L>
inline void fill_mrt(double omega, double s_other, KParams& k) {
  for (int j = 0; j < 19; ++j) k.mrt_r[j] = 0.f;
  k.mrt_diag = (float)(1.0 - s_other);
  for (int j = 0; j < L::NMOM; ++j) {
    double D = 0.0;
    for (int i = 0; i < L::Q; ++i) D += double(L::U(j, i)) * double(L::U(j, i));
    if (L::stress(j)) k.mrt_r[j] = (float)((s_other - omega) / D);
    if (L::conserved(j)) k.mrt_r[j] = (float)(s_other / D);
  }
}

// Reference offsets of 16-bit storage: dev_off[i] = f_eq,i(1, u_ref) - w_i =
// w_i (3 e.u + 4.5 (e.u)^2 - 1.5 u.u) at the reference velocity u_ref
template <class L>
inline void fill_dev_off(const double* u_ref, KParams& k) {
  for (int j = 0; j < 19; ++j) k.dev_off[j] = 0.f;
  const double uu = u_ref[0] * u_ref[0] + u_ref[1] * u_ref[1] + u_ref[2] * u_ref[2];
  double s0 = 0.0, s1[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < L::Q; ++i) {
    const double eu = L::ex(i) * u_ref[0] + L::ey(i) * u_ref[1] + L::ez(i) * u_ref[2];
    k.dev_off[i] = (float)(double(L::w(i)) * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
    s0 += k.dev_off[i];
    s1[0] += L::ex(i) * (double)k.dev_off[i];
    s1[1] += L::ey(i) * (double)k.dev_off[i];
    s1[2] += L::ez(i) * (double)k.dev_off[i];
  }
  k.drho_off = (float)s0;
  for (int a = 0; a < 3; ++a) k.j_off[a] = (float)s1[a];
}

// ---------------------------------------------------------------------------
// porosity G(theta) (Sec. 3.2, theta = 1 - w) and diffusivity interpolation
// ---------------------------------------------------------------------------
__device__ __forceinline__ void porosity_G(const KParams& P, float th, float& G, float& dG) {
  if (P.porosity == POR_LINEAR) {
    G = 1.0f - th;
    dG = -1.0f;
  } else if (P.porosity == POR_POWER) {
    const float q = P.por_q;
    const float tq1 = th > 0.0f ? __powf(th, q - 1.0f) : (q == 1.0f ? 1.0f : 0.0f);
    G = 1.0f - tq1 * th;
    dG = -q * tq1;
  } else {
    const float den = 1.0f / (1.0f + P.por_q * th);
    G = (1.0f - th) * den;
    dG = -(1.0f + P.por_q) * den * den;
  }
}

template <class LS>
__device__ __forceinline__ void scalar_rate(const KParams& P, float th, float& om, float& dom) {
  const float alpha = (1.0f - th) * P.alpha_f + th * P.alpha_s;
  om = rcp(0.5f + alpha * (1.0f / LS::cs2));
  dom = -om * om * (P.alpha_s - P.alpha_f) * (1.0f / LS::cs2);
}

// ---------------------------------------------------------------------------
// Node kernels for fluid lattice L with NS scalar lattices
// ---------------------------------------------------------------------------
template <class L, int NS, bool MRT>
struct NodeOps {
  using LS = typename ScalarOf<L>::type;
  static constexpr int Q = L::Q;
  static constexpr int QS = LS::Q;
  static constexpr int M = Q + NS * QS;
  static constexpr int NSA = NS > 0 ? NS : 1;

  // y = U^-1 (I - T) U x.  U has orthogonal rows, so U^-1 = U^T D^-1 and
  // sum_k U_k U_k^T / D_k = I; all non-stress, non-conserved moments share
  // one rate s, hence
  //   U^-1 (I - T) U = (1 - s) I + sum_{k stress, conserved} c_k U_k U_k^T,
  //   c_k = (s - s_k) / D_k   (s_k = omega for stress moments, 0 for rho, j),
  // a symmetric operator needing 9 (D3Q19) or 5 (D2Q9) moments, not 19 / 9.
  // P.mrt_r[k] holds c_k and P.mrt_diag holds 1 - s (set by fill_mrt).
  __device__ static __forceinline__ void mrt_op(const KParams& P, const float* x, float* y) {
    float m[L::NMOM];
    mrt_op_m(P, x, y, m);
  }

  // mrt_op that also returns m[k] = c_k (U_k . x) for the stress and
  // conserved moments (the rank-one weights; other entries unset)
  __device__ static __forceinline__ void mrt_op_m(const KParams& P, const float* x, float* y,
                                                  float* m) {
#if ALBM_MRT_FULL
    // the same operator through all moments: y = sum_k r_k U_k (U_k . x)
    float mf[L::NMOM];
#pragma unroll
    for (int k = 0; k < L::NMOM; ++k) {
      float a = 0.0f;
#pragma unroll
      for (int i = 0; i < Q; ++i)
        if (L::U(k, i) != 0) a += float(L::U(k, i)) * x[i];
      const float D = float(Dsq(k));
      const float rk = L::stress(k) ? (P.mrt_diag + P.mrt_r[k] * D)
                                    : (L::conserved(k) ? (P.mrt_diag + P.mrt_r[k] * D) : P.mrt_diag);
      mf[k] = a * rk / D;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float v = 0.0f;
#pragma unroll
      for (int k = 0; k < L::NMOM; ++k)
        if (L::U(k, i) != 0) v += float(L::U(k, i)) * mf[k];
      y[i] = v;
    }
    return;
#endif
#pragma unroll
    for (int k = 0; k < L::NMOM; ++k) {
      m[k] = 0.0f;
      if (!rank_one(k)) continue;
#pragma unroll
      for (int i = 0; i < Q; ++i)
        if (L::U(k, i) != 0) m[k] += float(L::U(k, i)) * x[i];
      m[k] *= P.mrt_r[k];
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float v = P.mrt_diag * x[i];
#pragma unroll
      for (int k = 0; k < L::NMOM; ++k)
        if (rank_one(k) && L::U(k, i) != 0) v += float(L::U(k, i)) * m[k];
      y[i] = v;
    }
  }

  // moments carried by the rank-one terms of mrt_op
  __host__ __device__ static constexpr bool rank_one(int k) {
    return L::stress(k) || (ALBM_MRT_CONSERVED && L::conserved(k));
  }

  // Weighted moments of the rows of U, sum_i w_i U(k,i) (e_ia (e_ib)), from
  // the weights times 36 (integers for D2Q9 and D3Q19), so that the entries
  // that vanish by symmetry are exact zeros and drop out at compile time.
  __host__ __device__ static constexpr int w36(int i) { return int(L::w(i) * 36.0f + 0.5f); }
  __host__ __device__ static constexpr int ecomp(int i, int a) {
    return a == 0 ? L::ex(i) : (a == 1 ? L::ey(i) : L::ez(i));
  }
  __host__ __device__ static constexpr int UW0(int k) {
    int s = 0;
    for (int i = 0; i < Q; ++i) s += w36(i) * L::U(k, i);
    return s;
  }
  __host__ __device__ static constexpr int UW1(int k, int a) {
    int s = 0;
    for (int i = 0; i < Q; ++i) s += w36(i) * ecomp(i, a) * L::U(k, i);
    return s;
  }
  __host__ __device__ static constexpr int UW2(int k, int a, int b) {
    int s = 0;
    for (int i = 0; i < Q; ++i) s += w36(i) * ecomp(i, a) * ecomp(i, b) * L::U(k, i);
    return s;
  }

  // C += m_k (weighted moments of U_k) for one rank-one moment k; the
  // weights are constant expressions, so zero terms vanish in the front end
  template <int k>
  __device__ static __forceinline__ void add_row_moment(float m, float& C0, float* C1,
                                                        float (*C2)[3]) {
    if constexpr (rank_one(k)) {
      constexpr float s = 1.0f / 36.0f;
      if constexpr (UW0(k) != 0) C0 += (float(UW0(k)) * s) * m;
      if constexpr (UW1(k, 0) != 0) C1[0] += (float(UW1(k, 0)) * s) * m;
      if constexpr (UW1(k, 1) != 0) C1[1] += (float(UW1(k, 1)) * s) * m;
      if constexpr (UW1(k, 2) != 0) C1[2] += (float(UW1(k, 2)) * s) * m;
      if constexpr (UW2(k, 0, 0) != 0) C2[0][0] += (float(UW2(k, 0, 0)) * s) * m;
      if constexpr (UW2(k, 0, 1) != 0) C2[0][1] += (float(UW2(k, 0, 1)) * s) * m;
      if constexpr (UW2(k, 0, 2) != 0) C2[0][2] += (float(UW2(k, 0, 2)) * s) * m;
      if constexpr (UW2(k, 1, 1) != 0) C2[1][1] += (float(UW2(k, 1, 1)) * s) * m;
      if constexpr (UW2(k, 1, 2) != 0) C2[1][2] += (float(UW2(k, 1, 2)) * s) * m;
      if constexpr (UW2(k, 2, 2) != 0) C2[2][2] += (float(UW2(k, 2, 2)) * s) * m;
    }
  }
  template <int... K>
  __device__ static __forceinline__ void add_row_moments(std::integer_sequence<int, K...>,
                                                         const float* mk, float& C0, float* C1,
                                                         float (*C2)[3]) {
    (add_row_moment<K>(mk[K], C0, C1, C2), ...);
  }

  __host__ __device__ static constexpr int Dsq(int k) {
    int d = 0;
    for (int i = 0; i < Q; ++i) d += L::U(k, i) * L::U(k, i);
    return d;
  }

  // Zou-He (Sec. 3): reconstruct the unknown populations of an x face in
  // place and return rho, drho, u.  Unknowns have e.n > 0 for the inward
  // normal n; rho (1 - u.n) = s0 + 2 s_out from mass and normal momentum;
  // each unknown is its opposite plus 2 w_i rho (e_i.u) / cs2, minus the
  // transverse correction sum_t e_it N_t, N_t = 1/2 sum_{e.n = 0} f_k e_kt.
  // In deviations the weights cancel: s0 + 2 s_out = 1 + D0 + 2 D_out.
  // The inlet is a velocity face (u = u_in, rho from the balance) or, for a
  // pressure inlet (Sec. 4), a pressure face (rho = rho_in, u = 1 - (1 + D0 +
  // 2 D_out) / rho_in) as long as that u stays within the cap u_in, else a
  // velocity face at the cap; pface reports a pressure face (the outlet
  // always is one).
  __device__ static __forceinline__ void zou_he(const KParams& P, bool inlet, float* d, float& rho,
                                                float& drho, float* u) {
    bool pface;
    zou_he(P, inlet, d, rho, drho, u, pface);
  }
  __device__ static __forceinline__ void zou_he(const KParams& P, bool inlet, float* d, float& rho,
                                                float& drho, float* u, bool& pface) {
    float D0 = 0.0f, Dout = 0.0f, Ny = 0.0f, Nz = 0.0f;
    const int sgn = inlet ? 1 : -1;  // inward normal along x
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int en = L::ex(i) * sgn;
      if (en == 0) {
        D0 += d[i];
        if (L::ey(i)) Ny += float(L::ey(i)) * d[i];
        if (L::ez(i)) Nz += float(L::ez(i)) * d[i];
      } else if (en < 0) {
        Dout += d[i];
      }
    }
    Ny *= 0.5f;
    Nz *= 0.5f;
    if (inlet) {
      pface = false;
      if (P.inlet_kind == 1) {
        const float up = (P.drho_in - D0 - 2.0f * Dout) * P.inv_rho_in;
        if (up <= P.u_in) {
          pface = true;
          rho = P.rho_in;
          drho = P.drho_in;
          u[0] = up;
        }
      }
      if (!pface) {
        drho = (D0 + 2.0f * Dout + P.u_in) * P.inv_1m_uin;
        rho = 1.0f + drho;
        u[0] = P.u_in;
      }
    } else {
      pface = true;
      rho = P.rho_out;
      drho = P.drho_out;
      u[0] = (D0 + 2.0f * Dout + P.one_m_rho_out) / P.rho_out;
    }
    u[1] = 0.0f;
    u[2] = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (L::ex(i) * sgn > 0) {
        float v = d[L::opp(i)] + 6.0f * L::w(i) * rho * float(L::ex(i)) * u[0];
        if (L::ey(i)) v -= float(L::ey(i)) * Ny;
        if (L::ez(i)) v -= float(L::ez(i)) * Nz;
        d[i] = v;
      }
    }
  }

  __device__ static __forceinline__ void moments(const float* d, float& rho, float& drho, float* u) {
    float s = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      s += d[i];
      if (L::ex(i)) jx += float(L::ex(i)) * d[i];
      if (L::ey(i)) jy += float(L::ey(i)) * d[i];
      if (L::ez(i)) jz += float(L::ez(i)) * d[i];
    }
    drho = s;
    rho = 1.0f + s;
    const float ir = rcp(rho);
    u[0] = jx * ir;
    u[1] = jy * ir;
    u[2] = jz * ir;
  }

  __device__ static __forceinline__ float deq(int i, float rho, float drho, const float* u, float uu) {
    const float eu = float(L::ex(i)) * u[0] + float(L::ey(i)) * u[1] + float(L::ez(i)) * u[2];
    return L::w(i) * (drho + rho * (3.0f * eu + 4.5f * eu * eu - 1.5f * uu));
  }

  // Outlet scalar: unknowns (e_x < 0) at equilibrium with the node's own
  // value T*, T* = sum_known g / (1 - sum_unknown w_i (1 + e_i.v / cs2)).
  __device__ static __forceinline__ void scalar_outlet(float* g, const float* v, float& T, float& den) {
    float sk = 0.0f, su = 0.0f;
#pragma unroll
    for (int i = 0; i < QS; ++i) {
      if (LS::ex(i) >= 0) {
        sk += g[i];
      } else {
        const float ev = float(LS::ex(i)) * v[0] + float(LS::ey(i)) * v[1] + float(LS::ez(i)) * v[2];
        su += LS::w(i) * (1.0f + ev * (1.0f / LS::cs2));
      }
    }
    den = 1.0f - su;
    T = sk / den;
#pragma unroll
    for (int i = 0; i < QS; ++i) {
      if (LS::ex(i) < 0) {
        const float ev = float(LS::ex(i)) * v[0] + float(LS::ey(i)) * v[1] + float(LS::ez(i)) * v[2];
        g[i] = LS::w(i) * T * (1.0f + ev * (1.0f / LS::cs2));
      }
    }
  }

  // prescribed inlet value of scalar s on row y: 1 halves (0 below ny/2, 1
  // above, odd scalars 1 - c), 2 signed (-1 below, +1 above, odd scalars -c)
  __device__ static __forceinline__ float inlet_value(const KParams& P, int s, int y) {
    const bool upper = y >= P.ny / 2;
    if (P.scalar_inlet == 1) {
      const float c = upper ? 1.0f : 0.0f;
      return (s & 1) ? 1.0f - c : c;
    }
    if (P.scalar_inlet == 2) {
      const float c = upper ? 1.0f : -1.0f;
      return (s & 1) ? -c : c;
    }
    return 0.0f;
  }

  // -------------------------------------------------------------------------
  // Fluid collision of a node in polynomial form.  With r the factor that
  // BGK keeps of the non-equilibrium part (1 - omega), or that MRT keeps of
  // the moments outside the stress set (1 - s_other),
  //   deq(v) + r (d - deq(u))                               (BGK)
  //   deq(v) + r (d - deq(u)) + sum_k U_k m_k               (MRT, k stress)
  // where m_k = c_k U_k.(d - deq(u)).  Because deq_i(rho, u) = w_i (drho +
  // rho (3 e.u + 4.5 (e.u)^2 - 1.5 u.u)) is a quadratic polynomial in e_i,
  //   deq_i(v) - r deq_i(u) = w_i (K0 + e_i.A + e_i^T Pi e_i),
  //   K0 = (1 - r) drho - 1.5 rho (v.v - r u.u),   A = 3 rho (v - r u),
  //   Pi = 4.5 rho (v v^T - r u u^T),
  // a handful of node constants instead of two equilibria per population;
  // the stress moments of deq(u) are rho 4.5 u^T M_k u with the constant
  // weighted second moments M_k = sum_i w_i U_ki e_i e_i^T (its zeroth and
  // first weighted moments vanish for the stress rows).  Same operator as
  // the direct form (ALBM_COLLIDE_DIRECT), up to rounding.
  // -------------------------------------------------------------------------
  // With FOLD, d holds the stored values d - dev_off of 16-bit storage on
  // entry and on exit: the offsets enter the stress moments (their stress
  // moments are rho = 1, u = u_ref ones) and the output through the
  // constant (r - 1) dev_off_i.
  template <bool FOLD = false>
  __device__ static __forceinline__ void collide_fluid(const KParams& P, float* d, float rho,
                                                       float drho, const float* u, const float* v,
                                                       float uu, float vv) {
    const float r = MRT ? P.mrt_diag : P.one_m_omega;
    const float K0 = (1.0f - r) * drho - 1.5f * rho * (vv - r * uu);
    float A[3], Pm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      A[a] = 3.0f * rho * (v[a] - r * u[a]);
#pragma unroll
      for (int b = a; b < 3; ++b) Pm[a][b] = 4.5f * rho * (v[a] * v[b] - r * (u[a] * u[b]));
    }
    float mk[L::NMOM];
    if constexpr (MRT) {
      // stress moments of d - deq(u), weighted by c_k
#pragma unroll
      for (int k = 0; k < L::NMOM; ++k) {
        mk[k] = 0.0f;
        if (!L::stress(k)) continue;
        float a = 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i)
          if (L::U(k, i) != 0) a += float(L::U(k, i)) * d[i];
        float eq = 0.0f, eo = 0.0f;
#pragma unroll
        for (int p_ = 0; p_ < 3; ++p_)
#pragma unroll
          for (int q_ = 0; q_ < 3; ++q_)
            if (UW2(k, p_, q_) != 0) {
              eq += (float(UW2(k, p_, q_)) * (4.5f / 36.0f)) * (u[p_] * u[q_]);
              if (FOLD) eo += (float(UW2(k, p_, q_)) * (4.5f / 36.0f)) * (P.j_off[p_] * P.j_off[q_]);
            }
        mk[k] = P.mrt_r[k] * (a + eo - rho * eq);
      }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
      float quad = K0;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b)
          if (e[a] * e[b] != 0) quad += float((a == b ? 1 : 2) * e[a] * e[b]) * Pm[a][b];
      float lin = 0.0f;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (e[a] != 0) lin += float(e[a]) * A[a];
      float y = r * d[i] + L::w(i) * (quad + lin);
      if constexpr (FOLD) y += (r - 1.0f) * P.dev_off[i];
      if constexpr (MRT) {
#pragma unroll
        for (int k = 0; k < L::NMOM; ++k)
          if (L::stress(k) && L::U(k, i) != 0) y += float(L::U(k, i)) * mk[k];
      }
      d[i] = y;
    }
  }

  // -------------------------------------------------------------------------
  // Forward: W^x applied to d (fluid deviations) and g (scalars) in place.
  // obj1/obj2 receive this node's objective terms F^x(f^n(x)).  OBJ is the
  // objective form compiled in (see obj_kind): 0 none, 1 outlet/inlet
  // objectives only, 2 all (with the dissipation of every fluid node).
  // -------------------------------------------------------------------------
  template <int OBJ = 2, bool FOLD = false>
  __device__ static __forceinline__ void forward(const KParams& P, uint8_t type, float th, int y,
                                                 float* d, float (*g)[QS], bool want_obj,
                                                 double& obj1, double& obj2) {
    if constexpr (FOLD) {
      // d holds the stored values of 16-bit storage (d - dev_off)
      if (type != FLUID) {
        // boundary nodes take the deviations themselves
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] += P.dev_off[i];
        forward<OBJ, false>(P, type, th, y, d, g, want_obj, obj1, obj2);
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] -= P.dev_off[i];
        return;
      }
      float sum = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        sum += d[i];
        if (L::ex(i)) jx += float(L::ex(i)) * d[i];
        if (L::ey(i)) jy += float(L::ey(i)) * d[i];
        if (L::ez(i)) jz += float(L::ez(i)) * d[i];
      }
      const float drho = sum + P.drho_off;
      const float rho = 1.0f + drho;
      const float ir = rcp(rho);
      float u[3] = {(jx + P.j_off[0]) * ir, (jy + P.j_off[1]) * ir, (jz + P.j_off[2]) * ir};
      if (OBJ == 2 && want_obj && P.objective == OBJ_DISSIPATION) {
        float dt[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) dt[i] = d[i] + P.dev_off[i];
        obj1 += (double)dissipation(P, dt, rho, drho, u);
      }
      float G, dG;
      porosity_G(P, th, G, dG);
      float v[3] = {G * u[0] + P.gx, G * u[1] + P.gy, G * u[2] + P.gz};
      const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
      const float vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
      collide_fluid<true>(P, d, rho, drho, u, v, uu, vv);
      scalars_forward<OBJ>(P, type, th, y, g, u, v, rho, want_obj, obj1, obj2);
      return;
    }
    if (type == WALL || type == HOT) {
      float t[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) t[i] = d[L::opp(i)];
#pragma unroll
      for (int i = 0; i < Q; ++i) d[i] = t[i];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (type == WALL) {
          float tg[QS];
#pragma unroll
          for (int i = 0; i < QS; ++i) tg[i] = g[s][LS::opp(i)];
#pragma unroll
          for (int i = 0; i < QS; ++i) g[s][i] = tg[i];
        } else {
#pragma unroll
          for (int i = 0; i < QS; ++i) g[s][i] = LS::w(i) * P.T_hot;
        }
      }
      return;
    }
    float rho, drho, u[3];
    if (type == INLET) {
      zou_he(P, true, d, rho, drho, u);
    } else if (type == OUTLET) {
      zou_he(P, false, d, rho, drho, u);
    } else {
      moments(d, rho, drho, u);
    }
    if (OBJ == 2 && want_obj && P.objective == OBJ_DISSIPATION && type == FLUID) {
      obj1 += (double)dissipation(P, d, rho, drho, u);
    }
    float G, dG;
    porosity_G(P, th, G, dG);
    float v[3] = {G * u[0] + P.gx, G * u[1] + P.gy, G * u[2] + P.gz};
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
#if ALBM_COLLIDE_DIRECT
    if (MRT) {
      float neq[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) neq[i] = d[i] - deq(i, rho, drho, u, uu);
      float mn[Q];
      mrt_op(P, neq, mn);
#pragma unroll
      for (int i = 0; i < Q; ++i) d[i] = deq(i, rho, drho, v, vv) + mn[i];
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        d[i] = deq(i, rho, drho, v, vv) + P.one_m_omega * (d[i] - deq(i, rho, drho, u, uu));
      }
    }
#else
    collide_fluid(P, d, rho, drho, u, v, uu, vv);
#endif
    scalars_forward<OBJ>(P, type, th, y, g, u, v, rho, want_obj, obj1, obj2);
  }

  // Scalar lattices of one node after its fluid collision (u: the fluid's
  // pre-collision or face velocity, v: its post-collision velocity), with
  // the outlet and inlet objective terms.
  template <int OBJ>
  __device__ static __forceinline__ void scalars_forward(const KParams& P, uint8_t type, float th,
                                                         int y, float (*g)[QS], const float* u,
                                                         const float* v, float rho, bool want_obj,
                                                         double& obj1, double& obj2) {
    if (NS == 0) return;
    float om, dom;
    scalar_rate<LS>(P, th, om, dom);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (type == INLET) {
        const float c = inlet_value(P, s, y);
#pragma unroll
        for (int i = 0; i < QS; ++i)
          g[s][i] = LS::w(i) * c * (1.0f + float(LS::ex(i)) * u[0] * (1.0f / LS::cs2));
        continue;
      }
      float T, den;
      if (type == OUTLET) {
        scalar_outlet(g[s], v, T, den);
        if (OBJ != 0 && want_obj && s == 0) {
          if (P.objective == OBJ_VARIANCE) {
            obj1 += (double)T;
            obj2 += (double)T * (double)T;
          } else if (P.objective == OBJ_HEATFLUX_DP || P.objective == OBJ_HEATFLUX) {
            obj1 += (double)v[0] * (double)T;
          } else if (P.objective == OBJ_MIXFLUX) {
            obj1 += (double)v[0] * (1.0 - (double)T * (double)T);
          }
        }
      } else {
        T = 0.0f;
#pragma unroll
        for (int i = 0; i < QS; ++i) T += g[s][i];
      }
#if ALBM_SCALAR_DIRECT
#pragma unroll
      for (int i = 0; i < QS; ++i) {
        const float ev = float(LS::ex(i)) * v[0] + float(LS::ey(i)) * v[1] + float(LS::ez(i)) * v[2];
        const float geq = LS::w(i) * T * (1.0f + ev * (1.0f / LS::cs2));
        g[s][i] = g[s][i] + om * (geq - g[s][i]);
      }
#else
      // (1 - om) g + om geq with om geq_i = w_i (a0 + e_i.a1): node
      // constants a0 = om T and a1 = om T v / cs2
      const float a0 = om * T;
      const float c1 = a0 * (1.0f / LS::cs2);
      const float a1[3] = {c1 * v[0], c1 * v[1], c1 * v[2]};
      const float keep = 1.0f - om;
#pragma unroll
      for (int i = 0; i < QS; ++i) {
        float t = a0;
        if (LS::ex(i)) t += float(LS::ex(i)) * a1[0];
        if (LS::ey(i)) t += float(LS::ey(i)) * a1[1];
        if (LS::ez(i)) t += float(LS::ez(i)) * a1[2];
        g[s][i] = keep * g[s][i] + LS::w(i) * t;
      }
#endif
    }
    if (want_obj && type == INLET && P.objective == OBJ_HEATFLUX_DP) {
      obj1 += -0.1 / 3.0 * (double)rho * (double)P.inv_A_in;
    }
  }

  // Viscous dissipation 2 rho nu S:S of one node with
  // S_ab = -(3 omega / (2 rho)) Pi_ab, Pi_ab = sum_i e_ia e_ib (f_i - feq_i)
  //      = sum_i e_ia e_ib d_i - drho/3 delta_ab - j_a j_b / rho.
  __device__ static __forceinline__ float dissipation(const KParams& P, const float* d, float rho,
                                                      float drho, const float* u) {
    float Pi[3][3];
    pi_neq(d, rho, drho, u, Pi);
    float s = 0.0f;
#pragma unroll
    for (int a = 0; a < L::DIM; ++a)
#pragma unroll
      for (int b = 0; b < L::DIM; ++b) s += Pi[a][b] * Pi[a][b];
    const float K = 9.0f * P.omega * P.omega * P.nu / rho;
    return 0.5f * K * s;
  }

  __device__ static __forceinline__ void pi_neq(const float* d, float rho, float drho, const float* u,
                                                float (*Pi)[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Pi[a][b] = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
#pragma unroll
      for (int a = 0; a < L::DIM; ++a)
#pragma unroll
        for (int b = a; b < L::DIM; ++b)
          if (e[a] * e[b] != 0) Pi[a][b] += float(e[a] * e[b]) * d[i];
    }
#pragma unroll
    for (int a = 0; a < L::DIM; ++a) {
#pragma unroll
      for (int b = a; b < L::DIM; ++b) {
        float v = Pi[a][b] - rho * u[a] * u[b];
        if (a == b) v -= drho * (1.0f / 3.0f);
        Pi[a][b] = v;
        Pi[b][a] = v;
      }
    }
  }

  // -------------------------------------------------------------------------
  // Reverse: given f^n(x) (d, g) and the adjoint weights a (fluid), b
  // (scalars) of the node's outputs W^x, compute
  //   lam_k  = sum_j a_j dW_j/dd_k + ws dF/dd_k,   lamg likewise,
  //   dth    = sum_j a_j dW_j/dtheta + ws dF/dtheta.
  // ws is the objective weight c_n of this step, cbar the outlet mean of
  // scalar 0 at this step (variance objective).
  // -------------------------------------------------------------------------
  // The adjoint weights are fetched by load(a, b) only after the forward
  // quantities are recomputed (two phases: f^n first, lambda^{n+1} second),
  // which bounds the number of values live in registers at once.  SRC is
  // the source form compiled in (see obj_kind): 0 none, for steps whose
  // weight ws is zero (the sources would add exact zeros), 1 outlet/inlet
  // objectives only, 2 all (the dissipation source of every fluid node).
  template <class Loader, int SRC = 2>
  __device__ static __forceinline__ void reverse(const KParams& P, uint8_t type, float th, int y,
                                                 const float* d_in, float (*g)[QS],
                                                 const Loader& load, float ws, float cbar,
                                                 float* lam, float (*lamg)[QS], float& dth) {
    dth = 0.0f;
    float a[Q], b[NSA][QS];
    if (type == WALL || type == HOT) {
      load(a, b);
#pragma unroll
      for (int k = 0; k < Q; ++k) lam[k] = a[L::opp(k)];
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int k = 0; k < QS; ++k) lamg[s][k] = (type == WALL) ? b[s][LS::opp(k)] : 0.0f;
      return;
    }
    // ---- forward recomputation ----
    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = d_in[i];
    float rho, drho, u[3];
    bool pface = false;   // the face of a boundary node holds rho (u follows)
    if (type == INLET) {
      zou_he(P, true, d, rho, drho, u, pface);
    } else if (type == OUTLET) {
      zou_he(P, false, d, rho, drho, u, pface);
    } else {
      moments(d, rho, drho, u);
    }
    float G, dG;
    porosity_G(P, th, G, dG);
    const float v[3] = {G * u[0] + P.gx, G * u[1] + P.gy, G * u[2] + P.gz};
    float dv[3] = {0.0f, 0.0f, 0.0f};
    float ddrho = 0.0f;
    float src[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) src[k] = 0.0f;
    float dT0 = 0.0f;  // d(objective)/d(T of scalar 0)
    float T[NSA], den[NSA];
    float om = 1.0f, dom = 0.0f;
    if (NS > 0) {
      scalar_rate<LS>(P, th, om, dom);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        den[s] = 1.0f;
        if (type == OUTLET) {
          scalar_outlet(g[s], v, T[s], den[s]);
        } else {
          float t = 0.0f;
#pragma unroll
          for (int i = 0; i < QS; ++i) t += g[s][i];
          T[s] = t;
        }
      }
    }
    // ---- objective sources ws * dF^x ----
    if (SRC != 0 && ws != 0.0f) {
      if (SRC == 2 && P.objective == OBJ_DISSIPATION && type == FLUID) {
        float Pi[3][3];
        pi_neq(d, rho, drho, u, Pi);
        float s2 = 0.0f, tr = 0.0f;
#pragma unroll
        for (int a_ = 0; a_ < L::DIM; ++a_) {
          tr += Pi[a_][a_];
#pragma unroll
          for (int b_ = 0; b_ < L::DIM; ++b_) s2 += Pi[a_][b_] * Pi[a_][b_];
        }
        const float ir = rcp(rho);
        const float K = 9.0f * P.omega * P.omega * P.nu * ir;
        const float Phi = 0.5f * K * s2;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          const float e[3] = {float(L::ex(k)) - u[0], float(L::ey(k)) - u[1], float(L::ez(k)) - u[2]};
          float q = 0.0f;
#pragma unroll
          for (int a_ = 0; a_ < L::DIM; ++a_)
#pragma unroll
            for (int b_ = 0; b_ < L::DIM; ++b_) q += e[a_] * Pi[a_][b_] * e[b_];
          src[k] = ws * (K * (q - tr * (1.0f / 3.0f)) - Phi * ir);
        }
      } else if (NS > 0 && type == OUTLET) {
        const float T0 = T[0];
        if (P.objective == OBJ_VARIANCE) {
          dT0 = ws * 2.0f * (T0 - cbar) * P.inv_A_out;
        } else if (P.objective == OBJ_HEATFLUX_DP || P.objective == OBJ_HEATFLUX) {
          dv[0] += ws * T0;
          dT0 = ws * v[0];
        } else if (P.objective == OBJ_MIXFLUX) {
          dv[0] += ws * (1.0f - T0 * T0);
          dT0 = ws * (-2.0f * v[0] * T0);
        }
      } else if (type == INLET && P.objective == OBJ_HEATFLUX_DP) {
        ddrho += ws * (-0.1f / 3.0f) * P.inv_A_in;
      }
    }
#if ALBM_ADJ_TWO_PHASE
    asm volatile("" ::: "memory");  // keep the lambda gathers after this point
#endif
    load(a, b);
    // ---- scalar lattices ----
    float du_in = 0.0f;   // d(objective)/d(u_x) through the inlet scalars of a pressure face
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (type == INLET) {
        if (pface) {
          // g_i = w_i c (1 + e_ix u_x / cs2) with the face velocity u_x
          const float c = inlet_value(P, s, y);
#pragma unroll
          for (int k = 0; k < QS; ++k)
            if (LS::ex(k)) du_in += b[s][k] * (LS::w(k) * c * float(LS::ex(k)) * (1.0f / LS::cs2));
        }
#pragma unroll
        for (int k = 0; k < QS; ++k) lamg[s][k] = 0.0f;
        continue;
      }
      float B0 = 0.0f, B1[3] = {0.0f, 0.0f, 0.0f}, bgsum = 0.0f;
#pragma unroll
      for (int i = 0; i < QS; ++i) {
        const float bw = b[s][i] * LS::w(i);
        B0 += bw;
        if (LS::ex(i)) B1[0] += float(LS::ex(i)) * bw;
        if (LS::ey(i)) B1[1] += float(LS::ey(i)) * bw;
        if (LS::ez(i)) B1[2] += float(LS::ez(i)) * bw;
        const float ev = float(LS::ex(i)) * v[0] + float(LS::ey(i)) * v[1] + float(LS::ez(i)) * v[2];
        bgsum += b[s][i] * (LS::w(i) * T[s] * (1.0f + ev * (1.0f / LS::cs2)) - g[s][i]);
      }
      const float B1v = B1[0] * v[0] + B1[1] * v[1] + B1[2] * v[2];
      float dTs = om * (B0 + B1v * (1.0f / LS::cs2)) + (s == 0 ? dT0 : 0.0f);
      const float cT = om * T[s] * (1.0f / LS::cs2);
      dv[0] += cT * B1[0];
      dv[1] += cT * B1[1];
      dv[2] += cT * B1[2];
      dth += dom * bgsum;
      if (type == OUTLET) {
        // chain through g_i = w_i T* phi_i (unknowns) and T* = S_known / den
        float dTstar = dTs;
        float wex = 0.0f, wey = 0.0f, wez = 0.0f;  // sum over unknowns of w_i e_i
#pragma unroll
        for (int i = 0; i < QS; ++i) {
          if (LS::ex(i) < 0) {
            const float lg = (1.0f - om) * b[s][i];
            const float ev = float(LS::ex(i)) * v[0] + float(LS::ey(i)) * v[1] + float(LS::ez(i)) * v[2];
            dTstar += lg * LS::w(i) * (1.0f + ev * (1.0f / LS::cs2));
            const float c = lg * LS::w(i) * T[s] * (1.0f / LS::cs2);
            dv[0] += c * float(LS::ex(i));
            dv[1] += c * float(LS::ey(i));
            dv[2] += c * float(LS::ez(i));
            wex += LS::w(i) * float(LS::ex(i));
            wey += LS::w(i) * float(LS::ey(i));
            wez += LS::w(i) * float(LS::ez(i));
          }
        }
        const float iden = 1.0f / den[s];
        const float cv = dTstar * T[s] * iden * (1.0f / LS::cs2);
        dv[0] += cv * wex;
        dv[1] += cv * wey;
        dv[2] += cv * wez;
#pragma unroll
        for (int k = 0; k < QS; ++k)
          lamg[s][k] = (LS::ex(k) >= 0) ? (1.0f - om) * b[s][k] + dTstar * iden : 0.0f;
      } else {
#pragma unroll
        for (int k = 0; k < QS; ++k) lamg[s][k] = (1.0f - om) * b[s][k] + dTs;
      }
    }
    // ---- fluid collision ----
    // c = (d W / d f_noneq)^T a: (1 - omega) a for BGK; the symmetric MRT
    // operator diag a + sum_k U_k m_k (stress and conserved moments k)
    float c[Q], mk[L::NMOM];
    if (MRT) {
      mrt_op_m(P, a, c, mk);
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) c[i] = P.one_m_omega * a[i];
    }
    // weighted moments A of a and C of c (0th, 1st, 2nd order in e)
    float A0 = 0.0f, A1[3] = {0.0f, 0.0f, 0.0f}, A2[3][3];
    float C0, C1[3], C2[3][3];
#pragma unroll
    for (int p_ = 0; p_ < 3; ++p_)
#pragma unroll
      for (int q_ = 0; q_ < 3; ++q_) A2[p_][q_] = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
      const float aw = a[i] * L::w(i);
      A0 += aw;
#pragma unroll
      for (int p_ = 0; p_ < 3; ++p_) {
        if (e[p_]) {
          A1[p_] += float(e[p_]) * aw;
#pragma unroll
          for (int q_ = p_; q_ < 3; ++q_)
            if (e[q_]) A2[p_][q_] += float(e[p_] * e[q_]) * aw;
        }
      }
    }
#if ALBM_MRT_FULL || ALBM_C_LOOP
    if (MRT || ALBM_C_LOOP) {
      C0 = 0.0f;
#pragma unroll
      for (int p_ = 0; p_ < 3; ++p_) {
        C1[p_] = 0.0f;
#pragma unroll
        for (int q_ = 0; q_ < 3; ++q_) C2[p_][q_] = 0.0f;
      }
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
        const float cw = c[i] * L::w(i);
        C0 += cw;
#pragma unroll
        for (int p_ = 0; p_ < 3; ++p_) {
          if (e[p_]) {
            C1[p_] += float(e[p_]) * cw;
#pragma unroll
            for (int q_ = p_; q_ < 3; ++q_)
              if (e[q_]) C2[p_][q_] += float(e[p_] * e[q_]) * cw;
          }
        }
      }
    } else
#endif
    {
      // C = diag A + sum_k m_k (weighted moments of U_k): the moments of the
      // rows of U are compile-time constants, mostly zero by symmetry
      const float diag = MRT ? P.mrt_diag : P.one_m_omega;
      C0 = diag * A0;
#pragma unroll
      for (int p_ = 0; p_ < 3; ++p_) {
        C1[p_] = diag * A1[p_];
#pragma unroll
        for (int q_ = p_; q_ < 3; ++q_) C2[p_][q_] = diag * A2[p_][q_];
      }
      if (MRT) add_row_moments(std::make_integer_sequence<int, L::NMOM>{}, mk, C0, C1, C2);
    }
#pragma unroll
    for (int p_ = 0; p_ < 3; ++p_)
#pragma unroll
      for (int q_ = 0; q_ < p_; ++q_) {
        A2[p_][q_] = A2[q_][p_];
        C2[p_][q_] = C2[q_][p_];
      }
    float A2v[3], C2u[3];
#pragma unroll
    for (int p_ = 0; p_ < 3; ++p_) {
      A2v[p_] = A2[p_][0] * v[0] + A2[p_][1] * v[1] + A2[p_][2] * v[2];
      C2u[p_] = C2[p_][0] * u[0] + C2[p_][1] * u[1] + C2[p_][2] * u[2];
    }
    const float vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float Qa = 3.0f * (A1[0] * v[0] + A1[1] * v[1] + A1[2] * v[2]) +
                     4.5f * (A2v[0] * v[0] + A2v[1] * v[1] + A2v[2] * v[2]) - 1.5f * A0 * vv;
    const float Qc = 3.0f * (C1[0] * u[0] + C1[1] * u[1] + C1[2] * u[2]) +
                     4.5f * (C2u[0] * u[0] + C2u[1] * u[1] + C2u[2] * u[2]) - 1.5f * C0 * uu;
    ddrho += (A0 + Qa) - (C0 + Qc);
    float du[3];
#pragma unroll
    for (int p_ = 0; p_ < 3; ++p_) {
      dv[p_] += rho * (3.0f * A1[p_] + 9.0f * A2v[p_] - 3.0f * A0 * v[p_]);
      du[p_] = G * dv[p_] - rho * (3.0f * C1[p_] + 9.0f * C2u[p_] - 3.0f * C0 * u[p_]);
    }
    dth += dG * (u[0] * dv[0] + u[1] * dv[1] + u[2] * dv[2]);
#pragma unroll
    for (int k = 0; k < Q; ++k) lam[k] = c[k] + src[k];
    if (type == FLUID) {
      const float ir = rcp(rho);
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const float eu = (float(L::ex(k)) - u[0]) * du[0] + (float(L::ey(k)) - u[1]) * du[1] +
                         (float(L::ez(k)) - u[2]) * du[2];
        lam[k] += ddrho + eu * ir;
      }
      return;
    }
    // ---- Zou-He transpose ----
    const bool inlet = (type == INLET);
    const int sgn = inlet ? 1 : -1;
    // total sensitivity of the face's free scalar: rho on a velocity face,
    // u_x on a pressure face (the outlet, an uncapped pressure inlet)
    float dface = pface ? du[0] + du_in : ddrho;
    float dNy = 0.0f, dNz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (L::ex(i) * sgn > 0) {
        const float coef = 6.0f * L::w(i) * float(L::ex(i));
        dface += lam[i] * coef * (pface ? rho : u[0]);
        if (L::ey(i)) dNy -= lam[i] * float(L::ey(i));
        if (L::ez(i)) dNz -= lam[i] * float(L::ez(i));
      }
    }
    // d(face scalar)/d(D0) and /d(Dout) = k1, 2 k1: velocity face rho = (1 +
    // D0 + 2 Dout) / (1 - u_in); outlet u_x = (1 + D0 + 2 Dout) / rho_out - 1;
    // pressure inlet u_x = 1 - (1 + D0 + 2 Dout) / rho_in
    const float k1 = !pface ? P.inv_1m_uin : (inlet ? -P.inv_rho_in : 1.0f / P.rho_out);
    float out[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int en = L::ex(k) * sgn;
      if (en > 0) {
        out[k] = 0.0f;
      } else if (en < 0) {
        out[k] = lam[k] + lam[L::opp(k)] + 2.0f * k1 * dface;
      } else {
        out[k] = lam[k] + k1 * dface + 0.5f * (float(L::ey(k)) * dNy + float(L::ez(k)) * dNz);
      }
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) lam[k] = out[k];
  }
};

}  // namespace albm
