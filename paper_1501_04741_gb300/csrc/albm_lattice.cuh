// Velocity sets and MRT moment polynomials for the device kernels.
//
// D3Q19 is the list e1..e19 of Sec. 3 in the paper's order (index 0 = rest);
// D3Q7 is its first 7 vectors (heat transfer, Sec. 3); D2Q9 keeps the z = 0
// members of that list in order ({e1..e5, e8..e11}, "reduced to 9" in 2D).
// Weights are the standard ones of each set; c_s^2 = 1/3 for the fluid sets
// and 1/4 for D3Q7.
//
// The MRT matrix U of Sec. 3.1 is the orthogonal polynomial basis of
// d'Humieres et al. (2002) for D3Q19 and of Lallemand & Luo (2000) for
// D2Q9.  Every entry is a constexpr function of the integer velocity, so
// fully unrolled loops fold the zeros and unit coefficients away.
#pragma once

namespace albm {

struct D2Q9 {
  static constexpr int Q = 9;
  static constexpr int DIM = 2;
  static constexpr float cs2 = 1.0f / 3.0f;
  __host__ __device__ static constexpr int ex(int i) {
    constexpr int t[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    return t[i];
  }
  __host__ __device__ static constexpr int ey(int i) {
    constexpr int t[9] = {0, 0, 0, 1, -1, 1, 1, -1, -1};
    return t[i];
  }
  __host__ __device__ static constexpr int ez(int) { return 0; }
  __host__ __device__ static constexpr int opp(int i) {
    constexpr int t[9] = {0, 2, 1, 4, 3, 8, 7, 6, 5};
    return t[i];
  }
  __host__ __device__ static constexpr float w(int i) {
    return i == 0 ? 4.0f / 9.0f : (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
  }
  // Lallemand & Luo moments: rho, e, eps, jx, qx, jy, qy, pxx, pxy
  static constexpr int NMOM = 9;
  __host__ __device__ static constexpr int U(int k, int i) {
    const int x = ex(i), y = ey(i), c2 = x * x + y * y;
    switch (k) {
      case 0: return 1;
      case 1: return -4 + 3 * c2;
      case 2: return (8 - 21 * c2 + 9 * c2 * c2) / 2;
      case 3: return x;
      case 4: return (-5 + 3 * c2) * x;
      case 5: return y;
      case 6: return (-5 + 3 * c2) * y;
      case 7: return x * x - y * y;
      default: return x * y;
    }
  }
  __host__ __device__ static constexpr bool conserved(int k) { return k == 0 || k == 3 || k == 5; }
  __host__ __device__ static constexpr bool stress(int k) { return k == 7 || k == 8; }
};

struct D3Q19 {
  static constexpr int Q = 19;
  static constexpr int DIM = 3;
  static constexpr float cs2 = 1.0f / 3.0f;
  __host__ __device__ static constexpr int ex(int i) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
  }
  __host__ __device__ static constexpr int ey(int i) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
  }
  __host__ __device__ static constexpr int ez(int i) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
    return t[i];
  }
  __host__ __device__ static constexpr int opp(int i) {
    constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15};
    return t[i];
  }
  __host__ __device__ static constexpr float w(int i) {
    return i == 0 ? 1.0f / 3.0f : (i < 7 ? 1.0f / 18.0f : 1.0f / 36.0f);
  }
  // d'Humieres et al. moments: rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx,
  // 3pixx, pww, piww, pxy, pyz, pxz, mx, my, mz
  static constexpr int NMOM = 19;
  __host__ __device__ static constexpr int U(int k, int i) {
    const int x = ex(i), y = ey(i), z = ez(i), c2 = x * x + y * y + z * z;
    switch (k) {
      case 0: return 1;
      case 1: return 19 * c2 - 30;
      case 2: return (21 * c2 * c2 - 53 * c2 + 24) / 2;
      case 3: return x;
      case 4: return (5 * c2 - 9) * x;
      case 5: return y;
      case 6: return (5 * c2 - 9) * y;
      case 7: return z;
      case 8: return (5 * c2 - 9) * z;
      case 9: return 3 * x * x - c2;
      case 10: return (3 * c2 - 5) * (3 * x * x - c2);
      case 11: return y * y - z * z;
      case 12: return (3 * c2 - 5) * (y * y - z * z);
      case 13: return x * y;
      case 14: return y * z;
      case 15: return x * z;
      case 16: return (y * y - z * z) * x;
      case 17: return (z * z - x * x) * y;
      default: return (x * x - y * y) * z;
    }
  }
  __host__ __device__ static constexpr bool conserved(int k) {
    return k == 0 || k == 3 || k == 5 || k == 7;
  }
  __host__ __device__ static constexpr bool stress(int k) {
    return k == 9 || k == 11 || k == 13 || k == 14 || k == 15;
  }
};

struct D3Q7 {
  static constexpr int Q = 7;
  static constexpr float cs2 = 0.25f;
  __host__ __device__ static constexpr int ex(int i) { return D3Q19::ex(i); }
  __host__ __device__ static constexpr int ey(int i) { return D3Q19::ey(i); }
  __host__ __device__ static constexpr int ez(int i) { return D3Q19::ez(i); }
  __host__ __device__ static constexpr int opp(int i) { return D3Q19::opp(i); }
  __host__ __device__ static constexpr float w(int i) { return i == 0 ? 0.25f : 0.125f; }
};

// Scalar lattice paired with each fluid lattice (Sec. 3).
template <class L> struct ScalarOf;
template <> struct ScalarOf<D2Q9> { using type = D2Q9; };
template <> struct ScalarOf<D3Q19> { using type = D3Q7; };

}  // namespace albm
