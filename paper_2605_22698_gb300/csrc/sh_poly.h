// Real spherical harmonics up to l = 3 as Cartesian polynomials of a unit
// vector (x, y, z), orthonormal on the sphere, no Condon-Shortley phase,
// components m = -l..l at index l*l + m + l.  Y_1 = sqrt(3/4pi) (y, z, x).
// These are the angular features of the NequIP/MACE family the paper's
// library implements (Sec. 2; Tables tbl:nequip_params and tbl:mace_params
// list l_max 2 and 3).  Used by the device kernels (float) and by the host
// table generator (double).
#pragma once

#ifdef __CUDACC__
#define MLIP_HD __host__ __device__ __forceinline__
#else
#define MLIP_HD inline
#endif

namespace mlip {

struct ShConst {
  static constexpr double c0 = 0.28209479177387814;   // 1/(2 sqrt(pi))
  static constexpr double c1 = 0.48860251190291992;   // sqrt(3/(4 pi))
  static constexpr double c2a = 1.0925484305920792;   // sqrt(15/pi)/2
  static constexpr double c2b = 0.31539156525252005;  // sqrt(5/pi)/4
  static constexpr double c2c = 0.54627421529603959;  // sqrt(15/pi)/4
  static constexpr double c3a = 0.59004358992664352;  // sqrt(35/(2 pi))/4
  static constexpr double c3b = 2.8906114426405538;   // sqrt(105/pi)/2
  static constexpr double c3c = 0.45704579946446572;  // sqrt(21/(2 pi))/4
  static constexpr double c3d = 0.37317633259011540;  // sqrt(7/pi)/4
  static constexpr double c3e = 1.4453057213202769;   // sqrt(105/pi)/4
};

// Y[0..15] for l <= 3.
template <class T>
MLIP_HD void sh3(T x, T y, T z, T* Y) {
  using K = ShConst;
  const T x2 = x * x, y2 = y * y, z2 = z * z;
  Y[0] = T(K::c0);
  Y[1] = T(K::c1) * y;
  Y[2] = T(K::c1) * z;
  Y[3] = T(K::c1) * x;
  Y[4] = T(K::c2a) * x * y;
  Y[5] = T(K::c2a) * y * z;
  Y[6] = T(K::c2b) * (T(3) * z2 - T(1));
  Y[7] = T(K::c2a) * x * z;
  Y[8] = T(K::c2c) * (x2 - y2);
  Y[9] = T(K::c3a) * y * (T(3) * x2 - y2);
  Y[10] = T(K::c3b) * x * y * z;
  Y[11] = T(K::c3c) * y * (T(5) * z2 - T(1));
  Y[12] = T(K::c3d) * z * (T(5) * z2 - T(3));
  Y[13] = T(K::c3c) * x * (T(5) * z2 - T(1));
  Y[14] = T(K::c3e) * z * (x2 - y2);
  Y[15] = T(K::c3a) * x * (x2 - T(3) * y2);
}

// Contract the polynomial gradients with a cotangent: out = sum_k dY[k] grad P_k
// (gradient of the polynomial in free variables x, y, z; the caller projects
// out the radial part).
template <class T>
MLIP_HD void sh3_vjp(T x, T y, T z, const T* dY, T& gx, T& gy, T& gz) {
  using K = ShConst;
  const T x2 = x * x, y2 = y * y, z2 = z * z;
  T ax = T(0), ay = T(0), az = T(0);
  // l = 1
  ay += T(K::c1) * dY[1];
  az += T(K::c1) * dY[2];
  ax += T(K::c1) * dY[3];
  // l = 2
  ax += T(K::c2a) * y * dY[4];  ay += T(K::c2a) * x * dY[4];
  ay += T(K::c2a) * z * dY[5];  az += T(K::c2a) * y * dY[5];
  az += T(6 * K::c2b) * z * dY[6];
  ax += T(K::c2a) * z * dY[7];  az += T(K::c2a) * x * dY[7];
  ax += T(2 * K::c2c) * x * dY[8];  ay -= T(2 * K::c2c) * y * dY[8];
  // l = 3
  ax += T(6 * K::c3a) * x * y * dY[9];
  ay += T(3 * K::c3a) * (x2 - y2) * dY[9];
  ax += T(K::c3b) * y * z * dY[10];
  ay += T(K::c3b) * x * z * dY[10];
  az += T(K::c3b) * x * y * dY[10];
  ay += T(K::c3c) * (T(5) * z2 - T(1)) * dY[11];
  az += T(10 * K::c3c) * y * z * dY[11];
  az += T(K::c3d) * (T(15) * z2 - T(3)) * dY[12];
  ax += T(K::c3c) * (T(5) * z2 - T(1)) * dY[13];
  az += T(10 * K::c3c) * x * z * dY[13];
  ax += T(2 * K::c3e) * x * z * dY[14];
  ay -= T(2 * K::c3e) * y * z * dY[14];
  az += T(K::c3e) * (x2 - y2) * dY[14];
  ax += T(3 * K::c3a) * (x2 - y2) * dY[15];
  ay -= T(6 * K::c3a) * x * y * dY[15];
  gx = ax; gy = ay; gz = az;
}

}  // namespace mlip
