// FP64 CPU oracle for the equivariant interaction potential (test infrastructure).
//
// This file is the reference against which the CUDA library is checked. It is
// test infrastructure only: the tests, the smoke check and the CPU-baseline leg
// of the benchmark load it; the library never does. It shares no code, header,
// table or generator with the CUDA path.
//
// What it computes follows the method of arxiv 2605.22698 ("mlip v2"): an
// equivariant message-passing interatomic potential of the NequIP/MACE family
// (Sec. 2 "Background and related work", Sec. 4 "Accelerating equivariant
// operations with e3j"), with energy as a per-atom readout plus reference
// energies (Eq. multihead_readout, one head) and forces as the negative
// position gradient (Eq. full_hessian, first derivative).  The paper prints no
// formula for the layer itself, so the definitions below are the textbook ones
// (real spherical harmonics, Racah's Clebsch-Gordan formula, Bessel basis with
// a polynomial envelope, radial MLP, scatter-sum, channel mix); each function
// names the definition it writes out.  Everything is double precision; the
// model arithmetic is templated on the scalar so that forward-mode dual
// numbers give exact derivatives as an independent check of the hand-written
// reverse pass.  Build with -ffp-contract=off: the neighbour test is defined
// without fused multiply-add.
//
// Parity pins (tests/test_oracle_*.py): closed forms and orthonormality of the
// harmonics, textbook CG values, CG orthogonality and Wigner-D intertwining,
// real CG proportional to Gaunt integrals, rotation/translation/permutation/
// image invariance, supercell extensivity, forces vs dual numbers and finite
// differences, stress vs strain finite differences, dimer closed form,
// brute-force neighbour sets, velocity-Verlet time reversibility.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return {s, a.d / (2.0 * s)}; }
inline Dual sin(Dual a) { return {std::sin(a.v), a.d * std::cos(a.v)}; }
inline Dual exp(Dual a) { double e = std::exp(a.v); return {e, a.d * e}; }
inline double val(double x) { return x; }
inline double val(Dual x) { return x.v; }
using std::sqrt; using std::sin; using std::exp;

// Hyper-dual numbers v + a e1 + b e2 + ab e1 e2 (e1^2 = e2^2 = 0): one pass of
// the templated energy with e1 on coordinate x and e2 on coordinate y gives
// d2E / dx dy exactly in the ab part (forward-over-forward, for the Hessian).
struct HDual {
  double v, a, b, ab;
  HDual() : v(0), a(0), b(0), ab(0) {}
  HDual(double x) : v(x), a(0), b(0), ab(0) {}
  HDual(double x, double da, double db, double dab) : v(x), a(da), b(db), ab(dab) {}
};
// f(x) for a unary function with value f0 and derivatives f1, f2 at x.v
inline HDual chain(const HDual& x, double f0, double f1, double f2) {
  return {f0, f1 * x.a, f1 * x.b, f1 * x.ab + f2 * x.a * x.b};
}
inline HDual operator+(HDual x, HDual y) { return {x.v + y.v, x.a + y.a, x.b + y.b, x.ab + y.ab}; }
inline HDual operator-(HDual x, HDual y) { return {x.v - y.v, x.a - y.a, x.b - y.b, x.ab - y.ab}; }
inline HDual operator-(HDual x) { return {-x.v, -x.a, -x.b, -x.ab}; }
inline HDual operator*(HDual x, HDual y) {
  return {x.v * y.v, x.a * y.v + x.v * y.a, x.b * y.v + x.v * y.b, x.ab * y.v + x.a * y.b + x.b * y.a + x.v * y.ab};
}
inline HDual operator/(HDual x, HDual y) {
  const double iv = 1.0 / y.v;
  return x * chain(y, iv, -iv * iv, 2.0 * iv * iv * iv);
}
inline HDual& operator+=(HDual& x, HDual y) { x = x + y; return x; }
inline HDual& operator-=(HDual& x, HDual y) { x = x - y; return x; }
inline HDual& operator*=(HDual& x, HDual y) { x = x * y; return x; }
inline HDual sqrt(HDual x) { const double s = std::sqrt(x.v); return chain(x, s, 0.5 / s, -0.25 / (s * x.v)); }
inline HDual sin(HDual x) { return chain(x, std::sin(x.v), std::cos(x.v), -std::sin(x.v)); }
inline HDual exp(HDual x) { const double e = std::exp(x.v); return chain(x, e, e, e); }
inline double val(HDual x) { return x.v; }

double factorial(int n) {
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= k;
  return f;
}

// ------------------------------------------------- real spherical harmonics
// Definition: for a unit vector with polar cosine z and azimuth phi,
//   Y_{l,m}  = sqrt(2) N_l^{|m|} P_l^{|m|}(z) cos(m phi)      (m > 0)
//   Y_{l,m}  = sqrt(2) N_l^{|m|} P_l^{|m|}(z) sin(|m| phi)    (m < 0)
//   Y_{l,0}  = N_l^0 P_l(z),
//   N_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
// with P_l^m the associated Legendre function WITHOUT the Condon-Shortley
// phase, P_l^m(z) = (1-z^2)^{m/2} d^m/dz^m P_l(z).  On the unit sphere
// (1-z^2)^{m/2} cos(m phi) = Re (x+iy)^m and (1-z^2)^{m/2} sin(m phi) =
// Im (x+iy)^m, so every value is a polynomial in (x, y, z).  Components are
// stored at index l*l + (m + l), m = -l..l.

// Coefficients of d^m/dz^m P_l(z) as a polynomial in z (index = power).
std::vector<double> legendre_deriv_coeffs(int l, int m) {
  // Rodrigues expansion: P_l(z) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l) z^{l-2k}
  std::vector<double> a(l + 1, 0.0);
  for (int k = 0; 2 * k <= l; ++k) {
    double c = factorial(l) / (factorial(k) * factorial(l - k)) *
               factorial(2 * l - 2 * k) / (factorial(l) * factorial(l - 2 * k));
    a[l - 2 * k] = ((k % 2) ? -c : c) / std::ldexp(1.0, l);
  }
  for (int d = 0; d < m; ++d) {
    std::vector<double> b(a.size(), 0.0);
    for (size_t n = 1; n < a.size(); ++n) b[n - 1] = a[n] * double(n);
    a = b;
  }
  return a;
}

// Cached coefficient table for l <= 8 (built once, read-only afterwards).
struct LegendreTable {
  std::vector<double> q[9][9];
  double N[9][9];
  LegendreTable() {
    for (int l = 0; l <= 8; ++l)
      for (int m = 0; m <= l; ++m) {
        q[l][m] = legendre_deriv_coeffs(l, m);
        N[l][m] = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * factorial(l - m) / factorial(l + m));
      }
  }
};
const LegendreTable& legendre_table() {
  static const LegendreTable t;
  return t;
}

template <class T>
void real_sh_unit(int lmax, T x, T y, T z, T* out) {
  const LegendreTable& tab = legendre_table();
  for (int l = 0; l <= lmax; ++l) {
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      const double N = tab.N[l][am];
      const std::vector<double>& q = tab.q[l][am];
      T Q = T(0.0), zp = T(1.0);
      for (size_t n = 0; n < q.size(); ++n) { Q = Q + T(q[n]) * zp; zp = zp * z; }
      // (x + i y)^am
      T cr = T(1.0), ci = T(0.0);
      for (int k = 0; k < am; ++k) {
        T nr = cr * x - ci * y;
        T ni = cr * y + ci * x;
        cr = nr; ci = ni;
      }
      T v;
      if (m > 0) v = T(std::sqrt(2.0) * N) * Q * cr;
      else if (m < 0) v = T(std::sqrt(2.0) * N) * Q * ci;
      else v = T(N) * Q;
      out[l * l + m + l] = v;
    }
  }
}

// Harmonics of the direction of an arbitrary nonzero vector.
template <class T>
void real_sh_vec(int lmax, T vx, T vy, T vz, T* out) {
  T r = sqrt(vx * vx + vy * vy + vz * vz);
  real_sh_unit(lmax, vx / r, vy / r, vz / r, out);
}

// Complex harmonics with the Condon-Shortley phase:
//   Y_l^m = (-1)^m N_l^m P_l^m(z) e^{i m phi} (m >= 0),  Y_l^{-m} = (-1)^m conj(Y_l^m).
void complex_sh_unit(int l, double x, double y, double z, std::complex<double>* out) {
  for (int m = 0; m <= l; ++m) {
    double N = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * factorial(l - m) / factorial(l + m));
    std::vector<double> q = legendre_deriv_coeffs(l, m);
    double Q = 0, zp = 1;
    for (size_t n = 0; n < q.size(); ++n) { Q += q[n] * zp; zp *= z; }
    std::complex<double> p(1.0, 0.0), b(x, y);
    for (int k = 0; k < m; ++k) p *= b;
    std::complex<double> ypos = ((m % 2) ? -1.0 : 1.0) * N * Q * p;
    out[l + m] = ypos;
    if (m > 0) out[l - m] = ((m % 2) ? -1.0 : 1.0) * std::conj(ypos);
  }
}

// Unitary U_l with Y^real_{l,m} = sum_mu U[m][mu] Y^complex_{l,mu} (rows m, columns mu,
// both -l..l).  From Y^c_{mu} = (-1)^mu N P e^{i mu phi} and Y^c_{-mu} = N P e^{-i mu phi}:
//   m > 0:  Y^r_m  = ((-1)^m Y^c_m + Y^c_{-m}) / sqrt 2
//   m < 0:  Y^r_m  = i (Y^c_{m} - (-1)^{|m|} Y^c_{|m|}) / sqrt 2
//   m = 0:  Y^r_0  = Y^c_0
// The tests verify U Y^c = Y^r at random points rather than trusting this algebra.
void real_basis_U(int l, std::complex<double>* U) {
  int n = 2 * l + 1;
  for (int k = 0; k < n * n; ++k) U[k] = 0.0;
  const double s = 1.0 / std::sqrt(2.0);
  for (int m = -l; m <= l; ++m) {
    int row = m + l;
    if (m == 0) {
      U[row * n + l] = 1.0;
    } else if (m > 0) {
      double sg = (m % 2) ? -1.0 : 1.0;
      U[row * n + (m + l)] = sg * s;
      U[row * n + (-m + l)] = s;
    } else {
      int am = -m;
      double sg = (am % 2) ? -1.0 : 1.0;
      U[row * n + (m + l)] = std::complex<double>(0.0, s);
      U[row * n + (am + l)] = std::complex<double>(0.0, -sg * s);
    }
  }
}

// ------------------------------------------------------------ Clebsch-Gordan
// Complex <l1 m1 l2 m2 | l3 m3> from Racah's closed form.
double cg_complex(int l1, int m1, int l2, int m2, int l3, int m3) {
  if (m3 != m1 + m2) return 0.0;
  if (l3 < std::abs(l1 - l2) || l3 > l1 + l2) return 0.0;
  if (std::abs(m1) > l1 || std::abs(m2) > l2 || std::abs(m3) > l3) return 0.0;
  double pre = std::sqrt((2.0 * l3 + 1.0) * factorial(l3 + l1 - l2) * factorial(l3 - l1 + l2) *
                         factorial(l1 + l2 - l3) / factorial(l1 + l2 + l3 + 1));
  pre *= std::sqrt(factorial(l3 + m3) * factorial(l3 - m3) * factorial(l1 - m1) * factorial(l1 + m1) *
                   factorial(l2 - m2) * factorial(l2 + m2));
  double sum = 0.0;
  for (int k = 0; k <= l1 + l2 + l3 + 1; ++k) {
    int a[6] = {k, l1 + l2 - l3 - k, l1 - m1 - k, l2 + m2 - k, l3 - l2 + m1 + k, l3 - l1 - m2 + k};
    bool ok = true;
    for (int q = 0; q < 6; ++q) if (a[q] < 0) ok = false;
    if (!ok) continue;
    double den = 1.0;
    for (int q = 0; q < 6; ++q) den *= factorial(a[q]);
    sum += ((k % 2) ? -1.0 : 1.0) / den;
  }
  return pre * sum;
}

// Real CG tensor C[m3][m1][m2] (each index -l..l, row-major) of a
// triangle-valid triple: C^r = U_l3 C^c (U_l1^* (x) U_l2^*).  The result is
// real up to one global phase (a power of i: imaginary for odd l1 + l2 + l3,
// the pseudotensor couplings of mixed-parity models), which is removed; then
// the overall sign is fixed so that
// the first entry (lexicographic in m3, m1, m2) with |c| > 1e-8 is positive.
// Entries below 1e-14 in magnitude are set to zero.
void real_cg(int l1, int l2, int l3, double* out) {
  int n1 = 2 * l1 + 1, n2 = 2 * l2 + 1, n3 = 2 * l3 + 1;
  std::vector<std::complex<double>> U1(n1 * n1), U2(n2 * n2), U3(n3 * n3);
  real_basis_U(l1, U1.data()); real_basis_U(l2, U2.data()); real_basis_U(l3, U3.data());
  std::vector<std::complex<double>> R(n3 * n1 * n2, 0.0);
  for (int a = 0; a < n3; ++a)
    for (int b = 0; b < n1; ++b)
      for (int c = 0; c < n2; ++c) {
        std::complex<double> acc = 0.0;
        for (int mu3 = 0; mu3 < n3; ++mu3) {
          if (U3[a * n3 + mu3] == 0.0) continue;
          for (int mu1 = 0; mu1 < n1; ++mu1) {
            if (U1[b * n1 + mu1] == 0.0) continue;
            for (int mu2 = 0; mu2 < n2; ++mu2) {
              if (U2[c * n2 + mu2] == 0.0) continue;
              double cg = cg_complex(l1, mu1 - l1, l2, mu2 - l2, l3, mu3 - l3);
              if (cg == 0.0) continue;
              acc += U3[a * n3 + mu3] * cg * std::conj(U1[b * n1 + mu1]) * std::conj(U2[c * n2 + mu2]);
            }
          }
        }
        R[(a * n1 + b) * n2 + c] = acc;
      }
  // global phase from the largest-magnitude entry
  size_t imax = 0;
  for (size_t k = 0; k < R.size(); ++k) if (std::abs(R[k]) > std::abs(R[imax])) imax = k;
  std::complex<double> ph = R[imax] / std::abs(R[imax]);
  for (size_t k = 0; k < R.size(); ++k) {
    double v = (R[k] * std::conj(ph)).real();
    out[k] = std::fabs(v) < 1e-14 ? 0.0 : v;
  }
  for (size_t k = 0; k < R.size(); ++k) {
    if (std::fabs(out[k]) > 1e-8) {
      if (out[k] < 0) for (size_t q = 0; q < R.size(); ++q) out[q] = -out[q];
      break;
    }
  }
}

// ------------------------------------------------------------------ paths
// Every (l1 <= L, l2 <= Lsh, l3 <= L) with |l1-l2| <= l3 <= l1+l2, in
// lexicographic order of (l1, l2, l3): with l1+l2+l3 even only (natural
// parity), or all of them (all_parities: the mixed-parity model, whose odd
// paths couple features into the opposite parity block).
struct CGEntry { int m3, m1, m2; double c; };
struct Path { int l1, l2, l3; std::vector<CGEntry> nz; };

std::vector<Path> build_paths(int L, int Lsh, bool all_parities = false) {
  std::vector<Path> ps;
  for (int l1 = 0; l1 <= L; ++l1)
    for (int l2 = 0; l2 <= Lsh; ++l2)
      for (int l3 = 0; l3 <= L; ++l3) {
        if (l3 < std::abs(l1 - l2) || l3 > l1 + l2) continue;
        if (!all_parities && (l1 + l2 + l3) % 2) continue;
        Path p{l1, l2, l3, {}};
        int n1 = 2 * l1 + 1, n2 = 2 * l2 + 1, n3 = 2 * l3 + 1;
        std::vector<double> C(n3 * n1 * n2);
        real_cg(l1, l2, l3, C.data());
        for (int a = 0; a < n3; ++a)
          for (int b = 0; b < n1; ++b)
            for (int c = 0; c < n2; ++c) {
              double v = C[(a * n1 + b) * n2 + c];
              if (v != 0.0) p.nz.push_back({a - l3, b - l1, c - l2, v});
            }
        ps.push_back(p);
      }
  return ps;
}

inline int lm(int l, int m) { return l * l + m + l; }

// Couplings of the symmetric contraction of correlation order 2 (MACE's
// product basis, Sec. "Background and related work" and the MACE table's
// "correlation 2"): the node's aggregated features A of orders l1 <= l2 <= L
// are coupled with themselves into order l3 <= L.  Only l1 <= l2 is kept: the
// (l2, l1) coupling of the same A is the same quadratic form (the real CG
// tensor of a natural-parity triple is symmetric under swapping its two
// inputs), and for l1 = l2 natural parity leaves only even l3, whose coupling
// is symmetric, so no kept path vanishes identically.  Lexicographic in
// (l1, l2, l3).
std::vector<Path> build_sc_paths(int L) {
  std::vector<Path> ps;
  for (const Path& p : build_paths(L, L))
    if (p.l1 <= p.l2) ps.push_back(p);
  return ps;
}

// --------------------------------------------------------------- radial part
// Bessel basis B_n(r) = sqrt(2/rc) sin(n pi r / rc) / r and the polynomial
// envelope u(x) = 1 - (p+1)(p+2)/2 x^p + p(p+2) x^{p+1} - p(p+1)/2 x^{p+2}
// for x < 1, 0 otherwise.
template <class T>
T bessel(int n, T r, double rc) {
  return T(std::sqrt(2.0 / rc)) * sin(T(n * kPi / rc) * r) / r;
}
template <class T>
T envelope(T x, int p) {
  if (val(x) >= 1.0) return T(0.0);
  T xp = T(1.0);
  for (int k = 0; k < p; ++k) xp = xp * x;
  double a = (p + 1.0) * (p + 2.0) / 2.0, b = p * (p + 2.0), c = p * (p + 1.0) / 2.0;
  return T(1.0) - T(a) * xp + T(b) * xp * x - T(c) * xp * x * x;
}
template <class T>
T silu(T x) { return x / (T(1.0) + exp(-x)); }
template <class T>
T sigmoid(T x) { return T(1.0) / (T(1.0) + exp(-x)); }
double silu_grad(double x) {
  double s = 1.0 / (1.0 + std::exp(-x));
  return s * (1.0 + x * (1.0 - s));
}

// tanh through the exponential, tanh(x) = 1 - 2 / (exp(2x) + 1): odd, so it
// keeps the parity of an odd scalar (mixed-parity models' 0o channels)
template <class T>
T tanh_t(T x) { return T(1.0) - T(2.0) / (exp(T(2.0) * x) + T(1.0)); }
double tanh_grad(double x) { const double t = std::tanh(x); return 1.0 - t * t; }

// Mixed-parity models (parity = 1): channel c < C/2 is the even-parity block,
// c >= C/2 the odd block.  A path with odd l2 (odd harmonics) takes its input
// from the other block (the output parity is the input parity times (-1)^l2).
inline int src_channel(int c, int C, int l2, int parity) { return (parity && (l2 & 1)) ? (c + C / 2) % C : c; }
// The scalar update's activation: SiLU on even scalars, tanh on odd ones.
template <class T>
T scalar_act(T x, int c, int C, int parity) { return (parity && c >= C / 2) ? tanh_t(x) : silu(x); }
inline double scalar_act_grad(double x, int c, int C, int parity) {
  return (parity && c >= C / 2) ? tanh_grad(x) : silu_grad(x);
}

// ------------------------------------------------------------------ model
struct Hyper {
  int S, T, C, L, Lsh, NB, H, p;
  double rc, avg_nb;
  int corr;  // 0: no symmetric contraction; 2: correlation order 2
  int charges;  // 1: charge head, charge correction and Coulomb term (open systems)
  double r0;    // soft-core radius of the Coulomb term, A
  int gate;     // 1: species self-connection and gated update of the l > 0 features
  int parity;   // 1: mixed-parity features (channel blocks of even and odd parity; pseudotensor paths)
};

struct Model {
  Hyper hp;
  int D, DY, P;
  std::vector<Path> paths, sc;
  std::vector<double> W_emb, W_out, E0, W_q, q0;
  double qtot = 0.0;  // total charge of the system being evaluated
  std::vector<std::vector<double>> W1, W2, W3, Wmix, Wsc1, Wsc2;
  // gated update: Wself [S][L+1][C][C], Wgate [C][L C], Wselfgate [S][C][L C] per layer
  std::vector<std::vector<double>> Wself, Wgate, Wselfgate;
};

int64_t num_weights(const Hyper& h, int P) {
  const int64_t Q = h.corr == 2 ? (int64_t)build_sc_paths(h.L).size() : 0;
  const int64_t sc = h.corr == 2 ? int64_t(h.S) * (h.L + 1 + Q) * h.C : 0;
  const int64_t gt = h.gate ? int64_t(h.S) * (h.L + 1) * h.C * h.C + int64_t(h.C) * h.L * h.C +
                                  int64_t(h.S) * h.C * h.L * h.C
                           : 0;
  return int64_t(h.S) * h.C +
         int64_t(h.T) * (int64_t(h.NB) * h.H + int64_t(h.H) * h.H + int64_t(h.H) * P * h.C +
                         int64_t(h.L + 1) * h.C * h.C + sc + gt) +
         int64_t(h.S) * h.C + h.S + (h.charges ? int64_t(h.S) * h.C + h.S : 0);
}

// ------------------------------------------------------------ electrostatics
// Coulomb's constant e^2 / (4 pi eps0) in eV A.
constexpr double kCoulomb = 14.3996454784;

// Soft-core pair function 1/chi(r) of the long-range term (Eq.
// long_range_interaction; chi follows PhysNet: equal to r beyond r0, smoothly
// regularised below):
//   1/chi(r) = phi(r/r0) / sqrt(r^2 + 1) + (1 - phi(r/r0)) / r,
//   phi(x) = 1 - 6 x^5 + 15 x^4 - 10 x^3 for x < 1, 0 otherwise.
template <class T>
T inv_chi(T r, double r0) {
  const T x = r / T(r0);
  if (val(x) >= 1.0) return T(1.0) / r;
  const T x3 = x * x * x;
  const T phi = T(1.0) - T(6.0) * x3 * x * x + T(15.0) * x3 * x - T(10.0) * x3;
  return phi / sqrt(r * r + T(1.0)) + (T(1.0) - phi) / r;
}
// d(1/chi)/dr, written out for the reverse pass
double inv_chi_grad(double r, double r0) {
  const double x = r / r0;
  if (x >= 1.0) return -1.0 / (r * r);
  const double x2 = x * x, x3 = x2 * x;
  const double phi = 1.0 - 6.0 * x3 * x2 + 15.0 * x3 * x - 10.0 * x3;
  const double dphi = (-30.0 * x2 * x2 + 60.0 * x3 - 30.0 * x2) / r0;
  const double s = std::sqrt(r * r + 1.0);
  return dphi * (1.0 / s - 1.0 / r) - phi * r / (s * s * s) - (1.0 - phi) / (r * r);
}

// Charge correction (Eq. charge_correction): qt_i = q_i - (sum_j q_j - Q) / N.
template <class T>
void correct_charges(std::vector<T>& q, double Q) {
  T sum = T(0.0);
  for (const T& v : q) sum += v;
  const T shift = (sum - T(Q)) / T((double)q.size());
  for (T& v : q) v = v - shift;
}

// E_LR = k sum_{i<j} qt_i qt_j / chi(r_ij) over all pairs of an open system
// (Eq. long_range_interaction, each unordered pair once).  atom_e (nullable)
// receives the half-pair shares k qt_i / 2 sum_{j != i} qt_j / chi(r_ij).
template <class T>
T coulomb_energy(const T* pos, const std::vector<T>& qt, int n, double r0, T* atom_e) {
  T E = T(0.0);
  for (int i = 0; i < n; ++i) {
    T ei = T(0.0);
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      const T dx = pos[3 * j] - pos[3 * i], dy = pos[3 * j + 1] - pos[3 * i + 1], dz = pos[3 * j + 2] - pos[3 * i + 2];
      ei += qt[j] * inv_chi(sqrt(dx * dx + dy * dy + dz * dz), r0);
    }
    ei = T(0.5 * kCoulomb) * qt[i] * ei;
    if (atom_e) atom_e[i] = ei;
    E += ei;
  }
  return E;
}

// Symmetric contraction of one node (correlation order 2), species z:
//   B[l3 m3][c] = w1[z][l3][c] A[l3 m3][c]
//               + sum_q w2[z][q][c] sum C^q[m3][m1][m2] A[l1 m1][c] A[l2 m2][c]
// over the couplings q = (l1 <= l2, l3) of build_sc_paths.  A, B: [D][C].
template <class T>
void sym_contract(const std::vector<Path>& sc, int L, int C, const T* A, const double* w1, const double* w2, T* B) {
  for (int l = 0; l <= L; ++l)
    for (int mm = -l; mm <= l; ++mm)
      for (int c = 0; c < C; ++c) B[(size_t)lm(l, mm) * C + c] = T(w1[(size_t)l * C + c]) * A[(size_t)lm(l, mm) * C + c];
  for (size_t q = 0; q < sc.size(); ++q) {
    const Path& pa = sc[q];
    for (const CGEntry& ce : pa.nz) {
      const int i3 = lm(pa.l3, ce.m3), i1 = lm(pa.l1, ce.m1), i2 = lm(pa.l2, ce.m2);
      for (int c = 0; c < C; ++c)
        B[(size_t)i3 * C + c] += T(w2[q * C + c] * ce.c) * A[(size_t)i1 * C + c] * A[(size_t)i2 * C + c];
    }
  }
}

// Its adjoint: GA = dE/dA from GB = dE/dB at the node's A (the product rule on
// both factors of every coupling).
void sym_contract_adjoint(const std::vector<Path>& sc, int L, int C, const double* A, const double* w1,
                          const double* w2, const double* GB, double* GA) {
  for (int l = 0; l <= L; ++l)
    for (int mm = -l; mm <= l; ++mm)
      for (int c = 0; c < C; ++c) GA[(size_t)lm(l, mm) * C + c] = w1[(size_t)l * C + c] * GB[(size_t)lm(l, mm) * C + c];
  for (size_t q = 0; q < sc.size(); ++q) {
    const Path& pa = sc[q];
    for (const CGEntry& ce : pa.nz) {
      const int i3 = lm(pa.l3, ce.m3), i1 = lm(pa.l1, ce.m1), i2 = lm(pa.l2, ce.m2);
      for (int c = 0; c < C; ++c) {
        const double g = w2[q * C + c] * ce.c * GB[(size_t)i3 * C + c];
        GA[(size_t)i1 * C + c] += g * A[(size_t)i2 * C + c];
        GA[(size_t)i2 * C + c] += g * A[(size_t)i1 * C + c];
      }
    }
  }
}

struct Edge { int i, j; int s0, s1, s2; };

// ------------------------------------------------------------ neighbours
// The set of directed pairs (receiver i, sender j, image S) with
//   sx = (S0*h00 + S1*h10) + S2*h20   (likewise y, z; h rows = lattice vectors)
//   dx = (xj - xi) + sx, ...;  d2 = (dx*dx + dy*dy) + dz*dz < rc*rc,
// excluding i == j with S = 0, S_k = 0 on open axes.  Brute force over all
// pairs and every image that can be within reach, sorted by (i, j, S).
bool invert3(const double* h, double* inv, double* det_out) {
  double det = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
               h[2] * (h[3] * h[7] - h[4] * h[6]);
  if (det_out) *det_out = det;
  if (!(std::fabs(det) > 1e-12)) return false;
  double id = 1.0 / det;
  inv[0] = (h[4] * h[8] - h[5] * h[7]) * id;
  inv[1] = (h[2] * h[7] - h[1] * h[8]) * id;
  inv[2] = (h[1] * h[5] - h[2] * h[4]) * id;
  inv[3] = (h[5] * h[6] - h[3] * h[8]) * id;
  inv[4] = (h[0] * h[8] - h[2] * h[6]) * id;
  inv[5] = (h[2] * h[3] - h[0] * h[5]) * id;
  inv[6] = (h[3] * h[7] - h[4] * h[6]) * id;
  inv[7] = (h[1] * h[6] - h[0] * h[7]) * id;
  inv[8] = (h[0] * h[4] - h[1] * h[3]) * id;
  return true;
}

int brute_neighbors(const double* pos, int n, const double* cell, const uint8_t* pbc, double rc,
                    std::vector<Edge>& out) {
  out.clear();
  bool anyp = pbc[0] || pbc[1] || pbc[2];
  double inv[9] = {0}, det = 0;
  int reach[3] = {0, 0, 0};
  std::vector<int> base(3 * (size_t)n, 0);
  if (anyp) {
    if (!invert3(cell, inv, &det)) return -1;
    double vol = std::fabs(det);
    for (int k = 0; k < 3; ++k) {
      if (!pbc[k]) continue;
      const double* a = cell + 3 * ((k + 1) % 3);
      const double* b = cell + 3 * ((k + 2) % 3);
      double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
      double w = vol / std::sqrt(cx * cx + cy * cy + cz * cz);  // perpendicular width
      reach[k] = (int)std::ceil(rc / w + 1.0 + 1e-6) - 1;
    }
    // integer part of each atom's fractional coordinate on periodic axes
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < 3; ++k) {
        if (!pbc[k]) continue;
        double s = pos[3 * i] * inv[0 * 3 + k] + pos[3 * i + 1] * inv[1 * 3 + k] + pos[3 * i + 2] * inv[2 * 3 + k];
        base[3 * i + k] = (int)std::floor(s);
      }
  }
  const double rc2 = rc * rc;
  std::vector<std::vector<Edge>> per(n);
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      int c0[3];
      for (int k = 0; k < 3; ++k) c0[k] = base[3 * i + k] - base[3 * j + k];
      for (int a = -reach[0]; a <= reach[0]; ++a)
        for (int b = -reach[1]; b <= reach[1]; ++b)
          for (int c = -reach[2]; c <= reach[2]; ++c) {
            int S0 = c0[0] + a, S1 = c0[1] + b, S2 = c0[2] + c;
            if (i == j && S0 == 0 && S1 == 0 && S2 == 0) continue;
            double sx = (S0 * cell[0] + S1 * cell[3]) + S2 * cell[6];
            double sy = (S0 * cell[1] + S1 * cell[4]) + S2 * cell[7];
            double sz = (S0 * cell[2] + S1 * cell[5]) + S2 * cell[8];
            if (!anyp) { sx = sy = sz = 0.0; }
            double dx = (pos[3 * j] - pos[3 * i]) + sx;
            double dy = (pos[3 * j + 1] - pos[3 * i + 1]) + sy;
            double dz = (pos[3 * j + 2] - pos[3 * i + 2]) + sz;
            double d2 = (dx * dx + dy * dy) + dz * dz;
            if (d2 < rc2) per[i].push_back({i, j, S0, S1, S2});
          }
    }
    std::sort(per[i].begin(), per[i].end(), [](const Edge& x, const Edge& y) {
      if (x.j != y.j) return x.j < y.j;
      if (x.s0 != y.s0) return x.s0 < y.s0;
      if (x.s1 != y.s1) return x.s1 < y.s1;
      return x.s2 < y.s2;
    });
  }
  for (int i = 0; i < n; ++i) out.insert(out.end(), per[i].begin(), per[i].end());
  return 0;
}

// --------------------------------------------------------------- forward
// One evaluation of E for positions of scalar type T (double, or Dual for a
// forward-mode derivative).  Layer t maps node features h (N x D x C,
// component index lm(l,m)) to
//   x_e   = (r_j - r_i) + S.h                           edge vector
//   Y_e   = Y_{l2 m2}(x_e / |x_e|),  b_e[n] = B_n(|x_e|) u(|x_e|/rc)
//   w_e   = W3^T silu(W2^T silu(W1^T b_e))              [P][C], no biases
//   m_i   = s sum_{e: recv=i} sum_p w_e[p][c] sum C^p[m3][m1][m2] h_j[l1 m1][c] Y_e[l2 m2]
//   m_i  <- sym_contract(m_i)   (only with correlation order 2)
//   u_i,l = m_i,l W_l   (u[c'] = sum_c m[c] W_l[c][c'])
//   h_i,0 += silu(u_i,0);  h_i,l>0 += u_i,l
// and E = sum_i (sum_c W_out[z_i][c] h_i,0[c] + E0[z_i]).
template <class T>
T model_energy(const Model& M, const std::vector<Edge>& edges, const std::vector<int>& row_ptr,
               const T* pos, const int* species, int n, const double* cell, double* atom_e,
               std::vector<std::vector<double>>* h_store, std::vector<std::vector<double>>* u_store,
               std::vector<std::vector<double>>* a_store = nullptr,
               std::vector<std::vector<double>>* g_store = nullptr) {
  const Hyper& hp = M.hp;
  const int D = M.D, C = hp.C, H = hp.H, P = M.P, NB = hp.NB, DY = M.DY;
  const double s = 1.0 / hp.avg_nb;
  std::vector<T> h((size_t)n * D * C, T(0.0));
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < C; ++c) h[((size_t)i * D) * C + c] = T(M.W_emb[(size_t)species[i] * C + c]);
  for (int t = 0; t < hp.T; ++t) {
    if (h_store) { (*h_store)[t].resize(h.size()); for (size_t k = 0; k < h.size(); ++k) (*h_store)[t][k] = val(h[k]); }
    std::vector<T> m((size_t)n * D * C, T(0.0));
    const std::vector<double>& W1 = M.W1[t];
    const std::vector<double>& W2 = M.W2[t];
    const std::vector<double>& W3 = M.W3[t];
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < n; ++i) {
      std::vector<T> Y(DY), b(NB), a1(H), z1(H), a2(H), z2(H), w((size_t)P * C);
      for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const Edge& E = edges[e];
        const int j = E.j;
        T x[3];
        for (int k = 0; k < 3; ++k) {
          double sk = (E.s0 * cell[k] + E.s1 * cell[3 + k]) + E.s2 * cell[6 + k];
          x[k] = (pos[3 * j + k] - pos[3 * i + k]) + T(sk);
        }
        T r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        real_sh_vec(hp.Lsh, x[0], x[1], x[2], Y.data());
        T u = envelope(r / T(hp.rc), hp.p);
        for (int q = 0; q < NB; ++q) b[q] = bessel(q + 1, r, hp.rc) * u;
        for (int k = 0; k < H; ++k) {
          T acc = T(0.0);
          for (int q = 0; q < NB; ++q) acc += b[q] * T(W1[(size_t)q * H + k]);
          a1[k] = acc; z1[k] = silu(acc);
        }
        for (int k = 0; k < H; ++k) {
          T acc = T(0.0);
          for (int q = 0; q < H; ++q) acc += z1[q] * T(W2[(size_t)q * H + k]);
          a2[k] = acc; z2[k] = silu(acc);
        }
        for (int pc = 0; pc < P * C; ++pc) {
          T acc = T(0.0);
          for (int k = 0; k < H; ++k) acc += z2[k] * T(W3[(size_t)k * P * C + pc]);
          w[pc] = acc;
        }
        for (int p = 0; p < P; ++p) {
          const Path& pa = M.paths[p];
          for (const CGEntry& ce : pa.nz) {
            const int i3 = lm(pa.l3, ce.m3), i1 = lm(pa.l1, ce.m1), i2 = lm(pa.l2, ce.m2);
            for (int c = 0; c < C; ++c)
              m[((size_t)i * D + i3) * C + c] += T(s) * w[(size_t)p * C + c] * T(ce.c) *
                                                   h[((size_t)j * D + i1) * C + src_channel(c, C, pa.l2, hp.parity)] *
                                                   Y[i2];
          }
        }
      }
    }
    if (hp.corr == 2) {
      if (a_store) { (*a_store)[t].resize(m.size()); for (size_t k = 0; k < m.size(); ++k) (*a_store)[t][k] = val(m[k]); }
      std::vector<T> B(m.size());
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i)
        sym_contract<T>(M.sc, hp.L, C, &m[(size_t)i * D * C], &M.Wsc1[t][(size_t)species[i] * (hp.L + 1) * C],
                        &M.Wsc2[t][(size_t)species[i] * M.sc.size() * C], &B[(size_t)i * D * C]);
      m.swap(B);
    }
    const std::vector<double>& Wm = M.Wmix[t];
    std::vector<T> hn(h);
    if (u_store) (*u_store)[t].assign((size_t)n * D * C, 0.0);
    if (hp.gate) {
      // pre_l = m_l W_l + h_l Wself[z][l];  g_l = m_0 Wgate_l + h_0 Wselfgate[z]_l (l >= 1, per channel)
      // h_0 += silu(pre_0);  h_l += sigmoid(g_l) pre_l
      const int LC = hp.L * C;
      if (g_store) (*g_store)[t].assign((size_t)n * LC, 0.0);
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) {
        const int z = species[i];
        const double* Ws = &M.Wself[t][(size_t)z * (hp.L + 1) * C * C];
        const double* Wsg = &M.Wselfgate[t][(size_t)z * C * LC];
        std::vector<T> g(LC);
        for (int q = 0; q < LC; ++q) {
          T acc = T(0.0);
          for (int c1 = 0; c1 < C; ++c1)
            acc += m[((size_t)i * D) * C + c1] * T(M.Wgate[t][(size_t)c1 * LC + q]) +
                   h[((size_t)i * D) * C + c1] * T(Wsg[(size_t)c1 * LC + q]);
          g[q] = acc;
          if (g_store) (*g_store)[t][(size_t)i * LC + q] = val(acc);
        }
        for (int l = 0; l <= hp.L; ++l)
          for (int mm = -l; mm <= l; ++mm) {
            const int ci = lm(l, mm);
            for (int c2 = 0; c2 < C; ++c2) {
              T acc = T(0.0);
              for (int c1 = 0; c1 < C; ++c1)
                acc += m[((size_t)i * D + ci) * C + c1] * T(Wm[((size_t)l * C + c1) * C + c2]) +
                       h[((size_t)i * D + ci) * C + c1] * T(Ws[((size_t)l * C + c1) * C + c2]);
              if (u_store) (*u_store)[t][((size_t)i * D + ci) * C + c2] = val(acc);
              hn[((size_t)i * D + ci) * C + c2] += (l == 0) ? silu(acc) : sigmoid(g[(l - 1) * C + c2]) * acc;
            }
          }
      }
      h.swap(hn);
      continue;
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
      for (int l = 0; l <= hp.L; ++l)
        for (int mm = -l; mm <= l; ++mm) {
          const int ci = lm(l, mm);
          for (int c2 = 0; c2 < C; ++c2) {
            T acc = T(0.0);
            for (int c1 = 0; c1 < C; ++c1)
              acc += m[((size_t)i * D + ci) * C + c1] * T(Wm[((size_t)l * C + c1) * C + c2]);
            if (u_store) (*u_store)[t][((size_t)i * D + ci) * C + c2] = val(acc);
            hn[((size_t)i * D + ci) * C + c2] += (l == 0) ? scalar_act(acc, c2, C, hp.parity) : acc;
          }
        }
    h.swap(hn);
  }
  if (h_store) { (*h_store)[hp.T].resize(h.size()); for (size_t k = 0; k < h.size(); ++k) (*h_store)[hp.T][k] = val(h[k]); }
  T E = T(0.0);
  for (int i = 0; i < n; ++i) {
    T ei = T(M.E0[species[i]]);
    for (int c = 0; c < C; ++c) ei += T(M.W_out[(size_t)species[i] * C + c]) * h[((size_t)i * D) * C + c];
    if (atom_e) atom_e[i] = val(ei);
    E += ei;
  }
  if (hp.charges) {
    // charge head q_i = W_q[z_i] . h_i,0 + q0[z_i], corrected to the total charge, and the Coulomb term
    std::vector<T> q(n);
    for (int i = 0; i < n; ++i) {
      T qi = T(M.q0[species[i]]);
      for (int c = 0; c < C; ++c) qi += T(M.W_q[(size_t)species[i] * C + c]) * h[((size_t)i * D) * C + c];
      q[i] = qi;
    }
    correct_charges(q, M.qtot);
    std::vector<T> ae(n);
    E += coulomb_energy<T>(pos, q, n, hp.r0, ae.data());
    if (atom_e)
      for (int i = 0; i < n; ++i) atom_e[i] += val(ae[i]);
  }
  return E;
}

std::vector<int> receiver_row_ptr(const std::vector<Edge>& edges, int n) {
  std::vector<int> rp(n + 1, 0);
  for (const Edge& e : edges) rp[e.i + 1]++;
  for (int i = 0; i < n; ++i) rp[i + 1] += rp[i];
  return rp;
}

// --------------------------------------------------------------- reverse
// Hand-written adjoint of model_energy.  G = dE/dh^t runs backwards through
// the layers; per edge the harmonics, basis and MLP are recomputed, and the
// Jacobians dY/dx and db/dx come from forward-mode dual numbers on the edge
// vector.  g_e = dE/dx_e; F_i = sum_{e: recv=i} g_e - sum_{e: send=i} g_e;
// stress = (1/V) sum_e x_e (x) g_e.
double model_energy_forces(const Model& M, const std::vector<Edge>& edges, const double* pos,
                           const int* species, int n, const double* cell, double* forces,
                           double* virial, double* atom_e) {
  const Hyper& hp = M.hp;
  const int D = M.D, C = hp.C, H = hp.H, P = M.P, NB = hp.NB, DY = M.DY;
  const double s = 1.0 / hp.avg_nb;
  const int E = (int)edges.size();
  std::vector<int> rp = receiver_row_ptr(edges, n);
  std::vector<std::vector<double>> hs(hp.T + 1), us(hp.T), as(hp.T), gs(hp.T);
  double energy = model_energy<double>(M, edges, rp, pos, species, n, cell, atom_e, &hs, &us, &as, &gs);

  // sender-sorted index of edges
  std::vector<int> sp(n + 1, 0), sidx(E);
  for (const Edge& e : edges) sp[e.j + 1]++;
  for (int i = 0; i < n; ++i) sp[i + 1] += sp[i];
  {
    std::vector<int> fill(sp.begin(), sp.end() - 1);
    for (int e = 0; e < E; ++e) sidx[fill[edges[e].j]++] = e;
  }
  // per-edge geometry and Jacobians
  std::vector<double> xe((size_t)E * 3), JY((size_t)E * DY * 3), Jb((size_t)E * NB * 3);
#pragma omp parallel for schedule(static)
  for (int e = 0; e < E; ++e) {
    const Edge& ed = edges[e];
    for (int k = 0; k < 3; ++k) {
      double sk = (ed.s0 * cell[k] + ed.s1 * cell[3 + k]) + ed.s2 * cell[6 + k];
      xe[(size_t)e * 3 + k] = (pos[3 * ed.j + k] - pos[3 * ed.i + k]) + sk;
    }
    for (int a = 0; a < 3; ++a) {
      Dual x[3];
      for (int k = 0; k < 3; ++k) x[k] = Dual(xe[(size_t)e * 3 + k], k == a ? 1.0 : 0.0);
      std::vector<Dual> Y(DY);
      real_sh_vec(hp.Lsh, x[0], x[1], x[2], Y.data());
      Dual r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
      Dual u = envelope(r / Dual(hp.rc), hp.p);
      for (int k = 0; k < DY; ++k) JY[((size_t)e * DY + k) * 3 + a] = Y[k].d;
      for (int q = 0; q < NB; ++q) Jb[((size_t)e * NB + q) * 3 + a] = (bessel(q + 1, r, hp.rc) * u).d;
    }
  }
  std::vector<double> dY((size_t)E * DY, 0.0), db((size_t)E * NB, 0.0);
  // dE/dh^T
  std::vector<double> G((size_t)n * D * C, 0.0);
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < C; ++c) G[((size_t)i * D) * C + c] = M.W_out[(size_t)species[i] * C + c];
  std::vector<double> qt, Fc;  // corrected charges and the Coulomb term's direct forces
  if (hp.charges) {
    const std::vector<double>& hT = hs[hp.T];
    qt.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
      double qi = M.q0[species[i]];
      for (int c = 0; c < C; ++c) qi += M.W_q[(size_t)species[i] * C + c] * hT[((size_t)i * D) * C + c];
      qt[i] = qi;
    }
    correct_charges(qt, M.qtot);
    // gt_i = dE/dqt_i = k sum_{j != i} qt_j / chi(r_ij); direct force -dE/dr_i at fixed charges
    std::vector<double> gt(n, 0.0);
    Fc.assign(3 * (size_t)n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        const double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1], pos[3 * j + 2] - pos[3 * i + 2]};
        const double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        gt[i] += kCoulomb * qt[j] * inv_chi(r, hp.r0);
        // E contains k qt_i qt_j f(r_ij) once per pair; d/dr_i of it is -k qt_i qt_j f'(r) d / r
        const double fr = kCoulomb * qt[i] * qt[j] * inv_chi_grad(r, hp.r0) / r;
        for (int a = 0; a < 3; ++a) Fc[3 * (size_t)i + a] += fr * d[a];
      }
    // through the correction: dE/dq_i = gt_i - mean(gt)
    double mean = 0.0;
    for (int i = 0; i < n; ++i) mean += gt[i];
    mean /= n;
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < C; ++c)
        G[((size_t)i * D) * C + c] += (gt[i] - mean) * M.W_q[(size_t)species[i] * C + c];
  }
  for (int t = hp.T - 1; t >= 0; --t) {
    const std::vector<double>& hprev = hs[t];
    const std::vector<double>& u = us[t];
    const std::vector<double>& Wm = M.Wmix[t];
    // through the residual update and the channel mix
    std::vector<double> Gm((size_t)n * D * C, 0.0);
    std::vector<double> Gself;  // gated update: the self-connection's share of dE/dh^t
    if (hp.gate) {
      const int LC = hp.L * C;
      Gself.assign((size_t)n * D * C, 0.0);
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) {
        const int z = species[i];
        const double* Ws = &M.Wself[t][(size_t)z * (hp.L + 1) * C * C];
        const double* Wsg = &M.Wselfgate[t][(size_t)z * C * LC];
        const double* g = &gs[t][(size_t)i * LC];
        // dE/dpre and dE/dg
        std::vector<double> dpre((size_t)D * C), dg(LC, 0.0);
        for (int l = 0; l <= hp.L; ++l)
          for (int mm = -l; mm <= l; ++mm) {
            const int ci = lm(l, mm);
            for (int c2 = 0; c2 < C; ++c2) {
              const size_t k = ((size_t)i * D + ci) * C + c2;
              if (l == 0) {
                dpre[(size_t)ci * C + c2] = G[k] * silu_grad(u[k]);
              } else {
                const double sg = 1.0 / (1.0 + std::exp(-g[(l - 1) * C + c2]));
                dpre[(size_t)ci * C + c2] = G[k] * sg;
                dg[(l - 1) * C + c2] += G[k] * u[k] * sg * (1.0 - sg);
              }
            }
          }
        for (int l = 0; l <= hp.L; ++l)
          for (int mm = -l; mm <= l; ++mm) {
            const int ci = lm(l, mm);
            for (int c1 = 0; c1 < C; ++c1) {
              double am = 0.0, ah = 0.0;
              for (int c2 = 0; c2 < C; ++c2) {
                am += Wm[((size_t)l * C + c1) * C + c2] * dpre[(size_t)ci * C + c2];
                ah += Ws[((size_t)l * C + c1) * C + c2] * dpre[(size_t)ci * C + c2];
              }
              if (l == 0)
                for (int q = 0; q < LC; ++q) {
                  am += M.Wgate[t][(size_t)c1 * LC + q] * dg[q];
                  ah += Wsg[(size_t)c1 * LC + q] * dg[q];
                }
              Gm[((size_t)i * D + ci) * C + c1] = am;
              Gself[((size_t)i * D + ci) * C + c1] = ah;
            }
          }
      }
    } else {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
      for (int l = 0; l <= hp.L; ++l)
        for (int mm = -l; mm <= l; ++mm) {
          const int ci = lm(l, mm);
          std::vector<double> gu(C);
          for (int c2 = 0; c2 < C; ++c2) {
            size_t k = ((size_t)i * D + ci) * C + c2;
            gu[c2] = (l == 0) ? G[k] * scalar_act_grad(u[k], c2, C, hp.parity) : G[k];
          }
          for (int c1 = 0; c1 < C; ++c1) {
            double acc = 0.0;
            for (int c2 = 0; c2 < C; ++c2) acc += Wm[((size_t)l * C + c1) * C + c2] * gu[c2];
            Gm[((size_t)i * D + ci) * C + c1] = acc;
          }
        }
    }
    if (hp.corr == 2) {  // through the symmetric contraction: Gm = dE/dB -> dE/dA
      std::vector<double> GA(Gm.size());
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i)
        sym_contract_adjoint(M.sc, hp.L, C, &as[t][(size_t)i * D * C], &M.Wsc1[t][(size_t)species[i] * (hp.L + 1) * C],
                             &M.Wsc2[t][(size_t)species[i] * M.sc.size() * C], &Gm[(size_t)i * D * C],
                             &GA[(size_t)i * D * C]);
      Gm.swap(GA);
    }
    std::vector<double> Gprev(G);  // residual path
    if (hp.gate)
      for (size_t k = 0; k < Gprev.size(); ++k) Gprev[k] += Gself[k];
    const std::vector<double>& W1 = M.W1[t];
    const std::vector<double>& W2 = M.W2[t];
    const std::vector<double>& W3 = M.W3[t];
    // loop over senders j so that each thread owns Gprev[j]
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < n; ++j) {
      std::vector<double> Y(DY), b(NB), a1(H), z1(H), a2(H), z2(H), w((size_t)P * C), dw((size_t)P * C);
      std::vector<double> dz2(H), da2(H), dz1(H), da1(H);
      for (int q = sp[j]; q < sp[j + 1]; ++q) {
        const int e = sidx[q];
        const int i = edges[e].i;
        const double* x = &xe[(size_t)e * 3];
        double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        real_sh_vec(hp.Lsh, x[0], x[1], x[2], Y.data());
        double uu = envelope(r / hp.rc, hp.p);
        for (int k = 0; k < NB; ++k) b[k] = bessel(k + 1, r, hp.rc) * uu;
        for (int k = 0; k < H; ++k) {
          double acc = 0;
          for (int qq = 0; qq < NB; ++qq) acc += b[qq] * W1[(size_t)qq * H + k];
          a1[k] = acc; z1[k] = silu(acc);
        }
        for (int k = 0; k < H; ++k) {
          double acc = 0;
          for (int qq = 0; qq < H; ++qq) acc += z1[qq] * W2[(size_t)qq * H + k];
          a2[k] = acc; z2[k] = silu(acc);
        }
        for (int pc = 0; pc < P * C; ++pc) {
          double acc = 0;
          for (int k = 0; k < H; ++k) acc += z2[k] * W3[(size_t)k * P * C + pc];
          w[pc] = acc;
        }
        std::fill(dw.begin(), dw.end(), 0.0);
        double* dYe = &dY[(size_t)e * DY];
        for (int p = 0; p < P; ++p) {
          const Path& pa = M.paths[p];
          for (const CGEntry& ce : pa.nz) {
            const int i3 = lm(pa.l3, ce.m3), i1 = lm(pa.l1, ce.m1), i2 = lm(pa.l2, ce.m2);
            for (int c = 0; c < C; ++c) {
              const int cs = src_channel(c, C, pa.l2, hp.parity);
              const double gt = s * Gm[((size_t)i * D + i3) * C + c];
              const double hj = hprev[((size_t)j * D + i1) * C + cs];
              const double wp = w[(size_t)p * C + c];
              Gprev[((size_t)j * D + i1) * C + cs] += wp * ce.c * Y[i2] * gt;
              dYe[i2] += wp * ce.c * hj * gt;
              dw[(size_t)p * C + c] += ce.c * hj * Y[i2] * gt;
            }
          }
        }
        for (int k = 0; k < H; ++k) {
          double acc = 0;
          for (int pc = 0; pc < P * C; ++pc) acc += W3[(size_t)k * P * C + pc] * dw[pc];
          dz2[k] = acc; da2[k] = acc * silu_grad(a2[k]);
        }
        for (int k = 0; k < H; ++k) {
          double acc = 0;
          for (int qq = 0; qq < H; ++qq) acc += W2[(size_t)k * H + qq] * da2[qq];
          dz1[k] = acc; da1[k] = acc * silu_grad(a1[k]);
        }
        for (int qq = 0; qq < NB; ++qq) {
          double acc = 0;
          for (int k = 0; k < H; ++k) acc += W1[(size_t)qq * H + k] * da1[k];
          db[(size_t)e * NB + qq] += acc;
        }
      }
    }
    G.swap(Gprev);
  }
  // edge gradients, forces, virial
  std::vector<double> g((size_t)E * 3, 0.0);
  for (int e = 0; e < E; ++e)
    for (int a = 0; a < 3; ++a) {
      double acc = 0;
      for (int k = 0; k < DY; ++k) acc += dY[(size_t)e * DY + k] * JY[((size_t)e * DY + k) * 3 + a];
      for (int q = 0; q < NB; ++q) acc += db[(size_t)e * NB + q] * Jb[((size_t)e * NB + q) * 3 + a];
      g[(size_t)e * 3 + a] = acc;
    }
  if (forces) {
    std::fill(forces, forces + 3 * (size_t)n, 0.0);
    for (int e = 0; e < E; ++e)
      for (int a = 0; a < 3; ++a) {
        forces[3 * edges[e].i + a] += g[(size_t)e * 3 + a];
        forces[3 * edges[e].j + a] -= g[(size_t)e * 3 + a];
      }
    if (hp.charges)
      for (size_t k = 0; k < 3 * (size_t)n; ++k) forces[k] += Fc[k];
  }
  if (virial) {
    for (int k = 0; k < 9; ++k) virial[k] = 0.0;
    for (int e = 0; e < E; ++e)
      for (int a = 0; a < 3; ++a)
        for (int b2 = 0; b2 < 3; ++b2) virial[a * 3 + b2] += xe[(size_t)e * 3 + a] * g[(size_t)e * 3 + b2];
  }
  return energy;
}

}  // namespace

// =================================================================== C API
extern "C" {

int oracle_version(void) { return 1; }

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Real harmonics Y_{l,m}(v/|v|), l <= lmax, out[l*l + m + l].
int oracle_real_sh(int lmax, const double* v, double* out) {
  if (lmax < 0 || lmax > 8) return -1;
  real_sh_vec<double>(lmax, v[0], v[1], v[2], out);
  return 0;
}

// Jacobian d Y_{lm}(v/|v|) / d v_a, out[(l*l+m+l)*3 + a].
int oracle_real_sh_grad(int lmax, const double* v, double* out) {
  if (lmax < 0 || lmax > 8) return -1;
  int n = (lmax + 1) * (lmax + 1);
  std::vector<Dual> Y(n);
  for (int a = 0; a < 3; ++a) {
    Dual x[3];
    for (int k = 0; k < 3; ++k) x[k] = Dual(v[k], k == a ? 1.0 : 0.0);
    real_sh_vec(lmax, x[0], x[1], x[2], Y.data());
    for (int k = 0; k < n; ++k) out[k * 3 + a] = Y[k].d;
  }
  return 0;
}

// Complex harmonics (Condon-Shortley phase), m = -l..l.
int oracle_complex_sh(int l, const double* v, double* re, double* im) {
  double r = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  std::vector<std::complex<double>> y(2 * l + 1);
  complex_sh_unit(l, v[0] / r, v[1] / r, v[2] / r, y.data());
  for (int k = 0; k < 2 * l + 1; ++k) { re[k] = y[k].real(); im[k] = y[k].imag(); }
  return 0;
}

double oracle_cg_complex(int l1, int m1, int l2, int m2, int l3, int m3) {
  return cg_complex(l1, m1, l2, m2, l3, m3);
}

int oracle_real_basis_U(int l, double* re, double* im) {
  int n = 2 * l + 1;
  std::vector<std::complex<double>> U(n * n);
  real_basis_U(l, U.data());
  for (int k = 0; k < n * n; ++k) { re[k] = U[k].real(); im[k] = U[k].imag(); }
  return 0;
}

int oracle_real_cg(int l1, int l2, int l3, double* out) {
  if (l3 < std::abs(l1 - l2) || l3 > l1 + l2) return -1;
  real_cg(l1, l2, l3, out);
  return 0;
}

// Paths (l1, l2, l3) in order; returns their count, writes 3 ints each if out != NULL.
int oracle_paths(int L, int Lsh, int* out) {
  std::vector<Path> ps = build_paths(L, Lsh);
  if (out)
    for (size_t k = 0; k < ps.size(); ++k) {
      out[3 * k] = ps[k].l1; out[3 * k + 1] = ps[k].l2; out[3 * k + 2] = ps[k].l3;
    }
  return (int)ps.size();
}

// Paths of the mixed-parity model: every triangle-valid (l1, l2, l3), both parities.
int oracle_paths_all(int L, int Lsh, int* out) {
  std::vector<Path> ps = build_paths(L, Lsh, true);
  if (out)
    for (size_t k = 0; k < ps.size(); ++k) {
      out[3 * k] = ps[k].l1; out[3 * k + 1] = ps[k].l2; out[3 * k + 2] = ps[k].l3;
    }
  return (int)ps.size();
}

double oracle_bessel(int n, double r, double rc) { return bessel<double>(n, r, rc); }
double oracle_envelope(double x, int p) { return envelope<double>(x, p); }

// hyper = {S, T, C, L, Lsh, NB, H, p, correlation, charges, gate}, dhyper = {rc, avg_num_neighbors, r0}
int64_t oracle_num_weights(const int* hyper) {
  Hyper h{hyper[0], hyper[1], hyper[2], hyper[3], hyper[4], hyper[5], hyper[6], hyper[7], 0, 0, hyper[8], hyper[9], 0,
          hyper[10], hyper[11]};
  int P = (int)build_paths(h.L, h.Lsh, h.parity != 0).size();
  return num_weights(h, P);
}

void* oracle_model_create(const int* hyper, const double* dhyper, const float* wts) {
  Model* M = new Model();
  Hyper& h = M->hp;
  h = Hyper{hyper[0], hyper[1], hyper[2], hyper[3], hyper[4], hyper[5], hyper[6], hyper[7], dhyper[0], dhyper[1],
            hyper[8], hyper[9], dhyper[2], hyper[10], hyper[11]};
  if (h.parity && (h.corr || h.gate || h.charges || h.C % 2)) { delete M; return nullptr; }
  M->paths = build_paths(h.L, h.Lsh, h.parity != 0);
  if (h.corr == 2) M->sc = build_sc_paths(h.L);
  M->P = (int)M->paths.size();
  M->D = (h.L + 1) * (h.L + 1);
  M->DY = (h.Lsh + 1) * (h.Lsh + 1);
  const float* q = wts;
  auto take = [&](std::vector<double>& v, size_t cnt) {
    v.resize(cnt);
    for (size_t k = 0; k < cnt; ++k) v[k] = (double)q[k];
    q += cnt;
  };
  take(M->W_emb, (size_t)h.S * h.C);
  M->W1.resize(h.T); M->W2.resize(h.T); M->W3.resize(h.T); M->Wmix.resize(h.T);
  M->Wsc1.resize(h.T); M->Wsc2.resize(h.T);
  M->Wself.resize(h.T); M->Wgate.resize(h.T); M->Wselfgate.resize(h.T);
  for (int t = 0; t < h.T; ++t) {
    take(M->W1[t], (size_t)h.NB * h.H);
    take(M->W2[t], (size_t)h.H * h.H);
    take(M->W3[t], (size_t)h.H * M->P * h.C);
    take(M->Wmix[t], (size_t)(h.L + 1) * h.C * h.C);
    if (h.corr == 2) {
      take(M->Wsc1[t], (size_t)h.S * (h.L + 1) * h.C);
      take(M->Wsc2[t], (size_t)h.S * M->sc.size() * h.C);
    }
    if (h.gate) {
      take(M->Wself[t], (size_t)h.S * (h.L + 1) * h.C * h.C);
      take(M->Wgate[t], (size_t)h.C * h.L * h.C);
      take(M->Wselfgate[t], (size_t)h.S * h.C * h.L * h.C);
    }
  }
  take(M->W_out, (size_t)h.S * h.C);
  take(M->E0, (size_t)h.S);
  if (h.parity) {
    // the definition of the mixed-parity model: the embedding and the readout
    // act on even scalars only (the energy is a true scalar), and the channel
    // mixes keep each parity block (block-diagonal W_l): the weights outside
    // those blocks are ignored
    const int Ch = h.C / 2;
    for (int z = 0; z < h.S; ++z)
      for (int c = Ch; c < h.C; ++c) M->W_emb[(size_t)z * h.C + c] = M->W_out[(size_t)z * h.C + c] = 0.0;
    for (int t = 0; t < h.T; ++t)
      for (int l = 0; l <= h.L; ++l)
        for (int c1 = 0; c1 < h.C; ++c1)
          for (int c2 = 0; c2 < h.C; ++c2)
            if ((c1 < Ch) != (c2 < Ch)) M->Wmix[t][((size_t)l * h.C + c1) * h.C + c2] = 0.0;
  }
  if (h.charges) {
    take(M->W_q, (size_t)h.S * h.C);
    take(M->q0, (size_t)h.S);
  }
  return M;
}

void oracle_model_free(void* m) { delete static_cast<Model*>(m); }

// Total charge Q of the systems evaluated next (models with the charge head).
void oracle_model_set_total_charge(void* m, double Q) { static_cast<Model*>(m)->qtot = Q; }

// Corrected charges of the charge head for one system (n values).
int oracle_charges(void* model, const double* pos, const int32_t* species, int64_t n, double* q_out) {
  const Model& M = *static_cast<Model*>(model);
  if (!M.hp.charges) return -4;
  std::vector<Edge> edges;
  double zero[9] = {0};
  uint8_t np[3] = {0, 0, 0};
  if (brute_neighbors(pos, (int)n, zero, np, M.hp.rc, edges) != 0) return -1;
  std::vector<int> rp = receiver_row_ptr(edges, (int)n);
  std::vector<int> sp(species, species + n);
  std::vector<std::vector<double>> hs(M.hp.T + 1);
  model_energy<double>(M, edges, rp, pos, sp.data(), (int)n, zero, nullptr, &hs, nullptr);
  const int D = M.D, C = M.hp.C;
  std::vector<double> q(n);
  for (int64_t i = 0; i < n; ++i) {
    double qi = M.q0[sp[i]];
    for (int c = 0; c < C; ++c) qi += M.W_q[(size_t)sp[i] * C + c] * hs[M.hp.T][((size_t)i * D) * C + c];
    q[i] = qi;
  }
  correct_charges(q, M.qtot);
  for (int64_t i = 0; i < n; ++i) q_out[i] = q[i];
  return 0;
}

// The Coulomb term alone for given corrected charges: E, dE/dqt [n], forces [n][3].
int oracle_coulomb(const double* pos, const double* qt, int64_t n, double r0, double* E, double* dEdq,
                   double* forces) {
  std::vector<double> q(qt, qt + n);
  *E = coulomb_energy<double>(pos, q, (int)n, r0, nullptr);
  for (int64_t i = 0; i < n; ++i) {
    double g = 0.0, F[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      const double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1], pos[3 * j + 2] - pos[3 * i + 2]};
      const double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      g += kCoulomb * q[j] * inv_chi(r, r0);
      const double fr = kCoulomb * q[i] * q[j] * inv_chi_grad(r, r0) / r;
      for (int a = 0; a < 3; ++a) F[a] += fr * d[a];
    }
    dEdq[i] = g;
    for (int a = 0; a < 3; ++a) forces[3 * i + a] = F[a];
  }
  return 0;
}

double oracle_inv_chi(double r, double r0) { return inv_chi<double>(r, r0); }

// Brute-force neighbour list, sorted by (recv, send, S).  Returns the number of
// edges (writing at most cap of them), -1 for a singular periodic cell.
int64_t oracle_neighbors(const double* pos, int64_t n, const double* cell, const uint8_t* pbc, double rc,
                         int32_t* recv, int32_t* send, int32_t* shift, int64_t cap) {
  std::vector<Edge> e;
  double zero[9] = {0};
  uint8_t np[3] = {0, 0, 0};
  bool anyp = pbc[0] || pbc[1] || pbc[2];
  if (brute_neighbors(pos, (int)n, anyp ? cell : zero, anyp ? pbc : np, rc, e) != 0) return -1;
  for (int64_t k = 0; k < (int64_t)e.size() && k < cap; ++k) {
    recv[k] = e[k].i; send[k] = e[k].j;
    shift[3 * k] = e[k].s0; shift[3 * k + 1] = e[k].s1; shift[3 * k + 2] = e[k].s2;
  }
  return (int64_t)e.size();
}

static double cell_volume(const double* h) {
  return std::fabs(h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                   h[2] * (h[3] * h[7] - h[4] * h[6]));
}

// Energy, forces (N x 3, nullable), stress (3 x 3 eV/A^3, nullable: needs a fully
// periodic cell), per-atom energies (nullable).  Returns 0 or a negative error.
int oracle_energy_forces(void* model, const double* pos, const int32_t* species, int64_t n,
                         const double* cell, const uint8_t* pbc, double* energy, double* forces,
                         double* stress, double* atom_e) {
  const Model& M = *static_cast<Model*>(model);
  bool anyp = pbc[0] || pbc[1] || pbc[2];
  if (M.hp.charges && anyp) return -3;  // the Coulomb term is defined for open systems
  double zero[9] = {0};
  uint8_t np[3] = {0, 0, 0};
  const double* cl = anyp ? cell : zero;
  std::vector<Edge> edges;
  if (brute_neighbors(pos, (int)n, cl, anyp ? pbc : np, M.hp.rc, edges) != 0) return -1;
  std::vector<int> sp(species, species + n);
  double vir[9];
  double E = model_energy_forces(M, edges, pos, sp.data(), (int)n, cl, forces, vir, atom_e);
  *energy = E;
  if (stress) {
    if (!(pbc[0] && pbc[1] && pbc[2])) return -2;
    double V = cell_volume(cell);
    for (int k = 0; k < 9; ++k) stress[k] = vir[k] / V;
  }
  return 0;
}

// Energy only (no reverse pass), with the per-atom energies if atom_e != NULL.
int oracle_energy(void* model, const double* pos, const int32_t* species, int64_t n,
                  const double* cell, const uint8_t* pbc, double* energy, double* atom_e) {
  const Model& M = *static_cast<Model*>(model);
  bool anyp = pbc[0] || pbc[1] || pbc[2];
  if (M.hp.charges && anyp) return -3;  // the Coulomb term is defined for open systems
  double zero[9] = {0};
  uint8_t np[3] = {0, 0, 0};
  const double* cl = anyp ? cell : zero;
  std::vector<Edge> edges;
  if (brute_neighbors(pos, (int)n, cl, anyp ? pbc : np, M.hp.rc, edges) != 0) return -1;
  std::vector<int> rp = receiver_row_ptr(edges, (int)n);
  std::vector<int> sp(species, species + n);
  *energy = model_energy<double>(M, edges, rp, pos, sp.data(), (int)n, cl, atom_e, nullptr, nullptr);
  return 0;
}

// Forward-mode derivative dE/d r_{atom, axis} with dual numbers (edge set fixed
// at the given positions).
int oracle_energy_dual(void* model, const double* pos, const int32_t* species, int64_t n,
                       const double* cell, const uint8_t* pbc, int64_t atom, int axis, double* energy,
                       double* dE) {
  const Model& M = *static_cast<Model*>(model);
  bool anyp = pbc[0] || pbc[1] || pbc[2];
  if (M.hp.charges && anyp) return -3;  // the Coulomb term is defined for open systems
  double zero[9] = {0};
  uint8_t np[3] = {0, 0, 0};
  const double* cl = anyp ? cell : zero;
  std::vector<Edge> edges;
  if (brute_neighbors(pos, (int)n, cl, anyp ? pbc : np, M.hp.rc, edges) != 0) return -1;
  std::vector<int> rp = receiver_row_ptr(edges, (int)n);
  std::vector<Dual> p(3 * n);
  for (int64_t k = 0; k < 3 * n; ++k) p[k] = Dual(pos[k], (k == 3 * atom + axis) ? 1.0 : 0.0);
  std::vector<int> sp(species, species + n);
  Dual E = model_energy<Dual>(M, edges, rp, p.data(), sp.data(), (int)n, cl, nullptr, nullptr, nullptr);
  *energy = E.v;
  *dE = E.d;
  return 0;
}

// Node features h^layer [n][(L+1)^2][C] (layer 0: the embedding; layer t:
// after t interaction layers), for feature-level equivariance pins.
int oracle_node_features(void* model, const double* pos, const int32_t* species, int64_t n, const double* cell,
                         const uint8_t* pbc, int layer, double* out) {
  const Model& M = *static_cast<Model*>(model);
  if (layer < 0 || layer > M.hp.T) return -2;
  bool anyp = pbc[0] || pbc[1] || pbc[2];
  double zero[9] = {0};
  uint8_t np[3] = {0, 0, 0};
  const double* cl = anyp ? cell : zero;
  std::vector<Edge> edges;
  if (brute_neighbors(pos, (int)n, cl, anyp ? pbc : np, M.hp.rc, edges) != 0) return -1;
  std::vector<int> rp = receiver_row_ptr(edges, (int)n);
  std::vector<std::vector<double>> hs(M.hp.T + 1), us(M.hp.T), as(M.hp.T), gs(M.hp.T);
  model_energy<double>(M, edges, rp, pos, species, (int)n, cl, nullptr, &hs, &us, &as, &gs);
  std::copy(hs[layer].begin(), hs[layer].end(), out);
  return 0;
}

// Row (atom, axis) of the Hessian d2E / dr_{atom,axis} dr_{j,b} for every j, b
// (out [n][3]), one hyper-dual pass per column; the edge set is fixed at the
// given positions.  -dF_j,b / dr_atom,axis by symmetry: the subsampled Hessian
// rows of Eq. sampled_hessian2 for one graph.
int oracle_hessian_row(void* model, const double* pos, const int32_t* species, int64_t n, const double* cell,
                       const uint8_t* pbc, int64_t atom, int axis, double* out) {
  const Model& M = *static_cast<Model*>(model);
  bool anyp = pbc[0] || pbc[1] || pbc[2];
  if (M.hp.charges && anyp) return -3;
  double zero[9] = {0};
  uint8_t np[3] = {0, 0, 0};
  const double* cl = anyp ? cell : zero;
  std::vector<Edge> edges;
  if (brute_neighbors(pos, (int)n, cl, anyp ? pbc : np, M.hp.rc, edges) != 0) return -1;
  std::vector<int> rp = receiver_row_ptr(edges, (int)n);
  std::vector<int> sp(species, species + n);
  const int64_t row = 3 * atom + axis;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t col = 0; col < 3 * n; ++col) {
    std::vector<HDual> p(3 * n);
    for (int64_t k = 0; k < 3 * n; ++k) p[k] = HDual(pos[k], k == row ? 1.0 : 0.0, k == col ? 1.0 : 0.0, 0.0);
    HDual E = model_energy<HDual>(M, edges, rp, p.data(), sp.data(), (int)n, cl, nullptr, nullptr, nullptr);
    out[col] = E.ab;
  }
  return 0;
}

// Feature-level tensor product of one edge:
//   t[l3 m3][c] = sum_p w[p][c] sum C^p[m3][m1][m2] h[l1 m1][c] Y_{l2 m2}(v/|v|)
// h, t: [(L+1)^2][C]; w: [P][C].
int oracle_tp(int L, int Lsh, int C, const double* h, const double* v, const double* w, double* t) {
  std::vector<Path> ps = build_paths(L, Lsh);
  int D = (L + 1) * (L + 1);
  std::vector<double> Y((Lsh + 1) * (Lsh + 1));
  real_sh_vec<double>(Lsh, v[0], v[1], v[2], Y.data());
  std::fill(t, t + (size_t)D * C, 0.0);
  for (size_t p = 0; p < ps.size(); ++p)
    for (const CGEntry& ce : ps[p].nz) {
      int i3 = lm(ps[p].l3, ce.m3), i1 = lm(ps[p].l1, ce.m1), i2 = lm(ps[p].l2, ce.m2);
      for (int c = 0; c < C; ++c) t[(size_t)i3 * C + c] += w[p * C + c] * ce.c * h[(size_t)i1 * C + c] * Y[i2];
    }
  return 0;
}

// Couplings (l1, l2, l3) of the symmetric contraction for node order L;
// returns their count, writes 3 ints each if out != NULL.
int oracle_sc_paths(int L, int* out) {
  std::vector<Path> ps = build_sc_paths(L);
  if (out)
    for (size_t k = 0; k < ps.size(); ++k) {
      out[3 * k] = ps[k].l1; out[3 * k + 1] = ps[k].l2; out[3 * k + 2] = ps[k].l3;
    }
  return (int)ps.size();
}

// Symmetric contraction of one node: A, B [(L+1)^2][C]; w1 [L+1][C]; w2 [Q][C].
int oracle_sym_contract(int L, int C, const double* A, const double* w1, const double* w2, double* B) {
  std::vector<Path> ps = build_sc_paths(L);
  sym_contract<double>(ps, L, C, A, w1, w2, B);
  return 0;
}

// Its adjoint: GA = dE/dA for GB = dE/dB at A.
int oracle_sym_contract_adjoint(int L, int C, const double* A, const double* w1, const double* w2,
                                const double* GB, double* GA) {
  std::vector<Path> ps = build_sc_paths(L);
  sym_contract_adjoint(ps, L, C, A, w1, w2, GB, GA);
  return 0;
}

// Velocity Verlet, NVE, FP64.  Units: A, fs, amu, eV; kappa converts eV/A/amu
// to A/fs^2.  The neighbour list is rebuilt (brute force) at every force call.
//   v += dt/2 F/m kappa;  r += dt v;  F = F(r);  v += dt/2 F/m kappa.
// pe/ke receive n_steps+1 values (the start and after each step).
int oracle_vv_nve(void* model, double* pos, double* vel, const int32_t* species, const double* mass, int64_t n,
                  const double* cell, const uint8_t* pbc, double dt, int64_t n_steps, double* pe, double* ke) {
  const double kappa = 9.648533212e-3;
  std::vector<double> F(3 * n);
  double E;
  int rc = oracle_energy_forces(model, pos, species, n, cell, pbc, &E, F.data(), nullptr, nullptr);
  if (rc) return rc;
  auto kin = [&]() {
    double k = 0;
    for (int64_t i = 0; i < n; ++i)
      for (int a = 0; a < 3; ++a) k += 0.5 * mass[species[i]] * vel[3 * i + a] * vel[3 * i + a] / kappa;
    return k;
  };
  if (pe) pe[0] = E;
  if (ke) ke[0] = kin();
  for (int64_t s = 0; s < n_steps; ++s) {
    for (int64_t i = 0; i < n; ++i)
      for (int a = 0; a < 3; ++a) vel[3 * i + a] += 0.5 * dt * F[3 * i + a] / mass[species[i]] * kappa;
    for (int64_t k = 0; k < 3 * n; ++k) pos[k] += dt * vel[k];
    rc = oracle_energy_forces(model, pos, species, n, cell, pbc, &E, F.data(), nullptr, nullptr);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i)
      for (int a = 0; a < 3; ++a) vel[3 * i + a] += 0.5 * dt * F[3 * i + a] / mass[species[i]] * kappa;
    if (pe) pe[s + 1] = E;
    if (ke) ke[s + 1] = kin();
  }
  return 0;
}

}  // extern "C"
