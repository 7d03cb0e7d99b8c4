// Build-time generator of the coupling tables baked into the kernels.
//
// For node l_max L in {2, 3} and edge l_max 3 it enumerates the coupling paths
// (l1, l2, l3) in lexicographic order and computes each path's real coupling
// tensor C[m3][m1][m2] as an invariant integral over the sphere, normalised so
// that every m3 row has unit norm (the invariant tensor of a triangle-valid
// triple is unique up to scale, so this is the real Clebsch-Gordan tensor),
// with the sign fixed so that the first entry (lexicographic in m3, m1, m2)
// above 1e-8 in magnitude is positive:
//   l1 + l2 + l3 even (natural parity):  the Gaunt integral of
//       Y_{l3 m3} Y_{l1 m1} Y_{l2 m2};
//   l1 + l2 + l3 odd (pseudotensor paths, mixed-parity models): the integral of
//       Y_{l3 m3} r.(grad Y_{l1 m1} x grad Y_{l2 m2}), the triple product of the
//       surface gradients, which is rotation invariant and odd under inversion,
//       so it vanishes unless l1 + l2 + l3 is odd.
// The integrals use Gauss-Legendre nodes in cos(theta) (found by Newton's
// method) times a uniform grid in phi, exact for these polynomial degrees.
// Output: a C++ header of constexpr arrays: CGTable<L> (natural-parity paths)
// and CGTableP<L> (every triangle-valid path, both parities).
//
// Usage: gen_tables <output.inc>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "sh_poly.h"

namespace {

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n); w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
      double dp = n * (z * p1 - p0) / (z * z - 1);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1, p1 = z;
    for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
    double dp = n * (z * p1 - p0) / (z * z - 1);
    x[i] = z;
    w[i] = 2.0 / ((1 - z * z) * dp * dp);
  }
}

struct Entry { int p, i3, i1, i2; double c; };
struct PathT { int l1, l2, l3; };

void build(int L, bool all_parities, std::vector<PathT>& paths, std::vector<Entry>& entries) {
  const int nt = 12, np = 24;
  std::vector<double> zx, zw;
  gauss_legendre(nt, zx, zw);
  std::vector<std::vector<double>> Ys, dYs;  // harmonics and their gradients [16][3] at the nodes
  std::vector<std::array<double, 3>> rs;
  std::vector<double> qw;
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < np; ++b) {
      double phi = 2 * M_PI * b / np, z = zx[a], s = std::sqrt(1 - z * z);
      const double x = s * std::cos(phi), y = s * std::sin(phi);
      std::vector<double> Y(16), dY(48);
      mlip::sh3<double>(x, y, z, Y.data());
      for (int k = 0; k < 16; ++k) {  // gradient of polynomial k: its cotangent is e_k
        double e[16] = {0};
        e[k] = 1.0;
        mlip::sh3_vjp<double>(x, y, z, e, dY[3 * k], dY[3 * k + 1], dY[3 * k + 2]);
      }
      Ys.push_back(Y);
      dYs.push_back(dY);
      rs.push_back({x, y, z});
      qw.push_back(zw[a] * 2 * M_PI / np);
    }
  for (int l1 = 0; l1 <= L; ++l1)
    for (int l2 = 0; l2 <= 3; ++l2)
      for (int l3 = 0; l3 <= L; ++l3) {
        if (l3 < std::abs(l1 - l2) || l3 > l1 + l2) continue;
        const bool odd = (l1 + l2 + l3) % 2 != 0;
        if (odd && !all_parities) continue;
        const int n1 = 2 * l1 + 1, n2 = 2 * l2 + 1, n3 = 2 * l3 + 1;
        std::vector<double> G(n3 * n1 * n2, 0.0);
        for (size_t q = 0; q < qw.size(); ++q)
          for (int a = 0; a < n3; ++a)
            for (int b = 0; b < n1; ++b)
              for (int c = 0; c < n2; ++c) {
                double f;
                if (!odd) {
                  f = Ys[q][l1 * l1 + b] * Ys[q][l2 * l2 + c];
                } else {  // r . (grad Y1 x grad Y2)
                  const double* g1 = &dYs[q][3 * (l1 * l1 + b)];
                  const double* g2 = &dYs[q][3 * (l2 * l2 + c)];
                  const double cx = g1[1] * g2[2] - g1[2] * g2[1], cy = g1[2] * g2[0] - g1[0] * g2[2],
                               cz = g1[0] * g2[1] - g1[1] * g2[0];
                  f = rs[q][0] * cx + rs[q][1] * cy + rs[q][2] * cz;
                }
                G[(a * n1 + b) * n2 + c] += qw[q] * Ys[q][l3 * l3 + a] * f;
              }
        double nrm = 0;
        for (int b = 0; b < n1 * n2; ++b) nrm += G[b] * G[b];
        nrm = std::sqrt(nrm);
        double sign = 0;
        for (double v : G) if (std::fabs(v / nrm) > 1e-8) { sign = v > 0 ? 1 : -1; break; }
        const int p = (int)paths.size();
        paths.push_back({l1, l2, l3});
        for (int a = 0; a < n3; ++a)
          for (int b = 0; b < n1; ++b)
            for (int c = 0; c < n2; ++c) {
              double v = sign * G[(a * n1 + b) * n2 + c] / nrm;
              if (std::fabs(v) < 1e-12) continue;
              entries.push_back({p, l3 * l3 + a, l1 * l1 + b, l2 * l2 + c, v});
            }
      }
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 2) { std::fprintf(stderr, "usage: gen_tables out.inc\n"); return 2; }
  FILE* f = std::fopen(argv[1], "w");
  if (!f) return 1;
  std::fprintf(f, "// Generated by gen_tables.cpp: coupling paths and real Clebsch-Gordan entries.\n#pragma once\n");
  for (int variant = 0; variant < 4; ++variant) {
    const int L = 2 + (variant & 1);
    const bool all = variant >= 2;
    std::vector<PathT> paths;
    std::vector<Entry> e;
    build(L, all, paths, e);
    std::fprintf(f, "template <> struct %s<%d> {\n", all ? "CGTableP" : "CGTable", L);
    std::fprintf(f, "  static constexpr int P = %d;\n  static constexpr int NNZ = %d;\n", (int)paths.size(), (int)e.size());
    auto arr = [&](const char* name, auto get, int n) {
      std::fprintf(f, "  static constexpr int %s[%d] = {", name, n);
      for (int k = 0; k < n; ++k) std::fprintf(f, "%s%d", k ? "," : "", get(k));
      std::fprintf(f, "};\n");
    };
    arr("l1", [&](int k) { return paths[k].l1; }, (int)paths.size());
    arr("l2", [&](int k) { return paths[k].l2; }, (int)paths.size());
    arr("l3", [&](int k) { return paths[k].l3; }, (int)paths.size());
    // first entry of each path (P + 1 offsets)
    std::vector<int> off(paths.size() + 1, 0);
    for (auto& x : e) off[x.p + 1]++;
    for (size_t k = 0; k < paths.size(); ++k) off[k + 1] += off[k];
    arr("off", [&](int k) { return off[k]; }, (int)off.size());
    arr("ep", [&](int k) { return e[k].p; }, (int)e.size());
    arr("e3", [&](int k) { return e[k].i3; }, (int)e.size());
    arr("e1", [&](int k) { return e[k].i1; }, (int)e.size());
    arr("e2", [&](int k) { return e[k].i2; }, (int)e.size());
    std::fprintf(f, "  static constexpr float ec[%d] = {", (int)e.size());
    for (size_t k = 0; k < e.size(); ++k) std::fprintf(f, "%s%.9ef", k ? "," : "", e[k].c);
    std::fprintf(f, "};\n");
    std::fprintf(f, "  static constexpr double ecd[%d] = {", (int)e.size());
    for (size_t k = 0; k < e.size(); ++k) std::fprintf(f, "%s%.17e", k ? "," : "", e[k].c);
    std::fprintf(f, "};\n};\n");
  }
  std::fclose(f);
  return 0;
}
