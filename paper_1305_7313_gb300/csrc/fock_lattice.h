// fock_lattice.h — cell, reciprocal lattice, plane-wave spheres and Coulomb
// kernels on the host, shared by the Gamma-point and the k-point plans.
//
// Built with -ffp-contract=off: the spheres' order is defined by a fixed
// sequence of IEEE operations (no fused multiply-add), so every machine builds
// the same lists.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "fock.h"

namespace fockx {
namespace lattice {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 2.0 * 3.14159265358979323846;

inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Rows b_i = (2 pi / Omega) (a_j x a_k); returns the signed volume a1 . (a2 x a3).
inline double reciprocal(const double* cell, double* recip) {
  double c23[3], c31[3], c12[3];
  cross3(cell + 3, cell + 6, c23);
  cross3(cell + 6, cell + 0, c31);
  cross3(cell + 0, cell + 3, c12);
  const double vol = (cell[0] * c23[0] + cell[1] * c23[1]) + cell[2] * c23[2];
  const double fac = kTwoPi / vol;
  for (int x = 0; x < 3; ++x) {
    recip[0 + x] = c23[x] * fac;
    recip[3 + x] = c31[x] * fac;
    recip[6 + x] = c12[x] * fac;
  }
  return vol;
}

// |k + G|^2 with G = m1 b1 + m2 b2 + m3 b3 and k = kf1 b1 + kf2 b2 + kf3 b3:
// each component ((m1 + kf1) b1x + (m2 + kf2) b2x) + (m3 + kf3) b3x, then
// (x^2 + y^2) + z^2.  kf = 0 gives |G|^2 exactly.
inline double g2_of(const double* b, int m1, int m2, int m3, const double* kf = nullptr) {
  const double u1 = kf ? double(m1) + kf[0] : double(m1);
  const double u2 = kf ? double(m2) + kf[1] : double(m2);
  const double u3 = kf ? double(m3) + kf[2] : double(m3);
  double c[3];
  for (int x = 0; x < 3; ++x) c[x] = (u1 * b[0 + x] + u2 * b[3 + x]) + u3 * b[6 + x];
  return (c[0] * c[0] + c[1] * c[1]) + c[2] * c[2];
}

struct GEntry {
  double g2;
  int m[3];
};

// The sphere |k + G|^2 <= 2 Ecut sorted by (|k + G|^2, m1, m2, m3); false if it
// does not fit on an N^3 grid (2 |m_a| >= N).
inline bool build_sphere(const double* cell, const double* recip, double ecut, int n, std::vector<GEntry>& sph,
                         const double* kf = nullptr) {
  const double gmax = std::sqrt(2.0 * ecut);
  int mmax[3];
  for (int i = 0; i < 3; ++i) {
    const double* a = cell + 3 * i;
    const double len = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    mmax[i] = (int)std::floor(gmax * len / kTwoPi + (kf ? std::fabs(kf[i]) : 0.0)) + 1;
  }
  sph.clear();
  for (int m1 = -mmax[0]; m1 <= mmax[0]; ++m1)
    for (int m2 = -mmax[1]; m2 <= mmax[1]; ++m2)
      for (int m3 = -mmax[2]; m3 <= mmax[2]; ++m3) {
        const double g2 = g2_of(recip, m1, m2, m3, kf);
        if (g2 <= 2.0 * ecut) sph.push_back(GEntry{g2, {m1, m2, m3}});
      }
  std::sort(sph.begin(), sph.end(), [](const GEntry& x, const GEntry& y) {
    if (x.g2 != y.g2) return x.g2 < y.g2;
    if (x.m[0] != y.m[0]) return x.m[0] < y.m[0];
    if (x.m[1] != y.m[1]) return x.m[1] < y.m[1];
    return x.m[2] < y.m[2];
  });
  for (const GEntry& e : sph)
    for (int a = 0; a < 3; ++a)
      if (2 * std::abs(e.m[a]) >= n) return false;
  return true;
}

inline int freq_of(int k, int n) { return k < (n + 1) / 2 ? k : k - n; }

// v(G) and dv/domega for |G|^2 = g2 (Spencer-Alavi: Rc = (3 Omega / 4 pi)^(1/3)).
inline void kernel_value(fock_kernel kind, double vol, double omega, double g2, double* v, double* dv) {
  if (kind == FOCK_KERNEL_SPENCER_ALAVI) {
    const double rc = std::cbrt(3.0 * vol / (4.0 * kPi));
    if (g2 == 0.0) {
      *v = 2.0 * kPi * rc * rc;
    } else {
      const double s = std::sin(0.5 * std::sqrt(g2) * rc);
      *v = 8.0 * kPi * s * s / g2;
    }
    *dv = 0.0;
  } else {
    const double w = omega;
    *v = (g2 == 0.0) ? kPi / (w * w) : -4.0 * kPi * std::expm1(-g2 / (4.0 * w * w)) / g2;
    *dv = -(2.0 * kPi / (w * w * w)) * std::exp(-g2 / (4.0 * w * w));
  }
}

}  // namespace lattice
}  // namespace fockx
