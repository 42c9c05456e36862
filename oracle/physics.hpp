// Oracle physics: four-vectors, LO matrix element, running coupling, splitting
// kernels, the final-final dipole splitting map, and colour bookkeeping.
// Test infrastructure only (see oracle_api.h); plain FP64, no reordering
// beyond what the formulas state.
#pragma once
#include <cmath>
#include <cstdint>

namespace oracle {

constexpr double kPi = 3.14159265358979323846;
// QCD colour factors.
constexpr double kCF = 4.0 / 3.0;
constexpr double kCA = 3.0;
constexpr double kTR = 0.5;
constexpr double kNc = 3.0;
// Electroweak inputs of the LO cross section.  The paper names none; these are
// the values adopted for this build (Z mass and width, alpha_QED at the Z,
// sin^2 theta_W) and every pin is self-consistent with them.
constexpr double kMZ = 91.1876;
constexpr double kGammaZ = 2.4952;
constexpr double kAlphaQED = 1.0 / 128.802;
constexpr double kSin2W = 0.222;
constexpr double kGeV2ToPb = 0.389379e9;
constexpr int kGluon = 21;

struct Vec4 {
  double e, x, y, z;  // contravariant (E, px, py, pz)
};

inline Vec4 operator+(const Vec4& a, const Vec4& b) { return {a.e + b.e, a.x + b.x, a.y + b.y, a.z + b.z}; }
inline Vec4 operator-(const Vec4& a, const Vec4& b) { return {a.e - b.e, a.x - b.x, a.y - b.y, a.z - b.z}; }
inline Vec4 operator*(double s, const Vec4& a) { return {s * a.e, s * a.x, s * a.y, s * a.z}; }
// Minkowski product, metric (+,-,-,-).
inline double dot(const Vec4& a, const Vec4& b) { return a.e * b.e - a.x * b.x - a.y * b.y - a.z * b.z; }
inline double p3abs(const Vec4& a) { return std::sqrt(a.x * a.x + a.y * a.y + a.z * a.z); }

// ---------------------------------------------------------------- ME (App. B)
// Electroweak charges of the electron and of quark flavour f (PDG 1..5:
// d u s c b).  V = T3 - 2 Q sin^2(theta_W), A = T3.
struct Couplings {
  double q, v, a;
};
inline Couplings quark_couplings(int f) {
  const bool up = (f == 2 || f == 4);
  const double q = up ? 2.0 / 3.0 : -1.0 / 3.0;
  const double t3 = up ? 0.5 : -0.5;
  return {q, t3 - 2.0 * q * kSin2W, t3};
}
inline Couplings electron_couplings() {
  const double q = -1.0, t3 = -0.5;
  return {q, t3 - 2.0 * q * kSin2W, t3};
}

// d sigma / d cos(theta) for e+e- -> f fbar at LO with gamma/Z exchange and
// interference (Ellis-Stirling-Webber form), in pb.  theta is the angle of the
// quark to the electron beam (+z).  drop_interference is a planted mistake.
inline double dsigma_dcos(double s, int f, double cth, bool drop_interference) {
  const Couplings e = electron_couplings();
  const Couplings q = quark_couplings(f);
  const double kappa = 1.0 / (4.0 * kSin2W * (1.0 - kSin2W));
  const double den = (s - kMZ * kMZ) * (s - kMZ * kMZ) + kGammaZ * kGammaZ * kMZ * kMZ;
  double chi1 = kappa * s * (s - kMZ * kMZ) / den;
  const double chi2 = kappa * kappa * s * s / den;
  if (drop_interference) chi1 = 0.0;
  const double a0 = e.q * e.q * q.q * q.q + 2.0 * e.q * q.q * e.v * q.v * chi1 +
                    (e.a * e.a + e.v * e.v) * (q.a * q.a + q.v * q.v) * chi2;
  const double a1 = 2.0 * e.q * q.q * e.a * q.a * chi1 + 4.0 * e.a * e.v * q.a * q.v * chi2;
  const double pref = kPi * kAlphaQED * kAlphaQED / (2.0 * s) * kNc;
  return pref * ((1.0 + cth * cth) * a0 + 2.0 * cth * a1) * kGeV2ToPb;
}

// ------------------------------------------------------ running coupling
// One-loop alpha_s(t) = alpha_s(mZ^2) / (1 + alpha_s(mZ^2) b0 ln(t / mZ^2)),
// b0 = (33 - 2 nf) / (12 pi).  fixed = 1 returns alpha_s(mZ) everywhere.
inline double alphas_at(double t, double alphas_mz, int nf, bool fixed) {
  if (fixed) return alphas_mz;
  const double b0 = (33.0 - 2.0 * nf) / (12.0 * kPi);
  return alphas_mz / (1.0 + alphas_mz * b0 * std::log(t / (kMZ * kMZ)));
}

// ------------------------------------------------------ splitting kernels
// Kernel kinds; a gluon splitter carries half of each gluon kernel per dipole.
enum Kind { kQtoQG = 0, kGtoGG = 1, kGtoQQ = 2 };

// P(z, y): the splitting function entering the veto (App. A, Eq. (A.9)).
inline double kernel_value(int kind, double z, double y) {
  switch (kind) {
    case kQtoQG: return kCF * (2.0 / (1.0 - z * (1.0 - y)) - (1.0 + z));
    case kGtoGG: return kCA / 2.0 * (2.0 / (1.0 - z * (1.0 - y)) - 2.0 + z * (1.0 - z));
    default: return kTR / 2.0 * (1.0 - 2.0 * z * (1.0 - z));
  }
}
// P^over(z) >= P(z, y) for 0 < y < 1 (App. A, Eq. (A.4)).
inline double kernel_estimate(int kind, double z) {
  switch (kind) {
    case kQtoQG: return 2.0 * kCF / (1.0 - z);
    case kGtoGG: return kCA / (1.0 - z);
    default: return kTR / 2.0;
  }
}
// I^over(z), a primitive of P^over (App. A, after Eq. (A.8)).
inline double kernel_primitive(int kind, double z) {
  switch (kind) {
    case kQtoQG: return -2.0 * kCF * std::log(1.0 - z);
    case kGtoGG: return -kCA * std::log(1.0 - z);
    default: return kTR / 2.0 * z;
  }
}
// (I^over)^{-1}(x).
inline double kernel_primitive_inverse(int kind, double x) {
  switch (kind) {
    case kQtoQG: return 1.0 - std::exp(-x / (2.0 * kCF));
    case kGtoGG: return 1.0 - std::exp(-x / kCA);
    default: return x / (kTR / 2.0);
  }
}
// The integral of P^over over [zm, zp]: I(zp) - I(zm).
inline double kernel_integral(int kind, double zm, double zp) {
  return kernel_primitive(kind, zp) - kernel_primitive(kind, zm);
}
// z from Eq. (A.8): z = I^-1[I(zm) + (I(zp) - I(zm)) r].
inline double kernel_generate_z(int kind, double zm, double zp, double r, bool z_uniform) {
  if (z_uniform) return zm + (zp - zm) * r;  // planted mistake
  const double x = kernel_primitive(kind, zm) + (kernel_primitive(kind, zp) - kernel_primitive(kind, zm)) * r;
  return kernel_primitive_inverse(kind, x);
}

// ----------------------------------------------- final-final dipole map
// Minkowski-orthogonal complement of three four-vectors: the vector N with
// N.X = det[X; a; b; c] for every X (rows = contravariant components).
inline Vec4 levi_civita(const Vec4& a, const Vec4& b, const Vec4& c) {
  auto det3 = [](double a1, double a2, double a3, double b1, double b2, double b3, double c1,
                 double c2, double c3) {
    return a1 * (b2 * c3 - b3 * c2) - a2 * (b1 * c3 - b3 * c1) + a3 * (b1 * c2 - b2 * c1);
  };
  const double cof0 = det3(a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z);
  const double cof1 = -det3(a.e, a.y, a.z, b.e, b.y, b.z, c.e, c.y, c.z);
  const double cof2 = det3(a.e, a.x, a.z, b.e, b.x, b.z, c.e, c.x, c.z);
  const double cof3 = -det3(a.e, a.x, a.y, b.e, b.x, b.y, c.e, c.x, c.y);
  return {cof0, -cof1, -cof2, -cof3};
}

// Two unit spacelike vectors n1, n2, Minkowski-orthogonal to the massless
// dipole legs a, b and to each other.  n1 is built from the first reference
// direction r of (1,1,0,0), (1,0,1,0), (1,0,0,1) that is not within about
// 0.01 rad of either leg (|n1^2| >= 1e-4 before normalisation).
inline void transverse_basis(const Vec4& a, const Vec4& b, Vec4& n1, Vec4& n2) {
  const Vec4 refs[3] = {{1, 1, 0, 0}, {1, 0, 1, 0}, {1, 0, 0, 1}};
  const double ab = dot(a, b);
  for (int r = 0; r < 3; ++r) {
    const Vec4& ref = refs[r];
    n1 = ref - (dot(ref, b) / ab) * a - (dot(ref, a) / ab) * b;
    if (std::fabs(dot(n1, n1)) >= 1e-4 || r == 2) break;
  }
  n1 = (1.0 / std::sqrt(-dot(n1, n1))) * n1;
  n2 = levi_civita(a, b, n1);
  n2 = (1.0 / std::sqrt(-dot(n2, n2))) * n2;
}

// Catani-Seymour final-final map: splitter pij and spectator pk (massless)
// become p_i, p_j, p_k with
//   p_i = z pij + (1-z) y pk + k_perp,  p_j = (1-z) pij + z y pk - k_perp,
//   p_k = (1-y) pk,  k_perp^2 = -z(1-z) y Q^2,  Q^2 = 2 pij.pk.
struct MapMutations {
  bool no_recoil, kt_sign, z_swap;
};
inline void splitting_map(const Vec4& pij, const Vec4& pk, double z, double y, double phi,
                          const MapMutations& mut, Vec4& pi, Vec4& pj, Vec4& pk_new) {
  const double q2 = 2.0 * dot(pij, pk);
  Vec4 n1, n2;
  transverse_basis(pij, pk, n1, n2);
  const double kt = std::sqrt(z * (1.0 - z) * y * q2);
  const Vec4 kperp = kt * (std::cos(phi) * n1 + std::sin(phi) * n2);
  const double zi = mut.z_swap ? 1.0 - z : z;
  pi = zi * pij + ((1.0 - zi) * y) * pk + kperp;
  pj = (1.0 - zi) * pij + (zi * y) * pk + (mut.kt_sign ? kperp : (-1.0) * kperp);
  pk_new = mut.no_recoil ? pk : (1.0 - y) * pk;
}

}  // namespace oracle
