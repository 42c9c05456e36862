// Oracle: Durham jet rates, thrust, heavy-jet mass, validation and
// histogram binning (Sec. 3.1).  Test infrastructure only (see oracle_api.h).
#include <algorithm>
#include <cmath>
#include <map>

#include "oracle_internal.hpp"

namespace oracle {

// Durham (k_T) clustering in the E-scheme.  The measure of a pair is
//   y_ij = 2 min(E_i^2, E_j^2) (1 - cos theta_ij) / s;
// the pair with the smallest y_ij is merged by four-vector addition until one
// jet is left.  The y_min of the merge that takes n+1 jets to n is the jet
// resolution y_{n,n+1}; y_out = (y23, y34, y45, y56), -1 where the event never
// had n+1 partons.  Ties go to the first pair (i < j, lexicographic); the
// merged jet takes index i and the last jet moves into index j.
void durham(const std::vector<Vec4>& moms, double s, int mutation, double y_out[4]) {
  std::vector<Vec4> jets = moms;
  for (int m = 0; m < 4; ++m) y_out[m] = -1.0;
  const bool use_max = (mutation & ORACLE_MUT_DURHAM_MAX) != 0;
  while (jets.size() > 1) {
    const int n = static_cast<int>(jets.size());
    double ymin = 0.0;
    int bi = -1, bj = -1;
    for (int i = 0; i < n; ++i) {
      for (int j = i + 1; j < n; ++j) {
        const Vec4& a = jets[i];
        const Vec4& b = jets[j];
        const double cos_ij = (a.x * b.x + a.y * b.y + a.z * b.z) / (p3abs(a) * p3abs(b));
        const double e2 = use_max ? std::max(a.e * a.e, b.e * b.e) : std::min(a.e * a.e, b.e * b.e);
        const double y = 2.0 * e2 * (1.0 - cos_ij) / s;
        if (bi < 0 || y < ymin) {
          ymin = y;
          bi = i;
          bj = j;
        }
      }
    }
    // n jets -> n-1 jets records y_{n-1,n}; y23 is index 0.
    const int idx = n - 3;
    if (idx >= 0 && idx < 4) y_out[idx] = ymin;
    jets[bi] = jets[bi] + jets[bj];
    jets[bj] = jets.back();
    jets.pop_back();
  }
}

// Exact thrust T = max_n sum_i |p_i . n| / sum_i |p_i|.  The optimal plane
// separating the two hemispheres can be rotated until it contains two
// particles j, k, so it suffices to try, for every pair with p_j x p_k != 0,
// the partition P = sum_{i != j,k} sign(p_i . (p_j x p_k)) p_i together with
// the four assignments P +- p_j +- p_k of the pair itself.  The thrust axis is
// the longest such P.  Collinear configurations (all cross products zero,
// including two back-to-back partons) have T = 1 along the first momentum.
double thrust(const std::vector<Vec4>& moms, int mutation, Vec4* axis) {
  const int n = static_cast<int>(moms.size());
  double sum_abs = 0.0;
  for (const Vec4& m : moms) sum_abs += p3abs(m);
  double best2 = -1.0;
  double bx = 0, by = 0, bz = 0;
  const bool only_plus = (mutation & ORACLE_MUT_THRUST_NOSIGNS) != 0;
  for (int j = 0; j < n; ++j) {
    for (int k = j + 1; k < n; ++k) {
      const Vec4& a = moms[j];
      const Vec4& b = moms[k];
      const double nx = a.y * b.z - a.z * b.y;
      const double ny = a.z * b.x - a.x * b.z;
      const double nz = a.x * b.y - a.y * b.x;
      if (nx == 0.0 && ny == 0.0 && nz == 0.0) continue;
      double px = 0, py = 0, pz = 0;
      for (int i = 0; i < n; ++i) {
        if (i == j || i == k) continue;
        const Vec4& c = moms[i];
        const double d = c.x * nx + c.y * ny + c.z * nz;
        if (d >= 0.0) {
          px += c.x; py += c.y; pz += c.z;
        } else {
          px -= c.x; py -= c.y; pz -= c.z;
        }
      }
      for (int sj = 0; sj < 2; ++sj) {
        for (int sk = 0; sk < 2; ++sk) {
          if (only_plus && (sj || sk)) continue;
          const double fj = sj ? -1.0 : 1.0;
          const double fk = sk ? -1.0 : 1.0;
          const double cx = px + fj * a.x + fk * b.x;
          const double cy = py + fj * a.y + fk * b.y;
          const double cz = pz + fj * a.z + fk * b.z;
          const double c2 = cx * cx + cy * cy + cz * cz;
          if (c2 > best2) {
            best2 = c2;
            bx = cx; by = cy; bz = cz;
          }
        }
      }
    }
  }
  if (best2 < 0.0) {  // collinear: T = 1 along the first momentum
    const double a = p3abs(moms[0]);
    if (axis) *axis = Vec4{0.0, moms[0].x / a, moms[0].y / a, moms[0].z / a};
    return 1.0;
  }
  const double len = std::sqrt(best2);
  if (axis) *axis = Vec4{0.0, bx / len, by / len, bz / len};
  return len / sum_abs;
}

// out = (y23, y34, y45, y56, 1 - T, rho_H, B_T, B_W).  The hemispheres
// split the event by the sign of p_i . n_T (zero goes to the "+" side).  The
// heavy-jet mass is rho_H = max(M+^2, M-^2) / s.  The jet broadenings
// (Table 1's observable list) sum the momenta transverse to the thrust axis:
// B_+- = sum over the hemisphere of |p_i x n_T| / (2 sum_i |p_i|),
// B_T = B_+ + B_-, B_W = max(B_+, B_-).
void event_shapes(const std::vector<Vec4>& moms, double s, int mutation, double out[8]) {
  durham(moms, s, mutation, out);
  Vec4 axis{};
  const double t = thrust(moms, mutation, &axis);
  out[4] = 1.0 - t;
  Vec4 hp{0, 0, 0, 0}, hm{0, 0, 0, 0};
  for (const Vec4& m : moms) {
    const double d = m.x * axis.x + m.y * axis.y + m.z * axis.z;
    if (d >= 0.0) hp = hp + m;
    else hm = hm + m;
  }
  const double mp = dot(hp, hp), mm = dot(hm, hm);
  const double heavy = (mutation & ORACLE_MUT_HJM_LIGHT) ? std::min(mp, mm) : std::max(mp, mm);
  out[5] = heavy / s;
  double sum_abs = 0.0, bp = 0.0, bm = 0.0;
  for (const Vec4& m : moms) {
    sum_abs += p3abs(m);
    const double d = m.x * axis.x + m.y * axis.y + m.z * axis.z;
    const double cx = m.y * axis.z - m.z * axis.y;
    const double cy = m.z * axis.x - m.x * axis.z;
    const double cz = m.x * axis.y - m.y * axis.x;
    const double pt = (mutation & ORACLE_MUT_BROAD_DOT) ? std::fabs(d) : std::sqrt(cx * cx + cy * cy + cz * cz);
    if (d >= 0.0) bp += pt;
    else bm += pt;
  }
  bp /= 2.0 * sum_abs;
  bm /= 2.0 * sum_abs;
  out[6] = bp + bm;
  out[7] = std::max(bp, bm);
}

// Validation bits: 1 momentum not conserved to 1e-10 GeV, 2 a parton off
// shell (|p^2| > 1e-10 E sqrt(s): the dipole map forms every component from
// momenta of the event's scale, so FP64 masslessness holds to ~eps E sqrt(s),
// not eps E^2), 4 non-positive energy, 8 broken colour flow,
// 16 flavour imbalance, 32 non-finite component.
int validate(const std::vector<Parton>& ps, double sqrt_s) {
  int bits = 0;
  Vec4 sum{0, 0, 0, 0};
  for (const Parton& q : ps) {
    const Vec4& m = q.p;
    if (!std::isfinite(m.e) || !std::isfinite(m.x) || !std::isfinite(m.y) || !std::isfinite(m.z))
      bits |= 32;
    sum = sum + m;
    if (!(m.e > 0.0)) bits |= 4;
    if (std::fabs(dot(m, m)) > 1e-10 * m.e * sqrt_s) bits |= 2;
  }
  if (std::fabs(sum.e - sqrt_s) > 1e-10 || std::fabs(sum.x) > 1e-10 || std::fabs(sum.y) > 1e-10 ||
      std::fabs(sum.z) > 1e-10)
    bits |= 1;
  // Colour: every line index appears once as colour and once as anticolour;
  // quarks carry (c, 0), antiquarks (0, a), gluons (c, a); following colour
  // lines from each quark visits every parton and ends on an antiquark.
  std::map<int, int> by_col, by_acol;
  bool ok = true;
  int nflav[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < static_cast<int>(ps.size()); ++i) {
    const Parton& q = ps[i];
    if (q.flav == kGluon) {
      ok = ok && q.col > 0 && q.acol > 0;
    } else if (q.flav >= 1 && q.flav <= 5) {
      ok = ok && q.col > 0 && q.acol == 0;
      nflav[q.flav] += 1;
    } else if (q.flav <= -1 && q.flav >= -5) {
      ok = ok && q.col == 0 && q.acol > 0;
      nflav[-q.flav] -= 1;
    } else {
      ok = false;
    }
    if (q.col > 0) ok = ok && by_col.emplace(q.col, i).second;
    if (q.acol > 0) ok = ok && by_acol.emplace(q.acol, i).second;
  }
  if (ok) {
    for (const auto& kv : by_col) ok = ok && by_acol.count(kv.first) == 1;
    for (const auto& kv : by_acol) ok = ok && by_col.count(kv.first) == 1;
  }
  if (ok) {
    std::vector<int> seen(ps.size(), 0);
    for (int i = 0; i < static_cast<int>(ps.size()) && ok; ++i) {
      if (!(ps[i].flav >= 1 && ps[i].flav <= 5)) continue;
      int cur = i;
      for (size_t guard = 0; guard <= ps.size(); ++guard) {
        if (seen[cur]) { ok = false; break; }
        seen[cur] = 1;
        if (ps[cur].col == 0) break;  // reached the antiquark
        cur = by_acol[ps[cur].col];
      }
      ok = ok && ps[cur].flav <= -1 && ps[cur].flav >= -5;
    }
    for (int v : seen) ok = ok && v == 1;
  }
  if (!ok) bits |= 8;
  for (int f = 1; f <= 5; ++f)
    if (nflav[f] != 0) bits |= 16;
  return bits;
}

// Binning: log10 y23..y56 on [-4.3, -0.3], 1-T and rho_H on [0, 0.5]; 100
// bins each plus underflow (row 0) and overflow (row 101).  Undefined values
// (y <= 0) are not filled.  1-T and rho_H are non-negative by definition
// (Sec. 3.1); a negative value is the rounding of an exact zero (a two-parton
// event) and is binned as zero, so that it never depends on the sign of an
// ulp.  B_T and B_W are binned on [0, 0.4].
void histogram_fill(double* hist, const double obs[8], double w) {
  for (int h = 0; h < kNObs; ++h) {
    double x, lo, hi;
    if (h < 4) {
      if (!(obs[h] > 0.0)) continue;
      x = std::log10(obs[h]);
      lo = -4.3;
      hi = -0.3;
    } else {
      x = obs[h] > 0.0 ? obs[h] : 0.0;
      lo = 0.0;
      hi = h < 6 ? 0.5 : 0.4;
    }
    const double f = (x - lo) / (hi - lo) * kNBins;
    int bin;
    if (f < 0.0) bin = 0;
    else if (f >= kNBins) bin = kNBins + 1;
    else bin = 1 + static_cast<int>(f);
    double* cell = hist + (h * kRow + bin) * 3;
    cell[0] += w;
    cell[1] += w * w;
    cell[2] += 1.0;
  }
}

}  // namespace oracle
