// Host-side ACE tables (no device code): the real Gaunt coefficients by the Racah
// 3j formula and the real/complex transform, the enumeration of the 325
// B-functions, the nu = 1 and nu = 2 coefficient arrays, the flattened nu = 3
// product terms and the merged nu = 3 monomials.  Compiled into the library and into the
// generator gen_nu3.cpp, which writes the monomial structure to ace_nu3.inc.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>

#include "ap_internal.cuh"

namespace ap {

// ------------------------------------------------------------------ host tables
namespace {

double fact(int n) {
  double r = 1.0;
  for (int k = 2; k <= n; ++k) r *= (double)k;
  return r;
}

// Wigner 3j symbol by the Racah formula.
double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
  double pre = std::sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) * fact(j3 + m3) *
                         fact(j3 - m3));
  double sum = 0.0;
  for (int k = 0; k <= j1 + j2 + j3; ++k) {
    int a1 = j3 - j2 + k + m1, a2 = j3 - j1 + k - m2, a3 = j1 + j2 - j3 - k, a4 = j1 - k - m1, a5 = j2 - k + m2;
    if (a1 < 0 || a2 < 0 || a3 < 0 || a4 < 0 || a5 < 0) continue;
    sum += ((k & 1) ? -1.0 : 1.0) / (fact(k) * fact(a1) * fact(a2) * fact(a3) * fact(a4) * fact(a5));
  }
  int ph = j1 - j2 - m3;
  return ((ph % 2 != 0) ? -1.0 : 1.0) * pre * sum;
}

// Integral of three complex spherical harmonics (Condon-Shortley phase).
double gaunt_complex(int l1, int m1, int l2, int m2, int l3, int m3) {
  double w0 = wigner3j(l1, l2, l3, 0, 0, 0);
  if (w0 == 0.0) return 0.0;
  return std::sqrt((2.0 * l1 + 1.0) * (2.0 * l2 + 1.0) * (2.0 * l3 + 1.0) / (4.0 * M_PI)) * w0 *
         wigner3j(l1, l2, l3, m1, m2, m3);
}

// Real harmonic (no Condon-Shortley phase, Y_1,-1 ~ y, Y_11 ~ x) as a combination
// of complex ones: returns the coefficient of Y_l^m in R_l,mu.
std::complex<double> real_from_complex(int mu, int m) {
  const double s = 1.0 / std::sqrt(2.0);
  if (mu == 0) return m == 0 ? 1.0 : 0.0;
  int a = std::abs(mu);
  double sg = (a & 1) ? -1.0 : 1.0;
  if (mu > 0) {
    if (m == a) return sg * s;
    if (m == -a) return s;
    return 0.0;
  }
  if (m == a) return std::complex<double>(0.0, -sg * s);
  if (m == -a) return std::complex<double>(0.0, s);
  return 0.0;
}

double gaunt_real(int l1, int u1, int l2, int u2, int l3, int u3) {
  std::complex<double> acc = 0.0;
  int m1s[2] = {std::abs(u1), -std::abs(u1)};
  int m2s[2] = {std::abs(u2), -std::abs(u2)};
  int m3s[2] = {std::abs(u3), -std::abs(u3)};
  for (int a = 0; a < (u1 ? 2 : 1); ++a)
    for (int b = 0; b < (u2 ? 2 : 1); ++b)
      for (int c = 0; c < (u3 ? 2 : 1); ++c) {
        int m1 = m1s[a], m2 = m2s[b], m3 = m3s[c];
        std::complex<double> k =
            real_from_complex(u1, m1) * real_from_complex(u2, m2) * real_from_complex(u3, m3);
        if (k == std::complex<double>(0.0, 0.0)) continue;
        acc += k * gaunt_complex(l1, m1, l2, m2, l3, m3);
      }
  return acc.real();
}

inline int aidx(int n, int l, int m) { return n * 25 + l * l + l + m; }

}  // namespace

void build_ace_tables(const ap_config& cfg, AceTables& t) {
  t.gaunt.assign(4 * 7 * 4 * 7 * 4 * 7, 0.0);
  auto G = [&](int l1, int m1, int l2, int m2, int l3, int m3) -> double& {
    return t.gaunt[((((l1 * 7 + m1 + 3) * 4 + l2) * 7 + m2 + 3) * 4 + l3) * 7 + m3 + 3];
  };
  for (int l1 = 0; l1 <= 3; ++l1)
    for (int m1 = -l1; m1 <= l1; ++m1)
      for (int l2 = 0; l2 <= 3; ++l2)
        for (int m2 = -l2; m2 <= l2; ++m2)
          for (int l3 = 0; l3 <= 3; ++l3)
            for (int m3 = -l3; m3 <= l3; ++m3) G(l1, m1, l2, m2, l3, m3) = gaunt_real(l1, m1, l2, m2, l3, m3);
  // enumeration: nu=1 by n; nu=2 by (n1 <= n2, l); nu=3 by (p1 <= p2 <= p3), p = 4n + l
  t.desc.clear();
  for (int n = 0; n < 8; ++n) t.desc.insert(t.desc.end(), {1, n, 0, 0, 0, 0, 0});
  for (int n1 = 0; n1 < 8; ++n1)
    for (int n2 = n1; n2 < 8; ++n2)
      for (int l = 0; l <= 4; ++l) t.desc.insert(t.desc.end(), {2, n1, n2, 0, l, l, 0});
  for (int p1 = 0; p1 < 12; ++p1)
    for (int p2 = p1; p2 < 12; ++p2)
      for (int p3 = p2; p3 < 12; ++p3) {
        int l1 = p1 & 3, l2 = p2 & 3, l3 = p3 & 3;
        if (l3 < std::abs(l1 - l2) || l3 > l1 + l2 || ((l1 + l2 + l3) & 1)) continue;
        double mx = 0.0;
        for (int m1 = -l1; m1 <= l1; ++m1)
          for (int m2 = -l2; m2 <= l2; ++m2)
            for (int m3 = -l3; m3 <= l3; ++m3) mx = std::fmax(mx, std::fabs(G(l1, m1, l2, m2, l3, m3)));
        if (mx < 1e-12) continue;
        t.desc.insert(t.desc.end(), {3, p1 >> 2, p2 >> 2, p3 >> 2, l1, l2, l3});
      }
  t.nb = (int)(t.desc.size() / 7);
  // nu = 1: E1 = sum_n c1[n] A_n00.
  // nu = 2: E2 = 1/2 sum_lm A_lm^T M_l A_lm with the symmetric 8x8 matrices
  //         M_l[n1][n2] = c(n1,n2,l) (n1 != n2), M_l[n][n] = 2 c(n,n,l), so that
  //         dE2/dA_{n,lm} = sum_n2 M_l[n][n2] A_{n2,lm}.
  // nu = 3: flattened Gaunt product terms coef * A[a1] A[a2] A[a3] (coef = c_v G),
  //         interleaved across functions so that neighbouring terms touch
  //         different A entries.
  // The nu = 3 Gaunt product terms of every function (structure only).
  struct Term {
    int idx;     // a1 | a2 << 8 | a3 << 16 over the 200 A entries
    int fn;      // the B-function v
    double g;    // real Gaunt coefficient
  };
  std::vector<std::vector<Term>> per_fn;
  for (int v = 0; v < t.nb; ++v) {
    const int* d = &t.desc[7 * v];
    if (d[0] != 3) continue;
    int l1 = d[4], l2 = d[5], l3 = d[6];
    std::vector<Term> terms;
    for (int m1 = -l1; m1 <= l1; ++m1)
      for (int m2 = -l2; m2 <= l2; ++m2)
        for (int m3 = -l3; m3 <= l3; ++m3) {
          double g = G(l1, m1, l2, m2, l3, m3);
          if (std::fabs(g) < 1e-14) continue;
          terms.push_back({aidx(d[1], l1, m1) | (aidx(d[2], l2, m2) << 8) | (aidx(d[3], l3, m3) << 16), v, g});
        }
    per_fn.push_back(terms);
  }
  // flattened, interleaved across functions
  std::vector<Term> flat;
  for (size_t k = 0;; ++k) {
    bool any = false;
    for (auto& fn : per_fn)
      if (k < fn.size()) {
        flat.push_back(fn[k]);
        any = true;
      }
    if (!any) break;
  }
  t.n_terms = (int)flat.size();
  t.term_idx.clear();
  for (const Term& u : flat) t.term_idx.push_back(u.idx);

  auto c48 = [](int a) { return (a / 25) * 16 + (a % 25); };   // n <= 2, lm < 16
  // nu = 3 as merged monomials: every term coef*A1*A2*A3 with its three indices in
  // the 48-entry numbering, sorted (a <= b <= c), and the coefficients of equal
  // monomials summed (E3 is a sum of monomials, so merging is exact algebra).
  // Ordered by the packed key c | b << 6 | a << 12, i.e. by (a, b, c); the structure
  // does not depend on the coefficients (terms with c_v = 0 stay, coefficient 0).
  std::vector<uint32_t> key_of(flat.size());
  std::map<uint32_t, int> slot;
  for (size_t k = 0; k < flat.size(); ++k) {
    int pk = flat[k].idx;
    int v[3] = {c48(pk & 255), c48((pk >> 8) & 255), c48((pk >> 16) & 255)};
    std::sort(v, v + 3);
    key_of[k] = (uint32_t)v[2] | ((uint32_t)v[1] << 6) | ((uint32_t)v[0] << 12);
    slot[key_of[k]] = 0;
  }
  t.nu3_key.clear();
  for (auto& kv : slot) {
    kv.second = (int)t.nu3_key.size();
    t.nu3_key.push_back(kv.first);
  }

  // Coefficient-dependent tables of one coefficient vector c:
  // nu = 1: E1 = sum_n c1[n] A_n00.
  // nu = 2: E2 = 1/2 sum_lm A_lm^T M_l A_lm with the symmetric 8x8 matrices
  //         M_l[n1][n2] = c(n1,n2,l) (n1 != n2), M_l[n][n] = 2 c(n,n,l), so that
  //         dE2/dA_{n,lm} = sum_n2 M_l[n][n2] A_{n2,lm}.
  // nu = 3: term coefficients c_v G and the merged monomial coefficients.
  auto coef_tables = [&](const double* c, int nc, std::vector<double>& c1, std::vector<double>& m2,
                         std::vector<double>& term_coef, std::vector<double>& nu3) {
    c1.assign(8, 0.0);
    m2.assign(5 * 64, 0.0);
    for (int v = 0; v < t.nb; ++v) {
      const int* d = &t.desc[7 * v];
      const double cv = (v < nc) ? c[v] : 0.0;
      if (d[0] == 1) {
        c1[d[1]] = cv;
      } else if (d[0] == 2) {
        int l = d[4], n1 = d[1], n2 = d[2];
        if (n1 == n2) {
          m2[l * 64 + n1 * 8 + n1] = 2.0 * cv;
        } else {
          m2[l * 64 + n1 * 8 + n2] = cv;
          m2[l * 64 + n2 * 8 + n1] = cv;
        }
      }
    }
    term_coef.assign(flat.size(), 0.0);
    nu3.assign(t.nu3_key.size(), 0.0);
    for (size_t k = 0; k < flat.size(); ++k) {
      const double cv = (flat[k].fn < nc) ? c[flat[k].fn] : 0.0;
      term_coef[k] = cv * flat[k].g;
      nu3[slot[key_of[k]]] += term_coef[k];
    }
  };
  coef_tables(cfg.ace_c, cfg.ace_nc, t.c1, t.m2, t.term_coef, t.nu3_coef);
  std::vector<double> unused;
  if (cfg.ace_fs_on)
    coef_tables(cfg.ace_c2, cfg.ace_nc, t.c1b, t.m2b, unused, t.nu3_coef2);
  else
    coef_tables(nullptr, 0, t.c1b, t.m2b, unused, t.nu3_coef2);
}

}  // namespace ap
