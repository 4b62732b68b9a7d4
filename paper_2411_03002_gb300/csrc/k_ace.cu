// Linear atomic cluster expansion (Eq. energy_ace, linear part) for the atoms of
// the precise work queue, and its hand-written adjoint (forces).
//
// Basis (project-defined; the paper specifies ACE only by reference):
//   g_k(r)  = T_k(2r/rc - 1) f_cut(r/rc), k = 0..7          (f_cut of Appendix B)
//   R_nl(r) = sum_k W[l][n][k] g_k(r),    n = 0..7, l = 0..4
//   A_nlm   = (1/N0) sum_j R_nl(r_ij) Y_lm(r_ij/|r_ij|)     (real orthonormal Y_lm)
//   B: nu=1 A_n00; nu=2 sum_m A_n1lm A_n2lm; nu=3 sum_m G A A A (real Gaunt G)
//   E_i = sum_v c_v B_iv
// Because R is linear in g, A = W . G with G_klm = sum_j g_k Y_lm, and the force
// needs only u_klm = (1/N0) sum_n W[l][n][k] dE/dA_nlm per atom:
//   dE_i/dr_ij = sum_lm [ (sum_k u_klm g'_k) Y_lm r^ + (sum_k u_klm g_k) grad Y_lm ].
// One warp per precise atom, persistent CTAs pulling atoms from the queue:
//   pass 0   the row entries inside r_c are compacted (j and r_ij) into shared memory;
//   stage A  lanes evaluate g and Y for 32 neighbours into a shared tile, then
//            contract G = g^T Y with 4-wide vector loads along the neighbour axis;
//   stage B  nu=3 through per-lane gradient programs (no atomics per term), nu=2 as
//            symmetric 8x8 matrix-vector products per (l,m), nu=1 directly;
//   stage C  lanes recompute g, g', Y, grad Y per neighbour (no A tiles stored),
//            contract with u and scatter -w_i p_ij to neighbour j, +w_i sum p to i.
#include <complex>
#include <algorithm>
#include <cstring>
#include <cmath>

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
  t.c1.assign(8, 0.0);
  t.m2.assign(5 * 64, 0.0);
  std::vector<std::vector<std::pair<int, double>>> per_fn;
  for (int v = 0; v < t.nb; ++v) {
    const int* d = &t.desc[7 * v];
    double cv = (v < cfg.ace_nc) ? cfg.ace_c[v] : 0.0;
    if (d[0] == 1) {
      t.c1[d[1]] = cv;
    } else if (d[0] == 2) {
      int l = d[4], n1 = d[1], n2 = d[2];
      if (n1 == n2) {
        t.m2[l * 64 + n1 * 8 + n1] = 2.0 * cv;
      } else {
        t.m2[l * 64 + n1 * 8 + n2] = cv;
        t.m2[l * 64 + n2 * 8 + n1] = cv;
      }
    } else {
      int l1 = d[4], l2 = d[5], l3 = d[6];
      std::vector<std::pair<int, double>> terms;
      for (int m1 = -l1; m1 <= l1; ++m1)
        for (int m2 = -l2; m2 <= l2; ++m2)
          for (int m3 = -l3; m3 <= l3; ++m3) {
            double g = G(l1, m1, l2, m2, l3, m3);
            if (std::fabs(g) < 1e-14) continue;
            terms.push_back({aidx(d[1], l1, m1) | (aidx(d[2], l2, m2) << 8) | (aidx(d[3], l3, m3) << 16), cv * g});
          }
      per_fn.push_back(terms);
    }
  }
  t.term_idx.clear();
  t.term_coef.clear();
  for (size_t k = 0;; ++k) {
    bool any = false;
    for (auto& fn : per_fn)
      if (k < fn.size()) {
        t.term_idx.push_back(fn[k].first);
        t.term_coef.push_back(fn[k].second);
        any = true;
      }
    if (!any) break;
  }
  t.n_terms = (int)t.term_idx.size();

  // nu = 3 gradient as 32 balanced per-lane programs.  Each term coef*A1*A2*A3
  // contributes coef*A2*A3 to dE/dA1, coef*A1*A3 to dE/dA2 and coef*A1*A2 to dE/dA3;
  // the entries are sorted by output, cut into 32 contiguous ranges of equal
  // length, and a lane flushes its register sum whenever its output changes.
  auto c48 = [](int a) { return (a / 25) * 16 + (a % 25); };   // n <= 2, lm < 16
  struct E3 {
    int out, b, c;
    double coef;
  };
  std::vector<E3> ent;
  for (int k = 0; k < t.n_terms; ++k) {
    int pk = t.term_idx[k];
    int a1 = c48(pk & 255), a2 = c48((pk >> 8) & 255), a3 = c48((pk >> 16) & 255);
    double cf = t.term_coef[k];
    ent.push_back({a1, a2, a3, cf});
    ent.push_back({a2, a1, a3, cf});
    ent.push_back({a3, a1, a2, cf});
  }
  std::stable_sort(ent.begin(), ent.end(), [](const E3& x, const E3& y) { return x.out < y.out; });
  const int total = (int)ent.size();
  const int per = (total + 31) / 32;
  t.e3_len = per;
  t.e3_idx.assign((size_t)per * 32, 0u);
  t.e3_coef.assign((size_t)per * 32, 0.0);
  for (int lane = 0; lane < 32; ++lane) {
    int b0 = lane * per, b1 = std::min(total, b0 + per);
    for (int q = b0; q < b1; ++q) {
      bool flush = (q + 1 == b1) || ent[q + 1].out != ent[q].out;
      uint32_t p = (uint32_t)ent[q].b | ((uint32_t)ent[q].c << 6) | ((uint32_t)ent[q].out << 12) |
                   (flush ? (1u << 24) : 0u);
      t.e3_idx[(size_t)(q - b0) * 32 + lane] = p;
      t.e3_coef[(size_t)(q - b0) * 32 + lane] = ent[q].coef;
    }
  }
}

// ------------------------------------------------------------------ device code
namespace {

constexpr int kCols = 36;            // 32 neighbour slots + 4 pad (16-byte rows, conflict-free)
constexpr int kRows = 33;            // 8 radial + 25 angular rows
// Warps per CTA and the minimum resident CTAs per SM
// the compiler budgets registers for; compile-time tuning parameters.
#ifndef AP_ACE_WARPS
#define AP_ACE_WARPS 6
#endif
#ifndef AP_ACE_MINB
#define AP_ACE_MINB 4   // FP32 only: four 6-warp CTAs per SM (shared memory and <= 85 registers)
#endif
template <typename R>
constexpr int kWarps = sizeof(R) == 4 ? AP_ACE_WARPS : 4;

template <typename R>
struct V;
template <>
struct V<float> {
  using S4 = float4;
  using R4 = float4;
  static __device__ inline int code(const float4& s) { return __float_as_int(s.w); }
};
template <>
struct V<double> {
  using S4 = double4_32a;
  using R4 = double4_32a;
  static __device__ inline int code(const double4_32a& s) { return (int)s.w; }
};

__device__ inline float rsqrt_(float v) { return rsqrtf(v); }
__device__ inline double rsqrt_(double v) { return rsqrt(v); }

template <typename R>
__device__ inline typename V<R>::R4 ld4(const R* p) {
  return *reinterpret_cast<const typename V<R>::R4*>(p);
}

__device__ inline int l_of(int lm) { return lm >= 16 ? 4 : lm >= 9 ? 3 : lm >= 4 ? 2 : lm >= 1 ? 1 : 0; }

// Radial functions g_k and (optionally) dg_k/dr for r < rc.
template <typename R, bool D>
__device__ inline void radial(R r, R inv_rc, int mode, R g[8], R dg[8]) {
  R x = r * inv_rc;
  R t = mode == 1 ? R(2) * x - R(1) : x;
  R t2 = t * t;
  R poly = R(1) - R(1.875) * t + R(1.25) * t2 * t - R(0.375) * t2 * t2 * t;
  R fc = mode == 1 ? R(0.5) * poly : poly;
  R dfc = (R(-1.875) + R(3.75) * t2 - R(1.875) * t2 * t2) * inv_rc;
  R c = R(2) * x - R(1);
  R T0 = R(1), T1 = c, dT0 = R(0), dT1 = R(1);
  g[0] = fc;
  g[1] = c * fc;
  if (D) {
    dg[0] = dfc;
    dg[1] = R(2) * inv_rc * fc + c * dfc;
  }
#pragma unroll
  for (int k = 2; k < 8; ++k) {
    R T2 = R(2) * c * T1 - T0;
    R dT2 = R(2) * T1 + R(2) * c * dT1 - dT0;
    g[k] = T2 * fc;
    if (D) dg[k] = dT2 * R(2) * inv_rc * fc + T2 * dfc;
    T0 = T1;
    T1 = T2;
    dT0 = dT1;
    dT1 = dT2;
  }
}

// Real spherical harmonics of a unit vector (x, y, z), index lm = l^2 + l + m.
template <typename R>
__device__ inline void sh_values(R x, R y, R z, R Y[25]) {
  const R x2 = x * x, y2 = y * y, z2 = z * z;
  Y[0] = R(0.28209479177387814);
  Y[1] = R(0.4886025119029199) * y;
  Y[2] = R(0.4886025119029199) * z;
  Y[3] = R(0.4886025119029199) * x;
  Y[4] = R(1.0925484305920792) * x * y;
  Y[5] = R(1.0925484305920792) * y * z;
  Y[6] = R(0.31539156525252005) * (R(2) * z2 - x2 - y2);
  Y[7] = R(1.0925484305920792) * x * z;
  Y[8] = R(0.5462742152960396) * (x2 - y2);
  Y[9] = R(0.5900435899266435) * y * (R(3) * x2 - y2);
  Y[10] = R(2.890611442640554) * x * y * z;
  Y[11] = R(0.4570457994644658) * y * (R(4) * z2 - x2 - y2);
  Y[12] = R(0.3731763325901154) * z * (R(2) * z2 - R(3) * x2 - R(3) * y2);
  Y[13] = R(0.4570457994644658) * x * (R(4) * z2 - x2 - y2);
  Y[14] = R(1.445305721320277) * z * (x2 - y2);
  Y[15] = R(0.5900435899266435) * x * (x2 - R(3) * y2);
  const R rho = x2 + y2;
  Y[16] = R(2.5033429417967046) * x * y * (x2 - y2);
  Y[17] = R(1.7701307697799304) * y * z * (R(3) * x2 - y2);
  Y[18] = R(0.9461746957575601) * x * y * (R(6) * z2 - rho);
  Y[19] = R(0.6690465435572892) * y * z * (R(4) * z2 - R(3) * rho);
  Y[20] = R(0.10578554691520431) * (R(8) * z2 * z2 - R(24) * z2 * rho + R(3) * rho * rho);
  Y[21] = R(0.6690465435572892) * x * z * (R(4) * z2 - R(3) * rho);
  Y[22] = R(0.47308734787878004) * (x2 - y2) * (R(6) * z2 - rho);
  Y[23] = R(1.7701307697799304) * x * z * (x2 - R(3) * y2);
  Y[24] = R(0.6258357354491761) * (x2 * x2 - R(6) * x2 * y2 + y2 * y2);
}

// Block l of the homogeneous solid harmonics Z_lm (= Y_lm on the unit sphere) and
// their Cartesian gradients; the tangential gradient is grad Z - l Z u.
template <typename R, int L>
__device__ inline void sh_block(R x, R y, R z, R* Y, R* gx, R* gy, R* gz) {
  const R x2 = x * x, y2 = y * y, z2 = z * z;
  if constexpr (L == 0) {
    Y[0] = R(0.28209479177387814);
    gx[0] = gy[0] = gz[0] = R(0);
  } else if constexpr (L == 1) {
    const R c = R(0.4886025119029199);
    Y[0] = c * y; gx[0] = R(0); gy[0] = c; gz[0] = R(0);
    Y[1] = c * z; gx[1] = R(0); gy[1] = R(0); gz[1] = c;
    Y[2] = c * x; gx[2] = c; gy[2] = R(0); gz[2] = R(0);
  } else if constexpr (L == 2) {
    const R a = R(1.0925484305920792), b = R(0.31539156525252005), e = R(0.5462742152960396);
    Y[0] = a * x * y; gx[0] = a * y; gy[0] = a * x; gz[0] = R(0);
    Y[1] = a * y * z; gx[1] = R(0); gy[1] = a * z; gz[1] = a * y;
    Y[2] = b * (R(2) * z2 - x2 - y2); gx[2] = R(-2) * b * x; gy[2] = R(-2) * b * y; gz[2] = R(4) * b * z;
    Y[3] = a * x * z; gx[3] = a * z; gy[3] = R(0); gz[3] = a * x;
    Y[4] = e * (x2 - y2); gx[4] = R(2) * e * x; gy[4] = R(-2) * e * y; gz[4] = R(0);
  } else if constexpr (L == 3) {
    const R c3 = R(0.5900435899266435), c2 = R(2.890611442640554), c1 = R(0.4570457994644658);
    const R c0 = R(0.3731763325901154), c2h = R(1.445305721320277);
    Y[0] = c3 * y * (R(3) * x2 - y2); gx[0] = c3 * R(6) * x * y; gy[0] = c3 * (R(3) * x2 - R(3) * y2); gz[0] = R(0);
    Y[1] = c2 * x * y * z; gx[1] = c2 * y * z; gy[1] = c2 * x * z; gz[1] = c2 * x * y;
    Y[2] = c1 * y * (R(4) * z2 - x2 - y2); gx[2] = c1 * R(-2) * x * y;
    gy[2] = c1 * (R(4) * z2 - x2 - R(3) * y2); gz[2] = c1 * R(8) * y * z;
    Y[3] = c0 * z * (R(2) * z2 - R(3) * x2 - R(3) * y2); gx[3] = c0 * R(-6) * x * z; gy[3] = c0 * R(-6) * y * z;
    gz[3] = c0 * (R(6) * z2 - R(3) * x2 - R(3) * y2);
    Y[4] = c1 * x * (R(4) * z2 - x2 - y2); gx[4] = c1 * (R(4) * z2 - R(3) * x2 - y2);
    gy[4] = c1 * R(-2) * x * y; gz[4] = c1 * R(8) * x * z;
    Y[5] = c2h * z * (x2 - y2); gx[5] = c2h * R(2) * x * z; gy[5] = c2h * R(-2) * y * z; gz[5] = c2h * (x2 - y2);
    Y[6] = c3 * x * (x2 - R(3) * y2); gx[6] = c3 * (R(3) * x2 - R(3) * y2); gy[6] = c3 * R(-6) * x * y; gz[6] = R(0);
  } else {
    const R a = R(2.5033429417967046), b = R(1.7701307697799304), c = R(0.9461746957575601);
    const R d = R(0.6690465435572892), e = R(0.10578554691520431), f = R(0.47308734787878004);
    const R g = R(0.6258357354491761);
    const R rho = x2 + y2;
    Y[0] = a * x * y * (x2 - y2); gx[0] = a * (R(3) * x2 * y - y2 * y); gy[0] = a * (x2 * x - R(3) * x * y2); gz[0] = R(0);
    Y[1] = b * y * z * (R(3) * x2 - y2); gx[1] = b * R(6) * x * y * z; gy[1] = b * (R(3) * x2 * z - R(3) * y2 * z);
    gz[1] = b * (R(3) * x2 * y - y2 * y);
    Y[2] = c * x * y * (R(6) * z2 - rho); gx[2] = c * (R(6) * y * z2 - R(3) * x2 * y - y2 * y);
    gy[2] = c * (R(6) * x * z2 - x2 * x - R(3) * x * y2); gz[2] = c * R(12) * x * y * z;
    Y[3] = d * y * z * (R(4) * z2 - R(3) * rho); gx[3] = d * R(-6) * x * y * z;
    gy[3] = d * (R(4) * z2 * z - R(3) * x2 * z - R(9) * y2 * z); gz[3] = d * (R(12) * y * z2 - R(3) * x2 * y - R(3) * y2 * y);
    Y[4] = e * (R(8) * z2 * z2 - R(24) * z2 * rho + R(3) * rho * rho);
    gx[4] = e * x * (R(12) * rho - R(48) * z2); gy[4] = e * y * (R(12) * rho - R(48) * z2);
    gz[4] = e * (R(32) * z2 * z - R(48) * z * rho);
    Y[5] = d * x * z * (R(4) * z2 - R(3) * rho); gx[5] = d * (R(4) * z2 * z - R(9) * x2 * z - R(3) * y2 * z);
    gy[5] = d * R(-6) * x * y * z; gz[5] = d * (R(12) * x * z2 - R(3) * x2 * x - R(3) * x * y2);
    Y[6] = f * (x2 - y2) * (R(6) * z2 - rho); gx[6] = f * (R(12) * x * z2 - R(4) * x2 * x);
    gy[6] = f * (R(-12) * y * z2 + R(4) * y2 * y); gz[6] = f * (R(12) * x2 * z - R(12) * y2 * z);
    Y[7] = b * x * z * (x2 - R(3) * y2); gx[7] = b * (R(3) * x2 * z - R(3) * y2 * z); gy[7] = b * R(-6) * x * y * z;
    gz[7] = b * (x2 * x - R(3) * x * y2);
    Y[8] = g * (x2 * x2 - R(6) * x2 * y2 + y2 * y2); gx[8] = g * (R(4) * x2 * x - R(12) * x * y2);
    gy[8] = g * (R(-12) * x2 * y + R(4) * y2 * y); gz[8] = R(0);
  }
}

template <typename R>
__device__ inline void pair_disp(const SysInfo& S, const typename V<R>::S4& si, const typename V<R>::S4& sj,
                                 const int* off, size_t e, R d[3]) {
  int k0, k1, k2;
  if (off) {
    int p = off[e];
    k0 = off_x(p);
    k1 = off_y(p);
    k2 = off_z(p);
  } else {
    int wi = V<R>::code(si), wj = V<R>::code(sj);
    k0 = wrap_off(cell_x(wj) - cell_x(wi), S.nc[0], S.periodic[0]);
    k1 = wrap_off(cell_y(wj) - cell_y(wi), S.nc[1], S.periodic[1]);
    k2 = wrap_off(cell_z(wj) - cell_z(wi), S.nc[2], S.periodic[2]);
  }
  if constexpr (sizeof(R) == 4) {
    d[0] = (R)k0 * S.hf[0] + (sj.x - si.x);
    d[1] = (R)k1 * S.hf[1] + (sj.y - si.y);
    d[2] = (R)k2 * S.hf[2] + (sj.z - si.z);
  } else {
    d[0] = (R)k0 * S.h[0] + (sj.x - si.x);
    d[1] = (R)k1 * S.h[1] + (sj.y - si.y);
    d[2] = (R)k2 * S.h[2] + (sj.z - si.z);
  }
}

template <typename R>
__device__ inline void add_force(float4* facc32, double* facc64, int j, R sx, R sy, R sz) {
  if constexpr (sizeof(R) == 4) {
    atomicAdd(&facc32[j], make_float4(sx, sy, sz, 0.f));
  } else {
    atomicAdd(&facc64[3 * j + 0], sx);
    atomicAdd(&facc64[3 * j + 1], sy);
    atomicAdd(&facc64[3 * j + 2], sz);
  }
}

template <typename R, int L>
__device__ inline void force_block(const R* __restrict__ U, R ux, R uy, R uz, const R g[8], const R dg[8], R& pr,
                                   R& ptx, R& pty, R& ptz) {
  R Y[2 * L + 1], gx[2 * L + 1], gy[2 * L + 1], gz[2 * L + 1];
  sh_block<R, L>(ux, uy, uz, Y, gx, gy, gz);
#pragma unroll
  for (int m = 0; m < 2 * L + 1; ++m) {
    const int lm = L * L + m;
    auto ua = ld4<R>(&U[lm * 8]);
    auto ub = ld4<R>(&U[lm * 8 + 4]);
    R S = (ua.x * g[0] + ua.y * g[1]) + (ua.z * g[2] + ua.w * g[3]) + ((ub.x * g[4] + ub.y * g[5]) + (ub.z * g[6] + ub.w * g[7]));
    R Sp = (ua.x * dg[0] + ua.y * dg[1]) + (ua.z * dg[2] + ua.w * dg[3]) +
           ((ub.x * dg[4] + ub.y * dg[5]) + (ub.z * dg[6] + ub.w * dg[7]));
    pr += Sp * Y[m];
    R lz = R(L) * Y[m];
    ptx += S * (gx[m] - lz * ux);
    pty += S * (gy[m] - lz * uy);
    ptz += S * (gz[m] - lz * uz);
  }
}

template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline float pack_j(int j, float) { return __int_as_float(j); }
__device__ inline double pack_j(int j, double) { return __longlong_as_double((long long)j); }
__device__ inline int unpack_j(float v) { return __float_as_int(v); }
__device__ inline int unpack_j(double v) { return (int)__double_as_longlong(v); }

constexpr int kListCap = 192;   // neighbours inside ace_rc kept per precise atom (FCC bulk: 134)

template <typename R>
struct AceArgs {
  const int* queue;
  const DevScalars* sc;
  DevScalars* stats;
  int* counter;
  const SysInfo* sys;
  const int* atom_sys;
  const typename V<R>::S4* sh;
  const int* nbr;
  const int* off;
  const int* cnt;
  int cap;
  const double* lam;
  const int* term_idx;
  const R* term_coef;
  int n_terms;
  const uint32_t* e3_idx;
  const R* e3_coef;
  const uint2* e3_pack;   // FP32 programs as (index, coefficient bits) pairs
  int e3_len;
  const R* W;
  const R* M2;
  const R* C1;
  R rc2, inv_rc, inv_n0;
  int mode;
  double* e_prec;
  float4* facc32;
  double* facc64;
};

template <typename R, bool FORCES>
__global__ void __launch_bounds__(kWarps<R> * 32, sizeof(R) == 4 ? AP_ACE_MINB : 1) k_ace(AceArgs<R> a) {
  // Shared memory (every region a multiple of 32 bytes, so 4-wide FP64 loads stay aligned):
  //   W [320] | M2 [320] | C1 [8] |
  //   per warp: compacted neighbours [kListCap][4] | tile [kRows][kCols]
  // A, dA, U, the G scratch and the 48 nu=3 inputs alias the tile once stage A's
  // contraction is done.  The nu=3 gradient programs stay in global memory (L1).
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R* Ws = reinterpret_cast<R*>(smem_raw);
  R* M2 = Ws + 320;
  R* C1 = M2 + 320;
  R* wbase = C1 + 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R* list = wbase + warp * (4 * kListCap + kRows * kCols);
  R* tile = list + 4 * kListCap;
  R* A = tile;
  R* dA = tile + 200;
  R* U = tile + 400;
  R* Gs = tile + 600;
  R* A48 = tile + 800;
  for (int t = threadIdx.x; t < 320; t += blockDim.x) {
    Ws[t] = a.W[t];
    M2[t] = a.M2[t];
  }
  if (threadIdx.x < 8) C1[threadIdx.x] = a.C1[threadIdx.x];
  __syncthreads();
  const int m = a.sc->n_precise;
  const int kq = lane & 7, grp = lane >> 3;
  const unsigned lt_mask = (1u << lane) - 1u;
  while (true) {
    int q = 0;
    if (lane == 0) q = atomicAdd(a.counter, 1);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= m) break;
    const int i = a.queue[q];
    const SysInfo& S = a.sys[a.atom_sys ? a.atom_sys[i] : 0];
    const auto si = a.sh[i];
    const int c = a.cnt[q];
    const size_t row = (size_t)q * a.cap;

    // ---------------- pass 0: compact the row entries inside ace_rc (j and r_ij)
    int nin = 0;
    for (int base = 0; base < c; base += 32) {
      const int slot = base + lane;
      bool in = false;
      R d[3] = {R(0), R(0), R(0)};
      int j = 0;
      if (slot < c) {
        j = a.nbr[row + slot];
        auto sj = a.sh[j];
        pair_disp<R>(S, si, sj, a.off, row + slot, d);
        in = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < a.rc2;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, in);
      const int pos = nin + __popc(mask & lt_mask);
      if (in && pos < kListCap) {
        R* e = &list[4 * pos];
        e[0] = d[0];
        e[1] = d[1];
        e[2] = d[2];
        e[3] = pack_j(j, R(0));
      }
      nin += __popc(mask);
    }
    if (nin > kListCap) {
      if (lane == 0) atomicOr(&a.stats->err, kErrCapacity);
      nin = kListCap;
    }
    __syncwarp();

    // ---------------- stage A: G_klm = sum_j g_k Y_lm over the compacted neighbours
    R acc[7];
#pragma unroll
    for (int t = 0; t < 7; ++t) acc[t] = R(0);
    for (int base = 0; base < nin; base += 32) {
      const int slot = base + lane;
      R g[8], Y[25];
      if (slot < nin) {
        auto e = ld4<R>(&list[4 * slot]);
        R r2 = e.x * e.x + e.y * e.y + e.z * e.z;
        R ir = rsqrt_(r2);
        radial<R, false>(r2 * ir, a.inv_rc, a.mode, g, nullptr);
        sh_values<R>(e.x * ir, e.y * ir, e.z * ir, Y);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) g[k] = R(0);
#pragma unroll
        for (int k = 0; k < 25; ++k) Y[k] = R(0);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) tile[k * kCols + lane] = g[k];
#pragma unroll
      for (int k = 0; k < 25; ++k) tile[(8 + k) * kCols + lane] = Y[k];
      __syncwarp();
      const int nv = min(32, nin - base);
      for (int s4 = 0; s4 < (nv + 3) / 4; ++s4) {
        auto g4 = ld4<R>(&tile[kq * kCols + 4 * s4]);
#pragma unroll
        for (int t = 0; t < 7; ++t) {
          const int lm = grp + 4 * t;
          if (lm < 25) {
            auto y4 = ld4<R>(&tile[(8 + lm) * kCols + 4 * s4]);
            acc[t] += g4.x * y4.x + g4.y * y4.y + g4.z * y4.z + g4.w * y4.w;
          }
        }
      }
      __syncwarp();
    }
    // G into the scratch, then A = (1/N0) W . G
#pragma unroll
    for (int t = 0; t < 7; ++t) {
      const int lm = grp + 4 * t;
      if (lm < 25) Gs[kq * 25 + lm] = acc[t];
    }
    __syncwarp();
    for (int o = lane; o < 200; o += 32) {
      const int n = o / 25, lm = o - 25 * n, l = l_of(lm);
      const R* w = &Ws[(l * 8 + n) * 8];
      R s = R(0);
#pragma unroll
      for (int k = 0; k < 8; ++k) s += w[k] * Gs[k * 25 + lm];
      A[o] = s * a.inv_n0;
      dA[o] = R(0);
    }
    __syncwarp();

    // ---------------- stage B: E and dE/dA
    // nu = 3: each lane runs its gradient program over the 48 A entries with
    // n <= 2, l <= 3 and flushes one register sum per output; E3 follows from
    // Euler's identity for a homogeneous cubic, E3 = (1/3) sum_a A_a dE3/dA_a.
    // Then nu = 2 and nu = 1 for the outputs each lane owns.
    for (int v = lane; v < 48; v += 32) A48[v] = A[(v >> 4) * 25 + (v & 15)];
    __syncwarp();
    {
      R acc = R(0);
      const uint32_t* pi = a.e3_idx + lane;
      const R* pc = a.e3_coef + lane;
      const uint2* pp = a.e3_pack + lane;
#pragma unroll 4
      for (int k = 0; k < a.e3_len; ++k) {
        uint32_t p;
        R cf;
        if constexpr (sizeof(R) == 4) {
          const uint2 v = __ldg(pp + 32 * k);   // index and FP32 coefficient in one load
          p = v.x;
          cf = __uint_as_float(v.y);
        } else {
          p = __ldg(pi + 32 * k);
          cf = __ldg(pc + 32 * k);
        }
        acc += cf * A48[p & 63u] * A48[(p >> 6) & 63u];
        if (p & (1u << 24)) {
          const int o = (int)((p >> 12) & 63u);
          atomicAdd(&dA[(o >> 4) * 25 + (o & 15)], acc);
          acc = R(0);
        }
      }
    }
    __syncwarp();
    R e = R(0);
    for (int v = lane; v < 48; v += 32) e += A48[v] * dA[(v >> 4) * 25 + (v & 15)];
    e *= R(1.0 / 3.0);
    for (int o = lane; o < 200; o += 32) {
      const int n = o / 25, lm = o - 25 * n, l = l_of(lm);
      const R* mrow = &M2[l * 64 + n * 8];
      R s = R(0);
#pragma unroll
      for (int n2 = 0; n2 < 8; ++n2) s += mrow[n2] * A[n2 * 25 + lm];
      const R lin = lm == 0 ? C1[n] : R(0);
      e += A[o] * (R(0.5) * s + lin);
      if (FORCES) dA[o] += s + lin;
    }
    double E = warp_sum<double>((double)e);
    if (lane == 0) {
      a.e_prec[i] = E;
      atomicAdd(&a.stats->ace_pairs, (unsigned long long)nin);
      atomicAdd(&a.stats->ace_atoms, 1ull);
    }
    if (!FORCES) {
      __syncwarp();
      continue;
    }
    __syncwarp();
    // ---------------- stage C: u_klm and forces over the compacted neighbours
    for (int o = lane; o < 200; o += 32) {
      const int lm = o >> 3, k = o & 7, l = l_of(lm);
      R s = R(0);
#pragma unroll
      for (int n = 0; n < 8; ++n) s += Ws[(l * 8 + n) * 8 + k] * dA[n * 25 + lm];
      U[o] = s * a.inv_n0;
    }
    __syncwarp();
    const R wgt = (R)(1.0 - (a.lam ? a.lam[i] : 0.0));
    R pix = R(0), piy = R(0), piz = R(0);
    for (int base = 0; base < nin; base += 32) {
      const int slot = base + lane;
      if (slot >= nin) continue;
      auto ev = ld4<R>(&list[4 * slot]);
      const int j = unpack_j(ev.w);
      R r2 = ev.x * ev.x + ev.y * ev.y + ev.z * ev.z;
      R ir = rsqrt_(r2);
      R ux = ev.x * ir, uy = ev.y * ir, uz = ev.z * ir;
      R g[8], dg[8];
      radial<R, true>(r2 * ir, a.inv_rc, a.mode, g, dg);
      R pr = R(0), ptx = R(0), pty = R(0), ptz = R(0);
      force_block<R, 0>(U, ux, uy, uz, g, dg, pr, ptx, pty, ptz);
      force_block<R, 1>(U, ux, uy, uz, g, dg, pr, ptx, pty, ptz);
      force_block<R, 2>(U, ux, uy, uz, g, dg, pr, ptx, pty, ptz);
      force_block<R, 3>(U, ux, uy, uz, g, dg, pr, ptx, pty, ptz);
      force_block<R, 4>(U, ux, uy, uz, g, dg, pr, ptx, pty, ptz);
      R px = pr * ux + ptx * ir, py = pr * uy + pty * ir, pz = pr * uz + ptz * ir;
      pix += px;
      piy += py;
      piz += pz;
      add_force<R>(a.facc32, a.facc64, j, -wgt * px, -wgt * py, -wgt * pz);
    }
    pix = warp_sum<R>(pix);
    piy = warp_sum<R>(piy);
    piz = warp_sum<R>(piz);
    if (lane == 0) add_force<R>(a.facc32, a.facc64, i, wgt * pix, wgt * piy, wgt * piz);
    __syncwarp();
  }
}

__global__ void k_ace_finalize32(int n, const float4* __restrict__ acc, double* __restrict__ f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 v = acc[i];
  f[3 * i + 0] += (double)v.x;
  f[3 * i + 1] += (double)v.y;
  f[3 * i + 2] += (double)v.z;
}

__global__ void k_ace_finalize64(int n, const double* __restrict__ acc, double* __restrict__ f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  f[i] += acc[i];
}

template <typename R>
size_t ace_smem() {
  return sizeof(R) * (320 + 320 + 8) + sizeof(R) * kWarps<R> * (4 * kListCap + kRows * kCols);
}

template <typename R>
void run_ace(ap_ctx* c, const double* d_lam, const int* d_queue, double* d_e_prec, bool forces, cudaStream_t s) {
  AceArgs<R> a;
  a.queue = d_queue;
  a.sc = c->d_sc;
  a.stats = c->d_sc;
  a.counter = &c->d_sc->work_counter;
  a.sys = c->d_sys;
  a.atom_sys = c->d_atom_sys;
  if constexpr (sizeof(R) == 4)
    a.sh = c->d_sh32;
  else
    a.sh = c->d_sh64;
  a.nbr = c->d_nbr_ace;
  a.off = c->stored_off ? c->d_off_ace : nullptr;
  a.cnt = c->d_cnt_ace;
  a.cap = c->cap_ace;
  a.lam = d_lam;
  a.term_idx = c->d_term_idx;
  if constexpr (sizeof(R) == 4) {
    a.term_coef = c->d_term_coef32;
    a.W = c->d_W32;
    a.facc32 = c->d_facc32;
    a.facc64 = nullptr;
  } else {
    a.term_coef = c->d_term_coef64;
    a.W = c->d_W64;
    a.facc32 = nullptr;
    a.facc64 = c->d_facc64;
  }
  a.M2 = a.W + 320;   // the parameter block is [W (320) | M2 (320) | C1 (8)]
  a.C1 = a.W + 640;
  a.n_terms = c->ace.n_terms;
  a.e3_idx = c->d_e3_idx;
  a.e3_pack = c->d_e3_pack;
  a.e3_len = c->ace.e3_len;
  if constexpr (sizeof(R) == 4)
    a.e3_coef = c->d_e3_coef32;
  else
    a.e3_coef = c->d_e3_coef64;
  a.rc2 = (R)(c->cfg.ace_rc * c->cfg.ace_rc);
  a.inv_rc = (R)(1.0 / c->cfg.ace_rc);
  a.inv_n0 = (R)(1.0 / c->cfg.ace_n0);
  a.mode = c->cfg.fcut_mode;
  a.e_prec = d_e_prec;
  size_t smem = ace_smem<R>();
  auto kern = forces ? k_ace<R, true> : k_ace<R, false>;
  static int configured[2][2] = {{0, 0}, {0, 0}};
  static int blocks_per_sm[2][2] = {{0, 0}, {0, 0}};
  int pi = sizeof(R) == 4 ? 0 : 1, fi = forces ? 1 : 0;
  if (!configured[pi][fi]) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kWarps<R> * 32, smem);
    blocks_per_sm[pi][fi] = b > 0 ? b : 1;
    configured[pi][fi] = 1;
  }
  if (forces) {
    if constexpr (sizeof(R) == 4)
      cudaMemsetAsync(c->d_facc32, 0, sizeof(float4) * (size_t)c->n, s);
    else
      cudaMemsetAsync(c->d_facc64, 0, sizeof(double) * 3 * (size_t)c->n, s);
  }
  cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  int grid = c->num_sms * blocks_per_sm[pi][fi];
  kern<<<grid, kWarps<R> * 32, smem, s>>>(a);
  c->kernels += 1;
}

}  // namespace

void upload_ace_tables(ap_ctx* c) {
  const AceTables& t = c->ace;
  std::vector<float> cf32(t.term_coef.begin(), t.term_coef.end());
  std::vector<double> p64(c->cfg.ace_W, c->cfg.ace_W + 320);
  p64.insert(p64.end(), t.m2.begin(), t.m2.end());
  p64.insert(p64.end(), t.c1.begin(), t.c1.end());
  std::vector<float> p32(p64.begin(), p64.end());
  cudaMalloc(&c->d_term_idx, sizeof(int) * t.n_terms);
  cudaMalloc(&c->d_term_coef32, sizeof(float) * t.n_terms);
  cudaMalloc(&c->d_term_coef64, sizeof(double) * t.n_terms);
  cudaMalloc(&c->d_W32, sizeof(float) * p32.size());
  cudaMalloc(&c->d_W64, sizeof(double) * p64.size());
  cudaMemcpy(c->d_term_idx, t.term_idx.data(), sizeof(int) * t.n_terms, cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_term_coef32, cf32.data(), sizeof(float) * t.n_terms, cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_term_coef64, t.term_coef.data(), sizeof(double) * t.n_terms, cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_W32, p32.data(), sizeof(float) * p32.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_W64, p64.data(), sizeof(double) * p64.size(), cudaMemcpyHostToDevice);
  const size_t ne = t.e3_idx.size();
  std::vector<float> e32(t.e3_coef.begin(), t.e3_coef.end());
  cudaMalloc(&c->d_e3_idx, sizeof(uint32_t) * ne);
  cudaMalloc(&c->d_e3_coef32, sizeof(float) * ne);
  cudaMalloc(&c->d_e3_coef64, sizeof(double) * ne);
  cudaMemcpy(c->d_e3_idx, t.e3_idx.data(), sizeof(uint32_t) * ne, cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_e3_coef32, e32.data(), sizeof(float) * ne, cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_e3_coef64, t.e3_coef.data(), sizeof(double) * ne, cudaMemcpyHostToDevice);
  std::vector<uint2> pack(ne);
  for (size_t k = 0; k < ne; ++k) {
    float cf = (float)t.e3_coef[k];
    uint32_t bits;
    std::memcpy(&bits, &cf, sizeof(bits));
    pack[k] = make_uint2(t.e3_idx[k], bits);
  }
  cudaMalloc(&c->d_e3_pack, sizeof(uint2) * ne);
  cudaMemcpy(c->d_e3_pack, pack.data(), sizeof(uint2) * ne, cudaMemcpyHostToDevice);
}

void launch_ace(ap_ctx* c, const double* d_lam, const int* d_queue, double* d_e_prec, bool forces, cudaStream_t s) {
  if (c->cfg.precision == AP_PREC_FP64)
    run_ace<double>(c, d_lam, d_queue, d_e_prec, forces, s);
  else
    run_ace<float>(c, d_lam, d_queue, d_e_prec, forces, s);
}

void launch_ace_finalize(ap_ctx* c, double* d_f, cudaStream_t s) {
  c->kernels += 1;
  if (c->cfg.precision == AP_PREC_FP64)
    k_ace_finalize64<<<(int)((3 * c->n + 255) / 256), 256, 0, s>>>((int)c->n, c->d_facc64, d_f);
  else
    k_ace_finalize32<<<(int)((c->n + 255) / 256), 256, 0, s>>>((int)c->n, c->d_facc32, d_f);
}

}  // namespace ap
