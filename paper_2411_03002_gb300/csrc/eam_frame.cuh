// Shared device helpers of the kernels that walk the EAM rows (the EAM passes and
// the selector features): analytic EAM parameters in the working precision, the
// cell-relative shadow types, and the per-atom frame that turns a row entry into
// the pair displacement d = k h + s_j - s_i.
#pragma once

#include "ap_internal.cuh"

namespace ap {

template <typename R>
struct EamP {
  R beta, beta_r0, alpha, A, D, rp, rc, rc2, inv_h;
};

template <typename R>
struct Shadow;
template <>
struct Shadow<float> {
  using T = float4;
  static __device__ inline int code(const float4& s) { return __float_as_int(s.w); }
};
template <>
struct Shadow<double> {
  using T = double4_32a;
  static __device__ inline int code(const double4_32a& s) { return (int)s.w; }
};

template <typename R>
struct Q2;
template <>
struct Q2<float> {
  using T = float2;
  static __device__ inline float2 make(float a, float b) { return make_float2(a, b); }
};
template <>
struct Q2<double> {
  using T = double2;
  static __device__ inline double2 make(double a, double b) { return make_double2(a, b); }
};

__device__ inline float rexp(float v) { return __expf(v); }
__device__ inline double rexp(double v) { return exp(v); }
__device__ inline float rsqrt_(float v) { return rsqrtf(v); }
__device__ inline double rsqrt_(double v) { return rsqrt(v); }
// Tuning parameters of the EAM passes (compile-time): lanes per atom, minimum
// resident blocks per SM (register cap), unroll depth of the neighbour loops, and
// the FP32 reciprocal (1: approximate MUFU reciprocal, 0: correctly rounded).
#ifndef AP_EAM_LANES
#define AP_EAM_LANES 4
#endif
#ifndef AP_EAM_MINB
#define AP_EAM_MINB 5   // FP32 only: <= 51 registers, 40 resident warps per SM
#endif
#ifndef AP_EAM_UNROLL
#define AP_EAM_UNROLL 8   // unroll depth of the per-lane neighbour loops
#endif
#ifndef AP_EAM_FAST_RCP
#define AP_EAM_FAST_RCP 1
#endif
constexpr int kEamUnroll = AP_EAM_UNROLL;   // (#pragma unroll takes a constant expression, not a macro)

__device__ inline float rcp_(float v) {
#if AP_EAM_FAST_RCP
  return __fdividef(1.f, v);
#else
  return __frcp_rn(v);
#endif
}
__device__ inline double rcp_(double v) { return 1.0 / v; }

// Per-atom frame: cell code and box constants of atom i, held in registers.
template <typename R, bool STORED>
struct Frame {
  R hx, hy, hz;
  int cx, cy, cz;
  int nx, ny, nz;
  int halfx, halfy, halfz;   // nc/2 in periodic dimensions, a huge value otherwise
  R sx, sy, sz;

  template <typename S4>
  __device__ inline Frame(const SysInfo& S, const S4& si) {
    if constexpr (sizeof(R) == 4) {
      hx = S.hf[0];
      hy = S.hf[1];
      hz = S.hf[2];
    } else {
      hx = S.h[0];
      hy = S.h[1];
      hz = S.h[2];
    }
    int w = Shadow<R>::code(si);
    cx = cell_x(w);
    cy = cell_y(w);
    cz = cell_z(w);
    nx = S.nc[0];
    ny = S.nc[1];
    nz = S.nc[2];
    halfx = S.periodic[0] ? nx / 2 : 0x3fffffff;
    halfy = S.periodic[1] ? ny / 2 : 0x3fffffff;
    halfz = S.periodic[2] ? nz / 2 : 0x3fffffff;
    sx = si.x;
    sy = si.y;
    sz = si.z;
  }

  __device__ static inline int unwrap(int d, int n, int half) {
    d += (d < -half) ? n : 0;
    d -= (d > half) ? n : 0;
    return d;
  }

  template <typename S4>
  __device__ inline void disp(const S4& sj, const int* __restrict__ off, size_t e, R d[3]) const {
    int kx, ky, kz;
    if constexpr (STORED) {
      int p = off[e];
      kx = off_x(p);
      ky = off_y(p);
      kz = off_z(p);
    } else {
      int w = Shadow<R>::code(sj);
      kx = unwrap(cell_x(w) - cx, nx, halfx);
      ky = unwrap(cell_y(w) - cy, ny, halfy);
      kz = unwrap(cell_z(w) - cz, nz, halfz);
    }
    d[0] = (R)kx * hx + (sj.x - sx);
    d[1] = (R)ky * hy + (sj.y - sy);
    d[2] = (R)kz * hz + (sj.z - sz);
  }
};

template <typename T, int G>
__device__ inline T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

template <typename R>
EamP<R> make_params(const ap_config& c) {
  EamP<R> p;
  p.beta = (R)c.eam_beta;
  p.beta_r0 = (R)(c.eam_beta / c.eam_r0);
  p.alpha = (R)c.eam_alpha;
  p.A = (R)c.eam_A;
  p.D = (R)c.eam_D;
  p.rp = (R)c.eam_rp;
  p.rc = (R)c.eam_rc;
  p.rc2 = (R)(c.eam_rc * c.eam_rc);
  p.inv_h = (R)(1.0 / c.eam_h);
  return p;
}

// Accurate exponential for forms whose large terms cancel (the Mishin pair).
__device__ inline float rexp_acc(float v) { return expf(v); }
__device__ inline double rexp_acc(double v) { return exp(v); }
// Correctly rounded operations that the compiler may not contract into FMAs (the
// error-carrying sums below depend on each operation being rounded on its own).
__device__ inline float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ inline double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ inline float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ inline double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// The fast potential of the EAM passes as a functor over the pair distance r < rc:
//   zeta(r)                        density contribution,
//   pair(r, dzeta, phi, dphi)      zeta'(r), Phi(r), Phi'(r),
//   embed(rho, xi, dxi)            xi(rho), xi'(rho),
// and kMinBlocks, the resident 256-thread blocks per SM its FP32 kernels are
// compiled for (the register budget).
// PotSynth: the analytic synthetic EAM (zeta = exp(-beta (r/r0 - 1)) psi, Phi = Morse psi,
// xi = -A sqrt(rho)).  PotMishin: the Mishin EAM2 forms of Appendix E.
template <typename R>
struct PotSynth {
  static constexpr int kMinBlocks = AP_EAM_MINB;
  EamP<R> p;
  R rc2;
  __device__ inline R zeta(R r) const {
    const R u = (r - p.rc) * p.inv_h;
    const R u2 = u * u;
    const R u4 = u2 * u2;
    return rexp(p.beta - p.beta_r0 * r) * (u4 * rcp_(R(1) + u4));
  }
  __device__ inline void pair(R r, R& dzeta, R& phi, R& dphi) const {
    const R u = (r - p.rc) * p.inv_h;
    const R u2 = u * u;
    const R u4 = u2 * u2;
    const R inv = rcp_(R(1) + u4);
    const R ps = u4 * inv;
    const R dps = R(4) * u2 * u * inv * inv * p.inv_h;
    const R ez = rexp(p.beta - p.beta_r0 * r);
    dzeta = ez * (dps - p.beta_r0 * ps);
    const R e1 = rexp(-p.alpha * (r - p.rp));
    const R e2 = e1 * e1;
    const R m = p.D * (e2 - R(2) * e1);
    const R dm = R(2) * p.alpha * p.D * (e1 - e2);
    dphi = dm * ps + m * dps;
    phi = m * ps;
  }
  __device__ inline void embed(R rho, R& xi, R& dxi) const {
    xi = R(0);
    dxi = R(0);
    if (rho > R(0)) {
      const R s = sqrt(rho);
      xi = -p.A * s;
      dxi = R(-0.5) * p.A * rcp_(s);
    }
  }
};

// Mishin EAM2 (Appendix E):
//   Phi(r)  = (E1 M(r, r01, a1) + E2 M(r, r02, a2) + delta) psi((r - rc)/h) - sum_n Theta(rs_n - r) S_n (rs_n - r)^4
//   zeta(r) = (a exp(-b1 (r - r03)^2) + exp(-b2 (r - r04))) psi((r - rc)/h)
//   xi(x)   = xi0 + xi2/2 y^2 + q1 y^3 + q2 y^4 + q3 y^5 + q4 y^6                     (x <= 1, y = x - 1)
//           = (xi0 + xi2/2 y^2 + q1 y^3 + Q1 y^4) / (1 + Q2 y^3)                      (x > 1)
//   plus the fitted offset F0; M(r, r0, a) = exp(-2a(r - r0)) - 2 exp(-a(r - r0)).  The
// second density exponent is taken only above the precision's underflow limit.
//
// Near the first shell E1 M1 and E2 M2 are a few eV each and cancel to a fraction of
// an eV, and the pairs of an atom sit at similar r.  Rounding E, a and r0 to FP32
// (and the inexact r - r01) would then shift every pair the same way, by a few 1e-6 eV
// per atom.  So each Morse term keeps E, a, r0 as (hi, lo) pairs (lo = 0 in FP64) and
// forms a (r - r0) with the errors of the subtraction (TwoSum) and of the product
// (FMA) carried: the exponent is within half an ulp of its exact value, unbiased.
template <typename R>
struct PotMishin {
  static constexpr int kMinBlocks = 4;   // <= 64 registers: the compensated terms fit unspilled
  R E1, E2, delta, F0, xi0, xi2, inv_h, q1, q2, q3, q4, Q1, Q2, S1, S2, S3, a, a1, a2, b1, b2, r01, r02, r03, r04,
      rs1, rs2, rs3, rc;
  R E1l, E2l, a1l, a2l, r01l, r02l;      // low parts of the Morse constants
  R rc2;
  __device__ inline void psi(R r, R& ps, R& dps) const {
    const R u = (r - rc) * inv_h;
    const R u2 = u * u;
    const R u4 = u2 * u2;
    const R inv = rcp_(R(1) + u4);
    ps = u4 * inv;
    dps = R(4) * u2 * u * inv * inv * inv_h;
  }
  // E (exp(-2a(r - r0)) - 2 exp(-a(r - r0))) and its r-derivative
  __device__ inline void morse(R r, R Eh, R El, R ah, R al, R r0h, R r0l, R& m, R& dm) const {
    const R b = -r0h;
    const R s = add_rn(r, b);
    const R bb = add_rn(s, -r);
    const R te = add_rn(add_rn(r, -add_rn(s, -bb)), add_rn(b, -bb));   // r - r0h = s + te exactly
    const R p = mul_rn(ah, s);
    const R pe = fma(ah, s, -p);                                         // ah s = p + pe exactly
    const R arg = -add_rn(p, add_rn(pe, fma(ah, add_rn(te, -r0l), mul_rn(al, s))));
    const R e = rexp_acc(arg);
    const R u = e * (e - R(2));
    m = fma(Eh, u, El * u);
    dm = R(2) * Eh * ah * e * (R(1) - e);
  }
  __device__ inline void rho0(R r, R& g, R& dg) const {
    const R x = r - r03;
    const R e = rexp_acc(-b1 * x * x);
    const R arg = -b2 * (r - r04);
    const R e2 = arg > (sizeof(R) == 4 ? R(-80) : R(-700)) ? rexp_acc(arg) : R(0);
    g = a * e + e2;
    dg = R(-2) * b1 * x * a * e - b2 * e2;
  }
  __device__ inline R zeta(R r) const {
    R ps, dps, g, dg;
    psi(r, ps, dps);
    rho0(r, g, dg);
    return g * ps;
  }
  __device__ inline void pair(R r, R& dzeta, R& phi, R& dphi) const {
    R ps, dps, g, dg;
    psi(r, ps, dps);
    rho0(r, g, dg);
    dzeta = dg * ps + g * dps;
    R m1, dm1, m2, dm2;
    morse(r, E1, E1l, a1, a1l, r01, r01l, m1, dm1);
    morse(r, E2, E2l, a2, a2l, r02, r02l, m2, dm2);
    const R core = m1 + m2 + delta;
    const R dcore = dm1 + dm2;
    phi = core * ps;
    dphi = dcore * ps + core * dps;
    const R rs[3] = {rs1, rs2, rs3}, S[3] = {S1, S2, S3};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const R t = rs[k] - r;
      if (t >= R(0)) {
        const R t3 = t * t * t;
        phi -= S[k] * t3 * t;
        dphi += R(4) * S[k] * t3;
      }
    }
  }
  __device__ inline void embed(R x, R& xi, R& dxi) const {
    const R y = x - R(1), y2 = y * y, y3 = y2 * y;
    if (x <= R(1)) {
      const R y4 = y3 * y, y5 = y4 * y;
      xi = xi0 + R(0.5) * xi2 * y2 + q1 * y3 + q2 * y4 + q3 * y5 + q4 * y5 * y;
      dxi = xi2 * y + R(3) * q1 * y2 + R(4) * q2 * y3 + R(5) * q3 * y4 + R(6) * q4 * y5;
    } else {
      const R num = xi0 + R(0.5) * xi2 * y2 + q1 * y3 + Q1 * y3 * y;
      const R dnum = xi2 * y + R(3) * q1 * y2 + R(4) * Q1 * y3;
      const R den = R(1) + Q2 * y3, dden = R(3) * Q2 * y2;
      xi = num / den;
      dxi = (dnum * den - num * dden) / (den * den);
    }
    xi += F0;
  }
};

template <typename R>
PotSynth<R> make_synth(const ap_config& c) {
  PotSynth<R> s;
  s.p = make_params<R>(c);
  s.rc2 = s.p.rc2;
  return s;
}

// c.eam_mishin holds the 29 parameters in the order E1, E2, delta, F0, xi0, xi2, h,
// q1..q4, Q1, Q2, S1..S3, a, a1, a2, b1, b2, r01..r04, rs1..rs3, rc.
template <typename R>
PotMishin<R> make_mishin(const ap_config& c) {
  const double* m = c.eam_mishin;
  PotMishin<R> p;
  R* dst[29] = {&p.E1, &p.E2, &p.delta, &p.F0, &p.xi0, &p.xi2, &p.inv_h, &p.q1, &p.q2, &p.q3, &p.q4, &p.Q1, &p.Q2,
                &p.S1, &p.S2, &p.S3, &p.a, &p.a1, &p.a2, &p.b1, &p.b2, &p.r01, &p.r02, &p.r03, &p.r04, &p.rs1,
                &p.rs2, &p.rs3, &p.rc};
  for (int k = 0; k < 29; ++k) *dst[k] = (R)m[k];
  auto lo = [](double v) { return (R)(v - (double)(R)v); };
  p.E1l = lo(m[0]);
  p.E2l = lo(m[1]);
  p.a1l = lo(m[17]);
  p.a2l = lo(m[18]);
  p.r01l = lo(m[21]);
  p.r02l = lo(m[22]);
  p.inv_h = (R)(1.0 / m[6]);
  p.rc2 = (R)(m[28] * m[28]);
  return p;
}

}  // namespace ap
