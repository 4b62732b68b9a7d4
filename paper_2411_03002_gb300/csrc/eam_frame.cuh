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
// resident blocks per SM (register cap), and the FP32 reciprocal (1: approximate
// MUFU reciprocal, 0: correctly rounded).
#ifndef AP_EAM_LANES
#define AP_EAM_LANES 4
#endif
#ifndef AP_EAM_MINB
#define AP_EAM_MINB 6   // FP32 only: <= 42 registers, 48 resident warps per SM
#endif
#ifndef AP_EAM_FAST_RCP
#define AP_EAM_FAST_RCP 0
#endif

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

}  // namespace ap
