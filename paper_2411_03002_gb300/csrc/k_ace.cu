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
// Three kernels per evaluation, communicating through per-queue-position scratch:
//   k_ace_basis    one warp per precise atom (persistent CTAs, atomic work counter):
//                  row entries inside r_c compacted; G = g^T Y over 32-neighbour
//                  shared tiles; A = (1/N0) W . G; nu = 1, 2 energy and gradient;
//   k_ace_nu3      one lane per precise atom: the nu = 3 energy and gradient with A
//                  and dE/dA in registers, straight-line code over the merged
//                  monomials generated from the basis (ace_nu3.inc);
//   k_ace_adjoint  one warp per precise atom: u = W^T dE/dA / N0; lanes recompute g,
//                  g', Y, grad Y per in-range neighbour, contract with u, and scatter
//                  -w_i p_ij to neighbour j and +w_i sum p to i.
#include <complex>
#include <algorithm>
#include <cstring>
#include <cmath>

#include "ap_internal.cuh"

namespace ap {

// ------------------------------------------------------------------ device code
namespace {

constexpr int kCols = 36;            // 32 neighbour slots + 4 pad (16-byte rows, conflict-free)
constexpr int kRows = 33;            // 8 radial + 25 angular rows
// Tensor-core staging of one 32-neighbour batch (FP32 path), per k-step of 8 neighbours:
// the Y^T operand fragments [m-tile 2][lane 32][4] + 16 pad floats, and the g operand
// fragments [lane 32][2] + 8 pad floats.  The pads put the four k-steps of one store
// on different banks.
constexpr int kTyStep = 2 * 128 + 16;
constexpr int kTgStep = 64 + 8;
template <typename R>
constexpr int kTileWords = sizeof(R) == 4 ? 4 * kTyStep + 4 * kTgStep : kRows * kCols;
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

// Fixed-point force accumulation (ace_deterministic): contributions rounded to multiples
// of 2^-36 eV/A, summed with exact, order-independent 64-bit integer atomics.
constexpr double kFixScale = 68719476736.0;   // 2^36
__device__ inline unsigned long long to_fix(double v) { return (unsigned long long)llrint(v * kFixScale); }

template <typename R>
__device__ inline void add_force(float4* facc32, double* facc64, unsigned long long* fix, int j, R sx, R sy, R sz) {
  if (fix) {
    atomicAdd(&fix[3 * j + 0], to_fix((double)sx));
    atomicAdd(&fix[3 * j + 1], to_fix((double)sy));
    atomicAdd(&fix[3 * j + 2], to_fix((double)sz));
    return;
  }
  if constexpr (sizeof(R) == 4) {
    atomicAdd(&facc32[j], make_float4(sx, sy, sz, 0.f));
  } else {
    atomicAdd(&facc64[3 * j + 0], sx);
    atomicAdd(&facc64[3 * j + 1], sy);
    atomicAdd(&facc64[3 * j + 2], sz);
  }
}

// Block l of the force contraction for one neighbour: with S_m = sum_k u_k,lm g_k and
// S'_m = sum_k u_k,lm g'_k, accumulates pr += sum_m S'_m Z_m and the tangential part
// sum_m S_m (grad Z_m - l Z_m u) as (ptx, pty, ptz) += sum_m S_m grad Z_m and
// pz_l += l sum_m S_m Z_m (the caller subtracts pz_l u once).
template <typename R, int L>
__device__ inline void force_block(const R* __restrict__ U, R ux, R uy, R uz, const R g[8], const R dg[8], R& pr,
                                   R& ptx, R& pty, R& ptz, R& pzl) {
  R Y[2 * L + 1], gx[2 * L + 1], gy[2 * L + 1], gz[2 * L + 1];
  sh_block<R, L>(ux, uy, uz, Y, gx, gy, gz);
  R q = R(0);
#pragma unroll
  for (int m = 0; m < 2 * L + 1; ++m) {
    const int lm = L * L + m;
    auto ua = ld4<R>(&U[lm * 8]);
    auto ub = ld4<R>(&U[lm * 8 + 4]);
    R S = ua.x * g[0];
    S = fma(ua.y, g[1], S);
    S = fma(ua.z, g[2], S);
    S = fma(ua.w, g[3], S);
    S = fma(ub.x, g[4], S);
    S = fma(ub.y, g[5], S);
    S = fma(ub.z, g[6], S);
    S = fma(ub.w, g[7], S);
    R Sp = ua.x * dg[0];
    Sp = fma(ua.y, dg[1], Sp);
    Sp = fma(ua.z, dg[2], Sp);
    Sp = fma(ua.w, dg[3], Sp);
    Sp = fma(ub.x, dg[4], Sp);
    Sp = fma(ub.y, dg[5], Sp);
    Sp = fma(ub.z, dg[6], Sp);
    Sp = fma(ub.w, dg[7], Sp);
    pr = fma(Sp, Y[m], pr);
    if (L > 0) {
      q = fma(S, Y[m], q);
      ptx = fma(S, gx[m], ptx);
      pty = fma(S, gy[m], pty);
      ptz = fma(S, gz[m], ptz);
    }
  }
  if (L > 0) pzl = fma(R(L), q, pzl);
}

template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- 3xTF32 on warp-level tensor cores (FP32 path).  An FP32 value x is carried as
// hi + lo: hi = x rounded to the 10-bit TF32 significand (ties away from zero), lo =
// x - hi (exact in FP32); the tensor core reads the leading TF32 bits of lo.  A
// product of two such pairs drops lo * lo', which leaves about the error of an FP32
// product (relative 2^-21 per term).
__device__ inline void tf32_split(float x, uint32_t& h, uint32_t& l) {
  h = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
  l = __float_as_uint(x - __uint_as_float(h));
}

// D += A B on one m16n8k8 tile (A 16x8 row-major, B 8x8 column-major, TF32 inputs, FP32
// accumulation).  Fragments of lane (g = lane / 4, t = lane % 4):
//   a = A[g][t], A[g+8][t], A[g][t+4], A[g+8][t+4];  b = B[t][g], B[t+4][g];
//   d = D[g][2t], D[g][2t+1], D[g+8][2t], D[g+8][2t+1].
__device__ inline void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// D += (Ah + Al)(Bh + Bl) without Al Bl, the small products first.
__device__ inline void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], uint32_t bh0,
                            uint32_t bh1, uint32_t bl0, uint32_t bl1) {
  mma_tf32(d, al, bh0, bh1);
  mma_tf32(d, ah, bl0, bl1);
  mma_tf32(d, ah, bh0, bh1);
}

// out[lm][n] = sum_k in[lm][k] F[l(lm)][n][k] for the 25 (l, m) rows (two m-tiles, rows
// 25..31 zero) and an 8 x 8 factor per l (F in shared memory, F[(l * 8 + n) * 8 + k]).
// `in` is held as m16n8k8 accumulator fragments (rows lm = 16 mt + g, + 8; columns
// k = 2t, 2t + 1), and so is `out`: the accumulator feeds the next product directly,
// with the contraction index relabelled (operand column t <-> k = 2t, t + 4 <-> 2t + 1,
// and B's rows the same way).  Rows of one m-tile carry several l, so tile 0 takes one
// product per l = 0..3 and every lane keeps the rows of its own l; tile 1 is l = 4.
__device__ inline void lm_mix(const float (&in)[2][4], const float* __restrict__ F, int g, int t,
                              float (&out)[2][4]) {
  uint32_t ah[2][4], al[2][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    tf32_split(in[mt][0], ah[mt][0], al[mt][0]);
    tf32_split(in[mt][2], ah[mt][1], al[mt][1]);
    tf32_split(in[mt][1], ah[mt][2], al[mt][2]);
    tf32_split(in[mt][3], ah[mt][3], al[mt][3]);
  }
  const int l0 = g == 0 ? 0 : g < 4 ? 1 : 2;   // l of row g
  const int l1 = g == 0 ? 2 : 3;               // l of row g + 8
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    const float2 f = *reinterpret_cast<const float2*>(&F[l * 64 + g * 8 + 2 * t]);
    uint32_t bh0, bl0, bh1, bl1;
    tf32_split(f.x, bh0, bl0);
    tf32_split(f.y, bh1, bl1);
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    if (l < 4) {
      mma3(d, ah[0], al[0], bh0, bh1, bl0, bl1);
      if (l == l0) {
        out[0][0] = d[0];
        out[0][1] = d[1];
      }
      if (l == l1) {
        out[0][2] = d[2];
        out[0][3] = d[3];
      }
    } else {
      mma3(d, ah[1], al[1], bh0, bh1, bl0, bl1);
#pragma unroll
      for (int e = 0; e < 4; ++e) out[1][e] = d[e];
    }
  }
}

__device__ inline float pack_j(int j, float) { return __int_as_float(j); }
__device__ inline double pack_j(int j, double) { return __longlong_as_double((long long)j); }
__device__ inline int unpack_j(float v) { return __float_as_int(v); }
__device__ inline float4 make_r4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
__device__ inline double4_32a make_r4(double a, double b, double c, double d) { return make_double4_32a(a, b, c, d); }
__device__ inline int unpack_j(double v) { return (int)__double_as_longlong(v); }

constexpr int kListCap = 192;   // in-range records per precise atom cached in shared memory (FCC bulk: 134)
#ifndef AP_ACE3_WARPS
#define AP_ACE3_WARPS 6
#endif
#ifndef AP_ACE3_MINB
#define AP_ACE3_MINB 4
#endif
template <typename R>
constexpr int kWarps3 = sizeof(R) == 4 ? AP_ACE3_WARPS : 4;   // warps per CTA of the adjoint kernel

#include "ace_nu3.inc"

// Arguments of the three ACE kernels.  Scratch indexed by the queue position q
// carries the per-atom state from one kernel to the next.
template <typename R>
struct AceArgs {
  const int* queue;
  const int* count;        // queue length (device)
  DevScalars* stats;
  int* counter;
  int* counter2;
  const SysInfo* sys;
  const int* atom_sys;
  const typename V<R>::S4* sh;
  const int* nbr;
  const int* off;
  const int* cnt;
  int cap;
  const double* lam;
  const double* wgt;       // explicit weights w_i (NULL: w_i = 1 - lambda_i)
  const R* W;
  const R* M2;
  const R* C1;
  const R* M2b;      // phi^(2) tables of the Finnis-Sinclair form
  const R* C1b;
  R rc2, inv_rc, inv_n0;
  int mode;
  int fs_on;
  double fs_eps;
  double* e_prec;
  float4* facc32;
  double* facc64;
  unsigned long long* faccfix;   // fixed-point accumulator [n][3], or NULL (float atomics)
  typename V<R>::R4* list4;   // [q][rec] in-range (d, j) records in row order (kernel 1 -> 3)
  int rec;                    // record slots per queue position (>= every ACE row's length)
  int* nin;          // [q] their number
  R* a48;            // [q][48] A entries with n <= 2, l <= 3 (input of nu = 3)
  R* dA;             // [q][200] dE/dA of nu = 1, 2
  double* e12;       // [q] E of nu = 1, 2
  R* de3;            // [q][48] dE3/dA (Finnis-Sinclair form: of phi^(1) + F' phi^(2))
  double* e3;        // [q] E3 (of phi^(1))
  R* dAb;            // [q][200] dphi^(2)_12/dA                 (Finnis-Sinclair form only)
  double* e12b;      // [q] phi^(2)_12                          (Finnis-Sinclair form only)
  double* fs;        // [q][2] F(phi^(2)), F'(phi^(2))          (Finnis-Sinclair form only)
};

// nu = 3 coefficients, passed by value (kernel parameter space), in the order of kNu3Key.
template <typename R>
struct Nu3Coef {
  R c[AP_NU3_N];
};

// Kernel 1, one warp per precise atom (persistent CTAs, atomic work counter):
//   pass 0   row entries inside r_c compacted (displacement and j) into shared memory,
//            their row positions kept for kernel 3;
//   stage A  lanes evaluate g and Y for 32 neighbours into a shared tile, then
//            contract G = g^T Y; A = (1/N0) W . G;
//   nu = 1, 2: E12 and dE12/dA (symmetric 8x8 matrix-vector products per (l, m)).
// FP32: the three contractions run on the tensor cores (warp-level m16n8k8 TF32 MMAs
// with the 3xTF32 split, FP32 accumulation), G and A staying in accumulator fragments.
// FP64: SIMT loops, G with 4-wide vector loads along the neighbour axis.
template <typename R>
__global__ void __launch_bounds__(kWarps<R> * 32, sizeof(R) == 4 ? AP_ACE_MINB : 1) k_ace_basis(AceArgs<R> a) {
  // Shared memory: W [320] | M2 [320] | C1 [8] | M2b [320] | C1b [8] | per warp: list
  // [kListCap][4] | tile [kTileWords] (FP32: operand fragments of one batch; FP64: the
  // g/Y tile [kRows][kCols], which A and the G scratch alias after stage A).
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R* Ws = reinterpret_cast<R*>(smem_raw);
  R* M2 = Ws + 320;
  R* C1 = M2 + 320;
  R* M2b = C1 + 8;
  R* C1b = M2b + 320;
  R* wbase = C1b + 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R* list = wbase + warp * (4 * kListCap + kTileWords<R>);
  R* tile = list + 4 * kListCap;
  for (int t = threadIdx.x; t < 320; t += blockDim.x) {
    Ws[t] = a.W[t];
    M2[t] = a.M2[t];
    M2b[t] = a.M2b[t];
  }
  if (threadIdx.x < 8) {
    C1[threadIdx.x] = a.C1[threadIdx.x];
    C1b[threadIdx.x] = a.C1b[threadIdx.x];
  }
  __syncthreads();
  const int m = *a.count;
  const int kq = lane & 7, grp = lane >> 3;
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned long long cnt_pairs = 0, cnt_atoms = 0, cnt_mma = 0;   // profiling counts of this warp
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

    // ---------------- pass 0: compact the row entries inside ace_rc.  The dependent loads
    // (row entry, then its shadow) run ahead of their use: the entry two batches ahead,
    // the shadow one batch ahead.
    int nin = 0;
    int j_a = lane < c ? a.nbr[row + lane] : 0;
    auto s_a = lane < c ? a.sh[j_a] : si;
    int j_b = lane + 32 < c ? a.nbr[row + lane + 32] : 0;
    for (int base = 0; base < c; base += 32) {
      const int slot = base + lane;
      const int j = j_a;
      const auto sj = s_a;
      j_a = j_b;
      if (slot + 32 < c) s_a = a.sh[j_a];
      j_b = slot + 64 < c ? a.nbr[row + slot + 64] : 0;
      bool in = false;
      R d[3] = {R(0), R(0), R(0)};
      if (slot < c) {
        pair_disp<R>(S, si, sj, a.off, row + slot, d);
        in = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < a.rc2;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, in);
      const int pos = nin + __popc(mask & lt_mask);   // < c <= rec
      if (in) {
        const auto rec = make_r4(d[0], d[1], d[2], pack_j(j, R(0)));
        a.list4[(size_t)q * a.rec + pos] = rec;
        if (pos < kListCap) *reinterpret_cast<typename V<R>::R4*>(&list[4 * pos]) = rec;
      }
      nin += __popc(mask);
    }
    if (lane == 0) a.nin[q] = nin;
    __syncwarp();   // also orders this warp's record stores before the reads of stage A

    // ---------------- stage A: G_klm = sum_j g_k Y_lm over the compacted neighbours,
    // then A = (1/N0) W . G and nu = 1, 2: E12 and dE12/dA
    R e = R(0);
    if constexpr (sizeof(R) == 4) {
      // Tensor cores, 3xTF32: per k-step of 8 neighbours, D[lm][k] += Y^T[lm][j] g[j][k]
      // for two m-tiles of 16 (l, m) rows.  Each lane evaluates g and Y of one neighbour
      // and stores them as operand fragments; the accumulators end as G in fragment form.
      const int g8 = lane >> 2, t4 = lane & 3;
      float* ty = tile;
      float* tg = tile + 4 * kTyStep;
      float acc[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[mt][u] = 0.f;
      // this lane's neighbour slot c of k-step ks: Y pairs (rows r, r + 8) go to the
      // fragment of lane (r % 8) * 4 + c % 4, elements 2 (c / 4) and 2 (c / 4) + 1; g_k
      // to lane k * 4 + c % 4, element c / 4
      const int pks = lane >> 3, pc = lane & 7;
      float* yb = ty + pks * kTyStep + (pc & 3) * 4 + (pc >> 2) * 2;
      float* gb = tg + pks * kTgStep + (pc & 3) * 2 + (pc >> 2);
      for (int base = 0; base < nin; base += 32) {
        const int slot = base + lane;
        float g[8], Y[25];
        if (slot < nin) {
          const auto en = slot < kListCap ? ld4<R>(&list[4 * slot]) : a.list4[(size_t)q * a.rec + slot];
          float r2 = en.x * en.x + en.y * en.y + en.z * en.z;
          float ir = rsqrt_(r2);
          radial<float, false>(r2 * ir, a.inv_rc, a.mode, g, nullptr);
          sh_values<float>(en.x * ir, en.y * ir, en.z * ir, Y);
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) g[k] = 0.f;
#pragma unroll
          for (int k = 0; k < 25; ++k) Y[k] = 0.f;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          *reinterpret_cast<float2*>(yb + r * 16) = make_float2(Y[r], Y[r + 8]);
          *reinterpret_cast<float2*>(yb + 128 + r * 16) = make_float2(Y[16 + r], r == 0 ? Y[24] : 0.f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) gb[k * 8] = g[k];
        __syncwarp();
        const int nks = (min(32, nin - base) + 7) >> 3;
        for (int ks = 0; ks < nks; ++ks) {
          const float4 y0 = *reinterpret_cast<const float4*>(ty + ks * kTyStep + lane * 4);
          const float4 y1 = *reinterpret_cast<const float4*>(ty + ks * kTyStep + 128 + lane * 4);
          const float2 gg = *reinterpret_cast<const float2*>(tg + ks * kTgStep + lane * 2);
          uint32_t yh0[4], yl0[4], yh1[4], yl1[4], gh0, gl0, gh1, gl1;
          tf32_split(y0.x, yh0[0], yl0[0]);
          tf32_split(y0.y, yh0[1], yl0[1]);
          tf32_split(y0.z, yh0[2], yl0[2]);
          tf32_split(y0.w, yh0[3], yl0[3]);
          tf32_split(y1.x, yh1[0], yl1[0]);
          tf32_split(y1.y, yh1[1], yl1[1]);
          tf32_split(y1.z, yh1[2], yl1[2]);
          tf32_split(y1.w, yh1[3], yl1[3]);
          tf32_split(gg.x, gh0, gl0);
          tf32_split(gg.y, gh1, gl1);
          // each k-step's products from zero, summed into acc with round-to-nearest FP32
          // adds: the tensor core's own accumulation does not round to nearest, and 48
          // chained MMAs would bias G
          float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
          mma3(d0, yh0, yl0, gh0, gh1, gl0, gl1);
          mma3(d1, yh1, yl1, gh0, gh1, gl0, gl1);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            acc[0][u] += d0[u];
            acc[1][u] += d1[u];
          }
        }
        __syncwarp();
      }
      // acc = G^T as fragments (rows lm, columns k); A = W G, then S = M2 A per l
      float am[2][4], sm[2][4];
      lm_mix(acc, Ws, g8, t4, am);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int u = 0; u < 4; ++u) am[mt][u] *= a.inv_n0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {   // the nu = 3 inputs: n <= 2, lm < 16 (tile 0)
        const int lm = g8 + 8 * (u >> 1), n = 2 * t4 + (u & 1);
        if (n < 3) a.a48[(size_t)q * 48 + n * 16 + lm] = am[0][u];
      }
      lm_mix(am, M2, g8, t4, sm);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int lm = 16 * mt + g8 + 8 * (u >> 1), n = 2 * t4 + (u & 1);
          if (lm < 25) {
            const float lin = lm == 0 ? C1[n] : 0.f;
            e += am[mt][u] * (0.5f * sm[mt][u] + lin);
            a.dA[(size_t)q * 200 + n * 25 + lm] = sm[mt][u] + lin;
          }
        }
      if (a.fs_on) {   // the same products with the phi^(2) coefficients
        lm_mix(am, M2b, g8, t4, sm);
        float eb = 0.f;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int lm = 16 * mt + g8 + 8 * (u >> 1), n = 2 * t4 + (u & 1);
            if (lm < 25) {
              const float lin = lm == 0 ? C1b[n] : 0.f;
              eb += am[mt][u] * (0.5f * sm[mt][u] + lin);
              a.dAb[(size_t)q * 200 + n * 25 + lm] = sm[mt][u] + lin;
            }
          }
        const double Eb = warp_sum<double>((double)eb);
        if (lane == 0) a.e12b[q] = Eb;
      }
    } else {
      // FP64: SIMT, G = g^T Y with 4-wide vector loads along the neighbour axis
      R* A = tile;
      R* Gs = tile + 600;
      R acc[7];
#pragma unroll
      for (int t = 0; t < 7; ++t) acc[t] = R(0);
      for (int base = 0; base < nin; base += 32) {
        const int slot = base + lane;
        R g[8], Y[25];
        if (slot < nin) {
          const auto en = slot < kListCap ? ld4<R>(&list[4 * slot]) : a.list4[(size_t)q * a.rec + slot];
          R r2 = en.x * en.x + en.y * en.y + en.z * en.z;
          R ir = rsqrt_(r2);
          radial<R, false>(r2 * ir, a.inv_rc, a.mode, g, nullptr);
          sh_values<R>(en.x * ir, en.y * ir, en.z * ir, Y);
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
      }
      __syncwarp();
      for (int v = lane; v < 48; v += 32) a.a48[(size_t)q * 48 + v] = A[(v >> 4) * 25 + (v & 15)];
      for (int o = lane; o < 200; o += 32) {
        const int n = o / 25, lm = o - 25 * n, l = l_of(lm);
        const R* mrow = &M2[l * 64 + n * 8];
        R s = R(0);
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) s += mrow[n2] * A[n2 * 25 + lm];
        const R lin = lm == 0 ? C1[n] : R(0);
        e += A[o] * (R(0.5) * s + lin);
        a.dA[(size_t)q * 200 + o] = s + lin;
      }
      if (a.fs_on) {   // the same products with the phi^(2) coefficients
        R eb = R(0);
        for (int o = lane; o < 200; o += 32) {
          const int n = o / 25, lm = o - 25 * n, l = l_of(lm);
          const R* mrow = &M2b[l * 64 + n * 8];
          R sb = R(0);
#pragma unroll
          for (int n2 = 0; n2 < 8; ++n2) sb += mrow[n2] * A[n2 * 25 + lm];
          const R lin = lm == 0 ? C1b[n] : R(0);
          eb += A[o] * (R(0.5) * sb + lin);
          a.dAb[(size_t)q * 200 + o] = sb + lin;
        }
        const double Eb = warp_sum<double>((double)eb);
        if (lane == 0) a.e12b[q] = Eb;
      }
    }
    const double E = warp_sum<double>((double)e);
    if (lane == 0) a.e12[q] = E;
    cnt_pairs += nin;
    cnt_atoms += 1;
    // tensor-core tiles: 6 per k-step of 8 neighbours, 15 per lm_mix
    if (sizeof(R) == 4) cnt_mma += 6 * ((nin + 7) / 8) + (a.fs_on ? 45 : 30);
    __syncwarp();
  }
  if (lane == 0 && cnt_atoms > 0) {   // the warp's counts, added once
    atomicAdd(&a.stats->ace_pairs, cnt_pairs);
    atomicAdd(&a.stats->ace_atoms, cnt_atoms);
    if (sizeof(R) == 4) atomicAdd(&a.stats->ace_mma, cnt_mma);
  }
}

// Kernel 2, one lane per precise atom: nu = 3 energy and gradient with the 48 A
// entries and their gradient in registers, as straight-line code over the merged
// monomials (ace_nu3.inc); coefficients are read from the parameter space.  E3
// follows from Euler's identity for a homogeneous cubic, E3 = (1/3) sum A dE3/dA.
// Finnis-Sinclair form (FS): a first pass gives the nu = 3 part of phi^(2), hence
// phi^(2), F and F'; the gradient pass then uses the coefficients c1 + F' c2, and
// E3 of phi^(1) is E3(c1 + F' c2) - F' E3(c2).
#ifndef AP_NU3_MINB
#define AP_NU3_MINB 0   // FP32: resident 128-thread blocks per SM the nu = 3 kernel is compiled for (0: no bound)
#endif
#if AP_NU3_MINB > 0
#define AP_NU3_BOUNDS __launch_bounds__(sizeof(R) == 4 ? 128 : 64, sizeof(R) == 4 ? AP_NU3_MINB : 1)
#else
#define AP_NU3_BOUNDS __launch_bounds__(sizeof(R) == 4 ? 128 : 64)
#endif
#ifndef AP_NU3_VEC
#define AP_NU3_VEC 1    // 4-wide loads of A and stores of dE3/dA
#endif
template <typename R, bool FS>
__global__ void AP_NU3_BOUNDS k_ace_nu3(AceArgs<R> a, const Nu3Coef<R> P,
                                                                       const Nu3Coef<R> Q) {
  const int m = *a.count;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
    R A[48], dA[48];
#if AP_NU3_VEC
    // 4-wide loads (the rows of a48 are 48 entries, a multiple of 4)
    const auto* src = reinterpret_cast<const typename V<R>::R4*>(a.a48 + (size_t)q * 48);
#pragma unroll
    for (int v = 0; v < 12; ++v) {
      const auto t = src[v];
      A[4 * v] = t.x;
      A[4 * v + 1] = t.y;
      A[4 * v + 2] = t.z;
      A[4 * v + 3] = t.w;
    }
#else
    const R* src = a.a48 + (size_t)q * 48;
#pragma unroll
    for (int v = 0; v < 48; ++v) A[v] = src[v];
#endif
#pragma unroll
    for (int v = 0; v < 48; ++v) dA[v] = R(0);
    R fp = R(0);
    double e3b = 0.0, Fv = 0.0;
    if constexpr (FS) {
      R eb = R(0);
#define NU3_GROUP_BEGIN(x, y) \
  {                           \
    const R p_ = A[x] * A[y]; \
    R s_ = R(0);
#define NU3_TERM(t, z) s_ = fma(Q.c[t], A[z], s_);
#define NU3_GROUP_END(x, y) \
  eb = fma(p_, s_, eb);     \
  }
      AP_NU3_BODY
#undef NU3_GROUP_BEGIN
#undef NU3_TERM
#undef NU3_GROUP_END
      e3b = (double)eb;
      const double phi2 = a.e12b[q] + e3b;
      const double sq = sqrt(fabs(phi2) + a.fs_eps * a.fs_eps);
      Fv = phi2 > 0.0 ? sq - a.fs_eps : (phi2 < 0.0 ? a.fs_eps - sq : 0.0);
      fp = (R)(0.5 / sq);
    }
#define NU3_GROUP_BEGIN(x, y) \
  {                           \
    const R p_ = A[x] * A[y]; \
    R s_ = R(0);
#define NU3_COEF(t) (FS ? fma(fp, Q.c[t], P.c[t]) : P.c[t])
#define NU3_TERM(t, z)             \
  s_ = fma(NU3_COEF(t), A[z], s_); \
  dA[z] = fma(NU3_COEF(t), p_, dA[z]);
#define NU3_GROUP_END(x, y)     \
  dA[x] = fma(s_, A[y], dA[x]); \
  dA[y] = fma(s_, A[x], dA[y]); \
  }
    AP_NU3_BODY
#undef NU3_GROUP_BEGIN
#undef NU3_COEF
#undef NU3_TERM
#undef NU3_GROUP_END
    R e = R(0);
#pragma unroll
    for (int v = 0; v < 48; ++v) e = fma(A[v], dA[v], e);
#if AP_NU3_VEC
    auto* dst = reinterpret_cast<typename V<R>::R4*>(a.de3 + (size_t)q * 48);
#pragma unroll
    for (int v = 0; v < 12; ++v) dst[v] = make_r4(dA[4 * v], dA[4 * v + 1], dA[4 * v + 2], dA[4 * v + 3]);
#else
    R* dst = a.de3 + (size_t)q * 48;
#pragma unroll
    for (int v = 0; v < 48; ++v) dst[v] = dA[v];
#endif
    a.e3[q] = (double)e * (1.0 / 3.0) - (FS ? (double)fp * e3b : 0.0);
    if (FS) {
      a.fs[2 * (size_t)q] = Fv;
      a.fs[2 * (size_t)q + 1] = (double)fp;
    }
  }
}

// Kernel 3, one warp per precise atom (persistent): E_i = E12 + E3 -> e_prec, then
// u_klm = (1/N0) sum_n W[l][n][k] dE/dA_nlm and the forces: lanes recompute g, g',
// Y, grad Y per in-range neighbour (from the kept row positions), contract with u
// and scatter -w_i p_ij to neighbour j, +w_i sum_j p_ij to i.
template <typename R, bool FORCES, bool FS>
__global__ void __launch_bounds__(kWarps3<R> * 32, sizeof(R) == 4 ? AP_ACE3_MINB : 1) k_ace_adjoint(AceArgs<R> a) {
  // Shared memory: W [320] | per warp: dA [200] | U [200]
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R* Ws = reinterpret_cast<R*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R* dA = Ws + 320 + warp * 400;
  R* U = dA + 200;
  for (int t = threadIdx.x; t < 320; t += blockDim.x) Ws[t] = a.W[t];
  __syncthreads();
  const int m = *a.count;
  while (true) {
    int q = 0;
    if (lane == 0) q = atomicAdd(a.counter2, 1);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= m) break;
    const int i = a.queue[q];
    if (lane == 0) a.e_prec[i] = a.e12[q] + a.e3[q] + (FS ? a.fs[2 * (size_t)q] : 0.0);
    if (!FORCES) continue;
    if (FS) {
      const R fp = (R)a.fs[2 * (size_t)q + 1];
      for (int o = lane; o < 200; o += 32) dA[o] = fma(fp, a.dAb[(size_t)q * 200 + o], a.dA[(size_t)q * 200 + o]);
    } else {
      for (int o = lane; o < 200; o += 32) dA[o] = a.dA[(size_t)q * 200 + o];
    }
    __syncwarp();
    for (int v = lane; v < 48; v += 32) dA[(v >> 4) * 25 + (v & 15)] += a.de3[(size_t)q * 48 + v];
    __syncwarp();
    for (int o = lane; o < 200; o += 32) {
      const int lm = o >> 3, k = o & 7, l = l_of(lm);
      R s = R(0);
#pragma unroll
      for (int n = 0; n < 8; ++n) s += Ws[(l * 8 + n) * 8 + k] * dA[n * 25 + lm];
      U[o] = s * a.inv_n0;
    }
    __syncwarp();
    const int nin = a.nin[q];
    const R wgt = (R)(a.wgt ? a.wgt[i] : 1.0 - (a.lam ? a.lam[i] : 0.0));
    R pix = R(0), piy = R(0), piz = R(0);
    // the pair records kernel 1 kept (displacement and j, coalesced), the lane's next
    // one loaded an iteration ahead
    const typename V<R>::R4* lst = a.list4 + (size_t)q * a.rec;
    typename V<R>::R4 e_n = make_r4(R(0), R(0), R(0), R(0));
    if (lane < nin) e_n = lst[lane];
    for (int base = 0; base < nin; base += 32) {
      const int slot = base + lane;
      const auto e = e_n;
      if (slot + 32 < nin) e_n = lst[slot + 32];
      if (slot >= nin) continue;
      const int j = unpack_j(e.w);
      const R d[3] = {e.x, e.y, e.z};
      R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      R ir = rsqrt_(r2);
      R ux = d[0] * ir, uy = d[1] * ir, uz = d[2] * ir;
      R g[8], dg[8];
      radial<R, true>(r2 * ir, a.inv_rc, a.mode, g, dg);
      R pr = R(0), ptx = R(0), pty = R(0), ptz = R(0), pzl = R(0);
      force_block<R, 0>(U, ux, uy, uz, g, dg, pr, ptx, pty, ptz, pzl);
      force_block<R, 1>(U, ux, uy, uz, g, dg, pr, ptx, pty, ptz, pzl);
      force_block<R, 2>(U, ux, uy, uz, g, dg, pr, ptx, pty, ptz, pzl);
      force_block<R, 3>(U, ux, uy, uz, g, dg, pr, ptx, pty, ptz, pzl);
      force_block<R, 4>(U, ux, uy, uz, g, dg, pr, ptx, pty, ptz, pzl);
      ptx = fma(-pzl, ux, ptx);
      pty = fma(-pzl, uy, pty);
      ptz = fma(-pzl, uz, ptz);
      R px = pr * ux + ptx * ir, py = pr * uy + pty * ir, pz = pr * uz + ptz * ir;
      pix += px;
      piy += py;
      piz += pz;
      add_force<R>(a.facc32, a.facc64, a.faccfix, j, -wgt * px, -wgt * py, -wgt * pz);
    }
    pix = warp_sum<R>(pix);
    piy = warp_sum<R>(piy);
    piz = warp_sum<R>(piz);
    if (lane == 0) add_force<R>(a.facc32, a.facc64, a.faccfix, i, wgt * pix, wgt * piy, wgt * piz);
    __syncwarp();
  }
}

__global__ void k_ace_finalize32(int n, const float4* __restrict__ acc, double* __restrict__ f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 v = acc[i];
  if (v.x == 0.f && v.y == 0.f && v.z == 0.f) return;   // no precise atom in reach (most atoms)
  f[3 * i + 0] += (double)v.x;
  f[3 * i + 1] += (double)v.y;
  f[3 * i + 2] += (double)v.z;
}

__global__ void k_ace_finalize_fix(int n, const unsigned long long* __restrict__ acc, double* __restrict__ f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  const long long v = (long long)acc[i];
  if (v != 0) f[i] += (double)v * (1.0 / kFixScale);
}

__global__ void k_ace_finalize64(int n, const double* __restrict__ acc, double* __restrict__ f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  f[i] += acc[i];
}

template <typename R>
size_t basis_smem() {
  return sizeof(R) * (320 + 320 + 8 + 320 + 8) + sizeof(R) * kWarps<R> * (4 * kListCap + kTileWords<R>);
}

template <typename R>
size_t adjoint_smem() {
  return sizeof(R) * (320 + kWarps3<R> * 400);
}

template <typename K>
int resident_blocks(K kern, int threads, size_t smem) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem);
  return b > 0 ? b : 1;
}

template <typename R>
void run_ace(ap_ctx* c, const double* d_lam, const double* d_wgt, const int* d_queue, const int* d_count,
             double* d_e_prec, bool forces, cudaStream_t s) {
  AceArgs<R> a;
  a.queue = d_queue;
  a.count = d_count ? d_count : &c->d_sc->n_precise;
  a.stats = c->d_sc;
  a.counter = &c->d_sc->work_counter;
  a.counter2 = &c->d_sc->work_counter2;
  a.sys = c->d_sys;
  a.atom_sys = c->d_atom_sys;
  if constexpr (sizeof(R) == 4) {
    a.sh = c->d_sh32;
    a.W = c->d_W32;
    a.facc32 = c->d_facc32;
    a.facc64 = nullptr;
  } else {
    a.sh = c->d_sh64;
    a.W = c->d_W64;
    a.facc32 = nullptr;
    a.facc64 = c->d_facc64;
  }
  a.nbr = c->d_nbr_ace;
  a.off = c->stored_off ? c->d_off_ace : nullptr;
  a.cnt = c->d_cnt_ace;
  a.cap = c->cap_ace;
  a.lam = d_lam;
  a.wgt = d_wgt;
  a.faccfix = c->cfg.ace_deterministic ? c->d_faccfix : nullptr;
  a.M2 = a.W + 320;   // the parameter block is [W (320) | M2 (320) | C1 (8) | M2b (320) | C1b (8)]
  a.C1 = a.W + 640;
  a.M2b = a.W + 648;
  a.C1b = a.W + 968;
  a.fs_on = c->cfg.ace_fs_on;
  a.fs_eps = c->cfg.ace_fs_eps;
  a.dAb = reinterpret_cast<R*>(c->d_ace_dAb);
  a.e12b = c->d_ace_e12b;
  a.fs = c->d_ace_fs;
  a.rc2 = (R)(c->cfg.ace_rc * c->cfg.ace_rc);
  a.inv_rc = (R)(1.0 / c->cfg.ace_rc);
  a.inv_n0 = (R)(1.0 / c->cfg.ace_n0);
  a.mode = c->cfg.fcut_mode;
  a.e_prec = d_e_prec;
  a.list4 = reinterpret_cast<typename V<R>::R4*>(c->d_ace_list);
  a.rec = c->ace_rec_cap;
  a.nin = c->d_ace_nin;
  a.a48 = reinterpret_cast<R*>(c->d_ace_a48);
  a.dA = reinterpret_cast<R*>(c->d_ace_dA);
  a.e12 = c->d_ace_e12;
  a.de3 = reinterpret_cast<R*>(c->d_ace_de3);
  a.e3 = c->d_ace_e3;
  static Nu3Coef<R> P, Q;
  for (int t = 0; t < AP_NU3_N; ++t) {
    P.c[t] = (R)c->ace.nu3_coef[t];
    Q.c[t] = (R)c->ace.nu3_coef2[t];
  }
  const bool fs = c->cfg.ace_fs_on != 0;

  const int pi = sizeof(R) == 4 ? 0 : 1;
  static int b1[2] = {0, 0}, b3[2][2][2] = {};
  const size_t s1 = basis_smem<R>(), s3 = adjoint_smem<R>();
  if (!b1[pi]) b1[pi] = resident_blocks(k_ace_basis<R>, kWarps<R> * 32, s1);
  auto k3 = forces ? (fs ? k_ace_adjoint<R, true, true> : k_ace_adjoint<R, true, false>)
                   : (fs ? k_ace_adjoint<R, false, true> : k_ace_adjoint<R, false, false>);
  if (!b3[pi][forces][fs]) b3[pi][forces][fs] = resident_blocks(k3, kWarps3<R> * 32, s3);
  if (forces) {
    if (a.faccfix)
      cudaMemsetAsync(c->d_faccfix, 0, sizeof(unsigned long long) * 3 * (size_t)c->n, s);
    else if constexpr (sizeof(R) == 4)
      cudaMemsetAsync(c->d_facc32, 0, sizeof(float4) * (size_t)c->n, s);
    else
      cudaMemsetAsync(c->d_facc64, 0, sizeof(double) * 3 * (size_t)c->n, s);
  }
  cudaMemsetAsync(a.counter, 0, 2 * sizeof(int), s);   // work_counter and work_counter2
  const int tb = prof_mark(c, s);
  k_ace_basis<R><<<c->num_sms * b1[pi], kWarps<R> * 32, s1, s>>>(a);
  prof_add(c, AP_PHASE_ACE_BASIS, tb, prof_mark(c, s));
  const int t2 = sizeof(R) == 4 ? 128 : 64;
  if (fs)
    k_ace_nu3<R, true><<<c->num_sms * (sizeof(R) == 4 ? 8 : 16), t2, 0, s>>>(a, P, Q);
  else
    k_ace_nu3<R, false><<<c->num_sms * (sizeof(R) == 4 ? 8 : 16), t2, 0, s>>>(a, P, Q);
  const int t0 = prof_mark(c, s);
  k3<<<c->num_sms * b3[pi][forces][fs], kWarps3<R> * 32, s3, s>>>(a);
  prof_add(c, AP_PHASE_ACE_ADJOINT, t0, prof_mark(c, s));
  c->kernels += 3;
}

}  // namespace

// The compiled nu = 3 code must match the host enumeration of the basis.
bool ace_nu3_matches(const AceTables& t) {
  if (t.nu3_key.size() != (size_t)AP_NU3_N) return false;
  for (int k = 0; k < AP_NU3_N; ++k)
    if (t.nu3_key[k] != kNu3Key[k]) return false;
  return true;
}

void upload_ace_tables(ap_ctx* c) {
  const AceTables& t = c->ace;
  std::vector<double> p64(c->cfg.ace_W, c->cfg.ace_W + 320);
  p64.insert(p64.end(), t.m2.begin(), t.m2.end());
  p64.insert(p64.end(), t.c1.begin(), t.c1.end());
  p64.insert(p64.end(), t.m2b.begin(), t.m2b.end());
  p64.insert(p64.end(), t.c1b.begin(), t.c1b.end());
  std::vector<float> p32(p64.begin(), p64.end());
  cudaMalloc(&c->d_W32, sizeof(float) * p32.size());
  cudaMalloc(&c->d_W64, sizeof(double) * p64.size());
  cudaMemcpy(c->d_W32, p32.data(), sizeof(float) * p32.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_W64, p64.data(), sizeof(double) * p64.size(), cudaMemcpyHostToDevice);
}

void launch_ace(ap_ctx* c, const double* d_lam, const int* d_queue, double* d_e_prec, bool forces, cudaStream_t s,
                const double* d_wgt, const int* d_count) {
  if (c->cfg.precision == AP_PREC_FP64)
    run_ace<double>(c, d_lam, d_wgt, d_queue, d_count, d_e_prec, forces, s);
  else
    run_ace<float>(c, d_lam, d_wgt, d_queue, d_count, d_e_prec, forces, s);
}

void launch_ace_finalize(ap_ctx* c, double* d_f, cudaStream_t s) {
  c->kernels += 1;
  if (c->cfg.ace_deterministic)
    k_ace_finalize_fix<<<(int)((3 * c->n + 255) / 256), 256, 0, s>>>((int)c->n, c->d_faccfix, d_f);
  else if (c->cfg.precision == AP_PREC_FP64)
    k_ace_finalize64<<<(int)((3 * c->n + 255) / 256), 256, 0, s>>>((int)c->n, c->d_facc64, d_f);
  else
    k_ace_finalize32<<<(int)((c->n + 255) / 256), 256, 0, s>>>((int)c->n, c->d_facc32, d_f);
}

}  // namespace ap
