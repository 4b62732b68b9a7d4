// EAM site energies (Eq. energy_eam) and the lambda-weighted force of Eq. F_i_d at
// fixed lambda.  Two passes over the neighbour rows, G lanes per atom with
// shuffle reductions:
//   density: rho_i = sum_j zeta(r_ij); q_i = (lambda_i xi'(rho_i), lambda_i)
//   force:   F_i = sum_j g_ij (x_j - x_i)/r_ij with
//            g_ij = (lambda_i xi'_i + lambda_j xi'_j) zeta'(r_ij) + (lambda_i + lambda_j)/2 Phi'(r_ij),
//            which is -grad_i sum_k lambda_k E_k^(f) gathered without atomics;
//            E_i^(f) = xi_i + 1/2 sum_j Phi(r_ij).
// Analytic forms: zeta(r) = exp(-beta (r/r0 - 1)) psi, Phi(r) = D (e^{-2a(r-rp)} -
// 2 e^{-a(r-rp)}) psi, xi(rho) = -A sqrt(rho), psi = u^4/(1+u^4), u = (r - rc)/h < 0.
#include "ap_internal.cuh"

namespace ap {

namespace {

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

__device__ inline const SysInfo& sys_of(const SysInfo* sys, const int* atom_sys, int i) {
  return sys[atom_sys ? atom_sys[i] : 0];
}

template <typename R, typename S4>
__device__ inline void pair_disp(const SysInfo& S, const S4& si, const S4& sj, const int* off, size_t e, R d[3]) {
  int k0, k1, k2;
  if (off) {
    int p = off[e];
    k0 = off_x(p);
    k1 = off_y(p);
    k2 = off_z(p);
  } else {
    int wi = Shadow<R>::code(si), wj = Shadow<R>::code(sj);
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

// psi(u) = u^4/(1+u^4) and dpsi/du, for u < 0
template <typename R>
__device__ inline void psi_fn(R u, R& ps, R& dps) {
  R u2 = u * u;
  R u4 = u2 * u2;
  R inv = R(1) / (R(1) + u4);
  ps = u4 * inv;
  dps = R(4) * u2 * u * inv * inv;
}

template <typename T, int G>
__device__ inline T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

template <typename R, int G>
__global__ void __launch_bounds__(256) k_eam_density(int n, const SysInfo* __restrict__ sys,
                                                     const int* __restrict__ atom_sys,
                                                     const typename Shadow<R>::T* __restrict__ sh,
                                                     const int* __restrict__ nbr, const int* __restrict__ off,
                                                     const int* __restrict__ cnt, int cap, EamP<R> p,
                                                     const double* __restrict__ lam,
                                                     typename Q2<R>::T* __restrict__ q, double* __restrict__ xi_out) {
  const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int sub = threadIdx.x & (G - 1);
  const bool active = gid < n;
  const int i = active ? gid : n - 1;
  const SysInfo& S = sys_of(sys, atom_sys, i);
  const auto si = sh[i];
  const int c = active ? cnt[i] : 0;
  const size_t row = (size_t)i * cap;
  R rho = R(0);
  for (int t = sub; t < c; t += G) {
    int j = nbr[row + t];
    auto sj = sh[j];
    R d[3];
    pair_disp<R>(S, si, sj, off, row + t, d);
    R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 < p.rc2) {
      R r = r2 * rsqrt_(r2);
      R ps, dps;
      psi_fn<R>((r - p.rc) * p.inv_h, ps, dps);
      rho += rexp(p.beta - p.beta_r0 * r) * ps;
    }
  }
  double rho_d = group_sum<double, G>((double)rho);
  if (active && sub == 0) {
    double li = lam ? lam[i] : 1.0;
    double xi = 0.0, dxi = 0.0;
    if (rho_d > 0.0) {
      double s = sqrt(rho_d);
      xi = -(double)p.A * s;
      dxi = -(double)p.A / (2.0 * s);
    }
    q[i] = Q2<R>::make((R)(li * dxi), (R)li);
    xi_out[i] = xi;
  }
}

template <typename R, int G>
__global__ void __launch_bounds__(256) k_eam_force(int n, const SysInfo* __restrict__ sys,
                                                   const int* __restrict__ atom_sys,
                                                   const typename Shadow<R>::T* __restrict__ sh,
                                                   const int* __restrict__ nbr, const int* __restrict__ off,
                                                   const int* __restrict__ cnt, int cap, EamP<R> p,
                                                   const typename Q2<R>::T* __restrict__ q,
                                                   const double* __restrict__ xi, double* __restrict__ e_fast,
                                                   double* __restrict__ f, int accumulate) {
  const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int sub = threadIdx.x & (G - 1);
  const bool active = gid < n;
  const int i = active ? gid : n - 1;
  const SysInfo& S = sys_of(sys, atom_sys, i);
  const auto si = sh[i];
  const auto qi = q[i];
  const int c = active ? cnt[i] : 0;
  const size_t row = (size_t)i * cap;
  R fx = R(0), fy = R(0), fz = R(0), phi = R(0);
  for (int t = sub; t < c; t += G) {
    int j = nbr[row + t];
    auto sj = sh[j];
    R d[3];
    pair_disp<R>(S, si, sj, off, row + t, d);
    R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 < p.rc2) {
      auto qj = q[j];
      R inv_r = rsqrt_(r2);
      R r = r2 * inv_r;
      R ps, dps;
      psi_fn<R>((r - p.rc) * p.inv_h, ps, dps);
      dps *= p.inv_h;
      R ez = rexp(p.beta - p.beta_r0 * r);
      R dzeta = ez * (dps - p.beta_r0 * ps);
      R e1 = rexp(-p.alpha * (r - p.rp));
      R e2 = e1 * e1;
      R m = p.D * (e2 - R(2) * e1);
      R dm = R(2) * p.alpha * p.D * (e1 - e2);
      R dphi = dm * ps + m * dps;
      phi += m * ps;
      R g = (qi.x + qj.x) * dzeta + R(0.5) * (qi.y + qj.y) * dphi;
      R s = g * inv_r;
      fx += s * d[0];
      fy += s * d[1];
      fz += s * d[2];
    }
  }
  double Fx = group_sum<double, G>((double)fx);
  double Fy = group_sum<double, G>((double)fy);
  double Fz = group_sum<double, G>((double)fz);
  double Ph = group_sum<double, G>((double)phi);
  if (active && sub == 0) {
    if (accumulate) {
      f[3 * i + 0] += Fx;
      f[3 * i + 1] += Fy;
      f[3 * i + 2] += Fz;
    } else {
      f[3 * i + 0] = Fx;
      f[3 * i + 1] = Fy;
      f[3 * i + 2] = Fz;
    }
    if (e_fast) e_fast[i] = xi[i] + 0.5 * Ph;
  }
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

template <typename R>
void run_eam(ap_ctx* c, const typename Shadow<R>::T* sh, const double* d_lam, double* d_e_fast, double* d_f,
             bool accumulate, cudaStream_t s) {
  constexpr int G = 8;
  const int threads = 256;
  int blocks = (int)((c->n * G + threads - 1) / threads);
  EamP<R> p = make_params<R>(c->cfg);
  auto* q = reinterpret_cast<typename Q2<R>::T*>(c->d_q);
  const int* off = c->stored_off ? c->d_off_eam : nullptr;
  k_eam_density<R, G><<<blocks, threads, 0, s>>>((int)c->n, c->d_sys, c->d_atom_sys, sh, c->d_nbr_eam, off,
                                                 c->d_cnt_eam, c->cap_eam, p, d_lam, q, c->d_xi);
  k_eam_force<R, G><<<blocks, threads, 0, s>>>((int)c->n, c->d_sys, c->d_atom_sys, sh, c->d_nbr_eam, off,
                                               c->d_cnt_eam, c->cap_eam, p, q, c->d_xi, d_e_fast, d_f,
                                               accumulate ? 1 : 0);
  c->kernels += 2;
}

}  // namespace

void launch_eam(ap_ctx* c, const double* d_lam, double* d_e_fast, double* d_f, bool accumulate, cudaStream_t s) {
  if (c->n <= 0) return;
  if (c->cfg.precision == AP_PREC_FP64)
    run_eam<double>(c, c->d_sh64, d_lam, d_e_fast, d_f, accumulate, s);
  else
    run_eam<float>(c, c->d_sh32, d_lam, d_e_fast, d_f, accumulate, s);
}

}  // namespace ap
