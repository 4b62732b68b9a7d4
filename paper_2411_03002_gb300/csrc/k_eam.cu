// EAM site energies (Eq. energy_eam) and the lambda-weighted force of Eq. F_i_d at
// fixed lambda.  Two passes over the neighbour rows, G lanes per atom with
// shuffle reductions:
//   density: rho_i = sum_j zeta(r_ij); q_i = (lambda_i xi'(rho_i), lambda_i)
//   force:   F_i = sum_j g_ij (x_j - x_i)/r_ij with
//            g_ij = (lambda_i xi'_i + lambda_j xi'_j) zeta'(r_ij) + (lambda_i + lambda_j)/2 Phi'(r_ij),
//            which is -grad_i sum_k lambda_k E_k^(f) gathered without atomics;
//            E_i^(f) = xi_i + 1/2 sum_j Phi(r_ij)  (the Phi sum reduced in FP64).
// Analytic forms: zeta(r) = exp(-beta (r/r0 - 1)) psi, Phi(r) = D (e^{-2a(r-rp)} -
// 2 e^{-a(r-rp)}) psi, xi(rho) = -A sqrt(rho), psi = u^4/(1+u^4), u = (r - rc)/h < 0.
//
// Pair displacements come from cell-relative shadows: d = k h + s_j - s_i with k
// the pair's cell offset, either stored per entry (small periodic boxes) or
// unwrapped from the packed cell codes (branch-free, per-atom constants hoisted).
#include "ap_internal.cuh"
#include "eam_frame.cuh"

namespace ap {

namespace {

template <typename R, int G, bool STORED>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? AP_EAM_MINB : 1) k_eam_density(int n, const SysInfo* __restrict__ sys,
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
  const auto si = sh[i];
  const Frame<R, STORED> fr(sys[atom_sys ? atom_sys[i] : 0], si);
  const int c = active ? cnt[i] : 0;
  const size_t row = (size_t)i * cap;
  R rho = R(0);
#pragma unroll 4
  for (int t = sub; t < c; t += G) {
    const int j = nbr[row + t];
    const auto sj = sh[j];
    R d[3];
    fr.disp(sj, off, row + t, d);
    const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 < p.rc2) {
      const R r = r2 * rsqrt_(r2);
      const R u = (r - p.rc) * p.inv_h;
      const R u2 = u * u;
      const R u4 = u2 * u2;
      rho += rexp(p.beta - p.beta_r0 * r) * (u4 * rcp_(R(1) + u4));
    }
  }
  rho = group_sum<R, G>(rho);
  if (active && sub == 0) {
    const R li = lam ? (R)lam[i] : R(1);
    R xi = R(0), dxi = R(0);
    if (rho > R(0)) {
      const R s = sqrt(rho);
      xi = -p.A * s;
      dxi = R(-0.5) * p.A * rcp_(s);
    }
    q[i] = Q2<R>::make(li * dxi, li);
    xi_out[i] = (double)xi;
  }
}

template <typename R, int G, bool STORED>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? AP_EAM_MINB : 1) k_eam_force(int n, const SysInfo* __restrict__ sys,
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
  const auto si = sh[i];
  const Frame<R, STORED> fr(sys[atom_sys ? atom_sys[i] : 0], si);
  const auto qi = q[i];
  const int c = active ? cnt[i] : 0;
  const size_t row = (size_t)i * cap;
  R fx = R(0), fy = R(0), fz = R(0), phi = R(0);
#pragma unroll 4
  for (int t = sub; t < c; t += G) {
    const int j = nbr[row + t];
    const auto sj = sh[j];
    const auto qj = q[j];
    R d[3];
    fr.disp(sj, off, row + t, d);
    const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 < p.rc2) {
      const R inv_r = rsqrt_(r2);
      const R r = r2 * inv_r;
      const R u = (r - p.rc) * p.inv_h;
      const R u2 = u * u;
      const R u4 = u2 * u2;
      const R inv = rcp_(R(1) + u4);
      const R ps = u4 * inv;
      const R dps = R(4) * u2 * u * inv * inv * p.inv_h;
      const R ez = rexp(p.beta - p.beta_r0 * r);
      const R dzeta = ez * (dps - p.beta_r0 * ps);
      const R e1 = rexp(-p.alpha * (r - p.rp));
      const R e2 = e1 * e1;
      const R m = p.D * (e2 - R(2) * e1);
      const R dm = R(2) * p.alpha * p.D * (e1 - e2);
      const R dphi = dm * ps + m * dps;
      phi += m * ps;
      const R g = (qi.x + qj.x) * dzeta + R(0.5) * (qi.y + qj.y) * dphi;
      const R s = g * inv_r;
      fx += s * d[0];
      fy += s * d[1];
      fz += s * d[2];
    }
  }
  fx = group_sum<R, G>(fx);
  fy = group_sum<R, G>(fy);
  fz = group_sum<R, G>(fz);
  const double ph = group_sum<double, G>((double)phi);
  if (active && sub == 0) {
    if (accumulate) {
      f[3 * i + 0] += (double)fx;
      f[3 * i + 1] += (double)fy;
      f[3 * i + 2] += (double)fz;
    } else {
      f[3 * i + 0] = (double)fx;
      f[3 * i + 1] = (double)fy;
      f[3 * i + 2] = (double)fz;
    }
    if (e_fast) e_fast[i] = xi[i] + 0.5 * ph;
  }
}

template <typename R, bool STORED>
void run_eam(ap_ctx* c, const typename Shadow<R>::T* sh, const double* d_lam, double* d_e_fast, double* d_f,
             bool accumulate, cudaStream_t s) {
  constexpr int G = AP_EAM_LANES;
  const int threads = 256;
  int blocks = (int)((c->n * G + threads - 1) / threads);
  EamP<R> p = make_params<R>(c->cfg);
  auto* q = reinterpret_cast<typename Q2<R>::T*>(c->d_q);
  const int* off = STORED ? c->d_off_eam : nullptr;
  k_eam_density<R, G, STORED><<<blocks, threads, 0, s>>>((int)c->n, c->d_sys, c->d_atom_sys, sh, c->d_nbr_eam,
                                                         off, c->d_cnt_eam, c->cap_eam, p, d_lam, q, c->d_xi);
  k_eam_force<R, G, STORED><<<blocks, threads, 0, s>>>((int)c->n, c->d_sys, c->d_atom_sys, sh, c->d_nbr_eam, off,
                                                       c->d_cnt_eam, c->cap_eam, p, q, c->d_xi, d_e_fast, d_f,
                                                       accumulate ? 1 : 0);
  c->kernels += 2;
}

}  // namespace

void launch_eam(ap_ctx* c, const double* d_lam, double* d_e_fast, double* d_f, bool accumulate, cudaStream_t s) {
  if (c->n <= 0) return;
  if (c->cfg.precision == AP_PREC_FP64) {
    if (c->stored_off)
      run_eam<double, true>(c, c->d_sh64, d_lam, d_e_fast, d_f, accumulate, s);
    else
      run_eam<double, false>(c, c->d_sh64, d_lam, d_e_fast, d_f, accumulate, s);
  } else {
    if (c->stored_off)
      run_eam<float, true>(c, c->d_sh32, d_lam, d_e_fast, d_f, accumulate, s);
    else
      run_eam<float, false>(c, c->d_sh32, d_lam, d_e_fast, d_f, accumulate, s);
  }
}

}  // namespace ap
