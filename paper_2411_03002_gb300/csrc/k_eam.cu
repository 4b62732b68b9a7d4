// EAM site energies (Eq. energy_eam) and the lambda-weighted force of Eq. F_i_d at
// fixed lambda.  Two passes over the neighbour rows, G lanes per atom with
// shuffle reductions:
//   density: rho_i = sum_j zeta(r_ij); q_i = (lambda_i xi'(rho_i), lambda_i)
//   force:   F_i = sum_j g_ij (x_j - x_i)/r_ij with
//            g_ij = (lambda_i xi'_i + lambda_j xi'_j) zeta'(r_ij) + (lambda_i + lambda_j)/2 Phi'(r_ij),
//            which is -grad_i sum_k lambda_k E_k^(f) gathered without atomics;
//            E_i^(f) = xi_i + 1/2 sum_j Phi(r_ij)  (E_i^(f) formed in FP64).
// The potential P is a functor (eam_frame.cuh): the analytic synthetic EAM or the
// Mishin EAM2 of Appendix E, selected by ap_config.eam_type.
//
// Pair displacements come from cell-relative shadows: d = k h + s_j - s_i with k
// the pair's cell offset, either stored per entry (small periodic boxes) or
// unwrapped from the packed cell codes (branch-free, per-atom constants hoisted).
//
// Rows hold every neighbour within r_c + skin, the ones inside r_c first (the row
// build orders them so).  The density pass tests every entry and stores lim_i, one
// past the last entry it found inside r_c; the force pass walks entries [0, lim_i)
// only, with the same test, so the entries it skips are exactly ones that add nothing.
#include "ap_internal.cuh"
#include "eam_frame.cuh"

namespace ap {

namespace {

// The per-lane walk over row entries t = sub, sub + G, ... < c, calling body(j, t),
// unrolled kEamUnroll deep.  (Loading the next group's row entries ahead of the current
// group by hand was measured slower than the compiler's schedule of this loop.)
template <int G, typename F>
__device__ __forceinline__ void walk_row(const int* __restrict__ rowp, int sub, int c, F&& body) {
#pragma unroll kEamUnroll
  for (int t = sub; t < c; t += G) body(rowp[t], t);
}

template <int G>
__device__ inline int group_max(int v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o, G));
  return v;
}

template <typename R, int G, bool STORED, typename P>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? P::kMinBlocks : 1) k_eam_density(int n, const SysInfo* __restrict__ sys,
                                                     const int* __restrict__ atom_sys,
                                                     const typename Shadow<R>::T* __restrict__ sh,
                                                     const int* __restrict__ nbr, const int* __restrict__ off,
                                                     const int* __restrict__ cnt, int cap, P p,
                                                     const double* __restrict__ lam,
                                                     typename Q2<R>::T* __restrict__ q, double* __restrict__ xi_out,
                                                     int* __restrict__ lim) {
  const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int sub = threadIdx.x & (G - 1);
  const bool active = gid < n;
  const int i = active ? gid : n - 1;
  const auto si = sh[i];
  const Frame<R, STORED> fr(sys[atom_sys ? atom_sys[i] : 0], si);
  const int c = active ? cnt[i] : 0;
  const size_t row = (size_t)i * cap;
  R rho = R(0);
  int last = -1;
  walk_row<G>(nbr + row, sub, c, [&](int j, int t) {
    const auto sj = sh[j];
    R d[3];
    fr.disp(sj, off, row + t, d);
    const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 < p.rc2) {
      rho += p.zeta(r2 * rsqrt_(r2));
      last = t;
    }
  });
  rho = group_sum<R, G>(rho);
  last = group_max<G>(last);
  if (active && sub == 0) {
    lim[i] = last + 1;
    const R li = lam ? (R)lam[i] : R(1);
    R xi, dxi;
    p.embed(rho, xi, dxi);
    q[i] = Q2<R>::make(li * dxi, li);
    xi_out[i] = (double)xi;
  }
}

template <typename R, int G, bool STORED, typename P>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? P::kMinBlocks : 1) k_eam_force(int n, const SysInfo* __restrict__ sys,
                                                   const int* __restrict__ atom_sys,
                                                   const typename Shadow<R>::T* __restrict__ sh,
                                                   const int* __restrict__ nbr, const int* __restrict__ off,
                                                   const int* __restrict__ cnt, int cap, P p,
                                                   const typename Q2<R>::T* __restrict__ q,
                                                   const double* __restrict__ xi, const int* __restrict__ lim,
                                                   double* __restrict__ e_fast, double* __restrict__ f,
                                                   int accumulate) {
  const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int sub = threadIdx.x & (G - 1);
  const bool active = gid < n;
  const int i = active ? gid : n - 1;
  const auto si = sh[i];
  const Frame<R, STORED> fr(sys[atom_sys ? atom_sys[i] : 0], si);
  const auto qi = q[i];
  const int c = active ? lim[i] : 0;
  const size_t row = (size_t)i * cap;
  R fx = R(0), fy = R(0), fz = R(0), phi = R(0);
  walk_row<G>(nbr + row, sub, c, [&](int j, int t) {
    const auto sj = sh[j];
    const auto qj = q[j];
    R d[3];
    fr.disp(sj, off, row + t, d);
    const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 < p.rc2) {
      const R inv_r = rsqrt_(r2);
      const R r = r2 * inv_r;
      R dzeta, ph, dphi;
      p.pair(r, dzeta, ph, dphi);
      phi += ph;
      const R g = (qi.x + qj.x) * dzeta + R(0.5) * (qi.y + qj.y) * dphi;
      const R s = g * inv_r;
      fx += s * d[0];
      fy += s * d[1];
      fz += s * d[2];
    }
  });
  fx = group_sum<R, G>(fx);
  fy = group_sum<R, G>(fy);
  fz = group_sum<R, G>(fz);
  // the G partial Phi sums are combined in the working precision, then widened once
  const double ph = (double)group_sum<R, G>(phi);
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

template <typename R, bool STORED, typename P>
void run_eam(ap_ctx* c, const P& p, const typename Shadow<R>::T* sh, const double* d_lam, double* d_e_fast,
             double* d_f, bool accumulate, cudaStream_t s) {
  constexpr int G = AP_EAM_LANES;
  const int threads = 256;
  int blocks = (int)((c->n * G + threads - 1) / threads);
  auto* q = reinterpret_cast<typename Q2<R>::T*>(c->d_q);
  const int* off = STORED ? c->d_off_eam : nullptr;
  k_eam_density<R, G, STORED, P><<<blocks, threads, 0, s>>>((int)c->n, c->d_sys, c->d_atom_sys, sh, c->d_nbr_eam,
                                                         off, c->d_cnt_eam, c->cap_eam, p, d_lam, q, c->d_xi,
                                                         c->d_lim_eam);
  const int t0 = prof_mark(c, s);
  k_eam_force<R, G, STORED, P><<<blocks, threads, 0, s>>>((int)c->n, c->d_sys, c->d_atom_sys, sh, c->d_nbr_eam, off,
                                                       c->d_cnt_eam, c->cap_eam, p, q, c->d_xi, c->d_lim_eam,
                                                       d_e_fast, d_f, accumulate ? 1 : 0);
  prof_add(c, AP_PHASE_EAM_FORCE, t0, prof_mark(c, s));
  c->kernels += 2;
  c->lim_valid = true;
}

template <typename R>
void run_eam_pot(ap_ctx* c, const typename Shadow<R>::T* sh, const double* d_lam, double* d_e_fast, double* d_f,
                 bool accumulate, cudaStream_t s) {
  if (c->cfg.eam_type == AP_EAM_MISHIN) {
    const PotMishin<R> p = make_mishin<R>(c->cfg);
    if (c->stored_off)
      run_eam<R, true>(c, p, sh, d_lam, d_e_fast, d_f, accumulate, s);
    else
      run_eam<R, false>(c, p, sh, d_lam, d_e_fast, d_f, accumulate, s);
  } else {
    const PotSynth<R> p = make_synth<R>(c->cfg);
    if (c->stored_off)
      run_eam<R, true>(c, p, sh, d_lam, d_e_fast, d_f, accumulate, s);
    else
      run_eam<R, false>(c, p, sh, d_lam, d_e_fast, d_f, accumulate, s);
  }
}

}  // namespace

void launch_eam(ap_ctx* c, const double* d_lam, double* d_e_fast, double* d_f, bool accumulate, cudaStream_t s) {
  if (c->n <= 0) return;
  if (c->cfg.precision == AP_PREC_FP64)
    run_eam_pot<double>(c, c->d_sh64, d_lam, d_e_fast, d_f, accumulate, s);
  else
    run_eam_pot<float>(c, c->d_sh32, d_lam, d_e_fast, d_f, accumulate, s);
}

}  // namespace ap
