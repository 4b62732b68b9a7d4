// Velocity Verlet with the lambda step (Eq. vv), the external indenter, the
// blended energy E_i = lambda_i E_i^(f) + (1 - lambda_i) E_i^(p) (Eq. energy_hyb)
// and fixed-order FP64 reductions (bitwise reproducible for a given n).
#include "ap_internal.cuh"

namespace ap {

namespace {

// 1 eV/(A amu) in A/fs^2, from 1 eV = 1.602176634e-19 J and 1 amu = 1.66053906660e-27 kg
constexpr double kAcc = 1.602176634e-19 / 1.66053906660e-27 * 1e-20 / 1e-10;
constexpr int kRedBlocks = 512;
constexpr int kRedThreads = 256;
constexpr int kVvThreads = 256;   // block size of k_vv_first (its block reduction)

// Half-kick factor s_i = 0.5 dt ACC / m_i, once per ap_step call (FP64 division is
// slow on this GPU; the kicks then need one FMA per component).
__global__ void k_vscale(int n, const double* __restrict__ mass, double dt, double* __restrict__ vs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) vs[i] = 0.5 * dt * kAcc / mass[i];
}

// Half kick and drift, and the new positions' cell-relative shadows (the k_shadow
// arithmetic, relative to the cells of the last build).  The displacement since the
// build (skin check) is the difference of the FP32 shadow and the build's shadow s32b:
// both are relative to the same cell, so it is exact to a few 1e-7 A.
__global__ void k_vv_first(int n, double* __restrict__ x, double* __restrict__ v, const double* __restrict__ f,
                           const double* __restrict__ vs, const uint8_t* __restrict__ fixed, double dt,
                           const SysInfo* __restrict__ sys, const int* __restrict__ atom_sys,
                           const double* __restrict__ org, const int4* __restrict__ cunw, float4* __restrict__ s32,
                           double4_32a* __restrict__ s64,
                           const float4* __restrict__ s32b, const float4* __restrict__ s32a, DevScalars* sc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  float d2 = 0.f, d2a = 0.f;   // squared displacement since the build / the ACE row build
  if (i < n) {
    double xx[3];
    const bool mobile = !(fixed && fixed[i]);
    if (!mobile) {
      v[3 * i + 0] = v[3 * i + 1] = v[3 * i + 2] = 0.0;
      for (int a = 0; a < 3; ++a) xx[a] = x[3 * i + a];
    } else {
      const double s = vs[i];
      bool bad = false;
      for (int a = 0; a < 3; ++a) {
        double vv = v[3 * i + a] + s * f[3 * i + a];
        xx[a] = x[3 * i + a] + dt * vv;
        v[3 * i + a] = vv;
        x[3 * i + a] = xx[a];
        bad |= (__double2hiint(xx[a]) & 0x7ff00000) == 0x7ff00000;   // inf or nan (exponent bits)
      }
      if (bad) atomicOr(&sc->err, kErrNonfinite);
    }
    const SysInfo& S = sys[atom_sys ? atom_sys[i] : 0];
    const int4 c = cunw[i];
    double sh[3];
    cell_shadow(S, org, c, xx, sh);
    const float4 s4 = make_float4((float)sh[0], (float)sh[1], (float)sh[2], __int_as_float(c.w));
    s32[i] = s4;
    if (s64) s64[i] = make_double4_32a(sh[0], sh[1], sh[2], (double)c.w);
    if (mobile) {
      const float4 b = s32b[i];
      const float ex = s4.x - b.x, ey = s4.y - b.y, ez = s4.z - b.z;
      d2 = ex * ex + ey * ey + ez * ez;
      if (s32a) {
        const float4 ba = s32a[i];
        const float ax = s4.x - ba.x, ay = s4.y - ba.y, az = s4.z - ba.z;
        d2a = ax * ax + ay * ay + az * az;
      }
    }
  }
  // block maxima first: one atomic per block and quantity (same-address atomics from every
  // warp serialise in L2 and cost more than the rest of the kernel)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    d2a = fmaxf(d2a, __shfl_xor_sync(0xffffffffu, d2a, o));
  }
  __shared__ float red[2][kVvThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = d2;
    red[1][wid] = d2a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      d2 = fmaxf(d2, red[0][k]);
      d2a = fmaxf(d2a, red[1][k]);
    }
    if (d2 > 0.f) atomicMax(&sc->max_disp2_bits, __float_as_uint(d2));
    if (s32a && d2a > 0.f) atomicMax(&sc->max_dispa2_bits, __float_as_uint(d2a));
  }
}

__global__ void k_vv_second(int n, double* __restrict__ v, const double* __restrict__ f,
                            const double* __restrict__ vs, const uint8_t* __restrict__ fixed) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (fixed && fixed[i]) {
    v[3 * i + 0] = v[3 * i + 1] = v[3 * i + 2] = 0.0;
    return;
  }
  const double s = vs[i];
  for (int a = 0; a < 3; ++a) v[3 * i + a] += s * f[3 * i + a];
}

// Spherical indenter: F = k (R - r)^2 (x - c)/r, E = k (R - r)^3 / 3 for r < R.
__global__ void k_indenter(int n, const double* __restrict__ x, double* __restrict__ f, double* __restrict__ e_ext,
                           double cx, double cy, double cz, double R, double k) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double dz = x[3 * i + 2] - cz;
  if (!(dz < R && dz > -R)) {   // r^2 < R^2 needs |dz| < R: most atoms stop here
    if (e_ext) e_ext[i] = 0.0;
    return;
  }
  double dx = x[3 * i] - cx, dy = x[3 * i + 1] - cy;
  double r2 = dx * dx + dy * dy + dz * dz;
  double e = 0.0;
  if (r2 < R * R && r2 > 0.0) {
    double r = sqrt(r2);
    double g = k * (R - r) * (R - r) / r;
    f[3 * i + 0] += g * dx;
    f[3 * i + 1] += g * dy;
    f[3 * i + 2] += g * dz;
    e = k * (R - r) * (R - r) * (R - r) / 3.0;
  }
  if (e_ext) e_ext[i] = e;
}

template <typename F>
__device__ inline void block_reduce_store(double v, double* out) {
  __shared__ double sh[kRedThreads];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// Fixed partition: block b owns [b*chunk, (b+1)*chunk); thread t sums a strided
// sequence in order; the tree order is fixed.  Same n -> same bits.
__global__ void k_blend_partial(int n, const double* __restrict__ lam, const double* __restrict__ ef,
                                const double* __restrict__ ep, const double* __restrict__ e_ext,
                                double* __restrict__ e_atom, double* __restrict__ part) {
  int chunk = (n + gridDim.x - 1) / gridDim.x;
  int b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  double s = 0.0;
  for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    double l = lam ? lam[i] : 1.0;
    double e = l * ef[i] + (1.0 - l) * (ep ? ep[i] : 0.0);
    if (e_atom) e_atom[i] = e;
    if (e_ext) e += e_ext[i];
    s += e;
  }
  block_reduce_store<double>(s, &part[blockIdx.x]);
}

__global__ void k_kin_partial(int n, const double* __restrict__ v, const double* __restrict__ mass,
                              double* __restrict__ part) {
  int chunk = (n + gridDim.x - 1) / gridDim.x;
  int b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  double s = 0.0;
  for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    double vv = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
    s += 0.5 * mass[i] * vv / kAcc;
  }
  block_reduce_store<double>(s, &part[blockIdx.x]);
}

__global__ void k_final_sum(int m, const double* __restrict__ part, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += part[i];
  block_reduce_store<double>(s, out);
}

__global__ void k_fill(int n, double* __restrict__ a, double v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

void launch_vscale(ap_ctx* c, const double* d_mass, cudaStream_t s) {
  k_vscale<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, d_mass, c->cfg.dt, c->d_vscale);
  c->kernels += 1;
}

void launch_vv_first(ap_ctx* c, double* d_x, double* d_v, const double* d_f, const double* d_mass,
                     const uint8_t* d_fixed, cudaStream_t s) {
  (void)d_mass;   // the half-kick factors come from launch_vscale
  k_vv_first<<<nblk(c->n, kVvThreads), kVvThreads, 0, s>>>((int)c->n, d_x, d_v, d_f, c->d_vscale, d_fixed, c->cfg.dt, c->d_sys,
                                             c->d_atom_sys, c->d_org, c->d_cunw, c->d_sh32,
                                             c->cfg.precision == AP_PREC_FP64 ? c->d_sh64 : nullptr, c->d_sh32b,
                                             c->cfg.rebuild_every == AP_REBUILD_SKIN ? c->d_sh32a : nullptr, c->d_sc);
  c->kernels += 1;
}

void launch_vv_second(ap_ctx* c, double* d_v, const double* d_f, const double* d_mass, const uint8_t* d_fixed,
                      cudaStream_t s) {
  (void)d_mass;
  k_vv_second<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, d_v, d_f, c->d_vscale, d_fixed);
  c->kernels += 1;
}

void launch_indenter(ap_ctx* c, const double* d_x, double* d_f, double t, cudaStream_t s) {
  const ap_config& g = c->cfg;
  k_indenter<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, d_x, d_f, c->d_eext, g.ind_c0[0] + g.ind_v[0] * t,
                                             g.ind_c0[1] + g.ind_v[1] * t, g.ind_c0[2] + g.ind_v[2] * t, g.ind_R,
                                             g.ind_k);
  c->kernels += 1;
}

void launch_blend(ap_ctx* c, const double* d_lam, const double* d_ef, const double* d_ep, const double* d_e_ext,
                  double* d_e_atom, double* d_e_total, cudaStream_t s) {
  k_blend_partial<<<kRedBlocks, kRedThreads, 0, s>>>((int)c->n, d_lam, d_ef, d_ep, d_e_ext, d_e_atom, c->d_red);
  k_final_sum<<<1, kRedThreads, 0, s>>>(kRedBlocks, c->d_red, d_e_total);
  c->kernels += 2;
}

void launch_kinetic(ap_ctx* c, const double* d_v, const double* d_mass, double* d_out, cudaStream_t s) {
  k_kin_partial<<<kRedBlocks, kRedThreads, 0, s>>>((int)c->n, d_v, d_mass, c->d_red + kRedBlocks);
  k_final_sum<<<1, kRedThreads, 0, s>>>(kRedBlocks, c->d_red + kRedBlocks, d_out);
  c->kernels += 2;
}

void launch_fill_lambda(ap_ctx* c, double* d_lam, double value, cudaStream_t s) {
  k_fill<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, d_lam, value);
  c->kernels += 1;
}

}  // namespace ap
