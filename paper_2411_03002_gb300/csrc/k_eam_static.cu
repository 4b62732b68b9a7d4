// Allocation-free EAM evaluation (ap_eval_eam_static).
//
// Some callers cannot allocate device memory at all: code running inside a
// host process whose allocator is owned by someone else (a plugin living in
// another framework's memory pool, a pre-sized embedded deployment, a process
// that has already handed its memory budget to another runtime).  For them this
// entry point computes the same quantities as ap_eval_eam -- EAM site energies and
// the lambda-weighted EAM force -- for one small system without a context,
// without neighbour rows and without any cudaMalloc.  Pairs are found by brute
// force over all atoms and periodic images, so it is meant for small systems.
//
// The per-atom scratch it needs between the density pass and the force pass
// (lambda xi'(rho), lambda and xi(rho) of every atom) lives in one file-scope
// device array of fixed size, so at most kStaticMaxAtoms atoms are accepted.
// Every GPU that loads the library holds that array until the process exits.
// All calls share the array: two calls whose kernels overlap on the GPU (for
// example on different streams) race and give wrong results; serialise them.
// Each call overwrites the scratch of atoms 0..n-1 before reading it, so nothing
// has to be cleared between calls.
#include <mutex>

#include "ap_internal.cuh"

namespace ap {
namespace {

constexpr int kStaticMaxAtoms = 32768;
// (lambda xi', lambda, xi) per atom
static __device__ __align__(256) double g_eam_scratch[3 * kStaticMaxAtoms];

struct StaticBox {
  double lo[3], L[3];
  int periodic[3];
};

struct StaticEam {
  double beta, beta_r0, alpha, A, D, rp, rc, rc2, inv_h;
};

// psi(u) = u^4/(1+u^4) and dpsi/du for u < 0
__device__ inline void psi_d(double u, double& ps, double& dps) {
  double u2 = u * u, u4 = u2 * u2, inv = 1.0 / (1.0 + u4);
  ps = u4 * inv;
  dps = 4.0 * u2 * u * inv * inv;
}

// Image range along one dimension that can bring displacement d0 within rc.
__device__ inline void image_range(const StaticBox& b, int d, double d0, double rc, int& lo, int& hi) {
  if (!b.periodic[d]) {
    lo = hi = 0;
    return;
  }
  lo = (int)ceil((-rc - d0) / b.L[d]) - 1;
  hi = (int)floor((rc - d0) / b.L[d]) + 1;
}

template <typename F>
__device__ inline void for_each_image(int n, const double* __restrict__ x, const StaticBox& b, double rc2, double rc,
                                      int i, F&& f) {
  const double xi0 = x[3 * i], xi1 = x[3 * i + 1], xi2 = x[3 * i + 2];
  for (int j = 0; j < n; ++j) {
    const double d0[3] = {x[3 * j] - xi0, x[3 * j + 1] - xi1, x[3 * j + 2] - xi2};
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) image_range(b, d, d0[d], rc, lo[d], hi[d]);
    for (int sx = lo[0]; sx <= hi[0]; ++sx)
      for (int sy = lo[1]; sy <= hi[1]; ++sy)
        for (int sz = lo[2]; sz <= hi[2]; ++sz) {
          if (j == i && sx == 0 && sy == 0 && sz == 0) continue;
          const double dx = d0[0] + sx * b.L[0], dy = d0[1] + sy * b.L[1], dz = d0[2] + sz * b.L[2];
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < rc2) f(j, dx, dy, dz, r2);
        }
  }
}

__global__ void k_eam_static_density(int n, const double* __restrict__ x, StaticBox b, StaticEam p,
                                     const double* __restrict__ lam, double* __restrict__ scratch) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double rho = 0.0;
  for_each_image(n, x, b, p.rc2, p.rc, i, [&](int, double, double, double, double r2) {
    double r = sqrt(r2), ps, dps;
    psi_d((r - p.rc) * p.inv_h, ps, dps);
    rho += exp(p.beta - p.beta_r0 * r) * ps;
  });
  double xi = 0.0, dxi = 0.0;
  if (rho > 0.0) {
    double s = sqrt(rho);
    xi = -p.A * s;
    dxi = -p.A / (2.0 * s);
  }
  double li = lam ? lam[i] : 1.0;
  scratch[3 * i + 0] = li * dxi;
  scratch[3 * i + 1] = li;
  scratch[3 * i + 2] = xi;
}

__global__ void k_eam_static_force(int n, const double* __restrict__ x, StaticBox b, StaticEam p,
                                   const double* __restrict__ scratch, double* __restrict__ e_fast,
                                   double* __restrict__ f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double qi = scratch[3 * i], li = scratch[3 * i + 1];
  double fx = 0.0, fy = 0.0, fz = 0.0, phi = 0.0;
  for_each_image(n, x, b, p.rc2, p.rc, i, [&](int j, double dx, double dy, double dz, double r2) {
    double r = sqrt(r2), ps, dps;
    psi_d((r - p.rc) * p.inv_h, ps, dps);
    dps *= p.inv_h;
    double ez = exp(p.beta - p.beta_r0 * r);
    double dzeta = ez * (dps - p.beta_r0 * ps);
    double e1 = exp(-p.alpha * (r - p.rp)), e2 = e1 * e1;
    double m = p.D * (e2 - 2.0 * e1), dm = 2.0 * p.alpha * p.D * (e1 - e2);
    phi += m * ps;
    double g = (qi + scratch[3 * j]) * dzeta + 0.5 * (li + scratch[3 * j + 1]) * (dm * ps + m * dps);
    double s = g / r;
    fx += s * dx;
    fy += s * dy;
    fz += s * dz;
  });
  f[3 * i + 0] += fx;
  f[3 * i + 1] += fy;
  f[3 * i + 2] += fz;
  e_fast[i] = scratch[3 * i + 2] + 0.5 * phi;
}

// Device address of the scratch array, looked up once per device.
std::mutex g_mu;
void* g_ptr[128] = {};

ap_status scratch_address(double** out, int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return AP_ERR_CUDA;
  *dev_out = dev;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_eam_scratch) != cudaSuccess || !p) return AP_ERR_CUDA;
    g_ptr[dev] = p;
  }
  *out = static_cast<double*>(g_ptr[dev]);
  return AP_OK;
}

}  // namespace
}  // namespace ap

extern "C" ap_status ap_eval_eam_static(const ap_config* h_cfg, int64_t n, const double* d_x, const ap_box* h_box,
                                        const double* d_lam, double* d_e_fast, double* d_f, void* stream) {
  using namespace ap;
  if (!h_cfg || !h_box || n < 0) return AP_ERR_ARG;
  if (n > kStaticMaxAtoms) return AP_ERR_ARG;
  if (n == 0) return AP_OK;
  if (!d_x || !d_e_fast || !d_f) return AP_ERR_ARG;
  const ap_config& c = *h_cfg;
  if (c.eam_type != AP_EAM_ANALYTIC) return AP_ERR_ARG;
  if (!(c.eam_rc > 0 && c.eam_h > 0 && c.eam_r0 > 0)) return AP_ERR_ARG;
  StaticBox b;
  for (int d = 0; d < 3; ++d) {
    b.lo[d] = h_box->lo[d];
    b.L[d] = h_box->hi[d] - h_box->lo[d];
    b.periodic[d] = h_box->periodic[d] ? 1 : 0;
    if (!(b.L[d] > 0)) return AP_ERR_ARG;
  }
  StaticEam p{c.eam_beta, c.eam_beta / c.eam_r0, c.eam_alpha, c.eam_A, c.eam_D, c.eam_rp, c.eam_rc,
              c.eam_rc * c.eam_rc, 1.0 / c.eam_h};
  double* scratch = nullptr;
  int dev = 0;
  ap_status st = scratch_address(&scratch, &dev);
  if (st != AP_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (s) {   // the scratch address is the current device's, so the stream must run there too
    int sdev = -1;
    if (cudaStreamGetDevice(s, &sdev) == cudaSuccess && sdev != dev) return AP_ERR_ARG;
    cudaGetLastError();
  }
  const int threads = 128, blocks = (int)((n + threads - 1) / threads);
  k_eam_static_density<<<blocks, threads, 0, s>>>((int)n, d_x, b, p, d_lam, scratch);
  k_eam_static_force<<<blocks, threads, 0, s>>>((int)n, d_x, b, p, scratch, d_e_fast, d_f);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}
