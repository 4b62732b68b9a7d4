// Local thermostat (Appendix C): energy errors of a lambda update and their
// momentum-conserving correction.
//
//   k_th_delta     Delta lambda_i = lambda_i^c - lambda_i^d and the ACE weights -Delta lambda_i
//                  of the difference force (F^c - F^d is linear in Delta lambda: an EAM
//                  pass with weights Delta lambda plus an ACE pass over K = {Delta lambda != 0}
//                  with weights -Delta lambda, run by the caller);
//   k_th_energy    Delta E_i = Delta T_i + Delta V_i (Eqs. Delta_T_i, Delta_V_i, Delta_E_i)
//                  from F^d, F^c - F^d, v(t + dt/2), E^f and E^p, for mobile atoms;
//   k_th_bin/...   the atoms with Delta E_i != 0 binned into sweep cells of edge
//                  >= 2 (r_row + skin), sorted by index inside a cell;
//   k_th_rescale   one warp per cell of one colour (8 launches): for every atom of
//                  the cell in ascending index, Omega_i = {i} + the distinct mobile
//                  atoms of its EAM row, v_cm, the relative kinetic energy, beta
//                  (Eq. beta_omega_i) and v_j <- v_cm + beta (v_j - v_cm)
//                  (Eq. p_resc_omega).  Cells of one colour are a cell apart, so
//                  their groups are disjoint and run concurrently.
#include <cmath>

#include "ap_internal.cuh"

namespace ap {

namespace {

constexpr double kAcc = 1.602176634e-19 / 1.66053906660e-27 * 1e-20 / 1e-10;   // A/fs^2 per eV/(A amu)

__global__ void k_th_delta(int n, const double* __restrict__ lam_c, const double* __restrict__ lam_d,
                           double* __restrict__ dlam, double* __restrict__ wneg, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = lam_c[i] - lam_d[i];
  dlam[i] = d;
  wneg[i] = -d;
  flag[i] = d != 0.0 ? 1 : 0;
}

__global__ void k_th_energy(int n, const double* __restrict__ dlam, const double* __restrict__ e_fast,
                            const double* __restrict__ e_prec_k, const double* __restrict__ f_d,
                            const double* __restrict__ df, const double* __restrict__ v_half,
                            const double* __restrict__ mass, const uint8_t* __restrict__ fixed, double dt,
                            double* __restrict__ dE, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double e = 0.0;
  if (!(fixed && fixed[i])) {
    // F^c^2 - F^d^2 written as d (2 F^d + d) with d = F^c - F^d: exactly 0 where the
    // difference force is 0 (a contracted fc*fc - fd*fd would leave a rounding residue).
    const double c1 = dt * dt * kAcc / (8.0 * mass[i]);
    for (int a = 0; a < 3; ++a) {
      const double fd = f_d[3 * i + a];
      const double d = df[3 * i + a];
      e += d * (c1 * (2.0 * fd + d) + 0.5 * dt * v_half[3 * i + a]);
    }
    const double dl = dlam[i];
    if (dl != 0.0) e += dl * (e_fast[i] - e_prec_k[i]);
  }
  dE[i] = e;
  flag[i] = e != 0.0 ? 1 : 0;
}

struct ThCells {
  double lo[3], h[3];
  int nc[3], periodic[3];
  double L[3];
};

__device__ inline int th_cell(const ThCells& T, const double* x) {
  int c[3];
  for (int d = 0; d < 3; ++d) {
    double s = x[d] - T.lo[d];
    if (T.periodic[d]) {
      s = fmod(s, T.L[d]);
      if (s < 0) s += T.L[d];
    }
    int k = (int)floor(s / T.h[d]);
    c[d] = k < 0 ? 0 : (k >= T.nc[d] ? T.nc[d] - 1 : k);
  }
  return (c[2] * T.nc[1] + c[1]) * T.nc[0] + c[0];
}

__global__ void k_th_count(const int* __restrict__ q, const int* __restrict__ m, const double* __restrict__ x,
                           ThCells T, int* __restrict__ cell_of, int* __restrict__ count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *m) return;
  const int c = th_cell(T, &x[3 * q[k]]);
  cell_of[k] = c;
  atomicAdd(&count[c], 1);
}

__global__ void k_th_scatter(const int* __restrict__ q, const int* __restrict__ m, const int* __restrict__ cell_of,
                             const int* __restrict__ start, int* __restrict__ fill, int* __restrict__ atoms) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *m) return;
  const int c = cell_of[k];
  atoms[start[c] + atomicAdd(&fill[c], 1)] = q[k];
}

// Ascending index inside every cell (insertion sort; cells hold a few hundred atoms).
__global__ void k_th_sort(int n_cells, const int* __restrict__ start, int* __restrict__ atoms) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const int b = start[c], e = start[c + 1];
  for (int a = b + 1; a < e; ++a) {
    const int v = atoms[a];
    int p = a - 1;
    while (p >= b && atoms[p] > v) {
      atoms[p + 1] = atoms[p];
      --p;
    }
    atoms[p + 1] = v;
  }
}

template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Member test for row entry t of atom i: a mobile atom other than i that does not
// appear earlier in the row (rows may hold several images of one atom).
__device__ inline bool member(const int* __restrict__ row, int t, int i, const uint8_t* __restrict__ fixed) {
  const int j = row[t];
  if (j == i || (fixed && fixed[j])) return false;
  for (int u = 0; u < t; ++u)
    if (row[u] == j) return false;
  return true;
}

__global__ void k_th_rescale(ThCells T, int color, const int* __restrict__ start, const int* __restrict__ atoms,
                             const int* __restrict__ nbr, const int* __restrict__ cnt, int cap,
                             const uint8_t* __restrict__ fixed, const double* __restrict__ mass,
                             const double* __restrict__ dE, double* __restrict__ v, DevScalars* __restrict__ sc) {
  const int lane = threadIdx.x & 31;
  const int px = color & 1, py = (color >> 1) & 1, pz = (color >> 2) & 1;
  const int mx = (T.nc[0] + 1 - px) / 2, my = (T.nc[1] + 1 - py) / 2, mz = (T.nc[2] + 1 - pz) / 2;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= mx * my * mz) return;
  const int cx = 2 * (w % mx) + px, cy = 2 * ((w / mx) % my) + py, cz = 2 * (w / (mx * my)) + pz;
  const int cell = (cz * T.nc[1] + cy) * T.nc[0] + cx;
  for (int a = start[cell]; a < start[cell + 1]; ++a) {
    const int i = atoms[a];
    const double de = dE[i];
    const int c = cnt[i];
    const int* row = nbr + (size_t)i * cap;
    // pass 1: total mass and momentum of Omega_i
    double sm = 0.0, spx = 0.0, spy = 0.0, spz = 0.0;
    if (lane == 0) {
      const double mi = mass[i];
      sm = mi;
      spx = mi * v[3 * i];
      spy = mi * v[3 * i + 1];
      spz = mi * v[3 * i + 2];
    }
    for (int t = lane; t < c; t += 32) {
      if (!member(row, t, i, fixed)) continue;
      const int j = row[t];
      const double mj = mass[j];
      sm += mj;
      spx += mj * v[3 * j];
      spy += mj * v[3 * j + 1];
      spz += mj * v[3 * j + 2];
    }
    sm = warp_sum(sm);
    const double vcx = warp_sum(spx) / sm, vcy = warp_sum(spy) / sm, vcz = warp_sum(spz) / sm;
    // pass 2: relative kinetic energy
    double k = 0.0;
    if (lane == 0) {
      const double ax = v[3 * i] - vcx, ay = v[3 * i + 1] - vcy, az = v[3 * i + 2] - vcz;
      k = 0.5 * mass[i] * (ax * ax + ay * ay + az * az);
    }
    for (int t = lane; t < c; t += 32) {
      if (!member(row, t, i, fixed)) continue;
      const int j = row[t];
      const double ax = v[3 * j] - vcx, ay = v[3 * j + 1] - vcy, az = v[3 * j + 2] - vcz;
      k += 0.5 * mass[j] * (ax * ax + ay * ay + az * az);
    }
    k = warp_sum(k) / kAcc;
    const double rad = k > 0.0 ? de / k + 1.0 : (de == 0.0 ? 1.0 : -1.0);
    if (rad < 0.0) {
      if (lane == 0) {
        atomicOr(&sc->err, kErrRadicand);
        atomicAdd(&sc->th_bad, 1ull);
      }
      __syncwarp();
      continue;
    }
    const double beta = sqrt(rad);
    // pass 3: rescale the relative velocities (every member written by one lane)
    if (lane == 0) {
      v[3 * i] = vcx + beta * (v[3 * i] - vcx);
      v[3 * i + 1] = vcy + beta * (v[3 * i + 1] - vcy);
      v[3 * i + 2] = vcz + beta * (v[3 * i + 2] - vcz);
      atomicAdd(&sc->th_n, 1ull);
      atomicAdd(&sc->th_e, de);
    }
    for (int t = lane; t < c; t += 32) {
      if (!member(row, t, i, fixed)) continue;
      const int j = row[t];
      v[3 * j] = vcx + beta * (v[3 * j] - vcx);
      v[3 * j + 1] = vcy + beta * (v[3 * j + 1] - vcy);
      v[3 * j + 2] = vcz + beta * (v[3 * j + 2] - vcz);
    }
    __syncwarp();
  }
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

ThCells th_cells(const ap_ctx* c) {
  const SysInfo& S = c->h_sys[0];
  ThCells T;
  const double hmin = 2.0 * (c->cfg.eam_rc + c->cfg.skin + c->cfg.skin);
  for (int d = 0; d < 3; ++d) {
    int nc = (int)std::floor(S.L[d] / hmin);
    if (nc < 1) nc = 1;
    if (S.periodic[d] && nc > 1 && (nc & 1)) --nc;
    T.nc[d] = nc;
    T.lo[d] = S.lo[d];
    T.L[d] = S.L[d];
    T.h[d] = S.L[d] / nc;
    T.periodic[d] = S.periodic[d];
  }
  return T;
}

}  // namespace

int th_cell_count(const ap_ctx* c) {
  ThCells T = th_cells(c);
  return T.nc[0] * T.nc[1] * T.nc[2];
}

void launch_th_delta(ap_ctx* c, const double* d_lam_c, const double* d_lam_d, cudaStream_t s) {
  const int n = (int)c->n;
  k_th_delta<<<nblk(n, 256), 256, 0, s>>>(n, d_lam_c, d_lam_d, c->d_th_dlam, c->d_th_w, c->d_flag);
  c->kernels += 1;
}

void launch_th_energy(ap_ctx* c, const double* d_f, const double* d_v, const double* d_mass, const uint8_t* d_fixed,
                      cudaStream_t s) {
  const int n = (int)c->n;
  k_th_energy<<<nblk(n, 256), 256, 0, s>>>(n, c->d_th_dlam, c->d_efast, c->d_th_ep, d_f, c->d_th_df, d_v, d_mass,
                                           d_fixed, c->cfg.dt, c->d_th_de, c->d_flag);
  c->kernels += 1;
}

// Bin the queue d_q (count *d_m) into sweep cells and run the 8 colour sweeps.
void launch_th_correct(ap_ctx* c, const int* d_q, const int* d_m, const double* d_x, const uint8_t* d_fixed,
                       const double* d_mass, double* d_v, cudaStream_t s) {
  const int n = (int)c->n;
  ThCells T = th_cells(c);
  const int nc = T.nc[0] * T.nc[1] * T.nc[2];
  cudaMemsetAsync(c->d_th_ccount, 0, sizeof(int) * (size_t)nc, s);
  k_th_count<<<nblk(n, 256), 256, 0, s>>>(d_q, d_m, d_x, T, c->d_th_cellof, c->d_th_ccount);
  c->kernels += 1 + scan_exclusive(c->d_th_ccount, c->d_th_cstart, nc, c->d_scan_tmp, s);
  cudaMemsetAsync(c->d_th_ccount, 0, sizeof(int) * (size_t)nc, s);
  k_th_scatter<<<nblk(n, 256), 256, 0, s>>>(d_q, d_m, c->d_th_cellof, c->d_th_cstart, c->d_th_ccount, c->d_th_atoms);
  k_th_sort<<<nblk(nc, 128), 128, 0, s>>>(nc, c->d_th_cstart, c->d_th_atoms);
  c->kernels += 2;
  for (int color = 0; color < 8; ++color) {
    const int px = color & 1, py = (color >> 1) & 1, pz = (color >> 2) & 1;
    const int cells = ((T.nc[0] + 1 - px) / 2) * ((T.nc[1] + 1 - py) / 2) * ((T.nc[2] + 1 - pz) / 2);
    if (cells <= 0) continue;
    k_th_rescale<<<nblk(32 * cells, 128), 128, 0, s>>>(T, color, c->d_th_cstart, c->d_th_atoms, c->d_nbr_eam,
                                                       c->d_cnt_eam, c->cap_eam, d_fixed, d_mass, c->d_th_de, d_v,
                                                       c->d_sc);
    c->kernels += 1;
  }
}

}  // namespace ap
