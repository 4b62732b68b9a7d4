/*
 * CPU oracle for the adaptive-precision EAM/ACE force evaluation (arXiv 2411.03002).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and may be
 * used by tests/, by __graft_entry__.smoke() and by bench.py's CPU-baseline leg.
 * The product path never loads it.  It shares no code, header, table or helper
 * with the CUDA library.
 *
 * Plain, slow, FP64, written from the definitions:
 *   - neighbour sets: j in nbr(i) iff (j,s) != (i,0) and |x_j + s L - x_i|^2 < rc^2
 *     (strict, as in Omega_lambda of Eq. lambda_2_i, Appendix B); every periodic
 *     image s inside the cutoff is enumerated.
 *   - centro-symmetry (LAMMPS definition, Appendix A, Eq. csp_1_i): the N = 12
 *     nearest neighbours, the N/2 smallest |r_a + r_b|^2 over all pairs, summed.
 *   - switching function f_cut, lambda_0 (Eq. lambda_1_i), lambda_min (Eq. lambda_2_i).
 *   - EAM site energy (Eq. energy_eam) with the analytic synthetic functions.
 *   - linear ACE site energy E_i = sum_v c_v B_iv (Eq. energy_ace, linear part)
 *     with the project's radial/angular basis; Gaunt couplings by quadrature.
 *   - forces F_k = -grad_k sum_i w_i E_i at fixed weights (Eq. F_i_d, section 2.3).
 *
 * Compile with -O2 -ffp-contract=off so that no multiply-add is fused.
 * Parallelism (OpenMP) is only over independent atoms; every per-atom sum runs
 * in a fixed serial order, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double lo[3];
  double hi[3];
  int periodic[3];
} orc_box;

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ geometry */

/* Range of image shifts s along dimension d that can bring a displacement d0
 * within rc.  One extra shift on each side; the exact test decides. */
static void image_range(const orc_box* b, int d, double d0, double rc, int* smin, int* smax) {
  if (!b->periodic[d]) {
    *smin = 0;
    *smax = 0;
    return;
  }
  double L = b->hi[d] - b->lo[d];
  *smin = (int)ceil((-rc - d0) / L) - 1;
  *smax = (int)floor((rc - d0) / L) + 1;
}

/* The defining displacement of image (j,s) seen from i: (x_j + s*L) - x_i. */
static void displacement(const orc_box* b, const double* xi, const double* xj, const int* s, double* d) {
  for (int k = 0; k < 3; ++k) {
    double L = b->hi[k] - b->lo[k];
    double shifted = xj[k] + (double)s[k] * L;
    d[k] = shifted - xi[k];
  }
}

static double norm2(const double* d) { return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]; }

/* Brute-force neighbour sets.  Row i holds cnt[i] entries (j, s) ordered by
 * j, then s lexicographically.  Returns the maximum count (may exceed cap, in
 * which case rows are truncated and the caller must retry). */
int orc_neighbors(int n, const double* x, const orc_box* b, double rc, int cap, int* cnt, int* jl, int* sl) {
  double rc2 = rc * rc;
  int maxc = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : maxc)
  for (int i = 0; i < n; ++i) {
    int c = 0;
    for (int j = 0; j < n; ++j) {
      double d0[3];
      for (int k = 0; k < 3; ++k) d0[k] = x[3 * j + k] - x[3 * i + k];
      int lo[3], hi[3];
      for (int k = 0; k < 3; ++k) image_range(b, k, d0[k], rc, &lo[k], &hi[k]);
      int s[3];
      for (s[0] = lo[0]; s[0] <= hi[0]; ++s[0])
        for (s[1] = lo[1]; s[1] <= hi[1]; ++s[1])
          for (s[2] = lo[2]; s[2] <= hi[2]; ++s[2]) {
            if (j == i && s[0] == 0 && s[1] == 0 && s[2] == 0) continue;
            double d[3];
            displacement(b, &x[3 * i], &x[3 * j], s, d);
            if (norm2(d) < rc2) {
              if (c < cap) {
                jl[(size_t)i * cap + c] = j;
                for (int k = 0; k < 3; ++k) sl[((size_t)i * cap + c) * 3 + k] = s[k];
              }
              ++c;
            }
          }
    }
    cnt[i] = c;
    if (c > maxc) maxc = c;
  }
  return maxc;
}

/* Neighbour sets of a subset of atoms (rows for ids[0..m)); same rules. */
int orc_neighbors_of(int n, const double* x, const orc_box* b, double rc, int m, const int* ids, int cap, int* cnt,
                     int* jl, int* sl) {
  double rc2 = rc * rc;
  int maxc = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(max : maxc)
  for (int q = 0; q < m; ++q) {
    int i = ids[q];
    int c = 0;
    for (int j = 0; j < n; ++j) {
      double d0[3];
      for (int k = 0; k < 3; ++k) d0[k] = x[3 * j + k] - x[3 * i + k];
      int lo[3], hi[3];
      for (int k = 0; k < 3; ++k) image_range(b, k, d0[k], rc, &lo[k], &hi[k]);
      int s[3];
      for (s[0] = lo[0]; s[0] <= hi[0]; ++s[0])
        for (s[1] = lo[1]; s[1] <= hi[1]; ++s[1])
          for (s[2] = lo[2]; s[2] <= hi[2]; ++s[2]) {
            if (j == i && s[0] == 0 && s[1] == 0 && s[2] == 0) continue;
            double d[3];
            displacement(b, &x[3 * i], &x[3 * j], s, d);
            if (norm2(d) < rc2) {
              if (c < cap) {
                jl[(size_t)q * cap + c] = j;
                for (int k = 0; k < 3; ++k) sl[((size_t)q * cap + c) * 3 + k] = s[k];
              }
              ++c;
            }
          }
    }
    cnt[q] = c;
    if (c > maxc) maxc = c;
  }
  return maxc;
}

/* ------------------------------------------------------------------ switching function */

/* f_cut of Appendix B.  mode 0: the polynomial exactly as printed,
 * 1 - 1.875x + 1.25x^3 - 0.375x^5 on [0,1].  mode 1: the C2-symmetric reading
 * 0.5*(1 - 1.875y + 1.25y^3 - 0.375y^5) with y = 2x - 1.  Both are 1 for x < 0
 * and 0 for x > 1. */
double orc_fcut(double x, int mode) {
  if (x < 0.0) return 1.0;
  if (x > 1.0) return 0.0;
  double t = x;
  if (mode == 1) t = 2.0 * x - 1.0;
  double t2 = t * t;
  double t3 = t2 * t;
  double t5 = t3 * t2;
  double p = ((1.0 - 1.875 * t) + 1.25 * t3) - 0.375 * t5;
  if (mode == 1) p = 0.5 * p;
  return p;
}

double orc_dfcut(double x, int mode) {
  if (x < 0.0 || x > 1.0) return 0.0;
  double t = (mode == 1) ? 2.0 * x - 1.0 : x;
  double t2 = t * t;
  double t4 = t2 * t2;
  /* d/dt of the polynomial; the chain factor 2 of mode 1 cancels the 0.5 */
  return (-1.875 + 3.75 * t2) - 1.875 * t4;
}

/* ------------------------------------------------------------------ centro-symmetry */

typedef struct {
  double r2;
  int j;
  int s[3];
  double d[3];
} orc_cand;

static int cand_less(const orc_cand* a, const orc_cand* b) {
  if (a->r2 != b->r2) return a->r2 < b->r2;
  if (a->j != b->j) return a->j < b->j;
  for (int k = 0; k < 3; ++k)
    if (a->s[k] != b->s[k]) return a->s[k] < b->s[k];
  return 0;
}

/* CSP_i per the LAMMPS definition (Appendix A) with N = 12, N_buffer = 0.  The
 * candidate set is every image within r_search (a neighbour list built with rc =
 * r_search).  Fewer than 12 candidates gives +inf.  Atoms with changeable[i] == 0
 * get 0. */
void orc_csp(int n, const double* x, const orc_box* b, const int* cnt, const int* jl, const int* sl, int cap,
             const uint8_t* changeable, double* csp) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    if (changeable && !changeable[i]) {
      csp[i] = 0.0;
      continue;
    }
    int c = cnt[i];
    if (c < 12) {
      csp[i] = INFINITY;
      continue;
    }
    orc_cand* cd = (orc_cand*)malloc(sizeof(orc_cand) * (size_t)c);
    for (int q = 0; q < c; ++q) {
      cd[q].j = jl[(size_t)i * cap + q];
      for (int k = 0; k < 3; ++k) cd[q].s[k] = sl[((size_t)i * cap + q) * 3 + k];
      displacement(b, &x[3 * i], &x[3 * cd[q].j], cd[q].s, cd[q].d);
      cd[q].r2 = norm2(cd[q].d);
    }
    /* insertion sort by (r2, j, s) */
    for (int a = 1; a < c; ++a) {
      orc_cand t = cd[a];
      int p = a - 1;
      while (p >= 0 && cand_less(&t, &cd[p])) {
        cd[p + 1] = cd[p];
        --p;
      }
      cd[p + 1] = t;
    }
    double v[66];
    int nv = 0;
    for (int a = 0; a < 12; ++a)
      for (int q = a + 1; q < 12; ++q) {
        double sx = cd[a].d[0] + cd[q].d[0];
        double sy = cd[a].d[1] + cd[q].d[1];
        double sz = cd[a].d[2] + cd[q].d[2];
        v[nv++] = (sx * sx + sy * sy) + sz * sz;
      }
    for (int a = 1; a < 66; ++a) {
      double t = v[a];
      int p = a - 1;
      while (p >= 0 && v[p] > t) {
        v[p + 1] = v[p];
        --p;
      }
      v[p + 1] = t;
    }
    double sum = v[0];
    for (int a = 1; a < 6; ++a) sum = sum + v[a];
    csp[i] = sum;
    free(cd);
  }
}

/* lambda_0 = 1 - f_cut((CSP_hi - CSP_avg)/(CSP_hi - CSP_lo)) (Eq. lambda_1_i with the
 * argument oriented as the paper requires: 0 for atoms computed exactly, 1 for
 * atoms computed fast).  Non-changeable atoms get 1. */
void orc_lambda0(int n, const double* csp_avg, double csp_lo, double csp_hi, int mode, const uint8_t* changeable,
                 double* lam0) {
  for (int i = 0; i < n; ++i) {
    if (changeable && !changeable[i]) {
      lam0[i] = 1.0;
      continue;
    }
    double y = (csp_hi - csp_avg[i]) / (csp_hi - csp_lo);
    lam0[i] = 1.0 - orc_fcut(y, mode);
  }
}

/* lambda_min (Eq. lambda_2_i): start from lambda_0,j and take the minimum over every
 * detected atom i (lambda_0,i < 1) and every image with r_ij < r_hi of
 * 1 - (1 - lambda_0,i) f_cut((r_ij - r_lo)/(r_hi - r_lo)), r_ij measured from i.
 * Non-changeable atoms keep 1.  Brute force over all pairs. */
void orc_lambda_min(int n, const double* x, const orc_box* b, const double* lam0, const uint8_t* changeable,
                    double r_lo, double r_hi, int mode, double* lam_min) {
  double rh2 = r_hi * r_hi;
  double width = r_hi - r_lo;
#pragma omp parallel for schedule(dynamic, 16)
  for (int j = 0; j < n; ++j) {
    if (changeable && !changeable[j]) {
      lam_min[j] = 1.0;
      continue;
    }
    double m = lam0[j];
    for (int i = 0; i < n; ++i) {
      if (!(lam0[i] < 1.0)) continue;
      if (changeable && !changeable[i]) continue;
      double d0[3];
      for (int k = 0; k < 3; ++k) d0[k] = x[3 * j + k] - x[3 * i + k];
      int lo[3], hi[3];
      for (int k = 0; k < 3; ++k) image_range(b, k, d0[k], r_hi, &lo[k], &hi[k]);
      int s[3];
      for (s[0] = lo[0]; s[0] <= hi[0]; ++s[0])
        for (s[1] = lo[1]; s[1] <= hi[1]; ++s[1])
          for (s[2] = lo[2]; s[2] <= hi[2]; ++s[2]) {
            if (j == i && s[0] == 0 && s[1] == 0 && s[2] == 0) continue;
            double d[3];
            displacement(b, &x[3 * i], &x[3 * j], s, d);
            double r2 = norm2(d);
            if (r2 < rh2) {
              double r = sqrt(r2);
              double val = 1.0 - (1.0 - lam0[i]) * orc_fcut((r - r_lo) / width, mode);
              if (val < m) m = val;
            }
          }
    }
    lam_min[j] = m;
  }
}

/* ------------------------------------------------------------------ EAM */

typedef struct {
  double beta, alpha, A, D, rp, r0, rc, h;
} orc_eam_params;

/* psi(x) = x^4/(1+x^4) for x < 0, else 0 */
static double psi(double x) {
  if (x >= 0.0) return 0.0;
  double x4 = x * x * x * x;
  return x4 / (1.0 + x4);
}
static double dpsi(double x) {
  if (x >= 0.0) return 0.0;
  double x3 = x * x * x;
  double den = 1.0 + x3 * x;
  return 4.0 * x3 / (den * den);
}

/* zeta(r) = exp(-beta (r/r0 - 1)) psi((r - rc)/h) */
static void eam_zeta(const orc_eam_params* p, double r, double* z, double* dz) {
  double e = exp(-p->beta * (r / p->r0 - 1.0));
  double u = (r - p->rc) / p->h;
  *z = e * psi(u);
  *dz = (-p->beta / p->r0) * e * psi(u) + e * dpsi(u) / p->h;
}

/* Phi(r) = D [exp(-2 alpha (r - rp)) - 2 exp(-alpha (r - rp))] psi((r - rc)/h) */
static void eam_phi(const orc_eam_params* p, double r, double* f, double* df) {
  double e1 = exp(-p->alpha * (r - p->rp));
  double e2 = exp(-2.0 * p->alpha * (r - p->rp));
  double m = p->D * (e2 - 2.0 * e1);
  double dm = p->D * (-2.0 * p->alpha * e2 + 2.0 * p->alpha * e1);
  double u = (r - p->rc) / p->h;
  *f = m * psi(u);
  *df = dm * psi(u) + m * dpsi(u) / p->h;
}

/* xi(rho) = -A sqrt(rho); rho <= 0 gives 0 and 0 */
static void eam_xi(const orc_eam_params* p, double rho, double* xi, double* dxi) {
  if (rho <= 0.0) {
    *xi = 0.0;
    *dxi = 0.0;
    return;
  }
  double s = sqrt(rho);
  *xi = -p->A * s;
  *dxi = -p->A / (2.0 * s);
}

/* ------------------------------------------------------------------ Mishin EAM2 (Appendix E)
 * Pair:      Phi(r) = (E1 M(r, r01, a1) + E2 M(r, r02, a2) + delta) psi((r - rc)/h)
 *                     - sum_n Theta(rs_n - r) S_n (rs_n - r)^4,
 *            M(r, r0, a) = exp(-2a(r - r0)) - 2 exp(-a(r - r0)), psi(x) = x^4/(1+x^4) for x < 0.
 * Embedding: xi(x) = xi0 + xi2/2 (x-1)^2 + sum_{n=1..4} q_n (x-1)^(n+2)                 (x <= 1)
 *            xi(x) = (xi0 + xi2/2 (x-1)^2 + q1 (x-1)^3 + Q1 (x-1)^4) / (1 + Q2 (x-1)^3)  (x > 1)
 *            plus the fitted offset F0.
 * Density:   zeta(r) = (a exp(-b1 (r - r03)^2) + exp(-b2 (r - r04))) psi((r - rc)/h); the second
 *            exponent is evaluated only when it is above -700 (for the published r04, b2 it
 *            underflows to 0 at every r > 0). */
typedef struct {
  double E1, E2, delta, F0, xi0, xi2, h, q1, q2, q3, q4, Q1, Q2, S1, S2, S3, a, a1, a2, b1, b2, r01, r02, r03, r04,
      rs1, rs2, rs3, rc;
} orc_mishin;

static void morse(double r, double r0, double al, double* m, double* dm) {
  double e1 = exp(-al * (r - r0));
  *m = e1 * e1 - 2.0 * e1;
  *dm = -2.0 * al * e1 * e1 + 2.0 * al * e1;
}

void orc_mishin_pair(const orc_mishin* p, double r, double* phi, double* dphi, double* z, double* dz) {
  double u = (r - p->rc) / p->h;
  double ps = psi(u), dps = dpsi(u) / p->h;
  double m1, dm1, m2, dm2;
  morse(r, p->r01, p->a1, &m1, &dm1);
  morse(r, p->r02, p->a2, &m2, &dm2);
  double core = p->E1 * m1 + p->E2 * m2 + p->delta;
  double dcore = p->E1 * dm1 + p->E2 * dm2;
  double ph = core * ps, dph = dcore * ps + core * dps;
  const double rs[3] = {p->rs1, p->rs2, p->rs3}, S[3] = {p->S1, p->S2, p->S3};
  for (int k = 0; k < 3; ++k)
    if (rs[k] - r >= 0.0) {
      double t = rs[k] - r;
      ph -= S[k] * t * t * t * t;
      dph += 4.0 * S[k] * t * t * t;
    }
  double g = exp(-p->b1 * (r - p->r03) * (r - p->r03));
  double dg = -2.0 * p->b1 * (r - p->r03) * g;
  double arg = -p->b2 * (r - p->r04);
  double e2 = arg > -700.0 ? exp(arg) : 0.0;
  double rho0 = p->a * g + e2, drho0 = p->a * dg - p->b2 * e2;
  *phi = ph;
  *dphi = dph;
  *z = rho0 * ps;
  *dz = drho0 * ps + rho0 * dps;
}

void orc_mishin_embed(const orc_mishin* p, double x, double* xi, double* dxi) {
  double y = x - 1.0, y2 = y * y, y3 = y2 * y;
  if (x <= 1.0) {
    double y4 = y3 * y, y5 = y4 * y, y6 = y5 * y;
    *xi = p->xi0 + 0.5 * p->xi2 * y2 + p->q1 * y3 + p->q2 * y4 + p->q3 * y5 + p->q4 * y6;
    *dxi = p->xi2 * y + 3.0 * p->q1 * y2 + 4.0 * p->q2 * y3 + 5.0 * p->q3 * y4 + 6.0 * p->q4 * y5;
  } else {
    double num = p->xi0 + 0.5 * p->xi2 * y2 + p->q1 * y3 + p->Q1 * y3 * y;
    double dnum = p->xi2 * y + 3.0 * p->q1 * y2 + 4.0 * p->Q1 * y3;
    double den = 1.0 + p->Q2 * y3, dden = 3.0 * p->Q2 * y2;
    *xi = num / den;
    *dxi = (dnum * den - num * dden) / (den * den);
  }
  *xi += p->F0;
}

/* EAM site energies and weighted forces with the Mishin functions; same contract as orc_eam. */
void orc_eam_mishin(int n, const double* x, const orc_box* b, const int* cnt, const int* jl, const int* sl, int cap,
                    const orc_mishin* p, const double* wt, double* e_site, double* f, double* rho_out,
                    double* dxi_out) {
  double* dxi = (double*)malloc(sizeof(double) * (size_t)n);
  double* gp = (double*)calloc((size_t)n * cap * 3, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    double r_sum = 0.0, phi_sum = 0.0;
    for (int q = 0; q < cnt[i]; ++q) {
      int j = jl[(size_t)i * cap + q];
      double d[3];
      displacement(b, &x[3 * i], &x[3 * j], &sl[((size_t)i * cap + q) * 3], d);
      double r = sqrt(norm2(d));
      if (r >= p->rc) continue;
      double ph, dph, z, dz;
      orc_mishin_pair(p, r, &ph, &dph, &z, &dz);
      r_sum += z;
      phi_sum += ph;
    }
    double xi, dx;
    orc_mishin_embed(p, r_sum, &xi, &dx);
    if (rho_out) rho_out[i] = r_sum;
    dxi[i] = dx;
    e_site[i] = xi + 0.5 * phi_sum;
    for (int q = 0; q < cnt[i]; ++q) {
      int j = jl[(size_t)i * cap + q];
      double d[3];
      displacement(b, &x[3 * i], &x[3 * j], &sl[((size_t)i * cap + q) * 3], d);
      double r = sqrt(norm2(d));
      if (r >= p->rc) continue;
      double ph, dph, z, dz;
      orc_mishin_pair(p, r, &ph, &dph, &z, &dz);
      double g = dx * dz + 0.5 * dph;
      for (int k = 0; k < 3; ++k) gp[((size_t)i * cap + q) * 3 + k] = g * d[k] / r;
    }
  }
  for (int k = 0; k < 3 * n; ++k) f[k] = 0.0;
  for (int i = 0; i < n; ++i) {
    double w = wt ? wt[i] : 1.0;
    if (w == 0.0) continue;
    for (int q = 0; q < cnt[i]; ++q) {
      int j = jl[(size_t)i * cap + q];
      for (int k = 0; k < 3; ++k) {
        double g = gp[((size_t)i * cap + q) * 3 + k];
        f[3 * j + k] -= w * g;
        f[3 * i + k] += w * g;
      }
    }
  }
  if (dxi_out) memcpy(dxi_out, dxi, sizeof(double) * (size_t)n);
  free(dxi);
  free(gp);
}

/* zeta, zeta', Phi, Phi' at m distances (the selector features use the pair terms). */
void orc_eam_pair(const orc_eam_params* p, int m, const double* r, double* z, double* dz, double* ph, double* dph) {
  for (int k = 0; k < m; ++k) {
    eam_zeta(p, r[k], &z[k], &dz[k]);
    eam_phi(p, r[k], &ph[k], &dph[k]);
  }
}

/* EAM site energies E_i^f = xi(sum_j zeta) + 1/2 sum_j Phi (Eq. energy_eam) and the
 * weighted force F_k = -grad_k sum_i wt_i E_i^f.  The neighbour list (cap, cnt,
 * jl, sl) may use a radius >= rc; pairs with r >= rc contribute nothing.
 * f is overwritten.  rho and dxi (optional) receive the densities and xi'(rho). */
void orc_eam(int n, const double* x, const orc_box* b, const int* cnt, const int* jl, const int* sl, int cap,
             const orc_eam_params* p, const double* wt, double* e_site, double* f, double* rho_out,
             double* dxi_out) {
  double* rho = (double*)malloc(sizeof(double) * (size_t)n);
  double* dxi = (double*)malloc(sizeof(double) * (size_t)n);
  /* per-pair gradient dE_i/dx_j, stored in the list layout */
  double* gp = (double*)calloc((size_t)n * cap * 3, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    double r_sum = 0.0, phi_sum = 0.0;
    for (int q = 0; q < cnt[i]; ++q) {
      int j = jl[(size_t)i * cap + q];
      double d[3];
      displacement(b, &x[3 * i], &x[3 * j], &sl[((size_t)i * cap + q) * 3], d);
      double r = sqrt(norm2(d));
      if (r >= p->rc) continue;
      double z, dz, ph, dph;
      eam_zeta(p, r, &z, &dz);
      eam_phi(p, r, &ph, &dph);
      r_sum += z;
      phi_sum += ph;
    }
    double xi, dx;
    eam_xi(p, r_sum, &xi, &dx);
    rho[i] = r_sum;
    dxi[i] = dx;
    e_site[i] = xi + 0.5 * phi_sum;
    /* dE_i/dx_j = (xi'(rho_i) zeta'(r) + 1/2 Phi'(r)) * d/r  (d = x_j - x_i) */
    for (int q = 0; q < cnt[i]; ++q) {
      int j = jl[(size_t)i * cap + q];
      double d[3];
      displacement(b, &x[3 * i], &x[3 * j], &sl[((size_t)i * cap + q) * 3], d);
      double r = sqrt(norm2(d));
      if (r >= p->rc) continue;
      double z, dz, ph, dph;
      eam_zeta(p, r, &z, &dz);
      eam_phi(p, r, &ph, &dph);
      double g = dx * dz + 0.5 * dph;
      for (int k = 0; k < 3; ++k) gp[((size_t)i * cap + q) * 3 + k] = g * d[k] / r;
    }
  }
  /* F_k = -sum_i wt_i dE_i/dx_k: dE_i/dx_j = gp_ij, dE_i/dx_i = -sum_j gp_ij (serial) */
  for (int k = 0; k < 3 * n; ++k) f[k] = 0.0;
  for (int i = 0; i < n; ++i) {
    double w = wt ? wt[i] : 1.0;
    if (w == 0.0) continue;
    for (int q = 0; q < cnt[i]; ++q) {
      int j = jl[(size_t)i * cap + q];
      for (int k = 0; k < 3; ++k) {
        double g = gp[((size_t)i * cap + q) * 3 + k];
        f[3 * j + k] -= w * g;
        f[3 * i + k] += w * g;
      }
    }
  }
  if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)n);
  if (dxi_out) memcpy(dxi_out, dxi, sizeof(double) * (size_t)n);
  free(rho);
  free(dxi);
  free(gp);
}

/* ------------------------------------------------------------------ ACE basis */

#define ACE_NMAX 8
#define ACE_LMAX 4
#define ACE_NLM (ACE_NMAX * (ACE_LMAX + 1) * (ACE_LMAX + 1)) /* 200 */
#define NU3_NMAX 3
#define NU3_LMAX 3

typedef struct {
  int nu;
  int n[3];
  int l[3];
} orc_bfunc;

typedef struct {
  double W[ACE_LMAX + 1][ACE_NMAX][ACE_NMAX]; /* [l][n][k] */
  double* c;
  double rc, n0;
  int fcut_mode;
  int nb;
  orc_bfunc* bf;
  /* real Gaunt coefficients for l1,l2,l3 <= 3, by quadrature: G[l1][m1+3][l2][m2+3][l3][m3+3] */
  double G[4][7][4][7][4][7];
  /* power-basis coefficients of Chebyshev T_k */
  double cheb[ACE_NMAX][ACE_NMAX];
  /* power-basis coefficients of the m-th derivative of Legendre P_l, [l][m][power] */
  double legd[ACE_LMAX + 1][ACE_LMAX + 1][ACE_LMAX + 1];
  double ynorm[ACE_LMAX + 1][ACE_LMAX + 1];
} orc_ace;

static double factorial(int k) {
  double r = 1.0;
  for (int i = 2; i <= k; ++i) r *= (double)i;
  return r;
}
static double binom(int a, int b) { return factorial(a) / (factorial(b) * factorial(a - b)); }

/* Real orthonormal spherical harmonic Y_lm and its gradient with respect to the
 * argument u, evaluated as a polynomial in (ux, uy, uz):
 *   Y_lm = c_lm * Re[(ux + i uy)^m] * d^m P_l/dz^m (uz)       m > 0
 *   Y_l0 = c_l0 * P_l(uz)
 *   Y_lm = c_lm * Im[(ux + i uy)^|m|] * d^|m| P_l/dz^|m| (uz)   m < 0
 * c_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) * (sqrt(2) for m != 0).
 * This equals sqrt(2) N P_l^m(cos t) cos(m p) on the unit sphere (no
 * Condon-Shortley phase); Y_1,-1 ~ y, Y_10 ~ z, Y_11 ~ x. */
static void ylm_poly(const orc_ace* a, int l, int m, const double* u, double* y, double* gy) {
  int am = m < 0 ? -m : m;
  /* complex power (ux + i uy)^k for k = am and am - 1 */
  double re = 1.0, im = 0.0, re1 = 1.0, im1 = 0.0;
  for (int k = 0; k < am; ++k) {
    re1 = re;
    im1 = im;
    double nr = re * u[0] - im * u[1];
    double ni = re * u[1] + im * u[0];
    re = nr;
    im = ni;
  }
  /* Q(z) = d^am P_l / dz^am and Q'(z) */
  double q = 0.0, dq = 0.0, zp = 1.0;
  for (int p = 0; p <= l - am; ++p) {
    q += a->legd[l][am][p] * zp;
    zp *= u[2];
  }
  zp = 1.0;
  for (int p = 1; p <= l - am; ++p) {
    dq += (double)p * a->legd[l][am][p] * zp;
    zp *= u[2];
  }
  double c = a->ynorm[l][am];
  double pi_v, dpx, dpy;
  if (m > 0) {
    pi_v = re;
    dpx = (double)am * re1;
    dpy = -(double)am * im1;
  } else if (m < 0) {
    pi_v = im;
    dpx = (double)am * im1;
    dpy = (double)am * re1;
  } else {
    pi_v = 1.0;
    dpx = 0.0;
    dpy = 0.0;
  }
  *y = c * pi_v * q;
  if (gy) {
    gy[0] = c * dpx * q;
    gy[1] = c * dpy * q;
    gy[2] = c * pi_v * dq;
  }
}

/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n. */
static void gauss_legendre(int n, double* xs, double* ws) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    xs[i] = z;
    ws[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* Enumerate the B-functions in the canonical order:
 *   nu=1: n = 0..7                                                  (8)
 *   nu=2: (n1, n2, l), n1 <= n2 <= 7, l = 0..4, lexicographic        (180)
 *   nu=3: (p1, p2, p3), p = 4n + l with n <= 2, l <= 3, p1 <= p2 <= p3,
 *         lexicographic; kept iff |l1 - l2| <= l3 <= l1 + l2, l1+l2+l3 even,
 *         and the coupling sum G A A A is not identically zero.         */
static int ace_enumerate(orc_ace* a, orc_bfunc* out) {
  int nb = 0;
  for (int n = 0; n < ACE_NMAX; ++n) {
    if (out) {
      out[nb].nu = 1;
      out[nb].n[0] = n;
      out[nb].l[0] = 0;
    }
    ++nb;
  }
  for (int n1 = 0; n1 < ACE_NMAX; ++n1)
    for (int n2 = n1; n2 < ACE_NMAX; ++n2)
      for (int l = 0; l <= ACE_LMAX; ++l) {
        if (out) {
          out[nb].nu = 2;
          out[nb].n[0] = n1;
          out[nb].n[1] = n2;
          out[nb].l[0] = l;
          out[nb].l[1] = l;
        }
        ++nb;
      }
  int np = NU3_NMAX * (NU3_LMAX + 1);
  for (int p1 = 0; p1 < np; ++p1)
    for (int p2 = p1; p2 < np; ++p2)
      for (int p3 = p2; p3 < np; ++p3) {
        int l1 = p1 % 4, l2 = p2 % 4, l3 = p3 % 4;
        int dl = l1 > l2 ? l1 - l2 : l2 - l1;
        if (l3 < dl || l3 > l1 + l2) continue;
        if ((l1 + l2 + l3) % 2) continue;
        double mx = 0.0;
        for (int m1 = -l1; m1 <= l1; ++m1)
          for (int m2 = -l2; m2 <= l2; ++m2)
            for (int m3 = -l3; m3 <= l3; ++m3) {
              double g = fabs(a->G[l1][m1 + 3][l2][m2 + 3][l3][m3 + 3]);
              if (g > mx) mx = g;
            }
        if (mx < 1e-12) continue;
        if (out) {
          out[nb].nu = 3;
          out[nb].n[0] = p1 / 4;
          out[nb].n[1] = p2 / 4;
          out[nb].n[2] = p3 / 4;
          out[nb].l[0] = l1;
          out[nb].l[1] = l2;
          out[nb].l[2] = l3;
        }
        ++nb;
      }
  return nb;
}

/* W: [5][8][8] indexed [l][n][k]; c: at least n_basis coefficients. */
orc_ace* orc_ace_create(const double* W, const double* c, int nc, double rc, double n0, int fcut_mode) {
  orc_ace* a = (orc_ace*)calloc(1, sizeof(orc_ace));
  memcpy(a->W, W, sizeof(a->W));
  a->rc = rc;
  a->n0 = n0;
  a->fcut_mode = fcut_mode;
  /* Chebyshev T_k in the power basis: T0 = 1, T1 = t, T_{k+1} = 2 t T_k - T_{k-1} */
  memset(a->cheb, 0, sizeof(a->cheb));
  a->cheb[0][0] = 1.0;
  a->cheb[1][1] = 1.0;
  for (int k = 1; k + 1 < ACE_NMAX; ++k)
    for (int p = 0; p < ACE_NMAX; ++p) {
      double v = -a->cheb[k - 1][p];
      if (p > 0) v += 2.0 * a->cheb[k][p - 1];
      a->cheb[k + 1][p] = v;
    }
  /* Legendre P_l(z) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l) z^(l-2k), and its derivatives */
  memset(a->legd, 0, sizeof(a->legd));
  for (int l = 0; l <= ACE_LMAX; ++l) {
    double pc[ACE_LMAX + 1] = {0};
    for (int k = 0; 2 * k <= l; ++k)
      pc[l - 2 * k] = ((k % 2) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l) / pow(2.0, l);
    for (int m = 0; m <= l; ++m) {
      for (int p = 0; p + m <= l; ++p) a->legd[l][m][p] = pc[p + m] * factorial(p + m) / factorial(p);
      a->ynorm[l][m] = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m)) *
                       (m ? sqrt(2.0) : 1.0);
    }
  }
  /* Real Gaunt coefficients by Gauss-Legendre (cos theta) x trapezoid (phi); exact
   * for the polynomial degrees involved (<= 9). */
  {
    const int NT = 12, NP = 24;
    double xs[12], ws[12];
    gauss_legendre(NT, xs, ws);
    memset(a->G, 0, sizeof(a->G));
    for (int it = 0; it < NT; ++it)
      for (int ip = 0; ip < NP; ++ip) {
        double ph = 2.0 * M_PI * ip / NP;
        double st = sqrt(1.0 - xs[it] * xs[it]);
        double u[3] = {st * cos(ph), st * sin(ph), xs[it]};
        double w = ws[it] * 2.0 * M_PI / NP;
        double Y[4][7];
        for (int l = 0; l <= 3; ++l)
          for (int m = -l; m <= l; ++m) ylm_poly(a, l, m, u, &Y[l][m + 3], NULL);
        for (int l1 = 0; l1 <= 3; ++l1)
          for (int m1 = -l1; m1 <= l1; ++m1)
            for (int l2 = 0; l2 <= 3; ++l2)
              for (int m2 = -l2; m2 <= l2; ++m2)
                for (int l3 = 0; l3 <= 3; ++l3)
                  for (int m3 = -l3; m3 <= l3; ++m3)
                    a->G[l1][m1 + 3][l2][m2 + 3][l3][m3 + 3] += w * Y[l1][m1 + 3] * Y[l2][m2 + 3] * Y[l3][m3 + 3];
      }
  }
  a->nb = ace_enumerate(a, NULL);
  a->bf = (orc_bfunc*)calloc((size_t)a->nb, sizeof(orc_bfunc));
  ace_enumerate(a, a->bf);
  a->c = (double*)calloc((size_t)a->nb, sizeof(double));
  for (int v = 0; v < a->nb && v < nc; ++v) a->c[v] = c[v];
  return a;
}

void orc_ace_destroy(orc_ace* a) {
  if (!a) return;
  free(a->bf);
  free(a->c);
  free(a);
}

int orc_ace_nbasis(const orc_ace* a) { return a->nb; }

/* desc[v*7 + 0..6] = nu, n1, n2, n3, l1, l2, l3 */
void orc_ace_basis_desc(const orc_ace* a, int* desc) {
  for (int v = 0; v < a->nb; ++v) {
    desc[v * 7 + 0] = a->bf[v].nu;
    for (int k = 0; k < 3; ++k) desc[v * 7 + 1 + k] = a->bf[v].n[k];
    for (int k = 0; k < 3; ++k) desc[v * 7 + 4 + k] = a->bf[v].l[k];
  }
}

/* Real Gaunt coefficient table, out[l1][m1+3][l2][m2+3][l3][m3+3] (4*7*4*7*4*7). */
void orc_ace_gaunt(const orc_ace* a, double* out) { memcpy(out, a->G, sizeof(a->G)); }

void orc_ylm(const orc_ace* a, int l, int m, const double* u, double* y, double* gy) { ylm_poly(a, l, m, u, y, gy); }

/* radial g_k(r) = T_k(2r/rc - 1) f_cut(r/rc) and its r-derivative */
static void ace_radial_g(const orc_ace* a, double r, double* g, double* dg) {
  double t = 2.0 * r / a->rc - 1.0;
  double fc = orc_fcut(r / a->rc, a->fcut_mode);
  double dfc = orc_dfcut(r / a->rc, a->fcut_mode) / a->rc;
  for (int k = 0; k < ACE_NMAX; ++k) {
    double tv = 0.0, dtv = 0.0, tp = 1.0;
    for (int p = 0; p < ACE_NMAX; ++p) {
      tv += a->cheb[k][p] * tp;
      tp *= t;
    }
    tp = 1.0;
    for (int p = 1; p < ACE_NMAX; ++p) {
      dtv += (double)p * a->cheb[k][p] * tp;
      tp *= t;
    }
    g[k] = tv * fc;
    dg[k] = dtv * (2.0 / a->rc) * fc + tv * dfc;
  }
}

#define AIDX(n, l, m) ((n) * 25 + (l) * (l) + (l) + (m))

/* A-basis of one atom: A[n][l][m] = (1/N0) sum_j R_nl(r_ij) Y_lm(r_ij / r_ij). */
static void ace_A(const orc_ace* a, const double* x, const orc_box* b, int i, const int* jl, const int* sl, int c,
                  double* A) {
  for (int q = 0; q < ACE_NLM; ++q) A[q] = 0.0;
  for (int q = 0; q < c; ++q) {
    double d[3];
    displacement(b, &x[3 * i], &x[3 * jl[q]], &sl[3 * q], d);
    double r = sqrt(norm2(d));
    if (r >= a->rc) continue;
    double u[3] = {d[0] / r, d[1] / r, d[2] / r};
    double g[ACE_NMAX], dg[ACE_NMAX];
    ace_radial_g(a, r, g, dg);
    for (int l = 0; l <= ACE_LMAX; ++l)
      for (int m = -l; m <= l; ++m) {
        double y;
        ylm_poly(a, l, m, u, &y, NULL);
        for (int n = 0; n < ACE_NMAX; ++n) {
          double R = 0.0;
          for (int k = 0; k < ACE_NMAX; ++k) R += a->W[l][n][k] * g[k];
          A[AIDX(n, l, m)] += R * y / a->n0;
        }
      }
  }
}

/* B-values and energy from A; optionally dE/dA. */
static double ace_B_E(const orc_ace* a, const double* A, double* B, double* dA) {
  double E = 0.0;
  if (dA)
    for (int q = 0; q < ACE_NLM; ++q) dA[q] = 0.0;
  for (int v = 0; v < a->nb; ++v) {
    const orc_bfunc* f = &a->bf[v];
    double cv = a->c[v];
    double bv = 0.0;
    if (f->nu == 1) {
      bv = A[AIDX(f->n[0], 0, 0)];
      if (dA) dA[AIDX(f->n[0], 0, 0)] += cv;
    } else if (f->nu == 2) {
      int l = f->l[0];
      for (int m = -l; m <= l; ++m) {
        double a1 = A[AIDX(f->n[0], l, m)], a2 = A[AIDX(f->n[1], l, m)];
        bv += a1 * a2;
        if (dA) {
          dA[AIDX(f->n[0], l, m)] += cv * a2;
          dA[AIDX(f->n[1], l, m)] += cv * a1;
        }
      }
    } else {
      int l1 = f->l[0], l2 = f->l[1], l3 = f->l[2];
      for (int m1 = -l1; m1 <= l1; ++m1)
        for (int m2 = -l2; m2 <= l2; ++m2)
          for (int m3 = -l3; m3 <= l3; ++m3) {
            double g = a->G[l1][m1 + 3][l2][m2 + 3][l3][m3 + 3];
            double a1 = A[AIDX(f->n[0], l1, m1)], a2 = A[AIDX(f->n[1], l2, m2)], a3 = A[AIDX(f->n[2], l3, m3)];
            bv += g * a1 * a2 * a3;
            if (dA) {
              dA[AIDX(f->n[0], l1, m1)] += cv * g * a2 * a3;
              dA[AIDX(f->n[1], l2, m2)] += cv * g * a1 * a3;
              dA[AIDX(f->n[2], l3, m3)] += cv * g * a1 * a2;
            }
          }
    }
    if (B) B[v] = bv;
    E += cv * bv;
  }
  return E;
}

/* A and B vectors of selected atoms (rows ids[0..m) of the list) */
void orc_ace_basis(const orc_ace* a, int m, const int* ids, const double* x, const orc_box* b, const int* cnt,
                   const int* jl, const int* sl, int cap, double* A_out, double* B_out) {
  for (int q = 0; q < m; ++q) {
    double A[ACE_NLM];
    ace_A(a, x, b, ids[q], &jl[(size_t)q * cap], &sl[(size_t)q * cap * 3], cnt[q], A);
    if (A_out) memcpy(&A_out[(size_t)q * ACE_NLM], A, sizeof(A));
    if (B_out) ace_B_E(a, A, &B_out[(size_t)q * a->nb], NULL);
  }
}

/* ACE site energies E_i^p = sum_v c_v B_iv for atoms with wt[i] != 0 (or all if
 * wt is NULL; 0 elsewhere), and the weighted force F_k = -grad_k sum_i wt_i E_i^p.
 * f is overwritten.  Neighbour rows are the full list (radius >= rc). */
void orc_ace_eval(const orc_ace* a, int n, const double* x, const orc_box* b, const int* cnt, const int* jl,
                  const int* sl, int cap, const double* wt, double* e_site, double* f) {
  double* gp = (double*)calloc((size_t)n * cap * 3, sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
  for (int i = 0; i < n; ++i) {
    if (wt && wt[i] == 0.0) {
      e_site[i] = 0.0;
      continue;
    }
    const int* ji = &jl[(size_t)i * cap];
    const int* si = &sl[(size_t)i * cap * 3];
    double A[ACE_NLM], dA[ACE_NLM];
    ace_A(a, x, b, i, ji, si, cnt[i], A);
    e_site[i] = ace_B_E(a, A, NULL, dA);
    /* dE_i/dx_j = (1/N0) sum_nlm dE/dA_nlm grad_d [R_nl(|d|) Y_lm(d/|d|)] */
    for (int q = 0; q < cnt[i]; ++q) {
      double d[3];
      displacement(b, &x[3 * i], &x[3 * ji[q]], &si[3 * q], d);
      double r = sqrt(norm2(d));
      if (r >= a->rc) continue;
      double u[3] = {d[0] / r, d[1] / r, d[2] / r};
      double g[ACE_NMAX], dg[ACE_NMAX];
      ace_radial_g(a, r, g, dg);
      double acc[3] = {0.0, 0.0, 0.0};
      for (int l = 0; l <= ACE_LMAX; ++l)
        for (int m = -l; m <= l; ++m) {
          double y, gy[3];
          ylm_poly(a, l, m, u, &y, gy);
          double ug = u[0] * gy[0] + u[1] * gy[1] + u[2] * gy[2];
          double gY[3];
          for (int k = 0; k < 3; ++k) gY[k] = (gy[k] - u[k] * ug) / r;
          for (int n2 = 0; n2 < ACE_NMAX; ++n2) {
            double R = 0.0, dR = 0.0;
            for (int k = 0; k < ACE_NMAX; ++k) {
              R += a->W[l][n2][k] * g[k];
              dR += a->W[l][n2][k] * dg[k];
            }
            double wgt = dA[AIDX(n2, l, m)] / a->n0;
            for (int k = 0; k < 3; ++k) acc[k] += wgt * (dR * u[k] * y + R * gY[k]);
          }
        }
      for (int k = 0; k < 3; ++k) gp[((size_t)i * cap + q) * 3 + k] = acc[k];
    }
  }
  for (int k = 0; k < 3 * n; ++k) f[k] = 0.0;
  for (int i = 0; i < n; ++i) {
    double w = wt ? wt[i] : 1.0;
    if (w == 0.0) continue;
    for (int q = 0; q < cnt[i]; ++q) {
      int j = jl[(size_t)i * cap + q];
      for (int k = 0; k < 3; ++k) {
        double g = gp[((size_t)i * cap + q) * 3 + k];
        f[3 * j + k] -= w * g;
        f[3 * i + k] += w * g;
      }
    }
  }
  free(gp);
}
