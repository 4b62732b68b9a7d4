// Precision classification (Appendix A and B): centro-symmetry parameter,
// moving averages, lambda_0, lambda_min spread, minimum-step hysteresis and the
// compacted precise-atom work queue.  Every value that decides a set is computed
// in FP64 with explicit round-to-nearest operations in the order of the
// definitions, so the detected and precise sets are reproducible bit for bit.
// FP32 is used only to pick candidates, with a guard band and an exact fallback.
#include "ap_internal.cuh"

namespace ap {

namespace {

constexpr float kBand = 1e-3f;     // FP32 guard band (A^2) on squared lengths
constexpr int kNN = 12;            // N nearest neighbours of FCC (N_buffer = 0)
constexpr int kHalf = kNN / 2;

__device__ inline const SysInfo& sys_of(const SysInfo* sys, const int* atom_sys, int i) {
  return sys[atom_sys ? atom_sys[i] : 0];
}
__device__ inline int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// f_cut of Appendix B in FP64 with the oracle's operation order.
__device__ inline double fcut_exact(double x, int mode) {
  if (x < 0.0) return 1.0;
  if (x > 1.0) return 0.0;
  double t = x;
  if (mode == 1) t = __dsub_rn(__dmul_rn(2.0, x), 1.0);
  double t2 = __dmul_rn(t, t);
  double t3 = __dmul_rn(t2, t);
  double t5 = __dmul_rn(t3, t2);
  double p = __dsub_rn(__dadd_rn(__dsub_rn(1.0, __dmul_rn(1.875, t)), __dmul_rn(1.25, t3)), __dmul_rn(0.375, t5));
  if (mode == 1) p = __dmul_rn(0.5, p);
  return p;
}

// f_cut in FP32, used only to screen candidates.
__device__ inline float fcut_f(float x, int mode) {
  if (x < 0.f) return 1.f;
  if (x > 1.f) return 0.f;
  const float t = mode == 1 ? 2.f * x - 1.f : x;
  const float t2 = t * t;
  const float p = 1.f - 1.875f * t + 1.25f * t2 * t - 0.375f * t2 * t2 * t;
  return mode == 1 ? 0.5f * p : p;
}

// Cell offset k of a row entry.
__device__ inline void entry_offset(const int* off, size_t e, const SysInfo& S, int wi, int wj, int k[3]) {
  if (off) {
    int p = off[e];
    k[0] = off_x(p);
    k[1] = off_y(p);
    k[2] = off_z(p);
  } else {
    k[0] = wrap_off(cell_x(wj) - cell_x(wi), S.nc[0], S.periodic[0]);
    k[1] = wrap_off(cell_y(wj) - cell_y(wi), S.nc[1], S.periodic[1]);
    k[2] = wrap_off(cell_z(wj) - cell_z(wi), S.nc[2], S.periodic[2]);
  }
}

// Exact displacement (x_j + S L) - x_i for a row entry with cell offset k.
__device__ inline void exact_disp(const double* __restrict__ x, const SysInfo& S, int i, int j, const int4& ci,
                                  const int4& cj, const int k[3], double d[3]) {
  int cu_i[3] = {ci.x, ci.y, ci.z}, cu_j[3] = {cj.x, cj.y, cj.z};
  for (int a = 0; a < 3; ++a) {
    // whole periods between the pair's cell offset and its unwrapped cells (the integer
    // division only where they differ)
    const int t = k[a] - (cu_j[a] - cu_i[a]);
    const int sd = (S.periodic[a] && t != 0) ? t / S.nc[a] : 0;
    // x_j + 0 L is x_j exactly: the FP64 multiply-add (slow on this GPU) only for images
    double shifted = sd == 0 ? x[3 * j + a] : __dadd_rn(x[3 * j + a], __dmul_rn((double)sd, S.L[a]));
    d[a] = __dsub_rn(shifted, x[3 * i + a]);
  }
}

__device__ inline double norm2_exact(const double d[3]) {
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

// Candidate order (r^2, j, s) of the definition.
__device__ inline bool cand_less(double ra, int ja, const int* sa, double rb, int jb, const int* sb) {
  if (ra != rb) return ra < rb;
  if (ja != jb) return ja < jb;
  for (int a = 0; a < 3; ++a)
    if (sa[a] != sb[a]) return sa[a] < sb[a];
  return false;
}

__device__ inline void image_of(const SysInfo& S, const int4& ci, const int4& cj, const int k[3], int s[3]) {
  int cu_i[3] = {ci.x, ci.y, ci.z}, cu_j[3] = {cj.x, cj.y, cj.z};
  for (int a = 0; a < 3; ++a) {
    const int t = k[a] - (cu_j[a] - cu_i[a]);
    s[a] = (S.periodic[a] && t != 0) ? t / S.nc[a] : 0;
  }
}

// Row position q of atom i's entry -> exact FP64 displacement.
__device__ inline void exact_entry(const double* __restrict__ x, const SysInfo& S, int i, const int4& ci,
                                   const int* __restrict__ nbr, const int* __restrict__ off,
                                   const int4* __restrict__ cunw, size_t row, int q, double d[3], int& j,
                                   int s[3]) {
  j = nbr[row + q];
  const int4 cj = cunw[j];
  int k[3];
  entry_offset(off, row + q, S, ci.w, cj.w, k);
  exact_disp(x, S, i, j, ci, cj, k, d);
  image_of(S, ci, cj, k, s);
}

// (r2, j, s) ordering of two row entries with equal or different exact r2.
__device__ inline bool entry_less(const double* __restrict__ x, const SysInfo& S, int i, const int4& ci,
                                  const int* __restrict__ nbr, const int* __restrict__ off,
                                  const int4* __restrict__ cunw, size_t row, double ra, int qa, double rb, int qb) {
  if (ra != rb) return ra < rb;
  if (qb < 0) return true;
  double d[3];
  int ja, jb, sa[3], sb[3];
  exact_entry(x, S, i, ci, nbr, off, cunw, row, qa, d, ja, sa);
  exact_entry(x, S, i, ci, nbr, off, cunw, row, qb, d, jb, sb);
  return cand_less(ra, ja, sa, rb, jb, sb);
}

// ------------------------------------------------------------------ CSP
#ifndef AP_CSP_PREFETCH
#define AP_CSP_PREFETCH 1   // software-pipelined row walk in the CSP selection (compile-time tuning)
#endif

// One thread per atom.  All selection arrays are indexed with compile-time
// indices (fully unrolled insertion), so they live in registers.
// FAST: every atom, FP32 selections only; an atom whose selection the FP32 values
// cannot decide (an r_search band hit, an ambiguous 12/13 or 6/7 boundary) is
// appended to `slow`.  !FAST: the atoms of `slow`, with the exact FP64 selections.
// CSP of atom i (128-thread blocks: the shared arrays are indexed by threadIdx.x).
// nin (FAST, rows built at these positions, else null): the row's first nin[i] entries
// are the ones inside r_c^2 = rpf2 at the build (FP32), the rest lie beyond it.  When the
// 13th smallest r^2 of that part lies more than two guard bands inside rpf2, no skin
// entry can enter the 13 nearest or come within a band of the 12/13 boundary, and the
// skin part is skipped; otherwise it is walked too.
template <bool FAST>
__device__ __forceinline__ void csp_atom(int i, const double* __restrict__ x, const uint8_t* __restrict__ ch,
                                         const SysInfo* __restrict__ sys, const int* __restrict__ atom_sys,
                                         const float4* __restrict__ s32, const int4* __restrict__ cunw,
                                         const int* __restrict__ nbr, const int* __restrict__ off,
                                         const int* __restrict__ cnt, int cap, float rsf2, double rs2,
                                         double* __restrict__ csp, int* __restrict__ slow, int* __restrict__ n_slow,
                                         const int* __restrict__ nin = nullptr, float rpf2 = 0.f,
                                         float stale2 = 0.f, int* __restrict__ n_stale = nullptr) {
  static_assert(kNN <= 255, "neighbour slots are packed in 8 bits");
  if (ch && !ch[i]) {
    csp[i] = 0.0;
    return;
  }
  const SysInfo& S = sys_of(sys, atom_sys, i);
  const float4 si = s32[i];
  const int4 ci = cunw[i];
  const int c = cnt[i];
  const size_t row = (size_t)i * cap;

  // 1. the 13 smallest FP32 r^2 among candidates inside r_search
  float tr[kNN + 1];
  int tq[kNN + 1];
#pragma unroll
  for (int a = 0; a <= kNN; ++a) {
    tr[a] = INFINITY;
    tq[a] = -1;
  }
  int n_in = 0;
  int q_end = (FAST && nin) ? nin[i] : c;
#if AP_CSP_PREFETCH
  // loads run ahead of the selection: the next entry's shadow and the entry after it
  int j_a = c > 0 ? nbr[row] : 0;
  float4 s_a = s32[j_a];
  int j_b = c > 1 ? nbr[row + 1] : 0;
#endif
  for (int q = 0; q < c; ++q) {
    if (q == q_end) {   // end of the in-range part (FAST with nin only)
      if (tr[kNN] + 2.f * kBand < rpf2) break;
      q_end = c;
    }
#if AP_CSP_PREFETCH
    const int j = j_a;
    const float4 sj = s_a;
    j_a = j_b;
    if (q + 1 < c) s_a = s32[j_a];
    if (q + 2 < c) j_b = nbr[row + q + 2];
#else
    const int j = nbr[row + q];
    const float4 sj = s32[j];
#endif
    int k[3];
    entry_offset(off, row + q, S, ci.w, __float_as_int(sj.w), k);
    const float dx = (float)k[0] * S.hf[0] + sj.x - si.x;
    const float dy = (float)k[1] * S.hf[1] + sj.y - si.y;
    const float dz = (float)k[2] * S.hf[2] + sj.z - si.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (r2 > rsf2 + kBand) continue;
    if (r2 >= rsf2 - kBand) {
      if constexpr (FAST) {
        slow[atomicAdd(n_slow, 1)] = i;
        return;
      }
      double d[3];
      exact_disp(x, S, i, j, ci, cunw[j], k, d);
      if (!(norm2_exact(d) < rs2)) continue;
    }
    ++n_in;
    if (r2 < tr[kNN]) {
      tr[kNN] = r2;
      tq[kNN] = q;
#pragma unroll
      for (int p = kNN; p > 0; --p) {
        if (tr[p] < tr[p - 1]) {
          const float t = tr[p];
          tr[p] = tr[p - 1];
          tr[p - 1] = t;
          const int u = tq[p];
          tq[p] = tq[p - 1];
          tq[p - 1] = u;
        }
      }
    }
  }
  // Rows older than the positions (stale2 > 0): every atom outside the row lies beyond
  // r_search - 2 m (m the largest displacement since the build), stale2 = that radius
  // squared.  The row's selection is exact when 12 candidates lie inside it with a
  // guard band; otherwise (a nearly isolated atom) the atom is counted and the caller
  // rebuilds the rows and computes the CSP again.
  if (stale2 > 0.f && !(n_in >= kNN && tr[kNN - 1] + 2.f * kBand < stale2)) atomicAdd(n_stale, 1);
  if (n_in < kNN) {
    csp[i] = INFINITY;
    return;
  }
  // 2. exact (r2, j, s) selection when the 12/13 boundary lies within the guard band
  if (n_in > kNN && tr[kNN] - tr[kNN - 1] <= 2.f * kBand) {
    if constexpr (FAST) {
      slow[atomicAdd(n_slow, 1)] = i;
      return;
    }
    double br[kNN];
    int bq[kNN];
#pragma unroll
    for (int a = 0; a < kNN; ++a) {
      br[a] = INFINITY;
      bq[a] = -1;
    }
    for (int q = 0; q < c; ++q) {
      double d[3];
      int j, s[3];
      exact_entry(x, S, i, ci, nbr, off, cunw, row, q, d, j, s);
      const double r2 = norm2_exact(d);
      if (!(r2 < rs2)) continue;
      if (!entry_less(x, S, i, ci, nbr, off, cunw, row, r2, q, br[kNN - 1], bq[kNN - 1])) continue;
      br[kNN - 1] = r2;
      bq[kNN - 1] = q;
#pragma unroll
      for (int p = kNN - 1; p > 0; --p) {
        if (entry_less(x, S, i, ci, nbr, off, cunw, row, br[p], bq[p], br[p - 1], bq[p - 1])) {
          const double t = br[p];
          br[p] = br[p - 1];
          br[p - 1] = t;
          const int u = bq[p];
          bq[p] = bq[p - 1];
          bq[p - 1] = u;
        }
      }
    }
#pragma unroll
    for (int a = 0; a < kNN; ++a) tq[a] = bq[a];
  }
  // 3. FP32 vectors of the 12 and the 7 smallest pair values |r_a + r_b|^2.  The 12
  // vectors and row positions live in shared memory, component-major (thread index
  // fastest, conflict-free), not in registers.
  __shared__ float s_v[3][kNN][128];
  __shared__ int s_tq[kNN][128];
  const int tx = threadIdx.x;
#pragma unroll
  for (int a = 0; a < kNN; ++a) {
    const int q = tq[a];
    s_tq[a][tx] = q;
    const int j = nbr[row + q];
    const float4 sj = s32[j];
    int k[3];
    entry_offset(off, row + q, S, ci.w, __float_as_int(sj.w), k);
    s_v[0][a][tx] = (float)k[0] * S.hf[0] + sj.x - si.x;
    s_v[1][a][tx] = (float)k[1] * S.hf[1] + sj.y - si.y;
    s_v[2][a][tx] = (float)k[2] * S.hf[2] + sj.z - si.z;
  }
  float pv[kHalf + 1];
  int pc[kHalf + 1];   // neighbour slots a | b << 8
#pragma unroll
  for (int a = 0; a <= kHalf; ++a) {
    pv[a] = INFINITY;
    pc[a] = 0;
  }
#pragma unroll
  for (int a = 0; a < kNN; ++a) {
    const float ax = s_v[0][a][tx], ay = s_v[1][a][tx], az = s_v[2][a][tx];
#pragma unroll
    for (int b = a + 1; b < kNN; ++b) {
      const float sx = ax + s_v[0][b][tx], sy = ay + s_v[1][b][tx], sz = az + s_v[2][b][tx];
      const float v = sx * sx + sy * sy + sz * sz;
      if (v < pv[kHalf]) {
        pv[kHalf] = v;
        pc[kHalf] = a | (b << 8);
#pragma unroll
        for (int p = kHalf; p > 0; --p) {
          if (pv[p] < pv[p - 1]) {
            const float t = pv[p];
            pv[p] = pv[p - 1];
            pv[p - 1] = t;
            const int u = pc[p];
            pc[p] = pc[p - 1];
            pc[p - 1] = u;
          }
        }
      }
    }
  }
  // 4. exact values of the six smallest pairs (all 66 in FP64 if the 6/7 boundary is ambiguous)
  double chosen[kHalf];
  if (pv[kHalf] - pv[kHalf - 1] > 2.f * kBand) {
#pragma unroll
    for (int t = 0; t < kHalf; ++t) {
      double da[3], db[3];
      int ja, jb, sa[3], sb[3];
      exact_entry(x, S, i, ci, nbr, off, cunw, row, s_tq[pc[t] & 0xff][tx], da, ja, sa);
      exact_entry(x, S, i, ci, nbr, off, cunw, row, s_tq[pc[t] >> 8][tx], db, jb, sb);
      const double s3[3] = {__dadd_rn(da[0], db[0]), __dadd_rn(da[1], db[1]), __dadd_rn(da[2], db[2])};
      chosen[t] = norm2_exact(s3);
    }
  } else {
    if constexpr (FAST) {
      slow[atomicAdd(n_slow, 1)] = i;
      return;
    }
#pragma unroll
    for (int t = 0; t < kHalf; ++t) chosen[t] = INFINITY;
    double ex[kNN][3];
#pragma unroll
    for (int a = 0; a < kNN; ++a) {
      int j, s[3];
      exact_entry(x, S, i, ci, nbr, off, cunw, row, s_tq[a][tx], ex[a], j, s);
    }
#pragma unroll
    for (int a = 0; a < kNN; ++a)
#pragma unroll
      for (int b = a + 1; b < kNN; ++b) {
        const double s3[3] = {__dadd_rn(ex[a][0], ex[b][0]), __dadd_rn(ex[a][1], ex[b][1]),
                              __dadd_rn(ex[a][2], ex[b][2])};
        const double v = norm2_exact(s3);
        if (v < chosen[kHalf - 1]) {
          chosen[kHalf - 1] = v;
#pragma unroll
          for (int p = kHalf - 1; p > 0; --p) {
            if (chosen[p] < chosen[p - 1]) {
              const double t = chosen[p];
              chosen[p] = chosen[p - 1];
              chosen[p - 1] = t;
            }
          }
        }
      }
  }
  // 5. ascending sum of the six values
#pragma unroll
  for (int a = 1; a < kHalf; ++a)
#pragma unroll
    for (int p = a; p > 0; --p)
      if (chosen[p] < chosen[p - 1]) {
        const double t = chosen[p];
        chosen[p] = chosen[p - 1];
        chosen[p - 1] = t;
      }
  double sum = chosen[0];
#pragma unroll
  for (int a = 1; a < kHalf; ++a) sum = __dadd_rn(sum, chosen[a]);
  csp[i] = sum;
}

__global__ void __launch_bounds__(128) k_csp(int n, const double* __restrict__ x, const uint8_t* __restrict__ ch,
                                                const SysInfo* __restrict__ sys, const int* __restrict__ atom_sys,
                                                const float4* __restrict__ s32, const int4* __restrict__ cunw,
                                                const int* __restrict__ nbr, const int* __restrict__ off,
                                                const int* __restrict__ cnt, int cap, float rsf2, double rs2,
                                                double* __restrict__ csp, int* __restrict__ slow,
                                                int* __restrict__ n_slow, const int* __restrict__ nin, float rpf2,
                                                float stale2, int* __restrict__ n_stale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n)
    csp_atom<true>(i, x, ch, sys, atom_sys, s32, cunw, nbr, off, cnt, cap, rsf2, rs2, csp, slow, n_slow, nin, rpf2,
                   stale2, n_stale);
}

__global__ void __launch_bounds__(128) k_csp_exact(const double* __restrict__ x, const uint8_t* __restrict__ ch,
                                                   const SysInfo* __restrict__ sys, const int* __restrict__ atom_sys,
                                                   const float4* __restrict__ s32, const int4* __restrict__ cunw,
                                                   const int* __restrict__ nbr, const int* __restrict__ off,
                                                   const int* __restrict__ cnt, int cap, float rsf2, double rs2,
                                                   double* __restrict__ csp, const int* __restrict__ slow,
                                                   const int* __restrict__ n_slow, float stale2,
                                                   int* __restrict__ n_stale) {
  const int m = *n_slow;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x)
    csp_atom<false>(slow[t], x, ch, sys, atom_sys, s32, cunw, nbr, off, cnt, cap, rsf2, rs2, csp, nullptr, nullptr,
                    nullptr, 0.f, stale2, n_stale);
}

// Canonical moving average over a ring buffer [ns][n]: oldest -> newest, then / ns.
__device__ inline double ring_mean(const double* __restrict__ hist, int ns, int newest, size_t n, int i) {
  int q0 = (newest + 1) % ns;
  double s = hist[(size_t)q0 * n + i];
  for (int q = 1; q < ns; ++q) s = __dadd_rn(s, hist[(size_t)((newest + 1 + q) % ns) * n + i]);
  return __ddiv_rn(s, (double)ns);
}

// Push CSP, average, lambda_0 (Eq. lambda_1_i), detected flag, lambda_min init.
__global__ void k_lambda0(int n, const uint8_t* __restrict__ ch, const double* __restrict__ csp,
                          double* __restrict__ hist, int ns, int pos, int fill, double csp_lo, double csp_hi,
                          int mode, double* __restrict__ csp_avg, double* __restrict__ lam0,
                          double* __restrict__ lam_min, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double c = csp[i];
  if (fill) {
    for (int q = 0; q < ns; ++q) hist[(size_t)q * n + i] = c;
  } else {
    hist[(size_t)pos * n + i] = c;
  }
  double avg = ring_mean(hist, ns, pos, (size_t)n, i);
  csp_avg[i] = avg;
  bool changeable = !ch || ch[i];
  double l0 = 1.0;
  if (changeable) {
    double y = __ddiv_rn(__dsub_rn(csp_hi, avg), __dsub_rn(csp_hi, csp_lo));
    l0 = __dsub_rn(1.0, fcut_exact(y, mode));
  }
  lam0[i] = l0;
  lam_min[i] = changeable ? l0 : 1.0;
  flag[i] = (changeable && l0 < 1.0) ? 1 : 0;
}

__global__ void k_compact(int n, const int* __restrict__ flag, const int* __restrict__ scan, int* __restrict__ out,
                          int* __restrict__ count32, long long* __restrict__ count64) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) out[scan[i]] = i;
  if (i == 0) {
    int tot = scan[n];
    if (count32) *count32 = tot;
    if (count64) *count64 = tot;
  }
}

// lambda_min spread (Eq. lambda_2_i): one warp per detected atom i scans the cells
// within r_hi; for every image j with r_ij < r_hi it lowers lambda_min,j to
// 1 - (1 - lambda_0,i) f_cut((r_ij - r_lo)/(r_hi - r_lo)) by a 64-bit atomicMin on
// the bit pattern (order-free and exact for non-negative doubles).
// The warp takes the stencil cells 32 at a time; the cells that can reach r_hi form,
// through a warp scan of their atom counts, one stream of candidate atoms that the
// lanes share out (lane k takes candidates k, k + 32, ...; its cell is found by a
// binary search over the 32 prefix sums), so lanes stay busy whatever the cells hold.
constexpr int kSpreadWarps = 8;

// The exact value 1 - (1 - lambda_0,i) f_cut((r_ij - r_lo)/(r_hi - r_lo)) of pair (i, j),
// j in the stencil cell of periodic image img relative to i's wrapped cell cw_i; false if
// r_ij >= r_hi.  Image relative to the input positions: s = img + nwrap_i - nwrap_j.
__device__ inline bool spread_value(const double* __restrict__ x, const SysInfo& S, int i, int j, const int4& ci,
                                    const int4& cj, const int img[3], double rh2, double r_lo, double width,
                                    double one_minus, int mode, double& v) {
  const int cwi[3] = {cell_x(ci.w), cell_y(ci.w), cell_z(ci.w)};
  const int cwj[3] = {cell_x(cj.w), cell_y(cj.w), cell_z(cj.w)};
  const int cu_i[3] = {ci.x, ci.y, ci.z}, cu_j[3] = {cj.x, cj.y, cj.z};
  double d[3];
  for (int q = 0; q < 3; ++q) {
    int sd = 0;
    if (S.periodic[q]) sd = img[q] + (cu_i[q] - cwi[q]) / S.nc[q] - (cu_j[q] - cwj[q]) / S.nc[q];
    const double shifted = sd == 0 ? x[3 * j + q] : __dadd_rn(x[3 * j + q], __dmul_rn((double)sd, S.L[q]));
    d[q] = __dsub_rn(shifted, x[3 * i + q]);
  }
  const double r2 = norm2_exact(d);
  if (!(r2 < rh2)) return false;
  const double r = __dsqrt_rn(r2);
  const double f = fcut_exact(__ddiv_rn(__dsub_rn(r, r_lo), width), mode);
  v = __dsub_rn(1.0, __dmul_rn(one_minus, f));
  return true;
}
#ifndef AP_SPREAD_UNROLL
#define AP_SPREAD_UNROLL 1   // unroll depth of the per-lane candidate loop (compile-time tuning)
#endif
constexpr int kSpreadUnroll = AP_SPREAD_UNROLL;
#ifndef AP_SPREAD_QUEUE
#define AP_SPREAD_QUEUE 1   // walk only the cells that can reach r_hi, 32 at a time (compile-time tuning)
#endif

// Two passes over the same candidates, since FP64 is slow on this GPU.  PHASE 0 (FP32): a
// pair surely inside r_lo has f_cut = 1, so its exact value 1 - (1 - lambda_0,i) needs no
// distance and goes straight into lambda_min,j; vmin_f[j] = the smallest FP32 estimate
// (error < 1e-5) over the pairs surely inside r_hi.  PHASE 1: the exact value of the other
// pairs only where it can set the final minimum: the estimate can go below the current
// lambda_min,j and, for a pair surely inside r_hi, lies within 1e-4 of vmin_f[j] (a pair in
// the guard band around r_hi is always evaluated).  Without the first pass every new
// running minimum, and every pair inside r_lo (they tie), took an exact value.
template <int PHASE>
__global__ void __launch_bounds__(kSpreadWarps * 32) k_spread(
    const int* __restrict__ det, const int* __restrict__ n_det, const double* __restrict__ x,
    const uint8_t* __restrict__ ch, const SysInfo* __restrict__ sys, const int* __restrict__ atom_sys,
    const float4* __restrict__ s32, const int4* __restrict__ cunw, const int* __restrict__ cstart,
    const int* __restrict__ catoms, const double* __restrict__ lam0, double r_lo, double r_hi, int mode, int sx,
    int sy, int sz, double* __restrict__ lam_min, float margin, float* __restrict__ vmin_f,
    int* __restrict__ det1, int* __restrict__ n_det1) {
  // per warp: inclusive prefix of candidate counts, first catoms slot, stencil offset
  __shared__ int s_pre[kSpreadWarps][32], s_beg[kSpreadWarps][32], s_t[kSpreadWarps][32], s_img[kSpreadWarps][32];
  __shared__ int4 s_q[kSpreadWarps][64];   // per warp: queued cells (first slot, count, stencil index, image)
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int m = *n_det;
  const double rh2 = __dmul_rn(r_hi, r_hi);
  const float rhf2 = (float)rh2;
  const float rlo2f = (float)__dmul_rn(r_lo, r_lo);
  // cells older than the positions (atoms up to `margin` from their cells): prune beyond r_hi + margin
  const float rprune = (float)r_hi + margin, prune2 = rprune * rprune;
  const double width = __dsub_rn(r_hi, r_lo);
  const float r_lo_f = (float)r_lo, inv_w_f = (float)(1.0 / width);
  const int wx = 2 * sx + 1, wy = 2 * sy + 1, wz = 2 * sz + 1;
  const int ncell = wx * wy * wz;
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < m; w += warps) {
    const int i = det[w];
    const SysInfo& S = sys_of(sys, atom_sys, i);
    const float4 si = s32[i];
    const int4 ci = cunw[i];
    const double one_minus = __dsub_rn(1.0, lam0[i]);
    const float one_minus_f = (float)one_minus;
    const double v_in = __dsub_rn(1.0, __dmul_rn(one_minus, 1.0));   // the value of a pair inside r_lo
    bool need = false;   // PHASE 0: a pair outside r_lo that can still go below lambda_min,j
    const int cw[3] = {cell_x(ci.w), cell_y(ci.w), cell_z(ci.w)};
    // the scan of a batch of cells' atom counts and the stream of their candidates
    auto walk = [&](int cnt, int beg, int t, int imgp) {
      int pre = cnt;   // inclusive warp scan of the counts
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
      }
      const int total = __shfl_sync(0xffffffffu, pre, 31);
      s_pre[wib][lane] = pre;
      s_beg[wib][lane] = beg;
      s_t[wib][lane] = t;
      s_img[wib][lane] = imgp;
      __syncwarp();
#if AP_SPREAD_UNROLL > 1
#pragma unroll kSpreadUnroll
#endif
      for (int k = lane; k < total; k += 32) {
        // cell of candidate k: the first c with s_pre[c] > k
        int lo = 0, hi = 31;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (s_pre[wib][mid] > k) hi = mid;
          else lo = mid + 1;
        }
        const int c = lo;
        const int a = s_beg[wib][c] + k - (c ? s_pre[wib][c - 1] : 0);
        const int tt = s_t[wib][c], ip = s_img[wib][c];
        const int dx = tt % wx - sx, dy = (tt / wx) % wy - sy, dz = tt / (wx * wy) - sz;
        const int j = catoms[a];
        if (j == i && dx == 0 && dy == 0 && dz == 0) continue;
        if (ch && !ch[j]) continue;
        const float ox = (float)dx * S.hf[0] - si.x;
        const float oy = (float)dy * S.hf[1] - si.y;
        const float oz = (float)dz * S.hf[2] - si.z;
        const float4 sj = s32[j];
        const float ddx = ox + sj.x, ddy = oy + sj.y, ddz = oz + sj.z;
        const float r2f = ddx * ddx + ddy * ddy + ddz * ddz;
        if (r2f > rhf2 + kBand) continue;
        // FP32 estimate of the candidate value (error < 1e-5)
        const float vf = fmaxf(0.f, 1.f - one_minus_f * fcut_f((sqrtf(r2f) - r_lo_f) * inv_w_f, mode));
        const bool inside = r2f < rhf2 - kBand;
        if constexpr (PHASE == 0) {
          // a pair that cannot go below the current lambda_min,j (which only decreases) is never the minimum
          if ((double)vf - 1e-4 >= __ldcg(&lam_min[j])) continue;
          if (r2f < rlo2f - kBand) {
            // surely inside r_lo: f_cut = 1, and the exact value 1 - (1 - lambda_0,i) needs no distance
            if (v_in < __ldcg(&lam_min[j]))
              atomicMin((unsigned long long*)&lam_min[j], (unsigned long long)__double_as_longlong(v_in));
            if (vf < __ldcg(&vmin_f[j])) atomicMin((unsigned int*)&vmin_f[j], __float_as_uint(vf));
            continue;
          }
          need = true;   // the second pass may take this pair's exact value
          if (inside && vf < __ldcg(&vmin_f[j])) atomicMin((unsigned int*)&vmin_f[j], __float_as_uint(vf));
          continue;
        }
        if (r2f < rlo2f - kBand) continue;   // applied by the first pass
        // if even its lower bound cannot go below the current lambda_min,j (which only
        // decreases), or a surely-inside pair's estimate lies above the smallest one by
        // more than twice the error, the exact value cannot be the final minimum
        if ((double)vf - 1e-4 >= __ldcg(&lam_min[j])) continue;
        if (inside && vf > __ldcg(&vmin_f[j]) + 1e-4f) continue;
        const int img[3] = {off_x(ip), off_y(ip), off_z(ip)};
        double v;
        if (!spread_value(x, S, i, j, ci, cunw[j], img, rh2, r_lo, width, one_minus, mode, v)) continue;
        atomicMin((unsigned long long*)&lam_min[j], (unsigned long long)__double_as_longlong(v));
      }
      __syncwarp();
    };
    int queued = 0;
    for (int t0 = 0; t0 < ncell; t0 += 32) {
      // this lane's cell of the chunk: kept if it exists and can reach r_hi
      const int t = t0 + lane;
      int cnt = 0, beg = 0, imgp = 0;
      if (t < ncell) {
        const int dx = t % wx - sx, dy = (t / wx) % wy - sy, dz = t / (wx * wy) - sz;
        int tc[3] = {cw[0] + dx, cw[1] + dy, cw[2] + dz};
        int img[3] = {0, 0, 0};
        bool skip = false;
        for (int a = 0; a < 3; ++a) {
          if (S.periodic[a]) {
            img[a] = floor_div(tc[a], S.nc[a]);
            tc[a] -= img[a] * S.nc[a];
          } else if (tc[a] < 0 || tc[a] >= S.nc[a]) {
            skip = true;
          }
        }
        if (!skip) {
          const float gx = fmaxf(0.f, fmaxf((float)dx * S.hf[0] - si.x, si.x - (float)(dx + 1) * S.hf[0]));
          const float gy = fmaxf(0.f, fmaxf((float)dy * S.hf[1] - si.y, si.y - (float)(dy + 1) * S.hf[1]));
          const float gz = fmaxf(0.f, fmaxf((float)dz * S.hf[2] - si.z, si.z - (float)(dz + 1) * S.hf[2]));
          if (gx * gx + gy * gy + gz * gz <= prune2 + kBand) {
            const int cid = S.cell_base + (tc[2] * S.nc[1] + tc[1]) * S.nc[0] + tc[0];
            beg = cstart[cid];
            cnt = cstart[cid + 1] - beg;
            // periodic image of the cell, 8 bits per component biased by 128
            imgp = pack_off(img[0], img[1], img[2]);
          }
        }
      }
#if AP_SPREAD_QUEUE
      // queue the cells that can reach r_hi; walk them 32 at a time
      const unsigned vm = __ballot_sync(0xffffffffu, cnt > 0);
      if (cnt > 0) s_q[wib][queued + __popc(vm & lt)] = make_int4(beg, cnt, t, imgp);
      queued += __popc(vm);
      __syncwarp();
      const bool last = t0 + 32 >= ncell;
      while (queued >= 32 || (last && queued > 0)) {
        const int take_n = queued < 32 ? queued : 32;
        const int4 e = lane < take_n ? s_q[wib][lane] : make_int4(0, 0, 0, 0);
        __syncwarp();
        if (lane + 32 < queued) s_q[wib][lane] = s_q[wib][lane + 32];
        queued -= take_n;
        __syncwarp();
        walk(e.y, e.x, e.z, e.w);
      }
#else
      walk(cnt, beg, t, imgp);
#endif
    }
    // the second pass visits only the detected atoms with such a pair (lambda_min only
    // decreases, so a pair screened out here stays out)
    if constexpr (PHASE == 0) {
      if (__any_sync(0xffffffffu, need) && lane == 0) det1[atomicAdd(n_det1, 1)] = i;
    }
  }
}

// Push lambda_min, average (Eq. lambda_3_i), hysteresis (Eq. lambda_4_i), flag precise.
__global__ void k_lambda_final(int n, const uint8_t* __restrict__ ch, const double* __restrict__ lam_min,
                               double* __restrict__ hist, int ns, int pos, int fill, double dlam_min,
                               double* __restrict__ lam_avg, double* __restrict__ lam_prev, double* __restrict__ lam,
                               int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double lm = lam_min[i];
  if (fill) {
    for (int q = 0; q < ns; ++q) hist[(size_t)q * n + i] = lm;
  } else {
    hist[(size_t)pos * n + i] = lm;
  }
  double avg = ring_mean(hist, ns, pos, (size_t)n, i);
  lam_avg[i] = avg;
  double prev = fill ? avg : lam_prev[i];
  bool take = fabs(__dsub_rn(avg, prev)) >= dlam_min || avg == 0.0 || avg == 1.0;
  double l = take ? avg : prev;
  if (ch && !ch[i]) l = 1.0;
  lam_prev[i] = l;
  lam[i] = l;
  flag[i] = l < 1.0 ? 1 : 0;
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

void launch_csp(ap_ctx* c, const double* d_x, const uint8_t* d_ch, cudaStream_t s, bool fresh_rows,
                double stale_disp) {
  double r = c->cfg.eam_rc + c->cfg.skin;
  double rs2 = r * r;
  const int* off = c->stored_off ? c->d_off_eam : nullptr;
  int* n_slow = &c->d_sc->n_csp_slow;
  cudaMemsetAsync(n_slow, 0, sizeof(int), s);
  // Rows older than the positions: stale2 = the radius inside which they are complete.
  // The build's split still bounds the skin part from below: its entries were beyond r_c
  // at the build and are now beyond r_c - 2 m, the radius the in-range part is tested
  // against before the skin part is skipped.
  float stale2 = 0.f;
  const int* nin = fresh_rows ? c->d_lim_eam : nullptr;
  float rpf2 = c->split_rpf2;
  if (stale_disp > 0.0) {
    const double rin = r - 2.0 * stale_disp;
    stale2 = rin > 0.0 ? (float)(rin * rin) : 1e-30f;
    cudaMemsetAsync(&c->d_sc->n_stale_bad, 0, sizeof(int), s);
    const double rp = std::sqrt((double)c->split_rpf2) - 2.0 * stale_disp;
    nin = c->d_split_eam;
    rpf2 = rp > 0.0 ? (float)(rp * rp) : 0.f;
  }
  k_csp<<<nblk(c->n, 128), 128, 0, s>>>((int)c->n, d_x, d_ch, c->d_sys, c->d_atom_sys, c->d_sh32, c->d_cunw,
                                              c->d_nbr_eam, off, c->d_cnt_eam, c->cap_eam, (float)rs2, rs2, c->d_csp,
                                              c->d_csp_slow, n_slow, nin, rpf2, stale2, &c->d_sc->n_stale_bad);
  // the handed-over atoms (a small fraction), grid-stride over the device-side count
  k_csp_exact<<<c->num_sms * 4, 128, 0, s>>>(d_x, d_ch, c->d_sys, c->d_atom_sys, c->d_sh32, c->d_cunw, c->d_nbr_eam,
                                             off, c->d_cnt_eam, c->cap_eam, (float)rs2, rs2, c->d_csp,
                                             c->d_csp_slow, n_slow, stale2, &c->d_sc->n_stale_bad);
  c->kernels += 2;
}

// d_score: the detection score pushed into the history (CSP, or the selector's p),
// with thresholds (lo, hi) in the f_cut argument (hi - avg)/(hi - lo).
void launch_lambda0(ap_ctx* c, const uint8_t* d_ch, const double* d_score, double lo, double hi, cudaStream_t s) {
  int ns = c->cfg.n_csp_avg;
  int fill = c->hist_started ? 0 : 1;
  int pos = fill ? 0 : (c->csp_pos + 1) % ns;
  c->csp_pos = pos;
  k_lambda0<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, d_ch, d_score, c->d_csp_hist, ns, pos, fill, lo, hi,
                                            c->cfg.fcut_mode, c->d_csp_avg, c->d_lam0, c->d_lam_min, c->d_flag);
  c->kernels += 2 + scan_exclusive(c->d_flag, c->d_scan, (int)c->n, c->d_scan_tmp, s);
  k_compact<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, c->d_flag, c->d_scan, c->d_detected, &c->d_sc->n_detected,
                                            nullptr);
}

void launch_spread(ap_ctx* c, const double* d_x, const uint8_t* d_ch, cudaStream_t s) {
  int grid = c->num_sms * 8;
  const int* st = c->cells_stale ? c->sten_spread_stale : c->sten_spread;
  const float margin = c->cells_stale ? (float)c->stale_m : 0.f;
  // +3.4e38 in every float: the FP32 minima start above any estimate
  cudaMemsetAsync(c->d_vmin_f, 0x7f, sizeof(float) * (size_t)c->n, s);
  cudaMemsetAsync(&c->d_sc->n_det1, 0, sizeof(int), s);
  k_spread<0><<<grid, kSpreadWarps * 32, 0, s>>>(c->d_detected, &c->d_sc->n_detected, d_x, d_ch, c->d_sys,
                                                 c->d_atom_sys, c->d_sh32, c->d_cunw, c->d_cell_start,
                                                 c->d_cell_atoms, c->d_lam0, c->cfg.r_lo, c->cfg.r_hi,
                                                 c->cfg.fcut_mode, st[0], st[1], st[2], c->d_lam_min, margin,
                                                 c->d_vmin_f, c->d_det1, &c->d_sc->n_det1);
  k_spread<1><<<grid, kSpreadWarps * 32, 0, s>>>(c->d_det1, &c->d_sc->n_det1, d_x, d_ch, c->d_sys,
                                                 c->d_atom_sys, c->d_sh32, c->d_cunw, c->d_cell_start,
                                                 c->d_cell_atoms, c->d_lam0, c->cfg.r_lo, c->cfg.r_hi,
                                                 c->cfg.fcut_mode, st[0], st[1], st[2], c->d_lam_min, margin,
                                                 c->d_vmin_f, nullptr, nullptr);
  c->kernels += 2;
}

void launch_lambda_final(ap_ctx* c, const uint8_t* d_ch, double* d_lam, int* d_queue, int64_t* d_nq64,
                         cudaStream_t s) {
  int ns = c->cfg.n_lam_avg;
  int fill = c->hist_started ? 0 : 1;
  int pos = fill ? 0 : (c->lam_pos + 1) % ns;
  c->lam_pos = pos;
  c->hist_started = true;
  k_lambda_final<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, d_ch, c->d_lam_min, c->d_lam_hist, ns, pos, fill,
                                                 c->cfg.dlam_min, c->d_lam_avg, c->d_lam_prev, d_lam, c->d_flag);
  c->kernels += 2 + scan_exclusive(c->d_flag, c->d_scan, (int)c->n, c->d_scan_tmp, s);
  k_compact<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, c->d_flag, c->d_scan, d_queue, &c->d_sc->n_precise,
                                            (long long*)(d_nq64 ? d_nq64 : (int64_t*)&c->d_sc->n_precise64));
}

}  // namespace ap
