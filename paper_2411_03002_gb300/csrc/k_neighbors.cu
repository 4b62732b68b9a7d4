// Cell list and neighbour rows (section 2.4: the per-domain neighbour search that
// the paper delegates to LAMMPS).  Row i of a list holds every image (j, s) with
// |x_j + s L - x_i|^2 < r_list^2, decided by that FP64 expression; an FP32
// cell-relative pre-filter only skips candidates that are clearly in or out.
#include <algorithm>
#include <cmath>

#include "ap_internal.cuh"

namespace ap {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_scan_block(const int* __restrict__ in, int* __restrict__ out, int m, int n_in,
                             int* __restrict__ bsum) {
  __shared__ int ws[kScanThreads / 32];
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int v[kScanItems];
  int tsum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int idx = base + k;
    v[k] = (idx < n_in) ? in[idx] : 0;
    tsum += v[k];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < kScanThreads / 32) ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) ws[lane] = w;
  }
  __syncthreads();
  int run = x - tsum + (wid > 0 ? ws[wid - 1] : 0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int idx = base + k;
    if (idx < m) out[idx] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = run;
}

__global__ void k_scan_add(int* __restrict__ out, int m, const int* __restrict__ offs) {
  int b = blockIdx.x;
  int add = offs[b];
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
    int idx = b * kScanTile + k;
    if (idx < m) out[idx] += add;
  }
}

int scan_rec(const int* in, int n_in, int* out, int m, int* tmp, cudaStream_t s) {
  int nb = (m + kScanTile - 1) / kScanTile;
  int k = 1;
  k_scan_block<<<nb, kScanThreads, 0, s>>>(in, out, m, n_in, tmp);
  if (nb > 1) {
    int* offs = tmp + nb;
    k += scan_rec(tmp, nb, offs, nb, tmp + 2 * nb, s);
    k_scan_add<<<nb, 256, 0, s>>>(out, m, offs);
    ++k;
  }
  return k;
}

__device__ inline int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__device__ inline const SysInfo& sys_of(const SysInfo* sys, const int* atom_sys, int i) {
  return sys[atom_sys ? atom_sys[i] : 0];
}

// ------------------------------------------------------------------ binning
__global__ void k_bin(int n, const double* __restrict__ x, const int32_t* __restrict__ species,
                      const SysInfo* __restrict__ sys, const int* __restrict__ atom_sys, int* __restrict__ cell,
                      int* __restrict__ slot, int4* __restrict__ cunw, int* __restrict__ cell_count,
                      DevScalars* sc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const SysInfo& S = sys_of(sys, atom_sys, i);
  int cw[3], cu[3];
  int bad = 0;
  if (species && species[i] != 0) bad |= kErrArg;
  for (int d = 0; d < 3; ++d) {
    double xv = x[3 * i + d];
    if (!isfinite(xv)) {
      bad |= kErrNonfinite;
      cw[d] = 0;
      cu[d] = 0;
      continue;
    }
    double rel = xv - S.lo[d];
    int nw = 0;
    if (S.periodic[d]) {
      nw = (int)floor(rel / S.L[d]);
      rel = rel - (double)nw * S.L[d];
    } else if (rel < 0.0 || rel >= S.L[d]) {
      bad |= kErrBox;
    }
    int c = (int)floor(rel / S.h[d]);
    c = c < 0 ? 0 : (c >= S.nc[d] ? S.nc[d] - 1 : c);
    cw[d] = c;
    cu[d] = c + nw * S.nc[d];
  }
  if (bad) atomicOr(&sc->err, bad);
  int id = S.cell_base + (cw[2] * S.nc[1] + cw[1]) * S.nc[0] + cw[0];
  cell[i] = id;
  cunw[i] = make_int4(cu[0], cu[1], cu[2], pack_cell(cw[0], cw[1], cw[2]));
  slot[i] = atomicAdd(&cell_count[id], 1);
}

__global__ void k_cell_scatter(int n, const int* __restrict__ cell, const int* __restrict__ slot,
                               const int* __restrict__ start, int* __restrict__ atoms) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  atoms[start[cell[i]] + slot[i]] = i;
}

// Sort each cell's atoms by index so that rows come out in a deterministic order.
__global__ void k_cell_sort(int n_cells, const int* __restrict__ start, int* __restrict__ atoms) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  int b = start[c], e = start[c + 1];
  for (int a = b + 1; a < e; ++a) {
    int t = atoms[a];
    int p = a - 1;
    while (p >= b && atoms[p] > t) {
      atoms[p + 1] = atoms[p];
      --p;
    }
    atoms[p + 1] = t;
  }
}

// Cell-relative coordinates s = (x - lo) - c_unw h; w = packed wrapped cell.
__global__ void k_shadow(int n, const double* __restrict__ x, const SysInfo* __restrict__ sys,
                         const int* __restrict__ atom_sys, const double* __restrict__ org,
                         const int4* __restrict__ cunw, float4* __restrict__ s32, double4_32a* __restrict__ s64) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const SysInfo& S = sys_of(sys, atom_sys, i);
  const int4 c = cunw[i];
  const double xi[3] = {x[3 * i + 0], x[3 * i + 1], x[3 * i + 2]};
  double sh[3];
  cell_shadow(S, org, c, xi, sh);
  s32[i] = make_float4((float)sh[0], (float)sh[1], (float)sh[2], __int_as_float(c.w));
  if (s64) s64[i] = make_double4_32a(sh[0], sh[1], sh[2], (double)c.w);
}

__global__ void k_wrap(int n, double* __restrict__ x, const SysInfo* __restrict__ sys, const int* __restrict__ atom_sys) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const SysInfo& S = sys_of(sys, atom_sys, i);
  for (int d = 0; d < 3; ++d) {
    if (!S.periodic[d]) continue;
    double xv = x[3 * i + d];
    double rel = xv - S.lo[d];
    if (rel >= 0.0 && rel < S.L[d]) continue;
    int nw = (int)floor(rel / S.L[d]);
    x[3 * i + d] = __dsub_rn(xv, __dmul_rn((double)nw, S.L[d]));
  }
}

// ------------------------------------------------------------------ row builds
// The exact decision: |(x_j + S L) - x_i|^2 < rc2 with explicit round-to-nearest
// operations (no contraction), S the image of j relative to the input positions.
__device__ inline bool exact_within(const double* __restrict__ x, const SysInfo& S, int i, int j, const int4& ci,
                                    const int4& cj, const int img[3], double rc2) {
  int cwi[3] = {cell_x(ci.w), cell_y(ci.w), cell_z(ci.w)};
  int cwj[3] = {cell_x(cj.w), cell_y(cj.w), cell_z(cj.w)};
  int cui[3] = {ci.x, ci.y, ci.z};
  int cuj[3] = {cj.x, cj.y, cj.z};
  double r2 = 0.0;
  double dd[3];
  for (int d = 0; d < 3; ++d) {
    int Sd = 0;
    if (S.periodic[d]) Sd = img[d] + (cui[d] - cwi[d]) / S.nc[d] - (cuj[d] - cwj[d]) / S.nc[d];
    double shifted = Sd == 0 ? x[3 * j + d] : __dadd_rn(x[3 * j + d], __dmul_rn((double)Sd, S.L[d]));
    dd[d] = __dsub_rn(shifted, x[3 * i + d]);
  }
  r2 = __dadd_rn(__dadd_rn(__dmul_rn(dd[0], dd[0]), __dmul_rn(dd[1], dd[1])), __dmul_rn(dd[2], dd[2]));
  return r2 < rc2;
}

// One warp builds one row (used for the long ACE rows).  The lanes test the stencil cells
// ((2 sten + 1)^3 around atom i's cell) 32 at a time against the cell-box distance and
// queue the cells that pass in a per-warp shared-memory buffer; each full batch of 32
// queued cells is walked with one cell per lane, the lanes iterating their cells' atoms in
// lock-step, and accepted (j, offset) are appended with ballot compaction.  Entry order:
// (batch, atom slot, lane) -- deterministic.  Returns the full count (may exceed cap).
// With cells older than the positions (atoms moved up to `margin` since the cell build),
// a cell is pruned only beyond r + margin, and the stencil must reach r + 2 margin.
// buf: this warp's 64-entry shared-memory queue (first atom slot, count, cell offset,
// image).
__device__ inline int build_row_warp(int i, const double* __restrict__ x, const SysInfo& S,
                                     const float4* __restrict__ s32, const int4* __restrict__ cunw,
                                     const int* __restrict__ cstart, const int* __restrict__ catoms, float rcf2,
                                     double rc2, float band, int cap, int* __restrict__ row,
                                     int* __restrict__ offrow, int sten, float margin, int4* buf) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const float4 si = s32[i];
  const int4 ci = cunw[i];
  const int cw[3] = {cell_x(ci.w), cell_y(ci.w), cell_z(ci.w)};
  const float rprune = sqrtf(rcf2) + margin, prune2 = rprune * rprune + band;
  const int W = 2 * sten + 1, ncell = W * W * W;
  int cnt = 0, queued = 0;
  for (int t0 = 0; t0 < ncell; t0 += 32) {
    const int t = t0 + lane;
    const int dx = t % W - sten, dy = (t / W) % W - sten, dz = t / (W * W) - sten;
    int tc[3] = {cw[0] + dx, cw[1] + dy, cw[2] + dz};
    int img[3] = {0, 0, 0};
    bool valid = t < ncell;
    for (int d = 0; d < 3 && valid; ++d) {
      if (S.periodic[d]) {
        img[d] = floor_div(tc[d], S.nc[d]);
        tc[d] -= img[d] * S.nc[d];
      } else if (tc[d] < 0 || tc[d] >= S.nc[d]) {
        valid = false;
      }
    }
    if (valid) {
      const float gx = fmaxf(0.f, fmaxf((float)dx * S.hf[0] - si.x, si.x - (float)(dx + 1) * S.hf[0]));
      const float gy = fmaxf(0.f, fmaxf((float)dy * S.hf[1] - si.y, si.y - (float)(dy + 1) * S.hf[1]));
      const float gz = fmaxf(0.f, fmaxf((float)dz * S.hf[2] - si.z, si.z - (float)(dz + 1) * S.hf[2]));
      valid = gx * gx + gy * gy + gz * gz <= prune2;
    }
    int b = 0, len = 0;
    if (valid) {
      const int cid = S.cell_base + (tc[2] * S.nc[1] + tc[1]) * S.nc[0] + tc[0];
      b = cstart[cid];
      len = cstart[cid + 1] - b;
    }
    const unsigned vm = __ballot_sync(0xffffffffu, len > 0);
    if (len > 0) buf[queued + __popc(vm & lt)] = make_int4(b, len, pack_off(dx, dy, dz), pack_off(img[0], img[1], img[2]));
    queued += __popc(vm);
    __syncwarp();
    // walk a full batch, or what is left after the last stencil cell
    const bool last = t0 + 32 >= ncell;
    while (queued >= 32 || (last && queued > 0)) {
      const int take_n = queued < 32 ? queued : 32;
      int4 e = make_int4(0, 0, 0, 0);
      if (lane < take_n) e = buf[lane];
      __syncwarp();
      if (lane + 32 < queued) buf[lane] = buf[lane + 32];   // the rest moves to the front
      queued -= take_n;
      __syncwarp();
      const int ox_i = off_x(e.z), oy_i = off_y(e.z), oz_i = off_z(e.z);
      const int im[3] = {off_x(e.w), off_y(e.w), off_z(e.w)};
      const float ox = (float)ox_i * S.hf[0] - si.x;
      const float oy = (float)oy_i * S.hf[1] - si.y;
      const float oz = (float)oz_i * S.hf[2] - si.z;
      const bool self_cell = ox_i == 0 && oy_i == 0 && oz_i == 0;
      const int maxlen = __reduce_max_sync(0xffffffffu, e.y);
      for (int k = 0; k < maxlen; ++k) {
        bool take = false;
        int j = 0;
        if (k < e.y) {
          j = catoms[e.x + k];
          if (!(j == i && self_cell)) {
            const float4 sj = s32[j];
            const float ddx = ox + sj.x, ddy = oy + sj.y, ddz = oz + sj.z;
            const float r2f = ddx * ddx + ddy * ddy + ddz * ddz;
            if (r2f < rcf2 - band) {
              take = true;
            } else if (r2f <= rcf2 + band) {
              take = exact_within(x, S, i, j, ci, cunw[j], im, rc2);
            }
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, take);
        const int pos = cnt + __popc(m & lt);
        if (take && pos < cap) {
          row[pos] = j;
          if (offrow) offrow[pos] = e.z;
        }
        cnt += __popc(m);
      }
    }
  }
  return cnt;
}

#ifndef AP_BUILD_MINB
#define AP_BUILD_MINB 9   // resident 128-thread blocks per SM the EAM row build is compiled for (<= 56 registers)
#endif
// Unroll depth of the per-cell candidate loop of the EAM row build (compile-time tuning).
#ifndef AP_BUILD_UNROLL
#define AP_BUILD_UNROLL 2
#endif
constexpr int kBuildUnroll = AP_BUILD_UNROLL;

// One thread builds one row (EAM rows of all atoms): scan the 5x5x5 stencil around atom i and keep the
// accepted (j, offset).  The row is ordered in two parts: first the entries whose FP32 distance
// lies inside the potential cutoff (rpf2 = r_c^2), in stencil order, then the skin entries;
// n_in_out receives the length of the first part.  The EAM density pass records, per atom,
// where the in-range entries end at the current positions (it re-tests every entry), so the
// force pass walks only that prefix; the split at build time only makes the prefix short.
// The CSP on rows built at its own positions may stop after the first part.  Candidates are
// read from s32c, the shadows in cell order; t_self is atom i's own position in that order.
__device__ inline int build_row(int i, int t_self, const double* __restrict__ x, const SysInfo& S,
                                const float4* __restrict__ s32, const float4* __restrict__ s32c,
                                const int4* __restrict__ cunw, const int* __restrict__ cstart,
                                const int* __restrict__ catoms, float rcf2, double rc2, float rpf2, float band,
                                int cap, int* __restrict__ row, int* __restrict__ offrow, int& n_in_out) {
  const float4 si = s32[i];
  const int4 ci = cunw[i];
  const int cw[3] = {cell_x(ci.w), cell_y(ci.w), cell_z(ci.w)};
  const float sv[3] = {si.x, si.y, si.z};
  const float rmax2 = rcf2 + band;
  int n_in = 0, n_skin = 0;   // in-range entries fill the row from the front, skin entries from the back
  for (int dz = -kStencil; dz <= kStencil; ++dz) {
    int tz = cw[2] + dz, iz = 0;
    if (S.periodic[2]) {
      iz = floor_div(tz, S.nc[2]);
      tz -= iz * S.nc[2];
    } else if (tz < 0 || tz >= S.nc[2]) {
      continue;
    }
    float gz = fmaxf(0.f, fmaxf((float)dz * S.hf[2] - sv[2], sv[2] - (float)(dz + 1) * S.hf[2]));
    for (int dy = -kStencil; dy <= kStencil; ++dy) {
      int ty = cw[1] + dy, iy = 0;
      if (S.periodic[1]) {
        iy = floor_div(ty, S.nc[1]);
        ty -= iy * S.nc[1];
      } else if (ty < 0 || ty >= S.nc[1]) {
        continue;
      }
      float gy = fmaxf(0.f, fmaxf((float)dy * S.hf[1] - sv[1], sv[1] - (float)(dy + 1) * S.hf[1]));
      if (gz * gz + gy * gy > rmax2) continue;
      for (int dx = -kStencil; dx <= kStencil; ++dx) {
        int tx = cw[0] + dx, ix = 0;
        if (S.periodic[0]) {
          ix = floor_div(tx, S.nc[0]);
          tx -= ix * S.nc[0];
        } else if (tx < 0 || tx >= S.nc[0]) {
          continue;
        }
        float gx = fmaxf(0.f, fmaxf((float)dx * S.hf[0] - sv[0], sv[0] - (float)(dx + 1) * S.hf[0]));
        if (gz * gz + gy * gy + gx * gx > rmax2) continue;
        int cid = S.cell_base + (tz * S.nc[1] + ty) * S.nc[0] + tx;
        int b = cstart[cid], e = cstart[cid + 1];
        const float ox = (float)dx * S.hf[0] - si.x;
        const float oy = (float)dy * S.hf[1] - si.y;
        const float oz = (float)dz * S.hf[2] - si.z;
#if AP_BUILD_UNROLL > 1
#pragma unroll kBuildUnroll
#endif
        for (int a = b; a < e; ++a) {
          // the shadows in cell order: the candidate's shadow and index load independently
          if (a == t_self && dx == 0 && dy == 0 && dz == 0) continue;
          const float4 sj = s32c[a];
          const int j = catoms[a];
          float ddx = ox + sj.x, ddy = oy + sj.y, ddz = oz + sj.z;
          float r2f = ddx * ddx + ddy * ddy + ddz * ddz;
          if (r2f > rcf2 + band) continue;
          bool take = r2f < rcf2 - band;
          if (!take) {
            int img[3] = {ix, iy, iz};
            take = exact_within(x, S, i, j, ci, cunw[j], img, rc2);
          }
          if (take) {
            const bool in = r2f < rpf2;
            if (n_in + n_skin < cap) {
              const int pos = in ? n_in : cap - 1 - n_skin;
              row[pos] = j;
              if (offrow) offrow[pos] = pack_off(dx, dy, dz);
            }
            if (in)
              ++n_in;
            else
              ++n_skin;
          }
        }
      }
    }
  }
  const int cnt = n_in + n_skin;
  n_in_out = n_in;
  if (cnt < cap) {
    // Close the gap: the skin entries move from [cap - n_skin, cap) to [n_in, cnt) in
    // chunks of 8, each chunk read in full before it is written.  A chunk's
    // destinations lie below every source of the later chunks (n_in + n_skin < cap),
    // so no entry is overwritten before it is read.  (A full row has no gap.)
    int* src = row + cap - n_skin;
    int* dst = row + n_in;
    for (int k0 = 0; k0 < n_skin; k0 += 8) {
      int v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = k0 + u < n_skin ? src[k0 + u] : 0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k0 + u < n_skin) dst[k0 + u] = v[u];
    }
    if (offrow) {
      int* osrc = offrow + cap - n_skin;
      int* odst = offrow + n_in;
      for (int k0 = 0; k0 < n_skin; k0 += 8) {
        int v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = k0 + u < n_skin ? osrc[k0 + u] : 0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (k0 + u < n_skin) odst[k0 + u] = v[u];
      }
    }
  }
  return cnt;
}

// FP32 shadows in cell order (s32c[a] = s32[catoms[a]]), for the EAM row build.
__global__ void k_shadow_cells(int n, const int* __restrict__ catoms, const float4* __restrict__ s32,
                               float4* __restrict__ s32c) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) s32c[a] = s32[catoms[a]];
}

__global__ void __launch_bounds__(128, AP_BUILD_MINB) k_build_eam(int n, const double* __restrict__ x, const SysInfo* __restrict__ sys,
                            const int* __restrict__ atom_sys, const float4* __restrict__ s32,
                            const float4* __restrict__ s32c,
                            const int4* __restrict__ cunw, const int* __restrict__ cstart,
                            const int* __restrict__ catoms, float rcf2, double rc2, float rpf2, float band,
                            int cap, int* __restrict__ nbr, int* __restrict__ off, int* __restrict__ cnt,
                            int* __restrict__ nin, DevScalars* sc) {
  // Threads take the atoms in cell order: the atoms of one cell walk the same stencil
  // cells with the same atom counts, so a warp diverges only on the per-atom gap test.
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = catoms[t];
  const SysInfo& S = sys_of(sys, atom_sys, i);
  int a = 0;
  int c = build_row(i, t, x, S, s32, s32c, cunw, cstart, catoms, rcf2, rc2, rpf2, band, cap, nbr + (size_t)i * cap,
                    off ? off + (size_t)i * cap : nullptr, a);
  // an overflowing row holds cap valid entries (the capacity error makes the caller
  // rebuild or fail before any result is used)
  cnt[i] = c < cap ? c : cap;
  nin[i] = a < cap ? a : cap;   // the in-range part (read by the CSP on rows built at its positions)
  if (c > cap) {
    atomicMax(&sc->need_eam, c);
    atomicOr(&sc->err, kErrCapacity);
  }
}

__global__ void __launch_bounds__(256) k_build_ace(const int* __restrict__ queue, const int* __restrict__ nq,
                                                   const double* __restrict__ x, const SysInfo* __restrict__ sys,
                                                   const int* __restrict__ atom_sys, const float4* __restrict__ s32,
                                                   const int4* __restrict__ cunw, const int* __restrict__ cstart,
                                                   const int* __restrict__ catoms, float rcf2, double rc2,
                                                   float band, int cap, int* __restrict__ nbr, int* __restrict__ off,
                                                   int* __restrict__ cnt, DevScalars* sc, int sten, float margin) {
  __shared__ int4 s_buf[8][64];   // per warp: the stencil cells queued for the walk
  const int wib = threadIdx.x >> 5;
  const int m = *nq;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < m; q += warps) {
    const int i = queue[q];
    const SysInfo& S = sys_of(sys, atom_sys, i);
    const int c = build_row_warp(i, x, S, s32, cunw, cstart, catoms, rcf2, rc2, band, cap, nbr + (size_t)q * cap,
                                 off ? off + (size_t)q * cap : nullptr, sten, margin, s_buf[wib]);
    if ((threadIdx.x & 31) == 0) {
      cnt[q] = c < cap ? c : cap;
      const int kept_c = c < cap ? c : cap;   // only a new maximum takes the (same-address) atomic
      if (kept_c > __ldcg(&sc->ace_row_max)) atomicMax(&sc->ace_row_max, kept_c);
      if (c > cap) {
        atomicMax(&sc->need_ace, c);
        atomicOr(&sc->err, kErrCapacity);
      }
    }
  }
}

// Export: entry (j, k) -> image s relative to the build positions.
__global__ void k_export(int rows, int cap_in, int cap_out, const int* __restrict__ row_atom,
                         const int* __restrict__ nbr, const int* __restrict__ off, const int* __restrict__ cnt_in,
                         const SysInfo* __restrict__ sys, const int* __restrict__ atom_sys,
                         const int4* __restrict__ cunw, int* __restrict__ cnt_out, int* __restrict__ idx_out,
                         int* __restrict__ shift_out) {
  int r = blockIdx.x;
  if (r >= rows) return;
  int i = row_atom ? row_atom[r] : r;
  const SysInfo& S = sys_of(sys, atom_sys, i);
  int c = cnt_in[r];
  if (threadIdx.x == 0) cnt_out[r] = c < cap_out ? c : cap_out;
  int4 ci = cunw[i];
  for (int q = threadIdx.x; q < c && q < cap_out; q += blockDim.x) {
    int j = nbr[(size_t)r * cap_in + q];
    int4 cj = cunw[j];
    int k[3];
    if (off) {
      int p = off[(size_t)r * cap_in + q];
      k[0] = off_x(p);
      k[1] = off_y(p);
      k[2] = off_z(p);
    } else {
      k[0] = wrap_off(cell_x(cj.w) - cell_x(ci.w), S.nc[0], S.periodic[0]);
      k[1] = wrap_off(cell_y(cj.w) - cell_y(ci.w), S.nc[1], S.periodic[1]);
      k[2] = wrap_off(cell_z(cj.w) - cell_z(ci.w), S.nc[2], S.periodic[2]);
    }
    int cu_i[3] = {ci.x, ci.y, ci.z}, cu_j[3] = {cj.x, cj.y, cj.z};
    idx_out[(size_t)r * cap_out + q] = j;
    for (int d = 0; d < 3; ++d) {
      int sd = 0;
      if (S.periodic[d]) sd = (k[d] - (cu_j[d] - cu_i[d])) / S.nc[d];
      shift_out[((size_t)r * cap_out + q) * 3 + d] = sd;
    }
  }
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

size_t scan_tmp_bytes(int n) { return sizeof(int) * ((size_t)n / 512 + 256); }

int scan_exclusive(const int* d_in, int* d_out, int n, int* d_tmp, cudaStream_t s) {
  return scan_rec(d_in, n, d_out, n + 1, d_tmp, s);
}

void launch_wrap_positions(ap_ctx* c, double* d_x, cudaStream_t s) {
  k_wrap<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, d_x, c->d_sys, c->d_atom_sys);
  c->kernels += 1;
}

void launch_bin(ap_ctx* c, const double* d_x, const int32_t* d_species, cudaStream_t s) {
  cudaMemsetAsync(c->d_cell_count, 0, sizeof(int) * (size_t)c->n_cells, s);
  k_bin<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, d_x, d_species, c->d_sys, c->d_atom_sys, c->d_cell, c->d_slot,
                                        c->d_cunw, c->d_cell_count, c->d_sc);
  c->kernels += 1;
}

void launch_cell_sort(ap_ctx* c, cudaStream_t s) {
  c->kernels += 2 + scan_exclusive(c->d_cell_count, c->d_cell_start, c->n_cells, c->d_scan_tmp, s);
  k_cell_scatter<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, c->d_cell, c->d_slot, c->d_cell_start, c->d_cell_atoms);
  k_cell_sort<<<nblk(c->n_cells, 128), 128, 0, s>>>(c->n_cells, c->d_cell_start, c->d_cell_atoms);
}

void launch_shadow(ap_ctx* c, const double* d_x, cudaStream_t s) {
  k_shadow<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, d_x, c->d_sys, c->d_atom_sys, c->d_org, c->d_cunw, c->d_sh32,
                                           c->cfg.precision == AP_PREC_FP64 ? c->d_sh64 : nullptr);
  c->kernels += 1;
}

static constexpr float kBand = 1e-3f;   // guard band on r^2 (A^2) around the cutoff

// Sum of the row counts (block sums, one 64-bit atomic per block).
__global__ void k_row_total(int rows, const int* __restrict__ cnt, unsigned long long* __restrict__ out) {
  __shared__ unsigned long long part[8];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = i < rows ? (unsigned long long)cnt[i] : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
    atomicAdd(out, s);
  }
}

void launch_row_total(ap_ctx* c, int which, int rows, cudaStream_t s) {
  cudaMemsetAsync(&c->d_sc->row_total, 0, sizeof(unsigned long long), s);
  if (rows > 0)
    k_row_total<<<nblk(rows, 256), 256, 0, s>>>(
        rows, which == 0 ? c->d_cnt_eam : which == 1 ? c->d_cnt_ace : c->d_lim_eam, &c->d_sc->row_total);
}

void launch_build_eam(ap_ctx* c, const double* d_x, cudaStream_t s) {
  double r = c->cfg.eam_rc + c->cfg.skin;
  double rc2 = r * r;
  // the potential's own cutoff: rows are split at it (the Mishin rc may lie below eam_rc)
  const double rp = c->cfg.eam_type == AP_EAM_MISHIN ? c->cfg.eam_mishin[28] : c->cfg.eam_rc;
  c->split_rpf2 = (float)(rp * rp);
  k_shadow_cells<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, c->d_cell_atoms, c->d_sh32, c->d_sh32c);
  c->kernels += 1;
  k_build_eam<<<nblk(c->n, 128), 128, 0, s>>>((int)c->n, d_x, c->d_sys, c->d_atom_sys, c->d_sh32, c->d_sh32c,
                                              c->d_cunw,
                                              c->d_cell_start, c->d_cell_atoms, (float)rc2, rc2, c->split_rpf2,
                                              kBand, c->cap_eam, c->d_nbr_eam,
                                              c->stored_off ? c->d_off_eam : nullptr, c->d_cnt_eam, c->d_lim_eam,
                                              c->d_sc);
  c->kernels += 1;
}

void launch_build_ace(ap_ctx* c, const double* d_x, const int* d_queue, const int* d_nq, cudaStream_t s) {
  const double r = c->cfg.ace_rc + c->cfg.skin;
  // Cells older than the positions (ap_step kept the EAM lists): the atoms moved up to
  // m = stale_m since the cell build, so a cell is pruned only beyond r + m and the
  // stencil reaches r + 2 m.  The rows stay complete while no atom moves more than skin/2
  // from its position at this build, which ap_step checks after every drift.
  int sten = kStencil;
  float margin = 0.f;
  if (c->cells_stale) {
    margin = (float)c->stale_m;
    for (const SysInfo& S : c->h_sys)
      for (int d = 0; d < 3; ++d) sten = std::max(sten, (int)std::ceil((r + 2.0 * c->stale_m) / S.h[d]));
  }
  double rc2 = r * r;
  int grid = c->num_sms * 8;
  k_build_ace<<<grid, 256, 0, s>>>(d_queue, d_nq, d_x, c->d_sys, c->d_atom_sys, c->d_sh32, c->d_cunw,
                                   c->d_cell_start, c->d_cell_atoms, (float)rc2, rc2, kBand, c->cap_ace,
                                   c->d_nbr_ace, c->stored_off ? c->d_off_ace : nullptr, c->d_cnt_ace, c->d_sc, sten,
                                   margin);
  c->kernels += 1;
}

void launch_export_rows(ap_ctx* c, int which, int rows, int cap_out, int* d_cnt, int* d_idx, int* d_shift,
                        cudaStream_t s) {
  if (rows <= 0) return;
  if (which == 0)
    k_export<<<rows, 128, 0, s>>>(rows, c->cap_eam, cap_out, nullptr, c->d_nbr_eam,
                                  c->stored_off ? c->d_off_eam : nullptr, c->d_cnt_eam, c->d_sys, c->d_atom_sys,
                                  c->d_cunw, d_cnt, d_idx, d_shift);
  else
    k_export<<<rows, 128, 0, s>>>(rows, c->cap_ace, cap_out, c->d_precise, c->d_nbr_ace,
                                  c->stored_off ? c->d_off_ace : nullptr, c->d_cnt_ace, c->d_sys, c->d_atom_sys,
                                  c->d_cunw, d_cnt, d_idx, d_shift);
}

}  // namespace ap
