// C-ABI entry points (include/ap.h) and the host-side orchestration.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "ap_internal.cuh"

using namespace ap;

namespace {

ap_status fail(ap_ctx* c, ap_status st, const std::string& msg) {
  if (c) c->err_msg = msg;
  return st;
}

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(c, AP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
cudaError_t dalloc(T*& p, size_t count) {
  dfree(p);
  if (count == 0) count = 1;
  return cudaMalloc((void**)&p, sizeof(T) * count);
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

ap_status validate(const ap_config& g, std::string& why) {
  auto bad = [&](const char* m) {
    why = m;
    return AP_ERR_ARG;
  };
  if (g.eam_type != AP_EAM_ANALYTIC && g.eam_type != AP_EAM_MISHIN) return bad("unknown eam_type");
  if (g.eam_type == AP_EAM_ANALYTIC && !(g.eam_rc > 0 && g.eam_h > 0 && g.eam_r0 > 0))
    return bad("EAM cutoff, h and r0 must be positive");
  if (g.eam_type == AP_EAM_MISHIN) {
    const double h = g.eam_mishin[6], rc = g.eam_mishin[28];
    if (!(h > 0 && rc > 0)) return bad("Mishin h and rc must be positive");
    if (!(g.eam_rc >= rc)) return bad("eam_rc must be >= the Mishin rc (it sets the EAM rows)");
    if (g.detector == AP_DETECT_SELECTOR) return bad("the selector detector needs eam_type AP_EAM_ANALYTIC");
  }
  if (!(g.ace_rc > 0 && g.ace_n0 > 0)) return bad("ACE cutoff and N0 must be positive");
  if (!(g.skin >= 0)) return bad("skin must be >= 0");
  if (!(g.csp_hi > g.csp_lo)) return bad("csp_hi must exceed csp_lo");
  if (!(g.r_hi > g.r_lo && g.r_lo >= 0)) return bad("need 0 <= r_lo < r_hi");
  if (g.n_csp_avg < 1 || g.n_lam_avg < 1) return bad("averaging windows must be >= 1");
  if (g.precision != AP_PREC_FP64 && g.precision != AP_PREC_MIXED) return bad("unknown precision");
  if (g.fcut_mode != AP_FCUT_PRINTED && g.fcut_mode != AP_FCUT_C2) return bad("unknown fcut_mode");
  if (g.ace_nc < 0 || g.ace_nc > 512) return bad("ace_nc out of range");
  if (g.cap_eam < 0 || g.cap_ace < 0 || g.cap_eam > 4096 || g.cap_ace > 4096) return bad("row capacity out of range");
  if (g.lambda_every < 1) return bad("lambda_every must be >= 1");
  if (g.rebuild_every < AP_REBUILD_SKIN) return bad("rebuild_every must be >= 0 or AP_REBUILD_SKIN");
  if (g.detector != AP_DETECT_CSP && g.detector != AP_DETECT_SELECTOR) return bad("unknown detector");
  if (g.detector == AP_DETECT_SELECTOR && !(g.sel_p_lo >= 0 && g.sel_p_hi > g.sel_p_lo))
    return bad("need 0 <= sel_p_lo < sel_p_hi");
  if (g.thermostat_on != 0 && g.thermostat_on != 1) return bad("thermostat_on must be 0 or 1");
  if (g.ace_fs_on != 0 && g.ace_fs_on != 1) return bad("ace_fs_on must be 0 or 1");
  if (g.ace_fs_on && !(g.ace_fs_eps > 0)) return bad("ace_fs_eps must be positive");
  return AP_OK;
}

// Cell grid of every system: edge >= (largest list radius)/2, so a 5x5x5 stencil
// covers both lists.
ap_status set_systems(ap_ctx* c, int n_sys, const int64_t* offsets, const ap_box* boxes) {
  const ap_config& g = c->cfg;
  double rlist = std::max(g.eam_rc, g.ace_rc) + g.skin;
  double htarget = rlist / kStencil;
  std::vector<SysInfo> sys(n_sys);
  std::vector<double> org;
  int base = 0;
  bool stored = false;
  int spread[3] = {0, 0, 0}, spread_stale[3] = {0, 0, 0};
  // With the skin criterion ACE rows (reaching ace_rc + skin) are built from cells up to
  // m = skin/2 old: pair cell offsets up to ceil((ace_rc + skin + 2m)/h).  Without stored
  // offsets they are recovered from the wrapped cells, which needs 2 offset + 1 cells in
  // every periodic dimension.
  bool wide = true;
  for (int s = 0; s < n_sys; ++s) {
    SysInfo& I = sys[s];
    std::memset(&I, 0, sizeof(I));
    for (int d = 0; d < 3; ++d) {
      double L = boxes[s].hi[d] - boxes[s].lo[d];
      if (!(L > 0)) return fail(c, AP_ERR_ARG, "box hi must exceed lo in every dimension");
      int nc = (int)std::floor(L / htarget);
      if (nc < 1) nc = 1;
      if (nc > kMaxCellsPerDim) return fail(c, AP_ERR_ARG, "box too large for the cell grid (1023 cells per dimension)");
      I.lo[d] = boxes[s].lo[d];
      I.L[d] = L;
      I.nc[d] = nc;
      I.h[d] = L / nc;
      I.hf[d] = (float)I.h[d];
      I.periodic[d] = boxes[s].periodic[d] ? 1 : 0;
      if (I.periodic[d] && nc < 2 * kStencil + 1) stored = true;
      int sp = (int)std::ceil(g.r_hi / I.h[d]);
      if (!I.periodic[d]) sp = std::min(sp, nc);
      spread[d] = std::max(spread[d], sp);
      int sps = (int)std::ceil((g.r_hi + g.skin) / I.h[d]);   // atoms up to skin/2 from their cells
      if (!I.periodic[d]) sps = std::min(sps, nc);
      spread_stale[d] = std::max(spread_stale[d], sps);
      const int reach = (int)std::ceil((g.ace_rc + 2.0 * g.skin) / I.h[d]);
      if (I.periodic[d] && nc < 2 * reach + 1) wide = false;
    }
    I.cell_base = base;
    base += I.nc[0] * I.nc[1] * I.nc[2];
    for (int d = 0; d < 3; ++d) {   // the cell origins lo + c h of the shadows
      I.org[d] = (int)org.size();
      for (int k = 0; k < I.nc[d]; ++k) org.push_back(std::fma((double)k, I.h[d], I.lo[d]));
    }
  }
  bool same = (n_sys == c->n_sys) && c->h_offsets.size() == (size_t)n_sys + 1 &&
              std::equal(offsets, offsets + n_sys + 1, c->h_offsets.begin()) &&
              std::memcmp(sys.data(), c->h_sys.data(), sizeof(SysInfo) * n_sys) == 0;
  if (same) return AP_OK;
  c->h_sys = sys;
  c->h_offsets.assign(offsets, offsets + n_sys + 1);
  c->n_sys = n_sys;
  c->n_cells = base;
  c->stored_off = stored;
  for (int d = 0; d < 3; ++d) {
    c->sten_spread[d] = spread[d];
    c->sten_spread_stale[d] = spread_stale[d];
  }
  c->stale_ok = stored || wide;
  CK(dalloc(c->d_sys, n_sys));
  CK(cudaMemcpy(c->d_sys, sys.data(), sizeof(SysInfo) * n_sys, cudaMemcpyHostToDevice));
  CK(dalloc(c->d_org, org.size()));
  CK(cudaMemcpy(c->d_org, org.data(), sizeof(double) * org.size(), cudaMemcpyHostToDevice));
  dfree(c->d_atom_sys);
  int64_t n = offsets[n_sys];
  if (n_sys > 1 && n > 0) {
    std::vector<int> as(n);
    for (int s = 0; s < n_sys; ++s)
      for (int64_t i = offsets[s]; i < offsets[s + 1]; ++i) as[i] = s;
    CK(dalloc(c->d_atom_sys, n));
    CK(cudaMemcpy(c->d_atom_sys, as.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  }
  if (c->n_cells + 1 > c->cells_cap) {
    c->cells_cap = c->n_cells + 1;
    CK(dalloc(c->d_cell_start, c->cells_cap + 1));
    CK(dalloc(c->d_cell_count, c->cells_cap));
  }
  size_t need_tmp = scan_tmp_bytes(std::max<int64_t>(c->n_cells + 1, n + 1)) / sizeof(int) + 1;
  if (need_tmp > c->scan_tmp_cap) {
    c->scan_tmp_cap = need_tmp;
    CK(dalloc(c->d_scan_tmp, need_tmp));
  }
  c->built = false;
  return AP_OK;
}

ap_status alloc_rows(ap_ctx* c, bool eam, bool ace) {
  if (eam) {
    CK(dalloc(c->d_nbr_eam, (size_t)c->n_cap * c->cap_eam));
    if (c->stored_off) CK(dalloc(c->d_off_eam, (size_t)c->n_cap * c->cap_eam));
  }
  if (ace) {
    CK(dalloc(c->d_nbr_ace, (size_t)c->ace_q_cap * c->cap_ace));
    if (c->stored_off) CK(dalloc(c->d_off_ace, (size_t)c->ace_q_cap * c->cap_ace));
  }
  return AP_OK;
}

cudaError_t dalloc_bytes(void*& p, size_t bytes) {
  if (p) cudaFree(p);
  p = nullptr;
  return cudaMalloc(&p, bytes ? bytes : 16);
}

// Pair-record slots per queue position for rows of up to `need` entries (rounded up
// to 8), reallocated when they grow.
ap_status ensure_ace_records(ap_ctx* c, int need) {
  const int r = (need + 7) & ~7;
  if (c->d_ace_list && r <= c->ace_rec_cap) return AP_OK;
  c->ace_rec_cap = std::max(r, c->ace_rec_cap);
  const size_t rb = c->cfg.precision == AP_PREC_FP64 ? sizeof(double) : sizeof(float);
  CK(dalloc_bytes(c->d_ace_list, rb * 4 * (size_t)c->ace_rec_cap * (size_t)c->ace_q_cap));
  return AP_OK;
}

// ACE rows, pair records and per-atom ACE scratch for at least `need` queue positions:
// sized by the precise queue, not by the atom count, and grown by half again when a
// longer queue arrives (at most n_cap).
ap_status ensure_ace_queue(ap_ctx* c, int64_t need) {
  if (need <= c->ace_q_cap && c->d_cnt_ace) return AP_OK;
  int64_t m = std::max<int64_t>(need + need / 2, 1024);
  m = std::max<int64_t>(std::min<int64_t>(m, c->n_cap), need);
  c->ace_q_cap = m;
  CK(dalloc(c->d_cnt_ace, m));
  ap_status st = alloc_rows(c, false, true);
  if (st) return st;
  const size_t rb = c->cfg.precision == AP_PREC_FP64 ? sizeof(double) : sizeof(float);
  CK(dalloc(c->d_ace_nin, m));
  CK(dalloc(c->d_ace_e12, m));
  CK(dalloc(c->d_ace_e3, m));
  CK(dalloc_bytes(c->d_ace_a48, rb * 48 * (size_t)m));
  CK(dalloc_bytes(c->d_ace_dA, rb * 200 * (size_t)m));
  CK(dalloc_bytes(c->d_ace_de3, rb * 48 * (size_t)m));
  CK(dalloc_bytes(c->d_ace_dAb, rb * (c->cfg.ace_fs_on ? 200 : 1) * (size_t)m));
  if (c->cfg.ace_fs_on) {
    CK(dalloc(c->d_ace_e12b, m));
    CK(dalloc(c->d_ace_fs, 2 * m));
  }
  if (c->d_ace_list) {   // keep the record width, resize for the new queue length
    cudaFree(c->d_ace_list);
    c->d_ace_list = nullptr;
  }
  return ensure_ace_records(c, std::max(c->ace_rec_cap, 8));
}

ap_status ensure_capacity(ap_ctx* c, int64_t n) {
  if (n > 0x7fffffff / 4) return fail(c, AP_ERR_ARG, "too many atoms for 32-bit indices");
  bool stored_changed = c->stored_off && (!c->d_off_eam || !c->d_off_ace);
  if (n <= c->n_cap && !stored_changed) return AP_OK;
  int64_t m = std::max<int64_t>(n, c->n_cap);
  c->n_cap = m;
  CK(dalloc(c->d_cell, m));
  CK(dalloc(c->d_cunw, m));
  CK(dalloc(c->d_cell_atoms, m));
  CK(dalloc(c->d_slot, m));
  CK(dalloc(c->d_sh32, m));
  CK(dalloc(c->d_sh32c, m));
  CK(dalloc(c->d_sh64, m));
  CK(dalloc(c->d_sh32b, m));
  CK(dalloc(c->d_vscale, m));
  CK(dalloc(c->d_cnt_eam, m));
  CK(dalloc(c->d_lim_eam, m));
  if (c->cfg.rebuild_every == AP_REBUILD_SKIN) {
    CK(dalloc(c->d_split_eam, m));
    CK(dalloc(c->d_sh32a, m));
  }
  ap_status st = alloc_rows(c, true, true);
  if (st) return st;
  CK(dalloc(c->d_csp, m));
  CK(dalloc(c->d_csp_slow, m));
  CK(dalloc(c->d_csp_avg, m));
  CK(dalloc(c->d_lam0, m));
  CK(dalloc(c->d_lam_min, m));
  CK(dalloc(c->d_lam_avg, m));
  CK(dalloc(c->d_lam_prev, m));
  CK(dalloc(c->d_csp_hist, (size_t)c->cfg.n_csp_avg * m));
  CK(dalloc(c->d_lam_hist, (size_t)c->cfg.n_lam_avg * m));
  CK(dalloc(c->d_flag, m));
  CK(dalloc(c->d_scan, m + 1));
  CK(dalloc(c->d_detected, m));
  CK(dalloc(c->d_vmin_f, m));
  CK(dalloc(c->d_det1, m));
  CK(dalloc(c->d_precise, m));
  CK(dalloc(c->d_lam_int, m));
  void* q = c->d_q;
  if (q) cudaFree(q);
  CK(cudaMalloc(&c->d_q, 16 * (size_t)m));
  CK(dalloc(c->d_xi, m));
  CK(dalloc(c->d_facc32, m));
  CK(dalloc(c->d_facc64, 3 * m));
  if (c->cfg.ace_deterministic) CK(dalloc(c->d_faccfix, 3 * m));
  CK(dalloc(c->d_efast, m));
  CK(dalloc(c->d_eprec, m));
  CK(dalloc(c->d_eatom, m));
  CK(dalloc(c->d_eext, m));
  CK(dalloc(c->d_changeable, m));
  size_t need_tmp = scan_tmp_bytes(std::max<int64_t>(c->n_cells + 1, m + 1)) / sizeof(int) + 1;
  if (need_tmp > c->scan_tmp_cap) {
    c->scan_tmp_cap = need_tmp;
    CK(dalloc(c->d_scan_tmp, need_tmp));
  }
  if (!c->d_red) CK(dalloc(c->d_red, 2048));
  c->hist_started = false;
  c->lam_ready = false;
  c->md_ready = false;
  return AP_OK;
}

ap_status read_scalars(ap_ctx* c, cudaStream_t s) {
  CK(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return AP_OK;
}

ap_status check_err_bits(ap_ctx* c) {
  int e = c->h_sc->err;
  if (e & kErrArg)
    return fail(c, AP_ERR_ARG, "invalid device input: nonzero species (single-species potentials) or queue index out of range");
  if (e & kErrNonfinite) return fail(c, AP_ERR_NONFINITE, "non-finite position");
  if (e & kErrBox) return fail(c, AP_ERR_BOX, "atom outside a non-periodic box dimension");
  if (e & kErrCapacity) {
    c->need = std::max(c->h_sc->need_eam, c->h_sc->need_ace);
    return fail(c, AP_ERR_CAPACITY, "neighbour row capacity exceeded");
  }
  if (e & kErrSkin) return fail(c, AP_ERR_SKIN, "an atom moved more than skin/2 between rebuilds");
  if (e & kErrTimeout) return fail(c, AP_ERR_TIMEOUT, "a bounded tensor-core wait gave up");
  if (e & kErrRadicand) return fail(c, AP_ERR_RADICAND, "a local-thermostat correction had a negative radicand");
  return AP_OK;
}

ap_status clear_err(ap_ctx* c, cudaStream_t s) {
  CK(cudaMemsetAsync(&c->d_sc->err, 0, sizeof(int), s));
  CK(cudaMemsetAsync(&c->d_sc->need_eam, 0, 2 * sizeof(int), s));
  return AP_OK;
}

// Bin, sort, shadow and EAM rows at the given positions (asynchronous).
void build_async(ap_ctx* c, const double* d_x, const int32_t* d_species, cudaStream_t s) {
  launch_bin(c, d_x, d_species, s);
  launch_cell_sort(c, s);
  launch_shadow(c, d_x, s);
  launch_build_eam(c, d_x, s);
  if (c->d_split_eam)   // the split of the rows, for a CSP on them after the atoms have moved
    cudaMemcpyAsync(c->d_split_eam, c->d_lim_eam, sizeof(int) * (size_t)c->n, cudaMemcpyDeviceToDevice, s);
  c->lim_valid = false;
  c->cells_stale = false;
  c->stale_m = 0.0;
  cudaMemcpyAsync(c->d_sh32b, c->d_sh32, sizeof(float4) * (size_t)c->n, cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(&c->d_sc->max_disp2_bits, 0, sizeof(unsigned int), s);
  // the ACE rows' reference shadows belong to the old cells: +3.4e38 until the next ACE build
  cudaMemsetAsync(&c->d_sc->max_dispa2_bits, 0x7f, sizeof(unsigned int), s);
  c->rebuilds++;
}

// Build with a capacity check; grows the rows once if needed.  Synchronises.
ap_status build_checked(ap_ctx* c, const double* d_x, const int32_t* d_species, cudaStream_t s) {
  for (int attempt = 0; attempt < 2; ++attempt) {
    ap_status st = clear_err(c, s);
    if (st) return st;
    build_async(c, d_x, d_species, s);
    CK(cudaGetLastError());
    st = read_scalars(c, s);
    if (st) return st;
    int e = c->h_sc->err;
    if ((e & kErrCapacity) && attempt == 0 && c->cfg.cap_eam == 0) {
      c->cap_eam = c->h_sc->need_eam + 16;
      st = alloc_rows(c, true, false);
      if (st) return st;
      continue;
    }
    st = check_err_bits(c);
    if (st) return st;
    break;
  }
  c->built = true;
  return AP_OK;
}

// ACE rows of a queue whose length is the device scalar d_count (a field of
// c->d_sc), with the ACE storage sized for that length first and the pair records for
// the longest row after; grows the row capacity once on overflow.  Synchronises.
ap_status build_ace_checked(ap_ctx* c, const double* d_x, const int* d_queue, const int* d_count, cudaStream_t s) {
  const size_t off = (size_t)((const char*)d_count - (const char*)c->d_sc);
  if (off + sizeof(int) > sizeof(DevScalars)) return fail(c, AP_ERR_ARG, "queue length outside the device scalars");
  for (int attempt = 0; attempt < 2; ++attempt) {
    ap_status st = clear_err(c, s);
    if (st) return st;
    CK(cudaMemsetAsync(&c->d_sc->ace_row_max, 0, sizeof(int), s));
    st = read_scalars(c, s);
    if (st) return st;
    int m = 0;
    std::memcpy(&m, (const char*)c->h_sc + off, sizeof(int));
    st = ensure_ace_queue(c, m);
    if (st) return st;
    launch_build_ace(c, d_x, d_queue, d_count, s);
    CK(cudaGetLastError());
    st = read_scalars(c, s);
    if (st) return st;
    if ((c->h_sc->err & kErrCapacity) && attempt == 0 && c->cfg.cap_ace == 0) {
      c->cap_ace = c->h_sc->need_ace + 16;
      st = alloc_rows(c, false, true);
      if (st) return st;
      continue;
    }
    st = check_err_bits(c);
    if (st) return st;
    return ensure_ace_records(c, c->h_sc->ace_row_max);
  }
  return AP_OK;
}

// The precise queue's ACE rows were just built at the current positions: their reference
// shadows for the displacement check of the skin criterion (no-op otherwise).
void ace_ref(ap_ctx* c, cudaStream_t s) {
  if (!c->d_sh32a) return;
  cudaMemcpyAsync(c->d_sh32a, c->d_sh32, sizeof(float4) * (size_t)c->n, cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(&c->d_sc->max_dispa2_bits, 0, sizeof(unsigned int), s);
}

// Queue length from the caller's device int64, clamped to [0, n].
__global__ void k_set_count(const long long* src, int n, int* dst32, long long* dst64) {
  long long v = *src;
  v = v < 0 ? 0 : (v > n ? n : v);
  *dst32 = (int)v;
  if (dst64) *dst64 = v;
}

// Copy the caller's queue (its first *count entries only); indices outside [0, n)
// are replaced by 0 and flagged as an argument error.
__global__ void k_copy_queue(const int* __restrict__ src, const int* __restrict__ count, int n, int* __restrict__ dst,
                             DevScalars* sc) {
  const int m = *count;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
    int i = src[q];
    if (i < 0 || i >= n) {
      atomicOr(&sc->err, kErrArg);
      i = 0;
    }
    dst[q] = i;
  }
}

__global__ void k_changeable(int n, const uint8_t* fixed, uint8_t* ch) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ch[i] = fixed[i] ? 0 : 1;
}

__global__ void k_check_skin(DevScalars* sc, float limit2) {
  if (__uint_as_float(sc->max_disp2_bits) > limit2) atomicOr(&sc->err, kErrSkin);
}

__global__ void k_flag_precise(int n, const double* lam, int* flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = lam[i] < 1.0 ? 1 : 0;
}

__global__ void k_compact_q(int n, const int* flag, const int* scan, int* out, int* count32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) out[scan[i]] = i;
  if (i == 0) *count32 = scan[n];
}

__global__ void k_flag_lam(int n, const double* lam, int* flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = lam[i] < 1.0 ? 1 : 0;
}

__global__ void k_compact_q64(int n, const int* flag, const int* scan, int* out, long long* count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) out[scan[i]] = i;
  if (i == 0) *count = scan[n];
}

// Precise queue from an imported lambda (restart without a new lambda sample).
void queue_from_lambda(ap_ctx* c, cudaStream_t s) {
  int n = (int)c->n;
  k_flag_precise<<<(n + 255) / 256, 256, 0, s>>>(n, c->d_lam_int, c->d_flag);
  scan_exclusive(c->d_flag, c->d_scan, n, c->d_scan_tmp, s);
  k_compact_q<<<(n + 255) / 256, 256, 0, s>>>(n, c->d_flag, c->d_scan, c->d_precise, &c->d_sc->n_precise);
}

}  // namespace

namespace ap {
int prof_mark(ap_ctx* c, cudaStream_t s) {
  if (!c->prof_on) return -1;
  if (c->ev_used == (int)c->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev_pool.push_back(e);
  }
  const int k = c->ev_used++;
  cudaEventRecord(c->ev_pool[k], s);
  return k;
}

void prof_add(ap_ctx* c, int phase, int start, int end) {
  if (start >= 0 && end >= 0) c->ev_pairs_phase.push_back({phase, start, end});
}
}  // namespace ap

namespace {

// Event pair around one phase of ap_step (only when profiling is on).
struct PhaseTimer {
  ap_ctx* c;
  cudaStream_t s;
  int phase;
  int start;
  PhaseTimer(ap_ctx* c_, cudaStream_t s_, int phase_) : c(c_), s(s_), phase(phase_) { start = prof_mark(c, s); }
  ~PhaseTimer() {
    if (start >= 0) prof_add(c, phase, start, prof_mark(c, s));
  }
};

void collect_profile(ap_ctx* c) {
  for (auto& pr : c->ev_pairs_phase) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[pr.start], c->ev_pool[pr.end]) == cudaSuccess) {
      c->prof_ms[pr.phase] += ms;
      c->prof_calls[pr.phase] += 1;
    }
  }
  c->ev_pairs_phase.clear();
  c->ev_used = 0;
}

// Selector scratch for n atoms (features, pre-pass densities, score).
ap_status ensure_sel_feat(ap_ctx* c, int64_t n) {
  if (n <= c->sel_feat_cap && c->d_sel_feat) return AP_OK;
  CK(dalloc(c->d_sel_rho, n));
  CK(dalloc(c->d_sel_feat, 24 * n));
  CK(dalloc(c->d_sel_score, n));
  c->sel_feat_cap = n;
  return AP_OK;
}

// Local-thermostat scratch for n atoms and the sweep cells of the current box.
ap_status ensure_th(ap_ctx* c) {
  const int64_t n = c->n;
  if (n > c->th_cap || !c->d_th_lamc) {
    CK(dalloc(c->d_th_lamc, n));
    CK(dalloc(c->d_th_dlam, n));
    CK(dalloc(c->d_th_w, n));
    CK(dalloc(c->d_th_df, 3 * n));
    CK(dalloc(c->d_th_ep, n));
    CK(dalloc(c->d_th_de, n));
    CK(dalloc(c->d_th_qk, n));
    CK(dalloc(c->d_th_qe, n));
    CK(dalloc(c->d_th_cellof, n));
    CK(dalloc(c->d_th_atoms, n));
    c->th_cap = n;
  }
  const int64_t nc = th_cell_count(c);
  if (nc + 1 > c->th_cells_cap) {
    CK(dalloc(c->d_th_ccount, nc + 1));
    CK(dalloc(c->d_th_cstart, nc + 2));
    c->th_cells_cap = nc + 1;
  }
  size_t need_tmp = scan_tmp_bytes(std::max<int64_t>(nc + 1, n + 1)) / sizeof(int) + 1;
  if (need_tmp > c->scan_tmp_cap) {
    c->scan_tmp_cap = need_tmp;
    CK(dalloc(c->d_scan_tmp, need_tmp));
  }
  return AP_OK;
}

// F^c - F^d of a lambda update (linear in Delta lambda = lambda^c - lambda^d): the ACE
// part over K = {Delta lambda != 0} with weights -Delta lambda (which also gives E^p
// of K for Delta V), then the EAM part with weights Delta lambda.  Runs before the
// ACE rows of the new precise queue are built.
ap_status th_difference(ap_ctx* c, const double* d_x, cudaStream_t s) {
  const int n = (int)c->n;
  launch_th_delta(c, c->d_th_lamc, c->d_lam_int, s);
  c->kernels += scan_exclusive(c->d_flag, c->d_scan, n, c->d_scan_tmp, s) + 1;
  k_compact_q<<<(n + 255) / 256, 256, 0, s>>>(n, c->d_flag, c->d_scan, c->d_th_qk, &c->d_sc->n_th_k);
  CK(cudaMemsetAsync(c->d_th_df, 0, sizeof(double) * 3 * (size_t)n, s));
  CK(cudaMemsetAsync(c->d_th_ep, 0, sizeof(double) * (size_t)n, s));
  ap_status st = build_ace_checked(c, d_x, c->d_th_qk, &c->d_sc->n_th_k, s);
  if (st) return st;
  launch_ace(c, nullptr, c->d_th_qk, c->d_th_ep, true, s, c->d_th_w, &c->d_sc->n_th_k);
  launch_ace_finalize(c, c->d_th_df, s);
  launch_eam(c, c->d_th_dlam, nullptr, c->d_th_df, true, s);
  return AP_OK;
}

// Delta E of every mobile atom from F^d (interatomic forces only) and the queue of
// atoms with Delta E != 0.
void th_energy(ap_ctx* c, const double* d_f, const double* d_v, const double* d_mass, const uint8_t* d_fixed,
               cudaStream_t s) {
  const int n = (int)c->n;
  launch_th_energy(c, d_f, d_v, d_mass, d_fixed, s);
  c->kernels += scan_exclusive(c->d_flag, c->d_scan, n, c->d_scan_tmp, s) + 1;
  k_compact_q<<<(n + 255) / 256, 256, 0, s>>>(n, c->d_flag, c->d_scan, c->d_th_qe, &c->d_sc->n_th_e);
}

// What the configured detector needs before a classification.
ap_status prep_detector(ap_ctx* c) {
  if (c->cfg.detector != AP_DETECT_SELECTOR) return AP_OK;
  if (!c->sel_ready) return fail(c, AP_ERR_STATE, "detector = selector needs ap_sel_set_model first");
  return ensure_sel_feat(c, c->n);
}

// fresh_rows: the EAM rows were built at d_x in this call (ap_step); csp_done: d_csp
// already holds the CSP at d_x.
void classify_async(ap_ctx* c, const double* d_x, const uint8_t* d_ch, double* d_lam, int* d_queue,
                    int64_t* d_nq64, cudaStream_t s, bool fresh_rows = false, bool csp_done = false) {
  if (!csp_done) launch_csp(c, d_x, d_ch, s, fresh_rows);
  if (c->cfg.detector == AP_DETECT_SELECTOR) {
    launch_sel_features(c, c->d_sel_feat, s);
    launch_sel_mlp(c, c->n, c->d_sel_feat, nullptr, nullptr, c->d_sel_score, nullptr, nullptr, nullptr, s);
    launch_lambda0(c, d_ch, c->d_sel_score, c->cfg.sel_p_lo, c->cfg.sel_p_hi, s);
  } else {
    launch_lambda0(c, d_ch, c->d_csp, c->cfg.csp_lo, c->cfg.csp_hi, s);
  }
  launch_spread(c, d_x, d_ch, s);
  launch_lambda_final(c, d_ch, d_lam, d_queue, d_nq64, s);
}

}  // namespace

// ====================================================================== ABI
extern "C" {

ap_status ap_create(const ap_config* h_cfg, ap_ctx** out) {
  if (!h_cfg || !out) return AP_ERR_ARG;
  *out = nullptr;
  std::string why;
  if (validate(*h_cfg, why) != AP_OK) return AP_ERR_ARG;
  ap_ctx* c = new ap_ctx();
  c->cfg = *h_cfg;
  c->cap_eam = h_cfg->cap_eam ? h_cfg->cap_eam : 160;
  c->cap_ace = h_cfg->cap_ace ? h_cfg->cap_ace : 288;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete c;
    return AP_ERR_CUDA;
  }
  build_ace_tables(c->cfg, c->ace);
  if (c->cfg.ace_nc < c->ace.nb) {
    delete c;
    return AP_ERR_ARG;
  }
  if (!ace_nu3_matches(c->ace)) {   // the generated nu = 3 code is out of date
    delete c;
    return AP_ERR_STATE;
  }
  upload_ace_tables(c);
  e = cudaMalloc(&c->d_sc, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_sc, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaMemset(c->d_sc, 0, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    ap_destroy(c);
    return AP_ERR_CUDA;
  }
  std::memset(c->h_sc, 0, sizeof(DevScalars));
  *out = c;
  return AP_OK;
}

void ap_destroy(ap_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  void* ptrs[] = {c->d_sys, c->d_atom_sys, c->d_cell, c->d_cunw, c->d_cell_start, c->d_cell_count, c->d_cell_atoms,
                  c->d_slot, c->d_sh32, c->d_sh32c, c->d_sh64, c->d_sh32b, c->d_sh32a, c->d_org, c->d_vscale, c->d_nbr_eam, c->d_off_eam, c->d_cnt_eam,
                  c->d_lim_eam, c->d_split_eam, c->d_nbr_ace, c->d_off_ace, c->d_cnt_ace, c->d_csp, c->d_csp_slow, c->d_csp_avg, c->d_lam0, c->d_lam_min,
                  c->d_lam_avg, c->d_lam_prev, c->d_csp_hist, c->d_lam_hist, c->d_flag, c->d_scan, c->d_detected, c->d_vmin_f, c->d_det1,
                  c->d_precise, c->d_lam_int, c->d_q, c->d_xi, c->d_facc32, c->d_facc64, c->d_faccfix, c->d_efast, c->d_eprec,
                  c->d_eatom, c->d_eext, c->d_changeable, c->d_W32, c->d_W64, c->d_ace_list, c->d_ace_nin,
                  c->d_ace_a48, c->d_ace_dA, c->d_ace_e12, c->d_ace_de3, c->d_ace_e3, c->d_ace_dAb, c->d_ace_e12b,
                  c->d_ace_fs, c->d_scan_tmp, c->d_red,
                  c->d_sel_model, c->d_sel_master, c->d_sel_m1, c->d_sel_m2, c->d_sel_grad, c->d_sel_partial,
                  c->d_sel_rho, c->d_sel_feat, c->d_sel_score, c->d_sel_z, c->d_sel_h1, c->d_sel_h2,
                  c->d_th_lamc, c->d_th_dlam, c->d_th_w, c->d_th_df, c->d_th_ep, c->d_th_de, c->d_th_qk, c->d_th_qe,
                  c->d_th_cellof, c->d_th_atoms, c->d_th_ccount, c->d_th_cstart, c->d_sc};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_sc) cudaFreeHost(c->h_sc);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

const char* ap_last_error(const ap_ctx* c) { return c ? c->err_msg.c_str() : "null context"; }

int64_t ap_need(const ap_ctx* c) { return c ? c->need : 0; }

static const AceTables& default_tables() {
  static AceTables t;
  static bool done = false;
  if (!done) {
    ap_config g;
    std::memset(&g, 0, sizeof(g));
    build_ace_tables(g, t);
    done = true;
  }
  return t;
}

int32_t ap_ace_nbasis(const ap_ctx* c) { return c ? c->ace.nb : default_tables().nb; }

ap_status ap_ace_basis_desc(const ap_ctx* c, int32_t* h_desc) {
  if (!h_desc) return AP_ERR_ARG;
  const AceTables& t = c ? c->ace : default_tables();
  std::memcpy(h_desc, t.desc.data(), sizeof(int32_t) * t.desc.size());
  return AP_OK;
}

ap_status ap_ace_gaunt(const ap_ctx* c, double* h_out) {
  if (!h_out) return AP_ERR_ARG;
  const AceTables& t = c ? c->ace : default_tables();
  std::memcpy(h_out, t.gaunt.data(), sizeof(double) * t.gaunt.size());
  return AP_OK;
}

ap_status ap_build_neighbors_batch(ap_ctx* c, int32_t n_sys, const int64_t* h_offsets, const ap_box* h_boxes,
                                   const double* d_x, const int32_t* d_species, void* stream) {
  if (!c) return AP_ERR_ARG;
  if (n_sys < 1 || !h_offsets || !h_boxes) return fail(c, AP_ERR_ARG, "need n_sys >= 1, offsets and boxes");
  if (h_offsets[0] != 0) return fail(c, AP_ERR_ARG, "offsets must start at 0");
  for (int s = 0; s < n_sys; ++s)
    if (h_offsets[s + 1] < h_offsets[s]) return fail(c, AP_ERR_ARG, "offsets must be non-decreasing");
  int64_t n = h_offsets[n_sys];
  if (n > 0 && !d_x) return fail(c, AP_ERR_ARG, "null positions");
  ap_status st = set_systems(c, n_sys, h_offsets, h_boxes);
  if (st) return st;
  st = ensure_capacity(c, n);
  if (st) return st;
  if (n != c->n) {
    c->hist_started = false;
    c->lam_ready = false;
    c->md_ready = false;
  }
  c->n = n;
  if (n == 0) {
    c->built = true;
    return AP_OK;
  }
  return build_checked(c, d_x, d_species, S(stream));
}

ap_status ap_build_neighbors(ap_ctx* c, int64_t n, const double* d_x, const int32_t* d_species, const ap_box* h_box,
                             void* stream) {
  if (!c) return AP_ERR_ARG;
  if (n < 0 || !h_box) return fail(c, AP_ERR_ARG, "need n >= 0 and a box");
  int64_t off[2] = {0, n};
  return ap_build_neighbors_batch(c, 1, off, h_box, d_x, d_species, stream);
}

ap_status ap_get_neighbors(ap_ctx* c, int32_t which, int32_t* d_cnt, int32_t* d_idx, int32_t* d_shift, int64_t cap,
                           int64_t* h_rows) {
  if (!c) return AP_ERR_ARG;
  if (!c->built) return fail(c, AP_ERR_STATE, "no neighbour build yet");
  if (which != 0 && which != 1) return fail(c, AP_ERR_ARG, "which must be 0 (EAM) or 1 (ACE)");
  ap_status st = read_scalars(c, 0);
  if (st) return st;
  int64_t rows = which == 0 ? c->n : c->h_sc->n_precise;
  if (h_rows) *h_rows = rows;
  if (rows > 0 && (!d_cnt || !d_idx || !d_shift || cap <= 0)) return fail(c, AP_ERR_ARG, "null output or cap <= 0");
  launch_export_rows(c, which, (int)rows, (int)cap, d_cnt, d_idx, d_shift, 0);
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  return AP_OK;
}

ap_status ap_spatial_order(ap_ctx* c, int32_t* d_order, void* stream) {
  if (!c) return AP_ERR_ARG;
  if (!c->built) return fail(c, AP_ERR_STATE, "no neighbour build yet");
  if (!d_order) return fail(c, AP_ERR_ARG, "null order");
  if (c->n > 0)
    CK(cudaMemcpyAsync(d_order, c->d_cell_atoms, sizeof(int) * (size_t)c->n, cudaMemcpyDeviceToDevice, S(stream)));
  return AP_OK;
}

ap_status ap_neighbor_total(ap_ctx* c, int32_t which, int64_t* h_total) {
  if (!c) return AP_ERR_ARG;
  if (!h_total) return fail(c, AP_ERR_ARG, "null argument");
  if (!c->built) return fail(c, AP_ERR_STATE, "no neighbour build yet");
  if (which < 0 || which > 2) return fail(c, AP_ERR_ARG, "which must be 0 (EAM), 1 (ACE) or 2 (EAM force prefixes)");
  if (which == 2 && !c->lim_valid) return fail(c, AP_ERR_STATE, "no EAM evaluation on the current rows");
  ap_status st = read_scalars(c, 0);
  if (st) return st;
  const int64_t rows = which == 1 ? c->h_sc->n_precise : c->n;
  launch_row_total(c, which, (int)rows, 0);
  unsigned long long t = 0;
  CK(cudaMemcpy(&t, &c->d_sc->row_total, sizeof(t), cudaMemcpyDeviceToHost));
  CK(cudaGetLastError());
  *h_total = (int64_t)t;
  return AP_OK;
}

ap_status ap_classify(ap_ctx* c, int64_t n, const double* d_x, const uint8_t* d_changeable, int32_t sample_now,
                      double* d_lam, int32_t* d_precise_idx, int64_t* d_n_precise, void* stream) {
  if (!c) return AP_ERR_ARG;
  if (!c->built || n != c->n) return fail(c, AP_ERR_STATE, "ap_classify needs ap_build_neighbors on the same atoms");
  if (n > 0 && (!d_x || !d_lam || !d_precise_idx)) return fail(c, AP_ERR_ARG, "null argument");
  cudaStream_t s = S(stream);
  if (n == 0) {
    if (d_n_precise) CK(cudaMemsetAsync(d_n_precise, 0, sizeof(int64_t), s));
    CK(cudaMemsetAsync(&c->d_sc->n_precise, 0, sizeof(int), s));
    return AP_OK;
  }
  if (!sample_now) {   // no new sample: the lambda of the last update and its queue
    if (!c->lam_ready || !c->hist_started)
      return fail(c, AP_ERR_STATE, "ap_classify with sample_now = 0 needs an earlier classification");
    const int nn = (int)n;
    CK(cudaMemcpyAsync(d_lam, c->d_lam_prev, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    k_flag_lam<<<(nn + 255) / 256, 256, 0, s>>>(nn, d_lam, c->d_flag);
    scan_exclusive(c->d_flag, c->d_scan, nn, c->d_scan_tmp, s);
    k_compact_q64<<<(nn + 255) / 256, 256, 0, s>>>(
        nn, c->d_flag, c->d_scan, d_precise_idx, d_n_precise ? (long long*)d_n_precise : &c->d_sc->n_precise64);
    CK(cudaGetLastError());
    return AP_OK;
  }
  ap_status st = prep_detector(c);
  if (st) return st;
  launch_shadow(c, d_x, s);
  classify_async(c, d_x, d_changeable, d_lam, d_precise_idx, d_n_precise, s);
  CK(cudaGetLastError());
  c->lam_ready = true;
  return AP_OK;
}

ap_status ap_precise_queue(ap_ctx* c, int64_t n, const double* d_lam, int32_t* d_queue, int64_t* d_n_queue,
                           void* stream) {
  if (!c) return AP_ERR_ARG;
  if (n < 0 || !d_n_queue || (n > 0 && (!d_lam || !d_queue))) return fail(c, AP_ERR_ARG, "null argument");
  if (n > c->n_cap) return fail(c, AP_ERR_STATE, "ap_precise_queue needs a neighbour build on at least n atoms");
  cudaStream_t s = S(stream);
  if (n == 0) {
    CK(cudaMemsetAsync(d_n_queue, 0, sizeof(int64_t), s));
    return AP_OK;
  }
  const int nn = (int)n;
  k_flag_lam<<<(nn + 255) / 256, 256, 0, s>>>(nn, d_lam, c->d_flag);
  scan_exclusive(c->d_flag, c->d_scan, nn, c->d_scan_tmp, s);
  k_compact_q64<<<(nn + 255) / 256, 256, 0, s>>>(nn, c->d_flag, c->d_scan, d_queue, (long long*)d_n_queue);
  CK(cudaGetLastError());
  return AP_OK;
}

ap_status ap_reset_lambda(ap_ctx* c) {
  if (!c) return AP_ERR_ARG;
  c->hist_started = false;
  c->csp_pos = c->lam_pos = -1;
  c->lam_ready = false;
  c->md_ready = false;
  return AP_OK;
}

ap_status ap_get_lambda_state(ap_ctx* c, double* d_csp, double* d_csp_avg, double* d_lam0, double* d_lam_min,
                              double* d_lam_avg, void* stream) {
  if (!c) return AP_ERR_ARG;
  if (!c->lam_ready) return fail(c, AP_ERR_STATE, "no classification yet");
  cudaStream_t s = S(stream);
  size_t b = sizeof(double) * (size_t)c->n;
  if (b == 0) return AP_OK;
  if (d_csp) CK(cudaMemcpyAsync(d_csp, c->d_csp, b, cudaMemcpyDeviceToDevice, s));
  if (d_csp_avg) CK(cudaMemcpyAsync(d_csp_avg, c->d_csp_avg, b, cudaMemcpyDeviceToDevice, s));
  if (d_lam0) CK(cudaMemcpyAsync(d_lam0, c->d_lam0, b, cudaMemcpyDeviceToDevice, s));
  if (d_lam_min) CK(cudaMemcpyAsync(d_lam_min, c->d_lam_min, b, cudaMemcpyDeviceToDevice, s));
  if (d_lam_avg) CK(cudaMemcpyAsync(d_lam_avg, c->d_lam_avg, b, cudaMemcpyDeviceToDevice, s));
  return AP_OK;
}

ap_status ap_eval_eam(ap_ctx* c, int64_t n, const double* d_x, const double* d_lam, double* d_e_fast, double* d_f,
                      float* d_feat, void* stream) {
  if (!c) return AP_ERR_ARG;
  if (!c->built || n != c->n) return fail(c, AP_ERR_STATE, "ap_eval_eam needs ap_build_neighbors on the same atoms");
  if (n == 0) return AP_OK;
  if (!d_x || !d_e_fast || !d_f) return fail(c, AP_ERR_ARG, "null argument");
  if (d_feat && c->cfg.eam_type != AP_EAM_ANALYTIC)
    return fail(c, AP_ERR_ARG, "selector features need eam_type AP_EAM_ANALYTIC");
  cudaStream_t s = S(stream);
  launch_shadow(c, d_x, s);
  launch_eam(c, d_lam, d_e_fast, d_f, true, s);
  if (d_feat) {   // the selector's EAM-level features from the same rows and shadows
    ap_status st = ensure_sel_feat(c, n);
    if (st) return st;
    launch_csp(c, d_x, nullptr, s);
    launch_sel_features(c, d_feat, s);
  }
  CK(cudaGetLastError());
  return AP_OK;
}

ap_status ap_eval_ace(ap_ctx* c, int64_t n, const double* d_x, const double* d_lam, const int32_t* d_precise_idx,
                      const int64_t* d_n_precise, double* d_e_prec, double* d_f, void* stream) {
  if (!c) return AP_ERR_ARG;
  if (!c->built || n != c->n) return fail(c, AP_ERR_STATE, "ap_eval_ace needs ap_build_neighbors on the same atoms");
  if (n == 0) return AP_OK;
  if (!d_x || !d_precise_idx || !d_n_precise || !d_e_prec) return fail(c, AP_ERR_ARG, "null argument");
  cudaStream_t s = S(stream);
  launch_shadow(c, d_x, s);
  k_set_count<<<1, 1, 0, s>>>((const long long*)d_n_precise, (int)n, &c->d_sc->n_precise, &c->d_sc->n_precise64);
  k_copy_queue<<<c->num_sms * 4, 256, 0, s>>>(d_precise_idx, &c->d_sc->n_precise, (int)n, c->d_precise, c->d_sc);
  ap_status st = build_ace_checked(c, d_x, c->d_precise, &c->d_sc->n_precise, s);
  if (st) return st;
  CK(cudaMemsetAsync(d_e_prec, 0, sizeof(double) * (size_t)n, s));
  launch_ace(c, d_lam, c->d_precise, d_e_prec, d_f != nullptr, s);
  if (d_f) launch_ace_finalize(c, d_f, s);
  CK(cudaGetLastError());
  return AP_OK;
}

ap_status ap_blend_forces(ap_ctx* c, int64_t n, const double* d_lam, const double* d_e_fast, const double* d_e_prec,
                          double* d_e_atom, double* d_e_total, void* stream) {
  if (!c) return AP_ERR_ARG;
  if (n != c->n) return fail(c, AP_ERR_STATE, "n differs from the last neighbour build");
  if (!d_e_fast || !d_e_total) return fail(c, AP_ERR_ARG, "null argument");
  cudaStream_t s = S(stream);
  launch_blend(c, d_lam, d_e_fast, d_e_prec, nullptr, d_e_atom, d_e_total, s);
  CK(cudaGetLastError());
  return AP_OK;
}

ap_status ap_step(ap_ctx* c, int64_t n, double* d_x, double* d_v, double* d_f, const double* d_mass,
                  const uint8_t* d_fixed, double* d_lam, int64_t nsteps, ap_step_stats* h_stats, void* stream) {
  if (!c) return AP_ERR_ARG;
  if (nsteps < 0) return fail(c, AP_ERR_ARG, "nsteps < 0");
  if (!c->n_sys || n != c->n) return fail(c, AP_ERR_STATE, "ap_step needs ap_build_neighbors on the same atoms");
  if (n == 0) return AP_OK;
  if (!d_x || !d_v || !d_f || !d_mass || !d_lam) return fail(c, AP_ERR_ARG, "null argument");
  if (!(c->cfg.dt > 0)) return fail(c, AP_ERR_ARG, "dt must be positive");
  cudaStream_t s = S(stream);
  const uint8_t* ch = nullptr;
  if (d_fixed) {
    k_changeable<<<(int)((n + 255) / 256), 256, 0, s>>>((int)n, d_fixed, c->d_changeable);
    c->kernels += 1;
    ch = c->d_changeable;
  }
  const ap_config& g = c->cfg;
  ap_status st = prep_detector(c);
  if (st) return st;
  const bool thermo = g.thermostat_on != 0;
  if (thermo) {
    if (c->n_sys != 1) return fail(c, AP_ERR_ARG, "the local thermostat needs a single system");
    st = ensure_th(c);
    if (st) return st;
  }
  if (!c->md_ready) {
    launch_wrap_positions(c, d_x, s);
    st = build_checked(c, d_x, nullptr, s);
    if (st) return st;
    if (c->restart_pending) {
      queue_from_lambda(c, s);
      c->restart_pending = false;
    } else {
      classify_async(c, d_x, ch, c->d_lam_int, c->d_precise, nullptr, s, true);
    }
    st = build_ace_checked(c, d_x, c->d_precise, &c->d_sc->n_precise, s);
    if (st) return st;
    ace_ref(c, s);
    CK(cudaMemsetAsync(c->d_eprec, 0, sizeof(double) * (size_t)n, s));
    launch_eam(c, c->d_lam_int, c->d_efast, d_f, false, s);
    launch_ace(c, c->d_lam_int, c->d_precise, c->d_eprec, true, s);
    launch_ace_finalize(c, d_f, s);
    if (g.indenter_on) launch_indenter(c, d_x, d_f, c->step * g.dt, s);
    c->lam_ready = true;
    c->md_ready = true;
  }
  st = clear_err(c, s);
  if (st) return st;
  const float skin_lim2 = (float)(0.25 * g.skin * g.skin);
  // Skin criterion: the lists are checked after every drift; a lambda update keeps them
  // (stale cells and rows) where the detector and the box allow it.
  const bool skin_rule = g.rebuild_every == AP_REBUILD_SKIN;
  const bool keep_ok = skin_rule && c->stale_ok && g.detector == AP_DETECT_CSP && !thermo;
  if (nsteps > 0) {
    PhaseTimer t(c, s, AP_PHASE_OTHER);
    launch_vscale(c, d_mass, s);   // the half-kick factors of this call's masses
  }
  for (int64_t k = 0; k < nsteps; ++k) {
    c->step++;
    {
      PhaseTimer t(c, s, AP_PHASE_OTHER);
      launch_vv_first(c, d_x, d_v, d_f, d_mass, d_fixed, s);
    }
    const bool lam_step = c->step % g.lambda_every == 0;
    bool build = false, keep = false, ace_only = false;
    double m = 0.0;   // the largest displacement since the last build (skin criterion)
    if (skin_rule) {
      PhaseTimer t(c, s, AP_PHASE_NEIGHBORS);
      st = read_scalars(c, s);   // an error so far (non-finite position) ends the call here
      if (st) return st;
      st = check_err_bits(c);
      if (st) return st;
      float d2, d2a;
      std::memcpy(&d2, &c->h_sc->max_disp2_bits, sizeof(float));
      std::memcpy(&d2a, &c->h_sc->max_dispa2_bits, sizeof(float));
      // from FP32 shadows (a few 1e-7 A per component): headroom
      m = std::sqrt((double)d2) * (1.0 + 1e-5) + 1e-5;
      const double ma = std::sqrt((double)d2a) * (1.0 + 1e-5) + 1e-5;   // since the ACE row build
      build = m > 0.5 * g.skin;
      keep = lam_step && !build && keep_ok && m <= kKeepFrac * g.skin;
      build = build || (lam_step && !keep);
      // the ACE rows reach ace_rc + skin at their build: rebuilt alone when an atom has moved
      // more than skin/2 since then while the EAM lists still hold (from their cells, m old)
      if (!build && !lam_step && ma > 0.5 * g.skin) {
        if (c->stale_ok) ace_only = true;
        else build = true;
      }
    } else {
      const int rb = g.rebuild_every > 0 ? g.rebuild_every : g.lambda_every;
      build = lam_step || c->step % rb == 0;
    }
    if (build || lam_step) {
      if (build) {
        PhaseTimer t(c, s, AP_PHASE_NEIGHBORS);
        if (!skin_rule) {
          k_check_skin<<<1, 1, 0, s>>>(c->d_sc, skin_lim2);
          c->kernels += 1;
          // an error so far (skin, non-finite position) ends the call here
          st = read_scalars(c, s);
          if (st) return st;
          st = check_err_bits(c);
          if (st) return st;
        }
        launch_wrap_positions(c, d_x, s);
        st = build_checked(c, d_x, nullptr, s);   // grows the EAM rows if one overflows
        if (st) return st;
      }
      bool csp_done = false;
      if (keep) {   // CSP from the kept rows; any atom they cannot decide sends the update to a rebuild
        PhaseTimer t(c, s, AP_PHASE_CLASSIFY);
        launch_csp(c, d_x, ch, s, false, m);   // the drift wrote the shadows of d_x
        st = read_scalars(c, s);
        if (st) return st;
        if (c->h_sc->n_stale_bad == 0) {
          c->cells_stale = true;
          c->stale_m = m;
          c->kept++;
          csp_done = true;
        } else {
          PhaseTimer t2(c, s, AP_PHASE_NEIGHBORS);
          launch_wrap_positions(c, d_x, s);
          st = build_checked(c, d_x, nullptr, s);
          if (st) return st;
          keep = false;
        }
      }
      {
        PhaseTimer t(c, s, AP_PHASE_CLASSIFY);
        if (lam_step) {
          if (thermo)
            CK(cudaMemcpyAsync(c->d_th_lamc, c->d_lam_int, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
          classify_async(c, d_x, ch, c->d_lam_int, c->d_precise, nullptr, s, !keep, csp_done);
        }
      }
      if (lam_step && thermo) {
        PhaseTimer t(c, s, AP_PHASE_THERMOSTAT);
        st = th_difference(c, d_x, s);
        if (st) return st;
      }
      {
        PhaseTimer t(c, s, AP_PHASE_CLASSIFY);
        // the new queue's ACE rows, with its storage sized first (synchronises)
        st = build_ace_checked(c, d_x, c->d_precise, &c->d_sc->n_precise, s);
        if (st) return st;
        ace_ref(c, s);
      }
    } else if (ace_only) {
      PhaseTimer t(c, s, AP_PHASE_NEIGHBORS);
      c->cells_stale = true;   // the atoms moved up to m since the cell build
      c->stale_m = m;
      st = build_ace_checked(c, d_x, c->d_precise, &c->d_sc->n_precise, s);
      if (st) return st;
      ace_ref(c, s);
      c->ace_rebuilds++;
    }
    {
      PhaseTimer t(c, s, AP_PHASE_EAM);
      launch_eam(c, c->d_lam_int, c->d_efast, d_f, false, s);
    }
    {
      PhaseTimer t(c, s, AP_PHASE_ACE);
      CK(cudaMemsetAsync(c->d_eprec, 0, sizeof(double) * (size_t)n, s));
      launch_ace(c, c->d_lam_int, c->d_precise, c->d_eprec, true, s);
    }
    {
      PhaseTimer t(c, s, AP_PHASE_OTHER);
      launch_ace_finalize(c, d_f, s);
    }
    if (lam_step && thermo) {   // Delta E from the interatomic forces, before the external force
      PhaseTimer t(c, s, AP_PHASE_THERMOSTAT);
      th_energy(c, d_f, d_v, d_mass, d_fixed, s);
    }
    {
      PhaseTimer t(c, s, AP_PHASE_OTHER);
      if (g.indenter_on) launch_indenter(c, d_x, d_f, c->step * g.dt, s);
      launch_vv_second(c, d_v, d_f, d_mass, d_fixed, s);
    }
    if (lam_step && thermo) {   // corrections of v(t + dt)
      PhaseTimer t(c, s, AP_PHASE_THERMOSTAT);
      launch_th_correct(c, c->d_th_qe, &c->d_sc->n_th_e, d_x, d_fixed, d_mass, d_v, s);
    }
  }
  {
    PhaseTimer t(c, s, AP_PHASE_OTHER);
    k_check_skin<<<1, 1, 0, s>>>(c->d_sc, skin_lim2);
    c->kernels += 1;
    launch_blend(c, c->d_lam_int, c->d_efast, c->d_eprec, g.indenter_on ? c->d_eext : nullptr, c->d_eatom,
                 &c->d_sc->e_total, s);
    launch_kinetic(c, d_v, d_mass, &c->d_sc->e_kin, s);
  }
  CK(cudaMemcpyAsync(d_lam, c->d_lam_int, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  CK(cudaGetLastError());
  st = read_scalars(c, s);
  if (st) return st;
  collect_profile(c);
  if (h_stats) {
    h_stats->step = c->step;
    h_stats->n_precise = c->h_sc->n_precise;
    h_stats->n_detected = c->h_sc->n_detected;
    h_stats->rebuilds = c->rebuilds;
    h_stats->e_pot = c->h_sc->e_total;
    h_stats->e_kin = c->h_sc->e_kin;
    float d2;
    std::memcpy(&d2, &c->h_sc->max_disp2_bits, sizeof(float));
    h_stats->max_disp = std::sqrt((double)d2);
    h_stats->error_bits = c->h_sc->err;
    h_stats->th_corrected = (int64_t)c->h_sc->th_n;
    h_stats->th_refused = (int64_t)c->h_sc->th_bad;
    h_stats->th_energy = c->h_sc->th_e;
    h_stats->kept = c->kept;
    h_stats->ace_rebuilds = c->ace_rebuilds;
  }
  return check_err_bits(c);
}

// ---------------------------------------------------------------------- selector
ap_status ap_sel_set_model(ap_ctx* c, const float* h_params, const float* h_mu, const float* h_inv_sigma) {
  if (!c) return AP_ERR_ARG;
  if (!h_params || !h_mu || !h_inv_sigma) return fail(c, AP_ERR_ARG, "null model array");
  for (int k = 0; k < AP_SEL_NPARAMS; ++k)
    if (!std::isfinite(h_params[k])) return fail(c, AP_ERR_ARG, "non-finite model parameter");
  for (int k = 0; k < AP_SEL_NFEAT; ++k)
    if (!std::isfinite(h_mu[k]) || !std::isfinite(h_inv_sigma[k])) return fail(c, AP_ERR_ARG, "non-finite mu or inv_sigma");
  CK(sel_mlp_attr());
  if (!c->d_sel_model) {
    CK(dalloc(c->d_sel_model, 1));
    CK(dalloc(c->d_sel_master, AP_SEL_NPARAMS));
    CK(dalloc(c->d_sel_m1, AP_SEL_NPARAMS));
    CK(dalloc(c->d_sel_m2, AP_SEL_NPARAMS));
    CK(dalloc(c->d_sel_grad, AP_SEL_NPARAMS + 1));
    CK(dalloc(c->d_sel_partial, sel_partial_floats(c)));
  }
  CK(cudaDeviceSynchronize());
  CK(cudaMemset(c->d_sel_model, 0, sizeof(SelDev)));
  CK(cudaMemset(c->d_sel_m1, 0, sizeof(float) * AP_SEL_NPARAMS));
  CK(cudaMemset(c->d_sel_m2, 0, sizeof(float) * AP_SEL_NPARAMS));
  CK(cudaMemset(c->d_sel_grad, 0, sizeof(float) * (AP_SEL_NPARAMS + 1)));
  CK(cudaMemcpy(c->d_sel_master, h_params, sizeof(float) * AP_SEL_NPARAMS, cudaMemcpyHostToDevice));
  float* vec = reinterpret_cast<float*>(reinterpret_cast<char*>(c->d_sel_model) + offsetof(SelDev, vec));
  CK(cudaMemcpy(vec + SelDev::kMu, h_mu, sizeof(float) * AP_SEL_NFEAT, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(vec + SelDev::kInvS, h_inv_sigma, sizeof(float) * AP_SEL_NFEAT, cudaMemcpyHostToDevice));
  launch_sel_adam(c, false, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, 0);
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  c->sel_ready = true;
  c->sel_t = 0;
  return AP_OK;
}

ap_status ap_sel_get_model(ap_ctx* c, float* h_params, float* h_mu, float* h_inv_sigma) {
  if (!c) return AP_ERR_ARG;
  if (!c->sel_ready) return fail(c, AP_ERR_STATE, "no selector model");
  CK(cudaDeviceSynchronize());
  const float* vec = reinterpret_cast<const float*>(reinterpret_cast<const char*>(c->d_sel_model) + offsetof(SelDev, vec));
  if (h_params) CK(cudaMemcpy(h_params, c->d_sel_master, sizeof(float) * AP_SEL_NPARAMS, cudaMemcpyDeviceToHost));
  if (h_mu) CK(cudaMemcpy(h_mu, vec + SelDev::kMu, sizeof(float) * AP_SEL_NFEAT, cudaMemcpyDeviceToHost));
  if (h_inv_sigma) CK(cudaMemcpy(h_inv_sigma, vec + SelDev::kInvS, sizeof(float) * AP_SEL_NFEAT, cudaMemcpyDeviceToHost));
  return AP_OK;
}

ap_status ap_sel_features(ap_ctx* c, int64_t n, const double* d_x, const uint8_t* d_changeable, float* d_feat,
                          void* stream) {
  if (!c) return AP_ERR_ARG;
  if (!c->built || n != c->n) return fail(c, AP_ERR_STATE, "ap_sel_features needs ap_build_neighbors on the same atoms");
  if (c->cfg.eam_type != AP_EAM_ANALYTIC) return fail(c, AP_ERR_ARG, "selector features need eam_type AP_EAM_ANALYTIC");
  if (n == 0) return AP_OK;
  if (!d_x || !d_feat) return fail(c, AP_ERR_ARG, "null argument");
  ap_status st = ensure_sel_feat(c, n);
  if (st) return st;
  cudaStream_t s = S(stream);
  launch_shadow(c, d_x, s);
  launch_csp(c, d_x, d_changeable, s);
  launch_sel_features(c, d_feat, s);
  CK(cudaGetLastError());
  return AP_OK;
}

ap_status ap_sel_predict(ap_ctx* c, int64_t n, const float* d_feat, float* d_p, float* d_logit, void* stream) {
  if (!c) return AP_ERR_ARG;
  if (!c->sel_ready) return fail(c, AP_ERR_STATE, "no selector model");
  if (n < 0 || n > 0x7fffffff) return fail(c, AP_ERR_ARG, "n out of range");
  if (n == 0) return AP_OK;
  if (!d_feat) return fail(c, AP_ERR_ARG, "null features");
  launch_sel_mlp(c, n, d_feat, nullptr, d_p, nullptr, d_logit, nullptr, nullptr, S(stream));
  CK(cudaGetLastError());
  return AP_OK;
}

ap_status ap_sel_train_step(ap_ctx* c, int64_t b, const float* d_feat, const int32_t* d_idx, const float* d_label,
                            const float* d_weight, float lr, float beta1, float beta2, float eps, float* d_loss,
                            void* stream) {
  if (!c) return AP_ERR_ARG;
  if (!c->sel_ready) return fail(c, AP_ERR_STATE, "no selector model");
  if (b < 1 || b > 0x7fffffff / 64) return fail(c, AP_ERR_ARG, "batch size out of range");
  if (!d_feat || !d_label || !d_weight) return fail(c, AP_ERR_ARG, "null argument");
  if (!(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return fail(c, AP_ERR_ARG, "bad Adam hyper-parameters");
  cudaStream_t s = S(stream);
  if (b > c->sel_train_cap) {
    CK(cudaStreamSynchronize(s));
    CK(dalloc(c->d_sel_z, b));
    float* h1 = nullptr;
    if (c->d_sel_h1) cudaFree(c->d_sel_h1);
    c->d_sel_h1 = nullptr;
    CK(cudaMalloc((void**)&h1, sizeof(uint16_t) * 64 * (size_t)b));
    c->d_sel_h1 = h1;
    CK(dalloc(c->d_sel_h2, 64 * (size_t)b));
    c->sel_train_cap = b;
  }
  launch_sel_mlp(c, b, d_feat, d_idx, nullptr, nullptr, c->d_sel_z, c->d_sel_h1, c->d_sel_h2, s);
  launch_sel_backward(c, b, d_feat, d_idx, d_label, d_weight, s);
  c->sel_t += 1;
  const double bc1 = 1.0 - std::pow((double)beta1, (double)c->sel_t);
  const double bc2 = 1.0 - std::pow((double)beta2, (double)c->sel_t);
  launch_sel_adam(c, true, lr, beta1, beta2, eps, (float)(1.0 / bc1), (float)(1.0 / bc2), s);
  if (d_loss) CK(cudaMemcpyAsync(d_loss, c->d_sel_grad + AP_SEL_NPARAMS, sizeof(float), cudaMemcpyDeviceToDevice, s));
  CK(cudaGetLastError());
  return AP_OK;
}

ap_status ap_sel_get_grad(ap_ctx* c, float* h_grad, float* h_loss) {
  if (!c) return AP_ERR_ARG;
  if (!c->sel_ready) return fail(c, AP_ERR_STATE, "no selector model");
  CK(cudaDeviceSynchronize());
  if (h_grad) CK(cudaMemcpy(h_grad, c->d_sel_grad, sizeof(float) * AP_SEL_NPARAMS, cudaMemcpyDeviceToHost));
  if (h_loss) CK(cudaMemcpy(h_loss, c->d_sel_grad + AP_SEL_NPARAMS, sizeof(float), cudaMemcpyDeviceToHost));
  ap_status st = read_scalars(c, 0);
  if (st) return st;
  return check_err_bits(c);
}

ap_status ap_profile_enable(ap_ctx* c, int32_t on) {
  if (!c) return AP_ERR_ARG;
  c->prof_on = on != 0;
  for (int p = 0; p < AP_NUM_PHASES; ++p) {
    c->prof_ms[p] = 0.0;
    c->prof_calls[p] = 0;
  }
  c->ev_pairs_phase.clear();
  c->ev_used = 0;
  c->kernels = 0;
  CK(cudaDeviceSynchronize());
  CK(cudaMemset(&c->d_sc->ace_pairs, 0, 3 * sizeof(unsigned long long)));
  c->h_sc->ace_pairs = c->h_sc->ace_atoms = c->h_sc->ace_mma = 0;
  return AP_OK;
}

ap_status ap_profile_read(ap_ctx* c, double* h_ms, int64_t* h_calls, int64_t* h_kernels, int64_t* h_ace_pairs,
                          int64_t* h_ace_atoms) {
  if (!c) return AP_ERR_ARG;
  for (int p = 0; p < AP_NUM_PHASES; ++p) {
    if (h_ms) h_ms[p] = c->prof_ms[p];
    if (h_calls) h_calls[p] = c->prof_calls[p];
  }
  if (h_kernels) *h_kernels = c->kernels;
  if (h_ace_pairs) *h_ace_pairs = (int64_t)c->h_sc->ace_pairs;
  if (h_ace_atoms) *h_ace_atoms = (int64_t)c->h_sc->ace_atoms;
  return AP_OK;
}

ap_status ap_profile_mma(ap_ctx* c, int64_t* h_mma) {
  if (!c || !h_mma) return AP_ERR_ARG;
  *h_mma = (int64_t)c->h_sc->ace_mma;
  return AP_OK;
}

ap_status ap_state_export(ap_ctx* c, void* h_buf, size_t* h_len) {
  if (!c || !h_len) return AP_ERR_ARG;
  const size_t n = (size_t)c->n;
  const size_t hdr = 8 * sizeof(int64_t);
  const size_t body = sizeof(double) * n * ((size_t)c->cfg.n_csp_avg + c->cfg.n_lam_avg + 2);
  if (!h_buf) {
    *h_len = hdr + body;
    return AP_OK;
  }
  if (*h_len < hdr + body) return fail(c, AP_ERR_ARG, "buffer too small");
  CK(cudaDeviceSynchronize());
  int64_t* h = (int64_t*)h_buf;
  h[0] = 0x41505354;  // "APST"
  h[1] = (int64_t)n;
  h[2] = c->cfg.n_csp_avg;
  h[3] = c->cfg.n_lam_avg;
  h[4] = c->csp_pos;
  h[5] = c->lam_pos;
  h[6] = c->hist_started ? 1 : 0;
  h[7] = c->step;
  char* p = (char*)h_buf + hdr;
  if (n) {
    CK(cudaMemcpy(p, c->d_csp_hist, sizeof(double) * n * c->cfg.n_csp_avg, cudaMemcpyDeviceToHost));
    p += sizeof(double) * n * c->cfg.n_csp_avg;
    CK(cudaMemcpy(p, c->d_lam_hist, sizeof(double) * n * c->cfg.n_lam_avg, cudaMemcpyDeviceToHost));
    p += sizeof(double) * n * c->cfg.n_lam_avg;
    CK(cudaMemcpy(p, c->d_lam_prev, sizeof(double) * n, cudaMemcpyDeviceToHost));
    p += sizeof(double) * n;
    CK(cudaMemcpy(p, c->d_lam_int, sizeof(double) * n, cudaMemcpyDeviceToHost));
  }
  *h_len = hdr + body;
  return AP_OK;
}

ap_status ap_state_import(ap_ctx* c, const void* h_buf, size_t h_len) {
  if (!c || !h_buf) return AP_ERR_ARG;
  const int64_t* h = (const int64_t*)h_buf;
  const size_t hdr = 8 * sizeof(int64_t);
  if (h_len < hdr || h[0] != 0x41505354) return fail(c, AP_ERR_ARG, "not an ap state buffer");
  const size_t n = (size_t)h[1];
  if ((int64_t)n != c->n) return fail(c, AP_ERR_STATE, "state was saved for a different atom count");
  if (h[2] != c->cfg.n_csp_avg || h[3] != c->cfg.n_lam_avg) return fail(c, AP_ERR_ARG, "window sizes differ");
  const size_t body = sizeof(double) * n * ((size_t)c->cfg.n_csp_avg + c->cfg.n_lam_avg + 2);
  if (h_len < hdr + body) return fail(c, AP_ERR_ARG, "buffer too small");
  c->csp_pos = (int)h[4];
  c->lam_pos = (int)h[5];
  c->hist_started = h[6] != 0;
  c->step = h[7];
  const char* p = (const char*)h_buf + hdr;
  if (n) {
    CK(cudaMemcpy(c->d_csp_hist, p, sizeof(double) * n * c->cfg.n_csp_avg, cudaMemcpyHostToDevice));
    p += sizeof(double) * n * c->cfg.n_csp_avg;
    CK(cudaMemcpy(c->d_lam_hist, p, sizeof(double) * n * c->cfg.n_lam_avg, cudaMemcpyHostToDevice));
    p += sizeof(double) * n * c->cfg.n_lam_avg;
    CK(cudaMemcpy(c->d_lam_prev, p, sizeof(double) * n, cudaMemcpyHostToDevice));
    p += sizeof(double) * n;
    CK(cudaMemcpy(c->d_lam_int, p, sizeof(double) * n, cudaMemcpyHostToDevice));
  }
  c->md_ready = false;
  c->restart_pending = true;
  return AP_OK;
}

}  // extern "C"
