// Learned detection score (the selector).  The paper lets any detector supply the
// argument of f_cut in Eq. lambda_1_i, as long as it is 0 for atoms to be computed
// precisely and 1 for atoms to be computed fast (Appendix B, the remark after f_cut);
// this file computes the project's learned score p_i = sigmoid(MLP(features_i)).
//
//   k_sel_rho       rho_i and xi'(rho_i) in FP32 over the EAM rows (pre-pass).
//   k_sel_features  24 features per atom (FP32) over the EAM rows, thread per atom.
//   k_sel_mlp       MLP 24-64-64-1 on 128-atom tiles with tcgen05: standardised
//                   bf16 inputs and bf16 weights in shared memory, FP32 accumulators
//                   in tensor memory, ReLU/bf16 epilogue between the layers, the last
//                   layer (64 -> 1) and the sigmoid in registers.
//   k_sel_bwd       backward pass of the weighted binary cross-entropy, FP32 SIMT,
//                   per-block partial gradients in a fixed sample order.
//   k_sel_reduce    fixed-order sum of the partials (bitwise reproducible).
//   k_sel_adam      Adam on the FP32 master weights; rewrites the bf16 operand images.
//
// Feature definitions (N = pairs with r < 5.5 A; S1 r < 3.09, S2 3.09 <= r < 4.02,
// S3 4.02 <= r < 4.77 A; empty sets give 0):
//   0 rho  1 xi(rho)  2 xi'(rho)  3 1/2 sum Phi  4-6 |S1| |S2| |S3|  7 min(CSP, 100)
//   8 sum_{j in S2} min(r_j^2, min_{k in S2, k != j} |r_j + r_k|^2)
//   9-11 |sum r_j| over S1, S2, N   12 |sum_N zeta'(r) r_j/r|   13 rho_i - mean_S1 rho_j
//   14-17 mean, std, min, max of r over S1   18-21 mean, std, 3rd, 4th central moment over N
//   22 |N|   23 mean_N xi'_j - xi'_i
#include <cuda_bf16.h>

#include "ap_internal.cuh"
#include "eam_frame.cuh"

namespace ap {

namespace {

constexpr float kRFeat = 5.5f;
constexpr float kShell1 = 3.09f, kShell2 = 4.02f, kShell3 = 4.77f;
constexpr float kCspCap = 100.f;
constexpr int kS2Max = 24;

// ------------------------------------------------------------------ density pre-pass
template <bool STORED>
__global__ void __launch_bounds__(128) k_sel_rho(int n, const SysInfo* __restrict__ sys,
                                                 const int* __restrict__ atom_sys, const float4* __restrict__ sh,
                                                 const int* __restrict__ nbr, const int* __restrict__ off,
                                                 const int* __restrict__ cnt, int cap, EamP<float> p,
                                                 float2* __restrict__ rho_dxi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 si = sh[i];
  const Frame<float, STORED> fr(sys[atom_sys ? atom_sys[i] : 0], si);
  const int c = cnt[i];
  const size_t row = (size_t)i * cap;
  const float rf2 = kRFeat * kRFeat;
  float rho = 0.f;
  for (int t = 0; t < c; ++t) {
    const int j = nbr[row + t];
    float d[3];
    fr.disp(sh[j], off, row + t, d);
    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 < rf2 && r2 < p.rc2) {
      const float r = sqrtf(r2);
      const float u = (r - p.rc) * p.inv_h;
      const float u4 = (u * u) * (u * u);
      rho += expf(p.beta - p.beta_r0 * r) * (u4 / (1.f + u4));
    }
  }
  float dxi = 0.f;
  if (rho > 0.f) dxi = -0.5f * p.A / sqrtf(rho);
  rho_dxi[i] = make_float2(rho, dxi);
}

// ------------------------------------------------------------------ features
template <bool STORED>
__global__ void __launch_bounds__(128) k_sel_features(int n, const SysInfo* __restrict__ sys,
                                                      const int* __restrict__ atom_sys,
                                                      const float4* __restrict__ sh, const int* __restrict__ nbr,
                                                      const int* __restrict__ off, const int* __restrict__ cnt,
                                                      int cap, EamP<float> p, const float2* __restrict__ rho_dxi,
                                                      const double* __restrict__ csp, float* __restrict__ feat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 si = sh[i];
  const Frame<float, STORED> fr(sys[atom_sys ? atom_sys[i] : 0], si);
  const int c = cnt[i];
  const size_t row = (size_t)i * cap;
  const float rf2 = kRFeat * kRFeat;
  const float2 me = rho_dxi[i];

  float phi = 0.f, sum_r = 0.f, sum_r1 = 0.f, rmin1 = 0.f, rmax1 = 0.f, rho_nb1 = 0.f, dxi_nb = 0.f;
  float v1[3] = {0.f, 0.f, 0.f}, v2[3] = {0.f, 0.f, 0.f}, va[3] = {0.f, 0.f, 0.f}, gz[3] = {0.f, 0.f, 0.f};
  int n_all = 0, n1 = 0, n2 = 0, n3 = 0;
  float s2v[kS2Max][3];
  for (int t = 0; t < c; ++t) {
    const int j = nbr[row + t];
    float d[3];
    fr.disp(sh[j], off, row + t, d);
    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 < rf2)) continue;
    const float r = sqrtf(r2);
    if (r2 < p.rc2) {
      const float u = (r - p.rc) * p.inv_h;
      const float u2 = u * u;
      const float u4 = u2 * u2;
      const float inv = 1.f / (1.f + u4);
      const float ps = u4 * inv;
      const float dps = 4.f * u2 * u * inv * inv * p.inv_h;
      const float ez = expf(p.beta - p.beta_r0 * r);
      const float dzeta = ez * (dps - p.beta_r0 * ps);
      const float e1 = expf(-p.alpha * (r - p.rp));
      phi += p.D * (e1 * e1 - 2.f * e1) * ps;
      const float s = dzeta / r;
      gz[0] += s * d[0];
      gz[1] += s * d[1];
      gz[2] += s * d[2];
    }
    ++n_all;
    sum_r += r;
    va[0] += d[0];
    va[1] += d[1];
    va[2] += d[2];
    const float2 nb = rho_dxi[j];
    dxi_nb += nb.y;
    if (r < kShell1) {
      rmin1 = n1 ? fminf(rmin1, r) : r;
      rmax1 = n1 ? fmaxf(rmax1, r) : r;
      ++n1;
      sum_r1 += r;
      rho_nb1 += nb.x;
      v1[0] += d[0];
      v1[1] += d[1];
      v1[2] += d[2];
    } else if (r < kShell2) {
      if (n2 < kS2Max) {
        s2v[n2][0] = d[0];
        s2v[n2][1] = d[1];
        s2v[n2][2] = d[2];
      }
      ++n2;
      v2[0] += d[0];
      v2[1] += d[1];
      v2[2] += d[2];
    } else if (r < kShell3) {
      ++n3;
    }
  }
  // second pass: central moments about the means
  const float mean = n_all ? sum_r / (float)n_all : 0.f;
  const float mean1 = n1 ? sum_r1 / (float)n1 : 0.f;
  float m2 = 0.f, m3 = 0.f, m4 = 0.f, m21 = 0.f;
  for (int t = 0; t < c; ++t) {
    const int j = nbr[row + t];
    float d[3];
    fr.disp(sh[j], off, row + t, d);
    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 < rf2)) continue;
    const float r = sqrtf(r2);
    const float e = r - mean;
    const float e2 = e * e;
    m2 += e2;
    m3 += e2 * e;
    m4 += e2 * e2;
    if (r < kShell1) {
      const float e1 = r - mean1;
      m21 += e1 * e1;
    }
  }
  // second-shell centro-symmetry
  float cs2 = 0.f;
  if (n2 <= kS2Max) {
    for (int a = 0; a < n2; ++a) {
      float best = s2v[a][0] * s2v[a][0] + s2v[a][1] * s2v[a][1] + s2v[a][2] * s2v[a][2];
      for (int b = 0; b < n2; ++b) {
        if (b == a) continue;
        const float x = s2v[a][0] + s2v[b][0], y = s2v[a][1] + s2v[b][1], z = s2v[a][2] + s2v[b][2];
        best = fminf(best, x * x + y * y + z * z);
      }
      cs2 += best;
    }
  } else {
    // more second-shell entries than registers hold (strong disorder): pair loop over the row
    for (int ta = 0; ta < c; ++ta) {
      float da[3];
      fr.disp(sh[nbr[row + ta]], off, row + ta, da);
      const float ra2 = da[0] * da[0] + da[1] * da[1] + da[2] * da[2];
      if (!(ra2 < rf2)) continue;
      const float ra = sqrtf(ra2);
      if (!(ra >= kShell1 && ra < kShell2)) continue;
      float best = ra2;
      for (int tb = 0; tb < c; ++tb) {
        if (tb == ta) continue;
        float db[3];
        fr.disp(sh[nbr[row + tb]], off, row + tb, db);
        const float rb2 = db[0] * db[0] + db[1] * db[1] + db[2] * db[2];
        if (!(rb2 < rf2)) continue;
        const float rb = sqrtf(rb2);
        if (!(rb >= kShell1 && rb < kShell2)) continue;
        const float x = da[0] + db[0], y = da[1] + db[1], z = da[2] + db[2];
        best = fminf(best, x * x + y * y + z * z);
      }
      cs2 += best;
    }
  }
  float o[24];
  o[0] = me.x;
  o[1] = me.x > 0.f ? -p.A * sqrtf(me.x) : 0.f;
  o[2] = me.y;
  o[3] = 0.5f * phi;
  o[4] = (float)n1;
  o[5] = (float)n2;
  o[6] = (float)n3;
  o[7] = (float)fmin(csp[i], (double)kCspCap);
  o[8] = cs2;
  o[9] = sqrtf(v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2]);
  o[10] = sqrtf(v2[0] * v2[0] + v2[1] * v2[1] + v2[2] * v2[2]);
  o[11] = sqrtf(va[0] * va[0] + va[1] * va[1] + va[2] * va[2]);
  o[12] = sqrtf(gz[0] * gz[0] + gz[1] * gz[1] + gz[2] * gz[2]);
  o[13] = n1 ? me.x - rho_nb1 / (float)n1 : 0.f;
  o[14] = mean1;
  o[15] = n1 ? sqrtf(m21 / (float)n1) : 0.f;
  o[16] = rmin1;
  o[17] = rmax1;
  o[18] = mean;
  o[19] = n_all ? sqrtf(m2 / (float)n_all) : 0.f;
  o[20] = n_all ? m3 / (float)n_all : 0.f;
  o[21] = n_all ? m4 / (float)n_all : 0.f;
  o[22] = (float)n_all;
  o[23] = n_all ? dxi_nb / (float)n_all - me.y : 0.f;
  float4* dst = reinterpret_cast<float4*>(feat + (size_t)i * 24);
#pragma unroll
  for (int k = 0; k < 6; ++k) dst[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
}

// ------------------------------------------------------------------ tcgen05 helpers
// Shared-memory matrix descriptor, canonical K-major layout without swizzle: the
// operand is a grid of 8-row x 16-byte core matrices (rows 16 B apart inside a
// core matrix); lbo = byte distance between core matrices adjacent along K,
// sbo = byte distance between core matrices adjacent along M (or N).
__device__ inline uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the tcgen05 family; base offset 0; no swizzle
  return d;
}

// Instruction descriptor of kind::f16: D = FP32, A = B = bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t mma_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ inline void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ inline void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ inline void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ inline uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the mbarrier phase with the given parity; gives up after ~1 s.
__device__ inline bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > 1000000000ull) return false;
  }
}

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape), waited.
__device__ inline void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ inline uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// ------------------------------------------------------------------ MLP forward (tcgen05)
// Shared-memory map (bytes).  Operand images use the canonical no-swizzle K-major
// layout with core matrix (row block rb, K block kb) at (kb * rows/8 + rb) * 128.
constexpr int kSmB1 = 0;                       // W1^T: 64 x 32 bf16   (4 KiB)
constexpr int kSmB2 = kSmB1 + 4096;            // W2^T: 64 x 64 bf16   (8 KiB)
constexpr int kSmA1 = kSmB2 + 8192;            // x~:  128 x 32 bf16   (8 KiB)
constexpr int kSmA2 = kSmA1 + 8192;            // h1:  128 x 64 bf16   (16 KiB)
constexpr int kSmF = kSmA2 + 16384;            // FP32 vectors (SelDev::vec)
constexpr int kSmBar = kSmF + 1024;            // mbarrier (8 B), TMEM base (4 B), abort flag (4 B)
constexpr int kSmUsed = kSmBar + 16;
// Padding so that every address a descriptor can form from these images stays
// inside the allocation.
constexpr int kSmTotal = 72 * 1024;
constexpr int kTmemCols = 128;                 // D1 in columns [0, 64), D2 in [64, 128)
constexpr uint32_t kIdesc = mma_idesc(128, 64);

__global__ void __launch_bounds__(128) k_sel_mlp(int n, const float* __restrict__ feat, const int* __restrict__ idx,
                                                 const SelDev* __restrict__ model, float* __restrict__ p_out,
                                                 double* __restrict__ score_out, float* __restrict__ z_out,
                                                 __nv_bfloat16* __restrict__ h1_out, float* __restrict__ h2_out,
                                                 DevScalars* __restrict__ sc) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int t = threadIdx.x;
  const int warp = t >> 5;
  float* vec = reinterpret_cast<float*>(sm + kSmF);
  const float* w3 = vec + SelDev::kW3;
  const float* b1 = vec + SelDev::kB1;
  const float* b2 = vec + SelDev::kB2;
  const float* mu = vec + SelDev::kMu;
  const float* inv_s = vec + SelDev::kInvS;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kSmBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kSmBar + 8);
  int* abort_flag = reinterpret_cast<int*>(sm + kSmBar + 12);

  // operand images and FP32 vectors -> shared memory
  {
    const uint4* src = reinterpret_cast<const uint4*>(model->img);
    uint4* dst = reinterpret_cast<uint4*>(sm + kSmB1);
    for (int k = t; k < (4096 + 8192) / 16; k += blockDim.x) dst[k] = src[k];
    for (int k = t; k < SelDev::kVec; k += blockDim.x) vec[k] = model->vec[k];
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t mbar = smem_u32(bar);
  const uint32_t sa1 = smem_u32(sm + kSmA1), sa2 = smem_u32(sm + kSmA2);
  const uint32_t sb1 = smem_u32(sm + kSmB1), sb2 = smem_u32(sm + kSmB2);
  // A (128 rows): lbo = 16 core matrices * 128 B along K; B (64 rows): 8 * 128 B
  constexpr uint32_t kLboA = 16 * 128, kLboB = 8 * 128, kSbo = 128;
  uint32_t phase = 0;
  const int n_tiles = (n + 127) / 128;
  const int row_off = ((t >> 3) * 128) + ((t & 7) * 16);   // this thread's row inside a K block

  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int row = tile * 128 + t;
    const bool valid = row < n;
    // ---- A1 <- bf16((x - mu) * inv_sigma), K padded to 32 with zeros
    {
      float x[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) x[k] = 0.f;
      if (valid) {
        const int src = idx ? idx[row] : row;
        const float4* fp = reinterpret_cast<const float4*>(feat + (size_t)src * 24);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float4 v = __ldg(fp + k);
          x[4 * k] = (v.x - mu[4 * k]) * inv_s[4 * k];
          x[4 * k + 1] = (v.y - mu[4 * k + 1]) * inv_s[4 * k + 1];
          x[4 * k + 2] = (v.z - mu[4 * k + 2]) * inv_s[4 * k + 2];
          x[4 * k + 3] = (v.w - mu[4 * k + 3]) * inv_s[4 * k + 3];
        }
      }
#pragma unroll
      for (int kb = 0; kb < 4; ++kb) {
        uint4 u;
        u.x = pack_bf16(x[8 * kb], x[8 * kb + 1]);
        u.y = pack_bf16(x[8 * kb + 2], x[8 * kb + 3]);
        u.z = pack_bf16(x[8 * kb + 4], x[8 * kb + 5]);
        u.w = pack_bf16(x[8 * kb + 6], x[8 * kb + 7]);
        *reinterpret_cast<uint4*>(sm + kSmA1 + kb * kLboA + row_off) = u;
      }
    }
    fence_async_smem();
    __syncthreads();
    // ---- layer 1: D1 = A1 * W1 (K = 32: two MMAs of K = 16)
    if (t == 0) {
      fence_after_sync();
#pragma unroll
      for (int s = 0; s < 2; ++s)
        mma_bf16(tmem, smem_desc(sa1 + s * 2 * kLboA, kLboA, kSbo), smem_desc(sb1 + s * 2 * kLboB, kLboB, kSbo),
                 kIdesc, s > 0);
      mma_commit(mbar);
    }
    if (!mbar_wait(mbar, phase)) atomicOr(abort_flag, 1);
    phase ^= 1u;
    fence_after_sync();
    __syncthreads();
    if (*abort_flag) break;
    // ---- epilogue 1: h1 = bf16(relu(D1 + b1)) -> A2 (and h1_out)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float a[16];
      tmem_ld16(tmem + lane_base + 16 * q, a);
#pragma unroll
      for (int k = 0; k < 16; ++k) a[k] = fmaxf(a[k] + b1[16 * q + k], 0.f);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint4 u;
        u.x = pack_bf16(a[8 * h], a[8 * h + 1]);
        u.y = pack_bf16(a[8 * h + 2], a[8 * h + 3]);
        u.z = pack_bf16(a[8 * h + 4], a[8 * h + 5]);
        u.w = pack_bf16(a[8 * h + 6], a[8 * h + 7]);
        const int kb = 2 * q + h;
        *reinterpret_cast<uint4*>(sm + kSmA2 + kb * kLboA + row_off) = u;
        if (h1_out && valid) *reinterpret_cast<uint4*>(h1_out + (size_t)row * 64 + 8 * kb) = u;
      }
    }
    fence_before_sync();
    fence_async_smem();
    __syncthreads();
    // ---- layer 2: D2 = A2 * W2 (K = 64: four MMAs)
    if (t == 0) {
      fence_after_sync();
#pragma unroll
      for (int s = 0; s < 4; ++s)
        mma_bf16(tmem + 64, smem_desc(sa2 + s * 2 * kLboA, kLboA, kSbo), smem_desc(sb2 + s * 2 * kLboB, kLboB, kSbo),
                 kIdesc, s > 0);
      mma_commit(mbar);
    }
    if (!mbar_wait(mbar, phase)) atomicOr(abort_flag, 1);
    phase ^= 1u;
    fence_after_sync();
    __syncthreads();
    if (*abort_flag) break;
    // ---- epilogue 2: h2 = relu(D2 + b2); z = sum_k h2_k w3_k + b3; p = sigmoid(z)
    float z = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float a[16];
      tmem_ld16(tmem + lane_base + 64 + 16 * q, a);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float h = fmaxf(a[k] + b2[16 * q + k], 0.f);
        a[k] = h;
        z = fmaf(h, w3[16 * q + k], z);
      }
      if (h2_out && valid) {
        float4* d = reinterpret_cast<float4*>(h2_out + (size_t)row * 64 + 16 * q);
#pragma unroll
        for (int k = 0; k < 4; ++k) d[k] = make_float4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
      }
    }
    z += vec[SelDev::kB3];
    if (valid) {
      const float pz = 1.f / (1.f + expf(-z));
      if (p_out) p_out[row] = pz;
      if (score_out) score_out[row] = (double)pz;
      if (z_out) z_out[row] = z;
    }
    fence_before_sync();
    __syncthreads();
  }
  // an abandoned wait: give the MMAs in flight one more bounded wait before freeing TMEM
  __syncthreads();
  if (*abort_flag) {
    if (t == 0) atomicOr(&sc->err, kErrTimeout);
    mbar_wait(mbar, phase ^ 1u);   // the parity of the wait that gave up
  }
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ------------------------------------------------------------------ backward (FP32 SIMT)
constexpr int kChunk = 64;
constexpr int kBwdThreads = 256;
// shared: h1 [64][64], h2 [64][64], dz2 [64][64], dz1 [64][64], xt [64][24], W2r [64][64],
// gz [64], loss [64]
constexpr int kBwdSmem = (5 * 64 * 64 + 64 * 24 + 2 * 64) * 4;

__global__ void __launch_bounds__(kBwdThreads) k_sel_bwd(int b, const float* __restrict__ feat,
                                                         const int* __restrict__ idx,
                                                         const float* __restrict__ label,
                                                         const float* __restrict__ weight,
                                                         const SelDev* __restrict__ model,
                                                         const float* __restrict__ z,
                                                         const __nv_bfloat16* __restrict__ h1g,
                                                         const float* __restrict__ h2g, float* __restrict__ partial) {
  extern __shared__ float sf[];
  float* h1 = sf;
  float* h2 = h1 + 64 * 64;
  float* dz2 = h2 + 64 * 64;
  float* dz1 = dz2 + 64 * 64;
  float* W2 = dz1 + 64 * 64;
  float* xt = W2 + 64 * 64;
  float* gz = xt + 64 * 24;
  float* lv = gz + 64;
  const int t = threadIdx.x;
  for (int k = t; k < 64 * 64; k += kBwdThreads) W2[k] = model->W2r[k];
  const float* vec = model->vec;
  // owned gradients: dW2 entries e = t + 256 u (k = e/64, n = e%64); dW1 entries
  // e = t + 256 u, u < 6 (f = e/64, k = e%64); t < 64: db1[t]; 64 <= t < 128: db2;
  // 128 <= t < 192: dw3; t == 192: db3 and the loss.
  float gW2[16], gW1[6], gv = 0.f, gl = 0.f;
#pragma unroll
  for (int u = 0; u < 16; ++u) gW2[u] = 0.f;
#pragma unroll
  for (int u = 0; u < 6; ++u) gW1[u] = 0.f;
  const int n_chunks = (b + kChunk - 1) / kChunk;
  for (int ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const int s0 = ch * kChunk;
    __syncthreads();
    for (int e = t; e < 64 * 64; e += kBwdThreads) {
      const int s = e >> 6, k = e & 63;
      const bool ok = s0 + s < b;
      h1[e] = ok ? __bfloat162float(h1g[(size_t)(s0 + s) * 64 + k]) : 0.f;
      h2[e] = ok ? h2g[(size_t)(s0 + s) * 64 + k] : 0.f;
    }
    for (int e = t; e < 64 * 24; e += kBwdThreads) {
      const int s = e / 24, f = e - 24 * (e / 24);
      float v = 0.f;
      if (s0 + s < b) {
        const int src = idx ? idx[s0 + s] : s0 + s;
        v = __bfloat162float(__float2bfloat16_rn((feat[(size_t)src * 24 + f] - vec[SelDev::kMu + f]) *
                                                 vec[SelDev::kInvS + f]));
      }
      xt[e] = v;
    }
    if (t < 64) {
      float g = 0.f, l = 0.f;
      if (s0 + t < b) {
        const int src = idx ? idx[s0 + t] : s0 + t;
        const float y = label[src], w = weight[src], zz = z[s0 + t];
        const float pz = 1.f / (1.f + expf(-zz));
        g = w * (pz - y);
        l = w * (fmaxf(zz, 0.f) + log1pf(expf(-fabsf(zz))) - y * zz);
      }
      gz[t] = g;
      lv[t] = l;
    }
    __syncthreads();
    for (int e = t; e < 64 * 64; e += kBwdThreads) {
      const int s = e >> 6, n = e & 63;
      dz2[e] = h2[e] > 0.f ? gz[s] * vec[SelDev::kW3 + n] : 0.f;
    }
    __syncthreads();
    // dW2 and dz1 (the latter through the bf16-valued W2)
#pragma unroll 1
    for (int u = 0; u < 16; ++u) {
      const int e = t + kBwdThreads * u;
      const int k = e >> 6, n = e & 63;
      float a = 0.f, dh = 0.f;
      for (int s = 0; s < kChunk; ++s) a = fmaf(h1[s * 64 + k], dz2[s * 64 + n], a);
      gW2[u] += a;
      // reuse (s = k, j = n) as an entry of dz1[s][j]
      const int s = k, j = n;
      for (int m = 0; m < 64; ++m) dh = fmaf(W2[j * 64 + m], dz2[s * 64 + m], dh);
      dz1[s * 64 + j] = h1[s * 64 + j] > 0.f ? dh : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const int e = t + kBwdThreads * u;
      const int f = e >> 6, k = e & 63;
      float a = 0.f;
      for (int s = 0; s < kChunk; ++s) a = fmaf(xt[s * 24 + f], dz1[s * 64 + k], a);
      gW1[u] += a;
    }
    if (t < 64) {
      float a = 0.f;
      for (int s = 0; s < kChunk; ++s) a += dz1[s * 64 + t];
      gv += a;
    } else if (t < 128) {
      float a = 0.f;
      for (int s = 0; s < kChunk; ++s) a += dz2[s * 64 + (t - 64)];
      gv += a;
    } else if (t < 192) {
      float a = 0.f;
      for (int s = 0; s < kChunk; ++s) a = fmaf(gz[s], h2[s * 64 + (t - 128)], a);
      gv += a;
    } else if (t == 192) {
      float a = 0.f, l = 0.f;
      for (int s = 0; s < kChunk; ++s) {
        a += gz[s];
        l += lv[s];
      }
      gv += a;
      gl += l;
    }
  }
  float* out = partial + (size_t)blockIdx.x * (SelDev::kParams + 1);
#pragma unroll
  for (int u = 0; u < 6; ++u) out[t + kBwdThreads * u] = gW1[u];             // W1 [f][k] at f*64 + k
#pragma unroll
  for (int u = 0; u < 16; ++u) out[SelDev::kOffW2 + t + kBwdThreads * u] = gW2[u];
  if (t < 64) out[SelDev::kOffB1 + t] = gv;
  else if (t < 128) out[SelDev::kOffB2 + t - 64] = gv;
  else if (t < 192) out[SelDev::kOffW3 + t - 128] = gv;
  else if (t == 192) {
    out[SelDev::kOffB3] = gv;
    out[SelDev::kParams] = gl;
  }
}

__global__ void k_sel_reduce(int parts, const float* __restrict__ partial, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > SelDev::kParams) return;
  float s = 0.f;
  for (int g = 0; g < parts; ++g) s += partial[(size_t)g * (SelDev::kParams + 1) + p];
  grad[p] = s;
}

// Adam step on the FP32 master (update != 0), then the bf16 operand images, the
// bf16-valued W2 copy and the FP32 vectors are rewritten from the master.
__global__ void k_sel_adam(float* __restrict__ master, float* __restrict__ m1, float* __restrict__ m2,
                           const float* __restrict__ grad, SelDev* __restrict__ model, int update, float lr,
                           float beta1, float beta2, float eps, float inv_bc1, float inv_bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= SelDev::kParams) return;
  float w = master[p];
  if (update) {
    const float g = grad[p];
    const float a = beta1 * m1[p] + (1.f - beta1) * g;
    const float v = beta2 * m2[p] + (1.f - beta2) * g * g;
    m1[p] = a;
    m2[p] = v;
    w -= lr * (a * inv_bc1) / (sqrtf(v * inv_bc2) + eps);
    master[p] = w;
  }
  const __nv_bfloat16 hb = __float2bfloat16_rn(w);
  __nv_bfloat16* img = reinterpret_cast<__nv_bfloat16*>(model->img);
  if (p < SelDev::kOffB1) {                      // W1[f][k]: B1 image row k (output), K = f
    const int f = p >> 6, k = p & 63;
    img[(((f >> 3) * 8 + (k >> 3)) * 128 + (k & 7) * 16 + (f & 7) * 2) / 2] = hb;
  } else if (p < SelDev::kOffW2) {
    model->vec[SelDev::kB1 + p - SelDev::kOffB1] = w;
  } else if (p < SelDev::kOffB2) {               // W2[k][n]: B2 image row n, K = k
    const int e = p - SelDev::kOffW2, k = e >> 6, n = e & 63;
    img[(4096 + ((k >> 3) * 8 + (n >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2) / 2] = hb;
    model->W2r[e] = __bfloat162float(hb);
  } else if (p < SelDev::kOffW3) {
    model->vec[SelDev::kB2 + p - SelDev::kOffB2] = w;
  } else if (p < SelDev::kOffB3) {
    model->vec[SelDev::kW3 + p - SelDev::kOffW3] = __bfloat162float(hb);
  } else {
    model->vec[SelDev::kB3] = w;
  }
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------------ launchers
void launch_sel_features(ap_ctx* c, float* d_feat, cudaStream_t s) {
  const int n = (int)c->n;
  if (n <= 0) return;
  EamP<float> p = make_params<float>(c->cfg);
  const int* off = c->stored_off ? c->d_off_eam : nullptr;
  if (c->stored_off) {
    k_sel_rho<true><<<nblk(n, 128), 128, 0, s>>>(n, c->d_sys, c->d_atom_sys, c->d_sh32, c->d_nbr_eam, off,
                                                   c->d_cnt_eam, c->cap_eam, p, c->d_sel_rho);
    k_sel_features<true><<<nblk(n, 128), 128, 0, s>>>(n, c->d_sys, c->d_atom_sys, c->d_sh32, c->d_nbr_eam, off,
                                                        c->d_cnt_eam, c->cap_eam, p, c->d_sel_rho, c->d_csp,
                                                        d_feat);
  } else {
    k_sel_rho<false><<<nblk(n, 128), 128, 0, s>>>(n, c->d_sys, c->d_atom_sys, c->d_sh32, c->d_nbr_eam, off,
                                                    c->d_cnt_eam, c->cap_eam, p, c->d_sel_rho);
    k_sel_features<false><<<nblk(n, 128), 128, 0, s>>>(n, c->d_sys, c->d_atom_sys, c->d_sh32, c->d_nbr_eam, off,
                                                         c->d_cnt_eam, c->cap_eam, p, c->d_sel_rho, c->d_csp,
                                                         d_feat);
  }
  c->kernels += 2;
}

cudaError_t sel_mlp_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_sel_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmTotal);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sel_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdSmem);
  if (e == cudaSuccess) done = true;
  return e;
}

void launch_sel_mlp(ap_ctx* c, int64_t n, const float* d_feat, const int* d_idx, float* d_p, double* d_score,
                    float* d_z, void* d_h1, float* d_h2, cudaStream_t s) {
  if (n <= 0) return;
  const int tiles = nblk(n, 128);
  const int grid = tiles < 3 * c->num_sms ? tiles : 3 * c->num_sms;
  k_sel_mlp<<<grid, 128, kSmTotal, s>>>((int)n, d_feat, d_idx, c->d_sel_model, d_p, d_score, d_z,
                                       reinterpret_cast<__nv_bfloat16*>(d_h1), d_h2, c->d_sc);
  c->kernels += 1;
}

int sel_bwd_parts(ap_ctx* c, int64_t b) {
  const int chunks = nblk(b, kChunk);
  return chunks < 2 * c->num_sms ? chunks : 2 * c->num_sms;
}

void launch_sel_backward(ap_ctx* c, int64_t b, const float* d_feat, const int* d_idx, const float* d_label,
                         const float* d_weight, cudaStream_t s) {
  const int parts = sel_bwd_parts(c, b);
  k_sel_bwd<<<parts, kBwdThreads, kBwdSmem, s>>>((int)b, d_feat, d_idx, d_label, d_weight, c->d_sel_model,
                                                 c->d_sel_z, reinterpret_cast<const __nv_bfloat16*>(c->d_sel_h1),
                                                 c->d_sel_h2, c->d_sel_partial);
  k_sel_reduce<<<nblk(SelDev::kParams + 1, 256), 256, 0, s>>>(parts, c->d_sel_partial, c->d_sel_grad);
  c->kernels += 2;
}

void launch_sel_adam(ap_ctx* c, bool update, float lr, float beta1, float beta2, float eps, float inv_bc1,
                     float inv_bc2, cudaStream_t s) {
  k_sel_adam<<<nblk(SelDev::kParams, 256), 256, 0, s>>>(c->d_sel_master, c->d_sel_m1, c->d_sel_m2, c->d_sel_grad,
                                                        c->d_sel_model, update ? 1 : 0, lr, beta1, beta2, eps,
                                                        inv_bc1, inv_bc2);
  c->kernels += 1;
}

size_t sel_partial_floats(ap_ctx* c) { return (size_t)(2 * c->num_sms) * (SelDev::kParams + 1); }

}  // namespace ap
