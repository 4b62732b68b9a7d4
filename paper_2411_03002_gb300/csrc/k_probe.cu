// Measured throughput peaks of the GPU the library runs on: the FP32 FFMA rate and
// the rate of warp-level TF32 tensor-core MMAs (m16n8k8), the denominators of the
// arithmetic rooflines of the ACE kernels.  Instrumentation; no paper counterpart.
//
// Each thread of sms x 4 blocks of 256 threads runs 8 independent dependency chains
// (FFMA: x = x a + b; MMA: D += A B on one tile per chain), enough independent work
// per scheduler to keep the pipe busy.  Block 0's thread 0 reads the SM cycle counter
// and the global nanosecond timer at its start and end, which gives the SM clock
// during the probe.
#include <cuda_runtime.h>

#include "ap_internal.cuh"

namespace ap {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(kThreads) k_probe_ffma(int iters, float a, float b, float* __restrict__ out,
                                                         unsigned long long* __restrict__ clk) {
  const bool rec = blockIdx.x == 0 && threadIdx.x == 0;
  unsigned long long c0 = 0, t0 = 0;
  if (rec) {
    t0 = global_ns();
    c0 = clock64();
  }
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3f + k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (rec) {
    clk[0] = clock64() - c0;
    clk[1] = global_ns() - t0;
  }
}

__global__ void __launch_bounds__(kThreads) k_probe_mma_tf32(int iters, float* __restrict__ out,
                                                             unsigned long long* __restrict__ clk) {
  const bool rec = blockIdx.x == 0 && threadIdx.x == 0;
  unsigned long long c0 = 0, t0 = 0;
  if (rec) {
    t0 = global_ns();
    c0 = clock64();
  }
  const uint32_t a0 = __float_as_uint(1e-3f * (threadIdx.x + 1)) & 0xffffe000u;
  const uint32_t a1 = a0 ^ 0x4000u, a2 = a0 ^ 0x8000u, a3 = a0 ^ 0xc000u;
  const uint32_t b0 = __float_as_uint(1e-3f) & 0xffffe000u, b1 = b0;
  float d[kChains][4];
#pragma unroll
  for (int t = 0; t < kChains; ++t)
#pragma unroll
    for (int u = 0; u < 4; ++u) d[t][u] = 0.f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int t = 0; t < kChains; ++t)
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+f"(d[t][0]), "+f"(d[t][1]), "+f"(d[t][2]), "+f"(d[t][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float s = 0.f;
#pragma unroll
  for (int t = 0; t < kChains; ++t) s += d[t][0] + d[t][1] + d[t][2] + d[t][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (rec) {
    clk[0] = clock64() - c0;
    clk[1] = global_ns() - t0;
  }
}

}  // namespace
}  // namespace ap

extern "C" ap_status ap_probe_peak(int32_t which, int32_t reps, void* stream, double* h_tflops, double* h_sm_mhz) {
  using namespace ap;
  if ((which != 0 && which != 1) || reps < 2 || reps > 100 || !h_tflops) return AP_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AP_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return AP_ERR_CUDA;
  const int blocks = sms * kBlocksPerSm;
  const int ffma_iters = 20000, mma_iters = 2500;
  float* d_out = nullptr;
  unsigned long long* d_clk = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ap_status st = AP_OK;
  double best_ms = 1e30, best_mhz = 0.0;
  if (cudaMalloc(&d_out, sizeof(float) * (size_t)blocks * kThreads) != cudaSuccess ||
      cudaMalloc(&d_clk, 2 * sizeof(unsigned long long)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = AP_ERR_CUDA;
  } else {
    for (int r = 0; r < reps && st == AP_OK; ++r) {   // the first run is a warm-up
      cudaEventRecord(e0, s);
      if (which == 0)
        k_probe_ffma<<<blocks, kThreads, 0, s>>>(ffma_iters, 0.999f, 1e-4f, d_out, d_clk);
      else
        k_probe_mma_tf32<<<blocks, kThreads, 0, s>>>(mma_iters, d_out, d_clk);
      cudaEventRecord(e1, s);
      unsigned long long clk[2] = {0, 0};
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
          cudaMemcpy(clk, d_clk, sizeof(clk), cudaMemcpyDeviceToHost) != cudaSuccess) {
        st = AP_ERR_CUDA;
        break;
      }
      if (r > 0 && ms < best_ms) {
        best_ms = ms;
        best_mhz = clk[1] > 0 ? 1e3 * (double)clk[0] / (double)clk[1] : 0.0;
      }
    }
  }
  if (st == AP_OK) {
    const double threads = (double)blocks * kThreads;
    const double flops = which == 0 ? 2.0 * kChains * ffma_iters * threads
                                    : 2.0 * 16 * 8 * 8 * (double)kChains * mma_iters * threads / 32.0;
    *h_tflops = flops / (best_ms * 1e-3) / 1e12;
    if (h_sm_mhz) *h_sm_mhz = best_mhz;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_clk) cudaFree(d_clk);
  if (d_out) cudaFree(d_out);
  return st;
}
