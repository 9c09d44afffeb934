// Roofline denominators of the arithmetic pipes, measured on the device:
// dependent chains of one instruction kind on eight independent
// accumulators per thread, enough warps per SM that the pipe, not the
// latency of a chain, bounds the rate.  The caller times a launch and
// divides the operations by the time.  No counterpart in the paper.
#include "internal.cuh"

namespace dsmc {

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ float ex2_f(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int K>
__global__ void __launch_bounds__(256) k_peak(int32_t iters, float* __restrict__ sink) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  float a[kChains];
  float2 p[kChains];
  double d[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) {
    a[q] = 0.5f + 1e-3f * (float)((t + q) & 63);
    p[q] = make_float2(a[q], a[q] + 0.25f);
    d[q] = (double)a[q];
  }
  const float2 m2 = make_float2(0.9999f, 0.9998f), c2 = make_float2(1e-4f, 2e-4f);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int q = 0; q < kChains; ++q) {
        if (K == 0) a[q] = fmaf(a[q], 0.9999f, 1e-4f);
        if (K == 1) p[q] = __ffma2_rn(p[q], m2, c2);
        if (K == 2) d[q] = fma(d[q], 0.9999, 1e-4);
        if (K == 3) a[q] = ex2_f(-a[q]);
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += K == 1 ? p[q].x + p[q].y : K == 2 ? (float)d[q] : a[q];
  sink[t] = s;
}

}  // namespace

// operations one thread performs: FLOPs for the FMA kinds (2 per FMA, 4 per
// paired FMA), special-function results for MUFU
int64_t peak_ops_per_thread(int which, int32_t iters) {
  const int64_t inst = (int64_t)iters * 4 * kChains;
  return which == 0 ? 2 * inst : which == 1 ? 4 * inst : which == 2 ? 2 * inst : inst;
}

int launch_peak(Ctx* c, int which, int32_t blocks, int32_t threads, int32_t iters, float* sink, cudaStream_t s) {
  switch (which) {
    case 0: k_peak<0><<<blocks, threads, 0, s>>>(iters, sink); break;
    case 1: k_peak<1><<<blocks, threads, 0, s>>>(iters, sink); break;
    case 2: k_peak<2><<<blocks, threads, 0, s>>>(iters, sink); break;
    default: k_peak<3><<<blocks, threads, 0, s>>>(iters, sink); break;
  }
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : record(c, DSMC_ERR_CUDA, "selftest_peak: launch failed");
}

}  // namespace dsmc
