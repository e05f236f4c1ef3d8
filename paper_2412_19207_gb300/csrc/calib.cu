// Device calibration: the measured rates of the arithmetic the double-float
// and float64 kernels are bound by, for their roofline denominators.
//   df32: the double-float multiply-add of the Schwarz apply and the inner
//         operator (df_mac_f_x2: exact product, two-sum, low-order terms by
//         FMAs, two at a time in packed float32x2 operations), counted as 2
//         flops each;
//   fp64: float64 FMAs, 2 flops each.
// Each thread runs 8 independent chains (enough to cover the pipelines'
// latency at full occupancy); the grid fills every SM several times over.
#include "common.cuh"
#include "df32.cuh"

namespace {

constexpr int CAL_T = 256;
constexpr int CAL_CHAINS = 8;

// the packed form the kernels use (df_mac_f_x2: two chains per call)
__global__ void __launch_bounds__(CAL_T) df_rate_kernel(int iters, float seed, float* __restrict__ sink) {
  float2 h[CAL_CHAINS / 2], l[CAL_CHAINS / 2];
  const float2 ah = make_float2(1.0f + seed * 1e-7f, 1.0f - seed * 1e-7f), al = make_float2(seed * 1e-15f, 0.f);
  const float2 xh = make_float2(0.999999f, 0.999998f), xl = make_float2(1e-9f * seed, -1e-9f * seed);
#pragma unroll
  for (int c = 0; c < CAL_CHAINS / 2; ++c) {
    h[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)(threadIdx.x - c) * 1e-3f);
    l[c] = make_float2(0.f, 0.f);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CAL_CHAINS / 2; ++c) df_mac_f_x2(h[c], l[c], ah, al, xh, xl);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CAL_CHAINS / 2; ++c) s += h[c].x + l[c].x + h[c].y + l[c].y;
  if (s == 1234.5f) sink[blockIdx.x] = s;     // never true in practice: keeps the chains live
}

__global__ void __launch_bounds__(CAL_T) fp64_rate_kernel(int iters, double seed, double* __restrict__ sink) {
  double v[CAL_CHAINS];
#pragma unroll
  for (int c = 0; c < CAL_CHAINS; ++c) v[c] = (double)(threadIdx.x + c) * 1e-3;
  const double a = 1.0 - seed * 1e-12, b = seed * 1e-9;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CAL_CHAINS; ++c) v[c] = fma(v[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CAL_CHAINS; ++c) s += v[c];
  if (s == 1234.5) sink[blockIdx.x] = s;
}

template <typename F>
cudaError_t time_ms(F launch, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  launch();                                  // warm-up
  cudaEventRecord(e0, 0);
  launch();
  cudaEventRecord(e1, 0);
  e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" rann_status rann_dd_device_rates(double* df32_tflops, double* fp64_tflops) {
  if (!df32_tflops && !fp64_tflops) return RANN_OK;
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = nsm * 8;
  void* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * (size_t)blocks) != cudaSuccess) {
    rann_set_error("rann_dd_device_rates: allocation failed");
    return RANN_ENOMEM;
  }
  cudaError_t e = cudaSuccess;
  if (df32_tflops) {
    const int iters = 4096;
    float ms = 0.f;
    e = time_ms([&] { df_rate_kernel<<<blocks, CAL_T>>>(iters, 0.5f, (float*)sink); }, &ms);
    if (e == cudaSuccess) *df32_tflops = 2.0 * blocks * CAL_T * (double)iters * CAL_CHAINS / (ms * 1e-3) / 1e12;
  }
  if (e == cudaSuccess && fp64_tflops) {
    const int iters = 1024;
    float ms = 0.f;
    e = time_ms([&] { fp64_rate_kernel<<<blocks, CAL_T>>>(iters, 0.5, (double*)sink); }, &ms);
    if (e == cudaSuccess) *fp64_tflops = 2.0 * blocks * CAL_T * (double)iters * CAL_CHAINS / (ms * 1e-3) / 1e12;
  }
  cudaFree(sink);
  if (e != cudaSuccess) {
    rann_set_error("rann_dd_device_rates: %s", cudaGetErrorString(e));
    return RANN_ECUDA;
  }
  return RANN_OK;
}
