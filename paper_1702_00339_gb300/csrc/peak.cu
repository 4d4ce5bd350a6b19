// Measured arithmetic peaks of the device (the denominators of the FP64- and
// FP32-pipe roofline fractions the benchmark reports).  A grid of a few CTAs
// per SM runs, per thread, eight independent dependent chains of fused
// multiply-adds (enough independent work per warp to keep the pipe issuing);
// the count of FMAs is known exactly, so FLOP/s = 2 * FMAs / event time.
#include <cuda_runtime.h>

#include "../../include/fock.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T b, T c) {
  T a0 = (T)(threadIdx.x + 1) * (T)1e-3, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
  T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
    a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
  }
  const T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (s == (T)-1) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true; keeps the chains live
}

template <class T>
int measure(int device, int ctas_per_sm, int iters, double* tflops) {
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return FOCK_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int grid = sms * ctas_per_sm, threads = 256;
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FOCK_OK;
  if (cudaMalloc(&out, (size_t)grid * threads * sizeof(T)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = FOCK_ECUDA;
  } else {
    k_fma_peak<T><<<grid, threads>>>(out, iters / 8, (T)0.9999999, (T)1e-7);   // warm-up
    float best = 0.f;
    for (int r = 0; r < 3 && rc == FOCK_OK; ++r) {
      cudaEventRecord(e0);
      k_fma_peak<T><<<grid, threads>>>(out, iters, (T)0.9999999, (T)1e-7);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = FOCK_ECUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (best == 0.f || ms < best) best = ms;
    }
    if (rc == FOCK_OK) *tflops = 2.0 * 8.0 * (double)iters * grid * threads / (best * 1e-3) / 1e12;
  }
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) rc = FOCK_ECUDA;
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

}  // namespace

extern "C" int fock_measure_peaks(int device, double* fp64_tflops, double* fp32_tflops) {
  if (!fp64_tflops || !fp32_tflops) return FOCK_EINVAL;
  int rc = measure<double>(device, 8, 1 << 12, fp64_tflops);
  if (rc == FOCK_OK) rc = measure<float>(device, 8, 1 << 16, fp32_tflops);
  return rc;
}
