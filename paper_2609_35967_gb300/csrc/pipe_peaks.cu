// pipe_peaks.cu -- FMA-chain microbenchmarks of the FP32 and FP64 pipes (libgdpeaks.so).
//
// Measurement only: the roofline denominators of the arithmetic pipes.  Each thread runs
// CH independent dependent chains y <- y * b + a (one FMA, two flops each), enough to keep
// the pipe busy at full occupancy; the grid is 8 blocks of 256 threads per SM.  The chains
// converge to a / (1 - b) = 1 and stay finite; the sum is written only when it equals a
// value it never takes, so the compiler cannot drop the chains.  Timed with CUDA events
// around repeated launches (best of the repetitions).  Nothing here changes a clock or
// any other setting of the GPU.
#include <cuda_runtime.h>

namespace {

template <typename T, int CH>
__global__ void __launch_bounds__(256) k_fma_chain(T* out, T a, T b, int iters) {
  T y[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) y[c] = (T)threadIdx.x * (T)1e-7 + (T)c * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < CH; ++c) y[c] = fma(y[c], b, a);
    }
  }
  T s = (T)0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += y[c];
  if (s == (T)-1.25) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, int CH>
int run(double* tflops, double* ms_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -2;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -2;
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(T) == 4 ? 4096 : 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -3;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T a = (T)1e-6, b = (T)(1.0 - 1e-6);
  float best = 1e30f;
  int rc = 0;
  for (int rep = 0; rep < 6 && rc == 0; ++rep) {
    cudaEventRecord(e0);
    k_fma_chain<T, CH><<<blocks, threads>>>(out, a, b, iters);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = -2; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;     // the first launch warms up
  }
  if (cudaGetLastError() != cudaSuccess) rc = -2;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != 0) return rc;
  const double flops = 2.0 * CH * 16.0 * (double)iters * (double)blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return 0;
}

}  // namespace

// Peak FMA throughput of one pipe in TFLOP/s (2 flops per FMA): fp64 = 0 the FP32 pipe,
// 1 the FP64 pipe.  ms_out (HOST, or NULL): the best launch time.  Returns 0, or a
// negative code when a CUDA call failed.  Synchronises the device.
extern "C" int gdp_fma_tflops(int fp64, double* tflops_out, double* ms_out) {
  if (!tflops_out) return -1;
  return fp64 ? run<double, 8>(tflops_out, ms_out) : run<float, 8>(tflops_out, ms_out);
}
