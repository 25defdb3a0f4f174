// Measured arithmetic peaks of the device: the FP64 (DFMA) and FP32 (FFMA) rates that bound the
// FP64 path and the ALU-bound stages of the mixed forms (the noise filter, the ring DFTs).
//
// Each thread runs eight independent fused multiply-add chains; the grid holds eight 256-thread
// blocks per SM, enough warps to keep every pipe busy.  Two warm-up launches, then the median of
// five launches timed with CUDA events on a private stream.  The chains cannot be folded by the
// compiler (the multiplier and addend are kernel arguments and every chain feeds the output).
#include <algorithm>
#include <vector>

#include "fnl_internal.cuh"

namespace fnl {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  T t = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) t += x[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

template <typename T>
double fma_rate(int device, int iters) {
  int sms = 0;
  FNL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int blocks = sms * 8, threads = 256;
  TempDev out(sizeof(T) * (size_t)blocks * threads);
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FNL_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  std::vector<float> ms;
  try {
    FNL_CUDA(cudaEventCreate(&e0));
    FNL_CUDA(cudaEventCreate(&e1));
    for (int w = 0; w < 2; ++w) k_fma_chains<T><<<blocks, threads, 0, st>>>(out.as<T>(), iters, (T)0.999, (T)0.5);
    FNL_CUDA(cudaGetLastError());
    for (int r = 0; r < 5; ++r) {
      FNL_CUDA(cudaEventRecord(e0, st));
      k_fma_chains<T><<<blocks, threads, 0, st>>>(out.as<T>(), iters, (T)0.999, (T)0.5);
      FNL_CUDA(cudaEventRecord(e1, st));
      FNL_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      FNL_CUDA(cudaEventElapsedTime(&t, e0, e1));
      ms.push_back(t);
    }
  } catch (...) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FNL_CUDA(cudaStreamDestroy(st));
  std::sort(ms.begin(), ms.end());
  const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  return flops / (ms[ms.size() / 2] * 1e-3) / 1e12;
}

}  // namespace

}  // namespace fnl

extern "C" fnl_status fnl_measure_fma_peaks(int device, double* fp64_tflops, double* fp32_tflops) {
  using namespace fnl;
  return guard([&] {
    int ndev = 0;
    FNL_CUDA(cudaGetDeviceCount(&ndev));
    FNL_REQUIRE(device >= 0 && device < ndev, "no such CUDA device");
    DeviceScope scope(device);
    // about 10 ms per timed launch at the nominal GB300 rates (1.25 and 80 TFLOP/s)
    if (fp64_tflops) *fp64_tflops = fma_rate<double>(device, 2500);
    if (fp32_tflops) *fp32_tflops = fma_rate<float>(device, 160000);
  });
}
