// jz_peak.cu -- measured fused multiply-add throughput of the current GPU,
// the denominator of the ALU rooflines: FP64 for the FP64 stage kernel,
// which GB300's FP64 rate bounds long before HBM does, and FP32 for the FP32
// kernel's arithmetic figure.
//
// Every thread runs eight independent FMA chains a <- a * b + c (b just below
// one, so the values settle instead of growing); 8 blocks of 256 threads per
// SM keep the pipes fed.  Timed with CUDA events after one warm-up launch,
// best of three.
#include <cmath>

#include "jz_internal.h"

namespace jz {

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PK_THREADS) k_fma_chains(T* sink, int iters, T b, T c) {
  T a[PK_CHAINS];
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
  if (s == T(-1)) *sink = s;  // never true; keeps the chains live
}

template <typename T>
int measure(int iters, double* tflops, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return record_error(JZ_ECUDA, "cannot query the device");
  const int blocks = 8 * sms;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return record_error(JZ_ECUDA, "cudaEventCreate failed");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return record_error(JZ_ECUDA, "cudaEventCreate failed");
  }
  double best = 0.0;
  cudaError_t err = cudaSuccess;
  for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_chains<T><<<blocks, PK_THREADS, 0, s>>>(nullptr, iters, T(0.999999), T(1e-6));
    count_launches(1);
    cudaEventRecord(e1, s);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && rep > 0 && ms > 0.f) {
      const double flops = 2.0 * PK_CHAINS * (double)iters * (double)blocks * PK_THREADS;
      best = fmax(best, flops / (ms * 1e-3) / 1e12);
    }
  }
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return record_error(JZ_ECUDA, cudaGetErrorString(err));
  *tflops = best;
  return JZ_OK;
}

}  // namespace

}  // namespace jz

using namespace jz;

extern "C" int jz_fma_peak(int fp64, double* tflops, void* stream) {
  if (!tflops) return record_error(JZ_EINVAL, "null output");
  if (fp64 != 0 && fp64 != 1) return record_error(JZ_EINVAL, "fp64 must be 0 or 1");
  cudaStream_t s = (cudaStream_t)stream;
  return fp64 ? measure<double>(1 << 12, tflops, s) : measure<float>(1 << 16, tflops, s);
}
