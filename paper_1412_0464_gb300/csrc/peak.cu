// hz_alu_peak: measured FP32 / FP64 fused multiply-add throughput of the
// device (the denominator of the ALU rooflines the benchmark reports for the
// Gauss-Jordan factorisation, which is bound by plain FMA arithmetic).
//
// Every thread runs kChains independent FMA recurrences (enough to hide the
// pipeline latency) for `iters` rounds; the grid holds 8 blocks of 256
// threads per SM.  The result is written so the compiler keeps the work.
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T a, T b, T* out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += x[c];
  if (acc == (T)-1.2345) out[blockIdx.x] = acc;   // practically never true
}

template <typename T>
double run_peak(int sms, cudaStream_t s, T* sink) {
  const int blocks = 8 * sms, threads = 256;
  const int iters = sizeof(T) == 4 ? 1 << 16 : 1 << 12;
  cudaEvent_t e0, e1;
  HZ_CU(cudaEventCreate(&e0));
  HZ_CU(cudaEventCreate(&e1));
  double best = 0;
  for (int rep = 0; rep < 4; ++rep) {     // the first run is a warm-up
    HZ_CU(cudaEventRecord(e0, s));
    fma_peak_kernel<T><<<blocks, threads, 0, s>>>(iters, (T)0.999, (T)1e-3, sink);
    HZ_CU(cudaEventRecord(e1, s));
    HZ_CU(cudaEventSynchronize(e1));
    float ms = 0;
    HZ_CU(cudaEventElapsedTime(&ms, e0, e1));
    const double flop = 2.0 * kChains * (double)iters * blocks * threads;
    if (rep > 0) best = std::max(best, flop / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

}  // namespace
}  // namespace hz

using namespace hz;

extern "C" hz_status hz_alu_peak(int precision, double* tflops, void* stream) {
  return run_guarded(nullptr, [&] {
    if (!tflops || (precision != HZ_PLAIN_FP64 && precision != HZ_MIXED))
      throw Failure(HZ_EINVAL, "hz_alu_peak: bad arguments");
    int dev = 0, sms = 1;
    HZ_CU(cudaGetDevice(&dev));
    HZ_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = (cudaStream_t)stream;
    void* sink = dmalloc(sizeof(double) * 8 * sms);
    try {
      *tflops = precision == HZ_MIXED ? run_peak<float>(sms, s, (float*)sink)
                                      : run_peak<double>(sms, s, (double*)sink);
    } catch (...) {
      dfree(sink);
      throw;
    }
    dfree(sink);
  });
}
