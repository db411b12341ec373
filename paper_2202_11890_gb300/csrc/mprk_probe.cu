// mprk_probe.cu — measures the GPU's FP64 fused multiply-add throughput,
// the denominator of the FP64 path's arithmetic roofline.
//
// Every thread runs NCHAIN independent dependency chains of double FMAs on
// registers only (no memory traffic inside the timed loop), on enough CTAs
// to fill every SM several times over. The result is stored only where it
// cannot be predicted, so the compiler keeps every FMA.
#include <cuda_runtime.h>

#include "mprk.h"
#include "mprk_internal.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int NCHAIN = 8;

__global__ void __launch_bounds__(PROBE_THREADS) fp64_fma_probe(long long iters, double b, double c,
                                                                 double* sink, long long* cycles) {
  double x[NCHAIN];
#pragma unroll
  for (int j = 0; j < NCHAIN; j++) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  const long long t0 = clock64();
  for (long long it = 0; it < iters; it++) {
#pragma unroll
    for (int j = 0; j < NCHAIN; j++) x[j] = fma(x[j], b, c);
  }
  const long long t1 = clock64();
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < NCHAIN; j++) s += x[j];
  if (s == -1.0) sink[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;  // never true for b, c > 0
  if (threadIdx.x == 0 && blockIdx.x == 0) *cycles = t1 - t0;
}

}  // namespace

extern "C" int mprk_probe_fp64(long long iters, double* gflops, double* dfma_per_clk_per_sm, double* sm_mhz,
                               int* sms) {
  if (iters < 1 || !gflops || !dfma_per_clk_per_sm || !sm_mhz || !sms) {
    mprk::set_last_error("mprk_probe_fp64: bad argument");
    return MPRK_EINVAL;
  }
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || nsm < 1) {
    mprk::set_last_error(std::string("mprk_probe_fp64: ") + cudaGetErrorString(e));
    return MPRK_ECUDA;
  }
  const int blocks = nsm * 8;  // eight CTAs of eight warps per SM
  double* sink = nullptr;
  long long* cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s = nullptr;
  int rc = MPRK_OK;
  float ms = 0.f;
  long long cycles = 0;
  e = cudaMalloc(&sink, sizeof(double) * blocks * PROBE_THREADS);
  if (e == cudaSuccess) e = cudaMalloc(&cyc, sizeof(long long));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    // one short warm-up launch, then the timed one
    fp64_fma_probe<<<blocks, PROBE_THREADS, 0, s>>>(iters / 16 + 1, 0.999999, 1e-6, sink, cyc);
    cudaEventRecord(e0, s);
    fp64_fma_probe<<<blocks, PROBE_THREADS, 0, s>>>(iters, 0.999999, 1e-6, sink, cyc);
    cudaEventRecord(e1, s);
    e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaMemcpy(&cycles, cyc, sizeof(long long), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    mprk::set_last_error(std::string("mprk_probe_fp64: ") + cudaGetErrorString(e));
    rc = MPRK_ECUDA;
  } else {
    const double fmas = (double)blocks * PROBE_THREADS * NCHAIN * (double)iters;
    const double sec = ms * 1e-3;
    *gflops = 2.0 * fmas / sec / 1e9;
    *sm_mhz = cycles / sec / 1e6;  // CTA 0's clock over the launch
    *dfma_per_clk_per_sm = fmas / (sec * (*sm_mhz) * 1e6) / nsm;
    *sms = nsm;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (sink) cudaFree(sink);
  if (cyc) cudaFree(cyc);
  return rc;
}
