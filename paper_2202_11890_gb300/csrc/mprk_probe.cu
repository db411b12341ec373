// mprk_probe.cu — measures the GPU's FP64 fused multiply-add throughput,
// the denominator of the FP64 path's arithmetic roofline.
//
// Every thread runs NCHAIN independent dependency chains of double FMAs on
// registers only (no memory traffic inside the timed loop). The grid is one
// full wave: as many CTAs as fit on every SM at once, all running the same
// number of FMAs. Each CTA records its own SM-clock cycles (clock64) and
// nanoseconds (globaltimer) between two block-wide barriers, which gives
// the SM clock and the FMAs per SM clock independent of launch overhead.
// The result is stored only where it cannot be predicted, so the compiler
// keeps every FMA.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "mprk.h"
#include "mprk_internal.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int NCHAIN = 16;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(PROBE_THREADS) fp64_fma_probe(int iters, double b, double c, double* sink,
                                                                 long long* cycles, long long* nanos) {
  double x[NCHAIN];
#pragma unroll
  for (int j = 0; j < NCHAIN; j++) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  __syncthreads();
  const long long c0 = clock64();
  const unsigned long long n0 = global_ns();
#pragma unroll 2
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int j = 0; j < NCHAIN; j++) x[j] = fma(x[j], b, c);
  }
  __syncthreads();
  const long long c1 = clock64();
  const unsigned long long n1 = global_ns();
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < NCHAIN; j++) s += x[j];
  if (s == -1.0) sink[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;  // never true for b, c > 0
  if (threadIdx.x == 0) {
    cycles[blockIdx.x] = c1 - c0;
    nanos[blockIdx.x] = (long long)(n1 - n0);
  }
}

}  // namespace

extern "C" int mprk_probe_fp64(long long iters, double* gflops, double* dfma_per_clk_per_sm, double* sm_mhz,
                               int* sms) {
  if (iters < 1 || iters > (1ll << 30) || !gflops || !dfma_per_clk_per_sm || !sm_mhz || !sms) {
    mprk::set_last_error("mprk_probe_fp64: bad argument");
    return MPRK_EINVAL;
  }
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_fma_probe, PROBE_THREADS, 0);
  if (e != cudaSuccess || nsm < 1 || per_sm < 1) {
    mprk::set_last_error(std::string("mprk_probe_fp64: ") + cudaGetErrorString(e));
    return MPRK_ECUDA;
  }
  const int blocks = nsm * per_sm;  // one full wave
  double* sink = nullptr;
  long long* cyc = nullptr;
  long long* ns = nullptr;
  cudaStream_t s = nullptr;
  int rc = MPRK_OK;
  std::vector<long long> hc(blocks), hn(blocks);
  e = cudaMalloc(&sink, sizeof(double) * blocks * PROBE_THREADS);
  if (e == cudaSuccess) e = cudaMalloc(&cyc, sizeof(long long) * blocks);
  if (e == cudaSuccess) e = cudaMalloc(&ns, sizeof(long long) * blocks);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    // a short warm-up launch, then the measured one
    fp64_fma_probe<<<blocks, PROBE_THREADS, 0, s>>>((int)(iters / 16 + 1), 0.999999, 1e-6, sink, cyc, ns);
    fp64_fma_probe<<<blocks, PROBE_THREADS, 0, s>>>((int)iters, 0.999999, 1e-6, sink, cyc, ns);
    e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hn.data(), ns, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    mprk::set_last_error(std::string("mprk_probe_fp64: ") + cudaGetErrorString(e));
    rc = MPRK_ECUDA;
  } else {
    // medians over the CTAs: cycles and nanoseconds of one CTA's loop; all
    // CTAs of the wave share their SM's FP64 units the whole time
    std::vector<double> clk(blocks);
    for (int j = 0; j < blocks; j++) clk[j] = hn[j] > 0 ? (double)hc[j] / (double)hn[j] : 0.0;  // cycles per ns
    std::sort(clk.begin(), clk.end());
    std::sort(hc.begin(), hc.end());
    std::sort(hn.begin(), hn.end());
    const double cyc_med = (double)hc[blocks / 2], ns_med = (double)hn[blocks / 2];
    const double fmas_per_sm = (double)per_sm * PROBE_THREADS * NCHAIN * (double)iters;
    *dfma_per_clk_per_sm = fmas_per_sm / cyc_med;
    *sm_mhz = clk[blocks / 2] * 1e3;
    *gflops = 2.0 * fmas_per_sm * nsm / (ns_med * 1e-9) / 1e9;
    *sms = nsm;
  }
  if (s) cudaStreamDestroy(s);
  if (sink) cudaFree(sink);
  if (cyc) cudaFree(cyc);
  if (ns) cudaFree(ns);
  return rc;
}
