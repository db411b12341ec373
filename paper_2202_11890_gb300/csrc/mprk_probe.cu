// mprk_probe.cu — measures the GPU's FP64 fused multiply-add throughput,
// the denominator of the FP64 path's arithmetic roofline.
//
// Every thread runs NCHAIN independent dependency chains of double FMAs on
// registers only (no memory traffic inside the timed loop); four variants
// (8 or 16 chains, operands in registers or literals) run, and the fastest
// counts. The grid is one
// full wave: as many CTAs as fit on every SM at once, all running the same
// number of FMAs. Each CTA records its SM-clock cycles (clock64) and its
// start and end on the global nanosecond timer, between two block-wide
// barriers. The cycles over the nanoseconds of each CTA give
// the SM clock. The FMA rate is all FMAs over the span from the first CTA's
// start to the last CTA's end on the global timer: CTAs sharing an SM do
// not progress at the same pace (the oldest warps tend to win issue), so a
// single CTA's duration would not do.
// The result is stored only where it cannot be predicted, so the compiler
// keeps every FMA.
//
// It also holds the test hook of the FP64 tiles' reciprocal, reciprocal
// square root and square root (fp64_recip.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fp64_recip.cuh"
#include "mprk.h"
#include "mprk_internal.h"

namespace {

constexpr int PROBE_THREADS = 256;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// NCHAIN chains per thread; IMM: the FMA's multiplier and addend are
// literals (0.5, 0.25: x converges to 0.5) instead of registers.
template <int NCHAIN, bool IMM>
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
    for (int j = 0; j < NCHAIN; j++) x[j] = IMM ? fma(x[j], 0.5, 0.25) : fma(x[j], b, c);
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
    nanos[2 * blockIdx.x] = (long long)n0;  // the global timer is one clock for all SMs
    nanos[2 * blockIdx.x + 1] = (long long)n1;
  }
}

__global__ void recip_check_kernel(const double* x, int n, double* rcp, double* rsq, double* sq) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double v = x[j];
  rcp[j] = mprk::recip_f64(v);
  rsq[j] = mprk::rsqrt_f64(v);
  sq[j] = mprk::sqrt_f64(v);
}

}  // namespace

namespace {

struct ProbeResult {
  double gflops, dfma_per_clk, mhz;
};

// One variant: a warm-up launch and a measured one of a full wave.
template <int NCHAIN, bool IMM>
cudaError_t run_probe(long long iters, int nsm, cudaStream_t s, ProbeResult* out) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_fma_probe<NCHAIN, IMM>, PROBE_THREADS, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int blocks = nsm * per_sm;  // one full wave
  double* sink = nullptr;
  long long* cyc = nullptr;
  long long* ns = nullptr;
  std::vector<long long> hc(blocks), hn(2 * blocks);
  e = cudaMalloc(&sink, sizeof(double) * blocks * PROBE_THREADS);
  if (e == cudaSuccess) e = cudaMalloc(&cyc, sizeof(long long) * blocks);
  if (e == cudaSuccess) e = cudaMalloc(&ns, sizeof(long long) * 2 * blocks);
  if (e == cudaSuccess) {
    fp64_fma_probe<NCHAIN, IMM><<<blocks, PROBE_THREADS, 0, s>>>((int)(iters / 16 + 1), 0.999999, 1e-6, sink, cyc, ns);
    fp64_fma_probe<NCHAIN, IMM><<<blocks, PROBE_THREADS, 0, s>>>((int)iters, 0.999999, 1e-6, sink, cyc, ns);
    e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hn.data(), ns, sizeof(long long) * 2 * blocks, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    // the SM clock: the median over the CTAs of cycles per nanosecond; the
    // FMA rate: every FMA over first start to last end
    std::vector<double> clk(blocks);
    long long t_start = hn[0], t_end = hn[1];
    for (int j = 0; j < blocks; j++) {
      const long long d = hn[2 * j + 1] - hn[2 * j];
      clk[j] = d > 0 ? (double)hc[j] / (double)d : 0.0;
      t_start = std::min(t_start, hn[2 * j]);
      t_end = std::max(t_end, hn[2 * j + 1]);
    }
    std::sort(clk.begin(), clk.end());
    const double fmas = (double)blocks * PROBE_THREADS * NCHAIN * (double)iters;
    const double sec = (double)std::max(1ll, t_end - t_start) * 1e-9;
    out->mhz = clk[blocks / 2] * 1e3;
    out->gflops = 2.0 * fmas / sec / 1e9;
    out->dfma_per_clk = fmas / sec / (out->mhz * 1e6) / nsm;
  }
  if (sink) cudaFree(sink);
  if (cyc) cudaFree(cyc);
  if (ns) cudaFree(ns);
  return e;
}

}  // namespace

extern "C" int mprk_probe_fp64(long long iters, double* gflops, double* dfma_per_clk_per_sm, double* sm_mhz,
                               int* sms, double* max_mhz) {
  if (iters < 1 || iters > (1ll << 30) || !gflops || !dfma_per_clk_per_sm || !sm_mhz || !sms || !max_mhz) {
    mprk::set_last_error("mprk_probe_fp64: bad argument");
    return MPRK_EINVAL;
  }
  int dev = 0, nsm = 0, khz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  cudaStream_t s = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  // the fastest of four kernels: 8 or 16 chains per thread, FMA operands in
  // registers or literals (the chain count sets the work per thread, so the
  // 8-chain runs take twice the iterations)
  ProbeResult best{0.0, 0.0, 0.0}, r{0.0, 0.0, 0.0};
  auto keep = [&](cudaError_t er) {
    if (er == cudaSuccess && r.gflops > best.gflops) best = r;
    return er;
  };
  if (e == cudaSuccess) e = keep(run_probe<16, false>(iters, nsm, s, &r));
  if (e == cudaSuccess) e = keep(run_probe<16, true>(iters, nsm, s, &r));
  if (e == cudaSuccess) e = keep(run_probe<8, false>(2 * iters, nsm, s, &r));
  if (e == cudaSuccess) e = keep(run_probe<8, true>(2 * iters, nsm, s, &r));
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess || nsm < 1) {
    mprk::set_last_error(std::string("mprk_probe_fp64: ") + cudaGetErrorString(e));
    return MPRK_ECUDA;
  }
  *gflops = best.gflops;
  *dfma_per_clk_per_sm = best.dfma_per_clk;
  *sm_mhz = best.mhz;
  *sms = nsm;
  *max_mhz = khz * 1e-3;
  return MPRK_OK;
}

extern "C" int mprk_selftest_recip(const double* in_dev, int n, double* recip_dev, double* rsqrt_dev,
                                   double* sqrt_dev) {
  if (!in_dev || !recip_dev || !rsqrt_dev || !sqrt_dev || n < 0) {
    mprk::set_last_error("mprk_selftest_recip: bad argument");
    return MPRK_EINVAL;
  }
  if (n > 0) recip_check_kernel<<<(n + 255) / 256, 256>>>(in_dev, n, recip_dev, rsqrt_dev, sqrt_dev);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) {
    mprk::set_last_error(std::string("mprk_selftest_recip: ") + cudaGetErrorString(e));
    return MPRK_ECUDA;
  }
  return MPRK_OK;
}
