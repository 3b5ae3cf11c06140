// sc_measure.cu -- the FP64 issue rates of the current GPU, measured.
//
// Every kernel on this library's path is bound by the FP64 pipe, and its
// rate depends on the operands: a general fused multiply-add issues faster
// than an addition or a multiplication (or an FMA with a unit multiplier).
// The roofline of each kernel is therefore taken against measured rates of
// both kinds, beside the nominal unit count x clock figure.
#include <cuda_runtime.h>

#include "sc_internal.h"

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

// kind 0: x = fma(x, b, a) with b != 1 (a general DFMA); kind 1: x = x + a.
// a and b arrive as arguments so nothing folds; one value per thread is
// written so nothing is removed.
template <int KIND>
__global__ void fp64_chain_kernel(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * threadIdx.x + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = KIND == 0 ? fma(x[c], b, a) : x[c] + a;
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best of three timed launches after one untimed launch of the same length
// (the first launches of a process can run before the clocks have settled).
template <int KIND>
sc_status chain_rate(double* out, int blocks, int threads, int iters, cudaStream_t s, double* g_per_s) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return sc::set_last_error(SC_ECUDA, "cudaEventCreate failed");
  fp64_chain_kernel<KIND><<<blocks, threads, 0, s>>>(out, iters, 1e-9, 1.0000001);
  float best = 0.f;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    fp64_chain_kernel<KIND><<<blocks, threads, 0, s>>>(out, iters, 1e-9, 1.0000001);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 0.f && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || best <= 0.f) return sc::set_last_error(SC_ECUDA, "FP64 rate kernel failed");
  *g_per_s = (double)kChains * iters * blocks * threads / (best * 1e-3) / 1e9;
  return SC_OK;
}

}  // namespace

extern "C" sc_status sc_measure_fp64_peak(void* cuda_stream, double* dfma_g_per_s, double* dadd_g_per_s, int* sms,
                                          double* sm_clock_mhz) {
  if (!dfma_g_per_s || !dadd_g_per_s || !sms || !sm_clock_mhz) return sc::set_last_error(SC_EINVAL, "null argument");
  int dev = 0, nsm = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) ||
      cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev))
    return sc::set_last_error(SC_ECUDA, "device query failed");
  const int blocks = nsm * 8, threads = 256, iters = 4000;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads) != cudaSuccess) {
    cudaGetLastError();
    return sc::set_last_error(SC_ENOMEM, "device allocation failed");
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  sc_status st = chain_rate<0>(out, blocks, threads, iters, s, dfma_g_per_s);
  if (st == SC_OK) st = chain_rate<1>(out, blocks, threads, iters, s, dadd_g_per_s);
  cudaFree(out);
  *sms = nsm;
  *sm_clock_mhz = khz / 1e3;
  return st;
}
