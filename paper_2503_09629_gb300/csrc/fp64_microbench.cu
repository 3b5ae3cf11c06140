// fp64_microbench.cu -- FP64 issue-rate microbenchmark (standalone program,
// not part of libsubcyc.so).  It measures how fast this GPU issues the FP64
// instructions the stencil and right-hand-side kernels are made of, which
// decides how those kernels write their arithmetic:
//   * DADD, DMUL and DFMA with 8 independent dependency chains per thread;
//   * fma(x, 1.0, a) with a literal 1 (the compiler folds it to a DADD) and
//     with a 1 passed as a kernel argument (stays a DFMA, bitwise x + a);
//   * DFMA throughput against warps per SM and chains per thread.
// Every kernel writes one value per thread so nothing is optimised away;
// out has room for the largest grid launched (blocks * threads doubles).
#include <cstdio>

#include <cuda_runtime.h>

namespace {

enum { kAdd = 0, kMul = 1, kFma = 2, kFmaLiteralOne = 3, kFmaArgOne = 4 };

template <int OP, int CHAINS>
__global__ void chains_kernel(double* out, int iters, double a, double b, double one) {
  double x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x * 1e-3 + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      if (OP == kAdd) x[c] = x[c] + a;
      if (OP == kMul) x[c] = x[c] * b;
      if (OP == kFma) x[c] = fma(x[c], b, a);
      if (OP == kFmaLiteralOne) x[c] = fma(x[c], 1.0, a);
      if (OP == kFmaArgOne) x[c] = fma(x[c], one, a);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// G instructions per second of one launch (after one untimed warm-up launch).
template <int OP, int CHAINS>
double rate(double* out, int blocks, int threads, int iters) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  chains_kernel<OP, CHAINS><<<blocks, threads>>>(out, 16, 1e-9, 1.0000001, 1.0);
  cudaEventRecord(e0);
  chains_kernel<OP, CHAINS><<<blocks, threads>>>(out, iters, 1e-9, 1.0000001, 1.0);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (double)CHAINS * iters * blocks * threads / (ms * 1e-3) / 1e9;
}

}  // namespace

int main() {
  int sms = 0, clock_khz = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, 0);
  const int max_blocks = sms * 8, threads = 256, iters = 4000;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * (size_t)max_blocks * threads) != cudaSuccess) {
    std::printf("cudaMalloc failed\n");
    return 1;
  }
  std::printf("SMs %d, max SM clock %.0f MHz, nominal DFMA issue %.1f G/s (2 per SM per clock)\n", sms,
              clock_khz / 1e3, sms * 2.0 * clock_khz / 1e6);
  const char* names[5] = {"DADD x+a", "DMUL x*b", "DFMA fma(x,b,a)", "fma(x,1.0,a) literal", "fma(x,one,a) argument"};
  for (int bpsm : {4, 8}) {
    const int blocks = sms * bpsm;
    const double r[5] = {rate<kAdd, 8>(out, blocks, threads, iters), rate<kMul, 8>(out, blocks, threads, iters),
                         rate<kFma, 8>(out, blocks, threads, iters),
                         rate<kFmaLiteralOne, 8>(out, blocks, threads, iters),
                         rate<kFmaArgOne, 8>(out, blocks, threads, iters)};
    for (int m = 0; m < 5; ++m)
      std::printf("blocks/SM %d, 8 chains  %-24s %7.1f G instr/s\n", bpsm, names[m], r[m]);
  }
  // DFMA against warps per SM (blocks of 32 threads) and chains per thread
  for (int warps : {1, 2, 4, 8}) {
    const int blocks = sms * warps;
    std::printf("warps/SM %d  DFMA G/s: 1 chain %7.1f  2 chains %7.1f  4 chains %7.1f  8 chains %7.1f\n", warps,
                rate<kFma, 1>(out, blocks, 32, iters), rate<kFma, 2>(out, blocks, 32, iters),
                rate<kFma, 4>(out, blocks, 32, iters), rate<kFma, 8>(out, blocks, 32, iters));
  }
  const cudaError_t e = cudaDeviceSynchronize();
  std::printf("status %s\n", cudaGetErrorString(e));
  cudaFree(out);
  return e == cudaSuccess ? 0 : 1;
}
