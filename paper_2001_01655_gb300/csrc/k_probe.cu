// FP64 fused multiply-add throughput of the CUDA cores.  The FP64 outer operator is bound by
// this rate, so its roofline needs it as a denominator; like the copy bandwidth and the GEMM
// rate of the other bounds it is measured rather than taken from the data sheet.  Every
// thread runs eight independent FMA chains (enough to cover the pipeline latency at full
// occupancy) for a fixed number of steps.
#include "ops.h"

namespace tomg {

namespace {

constexpr int CHAINS = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(int iters, double a, double b, double* sink) {
  double v[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; k++) v[k] = 1e-3 * (double)(threadIdx.x + k);
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int k = 0; k < CHAINS; k++) v[k] = fma(v[k], a, b);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CHAINS; k++) s += v[k];
  // the chains stay positive, so this store never happens; it keeps them live
  if (s < 0.0) sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

double fp64_fma_tflops(cudaStream_t s, int device) {
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int blocks = 8 * sms, threads = 256, iters = 2048;
  DBuf<double> sink;
  sink.resize((int64_t)blocks * threads);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 0.f;
  for (int rep = 0; rep < 6; rep++) {  // the first launch warms up
    CK(cudaEventRecord(e0, s));
    LAUNCH(k_fp64_fma, blocks, threads, 0, s, iters, 0.999999, 1e-6, sink.p);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * CHAINS * (double)iters * blocks * threads;
  return flops / (best * 1e-3) / 1e12;
}

}  // namespace tomg
