// Measurement and self-test hooks of the library (not part of the method):
//   - the pivot reciprocal recip_nr applied element-wise, so that a test can
//     compare it with the IEEE division 1.0/d over any set of inputs;
//   - FP64 throughput probes (plain FMA and the f64 mma.sync tensor-core
//     instruction) that measure the FP64 peak the factorization's roofline is
//     judged against.
#include <cuda_runtime.h>

#include "../../include/nmpc.h"
#include "kernels.h"

using namespace nmpc;

namespace {

__device__ double g_probe_sink;  // written only if a probe's result takes an impossible value

__global__ void k_recip_apply(const double* in, double* out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = recip_nr(in[i]);
}

// FP64 FMA probe: every thread runs CH independent chains of dependent FMAs
// (x <- x * a + b), so the FP64 pipe, not a chain's latency, sets the pace.
// The values stay bounded (a < 1) and are written out so nothing is removed.
constexpr int CH = 8;
__global__ void __launch_bounds__(256) k_probe_fma(int iters, double a, double b) {
  double x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  if (s == 12345.678) g_probe_sink = s;  // never true (x tends to 0.1); keeps the chains live
}

// FP64 tensor-core probe: per warp, CH independent 8x8 accumulators updated
// by mma.sync.m8n8k4 (f64 inputs and accumulators; 512 flops per instruction).
__global__ void __launch_bounds__(256) k_probe_dmma(int iters, double a, double b) {
  double acc[CH][2];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c][0] = acc[c][1] = 0.0;
  const double fa = a * (1.0 + 1e-6 * (threadIdx.x & 31)), fb = b;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(acc[c][0]), "+d"(acc[c][1])
                   : "d"(fa), "d"(fb));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += acc[c][0] + acc[c][1];
  if (s == 12345.678) g_probe_sink = s;
}

}  // namespace

extern "C" {

nmpc_status nmpc_debug_recip(const double* in, double* out, long long n, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!in || !out))) return NMPC_ERR_INVALID;
  if (n == 0) return NMPC_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  k_recip_apply<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
  return cudaGetLastError() == cudaSuccess ? NMPC_OK : NMPC_ERR_CUDA;
}

nmpc_status nmpc_probe_fp64(int kind, int blocks_per_sm, int iters, void* cuda_stream, double* tflops) {
  if ((kind != 0 && kind != 1) || blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || !tflops)
    return NMPC_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return NMPC_ERR_CUDA;
  const int blocks = sms * blocks_per_sm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return NMPC_ERR_CUDA;
  // warm-up launch, then the timed one
  for (int rep = 0; rep < 2; ++rep) {
    if (rep == 1) cudaEventRecord(e0, st);
    if (kind == 0) k_probe_fma<<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-7);
    else k_probe_dmma<<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-7);
  }
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) return NMPC_ERR_CUDA;
  const double threads = (double)blocks * 256.0;
  const double flops = kind == 0 ? threads * iters * CH * 2.0                 // one FMA per chain step
                                 : (threads / 32.0) * iters * CH * 512.0;     // 8x8x4 multiply-adds per mma
  *tflops = flops / (ms * 1e-3) / 1e12;
  return NMPC_OK;
}

}  // extern "C"
