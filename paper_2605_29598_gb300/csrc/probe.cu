// FMA-throughput probe: measures the FP64 and FP32 arithmetic roofs that
// the cell kernels of this library are bound by, on the GPU it runs on.
//
// Every thread runs CHAINS independent fused multiply-add chains
// x <- x * a + b for `iters` rounds (2 flops each); the grid fills every SM
// to its resident-thread limit, so the issue rate, not latency, limits the
// kernel.  a and b are kernel arguments, so the compiler cannot fold the
// chains; the results are stored so that they stay live.
#include "common.cuh"

namespace dg {

namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(T* __restrict__ out, int iters, T a, T b) {
  T x[PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run_probe(int device, int iters, double* tflops, double* ms_out, cudaStream_t st) {
  int sms = 0, per_sm = 0;
  DG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T>, PROBE_THREADS, 0));
  if (per_sm < 1) per_sm = 1;
  const int blocks = sms * per_sm;
  T* out = nullptr;
  DG_CUDA(cudaMalloc(&out, sizeof(T) * (size_t)blocks * PROBE_THREADS));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = DG_OK;
  float ms = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = cuda_fail(cudaGetLastError(), "cudaEventCreate");
  } else {
    const T a = (T)0.999999, b = (T)1e-7;
    for (int w = 0; w < 2; ++w) k_fma_probe<T><<<blocks, PROBE_THREADS, 0, st>>>(out, iters, a, b);
    cudaEventRecord(e0, st);
    k_fma_probe<T><<<blocks, PROBE_THREADS, 0, st>>>(out, iters, a, b);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "fma probe");
    else cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != DG_OK) return rc;
  const double flops = 2.0 * PROBE_CHAINS * (double)iters * blocks * PROBE_THREADS;
  *tflops = flops / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return DG_OK;
}

}  // namespace

}  // namespace dg

using namespace dg;

extern "C" int dg_probe_fma(dg_ctx* ctx, int bits, int iters, double* tflops, double* ms, void* stream) {
  if (!ctx || !tflops || (bits != 32 && bits != 64) || iters < 1) {
    set_error("dg_probe_fma: context, bits 32 or 64, iters >= 1 and an output are required");
    return DG_ERR_ARG;
  }
  int dev = -1;
  DG_CUDA(cudaGetDevice(&dev));
  if (dev != ctx->device) {
    set_error("dg_probe_fma: current device %d is not the context's device %d", dev, ctx->device);
    return DG_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  return bits == 64 ? run_probe<double>(dev, iters, tflops, ms, st) : run_probe<float>(dev, iters, tflops, ms, st);
}
