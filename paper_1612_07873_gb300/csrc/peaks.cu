// Measured CUDA-core arithmetic peaks (FP32 and FP64 fused multiply-add),
// the denominators of the rooflines of the kernels bound by the FP32 pipe
// (the Galerkin product) and the FP64 pipe (the block Gram-Schmidt, the
// FP64 fine operator).  Each thread runs CH independent FMA chains; the
// grid fills every SM several times over; the result is timed with CUDA
// events on the caller's stream.
#include "kernels.cuh"

namespace gbmg {

namespace {

template <typename R, int CH>
__global__ void __launch_bounds__(256) k_fma_chains(R* __restrict__ sink, int iters, R a, R b) {
  R v[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) v[c] = R(threadIdx.x + c) * R(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < CH; ++c) v[c] = fma(v[c], a, b);
  }
  R s = R(0);
#pragma unroll
  for (int c = 0; c < CH; ++c) s += v[c];
  // a store the compiler cannot prove dead: sink is written only when the
  // chains produce an exact sentinel, which a, b chosen by the host avoid
  if (s == R(-1.25)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename R>
double time_fma(cudaStream_t st) {
  constexpr int CH = 8;
  int dev = 0, sms = 0;
  GB_CHECK(cudaGetDevice(&dev));
  GB_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(R) == 4 ? 4096 : 256;
  DevBuf sink;
  sink.alloc(size_t(blocks) * threads * sizeof(R));
  // a slightly below 1 and b small keep the chains finite and away from -1.25
  const R a = R(0.999999), b = R(1e-7);
  k_fma_chains<R, CH><<<blocks, threads, 0, st>>>(sink.as<R>(), iters, a, b);  // warm-up
  GB_LAUNCH_CHECK();
  cudaEvent_t e0, e1;
  GB_CHECK(cudaEventCreate(&e0));
  GB_CHECK(cudaEventCreate(&e1));
  constexpr int reps = 5;
  GB_CHECK(cudaEventRecord(e0, st));
  for (int r = 0; r < reps; ++r)
    k_fma_chains<R, CH><<<blocks, threads, 0, st>>>(sink.as<R>(), iters, a, b);
  GB_CHECK(cudaEventRecord(e1, st));
  GB_CHECK(cudaEventSynchronize(e1));
  float ms = 0.f;
  GB_CHECK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  GB_LAUNCH_CHECK();
  const double flops = 2.0 * double(blocks) * threads * double(iters) * 16 * CH * reps;
  return flops / (double(ms) * 1e-3) / 1e12;
}

}  // namespace

}  // namespace gbmg

extern "C" mg_status mg_fma_peak(int prec, double* tflops, void* stream) {
  using namespace gbmg;
  try {
    GB_REQUIRE(tflops, MG_ERR_ARG, "fma_peak: null output");
    GB_REQUIRE(prec == MG_F32 || prec == MG_F64, MG_ERR_ARG, "fma_peak: prec must be F32 or F64");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    *tflops = prec == MG_F32 ? time_fma<float>(st) : time_fma<double>(st);
    return MG_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}
