// Measured throughput of the arithmetic units that bound the library's kernels: the
// transcendental unit (tanh.approx, ex2.approx, rcp.approx: the activations of the
// embedding and fitting nets), FP32 FMA and FP64 FMA.  The denominators of the rooflines
// that are not a tensor-core or memory bound come from here, measured on the device in
// use rather than assumed.
//
// Each thread runs kChains independent dependent chains of one instruction; the grid
// fills every SM with 8 blocks of 256 threads, so the unit is throughput-bound, not
// latency-bound.  Timed with CUDA events on a private stream after one warm-up launch;
// the fastest of three launches is reported.
#include "common.cuh"

namespace dpg {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

enum PeakOp { P_TANH = 0, P_EX2 = 1, P_RCP = 2, P_FFMA = 3, P_DFMA = 4 };

template <int OP>
struct PeakT { using type = float; };
template <>
struct PeakT<P_DFMA> { using type = double; };

template <int OP>
__device__ __forceinline__ typename PeakT<OP>::type peak_step(typename PeakT<OP>::type x,
                                                              typename PeakT<OP>::type mul,
                                                              typename PeakT<OP>::type add) {
  if constexpr (OP == P_TANH) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  } else if constexpr (OP == P_EX2) {
    float y;  // 2^-x keeps the chain inside (0, 1)
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    return y;
  } else if constexpr (OP == P_RCP) {
    float y;  // 1 / (x + 1): the added one keeps rcp(rcp(x)) from folding to x
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x + 1.f));
    return y;
  } else if constexpr (OP == P_FFMA) {
    return fmaf(x, mul, add);
  } else {
    return fma(x, mul, add);
  }
}

// Never written in practice: the chains' sum is compared with a value it cannot take, which
// keeps the compiler from dropping them without any memory traffic or allocation.
__device__ float g_sink_f;
__device__ double g_sink_d;

// mul and add arrive as kernel arguments, so the FMA operands are registers (not constants).
template <int OP>
__global__ void __launch_bounds__(kPeakThreads) k_peak(int iters, typename PeakT<OP>::type mul,
                                                       typename PeakT<OP>::type add) {
  using T = typename PeakT<OP>::type;
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(0.25) + T(0.01) * T((threadIdx.x + c) & 31);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = peak_step<OP>(x[c], mul, add);
  }
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += x[c];
  if (acc == T(-12345.0)) {
    if constexpr (sizeof(T) == 8) g_sink_d = acc;
    else g_sink_f = acc;
  }
}

template <int OP>
dp_status time_peak(int iters, double per_instr, double* rate, std::string& why) {
  const int grid = 8 * num_sms();
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  dp_status status = DP_OK;
  float best = 1e30f;
  auto fail = [&](const char* what, cudaError_t e) {
    why = std::string(what) + ": " + cudaGetErrorString(e);
    status = DP_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) fail("stream", e);
  if (status == DP_OK && (e = cudaEventCreate(&e0)) != cudaSuccess) fail("event", e);
  if (status == DP_OK && (e = cudaEventCreate(&e1)) != cudaSuccess) fail("event", e);
  for (int r = 0; r < 4 && status == DP_OK; ++r) {  // launch 0 warms up
    cudaEventRecord(e0, st);
    k_peak<OP><<<grid, kPeakThreads, 0, st>>>(iters, typename PeakT<OP>::type(0.9999),
                                              typename PeakT<OP>::type(1e-4));
    cudaEventRecord(e1, st);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) {
      fail("peak kernel", e);
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < best) best = ms;
  }
  if (st) cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (status == DP_OK) {
    const double ops = (double)grid * kPeakThreads * kChains * (double)iters * per_instr;
    *rate = ops / (best * 1e-3);
  }
  return status;
}

}  // namespace
}  // namespace dpg

using namespace dpg;

extern "C" dp_status dp_measure_peak(int which, double* rate) {
  if (!rate) return DP_ERR_ARG;
  std::string why;
  dp_status st;
  switch (which) {
    case P_TANH: st = time_peak<P_TANH>(16384, 1.0, rate, why); break;
    case P_EX2: st = time_peak<P_EX2>(16384, 1.0, rate, why); break;
    case P_RCP: st = time_peak<P_RCP>(16384, 1.0, rate, why); break;
    case P_FFMA: st = time_peak<P_FFMA>(65536, 2.0, rate, why); break;
    case P_DFMA: st = time_peak<P_DFMA>(1024, 2.0, rate, why); break;
    default: return DP_ERR_ARG;
  }
  return st;
}
