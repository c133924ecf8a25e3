// Tensor-core (tcgen05 / TMEM) support of the mixed-precision path: the
// built-in operand-layout self check, device capability query, and the 16-bit
// weight copies used by the mixed-precision kernels.
#include "tc_common.cuh"

namespace dpg {

bool tc_available(const Model*) {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3;
}

namespace {

// One CTA: D[128 x N] = A[128 x 64*KB] * B[N x 64*KB]^T with small exact values, A and
// B written by threads into K-major SW128 blocks; every output compared with the
// exact integer-valued reference.  out[0] = max |error|, out[1] = max |reference|.
template <int N, int KB, bool F16>
__global__ void __launch_bounds__(128) k_mma_selftest(float* out, int* err) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  unsigned char* sm = sm_raw + ((1024u - (tc::smem_u32(sm_raw) & 1023u)) & 1023u);
  unsigned char* A = sm;                         // KB blocks of 128 x 128 B
  unsigned char* B = sm + KB * 128 * 128;        // KB blocks of N x 128 B
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int t = threadIdx.x, w = t >> 5;
  auto aval = [](int r, int k) { return (float)(((r * 7 + k * 3) % 17) - 8) * 0.125f; };
  auto bval = [](int n, int k) { return (float)(((n * 5 + k * 11) % 13) - 6) * 0.25f; };
  for (int kb = 0; kb < KB; ++kb)
    for (int k0 = 0; k0 < 64; k0 += 8) {
      uint4 v;
      uint32_t* p = reinterpret_cast<uint32_t*>(&v);
      for (int q = 0; q < 4; ++q)
        p[q] = tc::pack2<F16>(aval(t, kb * 64 + k0 + 2 * q), aval(t, kb * 64 + k0 + 2 * q + 1));
      tc::st_chunk(A + kb * 16384, t, k0, v);
    }
  for (int n = t; n < N; n += 128)
    for (int kb = 0; kb < KB; ++kb)
      for (int k0 = 0; k0 < 64; k0 += 8) {
        uint4 v;
        uint32_t* p = reinterpret_cast<uint32_t*>(&v);
        for (int q = 0; q < 4; ++q)
          p[q] = tc::pack2<F16>(bval(n, kb * 64 + k0 + 2 * q), bval(n, kb * 64 + k0 + 2 * q + 1));
        tc::st_chunk(B + kb * N * 128, n, k0, v);
      }
  if (t == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
  }
  if (w == 0) {
    tc::tmem_alloc(&tslot, 256);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tslot;
  if (t == 0) {
    constexpr uint32_t idesc = tc::idesc_f16(128, N, F16);
    for (int kb = 0; kb < KB; ++kb)
      tc::mma_kblock(tmem, tc::smem_u32(A + kb * 16384), tc::smem_u32(B + kb * N * 128), idesc, kb > 0);
    tc::mma_commit(&bar);
  }
  bool ok = tc::mbar_wait(&bar, 0, err);
  tc::tc_fence_after();
  float emax = 0.f, rmax = 0.f;
  if (ok) {
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * w) << 16) + c0, v);
      tc::tmem_wait_ld();
      for (int u = 0; u < 16; ++u) {
        float ref = 0.f;
        for (int k = 0; k < 64 * KB; ++k) ref += aval(t, k) * bval(c0 + u, k);
        emax = fmaxf(emax, fabsf(v[u] - ref));
        rmax = fmaxf(rmax, fabsf(ref));
      }
    }
  } else {
    emax = 1e30f;
  }
  atomicMax(reinterpret_cast<int*>(out), __float_as_int(emax));
  atomicMax(reinterpret_cast<int*>(out + 1), __float_as_int(rmax));
  tc::tc_fence_before();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tmem, 256);
}

// As k_mma_selftest with K = 64 and either operand stored MN-major (rows = K, 64-wide
// MN blocks 8 KB apart), read through the MN-major descriptor and the transpose bits.
template <int N, bool F16, bool AMN, bool BMN>
__global__ void __launch_bounds__(128) k_mma_selftest_mn(float* out, int* err) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  unsigned char* sm = sm_raw + ((1024u - (tc::smem_u32(sm_raw) & 1023u)) & 1023u);
  unsigned char* A = sm;              // 16 KB
  unsigned char* B = sm + 16384;      // up to 16 KB
  constexpr uint32_t kLbo = 8192;     // 64 K-rows x 128 B per 64-wide MN block
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int t = threadIdx.x, w = t >> 5;
  auto aval = [](int r, int k) { return (float)(((r * 7 + k * 3) % 17) - 8) * 0.125f; };
  auto bval = [](int n, int k) { return (float)(((n * 5 + k * 11) % 13) - 6) * 0.25f; };
  for (int k = 0; k < 64; ++k) {
    const float v = aval(t, k);
    const uint32_t bits = tc::pack2<F16>(v, 0.f) & 0xFFFFu;
    const uint32_t off = AMN ? tc::sw128_mn_off(t, k, kLbo) : tc::sw128_off(t, k & ~7) + (k & 7) * 2;
    *reinterpret_cast<unsigned short*>(A + off) = (unsigned short)bits;
  }
  for (int n = t; n < N; n += 128)
    for (int k = 0; k < 64; ++k) {
      const uint32_t bits = tc::pack2<F16>(bval(n, k), 0.f) & 0xFFFFu;
      const uint32_t off = BMN ? tc::sw128_mn_off(n, k, kLbo) : tc::sw128_off(n, k & ~7) + (k & 7) * 2;
      *reinterpret_cast<unsigned short*>(B + off) = (unsigned short)bits;
    }
  if (t == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
  }
  if (w == 0) {
    tc::tmem_alloc(&tslot, 128);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tslot;
  if (t == 0) {
    constexpr uint32_t idesc = tc::idesc_mn(tc::idesc_f16(128, N, F16), AMN, BMN);
    for (int k = 0; k < 4; ++k) {
      const uint32_t as = tc::smem_u32(A) + (AMN ? 2048u * k : 32u * k);
      const uint32_t bs = tc::smem_u32(B) + (BMN ? 2048u * k : 32u * k);
      const uint64_t ad = AMN ? tc::sdesc_sw128_mn(as, kLbo) : tc::sdesc_sw128(as);
      const uint64_t bd = BMN ? tc::sdesc_sw128_mn(bs, kLbo) : tc::sdesc_sw128(bs);
      tc::mma_f16(tmem, ad, bd, idesc, k > 0 ? 1u : 0u);
    }
    tc::mma_commit(&bar);
  }
  bool ok = tc::mbar_wait(&bar, 0, err);
  tc::tc_fence_after();
  float emax = 0.f, rmax = 0.f;
  if (ok) {
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * w) << 16) + c0, v);
      tc::tmem_wait_ld();
      for (int u = 0; u < 16; ++u) {
        float ref = 0.f;
        for (int k = 0; k < 64; ++k) ref += aval(t, k) * bval(c0 + u, k);
        emax = fmaxf(emax, fabsf(v[u] - ref));
        rmax = fmaxf(rmax, fabsf(ref));
      }
    }
  } else {
    emax = 1e30f;
  }
  atomicMax(reinterpret_cast<int*>(out), __float_as_int(emax));
  atomicMax(reinterpret_cast<int*>(out + 1), __float_as_int(rmax));
  tc::tc_fence_before();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tmem, 128);
}

template <int N, bool F16, bool AMN, bool BMN>
dp_status run_selftest_mn(float* dout, int* derr, float* host) {
  // operands need 32 KB; the window is sized so that any misread stride stays inside it
  const size_t smem = 64 * 1024 + 1024;
  const void* fn = reinterpret_cast<const void*>(k_mma_selftest_mn<N, F16, AMN, BMN>);
  if (ensure_smem(fn, smem) != cudaSuccess) return DP_ERR_CUDA;
  if (cudaMemset(dout, 0, 8) != cudaSuccess) return DP_ERR_CUDA;
  k_mma_selftest_mn<N, F16, AMN, BMN><<<1, 128, smem>>>(dout, derr);
  if (cudaDeviceSynchronize() != cudaSuccess) return DP_ERR_CUDA;
  if (cudaMemcpy(host, dout, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return DP_ERR_CUDA;
  return DP_OK;
}

template <int N, int KB, bool F16>
dp_status run_selftest(float* dout, int* derr, float* host) {
  size_t smem = (size_t)KB * 128 * 128 + (size_t)KB * N * 128 + 1024;
  if (ensure_smem(reinterpret_cast<const void*>(k_mma_selftest<N, KB, F16>), smem) != cudaSuccess)
    return DP_ERR_CUDA;
  if (cudaMemset(dout, 0, 8) != cudaSuccess) return DP_ERR_CUDA;
  k_mma_selftest<N, KB, F16><<<1, 128, smem>>>(dout, derr);
  if (cudaDeviceSynchronize() != cudaSuccess) return DP_ERR_CUDA;
  if (cudaMemcpy(host, dout, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return DP_ERR_CUDA;
  return DP_OK;
}

}  // namespace

dp_status launch_tc_setup(Model* m) { return mix_fit_setup(m); }

}  // namespace dpg

using namespace dpg;

// Built-in self checks of the tensor-core operand layouts (see include/dp.h).
extern "C" dp_status dp_selftest(int which, double* result) {
  if (!result) return DP_ERR_ARG;
  if (!tc_available(nullptr)) return DP_ERR_UNSUPPORTED;
  float* d = nullptr;
  int* e = nullptr;
  if (cudaMalloc(&d, 16) != cudaSuccess || cudaMalloc(&e, 16) != cudaSuccess) return DP_ERR_OOM;
  cudaMemset(e, 0, 16);
  float h[2] = {0, 0};
  dp_status st = DP_ERR_ARG;
  switch (which) {
    case 0: st = run_selftest<64, 1, false>(d, e, h); break;
    case 1: st = run_selftest<112, 1, false>(d, e, h); break;
    case 2: st = run_selftest<240, 4, false>(d, e, h); break;
    case 3: st = run_selftest<32, 1, true>(d, e, h); break;
    case 4: st = run_selftest<160, 4, true>(d, e, h); break;
    case 5: st = run_selftest_mn<64, false, false, true>(d, e, h); break;
    case 6: st = run_selftest_mn<64, true, true, false>(d, e, h); break;
    case 7: st = run_selftest_mn<128, true, true, true>(d, e, h); break;
    default: break;
  }
  int eh = 0;
  cudaMemcpy(&eh, e, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  cudaFree(e);
  if (st != DP_OK) return st;
  if (eh) return DP_ERR_WAIT_TIMEOUT;
  result[0] = h[0];
  result[1] = h[1];
  return DP_OK;
}

// ---------------------------------------------------------------------------
// Check of the bounded-wait error path: one thread initialises an mbarrier that
// expects one arrival and waits for its first phase with the kernels' bounded wait
// routine, which nothing will complete.  No copy or MMA is issued, so nothing is in
// flight when the wait gives up; the kernel sets the timeout bit and returns.

namespace dpg {
namespace {

static __device__ int g_wait_selftest_err;

__global__ void k_wait_selftest(uint32_t limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) tc::mbar_wait_limit(&bar, 0, &g_wait_selftest_err, limit);
  __syncthreads();
}

}  // namespace
}  // namespace dpg

extern "C" dp_status dp_wait_selftest(unsigned int spin_limit) {
  if (spin_limit < 1 || spin_limit > tc::kSpinLimit) return DP_ERR_ARG;
  if (!tc_available(nullptr)) return DP_ERR_UNSUPPORTED;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_wait_selftest_err, &zero, sizeof(int)) != cudaSuccess) return DP_ERR_CUDA;
  k_wait_selftest<<<1, 32>>>(spin_limit);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return DP_ERR_CUDA;
  int bits = 0;
  if (cudaMemcpyFromSymbol(&bits, g_wait_selftest_err, sizeof(int)) != cudaSuccess) return DP_ERR_CUDA;
  return (bits & ERR_TIMEOUT) ? DP_ERR_WAIT_TIMEOUT : DP_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the self check.
//
// dp_selftest above takes its 32 bytes of device scratch from cudaMalloc and
// hands them back with cudaFree on every call.  Some callers cannot do that: a
// serving process that has already given the whole device to its own memory
// pool gets an out-of-memory error exactly when it wants to re-check a device,
// and a health monitor running beside live work must not pay for cudaFree,
// which waits for the whole device.  This variant keeps its scratch in a fixed
// array compiled into the library, so a call allocates nothing.

#include <cstring>
#include <mutex>

namespace dpg {
namespace {

// Per case 16 bytes: two floats that the kernel raises with atomicMax (max
// |error|, max |value|; both must start at 0) and the wait-timeout word (must
// start at 0), padded to 16 bytes.  Every call zeroes the slots it uses.
constexpr int kNoAllocCases = DP_SELFTEST_NOALLOC_MAX_CASES;
static __device__ __align__(256) unsigned int g_selftest_scratch[kNoAllocCases * 4];

constexpr int kNoAllocDevices = 64;
std::mutex g_noalloc_mu;
unsigned int* g_noalloc_scratch[kNoAllocDevices] = {nullptr};

template <int N, int KB>
constexpr size_t selftest_smem() { return (size_t)KB * 128 * 128 + (size_t)KB * N * 128 + 1024; }

template <int N, int KB, bool F16>
cudaError_t noalloc_prepare() {
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(k_mma_selftest<N, KB, F16>),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)selftest_smem<N, KB>());
}

template <int N, int KB, bool F16>
cudaError_t noalloc_launch(unsigned int* slot) {
  k_mma_selftest<N, KB, F16><<<1, 128, selftest_smem<N, KB>()>>>(reinterpret_cast<float*>(slot),
                                                                 reinterpret_cast<int*>(slot + 2));
  return cudaGetLastError();
}

// Once per device: the device address of the scratch array (the module holding it
// is loaded on first use) and the shared-memory limits of the five kernels.
dp_status noalloc_setup(unsigned int** scratch) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DP_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocDevices) return DP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_scratch[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_selftest_scratch) != cudaSuccess || !p) return DP_ERR_CUDA;
    if (noalloc_prepare<64, 1, false>() != cudaSuccess || noalloc_prepare<112, 1, false>() != cudaSuccess ||
        noalloc_prepare<240, 4, false>() != cudaSuccess || noalloc_prepare<32, 1, true>() != cudaSuccess ||
        noalloc_prepare<160, 4, true>() != cudaSuccess)
      return DP_ERR_CUDA;
    g_noalloc_scratch[dev] = static_cast<unsigned int*>(p);
  }
  *scratch = g_noalloc_scratch[dev];
  return DP_OK;
}

}  // namespace
}  // namespace dpg

extern "C" dp_status dp_selftest_noalloc(const int* which, int ncases, double* results) {
  if (ncases < 0) return DP_ERR_ARG;
  if (ncases > kNoAllocCases) return DP_ERR_CAPACITY;
  if (ncases > 0 && (!which || !results)) return DP_ERR_ARG;
  for (int i = 0; i < ncases; ++i)
    if (which[i] < 0 || which[i] > 4) return DP_ERR_ARG;
  if (!tc_available(nullptr)) return DP_ERR_UNSUPPORTED;
  unsigned int* scratch = nullptr;
  dp_status st = noalloc_setup(&scratch);
  if (st != DP_OK || ncases == 0) return st;

  // legacy default stream: the zeroing, the launches and the read-back are ordered
  if (cudaMemsetAsync(scratch, 0, (size_t)ncases * 16, 0) != cudaSuccess) return DP_ERR_CUDA;
  for (int i = 0; i < ncases; ++i) {
    unsigned int* slot = scratch + 4 * i;
    cudaError_t e = cudaErrorInvalidValue;
    switch (which[i]) {
      case 0: e = noalloc_launch<64, 1, false>(slot); break;
      case 1: e = noalloc_launch<112, 1, false>(slot); break;
      case 2: e = noalloc_launch<240, 4, false>(slot); break;
      case 3: e = noalloc_launch<32, 1, true>(slot); break;
      case 4: e = noalloc_launch<160, 4, true>(slot); break;
      default: break;
    }
    if (e != cudaSuccess) return DP_ERR_CUDA;
  }
  unsigned int host[kNoAllocCases * 4];
  if (cudaMemcpy(host, scratch, (size_t)ncases * 16, cudaMemcpyDeviceToHost) != cudaSuccess) return DP_ERR_CUDA;
  st = DP_OK;
  for (int i = 0; i < ncases; ++i) {
    float v[2];
    memcpy(v, host + 4 * i, sizeof(v));
    results[2 * i] = v[0];
    results[2 * i + 1] = v[1];
    if (host[4 * i + 2] != 0) st = DP_ERR_WAIT_TIMEOUT;
  }
  return st;
}
