// Tabulated (compressed) embedding net, Section II-A's compressed model: every output of each
// embedding net becomes a piecewise quintic in the net's input on n uniform intervals of width h
// from x0, matching the net's value, first and second derivative at both ends of every interval
// (a C2 interpolant; its error falls as h^6).  The table replaces the net in the forward and in
// the force backward (dG/dx is the derivative of the quintic).
//
// Layout (FP64 and FP32 copies): tab[((pair * n + i) * 100 + q) * 8 + p], p = 0..5 the
// coefficient of u^p with u = (x - x_i) / h in [0, 1); entries 6, 7 are zero (32-byte rows for
// vector loads).  An input below x0 or above x0 + n h uses the edge interval's polynomial.
#include "common.cuh"

namespace dpg {
namespace {

// Node values of the net of pair blockIdx.y at x_i = x0 + i h (i = blockIdx.x): G, G', G'' of
// every output by forward-mode differentiation written out per layer (FP64):
//   a = x W1 + b1, h1 = tanh(a):   h1' = (1 - h1^2) W1,            h1'' = -2 h1 (1 - h1^2) W1^2
//   a = h W + b,   t = tanh(a):    t'  = (1 - t^2) a',             t''  = (1 - t^2) a'' - 2 t (1 - t^2) a'^2
// with the residuals h2 = [h1, h1] + t2, G = [h2, h2] + t3 carried with their derivatives.
__global__ void __launch_bounds__(128) k_tab_nodes(int n, double x0, double h, const double* __restrict__ w,
                                                   double* __restrict__ v) {
  const int pair = blockIdx.y, i = blockIdx.x, tid = threadIdx.x;
  const double* W = w + (size_t)pair * kEmbParams;
  __shared__ double s1[kN1][3], s2[kN2][3];
  const double x = x0 + i * h;
  if (tid < kN1) {
    const double w1 = W[kEW1 + tid];
    const double t = tanh(x * w1 + W[kEb1 + tid]), t1 = 1.0 - t * t;
    s1[tid][0] = t;
    s1[tid][1] = t1 * w1;
    s1[tid][2] = -2.0 * t * t1 * w1 * w1;
  }
  __syncthreads();
  if (tid < kN2) {
    double a0 = W[kEb2 + tid], a1 = 0.0, a2 = 0.0;
    for (int k = 0; k < kN1; ++k) {
      const double wk = W[kEW2 + k * kN2 + tid];
      a0 += s1[k][0] * wk;
      a1 += s1[k][1] * wk;
      a2 += s1[k][2] * wk;
    }
    const double t = tanh(a0), t1 = 1.0 - t * t;
    const int r = tid % kN1;
    s2[tid][0] = s1[r][0] + t;
    s2[tid][1] = s1[r][1] + t1 * a1;
    s2[tid][2] = s1[r][2] + t1 * a2 - 2.0 * t * t1 * a1 * a1;
  }
  __syncthreads();
  if (tid < kN3) {
    double a0 = W[kEb3 + tid], a1 = 0.0, a2 = 0.0;
    for (int k = 0; k < kN2; ++k) {
      const double wk = W[kEW3 + k * kN3 + tid];
      a0 += s2[k][0] * wk;
      a1 += s2[k][1] * wk;
      a2 += s2[k][2] * wk;
    }
    const double t = tanh(a0), t1 = 1.0 - t * t;
    const int r = tid % kN2;
    double* o = v + (((size_t)pair * (n + 1) + i) * kN3 + tid) * 3;
    o[0] = s2[r][0] + t;
    o[1] = s2[r][1] + t1 * a1;
    o[2] = s2[r][2] + t1 * a2 - 2.0 * t * t1 * a1 * a1;
  }
}

// Quintic of interval i of output q: with f, f', f'' at the left (l) and right (r) nodes,
//   c0 = f_l, c1 = h f'_l, c2 = h^2 f''_l / 2,
//   A = f_r - (c0 + c1 + c2), B = h f'_r - (c1 + 2 c2), C = h^2 f''_r - 2 c2,
//   c3 = 10 A - 4 B + C / 2, c4 = -15 A + 7 B - C, c5 = 6 A - 3 B + C / 2
// (the solution of P(1) = f_r, P'(1) = h f'_r, P''(1) = h^2 f''_r for the top three coefficients).
__global__ void k_tab_coef(int npairs, int n, double h, const double* __restrict__ v, double* __restrict__ tab64,
                           float* __restrict__ tab32) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)npairs * n * kN3;
  if (idx >= total) return;
  const int q = (int)(idx % kN3);
  const size_t pi = idx / kN3;  // pair * n + i
  const int i = (int)(pi % n), pair = (int)(pi / n);
  const double* l = v + (((size_t)pair * (n + 1) + i) * kN3 + q) * 3;
  const double* r = l + (size_t)kN3 * 3;
  const double c0 = l[0], c1 = h * l[1], c2 = 0.5 * h * h * l[2];
  const double A = r[0] - (c0 + c1 + c2), B = h * r[1] - (c1 + 2.0 * c2), C = h * h * r[2] - 2.0 * c2;
  const double c[8] = {c0, c1, c2, 10.0 * A - 4.0 * B + 0.5 * C, -15.0 * A + 7.0 * B - C, 6.0 * A - 3.0 * B + 0.5 * C,
                       0.0, 0.0};
  double* d = tab64 + idx * 8;
  float* f = tab32 + idx * 8;
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    d[p] = c[p];
    f[p] = (float)c[p];
  }
}

}  // namespace

dp_status launch_tabulate(Model* m, double x0, double x1, int n) {
  DP_CUDA_TRY(m, cudaStreamSynchronize(m->stream));
  if (m->tab_mem) {
    DP_CUDA_TRY(m, cudaFree(m->tab_mem));
    m->tab_mem = nullptr;
    m->tab64 = nullptr;
    m->tab32 = nullptr;
  }
  m->tab_n = 0;
  if (n == 0) return DP_OK;
  const int npairs = m->ntypes * m->ntypes;
  const size_t nodes = (size_t)npairs * (n + 1) * kN3 * 3;        // doubles
  const size_t coef = (size_t)npairs * n * kN3 * 8;               // entries
  const size_t bytes = nodes * 8 + coef * 8 + coef * 4;
  void* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, bytes);
  if (e != cudaSuccess) {
    m->last_error = std::string("table allocation: ") + cudaGetErrorString(e);
    return DP_ERR_OOM;
  }
  m->tab_mem = mem;
  double* v = static_cast<double*>(mem);
  m->tab64 = v + nodes;
  m->tab32 = reinterpret_cast<float*>(m->tab64 + coef);
  const double h = (x1 - x0) / n;
  k_tab_nodes<<<dim3(n + 1, npairs), 128, 0, m->stream>>>(n, x0, h, m->w64, v);
  const size_t total = (size_t)npairs * n * kN3;
  k_tab_coef<<<(unsigned)((total + 255) / 256), 256, 0, m->stream>>>(npairs, n, h, v, m->tab64, m->tab32);
  m->launches += 2;
  DP_LAUNCH_CHECK(m);
  DP_CUDA_TRY(m, cudaStreamSynchronize(m->stream));
  m->tab_n = n;
  m->tab_x0 = x0;
  m->tab_h = h;
  return DP_OK;
}

}  // namespace dpg
