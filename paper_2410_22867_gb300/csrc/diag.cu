// Diagnostics of a computed state: the pair-distance histogram behind the radial distribution
// function (the structural check of Section IV-A, Fig. 6) and the per-atom virial.
#include "common.cuh"

namespace dpg {
namespace {

template <class V> struct PairT;
template <> struct PairT<float4> { using type = float; };
template <> struct PairT<dvec4> { using type = double; };

// One thread per neighbour slot of the formatted list (pairs within r_c of the last
// evaluation): the slot's pair (centre type ti, neighbour type tj) at distance r < r_max adds one
// to bin floor(r / dr) of histogram ti * nt + tj.  A block histogram in shared memory (32-bit),
// added to the global 64-bit one.  r^2 is summed as ((dx dx) + (dy dy)) + dz dz without FMA.
template <class V>
__global__ void k_rdf(int N, int nt, int S, int4 sel_off, const int* __restrict__ itype,
                      const int* __restrict__ nl_count, const V* __restrict__ nl_d, int nbins, double dr_inv,
                      double rmax2, unsigned long long* __restrict__ hist) {
  using T = typename PairT<V>::type;
  extern __shared__ unsigned int sh[];
  const int nh = nt * nt * nbins;
  for (int q = threadIdx.x; q < nh; q += blockDim.x) sh[q] = 0u;
  __syncthreads();
  const int so[4] = {sel_off.x, sel_off.y, sel_off.z, sel_off.w};
  const size_t total = (size_t)N * S;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / S), k = (int)(e % S);
    int tj = 0;
    while (tj + 1 < nt && k >= so[tj + 1]) ++tj;
    if (k - so[tj] >= nl_count[(size_t)i * nt + tj]) continue;
    const V d = nl_d[e];
    double r2;
    if constexpr (sizeof(T) == 8)
      r2 = __dadd_rn(__dadd_rn(__dmul_rn(d.x, d.x), __dmul_rn(d.y, d.y)), __dmul_rn(d.z, d.z));
    else
      r2 = (double)__fadd_rn(__fadd_rn(__fmul_rn(d.x, d.x), __fmul_rn(d.y, d.y)), __fmul_rn(d.z, d.z));
    if (!(r2 < rmax2)) continue;
    int b = (int)floor(sqrt(r2) * dr_inv);
    b = min(b, nbins - 1);
    atomicAdd(&sh[(itype[i] * nt + tj) * nbins + b], 1u);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nh; q += blockDim.x)
    if (sh[q]) atomicAdd(&hist[q], (unsigned long long)sh[q]);
}

__global__ void k_vir_user(int N, const int* __restrict__ perm, const double* __restrict__ vir_atom, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int u = perm[k];
#pragma unroll
  for (int q = 0; q < 9; ++q) out[(size_t)u * 9 + q] = vir_atom[(size_t)k * 9 + q];
}

}  // namespace

dp_status launch_rdf(Model* m, int nbins, double r_max, unsigned long long* hist_dev) {
  const int N = m->natoms, nt = m->ntypes;
  int4 so = make_int4(m->sel_off[0], m->sel_off[1], m->sel_off[2], m->sel_off[3]);
  const size_t smem = sizeof(unsigned int) * (size_t)nt * nt * nbins;
  DP_CUDA_TRY(m, cudaMemsetAsync(hist_dev, 0, sizeof(unsigned long long) * (size_t)nt * nt * nbins, m->stream));
  const double dr_inv = nbins / r_max;
  const int grid = 2 * num_sms();
  if (m->prec == DP_FP64) {
    DP_CUDA_TRY(m, ensure_smem(reinterpret_cast<const void*>(k_rdf<dvec4>), smem));
    k_rdf<dvec4><<<grid, 256, smem, m->stream>>>(N, nt, m->S, so, m->itype, m->nl_count,
                                                  static_cast<const dvec4*>(m->nl_d), nbins, dr_inv, r_max * r_max,
                                                  hist_dev);
  } else {
    DP_CUDA_TRY(m, ensure_smem(reinterpret_cast<const void*>(k_rdf<float4>), smem));
    k_rdf<float4><<<grid, 256, smem, m->stream>>>(N, nt, m->S, so, m->itype, m->nl_count,
                                                   static_cast<const float4*>(m->nl_d), nbins, dr_inv,
                                                   r_max * r_max, hist_dev);
  }
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_atom_virial_out(Model* m, int N, double* out) {
  k_vir_user<<<cdiv(N, 256), 256, 0, m->stream>>>(N, m->perm, m->vir_atom, out);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

}  // namespace dpg
