// Output reductions and the velocity-Verlet step (Section II-A: the MD engine
// updates velocities and positions of the atoms after the force evaluation and
// reports energies and pressure-related quantities).  Positions, velocities,
// forces, energies and virials are FP64 in every precision.
#include "common.cuh"

namespace dpg {
namespace {

constexpr double kKappa = 9.648533e-3;  // A fs^-2 per (eV / A / amu)

__global__ void k_unpermute(int N, const int* __restrict__ perm, const double* __restrict__ e_atom,
                            const double* __restrict__ vir_atom, const double* __restrict__ force, double* e_user,
                            double* vir_user, double* forces_user) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  int u = perm[k];
  e_user[u] = e_atom[k];
#pragma unroll
  for (int q = 0; q < 9; ++q) vir_user[(size_t)u * 9 + q] = vir_atom[(size_t)k * 9 + q];
  if (forces_user) {
#pragma unroll
    for (int q = 0; q < 3; ++q) forces_user[(size_t)u * 3 + q] = force[(size_t)k * 3 + q];
  }
}

// Per-replica energy and virial: sums of the per-atom values (caller order), or for the
// virial the per-replica accumulator vir_rep when the backward produced one.  Deterministic:
// block (c, r) sums chunk c (kRedChunk atoms) of replica r over a fixed strided partition (four
// independent loads per pass) and a fixed tree; with one chunk per replica it writes the result,
// otherwise its partial, which k_rep_final adds in chunk order.
constexpr int kRedThreads = 256;
constexpr int kRedChunk = 8192;
__global__ void __launch_bounds__(kRedThreads) k_rep_reduce(int nrep, int nchunk, const int* __restrict__ rep_off,
                                                           const double* __restrict__ e_user,
                                                           const double* __restrict__ vir_user,
                                                           const double* __restrict__ vir_rep, double* energy,
                                                           double* virial, double* part_out,
                                                           const int* __restrict__ err) {
  __shared__ double part[10][kRedThreads];
  const int r = blockIdx.y, c = blockIdx.x;
  if (r >= nrep) return;
  const int rb = rep_off[r], re = rep_off[r + 1];
  const int beg = min(re, rb + c * kRedChunk), end = min(re, beg + kRedChunk);
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int u0 = beg + threadIdx.x; u0 < end; u0 += 4 * kRedThreads) {
    double e[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int u = u0 + k * kRedThreads;
      e[k] = u < end ? e_user[u] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[0] += e[k];
    if (vir_user) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int u = u0 + k * kRedThreads;
        if (u < end)
          for (int q = 0; q < 9; ++q) acc[1 + q] += vir_user[(size_t)u * 9 + q];
      }
    }
  }
  for (int q = 0; q < 10; ++q) part[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int st = kRedThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int q = 0; q < 10; ++q) part[q][threadIdx.x] += part[q][threadIdx.x + st];
    __syncthreads();
  }
  if (nchunk > 1) {
    if (threadIdx.x < 10) part_out[((size_t)r * nchunk + c) * 10 + threadIdx.x] = part[threadIdx.x][0];
    return;
  }
  if (threadIdx.x == 0) {
    bool bad = err && *err != 0;
    if (energy) energy[r] = bad ? __longlong_as_double(0x7ff8000000000000ll) : part[0][0];
    if (virial)
      for (int q = 0; q < 9; ++q) virial[r * 9 + q] = vir_rep ? vir_rep[r * 9 + q] : part[1 + q][0];
  }
}

// The chunk partials of each replica added in chunk order (lane q: quantity q).
__global__ void k_rep_final(int nrep, int nchunk, const double* __restrict__ part, const double* __restrict__ vir_rep,
                            double* energy, double* virial, const int* __restrict__ err) {
  const int r = blockIdx.x, q = threadIdx.x;
  if (r >= nrep || q >= 10) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[((size_t)r * nchunk + c) * 10 + q];
  if (q == 0) {
    bool bad = err && *err != 0;
    if (energy) energy[r] = bad ? __longlong_as_double(0x7ff8000000000000ll) : s;
  } else if (virial) {
    virial[r * 9 + q - 1] = vir_rep ? vir_rep[r * 9 + q - 1] : s;
  }
}

__global__ void k_kick_drift(int N, dvec4* x, dvec4* v, const double* __restrict__ F,
                             const double* __restrict__ mass, double dt) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double a = 0.5 * dt * kKappa / mass[k];
  dvec4 vv = v[k], xx = x[k];
  vv.x += a * F[3 * k]; vv.y += a * F[3 * k + 1]; vv.z += a * F[3 * k + 2];
  xx.x += dt * vv.x; xx.y += dt * vv.y; xx.z += dt * vv.z;
  v[k] = vv;
  x[k] = xx;
}

__global__ void k_kick(int N, dvec4* v, const double* __restrict__ F, const double* __restrict__ mass, double dt) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double a = 0.5 * dt * kKappa / mass[k];
  dvec4 vv = v[k];
  vv.x += a * F[3 * k]; vv.y += a * F[3 * k + 1]; vv.z += a * F[3 * k + 2];
  v[k] = vv;
}

__global__ void k_load_state(int N, const int* __restrict__ perm, const int* __restrict__ itype,
                             const double* __restrict__ v_user, const double* __restrict__ mass_by_type,
                             dvec4* v, double* mass) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  int u = perm[k];
  v[k] = make_dvec4(v_user[3 * u], v_user[3 * u + 1], v_user[3 * u + 2], 0.0);
  mass[k] = mass_by_type[itype[k]];
}

__global__ void k_store_state(int N, const int* __restrict__ perm, const dvec4* __restrict__ x,
                              const dvec4* __restrict__ v, double* x_user, double* v_user) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  int u = perm[k];
  dvec4 p = x[k], q = v[k];
  x_user[3 * u] = p.x; x_user[3 * u + 1] = p.y; x_user[3 * u + 2] = p.z;
  v_user[3 * u] = q.x; v_user[3 * u + 1] = q.y; v_user[3 * u + 2] = q.z;
}

__global__ void k_kinetic_atoms(int N, const int* __restrict__ perm, const dvec4* __restrict__ v,
                                const double* __restrict__ mass, double* ke_user) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  dvec4 q = v[k];
  ke_user[perm[k]] = 0.5 * mass[k] * (q.x * q.x + q.y * q.y + q.z * q.z) / kKappa;
}

__global__ void k_nan(double* p, int n) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) p[k] = __longlong_as_double(0x7ff8000000000000ll);
}

}  // namespace

// Chunk slots of the reduction workspace: every replica may need ceil(max_atoms / kRedChunk).
size_t rep_reduce_slots(int max_atoms, int max_reps) {
  return (size_t)max_reps * ((size_t)max_atoms / kRedChunk + 1);
}

namespace {

// Per-replica sums of per-atom values (energy, and the per-atom virial unless vir_rep holds it).
dp_status launch_rep_reduce(Model* m, const double* e_user, const double* vir_user, const double* vir_rep,
                            double* energy, double* virial, const int* err) {
  const int nchunk = std::max(1, (m->max_rep_atoms + kRedChunk - 1) / kRedChunk);
  if (nchunk > 1 && (size_t)m->nrep * nchunk > m->red_cap) {
    m->last_error = "reduction workspace too small";
    return DP_ERR_CAPACITY;
  }
  k_rep_reduce<<<dim3(nchunk, m->nrep), kRedThreads, 0, m->stream>>>(m->nrep, nchunk, m->rep_off_dev, e_user, vir_user,
                                                                     vir_rep, energy, virial, m->red_part, err);
  m->launches += 1;
  if (nchunk > 1) {
    k_rep_final<<<m->nrep, 32, 0, m->stream>>>(m->nrep, nchunk, m->red_part, vir_rep, energy, virial, err);
    m->launches += 1;
  }
  return DP_OK;
}

}  // namespace

dp_status launch_outputs(Model* m, int N, double* energy_rep, double* atom_energy, double* forces,
                         double* virial_rep) {
  k_unpermute<<<cdiv(N, 256), 256, 0, m->stream>>>(N, m->perm, m->e_atom, m->vir_atom, m->force, m->e_user,
                                                   m->vir_user, forces);
  const bool mixed = is_mixed(m);
  const dp_status rs = launch_rep_reduce(m, m->e_user, mixed ? nullptr : m->vir_user, mixed ? m->vir_rep : nullptr,
                                         energy_rep, virial_rep, m->err);
  if (rs != DP_OK) return rs;
  m->launches += 1;
  if (atom_energy)
    DP_CUDA_TRY(m, cudaMemcpyAsync(atom_energy, m->e_user, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                                   m->stream));
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_zero_forces(Model* m, int N) {
  DP_CUDA_TRY(m, cudaMemsetAsync(m->force, 0, sizeof(double) * 3 * N, m->stream));
  return DP_OK;
}

dp_status launch_kick_drift(Model* m, int N, double dt) {
  k_kick_drift<<<cdiv(N, 256), 256, 0, m->stream>>>(N, m->x, m->v, m->force, m->mass, dt);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_kick(Model* m, int N, double dt) {
  k_kick<<<cdiv(N, 256), 256, 0, m->stream>>>(N, m->v, m->force, m->mass, dt);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_load_state(Model* m, int N, const double* v_user, const double* mass_by_type_dev) {
  k_load_state<<<cdiv(N, 256), 256, 0, m->stream>>>(N, m->perm, m->itype, v_user, mass_by_type_dev, m->v,
                                                    m->mass);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_store_state(Model* m, int N, double* x_user, double* v_user) {
  k_store_state<<<cdiv(N, 256), 256, 0, m->stream>>>(N, m->perm, m->x, m->v, x_user, v_user);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_kinetic(Model* m, int N, double* ke_rep) {
  k_kinetic_atoms<<<cdiv(N, 256), 256, 0, m->stream>>>(N, m->perm, m->v, m->mass, m->ke_user);
  const dp_status rs = launch_rep_reduce(m, m->ke_user, nullptr, nullptr, ke_rep, nullptr, nullptr);
  if (rs != DP_OK) return rs;
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_nan_energy(Model* m, double* energy, int n) {
  k_nan<<<cdiv(n, 256), 256, 0, m->stream>>>(energy, n);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

}  // namespace dpg
