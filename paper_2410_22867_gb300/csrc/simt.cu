// SIMT (CUDA-core) kernels of the FP64 and FP32 paths: environment matrix,
// embedding net, descriptor, fitting net forward/backward, and the embedding
// backward that produces forces and virials.
//
// Model (Section II-A, Fig. 1(b)): for each neighbour j of atom i,
//   s = sw(r)/r, R_hat = ((s, s dx/r, s dy/r, s dz/r) - davg[ti]) / dstd[ti],
//   G_j = embedding_{ti,tj}(R_hat_0)   (1 -> 25 -> 50 -> 100, tanh, residual),
//   T = (1/S) sum_j R_hat_j^T G_j (4 x 100), D = T^T T[:, :16] (100 x 16),
//   E_i = fitting_{ti}(D) (1600 -> 240 -> 240 -> 240 -> 1) + e_bias[ti],
// and F = -dE/dx by backward propagation through every step.  Activations of
// the embedding net are recomputed in the backward instead of being stored.
// The fitting backward multiplies by pre-transposed weights (the GEMM-NT to
// GEMM-NN conversion of Section III-B2).
#include "common.cuh"

namespace dpg {
namespace {

template <class T> __device__ __forceinline__ T dtanh(T x);
template <> __device__ __forceinline__ float dtanh<float>(float x) { return tanhf(x); }
template <> __device__ __forceinline__ double dtanh<double>(double x) { return tanh(x); }

template <class T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = dvec4; };

// Switch function and its derivative (quintic C2 or cosine), s = sw/r.
template <class T>
__device__ __forceinline__ void switch_fn(T r, T rs, T rc, int kind, T& sw, T& dsw) {
  if (r < rs) { sw = T(1); dsw = T(0); return; }
  if (r >= rc) { sw = T(0); dsw = T(0); return; }
  T w = rc - rs;
  T u = (r - rs) / w;
  if (kind == 1) {
    const T pi = T(3.14159265358979323846);
    sw = T(0.5) * cos(pi * u) + T(0.5);
    dsw = T(-0.5) * pi * sin(pi * u) / w;
  } else {
    T u2 = u * u;
    sw = u2 * u * (T(-6) * u2 + T(15) * u - T(10)) + T(1);
    dsw = T(-30) * u2 * (u - T(1)) * (u - T(1)) / w;
  }
}

template <class T>
struct EmbArgs {
  int N, ntypes, S;
  int sel_off[kMaxTypes + 1];
  T rc, rs, invS;
  int switch_kind;
  const T* w;          // theta
  const T* stat;       // davg [nt][4] then 1/dstd [nt][4]
  const T* pad;        // [nt][nt][4][100] padded-slot term, or null (every davg is 0)
  int sel[kMaxTypes];
  const T* tab;        // tabulated embedding: [pair][interval][100][8] quintic coefficients (TAB kernels)
  int tab_n;
  T tab_x0, tab_ih;    // first node, 1 / interval width
  const int* itype;
  const int* nl_j;
  const void* nl_d;
  const int* nl_count;
  T* Tm;               // [N][4][100]
  T* Dm;               // [N][1600]
  const T* dD;         // [N][1600]
  double* force;       // [N][3]
  double* vir_atom;    // [N][9]
};

// Threads per block of the embedding kernels (= neighbour rows per chunk).
template <class T> struct EB { static constexpr int v = (sizeof(T) == 8) ? 64 : 128; };
constexpr int kGP = kN3 + 1;  // padded G row
constexpr int kH = kN2;       // rows of the per-thread residual staging column

template <class T>
__device__ __forceinline__ void load_pair_vec(const void* nl_d, size_t idx, T* d);
template <>
__device__ __forceinline__ void load_pair_vec<float>(const void* nl_d, size_t idx, float* d) {
  float4 v = static_cast<const float4*>(nl_d)[idx];
  d[0] = v.x; d[1] = v.y; d[2] = v.z;
}
template <>
__device__ __forceinline__ void load_pair_vec<double>(const void* nl_d, size_t idx, double* d) {
  dvec4 v = static_cast<const dvec4*>(nl_d)[idx];
  d[0] = v.x; d[1] = v.y; d[2] = v.z;
}

// Tabulated embedding: the coefficient rows of the interval holding x (edge intervals beyond
// the ends) and the offset u = (x - x_i) / h in it.
template <class T>
__device__ __forceinline__ const T* tab_rows(const EmbArgs<T>& a, int pair, T x, T& u) {
  const T f = (x - a.tab_x0) * a.tab_ih;
  int i = (int)floor(f);
  i = min(max(i, 0), a.tab_n - 1);
  u = f - T(i);
  return a.tab + ((size_t)pair * a.tab_n + i) * kN3 * 8;
}
// G = P(u) and dG/du = P'(u) of one output from its six coefficients.
template <class T>
__device__ __forceinline__ void tab_poly(const T* c, T u, T& g, T& gu) {
  g = c[0] + u * (c[1] + u * (c[2] + u * (c[3] + u * (c[4] + u * c[5]))));
  gu = c[1] + u * (T(2) * c[2] + u * (T(3) * c[3] + u * (T(4) * c[4] + u * T(5) * c[5])));
}

// Layers 1 and 2 of the embedding net for input x: h1 [25], h2 [50] = [h1, h1] + tanh(h1 W2 + b2).
template <class T>
__device__ __forceinline__ void emb12(const T* __restrict__ W, T x, T* h1, T* h2) {
#pragma unroll
  for (int k = 0; k < kN1; ++k) h1[k] = dtanh<T>(x * W[kEW1 + k] + W[kEb1 + k]);
#pragma unroll
  for (int m = 0; m < kN2; m += 2) {
    T z0 = W[kEb2 + m], z1 = W[kEb2 + m + 1];
#pragma unroll
    for (int k = 0; k < kN1; ++k) {
      z0 += h1[k] * W[kEW2 + k * kN2 + m];
      z1 += h1[k] * W[kEW2 + k * kN2 + m + 1];
    }
    h2[m] = h1[m % kN1] + dtanh<T>(z0);
    h2[m + 1] = h1[(m + 1) % kN1] + dtanh<T>(z1);
  }
}

// Load the embedding weights of every (ti, tj) pair for centre type ti into smem.
template <class T>
__device__ void load_emb_weights(T* sW, const T* __restrict__ w, int ti, int ntypes) {
  const T* src = w + (size_t)ti * ntypes * kEmbParams;
  for (int q = threadIdx.x; q < ntypes * kEmbParams; q += blockDim.x) sW[q] = src[q];
}

template <class T>
__device__ __forceinline__ void env_row(const T* d, T rs, T rc, int kind, const T* avg, const T* isd, T* R, T& r,
                                        T& sw, T& dsw) {
  r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  switch_fn<T>(r, rs, rc, kind, sw, dsw);
  T s = sw / r;
  R[0] = s; R[1] = s * d[0] / r; R[2] = s * d[1] / r; R[3] = s * d[2] / r;
#pragma unroll
  for (int c = 0; c < 4; ++c) R[c] = (R[c] - avg[c]) * isd[c];
}

// Forward: per atom, R_hat rows and G rows of a chunk of neighbours are staged in
// shared memory; T = (1/S) R_hat^T G is accumulated by the first 100 threads
// (one output column each); D = T^T T[:, :16] follows.
template <class T, bool TAB>
__global__ void __launch_bounds__(EB<T>::v) k_embed_fwd(EmbArgs<T> a) {
  constexpr int NB = EB<T>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sW = reinterpret_cast<T*>(smem_raw);                 // [ntypes][kEmbParams]
  T* sG = sW + a.ntypes * kEmbParams;                     // [NB][kGP]
  T* sR = sG + NB * kGP;                                  // [NB][4]
  T* sT = sR + NB * 4;                                    // [4][kN3]
  const int tid = threadIdx.x;
  const int per = cdiv_dev(a.N, gridDim.x);
  const int i0 = blockIdx.x * per, i1 = min(a.N, i0 + per);
  int cur_ti = -1;
  for (int i = i0; i < i1; ++i) {
    const int ti = a.itype[i];
    if (ti != cur_ti) {
      __syncthreads();
      load_emb_weights(sW, a.w, ti, a.ntypes);
      cur_ti = ti;
      __syncthreads();
    }
    T avg[4], isd[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) { avg[c] = a.stat[ti * 4 + c]; isd[c] = a.stat[(a.ntypes + ti) * 4 + c]; }
    constexpr int NCOL = (kN3 + NB - 1) / NB;  // T columns owned by each thread
    T acc[NCOL][4];
#pragma unroll
    for (int u = 0; u < NCOL; ++u)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[u][c] = T(0);
    for (int tj = 0; tj < a.ntypes; ++tj) {
      const int cnt = a.nl_count[(size_t)i * a.ntypes + tj];
      const T* W = sW + tj * kEmbParams;
      for (int base = 0; base < cnt; base += NB) {
        const int rows = min(NB, cnt - base);
        if (tid < rows) {
          T d[3], R[4], r, sw, dsw;
          load_pair_vec<T>(a.nl_d, (size_t)i * a.S + a.sel_off[tj] + base + tid, d);
          env_row<T>(d, a.rs, a.rc, a.switch_kind, avg, isd, R, r, sw, dsw);
#pragma unroll
          for (int c = 0; c < 4; ++c) sR[tid * 4 + c] = R[c];
          T* g = sG + tid * kGP;
          if (TAB) {
            T u, gu;
            const T* rows = tab_rows<T>(a, ti * a.ntypes + tj, R[0], u);
            for (int q = 0; q < kN3; ++q) tab_poly<T>(rows + 8 * q, u, g[q], gu);
          } else {
          T h1[kN1], h2[kN2];
          emb12<T>(W, R[0], h1, h2);
#pragma unroll
          for (int m = 0; m < kN2; ++m) g[m] = h2[m];  // staged residual, overwritten by G below
          for (int q = 0; q < kN2; ++q) {
            T za = W[kEb3 + q], zb = W[kEb3 + q + kN2];
#pragma unroll
            for (int mm = 0; mm < kN2; ++mm) {
              za += h2[mm] * W[kEW3 + mm * kN3 + q];
              zb += h2[mm] * W[kEW3 + mm * kN3 + q + kN2];
            }
            T res = g[q];
            g[q] = res + dtanh<T>(za);
            g[q + kN2] = res + dtanh<T>(zb);
          }
          }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NCOL; ++u) {
          const int col = tid + u * NB;
          if (col < kN3) {
            for (int rr = 0; rr < rows; ++rr) {
              T gv = sG[rr * kGP + col];
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[u][c] += sR[rr * 4 + c] * gv;
            }
          }
        }
        __syncthreads();
      }
    }
    if (a.pad) {  // padded slots: (sel - count) copies of the normalised zero row
      for (int tj = 0; tj < a.ntypes; ++tj) {
        const T np = T(a.sel[tj] - a.nl_count[(size_t)i * a.ntypes + tj]);
        const T* P = a.pad + (size_t)(ti * a.ntypes + tj) * 4 * kN3;
#pragma unroll
        for (int u = 0; u < NCOL; ++u) {
          const int col = tid + u * NB;
          if (col < kN3)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[u][c] += np * P[c * kN3 + col];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < NCOL; ++u) {
      const int col = tid + u * NB;
      if (col < kN3) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          T v = acc[u][c] * a.invS;
          sT[c * kN3 + col] = v;
          a.Tm[(size_t)i * 4 * kN3 + c * kN3 + col] = v;
        }
      }
    }
    __syncthreads();
    for (int q = tid; q < kN3; q += NB) {
      T out[kM2];
#pragma unroll
      for (int b = 0; b < kM2; ++b) {
        T v = T(0);
#pragma unroll
        for (int c = 0; c < 4; ++c) v += sT[c * kN3 + q] * sT[c * kN3 + b];
        out[b] = v;
      }
#pragma unroll
      for (int b = 0; b < kM2; ++b) a.Dm[(size_t)i * kKD + q * kM2 + b] = out[b];
    }
    __syncthreads();
  }
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Backward: dT from dE/dD and T; per neighbour the embedding is recomputed, then
// dR_hat = dT G, dG = R_hat dT, reverse through the embedding to d s_hat, the
// analytic Jacobian of the environment row gives g = dE/dd; F_i += g, F_j -= g
// (FP64 atomics), per-atom virial -sum g (x) d.
template <class T, bool TAB>
__global__ void __launch_bounds__(EB<T>::v) k_embed_bwd(EmbArgs<T> a) {
  constexpr int NB = EB<T>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sW = reinterpret_cast<T*>(smem_raw);                 // [ntypes][kEmbParams]
  T* sT = sW + a.ntypes * kEmbParams;                     // [4][kN3]
  T* sdT = sT + 4 * kN3;                                  // [4][kN3] (includes 1/S)
  T* sdD = sdT + 4 * kN3;                                 // [kKD]
  T* sH = sdD + kKD;                                      // [kH][NB] residual staging
  __shared__ double red[NB / 32][12];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int per = cdiv_dev(a.N, gridDim.x);
  const int i0 = blockIdx.x * per, i1 = min(a.N, i0 + per);
  int cur_ti = -1;
  for (int i = i0; i < i1; ++i) {
    const int ti = a.itype[i];
    __syncthreads();
    if (ti != cur_ti) {
      load_emb_weights(sW, a.w, ti, a.ntypes);
      cur_ti = ti;
    }
    for (int q = tid; q < 4 * kN3; q += NB) sT[q] = a.Tm[(size_t)i * 4 * kN3 + q];
    for (int q = tid; q < kKD; q += NB) sdD[q] = a.dD[(size_t)i * kKD + q];
    __syncthreads();
    // dT[c][a] = sum_b dD[a][b] T[c][b] + [a < 16] sum_a' dD[a'][a] T[c][a']
    for (int q = tid; q < kN3; q += NB) {
      for (int c = 0; c < 4; ++c) {
        T v = T(0);
#pragma unroll
        for (int b = 0; b < kM2; ++b) v += sdD[q * kM2 + b] * sT[c * kN3 + b];
        if (q < kM2)
          for (int a2 = 0; a2 < kN3; ++a2) v += sdD[a2 * kM2 + q] * sT[c * kN3 + a2];
        sdT[c * kN3 + q] = v * a.invS;
      }
    }
    __syncthreads();
    T avg[4], isd[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) { avg[c] = a.stat[ti * 4 + c]; isd[c] = a.stat[(a.ntypes + ti) * 4 + c]; }
    double fi[3] = {0, 0, 0}, vi[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int tj = 0; tj < a.ntypes; ++tj) {
      const int cnt = a.nl_count[(size_t)i * a.ntypes + tj];
      const T* W = sW + tj * kEmbParams;
      for (int base = 0; base < cnt; base += NB) {
        if (tid < cnt - base) {
          const size_t e = (size_t)i * a.S + a.sel_off[tj] + base + tid;
          const int j = a.nl_j[e];
          T d[3], R[4], r, sw, dsw;
          load_pair_vec<T>(a.nl_d, e, d);
          env_row<T>(d, a.rs, a.rc, a.switch_kind, avg, isd, R, r, sw, dsw);
          T dR[4] = {T(0), T(0), T(0), T(0)};
          if (TAB) {
            // G and dG/dx from the table: dR_hat = dT G, dG = R_hat . dT, d s_hat = sum dG dG/dx
            T u, g, gu, ds = T(0);
            const T* rows = tab_rows<T>(a, ti * a.ntypes + tj, R[0], u);
            for (int q = 0; q < kN3; ++q) {
              tab_poly<T>(rows + 8 * q, u, g, gu);
              T dg = T(0);
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const T dt = sdT[c * kN3 + q];
                dR[c] += dt * g;
                dg += R[c] * dt;
              }
              ds += dg * gu;
            }
            dR[0] += ds * a.tab_ih;
          } else {
          T h1[kN1], h2[kN2], dh2[kN2];
          emb12<T>(W, R[0], h1, h2);
#pragma unroll
          for (int m = 0; m < kN2; ++m) { sH[m * NB + tid] = h2[m]; dh2[m] = T(0); }
          for (int q = 0; q < kN2; ++q) {
            T za = W[kEb3 + q], zb = W[kEb3 + q + kN2];
#pragma unroll
            for (int mm = 0; mm < kN2; ++mm) {
              za += h2[mm] * W[kEW3 + mm * kN3 + q];
              zb += h2[mm] * W[kEW3 + mm * kN3 + q + kN2];
            }
            const T ta = dtanh<T>(za), tb = dtanh<T>(zb);
            const T res = sH[q * NB + tid];
            const T ga = res + ta, gb = res + tb;
            T dga = T(0), dgb = T(0);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const T da = sdT[c * kN3 + q], db = sdT[c * kN3 + q + kN2];
              dR[c] += da * ga + db * gb;
              dga += R[c] * da;
              dgb += R[c] * db;
            }
            const T dza = dga * (T(1) - ta * ta), dzb = dgb * (T(1) - tb * tb);
#pragma unroll
            for (int mm = 0; mm < kN2; ++mm)
              dh2[mm] += dza * W[kEW3 + mm * kN3 + q] + dzb * W[kEW3 + mm * kN3 + q + kN2];
            sH[q * NB + tid] = dga + dgb;  // residual gradient into dh2[q]
          }
          T dh1[kN1];
#pragma unroll
          for (int k = 0; k < kN1; ++k) dh1[k] = T(0);
#pragma unroll
          for (int mm = 0; mm < kN2; ++mm) {
            const T g2 = dh2[mm] + sH[mm * NB + tid];
            const T t2 = h2[mm] - h1[mm % kN1];
            const T dz = g2 * (T(1) - t2 * t2);
            dh1[mm % kN1] += g2;
#pragma unroll
            for (int k = 0; k < kN1; ++k) dh1[k] += dz * W[kEW2 + k * kN2 + mm];
          }
          T ds_in = T(0);
#pragma unroll
          for (int k = 0; k < kN1; ++k) ds_in += dh1[k] * (T(1) - h1[k] * h1[k]) * W[kEW1 + k];
          dR[0] += ds_in;
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) dR[c] *= isd[c];
          // Jacobian of (s, s d/r) with respect to d
          const T rinv = T(1) / r;
          const T ds = dsw * rinv - sw * rinv * rinv;
          const T qv = sw * rinv * rinv;
          const T dq = dsw * rinv * rinv - T(2) * sw * rinv * rinv * rinv;
          const T proj = dR[1] * d[0] + dR[2] * d[1] + dR[3] * d[2];
          const T common = (dR[0] * ds + dq * proj) * rinv;
          double g3[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) g3[c] = (double)(common * d[c] + qv * dR[1 + c]);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            fi[c] += g3[c];
            atomicAdd(&a.force[3 * (size_t)j + c], -g3[c]);
          }
#pragma unroll
          for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) vi[p * 3 + q] -= g3[p] * (double)d[q];
        }
      }
    }
    // block reduction of the centre force and the per-atom virial
    double vals[12] = {fi[0], fi[1], fi[2], vi[0], vi[1], vi[2], vi[3], vi[4], vi[5], vi[6], vi[7], vi[8]};
#pragma unroll
    for (int q = 0; q < 12; ++q) vals[q] = warp_sum<double>(vals[q]);
    if (lane == 0)
      for (int q = 0; q < 12; ++q) red[wid][q] = vals[q];
    __syncthreads();
    if (tid < 12) {
      double v = 0;
      for (int w = 0; w < NB / 32; ++w) v += red[w][tid];
      if (tid < 3) atomicAdd(&a.force[3 * (size_t)i + tid], v);
      else a.vir_atom[(size_t)i * 9 + tid - 3] = v;
    }
  }
}

// One padded neighbour slot per (ti, tj), block ti * nt + tj: the normalised zero row
// R_pad = (0 - davg[ti]) / dstd[ti], its embedding G = N_{ti,tj}(R_pad_0), and the product
// R_pad[c] G[a] that every padded slot of segment tj adds to S*T.  FP64, stored in FP64 and FP32.
__global__ void __launch_bounds__(128) k_pad_rows(int nt, const double* __restrict__ w,
                                                  const double* __restrict__ stat, double* pad64, float* pad32) {
  const int ti = blockIdx.x / nt, tj = blockIdx.x % nt, tid = threadIdx.x;
  const double* W = w + (size_t)(ti * nt + tj) * kEmbParams;
  __shared__ double Rp[4], h1[kN1], h2[kN2];
  if (tid < 4) Rp[tid] = (0.0 - stat[ti * 4 + tid]) * stat[(nt + ti) * 4 + tid];
  __syncthreads();
  const double x = Rp[0];
  if (tid < kN1) h1[tid] = tanh(x * W[kEW1 + tid] + W[kEb1 + tid]);
  __syncthreads();
  if (tid < kN2) {
    double z = W[kEb2 + tid];
    for (int k = 0; k < kN1; ++k) z += h1[k] * W[kEW2 + k * kN2 + tid];
    h2[tid] = h1[tid % kN1] + tanh(z);
  }
  __syncthreads();
  if (tid < kN3) {
    double z = W[kEb3 + tid];
    for (int mm = 0; mm < kN2; ++mm) z += h2[mm] * W[kEW3 + mm * kN3 + tid];
    const double g = h2[tid % kN2] + tanh(z);
    for (int c = 0; c < 4; ++c) {
      const size_t o = ((size_t)(ti * nt + tj) * 4 + c) * kN3 + tid;
      pad64[o] = Rp[c] * g;
      pad32[o] = (float)(Rp[c] * g);
    }
  }
}

// ------------------------------------------------------------------ fitting net
enum EpiMode { EPI_TANH = 0, EPI_RES_TANH = 1, EPI_BWD = 2, EPI_NONE = 3 };

template <class T>
struct GemmArgs {
  const int* type_off;   // device: first row of each type
  const int* type_count; // device: rows of each type
  int type;
  int K, Ncol;
  const T* A;            // [rows][K]
  const T* B;            // [K][Ncol]
  T* C;                  // [rows][Ncol]
  const T* bias;         // [Ncol] (EPI_TANH, EPI_RES_TANH)
  const T* res;          // [rows][Ncol] or [Ncol] (res_vec)
  int res_vec;
  const T* aux_in;       // [rows][Ncol]: EPI_BWD factor source
  T* aux_out;            // [rows][Ncol]: EPI_RES_TANH tanh output / EPI_BWD pre-factor gradient
  int mode;
};

constexpr int GBM = 64, GBN = 80, GBK = 16;

template <class T>
__global__ void __launch_bounds__(256) k_fit_gemm(GemmArgs<T> g) {
  __shared__ T As[GBK][GBM + 1];
  __shared__ T Bs[GBK][GBN];
  const int rows = g.type_count[g.type];
  const int r0 = blockIdx.x * GBM;
  if (r0 >= rows) return;
  const int row_base = g.type_off[g.type];
  const int c0 = blockIdx.y * GBN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][5];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[p][q] = T(0);
  const T* A = g.A + (size_t)row_base * g.K;
  for (int k0 = 0; k0 < g.K; k0 += GBK) {
    for (int e = threadIdx.x; e < GBM * GBK; e += 256) {
      int rr = e / GBK, kk = e % GBK;
      int row = r0 + rr;
      As[kk][rr] = (row < rows && k0 + kk < g.K) ? A[(size_t)row * g.K + k0 + kk] : T(0);
    }
    for (int e = threadIdx.x; e < GBK * GBN; e += 256) {
      int kk = e / GBN, cc = e % GBN;
      Bs[kk][cc] = (k0 + kk < g.K) ? g.B[(size_t)(k0 + kk) * g.Ncol + c0 + cc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      T av[4], bv[5];
#pragma unroll
      for (int p = 0; p < 4; ++p) av[p] = As[kk][ty * 4 + p];
#pragma unroll
      for (int q = 0; q < 5; ++q) bv[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[p][q] += av[p] * bv[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    int row = r0 + ty * 4 + p;
    if (row >= rows) continue;
    size_t grow = (size_t)(row_base + row);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      int col = c0 + tx + 16 * q;
      size_t o = grow * g.Ncol + col;
      T v = acc[p][q];
      if (g.mode == EPI_TANH) {
        g.C[o] = dtanh<T>(v + g.bias[col]);
      } else if (g.mode == EPI_RES_TANH) {
        T t = dtanh<T>(v + g.bias[col]);
        g.aux_out[o] = t;
        g.C[o] = g.res[o] + t;
      } else if (g.mode == EPI_BWD) {
        T h = v + (g.res_vec ? g.res[col] : g.res[o]);
        T f = g.aux_in[o];
        if (g.aux_out) g.aux_out[o] = h;
        g.C[o] = h * (T(1) - f * f);
      } else {
        g.C[o] = v;
      }
    }
  }
}

// E_i = H3 . w4 + b4 + e_bias[t];  dZ3 = w4 * (1 - T3^2) written over H3.
template <class T>
__global__ void k_fit_head(const int* type_off, const int* type_count, int type, T* H3, const T* T3,
                           const T* w4, const T* b4, const T* ebias, double* e_atom) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= type_count[type]) return;
  const size_t r = (size_t)(type_off[type] + row);
  T e = T(0);
  for (int n = lane; n < kF; n += 32) {
    T h = H3[r * kF + n], t = T3[r * kF + n], w = w4[n];
    e += h * w;
    H3[r * kF + n] = w * (T(1) - t * t);
  }
  e = warp_sum<T>(e);
  if (lane == 0) e_atom[r] = (double)e + (double)b4[0] + (double)ebias[type];
}

template <class T>
dp_status run_fitting(Model* m, int N) {
  const T* w = (sizeof(T) == 8) ? reinterpret_cast<const T*>(m->w64) : reinterpret_cast<const T*>(m->w32);
  const T* wT = (sizeof(T) == 8) ? reinterpret_cast<const T*>(m->fitT64) : reinterpret_cast<const T*>(m->fitT32);
  T* act[5];
  for (int q = 0; q < 5; ++q) act[q] = static_cast<T*>(m->act[q]);
  const size_t emb_total = (size_t)m->ntypes * m->ntypes * kEmbParams;
  const size_t ebias_off = emb_total + (size_t)m->ntypes * kFitParams;
  const int gx = cdiv(N, GBM);
  for (int t = 0; t < m->ntypes; ++t) {
    const T* P = w + emb_total + (size_t)t * kFitParams;
    const T* PT = wT + (size_t)t * (kF * kKD + 2 * kF * kF);
    GemmArgs<T> g{};
    g.type_off = m->type_off; g.type_count = m->type_count; g.type = t;
    // F1: H1 = tanh(D W1 + b1)
    g.K = kKD; g.Ncol = kF; g.A = static_cast<const T*>(m->Dm); g.B = P + kFW1; g.C = act[0];
    g.bias = P + kFb1; g.mode = EPI_TANH;
    k_fit_gemm<T><<<dim3(gx, kF / GBN), 256, 0, m->stream>>>(g);
    // F2: T2 = tanh(H1 W2 + b2), H2 = H1 + T2
    g.K = kF; g.A = act[0]; g.B = P + kFW2; g.C = act[2]; g.bias = P + kFb2; g.res = act[0]; g.res_vec = 0;
    g.aux_out = act[1]; g.mode = EPI_RES_TANH;
    k_fit_gemm<T><<<dim3(gx, kF / GBN), 256, 0, m->stream>>>(g);
    // F3: T3 = tanh(H2 W3 + b3), H3 = H2 + T3
    g.A = act[2]; g.B = P + kFW3; g.C = act[4]; g.bias = P + kFb3; g.res = act[2]; g.aux_out = act[3];
    k_fit_gemm<T><<<dim3(gx, kF / GBN), 256, 0, m->stream>>>(g);
    // head: E_i, dZ3 = w4 (1 - T3^2) over H3
    k_fit_head<T><<<cdiv(N, 8), 256, 0, m->stream>>>(m->type_off, m->type_count, t, act[4], act[3], P + kFw4,
                                                     P + kFb4, w + ebias_off, m->e_atom);
    // B3: dH2 = w4 + dZ3 W3^T ; dZ2 = dH2 (1 - T2^2)  (dH2 -> act[3], dZ2 -> act[2])
    g.A = act[4]; g.B = PT + kF * kKD + kF * kF; g.C = act[2]; g.res = P + kFw4; g.res_vec = 1;
    g.aux_in = act[1]; g.aux_out = act[3]; g.mode = EPI_BWD;
    k_fit_gemm<T><<<dim3(gx, kF / GBN), 256, 0, m->stream>>>(g);
    // B2: dH1 = dH2 + dZ2 W2^T ; dZ1 = dH1 (1 - H1^2)  (dZ1 -> act[1])
    g.A = act[2]; g.B = PT + kF * kKD; g.C = act[1]; g.res = act[3]; g.res_vec = 0; g.aux_in = act[0];
    g.aux_out = nullptr;
    k_fit_gemm<T><<<dim3(gx, kF / GBN), 256, 0, m->stream>>>(g);
    // B1: dD = dZ1 W1^T
    g.K = kF; g.Ncol = kKD; g.A = act[1]; g.B = PT; g.C = static_cast<T*>(m->dD); g.mode = EPI_NONE;
    k_fit_gemm<T><<<dim3(gx, kKD / GBN), 256, 0, m->stream>>>(g);
    m->launches += 7;
  }
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

template <class T>
EmbArgs<T> make_emb_args(Model* m, int N) {
  EmbArgs<T> a{};
  a.N = N; a.ntypes = m->ntypes; a.S = m->S;
  for (int t = 0; t <= m->ntypes; ++t) a.sel_off[t] = m->sel_off[t];
  a.rc = (T)m->rc; a.rs = (T)m->rs; a.invS = T(1) / (T)m->S; a.switch_kind = m->switch_kind;
  a.w = (sizeof(T) == 8) ? reinterpret_cast<const T*>(m->w64) : reinterpret_cast<const T*>(m->w32);
  a.stat = (sizeof(T) == 8) ? reinterpret_cast<const T*>(m->stat64) : reinterpret_cast<const T*>(m->stat32);
  a.pad = !m->has_pad ? nullptr
                      : (sizeof(T) == 8) ? reinterpret_cast<const T*>(m->pad64) : reinterpret_cast<const T*>(m->pad32);
  for (int t = 0; t < m->ntypes; ++t) a.sel[t] = m->sel[t];
  a.tab = (m->tab_n == 0) ? nullptr
          : (sizeof(T) == 8) ? reinterpret_cast<const T*>(m->tab64) : reinterpret_cast<const T*>(m->tab32);
  a.tab_n = m->tab_n;
  a.tab_x0 = (T)m->tab_x0;
  a.tab_ih = m->tab_n ? (T)(1.0 / m->tab_h) : T(0);
  a.itype = m->itype; a.nl_j = m->nl_j; a.nl_d = m->nl_d; a.nl_count = m->nl_count;
  a.Tm = static_cast<T*>(m->Tm); a.Dm = static_cast<T*>(m->Dm); a.dD = static_cast<const T*>(m->dD);
  a.force = m->force; a.vir_atom = m->vir_atom;
  return a;
}

template <class K>
int resident_grid(K kernel, int threads, size_t smem, int work) {
  int per_sm = blocks_per_sm(reinterpret_cast<const void*>(kernel), threads, smem);
  return std::max(1, std::min(work, num_sms() * per_sm));
}

template <class T>
dp_status run_descriptor(Model* m, int N) {
  constexpr int NB = EB<T>::v;
  EmbArgs<T> a = make_emb_args<T>(m, N);
  size_t smem = sizeof(T) * ((size_t)m->ntypes * kEmbParams + NB * kGP + NB * 4 + 4 * kN3);
  auto fn = (m->tab_n > 0) ? k_embed_fwd<T, true> : k_embed_fwd<T, false>;
  DP_CUDA_TRY(m, ensure_smem(reinterpret_cast<const void*>(fn), smem));
  int grid = resident_grid(fn, NB, smem, N);
  fn<<<grid, NB, smem, m->stream>>>(a);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

template <class T>
dp_status run_embed_backward(Model* m, int N) {
  constexpr int NB = EB<T>::v;
  EmbArgs<T> a = make_emb_args<T>(m, N);
  size_t smem = sizeof(T) * ((size_t)m->ntypes * kEmbParams + 8 * kN3 + kKD + (size_t)kH * NB);
  auto fn = (m->tab_n > 0) ? k_embed_bwd<T, true> : k_embed_bwd<T, false>;
  DP_CUDA_TRY(m, ensure_smem(reinterpret_cast<const void*>(fn), smem));
  int grid = resident_grid(fn, NB, smem, N);
  fn<<<grid, NB, smem, m->stream>>>(a);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

}  // namespace

dp_status launch_pad_rows(Model* m) {
  m->has_pad = false;
  for (double v : m->davg_host) m->has_pad = m->has_pad || v != 0.0;
  if (!m->has_pad) return DP_OK;
  k_pad_rows<<<m->ntypes * m->ntypes, 128>>>(m->ntypes, m->w64, m->stat64, m->pad64, m->pad32);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_descriptor(Model* m, int N) {
  if (is_mixed(m)) return launch_mix_descriptor(m, N);
  return m->prec == DP_FP64 ? run_descriptor<double>(m, N) : run_descriptor<float>(m, N);
}
dp_status launch_fitting(Model* m, int N) {
  if (is_mixed(m)) return launch_mix_fitting(m, N);
  return m->prec == DP_FP64 ? run_fitting<double>(m, N) : run_fitting<float>(m, N);
}
dp_status launch_embed_backward(Model* m, int N) {
  if (is_mixed(m)) return launch_mix_embed_backward(m, N);
  return m->prec == DP_FP64 ? run_embed_backward<double>(m, N) : run_embed_backward<float>(m, N);
}

}  // namespace dpg
