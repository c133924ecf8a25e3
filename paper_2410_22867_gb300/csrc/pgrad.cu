// Parameter gradient of the training loss
//   L = cE (E - E0)^2 + cF sum_k |F_k - F0_k|^2
// with respect to every network parameter theta (embedding nets, fitting nets,
// e_bias) of the model of Section II-A / Fig. 1, in FP64 or FP32.
//
// With alpha = 2 cE (E - E0) and w = 2 cF (F - F0) held fixed, and F = -dE/dx,
//   dL/dtheta = alpha dE/dtheta - d/dtheta [ sum_k w_k . dE/dx_k ],
// i.e. the gradient of Psi = alpha E - D_w E, where D_w E is the directional
// derivative of E along the displacement field w.  D_w E is computed by carrying
// a tangent (derivative along w) beside every value of the forward pass:
// pair vectors get d' = w_j - w_i, and the tangent runs through the environment
// row, the embedding net, T, the descriptor and the fitting net to E_i'.  A
// reverse sweep over that (value, tangent) computation then gives dPsi/dtheta.
//
// Work runs per chunk of centre atoms of one type (at most pg_cap atoms):
//   1. embedding forward with tangents -> T, T' per atom;
//   2. descriptor D, D' per atom, stacked as the 2n rows [D; D'];
//   3. fitting net forward on the stacked rows (GEMMs), activations kept;
//   4. fitting reverse: adjoint rows [u_bar; v_bar] per layer, weight gradients as
//      GEMMs over the atoms, and [D_bar; D'_bar];
//   5. descriptor reverse -> T_bar, T'_bar per atom;
//   6. embedding reverse per neighbour row (activations recomputed), in row
//      chunks of at most kPgRows: each row writes its layer inputs and
//      pre-activation adjoints, whose products summed over rows are the weight
//      gradients (GEMMs with the rows as the reduction dimension).
// Weight gradients are accumulated with FP64 atomics.
#include "common.cuh"

namespace dpg {
namespace {

template <class T> __device__ __forceinline__ T tanh_t(T x);
template <> __device__ __forceinline__ float tanh_t<float>(float x) { return tanhf(x); }
template <> __device__ __forceinline__ double tanh_t<double>(double x) { return tanh(x); }

template <class T>
__device__ __forceinline__ void switch_t(T r, T rs, T rc, int kind, T& sw, T& dsw) {
  if (r < rs) { sw = T(1); dsw = T(0); return; }
  if (r >= rc) { sw = T(0); dsw = T(0); return; }
  const T wd = rc - rs;
  const T u = (r - rs) / wd;
  if (kind == 1) {
    const T pi = T(3.14159265358979323846);
    sw = T(0.5) * cos(pi * u) + T(0.5);
    dsw = T(-0.5) * pi * sin(pi * u) / wd;
  } else {
    const T u2 = u * u;
    sw = u2 * u * (T(-6) * u2 + T(15) * u - T(10)) + T(1);
    dsw = T(-30) * u2 * (u - T(1)) * (u - T(1)) / wd;
  }
}

template <class T>
__device__ __forceinline__ void pair_vec(const void* nl_d, size_t e, T* d);
template <>
__device__ __forceinline__ void pair_vec<float>(const void* nl_d, size_t e, float* d) {
  const float4 v = static_cast<const float4*>(nl_d)[e];
  d[0] = v.x; d[1] = v.y; d[2] = v.z;
}
template <>
__device__ __forceinline__ void pair_vec<double>(const void* nl_d, size_t e, double* d) {
  const dvec4 v = static_cast<const dvec4*>(nl_d)[e];
  d[0] = v.x; d[1] = v.y; d[2] = v.z;
}

template <class T>
struct PgArgs {
  int N, ntypes, S;
  int sel_off[kMaxTypes + 1];
  T rc, rs, invS;
  int switch_kind;
  const T* w;            // theta
  const T* stat;         // davg [nt][4], 1/dstd [nt][4]
  const int* nl_j;
  const void* nl_d;
  const int* nl_count;   // [N][nt]
  const double* wdir;    // [N][3] tangent direction w (internal order)
  const T* pad;          // [nt][nt][4][100] padded-slot term of T, or null (every davg is 0)
  int sel[kMaxTypes];
};

// Environment row R_hat and its tangent along d' (Jacobian of (s, s d/r), s = sw/r).
template <class T>
__device__ __forceinline__ void env_tangent(const PgArgs<T>& a, int ti, const T* d, const T* dd, T* R, T* Rd) {
  const T r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  T sw, dsw;
  switch_t<T>(r, a.rs, a.rc, a.switch_kind, sw, dsw);
  const T rinv = T(1) / r;
  const T s = sw * rinv;
  const T q = sw * rinv * rinv;
  const T rdot = (d[0] * dd[0] + d[1] * dd[1] + d[2] * dd[2]) * rinv;  // dr along d'
  const T sdot = (dsw * rinv - sw * rinv * rinv) * rdot;
  const T qdot = (dsw * rinv * rinv - T(2) * sw * rinv * rinv * rinv) * rdot;
  R[0] = s;
  Rd[0] = sdot;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R[1 + c] = q * d[c];
    Rd[1 + c] = qdot * d[c] + q * dd[c];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const T isd = a.stat[(a.ntypes + ti) * 4 + c];
    R[c] = (R[c] - a.stat[ti * 4 + c]) * isd;
    Rd[c] *= isd;
  }
}

template <class T>
__device__ __forceinline__ void row_geometry(const PgArgs<T>& a, int i, int ti, size_t e, T* R, T* Rd) {
  T d[3], dd[3];
  pair_vec<T>(a.nl_d, e, d);
  const int j = a.nl_j[e];
#pragma unroll
  for (int c = 0; c < 3; ++c) dd[c] = (T)(a.wdir[3 * (size_t)j + c] - a.wdir[3 * (size_t)i + c]);
  env_tangent<T>(a, ti, d, dd, R, Rd);
}

// Embedding layers 1 and 2 with tangents: h1, h1' [25]; h2, h2' [50]; v1 = x' W1; z2' [50].
template <class T>
__device__ __forceinline__ void emb12_tangent(const T* __restrict__ W, T x, T xd, T* h1, T* hd1, T* v1, T* h2,
                                              T* hd2, T* zd2) {
#pragma unroll 1
  for (int k = 0; k < kN1; ++k) {
    h1[k] = tanh_t<T>(x * W[kEW1 + k] + W[kEb1 + k]);
    v1[k] = xd * W[kEW1 + k];
    hd1[k] = (T(1) - h1[k] * h1[k]) * v1[k];
  }
#pragma unroll 1
  for (int m = 0; m < kN2; ++m) {
    T z = W[kEb2 + m], zd = T(0);
#pragma unroll 5
    for (int k = 0; k < kN1; ++k) {
      z += h1[k] * W[kEW2 + k * kN2 + m];
      zd += hd1[k] * W[kEW2 + k * kN2 + m];
    }
    const T t2 = tanh_t<T>(z);
    h2[m] = h1[m % kN1] + t2;
    hd2[m] = hd1[m % kN1] + (T(1) - t2 * t2) * zd;
    zd2[m] = zd;
  }
}

// 1. T and T' of each atom of the chunk: CTA per atom, rows staged in shared memory.
constexpr int kPgNB = 64;
constexpr int kPgGP = kN3 + 1;

template <class T>
__global__ void __launch_bounds__(kPgNB) k_pg_emb_fwd(PgArgs<T> a, int ti, int a0, int n, T* TT) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sG = reinterpret_cast<T*>(smem_raw);  // [NB][GP]
  T* sGd = sG + kPgNB * kPgGP;             // [NB][GP]
  T* sR = sGd + kPgNB * kPgGP;             // [NB][4]
  T* sRd = sR + kPgNB * 4;                 // [NB][4]
  const int tid = threadIdx.x;
  for (int li = blockIdx.x; li < n; li += gridDim.x) {
    const int i = a0 + li;
    T acc[2][4], accd[2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[u][c] = accd[u][c] = T(0);
    for (int tj = 0; tj < a.ntypes; ++tj) {
      const int cnt = a.nl_count[(size_t)i * a.ntypes + tj];
      const T* W = a.w + (size_t)(ti * a.ntypes + tj) * kEmbParams;
      for (int base = 0; base < cnt; base += kPgNB) {
        const int rows = min(kPgNB, cnt - base);
        if (tid < rows) {
          T R[4], Rd[4];
          row_geometry<T>(a, i, ti, (size_t)i * a.S + a.sel_off[tj] + base + tid, R, Rd);
#pragma unroll
          for (int c = 0; c < 4; ++c) { sR[tid * 4 + c] = R[c]; sRd[tid * 4 + c] = Rd[c]; }
          T h1[kN1], hd1[kN1], v1[kN1], h2[kN2], hd2[kN2], zd2[kN2];
          emb12_tangent<T>(W, R[0], Rd[0], h1, hd1, v1, h2, hd2, zd2);
          T* g = sG + tid * kPgGP;
          T* gd = sGd + tid * kPgGP;
#pragma unroll 1
          for (int q = 0; q < kN3; ++q) {
            T z = W[kEb3 + q], zd = T(0);
#pragma unroll 5
            for (int m = 0; m < kN2; ++m) {
              z += h2[m] * W[kEW3 + m * kN3 + q];
              zd += hd2[m] * W[kEW3 + m * kN3 + q];
            }
            const T t3 = tanh_t<T>(z);
            g[q] = h2[q % kN2] + t3;
            gd[q] = hd2[q % kN2] + (T(1) - t3 * t3) * zd;
          }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int col = tid + u * kPgNB;
          if (col < kN3) {
            for (int rr = 0; rr < rows; ++rr) {
              const T gv = sG[rr * kPgGP + col], gdv = sGd[rr * kPgGP + col];
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                acc[u][c] += sR[rr * 4 + c] * gv;
                accd[u][c] += sRd[rr * 4 + c] * gv + sR[rr * 4 + c] * gdv;
              }
            }
          }
        }
        __syncthreads();
      }
    }
    if (a.pad)  // padded slots: constant in the positions, so they add to T but not to T'
      for (int tj = 0; tj < a.ntypes; ++tj) {
        const T np = T(a.sel[tj] - a.nl_count[(size_t)i * a.ntypes + tj]);
        const T* P = a.pad + (size_t)(ti * a.ntypes + tj) * 4 * kN3;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int col = tid + u * kPgNB;
          if (col < kN3)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[u][c] += np * P[c * kN3 + col];
        }
      }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int col = tid + u * kPgNB;
      if (col < kN3)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          TT[(size_t)li * 800 + c * kN3 + col] = acc[u][c] * a.invS;
          TT[(size_t)li * 800 + 400 + c * kN3 + col] = accd[u][c] * a.invS;
        }
    }
  }
}

// 2. D = T^T T[:, :16] and D' = T'^T T< + T^T T'< as rows li and n + li of Y.
template <class T>
__global__ void k_pg_desc(int n, const T* TT, T* Y) {
  __shared__ T s[800];
  for (int li = blockIdx.x; li < n; li += gridDim.x) {
    __syncthreads();
    for (int q = threadIdx.x; q < 800; q += blockDim.x) s[q] = TT[(size_t)li * 800 + q];
    __syncthreads();
    const T* Tp = s;
    const T* Td = s + 400;
    for (int o = threadIdx.x; o < kKD; o += blockDim.x) {
      const int aa = o / kM2, b = o % kM2;
      T v = T(0), vd = T(0);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        v += Tp[c * kN3 + aa] * Tp[c * kN3 + b];
        vd += Td[c * kN3 + aa] * Tp[c * kN3 + b] + Tp[c * kN3 + aa] * Td[c * kN3 + b];
      }
      Y[(size_t)li * kKD + o] = v;
      Y[(size_t)(n + li) * kKD + o] = vd;
    }
  }
}

// 5. T_bar and T'_bar from D_bar (row li of Yb) and D'_bar (row n + li).
template <class T>
__global__ void k_pg_desc_bwd(int n, const T* TT, const T* Yb, T* TB) {
  __shared__ T s[800 + 2 * kKD];
  for (int li = blockIdx.x; li < n; li += gridDim.x) {
    __syncthreads();
    for (int q = threadIdx.x; q < 800; q += blockDim.x) s[q] = TT[(size_t)li * 800 + q];
    for (int q = threadIdx.x; q < kKD; q += blockDim.x) {
      s[800 + q] = Yb[(size_t)li * kKD + q];
      s[800 + kKD + q] = Yb[(size_t)(n + li) * kKD + q];
    }
    __syncthreads();
    const T* Tp = s;
    const T* Td = s + 400;
    const T* Db = s + 800;
    const T* Ddb = s + 800 + kKD;
    for (int o = threadIdx.x; o < 400; o += blockDim.x) {
      const int c = o / kN3, aa = o % kN3;
      T tb = T(0), tdb = T(0);
#pragma unroll
      for (int b = 0; b < kM2; ++b) {
        tb += Db[aa * kM2 + b] * Tp[c * kN3 + b] + Ddb[aa * kM2 + b] * Td[c * kN3 + b];
        tdb += Ddb[aa * kM2 + b] * Tp[c * kN3 + b];
      }
      if (aa < kM2) {
        for (int a2 = 0; a2 < kN3; ++a2) {
          tb += Db[a2 * kM2 + aa] * Tp[c * kN3 + a2] + Ddb[a2 * kM2 + aa] * Td[c * kN3 + a2];
          tdb += Ddb[a2 * kM2 + aa] * Tp[c * kN3 + a2];
        }
      }
      TB[(size_t)li * 800 + o] = tb;
      TB[(size_t)li * 800 + 400 + o] = tdb;
    }
  }
}

// 5b. Parameter gradient through the padded slots of centre type ti, one block per neighbour
//     type tj.  Every padded slot of segment tj holds the row R_pad = -davg[ti] / dstd[ti] and
//     G = N_{ti,tj}(R_pad_0), so with T_bar the adjoint of T (row li of TB, primal half):
//       G_bar[a] = (1/S) sum_li (sel[tj] - count_li,tj) sum_c T_bar_li[c][a] R_pad[c],
//     and the reverse of the embedding net at the single input R_pad_0 gives the parameter
//     gradients (FP64 atomics).  The input is a constant (davg, dstd are not parameters).
template <class T>
__global__ void __launch_bounds__(128) k_pg_pad_rev(PgArgs<T> a, int ti, int a0, int n, const T* __restrict__ TB,
                                                   double* grad) {
  const int tj = blockIdx.x, tid = threadIdx.x;
  const T* W = a.w + (size_t)(ti * a.ntypes + tj) * kEmbParams;
  double* gW = grad + (size_t)(ti * a.ntypes + tj) * kEmbParams;
  __shared__ T Rp[4], h1[kN1], t2[kN2], h2[kN2], gG[kN3], dz3[kN3], dh2[kN2], dz2[kN2];
  if (tid < 4) Rp[tid] = (T(0) - a.stat[ti * 4 + tid]) * a.stat[(a.ntypes + ti) * 4 + tid];
  __syncthreads();
  if (tid < kN3) {
    T acc = T(0);
    for (int li = 0; li < n; ++li) {
      const T np = T(a.sel[tj] - a.nl_count[(size_t)(a0 + li) * a.ntypes + tj]);
      const T* tb = TB + (size_t)li * 800;
      acc += np * (tb[tid] * Rp[0] + tb[kN3 + tid] * Rp[1] + tb[2 * kN3 + tid] * Rp[2] + tb[3 * kN3 + tid] * Rp[3]);
    }
    gG[tid] = acc * a.invS;
  }
  const T x = Rp[0];
  if (tid < kN1) h1[tid] = tanh_t<T>(x * W[kEW1 + tid] + W[kEb1 + tid]);
  __syncthreads();
  if (tid < kN2) {
    T z = W[kEb2 + tid];
    for (int k = 0; k < kN1; ++k) z += h1[k] * W[kEW2 + k * kN2 + tid];
    t2[tid] = tanh_t<T>(z);
    h2[tid] = h1[tid % kN1] + t2[tid];
  }
  __syncthreads();
  if (tid < kN3) {  // G[a] = h2[a % 50] + tanh(z3[a])
    T z = W[kEb3 + tid];
    for (int mm = 0; mm < kN2; ++mm) z += h2[mm] * W[kEW3 + mm * kN3 + tid];
    const T t3 = tanh_t<T>(z);
    dz3[tid] = gG[tid] * (T(1) - t3 * t3);
    atomicAdd(&gW[kEb3 + tid], (double)dz3[tid]);
  }
  __syncthreads();
  for (int q = tid; q < kN2 * kN3; q += blockDim.x)
    atomicAdd(&gW[kEW3 + q], (double)(h2[q / kN3] * dz3[q % kN3]));
  if (tid < kN2) {
    T v = gG[tid] + gG[tid + kN2];
    for (int aa = 0; aa < kN3; ++aa) v += W[kEW3 + tid * kN3 + aa] * dz3[aa];
    dh2[tid] = v;
    dz2[tid] = v * (T(1) - t2[tid] * t2[tid]);
    atomicAdd(&gW[kEb2 + tid], (double)dz2[tid]);
  }
  __syncthreads();
  for (int q = tid; q < kN1 * kN2; q += blockDim.x)
    atomicAdd(&gW[kEW2 + q], (double)(h1[q / kN2] * dz2[q % kN2]));
  if (tid < kN1) {
    T v = dh2[tid] + dh2[tid + kN1];
    for (int mm = 0; mm < kN2; ++mm) v += W[kEW2 + tid * kN2 + mm] * dz2[mm];
    const T dz1 = v * (T(1) - h1[tid] * h1[tid]);
    atomicAdd(&gW[kEb1 + tid], (double)dz1);
    atomicAdd(&gW[kEW1 + tid], (double)(x * dz1));
  }
}

// Plain tiled GEMM C[M x N] = op(A)[M x K] op(B)[K x N] (row-major storage, op = transpose
// when TA / TB).  OUT 0: store; 1: C += result; 2: atomicAdd into FP64 C, with the K range
// split over gridDim.z.
constexpr int kGM = 64, kGN = 64, kGK = 16;

template <class T, bool TA, bool TB, int OUT>
__global__ void __launch_bounds__(256) k_pg_gemm(int M, int N, int K, const T* __restrict__ A, int lda,
                                               const T* __restrict__ B, int ldb, void* Cv, int ldc) {
  __shared__ T As[kGK][kGM + 1];
  __shared__ T Bs[kGK][kGN + 1];
  const int m0 = blockIdx.y * kGM, n0 = blockIdx.x * kGN;
  const int kchunk = (K + gridDim.z - 1) / gridDim.z;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = T(0);
  for (int k0 = kbeg; k0 < kend; k0 += kGK) {
    for (int e = threadIdx.x; e < kGM * kGK; e += 256) {
      const int mm = TA ? e % kGM : e / kGK, kk = TA ? e / kGM : e % kGK;
      const int gm = m0 + mm, gk = k0 + kk;
      T v = T(0);
      if (gm < M && gk < kend) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < kGK * kGN; e += 256) {
      const int nn = TB ? e / kGK : e % kGN, kk = TB ? e % kGK : e / kGN;
      const int gn = n0 + nn, gk = k0 + kk;
      T v = T(0);
      if (gn < N && gk < kend) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) av[p] = As[kk][ty * 4 + p];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] += av[p] * bv[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int gm = m0 + ty * 4 + p;
    if (gm >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gn = n0 + tx + 16 * q;
      if (gn >= N) continue;
      const size_t o = (size_t)gm * ldc + gn;
      if (OUT == 2) {
        atomicAdd(static_cast<double*>(Cv) + o, (double)acc[p][q]);
      } else {
        T* C = static_cast<T*>(Cv);
        C[o] = (OUT == 1 ? C[o] : T(0)) + acc[p][q];
      }
    }
  }
}

// 3. Fitting activations on the stacked rows F = [z; z'] (raw GEMM output, 2n x 240):
//    layer 1: F <- [h1; v1], H <- [h1; h1'];  layer L > 1: F <- [k_L; v_L], and for L = 2
//    H <- H + [k2; (1 - k2^2) v2] (H then holds [h2; h2']).
template <class T>
__global__ void k_pg_fit_act(int n, int layer, const T* __restrict__ bias, T* F, T* H) {
  const size_t total = (size_t)n * kF;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int col = (int)(e % kF);
    const size_t rp = e, rt = e + total;
    const T k = tanh_t<T>(F[rp] + bias[col]);
    F[rp] = k;
    const T v = F[rt];
    if (layer == 1) {
      H[rp] = k;
      H[rt] = (T(1) - k * k) * v;
    } else if (layer == 2) {
      H[rp] += k;
      H[rt] += (T(1) - k * k) * v;
    }
  }
}

// 4a. Head: h3 = h2 + k3, h3' = h2' + (1 - k3^2) v3; gradient of w4 (sum over atoms of
//     alpha h3 - h3'); adjoints of (h3, h3') = (alpha w4, -w4) into G.
template <class T>
__global__ void k_pg_head(int n, const T* __restrict__ H, const T* __restrict__ F3, const T* __restrict__ w4,
                          const double* scal, T* G, double* gw4) {
  const T alpha = (T)scal[0];
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= kF) return;
  const size_t nt = (size_t)n * kF;
  double acc = 0.0;
  const T wv = w4[col];
  for (int r = blockIdx.y; r < n; r += gridDim.y) {
    const size_t e = (size_t)r * kF + col;
    const T k3 = F3[e], v3 = F3[e + nt];
    const T h3 = H[e] + k3;
    const T h3d = H[e + nt] + (T(1) - k3 * k3) * v3;
    acc += (double)(alpha * h3 - h3d);
    G[e] = alpha * wv;
    G[e + nt] = -wv;
  }
  atomicAdd(gw4 + col, acc);
}

// 4b. Layer reverse: from the adjoints (A, A') of (h_L, h_L') held in G and F_L = [k; v]:
//     k_bar = A - 2 k (A' v), u_bar = k_bar (1 - k^2), v_bar = A' (1 - k^2)  -> U = [u_bar; v_bar];
//     bias gradient += sum over atoms of u_bar.  For layer 2 also H <- [h1; h1'] from F1.
template <class T>
__global__ void k_pg_fit_rev(int n, int layer, const T* __restrict__ G, const T* __restrict__ FL,
                             const T* __restrict__ F1, T* U, T* H, double* gbias) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= kF) return;
  const size_t nt = (size_t)n * kF;
  double acc = 0.0;
  for (int r = blockIdx.y; r < n; r += gridDim.y) {
    const size_t e = (size_t)r * kF + col;
    const T k = FL[e], v = FL[e + nt];
    const T q = T(1) - k * k;
    const T Ap = G[e], At = G[e + nt];
    const T kb = Ap - T(2) * k * (At * v);
    const T ub = kb * q;
    U[e] = ub;
    U[e + nt] = At * q;
    acc += (double)ub;
    if (layer == 2) {
      const T h1 = F1[e];
      H[e] = h1;
      H[e + nt] = (T(1) - h1 * h1) * F1[e + nt];
    }
  }
  atomicAdd(gbias + col, acc);
}

// alpha * (number of atoms) into b4 and e_bias of the type.
__global__ void k_pg_counts(int n, const double* scal, double* gb4, double* gebias) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    atomicAdd(gb4, scal[0] * n);
    atomicAdd(gebias, scal[0] * n);
  }
}

// 6. Embedding reverse, one thread per neighbour row of pair (ti, tj); rows of the chunk's
//    atoms [b0, b0 + nb) are numbered by roff (exclusive offsets, nb + 1 entries).  Each
//    row writes X3 = [h2; h2'], Y3 = [z3_bar; z3'_bar], X2 = [h1; h1'], Y2 = [z2_bar;
//    z2'_bar] (primal at row r, tangent at row R + r) and C1 = [x z1_bar + x' v1_bar, z1_bar].
template <class T>
__global__ void __launch_bounds__(128) k_pg_emb_rev(PgArgs<T> a, int ti, int tj, int a0, int b0, int nb,
                                                   const int* __restrict__ roff, int R, const T* __restrict__ TB,
                                                   T* X3, T* Y3, T* X2, T* Y2, T* C1) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  int lo = 0, hi = nb - 1;  // last atom k with roff[k] <= r
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (roff[mid] <= r) lo = mid; else hi = mid - 1;
  }
  const int i = b0 + lo;
  const size_t e = (size_t)i * a.S + a.sel_off[tj] + (r - roff[lo]);
  const T* W = a.w + (size_t)(ti * a.ntypes + tj) * kEmbParams;
  const T* Tb = TB + (size_t)(i - a0) * 800;
  const T* Tdb = Tb + 400;
  T R4[4], Rd[4];
  row_geometry<T>(a, i, ti, e, R4, Rd);
  const T x = R4[0], xd = Rd[0];
  T h1[kN1], hd1[kN1], v1[kN1], h2[kN2], hd2[kN2], zd2[kN2];
  emb12_tangent<T>(W, x, xd, h1, hd1, v1, h2, hd2, zd2);
  T hb2[kN2], hdb2[kN2];
#pragma unroll 1
  for (int m = 0; m < kN2; ++m) {
    hb2[m] = hdb2[m] = T(0);
    X3[(size_t)r * kN2 + m] = h2[m];
    X3[(size_t)(R + r) * kN2 + m] = hd2[m];
  }
#pragma unroll 1
  for (int q = 0; q < kN3; ++q) {
    T z = W[kEb3 + q], zd = T(0);
#pragma unroll 5
    for (int m = 0; m < kN2; ++m) {
      z += h2[m] * W[kEW3 + m * kN3 + q];
      zd += hd2[m] * W[kEW3 + m * kN3 + q];
    }
    const T t3 = tanh_t<T>(z);
    const T q3 = T(1) - t3 * t3;
    T gb = T(0), gdb = T(0);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      gb += R4[c] * Tb[c * kN3 + q] + Rd[c] * Tdb[c * kN3 + q];
      gdb += R4[c] * Tdb[c * kN3 + q];
    }
    gb *= a.invS;
    gdb *= a.invS;
    const T tb = gb - T(2) * t3 * (gdb * zd);
    const T zb = tb * q3, zdb = gdb * q3;
    hb2[q % kN2] += gb;
    hdb2[q % kN2] += gdb;
#pragma unroll 5
    for (int m = 0; m < kN2; ++m) {
      hb2[m] += zb * W[kEW3 + m * kN3 + q];
      hdb2[m] += zdb * W[kEW3 + m * kN3 + q];
    }
    Y3[(size_t)r * kN3 + q] = zb;
    Y3[(size_t)(R + r) * kN3 + q] = zdb;
  }
  T hb1[kN1], hdb1[kN1];
#pragma unroll 1
  for (int k = 0; k < kN1; ++k) {
    hb1[k] = hdb1[k] = T(0);
    X2[(size_t)r * kN1 + k] = h1[k];
    X2[(size_t)(R + r) * kN1 + k] = hd1[k];
  }
#pragma unroll 1
  for (int m = 0; m < kN2; ++m) {
    const T t2 = h2[m] - h1[m % kN1];
    const T q2 = T(1) - t2 * t2;
    const T tb = hb2[m] - T(2) * t2 * (hdb2[m] * zd2[m]);
    const T zb = tb * q2, zdb = hdb2[m] * q2;
    hb1[m % kN1] += hb2[m];
    hdb1[m % kN1] += hdb2[m];
#pragma unroll 5
    for (int k = 0; k < kN1; ++k) {
      hb1[k] += zb * W[kEW2 + k * kN2 + m];
      hdb1[k] += zdb * W[kEW2 + k * kN2 + m];
    }
    Y2[(size_t)r * kN2 + m] = zb;
    Y2[(size_t)(R + r) * kN2 + m] = zdb;
  }
#pragma unroll 1
  for (int k = 0; k < kN1; ++k) {
    const T q1 = T(1) - h1[k] * h1[k];
    const T kb = hb1[k] - T(2) * h1[k] * (hdb1[k] * v1[k]);
    const T zb = kb * q1, vb = hdb1[k] * q1;
    C1[(size_t)r * 2 * kN1 + k] = x * zb + xd * vb;
    C1[(size_t)r * 2 * kN1 + kN1 + k] = zb;
  }
}

// Column sums of X [rows x cols] (leading dimension ld) added to out (FP64 atomics).
template <class T>
__global__ void k_pg_colsum(int rows, int cols, int ld, const T* __restrict__ X, double* out) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= cols) return;
  double acc = 0.0;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) acc += (double)X[(size_t)r * ld + col];
  atomicAdd(out + col, acc);
}

// alpha, loss, and the tangent direction w = 2 cF (F - F0) in internal order.
__global__ void k_pg_setup(int N, const double* __restrict__ e_atom, const double* __restrict__ force,
                           const double* __restrict__ F0, const int* __restrict__ perm, double E0, double cE,
                           double cF, double* wdir, double* scal) {
  __shared__ double sE[32], sL[32];
  double e = 0.0, l = 0.0;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    e += e_atom[k];
    const int u = perm[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double df = force[3 * (size_t)k + c] - F0[3 * (size_t)u + c];
      l += df * df;
      wdir[3 * (size_t)k + c] = 2.0 * cF * df;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    l += __shfl_xor_sync(0xffffffffu, l, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sE[wid] = e; sL[wid] = l; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double E = 0.0, L = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { E += sE[q]; L += sL[q]; }
    scal[0] = 2.0 * cE * (E - E0);
    scal[1] = cE * (E - E0) * (E - E0) + cF * L;
    scal[2] = E;
  }
}

template <class T, bool TA, bool TB, int OUT>
void gemm(Model* m, int M, int N, int K, const T* A, int lda, const T* B, int ldb, void* C, int ldc, int splitk = 1) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  dim3 grid(cdiv(N, kGN), cdiv(M, kGM), std::max(1, std::min(splitk, cdiv(K, kGK))));
  k_pg_gemm<T, TA, TB, OUT><<<grid, 256, 0, m->stream>>>(M, N, K, A, lda, B, ldb, C, ldc);
  m->launches += 1;
}

template <class T>
dp_status run_param_grad(Model* m, int N, double* grad) {
  const int nt = m->ntypes;
  PgArgs<T> a{};
  a.N = N; a.ntypes = nt; a.S = m->S;
  for (int t = 0; t <= nt; ++t) a.sel_off[t] = m->sel_off[t];
  a.rc = (T)m->rc; a.rs = (T)m->rs; a.invS = T(1) / (T)m->S; a.switch_kind = m->switch_kind;
  const T* theta = (sizeof(T) == 8) ? reinterpret_cast<const T*>(m->w64) : reinterpret_cast<const T*>(m->w32);
  a.w = theta;
  a.stat = (sizeof(T) == 8) ? reinterpret_cast<const T*>(m->stat64) : reinterpret_cast<const T*>(m->stat32);
  a.nl_j = m->nl_j; a.nl_d = m->nl_d; a.nl_count = m->nl_count; a.wdir = m->pg_w;
  a.pad = !m->has_pad ? nullptr
                      : (sizeof(T) == 8) ? reinterpret_cast<const T*>(m->pad64) : reinterpret_cast<const T*>(m->pad32);
  for (int t = 0; t < nt; ++t) a.sel[t] = m->sel[t];

  // host copies of the type ranges and per-atom neighbour counts (chunking)
  std::vector<int> cnt((size_t)N * nt), tc(kMaxTypes + 1);
  DP_CUDA_TRY(m, cudaMemcpyAsync(cnt.data(), m->nl_count, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost,
                                 m->stream));
  DP_CUDA_TRY(m, cudaMemcpyAsync(tc.data(), m->type_count, sizeof(int) * (kMaxTypes + 1), cudaMemcpyDeviceToHost,
                                 m->stream));
  DP_CUDA_TRY(m, cudaStreamSynchronize(m->stream));

  // row offsets of every (centre chunk, neighbour type, row chunk), uploaded once
  struct RowChunk { int ti, tj, a0, b0, nb, R; size_t off; };
  struct AtomChunk { int ti, a0, n; };
  std::vector<AtomChunk> achunks;
  std::vector<RowChunk> rchunks;
  std::vector<int> roffs;
  const int cap = m->pg_cap;
  for (int t = 0; t < nt; ++t)
    if (m->sel[t] > kPgRows) {
      m->last_error = "param_grad: sel larger than the row chunk";
      return DP_ERR_UNSUPPORTED;
    }
  int start = 0;
  for (int ti = 0; ti < nt; ++ti) {
    const int cnt_t = tc[ti];
    for (int c0 = 0; c0 < cnt_t; c0 += cap) {
      AtomChunk ac{ti, start + c0, std::min(cap, cnt_t - c0)};
      achunks.push_back(ac);
      for (int tj = 0; tj < nt; ++tj) {
        int b = ac.a0;
        const int bend = ac.a0 + ac.n;
        while (b < bend) {
          RowChunk rc{ti, tj, ac.a0, b, 0, 0, roffs.size()};
          int rows = 0;
          roffs.push_back(0);
          while (b < bend && rows + cnt[(size_t)b * nt + tj] <= kPgRows) {
            rows += cnt[(size_t)b * nt + tj];
            roffs.push_back(rows);
            ++b;
          }
          rc.nb = b - rc.b0;
          rc.R = rows;
          rchunks.push_back(rc);
        }
      }
    }
    start += cnt_t;
  }
  if (roffs.size() > m->pg_roff_cap) {
    m->last_error = "param_grad: row-offset table larger than allocated";
    return DP_ERR_CAPACITY;
  }
  if (!roffs.empty())
    DP_CUDA_TRY(m, cudaMemcpyAsync(m->pg_roff, roffs.data(), sizeof(int) * roffs.size(), cudaMemcpyHostToDevice,
                                   m->stream));

  // workspace
  T* ws = static_cast<T*>(m->pg_ws);
  const size_t C = (size_t)cap;
  T* TT = ws;
  T* Y = TT + C * 800;
  T* Yb = Y + 2 * C * kKD;
  T* F1 = Yb + 2 * C * kKD;
  T* F2 = F1 + 2 * C * kF;
  T* F3 = F2 + 2 * C * kF;
  T* H = F3 + 2 * C * kF;
  T* U = H + 2 * C * kF;
  T* G = U + 2 * C * kF;
  T* TB = G + 2 * C * kF;
  T* X3 = TB + C * 800;
  T* Y3 = X3 + 2 * (size_t)kPgRows * kN2;
  T* X2 = Y3 + 2 * (size_t)kPgRows * kN3;
  T* Y2 = X2 + 2 * (size_t)kPgRows * kN1;
  T* C1 = Y2 + 2 * (size_t)kPgRows * kN2;

  const size_t emb_total = (size_t)nt * nt * kEmbParams;
  const size_t fsmem = (size_t)(2 * kPgNB * kPgGP + 8 * kPgNB) * sizeof(T);
  DP_CUDA_TRY(m, ensure_smem(reinterpret_cast<const void*>(k_pg_emb_fwd<T>), fsmem));
  const int sms = num_sms();

  for (const AtomChunk& ac : achunks) {
    const int n = ac.n, ti = ac.ti;
    const size_t fb = emb_total + (size_t)ti * kFitParams;  // fitting block of ti
    const T* P = theta + fb;
    double* gP = grad + fb;
    // 1-2: T, T', D, D'
    k_pg_emb_fwd<T><<<std::min(n, 8 * sms), kPgNB, fsmem, m->stream>>>(a, ti, ac.a0, n, TT);
    k_pg_desc<T><<<std::min(n, 8 * sms), 128, 0, m->stream>>>(n, TT, Y);
    m->launches += 2;
    // 3: fitting forward on [D; D']
    const int M2 = 2 * n;
    const int eg = std::min(cdiv((long)n * kF, 256), 8 * sms);
    gemm<T, false, false, 0>(m, M2, kF, kKD, Y, kKD, P + kFW1, kF, F1, kF);
    k_pg_fit_act<T><<<eg, 256, 0, m->stream>>>(n, 1, P + kFb1, F1, H);
    gemm<T, false, false, 0>(m, M2, kF, kF, H, kF, P + kFW2, kF, F2, kF);
    k_pg_fit_act<T><<<eg, 256, 0, m->stream>>>(n, 2, P + kFb2, F2, H);
    gemm<T, false, false, 0>(m, M2, kF, kF, H, kF, P + kFW3, kF, F3, kF);
    k_pg_fit_act<T><<<eg, 256, 0, m->stream>>>(n, 3, P + kFb3, F3, H);
    m->launches += 3;
    // 4: fitting reverse
    const dim3 cg(cdiv(kF, 128), std::min(n, 64));
    k_pg_head<T><<<cg, 128, 0, m->stream>>>(n, H, F3, P + kFw4, m->pg_scal, G, gP + kFw4);
    k_pg_counts<<<1, 32, 0, m->stream>>>(n, m->pg_scal, gP + kFb4, grad + emb_total + (size_t)nt * kFitParams + ti);
    k_pg_fit_rev<T><<<cg, 128, 0, m->stream>>>(n, 3, G, F3, F1, U, H, gP + kFb3);
    m->launches += 3;
    const int sk = std::max(1, std::min(64, M2 / 256));
    gemm<T, true, false, 2>(m, kF, kF, M2, H, kF, U, kF, gP + kFW3, kF, sk);   // W3 grad: [h2; h2']^T U
    gemm<T, false, true, 1>(m, M2, kF, kF, U, kF, P + kFW3, kF, G, kF);        // G += U W3^T
    k_pg_fit_rev<T><<<cg, 128, 0, m->stream>>>(n, 2, G, F2, F1, U, H, gP + kFb2);
    m->launches += 1;
    gemm<T, true, false, 2>(m, kF, kF, M2, H, kF, U, kF, gP + kFW2, kF, sk);   // W2 grad: [h1; h1']^T U
    gemm<T, false, true, 1>(m, M2, kF, kF, U, kF, P + kFW2, kF, G, kF);        // G += U W2^T
    k_pg_fit_rev<T><<<cg, 128, 0, m->stream>>>(n, 1, G, F1, F1, U, H, gP + kFb1);
    m->launches += 1;
    gemm<T, true, false, 2>(m, kKD, kF, M2, Y, kKD, U, kF, gP + kFW1, kF, sk);  // W1 grad: [D; D']^T U
    gemm<T, false, true, 0>(m, M2, kKD, kF, U, kF, P + kFW1, kF, Yb, kKD);      // [D_bar; D'_bar] = U W1^T
    // 5: T_bar, T'_bar
    k_pg_desc_bwd<T><<<std::min(n, 8 * sms), 128, 0, m->stream>>>(n, TT, Yb, TB);
    m->launches += 1;
    if (a.pad) {
      k_pg_pad_rev<T><<<nt, 128, 0, m->stream>>>(a, ti, ac.a0, n, TB, grad);
      m->launches += 1;
    }
    // 6: embedding reverse per neighbour row
    for (const RowChunk& rc : rchunks) {
      if (rc.ti != ti || rc.a0 != ac.a0 || rc.R == 0) continue;
      const int R = rc.R;
      const size_t eb = (size_t)(ti * nt + rc.tj) * kEmbParams;
      k_pg_emb_rev<T><<<cdiv(R, 128), 128, 0, m->stream>>>(a, ti, rc.tj, ac.a0, rc.b0, rc.nb, m->pg_roff + rc.off,
                                                           R, TB, X3, Y3, X2, Y2, C1);
      m->launches += 1;
      const int skr = std::max(1, std::min(128, 2 * R / 512));
      gemm<T, true, false, 2>(m, kN2, kN3, 2 * R, X3, kN2, Y3, kN3, grad + eb + kEW3, kN3, skr);
      gemm<T, true, false, 2>(m, kN1, kN2, 2 * R, X2, kN1, Y2, kN2, grad + eb + kEW2, kN2, skr);
      const int ry = std::min(R, 256);
      k_pg_colsum<T><<<dim3(1, ry), 128, 0, m->stream>>>(R, kN3, kN3, Y3, grad + eb + kEb3);
      k_pg_colsum<T><<<dim3(1, ry), 128, 0, m->stream>>>(R, kN2, kN2, Y2, grad + eb + kEb2);
      k_pg_colsum<T><<<dim3(1, ry), 128, 0, m->stream>>>(R, 2 * kN1, 2 * kN1, C1, grad + eb + kEW1);
      m->launches += 3;
    }
  }
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

}  // namespace

size_t param_grad_workspace_bytes(int cap, bool fp64) {
  const size_t per_atom = 800 + 2 * 2 * (size_t)kKD + 6 * 2 * (size_t)kF + 800;
  const size_t per_row = 2 * (size_t)(kN2 + kN3 + kN1 + kN2) + 2 * kN1;
  return ((size_t)cap * per_atom + (size_t)kPgRows * per_row) * (fp64 ? 8 : 4);
}

dp_status launch_param_grad(Model* m, int N, const double* F0, double E0, double cE, double cF, double* grad,
                            double* loss) {
  DP_CUDA_TRY(m, cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)m->ntheta, m->stream));
  k_pg_setup<<<1, 1024, 0, m->stream>>>(N, m->e_atom, m->force, F0, m->perm, E0, cE, cF, m->pg_w, m->pg_scal);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  dp_status st = (m->prec == DP_FP64) ? run_param_grad<double>(m, N, grad) : run_param_grad<float>(m, N, grad);
  if (st != DP_OK) return st;
  if (loss) DP_CUDA_TRY(m, cudaMemcpyAsync(loss, m->pg_scal + 1, sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  return DP_OK;
}

}  // namespace dpg
