// Neighbour search: type sort, wrap and cell binning, Verlet list within
// r_c + skin with periodic images, and the per-step formatted list within r_c.
//
// The neighbour list is the one LAMMPS builds for the DP pair style (Section
// II-A, Fig. 1(a)), kept per neighbour type so no slicing is needed later
// (the type pre-classified environment matrix of Section III-B1), built with a
// cell list (the cell-list method cited in Section II-A) and a 2 A skin
// rebuilt every k steps (Section IV).
//
// Bit-exactness: a pair (j, n) is in the list iff the FP64 value
//   r2 = ((dx*dx) + (dy*dy)) + (dz*dz),  dx = (x_j + (n H)_x) - x_i,
//   (n H)_x = ((n0 H00 + n1 H10) + n2 H20)
// (round-to-nearest, no FMA) is below the squared cutoff; for an orthorhombic cell (n H)_x is
// n0 L_x exactly.  The kernels first
// classify in FP32 and fall back to that exact FP64 test whenever the FP32
// value lies inside a band wider than its worst-case rounding error, so the
// result equals the FP64 definition while doing FP32 work for almost all pairs
// (FP64 throughput is low on this GPU).
#include "common.cuh"

namespace dpg {
namespace {

__device__ __forceinline__ void set_err(int* err, int bit) { atomicOr(err, bit); }

// Wrap one coordinate into [0, L): w = x - L*floor(x/L); rounding cases that land
// on w < 0 or w >= L become 0.
__device__ __forceinline__ double wrap1(double x, double L) {
  double t = floor(__ddiv_rn(x, L));
  double p = __dmul_rn(t, L);
  double w = __dsub_rn(x, p);
  if (w < 0.0 || w >= L) w = 0.0;
  return w;
}

// Exact FP64 pair vector and squared length in the fixed operation order.
// Component c of the image shift n H in the fixed order ((n0 H0c + n1 H1c) + n2 H2c); for an
// orthorhombic cell (tri = 0) the two zero products drop out and it is n_c L_c, computed as such.
__device__ __forceinline__ double img_shift(const double* H, int tri, int n0, int n1, int n2, int c) {
  if (!tri) return __dmul_rn((double)(c == 0 ? n0 : c == 1 ? n1 : n2), H[4 * c]);
  return __dadd_rn(__dadd_rn(__dmul_rn((double)n0, H[c]), __dmul_rn((double)n1, H[3 + c])),
                   __dmul_rn((double)n2, H[6 + c]));
}

__device__ __forceinline__ double exact_r2(const dvec4& xi, const dvec4& xj, int nx, int ny, int nz,
                                           const RepGeom& g, double* d) {
  d[0] = __dsub_rn(__dadd_rn(xj.x, img_shift(g.H, g.tri, nx, ny, nz, 0)), xi.x);
  d[1] = __dsub_rn(__dadd_rn(xj.y, img_shift(g.H, g.tri, nx, ny, nz, 1)), xi.y);
  d[2] = __dsub_rn(__dadd_rn(xj.z, img_shift(g.H, g.tri, nx, ny, nz, 2)), xi.z);
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__device__ __forceinline__ int pack_img(int nx, int ny, int nz) {
  return ((nx + 512) << 20) | ((ny + 512) << 10) | (nz + 512);
}
__device__ __forceinline__ void unpack_img(int c, int& nx, int& ny, int& nz) {
  nx = ((c >> 20) & 1023) - 512;
  ny = ((c >> 10) & 1023) - 512;
  nz = (c & 1023) - 512;
}

__device__ __forceinline__ int floor_div(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

// ------------------------------------------------------------------ type sort
constexpr int kSortBlock = 1024;

__device__ __forceinline__ int rep_of(const int* rep_off, int nrep, int u) {
  int lo = 0, hi = nrep - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (rep_off[mid] <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_type_count(const int* __restrict__ types, int N, int ntypes, int* blk_count, int* err) {
  __shared__ int cnt[kMaxTypes];
  if (threadIdx.x < kMaxTypes) cnt[threadIdx.x] = 0;
  __syncthreads();
  int u = blockIdx.x * kSortBlock + threadIdx.x;
  if (u < N) {
    int t = types[u];
    if (t < 0 || t >= ntypes) { set_err(err, ERR_TYPE); t = 0; }
    atomicAdd(&cnt[t], 1);
  }
  __syncthreads();
  if (threadIdx.x < kMaxTypes) blk_count[blockIdx.x * kMaxTypes + threadIdx.x] = cnt[threadIdx.x];
}

__global__ void k_type_scan(int nblk, int ntypes, int* blk_count, int* type_count, int* type_off) {
  // single thread: nblk <= a few hundred
  if (threadIdx.x != 0) return;
  int off = 0;
  for (int t = 0; t < ntypes; ++t) {
    type_off[t] = off;
    int run = off;
    for (int b = 0; b < nblk; ++b) {
      int c = blk_count[b * kMaxTypes + t];
      blk_count[b * kMaxTypes + t] = run;
      run += c;
    }
    type_count[t] = run - off;
    off = run;
  }
  type_off[ntypes] = off;
  type_count[kMaxTypes] = off;
}

__global__ void k_type_scatter(const int* __restrict__ types, int N, int ntypes, const int* blk_off,
                               const int* rep_off, int nrep, int* perm, int* inv, int* itype, int* irep) {
  __shared__ int wcnt[kSortBlock / 32][kMaxTypes];
  int u = blockIdx.x * kSortBlock + threadIdx.x;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int t = (u < N) ? types[u] : -1;
  if (t >= ntypes) t = 0;
  if (t < 0 && u < N) t = 0;
  unsigned lt = (1u << lane) - 1u;
  int rank_in_warp = 0;
  for (int q = 0; q < ntypes; ++q) {
    unsigned mask = __ballot_sync(0xffffffffu, t == q);
    if (t == q) rank_in_warp = __popc(mask & lt);
    if (lane == 0) wcnt[w][q] = __popc(mask);
  }
  __syncthreads();
  if (u < N) {
    int before = 0;
    for (int ww = 0; ww < w; ++ww) before += wcnt[ww][t];
    int k = blk_off[blockIdx.x * kMaxTypes + t] + before + rank_in_warp;
    perm[k] = u;
    inv[u] = k;
    itype[k] = t;
    irep[k] = rep_of(rep_off, nrep, u);
  }
}

__global__ void k_load_positions(const double* __restrict__ coords, const int* __restrict__ perm, int N,
                                 dvec4* x) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  int u = perm[k];
  x[k] = make_dvec4(coords[3 * u], coords[3 * u + 1], coords[3 * u + 2], 0.0);
}

// ------------------------------------------------------------------ cells
// xf.w carries the atom's type (bit pattern), read by the Verlet-list gather; xq holds the
// wrapped position in fixed point for exact pair vectors.
__global__ void k_wrap_bin(int N, const int* __restrict__ irep, const int* __restrict__ itype,
                           const RepGeom* __restrict__ geom, dvec4* x, dvec4* xref, float4* xf, qvec4* xq,
                           float4* delta, int* cell_of, int* cell_count) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const RepGeom& g = geom[irep[k]];
  dvec4 p = x[k];
  double w[3], sf[3] = {0.0, 0.0, 0.0};
  if (!g.tri) {
    w[0] = wrap1(p.x, g.L[0]);
    w[1] = wrap1(p.y, g.L[1]);
    w[2] = wrap1(p.z, g.L[2]);
  } else {
    // t = floor(x Hinv) (fixed order), w = x - t H; sf = the fractional coordinate minus t
    const double pc[3] = {p.x, p.y, p.z};
    int t[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double s = __dadd_rn(__dadd_rn(__dmul_rn(pc[0], g.Hinv[c]), __dmul_rn(pc[1], g.Hinv[3 + c])),
                                 __dmul_rn(pc[2], g.Hinv[6 + c]));
      const double f = floor(s);
      t[c] = (int)f;
      sf[c] = s - f;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) w[c] = __dsub_rn(pc[c], img_shift(g.H, 1, t[0], t[1], t[2], c));
  }
  dvec4 q = make_dvec4(w[0], w[1], w[2], 0.0);
  x[k] = q;
  xref[k] = q;
  xf[k] = make_float4((float)w[0], (float)w[1], (float)w[2], __int_as_float(itype[k]));
  qvec4 qk;
  qk.x = llrint(w[0] * 4294967296.0); qk.y = llrint(w[1] * 4294967296.0); qk.z = llrint(w[2] * 4294967296.0);
  qk.w = 0;
  xq[k] = qk;
  delta[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  int c[3];
  for (int a = 0; a < 3; ++a) {
    int ci = g.tri ? (int)floor(sf[a] * g.nc[a]) : (int)floor(w[a] / g.edge[a]);
    c[a] = min(max(ci, 0), g.nc[a] - 1);
  }
  int cid = g.cell_off + (c[0] * g.nc[1] + c[1]) * g.nc[2] + c[2];
  cell_of[k] = cid;
  atomicAdd(&cell_count[cid], 1);
}

// Exclusive scan of the cell counts by one CTA: four consecutive cells per thread, 4096 per
// pass, warp-shuffle scans of the thread sums.
__global__ void __launch_bounds__(1024) k_scan_cells(int ncells, const int* __restrict__ cell_count,
                                                    int* cell_start) {
  __shared__ int ws[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ncells; base += 4096) {
    const int i0 = base + 4 * threadIdx.x;
    int v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = i0 + k < ncells ? cell_count[i0 + k] : 0;
    const int sum = (v[0] + v[1]) + (v[2] + v[3]);
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
      int t = ws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      ws[lane] = t;
    }
    __syncthreads();
    const int c0 = carry;
    int e = c0 + (w > 0 ? ws[w - 1] : 0) + x - sum;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (i0 + k < ncells) cell_start[i0 + k] = e;
      e += v[k];
    }
    const int total = ws[31];
    __syncthreads();  // carry and ws are read before they change
    if (threadIdx.x == 0) carry = c0 + total;
  }
  __syncthreads();
  if (threadIdx.x == 0) cell_start[ncells] = carry;
}

// Counting-sort scatter: the atoms of each cell, and their FP32 positions in the same order
// (so the Verlet walk reads index and position of a candidate with two independent loads).
__global__ void k_fill_cells(int N, const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                             const float4* __restrict__ xf, int* cell_fill, int* cell_atoms, float4* cell_xf) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  int cid = cell_of[k];
  int pos = cell_start[cid] + atomicAdd(&cell_fill[cid], 1);
  cell_atoms[pos] = k;
  cell_xf[pos] = xf[k];
}

// ------------------------------------------------------------------ Verlet list
struct VerletArgs {
  int N, ntypes, VS;
  int vcap[kMaxTypes], vcap_off[kMaxTypes + 1];
  double rcs2;
  float rcs2_hi;               // fp32 prefilter bound (rcs2 + band)
  const int* itype;
  const int* irep;
  const RepGeom* geom;
  const dvec4* x;
  const float4* xf;
  const qvec4* xq;
  const int* cell_of;
  const int* cell_start;
  const int* cell_atoms;
  const float4* cell_xf;
  float4* vl_e;                // entry: pair vector at rebuild (fp32), w = neighbour index (bits)
  int* vl_img;                 // entry: image code (read by the format near the cutoff only)
  int* vcount;
  int* work;                   // atoms left to k_verlet by k_verlet_cell (null: all atoms)
  int* work_n;                 // their number
  int* err;
};

constexpr int kVerletWarps = 4;

// One component of d = x_j + n H - x_i from fixed-point positions (units of 2^-32 A; shq is the
// image shift in the same units): the integer difference D = hi * 2^32 + lo (lo in [0, 2^32)) is
// exact; the float result is hi + lo * 2^-32 with one final rounding (within one ulp of d, up to
// the 2^-32 A rounding of H).  Integer work only: FP64 runs at a small fraction of the FP32 rate
// on this GPU.
__device__ __forceinline__ float fixed_diff(long long qj, long long qi, long long shq) {
  const long long D = qj + shq - qi;
  const int hi = (int)(D >> 32);
  const unsigned lo = (unsigned)(D & 0xffffffffll);
  return fmaf((float)lo, 2.3283064365386963e-10f, (float)hi);
}

// Verlet list of atom i (one warp per atom).  The list only has to contain every pair
// within r_c + skin (the per-step format keeps exactly the pairs within r_c, with an exact
// FP64 test near the cutoff), so a pair is taken when its FP32 r^2 is below (r_c + skin)^2
// plus a band wider than the FP32 rounding error: no FP64 in the candidate test.  The
// stencil's cells are taken 32 at a time; their candidates form one flat range that the
// lanes walk four at a time (independent loads of the cell-ordered index and position in
// flight).  Accepted pairs go straight to
// the list, grouped by neighbour type, in the order found: every consumer is independent
// of the order within a type (the descriptor is a sum over neighbours; the format is a
// compaction), and dp_get_nlist sorts a copy into the canonical order.  The pair vector at
// rebuild is formed exactly from fixed-point positions and stored in FP32, with the neighbour's
// index in its fourth word, so that the per-step format reads one 16-byte entry.
__global__ void __launch_bounds__(32 * kVerletWarps) k_verlet(VerletArgs a) {
  __shared__ int cnt[kVerletWarps][kMaxTypes];
  __shared__ int s_beg[kVerletWarps][32], s_off[kVerletWarps][32], s_img[kVerletWarps][32];
  __shared__ float s_sh[kVerletWarps][32][3];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nwork = a.work ? *a.work_n : a.N;
  for (int wi = blockIdx.x * kVerletWarps + w; wi < nwork; wi += gridDim.x * kVerletWarps) {
  const int i = a.work ? a.work[wi] : wi;
  __syncwarp();
  if (lane < kMaxTypes) cnt[w][lane] = 0;
  __syncwarp();
  const RepGeom& g = a.geom[a.irep[i]];
  const qvec4 qi = a.xq[i];
  const float4 xfi = a.xf[i];
  const int cid = a.cell_of[i];
  const int rel = cid - g.cell_off;
  const int ci[3] = {rel / (g.nc[1] * g.nc[2]), (rel / g.nc[2]) % g.nc[1], rel % g.nc[2]};
  const unsigned lt = (1u << lane) - 1u;
  const int sy = 2 * g.m[1] + 1, sz = 2 * g.m[2] + 1;
  const int ncell = (2 * g.m[0] + 1) * sy * sz;
  const int self_code = pack_img(0, 0, 0);
  const size_t ebase = (size_t)i * a.VS;

  auto fetch = [&](int q, int total, int nb, bool& acc, int& j, int& tj, int& code) {
    acc = false; j = -1; tj = 0; code = 0;
    if (q >= total) return;
    int lo = 0, hi = nb - 1;  // the batch cell holding flat index q
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_off[w][mid] <= q) lo = mid; else hi = mid - 1;
    }
    const int idx = s_beg[w][lo] + q - s_off[w][lo];
    j = a.cell_atoms[idx];
    const float4 xfj = a.cell_xf[idx];
    code = s_img[w][lo];
    if (j == i && code == self_code) return;
    const float dx = (xfj.x + s_sh[w][lo][0]) - xfi.x;
    const float dy = (xfj.y + s_sh[w][lo][1]) - xfi.y;
    const float dz = (xfj.z + s_sh[w][lo][2]) - xfi.z;
    acc = dx * dx + dy * dy + dz * dz < a.rcs2_hi;
    tj = __float_as_int(xfj.w);
  };
  auto append = [&](bool acc, int j, int tj, int code) {
    for (int t = 0; t < a.ntypes; ++t) {
      const unsigned mask = __ballot_sync(0xffffffffu, acc && tj == t);
      if (mask == 0u) continue;
      const int start = cnt[w][t];
      if (acc && tj == t) {
        const int pos = start + __popc(mask & lt);
        if (pos < a.vcap[t]) {
          int n0, n1, n2;
          unpack_img(code, n0, n1, n2);
          const qvec4 qj = a.xq[j];
          const size_t e = ebase + a.vcap_off[t] + pos;
          a.vl_img[e] = code;
          long long shq[3];
          if (!g.tri) {
            shq[0] = (long long)n0 * g.Hq[0];
            shq[1] = (long long)n1 * g.Hq[4];
            shq[2] = (long long)n2 * g.Hq[8];
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c)
              shq[c] = (long long)n0 * g.Hq[c] + (long long)n1 * g.Hq[3 + c] + (long long)n2 * g.Hq[6 + c];
          }
          a.vl_e[e] = make_float4(fixed_diff(qj.x, qi.x, shq[0]), fixed_diff(qj.y, qi.y, shq[1]),
                                  fixed_diff(qj.z, qi.z, shq[2]), __int_as_float(j));
        }
      }
      __syncwarp();
      if (lane == 0) cnt[w][t] = start + __popc(mask);
      __syncwarp();
    }
  };

  for (int cb = 0; cb < ncell; cb += 32) {
    const int k = cb + lane;
    int beg = 0, num = 0, code = 0;
    float sh[3] = {0.f, 0.f, 0.f};
    if (k < ncell) {
      const int o[3] = {k / (sy * sz) - g.m[0], (k / sz) % sy - g.m[1], k % sz - g.m[2]};
      int n[3], cc[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int v = ci[q] + o[q];
        n[q] = floor_div(v, g.nc[q]);
        cc[q] = v - n[q] * g.nc[q];
      }
#pragma unroll
      for (int q = 0; q < 3; ++q)
        sh[q] = ((float)n[0] * g.Hf[q] + (float)n[1] * g.Hf[3 + q]) + (float)n[2] * g.Hf[6 + q];
      const int c = g.cell_off + (cc[0] * g.nc[1] + cc[1]) * g.nc[2] + cc[2];
      beg = a.cell_start[c];
      num = a.cell_start[c + 1] - beg;
      code = pack_img(n[0], n[1], n[2]);
    }
    int incl = num;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    s_beg[w][lane] = beg;
    s_off[w][lane] = incl - num;
    s_img[w][lane] = code;
    s_sh[w][lane][0] = sh[0]; s_sh[w][lane][1] = sh[1]; s_sh[w][lane][2] = sh[2];
    __syncwarp();
    const int nb = min(32, ncell - cb);
    for (int base = 0; base < total; base += 128) {
      bool acc[4];
      int jj[4], tt[4], cc[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) fetch(base + 32 * h + lane, total, nb, acc[h], jj[h], tt[h], cc[h]);
#pragma unroll
      for (int h = 0; h < 4; ++h) append(acc[h], jj[h], tt[h], cc[h]);
    }
    __syncwarp();
  }
  __syncwarp();
  if (lane < a.ntypes) {
    int nt_ = cnt[w][lane];
    if (nt_ > a.vcap[lane]) {
      set_err(a.err, ERR_VCAP);
      nt_ = a.vcap[lane];
    }
    a.vcount[(size_t)i * a.ntypes + lane] = nt_;
  }
  }  // atoms of the work list
}

// Verlet list by cell: one CTA per cell stages the candidates of the cell's whole stencil in
// shared memory once (index, position plus image shift, stencil slot), and each of its warps
// tests one of the cell's atoms against them, with the same FP32 test and image codes as
// k_verlet.  A cell's atoms share one stencil, so its candidates are read from L2 once per cell
// instead of once per atom.  Accepted candidates go to a per-warp queue with their list slots;
// the exact pair vectors (an L2 gather of the fixed-point position and integer arithmetic) are
// formed 32 at a time from the queue, with every lane busy, instead of in the test loop where a
// quarter of the lanes or fewer accept.  Cells whose stencil has more than kMaxStencil cells or
// more than kCellCap candidates (small, sparse or triclinic boxes) hand their atoms to k_verlet.
constexpr int kCellWarps = 8;
constexpr int kCellCap = 2048;
constexpr int kMaxStencil = 125;
constexpr int kQueue = 64;
constexpr size_t kCellSmem = (size_t)kCellCap * (sizeof(float4) + sizeof(int));

__global__ void __launch_bounds__(32 * kCellWarps) k_verlet_cell(VerletArgs a) {
  extern __shared__ float4 s_cx[];                      // [kCellCap] position + shift, w = type | stencil slot << 8
  int* s_cj = reinterpret_cast<int*>(s_cx + kCellCap);  // [kCellCap] atom
  __shared__ int s_beg[kMaxStencil], s_off[kMaxStencil + 1], s_code[kMaxStencil];
  __shared__ float s_sh[kMaxStencil][3];
  __shared__ long long s_shq[kMaxStencil][3];
  __shared__ int s_wsum[kCellWarps], s_total, s_wbase;
  __shared__ int s_qj[kCellWarps][kQueue], s_qe[kCellWarps][kQueue];  // queue: atom, slot in the row
  __shared__ unsigned char s_qk[kCellWarps][kQueue];                  // queue: stencil slot
  const int cid = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int cb = a.cell_start[cid], ce = a.cell_start[cid + 1];
  if (cb == ce) return;
  // the cell's atoms go to k_verlet's work list (a decision the whole CTA takes together)
  auto hand_over = [&]() {
    if (t == 0) s_wbase = atomicAdd(a.work_n, ce - cb);
    __syncthreads();
    for (int q = t; q < ce - cb; q += 32 * kCellWarps) a.work[s_wbase + q] = a.cell_atoms[cb + q];
  };
  const RepGeom& g = a.geom[a.irep[a.cell_atoms[cb]]];
  const int sy = 2 * g.m[1] + 1, sz = 2 * g.m[2] + 1;
  const int ncell = (2 * g.m[0] + 1) * sy * sz;
  if (ncell > kMaxStencil) {
    hand_over();
    return;
  }
  // the slot of offset (0, 0, 0): the only one with image (0, 0, 0) and this very cell, so a
  // candidate is the centre itself exactly when it is atom i in this slot
  const int kc = (g.m[0] * sy + g.m[1]) * sz + g.m[2];
  const int rel = cid - g.cell_off;
  const int ci[3] = {rel / (g.nc[1] * g.nc[2]), (rel / g.nc[2]) % g.nc[1], rel % g.nc[2]};
  int num = 0;
  if (t < ncell) {
    const int o[3] = {t / (sy * sz) - g.m[0], (t / sz) % sy - g.m[1], t % sz - g.m[2]};
    int n[3], cc[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int v = ci[q] + o[q];
      n[q] = floor_div(v, g.nc[q]);
      cc[q] = v - n[q] * g.nc[q];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      s_sh[t][q] = ((float)n[0] * g.Hf[q] + (float)n[1] * g.Hf[3 + q]) + (float)n[2] * g.Hf[6 + q];
      s_shq[t][q] = g.tri ? (long long)n[0] * g.Hq[q] + (long long)n[1] * g.Hq[3 + q] + (long long)n[2] * g.Hq[6 + q]
                          : (long long)n[q] * g.Hq[4 * q];
    }
    const int c = g.cell_off + (cc[0] * g.nc[1] + cc[1]) * g.nc[2] + cc[2];
    s_beg[t] = a.cell_start[c];
    num = a.cell_start[c + 1] - s_beg[t];
    s_code[t] = pack_img(n[0], n[1], n[2]);
  }
  // exclusive prefix of the stencil cells' sizes (ncell <= 125 < 32 * kCellWarps)
  int incl = num;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_wsum[w] = incl;
  __syncthreads();
  int base = 0;
  for (int u = 0; u < w; ++u) base += s_wsum[u];
  if (t < ncell) s_off[t] = base + incl - num;
  if (t == 32 * kCellWarps - 1) s_total = base + incl;
  __syncthreads();
  const int T = s_total;
  if (T > kCellCap) {
    hand_over();
    return;
  }
  if (t == 0) s_off[ncell] = T;
  // staging: four candidates per thread per pass, their loads issued together
  constexpr int kSt = 4;
  for (int q0 = t; q0 < T; q0 += kSt * 32 * kCellWarps) {
    int idx[kSt], slot[kSt];
#pragma unroll
    for (int u = 0; u < kSt; ++u) {
      const int q = q0 + u * 32 * kCellWarps;
      idx[u] = 0;
      slot[u] = 0;
      if (q < T) {
        int lo = 0, hi = ncell - 1;  // the stencil slot holding candidate q
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_off[mid] <= q) lo = mid; else hi = mid - 1;
        }
        slot[u] = lo;
        idx[u] = s_beg[lo] + q - s_off[lo];
      }
    }
    float4 xf[kSt];
    int ja[kSt];
#pragma unroll
    for (int u = 0; u < kSt; ++u) {
      const bool in = q0 + u * 32 * kCellWarps < T;
      xf[u] = in ? a.cell_xf[idx[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
      ja[u] = in ? a.cell_atoms[idx[u]] : 0;
    }
#pragma unroll
    for (int u = 0; u < kSt; ++u) {
      const int q = q0 + u * 32 * kCellWarps;
      if (q < T) {
        const int k = slot[u];
        s_cx[q] = make_float4(xf[u].x + s_sh[k][0], xf[u].y + s_sh[k][1], xf[u].z + s_sh[k][2],
                              __int_as_float(__float_as_int(xf[u].w) | (k << 8)));
        s_cj[q] = ja[u];
      }
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  for (int ca = cb + w; ca < ce; ca += kCellWarps) {
    const int i = a.cell_atoms[ca];
    const float4 xfi = a.xf[i];
    const qvec4 qi = a.xq[i];
    const size_t ebase = (size_t)i * a.VS;
    // the queued entries [0, qn): exact pair vectors and the list writes, one entry per lane
    auto drain = [&](int qn) {
      __syncwarp();
      if (lane < qn) {
        const int j = s_qj[w][lane], k = s_qk[w][lane];
        const size_t e = ebase + s_qe[w][lane];
        const qvec4 qj = a.xq[j];
        a.vl_img[e] = s_code[k];
        a.vl_e[e] = make_float4(fixed_diff(qj.x, qi.x, s_shq[k][0]), fixed_diff(qj.y, qi.y, s_shq[k][1]),
                                fixed_diff(qj.z, qi.z, s_shq[k][2]), __int_as_float(j));
      }
      __syncwarp();
    };
    int cnt[kMaxTypes] = {0, 0, 0, 0};  // the same in every lane
    int qn = 0;                         // queue fill, the same in every lane
    // the next batch's candidate is read from shared memory one pass ahead
    float4 c4n = lane < T ? s_cx[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    int jn = lane < T ? s_cj[lane] : -1;
    for (int b = 0; b < T; b += 32) {
      const int q = b + lane;
      const float4 c4 = c4n;
      const int j = jn;
      if (q + 32 < T) {
        c4n = s_cx[q + 32];
        jn = s_cj[q + 32];
      }
      bool acc = false;
      int tj = 0, k = 0;
      if (q < T) {
        const int wk = __float_as_int(c4.w);
        k = wk >> 8;
        if (!(j == i && k == kc)) {
          const float dx = c4.x - xfi.x, dy = c4.y - xfi.y, dz = c4.z - xfi.z;
          acc = dx * dx + dy * dy + dz * dz < a.rcs2_hi;
          tj = wk & 0xff;
        }
      }
      int off = -1;  // this lane's slot in the row (vcap_off + position), -1: none
#pragma unroll
      for (int tt = 0; tt < kMaxTypes; ++tt) {
        if (tt >= a.ntypes) break;
        const unsigned mask = __ballot_sync(0xffffffffu, acc && tj == tt);
        if (acc && tj == tt) {
          const int pos = cnt[tt] + __popc(mask & lt);
          if (pos < a.vcap[tt]) off = a.vcap_off[tt] + pos;
        }
        cnt[tt] += __popc(mask);
      }
      const unsigned qm = __ballot_sync(0xffffffffu, off >= 0);
      if (off >= 0) {
        const int qs = qn + __popc(qm & lt);
        s_qj[w][qs] = j;
        s_qk[w][qs] = (unsigned char)k;
        s_qe[w][qs] = off;
      }
      qn += __popc(qm);
      if (qn >= 32) {
        drain(32);
        // move the rest (fewer than 32) to the front
        int rj = 0, re = 0, rk = 0;
        if (lane < qn - 32) { rj = s_qj[w][32 + lane]; re = s_qe[w][32 + lane]; rk = s_qk[w][32 + lane]; }
        __syncwarp();
        if (lane < qn - 32) { s_qj[w][lane] = rj; s_qe[w][lane] = re; s_qk[w][lane] = (unsigned char)rk; }
        qn -= 32;
      }
    }
    drain(qn);
#pragma unroll
    for (int tt = 0; tt < kMaxTypes; ++tt)
      if (lane == tt && tt < a.ntypes) {
        int nt_ = cnt[tt];
        if (nt_ > a.vcap[tt]) {
          set_err(a.err, ERR_VCAP);
          nt_ = a.vcap[tt];
        }
        a.vcount[(size_t)i * a.ntypes + tt] = nt_;
      }
  }
}

// ------------------------------------------------------------------ per-step
__global__ void k_delta(int N, const dvec4* __restrict__ x, const dvec4* __restrict__ xref, float4* delta,
                        double lim2, int* err) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  dvec4 p = x[k], q = xref[k];
  double dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
  delta[k] = make_float4((float)dx, (float)dy, (float)dz, 0.f);
  if (dx * dx + dy * dy + dz * dz > lim2) set_err(err, ERR_SKIN);
}

struct FormatArgs {
  int N, ntypes, VS, S;
  int vcap_off[kMaxTypes + 1];
  int sel[kMaxTypes], sel_off[kMaxTypes + 1];
  double rc2;
  float rc2_lo, rc2_hi;
  const int* irep;
  const int* perm;             // internal -> caller index (truncation tie-break)
  const RepGeom* geom;
  const dvec4* x;
  const float4* delta;
  const float4* vl_e;
  const int* vl_img;
  const int* vcount;
  int* nl_j;
  int* nl_img;                 // null: image codes not written (only the test hook reads them)
  void* nl_d;
  int* nl_count;
  int* err;
};

// Nearest-first truncation of one overflowing (atom i, type t) segment by its warp: every
// Verlet entry within r_c is ranked by (exact FP64 r^2, caller index of j, image code), the same
// order the neighbour list's canonical key uses for ties; the sel_t entries of rank < sel_t are
// written in Verlet order.  O(n^2 / 32) per lane, taken only when the segment overflows.
template <bool kFP64>
__device__ int keep_nearest(const FormatArgs& a, const RepGeom& g, const dvec4& xi, const float4& di, int n,
                            size_t vb, size_t ob, int sel, int lane) {
  const unsigned lt = (1u << lane) - 1u;
  int kept = 0;
  for (int b = 0; b < n; b += 32) {
    const int q = b + lane;
    bool in = false;
    double r2 = 0.0, dd[3] = {0.0, 0.0, 0.0};
    unsigned long long tie = 0;
    int j = 0, code = 0;
    if (q < n) {
      j = __float_as_int(a.vl_e[vb + q].w);
      code = a.vl_img[vb + q];
      int n0, n1, n2;
      unpack_img(code, n0, n1, n2);
      r2 = exact_r2(xi, a.x[j], n0, n1, n2, g, dd);
      in = r2 < a.rc2;
      tie = ((unsigned long long)(unsigned)a.perm[j] << 32) | (unsigned)code;
    }
    int rank = 0;
    for (int c = 0; c < n; c += 32) {
      const int p = c + lane;
      int pin = 0;
      double pr2 = 0.0, pd[3];
      unsigned long long ptie = 0;
      if (p < n) {
        const int pj = __float_as_int(a.vl_e[vb + p].w), pcode = a.vl_img[vb + p];
        int m0, m1, m2;
        unpack_img(pcode, m0, m1, m2);
        pr2 = exact_r2(xi, a.x[pj], m0, m1, m2, g, pd);
        pin = pr2 < a.rc2;
        ptie = ((unsigned long long)(unsigned)a.perm[pj] << 32) | (unsigned)pcode;
      }
      for (int s = 0; s < 32; ++s) {
        const double r2s = __shfl_sync(0xffffffffu, pr2, s);
        const unsigned long long ties = __shfl_sync(0xffffffffu, ptie, s);
        const int ins = __shfl_sync(0xffffffffu, pin, s);
        if (ins && (r2s < r2 || (r2s == r2 && ties < tie))) ++rank;
      }
    }
    const bool keep = in && rank < sel;
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    const int pos = kept + __popc(mask & lt);
    if (keep) {
      a.nl_j[ob + pos] = j;
      if (a.nl_img) a.nl_img[ob + pos] = code;
      if (kFP64) {
        static_cast<dvec4*>(a.nl_d)[ob + pos] = make_dvec4(dd[0], dd[1], dd[2], 0.0);
      } else {
        const float4 d0 = a.vl_e[vb + q];
        const float4 dj = a.delta[j];
        static_cast<float4*>(a.nl_d)[ob + pos] =
            make_float4(d0.x + (dj.x - di.x), d0.y + (dj.y - di.y), d0.z + (dj.z - di.z), 0.f);
      }
    }
    kept += __popc(mask);
  }
  return kept;
}

// kNearest selects the overflow policy at compile time, so the default (error) variant carries
// none of the selection's registers.
template <bool kFP64, bool kNearest>
__global__ void __launch_bounds__(128) k_format(FormatArgs a) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= a.N) return;
  const unsigned lt = (1u << lane) - 1u;
  const RepGeom& g = a.geom[a.irep[i]];
  const dvec4 xi = a.x[i];
  const float4 di = a.delta[i];
  for (int t = 0; t < a.ntypes; ++t) {
    const int n = a.vcount[(size_t)i * a.ntypes + t];
    const size_t vb = (size_t)i * a.VS + a.vcap_off[t];
    const size_t ob = (size_t)i * a.S + a.sel_off[t];
    int cnt = 0;
    if (kFP64) {
      for (int b = 0; b < n; b += 32) {
        const int q = b + lane;
        bool in = false;
        int j = 0, code = 0;
        double dd[3];
        if (q < n) {
          j = __float_as_int(a.vl_e[vb + q].w);
          code = a.vl_img[vb + q];
          int n0, n1, n2;
          unpack_img(code, n0, n1, n2);
          in = exact_r2(xi, a.x[j], n0, n1, n2, g, dd) < a.rc2;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, in);
        const int pos = cnt + __popc(mask & lt);
        if (in && pos < a.sel[t]) {
          a.nl_j[ob + pos] = j;
          if (a.nl_img) a.nl_img[ob + pos] = code;
          static_cast<dvec4*>(a.nl_d)[ob + pos] = make_dvec4(dd[0], dd[1], dd[2], 0.0);
        }
        cnt += __popc(mask);
      }
    } else {
      // Pipeline over the 32-entry batches: the entries of batches b + 1 .. b + 3 and the
      // neighbours' displacements of batch b + 1 are in flight while batch b is filtered.
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      float4 e0 = lane < n ? a.vl_e[vb + lane] : z4;
      float4 e1 = lane + 32 < n ? a.vl_e[vb + 32 + lane] : z4;
      float4 e2 = lane + 64 < n ? a.vl_e[vb + 64 + lane] : z4;
      float4 dj0 = lane < n ? a.delta[__float_as_int(e0.w)] : z4;
      for (int b = 0; b < n; b += 32) {
        const int q = b + lane;
        const float4 dj1 = q + 32 < n ? a.delta[__float_as_int(e1.w)] : z4;
        const float4 e3 = q + 96 < n ? a.vl_e[vb + q + 96] : z4;
        bool in = false;
        const int j = __float_as_int(e0.w);
        const float dfx = e0.x + (dj0.x - di.x), dfy = e0.y + (dj0.y - di.y), dfz = e0.z + (dj0.z - di.z);
        if (q < n) {
          const float r2f = dfx * dfx + dfy * dfy + dfz * dfz;
          if (r2f < a.rc2_lo) {
            in = true;
          } else if (r2f < a.rc2_hi) {
            // exact FP64 test near the cutoff: the only place the image code is read
            int n0, n1, n2;
            unpack_img(a.vl_img[vb + q], n0, n1, n2);
            double dd[3];
            in = exact_r2(a.x[i], a.x[j], n0, n1, n2, g, dd) < a.rc2;  // x_i re-read: fewer live registers
          }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, in);
        const int pos = cnt + __popc(mask & lt);
        if (in && pos < a.sel[t]) {
          a.nl_j[ob + pos] = j;
          if (a.nl_img) a.nl_img[ob + pos] = a.vl_img[vb + q];
          static_cast<float4*>(a.nl_d)[ob + pos] = make_float4(dfx, dfy, dfz, 0.f);
        }
        cnt += __popc(mask);
        e0 = e1;
        e1 = e2;
        e2 = e3;
        dj0 = dj1;
      }
    }
    if (cnt > a.sel[t]) {
      if (kNearest) {
        cnt = keep_nearest<kFP64>(a, g, xi, di, n, vb, ob, a.sel[t], lane);
      } else {
        if (lane == 0) set_err(a.err, ERR_SEL);
        cnt = a.sel[t];
      }
    }
    if (lane == 0) a.nl_count[(size_t)i * a.ntypes + t] = cnt;
  }
}

// Canonical copy of the formatted list for the caller: rows in the caller's atom order, each
// neighbour-type segment sorted by (caller index j, image nx, ny, nz), padded with -1 / 0.
// One CTA per atom; keys sorted in shared memory (bitonic).  A test hook, not on the MD path.
__global__ void k_get_nlist(int N, int ntypes, int S, const int* sel, const int* sel_off, const int* inv,
                            const int* perm, const int* nl_j, const int* nl_img, const int* nl_count,
                            int* out_nl, int* out_img) {
  extern __shared__ unsigned long long keys[];
  const int u = blockIdx.x;
  if (u >= N) return;
  const int i = inv[u];
  for (int t = 0; t < ntypes; ++t) {
    const int c = nl_count[(size_t)i * ntypes + t];
    int P = 1;
    while (P < c) P <<= 1;
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
      const size_t src = (size_t)i * S + sel_off[t] + q;
      keys[q] = (q < c) ? (((unsigned long long)(unsigned)perm[nl_j[src]] << 32) | (unsigned)nl_img[src])
                        : ~0ull;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
      for (int jj = k >> 1; jj > 0; jj >>= 1) {
        for (int q = threadIdx.x; q < P; q += blockDim.x) {
          const int p = q ^ jj;
          if (p > q) {
            const unsigned long long k0 = keys[q], k1 = keys[p];
            if ((k0 > k1) == ((q & k) == 0)) { keys[q] = k1; keys[p] = k0; }
          }
        }
        __syncthreads();
      }
    for (int q = threadIdx.x; q < sel[t]; q += blockDim.x) {
      const size_t dst = (size_t)u * S + sel_off[t] + q;
      out_nl[dst] = (q < c) ? (int)(keys[q] >> 32) : -1;
      out_img[dst] = (q < c) ? (int)(keys[q] & 0xffffffffu) : 0;
    }
    __syncthreads();
  }
}

}  // namespace

// ====================================================================== launchers
dp_status launch_type_sort(Model* m, const int* types_user, int N) {
  int nblk = cdiv(N, kSortBlock);
  k_type_count<<<nblk, kSortBlock, 0, m->stream>>>(types_user, N, m->ntypes, m->blk_count, m->err);
  k_type_scan<<<1, 32, 0, m->stream>>>(nblk, m->ntypes, m->blk_count, m->type_count, m->type_off);
  k_type_scatter<<<nblk, kSortBlock, 0, m->stream>>>(types_user, N, m->ntypes, m->blk_count, m->rep_off_dev,
                                                     m->nrep, m->perm, m->inv, m->itype, m->irep);
  m->launches += 3;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_load_positions(Model* m, const double* coords_user, int N) {
  k_load_positions<<<cdiv(N, 256), 256, 0, m->stream>>>(coords_user, m->perm, N, m->x);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

// Largest |x| a wrapped coordinate or a single-cell shift can have: max over rows of sum |H_ac|.
static double max_box_length(const Model* m) {
  double Lmax = 0;
  for (int r = 0; r < m->nrep; ++r)
    for (int a = 0; a < 3; ++a) {
      const double* h = m->geom_host[r].H + 3 * a;
      const double v = std::fabs(h[0]) + std::fabs(h[1]) + std::fabs(h[2]);
      Lmax = Lmax > v ? Lmax : v;
    }
  return Lmax;
}

dp_status launch_rebuild(Model* m, int N, bool with_skin) {
  cudaStream_t s = m->stream;
  DP_CUDA_TRY(m, cudaMemsetAsync(m->cell_count, 0, sizeof(int) * m->ncells, s));
  DP_CUDA_TRY(m, cudaMemsetAsync(m->cell_fill, 0, sizeof(int) * m->ncells, s));
  k_wrap_bin<<<cdiv(N, 256), 256, 0, s>>>(N, m->irep, m->itype, m->geom, m->x, m->xref, m->xf, m->xq,
                                          m->delta, m->cell_of, m->cell_count);
  k_scan_cells<<<1, 1024, 0, s>>>(m->ncells, m->cell_count, m->cell_start);
  k_fill_cells<<<cdiv(N, 256), 256, 0, s>>>(N, m->cell_of, m->cell_start, m->xf, m->cell_fill, m->cell_atoms,
                                            m->cell_xf);
  VerletArgs a;
  a.N = N; a.ntypes = m->ntypes; a.VS = m->VS;
  for (int t = 0; t < m->ntypes; ++t) {
    a.vcap[t] = m->vcap[t];
    a.vcap_off[t] = m->vcap_off[t];
  }
  a.vcap_off[m->ntypes] = m->vcap_off[m->ntypes];
  const double rcs = m->rc + (with_skin ? m->skin : 0.0);
  a.rcs2 = rcs * rcs;
  // worst-case FP32 error of the prefilter's r^2 is ~1.3e-6 * rcs * Lmax; use 10x that
  double band = 1.25e-5 * rcs * (max_box_length(m) + rcs) + 1e-3;
  a.rcs2_hi = (float)(a.rcs2 + band);
  a.itype = m->itype; a.irep = m->irep; a.geom = m->geom; a.x = m->x; a.xf = m->xf; a.xq = m->xq;
  a.cell_of = m->cell_of; a.cell_start = m->cell_start; a.cell_atoms = m->cell_atoms; a.cell_xf = m->cell_xf;
  a.vl_e = m->vl_e; a.vl_img = m->vl_img; a.vcount = m->vcount; a.err = m->err;
  // cells by k_verlet_cell; the atoms of the cells it hands over by k_verlet, whose grid-stride
  // loop over the work list costs little when the list is empty
  a.work = m->vl_work;
  a.work_n = m->vl_work + m->max_atoms;
  DP_CUDA_TRY(m, cudaMemsetAsync(a.work_n, 0, sizeof(int), s));
  DP_CUDA_TRY(m, ensure_smem(reinterpret_cast<const void*>(k_verlet_cell), kCellSmem));
  k_verlet_cell<<<m->ncells, 32 * kCellWarps, kCellSmem, s>>>(a);
  k_verlet<<<std::min(cdiv(N, kVerletWarps), 8 * num_sms()), 32 * kVerletWarps, 0, s>>>(a);
  m->launches += 5;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_delta(Model* m, int N) {
  double h = 0.5 * m->skin;
  k_delta<<<cdiv(N, 256), 256, 0, m->stream>>>(N, m->x, m->xref, m->delta, h * h, m->err);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_format(Model* m, int N, bool images) {
  FormatArgs a;
  a.N = N; a.ntypes = m->ntypes; a.VS = m->VS; a.S = m->S;
  for (int t = 0; t <= m->ntypes; ++t) { a.vcap_off[t] = m->vcap_off[t]; a.sel_off[t] = m->sel_off[t]; }
  for (int t = 0; t < m->ntypes; ++t) a.sel[t] = m->sel[t];
  a.rc2 = m->rc * m->rc;
  // FP32 pair vector d0 + (delta_j - delta_i) is within ~2e-7 (rc + skin + 2) per component
  // of the exact one; the r^2 error is below 1e-6 rc (rc + skin + 2).  Band: 100x.
  double band = 1e-4 * m->rc * (m->rc + m->skin + 2.0) + 1e-4;
  a.rc2_lo = (float)(a.rc2 - band);
  a.rc2_hi = (float)(a.rc2 + band);
  a.irep = m->irep; a.perm = m->perm; a.geom = m->geom; a.x = m->x; a.delta = m->delta;
  a.vl_e = m->vl_e; a.vl_img = m->vl_img; a.vcount = m->vcount;
  a.nl_j = m->nl_j; a.nl_img = images ? m->nl_img : nullptr; a.nl_d = m->nl_d; a.nl_count = m->nl_count;
  a.err = m->err;
  const dim3 grid(cdiv(N, 4));
  if (m->prec == DP_FP64) {
    if (m->nearest) k_format<true, true><<<grid, 128, 0, m->stream>>>(a);
    else k_format<true, false><<<grid, 128, 0, m->stream>>>(a);
  } else {
    if (m->nearest) k_format<false, true><<<grid, 128, 0, m->stream>>>(a);
    else k_format<false, false><<<grid, 128, 0, m->stream>>>(a);
  }
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_get_nlist(Model* m, int N, int* nlist, int* images) {
  int* dsel = m->small_i;
  int hsel[2 * kMaxTypes + 1];
  for (int t = 0; t < m->ntypes; ++t) hsel[t] = m->sel[t];
  for (int t = 0; t <= m->ntypes; ++t) hsel[kMaxTypes + t] = m->sel_off[t];
  DP_CUDA_TRY(m, cudaMemcpyAsync(dsel, hsel, sizeof(hsel), cudaMemcpyHostToDevice, m->stream));
  int Pmax = 1;
  for (int t = 0; t < m->ntypes; ++t)
    while (Pmax < m->sel[t]) Pmax <<= 1;
  const size_t ksm = sizeof(unsigned long long) * (size_t)Pmax;
  DP_CUDA_TRY(m, ensure_smem(reinterpret_cast<const void*>(k_get_nlist), ksm));
  k_get_nlist<<<N, 128, ksm, m->stream>>>(N, m->ntypes, m->S, dsel, dsel + kMaxTypes, m->inv, m->perm, m->nl_j,
                                          m->nl_img, m->nl_count, nlist, images);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

}  // namespace dpg
