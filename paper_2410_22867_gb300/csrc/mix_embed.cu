// Mixed-precision embedding net, descriptor and embedding backward on the
// tensor cores (tcgen05 / TMEM), Section III-B3's mixed precision mapped to
// Blackwell: the 25->50 and 50->100 layers of the embedding net (and their
// backward) are MMAs with 16-bit operands and FP32 accumulation in TMEM; the
// environment matrix, the 1->25 layer, all tanh (on the SFU) and residuals stay
// FP32 on the CUDA cores.  The reduction T = R_hat^T G of the descriptor (Section II-A) is a third MMA
// per tile with fp16 operands: G^T [feature][row] against a block-sparse R_hat^T
// whose column (atom slot, c) is non-zero only on that atom's rows, so one
// 128x32x128 product yields the partial T of every atom in the tile.
//
// Work decomposition.  For each neighbour type tj the real neighbours of all
// atoms form one "row stream" (atoms in internal, type-sorted order; rows of an
// atom contiguous).  The concatenated streams are split into one contiguous chunk
// per CTA, walked in tiles of at most 128 rows (one row per thread and TMEM lane)
// that never cross a centre-type boundary and hold at most kMaxAtoms atoms.  The
// partial T of an atom that continues into the next tile stays in registers
// (thread = feature) and is written once the atom is complete; only atoms split
// between two CTAs use global atomics.  Activations of the embedding net are
// recomputed in the backward instead of being stored.
//
// Latency.  Both kernels run 3 CTAs of 4 warps per SM.  Thread 0 issues the MMAs; warp 1
// locates the next tile while the last product of a tile runs, and the tile's data (rows
// by per-thread cp.async, dE/dT by one bulk copy) arrive in shared memory before it starts.
#include "tc_common.cuh"

namespace dpg {
namespace {

constexpr int kRows = 128;     // rows per tile = threads per CTA = TMEM lanes
constexpr int kMaxAtoms = 4;   // atom segments per tile (columns (atom, c) of the T product: 16)
constexpr uint32_t kTmemCols = 128;  // per CTA: D2/D3 share columns 0..111
constexpr int kLocWarp = 1;    // the warp that locates tiles (thread 0 issues the MMAs)

struct MixArgs {
  int N, ntypes, S;
  int sel_off[kMaxTypes + 1];
  float rc, rs, invS;
  int switch_kind;
  const float* w;        // theta (fp32)
  const float* stat;     // davg [nt][4], 1/dstd [nt][4]
  const int* itype;
  const int* type_off;   // device [nt + 1]
  const int* rowoff;     // [nt][N + 1] exclusive scan of nl_count over atoms, per neighbour type
  const int* nl_j;
  const float4* nl_d;
  float* Tseg;           // [nt][N][400] partial T per neighbour type
  const float4* dT;      // [N][100]: dE/dT[c][a] * (1/S), c in x..w
  double* force;         // [N][3]
  float* force32;        // [N][4] FP32 accumulator, x y z and a pad (folded into force after the backward)
  double* vir_atom;      // [N][9] (unused by the mixed backward)
  double* vir_rep;       // [nrep][9] per-replica virial
  const int* irep;       // [N] replica of each internal atom
  const unsigned char* img;  // per pair: the operand blocks of load_fwd_weights / load_bwd_ops
  const float4* tab;     // tabulated embedding: [pair][interval][100][2] float4 quintic coefficients
  int tab_n;
  float tab_x0, tab_ih;  // first node, 1 / interval width
  int* err;
};

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  uint32_t a = tc::smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// Smooth switch sw(r) and its derivative; winv = 1 / (rc - rs).
__device__ __forceinline__ void switch_fn(float r, float rs, float rc, float winv, int kind, float& sw, float& dsw) {
  if (r < rs) { sw = 1.f; dsw = 0.f; return; }
  if (r >= rc) { sw = 0.f; dsw = 0.f; return; }
  const float u = (r - rs) * winv;
  if (kind == 1) {
    const float pi = 3.14159265358979323846f;
    sw = 0.5f * cosf(pi * u) + 0.5f;
    dsw = -0.5f * pi * sinf(pi * u) * winv;
  } else {
    const float u2 = u * u;
    sw = u2 * u * (-6.f * u2 + 15.f * u - 10.f) + 1.f;
    dsw = -30.f * u2 * (u - 1.f) * (u - 1.f) * winv;
  }
}

// Shared state of a tile walk.
struct TileInfo {
  int tj, ti, p, nrows, a0, cs, ce;  // stream, centre type, first row (stream coords), rows, first atom, chunk
  // for the forward's write-out: slot of the tile's last atom, whether the tile completes it,
  // and the slots whose atom starts before or ends after this CTA's chunk
  int last_la, last_done, shared_mask;
};

// Walk state of one CTA over the concatenated streams (held uniformly by the locating warp).
struct Walk {
  int tj, base, hint;  // current stream, its first row in concatenated coordinates, atom at or before the tile
};

// Per-CTA tables: tot[tj] rows of stream tj; tiend[tj * nt + ti] end row of centre type ti in stream tj.
__device__ void walk_tables(const MixArgs& a, int* tot, int* tiend) {
  if (threadIdx.x == 0) {
    for (int tj = 0; tj < a.ntypes; ++tj) {
      const int* ro = a.rowoff + (size_t)tj * (a.N + 1);
      tot[tj] = ro[a.N];
      for (int ti = 0; ti < a.ntypes; ++ti) tiend[tj * a.ntypes + ti] = ro[a.type_off[ti + 1]];
    }
  }
}

// The locating warp, at the start of a tile: enters the stream of the next tile (starting at
// global row `next`) and starts the copy of the 32 row offsets from the hint atom into sWin
// (lane l copies entry l).  locate_tile reads them much later in the tile, so the copy's
// latency is hidden and no register waits for it.
__device__ __forceinline__ void locate_window(const MixArgs& a, int next, Walk& wk, const int* tot, int* sWin) {
  while (wk.tj < a.ntypes - 1 && next >= wk.base + tot[wk.tj]) {
    wk.base += tot[wk.tj];
    wk.tj += 1;
    wk.hint = -1;
  }
  if (wk.hint < 0) return;
  const int lane = threadIdx.x & 31;
  tc::cp_async4(sWin + lane, a.rowoff + (size_t)wk.tj * (a.N + 1) + min(wk.hint + lane, a.N));
}

// The locating warp finds the tile starting at global row `cur` of chunk [c0, c1).  The window
// of 32 row offsets from the hint atom (in sWin from locate_window when `have_win`) finds the
// first atom and, when it reaches far enough, the tile's atom offsets too; a binary search runs
// only when a CTA enters a stream.  With `sNat`, lane 0 also stores the tile's atom count.
__device__ __forceinline__ void locate_tile(const MixArgs& a, int cur, int c0, int c1, Walk& wk, const int* tot,
                                            const int* tiend, TileInfo* ti_out, int* sRow,
                                            const int* sWin = nullptr, bool have_win = false, int* sNat = nullptr) {
  const int lane = threadIdx.x & 31;
  while (wk.tj < a.ntypes - 1 && cur >= wk.base + tot[wk.tj]) {
    wk.base += tot[wk.tj];
    wk.tj += 1;
    wk.hint = -1;
    have_win = false;
  }
  const int tj = wk.tj;
  const int* ro = a.rowoff + (size_t)tj * (a.N + 1);
  const int p = cur - wk.base;
  int a0 = -1;
  const int hint = wk.hint;
  int v = 0;
  if (hint >= 0) {
    if (have_win) {
      tc::cp_async_wait_all();  // this lane's window entry (its only copy in flight)
      v = sWin[lane];
    } else {
      v = ro[min(hint + lane, a.N)];
    }
    const unsigned m = __ballot_sync(0xffffffffu, v <= p);  // a prefix of the lanes (offsets ascend)
    if (m != 0xffffffffu && m != 0u) a0 = hint + __popc(m) - 1;
  }
  const bool in_win = a0 >= 0 && a0 - hint + kMaxAtoms <= 31;
  if (a0 < 0) {  // largest atom i with ro[i] <= p
    int lo = 0, hi = a.N - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (ro[mid] <= p) lo = mid; else hi = mid - 1;
    }
    a0 = lo;
  }
  int ti = 0;
  while (ti < a.ntypes - 1 && p >= tiend[tj * a.ntypes + ti]) ++ti;
  // ro[min(a0 + k, N)] for k <= kMaxAtoms: lane a0 - hint + k of the window when it is there
  const int k = lane < kMaxAtoms + 1 ? lane : 0;
  int rk = __shfl_sync(0xffffffffu, v, in_win ? a0 - hint + k : 0);
  if (!in_win) rk = tc::ld_global_once(ro + min(a0 + k, a.N));
  if (lane <= kMaxAtoms) sRow[lane] = rk;
  const int r8 = __shfl_sync(0xffffffffu, rk, kMaxAtoms);
  int end = min(c1 - wk.base, tot[tj]);
  end = min(end, tiend[tj * a.ntypes + ti]);
  end = min(end, r8);
  end = min(end, p + kRows);
  // lanes 1 .. kMaxAtoms - 1 hold the offsets of the atoms after a0: the tile's last atom is the
  // last one starting before its end (also the hint for the next tile)
  const int last = a0 + __popc(__ballot_sync(0xffffffffu, lane >= 1 && lane < kMaxAtoms && rk <= end - 1));
  const int cs = c0 - wk.base, ce = c1 - wk.base;
  const int rk_next = __shfl_down_sync(0xffffffffu, rk, 1);  // ro[a0 + lane + 1]
  const unsigned shared = __ballot_sync(0xffffffffu, lane < kMaxAtoms && (rk < cs || rk_next > ce));
  const int rk_after_last = __shfl_sync(0xffffffffu, rk, last - a0 + 1);
  if (lane == 0) {
    TileInfo t;
    t.tj = tj; t.ti = ti; t.p = p; t.nrows = end - p; t.a0 = a0; t.cs = cs; t.ce = ce;
    t.last_la = last - a0;
    t.last_done = (end == rk_after_last) ? 1 : 0;
    t.shared_mask = (int)shared;
    *ti_out = t;
  }
  wk.hint = last;
  if (sNat != nullptr && lane == 0) *sNat = last - a0 + 1;
}

// dE/dT of `nat` atoms from atom a0 into sdT by one bulk copy, completing on dbar.
__device__ __forceinline__ void fetch_dT(const MixArgs& a, int a0, int nat, float4* sdT, uint64_t* dbar) {
  const uint32_t bytes = (uint32_t)nat * kN3 * 16u;
  tc::mbar_arrive_expect_tx(dbar, bytes);
  tc::bulk_load(sdT, a.dT + (size_t)a0 * kN3, bytes, dbar);
}

// The layer biases enter the tensor-core products: the A operands carry ones in the two K
// columns after the last unit, and the B blocks carry the bias split into a 16-bit head and
// the 16-bit rounding of the remainder there, so z = h W + b_hi + b_lo is accumulated in FP32
// with the bias exact to about 2^-22 relative.
template <bool F16>
__device__ __forceinline__ float split_hi(float b) {
  if (F16) return __half2float(__float2half_rn(b));
  return __bfloat162float(__float2bfloat16_rn(b));
}

// Element (k, n) of the layer-2 block: W2[k][n] (k < 25), the bias b2[n] at k = 25, 26.
template <bool F16>
__device__ __forceinline__ float w2_elem(const float* __restrict__ W, int k, int n) {
  if (n >= kN2) return 0.f;
  if (k < kN1) return W[kEW2 + k * kN2 + n];
  if (k == kN1 || k == kN1 + 1) {
    const float b = W[kEb2 + n], hi = split_hi<F16>(b);
    return k == kN1 ? hi : b - hi;
  }
  return 0.f;
}

// Element (k, f) of the layer-3 block: W3[k][f] (k < 50), the bias b3[f] at k = 50, 51.
template <bool F16>
__device__ __forceinline__ float w3_elem(const float* __restrict__ W, int k, int f) {
  if (f < 0 || f >= kN3) return 0.f;
  if (k < kN2) return W[kEW3 + k * kN3 + f];
  if (k == kN2 || k == kN2 + 1) {
    const float b = W[kEb3 + f], hi = split_hi<F16>(b);
    return k == kN2 ? hi : b - hi;
  }
  return 0.f;
}

// Layer-1 weights in FP32 for the CUDA cores (16-byte aligned slots for vector loads):
// small[0..31] = W1 (25 used), small[32..63] = b1 (25 used).
constexpr int kSmall = 64;
// Forward operand image of one embedding pair (built once per weight upload, copied into shared
// memory by three bulk copies per pair change): B2 | B3 (head, remainder) | small.
constexpr uint32_t kImgFwdB3 = 8192, kImgFwdSmall = kImgFwdB3 + 2 * 14336, kImgFwd = kImgFwdSmall + kSmall * 4;
constexpr uint32_t kImgBytes = kImgFwd;

// The three bulk copies of one operand image (B2 | B3 | small, `b3` and `sm_off` bytes in) into
// shared memory on mbarrier `bar`; issued by one thread.  Out of line: the kernels' register
// allocation stays that of their main loops.
__device__ __noinline__ void fetch_image(const unsigned char* img, uint32_t b3, uint32_t sm_off, uint32_t total,
                                         unsigned char* sB2, unsigned char* sB3, float* small, uint64_t* bar) {
  tc::mbar_arrive_expect_tx(bar, total);
  tc::bulk_load(sB2, img, b3, bar);
  tc::bulk_load(sB3, img + b3, sm_off - b3, bar);
  tc::bulk_load(small, img + sm_off, total - sm_off, bar);
}
__device__ __forceinline__ void load_small(const float* __restrict__ W, float* small) {
  for (int q = threadIdx.x; q < kSmall; q += blockDim.x)
    small[q] = (q & 31) < kN1 ? W[(q < 32 ? kEW1 : kEb1) + (q & 31)] : 0.f;
}

// The forward's weights enter the products split into a 16-bit head and the 16-bit rounding of
// the remainder: z = h W_hi + h W_lo, exact in the weights to about 2^-22 (fp16) or 2^-16 (bf16)
// relative.  With a single 16-bit copy every neighbour row would see the same rounding error,
// which does not average out in T and biases the energy (the activations' rounding differs from
// row to row and mostly does).  Layer 2: W_hi in K slots 0..31 and W_lo in 32..63 of one block,
// against [h1, 1, 1 | h1] in A (the bias rides in the head half).  Layer 3: a second B3 block.
template <bool F16>
__device__ __forceinline__ float lo_part(float w) {
  return w - split_hi<F16>(w);
}
// Element (k, n) of the split layer-2 block (k < 64).
template <bool F16>
__device__ __forceinline__ float w2_split_elem(const float* __restrict__ W, int k, int n) {
  if (k < 32) return split_hi<F16>(w2_elem<F16>(W, k, n));  // bias rows hold head and remainder already
  return (k - 32 < kN1) ? lo_part<F16>(w2_elem<F16>(W, k - 32, n)) : 0.f;
}
// Embedding weights of pair (ti, tj) into the forward's MMA operand blocks and small fp32 arrays.
//   B2: [64 x 64] rows n (layer-2 output), K slots 0..31 the 16-bit head of W2 (25 units, bias at
//       25/26), 32..56 the remainder of W2
//   B3: two [112 x 64] blocks (head, remainder), rows a (layer-3 output), K = layer-2 unit (50
//       used, bias head and remainder at 50/51 of the head block)
template <bool F16>
__device__ void load_fwd_weights(const float* __restrict__ W, unsigned char* sB2, unsigned char* sB3, float* small) {
  const int t = threadIdx.x;
  for (int q = t; q < 64 * 8; q += kRows) {
    int n = q >> 3, k0 = (q & 7) * 8;
    uint32_t p[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      int k = k0 + 2 * h;
      p[h] = tc::pack2<F16>(w2_split_elem<F16>(W, k, n), w2_split_elem<F16>(W, k + 1, n));
    }
    tc::st_chunk(sB2, n, k0, make_uint4(p[0], p[1], p[2], p[3]));
  }
  for (int q = t; q < 2 * 112 * 8; q += kRows) {
    const int part = q / (112 * 8), n = (q >> 3) % 112, k0 = (q & 7) * 8;
    uint32_t p[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      int k = k0 + 2 * h;
      float v0 = w3_elem<F16>(W, k, n), v1 = w3_elem<F16>(W, k + 1, n);
      if (part == 0) {
        v0 = split_hi<F16>(v0);
        v1 = split_hi<F16>(v1);
      } else {
        v0 = k < kN2 ? lo_part<F16>(v0) : 0.f;
        v1 = k + 1 < kN2 ? lo_part<F16>(v1) : 0.f;
      }
      p[h] = tc::pack2<F16>(v0, v1);
    }
    tc::st_chunk(sB3 + part * 14336, n, k0, make_uint4(p[0], p[1], p[2], p[3]));
  }
  load_small(W, small);
}

// Per-row front end shared by forward and backward: environment row and layer 1.
struct RowFront {
  float d[3], R[4], r, rinv, sw, dsw;
  int atom, la, j;
};

__device__ __forceinline__ int local_atom(const int* sRow, int row) {
  int la = 0;
#pragma unroll
  for (int k = 1; k < kMaxAtoms; ++k) la += (sRow[k] <= row) ? 1 : 0;
  return la;
}

// Thread t's row of tile `ti` (pair vector, neighbour index, replica of the centre atom) copied
// asynchronously into shared memory; waited for with cp_async_wait_all.
__device__ __forceinline__ void stage_row(const MixArgs& a, const TileInfo& ti, const int* sRow, int t, float4* sNd,
                                          int* sNj, int* sRep) {
  const int row = ti.p + t;
  const int la = local_atom(sRow, row);
  const size_t e = (size_t)(ti.a0 + la) * a.S + a.sel_off[ti.tj] + (row - sRow[la]);
  tc::cp_async16(sNd + t, a.nl_d + e);
  tc::cp_async4(sNj + t, a.nl_j + e);
  tc::cp_async4(sRep + t, a.irep + ti.a0 + la);
}

// Thread t's pair vector of tile `ti`, loaded into registers (used at the start of the tile).
__device__ __forceinline__ float4 pair_of(const MixArgs& a, const TileInfo& ti, const int* sRow, int t) {
  const int row = ti.p + t;
  const int la = local_atom(sRow, row);
  return __ldg(a.nl_d + (size_t)(ti.a0 + la) * a.S + a.sel_off[ti.tj] + (row - sRow[la]));
}

// Tabulated embedding: coefficient rows (two float4 per output: c0..c3, c4, c5, 0, 0) of the
// interval holding x (edge intervals beyond the ends) and u = (x - x_i) / h.
__device__ __forceinline__ const float4* tab_rows(const MixArgs& a, int pair, float x, float& u) {
  const float f = (x - a.tab_x0) * a.tab_ih;
  int i = (int)floorf(f);
  i = min(max(i, 0), a.tab_n - 1);
  u = f - (float)i;
  return a.tab + ((size_t)pair * a.tab_n + i) * (kN3 * 2);
}
// G = P(u) and dG/du = P'(u) of output q.
__device__ __forceinline__ void tab_poly(const float4* rows, int q, float u, float& g, float& gu) {
  const float4 lo = __ldg(rows + 2 * q), hi = __ldg(rows + 2 * q + 1);
  g = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, hi.y, hi.x), lo.w), lo.z), lo.y), lo.x);
  gu = fmaf(u, fmaf(u, fmaf(u, fmaf(u, 5.f * hi.y, 4.f * hi.x), 3.f * lo.w), 2.f * lo.z), lo.y);
}

// 1/r from one reciprocal square root (a few ulp; the row feeds 16-bit operands and FP32
// sums), r = r^2 / r, and no divisions on the row's critical path.
__device__ __forceinline__ void row_compute(const MixArgs& a, const TileInfo& ti, float4 dv, float winv,
                                            RowFront& f) {
  f.d[0] = dv.x; f.d[1] = dv.y; f.d[2] = dv.z;
  const float r2 = dv.x * dv.x + dv.y * dv.y + dv.z * dv.z;
  f.rinv = rsqrtf(r2);
  f.r = r2 * f.rinv;
  switch_fn(f.r, a.rs, a.rc, winv, a.switch_kind, f.sw, f.dsw);
  const float s = f.sw * f.rinv, sr = s * f.rinv;
  f.R[0] = s; f.R[1] = sr * dv.x; f.R[2] = sr * dv.y; f.R[3] = sr * dv.z;
#pragma unroll
  for (int c = 0; c < 4; ++c) f.R[c] = (f.R[c] - a.stat[ti.ti * 4 + c]) * a.stat[(a.ntypes + ti.ti) * 4 + c];
}

// h1 = tanh(s_hat W1 + b1) and its 16-bit copy into the A block (K = 32: 25 units, then the
// two bias ones; with SPLIT the copy again in K slots 32..63 for the remainder of W2).
template <bool F16, bool SPLIT = false>
__device__ __forceinline__ void layer1(const float* small, float x, float* h1, unsigned char* sA, int t) {
#pragma unroll
  for (int k4 = 0; k4 < 7; ++k4) {
    const float4 wv = reinterpret_cast<const float4*>(small)[k4];
    const float4 bv = reinterpret_cast<const float4*>(small)[8 + k4];
    const float w4[4] = {wv.x, wv.y, wv.z, wv.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (4 * k4 + u < kN1) h1[4 * k4 + u] = tc::tanh_fast(fmaf(x, w4[u], b4[u]));
  }
#pragma unroll
  for (int k0 = 0; k0 < 32; k0 += 8) {
    uint32_t p[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      int k = k0 + 2 * h;
      p[h] = tc::pack2<F16>(k < kN1 ? h1[k] : (k <= kN1 + 1 ? 1.f : 0.f),
                            k + 1 < kN1 ? h1[k + 1] : (k + 1 <= kN1 + 1 ? 1.f : 0.f));
    }
    tc::st_chunk(sA, t, k0, make_uint4(p[0], p[1], p[2], p[3]));
    if (SPLIT) {
      uint32_t q[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        int k = k0 + 2 * h;
        q[h] = tc::pack2<F16>(k < kN1 ? h1[k] : 0.f, k + 1 < kN1 ? h1[k + 1] : 0.f);
      }
      tc::st_chunk(sA, t, 32 + k0, make_uint4(q[0], q[1], q[2], q[3]));
    }
  }
}

// Layer-2 epilogue: h2 = [h1, h1] + tanh(z2) (z2 includes b2); 16-bit copy into the A block
// (K = 64: 50 units, then the two bias ones).
template <bool F16>
__device__ __forceinline__ void layer2_epi(uint32_t tl, const float* small, const float* h1, float* h2,
                                           unsigned char* sA, int t) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float z[16];
    tc::tmem_ld16(tl + 16 * c, z);
    tc::tmem_wait_ld();
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int m = 16 * c + u;
      if (m < kN2) h2[m] = h1[m % kN1] + tc::tanh_fast(z[u]);
    }
  }
#pragma unroll
  for (int k0 = 0; k0 < 64; k0 += 8) {
    uint32_t p[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      int m = k0 + 2 * h;
      p[h] = tc::pack2<F16>(m < kN2 ? h2[m] : (m <= kN2 + 1 ? 1.f : 0.f),
                            m + 1 < kN2 ? h2[m + 1] : (m + 1 <= kN2 + 1 ? 1.f : 0.f));
    }
    tc::st_chunk(sA, t, k0, make_uint4(p[0], p[1], p[2], p[3]));
  }
}

__device__ __forceinline__ void mma_sync_wait(uint64_t* bar, uint32_t& phase, int* err, bool& ok) {
  ok = tc::mbar_wait(bar, phase, err) && ok;
  phase ^= 1u;
  tc::tc_fence_after();
}

__device__ __forceinline__ void operand_barrier() {
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
}

// ------------------------------------------------------------------ forward
// Embedding forward and T: per 128-row tile the environment row and layer 1 on the CUDA
// cores, z2 = h1 W2 and z3 = h2 W3 on the tensor core (biases folded in), G = [h2, h2] +
// tanh(z3), and the T product of G^T against the block-sparse R_hat^T.
template <bool F16, bool TAB>
__global__ void __launch_bounds__(kRows, 3) k_mix_embed_fwd(MixArgs a) {
  extern __shared__ unsigned char sraw[];
  unsigned char* sm = align1024(sraw);
  unsigned char* sA = sm;                          // 16 KB operand block (h1, then h2)
  unsigned char* sGt = sm;                         // 32 KB: G^T fp16 (MN-major: [row][feature]), aliases sA after MMA 2
  unsigned char* sRs = sm + 32768;                 // 4 KB: block-sparse R_hat^T [(atom, c)][row] fp16
  unsigned char* sB2 = sRs + 4096;                 // 8 KB: W2 head | remainder along K
  unsigned char* sB3 = sB2 + 8192;                 // 2 x 14 KB: W3 head, remainder
  float* small = reinterpret_cast<float*>(sB3 + 2 * 14336);  // kSmall
  int* sRow = reinterpret_cast<int*>(small + kSmall);    // kMaxAtoms + 1
  int* sWin = sRow + 8;                                  // 32 row offsets (next tile's window)
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ TileInfo sti;
  __shared__ int s_tot[kMaxTypes], s_tiend[kMaxTypes * kMaxTypes];
  const int t = threadIdx.x, w = t >> 5;
  const float winv = 1.f / (a.rc - a.rs);

  int total = 0;
  for (int tj = 0; tj < a.ntypes; ++tj) total += a.rowoff[(size_t)tj * (a.N + 1) + a.N];
  // at least one full tile per CTA: with few rows (a small box) the CTAs past the last tile
  // return at once instead of each paying the weight staging for a sliver of rows
  const int per = max(kRows, (total + gridDim.x - 1) / gridDim.x);
  const int c0 = min(total, blockIdx.x * per), c1 = min(total, c0 + per);

  if (t == 0) { tc::mbar_init(&bar, 1); tc::mbar_fence_init(); }
  if (w == 0) { tc::tmem_alloc(&tslot, kTmemCols); tc::tmem_relinquish(); }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tslot;
  const uint32_t tl = tmem + ((uint32_t)(32 * w) << 16);
  uint32_t phase = 0;
  bool ok = true;
  int pair = -1;
  walk_tables(a, s_tot, s_tiend);
  __syncthreads();
  Walk wk{0, 0, -1};
  // T partial sums of the tile's atom slots for feature t (thread t = TMEM lane t of
  // the T product); slot 0 carries an atom that continues into the next tile.
  float tacc[kMaxAtoms][4];
#pragma unroll
  for (int s = 0; s < kMaxAtoms; ++s)
#pragma unroll
    for (int c = 0; c < 4; ++c) tacc[s][c] = 0.f;
  long long carry = -1;  // (tj, atom) whose partial T sits in slot 0

  // the first tile is located here; each later one by the locating warp during the previous
  // tile's T product (the tile's own sRow facts are kept in registers by then), after which
  // every thread starts the copy of its row's pair vector into shared memory
  if (w == kLocWarp && c0 < c1) locate_tile(a, c0, c0, c1, wk, s_tot, s_tiend, &sti, sRow);
  __syncthreads();
  // each thread's pair vector of the next tile is loaded into registers while the current
  // tile's T product runs (no shared-memory staging)
  float4 nd = make_float4(0.f, 0.f, 0.f, 1.f);
  if (c0 < c1 && t < sti.nrows) nd = pair_of(a, sti, sRow, t);
  for (int cur = c0; cur < c1 && ok;) {
    // the R_hat^T operand starts from zero (rows of other atoms stay zero)
    {
      uint4* z = reinterpret_cast<uint4*>(sRs);
      for (int q = t; q < 4096 / 16; q += kRows) z[q] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    const TileInfo ti = sti;
    if (w == kLocWarp && cur + ti.nrows < c1) locate_window(a, cur + ti.nrows, wk, s_tot, sWin);
    // the write-out's facts about this tile's atom slots (from the lookup)
    const int last_la = ti.last_la;
    const bool last_done = ti.last_done != 0;
    const unsigned shared_mask = (unsigned)ti.shared_mask;
    const int np = ti.ti * a.ntypes + ti.tj;
    if (np != pair) {
      if (!TAB) {  // the pair's operand blocks from its image, on the product barrier (idle here:
                   // every earlier product has completed)
        if (t == 0)
          fetch_image(a.img + (size_t)np * kImgBytes, kImgFwdB3, kImgFwdSmall, kImgFwd, sB2, sB3, small, &bar);
        ok = tc::mbar_wait(&bar, phase, a.err) && ok;
        phase ^= 1u;
      }
      pair = np;
      __syncthreads();
    }
    const long long key0 = (long long)ti.tj * a.N + ti.a0;
    if (carry != key0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) tacc[0][c] = 0.f;
    }

    // environment row and layer 1
    float h1[kN1], h2[kN2];
    RowFront f;
    const bool valid = t < ti.nrows;
    if (valid) {
      f.la = local_atom(sRow, ti.p + t);
      f.atom = ti.a0 + f.la;
      row_compute(a, ti, nd, winv, f);
    } else {
      f.R[0] = f.R[1] = f.R[2] = f.R[3] = 0.f;
      f.la = 0;
    }
    if constexpr (TAB) {
      // the tabulated embedding: G straight from the table into the G^T operand (fp16, MN-major)
      float u;
      const float4* rows = tab_rows(a, np, f.R[0], u);
#pragma unroll 1
      for (int c = 0; c < 7; ++c) {
        float g[16];
#pragma unroll
        for (int v = 0; v < 16; ++v) {
          const int q = 16 * c + v;
          float gu;
          g[v] = 0.f;
          if (q < kN3) tab_poly(rows, q, u, g[v], gu);
        }
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int q0 = 16 * c + 8 * hh;
          if (q0 < kN3)
            *reinterpret_cast<uint4*>(sGt + tc::sw128_mn_off(q0, t, 16384)) =
                make_uint4(tc::pack2<true>(g[8 * hh], g[8 * hh + 1]), tc::pack2<true>(g[8 * hh + 2], g[8 * hh + 3]),
                           tc::pack2<true>(g[8 * hh + 4], g[8 * hh + 5]), tc::pack2<true>(g[8 * hh + 6], g[8 * hh + 7]));
        }
      }
    } else {
    layer1<F16, true>(small, f.R[0], h1, sA, t);
    operand_barrier();
    if (t == 0) {
      tc::mma_kblock(tmem, tc::smem_u32(sA), tc::smem_u32(sB2), tc::idesc_f16(128, 64, F16), false, 4);
      tc::mma_commit(&bar);
    }
    mma_sync_wait(&bar, phase, a.err, ok);
    layer2_epi<F16>(tl, small, h1, h2, sA, t);
    operand_barrier();
    // layer 3 reuses the TMEM columns of layer 2 (already read)
    if (t == 0) {
      tc::mma_kblock(tmem, tc::smem_u32(sA), tc::smem_u32(sB3), tc::idesc_f16(128, 112, F16), false, 4);
      tc::mma_kblock(tmem, tc::smem_u32(sA), tc::smem_u32(sB3 + 14336), tc::idesc_f16(128, 112, F16), true, 4);
      tc::mma_commit(&bar);
    }
    mma_sync_wait(&bar, phase, a.err, ok);
    // layer-3 epilogue: G = [h2, h2] + tanh(z3) (z3 includes b3); G^T and this row's R_hat column go to
    // the fp16 operands of the T product T_slot[c][a] = sum_rows R_hat[row][c] G[row][a]
    {
      // G^T is the A operand stored MN-major: row = tile row (K), 64 features per 128-byte
      // row, features 64..127 in a second block 16 KB on; each thread writes its own row
#pragma unroll
      for (int c = 0; c < 7; ++c) {
        float z[16];
        tc::tmem_ld16(tl + 16 * c, z);
        tc::tmem_wait_ld();
        float g[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int q = 16 * c + u;
          g[u] = (q < kN3) ? h2[q % kN2] + tc::tanh_fast(z[u]) : 0.f;
        }
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int q0 = 16 * c + 8 * hh;
          if (q0 < kN3)  // features 104.. only feed output rows that are never read
            *reinterpret_cast<uint4*>(sGt + tc::sw128_mn_off(q0, t, 16384)) =
                make_uint4(tc::pack2<true>(g[8 * hh], g[8 * hh + 1]), tc::pack2<true>(g[8 * hh + 2], g[8 * hh + 3]),
                           tc::pack2<true>(g[8 * hh + 4], g[8 * hh + 5]), tc::pack2<true>(g[8 * hh + 6], g[8 * hh + 7]));
        }
      }
    }
    }
    // this row's R_hat column of the block-sparse operand
    if (valid) {
      const uint32_t kr = (uint32_t)(t & 63);
      unsigned char* rcol = sRs + (uint32_t)(t >> 6) * 2048u + (kr & 7) * 2;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int n = f.la * 4 + c;
        *reinterpret_cast<__half*>(rcol + n * 128 + (((kr >> 3) ^ (n & 7)) << 4)) = __float2half_rn(f.R[c]);
      }
    }
    operand_barrier();
    // T product on the tensor core: D[feature][(slot, c)] over the 128 rows (8 K steps;
    // A = G^T read MN-major, B = R_hat^T K-major)
    if (t == 0) {
      const uint32_t id = tc::idesc_mn(tc::idesc_f16(128, 4 * kMaxAtoms, true), true, false);
      const uint64_t a0 = tc::sdesc_sw128_mn(tc::smem_u32(sGt), 16384), b0 = tc::sdesc_sw128(tc::smem_u32(sRs));
      for (int k = 0; k < 8; ++k)
        tc::mma_f16(tmem, tc::sdesc_add(a0, 2048 * k), tc::sdesc_add(b0, (k >> 2) * 2048 + 32 * (k & 3)), id,
                    k > 0 ? 1u : 0u);
      tc::mma_commit(&bar);
    }
    __syncwarp();
    // while the T product runs: locate the next tile and start the copies of its rows
    if (cur + ti.nrows < c1) {
      if (w == kLocWarp) locate_tile(a, cur + ti.nrows, c0, c1, wk, s_tot, s_tiend, &sti, sRow, sWin, true);
      __syncthreads();
      const TileInfo nx = sti;
      if (t < nx.nrows) nd = pair_of(a, nx, sRow, t);
    }
    mma_sync_wait(&bar, phase, a.err, ok);
    {
      float v[16];
      tc::tmem_ld16(tl, v);
      tc::tmem_wait_ld();
#pragma unroll
      for (int s = 0; s < kMaxAtoms; ++s)
#pragma unroll
        for (int c = 0; c < 4; ++c) tacc[s][c] += v[4 * s + c];
    }
    // write complete atoms (feature t of each); carry the open one into slot 0
    const int n_out = last_done ? last_la + 1 : last_la;
    if (t < kN3) {
#pragma unroll
      for (int s = 0; s < kMaxAtoms; ++s) {
        if (s < n_out) {
          const bool shared = (shared_mask >> s) & 1u;
          float* dst = a.Tseg + ((size_t)ti.tj * a.N + ti.a0 + s) * 400 + t;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (shared) atomicAdd(dst + c * kN3, tacc[s][c]);
            else dst[c * kN3] = tacc[s][c];
          }
        }
      }
    }
    float keep[4] = {0.f, 0.f, 0.f, 0.f};
    if (!last_done) {
#pragma unroll
      for (int s = 0; s < kMaxAtoms; ++s)
        if (s == last_la)
#pragma unroll
          for (int c = 0; c < 4; ++c) keep[c] = tacc[s][c];
      carry = (long long)ti.tj * a.N + ti.a0 + last_la;
    } else {
      carry = -1;
    }
#pragma unroll
    for (int s = 0; s < kMaxAtoms; ++s)
#pragma unroll
      for (int c = 0; c < 4; ++c) tacc[s][c] = (s == 0) ? keep[c] : 0.f;
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    cur += ti.nrows;
  }
  tc::cp_async_wait_all();  // copies in flight after an early exit
  // an atom left open at the chunk end continues in the next CTA
  if (carry >= 0 && t < kN3) {
    float* dst = a.Tseg + (size_t)carry * 400 + t;
#pragma unroll
    for (int c = 0; c < 4; ++c) atomicAdd(dst + c * kN3, tacc[0][c]);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// ------------------------------------------------------------------ backward
// Layer-3 column order of the backward: feature q < 50 at column q, q >= 50 at column q + 14,
// so that the two features q = m and q = m + 50 that share the residual h2[m] sit 64 columns
// apart (16-column aligned TMEM loads, N = 128 with zero padding).
__device__ __forceinline__ int bwd_q_of(int n) {
  return n < kN2 ? n : (n >= 64 && n < 64 + kN2 ? n - 14 : -1);
}

// Backward operand blocks of pair (ti, tj): B2 as in the forward ([64 x 64], rows = layer-2
// unit, K = layer-1 unit) and B3 with 128 rows in the column order above (K = layer-2
// unit).  The transposed products dz3 W3^T and dz2 W2^T read the same two blocks as MN-major
// operands (their bias rows land in result columns that are never read).  small: W1, b1.
template <bool F16>
__device__ void load_bwd_ops(const float* __restrict__ W, unsigned char* sB2, unsigned char* sB3, float* small) {
  const int t = threadIdx.x;
  for (int q = t; q < 64 * 8; q += kRows) {
    const int n = q >> 3, k0 = (q & 7) * 8;
    uint32_t p[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int k = k0 + 2 * h;
      p[h] = tc::pack2<F16>(w2_elem<F16>(W, k, n), w2_elem<F16>(W, k + 1, n));
    }
    tc::st_chunk(sB2, n, k0, make_uint4(p[0], p[1], p[2], p[3]));
  }
  for (int q = t; q < 128 * 8; q += kRows) {
    const int n = q >> 3, k0 = (q & 7) * 8;
    const int f = bwd_q_of(n);
    uint32_t p[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int k = k0 + 2 * h;
      p[h] = tc::pack2<F16>(w3_elem<F16>(W, k, f), w3_elem<F16>(W, k + 1, f));
    }
    tc::st_chunk(sB3, n, k0, make_uint4(p[0], p[1], p[2], p[3]));
  }
  load_small(W, small);
}

// Embedding backward with recompute, prod_force and the per-replica virial.  One row per
// thread and TMEM lane; per tile four tensor-core products (z2 = h1 W2, z3 = h2 W3, dh2' = dz3 W3^T,
// dh1' = dz2 W2^T; the last two read B3 / B2 MN-major).  The layer-3 epilogue takes the
// features m and m + 50 together, so the residual part dG[m] + dG[m + 50] of dE/dh2 is final
// when formed; it is parked in the TMEM columns of z3 just read, and added back after the
// dh2' product.  dR_hat and dG use dE/dT and G in FP32 on the CUDA cores.
// ATOMVIR: a second pass over the stored state that accumulates only the per-atom (centre)
// virial -sum g (x) d into a.vir_atom (FP64) and leaves forces and per-replica virials alone.
template <bool F16, bool TAB, bool ATOMVIR = false>
__global__ void __launch_bounds__(kRows, 3) k_mix_embed_bwd(MixArgs a) {
  extern __shared__ unsigned char sraw[];
  unsigned char* sm = align1024(sraw);
  unsigned char* sA = sm;                          // 32 KB: h1 / h2 (blk 0), dz3 (blks 0-1), dz2 (blk 0)
  unsigned char* sB2 = sm + 32768;                 // 8 KB
  unsigned char* sB3 = sB2 + 8192;                 // 16 KB (128 rows, backward column order)
  float4* sdT = reinterpret_cast<float4*>(sB3 + 16384);              // [kMaxAtoms][100], paired layout
  float4* sNd = sdT + kMaxAtoms * kN3;                               // [kRows] pair vectors
  int* sNj = reinterpret_cast<int*>(sNd + kRows);                    // [kRows] neighbour index
  int* sRep = sNj + kRows;                                           // [2][kRows] replica, by tile parity
  float* small = reinterpret_cast<float*>(sRep + 2 * kRows);         // kSmall
  int* sRow = reinterpret_cast<int*>(small + kSmall);                // kMaxAtoms + 1
  int* sWin = sRow + 8;                                              // 32 row offsets
  __shared__ uint64_t bar, dbar;
  __shared__ int sNat;
  __shared__ uint32_t tslot;
  __shared__ TileInfo sti;
  __shared__ int s_tot[kMaxTypes], s_tiend[kMaxTypes * kMaxTypes];
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const float winv = 1.f / (a.rc - a.rs);

  int total = 0;
  for (int tj = 0; tj < a.ntypes; ++tj) total += a.rowoff[(size_t)tj * (a.N + 1) + a.N];
  // at least one full tile per CTA: with few rows (a small box) the CTAs past the last tile
  // return at once instead of each paying the weight staging for a sliver of rows
  const int per = max(kRows, (total + gridDim.x - 1) / gridDim.x);
  const int c0 = min(total, blockIdx.x * per), c1 = min(total, c0 + per);

  if (t == 0) { tc::mbar_init(&bar, 1); tc::mbar_init(&dbar, 1); tc::mbar_fence_init(); }
  if (w == 0) { tc::tmem_alloc(&tslot, kTmemCols); tc::tmem_relinquish(); }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tslot;
  const uint32_t tl = tmem + ((uint32_t)(32 * w) << 16);
  uint32_t phase = 0, dphase = 0;
  bool ok = true;
  int pair = -1;
  walk_tables(a, s_tot, s_tiend);
  __syncthreads();
  Walk wk{0, 0, -1};
  // per-thread virial -sum g (x) d over this thread's rows, per replica (flushed with FP64
  // atomics when the replica changes and at the end)
  float vacc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) vacc[q] = 0.f;
  int vrep = -1;
  const uint32_t id64 = tc::idesc_f16(128, 64, F16);
  const uint32_t id128 = tc::idesc_f16(128, 128, F16);
  const uint32_t idH2 = tc::idesc_mn(tc::idesc_f16(128, 64, F16), false, true);
  const uint32_t idH1 = tc::idesc_mn(tc::idesc_f16(128, 32, F16), false, true);

  // the first tile is located here; each later one by the locating warp in the middle of the
  // previous tile (after the last reads of sti, sRow and sdT), followed by the copies of the
  // tile's dE/dT (bulk, on dbar) and rows (per thread) into shared memory
  if (w == kLocWarp && c0 < c1) locate_tile(a, c0, c0, c1, wk, s_tot, s_tiend, &sti, sRow, nullptr, false, &sNat);
  __syncthreads();
  if (c0 < c1) {
    if (t == 32 * kLocWarp) fetch_dT(a, sti.a0, sNat, sdT, &dbar);
    if (t < sti.nrows) stage_row(a, sti, sRow, t, sNd, sNj, sRep);
  }
  bool dT_pending = c0 < c1;
  int it = 0;
  for (int cur = c0; cur < c1 && ok; ++it) {
    __syncthreads();
    const TileInfo ti = sti;
    tc::cp_async_wait_all();  // this thread's row, copied during the previous tile
    if (w == kLocWarp && cur + ti.nrows < c1) locate_window(a, cur + ti.nrows, wk, s_tot, sWin);
    const int np = ti.ti * a.ntypes + ti.tj;
    if (np != pair) {
      // the backward builds its operand blocks itself: fetching them from the image (bulk or
      // cooperative copy) changed the register allocation of its main loop and cost 4-8%
      if (!TAB) load_bwd_ops<F16>(a.w + (size_t)np * kEmbParams, sB2, sB3, small);
      pair = np;
      __syncthreads();
    }
    // the tile's dE/dT, copied during the previous tile
    RowFront f;
    const bool valid = t < ti.nrows;
    ok = tc::mbar_wait(&dbar, dphase, a.err) && ok;
    dphase ^= 1u;
    dT_pending = false;
    float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
      f.la = local_atom(sRow, ti.p + t);
      f.atom = ti.a0 + f.la;
      f.j = sNj[t];
      dv = sNd[t];
    }

    float h1[kN1], h2[kN2];
    if (valid) {
      row_compute(a, ti, dv, winv, f);
    } else {
      f.R[0] = f.R[1] = f.R[2] = f.R[3] = 0.f;
      f.la = 0; f.j = 0; f.atom = ti.a0;
    }
    float dR[4] = {0.f, 0.f, 0.f, 0.f};
    float ds = 0.f;
    if constexpr (TAB) {
      // the tabulated embedding (no tensor-core products): G and dG/dx of each pair (m, m + 50)
      // from the table, dR_hat += dT G (packed pairs), dG = R_hat . dT, d s_hat += dG dG/dx
      const float4* dTa = sdT + f.la * kN3;
      float u;
      const float4* rows = tab_rows(a, np, f.R[0], u);
      uint64_t ax = tc::f2(0.f, 0.f), ay = ax, az = ax, aw = ax;
#pragma unroll 2
      for (int m = 0; m < kN2; ++m) {
        float ga_, gua, gb_, gub;
        tab_poly(rows, m, u, ga_, gua);
        tab_poly(rows, m + kN2, u, gb_, gub);
        const uint64_t G2 = tc::f2(ga_, gb_);
        const float4 plo = dTa[2 * m], phi = dTa[2 * m + 1];
        ax = tc::f2fma(tc::f2(plo.x, plo.y), G2, ax);
        ay = tc::f2fma(tc::f2(plo.z, plo.w), G2, ay);
        az = tc::f2fma(tc::f2(phi.x, phi.y), G2, az);
        aw = tc::f2fma(tc::f2(phi.z, phi.w), G2, aw);
        const float ga = fmaf(f.R[3], phi.z, fmaf(f.R[2], phi.x, fmaf(f.R[1], plo.z, f.R[0] * plo.x)));
        const float gb = fmaf(f.R[3], phi.w, fmaf(f.R[2], phi.y, fmaf(f.R[1], plo.w, f.R[0] * plo.y)));
        ds = fmaf(ga, gua, fmaf(gb, gub, ds));
      }
      dR[0] = tc::f2lo(ax) + tc::f2hi(ax);
      dR[1] = tc::f2lo(ay) + tc::f2hi(ay);
      dR[2] = tc::f2lo(az) + tc::f2hi(az);
      dR[3] = tc::f2lo(aw) + tc::f2hi(aw);
      ds *= a.tab_ih;
      __syncthreads();  // every thread is done with sdT and sRow before the next tile's lookup
      if (w == kLocWarp && cur + ti.nrows < c1) {
        locate_tile(a, cur + ti.nrows, c0, c1, wk, s_tot, s_tiend, &sti, sRow, sWin, true, &sNat);
        if (lane == 0) fetch_dT(a, sti.a0, sNat, sdT, &dbar);
      }
      if (cur + ti.nrows < c1) {
        dT_pending = true;
        __syncthreads();  // the next tile's sti / sRow
        const TileInfo nx = sti;
        if (t < nx.nrows) stage_row(a, nx, sRow, t, sNd, sNj, sRep + ((it + 1) & 1) * kRows);
      }
    } else {
    layer1<F16>(small, f.R[0], h1, sA, t);
    operand_barrier();
    if (t == 0) {
      tc::mma_kblock(tmem, tc::smem_u32(sA), tc::smem_u32(sB2), id64, false, 2);
      tc::mma_commit(&bar);
    }
    __syncwarp();
    mma_sync_wait(&bar, phase, a.err, ok);
    layer2_epi<F16>(tl, small, h1, h2, sA, t);
    operand_barrier();
    if (t == 0) {
      tc::mma_kblock(tmem, tc::smem_u32(sA), tc::smem_u32(sB3), id128, false, 4);
      tc::mma_commit(&bar);
    }
    __syncwarp();
    mma_sync_wait(&bar, phase, a.err, ok);

    // layer-3 epilogue over the feature pairs (m, m + 50): G, dR_hat, dG, dz3 -> sA (blk 0:
    // column m, blk 1: column m + 64), residual dG[m] + dG[m + 50] -> TMEM column 64 + m.  The
    // two members of a pair run as packed FP32 pairs against the paired dE/dT layout (entries 2m,
    // 2m + 1: x, y then z, w of units m and m + 50).  dz3 is stored negated ((t^2 - 1) g instead of
    // (1 - t^2) g, one instruction less); the layer-2 backward takes the sign back.
    {
      const float4* dTa = sdT + f.la * kN3;
      const uint64_t m1 = tc::f2(-1.f, -1.f);
      uint64_t ax = tc::f2(0.f, 0.f), ay = ax, az = ax, aw = ax;
#pragma unroll
      for (int c = 0; c < 8; ++c) {  // columns 8 c .. 8 c + 7 of each member
        if (8 * c >= kN2) break;
        float za[8], zb[8];
        tc::tmem_ld8(tl + 8 * c, za);
        tc::tmem_ld8(tl + 64 + 8 * c, zb);
        tc::tmem_wait_ld();
        float da[8], db[8], r[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int m = 8 * c + u;
          da[u] = db[u] = r[u] = 0.f;
          if (m < kN2) {
            const float ta = tc::tanh_fast(za[u]), tb = tc::tanh_fast(zb[u]);
            const uint64_t T2 = tc::f2(ta, tb);
            const uint64_t G2 = tc::f2add(tc::f2(h2[m], h2[m]), T2);
            const float4 plo = dTa[2 * m], phi = dTa[2 * m + 1];
            const uint64_t Px = tc::f2(plo.x, plo.y), Py = tc::f2(plo.z, plo.w), Pz = tc::f2(phi.x, phi.y),
                           Pw = tc::f2(phi.z, phi.w);
            ax = tc::f2fma(Px, G2, ax);
            ay = tc::f2fma(Py, G2, ay);
            az = tc::f2fma(Pz, G2, az);
            aw = tc::f2fma(Pw, G2, aw);
            const float ga = fmaf(f.R[3], phi.z, fmaf(f.R[2], phi.x, fmaf(f.R[1], plo.z, f.R[0] * plo.x)));
            const float gb = fmaf(f.R[3], phi.w, fmaf(f.R[2], phi.y, fmaf(f.R[1], plo.w, f.R[0] * plo.y)));
            const uint64_t g = tc::f2(ga, gb);
            const uint64_t dzn = tc::f2mul(g, tc::f2fma(T2, T2, m1));  // -dz3 of (m, m + 50)
            da[u] = tc::f2lo(dzn);
            db[u] = tc::f2hi(dzn);
            r[u] = tc::f2lo(g) + tc::f2hi(g);
          }
        }
        const int k0 = 8 * c;
        tc::st_chunk(sA, t, k0, make_uint4(tc::pack2<F16>(da[0], da[1]), tc::pack2<F16>(da[2], da[3]),
                                           tc::pack2<F16>(da[4], da[5]), tc::pack2<F16>(da[6], da[7])));
        tc::st_chunk(sA + 16384, t, k0, make_uint4(tc::pack2<F16>(db[0], db[1]), tc::pack2<F16>(db[2], db[3]),
                                                   tc::pack2<F16>(db[4], db[5]), tc::pack2<F16>(db[6], db[7])));
        tc::tmem_st8(tl + 64 + k0, r);
      }
      // the last dz3 chunk of each half (columns 56..63 / 120..127) stays zero
      tc::st_chunk(sA, t, 56, make_uint4(0, 0, 0, 0));
      tc::st_chunk(sA + 16384, t, 56, make_uint4(0, 0, 0, 0));
      dR[0] = tc::f2lo(ax) + tc::f2hi(ax);
      dR[1] = tc::f2lo(ay) + tc::f2hi(ay);
      dR[2] = tc::f2lo(az) + tc::f2hi(az);
      dR[3] = tc::f2lo(aw) + tc::f2hi(aw);
    }
    tc::tmem_wait_st();
    operand_barrier();
    // dh2' = dz3 W3^T (B = the rows of B3 read MN-major: K = layer-3 column, N = layer-2 unit)
    if (t == 0) {
      const uint64_t a0 = tc::sdesc_sw128(tc::smem_u32(sA)), b0 = tc::sdesc_sw128_mn(tc::smem_u32(sB3), 8192);
      for (int k = 0; k < 8; ++k)
        tc::mma_f16(tmem, tc::sdesc_add(a0, (k >> 2) * 16384 + 32 * (k & 3)), tc::sdesc_add(b0, 2048 * k), idH2,
                    k > 0 ? 1u : 0u);
      tc::mma_commit(&bar);
    }
    __syncwarp();
    // while the MMA runs: locate the next tile and start the copies of its dE/dT (sdT is free
    // now) and rows
    if (w == kLocWarp && cur + ti.nrows < c1) {
      locate_tile(a, cur + ti.nrows, c0, c1, wk, s_tot, s_tiend, &sti, sRow, sWin, true, &sNat);
      if (lane == 0) fetch_dT(a, sti.a0, sNat, sdT, &dbar);  // values this lane has just written
    }
    mma_sync_wait(&bar, phase, a.err, ok);
    if (cur + ti.nrows < c1) {
      dT_pending = true;
      __syncthreads();  // the next tile's sti / sRow
      const TileInfo nx = sti;
      if (t < nx.nrows) stage_row(a, nx, sRow, t, sNd, sNj, sRep + ((it + 1) & 1) * kRows);
    }
    // layer-2 backward: g2 = dh2' + residual, dz2 = g2 (1 - t2^2) -> sA; h2's residual into dh1
    float dh1[kN1];
#pragma unroll
    for (int k = 0; k < kN1; ++k) dh1[k] = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float z[16], rr[16];
      tc::tmem_ld16(tl + 16 * c, z);
      tc::tmem_ld16(tl + 64 + 16 * c, rr);
      tc::tmem_wait_ld();
      float d2[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int m = 16 * c + u;
        d2[u] = 0.f;
        if (m < kN2) {
          const float g2 = rr[u] - z[u];  // dh2' comes out negated (dz3 was stored negated)
          const float t2 = h2[m] - h1[m % kN1];
          d2[u] = g2 * (1.f - t2 * t2);
          dh1[m % kN1] += g2;
        }
      }
#pragma unroll
      for (int hh = 0; hh < 2; ++hh)
        tc::st_chunk(sA, t, 16 * c + 8 * hh,
                     make_uint4(tc::pack2<F16>(d2[8 * hh], d2[8 * hh + 1]), tc::pack2<F16>(d2[8 * hh + 2], d2[8 * hh + 3]),
                                tc::pack2<F16>(d2[8 * hh + 4], d2[8 * hh + 5]),
                                tc::pack2<F16>(d2[8 * hh + 6], d2[8 * hh + 7])));
    }
    operand_barrier();
    // dh1' = dz2 W2^T (B = the rows of B2 read MN-major: K = layer-2 unit, N = layer-1 unit)
    if (t == 0) {
      const uint64_t a0 = tc::sdesc_sw128(tc::smem_u32(sA)), b0 = tc::sdesc_sw128_mn(tc::smem_u32(sB2), 8192);
      for (int k = 0; k < 4; ++k)
        tc::mma_f16(tmem, tc::sdesc_add(a0, 32 * k), tc::sdesc_add(b0, 2048 * k), idH1, k > 0 ? 1u : 0u);
      tc::mma_commit(&bar);
    }
    __syncwarp();
    mma_sync_wait(&bar, phase, a.err, ok);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float z[16];
      tc::tmem_ld16(tl + 16 * c, z);
      tc::tmem_wait_ld();
#pragma unroll
      for (int u4 = 0; u4 < 4; ++u4) {
        const float4 wv = reinterpret_cast<const float4*>(small)[4 * c + u4];
        const float w4[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = 16 * c + 4 * u4 + u;
          if (k < kN1) {
            const float g1 = z[4 * u4 + u] + dh1[k];
            ds = fmaf(g1 * (1.f - h1[k] * h1[k]), w4[u], ds);
          }
        }
      }
    }
    }  // network path
    // chain rule through the normalisation and the environment row.  Per-row terms,
    // the per-warp partial sums and the force accumulation are FP32 (FP64 arithmetic
    // runs at a small fraction of the FP32 rate on this GPU; ~180 terms per atom add
    // ~1e-6 relative rounding); the per-atom virial is accumulated in FP64.
    float g3[3] = {0.f, 0.f, 0.f};
    if (valid) {
      dR[0] += ds;
#pragma unroll
      for (int c = 0; c < 4; ++c) dR[c] *= a.stat[(a.ntypes + ti.ti) * 4 + c];
      const float rinv = f.rinv;
      const float dsr = f.dsw * rinv - f.sw * rinv * rinv;
      const float qv = f.sw * rinv * rinv;
      const float dq = f.dsw * rinv * rinv - 2.f * f.sw * rinv * rinv * rinv;
      const float proj = dR[1] * f.d[0] + dR[2] * f.d[1] + dR[3] * f.d[2];
      const float common = (dR[0] * dsr + dq * proj) * rinv;
#pragma unroll
      for (int c = 0; c < 3; ++c) g3[c] = common * f.d[c] + qv * dR[1 + c];
    }
    if (ATOMVIR) {
      // this row's -g (x) d, summed over the rows of each centre atom of the warp
      float vr[9];
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) vr[3 * p + q] = valid ? -g3[p] * f.d[q] : 0.f;
      const int my = valid ? f.la : -1;
      unsigned todo = __ballot_sync(0xffffffffu, valid);
      while (todo) {
        const int leader = __ffs(todo) - 1;
        const int seg = __shfl_sync(0xffffffffu, my, leader);
        const bool in = (my == seg);
        const unsigned mask = __ballot_sync(0xffffffffu, in);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          float v = in ? vr[q] : 0.f;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == leader) atomicAdd(&a.vir_atom[((size_t)ti.a0 + seg) * 9 + q], (double)v);
        }
        todo &= ~mask;
      }
      __syncthreads();
      cur += ti.nrows;
      continue;
    }
    if (valid) {
      tc::red_add_v4(a.force32 + 4 * (size_t)f.j, -g3[0], -g3[1], -g3[2], 0.f);
      const int rep = sRep[(it & 1) * kRows + t];
      if (rep != vrep) {
        if (vrep >= 0)
#pragma unroll
          for (int q = 0; q < 9; ++q) atomicAdd(&a.vir_rep[9 * vrep + q], (double)vacc[q]);
#pragma unroll
        for (int q = 0; q < 9; ++q) vacc[q] = 0.f;
        vrep = rep;
      }
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) vacc[3 * p + q] = fmaf(-g3[p], f.d[q], vacc[3 * p + q]);
    }
    // centre force: warp-segmented sums over rows of the same atom (the three components
    // reduced together, one vector atomic per segment)
    const int my = valid ? f.la : -1;
    unsigned todo = __ballot_sync(0xffffffffu, valid);
    while (todo) {
      const int leader = __ffs(todo) - 1;
      const int seg = __shfl_sync(0xffffffffu, my, leader);
      const bool in = (my == seg);
      const unsigned mask = __ballot_sync(0xffffffffu, in);
      float v0 = in ? g3[0] : 0.f, v1 = in ? g3[1] : 0.f, v2 = in ? g3[2] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
      }
      if (lane == leader) tc::red_add_v4(a.force32 + 4 * ((size_t)ti.a0 + seg), v0, v1, v2, 0.f);
      todo &= ~mask;
    }
    __syncthreads();
    cur += ti.nrows;
  }
  // copies still in flight after an early exit
  tc::cp_async_wait_all();
  if (dT_pending) tc::mbar_wait(&dbar, dphase, a.err);
  // flush the virial accumulators: one warp reduction when all lanes hold the same replica
  if (!ATOMVIR) {
    const int r0 = __shfl_sync(0xffffffffu, vrep, 0);
    if (__all_sync(0xffffffffu, vrep == r0)) {
      if (r0 >= 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          float v = vacc[q];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) atomicAdd(&a.vir_rep[9 * r0 + q], (double)v);
        }
      }
    } else if (vrep >= 0) {
#pragma unroll
      for (int q = 0; q < 9; ++q) atomicAdd(&a.vir_rep[9 * vrep + q], (double)vacc[q]);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// ------------------------------------------------------------------ small kernels
// Exclusive scan of nl_count[i][tj] over atoms, per neighbour type: local (1024 per block),
// block totals, fix-up.
__global__ void k_scan_local(int N, int ntypes, const int* __restrict__ cnt, int* rowoff, int* blk) {
  __shared__ int ws[32];
  const int tj = blockIdx.y;
  const int i = blockIdx.x * 1024 + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int v = (i < N) ? cnt[(size_t)i * ntypes + tj] : 0;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  const int excl = x - v + (w > 0 ? ws[w - 1] : 0);
  if (i < N) rowoff[(size_t)tj * (N + 1) + i] = excl;
  if (threadIdx.x == 1023) blk[tj * gridDim.x + blockIdx.x] = ws[31];
}

__global__ void k_scan_fix(int N, int nblk, int* rowoff, const int* blk) {
  const int tj = blockIdx.y;
  __shared__ int off;
  if (threadIdx.x == 0) {
    int s = 0;
    for (int b = 0; b < blockIdx.x; ++b) s += blk[tj * nblk + b];
    off = s;
    if (blockIdx.x == nblk - 1) {
      int tot = s;
      tot += blk[tj * nblk + blockIdx.x];
      rowoff[(size_t)tj * (N + 1) + N] = tot;
    }
  }
  __syncthreads();
  const int i = blockIdx.x * 1024 + threadIdx.x;
  if (i < N) rowoff[(size_t)tj * (N + 1) + i] += off;
}

// T = sum over neighbour types of the partial sums, scaled by 1/S (kept in FP32, feature-major,
// for the dE/dT kernel); D = T^T T[:, :16] in 16 bits for the fitting net.  One warp per atom
// at a time: the atom's partial sums (one 1.6 KB segment per neighbour type) are copied into a
// per-warp double buffer in dynamic shared memory by cp.async one atom ahead; T[c][b < 16] is
// held in registers and lane -> rows a = lane, lane + 32, ... of D (16 values, two 16-byte
// stores).
// Padded neighbour slots add (sel[tj] - count) copies of the normalised zero row's term
// (pad: [nt][nt][4][100], c-major, or null when every davg is 0).
constexpr int kDescWarps = 4;

struct PadArgs {
  const float* pad;
  const int* itype;
  const int* nl_count;
  int sel[kMaxTypes];
};

template <bool F16>
__global__ void __launch_bounds__(32 * kDescWarps) k_mix_descriptor(int N, int ntypes, float invS,
                                                                   const float* __restrict__ Tseg, float4* Tm,
                                                                   unsigned short* Dm, PadArgs pa) {
  extern __shared__ float4 sbuf[];  // [kDescWarps][2][ntypes][100]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float4* mine = sbuf + (size_t)w * 2 * ntypes * kN3;
  const int stride = gridDim.x * kDescWarps;
  auto issue = [&](int atom, int buf) {
    float4* dst = mine + buf * ntypes * kN3;
    for (int tj = 0; tj < ntypes; ++tj) {
      const float4* src = reinterpret_cast<const float4*>(Tseg + ((size_t)tj * N + atom) * 400);
      for (int q = lane; q < kN3; q += 32) tc::cp_async16(dst + tj * kN3 + q, src + q);
    }
    tc::cp_async_commit();
  };
  int i = blockIdx.x * kDescWarps + w;
  if (i < N) issue(i, 0);
  for (int buf = 0; i < N; i += stride, buf ^= 1) {
    if (i + stride < N) {
      issue(i + stride, buf ^ 1);
      tc::cp_async_wait_group<1>();
    } else {
      tc::cp_async_wait_group<0>();
    }
    __syncwarp();
    float4* seg = mine + buf * ntypes * kN3;
    // T (c-major, 400 floats) in place of the first segment
    const int ti = pa.pad ? pa.itype[i] : 0;
    for (int q = lane; q < kN3; q += 32) {
      float4 v = seg[q];
      for (int tj = 1; tj < ntypes; ++tj) {
        const float4 u = seg[tj * kN3 + q];
        v.x += u.x; v.y += u.y; v.z += u.z; v.w += u.w;
      }
      if (pa.pad)
        for (int tj = 0; tj < ntypes; ++tj) {
          const float np = (float)(pa.sel[tj] - pa.nl_count[(size_t)i * ntypes + tj]);
          const float4 u = reinterpret_cast<const float4*>(pa.pad + (size_t)(ti * ntypes + tj) * 400)[q];
          v.x = fmaf(np, u.x, v.x); v.y = fmaf(np, u.y, v.y); v.z = fmaf(np, u.z, v.z); v.w = fmaf(np, u.w, v.w);
        }
      v.x *= invS; v.y *= invS; v.z *= invS; v.w *= invS;
      seg[q] = v;
    }
    __syncwarp();
    const float* T = reinterpret_cast<const float*>(seg);
    float tb[4][kM2];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int b4 = 0; b4 < kM2 / 4; ++b4) {
        const float4 v = seg[(c * kN3) / 4 + b4];
        tb[c][4 * b4] = v.x; tb[c][4 * b4 + 1] = v.y; tb[c][4 * b4 + 2] = v.z; tb[c][4 * b4 + 3] = v.w;
      }
    for (int aa = lane; aa < kN3; aa += 32) {
      const float t0 = T[aa], t1 = T[kN3 + aa], t2 = T[2 * kN3 + aa], t3 = T[3 * kN3 + aa];
      Tm[(size_t)i * kN3 + aa] = make_float4(t0, t1, t2, t3);
      uint32_t pk[8];
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        float o[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int b = 2 * h + e;
          o[e] = fmaf(t3, tb[3][b], fmaf(t2, tb[2][b], fmaf(t1, tb[1][b], t0 * tb[0][b])));
        }
        pk[h] = tc::pack2<F16>(o[0], o[1]);
      }
      uint4* dst = reinterpret_cast<uint4*>(Dm + (size_t)i * kKD + aa * kM2);
      dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
    __syncwarp();  // every lane is done with this buffer before it is refilled
  }
}

// dT[c][a] = (1/S) (sum_b dD[a][b] T[c][b] + [a < 16] sum_a' dD[a'][a] T[c][a']), stored per atom
// as 100 float4 paired for the embedding backward: entries 2m = (x_m, x_m+50, y_m, y_m+50) and
// 2m + 1 = (z_m, z_m+50, w_m, w_m+50) for m < 50.  dD (dE/dD from the fitting kernel) is fp16 and
// T is stored feature-major ([N][100] float4 of the four components).
// One warp per atom at a time: the atom's T and dD are copied into a per-warp double buffer by
// cp.async one atom ahead, so the copies of the next atom overlap this one's arithmetic.  The
// second term's 64 outputs (c, a < 16) take lanes (a, half of the a' range) and one shuffle.
constexpr int kDtWarps = 4;

__global__ void __launch_bounds__(32 * kDtWarps) k_mix_dT(int N, float invS, const float4* __restrict__ Tm,
                                                         const unsigned short* __restrict__ dD,
                                                         float4* __restrict__ dT) {
  __shared__ __align__(16) float4 sT[kDtWarps][2][kN3];
  __shared__ __align__(16) unsigned short sD[kDtWarps][2][kKD];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int stride = gridDim.x * kDtWarps;
  auto issue = [&](int atom, int buf) {
    const float4* Ti = Tm + (size_t)atom * kN3;
    for (int q = lane; q < kN3; q += 32) tc::cp_async16(&sT[w][buf][q], Ti + q);
    const uint4* Di = reinterpret_cast<const uint4*>(dD + (size_t)atom * kKD);
    uint4* Ds = reinterpret_cast<uint4*>(sD[w][buf]);
    for (int q = lane; q < kKD / 8; q += 32) tc::cp_async16(Ds + q, Di + q);
    tc::cp_async_commit();
  };
  int i = blockIdx.x * kDtWarps + w;
  if (i < N) issue(i, 0);
  for (int buf = 0; i < N; i += stride, buf ^= 1) {
    if (i + stride < N) {
      issue(i + stride, buf ^ 1);
      tc::cp_async_wait_group<1>();
    } else {
      tc::cp_async_wait_group<0>();
    }
    __syncwarp();
    const float4* T = sT[w][buf];
    const __half* D = reinterpret_cast<const __half*>(sD[w][buf]);
    // second term: lane -> a = lane % 16 over a' in [50 h, 50 h + 50), h = lane / 16
    float u[4] = {0.f, 0.f, 0.f, 0.f};
    {
      const int a = lane & 15, h = lane >> 4;
#pragma unroll 5
      for (int a2 = 50 * h; a2 < 50 * h + 50; ++a2) {
        const float d = __half2float(D[a2 * kM2 + a]);
        const float4 tv = T[a2];
        u[0] = fmaf(d, tv.x, u[0]); u[1] = fmaf(d, tv.y, u[1]);
        u[2] = fmaf(d, tv.z, u[2]); u[3] = fmaf(d, tv.w, u[3]);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) u[c] += __shfl_xor_sync(0xffffffffu, u[c], 16);
    }
    // first term: lane -> pairs m = lane, lane + 32 (units m and m + 50); T[b] for b < 16 held
    // in registers
    float4 tb[kM2];
#pragma unroll
    for (int b = 0; b < kM2; ++b) tb[b] = T[b];
#pragma unroll
    for (int pp = 0; pp < 2; ++pp) {
      const int m = lane + 32 * pp;
      float ua[4];  // second term of unit m < 16, held by lane m
#pragma unroll
      for (int c = 0; c < 4; ++c) ua[c] = __shfl_sync(0xffffffffu, u[c], m & 15);
      if (m < kN2) {
        float v[2][4];
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
          const int a = m + kN2 * e2;
#pragma unroll
          for (int c = 0; c < 4; ++c) v[e2][c] = (a < kM2) ? ua[c] : 0.f;
          const uint4* Drow = reinterpret_cast<const uint4*>(D + a * kM2);
#pragma unroll
          for (int hc = 0; hc < 2; ++hc) {
            const uint4 raw = Drow[hc];
            const uint32_t q[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float2 d2 = __half22float2(*reinterpret_cast<const __half2*>(&q[e]));
              const float4 t0 = tb[8 * hc + 2 * e], t1 = tb[8 * hc + 2 * e + 1];
              v[e2][0] = fmaf(d2.x, t0.x, v[e2][0]); v[e2][1] = fmaf(d2.x, t0.y, v[e2][1]);
              v[e2][2] = fmaf(d2.x, t0.z, v[e2][2]); v[e2][3] = fmaf(d2.x, t0.w, v[e2][3]);
              v[e2][0] = fmaf(d2.y, t1.x, v[e2][0]); v[e2][1] = fmaf(d2.y, t1.y, v[e2][1]);
              v[e2][2] = fmaf(d2.y, t1.z, v[e2][2]); v[e2][3] = fmaf(d2.y, t1.w, v[e2][3]);
            }
          }
        }
        float4* o = dT + (size_t)i * kN3 + 2 * m;
        o[0] = make_float4(v[0][0] * invS, v[1][0] * invS, v[0][1] * invS, v[1][1] * invS);
        o[1] = make_float4(v[0][2] * invS, v[1][2] * invS, v[0][3] * invS, v[1][3] * invS);
      }
    }
    __syncwarp();  // every lane is done with this buffer before it is refilled
  }
}

// force (FP64, [N][3]) += force32 (the mixed backward's FP32 accumulation, [N][4]).
__global__ void k_fold_force32(int n3, const float* __restrict__ f32, double* __restrict__ force) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n3) force[k] += (double)f32[4 * (k / 3) + k % 3];
}

MixArgs make_mix_args(Model* m, int N) {
  MixArgs a{};
  a.N = N; a.ntypes = m->ntypes; a.S = m->S;
  for (int t = 0; t <= m->ntypes; ++t) a.sel_off[t] = m->sel_off[t];
  a.rc = (float)m->rc; a.rs = (float)m->rs; a.invS = 1.f / (float)m->S; a.switch_kind = m->switch_kind;
  a.w = m->w32; a.stat = m->stat32; a.itype = m->itype; a.type_off = m->type_off; a.rowoff = m->rowoff;
  a.tab = reinterpret_cast<const float4*>(m->tab32);
  a.img = static_cast<const unsigned char*>(m->emb_img);
  a.tab_n = m->tab_n;
  a.tab_x0 = (float)m->tab_x0;
  a.tab_ih = m->tab_n ? (float)(1.0 / m->tab_h) : 0.f;
  a.nl_j = m->nl_j; a.nl_d = static_cast<const float4*>(m->nl_d);
  a.Tseg = m->Tseg; a.dT = static_cast<const float4*>(m->dTm);
  a.force = m->force; a.force32 = m->force32; a.vir_atom = m->vir_atom; a.err = m->err;
  a.vir_rep = m->vir_rep; a.irep = m->irep;
  return a;
}

// (+ 160: sRow (8 ints) and sWin (32 ints); + 1024: alignment of the operand blocks)
// The forward operand image of every embedding pair: one CTA per pair runs the forward's
// shared-memory staging into global memory (the same bytes, swizzle included).
template <bool F16>
__global__ void __launch_bounds__(kRows) k_emb_images(const float* __restrict__ w, unsigned char* img) {
  const float* W = w + (size_t)blockIdx.x * kEmbParams;
  unsigned char* r = img + (size_t)blockIdx.x * kImgBytes;
  load_fwd_weights<F16>(W, r, r + kImgFwdB3, reinterpret_cast<float*>(r + kImgFwdSmall));
}
static_assert(kImgFwd % 16 == 0 && kImgFwdB3 % 16 == 0 && kImgFwdSmall % 16 == 0,
              "bulk copies need 16-byte sizes and offsets");

constexpr size_t kFwdSmem = 32768 + 4096 + 8192 + 2 * 14336 + kSmall * 4 + 160 + 1024;
constexpr size_t kBwdSmem =
    32768 + 8192 + 16384 + kMaxAtoms * kN3 * 16 + kRows * (16 + 4 + 8) + kSmall * 4 + 160 + 1024;

}  // namespace

size_t mix_emb_image_bytes(int ntypes) { return (size_t)ntypes * ntypes * kImgBytes; }

dp_status launch_emb_images(Model* m) {
  const int npairs = m->ntypes * m->ntypes;
  if (m->prec == DP_MIX_FP16)
    k_emb_images<true><<<npairs, kRows, 0, m->stream>>>(m->w32, static_cast<unsigned char*>(m->emb_img));
  else
    k_emb_images<false><<<npairs, kRows, 0, m->stream>>>(m->w32, static_cast<unsigned char*>(m->emb_img));
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_mix_descriptor(Model* m, int N) {
  const int nblk = cdiv(N, 1024);
  k_scan_local<<<dim3(nblk, m->ntypes), 1024, 0, m->stream>>>(N, m->ntypes, m->nl_count, m->rowoff, m->scan_blk);
  k_scan_fix<<<dim3(nblk, m->ntypes), 1024, 0, m->stream>>>(N, nblk, m->rowoff, m->scan_blk);
  DP_CUDA_TRY(m, cudaMemsetAsync(m->Tseg, 0, sizeof(float) * 400 * (size_t)N * m->ntypes, m->stream));
  MixArgs a = make_mix_args(m, N);
  const bool f16 = m->prec == DP_MIX_FP16;
  const bool tab = m->tab_n > 0;
  auto fk = f16 ? (tab ? k_mix_embed_fwd<true, true> : k_mix_embed_fwd<true, false>)
                : (tab ? k_mix_embed_fwd<false, true> : k_mix_embed_fwd<false, false>);
  const void* fn = reinterpret_cast<const void*>(fk);
  DP_CUDA_TRY(m, ensure_smem(fn, kFwdSmem));
  const int grid = tuned_grid(m, 0, num_sms() * blocks_per_sm(fn, kRows, kFwdSmem, kTmemCols));
  fk<<<grid, kRows, kFwdSmem, m->stream>>>(a);
  if (m->sub_ev[0]) DP_CUDA_TRY(m, cudaEventRecord(m->sub_ev[0], m->stream));
  const int dgrid = std::max(1, std::min((N + kDescWarps - 1) / kDescWarps, tuned_grid(m, 3, 8 * num_sms())));
  const size_t dsm = (size_t)kDescWarps * 2 * m->ntypes * kN3 * sizeof(float4);
  const void* dfn = f16 ? reinterpret_cast<const void*>(k_mix_descriptor<true>)
                        : reinterpret_cast<const void*>(k_mix_descriptor<false>);
  DP_CUDA_TRY(m, ensure_smem(dfn, dsm));
  PadArgs pa{};
  pa.pad = m->has_pad ? m->pad32 : nullptr;
  pa.itype = m->itype;
  pa.nl_count = m->nl_count;
  for (int t = 0; t < m->ntypes; ++t) pa.sel[t] = m->sel[t];
  if (f16)
    k_mix_descriptor<true><<<dgrid, 32 * kDescWarps, dsm, m->stream>>>(
        N, m->ntypes, 1.f / (float)m->S, m->Tseg, static_cast<float4*>(m->Tm), static_cast<unsigned short*>(m->Dm),
        pa);
  else
    k_mix_descriptor<false><<<dgrid, 32 * kDescWarps, dsm, m->stream>>>(
        N, m->ntypes, 1.f / (float)m->S, m->Tseg, static_cast<float4*>(m->Tm), static_cast<unsigned short*>(m->Dm),
        pa);
  m->launches += 4;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_mix_embed_backward(Model* m, int N) {
  const int dt_grid = std::max(1, std::min((N + kDtWarps - 1) / kDtWarps, tuned_grid(m, 2, 5 * num_sms())));
  k_mix_dT<<<dt_grid, 32 * kDtWarps, 0, m->stream>>>(N, 1.f / (float)m->S, static_cast<const float4*>(m->Tm),
                                                              static_cast<const unsigned short*>(m->dD),
                                                              static_cast<float4*>(m->dTm));
  DP_CUDA_TRY(m, cudaMemsetAsync(m->vir_rep, 0, sizeof(double) * 9 * (size_t)m->nrep, m->stream));
  DP_CUDA_TRY(m, cudaMemsetAsync(m->force32, 0, sizeof(float) * 4 * (size_t)N, m->stream));
  if (m->sub_ev[1]) DP_CUDA_TRY(m, cudaEventRecord(m->sub_ev[1], m->stream));
  MixArgs a = make_mix_args(m, N);
  const bool f16 = m->prec == DP_MIX_FP16;
  const bool tab = m->tab_n > 0;
  auto bk = f16 ? (tab ? k_mix_embed_bwd<true, true> : k_mix_embed_bwd<true, false>)
                : (tab ? k_mix_embed_bwd<false, true> : k_mix_embed_bwd<false, false>);
  const void* fn = reinterpret_cast<const void*>(bk);
  DP_CUDA_TRY(m, ensure_smem(fn, kBwdSmem));
  const int grid = tuned_grid(m, 1, num_sms() * blocks_per_sm(fn, kRows, kBwdSmem, kTmemCols));
  bk<<<grid, kRows, kBwdSmem, m->stream>>>(a);
  k_fold_force32<<<cdiv(3L * N, 256), 256, 0, m->stream>>>(3 * N, m->force32, m->force);
  m->launches += 3;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

dp_status launch_mix_atom_virial(Model* m, int N) {
  MixArgs a = make_mix_args(m, N);
  const bool f16 = m->prec == DP_MIX_FP16;
  const bool tab = m->tab_n > 0;
  auto bk = f16 ? (tab ? k_mix_embed_bwd<true, true, true> : k_mix_embed_bwd<true, false, true>)
                : (tab ? k_mix_embed_bwd<false, true, true> : k_mix_embed_bwd<false, false, true>);
  const void* fn = reinterpret_cast<const void*>(bk);
  DP_CUDA_TRY(m, ensure_smem(fn, kBwdSmem));
  const int grid = tuned_grid(m, 1, num_sms() * blocks_per_sm(fn, kRows, kBwdSmem, kTmemCols));
  bk<<<grid, kRows, kBwdSmem, m->stream>>>(a);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

}  // namespace dpg
