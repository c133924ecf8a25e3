// Mixed-precision fitting net on the tensor cores: forward 1600 -> 240 -> 240 ->
// 240 -> 1 and the data-gradient backward to dE/dD, fused in one persistent
// kernel per 128-atom tile of one centre type (Section II-A fitting net; Section
// III-B2: the backward multiplies by pre-arranged weight copies so every GEMM is
// of the same "NN" form; Section III-B3: the wide first-layer GEMM in 16 bits, the
// rest at FP32-level accuracy).
//
// Per tile (one TMEM lane per atom; two warpgroups split the 240 columns):
//   L1  z1 = D W1 + b1          16-bit operands, A (D) and B by TMA      h1 = tanh(z1)
//   L2  h2 = h1 + tanh(h1 W2 + b2)                 split 16-bit (3 MMAs)
//   L3  h3 = h2 + tanh(h2 W3 + b3);  E_i = h3 . w4 + b4 + e_bias   split
//   B3  dh2 = w4 + dz3 W3^T,  dz3 = w4 (1 - t3^2)  split
//   B2  dh1 = dh2 + dz2 W2^T, dz2 = dh2 (1 - t2^2) split
//   B1  dE/dD = dz1 W1^T,     dz1 = dh1 (1 - h1^2)  16-bit, N = 1600 in 10 chunks
// "Split": x = x_hi + x_lo with both halves 16-bit, x*w ~ x_hi w_hi + x_hi w_lo +
// x_lo w_hi, which keeps ~16 mantissa bits; rounding the 240 x 240 layers to plain
// 16 bits biases E_i by ~1e-3 eV (bf16), above the 1e-4 eV/atom target.
// The activations tanh come from e^{2x} (hardware base-2 exponential and reciprocal), within
// ~1e-6 absolute: an E_i error far below the 1e-4 eV/atom target.
// dE/dD is written in fp16 for the dE/dT kernel.
// The activation operand X (hi and lo) lives in shared memory, the FP32 residual
// stream (h1, h2, dh2) in TMEM columns 256..495, the factors 1 - h1^2 and 1 - t2^2
// in a small global scratch between forward and backward.  TMA loads run several
// jobs ahead of the MMAs in slots carved from whichever buffers the current GEMM
// does not read.
#include <cstring>
#include <deque>
#include <mutex>

#include "tc_common.cuh"

namespace dpg {
namespace {

constexpr int kFR = 128;                  // rows (atoms) per tile = TMEM lanes
constexpr int kThreads = 256;             // two warpgroups
constexpr int kBChunk = 160;              // N chunk of the B1 GEMM
constexpr uint32_t kBlk = 16384;          // one [128 x 64] 16-bit operand block
constexpr uint32_t kWB = 240 * 128;       // one [240 x 64] 16-bit weight block (30 KB)
constexpr uint32_t kXHi = 0;              // X_hi: 4 blocks
constexpr uint32_t kXLo = 4 * kBlk;       // X_lo: 4 blocks
constexpr uint32_t kSt = 8 * kBlk;        // 64 KB: four split staging slots
constexpr uint32_t kSSlot = 128 * 128;    // split job: [128 x 64] 16-bit weight block (16 KB)
constexpr int kSSlots = 4;
constexpr uint32_t kStageRow = kBChunk * 2 + 16;  // padded row of the dE/dD staging tile (bytes)
constexpr uint32_t kL1Slot = kBlk + kWB;  // L1 job: A block + W1T block (46 KB), slots over [0, kPrm)
constexpr int kL1Slots = 4;
constexpr uint32_t kB1Slot = kBChunk * 128;  // B1 job: W1 block [160 x 64] (20 KB), slots over [kXLo, kPrm)
constexpr int kB1Slots = 5;
// dE/dD of one B1 chunk is staged here [128 rows x 160 fp16] and written out in whole row
// segments; it overlays L1 slot 3 and the split slots, both idle during B1
constexpr uint32_t kStage = kXLo + kB1Slots * kB1Slot;
constexpr uint32_t kPrm = kStage + kFR * kStageRow;  // b1, b2, b3, w4
constexpr int kSplitSlot = 6;             // barrier index of the first split staging slot (6..9)
constexpr int kSplitJobs = 16;            // per split GEMM: 4 K blocks x 2 N halves x {hi, lo}
constexpr int kL1Jobs = kKD / 64;         // 25
constexpr int kB1Jobs = 4 * (kKD / kBChunk);  // 40

struct FitMaps {
  CUtensorMap D;                     // [rows = max_atoms][1600]
  CUtensorMap W1T[kMaxTypes];        // [240][1600]        L1 B
  CUtensorMap W1[kMaxTypes];         // [1600][240]        B1 B
  CUtensorMap S[kMaxTypes][4][2];    // split [240][240]: W2T, W3T, W3, W2 x {hi, lo}
};

struct FitArgs {
  int N, ntypes;
  const int* type_off;
  const int* type_count;
  const float* w;          // theta fp32
  long fit_base;           // offset of the first fitting block in theta
  long ebias_off;
  unsigned short* f1;      // [N][240] 16-bit: 1 - h1^2
  unsigned short* f2;      // [N][240] 16-bit: 1 - t2^2
  unsigned short* dD;      // [N][1600] fp16
  double* e_atom;
  int* err;
};

// Staging slots: one full/empty mbarrier pair each; `uses` counts completed jobs per slot.
struct Slots {
  uint64_t* full;   // [10]: L1 0..3, B1 0..5, split 6..9
  uint64_t* empty;  // [10]
  uint32_t uses[10];
};

__device__ __forceinline__ unsigned char* align1k(unsigned char* p) {
  uint32_t a = tc::smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// Before loading into slot k: wait until the MMAs of its previous job released it.
__device__ __forceinline__ void slot_acquire(Slots& s, int k, uint32_t loads_done, int* err, bool& ok) {
  if (loads_done > 0) ok = tc::mbar_wait(&s.empty[k], (loads_done - 1) & 1u, err) && ok;
}

template <bool F16>
__device__ __forceinline__ void store_x16(unsigned char* sm, int row, int col0, const float* v, bool split) {
  // 16 consecutive K elements of row `row` starting at col0 (multiple of 16): hi, and lo if split
  uint32_t ph[8], pl[8];
#pragma unroll
  for (int h = 0; h < 8; ++h) {
    ph[h] = tc::pack2<F16>(v[2 * h], v[2 * h + 1]);
    if (split) {
      float a0, a1;
      if (F16) {
        float2 f = __half22float2(*reinterpret_cast<__half2*>(&ph[h]));
        a0 = f.x; a1 = f.y;
      } else {
        float2 f = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&ph[h]));
        a0 = f.x; a1 = f.y;
      }
      pl[h] = tc::pack2<F16>(v[2 * h] - a0, v[2 * h + 1] - a1);
    }
  }
  const uint32_t blk = (col0 >> 6) * kBlk;
  tc::st_chunk(sm + kXHi + blk, row, col0 & 63, make_uint4(ph[0], ph[1], ph[2], ph[3]));
  tc::st_chunk(sm + kXHi + blk, row, (col0 & 63) + 8, make_uint4(ph[4], ph[5], ph[6], ph[7]));
  if (split) {
    tc::st_chunk(sm + kXLo + blk, row, col0 & 63, make_uint4(pl[0], pl[1], pl[2], pl[3]));
    tc::st_chunk(sm + kXLo + blk, row, (col0 & 63) + 8, make_uint4(pl[4], pl[5], pl[6], pl[7]));
  }
}

template <bool F16>
__device__ __forceinline__ void store_g16(unsigned short* g, const float* v) {
  uint32_t p[8];
#pragma unroll
  for (int h = 0; h < 8; ++h) p[h] = tc::pack2<F16>(v[2 * h], v[2 * h + 1]);
  uint4* d = reinterpret_cast<uint4*>(g);
  d[0] = make_uint4(p[0], p[1], p[2], p[3]);
  d[1] = make_uint4(p[4], p[5], p[6], p[7]);
}

template <bool F16>
__device__ __forceinline__ void unpack_g16(uint4 q0, uint4 q1, float* v) {
  const uint32_t p[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
  for (int h = 0; h < 8; ++h) {
    if (F16) {
      float2 f = __half22float2(*reinterpret_cast<const __half2*>(&p[h]));
      v[2 * h] = f.x; v[2 * h + 1] = f.y;
    } else {
      float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&p[h]));
      v[2 * h] = f.x; v[2 * h + 1] = f.y;
    }
  }
}

// ---- issuing thread (thread 0) helpers
struct Issuer {
  Slots* s;
  unsigned char* sm;
  const FitMaps* mp;
  int ty, row0;
  int* err;
  bool* ok;
  uint64_t keep, stream;  // L2 policies: weights (evict_last), streamed D (evict_first)
  // Every CTA walks the shared weight matrices starting at a different block, so the
  // SMs do not all request the same L2 lines at the same moment.
  int rot_l1, rot_s, rot_b1;
  __device__ int l1_block(int j) const { return (j + rot_l1) % kL1Jobs; }
  __device__ int split_block(int kb) const { return (kb + rot_s) & 3; }
  __device__ int b1_chunk(int n) const { return (n + rot_b1) % (kKD / kBChunk); }

  // L1 job j: A (D rows row0.., K block l1_block(j)) + the matching W1T block into slot j % 4
  __device__ void load_l1(int j) {
    const int k = j % kL1Slots;
    slot_acquire(*s, k, s->uses[k], err, *ok);
    unsigned char* a = sm + k * kL1Slot;
    const int kb = l1_block(j);
    tc::mbar_arrive_expect_tx(&s->full[k], kL1Slot);
    tc::tma_load_2d_hint(a, &mp->D, &s->full[k], 64 * kb, row0, stream);
    tc::tma_load_2d_hint(a + kBlk, &mp->W1T[ty], &s->full[k], 64 * kb, 0, keep);
  }
  // B1 job j: W1 rows of chunk b1_chunk(j / 4), K block j % 4, into slot j % 6 (X_lo + split area)
  __device__ void load_b1(int j) {
    const int k = j % kB1Slots;
    slot_acquire(*s, k, s->uses[k], err, *ok);
    tc::mbar_arrive_expect_tx(&s->full[k], kB1Slot);
    tc::tma_load_2d_hint(sm + kXLo + k * kB1Slot, &mp->W1[ty], &s->full[k], 64 * (j & 3), kBChunk * b1_chunk(j >> 2),
                         keep);
  }
  // split job i of GEMM g: weight half i & 1 (0 = hi, 1 = lo), N half (i >> 1) & 1 (rows 0..127
  // or 128..255; rows past 240 are zero-filled by the TMA) of K block split_block(i >> 2),
  // into split slot i & 3
  __device__ void load_split(int g, int i) {
    const int k = kSplitSlot + (i & 3);
    slot_acquire(*s, k, s->uses[k], err, *ok);
    tc::mbar_arrive_expect_tx(&s->full[k], kSSlot);
    tc::tma_load_2d_hint(sm + kSt + (i & 3) * kSSlot, &mp->S[ty][g][i & 1], &s->full[k], 64 * split_block(i >> 2),
                         128 * ((i >> 1) & 1), keep);
  }
  // the first three jobs of split GEMM g (issued under the preceding epilogue)
  __device__ void prefetch_split(int g) {
    for (int i = 0; i < kSSlots - 1; ++i) load_split(g, i);
  }
  // wait for the data of the oldest outstanding job in slot k and mark it consumed after the MMAs
  __device__ void consume_begin(int k) {
    *ok = tc::mbar_wait(&s->full[k], s->uses[k] & 1u, err) && *ok;
    tc::tc_fence_after();
  }
  __device__ void consume_end(int k) {
    tc::mma_commit(&s->empty[k]);
    s->uses[k] += 1;
  }
};

template <bool F16>
__global__ void __launch_bounds__(kThreads, 1) k_mix_fit(const __grid_constant__ FitMaps maps, FitArgs a) {
  extern __shared__ unsigned char sraw[];
  unsigned char* sm = align1k(sraw);
  float* prm = reinterpret_cast<float*>(sm + kPrm);  // b1, b2, b3, w4 [4][240]
  __shared__ uint64_t full[10], empty[10], accb[2];
  __shared__ uint32_t tslot;
  __shared__ int s_tiles[kMaxTypes + 1];
  __shared__ float sE[kFR];
  const int t = threadIdx.x, w = t >> 5;
  const int row = t & (kFR - 1), half = t >> 7;  // TMEM lane / atom, column half

  if (t == 0) {
    for (int q = 0; q < 10; ++q) { tc::mbar_init(&full[q], 1); tc::mbar_init(&empty[q], 1); }
    for (int q = 0; q < 2; ++q) tc::mbar_init(&accb[q], 1);
    tc::mbar_fence_init();
    int acc = 0;
    for (int ty = 0; ty < a.ntypes; ++ty) { s_tiles[ty] = acc; acc += (a.type_count[ty] + kFR - 1) / kFR; }
    s_tiles[a.ntypes] = acc;
    tc::tma_prefetch_desc(&maps.D);
  }
  if (w == 0) { tc::tmem_alloc(&tslot, 512); tc::tmem_relinquish(); }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tslot;
  const uint32_t lane_off = (uint32_t)(32 * (w & 3)) << 16;
  const uint32_t acc0 = tmem + lane_off, acc1 = tmem + 256 + lane_off;
  const uint32_t resid = acc1;
  Slots sl;
  sl.full = full; sl.empty = empty;
  for (int q = 0; q < 10; ++q) sl.uses[q] = 0;
  uint32_t aph[2] = {0, 0};
  bool ok = true;
  int cur_type = -1;
  const int ntiles = s_tiles[a.ntypes];
  const uint32_t id240 = tc::idesc_f16(128, 240, F16), id160 = tc::idesc_f16(128, kBChunk, F16);
  const uint32_t id128 = tc::idesc_f16(128, 128, F16);
  // columns of this thread's half: 16-column chunks [c_beg, c_end) of 15 (240 columns)
  const int c_beg = half ? 8 : 0, c_end = half ? 15 : 8;
  Issuer is;
  is.s = &sl; is.sm = sm; is.mp = &maps; is.err = a.err; is.ok = &ok;
  is.keep = tc::make_policy_evict_last();
  is.stream = tc::make_policy_evict_first();
  is.rot_l1 = blockIdx.x % kL1Jobs;
  is.rot_s = blockIdx.x & 3;
  is.rot_b1 = blockIdx.x % (kKD / kBChunk);

  auto sync_all = [&]() {
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
  };
  auto wait_acc = [&](int r) {
    ok = tc::mbar_wait(&accb[r], aph[r], a.err) && ok;
    aph[r] ^= 1u;
    tc::tc_fence_after();
  };
  // thread 0: the MMAs of split GEMM g (its first three jobs were prefetched).  Each job is
  // one N half (128 output columns) of one K block, hi or lo weights; after issuing job i the
  // slot of job i - 1 is refilled, so three loads stay in flight behind the MMAs.
  auto issue_split = [&](int g) {
    for (int i = 0; i < kSplitJobs && ok; ++i) {
      const int k = kSplitSlot + (i & 3);
      is.consume_begin(k);
      const int kx = is.split_block(i >> 2);
      const uint32_t d = tmem + 128u * (uint32_t)((i >> 1) & 1);
      const uint32_t xh = tc::smem_u32(sm + kXHi + kx * kBlk), xl = tc::smem_u32(sm + kXLo + kx * kBlk);
      const uint32_t wv = tc::smem_u32(sm + kSt + (i & 3) * kSSlot);
      if ((i & 1) == 0) {  // hi weights: x_hi w_hi + x_lo w_hi
        tc::mma_kblock(d, xh, wv, id128, i >= 4, 4);
        tc::mma_kblock(d, xl, wv, id128, true, 4);
      } else {             // lo weights: x_hi w_lo
        tc::mma_kblock(d, xh, wv, id128, true, 4);
      }
      is.consume_end(k);
      if (i + kSSlots - 1 < kSplitJobs) is.load_split(g, i + kSSlots - 1);
    }
    tc::mma_commit(&accb[0]);
  };

  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    int ty = 0;
    while (ty + 1 < a.ntypes && tile >= s_tiles[ty + 1]) ++ty;
    const int k = tile - s_tiles[ty];
    const int row0 = a.type_off[ty] + k * kFR;
    const int nrow = min(kFR, a.type_count[ty] - k * kFR);
    const bool valid = row < nrow;
    const size_t grow = (size_t)row0 + row;
    const float* P = a.w + a.fit_base + (long)ty * kFitParams;
    is.ty = ty; is.row0 = row0;
    if (ty != cur_type) {
      for (int q = t; q < 4 * kF; q += kThreads) {
        const int which = q / kF, c = q - which * kF;
        const long off = which == 0 ? kFb1 : which == 1 ? kFb2 : which == 2 ? kFb3 : kFw4;
        prm[q] = P[off + c];
      }
      cur_type = ty;
      __syncthreads();
    }
    const float* b1 = prm;
    const float* b2 = prm + kF;
    const float* b3 = prm + 2 * kF;
    const float* w4 = prm + 3 * kF;

    // ---- L1: z1 = D W1, 4 slots over [0, kPrm), three jobs ahead
    if (t == 0) {
      for (int j = 0; j < kL1Slots - 1; ++j) is.load_l1(j);
      for (int j = 0; j < kL1Jobs && ok; ++j) {
        const int s = j % kL1Slots;
        is.consume_begin(s);
        unsigned char* st = sm + s * kL1Slot;
        tc::mma_kblock(tmem, tc::smem_u32(st), tc::smem_u32(st + kBlk), id240, j > 0, 4);
        is.consume_end(s);
        // refill the slot of job j - 1 (MMAs of job j stay queued meanwhile)
        if (j + kL1Slots - 1 < kL1Jobs) is.load_l1(j + kL1Slots - 1);
      }
      tc::mma_commit(&accb[0]);
    }
    __syncwarp();  // lanes 1..31 of warp 0 wait here, not in a polling loop beside the issuer
    wait_acc(0);
    if (t == 0) is.prefetch_split(0);  // prefetch under the epilogue
    __syncwarp();
    // f1/f2 factors of this row are fetched ahead of the TMEM loop below
#pragma unroll 1
    for (int c = c_beg; c < c_end; ++c) {
      float z[16], h[16], f[16];
      tc::tmem_ld16(acc0 + 16 * c, z);
      tc::tmem_wait_ld();
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        h[u] = tc::tanh_exp(z[u] + b1[16 * c + u]);
        f[u] = 1.f - h[u] * h[u];
      }
      store_x16<F16>(sm, row, 16 * c, h, true);
      tc::tmem_st16(resid + 16 * c, h);
      if (valid) store_g16<F16>(a.f1 + grow * kF + 16 * c, f);
    }
    if (half == 1) {  // K columns 240..255 stay zero (hi and lo)
      tc::st_chunk(sm + kXHi + 3 * kBlk, row, 48, make_uint4(0, 0, 0, 0));
      tc::st_chunk(sm + kXHi + 3 * kBlk, row, 56, make_uint4(0, 0, 0, 0));
      tc::st_chunk(sm + kXLo + 3 * kBlk, row, 48, make_uint4(0, 0, 0, 0));
      tc::st_chunk(sm + kXLo + 3 * kBlk, row, 56, make_uint4(0, 0, 0, 0));
    }
    tc::tmem_wait_st();
    sync_all();

    // ---- L2: h2 = h1 + tanh(h1 W2 + b2)
    if (t == 0) issue_split(0);
    __syncwarp();
    wait_acc(0);
    if (t == 0) is.prefetch_split(1);
    __syncwarp();
#pragma unroll 1
    for (int c = c_beg; c < c_end; ++c) {
      float z[16], r[16], f[16];
      tc::tmem_ld16(acc0 + 16 * c, z);
      tc::tmem_ld16(resid + 16 * c, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float t2 = tc::tanh_exp(z[u] + b2[16 * c + u]);
        r[u] += t2;
        f[u] = 1.f - t2 * t2;
      }
      store_x16<F16>(sm, row, 16 * c, r, true);
      tc::tmem_st16(resid + 16 * c, r);
      if (valid) store_g16<F16>(a.f2 + grow * kF + 16 * c, f);
    }
    tc::tmem_wait_st();
    sync_all();

    // ---- L3: h3 = h2 + tanh(h2 W3 + b3), E_i, dz3
    if (t == 0) issue_split(1);
    __syncwarp();
    wait_acc(0);
    if (t == 0) is.prefetch_split(2);
    __syncwarp();
    float e = 0.f;
#pragma unroll 1
    for (int c = c_beg; c < c_end; ++c) {
      float z[16], r[16], dz[16];
      tc::tmem_ld16(acc0 + 16 * c, z);
      tc::tmem_ld16(resid + 16 * c, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float t3 = tc::tanh_exp(z[u] + b3[16 * c + u]);
        const float wv = w4[16 * c + u];
        e = fmaf(r[u] + t3, wv, e);
        dz[u] = wv * (1.f - t3 * t3);
      }
      store_x16<F16>(sm, row, 16 * c, dz, true);
    }
    if (half == 1) sE[row] = e;
    sync_all();
    if (half == 0 && valid)
      a.e_atom[grow] = (double)e + (double)sE[row] + (double)P[kFb4] + (double)a.w[a.ebias_off + ty];

    // ---- B3: dh2 = w4 + dz3 W3^T ; dz2 = dh2 (1 - t2^2)
    if (t == 0) issue_split(2);
    __syncwarp();
    {  // fetch this row's 1 - t2^2 factors while the MMAs run
      uint4 fq[16];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int cc = c_beg + c;
        if (valid && cc < c_end) {
          const uint4* src = reinterpret_cast<const uint4*>(a.f2 + grow * kF + 16 * cc);
          fq[2 * c] = src[0];
          fq[2 * c + 1] = src[1];
        } else {
          fq[2 * c] = fq[2 * c + 1] = make_uint4(0, 0, 0, 0);
        }
      }
      wait_acc(0);
      if (t == 0) is.prefetch_split(3);
      __syncwarp();
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int cc = c_beg + c;
        if (cc < c_end) {
          float z[16], f[16];
          tc::tmem_ld16(acc0 + 16 * cc, z);
          tc::tmem_wait_ld();
          unpack_g16<F16>(fq[2 * c], fq[2 * c + 1], f);
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            z[u] += w4[16 * cc + u];  // dh2
            f[u] *= z[u];             // dz2
          }
          tc::tmem_st16(resid + 16 * cc, z);
          store_x16<F16>(sm, row, 16 * cc, f, true);
        }
      }
    }
    tc::tmem_wait_st();
    sync_all();

    // ---- B2: dh1 = dh2 + dz2 W2^T ; dz1 = dh1 (1 - h1^2)
    if (t == 0) issue_split(3);
    __syncwarp();
    {
      uint4 fq[16];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int cc = c_beg + c;
        if (valid && cc < c_end) {
          const uint4* src = reinterpret_cast<const uint4*>(a.f1 + grow * kF + 16 * cc);
          fq[2 * c] = src[0];
          fq[2 * c + 1] = src[1];
        } else {
          fq[2 * c] = fq[2 * c + 1] = make_uint4(0, 0, 0, 0);
        }
      }
      wait_acc(0);
      // the B1 slots overlay X_lo and the split staging, both free once B2's MMAs are done;
      // its weights stream in under this epilogue
      if (t == 0)
        for (int j = 0; j < kB1Slots - 1; ++j) is.load_b1(j);
      __syncwarp();
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int cc = c_beg + c;
        if (cc < c_end) {
          float z[16], r[16], f[16];
          tc::tmem_ld16(acc0 + 16 * cc, z);
          tc::tmem_ld16(resid + 16 * cc, r);
          tc::tmem_wait_ld();
          unpack_g16<F16>(fq[2 * c], fq[2 * c + 1], f);
#pragma unroll
          for (int u = 0; u < 16; ++u) f[u] *= (z[u] + r[u]);
          store_x16<F16>(sm, row, 16 * cc, f, false);  // B1 is a plain 16-bit GEMM
        }
      }
    }
    sync_all();

    // ---- B1: dE/dD = dz1 W1^T in N chunks of 160 (4 K jobs each); TMEM regions alternate,
    //      chunk n + 2 is issued once chunk n has been drained
    constexpr int nch = kKD / kBChunk;
    int next_load = kB1Slots - 1;
    auto issue_b1_chunk = [&](int n) {
      for (int kb = 0; kb < 4 && ok; ++kb) {
        const int j = 4 * n + kb;
        const int s = j % kB1Slots;
        is.consume_begin(s);
        tc::mma_kblock(tmem + 256 * (n & 1), tc::smem_u32(sm + kXHi + kb * kBlk),
                       tc::smem_u32(sm + kXLo + s * kB1Slot), id160, kb > 0, 4);
        is.consume_end(s);
        // refill freed slots (the slot of job j - 1 at the latest) while job j's MMAs run
        while (next_load < kB1Jobs && next_load <= j + kB1Slots - 1) is.load_b1(next_load++);
      }
      tc::mma_commit(&accb[n & 1]);
    };
    if (t == 0) {
      issue_b1_chunk(0);
      issue_b1_chunk(1);
    }
    __syncwarp();
    for (int n = 0; n < nch; ++n) {
      const int rg = n & 1;
      wait_acc(rg);
      const uint32_t src = rg ? acc1 : acc0;
      // this thread's 80 columns of its row into the staging tile (fp16): five TMEM loads in
      // flight, one wait
      {
        const int cb = half ? 5 : 0;
        float z[5][16];
#pragma unroll
        for (int c = 0; c < 5; ++c) tc::tmem_ld16(src + 16 * (cb + c), z[c]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          uint32_t p[8];
#pragma unroll
          for (int h = 0; h < 8; ++h) p[h] = tc::pack2<true>(z[c][2 * h], z[c][2 * h + 1]);
          uint4* d = reinterpret_cast<uint4*>(sm + kStage + row * kStageRow + 32 * (cb + c));
          d[0] = make_uint4(p[0], p[1], p[2], p[3]);
          d[1] = make_uint4(p[4], p[5], p[6], p[7]);
        }
      }
      __syncthreads();
      // whole row segments (320 B) to dE/dD: warp w writes rows w, w + 8, ...; lanes 0..19
      {
        const int col0 = kBChunk * is.b1_chunk(n);
        for (int r = w; r < nrow; r += kThreads / 32)
          if ((t & 31) < kBChunk / 8) {
            const uint4 v = *reinterpret_cast<const uint4*>(sm + kStage + r * kStageRow + 16 * (t & 31));
            __stcs(reinterpret_cast<uint4*>(a.dD + (size_t)(row0 + r) * kKD + col0 + 8 * (t & 31)), v);
          }
      }
      tc::tc_fence_before();
      __syncthreads();
      tc::tc_fence_after();
      if (t == 0 && n + 2 < nch && ok) issue_b1_chunk(n + 2);
      __syncwarp();
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tmem, 512);
}

// 16-bit copies of the fitting weights of every type, laid out as the kernel's B operands:
// W1T [240][1600], W1 [1600][240], then for W2T, W3T, W3, W2 ([240][240]) a hi and a lo copy.
template <class H>
void make_fit_copies(const std::vector<double>& theta, long fit_base, int nt, std::vector<H>& out, H (*cvt)(float),
                     float (*back)(H)) {
  const size_t per = (size_t)kF * kKD * 2 + (size_t)kF * kF * 8;
  out.resize(per * nt);
  for (int ty = 0; ty < nt; ++ty) {
    const double* P = theta.data() + fit_base + (size_t)ty * kFitParams;
    H* W1T = out.data() + per * ty;
    H* W1 = W1T + (size_t)kF * kKD;
    H* S = W1 + (size_t)kF * kKD;
    for (int k = 0; k < kKD; ++k)
      for (int o = 0; o < kF; ++o) {
        const float v = (float)P[kFW1 + (size_t)k * kF + o];
        W1T[(size_t)o * kKD + k] = cvt(v);
        W1[(size_t)k * kF + o] = cvt(v);
      }
    auto put = [&](int g, size_t idx, double v) {
      const float f = (float)v;
      const H hi = cvt(f);
      S[(size_t)(2 * g) * kF * kF + idx] = hi;
      S[(size_t)(2 * g + 1) * kF * kF + idx] = cvt(f - back(hi));
    };
    for (int k = 0; k < kF; ++k)
      for (int o = 0; o < kF; ++o) {
        put(0, (size_t)o * kF + k, P[kFW2 + (size_t)k * kF + o]);  // W2T
        put(1, (size_t)o * kF + k, P[kFW3 + (size_t)k * kF + o]);  // W3T
        put(2, (size_t)k * kF + o, P[kFW3 + (size_t)k * kF + o]);  // W3
        put(3, (size_t)k * kF + o, P[kFW2 + (size_t)k * kF + o]);  // W2
      }
  }
}

__nv_bfloat16 to_bf16(float x) { return __float2bfloat16_rn(x); }
__half to_f16(float x) { return __float2half_rn(x); }
float from_bf16(__nv_bfloat16 x) { return __bfloat162float(x); }
float from_f16(__half x) { return __half2float(x); }

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D map over a row-major [rows][cols] 16-bit matrix, box [box_rows][64], 128-byte swizzle.
bool make_map(CUtensorMap* map, void* base, bool f16, uint64_t cols, uint64_t rows, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// The model's tensor maps, created with its weights (mix_fit_setup) and freed by dp_destroy.
FitMaps* maps_of(Model* m) {
  if (!m->fit_maps) m->fit_maps = new FitMaps{};
  return static_cast<FitMaps*>(m->fit_maps);
}

constexpr size_t kFitSmem = kPrm + 4 * kF * 4 + 1024;
static_assert(kL1Slots * kL1Slot <= kPrm, "L1 slots exceed the staging area");
static_assert(kXLo + kB1Slots * kB1Slot <= kStage, "B1 slots overlap the dE/dD staging tile");
static_assert(kSt + kSSlots * kSSlot <= kPrm, "split slots exceed the staging area");

}  // namespace

void mix_fit_release(Model* m) {
  delete static_cast<FitMaps*>(m->fit_maps);
  m->fit_maps = nullptr;
}

// Build the 16-bit weight copies and the tensor maps (at model creation).
dp_status mix_fit_setup(Model* m) {
  const bool f16 = m->prec == DP_MIX_FP16;
  const long fit_base = (long)m->ntypes * m->ntypes * kEmbParams;
  const size_t per = (size_t)kF * kKD * 2 + (size_t)kF * kF * 8;
  std::vector<unsigned short> host;
  if (f16) {
    std::vector<__half> h;
    make_fit_copies<__half>(m->theta_host, fit_base, m->ntypes, h, to_f16, from_f16);
    host.resize(h.size());
    std::memcpy(host.data(), h.data(), 2 * h.size());
  } else {
    std::vector<__nv_bfloat16> h;
    make_fit_copies<__nv_bfloat16>(m->theta_host, fit_base, m->ntypes, h, to_bf16, from_bf16);
    host.resize(h.size());
    std::memcpy(host.data(), h.data(), 2 * h.size());
  }
  DP_CUDA_TRY(m, cudaMemcpy(m->tc_weights, host.data(), 2 * host.size(), cudaMemcpyHostToDevice));
  FitMaps* fm = maps_of(m);
  unsigned short* base = static_cast<unsigned short*>(m->tc_weights);
  bool ok = make_map(&fm->D, m->Dm, f16, kKD, (uint64_t)m->max_atoms, 128);
  for (int ty = 0; ty < m->ntypes; ++ty) {
    unsigned short* W1T = base + per * ty;
    unsigned short* W1 = W1T + (size_t)kF * kKD;
    unsigned short* S = W1 + (size_t)kF * kKD;
    ok = ok && make_map(&fm->W1T[ty], W1T, f16, kKD, kF, kF);
    ok = ok && make_map(&fm->W1[ty], W1, f16, kF, kKD, kBChunk);
    for (int g = 0; g < 4; ++g)
      for (int h = 0; h < 2; ++h)
        ok = ok && make_map(&fm->S[ty][g][h], S + (size_t)(2 * g + h) * kF * kF, f16, kF, kF, 128);
  }
  if (!ok) {
    m->last_error = "cuTensorMapEncodeTiled failed";
    return DP_ERR_CUDA;
  }
  return DP_OK;
}

size_t mix_fit_weight_bytes(int ntypes) { return 2 * ((size_t)kF * kKD * 2 + (size_t)kF * kF * 8) * ntypes; }

dp_status launch_mix_fitting(Model* m, int N) {
  FitArgs a{};
  a.N = N; a.ntypes = m->ntypes; a.type_off = m->type_off; a.type_count = m->type_count; a.w = m->w32;
  a.fit_base = (long)m->ntypes * m->ntypes * kEmbParams;
  a.ebias_off = a.fit_base + (long)m->ntypes * kFitParams;
  a.f1 = static_cast<unsigned short*>(m->act[0]);
  a.f2 = static_cast<unsigned short*>(m->act[1]);
  a.dD = static_cast<unsigned short*>(m->dD);
  a.e_atom = m->e_atom;
  a.err = m->err;
  const bool f16 = m->prec == DP_MIX_FP16;
  const void* fn = f16 ? reinterpret_cast<const void*>(k_mix_fit<true>) : reinterpret_cast<const void*>(k_mix_fit<false>);
  DP_CUDA_TRY(m, ensure_smem(fn, kFitSmem));
  const int tiles_upper = cdiv(N, kFR) + m->ntypes;
  const int grid = std::max(1, std::min(num_sms(), tiles_upper));
  if (f16) k_mix_fit<true><<<grid, kThreads, kFitSmem, m->stream>>>(*maps_of(m), a);
  else k_mix_fit<false><<<grid, kThreads, kFitSmem, m->stream>>>(*maps_of(m), a);
  m->launches += 1;
  DP_LAUNCH_CHECK(m);
  return DP_OK;
}

}  // namespace dpg
