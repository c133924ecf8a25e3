// Mixed-precision fitting net on the tensor cores: forward 1600 -> 240 -> 240 ->
// 240 -> 1 and the data-gradient backward to dE/dD, fused in one persistent
// kernel per 128-atom tile of one centre type (Section II-A fitting net; Section
// III-B2: the backward multiplies by pre-arranged weight copies so every GEMM is
// of the same "NN" form; Section III-B3: the wide first-layer GEMM in 16 bits, the
// rest at FP32-level accuracy).
//
// Per tile (one TMEM lane per atom; two warpgroups split the 240 columns):
//   L1  z1 = D W1 + b1          16-bit operands, A (D) and B by TMA      h1 = tanh(z1)
//   L2  h2 = h1 + tanh(h1 W2 + b2)                 split 16-bit (3 MMAs of N = 240)
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
constexpr int kEpi = 256;                 // epilogue threads: warps 0..7, two per TMEM lane quarter
constexpr int kMmaWarp = 8;               // lane 0 issues every tcgen05.mma
constexpr int kLoadWarp = 9;              // lane 0 of warps 9..11 issue the TMA loads
constexpr int kLoaders = 3;
constexpr int kThreads = kEpi + 32 + 32 * kLoaders;
constexpr int kBChunk = 160;              // N chunk of the B1 GEMM
constexpr uint32_t kBlk = 16384;          // one [128 x 64] 16-bit operand block
constexpr uint32_t kWB = 240 * 128;       // one [240 x 64] 16-bit weight block (30 KB)
constexpr uint32_t kXHi = 0;              // X_hi: 4 blocks
constexpr uint32_t kXLo = 4 * kBlk;       // X_lo: 4 blocks
constexpr uint32_t kSt = 8 * kBlk;        // 90 KB: three split staging slots
constexpr uint32_t kSSlot = kWB;          // split job: [240 x 64] 16-bit weight block (30 KB)
constexpr int kSSlots = 3;
constexpr uint32_t kStageRow = kBChunk * 2 + 16;  // padded row of the dE/dD staging tile (bytes)
constexpr uint32_t kL1Slot = kBlk + kWB;  // L1 job: A block + W1T block (46 KB)
constexpr int kL1Slots = 3;               // slots over [0, kStage)
// B1 job: two W1 blocks [160 x 64] (K blocks 2h and 2h + 1 of one chunk, 40 KB), slots over
// [kXLo, kStage).  Every job costs the issuing thread a barrier wait and a commit (~0.15-0.2 us
// each on this GPU), so jobs carry two K blocks: eight products per wait.
constexpr uint32_t kB1Box = kBChunk * 128;
constexpr uint32_t kB1Slot = 2 * kB1Box;
constexpr int kB1Slots = 2;
// dE/dD of one B1 chunk is staged here [128 rows x 160 fp16] and written out in whole row
// segments; it overlays the split slots, idle during B1
constexpr uint32_t kStage = kXLo + kB1Slots * kB1Slot;
constexpr uint32_t kPrm = kSt + kSSlots * kSSlot;  // b1, b2, b3, w4
constexpr int kSplitSlot = 6;             // barrier index of the first split staging slot (6..8)
constexpr int kSplitJobs = 8;             // per split GEMM: 4 K blocks x {hi, lo}, all 240 output columns
constexpr int kL1Jobs = kKD / 64;         // 25
constexpr int kB1Chunks = kKD / kBChunk;  // 10
constexpr int kB1Jobs = 2 * kB1Chunks;    // 20

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

__device__ __forceinline__ unsigned char* align1k(unsigned char* p) {
  uint32_t a = tc::smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// The staging slots: barrier k (full: data landed; empty: the MMAs that read it completed) for
// L1 slots 0..2, B1 slots 0..1 and split slots 6..8.  `uses[k]` counts the jobs through slot k.
//   L1 job j      -> slot j % 3        B1 job j -> slot j % 2        split job i -> slot 6 + i % 3
//
// Each TMA thread processes its own copies one after another (about 0.3 us each from L2,
// whatever the box size), so three loader threads share the slots: slot k belongs to loader
// k % 3, which keeps the successive uses of a slot in one thread's program order.  The loaders
// sit in separate warps: lanes of one warp waiting on different barriers would take turns.
struct Loader {
  uint64_t* full;
  uint64_t* empty;
  unsigned char* sm;
  const FitMaps* mp;
  int lane;               // loader index 0..2
  int* err;
  bool ok;
  uint32_t uses[10];
  uint32_t issued[10];     // copies this lane started into slot k (for the final drain)
  uint64_t keep, stream;   // L2 policies: weights (evict_last), streamed D (evict_first)
  // Every CTA walks the shared weight matrices starting at a different block, so the SMs do
  // not all request the same L2 lines at the same moment.
  int rot_l1, rot_s, rot_b1;

  __device__ bool begin(int k, uint32_t bytes) {
    if (k % kLoaders != lane || !ok) return false;
    if (uses[k] > 0) ok = tc::mbar_wait(&empty[k], (uses[k] - 1) & 1u, err) && ok;
    if (!ok) return false;
    tc::mbar_arrive_expect_tx(&full[k], bytes);
    issued[k] = uses[k] + 1;
    return true;
  }
  // L1 job j: D rows row0.. and the W1T block of K block (j + rot) % 25
  __device__ void l1(int ty, int row0, int j) {
    const int k = j % kL1Slots, kb = (j + rot_l1) % kL1Jobs;
    if (begin(k, kL1Slot)) {
      unsigned char* a = sm + k * kL1Slot;
      tc::tma_load_2d_hint(a, &mp->D, &full[k], 64 * kb, row0, stream);
      tc::tma_load_2d_hint(a + kBlk, &mp->W1T[ty], &full[k], 64 * kb, 0, keep);
    }
    uses[k] += 1;
  }
  // split job i of GEMM g: weight half i & 1 (0 = hi, 1 = lo) of K block ((i >> 1) + rot) % 4,
  // all 240 rows
  __device__ void split(int ty, int g, int i) {
    const int s = i % kSSlots, k = kSplitSlot + s;
    if (begin(k, kSSlot))
      tc::tma_load_2d_hint(sm + kSt + s * kSSlot, &mp->S[ty][g][i & 1], &full[k], 64 * (((i >> 1) + rot_s) & 3), 0,
                           keep);
    uses[k] += 1;
  }
  // B1 job j: W1 rows of chunk (j / 2 + rot) % 10, K blocks 2 (j % 2) and 2 (j % 2) + 1
  __device__ void b1(int ty, int j) {
    const int k = j % kB1Slots;
    if (begin(k, kB1Slot)) {
      const int row = kBChunk * (((j >> 1) + rot_b1) % kB1Chunks), kb = 2 * (j & 1);
      unsigned char* dst = sm + kXLo + k * kB1Slot;
      tc::tma_load_2d_hint(dst, &mp->W1[ty], &full[k], 64 * kb, row, keep);
      tc::tma_load_2d_hint(dst + kB1Box, &mp->W1[ty], &full[k], 64 * (kb + 1), row, keep);
    }
    uses[k] += 1;
  }
};

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

// Tile order shared by every role: tile -> (type, first row, rows).
struct TileOf {
  int ty, row0, nrow;
};
__device__ __forceinline__ TileOf tile_of(int tile, const int* s_tiles, const FitArgs& a) {
  int ty = 0;
  while (ty + 1 < a.ntypes && tile >= s_tiles[ty + 1]) ++ty;
  const int k = tile - s_tiles[ty];
  return {ty, a.type_off[ty] + k * kFR, min(kFR, a.type_count[ty] - k * kFR)};
}

// Three warp roles run each tile's pipeline concurrently:
//   warps 9..11 (lane 0) TMA loads into the staging slots, as soon as a slot is free and the
//                        buffer it overlays is no longer read (events rf: L1 MMAs done, B2 MMAs
//                        done, B1 MMAs done);
//   warp 8 (lane 0)      the MMAs of each GEMM once its operands landed and the epilogue that
//                        writes its A operand finished (events epi, alternating barriers);
//   warps 0..7           the epilogues after each GEMM's accumulator is complete (accb).
// Each waits only with bounded polls; a role that gives up sets the shared abort flag and the
// others leave their loops at their next wait.
template <bool F16>
__global__ void __launch_bounds__(kThreads, 1) k_mix_fit(const __grid_constant__ FitMaps maps, FitArgs a) {
  extern __shared__ unsigned char sraw[];
  unsigned char* sm = align1k(sraw);
  float* prm = reinterpret_cast<float*>(sm + kPrm);  // b1, b2, b3, w4 [4][240]
  __shared__ uint64_t full[10], empty[10], accb[2], epib[2], rf[3], fin;
  __shared__ uint32_t tslot;
  __shared__ int s_tiles[kMaxTypes + 1];
  __shared__ int s_abort;
  __shared__ float sE[kFR];
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;

  if (t == 0) {
    for (int q = 0; q < 10; ++q) { tc::mbar_init(&full[q], 1); tc::mbar_init(&empty[q], 1); }
    for (int q = 0; q < 2; ++q) { tc::mbar_init(&accb[q], 1); tc::mbar_init(&epib[q], 1); }
    for (int q = 0; q < 3; ++q) tc::mbar_init(&rf[q], 1);
    tc::mbar_init(&fin, 1);
    tc::mbar_fence_init();
    int acc = 0;
    for (int ty = 0; ty < a.ntypes; ++ty) { s_tiles[ty] = acc; acc += (a.type_count[ty] + kFR - 1) / kFR; }
    s_tiles[a.ntypes] = acc;
    s_abort = 0;
  }
  if (w == 0) { tc::tmem_alloc(&tslot, 512); tc::tmem_relinquish(); }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tslot;
  const int ntiles = s_tiles[a.ntypes];
  volatile int* abort_flag = &s_abort;

  if (w >= kLoadWarp) {
    // ------------------------------------------------------------------ TMA loads
    if (lane == 0) {
      if (w == kLoadWarp) tc::tma_prefetch_desc(&maps.D);
      Loader L;
      L.full = full; L.empty = empty; L.sm = sm; L.mp = &maps; L.lane = w - kLoadWarp; L.err = a.err; L.ok = true;
      for (int q = 0; q < 10; ++q) L.uses[q] = L.issued[q] = 0;
      L.keep = tc::make_policy_evict_last();
      L.stream = tc::make_policy_evict_first();
      L.rot_l1 = blockIdx.x % kL1Jobs;
      L.rot_s = blockIdx.x & 3;
      L.rot_b1 = blockIdx.x % kB1Chunks;
      uint32_t rph[3] = {0, 0, 0};
      auto wait_rf = [&](int r) {
        L.ok = L.ok && tc::mbar_wait(&rf[r], rph[r] & 1u, a.err);
        rph[r] += 1;
      };
      for (int tile = blockIdx.x; tile < ntiles && L.ok && !*abort_flag; tile += gridDim.x) {
        const TileOf T = tile_of(tile, s_tiles, a);
        if (tile != (int)blockIdx.x) wait_rf(2);  // the B1 MMAs of the previous tile read X and the B1 slots
        for (int j = 0; j < kL1Jobs; ++j) L.l1(T.ty, T.row0, j);
        wait_rf(0);  // the split slots overlay L1 slot 2
        for (int g = 0; g < 4; ++g)
          for (int i = 0; i < kSplitJobs; ++i) L.split(T.ty, g, i);
        wait_rf(1);  // the B1 slots overlay X_lo (read by the B2 MMAs) and the split slots
        for (int j = 0; j < kB1Jobs; ++j) L.b1(T.ty, j);
      }
      if (!L.ok) *abort_flag = 1;
      // copies still in flight land before the CTA can finish
      for (int q = 0; q < 10; ++q)
        if (L.issued[q] > 0) tc::mbar_wait(&full[q], (L.issued[q] - 1) & 1u, a.err);
    }
    __syncwarp();
  } else if (w == kMmaWarp) {
    // ------------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t id240 = tc::idesc_f16(128, 240, F16), id160 = tc::idesc_f16(128, kBChunk, F16);
      const int rot_s = blockIdx.x & 3;
      uint32_t uses[10];
      for (int q = 0; q < 10; ++q) uses[q] = 0;
      bool ok = true;
      uint32_t ev = 0;
      auto consume = [&](int k) {
        ok = ok && tc::mbar_wait(&full[k], uses[k] & 1u, a.err);
        tc::tc_fence_after();
        return ok;
      };
      auto release = [&](int k) {
        tc::mma_commit(&empty[k]);
        uses[k] += 1;
      };
      auto wait_epi = [&]() {
        ok = ok && tc::mbar_wait(&epib[ev & 1], (ev >> 1) & 1u, a.err);
        ev += 1;
        tc::tc_fence_after();
        return ok;
      };
      // split GEMM: job i is one K block with the hi or the lo weights, N = 240 (one read of
      // the A operand serves all output columns: a 128 x 128 product would need as many shared
      // memory bytes per clock as the SM has)
      auto issue_split = [&]() {
        for (int i = 0; i < kSplitJobs; ++i) {
          const int s = i % kSSlots, k = kSplitSlot + s;
          if (!consume(k)) return;
          const int kx = ((i >> 1) + rot_s) & 3;
          const uint32_t xh = tc::smem_u32(sm + kXHi + kx * kBlk), xl = tc::smem_u32(sm + kXLo + kx * kBlk);
          const uint32_t wv = tc::smem_u32(sm + kSt + s * kSSlot);
          if ((i & 1) == 0) {  // hi weights: x_hi w_hi + x_lo w_hi
            tc::mma_kblock(tmem, xh, wv, id240, i >= 2, 4);
            tc::mma_kblock(tmem, xl, wv, id240, true, 4);
          } else {             // lo weights: x_hi w_lo
            tc::mma_kblock(tmem, xh, wv, id240, true, 4);
          }
          release(k);
        }
      };
      // B1 chunk n (TMEM region n & 1): four K blocks of dz1 (X_hi) against W1 rows, two jobs
      auto issue_b1 = [&](int n) {
        for (int h = 0; h < 2; ++h) {
          const int k = (2 * n + h) % kB1Slots;
          if (!consume(k)) return;
          const unsigned char* slot = sm + kXLo + k * kB1Slot;
#pragma unroll
          for (int q = 0; q < 2; ++q)
            tc::mma_kblock(tmem + 256 * (n & 1), tc::smem_u32(sm + kXHi + (2 * h + q) * kBlk),
                           tc::smem_u32(slot + q * kB1Box), id160, (h | q) > 0, 4);
          release(k);
        }
        tc::mma_commit(&accb[n & 1]);
      };
      for (int tile = blockIdx.x; tile < ntiles && ok && !*abort_flag; tile += gridDim.x) {
        // L1: z1 = D W1 into columns 0..239 (free: the previous tile's B1 drains are done)
        for (int j = 0; j < kL1Jobs && ok; ++j) {
          const int k = j % kL1Slots;
          if (!consume(k)) break;
          unsigned char* st = sm + k * kL1Slot;
          tc::mma_kblock(tmem, tc::smem_u32(st), tc::smem_u32(st + kBlk), id240, j > 0, 4);
          release(k);
        }
        tc::mma_commit(&accb[0]);
        tc::mma_commit(&rf[0]);
        // L2, L3, B3, B2: each after the epilogue that wrote its A operand
        for (int g = 0; g < 4 && ok; ++g) {
          if (!wait_epi()) break;
          issue_split();
          tc::mma_commit(&accb[0]);
          if (g == 3) tc::mma_commit(&rf[1]);
        }
        // B1 in ten chunks over two TMEM regions: chunk n + 2 once chunk n has been drained
        if (ok && wait_epi()) {
          issue_b1(0);
          issue_b1(1);
          for (int n = 0; n < kB1Chunks && ok; ++n) {
            if (!wait_epi()) break;
            if (n + 2 < kB1Chunks) issue_b1(n + 2);
            if (n + 2 == kB1Chunks - 1) tc::mma_commit(&rf[2]);
          }
        }
      }
      if (!ok) *abort_flag = 1;
      // every MMA has completed before the TMEM is released
      tc::mma_commit(&fin);
      tc::mbar_wait(&fin, 0, a.err);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------------ epilogues
    const int row = t & (kFR - 1), half = t >> 7;  // TMEM lane / atom, column half
    const uint32_t lane_off = (uint32_t)(32 * (w & 3)) << 16;
    const uint32_t acc0 = tmem + lane_off, acc1 = tmem + 256 + lane_off;
    const uint32_t resid = acc1;
    // columns of this thread's half: 16-column chunks [c_beg, c_end) of 15 (240 columns)
    const int c_beg = half ? 8 : 0, c_end = half ? 15 : 8;
    uint32_t aph[2] = {0, 0};
    uint32_t ev = 0;
    bool ok = true;
    int cur_type = -1;
    auto wait_acc = [&](int r) {
      ok = tc::mbar_wait(&accb[r], aph[r], a.err) && ok;
      aph[r] ^= 1u;
      tc::tc_fence_after();
    };
    // all epilogue threads: shared-memory and TMEM writes done, abort decided uniformly
    auto sync_epi = [&]() {
      tc::fence_async_smem();
      tc::tc_fence_before();
      ok = tc::bar_and(1, kEpi, ok && !*abort_flag);
      return ok;
    };
    // ... and the MMA issuer may go on
    auto signal = [&]() {
      if (t == 0) tc::mbar_arrive(&epib[ev & 1]);
      ev += 1;
    };

    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const TileOf T = tile_of(tile, s_tiles, a);
      const int ty = T.ty, row0 = T.row0, nrow = T.nrow;
      const bool valid = row < nrow;
      const size_t grow = (size_t)row0 + row;
      const float* P = a.w + a.fit_base + (long)ty * kFitParams;
      if (ty != cur_type) {
        for (int q = t; q < 4 * kF; q += kEpi) {
          const int which = q / kF, c = q - which * kF;
          const long off = which == 0 ? kFb1 : which == 1 ? kFb2 : which == 2 ? kFb3 : kFw4;
          prm[q] = P[off + c];
        }
        cur_type = ty;
        if (!sync_epi()) break;
      }
      const float* b1 = prm;
      const float* b2 = prm + kF;
      const float* b3 = prm + 2 * kF;
      const float* w4 = prm + 3 * kF;

      // ---- L1 epilogue: h1 = tanh(z1 + b1)
      wait_acc(0);
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
      if (!sync_epi()) break;
      signal();

      // ---- L2 epilogue: h2 = h1 + tanh(h1 W2 + b2)
      wait_acc(0);
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
      if (!sync_epi()) break;
      signal();

      // ---- L3 epilogue: h3 = h2 + tanh(h2 W3 + b3), E_i, dz3
      wait_acc(0);
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
      if (!sync_epi()) break;
      signal();
      if (half == 0 && valid)
        a.e_atom[grow] = (double)e + (double)sE[row] + (double)P[kFb4] + (double)a.w[a.ebias_off + ty];

      // ---- B3 epilogue: dh2 = w4 + dz3 W3^T ; dz2 = dh2 (1 - t2^2)
      {  // this row's 1 - t2^2 factors are fetched while the MMAs run
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
      if (!sync_epi()) break;
      signal();

      // ---- B2 epilogue: dh1 = dh2 + dz2 W2^T ; dz1 = dh1 (1 - h1^2), X_hi only (B1 is a plain
      //      16-bit GEMM; its weights stream into X_lo meanwhile)
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
            store_x16<F16>(sm, row, 16 * cc, f, false);
          }
        }
      }
      if (!sync_epi()) break;
      signal();

      // ---- B1 drains: dE/dD = dz1 W1^T, chunk n from TMEM region n & 1 through the staging tile
      for (int n = 0; n < kB1Chunks; ++n) {
        const int rg = n & 1;
        wait_acc(rg);
        const uint32_t src = rg ? acc1 : acc0;
        {  // this thread's 80 columns of its row (fp16): five TMEM loads in flight, one wait
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
        if (!sync_epi()) break;
        // TMEM region n & 1 is free: chunk n + 2 may start under the write-out
        if (n + 1 < kB1Chunks) signal();
        // whole row segments (320 B) to dE/dD: warp w writes rows w, w + 8, ...; lanes 0..19
        {
          const int col0 = kBChunk * (((blockIdx.x % kB1Chunks) + n) % kB1Chunks);
          for (int r = w; r < nrow; r += kEpi / 32)
            if (lane < kBChunk / 8) {
              const uint4 v = *reinterpret_cast<const uint4*>(sm + kStage + r * kStageRow + 16 * lane);
              __stcs(reinterpret_cast<uint4*>(a.dD + (size_t)(row0 + r) * kKD + col0 + 8 * lane), v);
            }
        }
        if (!sync_epi()) break;
        // the last chunk's signal also frees the staging tile, which the next tile's split
        // slots overlay
        if (n + 1 == kB1Chunks) signal();
      }
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
static_assert(kL1Slots * kL1Slot <= kStage, "L1 slots overlap the dE/dD staging tile");
static_assert(kStage + kFR * kStageRow <= kPrm, "dE/dD staging tile overlaps the parameters");
static_assert(kXLo + kB1Slots * kB1Slot <= kStage, "B1 slots overlap the dE/dD staging tile");


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
        ok = ok && make_map(&fm->S[ty][g][h], S + (size_t)(2 * g + h) * kF * kF, f16, kF, kF, kF);
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
