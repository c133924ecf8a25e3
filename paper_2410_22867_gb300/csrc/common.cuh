// Internal declarations shared by the CUDA translation units of libdpgb300.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dp.h"

namespace dpg {

// Network sizes fixed by the model (Section II-A; fitting widths of Section IV).
constexpr int kN1 = 25, kN2 = 50, kN3 = 100, kM2 = 16;
constexpr int kF = 240;
constexpr int kKD = kN3 * kM2;  // 1600, descriptor length
constexpr int kEmbParams = kN1 + kN1 + kN1 * kN2 + kN2 + kN2 * kN3 + kN3;       // 6450
constexpr int kFitParams = kKD * kF + kF + kF * kF + kF + kF * kF + kF + kF + 1;  // 500161
constexpr int kMaxTypes = 4;
constexpr int kRdfMaxCells = 24576;  // dp_rdf: ntypes^2 * nbins histogram cells at most
// parameter gradient: centre atoms per chunk, neighbour rows per chunk of the embedding reverse
constexpr int kPgAtoms = 2048, kPgRows = 16384;

// offsets inside one embedding block
constexpr int kEW1 = 0, kEb1 = kN1, kEW2 = 2 * kN1, kEb2 = kEW2 + kN1 * kN2, kEW3 = kEb2 + kN2,
              kEb3 = kEW3 + kN2 * kN3;
// offsets inside one fitting block
constexpr long kFW1 = 0, kFb1 = (long)kKD * kF, kFW2 = kFb1 + kF, kFb2 = kFW2 + kF * kF,
               kFW3 = kFb2 + kF, kFb3 = kFW3 + kF * kF, kFw4 = kFb3 + kF, kFb4 = kFw4 + kF;

// sticky device error bits
enum : int { ERR_SEL = 1, ERR_SKIN = 2, ERR_VCAP = 4, ERR_TIMEOUT = 8, ERR_CELLCAP = 16, ERR_TYPE = 32 };

// 32-byte aligned FP64 4-vector (positions, velocities, pair vectors).
struct __align__(32) dvec4 {
  double x, y, z, w;
};
__host__ __device__ __forceinline__ dvec4 make_dvec4(double x, double y, double z, double w) {
  dvec4 r;
  r.x = x; r.y = y; r.z = z; r.w = w;
  return r;
}

// Fixed-point position (x * 2^32, rounded) for exact pair vectors without FP64 arithmetic.
struct __align__(32) qvec4 {
  long long x, y, z, w;
};

// Per-replica geometry (orthorhombic box and cell grid).
// Periodic cell of one replica: cell vectors a, b, c as the rows of H; an image n = (n0, n1, n2)
// of an atom sits at x + n H, each component summed as ((n0 H0c + n1 H1c) + n2 H2c), which for
// an orthorhombic cell is n_c L_c exactly.
struct RepGeom {
  double H[9];        // cell vectors (rows)
  double Hinv[9];     // fractional coordinates s = x Hinv (row vector)
  double L[3];        // diagonal of H: the edges of an orthorhombic cell
  long long Hq[9];    // H in fixed point (H * 2^32, rounded)
  float Hf[9];        // H in fp32
  int nc[3];          // cells per axis
  int m[3];           // stencil half width per axis
  double edge[3];     // cell edge (orthorhombic, A) or 1 / nc (triclinic, fractional)
  int tri;            // 1: some off-diagonal entry of H is nonzero (cells in fractional coordinates)
  int cell_off;       // first global cell id of this replica
  int atom_off;       // first caller-order atom of this replica
  int natoms;
};

struct Model {
  // configuration
  int ntypes = 0, switch_kind = 0;
  double rc = 0, rs = 0, skin = 0;
  int sel[kMaxTypes] = {0}, sel_off[kMaxTypes + 1] = {0}, S = 0;
  int vcap[kMaxTypes] = {0}, vcap_off[kMaxTypes + 1] = {0}, VS = 0;
  dp_precision prec = DP_FP64;
  int max_atoms = 0, max_reps = 0, max_cells = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;  // owned; graphs are captured here, replayed on `stream`
  std::string last_error;
  long long ntheta = 0;
  std::vector<double> theta_host;
  std::vector<double> davg_host, dstd_host;

  // weights (device)
  double* w64 = nullptr;      // theta FP64 (blob order)
  float* w32 = nullptr;       // theta FP32
  double* fitT64 = nullptr;   // per type: W1^T [kF][kKD], W2^T [kF][kF], W3^T [kF][kF]
  float* fitT32 = nullptr;
  double* stat64 = nullptr;   // davg [nt][4], 1/dstd [nt][4]
  float* stat32 = nullptr;
  // One padded neighbour slot's contribution to S*T per (ti, tj): R_pad^T G(R_pad_0), c-major
  // [nt][nt][4][100], with R_pad = -davg[ti] / dstd[ti] (the normalised zero row).  Padded slots
  // add (sel[tj] - count) times it.  has_pad is false when every davg is 0 (then R_pad = 0).
  double* pad64 = nullptr;
  float* pad32 = nullptr;
  bool has_pad = false;
  // Tabulated embedding (dp_tabulate): tab_n > 0 intervals of width tab_h from tab_x0; quintic
  // coefficients [pair][interval][100][8] in FP64 and FP32 (tab.cu).  tab_mem owns both.
  int tab_n = 0;
  double tab_x0 = 0.0, tab_h = 0.0;
  unsigned long long* rdf_hist = nullptr;  // [kRdfMaxCells] pair-distance histogram (dp_rdf)
  double* tab64 = nullptr;
  float* tab32 = nullptr;
  void* tab_mem = nullptr;
  // 16-bit operand copies for the tensor-core kernels (per type), laid out by those kernels
  void* tc_weights = nullptr;
  void* emb_img = nullptr;    // mixed precision: per embedding pair, the forward's MMA operand
                              // blocks in their shared-memory byte layout
  size_t tc_weights_bytes = 0;

  // atoms (internal, type-sorted order)
  int* perm = nullptr;        // internal -> caller index
  bool nearest = false;       // nearest-first sel truncation instead of DP_ERR_SEL_OVERFLOW
  int* inv = nullptr;         // caller -> internal index
  int* itype = nullptr;
  int* irep = nullptr;
  int* type_count = nullptr;  // [kMaxTypes + 1] device: counts then total (offsets are derived)
  int* type_off = nullptr;    // [kMaxTypes + 1]
  int* blk_count = nullptr;   // scratch for the type sort
  dvec4* x = nullptr;       // positions (wrapped at rebuild, drifting between)
  dvec4* xref = nullptr;    // positions at the last rebuild
  dvec4* v = nullptr;       // velocities
  float4* delta = nullptr;    // x - xref in fp32
  float4* xf = nullptr;       // wrapped positions in fp32 (rebuild prefilter)
  qvec4* xq = nullptr;        // wrapped positions at rebuild in fixed point (x * 2^32)
  double* force = nullptr;    // [N*3]
  double* mass = nullptr;     // [N] per internal atom

  // replicas
  RepGeom* geom = nullptr;    // device [max_reps]
  RepGeom* geom_host = nullptr;  // the current geometry: one of the two staging buffers below
  RepGeom* geom_stage[2] = {nullptr, nullptr};  // pinned host staging, written alternately
  cudaEvent_t geom_ev[2] = {nullptr, nullptr};  // recorded after the copies out of each buffer
  int nrep = 0;
  int max_rep_atoms = 0;      // atoms of the largest replica (chunks of the per-replica sums)
  int ncells = 0;
  double* red_part = nullptr;  // per-replica sums: chunk partials [nrep][nchunk][10]
  size_t red_cap = 0;          // chunk slots of red_part

  // cell list
  int* cell_of = nullptr;
  int* cell_count = nullptr;
  int* cell_start = nullptr;
  int* cell_fill = nullptr;
  int* cell_atoms = nullptr;
  float4* cell_xf = nullptr;  // [N] FP32 positions in cell order (beside cell_atoms)

  // Verlet list (r_c + skin)
  float4* vl_e = nullptr;     // [N*VS] pair vector at rebuild (fp32), w = neighbour index
  int* vl_img = nullptr;      // [N*VS] image code
  int* vl_work = nullptr;     // [N + 1] atoms the per-atom Verlet kernel builds, their count last
  int* vcount = nullptr;      // [N*nt]

  // formatted list (r_c), compacted per type segment
  int* nl_j = nullptr;        // [N*S]
  int* nl_img = nullptr;      // [N*S] image codes, written only for dp_get_nlist
  void* nl_d = nullptr;       // [N*S] float4 (fp32 modes) or dvec4 (fp64)
  int* nl_count = nullptr;    // [N*nt]

  // descriptor and fitting buffers (element type depends on precision)
  void* Tm = nullptr;         // [N][4][kN3]
  void* Dm = nullptr;         // [N][kKD]
  void* dD = nullptr;         // [N][kKD]
  void* act[5] = {nullptr};   // fitting activations [N][kF]
  double* e_atom = nullptr;   // [N] internal order
  double* vir_atom = nullptr; // [N][9] internal order
  double* e_user = nullptr;   // [N] caller order
  double* vir_user = nullptr; // [N][9] caller order
  double* ke_user = nullptr;  // [N] caller order
  double* red_out = nullptr;  // [max_reps * 20] reductions scratch
  int* rep_off_dev = nullptr; // [max_reps + 1]
  int* err = nullptr;         // sticky error word
  int* err_host = nullptr;    // pinned
  int* small_i = nullptr;     // [64] device: small integer tables (sel, offsets)
  // mixed-precision path
  int* rowoff = nullptr;      // [nt][N + 1] row offsets of each atom in the per-type neighbour streams
  int* scan_blk = nullptr;    // [nt][N / 1024 + 1]
  float* Tseg = nullptr;      // [nt][N][400] partial T per neighbour type
  void* dTm = nullptr;        // [N][100] float4
  float* force32 = nullptr;   // [N*4] FP32 force accumulator of the mixed-precision backward (x y z pad)
  double* vir_rep = nullptr;  // [max_reps][9] per-replica virial accumulated by the mixed backward
  // parameter gradient
  void* pg_ws = nullptr;      // per-chunk activations and adjoints (FP64 or FP32)
  int pg_cap = 0;             // centre atoms per chunk
  int* pg_roff = nullptr;     // row offsets of every row chunk of one call
  size_t pg_roff_cap = 0;
  double* pg_w = nullptr;     // [N][3] tangent direction 2 cF (F - F0), internal order
  double* pg_scal = nullptr;  // alpha, loss, E

  // MD bookkeeping
  int natoms = 0;             // atoms of the current call
  bool lists_valid = false;
  bool md_valid = false;      // internal x, v, F, lists belong to the last MD call
  long long launches = 0;     // kernels launched (graph replays add their kernel count)
  cudaEvent_t sub_ev[2] = {nullptr, nullptr};  // set only inside dp_phase_times: kernel-level split
  // launch grids chosen by dp_autotune (0 = occupancy default): embedding forward,
  // embedding backward, dE/dT, descriptor
  int tune_grid[4] = {0, 0, 0, 0};
  unsigned long long tuned_key = 0;
  // captured MD steps (between rebuilds, with a rebuild) and the configuration they were
  // captured for; owned by the model and destroyed with it
  struct GraphCache {
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    long long kernels[2] = {0, 0};
    int N = -1, nrep = -1;
    double dt = 0;
    unsigned long long geom_hash = 0;
  } graphs;
  void* fit_maps = nullptr;   // tensor maps of the mixed fitting kernel (mix_fit.cu), owned
  // every device / pinned host allocation of dp_create, released by dp_destroy
  std::vector<void*> dev_allocs, host_allocs;
};

// ---------------------------------------------------------------------------
// error helpers
#define DP_CUDA_TRY(m, call)                                                       \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      (m)->last_error = std::string(#call) + ": " + cudaGetErrorString(e_);        \
      return DP_ERR_CUDA;                                                          \
    }                                                                              \
  } while (0)

#define DP_LAUNCH_CHECK(m)                                                         \
  do {                                                                             \
    cudaError_t e_ = cudaGetLastError();                                           \
    if (e_ != cudaSuccess) {                                                       \
      (m)->last_error = std::string("kernel launch: ") + cudaGetErrorString(e_);   \
      return DP_ERR_CUDA;                                                          \
    }                                                                              \
  } while (0)

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// Raise a kernel's dynamic shared-memory limit once (not from inside stream capture
// after the first call: the attribute call is skipped when already large enough).
inline cudaError_t ensure_smem(const void* fn, size_t smem) {
  static std::mutex mu;  // models may be driven from several host threads
  static std::vector<std::pair<const void*, size_t>> done;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& e : done)
    if (e.first == fn && e.second >= smem) return cudaSuccess;
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err == cudaSuccess)  // prefer the largest shared-memory carveout so several CTAs fit per SM
    err = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (err == cudaSuccess) done.push_back({fn, smem});
  return err;
}

// Resident blocks per SM for a launch shape, from the kernel's registers and static
// shared memory, the dynamic shared memory, and an optional TMEM column budget
// (tcgen05 kernels hold `tmem_cols` of the SM's 512 columns each).  Cached.
inline int blocks_per_sm(const void* fn, int threads, size_t smem, int tmem_cols = 0) {
  struct E { const void* f; int t; size_t s; int c; int n; };
  static std::mutex mu;
  static std::vector<E> cache;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& e : cache)
    if (e.f == fn && e.t == threads && e.s == smem && e.c == tmem_cols) return e.n;
  int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaFuncAttributes fa;
  int n = 1;
  if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess && smem_sm > 0 && regs_sm > 0) {
    const size_t per_block = smem + fa.sharedSizeBytes + 1024;  // 1 KB reserved per block
    const int regs = ((fa.numRegs + 7) / 8) * 8 * threads;       // allocation granularity 8 per thread
    n = (int)(smem_sm / per_block);
    if (regs > 0) n = std::min(n, regs_sm / regs);
    if (thr_sm > 0) n = std::min(n, thr_sm / threads);
    if (tmem_cols > 0) n = std::min(n, 512 / tmem_cols);
    n = std::max(1, std::min(n, 32));
  }
  cache.push_back({fn, threads, smem, tmem_cols, n});
  return n;
}

inline int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}
__host__ __device__ __forceinline__ int cdiv_dev(int a, int b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// host-side launchers (each returns DP_OK or DP_ERR_CUDA)
// nlist.cu
dp_status launch_type_sort(Model* m, const int* types_user, int N);
dp_status launch_load_positions(Model* m, const double* coords_user, int N);
// Cell binning and the Verlet list of every atom.  with_skin: pairs within r_c + skin (MD: the
// list serves the next steps); otherwise within r_c (a single evaluation: the list is rebuilt on
// every call, so the skin would only add entries).
dp_status launch_rebuild(Model* m, int N, bool with_skin);
dp_status launch_delta(Model* m, int N);
dp_status launch_format(Model* m, int N, bool images = false);  // images: also the image codes
dp_status launch_get_nlist(Model* m, int N, int* nlist, int* images);
// tab.cu
dp_status launch_tabulate(Model* m, double x0, double x1, int n);
// diag.cu
dp_status launch_rdf(Model* m, int nbins, double r_max, unsigned long long* hist_dev);
dp_status launch_atom_virial_out(Model* m, int N, double* out);
// mix_embed.cu: the embedding backward again, accumulating only the per-atom (centre) virial into vir_atom
dp_status launch_mix_atom_virial(Model* m, int N);  // synchronous; n = 0 drops the table
// simt.cu
dp_status launch_pad_rows(Model* m);  // pad64 / pad32 from the current weights (synchronous caller)
dp_status launch_descriptor(Model* m, int N);
dp_status launch_fitting(Model* m, int N);
dp_status launch_embed_backward(Model* m, int N);
// mix_embed.cu (tensor-core embedding net)
dp_status launch_mix_descriptor(Model* m, int N);
dp_status launch_mix_embed_backward(Model* m, int N);
// mix_fit.cu (tensor-core fitting net)
dp_status mix_fit_setup(Model* m);
size_t mix_fit_weight_bytes(int ntypes);
size_t mix_emb_image_bytes(int ntypes);
dp_status launch_emb_images(Model* m);
dp_status launch_mix_fitting(Model* m, int N);
void mix_fit_release(Model* m);
// grid of a tunable mixed kernel: the autotuned value if set, else the default
inline int tuned_grid(const Model* m, int which, int dflt) { return m->tune_grid[which] > 0 ? m->tune_grid[which] : dflt; }
// parameter gradient (pgrad.cu)
size_t param_grad_workspace_bytes(int cap, bool fp64);
dp_status launch_param_grad(Model* m, int N, const double* F0, double E0, double cE, double cF, double* grad,
                            double* loss);
inline bool is_mixed(const Model* m) { return m->prec == DP_MIX_BF16 || m->prec == DP_MIX_FP16; }
// md.cu
dp_status launch_outputs(Model* m, int N, double* energy_rep, double* atom_energy, double* forces,
                         double* virial_rep);
dp_status launch_zero_forces(Model* m, int N);
dp_status launch_kick_drift(Model* m, int N, double dt);
dp_status launch_kick(Model* m, int N, double dt);
dp_status launch_load_state(Model* m, int N, const double* v_user, const double* mass_by_type);
dp_status launch_store_state(Model* m, int N, double* x_user, double* v_user);
dp_status launch_kinetic(Model* m, int N, double* ke_rep);
size_t rep_reduce_slots(int max_atoms, int max_reps);  // chunk slots of red_part (10 doubles each)
dp_status launch_nan_energy(Model* m, double* energy, int n);

}  // namespace dpg
