// C-ABI entry points (declared in include/dp.h): model creation from a weight
// blob, force evaluation, batched evaluation, velocity-Verlet MD with CUDA-graph
// replay, neighbour-list export, error reporting.  All device memory is
// allocated in dp_create (Section III-B1: memory for all computations is
// allocated in the initial phase, no dynamic allocation during the run).
#include <cmath>
#include <cstdio>
#include <array>
#include <cstring>
#include <map>
#include <mutex>

#include "common.cuh"

namespace dpg {

dp_status launch_tc_setup(Model* m);  // tensor-core weights (tc kernels)
bool tc_available(const Model* m);

namespace {

template <class P>
dp_status dalloc(Model* m, P** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    m->last_error = std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e);
    return DP_ERR_OOM;
  }
  m->dev_allocs.push_back(q);
  *p = static_cast<P*>(q);
  return DP_OK;
}

template <class P>
dp_status halloc(Model* m, P** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMallocHost(&q, bytes);
  if (e != cudaSuccess) {
    m->last_error = std::string("cudaMallocHost: ") + cudaGetErrorString(e);
    return DP_ERR_OOM;
  }
  m->host_allocs.push_back(q);
  *p = static_cast<P*>(q);
  return DP_OK;
}

#define DP_TRY(x)                     \
  do {                                \
    dp_status s_ = (x);               \
    if (s_ != DP_OK) return s_;       \
  } while (0)

// ------------------------------------------------------------------ weight blob
struct Parsed {
  int ntypes = 0, switch_kind = 0;
  double rc = 0, rs = 0;
  int emb[3] = {0, 0, 0}, axis = 0, fit[3] = {0, 0, 0};
  std::vector<int> sel;
  std::vector<std::string> names;
  std::vector<double> theta, davg, dstd;
};

dp_status parse_blob(const unsigned char* p, size_t n, Parsed& o, std::string& why) {
  auto need = [&](size_t end) { return end <= n; };
  if (!need(64) || std::memcmp(p, "DPW1", 4) != 0) { why = "bad magic or truncated header"; return DP_ERR_WEIGHTS; }
  int32_t ver, nt, sk;
  std::memcpy(&ver, p + 4, 4); std::memcpy(&nt, p + 8, 4); std::memcpy(&sk, p + 12, 4);
  if (ver != 1 || nt < 1 || nt > kMaxTypes) { why = "unsupported version or ntypes"; return DP_ERR_WEIGHTS; }
  o.ntypes = nt; o.switch_kind = sk;
  std::memcpy(&o.rc, p + 16, 8); std::memcpy(&o.rs, p + 24, 8);
  std::memcpy(o.emb, p + 32, 12); std::memcpy(&o.axis, p + 44, 4); std::memcpy(o.fit, p + 48, 12);
  size_t off = 64;
  size_t nsel = (size_t)nt + (nt % 2);
  if (!need(off + 4 * nsel + 8 * (size_t)nt)) { why = "truncated sel/type names"; return DP_ERR_WEIGHTS; }
  o.sel.resize(nt);
  std::memcpy(o.sel.data(), p + off, 4 * (size_t)nt);
  off += 4 * nsel;
  for (int t = 0; t < nt; ++t) {
    char buf[9] = {0};
    std::memcpy(buf, p + off + 8 * t, 8);
    o.names.push_back(buf);
  }
  off += 8 * (size_t)nt;
  if (o.emb[0] != kN1 || o.emb[1] != kN2 || o.emb[2] != kN3 || o.axis != kM2 || o.fit[0] != kF ||
      o.fit[1] != kF || o.fit[2] != kF) {
    why = "network sizes differ from 25/50/100, axis 16, fitting 240x3";
    return DP_ERR_UNSUPPORTED;
  }
  size_t ntheta = (size_t)nt * nt * kEmbParams + (size_t)nt * kFitParams + nt;
  if (!need(off + 8 * (ntheta + 8 * (size_t)nt))) { why = "truncated parameters"; return DP_ERR_WEIGHTS; }
  o.theta.resize(ntheta);
  std::memcpy(o.theta.data(), p + off, 8 * ntheta);
  off += 8 * ntheta;
  o.davg.resize(4 * nt); o.dstd.resize(4 * nt);
  std::memcpy(o.davg.data(), p + off, 8 * 4 * (size_t)nt); off += 8 * 4 * (size_t)nt;
  std::memcpy(o.dstd.data(), p + off, 8 * 4 * (size_t)nt);
  for (double s : o.dstd)
    if (!(s > 0)) { why = "dstd must be positive"; return DP_ERR_WEIGHTS; }
  return DP_OK;
}

// ------------------------------------------------------------------ replicas
// with_skin: cells for the r_c + skin list of an MD run; otherwise for the r_c list of a single
// evaluation (smaller cells, fewer candidates per atom).
dp_status setup_replicas(Model* m, int nrep, const int* offs, const double* boxes, int N, bool with_skin) {
  if (nrep < 1 || nrep > m->max_reps) { m->last_error = "nrep out of range"; return DP_ERR_CAPACITY; }
  // Two pinned staging buffers, written alternately: the one written now fed the copies of the
  // call before last, and the event recorded after those copies has (almost always) completed,
  // so consecutive calls do not wait for the device.  The current one is switched only on success.
  const int sb = (m->geom_host == m->geom_stage[0]) ? 1 : 0;
  DP_CUDA_TRY(m, cudaEventSynchronize(m->geom_ev[sb]));
  RepGeom* gh = m->geom_stage[sb];
  int* off_h = reinterpret_cast<int*>(gh + m->max_reps);
  const double rcs = m->rc + (with_skin ? m->skin : 0.0);
  // Cells of edge >= (r_c + skin) / 2 and a 5 x 5 x 5 stencil when they fit the allocated cell
  // list (about half the candidates of edge >= r_c + skin with 3 x 3 x 3), else full-size cells.
  int cells = 0;
  for (int div = 2; div >= 1; --div) {
    cells = 0;
    for (int r = 0; r < nrep; ++r) {
      const double* b = boxes + 9 * r;
      RepGeom& g = gh[r];
      std::memset(&g, 0, sizeof(g));
      // any right-handed cell: finite entries, positive volume; inverse = adjugate / det
      double cof[9];
      for (int q = 0; q < 9; ++q) {
        if (!std::isfinite(b[q]) || std::fabs(b[q]) >= 268435456.0) {
          m->last_error = "box entries must be finite and below 2^28 A";
          return DP_ERR_ARG;
        }
        g.H[q] = b[q];
        g.Hf[q] = (float)b[q];
        g.Hq[q] = std::llrint(b[q] * 4294967296.0);
      }
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c)
          if (a != c && b[3 * a + c] != 0.0) g.tri = 1;
      cof[0] = b[4] * b[8] - b[5] * b[7];
      cof[1] = b[5] * b[6] - b[3] * b[8];
      cof[2] = b[3] * b[7] - b[4] * b[6];
      cof[3] = b[2] * b[7] - b[1] * b[8];
      cof[4] = b[0] * b[8] - b[2] * b[6];
      cof[5] = b[1] * b[6] - b[0] * b[7];
      cof[6] = b[1] * b[5] - b[2] * b[4];
      cof[7] = b[2] * b[3] - b[0] * b[5];
      cof[8] = b[0] * b[4] - b[1] * b[3];
      const double det = (b[0] * cof[0] + b[1] * cof[1]) + b[2] * cof[2];
      if (!(det > 0.0)) { m->last_error = "the box must be a right-handed cell of positive volume"; return DP_ERR_ARG; }
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) g.Hinv[3 * a + c] = cof[3 * c + a] / det;
      const double eff = rcs * (1.0 + 1e-9);
      int ncr = 1;
      for (int a = 0; a < 3; ++a) {
        g.L[a] = b[4 * a];
        if (!g.tri && !(g.L[a] > 0.0)) { m->last_error = "box length must be positive"; return DP_ERR_ARG; }
        // perpendicular width of the cell along axis a: V / |cross product of the other rows|
        const double* k = cof + 3 * a;
        const double width = g.tri ? det / std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]) : g.L[a];
        int nc = (int)std::floor(div * width / eff);
        if (nc < 1) nc = 1;
        if (nc > 1024) nc = 1024;
        g.nc[a] = nc;
        // triclinic cells are binned by fractional coordinate, one more stencil layer covers an
        // atom whose rounded fractional coordinate lands in the neighbouring cell
        g.edge[a] = g.tri ? 1.0 / nc : g.L[a] / nc;
        g.m[a] = (int)std::ceil(eff / (width / nc)) + g.tri;
        if (g.m[a] > 200) { m->last_error = "box too small for the cutoff"; return DP_ERR_UNSUPPORTED; }
        ncr *= nc;
      }
      g.cell_off = cells;
      g.atom_off = offs ? offs[r] : 0;
      g.natoms = offs ? offs[r + 1] - offs[r] : N;
      cells += ncr;
      off_h[r] = g.atom_off;
    }
    if (cells <= m->max_cells) break;
  }
  off_h[nrep] = offs ? offs[nrep] : N;
  if (off_h[nrep] != N || off_h[0] != 0) { m->last_error = "atom_offsets must run from 0 to natoms"; return DP_ERR_ARG; }
  for (int r = 0; r < nrep; ++r)
    if (off_h[r + 1] < off_h[r]) { m->last_error = "atom_offsets must be non-decreasing"; return DP_ERR_ARG; }
  if (cells > m->max_cells) { m->last_error = "too many cells for the allocated cell list"; return DP_ERR_CAPACITY; }
  m->nrep = nrep;
  m->ncells = cells;
  m->max_rep_atoms = 0;
  for (int r = 0; r < nrep; ++r) m->max_rep_atoms = std::max(m->max_rep_atoms, off_h[r + 1] - off_h[r]);
  DP_CUDA_TRY(m, cudaMemcpyAsync(m->geom, gh, sizeof(RepGeom) * nrep, cudaMemcpyHostToDevice, m->stream));
  DP_CUDA_TRY(m, cudaMemcpyAsync(m->rep_off_dev, off_h, sizeof(int) * (nrep + 1), cudaMemcpyHostToDevice,
                                 m->stream));
  DP_CUDA_TRY(m, cudaEventRecord(m->geom_ev[sb], m->stream));
  m->geom_host = gh;
  return DP_OK;
}

// One force evaluation on the current internal positions (lists already valid):
// format -> descriptor -> fitting -> embedding backward (forces, virials).
dp_status force_eval(Model* m, int N) {
  DP_TRY(launch_format(m, N));
  DP_TRY(launch_zero_forces(m, N));
  DP_TRY(launch_descriptor(m, N));
  DP_TRY(launch_fitting(m, N));
  DP_TRY(launch_embed_backward(m, N));
  return DP_OK;
}

dp_status map_err_bits(Model* m, int bits) {
  if (!bits) return DP_OK;
  std::string s = "device error:";
  if (bits & ERR_TYPE) s += " atom type out of range;";
  if (bits & ERR_SEL) s += " neighbour count above sel;";
  if (bits & ERR_SKIN) s += " atom moved more than skin/2 since the last rebuild;";
  if (bits & ERR_VCAP) s += " Verlet list capacity exceeded;";
  if (bits & ERR_CELLCAP) s += " cell capacity exceeded;";
  if (bits & ERR_TIMEOUT) s += " bounded wait timed out;";
  m->last_error = s;
  if (bits & ERR_TYPE) return DP_ERR_ARG;
  if (bits & ERR_SEL) return DP_ERR_SEL_OVERFLOW;
  if (bits & ERR_SKIN) return DP_ERR_SKIN_EXCEEDED;
  if (bits & ERR_TIMEOUT) return DP_ERR_WAIT_TIMEOUT;
  return DP_ERR_CAPACITY;
}

dp_status md_step(Model* m, int N, double dt, bool rebuild) {
  DP_TRY(launch_kick_drift(m, N, dt));
  if (rebuild) {
    DP_TRY(launch_rebuild(m, N, true));
  } else {
    DP_TRY(launch_delta(m, N));
  }
  DP_TRY(force_eval(m, N));
  DP_TRY(launch_kick(m, N, dt));
  return DP_OK;
}

void drop_graphs(Model* m) {
  Model::GraphCache& g = m->graphs;
  for (auto& e : g.exec)
    if (e) { cudaGraphExecDestroy(e); e = nullptr; }
  g.N = -1;
}

unsigned long long hash_geom(const Model* m) {
  unsigned long long h = 1469598103934665603ull;
  const unsigned char* p = reinterpret_cast<const unsigned char*>(m->geom_host);
  for (size_t k = 0; k < sizeof(RepGeom) * m->nrep; ++k) h = (h ^ p[k]) * 1099511628211ull;
  return h;
}

dp_status capture_step(Model* m, int N, double dt, bool rebuild, cudaGraphExec_t* out, long long* kernels) {
  cudaGraph_t graph = nullptr;
  // capture on the model's own stream (the caller's may be the uncapturable legacy stream)
  cudaStream_t user = m->stream;
  m->stream = m->capture_stream;
  cudaError_t e0 = cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal);
  if (e0 != cudaSuccess) {
    m->stream = user;
    m->last_error = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e0);
    return DP_ERR_CUDA;
  }
  const long long before = m->launches;
  dp_status st = md_step(m, N, dt, rebuild);
  *kernels = m->launches - before;  // counted when the graph is replayed, not now
  m->launches = before;
  cudaError_t e = cudaStreamEndCapture(m->stream, &graph);
  m->stream = user;
  if (st != DP_OK) { if (graph) cudaGraphDestroy(graph); return st; }
  if (e != cudaSuccess) { m->last_error = std::string("stream capture: ") + cudaGetErrorString(e); return DP_ERR_CUDA; }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) { m->last_error = std::string("graph instantiate: ") + cudaGetErrorString(e); return DP_ERR_CUDA; }
  return DP_OK;
}

// ---------------------------------------------------------------- autotuner
// Launch grids of the mixed-precision kernels whose shape is a real choice: the two embedding
// kernels (CTAs per SM, which also sets the length of each CTA's contiguous row chunk and so
// the balance between tail effects and atoms split across CTAs), the dE/dT and the descriptor
// kernels.  Each candidate is timed over full force evaluations on the model's current state
// (CUDA events on its stream); the fastest is kept.  Choices are cached per process by
// (precision, atoms, replicas, types, SMs).
std::mutex g_tune_mu;
std::map<unsigned long long, std::array<int, 4>> g_tune_cache;

unsigned long long tune_key(const Model* m, int N) {
  unsigned long long k = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) { k = (k ^ v) * 1099511628211ull; };
  mix((unsigned long long)m->prec); mix((unsigned long long)N); mix((unsigned long long)m->nrep);
  mix((unsigned long long)m->ntypes); mix((unsigned long long)num_sms()); mix((unsigned long long)m->tab_n);
  return k == 0 ? 1 : k;
}

dp_status autotune(Model* m, int N, int repeats) {
  if (!is_mixed(m)) return DP_OK;  // the SIMT paths have no tunable launch shapes
  const int sms = num_sms();
  const std::vector<int> cand[4] = {{1 * sms, 2 * sms, 3 * sms, 6 * sms},
                                    {1 * sms, 2 * sms, 3 * sms, 6 * sms},
                                    {2 * sms, 4 * sms, 5 * sms, 10 * sms},
                                    {4 * sms, 8 * sms, 16 * sms}};
  cudaEvent_t e0, e1;
  DP_CUDA_TRY(m, cudaEventCreate(&e0));
  DP_CUDA_TRY(m, cudaEventCreate(&e1));
  dp_status st = DP_OK;
  for (int k = 0; k < 4 && st == DP_OK; ++k) {
    float best = 1e30f;
    int pick = 0;
    for (int c : cand[k]) {
      m->tune_grid[k] = c;
      if ((st = force_eval(m, N)) != DP_OK) break;  // warm
      cudaEventRecord(e0, m->stream);
      for (int r = 0; r < repeats && st == DP_OK; ++r) st = force_eval(m, N);
      cudaEventRecord(e1, m->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { m->last_error = "autotune timing failed"; st = DP_ERR_CUDA; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (st == DP_OK && ms < best) { best = ms; pick = c; }
    }
    m->tune_grid[k] = pick;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == DP_OK) st = force_eval(m, N);  // leave forces of the chosen configuration
  return st;
}

// Apply cached choices or tune; returns whether the launch configuration changed.
dp_status ensure_tuned(Model* m, int N, bool* changed) {
  *changed = false;
  if (!is_mixed(m)) return DP_OK;
  const unsigned long long key = tune_key(m, N);
  if (m->tuned_key == key) return DP_OK;
  std::array<int, 4> old{m->tune_grid[0], m->tune_grid[1], m->tune_grid[2], m->tune_grid[3]};
  bool hit = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      for (int k = 0; k < 4; ++k) m->tune_grid[k] = it->second[k];
      hit = true;
    }
  }
  if (hit) {
    DP_TRY(force_eval(m, N));
  } else {
    DP_TRY(autotune(m, N, 3));
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = {m->tune_grid[0], m->tune_grid[1], m->tune_grid[2], m->tune_grid[3]};
  }
  m->tuned_key = key;
  for (int k = 0; k < 4; ++k) *changed = *changed || (old[k] != m->tune_grid[k]);
  return DP_OK;
}

dp_status run_md(Model* m, dp_md_state* st, double dt, int nsteps, int capture, bool tune = false) {
  if (!st || !st->x || !st->v || !st->types || !st->mass_by_type || !st->boxes) {
    m->last_error = "dp_md_state has a null pointer";
    return DP_ERR_ARG;
  }
  const int N = st->natoms;
  if (N < 1 || N > m->max_atoms) { m->last_error = "natoms out of range"; return DP_ERR_CAPACITY; }
  if (st->rebuild_every < 1 || nsteps < 0 || !(dt > 0)) { m->last_error = "bad MD parameters"; return DP_ERR_ARG; }
  for (int t = 0; t < m->ntypes; ++t)
    if (!(st->mass_by_type[t] > 0)) { m->last_error = "masses must be positive"; return DP_ERR_ARG; }
  int nrep = st->atom_offsets ? st->nrep : 1;
  const bool resume = st->resume && m->md_valid && m->natoms == N && m->nrep == nrep;
  if (st->resume && !resume) {
    m->last_error = "resume requested but the model holds no matching MD state";
    return DP_ERR_ARG;
  }
  if (!resume) {
    m->md_valid = false;
    DP_TRY(setup_replicas(m, nrep, st->atom_offsets, st->boxes, N, true));
    m->natoms = N;
    // masses per type into the device small table (as doubles after the int area)
    double* mass_t_dev = reinterpret_cast<double*>(m->small_i + 32);
    DP_CUDA_TRY(m, cudaMemcpyAsync(mass_t_dev, st->mass_by_type, sizeof(double) * m->ntypes,
                                   cudaMemcpyHostToDevice, m->stream));
    DP_TRY(launch_type_sort(m, st->types, N));
    DP_TRY(launch_load_positions(m, st->x, N));
    DP_TRY(launch_load_state(m, N, st->v, mass_t_dev));
    DP_TRY(launch_rebuild(m, N, true));
    DP_TRY(force_eval(m, N));
  }
  Model::GraphCache& gc = m->graphs;
  if (tune) {
    bool changed = false;
    DP_TRY(ensure_tuned(m, N, &changed));
    if (changed) drop_graphs(m);  // captured graphs hold the old launch shapes
  }
  if (capture) {
    unsigned long long h = hash_geom(m);
    if (gc.N != N || gc.nrep != nrep || gc.dt != dt || gc.geom_hash != h) {
      drop_graphs(m);
      DP_TRY(capture_step(m, N, dt, false, &gc.exec[0], &gc.kernels[0]));
      DP_TRY(capture_step(m, N, dt, true, &gc.exec[1], &gc.kernels[1]));
      gc.N = N; gc.nrep = nrep; gc.dt = dt; gc.geom_hash = h;
    }
  }
  for (int s = 0; s < nsteps; ++s) {
    long long step = st->step + s + 1;
    bool rebuild = (step % st->rebuild_every) == 0;
    if (capture) {
      DP_CUDA_TRY(m, cudaGraphLaunch(gc.exec[rebuild ? 1 : 0], m->stream));
      m->launches += gc.kernels[rebuild ? 1 : 0];
    } else {
      DP_TRY(md_step(m, N, dt, rebuild));
    }
  }
  st->step += nsteps;
  m->md_valid = true;
  DP_TRY(launch_outputs(m, N, st->potential, nullptr, st->forces, st->virial));
  if (st->kinetic) DP_TRY(launch_kinetic(m, N, st->kinetic));
  DP_TRY(launch_store_state(m, N, st->x, st->v));
  return DP_OK;
}

}  // namespace
}  // namespace dpg

using namespace dpg;

struct dp_model {
  Model m;
};

extern "C" {

const char* dp_version(void) { return "dpgb300 0.1"; }

// Device copies of the parameters from m->theta_host (and davg / dstd): theta in FP64 and
// FP32, transposed fitting weights, normalisation statistics, and for the mixed precisions
// the 16-bit tensor-core operand copies.  Synchronous.
dp_status upload_weights(Model* m) {
  const int nt = m->ntypes;
  const std::vector<double>& theta = m->theta_host;
  const size_t tsz = (size_t)kF * kKD + 2 * (size_t)kF * kF;
  std::vector<float> t32(theta.begin(), theta.end());
  std::vector<double> wT(tsz * nt);
  const size_t emb_total = (size_t)nt * nt * kEmbParams;
  for (int t = 0; t < nt; ++t) {
    const double* Pf = theta.data() + emb_total + (size_t)t * kFitParams;
    double* dst = wT.data() + t * tsz;
    for (int k = 0; k < kKD; ++k)
      for (int o = 0; o < kF; ++o) dst[(size_t)o * kKD + k] = Pf[kFW1 + (size_t)k * kF + o];
    double* d2 = dst + (size_t)kF * kKD;
    double* d3 = d2 + (size_t)kF * kF;
    for (int k = 0; k < kF; ++k)
      for (int o = 0; o < kF; ++o) {
        d2[(size_t)o * kF + k] = Pf[kFW2 + (size_t)k * kF + o];
        d3[(size_t)o * kF + k] = Pf[kFW3 + (size_t)k * kF + o];
      }
  }
  std::vector<float> wT32(wT.begin(), wT.end());
  std::vector<double> stat(8 * nt);
  for (int q = 0; q < 4 * nt; ++q) { stat[q] = m->davg_host[q]; stat[4 * nt + q] = 1.0 / m->dstd_host[q]; }
  std::vector<float> stat32(stat.begin(), stat.end());
  DP_CUDA_TRY(m, cudaMemcpy(m->w64, theta.data(), 8 * theta.size(), cudaMemcpyHostToDevice));
  DP_CUDA_TRY(m, cudaMemcpy(m->w32, t32.data(), 4 * t32.size(), cudaMemcpyHostToDevice));
  DP_CUDA_TRY(m, cudaMemcpy(m->fitT64, wT.data(), 8 * wT.size(), cudaMemcpyHostToDevice));
  DP_CUDA_TRY(m, cudaMemcpy(m->fitT32, wT32.data(), 4 * wT32.size(), cudaMemcpyHostToDevice));
  DP_CUDA_TRY(m, cudaMemcpy(m->stat64, stat.data(), 8 * stat.size(), cudaMemcpyHostToDevice));
  DP_CUDA_TRY(m, cudaMemcpy(m->stat32, stat32.data(), 4 * stat32.size(), cudaMemcpyHostToDevice));
  DP_TRY(launch_pad_rows(m));
  if (m->prec == DP_MIX_BF16 || m->prec == DP_MIX_FP16) {
    DP_TRY(launch_tc_setup(m));
    DP_TRY(launch_emb_images(m));
  }
  return DP_OK;
}

dp_status dp_create(dp_model** out, int ntypes, const char* const* type_map, double rcut, double rcut_smth,
                    const int* sel, const char* weight_path, const void* weight_blob, size_t blob_bytes,
                    dp_precision prec, int max_atoms, int max_replicas, double skin, void* cuda_stream) {
  if (!out) return DP_ERR_ARG;
  *out = nullptr;
  if (ntypes < 1 || ntypes > kMaxTypes || !sel || max_atoms < 1 || max_replicas < 1 || !(skin >= 0))
    return DP_ERR_ARG;
  if (prec < DP_FP64 || prec > DP_MIX_FP16) return DP_ERR_ARG;
  std::vector<unsigned char> file;
  const unsigned char* blob = static_cast<const unsigned char*>(weight_blob);
  if (weight_path) {
    FILE* f = std::fopen(weight_path, "rb");
    if (!f) return DP_ERR_WEIGHTS;
    std::fseek(f, 0, SEEK_END);
    long len = std::ftell(f);
    std::fseek(f, 0, SEEK_SET);
    file.resize(len > 0 ? (size_t)len : 0);
    size_t got = len > 0 ? std::fread(file.data(), 1, (size_t)len, f) : 0;
    std::fclose(f);
    if (got != file.size()) return DP_ERR_WEIGHTS;
    blob = file.data();
    blob_bytes = file.size();
  }
  if (!blob) return DP_ERR_ARG;
  dp_model* h = new dp_model();
  Model* m = &h->m;
  Parsed P;
  std::string why;
  dp_status st = parse_blob(blob, blob_bytes, P, why);
  auto fail = [&](dp_status s, const std::string& msg) {
    m->last_error = msg;
    dp_destroy(h);
    return s;
  };
  if (st != DP_OK) return fail(st, why);
  if (P.ntypes != ntypes) return fail(DP_ERR_WEIGHTS, "ntypes differs from the weights");
  if (std::fabs(P.rc - rcut) > 1e-12 * rcut || std::fabs(P.rs - rcut_smth) > 1e-12 * (rcut_smth + 1))
    return fail(DP_ERR_WEIGHTS, "rcut / rcut_smth differ from the weights");
  if (!(P.rs >= 0 && P.rs < P.rc)) return fail(DP_ERR_WEIGHTS, "need 0 <= rcut_smth < rcut");
  for (int t = 0; t < ntypes; ++t) {
    if (P.sel[t] != sel[t] || sel[t] < 1) return fail(DP_ERR_WEIGHTS, "sel differs from the weights");
    if (type_map && type_map[t] && P.names[t] != type_map[t])
      return fail(DP_ERR_WEIGHTS, "type_map differs from the weights");
  }
  m->ntypes = ntypes; m->switch_kind = P.switch_kind; m->rc = P.rc; m->rs = P.rs; m->skin = skin; m->prec = prec;
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(DP_ERR_CUDA, "cannot create the capture stream");
  m->max_atoms = max_atoms; m->max_reps = max_replicas;
  m->max_cells = max_atoms + 64 * max_replicas + 1024;
  m->sel_off[0] = 0; m->vcap_off[0] = 0;
  const double vol = std::pow((P.rc + skin) / P.rc, 3.0);
  for (int t = 0; t < ntypes; ++t) {
    m->sel[t] = sel[t];
    m->sel_off[t + 1] = m->sel_off[t] + sel[t];
    int cap = (int)std::ceil(1.3 * sel[t] * vol);
    m->vcap[t] = (cap + 31) / 32 * 32;
    m->vcap_off[t + 1] = m->vcap_off[t] + m->vcap[t];
  }
  m->S = m->sel_off[ntypes];
  m->VS = m->vcap_off[ntypes];
  m->ntheta = (long long)P.theta.size();
  m->theta_host = P.theta;
  m->davg_host = P.davg; m->dstd_host = P.dstd;
  if ((prec == DP_MIX_BF16 || prec == DP_MIX_FP16) && !tc_available(m))
    return fail(DP_ERR_UNSUPPORTED, "mixed precision needs the tensor-core kernels (sm_103a GPU)");

  const size_t N = (size_t)max_atoms, R = (size_t)max_replicas;
  const size_t es = (prec == DP_FP64) ? 8 : 4;
  const int nt = ntypes;
#define A_(p, bytes) do { dp_status s_ = dalloc(m, &m->p, (bytes)); if (s_ != DP_OK) return fail(s_, m->last_error); } while (0)
  A_(w64, 8 * P.theta.size());
  A_(w32, 4 * P.theta.size());
  const size_t tsz = (size_t)kF * kKD + 2 * (size_t)kF * kF;
  A_(fitT64, 8 * tsz * nt);
  A_(fitT32, 4 * tsz * nt);
  A_(stat64, 8 * 8 * nt);
  A_(stat32, 4 * 8 * nt);
  A_(pad64, 8 * (size_t)nt * nt * 4 * kN3);
  A_(rdf_hist, sizeof(unsigned long long) * kRdfMaxCells);
  A_(pad32, 4 * (size_t)nt * nt * 4 * kN3);
  A_(perm, 4 * N); A_(inv, 4 * N); A_(itype, 4 * N); A_(irep, 4 * N);
  A_(type_count, 4 * (kMaxTypes + 1)); A_(type_off, 4 * (kMaxTypes + 1));
  A_(blk_count, 4 * (size_t)kMaxTypes * (N / 1024 + 2));
  A_(x, 32 * N); A_(xref, 32 * N); A_(v, 32 * N); A_(delta, 16 * N); A_(xf, 16 * N); A_(xq, 32 * N);
  A_(force, 24 * N); A_(mass, 8 * N);
  A_(geom, sizeof(RepGeom) * R);
  A_(cell_of, 4 * N);
  A_(cell_count, 4 * (size_t)m->max_cells); A_(cell_start, 4 * ((size_t)m->max_cells + 1));
  A_(cell_fill, 4 * (size_t)m->max_cells); A_(cell_atoms, 4 * N); A_(cell_xf, 16 * N);
  A_(vl_e, 16 * N * m->VS); A_(vl_img, 4 * N * m->VS); A_(vl_work, 4 * (N + 1)); A_(vcount, 4 * N * nt);
  A_(nl_j, 4 * N * m->S); A_(nl_img, 4 * N * m->S);
  A_(nl_d, (prec == DP_FP64 ? 32 : 16) * N * m->S);
  A_(nl_count, 4 * N * nt);
  A_(Tm, es * N * 4 * kN3); A_(Dm, es * N * kKD); A_(dD, es * N * kKD);
  for (int q = 0; q < 5; ++q) A_(act[q], es * N * kF);
  A_(e_atom, 8 * N); A_(vir_atom, 72 * N); A_(e_user, 8 * N); A_(vir_user, 72 * N); A_(ke_user, 8 * N);
  A_(red_out, 8 * 20 * R + 64);
  A_(rep_off_dev, 4 * (R + 1));
  A_(err, 16);
  A_(small_i, 4 * 64 + 8 * kMaxTypes);
  if (prec == DP_MIX_BF16 || prec == DP_MIX_FP16) {
    A_(rowoff, 4 * (size_t)nt * (N + 1));
    A_(scan_blk, 4 * (size_t)nt * (N / 1024 + 2));
    A_(Tseg, 4 * (size_t)nt * N * 400);
    A_(dTm, 16 * N * kN3);
    A_(force32, 16 * N);
    A_(vir_rep, 72 * R + 64);
    A_(tc_weights, mix_fit_weight_bytes(nt));
    A_(emb_img, mix_emb_image_bytes(nt));
  }
  m->pg_cap = std::min(max_atoms, kPgAtoms);
  m->pg_roff_cap = 2 * (size_t)nt * N + 64;
  A_(pg_ws, param_grad_workspace_bytes(m->pg_cap, prec == DP_FP64));
  A_(pg_roff, 4 * m->pg_roff_cap);
  A_(pg_w, 24 * N);
  A_(pg_scal, 64);
  m->red_cap = rep_reduce_slots(max_atoms, max_replicas);
  A_(red_part, 80 * m->red_cap);
#undef A_
  for (int b = 0; b < 2; ++b) {
    if (halloc(m, &m->geom_stage[b], sizeof(RepGeom) * R + sizeof(int) * (R + 1) + 64) != DP_OK)
      return fail(DP_ERR_OOM, m->last_error);
    if (cudaEventCreateWithFlags(&m->geom_ev[b], cudaEventDisableTiming) != cudaSuccess)
      return fail(DP_ERR_CUDA, "cannot create an event");
  }
  m->geom_host = m->geom_stage[0];
  if (halloc(m, &m->err_host, 64) != DP_OK) return fail(DP_ERR_OOM, m->last_error);

  {
    dp_status s1 = upload_weights(m);
    if (s1 != DP_OK) return fail(s1, m->last_error);
  }
  if (cudaMemset(m->err, 0, 16) != cudaSuccess) return fail(DP_ERR_CUDA, "memset failed");
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(DP_ERR_CUDA, "device sync after create failed");
  *out = h;
  return DP_OK;
}

dp_status dp_compute_batch(dp_model* h, int nrep, const int* atom_offsets, const double* coords, const int* types,
                           const double* boxes, double* energies, double* atom_energy, double* forces,
                           double* virials) {
  if (!h) return DP_ERR_ARG;
  Model* m = &h->m;
  if (!atom_offsets || !coords || !types || !boxes || !energies || !forces) {
    m->last_error = "null argument";
    return DP_ERR_ARG;
  }
  if (nrep < 1) { m->last_error = "nrep < 1"; return DP_ERR_ARG; }
  const int N = atom_offsets[nrep];
  if (N < 1 || N > m->max_atoms) { m->last_error = "natoms out of range"; return DP_ERR_CAPACITY; }
  m->md_valid = false;
  DP_TRY(setup_replicas(m, nrep, atom_offsets, boxes, N, false));
  m->natoms = N;
  DP_TRY(launch_type_sort(m, types, N));
  DP_TRY(launch_load_positions(m, coords, N));
  DP_TRY(launch_rebuild(m, N, false));
  DP_TRY(force_eval(m, N));
  DP_TRY(launch_outputs(m, N, energies, atom_energy, forces, virials));
  return DP_OK;
}

dp_status dp_compute(dp_model* h, int natoms, const double* coords, const int* types, const double* box,
                     double* energy, double* atom_energy, double* forces, double* virial) {
  if (!h) return DP_ERR_ARG;
  if (!box) { h->m.last_error = "null box"; return DP_ERR_ARG; }
  if (natoms < 1) { h->m.last_error = "natoms < 1"; return DP_ERR_ARG; }
  int offs[2] = {0, natoms};
  return dp_compute_batch(h, 1, offs, coords, types, box, energy, atom_energy, forces, virial);
}

dp_status dp_verlet_step(dp_model* h, dp_md_state* st, double dt_fs, int nsteps, int capture_graph) {
  if (!h) return DP_ERR_ARG;
  return run_md(&h->m, st, dt_fs, nsteps, capture_graph, capture_graph != 0);
}

dp_status dp_md_run_batch(dp_model* h, dp_md_state* st, double dt_fs, int nsteps) {
  if (!h) return DP_ERR_ARG;
  return run_md(&h->m, st, dt_fs, nsteps, 1, true);
}

dp_status dp_autotune(dp_model* h, int repeats, int* grids) {
  if (!h || repeats < 0) return DP_ERR_ARG;
  Model* m = &h->m;
  if (repeats == 0) {  // query only
    if (grids)
      for (int k = 0; k < 4; ++k) grids[k] = m->tune_grid[k];
    return DP_OK;
  }
  if (m->natoms < 1) { m->last_error = "no state to tune on"; return DP_ERR_ARG; }
  drop_graphs(m);
  DP_TRY(autotune(m, m->natoms, repeats));
  m->tuned_key = tune_key(m, m->natoms);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[m->tuned_key] = {m->tune_grid[0], m->tune_grid[1], m->tune_grid[2], m->tune_grid[3]};
  }
  if (grids)
    for (int k = 0; k < 4; ++k) grids[k] = m->tune_grid[k];
  DP_CUDA_TRY(m, cudaStreamSynchronize(m->stream));
  return DP_OK;
}

dp_status dp_set_params(dp_model* h, const double* theta, long long ntheta) {
  if (!h) return DP_ERR_ARG;
  Model* m = &h->m;
  if (!theta) { m->last_error = "null theta"; return DP_ERR_ARG; }
  if (ntheta != m->ntheta) { m->last_error = "ntheta does not match the model"; return DP_ERR_ARG; }
  for (long long q = 0; q < ntheta; ++q)
    if (!std::isfinite(theta[q])) { m->last_error = "non-finite parameter"; return DP_ERR_WEIGHTS; }
  DP_CUDA_TRY(m, cudaStreamSynchronize(m->stream));
  m->theta_host.assign(theta, theta + ntheta);
  DP_TRY(upload_weights(m));
  DP_CUDA_TRY(m, cudaDeviceSynchronize());
  if (m->tab_n > 0) DP_TRY(launch_tabulate(m, m->tab_x0, m->tab_x0 + m->tab_n * m->tab_h, m->tab_n));
  return DP_OK;
}

dp_status dp_rdf(dp_model* h, int nbins, double r_max, unsigned long long* counts) {
  if (!h || !counts) return DP_ERR_ARG;
  Model* m = &h->m;
  if (m->natoms < 1) { m->last_error = "no state to analyse"; return DP_ERR_ARG; }
  if (nbins < 1 || nbins * m->ntypes * m->ntypes > kRdfMaxCells || !(r_max > 0) || r_max > m->rc) {
    m->last_error = "need 1 <= nbins, ntypes^2 * nbins <= 24576 and 0 < r_max <= rcut";
    return DP_ERR_ARG;
  }
  DP_TRY(launch_rdf(m, nbins, r_max, m->rdf_hist));
  DP_CUDA_TRY(m, cudaMemcpyAsync(counts, m->rdf_hist, sizeof(unsigned long long) * (size_t)m->ntypes * m->ntypes * nbins,
                                 cudaMemcpyDeviceToHost, m->stream));
  DP_CUDA_TRY(m, cudaStreamSynchronize(m->stream));
  return DP_OK;
}

dp_status dp_atom_virial(dp_model* h, double* atom_virial) {
  if (!h || !atom_virial) return DP_ERR_ARG;
  Model* m = &h->m;
  if (m->natoms < 1) { m->last_error = "no state to evaluate"; return DP_ERR_ARG; }
  const int N = m->natoms;
  if (is_mixed(m)) {
    DP_CUDA_TRY(m, cudaMemsetAsync(m->vir_atom, 0, sizeof(double) * 9 * (size_t)N, m->stream));
    DP_TRY(launch_mix_atom_virial(m, N));
  }
  return launch_atom_virial_out(m, N, atom_virial);
}

dp_status dp_tabulate(dp_model* h, double x_min, double x_max, int n_intervals) {
  if (!h) return DP_ERR_ARG;
  Model* m = &h->m;
  if (n_intervals < 0 || n_intervals > (1 << 20) ||
      (n_intervals > 0 && (!(x_max > x_min) || !std::isfinite(x_min) || !std::isfinite(x_max)))) {
    m->last_error = "need 0 <= n_intervals <= 2^20 and finite x_min < x_max";
    return DP_ERR_ARG;
  }
  drop_graphs(m);
  m->tuned_key = 0;
  return launch_tabulate(m, x_min, x_max, n_intervals);
}

dp_status dp_set_truncation(dp_model* h, int nearest) {
  if (!h) return DP_ERR_ARG;
  Model* m = &h->m;
  if (nearest != 0 && nearest != 1) {
    m->last_error = "nearest must be 0 or 1";
    return DP_ERR_ARG;
  }
  drop_graphs(m);
  m->nearest = nearest != 0;
  return DP_OK;
}

long long dp_ntheta(const dp_model* h) { return h ? h->m.ntheta : 0; }

dp_status dp_get_nlist(dp_model* h, int* nlist, int* images) {
  if (!h || !nlist || !images) return DP_ERR_ARG;
  Model* m = &h->m;
  if (m->natoms < 1) { m->last_error = "no neighbour list yet"; return DP_ERR_ARG; }
  // the per-step format leaves the image codes out; this pass repeats it with them
  DP_TRY(launch_format(m, m->natoms, true));
  DP_TRY(launch_get_nlist(m, m->natoms, nlist, images));
  DP_CUDA_TRY(m, cudaStreamSynchronize(m->stream));
  return DP_OK;
}

dp_status dp_sync(dp_model* h) {
  if (!h) return DP_ERR_ARG;
  Model* m = &h->m;
  DP_CUDA_TRY(m, cudaStreamSynchronize(m->stream));
  DP_CUDA_TRY(m, cudaMemcpy(m->err_host, m->err, sizeof(int), cudaMemcpyDeviceToHost));
  int bits = *m->err_host;
  if (bits) DP_CUDA_TRY(m, cudaMemset(m->err, 0, sizeof(int)));
  return map_err_bits(m, bits);
}

const char* dp_last_error(const dp_model* h) { return h ? h->m.last_error.c_str() : "null model"; }

long long dp_kernel_launches(const dp_model* h) { return h ? h->m.launches : 0; }

dp_status dp_phase_times(dp_model* h, int repeats, float* ms) {
  if (!h || !ms || repeats < 1) return DP_ERR_ARG;
  Model* m = &h->m;
  if (m->natoms < 1) { m->last_error = "no state to evaluate"; return DP_ERR_ARG; }
  const int N = m->natoms;
  cudaEvent_t ev[5];
  for (auto& e : ev) DP_CUDA_TRY(m, cudaEventCreate(&e));
  const bool split = is_mixed(m);  // the mixed launchers record the kernel-level split
  if (split)
    for (auto& e : m->sub_ev) DP_CUDA_TRY(m, cudaEventCreate(&e));
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  dp_status st = DP_OK;
  for (int r = 0; r < repeats && st == DP_OK; ++r) {
    cudaEventRecord(ev[0], m->stream);
    st = launch_format(m, N);
    cudaEventRecord(ev[1], m->stream);
    if (st == DP_OK) st = launch_zero_forces(m, N);
    if (st == DP_OK) st = launch_descriptor(m, N);
    cudaEventRecord(ev[2], m->stream);
    if (st == DP_OK) st = launch_fitting(m, N);
    cudaEventRecord(ev[3], m->stream);
    if (st == DP_OK) st = launch_embed_backward(m, N);
    cudaEventRecord(ev[4], m->stream);
    if (cudaEventSynchronize(ev[4]) != cudaSuccess) { m->last_error = "phase timing failed"; st = DP_ERR_CUDA; }
    for (int q = 0; q < 4 && st == DP_OK; ++q) {
      float t = 0;
      cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
      acc[q] += t;
    }
    float tot = 0;
    cudaEventElapsedTime(&tot, ev[0], ev[4]);
    acc[4] += tot;
    if (split && st == DP_OK) {
      float f = 0, b = 0;
      cudaEventElapsedTime(&f, ev[1], m->sub_ev[0]);
      cudaEventElapsedTime(&b, m->sub_ev[1], ev[4]);
      acc[5] += f;
      acc[6] += b;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (split)
    for (auto& e : m->sub_ev) { cudaEventDestroy(e); e = nullptr; }
  if (!split) { acc[5] = acc[1]; acc[6] = acc[3]; }
  for (int q = 0; q < 8; ++q) ms[q] = q < 7 ? (float)(acc[q] / repeats) : 0.f;
  return st;
}

void dp_destroy(dp_model* h) {
  if (!h) return;
  Model* m = &h->m;
  cudaStreamSynchronize(m->stream);
  drop_graphs(m);
  if (m->capture_stream) cudaStreamDestroy(m->capture_stream);
  for (auto& e : m->geom_ev)
    if (e) cudaEventDestroy(e);
  for (void* p : m->dev_allocs) cudaFree(p);
  for (void* p : m->host_allocs) cudaFreeHost(p);
  m->dev_allocs.clear();
  m->host_allocs.clear();
  mix_fit_release(m);
  if (m->tab_mem) cudaFree(m->tab_mem);
  m->tab_mem = nullptr;
  delete h;
}

}  // extern "C"

extern "C" dp_status dp_param_grad(dp_model* h, int natoms, const double* coords, const int* types,
                                   const double* box, double E0, const double* F0, double cE, double cF,
                                   double* grad, double* loss) {
  if (!h) return DP_ERR_ARG;
  Model* m = &h->m;
  if (!coords || !types || !box || !F0 || !grad) { m->last_error = "null argument"; return DP_ERR_ARG; }
  if (natoms < 1) { m->last_error = "natoms < 1"; return DP_ERR_ARG; }
  if (natoms > m->max_atoms) { m->last_error = "natoms out of range"; return DP_ERR_CAPACITY; }
  if (m->tab_n > 0) {
    m->last_error = "the parameter gradient needs the embedding networks, not their tables";
    return DP_ERR_UNSUPPORTED;
  }
  const int offs[2] = {0, natoms};
  m->md_valid = false;
  DP_TRY(setup_replicas(m, 1, offs, box, natoms, false));
  m->natoms = natoms;
  DP_TRY(launch_type_sort(m, types, natoms));
  DP_TRY(launch_load_positions(m, coords, natoms));
  DP_TRY(launch_rebuild(m, natoms, false));
  DP_TRY(force_eval(m, natoms));
  return launch_param_grad(m, natoms, F0, E0, cE, cF, grad, loss);
}
