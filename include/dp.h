/*
 * dp.h -- C ABI of the GB300 Deep Potential library (libdpgb300.so).
 *
 * The library evaluates the per-atom energy, forces and virial of a
 * smooth-edition two-body Deep Potential model and advances velocity-Verlet
 * molecular dynamics with it, on one GPU.  This is the force-field evaluation
 * of the paper's Section II-A and Fig. 1: the neighbour list within r_c, the
 * environment matrix R with its smoothed first column, the three-layer
 * embedding net, the descriptor, the three-layer fitting net giving E_i, and
 * the forces F_i obtained by backward propagation (Fig. 1(b)); the MD step
 * updates velocities and positions and reports pressure-related virials
 * (Section II-A).  Sizes follow Section IV: r_c 6 A (water) / 8 A (Cu),
 * neighbour caps 46/92 (water) and 512 (Cu), fitting net (240, 240, 240),
 * skin 2 A.  Mixed precision follows Section III-B3 (FP32 descriptor and
 * activations, 16-bit GEMM operands).
 *
 * Conventions for every entry point
 *  - All array arguments are caller-owned.  "device" arrays must be device
 *    memory of the model's GPU, valid until the model's stream reaches the
 *    call.  "host" arrays are read before the call returns.
 *  - Calls are asynchronous on the stream given to dp_create (NULL = the
 *    legacy default stream).  Argument errors are returned synchronously.
 *    Errors detected on the device (neighbour overflow, skin exceeded) are
 *    sticky: dp_sync() waits for the stream and returns them, and clears them.
 *  - Units: Angstrom, eV, fs, amu.  Forces are eV/A; the virial is in eV and
 *    is the negative strain derivative of the energy, Xi = -sum_pairs g (x) d
 *    with g = dE/dd for the pair vector d = x_j + n H - x_i.
 *  - Boxes are 3x3 row-major, the rows the cell vectors a, b, c; an image
 *    n = (n0, n1, n2) of atom j sits at x_j + n H.  Any right-handed cell of
 *    positive volume with entries below 2^28 A (else DP_ERR_ARG); orthorhombic
 *    cells (off-diagonal entries 0) wrap and bin per axis, triclinic ones by
 *    fractional coordinate s = x H^-1.
 *  - Atom arrays are in the caller's order; the library sorts atoms by type
 *    internally and un-permutes every output.
 *  - No call allocates device memory after dp_create (except dp_tabulate, a set-up
 *    call that allocates its tables): all buffers are sized there from max_atoms
 *    and max_replicas (preallocated memory, Section III-B1 "allocated in the
 *    initial phase").  Larger inputs return DP_ERR_CAPACITY.
 */
#ifndef DP_GB300_H
#define DP_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dp_model dp_model;

typedef enum {
  DP_OK = 0,
  DP_ERR_ARG = 1,           /* bad argument (null pointer, size, mismatch) */
  DP_ERR_CUDA = 2,          /* a CUDA runtime call failed; see dp_last_error */
  DP_ERR_OOM = 3,           /* device allocation failed in dp_create */
  DP_ERR_UNSUPPORTED = 4,   /* cell too small for the cutoff, unsupported network size or precision */
  DP_ERR_SEL_OVERFLOW = 5,  /* more real neighbours of one type than sel[type] */
  DP_ERR_SKIN_EXCEEDED = 6, /* an atom moved more than skin/2 since the last neighbour rebuild */
  DP_ERR_WAIT_TIMEOUT = 7,  /* a bounded device-side wait gave up */
  DP_ERR_CAPACITY = 8,      /* more atoms/replicas/cells/Verlet entries than allocated */
  DP_ERR_WEIGHTS = 9        /* weight blob malformed or inconsistent with the arguments */
} dp_status;

typedef enum {
  DP_FP64 = 0,     /* everything in FP64 */
  DP_FP32 = 1,     /* R, networks and per-pair force terms in FP32; positions,
                      Verlet update, force accumulation, energy and virial sums in FP64 */
  DP_MIX_BF16 = 2, /* as DP_FP32, with the embedding and fitting GEMM operands in BF16
                      on the tensor cores, FP32 accumulation; forces accumulated in FP32
                      (then added to the FP64 force array) */
  DP_MIX_FP16 = 3  /* as DP_MIX_BF16 with FP16 operands */
} dp_precision;

/*
 * dp_create -- build a model on the current CUDA device.
 *   out          receives the handle.
 *   ntypes       number of atom types; type_map[ntypes] their names (e.g. {"O","H"}),
 *                checked against the names stored in the weights (nullable: no check).
 *   rcut, rcut_smth  cutoff and start of the smooth switch (A); must equal the weights'.
 *   sel[ntypes]  per-neighbour-type caps; must equal the weights'.
 *   weight_path  file holding a weight blob, or NULL to use weight_blob/blob_bytes.
 *   weight_blob  host pointer to the blob (layout: magic "DPW1", header of sizes,
 *                sel, type names, then FP64 parameters in the documented order).
 *   prec         arithmetic policy (dp_precision).
 *   max_atoms    capacity in atoms summed over replicas; max_replicas capacity in boxes.
 *   skin         Verlet-list skin (A); the list of an MD run holds pairs within rcut + skin.
 *   cuda_stream  cudaStream_t to run on (NULL = default stream).
 * Weights are copied to device memory owned by the model.
 */
dp_status dp_create(dp_model** out, int ntypes, const char* const* type_map, double rcut,
                    double rcut_smth, const int* sel, const char* weight_path,
                    const void* weight_blob, size_t blob_bytes, dp_precision prec, int max_atoms,
                    int max_replicas, double skin, void* cuda_stream);

/*
 * dp_compute -- energy, per-atom energy, forces and virial of one periodic box.
 *   coords [natoms*3] device FP64, types [natoms] device int32 in [0, ntypes),
 *   box [9] host.  Outputs (device FP64): energy [1], atom_energy [natoms]
 *   (nullable), forces [natoms*3], virial [9] (nullable).
 * Positions are wrapped into the box and the neighbour list is rebuilt on every
 * call, within rcut only (no skin: nothing reuses it).  The call invalidates the
 * MD state held by the model (a later dp_verlet_step with resume set is refused).
 * On a device-side error the outputs are undefined and energy is NaN; dp_sync
 * returns the error.
 */
dp_status dp_compute(dp_model* m, int natoms, const double* coords, const int* types,
                     const double* box, double* energy, double* atom_energy, double* forces,
                     double* virial);

/*
 * dp_compute_batch -- dp_compute over nrep independent boxes in one pass.
 *   atom_offsets [nrep+1] host, CSR offsets of each replica's atoms in coords/types;
 *   boxes [nrep*9] host.  energies [nrep] and virials [nrep*9] device outputs
 *   (virials nullable); atom_energy [N] (nullable) and forces [N*3] device outputs.
 */
dp_status dp_compute_batch(dp_model* m, int nrep, const int* atom_offsets, const double* coords,
                           const int* types, const double* boxes, double* energies,
                           double* atom_energy, double* forces, double* virials);

/* Molecular-dynamics state, all in the caller's atom order. */
typedef struct {
  int natoms;                 /* total atoms over replicas */
  int nrep;                   /* number of independent boxes (>= 1) */
  const int* atom_offsets;    /* host [nrep+1]; NULL means one replica */
  const double* boxes;        /* host [nrep*9] */
  double* x;                  /* device [natoms*3] positions, updated in place */
  double* v;                  /* device [natoms*3] velocities (A/fs), updated in place */
  const int* types;           /* device [natoms] */
  const double* mass_by_type; /* host [ntypes], amu */
  double* forces;             /* device [natoms*3] out: forces after the last step (nullable) */
  double* potential;          /* device [nrep] out: potential energy after the last step (nullable) */
  double* kinetic;            /* device [nrep] out: kinetic energy after the last step (nullable) */
  double* virial;             /* device [nrep*9] out: virial after the last step (nullable) */
  long long step;             /* in/out: step counter; rebuilds happen when step % rebuild_every == 0 */
  int rebuild_every;          /* neighbour rebuild interval in steps (>= 1) */
  int resume;                 /* 0: read x, v, rebuild lists and evaluate F(x) first;
                                 1: continue from the model's internal state left by the previous
                                 MD call on this model (x, v are not re-read; same atoms and boxes) */
} dp_md_state;

/*
 * dp_verlet_step -- advance nsteps velocity-Verlet NVE steps of time step dt_fs:
 *   v += dt/2 * kappa F/m; x += dt v; rebuild the neighbour list every
 *   rebuild_every steps (positions wrapped then), otherwise check that no atom
 *   moved more than skin/2; F = F(x); v += dt/2 * kappa F/m;
 *   kappa = 9.648533e-3 A fs^-2 per eV A^-1 amu^-1.
 * Positions and velocities stay FP64 in every precision.  With capture_graph
 * != 0 the steps between rebuilds are captured once into a CUDA graph and
 * replayed; before the first capture for a configuration the launch grids of the
 * mixed-precision kernels are chosen by the autotuner (dp_autotune).  The state's x and v are read at the start and written at the end
 * of the call.  Works for one replica or many (nrep > 1).
 */
dp_status dp_verlet_step(dp_model* m, dp_md_state* st, double dt_fs, int nsteps, int capture_graph);

/*
 * dp_md_run_batch -- dp_verlet_step for many replicas of uneven size (st->nrep
 * boxes, atoms concatenated by st->atom_offsets).  Every phase is one launch over
 * the atoms and neighbour rows of all replicas (the kernels walk the concatenated
 * arrays), and the steps between neighbour rebuilds always run as a captured CUDA
 * graph.  On the first call for a configuration (precision, atoms, replicas) the
 * launch grids are chosen by the autotuner (dp_autotune; choices cached per process)
 * before the graph is captured.  Energies, kinetic energies and virials are reported
 * per replica.
 */
dp_status dp_md_run_batch(dp_model* m, dp_md_state* st, double dt_fs, int nsteps);

/*
 * dp_autotune -- time the candidate launch grids of the mixed-precision kernels whose
 * shape is a choice (embedding forward and backward: 1, 2, 3 or 6 CTAs per SM; the
 * dE/dT and descriptor kernels) over `repeats` full force evaluations each, on the
 * model's current state (after dp_compute or an MD call), and keep the fastest.
 * grids[4] (host, nullable) receives the chosen grids (embedding forward, embedding
 * backward, dE/dT, descriptor; 0 = not tuned, as for FP64 / FP32 models).  Drops the
 * model's captured MD graphs; leaves the forces of the chosen configuration; synchronous.
 * repeats = 0 only reports the current choices.
 */
dp_status dp_autotune(dp_model* m, int repeats, int* grids);

/*
 * dp_param_grad -- gradient of the loss
 *   L = cE * (E - E0)^2 + cF * sum_k |F_k - F0_k|^2
 * with respect to every model parameter theta (the FP64 parameter block of the
 * weight blob: embedding nets, fitting nets, e_bias; davg/dstd are not
 * parameters).  One box as in dp_compute; E0 host scalar; F0 [natoms*3] device
 * (caller order).  grad [ntheta] device FP64 output (overwritten); loss [1]
 * device output (nullable).  The force term is the derivative of the
 * directional derivative of E along w = 2 cF (F - F0), computed by a
 * tangent-forward sweep followed by a reverse sweep; embedding activations are
 * recomputed, not stored.  Runs in FP64 or FP32 according to the model's
 * precision (mixed precisions use FP32 here).
 */
dp_status dp_param_grad(dp_model* m, int natoms, const double* coords, const int* types,
                        const double* box, double E0, const double* F0, double cE, double cF,
                        double* grad, double* loss);

/*
 * dp_tabulate -- replace every embedding net by its table (the compressed model of Section
 * II-A): each of the 100 outputs of each net (ti, tj) becomes a piecewise quintic in the net's
 * input s_hat on n_intervals uniform intervals of [x_min, x_max], matching the net's value,
 * first and second derivative at both ends of every interval (C2; the error falls as h^6 with
 * the interval width h).  Inputs outside [x_min, x_max] use the edge interval's polynomial, so
 * the range should cover the normalised input of a neighbour at r_c (-davg/dstd) up to that of
 * the closest approach expected.  Forward and force backward then evaluate the table instead
 * of the net, in every precision (mixed precisions keep the 16-bit fitting net and T product).
 * n_intervals = 0 goes back to the nets.  The tables are built on the device in FP64 from the
 * current parameters (rebuilt by dp_set_params) and kept in FP64 and FP32.  Unlike the other
 * calls this one allocates device memory (the tables: 36 n bytes per output and pair).  Drops
 * captured MD graphs; synchronous.  dp_param_grad returns DP_ERR_UNSUPPORTED while a table is
 * in use.  Errors: DP_ERR_ARG (n_intervals < 0 or > 2^20, x_min >= x_max), DP_ERR_OOM, DP_ERR_CUDA.
 */
dp_status dp_tabulate(dp_model* m, double x_min, double x_max, int n_intervals);

/*
 * dp_rdf -- pair-distance histogram of the last evaluation (dp_compute, dp_compute_batch or
 * an MD call), behind the radial distribution function of Section IV-A (Fig. 6): for every
 * centre atom i of type ti and neighbour (j, image n) of type tj at distance r < r_max,
 * counts[(ti * ntypes + tj) * nbins + floor(r / (r_max / nbins))] += 1.  Each unordered pair is
 * counted from both ends.  The pairs are those of the formatted neighbour list, so
 * r_max <= rcut.  g_ab(r) = counts_ab / (N_a rho_b 4 pi r^2 dr) with rho_b = N_b / V (N_b - 1
 * for a = b).  counts [ntypes * ntypes * nbins] host output.  Distances in the model's
 * precision of the pair vectors (FP64 for DP_FP64, else FP32).  Synchronous.
 * Errors: DP_ERR_ARG (no state, nbins < 1, ntypes^2 nbins > 24576, r_max outside (0, rcut]).
 */
dp_status dp_rdf(dp_model* m, int nbins, double r_max, unsigned long long* counts);

/*
 * dp_atom_virial -- per-atom virial of the last evaluation, caller order: atom_virial
 * [natoms * 9] device, row-major 3 x 3 per atom, W_i = -sum over the neighbours (j, n) of i of
 * g_ijn (x) d_ijn with g = dE/dd (each pair term assigned to its centre atom i; the W_i sum to
 * the virial of dp_compute).  FP64 / FP32 models compute it in every evaluation; the mixed
 * precisions compute it here with a second pass of the force backward on the stored state (the
 * forces are not touched).  Asynchronous on the model's stream.
 * Errors: DP_ERR_ARG (null, no state), DP_ERR_CUDA.
 */
dp_status dp_atom_virial(dp_model* m, double* atom_virial);

/*
 * dp_set_truncation -- neighbour overflow policy.  nearest = 0 (default): a centre with more than
 * sel[t] neighbours of type t within rcut makes the evaluation fail with DP_ERR_SEL_OVERFLOW.
 * nearest = 1: such a neighbour type keeps its sel[t] nearest neighbours, DeePMD's convention for
 * a full neighbour list (Section II-A's fixed-size environment matrix); ranks are by the FP64
 * squared distance, ties by the caller's index of j, then the image (n_x, n_y, n_z).  The energy
 * is then discontinuous where two neighbours swap ranks across the cut.  Drops captured MD
 * graphs.  Errors: DP_ERR_ARG (null model, nearest not 0 or 1).
 */
dp_status dp_set_truncation(dp_model* m, int nearest);

/* Number of parameters in theta (the length of dp_param_grad's grad). */
long long dp_ntheta(const dp_model* m);

/*
 * dp_set_params -- replace the model's network parameters (training step).  theta
 * [ntheta] host FP64 in the layout of the weight blob's parameter block (embedding
 * nets per (ti, tj), fitting nets per type, e_bias); ntheta must equal dp_ntheta(m).
 * All derived device copies (FP32, transposed fitting weights, 16-bit tensor-core
 * copies) are rebuilt.  Waits for the model's stream first; synchronous.  Captured
 * MD graphs stay valid (the device buffers do not move).
 * Errors: DP_ERR_ARG (null, wrong size), DP_ERR_WEIGHTS (non-finite value), DP_ERR_CUDA.
 */
dp_status dp_set_params(dp_model* m, const double* theta, long long ntheta);

/*
 * dp_get_nlist -- copy the formatted neighbour list of the last dp_compute /
 * MD step: nlist [natoms*S] and images [natoms*S] device int32 in caller order,
 * S = sum(sel).  Row i holds, per neighbour type t in order, the neighbours of
 * type t in canonical order (ascending caller index j, then image nx, ny, nz),
 * padded with -1 (nlist) and 0 (images) to sel[t].  Image code:
 * ((nx+512)<<20) | ((ny+512)<<10) | (nz+512).  Waits for the stream.
 */
dp_status dp_get_nlist(dp_model* m, int* nlist, int* images);

/*
 * dp_phase_times -- measurement hook: run `repeats` force evaluations on the
 * model's current internal state (left by the last dp_compute / MD call) with
 * CUDA events on the model's stream around each phase, and write the mean
 * milliseconds per phase to ms[8]: [0] list format, [1] descriptor (environment
 * matrix, embedding, T, D), [2] fitting forward+backward, [3] embedding backward
 * with force and virial scatter, [4] whole evaluation, [5] the embedding
 * forward kernel alone (mixed precision; else = [1]), [6] the embedding backward
 * kernel alone (mixed precision: without the dE/dT kernel; else = [3]), [7] 0.
 * Synchronous.  Leaves forces/energies of the last evaluation in place.
 */
dp_status dp_phase_times(dp_model* m, int repeats, float* ms);

/* Number of kernels this model has launched so far (graph replays count every
   kernel in the graph).  Host-side counter; no synchronisation. */
long long dp_kernel_launches(const dp_model* m);

/*
 * dp_selftest -- built-in check of the tensor-core operand layouts on the current
 * device: runs one tcgen05 MMA of a known small-integer problem (case `which`:
 * 0..4 = shapes N 64/112/240/32/160, bf16 or fp16 operands, both K-major;
 * 5..7 = K 64 with an MN-major B (N 64), an MN-major A (N 64), or both MN-major
 * (N 128)) and writes
 * result[0] = max |error| against the exact product, result[1] = max |value|.
 * Returns DP_ERR_UNSUPPORTED on a device without tcgen05.
 */
dp_status dp_selftest(int which, double* result);

/*
 * dp_selftest_noalloc -- the checks of dp_selftest for several cases in one call,
 * without allocating memory.  The paper has no counterpart: this is a device
 * health check of the library for callers that cannot allocate (a process whose
 * device memory already belongs to its own pool, or a monitor that must not
 * trigger the device-wide wait of cudaFree, which dp_selftest calls).
 *   which[ncases]      host: case numbers 0..4 (the K-major cases of dp_selftest).
 *   ncases             0..DP_SELFTEST_NOALLOC_MAX_CASES; 0 performs only the set-up.
 *   results[2*ncases]  host, caller-owned: per case max |error| and max |value|.
 * Scratch: 16 bytes per case in a fixed 256-byte device array inside the library
 * (one copy per device).  Every call zeroes the slots it uses before its kernels
 * run, so nothing has to be cleared by the caller.  The first call on a device
 * does the set-up (looks up that array's address, sets kernel attributes); make
 * it before any stream capture on that device.  Calls that overlap in time on
 * one device (other host threads or streams) share the array and race: the
 * caller must serialise them.  Work runs on the legacy default stream; the call
 * returns when the results are on the host.
 * Errors: DP_ERR_CAPACITY if ncases > DP_SELFTEST_NOALLOC_MAX_CASES (nothing runs);
 * DP_ERR_ARG for ncases < 0, a null array with ncases > 0, or a case outside 0..4;
 * DP_ERR_UNSUPPORTED on a device without tcgen05; DP_ERR_CUDA if the set-up, a
 * launch or the copy failed; DP_ERR_WAIT_TIMEOUT if an MMA wait gave up.
 */
#define DP_SELFTEST_NOALLOC_MAX_CASES 16
dp_status dp_selftest_noalloc(const int* which, int ncases, double* results);

/*
 * dp_wait_selftest -- check of the bounded-wait error path on the current device.  A
 * kernel waits, with the same bounded wait routine the tensor-core kernels use, on an
 * mbarrier phase that nothing completes (no copy or MMA is issued, so nothing is in
 * flight).  After spin_limit polls (1 .. 2^22) the wait gives up, sets the timeout bit
 * and the kernel returns; the device stays usable.  Returns DP_ERR_WAIT_TIMEOUT when
 * the wait gave up (the expected outcome), DP_OK if it did not, DP_ERR_ARG for a
 * spin_limit out of range, DP_ERR_UNSUPPORTED without tcgen05, DP_ERR_CUDA if the launch
 * failed.  Uses the legacy default stream; synchronous; allocates nothing.
 */
dp_status dp_wait_selftest(unsigned int spin_limit);

/*
 * dp_measure_peak -- measured throughput of an arithmetic unit on the current device
 * (measurement hook for rooflines): which = 0 tanh.approx.f32, 1 ex2.approx.f32,
 * 2 rcp.approx.f32 (results per second; each step also adds one, so that the chain
 * cannot fold), 3 FP32 FMA, 4 FP64 FMA (FLOP per second, two per FMA).  Every SM runs eight blocks of 256 threads, each thread eight independent
 * dependent chains of the instruction; CUDA events on a private stream, the fastest of
 * three launches after a warm-up.  rate [1] host output.  Synchronous; allocates
 * nothing.  DP_ERR_ARG for an unknown `which` or a null rate, DP_ERR_CUDA on failure.
 */
dp_status dp_measure_peak(int which, double* rate);

/* Wait for the model's stream; return and clear the sticky device error (DP_OK if none). */
dp_status dp_sync(dp_model* m);

/* Human-readable description of the last error on this model (never NULL). */
const char* dp_last_error(const dp_model* m);

/* Free every resource of the model (waits for its stream first).  NULL is a no-op. */
void dp_destroy(dp_model* m);

/* Library version string. */
const char* dp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DP_GB300_H */
