/*
 * misa.h -- C ABI of the GB300 (sm_103a) EAM lattice-list molecular dynamics
 * library: the per-timestep hot path of MISA-MD (Chu et al., arXiv:2107.07866).
 *
 * One simulation handle owns one periodic bcc crystal of nx x ny x nz cubic
 * cells (2 nx ny nz lattice sites and as many atoms) on one GPU.  Atoms live
 * in the lattice list of Sec. 3: a hash array with one slot per lattice site
 * (index = 2 nx ny z + 2 nx y + x, x in [0, 2 nx): even x = cube corner,
 * odd x = body centre) and a run-away list for atoms that have left their
 * site (the paper's hash-clash tree).  Each step evaluates the EAM potential
 * (Eq. eam_base, Eq. eam_force_ij, the five steps of Sec. 2.2) with spline
 * tables (Sec. 4.1) by a full-neighbour gather through the neighbour offset
 * index, then advances velocity Verlet (Fig. 1).
 *
 * Conventions
 *  - Units: Angstrom, eV, fs, amu, K.
 *  - Atom ids are 0 .. natoms-1; per-atom host arrays are indexed by atom id
 *    and hold x,y,z (or vx,vy,vz ...) interleaved: a[3*id + d].
 *  - Host array arguments may also be device pointers (copies use unified
 *    addressing); the caller keeps ownership of every buffer it passes.
 *  - Every call is asynchronous on the handle's stream except those that
 *    return host data (misa_get_*, misa_stats), which synchronise it.
 *  - Return value: MISA_OK (0) or a negative MISA_E* code; the message is in
 *    misa_last_error().  No call traps or aborts; device-side problems are
 *    reported through status bits (misa_stats) and MISA_EUNSTABLE /
 *    MISA_ERUNAWAY_OVERFLOW from the next synchronising call.
 *  - A handle is not thread-safe: one host thread and one stream per handle.
 */
#ifndef MISA_H
#define MISA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define MISA_OK 0
#define MISA_EINVAL (-1)             /* bad argument or parameter */
#define MISA_EOOM (-2)               /* device allocation failed */
#define MISA_ECUDA (-3)              /* a CUDA runtime call failed */
#define MISA_ERUNAWAY_OVERFLOW (-4)  /* more run-away atoms than the list holds */
#define MISA_EUNSTABLE (-5)          /* non-finite force or velocity */
#define MISA_ETIMEOUT (-6)           /* a bounded device wait gave up */

/* arithmetic of the force path */
#define MISA_FP64 0       /* everything in FP64 */
#define MISA_FP32_FORCE 1 /* FP32 density/force arithmetic with compensated sums; FP64 integration */

/* status bits (misa_stats.status), sticky until misa_clear_status */
#define MISA_ST_RUNAWAY_OVERFLOW 0x1u /* run-away list full: atoms were dropped from the physics */
#define MISA_ST_NONFINITE 0x2u        /* NaN/Inf in a force or velocity */
#define MISA_ST_RFLOOR 0x4u           /* a pair closer than 1e-4 A (value clamped, no force) */
#define MISA_ST_RHO_EXTRAP 0x8u       /* a density above the embedding table (linear tail used) */

/* Optional device allocator: the library calls alloc(bytes, ctx) for every
 * device buffer it owns and free(ptr, bytes, ctx) on destroy.  NULL: the
 * library uses cudaMalloc / cudaFree. */
typedef void *(*misa_alloc_fn)(size_t bytes, void *ctx);
typedef void (*misa_free_fn)(void *ptr, size_t bytes, void *ctx);

typedef struct misa_params {
    int32_t nx, ny, nz;       /* cubic cells per axis, each >= 6 */
    double a0;                /* lattice constant (A) */
    double mass;              /* atomic mass (amu) */
    double rc;                /* cutoff (A); f and phi are zero at and beyond it */
    double skin;              /* delta (A): an array atom farther than this from its site
                                 becomes a run-away; (rc + 2 skin) / (a0/2) must be < sqrt(27) */
    int32_t n_knots;          /* knots per table (>= 8) */
    const double *f_knots;    /* electron density f(r) at r_k = k rc/(n-1)      (Sec. 4.1) */
    const double *phi_knots;  /* pair potential phi(r) at the same r_k          (Sec. 4.1) */
    const double *F_knots;    /* embedding F(rho) at rho_k = k rho_max/(n-1)    (Sec. 4.1) */
    double rho_max;           /* end of the embedding table; linear beyond */
    int32_t precision;        /* MISA_FP64 or MISA_FP32_FORCE */
    int32_t reassign_period;  /* steps between hash updates that move run-aways back (Alg. 2) */
    double dt_max;            /* timestep cap (fs) */
    double dx_max;            /* adaptive step: dt = min(dt_max, dx_max / max|v|); 0 = fixed dt */
    int64_t runaway_capacity; /* run-away list size; 0 = max(4096, natoms/64); at most 16384 */
    misa_alloc_fn alloc;      /* optional allocator hooks (both or neither) */
    misa_free_fn free;
    void *alloc_ctx;
    int32_t tile;             /* gather tile choice: 0 = autotuned, else a misa_tile_* index */
} misa_params;

typedef struct misa_stats {
    int64_t step;       /* steps taken since create */
    double time;        /* simulated time (fs) */
    double dt;          /* timestep the next step will use (fs) */
    int64_t natoms;
    int64_t nsites;
    int64_t n_runaway;  /* atoms in the run-away list */
    int64_t n_vacant;   /* lattice sites without an atom (equals n_runaway) */
    uint32_t status;    /* MISA_ST_* bits */
    double vmax;        /* largest speed (A/fs) at the last step end */
    int64_t launches;   /* kernels this handle has launched (host-side count) */
} misa_stats;

/* Phases timed by misa_timing_get, in step order. */
#define MISA_PHASE_KICK_DRIFT 0   /* opening half kick + drift + demotions */
#define MISA_PHASE_LIST 1         /* hash update (Alg. 2), run-away list sort, tile marks */
#define MISA_PHASE_DENSITY 2      /* array density pass + embedding derivative */
#define MISA_PHASE_RA_DENSITY 3   /* run-away density */
#define MISA_PHASE_FORCE 4        /* array force pass + closing half kick */
#define MISA_PHASE_RA_FORCE 5     /* run-away force + closing half kick */
#define MISA_PHASE_END 6          /* step bookkeeping */
#define MISA_NPHASE 7

typedef struct misa_sim misa_sim;

/* Fills p with the analytic-potential-free defaults (a0 2.855, mass 55.845,
 * rc 5.6, skin 0.6, FP32_FORCE, reassign 10, dt_max 1, dx_max 0); the caller
 * still sets the box and the three knot tables. */
void misa_default_params(misa_params *p);

/* Creates the lattice list of a perfect crystal (Sec. 3, hash
 * initialization: every atom on its own site, no clashes; atom id = lattice
 * id), builds the neighbour offset index and the spline coefficients
 * (Sec. 4.1) on the device, sets velocities to zero and evaluates the
 * initial forces.  stream: a cudaStream_t (NULL = default stream).  The
 * knot arrays are copied.  On success *out owns all device memory. */
int misa_create(const misa_params *p, void *stream, misa_sim **out);

/* Batch of nrep independent replicas (Sec. 1 feature list: batch execution
 * of simulations) in one handle: replica r is a perfect crystal of
 * dims[3r] x dims[3r+1] x dims[3r+2] cells (each >= 6); p's own nx, ny, nz are
 * ignored.  All replicas share the potential, a0, skin, precision and tile
 * shape, and every step kernel serves all of them in one launch (one
 * persistent tile launch per pass); each replica keeps its own adaptive
 * timestep, time and run-away list.  Atom ids are concatenated in replica
 * order: replica r owns ids [atom_base(r), atom_base(r) + 2 n_x n_y n_z).
 * Every per-atom call below takes all atoms of the batch.  misa_create is
 * misa_create_batch with one replica. */
int misa_create_batch(const misa_params *p, int32_t nrep, const int32_t *dims, void *stream, misa_sim **out);

/* Replica count, and box / first atom id / atom count of replica r. */
int misa_replica_count(const misa_sim *s);
int misa_replica_info(const misa_sim *s, int32_t r, int32_t dims[3], int64_t *atom_base, int64_t *natoms);

/* Frees the handle and its device memory (after synchronising its stream). */
void misa_destroy(misa_sim *s);

/* Message of the last failed call on s (or of the last failed create when
 * s is NULL).  Valid until the next call on s. */
const char *misa_last_error(const misa_sim *s);

/* Replaces positions x (3 natoms, A, any periodic image) and, if v is not
 * NULL, velocities (3 natoms, A/fs); n must equal natoms.  Atoms are hashed to
 * their nearest sites (Sec. 3): an atom takes its site if the site is free
 * and the atom lies within skin of it (lowest atom id first), else it joins
 * the run-away list.  Then the forces of the new positions are evaluated. */
int misa_set_state(misa_sim *s, const double *x, const double *v, int64_t n);

/* Starts copying positions x and, if v is not NULL, velocities v (3 natoms
 * each, host or device memory, layout as in misa_set_state) into staging
 * buffers of the handle (48 B per atom of device memory, allocated on first
 * use) on a copy stream of its own, and returns at once: the copy runs
 * beside the steps already launched, so the next state streams in while
 * the current one is simulated.  The new copy waits on the device for the
 * previous staged state to have been read, and the call waits on the host
 * for the previous staged copy to be complete.  x and v must stay valid and
 * unchanged until this copy is complete: once the next misa_stage_state has
 * returned, the handle's stream has passed misa_set_state_staged, or
 * misa_destroy has returned (from pageable host memory the copy completes
 * before the call returns).  A second call before misa_set_state_staged
 * replaces the staged state.  MISA_EOOM if the staging buffers cannot be
 * allocated. */
int misa_stage_state(misa_sim *s, const double *x, const double *v, int64_t n);

/* misa_set_state from the state staged by misa_stage_state: the handle's
 * stream waits for the staged copy, then the atoms are hashed to their sites
 * and the forces of the new positions are evaluated, exactly as in
 * misa_set_state.  Velocities are set to zero if none were staged.
 * MISA_EINVAL if nothing is staged. */
int misa_set_state_staged(misa_sim *s);

/* Replaces the velocities (3 natoms, A/fs). */
int misa_set_velocities(misa_sim *s, const double *v, int64_t n);

/* Primary knock-on atom (Sec. 5.1): atom gets kinetic energy energy_eV along
 * dir (normalised here); atom = -1 picks the atom on the cube corner of cell
 * (nx/2, ny/2, nz/2), the box centre. */
int misa_insert_pka(misa_sim *s, int64_t atom, double energy_eV, const double dir[3]);

/* PKA of replica r: the atom at the centre of replica r's box. */
int misa_insert_pka_replica(misa_sim *s, int32_t r, double energy_eV, const double dir[3]);

/* Advances n steps of NVE velocity Verlet: kick, drift (array atoms leaving
 * their skin move to the run-away list), hash update every reassign_period
 * steps (Alg. 2), EAM density / embedding derivative / force passes
 * (Alg. 1 with the offset index), kick, next adaptive timestep.  Launches
 * only; never synchronises. */
int misa_step(misa_sim *s, int n);

/* misa_step(s, n) whose last step also evaluates the per-atom energies E_i
 * (Eq. eam_base: F(rho_i) + half the pair terms) inside its own density and
 * force passes -- the "calculate and output physical quantities" stage of
 * Fig. 1's MD loop at the output cadence -- so that a following
 * misa_get_energies / misa_replica_energies reads them without evaluating
 * the potential again.  Results are bitwise those of misa_step followed by
 * misa_get_energies.  The energies stay valid until the positions, the
 * tables or the species change.  MISA_EINVAL for n < 1.  Launches only. */
int misa_step_energies(misa_sim *s, int n);

/* misa_step captures one step as a CUDA graph on an internal stream (joined
 * to the handle's stream by events) and replays it; enable = 0 launches the
 * kernels one by one instead.  Timing (misa_timing_enable) always launches
 * directly. */
int misa_set_graphs(misa_sim *s, int enable);

/* Potential energy (sum of E_i, Eq. eam_base) and kinetic energy (eV) of
 * the current state; per_atom (natoms, may be NULL) receives E_i.
 * Synchronises. */
int misa_get_energies(misa_sim *s, double *pe, double *ke, double *per_atom);

/* Potential and kinetic energy of every replica (arrays of nrep). */
int misa_replica_energies(misa_sim *s, double *pe, double *ke);

/* E_i of every atom (Eq. eam_base) of the current state into per_atom
 * (n >= natoms doubles, indexed by atom id, host or device memory) without
 * waiting: the handle's stream writes them into a buffer of the handle (from
 * the last misa_step_energies, else after one evaluation of the potential)
 * and an output stream of the handle copies them to per_atom, so that the
 * caller's next calls (a new state, more steps) run beside the copy.  From
 * pinned host memory the copy is asynchronous; from pageable memory it may
 * complete before the call returns.  per_atom must stay valid, and its
 * contents are undefined, until misa_wait_outputs returns.  A later call
 * waits on the device for the previous copy before it overwrites the
 * buffer.  MISA_EOOM if the buffer (8 bytes per atom) cannot be allocated. */
int misa_get_energies_async(misa_sim *s, double *per_atom, int64_t n);

/* Waits for the copies started by misa_get_energies_async; status as for
 * the synchronous calls.  Synchronises. */
int misa_wait_outputs(misa_sim *s);

/* Per-atom host outputs (3 natoms doubles, or natoms for the density),
 * indexed by atom id; n must be >= natoms.  Positions are wrapped into the
 * box.  Forces are those of the current positions (eV/A).  Synchronise. */
int misa_get_positions(misa_sim *s, double *x, int64_t n);
int misa_get_velocities(misa_sim *s, double *v, int64_t n);
int misa_get_forces(misa_sim *s, double *f, int64_t n);
int misa_get_density(misa_sim *s, double *rho, int64_t n);

/* Lattice-list storage (for checks): site_atom (nsites) = atom id per site
 * or -1; runaway_ids (cap) = run-away atom ids in list order; *n_runaway =
 * their count.  Synchronises. */
int misa_get_site_map(misa_sim *s, int64_t *site_atom, int64_t *runaway_ids, int64_t cap,
                      int64_t *n_runaway);

/* Per-phase device timing of misa_step (CUDA events on the handle's
 * stream, recorded only while enabled).  misa_timing_get synchronises and
 * writes, for each of the MISA_NPHASE phases, the summed milliseconds
 * (ms[phase]) over the steps taken since timing was enabled or last read,
 * and their count (*steps); then it restarts the sums. */
int misa_timing_enable(misa_sim *s, int enable);
int misa_timing_get(misa_sim *s, double ms[MISA_NPHASE], int64_t *steps);

/* Counters and status bits of the batch (run-aways summed over replicas,
 * step / time / dt of replica 0; dt is 0 for batches), and of one replica.
 * The status bits are shared by the batch.  Synchronise. */
int misa_stats_get(misa_sim *s, misa_stats *out);
int misa_replica_stats(misa_sim *s, int32_t r, misa_stats *out);
int misa_clear_status(misa_sim *s);

/* Checkpoint / restart of the full dynamic state (positions, velocities,
 * accelerations, lattice list, step, time, dt) to a binary file. */
int misa_save(misa_sim *s, const char *path);
int misa_load(misa_sim *s, const char *path);

/* Replaces the knot values of the three tables (same count and grids as at
 * create; host or device pointers), rebuilds the spline coefficients on the
 * device (Sec. 4.1) and re-evaluates the forces of the current positions. */
int misa_set_tables(misa_sim *s, const double *f_knots, const double *phi_knots, const double *F_knots);

/* Alloys (Sec. 2.2: Eq. eam_base and Eq. eam_force_ij with atom types; the
 * n(n+1)/2 + 3n functions of an n-type system).  Replaces the potential by
 * n_species (1..4) types on the grids given at create:
 *   f_knots    n_species x n_knots  density function rho_a(r) of each type
 *   F_knots    n_species x n_knots  embedding function F_a(rho) of each type
 *   phi_knots  n_species (n_species + 1)/2 x n_knots  pair functions phi_ab(r),
 *              rows (a, b), a <= b, in the order (0,0), (0,1), .., (0,n-1), (1,1), ..
 *   types      natoms bytes: type of each atom id (ignored for one species)
 * Host or device pointers.  Types stay with the atoms; with one species the
 * single-type tables and gathers are used.  Recomputes the forces of the
 * current positions and drops a captured step graph; synchronises;
 * MISA_EINVAL for a type outside [0, n_species) or when no tile shape fits
 * the alloy passes' shared memory.  FP32 handles run the packed tile
 * gathers with the species of every staged site, the most populous
 * species' density window in shared memory and the other tables through
 * the texture path (the tile shapes are re-chosen if the current ones do not
 * fit); FP64 handles run one thread per site with tables in global memory.
 * misa_loss_grad and misa_save keep to one type.  misa_set_tables returns
 * to one type. */
int misa_set_species(misa_sim *s, int n_species, const double *f_knots, const double *F_knots,
                     const double *phi_knots, const int8_t *types);

/* Potential fitting (no counterpart in the paper): loss and its gradient
 * with respect to the 3 n_knots knot values, for the current positions of
 * every replica against target forces Fref (3 natoms doubles, eV/A, by atom
 * id) and target energies Eref (nrep doubles, eV):
 *   loss = sum_r [ (1/(3 N_r)) sum_i |F_i - Fref_i|^2 + ((E_r - Eref_r)/N_r)^2 ]
 * (Eq. eam_base for E, Eq. eam_force_ij for F).  grad (3 n_knots doubles,
 * host or device; may be NULL) receives d loss / d knot in the order f knots,
 * phi knots, F knots.  Pair arithmetic and the per-CTA shared-memory bins
 * (5 n_knots values: the pair terms go to the values and slopes of their
 * segment's end knots) in the handle's precision, one ordered FP64
 * reduction over CTAs.  MISA_EINVAL for a handle with several species or
 * when the bins exceed a block's shared memory (n_knots > 11622 for FP32,
 * > 5811 for FP64).  Synchronises. */
int misa_loss_grad(misa_sim *s, const double *Fref, const double *Eref, double *loss, double *grad);

/* Number of built gather tile shapes, and the shape of each (cells). */
int misa_tile_count(void);
int misa_tile_shape(int index, int *tx, int *ty, int *tz);

/* Self-test of two shortcuts of the library that have no counterpart in the
 * paper.  (1) The float <-> double conversions done with integer operations
 * (used by the FP64 integration kernels), against the GPU's own conversions
 * on n generated bit patterns: mismatches[0] counts double -> float,
 * mismatches[1] float -> double disagreements (a subnormal result flushed to
 * a signed zero is not one).  (2) The hash of Sec. 3 with the site decided
 * in FP32 under a certifying margin (used when a state is set), against the
 * all-FP64 hash on n generated positions (thermal, near floor and distance
 * ties, exact ties, uniform): mismatches[2] counts positions whose site or
 * displacement differs in any bit.  mismatches holds 3 values.  Runs on the
 * current device, synchronises; MISA_EINVAL for n <= 0 or a null pointer,
 * MISA_ECUDA on a CUDA error. */
int misa_selftest(long long n, long long *mismatches);

/* 1 if shape `index` (1-based) is built for `precision`, else 0.  The FP64
 * gathers run one thread per site (2 tx ty tz <= 1024); the FP32 gathers run
 * two sites per thread, the tile folded in z (tz even, tx ty tz <= 1024).
 * Creating a handle with a shape its precision lacks returns MISA_EINVAL. */
int misa_tile_valid(int precision, int index);

/* Tile shapes in use (1-based indices) by the density pass and by the force
 * pass.  With misa_params.tile = 0 the autotuner times both passes of the
 * initial state for every shape built for the precision whose table window
 * and staged tile fit the shared memory of a block, and keeps the fastest
 * shape of each pass; otherwise both passes use misa_params.tile. */
int misa_tile_current(const misa_sim *s);
int misa_tile_current_force(const misa_sim *s);

/* Density-pass variant of an FP32 single-type handle.
 *   0  full-neighbour gather (default): every site evaluates all its pairs.
 *   1  Newton's third law inside a tile (Sec. 4.2's halving of the pair
 *      work): each dense-shell pair of two sites of one tile is evaluated
 *      once and its density handed to the partner through shared memory
 *      (no atomics); pairs that reach outside the tile are evaluated by the
 *      site itself.  Per-site sums keep a fixed order, so results do not
 *      depend on the tile shape; they differ from variant 0 in the last FP32
 *      bits (another summation order).
 * The force pass is the full-neighbour gather either way.  Recomputes the
 * forces of the current positions; drops a captured step graph;
 * synchronises.  MISA_EINVAL for another variant, for variant 1 on an FP64
 * or alloy handle, or when no tile shape fits the pass's shared memory. */
int misa_set_density_variant(misa_sim *s, int32_t variant);

/* Wigner-Seitz defect count of every replica (Sec. 5.1, the vacancy and
 * interstitial counts behind the Frenkel-pair curves): each atom belongs to
 * the cell of its nearest site -- an array atom to its own site, a run-away
 * to its home -- and since atoms = sites, vacancies = interstitials =
 * Frenkel pairs.  n_frenkel receives nrep counts (host memory).  Uses the
 * library's scratch; synchronises. */
int misa_defects(misa_sim *s, int64_t *n_frenkel);

/* Re-runs the tile autotuner on the current state (call it once after
 * loading a representative configuration, e.g. an equilibrated crystal:
 * the shapes that win on the perfect crystal of misa_create are not always
 * the ones that win at temperature).  Results do not depend on the shapes;
 * only speed does.  No-op when misa_params.tile fixed the shape.  Leaves
 * the forces of the current positions in place; drops a captured step
 * graph; synchronises. */
int misa_retune(misa_sim *s);

/* Issue-rate microbenchmarks of the current device (no counterpart in the
 * paper): the denominators of the arithmetic rooflines of the gathers and of
 * the FP64 path, measured rather than derived from unit counts and the
 * clock.  Each figure is the best of five timed launches (CUDA events on
 * `stream`, NULL = default stream) of a kernel that fills every warp slot of
 * every SM with independent dependency chains of one instruction:
 *   fp32_ffma_tflops    scalar FP32 FMA (2 flops each)
 *   fp32_ffma2_tflops   packed FP32x2 FMA (4 flops each)
 *   fp64_dfma_tflops    FP64 FMA (2 flops each)
 *   mufu_rsqrt_tops     approximate reciprocal square roots (1e12 per s)
 *   lds128_tbps         conflict-free 16-byte shared-memory loads (TB/s)
 *   sm_clock_mhz        SM clock during the FP32 probe (clock64 against the
 *                       global timer in one CTA)
 *   num_sms             multiprocessors of the device
 * Runs on the current device for ~0.2 s; changes no device setting;
 * synchronises the stream.  MISA_EINVAL for a null pointer, MISA_ECUDA on a
 * CUDA error. */
typedef struct misa_peaks {
    double fp32_ffma_tflops;
    double fp32_ffma2_tflops;
    double fp64_dfma_tflops;
    double mufu_rsqrt_tops;
    double lds128_tbps;
    double sm_clock_mhz;
    int32_t num_sms;
} misa_peaks;
int misa_measure_peaks(misa_peaks *out, void *stream);

/* Allocation-free force evaluation (the paper has no counterpart; it exists
 * for callers that must not allocate device memory).
 *
 * Some callers cannot call cudaMalloc: code that runs inside a framework
 * whose memory pool owns every device byte, code on a latency-critical path
 * where cudaMalloc's implicit device synchronisation is not acceptable, and
 * plug-ins loaded into a host program that has reserved the GPU's memory up
 * front.  For them this entry point computes what misa_set_state followed by
 * misa_get_forces / misa_get_energies computes -- per-atom EAM forces
 * (Eq. eam_force_ij) and per-atom energies E_i (Eq. eam_base) of an
 * explicit configuration -- without creating a handle and without any
 * device allocation: its working memory is one file-scope __device__ array
 * of the library (MISA_STATIC_SCRATCH_BYTES, about 9 MB), which every GPU
 * that loads the library holds until the process exits.
 *
 *   nx, ny, nz    box in cubic bcc cells (each >= 6); natoms = 2 nx ny nz
 *                 must not exceed MISA_STATIC_MAX_ATOMS
 *   a0, rc, skin  as in misa_params
 *   n_knots       knots per table, 8 .. MISA_STATIC_MAX_KNOTS (the FP32 path
 *                 keeps the reachable part of a table in shared memory beside
 *                 one 8x8x8-cell tile: up to 8192 knots fit a GB300 block;
 *                 a window that does not fit returns MISA_EINVAL)
 *   knots         DEVICE pointer, 3 n_knots doubles: f, phi, F knot values
 *                 (same grids as misa_params)
 *   rho_max       end of the embedding table
 *   precision     MISA_FP64 or MISA_FP32_FORCE
 *   x             DEVICE pointer, 3 natoms doubles, positions (A)
 *   forces        DEVICE pointer, 3 natoms doubles, output (eV/A), by atom id
 *   energies      DEVICE pointer, natoms doubles, output E_i (eV), or NULL
 *   stream        cudaStream_t to run on (NULL = default stream)
 * The caller owns all four buffers.  At most MISA_STATIC_RUNAWAY_CAP atoms
 * may be off their lattice sites (else MISA_ERUNAWAY_OVERFLOW).  Sizes
 * beyond the limits return MISA_EINVAL without touching the GPU; the
 * message is in misa_last_error(NULL).
 *
 * The first call on a device looks up the device address of the scratch
 * array (set-up, once per device, with that device current); make that
 * first call before any stream capture on the device.  Every call shares
 * the one array and clears the parts that must start from zero; calls that
 * overlap on the GPU (several streams or host threads at once) race on it
 * and must be serialised by the caller.  Returns when the outputs are
 * complete (it synchronises the stream). */
#define MISA_STATIC_MAX_ATOMS 32768
#define MISA_STATIC_MAX_KNOTS 8192
#define MISA_STATIC_RUNAWAY_CAP 1024
#define MISA_STATIC_SCRATCH_BYTES (9u * 1024u * 1024u)
int misa_eam_forces_static(int32_t nx, int32_t ny, int32_t nz, double a0, double rc, double skin,
                           int32_t n_knots, const double *knots, double rho_max, int32_t precision,
                           const double *x, double *forces, double *energies, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MISA_H */
