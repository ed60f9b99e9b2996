/*
 * slpic.h -- C ABI of libslpic, a GB300 (sm_103a) implementation of the
 * per-marker step of speed-limited particle-in-cell with Monte-Carlo
 * collisions (SLPIC-MCC) for a 1D3V argon-filled parallel-plate gap
 * (Theis, Werner, Jenkins, Cary, "Computing the Paschen curve for argon with
 * speed-limited particle-in-cell simulation").
 *
 * One context holds one or more independent instances (gaps at their own
 * pressure and voltage); every instance has an electron and an Ar+ species.
 * All instances advance together in one batched launch per phase.
 *
 * Conventions used by every call:
 *  - SI units, except energies, which are in eV.
 *  - Cathode at x = 0 (phi = 0), anode at x = d (phi = V); E_x = -dphi/dx.
 *  - Species index: SLPIC_ELECTRON (0) or SLPIC_ION (1).
 *  - Marker storage (FP32 path): struct-of-arrays of int32 cell in [0, N),
 *    float offset in [0, 1) inside the cell, float vx, vy, vz [m/s], float
 *    flux weight w_j (physical particles represented per crossing, constant
 *    along a trajectory, Sec. II.B), uint32 id.  Bit 31 of the id is the
 *    generation flag (0: descends from a seeded electron without passing
 *    through secondary emission); bits 0-30 are a serial number unique within
 *    the species.
 *  - Host pointers are read or written only during the call; the library
 *    never keeps them.  Device pointers passed to *_device calls must point
 *    to memory of the context's device and stay valid during the call.
 *  - Every call returns SLPIC_OK (0) or a negative SLPIC_ERR_* code and then
 *    leaves a message in slpic_last_error().  Errors raised on the GPU during
 *    slpic_step (capacity, wait time-out) are latched in device memory and
 *    returned by the next call that synchronises (reads, slpic_synchronize);
 *    after such an error further steps are no-ops until slpic_clear_error(),
 *    and the markers of the failed step are in an unspecified state (the step
 *    updates the stores in place): load or seed them again.
 *  - A context is not thread-safe; use one host thread per context.
 */
#ifndef SLPIC_H
#define SLPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SLPIC_OK 0
#define SLPIC_ERR_INVALID_ARG (-1)
#define SLPIC_ERR_STATE (-2)
#define SLPIC_ERR_CAPACITY (-3)
#define SLPIC_ERR_CUDA (-4)
#define SLPIC_ERR_TIMEOUT (-5)
#define SLPIC_ERR_NUMERIC (-6)

#define SLPIC_ELECTRON 0
#define SLPIC_ION 1

#define SLPIC_FIELD_FROZEN 0  /* vacuum field -V/d at every node, never solved */
#define SLPIC_FIELD_POISSON 1 /* 1D Poisson solve after every step's deposit */

#define SLPIC_SEED_CATHODE 0  /* uniform in cell 0, energy e0, forward hemisphere */
#define SLPIC_SEED_REST 1     /* at x = 0 with zero velocity (the paper's seeding) */
#define SLPIC_SEED_GAP 2      /* uniform over the gap, energy log-uniform, isotropic */
#define SLPIC_SEED_THERMAL 3  /* uniform over the gap, gas-temperature Maxwellian */

typedef struct slpic_ctx slpic_ctx;

/* FP32 marker arrays (host or device pointers, as the call states). */
typedef struct {
  int32_t* cell;
  float* off;
  float* vx;
  float* vy;
  float* vz;
  float* wj;
  uint32_t* id;
} slpic_soa_f32;

/* FP64 marker arrays, for contexts whose marker path is FP64. */
typedef struct {
  int32_t* cell;
  double* off;
  double* vx;
  double* vy;
  double* vz;
  double* wj;
  uint32_t* id;
} slpic_soa_f64;

/* What happened in one step of one instance (or, from slpic_read_tallies, the
 * sums over all steps since the last seed/load).  Counts are exact; weight
 * sums are exact integer sums of w_j in units of 2^-charge_shift converted to
 * double at read time. */
typedef struct {
  int64_t step;            /* index of the step (last step for sums) */
  int64_t n_live[2];       /* live markers after the step */
  double w_live[2];        /* sum of w_j of live markers after the step */
  int64_t n_coll[3];       /* real collisions: elastic, excitation, ionization */
  int64_t n_candidates;    /* null-collision candidates (u1 < P0) */
  int64_t n_abs[2][2];     /* absorbed [species][0 cathode, 1 anode] */
  double w_abs[2][2];      /* their sum of w_j (flux through the electrode, Eq. j) */
  int64_t n_see;           /* secondary electrons emitted at the cathode */
  double w_see;
  double w_ionz;           /* sum of w_j of ionizing electrons (= born ions) */
  double w_cath_ion;       /* sum of w_j of ions absorbed at the cathode */
  double w_cath_ion_gen0;  /* same, first-generation ions only */
  int64_t n_clamp;         /* energies clamped at 0 after an inelastic event */
  int64_t n_majorant;      /* electrons whose beta*v exceeded the majorant's cap */
  int64_t marker_steps;    /* markers advanced (both species) */
  double w_gain_gen0;      /* sum of yield * w_j of first-generation ions at
                              the cathode (the gain's numerator) */
} slpic_tallies;

/* Library version as an integer MMmmpp. */
int slpic_version(void);

/* Message of the last failed call on ctx (owned by ctx; valid until the next
 * call).  With ctx = NULL: the last failure of slpic_create or
 * slpic_philox_static. */
const char* slpic_last_error(const slpic_ctx* ctx);

/* Create a context on CUDA device `device` with `n_instances` >= 1 instances.
 * Nothing is allocated on the device until the first seed/load/step. */
int slpic_create(slpic_ctx** out, int device, int n_instances);
int slpic_destroy(slpic_ctx* ctx);

/* Stream for all device work of ctx (a cudaStream_t, e.g. PyTorch's current
 * stream); NULL = the legacy default stream. */
int slpic_set_stream(slpic_ctx* ctx, void* cuda_stream);

/* Gap of instance `inst` (Sec. IV): width d [m], n_cells >= 2 uniform cells,
 * anode potential V [V], field mode (SLPIC_FIELD_*), electrode area [m^2]
 * that the flux weights refer to (charge density = sum e w_p / (area dx)). */
int slpic_set_gap(slpic_ctx* ctx, int inst, double d, int n_cells, double V,
                  int field_mode, double area);
/* Change only the anode potential (allowed between runs, e.g. bisection over
 * V); the vacuum field is reset to -V/d. */
int slpic_set_voltage(slpic_ctx* ctx, int inst, double V);
/* Background argon at rest: pressure [Pa], temperature [K]; n_g = p/(k T). */
int slpic_set_gas(slpic_ctx* ctx, int inst, double p_Pa, double T_K);
/* Electron-argon cross sections [m^2] at the nodes of an octave-uniform
 * energy grid: node j = o 2^log2_sub + m sits at 2^(lo_exp2 + o)
 * (1 + m / 2^log2_sub) eV, j = 0 .. octaves 2^log2_sub (inclusive).  Values
 * are interpolated linearly in energy and held constant outside the grid.
 * Elastic (Vahedi-Surendra angles), one excitation level (threshold e_ex, eV)
 * and ionization (threshold e_io, eV), Sec. IV.  Host arrays, copied.
 * inst = -1 sets every instance. */
int slpic_set_cross_sections(slpic_ctx* ctx, int inst, int lo_exp2,
                             int log2_sub, int octaves, const float* sig_el,
                             const float* sig_ex, double e_ex,
                             const float* sig_io, double e_io);
/* The same with n_exc (1..3) excitation levels: the five processes of
 * Sec. IV (elastic, three excitations, ionization).
 * - sig_ex[k] and e_ex[k] are level k's cross sections and threshold [eV].
 * - A collision picks the first process, in the order elastic, level 1 ..
 *   n_exc, ionization, whose cumulative rate exceeds the draw.
 * - An excitation removes its level's threshold and scatters isotropically.
 * - The tallies count every excitation level under n_coll[1]. */
int slpic_set_cross_sections_levels(slpic_ctx* ctx, int inst, int lo_exp2,
                                    int log2_sub, int octaves, const float* sig_el,
                                    int n_exc, const float* const* sig_ex,
                                    const double* e_ex, const float* sig_io,
                                    double e_io);
/* Species: mass [kg], charge [C], speed limit v_lim [m/s] of Eq. betaAbrupt
 * (beta = min(1, v_lim/|v|); v_lim <= 0 or +inf gives beta = 1, i.e. PIC),
 * capacity = maximum live markers (rounded up to whole tiles of 128 markers,
 * plus one tile).  Only electrons collide (Sec. IV).  Device memory per slot
 * of capacity: two buffers of the seven marker fields (56 B in FP32, 96 B in
 * FP64), and for electrons a null-collision candidate record (32 B in FP32,
 * 64 B in FP64) and the staging of emitted electrons (28 B or 48 B per ion
 * slot). */
int slpic_set_species(slpic_ctx* ctx, int inst, int species, double mass,
                      double charge, double v_lim, int64_t capacity);
/* Ion-induced secondary-electron yield gamma at the cathode (constant; the
 * emitted electron starts at x = 0 with zero velocity, Sec. IV). */
int slpic_set_emission(slpic_ctx* ctx, int inst, double gamma_se);
/* Yield model: SLPIC_EMISSION_CONSTANT (gamma of slpic_set_emission, the
 * default) or SLPIC_EMISSION_ENERGY, the energy-dependent yield of Eq. sey:
 * 0.09 (eps_i / 700 eV)^0.05 below 700 eV and 0.09 (eps_i / 700 eV)^0.72
 * from 700 eV on, eps_i the ion's kinetic energy when it crosses the
 * cathode.  An ion emits when its Philox draw is below the yield; the
 * expected yield of first-generation ions is tallied in w_gain_gen0. */
#define SLPIC_EMISSION_CONSTANT 0
#define SLPIC_EMISSION_ENERGY 1
int slpic_set_emission_model(slpic_ctx* ctx, int inst, int model);
/* Time step [s]. */
int slpic_set_dt(slpic_ctx* ctx, int inst, double dt);
/* Random stream: 64-bit Philox key of the instance. */
int slpic_set_seed(slpic_ctx* ctx, int inst, uint64_t seed);
/* Fixed point of the deposit: one unit of charge = 2^-shift flux weights
 * (0 <= shift <= 40; the weights times 2^shift must stay below 2^39). */
int slpic_set_charge_shift(slpic_ctx* ctx, int inst, int shift);

/* Time-step rules of Sec. IV for a gap of n_cells cells at voltage V:
 * mode 0 (SLPIC) dt = dx / v0 with v0 = sqrt(2 e V / m_ion); mode 1 (PIC)
 * dt = dx / sqrt(2 e V / m_e).  Host arithmetic only. */
int slpic_suggest_dt(double d, int n_cells, double V, double m_ion, int mode,
                     double* dt_out);

/* Seed n markers of `species` on the device (appended to the live ones),
 * drawn from the instance's Philox stream (counter word 1 = 0xFFFFFFFF):
 * mode SLPIC_SEED_*; e0 [eV] for SEED_CATHODE; [e_lo, e_hi] eV for SEED_GAP;
 * every marker gets flux weight wj.  Seeded electrons add to the instance's
 * seeded weight (the gain's denominator); the step counter and the tallies
 * go on (slpic_reset_counters restarts them). */
int slpic_seed(slpic_ctx* ctx, int inst, int species, int64_t n, int mode,
               double e0, double e_lo, double e_hi, double wj);
/* Arithmetic type of the marker path: 32 (default; positions, velocities and
 * weights in float, the deposit in int64 fixed point, the field solve and
 * tallies in double) or 64 (everything of the marker path in double, the
 * plain FP64 form).  Set before the first use of the context; the FP32
 * marker calls then fail with SLPIC_ERR_STATE and the _f64 ones are used. */
int slpic_set_precision(slpic_ctx* ctx, int bits);

/* Replace the markers of `species` by n markers from host arrays (FP32 SoA);
 * next_id = serial number of the next born marker.  Cells must lie in
 * [0, N) and offsets in [0, 1).  For electrons the loaded weight becomes the
 * seeded weight; the step counter and the tallies go on
 * (slpic_reset_counters restarts them). */
int slpic_load_particles(slpic_ctx* ctx, int inst, int species,
                         const slpic_soa_f32* host, int64_t n,
                         uint32_t next_id);
/* Same from device arrays (device-to-device copies, no host staging). */
int slpic_load_particles_device(slpic_ctx* ctx, int inst, int species,
                                const slpic_soa_f32* dev, int64_t n,
                                uint32_t next_id);
/* slpic_load_particles for an FP64 context (host FP64 SoA). */
int slpic_load_particles_f64(slpic_ctx* ctx, int inst, int species,
                             const slpic_soa_f64* host, int64_t n,
                             uint32_t next_id);
/* Reset the step counter and tallies without touching the markers. */
int slpic_reset_counters(slpic_ctx* ctx, int inst);

/* Advance every instance by n_steps steps (asynchronous on the context's
 * stream).  One step: gather, speed-limited kick and drift, absorption and
 * secondary emission, null-collision MCC with births, stable compaction and
 * append, fixed-point deposit, field solve, tallies. */
int slpic_step(slpic_ctx* ctx, int64_t n_steps);
/* Steps of small populations (Sec. V: the breakdown runs start from 100
 * electrons and stay near that size): up to n_steps steps of every instance
 * in one launch, one CTA of the device per instance, with no per-step launch.
 * Synchronous.  Runs only while every store has at most the small-path limit
 * of tiles (128 markers each, slpic_set_small_limit) when a step starts, and
 * stops before the first step at which one has more; *steps_done gets the
 * steps run (0 when the path does not apply: a store above the limit, a store
 * too small to take one step's births from there (3 x the limit for
 * electrons, 2 x for ions), a field-mode-1 grid too large for shared memory,
 * more instances than fit on the device at once, or profiling on).  The
 * results are those of slpic_step, bit for bit; continue with slpic_step for
 * the remaining steps.  The tallies, history, counts and fields read after
 * it are those of the last step run. */
int slpic_step_small(slpic_ctx* ctx, int64_t n_steps, int64_t* steps_done);
/* Small-path limit: most tiles (128 marker slots each) a store may hold when
 * a step of slpic_step_small starts, 0..32 (default 32; 0 switches the path
 * off).  slpic_ion_trend and slpic_paschen_bisect take the small path by
 * themselves while the populations are within it. */
int slpic_set_small_limit(slpic_ctx* ctx, int max_tiles);
/* Wait for the context's work; returns the latched device error, if any. */
int slpic_synchronize(slpic_ctx* ctx);
/* Forget a latched device error (load or seed the markers again after it). */
int slpic_clear_error(slpic_ctx* ctx);

/* Reads (synchronise first).  Host buffers are caller-owned. */
int slpic_count(slpic_ctx* ctx, int inst, int species, int64_t* n_out);
int slpic_read_particles(slpic_ctx* ctx, int inst, int species,
                         const slpic_soa_f32* host, int64_t capacity,
                         int64_t* n_out);
/* slpic_read_particles for an FP64 context. */
int slpic_read_particles_f64(slpic_ctx* ctx, int inst, int species,
                             const slpic_soa_f64* host, int64_t capacity,
                             int64_t* n_out);
/* Fixed-point deposit of the last step (n_cells + 1 int64 node values;
 * all zero before the first step and after slpic_reset_counters).  A step's
 * deposit is a function of the markers after it: each live marker adds
 * round(beta(|v|) w_j 2^shift) split linearly between its cell's nodes.
 * With field_mode 1 the step forms it (the Poisson solve needs it); with an
 * imposed field the step deposits nothing and this call (or a load or seed,
 * before it changes the markers) forms it from the markers.  The integers are
 * the same either way.  Synchronises; returns a latched device error. */
int slpic_read_charge(slpic_ctx* ctx, int inst, int species, int64_t* host,
                      int64_t n);
/* Number density at the nodes [m^-3] of the last step's deposit (boundary
 * nodes count half a cell). */
int slpic_read_density(slpic_ctx* ctx, int inst, int species, double* host,
                       int64_t n);
/* Potential [V] and field [V/m] at the n_cells + 1 nodes. */
int slpic_read_field(slpic_ctx* ctx, int inst, double* phi, double* E,
                     int64_t n);
/* Sums over all steps since the last seed/load/reset. */
int slpic_read_tallies(slpic_ctx* ctx, int inst, slpic_tallies* out);
/* Per-step records of the last min(n_steps, ring) steps, oldest first. */
int slpic_read_history(slpic_ctx* ctx, int inst, slpic_tallies* out,
                       int64_t capacity, int64_t* n_out);
/* Electrode currents of the last step [A]: e * (sum of w_j crossing) / dt,
 * positive for charge flowing into the gap's external circuit direction
 * x = 0 -> d. */
int slpic_read_current(slpic_ctx* ctx, int inst, double* I_anode,
                       double* I_cathode);
/* First-generation secondary-emission gain G = (sum of yield * w_j over
 * first-generation ions absorbed at the cathode) / (sum of seeded w_j):
 * expected emitted electrons per seed electron (with a constant yield,
 * gamma times the ions' flux weight); G >= 1 is the Townsend breakdown
 * criterion gamma (e^(alpha d) - 1) >= 1 (Sec. II.A). */
int slpic_read_gain(slpic_ctx* ctx, int inst, double* G);

/* Breakdown-voltage search over a batch (Sec. V, Fig. paschen): the context
 * holds n_pd * n_v configured instances, instance p * n_v + j being voltage j
 * of pd point p (gap, gas, cross sections, species capacities and gamma set
 * by the caller).  Every round, each pd point's bracket [lo, hi] is cut at
 * n_v interior voltages V_j = lo + (hi - lo)(j + 1)/(n_v + 1), one per
 * instance, and each instance runs one avalanche:
 *  - electron v_lim = vlim_factor sqrt(2 e V / M) and dt = dx / v_lim
 *    (vlim_factor <= 0: standard PIC, beta = 1, dt = dx / sqrt(2 e V / m_e));
 *  - its markers are replaced by n_seed electrons at the cathode (energy e0,
 *    SLPIC_SEED_CATHODE, unit weight), with the instance's seed advanced by
 *    the round;
 *  - secondary emission is switched off during the run (the yield model
 *    stays), and the gain G = (yield * flux weight of first-generation ions
 *    reaching the cathode) / (seeded weight) is its expected value
 *    (Townsend: G >= 1 is breakdown, Sec. II.A);
 *  - the batch steps until every instance has no marker left, or
 *    max_steps, in chunks of at most chunk_steps steps between checks of the
 *    live counts: a chunk is shortened so that no store can overflow in it
 *    (electrons at most double per step); an instance with more than
 *    (1 + 1/gamma) n_seed live electrons or at least n_seed/gamma live ions
 *    is above breakdown for certain (each ionization leaves an ion that
 *    reaches the cathode; gamma is the constant yield, or for Eq. sey the
 *    yield 0.09 (0.1 eV / 700 eV)^0.05 of an ion that fell through 0.1 V,
 *    a bound for every ion born more than 0.1 V from the cathode): it is
 *    emptied and counts as G = +inf.  Every instance needs gamma > 0 and
 *    capacities of at least
 *    2 (1 + 1/gamma) n_seed electrons and n_seed/gamma + (1 + 1/gamma) n_seed
 *    ions, else SLPIC_ERR_INVALID_ARG.
 * Then each bracket shrinks to [V_{j-1}, V_j] around the first j with
 * G >= 1 (V_{-1} = lo, V_{n_v} = hi).  On return Vb_lo/Vb_hi [n_pd] hold the
 * final brackets and, if not NULL, gain [n_pd * n_v] the last round's G.  The
 * instances keep the last round's voltage, v_lim and dt; emission is on again.
 * Errors as the other calls (a capacity error cannot occur: see above). */
typedef struct {
  int n_pd;            /* pd points */
  int n_v;             /* voltages per pd point and round */
  int rounds;          /* section-search rounds (>= 1) */
  int64_t n_seed;      /* electrons seeded per instance and round */
  double e0;           /* their energy [eV] */
  double vlim_factor;  /* see above */
  int64_t chunk_steps; /* most steps between checks of the live counts */
  int64_t max_steps;   /* per round */
  const double* V_lo;  /* [n_pd] initial bracket [V] */
  const double* V_hi;  /* [n_pd] */
} slpic_paschen_spec;
int slpic_paschen_bisect(slpic_ctx* ctx, const slpic_paschen_spec* spec, double* Vb_lo,
                         double* Vb_hi, double* gain);

/* The paper's breakdown test (Sec. V): advance every instance by n_windows
 * windows of steps_per_window steps and write each instance's mean number of
 * live ions per window to means [n_inst * n_windows] (instance-major).
 * - Below breakdown the ion population falls back to zero after its first
 *   rise; above it, it keeps growing.
 * - above [n_inst] (may be NULL) is 1 when the last window's mean is
 *   positive and exceeds every earlier window's, else 0.
 * - An instance whose live markers (both species) pass a third of the
 *   smaller store's capacity is above breakdown. It is emptied, its
 *   remaining windows read -1, and it counts as above.  When every instance
 *   has stopped so, no further step is taken.
 * - Steps run in chunks short enough that no store can overflow in between
 *   (growth at most x3 per step with emission).
 * - With the paper's setup: seed electrons at rest (SLPIC_SEED_REST),
 *   n_windows * steps_per_window = 30 ion crossing times, the Eq. sey yield. */
int slpic_ion_trend(slpic_ctx* ctx, int64_t steps_per_window, int n_windows, double* means,
                    int* above);

/* Checkpoint and resume.  slpic_save writes the context's state to a host
 * buffer: per instance the live markers of both species in store order and
 * their next serial numbers, the step counters (step index, steps done,
 * seeded and live weights, live-ion sum), the tally totals and the history
 * ring, the node field (phi and E) and the last deposit.  The configuration
 * (gap, gas, tables, species, emission, dt, seed, capacities) is not in it.
 * With buf = NULL only *size_out (the snapshot's bytes) is written; with a
 * buffer smaller than that, SLPIC_ERR_CAPACITY.  Synchronises.
 * slpic_load restores such a snapshot into a context configured as the
 * saved one was (same instance count, precision, cells and ring length,
 * capacities holding the markers; else SLPIC_ERR_INVALID_ARG or
 * SLPIC_ERR_CAPACITY).  Steps after a load give, bit for bit, the results
 * the saved context would have given.  A library utility; the method has no
 * counterpart. */
int slpic_save(slpic_ctx* ctx, void* buf, size_t capacity, size_t* size_out);
int slpic_load(slpic_ctx* ctx, const void* buf, size_t size);

/* Bounded waits: every wait of a kernel on data another thread block
 * produces (bulk-copy barriers, the ordered scans' look-back, the single-CTA
 * path's grid barrier) gives up after this many polls, latches
 * SLPIC_ERR_TIMEOUT and lets the kernel return; the next synchronising call
 * returns the error and steps are no-ops until slpic_clear_error.  0 restores
 * the default (2^22 polls, seconds).  A library utility; the method has no
 * counterpart. */
int slpic_set_spin_limit(slpic_ctx* ctx, uint32_t polls);
/* Test hook for the bounded waits: once, in a launch of the single-CTA path
 * with more than one instance, the thread block of instance `inst` leaves
 * out its arrival at grid barrier `barrier` (the barrier taken after
 * barrier - 1 steps of the launch; 1 = before its first step).  Every
 * block's wait at that barrier then runs out after the spin limit, the
 * launch ends there, and the call that stepped returns SLPIC_ERR_TIMEOUT.
 * inst = -1 switches the hook off.  After the timeout, slpic_clear_error and
 * a fresh load or seed make the context usable again.  A library utility;
 * the method has no counterpart. */
int slpic_test_skip_barrier(slpic_ctx* ctx, int inst, int64_t barrier);

/* Multiplication per ion transit (Sec. V: the population over windows of
 * one ion crossing time sqrt(2 M d / (e E))).  Advances every instance by
 * n_windows windows of steps_per_window steps (the single-CTA path while the
 * stores are small, then the batched kernels) and writes:
 * - see [n_inst * n_windows] (instance-major): the flux weight of the
 *   electrons emitted at the cathode in each window (the sum of their w_j,
 *   Eq. j), from the FP64 running totals the step keeps on the device;
 * - M [n_inst * (n_windows - 1)] (may be NULL): the multiplication of each
 *   window over the one before, see_k / see_{k-1} (NaN after a window with
 *   no emission).
 * Below breakdown M < 1 and the emission dies out; above it M > 1.  The
 * caller sizes the stores for the growth it expects: a store that
 * overflows ends the call with SLPIC_ERR_CAPACITY, as slpic_step does. */
int slpic_multiplication(slpic_ctx* ctx, int64_t steps_per_window, int n_windows, double* see,
                         double* M);

/* Launch shape of the step: warps per CTA of the particle kernel (a
 * multiple of 4, at most 20; each warp owns a 128-slot tile) and CTAs per
 * SM of the collision kernel (1..32).  While the warps' stages leave room
 * for the largest instance's charge grid in shared memory the kernel
 * deposits there; with more warps it deposits to global memory.  The
 * library's own choice is the most warps that leave that room, and 8.
 * Results do not depend on the shape, bit for bit: tiles are independent,
 * deposits are integer sums and births are ordered by (tile, slot). */
int slpic_set_launch_shape(slpic_ctx* ctx, int push_warps, int collide_ctas_per_sm);
int slpic_get_launch_shape(slpic_ctx* ctx, int* push_warps, int* collide_ctas_per_sm);
/* Autotuner: times candidate shapes on the context's own markers and keeps
 * the fastest per marker-step; writes it to the out arguments (may be
 * NULL).  It tries every warp count, then collision CTAs per SM of
 * 2, 4, 8 and 16, running steps_each steps of the simulation for each.
 * These are real steps: the state advances by (push candidates + 4) *
 * steps_each steps, exactly as slpic_step would have advanced it. */
int slpic_autotune(slpic_ctx* ctx, int64_t steps_each, int* push_warps,
                   int* collide_ctas_per_sm);

/* Per-step timing of the particle kernel: when on, slpic_step launches each
 * step without a CUDA graph and brackets every particle-kernel launch with
 * CUDA events on the context's stream. */
int slpic_set_profiling(slpic_ctx* ctx, int on);
/* Total device time [ms] and number of particle-kernel launches timed since
 * profiling was switched on (synchronises). */
int slpic_read_profile(slpic_ctx* ctx, double* push_ms, int64_t* launches);
/* Look-back statistics of the particle kernel since the last call: how many
 * times a tile found its predecessor's count not yet published, and the
 * longest such wait in polls (about 0.1 us each).  Synchronises; resets. */
int slpic_read_wait_stats(slpic_ctx* ctx, int64_t* waits, int64_t* longest);
/* Device-side kernel launches made by the last slpic_step call. */
int slpic_launch_count(slpic_ctx* ctx, int64_t* launches);

/* Philox4x32-10 evaluated by the device: out[4i..4i+3] = Philox(ctr[4i..],
 * key = seed).  Host arrays; for checking the random stream.  A step of
 * instance i draws, for marker id of species s, counter (id, step,
 * 2 i + s, block): block 0 = (unused, process, two angles) of a collision
 * candidate or (emission test, ...) of an ion at the cathode; block 1 =
 * (energy split, secondary's two angles); block 2 = born ion's Maxwellian;
 * seeding uses step = 0xFFFFFFFF. */
int slpic_philox(int device, uint64_t seed, const uint32_t* ctr, int64_t n,
                 uint32_t* out);

/* Philox2x32-10 evaluated by the device: out[2i..2i+1] = Philox(ctr[2i..],
 * key).  The null-collision draw of an electron in a step is word 0 of
 * Philox2x32-10 with counter (id, step) and key
 * lo32(seed) ^ hi32(seed) ^ (0x85EBCA6B * (instance + 1)) mod 2^32. */
int slpic_philox2x32(int device, uint32_t key, const uint32_t* ctr, int64_t n,
                     uint32_t* out);

/* Largest n that slpic_philox_static accepts: its device scratch holds this
 * many 16-byte counters and as many 16-byte outputs (1 MiB in all). */
#define SLPIC_PHILOX_STATIC_MAX 32768

/* slpic_philox without any device allocation.  A library utility; the method
 * has no counterpart.  Same arguments and results as slpic_philox, but the
 * counters and outputs are staged in one fixed device array that the library
 * owns (SLPIC_PHILOX_STATIC_MAX counters and as many outputs, 1 MiB, held on
 * every device that loads the library's device code until the process
 * exits), so the call makes no cudaMalloc or cudaFree.  It is for callers
 * that must not allocate device memory at the time of the call: a process
 * whose memory pool already holds all of the device, or one that checks the
 * random stream while a simulation runs on another stream of the same device
 * (the cudaFree in slpic_philox synchronises the whole device and would stall
 * that stream).
 *  - n > SLPIC_PHILOX_STATIC_MAX, n < 0 or a NULL array: SLPIC_ERR_INVALID_ARG
 *    before anything runs; the message is in slpic_last_error(NULL).  CUDA
 *    failures return SLPIC_ERR_CUDA with the message there too.
 *  - Set-up, once per device and context, with that device current: the
 *    array's address (cudaGetSymbolAddress), a private non-blocking stream,
 *    and the load of the library's device code that holds the array and the
 *    kernel.  CUDA loads device code lazily, and that first load reserves the
 *    1 MiB: slpic_create does the set-up for its device, and otherwise the
 *    first call on a device does it.  Create a context (or make one call) on
 *    each device before filling a memory pool or beginning a stream capture
 *    there.  After cudaDeviceReset the next call sets up again.
 *  - The copies and the kernel run on the private non-blocking stream: the
 *    call neither waits for nor delays work on other streams, and returns
 *    once out is written.  It makes `device` current for the calling thread.
 *  - Nothing in the scratch has to start at zero: each call copies its n
 *    counters in before the kernel reads them, and copies back only the n
 *    outputs the kernel has written.
 *  - There is one scratch array per device in a process: calls that overlap
 *    on one device (made from several host threads) race on it and return
 *    wrong words; serialise them. */
int slpic_philox_static(int device, uint64_t seed, const uint32_t* ctr, int64_t n,
                        uint32_t* out);

#ifdef __cplusplus
}
#endif

#endif /* SLPIC_H */
