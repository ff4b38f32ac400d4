/*
 * pic.h -- C ABI of the GB300 (sm_103a) 1d3v electrostatic PIC/MCC library.
 *
 * The library advances electrons and one positive ion species between two
 * parallel plates, the kinetic method of Becker, Kaehlert, Sun, Bonitz,
 * Loffhagen, arXiv:1608.04601, section "PIC/MCC simulation procedure":
 *   - superparticles of constant weight, one space coordinate and three
 *     velocity components (1d3v);
 *   - cloud-in-cell charge assignment and field interpolation;
 *   - Eq. (poisson) on N cells with phi(0,t) = V0 sin(2 pi f t), phi(d,t) = 0
 *     (section "Boundary conditions and initial values"), second-order
 *     central differences;
 *   - velocity Verlet push; collisions act on the synchronised velocity;
 *   - full absorption at both electrodes (optional secondary electrons);
 *   - null-collision Monte Carlo collisions with the processes of Table
 *     "reactions": electron elastic, excitation (1 or 2 levels), ionization
 *     (remaining energy shared equally); ion isotropic and backward elastic.
 *
 * Conventions for every entry point:
 *   - Return a pic_status; PIC_OK is 0. No C++ exception crosses the ABI.
 *     pic_last_error() gives a text for the last failure of a context.
 *   - Pointers named host_* or documented "host" are host memory owned by
 *     the caller, read or written before the call returns. The library owns
 *     all device memory it allocates; nothing is kept of caller pointers
 *     after a call returns.
 *   - Work is enqueued on the context's CUDA stream (the caller's, if given
 *     in pic_options.cuda_stream). Calls that return host data synchronise
 *     that stream first; pic_sync() synchronises and reports errors that the
 *     device raised (capacity overflow, bounded-wait timeout, non-finite state).
 *   - Species index 0 = electrons, 1 = ions. Discharge index counts from 0 in
 *     the order given to pic_batch_create.
 *   - Particle state is structure-of-arrays: int32 cell c in [0, N), in-cell
 *     offset f in [0, 1), velocities vx, vy, vz in m/s, with z = (c + f) d/N.
 *     The stored v_z is the Verlet half-step velocity v_n + (q/m) E_n dt/2.
 *     Real arrays are float (PIC_FP32) or double (PIC_FP64), per context.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx;

typedef enum {
    PIC_OK = 0,
    PIC_ERR_ARG = -1,        /* invalid argument (sizes, NULL, ranges)          */
    PIC_ERR_CUDA = -2,       /* a CUDA call failed                              */
    PIC_ERR_CAPACITY = -3,   /* a particle or birth buffer would overflow       */
    PIC_ERR_TIMEOUT = -4,    /* a bounded device-side wait gave up              */
    PIC_ERR_TABLE = -5,      /* cross-section table rejected (negative, NaN)    */
    PIC_ERR_NONFINITE = -6,  /* a non-finite particle coordinate was met        */
    PIC_ERR_STATE = -7       /* call not valid in the context's current state   */
} pic_status;

enum { PIC_ELECTRONS = 0, PIC_IONS = 1 };
enum { PIC_FP32 = 0, PIC_FP64 = 1 };
enum { PIC_MAX_DISCHARGES = 64, PIC_MAX_CELLS = 4096 };

/* Background gas with its cross sections (Table "reactions"), tabulated on
 * eps_k = k de_eV, k = 0..n_pts-1 (host arrays, copied at create time):
 *   sigma_e[k*(2+n_exc) + j] m^2, lab energy: j = 0 elastic, 1..n_exc
 *                                  excitation levels, 1+n_exc ionization;
 *   sigma_i[k*2 + j] m^2, centre-of-mass energy: j = 0 isotropic elastic,
 *                                  1 backward elastic (charge exchange).   */
typedef struct {
    double mass_kg;
    int32_t n_exc;           /* 1 or 2                                      */
    int32_t n_pts;           /* >= 2, <= 2^24                               */
    double de_eV;
    double eps_exc_eV[2];
    double eps_iz_eV;
    const double* sigma_e;
    const double* sigma_i;
} pic_gas;

/* Superparticle weights, initial population and store capacity. */
typedef struct {
    double w_e, w_i;         /* physical particles per superparticle per m^2 */
    int64_t n_e0, n_i0;      /* loaded at create (uniform, Maxwellian)       */
    int64_t capacity_e;      /* maximum superparticles held per species      */
    int64_t capacity_i;
    double T_e0_eV, T_i0_K;  /* temperatures of the initial Maxwellians      */
    double gamma_see;        /* secondary electrons per absorbed ion (0: off) */
    int32_t steps_per_period;/* rf period in steps (diagnostic bookkeeping)  */
    int32_t reserved;
} pic_weights;

/* One discharge of a batch. */
typedef struct {
    int32_t gas;             /* index into the gas array                    */
    int32_t n_cells;         /* N, 1..PIC_MAX_CELLS                         */
    double gap_m, p_Pa, T_gas_K, f_rf_Hz, V_rf_V, dt_s;
    pic_weights weights;
    uint32_t discharge_id;   /* fourth word of every random-stream counter  */
    int32_t reserved;
} pic_discharge;

typedef struct {
    int32_t precision;       /* PIC_FP32 (default) or PIC_FP64                */
    int32_t sort_every;      /* 0: never sort; K > 0: stable sort by cell    */
                             /* after every step n with (n+1) % K == 0       */
    int32_t block;           /* sweep threads per CTA: 128, 256 (default), 512 (PPT 2 or 4) */
    int32_t ppt;             /* sweep particles per thread: 2, 4 (default), 8 */
    int32_t ctas_per_sm;     /* persistent sweep CTAs per SM (0: occupancy)  */
    int32_t use_graph;       /* 1: replay pic_step in CUDA graphs of one rf  */
                             /* period (requires sort_every | steps/period)  */
    void* cuda_stream;       /* cudaStream_t to enqueue on; NULL = own stream */
    int32_t load;            /* 1 (default): load n_e0 / n_i0 at create      */
    int32_t leapfrog;        /* 0 (default): velocity Verlet, collisions at  */
                             /* v_n between the two half kicks (the paper's  */
                             /* scheme); 1: leapfrog variant, collisions at  */
                             /* v_{n+1/2} after both kicks, newborns drift   */
                             /* with their birth velocity                    */
} pic_options;

/* Fills *opt with the defaults documented above. */
void pic_default_options(pic_options* opt);

/* Creates a batch of independent discharges that advance together (one
 * sweep launch and one field launch per step for all of them). seed keys
 * every random stream (Philox4x32-10). opt may be NULL (defaults).
 * On PIC_OK, *out owns all device memory; release it with pic_destroy.   */
pic_status pic_batch_create(pic_ctx** out, const pic_gas* gases, int32_t n_gases,
                            const pic_discharge* discharges, int32_t n_discharges,
                            uint64_t seed, const pic_options* opt);

/* One discharge: gas and its tables, gap, pressure, gas temperature, rf
 * frequency and amplitude, cells, time step, weights, seed.              */
pic_status pic_create(pic_ctx** out, const pic_gas* gas, double gap_m, double p_Pa,
                      double T_gas_K, double f_rf_Hz, double V_rf_V, int32_t n_cells,
                      double dt_s, const pic_weights* weights, uint64_t seed,
                      const pic_options* opt);

/* Enqueues n_steps full time steps: sweep (gather, half kick, MCC, half
 * kick, drift, walls, compaction, deposit), births appended, periodic sort,
 * Poisson at t_{n+1}, moments accumulated. Asynchronous.
 * Order of a store after a sweep: the survivors in input-slot order, then
 * the newborns in parent-slot order (electrons: ionization electrons, then
 * secondary electrons of absorbed ions; ions: ionization ions). The slot
 * order keys every random stream, so the order is part of the result.    */
pic_status pic_step(pic_ctx* ctx, int64_t n_steps);

/* The parts of one step, for tests and custom drivers:
 *   pic_sweep  -- sweep of all discharges at the current step with the
 *                 current node field, births appended, counts updated;
 *   pic_sort   -- stable counting sort of every store by cell;
 *   pic_solve  -- charge density, Poisson at t_{n+1}, node field, moments
 *                 accumulated, step counter advanced.                     */
pic_status pic_sweep(pic_ctx* ctx);
pic_status pic_sort(pic_ctx* ctx);
pic_status pic_solve(pic_ctx* ctx);

/* Waits for the stream; returns the first device-raised error, if any.   */
pic_status pic_sync(pic_ctx* ctx);

/* Cycle-averaged moments of one discharge since the last reset (host
 * arrays of N+1 nodes, caller-owned, each may be NULL).                   */
typedef struct {
    double* n_e;             /* electron density, m^-3                       */
    double* n_i;             /* ion density, m^-3                            */
    double* mean_eps;        /* mean electron energy, eV                     */
    int64_t steps;           /* steps accumulated                            */
    int64_t count[2];        /* superparticles now, per species              */
    double absorbed[2][2];   /* superparticles absorbed [species][electrode] */
    double flux[2][2];       /* particle flux to [species][electrode], m^-2 s^-1 */
    double surface_charge;   /* eps0 E(0) at the last solve, C m^-2          */
    /* rf periods and the periodic steady state, computed by the library from the mean
     * superparticle count of each species per period (pic_period_counts): the state is
     * steady from the first period k (counted from 1) at which, for both species, the means
     * over the periods [k-W, k) and [k-2W, k-W) differ by less than PIC_STEADY_TOL relative
     * to the first, W = PIC_STEADY_BLOCK. The paper notes that its discharges needed about
     * 1000 to 4000 periods (section "Numerical parameters and initial values").           */
    int64_t periods_done;    /* complete rf periods since step 0                 */
    int64_t steady_period;   /* first period at which the test held, -1 if none  */
    double steady_metric;    /* the test's largest relative difference at the last
                                complete period (-1 before 2 W periods)         */
    int32_t steady;          /* 1 if steady_period >= 0                          */
    int32_t reserved;
    /* Discharge current density J(t) = eps0 dE(0,t)/dt + e0 (Gamma_i - Gamma_e)(0,t)
     * (section "Boundary conditions"), FP64 on the device every step: */
    double J_amp;            /* first-harmonic amplitude over the last complete
                                period, A m^-2 (0 before the first period)      */
    double J_last;           /* over the last step, A m^-2                       */
} pic_moments_t;
#define PIC_STEADY_BLOCK 50
#define PIC_STEADY_TOL 1e-3
pic_status pic_moments(pic_ctx* ctx, int32_t discharge, pic_moments_t* out);

/* J(t) of every step first .. first+n-1 into host out[2 k] (at z = 0, the paper's
 * definition) and out[2 k + 1] (the same expression at z = d; the two agree to rounding
 * when both species have equal weights, by conservation of charge). The current of step n
 * spans t_n .. t_{n+1}: eps0 times the change of the electrode field between the solves at
 * t_n and t_{n+1}, over dt, plus the charge of the superparticles absorbed (and secondary
 * electrons emitted) at that electrode during the sweep of step n, over dt. Zero for the
 * first step after a load. The last 4 rf periods (4096 steps if steps_per_period is 0) are
 * kept; *steps_done receives the steps completed.                                        */
pic_status pic_current(pic_ctx* ctx, int32_t discharge, int64_t first, int64_t n, double* out,
                       int64_t* steps_done);
/* First-harmonic amplitude of J(t) at z = 0 over rf periods first .. first+n-1: with
 * a = (2/P) sum_k J_k sin(w t_k), b = (2/P) sum_k J_k cos(w t_k) over the P steps of the
 * period at their midpoints t_k, the amplitude is sqrt(a^2 + b^2) (the J_calc of Eq.
 * adaptivevoltage). Requires a time step that divides the period (PIC_ERR_STATE). */
pic_status pic_current_amplitude(pic_ctx* ctx, int32_t discharge, int64_t first, int64_t n, double* out,
                                 int64_t* periods_done);
/* Current-driven mode (Eq. adaptivevoltage, section "Boundary conditions"): with J0 > 0 (A/m^2),
 * after every rf period of discharge d the amplitude of the applied voltage is multiplied by
 * J0 / J_calc, J_calc the period's first-harmonic amplitude of J(0,t) (pic_current_amplitude);
 * J0 = 0 keeps the amplitude in effect fixed. The paper adapts the voltage of its fluid models
 * this way; here it drives the particle model. Requires a time step that divides the rf period
 * (PIC_ERR_STATE). Synchronises the stream; takes effect from the next completed period.     */
pic_status pic_set_current_drive(pic_ctx* ctx, int32_t discharge, double J0);
/* Voltage amplitude V0 applied in rf periods first .. first+n-1 into host out[k] (the last
 * PERIOD_HIST periods are kept); *V0_now the amplitude in effect now (either may be NULL).   */
pic_status pic_voltage_amplitude(pic_ctx* ctx, int32_t discharge, int64_t first, int64_t n, double* out,
                                 int64_t* periods_done, double* V0_now);
pic_status pic_reset_moments(pic_ctx* ctx);

/* ---- kinetic diagnostics of the electrons (section "Results") -------------
 * Taken from the electron store at (x_n, v_n), before the sweep of step n of pic_step, on
 * the device (one or two extra launches at such a step, none at other steps):
 *   - rf-phase snapshots at every step n with period_steps > 0 and n % period_steps ==
 *     phase_step (the paper's profiles at t f = 0.25 take period_steps = steps_per_period,
 *     phase_step = steps_per_period / 4): the node field E and the cloud-in-cell node moments
 *     density n_e, mean energy, particle flux Gamma_e, energy flux Q_e, ionization rate S (each
 *     electron's sigma_iz v times n_gas), heating -e0 E Gamma_e and fast-electron density
 *     (energy above fast_eV; the paper takes e0 V0 / 4);
 *   - samples at every step n with sample_every > 0 and n % sample_every == 0: the energy
 *     histogram of eedf_bins bins of eedf_de_eV (the last bin also takes higher energies) and
 *     the fast-electron density.
 * Per electron: the gathered field and the first half kick as in the sweep, its energy in
 * 2^-12 eV (clamped at 2^26), and per node moment an integer (rounded in the particle
 * precision) split between the two nodes of its cell like the charge; density 2^32 per
 * particle, energy 2^-12 eV, v_z 2^-6 m/s, energy x v_z 2^-4 eV m/s, sigma_iz v 2^-72 m^3/s.
 * The sums are exact, hence independent of the order of the particles.
 * With graphs (pic_options.use_graph), rf periods run as graphs only while both schedules
 * repeat every rf period (period_steps and sample_every divide steps_per_period, or are 0);
 * otherwise steps are launched one by one.                                                 */
typedef struct {
    int32_t period_steps;   /* 0: no snapshots                                            */
    int32_t phase_step;     /* 0 .. period_steps - 1                                      */
    int32_t sample_every;   /* 0: no samples                                              */
    int32_t eedf_bins;      /* 1 .. PIC_DIAG_MAX_BINS                                     */
    double eedf_de_eV;      /* bin width, > 0                                             */
    double fast_eV;         /* fast-electron threshold, >= 0                              */
} pic_diag_config;
#define PIC_DIAG_MAX_BINS 16384
/* Configures (cfg) or switches off (cfg NULL) the diagnostics of every discharge; clears the
 * accumulators. Allocates device memory (and so synchronises the context's stream); not
 * allowed while the stream is being captured. PIC_ERR_ARG for a configuration out of range. */
pic_status pic_set_diagnostics(pic_ctx* ctx, const pic_diag_config* cfg);
/* Clears the accumulators (stream-ordered). PIC_ERR_STATE if not configured.             */
pic_status pic_reset_diagnostics(pic_ctx* ctx);
/* Read-out of one discharge (host arrays, each may be NULL): E [V/m], n_e [m^-3], mean_eps
 * [eV], gamma_e [m^-2 s^-1], q_e [W m^-2], heating [W m^-3], ion_rate [m^-3 s^-1], n_fast
 * [m^-3] averaged over the snapshots, n_fast_avg [m^-3] over the samples (N+1 nodes each; the
 * wall nodes own half a cell); eedf [eedf_bins]: f0(U)/n_e at the bin centres U [eV^-3/2],
 * normalised so that sum_b eedf_b sqrt(U_b) eedf_de_eV = 1; snapshots and samples taken.
 * Synchronises the stream. PIC_ERR_STATE if not configured.                                 */
pic_status pic_diagnostics(pic_ctx* ctx, int32_t discharge, double* E, double* n_e, double* mean_eps,
                           double* gamma_e, double* q_e, double* heating, double* ion_rate, double* n_fast,
                           double* n_fast_avg, double* eedf, int64_t* snapshots, int64_t* samples);

void        pic_destroy(pic_ctx* ctx);         /* NULL-safe                 */
const char* pic_last_error(const pic_ctx* ctx);
const char* pic_status_string(pic_status s);

/* ---- state access (host buffers; synchronous) --------------------------- */
pic_status pic_get_count(pic_ctx* ctx, int32_t d, int32_t species, int64_t* n);
/* Copies the store of (d, species) into host arrays of at least `cap`
 * entries (any of them may be null: not copied); *n receives the count.
 * Real arrays per the context precision. A count above cap returns
 * PIC_ERR_ARG with the arrays untouched. pic_set_state replaces the store by
 * n particles (cells c in [0, N), else PIC_ERR_ARG and an empty store; above
 * the store's capacity PIC_ERR_CAPACITY). Both synchronise the context's
 * stream before they return. Host arrays in pinned, mapped memory
 * (cudaHostAlloc, cudaHostRegister, a pinned torch tensor) are read or
 * written by the device directly over the host link, fastest when each
 * starts on a 16-byte boundary; pageable arrays go through device staging
 * and copies. Both ways give the same store, bit for bit.               */
pic_status pic_get_state(pic_ctx* ctx, int32_t d, int32_t species, int64_t cap, int32_t* c,
                         void* f, void* vx, void* vy, void* vz, int64_t* n);
pic_status pic_set_state(pic_ctx* ctx, int32_t d, int32_t species, int64_t n, const int32_t* c,
                         const void* f, const void* vx, const void* vy, const void* vz);
/* Node field used by the gather (N+1 reals); FP64 potential and field.   */
pic_status pic_get_field(pic_ctx* ctx, int32_t d, void* E, double* E64, double* phi);
pic_status pic_set_field(pic_ctx* ctx, int32_t d, const void* E);
/* 64-bit fixed-point CIC deposits of the last sweep (2^32 per particle). */
pic_status pic_get_deposit(pic_ctx* ctx, int32_t d, int32_t species, int64_t* D);
pic_status pic_set_deposit(pic_ctx* ctx, int32_t d, int32_t species, const int64_t* D);
/* Electron energy moment of the last sweep at (x_n, v_n), 2^-12 eV units
 * (per-particle energies clamped at 16384 eV). */
pic_status pic_get_energy_deposit(pic_ctx* ctx, int32_t d, int64_t* Q);
pic_status pic_get_step(pic_ctx* ctx, int64_t* step);
pic_status pic_set_step(pic_ctx* ctx, int64_t step);

/* Event counters since creation. */
typedef struct {
    int64_t absorbed[2][2];
    int64_t collisions_e[4]; /* elastic, excitation 1, excitation 2, ionization */
    int64_t collisions_i[2]; /* isotropic, backward                          */
    int64_t null_inelastic;  /* inelastic process selected below threshold   */
    int64_t see_emitted;
    int64_t candidates[2];
    int64_t table_clamped[2];
} pic_counters;
pic_status pic_get_counters(pic_ctx* ctx, int32_t d, pic_counters* out);

/* Derived per-discharge constants (host FP64 values before rounding). */
typedef struct {
    double dx, n_gas, kmax_e, kmax_i, numax_e, numax_i, pnull_e, pnull_i;
    uint32_t thr_e, thr_i;
    double K_e, K_i, dtdx, kappa_e, kappa_i, kappa_E, beta_e, omb_e;
    double de2_exc[2], de2_iz, sig_n, sig_e0, sig_i0, sig_see, sig_see_n;
} pic_derived;
pic_status pic_get_derived(pic_ctx* ctx, int32_t d, pic_derived* out);
/* Cumulative rate-coefficient tables of one gas: Te n_pts x 4, Ti n_pts x 2. */
pic_status pic_get_tables(pic_ctx* ctx, int32_t gas, void* Te, void* Ti);

/* Warm start: replaces every store by superparticles sampled from given
 * cycle-averaged profiles, instead of the uniform cold load. profiles is a host
 * array [n_discharges][3][n_pts] on the uniform grid z_j = j gap / (n_pts-1):
 * electron density, ion density (m^-3), mean electron energy (eV). Counts are
 * the profile integrals over the weights; positions follow the inverse of the
 * piecewise-constant CDF; electrons are Maxwellian at kT = 2/3 <eps>(z), ions at
 * T_i0 (Philox calls 0xF2, 0xF3 at step 0). Then, as after the cold load:
 * deposit, field at t = 0, half back-kick. Only before the first step
 * (PIC_ERR_STATE otherwise); PIC_ERR_CAPACITY if a count exceeds capacity.
 * The paper notes that initial values change the time to the periodic state,
 * not the state (section "Numerical parameters and initial values").        */
pic_status pic_load_profiles(pic_ctx* ctx, int32_t n_pts, const double* profiles);

/* Mean superparticle count of each species over rf periods first .. first+n-1
 * (periods counted from step 0; a period ends after steps_per_period steps),
 * into host out[2*k + species]. *periods_done receives the periods completed.
 * The last 65536 periods are kept. The steady-state criterion of the warm start
 * compares these means 50 periods apart.                                    */
pic_status pic_period_counts(pic_ctx* ctx, int32_t d, int64_t first, int64_t n, double* out,
                             int64_t* periods_done);

/* Timing of the last pic_step call's sweep launches (CUDA events on the
 * context stream): total milliseconds and launches.                       */
pic_status pic_sweep_timing(pic_ctx* ctx, int32_t enable, double* total_ms, int64_t* launches);

/* ---- self-checks of the device building blocks (host buffers) ---------- */
/* Philox4x32-10 (Salmon et al., SC'11) on n counters (4 words each).      */
/* The bounded device-side wait of the sweep's bulk-copy staging, on its own: one mbarrier that
 * expects one arrival, polled at most `tries` times (1 .. 2^20). arrive = 0: nothing arrives, the
 * wait gives up and the call returns PIC_ERR_TIMEOUT with the device context intact (nothing is
 * left in flight); arrive = 1: PIC_OK. Synchronous, default stream.                        */
pic_status pic_debug_wait(int32_t arrive, int32_t tries);
pic_status pic_debug_philox(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out);
/* Own log, sin(pi y), cos(pi y), Box-Muller and isotropic direction as used
 * by the kernels, on n inputs.                                            */
pic_status pic_debug_math(int64_t n, const float* x, const float* y, float* log_out,
                          float* sin_out, float* cos_out);

/* ---- allocation-free entry point ----------------------------------------
 * The paper has no counterpart to this entry point. It serves callers that
 * cannot allocate device memory while they run -- code with its own memory
 * arena that forbids cudaMalloc/cudaFree (they synchronise the device and can
 * fail late), plug-ins that are handed only device pointers, services that
 * must not grow their footprint. pic_sort_noalloc stably sorts one particle
 * store by cell index (the same order as pic_sort):
 *   c_in, rec_in   device arrays of n cells and n records {f, vx, vy, vz}
 *                  (float4, or four doubles for PIC_FP64), caller-owned;
 *   c_out, rec_out device arrays of n entries, caller-owned, not overlapping
 *                  the inputs; cells must lie in [0, n_cells);
 *   cuda_stream    stream to enqueue on (NULL: the legacy default stream).
 * Alignment: rec_in and rec_out must be 16-byte aligned (PIC_FP32) or 32-byte
 * aligned (PIC_FP64), c_in and c_out 4-byte aligned; otherwise PIC_ERR_ARG
 * and nothing is launched. A cell outside [0, n_cells) is not placed: the
 * call still returns PIC_OK, and the last entries of c_out and rec_out (one
 * per such cell) keep whatever they held before (the context sort,
 * pic_sort, reports such cells through pic_sync instead).
 * Its scratch is a fixed array of PIC_NOALLOC_SCRATCH_BYTES compiled into the
 * library (every GPU that loads the library holds it until the process
 * exits); the call allocates nothing. Limit: n_cells * (1 + ceil(n / 4096))
 * <= PIC_NOALLOC_SCRATCH_BYTES / 4, else PIC_ERR_CAPACITY (e.g. 512 cells:
 * up to 8.38e6 particles; 2048 cells: up to 2.09e6). The first call on a
 * device looks up the array's device address; make that first call before
 * any stream capture. All calls share the one array and each call rewrites
 * all of it that it reads, so consecutive calls are independent, but calls
 * that overlap on the GPU (other streams or threads) race: serialise them.
 * Returns PIC_ERR_ARG for invalid arguments, PIC_ERR_CUDA if a launch fails
 * or if an earlier CUDA error is pending on the calling thread (it is left
 * pending for the caller, and nothing is launched); asynchronous otherwise. */
#define PIC_NOALLOC_SCRATCH_BYTES (4u << 20)
pic_status pic_sort_noalloc(const int32_t* c_in, const void* rec_in, int32_t* c_out, void* rec_out,
                            int64_t n, int32_t n_cells, int32_t precision, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
