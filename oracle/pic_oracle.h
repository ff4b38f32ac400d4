/*
 * pic_oracle.h -- plain CPU oracle of the 1d3v electrostatic PIC/MCC time step
 * of Becker, Kaehlert, Sun, Bonitz, Loffhagen (arXiv:1608.04601), section
 * "PIC/MCC simulation procedure" (superparticles of constant weight, cloud-in-
 * cell charge assignment, Poisson equation Eq. (poisson) with the rf Dirichlet
 * boundary of section "Boundary conditions", velocity Verlet, full absorption
 * at both electrodes, null-collision Monte Carlo collisions with the reactions
 * of Table "reactions").
 *
 * TEST INFRASTRUCTURE. This oracle exists to check the CUDA library. Only the
 * test suite, the smoke check and the benchmark's CPU-baseline / reference arm
 * may load it. The CUDA library never includes, links or calls it, and it
 * includes nothing of the library.
 *
 * The same source is compiled twice:
 *   liboracle_f64.so  (ORC_F32 undefined): every per-particle value in double.
 *   liboracle_f32.so  (-DORC_F32):         every per-particle value in float,
 *       op by op as written in pic_oracle.c, so that each floating-point value
 *       that decides an integer (candidate, process, new cell, fixed-point
 *       deposit) is taken in the precision of the FP32 kernel.
 * Field solve, densities and diagnostics are FP64 in both builds.
 * Parity status of every function is listed in pic_oracle.c's header.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Background gas and its cross sections (Table "reactions"). Cross sections
 * are tabulated on the uniform energy grid eps_k = k*de_eV, k = 0..n_pts-1.
 *   sigma_e[k*(2+n_exc) + j], m^2: j = 0 elastic, 1..n_exc excitation levels,
 *                                  1+n_exc ionization; lab-frame energy.
 *   sigma_i[k*2 + j],         m^2: j = 0 isotropic, 1 backward elastic;
 *                                  centre-of-mass energy.                    */
typedef struct {
    double mass_kg;          /* neutral (and ion) mass                       */
    int32_t n_exc;           /* 1 or 2 excitation levels                     */
    int32_t n_pts;           /* energy grid points (>= 2)                    */
    double de_eV;            /* grid spacing                                 */
    double eps_exc_eV[2];    /* excitation thresholds                        */
    double eps_iz_eV;        /* ionization threshold                         */
    const double* sigma_e;
    const double* sigma_i;
} orc_gas;

typedef struct {
    double gap_m, p_Pa, T_gas_K, f_rf_Hz, V_rf_V, dt_s;
    double w_e, w_i;         /* superparticle weights, m^-2                  */
    double T_e0_eV, T_i0_K;  /* temperatures of the initial Maxwellians      */
    double gamma_see;        /* electrons emitted per absorbed ion           */
    int64_t n_e0, n_i0;      /* initial superparticles per species           */
    uint64_t seed;
    int32_t n_cells;
    int32_t sort_every;      /* 0: never; K: after every step n with (n+1)%K==0 */
    uint32_t discharge_id;   /* fourth Philox counter word                   */
    int32_t pad_;
} orc_params;

/* Per-step event counters (cumulative since creation). */
typedef struct {
    int64_t absorbed[2][2];  /* [species][electrode 0 at z=0, 1 at z=d]      */
    int64_t collisions_e[4]; /* elastic, exc1, exc2, ionization              */
    int64_t collisions_i[2]; /* isotropic, backward                          */
    int64_t null_inelastic;  /* selected inelastic below threshold           */
    int64_t see_emitted;
    int64_t candidates[2];
    int64_t table_clamped[2];
} orc_counters;

typedef struct orc_ctx orc_ctx;

orc_ctx* orc_create(const orc_gas* gas, const orc_params* p);
void     orc_destroy(orc_ctx* o);
int      orc_real_bytes(void);               /* 4 or 8                       */

/* Initial loading (uniform positions, Maxwellian velocities), initial
 * deposit, field solve at t = 0 and the half back-kick of v_z.            */
int      orc_load(orc_ctx* o);

/* Warm start: replaces both stores by particles sampled from profiles on a
 * uniform grid of n_pts points over [0, d]: n_e, n_i (m^-3), mean electron
 * energy (eV). Counts = integral / weight; positions by the inverse of the
 * piecewise-constant CDF; velocities Maxwellian, electrons at kT = 2/3 <eps>(z),
 * ions at T_i0. Then deposit, field at t = 0 and the half back-kick.        */
int      orc_load_profiles(orc_ctx* o, int n_pts, const double* n_e, const double* n_i,
                           const double* mean_eps);

/* The parts of one time step, and the whole step. */
int      orc_sweep(orc_ctx* o);     /* gather, Verlet, MCC, walls, compaction, deposit */
int      orc_sort(orc_ctx* o);      /* stable counting sort of both species by cell   */
int      orc_solve(orc_ctx* o);     /* Poisson at t_{n+1}, node field, advance n      */
int      orc_step(orc_ctx* o, int64_t n_steps);

/* State access. Arrays are SoA; velocities in m/s; f in [0,1). */
int64_t  orc_count(const orc_ctx* o, int species);
int      orc_get_state(const orc_ctx* o, int species, int32_t* c, void* f,
                       void* vx, void* vy, void* vz);
int      orc_set_state(orc_ctx* o, int species, int64_t n, const int32_t* c,
                       const void* f, const void* vx, const void* vy, const void* vz);
int      orc_get_field(const orc_ctx* o, void* E);          /* N+1 reals, V/m  */
int      orc_set_field(orc_ctx* o, const void* E);
int      orc_get_phi(const orc_ctx* o, double* phi);        /* N+1, V, FP64    */
int      orc_get_efield64(const orc_ctx* o, double* E);     /* N+1, FP64       */
int      orc_get_deposit(const orc_ctx* o, int species, int64_t* D);   /* N+1 */
int      orc_set_deposit(orc_ctx* o, int species, const int64_t* D);
int      orc_get_energy_deposit(const orc_ctx* o, int64_t* Q);         /* N+1, 2^-12 eV */
int64_t  orc_get_step(const orc_ctx* o);
void     orc_set_step(orc_ctx* o, int64_t n);
void     orc_get_counters(const orc_ctx* o, orc_counters* out);

/* Derived per-discharge constants, for bitwise comparison with the library. */
typedef struct {
    double dx, n_gas, kmax_e, kmax_i, numax_e, numax_i, pnull_e, pnull_i;
    uint32_t thr_e, thr_i;
    double K_e, K_i, dtdx, kappa_e, kappa_i, kappa_E, beta_e, omb_e;
    double de2_exc[2], de2_iz, sig_n, sig_e0, sig_i0, sig_see, sig_see_n;
} orc_derived;
void     orc_get_derived(const orc_ctx* o, orc_derived* out);
int      orc_get_tables(const orc_ctx* o, void* Te /* n_pts*4 */, void* Ti /* n_pts*2 */);

/* Cycle-averaged diagnostics since the last reset. */
typedef struct {
    int64_t steps;
    double  absorbed[2][2];  /* superparticles, summed over the steps        */
} orc_moment_info;
int      orc_moments(const orc_ctx* o, double* n_e, double* n_i, double* mean_eps,
                     orc_moment_info* info);
void     orc_reset_moments(orc_ctx* o);

/* Discharge current density (section "Boundary conditions", equation for J(t)) over the step of
 * the last solve, J = eps0 dE/dt + e0 (Gamma_i - Gamma_e), in A m^-2: J[0] at z = 0 (the
 * powered electrode, the paper's definition), J[1] the same expression at z = d. Both are zero
 * after the first solve of a run (no previous field).                                         */
void     orc_last_current(const orc_ctx* o, double J[2]);
/* Per rf period of period_steps steps (counted from step 0; 0: off): the first-harmonic amplitude
 * J_calc of J(0,t) at the step midpoints, and with J_target > 0 the current-driven mode of Eq.
 * (adaptivevoltage): after every period V0 <- V0 J_target / J_calc (section "Boundary
 * conditions"; the paper applies it to its fluid models, here it drives the particle model).  */
int      orc_set_current_drive(orc_ctx* o, int period_steps, double J_target);
/* Push scheme (section "PIC/MCC simulation procedure": the method uses velocity Verlet and notes
 * that it converges faster in dt than leapfrog). 0 (default): velocity Verlet, the collision acts
 * on v_n between the two half kicks; 1: leapfrog variant, both half kicks first (v_{n+1/2} =
 * v_{n-1/2} + a_n dt, the same two operations) and the collision acts on v_{n+1/2}, newborns
 * drift with their birth velocity. Diagnostics at v_n in both.                                */
int      orc_set_scheme(orc_ctx* o, int leapfrog);
/* Completed periods; their amplitudes J_calc and applied V0 (up to cap of each), V0 in effect. */
int64_t  orc_period_history(const orc_ctx* o, double* amp, double* V0, int64_t cap, double* V_now);

/* Kinetic diagnostics of the electrons (section "Results": the EEDF figure, the fast-electron
 * density and the profiles at t f = 0.25), taken at (x_n, v_n) before the sweep of step n:
 *   - phase-resolved: at every step n with n % period_steps == phase_step, the node field E and
 *     the cloud-in-cell moments density, mean energy, particle flux Gamma_e, energy flux Q_e,
 *     ionization rate S (the rate coefficient sigma_iz v of each electron times n_gas), fast
 *     electrons (energy above fast_eV), accumulated over such steps;
 *   - sampled every sample_every steps: the energy histogram (eedf_bins bins of eedf_de_eV, the
 *     last bin also takes higher energies) and the fast-electron density.
 * Every per-particle value is formed in the particle precision and rounded to an integer, so the
 * accumulators are exact sums. The read-out gives physical units (see orc_diagnostics).       */
typedef struct {
    int32_t period_steps, phase_step, sample_every, eedf_bins;
    double eedf_de_eV, fast_eV;
} orc_diag_config;
int  orc_set_diagnostics(orc_ctx* o, const orc_diag_config* cfg);   /* resets the accumulators */
void orc_reset_diagnostics(orc_ctx* o);
/* Read-out (each array may be NULL): E [V/m], n_e [m^-3], mean_eps [eV], gamma_e [m^-2 s^-1],
 * q_e [W m^-2], heating = -e0 E Gamma_e [W m^-3], ion_rate [m^-3 s^-1], n_fast [m^-3] averaged
 * over the phase snapshots (N+1 nodes each); n_fast_avg [m^-3] over the samples; eedf
 * [eedf_bins] f0(U)/n_e at the bin centres [eV^-3/2]; snapshots and samples counted.          */
int  orc_diagnostics(const orc_ctx* o, double* E, double* n_e, double* mean_eps, double* gamma_e, double* q_e,
                     double* heating, double* ion_rate, double* n_fast, double* n_fast_avg, double* eedf,
                     int64_t* snapshots, int64_t* samples);

/* Building blocks, exported for the pins. */
void     orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
float    orc_uniform(uint32_t x);
float    orc_logf(float x);
void     orc_sincospif(float y, float* s, float* c);
void     orc_box_muller(float ua, float ub, float* n0, float* n1);
void     orc_isotropic(float ua, float ub, float* nx, float* ny, float* nz);
/* Dirichlet Poisson solve by the Thomas algorithm: rho[0..N] in C/m^3,
 * phi[0..N] out, E[0..N] out (node field, see orc_solve).                  */
void     orc_poisson(int N, double dx, double V0, double VN, const double* rho,
                     double* phi, double* E);

#ifdef __cplusplus
}
#endif
#endif
