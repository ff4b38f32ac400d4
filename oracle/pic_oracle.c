/*
 * pic_oracle.c -- plain, slow CPU oracle of the 1d3v electrostatic PIC/MCC
 * time step of arXiv:1608.04601 (Becker et al.), section "PIC/MCC simulation
 * procedure". TEST INFRASTRUCTURE ONLY (see pic_oracle.h): the CUDA library
 * never links, includes or calls this file, and this file uses nothing of it.
 *
 * What each part follows, and how it is pinned (tests/test_oracle_*.py):
 *   philox4x32_10   Salmon et al., SC'11, "Parallel random numbers: as easy as
 *                   1, 2, 3" (Philox-4x32, 10 rounds). Pinned by the published
 *                   known-answer vectors (tests/golden/philox4x32_10_kat.txt).
 *   orc_logf,       own elementary functions so that the CUDA path can take
 *   orc_sincospif   the same values bit for bit: log by exponent split and the
 *                   atanh series ln m = 2(t + t^3/3 + t^5/5 + t^7/7 + t^9/9),
 *                   t = (m-1)/(m+1); sin/cos(pi r) by quadrant reduction and
 *                   their Taylor series on |r| <= 1/4. Pinned against libm to
 *                   a few ulp.
 *   load            uniform positions, Maxwellian velocities (Table
 *                   "numericalparameters": homogeneous quasi-neutral start).
 *                   Pinned by moments and a KS test.
 *   field solve     Eq. (poisson) with phi(0,t) = V0 sin(2 pi f t), phi(d,t) = 0
 *                   (section "Boundary conditions"), second-order central
 *                   differences (section "Numerical solution of fluid
 *                   models"), Thomas algorithm. Pinned by the closed form for
 *                   uniform charge (exact for quadratics) and a dense solve.
 *   gather/deposit  cloud-in-cell, linear weights (section "PIC/MCC ..."),
 *                   64-bit fixed point. Pinned by exact charge conservation
 *                   and the node/half-node special cases.
 *   push            velocity Verlet (section "PIC/MCC ..."), collisions on the
 *                   synchronised velocity v_n. Pinned by field-free energy
 *                   conservation and the exact constant-field parabola.
 *   MCC             null-collision method; isotropic scattering except the
 *                   backward ion-neutral elastic process; ionization shares
 *                   the remaining energy equally (section "PIC/MCC ...",
 *                   Table "reactions"). Pinned by brute-force collision
 *                   probabilities, exponential free flight (KS), energy and
 *                   momentum bookkeeping, isotropy.
 *   walls           full absorption at z = 0 and z = d. Pinned by the
 *                   one-sided Maxwellian flux n v_th / 4 (Eq. BCparticles).
 *   moments         cycle averages (section "Results"). Pinned by the
 *                   uniform static load.
 * Secondary electron emission is not in the paper (it assumes none); it is
 * an added option. Pinned by its emitted count (binomial in the absorbed
 * ions) and the emitted velocities (the flux of a Maxwellian at 2 eV:
 * Rayleigh normal speed, normal tangential components, independent, mean
 * energy 2 T).
 *
 * Every per-particle value is of type real (float or double, see the
 * header); values drawn from the random streams (directions, normals) are
 * always formed in float by the own functions below and then widened.
 * Build with -ffp-contract=off: only the explicit FMAs below are fused.
 */
#include "pic_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORC_F32
typedef float real;
#define R_FMA(a, b, c) fmaf((a), (b), (c))
#define R_SQRT(x) sqrtf(x)
#define R_FLOOR(x) floorf(x)
#define R_RINT(x) llrintf(x)
#define R_ONE_MINUS_ULP 0x1.fffffep-1f
#else
typedef double real;
#define R_FMA(a, b, c) fma((a), (b), (c))
#define R_SQRT(x) sqrt(x)
#define R_FLOOR(x) floor(x)
#define R_RINT(x) llrint(x)
#define R_ONE_MINUS_ULP 0x1.fffffffffffffp-1
#endif

/* CODATA 2018 values. */
#define E_CHARGE 1.602176634e-19
#define M_ELEC 9.1093837015e-31
#define EPS0 8.8541878128e-12
#define K_BOLTZ 1.380649e-23
#define PI_D 3.14159265358979323846
#define T_SEE_EV 2.0          /* temperature of emitted secondary electrons */
#define TWO32 4294967296.0

enum { SP_E = 0, SP_I = 1 };
enum { CALL_MAIN = 0, CALL_AUX = 1, CALL_AUX2 = 2, CALL_SEE = 3, CALL_CAND = 4,
       CALL_LOAD0 = 0xF0, CALL_LOAD1 = 0xF1, CALL_WARM0 = 0xF2, CALL_WARM1 = 0xF3 };

typedef struct {
    int32_t* c;
    real *f, *vx, *vy, *vz;
    int64_t n, cap;
} store;

struct orc_ctx {
    orc_params p;
    orc_gas gas;
    int N, n_pts, n_proc_e;
    orc_derived d;
    /* real-typed copies of the derived constants used per particle */
    real K_e, K_i, dtdx, kappa_e, kappa_i, kappa_E, beta_e, omb_e, de2_exc[2], de2_iz;
    real sig_n, sig_e0, sig_i0, sig_see, sig_see_n, kmax_e, kmax_i, gamma;
    real* Te;    /* n_pts x 4, cumulative rate coefficient sigma*v, m^3/s     */
    real* Ti;    /* n_pts x 2                                                  */
    store s[2];
    real* E;     /* node field used by the gather                              */
    double *E64, *phi, *rho;
    int64_t *D[2], *Dprev_e, *Q;
    int64_t step;
    orc_counters cnt;
    /* moment accumulators */
    double *acc_D[2], *acc_Q, *acc_Dprev;
    int64_t acc_steps;
    orc_counters cnt_at_reset;
    /* discharge current density (Eq. for J(t), section "Boundary conditions"): electrode fields and
     * particle counts at the last solve, secondary electrons emitted per electrode, and the last
     * step's J at z = 0 and at z = d */
    int have_solve;
    double E_wall_prev[2];
    int64_t abs_prev[2][2], see_side[2], see_prev[2];
    double J_last[2];
    /* current-driven mode (Eq. adaptivevoltage): amplitude in effect, target (0: fixed voltage),
     * first-harmonic projections of J(0,t) over the current rf period, per-period history       */
    double V_amp, J_target, proj_a, proj_b;
    int leapfrog;  /* 1: collisions at v_{n+1/2} (leapfrog variant); 0: at v_n (velocity Verlet) */
    int period_steps;
    double *amp_hist, *V_hist;
    int64_t hist_n, hist_cap;
    /* kinetic diagnostics */
    orc_diag_config dg;
    int dg_on;
    int64_t *dg_D, *dg_U, *dg_V, *dg_W, *dg_K, *dg_F, *dg_Fa, *dg_eedf;
    double* dg_E;
    int64_t dg_snap, dg_samples;
};

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). The round multiplies
 * counter words 0 and 2 by two fixed odd constants, keeps the 32-bit halves,
 * and mixes the high halves with the other counter words and the round key;
 * the key is bumped by two Weyl constants between rounds.                   */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout: (slot, step low word, step bits 32..47 << 16 | species << 8
 * | call, discharge id); key = the 64-bit seed.                            */
static void draw(const orc_ctx* o, uint32_t slot, int species, int call, uint32_t r[4]) {
    uint64_t n = (uint64_t)o->step;
    uint32_t ctr[4] = {slot, (uint32_t)n,
                       ((uint32_t)((n >> 32) & 0xFFFFu) << 16) | ((uint32_t)species << 8) | (uint32_t)call,
                       o->p.discharge_id};
    uint32_t key[2] = {(uint32_t)o->p.seed, (uint32_t)(o->p.seed >> 32)};
    orc_philox4x32_10(ctr, key, r);
}

/* Candidate word of a slot: slots 4q..4q+3 share one Philox call (call 4,
 * first counter word q) and take its words 0..3 in order.                   */
static uint32_t candidate_word(const orc_ctx* o, uint32_t slot, int species) {
    uint32_t r[4];
    draw(o, slot >> 2, species, CALL_CAND, r);
    return r[slot & 3];
}

/* u = (top 23 bits + 1/2) * 2^-23, in [2^-24, 1 - 2^-24], exact in float
 * (24 significant bits) and hence in double.                               */
float orc_uniform(uint32_t x) { return ((float)(x >> 9) + 0.5f) * 0x1p-23f; }
#define U24 orc_uniform

/* Natural log of a positive normal float: x = m 2^e with m in [sqrt(1/2),
 * sqrt(2)); ln m = 2 atanh(t), t = (m-1)/(m+1), |t| <= 0.1716, by its Taylor
 * series to t^9 (truncation < 1e-9 relative).                             */
float orc_logf(float x) {
    uint32_t b;
    memcpy(&b, &x, 4);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    uint32_t mb = (b & 0x007FFFFFu) | 0x3F800000u;
    float m;
    memcpy(&m, &mb, 4);
    if (m > 0x1.6a09e6p+0f) {
        m = m * 0.5f;
        e = e + 1;
    }
    float t = (m - 1.0f) / (m + 1.0f);
    float t2 = t * t;
    float p = fmaf(t2, 0x1.c71c72p-4f, 0x1.24924ap-3f); /* 1/9, 1/7 */
    p = fmaf(t2, p, 0x1.99999ap-3f);                     /* 1/5 */
    p = fmaf(t2, p, 0x1.555556p-2f);                     /* 1/3 */
    float t2x = 2.0f * t;
    float lm = fmaf(t2x, t2 * p, t2x);
    float ef = (float)e;
    return fmaf(ef, 0x1.62e430p-1f, fmaf(ef, -0x1.05c610p-29f, lm)); /* ln 2 = hi + lo */
}

/* sin(pi y), cos(pi y) for y in [0, 2]: y = r + q/2 with q = rint(2y),
 * |r| <= 1/4 (exact), then the Taylor series of sin(pi r) to r^9 and of
 * cos(pi r) to r^10, and the quadrant q mod 4.                             */
void orc_sincospif(float y, float* s, float* c) {
    float q = rintf(2.0f * y);
    float r = fmaf(q, -0.5f, y);
    int iq = ((int)q) & 3;
    float r2 = r * r;
    float ps = fmaf(r2, 0x1.507834p-4f, -0x1.32d2ccp-1f); /* pi^9/9!, -pi^7/7! */
    ps = fmaf(r2, ps, 0x1.466bc6p+1f);                     /* pi^5/5! */
    ps = fmaf(r2, ps, -0x1.4abbcep+2f);                    /* -pi^3/3! */
    ps = fmaf(r2, ps, 0x1.921fb6p+1f);                     /* pi */
    float sn = r * ps;
    float pc = fmaf(r2, -0x1.a6d1f2p-6f, 0x1.e1f506p-3f); /* -pi^10/10!, pi^8/8! */
    pc = fmaf(r2, pc, -0x1.55d3c8p+0f);                    /* -pi^6/6! */
    pc = fmaf(r2, pc, 0x1.03c1f0p+2f);                     /* pi^4/4! */
    pc = fmaf(r2, pc, -0x1.3bd3ccp+2f);                    /* -pi^2/2! */
    float cs = fmaf(r2, pc, 1.0f);
    switch (iq) {
        case 0: *s = sn; *c = cs; break;
        case 1: *s = cs; *c = -sn; break;
        case 2: *s = -sn; *c = -cs; break;
        default: *s = -cs; *c = sn; break;
    }
}

/* Box-Muller: two independent standard normals from two uniforms. */
void orc_box_muller(float ua, float ub, float* n0, float* n1) {
    float rr = sqrtf(-2.0f * orc_logf(ua));
    float s, c;
    orc_sincospif(2.0f * ub, &s, &c);
    *n0 = rr * c;
    *n1 = rr * s;
}

/* Uniform direction on the unit sphere: cos(theta) = 1 - 2 ua, azimuth
 * 2 pi ub, z the polar axis.                                                */
void orc_isotropic(float ua, float ub, float* nx, float* ny, float* nz) {
    float ct = 1.0f - 2.0f * ua;
    float st = sqrtf(fmaxf(0.0f, fmaf(-ct, ct, 1.0f)));
    float s, c;
    orc_sincospif(2.0f * ub, &s, &c);
    *nx = st * c;
    *ny = st * s;
    *nz = ct;
}

/* The scattering direction in the particle precision: cos(theta) = 1 - 2 ua is
 * exact in float and double; in the double build sin(theta) is taken in
 * double and the float azimuth pair is renormalised in double, so that the
 * unit vector is unit to double round-off.                                   */
static void iso_dir(float ua, float ub, real* nx, real* ny, real* nz) {
#ifdef ORC_F32
    orc_isotropic(ua, ub, nx, ny, nz);
#else
    double ct = 1.0 - 2.0 * (double)ua;
    double st = sqrt(fmax(0.0, fma(-ct, ct, 1.0)));
    float sf, cf;
    orc_sincospif(2.0f * ub, &sf, &cf);
    double c = (double)cf, s = (double)sf;
    double h = sqrt(c * c + s * s);
    c = c / h;
    s = s / h;
    *nx = st * c;
    *ny = st * s;
    *nz = ct;
#endif
}

/* ------------------------------------------------------------------------ */
/* Poisson, Eq. (poisson), on nodes z_j = j dx with Dirichlet values at both
 * electrodes; 3-point central differences for the interior nodes solved by
 * the Thomas algorithm. Node field: central difference inside; at the two
 * electrodes Gauss's law over the half cell adjacent to the wall.          */
void orc_poisson(int N, double dx, double V0, double VN, const double* rho, double* phi, double* E) {
    int M = N - 1;
    phi[0] = V0;
    phi[N] = VN;
    if (M >= 1) {
        double* cp = (double*)malloc(sizeof(double) * (size_t)(M + 1));
        double* dp = (double*)malloc(sizeof(double) * (size_t)(M + 1));
        for (int j = 1; j <= M; ++j) {
            double b = -rho[j] * dx * dx / EPS0;
            if (j == 1) b -= V0;
            if (j == M) b -= VN;
            if (j == 1) {
                cp[j] = 1.0 / -2.0;
                dp[j] = b / -2.0;
            } else {
                double m = -2.0 - cp[j - 1];
                cp[j] = 1.0 / m;
                dp[j] = (b - dp[j - 1]) / m;
            }
        }
        phi[M] = dp[M];
        for (int j = M - 1; j >= 1; --j) phi[j] = dp[j] - cp[j] * phi[j + 1];
        free(cp);
        free(dp);
    }
    for (int j = 1; j < N; ++j) E[j] = (phi[j - 1] - phi[j + 1]) / (2.0 * dx);
    E[0] = (phi[0] - phi[1]) / dx - rho[0] * dx / (2.0 * EPS0);
    E[N] = (phi[N - 1] - phi[N]) / dx + rho[N] * dx / (2.0 * EPS0);
}

/* ------------------------------------------------------------------------ */
static int store_reserve(store* s, int64_t n) {
    if (n <= s->cap) return 0;
    int64_t cap = s->cap ? s->cap : 1024;
    while (cap < n) cap *= 2;
    s->c = (int32_t*)realloc(s->c, sizeof(int32_t) * (size_t)cap);
    s->f = (real*)realloc(s->f, sizeof(real) * (size_t)cap);
    s->vx = (real*)realloc(s->vx, sizeof(real) * (size_t)cap);
    s->vy = (real*)realloc(s->vy, sizeof(real) * (size_t)cap);
    s->vz = (real*)realloc(s->vz, sizeof(real) * (size_t)cap);
    if (!s->c || !s->f || !s->vx || !s->vy || !s->vz) return -1;
    s->cap = cap;
    return 0;
}

static void store_free(store* s) {
    free(s->c); free(s->f); free(s->vx); free(s->vy); free(s->vz);
    memset(s, 0, sizeof(*s));
}

static void store_push(store* s, int32_t c, real f, real vx, real vy, real vz) {
    if (s->n >= s->cap) store_reserve(s, s->n + 1);
    s->c[s->n] = c; s->f[s->n] = f; s->vx[s->n] = vx; s->vy[s->n] = vy; s->vz[s->n] = vz;
    s->n++;
}

int orc_real_bytes(void) { return (int)sizeof(real); }

/* Rate-coefficient tables k_j(eps) = sigma_j(eps) * v(eps) (m^3/s), summed
 * cumulatively over the processes in table order and rounded to real.
 * Electrons: v = sqrt(2 e eps / m_e), lab energy. Ions: relative speed
 * g = sqrt(4 e eps / M) for the centre-of-mass energy eps = M g^2 / 4.     */
static void build_tables(orc_ctx* o) {
    const orc_gas* g = &o->gas;
    int np = o->n_proc_e;
    double kmax_e = 0.0, kmax_i = 0.0;
    for (int k = 0; k < o->n_pts; ++k) {
        double eps = (double)k * g->de_eV;
        double v = sqrt(2.0 * E_CHARGE * eps / M_ELEC);
        double cum = 0.0;
        for (int j = 0; j < 4; ++j) {
            if (j < np) cum = cum + g->sigma_e[(size_t)k * np + j] * v;
            o->Te[(size_t)k * 4 + j] = (real)cum;
        }
        double gr = sqrt(4.0 * E_CHARGE * eps / g->mass_kg);
        cum = 0.0;
        for (int j = 0; j < 2; ++j) {
            cum = cum + g->sigma_i[(size_t)k * 2 + j] * gr;
            o->Ti[(size_t)k * 2 + j] = (real)cum;
        }
        if ((double)o->Te[(size_t)k * 4 + 3] > kmax_e) kmax_e = (double)o->Te[(size_t)k * 4 + 3];
        if ((double)o->Ti[(size_t)k * 2 + 1] > kmax_i) kmax_i = (double)o->Ti[(size_t)k * 2 + 1];
    }
    o->d.kmax_e = kmax_e;
    o->d.kmax_i = kmax_i;
}

static uint32_t null_threshold(double numax, double dt, double* pnull) {
    double P = -expm1(-numax * dt);
    *pnull = P;
    double t = floor(P * TWO32);
    if (t < 0.0) t = 0.0;
    if (t > 4294967295.0) t = 4294967295.0;
    return (uint32_t)t;
}

static void derive(orc_ctx* o) {
    const orc_params* p = &o->p;
    double M = o->gas.mass_kg, de = o->gas.de_eV, dt = p->dt_s;
    orc_derived* d = &o->d;
    d->dx = p->gap_m / (double)p->n_cells;
    d->n_gas = p->p_Pa / (K_BOLTZ * p->T_gas_K);
    d->K_e = (-E_CHARGE / M_ELEC) * (0.5 * dt);
    d->K_i = (E_CHARGE / M) * (0.5 * dt);
    d->dtdx = dt / d->dx;
    d->kappa_e = 0.5 * M_ELEC / (E_CHARGE * de);
    d->kappa_i = 0.25 * M / (E_CHARGE * de);
    d->kappa_E = 0.5 * M_ELEC / E_CHARGE * 4096.0;
    d->beta_e = M_ELEC / (M_ELEC + M);
    d->omb_e = M / (M_ELEC + M);
    for (int j = 0; j < 2; ++j) d->de2_exc[j] = 2.0 * E_CHARGE * o->gas.eps_exc_eV[j] / M_ELEC;
    d->de2_iz = 2.0 * E_CHARGE * o->gas.eps_iz_eV / M_ELEC;
    d->sig_n = sqrt(K_BOLTZ * p->T_gas_K / M);
    d->sig_e0 = sqrt(E_CHARGE * p->T_e0_eV / M_ELEC);
    d->sig_i0 = sqrt(K_BOLTZ * p->T_i0_K / M);
    d->sig_see = sqrt(E_CHARGE * T_SEE_EV / M_ELEC);
    d->sig_see_n = sqrt(2.0 * E_CHARGE * T_SEE_EV / M_ELEC);
    d->numax_e = d->n_gas * d->kmax_e;
    d->numax_i = d->n_gas * d->kmax_i;
    d->thr_e = null_threshold(d->numax_e, dt, &d->pnull_e);
    d->thr_i = null_threshold(d->numax_i, dt, &d->pnull_i);

    o->K_e = (real)d->K_e; o->K_i = (real)d->K_i; o->dtdx = (real)d->dtdx;
    o->kappa_e = (real)d->kappa_e; o->kappa_i = (real)d->kappa_i; o->kappa_E = (real)d->kappa_E;
    o->beta_e = (real)d->beta_e; o->omb_e = (real)d->omb_e;
    o->de2_exc[0] = (real)d->de2_exc[0]; o->de2_exc[1] = (real)d->de2_exc[1];
    o->de2_iz = (real)d->de2_iz;
    o->sig_n = (real)d->sig_n; o->sig_e0 = (real)d->sig_e0; o->sig_i0 = (real)d->sig_i0;
    o->sig_see = (real)d->sig_see; o->sig_see_n = (real)d->sig_see_n;
    o->kmax_e = (real)d->kmax_e; o->kmax_i = (real)d->kmax_i;
    o->gamma = (real)p->gamma_see;
}

orc_ctx* orc_create(const orc_gas* gas, const orc_params* p) {
    if (!gas || !p || p->n_cells < 1 || gas->n_pts < 2 || gas->n_exc < 1 || gas->n_exc > 2) return NULL;
    orc_ctx* o = (orc_ctx*)calloc(1, sizeof(orc_ctx));
    if (!o) return NULL;
    o->p = *p;
    o->V_amp = p->V_rf_V;
    o->gas = *gas;
    o->N = p->n_cells;
    o->n_pts = gas->n_pts;
    o->n_proc_e = 2 + gas->n_exc;
    size_t N1 = (size_t)o->N + 1;
    o->Te = (real*)malloc(sizeof(real) * (size_t)o->n_pts * 4);
    o->Ti = (real*)malloc(sizeof(real) * (size_t)o->n_pts * 2);
    o->E = (real*)calloc(N1, sizeof(real));
    o->E64 = (double*)calloc(N1, sizeof(double));
    o->phi = (double*)calloc(N1, sizeof(double));
    o->rho = (double*)calloc(N1, sizeof(double));
    o->D[0] = (int64_t*)calloc(N1, sizeof(int64_t));
    o->D[1] = (int64_t*)calloc(N1, sizeof(int64_t));
    o->Dprev_e = (int64_t*)calloc(N1, sizeof(int64_t));
    o->Q = (int64_t*)calloc(N1, sizeof(int64_t));
    o->acc_D[0] = (double*)calloc(N1, sizeof(double));
    o->acc_D[1] = (double*)calloc(N1, sizeof(double));
    o->acc_Q = (double*)calloc(N1, sizeof(double));
    o->acc_Dprev = (double*)calloc(N1, sizeof(double));
    build_tables(o);
    derive(o);
    /* the caller's table pointers are not kept */
    o->gas.sigma_e = NULL;
    o->gas.sigma_i = NULL;
    return o;
}

void orc_destroy(orc_ctx* o) {
    if (!o) return;
    store_free(&o->s[0]);
    store_free(&o->s[1]);
    free(o->Te); free(o->Ti); free(o->E); free(o->E64); free(o->phi); free(o->rho);
    free(o->D[0]); free(o->D[1]); free(o->Dprev_e); free(o->Q);
    free(o->acc_D[0]); free(o->acc_D[1]); free(o->acc_Q); free(o->acc_Dprev);
    free(o->dg_D); free(o->dg_U); free(o->dg_V); free(o->dg_W); free(o->dg_K); free(o->dg_F); free(o->dg_Fa);
    free(o->dg_eedf); free(o->dg_E);
    free(o->amp_hist); free(o->V_hist);
    free(o);
}

/* CIC deposit of one superparticle at (c, f): weight 1 - f to node c and f to
 * node c+1, as 64-bit fixed point with 2^32 per particle.                   */
static void deposit(int64_t* D, int32_t c, real f) {
    int64_t F = (int64_t)R_RINT(f * (real)TWO32);
    D[c] += (int64_t)4294967296LL - F;
    D[c + 1] += F;
}

static real gather(const orc_ctx* o, int32_t c, real f) {
    real E0 = o->E[c], E1 = o->E[c + 1];
    return R_FMA(f, E1 - E0, E0);
}

/* Drift by v_z dt in cell units; returns -1 if the particle stays inside,
 * else the electrode it reached (0: z = 0, 1: z = d).                       */
static int drift(const orc_ctx* o, int32_t c, real f, real vz, int32_t* cn, real* fn) {
    real s = R_FMA(vz, o->dtdx, f);
    if (!(s >= (real)(-c))) return 0;
    if (s >= (real)(o->N - c)) return 1;
    real fl = R_FLOOR(s);
    real fr = s - fl;
    if (fr >= (real)1) fr = R_ONE_MINUS_ULP;
    *cn = c + (int32_t)fl;
    *fn = fr;
    return -1;
}

/* Linear interpolation of a cumulative table at xi (grid units); beyond the
 * last point the last row is used.                                          */
static int lookup(const real* T, int ncol, int n_pts, real xi, real* C) {
    real top = (real)(n_pts - 1);
    if (!(xi < top)) {
        for (int j = 0; j < ncol; ++j) C[j] = T[(size_t)(n_pts - 1) * ncol + j];
        return 1;
    }
    int i = (int)xi;
    real fr = xi - (real)i;
    for (int j = 0; j < ncol; ++j) {
        real a = T[(size_t)i * ncol + j], b = T[(size_t)(i + 1) * ncol + j];
        C[j] = R_FMA(fr, b - a, a);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
int orc_load(orc_ctx* o) {
    int N = o->N;
    for (int sp = 0; sp < 2; ++sp) {
        store* s = &o->s[sp];
        int64_t n0 = sp == SP_E ? o->p.n_e0 : o->p.n_i0;
        real sig = sp == SP_E ? o->sig_e0 : o->sig_i0;
        s->n = 0;
        if (store_reserve(s, n0 > 0 ? n0 : 1)) return -1;
        for (int64_t k = 0; k < n0; ++k) {
            uint32_t r[4], q[4];
            int64_t saved = o->step;
            o->step = 0;
            draw(o, (uint32_t)k, sp, CALL_LOAD0, r);
            draw(o, (uint32_t)k, sp, CALL_LOAD1, q);
            o->step = saved;
            real x = (real)U24(r[0]) * (real)N;
            int32_t c = (int32_t)x;
            real f;
            if (c >= N) {
                c = N - 1;
                f = R_ONE_MINUS_ULP;
            } else {
                f = x - (real)c;
            }
            float n0f, n1f, n2f, n3f;
            orc_box_muller(U24(r[1]), U24(r[2]), &n0f, &n1f);
            orc_box_muller(U24(r[3]), U24(q[0]), &n2f, &n3f);
            (void)n3f;
            store_push(s, c, f, sig * (real)n0f, sig * (real)n1f, sig * (real)n2f);
        }
    }
    /* initial deposit and field at t = 0 */
    for (int sp = 0; sp < 2; ++sp) {
        memset(o->D[sp], 0, sizeof(int64_t) * (size_t)(N + 1));
        store* s = &o->s[sp];
        for (int64_t k = 0; k < s->n; ++k) deposit(o->D[sp], s->c[k], s->f[k]);
    }
    o->step = 0;
    {
        /* solve at t_0 = 0 */
        int64_t saved = o->step;
        o->step = -1;
        orc_solve(o);
        o->step = saved;
    }
    /* half back-kick: stored velocity is v_0 - a_0 dt / 2 */
    for (int sp = 0; sp < 2; ++sp) {
        store* s = &o->s[sp];
        real mK = -(sp == SP_E ? o->K_e : o->K_i);
        for (int64_t k = 0; k < s->n; ++k) s->vz[k] = R_FMA(mK, gather(o, s->c[k], s->f[k]), s->vz[k]);
    }
    memcpy(o->Dprev_e, o->D[SP_E], sizeof(int64_t) * (size_t)(N + 1));
    return 0;
}

/* The common end of a load: deposit, field at t = 0, half back-kick. */
static void finish_load(orc_ctx* o) {
    int N = o->N;
    for (int sp = 0; sp < 2; ++sp) {
        memset(o->D[sp], 0, sizeof(int64_t) * (size_t)(N + 1));
        store* s = &o->s[sp];
        for (int64_t k = 0; k < s->n; ++k) deposit(o->D[sp], s->c[k], s->f[k]);
    }
    o->step = -1;
    orc_solve(o);
    o->step = 0;
    for (int sp = 0; sp < 2; ++sp) {
        store* s = &o->s[sp];
        real mK = -(sp == SP_E ? o->K_e : o->K_i);
        for (int64_t k = 0; k < s->n; ++k) s->vz[k] = R_FMA(mK, gather(o, s->c[k], s->f[k]), s->vz[k]);
    }
    memcpy(o->Dprev_e, o->D[SP_E], sizeof(int64_t) * (size_t)(N + 1));
}

int orc_load_profiles(orc_ctx* o, int P, const double* n_e, const double* n_i, const double* mean_eps) {
    const int N = o->N;
    if (P < 2) return -1;
    real* cdf = (real*)malloc(sizeof(real) * (size_t)P);
    real* eps = (real*)malloc(sizeof(real) * (size_t)P);
    const double dz = o->p.gap_m / (double)(P - 1);
    const real scale = (real)((double)N / (double)(P - 1));
    const real K23 = (real)(2.0 * E_CHARGE / (3.0 * M_ELEC));
    for (int j = 0; j < P; ++j) eps[j] = (real)(mean_eps[j] > 0.0 ? mean_eps[j] : 0.0);
    for (int sp = 0; sp < 2; ++sp) {
        const double* prof = sp == SP_E ? n_e : n_i;
        const double w = sp == SP_E ? o->p.w_e : o->p.w_i;
        double A = 0.0;
        for (int j = 0; j + 1 < P; ++j) {
            double a = 0.5 * (fmax(prof[j], 0.0) + fmax(prof[j + 1], 0.0)) * dz;
            A += a;
        }
        int64_t n = A > 0.0 ? (int64_t)floor(A / w + 0.5) : 0;
        double run = 0.0;
        cdf[0] = (real)0;
        for (int j = 0; j + 1 < P; ++j) {
            run += 0.5 * (fmax(prof[j], 0.0) + fmax(prof[j + 1], 0.0)) * dz;
            cdf[j + 1] = (real)(A > 0.0 ? run / A : 0.0);
        }
        cdf[P - 1] = (real)1;
        store* s = &o->s[sp];
        s->n = 0;
        if (store_reserve(s, n > 0 ? n : 1)) return -1;
        for (int64_t k = 0; k < n; ++k) {
            uint32_t r[4], q[4];
            draw(o, (uint32_t)k, sp, CALL_WARM0, r);
            draw(o, (uint32_t)k, sp, CALL_WARM1, q);
            const real u = (real)U24(r[0]);
            int lo = 0, hi = P - 2;   /* largest j in [0, P-2] with cdf[j] <= u */
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (cdf[mid] <= u) lo = mid;
                else hi = mid - 1;
            }
            const int j = lo;
            const real den = cdf[j + 1] - cdf[j];
            real t = den > (real)0 ? (u - cdf[j]) / den : (real)0;
            if (t >= (real)1) t = R_ONE_MINUS_ULP;
            const real x = ((real)j + t) * scale;
            int32_t c = (int32_t)x;
            real f;
            if (c >= N) {
                c = N - 1;
                f = R_ONE_MINUS_ULP;
            } else {
                f = x - (real)c;
            }
            real sig;
            if (sp == SP_E) {
                real el = R_FMA(t, eps[j + 1] - eps[j], eps[j]);
                if (!(el > (real)0)) el = (real)0;
                sig = R_SQRT(el * K23);
            } else {
                sig = o->sig_i0;
            }
            float n0f, n1f, n2f, n3f;
            orc_box_muller(U24(r[1]), U24(r[2]), &n0f, &n1f);
            orc_box_muller(U24(r[3]), U24(q[0]), &n2f, &n3f);
            (void)n3f;
            store_push(s, c, f, sig * (real)n0f, sig * (real)n1f, sig * (real)n2f);
        }
    }
    free(cdf);
    free(eps);
    finish_load(o);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One sweep over both species at step n, from (x_n, v*) with the node field
 * E_n: v_n = v* + K E(x_n); collision on v_n; v* <- v_n + K E(x_n);
 * x_{n+1} = x_n + v*_z dt; absorption; deposit at x_{n+1}.
 * New arrays: the survivors in input-slot order, then the newborns that stay,
 * in parent-slot order: for electrons the ionization electrons, then the
 * secondary electrons of absorbed ions; for ions the ionization ions.       */
int orc_sweep(orc_ctx* o) {
    const int N = o->N;
    size_t N1 = (size_t)N + 1;
    /* out: survivors in input order; sec: ionization electrons in parent order; birth[sp]: newborns
     * of species sp made by the other species' sweep (ions from ionization, SEE electrons) */
    store out[2], birth[2], sec;
    memset(out, 0, sizeof(out));
    memset(birth, 0, sizeof(birth));
    memset(&sec, 0, sizeof(sec));
    if (store_reserve(&out[SP_E], o->s[SP_E].n * 2 + 16) || store_reserve(&out[SP_I], o->s[SP_I].n + 16) ||
        store_reserve(&birth[SP_E], 16) || store_reserve(&birth[SP_I], 16) || store_reserve(&sec, 16))
        return -1;
    memcpy(o->Dprev_e, o->D[SP_E], sizeof(int64_t) * N1);
    memset(o->Q, 0, sizeof(int64_t) * N1);
    memset(o->D[0], 0, sizeof(int64_t) * N1);
    memset(o->D[1], 0, sizeof(int64_t) * N1);
    const int ncol_e = 4;

    /* electrons */
    {
        store* s = &o->s[SP_E];
        for (int64_t k = 0; k < s->n; ++k) {
            uint32_t slot = (uint32_t)k;
            int32_t c = s->c[k];
            real f = s->f[k], vx = s->vx[k], vy = s->vy[k], vz = s->vz[k];
            real ef = gather(o, c, f);
            vz = R_FMA(o->K_e, ef, vz);
            real e2 = R_FMA(vx, vx, R_FMA(vy, vy, vz * vz));
            {   /* energy moment at (x_n, v_n), 2^-12 eV fixed point, clamped at 2^26 (16384 eV) */
                real eq = e2 * o->kappa_E;
                if (!(eq <= (real)0x1p26)) eq = (real)0x1p26;
                int64_t Et = (int64_t)R_RINT(eq);
                int64_t Eh = (int64_t)R_RINT(eq * f);
                o->Q[c] += Et - Eh;
                o->Q[c + 1] += Eh;
            }
            if (o->leapfrog) {  /* both half kicks first: the collision acts on v_{n+1/2} */
                vz = R_FMA(o->K_e, ef, vz);
                e2 = R_FMA(vx, vx, R_FMA(vy, vy, vz * vz));
            }
            int have_child = 0;
            real ce_vx = 0, ce_vy = 0, ce_vz = 0, ci_vx = 0, ci_vy = 0, ci_vz = 0;
            if (candidate_word(o, slot, SP_E) < o->d.thr_e) {
                uint32_t r[4];
                draw(o, slot, SP_E, CALL_MAIN, r);
                o->cnt.candidates[SP_E]++;
                real C[4];
                o->cnt.table_clamped[SP_E] += lookup(o->Te, ncol_e, o->n_pts, e2 * o->kappa_e, C);
                real R = (real)U24(r[1]) * o->kmax_e;
                int j = 0;
                while (j < 4 && !(R < C[j])) ++j;
                if (j < 4) {
                    real nx, ny, nz;
                    if (j == 0) {
                        /* elastic, target at rest: v' = beta v + (1-beta)|v| n */
                        real g = R_SQRT(e2);
                        iso_dir(U24(r[2]), U24(r[3]), &nx, &ny, &nz);
                        real og = o->omb_e * g;
                        vx = R_FMA(o->beta_e, vx, og * nx);
                        vy = R_FMA(o->beta_e, vy, og * ny);
                        vz = R_FMA(o->beta_e, vz, og * nz);
                        o->cnt.collisions_e[0]++;
                    } else if (j <= o->gas.n_exc) {
                        real e2n = e2 - o->de2_exc[j - 1];
                        if (e2n > (real)0) {
                            real sp = R_SQRT(e2n);
                            iso_dir(U24(r[2]), U24(r[3]), &nx, &ny, &nz);
                            vx = sp * nx;
                            vy = sp * ny;
                            vz = sp * nz;
                            o->cnt.collisions_e[j]++;
                        } else {
                            o->cnt.null_inelastic++;
                        }
                    } else {
                        real e2r = e2 - o->de2_iz;
                        if (e2r > (real)0) {
                            real sp = R_SQRT((real)0.5 * e2r);
                            iso_dir(U24(r[2]), U24(r[3]), &nx, &ny, &nz);
                            vx = sp * nx;
                            vy = sp * ny;
                            vz = sp * nz;
                            uint32_t q[4], w[4];
                            draw(o, slot, SP_E, CALL_AUX, q);
                            draw(o, slot, SP_E, CALL_AUX2, w);
                            iso_dir(U24(q[0]), U24(q[1]), &nx, &ny, &nz);
                            ce_vx = sp * nx;
                            ce_vy = sp * ny;
                            ce_vz = sp * nz;
                            float b0, b1, b2, b3;
                            orc_box_muller(U24(q[2]), U24(q[3]), &b0, &b1);
                            orc_box_muller(U24(w[0]), U24(w[1]), &b2, &b3);
                            (void)b3;
                            ci_vx = o->sig_n * (real)b0;
                            ci_vy = o->sig_n * (real)b1;
                            ci_vz = o->sig_n * (real)b2;
                            have_child = 1;
                            o->cnt.collisions_e[3]++;
                        } else {
                            o->cnt.null_inelastic++;
                        }
                    }
                }
            }
            if (!o->leapfrog) vz = R_FMA(o->K_e, ef, vz);  /* second half kick after the collision */
            int32_t cn;
            real fn;
            int side = drift(o, c, f, vz, &cn, &fn);
            if (side < 0) {
                store_push(&out[SP_E], cn, fn, vx, vy, vz);
                deposit(o->D[SP_E], cn, fn);
            } else {
                o->cnt.absorbed[SP_E][side]++;
            }
            if (have_child) {
                if (!o->leapfrog) ce_vz = R_FMA(o->K_e, ef, ce_vz);  /* newborns born at t_n: half kick */
                side = drift(o, c, f, ce_vz, &cn, &fn);
                if (side < 0) {
                    store_push(&sec, cn, fn, ce_vx, ce_vy, ce_vz);
                    deposit(o->D[SP_E], cn, fn);
                } else {
                    o->cnt.absorbed[SP_E][side]++;
                }
                if (!o->leapfrog) ci_vz = R_FMA(o->K_i, ef, ci_vz);
                side = drift(o, c, f, ci_vz, &cn, &fn);
                if (side < 0) {
                    store_push(&birth[SP_I], cn, fn, ci_vx, ci_vy, ci_vz);
                    deposit(o->D[SP_I], cn, fn);
                } else {
                    o->cnt.absorbed[SP_I][side]++;
                }
            }
        }
    }

    /* ions */
    {
        store* s = &o->s[SP_I];
        for (int64_t k = 0; k < s->n; ++k) {
            uint32_t slot = (uint32_t)k;
            int32_t c = s->c[k];
            real f = s->f[k], vx = s->vx[k], vy = s->vy[k], vz = s->vz[k];
            real ef = gather(o, c, f);
            vz = R_FMA(o->K_i, ef, vz);
            if (o->leapfrog) vz = R_FMA(o->K_i, ef, vz);  /* collision at v_{n+1/2} */
            if (candidate_word(o, slot, SP_I) < o->d.thr_i) {
                uint32_t r[4];
                draw(o, slot, SP_I, CALL_MAIN, r);
                o->cnt.candidates[SP_I]++;
                uint32_t q[4];
                draw(o, slot, SP_I, CALL_AUX, q);
                float a0, a1, a2, a3;
                orc_box_muller(U24(q[0]), U24(q[1]), &a0, &a1);
                orc_box_muller(U24(q[2]), U24(q[3]), &a2, &a3);
                (void)a3;
                real vnx = o->sig_n * (real)a0, vny = o->sig_n * (real)a1, vnz = o->sig_n * (real)a2;
                real gx = vx - vnx, gy = vy - vny, gz = vz - vnz;
                real g2 = R_FMA(gx, gx, R_FMA(gy, gy, gz * gz));
                real C[2];
                o->cnt.table_clamped[SP_I] += lookup(o->Ti, 2, o->n_pts, g2 * o->kappa_i, C);
                real R = (real)U24(r[1]) * o->kmax_i;
                if (R < C[0]) {
                    /* isotropic in the centre-of-mass frame, equal masses */
                    real hg = (real)0.5 * R_SQRT(g2);
                    real nx, ny, nz;
                    iso_dir(U24(r[2]), U24(r[3]), &nx, &ny, &nz);
                    vx = R_FMA(hg, nx, (vx + vnx) * (real)0.5);
                    vy = R_FMA(hg, ny, (vy + vny) * (real)0.5);
                    vz = R_FMA(hg, nz, (vz + vnz) * (real)0.5);
                    o->cnt.collisions_i[0]++;
                } else if (R < C[1]) {
                    /* backward elastic: the ion leaves with the neutral's velocity */
                    vx = vnx;
                    vy = vny;
                    vz = vnz;
                    o->cnt.collisions_i[1]++;
                }
            }
            if (!o->leapfrog) vz = R_FMA(o->K_i, ef, vz);
            int32_t cn;
            real fn;
            int side = drift(o, c, f, vz, &cn, &fn);
            if (side < 0) {
                store_push(&out[SP_I], cn, fn, vx, vy, vz);
                deposit(o->D[SP_I], cn, fn);
            } else {
                o->cnt.absorbed[SP_I][side]++;
                if (o->p.gamma_see > 0.0) {
                    uint32_t w[4];
                    draw(o, slot, SP_I, CALL_SEE, w);
                    if ((real)U24(w[0]) < o->gamma) {
                        real vn = o->sig_see_n * (real)sqrtf(-orc_logf(U24(w[1])));
                        float t0, t1;
                        orc_box_muller(U24(w[2]), U24(w[3]), &t0, &t1);
                        int32_t ce = side == 0 ? 0 : N - 1;
                        real fe = side == 0 ? (real)0 : R_ONE_MINUS_ULP;
                        store_push(&birth[SP_E], ce, fe, o->sig_see * (real)t0, o->sig_see * (real)t1,
                                   side == 0 ? vn : -vn);
                        deposit(o->D[SP_E], ce, fe);
                        o->cnt.see_emitted++;
                        o->see_side[side]++;
                    }
                }
            }
        }
    }

    /* newborns after the survivors, in parent order: electrons get the ionization electrons, then
     * the SEE electrons; ions get the ionization ions */
    for (int64_t k = 0; k < sec.n; ++k) store_push(&out[SP_E], sec.c[k], sec.f[k], sec.vx[k], sec.vy[k], sec.vz[k]);
    store_free(&sec);
    for (int sp = 0; sp < 2; ++sp) {
        store* b = &birth[sp];
        for (int64_t k = 0; k < b->n; ++k) store_push(&out[sp], b->c[k], b->f[k], b->vx[k], b->vy[k], b->vz[k]);
        store_free(b);
        store_free(&o->s[sp]);
        o->s[sp] = out[sp];
    }
    return 0;
}

/* Stable counting sort of each species by cell index. */
int orc_sort(orc_ctx* o) {
    int N = o->N;
    int64_t* start = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    if (!start) return -1;
    for (int sp = 0; sp < 2; ++sp) {
        store* s = &o->s[sp];
        store t;
        memset(&t, 0, sizeof(t));
        if (store_reserve(&t, s->n > 0 ? s->n : 1)) return -1;
        memset(start, 0, sizeof(int64_t) * ((size_t)N + 1));
        for (int64_t k = 0; k < s->n; ++k) start[s->c[k] + 1]++;
        for (int j = 0; j < N; ++j) start[j + 1] += start[j];
        for (int64_t k = 0; k < s->n; ++k) {
            int64_t dst = start[s->c[k]]++;
            t.c[dst] = s->c[k]; t.f[dst] = s->f[k]; t.vx[dst] = s->vx[k];
            t.vy[dst] = s->vy[k]; t.vz[dst] = s->vz[k];
        }
        t.n = s->n;
        store_free(s);
        *s = t;
    }
    free(start);
    return 0;
}

/* Charge density from the deposits (node volume dx inside, dx/2 at the
 * electrodes), Poisson at t_{n+1} = (n+1) dt, node field; then n <- n+1.   */
int orc_solve(orc_ctx* o) {
    int N = o->N;
    double dx = o->d.dx;
    double t = (double)(o->step + 1) * o->p.dt_s;
    for (int j = 0; j <= N; ++j) {
        double Vj = (j == 0 || j == N) ? 0.5 * dx : dx;
        o->rho[j] = E_CHARGE * (o->p.w_i * (double)o->D[SP_I][j] - o->p.w_e * (double)o->D[SP_E][j]) / (TWO32 * Vj);
    }
    double V0 = o->V_amp * sin(2.0 * PI_D * o->p.f_rf_Hz * t);
    orc_poisson(N, dx, V0, 0.0, o->rho, o->phi, o->E64);
    for (int j = 0; j <= N; ++j) o->E[j] = (real)o->E64[j];
    /* Discharge current density over the step just solved for (from the previous solve to this
     * one), J = eps0 dE/dt + e0 (Gamma_i - Gamma_e), fluxes counted positive towards +z:
     * at z = 0 absorbed ions (moving towards -z) carry -e w_i, absorbed electrons +e w_e, emitted
     * secondary electrons (moving towards +z) -e w_e; at z = d the signs of the absorbed
     * particles flip and emitted electrons move towards -z. */
    if (o->have_solve) {
        double dt = o->p.dt_s, we = o->p.w_e, wi = o->p.w_i;
        double dA[2][2], dS[2];
        for (int a = 0; a < 2; ++a) {
            for (int b = 0; b < 2; ++b) dA[a][b] = (double)(o->cnt.absorbed[a][b] - o->abs_prev[a][b]);
            dS[a] = (double)(o->see_side[a] - o->see_prev[a]);
        }
        double cond0 = E_CHARGE * (we * dA[SP_E][0] - wi * dA[SP_I][0] - we * dS[0]) / dt;
        double condN = E_CHARGE * (wi * dA[SP_I][1] - we * dA[SP_E][1] + we * dS[1]) / dt;
        o->J_last[0] = EPS0 * (o->E64[0] - o->E_wall_prev[0]) / dt + cond0;
        o->J_last[1] = EPS0 * (o->E64[N] - o->E_wall_prev[1]) / dt + condN;
    } else {
        o->J_last[0] = o->J_last[1] = 0.0;
    }
    o->have_solve = 1;
    o->E_wall_prev[0] = o->E64[0];
    o->E_wall_prev[1] = o->E64[N];
    for (int a = 0; a < 2; ++a) {
        for (int b = 0; b < 2; ++b) o->abs_prev[a][b] = o->cnt.absorbed[a][b];
        o->see_prev[a] = o->see_side[a];
    }
    o->step++;
    return 0;
}

void orc_last_current(const orc_ctx* o, double J[2]) {
    J[0] = o->J_last[0];
    J[1] = o->J_last[1];
}

/* End of step n (its solve done, J_last = J of step n): first-harmonic projections of J(0,t) over
 * the rf period at the step midpoints t_{n+1/2}; at the period's last step its amplitude
 * J_calc = sqrt(a^2 + b^2), a = (2/P) sum J sin(w t), b = (2/P) sum J cos(w t), and in the
 * current-driven mode V0 <- V0 J0 / J_calc for the next period (Eq. adaptivevoltage).           */
static void period_current(orc_ctx* o, int64_t n) {
    const int P = o->period_steps;
    if (P <= 0) return;
    const double w = 2.0 * PI_D * o->p.f_rf_Hz, th = w * ((double)(n % P) + 0.5) * o->p.dt_s;
    o->proj_a += o->J_last[0] * sin(th);
    o->proj_b += o->J_last[0] * cos(th);
    if (n % P != P - 1) return;
    const double a = 2.0 * o->proj_a / P, b = 2.0 * o->proj_b / P;
    const double amp = sqrt(a * a + b * b);
    if (o->hist_n == o->hist_cap) {
        o->hist_cap = o->hist_cap ? 2 * o->hist_cap : 64;
        o->amp_hist = (double*)realloc(o->amp_hist, sizeof(double) * (size_t)o->hist_cap);
        o->V_hist = (double*)realloc(o->V_hist, sizeof(double) * (size_t)o->hist_cap);
    }
    o->amp_hist[o->hist_n] = amp;
    o->V_hist[o->hist_n] = o->V_amp;  /* the amplitude applied during this period */
    o->hist_n++;
    if (o->J_target > 0.0 && amp > 0.0) o->V_amp = o->V_amp * (o->J_target / amp);
    o->proj_a = o->proj_b = 0.0;
}

int orc_set_scheme(orc_ctx* o, int leapfrog) {
    if (leapfrog != 0 && leapfrog != 1) return -1;
    o->leapfrog = leapfrog;
    return 0;
}

int orc_set_current_drive(orc_ctx* o, int period_steps, double J_target) {
    if (period_steps < 0 || !(J_target >= 0.0)) return -1;
    o->period_steps = period_steps;
    o->J_target = J_target;
    o->proj_a = o->proj_b = 0.0;
    return 0;
}

int64_t orc_period_history(const orc_ctx* o, double* amp, double* V0, int64_t cap, double* V_now) {
    const int64_t n = o->hist_n < cap ? o->hist_n : cap;
    if (amp) memcpy(amp, o->amp_hist, sizeof(double) * (size_t)n);
    if (V0) memcpy(V0, o->V_hist, sizeof(double) * (size_t)n);
    if (V_now) *V_now = o->V_amp;
    return o->hist_n;
}

static void diag_take(orc_ctx* o);

int orc_step(orc_ctx* o, int64_t n_steps) {
    int N = o->N;
    for (int64_t it = 0; it < n_steps; ++it) {
        if (o->dg_on) diag_take(o);
        if (orc_sweep(o)) return -1;
        int64_t n = o->step;
        if (o->p.sort_every > 0 && (n + 1) % o->p.sort_every == 0)
            if (orc_sort(o)) return -1;
        orc_solve(o);
        period_current(o, n);
        for (int j = 0; j <= N; ++j) {
            o->acc_D[0][j] += (double)o->D[0][j];
            o->acc_D[1][j] += (double)o->D[1][j];
            o->acc_Q[j] += (double)o->Q[j];
            o->acc_Dprev[j] += (double)o->Dprev_e[j];
        }
        o->acc_steps++;
    }
    return 0;
}

/* Densities n_s,j = w_s D_s,j / (2^32 V_j) averaged over the accumulated
 * steps; mean electron energy (eV) = energy moment / density moment, both
 * taken at (x_n, v_n).                                                      */
int orc_moments(const orc_ctx* o, double* n_e, double* n_i, double* mean_eps, orc_moment_info* info) {
    int N = o->N;
    double dx = o->d.dx;
    double ns = o->acc_steps > 0 ? (double)o->acc_steps : 1.0;
    for (int j = 0; j <= N; ++j) {
        double Vj = (j == 0 || j == N) ? 0.5 * dx : dx;
        if (n_e) n_e[j] = o->p.w_e * o->acc_D[0][j] / (TWO32 * Vj * ns);
        if (n_i) n_i[j] = o->p.w_i * o->acc_D[1][j] / (TWO32 * Vj * ns);
        if (mean_eps) mean_eps[j] = o->acc_Dprev[j] > 0.0 ? (o->acc_Q[j] / 4096.0) / (o->acc_Dprev[j] / TWO32) : 0.0;
    }
    if (info) {
        info->steps = o->acc_steps;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                info->absorbed[a][b] = (double)(o->cnt.absorbed[a][b] - o->cnt_at_reset.absorbed[a][b]);
    }
    return 0;
}

void orc_reset_moments(orc_ctx* o) {
    size_t N1 = (size_t)o->N + 1;
    memset(o->acc_D[0], 0, sizeof(double) * N1);
    memset(o->acc_D[1], 0, sizeof(double) * N1);
    memset(o->acc_Q, 0, sizeof(double) * N1);
    memset(o->acc_Dprev, 0, sizeof(double) * N1);
    o->acc_steps = 0;
    o->cnt_at_reset = o->cnt;
}

/* ------------------------------------------------------------------------ */
int64_t orc_count(const orc_ctx* o, int species) { return o->s[species & 1].n; }

int orc_get_state(const orc_ctx* o, int species, int32_t* c, void* f, void* vx, void* vy, void* vz) {
    const store* s = &o->s[species & 1];
    size_t n = (size_t)s->n;
    if (c) memcpy(c, s->c, n * sizeof(int32_t));
    if (f) memcpy(f, s->f, n * sizeof(real));
    if (vx) memcpy(vx, s->vx, n * sizeof(real));
    if (vy) memcpy(vy, s->vy, n * sizeof(real));
    if (vz) memcpy(vz, s->vz, n * sizeof(real));
    return 0;
}

int orc_set_state(orc_ctx* o, int species, int64_t n, const int32_t* c, const void* f, const void* vx,
                  const void* vy, const void* vz) {
    store* s = &o->s[species & 1];
    if (store_reserve(s, n > 0 ? n : 1)) return -1;
    for (int64_t k = 0; k < n; ++k)
        if (c[k] < 0 || c[k] >= o->N) return -2;
    memcpy(s->c, c, (size_t)n * sizeof(int32_t));
    memcpy(s->f, f, (size_t)n * sizeof(real));
    memcpy(s->vx, vx, (size_t)n * sizeof(real));
    memcpy(s->vy, vy, (size_t)n * sizeof(real));
    memcpy(s->vz, vz, (size_t)n * sizeof(real));
    s->n = n;
    return 0;
}

int orc_get_field(const orc_ctx* o, void* E) {
    memcpy(E, o->E, sizeof(real) * ((size_t)o->N + 1));
    return 0;
}
int orc_set_field(orc_ctx* o, const void* E) {
    memcpy(o->E, E, sizeof(real) * ((size_t)o->N + 1));
    return 0;
}
int orc_get_phi(const orc_ctx* o, double* phi) {
    memcpy(phi, o->phi, sizeof(double) * ((size_t)o->N + 1));
    return 0;
}
int orc_get_efield64(const orc_ctx* o, double* E) {
    memcpy(E, o->E64, sizeof(double) * ((size_t)o->N + 1));
    return 0;
}
int orc_get_deposit(const orc_ctx* o, int species, int64_t* D) {
    memcpy(D, o->D[species & 1], sizeof(int64_t) * ((size_t)o->N + 1));
    return 0;
}
int orc_set_deposit(orc_ctx* o, int species, const int64_t* D) {
    memcpy(o->D[species & 1], D, sizeof(int64_t) * ((size_t)o->N + 1));
    return 0;
}
int orc_get_energy_deposit(const orc_ctx* o, int64_t* Q) {
    memcpy(Q, o->Q, sizeof(int64_t) * ((size_t)o->N + 1));
    return 0;
}
int64_t orc_get_step(const orc_ctx* o) { return o->step; }
void orc_set_step(orc_ctx* o, int64_t n) { o->step = n; }
void orc_get_counters(const orc_ctx* o, orc_counters* out) { *out = o->cnt; }
void orc_get_derived(const orc_ctx* o, orc_derived* out) { *out = o->d; }
int orc_get_tables(const orc_ctx* o, void* Te, void* Ti) {
    if (Te) memcpy(Te, o->Te, sizeof(real) * (size_t)o->n_pts * 4);
    if (Ti) memcpy(Ti, o->Ti, sizeof(real) * (size_t)o->n_pts * 2);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Kinetic diagnostics (see pic_oracle.h). The field average is of the node field the particles
 * gather (the particle precision). Per electron at (x_n, v_n): the gathered field and the
 * first half kick as in the sweep, the energy e2 kappa_E in 2^-12 eV clamped at 2^26 as for the
 * energy moment, then each moment as an integer value X (rounded in the particle precision) split
 * between the two nodes of its cell like the charge: X - Xh to node c, Xh = rn(X f) to node c+1.
 * Units of X: density 2^32 per particle (the deposit's F split), energy 2^-12 eV, particle flux
 * v_z 2^6 (1/64 m/s), energy flux U v_z 2^-4 (16 eV m/s, formed as eq v_z 2^-16), ionization rate
 * coefficient sigma_iz v 2^72 (m^3/s).                                                         */
int orc_set_diagnostics(orc_ctx* o, const orc_diag_config* cfg) {
    if (!cfg || cfg->period_steps < 0 || cfg->eedf_bins < 1 || !(cfg->eedf_de_eV > 0)) return -1;
    o->dg = *cfg;
    size_t N1 = (size_t)o->N + 1;
    int64_t** arr[7] = {&o->dg_D, &o->dg_U, &o->dg_V, &o->dg_W, &o->dg_K, &o->dg_F, &o->dg_Fa};
    for (int k = 0; k < 7; ++k) {
        free(*arr[k]);
        *arr[k] = (int64_t*)calloc(N1, sizeof(int64_t));
    }
    free(o->dg_eedf);
    o->dg_eedf = (int64_t*)calloc((size_t)cfg->eedf_bins, sizeof(int64_t));
    free(o->dg_E);
    o->dg_E = (double*)calloc(N1, sizeof(double));
    o->dg_on = 1;
    orc_reset_diagnostics(o);
    return 0;
}

void orc_reset_diagnostics(orc_ctx* o) {
    if (!o->dg_on) return;
    size_t N1 = (size_t)o->N + 1;
    int64_t* arr[7] = {o->dg_D, o->dg_U, o->dg_V, o->dg_W, o->dg_K, o->dg_F, o->dg_Fa};
    for (int k = 0; k < 7; ++k) memset(arr[k], 0, sizeof(int64_t) * N1);
    memset(o->dg_eedf, 0, sizeof(int64_t) * (size_t)o->dg.eedf_bins);
    memset(o->dg_E, 0, sizeof(double) * N1);
    o->dg_snap = 0;
    o->dg_samples = 0;
}

static void split_add(int64_t* h, int32_t c, real x, real f) {
    int64_t X = (int64_t)R_RINT(x), Xh = (int64_t)R_RINT(x * f);
    h[c] += X - Xh;
    h[c + 1] += Xh;
}

static void diag_take(orc_ctx* o) {
    const int64_t n = o->step;
    const int P = o->dg.period_steps;
    const int phase = P > 0 && o->dg.phase_step >= 0 && n % P == o->dg.phase_step;
    const int sample = o->dg.sample_every > 0 && n % o->dg.sample_every == 0;
    if (!phase && !sample) return;
    const int N = o->N, bins = o->dg.eedf_bins;
    const real thr = (real)(o->dg.fast_eV * 4096.0);          /* 2^-12 eV */
    const real inv_bin = (real)(1.0 / (o->dg.eedf_de_eV * 4096.0));
    const int ciz = o->n_proc_e - 1;                          /* ionization column of the table */
    const store* s = &o->s[SP_E];
    if (phase) {
        for (int j = 0; j <= N; ++j) o->dg_E[j] += (double)o->E[j];
        o->dg_snap++;
    }
    if (sample) o->dg_samples++;
    for (int64_t k = 0; k < s->n; ++k) {
        const int32_t c = s->c[k];
        const real f = s->f[k], vx = s->vx[k], vy = s->vy[k];
        const real ef = gather(o, c, f);
        const real vz = R_FMA(o->K_e, ef, s->vz[k]);           /* v_n */
        const real e2 = R_FMA(vx, vx, R_FMA(vy, vy, vz * vz));
        real eq = e2 * o->kappa_E;
        if (!(eq <= (real)0x1p26)) eq = (real)0x1p26;
        const int64_t F = (int64_t)R_RINT(f * (real)TWO32);
        const int fast = eq > thr;
        if (phase) {
            o->dg_D[c] += (int64_t)4294967296LL - F;
            o->dg_D[c + 1] += F;
            split_add(o->dg_U, c, eq, f);
            split_add(o->dg_V, c, vz * (real)64.0, f);
            split_add(o->dg_W, c, (eq * vz) * (real)0x1p-16, f);
            real C[4];
            lookup(o->Te, 4, o->n_pts, e2 * o->kappa_e, C);
            split_add(o->dg_K, c, (C[ciz] - C[ciz - 1]) * (real)0x1p72, f);
            if (fast) {
                o->dg_F[c] += (int64_t)4294967296LL - F;
                o->dg_F[c + 1] += F;
            }
        }
        if (sample) {
            const real xb = eq * inv_bin;                     /* bin index, clamped before the conversion */
            const int b = xb < (real)bins ? (int)xb : bins - 1;
            o->dg_eedf[b]++;
            if (fast) {
                o->dg_Fa[c] += (int64_t)4294967296LL - F;
                o->dg_Fa[c + 1] += F;
            }
        }
    }
}

int orc_diagnostics(const orc_ctx* o, double* E, double* n_e, double* mean_eps, double* gamma_e, double* q_e,
                    double* heating, double* ion_rate, double* n_fast, double* n_fast_avg, double* eedf,
                    int64_t* snapshots, int64_t* samples) {
    if (!o->dg_on) return -1;
    const int N = o->N;
    const double dx = o->d.dx, w = o->p.w_e;
    const double ns = o->dg_snap > 0 ? (double)o->dg_snap : 1.0, nm = o->dg_samples > 0 ? (double)o->dg_samples : 1.0;
    for (int j = 0; j <= N; ++j) {
        const double Vj = (j == 0 || j == N) ? 0.5 * dx : dx;
        const double Ej = o->dg_E[j] / ns;
        const double g = w * (double)o->dg_V[j] / 64.0 / (Vj * ns);
        if (E) E[j] = Ej;
        if (n_e) n_e[j] = w * (double)o->dg_D[j] / (TWO32 * Vj * ns);
        if (mean_eps) mean_eps[j] = o->dg_D[j] > 0 ? ((double)o->dg_U[j] / 4096.0) / ((double)o->dg_D[j] / TWO32) : 0.0;
        if (gamma_e) gamma_e[j] = g;
        if (q_e) q_e[j] = w * E_CHARGE * (double)o->dg_W[j] * 16.0 / (Vj * ns);
        if (heating) heating[j] = -E_CHARGE * Ej * g;
        if (ion_rate) ion_rate[j] = o->d.n_gas * w * (double)o->dg_K[j] * 0x1p-72 / (Vj * ns);
        if (n_fast) n_fast[j] = w * (double)o->dg_F[j] / (TWO32 * Vj * ns);
        if (n_fast_avg) n_fast_avg[j] = w * (double)o->dg_Fa[j] / (TWO32 * Vj * nm);
    }
    if (eedf) {
        double tot = 0.0;
        for (int b = 0; b < o->dg.eedf_bins; ++b) tot += (double)o->dg_eedf[b];
        for (int b = 0; b < o->dg.eedf_bins; ++b) {
            const double U = (b + 0.5) * o->dg.eedf_de_eV;
            eedf[b] = tot > 0 ? (double)o->dg_eedf[b] / (tot * o->dg.eedf_de_eV * sqrt(U)) : 0.0;
        }
    }
    if (snapshots) *snapshots = o->dg_snap;
    if (samples) *samples = o->dg_samples;
    return 0;
}
