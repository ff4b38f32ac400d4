// pic_internal.h -- device-side data layout shared by the host runtime and the
// kernels of the PIC/MCC library (not part of the public ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pic {

constexpr int MAXD = 64;      // discharges per context
constexpr int MAXN = 4096;    // cells per discharge
constexpr int SLICE = 4096;   // sweep chunks per slice of the segment-table pass
constexpr int NCNT = 18;      // event counters per discharge

// Event counter slots (u64 each), per discharge.
enum {
    CNT_ABS = 0,       // 4: [species][electrode]
    CNT_COLL_E = 4,    // 4: elastic, exc1, exc2, ionization
    CNT_COLL_I = 8,    // 2: isotropic, backward
    CNT_NULL_INEL = 10,
    CNT_SEE = 11,
    CNT_CAND = 12,     // 2
    CNT_CLAMP = 14,    // 2
    CNT_SEE_SIDE = 16  // 2: secondary electrons emitted at electrode 0, 1
};

// Device error bits (Ctl::error).
enum : int { ERR_CAPACITY = 1, ERR_TIMEOUT = 2, ERR_NONFINITE = 4 };

// Per-particle constants of one discharge in the particle precision T.
template <typename T>
struct Consts {
    T K[2];            // (q/m) dt/2, electrons and ions
    T dtdx;            // dt / dx
    T kappa_e;         // (m_e/2e)/de : speed^2 -> grid index (lab energy)
    T kappa_i;         // (M/4e)/de   : relative speed^2 -> grid index (c.m. energy)
    T kappa_E;         // (m_e/2e) 2^12 : speed^2 -> energy in 2^-12 eV
    T beta, omb;       // m_e/(m_e+M), M/(m_e+M)
    T de2_exc[2];      // excitation thresholds in speed^2 units
    T de2_iz;          // ionization threshold in speed^2 units
    T sig_n;           // sqrt(kT_gas/M)
    T sig_see, sig_see_n;  // emitted electrons: tangential sigma, normal scale
    T kmax_e, kmax_i;  // table maxima (m^3/s)
    T gamma;           // secondary emission yield
    T sig0[2];         // initial Maxwellians
};

// A particle store (one species of one discharge) is a sequence of chunks of at most CHUNK
// slots; a sweep processes one chunk per warp and writes chunk k's survivors, compacted in slot
// order, to region k of the other buffer (records [k CHUNK, (k+1) CHUNK)). The layout of a buffer
// is (K, M, D0): chunks k < K are regions, chunk k holding slots [start[k], start[k+1]) at records
// k CHUNK + (slot - start[k]), start[K] = M; chunks k >= K are the dense part, slots
// M + (k - K) CHUNK + i at records D0 + (k - K) CHUNK + i. After a sweep the regions are the last
// sweep's chunks and the dense part its newborns, copied to D0 = R0; after a load, an upload, a sort
// or a repack the buffer is dense (K = 0, M = 0, D0 = 0). Slots, and so the random streams, number
// the particles exactly as a densely compacted store would.
struct Lay {
    int K;                    // region chunks
    int pad_;
    long long M;              // slots in the regions
    long long D0;             // record offset of the dense part
};

struct Disc {
    int N, n_exc, n_pts, gas;
    uint32_t thr[2];          // null-collision candidate thresholds (of 2^32)
    uint32_t discharge_id;
    int steps_per_period;
    double dx, dt, V_rf, f_rf, w[2];
    // Poisson constants (host-computed, so the FP64 solve needs no device division):
    // r_j = pc_r[1] D_i,j - pc_r[0] D_e,j = rho_j dx^2 / eps0 inside; wall charge density
    // rho = pc_w[1] D_i - pc_w[0] D_e (half-cell volume); 1/dx, -1/(2 dx), dx/(2 eps0), 1/N
    double pc_r[2], pc_w[2], inv_dx, m_inv_2dx, hdx_eps, inv_N, inv_dt;
    const double* V0tab;      // V_rf sin(2 pi f k dt), k < steps_per_period, or null (then sin on device)
    int has_see, tile;        // sweep tile (slots) of this context
    int leapfrog, pad_lf;     // push scheme: 0 velocity Verlet (collisions at v_n), 1 leapfrog (at v_{n+1/2})
    int chunk, warps;         // compaction unit: one warp's 32 PPT slots; warps per tile
    int rec_words;            // particle record size in 16-byte words (1: FP32, 2: FP64)
    Consts<float> cf;
    Consts<double> cd;
    const void* Te;           // n_pts rows x 4 (T): cumulative sigma*v, electrons
    const void* Ti;           // n_pts rows x 2 (T): cumulative sigma*g, ions
    int32_t* c[2][2];         // [buffer][species] cell index
    void* p[2][2];            // [buffer][species] {f, vx, vy, vz} records
    long long cap[2];         // capacity per species (superparticles)
    long long rmax[2];        // regions a store may have (more: capacity error; a repack or sort resets)
    long long ralloc[2];      // regions of a buffer: rmax + the newborn chunks of one step
    long long R0[2];          // ralloc chunk: offset of the newborn (dense) area of a record buffer
    long long rcap[2];        // records per buffer: R0 + the newborn area + one chunk
    int* start[2];            // [ralloc + 1] first slot of each region chunk; start[K] = M
    int* cnt_main[2];         // [ralloc] survivors of each sweep chunk
    int* cnt_birth[2];        // [ralloc] other-species newborns of each sweep chunk
    int* cnt_same;            // [ralloc] ionization electrons of each electron-sweep chunk
    int32_t* bc[2];           // newborns of the other species, by parent species:
    void* bp[2];              //   chunk k owns records [k chunk, (k+1) chunk)
    int32_t* sc;              // ionization electrons of the electron sweep, same chunk regions
    void* sp_;
    // per slice of SLICE sweep chunks of species sp, [parity][k][3]: 0 survivors, 1 other-species
    // newborns, 2 same-species newborns. The sweep adds into parity Ctl::slice_par; k_post reads
    // it and clears the other parity for the next sweep
    unsigned* slice_tot[2];
    int slice_n[2];           // slices per parity

    long long bcap;           // births region size in the record buffers
    void* E;                  // node field for the gather (T), N+1
    double* E64;              // node field, FP64
    double* phi;              // potential, FP64
    unsigned long long* D[2]; // CIC deposits at x_{n+1}, 2^32 per particle
    unsigned long long* Q;    // electron energy moment at x_n, 2^-12 eV
    unsigned long long* Dprev;// electron deposit at x_n
    unsigned __int128* acc_D[2];    // exact sums over the accumulated steps of D, Q, D at x_n
    unsigned __int128* acc_Q;
    unsigned __int128* acc_Dprev;
    unsigned long long* cnt;  // NCNT counters
    double* period_mean;      // [PERIOD_HIST][2] mean superparticle count of every rf period
    // discharge current density J(t) at z = 0 and z = d of every step, ring of jh steps, and the
    // first-harmonic amplitude of J at z = 0 of every rf period (ring of PERIOD_HIST)
    double* J_hist;           // [jh][2]
    int jh;
    const double* jtab;       // sin, cos of 2 pi f (k + 1/2) dt, k < steps_per_period, or null
    double* J_amp;            // [PERIOD_HIST]
    double* V_hist;           // [PERIOD_HIST] rf voltage amplitude applied in every period
    // kinetic diagnostics (null until configured): node accumulators [DG_ARRAYS][N+1], sum of the
    // node field over the snapshots [N+1], EEDF counts [bins], snapshots and samples taken [2]
    unsigned long long* dg;
    double* dg_E;
    unsigned long long* dg_eedf;
    unsigned long long* dg_n;
};

// Node arrays of the kinetic diagnostics (k_diag): density, energy, particle flux, energy flux,
// ionization rate, fast electrons (snapshots), fast electrons (samples).
enum { DG_D = 0, DG_U, DG_V, DG_W, DG_K, DG_F, DG_FA, DG_ARRAYS };
enum : int { DIAG_PHASE = 1, DIAG_SAMPLE = 2, DIAG_COUNT = 4 };
constexpr unsigned DG_PHASE_MASK = 0x3Fu, DG_SAMPLE_MASK = 1u << DG_FA;

// One k_diag launch: what it takes (DIAG_* bits; DIAG_COUNT: this launch also sums the field and
// counts the snapshot or sample), the node arrays it accumulates, the EEDF bins, the fast-electron
// threshold and the inverse bin width, both in 2^-12 eV units (rounded to the particle precision
// on the device).
struct DiagArgs {
    int mode;
    unsigned mask;
    int bins;
    int pad_;
    double thr, inv_bin;
};

// Control block; one per context, in device memory.
struct Ctl {
    long long step;           // current step index n
    unsigned int tile_ctr;    // sweep tile dispenser
    unsigned int done;        // sweep CTAs finished
    unsigned int fin_done;    // k_post CTAs finished
    int error;                // ERR_* bits
    long long count[MAXD][2]; // superparticles per store
    Lay lay[MAXD][2][2];      // [discharge][species][buffer] layout of the store in that buffer
    int chunks_in[MAXD][2];   // chunks the last sweep processed, per store
    int slice_par;            // parity of the slice sums the next sweep adds into
    long long acc_steps[MAXD];
    double E0_last[MAXD];
    // J(t): electrode fields and event counters at the last solve, first-harmonic sums of the
    // current period (sin, cos)
    int have_solve[MAXD];
    double E_wall[MAXD][2];
    unsigned long long cnt_solve[MAXD][6];
    double J_sum[MAXD][2];
    // current-driven mode (Eq. adaptivevoltage): the applied amplitude is V_rf V_scale, and with
    // J_drive > 0 V_scale <- V_scale J_drive / J_calc after every rf period
    double V_scale[MAXD];
    double J_drive[MAXD];
    double period_acc[MAXD][2];   // sum of the counts over the steps of the current rf period
    unsigned sort_rows_done[MAXD][2];  // k_sort_rows CTAs finished, per store (reset by the last)
};

// Chunks of a store with layout L and count n.
__host__ __device__ inline long long chunks_of(const Lay& L, long long n, int chunk) {
    return (long long)L.K + (n - L.M + chunk - 1) / chunk;
}

constexpr int PERIOD_HIST = 1 << 16;  // rf periods of mean counts kept per discharge (ring)

struct alignas(32) d4 {
    double x, y, z, w;
};

template <typename T> struct Rec;
template <> struct Rec<float> { using type = float4; };
template <> struct Rec<double> { using type = d4; };

}  // namespace pic
