// pic_api.cu -- host runtime and C ABI (include/pic.h) of the PIC/MCC library.
// Owns device memory, the stream, the per-discharge descriptors and the step
// sequence (sweep -> finalize -> periodic sort), optionally replayed from CUDA
// graphs of one rf period.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "pic_internal.h"
#include "pic_launch.h"

using namespace pic;

#define H_E_CHARGE 1.602176634e-19
#define H_M_ELEC 9.1093837015e-31
#define H_K_BOLTZ 1.380649e-23
#define H_TWO32 4294967296.0
#define H_T_SEE_EV 2.0
#define H_EPS0 8.8541878128e-12
#define H_PI 3.14159265358979323846

struct GasDev {
    int n_pts, n_exc;
    double de, mass;
    void* Te;
    void* Ti;
    double kmax_e, kmax_i;
};

struct pic_ctx {
    int fp64 = 0;
    pic_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int n_disc = 0, n_gas = 0, max_N = 0;
    unsigned long long seed = 0;
    std::vector<pic_discharge> dis;
    std::vector<GasDev> gas;
    std::vector<pic_derived> der;
    std::vector<Disc> hd;
    Disc* d_discs = nullptr;
    Ctl* d_ctl = nullptr;
    unsigned* sort_hist = nullptr;
    unsigned* sort_tot = nullptr;
    long long* sort_hoff = nullptr;
    unsigned* sort_kr = nullptr;    // per slot of every store: cell | rank in its sort tile << 16
    long long* sort_eoff = nullptr; // first slot of each store in sort_kr
    int repack_every = 0;           // order-preserving repack after every step n with (n+1) % this == 0
    std::vector<void*> allocs;
    int cur = 0;
    long long step = 0;
    bool deposits_zero = true;
    int sweep_grid = 0, num_sms = 0;
    int max_slices = 0;  // slices of sweep chunks of the largest store
    void* stage = nullptr;  // device staging of state transfers
    size_t stage_bytes = 0;
    void* h_pin = nullptr;  // pinned host scratch for read-backs (one stream sync per call)
    size_t h_pin_bytes = 0;
    std::string err;
    pic_counters cnt_at_reset[MAXD];
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    size_t ev_used = 0;
    // one-period graphs, keyed by (buffer parity at entry, step phase within the sort period)
    struct GraphEntry {
        int cur_in, phase, cur_out;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
    // kinetic diagnostics (pic_set_diagnostics): configuration, device allocations, whether both
    // schedules repeat every rf period (then periods may run as graphs)
    bool dg_on = false, dg_periodic = true;
    pic_diag_config dg{};
    std::vector<void*> dg_allocs;
};

static pic_status fail(pic_ctx* c, pic_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

static pic_status cuda_fail(pic_ctx* c, cudaError_t e, const char* what) {
    return fail(c, PIC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

static void* dalloc(pic_ctx* ctx, size_t bytes, cudaError_t* e) {
    void* p = nullptr;
    *e = cudaMalloc(&p, bytes ? bytes : 16);
    if (*e != cudaSuccess) return nullptr;
    ctx->allocs.push_back(p);
    *e = cudaMemsetAsync(p, 0, bytes ? bytes : 16, ctx->stream);
    return p;
}

extern "C" void pic_default_options(pic_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = PIC_FP32;
    o->sort_every = 0;
    o->block = 256;
    o->ppt = 4;
    o->ctas_per_sm = 0;
    o->use_graph = 0;
    o->cuda_stream = nullptr;
    o->load = 1;
}

extern "C" const char* pic_status_string(pic_status s) {
    switch (s) {
        case PIC_OK: return "ok";
        case PIC_ERR_ARG: return "invalid argument";
        case PIC_ERR_CUDA: return "CUDA error";
        case PIC_ERR_CAPACITY: return "particle capacity exceeded";
        case PIC_ERR_TIMEOUT: return "device wait timed out";
        case PIC_ERR_TABLE: return "cross-section table rejected";
        case PIC_ERR_NONFINITE: return "non-finite particle state";
        case PIC_ERR_STATE: return "invalid call in current state";
    }
    return "unknown";
}

extern "C" const char* pic_last_error(const pic_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

static uint32_t null_threshold(double numax, double dt, double* pnull) {
    const double P = -expm1(-numax * dt);
    *pnull = P;
    double t = floor(P * H_TWO32);
    if (t < 0.0) t = 0.0;
    if (t > 4294967295.0) t = 4294967295.0;
    return (uint32_t)t;
}

// Host FP64 derivation of the per-discharge constants (same expressions in the
// documented order, so that the rounded values are reproducible).
static void derive(const pic_discharge& d, const GasDev& g, const pic_gas& gi, pic_derived* o) {
    const double M = g.mass, de = g.de, dt = d.dt_s;
    o->dx = d.gap_m / (double)d.n_cells;
    o->n_gas = d.p_Pa / (H_K_BOLTZ * d.T_gas_K);
    o->K_e = (-H_E_CHARGE / H_M_ELEC) * (0.5 * dt);
    o->K_i = (H_E_CHARGE / M) * (0.5 * dt);
    o->dtdx = dt / o->dx;
    o->kappa_e = 0.5 * H_M_ELEC / (H_E_CHARGE * de);
    o->kappa_i = 0.25 * M / (H_E_CHARGE * de);
    o->kappa_E = 0.5 * H_M_ELEC / H_E_CHARGE * 4096.0;
    o->beta_e = H_M_ELEC / (H_M_ELEC + M);
    o->omb_e = M / (H_M_ELEC + M);
    for (int j = 0; j < 2; ++j) o->de2_exc[j] = 2.0 * H_E_CHARGE * (j < gi.n_exc ? gi.eps_exc_eV[j] : 0.0) / H_M_ELEC;
    o->de2_iz = 2.0 * H_E_CHARGE * gi.eps_iz_eV / H_M_ELEC;
    o->sig_n = sqrt(H_K_BOLTZ * d.T_gas_K / M);
    o->sig_e0 = sqrt(H_E_CHARGE * d.weights.T_e0_eV / H_M_ELEC);
    o->sig_i0 = sqrt(H_K_BOLTZ * d.weights.T_i0_K / M);
    o->sig_see = sqrt(H_E_CHARGE * H_T_SEE_EV / H_M_ELEC);
    o->sig_see_n = sqrt(2.0 * H_E_CHARGE * H_T_SEE_EV / H_M_ELEC);
    o->kmax_e = g.kmax_e;
    o->kmax_i = g.kmax_i;
    o->numax_e = o->n_gas * o->kmax_e;
    o->numax_i = o->n_gas * o->kmax_i;
    o->thr_e = null_threshold(o->numax_e, dt, &o->pnull_e);
    o->thr_i = null_threshold(o->numax_i, dt, &o->pnull_i);
}

template <typename T>
static void fill_consts(Consts<T>& k, const pic_derived& o, const pic_discharge& d) {
    k.K[0] = (T)o.K_e;
    k.K[1] = (T)o.K_i;
    k.dtdx = (T)o.dtdx;
    k.kappa_e = (T)o.kappa_e;
    k.kappa_i = (T)o.kappa_i;
    k.kappa_E = (T)o.kappa_E;
    k.beta = (T)o.beta_e;
    k.omb = (T)o.omb_e;
    k.de2_exc[0] = (T)o.de2_exc[0];
    k.de2_exc[1] = (T)o.de2_exc[1];
    k.de2_iz = (T)o.de2_iz;
    k.sig_n = (T)o.sig_n;
    k.sig_see = (T)o.sig_see;
    k.sig_see_n = (T)o.sig_see_n;
    k.kmax_e = (T)o.kmax_e;
    k.kmax_i = (T)o.kmax_i;
    k.gamma = (T)d.weights.gamma_see;
    k.sig0[0] = (T)o.sig_e0;
    k.sig0[1] = (T)o.sig_i0;
}

// Region bookkeeping of a store of capacity cap (superparticles) with sweep chunks of `chunk` slots
// and a newborn area of bcap records: a store may hold rmax regions (a quarter more than a dense
// store of cap particles needs, and 64), the output area has room for the newborn chunks of one step
// beyond that, and a layout never has more than maxchunks chunks.
struct RegionSizes {
    long long rmax, bchunks, ralloc, R0, rcap, maxchunks;
};
static RegionSizes region_sizes(long long cap, long long chunk, long long bcap) {
    RegionSizes r;
    r.rmax = (cap + chunk - 1) / chunk + (cap + 4 * chunk - 1) / (4 * chunk) + 64;
    r.bchunks = (bcap + chunk - 1) / chunk + 1;
    r.ralloc = r.rmax + r.bchunks;
    r.R0 = r.ralloc * chunk;
    r.rcap = r.R0 + r.bchunks * chunk + chunk;
    r.maxchunks = r.ralloc + r.bchunks;
    return r;
}

extern "C" void pic_destroy(pic_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    for (auto& e : ctx->ev) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    for (void* p : ctx->allocs) cudaFree(p);
    for (void* p : ctx->dg_allocs) cudaFree(p);
    if (ctx->stage) cudaFree(ctx->stage);
    if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

static pic_status enqueue_sweep(pic_ctx* ctx);
static pic_status enqueue_finalize(pic_ctx* ctx, int mode);
static pic_status enqueue_sort(pic_ctx* ctx);

extern "C" pic_status pic_batch_create(pic_ctx** out, const pic_gas* gases, int32_t n_gases,
                                       const pic_discharge* dis, int32_t n_dis, uint64_t seed,
                                       const pic_options* opt) {
    if (!out) return PIC_ERR_ARG;
    *out = nullptr;
    if (!gases || !dis || n_gases < 1 || n_dis < 1 || n_dis > MAXD) return PIC_ERR_ARG;
    pic_ctx* ctx = new pic_ctx();
    if (opt) ctx->opt = *opt;
    else pic_default_options(&ctx->opt);
    pic_options& o = ctx->opt;
    if (o.block != 128 && o.block != 256 && o.block != 512) o.block = 256;
    if (o.block == 512 && o.ppt == 8) o.ppt = 4;
    if (o.ppt != 2 && o.ppt != 4 && o.ppt != 8) o.ppt = 4;
    if (o.precision != PIC_FP32 && o.precision != PIC_FP64) {
        pic_destroy(ctx);
        return PIC_ERR_ARG;
    }
    ctx->fp64 = o.precision == PIC_FP64;
    ctx->seed = seed;
    ctx->n_disc = n_dis;
    ctx->n_gas = n_gases;
    const size_t rsz = ctx->fp64 ? sizeof(double) : sizeof(float);
    // validation
    for (int i = 0; i < n_gases; ++i) {
        const pic_gas& g = gases[i];
        if (g.n_exc < 1 || g.n_exc > 2 || g.n_pts < 2 || g.n_pts > (1 << 24) || !(g.de_eV > 0) ||
            !(g.mass_kg > 0) || !g.sigma_e || !g.sigma_i) {
            pic_destroy(ctx);
            return PIC_ERR_ARG;
        }
        const size_t ne = (size_t)g.n_pts * (2 + g.n_exc), ni = (size_t)g.n_pts * 2;
        for (size_t k = 0; k < ne; ++k)
            if (!(g.sigma_e[k] >= 0.0) || !std::isfinite(g.sigma_e[k])) {
                pic_destroy(ctx);
                return PIC_ERR_TABLE;
            }
        for (size_t k = 0; k < ni; ++k)
            if (!(g.sigma_i[k] >= 0.0) || !std::isfinite(g.sigma_i[k])) {
                pic_destroy(ctx);
                return PIC_ERR_TABLE;
            }
    }
    for (int i = 0; i < n_dis; ++i) {
        const pic_discharge& d = dis[i];
        const pic_weights& w = d.weights;
        if (d.gas < 0 || d.gas >= n_gases || d.n_cells < 1 || d.n_cells > MAXN || !(d.gap_m > 0) || !(d.dt_s > 0) ||
            !(d.p_Pa >= 0) || !(d.T_gas_K > 0) || w.n_e0 < 0 || w.n_i0 < 0 || w.capacity_e < w.n_e0 ||
            w.capacity_i < w.n_i0 || w.capacity_e > (1ll << 30) - 1 || w.capacity_i > (1ll << 30) - 1 ||
            !(w.gamma_see >= 0 && w.gamma_see <= 1)) {
            pic_destroy(ctx);
            return PIC_ERR_ARG;
        }
        ctx->max_N = std::max(ctx->max_N, d.n_cells);
        ctx->dis.push_back(d);
    }
    // stream
    if (o.cuda_stream) {
        ctx->stream = (cudaStream_t)o.cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            pic_status s = cuda_fail(ctx, e, "stream");
            pic_destroy(ctx);
            return s;
        }
        ctx->own_stream = true;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t ce;
#define ALLOC(ptr, type, bytes)                                          \
    do {                                                                 \
        ptr = (type)dalloc(ctx, (bytes), &ce);                           \
        if (ce != cudaSuccess) {                                         \
            pic_status s_ = cuda_fail(ctx, ce, "allocation");            \
            std::string m_ = ctx->err;                                   \
            pic_destroy(ctx);                                            \
            (void)m_;                                                    \
            return s_;                                                   \
        }                                                                \
    } while (0)

    // tables per gas
    for (int i = 0; i < n_gases; ++i) {
        const pic_gas& g = gases[i];
        GasDev gd{};
        gd.n_pts = g.n_pts;
        gd.n_exc = g.n_exc;
        gd.de = g.de_eV;
        gd.mass = g.mass_kg;
        const size_t ne = (size_t)g.n_pts * (2 + g.n_exc), ni = (size_t)g.n_pts * 2;
        double *se = nullptr, *si = nullptr;
        unsigned long long* km = nullptr;
        if (cudaMalloc(&se, ne * 8) != cudaSuccess || cudaMalloc(&si, ni * 8) != cudaSuccess ||
            cudaMalloc(&km, 16) != cudaSuccess) {
            cudaFree(se);
            cudaFree(si);
            pic_destroy(ctx);
            return PIC_ERR_CUDA;
        }
        cudaMemcpyAsync(se, g.sigma_e, ne * 8, cudaMemcpyHostToDevice, ctx->stream);
        cudaMemcpyAsync(si, g.sigma_i, ni * 8, cudaMemcpyHostToDevice, ctx->stream);
        cudaMemsetAsync(km, 0, 16, ctx->stream);
        ALLOC(gd.Te, void*, (size_t)g.n_pts * 4 * rsz);
        ALLOC(gd.Ti, void*, (size_t)g.n_pts * 2 * rsz);
        ce = launch_tables(ctx->fp64, g.n_pts, 2 + g.n_exc, g.de_eV, g.mass_kg, se, si, gd.Te, gd.Ti, km,
                           ctx->stream);
        unsigned long long kmh[2] = {0, 0};
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(kmh, km, 16, cudaMemcpyDeviceToHost, ctx->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
        cudaFree(se);
        cudaFree(si);
        cudaFree(km);
        if (ce != cudaSuccess) {
            pic_status s = cuda_fail(ctx, ce, "tables");
            pic_destroy(ctx);
            return s;
        }
        std::memcpy(&gd.kmax_e, &kmh[0], 8);
        std::memcpy(&gd.kmax_i, &kmh[1], 8);
        ctx->gas.push_back(gd);
    }

    const long long tile = (long long)o.block * o.ppt;
    const long long chunk = 32ll * o.ppt;
    auto bcap_of = [&](int i) {
        return std::max(ctx->dis[i].weights.capacity_e, ctx->dis[i].weights.capacity_i) / 8 + 4096;
    };
    // sort scratch: per store (cells x sort tiles) counts
    {
        std::vector<long long> hoff(2 * MAXD, 0);
        long long acc = 0;
        const long long st = sort_tile_chunks((int)chunk);
        for (int i = 0; i < n_dis; ++i)
            for (int sp = 0; sp < 2; ++sp) {
                hoff[2 * i + sp] = acc;
                const long long cap = sp ? ctx->dis[i].weights.capacity_i : ctx->dis[i].weights.capacity_e;
                const RegionSizes rs = region_sizes(cap, chunk, bcap_of(i));
                acc += (long long)ctx->dis[i].n_cells * ((rs.maxchunks + st - 1) / st + 1);
            }
        ALLOC(ctx->sort_hist, unsigned*, sizeof(unsigned) * (size_t)std::max(acc, 1ll));
        ALLOC(ctx->sort_tot, unsigned*, sizeof(unsigned) * (size_t)(2 * MAXD) * MAXN);
        ALLOC(ctx->sort_hoff, long long*, sizeof(long long) * 2 * MAXD);
        cudaMemcpyAsync(ctx->sort_hoff, hoff.data(), sizeof(long long) * 2 * MAXD, cudaMemcpyHostToDevice,
                        ctx->stream);
        std::vector<long long> eoff(2 * MAXD, 0);
        long long ea = 0;
        for (int i = 0; i < n_dis; ++i)
            for (int sp = 0; sp < 2; ++sp) {
                eoff[2 * i + sp] = ea;
                ea += sp ? ctx->dis[i].weights.capacity_i : ctx->dis[i].weights.capacity_e;
            }
        ALLOC(ctx->sort_kr, unsigned*, sizeof(unsigned) * (size_t)std::max(ea, 1ll));
        ALLOC(ctx->sort_eoff, long long*, sizeof(long long) * 2 * MAXD);
        cudaMemcpyAsync(ctx->sort_eoff, eoff.data(), sizeof(long long) * 2 * MAXD, cudaMemcpyHostToDevice,
                        ctx->stream);
    }

    // per-discharge buffers and descriptors
    for (int i = 0; i < n_dis; ++i) {
        const pic_discharge& d = ctx->dis[i];
        const GasDev& g = ctx->gas[d.gas];
        pic_derived der{};
        derive(d, g, gases[d.gas], &der);
        ctx->der.push_back(der);
        Disc D{};
        D.N = d.n_cells;
        D.n_exc = g.n_exc;
        D.n_pts = g.n_pts;
        D.gas = d.gas;
        D.thr[0] = der.thr_e;
        D.thr[1] = der.thr_i;
        D.discharge_id = d.discharge_id;
        D.steps_per_period = d.weights.steps_per_period;
        D.dx = der.dx;
        D.dt = d.dt_s;
        D.V_rf = d.V_rf_V;
        D.f_rf = d.f_rf_Hz;
        D.w[0] = d.weights.w_e;
        D.w[1] = d.weights.w_i;
        for (int sp = 0; sp < 2; ++sp) {
            D.pc_r[sp] = H_E_CHARGE * D.w[sp] * der.dx / (H_TWO32 * H_EPS0);
            D.pc_w[sp] = H_E_CHARGE * D.w[sp] / (H_TWO32 * 0.5 * der.dx);
        }
        D.inv_dx = 1.0 / der.dx;
        D.m_inv_2dx = -1.0 / (2.0 * der.dx);
        D.hdx_eps = der.dx / (2.0 * H_EPS0);
        D.inv_N = 1.0 / (double)d.n_cells;
        D.inv_dt = 1.0 / d.dt_s;
        D.V0tab = nullptr;
        D.jtab = nullptr;
        {
            // one rf period of V(t) when dt divides it (f dt steps_per_period = 1 to 1e-12)
            const int spp = d.weights.steps_per_period;
            if (spp > 0 && std::fabs(d.f_rf_Hz * d.dt_s * spp - 1.0) <= 1e-12) {
                std::vector<double> v((size_t)spp);
                for (int k = 0; k < spp; ++k)
                    v[(size_t)k] = d.V_rf_V * std::sin(2.0 * H_PI * d.f_rf_Hz * ((double)k * d.dt_s));
                double* dv = nullptr;
                ALLOC(dv, double*, sizeof(double) * (size_t)spp);
                if (cudaMemcpy(dv, v.data(), sizeof(double) * (size_t)spp, cudaMemcpyHostToDevice) != cudaSuccess) {
                    pic_status s_ = fail(ctx, PIC_ERR_CUDA, "voltage table");
                    pic_destroy(ctx);
                    return s_;
                }
                D.V0tab = dv;
                // sin and cos at the step midpoints (first harmonic of J(t))
                std::vector<double> jt(2 * (size_t)spp);
                for (int k = 0; k < spp; ++k) {
                    const double ph = 2.0 * H_PI * d.f_rf_Hz * (((double)k + 0.5) * d.dt_s);
                    jt[2 * (size_t)k] = std::sin(ph);
                    jt[2 * (size_t)k + 1] = std::cos(ph);
                }
                double* dj = nullptr;
                ALLOC(dj, double*, sizeof(double) * 2 * (size_t)spp);
                if (cudaMemcpy(dj, jt.data(), sizeof(double) * 2 * (size_t)spp, cudaMemcpyHostToDevice) !=
                    cudaSuccess) {
                    pic_status s_ = fail(ctx, PIC_ERR_CUDA, "current table");
                    pic_destroy(ctx);
                    return s_;
                }
                D.jtab = dj;
            }
        }
        D.jh = d.weights.steps_per_period > 0 ? 4 * d.weights.steps_per_period : 4096;
        ALLOC(D.J_hist, double*, sizeof(double) * 2 * (size_t)D.jh);
        ALLOC(D.J_amp, double*, sizeof(double) * PERIOD_HIST);
        ALLOC(D.V_hist, double*, sizeof(double) * PERIOD_HIST);
        D.has_see = d.weights.gamma_see > 0.0;
        D.leapfrog = o.leapfrog != 0;
        D.tile = (int)tile;
        D.chunk = 32 * o.ppt;
        D.warps = o.block / 32;
        D.rec_words = ctx->fp64 ? 2 : 1;
        fill_consts<float>(D.cf, der, d);
        fill_consts<double>(D.cd, der, d);
        D.Te = g.Te;
        D.Ti = g.Ti;
        D.cap[0] = d.weights.capacity_e;
        D.cap[1] = d.weights.capacity_i;
        D.bcap = bcap_of(i);
        const size_t rec = 4 * rsz;
        for (int sp = 0; sp < 2; ++sp) {
            // record buffers: one region per sweep chunk, then the newborn area
            const RegionSizes rs = region_sizes(D.cap[sp], chunk, D.bcap);
            D.rmax[sp] = rs.rmax;
            D.ralloc[sp] = rs.ralloc;
            D.R0[sp] = rs.R0;
            D.rcap[sp] = rs.rcap;
            if (D.rcap[sp] > 0x7FFFFFF0ll) {
                pic_status s_ = fail(ctx, PIC_ERR_ARG, "capacity too large for 32-bit record offsets");
                pic_destroy(ctx);
                return s_;
            }
        }
        for (int b = 0; b < 2; ++b)
            for (int sp = 0; sp < 2; ++sp) {
                ALLOC(D.c[b][sp], int32_t*, sizeof(int32_t) * (size_t)(D.rcap[sp] + 16));
                ALLOC(D.p[b][sp], void*, rec * (size_t)(D.rcap[sp] + 16));
            }
        for (int sp = 0; sp < 2; ++sp) {
            const size_t mc = (size_t)D.ralloc[sp], nrec = mc * (size_t)chunk;
            ALLOC(D.bc[sp], int32_t*, sizeof(int32_t) * (nrec + 16));
            ALLOC(D.bp[sp], void*, rec * (nrec + 16));
            ALLOC(D.start[sp], int*, sizeof(int) * (mc + 2));
            ALLOC(D.cnt_main[sp], int*, sizeof(int) * (mc + 1));
            ALLOC(D.cnt_birth[sp], int*, sizeof(int) * (mc + 1));
            const size_t ns = (mc + SLICE - 1) / SLICE + 1;
            ctx->max_slices = std::max(ctx->max_slices, (int)ns);
            D.slice_n[sp] = (int)ns;
            ALLOC(D.slice_tot[sp], unsigned*, sizeof(unsigned) * 2 * 3 * ns);  // two parities
            if (cudaMemset(D.slice_tot[sp], 0, sizeof(unsigned) * 2 * 3 * ns) != cudaSuccess) {
                pic_status s_ = fail(ctx, PIC_ERR_CUDA, "slice sums");
                pic_destroy(ctx);
                return s_;
            }
            if (sp == 0) {
                ALLOC(D.sc, int32_t*, sizeof(int32_t) * (nrec + 16));
                ALLOC(D.sp_, void*, rec * (nrec + 16));
                ALLOC(D.cnt_same, int*, sizeof(int) * (mc + 1));
            }
        }
        const size_t N1 = (size_t)d.n_cells + 1;
        ALLOC(D.E, void*, rsz * N1);
        ALLOC(D.E64, double*, 8 * N1);
        ALLOC(D.phi, double*, 8 * N1);
        ALLOC(D.D[0], unsigned long long*, 8 * N1);
        ALLOC(D.D[1], unsigned long long*, 8 * N1);
        ALLOC(D.Q, unsigned long long*, 8 * N1);
        ALLOC(D.Dprev, unsigned long long*, 8 * N1);
        // the four exact accumulators in one block (read back by one copy)
        ALLOC(D.acc_D[0], unsigned __int128*, 4 * 16 * N1);
        D.acc_D[1] = D.acc_D[0] + N1;
        D.acc_Q = D.acc_D[0] + 2 * N1;
        D.acc_Dprev = D.acc_D[0] + 3 * N1;
        ALLOC(D.cnt, unsigned long long*, 8 * NCNT);
        ALLOC(D.period_mean, double*, sizeof(double) * 2 * PERIOD_HIST);
        ctx->hd.push_back(D);
        std::memset(&ctx->cnt_at_reset[i], 0, sizeof(pic_counters));
    }
    ALLOC(ctx->d_discs, Disc*, sizeof(Disc) * n_dis);
    ALLOC(ctx->d_ctl, Ctl*, sizeof(Ctl));
#undef ALLOC
    cudaMemcpyAsync(ctx->d_discs, ctx->hd.data(), sizeof(Disc) * n_dis, cudaMemcpyHostToDevice, ctx->stream);
    {
        Ctl h{};
        for (int i = 0; i < n_dis; ++i) {
            h.count[i][0] = o.load ? ctx->dis[i].weights.n_e0 : 0;
            h.count[i][1] = o.load ? ctx->dis[i].weights.n_i0 : 0;
            h.V_scale[i] = 1.0;
            h.J_drive[i] = 0.0;
        }
        cudaMemcpyAsync(ctx->d_ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream);
        ce = launch_set_dense(ctx->d_discs, n_dis, ctx->d_ctl, 0, ctx->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
        if (ce != cudaSuccess) {
            pic_status s = cuda_fail(ctx, ce, "store set-up");
            pic_destroy(ctx);
            return s;
        }
    }
    // sweep grid: persistent CTAs
    {
        int occ = sweep_occupancy(ctx->fp64, o.block, o.ppt, ctx->max_N, n_dis);
        if (occ < 1) occ = 1;
        int per = o.ctas_per_sm > 0 ? std::min(o.ctas_per_sm, occ) : occ;
        ctx->sweep_grid = std::max(1, ctx->num_sms * per);
    }
    if (o.load) {
        const int gx = std::max(1, ctx->num_sms * 4);
        ce = launch_load(ctx->fp64, ctx->d_discs, n_dis, ctx->d_ctl, 0, seed, gx, ctx->stream);
        if (ce == cudaSuccess) ce = launch_deposit(ctx->fp64, ctx->d_discs, n_dis, ctx->d_ctl, 0, ctx->max_N, gx,
                                                   ctx->stream);
        if (ce == cudaSuccess) ce = launch_finalize(ctx->fp64, ctx->d_discs, n_dis, ctx->d_ctl, 0, 4, 0, ctx->max_N, ctx->stream);
        if (ce == cudaSuccess) ce = launch_backkick(ctx->fp64, ctx->d_discs, n_dis, ctx->d_ctl, 0, gx, ctx->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
        if (ce != cudaSuccess) {
            pic_status s = cuda_fail(ctx, ce, "initial load");
            pic_destroy(ctx);
            return s;
        }
    }
    ctx->cur = 0;
    ctx->step = 0;
    ctx->deposits_zero = true;
    // Sweeps append regions (one per chunk, plus the newborns' chunks); a sort makes a store dense
    // again. When it runs rarer than every 64 steps, an order-preserving repack does, every R steps
    // with R the largest divisor of the rf period up to 64 (so that one-period graphs stay periodic).
    {
        const int K = o.sort_every, P = ctx->dis[0].weights.steps_per_period;
        ctx->repack_every = 0;
        if (!(K > 0 && K <= 64)) {
            int R = 64;
            if (P > 0)
                for (R = std::min(P, 64); P % R != 0; --R) {
                }
            ctx->repack_every = R;
        }
    }
    *out = ctx;
    return PIC_OK;
}

extern "C" pic_status pic_create(pic_ctx** out, const pic_gas* gas, double gap_m, double p_Pa, double T_gas_K,
                                 double f_rf_Hz, double V_rf_V, int32_t n_cells, double dt_s,
                                 const pic_weights* weights, uint64_t seed, const pic_options* opt) {
    if (!gas || !weights) return PIC_ERR_ARG;
    pic_discharge d{};
    d.gas = 0;
    d.n_cells = n_cells;
    d.gap_m = gap_m;
    d.p_Pa = p_Pa;
    d.T_gas_K = T_gas_K;
    d.f_rf_Hz = f_rf_Hz;
    d.V_rf_V = V_rf_V;
    d.dt_s = dt_s;
    d.weights = *weights;
    d.discharge_id = 0;
    return pic_batch_create(out, gas, 1, &d, 1, seed, opt);
}

// ---------------------------------------------------------------------------
static pic_status enqueue_sweep(pic_ctx* ctx) {
    if (!ctx->deposits_zero) {
        for (auto& D : ctx->hd) {
            const size_t b = 8 * ((size_t)D.N + 1);
            CK(cudaMemsetAsync(D.D[0], 0, b, ctx->stream), "memset");
            CK(cudaMemsetAsync(D.D[1], 0, b, ctx->stream), "memset");
            CK(cudaMemsetAsync(D.Q, 0, b, ctx->stream), "memset");
        }
    }
    SweepLaunch L{};
    L.fp64 = ctx->fp64;
    L.block = ctx->opt.block;
    L.ppt = ctx->opt.ppt;
    L.grid = ctx->sweep_grid;
    L.max_N = ctx->max_N;
    L.n_disc = ctx->n_disc;
    L.in_buf = ctx->cur;
    L.discs = ctx->d_discs;
    L.ctl = ctx->d_ctl;
    L.seed = ctx->seed;
    L.stream = ctx->stream;
    std::pair<cudaEvent_t, cudaEvent_t>* evp = nullptr;
    if (ctx->timing) {
        if (ctx->ev_used == ctx->ev.size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            ctx->ev.push_back({a, b});
        }
        evp = &ctx->ev[ctx->ev_used++];
        cudaEventRecord(evp->first, ctx->stream);
    }
    CK(launch_sweep(L), "sweep launch");
    if (evp) cudaEventRecord(evp->second, ctx->stream);
    ctx->deposits_zero = false;
    return PIC_OK;
}

static pic_status enqueue_finalize(pic_ctx* ctx, int mode) {
    CK(launch_finalize(ctx->fp64, ctx->d_discs, ctx->n_disc, ctx->d_ctl, mode & 1 ? 1 - ctx->cur : ctx->cur, mode,
                       ctx->max_slices, ctx->max_N, ctx->stream),
       "finalize launch");
    if (mode & 1) ctx->cur = 1 - ctx->cur;
    if (mode & 2) ctx->step += 1;
    ctx->deposits_zero = true;
    return PIC_OK;
}

static pic_status enqueue_sort(pic_ctx* ctx) {
    const int gx = std::max(1, ctx->num_sms * 2);
    CK(launch_sort(ctx->fp64, ctx->d_discs, ctx->n_disc, ctx->d_ctl, ctx->cur, 1 - ctx->cur, ctx->sort_hist,
                   ctx->sort_hoff, ctx->sort_tot, ctx->sort_kr, ctx->sort_eoff, ctx->max_N, gx,
                   ctx->stream),
       "sort launch");
    ctx->cur = 1 - ctx->cur;
    return PIC_OK;
}

static pic_status enqueue_repack(pic_ctx* ctx) {
    const int gx = std::max(1, ctx->num_sms * 4);
    CK(launch_repack(ctx->fp64, ctx->d_discs, ctx->n_disc, ctx->d_ctl, ctx->cur, 1 - ctx->cur, gx, ctx->stream),
       "repack launch");
    ctx->cur = 1 - ctx->cur;
    return PIC_OK;
}

// Diagnostics of step n = ctx->step, before its sweep, when the schedules ask for them: one k_diag
// launch, or two when the node arrays of the snapshot do not fit the shared memory together.
static pic_status enqueue_diag(pic_ctx* ctx) {
    const pic_diag_config& g = ctx->dg;
    const long long n = ctx->step;
    const bool phase = g.period_steps > 0 && n % g.period_steps == g.phase_step;
    const bool sample = g.sample_every > 0 && n % g.sample_every == 0;
    if (!phase && !sample) return PIC_OK;
    unsigned left = (phase ? DG_PHASE_MASK : 0u) | (sample ? DG_SAMPLE_MASK : 0u);
    constexpr size_t budget = 200 * 1024;
    bool first = true;
    while (left) {
        DiagArgs A{};
        A.mode = first ? (phase ? DIAG_PHASE : 0) | (sample ? DIAG_SAMPLE : 0) | DIAG_COUNT : 0;
        A.bins = g.eedf_bins;
        A.thr = g.fast_eV * 4096.0;
        A.inv_bin = 1.0 / (g.eedf_de_eV * 4096.0);
        const int bins = (A.mode & DIAG_SAMPLE) ? g.eedf_bins : 0;
        for (int a = 0; a < DG_ARRAYS; ++a) {
            const unsigned bit = 1u << a;
            if ((left & bit) && (A.mask == 0 || diag_smem(ctx->max_N, A.mask | bit, bins) <= budget)) A.mask |= bit;
        }
        left &= ~A.mask;
        const size_t smem = diag_smem(ctx->max_N, A.mask, bins);
        const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (220 * 1024) / std::max<size_t>(smem, 1)));
        CK(launch_diag(ctx->fp64, ctx->d_discs, ctx->n_disc, ctx->d_ctl, ctx->cur, A, ctx->max_N,
                       std::max(1, ctx->num_sms * per_sm), ctx->stream),
           "diagnostics launch");
        first = false;
    }
    return PIC_OK;
}

// Sweep + births + solve: the sweep reads buffer cur and writes 1-cur; the
// finalize appends births into 1-cur; cur flips. Then the sort, or the repack, when due.
static pic_status enqueue_step(pic_ctx* ctx) {
    if (ctx->dg_on) {
        pic_status s0 = enqueue_diag(ctx);
        if (s0 != PIC_OK) return s0;
    }
    pic_status s = enqueue_sweep(ctx);
    if (s != PIC_OK) return s;
    s = enqueue_finalize(ctx, 3);
    if (s != PIC_OK) return s;
    const int K = ctx->opt.sort_every;
    if (K > 0 && ctx->step % K == 0) return enqueue_sort(ctx);
    if (ctx->repack_every > 0 && ctx->step % ctx->repack_every == 0) return enqueue_repack(ctx);
    return PIC_OK;
}

static pic_status run_graph_period(pic_ctx* ctx, int P) {
    // the period's sorts and repacks follow from the step at which it starts
    const int phase = (int)(ctx->step % P);
    for (auto& g : ctx->graphs)
        if (g.cur_in == ctx->cur && g.phase == phase) {
            CK(cudaGraphLaunch(g.exec, ctx->stream), "graph launch");
            ctx->cur = g.cur_out;
            ctx->step += P;
            ctx->deposits_zero = true;
            return PIC_OK;
        }
    // capture one period
    const int cur0 = ctx->cur;
    const long long step0 = ctx->step;
    const bool timing = ctx->timing;
    ctx->timing = false;
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    pic_status s = PIC_OK;
    for (int i = 0; i < P && s == PIC_OK; ++i) s = enqueue_step(ctx);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    ctx->timing = timing;
    if (s != PIC_OK) return s;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
    pic_ctx::GraphEntry ge{cur0, phase, ctx->cur, exec};
    ctx->graphs.push_back(ge);
    ctx->cur = cur0;
    ctx->step = step0;
    CK(cudaGraphLaunch(exec, ctx->stream), "graph launch");
    ctx->cur = ge.cur_out;
    ctx->step = step0 + P;
    ctx->deposits_zero = true;
    return PIC_OK;
}

extern "C" pic_status pic_step(pic_ctx* ctx, int64_t n_steps) {
    if (!ctx || n_steps < 0) return PIC_ERR_ARG;
    const int P = ctx->dis[0].weights.steps_per_period;
    const int K = ctx->opt.sort_every;
    const bool graphs = ctx->opt.use_graph && P > 0 && (K <= 0 || P % K == 0) && !ctx->timing &&
                        (!ctx->dg_on || ctx->dg_periodic);
    int64_t left = n_steps;
    while (left > 0) {
        if (graphs && left >= P) {
            pic_status s = run_graph_period(ctx, P);
            if (s != PIC_OK) return s;
            left -= P;
            continue;
        }
        pic_status s = enqueue_step(ctx);
        if (s != PIC_OK) return s;
        --left;
    }
    return PIC_OK;
}

extern "C" pic_status pic_sweep(pic_ctx* ctx) {
    if (!ctx) return PIC_ERR_ARG;
    pic_status s = enqueue_sweep(ctx);
    if (s != PIC_OK) return s;
    // births appended and counts updated; no solve, no step advance
    CK(launch_finalize(ctx->fp64, ctx->d_discs, ctx->n_disc, ctx->d_ctl, 1 - ctx->cur, 1 | 8, ctx->max_slices,
                       ctx->max_N, ctx->stream),
       "append launch");
    ctx->cur = 1 - ctx->cur;
    return PIC_OK;
}

extern "C" pic_status pic_sort(pic_ctx* ctx) {
    if (!ctx) return PIC_ERR_ARG;
    return enqueue_sort(ctx);
}

extern "C" pic_status pic_solve(pic_ctx* ctx) {
    if (!ctx) return PIC_ERR_ARG;
    return enqueue_finalize(ctx, 2);
}

extern "C" pic_status pic_sync(pic_ctx* ctx) {
    if (!ctx) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    int err = 0;
    CK(cudaMemcpy(&err, &ctx->d_ctl->error, sizeof(int), cudaMemcpyDeviceToHost), "error word");
    if (err & ERR_TIMEOUT) return fail(ctx, PIC_ERR_TIMEOUT, "a bounded device-side wait timed out");
    if (err & ERR_CAPACITY) return fail(ctx, PIC_ERR_CAPACITY, "particle or birth buffer capacity exceeded");
    if (err & ERR_NONFINITE) return fail(ctx, PIC_ERR_NONFINITE, "non-finite particle coordinate");
    return PIC_OK;
}

// ---------------------------------------------------------------------------
static bool bad_d(pic_ctx* ctx, int d) { return !ctx || d < 0 || d >= ctx->n_disc; }

// Pinned host scratch of at least `bytes` for read-backs: device -> host copies into it are
// queued on the context's stream and waited for with one synchronisation.
static pic_status pinned(pic_ctx* ctx, size_t bytes) {
    if (ctx->h_pin_bytes >= bytes) return PIC_OK;
    bytes = std::max(bytes, (size_t)1 << 16);
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
    ctx->h_pin = nullptr;
    ctx->h_pin_bytes = 0;
    CK(cudaMallocHost(&ctx->h_pin, bytes), "pinned scratch");
    ctx->h_pin_bytes = bytes;
    return PIC_OK;
}

extern "C" pic_status pic_get_count(pic_ctx* ctx, int32_t d, int32_t sp, int64_t* n) {
    if (bad_d(ctx, d) || (sp & ~1) || !n) return PIC_ERR_ARG;
    pic_status s = pinned(ctx, 64);
    if (s != PIC_OK) return s;
    long long* v = static_cast<long long*>(ctx->h_pin);
    CK(cudaMemcpyAsync(v, &ctx->d_ctl->count[d][sp], 8, cudaMemcpyDeviceToHost, ctx->stream), "count");
    CK(cudaStreamSynchronize(ctx->stream), "count");
    *n = *v;
    return PIC_OK;
}

// Device staging for state transfers (cells, then four real arrays), grown on demand.
static size_t pad16(size_t b) { return (b + 15) / 16 * 16; }

// Device staging of a state transfer: the cells and the four real arrays, each starting on a
// 16-byte boundary (the pack / unpack kernels then move whole 16-byte groups), and an error word.
static pic_status staging(pic_ctx* ctx, long long n) {
    const size_t r = ctx->fp64 ? 8 : 4;
    const size_t need = pad16((size_t)n * 4) + 4 * pad16((size_t)n * r) + 64;
    if (ctx->stage_bytes >= need) return PIC_OK;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    if (ctx->stage) cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    CK(cudaMalloc(&ctx->stage, need), "staging");
    ctx->stage_bytes = need;
    return PIC_OK;
}

// The device address of host memory the GPU can reach directly (pinned and mapped, e.g. from
// cudaHostAlloc or a registered buffer), or null (pageable memory, or a null pointer). State
// transfers with such buffers let the pack / unpack kernels read or write them over the host link
// instead of going through device staging and copies (measured: the link runs at the same rate
// either way, so this saves the staging pass and the per-array copies).
static void* mapped(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // not a CUDA pointer: clear the error, take the staged path
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

extern "C" pic_status pic_get_state(pic_ctx* ctx, int32_t d, int32_t sp, int64_t cap, int32_t* c, void* f,
                                    void* vx, void* vy, void* vz, int64_t* n_out) {
    if (bad_d(ctx, d) || (sp & ~1) || cap < 0) return PIC_ERR_ARG;
    void* hm[5] = {c, f, vx, vy, vz};
    bool direct = true;
    for (int q = 0; q < 5; ++q)
        if (hm[q]) {
            hm[q] = mapped(hm[q]);
            direct = direct && hm[q] != nullptr;
        }
    if (direct) {  // every requested array mapped: the unpack kernel writes the caller's arrays
        // directly, taking the count on the device; one synchronisation for the count
        pic_status s = pinned(ctx, 64);
        if (s != PIC_OK) return s;
        long long* hn = static_cast<long long*>(ctx->h_pin);
        const int grid = std::max(1, (int)std::min<long long>(ctx->num_sms * 8, (cap + 255) / 256));
        void* const v[4] = {hm[1], hm[2], hm[3], hm[4]};
        CK(launch_unpack_state(ctx->fp64, ctx->d_discs, ctx->d_ctl, d, sp, ctx->cur, cap,
                               static_cast<int32_t*>(hm[0]), v, grid, ctx->stream),
           "state gather");
        CK(cudaMemcpyAsync(hn, &ctx->d_ctl->count[d][sp], 8, cudaMemcpyDeviceToHost, ctx->stream), "count");
        CK(cudaStreamSynchronize(ctx->stream), "state copy");
        if (n_out) *n_out = *hn;
        if (*hn > cap) return fail(ctx, PIC_ERR_ARG, "host buffer too small");
        return PIC_OK;
    }
    int64_t n = 0;
    pic_status s = pic_get_count(ctx, d, sp, &n);
    if (s != PIC_OK) return s;
    if (n_out) *n_out = n;
    if (n > cap) return fail(ctx, PIC_ERR_ARG, "host buffer too small");
    if (n == 0) return PIC_OK;
    const int grid = std::max(1, std::min(ctx->num_sms * 8, (int)((n + 255) / 256)));
    s = staging(ctx, n);
    if (s != PIC_OK) return s;
    const size_t r = ctx->fp64 ? 8 : 4;
    int32_t* sc = static_cast<int32_t*>(ctx->stage);
    unsigned char* sv = static_cast<unsigned char*>(ctx->stage) + pad16((size_t)n * 4);
    const size_t sr = pad16((size_t)n * r);
    {
        void* const v[4] = {sv, sv + sr, sv + 2 * sr, sv + 3 * sr};
        CK(launch_unpack_state(ctx->fp64, ctx->d_discs, ctx->d_ctl, d, sp, ctx->cur, n, sc, v, grid, ctx->stream),
           "state gather");
    }
    if (c) CK(cudaMemcpyAsync(c, sc, 4 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream), "state c");
    void* outs[4] = {f, vx, vy, vz};
    for (int q = 0; q < 4; ++q)
        if (outs[q]) CK(cudaMemcpyAsync(outs[q], sv + q * sr, r * (size_t)n, cudaMemcpyDeviceToHost,
                                        ctx->stream), "state p");
    CK(cudaStreamSynchronize(ctx->stream), "state copy");
    return PIC_OK;
}

extern "C" pic_status pic_set_state(pic_ctx* ctx, int32_t d, int32_t sp, int64_t n, const int32_t* c,
                                    const void* f, const void* vx, const void* vy, const void* vz) {
    if (bad_d(ctx, d) || (sp & ~1) || n < 0 || (n && (!c || !f || !vx || !vy || !vz))) return PIC_ERR_ARG;
    const Disc& D = ctx->hd[d];
    if (n > D.cap[sp]) return fail(ctx, PIC_ERR_CAPACITY, "state larger than capacity");
    const size_t r = ctx->fp64 ? 8 : 4;
    pic_status s = staging(ctx, n > 0 ? n : 1);
    if (s != PIC_OK) return s;
    int32_t* sc = static_cast<int32_t*>(ctx->stage);
    unsigned char* sv = static_cast<unsigned char*>(ctx->stage) + pad16((size_t)n * 4);
    const size_t sr = pad16((size_t)n * r);
    unsigned* bad = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(ctx->stage) + ctx->stage_bytes - 64);
    CK(cudaMemsetAsync(bad, 0, sizeof(unsigned), ctx->stream), "state check");
    if (n) {
        const int grid = std::max(1, std::min(ctx->num_sms * 8, (int)((n + 255) / 256)));
        const void* hm[5] = {mapped(c), mapped(f), mapped(vx), mapped(vy), mapped(vz)};
        if (hm[0] && hm[1] && hm[2] && hm[3] && hm[4]) {  // mapped: the pack kernel reads them directly
            const void* const v[4] = {hm[1], hm[2], hm[3], hm[4]};
            CK(launch_pack_state(ctx->fp64, ctx->d_discs, d, sp, ctx->cur, n, static_cast<const int32_t*>(hm[0]), v,
                                 bad, grid, ctx->stream),
               "state pack");
        } else {
            CK(cudaMemcpyAsync(sc, c, 4 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream), "state c");
            const void* ins[4] = {f, vx, vy, vz};
            for (int q = 0; q < 4; ++q)
                CK(cudaMemcpyAsync(sv + q * sr, ins[q], r * (size_t)n, cudaMemcpyHostToDevice,
                                   ctx->stream),
                   "state p");
            const void* const v[4] = {sv, sv + sr, sv + 2 * sr, sv + 3 * sr};
            CK(launch_pack_state(ctx->fp64, ctx->d_discs, d, sp, ctx->cur, n, sc, v, bad, grid, ctx->stream),
               "state pack");
        }
    }
    // count and dense layout on the device (a rejected upload leaves an empty store), then one
    // synchronisation for the check word
    CK(launch_finish_upload(ctx->d_discs, ctx->d_ctl, d, sp, n, bad, ctx->cur, ctx->stream), "state finish");
    s = pinned(ctx, 64);
    if (s != PIC_OK) return s;
    unsigned* hbad = static_cast<unsigned*>(ctx->h_pin);
    CK(cudaMemcpyAsync(hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream), "state check");
    CK(cudaStreamSynchronize(ctx->stream), "state copy");
    if (*hbad) return fail(ctx, PIC_ERR_ARG, "cell index out of range");
    return PIC_OK;
}

extern "C" pic_status pic_get_field(pic_ctx* ctx, int32_t d, void* E, double* E64, double* phi) {
    if (bad_d(ctx, d)) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    const Disc& D = ctx->hd[d];
    const size_t N1 = (size_t)D.N + 1, r = ctx->fp64 ? 8 : 4;
    if (E) CK(cudaMemcpy(E, D.E, r * N1, cudaMemcpyDeviceToHost), "field");
    if (E64) CK(cudaMemcpy(E64, D.E64, 8 * N1, cudaMemcpyDeviceToHost), "field64");
    if (phi) CK(cudaMemcpy(phi, D.phi, 8 * N1, cudaMemcpyDeviceToHost), "phi");
    return PIC_OK;
}

extern "C" pic_status pic_set_field(pic_ctx* ctx, int32_t d, const void* E) {
    if (bad_d(ctx, d) || !E) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    const Disc& D = ctx->hd[d];
    CK(cudaMemcpy(D.E, E, (ctx->fp64 ? 8 : 4) * ((size_t)D.N + 1), cudaMemcpyHostToDevice), "field");
    return PIC_OK;
}

extern "C" pic_status pic_get_deposit(pic_ctx* ctx, int32_t d, int32_t sp, int64_t* Dh) {
    if (bad_d(ctx, d) || (sp & ~1) || !Dh) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    const Disc& D = ctx->hd[d];
    CK(cudaMemcpy(Dh, D.D[sp], 8 * ((size_t)D.N + 1), cudaMemcpyDeviceToHost), "deposit");
    return PIC_OK;
}

extern "C" pic_status pic_set_deposit(pic_ctx* ctx, int32_t d, int32_t sp, const int64_t* Dh) {
    if (bad_d(ctx, d) || (sp & ~1) || !Dh) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    const Disc& D = ctx->hd[d];
    CK(cudaMemcpy(D.D[sp], Dh, 8 * ((size_t)D.N + 1), cudaMemcpyHostToDevice), "deposit");
    ctx->deposits_zero = false;
    return PIC_OK;
}

extern "C" pic_status pic_get_energy_deposit(pic_ctx* ctx, int32_t d, int64_t* Q) {
    if (bad_d(ctx, d) || !Q) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    const Disc& D = ctx->hd[d];
    CK(cudaMemcpy(Q, D.Q, 8 * ((size_t)D.N + 1), cudaMemcpyDeviceToHost), "energy deposit");
    return PIC_OK;
}

extern "C" pic_status pic_get_step(pic_ctx* ctx, int64_t* step) {
    if (!ctx || !step) return PIC_ERR_ARG;
    *step = ctx->step;
    return PIC_OK;
}

extern "C" pic_status pic_set_step(pic_ctx* ctx, int64_t step) {
    if (!ctx || step < 0) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    long long v = step;
    CK(cudaMemcpy(&ctx->d_ctl->step, &v, 8, cudaMemcpyHostToDevice), "step");
    ctx->step = step;
    return PIC_OK;
}

static void parse_counters(const unsigned long long* c, pic_counters* o) {
    std::memset(o, 0, sizeof(*o));
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) o->absorbed[a][b] = (int64_t)c[CNT_ABS + 2 * a + b];
    for (int j = 0; j < 4; ++j) o->collisions_e[j] = (int64_t)c[CNT_COLL_E + j];
    for (int j = 0; j < 2; ++j) o->collisions_i[j] = (int64_t)c[CNT_COLL_I + j];
    o->null_inelastic = (int64_t)c[CNT_NULL_INEL];
    o->see_emitted = (int64_t)c[CNT_SEE];
    o->candidates[0] = (int64_t)c[CNT_CAND];
    o->candidates[1] = (int64_t)c[CNT_CAND + 1];
    o->table_clamped[0] = (int64_t)c[CNT_CLAMP];
    o->table_clamped[1] = (int64_t)c[CNT_CLAMP + 1];
}
static pic_status read_counters(pic_ctx* ctx, int d, pic_counters* o) {
    pic_status s = pinned(ctx, 8 * NCNT);
    if (s != PIC_OK) return s;
    unsigned long long* c = static_cast<unsigned long long*>(ctx->h_pin);
    CK(cudaMemcpyAsync(c, ctx->hd[d].cnt, 8 * NCNT, cudaMemcpyDeviceToHost, ctx->stream), "counters");
    CK(cudaStreamSynchronize(ctx->stream), "counters");
    parse_counters(c, o);
    return PIC_OK;
}

extern "C" pic_status pic_get_counters(pic_ctx* ctx, int32_t d, pic_counters* out) {
    if (bad_d(ctx, d) || !out) return PIC_ERR_ARG;
    return read_counters(ctx, d, out);
}

extern "C" pic_status pic_get_derived(pic_ctx* ctx, int32_t d, pic_derived* out) {
    if (bad_d(ctx, d) || !out) return PIC_ERR_ARG;
    *out = ctx->der[d];
    return PIC_OK;
}

extern "C" pic_status pic_get_tables(pic_ctx* ctx, int32_t g, void* Te, void* Ti) {
    if (!ctx || g < 0 || g >= ctx->n_gas) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    const GasDev& G = ctx->gas[g];
    const size_t r = ctx->fp64 ? 8 : 4;
    if (Te) CK(cudaMemcpy(Te, G.Te, (size_t)G.n_pts * 4 * r, cudaMemcpyDeviceToHost), "tables");
    if (Ti) CK(cudaMemcpy(Ti, G.Ti, (size_t)G.n_pts * 2 * r, cudaMemcpyDeviceToHost), "tables");
    return PIC_OK;
}

// Copies ring entries first .. first+n-1 (ring of len entries of bytes each) to host memory, in at
// most two contiguous copies.
static cudaError_t ring_copy(void* dst, const void* ring, long long first, long long n, long long len, size_t bytes) {
    const long long a = first % len, n1 = std::min(n, len - a);
    const unsigned char* r = static_cast<const unsigned char*>(ring);
    unsigned char* o = static_cast<unsigned char*>(dst);
    cudaError_t e = n1 > 0 ? cudaMemcpy(o, r + a * bytes, (size_t)n1 * bytes, cudaMemcpyDeviceToHost) : cudaSuccess;
    if (e == cudaSuccess && n > n1) e = cudaMemcpy(o + n1 * bytes, r, (size_t)(n - n1) * bytes, cudaMemcpyDeviceToHost);
    return e;
}

extern "C" pic_status pic_moments(pic_ctx* ctx, int32_t d, pic_moments_t* out) {
    if (bad_d(ctx, d) || !out) return PIC_ERR_ARG;
    const Disc& D = ctx->hd[d];
    const int N = D.N;
    const size_t N1 = (size_t)N + 1;
    // every read-back of the call into pinned memory, one synchronisation: the four exact
    // accumulators (one block), the control block, the counters, the last J(t) and the last
    // period's current amplitude
    const size_t acc = 16 * N1, o_ctl = 4 * acc, o_cnt = o_ctl + ((sizeof(Ctl) + 15) / 16) * 16;
    const size_t o_j = o_cnt + 8 * NCNT;
    pic_status s = pinned(ctx, o_j + 3 * sizeof(double));
    if (s != PIC_OK) return s;
    unsigned char* h = static_cast<unsigned char*>(ctx->h_pin);
    const int spp = ctx->dis[d].weights.steps_per_period;
    const long long done = spp > 0 ? ctx->step / spp : 0;
    double* hj = reinterpret_cast<double*>(h + o_j);
    hj[0] = hj[1] = hj[2] = 0.0;
    CK(cudaMemcpyAsync(h, D.acc_D[0], 4 * acc, cudaMemcpyDeviceToHost, ctx->stream), "moments");
    CK(cudaMemcpyAsync(h + o_ctl, ctx->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream), "moments");
    CK(cudaMemcpyAsync(h + o_cnt, D.cnt, 8 * NCNT, cudaMemcpyDeviceToHost, ctx->stream), "moments");
    if (ctx->step > 0) {
        CK(cudaMemcpyAsync(hj, D.J_hist + 2 * ((ctx->step - 1) % D.jh), 2 * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream), "current");
        if (done > 0 && D.jtab)
            CK(cudaMemcpyAsync(hj + 2, D.J_amp + (done - 1) % PERIOD_HIST, sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream), "current amplitude");
    }
    CK(cudaStreamSynchronize(ctx->stream), "moments");
    const Ctl& hc = *reinterpret_cast<const Ctl*>(h + o_ctl);
    if (hc.error & ERR_TIMEOUT) return fail(ctx, PIC_ERR_TIMEOUT, "a bounded device-side wait timed out");
    if (hc.error & ERR_CAPACITY) return fail(ctx, PIC_ERR_CAPACITY, "particle or birth buffer capacity exceeded");
    if (hc.error & ERR_NONFINITE) return fail(ctx, PIC_ERR_NONFINITE, "non-finite particle coordinate");
    const unsigned __int128* iD0 = reinterpret_cast<const unsigned __int128*>(h);
    const unsigned __int128* iD1 = reinterpret_cast<const unsigned __int128*>(h + acc);
    const unsigned __int128* iQ = reinterpret_cast<const unsigned __int128*>(h + 2 * acc);
    const unsigned __int128* iP = reinterpret_cast<const unsigned __int128*>(h + 3 * acc);
    const long long steps = hc.acc_steps[d];
    const double dx = D.dx, ns = steps > 0 ? (double)steps : 1.0;
    for (int j = 0; j <= N; ++j) {
        const double Vj = (j == 0 || j == N) ? 0.5 * dx : dx;
        const double aD0 = (double)iD0[j], aD1 = (double)iD1[j], aQ = (double)iQ[j], aP = (double)iP[j];
        if (out->n_e) out->n_e[j] = D.w[0] * aD0 / (H_TWO32 * Vj * ns);
        if (out->n_i) out->n_i[j] = D.w[1] * aD1 / (H_TWO32 * Vj * ns);
        if (out->mean_eps) out->mean_eps[j] = aP > 0.0 ? (aQ / 4096.0) / (aP / H_TWO32) : 0.0;
    }
    pic_counters c;
    parse_counters(reinterpret_cast<const unsigned long long*>(h + o_cnt), &c);
    out->steps = steps;
    out->count[0] = hc.count[d][0];
    out->count[1] = hc.count[d][1];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            out->absorbed[a][b] = (double)(c.absorbed[a][b] - ctx->cnt_at_reset[d].absorbed[a][b]);
            out->flux[a][b] = steps > 0 ? out->absorbed[a][b] * D.w[a] / ((double)steps * D.dt) : 0.0;
        }
    out->surface_charge = 8.8541878128e-12 * hc.E0_last[d];
    // rf periods, the steady-state criterion on the per-period mean counts, J(t)
    out->periods_done = done;
    out->steady_period = -1;
    out->steady_metric = -1.0;
    out->steady = 0;
    out->reserved = 0;
    out->J_last = hj[0];
    out->J_amp = hj[2];
    const long long keep = std::min(done, (long long)PERIOD_HIST);
    if (keep >= 2 * PIC_STEADY_BLOCK) {
        std::vector<double> pm(2 * (size_t)keep);
        CK(ring_copy(pm.data(), D.period_mean, done - keep, keep, PERIOD_HIST, 2 * sizeof(double)),
           "period counts");  // oldest kept period first
        std::vector<double> cum(2 * (size_t)(keep + 1), 0.0);
        for (long long k = 0; k < keep; ++k)
            for (int sp = 0; sp < 2; ++sp) cum[2 * (k + 1) + sp] = cum[2 * k + sp] + pm[2 * k + sp];
        const int W = PIC_STEADY_BLOCK;
        for (long long k = 2 * W; k <= keep; ++k) {
            double metric = 0.0;
            bool pos = true;
            for (int sp = 0; sp < 2; ++sp) {
                const double a = (cum[2 * k + sp] - cum[2 * (k - W) + sp]) / W;
                const double b = (cum[2 * (k - W) + sp] - cum[2 * (k - 2 * W) + sp]) / W;
                if (!(a > 0)) pos = false;
                else metric = std::max(metric, std::fabs(a - b) / a);
            }
            if (!pos) metric = INFINITY;
            if (k == keep) out->steady_metric = metric;
            if (out->steady_period < 0 && metric < PIC_STEADY_TOL) out->steady_period = done - keep + k;
        }
        out->steady = out->steady_period >= 0;
    }
    return PIC_OK;
}

extern "C" pic_status pic_current(pic_ctx* ctx, int32_t d, int64_t first, int64_t n, double* out,
                                  int64_t* steps_done) {
    if (bad_d(ctx, d) || first < 0 || n < 0 || (n && !out)) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    const Disc& D = ctx->hd[d];
    if (steps_done) *steps_done = ctx->step;
    if (first + n > ctx->step || ctx->step - first > D.jh) return fail(ctx, PIC_ERR_ARG, "steps not available");
    CK(ring_copy(out, D.J_hist, first, n, D.jh, 2 * sizeof(double)), "current");
    return PIC_OK;
}

extern "C" pic_status pic_current_amplitude(pic_ctx* ctx, int32_t d, int64_t first, int64_t n, double* out,
                                            int64_t* periods_done) {
    if (bad_d(ctx, d) || first < 0 || n < 0 || (n && !out)) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    const Disc& D = ctx->hd[d];
    const int spp = ctx->dis[d].weights.steps_per_period;
    const long long done = spp > 0 ? ctx->step / spp : 0;
    if (periods_done) *periods_done = done;
    if (!D.jtab && n > 0) return fail(ctx, PIC_ERR_STATE, "the time step does not divide the rf period");
    if (first + n > done || done - first > PERIOD_HIST) return fail(ctx, PIC_ERR_ARG, "periods not available");
    CK(ring_copy(out, D.J_amp, first, n, PERIOD_HIST, sizeof(double)), "current amplitude");
    return PIC_OK;
}

extern "C" pic_status pic_set_current_drive(pic_ctx* ctx, int32_t d, double J0) {
    if (bad_d(ctx, d) || !(J0 >= 0.0) || !std::isfinite(J0)) return PIC_ERR_ARG;
    if (!ctx->hd[d].jtab) return fail(ctx, PIC_ERR_STATE, "the time step does not divide the rf period");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    CK(cudaMemcpy(&ctx->d_ctl->J_drive[d], &J0, sizeof(double), cudaMemcpyHostToDevice), "current drive");
    return PIC_OK;
}

extern "C" pic_status pic_voltage_amplitude(pic_ctx* ctx, int32_t d, int64_t first, int64_t n, double* out,
                                            int64_t* periods_done, double* V0_now) {
    if (bad_d(ctx, d) || first < 0 || n < 0 || (n && !out)) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    const Disc& D = ctx->hd[d];
    const int spp = ctx->dis[d].weights.steps_per_period;
    const long long done = spp > 0 ? ctx->step / spp : 0;
    if (periods_done) *periods_done = done;
    if (V0_now) {
        double s = 1.0;
        CK(cudaMemcpy(&s, &ctx->d_ctl->V_scale[d], sizeof(double), cudaMemcpyDeviceToHost), "voltage");
        *V0_now = D.V_rf * s;
    }
    if (!D.jtab && n > 0) return fail(ctx, PIC_ERR_STATE, "the time step does not divide the rf period");
    if (first + n > done || done - first > PERIOD_HIST) return fail(ctx, PIC_ERR_ARG, "periods not available");
    CK(ring_copy(out, D.V_hist, first, n, PERIOD_HIST, sizeof(double)), "voltage amplitude");
    return PIC_OK;
}

extern "C" pic_status pic_reset_moments(pic_ctx* ctx) {
    if (!ctx) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    for (int d = 0; d < ctx->n_disc; ++d) {
        const Disc& D = ctx->hd[d];
        const size_t b = 16 * ((size_t)D.N + 1);
        CK(cudaMemset(D.acc_D[0], 0, 4 * b), "reset");  // the four accumulators, one block
        long long z = 0;
        CK(cudaMemcpy(&ctx->d_ctl->acc_steps[d], &z, 8, cudaMemcpyHostToDevice), "reset");
        pic_status s = read_counters(ctx, d, &ctx->cnt_at_reset[d]);
        if (s != PIC_OK) return s;
    }
    return PIC_OK;
}

// ---------------------------------------------------------------------------
// Kinetic diagnostics.
static void drop_graphs(pic_ctx* ctx) {
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
}

extern "C" pic_status pic_set_diagnostics(pic_ctx* ctx, const pic_diag_config* cfg) {
    if (!ctx) return PIC_ERR_ARG;
    if (cfg && (cfg->period_steps < 0 || cfg->sample_every < 0 || cfg->eedf_bins < 1 ||
                cfg->eedf_bins > PIC_DIAG_MAX_BINS || !(cfg->eedf_de_eV > 0) || !(cfg->fast_eV >= 0) ||
                !std::isfinite(cfg->eedf_de_eV) || !std::isfinite(cfg->fast_eV) ||
                (cfg->period_steps > 0 && (cfg->phase_step < 0 || cfg->phase_step >= cfg->period_steps))))
        return fail(ctx, PIC_ERR_ARG, "diagnostics configuration out of range");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(ctx->stream, &cs), "capture status");
    if (cs != cudaStreamCaptureStatusNone) return fail(ctx, PIC_ERR_STATE, "diagnostics configured during a capture");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    drop_graphs(ctx);  // their steps were captured with the old schedule
    for (void* p : ctx->dg_allocs) cudaFree(p);
    ctx->dg_allocs.clear();
    ctx->dg_on = false;
    for (auto& D : ctx->hd) D.dg = nullptr, D.dg_E = nullptr, D.dg_eedf = nullptr, D.dg_n = nullptr;
    if (cfg) {
        for (auto& D : ctx->hd) {
            const size_t N1 = (size_t)D.N + 1;
            void* p[4] = {nullptr, nullptr, nullptr, nullptr};
            const size_t bytes[4] = {8 * N1 * DG_ARRAYS, 8 * N1, 8 * (size_t)cfg->eedf_bins, 16};
            for (int q = 0; q < 4; ++q) {
                CK(cudaMalloc(&p[q], bytes[q]), "diagnostics allocation");
                ctx->dg_allocs.push_back(p[q]);
                CK(cudaMemsetAsync(p[q], 0, bytes[q], ctx->stream), "diagnostics clear");
            }
            D.dg = static_cast<unsigned long long*>(p[0]);
            D.dg_E = static_cast<double*>(p[1]);
            D.dg_eedf = static_cast<unsigned long long*>(p[2]);
            D.dg_n = static_cast<unsigned long long*>(p[3]);
        }
        ctx->dg = *cfg;
        const int P = ctx->dis[0].weights.steps_per_period;
        ctx->dg_periodic = P > 0 && (cfg->period_steps == 0 || P % cfg->period_steps == 0) &&
                           (cfg->sample_every == 0 || P % cfg->sample_every == 0);
    }
    CK(cudaMemcpyAsync(ctx->d_discs, ctx->hd.data(), sizeof(Disc) * ctx->n_disc, cudaMemcpyHostToDevice, ctx->stream),
       "descriptor upload");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    ctx->dg_on = cfg != nullptr;
    return PIC_OK;
}

extern "C" pic_status pic_reset_diagnostics(pic_ctx* ctx) {
    if (!ctx) return PIC_ERR_ARG;
    if (!ctx->dg_on) return fail(ctx, PIC_ERR_STATE, "diagnostics not configured");
    for (auto& D : ctx->hd) {
        const size_t N1 = (size_t)D.N + 1;
        CK(cudaMemsetAsync(D.dg, 0, 8 * N1 * DG_ARRAYS, ctx->stream), "diagnostics clear");
        CK(cudaMemsetAsync(D.dg_E, 0, 8 * N1, ctx->stream), "diagnostics clear");
        CK(cudaMemsetAsync(D.dg_eedf, 0, 8 * (size_t)ctx->dg.eedf_bins, ctx->stream), "diagnostics clear");
        CK(cudaMemsetAsync(D.dg_n, 0, 16, ctx->stream), "diagnostics clear");
    }
    return PIC_OK;
}

extern "C" pic_status pic_diagnostics(pic_ctx* ctx, int32_t d, double* E, double* n_e, double* mean_eps,
                                      double* gamma_e, double* q_e, double* heating, double* ion_rate,
                                      double* n_fast, double* n_fast_avg, double* eedf, int64_t* snapshots,
                                      int64_t* samples) {
    if (bad_d(ctx, d)) return PIC_ERR_ARG;
    if (!ctx->dg_on) return fail(ctx, PIC_ERR_STATE, "diagnostics not configured");
    const Disc& D = ctx->hd[d];
    const int N = D.N, bins = ctx->dg.eedf_bins;
    const size_t N1 = (size_t)N + 1;
    const size_t o_E = 8 * N1 * DG_ARRAYS, o_h = o_E + 8 * N1, o_n = o_h + 8 * (size_t)bins;
    pic_status s = pinned(ctx, o_n + 16);
    if (s != PIC_OK) return s;
    unsigned char* h = static_cast<unsigned char*>(ctx->h_pin);
    CK(cudaMemcpyAsync(h, D.dg, o_E, cudaMemcpyDeviceToHost, ctx->stream), "diagnostics");
    CK(cudaMemcpyAsync(h + o_E, D.dg_E, 8 * N1, cudaMemcpyDeviceToHost, ctx->stream), "diagnostics");
    CK(cudaMemcpyAsync(h + o_h, D.dg_eedf, 8 * (size_t)bins, cudaMemcpyDeviceToHost, ctx->stream), "diagnostics");
    CK(cudaMemcpyAsync(h + o_n, D.dg_n, 16, cudaMemcpyDeviceToHost, ctx->stream), "diagnostics");
    CK(cudaStreamSynchronize(ctx->stream), "diagnostics");
    const long long* A = reinterpret_cast<const long long*>(h);  // exact sums, two's complement
    const long long *aD = A + DG_D * N1, *aU = A + DG_U * N1, *aV = A + DG_V * N1, *aW = A + DG_W * N1,
                    *aK = A + DG_K * N1, *aF = A + DG_F * N1, *aFa = A + DG_FA * N1;
    const double* sE = reinterpret_cast<const double*>(h + o_E);
    const unsigned long long* hb = reinterpret_cast<const unsigned long long*>(h + o_h);
    const unsigned long long* cnt = reinterpret_cast<const unsigned long long*>(h + o_n);
    const double dx = D.dx, w = D.w[0], n_gas = ctx->der[d].n_gas;
    const double ns = cnt[0] > 0 ? (double)cnt[0] : 1.0, nm = cnt[1] > 0 ? (double)cnt[1] : 1.0;
    for (int j = 0; j <= N; ++j) {
        const double Vj = (j == 0 || j == N) ? 0.5 * dx : dx;
        const double Ej = sE[j] / ns;
        const double g = w * (double)aV[j] / 64.0 / (Vj * ns);
        if (E) E[j] = Ej;
        if (n_e) n_e[j] = w * (double)aD[j] / (H_TWO32 * Vj * ns);
        if (mean_eps) mean_eps[j] = aD[j] > 0 ? ((double)aU[j] / 4096.0) / ((double)aD[j] / H_TWO32) : 0.0;
        if (gamma_e) gamma_e[j] = g;
        if (q_e) q_e[j] = w * H_E_CHARGE * (double)aW[j] * 16.0 / (Vj * ns);
        if (heating) heating[j] = -H_E_CHARGE * Ej * g;
        if (ion_rate) ion_rate[j] = n_gas * w * (double)aK[j] * 0x1p-72 / (Vj * ns);
        if (n_fast) n_fast[j] = w * (double)aF[j] / (H_TWO32 * Vj * ns);
        if (n_fast_avg) n_fast_avg[j] = w * (double)aFa[j] / (H_TWO32 * Vj * nm);
    }
    if (eedf) {
        double tot = 0.0;
        for (int b = 0; b < bins; ++b) tot += (double)hb[b];
        for (int b = 0; b < bins; ++b) {
            const double U = (b + 0.5) * ctx->dg.eedf_de_eV;
            eedf[b] = tot > 0 ? (double)hb[b] / (tot * ctx->dg.eedf_de_eV * std::sqrt(U)) : 0.0;
        }
    }
    if (snapshots) *snapshots = (int64_t)cnt[0];
    if (samples) *samples = (int64_t)cnt[1];
    return PIC_OK;
}

extern "C" pic_status pic_sweep_timing(pic_ctx* ctx, int32_t enable, double* total_ms, int64_t* launches) {
    if (!ctx) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    double tot = 0.0;
    for (size_t i = 0; i < ctx->ev_used; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev[i].first, ctx->ev[i].second);
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = (int64_t)ctx->ev_used;
    ctx->ev_used = 0;
    ctx->timing = enable != 0;
    return PIC_OK;
}

// ---------------------------------------------------------------------------
extern "C" pic_status pic_debug_philox(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out) {
    if (n < 0 || (n && (!ctr || !key || !out))) return PIC_ERR_ARG;
    if (!n) return PIC_OK;
    uint32_t *dc = nullptr, *dout = nullptr;
    if (cudaMalloc(&dc, 16 * n) != cudaSuccess || cudaMalloc(&dout, 16 * n) != cudaSuccess) {
        cudaFree(dc);
        return PIC_ERR_CUDA;
    }
    cudaMemcpy(dc, ctr, 16 * n, cudaMemcpyHostToDevice);
    cudaError_t e = launch_debug_philox(n, dc, key[0], key[1], dout, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 16 * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dout);
    return e == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}

extern "C" pic_status pic_debug_wait(int32_t arrive, int32_t tries) {
    if (tries < 1 || tries > (1 << 20)) return PIC_ERR_ARG;
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return PIC_ERR_CUDA;
    int h = -1;
    cudaError_t e = cudaMemset(d, 0xFF, sizeof(int));
    if (e == cudaSuccess) e = launch_debug_wait(arrive ? 1 : 0, tries, d, 0);
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return PIC_ERR_CUDA;
    return h == 0 ? PIC_OK : h == ERR_TIMEOUT ? PIC_ERR_TIMEOUT : PIC_ERR_CUDA;
}

extern "C" pic_status pic_debug_math(int64_t n, const float* x, const float* y, float* lg, float* sn, float* cs) {
    if (n < 0 || (n && (!x || !y || !lg || !sn || !cs))) return PIC_ERR_ARG;
    if (!n) return PIC_OK;
    float* b = nullptr;
    if (cudaMalloc(&b, 20 * n) != cudaSuccess) return PIC_ERR_CUDA;
    cudaMemcpy(b, x, 4 * n, cudaMemcpyHostToDevice);
    cudaMemcpy(b + n, y, 4 * n, cudaMemcpyHostToDevice);
    cudaError_t e = launch_debug_math(n, b, b + n, b + 2 * n, b + 3 * n, b + 4 * n, 0);
    if (e == cudaSuccess) e = cudaMemcpy(lg, b + 2 * n, 4 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(sn, b + 3 * n, 4 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(cs, b + 4 * n, 4 * n, cudaMemcpyDeviceToHost);
    cudaFree(b);
    return e == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}

extern "C" pic_status pic_period_counts(pic_ctx* ctx, int32_t d, int64_t first, int64_t n, double* out,
                                        int64_t* periods_done) {
    if (bad_d(ctx, d) || first < 0 || n < 0 || (n && !out)) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    const int spp = ctx->dis[d].weights.steps_per_period;
    const long long done = spp > 0 ? ctx->step / spp : 0;
    if (periods_done) *periods_done = done;
    if (first + n > done || done - first > PERIOD_HIST) return fail(ctx, PIC_ERR_ARG, "periods not available");
    for (long long k = 0; k < n; ++k) {
        const long long slot = (first + k) % PERIOD_HIST;
        CK(cudaMemcpy(out + 2 * k, ctx->hd[d].period_mean + 2 * slot, 2 * sizeof(double), cudaMemcpyDeviceToHost),
           "period counts");
    }
    return PIC_OK;
}

// Warm start (see include/pic.h): profiles[d][3][n_pts] = n_e, n_i (m^-3), mean electron energy (eV).
extern "C" pic_status pic_load_profiles(pic_ctx* ctx, int32_t n_pts, const double* profiles) {
    if (!ctx || n_pts < 2 || !profiles) return PIC_ERR_ARG;
    if (ctx->step != 0) return fail(ctx, PIC_ERR_STATE, "profiles can only be loaded before the first step");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    const int P = n_pts, nd = ctx->n_disc;
    const size_t r = ctx->fp64 ? 8 : 4;
    std::vector<unsigned char> host((size_t)nd * 3 * P * r);
    std::vector<long long> counts((size_t)nd * 2);
    for (int d = 0; d < nd; ++d) {
        const double* pr = profiles + (size_t)d * 3 * P;
        const double dz = ctx->dis[d].gap_m / (double)(P - 1);
        for (int sp = 0; sp < 2; ++sp) {
            const double* prof = pr + (size_t)sp * P;
            const double w = sp == 0 ? ctx->dis[d].weights.w_e : ctx->dis[d].weights.w_i;
            double A = 0.0;
            for (int j = 0; j + 1 < P; ++j) {
                const double a = 0.5 * (std::fmax(prof[j], 0.0) + std::fmax(prof[j + 1], 0.0)) * dz;
                A += a;
            }
            const long long n = A > 0.0 ? (long long)std::floor(A / w + 0.5) : 0;
            const long long cap = sp == 0 ? ctx->dis[d].weights.capacity_e : ctx->dis[d].weights.capacity_i;
            if (n > cap) return fail(ctx, PIC_ERR_CAPACITY, "profile integral exceeds the store capacity");
            counts[2 * d + sp] = n;
            double run = 0.0;
            unsigned char* out = host.data() + ((size_t)d * 3 + sp) * P * r;
            for (int j = 0; j < P; ++j) {
                double v;
                if (j == 0) v = 0.0;
                else if (j == P - 1) v = 1.0;
                else {
                    run += 0.5 * (std::fmax(prof[j - 1], 0.0) + std::fmax(prof[j], 0.0)) * dz;
                    v = A > 0.0 ? run / A : 0.0;
                }
                if (ctx->fp64) std::memcpy(out + j * r, &v, 8);
                else {
                    const float fv = (float)v;
                    std::memcpy(out + j * r, &fv, 4);
                }
            }
        }
        unsigned char* out = host.data() + ((size_t)d * 3 + 2) * P * r;
        for (int j = 0; j < P; ++j) {
            const double v = std::fmax(pr[2 * (size_t)P + j], 0.0);
            if (ctx->fp64) std::memcpy(out + j * r, &v, 8);
            else {
                const float fv = (float)v;
                std::memcpy(out + j * r, &fv, 4);
            }
        }
    }
    void* dtab = nullptr;
    void* ddesc = nullptr;
    const size_t dsz = warm_desc_bytes(ctx->fp64);
    if (cudaMalloc(&dtab, host.size()) != cudaSuccess || cudaMalloc(&ddesc, dsz * nd) != cudaSuccess) {
        cudaFree(dtab);
        return fail(ctx, PIC_ERR_CUDA, "warm-start tables");
    }
    std::vector<unsigned char> desc(dsz * nd);
    const double K23 = 2.0 * H_E_CHARGE / (3.0 * H_M_ELEC);
    for (int d = 0; d < nd; ++d) {
        unsigned char* base = (unsigned char*)dtab + (size_t)d * 3 * P * r;
        warm_desc_fill(ctx->fp64, desc.data() + dsz * d, base, base + P * r, base + 2 * P * r, P,
                       (double)ctx->dis[d].n_cells / (double)(P - 1), K23);
    }
    cudaError_t e = cudaMemcpy(dtab, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ddesc, desc.data(), desc.size(), cudaMemcpyHostToDevice);
    for (int d = 0; d < nd && e == cudaSuccess; ++d)
        e = cudaMemcpy(&ctx->d_ctl->count[d][0], &counts[2 * d], 16, cudaMemcpyHostToDevice);
    for (auto& D : ctx->hd) {
        const size_t b = 8 * ((size_t)D.N + 1);
        if (e == cudaSuccess) e = cudaMemset(D.D[0], 0, b);
        if (e == cudaSuccess) e = cudaMemset(D.D[1], 0, b);
        if (e == cudaSuccess) e = cudaMemset(D.Q, 0, b);
    }
    const int gx = std::max(1, ctx->num_sms * 4);
    ctx->cur = 0;
    if (e == cudaSuccess)
        e = launch_load_profile(ctx->fp64, ctx->d_discs, nd, ctx->d_ctl, 0, ctx->seed, ddesc, gx, ctx->stream);
    if (e == cudaSuccess) e = launch_set_dense(ctx->d_discs, nd, ctx->d_ctl, 0, ctx->stream);
    if (e == cudaSuccess) e = launch_deposit(ctx->fp64, ctx->d_discs, nd, ctx->d_ctl, 0, ctx->max_N, gx, ctx->stream);
    if (e == cudaSuccess) e = launch_finalize(ctx->fp64, ctx->d_discs, nd, ctx->d_ctl, 0, 4, 0, ctx->max_N, ctx->stream);
    if (e == cudaSuccess) e = launch_backkick(ctx->fp64, ctx->d_discs, nd, ctx->d_ctl, 0, gx, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(dtab);
    cudaFree(ddesc);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "warm start");
    ctx->deposits_zero = true;
    return PIC_OK;
}
