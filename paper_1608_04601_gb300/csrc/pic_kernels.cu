// pic_kernels.cu -- CUDA kernels (sm_103a) of the 1d3v PIC/MCC time step of
// arXiv:1608.04601, section "PIC/MCC simulation procedure".
//
// One time step is two launches (and the sort every K steps):
//   k_sweep     persistent; tiles of BLOCK x PPT slots of all stores in a
//               static grid-stride order; each warp owns a chunk of 32 PPT
//               slots and loads, pushes (CIC gather of E_n from shared
//               memory, half kick, null-collision MCC on Philox streams, half
//               kick, drift, walls), collides and writes its survivors in slot
//               order into the chunk's own output region, newborns into the
//               chunk's newborn regions, with no barrier inside a tile. CIC
//               deposits go to warp-aggregated shared-memory int64 histograms,
//               flushed with global atomics. Chunk counts are summed per slice.
//   k_post      per slice of chunks: the region starts of the new layout and
//               the newborn copies; per discharge, concurrently: the store
//               totals (new counts) and Poisson (Eq. poisson, rf Dirichlet
//               boundary) from exact integer prefix sums of the deposits, node
//               field, cycle-average accumulators, J(t).
//   sort        every K steps: stable counting sort of each store by cell
//               into a dense store (else an order-preserving repack).
//   k_diag      at the steps the diagnostics schedule names, before the sweep:
//               the electrons' node moments and energy histogram.
#include "pic_internal.h"
#include "pic_device.cuh"

namespace pic {

#define E_CHARGE 1.602176634e-19
#define M_ELEC 9.1093837015e-31
#define EPS0 8.8541878128e-12
#define PI_D 3.14159265358979323846
#define TWO32_D 4294967296.0

constexpr unsigned FULL = 0xFFFFFFFFu;

template <typename T> __device__ __forceinline__ const Consts<T>& consts_of(const Disc& d);
template <> __device__ __forceinline__ const Consts<float>& consts_of<float>(const Disc& d) { return d.cf; }
template <> __device__ __forceinline__ const Consts<double>& consts_of<double>(const Disc& d) { return d.cd; }

template <typename T> struct T4;
template <> struct T4<float> { using type = float4; using two = float2; };
template <> struct T4<double> { using type = d4; using two = double2; };

template <int V>
struct IC {
    static constexpr int value = V;
};

template <typename T>
struct Part {
    int c;
    T f, vx, vy, vz;
};

// Segment (one store of one discharge) as seen by a sweep CTA.
template <typename T>
struct Seg {
    Consts<T> k;
    int d, sp, N, n_pts, has_see, n_exc, leapfrog;
    uint32_t thr, did;
    long long n, cap, bcap, tile0, ntiles;
    const int32_t* cin;
    const void* pin;
    int32_t* cout;
    void* pout;
    int32_t* bc;      // other-species newborns of this sweep, chunk regions
    void* bp;
    int32_t* sc;      // same-species newborns (ionization electrons), chunk regions
    void* sp_;
    const void* Te;
    const void* Ti;
    unsigned long long* Dg;
    unsigned long long* Dother;
    unsigned long long* Qg;
    unsigned long long* cnt;
    const int* start;  // region starts of the input layout
    int K;             // region chunks of the input layout
    long long M, D0;   // slots in the regions, record offset of the dense part
    long long ralloc;  // output regions
    int* cnt_main;
    int* cnt_birth;
    int* cnt_same;
    unsigned* slice_tot;
};

// Programmatic dependent launch (the kernels of a step, launched by launch_pdl): wait until the
// previous kernel in the stream has completed and its writes are visible. Every such kernel calls
// this before its first memory access (a no-op for a kernel launched without the attribute). No
// kernel triggers its dependents early: they launch as its CTAs exit, so no CTA of a later kernel
// shares an SM's L1 with a CTA that may still read data the kernel in between rewrites.
__device__ __forceinline__ void grid_dep_sync() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ int drift(int N, T dtdx, int c, T f, T vz, int& cn, T& fn, int& err) {
    const T s = fma_(vz, dtdx, f);
    if (!(s == s)) err |= ERR_NONFINITE;
    if (!(s >= (T)(-c))) return 0;
    if (s >= (T)(N - c)) return 1;
    const T fl = floor_(s);
    T fr = sub_(s, fl);
    if (fr >= (T)1) fr = one_minus_ulp<T>();
    cn = c + (int)fl;
    fn = fr;
    return -1;
}

// Exact 64-bit add into a shared-memory word with native 32-bit atomics: the low
// word's returned old value tells whether this add carried into the high word.
__device__ __forceinline__ void sadd64(unsigned long long* p, unsigned long long v) {
    unsigned* w = reinterpret_cast<unsigned*>(p);
    const unsigned lo = (unsigned)v, hi = (unsigned)(v >> 32);
    const unsigned old = atomicAdd(&w[0], lo);
    const unsigned up = hi + ((unsigned)(old + lo) < old ? 1u : 0u);
    if (up) atomicAdd(&w[1], up);
}

__device__ __forceinline__ void hist_add(unsigned long long* h, int c, unsigned long long F) {
    atomicAdd(&h[c], (1ull << 32) - F);
    if (F) atomicAdd(&h[c + 1], F);
}

// Same, into a shared-memory histogram.
__device__ __forceinline__ void shist_add(unsigned long long* h, int c, unsigned long long F) {
    sadd64(&h[c], (1ull << 32) - F);
    if (F) sadd64(&h[c + 1], F);
}

// Round-to-nearest-even conversion of a value in [0, 2^32) to an unsigned integer.
__device__ __forceinline__ unsigned long long rint_u32(float a) { return __float2uint_rn(a); }
__device__ __forceinline__ unsigned long long rint_u32(double a) { return __double2uint_rn(a); }

__device__ __forceinline__ unsigned long long cic_F(float f) {
    return (unsigned long long)__float2uint_rn(__fmul_rn(f, 4294967296.0f));  // f < 1: below 2^32
}
__device__ __forceinline__ unsigned long long cic_F(double f) {
    return __double2ull_rn(__dmul_rn(f, TWO32_D));  // may round to 2^32
}

// Warp-aggregated histogram updates (warp_dep, warp_energy below; k_diag): lanes with equal keys are
// grouped (match_any) and each group's sums reduced (redux) and added by its first lane. The group
// reductions of a warp run one after another (one per distinct member mask), so their cost grows
// with the number of groups: a warp with more than HIST_GROUPS distinct keys adds lane by lane
// instead (measured on C2 with the earlier 64-bit adds: the sweep of an unsorted store 140 -> 55
// us; two groups was the best threshold within a sort period). Integer adds: the same sums either way.
constexpr int HIST_GROUPS = 2;

// The sweep's shared-memory histograms hold exact sums in 32-bit pieces, added with atomics whose
// result is not read (no return trip, no carry logic):
//   deposit, per cell c: particles n_c, and the sum of F = rn(f 2^32) as low and high 16-bit parts;
//     node j then receives 2^32 n_j - F_j + F_{j-1} (the charge split (2^32 - F, F) of every
//     particle), formed in 64 bits when the CTA flushes;
//   energy moment, per node: the sum of its 26-bit values as low 13-bit and high parts.
// A piece sum stays below 2^32 while the CTA has added fewer than 2^15 particles (plus their
// newborns) since its last flush: the sweep flushes at least that often.
struct DepHist {
    unsigned* n;
    unsigned* lo;
    unsigned* hi;
};
__device__ __forceinline__ void dep_add(const DepHist& h, int c, unsigned long long F) {
    atomicAdd(&h.n[c], 1u);
    atomicAdd(&h.lo[c], (unsigned)(F & 0xFFFFu));
    atomicAdd(&h.hi[c], (unsigned)(F >> 16));
}
// Warp-aggregated deposit of one particle per lane (key = cell, < 0: none; F as above): lanes of
// equal keys are reduced (match_any, redux) and their first lane adds the group's sums, unless the
// warp's keys form more than HIST_GROUPS groups (then lane by lane).
__device__ __forceinline__ void warp_dep(const DepHist& h, int key, unsigned long long F, int lane) {
    const int k0 = __shfl_sync(FULL, key, 0);
    if (!__all_sync(FULL, key == k0)) {  // several cells (or empty lanes): lane by lane
        if (key >= 0) dep_add(h, key, F);
        return;
    }
    const unsigned lo = __reduce_add_sync(FULL, (unsigned)(F & 0xFFFFu));
    const unsigned hi = __reduce_add_sync(FULL, (unsigned)(F >> 16));
    if (lane == 0 && key >= 0) {
        atomicAdd(&h.n[key], 32u);
        if (lo) atomicAdd(&h.lo[key], lo);
        if (hi) atomicAdd(&h.hi[key], hi);
    }
}
// Warp-aggregated energy moment: a (< 2^26) to node key, b (< 2^26) to node key + 1.
__device__ __forceinline__ void warp_energy(unsigned* qlo, unsigned* qhi, int key, unsigned a, unsigned b, int lane) {
    const int k0 = __shfl_sync(FULL, key, 0);
    const unsigned peers = FULL;
    const bool leader = lane == 0;
    if (!__all_sync(FULL, key == k0)) {
        if (key >= 0) {
            if (a) {
                atomicAdd(&qlo[key], a & 0x1FFFu);
                atomicAdd(&qhi[key], a >> 13);
            }
            if (b) {
                atomicAdd(&qlo[key + 1], b & 0x1FFFu);
                atomicAdd(&qhi[key + 1], b >> 13);
            }
        }
        return;
    }
    const unsigned al = __reduce_add_sync(peers, a & 0x1FFFu), ah = __reduce_add_sync(peers, a >> 13);
    const unsigned bl = __reduce_add_sync(peers, b & 0x1FFFu), bh = __reduce_add_sync(peers, b >> 13);
    if (leader && key >= 0) {
        if (al) atomicAdd(&qlo[key], al);
        if (ah) atomicAdd(&qhi[key], ah);
        if (bl) atomicAdd(&qlo[key + 1], bl);
        if (bh) atomicAdd(&qhi[key + 1], bh);
    }
}

template <typename T>
__device__ __forceinline__ void store_rec(int32_t* c, void* p, unsigned i, const Part<T>& q);
template <>
__device__ __forceinline__ void store_rec<float>(int32_t* c, void* p, unsigned i, const Part<float>& q) {
    c[i] = q.c;
    reinterpret_cast<float4*>(p)[i] = make_float4(q.f, q.vx, q.vy, q.vz);
}
template <>
__device__ __forceinline__ void store_rec<double>(int32_t* c, void* p, unsigned i, const Part<double>& q) {
    c[i] = q.c;
    double2* pp = reinterpret_cast<double2*>(p) + 2 * i;
    pp[0] = make_double2(q.f, q.vx);
    pp[1] = make_double2(q.vy, q.vz);
}

template <typename T>
__device__ __forceinline__ void load_rec(const void* p, unsigned i, T& f, T& vx, T& vy, T& vz);
template <>
__device__ __forceinline__ void load_rec<float>(const void* p, unsigned i, float& f, float& vx, float& vy,
                                                float& vz) {
    const float4 a = __ldcs(reinterpret_cast<const float4*>(p) + i);
    f = a.x; vx = a.y; vy = a.z; vz = a.w;
}
template <>
__device__ __forceinline__ void load_rec<double>(const void* p, unsigned i, double& f, double& vx, double& vy,
                                                 double& vz) {
    const double2* pp = reinterpret_cast<const double2*>(p) + 2 * i;
    const double2 a = __ldcs(pp), b = __ldcs(pp + 1);
    f = a.x; vx = a.y; vy = b.x; vz = b.y;
}

// The collision candidates of a chunk are queued by their warp in shared memory as their indices
// in the chunk; the lane that processes one reads the particle from the staged records, collides
// it, writes the new velocity back into the staged record and flags the newborns it left after
// their first drift, which it stores at the candidate's rank in the chunk's newborn regions (the
// warp then compacts them into parent-slot order).
// A collision candidate of a chunk: its velocity v_n and gathered field on entry; the velocity after
// the collision on return; newborns flagged in `out` (bit 1: same species, bit 2: other species).
template <typename T>
struct Cand {
    T ef;
    T vx, vy, vz;
};

// The collision of a queued candidate (null-collision method: process
// selection against the cumulative rate tables, then the kinematics).
template <typename T>
__device__ __forceinline__ uint32_t collide(const Seg<T>& S, Cand<T>& q, int qc, T qf, uint32_t slot, uint32_t ridx,
                                         long long step, unsigned long long seed, const DepHist& sH, unsigned* sC,
                                         int& err) {
    using Row4 = typename T4<T>::type;
    using Row2 = typename T4<T>::two;
    const Consts<T>& K = S.k;
    const int N = S.N;
    T vx = q.vx, vy = q.vy, vz = q.vz;
    uint32_t out = 0;
    if (S.sp == 0) {
        const T e2 = fma_(vx, vx, fma_(vy, vy, mul_(vz, vz)));
        bool child = false;
        T cvx = 0, cvy = 0, cvz = 0, ivx = 0, ivy = 0, ivz = 0;
        const U4 r = draw(seed, slot, step, 0, 0, S.did);
        const T xi = mul_(e2, K.kappa_e);
        const Row4* Te = reinterpret_cast<const Row4*>(S.Te);
        T C0, C1, C2, C3;
        if (!(xi < (T)(S.n_pts - 1))) {
            const Row4 a = Te[S.n_pts - 1];
            C0 = a.x; C1 = a.y; C2 = a.z; C3 = a.w;
            atomicAdd(&sC[CNT_CLAMP + 0], 1u);
        } else {
            const int i = (int)xi;
            const T fr = sub_(xi, (T)i);
            const Row4 a = Te[i], b = Te[i + 1];
            C0 = fma_(fr, sub_(b.x, a.x), a.x);
            C1 = fma_(fr, sub_(b.y, a.y), a.y);
            C2 = fma_(fr, sub_(b.z, a.z), a.z);
            C3 = fma_(fr, sub_(b.w, a.w), a.w);
        }
        const T R = mul_((T)u01(r.y), K.kmax_e);
        const int j = (R < C0) ? 0 : (R < C1) ? 1 : (R < C2) ? 2 : (R < C3) ? 3 : 4;
        if (j < 4) {
            // the scattered electron's direction: the same draw for every process, so it is
            // formed once, outside the per-process branches
            T nx, ny, nz;
            iso_dir(u01(r.z), u01(r.w), nx, ny, nz);
            if (j == 0) {  // elastic, target at rest: v' = beta v + (1-beta)|v| n
                const T g = sqrt_(e2);
                const T og = mul_(K.omb, g);
                vx = fma_(K.beta, vx, mul_(og, nx));
                vy = fma_(K.beta, vy, mul_(og, ny));
                vz = fma_(K.beta, vz, mul_(og, nz));
                atomicAdd(&sC[CNT_COLL_E + 0], 1u);
            } else if (j <= S.n_exc) {  // excitation of level j
                const T e2n = sub_(e2, K.de2_exc[j - 1]);
                if (e2n > (T)0) {
                    const T sp = sqrt_(e2n);
                    vx = mul_(sp, nx);
                    vy = mul_(sp, ny);
                    vz = mul_(sp, nz);
                    atomicAdd(&sC[CNT_COLL_E + j], 1u);
                } else {
                    atomicAdd(&sC[CNT_NULL_INEL], 1u);
                }
            } else {  // ionization: remaining energy shared equally
                const T e2r = sub_(e2, K.de2_iz);
                if (e2r > (T)0) {
                    const T sp = sqrt_(mul_((T)0.5, e2r));
                    vx = mul_(sp, nx);
                    vy = mul_(sp, ny);
                    vz = mul_(sp, nz);
                    const U4 q1 = draw(seed, slot, step, 0, 1, S.did);
                    const U4 w = draw(seed, slot, step, 0, 2, S.did);
                    iso_dir(u01(q1.x), u01(q1.y), nx, ny, nz);
                    cvx = mul_(sp, nx);
                    cvy = mul_(sp, ny);
                    cvz = mul_(sp, nz);
                    float b0, b1, b2, b3;
                    box_muller(u01(q1.z), u01(q1.w), b0, b1);
                    box_muller(u01(w.x), u01(w.y), b2, b3);
                    ivx = mul_(K.sig_n, (T)b0);
                    ivy = mul_(K.sig_n, (T)b1);
                    ivz = mul_(K.sig_n, (T)b2);
                    child = true;
                    atomicAdd(&sC[CNT_COLL_E + 3], 1u);
                } else {
                    atomicAdd(&sC[CNT_NULL_INEL], 1u);
                }
            }
        }
        if (child) {  // newborns: second half kick and drift from the parent's position
            int cn;
            T fn;
            if (!S.leapfrog) cvz = fma_(K.K[0], q.ef, cvz);  // born at t_n (Verlet): the second half kick
            int side = drift(N, K.dtdx, qc, qf, cvz, cn, fn, err);
            if (side < 0) {
                store_rec<T>(S.sc, S.sp_, ridx, Part<T>{cn, fn, cvx, cvy, cvz});
                dep_add(sH, cn, cic_F(fn));
                out |= 2u;
            } else {
                atomicAdd(&sC[CNT_ABS + side], 1u);
            }
            if (!S.leapfrog) ivz = fma_(K.K[1], q.ef, ivz);
            side = drift(N, K.dtdx, qc, qf, ivz, cn, fn, err);
            if (side < 0) {
                store_rec<T>(S.bc, S.bp, ridx, Part<T>{cn, fn, ivx, ivy, ivz});
                hist_add(S.Dother, cn, cic_F(fn));
                out |= 4u;
            } else {
                atomicAdd(&sC[CNT_ABS + 2 + side], 1u);
            }
        }
    } else {
        const U4 r = draw(seed, slot, step, 1, 0, S.did);
        const U4 q1 = draw(seed, slot, step, 1, 1, S.did);
        float a0, a1, a2, a3;
        box_muller(u01(q1.x), u01(q1.y), a0, a1);
        box_muller(u01(q1.z), u01(q1.w), a2, a3);
        const T vnx = mul_(K.sig_n, (T)a0), vny = mul_(K.sig_n, (T)a1), vnz = mul_(K.sig_n, (T)a2);
        const T gx = sub_(vx, vnx), gy = sub_(vy, vny), gz = sub_(vz, vnz);
        const T g2 = fma_(gx, gx, fma_(gy, gy, mul_(gz, gz)));
        const T xi = mul_(g2, K.kappa_i);
        const Row2* Ti = reinterpret_cast<const Row2*>(S.Ti);
        T C0, C1;
        if (!(xi < (T)(S.n_pts - 1))) {
            const Row2 a = Ti[S.n_pts - 1];
            C0 = a.x; C1 = a.y;
            atomicAdd(&sC[CNT_CLAMP + 1], 1u);
        } else {
            const int i = (int)xi;
            const T fr = sub_(xi, (T)i);
            const Row2 a = Ti[i], b = Ti[i + 1];
            C0 = fma_(fr, sub_(b.x, a.x), a.x);
            C1 = fma_(fr, sub_(b.y, a.y), a.y);
        }
        const T R = mul_((T)u01(r.y), K.kmax_i);
        if (R < C0) {  // isotropic in the centre-of-mass frame, equal masses
            const T hg = mul_((T)0.5, sqrt_(g2));
            T nx, ny, nz;
            iso_dir(u01(r.z), u01(r.w), nx, ny, nz);
            vx = fma_(hg, nx, mul_(add_(vx, vnx), (T)0.5));
            vy = fma_(hg, ny, mul_(add_(vy, vny), (T)0.5));
            vz = fma_(hg, nz, mul_(add_(vz, vnz), (T)0.5));
            atomicAdd(&sC[CNT_COLL_I + 0], 1u);
        } else if (R < C1) {  // backward: the ion takes the atom's velocity
            vx = vnx;
            vy = vny;
            vz = vnz;
            atomicAdd(&sC[CNT_COLL_I + 1], 1u);
        }
    }
    q.vx = vx;
    q.vy = vy;
    q.vz = vz;
    return out;
}

// Secondary electron of an ion absorbed at electrode `side` (added option).
template <typename T>
__device__ __forceinline__ bool emit_see(const Seg<T>& S, uint32_t slot, long long step, unsigned long long seed,
                                      int side, Part<T>& p, unsigned* sC) {
    const Consts<T>& K = S.k;
    const U4 w = draw(seed, slot, step, 1, 3, S.did);
    if (!((T)u01(w.x) < K.gamma)) return false;
    const T vn = mul_(K.sig_see_n, (T)__fsqrt_rn(-own_logf(u01(w.y))));
    float t0, t1;
    box_muller(u01(w.z), u01(w.w), t0, t1);
    const int ce = side == 0 ? 0 : S.N - 1;
    const T fe = side == 0 ? (T)0 : one_minus_ulp<T>();
    p = Part<T>{ce, fe, mul_(K.sig_see, (T)t0), mul_(K.sig_see, (T)t1), side == 0 ? vn : -vn};
    hist_add(S.Dother, ce, cic_F(fe));
    atomicAdd(&sC[CNT_SEE], 1u);
    atomicAdd(&sC[CNT_SEE_SIDE + side], 1u);
    return true;
}

// Moves one record within a buffer (newborn compaction, dst <= src; nothing to do if equal).
template <typename T>
__device__ __forceinline__ void move_rec(int32_t* c, void* p, unsigned src, unsigned dst) {
    if (src == dst) return;
    using R = typename Rec<T>::type;
    R* pp = reinterpret_cast<R*>(p);
    const int cv = c[src];
    const R rv = pp[src];
    c[dst] = cv;
    pp[dst] = rv;
}

// Store totals after a sweep, for discharge d, by one warp of k_post: from the slice sums of parity
// par, the new counts and the layout of the output buffer (the sweep's chunks become its regions,
// the newborns its dense part at R0); on a full step the per-period mean counts; then the slice
// sums of the other parity cleared for the next sweep.
__device__ __forceinline__ void store_totals(const Disc& D, int d, Ctl* ctl, int lane, int par, bool full_step,
                                             int out_buf, int& err) {
    long long chunks[2], slices[2];
    for (int sp = 0; sp < 2; ++sp) {
        chunks[sp] = ctl->chunks_in[d][sp];
        slices[sp] = (chunks[sp] + SLICE - 1) / SLICE;
    }
    const unsigned* T0 = D.slice_tot[0] + (size_t)par * 3 * D.slice_n[0];
    const unsigned* T1 = D.slice_tot[1] + (size_t)par * 3 * D.slice_n[1];
    // survivors of both sweeps, ionization electrons and ions of the electron sweep, SEE electrons
    long long main0 = 0, main1 = 0, same0 = 0, see = 0, ions = 0;
    for (long long k = lane; k < max(slices[0], slices[1]); k += 32) {
        if (k < slices[0]) {
            main0 += T0[3 * k + 0];
            ions += T0[3 * k + 1];
            same0 += T0[3 * k + 2];
        }
        if (k < slices[1]) {
            main1 += T1[3 * k + 0];
            see += T1[3 * k + 1];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        main0 += __shfl_xor_sync(FULL, main0, o);
        main1 += __shfl_xor_sync(FULL, main1, o);
        same0 += __shfl_xor_sync(FULL, same0, o);
        see += __shfl_xor_sync(FULL, see, o);
        ions += __shfl_xor_sync(FULL, ions, o);
    }
    for (int sp = 0; sp < 2; ++sp) {
        const long long main_total = sp == 0 ? main0 : main1;
        const long long nb = sp == 0 ? same0 + see : ions;
        const long long bcap = D.bcap;
        const long long nbk = nb < bcap ? nb : bcap;
        const long long ch = chunks[sp];
        long long n_new = main_total + nbk;
        if (lane == 0) {
            if (nb > bcap) err |= ERR_CAPACITY;
            // more regions than the next sweep has output regions for: a sort or a repack is overdue
            if (ch > D.rmax[sp]) err |= ERR_CAPACITY;
            D.start[sp][ch] = (int)main_total;
            if (n_new > D.cap[sp]) {
                err |= ERR_CAPACITY;
                n_new = D.cap[sp];
            }
            ctl->count[d][sp] = n_new;
            Lay& L = ctl->lay[d][sp][out_buf];
            L.K = (int)ch;
            L.M = main_total;
            L.D0 = D.R0[sp];
            if (full_step) {  // per-period mean counts (steady-state criterion)
                const long long n_step = ctl->step;  // this step is n; the counts belong to n+1
                ctl->period_acc[d][sp] += (double)n_new;
                if (D.steps_per_period > 0 && (n_step + 1) % D.steps_per_period == 0) {
                    const long long per = (n_step + 1) / D.steps_per_period - 1;
                    D.period_mean[(per % PERIOD_HIST) * 2 + sp] = ctl->period_acc[d][sp] / D.steps_per_period;
                    ctl->period_acc[d][sp] = 0.0;
                }
            }
        }
        // the next sweep adds into the other parity
        unsigned* Tn = D.slice_tot[sp] + (size_t)(par ^ 1) * 3 * D.slice_n[sp];
        for (int k = lane; k < 3 * D.slice_n[sp]; k += 32) Tn[k] = 0;
    }
}

// Bulk copies into shared memory (the asynchronous copy engine) with an mbarrier per buffer.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(unsigned long long* mb) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mb)) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* mb, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mb)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* mb) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mb))
                 : "memory");
}
// Waits for phase `parity` of the barrier to complete, at most `tries` polls (each poll may block
// for a hardware-defined time); false if it gave up.
constexpr int MBAR_TRIES = 1 << 20;
__device__ __forceinline__ bool mbar_wait(unsigned long long* mb, unsigned parity, int tries = MBAR_TRIES) {
    const unsigned a = smem_u32(mb);
    for (int it = 0; it < tries; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Dynamic shared memory of the sweep: the node field (T, N+1), the deposit histogram (u32 n, lo, hi
// per cell) and the energy moment (u32 lo, hi per node); per warp two staging buffers of one chunk (records, then cells) and its candidate
// queue; per store the layout snapshot and the tile prefix.
template <typename T>
__host__ __device__ constexpr size_t sweep_hist_offset(int max_N) {  // after the node field
    return (((size_t)(max_N + 1) * sizeof(T) + 15) / 16) * 16;
}
template <typename T>
__host__ __device__ constexpr size_t sweep_stage_offset(int max_N) {
    return ((sweep_hist_offset<T>(max_N) + 4 * (3 * (size_t)max_N + 2 * ((size_t)max_N + 1)) + 127) / 128) * 128;
}
template <typename T, int PPT>
__host__ __device__ constexpr size_t sweep_stage_bytes() {  // one buffer of one warp
    return (size_t)32 * PPT * (sizeof(typename Rec<T>::type) + 4);
}
template <typename T, int BLOCK, int PPT>
__host__ __device__ constexpr size_t sweep_queue_offset(int max_N) {
    return sweep_stage_offset<T>(max_N) + 2 * (BLOCK / 32) * sweep_stage_bytes<T, PPT>();
}
template <typename T, int BLOCK, int PPT>
__host__ __device__ constexpr size_t sweep_store_offset(int max_N) {
    return ((sweep_queue_offset<T, BLOCK, PPT>(max_N) + (size_t)BLOCK * PPT + 15) / 16) * 16;
}
struct StoreSnap {  // layout of one input store, for the prefetches of any tile
    int K, chunks;
    long long M, D0, n;
};
template <typename T, int BLOCK, int PPT>
__host__ __device__ constexpr size_t sweep_smem(int max_N, int n_disc) {
    return sweep_store_offset<T, BLOCK, PPT>(max_N) + sizeof(StoreSnap) * 2 * (size_t)n_disc +
           sizeof(long long) * (2 * (size_t)n_disc + 1);
}

// Resident threads per SM the sweep is compiled for (the register budget is 65536 / that): the
// FP32 chunk state fits 64 registers at PPT <= 2 and 80 at PPT = 4; 512-thread CTAs at PPT = 4 are
// held to 64 registers so that two of them fit an SM.
template <typename T, int BLOCK, int PPT>
__host__ __device__ constexpr int sweep_threads_per_sm() {
    return sizeof(T) == 4 ? (PPT <= 2 ? 1024 : PPT == 4 ? (BLOCK >= 512 ? 1024 : 768) : 512) : 256;
}
template <typename T, int BLOCK, int PPT>
__host__ __device__ constexpr int sweep_min_blocks() {
    return sweep_threads_per_sm<T, BLOCK, PPT>() / BLOCK > 0 ? sweep_threads_per_sm<T, BLOCK, PPT>() / BLOCK : 1;
}

// ---------------------------------------------------------------------------
// The sweep. Persistent CTAs take the tiles of NW chunks of all stores (discharge, species) in a
// static grid-stride order; warp w of a tile owns the tile's chunk w (at most CHUNK = 32 PPT
// slots, a region or a run of the dense part of the input layout) and works on it alone, with no
// barrier: the chunk's records and cells arrive in the warp's staging buffer by a bulk copy issued
// while the warp was processing its previous chunk; the warp pushes its particles (gather, kick,
// energy moment, candidate test), runs one collision pass over the chunk's candidates, then kicks,
// drifts, deposits and writes the survivors in slot order to the chunk's own output region
// [CHUNK cs, ...), cs the chunk index. Newborns go in parent-slot order to the chunk's regions of
// the newborn buffers (same species: ionization electrons; other species: ionization ions, or SEE
// electrons of the ion sweep), and the chunk records the three counts. The CTA synchronises only
// where its tiles move to another store (histogram flush).
template <typename T, int BLOCK, int PPT>
__global__ void __launch_bounds__(BLOCK, sweep_min_blocks<T, BLOCK, PPT>())
    k_sweep(const Disc* __restrict__ discs, int n_disc, Ctl* __restrict__ ctl, int in_buf, unsigned long long seed,
            int max_N) {
    using R = typename Rec<T>::type;
    constexpr int NW = BLOCK / 32;
    constexpr int CHUNK = 32 * PPT;
    constexpr unsigned REC_BYTES = CHUNK * sizeof(R), CELL_BYTES = CHUNK * 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* s_E = reinterpret_cast<T*>(smem_raw);
    unsigned* s_h32 = reinterpret_cast<unsigned*>(smem_raw + sweep_hist_offset<T>(max_N));
    const DepHist s_dep{s_h32, s_h32 + max_N, s_h32 + 2 * max_N};
    unsigned* s_qlo = s_h32 + 3 * max_N;
    unsigned* s_qhi = s_qlo + (max_N + 1);
    const int h32_words = 3 * max_N + 2 * (max_N + 1);
    StoreSnap* s_store = reinterpret_cast<StoreSnap*>(smem_raw + sweep_store_offset<T, BLOCK, PPT>(max_N));
    long long* s_segstart = reinterpret_cast<long long*>(s_store + 2 * n_disc);

    __shared__ Seg<T> S;
    __shared__ long long s_step;
    __shared__ int s_par;
    __shared__ unsigned s_cnt[NCNT];
    __shared__ int s_err;
    __shared__ unsigned long long s_mbar[NW][2];
    // per warp: the chunk prefetched for its next tile (chunk index, first and end slot, valid), the
    // store of the last prefetch, and the barrier phases (kept here, not in registers)
    __shared__ int s_pf[NW][6];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned char* stage = smem_raw + sweep_stage_offset<T>(max_N) + (size_t)warp * 2 * sweep_stage_bytes<T, PPT>();
    // per warp: the chunk indices of its candidates, in slot order (CHUNK <= 256)
    uint8_t* Q = reinterpret_cast<uint8_t*>(smem_raw + sweep_queue_offset<T, BLOCK, PPT>(max_N)) + warp * CHUNK;
    if (lane == 0) {
        mbar_init(&s_mbar[warp][0]);
        mbar_init(&s_mbar[warp][1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    grid_dep_sync();
    if (tid == 0) {
        long long acc = 0;
        int err0 = 0;
        for (int s = 0; s < 2 * n_disc; ++s) {
            const int d = s >> 1, sp = s & 1;
            const Lay L = ctl->lay[d][sp][in_buf];
            const long long n = ctl->count[d][sp];
            long long ch = chunks_of(L, n, CHUNK);
            if (ch > discs[d].ralloc[sp]) {  // more chunks than output regions: reported, the rest dropped
                ch = discs[d].ralloc[sp];
                err0 |= ERR_CAPACITY;
            }
            s_store[s] = StoreSnap{L.K, (int)ch, L.M, L.D0, n};
            s_segstart[s] = acc;
            acc += (ch + NW - 1) / NW;
            if (blockIdx.x == 0) ctl->chunks_in[d][sp] = (int)ch;  // read by the post-sweep grid
        }
        s_segstart[2 * n_disc] = acc;
        s_step = ctl->step;
        s_par = ctl->slice_par;
        s_err = blockIdx.x == 0 ? err0 : 0;
    }
    __syncthreads();
    const int total_tiles = (int)s_segstart[2 * n_disc];  // tiles and chunks fit in 31 bits (record offsets do)
    const long long step = s_step;
    int cur_seg = -1, cur_d = -1;
    int err = 0;

    // Adds the CTA's histograms and counters of the current store to the global ones and clears them.
    auto flush = [&]() {
        __syncthreads();
        const int N = S.N;
        for (int j = tid; j <= N; j += BLOCK) {
            unsigned long long h = 0;
            if (j < N)
                h = ((unsigned long long)s_dep.n[j] << 32) -
                    ((unsigned long long)s_dep.lo[j] + ((unsigned long long)s_dep.hi[j] << 16));
            if (j > 0) h += (unsigned long long)s_dep.lo[j - 1] + ((unsigned long long)s_dep.hi[j - 1] << 16);
            if (h) atomicAdd(&S.Dg[j], h);
            if (S.sp == 0) {
                const unsigned long long q = (unsigned long long)s_qlo[j] + ((unsigned long long)s_qhi[j] << 13);
                if (q) atomicAdd(&S.Qg[j], q);
            }
        }
        if (tid < NCNT && s_cnt[tid]) atomicAdd(&S.cnt[tid], (unsigned long long)s_cnt[tid]);
        __syncthreads();
        for (int j = tid; j < h32_words; j += BLOCK) s_h32[j] = 0;
        if (tid < NCNT) s_cnt[tid] = 0;
        __syncthreads();
    };

    // Prefetch of this warp's chunk of tile gn into staging buffer b: the store of the tile, the
    // chunk's record offset (known without any table) and its first and end slot (regions: from
    // the start table, loaded now and used when the chunk is processed).
    int* pf = s_pf[warp];  // [0] chunk, [1] first slot, [2] end slot, [3] valid, [4] store, [5] phases
    auto prefetch = [&](int b, int gn) {
        if (lane == 0) pf[3] = 0;
        if (gn >= total_tiles) return;
        int sg = pf[4];
        while (sg + 1 < 2 * n_disc && s_segstart[sg + 1] <= gn) ++sg;
        const StoreSnap ss = s_store[sg];
        const int cs = (gn - (int)s_segstart[sg]) * NW + warp;
        if (cs >= ss.chunks) return;
        const int d = sg >> 1, sp = sg & 1;
        long long src;
        int pst0, pst1;
        if (cs < ss.K) {
            src = (long long)cs * CHUNK;
            const int* st = discs[d].start[sp];
            pst0 = __ldg(st + cs);
            pst1 = __ldg(st + cs + 1);
        } else {
            const long long j = (long long)(cs - ss.K);
            src = ss.D0 + j * CHUNK;
            pst0 = (int)(ss.M + j * CHUNK);
            pst1 = (int)min(ss.n, ss.M + (j + 1) * CHUNK);
        }
        if (lane == 0) {
            pf[0] = (int)cs;
            pf[1] = pst0;
            pf[2] = pst1;
            pf[3] = 1;
            pf[4] = sg;
            unsigned char* buf = stage + (size_t)b * sweep_stage_bytes<T, PPT>();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads and writes of the buffer
            mbar_expect(&s_mbar[warp][b], REC_BYTES + CELL_BYTES);
            bulk_g2s(buf, reinterpret_cast<const R*>(discs[d].p[in_buf][sp]) + src, REC_BYTES, &s_mbar[warp][b]);
            bulk_g2s(buf + REC_BYTES, discs[d].c[in_buf][sp] + src, CELL_BYTES, &s_mbar[warp][b]);
        }
    };

    const unsigned lt = (1u << lane) - 1u;
    if (lane == 0) {
        pf[4] = 0;
        pf[5] = 0;  // bit b: phase of buffer b's barrier the next wait expects
    }
    __syncwarp();
    prefetch(0, blockIdx.x);  // the chunk of the CTA's first tile, into buffer 0
    __syncwarp();

    // One warp's chunk of the store of species SP: push, collide, write (see above). Phases B and C
    // read each particle again from the staging buffer and repeat the gather and the first half kick
    // (the same operations, so the same values) instead of keeping them in registers or in the
    // queue; a collision writes the velocity after it back into the staged record, and phase C then
    // takes that velocity as v_n.
    auto chunk = [&](unsigned cs, int base, int cnt, R* srec, const int32_t* scell, auto spc) {
        constexpr int SP = decltype(spc)::value;
        const unsigned obase = cs * CHUNK;
        unsigned offA = obase, offB = obase, offS = obase;  // output cursors of the chunk's regions
        const int N = S.N;
        const T Ksp = S.k.K[SP];
        // particle i of the chunk: cell (-1 if none or out of range), offset, velocity, gathered field
        auto particle = [&](int i, int& c, T& f, T& vx, T& vy, T& vz, T& ef) {
            c = -1;
            f = vx = vy = vz = ef = (T)0;
            if (i < cnt) {
                c = scell[i];
                const R r = srec[i];
                f = r.x;
                vx = r.y;
                vy = r.z;
                vz = r.w;
                if (!((unsigned)c < (unsigned)N)) c = -1;
                else {
                    const T E0 = s_E[c], E1 = s_E[c + 1];
                    ef = fma_(f, sub_(E1, E0), E0);
                }
            }
        };
        if (cnt > 0) {
            // candidate words: slots 4q..4q+3 take the four words of one Philox call (call 4,
            // counter word 0 = q); lane l computes the calls q0 + l + 32 m, q0 = base / 4, compares
            // their words with the threshold and keeps the results as bits 4 m + w (word w); the
            // particle of slot s takes bit s % 4 of call s / 4 by one shuffle
            constexpr int NG = (CHUNK / 4 + 1 + 31) / 32;
            const uint32_t did = S.did, thr = S.thr;
            const unsigned q0 = (unsigned)base >> 2;
            // calls needed: q0 .. (base + cnt - 1) / 4; the last group of calls is drawn only if the
            // chunk reaches it (an unaligned first slot needs one call beyond CHUNK / 4)
            const int ncalls = (int)(((unsigned)base + cnt - 1) >> 2) - (int)q0 + 1;
            unsigned cbits = 0;
#pragma unroll
            for (int m = 0; m < NG; ++m)
                if (32 * m < ncalls) {
                    const U4 w = draw(seed, q0 + lane + 32 * m, step, SP, 4, did);
                    cbits |= ((w.x < thr ? 1u : 0u) | (w.y < thr ? 2u : 0u) | (w.z < thr ? 4u : 0u) |
                              (w.w < thr ? 8u : 0u))
                             << (4 * m);
                }
            // ---- phase A: gather, first half kick, energy moment, candidate test
            unsigned candm = 0;  // bit k: this lane's particle of row k is a candidate
            int qn = 0;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const int i = 32 * k + lane;
                int c;
                T f, vx, vy, vz, ef;
                particle(i, c, f, vx, vy, vz, ef);
                if (i < cnt && c < 0) err |= ERR_NONFINITE;  // corrupt cell index: dropped and reported
                const bool valid = c >= 0;
                unsigned qa = 0, qb = 0;
                if (valid) {
                    vz = fma_(Ksp, ef, vz);  // v_n
                    if (SP == 0) {  // energy moment at (x_n, v_n), 2^-12 eV, clamped at 2^26
                        const T e2 = fma_(vx, vx, fma_(vy, vy, mul_(vz, vz)));
                        T eq = mul_(e2, S.k.kappa_E);
                        if (!(eq <= (T)0x1p26)) eq = (T)0x1p26;
                        const unsigned long long Et = rint_u32(eq);
                        const unsigned long long Eh = rint_u32(mul_(eq, f));
                        qa = (unsigned)(Et - Eh);
                        qb = (unsigned)Eh;
                    }
                }
                if (SP == 0) warp_energy(s_qlo, s_qhi, c, qa, qb, lane);
                const unsigned slot = (unsigned)base + i;
                const unsigned r = (slot >> 2) - q0;
                const unsigned cb = __shfl_sync(FULL, cbits, r & 31);
                const bool cand = valid && ((cb >> (4 * (r >> 5) + (slot & 3))) & 1u);
                const unsigned cm = __ballot_sync(FULL, cand);
                if (lane == 0 && cm) atomicAdd(&s_cnt[CNT_CAND + SP], (unsigned)__popc(cm));
                if (cand) {
                    candm |= 1u << k;
                    Q[qn + __popc(cm & lt)] = (uint8_t)i;
                }
                qn += __popc(cm);
            }
            // ---- phase B: the chunk's candidates, 32 at a time; newborns in queue (= slot) order
            __syncwarp();
            for (int r0 = 0; r0 < qn; r0 += 32) {
                const int q = r0 + lane;
                uint32_t o = 0;
                if (q < qn) {
                    const int i = Q[q];
                    int c;
                    T f, vx, vy, vz, ef;
                    particle(i, c, f, vx, vy, vz, ef);  // a candidate has a valid cell
                    T vzc = fma_(Ksp, ef, vz);                 // v_n
                    if (S.leapfrog) vzc = fma_(Ksp, ef, vzc);  // leapfrog: the collision acts on v_{n+1/2}
                    Cand<T> e{ef, vx, vy, vzc};
                    o = collide<T>(S, e, c, f, (uint32_t)base + i, obase + q, step, seed, s_dep, s_cnt, err);
                    R& rec = srec[i];
                    rec.y = e.vx;
                    rec.z = e.vy;
                    rec.w = e.vz;
                }
                __syncwarp();
                if (SP == 0) {  // the round's newborns, from the candidates' ranks to parent-slot order (dst <= src)
                    const unsigned m1 = __ballot_sync(FULL, (o & 2u) != 0), m2 = __ballot_sync(FULL, (o & 4u) != 0);
                    if (o & 2u) move_rec<T>(S.sc, S.sp_, obase + q, offS + __popc(m1 & lt));
                    if (o & 4u) move_rec<T>(S.bc, S.bp, obase + q, offB + __popc(m2 & lt));
                    offS += __popc(m1);
                    offB += __popc(m2);
                    __syncwarp();
                }
            }
            // ---- phase C: second half kick, drift, walls, deposit, survivors in slot order
            const T dtdx = S.k.dtdx;
            int32_t* __restrict__ cout = S.cout;
            void* pout = S.pout;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const int i = 32 * k + lane;
                bool alive = false, see = false;
                Part<T> P0{}, Pse{};
                int c;
                T f, vx, vy, vz, ef;
                particle(i, c, f, vx, vy, vz, ef);
                if (c >= 0) {
                    // v_n as in phase A; a candidate's staged record already holds its velocity after
                    // the collision (at v_n, or at v_{n+1/2} in the leapfrog scheme, then final)
                    const bool coll = (candm >> k) & 1u;
                    if (!coll) vz = fma_(Ksp, ef, vz);
                    if (!(coll && S.leapfrog)) vz = fma_(Ksp, ef, vz);
                    int cn;
                    T fn;
                    const int side = drift(N, dtdx, c, f, vz, cn, fn, err);
                    if (side < 0) {
                        P0 = Part<T>{cn, fn, vx, vy, vz};
                        alive = true;
                    } else {
                        atomicAdd(&s_cnt[CNT_ABS + 2 * SP + side], 1u);
                        if (SP == 1 && S.has_see)
                            see = emit_see<T>(S, (uint32_t)base + i, step, seed, side, Pse, s_cnt);
                    }
                }
                warp_dep(s_dep, alive ? P0.c : -1, alive ? cic_F(P0.f) : 0ull, lane);
                const unsigned mA = __ballot_sync(FULL, alive);
                if (alive) store_rec<T>(cout, pout, offA + __popc(mA & lt), P0);
                offA += __popc(mA);
                if (SP == 1) {
                    const unsigned mB = __ballot_sync(FULL, see);
                    if (see) store_rec<T>(S.bc, S.bp, offB + __popc(mB & lt), Pse);
                    offB += __popc(mB);
                }
            }
        }
        if (lane == 0) {
            const unsigned a = offA - obase, b = offB - obase, c = offS - obase;
            S.cnt_main[cs] = (int)a;
            S.cnt_birth[cs] = (int)b;
            if (SP == 0) S.cnt_same[cs] = (int)c;
            unsigned* sl = S.slice_tot + 3 * (cs / SLICE);
            if (a) atomicAdd(&sl[0], a);
            if (b) atomicAdd(&sl[1], b);
            if (SP == 0 && c) atomicAdd(&sl[2], c);
        }
    };

    // tiles between flushes: at most 2^14 particles (and as many newborns) per flush, which keeps
    // every histogram piece below 2^32
    constexpr int FLUSH_TILES = (16384 / (BLOCK * PPT)) > 0 ? 16384 / (BLOCK * PPT) : 1;
    int it = 0, since = 0;
    for (int g = blockIdx.x; g < total_tiles; g += gridDim.x, ++it, ++since) {
        // the store of tile g: the CTA's tiles increase, so its store only moves forward
        int seg = cur_seg < 0 ? 0 : cur_seg;
        while (seg + 1 < 2 * n_disc && s_segstart[seg + 1] <= g) ++seg;
        if (seg == cur_seg && since >= FLUSH_TILES) {
            flush();
            since = 0;
        }
        if (seg != cur_seg) {
            since = 0;
            if (cur_seg >= 0) flush();
            const int d = seg >> 1, sp = seg & 1;
            if (tid == 0) {
                const Disc& D = discs[d];
                S.k = consts_of<T>(D);
                S.d = d;
                S.sp = sp;
                S.N = D.N;
                S.n_pts = D.n_pts;
                S.has_see = D.has_see;
                S.leapfrog = D.leapfrog;
                S.n_exc = D.n_exc;
                S.thr = D.thr[sp];
                S.did = D.discharge_id;
                S.n = s_store[seg].n;
                S.cap = D.cap[sp];
                S.bcap = D.bcap;
                S.cin = D.c[in_buf][sp];
                S.pin = D.p[in_buf][sp];
                S.cout = D.c[1 - in_buf][sp];
                S.pout = D.p[1 - in_buf][sp];
                S.bc = D.bc[sp];
                S.bp = D.bp[sp];
                S.sc = D.sc;
                S.sp_ = D.sp_;
                S.Te = D.Te;
                S.Ti = D.Ti;
                S.Dg = D.D[sp];
                S.Dother = D.D[1 - sp];
                S.Qg = D.Q;
                S.cnt = D.cnt;
                S.start = D.start[sp];
                S.K = s_store[seg].K;
                S.M = s_store[seg].M;
                S.D0 = s_store[seg].D0;
                S.ralloc = D.ralloc[sp];
                S.cnt_main = D.cnt_main[sp];
                S.cnt_birth = D.cnt_birth[sp];
                S.cnt_same = D.cnt_same;
                S.slice_tot = D.slice_tot[sp] + (size_t)s_par * 3 * D.slice_n[sp];
            }
            if (tid < NCNT) s_cnt[tid] = 0;
            __syncthreads();
            for (int j = tid; j < h32_words; j += BLOCK) s_h32[j] = 0;
            if (d != cur_d) {
                const T* E = reinterpret_cast<const T*>(discs[d].E);
                for (int j = tid; j <= S.N; j += BLOCK) s_E[j] = E[j];
                cur_d = d;
            }
            cur_seg = seg;
            __syncthreads();
        }

        const int b = it & 1;
        const bool mine = pf[3] != 0;
        const unsigned cs = (unsigned)pf[0];
        const int base = pf[1], end = pf[2];
        if (mine) {  // this tile's chunk: its staged data, then the next tile's prefetch into the other buffer
            if (!mbar_wait(&s_mbar[warp][b], ((unsigned)pf[5] >> b) & 1u)) err |= ERR_TIMEOUT;
        }
        __syncwarp();
        if (lane == 0 && mine) pf[5] ^= 1 << b;
        prefetch(b ^ 1, g + gridDim.x);
        __syncwarp();
        if (mine && !(err & ERR_TIMEOUT)) {
            unsigned char* buf = stage + (size_t)b * sweep_stage_bytes<T, PPT>();
            R* srec = reinterpret_cast<R*>(buf);
            const int32_t* scell = reinterpret_cast<const int32_t*>(buf + REC_BYTES);
            // slots and record offsets fit in 31 bits: the host caps every record buffer below 2^31
            if (S.sp == 0) chunk(cs, base, end - base, srec, scell, IC<0>{});
            else chunk(cs, base, end - base, srec, scell, IC<1>{});
        }
        __syncwarp();
    }
    // copies still in flight (a prefetch is issued only for a tile this CTA takes, so none should
    // be): wait for them, bounded, before the CTA's shared memory goes away
    if (pf[3] && !mbar_wait(&s_mbar[warp][it & 1], ((unsigned)pf[5] >> (it & 1)) & 1u)) err |= ERR_TIMEOUT;
    if (cur_seg >= 0) flush();
    if (err) atomicOr(&s_err, err);
    __syncthreads();
    if (tid == 0 && s_err) atomicOr(&ctl->error, s_err);
}


// ---------------------------------------------------------------------------
// Exact prefix terms of the Poisson solve for both species over a run of nodes: r = sum of the
// deposits D_k, m = sum of k D_k. With R_j = sum_{1<=k<=j} D_k and M_j = sum_{1<=k<=j} k D_k the
// double sum S_{j+1} = sum_{i<=j} R_i equals (j + 1) R_j - M_j, so one scan of plain integer sums
// gives both R and S (no products inside the scan; integer, so any order gives the same).
struct PSum {
    unsigned long long r[2];
    unsigned __int128 m[2];
};
__device__ __forceinline__ void psum_add(PSum& a, const PSum& b) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
        a.r[sp] += b.r[sp];
        a.m[sp] += b.m[sp];
    }
}
__device__ __forceinline__ PSum psum_shfl_up(const PSum& x, int o) {
    PSum y;
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
        y.r[sp] = __shfl_up_sync(FULL, x.r[sp], o);
        const unsigned long long lo = __shfl_up_sync(FULL, (unsigned long long)x.m[sp], o);
        const unsigned long long hi = __shfl_up_sync(FULL, (unsigned long long)(x.m[sp] >> 64), o);
        y.m[sp] = ((unsigned __int128)hi << 64) | lo;
    }
    return y;
}
// Exclusive scan of one PSum per thread over the first NT threads of the block (NT / 32 warps,
// named barrier 1; the other warps of the block do not take part), and the total over all of
// them. s_w: NT / 32 + 1 entries.
template <int NT>
__device__ __forceinline__ PSum block_exclusive_psum(const PSum& own, PSum* s_w, int lane, int warp, PSum& total) {
    constexpr int NW = NT / 32;
    PSum x = own;
#pragma unroll 1
    for (int o = 1; o < 32; o <<= 1) {
        const PSum y = psum_shfl_up(x, o);
        if (lane >= o) psum_add(x, y);
    }
    if (lane == 31) s_w[warp] = x;
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    if (warp == 0) {
        const PSum v = lane < NW ? s_w[lane] : PSum{};
        PSum w = v;
#pragma unroll 1
        for (int o = 1; o < NW; o <<= 1) {
            const PSum y = psum_shfl_up(w, o);
            if (lane >= o) psum_add(w, y);
        }
        if (lane == NW - 1) s_w[NW] = w;
        if (lane < NW) {
#pragma unroll
            for (int sp = 0; sp < 2; ++sp) {  // inclusive -> exclusive
                w.r[sp] -= v.r[sp];
                w.m[sp] -= v.m[sp];
            }
            s_w[lane] = w;
        }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    total = s_w[NW];
    PSum r = s_w[warp];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {  // + this warp's inclusive sum before the thread
        r.r[sp] += x.r[sp] - own.r[sp];
        r.m[sp] += x.m[sp] - own.m[sp];
    }
    return r;
}
// Nearest double of a 128-bit integer below 2^115 in magnitude (two roundings at most).
__device__ __forceinline__ double i128_to_double(__int128 x) {
    const long long hi = (long long)(x >> 64);
    const unsigned long long lo = (unsigned long long)x;
    return __fma_rn((double)hi, 0x1p64, __ull2double_rn(lo));
}

// After a sweep (mode bit 1) and for every solve, one grid (x = slice or role,
// y = store): CTAs x < nsl write the region starts of the chunks of slice x of
// store y (the first slot each chunk's survivors take in the new layout) and
// copy its newborns into the newborn area; CTA x = nsl, y even solves the field
// of discharge y / 2 and accumulates the moments; CTA x = nsl, y odd turns the
// slice sums of discharge y / 2 into the new counts and layouts and clears the
// sums of the other parity for the next sweep. mode bits: 1 layouts after a sweep; 2
// accumulate moments and advance the step; 4 initial solve at t = n dt (load);
// 8 segments only (no solve, deposits kept). The last CTA to finish advances
// the step (mode bit 2) and flips the slice parity (mode bit 1).
template <int BLOCK>
__device__ __forceinline__ void seg_apply(const Disc* __restrict__ discs, Ctl* __restrict__ ctl, int out_buf, int tid, int lane,
                          int warp) {
    constexpr int K = SLICE / BLOCK, NW = BLOCK / 32;
    static_assert(SLICE % BLOCK == 0 && NW <= 32 && NW >= 3, "seg_apply block shape");
    using R = float4;
    __shared__ int s_w[3][NW];
    // the slice's chunk counts (each at most one chunk of slots: 16 bits), loaded coalesced while
    // every thread scans K consecutive chunks
    __shared__ unsigned short s_cnt[3][SLICE];
    const int d = blockIdx.y >> 1, sp = blockIdx.y & 1;
    const Disc& D = discs[d];
    // every field is read before the first store (the stores could otherwise alias them)
    const int CHUNK = D.chunk;
    const int* __restrict__ cnt_m = D.cnt_main[sp];
    const int* __restrict__ cnt_b = D.cnt_birth[sp];
    const int* __restrict__ cnt_s = D.cnt_same;
    int* __restrict__ st = D.start[sp];
    const int q = 1 - sp;  // store of the other-species newborns
    const long long bcap = D.bcap;
    const int rw = D.rec_words;  // record size in 16-byte words
    int32_t* __restrict__ oc_q = D.c[out_buf][q] + D.R0[q];
    R* __restrict__ op_q = reinterpret_cast<R*>(D.p[out_buf][q]) + D.R0[q] * rw;
    int32_t* __restrict__ oc_0 = D.c[out_buf][0] + D.R0[0];
    R* __restrict__ op_0 = reinterpret_cast<R*>(D.p[out_buf][0]) + D.R0[0] * rw;
    const int32_t* __restrict__ bc = D.bc[sp];
    const R* __restrict__ bp = reinterpret_cast<const R*>(D.bp[sp]);
    const int32_t* __restrict__ sc = D.sc;
    const R* __restrict__ spr = reinterpret_cast<const R*>(D.sp_);
    const unsigned* __restrict__ slice0 = D.slice_tot[0];
    const unsigned* __restrict__ slice_s = D.slice_tot[sp];
    const int sn0 = D.slice_n[0], sn_s = D.slice_n[sp];
    const long long chunks = ctl->chunks_in[d][sp];
    const long long t0 = (long long)blockIdx.x * SLICE;
    if (t0 >= chunks) return;
    // output offsets of this slice: the sums of the slices before it (survivors, other-species
    // newborns, same-species newborns); the ion sweep's SEE electrons follow all ionization
    // electrons of the electron sweep
    __shared__ long long s_pre[3];
    if (warp == 0) {
        const int par = ctl->slice_par;
        const unsigned* Tp = slice_s + (size_t)par * 3 * sn_s;
        long long a = 0, b = 0, c = 0;
        for (int k = lane; k < (int)blockIdx.x; k += 32) {
            a += Tp[3 * k + 0];
            b += Tp[3 * k + 1];
            c += Tp[3 * k + 2];
        }
        if (sp == 1) {
            const long long ch0 = ctl->chunks_in[d][0];
            const unsigned* T0 = slice0 + (size_t)par * 3 * sn0;
            for (long long k = lane; k < (ch0 + SLICE - 1) / SLICE; k += 32) b += T0[3 * k + 2];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(FULL, a, o);
            b += __shfl_xor_sync(FULL, b, o);
            c += __shfl_xor_sync(FULL, c, o);
        }
        if (lane == 0) {
            s_pre[0] = a;
            s_pre[1] = b;
            s_pre[2] = c;
        }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int k = i * BLOCK + tid;
        const bool in = t0 + k < chunks;
        s_cnt[0][k] = (unsigned short)(in ? cnt_m[t0 + k] : 0);
        s_cnt[1][k] = (unsigned short)(in ? cnt_b[t0 + k] : 0);
        s_cnt[2][k] = (unsigned short)((in && sp == 0) ? cnt_s[t0 + k] : 0);
    }
    __syncthreads();
    const long long tb = t0 + (long long)tid * K;
    int rm = 0, rb = 0, rs = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        rm += s_cnt[0][tid * K + i];
        rb += s_cnt[1][tid * K + i];
        rs += s_cnt[2][tid * K + i];
    }
    int xm = rm, xb = rb, xs = rs;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ym = __shfl_up_sync(FULL, xm, o), yb = __shfl_up_sync(FULL, xb, o), ys = __shfl_up_sync(FULL, xs, o);
        if (lane >= o) {
            xm += ym;
            xb += yb;
            xs += ys;
        }
    }
    if (lane == 31) {
        s_w[0][warp] = xm;
        s_w[1][warp] = xb;
        s_w[2][warp] = xs;
    }
    __syncthreads();
    if (warp < 3) {  // warp k scans the NW warp sums of count k (NW <= 32)
        const int v = lane < NW ? s_w[warp][lane] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            const int y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane < NW) s_w[warp][lane] = x - v;
    }
    __syncthreads();
    long long em = s_pre[0] + s_w[0][warp] + xm - rm;
    const long long eb0 = s_pre[1] + s_w[1][warp] + xb - rb;  // this thread's first newborn of each kind
    const long long es0 = s_pre[2] + s_w[2][warp] + xs - rs;
#pragma unroll 1
    for (int i = 0; i < K; ++i) {  // rolled: this code runs once per step, from a cold instruction cache
        const long long t = tb + i;
        if (t < chunks) st[t] = (int)em;  // the first slot of region t of the new layout
        em += s_cnt[0][tid * K + i];
    }
    // The newborns of the warp's chunks, copied by the whole warp: newborn j of a kind belongs to the
    // last lane u whose first newborn is at or before j (a search over the lanes' starts), and within
    // lane u's K chunks to the one whose running count passes j. All lanes load, then all store.
    int err = 0;
#pragma unroll 1
    for (int kind = 0; kind < 2; ++kind) {
        if (kind == 1 && sp != 0) break;  // same-species newborns: the electron sweep's only
        const int row = kind == 0 ? 1 : 2;
        const long long e0 = kind == 0 ? eb0 : es0;
        const int r = kind == 0 ? rb : rs;
        const int32_t* __restrict__ cin = kind == 0 ? bc : sc;
        const R* __restrict__ pin = kind == 0 ? bp : spr;
        int32_t* __restrict__ cdst = kind == 0 ? oc_q : oc_0;
        R* __restrict__ pdst = kind == 0 ? op_q : op_0;
        const long long w0 = __shfl_sync(FULL, e0, 0), w1 = __shfl_sync(FULL, e0 + r, 31);
        for (long long jb = w0; jb < w1; jb += 32) {
            const long long j = jb + lane;
            int u = 0;  // last lane with start <= j
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long su = __shfl_sync(FULL, e0, u + o);
                if (su <= j) u += o;
            }
            const long long su = __shfl_sync(FULL, e0, u);
            if (j >= w1) continue;
            long long rem = j - su;
            int ci = 0;
            const int tw = (warp * 32 + u) * K;  // lane u's first chunk in the slice
            while (ci < K - 1 && rem >= s_cnt[row][tw + ci]) rem -= s_cnt[row][tw + ci++];
            const long long srcr = (t0 + tw + ci) * CHUNK + rem;
            if (j < bcap) {  // records of one (FP32) or two (FP64) 16-byte words; no runtime-indexed array
                const int cv = cin[srcr];
                const R r0 = pin[srcr * rw];
                const R r1 = rw == 2 ? pin[srcr * rw + 1] : r0;
                cdst[j] = cv;
                pdst[j * rw] = r0;
                if (rw == 2) pdst[j * rw + 1] = r1;
            } else {
                err = ERR_CAPACITY;
            }
        }
    }
    if (err) atomicOr(&ctl->error, err);
}

// Field of one discharge after its deposits are complete (the field role of k_post; all
// POST_BLOCK threads of the CTA). Poisson, Eq. (poisson): phi_{j-1} - 2 phi_j + phi_{j+1} = -r_j with
// r_j = rho_j dx^2 / eps0, phi_0 = V_rf sin(2 pi f t), phi_N = 0. With R_j = sum_{k<=j} r_k and
// S_j = sum_{i<j} R_i: phi_j = phi_0 + j g_1 - S_j, g_1 = (phi_N - phi_0 + S_N) / N. R and S are
// linear in the deposits: R_j = c_i IR_i,j - c_e IR_e,j, S_{j+1} = c_i IS_i,j - c_e IS_e,j with the
// exact integer sums IR_s,j = sum_{1<=k<=j} D_s,k (64 bits: a store holds below 2^30 particles of
// 2^32 each) and IS_s,j = sum_{i<=j} IR_s,i (128 bits), from one scan of plain sums (PSum). FP64
// (slow on this part) is used once per node, with no division (host reciprocals).
constexpr int POST_BLOCK = 512;  // threads per k_post CTA
constexpr int FIELD_SCAN = 256;  // threads of the integer scan

// Discharge current density over step n (section "Boundary conditions", equation for J(t)):
// J = eps0 dE/dt + e0 (Gamma_i - Gamma_e), with the particle fluxes counted positive towards +z
// from the step's absorbed and emitted superparticles: at z = 0 an absorbed ion (moving towards
// -z) carries -e w_i, an absorbed electron +e w_e, an emitted secondary electron (towards +z)
// -e w_e; at z = d the absorbed particles' signs flip and emitted electrons move towards -z.
// FP64, by one thread of the field CTA after the new electrode fields Ew are known. The initial
// solve of a load (mode bit 4) only records the fields and counters. On a full step the current at
// z = 0 is also projected onto the rf period's first harmonic (sin and cos at the step midpoint);
// at the end of a period the amplitude is stored.
__device__ __forceinline__ void discharge_current(const Disc& D, int d, Ctl* ctl, int mode, long long step,
                                               const double* Ew) {
    // counters as scalars (an array here would live in local memory, cold at every step)
    const unsigned long long c0 = D.cnt[CNT_ABS + 0], c1 = D.cnt[CNT_ABS + 1], c2 = D.cnt[CNT_ABS + 2],
                             c3 = D.cnt[CNT_ABS + 3];  // [species][electrode]
    const unsigned long long c4 = D.cnt[CNT_SEE_SIDE], c5 = D.cnt[CNT_SEE_SIDE + 1];
    if (!(mode & 4)) {  // a solve after a sweep (or a stand-alone solve): the current of step n
        double J0 = 0.0, JN = 0.0;  // no earlier solve: no current
        if (ctl->have_solve[d]) {
            const unsigned long long* cs = ctl->cnt_solve[d];
            const double dA0 = (double)(c0 - cs[0]), dA1 = (double)(c1 - cs[1]), dA2 = (double)(c2 - cs[2]),
                         dA3 = (double)(c3 - cs[3]);
            const double dS0 = (double)(c4 - cs[4]), dS1 = (double)(c5 - cs[5]);
            const double we = D.w[0], wi = D.w[1], rdt = D.inv_dt;  // FP64 division is slow on this part
            const double cond0 = E_CHARGE * (we * dA0 - wi * dA2 - we * dS0) * rdt;
            const double condN = E_CHARGE * (wi * dA3 - we * dA1 + we * dS1) * rdt;
            J0 = EPS0 * (Ew[0] - ctl->E_wall[d][0]) * rdt + cond0;
            JN = EPS0 * (Ew[1] - ctl->E_wall[d][1]) * rdt + condN;
        }
        const long long slot = step % D.jh;
        D.J_hist[2 * slot] = J0;
        D.J_hist[2 * slot + 1] = JN;
        if ((mode & 2) && D.jtab && D.steps_per_period > 0) {
            const int spp = D.steps_per_period;
            const int k = (int)(step % spp);
            ctl->J_sum[d][0] += J0 * D.jtab[2 * k];
            ctl->J_sum[d][1] += J0 * D.jtab[2 * k + 1];
            if (k == spp - 1) {
                const double a = 2.0 * ctl->J_sum[d][0] / spp, b = 2.0 * ctl->J_sum[d][1] / spp;
                const double amp = sqrt(a * a + b * b);
                D.J_amp[(step / spp) % PERIOD_HIST] = amp;
                D.V_hist[(step / spp) % PERIOD_HIST] = D.V_rf * ctl->V_scale[d];
                const double J0 = ctl->J_drive[d];
                if (J0 > 0.0 && amp > 0.0) ctl->V_scale[d] = ctl->V_scale[d] * (J0 / amp);  // Eq. (adaptivevoltage)
                ctl->J_sum[d][0] = 0.0;
                ctl->J_sum[d][1] = 0.0;
            }
        }
    }
    ctl->have_solve[d] = 1;
    ctl->E_wall[d][0] = Ew[0];
    ctl->E_wall[d][1] = Ew[1];
    unsigned long long* cs = ctl->cnt_solve[d];
    cs[0] = c0;
    cs[1] = c1;
    cs[2] = c2;
    cs[3] = c3;
    cs[4] = c4;
    cs[5] = c5;
}
template <typename T>
__device__ __forceinline__ void field_solve(const Disc& D, int d, Ctl* __restrict__ ctl, int mode, int tid, int lane,
                                            int warp, double* s_f, int max_N, PSum* s_ps, double* s_Ew) {
    constexpr int BLOCK = POST_BLOCK;
    // every field of the discharge is read before the first store
    const int N = D.N;
    unsigned long long* __restrict__ De = D.D[0];
    unsigned long long* __restrict__ Di = D.D[1];
    unsigned long long* __restrict__ Qd = D.Q;
    unsigned long long* __restrict__ Dp = D.Dprev;
    unsigned __int128* __restrict__ aDe = D.acc_D[0];
    unsigned __int128* __restrict__ aDi = D.acc_D[1];
    unsigned __int128* __restrict__ aQ = D.acc_Q;
    unsigned __int128* __restrict__ aDp = D.acc_Dprev;
    double* __restrict__ phi = D.phi;
    double* __restrict__ E64 = D.E64;
    T* __restrict__ Ef = reinterpret_cast<T*>(D.E);
    const double pr0 = D.pc_r[0], pr1 = D.pc_r[1], pw0 = D.pc_w[0], pw1 = D.pc_w[1];
    const double inv_dx = D.inv_dx, m_inv_2dx = D.m_inv_2dx, hdx_eps = D.hdx_eps, inv_N = D.inv_N;
    const long long step = ctl->step;
    const long long ns = (mode & 4) ? step : step + 1;  // time level of the solve
    const double V0 = (D.V0tab ? D.V0tab[ns % D.steps_per_period]
                               : D.V_rf * sin(2.0 * PI_D * D.f_rf * ((double)ns * D.dt))) *
                      ctl->V_scale[d];
    // one pass over the nodes: stage the deposits in shared memory, accumulate the moments (mode
    // bit 2) and hand the next sweep zeroed deposit arrays
    unsigned long long* sde = reinterpret_cast<unsigned long long*>(s_f);
    unsigned long long* sdi = sde + (max_N + 1);
    for (int j = tid; j <= N; j += BLOCK) {
        const unsigned long long de = De[j], di = Di[j], q = Qd[j], dp = Dp[j];
        if (mode & 2) {
            const unsigned __int128 a0 = aDe[j], a1 = aDi[j], aq = aQ[j], ap = aDp[j];
            aDe[j] = a0 + de;
            aDi[j] = a1 + di;
            aQ[j] = aq + q;
            aDp[j] = ap + dp;
        }
        Dp[j] = de;
        De[j] = 0;
        Di[j] = 0;
        Qd[j] = 0;
        sde[j] = de;
        sdi[j] = di;
    }
    if (tid == 0 && (mode & 2)) ctl->acc_steps[d] += 1;
    __syncthreads();
    if (tid >= FIELD_SCAN) return;
    // thread t owns nodes [lo, hi); node 0 carries no deposit term; node N is done by the owner of N - 1
    const int per = (N + FIELD_SCAN - 1) / FIELD_SCAN;
    const int lo = min(N, tid * per), hi = min(N, lo + per);
    PSum own{};
    for (int j = max(lo, 1); j < hi; ++j) {
        own.r[0] += sde[j];
        own.r[1] += sdi[j];
        own.m[0] += (unsigned __int128)j * sde[j];
        own.m[1] += (unsigned __int128)j * sdi[j];
    }
    PSum tot;
    PSum run = block_exclusive_psum<FIELD_SCAN>(own, s_ps, lane, warp, tot);
    // R_j -> r_j sums in FP64 (Rr), S_{j+1} = (j + 1) R_j - M_j -> FP64 (Sx), as c_i x_i - c_e x_e
    auto Rr_of = [&](const PSum& p) {
        return __fma_rn(pr1, (double)(long long)p.r[1], -pr0 * (double)(long long)p.r[0]);
    };
    auto Sx_of = [&](const PSum& p, int j1) {  // S at node j1 from the sums through node j1 - 1
        const __int128 S0 = (__int128)((unsigned __int128)j1 * p.r[0] - p.m[0]);
        const __int128 S1 = (__int128)((unsigned __int128)j1 * p.r[1] - p.m[1]);
        return __fma_rn(pr1, i128_to_double(S1), -pr0 * i128_to_double(S0));
    };
    const double g1 = (Sx_of(tot, N) - V0) * inv_N;  // S_N from the totals
    // g_j = phi_j - phi_{j-1} = g_1 - R_{j-1}; node field E_j = -(g_j + g_{j+1}) / (2 dx) inside
    // (the central difference of phi, without the cancellation of large phi values), and Gauss's
    // law over the half cells at the electrodes
    double Rprev = Rr_of(run);      // R_{lo-1}
    double Sprev = Sx_of(run, lo);  // S_lo
    for (int j = lo; j < hi; ++j) {
        if (j >= 1) {
            const unsigned long long e = sde[j], i = sdi[j];
            run.r[0] += e;
            run.r[1] += i;
            run.m[0] += (unsigned __int128)j * e;
            run.m[1] += (unsigned __int128)j * i;
        }
        const double Rj = Rr_of(run);
        double ph, E;
        if (j == 0) {
            ph = V0;
            const double rw = __fma_rn(pw1, (double)sdi[0], -pw0 * (double)sde[0]);
            E = -g1 * inv_dx - rw * hdx_eps;
            ctl->E0_last[d] = E;
            s_Ew[0] = E;
        } else {
            ph = V0 + (double)j * g1 - Sprev;
            E = ((g1 - Rprev) + (g1 - Rj)) * m_inv_2dx;
        }
        phi[j] = ph;
        E64[j] = E;
        Ef[j] = (T)E;
        Rprev = Rj;
        Sprev = Sx_of(run, j + 1);
    }
    if (lo < hi && hi == N) {  // the electrode at x = L
        const double rw = __fma_rn(pw1, (double)sdi[N], -pw0 * (double)sde[N]);
        const double E = -(g1 - Rprev) * inv_dx + rw * hdx_eps;
        phi[N] = 0.0;
        E64[N] = E;
        Ef[N] = (T)E;
        s_Ew[1] = E;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(FIELD_SCAN) : "memory");
    if (tid == 0) discharge_current(D, d, ctl, mode, step, s_Ew);
}

template <typename T>
__global__ void __launch_bounds__(POST_BLOCK, 1) k_post(const Disc* __restrict__ discs, int n_disc, Ctl* __restrict__ ctl,
                                                     int out_buf, int mode, int nsl, int max_N) {
    constexpr int BLOCK = POST_BLOCK;
    extern __shared__ __align__(16) double s_f[];
    __shared__ PSum s_ps[FIELD_SCAN / 32 + 1];
    __shared__ double s_Ew[2];
    __shared__ int s_err;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    grid_dep_sync();
    if (tid == 0) s_err = 0;
    __syncthreads();
    if ((int)blockIdx.x < nsl) {
        seg_apply<BLOCK>(discs, ctl, out_buf, tid, lane, warp);
    } else if ((mode & 1) && (blockIdx.y & 1) == 1) {  // store totals of discharge y / 2
        if (warp == 0) {
            int e2 = 0;
            store_totals(discs[blockIdx.y >> 1], blockIdx.y >> 1, ctl, lane, ctl->slice_par, (mode & 2) != 0, out_buf,
                         e2);
            if (e2 && lane == 0) atomicOr(&s_err, e2);
        }
    } else if (!(mode & 8) && (blockIdx.y & 1) == 0) {
        field_solve<T>(discs[blockIdx.y >> 1], blockIdx.y >> 1, ctl, mode, tid, lane, warp, s_f, max_N, s_ps, s_Ew);
    }
    __syncthreads();
    // the last CTA advances the step (bit 2) and, after a sweep, the slice parity. Every CTA has
    // consumed its reads of both before its count (data dependence), and the last CTA reads no other
    // CTA's results, so no fence: the kernel boundary publishes everything
    if (tid == 0) {
        if (s_err) atomicOr(&ctl->error, s_err);
        const unsigned prev = atomicAdd(&ctl->fin_done, 1u);
        if (prev == gridDim.x * gridDim.y - 1) {
            ctl->fin_done = 0;
            if (mode & 2) ctl->step = ctl->step + 1;
            if (mode & 1) ctl->slice_par = ctl->slice_par ^ 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Initial load: uniform positions, Maxwellian velocities (Philox calls 0xF0,
// 0xF1 at step 0). grid.y = store (d, species).
template <typename T>
__global__ void k_load(const Disc* __restrict__ discs, Ctl* __restrict__ ctl, int buf, unsigned long long seed) {
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const Disc& D = discs[d];
    const Consts<T>& K = consts_of<T>(D);
    const long long n = ctl->count[d][sp];
    const int N = D.N;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const U4 r = draw(seed, (uint32_t)k, 0, sp, 0xF0, D.discharge_id);
        const U4 q = draw(seed, (uint32_t)k, 0, sp, 0xF1, D.discharge_id);
        const T x = mul_((T)u01(r.x), (T)N);
        int c = (int)x;
        T f;
        if (c >= N) {
            c = N - 1;
            f = one_minus_ulp<T>();
        } else {
            f = sub_(x, (T)c);
        }
        float n0, n1, n2, n3;
        box_muller(u01(r.y), u01(r.z), n0, n1);
        box_muller(u01(r.w), u01(q.x), n2, n3);
        const T sg = K.sig0[sp];
        store_rec<T>(D.c[buf][sp], D.p[buf][sp], k, Part<T>{c, f, mul_(sg, (T)n0), mul_(sg, (T)n1), mul_(sg, (T)n2)});
    }
}

// Warm start: particles sampled from profiles on a uniform grid of P points
// (calls 0xF2, 0xF3 at step 0): position by inverse of the piecewise-constant
// CDF, electrons Maxwellian at kT = 2/3 <eps>(z), ions at T_i0.
template <typename T>
struct WarmDev {
    const T* cdf[2];  // per species, P entries, cdf[0] = 0, cdf[P-1] = 1
    const T* eps;     // P entries, eV
    int P, pad_;
    T scale;          // N / (P - 1)
    T K23;            // 2 e / (3 m_e)
};

template <typename T>
__global__ void k_load_profile(const Disc* __restrict__ discs, Ctl* __restrict__ ctl, int buf,
                               unsigned long long seed, const WarmDev<T>* __restrict__ warm) {
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const Disc& D = discs[d];
    const WarmDev<T>& W = warm[d];
    const long long n = ctl->count[d][sp];
    const int N = D.N, P = W.P;
    const T* cdf = W.cdf[sp];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const U4 r = draw(seed, (uint32_t)k, 0, sp, 0xF2, D.discharge_id);
        const U4 q = draw(seed, (uint32_t)k, 0, sp, 0xF3, D.discharge_id);
        const T u = (T)u01(r.x);
        int lo = 0, hi = P - 2;  // largest j in [0, P-2] with cdf[j] <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cdf[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        const int j = lo;
        const T den = sub_(cdf[j + 1], cdf[j]);
        T t = den > (T)0 ? div_(sub_(u, cdf[j]), den) : (T)0;
        if (t >= (T)1) t = one_minus_ulp<T>();
        const T x = mul_(add_((T)j, t), W.scale);
        int c = (int)x;
        T f;
        if (c >= N) {
            c = N - 1;
            f = one_minus_ulp<T>();
        } else {
            f = sub_(x, (T)c);
        }
        T sg;
        if (sp == 0) {
            T el = fma_(t, sub_(W.eps[j + 1], W.eps[j]), W.eps[j]);
            if (!(el > (T)0)) el = (T)0;
            sg = sqrt_(mul_(el, W.K23));
        } else {
            sg = consts_of<T>(D).sig0[1];
        }
        float n0, n1, n2, n3;
        box_muller(u01(r.y), u01(r.z), n0, n1);
        box_muller(u01(r.w), u01(q.x), n2, n3);
        store_rec<T>(D.c[buf][sp], D.p[buf][sp], k, Part<T>{c, f, mul_(sg, (T)n0), mul_(sg, (T)n1), mul_(sg, (T)n2)});
    }
}

// CIC deposit of whole stores (used after a load or a state upload).
template <typename T>
__global__ void k_deposit(const Disc* __restrict__ discs, const Ctl* __restrict__ ctl, int buf, int max_N) {
    extern __shared__ __align__(16) unsigned long long s_h[];
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const Disc& D = discs[d];
    const int N = D.N;
    for (int j = threadIdx.x; j <= N; j += blockDim.x) s_h[j] = 0;
    __syncthreads();
    const long long n = ctl->count[d][sp];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        T f, vx, vy, vz;
        load_rec<T>(D.p[buf][sp], k, f, vx, vy, vz);
        shist_add(s_h, D.c[buf][sp][k], cic_F(f));
    }
    __syncthreads();
    for (int j = threadIdx.x; j <= N; j += blockDim.x)
        if (s_h[j]) atomicAdd(&D.D[sp][j], s_h[j]);
}

// Half back-kick after the initial solve: stored v_z = v_0 - (q/m) E_0 dt / 2.
template <typename T>
__global__ void k_backkick(const Disc* __restrict__ discs, const Ctl* __restrict__ ctl, int buf) {
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const Disc& D = discs[d];
    const Consts<T>& K = consts_of<T>(D);
    const T* E = reinterpret_cast<const T*>(D.E);
    const long long n = ctl->count[d][sp];
    using R = typename Rec<T>::type;
    R* P = reinterpret_cast<R*>(D.p[buf][sp]);
    const T mK = -K.K[sp];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int c = D.c[buf][sp][k];
        R r = P[k];
        const T e0 = E[c], e1 = E[c + 1];
        const T ef = fma_(r.x, sub_(e1, e0), e0);
        r.w = fma_(mK, ef, r.w);
        P[k] = r;
    }
}

// Rate-coefficient tables sigma_j * v, cumulative over processes, rounded to T.
// Electrons: v = sqrt(2 e eps / m_e). Ions: g = sqrt(4 e eps / M) (c.m. energy).
template <typename T>
__global__ void k_tables(int n_pts, int n_proc, double de, double M, const double* __restrict__ se,
                         const double* __restrict__ si, T* __restrict__ Te, T* __restrict__ Ti,
                         unsigned long long* __restrict__ kmax) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pts) return;
    const double eps = (double)k * de;
    const double v = sqrt(2.0 * E_CHARGE * eps / M_ELEC);
    double cum = 0.0;
    for (int j = 0; j < 4; ++j) {
        if (j < n_proc) cum = __dadd_rn(cum, __dmul_rn(se[(size_t)k * n_proc + j], v));
        Te[(size_t)k * 4 + j] = (T)cum;
    }
    const double gr = sqrt(4.0 * E_CHARGE * eps / M);
    cum = 0.0;
    for (int j = 0; j < 2; ++j) {
        cum = __dadd_rn(cum, __dmul_rn(si[(size_t)k * 2 + j], gr));
        Ti[(size_t)k * 2 + j] = (T)cum;
    }
    atomicMax(&kmax[0], (unsigned long long)__double_as_longlong((double)Te[(size_t)k * 4 + 3]));
    atomicMax(&kmax[1], (unsigned long long)__double_as_longlong((double)Ti[(size_t)k * 2 + 1]));
}

// ---------------------------------------------------------------------------
// Chunk k of a store with layout L (see Lay): first slot, slots and record offset. Regions take
// their first and end slots from the start table.
struct ChunkDesc {
    long long src;
    int base, cnt;
};
__device__ __forceinline__ ChunkDesc chunk_desc(const Lay& L, long long n, const int* st, long long k, int chunk) {
    ChunkDesc c;
    if (k < L.K) {
        c.src = k * chunk;
        c.base = __ldg(st + k);
        c.cnt = __ldg(st + k + 1) - c.base;
    } else {
        const long long j = k - L.K;
        c.src = L.D0 + j * chunk;
        c.base = (int)(L.M + j * chunk);
        c.cnt = (int)min((long long)chunk, n - c.base);
    }
    return c;
}

// ---------------------------------------------------------------------------
// Kinetic diagnostics of the electrons (section "Results": the EEDF, the fast-electron density and
// the profiles at a fixed rf phase), taken from the store at (x_n, v_n) before the sweep of step n.
// Per electron: the gathered field and the first half kick as in the sweep, the energy in 2^-12 eV
// clamped at 2^26, then per node array an integer value X rounded in the particle precision and
// split like the charge (X - rn(X f) to node c, rn(X f) to node c + 1). Units of X:
//   DG_D  2^32 per particle (the deposit's F split)     DG_U  energy, 2^-12 eV
//   DG_V  v_z, 2^-6 m/s                                  DG_W  energy x v_z, formed as (eq v_z) 2^-16
//   DG_K  ionization rate coefficient, 2^-72 m^3/s       DG_F  2^32 per electron above the threshold
//   DG_FA as DG_F, at the EEDF samples
// Sums are exact (int64, mod 2^64); warp groups of equal cells are reduced in three 22/22/20-bit
// parts, so no partial sum overflows 32 bits.
template <typename T> __device__ __forceinline__ long long rint_ll(T x);
template <> __device__ __forceinline__ long long rint_ll<float>(float x) { return __float2ll_rn(x); }
template <> __device__ __forceinline__ long long rint_ll<double>(double x) { return __double2ll_rn(x); }

__device__ __forceinline__ unsigned long long group_sum64(unsigned peers, unsigned long long v) {
    const unsigned a = __reduce_add_sync(peers, (unsigned)(v & 0x3FFFFFu));
    const unsigned b = __reduce_add_sync(peers, (unsigned)((v >> 22) & 0x3FFFFFu));
    const unsigned c = __reduce_add_sync(peers, (unsigned)(v >> 44));
    return (unsigned long long)a + ((unsigned long long)b << 22) + ((unsigned long long)c << 44);
}

// a to node key, b to node key + 1 of a shared histogram: reduced over the lanes of `peers` and
// added by the leader, or (lanewise) added lane by lane.
__device__ __forceinline__ void warp_add_pair(unsigned long long* h, int key, unsigned long long a,
                                              unsigned long long b, unsigned peers, bool leader, bool lanewise) {
    if (lanewise) {
        if (key >= 0) {
            if (a) sadd64(&h[key], a);
            if (b) sadd64(&h[key + 1], b);
        }
        return;
    }
    const unsigned long long sa = group_sum64(peers, a), sb = group_sum64(peers, b);
    if (leader && key >= 0) {
        if (sa) sadd64(&h[key], sa);
        if (sb) sadd64(&h[key + 1], sb);
    }
}

template <typename T>
__device__ __forceinline__ void split_rint(T x, T f, unsigned long long& a, unsigned long long& b) {
    const long long X = rint_ll<T>(x), Xh = rint_ll<T>(mul_(x, f));
    a = (unsigned long long)(X - Xh);
    b = (unsigned long long)Xh;
}

template <typename T4r, typename T>
__device__ __forceinline__ T col4(const T4r& r, int j) {
    return j == 0 ? r.x : j == 1 ? r.y : j == 2 ? r.z : r.w;
}

constexpr int DIAG_BLOCK = 256, DIAG_NW = DIAG_BLOCK / 32;

template <typename T>
__global__ void __launch_bounds__(DIAG_BLOCK) k_diag(const Disc* __restrict__ discs, const Ctl* __restrict__ ctl,
                                                     int buf, DiagArgs A) {
    grid_dep_sync();
    extern __shared__ __align__(16) unsigned long long s_dg[];  // [arrays of the mask][N + 1], EEDF [bins] u32
    using R = typename Rec<T>::type;
    using Row4 = typename T4<T>::type;
    const int d = blockIdx.y;
    const Disc& D = discs[d];
    const int N = D.N, N1 = N + 1, CHUNK = D.chunk, RPC = CHUNK / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool phase = A.mode & DIAG_PHASE, sample = A.mode & DIAG_SAMPLE;
    const int nar = __popc(A.mask), nb = sample ? A.bins : 0;
    unsigned* s_eedf = reinterpret_cast<unsigned*>(s_dg + (size_t)nar * N1);
    for (int j = tid; j < nar * N1; j += DIAG_BLOCK) s_dg[j] = 0;
    for (int j = tid; j < nb; j += DIAG_BLOCK) s_eedf[j] = 0;
    const T* E = reinterpret_cast<const T*>(D.E);
    if (blockIdx.x == 0 && (A.mode & DIAG_COUNT)) {  // field sum of the snapshot, snapshot and sample counts
        if (phase)
            for (int j = tid; j <= N; j += DIAG_BLOCK) D.dg_E[j] += (double)E[j];
        if (tid == 0) {
            if (phase) D.dg_n[0] += 1;
            if (sample) D.dg_n[1] += 1;
        }
    }
    __syncthreads();
    unsigned long long* h[DG_ARRAYS];
#pragma unroll
    for (int a = 0; a < DG_ARRAYS; ++a) h[a] = s_dg + (size_t)__popc(A.mask & ((1u << a) - 1u)) * N1;
    const bool mD = A.mask & (1u << DG_D), mU = A.mask & (1u << DG_U), mV = A.mask & (1u << DG_V),
               mW = A.mask & (1u << DG_W), mK = A.mask & (1u << DG_K), mF = A.mask & (1u << DG_F),
               mFa = A.mask & (1u << DG_FA);
    const Consts<T>& K = consts_of<T>(D);
    const T thr = (T)A.thr, inv_bin = (T)A.inv_bin, top = (T)(D.n_pts - 1), binsT = (T)A.bins;
    const int ciz = 1 + D.n_exc;  // ionization column of the cumulative electron table
    const Row4* Te = reinterpret_cast<const Row4*>(D.Te);
    const long long n = ctl->count[d][0];
    const Lay L = ctl->lay[d][0][buf];
    const long long chunks = chunks_of(L, n, CHUNK);
    const int32_t* __restrict__ cc = D.c[buf][0];
    const R* __restrict__ P = reinterpret_cast<const R*>(D.p[buf][0]);
    for (long long k = (long long)blockIdx.x * DIAG_NW + warp; k < chunks; k += (long long)gridDim.x * DIAG_NW) {
        const ChunkDesc cd = chunk_desc(L, n, D.start[0], k, CHUNK);
        for (int r = 0; r < RPC; ++r) {
            const int i = 32 * r + lane;
            int c = -1;
            T f = 0, vx = 0, vy = 0, vz = 0;
            if (i < cd.cnt) {
                c = cc[cd.src + i];
                const R q = P[cd.src + i];
                f = q.x;
                vx = q.y;
                vy = q.z;
                vz = q.w;
                if (!((unsigned)c < (unsigned)N)) c = -1;
            }
            unsigned long long F = 0, uA = 0, uB = 0, vA = 0, vB = 0, wA = 0, wB = 0, kA = 0, kB = 0;
            bool fast = false;
            int bin = 0;
            if (c >= 0) {
                const T E0 = E[c], E1 = E[c + 1];
                const T ef = fma_(f, sub_(E1, E0), E0);
                vz = fma_(K.K[0], ef, vz);  // v_n
                const T e2 = fma_(vx, vx, fma_(vy, vy, mul_(vz, vz)));
                T eq = mul_(e2, K.kappa_E);
                if (!(eq <= (T)0x1p26)) eq = (T)0x1p26;
                F = cic_F(f);
                fast = eq > thr;
                if (mU) split_rint<T>(eq, f, uA, uB);
                if (mV) split_rint<T>(mul_(vz, (T)64), f, vA, vB);
                if (mW) split_rint<T>(mul_(mul_(eq, vz), (T)0x1p-16), f, wA, wB);
                if (mK) {
                    const T xi = mul_(e2, K.kappa_e);
                    T Cz, Cy;
                    if (!(xi < top)) {
                        const Row4 a = Te[D.n_pts - 1];
                        Cz = col4<Row4, T>(a, ciz);
                        Cy = col4<Row4, T>(a, ciz - 1);
                    } else {
                        const int ii = (int)xi;
                        const T fr = sub_(xi, (T)ii);
                        const Row4 a = Te[ii], b = Te[ii + 1];
                        const T az = col4<Row4, T>(a, ciz), ay = col4<Row4, T>(a, ciz - 1);
                        Cz = fma_(fr, sub_(col4<Row4, T>(b, ciz), az), az);
                        Cy = fma_(fr, sub_(col4<Row4, T>(b, ciz - 1), ay), ay);
                    }
                    split_rint<T>(mul_(sub_(Cz, Cy), (T)0x1p72), f, kA, kB);
                }
                if (sample) {
                    const T xb = mul_(eq, inv_bin);
                    bin = xb < binsT ? (int)xb : A.bins - 1;
                }
            }
            // a row of one cell (common on a cell-sorted store) is reduced across the warp, any other
            // row added lane by lane (grouping by match_any cost more than it saved in the sweep)
            const int c0 = __shfl_sync(FULL, c, 0);
            const bool lanewise = !__all_sync(FULL, c == c0);
            const unsigned peers = FULL;
            const bool leader = lane == 0;
            const unsigned long long dA = c >= 0 ? (1ull << 32) - F : 0ull, dB = c >= 0 ? F : 0ull;
            if (mD) warp_add_pair(h[DG_D], c, dA, dB, peers, leader, lanewise);
            if (mU) warp_add_pair(h[DG_U], c, uA, uB, peers, leader, lanewise);
            if (mV) warp_add_pair(h[DG_V], c, vA, vB, peers, leader, lanewise);
            if (mW) warp_add_pair(h[DG_W], c, wA, wB, peers, leader, lanewise);
            if (mK) warp_add_pair(h[DG_K], c, kA, kB, peers, leader, lanewise);
            if (mF) warp_add_pair(h[DG_F], c, fast ? dA : 0ull, fast ? dB : 0ull, peers, leader, lanewise);
            if (mFa) warp_add_pair(h[DG_FA], c, fast ? dA : 0ull, fast ? dB : 0ull, peers, leader, lanewise);
            if (sample && c >= 0) atomicAdd(&s_eedf[bin], 1u);
        }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < DG_ARRAYS; ++a)
        if (A.mask & (1u << a)) {
            unsigned long long* g = D.dg + (size_t)a * N1;
            for (int j = tid; j < N1; j += DIAG_BLOCK)
                if (h[a][j]) atomicAdd(&g[j], h[a][j]);
        }
    for (int j = tid; j < nb; j += DIAG_BLOCK)
        if (s_eedf[j]) atomicAdd(&D.dg_eedf[j], (unsigned long long)s_eedf[j]);
}

// Stable counting sort by cell. A sort tile is SORT_NW warps of SORT_R rows of 32 slots: warp w of
// tile t walks the store's chunks t SORT_NW CPW + w CPW .. + CPW - 1 (CPW = SORT_R 32 / CHUNK) in
// slot order.
constexpr int SORT_BLOCK = 256, SORT_NW = SORT_BLOCK / 32, SORT_R = 16;
__device__ __forceinline__ long long sort_tiles(long long chunks, int chunk) {
    const long long per = (long long)SORT_NW * (SORT_R * 32 / chunk);
    return (chunks + per - 1) / per;
}

// Stable counting sort of every store by cell:
//   k_sort_count   per tile: each slot's cell and its rank among the tile's
//                  slots of the same cell (in slot order), packed with the cell
//                  into kr[slot], and the tile's cell counts into
//                  hist[seg][t N + c];
//   k_sort_rows    per cell: exclusive scan of the counts over the tiles; the
//                  last CTA of a store scans the cell totals (first slot of
//                  every cell);
//   k_sort_scatter per tile, walking the same chunks: destination = first slot
//                  of its cell + the tile's offset in that cell + its rank; the
//                  sorted buffer's layout is dense.
__global__ void __launch_bounds__(SORT_BLOCK) k_sort_count(const Disc* __restrict__ discs, const Ctl* __restrict__ ctl,
                                                           int buf, unsigned* __restrict__ hist,
                                                           const long long* __restrict__ hoff,
                                                           unsigned* __restrict__ kr_all,
                                                           const long long* __restrict__ eoff, int max_N) {
    grid_dep_sync();
    extern __shared__ __align__(16) unsigned s_w[];  // [SORT_NW][max_N] per-warp counts, then prefixes
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const Disc& D = discs[d];
    const int N = D.N, CHUNK = D.chunk, RPC = CHUNK / 32, CPW = SORT_R / RPC;
    const long long n = ctl->count[d][sp];
    const Lay L = ctl->lay[d][sp][buf];
    const long long chunks = chunks_of(L, n, CHUNK);
    const long long Ts = sort_tiles(chunks, CHUNK);
    const int32_t* __restrict__ cc = D.c[buf][sp];
    const int* st = D.start[sp];
    unsigned* H = hist + hoff[seg];
    unsigned* KR = kr_all + eoff[seg];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned* Wc = s_w + warp * max_N;
    for (long long t = blockIdx.x; t < Ts; t += gridDim.x) {
        for (int j = tid; j < SORT_NW * max_N; j += SORT_BLOCK) s_w[j] = 0;
        __syncthreads();
        const long long k0 = (t * SORT_NW + warp) * CPW;
        unsigned kr[SORT_R];
        int slot[SORT_R];
        ChunkDesc cd{0, 0, 0};
#pragma unroll
        for (int r = 0; r < SORT_R; ++r) {  // all cell loads first
            const int ci = r / RPC, row = r % RPC;
            if (row == 0) cd = (k0 + ci < chunks) ? chunk_desc(L, n, st, k0 + ci, CHUNK) : ChunkDesc{0, 0, 0};
            const int i = 32 * row + lane;
            kr[r] = 0xFFFFu;
            slot[r] = -1;
            if (i < cd.cnt) {
                kr[r] = (unsigned)__ldcs(cc + cd.src + i);  // checked below, after all loads are issued
                slot[r] = cd.base + i;
            }
        }
#pragma unroll
        for (int r = 0; r < SORT_R; ++r) {  // rank among the warp's equal cells so far
            if (kr[r] >= (unsigned)N) kr[r] = 0xFFFFu;  // past the store, or a corrupt cell index: not placed
            const int k = (int)kr[r];
            const unsigned peers = __match_any_sync(FULL, k);
            if (k < N) {
                const unsigned b = Wc[k];
                kr[r] |= (b + __popc(peers & lt)) << 16;
                __syncwarp(peers);
                if (lane == __ffs(peers) - 1) Wc[k] = b + __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        for (int j = tid; j < N; j += SORT_BLOCK) {  // per cell: prefix over the warps, tile count
            unsigned run = 0;
#pragma unroll
            for (int w = 0; w < SORT_NW; ++w) {
                const unsigned v = s_w[w * max_N + j];
                s_w[w * max_N + j] = run;
                run += v;
            }
            H[(size_t)t * N + j] = run;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < SORT_R; ++r) {
            if (slot[r] >= 0) {
                const int k = (int)(kr[r] & 0xFFFFu);
                KR[slot[r]] = k < N ? (unsigned)k | ((Wc[k] + (kr[r] >> 16)) << 16) : 0xFFFFu;
            }
        }
        __syncthreads();
    }
}

// Exclusive scan of one store's N row totals in place -> the first slot of every cell (1024
// threads; the totals were written by other CTAs of the same grid, so they are read from L2).
__device__ __forceinline__ void cells_scan(unsigned* a, int N) {
    __shared__ unsigned s_v[MAXN];
    __shared__ unsigned s_w[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = tid; j < N; j += 1024) s_v[j] = __ldcg(a + j);
    __syncthreads();
    const int per = (N + 1023) / 1024, lo = tid * per, hi = min(N, lo + per);
    unsigned run = 0;
    for (int j = lo; j < hi; ++j) run += s_v[j];
    unsigned x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const unsigned w = s_w[lane];
        unsigned y = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(FULL, y, o);
            if (lane >= o) y += t;
        }
        s_w[lane] = y - w;
    }
    __syncthreads();
    unsigned e = s_w[warp] + x - run;
    for (int j = lo; j < hi; ++j) {
        const unsigned v = s_v[j];
        a[j] = e;
        e += v;
    }
}

// Per (store, group of 32 cells): exclusive scan over the tiles in place (lane = cell, each warp
// a contiguous range of tiles, so rows are read 128 bytes at a time); row totals out.
__global__ void __launch_bounds__(1024) k_sort_rows(const Disc* __restrict__ discs, Ctl* __restrict__ ctl, int buf,
                                                    unsigned* __restrict__ hist, const long long* __restrict__ hoff,
                                                    unsigned* __restrict__ tot) {
    grid_dep_sync();
    __shared__ unsigned s_sum[32][33];
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const int N = discs[d].N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    if (blockIdx.x * 32 >= N) return;
    const unsigned Ts = (unsigned)sort_tiles(chunks_of(ctl->lay[d][sp][buf], ctl->count[d][sp], discs[d].chunk),
                                             discs[d].chunk);
    unsigned* H = hist + hoff[seg];
    const unsigned per = (Ts + 31) / 32, t0 = min(Ts, warp * per), t1 = min(Ts, t0 + per);
    unsigned sum = 0;
    if (c < N)
        for (unsigned t = t0; t < t1; ++t) sum += H[(size_t)t * N + c];
    s_sum[warp][lane] = sum;
    __syncthreads();
    unsigned pre = 0;
    for (int w = 0; w < warp; ++w) pre += s_sum[w][lane];
    if (warp == 31 && c < N) tot[(long long)seg * MAXN + c] = pre + sum;
    if (c < N)
        for (unsigned t = t0; t < t1; ++t) {
            const unsigned v = H[(size_t)t * N + c];
            H[(size_t)t * N + c] = pre;
            pre += v;
        }
    // the last CTA of the store turns the row totals into the first slot of every cell
    __shared__ int s_last;
    if (warp == 31) __threadfence();  // this CTA's totals, before its count
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&ctl->sort_rows_done[d][sp], 1u);
        s_last = prev == (unsigned)((N + 31) / 32 - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    cells_scan(tot + (long long)seg * MAXN, N);
    if (threadIdx.x == 0) ctl->sort_rows_done[d][sp] = 0;
}

template <typename T>
__global__ void __launch_bounds__(SORT_BLOCK) k_sort_scatter(const Disc* __restrict__ discs,
                                                             Ctl* __restrict__ ctl, int src, int dst,
                                                             const unsigned* __restrict__ hist,
                                                             const long long* __restrict__ hoff,
                                                             const unsigned* __restrict__ tot,
                                                             const unsigned* __restrict__ kr_all,
                                                             const long long* __restrict__ eoff) {
    grid_dep_sync();
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const Disc& D = discs[d];
    const int N = D.N, CHUNK = D.chunk, RPC = CHUNK / 32, CPW = SORT_R / RPC;
    const long long n = ctl->count[d][sp];
    const Lay L = ctl->lay[d][sp][src];
    const long long chunks = chunks_of(L, n, CHUNK);
    const long long Ts = sort_tiles(chunks, CHUNK);
    using R = typename Rec<T>::type;
    const R* __restrict__ ps = reinterpret_cast<const R*>(D.p[src][sp]);
    R* __restrict__ pd = reinterpret_cast<R*>(D.p[dst][sp]);
    int32_t* __restrict__ cd = D.c[dst][sp];
    const int* st = D.start[sp];
    const unsigned* H = hist + hoff[seg];
    const unsigned* cstart = tot + (long long)seg * MAXN;
    const unsigned* KR = kr_all + eoff[seg];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->lay[d][sp][dst] = Lay{0, 0, 0, 0};  // the sorted store is dense
    for (long long t = blockIdx.x; t < Ts; t += gridDim.x) {
        const long long k0 = (t * SORT_NW + warp) * CPW;
        for (int ci = 0; ci < CPW && k0 + ci < chunks; ++ci) {
            const ChunkDesc c = chunk_desc(L, n, st, k0 + ci, CHUNK);
            for (int row = 0; row < RPC; ++row) {
                const int i = 32 * row + lane;
                if (i >= c.cnt) continue;
                const unsigned kr = __ldcs(KR + c.base + i);
                const int k = (int)(kr & 0xFFFFu);
                if (k >= N) continue;  // a corrupt cell index (reported by the sweep): dropped
                const unsigned long long o = (unsigned long long)cstart[k] + H[(size_t)t * N + k] + (kr >> 16);
                if (o < (unsigned long long)n) {
                    cd[o] = k;
                    pd[o] = ps[c.src + i];
                }
            }
        }
    }
}

// Order-preserving repack of every store into a dense buffer (the slots keep their order): bounds
// the number of regions when the sort runs rarely or never. One warp per chunk.
template <typename T>
__global__ void k_repack(const Disc* __restrict__ discs, Ctl* __restrict__ ctl, int src, int dst) {
    grid_dep_sync();
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const Disc& D = discs[d];
    const int CHUNK = D.chunk;
    const long long n = ctl->count[d][sp];
    const Lay L = ctl->lay[d][sp][src];
    const long long chunks = chunks_of(L, n, CHUNK);
    using R = typename Rec<T>::type;
    const R* __restrict__ ps = reinterpret_cast<const R*>(D.p[src][sp]);
    const int32_t* __restrict__ cs_ = D.c[src][sp];
    R* __restrict__ pd = reinterpret_cast<R*>(D.p[dst][sp]);
    int32_t* __restrict__ cd = D.c[dst][sp];
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = ((long long)gridDim.x * blockDim.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->lay[d][sp][dst] = Lay{0, 0, 0, 0};
    for (long long k = w0; k < chunks; k += nw) {
        const ChunkDesc c = chunk_desc(L, n, D.start[sp], k, CHUNK);
        for (int i = lane; i < c.cnt; i += 32) {
            cd[c.base + i] = __ldcs(cs_ + c.src + i);
            pd[c.base + i] = ps[c.src + i];
        }
    }
}

// 16-byte groups of the SoA arrays of a state transfer: W consecutive particles, their cells in
// one W-wide integer vector and each real array in one 16-byte vector.
template <typename T>
struct XferVec;
template <>
struct XferVec<float> {
    typedef int4 CV;
    typedef float4 RV;
    static constexpr int W = 4;
};
template <>
struct XferVec<double> {
    typedef int2 CV;
    typedef double2 RV;
    static constexpr int W = 2;
};

__device__ __forceinline__ bool aligned16(const void* a, const void* b, const void* c, const void* d,
                                          const void* e) {
    return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(c) |
             reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(e)) & 15) == 0;
}

// State upload: SoA arrays (device staging, or the caller's mapped pinned host arrays) -> the
// store's records; cells outside [0, N) are counted in *bad. With 16-byte aligned arrays each
// thread reads whole 16-byte groups (over the host link, wide loads keep more bytes in flight
// per thread), the ragged tail one by one.
template <typename T>
__global__ void k_pack_state(const Disc* __restrict__ discs, int d, int sp, int buf, long long n,
                             const int32_t* __restrict__ c, const T* __restrict__ f, const T* __restrict__ vx,
                             const T* __restrict__ vy, const T* __restrict__ vz, unsigned* __restrict__ bad) {
    typedef XferVec<T> X;
    const Disc& D = discs[d];
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
    const long long groups = aligned16(c, f, vx, vy, vz) ? n / X::W : 0;
    unsigned nbad = 0;
    for (long long g = t0; g < groups; g += nt) {
        const typename X::CV cv = reinterpret_cast<const typename X::CV*>(c)[g];
        const typename X::RV a = reinterpret_cast<const typename X::RV*>(f)[g];
        const typename X::RV b = reinterpret_cast<const typename X::RV*>(vx)[g];
        const typename X::RV e = reinterpret_cast<const typename X::RV*>(vy)[g];
        const typename X::RV h = reinterpret_cast<const typename X::RV*>(vz)[g];
        const int* cs = reinterpret_cast<const int*>(&cv);
        const T *as = reinterpret_cast<const T*>(&a), *bs = reinterpret_cast<const T*>(&b);
        const T *es = reinterpret_cast<const T*>(&e), *hs = reinterpret_cast<const T*>(&h);
#pragma unroll
        for (int k = 0; k < X::W; ++k) {
            nbad += (unsigned)cs[k] >= (unsigned)D.N;
            store_rec<T>(D.c[buf][sp], D.p[buf][sp], (unsigned)(g * X::W + k), Part<T>{cs[k], as[k], bs[k], es[k], hs[k]});
        }
    }
    for (long long i = groups * X::W + t0; i < n; i += nt) {
        const int ci = c[i];
        nbad += (unsigned)ci >= (unsigned)D.N;
        store_rec<T>(D.c[buf][sp], D.p[buf][sp], (unsigned)i, Part<T>{ci, f[i], vx[i], vy[i], vz[i]});
    }
    if (nbad) atomicAdd(bad, nbad);
}

// Position i of the state in the store: regions (binary search of the start table; empty regions
// share their start) and then the dense part by offset.
__device__ __forceinline__ long long state_slot(const Lay& L, const int* st, int chunk, long long i) {
    if (i >= L.M) return L.D0 + (i - L.M);
    int lo = 0, hi = L.K - 1;  // last region with start <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long long)st[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return (long long)lo * chunk + (i - st[lo]);
}

// State download: the store, read through its layout -> SoA arrays (device staging, or the
// caller's mapped pinned host arrays; null outputs are skipped). The count comes from the control
// block; above cap nothing is written. With 16-byte aligned outputs each thread writes whole
// 16-byte groups.
template <typename T>
__global__ void k_unpack_state(const Disc* __restrict__ discs, const Ctl* __restrict__ ctl, int d, int sp, int buf,
                               long long cap, int32_t* __restrict__ c, T* __restrict__ f, T* __restrict__ vx,
                               T* __restrict__ vy, T* __restrict__ vz) {
    typedef XferVec<T> X;
    const Disc& D = discs[d];
    const long long n = ctl->count[d][sp];
    if (n > cap) return;
    const Lay L = ctl->lay[d][sp][buf];
    const int* st = D.start[sp];
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
    const long long groups = aligned16(c, f, vx, vy, vz) ? n / X::W : 0;  // null is aligned
    for (long long g = t0; g < groups; g += nt) {
        typename X::CV cv;
        typename X::RV a, b, e, h;
        int* cs = reinterpret_cast<int*>(&cv);
        T *as = reinterpret_cast<T*>(&a), *bs = reinterpret_cast<T*>(&b);
        T *es = reinterpret_cast<T*>(&e), *hs = reinterpret_cast<T*>(&h);
#pragma unroll
        for (int k = 0; k < X::W; ++k) {
            const long long o = state_slot(L, st, D.chunk, g * X::W + k);
            load_rec<T>(D.p[buf][sp], (unsigned)o, as[k], bs[k], es[k], hs[k]);
            cs[k] = D.c[buf][sp][o];
        }
        if (c) reinterpret_cast<typename X::CV*>(c)[g] = cv;
        if (f) reinterpret_cast<typename X::RV*>(f)[g] = a;
        if (vx) reinterpret_cast<typename X::RV*>(vx)[g] = b;
        if (vy) reinterpret_cast<typename X::RV*>(vy)[g] = e;
        if (vz) reinterpret_cast<typename X::RV*>(vz)[g] = h;
    }
    for (long long i = groups * X::W + t0; i < n; i += nt) {
        const long long o = state_slot(L, st, D.chunk, i);
        T a, b, e, g;
        load_rec<T>(D.p[buf][sp], (unsigned)o, a, b, e, g);
        if (c) c[i] = D.c[buf][sp][o];
        if (f) f[i] = a;
        if (vx) vx[i] = b;
        if (vy) vy[i] = e;
        if (vz) vz[i] = g;
    }
}

// End of a state upload (one thread): the store holds n particles, or none if the pack kernel found a
// cell out of range, dense in buffer buf.
__global__ void k_finish_upload(const Disc* __restrict__ discs, Ctl* __restrict__ ctl, int d, int sp, long long n,
                                const unsigned* __restrict__ bad, int buf) {
    ctl->count[d][sp] = *bad ? 0 : n;
    ctl->lay[d][sp][buf] = Lay{0, 0, 0, 0};
}
// Every store dense in buffer buf (after a load).
__global__ void k_set_dense(const Disc* __restrict__ discs, int n_disc, Ctl* __restrict__ ctl, int buf) {
    grid_dep_sync();
    const int i = threadIdx.x;
    if (i >= 2 * n_disc) return;
    ctl->lay[i >> 1][i & 1][buf] = Lay{0, 0, 0, 0};
}

// ---------------------------------------------------------------------------
__global__ void k_debug_philox(long long n, const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1,
                               uint32_t* __restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const U4 r = philox4x32_10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

__global__ void k_debug_math(long long n, const float* __restrict__ x, const float* __restrict__ y,
                             float* __restrict__ lg, float* __restrict__ sn, float* __restrict__ cs) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    lg[i] = own_logf(x[i]);
    float s, c;
    own_sincospif(y[i], s, c);
    sn[i] = s;
    cs[i] = c;
}

}  // namespace pic

// ---------------------------------------------------------------------------
// Launch wrappers used by the host runtime.
#include <mutex>
#include <vector>

#include "pic_launch.h"

namespace pic {

// Bounded-wait check: one mbarrier expecting a single arrival. With arrive = 0 nothing arrives, so
// the wait gives up after `tries` polls and the kernel reports ERR_TIMEOUT in *out; nothing is in
// flight when it returns. With arrive = 1 the thread arrives first and the wait succeeds.
__global__ void k_debug_wait(int arrive, int tries, int* out) {
    __shared__ __align__(8) unsigned long long mb;
    if (threadIdx.x == 0) mbar_init(&mb);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&mb)) : "memory");
        *out = mbar_wait(&mb, 0u, tries) ? 0 : ERR_TIMEOUT;
    }
}

// Raises a kernel's dynamic shared-memory limit once per (kernel, size). Kernels
// are told apart by their address (instantiations can share a type).
template <typename K>
static cudaError_t smem_attr(K kern, size_t smem) {
    static std::mutex mu;
    static std::vector<std::pair<const void*, size_t>> done;
    std::lock_guard<std::mutex> lk(mu);
    const void* key = reinterpret_cast<const void*>(kern);
    for (auto& p : done)
        if (p.first == key) {
            if (smem <= p.second) return cudaSuccess;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) p.second = smem;
            return e;
        }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done.push_back({key, smem});
    return e;
}

// Launch with programmatic stream serialization: the grid may be scheduled while the kernel before
// it in the stream is still finishing (it takes SMs as they free up), and every such kernel starts
// with grid_dep_wait(), which returns once that kernel has completed and its memory is visible. So
// the kernel-to-kernel gap of a step shrinks while the ordering stays that of plain launches.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <typename T, int BLOCK, int PPT>
static cudaError_t launch_sweep_t(const SweepLaunch& L) {
    const size_t smem = sweep_smem<T, BLOCK, PPT>(L.max_N, L.n_disc);
    auto kern = k_sweep<T, BLOCK, PPT>;
    cudaError_t e = smem_attr(kern, smem);
    if (e != cudaSuccess) return e;
    e = launch_pdl(kern, dim3(L.grid), dim3(BLOCK), smem, L.stream, L.discs, L.n_disc, L.ctl, L.in_buf, L.seed,
                   L.max_N);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_sweep_p(const SweepLaunch& L) {
    if (L.block == 512) {
        if (L.ppt == 2) return launch_sweep_t<T, 512, 2>(L);
        return launch_sweep_t<T, 512, 4>(L);
    }
    if (L.block == 128) {
        if (L.ppt == 2) return launch_sweep_t<T, 128, 2>(L);
        if (L.ppt == 8) return launch_sweep_t<T, 128, 8>(L);
        return launch_sweep_t<T, 128, 4>(L);
    }
    if (L.ppt == 2) return launch_sweep_t<T, 256, 2>(L);
    if (L.ppt == 8) return launch_sweep_t<T, 256, 8>(L);
    return launch_sweep_t<T, 256, 4>(L);
}

cudaError_t launch_sweep(const SweepLaunch& L) {
    return L.fp64 ? launch_sweep_p<double>(L) : launch_sweep_p<float>(L);
}

template <typename T, int BLOCK, int PPT>
static int occ_t(int max_N, int n_disc) {
    int nb = 0;
    const size_t smem = sweep_smem<T, BLOCK, PPT>(max_N, n_disc);
    smem_attr(k_sweep<T, BLOCK, PPT>, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<T, BLOCK, PPT>, BLOCK, smem);
    return nb;
}
template <typename T>
static int occ_p(int block, int ppt, int max_N, int n_disc) {
    if (block == 512) {
        if (ppt == 2) return occ_t<T, 512, 2>(max_N, n_disc);
        return occ_t<T, 512, 4>(max_N, n_disc);
    }
    if (block == 128) {
        if (ppt == 2) return occ_t<T, 128, 2>(max_N, n_disc);
        if (ppt == 8) return occ_t<T, 128, 8>(max_N, n_disc);
        return occ_t<T, 128, 4>(max_N, n_disc);
    }
    if (ppt == 2) return occ_t<T, 256, 2>(max_N, n_disc);
    if (ppt == 8) return occ_t<T, 256, 8>(max_N, n_disc);
    return occ_t<T, 256, 4>(max_N, n_disc);
}
int sweep_occupancy(int fp64, int block, int ppt, int max_N, int n_disc) {
    return fp64 ? occ_p<double>(block, ppt, max_N, n_disc) : occ_p<float>(block, ppt, max_N, n_disc);
}

cudaError_t launch_finalize(int fp64, const Disc* discs, int n_disc, Ctl* ctl, int out_buf, int mode, int max_slices,
                            int max_N, cudaStream_t st) {
    const size_t smem = sizeof(double) * 2 * ((size_t)max_N + 1);
    const int nsl = (mode & 1) ? (max_slices > 0 ? max_slices : 1) : 0;
    const dim3 grid(nsl + 1, 2 * n_disc);
    if (fp64) {
        smem_attr(k_post<double>, smem);
        return launch_pdl(k_post<double>, grid, dim3(POST_BLOCK), smem, st, discs, n_disc, ctl, out_buf, mode, nsl,
                          max_N);
    } else {
        smem_attr(k_post<float>, smem);
        return launch_pdl(k_post<float>, grid, dim3(POST_BLOCK), smem, st, discs, n_disc, ctl, out_buf, mode, nsl,
                          max_N);
    }
}

cudaError_t launch_load(int fp64, const Disc* discs, int n_disc, Ctl* ctl, int buf, unsigned long long seed,
                        int grid_x, cudaStream_t st) {
    dim3 g(grid_x, 2 * n_disc);
    if (fp64) k_load<double><<<g, 256, 0, st>>>(discs, ctl, buf, seed);
    else k_load<float><<<g, 256, 0, st>>>(discs, ctl, buf, seed);
    return cudaGetLastError();
}

cudaError_t launch_load_profile(int fp64, const Disc* discs, int n_disc, Ctl* ctl, int buf, unsigned long long seed,
                                const void* warm, int grid_x, cudaStream_t st) {
    dim3 g(grid_x, 2 * n_disc);
    if (fp64) k_load_profile<double><<<g, 256, 0, st>>>(discs, ctl, buf, seed, (const WarmDev<double>*)warm);
    else k_load_profile<float><<<g, 256, 0, st>>>(discs, ctl, buf, seed, (const WarmDev<float>*)warm);
    return cudaGetLastError();
}

size_t warm_desc_bytes(int fp64) { return fp64 ? sizeof(WarmDev<double>) : sizeof(WarmDev<float>); }

void warm_desc_fill(int fp64, void* out, const void* cdf_e, const void* cdf_i, const void* eps, int P, double scale,
                    double K23) {
    if (fp64) {
        WarmDev<double> w{};
        w.cdf[0] = (const double*)cdf_e;
        w.cdf[1] = (const double*)cdf_i;
        w.eps = (const double*)eps;
        w.P = P;
        w.scale = scale;
        w.K23 = K23;
        *(WarmDev<double>*)out = w;
    } else {
        WarmDev<float> w{};
        w.cdf[0] = (const float*)cdf_e;
        w.cdf[1] = (const float*)cdf_i;
        w.eps = (const float*)eps;
        w.P = P;
        w.scale = (float)scale;
        w.K23 = (float)K23;
        *(WarmDev<float>*)out = w;
    }
}

cudaError_t launch_deposit(int fp64, const Disc* discs, int n_disc, const Ctl* ctl, int buf, int max_N, int grid_x,
                           cudaStream_t st) {
    dim3 g(grid_x, 2 * n_disc);
    const size_t smem = sizeof(unsigned long long) * (max_N + 1);
    if (fp64) k_deposit<double><<<g, 256, smem, st>>>(discs, ctl, buf, max_N);
    else k_deposit<float><<<g, 256, smem, st>>>(discs, ctl, buf, max_N);
    return cudaGetLastError();
}

cudaError_t launch_backkick(int fp64, const Disc* discs, int n_disc, const Ctl* ctl, int buf, int grid_x,
                            cudaStream_t st) {
    dim3 g(grid_x, 2 * n_disc);
    if (fp64) k_backkick<double><<<g, 256, 0, st>>>(discs, ctl, buf);
    else k_backkick<float><<<g, 256, 0, st>>>(discs, ctl, buf);
    return cudaGetLastError();
}

cudaError_t launch_tables(int fp64, int n_pts, int n_proc, double de, double M, const double* se, const double* si,
                          void* Te, void* Ti, unsigned long long* kmax, cudaStream_t st) {
    const int g = (n_pts + 255) / 256;
    if (fp64) k_tables<double><<<g, 256, 0, st>>>(n_pts, n_proc, de, M, se, si, (double*)Te, (double*)Ti, kmax);
    else k_tables<float><<<g, 256, 0, st>>>(n_pts, n_proc, de, M, se, si, (float*)Te, (float*)Ti, kmax);
    return cudaGetLastError();
}

cudaError_t launch_sort(int fp64, const Disc* discs, int n_disc, Ctl* ctl, int src, int dst, unsigned* hist,
                        const long long* hoff, unsigned* tot, unsigned* kr, const long long* eoff, int max_N,
                        int grid_x, cudaStream_t st) {
    dim3 g(grid_x, 2 * n_disc);
    const size_t smem = sizeof(unsigned) * SORT_NW * max_N;
    cudaError_t e = smem_attr(k_sort_count, smem);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_sort_count, g, dim3(SORT_BLOCK), smem, st, discs, ctl, src, hist, hoff, kr, eoff, max_N);
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_sort_rows, dim3((max_N + 31) / 32, 2 * n_disc), dim3(1024), 0, st, discs, ctl, src, hist, hoff,
                   tot);
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (fp64)
        return launch_pdl(k_sort_scatter<double>, g, dim3(SORT_BLOCK), 0, st, discs, ctl, src, dst, hist, hoff, tot, kr,
                          eoff);
    return launch_pdl(k_sort_scatter<float>, g, dim3(SORT_BLOCK), 0, st, discs, ctl, src, dst, hist, hoff, tot, kr,
                      eoff);
}

cudaError_t launch_repack(int fp64, const Disc* discs, int n_disc, Ctl* ctl, int src, int dst, int grid_x,
                          cudaStream_t st) {
    const dim3 g(grid_x, 2 * n_disc);
    if (fp64) return launch_pdl(k_repack<double>, g, dim3(256), 0, st, discs, ctl, src, dst);
    return launch_pdl(k_repack<float>, g, dim3(256), 0, st, discs, ctl, src, dst);
}

cudaError_t launch_pack_state(int fp64, const Disc* discs, int d, int sp, int buf, long long n, const int32_t* c,
                              const void* const v[4], unsigned* bad, int grid, cudaStream_t st) {
    if (fp64)
        k_pack_state<double><<<grid, 256, 0, st>>>(discs, d, sp, buf, n, c, (const double*)v[0], (const double*)v[1],
                                                   (const double*)v[2], (const double*)v[3], bad);
    else
        k_pack_state<float><<<grid, 256, 0, st>>>(discs, d, sp, buf, n, c, (const float*)v[0], (const float*)v[1],
                                                  (const float*)v[2], (const float*)v[3], bad);
    return cudaGetLastError();
}

cudaError_t launch_unpack_state(int fp64, const Disc* discs, const Ctl* ctl, int d, int sp, int buf, long long cap,
                                int32_t* c, void* const v[4], int grid, cudaStream_t st) {
    if (fp64)
        k_unpack_state<double><<<grid, 256, 0, st>>>(discs, ctl, d, sp, buf, cap, c, (double*)v[0], (double*)v[1],
                                                     (double*)v[2], (double*)v[3]);
    else
        k_unpack_state<float><<<grid, 256, 0, st>>>(discs, ctl, d, sp, buf, cap, c, (float*)v[0], (float*)v[1],
                                                    (float*)v[2], (float*)v[3]);
    return cudaGetLastError();
}


long long sort_tile_chunks(int chunk) { return (long long)SORT_NW * (SORT_R * 32 / chunk); }

cudaError_t launch_finish_upload(const Disc* discs, Ctl* ctl, int d, int sp, long long n, const unsigned* bad,
                                 int buf, cudaStream_t st) {
    k_finish_upload<<<1, 1, 0, st>>>(discs, ctl, d, sp, n, bad, buf);
    return cudaGetLastError();
}

// Dynamic shared memory of a k_diag launch: its node arrays and, for a sample, the EEDF (bins > 0).
size_t diag_smem(int max_N, unsigned mask, int bins) {
    return (size_t)__builtin_popcount(mask) * 8 * ((size_t)max_N + 1) + 4 * (size_t)bins;
}

cudaError_t launch_diag(int fp64, const Disc* discs, int n_disc, const Ctl* ctl, int buf, const DiagArgs& A,
                        int max_N, int grid_x, cudaStream_t st) {
    const size_t smem = diag_smem(max_N, A.mask, (A.mode & DIAG_SAMPLE) ? A.bins : 0);
    const dim3 g(grid_x, n_disc);
    if (fp64) {
        cudaError_t e = smem_attr(k_diag<double>, smem);
        if (e != cudaSuccess) return e;
        return launch_pdl(k_diag<double>, g, dim3(DIAG_BLOCK), smem, st, discs, ctl, buf, A);
    }
    cudaError_t e = smem_attr(k_diag<float>, smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_diag<float>, g, dim3(DIAG_BLOCK), smem, st, discs, ctl, buf, A);
}

cudaError_t launch_set_dense(const Disc* discs, int n_disc, Ctl* ctl, int buf, cudaStream_t st) {
    return launch_pdl(k_set_dense, dim3(1), dim3(128), 0, st, discs, n_disc, ctl, buf);
}

cudaError_t launch_debug_wait(int arrive, int tries, int* out, cudaStream_t st) {
    k_debug_wait<<<1, 32, 0, st>>>(arrive, tries, out);
    return cudaGetLastError();
}

cudaError_t launch_debug_philox(long long n, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out,
                                cudaStream_t st) {
    k_debug_philox<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, ctr, k0, k1, out);
    return cudaGetLastError();
}
cudaError_t launch_debug_math(long long n, const float* x, const float* y, float* lg, float* sn, float* cs,
                              cudaStream_t st) {
    k_debug_math<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, y, lg, sn, cs);
    return cudaGetLastError();
}

}  // namespace pic
