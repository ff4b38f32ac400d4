// pic_kernels.cu -- CUDA kernels (sm_103a) of the 1d3v PIC/MCC time step of
// arXiv:1608.04601, section "PIC/MCC simulation procedure".
//
// One time step is two launches (and the sort every K steps):
//   k_sweep     persistent; every CTA takes tiles of particles in increasing
//               order from a global dispenser. Per particle: CIC gather of E_n
//               (node field held in shared memory), half kick, null-collision
//               MCC on Philox streams, half kick, drift, wall test. A block
//               scan orders each tile's outputs (particles in slot order, each
//               followed by its same-species newborn), written into the tile's
//               own region of the output buffer; no tile waits for another.
//               CIC deposit into a shared-memory int64 histogram, flushed
//               with global atomics.
//   k_finalize  one CTA per discharge: the new segment tables (an exclusive
//               scan of the per-tile output counts), births of the other
//               species compacted behind them, Poisson (Eq. poisson, rf
//               Dirichlet boundary) in FP64 by two block scans, node field,
//               cycle-average accumulators.
//   sort        every K steps: stable counting sort of each store by cell
//               into a dense store.
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

template <typename T>
struct Part {
    int c;
    T f, vx, vy, vz;
};

// Segment (one store of one discharge) as seen by a sweep CTA.
template <typename T>
struct Seg {
    Consts<T> k;
    int d, sp, N, n_pts, has_see, n_exc;
    uint32_t thr, did;
    long long n, cap, bcap, tile0, ntiles;
    const int32_t* cin;
    const void* pin;
    int32_t* cout;
    void* pout;
    int32_t* bc;
    void* bp;
    const void* Te;
    const void* Ti;
    unsigned long long* Dg;
    unsigned long long* Dother;
    unsigned long long* Qg;
    unsigned long long* cnt;
    const int* seg_start;
    const int* seg_src;
    const int* first_seg;
    int nseg;
    int* cnt_main;
    int* cnt_birth;
};

// Window of the segment table staged in shared memory for one tile: segments
// k0 .. k0+nw-1 and the start of segment k0+nw.
constexpr int SEGWIN = 32;
struct SegWin {
    int k0, nw;
    int start[SEGWIN + 1];
    int src[SEGWIN];
};

// Loaded by one warp: the window starting at segment k0.
__device__ __forceinline__ void seg_window_load(SegWin& W, const int* __restrict__ seg_start,
                                                const int* __restrict__ seg_src, int nseg, int k0, int lane) {
    const int nw = min(SEGWIN, nseg - k0);
    if (lane == 0) {
        W.k0 = k0;
        W.nw = nw;
        W.start[SEGWIN] = 0x7FFFFFFF;
    }
    const int k = k0 + lane;
    W.start[lane] = (lane <= nw && k <= nseg) ? seg_start[k] : 0x7FFFFFFF;
    W.src[lane] = (lane < nw) ? seg_src[k] : 0;
    if (lane == 0 && nw == SEGWIN) W.start[SEGWIN] = seg_start[k0 + SEGWIN];
}

// Buffer offset of a slot: the last segment whose start is <= slot holds it.
__device__ __forceinline__ long long seg_offset(const SegWin& W, const int* __restrict__ seg_start,
                                                const int* __restrict__ seg_src, int nseg, long long slot) {
    if (slot < (long long)W.start[1]) return (long long)W.src[0] + (slot - W.start[0]);  // first segment
    if (slot < (long long)W.start[W.nw]) {
        int lo = 0, hi = W.nw - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((long long)W.start[mid] <= slot) lo = mid;
            else hi = mid - 1;
        }
        return (long long)W.src[lo] + (slot - W.start[lo]);
    }
    int lo = W.k0 + W.nw, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long long)seg_start[mid] <= slot) lo = mid;
        else hi = mid - 1;
    }
    return (long long)seg_src[lo] + (slot - seg_start[lo]);
}

// Drift x_{n+1} = x_n + v_z dt in cell units. Returns -1 (inside) with the new
// (cell, offset), or the electrode reached (0: z = 0, 1: z = d).
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

// Warp-aggregated shared-memory histogram update. key < 0: nothing. Lanes with
// equal keys are grouped (match_any); each group's sums are reduced in 32-bit
// parts (redux) and its first lane applies them:
//   deposit (PAIR = false): v = 2^40 + F  ->  node key += count 2^32 - sum F, node key+1 += sum F
//   moment  (PAIR = true):  v = lo + hi 2^32 (lo, hi < 2^26) -> node key += sum lo, key+1 += sum hi
template <bool PAIR>
__device__ __forceinline__ void warp_hist(unsigned long long* h, int key, unsigned long long v, int lane) {
    const unsigned peers = __match_any_sync(FULL, key);
    const bool leader = lane == __ffs(peers) - 1;
    if (PAIR) {
        const unsigned lo = __reduce_add_sync(peers, (unsigned)v);
        const unsigned hi = __reduce_add_sync(peers, (unsigned)(v >> 32));
        if (leader && key >= 0) {
            if (lo) sadd64(&h[key], lo);
            if (hi) sadd64(&h[key + 1], hi);
        }
    } else {
        const unsigned long long F = v & ((1ull << 40) - 1);  // <= 2^32
        const unsigned fh = __reduce_add_sync(peers, (unsigned)(F >> 16));
        const unsigned fl = __reduce_add_sync(peers, (unsigned)(F & 0xFFFFu));
        if (leader && key >= 0) {
            const unsigned long long sF = ((unsigned long long)fh << 16) + fl;
            sadd64(&h[key], ((unsigned long long)__popc(peers) << 32) - sF);
            if (sF) sadd64(&h[key + 1], sF);
        }
    }
}

// One collision candidate, queued by its warp in shared memory: the owner
// writes the particle (cell, offset, gathered field, v_n); the lane that
// processes the collision writes back the new velocity and the newborns after
// their first drift.
template <typename T>
struct QEnt {
    uint32_t slot;
    int c;
    uint32_t out;     // bit1 same-species newborn stays, bit2 other-species birth stays
    int pad_;
    T f, ef;
    T vx, vy, vz;     // in: v_n; out: velocity after the collision
    Part<T> p1, p2;   // newborns (same species, other species) at x_{n+1}
};

// The collision of a queued candidate (null-collision method: process
// selection against the cumulative rate tables, then the kinematics).
template <typename T>
__device__ __noinline__ void collide(const Seg<T>& S, QEnt<T>& q, long long step, unsigned long long seed,
                                     unsigned long long* sH, unsigned* sC, int& err) {
    using Row4 = typename T4<T>::type;
    using Row2 = typename T4<T>::two;
    const Consts<T>& K = S.k;
    const int N = S.N;
    const uint32_t slot = q.slot;
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
            T nx, ny, nz;
            if (j == 0) {  // elastic, target at rest: v' = beta v + (1-beta)|v| n
                const T g = sqrt_(e2);
                iso_dir(u01(r.z), u01(r.w), nx, ny, nz);
                const T og = mul_(K.omb, g);
                vx = fma_(K.beta, vx, mul_(og, nx));
                vy = fma_(K.beta, vy, mul_(og, ny));
                vz = fma_(K.beta, vz, mul_(og, nz));
                atomicAdd(&sC[CNT_COLL_E + 0], 1u);
            } else if (j <= S.n_exc) {  // excitation of level j
                const T e2n = sub_(e2, K.de2_exc[j - 1]);
                if (e2n > (T)0) {
                    const T sp = sqrt_(e2n);
                    iso_dir(u01(r.z), u01(r.w), nx, ny, nz);
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
                    iso_dir(u01(r.z), u01(r.w), nx, ny, nz);
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
            cvz = fma_(K.K[0], q.ef, cvz);
            int side = drift(N, K.dtdx, q.c, q.f, cvz, cn, fn, err);
            if (side < 0) {
                q.p1 = Part<T>{cn, fn, cvx, cvy, cvz};
                shist_add(sH, cn, cic_F(fn));
                out |= 2u;
            } else {
                atomicAdd(&sC[CNT_ABS + side], 1u);
            }
            ivz = fma_(K.K[1], q.ef, ivz);
            side = drift(N, K.dtdx, q.c, q.f, ivz, cn, fn, err);
            if (side < 0) {
                q.p2 = Part<T>{cn, fn, ivx, ivy, ivz};
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
    q.out = out;
}

// Secondary electron of an ion absorbed at electrode `side` (added option).
template <typename T>
__device__ __noinline__ bool emit_see(const Seg<T>& S, uint32_t slot, long long step, unsigned long long seed,
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
    return true;
}

template <typename T>
__device__ __forceinline__ void store_rec(int32_t* c, void* p, long long i, const Part<T>& q);
template <>
__device__ __forceinline__ void store_rec<float>(int32_t* c, void* p, long long i, const Part<float>& q) {
    c[i] = q.c;
    reinterpret_cast<float4*>(p)[i] = make_float4(q.f, q.vx, q.vy, q.vz);
}
template <>
__device__ __forceinline__ void store_rec<double>(int32_t* c, void* p, long long i, const Part<double>& q) {
    c[i] = q.c;
    double2* pp = reinterpret_cast<double2*>(p) + 2 * i;
    pp[0] = make_double2(q.f, q.vx);
    pp[1] = make_double2(q.vy, q.vz);
}

template <typename T>
__device__ __forceinline__ void load_rec(const void* p, long long i, T& f, T& vx, T& vy, T& vz);
template <>
__device__ __forceinline__ void load_rec<float>(const void* p, long long i, float& f, float& vx, float& vy,
                                                float& vz) {
    const float4 a = __ldcs(reinterpret_cast<const float4*>(p) + i);
    f = a.x; vx = a.y; vy = a.z; vz = a.w;
}
template <>
__device__ __forceinline__ void load_rec<double>(const void* p, long long i, double& f, double& vx, double& vy,
                                                 double& vz) {
    const double2* pp = reinterpret_cast<const double2*>(p) + 2 * i;
    const double2 a = __ldcs(pp), b = __ldcs(pp + 1);
    f = a.x; vx = a.y; vy = b.x; vz = b.y;
}

// Dynamic shared memory of the sweep: histogram and energy moment (u64, N+1
// each), the node field (T, N+1), then the warps' candidate queues.
template <typename T>
__host__ __device__ constexpr size_t sweep_queue_offset(int max_N) {
    return (((size_t)(max_N + 1) * (16 + sizeof(T)) + 15) / 16) * 16;
}
template <typename T, int BLOCK, int PPT>
__host__ __device__ constexpr size_t sweep_smem(int max_N) {
    return sweep_queue_offset<T>(max_N) + sizeof(QEnt<T>) * (BLOCK / 32) * 32 * (PPT < 2 ? PPT : 2);
}

// ---------------------------------------------------------------------------
// The sweep. Persistent CTAs take tiles of TILE = BLOCK x PPT slots of every
// store (discharge, species) in increasing order from a global dispenser.
// Tile t of a store reads its slots through the store's segment table and
// writes its outputs, in slot order, into its own region of the output buffer:
// same-species outputs at [2 TILE t, ...), other-species births at [TILE t, ...)
// of the birth buffer; it records both counts. No tile waits for another.
template <typename T, int BLOCK, int PPT>
__global__ void __launch_bounds__(BLOCK, (sizeof(T) == 4 ? 512 : 256) / BLOCK)
    k_sweep(const Disc* __restrict__ discs, int n_disc, Ctl* __restrict__ ctl, int in_buf, unsigned long long seed,
            int max_N) {
    constexpr int TILE = BLOCK * PPT;
    constexpr int NW = BLOCK / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* s_hist = reinterpret_cast<unsigned long long*>(smem_raw);
    unsigned long long* s_Q = s_hist + (max_N + 1);
    T* s_E = reinterpret_cast<T*>(s_Q + (max_N + 1));
    QEnt<T>* s_q = reinterpret_cast<QEnt<T>*>(smem_raw + sweep_queue_offset<T>(max_N));

    __shared__ long long s_segstart[2 * MAXD + 1];
    __shared__ Seg<T> S;
    __shared__ SegWin W;
    __shared__ unsigned int s_tile;
    __shared__ long long s_step;
    constexpr int BATCH = PPT < 2 ? PPT : 2;   // iterations whose candidates share one queue pass
    constexpr int QCAP = 32 * BATCH;           // queue entries per warp
    __shared__ uint32_t s_wsum[BATCH][NW];
    __shared__ uint32_t s_ktot[BATCH];
    __shared__ unsigned s_cnt[NCNT];
    __shared__ int s_err;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        long long acc = 0;
        for (int s = 0; s < 2 * n_disc; ++s) {
            s_segstart[s] = acc;
            const long long n = ctl->count[s >> 1][s & 1];
            acc += (n + TILE - 1) / TILE;
        }
        s_segstart[2 * n_disc] = acc;
        s_step = ctl->step;
        s_err = 0;
    }
    __syncthreads();
    const long long total_tiles = s_segstart[2 * n_disc];
    const long long step = s_step;
    int cur_seg = -1, cur_d = -1;
    int err = 0;

    auto flush = [&]() {
        __syncthreads();
        for (int j = tid; j <= S.N; j += BLOCK) {
            const unsigned long long h = s_hist[j];
            if (h) atomicAdd(&S.Dg[j], h);
            if (S.sp == 0) {
                const unsigned long long q = s_Q[j];
                if (q) atomicAdd(&S.Qg[j], q);
            }
        }
        if (tid < NCNT && s_cnt[tid]) atomicAdd(&S.cnt[tid], (unsigned long long)s_cnt[tid]);
        __syncthreads();
    };

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&ctl->tile_ctr, 1u);
        __syncthreads();
        const long long g = s_tile;
        if (g >= total_tiles) break;
        int seg = 0;
        {
            int lo = 0, hi = 2 * n_disc - 1;  // largest store with segstart <= g
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_segstart[mid] <= g) lo = mid;
                else hi = mid - 1;
            }
            seg = lo;
        }
        if (seg != cur_seg) {
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
                S.n_exc = D.n_exc;
                S.thr = D.thr[sp];
                S.did = D.discharge_id;
                S.n = ctl->count[d][sp];
                S.cap = D.cap[sp];
                S.bcap = D.bcap;
                S.tile0 = s_segstart[seg];
                S.ntiles = s_segstart[seg + 1] - s_segstart[seg];
                S.cin = D.c[in_buf][sp];
                S.pin = D.p[in_buf][sp];
                S.cout = D.c[1 - in_buf][sp];
                S.pout = D.p[1 - in_buf][sp];
                S.bc = D.bc[sp];
                S.bp = D.bp[sp];
                S.Te = D.Te;
                S.Ti = D.Ti;
                S.Dg = D.D[sp];
                S.Dother = D.D[1 - sp];
                S.Qg = D.Q;
                S.cnt = D.cnt;
                S.seg_start = D.seg_start[sp];
                S.seg_src = D.seg_src[sp];
                S.first_seg = D.first_seg[sp];
                S.nseg = ctl->nseg[d][sp];
                S.cnt_main = D.cnt_main[sp];
                S.cnt_birth = D.cnt_birth[sp];
            }
            if (tid < NCNT) s_cnt[tid] = 0;
            __syncthreads();
            for (int j = tid; j <= S.N; j += BLOCK) {
                s_hist[j] = 0;
                s_Q[j] = 0;
            }
            if (d != cur_d) {
                const T* E = reinterpret_cast<const T*>(discs[d].E);
                for (int j = tid; j <= S.N; j += BLOCK) s_E[j] = E[j];
                cur_d = d;
            }
            cur_seg = seg;
            __syncthreads();
        }

        const long long ts = g - S.tile0;
        const long long base = ts * TILE;
        if (warp == 0)
            seg_window_load(W, S.seg_start, S.seg_src, S.nseg, S.nseg <= 1 ? 0 : S.first_seg[ts], lane);
        __syncthreads();
        int cin[PPT];
        T fin[PPT], vxin[PPT], vyin[PPT], vzin[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const long long slot = base + (long long)k * BLOCK + tid;
            cin[k] = -1;
            if (slot < S.n) {
                const long long off = seg_offset(W, S.seg_start, S.seg_src, S.nseg, slot);
                const int cc = __ldcs(S.cin + off);
                load_rec<T>(S.pin, off, fin[k], vxin[k], vyin[k], vzin[k]);
                if ((unsigned)cc < (unsigned)S.N) cin[k] = cc;
                else err |= ERR_NONFINITE;  // corrupt cell index: dropped and reported
            }
        }
        // Candidate words: slots 4q..4q+3 take the four words of one Philox call (call 4,
        // counter word 0 = q). Lane l of warp w computes group q = (base + k BLOCK + 32 w) / 4 + j
        // for k = i / 8, j = i % 8, i = l + 32 m; iteration k takes its word by shuffle.
        constexpr int NG = (8 * PPT + 31) / 32;
        U4 cw[NG];
#pragma unroll
        for (int m = 0; m < NG; ++m) {
            const int i = lane + 32 * m;
            const long long q = (base + (long long)(i >> 3) * BLOCK + 32 * warp) / 4 + (i & 7);
            cw[m] = draw(seed, (uint32_t)q, step, S.sp, 4, S.did);
        }
        QEnt<T>* Q = s_q + warp * QCAP;
        const T Ksp = S.k.K[S.sp];
        long long offA = ts * (2 * TILE), offB = ts * TILE;
#pragma unroll
        for (int b = 0; b < PPT; b += BATCH) {
            // phase A: gather, first half kick, energy moment, candidate test; candidates queued
            T ef[BATCH];
            uint32_t fl[BATCH];
            int qi[BATCH];
            int qn = 0;
#pragma unroll
            for (int kk = 0; kk < BATCH; ++kk) {
                const int k = b + kk;
                const int src_lane = (8 * k + (lane >> 2)) & 31;
                const U4& g4 = cw[(8 * k) >> 5];
                const uint32_t w0 = __shfl_sync(FULL, g4.x, src_lane), w1 = __shfl_sync(FULL, g4.y, src_lane);
                const uint32_t w2 = __shfl_sync(FULL, g4.z, src_lane), w3 = __shfl_sync(FULL, g4.w, src_lane);
                const int wi = lane & 3;
                const uint32_t cword = wi == 0 ? w0 : wi == 1 ? w1 : wi == 2 ? w2 : w3;
                const bool valid = cin[k] >= 0;
                unsigned long long qv = 0;
                ef[kk] = 0;
                if (valid) {
                    const int c = cin[k];
                    const T E0 = s_E[c], E1 = s_E[c + 1];
                    ef[kk] = fma_(fin[k], sub_(E1, E0), E0);
                    vzin[k] = fma_(Ksp, ef[kk], vzin[k]);  // v_n
                    if (S.sp == 0) {  // energy moment at (x_n, v_n), 2^-12 eV, clamped at 2^26
                        const T e2 = fma_(vxin[k], vxin[k], fma_(vyin[k], vyin[k], mul_(vzin[k], vzin[k])));
                        T eq = mul_(e2, S.k.kappa_E);
                        if (!(eq <= (T)0x1p26)) eq = (T)0x1p26;
                        const unsigned long long Et = rint_u32(eq);
                        const unsigned long long Eh = rint_u32(mul_(eq, fin[k]));
                        qv = (Et - Eh) | (Eh << 32);
                    }
                }
                if (S.sp == 0) warp_hist<true>(s_Q, cin[k], qv, lane);
                const bool cand = valid && cword < S.thr;
                const unsigned cm = __ballot_sync(FULL, cand);
                if (lane == 0 && cm) atomicAdd(&s_cnt[CNT_CAND + S.sp], (unsigned)__popc(cm));
                qi[kk] = qn + __popc(cm & ((1u << lane) - 1u));
                if (cand) {
                    QEnt<T>& e = Q[qi[kk]];
                    e.slot = (uint32_t)(base + (long long)k * BLOCK + tid);
                    e.c = cin[k];
                    e.f = fin[k];
                    e.ef = ef[kk];
                    e.vx = vxin[k];
                    e.vy = vyin[k];
                    e.vz = vzin[k];
                }
                qn += __popc(cm);
                fl[kk] = cand ? 8u : 0u;
            }
            __syncwarp();
            // phase B: the warp works through its queue, 32 candidates at a time
            for (int q = lane; q < qn; q += 32) collide<T>(S, Q[q], step, seed, s_hist, s_cnt, err);
            __syncwarp();
            // phase C: second half kick, drift, walls, deposit
            Part<T> P0[BATCH], Pse[BATCH];
#pragma unroll
            for (int kk = 0; kk < BATCH; ++kk) {
                const int k = b + kk;
                bool alive = false;
                if (cin[k] >= 0) {
                    T vx = vxin[k], vy = vyin[k], vz = vzin[k];
                    if (fl[kk] & 8u) {
                        const QEnt<T>& e = Q[qi[kk]];
                        vx = e.vx;
                        vy = e.vy;
                        vz = e.vz;
                        fl[kk] |= e.out;
                    }
                    vz = fma_(Ksp, ef[kk], vz);
                    int cn;
                    T fn;
                    const int side = drift(S.N, S.k.dtdx, cin[k], fin[k], vz, cn, fn, err);
                    if (side < 0) {
                        P0[kk] = Part<T>{cn, fn, vx, vy, vz};
                        alive = true;
                        fl[kk] |= 1u;
                    } else {
                        atomicAdd(&s_cnt[CNT_ABS + 2 * S.sp + side], 1u);
                        if (S.sp == 1 && S.has_see &&
                            emit_see<T>(S, (uint32_t)(base + (long long)k * BLOCK + tid), step, seed, side, Pse[kk],
                                        s_cnt))
                            fl[kk] |= 4u;
                    }
                }
                warp_hist<false>(s_hist, alive ? P0[kk].c : -1, alive ? (1ull << 40) + cic_F(P0[kk].f) : 0ull,
                                 lane);
            }
            // block scan of (same-species outputs | births << 16) per k of the batch, in slot order
            uint32_t v[BATCH], incl[BATCH];
#pragma unroll
            for (int kk = 0; kk < BATCH; ++kk) {
                v[kk] = (fl[kk] & 1u) + ((fl[kk] >> 1) & 1u) + (((fl[kk] >> 2) & 1u) << 16);
                incl[kk] = v[kk];
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                for (int kk = 0; kk < BATCH; ++kk) {
                    const uint32_t t = __shfl_up_sync(FULL, incl[kk], o);
                    if (lane >= o) incl[kk] += t;
                }
            }
            if (lane == 31) {
#pragma unroll
                for (int kk = 0; kk < BATCH; ++kk) s_wsum[kk][warp] = incl[kk];
            }
            __syncthreads();
            if (warp == 0) {
#pragma unroll
                for (int kk = 0; kk < BATCH; ++kk) {
                    const uint32_t own = lane < NW ? s_wsum[kk][lane] : 0u;
                    uint32_t x = own;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t t = __shfl_up_sync(FULL, x, o);
                        if (lane >= o) x += t;
                    }
                    if (lane < NW) s_wsum[kk][lane] = x - own;
                    if (lane == NW - 1) s_ktot[kk] = x;
                }
            }
            __syncthreads();
            // phase D: write the batch's outputs into the tile's regions, in slot order
#pragma unroll
            for (int kk = 0; kk < BATCH; ++kk) {
                const uint32_t ex = incl[kk] - v[kk] + s_wsum[kk][warp];
                long long ia = offA + (ex & 0xFFFFu);
                const long long ib = offB + (ex >> 16);
                if (fl[kk] & 1u) {
                    store_rec<T>(S.cout, S.pout, ia, P0[kk]);
                    ++ia;
                }
                if (fl[kk] & 2u) store_rec<T>(S.cout, S.pout, ia, Q[qi[kk]].p1);
                if (fl[kk] & 4u) store_rec<T>(S.bc, S.bp, ib, S.sp == 0 ? Q[qi[kk]].p2 : Pse[kk]);
                offA += s_ktot[kk] & 0xFFFFu;
                offB += s_ktot[kk] >> 16;
            }
            __syncthreads();
        }
        if (tid == 0) {
            S.cnt_main[ts] = (int)(offA - ts * (2 * TILE));
            S.cnt_birth[ts] = (int)(offB - ts * TILE);
        }
        __syncthreads();
    }
    if (cur_seg >= 0) flush();
    if (err) atomicOr(&s_err, err);
    __syncthreads();
    if (tid == 0) {
        if (s_err) atomicOr(&ctl->error, s_err);
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->done, 1u);
        if (prev == gridDim.x - 1) {
            for (int i = 0; i < 2 * n_disc; ++i) ctl->count_in[i >> 1][i & 1] = ctl->count[i >> 1][i & 1];
            ctl->tile_ctr = 0;
            ctl->done = 0;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// Block-wide inclusive scan of doubles held as `per` consecutive elements per
// thread (fixed association order, hence deterministic).
template <int BLOCK>
__device__ void block_scan_inclusive(double* a, int n, double* s_warp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = BLOCK / 32;
    const int per = (n + BLOCK - 1) / BLOCK;
    const int lo = tid * per, hi = min(n, lo + per);
    double run = 0.0;
    for (int i = lo; i < hi; ++i) {
        run = __dadd_rn(run, a[i]);
        a[i] = run;
    }
    double x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x = __dadd_rn(x, t);
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const double own = lane < NW ? s_warp[lane] : 0.0;
        double y = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double t = __shfl_up_sync(FULL, y, o);
            if (lane >= o) y = __dadd_rn(y, t);
        }
        if (lane < NW) s_warp[lane] = __dsub_rn(y, own);
    }
    __syncthreads();
    const double add = __dadd_rn(__dsub_rn(x, run), s_warp[warp]);
    for (int i = lo; i < hi; ++i) a[i] = __dadd_rn(a[i], add);
    __syncthreads();
}

// Exclusive scan of n int counts (global memory) by a whole block: every thread
// takes a contiguous chunk; visit(t, prefix, count) is called for every entry in
// order within the chunk. Returns the total (to every thread).
template <int BLOCK, typename F>
__device__ long long block_chunk_scan(const int* __restrict__ cnt, long long n, long long* s_w, F&& visit) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = BLOCK / 32;
    const long long per = (n + BLOCK - 1) / BLOCK;
    const long long lo = tid * per, hi = min(n, lo + per);
    long long run = 0;
    for (long long t = lo; t < hi; ++t) run += cnt[t];
    long long x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const long long own = lane < NW ? s_w[lane] : 0;
        long long y = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long z = __shfl_up_sync(FULL, y, o);
            if (lane >= o) y += z;
        }
        if (lane < NW) s_w[lane] = y - own;
        if (lane == NW - 1) s_w[32] = y;
    }
    __syncthreads();
    long long ex = s_w[warp] + x - run;
    for (long long t = lo; t < hi; ++t) {
        const int c = cnt[t];
        visit(t, ex, c);
        ex += c;
    }
    const long long total = s_w[32];
    __syncthreads();
    return total;
}

// mode bits: 1 append births and update counts; 2 accumulate moments and
// advance the step; 4 initial solve at t = n dt (load); 8 births only (no
// solve, deposits kept).
template <typename T>
__global__ void __launch_bounds__(1024) k_finalize(const Disc* __restrict__ discs, int n_disc, Ctl* __restrict__ ctl,
                                                   int out_buf, int mode) {
    constexpr int BLOCK = 1024;
    extern __shared__ __align__(16) double s_f[];
    __shared__ double s_warp[32];
    __shared__ long long s_n[2][3];
    __shared__ long long s_lscan[33];
    __shared__ int s_err;
    const int d = blockIdx.x, tid = threadIdx.x, role = blockIdx.y;
    const Disc& D = discs[d];
    const int N = D.N;
    if (tid == 0) s_err = 0;
    __syncthreads();

    // role 1, 2: the new segment table and births of store role-1; role 0: the field
    if ((mode & 1) && role > 0) {
        // New segment tables from the sweep's per-tile counts: store sp's segments are its own
        // tiles' regions (slot order), then one segment of the births of sp that the other
        // species' tiles produced, compacted here into the births region.
        using R = typename Rec<T>::type;
        const int TILE = D.tile;
        if (tid == 0) {
            for (int sp = 0; sp < 2; ++sp) s_n[sp][0] = (ctl->count_in[d][sp] + TILE - 1) / TILE;  // input tiles
        }
        __syncthreads();
        {
            const int sp = role - 1;
            const int par = 1 - sp;
            const long long tiles = s_n[sp][0], ptiles = s_n[par][0];
            int* st = D.seg_start[sp];
            int* sr = D.seg_src[sp];
            const long long main_total = block_chunk_scan<BLOCK>(D.cnt_main[sp], tiles, s_lscan,
                [&](long long t, long long ex, int c) {
                    st[t] = (int)ex;
                    sr[t] = (int)(t * 2 * TILE);
                });
            int32_t* cdst = D.c[out_buf][sp];
            R* pdst = reinterpret_cast<R*>(D.p[out_buf][sp]);
            const int32_t* csrc = D.bc[par];
            const R* psrc = reinterpret_cast<const R*>(D.bp[par]);
            const long long R0 = D.R0[sp], bcap = D.bcap;
            const long long nb = block_chunk_scan<BLOCK>(D.cnt_birth[par], ptiles, s_lscan,
                [&](long long t, long long ex, int c) {
                    for (int k = 0; k < c; ++k) {
                        if (ex + k < bcap) {
                            cdst[R0 + ex + k] = csrc[t * TILE + k];
                            pdst[R0 + ex + k] = psrc[t * TILE + k];
                        } else {
                            s_err = ERR_CAPACITY;
                        }
                    }
                });
            const long long nbk = nb < bcap ? nb : bcap;
            const int nseg = (int)tiles + (nbk > 0 ? 1 : 0);
            long long n_new = main_total + nbk;
            if (tid == 0) {
                if (nbk > 0) {
                    st[tiles] = (int)main_total;
                    sr[tiles] = (int)R0;
                }
                st[nseg] = (int)n_new;
                if (n_new > D.cap[sp]) {
                    s_err = ERR_CAPACITY;
                    n_new = D.cap[sp];
                }
                ctl->count[d][sp] = n_new;
                ctl->nseg[d][sp] = nseg;
            }
            __syncthreads();
            // first segment of every tile of the next sweep: the segment holding slot j TILE
            const long long jmax = D.max_tiles[sp];
            for (int k = tid; k < nseg; k += BLOCK) {
                const long long s0 = st[k], s1 = st[k + 1];
                if (s1 > s0) {
                    const long long j1 = (s1 + TILE - 1) / TILE;
                    for (long long j = (s0 + TILE - 1) / TILE; j < j1 && j <= jmax; ++j) D.first_seg[sp][j] = k;
                }
            }
            __syncthreads();
        }
    }

    if (role > 0 || (mode & 8)) {
        __syncthreads();
        if (tid == 0 && s_err) atomicOr(&ctl->error, s_err);
        if (tid == 0 && (mode & 2)) {
            __threadfence();
            const unsigned prev = atomicAdd(&ctl->fin_done, 1u);
            if (prev == gridDim.x * gridDim.y - 1) {
                ctl->fin_done = 0;
                ctl->step = ctl->step + 1;
                __threadfence();
            }
        }
        return;
    }

    // Poisson, Eq. (poisson): phi_{j-1} - 2 phi_j + phi_{j+1} = -r_j, r_j = rho_j dx^2 / eps0,
    // phi_0 = V_rf sin(2 pi f t), phi_N = 0. With R_j = sum_{k<=j} r_k and S_j = sum_{i<j} R_i:
    // phi_j = phi_0 + j g_1 - S_j, g_1 = (phi_N - phi_0 + S_N) / N.
    double* a = s_f;               // N+1
    double* rho = s_f + (MAXN + 1);
    const double dx = D.dx;
    const long long step = ctl->step;
    const double t = (mode & 4) ? (double)step * D.dt : (double)(step + 1) * D.dt;
    const double V0 = D.V_rf * sin(2.0 * PI_D * D.f_rf * t);
    for (int j = tid; j <= N; j += BLOCK) {
        const double Vj = (j == 0 || j == N) ? 0.5 * dx : dx;
        rho[j] = E_CHARGE * (D.w[1] * (double)D.D[1][j] - D.w[0] * (double)D.D[0][j]) / (TWO32_D * Vj);
        a[j] = (j >= 1 && j <= N - 1) ? rho[j] * dx * dx / EPS0 : 0.0;
    }
    __syncthreads();
    block_scan_inclusive<BLOCK>(a, N, s_warp);  // a[j] = R_j, j = 0..N-1
    double* Rr = rho + (MAXN + 1);              // keep R for the field (third shared array)
    for (int j = tid; j < N; j += BLOCK) Rr[j] = a[j];
    __syncthreads();
    // exclusive scan of R into S: S_j = sum_{i<j} R_i, j = 0..N
    double* Sx = a;  // reuse: shift by one
    {
        // a[j] holds R_j (j < N); build S in place: S_0 = 0, S_{j+1} = S_j + R_j
        block_scan_inclusive<BLOCK>(a, N, s_warp);  // a[j] = sum_{i<=j} R_i = S_{j+1}
    }
    __syncthreads();
    const double SN = N > 0 ? Sx[N - 1] : 0.0;
    const double g1 = (0.0 - V0 + SN) / (double)N;
    // g_j = phi_j - phi_{j-1} = g_1 - R_{j-1}; node field E_j = -(g_j + g_{j+1}) / (2 dx) inside
    // (the central difference of phi, without the cancellation of large phi values), and Gauss's
    // law over the half cells at the electrodes.
    double* phi = D.phi;
    for (int j = tid; j <= N; j += BLOCK) {
        const double Sj = j == 0 ? 0.0 : Sx[j - 1];
        double ph = V0 + (double)j * g1 - Sj;
        if (j == N) ph = 0.0;
        if (j == 0) ph = V0;
        phi[j] = ph;
    }
    __syncthreads();
    for (int j = tid; j <= N; j += BLOCK) {
        double E;
        if (j == 0) E = -g1 / dx - rho[0] * dx / (2.0 * EPS0);
        else if (j == N) E = -(g1 - Rr[N - 1]) / dx + rho[N] * dx / (2.0 * EPS0);
        else E = -((g1 - Rr[j - 1]) + (g1 - Rr[j])) / (2.0 * dx);
        D.E64[j] = E;
        reinterpret_cast<T*>(D.E)[j] = (T)E;
        if (j == 0) ctl->E0_last[d] = E;
    }
    if (mode & 2) {
        for (int j = tid; j <= N; j += BLOCK) {
            D.acc_D[0][j] += (double)D.D[0][j];
            D.acc_D[1][j] += (double)D.D[1][j];
            D.acc_Q[j] += (double)D.Q[j];
            D.acc_Dprev[j] += (double)D.Dprev[j];
        }
        if (tid == 0) ctl->acc_steps[d] += 1;
    }
    for (int j = tid; j <= N; j += BLOCK) {
        D.Dprev[j] = D.D[0][j];
        D.D[0][j] = 0;
        D.D[1][j] = 0;
        D.Q[j] = 0;
    }
    __syncthreads();
    if (tid == 0) {
        if (s_err) atomicOr(&ctl->error, s_err);
        if (mode & 2) {
            __threadfence();
            const unsigned prev = atomicAdd(&ctl->fin_done, 1u);
            if (prev == gridDim.x * gridDim.y - 1) {
                ctl->fin_done = 0;
                ctl->step = step + 1;
                __threadfence();
            }
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
// Stable counting sort by cell. Tiles of SORT_TILE particles; inside a tile
// warp w owns a contiguous run of SORT_R x 32 particles in input order.
constexpr int SORT_BLOCK = 256, SORT_NW = SORT_BLOCK / 32, SORT_R = 16, SORT_TILE = SORT_BLOCK * SORT_R;

// Per tile: count of each cell -> hist[seg][c * T_s + t]. Input read through
// the store's segment table.
__global__ void __launch_bounds__(SORT_BLOCK) k_sort_count(const Disc* __restrict__ discs, const Ctl* __restrict__ ctl,
                                                           int buf, unsigned* __restrict__ hist,
                                                           const long long* __restrict__ hoff) {
    extern __shared__ __align__(16) unsigned s_c[];
    __shared__ SegWin W;
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const Disc& D = discs[d];
    const int N = D.N;
    const long long n = ctl->count[d][sp];
    const int nseg = ctl->nseg[d][sp];
    const long long Ts = (n + SORT_TILE - 1) / SORT_TILE;
    const int32_t* cc = D.c[buf][sp];
    unsigned* H = hist + hoff[seg];
    const int lane = threadIdx.x & 31;
    const int per_sweep_tile = SORT_TILE / D.tile;
    for (long long t = blockIdx.x; t < Ts; t += gridDim.x) {
        for (int j = threadIdx.x; j < N; j += SORT_BLOCK) s_c[j] = 0;
        if (threadIdx.x < 32)
            seg_window_load(W, D.seg_start[sp], D.seg_src[sp], nseg, nseg <= 1 ? 0 : D.first_seg[sp][t * per_sweep_tile],
                            lane);
        __syncthreads();
        for (int i = threadIdx.x; i < SORT_TILE; i += SORT_BLOCK) {
            const long long k = t * SORT_TILE + i;
            const int key = k < n ? cc[seg_offset(W, D.seg_start[sp], D.seg_src[sp], nseg, k)] : N;
            const unsigned peers = __match_any_sync(FULL, key);
            if ((unsigned)key < (unsigned)N && lane == __ffs(peers) - 1) atomicAdd(&s_c[key], (unsigned)__popc(peers));
        }
        __syncthreads();
        for (int j = threadIdx.x; j < N; j += SORT_BLOCK) H[(long long)j * Ts + t] = s_c[j];
        __syncthreads();
    }
}

// Per (store, cell) row: exclusive scan over the tiles in place; row total out.
__global__ void __launch_bounds__(1024) k_sort_rows(const Disc* __restrict__ discs, const Ctl* __restrict__ ctl,
                                                    unsigned* __restrict__ hist, const long long* __restrict__ hoff,
                                                    unsigned* __restrict__ tot) {
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const int N = discs[d].N;
    const int c = blockIdx.x;
    if (c >= N) return;
    const long long n = ctl->count[d][sp];
    const long long Ts = (n + SORT_TILE - 1) / SORT_TILE;
    unsigned* row = hist + hoff[seg] + (long long)c * Ts;
    __shared__ unsigned s_w[32];
    __shared__ unsigned s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (long long b0 = 0; b0 < Ts; b0 += 1024) {
        const long long i = b0 + tid;
        const unsigned own = i < Ts ? row[i] : 0u;
        unsigned x = own;
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
        const unsigned carry = s_carry;
        if (i < Ts) row[i] = carry + s_w[warp] + x - own;
        __syncthreads();
        if (tid == 1023) s_carry = carry + s_w[warp] + x;
        __syncthreads();
    }
    if (tid == 0) tot[(long long)seg * MAXN + c] = s_carry;
}

// Per store: exclusive scan of the row totals -> first slot of every cell.
__global__ void __launch_bounds__(1024) k_sort_cells(const Disc* __restrict__ discs, unsigned* __restrict__ tot) {
    const int seg = blockIdx.x, d = seg >> 1;
    const int N = discs[d].N;
    unsigned* a = tot + (long long)seg * MAXN;
    __shared__ unsigned s_v[MAXN];
    __shared__ unsigned s_w[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = tid; j < N; j += 1024) s_v[j] = a[j];
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

// Scatter: per-warp counts, prefix over warps, then each warp places its run
// in order (rank among equal cells by match_any). Input through the segment
// table; output dense.
template <typename T>
__global__ void __launch_bounds__(SORT_BLOCK) k_sort_scatter(const Disc* __restrict__ discs,
                                                             const Ctl* __restrict__ ctl, int src, int dst,
                                                             const unsigned* __restrict__ hist,
                                                             const long long* __restrict__ hoff,
                                                             const unsigned* __restrict__ tot, int max_N) {
    extern __shared__ __align__(16) unsigned s_w[];  // [SORT_NW][max_N]
    __shared__ SegWin W;
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const Disc& D = discs[d];
    const int N = D.N;
    const long long n = ctl->count[d][sp];
    const int nseg = ctl->nseg[d][sp];
    const long long Ts = (n + SORT_TILE - 1) / SORT_TILE;
    const int32_t* cs = D.c[src][sp];
    int32_t* cd = D.c[dst][sp];
    using R = typename Rec<T>::type;
    const R* ps = reinterpret_cast<const R*>(D.p[src][sp]);
    R* pd = reinterpret_cast<R*>(D.p[dst][sp]);
    const unsigned* H = hist + hoff[seg];
    const unsigned* cstart = tot + (long long)seg * MAXN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned* Wc = s_w + warp * max_N;
    const int per_sweep_tile = SORT_TILE / D.tile;
    for (long long t = blockIdx.x; t < Ts; t += gridDim.x) {
        for (int j = tid; j < SORT_NW * max_N; j += SORT_BLOCK) s_w[j] = 0;
        if (warp == 0)
            seg_window_load(W, D.seg_start[sp], D.seg_src[sp], nseg, nseg <= 1 ? 0 : D.first_seg[sp][t * per_sweep_tile],
                            lane);
        __syncthreads();
        const long long wbase = t * SORT_TILE + (long long)warp * (SORT_R * 32);
        for (int r = 0; r < SORT_R; ++r) {
            const long long k = wbase + r * 32 + lane;
            const int key = k < n ? cs[seg_offset(W, D.seg_start[sp], D.seg_src[sp], nseg, k)] : N;
            const unsigned peers = __match_any_sync(FULL, key);
            if ((unsigned)key < (unsigned)N && lane == __ffs(peers) - 1) Wc[key] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        for (int j = tid; j < N; j += SORT_BLOCK) {
            unsigned run = 0;
#pragma unroll
            for (int w = 0; w < SORT_NW; ++w) {
                const unsigned v = s_w[w * max_N + j];
                s_w[w * max_N + j] = run;
                run += v;
            }
        }
        __syncthreads();
        for (int r = 0; r < SORT_R; ++r) {
            const long long k = wbase + r * 32 + lane;
            long long off = 0;
            int key = N;
            if (k < n) {
                off = seg_offset(W, D.seg_start[sp], D.seg_src[sp], nseg, k);
                key = cs[off];
            }
            const unsigned peers = __match_any_sync(FULL, key);
            const unsigned b = (unsigned)key < (unsigned)N ? Wc[key] : 0u;
            __syncwarp();
            if ((unsigned)key < (unsigned)N) {
                const long long o = (long long)cstart[key] + H[(long long)key * Ts + t] + b + __popc(peers & lt);
                if (o < n) {
                    cd[o] = key;
                    pd[o] = ps[off];
                }
                if (lane == __ffs(peers) - 1) Wc[key] = b + __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
    }
}

// Every store becomes one dense segment [0, count) (after a load, an upload or a sort).
__global__ void k_set_dense(const Disc* __restrict__ discs, int n_disc, Ctl* __restrict__ ctl) {
    const int i = threadIdx.x;
    if (i >= 2 * n_disc) return;
    const int d = i >> 1, sp = i & 1;
    const Disc& D = discs[d];
    D.seg_start[sp][0] = 0;
    D.seg_start[sp][1] = (int)ctl->count[d][sp];
    D.seg_src[sp][0] = 0;
    D.first_seg[sp][0] = 0;
    ctl->nseg[d][sp] = 1;
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

template <typename T, int BLOCK, int PPT>
static cudaError_t launch_sweep_t(const SweepLaunch& L) {
    const size_t smem = sweep_smem<T, BLOCK, PPT>(L.max_N);
    auto kern = k_sweep<T, BLOCK, PPT>;
    cudaError_t e = smem_attr(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<L.grid, BLOCK, smem, L.stream>>>(L.discs, L.n_disc, L.ctl, L.in_buf, L.seed, L.max_N);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_sweep_p(const SweepLaunch& L) {
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
static int occ_t(int max_N) {
    int nb = 0;
    const size_t smem = sweep_smem<T, BLOCK, PPT>(max_N);
    smem_attr(k_sweep<T, BLOCK, PPT>, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<T, BLOCK, PPT>, BLOCK, smem);
    return nb;
}
template <typename T>
static int occ_p(int block, int ppt, int max_N) {
    if (block == 128) {
        if (ppt == 2) return occ_t<T, 128, 2>(max_N);
        if (ppt == 8) return occ_t<T, 128, 8>(max_N);
        return occ_t<T, 128, 4>(max_N);
    }
    if (ppt == 2) return occ_t<T, 256, 2>(max_N);
    if (ppt == 8) return occ_t<T, 256, 8>(max_N);
    return occ_t<T, 256, 4>(max_N);
}
int sweep_occupancy(int fp64, int block, int ppt, int max_N) {
    return fp64 ? occ_p<double>(block, ppt, max_N) : occ_p<float>(block, ppt, max_N);
}

cudaError_t launch_finalize(int fp64, const Disc* discs, int n_disc, Ctl* ctl, int out_buf, int mode,
                            cudaStream_t st) {
    const size_t smem = sizeof(double) * 3 * (MAXN + 1);
    if (fp64) {
        smem_attr(k_finalize<double>, smem);
        k_finalize<double><<<dim3(n_disc, 3), 1024, smem, st>>>(discs, n_disc, ctl, out_buf, mode);
    } else {
        smem_attr(k_finalize<float>, smem);
        k_finalize<float><<<dim3(n_disc, 3), 1024, smem, st>>>(discs, n_disc, ctl, out_buf, mode);
    }
    return cudaGetLastError();
}

cudaError_t launch_load(int fp64, const Disc* discs, int n_disc, Ctl* ctl, int buf, unsigned long long seed,
                        int grid_x, cudaStream_t st) {
    dim3 g(grid_x, 2 * n_disc);
    if (fp64) k_load<double><<<g, 256, 0, st>>>(discs, ctl, buf, seed);
    else k_load<float><<<g, 256, 0, st>>>(discs, ctl, buf, seed);
    return cudaGetLastError();
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

cudaError_t launch_sort(int fp64, const Disc* discs, int n_disc, const Ctl* ctl, int src, int dst, unsigned* hist,
                        const long long* hoff, unsigned* tot, int max_N, int grid_x, cudaStream_t st) {
    dim3 g(grid_x, 2 * n_disc);
    k_sort_count<<<g, SORT_BLOCK, sizeof(unsigned) * max_N, st>>>(discs, ctl, src, hist, hoff);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sort_rows<<<dim3(max_N, 2 * n_disc), 1024, 0, st>>>(discs, ctl, hist, hoff, tot);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sort_cells<<<2 * n_disc, 1024, 0, st>>>(discs, tot);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(unsigned) * SORT_NW * max_N;
    if (fp64) {
        smem_attr(k_sort_scatter<double>, smem);
        k_sort_scatter<double><<<g, SORT_BLOCK, smem, st>>>(discs, ctl, src, dst, hist, hoff, tot, max_N);
    } else {
        smem_attr(k_sort_scatter<float>, smem);
        k_sort_scatter<float><<<g, SORT_BLOCK, smem, st>>>(discs, ctl, src, dst, hist, hoff, tot, max_N);
    }
    return cudaGetLastError();
}

long long sort_tile() { return SORT_TILE; }

cudaError_t launch_set_dense(const Disc* discs, int n_disc, Ctl* ctl, cudaStream_t st) {
    k_set_dense<<<1, 128, 0, st>>>(discs, n_disc, ctl);
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
