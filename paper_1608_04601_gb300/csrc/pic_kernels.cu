// pic_kernels.cu -- CUDA kernels (sm_103a) of the 1d3v PIC/MCC time step of
// arXiv:1608.04601, section "PIC/MCC simulation procedure".
//
// One time step is three launches:
//   k_sweep     persistent; every CTA takes tiles of particles in increasing
//               order from a global dispenser. Per particle: CIC gather of E_n
//               (node field held in shared memory), half kick, null-collision
//               MCC on Philox streams, half kick, drift, wall test; per tile a
//               block scan and a decoupled look-back over the tiles of its
//               store give every surviving / newborn particle its output slot
//               (survivors in input order, each followed by its same-species
//               newborn); CIC deposit into a shared-memory int64 histogram
//               that is flushed with global atomics.
//   k_finalize  one CTA per discharge: births of the other species appended,
//               Poisson (Eq. poisson, rf Dirichlet boundary) in FP64 by two
//               block scans, node field, cycle-average accumulators.
//   sort        every K steps: stable counting sort of each store by cell.
#include "pic_internal.h"
#include "pic_device.cuh"

namespace pic {

#define E_CHARGE 1.602176634e-19
#define M_ELEC 9.1093837015e-31
#define EPS0 8.8541878128e-12
#define PI_D 3.14159265358979323846
#define TWO32_D 4294967296.0

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int LOOKBACK_SPIN_LIMIT = 1 << 22;  // ~seconds: then report ERR_TIMEOUT and go on

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
};

__device__ __forceinline__ unsigned long long mk_status(unsigned epoch, unsigned flag, unsigned long long v) {
    return ((unsigned long long)epoch << 32) | ((unsigned long long)flag << 30) | (v & 0x3FFFFFFFull);
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

// Warp-aggregated shared-memory histogram update. key < 0: nothing. Lanes whose keys equal their
// left neighbour's form a run (the store is kept cell-sorted, so runs are long); one 64-bit warp
// scan of the packed values gives each run's sum, and the run's last lane applies it:
//   deposit (pair = false): v = 2^40 + F  ->  node key += count 2^32 - sum F, node key+1 += sum F
//   moment  (pair = true):  v = lo + hi 2^32 -> node key += sum lo, node key+1 += sum hi
// When most keys in the warp differ, plain atomics are cheaper and are used instead.
template <bool PAIR>
__device__ __forceinline__ void warp_hist(unsigned long long* h, int key, unsigned long long v, int lane) {
    const int prev = __shfl_up_sync(FULL, key, 1);
    const bool head = lane == 0 || prev != key;
    const unsigned heads = __ballot_sync(FULL, head);
    if (__popc(heads) > 12) {
        if (key >= 0) {
            if (PAIR) {
                const unsigned long long lo = v & 0xFFFFFFFFull, hi = v >> 32;
                if (lo) sadd64(&h[key], lo);
                if (hi) sadd64(&h[key + 1], hi);
            } else {
                const unsigned long long F = v & ((1ull << 40) - 1);
                sadd64(&h[key], (1ull << 32) - F);
                if (F) sadd64(&h[key + 1], F);
            }
        }
        return;
    }
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += t;
    }
    const unsigned below = heads & (0xFFFFFFFFu >> (31 - lane));
    const int hl = 31 - __clz(below);
    const unsigned long long before = __shfl_sync(FULL, x, hl > 0 ? hl - 1 : 0);
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (tail && key >= 0) {
        const unsigned long long sum = x - (hl > 0 ? before : 0ull);
        if (PAIR) {
            const unsigned long long lo = sum & 0xFFFFFFFFull, hi = sum >> 32;
            if (lo) sadd64(&h[key], lo);
            if (hi) sadd64(&h[key + 1], hi);
        } else {
            const unsigned long long cnt = sum >> 40, F = sum & ((1ull << 40) - 1);
            sadd64(&h[key], (cnt << 32) - F);
            if (F) sadd64(&h[key + 1], F);
        }
    }
}

// Advance one particle by one step. Returns flags: bit0 particle stays,
// bit1 same-species newborn stays, bit2 other-species birth stays,
// bit3 candidate for a collision.
template <typename T>
__device__ __forceinline__ uint32_t advance(const Seg<T>& S, const T* __restrict__ sE, unsigned long long* sH,
                                            unsigned long long& qv, unsigned* sC, uint32_t slot,
                                            long long step, unsigned long long seed, int c, T f, T vx, T vy, T vz,
                                            Part<T>& p0, Part<T>& p1, Part<T>& p2, int& err) {
    using Row4 = typename T4<T>::type;
    using Row2 = typename T4<T>::two;
    const Consts<T>& K = S.k;
    const int N = S.N;
    uint32_t out = 0;
    const T E0 = sE[c], E1 = sE[c + 1];
    const T ef = fma_(f, sub_(E1, E0), E0);
    if (S.sp == 0) {
        vz = fma_(K.K[0], ef, vz);  // v_n
        const T e2 = fma_(vx, vx, fma_(vy, vy, mul_(vz, vz)));
        {   // energy moment at (x_n, v_n) in 2^-12 eV, clamped at 2^26 (16384 eV)
            T eq = mul_(e2, K.kappa_E);
            if (!(eq <= (T)0x1p26)) eq = (T)0x1p26;
            const unsigned long long Et = rint_u32(eq);
            const unsigned long long Eh = rint_u32(mul_(eq, f));
            qv = (Et - Eh) | (Eh << 32);
        }
        const U4 r = draw(seed, slot, step, 0, 0, S.did);
        bool child = false;
        T cvx = 0, cvy = 0, cvz = 0, ivx = 0, ivy = 0, ivz = 0;
        if (r.x < S.thr) {
            out |= 8u;
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
                } else if (j <= S.n_exc) {
                    // excitation of level j
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
                        const U4 q = draw(seed, slot, step, 0, 1, S.did);
                        const U4 w = draw(seed, slot, step, 0, 2, S.did);
                        iso_dir(u01(q.x), u01(q.y), nx, ny, nz);
                        cvx = mul_(sp, nx);
                        cvy = mul_(sp, ny);
                        cvz = mul_(sp, nz);
                        float b0, b1, b2, b3;
                        box_muller(u01(q.z), u01(q.w), b0, b1);
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
        }
        vz = fma_(K.K[0], ef, vz);
        int cn;
        T fn;
        int side = drift(N, K.dtdx, c, f, vz, cn, fn, err);
        if (side < 0) {
            p0 = Part<T>{cn, fn, vx, vy, vz};
            out |= 1u;
        } else {
            atomicAdd(&sC[CNT_ABS + side], 1u);
        }
        if (child) {
            cvz = fma_(K.K[0], ef, cvz);
            side = drift(N, K.dtdx, c, f, cvz, cn, fn, err);
            if (side < 0) {
                p1 = Part<T>{cn, fn, cvx, cvy, cvz};
                shist_add(sH, cn, cic_F(fn));
                out |= 2u;
            } else {
                atomicAdd(&sC[CNT_ABS + side], 1u);
            }
            ivz = fma_(K.K[1], ef, ivz);
            side = drift(N, K.dtdx, c, f, ivz, cn, fn, err);
            if (side < 0) {
                p2 = Part<T>{cn, fn, ivx, ivy, ivz};
                hist_add(S.Dother, cn, cic_F(fn));
                out |= 4u;
            } else {
                atomicAdd(&sC[CNT_ABS + 2 + side], 1u);
            }
        }
    } else {
        vz = fma_(K.K[1], ef, vz);  // v_n
        const U4 r = draw(seed, slot, step, 1, 0, S.did);
        if (r.x < S.thr) {
            out |= 8u;
            const U4 q = draw(seed, slot, step, 1, 1, S.did);
            float a0, a1, a2, a3;
            box_muller(u01(q.x), u01(q.y), a0, a1);
            box_muller(u01(q.z), u01(q.w), a2, a3);
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
        vz = fma_(K.K[1], ef, vz);
        int cn;
        T fn;
        const int side = drift(N, K.dtdx, c, f, vz, cn, fn, err);
        if (side < 0) {
            p0 = Part<T>{cn, fn, vx, vy, vz};
            out |= 1u;
        } else {
            atomicAdd(&sC[CNT_ABS + 2 + side], 1u);
            if (S.has_see) {
                const U4 w = draw(seed, slot, step, 1, 3, S.did);
                if ((T)u01(w.x) < K.gamma) {
                    const T vn = mul_(K.sig_see_n, (T)__fsqrt_rn(-own_logf(u01(w.y))));
                    float t0, t1;
                    box_muller(u01(w.z), u01(w.w), t0, t1);
                    const int ce = side == 0 ? 0 : N - 1;
                    const T fe = side == 0 ? (T)0 : one_minus_ulp<T>();
                    p2 = Part<T>{ce, fe, mul_(K.sig_see, (T)t0), mul_(K.sig_see, (T)t1), side == 0 ? vn : -vn};
                    hist_add(S.Dother, ce, cic_F(fe));
                    atomicAdd(&sC[CNT_SEE], 1u);
                    out |= 4u;
                }
            }
        }
    }
    return out;
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

// ---------------------------------------------------------------------------
template <typename T, int BLOCK, int PPT>
__global__ void __launch_bounds__(BLOCK, (sizeof(T) == 4 ? 512 : 256) / BLOCK) k_sweep(const Disc* __restrict__ discs, int n_disc, Ctl* __restrict__ ctl,
                                                 unsigned long long* __restrict__ st_main,
                                                 unsigned long long* __restrict__ st_bagg,
                                                 unsigned long long* __restrict__ st_binc, int in_buf,
                                                 unsigned long long seed, int max_N) {
    constexpr int TILE = BLOCK * PPT;
    constexpr int NW = BLOCK / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* s_hist = reinterpret_cast<unsigned long long*>(smem_raw);
    unsigned long long* s_Q = s_hist + (max_N + 1);
    T* s_E = reinterpret_cast<T*>(s_Q + (max_N + 1));

    __shared__ long long s_segstart[2 * MAXD + 1];
    __shared__ Seg<T> S;
    __shared__ unsigned int s_tile;
    __shared__ unsigned int s_epoch;
    __shared__ long long s_step;
    __shared__ uint32_t s_wsum[PPT][NW];
    __shared__ uint32_t s_ktot[PPT];
    __shared__ unsigned long long s_excl[2];
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
        s_epoch = ctl->epoch;
        s_step = ctl->step;
        s_err = 0;
    }
    __syncthreads();
    const long long total_tiles = s_segstart[2 * n_disc];
    const unsigned epoch = s_epoch;
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
            int lo = 0, hi = 2 * n_disc - 1;  // largest seg with segstart <= g and non-empty
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
        int cin[PPT];
        T fin[PPT], vxin[PPT], vyin[PPT], vzin[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const long long slot = base + (long long)k * BLOCK + tid;
            cin[k] = -1;
            if (slot < S.n) {
                const int cc = __ldcs(S.cin + slot);
                load_rec<T>(S.pin, slot, fin[k], vxin[k], vyin[k], vzin[k]);
                if ((unsigned)cc < (unsigned)S.N) cin[k] = cc;
                else err |= ERR_NONFINITE;  // corrupt cell index: dropped and reported
            }
        }
        Part<T> P0[PPT], P1[PPT], P2[PPT];
        uint32_t fl[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            fl[k] = 0;
            unsigned long long qv = 0;
            if (cin[k] >= 0) {
                const uint32_t slot = (uint32_t)(base + (long long)k * BLOCK + tid);
                fl[k] = advance<T>(S, s_E, s_hist, qv, s_cnt, slot, step, seed, cin[k], fin[k], vxin[k], vyin[k],
                                   vzin[k], P0[k], P1[k], P2[k], err);
            }
            const unsigned cm = __ballot_sync(FULL, (fl[k] & 8u) != 0);
            if (lane == 0 && cm) atomicAdd(&s_cnt[CNT_CAND + S.sp], (unsigned)__popc(cm));
            // deposit of the particle at x_{n+1}, and (electrons) the energy moment at x_n
            const bool alive = (fl[k] & 1u) != 0;
            warp_hist<false>(s_hist, alive ? P0[k].c : -1, alive ? (1ull << 40) + cic_F(P0[k].f) : 0ull, lane);
            if (S.sp == 0) warp_hist<true>(s_Q, cin[k], qv, lane);
        }
        // block scan of (same-species outputs | births << 16) per k, in slot order
        uint32_t v[PPT], incl[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            v[k] = (fl[k] & 1u) + ((fl[k] >> 1) & 1u) + (((fl[k] >> 2) & 1u) << 16);
            incl[k] = v[k];
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const uint32_t t = __shfl_up_sync(FULL, incl[k], o);
                if (lane >= o) incl[k] += t;
            }
        }
        if (lane == 31) {
#pragma unroll
            for (int k = 0; k < PPT; ++k) s_wsum[k][warp] = incl[k];
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const uint32_t own = lane < NW ? s_wsum[k][lane] : 0u;
                uint32_t x = own;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(FULL, x, o);
                    if (lane >= o) x += t;
                }
                if (lane < NW) s_wsum[k][lane] = x - own;
                if (lane == NW - 1) s_ktot[k] = x;
            }
        }
        __syncthreads();
        unsigned long long A = 0, B = 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            A += s_ktot[k] & 0xFFFFu;
            B += s_ktot[k] >> 16;
        }
        // decoupled look-back over the tiles of this store
        if (warp == 0) {
            unsigned long long exA = 0, exB = 0;
            const long long first = S.tile0;
            if (g == first) {
                if (lane == 0) {
                    st_binc[g] = B;
                    st_release(&st_main[g], mk_status(epoch, 2, A));
                }
            } else {
                if (lane == 0) {
                    st_bagg[g] = B;
                    st_release(&st_main[g], mk_status(epoch, 1, A));
                }
                // Look back in windows of LB_W x 32 predecessors: all of a window's status
                // words are requested at once, then its 32-tile groups are examined nearest
                // first; the walk stops at the nearest inclusive prefix.
                constexpr int LB_W = 8;
                long long j = g - 1;
                bool found = false;
                while (!found) {
                    unsigned long long w[LB_W];
#pragma unroll
                    for (int i = 0; i < LB_W; ++i) {
                        const long long idx = j - i * 32 - lane;
                        w[i] = idx >= first ? ld_acquire(&st_main[idx]) : mk_status(epoch, 2, 0);
                    }
#pragma unroll
                    for (int i = 0; i < LB_W && !found; ++i) {
                        const long long idx = j - i * 32 - lane;
                        unsigned flag = 2;
                        if (idx >= first) {
                            flag = ((unsigned)(w[i] >> 32) == epoch) ? (unsigned)(w[i] >> 30) & 3u : 0u;
                            for (int it = 0; !flag && it < LOOKBACK_SPIN_LIMIT; ++it) {
                                __nanosleep(32);
                                w[i] = ld_acquire(&st_main[idx]);
                                if ((unsigned)(w[i] >> 32) == epoch) flag = (unsigned)(w[i] >> 30) & 3u;
                            }
                            if (!flag) {
                                err |= ERR_TIMEOUT;
                                flag = 2;
                                w[i] = 0;
                            }
                        }
                        const unsigned long long va = idx >= first ? (w[i] & 0x3FFFFFFFull) : 0ull;
                        const unsigned pm = __ballot_sync(FULL, flag == 2);
                        const int L = pm ? __ffs(pm) - 1 : 31;
                        unsigned long long vb = 0;
                        if (idx >= first && lane <= L)
                            vb = (flag == 2) ? *((volatile unsigned long long*)&st_binc[idx])
                                             : *((volatile unsigned long long*)&st_bagg[idx]);
                        unsigned long long a = lane <= L ? va : 0ull, b = vb;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            a += __shfl_xor_sync(FULL, a, o);
                            b += __shfl_xor_sync(FULL, b, o);
                        }
                        exA += a;
                        exB += b;
                        if (pm) found = true;
                    }
                    j -= LB_W * 32;
                }
                if (lane == 0) {
                    st_binc[g] = exB + B;
                    st_release(&st_main[g], mk_status(epoch, 2, exA + A));
                }
            }
            if (lane == 0) {
                s_excl[0] = exA;
                s_excl[1] = exB;
                if (ts == S.ntiles - 1) {
                    ctl->out_main[S.d][S.sp] = (long long)(exA + A);
                    ctl->out_birth[S.d][S.sp] = (long long)(exB + B);
                }
            }
        }
        __syncthreads();
        // scatter the outputs
        unsigned long long offA = s_excl[0], offB = s_excl[1];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const uint32_t ex = incl[k] - v[k] + s_wsum[k][warp];
            unsigned long long ia = offA + (ex & 0xFFFFu);
            const unsigned long long ib = offB + (ex >> 16);
            if (fl[k] & 1u) {
                if ((long long)ia < S.cap) store_rec<T>(S.cout, S.pout, (long long)ia, P0[k]);
                else err |= ERR_CAPACITY;
                ++ia;
            }
            if (fl[k] & 2u) {
                if ((long long)ia < S.cap) store_rec<T>(S.cout, S.pout, (long long)ia, P1[k]);
                else err |= ERR_CAPACITY;
            }
            if (fl[k] & 4u) {
                if ((long long)ib < S.bcap) store_rec<T>(S.bc, S.bp, (long long)ib, P2[k]);
                else err |= ERR_CAPACITY;
            }
            offA += s_ktot[k] & 0xFFFFu;
            offB += s_ktot[k] >> 16;
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
            ctl->tile_ctr = 0;
            ctl->done = 0;
            ctl->epoch = epoch + 1;
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
    __shared__ int s_err;
    const int d = blockIdx.x, tid = threadIdx.x;
    const Disc& D = discs[d];
    const int N = D.N;
    if (tid == 0) s_err = 0;
    __syncthreads();

    if (mode & 1) {
        using R = typename Rec<T>::type;
        if (tid == 0) {
            for (int sp = 0; sp < 2; ++sp) {
                const long long n_in = ctl->count[d][sp];
                s_n[sp][0] = n_in > 0 ? ctl->out_main[d][sp] : 0;   // same-species outputs
                s_n[sp][1] = n_in > 0 ? ctl->out_birth[d][sp] : 0;  // births of the other species
            }
        }
        __syncthreads();
        for (int sp_new = 0; sp_new < 2; ++sp_new) {
            const int sp_par = 1 - sp_new;
            const long long nb = s_n[sp_par][1];
            const long long n0 = s_n[sp_new][0];
            int32_t* cdst = D.c[out_buf][sp_new];
            R* pdst = reinterpret_cast<R*>(D.p[out_buf][sp_new]);
            const int32_t* csrc = D.bc[sp_par];
            const R* psrc = reinterpret_cast<const R*>(D.bp[sp_par]);
            for (long long k = tid; k < nb; k += BLOCK) {
                const long long dst = n0 + k;
                if (k < D.bcap && dst < D.cap[sp_new]) {
                    cdst[dst] = csrc[k];
                    pdst[dst] = psrc[k];
                } else {
                    s_err = ERR_CAPACITY;
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            for (int sp = 0; sp < 2; ++sp) {
                long long n = s_n[sp][0] + s_n[1 - sp][1];
                if (s_n[sp][0] > D.cap[sp] || s_n[1 - sp][1] > D.bcap) s_err = ERR_CAPACITY;
                if (n > D.cap[sp]) {
                    n = D.cap[sp];
                    s_err = ERR_CAPACITY;
                }
                ctl->count[d][sp] = n;
            }
        }
    }

    if (mode & 8) {
        __syncthreads();
        if (tid == 0 && s_err) atomicOr(&ctl->error, s_err);
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
            if (prev == gridDim.x - 1) {
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

// Per tile: count of each cell -> hist[seg][c * T_s + t].
__global__ void __launch_bounds__(SORT_BLOCK) k_sort_count(const Disc* __restrict__ discs, const Ctl* __restrict__ ctl,
                                                           int buf, unsigned* __restrict__ hist,
                                                           const long long* __restrict__ hoff) {
    extern __shared__ __align__(16) unsigned s_c[];
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const Disc& D = discs[d];
    const int N = D.N;
    const long long n = ctl->count[d][sp];
    const long long Ts = (n + SORT_TILE - 1) / SORT_TILE;
    const int32_t* cc = D.c[buf][sp];
    unsigned* H = hist + hoff[seg];
    const int lane = threadIdx.x & 31;
    for (long long t = blockIdx.x; t < Ts; t += gridDim.x) {
        for (int j = threadIdx.x; j < N; j += SORT_BLOCK) s_c[j] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < SORT_TILE; i += SORT_BLOCK) {
            const long long k = t * SORT_TILE + i;
            const int key = k < n ? cc[k] : N;
            const unsigned peers = __match_any_sync(FULL, key);
            if (key < N && lane == __ffs(peers) - 1) atomicAdd(&s_c[key], (unsigned)__popc(peers));
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
// in order (rank among equal cells by match_any).
template <typename T>
__global__ void __launch_bounds__(SORT_BLOCK) k_sort_scatter(const Disc* __restrict__ discs,
                                                             const Ctl* __restrict__ ctl, int src, int dst,
                                                             const unsigned* __restrict__ hist,
                                                             const long long* __restrict__ hoff,
                                                             const unsigned* __restrict__ tot, int max_N) {
    extern __shared__ __align__(16) unsigned s_w[];  // [SORT_NW][max_N]
    const int seg = blockIdx.y, d = seg >> 1, sp = seg & 1;
    const Disc& D = discs[d];
    const int N = D.N;
    const long long n = ctl->count[d][sp];
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
    unsigned* W = s_w + warp * max_N;
    for (long long t = blockIdx.x; t < Ts; t += gridDim.x) {
        for (int j = tid; j < SORT_NW * max_N; j += SORT_BLOCK) s_w[j] = 0;
        __syncthreads();
        const long long wbase = t * SORT_TILE + (long long)warp * (SORT_R * 32);
        for (int r = 0; r < SORT_R; ++r) {
            const long long k = wbase + r * 32 + lane;
            const int key = k < n ? cs[k] : N;
            const unsigned peers = __match_any_sync(FULL, key);
            if (key < N && lane == __ffs(peers) - 1) W[key] += __popc(peers);
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
            const int key = k < n ? cs[k] : N;
            const unsigned peers = __match_any_sync(FULL, key);
            const unsigned b = key < N ? W[key] : 0u;
            __syncwarp();
            if (key < N) {
                const long long o = (long long)cstart[key] + H[(long long)key * Ts + t] + b + __popc(peers & lt);
                if (o < n) {
                    cd[o] = key;
                    pd[o] = ps[k];
                }
                if (lane == __ffs(peers) - 1) W[key] = b + __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
    }
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
    const size_t smem = (size_t)(L.max_N + 1) * (16 + sizeof(T));
    auto kern = k_sweep<T, BLOCK, PPT>;
    cudaError_t e = smem_attr(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<L.grid, BLOCK, smem, L.stream>>>(L.discs, L.n_disc, L.ctl, L.st_main, L.st_bagg, L.st_binc, L.in_buf,
                                            L.seed, L.max_N);
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
    const size_t smem = (size_t)(max_N + 1) * (16 + sizeof(T));
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
        k_finalize<double><<<n_disc, 1024, smem, st>>>(discs, n_disc, ctl, out_buf, mode);
    } else {
        smem_attr(k_finalize<float>, smem);
        k_finalize<float><<<n_disc, 1024, smem, st>>>(discs, n_disc, ctl, out_buf, mode);
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
