// mlp.cu -- the warm-start network: BF16 products on the tcgen05 tensor cores
// with FP32 accumulation in tensor memory, fused epilogues (bias, tanh,
// tanh'), MSE loss, Adam; C ABI in include/mlp.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mlp.h"
#include "pic_device.cuh"

namespace {

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------
// C[M x N] = A(M x K) B(K x N) on the 5th-generation tensor cores (tcgen05).
// A(m, k) = A[m lda + k] (a_t = 0) or A[k lda + m] (a_t = 1); B(k, n) =
// B[n ldb + k] (b_t = 0) or B[k ldb + n] (b_t = 1).
//
// One CTA of 128 threads per 128 x 64 tile of C, K in chunks of 64. The
// operands of a chunk sit in shared memory K-major without swizzle: 8 x 8 core
// matrices of 128 contiguous bytes (row r of a core matrix at 16 r bytes),
// core matrices adjacent in K 128 bytes apart (the descriptor's leading-
// dimension offset), 8-row groups 1024 bytes apart (its stride offset), zero
// outside the matrices. Two buffers: while the tensor core multiplies chunk i
// (one thread issues four tcgen05.mma kind::f16, M 128, N 64, K 16, BF16
// operands, FP32 accumulator in 64 columns of tensor memory, and commits them
// to the buffer's mbarrier), the threads already load chunk i + 1 into
// registers; a buffer is overwritten only after its mbarrier says the products
// that read it are done (bounded waits). The epilogue reads the accumulator
// with tcgen05.ld (warp w owns lanes 32 w .. 32 w + 31, the tile's rows),
// parks it in shared memory and writes C row by row, coalesced, applying the
// fused bias / tanh / tanh' step.
enum Epilogue {
    EP_STORE = 0,     // C32 = acc
    EP_BIAS_TANH = 1, // z = acc + bias; C32 = tanh z; C16 = bf16(C32)
    EP_BIAS = 2,      // C32 = acc + bias; C16 = bf16(C32)
    EP_DTANH = 3,     // C32 = acc (1 - yprev^2); C16 = bf16(C32)
};

struct GemmArgs {
    const bf16* A;
    const bf16* B;
    int lda, ldb, a_t, b_t;
    int M, N, K;
    int ep;
    const float* bias;
    const float* yprev;  // [M x N], ld = ldc
    float* C32;
    bf16* C16;
    int ldc;
    unsigned* err;       // set to MLP_ERR_TIMEOUT if a bounded wait gave up
};

constexpr int TBM = 128, TBN = 64, TBK = 64, TTHREADS = 128, TMEM_COLS = 64;
constexpr unsigned CM_BYTES = 128;                    // one 8 x 8 BF16 core matrix
constexpr unsigned LBO = CM_BYTES;                    // next core matrix along K
constexpr unsigned SBO = (TBK / 8) * CM_BYTES;        // next 8-row group
constexpr unsigned A_BYTES = TBM * TBK * 2, B_BYTES = TBN * TBK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr unsigned GEMM_SMEM = 2 * STAGE_BYTES;       // dynamic shared memory: two operand buffers
constexpr int UA = TBM * TBK / 8 / TTHREADS, UB = TBN * TBK / 8 / TTHREADS;  // 8-element units per thread
constexpr int TC_TRIES = 1 << 20;                     // polls of a bounded mbarrier wait
constexpr unsigned MLP_ERR_TIMEOUT = 1u;
static_assert((TBN + 1) * TBM * 4 <= GEMM_SMEM, "epilogue tile must fit in the operand buffers");

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 in bits 17-22, M / 16 in bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                           ((uint32_t)(TBM >> 4) << 24);

__device__ __forceinline__ uint32_t s_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address / 16 (bits 0-13), leading-dimension byte offset
// / 16 (16-29), stride byte offset / 16 (32-45), the fixed version field 0b001 (46-48), base
// offset 0, no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(SBO >> 4) << 32) |
           (1ull << 46);
}

// Byte offset of element (row r, k) of a staged operand tile.
__device__ __forceinline__ unsigned cm_off(int r, int k) {
    return (unsigned)(((r >> 3) * (TBK / 8) + (k >> 3)) * CM_BYTES + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ bool tc_wait(uint32_t mb, unsigned parity) {
    for (int it = 0; it < TC_TRIES; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mb), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// How a thread moves an operand: element gathers (any layout and alignment), 16-byte loads of
// k-contiguous rows, or (transposed operand, m contiguous) 16- / 8-byte loads of 8 rows of k that
// the thread transposes in registers.
enum StageMode { SM_GATHER = 0, SM_VEC = 1, SM_TVEC = 2 };

// Chosen on the host per operand; the product kernel is compiled for each pair of modes.
inline int stage_mode(const void* X, int ld, int t) {
    if ((ld % 8) != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0) return SM_GATHER;
    return t ? SM_TVEC : SM_VEC;
}

// Unit q of this thread (8 consecutive k of one row of the tile): its row and 8-column group.
// SM_VEC: the eight lanes of a quarter warp take the eight rows of one core matrix (its 128 bytes
// in one conflict-free store), the next eight lanes the next 8 k of the same rows. SM_GATHER:
// consecutive lanes take consecutive rows. SM_TVEC: the thread owns the U rows U (tid % (R / U))
// .. + U - 1 at the 8 k of group tid / (R / U), unit q being its row q.
template <int R, int U, int MODE>
__device__ __forceinline__ void unit_rk(int q, int& r, int& kc) {
    const int tid = threadIdx.x, u = tid + q * TTHREADS;
    if constexpr (MODE == SM_VEC) {
        r = (u >> 6) * 8 + (u & 7);
        kc = (u >> 3) & 7;
    } else if constexpr (MODE == SM_TVEC) {
        r = U * (tid % (R / U)) + q;
        kc = tid / (R / U);
    } else {
        r = u % R;
        kc = u / R;
    }
}

// One k row of a transposed block: U consecutive BF16 (rows m .. m + U - 1) as U / 2 words.
template <int U>
__device__ __forceinline__ void load_row(uint32_t (&w)[U / 2], const bf16* src, int avail) {
#pragma unroll
    for (int p = 0; p < U / 2; ++p) w[p] = 0u;
    if (avail >= U) {
        if constexpr (U == 8) {
            const uint4 x = *reinterpret_cast<const uint4*>(src);
            w[0] = x.x;
            w[1] = x.y;
            w[2] = x.z;
            w[3] = x.w;
        } else {
            const uint2 x = *reinterpret_cast<const uint2*>(src);
            w[0] = x.x;
            w[1] = x.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < U; ++e)
            if (e < avail) w[e >> 1] |= (uint32_t)__bfloat16_as_ushort(src[e]) << (16 * (e & 1));
    }
}

// Loads this thread's units of the chunk at k0 of an operand X (rows x K; element (r, k) at
// X[r ld + k], or X[k ld + r] if t) into registers, 8 BF16 per uint4 (k ascending), zero outside.
template <int R, int U, int MODE>
__device__ __forceinline__ void load_units(uint4 (&v)[U], const bf16* __restrict__ X, int ld, int t, int rows, int K,
                                           int r0, int k0) {
    static_assert(U == 4 || U == 8, "a transposed block is 8 k by 4 or 8 rows");
    if constexpr (MODE == SM_TVEC) {
        int r, kc;
        unit_rk<R, U, MODE>(0, r, kc);
        const int m = r0 + r;  // first of the thread's U rows (a multiple of U)
        uint32_t w[8][U / 2];  // w[i]: rows m .. m + U - 1 at k = k0 + 8 kc + i
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = k0 + 8 * kc + i;
            load_row<U>(w[i], X + (size_t)k * ld + m, k < K ? rows - m : 0);
        }
        // transpose: unit j (row m + j) word p holds k = 2p (low half) and 2p + 1 (high half)
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const unsigned sel = (j & 1) ? 0x7632u : 0x5410u;
            v[j] = make_uint4(__byte_perm(w[0][j >> 1], w[1][j >> 1], sel), __byte_perm(w[2][j >> 1], w[3][j >> 1], sel),
                              __byte_perm(w[4][j >> 1], w[5][j >> 1], sel), __byte_perm(w[6][j >> 1], w[7][j >> 1], sel));
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
        int r, kc;
        unit_rk<R, U, MODE>(q, r, kc);
        const int m = r0 + r, k = k0 + 8 * kc;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (m < rows) {
            if (MODE == SM_VEC && k + 8 <= K) {
                const uint4 x = *reinterpret_cast<const uint4*>(X + (size_t)m * ld + k);
                w[0] = x.x;
                w[1] = x.y;
                w[2] = x.z;
                w[3] = x.w;
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (k + j < K) {
                        const bf16 e = t ? X[(size_t)(k + j) * ld + m] : X[(size_t)m * ld + k + j];
                        w[j >> 1] |= (uint32_t)__bfloat16_as_ushort(e) << (16 * (j & 1));
                    }
            }
        }
        v[q] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

template <int R, int U, int MODE>
__device__ __forceinline__ void store_units(unsigned char* s, const uint4 (&v)[U]) {
#pragma unroll
    for (int q = 0; q < U; ++q) {
        int r, kc;
        unit_rk<R, U, MODE>(q, r, kc);
        *reinterpret_cast<uint4*>(s + cm_off(r, 8 * kc)) = v[q];
    }
}

template <int MA, int MB>  // staging modes of A and B
__global__ void __launch_bounds__(TTHREADS) k_gemm(GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem[];  // two buffers of A (128 x 64) then B (64 x 64)
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    const uint32_t mb0 = s_addr(&mbar[0]);  // buffer b's barrier at mb0 + 8 b
    if (warp == 0) {  // tensor memory for the accumulator: one warp allocates, the same warp frees
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0 + 8u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const int nk = (g.K + TBK - 1) / TBK;
    uint4 ra[UA], rb[UB];
    load_units<TBM, UA, MA>(ra, g.A, g.lda, g.a_t, g.M, g.K, m0, 0);
    load_units<TBN, UB, MB>(rb, g.B, g.ldb, g.b_t, g.N, g.K, n0, 0);
    bool ok = true;
    int last = -1;  // last chunk whose products were committed
    for (int i = 0; i < nk; ++i) {
        const int b = i & 1;
        // buffer b last held chunk i - 2: its products must be done before it is overwritten
        const bool done = i < 2 || tc_wait(mb0 + 8u * b, (((unsigned)i >> 1) & 1u) ^ 1u);
        if (__syncthreads_or(!done)) {  // one decision for the whole CTA
            ok = false;
            break;
        }
        unsigned char* sa = smem + b * STAGE_BYTES;
        store_units<TBM, UA, MA>(sa, ra);
        store_units<TBN, UB, MB>(sa + A_BYTES, rb);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the operands, to the tensor core's proxy
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = s_addr(sa), b0 = a0 + A_BYTES;
#pragma unroll
            for (int s = 0; s < TBK / 16; ++s) {  // K 16 per instruction: two core matrices along K
                const uint64_t ad = sdesc(a0 + 2 * s * CM_BYTES), bd = sdesc(b0 + 2 * s * CM_BYTES);
                const uint32_t accumulate = (i > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(IDESC), "r"(accumulate)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb0 + 8u * b)
                         : "memory");
        }
        last = i;
        if (i + 1 < nk) {  // the next chunk's loads overlap the products just issued
            load_units<TBM, UA, MA>(ra, g.A, g.lda, g.a_t, g.M, g.K, m0, (i + 1) * TBK);
            load_units<TBN, UB, MB>(rb, g.B, g.ldb, g.b_t, g.N, g.K, n0, (i + 1) * TBK);
        }
    }
    if (ok) {  // the last commit covers every product issued before it
        const bool done = tc_wait(mb0 + 8u * (last & 1), ((unsigned)last >> 1) & 1u);
        if (__syncthreads_or(!done)) ok = false;
    }
    if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // accumulator -> shared tile T[128][65] (thread = row: conflict-free with the odd stride)
        float* T = reinterpret_cast<float*>(smem);
        const int row = warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < TBN; c0 += 16) {
            uint32_t r[16];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) T[row * (TBN + 1) + c0 + j] = __uint_as_float(r[j]);
        }
        __syncthreads();
        // row by row: a warp writes 32 consecutive columns of one row. Each thread keeps one column
        // (its bias loaded once) and takes every second row; the loads of a batch of rows (yprev)
        // are all issued before its stores, which the compiler could not reorder (aliasing).
        const int cc = tid % TBN, rb = tid / TBN, n = n0 + cc;
        const bool nin = n < g.N;
        const float bn = (nin && (g.ep == EP_BIAS_TANH || g.ep == EP_BIAS)) ? g.bias[n] : 0.0f;
        constexpr int RSTEP = TTHREADS / TBN, BATCH = 16;
#pragma unroll 1
        for (int r0 = rb; r0 < TBM; r0 += RSTEP * BATCH) {
            float y[BATCH];
#pragma unroll
            for (int j = 0; j < BATCH; ++j) {
                const int m = m0 + r0 + RSTEP * j;
                y[j] = (g.ep == EP_DTANH && nin && m < g.M) ? g.yprev[(size_t)m * g.ldc + n] : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < BATCH; ++j) {
                const int rr = r0 + RSTEP * j, m = m0 + rr;
                if (!nin || m >= g.M) continue;
                float v = T[rr * (TBN + 1) + cc];
                if (g.ep == EP_BIAS_TANH) v = tanhf(v + bn);
                else if (g.ep == EP_BIAS) v = v + bn;
                else if (g.ep == EP_DTANH) v = v * (1.0f - y[j] * y[j]);
                const size_t o = (size_t)m * g.ldc + n;
                g.C32[o] = v;
                if (g.C16) g.C16[o] = __float2bfloat16_rn(v);
            }
        }
    } else if (tid == 0) {
        atomicOr(g.err, MLP_ERR_TIMEOUT);
        if (last >= 0) tc_wait(mb0 + 8u * (last & 1), ((unsigned)last >> 1) & 1u);  // a last bounded chance for the products in flight
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Column sums of g[rows x cols] (bias gradients): a block of 32 columns x 8 row groups, each
// thread summing every eighth row, then the eight partial sums in order (a fixed order per column).
__global__ void __launch_bounds__(256) k_colsum(const float* __restrict__ g, int rows, int cols,
                                                float* __restrict__ out) {
    __shared__ float s[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x, gy = threadIdx.y;
    float acc = 0.0f;
    if (c < cols)
        for (int r = gy; r < rows; r += 8) acc += g[(size_t)r * cols + c];
    s[gy][threadIdx.x] = acc;
    __syncthreads();
    if (gy == 0 && c < cols) {
        float t = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += s[k][threadIdx.x];
        out[c] = t;
    }
}

__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// Sum of a block's values in a fixed tree (warp shuffles, then the warps' sums); thread 0 gets it.
__device__ __forceinline__ float block_sum256(float v) {
    __shared__ float s_w[8];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.0f;
    if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) t += s_w[k];
    return t;
}

// Mean squared error over n = rows x cols values and its gradient 2 (y - t) / n (FP32 and BF16):
// each block strides over the values and leaves its partial sum; k_mse_final adds the partial sums
// in order (the grid depends on n only, so the reduction order is fixed).
constexpr int MSE_BLOCKS = 256;
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ y, const float* __restrict__ t, long long n,
                                             float* __restrict__ g32, bf16* __restrict__ g16,
                                             float* __restrict__ part) {
    const float sc = 2.0f / (float)n;
    float acc = 0.0f;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const float d = y[i] - t[i];
        acc += d * d;
        const float gv = sc * d;
        g32[i] = gv;
        g16[i] = __float2bfloat16_rn(gv);
    }
    const float b = block_sum256(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__global__ void __launch_bounds__(256) k_mse_final(const float* __restrict__ part, int nb, long long n,
                                                   float* __restrict__ loss) {
    const float b = block_sum256(threadIdx.x < nb ? part[threadIdx.x] : 0.0f);
    if (threadIdx.x == 0) *loss = b / (float)n;
}

// Adam on the FP32 master parameters; refreshes the BF16 weight copies
// (w16[i] for i < n16: the weights of every layer packed, biases skipped).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Weight copy of layer: master W (at p + off) -> bf16.
__global__ void k_weights_bf16(const float* __restrict__ p, long long off, long long n, bf16* __restrict__ w) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        w[i] = __float2bfloat16_rn(p[off + i]);
}

// Glorot-uniform initial weights from Philox (key = seed, counter = (index,
// layer, 0xA0, 0)), zero biases.
__global__ void k_init(float* __restrict__ p, long long off, long long nw, long long nb, int layer, float a,
                       unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw + nb; i += (long long)gridDim.x * blockDim.x) {
        if (i < nw) {
            const pic::U4 r = pic::philox4x32_10((uint32_t)i, (uint32_t)layer, 0xA0u, 0u, (uint32_t)seed,
                                                 (uint32_t)(seed >> 32));
            p[off + i] = a * (2.0f * pic::u01(r.x) - 1.0f);
        } else {
            p[off + i] = 0.0f;
        }
    }
}

}  // namespace

struct mlp_ctx {
    int L = 0;
    int sizes[MLP_MAX_LAYERS + 1] = {};
    int max_batch = 0;
    long long woff[MLP_MAX_LAYERS] = {}, boff[MLP_MAX_LAYERS] = {}, w16off[MLP_MAX_LAYERS] = {};
    long long n_params = 0, n_w = 0;
    float* p = nullptr;     // master parameters
    float* grad = nullptr;  // gradients (same layout)
    float* m = nullptr;
    float* v = nullptr;
    bf16* w16 = nullptr;    // weights, packed by layer
    bf16* x16 = nullptr;    // input [max_batch x sizes[0]]
    float* y32[MLP_MAX_LAYERS] = {};
    bf16* y16[MLP_MAX_LAYERS] = {};
    float* g32[2] = {};
    bf16* g16[2] = {};
    float* loss = nullptr;
    float* mse_part = nullptr;  // per-block partial sums of the loss
    unsigned* d_err = nullptr;  // device word: a product's bounded wait gave up
    long long step = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<void*> allocs;
    std::string err;
};

namespace {

pic_status fail(mlp_ctx* c, pic_status s, const char* what, cudaError_t e = cudaSuccess) {
    if (c) {
        c->err = what;
        if (e != cudaSuccess) {
            c->err += ": ";
            c->err += cudaGetErrorString(e);
        }
    }
    return s;
}

template <typename T>
bool dalloc(mlp_ctx* c, T** p, size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) return false;
    c->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return true;
}

typedef void (*GemmKernel)(GemmArgs);
GemmKernel gemm_kernel(int ma, int mb) {
    static const GemmKernel K[3][3] = {
        {k_gemm<SM_GATHER, SM_GATHER>, k_gemm<SM_GATHER, SM_VEC>, k_gemm<SM_GATHER, SM_TVEC>},
        {k_gemm<SM_VEC, SM_GATHER>, k_gemm<SM_VEC, SM_VEC>, k_gemm<SM_VEC, SM_TVEC>},
        {k_gemm<SM_TVEC, SM_GATHER>, k_gemm<SM_TVEC, SM_VEC>, k_gemm<SM_TVEC, SM_TVEC>}};
    return K[ma][mb];
}

cudaError_t gemm(mlp_ctx* c, const bf16* A, int lda, int a_t, const bf16* B, int ldb, int b_t, int M, int N, int K,
                 int ep, const float* bias, const float* yprev, float* C32, bf16* C16, int ldc) {
    GemmArgs g{A, B, lda, ldb, a_t, b_t, M, N, K, ep, bias, yprev, C32, C16, ldc, c->d_err};
    dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM);
    gemm_kernel(stage_mode(A, lda, a_t), stage_mode(B, ldb, b_t))<<<grid, TTHREADS, GEMM_SMEM, c->stream>>>(g);
    return cudaGetLastError();
}

// Synchronises the context's stream and reports a product whose bounded wait gave up.
pic_status sync_checked(mlp_ctx* c, const char* what) {
    unsigned h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, what, e);
    if (h) return fail(c, PIC_ERR_TIMEOUT, "a tensor-core product's bounded wait timed out");
    return PIC_OK;
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1024 ? (b > 0 ? b : 1) : 1024);
}

cudaError_t refresh_bf16(mlp_ctx* c) {
    for (int l = 0; l < c->L; ++l) {
        const long long nw = (long long)c->sizes[l] * c->sizes[l + 1];
        k_weights_bf16<<<grid_for(nw), 256, 0, c->stream>>>(c->p, c->woff[l], nw, c->w16 + c->w16off[l]);
    }
    return cudaGetLastError();
}

cudaError_t forward(mlp_ctx* c, int batch, const float* x) {
    const long long nx = (long long)batch * c->sizes[0];
    k_to_bf16<<<grid_for(nx), 256, 0, c->stream>>>(x, c->x16, nx);
    cudaError_t e = cudaGetLastError();
    for (int l = 0; l < c->L && e == cudaSuccess; ++l) {
        const int in = c->sizes[l], out = c->sizes[l + 1];
        const bf16* A = l == 0 ? c->x16 : c->y16[l - 1];
        e = gemm(c, A, in, 0, c->w16 + c->w16off[l], in, 0, batch, out, in,
                 l + 1 < c->L ? EP_BIAS_TANH : EP_BIAS, c->p + c->boff[l], nullptr, c->y32[l], c->y16[l], out);
    }
    return e;
}

}  // namespace

extern "C" {

pic_status mlp_create(mlp_ctx** out, int32_t n_layers, const int32_t* sizes, int32_t max_batch, uint64_t seed,
                      void* cuda_stream) {
    if (!out || !sizes || n_layers < 1 || n_layers > MLP_MAX_LAYERS || max_batch < 1) return PIC_ERR_ARG;
    *out = nullptr;
    for (int l = 0; l <= n_layers; ++l)
        if (sizes[l] < 1 || sizes[l] > MLP_MAX_WIDTH) return PIC_ERR_ARG;
    // the product's two operand buffers take 48 KB of dynamic shared memory (above the default limit
    // together with its barriers)
    for (int ma = 0; ma < 3; ++ma)
        for (int mb = 0; mb < 3; ++mb)
            if (cudaFuncSetAttribute(gemm_kernel(ma, mb), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM) !=
                cudaSuccess)
                return PIC_ERR_CUDA;
    mlp_ctx* c = new mlp_ctx();
    c->L = n_layers;
    c->max_batch = max_batch;
    int wmax = 0;
    for (int l = 0; l <= n_layers; ++l) {
        c->sizes[l] = sizes[l];
        wmax = wmax > sizes[l] ? wmax : sizes[l];
    }
    for (int l = 0; l < n_layers; ++l) {
        const long long nw = (long long)sizes[l] * sizes[l + 1];
        c->woff[l] = c->n_params;
        c->boff[l] = c->n_params + nw;
        c->n_params += nw + sizes[l + 1];
        c->w16off[l] = c->n_w;
        c->n_w += nw;
    }
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return PIC_ERR_CUDA;
        }
        c->own_stream = true;
    }
    const size_t P = (size_t)c->n_params;
    bool ok = dalloc(c, &c->p, P) && dalloc(c, &c->grad, P) && dalloc(c, &c->m, P) && dalloc(c, &c->v, P) &&
              dalloc(c, &c->w16, (size_t)c->n_w) && dalloc(c, &c->x16, (size_t)max_batch * sizes[0]) &&
              dalloc(c, &c->loss, 1) && dalloc(c, &c->d_err, 1) &&
              dalloc(c, &c->mse_part, (size_t)MSE_BLOCKS);
    for (int l = 0; l < n_layers && ok; ++l)
        ok = dalloc(c, &c->y32[l], (size_t)max_batch * sizes[l + 1]) && dalloc(c, &c->y16[l], (size_t)max_batch * sizes[l + 1]);
    for (int b = 0; b < 2 && ok; ++b)
        ok = dalloc(c, &c->g32[b], (size_t)max_batch * wmax) && dalloc(c, &c->g16[b], (size_t)max_batch * wmax);
    if (!ok) {
        mlp_destroy(c);
        return PIC_ERR_CUDA;
    }
    cudaMemsetAsync(c->m, 0, P * sizeof(float), c->stream);
    cudaMemsetAsync(c->v, 0, P * sizeof(float), c->stream);
    cudaMemsetAsync(c->grad, 0, P * sizeof(float), c->stream);
    cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream);
    for (int l = 0; l < n_layers; ++l) {
        const long long nw = (long long)sizes[l] * sizes[l + 1];
        const float a = std::sqrt(6.0f / (float)(sizes[l] + sizes[l + 1]));
        k_init<<<grid_for(nw + sizes[l + 1]), 256, 0, c->stream>>>(c->p, c->woff[l], nw, sizes[l + 1], l, a, seed);
    }
    cudaError_t e = refresh_bf16(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        mlp_destroy(c);
        return PIC_ERR_CUDA;
    }
    *out = c;
    return PIC_OK;
}

int64_t mlp_param_count(const mlp_ctx* c) { return c ? c->n_params : 0; }

pic_status mlp_set_params(mlp_ctx* c, const float* host) {
    if (!c || !host) return PIC_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(c->p, host, sizeof(float) * (size_t)c->n_params, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = refresh_bf16(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? PIC_OK : fail(c, PIC_ERR_CUDA, "set params", e);
}

pic_status mlp_get_params(mlp_ctx* c, float* host) {
    if (!c || !host) return PIC_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(host, c->p, sizeof(float) * (size_t)c->n_params, cudaMemcpyDeviceToHost, c->stream);
    return e == cudaSuccess ? sync_checked(c, "get params") : fail(c, PIC_ERR_CUDA, "get params", e);
}

pic_status mlp_forward(mlp_ctx* c, int32_t batch, const float* x, float* y) {
    if (!c || !x || !y || batch < 1 || batch > c->max_batch) return PIC_ERR_ARG;
    cudaError_t e = forward(c, batch, x);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(y, c->y32[c->L - 1], sizeof(float) * (size_t)batch * c->sizes[c->L],
                            cudaMemcpyDeviceToDevice, c->stream);
    return e == cudaSuccess ? PIC_OK : fail(c, PIC_ERR_CUDA, "forward", e);
}

pic_status mlp_loss_grad(mlp_ctx* c, int32_t batch, const float* x, const float* t, float* loss) {
    if (!c || !x || !t || batch < 1 || batch > c->max_batch) return PIC_ERR_ARG;
    cudaError_t e = forward(c, batch, x);
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "forward", e);
    const int L = c->L;
    const long long ny = (long long)batch * c->sizes[L];
    int cur = 0;
    const int nb = (int)std::min<long long>(MSE_BLOCKS, (ny + 255) / 256);
    k_mse<<<nb, 256, 0, c->stream>>>(c->y32[L - 1], t, ny, c->g32[cur], c->g16[cur], c->mse_part);
    k_mse_final<<<1, 256, 0, c->stream>>>(c->mse_part, nb, ny, loss ? loss : c->loss);
    e = cudaGetLastError();
    for (int l = L - 1; l >= 0 && e == cudaSuccess; --l) {
        const int in = c->sizes[l], out = c->sizes[l + 1];
        const bf16* X = l == 0 ? c->x16 : c->y16[l - 1];
        // dW_l = G^T X: M = out, N = in, K = batch
        e = gemm(c, c->g16[cur], out, 1, X, in, 1, out, in, batch, EP_STORE, nullptr, nullptr,
                 c->grad + c->woff[l], nullptr, in);
        if (e != cudaSuccess) break;
        k_colsum<<<(out + 31) / 32, dim3(32, 8), 0, c->stream>>>(c->g32[cur], batch, out, c->grad + c->boff[l]);
        e = cudaGetLastError();
        if (e != cudaSuccess || l == 0) break;
        // G_{l-1} = (G W_l) * (1 - y_{l-1}^2): M = batch, N = in, K = out
        e = gemm(c, c->g16[cur], out, 0, c->w16 + c->w16off[l], in, 1, batch, in, out, EP_DTANH, nullptr,
                 c->y32[l - 1], c->g32[1 - cur], c->g16[1 - cur], in);
        cur = 1 - cur;
    }
    return e == cudaSuccess ? PIC_OK : fail(c, PIC_ERR_CUDA, "backward", e);
}

pic_status mlp_get_grads(mlp_ctx* c, float* host) {
    if (!c || !host) return PIC_ERR_ARG;
    cudaError_t e =
        cudaMemcpyAsync(host, c->grad, sizeof(float) * (size_t)c->n_params, cudaMemcpyDeviceToHost, c->stream);
    return e == cudaSuccess ? sync_checked(c, "get grads") : fail(c, PIC_ERR_CUDA, "get grads", e);
}

pic_status mlp_adam(mlp_ctx* c, float lr, float beta1, float beta2, float eps) {
    if (!c || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0)) return PIC_ERR_ARG;
    c->step += 1;
    const float c1 = (float)(1.0 - std::pow((double)beta1, (double)c->step));
    const float c2 = (float)(1.0 - std::pow((double)beta2, (double)c->step));
    k_adam<<<grid_for(c->n_params), 256, 0, c->stream>>>(c->p, c->grad, c->m, c->v, c->n_params, lr, beta1, beta2, eps,
                                                         c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = refresh_bf16(c);
    return e == cudaSuccess ? PIC_OK : fail(c, PIC_ERR_CUDA, "adam", e);
}

pic_status mlp_train_step(mlp_ctx* c, int32_t batch, const float* x, const float* t, float lr, float* loss) {
    pic_status s = mlp_loss_grad(c, batch, x, t, loss);
    if (s != PIC_OK) return s;
    return mlp_adam(c, lr, 0.9f, 0.999f, 1e-8f);
}

pic_status mlp_sync(mlp_ctx* c) {
    if (!c) return PIC_ERR_ARG;
    return sync_checked(c, "synchronize");
}

void mlp_destroy(mlp_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (void* q : c->allocs) cudaFree(q);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* mlp_last_error(const mlp_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
