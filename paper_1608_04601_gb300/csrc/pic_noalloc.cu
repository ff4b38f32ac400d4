// pic_noalloc.cu -- pic_sort_noalloc: the stable sort by cell of one particle
// store, on buffers the caller owns, with no device allocation at all.
//
// Some callers cannot allocate device memory while they run: code that keeps
// its own arena and forbids cudaMalloc/cudaFree (which synchronise the device
// and may fail late), plug-ins that only receive device pointers from a host
// framework, and long-running services that must not fragment or grow memory.
// For them this entry point takes its scratch (per-tile cell counts and cell
// starts) from a fixed array compiled into the library, so a call allocates
// nothing. The array (PIC_NOALLOC_SCRATCH_BYTES) is held by every GPU that
// loads the library until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/pic.h"

namespace {

constexpr int NA_BLOCK = 256, NA_NW = NA_BLOCK / 32, NA_R = 16, NA_TILE = NA_BLOCK * NA_R;
constexpr long long NA_WORDS = PIC_NOALLOC_SCRATCH_BYTES / 4;
constexpr unsigned NA_FULL = 0xFFFFFFFFu;

// Shared scratch of every call: [0, N) cell starts, then N x tiles counts.
static __device__ __align__(256) unsigned g_sort_scratch[NA_WORDS];

struct alignas(32) D4 {
    double x, y, z, w;
};

std::mutex g_mu;
void* g_scratch_addr[256] = {};

__global__ void __launch_bounds__(NA_BLOCK) na_count(const int32_t* __restrict__ c, long long n, int N,
                                                    unsigned* __restrict__ hist, long long Ts) {
    extern __shared__ unsigned s_c[];
    const int lane = threadIdx.x & 31;
    for (long long t = blockIdx.x; t < Ts; t += gridDim.x) {
        for (int j = threadIdx.x; j < N; j += NA_BLOCK) s_c[j] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < NA_TILE; i += NA_BLOCK) {
            const long long k = t * NA_TILE + i;
            const int key = k < n ? c[k] : N;
            const unsigned peers = __match_any_sync(NA_FULL, key);
            if ((unsigned)key < (unsigned)N && lane == __ffs(peers) - 1) atomicAdd(&s_c[key], (unsigned)__popc(peers));
        }
        __syncthreads();
        for (int j = threadIdx.x; j < N; j += NA_BLOCK) hist[(long long)j * Ts + t] = s_c[j];
        __syncthreads();
    }
}

// One CTA per cell: exclusive scan over the tiles in place, row total to tot[c].
__global__ void __launch_bounds__(1024) na_rows(unsigned* __restrict__ hist, long long Ts, unsigned* __restrict__ tot) {
    __shared__ unsigned s_w[32];
    __shared__ unsigned s_carry;
    const int c = blockIdx.x;
    unsigned* row = hist + (long long)c * Ts;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (long long b0 = 0; b0 < Ts; b0 += 1024) {
        const long long i = b0 + tid;
        const unsigned own = i < Ts ? row[i] : 0u;
        unsigned x = own;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(NA_FULL, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const unsigned w = s_w[lane];
            unsigned y = w;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(NA_FULL, y, o);
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
    if (tid == 0) tot[c] = s_carry;
}

// One CTA: exclusive scan of the N row totals into cell starts (in place).
__global__ void __launch_bounds__(1024) na_cells(unsigned* __restrict__ tot, int N) {
    __shared__ unsigned s_v[PIC_MAX_CELLS];
    __shared__ unsigned s_w[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = tid; j < N; j += 1024) s_v[j] = tot[j];
    __syncthreads();
    const int per = (N + 1023) / 1024, lo = tid * per, hi = min(N, lo + per);
    unsigned run = 0;
    for (int j = lo; j < hi; ++j) run += s_v[j];
    unsigned x = run;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(NA_FULL, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const unsigned w = s_w[lane];
        unsigned y = w;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(NA_FULL, y, o);
            if (lane >= o) y += t;
        }
        s_w[lane] = y - w;
    }
    __syncthreads();
    unsigned e = s_w[warp] + x - run;
    for (int j = lo; j < hi; ++j) {
        const unsigned v = s_v[j];
        tot[j] = e;
        e += v;
    }
}

// Per tile: per-warp counts, prefix over warps, then every warp places its run
// of particles in input order (rank among equal cells by match_any).
template <typename R>
__global__ void __launch_bounds__(NA_BLOCK) na_scatter(const int32_t* __restrict__ cs, const R* __restrict__ ps,
                                                      int32_t* __restrict__ cd, R* __restrict__ pd, long long n,
                                                      int N, const unsigned* __restrict__ hist,
                                                      const unsigned* __restrict__ cstart, long long Ts) {
    extern __shared__ unsigned s_w[];  // [NA_NW][N]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned* W = s_w + warp * N;
    for (long long t = blockIdx.x; t < Ts; t += gridDim.x) {
        for (int j = tid; j < NA_NW * N; j += NA_BLOCK) s_w[j] = 0;
        __syncthreads();
        const long long wbase = t * NA_TILE + (long long)warp * (NA_R * 32);
        for (int r = 0; r < NA_R; ++r) {
            const long long k = wbase + r * 32 + lane;
            const int key = k < n ? cs[k] : N;
            const unsigned peers = __match_any_sync(NA_FULL, key);
            if ((unsigned)key < (unsigned)N && lane == __ffs(peers) - 1) W[key] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        for (int j = tid; j < N; j += NA_BLOCK) {
            unsigned run = 0;
            for (int w = 0; w < NA_NW; ++w) {
                const unsigned v = s_w[w * N + j];
                s_w[w * N + j] = run;
                run += v;
            }
        }
        __syncthreads();
        for (int r = 0; r < NA_R; ++r) {
            const long long k = wbase + r * 32 + lane;
            const int key = k < n ? cs[k] : N;
            const unsigned peers = __match_any_sync(NA_FULL, key);
            const unsigned b = (unsigned)key < (unsigned)N ? W[key] : 0u;
            __syncwarp();
            if ((unsigned)key < (unsigned)N) {
                const long long o = (long long)cstart[key] + hist[(long long)key * Ts + t] + b + __popc(peers & lt);
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

// Device address of the scratch array for the current device, looked up once
// per device (the host-side name of a __device__ array is not its address).
pic_status scratch_address(unsigned** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return PIC_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return PIC_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned*>(g_scratch_addr[dev]);
    return PIC_OK;
}

template <typename R>
pic_status run_sort(const int32_t* c_in, const void* rec_in, int32_t* c_out, void* rec_out, long long n, int N,
                    cudaStream_t st, unsigned* scratch) {
    const long long Ts = (n + NA_TILE - 1) / NA_TILE;
    unsigned* cstart = scratch;
    unsigned* hist = scratch + N;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PIC_ERR_CUDA;
    const int grid = (int)(Ts < 2LL * sms ? Ts : 2LL * sms);
    const size_t smem = sizeof(unsigned) * NA_NW * N;
    if (cudaFuncSetAttribute(na_scatter<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return PIC_ERR_CUDA;
    // each launch is checked on its own, so that a failure is reported by the launch that caused it
    na_count<<<grid, NA_BLOCK, sizeof(unsigned) * N, st>>>(c_in, n, N, hist, Ts);
    if (cudaGetLastError() != cudaSuccess) return PIC_ERR_CUDA;
    na_rows<<<N, 1024, 0, st>>>(hist, Ts, cstart);
    if (cudaGetLastError() != cudaSuccess) return PIC_ERR_CUDA;
    na_cells<<<1, 1024, 0, st>>>(cstart, N);
    if (cudaGetLastError() != cudaSuccess) return PIC_ERR_CUDA;
    na_scatter<R><<<grid, NA_BLOCK, smem, st>>>(c_in, static_cast<const R*>(rec_in), c_out, static_cast<R*>(rec_out),
                                                n, N, hist, cstart, Ts);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace

extern "C" pic_status pic_sort_noalloc(const int32_t* c_in, const void* rec_in, int32_t* c_out, void* rec_out,
                                       int64_t n, int32_t n_cells, int32_t precision, void* cuda_stream) {
    if (n < 0 || n_cells < 1 || n_cells > PIC_MAX_CELLS || (precision != PIC_FP32 && precision != PIC_FP64))
        return PIC_ERR_ARG;
    if (n > 0 && (!c_in || !rec_in || !c_out || !rec_out)) return PIC_ERR_ARG;
    // the kernels move records as float4 (16 bytes) or as 32-byte groups of four doubles, and cells
    // as int32: a misaligned buffer is rejected here, before any launch
    const size_t rec_align = precision == PIC_FP64 ? sizeof(D4) : sizeof(float4);
    if (n > 0 && (!aligned(rec_in, rec_align) || !aligned(rec_out, rec_align) || !aligned(c_in, 4) ||
                  !aligned(c_out, 4)))
        return PIC_ERR_ARG;
    const long long tiles = (n + NA_TILE - 1) / NA_TILE;
    if ((long long)n_cells + (long long)n_cells * tiles > NA_WORDS) return PIC_ERR_CAPACITY;
    // an error left over from the caller's earlier work is not this call's: report it without
    // clearing it and launch nothing
    if (n > 0 && cudaPeekAtLastError() != cudaSuccess) return PIC_ERR_CUDA;
    unsigned* scratch = nullptr;
    pic_status s = scratch_address(&scratch);
    if (s != PIC_OK || n == 0) return s;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == PIC_FP64) return run_sort<D4>(c_in, rec_in, c_out, rec_out, n, n_cells, st, scratch);
    return run_sort<float4>(c_in, rec_in, c_out, rec_out, n, n_cells, st, scratch);
}
