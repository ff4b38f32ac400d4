// mlp.cu -- the warm-start network: BF16 tensor-core products with FP32
// accumulation (mma.sync m16n8k16), fused epilogues (bias, tanh, tanh'),
// MSE loss, Adam; C ABI in include/mlp.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mlp.h"
#include "pic_device.cuh"

namespace {

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------
// C[M x N] = A(M x K) B(K x N) on the tensor cores. A(m, k) = A[m lda + k]
// (a_t = 0) or A[k lda + m] (a_t = 1); B(k, n) = B[n ldb + k] (b_t = 0) or
// B[k ldb + n] (b_t = 1). Tiles of 64 x 64 x 32: four warps of 32 x 32, each
// 2 x 4 products of 16 x 8 x 16. Operands are staged K-contiguous in shared
// memory (rows padded by 8 elements against bank conflicts) and read as the
// documented per-lane fragments: lane (g = lane / 4, t = lane % 4) holds A rows
// g and g + 8, columns 2t, 2t + 1 (+ 8); B columns n = g, rows 2t, 2t + 1
// (+ 8); accumulator rows g, g + 8, columns 2t, 2t + 1.
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
};

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8, GTHREADS = 128;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(GTHREADS) k_gemm(GemmArgs g) {
    __shared__ __align__(16) bf16 sA[GBM][GBK + GPAD];
    __shared__ __align__(16) bf16 sB[GBN][GBK + GPAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;  // warp tile (32 x 32) inside the block tile
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
    const bf16 zero = __float2bfloat16_rn(0.0f);

    for (int k0 = 0; k0 < g.K; k0 += GBK) {
        // stage A (GBM x GBK) and B (GBN x GBK), K-contiguous, zero outside the matrices
        for (int e = tid; e < GBM * GBK; e += GTHREADS) {
            int r, c;
            if (g.a_t) {  // consecutive threads walk m (contiguous in memory)
                r = e % GBM;
                c = e / GBM;
            } else {
                r = e / GBK;
                c = e % GBK;
            }
            const int m = m0 + r, k = k0 + c;
            bf16 v = zero;
            if (m < g.M && k < g.K) v = g.a_t ? g.A[(size_t)k * g.lda + m] : g.A[(size_t)m * g.lda + k];
            sA[r][c] = v;
        }
        for (int e = tid; e < GBN * GBK; e += GTHREADS) {
            int r, c;
            if (g.b_t) {
                r = e % GBN;
                c = e / GBN;
            } else {
                r = e / GBK;
                c = e % GBK;
            }
            const int n = n0 + r, k = k0 + c;
            bf16 v = zero;
            if (n < g.N && k < g.K) v = g.b_t ? g.B[(size_t)k * g.ldb + n] : g.B[(size_t)n * g.ldb + k];
            sB[r][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm * 32 + i * 16 + gq;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&sA[r][kk + 2 * tq]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&sA[r + 8][kk + 2 * tq]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&sA[r][kk + 2 * tq + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&sA[r + 8][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn * 32 + j * 8 + gq;
                bfr[j][0] = *reinterpret_cast<const uint32_t*>(&sB[c][kk + 2 * tq]);
                bfr[j][1] = *reinterpret_cast<const uint32_t*>(&sB[c][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
    // epilogue
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm * 32 + i * 16 + gq + (r >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + j * 8 + 2 * tq + (r & 1);
                if (m >= g.M || n >= g.N) continue;
                float v = acc[i][j][r];
                const size_t o = (size_t)m * g.ldc + n;
                if (g.ep == EP_BIAS_TANH) v = tanhf(v + g.bias[n]);
                else if (g.ep == EP_BIAS) v = v + g.bias[n];
                else if (g.ep == EP_DTANH) {
                    const float y = g.yprev[o];
                    v = v * (1.0f - y * y);
                }
                g.C32[o] = v;
                if (g.C16) g.C16[o] = __float2bfloat16_rn(v);
            }
}

// Column sums of g[rows x cols] (bias gradients), fixed order per column.
__global__ void k_colsum(const float* __restrict__ g, int rows, int cols, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += g[(size_t)r * cols + c];
    out[c] = s;
}

__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// Mean squared error over n = rows x cols values and its gradient 2 (y - t) / n
// (FP32 and BF16); one block, fixed reduction order.
__global__ void __launch_bounds__(1024) k_mse(const float* __restrict__ y, const float* __restrict__ t, long long n,
                                              float* __restrict__ g32, bf16* __restrict__ g16, float* __restrict__ loss) {
    __shared__ float s_w[32];
    const float sc = 2.0f / (float)n;
    float acc = 0.0f;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const float d = y[i] - t[i];
        acc += d * d;
        const float gv = sc * d;
        g32[i] = gv;
        g16[i] = __float2bfloat16_rn(gv);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? s_w[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
        if (threadIdx.x == 0) *loss = v / (float)n;
    }
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

cudaError_t gemm(cudaStream_t st, const bf16* A, int lda, int a_t, const bf16* B, int ldb, int b_t, int M, int N, int K,
                 int ep, const float* bias, const float* yprev, float* C32, bf16* C16, int ldc) {
    GemmArgs g{A, B, lda, ldb, a_t, b_t, M, N, K, ep, bias, yprev, C32, C16, ldc};
    dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
    k_gemm<<<grid, GTHREADS, 0, st>>>(g);
    return cudaGetLastError();
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
        e = gemm(c->stream, A, in, 0, c->w16 + c->w16off[l], in, 0, batch, out, in,
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
              dalloc(c, &c->loss, 1);
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
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? PIC_OK : fail(c, PIC_ERR_CUDA, "get params", e);
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
    k_mse<<<1, 1024, 0, c->stream>>>(c->y32[L - 1], t, ny, c->g32[cur], c->g16[cur], loss ? loss : c->loss);
    e = cudaGetLastError();
    for (int l = L - 1; l >= 0 && e == cudaSuccess; --l) {
        const int in = c->sizes[l], out = c->sizes[l + 1];
        const bf16* X = l == 0 ? c->x16 : c->y16[l - 1];
        // dW_l = G^T X: M = out, N = in, K = batch
        e = gemm(c->stream, c->g16[cur], out, 1, X, in, 1, out, in, batch, EP_STORE, nullptr, nullptr,
                 c->grad + c->woff[l], nullptr, in);
        if (e != cudaSuccess) break;
        k_colsum<<<(out + 255) / 256, 256, 0, c->stream>>>(c->g32[cur], batch, out, c->grad + c->boff[l]);
        e = cudaGetLastError();
        if (e != cudaSuccess || l == 0) break;
        // G_{l-1} = (G W_l) * (1 - y_{l-1}^2): M = batch, N = in, K = out
        e = gemm(c->stream, c->g16[cur], out, 0, c->w16 + c->w16off[l], in, 1, batch, in, out, EP_DTANH, nullptr,
                 c->y32[l - 1], c->g32[1 - cur], c->g16[1 - cur], in);
        cur = 1 - cur;
    }
    return e == cudaSuccess ? PIC_OK : fail(c, PIC_ERR_CUDA, "backward", e);
}

pic_status mlp_get_grads(mlp_ctx* c, float* host) {
    if (!c || !host) return PIC_ERR_ARG;
    cudaError_t e =
        cudaMemcpyAsync(host, c->grad, sizeof(float) * (size_t)c->n_params, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? PIC_OK : fail(c, PIC_ERR_CUDA, "get grads", e);
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
    cudaError_t e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? PIC_OK : fail(c, PIC_ERR_CUDA, "synchronize", e);
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
