/* mlp.h -- C ABI of the warm-start network (GB300, sm_103a).
 *
 * The paper proposes initial values closer to the periodic state to shorten
 * the 1000-4000 rf periods its PIC runs needed (section "Numerical parameters
 * and initial values"). This network maps discharge parameters to the
 * periodic-state profiles (n_e, n_i, mean electron energy on a uniform grid);
 * pic_load_profiles (pic.h) then samples the initial particles from them.
 *
 * A multilayer perceptron: layer l computes z_l = y_{l-1} W_l^T + b_l with
 * W_l [out_l x in_l]; hidden layers apply tanh, the last layer is linear.
 * Weights are BF16 copies of FP32 master weights; every product runs on the
 * tcgen05 tensor cores (BF16 operands from shared memory, FP32 accumulator in
 * tensor memory); activations feed the next product as BF16.
 * Training minimises the mean squared error over the outputs with Adam.
 *
 * Memory: the context owns all device memory (weights, Adam moments,
 * activations for max_batch rows). x, t, y and loss arguments are DEVICE
 * pointers to FP32 row-major arrays; calls are asynchronous on the context's
 * stream (mlp_sync waits). Host arrays are used only by mlp_set_params,
 * mlp_get_params and mlp_get_grads, which synchronise.
 * Parameter layout (host arrays): for each layer in order, W_l row-major
 * [out_l][in_l], then b_l [out_l].
 * Errors: PIC_ERR_ARG for bad sizes or pointers, PIC_ERR_CUDA for CUDA
 * failures (text in mlp_last_error); PIC_ERR_TIMEOUT from mlp_sync,
 * mlp_get_params or mlp_get_grads if a product's bounded wait on the tensor
 * core gave up (its outputs are then not written).                          */
#ifndef MLP_H
#define MLP_H

#include <stdint.h>

#include "pic.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlp_ctx mlp_ctx;

#define MLP_MAX_LAYERS 8
#define MLP_MAX_WIDTH 4096

/* sizes[0] inputs, sizes[1..n_layers] layer outputs; weights drawn uniform in
 * +-sqrt(6 / (in + out)) from Philox streams keyed by seed, biases zero.
 * cuda_stream NULL: the context creates its own stream.                     */
pic_status mlp_create(mlp_ctx** out, int32_t n_layers, const int32_t* sizes, int32_t max_batch, uint64_t seed,
                      void* cuda_stream);
int64_t mlp_param_count(const mlp_ctx* ctx);
pic_status mlp_set_params(mlp_ctx* ctx, const float* host);
pic_status mlp_get_params(mlp_ctx* ctx, float* host);

/* y[batch x sizes[n_layers]] = network(x[batch x sizes[0]]); batch <= max_batch. */
pic_status mlp_forward(mlp_ctx* ctx, int32_t batch, const float* x, float* y);

/* Forward and backward of L = mean over batch x outputs of (y - t)^2: *loss
 * (device, one float) and the gradients of all parameters (kept in the
 * context; FP32, same layout as the parameters).                            */
pic_status mlp_loss_grad(mlp_ctx* ctx, int32_t batch, const float* x, const float* t, float* loss);
pic_status mlp_get_grads(mlp_ctx* ctx, float* host);

/* One Adam step (Kingma and Ba) from the stored gradients on the FP32 master
 * weights, bias-corrected with the context's step count; refreshes the BF16
 * copies.                                                                   */
pic_status mlp_adam(mlp_ctx* ctx, float lr, float beta1, float beta2, float eps);

/* mlp_loss_grad then mlp_adam. */
pic_status mlp_train_step(mlp_ctx* ctx, int32_t batch, const float* x, const float* t, float lr, float* loss);

pic_status mlp_sync(mlp_ctx* ctx);
void mlp_destroy(mlp_ctx* ctx); /* NULL-safe */
const char* mlp_last_error(const mlp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
