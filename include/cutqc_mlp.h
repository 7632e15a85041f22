/* cutqc_mlp.h -- cut-scoring MLP kernels of libcutqc.
 *
 * The paper has no learned component.  This network (64 -> 256 -> 256 -> 1,
 * ReLU, mean squared error) predicts the log2 reconstruction cost of a
 * candidate wire cut from 64 structural features, so that many candidate
 * cuts can be ranked in one batched launch before the exact cost model
 * checks the best of them.
 *
 * Parameters (device): one flat FP32 array of cutqc_mlp_param_count floats,
 * [W1 (64 x 256) | b1 (256) | W2 (256 x 256) | b2 (256) | W3 (256 x 1) | b3],
 * W_l stored [in][out], plus a BF16 copy of the same layout that the forward
 * and backward passes read (refresh it with cutqc_mlp_sync_bf16 after writing
 * the FP32 array; cutqc_mlp_adam keeps it in step).  Activations and all
 * accumulations are FP32.  x is [batch][64] FP32, y and t are [batch] FP32.
 * Workspace: cutqc_mlp_workspace_size(batch) bytes (activations).
 * All calls are asynchronous on `stream` and return CUTQC_* codes.            */
#ifndef CUTQC_MLP_H
#define CUTQC_MLP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int cutqc_mlp_param_count(int64_t* n);
int cutqc_mlp_workspace_size(int batch, size_t* bytes);
/* params_bf16[i] = bf16(params[i]) */
int cutqc_mlp_sync_bf16(const float* params_dev, void* params_bf16_dev, void* stream);
/* y = network(x) */
int cutqc_mlp_forward(const float* params_dev, const void* params_bf16_dev, const float* x_dev, int batch,
                      float* y_dev, void* ws_dev, size_t ws_bytes, void* stream);
/* grad = d/dparams of mean (y - t)^2 at the BF16 weights; loss_dev (nullable,
 * float64 scalar) = the loss */
int cutqc_mlp_gradients(const float* params_dev, const void* params_bf16_dev, const float* x_dev, const float* t_dev,
                        int batch, float* grad_dev, double* loss_dev, void* ws_dev, size_t ws_bytes, void* stream);
/* Adam with bias correction (step >= 1) on the FP32 parameters; refreshes the
 * BF16 copy */
int cutqc_mlp_adam(float* params_dev, void* params_bf16_dev, const float* grad_dev, float* m_dev, float* v_dev,
                   int step, float lr, float beta1, float beta2, float eps, void* stream);
/* gradients + Adam (beta1 0.9, beta2 0.999, eps 1e-8) */
int cutqc_mlp_train_step(float* params_dev, void* params_bf16_dev, float* grad_dev, float* m_dev, float* v_dev,
                         int step, float lr, const float* x_dev, const float* t_dev, int batch, double* loss_dev,
                         void* ws_dev, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CUTQC_MLP_H */
