/* dpdlp_gnn.h -- C ABI of the learned warm start for families of LPs that share A.
 *
 * A bipartite message-passing network over the variable-constraint graph of A predicts a
 * start point (x, y) for the PDHG solver (pass it to dpdlp_set_start).  The paper itself
 * starts from zero (its algorithm takes any start point, Algorithm 1); the network is an
 * addition, trained on solutions of the plain solver, and cold PDHG from zero stays the
 * fallback.
 *
 * Network (H = 64 hidden units, F = 8 input features, L = 4 rounds):
 *   aggregation   R = diag(1 / max(1, sum_j |a_ij|)) A          (m x n, row means)
 *                 C = diag(1 / max(1, sum_i |a_ij|)) A^T        (n x m, column means)
 *   encoders      hv = relu(Fv Ev^T + ev)   (n x H),   hc = relu(Fc Ec^T + ec)   (m x H)
 *   round l       gc = R hv,  hc = relu(hc Uc_l^T + gc Vc_l^T + bc_l)
 *                 gv = C hc,  hv = relu(hv Uv_l^T + gv Vv_l^T + bv_l)
 *   heads         x_hat = hv wx + bx (n),   y_hat = hc wy + by (m)
 *   loss          mean_j (x_hat_j - tx_j)^2 + mean_i (y_hat_i - ty_i)^2
 * Weights (Ev, Ec, Uc, Vc, Uv, Vv, wx, wy) are used in BF16, biases in FP32; activations,
 * products and sums are FP32.  The master parameters are an FP32 vector in the order
 *   Ev[H][F], ev[H], Ec[H][F], ec[H],
 *   for l = 0..L-1: Uc[H][H], Vc[H][H], bc[H], Uv[H][H], Vv[H][H], bv[H],
 *   wx[H], bx, wy[H], by
 * (dpdlp_gnn_param_count() entries); the BF16 copies are refreshed from it by
 * dpdlp_gnn_set_params and dpdlp_gnn_adam.  Every reduction runs in a fixed order: results
 * are bitwise reproducible.
 *
 * Conventions: return 0 on success, < 0 on error (DPDLP_ERR_* of dpdlp.h), after which
 * dpdlp_gnn_last_error describes it.  Array arguments are HOST pointers unless
 * dpdlp_gnn_set_ptr_mode(g, 1) made the feature, target and output arrays DEVICE pointers
 * (on the handle's device).  Inputs are copied; the caller keeps its buffers.
 */
#ifndef DPDLP_GNN_H
#define DPDLP_GNN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DPDLP_GNN_HIDDEN 64
#define DPDLP_GNN_FEATURES 8
#define DPDLP_GNN_ROUNDS 4

typedef struct dpdlp_gnn dpdlp_gnn_t;

/* Number of FP32 master parameters. */
int64_t dpdlp_gnn_param_count(void);

/* Create a network on CUDA device `device` (parameters zero until set). */
int dpdlp_gnn_create(dpdlp_gnn_t** out, int device);
void dpdlp_gnn_destroy(dpdlp_gnn_t* g);
const char* dpdlp_gnn_last_error(const dpdlp_gnn_t* g);

/* 0: host arrays (default); 1: device arrays for features, targets and outputs. */
int dpdlp_gnn_set_ptr_mode(dpdlp_gnn_t* g, int device);

/* Master parameters (FP32, `count` = dpdlp_gnn_param_count()), HOST arrays always.
 * Setting them also resets the Adam moments. */
int dpdlp_gnn_set_params(dpdlp_gnn_t* g, const float* params, int64_t count);
int dpdlp_gnn_get_params(dpdlp_gnn_t* g, float* params, int64_t count);
/* Accumulated gradient of the loss (FP32), HOST array. */
int dpdlp_gnn_get_grads(dpdlp_gnn_t* g, float* grads, int64_t count);
int dpdlp_gnn_zero_grads(dpdlp_gnn_t* g);

/* The graph: A in CSR (m rows, n columns, HOST arrays, the layout of dpdlp_load_lp);
 * values may be any finite numbers.  Builds R and C (and their transposes for the
 * backward pass) on the device and sizes the activation buffers. */
int dpdlp_gnn_set_graph(dpdlp_gnn_t* g, int32_t n, int32_t m, const int64_t* row_ptr,
                        const int32_t* col_idx, const double* val);

/* Input features Fv[n][F] and Fc[m][F] (row-major FP32). */
int dpdlp_gnn_set_features(dpdlp_gnn_t* g, const float* fv, const float* fc);

/* Forward pass; writes x_hat[n] and y_hat[m] (FP32) when the pointers are not NULL. */
int dpdlp_gnn_forward(dpdlp_gnn_t* g, float* x_hat, float* y_hat);

/* After dpdlp_gnn_forward: loss against the targets tx[n], ty[m] (FP32) into *loss (may be
 * NULL) and its gradient added to the accumulated gradient. */
int dpdlp_gnn_backward(dpdlp_gnn_t* g, const float* tx, const float* ty, double* loss);

/* One Adam step on the master parameters with the accumulated gradient (step = 1, 2, ...
 * for the bias correction), then refresh the BF16 copies and zero the gradient. */
int dpdlp_gnn_adam(dpdlp_gnn_t* g, double lr, double beta1, double beta2, double eps,
                   int64_t step);

/* One whole training step on one instance: set the features fv[n][F], fc[m][F], forward pass,
 * loss and gradient against the targets tx[n], ty[m], one Adam step -- the same kernels in the
 * same order as dpdlp_gnn_set_features, dpdlp_gnn_forward, dpdlp_gnn_backward and
 * dpdlp_gnn_adam, so the parameters come out bitwise the same -- as one replay of a CUDA graph
 * captured at the first call after dpdlp_gnn_set_graph (arrays host or device per the pointer
 * mode).  *loss (may be NULL: then the call only enqueues the step and returns without waiting
 * for it) receives the step's loss.  Errors as the individual calls. */
int dpdlp_gnn_train_step(dpdlp_gnn_t* g, const float* fv, const float* fc, const float* tx,
                         const float* ty, double lr, double beta1, double beta2, double eps,
                         int64_t step, double* loss);

#ifdef __cplusplus
}
#endif

#endif /* DPDLP_GNN_H */
