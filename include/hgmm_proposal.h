/* Learned pose proposal for HGMM registration: C ABI.
 *
 * The paper registers from the identity and widens the basin of
 * convergence with its adaptive tree descent (Sec. 4, Algorithm 1).  This
 * part has no counterpart in the paper: a 3-layer perceptron reads the 64
 * level-1 GMM nodes (the paper's second level of 8-component GMMs, Sec. 3)
 * of both clouds and proposes an initial pose, which the plain method then
 * refines (hgmm_register / hgmm_batch_register), with the plain method from
 * the identity kept as the fallback: hgmm_pose_select keeps whichever of the
 * two refinements ends with the lower Eq. 11 objective.
 *
 * Canonical frame of a cloud (16 float64, "frame record"): c (3) = root
 * mean, s = sqrt(trace Sigma_root), V (9, row-major; columns = axes) = the
 * root eigenvectors the build used to seed level 0, third axis negated if
 * det V < 0, then flipped (1.0 if it was), 0, 0.
 *
 * Features of a cloud (640 BF16, stored as uint16): 64 nodes x 10 values,
 * node entry [64 pi_parent pi_child, V^T (mu - c) / s, 16 upper(V^T Sigma
 * V) / s^2] (upper = xx xy xz yy yz zz).  Level-0 node k fills group
 * k ^ (4 if flipped) (8 slots); its live children follow in order of
 * decreasing weight (ties by index); a live level-0 node whose children all
 * died fills the group's first slot itself; empty slots are zero.
 *
 * Network input of a pair (1280 BF16): [features(source), features(target)].
 * Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3,
 * 1280 -> 256 -> 256 -> 9, BF16 weights and activations on the tensor cores
 * (tcgen05, FP32 accumulation), FP32 master parameters and Adam state.
 * Output y (9 float32): y[0:3], y[3:6] = two columns whose Gram-Schmidt
 * orthonormalisation gives R', y[6:9] = t', in canonical coordinates:
 * x~_t = R' x~_s + t' with x~ = V^T (x - c) / s per cloud.  Hence
 * R = V_t R' V_s^T and t = c_t + s_t V_t t' - R c_s (pose source -> target).
 * Label of a pair (12 float32): R' row-major, t'.
 * Loss: mean over the batch of ||GS(y) - R'||_F^2 + w_t ||y_t - t'||^2.
 *
 * Flat parameter vector (HGMM_MLP_PARAMS float32): W1 (256 x 1280,
 * row-major), b1 (256), W2 (256 x 256), b2 (256), W3 (9 x 256), b3 (9).
 *
 * All device pointers belong to the caller unless stated; calls are
 * enqueued on `stream` (a cudaStream_t, NULL = legacy default stream) and
 * are graph-capturable unless marked synchronous.  Return values are the
 * HGMM_* codes of hgmm.h.
 */
#ifndef HGMM_PROPOSAL_H
#define HGMM_PROPOSAL_H

#include <stdint.h>

#include "hgmm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define HGMM_MLP_IN 1280
#define HGMM_MLP_HIDDEN 256
#define HGMM_MLP_OUT 9
#define HGMM_MLP_PARAMS 396041
#define HGMM_FEAT_PER_CLOUD 640
#define HGMM_FRAME_DOUBLES 16
#define HGMM_LABEL_FLOATS 12

typedef struct hgmm_mlp hgmm_mlp;

/* Network with room for batches of up to max_batch pairs (1..65536), on the
 * current device; parameters zero until hgmm_mlp_set_params. */
int hgmm_mlp_create(int32_t max_batch, hgmm_mlp** out);
void hgmm_mlp_destroy(hgmm_mlp* m);

/* Copy FP32 master parameters from the host (count must equal
 * HGMM_MLP_PARAMS), refresh the BF16 weight copies and reset the Adam
 * moments and step count.  Synchronous. */
int hgmm_mlp_set_params(hgmm_mlp* m, const float* h_params, int64_t count);
/* Copy the FP32 master parameters (resp. the gradients of the last
 * hgmm_mlp_gradients / hgmm_mlp_train_step) to the host.  Synchronous. */
int hgmm_mlp_get_params(hgmm_mlp* m, float* h_params, int64_t count);
int hgmm_mlp_read_grads(hgmm_mlp* m, float* h_grads, int64_t count);

/* y = network(x) for `batch` pairs: d_x batch x 1280 BF16 (16-byte aligned,
 * device), d_y batch x 9 float32 (device).  Errors: HGMM_EINVAL (batch not
 * in [1, max_batch], unaligned x), HGMM_ECUDA. */
int hgmm_mlp_forward(hgmm_mlp* m, const uint16_t* d_x, int32_t batch, float* d_y, void* stream);

/* Loss and gradients of the FP32 master parameters for one batch: rows
 * d_index[0..batch) of d_x / d_labels (n_rows rows each, device), or rows
 * 0..batch-1 when d_index is NULL.  The mean loss goes to d_loss (1 float32,
 * device) if not NULL.  An index outside [0, n_rows) is reported by
 * hgmm_mlp_sync as HGMM_EINVAL (its row counts as zero). */
int hgmm_mlp_gradients(hgmm_mlp* m, const uint16_t* d_x, const float* d_labels,
                       const int32_t* d_index, int32_t batch, int32_t n_rows, float w_t,
                       float* d_loss, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) of every
 * parameter from the current gradients, then refresh the BF16 weights. */
int hgmm_mlp_adam(hgmm_mlp* m, float lr, void* stream);

/* hgmm_mlp_gradients followed by hgmm_mlp_adam. */
int hgmm_mlp_train_step(hgmm_mlp* m, const uint16_t* d_x, const float* d_labels,
                        const int32_t* d_index, int32_t batch, int32_t n_rows, float w_t,
                        float lr, float* d_loss, void* stream);

/* Synchronise `stream` and return the first error the network's kernels
 * recorded since the last call (HGMM_ETIMEOUT: a tensor-core completion
 * wait ran out; HGMM_EINVAL: a bad batch index), clearing it. */
int hgmm_mlp_sync(hgmm_mlp* m, void* stream);

/* Features (640 BF16 at d_feat, 16-byte aligned) and frame record (16
 * float64 at d_frame) of the cloud of the tree's last build (depth >= 2). */
int hgmm_tree_features(hgmm_tree* t, uint16_t* d_feat, double* d_frame, void* stream);

/* Features of every planned pair's TARGET cloud in one persistent launch:
 * builds each target's tree (the plan's depths, all >= 2) and writes pair
 * i's features to d_feat + 640 i and its frame to d_frame + 16 i; no
 * registration runs.  Planning the source and target of pair j as entries
 * 2j and 2j+1 makes d_feat the network input (n x 1280) and d_frame the
 * per-pair frames (n x 32, source frame first) of hgmm_pose_decode. */
int hgmm_batch_features(hgmm_batch* b, const float* d_points, const hgmm_params* p,
                        uint16_t* d_feat, double* d_frame, void* stream);

/* The network's proposal for one pair in a single call: the features and
 * frames of the source tree `src` and the target tree `tgt` (each as
 * hgmm_tree_features gives them, depth >= 2), the forward pass and the
 * decode, i.e. d_T_out (16 float64, device, caller-owned) = the pose that
 * maps the source cloud into the target's frame, ready to start
 * hgmm_register on `tgt`.  Uses buffers of the network handle, so calls on
 * one handle must not overlap.  Enqueued on `stream`; graph-capturable.
 * Errors: HGMM_EINVAL (a NULL argument, a tree not built or of depth < 2),
 * HGMM_ECUDA. */
int hgmm_propose(hgmm_tree* tgt, hgmm_tree* src, hgmm_mlp* m, void* stream, double* d_T_out);

/* Poses (n x 16 float64, row-major 4x4) from network outputs (n x 9) and
 * the per-pair frames (n x 32: source frame, target frame). */
int hgmm_pose_decode(const float* d_y, const double* d_frames, int32_t n, double* d_T, void* stream);

/* Labels (n x 12 float32) of poses (n x 16 float64) in the per-pair frames. */
int hgmm_pose_encode(const double* d_T, const double* d_frames, int32_t n, float* d_labels,
                     void* stream);

/* Per pair: the pose whose objective is lower (a non-finite objective loses;
 * ties keep a) to d_T_out (n x 16), which one (0 = a, 1 = b) to d_choice and
 * its objective to d_obj_out, each if not NULL (d_T_out and d_obj_out may be
 * d_T_a and d_obj_a, so candidates can be folded in one by one). */
int hgmm_pose_select(int32_t n, const double* d_T_a, const double* d_obj_a, const double* d_T_b,
                     const double* d_obj_b, double* d_T_out, int32_t* d_choice, double* d_obj_out,
                     void* stream);

/* d_out[i] = d_A[i] d_B[i] for n pairs of 4x4 FP64 row-major poses (device,
 * n x 16 each; d_out may alias neither input). */
int hgmm_pose_compose(int32_t n, const double* d_A, const double* d_B, double* d_out, void* stream);

/* Checking entry point for the tensor-core GEMM the network runs on:
 * d_out[m * N + n] = sum_k A[m][k] B[n][k] (float32, device) with BF16
 * operands A[m][k] = d_A[m * a_m + k * a_k], B[n][k] = d_B[n * b_n + k * b_k]
 * (element strides; for each operand either the k stride or the row stride
 * is 1, the other a multiple of 8; a K stride of 1 needs K % 8 == 0, a row
 * stride of 1 needs the row count % 8 == 0; 16-byte aligned bases).  N <= 16
 * runs 128 x 16 tiles, larger N 128 x 256 tiles.  Errors: HGMM_EINVAL. */
int hgmm_debug_gemm(const uint16_t* d_A, int64_t a_m, int64_t a_k, const uint16_t* d_B, int64_t b_n,
                    int64_t b_k, int32_t M, int32_t N, int32_t K, float* d_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HGMM_PROPOSAL_H */
