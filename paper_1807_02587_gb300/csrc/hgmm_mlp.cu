// Learned pose proposal: the network's forward and backward passes on the
// tensor cores (hgmm_tc.cuh), its loss through the 6-D rotation
// representation, Adam, the canonical-frame features of a tree, and the
// pose encode / decode / fallback-select kernels.
//
// Forward (x: batch x 1280 BF16):
//   H1 = relu(x W1^T + b1)      tcgen05, N = 256, K = 1280, bias+ReLU epilogue -> BF16
//   H2 = relu(H1 W2^T + b2)     tcgen05, N = 256, K = 256
//   Y  = H2 W3^T + b3           tcgen05, N = 16 (rows 9..15 of W3 are zero), FP32 out
// Backward (dY from the loss kernel, BF16 for the tensor cores, FP32 kept):
//   dW3^T = H2^T dY             M = 256 hidden, N = 16, K = batch (both read transposed)
//   dZ2 = (dY W3) * [H2 > 0]    N = 256, K = 16, mask epilogue -> BF16
//   dW2 = dZ2^T H1              M = 256, N = 256, K = batch
//   dZ1 = (dZ2 W2) * [H1 > 0]
//   dW1 = dZ1^T x               M = 256, N = 1280, K = batch
//   db = column sums of dZ1, dZ2, dY (two-pass, fixed order: deterministic)
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <mutex>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/hgmm_proposal.h"
#include "hgmm_feat.cuh"
#include "hgmm_internal.cuh"
#include "hgmm_tc.cuh"

namespace hgmm {
namespace {

constexpr int IN = HGMM_MLP_IN, HID = HGMM_MLP_HIDDEN, OUT = HGMM_MLP_OUT, OUTP = 16;
constexpr int64_t OFF_W1 = 0;
constexpr int64_t OFF_B1 = OFF_W1 + int64_t(HID) * IN;
constexpr int64_t OFF_W2 = OFF_B1 + HID;
constexpr int64_t OFF_B2 = OFF_W2 + int64_t(HID) * HID;
constexpr int64_t OFF_W3 = OFF_B2 + HID;
constexpr int64_t OFF_B3 = OFF_W3 + int64_t(OUT) * HID;
constexpr int64_t N_PARAMS = OFF_B3 + OUT;
static_assert(N_PARAMS == HGMM_MLP_PARAMS, "parameter layout");
static_assert(FEAT_PER_CLOUD == HGMM_FEAT_PER_CLOUD && FRAME_DOUBLES == HGMM_FRAME_DOUBLES, "layout");

constexpr int ERR_TIMEOUT = 1;
constexpr int ERR_INDEX = 2;
constexpr int COLSUM_ROWS = 64;  // rows per partial column sum

using bf16 = __nv_bfloat16;

__global__ void k_tree_features(const RootDev* root, const NodeStat* stat, bf16* feat, double* frame) {
    __shared__ double fsm[FRAME_DOUBLES];
    tree_features_warp(root, stat, feat, frame, fsm);
}

// Rows idx[r] of x and labels -> row r of the gathered batch.
__global__ void k_gather(const bf16* __restrict__ X, const float* __restrict__ L,
                         const int* __restrict__ idx, int n_rows, bf16* __restrict__ Xo,
                         float* __restrict__ Lo, int* __restrict__ err) {
    const int r = blockIdx.x;
    const int src = idx[r];
    const bool good = src >= 0 && src < n_rows;
    if (!good && threadIdx.x == 0) atomicOr(err, ERR_INDEX);
    const uint4* xs = reinterpret_cast<const uint4*>(X + int64_t(good ? src : 0) * IN);
    uint4* xd = reinterpret_cast<uint4*>(Xo + int64_t(r) * IN);
    for (int i = threadIdx.x; i < IN / 8; i += blockDim.x)
        xd[i] = good ? __ldg(xs + i) : make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x < HGMM_LABEL_FLOATS)
        Lo[int64_t(r) * HGMM_LABEL_FLOATS + threadIdx.x] =
            good ? L[int64_t(src) * HGMM_LABEL_FLOATS + threadIdx.x] : 0.f;
}

__device__ __forceinline__ void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Gram-Schmidt of (a1, a2) into the columns b1, b2, b3 = b1 x b2.
__device__ __forceinline__ void gram_schmidt(const double* a1, const double* a2, double* b1,
                                             double* b2, double* b3, double* n1, double* dd,
                                             double* n2) {
    *n1 = sqrt(dot3(a1, a1));
    const double i1 = *n1 > 0.0 ? 1.0 / *n1 : 0.0;
    for (int i = 0; i < 3; ++i) b1[i] = a1[i] * i1;
    *dd = dot3(b1, a2);
    double u[3];
    for (int i = 0; i < 3; ++i) u[i] = a2[i] - *dd * b1[i];
    *n2 = sqrt(dot3(u, u));
    const double i2 = *n2 > 0.0 ? 1.0 / *n2 : 0.0;
    for (int i = 0; i < 3; ++i) b2[i] = u[i] * i2;
    cross3(b1, b2, b3);
}

// Loss of every row and dL/dy (mean over the batch); one CTA of 256
// threads, fixed-order block reduction of the loss.
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ Y, const float* __restrict__ L,
                                              int batch, float w_t, bf16* __restrict__ dY,
                                              float* __restrict__ dYf, float* __restrict__ loss) {
    __shared__ double red[256];
    double acc = 0.0;
    const double inv_b = 1.0 / double(batch);
    for (int r = threadIdx.x; r < batch; r += blockDim.x) {
        const float* y = Y + int64_t(r) * OUT;
        const float* l = L + int64_t(r) * HGMM_LABEL_FLOATS;
        double a1[3], a2[3], b1[3], b2[3], b3[3], n1, dd, n2;
        for (int i = 0; i < 3; ++i) {
            a1[i] = y[i];
            a2[i] = y[3 + i];
        }
        gram_schmidt(a1, a2, b1, b2, b3, &n1, &dd, &n2);
        double G1[3], G2[3], G3[3], e = 0.0;
        for (int i = 0; i < 3; ++i) {
            // label R' row-major: column k entry i at l[3 i + k]
            const double r0 = b1[i] - l[3 * i + 0], r1 = b2[i] - l[3 * i + 1], r2 = b3[i] - l[3 * i + 2];
            e += r0 * r0 + r1 * r1 + r2 * r2;
            G1[i] = 2.0 * r0;
            G2[i] = 2.0 * r1;
            G3[i] = 2.0 * r2;
        }
        double gt[3];
        for (int i = 0; i < 3; ++i) {
            const double d = double(y[6 + i]) - l[9 + i];
            e += double(w_t) * d * d;
            gt[i] = 2.0 * double(w_t) * d;
        }
        acc += e;
        // back through b3 = b1 x b2, b2 = u / |u|, u = a2 - (b1.a2) b1, b1 = a1 / |a1|
        double gb1[3], gb2[3], c[3];
        cross3(b2, G3, c);
        for (int i = 0; i < 3; ++i) gb1[i] = G1[i] + c[i];
        cross3(G3, b1, c);
        for (int i = 0; i < 3; ++i) gb2[i] = G2[i] + c[i];
        const double i2 = n2 > 0.0 ? 1.0 / n2 : 0.0, i1 = n1 > 0.0 ? 1.0 / n1 : 0.0;
        const double p2 = dot3(gb2, b2);
        double gu[3];
        for (int i = 0; i < 3; ++i) gu[i] = (gb2[i] - p2 * b2[i]) * i2;
        const double q = dot3(gu, b1);
        double ga2[3];
        for (int i = 0; i < 3; ++i) {
            ga2[i] = gu[i] - q * b1[i];
            gb1[i] += -q * a2[i] - dd * gu[i];
        }
        const double p1 = dot3(gb1, b1);
        double g[OUTP];
        for (int i = 0; i < 3; ++i) {
            g[i] = (gb1[i] - p1 * b1[i]) * i1 * inv_b;
            g[3 + i] = ga2[i] * inv_b;
            g[6 + i] = gt[i] * inv_b;
        }
        for (int i = OUT; i < OUTP; ++i) g[i] = 0.0;
        for (int i = 0; i < OUTP; ++i) {
            dYf[int64_t(r) * OUTP + i] = float(g[i]);
            dY[int64_t(r) * OUTP + i] = __double2bfloat16(g[i]);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = float(red[0] * inv_b);
}

// Column sums for the bias gradients, pass 1: block (chunk, matrix) sums
// COLSUM_ROWS rows of one column per thread.  matrix 0: dZ1, 1: dZ2 (BF16,
// 256 columns), 2: dY (FP32, 16 columns).
__global__ void __launch_bounds__(256) k_colsum_partial(const bf16* __restrict__ dZ1,
                                                        const bf16* __restrict__ dZ2,
                                                        const float* __restrict__ dYf, int batch,
                                                        float* __restrict__ part) {
    const int chunk = blockIdx.x, mat = blockIdx.y, j = threadIdx.x;
    const int r0 = chunk * COLSUM_ROWS, r1 = min(batch, r0 + COLSUM_ROWS);
    float s = 0.f;
    if (mat < 2) {
        const bf16* Z = mat == 0 ? dZ1 : dZ2;
        for (int r = r0; r < r1; ++r) s += __bfloat162float(Z[int64_t(r) * HID + j]);
    } else if (j < OUTP) {
        for (int r = r0; r < r1; ++r) s += dYf[int64_t(r) * OUTP + j];
    }
    part[(int64_t(chunk) * 3 + mat) * HID + j] = s;
}

// pass 2: fixed-order sum over the chunks into the bias gradients.
__global__ void __launch_bounds__(256) k_colsum_final(const float* __restrict__ part, int nchunks,
                                                      float* __restrict__ grads) {
    const int mat = blockIdx.x, j = threadIdx.x;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += part[(int64_t(c) * 3 + mat) * HID + j];
    if (mat == 0) grads[OFF_B1 + j] = float(s);
    else if (mat == 1) grads[OFF_B2 + j] = float(s);
    else if (j < OUT) grads[OFF_B3 + j] = float(s);
}

// BF16 copies of the weights the tensor cores read; W3 padded to 16 rows.
__device__ __forceinline__ void store_bf16_copy(int64_t i, float p, bf16* W1, bf16* W2, bf16* W3,
                                                float* b3p) {
    if (i < OFF_B1) W1[i - OFF_W1] = __float2bfloat16_rn(p);
    else if (i >= OFF_W2 && i < OFF_B2) W2[i - OFF_W2] = __float2bfloat16_rn(p);
    else if (i >= OFF_W3 && i < OFF_B3) W3[i - OFF_W3] = __float2bfloat16_rn(p);
    else if (i >= OFF_B3) b3p[i - OFF_B3] = p;
}

__global__ void k_refresh(const float* __restrict__ P, bf16* W1, bf16* W2, bf16* W3, float* b3p) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N_PARAMS;
         i += int64_t(gridDim.x) * blockDim.x)
        store_bf16_copy(i, P[i], W1, W2, W3, b3p);
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ Mo,
                       float* __restrict__ Vo, float lr, float c1, float c2, bf16* W1, bf16* W2,
                       bf16* W3, float* b3p) {
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N_PARAMS;
         i += int64_t(gridDim.x) * blockDim.x) {
        const float g = G[i];
        const float m = beta1 * Mo[i] + (1.f - beta1) * g;
        const float v = beta2 * Vo[i] + (1.f - beta2) * g * g;
        Mo[i] = m;
        Vo[i] = v;
        const float p = P[i] - lr * (m * c1) / (sqrtf(v * c2) + eps);
        P[i] = p;
        store_bf16_copy(i, p, W1, W2, W3, b3p);
    }
}

__device__ __forceinline__ void load_frame(const double* f, double* c, double& s, double* V) {
    for (int a = 0; a < 3; ++a) c[a] = f[a];
    s = f[3];
    for (int v = 0; v < 9; ++v) V[v] = f[4 + v];
}

__global__ void k_decode(const float* __restrict__ Y, const double* __restrict__ F, int n,
                         double* __restrict__ T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double cs[3], ct[3], Vs[9], Vt[9], ss, st;
    load_frame(F + 32 * int64_t(i), cs, ss, Vs);
    load_frame(F + 32 * int64_t(i) + 16, ct, st, Vt);
    const float* y = Y + int64_t(i) * OUT;
    double a1[3], a2[3], b[3][3], n1, dd, n2;
    for (int k = 0; k < 3; ++k) {
        a1[k] = y[k];
        a2[k] = y[3 + k];
    }
    gram_schmidt(a1, a2, b[0], b[1], b[2], &n1, &dd, &n2);
    // R' (columns b[0..2]); A = Vt R', R = A Vs^T
    double A[3][3], R[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) A[r][c] = Vt[3 * r] * b[c][0] + Vt[3 * r + 1] * b[c][1] + Vt[3 * r + 2] * b[c][2];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) R[r][c] = A[r][0] * Vs[3 * c] + A[r][1] * Vs[3 * c + 1] + A[r][2] * Vs[3 * c + 2];
    double* o = T + 16 * int64_t(i);
    for (int r = 0; r < 3; ++r) {
        const double vt = Vt[3 * r] * y[6] + Vt[3 * r + 1] * y[7] + Vt[3 * r + 2] * y[8];
        const double rc = R[r][0] * cs[0] + R[r][1] * cs[1] + R[r][2] * cs[2];
        for (int c = 0; c < 3; ++c) o[4 * r + c] = R[r][c];
        o[4 * r + 3] = ct[r] + st * vt - rc;
    }
    o[12] = 0.0;
    o[13] = 0.0;
    o[14] = 0.0;
    o[15] = 1.0;
}

__global__ void k_encode(const double* __restrict__ T, const double* __restrict__ F, int n,
                         float* __restrict__ L) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double cs[3], ct[3], Vs[9], Vt[9], ss, st;
    load_frame(F + 32 * int64_t(i), cs, ss, Vs);
    load_frame(F + 32 * int64_t(i) + 16, ct, st, Vt);
    const double* p = T + 16 * int64_t(i);
    double RVs[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            RVs[r][c] = p[4 * r] * Vs[c] + p[4 * r + 1] * Vs[3 + c] + p[4 * r + 2] * Vs[6 + c];
    float* l = L + int64_t(i) * HGMM_LABEL_FLOATS;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            l[3 * r + c] = float(Vt[r] * RVs[0][c] + Vt[3 + r] * RVs[1][c] + Vt[6 + r] * RVs[2][c]);
    double d[3];
    for (int r = 0; r < 3; ++r)
        d[r] = p[4 * r] * cs[0] + p[4 * r + 1] * cs[1] + p[4 * r + 2] * cs[2] + p[4 * r + 3] - ct[r];
    for (int a = 0; a < 3; ++a) l[9 + a] = float((Vt[a] * d[0] + Vt[3 + a] * d[1] + Vt[6 + a] * d[2]) / st);
}

// One thread per pair; inputs and outputs may alias (T_out = T_a, obj_out
// = obj_a): every value is read before it is written.
__global__ void k_select(int n, const double* Ta, const double* oa, const double* Tb, const double* ob,
                         double* To, int* __restrict__ choice, double* oo) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = oa[i], b = ob[i];
    const bool take_b = isfinite(b) && (!isfinite(a) || b < a);
    const double* src = (take_b ? Tb : Ta) + 16 * int64_t(i);
    double v[16];
    for (int k = 0; k < 16; ++k) v[k] = src[k];
    for (int k = 0; k < 16; ++k) To[16 * int64_t(i) + k] = v[k];
    if (choice) choice[i] = take_b ? 1 : 0;
    if (oo) oo[i] = take_b ? b : a;
}

__global__ void k_compose(int n, const double* __restrict__ A, const double* __restrict__ Bm,
                          double* __restrict__ O) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* a = A + 16 * int64_t(i);
    const double* b = Bm + 16 * int64_t(i);
    double* o = O + 16 * int64_t(i);
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c)
            o[4 * r + c] = a[4 * r] * b[c] + a[4 * r + 1] * b[4 + c] + a[4 * r + 2] * b[8 + c] + a[4 * r + 3] * b[12 + c];
}


// ---------------------------------------------------------------------------
// The whole forward pass of one 128-row block in one launch (warp-specialised
// tcgen05 with TMEM accumulators and TMA operand streams):
//   layer 1: acc1 (TMEM columns 0..255) = X[128 x 1280] W1^T, 20 K-steps of
//            TMA-fed 128 x 64 / 256 x 64 tiles in a 4-stage ring;
//   epilogue warps: h1 = relu(acc1 + b1) as BF16 to H1 (global, for the
//            backward pass; skipped when H1 is null) and into shared memory
//            in the 128-byte-swizzled K-major layout that TMA would write,
//            as layer 2's A operand;
//   layer 2: acc2 (columns 256..511) = h1 W2^T, W2 tiles streamed by TMA;
//   epilogue: h2 likewise (H2 if not null, and shared memory over h1);
//   layer 3: acc3 (columns 0..15) = h2 W3^T (W3 padded to 16 rows);
//   epilogue: Y = acc3 + b3 (9 columns, FP32).
// Warps 0-3 are the epilogue (warp w owns TMEM lanes 32w..32w+31, i.e.
// rows), one thread of warp 4 issues the TMA loads, one thread of warp 5
// the MMAs.  Every wait is bounded; on a timeout the kernel records the
// error, lets every role run out (commits and arrivals still happen) and
// drains its loads in flight before it frees TMEM.
constexpr int FW_THREADS = 192;
constexpr int FW_S1 = 4;                          // layer-1 stages
constexpr int FW_A = 128 * 128;                   // 128 rows x 64 BF16
constexpr int FW_B = 256 * 128;                   // 256 rows x 64 BF16
constexpr int FW_STAGE1 = FW_A + FW_B;            // 48 KB
constexpr int FW_H = 4 * FW_A;                    // 128 x 256 BF16: four 64-wide K chunks (64 KB)
constexpr int FW_W2_OFF = FW_H;                   // two 32 KB W2 stages after the h buffer
constexpr int FW_W3_OFF = FW_W2_OFF + 2 * FW_B;   // four 16 x 64 W3 tiles (8 KB)
constexpr int FW_W3_TILE = 16 * 128;
constexpr int FW_SMEM = FW_S1 * FW_STAGE1 + 1024; // the h buffer and W2/W3 reuse the layer-1 ring
static_assert(FW_W3_OFF + 4 * FW_W3_TILE <= FW_S1 * FW_STAGE1, "layer 2/3 buffers inside the ring");

// Row r's 16-byte unit u of a 64-wide K chunk in the 128-byte swizzled layout.
__device__ __forceinline__ uint32_t sw128_offset(int r, int u) {
    return uint32_t(r * 128 + ((u ^ (r & 7)) << 4));
}

// Epilogue of one hidden layer: relu(acc + bias) for this thread's row (all
// 256 columns) to the global row (16-byte stores, if grow is not null) and
// to the shared h buffer.
__device__ __forceinline__ void fw_hidden_epilogue(uint32_t tacc, const float* __restrict__ bias,
                                                   bf16* __restrict__ grow, uint32_t hbuf, int r) {
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
        float v[64];
        tc::tmem_ld64(tacc + uint32_t(c * 64), v);
        const float4* b4 = reinterpret_cast<const float4*>(bias + c * 64);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float4 ba = __ldg(b4 + 2 * u), bb = __ldg(b4 + 2 * u + 1);
            const float x[8] = {v[8 * u] + ba.x, v[8 * u + 1] + ba.y, v[8 * u + 2] + ba.z, v[8 * u + 3] + ba.w,
                                v[8 * u + 4] + bb.x, v[8 * u + 5] + bb.y, v[8 * u + 6] + bb.z, v[8 * u + 7] + bb.w};
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const __nv_bfloat162 p2 = __floats2bfloat162_rn(fmaxf(x[2 * h], 0.f), fmaxf(x[2 * h + 1], 0.f));
                w[h] = *reinterpret_cast<const uint32_t*>(&p2);
            }
            if (grow) reinterpret_cast<uint4*>(grow + c * 64)[u] = make_uint4(w[0], w[1], w[2], w[3]);
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                         :: "r"(hbuf + uint32_t(c * FW_A) + sw128_offset(r, u)), "r"(w[0]), "r"(w[1]), "r"(w[2]),
                            "r"(w[3]) : "memory");
        }
    }
}

__device__ __forceinline__ bool fw_wait(uint64_t* bar, uint32_t parity, int* fail) {
    if (*(volatile int*)fail) return false;
    if (tc::mbar_wait_bounded(bar, parity, tc::MBAR_SPIN_LIMIT)) return true;
    atomicExch(fail, 1);
    return false;
}

__global__ void __launch_bounds__(FW_THREADS, 1)
k_mlp_forward(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
              const __grid_constant__ CUtensorMap tmW2, const __grid_constant__ CUtensorMap tmW3,
              const float* __restrict__ b1, const float* __restrict__ b2, const float* __restrict__ b3p,
              bf16* __restrict__ H1, bf16* __restrict__ H2, float* __restrict__ Y, int batch,
              int* __restrict__ err) {
    extern __shared__ unsigned char fw_raw[];
    __shared__ __align__(8) uint64_t full1[FW_S1], empty1[FW_S1], full2[2], empty2[2];
    __shared__ __align__(8) uint64_t full3, done1, done2, done3, h1_ready, h2_ready;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    const uint32_t base = (tc::smem_u32(fw_raw) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * 128;
    constexpr int NK1 = IN / 64, NK2 = HID / 64;
    constexpr uint32_t ID1 = tc::idesc_bf16_f32(128, HID), ID3 = tc::idesc_bf16_f32(128, OUTP);
    if (warp == 4) {
        tc::tmem_alloc(&tmem_slot, 512);
        tc::tmem_relinquish();
    }
    if (threadIdx.x == 160) {
        for (int i = 0; i < FW_S1; ++i) {
            tc::mbar_init(&full1[i], 1);
            tc::mbar_init(&empty1[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&full2[i], 1);
            tc::mbar_init(&empty2[i], 1);
        }
        tc::mbar_init(&full3, 1);
        tc::mbar_init(&done1, 1);
        tc::mbar_init(&done2, 1);
        tc::mbar_init(&done3, 1);
        tc::mbar_init(&h1_ready, 128);
        tc::mbar_init(&h2_ready, 128);
        fail = 0;
        tc::fence_mbar_init();
        tc::prefetch_tmap(&tmX);
        tc::prefetch_tmap(&tmW1);
        tc::prefetch_tmap(&tmW2);
        tc::prefetch_tmap(&tmW3);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t hbuf = base;
    int issued1 = 0, issued2 = 0;
    bool issued3 = false;
    if (threadIdx.x == 128) {
        // ---- producer
        for (int kt = 0; kt < NK1; ++kt) {
            const int st = kt % FW_S1;
            if (kt >= FW_S1 && !fw_wait(&empty1[st], ((kt / FW_S1) - 1) & 1, &fail)) break;
            const uint32_t sa = base + st * FW_STAGE1;
            tc::mbar_arrive_expect_tx(&full1[st], uint32_t(FW_STAGE1));
            tc::tma_load_2d(sa, &tmX, kt * 64, m0, &full1[st]);
            tc::tma_load_2d(sa + FW_A, &tmW1, kt * 64, 0, &full1[st]);
            issued1 = kt + 1;
        }
        // layer 2 and 3 operands go where the layer-1 ring was: after its MMAs
        if (issued1 == NK1 && fw_wait(&done1, 0, &fail)) {
            tc::mbar_arrive_expect_tx(&full3, uint32_t(4 * FW_W3_TILE));
            for (int kt = 0; kt < NK2; ++kt)
                tc::tma_load_2d(base + FW_W3_OFF + kt * FW_W3_TILE, &tmW3, kt * 64, 0, &full3);
            issued3 = true;
            for (int kt = 0; kt < NK2; ++kt) {
                const int st = kt & 1;
                if (kt >= 2 && !fw_wait(&empty2[st], ((kt >> 1) - 1) & 1, &fail)) break;
                tc::mbar_arrive_expect_tx(&full2[st], uint32_t(FW_B));
                tc::tma_load_2d(base + FW_W2_OFF + st * FW_B, &tmW2, kt * 64, 0, &full2[st]);
                issued2 = kt + 1;
            }
        }
    } else if (threadIdx.x == 160) {
        // ---- MMA issuer
        bool ok = true;
        for (int kt = 0; kt < NK1 && ok; ++kt) {
            const int st = kt % FW_S1;
            ok = fw_wait(&full1[st], (kt / FW_S1) & 1, &fail);
            if (!ok) break;
            tc::fence_after_sync();
            const uint32_t sa = base + st * FW_STAGE1;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc::mma_bf16(tmem, tc::smem_desc_sw128(sa + kk * 32), tc::smem_desc_sw128(sa + FW_A + kk * 32), ID1,
                             (kt | kk) != 0 ? 1u : 0u);
            tc::mma_commit(&empty1[st]);
        }
        tc::mma_commit(&done1);
        ok = ok && fw_wait(&h1_ready, 0, &fail);
        for (int kt = 0; kt < NK2 && ok; ++kt) {
            const int st = kt & 1;
            ok = fw_wait(&full2[st], (kt >> 1) & 1, &fail);
            if (!ok) break;
            tc::fence_after_sync();
            const uint32_t sb = base + FW_W2_OFF + st * FW_B;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc::mma_bf16(tmem + 256u, tc::smem_desc_sw128(hbuf + kt * FW_A + kk * 32),
                             tc::smem_desc_sw128(sb + kk * 32), ID1, (kt | kk) != 0 ? 1u : 0u);
            tc::mma_commit(&empty2[st]);
        }
        tc::mma_commit(&done2);
        ok = ok && fw_wait(&h2_ready, 0, &fail) && fw_wait(&full3, 0, &fail);
        if (ok) {
            tc::fence_after_sync();
            for (int kt = 0; kt < NK2; ++kt)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc::mma_bf16(tmem, tc::smem_desc_sw128(hbuf + kt * FW_A + kk * 32),
                                 tc::smem_desc_sw128(base + FW_W3_OFF + kt * FW_W3_TILE + kk * 32), ID3,
                                 (kt | kk) != 0 ? 1u : 0u);
        }
        tc::mma_commit(&done3);
    } else if (warp < 4) {
        // ---- epilogue: thread = tile row
        const int r = warp * 32 + lane;
        const int m = m0 + r;
        const bool row_ok = m < batch;
        const uint32_t lanes = uint32_t(warp * 32) << 16;
        // warp-uniform decisions: the TMEM loads below are warp-collective
        const bool ok1 = __all_sync(0xffffffffu, fw_wait(&done1, 0, &fail));
        if (ok1) {
            tc::fence_after_sync();
            fw_hidden_epilogue(tmem + lanes, b1, (H1 && row_ok) ? H1 + int64_t(m) * HID : nullptr, hbuf, r);
            tc::fence_before_sync();
        }
        tc::fence_proxy_async();  // the h buffer, written here, is read by the tensor core
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tc::smem_u32(&h1_ready)) : "memory");
        const bool ok2 = __all_sync(0xffffffffu, ok1 && fw_wait(&done2, 0, &fail));
        if (ok2) {
            tc::fence_after_sync();
            fw_hidden_epilogue(tmem + lanes + 256u, b2, (H2 && row_ok) ? H2 + int64_t(m) * HID : nullptr, hbuf, r);
            tc::fence_before_sync();
        }
        tc::fence_proxy_async();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tc::smem_u32(&h2_ready)) : "memory");
        const bool ok3 = __all_sync(0xffffffffu, ok2 && fw_wait(&done3, 0, &fail));
        if (ok3) {
            tc::fence_after_sync();
            float v[16];
            tc::tmem_ld16(tmem + lanes, v);
            if (row_ok)
#pragma unroll
                for (int j = 0; j < OUT; ++j) Y[int64_t(m) * OUT + j] = v[j] + b3p[j];
        }
    }
    __syncwarp();
    if (threadIdx.x == 128) {
        // loads issued but never consumed: let them land before the CTA exits
        for (int kt = max(0, issued1 - FW_S1); kt < issued1; ++kt)
            tc::mbar_wait_bounded(&full1[kt % FW_S1], (kt / FW_S1) & 1, tc::MBAR_SPIN_LIMIT);
        for (int kt = max(0, issued2 - 2); kt < issued2; ++kt)
            tc::mbar_wait_bounded(&full2[kt & 1], (kt >> 1) & 1, tc::MBAR_SPIN_LIMIT);
        if (issued3) tc::mbar_wait_bounded(&full3, 0, tc::MBAR_SPIN_LIMIT);
    }
    if (threadIdx.x == 160) tc::mbar_wait_bounded(&done3, 0, tc::MBAR_SPIN_LIMIT);  // MMAs in flight
    __syncthreads();
    if (threadIdx.x == 0 && *(volatile int*)&fail) atomicOr(err, ERR_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 4) tc::tmem_dealloc(tmem, 512);
}

}  // namespace
}  // namespace hgmm

using namespace hgmm;
using hgmm::tc::GemmArgs;

struct hgmm_mlp {
    int device = 0;
    int max_batch = 0;
    int step = 0;
    std::vector<void*> allocs;
    float* P = nullptr;   // FP32 master parameters
    float* G = nullptr;   // gradients
    float* Mo = nullptr;  // Adam moments
    float* Vo = nullptr;
    bf16* W1 = nullptr;
    bf16* W2 = nullptr;
    bf16* W3 = nullptr;   // 16 x 256, rows >= 9 zero
    float* b3p = nullptr; // 16
    bf16* Xg = nullptr;   // gathered batch
    float* Lg = nullptr;
    bf16* H1 = nullptr;
    bf16* H2 = nullptr;
    float* Y = nullptr;   // batch x 9
    bf16* dY = nullptr;   // batch x 16
    float* dYf = nullptr;
    bf16* dZ2 = nullptr;
    bf16* dZ1 = nullptr;
    float* part = nullptr;
    float* loss = nullptr;
    int* err = nullptr;
    float* ws = nullptr;      // K-slice partials of the weight-gradient products
    long long ws_cap = 0;     // floats
    bf16* prop_x = nullptr;   // hgmm_propose: one pair's input (1280)
    double* prop_fr = nullptr;  // ... its frames (source, target: 32)
    float* prop_y = nullptr;  // ... the network's output (9)
};

namespace {

template <typename T>
bool malloc_into(hgmm_mlp* m, T** p, size_t count) {
    *p = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T)) != cudaSuccess) return false;
    m->allocs.push_back(*p);
    return cudaMemset(*p, 0, (count ? count : 1) * sizeof(T)) == cudaSuccess;
}

bool a16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Operand (rows x K) at base with element strides (rs, ks): the tile loader
// needs 16-byte vectors along K (ks == 1) or along the rows (rs == 1).
bool operand_ok(const void* base, long long rs, long long ks, int rows, int K) {
    if (!a16(base)) return false;
    if (ks == 1) return rs % 8 == 0 && K % 8 == 0;
    if (rs == 1) return ks % 8 == 0 && rows % 8 == 0;
    return false;
}

constexpr int MAX_SLICES = 32;

template <int BN>
int gemm_launch(const GemmArgs& g, int slices, cudaStream_t s) {
    const dim3 grid((g.M + tc::GEMM_BM - 1) / tc::GEMM_BM, (g.N + BN - 1) / BN, slices);
    tc::k_gemm_bf16<BN><<<grid, tc::GEMM_THREADS, tc::gemm_smem_bytes(BN), s>>>(g);
    return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}

// cuTensorMapEncodeTiled from the driver (resolved once), or null.
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of a K-contiguous BF16 operand (rows x K, row stride rs
// elements): dimensions (K, rows), box 64 x box_rows, 128-byte swizzle,
// zeros outside the matrix.
bool encode_operand(CUtensorMap* tm, const bf16* base, long long rs, int rows, int K, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
    const cuuint64_t strides[1] = {cuuint64_t(rs) * sizeof(bf16)};
    const cuuint32_t box[2] = {cuuint32_t(tc::GEMM_BK), cuuint32_t(box_rows)};
    const cuuint32_t estr[2] = {1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
int gemm_tma_launch(const GemmArgs& g, const CUtensorMap& ta, const CUtensorMap& tb, cudaStream_t s) {
    const dim3 grid((g.M + tc::GEMM_BM - 1) / tc::GEMM_BM, (g.N + BN - 1) / BN);
    tc::k_gemm_tma<BN><<<grid, tc::GEMM_THREADS, tc::tma_smem_bytes(BN), s>>>(ta, tb, g);
    return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}

// D = A B^T with the fused epilogue of g.  Both operands K-contiguous and
// no K slices: the warp-specialised TMA kernel.  Otherwise the cp.async
// kernel: N <= 16 runs 128 x 16 tiles, larger N 128 x 128 tiles; when the
// tiles alone cannot fill the GPU and K is long (the weight gradients: K =
// batch), K is cut into 64-multiple slices whose FP32 partials go to ws and
// are summed in a fixed order.
int gemm(GemmArgs g, cudaStream_t s, float* ws = nullptr, long long ws_cap = 0) {
    if (g.M < 1 || g.N < 1 || g.K < 1 || !operand_ok(g.A, g.a_m, g.a_k, g.M, g.K) ||
        !operand_ok(g.B, g.b_n, g.b_k, g.N, g.K))
        return HGMM_EINVAL;
    const int bn = g.N <= 16 ? 16 : 128;
    const int tiles = ((g.M + tc::GEMM_BM - 1) / tc::GEMM_BM) * ((g.N + bn - 1) / bn);
    const int kt = (g.K + tc::GEMM_BK - 1) / tc::GEMM_BK;
    int slices = 1;
    if (ws && g.epi == tc::EPI_F32 && tiles < 128) slices = std::min(std::min(MAX_SLICES, kt), (304 + tiles - 1) / tiles);
    g.k_split = ((kt + slices - 1) / slices) * tc::GEMM_BK;
    slices = (g.K + g.k_split - 1) / g.k_split;
    if (slices <= 1 && g.a_k == 1 && g.b_k == 1) {
        // (operand_ok has checked 16-byte bases and row strides % 8 == 0)
        CUtensorMap ta, tb;
        if (encode_operand(&ta, g.A, g.a_m, g.M, g.K, tc::GEMM_BM) &&
            encode_operand(&tb, g.B, g.b_n, g.N, g.K, bn)) {
            g.k_split = g.K;
            g.split_stride = 0;
            return bn == 16 ? gemm_tma_launch<16>(g, ta, tb, s) : gemm_tma_launch<128>(g, ta, tb, s);
        }
    }
    if (slices <= 1) {
        g.split_stride = 0;
        return bn == 16 ? gemm_launch<16>(g, 1, s) : gemm_launch<128>(g, 1, s);
    }
    // partials at the output's own offsets, one copy per slice
    const long long span = (long long)(g.M - 1) * g.o_m + (long long)(g.N - 1) * g.o_n + 1;
    if ((long long)slices * span > ws_cap) return HGMM_ECAPACITY;
    float* out = g.out_f32;
    g.out_f32 = ws;
    g.split_stride = span;
    const int rc = bn == 16 ? gemm_launch<16>(g, slices, s) : gemm_launch<128>(g, slices, s);
    if (rc) return rc;
    tc::k_sum_slices<<<304, 256, 0, s>>>(ws, slices, span, g.M, g.N, g.n_store, g.o_m, g.o_n, out);
    return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}

GemmArgs gargs(const bf16* A, long long a_m, long long a_k, const bf16* B, long long b_n,
               long long b_k, int M, int N, int K, int epi, int* err) {
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.A = A;
    g.a_m = a_m;
    g.a_k = a_k;
    g.B = B;
    g.b_n = b_n;
    g.b_k = b_k;
    g.M = M;
    g.N = N;
    g.K = K;
    g.n_store = N;
    g.k_split = K;
    g.split_stride = 0;
    g.epi = epi;
    g.err = err;
    return g;
}

// The fused forward (one launch for the three layers; the hidden layers go
// to m->H1 / m->H2 only when the backward pass needs them), or HGMM_ECUDA if
// its tensor maps cannot be encoded (the caller then runs the three GEMMs).
int forward_fused(hgmm_mlp* m, const bf16* X, int batch, float* Y, cudaStream_t s, bool keep_hidden) {
    CUtensorMap tx, t1, t2, t3;
    if (!encode_operand(&tx, X, IN, batch, IN, 128) || !encode_operand(&t1, m->W1, IN, HID, IN, HID) ||
        !encode_operand(&t2, m->W2, HID, HID, HID, HID) || !encode_operand(&t3, m->W3, HID, OUTP, HID, OUTP))
        return HGMM_ECUDA;
    k_mlp_forward<<<(batch + 127) / 128, FW_THREADS, FW_SMEM, s>>>(tx, t1, t2, t3, m->P + OFF_B1, m->P + OFF_B2,
                                                                 m->b3p, keep_hidden ? m->H1 : nullptr,
                                                                 keep_hidden ? m->H2 : nullptr, Y, batch, m->err);
    return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}

int forward_impl(hgmm_mlp* m, const bf16* X, int batch, float* Y, cudaStream_t s, bool keep_hidden = true) {
    if (forward_fused(m, X, batch, Y, s, keep_hidden) == HGMM_OK) return HGMM_OK;
    GemmArgs g = gargs(X, IN, 1, m->W1, IN, 1, batch, HID, IN, tc::EPI_BIAS_RELU_BF16, m->err);
    g.bias = m->P + OFF_B1;
    g.out_bf16 = m->H1;
    g.o_m = HID;
    g.o_n = 1;
    if (int rc = gemm(g, s, m->ws, m->ws_cap)) return rc;
    g = gargs(m->H1, HID, 1, m->W2, HID, 1, batch, HID, HID, tc::EPI_BIAS_RELU_BF16, m->err);
    g.bias = m->P + OFF_B2;
    g.out_bf16 = m->H2;
    g.o_m = HID;
    g.o_n = 1;
    if (int rc = gemm(g, s, m->ws, m->ws_cap)) return rc;
    g = gargs(m->H2, HID, 1, m->W3, HID, 1, batch, OUTP, HID, tc::EPI_BIAS_F32, m->err);
    g.bias = m->b3p;
    g.out_f32 = Y;
    g.o_m = OUT;
    g.o_n = 1;
    g.n_store = OUT;
    return gemm(g, s);
}

bool set_gemm_smem() {
    return cudaFuncSetAttribute(tc::k_gemm_bf16<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tc::gemm_smem_bytes(128)) == cudaSuccess &&
           cudaFuncSetAttribute(tc::k_gemm_bf16<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tc::gemm_smem_bytes(16)) == cudaSuccess &&
           cudaFuncSetAttribute(tc::k_gemm_tma<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tc::tma_smem_bytes(128)) == cudaSuccess &&
           cudaFuncSetAttribute(tc::k_gemm_tma<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tc::tma_smem_bytes(16)) == cudaSuccess &&
           cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM) == cudaSuccess;
}

int check_dev(const hgmm_mlp* m) {
    int cur = -1;
    return (cudaGetDevice(&cur) == cudaSuccess && cur == m->device) ? HGMM_OK : HGMM_EINVAL;
}

}  // namespace

extern "C" {

int hgmm_mlp_create(int32_t max_batch, hgmm_mlp** out) {
    if (!out) return HGMM_EINVAL;
    *out = nullptr;
    if (max_batch < 1 || max_batch > 65536) return HGMM_EINVAL;
    hgmm_mlp* m = new hgmm_mlp();
    if (cudaGetDevice(&m->device) != cudaSuccess) {
        delete m;
        return HGMM_ECUDA;
    }
    m->max_batch = max_batch;
    const size_t B = size_t(max_batch);
    const int nchunks = (max_batch + COLSUM_ROWS - 1) / COLSUM_ROWS;
    bool good = malloc_into(m, &m->P, N_PARAMS) && malloc_into(m, &m->G, N_PARAMS) &&
                malloc_into(m, &m->Mo, N_PARAMS) && malloc_into(m, &m->Vo, N_PARAMS) &&
                malloc_into(m, &m->W1, size_t(HID) * IN) && malloc_into(m, &m->W2, size_t(HID) * HID) &&
                malloc_into(m, &m->W3, size_t(OUTP) * HID) && malloc_into(m, &m->b3p, OUTP) &&
                malloc_into(m, &m->Xg, B * IN) && malloc_into(m, &m->Lg, B * HGMM_LABEL_FLOATS) &&
                malloc_into(m, &m->H1, B * HID) && malloc_into(m, &m->H2, B * HID) &&
                malloc_into(m, &m->Y, B * OUT) && malloc_into(m, &m->dY, B * OUTP) &&
                malloc_into(m, &m->dYf, B * OUTP) && malloc_into(m, &m->dZ2, B * HID) &&
                malloc_into(m, &m->dZ1, B * HID) && malloc_into(m, &m->part, size_t(nchunks) * 3 * HID) &&
                malloc_into(m, &m->loss, 1) && malloc_into(m, &m->err, 1) &&
                malloc_into(m, &m->prop_x, IN) && malloc_into(m, &m->prop_fr, 2 * HGMM_FRAME_DOUBLES) &&
                malloc_into(m, &m->prop_y, 16);
    m->ws_cap = (long long)MAX_SLICES * HID * IN;
    good = good && malloc_into(m, &m->ws, size_t(m->ws_cap));
    good = good && set_gemm_smem();
    if (!good) {
        hgmm_mlp_destroy(m);
        return HGMM_ENOMEM;
    }
    *out = m;
    return HGMM_OK;
}

void hgmm_mlp_destroy(hgmm_mlp* m) {
    if (!m) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(m->device);
    for (void* p : m->allocs) cudaFree(p);
    cudaSetDevice(cur);
    delete m;
}

int hgmm_mlp_set_params(hgmm_mlp* m, const float* h_params, int64_t count) {
    if (!m || !h_params || count != N_PARAMS) return HGMM_EINVAL;
    if (int rc = check_dev(m)) return rc;
    const size_t bytes = size_t(N_PARAMS) * sizeof(float);
    bool good = cudaMemcpy(m->P, h_params, bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                cudaMemset(m->Mo, 0, bytes) == cudaSuccess && cudaMemset(m->Vo, 0, bytes) == cudaSuccess &&
                cudaMemset(m->G, 0, bytes) == cudaSuccess;
    if (!good) return HGMM_ECUDA;
    k_refresh<<<512, 256>>>(m->P, m->W1, m->W2, m->W3, m->b3p);
    m->step = 0;
    return cudaDeviceSynchronize() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}

int hgmm_mlp_get_params(hgmm_mlp* m, float* h_params, int64_t count) {
    if (!m || !h_params || count != N_PARAMS) return HGMM_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return HGMM_ECUDA;
    return cudaMemcpy(h_params, m->P, size_t(N_PARAMS) * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
               ? HGMM_OK
               : HGMM_ECUDA;
}

int hgmm_mlp_read_grads(hgmm_mlp* m, float* h_grads, int64_t count) {
    if (!m || !h_grads || count != N_PARAMS) return HGMM_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return HGMM_ECUDA;
    return cudaMemcpy(h_grads, m->G, size_t(N_PARAMS) * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
               ? HGMM_OK
               : HGMM_ECUDA;
}

int hgmm_mlp_forward(hgmm_mlp* m, const uint16_t* d_x, int32_t batch, float* d_y, void* stream) {
    if (!m || !d_x || !d_y || batch < 1 || batch > m->max_batch || !a16(d_x)) return HGMM_EINVAL;
    if (int rc = check_dev(m)) return rc;
    return forward_impl(m, reinterpret_cast<const bf16*>(d_x), batch, d_y, static_cast<cudaStream_t>(stream),
                        false);
}

int hgmm_mlp_gradients(hgmm_mlp* m, const uint16_t* d_x, const float* d_labels, const int32_t* d_index,
                       int32_t batch, int32_t n_rows, float w_t, float* d_loss, void* stream) {
    if (!m || !d_x || !d_labels || batch < 1 || batch > m->max_batch || !a16(d_x) || !(w_t >= 0.f))
        return HGMM_EINVAL;
    if (d_index && n_rows < 1) return HGMM_EINVAL;
    if (int rc = check_dev(m)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bf16* X = reinterpret_cast<const bf16*>(d_x);
    const float* L = d_labels;
    if (d_index) {
        k_gather<<<batch, 160, 0, s>>>(X, d_labels, d_index, n_rows, m->Xg, m->Lg, m->err);
        X = m->Xg;
        L = m->Lg;
    }
    if (int rc = forward_impl(m, X, batch, m->Y, s)) return rc;
    k_loss<<<1, 256, 0, s>>>(m->Y, L, batch, w_t, m->dY, m->dYf, d_loss ? d_loss : m->loss);
    // dW3^T[h][o] = sum_r H2[r][h] dY[r][o]: A = H2^T, B = dY^T (both read along rows)
    GemmArgs g = gargs(m->H2, 1, HID, m->dY, 1, OUTP, HID, OUTP, batch, tc::EPI_F32, m->err);
    g.out_f32 = m->G + OFF_W3;
    g.o_m = 1;
    g.o_n = HID;
    g.n_store = OUT;
    if (int rc = gemm(g, s, m->ws, m->ws_cap)) return rc;
    // dZ2 = (dY W3) * [H2 > 0]: B[n = h][k = o] = W3[o][h]
    g = gargs(m->dY, OUTP, 1, m->W3, 1, HID, batch, HID, OUTP, tc::EPI_MASK_BF16, m->err);
    g.mask = m->H2;
    g.mask_m = HID;
    g.out_bf16 = m->dZ2;
    g.o_m = HID;
    g.o_n = 1;
    if (int rc = gemm(g, s, m->ws, m->ws_cap)) return rc;
    // dW2 = dZ2^T H1
    g = gargs(m->dZ2, 1, HID, m->H1, 1, HID, HID, HID, batch, tc::EPI_F32, m->err);
    g.out_f32 = m->G + OFF_W2;
    g.o_m = HID;
    g.o_n = 1;
    if (int rc = gemm(g, s, m->ws, m->ws_cap)) return rc;
    // dZ1 = (dZ2 W2) * [H1 > 0]
    g = gargs(m->dZ2, HID, 1, m->W2, 1, HID, batch, HID, HID, tc::EPI_MASK_BF16, m->err);
    g.mask = m->H1;
    g.mask_m = HID;
    g.out_bf16 = m->dZ1;
    g.o_m = HID;
    g.o_n = 1;
    if (int rc = gemm(g, s, m->ws, m->ws_cap)) return rc;
    // dW1 = dZ1^T x
    g = gargs(m->dZ1, 1, HID, X, 1, IN, HID, IN, batch, tc::EPI_F32, m->err);
    g.out_f32 = m->G + OFF_W1;
    g.o_m = IN;
    g.o_n = 1;
    if (int rc = gemm(g, s, m->ws, m->ws_cap)) return rc;
    const int nchunks = (batch + COLSUM_ROWS - 1) / COLSUM_ROWS;
    k_colsum_partial<<<dim3(nchunks, 3), 256, 0, s>>>(m->dZ1, m->dZ2, m->dYf, batch, m->part);
    k_colsum_final<<<3, 256, 0, s>>>(m->part, nchunks, m->G);
    return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}

int hgmm_mlp_adam(hgmm_mlp* m, float lr, void* stream) {
    if (!m || !(lr >= 0.f)) return HGMM_EINVAL;
    if (int rc = check_dev(m)) return rc;
    m->step += 1;
    const double c1 = 1.0 / (1.0 - std::pow(0.9, m->step));
    const double c2 = 1.0 / (1.0 - std::pow(0.999, m->step));
    k_adam<<<608, 256, 0, static_cast<cudaStream_t>(stream)>>>(m->P, m->G, m->Mo, m->Vo, lr, float(c1),
                                                              float(c2), m->W1, m->W2, m->W3, m->b3p);
    return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}

int hgmm_mlp_train_step(hgmm_mlp* m, const uint16_t* d_x, const float* d_labels, const int32_t* d_index,
                        int32_t batch, int32_t n_rows, float w_t, float lr, float* d_loss, void* stream) {
    if (int rc = hgmm_mlp_gradients(m, d_x, d_labels, d_index, batch, n_rows, w_t, d_loss, stream))
        return rc;
    return hgmm_mlp_adam(m, lr, stream);
}

int hgmm_mlp_sync(hgmm_mlp* m, void* stream) {
    if (!m) return HGMM_EINVAL;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return HGMM_ECUDA;
    int e = 0;
    if (cudaMemcpy(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(m->err, 0, sizeof(int)) != cudaSuccess)
        return HGMM_ECUDA;
    if (e & ERR_TIMEOUT) return HGMM_ETIMEOUT;
    if (e & ERR_INDEX) return HGMM_EINVAL;
    return HGMM_OK;
}

int hgmm_tree_features(hgmm_tree* t, uint16_t* d_feat, double* d_frame, void* stream) {
    if (!t || !d_feat || !d_frame || !t->built || t->depth < 2 || !a16(d_feat)) return HGMM_EINVAL;
    k_tree_features<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(
        t->root, t->stat, reinterpret_cast<bf16*>(d_feat), d_frame);
    return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}

int hgmm_propose(hgmm_tree* tgt, hgmm_tree* src, hgmm_mlp* m, void* stream, double* d_T_out) {
    if (!tgt || !src || !m || !d_T_out) return HGMM_EINVAL;
    if (int rc = check_dev(m)) return rc;
    uint16_t* x = reinterpret_cast<uint16_t*>(m->prop_x);
    // network input: [features(source), features(target)], frames likewise
    if (int rc = hgmm_tree_features(src, x, m->prop_fr, stream)) return rc;
    if (int rc = hgmm_tree_features(tgt, x + HGMM_FEAT_PER_CLOUD, m->prop_fr + HGMM_FRAME_DOUBLES, stream))
        return rc;
    if (int rc = hgmm_mlp_forward(m, x, 1, m->prop_y, stream)) return rc;
    return hgmm_pose_decode(m->prop_y, m->prop_fr, 1, d_T_out, stream);
}

int hgmm_pose_decode(const float* d_y, const double* d_frames, int32_t n, double* d_T, void* stream) {
    if (!d_y || !d_frames || !d_T || n < 1) return HGMM_EINVAL;
    k_decode<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(d_y, d_frames, n, d_T);
    return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}

int hgmm_pose_encode(const double* d_T, const double* d_frames, int32_t n, float* d_labels, void* stream) {
    if (!d_T || !d_frames || !d_labels || n < 1) return HGMM_EINVAL;
    k_encode<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(d_T, d_frames, n, d_labels);
    return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}

int hgmm_debug_gemm(const uint16_t* d_A, int64_t a_m, int64_t a_k, const uint16_t* d_B, int64_t b_n,
                    int64_t b_k, int32_t M, int32_t N, int32_t K, float* d_out, void* stream) {
    if (!d_A || !d_B || !d_out) return HGMM_EINVAL;
    static int* err = nullptr;  // error word of the checking launches
    if (!err && (cudaMalloc(&err, sizeof(int)) != cudaSuccess || cudaMemset(err, 0, sizeof(int)) != cudaSuccess))
        return HGMM_ECUDA;
    static bool attr = false;
    static float* ws = nullptr;
    const long long ws_cap = (long long)MAX_SLICES * 256 * 1536;
    if (!attr) {
        if (!set_gemm_smem() || cudaMalloc(&ws, size_t(ws_cap) * sizeof(float)) != cudaSuccess) return HGMM_ECUDA;
        attr = true;
    }
    GemmArgs g = gargs(reinterpret_cast<const bf16*>(d_A), a_m, a_k, reinterpret_cast<const bf16*>(d_B),
                       b_n, b_k, M, N, K, tc::EPI_F32, err);
    g.out_f32 = d_out;
    g.o_m = N;
    g.o_n = 1;
    return gemm(g, static_cast<cudaStream_t>(stream), ws, ws_cap);
}

int hgmm_pose_select(int32_t n, const double* d_T_a, const double* d_obj_a, const double* d_T_b,
                     const double* d_obj_b, double* d_T_out, int32_t* d_choice, double* d_obj_out,
                     void* stream) {
    if (n < 1 || !d_T_a || !d_obj_a || !d_T_b || !d_obj_b || !d_T_out) return HGMM_EINVAL;
    k_select<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(n, d_T_a, d_obj_a, d_T_b,
                                                                             d_obj_b, d_T_out, d_choice,
                                                                             d_obj_out);
    return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}

int hgmm_pose_compose(int32_t n, const double* d_A, const double* d_B, double* d_out, void* stream) {
    if (n < 1 || !d_A || !d_B || !d_out || d_out == d_A || d_out == d_B) return HGMM_EINVAL;
    k_compose<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(n, d_A, d_B, d_out);
    return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}

}  // extern "C"
