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

int forward_impl(hgmm_mlp* m, const bf16* X, int batch, float* Y, cudaStream_t s) {
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
                                tc::tma_smem_bytes(16)) == cudaSuccess;
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
    return forward_impl(m, reinterpret_cast<const bf16*>(d_x), batch, d_y, static_cast<cudaStream_t>(stream));
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
