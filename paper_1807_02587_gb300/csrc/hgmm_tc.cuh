// Fifth-generation tensor-core (tcgen05) GEMM for the pose-proposal network.
//
//   D[m][n] = sum_k A[m][k] * B[n][k]      (BF16 operands, FP32 accumulation)
//
// One CTA of 128 threads computes a 128 x BN tile with its accumulator in
// tensor memory (TMEM).  Operands are staged into shared memory in the
// canonical no-swizzle K-major layout: 8-row x 16-byte core matrices, core
// matrices adjacent along K 128 bytes apart (leading byte offset), 8-row
// groups 1024 bytes apart (stride byte offset), 64 K-elements per stage.
// Two stages: while the tensor core works on one, the threads fill the
// other; one elected thread issues tcgen05.mma and commits each stage to an
// mbarrier, whose phase tells the loaders the stage is free again.  A or B
// may be stored with K contiguous (16-byte vector loads along K) or with
// M (resp. N) contiguous (16-byte vector loads along M, scattered into the
// K-major tile), which is how the weight-gradient products read activations
// without a transposed copy.  Every mbarrier wait has an iteration limit: a
// wait that runs out records an error word and the kernel frees its TMEM and
// returns.  The epilogue reads the accumulator with tcgen05.ld (warp w owns
// TMEM lanes 32w..32w+31, i.e. tile rows) and applies one of the fused
// epilogues below.
#pragma once

#include "hgmm_async.cuh"
#include <cstdint>
#include <cuda_bf16.h>

namespace hgmm {
namespace tc {

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1, no swizzle, base offset 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// A and B BF16 (bits 7-9 = 1, bits 10-12 = 1), both K-major, N >> 3 at bit
// 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

// Arrive once on the mbarrier when every tcgen05.mma this thread issued so
// far has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}

// TMEM allocation by one whole warp; the column base lands in *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(dst)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape), and
// the wait for the load, in one statement so no use can be scheduled early.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ GEMM
enum Epilogue : int {
    EPI_F32 = 0,             // out_f32[m, n] = acc
    EPI_BIAS_F32 = 1,        // out_f32[m, n] = acc + bias[n]
    EPI_BIAS_RELU_BF16 = 2,  // out_bf16[m, n] = bf16(max(acc + bias[n], 0))
    EPI_MASK_BF16 = 3,       // out_bf16[m, n] = bf16(mask[m, n] > 0 ? acc : 0)
};

struct GemmArgs {
    const __nv_bfloat16* A;
    long long a_m, a_k;   // element strides: A[m][k] = A[m * a_m + k * a_k]
    const __nv_bfloat16* B;
    long long b_n, b_k;   // B[n][k] = B[n * b_n + k * b_k]
    int M, N, K;
    int k_split;          // K elements per blockIdx.z slice (multiple of 64)
    long long split_stride;  // EPI_F32 with slices: slice z writes out_f32 + z * split_stride
    int n_store;          // columns n >= n_store are not written
    int epi;
    const float* bias;
    const __nv_bfloat16* mask;
    long long mask_m;
    float* out_f32;
    __nv_bfloat16* out_bf16;
    long long o_m, o_n;   // out[m * o_m + n * o_n]
    int* err;
};

constexpr int GEMM_BM = 128;
constexpr int GEMM_BK = 64;
constexpr int GEMM_THREADS = 128;
constexpr int GEMM_STAGES = 4;
constexpr int GEMM_A_STAGE = GEMM_BM * GEMM_BK * 2;  // bytes
constexpr uint32_t CORE_LBO = 128;                   // core matrices adjacent along K
constexpr uint32_t CORE_SBO = (GEMM_BK / 8) * 128;   // 8-row groups

__host__ __device__ constexpr int gemm_b_stage(int bn) { return bn * GEMM_BK * 2; }
__host__ __device__ constexpr int gemm_smem_bytes(int bn) {
    return GEMM_STAGES * (GEMM_A_STAGE + gemm_b_stage(bn));
}
__host__ __device__ constexpr uint32_t gemm_tmem_cols(int bn) {
    return bn <= 32 ? 32u : (bn <= 64 ? 64u : (bn <= 128 ? 128u : 256u));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool pred) {
    // src-size 0 fills the 16 bytes with zeros and reads nothing
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(pred ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// Fill one K-major operand tile (rows x 64) of shared memory, element (row,
// k) from src[row * rs + k * ks]; rows >= nrows_valid and k >= k_end read
// zero.  ks == 1: 16-byte asynchronous copies along K (cp.async; the caller
// commits the group), consecutive threads on consecutive rows of one K
// chunk so that eight threads fill one 128-byte core matrix.  Otherwise
// rs == 1: 16-byte loads along the row index, scattered per element
// (synchronous).
__device__ __forceinline__ void stage_tile(unsigned char* dst, const __nv_bfloat16* src, int rows,
                                           int row0, int nrows_valid, long long rs, long long ks,
                                           int k0, int k_end) {
    if (ks == 1) {
        const uint32_t d0 = smem_u32(dst);
        for (int q = threadIdx.x; q < rows * 8; q += GEMM_THREADS) {
            const int r = q % rows, c = q / rows;
            const int row = row0 + r, k = k0 + c * 8;
            const bool ok = row < nrows_valid && k < k_end;
            cp_async16(d0 + (r >> 3) * CORE_SBO + c * CORE_LBO + (r & 7) * 16,
                       ok ? (const void*)(src + row * rs + k) : (const void*)src, ok);
        }
    } else {
        const int groups = rows >> 3;
        for (int q = threadIdx.x; q < groups * GEMM_BK; q += GEMM_THREADS) {
            const int kk = q % GEMM_BK, g = q / GEMM_BK;
            const int k = k0 + kk, row = row0 + g * 8;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (row < nrows_valid && k < k_end) v = __ldg(reinterpret_cast<const uint4*>(src + row + k * ks));
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
            unsigned char* d = dst + g * CORE_SBO + (kk >> 3) * CORE_LBO + (kk & 7) * 2;
#pragma unroll
            for (int j = 0; j < 8; ++j) *reinterpret_cast<__nv_bfloat16*>(d + j * 16) = e[j];
        }
    }
}

// One CTA: a 128 x BN tile of D over the K slice of blockIdx.z, in a ring of
// GEMM_STAGES shared-memory stages.  Tile kt is loaded GEMM_STAGES - 1
// steps ahead into the stage that tile kt - 1 used, after the mbarrier of
// that stage says its MMAs are done; before the MMAs of tile kt every
// thread waits for its own copies of that tile (cp.async.wait_group), makes
// them visible to the tensor core (fence.proxy.async) and meets the others.
template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS, 1) k_gemm_bf16(GemmArgs g) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "M = 128 needs N in [16, 256], step 16");
    constexpr int S = GEMM_STAGES;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[S];
    __shared__ uint32_t tmem_slot;
    constexpr uint32_t NCOLS = gemm_tmem_cols(BN);
    constexpr uint32_t IDESC = idesc_bf16_f32(GEMM_BM, BN);
    constexpr int STAGE = GEMM_A_STAGE + gemm_b_stage(BN);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * GEMM_BM, n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * g.k_split;
    const int ke = min(g.K, kb + g.k_split);

    if (warp == 0) {
        tmem_alloc(&tmem_slot, NCOLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < S; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;

    const int nk = ke > kb ? (ke - kb + GEMM_BK - 1) / GEMM_BK : 0;
    auto load = [&](int t) {
        unsigned char* sA = smem + (t % S) * STAGE;
        stage_tile(sA, g.A, GEMM_BM, m0, g.M, g.a_m, g.a_k, kb + t * GEMM_BK, ke);
        stage_tile(sA + GEMM_A_STAGE, g.B, BN, n0, g.N, g.b_n, g.b_k, kb + t * GEMM_BK, ke);
    };
#pragma unroll 1
    for (int t = 0; t < S - 1; ++t) {
        if (t < nk) load(t);
        cp_async_commit();
    }
    bool ok = true;
#pragma unroll 1
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % S;
        cp_async_wait<S - 2>();  // this thread's copies of tile kt have landed
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_after_sync();
            unsigned char* sA = smem + s * STAGE;
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sA + GEMM_A_STAGE);
#pragma unroll
            for (int kk = 0; kk < GEMM_BK / 16; ++kk) {
                // one K = 16 step spans two core matrices along K
                const uint64_t da = smem_desc(a0 + kk * 2 * CORE_LBO, CORE_LBO, CORE_SBO);
                const uint64_t db = smem_desc(b0 + kk * 2 * CORE_LBO, CORE_LBO, CORE_SBO);
                mma_bf16(tmem, da, db, IDESC, (kt | kk) != 0 ? 1u : 0u);
            }
            mma_commit(&bars[s]);
        }
        // refill the stage of tile kt - 1 with tile kt + S - 1
        const int nt = kt + S - 1;
        if (kt >= 1 && nt < nk) {
            const int ps = (kt - 1) % S;
            const bool w = mbar_wait_bounded(&bars[ps], ((kt - 1) / S) & 1, MBAR_SPIN_LIMIT);
            ok = __syncthreads_and(w) != 0;
            if (!ok) break;
        }
        if (nt < nk) load(nt);
        cp_async_commit();
    }
    cp_async_wait<0>();
    if (ok && nk > 0) {
        const int last = nk - 1;
        const bool w = mbar_wait_bounded(&bars[last % S], (last / S) & 1, MBAR_SPIN_LIMIT);
        ok = __syncthreads_and(w) != 0;
    }
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(g.err, 1);
        // give MMAs still in flight a bounded chance to finish before freeing
        if (nk > 0) mbar_wait_bounded(&bars[(nk - 1) % S], ((nk - 1) / S) & 1, MBAR_SPIN_LIMIT);
    } else {
        fence_after_sync();
        const int r = warp * 32 + lane;
        const int m = m0 + r;
        const uint32_t trow = tmem + (uint32_t(warp * 32) << 16);
        float* outf = g.out_f32 ? g.out_f32 + blockIdx.z * g.split_stride : nullptr;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            if (nk > 0) {
                tmem_ld16(trow + uint32_t(c0), v);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.f;
            }
            if (m >= g.M) continue;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int n = n0 + c0 + i;
                if (n >= g.N || n >= g.n_store) continue;
                float x = v[i];
                const long long o = m * g.o_m + n * g.o_n;
                switch (g.epi) {
                    case EPI_F32: outf[o] = x; break;
                    case EPI_BIAS_F32: outf[o] = x + g.bias[n]; break;
                    case EPI_BIAS_RELU_BF16:
                        x += g.bias[n];
                        g.out_bf16[o] = __float2bfloat16_rn(x > 0.f ? x : 0.f);
                        break;
                    default: {
                        const float mk = __bfloat162float(g.mask[m * g.mask_m + n]);
                        g.out_bf16[o] = __float2bfloat16_rn(mk > 0.f ? x : 0.f);
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// Fixed-order sum of the K-slice partials: out[i] = sum_z ws[z * stride + i]
// for the n_store columns of an M x N (row stride o_m) output.
__global__ void k_sum_slices(const float* __restrict__ ws, int slices, long long stride, int M, int N,
                             int n_store, long long o_m, long long o_n, float* __restrict__ out) {
    const long long total = (long long)M * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int m = int(i / N), n = int(i % N);
        if (n >= n_store) continue;
        const long long o = m * o_m + n * o_n;
        float acc = 0.f;
        for (int z = 0; z < slices; ++z) acc += ws[z * stride + o];
        out[o] = acc;
    }
}

}  // namespace tc
}  // namespace hgmm
