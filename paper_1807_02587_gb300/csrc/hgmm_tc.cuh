// Fifth-generation tensor-core (tcgen05) GEMM for the pose-proposal network.
//
//   D[m][n] = sum_k A[m][k] * B[n][k]      (BF16 operands, FP32 accumulation)
//
// Two kernels compute a 128 x BN tile per CTA with the accumulator in
// tensor memory (TMEM):
//
// k_gemm_tma (both operands stored with K contiguous: the forward pass):
// warp-specialised.  One thread of warp 0 streams the operand tiles into a
// ring of shared-memory stages with TMA (cp.async.bulk.tensor, 128-byte
// swizzle, completion counted on each stage's "full" mbarrier); one thread
// of warp 1 waits for each full stage, issues the tcgen05.mma of its four
// K = 16 steps and commits them to the stage's "empty" mbarrier, which
// hands the stage back to the producer; after the last stage its commit on
// the "done" mbarrier releases the four epilogue warps.
//
// k_gemm_bf16 (any operand layout: the weight gradients read activations
// transposed, without a copy): all 128 threads stage operands with
// cp.async into the canonical no-swizzle K-major layout (8-row x 16-byte
// core matrices, adjacent along K 128 bytes apart, 8-row groups 1024 bytes
// apart, 64 K-elements per stage) in a ring of GEMM_STAGES stages filled
// GEMM_STAGES - 1 tiles ahead; one elected thread issues the MMAs and
// commits each stage to an mbarrier whose phase frees it for the loaders.
//
// Every mbarrier wait has an iteration limit: a wait that runs out records
// an error word; the kernel then waits (bounded) for its own copies and
// MMAs in flight, frees its TMEM and returns.  The epilogue reads the
// accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31, i.e. tile
// rows) and applies one of the fused epilogues below.
#pragma once

#include "hgmm_async.cuh"
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>

namespace hgmm {
namespace tc {

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1, no swizzle, base offset 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// The same for a K-major operand in the 128-byte swizzled layout that TMA
// writes with CU_TENSOR_MAP_SWIZZLE_128B: rows of 128 bytes (64 BF16 along
// K), 8-row atoms 1024 bytes apart (stride byte offset), the 16-byte chunks
// of row r permuted by r mod 8 (swizzle mode 2 at bits 61-63; the leading
// byte offset is not used by this layout and is set to 16 bytes).  The
// atoms must start on 1024-byte boundaries (base offset 0); a K step inside
// the 128-byte row advances the start address.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
           (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// 2-D TMA load of the box at (x, y) (x = innermost, elements) of the tensor
// map into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        :: "r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const void* tmap) {
    asm volatile("prefetch.tensormap [%0];" :: "l"(tmap) : "memory");
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

// 32 consecutive FP32 columns of this thread's TMEM lane, and the wait.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 consecutive FP32 columns of this thread's TMEM lane, and the wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
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

// Epilogue of one 16-column group of a row (shared by both kernels).
__device__ __forceinline__ void epilogue16(const GemmArgs& g, float* outf, int m, int n0c, const float (&v)[16]) {
    if (m >= g.M) return;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int n = n0c + i;
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

// Epilogue of 32 columns n0c.. of row m.  When all 32 columns are stored and
// the output rows are contiguous and 16-byte aligned, each thread writes its
// row's 32 values as full 16-byte vectors (64 bytes of BF16, 128 of FP32)
// and reads the bias as float4; otherwise element by element.
__device__ __forceinline__ void epilogue32(const GemmArgs& g, float* outf, int m, int n0c, const float (&v)[32]) {
    if (m >= g.M) return;
    const bool bf = g.epi == EPI_BIAS_RELU_BF16 || g.epi == EPI_MASK_BF16;
    const int lim = min(g.N, g.n_store);
    const long long o = m * g.o_m + n0c;
    const bool vec = n0c + 32 <= lim && g.o_n == 1 && g.epi != EPI_MASK_BF16 &&
                     ((bf ? reinterpret_cast<uintptr_t>(g.out_bf16 + o) : reinterpret_cast<uintptr_t>(outf + o)) &
                      15u) == 0 &&
                     (g.epi == EPI_F32 || (reinterpret_cast<uintptr_t>(g.bias + n0c) & 15u) == 0);
    if (!vec) {
        float a[16], b[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            a[i] = v[i];
            b[i] = v[16 + i];
        }
        epilogue16(g, outf, m, n0c, a);
        epilogue16(g, outf, m, n0c + 16, b);
        return;
    }
    float x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = v[i];
    if (g.epi != EPI_F32) {
        const float4* b4 = reinterpret_cast<const float4*>(g.bias + n0c);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 b = __ldg(b4 + j);
            x[4 * j] += b.x;
            x[4 * j + 1] += b.y;
            x[4 * j + 2] += b.z;
            x[4 * j + 3] += b.w;
        }
    }
    if (bf) {
        uint4* d = reinterpret_cast<uint4*>(g.out_bf16 + o);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float lo = fmaxf(x[8 * j + 2 * h], 0.f), hi = fmaxf(x[8 * j + 2 * h + 1], 0.f);
                const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
                w[h] = *reinterpret_cast<const uint32_t*>(&p);
            }
            d[j] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
        float4* d = reinterpret_cast<float4*>(outf + o);
#pragma unroll
        for (int j = 0; j < 8; ++j) d[j] = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
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
        if (BN % 32 == 0 && nk > 0) {
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                float v[32];
                tmem_ld32(trow + uint32_t(c0), v);
                epilogue32(g, outf, m, n0 + c0, v);
            }
        } else {
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                if (nk > 0) {
                    tmem_ld16(trow + uint32_t(c0), v);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = 0.f;
                }
                epilogue16(g, outf, m, n0 + c0, v);
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

constexpr int TMA_STAGES = 6;
constexpr int TMA_A_BYTES = GEMM_BM * 128;                       // 128 rows x 64 BF16
__host__ __device__ constexpr int tma_b_bytes(int bn) { return bn * 128; }
__host__ __device__ constexpr int tma_stage_bytes(int bn) { return TMA_A_BYTES + tma_b_bytes(bn); }
// dynamic shared memory: the stages, plus 1 KB so they can start on a 1024-byte boundary
__host__ __device__ constexpr int tma_smem_bytes(int bn) { return TMA_STAGES * tma_stage_bytes(bn) + 1024; }

// Warp-specialised TMA GEMM (operands K-contiguous; tmA / tmB map A as
// (K, M) and B as (K, N), box 64 x 128 and 64 x BN, 128-byte swizzle,
// zero fill outside the matrix).  Grid: (M tiles, N tiles), no K slices.
template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
k_gemm_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmArgs g) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "M = 128 needs N in [16, 256], step 16");
    constexpr int S = TMA_STAGES;
    constexpr int STAGE = tma_stage_bytes(BN);
    constexpr uint32_t NCOLS = gemm_tmem_cols(BN);
    constexpr uint32_t IDESC = idesc_bf16_f32(GEMM_BM, BN);
    extern __shared__ unsigned char tma_smem_raw[];
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    // stages on a 1024-byte boundary (the swizzle atoms' alignment)
    const uint32_t raw = smem_u32(tma_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * GEMM_BM, n0 = blockIdx.y * BN;
    const int nk = (g.K + GEMM_BK - 1) / GEMM_BK;

    if (warp == 0) {
        tmem_alloc(&tmem_slot, NCOLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 32) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&done, 1);
        fail = 0;
        fence_mbar_init();
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    int issued = 0;  // producer: stages whose loads were issued
    if (threadIdx.x == 0) {
        // ---- producer: stage kt % S gets tile kt once its previous tile's MMAs are done
        for (int kt = 0; kt < nk; ++kt) {
            const int st = kt % S;
            if (kt >= S && !mbar_wait_bounded(&empty[st], ((kt / S) - 1) & 1, MBAR_SPIN_LIMIT)) {
                atomicOr(g.err, 1);
                atomicExch(&fail, 1);
                break;
            }
            const uint32_t sa = base + st * STAGE;
            mbar_arrive_expect_tx(&full[st], uint32_t(STAGE));
            tma_load_2d(sa, &tmA, kt * GEMM_BK, m0, &full[st]);
            tma_load_2d(sa + TMA_A_BYTES, &tmB, kt * GEMM_BK, n0, &full[st]);
            issued = kt + 1;
        }
    } else if (threadIdx.x == 32) {
        // ---- MMA issuer
        int kt = 0;
        for (; kt < nk; ++kt) {
            const int st = kt % S;
            if (!mbar_wait_bounded(&full[st], (kt / S) & 1, MBAR_SPIN_LIMIT) || *(volatile int*)&fail) {
                atomicOr(g.err, 1);
                atomicExch(&fail, 1);
                break;
            }
            fence_after_sync();
            const uint32_t sa = base + st * STAGE;
#pragma unroll
            for (int kk = 0; kk < GEMM_BK / 16; ++kk) {
                // K = 16 BF16 = 32 bytes along the swizzled 128-byte row
                const uint64_t da = smem_desc_sw128(sa + kk * 32);
                const uint64_t db = smem_desc_sw128(sa + TMA_A_BYTES + kk * 32);
                mma_bf16(tmem, da, db, IDESC, (kt | kk) != 0 ? 1u : 0u);
            }
            mma_commit(&empty[st]);
        }
        // arrives when every MMA issued above has completed
        mma_commit(&done);
    }
    __syncwarp();
    // ---- epilogue: all four warps
    const bool ok = mbar_wait_bounded(&done, 0, MBAR_SPIN_LIMIT) && !*(volatile int*)&fail;
    if (!ok && lane == 0) atomicOr(g.err, 1);
    if (threadIdx.x == 0) {
        // loads issued but never consumed: let them land before the CTA exits
        for (int kt = max(0, issued - S); kt < issued; ++kt)
            mbar_wait_bounded(&full[kt % S], (kt / S) & 1, MBAR_SPIN_LIMIT);
    }
    if (__syncthreads_and(ok) && nk > 0) {
        fence_after_sync();
        const int m = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + (uint32_t(warp * 32) << 16);
        if (BN % 64 == 0) {
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 64) {
                float v[64], a[32], b[32];
                tmem_ld64(trow + uint32_t(c0), v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    a[i] = v[i];
                    b[i] = v[32 + i];
                }
                epilogue32(g, g.out_f32, m, n0 + c0, a);
                epilogue32(g, g.out_f32, m, n0 + c0 + 32, b);
            }
        } else {
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(trow + uint32_t(c0), v);
                epilogue16(g, g.out_f32, m, n0 + c0, v);
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
