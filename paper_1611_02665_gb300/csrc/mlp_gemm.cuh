// BF16 tensor-core GEMM for the surrogate network, written for sm_103a's
// fifth-generation tensor cores: C[M,N] = A[M,K] . B[N,K]^T with A and B
// bf16, K contiguous ("K-major"), FP32 accumulation in tensor memory (TMEM).
//
// One CTA computes one 128 x BN output tile (optionally a K slice of it):
//   warp 0 lane 0  TMA producer: 128x64 A and BNx64 B tiles, 128-byte
//                  swizzle, into a ring of STAGES shared-memory slots
//                  (full/empty mbarriers);
//   warp 1         allocates BN TMEM columns; lane 0 issues
//                  tcgen05.mma.cta_group::1.kind::f16 (M=128, N=BN, K=16)
//                  four times per 64-wide K block and commits each slot back
//                  to the producer with tcgen05.commit;
//   warps 0-3      epilogue: tcgen05.ld 32 lanes x 32 columns per warp, a
//                  fused elementwise stage, vectorised global stores.
// Every wait is bounded (2 s); a timeout sets the caller's status word and
// the CTA still releases its TMEM before returning.
//
// The fused epilogues implement the network's layers (see mlp.cu): bias +
// SiLU forward (saving the pre-activation and a transposed copy for the
// weight gradients), the SiLU backward, a split-K FP32 reduction, and the
// forward-mode (value, 3 first, 3 pure second derivative) propagation over 8
// stacked rows per position.
#pragma once

#include "bspline_internal.cuh"

namespace mlpk {

using bsg::mbar_arrive_expect_tx;
using bsg::mbar_init;
using bsg::mbar_try_wait;
using bsg::smem_u32;

constexpr int BM = 128;
constexpr int BK = 64;  // one 128-byte swizzle atom of bf16 along K
constexpr int STAGES = 4;
constexpr int kThreads = 128;

enum Epi {
    EPI_FWD_TRAIN = 0,  // a = silu(acc + b): a bf16 [M][ld0], a^T bf16 [N][ld1], z fp32 [M][ldz]
    EPI_FWD_INFER = 1,  // a = silu(acc + b): a bf16 [M][ld0]
    EPI_LINEAR = 2,     // out = acc + b: fp32 [M][ld0]
    EPI_BWD = 3,        // d = acc * silu'(z): d bf16 [M][ld0], d^T bf16 [N][ld1]; z fp32 [M][ldz] read
    EPI_ATOMIC = 4,     // out += acc: fp32 [M][ld0] (split-K partial sums)
    EPI_FM_HIDDEN = 5,  // forward mode over 8 stacked rows per position: bf16 [M][ld0]
    EPI_FM_OUT = 6,     // forward mode output: v [P][ld0], g [P][3][ld0], l [P][ld0] fp32
};

struct GemmArgs {
    int M, N, K;
    int kblocks_per_split;  // K blocks (of 64) per blockIdx.z
    const float *bias;      // [N] or null
    void *out0;
    int ld0;
    void *out1;
    int ld1;
    float *z;  // pre-activation save (FWD_TRAIN) / read (BWD)
    int ldz;
    float *g;  // EPI_FM_OUT gradients
    float *l;  // EPI_FM_OUT Laplacian
    int *status;
};

// ---- tcgen05 / TMA wrappers ----
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// 32 lanes x 32 consecutive 32-bit columns: thread i of the warp gets lane (base + i).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major bf16 tile written by TMA with
// 128-byte swizzle: 8-row x 128-byte swizzle atoms stacked along M/N every
// 1024 bytes (stride byte offset), version 1, layout type 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);        // start address
    d |= (uint64_t)1 << 16;                        // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset
    d |= (uint64_t)1 << 46;                        // descriptor version
    d |= (uint64_t)2 << 61;                        // swizzle mode: 128 bytes
    return d;
}

// Instruction descriptor: D fp32, A and B bf16, both K-major, M = 128, N = BN.
template <int BN> __host__ __device__ constexpr uint32_t idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

constexpr uint64_t kWaitNs = 2000000000ull;
__device__ __forceinline__ bool wait_bounded(uint64_t *bar, uint32_t parity, int *status) {
    return bsg::mbar_wait_bounded(bar, parity, status);
}

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + __expf(-z)); }

__device__ __forceinline__ void store_bf16x32(__nv_bfloat16 *dst, const float *v) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        __nv_bfloat162 h[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(v[8 * q + 2 * e], v[8 * q + 2 * e + 1]);
        *reinterpret_cast<uint4 *>(dst + 8 * q) = *reinterpret_cast<uint4 *>(h);
    }
}
__device__ __forceinline__ void store_f32x32(float *dst, const float *v) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
        *reinterpret_cast<float4 *>(dst + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
__device__ __forceinline__ void red_add_f32x4(float *dst, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

template <int BN> __host__ __device__ constexpr size_t gemm_smem_bytes() {
    return (size_t)STAGES * (BM * BK * 2 + BN * BK * 2) + 1024 /*align*/ + 256 /*barriers*/;
}

template <int BN, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                     const GemmArgs g) {
    constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sA = base;
    unsigned char *sB = base + (size_t)STAGES * A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + (size_t)STAGES * B_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
    const int kb_total = g.K / BK;
    const int kb_begin = blockIdx.z * g.kblocks_per_split;
    const int kb_end = min(kb_total, kb_begin + g.kblocks_per_split);
    const int nkb = max(0, kb_end - kb_begin);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        bsg::fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(s_tmem, BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp == 0 && lane == 0) {
        int issued = 0;
        for (int i = 0; i < nkb; ++i) {
            const int s = i % STAGES;
            if (i >= STAGES && !wait_bounded(&empty[s], (uint32_t)(((i / STAGES) - 1) & 1), g.status)) break;
            mbar_arrive_expect_tx(&full[s], A_BYTES + B_BYTES);
            const int kc = (kb_begin + i) * BK;
            tma_load_2d(sA + (size_t)s * A_BYTES, &mapA, &full[s], kc, m0);
            tma_load_2d(sB + (size_t)s * B_BYTES, &mapB, &full[s], kc, n0);
            issued = i + 1;
        }
        // every issued load has landed before the CTA may exit
        for (int j = max(0, issued - STAGES); j < issued; ++j)
            if (!wait_bounded(&full[j % STAGES], (uint32_t)((j / STAGES) & 1), g.status)) break;
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_bf16<BN>();
        for (int i = 0; i < nkb; ++i) {
            const int s = i % STAGES;
            if (!wait_bounded(&full[s], (uint32_t)((i / STAGES) & 1), g.status)) break;
            tc_fence_after();
            const uint64_t ad = smem_desc_sw128(smem_u32(sA + (size_t)s * A_BYTES));
            const uint64_t bd = smem_desc_sw128(smem_u32(sB + (size_t)s * B_BYTES));
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)  // +32 bytes along K per step = +2 in the address field
                umma_bf16(tmem, ad + 2 * k, bd + 2 * k, idesc, (i > 0 || k > 0) ? 1u : 0u);
            umma_commit(&empty[s]);
        }
        umma_commit(done);
    }
    __syncwarp();

    // ---------------- epilogue ----------------
    const bool ok = wait_bounded(done, 0, g.status);
    __syncwarp();
    tc_fence_after();
    if (ok && nkb > 0) {
        const int row = warp * 32 + lane;
        const int m = m0 + row;
        const bool live = m < g.M;
        const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tbase + c0, r);
            float acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = __uint_as_float(r[j]);
            const int n = n0 + c0;
            if constexpr (EPI == EPI_FWD_TRAIN || EPI == EPI_FWD_INFER) {
                float a[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float z = acc[j] + g.bias[n + j];
                    acc[j] = z;
                    a[j] = z * sigm(z);
                }
                if (live) {
                    store_bf16x32(static_cast<__nv_bfloat16 *>(g.out0) + (size_t)m * g.ld0 + n, a);
                    if constexpr (EPI == EPI_FWD_TRAIN) store_f32x32(g.z + (size_t)m * g.ldz + n, acc);
                }
                if constexpr (EPI == EPI_FWD_TRAIN) {
                    if (live) {
                        __nv_bfloat16 *t = static_cast<__nv_bfloat16 *>(g.out1) + (size_t)n * g.ld1 + m;
#pragma unroll
                        for (int j = 0; j < 32; ++j) t[(size_t)j * g.ld1] = __float2bfloat16_rn(a[j]);
                    }
                }
            } else if constexpr (EPI == EPI_LINEAR) {
                if (live) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) acc[j] += g.bias ? g.bias[n + j] : 0.f;
                    store_f32x32(static_cast<float *>(g.out0) + (size_t)m * g.ld0 + n, acc);
                }
            } else if constexpr (EPI == EPI_BWD) {
                if (live) {
                    const float *zr = g.z + (size_t)m * g.ldz + n;
                    float d[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float z = zr[j];
                        const float s = sigm(z);
                        d[j] = acc[j] * (s * (1.f + z * (1.f - s)));
                    }
                    store_bf16x32(static_cast<__nv_bfloat16 *>(g.out0) + (size_t)m * g.ld0 + n, d);
                    __nv_bfloat16 *t = static_cast<__nv_bfloat16 *>(g.out1) + (size_t)n * g.ld1 + m;
#pragma unroll
                    for (int j = 0; j < 32; ++j) t[(size_t)j * g.ld1] = __float2bfloat16_rn(d[j]);
                }
            } else if constexpr (EPI == EPI_ATOMIC) {
                if (live) {
                    float *o = static_cast<float *>(g.out0) + (size_t)m * g.ld0 + n;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        red_add_f32x4(o + 4 * q, acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
                }
            } else if constexpr (EPI == EPI_FM_HIDDEN || EPI == EPI_FM_OUT) {
                // Rows are (position, stream) with 8 streams per position in consecutive lanes:
                // 0 value, 1-3 d/dx_d, 4-6 d2/dx_d^2, 7 unused.
                const int s = lane & 7, grp = lane & ~7;
                const int src = (s >= 4 && s <= 6) ? s - 3 : s;
                float o[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float zacc = __shfl_sync(0xffffffffu, acc[j], grp);
                    const float dz = __shfl_sync(0xffffffffu, acc[j], grp + src);
                    if constexpr (EPI == EPI_FM_HIDDEN) {
                        const float z = zacc + g.bias[n + j];
                        const float sg = sigm(z);
                        const float d1 = sg * (1.f + z * (1.f - sg));
                        const float d2 = sg * (1.f - sg) * (2.f + z * (1.f - 2.f * sg));
                        float val;
                        if (s == 0) val = z * sg;
                        else if (s <= 3) val = d1 * acc[j];
                        else if (s <= 6) val = fmaf(d2, dz * dz, d1 * acc[j]);
                        else val = 0.f;
                        o[j] = val;
                    } else {
                        const float l4 = __shfl_sync(0xffffffffu, acc[j], grp + 4);
                        const float l5 = __shfl_sync(0xffffffffu, acc[j], grp + 5);
                        const float l6 = __shfl_sync(0xffffffffu, acc[j], grp + 6);
                        (void)dz;
                        o[j] = s == 0 ? zacc + g.bias[n + j] : (s <= 3 ? acc[j] : l4 + l5 + l6);
                    }
                }
                if (live) {
                    if constexpr (EPI == EPI_FM_HIDDEN) {
                        store_bf16x32(static_cast<__nv_bfloat16 *>(g.out0) + (size_t)m * g.ld0 + n, o);
                    } else {
                        const size_t p = (size_t)(m >> 3);
                        if (s == 0) store_f32x32(static_cast<float *>(g.out0) + p * g.ld0 + n, o);
                        else if (s <= 3) store_f32x32(g.g + (p * 3 + (s - 1)) * g.ld0 + n, o);
                        else if (s == 4) store_f32x32(g.l + p * g.ld0 + n, o);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, BN);
}

}  // namespace mlpk
