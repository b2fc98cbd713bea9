// BF16 tensor-core GEMM for the surrogate network, written for sm_103a's
// fifth-generation tensor cores: C[M,N] = A[M,K] . B[N,K]^T with A and B
// bf16, K contiguous ("K-major"), FP32 accumulation in tensor memory (TMEM).
//
// Persistent: each CTA walks 128 x BN output tiles (optionally K slices of
// them) round-robin. Warp roles:
//   warp 0 lane 0  TMA producer: 128x64 A and BNx64 B tiles, 128-byte
//                  swizzle, into a ring of shared-memory slots (gemm_stages)
//                  (full/empty mbarriers), continuously across tiles;
//   warp 1         allocates 2*BN TMEM columns (two accumulators); lane 0
//                  issues tcgen05.mma.cta_group::1.kind::f16 (M=128, N=BN,
//                  K=16) four times per 64-wide K block, frees each slot with
//                  tcgen05.commit, and hands a finished accumulator to the
//                  epilogue with another commit;
//   warps 2-17     epilogue: four warps per TMEM lane quarter, each reading
//                  a quarter of the BN columns with tcgen05.ld (32 lanes x 16
//                  columns), releasing the accumulator after its last load,
//                  then a fused elementwise stage and either a TMA store of
//                  the chunk staged in shared memory (single-output
//                  epilogues) or vectorised stores from registers.
// The epilogue of one tile overlaps the MMAs of the next. Every wait is
// bounded (2 s); a timeout sets the caller's status word and the CTA still
// releases its TMEM before returning.
//
// The fused epilogues implement the network's layers (see mlp.cu): bias +
// SiLU forward (saving the pre-activation and a transposed copy for the
// weight gradients), the SiLU backward, a split-K FP32 reduction, and the
// forward-mode propagation of value, gradient and Laplacian over 5 rows per
// position (fm_row).
//
// gemm_pair_kernel (end of the file) runs the same roles on clusters of two
// CTAs with tcgen05 cta_group::2 MMAs on 256 x 256 tiles.
#pragma once

#include "bspline_internal.cuh"
#include "tcgen05_ptx.cuh"

namespace mlpk {

using bsg::mbar_arrive_expect_tx;
using bsg::mbar_init;
using bsg::mbar_try_wait;
using bsg::smem_u32;

constexpr int BM = 128;
constexpr int BK = 64;  // one 128-byte swizzle atom of bf16 along K
constexpr int STAGES = 4;  // operand ring depth, except where gemm_stages says otherwise
constexpr int kEpiWarps = 16;  // 4 per TMEM lane quarter
constexpr int CW = 16;         // accumulator columns per tcgen05.ld
constexpr int kThreads = 64 + 32 * kEpiWarps;

enum Epi {
    EPI_FWD_TRAIN = 0,  // a = silu(acc + b): a bf16 [M][ld0], a^T bf16 [N][ld1], z fp32 [M][ldz]
    EPI_FWD_INFER = 1,  // a = silu(acc + b): a bf16 [M][ld0]
    EPI_LINEAR = 2,     // out = acc + b: fp32 [M][ld0]
    EPI_BWD = 3,        // d = acc * silu'(z): d bf16 [M][ld0], d^T bf16 [N][ld1]; z fp32 [M][ldz] read
    EPI_ATOMIC = 4,     // out += acc: fp32 [M][ld0] (split-K partial sums)
    EPI_FM_HIDDEN = 5,  // forward mode over 5 rows per position (fm_row): bf16 [M][ld0]
    EPI_FM_OUT = 6,     // forward mode output: v [P][ld0], g [P][3][ld0], l [P][ld0] fp32
    // training on values and gradients: 4 rows per position (vg_row: value, d/dx_d), tangents carry no bias
    EPI_VG_HIDDEN = 7,  // value a = silu(z), tangent a_d = silu'(z) z_d: bf16 [M][ld0] and [N][ld1]; z / z_d fp32 [M][ldz]
    EPI_VG_OUT = 8,     // value acc + b, tangent acc: fp32 [M][ld0]
    EPI_VG_BWD = 9,     // value dz = silu'(z) da + silu''(z) sum_d z_d da_d, tangent dz_d = silu'(z) da_d:
                        // bf16 [M][ld0] and [N][ld1]; z / z_d fp32 [M][ldz] read
};

struct GemmArgs {
    int M, N, K;
    int kblocks_per_split;  // K blocks (of 64) per K slice
    int splits;             // K slices per output tile
    const float *bias;      // [N] or null
    void *out0;
    int ld0;
    void *out1;
    int ld1;
    float *z;  // pre-activation save (FWD_TRAIN) / read (BWD)
    int ldz;
    float *g;  // EPI_FM_OUT gradients
    float *l;  // EPI_FM_OUT Laplacian
    int npos;  // EPI_FM_OUT positions
    int *status;
};

// Forward-mode row layout: every 32 rows hold 6 positions of 5 consecutive
// rows each - 0 value, 1-3 d/dx_d, 4 Laplacian - and two unused rows (30, 31),
// so a position never straddles a warp's 32 TMEM lanes. The Laplacian row
// carries sum_d d2/dx_d^2 directly: the pre-activation's Laplacian is linear in
// the previous layer's (W applied to it), and silu adds
// silu''(z) |grad z|^2 + silu'(z) lap z, which needs only the gradient rows.
constexpr int kFmStreams = 5, kFmPerWarp = 6;
__host__ __device__ constexpr long long fm_rows(long long npos) { return 32 * ((npos + kFmPerWarp - 1) / kFmPerWarp); }
__host__ __device__ constexpr long long fm_row(long long p, int stream) {
    return 32 * (p / kFmPerWarp) + kFmStreams * (p % kFmPerWarp) + stream;
}

// Training layout on values and gradients: position p owns the 4 consecutive rows 4p + s, s = 0 the value,
// s = 1..3 its derivative along axis s - 1, so a warp's 32 rows hold 8 whole positions.
constexpr int kVgStreams = 4;
__host__ __device__ constexpr long long vg_row(long long p, int stream) { return kVgStreams * p + stream; }

// ---- tcgen05 / TMA wrappers (tcgen05_ptx.cuh) ----
using bsg::smem_desc_sw128;
using bsg::tc_fence_after;
using bsg::tc_fence_before;
using bsg::tma_load_2d;
using bsg::tmem_alloc;
using bsg::tmem_dealloc;
using bsg::tmem_ld16;
using bsg::tmem_ld16_async;
using bsg::tmem_ld32;
using bsg::tmem_relinquish;
using bsg::tmem_wait16;
using bsg::umma_commit;

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    bsg::umma_f16(tmem_d, adesc, bdesc, idesc, accumulate);
}

// Instruction descriptor: D fp32, A and B bf16, both K-major, M x BN (M = 128 for one CTA, 256 for a pair).
template <int BN, int M = BM> __host__ __device__ constexpr uint32_t idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

constexpr uint64_t kWaitNs = 2000000000ull;
__device__ __forceinline__ bool wait_bounded(uint64_t *bar, uint32_t parity, int *status) {
    return bsg::mbar_wait_bounded(bar, parity, status);
}

// Logistic function through the hardware tanh: sigma(z) = (1 + tanh(z/2)) / 2.
// tanh.approx.f32 is accurate to about 2^-11, below the bfloat16 rounding the
// activations get next.
__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sigm(float z) { return fmaf(0.5f, tanh_approx(0.5f * z), 0.5f); }

// SiLU of two pre-activations with packed FP32 instructions: with h = z/2 (exact),
// silu(z) = z sigma(z) = h (1 + tanh h), one fused multiply-add after the tanh.
using bsg::f32x2;
__device__ __forceinline__ f32x2 silu2(f32x2 z) {
    const f32x2 h = bsg::mul2(z, bsg::pack2(0.5f, 0.5f));
    float h0, h1;
    bsg::unpack2(h, h0, h1);
    return bsg::fma2(h, bsg::pack2(tanh_approx(h0), tanh_approx(h1)), h);
}

// 16 bf16 values per lane (lane = row m of the warp's 32 rows, the warp's
// columns n..n+15), stored cooperatively: lanes trade halves through
// shuffles so that each store instruction writes whole 32-byte sectors of 16
// rows (lanes 2r and 2r+1 hold the two 16-byte halves of row r) instead of
// 16-byte halves of 32 rows. Every lane of the warp must call it; live says
// whether the calling lane's row exists.
__device__ __forceinline__ void store_bf16xCW_rows(__nv_bfloat16 *out, int ld, int m, int n, const float *v,
                                                   bool live, int lane) {
    static_assert(CW == 16, "two 16-byte halves per row");
    uint32_t pk[CW / 2];
#pragma unroll
    for (int w = 0; w < CW / 2; ++w) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * w], v[2 * w + 1]);
        pk[w] = *reinterpret_cast<const uint32_t *>(&h);
    }
    const int row0 = m - lane, half = lane & 1;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int src = (lane >> 1) + 16 * i;
        uint32_t o[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const uint32_t lo = __shfl_sync(0xffffffffu, pk[w], src), hi = __shfl_sync(0xffffffffu, pk[4 + w], src);
            o[w] = half ? hi : lo;
        }
        if (__shfl_sync(0xffffffffu, live ? 1 : 0, src)) {
            uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)(row0 + src) * ld + n + 8 * half);
            *dst = make_uint4(o[0], o[1], o[2], o[3]);
        }
    }
}

// 16 floats per lane stored cooperatively: dst is the calling lane's
// destination (its row, column n) or null if it stores nothing. Lanes trade
// values through shuffles so that each store instruction writes one whole
// 32-byte sector of each of 16 rows (lanes 2r and 2r+1 hold its halves).
// Every lane of the warp must call it.
__device__ __forceinline__ void store_f32xCW_coop(float *dst, const float *v, int lane) {
    static_assert(CW == 16, "two 32-byte sectors per row");
    const int half = lane & 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int src = (lane >> 1) + 16 * (i & 1), sector = i >> 1;
        float o[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const float lo = __shfl_sync(0xffffffffu, v[8 * sector + w], src);
            const float hi = __shfl_sync(0xffffffffu, v[8 * sector + 4 + w], src);
            o[w] = half ? hi : lo;
        }
        float *d = reinterpret_cast<float *>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(dst), src));
        if (d) *reinterpret_cast<float4 *>(d + 8 * sector + 4 * half) = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// As store_f32xCW_coop for a row-major matrix (row m = this lane's row of the
// warp's 32, column n): each lane computes the destinations of the rows it
// stores instead of receiving them, which saves the pointer shuffles. Rows at
// or past M are not stored.
__device__ __forceinline__ void store_f32xCW_rows(float *out, int ld, int m, int n, int M, const float *v,
                                                  int lane) {
    static_assert(CW == 16, "two 32-byte sectors per row");
    const int half = lane & 1, row0 = m - lane;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int src = (lane >> 1) + 16 * (i & 1), sector = i >> 1;
        float o[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const float lo = __shfl_sync(0xffffffffu, v[8 * sector + w], src);
            const float hi = __shfl_sync(0xffffffffu, v[8 * sector + 4 + w], src);
            o[w] = half ? hi : lo;
        }
        if (row0 + src < M)
            *reinterpret_cast<float4 *>(out + (size_t)(row0 + src) * ld + n + 8 * sector + 4 * half) =
                make_float4(o[0], o[1], o[2], o[3]);
    }
}

__device__ __forceinline__ void red_add_f32x4(float *dst, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// Epilogues whose output is one row-major matrix leave through TMA stores: each epilogue warp stages
// its 32 rows x CW columns in shared memory, in the output tensor map's box layout, and one lane stores
// the box. Row ends and rows past M are the tensor map's to clip. The other epilogues store from
// registers (several outputs, transposed copies, scattered rows or reductions).
template <int EPI> constexpr bool epi_tma_store() {
    return EPI == EPI_FWD_INFER || EPI == EPI_LINEAR || EPI == EPI_FM_HIDDEN;
}
template <int EPI> constexpr int epi_out_bytes() { return EPI == EPI_LINEAR ? 4 : 2; }
// staging boxes per epilogue warp: two for bf16, so that the next chunk is written while the last one is
// stored; one for fp32, which keeps the 4-slot operand ring within shared memory (measured on the 65,536 x
// 512 x 512 output layer: 39.6 us, against 42.3 us with two boxes and a 3-slot ring)
template <int EPI> constexpr int epi_stage_bufs() { return epi_tma_store<EPI>() ? (epi_out_bytes<EPI>() == 2 ? 2 : 1) : 0; }
constexpr int kStageRows = 32;
template <int EPI> constexpr uint32_t epi_stage_bytes() { return (uint32_t)(kStageRows * CW * epi_out_bytes<EPI>()); }

// Operand ring depth (slots of one 64-wide K block of A and B).
template <int BN, int EPI> __host__ __device__ constexpr int gemm_stages() { return STAGES; }
// Shared memory of a CTA with NST operand slots, EW epilogue warps and NBUF staging boxes per warp.
template <int BN, int EPI, int EW, int NST, int NBUF> __host__ __device__ constexpr size_t gemm_smem_bytes_of() {
    return (size_t)NST * (BM * BK * 2 + BN * BK * 2) + 1024 /*align*/ + 1024 /*barriers*/ +
           (size_t)EW * NBUF * epi_stage_bytes<EPI>();
}
template <int BN, int EPI> __host__ __device__ constexpr size_t gemm_smem_bytes() {
    return gemm_smem_bytes_of<BN, EPI, kEpiWarps, gemm_stages<BN, EPI>(), epi_stage_bufs<EPI>()>();
}

// Two CTAs per SM (gemm_bf16_kernel<128, EPI, kEpiWarps2, ...>, 2): 128 x 128 tiles, 8 epilogue warps, one
// staging box per warp, and the deepest operand ring (3 or 2 slots) with which two CTAs fit in an SM's
// 228 KB of shared memory (each CTA also takes 1 KB of it).
constexpr int kEpiWarps2 = 8;
template <int EPI> constexpr int two_cta_bufs() { return epi_stage_bufs<EPI>() < 1 ? epi_stage_bufs<EPI>() : 1; }
template <int EPI> constexpr bool two_cta_fit(int nst) {
    return 2 * ((nst == 3 ? gemm_smem_bytes_of<128, EPI, kEpiWarps2, 3, two_cta_bufs<EPI>()>()
                          : gemm_smem_bytes_of<128, EPI, kEpiWarps2, 2, two_cta_bufs<EPI>()>()) + 1024) <= 233472;
}
template <int EPI> constexpr int two_cta_stages() { return two_cta_fit<EPI>(3) ? 3 : 2; }
static_assert(gemm_smem_bytes<256, EPI_LINEAR>() <= 232448 && gemm_smem_bytes<256, EPI_FWD_INFER>() <= 232448 &&
                  gemm_smem_bytes<256, EPI_FWD_TRAIN>() <= 232448,
              "shared memory per CTA");

// One row of a staged box (this lane's row r of the warp's 32), in the layouts the output tensor maps
// declare. bf16: a row is 32 bytes, two 16-byte halves, with the 32-byte swizzle (address bit 4 ^= bit 7:
// half h of row r sits at h ^ bit 2 of r). fp32: a row is 64 bytes, four 16-byte quarters, with the
// 64-byte swizzle (bits 4-5 ^= bits 7-8: quarter q of row r sits at q ^ bits 1-2 of r). Either way the
// 8 rows one shared-memory wavefront serves land in 8 different 16-byte bank groups.
__device__ __forceinline__ void stage_bf16_row(unsigned char *box, int r, const float *v) {
    static_assert(CW == 16, "two 16-byte halves per row");
    uint32_t pk[CW / 2];
#pragma unroll
    for (int w = 0; w < CW / 2; ++w) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * w], v[2 * w + 1]);
        pk[w] = *reinterpret_cast<const uint32_t *>(&h);
    }
    uint4 *row = reinterpret_cast<uint4 *>(box + r * 32);
    const int x = (r >> 2) & 1;
    row[x] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    row[1 ^ x] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}
__device__ __forceinline__ void stage_f32_row(unsigned char *box, int r, const float *v) {
    static_assert(CW == 16, "four 16-byte quarters per row");
    float4 *row = reinterpret_cast<float4 *>(box + r * 64);
    const int x = (r >> 1) & 3;
#pragma unroll
    for (int q = 0; q < 4; ++q) row[q ^ x] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// Bias values of CW consecutive columns (vector loads; every lane reads the same addresses).
__device__ __forceinline__ void load_bias(const float *bias, int n, float (&b)[CW]) {
#pragma unroll
    for (int q = 0; q < CW / 4; ++q) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(bias + n) + q);
        b[4 * q] = v.x;
        b[4 * q + 1] = v.y;
        b[4 * q + 2] = v.z;
        b[4 * q + 3] = v.w;
    }
}

__device__ __forceinline__ void load_bias_or_zero(const float *bias, int n, float (&b)[CW]) {
    if (bias) {
        load_bias(bias, n, b);
    } else {
#pragma unroll
        for (int j = 0; j < CW; ++j) b[j] = 0.f;
    }
}

// Fused elementwise stage for CW consecutive columns n..n+CW-1 of row m (this
// thread's TMEM lane). acc holds the FP32 accumulators.
template <int EPI> constexpr bool epi_uses_bias() {
    return EPI == EPI_FWD_TRAIN || EPI == EPI_FWD_INFER || EPI == EPI_LINEAR || EPI == EPI_FM_HIDDEN ||
           EPI == EPI_FM_OUT || EPI == EPI_VG_HIDDEN || EPI == EPI_VG_OUT;
}

// Transposed bf16 copy of this lane's CW values: t[(n + j) * ld1 + m].
__device__ __forceinline__ void store_bf16xCW_transposed(void *out1, int ld1, int m, int n, const float *v) {
    __nv_bfloat16 *t = static_cast<__nv_bfloat16 *>(out1) + (size_t)n * ld1 + m;
#pragma unroll
    for (int j = 0; j < CW; ++j) t[(size_t)j * ld1] = __float2bfloat16_rn(v[j]);
}

// box: this warp's staging box for the epilogues that store through TMA (epi_tma_store), else unused.
template <int EPI>
__device__ __forceinline__ void epilogue_chunk(const GemmArgs &g, float (&acc)[CW], const float (&bb)[CW], int m,
                                               int n, bool live, int lane, unsigned char *box) {
    if constexpr (EPI == EPI_FWD_TRAIN || EPI == EPI_FWD_INFER) {
        float a[CW];
#pragma unroll
        for (int j = 0; j < CW; j += 2) {
            const f32x2 z = bsg::add2(bsg::pack2(acc[j], acc[j + 1]), bsg::pack2(bb[j], bb[j + 1]));
            bsg::unpack2(z, acc[j], acc[j + 1]);
            bsg::unpack2(silu2(z), a[j], a[j + 1]);
        }
        if constexpr (EPI == EPI_FWD_INFER) {
            stage_bf16_row(box, lane, a);
        } else {
            store_bf16xCW_rows(static_cast<__nv_bfloat16 *>(g.out0), g.ld0, m, n, a, live, lane);
            store_f32xCW_rows(g.z, g.ldz, m, n, g.M, acc, lane);
            if (live) {
                __nv_bfloat16 *t = static_cast<__nv_bfloat16 *>(g.out1) + (size_t)n * g.ld1 + m;
#pragma unroll
                for (int j = 0; j < CW; ++j) t[(size_t)j * g.ld1] = __float2bfloat16_rn(a[j]);
            }
        }
    } else if constexpr (EPI == EPI_LINEAR) {
#pragma unroll
        for (int j = 0; j < CW; j += 2)
            bsg::unpack2(bsg::add2(bsg::pack2(acc[j], acc[j + 1]), bsg::pack2(bb[j], bb[j + 1])), acc[j], acc[j + 1]);
        stage_f32_row(box, lane, acc);
    } else if constexpr (EPI == EPI_BWD) {
        float d[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) d[j] = 0.f;
        if (live) {
            const float *zr = g.z + (size_t)m * g.ldz + n;
#pragma unroll
            for (int q = 0; q < CW / 4; ++q) {
                const float4 z4 = *reinterpret_cast<const float4 *>(zr + 4 * q);
                const float zz[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float s = sigm(zz[e]);
                    d[4 * q + e] = acc[4 * q + e] * (s * fmaf(zz[e], 1.f - s, 1.f));
                }
            }
        }
        store_bf16xCW_rows(static_cast<__nv_bfloat16 *>(g.out0), g.ld0, m, n, d, live, lane);
        if (live) {
            __nv_bfloat16 *t = static_cast<__nv_bfloat16 *>(g.out1) + (size_t)n * g.ld1 + m;
#pragma unroll
            for (int j = 0; j < CW; ++j) t[(size_t)j * g.ld1] = __float2bfloat16_rn(d[j]);
        }
    } else if constexpr (EPI == EPI_ATOMIC) {
        if (live) {
            float *o = static_cast<float *>(g.out0) + (size_t)m * g.ld0 + n;
#pragma unroll
            for (int q = 0; q < CW / 4; ++q)
                red_add_f32x4(o + 4 * q, acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
    } else if constexpr (EPI == EPI_VG_HIDDEN || EPI == EPI_VG_OUT) {
        // row m = this lane: stream s of position m / 4; the value lane of the group is lane & ~3
        const int s = lane & 3, grp = lane & ~3;
        float o[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) {
            if constexpr (EPI == EPI_VG_HIDDEN) {
                const float z = __shfl_sync(0xffffffffu, acc[j], grp) + bb[j];
                const float sg = sigm(z);
                const float d1 = sg * fmaf(z, 1.f - sg, 1.f);
                o[j] = s == 0 ? z * sg : d1 * acc[j];
                acc[j] = s == 0 ? z : acc[j];  // saved for the backward pass: z, or the tangent z_d
            } else {
                o[j] = s == 0 ? acc[j] + bb[j] : acc[j];
            }
        }
        if constexpr (EPI == EPI_VG_HIDDEN) {
            store_bf16xCW_rows(static_cast<__nv_bfloat16 *>(g.out0), g.ld0, m, n, o, live, lane);
            store_f32xCW_rows(g.z, g.ldz, m, n, g.M, acc, lane);
            if (live) store_bf16xCW_transposed(g.out1, g.ld1, m, n, o);
        } else {
            store_f32xCW_rows(static_cast<float *>(g.out0), g.ld0, m, n, g.M, o, lane);
        }
    } else if constexpr (EPI == EPI_VG_BWD) {
        // acc = (dz_next W) for this row: da (value) or da_d (tangent). zown: this row's saved z or z_d.
        const int s = lane & 3, grp = lane & ~3;
        float zown[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) zown[j] = 0.f;
        if (live) {
            const float *zr = g.z + (size_t)m * g.ldz + n;
#pragma unroll
            for (int q = 0; q < CW / 4; ++q) {
                const float4 z4 = *reinterpret_cast<const float4 *>(zr + 4 * q);
                zown[4 * q] = z4.x, zown[4 * q + 1] = z4.y, zown[4 * q + 2] = z4.z, zown[4 * q + 3] = z4.w;
            }
        }
        float d[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) {
            const float z = __shfl_sync(0xffffffffu, zown[j], grp);
            const float tj = s == 0 ? 0.f : zown[j] * acc[j];  // z_d da_d on the tangent lanes
            const float tsum = __shfl_sync(0xffffffffu, tj, grp + 1) + __shfl_sync(0xffffffffu, tj, grp + 2) +
                               __shfl_sync(0xffffffffu, tj, grp + 3);
            const float sg = sigm(z);
            const float om = 1.f - sg;
            const float d1 = sg * fmaf(z, om, 1.f);
            const float d2 = sg * om * fmaf(z, 1.f - 2.f * sg, 2.f);
            d[j] = s == 0 ? fmaf(d2, tsum, d1 * acc[j]) : d1 * acc[j];
        }
        store_bf16xCW_rows(static_cast<__nv_bfloat16 *>(g.out0), g.ld0, m, n, d, live, lane);
        if (live) store_bf16xCW_transposed(g.out1, g.ld1, m, n, d);
    } else if constexpr (EPI == EPI_FM_HIDDEN || EPI == EPI_FM_OUT) {
        // Row m = this lane of the warp's 32 rows (m & 31 == lane): stream s of position 6 (m >> 5) + q
        // (fm_row); lanes 30 and 31 are unused and stay 0.
        const bool pad = lane >= kFmStreams * kFmPerWarp;
        const int q = pad ? 0 : lane / kFmStreams, s = pad ? 0 : lane - kFmStreams * q, grp = kFmStreams * q;
        // lane-uniform selectors keep the per-element work free of branches
        const bool isv = s == 0, isl = s == 4;
        float o[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) {
            const float zacc = __shfl_sync(0xffffffffu, acc[j], grp);
            if constexpr (EPI == EPI_FM_HIDDEN) {
                // value: silu(z); d/dx_d: silu'(z) dz_d; Laplacian: silu''(z) |grad z|^2 + silu'(z) lap z
                const float g1 = __shfl_sync(0xffffffffu, acc[j], grp + 1);
                const float g2 = __shfl_sync(0xffffffffu, acc[j], grp + 2);
                const float g3 = __shfl_sync(0xffffffffu, acc[j], grp + 3);
                const float z = zacc + bb[j];
                const float sg = sigm(z);
                const float om = 1.f - sg;
                const float d1 = sg * fmaf(z, om, 1.f);
                const float d2 = sg * om * fmaf(z, 1.f - 2.f * sg, 2.f);
                const float gg = fmaf(g1, g1, fmaf(g2, g2, g3 * g3));
                const float t = fmaf(isl ? d2 : 0.f, gg, d1 * acc[j]);
                o[j] = pad ? 0.f : (isv ? z * sg : t);
            } else {
                o[j] = isv ? zacc + bb[j] : acc[j];
            }
        }
        if constexpr (EPI == EPI_FM_HIDDEN) {
            stage_bf16_row(box, lane, o);
        } else {
            const long long p = (long long)(m >> 5) * kFmPerWarp + q;
            float *dst = nullptr;
            if (live && !pad && p < g.npos) {
                if (s == 0) dst = static_cast<float *>(g.out0) + (size_t)p * g.ld0 + n;
                else if (s <= 3) dst = g.g + ((size_t)p * 3 + (s - 1)) * g.ld0 + n;
                else dst = g.l + (size_t)p * g.ld0 + n;
            }
            store_f32xCW_coop(dst, o, lane);
        }
    }
}

// One accumulator tile's epilogue in one epilogue warp: TMEM lane quarter warp % 4, column quarter
// (epilogue warp) / 4 of the 128 x BN accumulator buf, output rows from m0 and columns from n0; release()
// (called by lane 0) hands the accumulator back to the MMA issuer once read. stg: this warp's staging boxes
// (NBUF of them, TMA-store epilogues), sc: the chunks it has staged so far.
// PW epilogue warps per TMEM lane quarter, each taking BN / PW of the tile's columns.
template <int BN, int EPI, int NBUF, class Release, int PW = kEpiWarps / 4>
__device__ __forceinline__ void epilogue_tile(const GemmArgs &g, const CUtensorMap *mapC, uint32_t tmem, int buf,
                                              unsigned char *stg, int &sc, int warp, int lane, int m0, int n0,
                                              Release release) {
    constexpr bool TS = epi_tma_store<EPI>();
    static_assert(!TS || NBUF >= 1, "staging boxes");
    constexpr uint32_t SB = epi_stage_bytes<EPI>();
    constexpr int COLS = BN / PW;
    const int quarter = warp & 3, part = (warp - 2) >> 2;
    const int m = m0 + quarter * 32 + lane;
    const bool live = m < g.M;
    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN + part * COLS);
    const int nbase = n0 + part * COLS;
    const int row0 = m0 + quarter * 32;  // the warp's first row: the staged box's row coordinate
    // One chunk of CW columns: its accumulator registers r (already waited for) and bias b.
    auto process = [&](uint32_t(&r)[CW], const float(&b)[CW], int c) {
        float acc[CW];
#pragma unroll
        for (int j2 = 0; j2 < CW; ++j2) acc[j2] = __uint_as_float(r[j2]);
        unsigned char *box = nullptr;
        if constexpr (TS) {
            // the store that last read this box (NBUF chunks ago) must have finished reading it
            box = stg + (size_t)(sc % NBUF) * SB;
            if (lane == 0) bsg::bulk_wait_group_read<NBUF - 1>();
            __syncwarp();
        }
        epilogue_chunk<EPI>(g, acc, b, m, nbase + c, live, lane, box);
        if constexpr (TS) {
            bsg::fence_proxy_async_smem();  // each lane's box writes, visible to the TMA unit
            __syncwarp();
            if (lane == 0 && row0 < g.M) {
                bsg::tma_store_2d(mapC, box, nbase + c, row0);
                bsg::bulk_commit_group();
            }
            ++sc;
        }
    };
    auto fetch = [&](uint32_t(&r)[CW], float(&b)[CW], int c) {
        tmem_ld16_async(taddr + c, r);
        if constexpr (epi_uses_bias<EPI>()) load_bias_or_zero(g.bias, nbase + c, b);
    };
    auto hand_back = [&]() {  // accumulator fully read: hand it back to the MMA issuer
        tc_fence_before();
        __syncwarp();
        if (lane == 0) release(buf);
    };
    // software pipeline over two register sets (no copies between them): the next chunk's accumulator
    // and bias are in flight while a chunk is processed
    static_assert(COLS % (2 * CW) == 0, "chunks in pairs");
    uint32_t r0[CW], r1[CW];
    float b0[CW], b1[CW];
    fetch(r0, b0, 0);
    tmem_wait16(r0);
#pragma unroll
    for (int c = 0; c < COLS; c += 2 * CW) {
        fetch(r1, b1, c + CW);
        process(r0, b0, c);
        tmem_wait16(r1);
        if (c + 2 * CW < COLS) fetch(r0, b0, c + 2 * CW);
        else hand_back();
        process(r1, b1, c + CW);
        if (c + 2 * CW < COLS) tmem_wait16(r0);
    }
}

// The epilogue warps of the single-GEMM kernels: tiles t0, t0 + tstep, ... < total alternate between the two
// accumulators (tfull[buf] says one is ready); decode(t, m0, n0, kb0, nkb) gives a tile's origin and row_off
// this CTA's first row in it.
template <int BN, int EPI, int NBUF, class Decode, class Release, int PW = kEpiWarps / 4>
__device__ __forceinline__ void epilogue_warps(const GemmArgs &g, const CUtensorMap *mapC, uint32_t tmem,
                                               uint64_t *tfull, unsigned char *staging, int warp, int lane, int t0,
                                               int tstep, int total, int row_off, Decode decode, Release release) {
    constexpr bool TS = epi_tma_store<EPI>();
    unsigned char *stg = staging + (size_t)(warp - 2) * NBUF * epi_stage_bytes<EPI>();
    int sc = 0;
    int local = 0;
    for (int t = t0; t < total; t += tstep, ++local) {
        int m0, n0, kb0, nkb;
        decode(t, m0, n0, kb0, nkb);
        const int buf = local & 1, use = local >> 1;
        if (!__all_sync(0xffffffffu, wait_bounded(&tfull[buf], (uint32_t)(use & 1), g.status))) break;
        tc_fence_after();
        epilogue_tile<BN, EPI, NBUF, Release, PW>(g, mapC, tmem, buf, stg, sc, warp, lane, m0 + row_off, n0,
                                                  release);
    }
    if constexpr (TS) {
        if (lane == 0) bsg::bulk_wait_group<0>();  // stores complete before the boxes go away
    }
}

// mapC: the output's tensor map (box CW x 32, epi_tma_store epilogues only; not read otherwise).
// EW epilogue warps (4 per TMEM lane quarter by default), NSTX operand slots (0: gemm_stages), NBMAX staging
// boxes per warp at most, MINB CTAs per SM.
template <int BN, int EPI, int EW = kEpiWarps, int NSTX = 0, int NBMAX = 2, int MINB = 1>
__global__ void __launch_bounds__(64 + 32 * EW, MINB)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                     const __grid_constant__ CUtensorMap mapC, const GemmArgs g) {
    static_assert(EW % 4 == 0 && BN % (EW / 4) == 0, "epilogue warps per lane quarter");
    constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    constexpr int NST = NSTX ? NSTX : gemm_stages<BN, EPI>();
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sA = base;
    unsigned char *sB = base + (size_t)NST * A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + (size_t)NST * B_BYTES);
    uint64_t *empty = full + NST;
    uint64_t *tfull = empty + NST;  // accumulator ready for the epilogue
    uint64_t *tempty = tfull + 2;      // accumulator drained by the epilogue
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(tempty + 2);
    // staging boxes: 1024 bytes past the barriers, so every box starts on a 1024-byte boundary
    unsigned char *staging = sB + (size_t)NST * B_BYTES + 1024;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_n = g.N / BN, tiles_m = (g.M + BM - 1) / BM;
    const int total = tiles_n * tiles_m * g.splits;
    const int kb_total = g.K / BK;

    bsg::pdl_trigger();  // the next kernel may take up free SM room now; it waits for this one to complete
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EW);
        }
        bsg::fence_mbar_init();
    }
    // The barriers are set up while the previous kernel in the stream drains; its outputs (this GEMM's
    // operands) are read only after it has completed. Tensor memory is allocated after the wait too, so a
    // waiting CTA never holds columns that a still-running kernel on the same SM may need.
    bsg::pdl_wait();
    if (warp == 1) {
        tmem_alloc(s_tmem, 2 * BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    // tile t -> (m block, n block, K slice); consecutive tiles share the A rows
    auto decode = [&](int t, int &m0, int &n0, int &kb0, int &nkb) {
        const int ks = t % g.splits;
        const int r = t / g.splits;
        n0 = (r % tiles_n) * BN;
        m0 = (r / tiles_n) * BM;
        kb0 = ks * g.kblocks_per_split;
        nkb = min(g.kblocks_per_split, kb_total - kb0);
    };

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                int m0, n0, kb0, nkb;
                decode(t, m0, n0, kb0, nkb);
                for (int i = 0; i < nkb; ++i, ++it) {
                    const int s = it % NST;
                    if (it >= NST && !wait_bounded(&empty[s], (uint32_t)(((it / NST) - 1) & 1), g.status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], A_BYTES + B_BYTES);
                    const int kc = (kb0 + i) * BK;
                    tma_load_2d(sA + (size_t)s * A_BYTES, &mapA, &full[s], kc, m0);
                    tma_load_2d(sB + (size_t)s * B_BYTES, &mapB, &full[s], kc, n0);
                }
            }
            // every issued load has landed before the CTA may exit
            for (int j2 = max(0, it - NST); j2 < it; ++j2)
                if (!wait_bounded(&full[j2 % NST], (uint32_t)((j2 / NST) & 1), g.status)) break;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16<BN>();
            int it = 0, local = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++local) {
                int m0, n0, kb0, nkb;
                decode(t, m0, n0, kb0, nkb);
                const int buf = local & 1, use = local >> 1;
                if (use >= 1 && !wait_bounded(&tempty[buf], (uint32_t)((use - 1) & 1), g.status)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * BN);
                for (int i = 0; i < nkb; ++i, ++it) {
                    const int s = it % NST;
                    if (!wait_bounded(&full[s], (uint32_t)((it / NST) & 1), g.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = smem_desc_sw128(smem_u32(sA + (size_t)s * A_BYTES));
                    const uint64_t bd = smem_desc_sw128(smem_u32(sB + (size_t)s * B_BYTES));
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)  // +32 bytes along K per step = +2 in the address field
                        umma_bf16(d, ad + 2 * k, bd + 2 * k, idesc, (i > 0 || k > 0) ? 1u : 0u);
                    umma_commit(&empty[s]);
                }
                umma_commit(&tfull[buf]);
            }
        }
    } else {
        constexpr int NB = epi_stage_bufs<EPI>() < NBMAX ? epi_stage_bufs<EPI>() : NBMAX;
        constexpr int NBUF = epi_tma_store<EPI>() ? NB : 1;
        auto release = [&](int buf) { bsg::mbar_arrive(&tempty[buf]); };
        epilogue_warps<BN, EPI, NBUF, decltype(decode), decltype(release), EW / 4>(
            g, &mapC, tmem, tfull, staging, warp, lane, (int)blockIdx.x, (int)gridDim.x, total, 0, decode, release);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, 2 * BN);
}

// ---------------------------------------------------------------------------
// CTA-pair GEMM (tcgen05 cta_group::2): a cluster of two CTAs computes a 256 x 256 output tile. Each CTA loads
// its own 128 rows of A and its half (128 rows) of the 256-row B tile; the even CTA issues M = 256, N = 256
// MMAs that read both CTAs' shared memory, and each CTA's tensor memory receives its 128 x 256 accumulator.
// Against one CTA's 128 x 256 tile this halves the B operand each SM streams from L2 (32 KB per 64-wide K
// block instead of 48 KB) and leaves the shared memory for a deeper operand ring. Roles as in
// gemm_bf16_kernel: the producers of both CTAs count their loads on the even CTA's full barrier, the even
// CTA's MMA commits free the slots of both CTAs and hand the accumulators to both CTAs' epilogues, whose
// warps all release them on the even CTA's barrier.
// ---------------------------------------------------------------------------
constexpr int kPairBN = 256;
// operand ring depth and staging boxes per warp, filling 226 KB of shared memory
template <int EPI> constexpr int pair_stages() {
    return !epi_tma_store<EPI>() ? 7 : (epi_out_bytes<EPI>() == 4 ? 5 : 6);
}
template <int EPI> constexpr int pair_stage_bufs() { return epi_tma_store<EPI>() ? 2 : 1; }
template <int EPI> __host__ __device__ constexpr size_t pair_smem_bytes() {
    return (size_t)pair_stages<EPI>() * (BM * BK * 2 + (kPairBN / 2) * BK * 2) + 1024 /*align*/ + 1024 /*barriers*/ +
           (epi_tma_store<EPI>() ? (size_t)kEpiWarps * pair_stage_bufs<EPI>() * epi_stage_bytes<EPI>() : 0);
}
static_assert(pair_smem_bytes<EPI_LINEAR>() <= 232448 && pair_smem_bytes<EPI_FWD_INFER>() <= 232448 &&
                  pair_smem_bytes<EPI_FWD_TRAIN>() <= 232448,
              "shared memory per CTA");

template <int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_pair_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                     const __grid_constant__ CUtensorMap mapC, const GemmArgs g) {
    constexpr int BN = kPairBN, BNH = BN / 2;
    constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BNH * BK * 2;
    constexpr int NST = pair_stages<EPI>();
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sA = base;
    unsigned char *sB = base + (size_t)NST * A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + (size_t)NST * B_BYTES);  // used in the even CTA
    uint64_t *empty = full + NST;
    uint64_t *tfull = empty + NST;
    uint64_t *tempty = tfull + 2;  // used in the even CTA
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(tempty + 2);
    unsigned char *staging = sB + (size_t)NST * B_BYTES + 1024;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = bsg::cluster_ctarank();
    const bool leader = rank == 0;
    const int pair = (int)blockIdx.x >> 1, npairs = (int)gridDim.x >> 1;
    const int tiles_n = g.N / BN, tiles_m = (g.M + 2 * BM - 1) / (2 * BM);
    const int total = tiles_n * tiles_m;
    const int kb_total = g.K / BK;

    bsg::pdl_trigger();
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 2 * kEpiWarps);
        }
        bsg::fence_mbar_init();
    }
    bsg::cluster_sync();  // both CTAs' barriers exist before either CTA signals the other's
    bsg::pdl_wait();
    if (warp == 1) {
        bsg::tmem_alloc_pair(s_tmem, 2 * BN);
        bsg::tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    auto decode = [&](int t, int &m0, int &n0, int &kb0, int &nkb) {
        n0 = (t % tiles_n) * BN;
        m0 = (t / tiles_n) * (2 * BM);
        kb0 = 0;
        nkb = kb_total;
    };

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int t = pair; t < total && ok; t += npairs) {
                int m0, n0, kb0, nkb;
                decode(t, m0, n0, kb0, nkb);
                for (int i = 0; i < nkb; ++i, ++it) {
                    const int s = it % NST;
                    if (it >= NST && !wait_bounded(&empty[s], (uint32_t)(((it / NST) - 1) & 1), g.status)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fbar = bsg::mapa_shared(smem_u32(&full[s]), 0);
                    if (leader) mbar_arrive_expect_tx(&full[s], 2 * (A_BYTES + B_BYTES));
                    const int kc = (kb0 + i) * BK;
                    bsg::tma_load_2d_pair(sA + (size_t)s * A_BYTES, &mapA, fbar, kc, m0 + (int)rank * BM);
                    bsg::tma_load_2d_pair(sB + (size_t)s * B_BYTES, &mapB, fbar, kc, n0 + (int)rank * BNH);
                }
            }
            // the even CTA sees every load of both CTAs land; the odd CTA's loads are covered by it and by the
            // cluster barrier before exit
            if (leader)
                for (int j2 = max(0, it - NST); j2 < it; ++j2)
                    if (!wait_bounded(&full[j2 % NST], (uint32_t)((j2 / NST) & 1), g.status)) break;
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            constexpr uint32_t idesc = idesc_bf16<BN, 2 * BM>();
            int it = 0, local = 0;
            bool ok = true;
            for (int t = pair; t < total && ok; t += npairs, ++local) {
                int m0, n0, kb0, nkb;
                decode(t, m0, n0, kb0, nkb);
                const int buf = local & 1, use = local >> 1;
                if (use >= 1 && !wait_bounded(&tempty[buf], (uint32_t)((use - 1) & 1), g.status)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * BN);
                for (int i = 0; i < nkb; ++i, ++it) {
                    const int s = it % NST;
                    if (!wait_bounded(&full[s], (uint32_t)((it / NST) & 1), g.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = smem_desc_sw128(smem_u32(sA + (size_t)s * A_BYTES));
                    const uint64_t bd = smem_desc_sw128(smem_u32(sB + (size_t)s * B_BYTES));
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)
                        bsg::umma_f16_pair(d, ad + 2 * k, bd + 2 * k, idesc, (i > 0 || k > 0) ? 1u : 0u);
                    bsg::umma_commit_pair(&empty[s], 0x3);
                }
                bsg::umma_commit_pair(&tfull[buf], 0x3);
            }
        }
    } else {
        epilogue_warps<BN, EPI, pair_stage_bufs<EPI>()>(
            g, &mapC, tmem, tfull, staging, warp, lane, pair, npairs, total, (int)rank * BM, decode,
            [&](int buf) { bsg::mbar_arrive_cluster(bsg::mapa_shared(smem_u32(&tempty[buf]), 0)); });
    }
    tc_fence_before();
    bsg::cluster_sync();  // neither CTA leaves while the other may still read its operands or signal it
    if (warp == 1) bsg::tmem_dealloc_pair(tmem, 2 * BN);
}

}  // namespace mlpk
