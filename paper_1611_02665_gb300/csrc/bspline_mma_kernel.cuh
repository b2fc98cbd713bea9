// Tensor-core evaluation of 16-bit tables (BSPLINE_VARIANT_MMA).
//
// At one position, every output of Eq. (TricubicValue) is a weighted sum over
// the 64 stencil points k = (a, b, c) of the table rows:
//     out_q[n] = f_q * s_n * sum_k W_q[k] * p[k][n],
// where W_q[k] = wx_q[a] wy_q[b] wz_q[c] multiplies the 1-D basis pieces (or
// their t-derivatives) that output q takes along each axis, f_q is its grid
// factor (n_x for d/dx, n_x n_y for d2/dxdy, ...), s_n the orbital's table
// scale and p[k][n] the 16-bit codes. For a block of 128 orbitals that is a
// small matrix product D[128 x outputs] = A[128 x 64] B[64 x outputs], which
// this kernel runs on the tensor cores (tcgen05.mma, kind::f16, FP32
// accumulation in tensor memory).
//
//   A  the unit's 64 stencil rows of 128 orbitals: two TMA boxes {64 orbitals,
//      4, 4, 4} with 128-byte swizzle. Orbital-contiguous rows for consecutive
//      k are the MN-major operand layout, so the boxes are used as loaded.
//   B  the weights, written by the producer warp. Each W_q is split into parts
//      of the table's type whose sum carries 22 (FP16: hi + lo) or 24 (BF16:
//      hi + mid + lo) significant bits; part j fills rows 16j..16j+15 (K-major,
//      128-byte swizzle). 16-bit x 16-bit products are exact in FP32, so the
//      sums differ from the FP32 FMA path only in rounding order.
//   D  FP32 in tensor memory, a ring of accumulators (256 columns per CTA:
//      8 for FP16, 4 for BF16), so the epilogues of earlier units overlap
//      the MMAs of later ones.
//
// Work unit = (position, 128-orbital block); persistent CTAs take positions
// round-robin and run their blocks in turn. Warp roles: warp 0 builds the weights (all lanes) and issues
// the TMA boxes (lane 0) into a ring of `stages` slots; warp 1 owns the
// tensor memory and lane 0 issues four K=16 MMAs per unit; warps 2-5 read the
// accumulator (one TMEM lane quarter each: thread = orbital), add the parts,
// scale and stream the outputs out. Every wait is bounded (2 s): a timeout
// sets the table's status word, the roles stop, in-flight copies and MMAs are
// waited for (bounded), and the tensor memory is freed before the CTA exits.
#pragma once

#include "bspline_internal.cuh"
#include "tcgen05_ptx.cuh"

namespace bsg {

constexpr int kMmaM = 128;                   // orbitals per unit (MMA M)
constexpr int kMmaThreads = 192;             // producer, MMA, 4 epilogue warps
constexpr uint32_t kMmaBoxBytes = 64u * 128u;  // one box: 64 rows x 64 orbitals x 2 bytes

template <typename T> constexpr int mma_parts() { return Elem<T>::dtype == BSPLINE_F16 ? 2 : 3; }
template <typename T> constexpr int mma_ncols() { return 16 * mma_parts<T>(); }
template <typename T> constexpr int mma_acc_cols() { return mma_ncols<T>() <= 32 ? 32 : 64; }
// Accumulators per CTA: 256 tensor-memory columns, so two CTAs fill an SM's 512.
template <typename T> constexpr int mma_nacc() { return 256 / mma_acc_cols<T>(); }
template <typename T> constexpr uint32_t mma_b_bytes() { return (uint32_t)mma_ncols<T>() * 128u; }
constexpr uint32_t kMmaStageBytes = 2 * kMmaBoxBytes;  // one unit's A tile
// Weight slots: enough positions to cover `stages` units (nmblk units per
// position), at least 2, at most `stages`.
inline int mma_wslots(int stages, int nmblk) {
    const int w = (stages + nmblk - 1) / nmblk + 1;
    return w < 2 ? 2 : (w > stages ? stages : w);
}
// Ratio sums (bspline_eval_ratio on this variant): per-quarter partial sums of
// up to 10 components, double-buffered, and their full / free barriers.
constexpr size_t kMmaRedBytes = 2 * 10 * 4 * sizeof(float) + 4 * 8;
// ub: orbital blocks per unit (a ring slot holds ub blocks, an accumulator ub blocks' columns).
template <typename T> inline size_t mma_smem_bytes(int stages, int nmblk, int ub = 1) {
    const int w = mma_wslots(stages, (nmblk + ub - 1) / ub);
    return 1024 + (size_t)stages * ub * kMmaStageBytes + (size_t)w * mma_b_bytes<T>() +
           (size_t)(2 * stages + 2 * mma_nacc<T>() + w) * 8 + 16 + kMmaRedBytes;
}

// Instruction descriptor: D fp32, A and B of the table's type, A MN-major
// (transposed), B K-major, M = 128, N = ncols.
template <typename T> __host__ __device__ constexpr uint32_t mma_idesc() {
    constexpr uint32_t ab = Elem<T>::dtype == BSPLINE_BF16 ? 1u : 0u;
    return (1u << 4) | (ab << 7) | (ab << 10) | (1u << 15) | ((uint32_t)(mma_ncols<T>() >> 3) << 17) |
           ((uint32_t)(kMmaM >> 4) << 24);
}

// Per-axis derivative orders of the outputs of KIND (the Laplacian row of VGL
// is assembled separately).
__device__ __forceinline__ void mma_orders(int q, int &ox, int &oy, int &oz) {
    constexpr int tab[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                                {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
    ox = tab[q][0];
    oy = tab[q][1];
    oz = tab[q][2];
}

// w[base + i] for a lane-dependent i in 0..3, by selects (no local-memory array).
__device__ __forceinline__ float pick4(const float (&w)[12], int base, int i) {
    return i == 0 ? w[base] : (i == 1 ? w[base + 1] : (i == 2 ? w[base + 2] : w[base + 3]));
}

template <typename T> __device__ __forceinline__ uint32_t mma_pack(float lo_k, float hi_k);
template <> __device__ __forceinline__ uint32_t mma_pack<__half>(float a, float b) {
    return (uint32_t)__half_as_ushort(__float2half_rn(a)) | ((uint32_t)__half_as_ushort(__float2half_rn(b)) << 16);
}
template <> __device__ __forceinline__ uint32_t mma_pack<__nv_bfloat16>(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}
template <typename T> __device__ __forceinline__ float mma_round(float w);
template <> __device__ __forceinline__ float mma_round<__half>(float w) { return __half2float(__float2half_rn(w)); }
template <> __device__ __forceinline__ float mma_round<__nv_bfloat16>(float w) {
    return __bfloat162float(__float2bfloat16_rn(w));
}

// Writes the weight parts of output row q for stencil points k0 = 2*lane and
// k0 + 1 into the K-major, 128-byte-swizzled B tile: element (row, k) sits at
// (row / 8) * 1024 + (row % 8) * 128 + ((k / 8) ^ (row % 8)) * 16 + (k % 8) * 2.
template <typename T>
__device__ __forceinline__ void mma_put_row(unsigned char *sB, int q, int lane, float w0, float w1) {
    constexpr int P = mma_parts<T>();
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const float h0 = mma_round<T>(w0), h1 = mma_round<T>(w1);
        const int row = 16 * j + q;
        const uint32_t off = (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * 128u +
                             ((uint32_t)((lane >> 2) ^ (row & 7)) << 4) + (uint32_t)(lane & 3) * 4u;
        *reinterpret_cast<uint32_t *>(sB + off) = mma_pack<T>(h0, h1);
        w0 -= h0;  // exact: the rounding residue of a 16-bit rounding is representable in FP32
        w1 -= h1;
    }
}

// Builds the B tile of one position (rows of KIND, all parts) from its cell
// offsets; called by the 32 lanes of the producer warp.
template <int KIND, typename T>
__device__ __forceinline__ void mma_build_weights(const EvalArgs &A, unsigned char *sB, int lane, float tx, float ty,
                                                  float tz) {
    constexpr int NO = nout_of(KIND);
    float wx[12], wy[12], wz[12];
    basis_weights(tx, 1.f, wx);
    basis_weights(ty, 1.f, wy);
    basis_weights(tz, 1.f, wz);
    // this lane's stencil points k = 2*lane, 2*lane + 1: a = k / 16, b = (k / 4) % 4, c = k % 4;
    // px[o] = o-th derivative piece of axis x at a (likewise y at b, z at c0 and c0 + 1)
    const int a = lane >> 3, b = (lane >> 1) & 3, c0 = (lane & 1) * 2;
    float px[3], py[3], pz0[3], pz1[3];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        px[o] = pick4(wx, 4 * o, a);
        py[o] = pick4(wy, 4 * o, b);
        pz0[o] = pick4(wz, 4 * o, c0);
        pz1[o] = pick4(wz, 4 * o, c0 + 1);
    }
    constexpr int NW = KIND == BSPLINE_VGL ? 4 : NO;  // rows that are one product of pieces
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        int ox, oy, oz;
        mma_orders(q, ox, oy, oz);
        const float wab = px[ox] * py[oy];
        mma_put_row<T>(sB, q, lane, wab * pz0[oz], wab * pz1[oz]);
    }
    if constexpr (KIND == BSPLINE_VGL) {
        // Laplacian row: sum over axes of n_d^2 times the pure second derivative, over S = max n_d^2
        const float nx2 = (float)A.nx * A.nx, ny2 = (float)A.ny * A.ny, nz2 = (float)A.nz * A.nz;
        const float inv = 1.f / fmaxf(nx2, fmaxf(ny2, nz2));
        const float lx = nx2 * inv, ly = ny2 * inv, lz = nz2 * inv;
        const float l0 = lx * px[2] * py[0] * pz0[0] + ly * px[0] * py[2] * pz0[0] + lz * px[0] * py[0] * pz0[2];
        const float l1 = lx * px[2] * py[0] * pz1[0] + ly * px[0] * py[2] * pz1[0] + lz * px[0] * py[0] * pz1[2];
        mma_put_row<T>(sB, 4, lane, l0, l1);
    }
}

// Grid factor of each output of KIND: n_d per first derivative, n_a n_b per
// second derivative, max n_d^2 for the normalised Laplacian row.
template <int KIND> __device__ __forceinline__ void mma_output_factors(const EvalArgs &A, float (&fq)[nout_of(KIND)]) {
    fq[0] = 1.f;
    if constexpr (KIND != BSPLINE_V) {
        const float n3[3] = {(float)A.nx, (float)A.ny, (float)A.nz};
        fq[1] = n3[0];
        fq[2] = n3[1];
        fq[3] = n3[2];
        if constexpr (KIND == BSPLINE_VGL) {
            fq[4] = fmaxf(n3[0] * n3[0], fmaxf(n3[1] * n3[1], n3[2] * n3[2]));
        } else {
#pragma unroll
            for (int q = 4; q < 10; ++q) {
                int ox, oy, oz;
                mma_orders(q, ox, oy, oz);
                float f = 1.f;
                for (int r = 0; r < ox; ++r) f *= n3[0];
                for (int r = 0; r < oy; ++r) f *= n3[1];
                for (int r = 0; r < oz; ++r) f *= n3[2];
                fq[q] = f;
            }
        }
    }
}

// Streaming stores of one orbital's outputs at one position.
template <int KIND>
__device__ __forceinline__ void mma_store(const EvalArgs &A, long long pos, int n, const float (&out)[nout_of(KIND)]) {
    const long long ld = A.ld;
    __stcs(A.o0 + pos * ld + n, out[0]);
    if constexpr (KIND != BSPLINE_V) {
#pragma unroll
        for (int d = 0; d < 3; ++d) __stcs(A.o1 + (pos * 3 + d) * ld + n, out[1 + d]);
    }
    if constexpr (KIND == BSPLINE_VGL) __stcs(A.o2 + pos * ld + n, out[4]);
    if constexpr (KIND == BSPLINE_VGH) {
#pragma unroll
        for (int d = 0; d < 6; ++d) __stcs(A.o2 + (pos * 6 + d) * ld + n, out[4 + d]);
    }
}

// Two CTAs per SM (ctas_per_sm = 2) must fit the register file: 2 blocks.
// LAT: general cell. Positions are Cartesian (reduced through u = r G), the
// tensor cores form the fractional derivatives of acc_kind (VGL takes the VGH
// set: the Laplacian mixes all six), and the epilogue turns them Cartesian.
// RAT: determinant-ratio sums instead of per-orbital outputs (Sec. "QMC and
// B-spline-based SPOs": sum_n phi_n(r) A^-1(n,e), and the same over the
// derivatives): each thread multiplies its orbital's components by
// u_n = uinv[pos*ldu + n] and keeps running sums over the position's blocks;
// at the position's last block the four epilogue warps reduce them in a fixed
// order (warp shuffles, then the quarters 0..3 through shared memory) and
// ratio[pos*nout + q] receives component q's sum.
// UB: orbital blocks per work unit (1 or 2). A unit of two blocks takes one ring slot of two table tiles and
// one accumulator of twice the columns, so every hand-off between the three roles covers 256 orbitals.
template <int KIND, typename T, bool LAT, bool RAT, int UB = 1>
__global__ void __launch_bounds__(kMmaThreads, 2)
    eval_mma_kernel(const __grid_constant__ CUtensorMap map, const EvalArgs A, int nmblk, int stages, int wslots,
                    const float *__restrict__ uinv, int ldu, float *__restrict__ ratio) {
    pdl_wait();
    pdl_trigger();
    constexpr int AK = acc_kind<KIND, LAT>();
    constexpr int NO = nout_of(AK);
    constexpr int P = mma_parts<T>();
    constexpr int ACC = mma_acc_cols<T>();
    constexpr int NACC = mma_nacc<T>() / UB;  // accumulators of UB * ACC columns
    constexpr uint32_t SB = UB * kMmaStageBytes;
    const int nunit = (nmblk + UB - 1) / UB;
    constexpr uint32_t BB = mma_b_bytes<T>();
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *wbase = base + (size_t)stages * SB;  // weight slots
    uint64_t *full = reinterpret_cast<uint64_t *>(wbase + (size_t)wslots * BB);
    uint64_t *empty = full + stages;
    uint64_t *tfull = empty + stages;
    uint64_t *tempty = tfull + NACC;
    uint64_t *wfree = tempty + NACC;
    uint64_t *redfull = wfree + wslots;  // [2] partial sums of a position written (4 arrivals)
    uint64_t *redfree = redfull + 2;     // [2] partial sums read (1 arrival)
    float *red = reinterpret_cast<float *>(redfree + 2);  // [2][10][4]
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(red + 2 * 10 * 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NACC; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        for (int w = 0; w < wslots; ++w) mbar_init(&wfree[w], 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&redfull[b], 4);
            mbar_init(&redfree[b], 1);
        }
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(s_tmem, NACC * UB * ACC);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    // Work order: each CTA takes position slots p = blockIdx.x, + gridDim.x, ...
    // and for each the nmblk orbital blocks in turn (unit counter it). The
    // weights of a position are built once, into weight slot (position
    // counter ip) % wslots, after the MMA lane has released that slot (its
    // commit to wfree after the last unit of the slot's previous position).
    const int G = gridDim.x;
    const int npos = A.npos;

    if (warp == 0) {
        // ---- producer: weights (all lanes), TMA boxes (lane 0) ----
        // Positions are fetched and reduced to cells 32 slots at a time (lane j
        // takes slot pb + j * G), so their load latency is paid once per 32
        // positions; each position then takes its cell from lane j.
        long long it = 0, ip = 0;
        bool ok = true;
        for (int pb = blockIdx.x; pb < npos && ok; pb += 32 * G) {
            const long long sj = pb + (long long)lane * G;
            int cj[3] = {0, 0, 0};
            float tj[3] = {0.f, 0.f, 0.f};
            if (sj < npos) {
                const long long pos = A.perm ? A.perm[sj] : sj;
                cell_reduce(LAT ? frac_coord(A, pos, 0) : A.x[pos], A.nx, cj[0], tj[0]);
                cell_reduce(LAT ? frac_coord(A, pos, 1) : A.y[pos], A.ny, cj[1], tj[1]);
                cell_reduce(LAT ? frac_coord(A, pos, 2) : A.z[pos], A.nz, cj[2], tj[2]);
            }
            const int nb = min(32, (npos - pb + G - 1) / G);
            for (int j = 0; j < nb && ok; ++j, ++ip) {
                const int ix = __shfl_sync(0xffffffffu, cj[0], j), iy = __shfl_sync(0xffffffffu, cj[1], j),
                          iz = __shfl_sync(0xffffffffu, cj[2], j);
                const float tx = __shfl_sync(0xffffffffu, tj[0], j), ty = __shfl_sync(0xffffffffu, tj[1], j),
                            tz = __shfl_sync(0xffffffffu, tj[2], j);
                const int ws = (int)(ip % wslots);
                unsigned char *sB = wbase + (size_t)ws * BB;
                for (int ub = 0; ub < nunit; ++ub, ++it) {
                    const int s = (int)(it % stages);
                    const uint32_t eph = (uint32_t)(((it / stages) - 1) & 1);
                    if (it >= stages && !__all_sync(0xffffffffu, mbar_wait_bounded(&empty[s], eph, A.status))) {
                        ok = false;
                        break;
                    }
                    if (ub == 0) {
                        const uint32_t wph = (uint32_t)(((ip / wslots) - 1) & 1);
                        if (ip >= wslots && !__all_sync(0xffffffffu, mbar_wait_bounded(&wfree[ws], wph, A.status))) {
                            ok = false;
                            break;
                        }
                        mma_build_weights<AK, T>(A, sB, lane, tx, ty, tz);
                        fence_proxy_async_smem();
                        __syncwarp();
                    }
                    if (lane == 0) {
                        unsigned char *sA = base + (size_t)s * SB;
                        // the unit's blocks; the upper half of a ragged last block stays unloaded, and so does a
                        // missing last block of the position
                        uint32_t bytes = 0;
#pragma unroll
                        for (int b = 0; b < UB; ++b) {
                            const int o0 = (ub * UB + b) * kMmaM;
                            if (o0 < A.Npad) bytes += o0 + 64 < A.Npad ? 2 * kMmaBoxBytes : kMmaBoxBytes;
                        }
                        mbar_arrive_expect_tx(&full[s], bytes);
#pragma unroll
                        for (int b = 0; b < UB; ++b) {
                            const int o0 = (ub * UB + b) * kMmaM;
                            if (o0 >= A.Npad) break;
                            unsigned char *dst = sA + (size_t)b * kMmaStageBytes;
                            tma_load_4d(dst, &map, &full[s], o0, iz, iy, ix);
                            if (o0 + 64 < A.Npad) tma_load_4d(dst + kMmaBoxBytes, &map, &full[s], o0 + 64, iz, iy, ix);
                        }
                    }
                }
            }
        }
        // every box this CTA issued has landed before the CTA may exit
        if (lane == 0)
            for (long long j = it > stages ? it - stages : 0; j < it; ++j)
                if (!mbar_wait_bounded(&full[j % stages], (uint32_t)((j / stages) & 1), A.status)) break;
    } else if (warp == 1) {
        // ---- MMA issue (lane 0) ----
        if (lane == 0) {
            constexpr uint32_t idesc = mma_idesc<T>();
            long long it = 0, ip = 0;
            bool ok = true;
            for (int p = blockIdx.x; p < npos && ok; p += G, ++ip) {
                const int ws = (int)(ip % wslots);
                const uint32_t b0 = smem_u32(wbase + (size_t)ws * BB);
                for (int ub = 0; ub < nunit; ++ub, ++it) {
                    const int s = (int)(it % stages);
                    const int acc = (int)(it % NACC);
                    const uint32_t tph = (uint32_t)(((it / NACC) - 1) & 1);
                    if (!mbar_wait_bounded(&full[s], (uint32_t)((it / stages) & 1), A.status) ||
                        (it >= NACC && !mbar_wait_bounded(&tempty[acc], tph, A.status))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int b = 0; b < UB; ++b) {
                        if (ub * UB + b >= nmblk) break;
                        const uint32_t a0 = smem_u32(base + (size_t)s * SB + (size_t)b * kMmaStageBytes);
                        const uint32_t d = tmem + (uint32_t)((acc * UB + b) * ACC);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks)  // K = 16 per MMA: 16 rows of A (2048 bytes), 32 bytes of B rows
                            umma_f16(d, smem_desc_sw128_mn(a0 + ks * 2048u, kMmaBoxBytes, 1024u),
                                     smem_desc_sw128(b0 + ks * 32u), idesc, ks > 0 ? 1u : 0u);
                    }
                    umma_commit(&empty[s]);
                    umma_commit(&tfull[acc]);
                    if (ub == nunit - 1) umma_commit(&wfree[ws]);  // the position's weights are no longer read
                }
            }
            // the last MMAs have finished before the tensor memory may be freed
            if (it > 0) mbar_wait_bounded(&tfull[(it - 1) % NACC], (uint32_t)(((it - 1) / NACC) & 1), A.status);
        }
        __syncwarp();
    } else {
        // ---- epilogue: thread = orbital (TMEM lane), one lane quarter per warp ----
        const int quarter = warp & 3;
        float fq[NO];
        mma_output_factors<AK>(A, fq);
        // The orbital scale depends on the block only; the next unit's scale is
        // loaded while this unit is processed, so its latency stays hidden.
        auto scale_of = [&](int mb) {
            const int n = mb * kMmaM + quarter * 32 + lane;
            return n < A.N ? A.scale[n] : 0.f;
        };
        float sc_next = scale_of(0);
        constexpr int NK = nout_of(KIND);
        float part[NK];  // RAT: running sums of the position's components
        long long it = 0, ip = 0;
        bool ok = true;
        for (int pb = blockIdx.x; pb < npos && ok; pb += 32 * G) {
            // output positions of 32 slots at a time (lane j: slot pb + j * G)
            const long long sj = pb + (long long)lane * G;
            const int posj = sj < npos ? (A.perm ? A.perm[sj] : (int)sj) : 0;
            const int nb = min(32, (npos - pb + G - 1) / G);
            // RAT: this thread's u_n of the next unit, loaded one unit ahead (like the scale)
            auto u_of = [&](long long p, int mb) {
                const int n = mb * kMmaM + quarter * 32 + lane;
                return n < A.N ? uinv[p * (long long)ldu + n] : 0.f;
            };
            float u_next = 0.f;
            if constexpr (RAT) u_next = u_of(__shfl_sync(0xffffffffu, posj, 0), 0);
            for (int j = 0; j < nb && ok; ++j, ++ip) {
                const long long pos = __shfl_sync(0xffffffffu, posj, j);
                const long long pos_after = __shfl_sync(0xffffffffu, posj, j + 1 < nb ? j + 1 : j);
                if constexpr (RAT) {
#pragma unroll
                    for (int q = 0; q < NK; ++q) part[q] = 0.f;
                    // u of the next position comes from DRAM: start its row toward L2 a position early
                    if (j + 1 < nb)
                        for (int n = quarter * 32 + lane; n < A.N; n += kMmaM)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(uinv + pos_after * (long long)ldu + n));
                }
                for (int ub = 0; ub < nunit; ++ub, ++it) {
                    const int acc = (int)(it % NACC);
                    const uint32_t fph = (uint32_t)((it / NACC) & 1);
                    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&tfull[acc], fph, A.status))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int b = 0; b < UB; ++b) {
                        const int mb = ub * UB + b;
                        if (mb >= nmblk) break;
                        const int n = mb * kMmaM + quarter * 32 + lane;
                        const float sc = sc_next;
                        sc_next = scale_of(mb + 1 < nmblk ? mb + 1 : 0);
                        float u_cur = 0.f;
                        if constexpr (RAT) {
                            u_cur = u_next;
                            if (mb + 1 < nmblk) u_next = u_of(pos, mb + 1);
                            else if (j + 1 < nb) u_next = u_of(pos_after, 0);
                        }
                        const uint32_t taddr =
                            tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((acc * UB + b) * ACC);
                        uint32_t r[32];
                        tmem_ld32(taddr, r);
                        uint32_t r3[16];
                        if constexpr (P == 3) tmem_ld16(taddr + 32, r3);
                        if (b == UB - 1 || mb + 1 >= nmblk) {  // the unit's accumulator is read: hand it back
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&tempty[acc]);
                        }
                        if (n < A.N) {
                            float out[NO];
#pragma unroll
                            for (int q = 0; q < NO; ++q) {
                                float v = __uint_as_float(r[16 + q]);
                                if constexpr (P == 3) v += __uint_as_float(r3[q]);
                                v += __uint_as_float(r[q]);
                                out[q] = v * fq[q] * sc;
                            }
                            float oc[NK];
                            if constexpr (LAT) {
                                float in1[NO][1], outc[NK][1];
#pragma unroll
                                for (int q = 0; q < NO; ++q) in1[q][0] = out[q];
                                to_cartesian<KIND, 1>(A, in1, outc);
#pragma unroll
                                for (int q = 0; q < NK; ++q) oc[q] = outc[q][0];
                            } else {
#pragma unroll
                                for (int q = 0; q < NK; ++q) oc[q] = out[q];
                            }
                            if constexpr (RAT) {
#pragma unroll
                                for (int q = 0; q < NK; ++q) part[q] = fmaf(oc[q], u_cur, part[q]);
                            } else {
                                mma_store<KIND>(A, pos, n, oc);
                            }
                        }
                    }
                }
                if constexpr (RAT) {
                    if (!ok) break;
                    // fixed-order reduction: the warp's 32 orbitals by shuffles, then quarters 0..3
                    const int b = (int)(ip & 1);
                    const uint32_t use = (uint32_t)(ip >> 1);
                    float *rb = red + b * 40;
#pragma unroll
                    for (int q = 0; q < NK; ++q) {
                        float v = part[q];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        part[q] = v;
                    }
                    if (ip >= 2 && !__all_sync(0xffffffffu, mbar_wait_bounded(&redfree[b], (use - 1) & 1, A.status))) {
                        ok = false;
                        break;
                    }
                    if (lane < NK) {
                        float v = part[0];
#pragma unroll
                        for (int q = 1; q < NK; ++q)
                            if (lane == q) v = part[q];
                        rb[lane * 4 + quarter] = v;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&redfull[b]);
                    if (warp == 2) {  // the reader: adds the quarters in order and writes the sums
                        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&redfull[b], use & 1, A.status))) {
                            ok = false;
                            break;
                        }
                        if (lane < NK)
                            ratio[pos * NK + lane] =
                                ((rb[lane * 4] + rb[lane * 4 + 1]) + rb[lane * 4 + 2]) + rb[lane * 4 + 3];
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&redfree[b]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, NACC * UB * ACC);
}

// Persistent launch: ctas_per_sm CTAs on every SM (at most one per position), units of nb / 128 orbital
// blocks (nb = 128 or 256). ratio non-null: the ratio sums of bspline_eval_ratio (uinv, ldu) instead of
// per-orbital outputs.
template <int KIND, typename T, bool LAT>
static bspline_status launch_mma(const EvalArgs &A, const CUtensorMap *map, int nb, int stages, int ctas_per_sm,
                                 int num_sms, cudaStream_t s, const float *uinv = nullptr, int ldu = 0,
                                 float *ratio = nullptr) {
    if constexpr (sizeof(T) != 2) {
        return BSPLINE_ERR_UNSUPPORTED;
    } else {
        if (!map || (nb != kMmaM && nb != 2 * kMmaM)) return BSPLINE_ERR_ARG;
        const int ub = nb / kMmaM;
        const int nmblk = (A.Npad + kMmaM - 1) / kMmaM;
        const long long want = (long long)num_sms * ctas_per_sm;
        const int grid = (int)(A.npos < want ? A.npos : want);
        const size_t smem = mma_smem_bytes<T>(stages, nmblk, ub);
        using Kern = void (*)(CUtensorMap, EvalArgs, int, int, int, const float *, int, float *);
        Kern kern = ub == 2 ? (ratio ? eval_mma_kernel<KIND, T, LAT, true, 2> : eval_mma_kernel<KIND, T, LAT, false, 2>)
                            : (ratio ? eval_mma_kernel<KIND, T, LAT, true, 1> : eval_mma_kernel<KIND, T, LAT, false, 1>);
        static bool attr_set[4] = {false, false, false, false};  // idempotent; a race only repeats the call
        const int ak = (ratio ? 1 : 0) + 2 * (ub - 1);
        if (!attr_set[ak]) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
            if (e != cudaSuccess) return cuda_status(e);
            attr_set[ak] = true;
        }
        return cuda_status(launch_k(kern, grid, kMmaThreads, smem, s, true, *map, A, nmblk, stages,
                                    mma_wslots(stages, (nmblk + ub - 1) / ub), uinv, ldu, ratio));
    }
}

}  // namespace bsg
