// Single-table evaluation kernels (V / VGL / VGH), templated on the stored
// element type. Included once per element type by bspline_eval_<type>.cu.
//
// Two launch shapes, both reading the padded table [nx+3][ny+3][nz+3][Npad]
// with orbitals innermost (the paper's P[Nx][Ny][Nz][N] with the row padding
// of Sec. "Baseline and miniQMC"):
//
//  DIRECT  One CTA per (group of ppc positions, block of NT*VEC orbitals).
//          Three threads reduce the positions to cells and weights in double
//          precision and publish them in shared memory; every thread then
//          owns VEC consecutive orbitals and streams the 64 stencil rows
//          straight from global memory with 128-bit (or 64-bit) loads, 16
//          rows in flight per x-plane.
//
//  TMA     Persistent CTAs, one producer warp and NBOX/32 consumer warps.
//          Per work item (position, block of NBOX orbitals) the producer lane
//          computes the cell and the 36 weights and issues ONE 4-D TMA box
//          {NBOX, 4, 4, 4} - the whole 64-row stencil slice - into a ring of
//          `stages` shared-memory slots guarded by mbarriers. Consumers take
//          one orbital per thread from shared memory.
//
// Both use the factorised z -> y -> x accumulation of accumulate().
#pragma once

#include "bspline_internal.cuh"
#include "bspline_mma_kernel.cuh"

namespace bsg {

constexpr int kMaxPpc = 8;
// Positions one DIRECT CTA holds weights for (several position groups when N
// is small, see eval_direct_kernel).
constexpr int kMaxCtaPos = 32;

// Where the arithmetic runs on packed pairs (accumulate_x2; identical results). Measured with every
// variant built both ways (outputs bitwise equal; 16^3 x 64 table at 16384 positions, 48^3 x 2048 at 4096,
// 48 x 48 x 60 x 128 at 65536):
//  - 16-bit tables, VGL and VGH: packed. Their DIRECT kernels are bound by instruction issue (a
//    conversion per element on top of the FMAs): FP16 VGH 27.9 -> 22.1 us, VGL 21.6 -> 19.6 us at 16384
//    positions; 48 x 48 x 60 x 128 VGH 230 -> 198 us; 48^3 x 2048 VGH 179 -> 173 us.
//  - 16-bit V: scalar (packed: 11.7 -> 14.0 us; its loads, not its 84 FMAs per orbital, set the pace).
//  - FP32, rows staged through the ring, VGH and VGL: packed in the plain layout (48^3 x 2048, 4096
//    sorted positions: VGH 216 -> 212 us, VGL 182 -> 177 us; 64^3 x 4096 VGL 840 -> 822 us; the batched
//    kernel's ring uses the same choice), scalar in the grouped one (48 x 48 x 60 x 128 VGH: 162 -> 169
//    us packed). FP32 V: scalar (packed was slower everywhere measured).
// The packed grouped kernels need more registers: VGH asks for 384 resident threads per SM (168
// registers; at 128 it spilled 288 bytes and took 24.8 instead of 22.1 us), VGL for 512 (19.6 against
// 20.7 us at 384).
template <typename T, int KIND> constexpr bool packed_direct() { return sizeof(T) == 2 && KIND != BSPLINE_V; }
template <int KIND> constexpr bool packed_staged_plain() { return KIND != BSPLINE_V; }
template <int KIND> constexpr int packed_grp_threads() { return KIND == BSPLINE_VGH ? 384 : 512; }
// The 16-unit ring of small launches (one CTA per SM, so registers are no constraint): packed for VGH
// (1024 positions of the 16^3 x 64 table, replayed from a graph: 4.08 -> 3.51 us; V and VGL unchanged).
template <int KIND> constexpr bool packed_small() { return KIND == BSPLINE_VGH; }

// CTAs per SM the DIRECT kernel asks registers for, as resident threads per
// SM (measured at 48^3 x 2048, 4096 sorted positions): 640 threads (VGH at 96
// registers, 20 warps, no spills) for 16-bit tables and for V, whose loads
// need more warps to cover their latency (FP16 VGH 0.253 -> 0.205 ms, FP32 V
// 0.227 -> 0.184 ms); 512 threads (128 registers) for FP32 VGH and VGL, which
// are faster with more loads in flight per thread (0.247 ms, against 0.274 ms
// at 640 threads and 0.328 ms at 256 threads / 242 registers).
template <int KIND, typename T, int NT> constexpr int direct_min_blocks() {
    return ((sizeof(T) == 2 || KIND == BSPLINE_V) ? 640 : 512) / NT;
}

// LAT: general cell (Cartesian positions and derivatives, see to_cartesian).
// GRP: grouped layout for small N. The plain layout gives each of the NT
// threads VEC orbitals of one position at a time (the CTA's NT*VEC orbitals).
// When a table's whole padded row fits in 2^lg < NT lanes, the grouped layout
// splits the CTA into NT >> lg position groups of 2^lg lanes that evaluate
// different positions side by side, so no thread idles for want of orbitals.
// A CTA takes cpos positions (group g evaluates positions g, g + groups, ...).
// PK: the arithmetic on pairs of orbitals with packed FP32 instructions (accumulate_x2; VEC = 4), same
// results; the weights are also kept as duplicated pairs in shared memory.
template <int KIND, typename T, int VEC, int NT, bool LAT = false, bool GRP = false, bool PK = false>
__global__ void __launch_bounds__(NT, (PK ? (GRP ? packed_grp_threads<acc_kind<KIND, LAT>()>() : 512) / NT
                                         : direct_min_blocks<acc_kind<KIND, LAT>(), T, NT>()))
    eval_direct_kernel(const EvalArgs A, int cpos, int nblk, int vst, int lg) {
    pdl_wait();
    pdl_trigger();
    constexpr int NB = NT * VEC;
    constexpr int AK = acc_kind<KIND, LAT>();
    constexpr int NO = nout_of(AK);
    constexpr int kPos = GRP ? kMaxCtaPos : kMaxPpc;
    __shared__ float sW[kPos][36];
    __shared__ f32x2 sW2[PK ? kPos : 1][36];
    __shared__ int sIdx[kPos][3];

    const int blk = (int)(blockIdx.x % (unsigned)nblk);
    const long long p0 = (long long)(blockIdx.x / (unsigned)nblk) * cpos;
    const int np = (int)min((long long)cpos, (long long)A.npos - p0);
    for (int r = threadIdx.x; r < np * 3; r += NT) {
        const int p = r / 3, d = r % 3;
        const double *X = d == 0 ? A.x : (d == 1 ? A.y : A.z);
        const int n = d == 0 ? A.nx : (d == 1 ? A.ny : A.nz);
        const long long pos = A.perm ? A.perm[p0 + p] : p0 + p;
        int i;
        float t;
        cell_reduce(LAT ? frac_coord(A, pos, d) : X[pos], n, i, t);
        basis_weights(t, (float)n, &sW[p][d * 12]);
        if constexpr (PK) {
#pragma unroll
            for (int k = 0; k < 12; ++k) sW2[p][d * 12 + k] = pack2(sW[p][d * 12 + k], sW[p][d * 12 + k]);
        }
        sIdx[p][d] = i;
    }
    __syncthreads();

    const int lane = GRP ? ((int)threadIdx.x & ((1 << lg) - 1)) : (int)threadIdx.x;
    const int p_first = GRP ? ((int)threadIdx.x >> lg) : 0;
    const int p_step = GRP ? (NT >> lg) : 1;
    const int n0 = blk * NB + lane * VEC;
    if (n0 >= A.Npad) return;
    const T *tab = static_cast<const T *>(A.table);

    float sc[VEC];
    if constexpr (sizeof(T) == 2 && !PK) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) sc[e] = A.scale[n0 + e];
    }

#pragma unroll 1
    for (int p = p_first; p < np; p += p_step) {
        const long long base =
            (long long)sIdx[p][0] * A.si + (long long)sIdx[p][1] * A.sj + (long long)sIdx[p][2] * A.Npad + n0;
        const T *rowp = tab + base;
        const long long si = A.si, sj = A.sj, sk = A.Npad;
        float out[NO][VEC];
        if constexpr (PK) {
            static_assert(VEC == 4, "packed accumulation takes 4 orbitals per thread");
            auto rows2 = [&](int a, int b, f32x2 (&pr)[4][2]) {
                const T *r = rowp + a * si + b * sj;
#pragma unroll
                for (int c = 0; c < 4; ++c) load_row_global_x2<T>(r + c * sk, pr[c]);
            };
            f32x2 acc2[NO][2];
            accumulate_x2<AK, 2>(&sW2[p][0], rows2, acc2);
            unpack_outputs(acc2, out);
        } else {
            auto rows = [&](int a, int b, float (&pr)[4][VEC]) {
                const T *r = rowp + a * si + b * sj;
#pragma unroll
                for (int c = 0; c < 4; ++c) load_row_global<T, VEC>(r + c * sk, pr[c]);
            };
            accumulate<AK, VEC>(&sW[p][0], rows, out);
        }
        if constexpr (sizeof(T) == 2) {
            if constexpr (PK) {  // loaded only now: no registers held across the accumulation
#pragma unroll
                for (int e = 0; e < VEC; ++e) sc[e] = A.scale[n0 + e];
            }
#pragma unroll
            for (int q = 0; q < NO; ++q)
#pragma unroll
                for (int e = 0; e < VEC; ++e) out[q][e] *= sc[e];
        }
        const long long pos = A.perm ? A.perm[p0 + p] : p0 + p;
        if constexpr (LAT) {
            float outc[nout_of(KIND)][VEC];
            to_cartesian<KIND, VEC>(A, out, outc);
            if (vst)
                store_outputs<KIND, VEC, true>(A, pos, n0, outc);
            else
                store_outputs<KIND, VEC, false>(A, pos, n0, outc);
        } else {
            if (vst)
                store_outputs<KIND, VEC, true>(A, pos, n0, out);
            else
                store_outputs<KIND, VEC, false>(A, pos, n0, out);
        }
    }
}

// ---------------------------------------------------------------------------
// DIRECT with the rows staged through shared memory (FP32 tables; launch
// shape DIRECT with stages = R in {3, 4, 6, 8}). The plain kernel loads an
// a-slice of 16 rows into registers, computes it, then loads the next, so its
// loads are in flight in bursts. Here each thread keeps a private ring of R
// units in shared memory - a unit is the 4 rows (c = 0..3) of one (a, b) - and
// cp.async keeps R of its 16 units in flight while it computes on the ones
// already there. A slot is refilled right after it is read, and the refill's
// address depends (by a zero term) on the data just read, so the copy cannot
// start before the read has returned.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// The rings live in dynamic shared memory rounded up to a 128-byte boundary (launches ask for
// kRingAlign bytes more). Dynamic shared memory follows the kernel's static shared memory, so its start
// moves with it; a ring that starts 16 bytes off a 32-byte boundary makes every 16-byte cp.async of a
// warp touch two sectors, which doubled the L2 read requests of the batched kernel (measured with ncu:
// 152 M against 76 M sectors for the same copies) and cost it a third of its speed.
constexpr size_t kRingAlign = 128;
__device__ __forceinline__ float4 *align_ring(void *dyn) {
    return reinterpret_cast<float4 *>((reinterpret_cast<uintptr_t>(dyn) + kRingAlign - 1) & ~uintptr_t(kRingAlign - 1));
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// A ring of at most 4 units (32 KB per CTA) leaves shared memory for 5 CTAs per SM, so the register
// budget is set for 5 (96 registers; 122 at 4 CTAs).
template <int KIND, int NT, int R> constexpr int async_min_blocks() {
    return R <= 4 ? 640 / NT : direct_min_blocks<KIND, float, NT>();
}

// The 4x4x4 accumulation of one position for the 4 orbitals at rowp (stencil point (0, 0, 0) of this
// thread's orbitals in an FP32 table with row strides si, sj, sk), the 16 units of 4 rows staged through
// this thread's ring of R units: mine is the thread's float4 in slot 0, row 0 of a [R][4][NT] float4
// array in shared memory. Issues the first R units, then refills each slot as soon as it is read.
template <int AK, int NT, int R>
__device__ __forceinline__ void accumulate_staged(const float *rowp, long long si, long long sj, long long sk,
                                                  float4 *mine, const float *W, float (&out)[nout_of(AK)][4]) {
    auto issue = [&](int u, const float *base) {
        const float *r = base + (u >> 2) * si + (u & 3) * sj;
        float4 *slot = mine + (u % R) * 4 * NT;
#pragma unroll
        for (int c = 0; c < 4; ++c) cp_async16(slot + c * NT, r + c * sk);
    };
#pragma unroll
    for (int u = 0; u < R; ++u) {
        issue(u, rowp);
        cp_async_commit();
    }
    int k = 0;  // unit the next call of rows reads: accumulate asks for (a, b) in the order a * 4 + b
    auto rows = [&](int a, int b, float (&pr)[4][4]) {
        cp_async_wait<R - 1>();
        const float4 *slot = mine + (k % R) * 4 * NT;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float4 v = slot[c * NT];
            pr[c][0] = v.x;
            pr[c][1] = v.y;
            pr[c][2] = v.z;
            pr[c][3] = v.w;
        }
        if (k + R < 16) {
            uint32_t dep;  // 0, but only once the reads above have returned
            asm volatile("and.b32 %0, %1, 0;" : "=r"(dep) : "r"(__float_as_uint(pr[3][3])));
            issue(k + R, rowp + dep);
        }
        cp_async_commit();
        ++k;
    };
    accumulate<AK, 4>(W, rows, out);
}

// accumulate_staged with the arithmetic on packed pairs (accumulate_x2); W2: the weights as duplicated pairs.
template <int AK, int NT, int R>
__device__ __forceinline__ void accumulate_staged_x2(const float *rowp, long long si, long long sj, long long sk,
                                                     float4 *mine, const f32x2 *W2, float (&out)[nout_of(AK)][4]) {
    auto issue = [&](int u, const float *base) {
        const float *r = base + (u >> 2) * si + (u & 3) * sj;
        float4 *slot = mine + (u % R) * 4 * NT;
#pragma unroll
        for (int c = 0; c < 4; ++c) cp_async16(slot + c * NT, r + c * sk);
    };
#pragma unroll
    for (int u = 0; u < R; ++u) {
        issue(u, rowp);
        cp_async_commit();
    }
    int k = 0;
    auto rows = [&](int a, int b, f32x2 (&pr)[4][2]) {
        cp_async_wait<R - 1>();
        const ulonglong2 *slot = reinterpret_cast<const ulonglong2 *>(mine + (k % R) * 4 * NT);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const ulonglong2 v = slot[c * NT];
            pr[c][0] = v.x;
            pr[c][1] = v.y;
        }
        if (k + R < 16) {
            uint32_t dep;  // 0, but only once the reads above have returned
            asm volatile("and.b32 %0, %1, 0;" : "=r"(dep) : "r"((uint32_t)(pr[3][1] >> 32)));
            issue(k + R, rowp + dep);
        }
        cp_async_commit();
        ++k;
    };
    f32x2 acc2[nout_of(AK)][2];
    accumulate_x2<AK, 2>(W2, rows, acc2);
    unpack_outputs(acc2, out);
}

// GRP: the grouped layout of eval_direct_kernel (a row of at most 256 orbitals; position groups of 2^lg
// lanes, cpos positions per CTA); each thread's ring is refilled from the start for each of its positions.
template <int KIND, int NT, int R, bool LAT, bool GRP = false, bool PK = false>
__global__ void __launch_bounds__(NT, (GRP ? (PK ? packed_grp_threads<acc_kind<KIND, LAT>()>() / NT
                                                 : direct_min_blocks<acc_kind<KIND, LAT>(), float, NT>())
                                           : async_min_blocks<acc_kind<KIND, LAT>(), NT, R>()))
    eval_direct_async_kernel(const EvalArgs A, int ppc, int nblk, int vst, int lg = 0) {
    pdl_wait();
    pdl_trigger();
    constexpr int VEC = 4, NB = NT * VEC;
    constexpr int AK = acc_kind<KIND, LAT>();
    constexpr int NO = nout_of(AK);
    constexpr int kPos = GRP ? kMaxCtaPos : kMaxPpc;
    extern __shared__ __align__(16) float4 ring_raw[];
    float4 *ring = align_ring(ring_raw);  // [R][4][NT]: slot, row c, thread
    __shared__ float sW[kPos][36];
    __shared__ f32x2 sW2[PK ? kPos : 1][36];
    __shared__ int sIdx[kPos][3];

    const int blk = (int)(blockIdx.x % (unsigned)nblk);
    const long long p0 = (long long)(blockIdx.x / (unsigned)nblk) * ppc;
    const int np = (int)min((long long)ppc, (long long)A.npos - p0);
    for (int r = threadIdx.x; r < np * 3; r += NT) {
        const int p = r / 3, d = r % 3;
        const double *X = d == 0 ? A.x : (d == 1 ? A.y : A.z);
        const int n = d == 0 ? A.nx : (d == 1 ? A.ny : A.nz);
        const long long pos = A.perm ? A.perm[p0 + p] : p0 + p;
        int i;
        float t;
        cell_reduce(LAT ? frac_coord(A, pos, d) : X[pos], n, i, t);
        basis_weights(t, (float)n, &sW[p][d * 12]);
        if constexpr (PK) {
#pragma unroll
            for (int k = 0; k < 12; ++k) sW2[p][d * 12 + k] = pack2(sW[p][d * 12 + k], sW[p][d * 12 + k]);
        }
        sIdx[p][d] = i;
    }
    __syncthreads();

    const int lane = GRP ? ((int)threadIdx.x & ((1 << lg) - 1)) : (int)threadIdx.x;
    const int p_first = GRP ? ((int)threadIdx.x >> lg) : 0;
    const int p_step = GRP ? (NT >> lg) : 1;
    const int n0 = blk * NB + lane * VEC;
    if (n0 >= A.Npad) return;
    const float *tab = static_cast<const float *>(A.table);
    const long long si = A.si, sj = A.sj, sk = A.Npad;
    float4 *mine = ring + threadIdx.x;

#pragma unroll 1
    for (int p = p_first; p < np; p += p_step) {
        const float *rowp =
            tab + (long long)sIdx[p][0] * si + (long long)sIdx[p][1] * sj + (long long)sIdx[p][2] * sk + n0;
        float out[NO][VEC];
        if constexpr (PK)
            accumulate_staged_x2<AK, NT, R>(rowp, si, sj, sk, mine, &sW2[p][0], out);
        else
            accumulate_staged<AK, NT, R>(rowp, si, sj, sk, mine, &sW[p][0], out);
        const long long pos = A.perm ? A.perm[p0 + p] : p0 + p;
        if constexpr (LAT) {
            float outc[nout_of(KIND)][VEC];
            to_cartesian<KIND, VEC>(A, out, outc);
            if (vst)
                store_outputs<KIND, VEC, true>(A, pos, n0, outc);
            else
                store_outputs<KIND, VEC, false>(A, pos, n0, outc);
        } else {
            if (vst)
                store_outputs<KIND, VEC, true>(A, pos, n0, out);
            else
                store_outputs<KIND, VEC, false>(A, pos, n0, out);
        }
    }
}

// ---------------------------------------------------------------------------
// Fused determinant-ratio consumer (Sec. "QMC and B-spline-based SPOs": the
// ratio det[A']/det[A] = sum_n phi_n(r_e) A^-1(n,e) of a one-electron move,
// and the same sum over grad phi_n for the gradient ratio). One CTA takes one
// position and all N orbitals, NT*VEC of them at a time: each component of
// the orbital outputs is multiplied by u_n = A^-1(n,e) (u = A.uinv + pos*ldu)
// and summed over the block's orbitals in a fixed tree (per thread, warp
// shuffles, warps in order); the block sums are added in block order, so the
// result is deterministic. out[pos*nout + q] receives the sum of component q
// (the same components, in the same order, as the per-orbital outputs of KIND).
// ---------------------------------------------------------------------------
// Reducing each block before the next keeps no running sums live across the
// stencil loop, so the FP32 kernel with rows staged through the ring has the
// staged kernel's register budget (640 resident threads per SM, 4-unit ring).
// 16-bit tables (rows in registers): VGL/VGH 384 resident threads per SM (168
// registers), V the DIRECT budget.
template <int KIND, typename T, int NT, int R> constexpr int ratio_min_blocks() {
    return R > 0 ? async_min_blocks<KIND, NT, R>() : (KIND == BSPLINE_V ? direct_min_blocks<KIND, T, NT>() : 384 / NT);
}

// R > 0 (FP32 tables): each block's rows are staged through a per-thread
// shared-memory ring of R 4-row units as in eval_direct_async_kernel (for VGL
// and VGH with packed arithmetic), the ring refilled for each block.
template <int KIND, typename T, int VEC, int NT, bool LAT = false, int R = 0>
__global__ void __launch_bounds__(NT, (ratio_min_blocks<acc_kind<KIND, LAT>(), T, NT, R>()))
    eval_ratio_kernel(const EvalArgs A, const float *__restrict__ uinv, int ldu, float *__restrict__ ratio) {
    pdl_wait();
    pdl_trigger();
    constexpr int NB = NT * VEC;
    constexpr int AK = acc_kind<KIND, LAT>();
    constexpr int NO = nout_of(KIND);
    constexpr bool PK = R > 0 && packed_staged_plain<AK>();  // packed pairs of orbitals (VGL/VGH)
    static_assert(R == 0 || (sizeof(T) == 4 && VEC == 4), "the staged ratio kernel takes FP32 rows, 4 orbitals per thread");
    __shared__ float sW[36];
    __shared__ f32x2 sW2[PK ? 36 : 1];
    __shared__ int sIdx[3];
    __shared__ float sRed[NO][NT / 32];

    const long long slot = blockIdx.x;
    const long long pos = A.perm ? A.perm[slot] : slot;
    if (threadIdx.x < 3) {
        const int d = threadIdx.x;
        const double *X = d == 0 ? A.x : (d == 1 ? A.y : A.z);
        const int n = d == 0 ? A.nx : (d == 1 ? A.ny : A.nz);
        int i;
        float t;
        cell_reduce(LAT ? frac_coord(A, pos, d) : X[pos], n, i, t);
        basis_weights(t, (float)n, &sW[d * 12]);
        if constexpr (PK) {
#pragma unroll
            for (int k = 0; k < 12; ++k) sW2[d * 12 + k] = pack2(sW[d * 12 + k], sW[d * 12 + k]);
        }
        sIdx[d] = i;
    }
    __syncthreads();
    const T *tab = static_cast<const T *>(A.table);
    const long long base = (long long)sIdx[0] * A.si + (long long)sIdx[1] * A.sj + (long long)sIdx[2] * A.Npad;
    const long long si = A.si, sj = A.sj, sk = A.Npad;
    const float *u = uinv + pos * (long long)ldu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    extern __shared__ __align__(16) float4 ratio_ring_raw[];
    float4 *mine = align_ring(ratio_ring_raw) + threadIdx.x;  // [R][4][NT]
    float total = 0.f;  // thread q < NO: the sum of component q over the blocks done so far
    const int nblk = (A.Npad + NB - 1) / NB;

    // every thread takes part in every block's reduction, also past the end of the padded row
#pragma unroll 1
    for (int b = 0; b < nblk; ++b) {
        const int n0 = b * NB + (int)threadIdx.x * VEC;
        float out[NO][VEC];
        float w[VEC];
        if (n0 < A.Npad) {
            float acc[nout_of(AK)][VEC];
            if constexpr (PK) {
                accumulate_staged_x2<AK, NT, R>(reinterpret_cast<const float *>(tab) + base + n0, si, sj, sk, mine,
                                                sW2, acc);
            } else if constexpr (R > 0) {
                accumulate_staged<AK, NT, R>(reinterpret_cast<const float *>(tab) + base + n0, si, sj, sk, mine, sW,
                                             acc);
            } else {
                const T *rowp = tab + base + n0;
                auto rows = [&](int a, int b2, float (&pr)[4][VEC]) {
                    const T *r = rowp + a * si + b2 * sj;
#pragma unroll
                    for (int c = 0; c < 4; ++c) load_row_global<T, VEC>(r + c * sk, pr[c]);
                };
                accumulate<AK, VEC>(sW, rows, acc);
            }
            if constexpr (LAT) {
                to_cartesian<KIND, VEC>(A, acc, out);
            } else {
#pragma unroll
                for (int q = 0; q < NO; ++q)
#pragma unroll
                    for (int e = 0; e < VEC; ++e) out[q][e] = acc[q][e];
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int n = n0 + e;
                w[e] = n < A.N ? u[n] : 0.f;
                if constexpr (sizeof(T) == 2) {
                    if (n < A.N) w[e] *= A.scale[n];
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < NO; ++q)
#pragma unroll
                for (int e = 0; e < VEC; ++e) out[q][e] = 0.f;
#pragma unroll
            for (int e = 0; e < VEC; ++e) w[e] = 0.f;
        }
        // this block's sums, one component at a time: this thread's orbitals in order, warp shuffles,
        // then the warps' totals in order
#pragma unroll
        for (int q = 0; q < NO; ++q) {
            float v = 0.f;
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                if (n0 + e < A.N) v = fmaf(out[q][e], w[e], v);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) sRed[q][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < NO) {
            float v = 0.f;
#pragma unroll
            for (int k = 0; k < NT / 32; ++k) v += sRed[threadIdx.x][k];
            total += v;
        }
        __syncthreads();  // sRed is rewritten by the next block
    }
    if (threadIdx.x < NO) ratio[pos * NO + threadIdx.x] = total;
}

// Shared-memory layout of the TMA kernel (bytes from a 128-byte aligned base):
//   [stages][64][NBOX] T   stencil slices, TMA destination
//   [stages][36] float     weights of the slot's position
//   [stages] uint64        full barriers (producer arrive + TMA bytes)
//   [stages] uint64        empty barriers (one arrive per consumer warp)
__host__ __device__ constexpr size_t tma_slot_bytes(int esize, int nbox) { return (size_t)64 * nbox * esize; }
__host__ __device__ constexpr size_t tma_layout_bytes(int esize, int nbox, int stages) {
    return tma_slot_bytes(esize, nbox) * stages + (size_t)stages * 36 * 4 + (size_t)stages * 16 + 128;
}

template <int KIND, typename T, int NBOX>
__global__ void __launch_bounds__(32 + NBOX, 1)
    eval_tma_kernel(const __grid_constant__ CUtensorMap map, const EvalArgs A, int nblk, int stages) {
    pdl_wait();
    pdl_trigger();
    constexpr int CW = NBOX / 32;  // consumer warps, one orbital per consumer thread
    constexpr int NO = nout_of(KIND);
    constexpr uint32_t kSlotBytes = 64u * NBOX * sizeof(T);
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    T *sTab = reinterpret_cast<T *>(base);
    float *sW = reinterpret_cast<float *>(base + (size_t)kSlotBytes * stages);
    uint64_t *full = reinterpret_cast<uint64_t *>(sW + stages * 36);
    uint64_t *empty = full + stages;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CW);
        }
        fence_mbar_init();
    }
    __syncthreads();

    const long long total = (long long)A.npos * nblk;
    if (warp == 0) {
        if (lane != 0) return;
        // Producer: cell + weights for the slot, then one TMA box per item.
        long long it = 0;
        for (long long w = blockIdx.x; w < total; w += gridDim.x, ++it) {
            const int s = (int)(it % stages);
            const uint32_t ph = (uint32_t)((it / stages) & 1);
            if (it >= stages && !mbar_wait_bounded(&empty[s], ph ^ 1u, A.status)) break;
            const long long slot = w / nblk;
            const int blk = (int)(w - slot * nblk);
            const long long pos = A.perm ? A.perm[slot] : slot;
            int ci, cj, ck;
            float tx, ty, tz;
            cell_reduce(A.x[pos], A.nx, ci, tx);
            cell_reduce(A.y[pos], A.ny, cj, ty);
            cell_reduce(A.z[pos], A.nz, ck, tz);
            float *W = sW + s * 36;
            basis_weights(tx, (float)A.nx, W);
            basis_weights(ty, (float)A.ny, W + 12);
            basis_weights(tz, (float)A.nz, W + 24);
            mbar_arrive_expect_tx(&full[s], kSlotBytes);
            tma_load_4d(sTab + (size_t)s * 64 * NBOX, &map, &full[s], blk * NBOX, ck, cj, ci);
        }
        // Every box this CTA issued has landed before the CTA may exit.
        const long long first = it > stages ? it - stages : 0;
        for (long long j = first; j < it; ++j) {
            const int s = (int)(j % stages);
            if (!mbar_wait_bounded(&full[s], (uint32_t)((j / stages) & 1), A.status)) break;
        }
        return;
    }

    // Consumers
    const int ct = threadIdx.x - 32;
    long long it = 0;
    for (long long w = blockIdx.x; w < total; w += gridDim.x, ++it) {
        const int s = (int)(it % stages);
        const uint32_t ph = (uint32_t)((it / stages) & 1);
        // warp-uniform outcome, so that a timed-out lane never leaves its warp behind
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[s], ph, A.status))) break;
        const long long slot = w / nblk;
        const int blk = (int)(w - slot * nblk);
        const long long pos = A.perm ? A.perm[slot] : slot;
        const T *st = sTab + (size_t)s * 64 * NBOX + ct;
        auto rows = [&](int a, int b, float (&pr)[4][1]) {
#pragma unroll
            for (int c = 0; c < 4; ++c) load_row_shared<T, 1>(st + ((a * 4 + b) * 4 + c) * NBOX, pr[c]);
        };
        float out[NO][1];
        accumulate<KIND, 1>(sW + s * 36, rows, out);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        const int n0 = blk * NBOX + ct;
        if (n0 < A.N) {
            if constexpr (sizeof(T) == 2) {
                const float sc = A.scale[n0];
#pragma unroll
                for (int q = 0; q < NO; ++q) out[q][0] *= sc;
            }
            store_outputs<KIND, 1, false>(A, pos, n0, out);
        }
    }
}

// ---------------------------------------------------------------------------
// Host dispatch for one element type
// ---------------------------------------------------------------------------
template <int KIND, typename T, int NBOX>
static bspline_status launch_tma(const EvalArgs &A, const CUtensorMap *map, int nblk, int stages, int grid,
                                 size_t smem, cudaStream_t s) {
    auto kern = eval_tma_kernel<KIND, T, NBOX>;
    static bool attr_set = false;  // idempotent; a race only repeats the call
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return cuda_status(e);
        attr_set = true;
    }
    return cuda_status(launch_k(kern, grid, 32 + NBOX, smem, s, true, *map, A, nblk, stages));
}



// Plain layout with NT threads, or, when the padded row fits in 64 lanes or
// fewer (Npad <= 256), the grouped layout with 128 threads: lanes = the
// smallest power of two that holds the row, ppc positions per group, at most
// kMaxCtaPos positions per CTA.
template <int KIND, typename T, int NT, bool LAT>
static bspline_status launch_direct(const EvalArgs &A, int ppc, cudaStream_t s) {
    constexpr int VEC = 4;
    const int vst = (A.ld % VEC == 0) && (reinterpret_cast<uintptr_t>(A.o0) % 16 == 0) &&
                    (!A.o1 || reinterpret_cast<uintptr_t>(A.o1) % 16 == 0) &&
                    (!A.o2 || reinterpret_cast<uintptr_t>(A.o2) % 16 == 0);
    if (A.Npad <= 64 * VEC) {
        constexpr int GNT = 128;
        int lg = 0;
        while ((1 << lg) * VEC < A.Npad) ++lg;
        const int groups = GNT >> lg;
        const int cpos = groups * (ppc < kMaxCtaPos / groups ? ppc : kMaxCtaPos / groups);
        const long long grid = ((long long)A.npos + cpos - 1) / cpos;
        if (grid > 0x7fffffffLL) return BSPLINE_ERR_ARG;
        return cuda_status(launch_k(eval_direct_kernel<KIND, T, VEC, GNT, LAT, true, packed_direct<T, KIND>()>,
                                    (unsigned)grid, GNT, 0, s, true, A, cpos, 1, vst, lg));
    }
    constexpr int NB = NT * VEC;
    const int nblk = (A.Npad + NB - 1) / NB;
    const long long grid = ((long long)A.npos + ppc - 1) / ppc * nblk;
    if (grid > 0x7fffffffLL) return BSPLINE_ERR_ARG;
    return cuda_status(launch_k(eval_direct_kernel<KIND, T, VEC, NT, LAT, false, packed_direct<T, KIND>()>,
                                (unsigned)grid, NT, 0, s, true, A, ppc, nblk, vst, 0));
}

// DIRECT with rows staged through shared memory: FP32 tables, 128 threads,
// ring of R units per thread (R * 8 KB of shared memory per CTA).
template <int KIND, typename T>
static bspline_status launch_direct_async(const EvalArgs &A, int ppc, int R, cudaStream_t s) {
    if constexpr (sizeof(T) != 4) {
        return BSPLINE_ERR_UNSUPPORTED;
    } else {
        constexpr int NT = 128, NB = NT * 4;
        const int nblk = (A.Npad + NB - 1) / NB;
        const long long grid = ((long long)A.npos + ppc - 1) / ppc * nblk;
        if (grid > 0x7fffffffLL) return BSPLINE_ERR_ARG;
        const int vst = (A.ld % 4 == 0) && (reinterpret_cast<uintptr_t>(A.o0) % 16 == 0) &&
                        (!A.o1 || reinterpret_cast<uintptr_t>(A.o1) % 16 == 0) &&
                        (!A.o2 || reinterpret_cast<uintptr_t>(A.o2) % 16 == 0);
        const size_t smem = (size_t)R * 4 * NT * sizeof(float4) + kRingAlign;
        if (A.Npad <= 64 * 4 && (R == 4 || R == 16)) {  // grouped layout (4-unit ring; 16 for small launches)
            int lg = 0;
            while ((1 << lg) * 4 < A.Npad) ++lg;
            const int groups = NT >> lg;
            const int cpos = groups * (ppc < kMaxCtaPos / groups ? ppc : kMaxCtaPos / groups);
            const long long ggrid = ((long long)A.npos + cpos - 1) / cpos;
            if (ggrid > 0x7fffffffLL) return BSPLINE_ERR_ARG;
            if (R == 16) {  // every unit of the stencil in flight at once (128 KB per CTA, one CTA per SM)
                if (A.lattice) return BSPLINE_ERR_UNSUPPORTED;
                auto kern = eval_direct_async_kernel<KIND, NT, 16, false, true, packed_small<KIND>()>;
                static bool dattr = false;  // idempotent; a race only repeats the call
                if (!dattr) {
                    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    if (e != cudaSuccess) return cuda_status(e);
                    dattr = true;
                }
                return cuda_status(launch_k(kern, (unsigned)ggrid, NT, smem, s, true, A, cpos, 1, vst, lg));
            }
            static bool gattr[2] = {false, false};  // [lattice]
            auto kern = A.lattice ? eval_direct_async_kernel<KIND, NT, 4, true, true>
                                  : eval_direct_async_kernel<KIND, NT, 4, false, true>;
            if (!gattr[A.lattice ? 1 : 0]) {
                cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return cuda_status(e);
                gattr[A.lattice ? 1 : 0] = true;
            }
            return cuda_status(launch_k(kern, (unsigned)ggrid, NT, smem, s, true, A, cpos, 1, vst, lg));
        }
        static bool attr_set[9][2] = {};  // [R][lattice]; idempotent, a race only repeats the call
#define BSG_ASYNC(RR)                                                                                        \
    {                                                                                                        \
        auto kern = A.lattice ? eval_direct_async_kernel<KIND, NT, RR, true, false, packed_staged_plain<KIND>()> \
                              : eval_direct_async_kernel<KIND, NT, RR, false, false, packed_staged_plain<KIND>()>;\
        if (!attr_set[RR][A.lattice ? 1 : 0]) {                                                            \
            cudaError_t e =                                                                                 \
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);         \
            if (e != cudaSuccess) return cuda_status(e);                                                   \
            attr_set[RR][A.lattice ? 1 : 0] = true;                                                        \
        }                                                                                                    \
        return cuda_status(launch_k(kern, (unsigned)grid, NT, smem, s, true, A, ppc, nblk, vst, 0));         \
    }
        switch (R) {
            case 3: BSG_ASYNC(3)
            case 4: BSG_ASYNC(4)
            case 6: BSG_ASYNC(6)
            case 8: BSG_ASYNC(8)
            default: return BSPLINE_ERR_ARG;
        }
#undef BSG_ASYNC
    }
}

// DIRECT positions per CTA when the launch shape leaves it to the call (ppc = 0): 1, except in the
// grouped layout (tables of at most 256 orbitals), where a call with many positions gives each group up
// to 4 positions in turn while at least 16 CTAs per SM remain. Measured at 48 x 48 x 60 x 128, VGH:
// 65536 positions 298 -> 276 us with 4; 4096 positions are fastest with 1.
inline int auto_ppc(const EvalArgs &A, int num_sms) {
    if (A.Npad > 64 * 4) return 1;
    int lg = 0;
    while ((1 << lg) * 4 < A.Npad) ++lg;
    const long long groups = 128 >> lg;
    const long long per = (long long)A.npos / (groups * 16LL * num_sms);
    return per < 1 ? 1 : (per > 4 ? 4 : (int)per);
}

// A call small enough that the grouped layout (rows of at most 256 FP32 orbitals) fills at most one CTA
// per SM: latency, not occupancy, bounds it, and a 4-unit ring would fetch a position's 16 units in four
// round trips to L2. When the launch shape leaves positions per CTA to the call (ppc = 0, the default),
// such a call stages all 16 units at once instead (eval_direct_async_kernel with R = 16); the arithmetic
// and so the results are those of every other FP32 kernel.
template <typename T>
inline bool small_grouped_launch(const EvalArgs &A, const bspline_tuning &tu, int num_sms) {
    if (sizeof(T) != 4 || A.lattice || tu.variant != BSPLINE_VARIANT_DIRECT || tu.ppc != 0 || tu.nb != 512 ||
        A.Npad > 64 * 4)
        return false;
    int lg = 0;
    while ((1 << lg) * 4 < A.Npad) ++lg;
    const long long groups = 128 >> lg;
    return ((long long)A.npos + groups - 1) / groups <= num_sms;
}

template <int KIND, typename T>
static bspline_status launch_kind(const bspline_tuning &tu, const EvalArgs &A, const CUtensorMap *map, int num_sms,
                                  cudaStream_t s) {
    if (tu.variant == BSPLINE_VARIANT_MMA) {
        if (A.lattice) return launch_mma<KIND, T, true>(A, map, tu.nb, tu.stages, tu.ppc, num_sms, s);
        return launch_mma<KIND, T, false>(A, map, tu.nb, tu.stages, tu.ppc, num_sms, s);
    }
    if (A.lattice) {
        if (tu.variant == BSPLINE_VARIANT_TMA) return BSPLINE_ERR_UNSUPPORTED;
        const int lppc = tu.ppc ? tu.ppc : auto_ppc(A, num_sms);
        // FP32 rows staged through the ring, as in the unit cell (48^3 x 2048, 4096 sorted positions, hexagonal
        // cell: VGH 236.5 -> 213.0 us, VGL 213.0 -> 190.9 us against rows in registers)
        if (sizeof(T) == 4 && tu.stages >= 3) return launch_direct_async<KIND, T>(A, lppc, tu.stages, s);
        return launch_direct<KIND, T, 128, true>(A, lppc, s);  // 128 threads only
    }
    if (tu.variant == BSPLINE_VARIANT_TMA) {
        const int nbox = tu.nb;
        const int stages = tu.stages;
        const int nblk = (A.Npad + nbox - 1) / nbox;
        const long long total = (long long)A.npos * nblk;
        const long long want = (long long)num_sms * tu.ppc;
        const int grid = (int)(total < want ? total : want);
        const size_t smem = tma_layout_bytes((int)sizeof(T), nbox, stages);
        if (!map) return BSPLINE_ERR_ARG;
        if (nbox == 256) return launch_tma<KIND, T, 256>(A, map, nblk, stages, grid, smem, s);
        if (nbox == 128) return launch_tma<KIND, T, 128>(A, map, nblk, stages, grid, smem, s);
        return BSPLINE_ERR_ARG;
    }
    const int ppc = tu.ppc ? tu.ppc : auto_ppc(A, num_sms);
    if (small_grouped_launch<T>(A, tu, num_sms)) return launch_direct_async<KIND, T>(A, 1, 16, s);
    if (tu.stages >= 3) return launch_direct_async<KIND, T>(A, ppc, tu.stages, s);
    const int nt = tu.nb / 4;
    if (nt == 64) return launch_direct<KIND, T, 64, false>(A, ppc, s);
    if (nt == 128) return launch_direct<KIND, T, 128, false>(A, ppc, s);
    if (nt == 256) return launch_direct<KIND, T, 256, false>(A, ppc, s);
    return BSPLINE_ERR_ARG;
}

template <typename T>
static bspline_status launch_eval_typed(int kind, const bspline_tuning &tu, const EvalArgs &A,
                                        const CUtensorMap *map, int num_sms, cudaStream_t s) {
    switch (kind) {
        case BSPLINE_V: return launch_kind<BSPLINE_V, T>(tu, A, map, num_sms, s);
        case BSPLINE_VGL: return launch_kind<BSPLINE_VGL, T>(tu, A, map, num_sms, s);
        case BSPLINE_VGH: return launch_kind<BSPLINE_VGH, T>(tu, A, map, num_sms, s);
        default: return BSPLINE_ERR_ARG;
    }
}

// Ratio sums on the tensor-core variant (16-bit tables): the launch shape tu.
template <typename T>
static bspline_status launch_ratio_mma_typed(int kind, const bspline_tuning &tu, const EvalArgs &A,
                                             const CUtensorMap *map, int num_sms, const float *uinv, int ldu,
                                             float *ratio, cudaStream_t s) {
#define BSG_MMA_RATIO(K)                                                                          \
    (A.lattice ? launch_mma<K, T, true>(A, map, tu.nb, tu.stages, tu.ppc, num_sms, s, uinv, ldu, ratio) \
               : launch_mma<K, T, false>(A, map, tu.nb, tu.stages, tu.ppc, num_sms, s, uinv, ldu, ratio))
    switch (kind) {
        case BSPLINE_V: return BSG_MMA_RATIO(BSPLINE_V);
        case BSPLINE_VGL: return BSG_MMA_RATIO(BSPLINE_VGL);
        case BSPLINE_VGH: return BSG_MMA_RATIO(BSPLINE_VGH);
        default: return BSPLINE_ERR_ARG;
    }
#undef BSG_MMA_RATIO
}

// Launch of the fused ratio kernel: one CTA of 128 threads per position.
template <typename T>
static bspline_status launch_ratio_typed(int kind, const EvalArgs &A, const float *uinv, int ldu, float *ratio,
                                         cudaStream_t s) {
    if (A.npos > 0x7fffffff) return BSPLINE_ERR_ARG;
    const unsigned grid = (unsigned)A.npos;
    // FP32 tables: rows staged through a 4-unit shared-memory ring (32 KB per CTA)
#define BSG_RATIO(K, L)                                                                                   \
    {                                                                                                     \
        constexpr int RR = sizeof(T) == 4 ? 4 : 0;                                                       \
        const size_t smem = RR > 0 ? (size_t)RR * 4 * 128 * sizeof(float4) + kRingAlign : 0;            \
        auto kern = eval_ratio_kernel<K, T, 4, 128, L, RR>;                                              \
        static bool attr = false; /* idempotent; a race only repeats the call */                         \
        if (RR > 0 && !attr) {                                                                            \
            cudaError_t e =                                                                              \
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);         \
            if (e != cudaSuccess) return cuda_status(e);                                                 \
            attr = true;                                                                                  \
        }                                                                                                 \
        const cudaError_t le = launch_k(kern, grid, 128, smem, s, true, A, uinv, ldu, ratio);             \
        if (le != cudaSuccess) return cuda_status(le);                                                    \
    }
    switch (kind) {
        case BSPLINE_V:
            if (A.lattice) BSG_RATIO(BSPLINE_V, true) else BSG_RATIO(BSPLINE_V, false) break;
        case BSPLINE_VGL:
            if (A.lattice) BSG_RATIO(BSPLINE_VGL, true) else BSG_RATIO(BSPLINE_VGL, false) break;
        case BSPLINE_VGH:
            if (A.lattice) BSG_RATIO(BSPLINE_VGH, true) else BSG_RATIO(BSPLINE_VGH, false) break;
        default: return BSPLINE_ERR_ARG;
    }
#undef BSG_RATIO
    return cuda_status(cudaGetLastError());
}

}  // namespace bsg
