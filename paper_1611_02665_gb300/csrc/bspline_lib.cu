// C ABI of the GB300 B-spline library: table lifetime, coefficient upload
// (periodic padding, per-orbital reduced-precision scaling), single-table
// evaluation entry points, the host-buffer path and the device status word.
//
// Paper: arXiv:1611.02665, Sec. "Baseline and miniQMC": the read-only table
// P[Nx][Ny][Nz][N] is created once and shared; V, VGL and VGH evaluate all N
// orbitals at one position. Eq. (SplineFunc) gives the stencil knots i-1..i+2
// that the padded rows hold.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "bspline_eval_kernels.cuh"

using namespace bsg;

namespace bsg {

bspline_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return BSPLINE_OK;
    if (e == cudaErrorMemoryAllocation) return BSPLINE_ERR_ALLOC;
    return BSPLINE_ERR_CUDA;
}

int default_stages(int dtype, int nbox) { return (dtype == BSPLINE_F32 && nbox == 256) ? 3 : 4; }

size_t tma_smem_bytes(int dtype, int nbox, int stages) {
    return tma_layout_bytes(dtype == BSPLINE_F32 ? 4 : 2, nbox, stages);
}

// ctas CTAs of the tensor-core variant fit an SM's 228 KB of shared memory
// (each CTA also reserves 1 KB).
bool mma_fits(int dtype, int stages, int Npad, int ctas, int nb) {
    return (mma_smem_bytes_dtype(dtype, stages, Npad, nb) + 1024) * (size_t)ctas <= 228u * 1024u;
}

// Dynamic shared memory of the tensor-core variant (16-bit tables only), units of nb orbitals.
size_t mma_smem_bytes_dtype(int dtype, int stages, int Npad, int nb) {
    const int nmblk = (Npad + kMmaM - 1) / kMmaM;
    const int ub = nb / kMmaM;
    return dtype == BSPLINE_F16 ? mma_smem_bytes<__half>(stages, nmblk, ub)
                                : mma_smem_bytes<__nv_bfloat16>(stages, nmblk, ub);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 4-D tensor map over the padded table: dims {Npad, nz+3, ny+3, nx+3}, box
// {nbox, 4, 4, 4} = one orbital block of the whole 4x4x4 stencil.
bspline_status get_tma_map(bspline_t t, int nbox, int swizzle, const CUtensorMap **out) {
    std::lock_guard<std::mutex> g(t->mu);
    for (int m = 0; m < t->nmaps; ++m)
        if (t->maps[m].nbox == nbox && t->maps[m].swizzle == swizzle) {
            *out = &t->maps[m].map;
            return BSPLINE_OK;
        }
    if (t->nmaps >= kMaxTmaMaps) return BSPLINE_ERR_ARG;
    auto enc = tensor_map_encoder();
    if (!enc) return BSPLINE_ERR_UNSUPPORTED;
    CUtensorMapDataType dt = t->dtype == BSPLINE_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                             : t->dtype == BSPLINE_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t es = (cuuint64_t)t->esize;
    cuuint64_t dims[4] = {(cuuint64_t)t->Npad, (cuuint64_t)t->nz + 3, (cuuint64_t)t->ny + 3, (cuuint64_t)t->nx + 3};
    cuuint64_t strides[3] = {dims[0] * es, dims[0] * dims[1] * es, dims[0] * dims[1] * dims[2] * es};
    cuuint32_t box[4] = {(cuuint32_t)nbox, 4, 4, 4};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    TmaMapEntry &e = t->maps[t->nmaps];
    CUresult r = enc(&e.map, dt, 4, t->table, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return BSPLINE_ERR_CUDA;
    e.nbox = nbox;
    e.swizzle = swizzle;
    ++t->nmaps;
    *out = &e.map;
    return BSPLINE_OK;
}

}  // namespace bsg

// ---------------------------------------------------------------------------
// Table construction kernels
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// Row of the source array that padded row (a, b, c) takes its values from.
__device__ __forceinline__ size_t source_row(size_t r, int nx, int ny, int nz, int src_padded) {
    if (src_padded) return r;
    const int c = (int)(r % (nz + 3));
    const size_t q = r / (nz + 3);
    const int b = (int)(q % (ny + 3));
    const int a = (int)(q / (ny + 3));
    return ((size_t)wrapi(a - 1, nx) * ny + wrapi(b - 1, ny)) * nz + wrapi(c - 1, nz);
}

// Per-orbital max |p| into bits[] (non-negative floats order like unsigned ints). A warp covers
// 32 * V consecutive orbitals of a row (V = 4: 16-byte loads, N % 4 == 0 and src 16-byte aligned),
// the CTA's 8 warps different rows; four rows per warp are loaded before they are compared.
template <int V>
__global__ void __launch_bounds__(256) absmax_kernel(const float *__restrict__ src, size_t nrows, int N,
                                                     unsigned *__restrict__ bits) {
    const int lane = threadIdx.x & 31, wrow = threadIdx.x >> 5;
    const int n = (blockIdx.x * 32 + lane) * V;
    const size_t step = (size_t)8 * gridDim.y;
    float m[V];
#pragma unroll
    for (int e = 0; e < V; ++e) m[e] = 0.f;
    if (n < N) {
        size_t r = (size_t)blockIdx.y * 8 + wrow;
        for (; r + 3 * step < nrows; r += 4 * step) {
            float v[4][V];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float *p = src + (r + u * step) * N + n;
                if constexpr (V == 4) {
                    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
                    v[u][0] = q.x, v[u][1] = q.y, v[u][2] = q.z, v[u][3] = q.w;
                } else {
                    v[u][0] = __ldg(p);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int e = 0; e < V; ++e) m[e] = fmaxf(m[e], fabsf(v[u][e]));
        }
        for (; r < nrows; r += step) {
            const float *p = src + r * N + n;
#pragma unroll
            for (int e = 0; e < V; ++e) m[e] = fmaxf(m[e], fabsf(__ldg(p + e)));
        }
    }
    __shared__ float red[8][32 * V + 1];
#pragma unroll
    for (int e = 0; e < V; ++e) red[wrow][lane * V + e] = m[e];
    __syncthreads();
    for (int c = threadIdx.x; c < 32 * V; c += blockDim.x) {
        const int nc = blockIdx.x * 32 * V + c;
        if (nc >= N) continue;
        float mm = red[0][c];
        for (int k = 1; k < 8; ++k) mm = fmaxf(mm, red[k][c]);
        atomicMax(&bits[nc], __float_as_uint(mm));
    }
}

__global__ void finalize_scale_kernel(unsigned *bits, int N, int Npad, int reduced) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= Npad) return;
    float s = 1.f;
    if (reduced && n < N) {
        s = __uint_as_float(bits[n]);
        if (!(s > 0.f)) s = 1.f;
    }
    reinterpret_cast<float *>(bits)[n] = s;
}

template <typename T> __device__ __forceinline__ T encode(float v, float s);
template <> __device__ __forceinline__ float encode<float>(float v, float) { return v; }
template <> __device__ __forceinline__ __half encode<__half>(float v, float s) {
    return __float2half_rn(__fdiv_rn(v, s));
}
template <> __device__ __forceinline__ __nv_bfloat16 encode<__nv_bfloat16>(float v, float s) {
    return __float2bfloat16_rn(__fdiv_rn(v, s));
}

// Four encoded values stored together (16 bytes of float, 8 of a 16-bit type).
template <typename T> __device__ __forceinline__ void store4(T *d, float4 v, float4 s) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(d) = v;
    } else {
        const T e[4] = {encode<T>(v.x, s.x), encode<T>(v.y, s.y), encode<T>(v.z, s.z), encode<T>(v.w, s.w)};
        uint2 u;
        memcpy(&u, e, sizeof(u));
        *reinterpret_cast<uint2 *>(d) = u;
    }
}

// One padded row per CTA iteration: the row's source is found once, then the
// threads copy its orbitals (coalesced) and zero the padding columns; four at
// a time (vec: N % 4 == 0 and src 16-byte aligned; Npad is a multiple of 32).
template <typename T>
__global__ void __launch_bounds__(256) pad_kernel(const float *__restrict__ src, int src_padded, T *__restrict__ dst,
                                                  const float *__restrict__ scale, int nx, int ny, int nz, int N,
                                                  int Npad, size_t rows, int vec) {
    for (size_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const float *srow = src + source_row(r, nx, ny, nz, src_padded) * N;
        T *drow = dst + r * Npad;
        if (vec) {
#pragma unroll 2
            for (int q = threadIdx.x; q < Npad / 4; q += blockDim.x) {
                const bool in = 4 * q < N;
                const float4 v = in ? __ldg(reinterpret_cast<const float4 *>(srow) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 sc = in ? __ldg(reinterpret_cast<const float4 *>(scale) + q) : make_float4(1.f, 1.f, 1.f, 1.f);
                store4<T>(drow + 4 * q, v, sc);
            }
        } else {
            for (int n = threadIdx.x; n < Npad; n += blockDim.x)
                drow[n] = encode<T>(n < N ? srow[n] : 0.f, n < N ? scale[n] : 1.f);
        }
    }
}

// One CTA waits on an mbarrier that nothing ever arrives at: the bounded wait
// must give up after limit_ns, record the timeout and let the kernel return.
__global__ void wait_selftest_kernel(int *status, unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    mbar_wait_bounded(&bar, 0, status, limit_ns);
}

// Read-bandwidth probe: every thread streams 16-byte vectors (grid-stride,
// four independent loads per round) with loads that allocate in L2 but not in
// L1, so a buffer smaller than L2 measures L2 bandwidth after its first pass.
// The sum goes to *sink only if it equals a value it never takes, which keeps
// the loads alive without a store per thread.
// The buffer is read `passes` times per launch, so a small (L2-sized) buffer
// still gives a launch long enough that launch latency does not count.
__global__ void __launch_bounds__(512)
    read_probe_kernel(const float4 *__restrict__ buf, size_t n16, int passes, float *sink) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    float acc = 0.f;
    for (int pass = 0; pass < passes; ++pass) {
        size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            float4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride), c = __ldcg(buf + i + 2 * stride),
                   d = __ldcg(buf + i + 3 * stride);
            acc += (a.x + b.y) + (c.z + d.w);
        }
        for (; i < n16; i += stride) acc += __ldcg(buf + i).x;
    }
    if (acc == -1.2345e30f) *sink = acc;
}

// ---------------------------------------------------------------------------
// Cell-sorted evaluation order: one CTA counting-sorts the positions by the
// Morton code of their coarse cell (i >> shift, j >> shift, k >> shift).
// ---------------------------------------------------------------------------
// Launched with the programmatic serialization attribute: it may start while the previous kernel in the
// stream (the previous call's evaluation) drains, and waits for it only before it writes perm.
__global__ void __launch_bounds__(kOrderThreads) cell_order_kernel(const EvalArgs A, int shift, int nbins, int *perm) {
    pdl_trigger();
    extern __shared__ int hist[];  // nbins counters, then (npos <= kOrderKeyCache) npos cached keys
    __shared__ int wsum[32];
    __shared__ float G[9];
    if (threadIdx.x < 9) G[threadIdx.x] = A.Gf[threadIdx.x];
    __syncthreads();
    int *keys = A.npos <= kOrderKeyCache ? hist + nbins : nullptr;
    block_cell_sort(A.x, A.y, A.z, A.npos, A.nx, A.ny, A.nz, shift, nbins, perm, hist, wsum, A.lattice ? G : nullptr,
                    keys);
}

// ---------------------------------------------------------------------------
// The same order for many positions, on many CTAs: keys and a histogram in
// global memory (order_keys_kernel), a one-CTA exclusive scan of the bins
// (order_scan_kernel), and a scatter that claims slots with atomics
// (order_scatter_kernel). The order of positions within one coarse cell then
// varies from run to run; each position's outputs do not depend on it.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) order_keys_kernel(const EvalArgs A, int shift, int *keys, int *hist) {
    __shared__ float G[9];
    if (threadIdx.x < 9) G[threadIdx.x] = A.Gf[threadIdx.x];
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < A.npos; p += stride) {
        const int k = cell_key(A.x, A.y, A.z, (int)p, A.nx, A.ny, A.nz, shift, A.lattice ? G : nullptr);
        keys[p] = k;
        atomicAdd(&hist[k], 1);
    }
}

// offsets = exclusive prefix sum of hist (nbins <= kOrderMaxBins), one CTA.
__global__ void __launch_bounds__(1024) order_scan_kernel(const int *hist, int *offsets, int nbins) {
    pdl_wait();
    pdl_trigger();
    __shared__ int bins[kOrderMaxBins];
    __shared__ int wsum[32];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) bins[b] = hist[b];
    __syncthreads();
    block_scan_bins(bins, nbins, wsum);
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) offsets[b] = bins[b];
}

// perm[slot] = position, each position taking the next slot of its bin. A slot
// at or past npos (which a correct histogram never yields) is not written and
// sets the table's status to BSPLINE_ERR_BOUNDS.
__global__ void __launch_bounds__(256) order_scatter_kernel(const int *keys, int npos, int *offsets, int *perm,
                                                            int *status) {
    pdl_wait();
    pdl_trigger();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npos; p += stride) {
        const int slot = atomicAdd(&offsets[keys[p]], 1);
        if (slot >= 0 && slot < npos)
            perm[slot] = (int)p;
        else
            atomicCAS(status, 0, (int)BSPLINE_ERR_BOUNDS);
    }
}

bool current_device_is(bspline_t t) {
    int d = -1;
    return cudaGetDevice(&d) == cudaSuccess && d == t->device;
}

bspline_status fill_table(bspline_t t, const float *src, int on_device, int src_padded, void *stream) {
    if (!t || !src) return BSPLINE_ERR_ARG;
    if (!current_device_is(t)) return BSPLINE_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t src_rows = src_padded ? t->rows : (size_t)t->nx * t->ny * t->nz;
    const size_t src_bytes = src_rows * t->N * sizeof(float);
    const float *dsrc = src;
    float *tmp = nullptr;
    cudaError_t e;
    if (!on_device) {
        e = cudaMalloc(&tmp, src_bytes);
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaMemcpyAsync(tmp, src, src_bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cuda_status(e);
        }
        dsrc = tmp;
    }
    unsigned *bits = reinterpret_cast<unsigned *>(t->scale);
    const int reduced = t->dtype != BSPLINE_F32;
    bspline_status st = BSPLINE_OK;
    e = cudaMemsetAsync(bits, 0, sizeof(float) * t->Npad, s);
    if (e == cudaSuccess && reduced) {
        const bool vec = t->N % 4 == 0 && reinterpret_cast<uintptr_t>(dsrc) % 16 == 0;
        const int cols = vec ? 128 : 32;  // orbitals per CTA
        const unsigned gx = (unsigned)((t->N + cols - 1) / cols);
        // about 8 CTAs per SM in all, each warp over at least 32 rows
        const size_t gy = std::max<size_t>(1, std::min<size_t>(src_rows / 256, ((size_t)t->num_sms * 8 + gx - 1) / gx));
        dim3 grid(gx, (unsigned)std::min<size_t>(gy, 65535));
        if (vec)
            absmax_kernel<4><<<grid, 256, 0, s>>>(dsrc, src_rows, t->N, bits);
        else
            absmax_kernel<1><<<grid, 256, 0, s>>>(dsrc, src_rows, t->N, bits);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        finalize_scale_kernel<<<(t->Npad + 255) / 256, 256, 0, s>>>(bits, t->N, t->Npad, reduced);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const size_t rows = t->rows;
        const unsigned blocks = (unsigned)std::min<size_t>(rows, (size_t)t->num_sms * 32);
        const int vec = t->N % 4 == 0 && reinterpret_cast<uintptr_t>(dsrc) % 16 == 0;
        switch (t->dtype) {
            case BSPLINE_F32:
                pad_kernel<float><<<blocks, 256, 0, s>>>(dsrc, src_padded, static_cast<float *>(t->table), t->scale,
                                                         t->nx, t->ny, t->nz, t->N, t->Npad, rows, vec);
                break;
            case BSPLINE_F16:
                pad_kernel<__half><<<blocks, 256, 0, s>>>(dsrc, src_padded, static_cast<__half *>(t->table),
                                                          t->scale, t->nx, t->ny, t->nz, t->N, t->Npad, rows, vec);
                break;
            default:
                pad_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(dsrc, src_padded,
                                                                 static_cast<__nv_bfloat16 *>(t->table), t->scale,
                                                                 t->nx, t->ny, t->nz, t->N, t->Npad, rows, vec);
        }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = cuda_status(e);
    if (tmp) {
        cudaError_t e2 = cudaStreamSynchronize(s);
        cudaFree(tmp);
        if (st == BSPLINE_OK && e2 != cudaSuccess) st = cuda_status(e2);
    }
    if (st == BSPLINE_OK) t->has_coefs = 1;
    return st;
}

// Measured on a 48^3 grid, 4096 sorted positions: for 16-bit tables the
// tensor-core variant (256-orbital units) is faster for VGL and VGH once a row
// holds 640 orbitals (FP16 VGH 57.2 against 70.0 us, BF16 61.9 against 70.0),
// and for FP16 already at 512 (VGL 42.9 against 48.3 us, VGH 46.5 against
// 49.0); BF16 at 512 is slower on it (VGH 58.6 against 48.8 us), and so is
// either type at 384 or below, where a position fills less than one unit. V
// stays on DIRECT (one output row does not cover the per-unit pipeline cost).
//
// Positions are cell-sorted (order 1) when the table is larger than L2: nearby
// positions then read their shared stencil rows from L2 instead of DRAM (FP32
// VGH at 48^3 x 2048: 0.349 -> 0.219 ms per 4096 positions). A table that
// fits in L2 gains nothing from it and pays for the sort (48 x 48 x 60 x 128,
// 4096 positions: 33 against 42 us).
bspline_tuning default_tuning(int dtype, int kind, int Npad, bool exceeds_l2) {
    bspline_tuning tu{};
    tu.order = exceeds_l2 ? 1 : 0;
    if (kind != BSPLINE_V && (dtype == BSPLINE_F16 ? Npad >= 512 : dtype == BSPLINE_BF16 && Npad > 512)) {
        // 2 CTAs per SM, the deepest ring that fits; units of two 128-orbital blocks, which halve the
        // hand-offs between producer, MMA lane and epilogue per orbital (FP16 at 48^3, 4096 sorted
        // positions, 128 -> 256 orbitals per unit: VGH 142.3 -> 132.0 us at N = 2048, 319.5 -> 304.6 at
        // 4096; VGL 131.6 -> 111.5 at 2048; VGH ratio sums 138.5 -> 125.3)
        tu.variant = BSPLINE_VARIANT_MMA;
        tu.nb = 256;
        tu.ppc = 2;
        return tu;
    }
    tu.variant = BSPLINE_VARIANT_DIRECT;
    tu.nb = 512;
    tu.ppc = 0;  // chosen per call from the number of positions (auto_ppc)
    // FP32 VGH and VGL: rows staged through a 4-unit shared-memory ring, 5 CTAs per SM (sorted steps at
    // 48^3 x 2048, 4096 positions: VGH 0.214 ms against 0.217 with a 6-unit ring at 4 CTAs per SM and
    // 0.222 with loads into registers; VGL 0.190 against 0.194 and 0.198). V is no faster staged.
    // Rows of at most 256 orbitals use the grouped staged kernel (4 CTAs per SM) where it measured
    // faster than the grouped register kernel: VGH at every width (48 x 48 x 60 x 128: 279 -> 160 us
    // at 65536 positions, 19.3 -> 15.0 us at 4096; 48^3 x 256: 37.9 -> 35.9 us; 16^3 x 64 at 16384
    // positions: 24.0 -> 23.6 us), VGL and V only at 128 orbitals (VGL 222 -> 140 us, V 167 -> 110 us;
    // 64 and 256 orbitals were 2-5 % slower staged).
    // (Rows of 65..128 orbitals share the 128-orbital layout: one warp per position.)
    const bool warp_rows = Npad > 64 && Npad <= 128;
    if (dtype == BSPLINE_F32 && kind == BSPLINE_VGH) tu.stages = 4;
    if (dtype == BSPLINE_F32 && kind == BSPLINE_VGL && (Npad > 256 || warp_rows)) tu.stages = 4;
    if (dtype == BSPLINE_F32 && kind == BSPLINE_V && warp_rows) tu.stages = 4;
    return tu;
}

// Fill zero fields with defaults and check the shape is one the library has kernels for.
bspline_status resolve_tuning(bspline_t t, int kind, const bspline_tuning &in, bspline_tuning *out) {
    bspline_tuning tu = in;
    if (tu.variant == BSPLINE_VARIANT_AUTO) tu = t->tuning[kind];
    if (tu.variant == BSPLINE_VARIANT_AUTO) tu = default_tuning(t->dtype, kind, t->Npad, t->table_bytes > t->l2_bytes);
    if (tu.variant == BSPLINE_VARIANT_DIRECT) {
        if (tu.nb == 0) tu.nb = 512;
        if (tu.nb != 256 && tu.nb != 512 && tu.nb != 1024) return BSPLINE_ERR_ARG;
        if (tu.ppc < 0 || tu.ppc > kMaxPpc) return BSPLINE_ERR_ARG;  // 0: chosen per call
        // stages: 0 = loads into registers; 3, 4, 6 or 8 = rows staged through shared memory (FP32)
        if (tu.stages != 0 && tu.stages != 3 && tu.stages != 4 && tu.stages != 6 && tu.stages != 8)
            return BSPLINE_ERR_ARG;
        if (tu.stages != 0 && (t->dtype != BSPLINE_F32 || tu.nb != 512)) return BSPLINE_ERR_UNSUPPORTED;
        if (tu.order < 0 || tu.order > 1) return BSPLINE_ERR_ARG;
    } else if (tu.variant == BSPLINE_VARIANT_TMA) {
        if (tu.nb == 0) tu.nb = 256;
        if (tu.nb != 128 && tu.nb != 256) return BSPLINE_ERR_ARG;
        if (tu.stages == 0) tu.stages = default_stages(t->dtype, tu.nb);
        if (tu.ppc == 0) tu.ppc = 1;
        if (tu.stages < 2 || tu.stages > 16) return BSPLINE_ERR_ARG;
        if (tu.ppc < 1 || tu.ppc > 8) return BSPLINE_ERR_ARG;
        if (tma_smem_bytes(t->dtype, tu.nb, tu.stages) > 227u * 1024u) return BSPLINE_ERR_ARG;
        if (tu.order < 0 || tu.order > 1) return BSPLINE_ERR_ARG;
    } else if (tu.variant == BSPLINE_VARIANT_MMA) {
        if (t->dtype == BSPLINE_F32) return BSPLINE_ERR_UNSUPPORTED;  // 16-bit tables only
        if (tu.nb == 0) tu.nb = 128;
        if (tu.ppc == 0) tu.ppc = 2;
        if ((tu.nb != 128 && tu.nb != 256) || tu.ppc < 1 || tu.ppc > 2) return BSPLINE_ERR_ARG;
        if (tu.stages == 0)  // the deepest ring up to 6 units that lets ppc CTAs share an SM
            for (tu.stages = 6; tu.stages > 2 && !mma_fits(t->dtype, tu.stages, t->Npad, tu.ppc, tu.nb); --tu.stages) {
            }
        if (tu.stages < 2 || tu.stages > 8 || !mma_fits(t->dtype, tu.stages, t->Npad, tu.ppc, tu.nb))
            return BSPLINE_ERR_ARG;
        if (tu.order < 0 || tu.order > 1) return BSPLINE_ERR_ARG;
    } else {
        return BSPLINE_ERR_ARG;
    }
    *out = tu;
    return BSPLINE_OK;
}

}  // namespace

namespace bsg {
// An FP32 table whose rows were written in place by a kernel of the caller's (the interpolation
// solve's last pass): unit per-orbital scales, and the table marked filled.
bspline_status finish_f32_table(bspline_t t, cudaStream_t s) {
    if (t->dtype != BSPLINE_F32) return BSPLINE_ERR_DTYPE;
    finalize_scale_kernel<<<(t->Npad + 255) / 256, 256, 0, s>>>(reinterpret_cast<unsigned *>(t->scale), t->N,
                                                                 t->Npad, 0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    t->has_coefs = 1;
    return BSPLINE_OK;
}

// Lattice fields of the launch arguments (general cell, if one is set).
void fill_lattice(bspline_t t, EvalArgs &A) {
    A.lattice = t->lattice;
    if (!t->lattice) return;
    for (int k = 0; k < 9; ++k) {
        A.G[k] = t->G[k];
        A.Gf[k] = (float)t->G[k];
    }
    double M[3][3];  // M = G^T G: trace(G H G^T) = sum_de M[d][e] H[d][e]
    for (int d = 0; d < 3; ++d)
        for (int e = 0; e < 3; ++e) {
            M[d][e] = 0.0;
            for (int i = 0; i < 3; ++i) M[d][e] += t->G[i * 3 + d] * t->G[i * 3 + e];
        }
    A.lapw[0] = (float)M[0][0];
    A.lapw[1] = (float)(2.0 * M[0][1]);
    A.lapw[2] = (float)(2.0 * M[0][2]);
    A.lapw[3] = (float)M[1][1];
    A.lapw[4] = (float)(2.0 * M[1][2]);
    A.lapw[5] = (float)M[2][2];
}

// Cell-sorted evaluation order for A: sorts A's positions into perm_scratch
// (order_scratch_ints(A.npos) ints) if given, else into the handle's scratch,
// and points A.perm at the result. Up to kOrderMultiMin positions one CTA
// sorts (launched to overlap the previous kernel, see cell_order_kernel);
// above, the many-CTA sort.
// Grows t->perm to npos positions; the caller holds t->mu. sync: what to wait for before the old
// scratch is freed (a stream, or the whole device when null and device_wide).
static bspline_status grow_order_scratch(bspline_t t, size_t npos, cudaStream_t sync, bool device_wide) {
    if (t->perm_cap >= npos) return BSPLINE_OK;
    cudaError_t e = device_wide ? cudaDeviceSynchronize() : cudaStreamSynchronize(sync);  // old scratch in use
    if (e != cudaSuccess) return cuda_status(e);
    cudaFree(t->perm);
    t->perm = nullptr;
    t->perm_cap = 0;
    e = cudaMalloc(&t->perm, sizeof(int) * order_scratch_ints(npos));
    if (e != cudaSuccess) return cuda_status(e);
    t->perm_cap = npos;
    return BSPLINE_OK;
}

bspline_status reserve_order_scratch(bspline_t t, size_t npos) {
    if (!t) return BSPLINE_ERR_ARG;
    std::lock_guard<std::mutex> g(t->mu);
    return grow_order_scratch(t, npos, nullptr, true);
}

bspline_status apply_order(bspline_t t, EvalArgs &A, cudaStream_t s, int *perm_scratch) {
    std::unique_lock<std::mutex> g(t->mu, std::defer_lock);
    int *perm = perm_scratch;  // caller-owned scratch (order_scratch_ints), else the handle's
    if (!perm) {
        g.lock();
        bspline_status st = grow_order_scratch(t, (size_t)A.npos, s, false);
        if (st != BSPLINE_OK) return st;
    }
    if (!perm) perm = t->perm;
    int shift = 0, nbins = 0;
    order_bins(t->nx, t->ny, t->nz, &shift, &nbins);
    if (A.npos > kOrderMultiMin) {
        int *keys = perm + A.npos, *hist = keys + A.npos, *offsets = hist + kOrderMaxBins;
        const unsigned grid = (unsigned)std::min<long long>(((long long)A.npos + 1023) / 1024, (long long)t->num_sms * 8);
        cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * nbins, s);
        if (e == cudaSuccess) {
            order_keys_kernel<<<grid, 256, 0, s>>>(A, shift, keys, hist);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = launch_k(order_scan_kernel, 1, 1024, 0, s, true, hist, offsets, nbins);
        if (e == cudaSuccess)
            e = launch_k(order_scatter_kernel, grid, 256, 0, s, true, keys, A.npos, offsets, perm, A.status);
        if (e != cudaSuccess) return cuda_status(e);
        A.perm = perm;
        return BSPLINE_OK;
    }
    static bool attr_set = false;  // idempotent; a race only repeats the call
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(cell_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(int) * (kOrderMaxBins + kOrderKeyCache)));
        if (e != cudaSuccess) return cuda_status(e);
        attr_set = true;
    }
    const size_t smem = sizeof(int) * (nbins + (A.npos <= kOrderKeyCache ? A.npos : 0));
    cudaError_t e = launch_k(cell_order_kernel, 1, kOrderThreads, smem, s, true, A, shift, nbins, perm);
    if (e != cudaSuccess) return cuda_status(e);
    A.perm = perm;
    return BSPLINE_OK;
}

// Launch one single-table evaluation (used by the eval entry points, the
// host-buffer path and the autotuner).
bspline_status launch_eval(bspline_t t, int kind, const bspline_tuning &want, int npos, const double *x,
                           const double *y, const double *z, float *o0, float *o1, float *o2, int ld, cudaStream_t s,
                           int *perm_scratch) {
    bspline_tuning tu;
    bspline_status st = resolve_tuning(t, kind, want, &tu);
    if (st != BSPLINE_OK) return st;
    if (npos == 0) return BSPLINE_OK;
    EvalArgs A;
    memset(&A, 0, sizeof A);
    A.table = t->table;
    A.scale = t->scale;
    A.nx = t->nx;
    A.ny = t->ny;
    A.nz = t->nz;
    A.N = t->N;
    A.Npad = t->Npad;
    A.sj = (long long)(t->nz + 3) * t->Npad;
    A.si = (long long)(t->ny + 3) * A.sj;
    A.npos = npos;
    A.x = x;
    A.y = y;
    A.z = z;
    A.o0 = o0;
    A.o1 = o1;
    A.o2 = o2;
    A.ld = ld;
    A.status = t->status;
    A.perm = nullptr;
    fill_lattice(t, A);
    if (tu.order == 1 && npos > 1) {
        st = apply_order(t, A, s, perm_scratch);
        if (st != BSPLINE_OK) return st;
    }
    const CUtensorMap *map = nullptr;
    if (tu.variant == BSPLINE_VARIANT_TMA || tu.variant == BSPLINE_VARIANT_MMA) {
        if (A.lattice && tu.variant == BSPLINE_VARIANT_TMA) return BSPLINE_ERR_UNSUPPORTED;  // fractional only
        st = tu.variant == BSPLINE_VARIANT_TMA ? get_tma_map(t, tu.nb, 0, &map) : get_tma_map(t, 64, 1, &map);
        if (st != BSPLINE_OK) return st;
    }
    switch (t->dtype) {
        case BSPLINE_F32: return launch_eval_f32(kind, tu, A, map, t->num_sms, s);
        case BSPLINE_F16: return launch_eval_f16(kind, tu, A, map, t->num_sms, s);
        case BSPLINE_BF16: return launch_eval_bf16(kind, tu, A, map, t->num_sms, s);
        default: return BSPLINE_ERR_DTYPE;
    }
}
}  // namespace bsg

namespace {

bspline_status check_eval_args(bspline_t t, int npos, const double *x, const double *y, const double *z,
                               const float *o0, const float *o1, const float *o2, int kind, int ld) {
    if (!t) return BSPLINE_ERR_ARG;
    if (!t->has_coefs) return BSPLINE_ERR_STATE;
    if (npos < 0 || ld < t->N) return BSPLINE_ERR_ARG;
    if (npos == 0) return BSPLINE_OK;
    if (!x || !y || !z || !o0) return BSPLINE_ERR_ARG;
    if (kind != BSPLINE_V && (!o1 || !o2)) return BSPLINE_ERR_ARG;
    if (!current_device_is(t)) return BSPLINE_ERR_ARG;
    return BSPLINE_OK;
}

}  // namespace

extern "C" {

int bspline_abi_version(void) { return BSPLINE_ABI_VERSION; }

const char *bspline_status_str(bspline_status s) {
    switch (s) {
        case BSPLINE_OK: return "ok";
        case BSPLINE_ERR_ARG: return "invalid argument";
        case BSPLINE_ERR_ALLOC: return "allocation failed";
        case BSPLINE_ERR_CUDA: return "CUDA error";
        case BSPLINE_ERR_DTYPE: return "unsupported element type";
        case BSPLINE_ERR_STATE: return "table has no coefficients";
        case BSPLINE_ERR_TIMEOUT: return "device wait timed out";
        case BSPLINE_ERR_UNSUPPORTED: return "unsupported on this device";
        case BSPLINE_ERR_BOUNDS: return "device-side index check failed";
        default: return "unknown status";
    }
}

bspline_status bspline_create(int nx, int ny, int nz, int N, int dtype, bspline_t *out) {
    if (!out) return BSPLINE_ERR_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || N < 1 || N > (1 << 20)) return BSPLINE_ERR_ARG;
    if (dtype != BSPLINE_F32 && dtype != BSPLINE_F16 && dtype != BSPLINE_BF16) return BSPLINE_ERR_DTYPE;
    if ((long long)(nx + 3) * (ny + 3) * (nz + 3) > (1LL << 31)) return BSPLINE_ERR_ARG;
    bspline_s *t = new (std::nothrow) bspline_s();
    if (!t) return BSPLINE_ERR_ALLOC;
    t->nx = nx;
    t->ny = ny;
    t->nz = nz;
    t->N = N;
    t->dtype = dtype;
    t->esize = dtype == BSPLINE_F32 ? 4 : 2;
    const int row_elems = 128 / t->esize;  // 128-byte rows
    t->Npad = (N + row_elems - 1) / row_elems * row_elems;
    t->rows = (size_t)(nx + 3) * (ny + 3) * (nz + 3);
    t->table_bytes = t->rows * t->Npad * t->esize;
    for (int k = 0; k < 3; ++k) t->tuning[k] = bspline_tuning{0, 0, 0, 0};
    cudaError_t e = cudaGetDevice(&t->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, t->device);
    int l2 = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, t->device);
    t->l2_bytes = (size_t)l2;
    if (e == cudaSuccess) e = cudaMalloc(&t->table, t->table_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&t->scale, sizeof(float) * t->Npad);
    if (e == cudaSuccess) e = cudaMalloc(&t->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(t->status, 0, sizeof(int));
    if (e != cudaSuccess) {
        bspline_destroy(t);
        return cuda_status(e);
    }
    *out = t;
    return BSPLINE_OK;
}

bspline_status bspline_destroy(bspline_t t) {
    if (!t) return BSPLINE_ERR_ARG;
    cudaDeviceSynchronize();
    cudaFree(t->table);
    cudaFree(t->scale);
    cudaFree(t->status);
    cudaFree(t->perm);
    for (int k = 0; k < 2; ++k) {
        cudaFree(t->staging.d_pos[k]);
        cudaFree(t->staging.d_out[k]);
        cudaFree(t->staging.d_perm[k]);
        cudaFree(t->staging.d_perm_direct);
        t->staging.d_perm_direct = nullptr;
        if (t->staging.stream[k]) cudaStreamDestroy(t->staging.stream[k]);
    }
    delete t;
    return BSPLINE_OK;
}

bspline_status bspline_set_coefs(bspline_t t, const float *coefs, int on_device, void *stream) {
    return fill_table(t, coefs, on_device, 0, stream);
}

bspline_status bspline_set_coefs_padded(bspline_t t, const float *padded, int on_device, void *stream) {
    return fill_table(t, padded, on_device, 1, stream);
}

bspline_status bspline_get_info(bspline_t t, bspline_info *out) {
    if (!t || !out) return BSPLINE_ERR_ARG;
    out->nx = t->nx;
    out->ny = t->ny;
    out->nz = t->nz;
    out->N = t->N;
    out->Npad = t->Npad;
    out->dtype = t->dtype;
    out->table_bytes = t->table_bytes;
    out->has_coefs = t->has_coefs;
    return BSPLINE_OK;
}

bspline_status bspline_get_table(bspline_t t, void *dst, float *scale) {
    if (!t || !dst) return BSPLINE_ERR_ARG;
    if (!t->has_coefs) return BSPLINE_ERR_STATE;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy2D(dst, (size_t)t->N * t->esize, t->table, (size_t)t->Npad * t->esize, (size_t)t->N * t->esize,
                         t->rows, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && scale) e = cudaMemcpy(scale, t->scale, sizeof(float) * t->N, cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

bspline_status bspline_eval_v(bspline_t t, int npos, const double *x, const double *y, const double *z, float *v,
                              int ld, void *stream) {
    bspline_status st = check_eval_args(t, npos, x, y, z, v, nullptr, nullptr, BSPLINE_V, ld);
    if (st != BSPLINE_OK || npos == 0) return st;
    return launch_eval(t, BSPLINE_V, bspline_tuning{0, 0, 0, 0}, npos, x, y, z, v, nullptr, nullptr, ld,
                       static_cast<cudaStream_t>(stream));
}

bspline_status bspline_eval_vgl(bspline_t t, int npos, const double *x, const double *y, const double *z, float *v,
                                float *g, float *l, int ld, void *stream) {
    bspline_status st = check_eval_args(t, npos, x, y, z, v, g, l, BSPLINE_VGL, ld);
    if (st != BSPLINE_OK || npos == 0) return st;
    return launch_eval(t, BSPLINE_VGL, bspline_tuning{0, 0, 0, 0}, npos, x, y, z, v, g, l, ld,
                       static_cast<cudaStream_t>(stream));
}

bspline_status bspline_eval_vgh(bspline_t t, int npos, const double *x, const double *y, const double *z, float *v,
                                float *g, float *h, int ld, void *stream) {
    bspline_status st = check_eval_args(t, npos, x, y, z, v, g, h, BSPLINE_VGH, ld);
    if (st != BSPLINE_OK || npos == 0) return st;
    return launch_eval(t, BSPLINE_VGH, bspline_tuning{0, 0, 0, 0}, npos, x, y, z, v, g, h, ld,
                       static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace {

// Device-usable address of a host buffer, or null if the GPU cannot reach it:
// pinned (page-locked, mapped) memory through its device alias, pageable
// memory only where the device reads the host's page tables (e.g. over
// NVLink-C2C on Grace-based nodes), device or managed memory as is.
const void *device_alias(const void *p, bool pageable_ok) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    return pageable_ok ? p : nullptr;
}

// Host buffers the kernel reads and writes in place (no staging copies).
bspline_status eval_host_direct(bspline_t t, int kind, int npos, const double *x, const double *y, const double *z,
                                float *v, float *g, float *hl, int ld, bool *used) {
    *used = false;
    HostStaging &S = t->staging;
    int pageable = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, t->device) != cudaSuccess) pageable = 0;
    const void *ptr[6] = {x, y, z, v, g, hl};
    const void *dev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    const int nptr = kind == BSPLINE_V ? 4 : 6;
    for (int k = 0; k < nptr; ++k) {
        dev[k] = device_alias(ptr[k], pageable != 0);
        if (!dev[k]) return BSPLINE_OK;  // not reachable: the caller stages instead
    }
    cudaError_t e = cudaSuccess;
    if (!S.stream[0]) e = cudaStreamCreateWithFlags(&S.stream[0], cudaStreamNonBlocking);
    if (e == cudaSuccess && S.direct_cap < (size_t)npos) {
        e = cudaStreamSynchronize(S.stream[0]);
        cudaFree(S.d_perm_direct);
        S.d_perm_direct = nullptr;
        S.direct_cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&S.d_perm_direct, sizeof(int) * order_scratch_ints((size_t)npos));
        if (e == cudaSuccess) S.direct_cap = (size_t)npos;
    }
    if (e != cudaSuccess) return cuda_status(e);
    *used = true;
    bspline_status st = launch_eval(t, kind, bspline_tuning{0, 0, 0, 0, 0}, npos, (const double *)dev[0],
                                    (const double *)dev[1], (const double *)dev[2], (float *)dev[3],
                                    (float *)dev[4], (float *)dev[5], ld, S.stream[0], S.d_perm_direct);
    e = cudaStreamSynchronize(S.stream[0]);
    if (st != BSPLINE_OK) return st;
    return cuda_status(e);
}

}  // namespace

extern "C" {

bspline_status bspline_set_host_mode(bspline_t t, int mode) {
    if (!t || mode < 0 || mode > 2) return BSPLINE_ERR_ARG;
    std::lock_guard<std::mutex> g_(t->staging_mu);
    t->staging.mode = mode;
    return BSPLINE_OK;
}

bspline_status bspline_eval_ratio(bspline_t t, int kind, int npos, const double *x, const double *y,
                                  const double *z, const float *uinv, int ldu, float *ratio, void *stream) {
    if (!t || kind < BSPLINE_V || kind > BSPLINE_VGH) return BSPLINE_ERR_ARG;
    if (!t->has_coefs) return BSPLINE_ERR_STATE;
    if (npos < 0 || ldu < t->N) return BSPLINE_ERR_ARG;
    if (npos == 0) return BSPLINE_OK;
    if (!x || !y || !z || !uinv || !ratio) return BSPLINE_ERR_ARG;
    if (!current_device_is(t)) return BSPLINE_ERR_ARG;
    bspline_tuning tu;
    bspline_status st = resolve_tuning(t, kind, bspline_tuning{0, 0, 0, 0, 0}, &tu);
    if (st != BSPLINE_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    EvalArgs A;
    memset(&A, 0, sizeof A);
    A.table = t->table;
    A.scale = t->scale;
    A.nx = t->nx;
    A.ny = t->ny;
    A.nz = t->nz;
    A.N = t->N;
    A.Npad = t->Npad;
    A.sj = (long long)(t->nz + 3) * t->Npad;
    A.si = (long long)(t->ny + 3) * A.sj;
    A.npos = npos;
    A.x = x;
    A.y = y;
    A.z = z;
    A.status = t->status;
    fill_lattice(t, A);
    if (tu.order == 1 && npos > 1) {
        st = apply_order(t, A, s, nullptr);
        if (st != BSPLINE_OK) return st;
    }
    if (tu.variant == BSPLINE_VARIANT_MMA) {  // 16-bit tables on the tensor cores
        const CUtensorMap *map = nullptr;
        st = get_tma_map(t, 64, 1, &map);
        if (st != BSPLINE_OK) return st;
        if (t->dtype == BSPLINE_F16) return launch_ratio_mma_f16(kind, tu, A, map, t->num_sms, uinv, ldu, ratio, s);
        return launch_ratio_mma_bf16(kind, tu, A, map, t->num_sms, uinv, ldu, ratio, s);
    }
    switch (t->dtype) {
        case BSPLINE_F32: return launch_ratio_f32(kind, A, uinv, ldu, ratio, s);
        case BSPLINE_F16: return launch_ratio_f16(kind, A, uinv, ldu, ratio, s);
        case BSPLINE_BF16: return launch_ratio_bf16(kind, A, uinv, ldu, ratio, s);
        default: return BSPLINE_ERR_DTYPE;
    }
}

bspline_status bspline_eval_host(bspline_t t, int kind, int npos, const double *x, const double *y, const double *z,
                                 float *v, float *g, float *hl, int ld) {
    if (kind < BSPLINE_V || kind > BSPLINE_VGH) return BSPLINE_ERR_ARG;
    bspline_status st = check_eval_args(t, npos, x, y, z, v, g, hl, kind, ld);
    if (st != BSPLINE_OK || npos == 0) return st;
    const int ncomp = nout_of(kind);
    const size_t per_pos = (size_t)ncomp * ld;  // floats
    std::lock_guard<std::mutex> g_(t->staging_mu);
    HostStaging &S = t->staging;
    if (S.mode != 1) {
        bool used = false;
        st = eval_host_direct(t, kind, npos, x, y, z, v, g, hl, ld, &used);
        if (used || st != BSPLINE_OK) return st;
        if (S.mode == 2) return BSPLINE_ERR_UNSUPPORTED;  // direct access asked for but not possible
    }
    // Chunks of about 32 MB of outputs, at least 64 positions.
    size_t chunk = std::max<size_t>(64, ((size_t)32 << 20) / (per_pos * sizeof(float)));
    chunk = std::min<size_t>(chunk, (size_t)npos);
    cudaError_t e = cudaSuccess;
    if (S.pos_cap < chunk || S.out_cap < chunk * per_pos) {
        e = cudaDeviceSynchronize();  // earlier calls may still use the old buffers
        for (int k = 0; k < 2; ++k) {
            cudaFree(S.d_pos[k]);
            cudaFree(S.d_out[k]);
            cudaFree(S.d_perm[k]);
            S.d_pos[k] = nullptr;
            S.d_out[k] = nullptr;
            S.d_perm[k] = nullptr;
        }
        S.pos_cap = S.out_cap = 0;
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaMalloc(&S.d_pos[k], sizeof(double) * 3 * chunk);
            if (e == cudaSuccess) e = cudaMalloc(&S.d_out[k], sizeof(float) * chunk * per_pos);
            if (e == cudaSuccess) e = cudaMalloc(&S.d_perm[k], sizeof(int) * order_scratch_ints(chunk));
        }
        if (e != cudaSuccess) return cuda_status(e);
        S.pos_cap = chunk;
        S.out_cap = chunk * per_pos;
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        if (!S.stream[k]) e = cudaStreamCreateWithFlags(&S.stream[k], cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_status(e);

    const size_t nchunks = ((size_t)npos + chunk - 1) / chunk;
    for (size_t c = 0; c < nchunks && st == BSPLINE_OK; ++c) {
        const int k = (int)(c & 1);
        cudaStream_t s = S.stream[k];
        const size_t p0 = c * chunk;
        const int np = (int)std::min(chunk, (size_t)npos - p0);
        double *dx = S.d_pos[k], *dy = dx + chunk, *dz = dy + chunk;
        float *dv = S.d_out[k];
        float *dg = dv + (size_t)np * ld;
        float *dh = kind == BSPLINE_VGL ? dg + (size_t)np * 3 * ld : dg + (size_t)np * 3 * ld;
        if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x + p0, sizeof(double) * np, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y + p0, sizeof(double) * np, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dz, z + p0, sizeof(double) * np, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        st = launch_eval(t, kind, bspline_tuning{0, 0, 0, 0, 0}, np, dx, dy, dz, dv,
                         kind == BSPLINE_V ? nullptr : dg, kind == BSPLINE_V ? nullptr : dh, ld, s, S.d_perm[k]);
        if (st != BSPLINE_OK) break;
        e = cudaMemcpyAsync(v + p0 * ld, dv, sizeof(float) * np * ld, cudaMemcpyDeviceToHost, s);
        if (kind != BSPLINE_V && e == cudaSuccess)
            e = cudaMemcpyAsync(g + p0 * 3 * ld, dg, sizeof(float) * np * 3 * ld, cudaMemcpyDeviceToHost, s);
        if (kind == BSPLINE_VGL && e == cudaSuccess)
            e = cudaMemcpyAsync(hl + p0 * ld, dh, sizeof(float) * np * ld, cudaMemcpyDeviceToHost, s);
        if (kind == BSPLINE_VGH && e == cudaSuccess)
            e = cudaMemcpyAsync(hl + p0 * 6 * ld, dh, sizeof(float) * np * 6 * ld, cudaMemcpyDeviceToHost, s);
    }
    cudaError_t e0 = cudaStreamSynchronize(S.stream[0]);
    cudaError_t e1 = cudaStreamSynchronize(S.stream[1]);
    if (st != BSPLINE_OK) return st;
    if (e == cudaSuccess) e = e0;
    if (e == cudaSuccess) e = e1;
    return cuda_status(e);
}

bspline_status bspline_device_status(bspline_t t, void *stream, int reset) {
    if (!t) return BSPLINE_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, t->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && reset) e = cudaMemsetAsync(t->status, 0, sizeof(int), s);
    if (e == cudaSuccess && reset) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    return (bspline_status)v;
}

bspline_status bspline_set_lattice(bspline_t t, const double *L) {
    if (!t) return BSPLINE_ERR_ARG;
    if (!L) {
        t->lattice = 0;
        return BSPLINE_OK;
    }
    const double a = L[0], b = L[1], c = L[2], d = L[3], e = L[4], f = L[5], g = L[6], h = L[7], i = L[8];
    const double det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
    double scale = 0.0;
    for (int k = 0; k < 9; ++k) {
        if (!std::isfinite(L[k])) return BSPLINE_ERR_ARG;
        scale = std::max(scale, std::fabs(L[k]));
    }
    if (!(std::fabs(det) > 1e-12 * scale * scale * scale)) return BSPLINE_ERR_ARG;  // singular cell
    const double inv[9] = {(e * i - f * h) / det, (c * h - b * i) / det, (b * f - c * e) / det,
                           (f * g - d * i) / det, (a * i - c * g) / det, (c * d - a * f) / det,
                           (d * h - e * g) / det, (b * g - a * h) / det, (a * e - b * d) / det};
    for (int k = 0; k < 9; ++k) {
        t->L[k] = L[k];
        t->G[k] = inv[k];
    }
    t->lattice = 1;
    return BSPLINE_OK;
}

bspline_status bspline_measure_read_bandwidth(size_t bytes, int reps, double *gbs, void *stream) {
    if (!gbs || reps < 1 || reps > 1000 || bytes < 16 || bytes % 16 != 0) return BSPLINE_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);
    float4 *buf = nullptr;
    float *sink = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    e = cudaMalloc(&buf, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, bytes, s);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    std::vector<float> ms;
    const unsigned grid = (unsigned)sms * 4;  // 4 CTAs of 512 threads per SM: 2048 resident threads
    const size_t min_read = (size_t)1 << 30;  // at least 1 GiB per timed launch
    const int passes = (int)std::max<size_t>(1, (min_read + bytes - 1) / bytes);
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // pass 0 warms the caches
        cudaEventRecord(ev[0], s);
        read_probe_kernel<<<grid, 512, 0, s>>>(buf, bytes / 16, passes, sink);
        e = cudaGetLastError();
        cudaEventRecord(ev[1], s);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float m = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&m, ev[0], ev[1]);
        if (r > 0) ms.push_back(m);
    }
    if (e == cudaSuccess) {
        std::sort(ms.begin(), ms.end());
        *gbs = (double)bytes * passes / (ms[ms.size() / 2] * 1e-3) / 1e9;
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    cudaFree(buf);
    cudaFree(sink);
    return cuda_status(e);
}

bspline_status bspline_selftest_wait_timeout(bspline_t t, int limit_us, void *stream) {
    if (!t || limit_us < 1 || limit_us > 2000000) return BSPLINE_ERR_ARG;
    if (!current_device_is(t)) return BSPLINE_ERR_ARG;
    wait_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(t->status,
                                                                          (unsigned long long)limit_us * 1000ull);
    return cuda_status(cudaGetLastError());
}

bspline_status bspline_set_tuning(bspline_t t, int kind, const bspline_tuning *tune) {
    if (!t || !tune || kind < BSPLINE_V || kind > BSPLINE_VGH) return BSPLINE_ERR_ARG;
    if (tune->variant == BSPLINE_VARIANT_AUTO) {
        t->tuning[kind] = bspline_tuning{0, 0, 0, 0};
        return BSPLINE_OK;
    }
    bspline_tuning tu;
    bspline_status st = resolve_tuning(t, kind, *tune, &tu);
    if (st != BSPLINE_OK) return st;
    t->tuning[kind] = tu;
    return BSPLINE_OK;
}

bspline_status bspline_get_tuning(bspline_t t, int kind, bspline_tuning *out) {
    if (!t || !out || kind < BSPLINE_V || kind > BSPLINE_VGH) return BSPLINE_ERR_ARG;
    return resolve_tuning(t, kind, bspline_tuning{0, 0, 0, 0}, out);
}

}  // extern "C"
