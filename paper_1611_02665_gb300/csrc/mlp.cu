// Learned surrogate of a B-spline orbital table: a periodic Fourier-feature
// MLP trained and evaluated with the tcgen05 GEMM of mlp_gemm.cuh. Not in
// arXiv:1611.02665; the spline library produces its targets and judges it.
//
// Layers: features (6*nfreq sin/cos, padded to kin) -> `layers` x [hidden,
// SiLU] -> linear nout. Training: forward with saved pre-activations and
// transposed bf16 copies, MSE loss, backward (dA via W^T, dW via split-K
// over the batch), Adam on FP32 master weights that also refreshes the bf16
// W and W^T copies. Inference: V with one row per position; VGL with 5 rows
// per position (value, 3 first derivatives, Laplacian; fm_row) propagated by
// the forward-mode epilogues.
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "mlp_gemm.cuh"
#include "mlp_surrogate.h"

using namespace mlpk;
using bsg::cuda_status;

namespace {

constexpr int kMaxLayers = 8;

struct LayerDev {
    long long w_off, b_off, wb_off;
    int in, out;
};
struct LayerTable {
    LayerDev l[kMaxLayers];
    int n;
};

}  // namespace

struct mlp_s {
    int nfreq = 0, hidden = 0, layers = 0, nout = 0, kin = 0;
    int device = 0, sms = 0;
    int gemm_kernel = 0;  // mlp_set_gemm_kernel: 0 the library's choice, 1 one CTA per tile, 2 CTA pairs,
                          // 3 two CTAs per SM
    LayerTable lt;
    size_t nparams = 0, nweights = 0;
    float *params = nullptr, *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
    long long step = 0;
    __nv_bfloat16 *wb = nullptr, *wbT = nullptr;
    int *status = nullptr;
    // training workspace (capacity tb rows)
    int tb = 0;
    __nv_bfloat16 *feat = nullptr, *featT = nullptr;
    std::vector<__nv_bfloat16 *> act, actT, d, dT;
    std::vector<float *> z;
    float *out = nullptr;
    float *loss = nullptr;
    float *lossp = nullptr;  // loss_kernel's per-block loss shares (room for the largest batch), then
    unsigned *lcount = nullptr;  // its finished-block counter, at a fixed place after the largest batch's shares
    // inference workspace (capacity ir rows)
    int ir = 0;
    __nv_bfloat16 *ifeat = nullptr, *h[2] = {nullptr, nullptr};
    std::map<std::tuple<const void *, int, int, int>, CUtensorMap> maps;
    // output tensor maps of the TMA-store epilogues: (pointer, rows, columns, row stride, element bytes)
    std::map<std::tuple<const void *, int, int, int, int>, CUtensorMap> omaps;
    std::mutex mu;
};

namespace {

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Features of a position: for axis d and frequency k = 1..nfreq, columns
// d*2*nfreq + 2(k-1) and + 1 hold sin(2 pi k x_d) and cos(2 pi k x_d); the
// columns from 6 nfreq to kin are zero. Row layouts (MODE):
//   kPlainRows  one row per position;
//   kFmRows     forward mode for inference (fm_row): 5 rows per position, value, d/dx_d (d = 0..2), and
//               the Laplacian, whose entries for axis d are d2/dx_d^2 of that axis' features (a feature
//               depends on one coordinate only);
//   kVgRows     training on values and gradients (vg_row): 4 rows per position, value and d/dx_d.
//
// One CTA builds the rows of PB consecutive positions in shared memory and
// writes them out as one contiguous block of 16-byte stores (and, for
// training, the transposed copy FT[f * ldT + row] with consecutive rows in
// consecutive threads). Each coordinate is wrapped into [0, 1) once, in double
// precision; the frequencies follow in single precision (see below). A first version computed each feature in
// its own thread in double precision and took 61 us for 65536 positions on
// GB300's slow FP64 units; one thread per (position, axis) writing straight
// to global memory took 37 us (scattered 4-byte stores).
constexpr int kPlainRows = 0, kFmRows = 1, kVgRows = 2;
// Shared-memory row stride (elements) of the feature kernels' tile: the row plus 16 bytes.
__host__ __device__ constexpr int feat_stride(int kin) { return kin + 8; }
__host__ __device__ constexpr long long feat_rows(int mode, long long npos) {
    return mode == kFmRows ? fm_rows(npos) : (mode == kVgRows ? kVgStreams * npos : npos);
}
__host__ __device__ constexpr long long feat_row(int mode, long long p, int stream) {
    return mode == kFmRows ? fm_row(p, stream) : (mode == kVgRows ? vg_row(p, stream) : p);
}

template <int MODE>
__global__ void __launch_bounds__(256)
    features_kernel(const double *x, const double *y, const double *z, int npos, int nfreq, int kin, int PB,
                    __nv_bfloat16 *F, __nv_bfloat16 *FT, int ldT) {
    bsg::pdl_wait();
    bsg::pdl_trigger();
    constexpr bool FM = MODE != kPlainRows;  // derivative rows
    extern __shared__ __align__(16) unsigned char feat_smem[];
    // [rows][ks]: rows padded by 16 bytes, so that the threads of a warp, which write the same feature
    // column of different rows, spread over the banks instead of sharing one
    const int ks = feat_stride(kin);
    __nv_bfloat16 *tile = reinterpret_cast<__nv_bfloat16 *>(feat_smem);
    const int p0 = blockIdx.x * PB;
    const int np = min(PB, npos - p0);
    const int rows = (int)feat_rows(MODE, np);
    float *cw = reinterpret_cast<float *>(tile + (size_t)feat_rows(MODE, PB) * ks);  // [PB][3]
    const int rw = kin / 8, srw = ks / 8;  // 16-byte words of a row in global / shared memory
    const int words = rows * rw;           // (kin is a multiple of 64)
    uint4 *t4 = reinterpret_cast<uint4 *>(tile);
    for (int i = threadIdx.x; i < rows * srw; i += blockDim.x) t4[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = threadIdx.x; i < np * 3; i += blockDim.x) {
        const int pl = i / 3, d = i % 3;
        const double c = d == 0 ? x[p0 + pl] : (d == 1 ? y[p0 + pl] : z[p0 + pl]);
        cw[i] = (float)(c - floor(c));
    }
    __syncthreads();
    // one thread per (position, axis): sin/cos of 2 pi x from sincospif, then of 2 pi k x for k = 2..nfreq
    // by the angle-addition recurrence (a few float ulps of drift by k = 64, far below the bf16 rounding
    // of the features)
    for (int i = threadIdx.x; i < np * 3; i += blockDim.x) {
        const int pl = i / 3, d = i % 3;
        float s1, c1;
        sincospif(2.f * cw[i], &s1, &c1);
        float sn = s1, cs = c1;
        const size_t r0 = (size_t)feat_row(MODE, pl, 0);
        __nv_bfloat16 *row0 = tile + r0 * ks + d * 2 * nfreq;
        for (int k = 1; k <= nfreq; ++k) {
            __nv_bfloat16 *row = row0 + 2 * (k - 1);
            *reinterpret_cast<__nv_bfloat162 *>(row) = __floats2bfloat162_rn(sn, cs);
            if constexpr (FM) {
                const float w = 6.283185307179586f * (float)k;
                // the derivative rows of position pl follow its value row (both layouts)
                *reinterpret_cast<__nv_bfloat162 *>(row + (size_t)(1 + d) * ks) =
                    __floats2bfloat162_rn(w * cs, -w * sn);
                if constexpr (MODE == kFmRows)
                    *reinterpret_cast<__nv_bfloat162 *>(row + (size_t)4 * ks) =
                        __floats2bfloat162_rn(-w * w * sn, -w * w * cs);
            }
            const float sn_next = fmaf(sn, c1, cs * s1);  // sin(a + b) = sin a cos b + cos a sin b
            cs = fmaf(cs, c1, -(sn * s1));                // cos(a + b) = cos a cos b - sin a sin b
            sn = sn_next;
        }
    }
    __syncthreads();
    const size_t rbase = (size_t)feat_rows(MODE, p0);
    uint4 *dst = reinterpret_cast<uint4 *>(F + rbase * kin);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = t4[(i / rw) * srw + i % rw];
    if (MODE != kFmRows && FT)
        for (int i = threadIdx.x; i < kin * rows; i += blockDim.x) {
            const int f = i / rows, rl = i % rows;
            FT[(size_t)f * ldT + rbase + rl] = tile[(size_t)rl * ks + f];
        }
}

// Positions per CTA (for the inference forward mode a multiple of 6: whole groups of 32 rows) and dynamic
// shared memory of the feature kernels.
inline int feature_block(int mode) { return mode == kFmRows ? 12 : (mode == kVgRows ? 16 : 64); }
inline size_t feature_smem(int mode, int kin) {
    const int pb = feature_block(mode);
    return (size_t)feat_rows(mode, pb) * feat_stride(kin) * 2 + (size_t)pb * 3 * 4;
}

template <int MODE>
cudaError_t launch_features(const double *x, const double *y, const double *z, int npos, int nfreq, int kin,
                            __nv_bfloat16 *F, __nv_bfloat16 *FT, int ldT, cudaStream_t s) {
    static bool attr_set = false;  // idempotent; a race only repeats the call
    const size_t smem = feature_smem(MODE, kin);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(features_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)feature_smem(MODE, 448));  // kin <= 448 (nfreq <= 64)
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int pb = feature_block(MODE);
    return bsg::launch_k(features_kernel<MODE>, (unsigned)((npos + pb - 1) / pb), 256, smem, s, true, x, y, z,
                         npos, nfreq, kin, pb, F, FT, ldT);
}

// MSE gradient d = 2 (out - y) / (B nout) as bf16 [B][nout] and [nout][B], and the loss
// sum (out-y)^2 / (B nout). One 32 x 64 tile per 32 x 8 block: a thread takes two adjacent columns of 4
// rows (8-byte loads of out, 4-byte bf16 pair stores of d), loaded before use; the transposed copy goes
// through shared memory as bf16 pairs of adjacent rows. Each block writes its share of the loss to
// lossp[block]; the block that finishes last (counted in *count, which it resets to 0) adds the shares in
// block order, so the loss is the same from run to run.
//
// VG (training on values and gradients, vg_row layout, B = 4 x positions rows): a value row m = 4p is
// compared with tgt[p][ld] and weighs 1 / (positions nout); a derivative row 4p + s with
// tgt_g[(p * 3 + s - 1) * ldt + n] and weighs lam / (3 positions nout). The gradient of a row is twice its
// weight times the difference, the loss the weighted sum of squares.
constexpr int kLossCols = 64;
template <bool VG>
__global__ void __launch_bounds__(256) loss_kernel(const float *out, const float *tgt, int ldt, int B, int nout,
                                                   __nv_bfloat16 *d, __nv_bfloat16 *dT, float *lossp,
                                                   unsigned *count, float *loss, const float *tgt_g, float lam) {
    bsg::pdl_wait();
    bsg::pdl_trigger();
    __shared__ float tile[kLossCols][33];  // [column][row] gradients
    __shared__ float wsum[8];
    __shared__ bool last;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int m0 = blockIdx.y * 32, n0 = blockIdx.x * kLossCols;
    const float npos = VG ? (float)(B / kVgStreams) : (float)B;
    const float inv = 1.0f / (npos * (float)nout);
    const float invg = lam / (3.f * npos * (float)nout);
    const int n = n0 + 2 * tx;  // this thread's two columns (nout is a multiple of 128)
    float2 o[4];
    float t[4][2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int m = m0 + ty + 8 * k;
        const bool live = m < B;
        o[k] = live ? *reinterpret_cast<const float2 *>(out + (size_t)m * nout + n) : make_float2(0.f, 0.f);
        const float *tr = tgt + (size_t)m * ldt + n;
        if constexpr (VG) {
            const int p = m / kVgStreams, st = m % kVgStreams;
            tr = st == 0 ? tgt + (size_t)p * ldt + n : tgt_g + ((size_t)p * 3 + st - 1) * ldt + n;
        }
        t[k][0] = live ? tr[0] : 0.f;
        t[k][1] = live ? tr[1] : 0.f;
    }
    float part = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int m = m0 + ty + 8 * k;
        const float w = VG ? (m % kVgStreams == 0 ? inv : invg) : inv;
        const float d0 = o[k].x - t[k][0], d1 = o[k].y - t[k][1];
        part += VG ? w * (d0 * d0 + d1 * d1) : d0 * d0 + d1 * d1;
        const float g0 = 2.f * d0 * w, g1 = 2.f * d1 * w;
        if (m < B) *reinterpret_cast<__nv_bfloat162 *>(d + (size_t)m * nout + n) = __floats2bfloat162_rn(g0, g1);
        tile[2 * tx][ty + 8 * k] = g0;
        tile[2 * tx + 1][ty + 8 * k] = g1;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if (tx == 0) wsum[ty] = part;
    __syncthreads();
    // transposed copy: pairs of adjacent rows of one column, 16 pairs (64 bytes) of a column per half warp
#pragma unroll
    for (int j = 0; j < kLossCols * 16 / 256; ++j) {
        const int q = tid + 256 * j, c = q >> 4, rp = q & 15, m = m0 + 2 * rp;
        if (m + 1 < B)
            *reinterpret_cast<__nv_bfloat162 *>(dT + (size_t)(n0 + c) * B + m) =
                __floats2bfloat162_rn(tile[c][2 * rp], tile[c][2 * rp + 1]);
        else if (m < B)
            dT[(size_t)(n0 + c) * B + m] = __float2bfloat16_rn(tile[c][2 * rp]);
    }
    const unsigned nblk = gridDim.x * gridDim.y;
    if (tid == 0) {
        float total = 0.f;
        for (int k = 0; k < 8; ++k) total += wsum[k];
        lossp[blockIdx.y * gridDim.x + blockIdx.x] = VG ? total : total * inv;
        __threadfence();
        last = atomicAdd(count, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    float acc = 0.f;
    for (unsigned b2 = tid; b2 < nblk; b2 += 256) acc += __ldcg(lossp + b2);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    __syncthreads();
    if (tx == 0) wsum[ty] = acc;
    __syncthreads();
    if (tid == 0) {
        float total = 0.f;
        for (int k = 0; k < 8; ++k) total += wsum[k];
        *loss = total;
        *count = 0;
    }
}

constexpr int kBiasRows = 4;  // bias-gradient rows per block
struct BiasGradArgs {
    const __nv_bfloat16 *dT[kMaxLayers];  // layer k's output gradient, [out_k][B]
    int row_end[kMaxLayers];              // running sum of out_k: block r belongs to the first k with r < row_end[k]
    int n;
};

// Bias gradients of every layer in one launch: grads[b_off_k + r] = sum_m dT_k[r][m]. kBiasRows rows per
// block (rows of all layers in sequence), 8 bf16 per load (B % 8 == 0). VG (vg_row layout): the bias reaches the
// value rows only (m = 0, 4, 8, ...), elements 0 and 4 of each 8.
template <bool VG>
__global__ void __launch_bounds__(256) bias_grad_kernel(BiasGradArgs a, LayerTable lt, int B, float *grads) {
    bsg::pdl_wait();
    bsg::pdl_trigger();
    __shared__ float wsum[kBiasRows][8];
    // rows kBiasRows * blockIdx.x ..: every layer's out is a multiple of kBiasRows, so a block stays in one
    // layer; all its rows' loads are issued before any sum
    const int r0 = (int)blockIdx.x * kBiasRows;
    int k = 0;
    while (k + 1 < a.n && r0 >= a.row_end[k]) ++k;
    const int rb = r0 - (k ? a.row_end[k - 1] : 0);
    float s[kBiasRows];
#pragma unroll
    for (int j = 0; j < kBiasRows; ++j) {
        const uint4 *row = reinterpret_cast<const uint4 *>(a.dT[k] + (size_t)(rb + j) * B);
        s[j] = 0.f;
#pragma unroll 4
        for (int q = threadIdx.x; q < B / 8; q += blockDim.x) {
            const uint4 u = row[q];
            if constexpr (VG) {
                s[j] += __uint_as_float(u.x << 16) + __uint_as_float(u.z << 16);
            } else {
                const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) s[j] += __uint_as_float(w[e] << 16) + __uint_as_float(w[e] & 0xffff0000u);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kBiasRows; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[j] += __shfl_xor_sync(0xffffffffu, s[j], o);
        if ((threadIdx.x & 31) == 0) wsum[j][threadIdx.x >> 5] = s[j];
    }
    __syncthreads();
    if (threadIdx.x < kBiasRows) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += wsum[threadIdx.x][w];
        grads[lt.l[k].b_off + rb + threadIdx.x] = t;
    }
}

struct AdamArgs {
    float lr, b1, b2, eps, bc1, bc2;
};

// One Adam step on parameter i (Algorithm 1 of Kingma & Ba), returning the new value.
__device__ __forceinline__ float adam_update(float *params, const float *grads, float *m1, float *m2, long long i,
                                             const AdamArgs &a) {
    const float g = grads[i];
    const float mm = a.b1 * m1[i] + (1.f - a.b1) * g;
    const float vv = a.b2 * m2[i] + (1.f - a.b2) * g * g;
    m1[i] = mm;
    m2[i] = vv;
    const float p = params[i] - a.lr * (mm / a.bc1) / (sqrtf(vv / a.bc2) + a.eps);
    params[i] = p;
    return p;
}

// Updates the parameters (UPDATE) and rewrites the BF16 weight copies wb ([out][in]) and wbT ([in][out]).
// blockIdx.y < lt.n: the 32 x 32 tiles of layer blockIdx.y's weights (in and out are multiples of 32);
// the transposed copy goes through a shared-memory tile so both stores are row-contiguous.
// blockIdx.y == lt.n: every layer's biases. Block 32 x 8.
template <bool UPDATE>
__global__ void __launch_bounds__(256) adam_kernel(float *params, const float *grads, float *m1, float *m2,
                                                   AdamArgs a, LayerTable lt, __nv_bfloat16 *wb, __nv_bfloat16 *wbT) {
    bsg::pdl_wait();
    bsg::pdl_trigger();
    __shared__ __nv_bfloat16 tile[32][34];
    const int tx = threadIdx.x, ty = threadIdx.y;
    if ((int)blockIdx.y == lt.n) {
        if (!UPDATE) return;
        for (int k = 0; k < lt.n; ++k) {
            const LayerDev &L = lt.l[k];
            for (int j = (int)blockIdx.x * 256 + ty * 32 + tx; j < L.out; j += (int)gridDim.x * 256)
                adam_update(params, grads, m1, m2, L.b_off + j, a);
        }
        return;
    }
    const LayerDev L = lt.l[blockIdx.y];
    const int tcols = L.in / 32, tiles = (L.out / 32) * tcols;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int o0 = (t / tcols) * 32, c0 = (t % tcols) * 32;
#pragma unroll
        for (int r = ty; r < 32; r += 8) {
            const long long q = (long long)(o0 + r) * L.in + c0 + tx;
            const float p = UPDATE ? adam_update(params, grads, m1, m2, L.w_off + q, a) : params[L.w_off + q];
            const __nv_bfloat16 b = __float2bfloat16_rn(p);
            wb[L.wb_off + q] = b;
            tile[r][tx] = b;
        }
        __syncthreads();
#pragma unroll
        for (int r = ty; r < 32; r += 8) wbT[L.wb_off + (long long)(c0 + r) * L.out + o0 + tx] = tile[tx][r];
        __syncthreads();
    }
}

dim3 adam_grid(const LayerTable &lt) {
    int tiles = 1;
    for (int k = 0; k < lt.n; ++k) tiles = std::max(tiles, (lt.l[k].in / 32) * (lt.l[k].out / 32));
    return dim3((unsigned)std::min(tiles, 512), (unsigned)(lt.n + 1));
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
bspline_status encode_bf16_map(const void *ptr, int rows, int cols, int boxrows, CUtensorMap *out) {
    auto enc = bsg::tensor_map_encoder();
    if (!enc) return BSPLINE_ERR_UNSUPPORTED;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)boxrows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? BSPLINE_OK : BSPLINE_ERR_CUDA;
}

bspline_status get_map(mlp_s *m, const void *ptr, int rows, int cols, int boxrows, CUtensorMap *out) {
    if (!m) return encode_bf16_map(ptr, rows, cols, boxrows, out);
    auto key = std::make_tuple(ptr, rows, cols, boxrows);
    auto it = m->maps.find(key);
    if (it != m->maps.end()) {
        *out = it->second;
        return BSPLINE_OK;
    }
    bspline_status st = encode_bf16_map(ptr, rows, cols, boxrows, out);
    if (st == BSPLINE_OK) m->maps[key] = *out;
    return st;
}

// Output map of the TMA-store epilogues: a row-major [rows][ld] matrix of bf16 (esize 2) or fp32 (4) of
// which the first cols columns are written, in boxes of CW columns x 32 rows staged with the 32-byte
// (bf16) or 64-byte (fp32) swizzle (stage_bf16_row / stage_f32_row).
bspline_status encode_out_map(void *ptr, int rows, int cols, int ld, int esize, CUtensorMap *out) {
    auto enc = bsg::tensor_map_encoder();
    if (!enc) return BSPLINE_ERR_UNSUPPORTED;
    if (reinterpret_cast<uintptr_t>(ptr) % 16 || ((size_t)ld * esize) % 16 || ld < cols) return BSPLINE_ERR_ARG;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
    cuuint32_t box[2] = {(cuuint32_t)CW, (cuuint32_t)kStageRows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(out, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     esize == 2 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? BSPLINE_OK : BSPLINE_ERR_CUDA;
}

bspline_status get_out_map(mlp_s *m, void *ptr, int rows, int cols, int ld, int esize, CUtensorMap *out) {
    if (!m) return encode_out_map(ptr, rows, cols, ld, esize, out);
    auto key = std::make_tuple((const void *)ptr, rows, cols, ld, esize);
    auto it = m->omaps.find(key);
    if (it != m->omaps.end()) {
        *out = it->second;
        return BSPLINE_OK;
    }
    bspline_status st = encode_out_map(ptr, rows, cols, ld, esize, out);
    if (st == BSPLINE_OK) {
        if (m->omaps.size() >= 256) m->omaps.clear();  // callers' output buffers come and go
        m->omaps[key] = *out;
    }
    return st;
}

// Launch configuration of gemm_bf16_kernel: BN, epilogue warps, operand slots, staging boxes per warp at most,
// CTAs per SM. Default: one CTA per SM (gemm_stages slots, up to two boxes); TwoCta: 128 x 128 tiles, two
// CTAs per SM.
template <int BN_, int EW_ = kEpiWarps, int NST_ = 0, int NBMAX_ = 2, int MINB_ = 1> struct GemmCfg {
    static constexpr int BN = BN_, EW = EW_, NST = NST_, NBMAX = NBMAX_, MINB = MINB_;
    template <int EPI> static constexpr size_t smem() {
        constexpr int nst = NST ? NST : gemm_stages<BN, EPI>();
        constexpr int nb = epi_stage_bufs<EPI>() < NBMAX ? epi_stage_bufs<EPI>() : NBMAX;
        return gemm_smem_bytes_of<BN, EPI, EW, nst, nb>();
    }
};
template <int EPI> using TwoCta = GemmCfg<128, kEpiWarps2, two_cta_stages<EPI>(), 1, 2>;

template <class C, int EPI> bspline_status set_smem_attr() {
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel<C::BN, EPI, C::EW, C::NST, C::NBMAX, C::MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::template smem<EPI>());
        if (e != cudaSuccess) return cuda_status(e);
        done = true;
    }
    return BSPLINE_OK;
}

// C tile grid over (N/BN, ceil(M/128), splits). A: [arows][K] bf16, B: [N][K] bf16.
template <int BN, int EPI, class Cfg = GemmCfg<BN>>
bspline_status run_gemm(mlp_s *m, const void *A, int arows, const void *B, int N, int K, int M, GemmArgs g,
                        int splits, cudaStream_t s) {
    static_assert(Cfg::BN == BN, "tile width");
    if (N % BN != 0 || K % BK != 0 || M < 1 || arows < M) return BSPLINE_ERR_ARG;
    CUtensorMap ma, mb, mc;
    memset(&mc, 0, sizeof mc);
    bspline_status st = get_map(m, A, arows, K, BM, &ma);
    if (st == BSPLINE_OK) st = get_map(m, B, N, K, BN, &mb);
    if (st == BSPLINE_OK && epi_tma_store<EPI>()) st = get_out_map(m, g.out0, M, N, g.ld0, epi_out_bytes<EPI>(), &mc);
    if (st == BSPLINE_OK) st = set_smem_attr<Cfg, EPI>();
    if (st != BSPLINE_OK) return st;
    const int kb = K / BK;
    splits = std::max(1, std::min(splits, kb));
    g.M = M;
    g.N = N;
    g.K = K;
    g.kblocks_per_split = (kb + splits - 1) / splits;
    g.splits = (kb + g.kblocks_per_split - 1) / g.kblocks_per_split;  // every slice non-empty
    const long long tiles = (long long)(N / BN) * ((M + BM - 1) / BM) * g.splits;
    int sms = 148;
    if (m) sms = m->sms;
    else {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int grid = (int)std::min<long long>(tiles, (long long)sms * Cfg::MINB);
    return cuda_status(bsg::launch_k(gemm_bf16_kernel<BN, EPI, Cfg::EW, Cfg::NST, Cfg::NBMAX, Cfg::MINB>, grid,
                                     64 + 32 * Cfg::EW, Cfg::template smem<EPI>(), s, true, ma, mb, mc, g));
}

// The CTA-pair kernel on clusters of two: (clusters that fit on the device at once, or 0 if none do).
template <int EPI> int pair_clusters() {
    static int n = -1;
    if (n < 0) {
        n = 0;
        if (cudaFuncSetAttribute(gemm_pair_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pair_smem_bytes<EPI>()) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = pair_smem_bytes<EPI>();
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int c = 0;
        if (cudaOccupancyMaxActiveClusters(&c, gemm_pair_kernel<EPI>, &cfg) == cudaSuccess) n = c;
        else cudaGetLastError();
    }
    return n;
}

// C pair tiles of 256 x 256 over (N/256, ceil(M/256)). A: [arows][K] bf16, B: [N][K] bf16.
template <int EPI>
bspline_status run_gemm_pair(mlp_s *m, const void *A, int arows, const void *B, int N, int K, int M, GemmArgs g,
                             int clusters, cudaStream_t s) {
    if (N % kPairBN != 0 || K % BK != 0 || M < 1 || arows < M || clusters < 1) return BSPLINE_ERR_ARG;
    CUtensorMap ma, mb, mc;
    memset(&mc, 0, sizeof mc);
    bspline_status st = get_map(m, A, arows, K, BM, &ma);
    if (st == BSPLINE_OK) st = get_map(m, B, N, K, kPairBN / 2, &mb);
    if (st == BSPLINE_OK && epi_tma_store<EPI>()) st = get_out_map(m, g.out0, M, N, g.ld0, epi_out_bytes<EPI>(), &mc);
    if (st != BSPLINE_OK) return st;
    g.M = M;
    g.N = N;
    g.K = K;
    g.kblocks_per_split = K / BK;
    g.splits = 1;
    const long long tiles = (long long)(N / kPairBN) * ((M + 2 * BM - 1) / (2 * BM));
    const int grid = 2 * (int)std::min<long long>(tiles, clusters);
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = pair_smem_bytes<EPI>();
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cuda_status(cudaLaunchKernelEx(&cfg, gemm_pair_kernel<EPI>, ma, mb, mc, g));
}

// Whether the library's choice takes CTA pairs where every cluster gets a tile.
constexpr bool kPairsByDefault = false;

// Which kernel a GEMM without a surrogate handle runs on: 0 = the library's choice, 1 = one CTA per tile,
// 2 = CTA pairs (where the shape allows them). Set only by mlp_gemm_bf16_ex, for tests and measurements; a
// surrogate's own GEMMs follow its gemm_kernel (mlp_set_gemm_kernel).
thread_local int g_gemm_kernel = 0;

// Tile width: 256 columns when N allows it and the 128 x 256 tiles fill every SM; else 128, so that the
// SMs are all busy and a CTA of the persistent kernel may have a next tile whose MMAs overlap the current
// tile's epilogue. Measured on the training step at 8192 rows (128 wide tiles on 148 SMs): 183.5 ->
// 173.2 us; at 16384 rows the wide tiles stay (256 tiles: 301.7 us, against 304.2 us with narrow ones).
inline int gemm_bn(int M, int N, int sms) {
    if (N % 256 != 0) return 128;
    const long long wide_tiles = (long long)((M + BM - 1) / BM) * (N / 256);
    return wide_tiles >= sms ? 256 : 128;
}

template <int EPI>
bspline_status gemm(mlp_s *m, const void *A, int arows, const void *B, int N, int K, int M, GemmArgs g, int splits,
                    cudaStream_t s) {
    int sms = 148;
    if (m) sms = m->sms;
    else {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    // CTA pairs where every cluster gets a 256 x 256 tile (no K split)
    const int choice = m ? m->gemm_kernel : g_gemm_kernel;
    if constexpr (EPI != EPI_ATOMIC) {
        if ((choice == 0 || choice == 2) && splits <= 1 && N % kPairBN == 0) {
            const int clusters = pair_clusters<EPI>();
            const long long pair_tiles = (long long)((M + 2 * BM - 1) / (2 * BM)) * (N / kPairBN);
            if (clusters > 0 && (choice == 2 || (kPairsByDefault && pair_tiles >= clusters)))
                return run_gemm_pair<EPI>(m, A, arows, B, N, K, M, g, clusters, s);
        }
    }
    if (choice == 3 && N % 128 == 0) return run_gemm<128, EPI, TwoCta<EPI>>(m, A, arows, B, N, K, M, g, splits, s);
    if (gemm_bn(M, N, sms) == 256) return run_gemm<256, EPI>(m, A, arows, B, N, K, M, g, splits, s);
    return run_gemm<128, EPI>(m, A, arows, B, N, K, M, g, splits, s);
}

GemmArgs blank_args(int *status) {
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.status = status;
    return g;
}

void free_train(mlp_s *m) {
    cudaFree(m->feat);
    cudaFree(m->featT);
    for (auto p : m->act) cudaFree(p);
    for (auto p : m->actT) cudaFree(p);
    for (auto p : m->d) cudaFree(p);
    for (auto p : m->dT) cudaFree(p);
    for (auto p : m->z) cudaFree(p);
    cudaFree(m->out);
    cudaFree(m->lossp);
    m->lossp = nullptr;
    m->lcount = nullptr;
    m->feat = m->featT = nullptr;
    m->act.clear();
    m->actT.clear();
    m->d.clear();
    m->dT.clear();
    m->z.clear();
    m->out = nullptr;
    m->tb = 0;
    m->maps.clear();
    m->omaps.clear();
}

void free_infer(mlp_s *m) {
    cudaFree(m->ifeat);
    cudaFree(m->h[0]);
    cudaFree(m->h[1]);
    m->ifeat = m->h[0] = m->h[1] = nullptr;
    m->ir = 0;
    m->maps.clear();
    m->omaps.clear();
}

template <typename T> cudaError_t alloc(T **p, size_t n) { return cudaMalloc(p, n * sizeof(T)); }

bspline_status ensure_train(mlp_s *m, int B) {
    if (m->tb >= B) return BSPLINE_OK;
    cudaDeviceSynchronize();
    free_train(m);
    const int H = m->hidden;
    cudaError_t e = alloc(&m->feat, (size_t)B * m->kin);
    if (e == cudaSuccess) e = alloc(&m->featT, (size_t)B * m->kin);
    for (int l = 0; l < m->layers && e == cudaSuccess; ++l) {
        __nv_bfloat16 *a = nullptr, *aT = nullptr;
        float *zz = nullptr;
        e = alloc(&a, (size_t)B * H);
        if (e == cudaSuccess) e = alloc(&aT, (size_t)B * H);
        if (e == cudaSuccess) e = alloc(&zz, (size_t)B * H);
        m->act.push_back(a);
        m->actT.push_back(aT);
        m->z.push_back(zz);
    }
    for (int l = 0; l <= m->layers && e == cudaSuccess; ++l) {
        const int w = l == m->layers ? m->nout : H;
        __nv_bfloat16 *a = nullptr, *aT = nullptr;
        e = alloc(&a, (size_t)B * w);
        if (e == cudaSuccess) e = alloc(&aT, (size_t)B * w);
        m->d.push_back(a);
        m->dT.push_back(aT);
    }
    if (e == cudaSuccess) e = alloc(&m->out, (size_t)B * m->nout);
    // one loss share per block of loss_kernel, then its finished-block counter
    const size_t nblk = (size_t)((B + 31) / 32) * ((m->nout + 31) / 32);
    if (e == cudaSuccess) e = alloc(&m->lossp, nblk + 1);
    if (e == cudaSuccess) m->lcount = reinterpret_cast<unsigned *>(m->lossp + nblk);
    if (e == cudaSuccess) e = cudaMemset(m->lcount, 0, 4);
    if (e != cudaSuccess) {
        free_train(m);
        return cuda_status(e);
    }
    m->tb = B;
    return BSPLINE_OK;
}

bspline_status ensure_infer(mlp_s *m, int rows) {
    rows = (rows + BM - 1) / BM * BM;
    if (m->ir >= rows) return BSPLINE_OK;
    cudaDeviceSynchronize();
    free_infer(m);
    cudaError_t e = alloc(&m->ifeat, (size_t)rows * m->kin);
    if (e == cudaSuccess) e = alloc(&m->h[0], (size_t)rows * m->hidden);
    if (e == cudaSuccess) e = alloc(&m->h[1], (size_t)rows * m->hidden);
    if (e != cudaSuccess) {
        free_infer(m);
        return cuda_status(e);
    }
    // rows beyond the live ones are read by the GEMMs; keep them finite
    e = cudaMemset(m->ifeat, 0, (size_t)rows * m->kin * 2);
    if (e == cudaSuccess) e = cudaMemset(m->h[0], 0, (size_t)rows * m->hidden * 2);
    if (e == cudaSuccess) e = cudaMemset(m->h[1], 0, (size_t)rows * m->hidden * 2);
    if (e != cudaSuccess) return cuda_status(e);
    m->ir = rows;
    return BSPLINE_OK;
}

bool current_device_is(mlp_s *m) {
    int d = -1;
    return cudaGetDevice(&d) == cudaSuccess && d == m->device;
}

bool aligned16(const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

bspline_status refresh(mlp_s *m, cudaStream_t s) {
    adam_kernel<false><<<adam_grid(m->lt), dim3(32, 8), 0, s>>>(m->params, nullptr, nullptr, nullptr, AdamArgs{},
                                                                  m->lt, m->wb, m->wbT);
    return cuda_status(cudaGetLastError());
}

double gemm_flops(long long M, long long N, long long K) { return 2.0 * M * N * K; }

}  // namespace

extern "C" {

bspline_status mlp_create(int nfreq, int hidden, int layers, int nout, mlp_t *out) {
    if (!out) return BSPLINE_ERR_ARG;
    *out = nullptr;
    if (nfreq < 1 || nfreq > 64 || hidden < 128 || hidden > 4096 || hidden % 128 || layers < 1 ||
        layers > kMaxLayers - 2 || nout < 128 || nout > 8192 || nout % 128)
        return BSPLINE_ERR_ARG;
    mlp_s *m = new (std::nothrow) mlp_s();
    if (!m) return BSPLINE_ERR_ALLOC;
    m->nfreq = nfreq;
    m->hidden = hidden;
    m->layers = layers;
    m->nout = nout;
    m->kin = (6 * nfreq + BK - 1) / BK * BK;
    if (m->kin % 128) m->kin += 64;  // the dW GEMM of layer 0 tiles N = kin by 128
    size_t off = 0, woff = 0;
    m->lt.n = layers + 1;
    for (int l = 0; l <= layers; ++l) {
        LayerDev &L = m->lt.l[l];
        L.in = l == 0 ? m->kin : hidden;
        L.out = l == layers ? nout : hidden;
        L.w_off = (long long)off;
        off += (size_t)L.in * L.out;
        L.b_off = (long long)off;
        off += L.out;
        L.wb_off = (long long)woff;
        woff += (size_t)L.in * L.out;
    }
    m->nparams = off;
    m->nweights = woff;
    cudaError_t e = cudaGetDevice(&m->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, m->device);
    if (e == cudaSuccess) e = alloc(&m->params, off);
    if (e == cudaSuccess) e = alloc(&m->grads, off);
    if (e == cudaSuccess) e = alloc(&m->m1, off);
    if (e == cudaSuccess) e = alloc(&m->m2, off);
    if (e == cudaSuccess) e = alloc(&m->wb, woff);
    if (e == cudaSuccess) e = alloc(&m->wbT, woff);
    if (e == cudaSuccess) e = alloc(&m->status, 1);
    if (e == cudaSuccess) e = alloc(&m->loss, 1);
    if (e == cudaSuccess) e = cudaMemset(m->params, 0, off * 4);
    if (e == cudaSuccess) e = cudaMemset(m->grads, 0, off * 4);
    if (e == cudaSuccess) e = cudaMemset(m->m1, 0, off * 4);
    if (e == cudaSuccess) e = cudaMemset(m->m2, 0, off * 4);
    if (e == cudaSuccess) e = cudaMemset(m->status, 0, 4);
    if (e == cudaSuccess) e = cudaMemset(m->wb, 0, woff * 2);
    if (e == cudaSuccess) e = cudaMemset(m->wbT, 0, woff * 2);
    if (e != cudaSuccess) {
        mlp_destroy(m);
        return cuda_status(e);
    }
    *out = m;
    return BSPLINE_OK;
}

bspline_status mlp_destroy(mlp_t m) {
    if (!m) return BSPLINE_ERR_ARG;
    cudaDeviceSynchronize();
    free_train(m);
    free_infer(m);
    cudaFree(m->params);
    cudaFree(m->grads);
    cudaFree(m->m1);
    cudaFree(m->m2);
    cudaFree(m->wb);
    cudaFree(m->wbT);
    cudaFree(m->status);
    cudaFree(m->loss);
    delete m;
    return BSPLINE_OK;
}

size_t mlp_param_count(mlp_t m) { return m ? m->nparams : 0; }
int mlp_feature_count(mlp_t m) { return m ? m->kin : 0; }

bspline_status mlp_device_status(mlp_t m, void *stream, int reset) {
    if (!m) return BSPLINE_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, m->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && reset) e = cudaMemsetAsync(m->status, 0, sizeof(int), s);
    if (e == cudaSuccess && reset) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    return (bspline_status)v;
}

bspline_status mlp_set_gemm_kernel(mlp_t m, int kernel) {
    if (!m || kernel < 0 || kernel > 3) return BSPLINE_ERR_ARG;
    std::lock_guard<std::mutex> lock(m->mu);
    m->gemm_kernel = kernel;
    return BSPLINE_OK;
}

bspline_status mlp_init(mlp_t m, unsigned long long seed) {
    if (!m || !current_device_is(m)) return BSPLINE_ERR_ARG;
    std::vector<float> p(m->nparams, 0.f);
    unsigned long long st = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    for (int l = 0; l < m->lt.n; ++l) {
        const LayerDev &L = m->lt.l[l];
        const int in_live = l == 0 ? 6 * m->nfreq : L.in;
        const float a = 0.5f * sqrtf(6.0f / (float)in_live);
        for (long long q = 0; q < (long long)L.in * L.out; ++q) {
            st = st * 6364136223846793005ull + 1442695040888963407ull;
            const float u = (float)((st >> 40) * (1.0 / 16777216.0));  // [0,1)
            const int c = (int)(q % L.in);
            p[L.w_off + q] = c < in_live ? a * (2.f * u - 1.f) : 0.f;
        }
    }
    return mlp_set_params(m, p.data(), p.size());
}

bspline_status mlp_set_params(mlp_t m, const float *host, size_t count) {
    if (!m || !host || count != m->nparams || !current_device_is(m)) return BSPLINE_ERR_ARG;
    cudaError_t e = cudaMemcpy(m->params, host, count * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m1, 0, count * 4);
    if (e == cudaSuccess) e = cudaMemset(m->m2, 0, count * 4);
    if (e != cudaSuccess) return cuda_status(e);
    m->step = 0;
    bspline_status st = refresh(m, nullptr);
    if (st != BSPLINE_OK) return st;
    return cuda_status(cudaDeviceSynchronize());
}

bspline_status mlp_get_params(mlp_t m, float *host, size_t count) {
    if (!m || !host || count != m->nparams) return BSPLINE_ERR_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host, m->params, count * 4, cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

bspline_status mlp_get_grads(mlp_t m, float *host, size_t count) {
    if (!m || !host || count != m->nparams) return BSPLINE_ERR_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host, m->grads, count * 4, cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

}  // extern "C"

namespace {

// One training step over R rows: R = B positions (value loss), or with VG R = 4 B rows in the vg_row layout
// (each position's value and its three derivatives, loss on both; tgt_g [B][3][ldt], weight lam).
template <bool VG>
bspline_status train_step(mlp_t m, int B, const double *x, const double *y, const double *z, const float *target,
                          int ldt, const float *tgt_g, float lam, float lr, float *loss_out, cudaStream_t s) {
    const int R = VG ? kVgStreams * B : B;
    std::lock_guard<std::mutex> lock(m->mu);
    bspline_status st = ensure_train(m, R);
    if (st != BSPLINE_OK) return st;
    const int H = m->hidden, L = m->layers, kin = m->kin;
    cudaError_t e = cudaMemsetAsync(m->grads, 0, m->nparams * 4, s);
    if (e != cudaSuccess) return cuda_status(e);

    // features, row-major and transposed
    e = launch_features<VG ? kVgRows : kPlainRows>(x, y, z, B, m->nfreq, kin, m->feat, m->featT, R, s);
    if (e != cudaSuccess) return cuda_status(e);
    // forward
    for (int l = 0; l < L && st == BSPLINE_OK; ++l) {
        const LayerDev &Ld = m->lt.l[l];
        GemmArgs g = blank_args(m->status);
        g.bias = m->params + Ld.b_off;
        g.out0 = m->act[l];
        g.ld0 = H;
        g.out1 = m->actT[l];
        g.ld1 = R;
        g.z = m->z[l];
        g.ldz = H;
        const void *A = l == 0 ? (const void *)m->feat : (const void *)m->act[l - 1];
        st = gemm<VG ? EPI_VG_HIDDEN : EPI_FWD_TRAIN>(m, A, R, m->wb + Ld.wb_off, H, Ld.in, R, g, 1, s);
    }
    if (st != BSPLINE_OK) return st;
    {
        const LayerDev &Ld = m->lt.l[L];
        GemmArgs g = blank_args(m->status);
        g.bias = m->params + Ld.b_off;
        g.out0 = m->out;
        g.ld0 = m->nout;
        st = gemm<VG ? EPI_VG_OUT : EPI_LINEAR>(m, m->act[L - 1], R, m->wb + Ld.wb_off, m->nout, H, R, g, 1, s);
        if (st != BSPLINE_OK) return st;
    }
    // loss and output gradient
    {
        dim3 grid(m->nout / kLossCols, (R + 31) / 32);
        e = bsg::launch_k(loss_kernel<VG>, grid, dim3(32, 8), 0, s, true, (const float *)m->out, target, ldt, R,
                          m->nout, m->d[L], m->dT[L], m->lossp, m->lcount, m->loss,
                          tgt_g, lam);
        if (e != cudaSuccess) return cuda_status(e);
    }
    // backward
    for (int l = L; l >= 0 && st == BSPLINE_OK; --l) {
        const LayerDev &Ld = m->lt.l[l];
        const int tiles = (Ld.out / BM) * (Ld.in / gemm_bn(Ld.out, Ld.in, m->sms));  // as gemm() tiles N
        const int splits = std::max(1, m->sms / std::max(tiles, 1));
        GemmArgs g = blank_args(m->status);
        g.out0 = m->grads + Ld.w_off;
        g.ld0 = Ld.in;
        const void *Bop = l == 0 ? (const void *)m->featT : (const void *)m->actT[l - 1];
        st = gemm<EPI_ATOMIC>(m, m->dT[l], Ld.out, Bop, Ld.in, R, Ld.out, g, splits, s);
        if (st != BSPLINE_OK) break;
        if (l > 0) {
            GemmArgs gb = blank_args(m->status);
            gb.out0 = m->d[l - 1];
            gb.ld0 = H;
            gb.out1 = m->dT[l - 1];
            gb.ld1 = R;
            gb.z = m->z[l - 1];
            gb.ldz = H;
            st = gemm<VG ? EPI_VG_BWD : EPI_BWD>(m, m->d[l], R, m->wbT + Ld.wb_off, H, Ld.out, R, gb, 1, s);
        }
    }
    if (st != BSPLINE_OK) return st;
    {
        BiasGradArgs ba{};
        ba.n = m->lt.n;
        int rows = 0;
        for (int l = 0; l < m->lt.n; ++l) {
            ba.dT[l] = m->dT[l];
            rows += m->lt.l[l].out;
            ba.row_end[l] = rows;
        }
        e = bsg::launch_k(bias_grad_kernel<VG>, rows / kBiasRows, 256, 0, s, true, ba, m->lt, R, m->grads);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (lr > 0.f) {
        ++m->step;
        const float b1 = 0.9f, b2 = 0.999f;
        const float bc1 = 1.f - powf(b1, (float)m->step), bc2 = 1.f - powf(b2, (float)m->step);
        e = bsg::launch_k(adam_kernel<true>, adam_grid(m->lt), dim3(32, 8), 0, s, true, m->params,
                          (const float *)m->grads, m->m1, m->m2, AdamArgs{lr, b1, b2, 1e-8f, bc1, bc2}, m->lt, m->wb,
                          m->wbT);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (loss_out) {
        e = cudaMemcpyAsync(loss_out, m->loss, 4, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return BSPLINE_OK;
}

}  // namespace

extern "C" {

bspline_status mlp_train_step(mlp_t m, int B, const double *x, const double *y, const double *z, const float *target,
                              int ldt, float lr, float *loss_out, void *stream) {
    if (!m || B < 128 || B % 128 || !x || !y || !z || !target || ldt < m->nout || !(lr >= 0.f))
        return BSPLINE_ERR_ARG;
    if (!current_device_is(m)) return BSPLINE_ERR_ARG;
    return train_step<false>(m, B, x, y, z, target, ldt, nullptr, 0.f, lr, loss_out, static_cast<cudaStream_t>(stream));
}

bspline_status mlp_train_step_vg(mlp_t m, int B, const double *x, const double *y, const double *z,
                                 const float *target_v, const float *target_g, int ldt, float lambda, float lr,
                                 float *loss_out, void *stream) {
    if (!m || B < 32 || B % 32 || !x || !y || !z || !target_v || !target_g || ldt < m->nout || !(lr >= 0.f) ||
        !(lambda >= 0.f) || !std::isfinite(lambda))
        return BSPLINE_ERR_ARG;
    if ((long long)B * kVgStreams > 0x7fffffffLL / 2) return BSPLINE_ERR_ARG;
    if (!current_device_is(m)) return BSPLINE_ERR_ARG;
    return train_step<true>(m, B, x, y, z, target_v, ldt, target_g, lambda, lr, loss_out,
                            static_cast<cudaStream_t>(stream));
}

static bspline_status check_eval(mlp_t m, int npos, const double *x, const double *y, const double *z,
                                 const float *v, int ld) {
    if (!m || npos < 0 || ld < m->nout || ld % 4) return BSPLINE_ERR_ARG;
    if (npos == 0) return BSPLINE_OK;
    if (!x || !y || !z || !v || !aligned16(v)) return BSPLINE_ERR_ARG;
    if (!current_device_is(m)) return BSPLINE_ERR_ARG;
    if ((long long)npos * 8 > 0x7fffffffLL / 2) return BSPLINE_ERR_ARG;
    return BSPLINE_OK;
}

bspline_status mlp_eval_v(mlp_t m, int npos, const double *x, const double *y, const double *z, float *v, int ld,
                          void *stream) {
    bspline_status st = check_eval(m, npos, x, y, z, v, ld);
    if (st != BSPLINE_OK || npos == 0) return st;
    std::lock_guard<std::mutex> lock(m->mu);
    st = ensure_infer(m, npos);
    if (st != BSPLINE_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_features<kPlainRows>(x, y, z, npos, m->nfreq, m->kin, m->ifeat, nullptr, 0, s);
    if (e != cudaSuccess) return cuda_status(e);
    const int rows = m->ir;
    for (int l = 0; l < m->layers && st == BSPLINE_OK; ++l) {
        const LayerDev &Ld = m->lt.l[l];
        GemmArgs g = blank_args(m->status);
        g.bias = m->params + Ld.b_off;
        g.out0 = m->h[l & 1];
        g.ld0 = m->hidden;
        const void *A = l == 0 ? (const void *)m->ifeat : (const void *)m->h[(l - 1) & 1];
        st = gemm<EPI_FWD_INFER>(m, A, rows, m->wb + Ld.wb_off, m->hidden, Ld.in, npos, g, 1, s);
    }
    if (st != BSPLINE_OK) return st;
    const LayerDev &Ld = m->lt.l[m->layers];
    GemmArgs g = blank_args(m->status);
    g.bias = m->params + Ld.b_off;
    g.out0 = v;
    g.ld0 = ld;
    return gemm<EPI_LINEAR>(m, m->h[(m->layers - 1) & 1], rows, m->wb + Ld.wb_off, m->nout, m->hidden, npos,
                                     g, 1, s);
}

bspline_status mlp_eval_vgl(mlp_t m, int npos, const double *x, const double *y, const double *z, float *v, float *g,
                            float *l, int ld, void *stream) {
    bspline_status st = check_eval(m, npos, x, y, z, v, ld);
    if (st != BSPLINE_OK || npos == 0) return st;
    if (!g || !l || !aligned16(g) || !aligned16(l)) return BSPLINE_ERR_ARG;
    std::lock_guard<std::mutex> lock(m->mu);
    const int R = (int)fm_rows(npos);
    st = ensure_infer(m, R);
    if (st != BSPLINE_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_features<kFmRows>(x, y, z, npos, m->nfreq, m->kin, m->ifeat, nullptr, 0, s);
    if (e != cudaSuccess) return cuda_status(e);
    const int rows = m->ir;
    for (int k = 0; k < m->layers && st == BSPLINE_OK; ++k) {
        const LayerDev &Ld = m->lt.l[k];
        GemmArgs ga = blank_args(m->status);
        ga.bias = m->params + Ld.b_off;
        ga.out0 = m->h[k & 1];
        ga.ld0 = m->hidden;
        const void *A = k == 0 ? (const void *)m->ifeat : (const void *)m->h[(k - 1) & 1];
        st = gemm<EPI_FM_HIDDEN>(m, A, rows, m->wb + Ld.wb_off, m->hidden, Ld.in, R, ga, 1, s);
    }
    if (st != BSPLINE_OK) return st;
    const LayerDev &Ld = m->lt.l[m->layers];
    GemmArgs ga = blank_args(m->status);
    ga.bias = m->params + Ld.b_off;
    ga.out0 = v;
    ga.ld0 = ld;
    ga.g = g;
    ga.l = l;
    ga.npos = npos;
    return gemm<EPI_FM_OUT>(m, m->h[(m->layers - 1) & 1], rows, m->wb + Ld.wb_off, m->nout, m->hidden, R,
                                     ga, 1, s);
}

bspline_status mlp_save(mlp_t m, const char *path) {
    if (!m || !path) return BSPLINE_ERR_ARG;
    std::vector<float> buf(m->nparams * 3);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(buf.data(), m->params, m->nparams * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + m->nparams, m->m1, m->nparams * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + 2 * m->nparams, m->m2, m->nparams * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    FILE *f = fopen(path, "wb");
    if (!f) return BSPLINE_ERR_ARG;
    fprintf(f,
            "{\"format\":\"bspline-mlp-v1\",\"nfreq\":%d,\"hidden\":%d,\"layers\":%d,\"nout\":%d,\"kin\":%d,"
            "\"nparams\":%zu,\"step\":%lld}\n",
            m->nfreq, m->hidden, m->layers, m->nout, m->kin, m->nparams, m->step);
    const size_t w = fwrite(buf.data(), 4, buf.size(), f);
    fclose(f);
    return w == buf.size() ? BSPLINE_OK : BSPLINE_ERR_ARG;
}

bspline_status mlp_load(mlp_t m, const char *path) {
    if (!m || !path || !current_device_is(m)) return BSPLINE_ERR_ARG;
    FILE *f = fopen(path, "rb");
    if (!f) return BSPLINE_ERR_ARG;
    char line[512];
    if (!fgets(line, sizeof line, f)) {
        fclose(f);
        return BSPLINE_ERR_ARG;
    }
    int nfreq = 0, hidden = 0, layers = 0, nout = 0, kin = 0;
    size_t np = 0;
    long long step = 0;
    if (sscanf(line,
               "{\"format\":\"bspline-mlp-v1\",\"nfreq\":%d,\"hidden\":%d,\"layers\":%d,\"nout\":%d,\"kin\":%d,"
               "\"nparams\":%zu,\"step\":%lld}",
               &nfreq, &hidden, &layers, &nout, &kin, &np, &step) != 7 ||
        nfreq != m->nfreq || hidden != m->hidden || layers != m->layers || nout != m->nout || kin != m->kin ||
        np != m->nparams) {
        fclose(f);
        return BSPLINE_ERR_ARG;
    }
    std::vector<float> buf(np * 3);
    const size_t r = fread(buf.data(), 4, buf.size(), f);
    fclose(f);
    if (r != buf.size()) return BSPLINE_ERR_ARG;
    cudaError_t e = cudaMemcpy(m->params, buf.data(), np * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->m1, buf.data() + np, np * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->m2, buf.data() + 2 * np, np * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_status(e);
    m->step = step;
    bspline_status st = refresh(m, nullptr);
    if (st != BSPLINE_OK) return st;
    return cuda_status(cudaDeviceSynchronize());
}

bspline_status mlp_gemm_bf16(const void *A, const void *B, float *C, int M, int N, int K, int ldc, int splitk,
                             void *stream) {
    return mlp_gemm_bf16_ex(A, B, C, M, N, K, ldc, splitk, 0, stream);
}

bspline_status mlp_gemm_bf16_ex(const void *A, const void *B, float *C, int M, int N, int K, int ldc, int splitk,
                                int kernel, void *stream) {
    if (!A || !B || !C || M < 1 || N < 128 || N % 128 || K < 64 || K % 64 || ldc < N || ldc % 4 || !aligned16(C) ||
        splitk < 1 || kernel < 0 || kernel > 3)
        return BSPLINE_ERR_ARG;
    struct Restore {
        int v;
        ~Restore() { g_gemm_kernel = v; }
    } restore{g_gemm_kernel};
    g_gemm_kernel = kernel;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GemmArgs g = blank_args(nullptr);
    g.out0 = C;
    g.ld0 = ldc;
    if (splitk > 1) {
        cudaError_t e = cudaMemset2DAsync(C, (size_t)ldc * 4, 0, (size_t)N * 4, M, s);
        if (e != cudaSuccess) return cuda_status(e);
        return gemm<EPI_ATOMIC>(nullptr, A, M, B, N, K, M, g, splitk, s);
    }
    return gemm<EPI_LINEAR>(nullptr, A, M, B, N, K, M, g, 1, s);
}

double mlp_flops(mlp_t m, int what, int n) {
    if (!m || n <= 0) return 0.0;
    const long long H = m->hidden;
    double f = 0.0;
    if (what == 0 || what == 1) {
        const long long rows = what == 0 ? n : fm_rows(n);
        const long long Mp = (rows + BM - 1) / BM * BM;
        for (int l = 0; l <= m->layers; ++l) f += gemm_flops(Mp, m->lt.l[l].out, m->lt.l[l].in);
    } else {
        if (what == 3) n *= kVgStreams;  // training on values and gradients: 4 rows per position
        for (int l = 0; l <= m->layers; ++l) {
            const LayerDev &L = m->lt.l[l];
            f += gemm_flops(n, L.out, L.in);       // forward
            f += gemm_flops(L.out, L.in, n);       // weight gradient
            if (l > 0) f += gemm_flops(n, L.in, L.out);  // activation gradient
        }
        (void)H;
    }
    return f;
}

}  // extern "C"
