// Internal definitions shared by the translation units of the GB300 B-spline
// library: the table handle, launch arguments, the per-position cell and
// weight stage, the factorised 4x4x4 accumulation and the PTX wrappers
// (mbarrier, TMA, cache-hinted loads).
//
// Paper: arXiv:1611.02665. Eq. (SplineFunc) and Eq. (TricubicValue) in
// Sec. "QMC and B-spline-based SPOs" define what is computed; Sec. "Baseline
// and miniQMC" (Fig. (baselineCode)) gives the V / VGL / VGH outputs and the
// 64 stride-one row reads per position.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <utility>
#include <string>

#include "bspline_gb300.h"

namespace bsg {

// ---------------------------------------------------------------------------
// Host-side handle
// ---------------------------------------------------------------------------
constexpr int kMaxTmaMaps = 4;

struct TmaMapEntry {
    int nbox = 0;
    int swizzle = 0;  // 1: 128-byte swizzle (the tensor-core variant's A operand)
    CUtensorMap map;  // 64-byte aligned type
};

struct HostStaging {
    size_t pos_cap = 0;   // positions per chunk buffer
    size_t out_cap = 0;   // floats per chunk buffer (all components)
    double *d_pos[2] = {nullptr, nullptr};
    float *d_out[2] = {nullptr, nullptr};
    int *d_perm[2] = {nullptr, nullptr};  // per-stream evaluation order scratch
    cudaStream_t stream[2] = {nullptr, nullptr};
    int *d_perm_direct = nullptr;  // order scratch of the direct-access path
    size_t direct_cap = 0;
    int mode = 0;                  // 0 auto, 1 staged copies, 2 direct access
};

}  // namespace bsg

struct bspline_s {
    int nx = 0, ny = 0, nz = 0, N = 0, Npad = 0;
    int dtype = BSPLINE_F32;
    int esize = 4;
    int device = 0;
    int num_sms = 0;
    size_t l2_bytes = 0;      // the device's L2 cache size
    size_t rows = 0;          // (nx+3)*(ny+3)*(nz+3)
    size_t table_bytes = 0;
    void *table = nullptr;    // device [nx+3][ny+3][nz+3][Npad] of dtype
    float *scale = nullptr;   // device [Npad] (all 1 for FP32 tables)
    int *status = nullptr;    // device status word
    int has_coefs = 0;
    bspline_tuning tuning[3];
    bsg::TmaMapEntry maps[bsg::kMaxTmaMaps];
    int nmaps = 0;
    std::mutex mu;            // guards maps and the perm scratch
    std::mutex staging_mu;    // serialises bspline_eval_host (its staging buffers)
    bsg::HostStaging staging;
    int *perm = nullptr;      // scratch: cell-sorted evaluation order
    size_t perm_cap = 0;
    int lattice = 0;          // 1: general cell set by bspline_set_lattice
    double L[9] = {0};        // lattice vectors as rows
    double G[9] = {0};        // L^-1
};

namespace bsg {

// Launch arguments of one single-table evaluation.
struct EvalArgs {
    const void *table;
    const float *scale;
    int nx, ny, nz;
    int N, Npad;
    long long sj;    // elements between rows j and j+1  = (nz+3)*Npad
    long long si;    // elements between rows i and i+1  = (ny+3)*(nz+3)*Npad
    int npos;
    const double *x, *y, *z;
    float *o0, *o1, *o2;  // v, g, h-or-l
    int ld;
    int *status;
    const int *perm;  // evaluation order (slot -> position), or null for input order
    // General cell (lattice != 0): positions are Cartesian, u = r . G with
    // G = L^-1 (row-major G[i*3+d]); outputs are Cartesian derivatives.
    int lattice;
    double G[9];
    float Gf[9];
    float lapw[6];  // Laplacian weights of the fractional Hessian (xx,xy,xz,yy,yz,zz)
};

// Fractional coordinate d of position pos (Cartesian positions are mapped
// through G in double precision when a lattice is set).
__device__ __forceinline__ double frac_coord(const EvalArgs &A, long long pos, int d) {
    if (!A.lattice) return d == 0 ? A.x[pos] : (d == 1 ? A.y[pos] : A.z[pos]);
    return A.x[pos] * A.G[d] + A.y[pos] * A.G[3 + d] + A.z[pos] * A.G[6 + d];
}

constexpr int nout_of(int kind) { return kind == BSPLINE_V ? 1 : (kind == BSPLINE_VGL ? 5 : 10); }

// Reduce one fractional coordinate to (cell index, offset) in double
// precision: wrap into the unit cell, scale by the grid, take the floor
// (Eq. (SplineFunc): i = floor(x / Delta)). A coordinate that rounds onto the
// far face wraps to cell 0 with offset 0. Double precision keeps the chosen
// stencil identical to the one a double-precision reference picks.
__device__ __forceinline__ void cell_reduce(double x, int n, int &i, float &t) {
    double xw = x - floor(x);
    double u = xw * (double)n;
    double fi = floor(u);
    double td = u - fi;
    int ii = (int)fi;
    if (ii >= n) {
        ii -= n;
        td = 0.0;
    }
    i = ii;
    t = (float)td;
}

// Cubic B-spline weights of the four stencil rows (knots i-1..i+2) at offset
// t, with first and second derivatives scaled by n and n^2 (the chain rule for
// u = x * n). Layout: w[0..3] value, w[4..7] first, w[8..11] second derivative.
__device__ __forceinline__ void basis_weights(float t, float n, float *w) {
    const float s = 1.0f - t;
    const float t2 = t * t, t3 = t2 * t;
    const float sixth = 1.0f / 6.0f;
    w[0] = sixth * s * s * s;
    w[1] = fmaf(0.5f, t3, 2.0f / 3.0f - t2);
    w[2] = sixth * fmaf(-3.0f, t3, fmaf(3.0f, t2, fmaf(3.0f, t, 1.0f)));
    w[3] = sixth * t3;
    w[4] = -0.5f * s * s * n;
    w[5] = t * fmaf(1.5f, t, -2.0f) * n;
    w[6] = fmaf(-1.5f, t2, t + 0.5f) * n;
    w[7] = 0.5f * t2 * n;
    const float n2 = n * n;
    w[8] = s * n2;
    w[9] = fmaf(3.0f, t, -2.0f) * n2;
    w[10] = fmaf(-3.0f, t, 1.0f) * n2;
    w[11] = t * n2;
}

// ---------------------------------------------------------------------------
// Element conversion and vector loads
// ---------------------------------------------------------------------------
template <typename T> struct Elem;
template <> struct Elem<float> {
    static constexpr int dtype = BSPLINE_F32;
};
template <> struct Elem<__half> {
    static constexpr int dtype = BSPLINE_F16;
};
template <> struct Elem<__nv_bfloat16> {
    static constexpr int dtype = BSPLINE_BF16;
};

// Read-only global loads that skip L1 allocation and ask L2 for 256-byte
// prefetch: each warp streams contiguous orbital runs of a row.
__device__ __forceinline__ uint32_t ldg_b32(const void *p) {
    uint32_t r;
    asm("ld.global.nc.L1::no_allocate.L2::256B.b32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}
__device__ __forceinline__ uint2 ldg_b64(const void *p) {
    uint2 r;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v2.b32 {%0, %1}, [%2];"
                 : "=r"(r.x), "=r"(r.y)
                 : "l"(p));
    return r;
}
__device__ __forceinline__ uint4 ldg_b128(const void *p) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

__device__ __forceinline__ float2 h2f(uint32_t u) {
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}
__device__ __forceinline__ float2 b2f(uint32_t u) {
    // bfloat16 -> float is a 16-bit shift of the bit pattern
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

// Load VEC consecutive elements of type T from global memory into floats.
template <typename T, int VEC> __device__ __forceinline__ void load_row_global(const T *p, float *out);

template <> __device__ __forceinline__ void load_row_global<float, 1>(const float *p, float *o) {
    o[0] = __uint_as_float(ldg_b32(p));
}
template <> __device__ __forceinline__ void load_row_global<float, 2>(const float *p, float *o) {
    uint2 r = ldg_b64(p);
    o[0] = __uint_as_float(r.x);
    o[1] = __uint_as_float(r.y);
}
template <> __device__ __forceinline__ void load_row_global<float, 4>(const float *p, float *o) {
    uint4 r = ldg_b128(p);
    o[0] = __uint_as_float(r.x);
    o[1] = __uint_as_float(r.y);
    o[2] = __uint_as_float(r.z);
    o[3] = __uint_as_float(r.w);
}
#define BSG_HALF_LOADS(T, CONV)                                                          \
    template <> __device__ __forceinline__ void load_row_global<T, 2>(const T *p, float *o) { \
        float2 a = CONV(ldg_b32(p));                                                     \
        o[0] = a.x;                                                                      \
        o[1] = a.y;                                                                      \
    }                                                                                    \
    template <> __device__ __forceinline__ void load_row_global<T, 4>(const T *p, float *o) { \
        uint2 r = ldg_b64(p);                                                            \
        float2 a = CONV(r.x), b = CONV(r.y);                                             \
        o[0] = a.x;                                                                      \
        o[1] = a.y;                                                                      \
        o[2] = b.x;                                                                      \
        o[3] = b.y;                                                                      \
    }                                                                                    \
    template <> __device__ __forceinline__ void load_row_global<T, 8>(const T *p, float *o) { \
        uint4 r = ldg_b128(p);                                                           \
        float2 a = CONV(r.x), b = CONV(r.y), c = CONV(r.z), d = CONV(r.w);               \
        o[0] = a.x;                                                                      \
        o[1] = a.y;                                                                      \
        o[2] = b.x;                                                                      \
        o[3] = b.y;                                                                      \
        o[4] = c.x;                                                                      \
        o[5] = c.y;                                                                      \
        o[6] = d.x;                                                                      \
        o[7] = d.y;                                                                      \
    }
BSG_HALF_LOADS(__half, h2f)
BSG_HALF_LOADS(__nv_bfloat16, b2f)
#undef BSG_HALF_LOADS

// Load VEC consecutive elements of type T from shared memory into floats.
template <typename T, int VEC> __device__ __forceinline__ void load_row_shared(const T *p, float *o) {
    if constexpr (sizeof(T) == 4) {
        if constexpr (VEC == 1) {
            o[0] = *reinterpret_cast<const float *>(p);
        } else if constexpr (VEC == 2) {
            float2 a = *reinterpret_cast<const float2 *>(p);
            o[0] = a.x;
            o[1] = a.y;
        } else {
            float4 a = *reinterpret_cast<const float4 *>(p);
            o[0] = a.x;
            o[1] = a.y;
            o[2] = a.z;
            o[3] = a.w;
        }
    } else {
        if constexpr (VEC == 1) {
            if constexpr (Elem<T>::dtype == BSPLINE_F16)
                o[0] = __half2float(*reinterpret_cast<const __half *>(p));
            else
                o[0] = __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(p));
        } else {
#pragma unroll
            for (int q = 0; q < VEC / 2; ++q) {
                uint32_t u = reinterpret_cast<const uint32_t *>(p)[q];
                float2 a = Elem<T>::dtype == BSPLINE_F16 ? h2f(u) : b2f(u);
                o[2 * q] = a.x;
                o[2 * q + 1] = a.y;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Factorised accumulation over the 4x4x4 stencil (Eq. (TricubicValue)).
// The triple sum is taken innermost-first: along z for each (a,b) row pair,
// then along y, then along x, so each loaded coefficient costs 1 (V), 3
// (VGL/VGH) FMAs in the z stage instead of one per output component.
// W: weights [3 axes][12] as produced by basis_weights.
// rows(a, b, p) fills p[c][VEC] with the four z-rows of plane (a, b).
// out[q][VEC]: V: v | VGL: v,gx,gy,gz,l | VGH: v,gx,gy,gz,hxx,hxy,hxz,hyy,hyz,hzz
// ---------------------------------------------------------------------------
template <int KIND, int VEC, class Rows>
__device__ __forceinline__ void accumulate(const float *__restrict__ W, Rows rows,
                                           float (&out)[nout_of(KIND)][VEC]) {
    constexpr int NO = nout_of(KIND);
#pragma unroll
    for (int q = 0; q < NO; ++q)
#pragma unroll
        for (int e = 0; e < VEC; ++e) out[q][e] = 0.f;

    const float *wx = W, *wy = W + 12, *wz = W + 24;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        float p[4][4][VEC];  // [b][c][e]
#pragma unroll
        for (int b = 0; b < 4; ++b) rows(a, b, p[b]);

        if constexpr (KIND == BSPLINE_V) {
            float t00[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) t00[e] = 0.f;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    float s0 = wz[0] * p[b][0][e];
                    s0 = fmaf(wz[1], p[b][1][e], s0);
                    s0 = fmaf(wz[2], p[b][2][e], s0);
                    s0 = fmaf(wz[3], p[b][3][e], s0);
                    t00[e] = fmaf(wy[b], s0, t00[e]);
                }
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) out[0][e] = fmaf(wx[a], t00[e], out[0][e]);
        } else {
            float t00[VEC], t01[VEC], t02[VEC], t10[VEC], t20[VEC], t11[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) t00[e] = t01[e] = t02[e] = t10[e] = t20[e] = t11[e] = 0.f;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    float s0 = wz[0] * p[b][0][e], s1 = wz[4] * p[b][0][e], s2 = wz[8] * p[b][0][e];
#pragma unroll
                    for (int c = 1; c < 4; ++c) {
                        s0 = fmaf(wz[c], p[b][c][e], s0);
                        s1 = fmaf(wz[4 + c], p[b][c][e], s1);
                        s2 = fmaf(wz[8 + c], p[b][c][e], s2);
                    }
                    t00[e] = fmaf(wy[b], s0, t00[e]);
                    t01[e] = fmaf(wy[b], s1, t01[e]);
                    t02[e] = fmaf(wy[b], s2, t02[e]);
                    t10[e] = fmaf(wy[4 + b], s0, t10[e]);
                    t20[e] = fmaf(wy[8 + b], s0, t20[e]);
                    if constexpr (KIND == BSPLINE_VGH) t11[e] = fmaf(wy[4 + b], s1, t11[e]);
                }
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const float x0 = wx[a], x1 = wx[4 + a], x2 = wx[8 + a];
                out[0][e] = fmaf(x0, t00[e], out[0][e]);
                out[1][e] = fmaf(x1, t00[e], out[1][e]);
                out[2][e] = fmaf(x0, t10[e], out[2][e]);
                out[3][e] = fmaf(x0, t01[e], out[3][e]);
                if constexpr (KIND == BSPLINE_VGL) {
                    out[4][e] = fmaf(x2, t00[e], fmaf(x0, t20[e] + t02[e], out[4][e]));
                } else {
                    out[4][e] = fmaf(x2, t00[e], out[4][e]);
                    out[5][e] = fmaf(x1, t10[e], out[5][e]);
                    out[6][e] = fmaf(x1, t01[e], out[6][e]);
                    out[7][e] = fmaf(x0, t20[e], out[7][e]);
                    out[8][e] = fmaf(x0, t11[e], out[8][e]);
                    out[9][e] = fmaf(x0, t02[e], out[9][e]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The same factorised accumulation on pairs of orbitals with packed FP32
// arithmetic (fma / mul / add .rn.f32x2: two IEEE single-precision operations
// per instruction, each rounded as the scalar one). Every output gets the
// same operations in the same order as in accumulate(), so the results are
// identical; the instructions issued for the arithmetic are halved, which
// matters where the evaluation is bound by instruction issue rather than by
// memory (tables that sit in L2, 16-bit tables that convert every element).
// W2: the 36 weights of basis_weights, each duplicated into a pair (w, w).
// rows(a, b, p) fills p[c][NP] with the four z-rows of plane (a, b) as NP
// pairs of consecutive orbitals. out[q][NP]: pairs, components as accumulate.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// A weight pair read from shared memory where it is used (the loads are not hoisted, so the x and y
// weights take no registers between their few uses; the z weights, used for every row, stay in registers).
__device__ __forceinline__ uint32_t smem_u32(const void *p);
__device__ __forceinline__ f32x2 lds_pair(const f32x2 *p) {
    f32x2 v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(smem_u32(p)));
    return v;
}
struct SmemPairs {
    const f32x2 *p;
    __device__ __forceinline__ f32x2 operator[](int k) const { return lds_pair(p + k); }
};

template <int KIND, int NP, class Rows>
__device__ __forceinline__ void accumulate_x2(const f32x2 *__restrict__ W2, Rows rows,
                                              f32x2 (&out)[nout_of(KIND)][NP]) {
    constexpr int NO = nout_of(KIND);
#pragma unroll
    for (int q = 0; q < NO; ++q)
#pragma unroll
        for (int e = 0; e < NP; ++e) out[q][e] = 0ull;

    const SmemPairs wx{W2}, wy{W2 + 12};
    f32x2 wz[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) wz[k] = W2[24 + k];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        if constexpr (KIND == BSPLINE_V) {
            f32x2 t00[NP];
#pragma unroll
            for (int e = 0; e < NP; ++e) t00[e] = 0ull;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                f32x2 p[4][NP];  // [c][pair]: the rows of plane (a, b), loaded where they are used
                rows(a, b, p);
                const f32x2 yb = wy[b];
#pragma unroll
                for (int e = 0; e < NP; ++e) {
                    f32x2 s0 = mul2(wz[0], p[0][e]);
                    s0 = fma2(wz[1], p[1][e], s0);
                    s0 = fma2(wz[2], p[2][e], s0);
                    s0 = fma2(wz[3], p[3][e], s0);
                    t00[e] = fma2(yb, s0, t00[e]);
                }
            }
            const f32x2 x0 = wx[a];
#pragma unroll
            for (int e = 0; e < NP; ++e) out[0][e] = fma2(x0, t00[e], out[0][e]);
        } else {
            f32x2 t00[NP], t01[NP], t02[NP], t10[NP], t20[NP], t11[NP];
#pragma unroll
            for (int e = 0; e < NP; ++e) t00[e] = t01[e] = t02[e] = t10[e] = t20[e] = t11[e] = 0ull;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                f32x2 p[4][NP];
                rows(a, b, p);
                const f32x2 y0 = wy[b], y1 = wy[4 + b], y2 = wy[8 + b];
#pragma unroll
                for (int e = 0; e < NP; ++e) {
                    f32x2 s0 = mul2(wz[0], p[0][e]), s1 = mul2(wz[4], p[0][e]), s2 = mul2(wz[8], p[0][e]);
#pragma unroll
                    for (int c = 1; c < 4; ++c) {
                        s0 = fma2(wz[c], p[c][e], s0);
                        s1 = fma2(wz[4 + c], p[c][e], s1);
                        s2 = fma2(wz[8 + c], p[c][e], s2);
                    }
                    t00[e] = fma2(y0, s0, t00[e]);
                    t01[e] = fma2(y0, s1, t01[e]);
                    t02[e] = fma2(y0, s2, t02[e]);
                    t10[e] = fma2(y1, s0, t10[e]);
                    t20[e] = fma2(y2, s0, t20[e]);
                    if constexpr (KIND == BSPLINE_VGH) t11[e] = fma2(y1, s1, t11[e]);
                }
            }
            const f32x2 x0 = wx[a], x1 = wx[4 + a], x2 = wx[8 + a];
#pragma unroll
            for (int e = 0; e < NP; ++e) {
                out[0][e] = fma2(x0, t00[e], out[0][e]);
                out[1][e] = fma2(x1, t00[e], out[1][e]);
                out[2][e] = fma2(x0, t10[e], out[2][e]);
                out[3][e] = fma2(x0, t01[e], out[3][e]);
                if constexpr (KIND == BSPLINE_VGL) {
                    out[4][e] = fma2(x2, t00[e], fma2(x0, add2(t20[e], t02[e]), out[4][e]));
                } else {
                    out[4][e] = fma2(x2, t00[e], out[4][e]);
                    out[5][e] = fma2(x1, t10[e], out[5][e]);
                    out[6][e] = fma2(x1, t01[e], out[6][e]);
                    out[7][e] = fma2(x0, t20[e], out[7][e]);
                    out[8][e] = fma2(x0, t11[e], out[8][e]);
                    out[9][e] = fma2(x0, t02[e], out[9][e]);
                }
            }
        }
    }
}

// Pairs of accumulate_x2 back to the floats of accumulate (orbital 2e and 2e + 1 of pair e).
template <int NO, int NP>
__device__ __forceinline__ void unpack_outputs(const f32x2 (&in)[NO][NP], float (&out)[NO][2 * NP]) {
#pragma unroll
    for (int q = 0; q < NO; ++q)
#pragma unroll
        for (int e = 0; e < NP; ++e) unpack2(in[q][e], out[q][2 * e], out[q][2 * e + 1]);
}

// Load 4 consecutive elements of type T from global memory as 2 pairs of floats.
template <typename T> __device__ __forceinline__ void load_row_global_x2(const T *p, f32x2 *o) {
    float f[4];
    load_row_global<T, 4>(p, f);
    o[0] = pack2(f[0], f[1]);
    o[1] = pack2(f[2], f[3]);
}

// Accumulation kind behind an output kind: in a general cell the Laplacian
// mixes all six fractional second derivatives, so VGL accumulates VGH.
template <int KIND, bool LAT> constexpr int acc_kind() { return (LAT && KIND == BSPLINE_VGL) ? BSPLINE_VGH : KIND; }

// Fractional derivatives (layout of acc_kind) to Cartesian ones (layout of
// KIND): g = G g_u, H = G H_u G^T, Laplacian = sum of lapw * H_u.
template <int KIND, int VEC>
__device__ __forceinline__ void to_cartesian(const EvalArgs &A, const float (&in)[nout_of(acc_kind<KIND, true>())][VEC],
                                             float (&out)[nout_of(KIND)][VEC]) {
    const float *G = A.Gf;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        out[0][e] = in[0][e];
        if constexpr (KIND != BSPLINE_V) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
                out[1 + i][e] = fmaf(G[i * 3], in[1][e], fmaf(G[i * 3 + 1], in[2][e], G[i * 3 + 2] * in[3][e]));
            const float hxx = in[4][e], hxy = in[5][e], hxz = in[6][e], hyy = in[7][e], hyz = in[8][e],
                        hzz = in[9][e];
            if constexpr (KIND == BSPLINE_VGL) {
                out[4][e] = fmaf(A.lapw[0], hxx, fmaf(A.lapw[1], hxy, fmaf(A.lapw[2], hxz,
                            fmaf(A.lapw[3], hyy, fmaf(A.lapw[4], hyz, A.lapw[5] * hzz)))));
            } else {
                const float Hu[3][3] = {{hxx, hxy, hxz}, {hxy, hyy, hyz}, {hxz, hyz, hzz}};
                float T[3][3];  // T = H_u G^T
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        T[a][j] = fmaf(Hu[a][0], G[j * 3], fmaf(Hu[a][1], G[j * 3 + 1], Hu[a][2] * G[j * 3 + 2]));
                const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const int i = ij[q][0], j = ij[q][1];
                    out[4 + q][e] = fmaf(G[i * 3], T[0][j], fmaf(G[i * 3 + 1], T[1][j], G[i * 3 + 2] * T[2][j]));
                }
            }
        }
    }
}

// Streaming store of one output component for orbitals n0..n0+VEC-1 of one
// position (elements >= N are skipped). VST: the vector store is aligned.
template <int VEC, bool VST>
__device__ __forceinline__ void store_vec(float *dst, int n0, int N, const float *val) {
    if (VST && n0 + VEC <= N) {
        if constexpr (VEC == 4) {
            __stcs(reinterpret_cast<float4 *>(dst + n0), make_float4(val[0], val[1], val[2], val[3]));
            return;
        } else if constexpr (VEC == 2) {
            __stcs(reinterpret_cast<float2 *>(dst + n0), make_float2(val[0], val[1]));
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e)
        if (n0 + e < N) __stcs(dst + n0 + e, val[e]);
}

// Write all components of one position for orbitals n0..n0+VEC-1.
template <int KIND, int VEC, bool VST>
__device__ __forceinline__ void store_outputs(const EvalArgs &A, long long pos, int n0,
                                              float (&out)[nout_of(KIND)][VEC]) {
    const long long ld = A.ld;
    store_vec<VEC, VST>(A.o0 + pos * ld, n0, A.N, out[0]);
    if constexpr (KIND != BSPLINE_V) {
#pragma unroll
        for (int d = 0; d < 3; ++d) store_vec<VEC, VST>(A.o1 + (pos * 3 + d) * ld, n0, A.N, out[1 + d]);
    }
    if constexpr (KIND == BSPLINE_VGL) store_vec<VEC, VST>(A.o2 + pos * ld, n0, A.N, out[4]);
    if constexpr (KIND == BSPLINE_VGH) {
#pragma unroll
        for (int d = 0; d < 6; ++d) store_vec<VEC, VST>(A.o2 + (pos * 6 + d) * ld, n0, A.N, out[4 + d]);
    }
}

// ---------------------------------------------------------------------------
// mbarrier / TMA wrappers (sm_90+ PTX, used on sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every wait in this library is bounded: after kWaitLimitNs the waiter records
// BSPLINE_ERR_TIMEOUT in the table's status word and gives up.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *status,
                                                  uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > limit_ns) {
            if (status) atomicExch(status, (int)BSPLINE_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// One 4-D tiled TMA load into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch (PTX griddepcontrol). A kernel launched with
// the programmatic stream serialization attribute may start while the kernel
// before it in the stream is still running, once every CTA of that kernel has
// executed pdl_trigger() (or exited). pdl_wait() then blocks until the earlier
// kernel has completed and its writes are visible; in a kernel launched
// without the attribute it returns at once. Every evaluation kernel is
// launched with the attribute and waits first, so its CTAs are resident when
// the kernel before it (a sort, or the previous call's evaluation) completes.
// The one-CTA cell sort computes its keys and histogram while the previous
// evaluation drains, and waits for it only before writing the permutation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// kern<<<grid, block, smem, s>>>(args...), with the programmatic stream
// serialization attribute when pdl is set (the kernel must then call
// pdl_wait() before it touches memory the previous kernel may still write).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                            Args &&...args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------
// Cell-sorted evaluation order: a counting sort of positions by the Morton
// code of their coarse cell (i >> shift, j >> shift, k >> shift), done by one
// CTA in shared memory.
// ---------------------------------------------------------------------------
constexpr int kOrderThreads = 1024;
constexpr int kOrderMaxBins = 8192;
constexpr int kOrderKeyCache = 16384;  // positions whose keys the single-table sort keeps in shared memory
constexpr int kOrderMultiMin = 8192;   // above this many positions the sort runs on many CTAs

// Ints of evaluation-order scratch for npos positions: the permutation, then
// (sort on many CTAs) the keys, the histogram and the bin offsets.
inline size_t order_scratch_ints(size_t npos) { return 2 * npos + 2 * (size_t)kOrderMaxBins; }

__device__ __forceinline__ unsigned spread_bits3(unsigned v) {
    // put bit b of v at bit 3b (v < 1024)
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// The sort key only decides which positions run together (locality), never
// a result, so single precision is enough here (the evaluation itself
// reduces cells in FP64).
__device__ __forceinline__ int coarse_coord(float xf, int n, int shift) {
    float u = (xf - floorf(xf)) * (float)n;
    int i = (int)u;
    i = i < 0 ? 0 : (i >= n ? n - 1 : i);
    return i >> shift;
}

// G (row-major L^-1 in single precision, or null): positions are Cartesian and map to u = r G, also in
// single precision (FP64 there doubled the one-CTA sort's time: 20.1 against 10.4 us at 4096 positions).
__device__ __forceinline__ int cell_key(const double *x, const double *y, const double *z, int p, int nx, int ny,
                                        int nz, int shift, const float *G) {
    float u0 = (float)x[p], u1 = (float)y[p], u2 = (float)z[p];
    if (G) {
        const float r0 = u0, r1 = u1, r2 = u2;
        u0 = r0 * G[0] + r1 * G[3] + r2 * G[6];
        u1 = r0 * G[1] + r1 * G[4] + r2 * G[7];
        u2 = r0 * G[2] + r1 * G[5] + r2 * G[8];
    }
    return (int)(spread_bits3((unsigned)coarse_coord(u0, nx, shift)) |
                 (spread_bits3((unsigned)coarse_coord(u1, ny, shift)) << 1) |
                 (spread_bits3((unsigned)coarse_coord(u2, nz, shift)) << 2));
}

// In-place exclusive prefix sum of hist[0 .. nbins) in shared memory. Called by
// every thread of one CTA (blockDim.x a multiple of 32, at most 1024); wsum:
// 32 ints of shared memory. Each thread owns ceil(nbins / blockDim.x)
// consecutive bins. Ends with the CTA synchronised.
__device__ __forceinline__ void block_scan_bins(int *hist, int nbins, int *wsum) {
    const int per = (nbins + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    int local = 0;
    for (int b = b0; b < min(nbins, b0 + per); ++b) local += hist[b];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += v;
        }
        wsum[lane] = w;  // inclusive prefix of warp totals
    }
    __syncthreads();
    int run = incl - local + (wid > 0 ? wsum[wid - 1] : 0);
    for (int b = b0; b < min(nbins, b0 + per); ++b) {
        const int c = hist[b];
        hist[b] = run;
        run += c;
    }
    __syncthreads();
}

// perm[slot] = position, slots ordered by key. Called by every thread of one
// CTA (blockDim.x a multiple of 32, at most 1024); hist: nbins ints and wsum:
// 32 ints of shared memory. keys: npos ints of shared memory that keep each
// position's key from the histogram pass for the scatter pass, or null (the
// scatter recomputes them). The histogram pass loads four positions per
// thread before it counts them, so their load latencies overlap.
__device__ __forceinline__ void block_cell_sort(const double *x, const double *y, const double *z, int npos, int nx,
                                                int ny, int nz, int shift, int nbins, int *perm, int *hist,
                                                int *wsum, const float *G = nullptr, int *keys = nullptr) {
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    constexpr int U = 4;
    for (int p0 = threadIdx.x; p0 < npos; p0 += U * blockDim.x) {
        int k[U];
#pragma unroll
        for (int e = 0; e < U; ++e) {
            const int p = p0 + e * (int)blockDim.x;
            k[e] = p < npos ? cell_key(x, y, z, p, nx, ny, nz, shift, G) : 0;
        }
#pragma unroll
        for (int e = 0; e < U; ++e) {
            const int p = p0 + e * (int)blockDim.x;
            if (p < npos) {
                atomicAdd(&hist[k[e]], 1);
                if (keys) keys[p] = k[e];
            }
        }
    }
    __syncthreads();
    block_scan_bins(hist, nbins, wsum);
    pdl_wait();  // the previous kernel may still read perm (returns at once without the launch attribute)
    for (int p = threadIdx.x; p < npos; p += blockDim.x)
        perm[atomicAdd(&hist[keys ? keys[p] : cell_key(x, y, z, p, nx, ny, nz, shift, G)], 1)] = p;
}

// Coarse cells of 2^shift grid cells per axis (shift >= 2), with at most
// kOrderMaxBins Morton bins.
inline void order_bins(int nx, int ny, int nz, int *shift, int *nbins) {
    const int nmax = nx > ny ? (nx > nz ? nx : nz) : (ny > nz ? ny : nz);
    int sh = 2, bits = 0;
    for (;;) {
        const int coarse = ((nmax - 1) >> sh) + 1;
        bits = 0;
        while ((1 << bits) < coarse) ++bits;
        if ((1 << (3 * bits)) <= kOrderMaxBins) break;
        ++sh;
    }
    *shift = sh;
    *nbins = 1 << (3 * bits);
}

// ---------------------------------------------------------------------------
// Host helpers shared by translation units
// ---------------------------------------------------------------------------
bspline_status cuda_status(cudaError_t e);
// cuTensorMapEncodeTiled from the driver (null if unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
bspline_status get_tma_map(bspline_t t, int nbox, int swizzle, const CUtensorMap **out);
int default_stages(int dtype, int nbox);
size_t tma_smem_bytes(int dtype, int nbox, int stages);
size_t mma_smem_bytes_dtype(int dtype, int stages, int Npad, int nb = 128);
bool mma_fits(int dtype, int stages, int Npad, int ctas, int nb = 128);

// One single-table evaluation: resolves the launch shape (want, else the
// handle's tuning, else the default), orders the positions if asked (in
// perm_scratch, order_scratch_ints(npos) ints, if given, else the handle's scratch) and
// launches the kernel for the table's element type.
bspline_status launch_eval(bspline_t t, int kind, const bspline_tuning &want, int npos, const double *x,
                           const double *y, const double *z, float *o0, float *o1, float *o2, int ld, cudaStream_t s,
                           int *perm_scratch = nullptr);

// Grows the handle's sort scratch to hold npos positions (synchronises the device if it reallocates).
bspline_status reserve_order_scratch(bspline_t t, size_t npos);
// FP32 tables filled in place by the caller's kernel: unit scales, has_coefs set (stream-ordered).
bspline_status finish_f32_table(bspline_t t, cudaStream_t s);

// Cell-sorted order of A's positions (sets A.perm); see launch_eval. perm_scratch, if given, holds
// order_scratch_ints(A.npos) ints.
bspline_status apply_order(bspline_t t, EvalArgs &A, cudaStream_t s, int *perm_scratch);

// Dispatch of one single-table evaluation with a resolved tuning (per dtype TU).
bspline_status launch_eval_f32(int kind, const bspline_tuning &tu, const EvalArgs &A, const CUtensorMap *map,
                               int num_sms, cudaStream_t s);
bspline_status launch_eval_f16(int kind, const bspline_tuning &tu, const EvalArgs &A, const CUtensorMap *map,
                               int num_sms, cudaStream_t s);
bspline_status launch_ratio_f32(int kind, const EvalArgs &A, const float *uinv, int ldu, float *ratio,
                                cudaStream_t s);
bspline_status launch_ratio_f16(int kind, const EvalArgs &A, const float *uinv, int ldu, float *ratio,
                                cudaStream_t s);
bspline_status launch_ratio_bf16(int kind, const EvalArgs &A, const float *uinv, int ldu, float *ratio,
                                 cudaStream_t s);
// Ratio sums on the tensor-core variant (16-bit tables only).
bspline_status launch_ratio_mma_f16(int kind, const bspline_tuning &tu, const EvalArgs &A, const CUtensorMap *map,
                                    int num_sms, const float *uinv, int ldu, float *ratio, cudaStream_t s);
bspline_status launch_ratio_mma_bf16(int kind, const bspline_tuning &tu, const EvalArgs &A, const CUtensorMap *map,
                                     int num_sms, const float *uinv, int ldu, float *ratio, cudaStream_t s);
bspline_status launch_eval_bf16(int kind, const bspline_tuning &tu, const EvalArgs &A, const CUtensorMap *map,
                                int num_sms, cudaStream_t s);

}  // namespace bsg
