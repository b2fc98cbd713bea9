// Coefficients from orbital values on the grid: the periodic cubic
// B-spline interpolation solve.
//
// The paper calls the coefficient tables interpolation tables (Sec. "QMC and
// B-spline-based SPOs"): coefficients are chosen so that the spline takes
// given values at the grid points. At a knot (t = 0 on every axis) the
// stencil weights are (1/6, 4/6, 1/6, 0) (Eq. (SplineFunc)), so the spline's
// knot values are the tensor product, over the three axes, of the circulant
// operator (T c)_j = (c_{j-1} + 4 c_j + c_{j+1}) / 6. The solve applies T^-1
// along x, then y, then z.
//
// T^-1 as a recursive filter (Unser, Aldroubi and Eden, "Fast B-spline
// transforms", 1991): with z = sqrt(3) - 2, the root of z^2 + 4 z + 1 = 0
// inside the unit circle, (w^-1 + 4 + w) = -(1/z)(1 - z w^-1)(1 - z w), so
//     T^-1 = -6 z / ((1 - z w^-1)(1 - z w)):
// a causal recursion c+_i = f_i + z c+_{i-1}, an anti-causal one
// d_i = c+_i + z d_{i+1}, and c_i = -6 z d_i. On a periodic line of n points
// each recursion starts from its input summed over every periodic image,
//     c+_0 = sum_{k<n} z^k f_{-k} / (1 - z^n),
//     d_{n-1} = sum_{k<n} z^k c+_{n-1+k} / (1 - z^n),
// where terms with |z|^k < 2^-45 (k >= 24) are dropped. About 4 n operations
// per line, against n^2 for the equivalent circular convolution with the
// inverse's taps.
//
// One warp per (line, block of 32 orbitals): lane o solves orbital n0 + o,
// staging its column of the line in shared memory (up to 1024 points, 128 KB
// per warp), so each pass reads and writes the data once, in place.
#include <math.h>

#include <algorithm>
#include <vector>

#include "bspline_internal.cuh"

using namespace bsg;

namespace {

constexpr int kInterpOrb = 32;     // orbitals per CTA (one warp)
constexpr int kInterpMaxN = 1024;  // points per line
constexpr int kInterpTerms = 24;   // terms of the periodic start sums (|z|^24 < 2^-45)

// data[line base + i*stride_i + n] for i < n_axis; one CTA per (line, orbital block).
// Lines are enumerated by (outer, inner): line base = outer * stride_outer + inner * stride_inner.
// zn_inv = 1 / (1 - z^n_axis).
__global__ void __launch_bounds__(kInterpOrb)
    interp_axis_kernel(float *data, int n_axis, long long stride_i, int n_inner, long long stride_outer,
                       long long stride_inner, int N, float zn_inv) {
    extern __shared__ float line[];  // [n_axis][kInterpOrb]: lane o uses column o only
    const float z = -0.267949192431122706f;  // sqrt(3) - 2
    const int line_id = blockIdx.x;
    const int outer = line_id / n_inner, inner = line_id % n_inner;
    const long long base = outer * stride_outer + inner * stride_inner;
    const int o = threadIdx.x;
    const int n = n_axis;
    const bool live = (int)blockIdx.y * kInterpOrb + o < N;
    float *col = line + o;
    const float *src = data + base + (long long)blockIdx.y * kInterpOrb + o;
#pragma unroll 8
    for (int i = 0; i < n; ++i) col[i * kInterpOrb] = live ? src[i * stride_i] : 0.f;
    const int K = min(n, kInterpTerms);
    // causal: c+_0 from the periodic sum, then c+_i = f_i + z c+_{i-1}
    float acc = 0.f, zk = 1.f;
    for (int k = 0; k < K; ++k) {
        acc = fmaf(zk, col[(k == 0 ? 0 : n - k) * kInterpOrb], acc);
        zk *= z;
    }
    float c = acc * zn_inv;
    col[0] = c;
    for (int i = 1; i < n; ++i) {
        c = fmaf(z, c, col[i * kInterpOrb]);
        col[i * kInterpOrb] = c;
    }
    // anti-causal: d_{n-1} from the periodic sum over c+, then d_i = c+_i + z d_{i+1}; c_i = -6 z d_i
    acc = 0.f;
    zk = 1.f;
    for (int k = 0; k < K; ++k) {
        acc = fmaf(zk, col[(k == 0 ? n - 1 : k - 1) * kInterpOrb], acc);
        zk *= z;
    }
    const float gain = -6.f * z;
    float d = acc * zn_inv;
    col[(n - 1) * kInterpOrb] = gain * d;
    for (int i = n - 2; i >= 0; --i) {
        d = fmaf(z, d, col[i * kInterpOrb]);
        col[i * kInterpOrb] = gain * d;
    }
    if (!live) return;
    float *dst = data + base + (long long)blockIdx.y * kInterpOrb + o;
#pragma unroll 8
    for (int i = 0; i < n; ++i) dst[i * stride_i] = col[i * kInterpOrb];
}

}  // namespace

extern "C" bspline_status bspline_set_values(bspline_t t, const float *values, int on_device, void *stream) {
    if (!t || !values) return BSPLINE_ERR_ARG;
    if (t->nx > kInterpMaxN || t->ny > kInterpMaxN || t->nz > kInterpMaxN) return BSPLINE_ERR_UNSUPPORTED;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != t->device) return BSPLINE_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nx = t->nx, ny = t->ny, nz = t->nz, N = t->N;
    const size_t elems = (size_t)nx * ny * nz * N;
    float *work = nullptr;
    cudaError_t e = cudaMalloc(&work, elems * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(work, values, elems * sizeof(float),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    static bool attr = false;
    if (e == cudaSuccess && !attr) {
        e = cudaFuncSetAttribute(interp_axis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float) * kInterpMaxN * kInterpOrb));
        attr = e == cudaSuccess;
    }
    const long long sN = N, sz = (long long)N, sy = (long long)nz * N, sx = (long long)ny * nz * N;
    const unsigned oblocks = (unsigned)((N + kInterpOrb - 1) / kInterpOrb);
    struct Pass {
        int n;
        long long stride;
        int lines, inner;
        long long so, si;
    };
    // x: lines over (j,k) = inner index of length ny*nz with stride N; y: outer i, inner k; z: lines over (i,j)
    const Pass passes[3] = {
        {nx, sx, ny * nz, ny * nz, 0, sN},
        {ny, sy, nx * nz, nz, sx, sz},
        {nz, sz, nx * ny, ny, sx, sy},
    };
    for (int p = 0; p < 3 && e == cudaSuccess; ++p) {
        const Pass &P = passes[p];
        const float zn_inv = (float)(1.0 / (1.0 - std::pow(std::sqrt(3.0) - 2.0, P.n)));
        dim3 grid((unsigned)P.lines, oblocks);
        interp_axis_kernel<<<grid, kInterpOrb, sizeof(float) * P.n * kInterpOrb, s>>>(work, P.n, P.stride, P.inner,
                                                                                     P.so, P.si, N, zn_inv);
        e = cudaGetLastError();
    }
    bspline_status st = cuda_status(e);
    if (st == BSPLINE_OK) st = bspline_set_coefs(t, work, 1, stream);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(work);
    if (st != BSPLINE_OK) return st;
    return cuda_status(e2);
}
