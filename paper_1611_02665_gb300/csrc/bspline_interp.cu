// Coefficients from orbital values on the grid: the periodic cubic
// B-spline interpolation solve.
//
// The paper calls the coefficient tables interpolation tables (Sec. "QMC and
// B-spline-based SPOs"): coefficients are chosen so that the spline takes
// given values at the grid points. At a knot (t = 0 on every axis) the
// stencil weights are (1/6, 4/6, 1/6, 0) (Eq. (SplineFunc)), so the spline's
// knot values are the tensor product, over the three axes, of the circulant
// operator (T c)_j = (c_{j-1} + 4 c_j + c_{j+1}) / 6. Its inverse on a
// periodic line of n points is a circular convolution with
//     G_k = sqrt(3) (lambda^k + lambda^(n-k)) / (1 - lambda^n),  lambda = sqrt(3) - 2,
// for k = 0..n-1 (the bi-infinite inverse sqrt(3) lambda^|k|, summed over
// periodic images). The solve applies it along x, then y, then z.
//
// One CTA per (line, block of 32 orbitals): the whole line of the block sits
// in shared memory (up to 1024 points, 128 KB), so each pass reads and writes
// the table once, in place.
#include <math.h>

#include <algorithm>
#include <vector>

#include "bspline_internal.cuh"

using namespace bsg;

namespace {

constexpr int kInterpOrb = 32;     // orbitals per CTA
constexpr int kInterpThreads = 256;
constexpr int kInterpMaxN = 1024;  // points per line

// data[line base + i*stride_i + n] for i < n_axis; one CTA per (line, orbital block).
// Lines are enumerated by (outer, inner): line base = outer * stride_outer + inner * stride_inner.
__global__ void __launch_bounds__(kInterpThreads)
    interp_axis_kernel(float *data, const float *__restrict__ taps, int n_axis, long long stride_i, int n_inner,
                       long long stride_outer, long long stride_inner, int N) {
    extern __shared__ float line[];  // [n_axis][kInterpOrb]
    const int line_id = blockIdx.x;
    const int outer = line_id / n_inner, inner = line_id % n_inner;
    const long long base = outer * stride_outer + inner * stride_inner;
    const int n0 = blockIdx.y * kInterpOrb;
    const int o = threadIdx.x % kInterpOrb;  // orbital within the block
    const int r0 = threadIdx.x / kInterpOrb;  // first point this thread handles
    constexpr int rstep = kInterpThreads / kInterpOrb;
    const bool live = n0 + o < N;
    for (int i = r0; i < n_axis; i += rstep)
        line[i * kInterpOrb + o] = live ? data[base + i * stride_i + n0 + o] : 0.f;
    __syncthreads();
    // Results go straight back to global memory: the inputs are read from the
    // shared copy of the line only, and other CTAs own other lines.
    for (int i = r0; i < n_axis; i += rstep) {
        float acc = 0.f;
        // c_i = sum_k G_k f_{(i - k) mod n}
        int src = i;
        for (int k = 0; k < n_axis; ++k) {
            acc = fmaf(taps[k], line[src * kInterpOrb + o], acc);
            src = src == 0 ? n_axis - 1 : src - 1;
        }
        if (live) data[base + i * stride_i + n0 + o] = acc;
    }
}

// Inverse-circulant taps of one axis, in double precision.
std::vector<float> interp_taps(int n) {
    const double s3 = std::sqrt(3.0), lam = s3 - 2.0;
    const double ln = std::pow(lam, n);
    std::vector<float> g(n);
    for (int k = 0; k < n; ++k) g[k] = (float)(s3 * (std::pow(lam, k) + std::pow(lam, n - k)) / (1.0 - ln));
    return g;
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
    float *work = nullptr, *dtaps = nullptr;
    cudaError_t e = cudaMalloc(&work, elems * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dtaps, sizeof(float) * (nx + ny + nz));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(work, values, elems * sizeof(float),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    std::vector<float> taps;
    for (int n : {nx, ny, nz}) {
        std::vector<float> g = interp_taps(n);
        taps.insert(taps.end(), g.begin(), g.end());
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtaps, taps.data(), sizeof(float) * taps.size(), cudaMemcpyHostToDevice, s);
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
        int tap_off;
    };
    // x: lines over (j,k) = inner index of length ny*nz with stride N; y: outer i, inner k; z: lines over (i,j)
    const Pass passes[3] = {
        {nx, sx, ny * nz, ny * nz, 0, sN, 0},
        {ny, sy, nx * nz, nz, sx, sz, nx},
        {nz, sz, nx * ny, ny, sx, sy, nx + ny},
    };
    for (int p = 0; p < 3 && e == cudaSuccess; ++p) {
        const Pass &P = passes[p];
        dim3 grid((unsigned)P.lines, oblocks);
        interp_axis_kernel<<<grid, kInterpThreads, sizeof(float) * P.n * kInterpOrb, s>>>(
            work, dtaps + P.tap_off, P.n, P.stride, P.inner, P.so, P.si, N);
        e = cudaGetLastError();
    }
    bspline_status st = cuda_status(e);
    if (st == BSPLINE_OK) st = bspline_set_coefs(t, work, 1, stream);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(work);
    cudaFree(dtaps);
    if (st != BSPLINE_OK) return st;
    return cuda_status(e2);
}
