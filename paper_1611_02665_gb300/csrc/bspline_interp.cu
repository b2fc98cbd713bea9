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
// per warp). The line's loads are all issued at once as asynchronous copies
// into shared memory. Consecutive CTAs take consecutive orbital blocks of one
// line, so each row is read and written in one contiguous run. For FP32
// tables from device samples the passes need no scratch: the x pass reads the
// samples and writes the padded table's interior rows, the y and z passes work
// there in place, and the z pass also writes the periodic copies of each row;
// the samples are read once and the table written once. Other tables and host
// samples run on a scratch copy, and 16-bit tables are quantised from it.
#include <math.h>

#include <algorithm>
#include <vector>

#include "bspline_internal.cuh"

using namespace bsg;

namespace {

constexpr int kInterpOrb = 32;     // orbitals per CTA (one warp)
constexpr int kInterpMaxN = 1024;  // points per line
constexpr int kInterpTerms = 24;   // terms of the periodic start sums (|z|^24 < 2^-45)

// Where a pass reads or writes its lines: element (line (outer, inner), point i, orbital n) at
// ptr[outer * so + inner * si + i * st + n].
struct LineArr {
    float *ptr;
    long long st, so, si;
};

// The padded FP32 table as the destination of the last pass (along z).
struct PadDst {
    float *table;
    int nx, ny, nz, Npad;
};

// Padded indices along an axis of n points that repeat point i: padded index a takes point (a - 1) mod n,
// a < n + 3 (one to four of them). Returns their count.
__device__ __forceinline__ int padded_copies(int i, int n, int (&out)[4]) {
    int c = 0;
#pragma unroll
    for (int m = -1; m <= 2; ++m) {
        const int a = i + 1 + m * n;
        if (a >= 0 && a < n + 3) out[c++] = a;
    }
    return c;
}

__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}

// One CTA (one warp) per (line, block of 32 orbitals), CTA g taking orbital block g % nob of line g / nob
// (lines (outer, inner) of n_axis points, inner fastest). Reads src, writes dst (the same array in place).
// PAD: the pass along z, lines (outer, inner) = (i, j), writing every padded row that repeats a point into
// pad.table instead of dst; lanes past N (up to Npad) write the zero padding columns. zn_inv =
// 1 / (1 - z^n_axis).
template <bool PAD>
__global__ void __launch_bounds__(kInterpOrb)
    interp_axis_kernel(const LineArr src, const LineArr dst, int n_axis, int n_inner, int nob, int N, float zn_inv,
                       PadDst pad) {
    extern __shared__ float line[];  // [n_axis][kInterpOrb]: lane o uses column o only
    const float z = -0.267949192431122706f;  // sqrt(3) - 2
    const long long g = blockIdx.x;
    const int line_id = (int)(g / nob), ob = (int)(g % nob);
    const int outer = line_id / n_inner, inner = line_id % n_inner;
    const int o = threadIdx.x;
    const int n = n_axis;
    const int col_n = ob * kInterpOrb + o;
    const bool live = col_n < N;
    float *col = line + o;
    if (live) {
        const float *s = src.ptr + outer * src.so + inner * src.si + col_n;
        for (int i = 0; i < n; ++i) cp_async4(col + i * kInterpOrb, s + i * src.st);
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    } else {
        for (int i = 0; i < n; ++i) col[i * kInterpOrb] = 0.f;
    }
    const int K = min(n, kInterpTerms);
    // causal: c+_0 from the periodic sum, then c+_i = f_i + z c+_{i-1}
    float acc = 0.f, zk = 1.f;
    for (int k = 0; k < K; ++k) {
        acc = fmaf(zk, col[(k == 0 ? 0 : n - k) * kInterpOrb], acc);
        zk *= z;
    }
    float c = acc * zn_inv;
    col[0] = c;
#pragma unroll 4
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
#pragma unroll 4
    for (int i = n - 2; i >= 0; --i) {
        d = fmaf(z, d, col[i * kInterpOrb]);
        col[i * kInterpOrb] = gain * d;
    }
    if constexpr (!PAD) {
        if (!live) return;
        float *out = dst.ptr + outer * dst.so + inner * dst.si + col_n;
#pragma unroll 8
        for (int i = 0; i < n; ++i) out[i * dst.st] = col[i * kInterpOrb];
    } else {
        if (col_n >= pad.Npad) return;
        int as[4], bs[4];
        const int na = padded_copies(outer, pad.nx, as), nb = padded_copies(inner, pad.ny, bs);
        const long long rows_c = pad.nz + 3, rows_bc = (long long)(pad.ny + 3) * rows_c;
        for (int ia = 0; ia < na; ++ia)
            for (int ib = 0; ib < nb; ++ib) {
                float *rowp = pad.table + (as[ia] * rows_bc + bs[ib] * rows_c) * pad.Npad + col_n;
                // padded rows 1..n along z repeat points 0..n-1; rows 0, n+1 and n+2 repeat n-1, 0 and 1 mod n
#pragma unroll 8
                for (int k = 0; k < n; ++k) rowp[(long long)(k + 1) * pad.Npad] = col[k * kInterpOrb];
                rowp[0] = col[(n - 1) * kInterpOrb];
                rowp[(long long)(n + 1) * pad.Npad] = col[0];
                rowp[(long long)(n + 2) * pad.Npad] = col[(1 % n) * kInterpOrb];
            }
    }
}

}  // namespace

extern "C" bspline_status bspline_set_values(bspline_t t, const float *values, int on_device, void *stream) {
    if (!t || !values) return BSPLINE_ERR_ARG;
    if (t->nx > kInterpMaxN || t->ny > kInterpMaxN || t->nz > kInterpMaxN) return BSPLINE_ERR_UNSUPPORTED;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != t->device) return BSPLINE_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nx = t->nx, ny = t->ny, nz = t->nz, N = t->N, Npad = t->Npad;
    const size_t elems = (size_t)nx * ny * nz * N;
    const bool to_table = t->dtype == BSPLINE_F32;  // the last pass writes the padded table
    // FP32 tables from device samples: the x pass reads the samples and writes the table's interior rows
    // (padded row (i+1, j+1, k+1) holds point (i, j, k)), the y pass works there in place, and the z pass
    // in place too, adding the periodic copies; those lie outside the interior, which is all any line reads.
    // Otherwise the passes run on a scratch copy of the samples.
    const bool in_table = to_table && on_device;
    float *work = nullptr;
    cudaError_t e = cudaSuccess;
    if (!in_table) {
        e = cudaMalloc(&work, elems * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(work, values, elems * sizeof(float),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    }
    static bool attr[2] = {false, false};  // idempotent; a race only repeats the call
    for (int pad = 0; pad < 2 && e == cudaSuccess; ++pad) {
        if (attr[pad]) continue;
        e = cudaFuncSetAttribute(pad ? interp_axis_kernel<true> : interp_axis_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float) * kInterpMaxN * kInterpOrb));
        attr[pad] = e == cudaSuccess;
    }
    // element strides of point (i, j, k): the samples' layout, and the padded table's
    const long long ux = (long long)ny * nz * N, uy = (long long)nz * N, uz = N;
    const long long px = (long long)(ny + 3) * (nz + 3) * Npad, py = (long long)(nz + 3) * Npad, pz = Npad;
    float *table = static_cast<float *>(t->table);
    float *interior = table + px + py + pz;  // padded row (1, 1, 1)
    // lines of each pass: x over (outer j, inner k), y over (i, k), z over (i, j)
    auto lines_of = [](int p, float *ptr, long long sx, long long sy, long long sz) {
        if (p == 0) return LineArr{ptr, sx, sy, sz};
        if (p == 1) return LineArr{ptr, sy, sx, sz};
        return LineArr{ptr, sz, sx, sy};
    };
    const int npts[3] = {nx, ny, nz}, ninner[3] = {nz, nz, ny}, nlines[3] = {ny * nz, nx * nz, nx * ny};
    const PadDst dst{table, nx, ny, nz, Npad};
    for (int p = 0; p < 3 && e == cudaSuccess; ++p) {
        const float zn_inv = (float)(1.0 / (1.0 - std::pow(std::sqrt(3.0) - 2.0, npts[p])));
        const bool pad = to_table && p == 2;
        LineArr src, out;
        if (in_table) {
            src = p == 0 ? lines_of(p, const_cast<float *>(values), ux, uy, uz) : lines_of(p, interior, px, py, pz);
            out = lines_of(p, interior, px, py, pz);
        } else {
            src = out = lines_of(p, work, ux, uy, uz);
        }
        const int nob = ((pad ? Npad : N) + kInterpOrb - 1) / kInterpOrb;
        const long long grid = (long long)nlines[p] * nob;
        if (grid > 0x7fffffffLL) {
            e = cudaErrorInvalidValue;
            break;
        }
        const size_t smem = sizeof(float) * npts[p] * kInterpOrb;
        if (pad)
            interp_axis_kernel<true><<<(unsigned)grid, kInterpOrb, smem, s>>>(src, out, npts[p], ninner[p], nob, N,
                                                                             zn_inv, dst);
        else
            interp_axis_kernel<false><<<(unsigned)grid, kInterpOrb, smem, s>>>(src, out, npts[p], ninner[p], nob, N,
                                                                              zn_inv, dst);
        e = cudaGetLastError();
    }
    bspline_status st = cuda_status(e);
    if (st == BSPLINE_OK) st = to_table ? finish_f32_table(t, s) : bspline_set_coefs(t, work, 1, stream);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (work) cudaFree(work);
    if (st != BSPLINE_OK) return st;
    return cuda_status(e2);
}
