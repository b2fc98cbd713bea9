/*
 * bspline_gb300.h - C ABI of the GB300 (sm_103a) tricubic B-spline orbital
 * evaluation library.
 *
 * The library evaluates N periodic tricubic B-spline orbitals at electron
 * positions in the three forms of arXiv:1611.02665 (Mathuriya et al.):
 *   V   - values                                   (Sec. "Baseline and miniQMC")
 *   VGL - values, gradients, Laplacians            (same section)
 *   VGH - values, gradients, Hessians, SoA outputs (Fig. (baselineCode) (b))
 * The function evaluated is Eq. (TricubicValue) of Sec. "QMC and
 * B-spline-based SPOs": phi_n(r) = sum over a 4x4x4 stencil of products of
 * cubic basis weights (Eq. (SplineFunc)) times coefficients p[i'][j'][k'][n].
 *
 * Conventions shared by every call:
 *  - Positions are fractional coordinates in the periodic unit cell, as three
 *    double arrays x[npos], y[npos], z[npos] (structure of arrays). Any real
 *    value is accepted and wrapped into [0,1).
 *  - Derivatives are with respect to those fractional coordinates.
 *  - Outputs are float and written, never accumulated. With leading dimension
 *    ld >= N (elements): v[p*ld + n]; g[(p*3 + d)*ld + n] for d = x,y,z;
 *    h[(p*6 + e)*ld + n] for e = xx,xy,xz,yy,yz,zz; l[p*ld + n]. Elements
 *    n in [N, ld) are left untouched.
 *  - Evaluation calls are asynchronous on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream). Pointers marked "device" must be device memory of
 *    the current device. The caller owns every buffer it passes; the library
 *    never frees or keeps them.
 *  - Argument errors are detected on the host before any launch and return
 *    BSPLINE_ERR_ARG with nothing enqueued. A failed launch returns
 *    BSPLINE_ERR_CUDA. Device-side conditions (a bounded wait that ran out)
 *    set a status word per table, read with bspline_device_status().
 *  - A table handle may be used for evaluation from several host threads at
 *    once; bspline_set_coefs*, bspline_set_tuning and bspline_destroy must not
 *    run concurrently with any other call on the same handle.
 */
#ifndef BSPLINE_GB300_H
#define BSPLINE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BSPLINE_ABI_VERSION 2

typedef struct bspline_s *bspline_t;
typedef struct bspline_plan_s *bspline_plan_t;

typedef enum {
    BSPLINE_OK = 0,
    BSPLINE_ERR_ARG = 1,       /* invalid argument (null, negative, too small, misaligned) */
    BSPLINE_ERR_ALLOC = 2,     /* device or host allocation failed */
    BSPLINE_ERR_CUDA = 3,      /* a CUDA runtime call or launch failed */
    BSPLINE_ERR_DTYPE = 4,     /* unsupported table element type */
    BSPLINE_ERR_STATE = 5,     /* table has no coefficients yet */
    BSPLINE_ERR_TIMEOUT = 6,   /* a bounded device-side wait ran out */
    BSPLINE_ERR_UNSUPPORTED = 7,/* request valid but not supported on this device */
    BSPLINE_ERR_BOUNDS = 8     /* a device-side index check failed (the access was skipped) */
} bspline_status;

/* Element type of the stored coefficient table. FP16/BF16 tables hold
 * p / s_n with s_n = max |p[.][.][.][n]| per orbital and rescale outputs by
 * s_n; accumulation is always FP32. (Reduced-precision storage is not in the
 * paper, which computes in single precision throughout.) */
typedef enum { BSPLINE_F32 = 0, BSPLINE_F16 = 1, BSPLINE_BF16 = 2 } bspline_dtype;

typedef enum { BSPLINE_V = 0, BSPLINE_VGL = 1, BSPLINE_VGH = 2 } bspline_kind;

/* Kernel variants (see bspline_tuning). */
typedef enum {
    BSPLINE_VARIANT_AUTO = 0,  /* the tuned (or default) choice */
    BSPLINE_VARIANT_DIRECT = 1,/* vectorised global loads straight into registers */
    BSPLINE_VARIANT_TMA = 2,   /* persistent; one 4-D TMA box per (position, orbital block) */
    BSPLINE_VARIANT_MMA = 3    /* 16-bit tables: the 64-point stencil sum on the tensor cores
                                  (tcgen05), table rows by TMA; persistent */
} bspline_variant;

typedef struct {
    int nx, ny, nz;     /* grid intervals per axis */
    int N;              /* orbitals */
    int Npad;           /* stored orbitals per row (N rounded up to a 128-byte row) */
    int dtype;          /* bspline_dtype */
    size_t table_bytes; /* (nx+3)*(ny+3)*(nz+3)*Npad*element size */
    int has_coefs;      /* 1 once bspline_set_coefs* completed */
} bspline_info;

/* Launch shape of one evaluation form. Any field 0 takes the default.
 *  variant: bspline_variant.
 *  nb:      orbitals per work unit (DIRECT: per CTA; TMA: per box, <= 256;
 *           MMA: 128 or 256, one or two 128-orbital blocks per hand-off).
 *  ppc:     DIRECT: positions per CTA (0: chosen per call - 1, or for
 *           tables of at most 256 orbitals up to 4 when a call has many
 *           positions). TMA: CTAs per SM. MMA: CTAs per SM (1 or 2).
 *  stages:  TMA and MMA: pipeline depth (work units in flight per CTA, MMA
 *           2..8). DIRECT: 0 = rows loaded into registers; 3, 4, 6 or 8 =
 *           rows staged through a per-thread shared-memory ring of that many
 *           4-row units with cp.async (FP32 tables, nb = 512 only).
 *  order:   0 = positions in input order; 1 = cell-sorted: before the
 *           evaluation a one-CTA counting sort groups the positions by
 *           coarse cell in Morton order, so positions that share stencil
 *           rows run together and read them from L2. Outputs still go to
 *           each position's own slot. Uses a scratch permutation owned by
 *           the handle (allocated on first use), so evaluations with
 *           order = 1 on one handle must not overlap on the GPU. The
 *           default shape (variant AUTO, nothing tuned) sorts when the table
 *           is larger than the device's L2 cache.
 *           The sort and the evaluation use programmatic dependent launch:
 *           the sort starts reading the positions while the kernel before
 *           it in the stream (for instance the previous call's evaluation)
 *           finishes, and waits for that kernel before it writes anything.
 *           A kernel that releases its dependents early (griddepcontrol /
 *           cudaTriggerProgrammaticLaunchCompletion) must therefore not
 *           still be writing the positions; ordinary kernels and copies
 *           are complete before the sort starts. */
typedef struct {
    int variant;
    int nb;
    int ppc;
    int stages;
    int order;
} bspline_tuning;

/* ---- table lifetime (Sec. "Baseline and miniQMC": the table P is created
 *      once, read-only and shared by all walkers) ---- */

/* Create an empty table for an nx*ny*nz periodic grid and N orbitals.
 * nx,ny,nz >= 1 (a grid of fewer than 4 intervals still works: rows wrap),
 * 1 <= N <= 1<<20, dtype a bspline_dtype. Allocates the padded device table
 * [nx+3][ny+3][nz+3][Npad] on the current device. *out receives the handle. */
bspline_status bspline_create(int nx, int ny, int nz, int N, int dtype, bspline_t *out);

/* Free the table and everything the handle owns. Synchronises the device first. */
bspline_status bspline_destroy(bspline_t t);

/* Fill the table from periodic coefficients coefs[nx][ny][nz][N] (float,
 * orbital innermost, host or device memory as on_device says). Builds the
 * padded rows pad[a][b][c] = coefs[(a-1) mod nx][(b-1) mod ny][(c-1) mod nz]
 * so that the stencil of cell i reads rows i..i+3 (knots i-1..i+2 of
 * Eq. (SplineFunc)) without wrapping. Reduced-precision tables compute the
 * per-orbital scale here. Asynchronous on stream for device input; a host
 * input is copied synchronously. */
bspline_status bspline_set_coefs(bspline_t t, const float *coefs, int on_device, void *stream);

/* Fill the table from an already padded float array [nx+3][ny+3][nz+3][N]
 * (host or device). Lets a caller store non-periodic fields, e.g. to check
 * polynomial reproduction. Same scale rule as bspline_set_coefs. */
bspline_status bspline_set_coefs_padded(bspline_t t, const float *padded, int on_device, void *stream);

/* Fill the table from orbital VALUES sampled on the grid, values[nx][ny][nz][N]
 * (float; host or device memory as on_device says): the value of orbital n
 * at the grid point (i/nx, j/ny, k/nz). The coefficients are the periodic
 * cubic B-spline interpolation of the samples (the paper's interpolation
 * tables, Sec. "QMC and B-spline-based SPOs"): at every grid point the spline
 * then equals the sample. The inverse of the knot operator
 * (c[j-1] + 4c[j] + c[j+1])/6 is applied along each axis as a causal and an
 * anti-causal first-order recursion started from periodic sums (exact up to
 * terms below 2^-45 of the largest), then the table is stored as by
 * bspline_set_coefs. Grids up to 1024 points per axis.
 * FP32 tables from device values are solved in the table itself (the values
 * are read, not modified); host values and 16-bit tables use a temporary
 * device copy of the values (nx*ny*nz*N floats, allocated and freed by the
 * call). Returns when the table is filled. */
bspline_status bspline_set_values(bspline_t t, const float *values, int on_device, void *stream);

/* General (non-orthorhombic) cell. L (9 doubles, row-major) holds the three
 * lattice vectors as rows: a Cartesian position is r = u0*L[0..2] +
 * u1*L[3..5] + u2*L[6..8] for fractional u. Once set, the single-table
 * evaluations (bspline_eval_v/vgl/vgh, bspline_eval_host, bspline_eval_ratio)
 * take Cartesian positions (wrapped into the cell through u = r L^-1 in
 * double precision) and return Cartesian derivatives: g = G g_u and
 * H = G H_u G^T with G = L^-1, the Laplacian the trace of H (so VGL also
 * forms the mixed fractional second derivatives). L = NULL returns to the
 * default unit cube, where positions are fractional. A singular or
 * non-finite L gives BSPLINE_ERR_ARG. With a lattice, DIRECT runs with 512
 * orbitals per CTA (FP32 rows staged through the shared-memory ring when the
 * launch shape has a ring depth, as in the unit cube) and the tensor-core
 * variant applies the transform in its epilogue; the TMA variant and batched
 * plans return BSPLINE_ERR_UNSUPPORTED. The cell-sorted order sorts by the
 * fractional cell. (The paper picks VGL or VGH by the simulation cell type,
 * Sec. "Baseline and miniQMC"; it does not give the transform.) */
bspline_status bspline_set_lattice(bspline_t t, const double *L);

bspline_status bspline_get_info(bspline_t t, bspline_info *out);

/* Copy the stored table to host memory, synchronously: dst receives
 * [nx+3][ny+3][nz+3][N] elements of the stored type (float or raw 16-bit
 * codes, orbital padding removed); scale (may be NULL) receives N floats
 * (all 1 for FP32 tables). */
bspline_status bspline_get_table(bspline_t t, void *dst, float *scale);

/* ---- evaluation (Fig. (baselineCode) (b): SoA outputs; Sec. "Baseline and
 *      miniQMC": 64N stride-one reads per position) ---- */

/* x,y,z: device, npos doubles each. v: device, npos*ld floats. npos >= 0
 * (0 is a no-op), ld >= N. */
bspline_status bspline_eval_v(bspline_t t, int npos, const double *x, const double *y,
                              const double *z, float *v, int ld, void *stream);

/* g: device, npos*3*ld floats; l: device, npos*ld floats. */
bspline_status bspline_eval_vgl(bspline_t t, int npos, const double *x, const double *y,
                                const double *z, float *v, float *g, float *l, int ld,
                                void *stream);

/* g: device, npos*3*ld floats; h: device, npos*6*ld floats. */
bspline_status bspline_eval_vgh(bspline_t t, int npos, const double *x, const double *y,
                                const double *z, float *v, float *g, float *h, int ld,
                                void *stream);

/* Fused determinant-ratio consumer (Sec. "QMC and B-spline-based SPOs":
 * for a move of electron e to r', det[A']/det[A] = sum_n phi_n(r') A^-1(n,e),
 * and the gradient ratio is the same sum over grad phi_n). For each position p
 * the caller passes the N inverse entries that multiply phi_n in that sum:
 * uinv[p*ldu + n], n < N (device, float, ldu >= N). With the Slater matrix
 * A[n][i] = phi_n(r_i) this is row e of A^-1 (the paper's A^-1(n,e) indexes
 * the inverse stored transposed). ratio (device, npos * ncomp floats) receives
 * ratio[p*ncomp + q] = sum_n c_q(phi_n)(r_p) * u_p[n] for each output
 * component c_q of `kind`, in the order of the per-orbital outputs:
 *   V   (ncomp 1):  value;
 *   VGL (ncomp 5):  value, d/dx, d/dy, d/dz, Laplacian;
 *   VGH (ncomp 10): value, d/dx, d/dy, d/dz, xx, xy, xz, yy, yz, zz.
 * The per-orbital values are never written to memory. Sums are formed in a
 * fixed order, so results are deterministic. Follows the handle's launch
 * shape of `kind` (bspline_get_tuning): its position order, and for 16-bit
 * tables whose shape is BSPLINE_VARIANT_MMA the sums are formed in that
 * variant's epilogue; otherwise one CTA per position runs the FMA stencil.
 * Asynchronous on stream. */
bspline_status bspline_eval_ratio(bspline_t t, int kind, int npos, const double *x,
                                  const double *y, const double *z, const float *uinv, int ldu,
                                  float *ratio, void *stream);

/* The same evaluation from and to HOST memory. kind picks the form; g and hl
 * are ignored for V; hl is l for VGL and h for VGH. Returns when the outputs
 * are in host memory. Two ways, chosen by bspline_set_host_mode:
 *  - direct: when the GPU can address every buffer (pinned memory, or any
 *    host memory on nodes where the device reads the host page tables, such
 *    as Grace-based nodes over NVLink-C2C), the kernel reads the positions
 *    and writes the outputs in place;
 *  - staged: positions are copied to device buffers, the evaluation runs in
 *    chunks of about 32 MB of outputs on two streams, and the outputs are
 *    copied back, overlapping copies with compute (pinned memory gives
 *    asynchronous copies).
 * Scratch buffers are allocated on first use and kept by the handle. Calls on
 * one handle are serialised. */
bspline_status bspline_eval_host(bspline_t t, int kind, int npos, const double *x,
                                 const double *y, const double *z, float *v, float *g,
                                 float *hl, int ld);

/* Host path of bspline_eval_host: 0 = direct access when every buffer is
 * reachable from the GPU, staged copies otherwise (default); 1 = always
 * staged copies; 2 = direct access only (BSPLINE_ERR_UNSUPPORTED if a buffer
 * is not reachable). */
bspline_status bspline_set_host_mode(bspline_t t, int mode);

/* Device status word of the table: BSPLINE_OK, BSPLINE_ERR_TIMEOUT if a
 * bounded wait inside a kernel ran out, or BSPLINE_ERR_BOUNDS if the
 * position sort met a slot outside its permutation, since the last reset
 * (the first condition met is kept). Synchronises
 * stream first. reset != 0 clears the word. */
bspline_status bspline_device_status(bspline_t t, void *stream, int reset);

/* Self-test of the bounded device waits (failure detection without a fault):
 * one CTA waits on an mbarrier that nothing ever arrives at, with a limit of
 * limit_us microseconds (1..2000000). The wait gives up, records
 * BSPLINE_ERR_TIMEOUT in the table's status word and the kernel returns, so
 * the context stays usable. Read and clear it with bspline_device_status. */
bspline_status bspline_selftest_wait_timeout(bspline_t t, int limit_us, void *stream);

/* ---- launch shape and autotuning (the paper's tunable tile N_b,
 *      Sec. "AoSoA transformation", re-derived for GB300) ---- */

bspline_status bspline_set_tuning(bspline_t t, int kind, const bspline_tuning *tune);
bspline_status bspline_get_tuning(bspline_t t, int kind, bspline_tuning *out);

/* Time candidate launch shapes for `kind` on npos_hint random positions
 * (CUDA events, median of several runs) and keep the fastest in the
 * handle. If wisdom_path is non-NULL: a matching record in that file
 * (same GPU name, grid, N, dtype, kind, npos_hint) is used without timing,
 * and a new result is appended to it as one JSON line. chosen (may be NULL)
 * receives the pick. Synchronous; allocates and frees its own scratch. */
bspline_status bspline_tune(bspline_t t, int kind, int npos_hint, const char *wisdom_path,
                            bspline_tuning *chosen);

/* ---- batched evaluation across walkers and tables (one launch;
 *      the paper's walker-level parallelism, Sec. "Baseline and miniQMC") ---- */

/* One table's share of a batch: npos positions (the concatenated positions
 * of its walkers; device x,y,z) and device outputs laid out as for the
 * single-table calls (hl is l for VGL, h for VGH, unused for V). */
typedef struct {
    bspline_t table;
    int npos;
    const double *x, *y, *z;
    float *v, *g, *hl;
    int ld;
} bspline_batch_item;

/* Build a reusable plan: validates the items, copies their descriptors to
 * device memory owned by the plan. All tables must hold coefficients and
 * share one element type (BSPLINE_ERR_DTYPE otherwise). nitems in 1..1024.
 * The caller keeps the tables and buffers alive while the plan is used.
 * Work is cut into units of (item, position, 512 orbitals), one CTA each, at
 * most 2^31 - 1 units (BSPLINE_ERR_ARG beyond). Launches of one plan must not
 * overlap on the GPU when its positions are cell-sorted (they share the
 * plan's permutation scratch). */
bspline_status bspline_plan_create(const bspline_batch_item *items, int nitems, int kind,
                                   bspline_plan_t *out);
/* Enqueue the batch as one launch on stream (after the sort, if ordered). */
bspline_status bspline_plan_run(bspline_plan_t plan, void *stream);
/* Enqueue the batch as a CUDA graph (captured on first use on a private
 * stream, then replayed on `stream`). */
bspline_status bspline_plan_run_graph(bspline_plan_t plan, void *stream);
/* Order of each item's positions in later runs of the plan: 0 = input order
 * (default), 1 = cell-sorted (one extra launch sorts every item's positions
 * by the Morton code of their coarse cell, one CTA per item, so positions
 * that share stencil rows run together; see bspline_tuning.order). Drops a
 * captured graph, which is captured again on the next run_graph. */
bspline_status bspline_plan_set_order(bspline_plan_t plan, int order);

/* How a plan runs (bspline_plan_set_mode):
 *  BSPLINE_PLAN_ONE_LAUNCH (default): the batched kernel over all items, one
 *    launch (after the sort if ordered), one CTA per unit of 512 orbitals.
 *  BSPLINE_PLAN_PER_TABLE: one single-table evaluation per item, in item
 *    order on the stream, each with its table's launch shape
 *    (bspline_get_tuning: tuned, else the default, with its own position
 *    order); the plan's order does not apply. Setting it sizes every
 *    table's sort scratch (may synchronise the device), so graph captures
 *    never allocate. Runs of such a plan must not overlap on the GPU with
 *    other sorted evaluations of its tables. A captured graph keeps the
 *    launch shapes the tables had when it was captured.
 * Changing the mode drops a captured graph. */
#define BSPLINE_PLAN_ONE_LAUNCH 0
#define BSPLINE_PLAN_PER_TABLE 1
bspline_status bspline_plan_set_mode(bspline_plan_t plan, int mode);
bspline_status bspline_plan_get_mode(bspline_plan_t plan, int *mode, int *order);

/* Staging depth of the one-launch kernel (the paper's tunable tile, Sec.
 * "AoSoA transformation", applied to how a unit's rows reach the SM):
 * 0 = each thread loads its 64 stencil rows into registers, a slice of 16
 * at a time; 4 or 6 = the rows go through a per-thread ring of that many
 * 4-row units in shared memory filled by cp.async (R * 8 KB per CTA), so
 * the next units are in flight while a thread computes, as in the
 * single-table staged launch shape. A new plan has 4 for FP32 tables and 0
 * for 16-bit ones. The ring takes FP32 plans only (BSPLINE_ERR_UNSUPPORTED
 * otherwise); other values give BSPLINE_ERR_ARG. Changing it drops a
 * captured graph. Results do not depend on it. */
bspline_status bspline_plan_set_stages(bspline_plan_t plan, int stages);
bspline_status bspline_plan_get_stages(bspline_plan_t plan, int *stages);

/* Autotune the plan (the paper's tile tuning, Sec. "AoSoA transformation",
 * at the level of a batch): times,
 * with CUDA events on stream, `reps` runs (1..100, after one warm-up) of
 * each candidate - one launch in input order or cell-sorted, each with rows
 * into registers or (FP32 plans) through the 4-unit shared-memory ring, and
 * one evaluation per table - and keeps the fastest (median), including its
 * staging depth (bspline_plan_get_stages). chosen_mode and
 * chosen_order (may be NULL) receive it. Synchronous; the outputs hold the
 * last run's results (every candidate writes the same values). */
bspline_status bspline_plan_tune(bspline_plan_t plan, int reps, void *stream, int *chosen_mode,
                                 int *chosen_order);
bspline_status bspline_plan_destroy(bspline_plan_t plan);

/* Convenience: create a plan, run it on stream, wait for the stream, and
 * release the plan. Returns after the outputs are written. */
bspline_status bspline_eval_batched(const bspline_batch_item *items, int nitems, int kind,
                                    void *stream);

/* The same batched evaluation without allocating anything (the paper has no
 * counterpart; this serves callers that cannot or must not allocate device
 * memory around an evaluation, e.g. an application whose own memory manager
 * owns all the device memory it may use, or a loop that must never reach
 * cudaMalloc/cudaFree because those can synchronise the device or fail under
 * memory pressure). The caller still passes every input and output; the
 * scratch (the item descriptors) lives in a fixed device array compiled into
 * the library: 8192 bytes on each GPU that loads the library, held until the
 * process exits.
 *  - nitems: 1..BSPLINE_NOALLOC_MAX_ITEMS; more returns BSPLINE_ERR_ARG with
 *    nothing enqueued. Tables, outputs and errors as for bspline_plan_create.
 *  - The first call on a device (with that device current) looks up the
 *    device address of the array and keeps it for the life of the process:
 *    do not use this entry point across a cudaDeviceReset.
 *  - Never call it on a stream that is capturing a CUDA graph: the
 *    descriptors are copied from the call's own stack frame, which a replayed
 *    graph would read after it is gone. A capturing stream (or the legacy
 *    stream while another stream captures) returns BSPLINE_ERR_UNSUPPORTED
 *    with nothing enqueued.
 *  - Every call shares the one array, which keeps the last call's contents.
 *    Calls on the same stream
 *    are ordered; calls that overlap on the GPU (different streams, or
 *    different host threads) race on the array and must not be made.
 *  - Asynchronous on stream: descriptors are copied from host stack memory
 *    with cudaMemcpyAsync, then one launch. Because that source is pageable
 *    memory, the copy may first wait for earlier work on the stream, so the
 *    call can block the host until then. */
#define BSPLINE_NOALLOC_MAX_ITEMS 64
bspline_status bspline_eval_batched_noalloc(const bspline_batch_item *items, int nitems, int kind,
                                            void *stream);

/* Read bandwidth of the current device's memory hierarchy for a working set
 * of `bytes` (a multiple of 16): allocates and zeroes a device buffer, reads
 * it once to warm the caches, then times `reps` (1..1000) launches with CUDA
 * events on `stream` and stores the median rate in *gbs (GB/s, 1e9 bytes/s).
 * Each launch reads the whole buffer as many times as it takes to read at
 * least 1 GiB, so launch latency does not count. A
 * buffer well below the L2 size gives the L2 read bandwidth (the roofline of
 * evaluations whose table stays in L2); one well above it, the DRAM read
 * bandwidth. Synchronous; frees what it allocated. */
bspline_status bspline_measure_read_bandwidth(size_t bytes, int reps, double *gbs, void *stream);

/* ---- misc ---- */
const char *bspline_status_str(bspline_status s);
int bspline_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BSPLINE_GB300_H */
