// Batched evaluation across walkers and tables in one launch.
//
// The paper runs one walker per thread over a shared table (Sec. "Baseline
// and miniQMC", Fig. (alg:bspline_thd)) and splits each walker's orbitals
// into independent tiles (Sec. "AoSoA transformation", Sec. "Exposing
// Parallelism Within Walker Update"). Here a batch may span several tables of
// different grids and orbital counts, each with its own walkers' positions.
// The work is cut into equal-cost units - (table, position, block of NB
// orbitals) - numbered table by table, one CTA per unit, so tables of uneven
// size share the GPU without a launch per table; the plan can also be
// replayed as a CUDA graph.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "bspline_eval_kernels.cuh"

using namespace bsg;

namespace {

constexpr int kMaxItems = 1024;
constexpr int kBatchNT = 128;               // threads per CTA
constexpr int kBatchVec = 4;                // orbitals per thread
constexpr int kBatchNB = kBatchNT * kBatchVec;  // orbitals per unit

// Device descriptor of one item of a batch.
struct BatchItemDev {
    const void *table;
    const float *scale;
    const double *x, *y, *z;
    float *o0, *o1, *o2;
    long long si, sj;
    long long unit_begin;  // first unit of this item
    int nx, ny, nz, N, Npad, ld, npos, nblk, vst;
};

// Register budget: the single-table kernel's for the same way of loading rows (direct_min_blocks into
// registers, async_min_blocks through the ring).
template <int KIND, typename T, int R> constexpr int batched_min_blocks() {
    return R > 0 ? async_min_blocks<KIND, kBatchNT, R>() : direct_min_blocks<KIND, T, kBatchNT>();
}

// One CTA per unit u = blockIdx.x. perm / perm_begin (both null for input
// order): item k's positions are taken in the order perm[perm_begin[k] + slot].
// R = 0: rows loaded into registers; R > 0 (FP32 tables): rows staged through
// a per-thread shared-memory ring of R 4-row units (accumulate_staged, the
// single-table staged kernel's loop), R * 8 KB of dynamic shared memory.
template <int KIND, typename T, int R>
__global__ void __launch_bounds__(kBatchNT, (batched_min_blocks<KIND, T, R>()))
    batched_kernel(const BatchItemDev *__restrict__ items, int nitems, const int *__restrict__ perm,
                   const int *__restrict__ perm_begin) {
    constexpr int NO = nout_of(KIND);
    constexpr bool PK = R > 0 && sizeof(T) == 4 && packed_staged_plain<KIND>();
    __shared__ float sW[36];
    __shared__ f32x2 sW2[PK ? 36 : 1];
    __shared__ int sIdx[3];
    __shared__ int sItem, sBlk;
    __shared__ long long sPos;

    const long long u = blockIdx.x;
    if (threadIdx.x < 32) {
        // item of u: the last k with unit_begin <= u (items[0] begins at 0)
        const int lane = threadIdx.x;
        int k;
        if (nitems <= 32) {
            const bool le = lane < nitems && items[lane].unit_begin <= u;
            k = 31 - __clz(__ballot_sync(0xffffffffu, le));
        } else {
            int lo = 0, hi = nitems - 1;
            if (lane == 0)
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (items[mid].unit_begin <= u) lo = mid;
                    else hi = mid - 1;
                }
            k = __shfl_sync(0xffffffffu, lo, 0);
        }
        if (lane < 3) {
            const BatchItemDev &it = items[k];
            const long long local = u - it.unit_begin;
            const long long slot = local / it.nblk;
            const long long pos = perm ? perm[perm_begin[k] + slot] : slot;
            const double *X = lane == 0 ? it.x : (lane == 1 ? it.y : it.z);
            const int n = lane == 0 ? it.nx : (lane == 1 ? it.ny : it.nz);
            int i;
            float t;
            cell_reduce(X[pos], n, i, t);
            basis_weights(t, (float)n, &sW[lane * 12]);
            if constexpr (PK) {
#pragma unroll
                for (int q = 0; q < 12; ++q) sW2[lane * 12 + q] = pack2(sW[lane * 12 + q], sW[lane * 12 + q]);
            }
            sIdx[lane] = i;
            if (lane == 0) {
                sItem = k;
                sBlk = (int)(local - slot * it.nblk);
                sPos = pos;
            }
        }
    }
    __syncthreads();
    const BatchItemDev &it = items[sItem];
    const long long pos = sPos;
    const int n0 = sBlk * kBatchNB + (int)threadIdx.x * kBatchVec;
    if (n0 >= it.Npad) return;
    const T *rowp = static_cast<const T *>(it.table) + (long long)sIdx[0] * it.si + (long long)sIdx[1] * it.sj +
                    (long long)sIdx[2] * it.Npad + n0;
    const long long si = it.si, sj = it.sj, sk = it.Npad;
    float out[NO][kBatchVec];
    if constexpr (R > 0 && sizeof(T) == 4) {
        extern __shared__ __align__(16) float4 batch_ring_raw[];
        float4 *batch_ring = align_ring(batch_ring_raw);  // [R][4][kBatchNT]
        if constexpr (PK)
            accumulate_staged_x2<KIND, kBatchNT, R>(reinterpret_cast<const float *>(rowp), si, sj, sk,
                                                    batch_ring + threadIdx.x, sW2, out);
        else
            accumulate_staged<KIND, kBatchNT, R>(reinterpret_cast<const float *>(rowp), si, sj, sk,
                                                 batch_ring + threadIdx.x, sW, out);
    } else {
        auto rows = [&](int a, int b, float (&pr)[4][kBatchVec]) {
            const T *r = rowp + a * si + b * sj;
#pragma unroll
            for (int c = 0; c < 4; ++c) load_row_global<T, kBatchVec>(r + c * sk, pr[c]);
        };
        accumulate<KIND, kBatchVec>(sW, rows, out);
    }
    if constexpr (sizeof(T) == 2) {
#pragma unroll
        for (int e = 0; e < kBatchVec; ++e) {
            const float sc = it.scale[n0 + e];
#pragma unroll
            for (int q = 0; q < NO; ++q) out[q][e] *= sc;
        }
    }
    EvalArgs A;
    A.N = it.N;
    A.ld = it.ld;
    A.o0 = it.o0;
    A.o1 = it.o1;
    A.o2 = it.o2;
    if (it.vst)
        store_outputs<KIND, kBatchVec, true>(A, pos, n0, out);
    else
        store_outputs<KIND, kBatchVec, false>(A, pos, n0, out);
}

template <typename T, int R>
const void *batched_kernel_ptr(int kind) {
    switch (kind) {
        case BSPLINE_V: return reinterpret_cast<const void *>(batched_kernel<BSPLINE_V, T, R>);
        case BSPLINE_VGL: return reinterpret_cast<const void *>(batched_kernel<BSPLINE_VGL, T, R>);
        default: return reinterpret_cast<const void *>(batched_kernel<BSPLINE_VGH, T, R>);
    }
}

// stages: 0 (rows into registers) for every element type; 4 or 6 (shared-memory ring) for FP32.
const void *kernel_for(int dtype, int kind, int stages = 0) {
    if (dtype == BSPLINE_F32) {
        if (stages == 4) return batched_kernel_ptr<float, 4>(kind);
        if (stages == 6) return batched_kernel_ptr<float, 6>(kind);
        return batched_kernel_ptr<float, 0>(kind);
    }
    if (dtype == BSPLINE_F16) return batched_kernel_ptr<__half, 0>(kind);
    return batched_kernel_ptr<__nv_bfloat16, 0>(kind);
}

size_t batched_smem(int stages) { return stages > 0 ? (size_t)stages * 4 * kBatchNT * sizeof(float4) + kRingAlign : 0; }

bool aligned16(const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

// One CTA per item: cell-sorted order of the item's positions into
// perm[perm_begin[k] ...] (sort[k] = {shift, nbins} of the item's grid).
// Shared memory: max_bins counters, then key_cap cached keys; an item with at
// most key_cap positions keeps its keys there for the scatter pass.
__global__ void __launch_bounds__(kOrderThreads) batched_order_kernel(const BatchItemDev *__restrict__ items,
                                                                      const int *__restrict__ perm_begin,
                                                                      const int2 *__restrict__ sort, int *perm,
                                                                      int max_bins, int key_cap) {
    extern __shared__ int hist[];
    __shared__ int wsum[32];
    const BatchItemDev &it = items[blockIdx.x];
    const int2 sb = sort[blockIdx.x];
    int *keys = it.npos <= key_cap ? hist + max_bins : nullptr;
    block_cell_sort(it.x, it.y, it.z, it.npos, it.nx, it.ny, it.nz, sb.x, sb.y, perm + perm_begin[blockIdx.x], hist,
                    wsum, nullptr, keys);
}

}  // namespace

struct bspline_plan_s {
    int kind = 0, dtype = 0, nitems = 0;
    long long total = 0;                      // units = CTAs of the launch
    BatchItemDev *d_items = nullptr;          // scratch: descriptors
    int order = 0;                            // 1: cell-sorted positions per item
    int *d_perm = nullptr;                    // scratch: per-item evaluation order
    int *d_perm_begin = nullptr;              // [nitems] offsets into d_perm
    int2 *d_sort = nullptr;                   // [nitems] {shift, nbins}
    int max_bins = 0;
    int key_cap = 0;                          // positions whose sort keys fit in the order kernel's shared memory
    int mode = BSPLINE_PLAN_ONE_LAUNCH;       // or BSPLINE_PLAN_PER_TABLE
    int stages = 0;                           // one launch: 0 rows into registers, 4 / 6 shared-memory ring
    std::vector<bspline_batch_item> host_items;  // the items, for per-table runs
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

bspline_status build_descriptors(const bspline_batch_item *items, int nitems, int kind,
                                 std::vector<BatchItemDev> *out, int *dtype, long long *total) {
    if (!items || nitems < 1 || nitems > kMaxItems || kind < BSPLINE_V || kind > BSPLINE_VGH)
        return BSPLINE_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSPLINE_ERR_CUDA;
    long long units = 0;
    out->resize(nitems);
    for (int k = 0; k < nitems; ++k) {
        const bspline_batch_item &s = items[k];
        bspline_t t = s.table;
        if (!t) return BSPLINE_ERR_ARG;
        if (!t->has_coefs) return BSPLINE_ERR_STATE;
        if (t->device != dev) return BSPLINE_ERR_ARG;
        if (t->lattice) return BSPLINE_ERR_UNSUPPORTED;  // batched plans take fractional positions
        if (k == 0) *dtype = t->dtype;
        if (t->dtype != *dtype) return BSPLINE_ERR_DTYPE;
        if (s.npos < 0 || s.ld < t->N) return BSPLINE_ERR_ARG;
        if (s.npos > 0 && (!s.x || !s.y || !s.z || !s.v)) return BSPLINE_ERR_ARG;
        if (s.npos > 0 && kind != BSPLINE_V && (!s.g || !s.hl)) return BSPLINE_ERR_ARG;
        BatchItemDev &d = (*out)[k];
        memset(&d, 0, sizeof d);
        d.table = t->table;
        d.scale = t->scale;
        d.x = s.x;
        d.y = s.y;
        d.z = s.z;
        d.o0 = s.v;
        d.o1 = kind == BSPLINE_V ? nullptr : s.g;
        d.o2 = kind == BSPLINE_V ? nullptr : s.hl;
        d.nx = t->nx;
        d.ny = t->ny;
        d.nz = t->nz;
        d.N = t->N;
        d.Npad = t->Npad;
        d.ld = s.ld;
        d.npos = s.npos;
        d.sj = (long long)(t->nz + 3) * t->Npad;
        d.si = (long long)(t->ny + 3) * d.sj;
        d.nblk = (t->Npad + kBatchNB - 1) / kBatchNB;
        d.vst = (s.ld % 4 == 0) && aligned16(s.v) && (kind == BSPLINE_V || (aligned16(s.g) && aligned16(s.hl)));
        d.unit_begin = units;
        units += (long long)s.npos * d.nblk;
    }
    *total = units;
    return BSPLINE_OK;
}

// One single-table evaluation per item, with each table's own launch shape (its tuning or the default).
bspline_status launch_per_table(bspline_plan_s *p, cudaStream_t s) {
    for (const bspline_batch_item &it : p->host_items) {
        if (it.npos == 0) continue;
        const bool v = p->kind == BSPLINE_V;
        bspline_status st = launch_eval(it.table, p->kind, bspline_tuning{0, 0, 0, 0, 0}, it.npos, it.x, it.y, it.z,
                                        it.v, v ? nullptr : it.g, v ? nullptr : it.hl, it.ld, s);
        if (st != BSPLINE_OK) return st;
    }
    return BSPLINE_OK;
}

// A captured graph holds the old launch sequence.
void drop_graph(bspline_plan_s *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
}

bspline_status launch_plan(bspline_plan_s *p, cudaStream_t s) {
    if (p->total == 0) return BSPLINE_OK;
    if (p->mode == BSPLINE_PLAN_PER_TABLE) return launch_per_table(p, s);
    const BatchItemDev *items = p->d_items;
    int nitems = p->nitems;
    const int *perm = nullptr, *perm_begin = nullptr;
    cudaError_t e;
    if (p->order) {
        const size_t smem = sizeof(int) * ((size_t)p->max_bins + p->key_cap);
        static bool attr_set = false;  // idempotent; a race only repeats the call
        if (!attr_set) {
            e = cudaFuncSetAttribute(batched_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(int) * (kOrderMaxBins + kOrderKeyCache)));
            if (e != cudaSuccess) return cuda_status(e);
            attr_set = true;
        }
        batched_order_kernel<<<nitems, kOrderThreads, smem, s>>>(p->d_items, p->d_perm_begin, p->d_sort, p->d_perm,
                                                                 p->max_bins, p->key_cap);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
        perm = p->d_perm;
        perm_begin = p->d_perm_begin;
    }
    const void *kern = kernel_for(p->dtype, p->kind, p->stages);
    if (p->stages > 0) {
        // the 6-unit ring (48 KB) and the kernel's static shared memory pass the default 48 KB of a launch
        static bool ring_attr[3][2] = {};  // [kind][4 or 6 units]; idempotent, a race only repeats the call
        bool &done = ring_attr[p->kind][p->stages == 6 ? 1 : 0];
        if (!done) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batched_smem(p->stages));
            if (e != cudaSuccess) return cuda_status(e);
            done = true;
        }
    }
    void *args[] = {(void *)&items, (void *)&nitems, (void *)&perm, (void *)&perm_begin};
    e = cudaLaunchKernel(kern, dim3((unsigned)p->total), dim3(kBatchNT), args, batched_smem(p->stages), s);
    return cuda_status(e);
}

void free_plan(bspline_plan_s *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    cudaFree(p->d_items);
    cudaFree(p->d_perm);
    cudaFree(p->d_perm_begin);
    cudaFree(p->d_sort);
    delete p;
}

}  // namespace

extern "C" {

bspline_status bspline_plan_create(const bspline_batch_item *items, int nitems, int kind, bspline_plan_t *out) {
    if (!out) return BSPLINE_ERR_ARG;
    *out = nullptr;
    std::vector<BatchItemDev> desc;
    int dtype = 0;
    long long total = 0;
    bspline_status st = build_descriptors(items, nitems, kind, &desc, &dtype, &total);
    if (st != BSPLINE_OK) return st;
    if (total > 0x7fffffffLL) return BSPLINE_ERR_ARG;  // one CTA per unit
    bspline_plan_s *p = new (std::nothrow) bspline_plan_s();
    if (!p) return BSPLINE_ERR_ALLOC;
    p->kind = kind;
    p->dtype = dtype;
    // FP32 plans stage their rows through the 4-unit ring by default: five-table VGL batch, one launch,
    // sorted 1.252 -> 1.136 ms, input order 1.954 -> 1.874 ms
    p->stages = dtype == BSPLINE_F32 ? 4 : 0;
    p->nitems = nitems;
    p->total = total;
    p->host_items.assign(items, items + nitems);
    cudaError_t e = cudaMalloc(&p->d_items, sizeof(BatchItemDev) * nitems);
    // evaluation-order scratch (used when bspline_plan_set_order asks for it)
    std::vector<int> pbeg(nitems);
    std::vector<int2> sorts(nitems);
    long long npos_total = 0;
    for (int k = 0; k < nitems; ++k) {
        pbeg[k] = (int)npos_total;
        npos_total += desc[k].npos;
        int sh = 0, nb = 0;
        order_bins(desc[k].nx, desc[k].ny, desc[k].nz, &sh, &nb);
        sorts[k] = make_int2(sh, nb);
        p->max_bins = std::max(p->max_bins, nb);
        p->key_cap = std::max(p->key_cap, std::min(desc[k].npos, kOrderKeyCache));
    }
    if (npos_total > 0x7fffffffLL) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaMalloc(&p->d_perm, sizeof(int) * std::max<long long>(npos_total, 1));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_perm_begin, sizeof(int) * nitems);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_sort, sizeof(int2) * nitems);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_perm_begin, pbeg.data(), sizeof(int) * nitems, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_sort, sorts.data(), sizeof(int2) * nitems, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_items, desc.data(), sizeof(BatchItemDev) * nitems, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_status(e);
    }
    *out = p;
    return BSPLINE_OK;
}

bspline_status bspline_plan_run(bspline_plan_t plan, void *stream) {
    if (!plan) return BSPLINE_ERR_ARG;
    return launch_plan(plan, static_cast<cudaStream_t>(stream));
}

bspline_status bspline_plan_run_graph(bspline_plan_t plan, void *stream) {
    if (!plan) return BSPLINE_ERR_ARG;
    cudaError_t e = cudaSuccess;
    if (!plan->exec) {
        cudaStream_t cap = nullptr;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        bspline_status st = BSPLINE_OK;
        if (e == cudaSuccess) {
            st = launch_plan(plan, cap);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cap, &g);
            if (st == BSPLINE_OK && e2 == cudaSuccess) {
                plan->graph = g;
                e = cudaGraphInstantiate(&plan->exec, g, 0);
            } else {
                if (g) cudaGraphDestroy(g);
                if (e2 != cudaSuccess) e = e2;
            }
        }
        cudaStreamDestroy(cap);
        if (st != BSPLINE_OK) return st;
        if (e != cudaSuccess) return cuda_status(e);
    }
    return cuda_status(cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream)));
}

bspline_status bspline_plan_set_order(bspline_plan_t plan, int order) {
    if (!plan || order < 0 || order > 1) return BSPLINE_ERR_ARG;
    if (plan->order != order) {
        plan->order = order;
        drop_graph(plan);
    }
    return BSPLINE_OK;
}

bspline_status bspline_plan_set_stages(bspline_plan_t plan, int stages) {
    if (!plan || (stages != 0 && stages != 4 && stages != 6)) return BSPLINE_ERR_ARG;
    if (stages != 0 && plan->dtype != BSPLINE_F32) return BSPLINE_ERR_UNSUPPORTED;
    if (plan->stages != stages) {
        plan->stages = stages;
        drop_graph(plan);
    }
    return BSPLINE_OK;
}

bspline_status bspline_plan_set_mode(bspline_plan_t plan, int mode) {
    if (!plan || (mode != BSPLINE_PLAN_ONE_LAUNCH && mode != BSPLINE_PLAN_PER_TABLE)) return BSPLINE_ERR_ARG;
    if (mode == BSPLINE_PLAN_PER_TABLE) {
        // size every table's sort scratch now, so a later graph capture never reallocates it
        for (const bspline_batch_item &it : plan->host_items) {
            bspline_status st = reserve_order_scratch(it.table, (size_t)it.npos);
            if (st != BSPLINE_OK) return st;
        }
    }
    if (plan->mode != mode) {
        plan->mode = mode;
        drop_graph(plan);
    }
    return BSPLINE_OK;
}

bspline_status bspline_plan_get_mode(bspline_plan_t plan, int *mode, int *order) {
    if (!plan) return BSPLINE_ERR_ARG;
    if (mode) *mode = plan->mode;
    if (order) *order = plan->order;
    return BSPLINE_OK;
}

bspline_status bspline_plan_get_stages(bspline_plan_t plan, int *stages) {
    if (!plan || !stages) return BSPLINE_ERR_ARG;
    *stages = plan->stages;
    return BSPLINE_OK;
}

bspline_status bspline_plan_tune(bspline_plan_t plan, int reps, void *stream, int *chosen_mode, int *chosen_order) {
    if (!plan || reps < 1 || reps > 100) return BSPLINE_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // {mode, order, stages}: one launch in input or cell-sorted order with rows into registers or (FP32)
    // through the shared-memory ring, and one evaluation per table
    const int cand[5][3] = {{BSPLINE_PLAN_ONE_LAUNCH, 0, 0}, {BSPLINE_PLAN_ONE_LAUNCH, 1, 0},
                            {BSPLINE_PLAN_ONE_LAUNCH, 0, 4}, {BSPLINE_PLAN_ONE_LAUNCH, 1, 4},
                            {BSPLINE_PLAN_PER_TABLE, 0, 0}};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    bspline_status st = cuda_status(e);
    float best = 0.f;
    int pick = -1;
    std::vector<float> ms;
    for (int c = 0; c < 5 && st == BSPLINE_OK; ++c) {
        if (cand[c][2] != 0 && plan->dtype != BSPLINE_F32) continue;  // the ring takes FP32 tables only
        st = bspline_plan_set_mode(plan, cand[c][0]);
        if (st == BSPLINE_OK) st = bspline_plan_set_order(plan, cand[c][1]);
        if (st == BSPLINE_OK) st = bspline_plan_set_stages(plan, cand[c][2]);
        if (st == BSPLINE_OK) st = launch_plan(plan, s);  // warm-up
        ms.clear();
        for (int r = 0; r < reps && st == BSPLINE_OK; ++r) {
            e = cudaEventRecord(ev[0], s);
            if (e == cudaSuccess) st = launch_plan(plan, s);
            if (st == BSPLINE_OK && e == cudaSuccess) e = cudaEventRecord(ev[1], s);
            if (st == BSPLINE_OK && e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            float t = 0.f;
            if (st == BSPLINE_OK && e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
            if (e != cudaSuccess) st = cuda_status(e);
            ms.push_back(t);
        }
        if (st != BSPLINE_OK) break;
        std::sort(ms.begin(), ms.end());
        const float med = ms[ms.size() / 2];
        if (pick < 0 || med < best) {
            best = med;
            pick = c;
        }
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (st != BSPLINE_OK) return st;
    st = bspline_plan_set_mode(plan, cand[pick][0]);
    if (st == BSPLINE_OK) st = bspline_plan_set_order(plan, cand[pick][1]);
    if (st == BSPLINE_OK) st = bspline_plan_set_stages(plan, cand[pick][2]);
    if (st != BSPLINE_OK) return st;
    if (chosen_mode) *chosen_mode = cand[pick][0];
    if (chosen_order) *chosen_order = cand[pick][1];
    return BSPLINE_OK;
}

bspline_status bspline_plan_destroy(bspline_plan_t plan) {
    if (!plan) return BSPLINE_ERR_ARG;
    cudaDeviceSynchronize();
    free_plan(plan);
    return BSPLINE_OK;
}

bspline_status bspline_eval_batched(const bspline_batch_item *items, int nitems, int kind, void *stream) {
    bspline_plan_t p = nullptr;
    bspline_status st = bspline_plan_create(items, nitems, kind, &p);
    if (st != BSPLINE_OK) return st;
    st = bspline_plan_run(p, stream);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    free_plan(p);
    if (st != BSPLINE_OK) return st;
    return cuda_status(e);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched evaluation that allocates nothing.
//
// Some callers cannot allocate GPU memory around an evaluation: for example
// an application whose own memory manager has already reserved the device
// memory it is allowed to use, or a latency-sensitive loop that must not hit
// cudaMalloc/cudaFree (they can synchronise the device and can fail under
// memory pressure). bspline_eval_batched_noalloc serves them. It runs the
// same batched kernel as the plans above, but its scratch (the item
// descriptors) lives in the fixed device array below instead of in memory
// the library allocates.
// ---------------------------------------------------------------------------
namespace {

struct NoAllocScratch {
    BatchItemDev items[BSPLINE_NOALLOC_MAX_ITEMS];
};

}  // namespace

// Shared by every call on a device and kept until the library is unloaded.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

namespace {

constexpr int kNoAllocMaxDevices = 64;

struct NoAllocDevice {
    bool ready;
    unsigned char *scratch;  // device address of g_noalloc_scratch on this device
};

NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// One-time set-up per device, with that device current: look up the device
// address of the scratch array (host code only sees a host-side stand-in for
// the symbol, which no kernel may be given).
bspline_status noalloc_setup(int dev, NoAllocDevice **out) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) return BSPLINE_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e);
        d.scratch = static_cast<unsigned char *>(ptr);
        d.ready = true;
    }
    *out = &d;
    return BSPLINE_OK;
}

// Descriptor of one item, written into caller-provided storage (no allocation).
bspline_status noalloc_descriptor(const bspline_batch_item &s, int kind, int dev, int *dtype, bool first,
                                  long long unit_begin, BatchItemDev *d) {
    bspline_t t = s.table;
    if (!t) return BSPLINE_ERR_ARG;
    if (!t->has_coefs) return BSPLINE_ERR_STATE;
    if (t->device != dev) return BSPLINE_ERR_ARG;
    if (t->lattice) return BSPLINE_ERR_UNSUPPORTED;  // batched evaluation takes fractional positions
    if (first) *dtype = t->dtype;
    if (t->dtype != *dtype) return BSPLINE_ERR_DTYPE;
    if (s.npos < 0 || s.ld < t->N) return BSPLINE_ERR_ARG;
    if (s.npos > 0 && (!s.x || !s.y || !s.z || !s.v)) return BSPLINE_ERR_ARG;
    if (s.npos > 0 && kind != BSPLINE_V && (!s.g || !s.hl)) return BSPLINE_ERR_ARG;
    memset(d, 0, sizeof *d);
    d->table = t->table;
    d->scale = t->scale;
    d->x = s.x;
    d->y = s.y;
    d->z = s.z;
    d->o0 = s.v;
    d->o1 = kind == BSPLINE_V ? nullptr : s.g;
    d->o2 = kind == BSPLINE_V ? nullptr : s.hl;
    d->nx = t->nx;
    d->ny = t->ny;
    d->nz = t->nz;
    d->N = t->N;
    d->Npad = t->Npad;
    d->ld = s.ld;
    d->npos = s.npos;
    d->sj = (long long)(t->nz + 3) * t->Npad;
    d->si = (long long)(t->ny + 3) * d->sj;
    d->nblk = (t->Npad + kBatchNB - 1) / kBatchNB;
    d->vst = (s.ld % 4 == 0) && aligned16(s.v) && (kind == BSPLINE_V || (aligned16(s.g) && aligned16(s.hl)));
    d->unit_begin = unit_begin;
    return BSPLINE_OK;
}

}  // namespace

extern "C" bspline_status bspline_eval_batched_noalloc(const bspline_batch_item *items, int nitems, int kind,
                                                       void *stream) {
    if (!items || nitems < 1 || kind < BSPLINE_V || kind > BSPLINE_VGH) return BSPLINE_ERR_ARG;
    if (nitems > BSPLINE_NOALLOC_MAX_ITEMS) return BSPLINE_ERR_ARG;  // beyond the fixed scratch
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The descriptors are copied from this call's stack frame: a graph that recorded the copy would read a
    // dead frame when replayed, so a capturing stream is refused before anything is enqueued.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce == cudaErrorStreamCaptureImplicit) {  // the legacy stream while another stream captures
        cudaGetLastError();
        return BSPLINE_ERR_UNSUPPORTED;
    }
    if (ce != cudaSuccess) return BSPLINE_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return BSPLINE_ERR_UNSUPPORTED;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSPLINE_ERR_CUDA;
    NoAllocDevice *D = nullptr;
    bspline_status st = noalloc_setup(dev, &D);
    if (st != BSPLINE_OK) return st;

    BatchItemDev desc[BSPLINE_NOALLOC_MAX_ITEMS];  // host staging on the stack
    int dtype = 0;
    long long units = 0;
    for (int k = 0; k < nitems; ++k) {
        st = noalloc_descriptor(items[k], kind, dev, &dtype, k == 0, units, &desc[k]);
        if (st != BSPLINE_OK) return st;
        units += (long long)desc[k].npos * desc[k].nblk;
    }
    if (units > 0x7fffffffLL) return BSPLINE_ERR_ARG;  // one CTA per unit
    const void *kern = kernel_for(dtype, kind);
    NoAllocScratch *scr = reinterpret_cast<NoAllocScratch *>(D->scratch);
    // Stream-ordered after any earlier call on the same stream; calls on other streams race.
    cudaError_t e = cudaMemcpyAsync(scr->items, desc, sizeof(BatchItemDev) * nitems, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (units == 0) return BSPLINE_OK;
    const BatchItemDev *ditems = scr->items;
    const int *no_perm = nullptr, *no_begin = nullptr;  // input order
    void *args[] = {(void *)&ditems, (void *)&nitems, (void *)&no_perm, (void *)&no_begin};
    return cuda_status(cudaLaunchKernel(kern, dim3((unsigned)units), dim3(kBatchNT), args, 0, s));
}
