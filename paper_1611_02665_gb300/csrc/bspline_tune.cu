// Autotuner for the single-table launch shape.
//
// The paper picks its orbital tile N_b per machine by hand and plans an
// FFTW-"wisdom"-like automatic choice (Sec. "AoSoA transformation" and
// Sec. "Experiments and Results"). Here the tunable shape is the kernel
// variant, the orbitals per work unit, positions per CTA (DIRECT) or CTAs per
// SM and pipeline depth (TMA). Each candidate is timed with CUDA events on a
// scratch batch of random positions; the fastest is kept in the handle and
// optionally appended to a JSON-lines wisdom file.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "bspline_internal.cuh"

using namespace bsg;

namespace {

bool find_num(const std::string &line, const char *key, double *out) {
    std::string k = std::string("\"") + key + "\":";
    size_t p = line.find(k);
    if (p == std::string::npos) return false;
    const char *b = line.c_str() + p + k.size();
    char *e = nullptr;
    double v = strtod(b, &e);
    if (e == b) return false;
    *out = v;
    return true;
}

bool find_str(const std::string &line, const char *key, std::string *out) {
    std::string k = std::string("\"") + key + "\":\"";
    size_t p = line.find(k);
    if (p == std::string::npos) return false;
    size_t q = line.find('"', p + k.size());
    if (q == std::string::npos) return false;
    *out = line.substr(p + k.size(), q - p - k.size());
    return true;
}

struct Key {
    std::string gpu;
    int nx, ny, nz, N, dtype, kind, npos;
};

bool lookup_wisdom(const char *path, const Key &k, bspline_tuning *out) {
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char buf[1024];
    bool found = false;
    while (fgets(buf, sizeof buf, f)) {
        std::string line(buf);
        std::string gpu;
        double v[12];
        const char *keys[12] = {"nx",      "ny", "nz",  "N",      "dtype", "kind",
                                "npos",    "variant", "nb", "ppc", "stages", "order"};
        bool ok = find_str(line, "gpu", &gpu);
        for (int i = 0; i < 12 && ok; ++i) ok = find_num(line, keys[i], &v[i]);
        if (!ok || gpu != k.gpu) continue;
        if ((int)v[0] != k.nx || (int)v[1] != k.ny || (int)v[2] != k.nz || (int)v[3] != k.N ||
            (int)v[4] != k.dtype || (int)v[5] != k.kind || (int)v[6] != k.npos)
            continue;
        *out = bspline_tuning{(int)v[7], (int)v[8], (int)v[9], (int)v[10], (int)v[11]};
        found = true;  // the last matching record wins
    }
    fclose(f);
    return found;
}

void append_wisdom(const char *path, const Key &k, const bspline_tuning &tu, double us) {
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f,
            "{\"gpu\":\"%s\",\"nx\":%d,\"ny\":%d,\"nz\":%d,\"N\":%d,\"dtype\":%d,\"kind\":%d,\"npos\":%d,"
            "\"variant\":%d,\"nb\":%d,\"ppc\":%d,\"stages\":%d,\"order\":%d,\"us\":%.3f}\n",
            k.gpu.c_str(), k.nx, k.ny, k.nz, k.N, k.dtype, k.kind, k.npos, tu.variant, tu.nb, tu.ppc, tu.stages,
            tu.order, us);
    fclose(f);
}

std::vector<bspline_tuning> candidates(int dtype, int Npad) {
    std::vector<bspline_tuning> c;
    for (int order : {0, 1}) {
        for (int nb : {256, 512, 1024})
            for (int ppc : {1, 2, 4}) c.push_back({BSPLINE_VARIANT_DIRECT, nb, ppc, 0, order});
        if (dtype == BSPLINE_F32)
            for (int ring : {4, 6}) c.push_back({BSPLINE_VARIANT_DIRECT, 512, 1, ring, order});
        for (int nb : {128, 256})
            for (int stages : {2, 3, 4, 6})
                for (int cps : {1, 2}) {
                    if (tma_smem_bytes(dtype, nb, stages) * cps > 228u * 1024u) continue;
                    if (tma_smem_bytes(dtype, nb, stages) > 227u * 1024u) continue;
                    c.push_back({BSPLINE_VARIANT_TMA, nb, cps, stages, order});
                }
        if (dtype != BSPLINE_F32)
            for (int nb : {128, 256})
                for (int stages : {2, 3, 4, 5, 6, 8})
                    for (int cps : {1, 2})
                        if ((nb == 256 || stages >= 4) && mma_fits(dtype, stages, Npad, cps, nb))
                            c.push_back({BSPLINE_VARIANT_MMA, nb, cps, stages, order});
    }
    return c;
}

}  // namespace

extern "C" bspline_status bspline_tune(bspline_t t, int kind, int npos_hint, const char *wisdom_path,
                                       bspline_tuning *chosen) {
    if (!t || kind < BSPLINE_V || kind > BSPLINE_VGH || npos_hint < 0) return BSPLINE_ERR_ARG;
    if (!t->has_coefs) return BSPLINE_ERR_STATE;
    const int npos = npos_hint > 0 ? npos_hint : 4096;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, t->device);
    if (e != cudaSuccess) return cuda_status(e);
    Key key{prop.name, t->nx, t->ny, t->nz, t->N, t->dtype, kind, npos};
    bspline_tuning best{0, 0, 0, 0, 0};
    if (wisdom_path && lookup_wisdom(wisdom_path, key, &best)) {
        bspline_status st = bspline_set_tuning(t, kind, &best);
        if (st == BSPLINE_OK) {
            if (chosen) bspline_get_tuning(t, kind, chosen);
            return BSPLINE_OK;
        }
    }

    // Scratch: random positions (64-bit LCG, fixed seed) and outputs with ld = N.
    std::vector<double> hpos((size_t)3 * npos);
    unsigned long long st64 = 0x9E3779B97F4A7C15ull;
    for (auto &v : hpos) {
        st64 = st64 * 6364136223846793005ull + 1442695040888963407ull;
        v = (double)(st64 >> 11) * (1.0 / 9007199254740992.0);
    }
    const int ncomp = nout_of(kind);
    double *dpos = nullptr;
    float *dout = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    e = cudaMalloc(&dpos, sizeof(double) * hpos.size());
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(float) * (size_t)npos * ncomp * t->N);
    if (e == cudaSuccess) e = cudaMemcpy(dpos, hpos.data(), sizeof(double) * hpos.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    bspline_status st = cuda_status(e);
    double best_us = 1e30;
    if (st == BSPLINE_OK) {
        const double *x = dpos, *y = dpos + npos, *z = dpos + 2 * (size_t)npos;
        float *o0 = dout, *o1 = dout + (size_t)npos * t->N, *o2 = o1 + (size_t)npos * 3 * t->N;
        for (const bspline_tuning &c : candidates(t->dtype, t->Npad)) {
            bspline_status ls = launch_eval(t, kind, c, npos, x, y, z, o0, kind == BSPLINE_V ? nullptr : o1,
                                            kind == BSPLINE_V ? nullptr : o2, t->N, s);
            if (ls != BSPLINE_OK) continue;
            std::vector<float> ms;
            for (int r = 0; r < 5; ++r) {
                cudaEventRecord(ev0, s);
                launch_eval(t, kind, c, npos, x, y, z, o0, kind == BSPLINE_V ? nullptr : o1,
                            kind == BSPLINE_V ? nullptr : o2, t->N, s);
                cudaEventRecord(ev1, s);
                if (cudaEventSynchronize(ev1) != cudaSuccess) break;
                float m = 0.f;
                cudaEventElapsedTime(&m, ev0, ev1);
                ms.push_back(m);
            }
            if (ms.size() != 5) {
                st = BSPLINE_ERR_CUDA;
                break;
            }
            std::sort(ms.begin(), ms.end());
            const double us = ms[2] * 1000.0;
            if (us < best_us) {
                best_us = us;
                best = c;
            }
        }
        e = cudaStreamSynchronize(s);
        if (st == BSPLINE_OK && e != cudaSuccess) st = cuda_status(e);
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (s) cudaStreamDestroy(s);
    cudaFree(dpos);
    cudaFree(dout);
    if (st != BSPLINE_OK) return st;
    if (best.variant == 0) return BSPLINE_ERR_CUDA;
    st = bspline_set_tuning(t, kind, &best);
    if (st != BSPLINE_OK) return st;
    if (wisdom_path) append_wisdom(wisdom_path, key, best, best_us);
    if (chosen) bspline_get_tuning(t, kind, chosen);
    return BSPLINE_OK;
}
