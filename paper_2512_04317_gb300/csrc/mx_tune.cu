// Launch-geometry autotuner.  Register-resident radix-2 pass: the number of
// transform groups per CTA; tensor-core pass: the tile (4096 points on 256
// threads, or 2048 on 128) and the resident CTAs per SM of its persistent
// grid.  Each is measured per (transform length, other
// extent, axis, element format, block size, batch class) and the fastest kept
// in a process-wide table, which the launchers consult and which can be saved
// to / merged from a JSON file.  Every geometry computes the same bits: each
// transform (tensor-core pass: each tile) is processed independently in a
// fixed order.
#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "mx_plan.h"

using namespace mxfft;

namespace {

// batch class: ceil(log2(batch)), so that a table entry covers batches of
// similar grid size
int batch_class(int batch) {
    int c = 0;
    while ((1 << c) < batch && c < 30) c++;
    return c;
}

// n, other, dim, fmt, m (tensor-core pass: vectors per MX block), batch class,
// kind (0 radix-2 groups per CTA, 1 tensor-core CTAs per SM)
using Key = std::tuple<int, int, int, int, int, int, int>;
struct Val {
    int ng;        // groups per CTA, or CTAs per SM
    double us;
    int tile = 0;  // tensor-core pass: points per tile
};

std::mutex g_mu;
std::map<Key, Val>& table() {
    static std::map<Key, Val> t;
    return t;
}

// Deterministic pseudo-random complex values in [-1, 1) for the scratch batch.
__global__ void fill_kernel(float2* x, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u ^ (uint32_t)(i >> 32);
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        x[i] = make_float2((float)(h & 0xffff) / 32768.0f - 1.0f, (float)(h >> 16) / 32768.0f - 1.0f);
    }
}

// Average duration (microseconds) of `reps` launches of the pass with ng
// groups per CTA, after `warm` untimed ones; negative on a launch error.
double time_ng(mxfft_plan_s* p, const PassArgs& a, int batch, int ng, cudaStream_t s, int warm, int reps) {
    for (int i = 0; i < warm; i++)
        if (launch_fast_pass_ng(a, p->d_twh[a.dim][0], p->twa[a.dim][0], batch, ng, s) != cudaSuccess)
            return -1.0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1.0; }
    double us = -1.0;
    cudaEventRecord(e0, s);
    bool ok = true;
    for (int i = 0; i < reps && ok; i++)
        ok = launch_fast_pass_ng(a, p->d_twh[a.dim][0], p->twa[a.dim][0], batch, ng, s) == cudaSuccess;
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        us = 1000.0 * ms / reps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return us;
}

// The same for the tensor-core pass with its tile and ctas CTAs per SM.
double time_tc16(const Tc16Args& t, int fmt, int batch, int tile, int ctas, cudaStream_t s, int warm,
                 int reps) {
    for (int i = 0; i < warm; i++)
        if (launch_tc16_pass_geo(t, fmt, batch, tile, ctas, s) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1.0; }
    double us = -1.0;
    cudaEventRecord(e0, s);
    bool ok = true;
    for (int i = 0; i < reps && ok; i++) ok = launch_tc16_pass_geo(t, fmt, batch, tile, ctas, s) == cudaSuccess;
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        us = 1000.0 * ms / reps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return us;
}

// Integer value of "key": in a flat JSON object text (no nesting).
bool json_int(const std::string& obj, const char* key, long* v) {
    const std::string k = std::string("\"") + key + "\"";
    size_t at = obj.find(k);
    if (at == std::string::npos) return false;
    at = obj.find(':', at + k.size());
    if (at == std::string::npos) return false;
    const char* c = obj.c_str() + at + 1;
    char* end = nullptr;
    errno = 0;
    const long x = std::strtol(c, &end, 10);
    if (end == c || errno != 0) return false;
    *v = x;
    return true;
}

}  // namespace

namespace mxfft {

int fast_ng_tuned(int n, int other, int dim, int fmt, int m, int batch) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = table().find(Key(n, other, dim, fmt, m, batch_class(batch), 0));
    return it == table().end() ? 0 : it->second.ng;
}

void fast_ng_store(int n, int other, int dim, int fmt, int m, int batch, int ng, double us) {
    std::lock_guard<std::mutex> lk(g_mu);
    table()[Key(n, other, dim, fmt, m, batch_class(batch), 0)] = Val{ng, us};
}

void tc16_geo_tuned(int n, int other, int dim, int fmt, int g, int batch, int* tile, int* ctas) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = table().find(Key(n, other, dim, fmt, g, batch_class(batch), 1));
    *tile = it == table().end() ? 0 : it->second.tile;
    *ctas = it == table().end() ? 0 : it->second.ng;
}

void tc16_geo_store(int n, int other, int dim, int fmt, int g, int batch, int tile, int ctas,
                    double us) {
    std::lock_guard<std::mutex> lk(g_mu);
    table()[Key(n, other, dim, fmt, g, batch_class(batch), 1)] = Val{ctas, us, tile};
}

}  // namespace mxfft

extern "C" {

int mxfft_tune(mxfft_plan_t p, int batch, void* stream, int* n_measured) {
    if (n_measured) *n_measured = 0;
    if (!p || batch < 1) return MXFFT_ERR_INVALID;
    if (p->path == 0 && p->force_generic) return MXFFT_OK;   // nothing to choose
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return MXFFT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t npts = (size_t)batch * p->n0 * p->n1;
    float2 *x = nullptr, *y = nullptr;
    SliceStats* st = nullptr;
    int rc = cuda_status(cudaMalloc(&x, npts * sizeof(float2)));
    if (rc == MXFFT_OK) rc = cuda_status(cudaMalloc(&y, npts * sizeof(float2)));
    if (rc == MXFFT_OK) rc = cuda_status(cudaMalloc(&st, (size_t)batch * sizeof(SliceStats)));
    if (rc == MXFFT_OK) rc = cuda_status(cudaMemsetAsync(st, 0, (size_t)batch * sizeof(SliceStats), s));
    if (rc == MXFFT_OK) {
        fill_kernel<<<1024, 256, 0, s>>>(x, npts);
        rc = cuda_status(cudaGetLastError());
    }
    int measured = 0;
    for (int dim = 1; dim >= 0 && rc == MXFFT_OK; dim--) {
        // out of place, so that every launch sees the same input
        PassArgs a = pass_args(p, dim, 0, x, y);
        a.st = st;
        a.prologue = dim == 1 ? PRO_PRESCALE : PRO_NONE;
        a.epilogue = dim == 1 ? EPI_RAW : EPI_UNSCALE;
        const int other = dim == 1 ? p->n0 : p->n1;
        if (p->path == 1) {
            // 256 threads: 1 or 2 CTAs per SM; 128 threads (n <= 1024): 2 to 6
            const Tc16Args t = tc16_args(p, a, 0);
            const int cand[][2] = {{4096, 1}, {4096, 2}, {2048, 2}, {2048, 3}, {2048, 4}, {2048, 5},
                                   {2048, 6}};
            int best = -1;
            double best_us = 0.0;
            for (int i = 0; i < 7 && rc == MXFFT_OK; i++) {
                if (cand[i][0] == 2048 && a.n > 1024) continue;
                const double us = time_tc16(t, p->fmt, batch, cand[i][0], cand[i][1], s, 2, 5);
                if (us < 0) { rc = MXFFT_ERR_CUDA; break; }
                measured++;
                if (best < 0 || us < best_us) { best = i; best_us = us; }
            }
            if (rc == MXFFT_OK && best >= 0)
                tc16_geo_store(a.n, other, dim, p->fmt, t.g, batch, cand[best][0], cand[best][1], best_us);
            continue;
        }
        if (!fast_pass_supported(a)) continue;
        int cand[16];
        const int nc = fast_ng_candidates(a.n, other, a.m, cand, 16);
        if (nc < 2) continue;
        int best = 0;
        double best_us = 0.0;
        for (int i = 0; i < nc; i++) {
            const double us = time_ng(p, a, batch, cand[i], s, 2, 5);
            if (us < 0) { rc = MXFFT_ERR_CUDA; break; }
            measured++;
            if (best == 0 || us < best_us) { best = cand[i]; best_us = us; }
        }
        if (rc == MXFFT_OK) fast_ng_store(a.n, other, dim, p->fmt, a.m, batch, best, best_us);
    }
    if (rc == MXFFT_OK) rc = cuda_status(cudaStreamSynchronize(s));
    if (x) cudaFree(x);
    if (y) cudaFree(y);
    if (st) cudaFree(st);
    if (n_measured) *n_measured = measured;
    return rc;
}

int mxfft_tune_save(const char* path) {
    if (!path) return MXFFT_ERR_INVALID;
    std::string out = "{\"mxfft_tune\": 1, \"entries\": [";
    {
        std::lock_guard<std::mutex> lk(g_mu);
        bool first = true;
        for (const auto& kv : table()) {
            char buf[256];
            if (std::get<6>(kv.first) == 1)
                std::snprintf(buf, sizeof buf,
                              "%s\n  {\"kind\": 1, \"n\": %d, \"other\": %d, \"dim\": %d, \"fmt\": %d, "
                              "\"m\": %d, \"batch_class\": %d, \"tile\": %d, \"ctas_per_sm\": %d, "
                              "\"us\": %.3f}",
                              first ? "" : ",", std::get<0>(kv.first), std::get<1>(kv.first),
                              std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first),
                              std::get<5>(kv.first), kv.second.tile ? kv.second.tile : 4096, kv.second.ng,
                              kv.second.us);
            else
                std::snprintf(buf, sizeof buf,
                              "%s\n  {\"n\": %d, \"other\": %d, \"dim\": %d, \"fmt\": %d, \"m\": %d, "
                              "\"batch_class\": %d, \"ng\": %d, \"us\": %.3f}",
                              first ? "" : ",", std::get<0>(kv.first), std::get<1>(kv.first),
                              std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first),
                              std::get<5>(kv.first), kv.second.ng, kv.second.us);
            out += buf;
            first = false;
        }
    }
    out += "\n]}\n";
    FILE* f = std::fopen(path, "wb");
    if (!f) return MXFFT_ERR_INVALID;
    const bool ok = std::fwrite(out.data(), 1, out.size(), f) == out.size();
    return (std::fclose(f) == 0 && ok) ? MXFFT_OK : MXFFT_ERR_INVALID;
}

int mxfft_tune_load(const char* path) {
    if (!path) return MXFFT_ERR_INVALID;
    FILE* f = std::fopen(path, "rb");
    if (!f) return MXFFT_ERR_INVALID;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    if (text.find("\"mxfft_tune\"") == std::string::npos) return MXFFT_ERR_INVALID;
    size_t at = text.find("\"entries\"");
    if (at == std::string::npos) return MXFFT_ERR_INVALID;
    std::vector<std::pair<Key, Val>> parsed;
    while ((at = text.find('{', at)) != std::string::npos) {
        const size_t end = text.find('}', at);
        if (end == std::string::npos) return MXFFT_ERR_INVALID;
        const std::string obj = text.substr(at, end - at + 1);
        long n, other, dim, fmt, m, bc, ng, kind = 0, tile = 4096;
        if (json_int(obj, "kind", &kind) && kind != 0 && kind != 1) return MXFFT_ERR_INVALID;
        if (!json_int(obj, "n", &n) || !json_int(obj, "other", &other) || !json_int(obj, "dim", &dim) ||
            !json_int(obj, "fmt", &fmt) || !json_int(obj, "m", &m) ||
            !json_int(obj, "batch_class", &bc) || !json_int(obj, kind == 1 ? "ctas_per_sm" : "ng", &ng))
            return MXFFT_ERR_INVALID;
        bool valid = false;
        if (kind == 1) {
            json_int(obj, "tile", &tile);
            valid = ng >= 1 && ng <= kTc16MaxCtasPerSm && tc16_supported((int)n, (int)other, (int)fmt) &&
                    (m == 1 || m == 2 || m == 4) && (tile == 4096 || (tile == 2048 && n <= 1024));
        } else {
            int cand[16];
            const int nc = fast_ng_candidates((int)n, (int)other, (int)m, cand, 16);
            for (int i = 0; i < nc; i++) valid = valid || cand[i] == ng;
        }
        if (!valid || (dim != 0 && dim != 1) || bc < 0 || bc > 30) return MXFFT_ERR_INVALID;
        parsed.push_back({Key((int)n, (int)other, (int)dim, (int)fmt, (int)m, (int)bc, (int)kind),
                          Val{(int)ng, 0.0, kind == 1 ? (int)tile : 0}});
        at = end + 1;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& kv : parsed) table()[kv.first] = kv.second;
    return MXFFT_OK;
}

int mxfft_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    table().clear();
    return MXFFT_OK;
}

}  // extern "C"
