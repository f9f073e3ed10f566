// Ragged batch executor: many independent 2D transforms of the method (Alg. 1
// prescale, then the Alg. 2 radix-2 passes along rows and columns, Eq. (1)
// round trips) enqueued as
//   table upload -> statistics records cleared -> one statistics launch over
//   every slice of every item -> one ragged rows launch and one ragged
//   columns launch over every (plan, direction) group whose passes fit the
//   ragged register-resident kernel (k = 32, n <= 1024) -> [round trips: one
//   statistics launch over the forward outputs -> one ragged inverse rows and
//   one inverse columns launch]
// so any mix of such plans runs in at most 6 launches.  Groups of other plans
// (tensor-core paths, other k, the generic pass) keep one launch per pass and
// group, as parallel branches on fork streams beside the ragged launches.
// Every pass kernel reads its slices' buffers and statistics records from a
// table in device memory (SliceRef), so a group is one launch whatever the
// addresses, and a captured graph stays valid when a later call passes other
// buffers: only the table content changes.  Per slice the arithmetic is that
// of mxfft_forward / mxfft_inverse / mxfft_roundtrip / mxfft_roundtrip_fused,
// so results are bit-identical to them.
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mx_plan.h"

using namespace mxfft;

namespace {

constexpr int kForkStreams = 8;
constexpr size_t kMaxGraphs = 64;

using PlanKey = std::tuple<int, int, int, int>;   // n0, n1, format, k

struct PassLaunch {
    mxfft_plan_s* p;
    int dim, dir, prologue, epilogue;
    int ref0, count;      // slice references [ref0, ref0 + count)
    int branch;           // fork branch within its stage
    int fused = 0;        // 1: forward + inverse columns of the fused round trip
    int whole = 0;        // 1: the fused 2D kernel (statistics, rows, columns)
    int stats_out = 0;    // 1: the pass accumulates its output's statistics into
                          // the references' st_out records (round trips, tensor-core path)
};

// One ragged launch: the register-resident passes of several plans along
// one axis (k = 32), every CTA 256 threads, its work from a table of
// (group, slice, first transform) entries; the groups' arguments travel as a
// kernel parameter.
struct RaggedPhase {
    int dim = 1;
    std::vector<char> groups;         // ngroups records of fast_ragged_arg_size() bytes
    int ngroups = 0;
    int cta0 = 0, ncta = 0;           // entries [cta0, cta0 + ncta) of Layout::rctas
    size_t smem = 0;                  // largest dynamic shared memory of its groups
};

// Host image of one run: the device tables and the launches that read them.
struct Layout {
    std::vector<SliceRef> refs;
    std::vector<StatsRef> srefs;
    std::vector<int2> ctas;
    std::vector<PassLaunch> stage1, stage2;
    std::vector<RssRef> rrefs;        // RSS outputs, in item order
    // ragged launches: stage-1 rows, stage-1 columns, stage-2 rows, stage-2 columns
    RaggedPhase rag[4];
    std::vector<int4> rctas;
    int nbranch1 = 0, nbranch2 = 0;
    int cta1 = 0, ncta1 = 0, cta2 = 0, ncta2 = 0;
    int nslices = 0;
    std::vector<char> rt;             // per slice: round trip
    size_t off_srefs = 0, off_ctas = 0, off_rss = 0, off_rctas = 0, bytes = 0;
    std::string signature;
};

// Buffers of one run shape: pinned staging and device copy of the tables, the
// statistics records (forward then inverse, nslices each), and the event of
// the last run that used them.
struct RunBuffers {
    void* h_blob = nullptr;
    void* d_blob = nullptr;
    size_t cap = 0;
    SliceStats* d_st = nullptr;
    int st_cap = 0;
    cudaEvent_t done = nullptr;
    bool pending = false;             // a run may still read h_blob
    std::vector<char> last;           // table bytes of the last upload
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    RunBuffers buf;
    int launches = 0;     // kernels in the captured graph
};

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

void free_buffers(RunBuffers& b) {
    if (b.h_blob) cudaFreeHost(b.h_blob);
    if (b.d_blob) cudaFree(b.d_blob);
    if (b.d_st) cudaFree(b.d_st);
    if (b.done) cudaEventDestroy(b.done);
    b = RunBuffers();
}

// Capacity for a layout; waits for the buffers' last run before reallocating.
int reserve(RunBuffers& b, const Layout& L) {
    if (!b.done) {
        int rc = cuda_status(cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming));
        if (rc) return rc;
    }
    if (L.bytes <= b.cap && L.nslices <= b.st_cap) return MXFFT_OK;
    if (b.pending) {
        int rc = cuda_status(cudaEventSynchronize(b.done));
        if (rc) return rc;
        b.pending = false;
    }
    if (L.bytes > b.cap) {
        if (b.h_blob) cudaFreeHost(b.h_blob);
        if (b.d_blob) cudaFree(b.d_blob);
        b.h_blob = b.d_blob = nullptr;
        b.cap = 0;
        size_t cap = 4096;
        while (cap < L.bytes) cap *= 2;
        int rc = cuda_status(cudaMallocHost(&b.h_blob, cap));
        if (rc == MXFFT_OK) rc = cuda_status(cudaMalloc(&b.d_blob, cap));
        if (rc) return rc;
        b.cap = cap;
        b.last.clear();
    }
    if (L.nslices > b.st_cap) {
        if (b.d_st) cudaFree(b.d_st);
        b.d_st = nullptr;
        b.st_cap = 0;
        int cap = 16;
        while (cap < L.nslices) cap *= 2;
        int rc = cuda_status(cudaMalloc(&b.d_st, 2 * (size_t)cap * sizeof(SliceStats)));
        if (rc) return rc;
        b.st_cap = cap;
        b.last.clear();
    }
    return MXFFT_OK;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const char* ca = (const char*)a;
    const char* cb = (const char*)b;
    return ca < cb + nb && cb < ca + na;
}

bool item_ok(const mxfft_item& it) {
    if (it.slices < 0 || it.op < 0 || it.op > 3 || it.reserved != 0) return false;
    if (it.slices == 0) return true;
    if (!it.in || !it.out || ((uintptr_t)it.in & 15u) || ((uintptr_t)it.out & 15u)) return false;
    const size_t bytes = (size_t)it.slices * it.n0 * it.n1 * sizeof(float2);
    if (it.in != it.out && overlap(it.in, bytes, it.out, bytes)) return false;
    if (it.rss) {
        if (it.coils < 1 || it.slices % it.coils || ((uintptr_t)it.rss & 15u)) return false;
        const size_t rb = (size_t)(it.slices / it.coils) * it.n0 * it.n1 * sizeof(float);
        if (overlap(it.rss, rb, it.in, bytes) || overlap(it.rss, rb, it.out, bytes)) return false;
    }
    return true;
}

}  // namespace

struct mxfft_engine_s {
    int device = -1;
    float tau = 0.f, target = 0.f;
    int flags = 0;
    std::map<PlanKey, mxfft_plan_t> plans;
    cudaStream_t capture = nullptr;             // stream the graphs are captured on
    cudaStream_t fork[kForkStreams] = {};
    std::vector<cudaEvent_t> evs;               // fork / join events
    RunBuffers direct;
    std::unordered_map<std::string, GraphEntry*> graphs;
    // last run, for mxfft_engine_get_status
    RunBuffers* last_buf = nullptr;
    int last_slices = 0;
    std::vector<char> last_rt;
    std::vector<mxfft_plan_s*> last_plans;
    int last_launches = 0;                      // kernels the last run enqueued
};

namespace {

int get_plan(mxfft_engine_s* e, const mxfft_item& it, mxfft_plan_s** out) {
    const PlanKey key(it.n0, it.n1, it.format, it.k);
    auto f = e->plans.find(key);
    if (f != e->plans.end()) { *out = f->second; return MXFFT_OK; }
    mxfft_plan_t p = nullptr;
    int rc = mxfft_plan(it.n0, it.n1, it.format, it.k, e->tau, e->target, &p);
    if (rc) return rc;
    if (e->flags & MXFFT_ENGINE_TC16) {
        // plans the tensor-core pass does not cover keep the radix-2 pass
        rc = mxfft_set_option(p, MXFFT_OPT_PATH, 1.0);
        if (rc != MXFFT_OK && rc != MXFFT_ERR_UNSUPPORTED) { mxfft_destroy(p); return rc; }
        if (rc == MXFFT_OK && (e->flags & MXFFT_ENGINE_FUSED2D))
            rc = mxfft_set_option(p, MXFFT_OPT_FUSED2D, 1.0);
        if (rc == MXFFT_OK && (e->flags & MXFFT_ENGINE_FOLD_STATS))
            rc = mxfft_set_option(p, MXFFT_OPT_FOLD_STATS, 1.0);
        if (rc != MXFFT_OK && rc != MXFFT_ERR_UNSUPPORTED) { mxfft_destroy(p); return rc; }
    }
    e->plans[key] = p;
    *out = p;
    return MXFFT_OK;
}

// Slices in item order get records st_f = d_st + g, st_i = d_st + cap + g.
int build_layout(mxfft_engine_s* e, const mxfft_item* items, int n, Layout& L,
                 std::vector<mxfft_plan_s*>& item_plan) {
    item_plan.assign(n, nullptr);
    std::string sig;
    for (int i = 0; i < n; i++) {
        if (items[i].slices == 0) continue;
        if (items[i].op == MXFFT_OP_ROUNDTRIP_FUSED && items[i].format == MXFFT_FP16)
            return MXFFT_ERR_UNSUPPORTED;
        int rc = get_plan(e, items[i], &item_plan[i]);
        if (rc) return rc;
        char b[128];
        std::snprintf(b, sizeof b, "%d,%d,%d,%d,%d,%d,%d;", items[i].n0, items[i].n1, items[i].format,
                      items[i].k, items[i].op, items[i].slices, items[i].rss ? items[i].coils : 0);
        sig += b;
        L.nslices += items[i].slices;
    }
    L.signature = sig;
    // table sizes: per slice two pass references (rows, columns) and a
    // statistics reference with its CTAs; round trips add one reference for
    // the inverse passes and a second statistics reference
    size_t refs = 0, srefs = 0, ctas = 0, rss = 0;
    for (int i = 0; i < n; i++) {
        const size_t sl = (size_t)items[i].slices;
        const size_t c = ((size_t)items[i].n0 * items[i].n1 + kStatsPtsPerCta - 1) / kStatsPtsPerCta;
        const size_t rt = items[i].op == MXFFT_OP_ROUNDTRIP ? 1 : 0;
        refs += sl * (2 + rt);
        srefs += sl * (1 + rt);
        ctas += sl * c * (1 + rt);
        rss += (sl > 0 && items[i].rss) ? 1 : 0;
    }
    // ragged CTA entries: at most (n0 + n1) / 8 per slice and stage (a CTA
    // holds at least 8 transforms), two stages
    size_t rctas = 0;
    for (int i = 0; i < n; i++) rctas += (size_t)items[i].slices * (items[i].n0 + items[i].n1) / 4;
    L.off_srefs = align16(refs * sizeof(SliceRef));
    L.off_ctas = align16(L.off_srefs + srefs * sizeof(StatsRef));
    L.off_rss = align16(L.off_ctas + ctas * sizeof(int2));
    L.off_rctas = align16(L.off_rss + rss * sizeof(RssRef));
    L.bytes = align16(L.off_rctas + rctas * sizeof(int4));
    return MXFFT_OK;
}

// Fill the tables for records at st_base (forward) and st_base + st_cap
// (inverse statistics of round trips).
// (d_blob: the device copy of the tables, whose slice references the ragged
// launches' arguments point into; ragged: use the ragged launches.)
void fill_layout(const mxfft_item* items, int n, const std::vector<mxfft_plan_s*>& item_plan,
                 SliceStats* st_base, int st_cap, const void* d_blob, bool ragged, Layout& L) {
    L.refs.clear();
    L.srefs.clear();
    L.ctas.clear();
    L.stage1.clear();
    L.stage2.clear();
    L.rt.assign(L.nslices, 0);
    // ragged launches of the register-resident pass (k = 32): a plan's group
    // joins them when both of its axes fit the ragged geometry
    for (int ph = 0; ph < 4; ph++) {
        L.rag[ph] = RaggedPhase();
        L.rag[ph].dim = (ph & 1) ? 0 : 1;
    }
    L.rctas.clear();
    std::vector<int4> rc[4];
    const SliceRef* d_refs = static_cast<const SliceRef*>(d_blob);
    const int max_groups = fast_ragged_max_groups();
    auto fits = [&](mxfft_plan_s* p) {
        return ragged && p->path == 0 && !p->force_generic &&
               fast_ragged_supported(pass_args(p, 1, 0, nullptr, nullptr)) &&
               fast_ragged_supported(pass_args(p, 0, 0, nullptr, nullptr));
    };
    // a stage uses the ragged launches when at least two groups fit them (a
    // single group keeps its tuned per-plan launches, as few in number)
    bool use = false;
    auto ragged_ok = [&](mxfft_plan_s* p, int ph_a, int ph_b, int ph_c) {
        if (!use || !fits(p)) return false;
        for (int ph : {ph_a, ph_b, ph_c})
            if (ph >= 0 && L.rag[ph].ngroups >= max_groups) return false;
        return true;
    };
    auto add_ragged = [&](int ph, mxfft_plan_s* p, int dim, int dir, int pro, int epi, int ref0,
                          int count, bool fused) {
        PassArgs a = pass_args(p, dim, dir, nullptr, nullptr);
        a.ref = d_refs + ref0;
        a.prologue = pro;
        a.epilogue = epi;
        RaggedPhase& R = L.rag[ph];
        const size_t sz = fast_ragged_arg_size();
        R.groups.resize((size_t)(R.ngroups + 1) * sz);
        int tpc = 0;
        size_t smem = 0;
        fast_ragged_fill(R.groups.data() + (size_t)R.ngroups * sz, a, p->d_twh[dim][dir], p->twa[dim][dir],
                         fused ? p->d_twh[0][1] : nullptr, fused ? &p->twa[0][1] : nullptr, &tpc, &smem);
        const int other = dim == 1 ? p->n0 : p->n1;
        for (int sl = 0; sl < count; sl++)
            for (int t0 = 0; t0 < other; t0 += tpc) rc[ph].push_back(make_int4(R.ngroups, sl, t0, 0));
        R.smem = std::max(R.smem, smem);
        R.ngroups++;
    };
    int branch = 0;   // fork branches of the per-plan launches
    std::vector<int> first(n, 0);
    for (int i = 0, g = 0; i < n; i++) { first[i] = g; g += items[i].slices; }
    auto add_stats = [&](const float2* x, SliceStats* st, int npts, const KParams& kp) {
        const int ctas = (npts + kStatsPtsPerCta - 1) / kStatsPtsPerCta;
        const int idx = (int)L.srefs.size();
        L.srefs.push_back(StatsRef{x, st, npts, (uint32_t)ctas, kp});
        for (int c = 0; c < ctas; c++) L.ctas.push_back(make_int2(idx, c));
    };
    // slices of plans that run the fused 2D kernel take their statistics on
    // chip (forward, inverse and both halves of round trips)
    auto whole2d = [&](int i) {
        return item_plan[i] && uses_tc2d(item_plan[i]) && items[i].op != MXFFT_OP_ROUNDTRIP_FUSED;
    };
    // round trips whose forward columns pass (tensor-core path) takes the
    // inverse's statistics of its output: no statistics launch for them
    auto folded = [&](int i) {
        return items[i].op == MXFFT_OP_ROUNDTRIP && item_plan[i] && tc16_folds_stats(item_plan[i]) &&
               !uses_tc2d(item_plan[i]);
    };
    // statistics of every other input
    L.cta1 = 0;
    for (int i = 0; i < n; i++) {
        const mxfft_item& it = items[i];
        const int np = it.n0 * it.n1;
        if (whole2d(i)) continue;
        for (int s = 0; s < it.slices; s++)
            add_stats((const float2*)it.in + (size_t)s * np, st_base + first[i] + s, np,
                      kparams(item_plan[i]));
    }
    L.ncta1 = (int)L.ctas.size();
    // stage 1 groups: (plan, kind) in order of first appearance; kind 0 forward
    // (also the first half of a round trip), 1 inverse, 2 fused round trip
    auto kind_of = [](int op) {
        return op == MXFFT_OP_INVERSE ? 1 : (op == MXFFT_OP_ROUNDTRIP_FUSED ? 2 : 0);
    };
    std::vector<std::pair<mxfft_plan_s*, int>> groups;
    for (int i = 0; i < n; i++) {
        if (items[i].slices == 0) continue;
        const std::pair<mxfft_plan_s*, int> key(item_plan[i], kind_of(items[i].op));
        if (std::find(groups.begin(), groups.end(), key) == groups.end()) groups.push_back(key);
    }
    {
        int fit = 0;
        for (const auto& g : groups)
            fit += fits(g.first) && (g.second == 2 || !uses_tc2d(g.first));
        use = fit >= 2;
    }
    for (size_t gi = 0; gi < groups.size(); gi++) {
        mxfft_plan_s* p = groups[gi].first;
        const int kind = groups[gi].second;
        const int dir = kind == 1 ? 1 : 0;
        const int np = p->n0 * p->n1;
        const int rows0 = (int)L.refs.size();
        std::vector<SliceStats*> st_out;   // per slice: inverse statistics folded into the columns pass
        for (int i = 0; i < n; i++) {
            if (item_plan[i] != p || kind_of(items[i].op) != kind) continue;
            for (int s = 0; s < items[i].slices; s++) {
                L.refs.push_back(SliceRef{(const float2*)items[i].in + (size_t)s * np,
                                          (float2*)items[i].out + (size_t)s * np,
                                          st_base + first[i] + s, nullptr});
                st_out.push_back(folded(i) ? st_base + st_cap + first[i] + s : nullptr);
            }
        }
        const int count = (int)L.refs.size() - rows0;
        const bool any_out = std::any_of(st_out.begin(), st_out.end(), [](SliceStats* q) { return q; });
        if (kind != 2 && uses_tc2d(p)) {
            // one launch: statistics, rows and columns of every slice of the group
            PassLaunch w{p, 2, dir, PRO_PRESCALE, EPI_UNSCALE, rows0, count, branch++};
            w.whole = 1;
            L.stage1.push_back(w);
            continue;
        }
        const int cols0 = (int)L.refs.size();
        for (int r = 0; r < count; r++) {
            SliceRef c = L.refs[rows0 + r];
            c.in = c.out;
            c.st_out = st_out[r];
            L.refs.push_back(c);
        }
        if (ragged_ok(p, 0, 1, kind == 2 ? 2 : -1)) {
            // rows and columns in the ragged launches; the fused round trip's
            // inverse rows join the stage-2 rows launch (they need only its columns)
            add_ragged(0, p, 1, dir, PRO_PRESCALE, EPI_RAW, rows0, count, false);
            add_ragged(1, p, 0, dir, PRO_NONE, kind == 2 ? EPI_RAW : EPI_UNSCALE, cols0, count, kind == 2);
            if (kind == 2) add_ragged(2, p, 1, 1, PRO_NONE, EPI_RT_FINAL, cols0, count, false);
            continue;
        }
        const int br = branch++;
        L.stage1.push_back(PassLaunch{p, 1, dir, PRO_PRESCALE, EPI_RAW, rows0, count, br});
        if (kind == 2) {
            // fused round trip: columns forward + inverse, then the inverse rows
            // with the one decode (2^(-k - log2(n0 n1)), k of the input)
            L.stage1.push_back(PassLaunch{p, 0, 0, PRO_NONE, EPI_RAW, cols0, count, br, 1});
            L.stage1.push_back(PassLaunch{p, 1, 1, PRO_NONE, EPI_RT_FINAL, cols0, count, br});
        } else {
            PassLaunch c{p, 0, dir, PRO_NONE, EPI_UNSCALE, cols0, count, br};
            c.stats_out = any_out ? 1 : 0;
            L.stage1.push_back(c);
        }
    }
    L.nbranch1 = branch;
    // round trips: statistics of the forward outputs, then the inverse passes
    L.cta2 = (int)L.ctas.size();
    std::vector<mxfft_plan_s*> rt_plans;
    for (int i = 0; i < n; i++) {
        if (items[i].op != MXFFT_OP_ROUNDTRIP || items[i].slices == 0) continue;
        const int np = items[i].n0 * items[i].n1;
        for (int s = 0; s < items[i].slices; s++) {
            if (!whole2d(i) && !folded(i))
                add_stats((const float2*)items[i].out + (size_t)s * np, st_base + st_cap + first[i] + s,
                          np, kparams(item_plan[i]));
            L.rt[first[i] + s] = 1;
        }
        if (std::find(rt_plans.begin(), rt_plans.end(), item_plan[i]) == rt_plans.end())
            rt_plans.push_back(item_plan[i]);
    }
    L.ncta2 = (int)L.ctas.size() - L.cta2;
    branch = 0;
    {
        int fit = L.rag[2].ngroups;   // fused round trips' inverse rows, already ragged
        for (mxfft_plan_s* p : rt_plans) fit += fits(p) && !uses_tc2d(p);
        use = fit >= 2;
    }
    for (size_t gi = 0; gi < rt_plans.size(); gi++) {
        mxfft_plan_s* p = rt_plans[gi];
        const int np = p->n0 * p->n1;
        const int r0 = (int)L.refs.size();
        for (int i = 0; i < n; i++) {
            if (item_plan[i] != p || items[i].op != MXFFT_OP_ROUNDTRIP) continue;
            for (int s = 0; s < items[i].slices; s++) {
                float2* y = (float2*)items[i].out + (size_t)s * np;
                L.refs.push_back(SliceRef{y, y, st_base + st_cap + first[i] + s, nullptr});
            }
        }
        const int count = (int)L.refs.size() - r0;
        if (uses_tc2d(p)) {
            PassLaunch w{p, 2, 1, PRO_PRESCALE, EPI_RT_FINAL, r0, count, branch++};
            w.whole = 1;
            L.stage2.push_back(w);
            continue;
        }
        if (ragged_ok(p, 2, 3, -1)) {
            add_ragged(2, p, 1, 1, PRO_PRESCALE, EPI_RAW, r0, count, false);
            add_ragged(3, p, 0, 1, PRO_NONE, EPI_RT_FINAL, r0, count, false);
            continue;
        }
        const int br = branch++;
        L.stage2.push_back(PassLaunch{p, 1, 1, PRO_PRESCALE, EPI_RAW, r0, count, br});
        L.stage2.push_back(PassLaunch{p, 0, 1, PRO_NONE, EPI_RT_FINAL, r0, count, br});
    }
    L.nbranch2 = branch;
    for (int ph = 0; ph < 4; ph++) {
        L.rag[ph].cta0 = (int)L.rctas.size();
        L.rag[ph].ncta = (int)rc[ph].size();
        L.rctas.insert(L.rctas.end(), rc[ph].begin(), rc[ph].end());
    }
    // root-sum-of-squares outputs of the items that ask for them
    L.rrefs.clear();
    for (int i = 0; i < n; i++)
        if (items[i].slices > 0 && items[i].rss)
            L.rrefs.push_back(RssRef{(const float2*)items[i].out, (float*)items[i].rss, items[i].coils,
                                     items[i].slices / items[i].coils,
                                     (long long)items[i].n0 * items[i].n1});
    L.off_srefs = align16(L.refs.size() * sizeof(SliceRef));
    L.off_ctas = align16(L.off_srefs + L.srefs.size() * sizeof(StatsRef));
    L.off_rss = align16(L.off_ctas + L.ctas.size() * sizeof(int2));
    L.off_rctas = align16(L.off_rss + L.rrefs.size() * sizeof(RssRef));
    L.bytes = align16(L.off_rctas + L.rctas.size() * sizeof(int4));
}

void pack(const Layout& L, char* dst) {
    std::memset(dst, 0, L.bytes);
    std::memcpy(dst, L.refs.data(), L.refs.size() * sizeof(SliceRef));
    std::memcpy(dst + L.off_srefs, L.srefs.data(), L.srefs.size() * sizeof(StatsRef));
    std::memcpy(dst + L.off_ctas, L.ctas.data(), L.ctas.size() * sizeof(int2));
    std::memcpy(dst + L.off_rss, L.rrefs.data(), L.rrefs.size() * sizeof(RssRef));
    std::memcpy(dst + L.off_rctas, L.rctas.data(), L.rctas.size() * sizeof(int4));
}

// One stage: main(s) enqueues the ragged launches on the run's own stream
// while the per-plan launches run as parallel branches on the fork streams.
template <class Main>
cudaError_t run_stage(mxfft_engine_s* e, const std::vector<PassLaunch>& stage, int nbranch,
                      const SliceRef* d_refs, cudaStream_t s, size_t& ev, Main main) {
    const int nf = std::min(nbranch, kForkStreams);
    cudaError_t err = cudaSuccess;
    if (nf > 1) {
        // fork: every branch stream waits for the work so far on s
        err = cudaEventRecord(e->evs[ev], s);
        for (int f = 0; f < nf && err == cudaSuccess; f++) err = cudaStreamWaitEvent(e->fork[f], e->evs[ev], 0);
        ev++;
    }
    if (err == cudaSuccess) err = main(s);
    for (const PassLaunch& pl : stage) {
        if (err != cudaSuccess) break;
        if (pl.whole) {
            Tc2dArgs t = tc2d_args(pl.p, pl.dir, nullptr, nullptr, nullptr, pl.epilogue);
            t.ref = d_refs + pl.ref0;
            err = timed_tc2d(pl.p, t, pl.count, nf > 1 ? e->fork[pl.branch % nf] : s);
            continue;
        }
        PassArgs a = pass_args(pl.p, pl.dim, pl.dir, nullptr, nullptr);
        a.ref = d_refs + pl.ref0;
        a.prologue = pl.prologue;
        a.epilogue = pl.epilogue;
        a.stats_out = pl.stats_out;
        cudaStream_t bs = nf > 1 ? e->fork[pl.branch % nf] : s;
        err = pl.fused ? fused_cols_pass(pl.p, a, pl.count, bs) : timed_pass(pl.p, a, pl.count, bs);
    }
    if (nf > 1) {
        // join
        for (int f = 0; f < nf && err == cudaSuccess; f++) {
            err = cudaEventRecord(e->evs[ev], e->fork[f]);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(s, e->evs[ev], 0);
            ev++;
        }
    }
    return err;
}

// Everything of one run after its tables are in device memory.
cudaError_t enqueue(mxfft_engine_s* e, const Layout& L, RunBuffers& b, cudaStream_t s) {
    char* d = (char*)b.d_blob;
    const SliceRef* d_refs = (const SliceRef*)d;
    const StatsRef* d_srefs = (const StatsRef*)(d + L.off_srefs);
    const int2* d_ctas = (const int2*)(d + L.off_ctas);
    size_t ev = 0;
    cudaError_t err = cudaMemsetAsync(b.d_st, 0, 2 * (size_t)b.st_cap * sizeof(SliceStats), s);
    // the plans' timeout flags report this run only
    std::vector<mxfft_plan_s*> seen;
    for (const std::vector<PassLaunch>* st : {&L.stage1, &L.stage2})
        for (const PassLaunch& pl : *st)
            if (err == cudaSuccess && pl.p->d_err && std::find(seen.begin(), seen.end(), pl.p) == seen.end()) {
                seen.push_back(pl.p);
                err = cudaMemsetAsync(pl.p->d_err, 0, sizeof(int), s);
            }
    const int4* d_rctas = (const int4*)(d + L.off_rctas);
    auto ragged = [&](int ph_a, int ph_b) {
        return [&, ph_a, ph_b](cudaStream_t ms) {
            cudaError_t r = cudaSuccess;
            for (int ph : {ph_a, ph_b}) {
                const RaggedPhase& R = L.rag[ph];
                if (r == cudaSuccess && R.ngroups > 0)
                    r = launch_fast_ragged(R.groups.data(), R.ngroups, d_rctas + R.cta0, R.ncta, R.dim,
                                           R.smem, ms);
            }
            return r;
        };
    };
    if (err == cudaSuccess) err = launch_stats_ref(d_srefs, d_ctas + L.cta1, L.ncta1, s);
    if (err == cudaSuccess) err = run_stage(e, L.stage1, L.nbranch1, d_refs, s, ev, ragged(0, 1));
    if (err == cudaSuccess && L.ncta2 > 0) err = launch_stats_ref(d_srefs, d_ctas + L.cta2, L.ncta2, s);
    if (err == cudaSuccess) err = run_stage(e, L.stage2, L.nbranch2, d_refs, s, ev, ragged(2, 3));
    const RssRef* d_rss = (const RssRef*)(d + L.off_rss);
    for (size_t j = 0; j < L.rrefs.size() && err == cudaSuccess; j++)
        err = launch_rss(L.rrefs[j], d_rss + j, L.rrefs[j].images, L.rrefs[j].npts, s);
    return err;
}

// Make the staging buffer hold the layout's tables; returns whether they
// changed.  Waits for the buffer's last run before rewriting it.
int stage_tables(RunBuffers& b, const Layout& L, bool* changed) {
    std::vector<char> img(L.bytes);
    pack(L, img.data());
    *changed = img != b.last;
    if (!*changed) return MXFFT_OK;
    if (b.pending) {
        int rc = cuda_status(cudaEventSynchronize(b.done));
        if (rc) return rc;
        b.pending = false;
    }
    std::memcpy(b.h_blob, img.data(), L.bytes);
    b.last.swap(img);
    return MXFFT_OK;
}

void clear_graphs(mxfft_engine_s* e) {
    for (auto& kv : e->graphs) {
        if (kv.second->buf.pending) cudaEventSynchronize(kv.second->buf.done);
        if (kv.second->exec) cudaGraphExecDestroy(kv.second->exec);
        free_buffers(kv.second->buf);
        delete kv.second;
    }
    e->graphs.clear();
    e->last_buf = nullptr;
}

}  // namespace

namespace mxfft {

cudaError_t engine_flags_async(mxfft_engine_t e, uint32_t* h_flags, cudaStream_t s) {
    if (!e || !h_flags) return cudaErrorInvalidValue;
    if (!e->last_buf || e->last_slices == 0) return cudaSuccess;
    const RunBuffers& b = *e->last_buf;
    return cudaMemcpy2DAsync(h_flags, sizeof(uint32_t),
                             (const char*)b.d_st + offsetof(SliceStats, nonfinite), sizeof(SliceStats),
                             sizeof(uint32_t), (size_t)e->last_slices, cudaMemcpyDeviceToHost, s);
}

}  // namespace mxfft

extern "C" {

int mxfft_engine_create(float tau, float target, int flags, mxfft_engine_t* out) {
    if (!out) return MXFFT_ERR_INVALID;
    *out = nullptr;
    if (!(tau > 0.0f && tau < 1.0f) || !(target > 0.0f) || (flags & ~31)) return MXFFT_ERR_INVALID;
    // validate tau / target the way a plan does
    mxfft_plan_t probe = nullptr;
    int rc = mxfft_plan(2, 2, MXFFT_E4M3, 2, tau, target, &probe);
    if (rc) return rc;
    mxfft_destroy(probe);
    mxfft_engine_s* e = new (std::nothrow) mxfft_engine_s;
    if (!e) return MXFFT_ERR_NOMEM;
    e->tau = tau;
    e->target = target;
    e->flags = flags;
    rc = cuda_status(cudaGetDevice(&e->device));
    if (rc == MXFFT_OK) rc = cuda_status(cudaStreamCreateWithFlags(&e->capture, cudaStreamNonBlocking));
    for (int f = 0; f < kForkStreams && rc == MXFFT_OK; f++)
        rc = cuda_status(cudaStreamCreateWithFlags(&e->fork[f], cudaStreamNonBlocking));
    // 2 fork + 2 * kForkStreams join events per stage, two stages
    e->evs.assign(2 * (1 + kForkStreams) + 2, nullptr);
    for (size_t i = 0; i < e->evs.size() && rc == MXFFT_OK; i++)
        rc = cuda_status(cudaEventCreateWithFlags(&e->evs[i], cudaEventDisableTiming));
    if (rc) { mxfft_engine_destroy(e); return rc; }
    *out = e;
    return MXFFT_OK;
}

int mxfft_engine_run(mxfft_engine_t e, const mxfft_item* items, int n_items, void* stream) {
    struct Range {   // NVTX range on the host timeline for the whole call
        Range() { nvtxRangePushA("mxfft_engine_run"); }
        ~Range() { nvtxRangePop(); }
    } range;
    if (!e || n_items < 0 || (n_items > 0 && !items)) return MXFFT_ERR_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != e->device) return MXFFT_ERR_CUDA;
    for (int i = 0; i < n_items; i++) {
        if (!item_ok(items[i])) return MXFFT_ERR_INVALID;
        if (items[i].slices == 0) continue;
        // the plan constructor checks the shape, format, k
        if (!pow2(items[i].n0) || !pow2(items[i].n1)) return MXFFT_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Layout L;
    std::vector<mxfft_plan_s*> item_plan;
    int rc = build_layout(e, items, n_items, L, item_plan);
    if (rc) return rc;
    if (L.nslices == 0) return MXFFT_OK;

    RunBuffers* b = &e->direct;
    GraphEntry* g = nullptr;
    if (e->flags & MXFFT_ENGINE_GRAPHS) {
        auto f = e->graphs.find(L.signature);
        if (f != e->graphs.end()) {
            g = f->second;
        } else {
            if (e->graphs.size() >= kMaxGraphs) clear_graphs(e);
            g = new (std::nothrow) GraphEntry;
            if (!g) return MXFFT_ERR_NOMEM;
            e->graphs[L.signature] = g;
        }
        b = &g->buf;
    }
    // (a signature fixes the table sizes and slice count, so a graph's
    // buffers are never reallocated under it)
    rc = reserve(*b, L);
    if (rc) return rc;
    fill_layout(items, n_items, item_plan, b->d_st, b->st_cap, b->d_blob,
                !(e->flags & MXFFT_ENGINE_NO_RAGGED), L);
    bool changed = false;
    rc = stage_tables(*b, L, &changed);
    if (rc) return rc;
    // the tables go up (stream-ordered, from the pinned staging buffer) only
    // when they differ from the last upload into these buffers
    cudaError_t err = cudaSuccess;
    // an earlier run of these buffers may still be on another stream: it
    // reads the same statistics records that this run clears first, so this
    // stream waits for it on the device (no host synchronisation)
    if (b->pending) err = cudaStreamWaitEvent(s, b->done, 0);
    if (err == cudaSuccess && changed)
        err = cudaMemcpyAsync(b->d_blob, b->h_blob, L.bytes, cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return cuda_status(err);
    if (g) {
        if (!g->exec) {
            // capture on the engine's own stream (the caller's may be the
            // legacy stream, which cannot be captured)
            cudaGraph_t graph = nullptr;
            err = cudaStreamBeginCapture(e->capture, cudaStreamCaptureModeThreadLocal);
            if (err == cudaSuccess) {
                const long long n0 = g_kernel_launches.load();
                cudaError_t e1 = enqueue(e, L, *b, e->capture);
                g->launches = (int)(g_kernel_launches.load() - n0);
                cudaError_t e2 = cudaStreamEndCapture(e->capture, &graph);
                err = e1 != cudaSuccess ? e1 : e2;
            }
            if (err == cudaSuccess) err = cudaGraphInstantiate(&g->exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (err != cudaSuccess) {
                g->exec = nullptr;
                return cuda_status(err);
            }
        }
        err = cudaGraphLaunch(g->exec, s);
        e->last_launches = g->launches;
    } else {
        const long long n0 = g_kernel_launches.load();
        err = enqueue(e, L, *b, s);
        e->last_launches = (int)(g_kernel_launches.load() - n0);
    }
    if (err == cudaSuccess) err = cudaEventRecord(b->done, s);
    if (err != cudaSuccess) return cuda_status(err);
    b->pending = true;
    e->last_buf = b;
    e->last_slices = L.nslices;
    e->last_rt = L.rt;
    e->last_plans.clear();
    for (auto* p : item_plan)
        if (p && std::find(e->last_plans.begin(), e->last_plans.end(), p) == e->last_plans.end())
            e->last_plans.push_back(p);
    return MXFFT_OK;
}

int mxfft_engine_launches(mxfft_engine_t e, int* launches) {
    if (!e || !launches) return MXFFT_ERR_INVALID;
    *launches = e->last_launches;
    return MXFFT_OK;
}

int mxfft_engine_get_status(mxfft_engine_t e, int* device_flags, int32_t* k_out, int k_out_len) {
    if (!e || !device_flags || (k_out && k_out_len < 0)) return MXFFT_ERR_INVALID;
    *device_flags = 0;
    if (!e->last_buf) return MXFFT_OK;
    RunBuffers& b = *e->last_buf;
    int rc = cuda_status(cudaEventSynchronize(b.done));
    if (rc) return rc;
    const int S = e->last_slices;
    std::vector<SliceStats> st(2 * (size_t)b.st_cap);
    rc = cuda_status(cudaMemcpy(st.data(), b.d_st, st.size() * sizeof(SliceStats), cudaMemcpyDeviceToHost));
    if (rc) return rc;
    int flags = 0;
    for (int g = 0; g < S; g++)
        if (st[g].nonfinite || (e->last_rt[g] && st[b.st_cap + g].nonfinite)) flags |= 1;
    for (mxfft_plan_s* p : e->last_plans) {
        if (!p->d_err) continue;
        int err = 0;
        rc = cuda_status(cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (rc) return rc;
        if (err) flags |= 2;
    }
    *device_flags = flags;
    if (k_out)
        for (int g = 0; g < S && 2 * g < k_out_len; g++) {
            k_out[2 * g] = st[g].k;
            if (2 * g + 1 < k_out_len) k_out[2 * g + 1] = e->last_rt[g] ? st[b.st_cap + g].k : 0;
        }
    return MXFFT_OK;
}

int mxfft_engine_destroy(mxfft_engine_t e) {
    if (!e) return MXFFT_ERR_INVALID;
    clear_graphs(e);
    if (e->direct.pending) cudaEventSynchronize(e->direct.done);
    free_buffers(e->direct);
    for (auto& kv : e->plans) mxfft_destroy(kv.second);
    for (cudaEvent_t ev : e->evs)
        if (ev) cudaEventDestroy(ev);
    for (int f = 0; f < kForkStreams; f++)
        if (e->fork[f]) cudaStreamDestroy(e->fork[f]);
    if (e->capture) cudaStreamDestroy(e->capture);
    delete e;
    return MXFFT_OK;
}

}  // extern "C"
