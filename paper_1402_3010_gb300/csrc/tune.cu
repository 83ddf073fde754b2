// Join tile shapes per instance size, and the autotuner that chooses them by measurement.
//
// An instance is joined with G query groups per CTA (G = 1, 2, 4, 8), each group holding a
// candidate window of JOIN_WMAX / G ids in shared memory: a small G gives long windows
// (fewer windows, so less fixed cost per query), a large G more queries in flight per SM.
// This is the block size of Sec. 5.1.9 turned into a CTA-level tile, and like the paper's
// block size it is a measured choice. The table maps an instance's size bucket to G; the
// bucket bounds are the work-split thresholds between the shapes.
#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "index.cuh"

namespace aps {
namespace {

const int64_t BOUNDS[APS_TUNE_BUCKETS] = {512, 1280, 2560, 5120, 10240, 20480, 40960, INT64_MAX};
const int GS[4] = {1, 2, 4, 8};

// Default for self-joins: the largest G whose window still holds the whole instance (one
// window per query), but at least 2 groups. Measured on the 200k-vector power-law set
// (join ms): G = 1: 71.7, 2: 65.0, 4: 65.6, 8: 72.9.
// Default for queryable indexes: the same. Their queries are (query, window) work items,
// so a long query's windows run on several CTAs; on the 1M-vector serving index G = 1 and
// G = 2 then serve alike (84.3k and 84.5k queries/s saturated). Before that split, a
// batch waited for its longest query on one group, and G = 1 (a whole CTA per query)
// served 47.0k against 23.5k with G = 2.
const aps_tuning DEFAULT_TUNING = {{8, 8, 8, 8, 4, 2, 2, 2}, {8, 8, 8, 8, 4, 2, 2, 2}};

std::mutex g_tune_mu;
aps_tuning g_tune = DEFAULT_TUNING;

constexpr int64_t SAMPLE_ROWS = 1 << 18;  // vectors per bucket sample (whole instances)

// Join time (least of reps) of the batch's instances `sel` (ascending ids) under table tu.
// The whole batch is indexed in place; a proper subset is first copied into its own CSR.
aps_status time_join(const std::vector<int> &sel, int32_t k, const int64_t *ro, const int64_t *hptr,
                     const int64_t *dp, const int32_t *di, const float *dv, const int32_t *m, const float *t,
                     uint32_t flags, const aps_tuning &tu, int reps, cudaStream_t s, float *ms) {
    std::vector<InstDesc> desc;
    DBuf<int64_t> sp;
    DBuf<int32_t> si;
    DBuf<float> sv;
    const int64_t *p = dp;
    const int32_t *ii = di;
    const float *vv = dv;
    for (int r : sel) {
        InstDesc I;
        memset(&I, 0, sizeof(I));
        I.n = (int32_t)(ro[r + 1] - ro[r]);
        I.m = m[r];
        I.t = t[r];
        desc.push_back(I);
    }
    if ((int32_t)sel.size() != k) {
        std::vector<int64_t> hp(1, 0);
        int64_t nz = 0;
        for (int r : sel) {
            for (int64_t x = ro[r]; x < ro[r + 1]; x++) hp.push_back(nz + hptr[x + 1] - hptr[ro[r]]);
            nz += hptr[ro[r + 1]] - hptr[ro[r]];
        }
        APS_TRY(sp.alloc(hp.size(), s));
        APS_TRY(si.alloc((size_t)std::max<int64_t>(nz, 1), s));
        APS_TRY(sv.alloc((size_t)std::max<int64_t>(nz, 1), s));
        APS_CUDA(cudaMemcpyAsync(sp.p, hp.data(), sizeof(int64_t) * hp.size(), cudaMemcpyHostToDevice, s));
        int64_t off = 0;
        for (int r : sel) {
            const int64_t a = hptr[ro[r]], c = hptr[ro[r + 1]] - a;
            if (c > 0) {
                APS_CUDA(cudaMemcpyAsync(si.p + off, di + a, sizeof(int32_t) * c, cudaMemcpyDeviceToDevice, s));
                APS_CUDA(cudaMemcpyAsync(sv.p + off, dv + a, sizeof(float) * c, cudaMemcpyDeviceToDevice, s));
            }
            off += c;
        }
        p = sp.p;
        ii = si.p;
        vv = sv.p;
    }
    aps_index *ix = new (std::nothrow) aps_index();
    if (!ix) return APS_ENOMEM;
    ix->flags = flags;
    ix->stream = s;
    cudaGetDevice(&ix->device);
    aps_status st = build_index_device(ix, p, ii, vv, desc, s, &tu);
    float best = -1.f;
    for (int r = 0; r < reps && st == APS_OK; r++) {
        aps_pairs out;
        memset(&out, 0, sizeof(out));
        st = join_all_pairs(ix, flags, &out, nullptr);
        if (st == APS_OK) {
            const float j = ix->stats.ms_join;
            best = best < 0.f ? j : std::min(best, j);
        }
        pairs_release(&out);
    }
    delete ix;
    cudaStreamSynchronize(s);
    *ms = best;
    return st;
}

}  // namespace

int tune_bucket(int64_t n) {
    int b = 0;
    while (b < APS_TUNE_BUCKETS - 1 && n > BOUNDS[b]) b++;
    return b;
}

aps_tuning tuning_default() { return DEFAULT_TUNING; }

aps_tuning tuning_current() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune;
}

bool tuning_valid(const aps_tuning &tu) {
    for (int b = 0; b < APS_TUNE_BUCKETS; b++)
        for (const int g : {tu.groups[b], tu.query_groups[b]})
            if (g != 1 && g != 2 && g != 4 && g != 8) return false;
    return true;
}

void tuning_set(const aps_tuning &tu) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune = tu;
}

aps_status autotune_batch(int32_t k, const int64_t *ro, const int64_t *hptr, const int64_t *dp, const int32_t *di,
                          const float *dv, const int32_t *m, const float *t, uint32_t flags, cudaStream_t s,
                          aps_tuning *out, aps_tune_report *rep) {
    aps_tune_report R;
    memset(&R, 0, sizeof(R));
    for (int b = 0; b < APS_TUNE_BUCKETS; b++)
        for (int gi = 0; gi < 4; gi++) R.ms[b][gi] = -1.f;
    const aps_tuning cur = tuning_current();
    aps_tuning tuned = cur;
    std::vector<std::vector<int>> members(APS_TUNE_BUCKETS);
    for (int r = 0; r < k; r++) members[tune_bucket(ro[r + 1] - ro[r])].push_back(r);
    for (int b = 0; b < APS_TUNE_BUCKETS; b++) {
        std::vector<int> &L = members[b];
        R.instances[b] = (int32_t)L.size();
        if (L.empty()) continue;
        // sample: q instances spread evenly over the bucket's size order, the most that fit
        // SAMPLE_ROWS vectors (at least one)
        std::vector<int> by_n = L;
        std::stable_sort(by_n.begin(), by_n.end(),
                         [&](int a, int c) { return ro[a + 1] - ro[a] < ro[c + 1] - ro[c]; });
        std::vector<int> sel;
        for (int64_t q = (int64_t)by_n.size(); q >= 1; q--) {
            sel.clear();
            int64_t rows = 0;
            for (int64_t i = 0; i < q; i++) {
                const int r = by_n[(size_t)(((2 * i + 1) * (int64_t)by_n.size()) / (2 * q))];
                sel.push_back(r);
                rows += ro[r + 1] - ro[r];
            }
            if (rows <= SAMPLE_ROWS || q == 1) break;
        }
        std::sort(sel.begin(), sel.end());
        R.sampled[b] = (int32_t)sel.size();
        float best = -1.f;
        int best_g = cur.groups[b];
        for (int gi = 0; gi < 4; gi++) {
            aps_tuning force = cur;
            for (int c = 0; c < APS_TUNE_BUCKETS; c++) force.groups[c] = GS[gi];
            float ms = -1.f;
            APS_TRY(time_join(sel, k, ro, hptr, dp, di, dv, m, t, flags, force, 3, s, &ms));
            R.ms[b][gi] = ms;
            if (ms >= 0.f && (best < 0.f || ms < best)) {
                best = ms;
                best_g = GS[gi];
            }
        }
        const int ci = cur.groups[b] == 1 ? 0 : cur.groups[b] == 2 ? 1 : cur.groups[b] == 4 ? 2 : 3;
        tuned.groups[b] = (R.ms[b][ci] >= 0.f && R.ms[b][ci] <= 1.02f * best) ? cur.groups[b] : best_g;
    }
    // the whole batch: the chosen table against the default
    std::vector<int> all((size_t)k);
    for (int r = 0; r < k; r++) all[(size_t)r] = r;
    aps_tuning def = DEFAULT_TUNING;
    memcpy(def.query_groups, cur.query_groups, sizeof(def.query_groups));  // the queryable column stays
    APS_TRY(time_join(all, k, ro, hptr, dp, di, dv, m, t, flags, def, 2, s, &R.ms_default));
    if (memcmp(&tuned, &def, sizeof(def)) == 0) {
        R.ms_tuned = R.ms_default;
    } else {
        APS_TRY(time_join(all, k, ro, hptr, dp, di, dv, m, t, flags, tuned, 2, s, &R.ms_tuned));
    }
    if (!(R.ms_tuned < R.ms_default)) {
        R.kept_default = memcmp(&tuned, &def, sizeof(def)) != 0;
        tuned = def;
    }
    tuning_set(tuned);
    *out = tuned;
    if (rep) *rep = R;
    return APS_OK;
}

}  // namespace aps
