// extern "C" entry points of libaps.so (declared in include/aps.h).
#include <cmath>
#include <cstring>
#include <new>

#include "index.cuh"

using namespace aps;

namespace {

struct HostCsrCopy {  // device copies of a host CSR
    DBuf<int64_t> indptr;
    DBuf<int32_t> idx;
    DBuf<float> val;
};

aps_status check_threshold(float t) {
    if (!(t > 0.f) || !(t <= 1.f)) {
        set_error("threshold t must be in (0, 1], got %g", (double)t);
        return APS_EINVAL;
    }
    return APS_OK;
}

// Bring one CSR to the device (or just borrow device pointers).
aps_status stage_csr(const int64_t *indptr, const int32_t *idx, const float *val, int64_t n, uint32_t flags,
                     cudaStream_t s, HostCsrCopy &c, const int64_t **dp, const int32_t **di, const float **dv) {
    if (!indptr) {
        set_error("indptr must not be NULL");
        return APS_EINVAL;
    }
    if (flags & APS_DEVICE_PTRS) {
        *dp = indptr;
        *di = idx;
        *dv = val;
        return APS_OK;
    }
    if (indptr[0] != 0) {
        set_error("indptr[0] must be 0");
        return APS_EINVAL;
    }
    const int64_t nnz = indptr[n];
    if (nnz < 0 || nnz >= (1ll << 31)) {
        set_error("nnz = %lld out of range [0, 2^31)", (long long)nnz);
        return APS_EINVAL;
    }
    if (nnz > 0 && (!idx || !val)) {
        set_error("idx and val must not be NULL when nnz > 0");
        return APS_EINVAL;
    }
    APS_TRY(c.indptr.alloc((size_t)n + 1, s));
    APS_TRY(c.idx.alloc((size_t)nnz, s));
    APS_TRY(c.val.alloc((size_t)nnz, s));
    APS_CUDA(cudaMemcpyAsync(c.indptr.p, indptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
    if (nnz) {
        APS_CUDA(cudaMemcpyAsync(c.idx.p, idx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
        APS_CUDA(cudaMemcpyAsync(c.val.p, val, sizeof(float) * nnz, cudaMemcpyHostToDevice, s));
    }
    *dp = c.indptr.p;
    *di = c.idx.p;
    *dv = c.val.p;
    return APS_OK;
}

aps_status build_single(const int64_t *indptr, const int32_t *idx, const float *val, int32_t n, int32_t m, float t,
                        uint32_t flags, cudaStream_t s, aps_index **out) {
    if (!out) {
        set_error("out must not be NULL");
        return APS_EINVAL;
    }
    *out = nullptr;
    if (n < 0 || m < 1) {
        set_error("need n >= 0 and m >= 1 (got n=%d m=%d)", n, m);
        return APS_EINVAL;
    }
    APS_TRY(check_threshold(t));
    aps_index *ix = new (std::nothrow) aps_index();
    if (!ix) {
        set_error("host allocation failed");
        return APS_ENOMEM;
    }
    cudaGetDevice(&ix->device);
    ix->flags = flags;
    ix->t = t;
    ix->stream = s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    aps_status st;
    {
        HostCsrCopy c;
        const int64_t *dp;
        const int32_t *di;
        const float *dv;
        st = stage_csr(indptr, idx, val, n, flags, s, c, &dp, &di, &dv);
        if (st == APS_OK) {
            std::vector<InstDesc> inst(1);
            memset(inst.data(), 0, sizeof(InstDesc));
            inst[0].n = n;
            inst[0].m = m;
            inst[0].t = t;
            st = build_index_device(ix, dp, di, dv, inst, s);
        }
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != APS_OK) {
        delete ix;
        return st;
    }
    ix->stats.ms_build = ms;
    *out = ix;
    return APS_OK;
}

template <class T>
aps_status export_array(T *dst, const DBuf<T> &src, size_t n, cudaStream_t s) {
    if (!dst || n == 0) return APS_OK;
    APS_CUDA(cudaMemcpyAsync(dst, src.p, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
    return APS_OK;
}

}  // namespace

extern "C" {

aps_status aps_build_index(const int64_t *indptr, const int32_t *idx, const float *val, int32_t n, int32_t m, float t,
                           uint32_t flags, void *stream, aps_index **out) {
    return build_single(indptr, idx, val, n, m, t, flags, static_cast<cudaStream_t>(stream), out);
}

aps_status aps_all_pairs(aps_index *index, uint32_t flags, aps_pairs *out) {
    if (!index || !out) {
        set_error("index and out must not be NULL");
        return APS_EINVAL;
    }
    memset(out, 0, sizeof(*out));
    if (index->k != 1) {
        set_error("aps_all_pairs needs a single-instance index");
        return APS_EINVAL;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, index->stream);
    aps_status st = join_all_pairs(index, flags, out, nullptr);
    if (st == APS_OK && (flags & APS_HOST_OUTPUT)) st = pairs_to_host(out, index->stream);
    cudaEventRecord(e1, index->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    index->stats.ms_total = ms;
    if (st != APS_OK) pairs_release(out);
    return st;
}

aps_status aps_all_pairs_split(aps_index *index, int32_t nblk, int64_t heavy, uint32_t flags, aps_pairs *out) {
    if (!index || !out) {
        set_error("index and out must not be NULL");
        return APS_EINVAL;
    }
    memset(out, 0, sizeof(*out));
    if (index->k != 1) {
        set_error("aps_all_pairs_split needs a single-instance index");
        return APS_EINVAL;
    }
    if (nblk < 2 || nblk > 8 || heavy < 0) {
        set_error("need 2 <= nblk <= 8 dimension blocks and heavy >= 0");
        return APS_EINVAL;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, index->stream);
    aps_status st = join_all_pairs(index, flags, out, nullptr, nblk, heavy);
    if (st == APS_OK && (flags & APS_HOST_OUTPUT)) st = pairs_to_host(out, index->stream);
    cudaEventRecord(e1, index->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    index->stats.ms_total = ms;
    if (st != APS_OK) pairs_release(out);
    return st;
}

aps_status aps_index_export(const aps_index *ix, int32_t *len, float *mw, int32_t *nnz_d, float *mw_d,
                            int32_t *rank_of_dim, int32_t *crank, float *cval, int32_t *split, int32_t *qsplit,
                            float *mw_pre, int64_t *list_ptr, int32_t *post_id, float *post_w) {
    if (!ix) {
        set_error("index must not be NULL");
        return APS_EINVAL;
    }
    cudaStream_t s = ix->stream;
    const IndexArrays &d = ix->d;
    APS_TRY(export_array(len, d.len, ix->N, s));
    APS_TRY(export_array(mw, d.mw, ix->N, s));
    APS_TRY(export_array(nnz_d, d.nnz_d, ix->M, s));
    APS_TRY(export_array(mw_d, d.mw_d, ix->M, s));
    APS_TRY(export_array(rank_of_dim, d.rank_of_dim, ix->M, s));
    APS_TRY(export_array(crank, d.crank, ix->nnz, s));
    APS_TRY(export_array(cval, d.cval, ix->nnz, s));
    APS_TRY(export_array(split, d.split, ix->N, s));
    APS_TRY(export_array(qsplit, d.qsplit, ix->N, s));
    APS_TRY(export_array(mw_pre, d.mwpre, ix->N, s));
    APS_TRY(export_array(list_ptr, d.lptr, ix->M + 1, s));
    if ((post_id || post_w) && ix->nsuf > 0) {
        std::vector<int2> tmp((size_t)ix->nsuf);
        APS_CUDA(cudaMemcpyAsync(tmp.data(), d.post.p, sizeof(int2) * ix->nsuf, cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaStreamSynchronize(s));
        const int32_t mask = (ix->k == 1 && ix->inst_h[0].packed) ? 0x00ffffff : 0x7fffffff;
        for (int64_t q = 0; q < ix->nsuf; q++) {
            if (post_id) post_id[q] = tmp[q].x & mask;
            if (post_w) memcpy(&post_w[q], &tmp[q].y, 4);
        }
    }
    APS_CUDA(cudaStreamSynchronize(s));
    return APS_OK;
}

aps_status aps_index_info(const aps_index *ix, int32_t *n, int32_t *m, int64_t *nnz, int64_t *indexed) {
    if (!ix) {
        set_error("index must not be NULL");
        return APS_EINVAL;
    }
    if (n) *n = (int32_t)ix->N;
    if (m) *m = (int32_t)ix->M;
    if (nnz) *nnz = ix->nnz;
    if (indexed) *indexed = ix->nsuf;
    return APS_OK;
}

aps_status aps_index_stats(const aps_index *ix, aps_stats *out) {
    if (!ix || !out) {
        set_error("index and out must not be NULL");
        return APS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(ix->stats_mu);
    *out = ix->stats;
    return APS_OK;
}

void aps_index_free(aps_index *ix) {
    if (!ix) return;
    cudaStream_t s = ix->stream;
    delete ix;  // DBuf members free on the index stream
    cudaStreamSynchronize(s);
}

void aps_pairs_free(aps_pairs *p) { pairs_release(p); }

aps_status aps_pairs_copy_to(const aps_pairs *p, int32_t *i, int32_t *j, float *score, void *stream) {
    if (!p) {
        set_error("pairs must not be NULL");
        return APS_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)p->count;
    if (n) {
        if (i) APS_CUDA(cudaMemcpyAsync(i, p->i, n * 4, cudaMemcpyDefault, s));
        if (j) APS_CUDA(cudaMemcpyAsync(j, p->j, n * 4, cudaMemcpyDefault, s));
        if (score) APS_CUDA(cudaMemcpyAsync(score, p->score, n * 4, cudaMemcpyDefault, s));
    }
    APS_CUDA(cudaStreamSynchronize(s));
    return APS_OK;
}

aps_status aps_batch_all_pairs(int32_t k, const aps_instance *inst, uint32_t flags, void *stream, aps_pairs *outs,
                               aps_stats *stats) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (k < 1 || !inst || !outs) {
        set_error("need k >= 1 instances and non-NULL inst/outs");
        return APS_EINVAL;
    }
    for (int i = 0; i < k; i++) memset(&outs[i], 0, sizeof(aps_pairs));
    // concatenate the instances' CSRs
    std::vector<InstDesc> desc((size_t)k);
    std::vector<int64_t> nnzs((size_t)k);
    int64_t N = 0, NNZ = 0;
    for (int i = 0; i < k; i++) {
        const aps_instance &I = inst[i];
        if (I.n < 0 || I.m < 1 || !I.indptr) {
            set_error("instance %d: need n >= 0, m >= 1 and indptr", i);
            return APS_EINVAL;
        }
        APS_TRY(check_threshold(I.t));
        int64_t nz = 0;
        if (flags & APS_DEVICE_PTRS) {
            APS_CUDA(cudaMemcpy(&nz, I.indptr + I.n, sizeof(int64_t), cudaMemcpyDeviceToHost));
        } else {
            if (I.indptr[0] != 0) {
                set_error("instance %d: indptr[0] must be 0", i);
                return APS_EINVAL;
            }
            nz = I.indptr[I.n];
        }
        if (nz < 0) {
            set_error("instance %d: negative nnz", i);
            return APS_EINVAL;
        }
        memset(&desc[i], 0, sizeof(InstDesc));
        desc[i].n = I.n;
        desc[i].m = I.m;
        desc[i].t = I.t;
        nnzs[i] = nz;
        N += I.n;
        NNZ += nz;
    }
    if (NNZ >= (1ll << 31)) {
        set_error("total nnz must be < 2^31");
        return APS_EINVAL;
    }
    aps_index *ix = new (std::nothrow) aps_index();
    if (!ix) return APS_ENOMEM;
    ix->flags = flags;
    ix->stream = s;
    cudaGetDevice(&ix->device);
    cudaEvent_t e0, e1, e2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    cudaEventRecord(e0, s);
    aps_status st = APS_OK;
    std::vector<int64_t> offs;
    {
        DBuf<int64_t> dptr;
        DBuf<int32_t> didx;
        DBuf<float> dval;
        st = dptr.alloc((size_t)N + 1, s);
        if (st == APS_OK) st = didx.alloc((size_t)NNZ, s);
        if (st == APS_OK) st = dval.alloc((size_t)NNZ, s);
        if (st == APS_OK) {
            std::vector<int64_t> hptr((size_t)N + 1);
            int64_t vb = 0, eb = 0;
            const cudaMemcpyKind kind = (flags & APS_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
            for (int i = 0; i < k && st == APS_OK; i++) {
                const aps_instance &I = inst[i];
                if (flags & APS_DEVICE_PTRS) {
                    std::vector<int64_t> tmp((size_t)I.n + 1);
                    if (cudaMemcpy(tmp.data(), I.indptr, sizeof(int64_t) * (I.n + 1), cudaMemcpyDeviceToHost) !=
                        cudaSuccess) {
                        st = APS_ECUDA;
                        break;
                    }
                    for (int r = 0; r <= I.n; r++) hptr[vb + r] = eb + tmp[r];
                } else {
                    for (int r = 0; r <= I.n; r++) hptr[vb + r] = eb + I.indptr[r];
                }
                if (nnzs[i]) {
                    if (cudaMemcpyAsync(didx.p + eb, I.idx, sizeof(int32_t) * nnzs[i], kind, s) != cudaSuccess ||
                        cudaMemcpyAsync(dval.p + eb, I.val, sizeof(float) * nnzs[i], kind, s) != cudaSuccess) {
                        set_error("copy of instance %d failed", i);
                        st = APS_ECUDA;
                    }
                }
                vb += I.n;
                eb += nnzs[i];
            }
            if (st == APS_OK && cudaMemcpyAsync(dptr.p, hptr.data(), sizeof(int64_t) * (N + 1),
                                                cudaMemcpyHostToDevice, s) != cudaSuccess)
                st = APS_ECUDA;
            if (st == APS_OK) st = cudaStreamSynchronize(s) == cudaSuccess ? APS_OK : APS_ECUDA;
            if (st == APS_OK) st = build_index_device(ix, dptr.p, didx.p, dval.p, desc, s);
        }
    }
    cudaEventRecord(e1, s);
    aps_pairs all;
    memset(&all, 0, sizeof(all));
    if (st == APS_OK) st = join_all_pairs(ix, flags, &all, &offs);
    if (st == APS_OK && (flags & APS_HOST_OUTPUT)) st = pairs_to_host(&all, s);
    cudaEventRecord(e2, s);
    cudaEventSynchronize(e2);
    if (st == APS_OK) {
        float mb = 0, mt = 0;
        cudaEventElapsedTime(&mb, e0, e1);
        cudaEventElapsedTime(&mt, e0, e2);
        ix->stats.ms_build = mb;
        ix->stats.ms_total = mt;
        if (stats) *stats = ix->stats;
        static_cast<PairsAlloc *>(all._priv)->refs = k;
        for (int i = 0; i < k; i++) {
            aps_pairs &o = outs[i];
            const int64_t a = offs[i], b = offs[i + 1];
            o.count = b - a;
            o.i = all.i + a;
            o.j = all.j + a;
            o.score = all.score + a;
            o.on_device = all.on_device;
            o._priv = all._priv;
        }
    } else {
        pairs_release(&all);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    delete ix;
    cudaStreamSynchronize(s);
    return st;
}

aps_status aps_batch_all_pairs_csr(int32_t k, const int64_t *row_offsets, const int64_t *indptr, const int32_t *idx,
                                   const float *val, const int32_t *m, const float *t, uint32_t flags, void *stream,
                                   aps_pairs *outs, aps_stats *stats) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (k < 1 || !row_offsets || !indptr || !m || !t || !outs) {
        set_error("need k >= 1 and non-NULL row_offsets, indptr, m, t, outs");
        return APS_EINVAL;
    }
    for (int i = 0; i < k; i++) memset(&outs[i], 0, sizeof(aps_pairs));
    if (row_offsets[0] != 0) {
        set_error("row_offsets[0] must be 0");
        return APS_EINVAL;
    }
    std::vector<InstDesc> desc((size_t)k);
    for (int i = 0; i < k; i++) {
        const int64_t n = row_offsets[i + 1] - row_offsets[i];
        if (n < 0 || n >= (1ll << 31) || m[i] < 1) {
            set_error("instance %d: need 0 <= n < 2^31 and m >= 1", i);
            return APS_EINVAL;
        }
        APS_TRY(check_threshold(t[i]));
        memset(&desc[i], 0, sizeof(InstDesc));
        desc[i].n = (int32_t)n;
        desc[i].m = m[i];
        desc[i].t = t[i];
    }
    const int64_t N = row_offsets[k];
    aps_index *ix = new (std::nothrow) aps_index();
    if (!ix) return APS_ENOMEM;
    ix->flags = flags;
    ix->stream = s;
    cudaGetDevice(&ix->device);
    cudaEvent_t e0, e1, e2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    cudaEventRecord(e0, s);
    aps_status st;
    std::vector<int64_t> offs;
    {
        HostCsrCopy c;
        const int64_t *dp;
        const int32_t *di;
        const float *dv;
        st = stage_csr(indptr, idx, val, N, flags, s, c, &dp, &di, &dv);
        if (st == APS_OK) st = build_index_device(ix, dp, di, dv, desc, s);
    }
    cudaEventRecord(e1, s);
    aps_pairs all;
    memset(&all, 0, sizeof(all));
    if (st == APS_OK) st = join_all_pairs(ix, flags, &all, &offs);
    if (st == APS_OK && (flags & APS_HOST_OUTPUT)) st = pairs_to_host(&all, s);
    cudaEventRecord(e2, s);
    cudaEventSynchronize(e2);
    if (st == APS_OK) {
        float mb = 0, mt = 0;
        cudaEventElapsedTime(&mb, e0, e1);
        cudaEventElapsedTime(&mt, e0, e2);
        ix->stats.ms_build = mb;
        ix->stats.ms_total = mt;
        if (stats) *stats = ix->stats;
        static_cast<PairsAlloc *>(all._priv)->refs = k;
        for (int i = 0; i < k; i++) {
            aps_pairs &o = outs[i];
            o.count = offs[i + 1] - offs[i];
            o.i = all.i + offs[i];
            o.j = all.j + offs[i];
            o.score = all.score + offs[i];
            o.on_device = all.on_device;
            o._priv = all._priv;
        }
    } else {
        pairs_release(&all);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    delete ix;
    cudaStreamSynchronize(s);
    return st;
}

int32_t aps_tune_bucket(int64_t n) { return tune_bucket(n); }

void aps_tuning_default(aps_tuning *out) {
    if (out) *out = tuning_default();
}

void aps_get_tuning(aps_tuning *out) {
    if (out) *out = tuning_current();
}

aps_status aps_set_tuning(const aps_tuning *tuning) {
    if (!tuning || !tuning_valid(*tuning)) {
        set_error("a tuning table needs 1, 2, 4 or 8 query groups in every bucket");
        return APS_EINVAL;
    }
    tuning_set(*tuning);
    return APS_OK;
}

aps_status aps_autotune_batch_csr(int32_t k, const int64_t *row_offsets, const int64_t *indptr, const int32_t *idx,
                                  const float *val, const int32_t *m, const float *t, uint32_t flags, void *stream,
                                  aps_tuning *out, aps_tune_report *report) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (k < 1 || !row_offsets || !indptr || !m || !t || !out) {
        set_error("need k >= 1 and non-NULL row_offsets, indptr, m, t, out");
        return APS_EINVAL;
    }
    if (row_offsets[0] != 0) {
        set_error("row_offsets[0] must be 0");
        return APS_EINVAL;
    }
    for (int i = 0; i < k; i++) {
        const int64_t n = row_offsets[i + 1] - row_offsets[i];
        if (n < 0 || n >= (1ll << 31) || m[i] < 1) {
            set_error("instance %d: need 0 <= n < 2^31 and m >= 1", i);
            return APS_EINVAL;
        }
        APS_TRY(check_threshold(t[i]));
    }
    const int64_t N = row_offsets[k];
    HostCsrCopy c;
    const int64_t *dp;
    const int32_t *di;
    const float *dv;
    APS_TRY(stage_csr(indptr, idx, val, N, flags, s, c, &dp, &di, &dv));
    // the sample CSRs are cut on the host side of the row pointers
    std::vector<int64_t> hptr;
    const int64_t *hp = indptr;
    if (flags & APS_DEVICE_PTRS) {
        hptr.resize((size_t)N + 1);
        APS_CUDA(cudaMemcpyAsync(hptr.data(), indptr, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaStreamSynchronize(s));
        hp = hptr.data();
    }
    // the self-join column is tuned: the timed joins take neither host output nor the
    // queryable split
    return autotune_batch(k, row_offsets, hp, dp, di, dv, m, t, flags & ~(uint32_t)(APS_HOST_OUTPUT | APS_QUERYABLE), s,
                          out, report);
}

aps_status aps_all_pairs_dense(const float *X, int32_t n, int32_t d, float t, uint32_t flags, void *stream,
                               aps_pairs *out, aps_stats *stats) {
    if (!out) {
        set_error("out must not be NULL");
        return APS_EINVAL;
    }
    memset(out, 0, sizeof(*out));
    if (stats) memset(stats, 0, sizeof(*stats));
    APS_TRY(check_threshold(t));
    if (n < 0 || d < 64 || d > 512 || d % 64 != 0 || (n > 0 && !X)) {
        set_error("need n >= 0, X != NULL and d a multiple of 64 in [64, 512] (got n=%d d=%d)", n, d);
        return APS_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    aps_status st = dense_all_pairs(X, n, d, t, flags, s, out, stats);
    if (st == APS_OK && (flags & APS_HOST_OUTPUT)) st = pairs_to_host(out, s);
    if (st != APS_OK) pairs_release(out);
    return st;
}

aps_status aps_dense_tensor_products(const float *X, int32_t n, int32_t d, float *raw, void *stream) {
    if (n < 0 || n > 16384 || d < 64 || d > 512 || d % 64 != 0 || (n > 0 && (!X || !raw))) {
        set_error("need 0 <= n <= 16384, device X and raw, and d a multiple of 64 in [64, 512] (got n=%d d=%d)", n,
                  d);
        return APS_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(X) & 15) {
        set_error("X must be 16-byte aligned");
        return APS_EINVAL;
    }
    if (n == 0) return APS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    APS_TRY(dense_tensor_products(X, n, d, s, raw));
    APS_CUDA(cudaStreamSynchronize(s));
    return APS_OK;
}

const char *aps_version(void) { return "aps 0.1 (sm_103a)"; }

void aps_debug_fail_alloc(int64_t k) { set_alloc_fault(k); }

void aps_debug_dense_stall(int64_t launches, uint64_t wait_ns) { dense_debug_stall(launches, wait_ns); }

void aps_debug_stage_cap(int64_t pairs) { debug_stage_cap(pairs); }

aps_status aps_graph_csr(const int32_t *i, const int32_t *j, const float *s, int64_t count, int32_t n,
                         uint32_t flags, void *stream, aps_graph *out) {
    if (!out) {
        set_error("out must not be NULL");
        return APS_EINVAL;
    }
    return graph_csr(i, j, s, count, n, flags, static_cast<cudaStream_t>(stream), out);
}

aps_status aps_graph_knn(const aps_graph *g, int32_t k, int32_t *nbr, float *wk, uint32_t flags, void *stream) {
    return graph_knn(g, k, nbr, wk, flags, static_cast<cudaStream_t>(stream));
}

aps_status aps_graph_copy_to(const aps_graph *g, int64_t *row_ptr, int32_t *col, float *w, void *stream) {
    if (!g || !g->_priv) {
        set_error("the graph must come from aps_graph_csr");
        return APS_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (row_ptr) APS_CUDA(cudaMemcpyAsync(row_ptr, g->row_ptr, 8 * ((size_t)g->n + 1), cudaMemcpyDefault, s));
    if (g->nnz) {
        if (col) APS_CUDA(cudaMemcpyAsync(col, g->col, 4 * (size_t)g->nnz, cudaMemcpyDefault, s));
        if (w) APS_CUDA(cudaMemcpyAsync(w, g->w, 4 * (size_t)g->nnz, cudaMemcpyDefault, s));
    }
    APS_CUDA(cudaStreamSynchronize(s));
    return APS_OK;
}

void aps_graph_free(aps_graph *g) { graph_release(g); }

aps_status aps_pairs_verify(const aps_pairs *lists, int32_t k, const int64_t *indptr, const int32_t *idx,
                            const float *val, int32_t n, int32_t m, float t, uint32_t flags, void *stream,
                            aps_pairs *out, int64_t *n_candidates) {
    if (!out || (k > 0 && !lists) || k < 0 || n < 0 || m < 1) {
        set_error("need out != NULL, k >= 0 lists, n >= 0 and m >= 1");
        return APS_EINVAL;
    }
    if (!(t > 0.f) || !(t <= 1.f)) {
        set_error("threshold t must be in (0, 1], got %g", (double)t);
        return APS_EINVAL;
    }
    memset(out, 0, sizeof(*out));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HostCsrCopy hc;
    const int64_t *dp = nullptr;
    const int32_t *di = nullptr;
    const float *dv = nullptr;
    APS_TRY(stage_csr(indptr, idx, val, n, flags, s, hc, &dp, &di, &dv));
    aps_status st = pairs_verify(lists, k, dp, di, dv, n, m, t, s, out, n_candidates);
    if (st == APS_OK && (flags & APS_HOST_OUTPUT)) st = pairs_to_host(out, s);
    if (st != APS_OK) pairs_release(out);
    return st;
}

}  // extern "C"
