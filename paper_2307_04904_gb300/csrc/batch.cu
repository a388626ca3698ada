// batch.cu -- planning and running batches of ragged DTW jobs (dtwgb_batch.h).
//
// Plan: every pair of every job gets its band (the same readings as
// dtw_pairwise) and a shape: (family, K) per length/band bucket from the
// instruction-count model or from timing candidates on sampled pairs
// (autotuner), then the exact G and masked tail per pair for rotated shapes.
// Pairs with equal (family, K, G, MT) form a class; each class is a work
// queue sorted by estimated cost, largest first, popped by one persistent
// kernel.  Run: reset the queue heads, stage every job's series into the
// padded buffer, launch every class (class 0 on the caller's stream, the
// others on side streams forked and joined by events, so they overlap), zero
// the diagonals -- captured once into a CUDA graph when asked.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dtwgb_batch.h"
#include "band_tworow.cuh"
#include "tstrip.cuh"

namespace dtwgb {
namespace {

struct ClassKey {
    int kind, K, G, MT;
    bool operator<(const ClassKey &o) const
    {
        if (kind != o.kind) return kind < o.kind;
        if (K != o.K) return K < o.K;
        if (G != o.G) return G < o.G;
        return MT < o.MT;
    }
};

struct ClassPlan {
    ClassKey key;
    std::vector<uint64_t> items;  // host, sorted
    int64_t cells = 0;
    int maxlen = 0;               // strip: longest row count of its pairs
    uint64_t *d_items = nullptr;  // points into the batch's item buffer
    float *d_bnd = nullptr;
    int64_t bnd_stride = 0, warps = 0;
};

struct PairInfo {
    int n, m, w;
    bool trivial;
};

int64_t band_cells_exact(int64_t n, int64_t m, int64_t w)
{
    // sum over rows i = 1..n of min(m, i+w) - max(1, i-w) + 1, for n <= m,
    // m - n <= w <= m - 1 (every row meets the band)
    const int64_t a = std::min(n, std::max<int64_t>(0, m - w));
    const int64_t s1 = a * (a + 1) / 2 + a * w + (n - a) * m;
    const int64_t b = std::min(n, w);
    const int64_t s2 = b + (n > w ? (n - w) * (n - w + 1) / 2 : 0);
    return s1 - s2 + n;
}

// Length/band bucket: shapes are decided per bucket.
uint64_t bucket_of(int n, int m, int w)
{
    const int W = 2 * w + 1;
    const int wq = (int)std::floor(4.0 * std::log2((double)W));
    const int nq = (int)std::floor(2.0 * std::log2((double)n));
    const int mq = (int)std::floor(2.0 * std::log2((double)m));
    return ((uint64_t)wq << 32) | ((uint64_t)nq << 16) | (uint64_t)mq;
}

struct Family {
    int kind, K;  // kind 0 rotated (G chosen per pair), 1 strip
};

bool rotated_fits(int W, int K, int &G, int &MT)
{
    G = 2;
    while (G * K < W && G < 32) G *= 2;
    if (G * K < W) return false;
    MT = rot_masked_tail(K, G, W);
    return rot_shape_compiled(K, MT, true);
}

// Right padding of every staged series of a batch.  It covers the reads past a
// series' end of every shape the planner can choose: the rotated kernel's
// prefetches reach G*K + K + G + 1 values (693 for G = 32, K = 20), the strips'
// 32K + 8 (520), the transposed strip's G*K (512); two-row shapes are admitted
// only while their G*2H + 2G + H + 4 fits.
constexpr int kBatchPR = 700;

// Two-row shapes on the work queue: K = 2H slots per lane, the fewest lanes G
// whose slots hold the band row, and the pair's masked tail.
bool tworow_fits(int W, int H, int &G, int &MT)
{
    G = 2;
    while (G * 2 * H < W && G < 32) G *= 2;
    if (G * 2 * H < W || tworow_pad_right(G, H) > kBatchPR) return false;
    MT = tworow_masked_tail(H, G, W);
    return tworow_queue_compiled(H, MT);
}

double family_cost(const Family &f, int n, int m, int w)
{
    if (f.kind == 1) return cost_strip(n, m, w, f.K);
    if (f.kind == 2) return cost_tstrip(n, m, w, f.K);
    int G, MT;
    if (f.kind == 3) {
        if (!tworow_fits(2 * w + 1, f.K / 2, G, MT)) return 1e300;
        return cost_tworow(n, f.K / 2, G, MT);
    }
    if (!rotated_fits(2 * w + 1, f.K, G, MT)) return 1e300;
    return cost_rotated(n, f.K, G, MT);
}

// kind 0 rotated (K slots), 1 column strip, 2 transposed strip, 3 two-row rotated (K = 2H)
const Family kFamilies[] = {{0, 4},  {0, 8},  {0, 10}, {0, 12}, {0, 13}, {0, 16}, {0, 18},
                            {0, 20}, {1, 4},  {1, 8},  {1, 16}, {2, 4},  {2, 8},  {2, 16},
                            {3, 12}, {3, 16}, {3, 20}, {3, 24}, {3, 26}, {3, 32}};

// The class of a pair under family f: kind 0 rotated band (K, G, masked tail),
// 1 column strip (K), 2 transposed strip (K, G); a family that cannot hold the
// pair falls back to the strip of K = 8.
ClassKey class_key(const Family &f, int n, int w)
{
    int G = 0, MT = 0;
    if (f.kind == 0 && rotated_fits(2 * w + 1, f.K, G, MT)) return ClassKey{0, f.K, G, MT};
    if (f.kind == 3 && tworow_fits(2 * w + 1, f.K / 2, G, MT)) return ClassKey{3, f.K, G, MT};
    if (f.kind == 2 && (G = tstrip_lanes(n, f.K)) > 0) return ClassKey{2, f.K, G, 0};
    if (f.kind == 1) return ClassKey{1, f.K, 32, 0};
    return ClassKey{1, 8, 32, 0};
}

// DTWGB_BATCH_FAMILY ("rot:K", "strip:K" or "tstrip:K") forces one family for
// every bucket, for tests and measurement.
bool forced_family(Family &out)
{
    const char *e = getenv("DTWGB_BATCH_FAMILY");
    if (!e || !*e) return false;
    int K = 0;
    if (sscanf(e, "tstrip:%d", &K) == 1) out = Family{2, K};
    else if (sscanf(e, "two:%d", &K) == 1) out = Family{3, 2 * K};
    else if (sscanf(e, "strip:%d", &K) == 1) out = Family{1, K};
    else if (sscanf(e, "rot:%d", &K) == 1) out = Family{0, K};
    else return false;
    for (const Family &f : kFamilies)
        if (f.kind == out.kind && f.K == out.K) return true;
    return false;
}

// Autotune results: (device, bucket) -> family, kept for the process and, if
// DTWGB_TUNE_CACHE names a file, in that file as JSON lines.
std::mutex g_tune_mu;
std::map<std::pair<std::string, uint64_t>, Family> g_tune;
bool g_tune_loaded = false;

std::string device_key()
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    char buf[300];
    snprintf(buf, sizeof(buf), "%s/sm%d%d/%d", prop.name, prop.major, prop.minor,
             prop.multiProcessorCount);
    return buf;
}

void tune_cache_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("DTWGB_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof(line), f)) {
        char dev[300];
        unsigned long long bucket = 0;
        int kind = 0, K = 0;
        if (sscanf(line, "{\"device\": \"%299[^\"]\", \"bucket\": %llu, \"kind\": %d, \"K\": %d}", dev,
                   &bucket, &kind, &K) == 4)
            g_tune[{std::string(dev), (uint64_t)bucket}] = Family{kind, K};
    }
    fclose(f);
}

void tune_cache_store(const std::string &dev, uint64_t bucket, const Family &f)
{
    g_tune[{dev, bucket}] = f;
    const char *path = getenv("DTWGB_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *fp = fopen(path, "a");
    if (!fp) return;
    fprintf(fp, "{\"device\": \"%s\", \"bucket\": %llu, \"kind\": %d, \"K\": %d}\n", dev.c_str(),
            (unsigned long long)bucket, f.kind, f.K);
    fclose(fp);
}

}  // namespace
}  // namespace dtwgb

using namespace dtwgb;

struct dtw_batch {
    int device = 0;
    uint32_t flags = 0;
    std::vector<dtw_job> jobs;
    std::vector<BandArgs> args;      // per job, device pointers filled in
    std::vector<int64_t> pad_base;   // per job: index of its staged set in d_padded
    std::vector<int64_t> qpad_base;  // per job: index of its staged query (or -1)
    int32_t PL = 0, PR = 0;
    std::vector<ClassPlan> classes;
    BandArgs *d_jobs = nullptr;
    float *d_padded = nullptr;
    uint64_t *d_items = nullptr;
    unsigned long long *d_heads = nullptr;
    float *d_bnd = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;  // ev[0] fork, ev[1..] joins
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t pairs = 0, cells = 0;
    int buckets_tuned = 0;
    // DTW_BATCH_POOLED: device buffers from the stream-ordered pool on pool_stream,
    // every class on the run's stream, released stream-ordered (no device sync)
    bool pooled = false;
    cudaStream_t pool_stream = nullptr;
};

namespace {

// Launch every class and the job epilogues on `st` (side streams for classes
// 1.., joined back into `st`).
int enqueue(dtw_batch *b, cudaStream_t st)
{
    const int nc = (int)b->classes.size();
    DTWGB_CUDA(cudaMemsetAsync(b->d_heads, 0, sizeof(unsigned long long) * (nc > 0 ? nc : 1), st));
    for (size_t j = 0; j < b->jobs.size(); ++j) {
        const dtw_job &J = b->jobs[j];
        int rc = launch_stage_set(J.values, J.offsets, J.p, b->PL, b->PR,
                                  b->d_padded + b->pad_base[j], st);
        if (rc) return rc;
        if (J.query) {
            rc = launch_stage_one(J.query, J.qlen, b->PL, b->PR, b->d_padded + b->qpad_base[j], st);
            if (rc) return rc;
        }
    }
    const bool fork = nc > 1 && !b->side.empty();  // pooled batches run every class on st
    if (fork) DTWGB_CUDA(cudaEventRecord(b->ev[0], st));
    for (int c = 0; c < nc; ++c) {
        const ClassPlan &C = b->classes[c];
        cudaStream_t s = st;
        if (c > 0 && fork) {
            s = b->side[(c - 1) % b->side.size()];
            DTWGB_CUDA(cudaStreamWaitEvent(s, b->ev[0], 0));
        }
        QueueSrc src;
        src.jobs = b->d_jobs;
        src.items = C.d_items;
        src.n_items = (int64_t)C.items.size();
        src.head = b->d_heads + c;
        src.G = C.key.G;
        src.log2G = 0;
        while ((1 << src.log2G) < src.G) ++src.log2G;
        int rc = C.key.kind == 0   ? launch_band1_queue(src, C.key.K, C.key.MT, s)
                 : C.key.kind == 2 ? launch_tstrip_queue(src, C.key.K, s)
                 : C.key.kind == 3 ? launch_tworow_queue(src, C.key.K / 2, C.key.MT, s)
                                   : launch_strip_queue(src, C.key.K, C.d_bnd, C.bnd_stride, C.warps, s);
        if (rc) return rc;
        if (c > 0 && fork) {
            DTWGB_CUDA(cudaEventRecord(b->ev[c], s));
            DTWGB_CUDA(cudaStreamWaitEvent(st, b->ev[c], 0));
        }
    }
    for (size_t j = 0; j < b->jobs.size(); ++j) {
        const dtw_job &J = b->jobs[j];
        if (!J.query && !(J.flags & DTW_OUT_PACKED_UPPER)) {
            int rc = launch_zero_diagonal(J.out, J.p, st);
            if (rc) return rc;
        }
    }
    return DTW_OK;
}

void release(dtw_batch *b)
{
    if (!b) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(b->device);
    if (b->pooled) {  // stream-ordered: after every run enqueued on pool_stream
        for (void *q : {(void *)b->d_jobs, (void *)b->d_padded, (void *)b->d_items,
                        (void *)b->d_heads, (void *)b->d_bnd})
            scratch_free(q, b->pool_stream);
        for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
        cudaSetDevice(cur);
        delete b;
        return;
    }
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaStream_t s : b->side) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    cudaFree(b->d_jobs);
    cudaFree(b->d_padded);
    cudaFree(b->d_items);
    cudaFree(b->d_heads);
    cudaFree(b->d_bnd);
    cudaSetDevice(cur);
    delete b;
}

int validate_job(const dtw_job &J, int idx)
{
    if (J.p < 1) { set_error("job %d: p = %d must be >= 1", idx, J.p); return DTW_EINVAL; }
    if (!J.values || !J.offsets || !J.offsets_host || !J.out) {
        set_error("job %d: NULL pointer argument", idx);
        return DTW_EINVAL;
    }
    if (J.query && J.qlen < 1) { set_error("job %d: qlen = %d must be >= 1", idx, J.qlen); return DTW_EINVAL; }
    if (J.offsets_host[0] < 0) { set_error("job %d: negative offsets[0]", idx); return DTW_EINVAL; }
    for (int32_t i = 0; i < J.p; ++i) {
        const int64_t len = J.offsets_host[i + 1] - J.offsets_host[i];
        if (len <= 0 || len > INT32_MAX / 4) {
            set_error("job %d: series %d is empty, too long or offsets decrease", idx, i);
            return DTW_EINVAL;
        }
    }
    return DTW_OK;
}

PairInfo pair_info(const dtw_job &J, int64_t la, int64_t lb)
{
    PairInfo P;
    P.n = (int)std::min(la, lb);
    P.m = (int)std::max(la, lb);
    const int diff = P.m - P.n;
    const int wb = J.window_permille > 0 ? (int)((int64_t)J.window_permille * P.m / 1000) : J.window;
    int w;
    if (wb < 0) w = P.m - 1;
    else if (J.flags & DTW_BAND_STRICT) w = wb;
    else w = std::max(wb, diff);
    if (w > P.m - 1) w = P.m - 1;
    P.w = w;
    P.trivial = diff > w;
    return P;
}

// Time one family on a sample of items (all exact classes of the sample,
// launched one after another); returns milliseconds or a negative code.
double time_family(dtw_batch *b, const Family &f, const std::vector<uint64_t> &sample,
                   const std::vector<PairInfo> &info, uint64_t *d_tmp, unsigned long long *d_head,
                   float *d_bnd, int64_t bnd_elems, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1)
{
    std::map<ClassKey, std::vector<uint64_t>> byclass;
    for (size_t i = 0; i < sample.size(); ++i) {
        const PairInfo &P = info[i];
        byclass[class_key(f, P.n, P.w)].push_back(sample[i]);
    }
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
        if (cudaEventRecord(e0, st) != cudaSuccess) return -1;
        for (auto &kv : byclass) {
            if (cudaMemcpyAsync(d_tmp, kv.second.data(), kv.second.size() * sizeof(uint64_t),
                                cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemsetAsync(d_head, 0, sizeof(unsigned long long), st) != cudaSuccess)
                return -1;
            QueueSrc src{b->d_jobs, d_tmp, (int64_t)kv.second.size(), d_head, kv.first.G, 0};
            while ((1 << src.log2G) < src.G) ++src.log2G;
            int rc;
            if (kv.first.kind == 0) {
                rc = launch_band1_queue(src, kv.first.K, kv.first.MT, st);
            } else if (kv.first.kind == 3) {
                rc = launch_tworow_queue(src, kv.first.K / 2, kv.first.MT, st);
            } else if (kv.first.kind == 2) {
                rc = launch_tstrip_queue(src, kv.first.K, st);
            } else {
                int64_t warps = 0;
                if ((rc = strip_warps(kv.first.K, src.n_items, &warps))) return -1;
                int maxlen = 0;
                for (size_t i = 0; i < sample.size(); ++i) maxlen = std::max(maxlen, info[i].n);
                const int64_t stride = strip_bnd_stride(maxlen);
                if (stride * warps > bnd_elems) warps = bnd_elems / stride / 8 * 8;
                if (warps < 8) return -1;
                rc = launch_strip_queue(src, kv.first.K, d_bnd, stride, warps, st);
            }
            if (rc) return -1;
        }
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
            return -1;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);  // first repetition warms up
    }
    return best;
}

}  // namespace

extern "C" int dtw_batch_create(const dtw_job *jobs, int32_t njobs, uint32_t flags, void *stream,
                                dtw_batch **out)
{
    clear_error();
    if (!out) { set_error("NULL out"); return DTW_EINVAL; }
    *out = nullptr;
    if (njobs < 1 || !jobs) { set_error("njobs = %d must be >= 1", njobs); return DTW_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    for (int32_t j = 0; j < njobs; ++j) {
        int rc = validate_job(jobs[j], j);
        if (rc) return rc;
    }
    if ((flags & DTW_BATCH_POOLED) && (flags & (DTW_BATCH_GRAPH | DTW_BATCH_AUTOTUNE))) {
        set_error("DTW_BATCH_POOLED excludes DTW_BATCH_GRAPH and DTW_BATCH_AUTOTUNE");
        return DTW_EINVAL;
    }
    dtw_batch *b = new dtw_batch();
    b->flags = flags;
    b->pooled = (flags & DTW_BATCH_POOLED) != 0;
    b->pool_stream = st;
    cudaGetDevice(&b->device);
    b->jobs.assign(jobs, jobs + njobs);
    auto fail = [&](int rc) {
        release(b);
        return rc;
    };

    // ---- enumerate pairs, their bands and buckets
    std::vector<uint64_t> items;
    std::vector<PairInfo> infos;
    int64_t total_pairs = 0;
    for (const dtw_job &J : b->jobs)
        total_pairs += J.query ? J.p : (int64_t)J.p * (J.p - 1) / 2;
    if (total_pairs >= (1ll << kItemShift)) { set_error("too many pairs in one job"); return fail(DTW_EINVAL); }
    items.reserve(total_pairs);
    infos.reserve(total_pairs);
    int wmax = 0, maxlen = 1;
    for (int32_t j = 0; j < njobs; ++j) {
        const dtw_job &J = b->jobs[j];
        const int64_t *o = J.offsets_host;
        for (int32_t i = 0; i < J.p; ++i) maxlen = std::max<int>(maxlen, (int)(o[i + 1] - o[i]));
        if (J.query) maxlen = std::max(maxlen, J.qlen);
        const uint64_t jb = (uint64_t)j << kItemShift;
        if (J.query) {
            for (int32_t t = 0; t < J.p; ++t) {
                infos.push_back(pair_info(J, J.qlen, o[t + 1] - o[t]));
                items.push_back(jb | (uint64_t)t);
            }
        } else {
            uint64_t t = 0;
            for (int32_t a = 0; a + 1 < J.p; ++a)
                for (int32_t c = a + 1; c < J.p; ++c, ++t) {
                    infos.push_back(pair_info(J, o[a + 1] - o[a], o[c + 1] - o[c]));
                    items.push_back(jb | t);
                }
        }
    }
    for (const PairInfo &P : infos)
        if (!P.trivial) wmax = std::max(wmax, P.w);

    // ---- shape family per bucket: model, or the autotuner / its cache
    std::map<uint64_t, std::vector<size_t>> buckets;
    for (size_t i = 0; i < infos.size(); ++i)
        if (!infos[i].trivial) buckets[bucket_of(infos[i].n, infos[i].m, infos[i].w)].push_back(i);
    std::map<uint64_t, Family> choice;
    Family forced_f{1, 8};
    const bool forced = forced_family(forced_f);
    double total_cost = 0.0;
    std::map<uint64_t, double> bucket_cost;
    for (auto &kv : buckets) {
        const PairInfo &R = infos[kv.second[kv.second.size() / 2]];  // a representative pair
        double best = 1e300;
        Family bf{1, 8};
        for (const Family &f : kFamilies) {
            const double c = family_cost(f, R.n, R.m, R.w);
            if (c < best) { best = c; bf = f; }
        }
        if (forced) {
            bf = forced_f;
            best = std::min(best, family_cost(bf, R.n, R.m, R.w));
        }
        choice[kv.first] = bf;
        bucket_cost[kv.first] = best * kv.second.size();
        total_cost += best * kv.second.size();
    }

    // ---- device state: job table, padded series, queue heads
    // pads for every family (see kBatchPR); on the left the band's first y window and
    // the two-row kernel's ramp rows (x down to 2 - 2G)
    b->PL = std::max(wmax, 64) + 2;
    b->PR = kBatchPR;
    const int64_t pad = b->PL + b->PR;
    int64_t elems = 0;
    b->pad_base.resize(njobs);
    b->qpad_base.assign(njobs, -1);
    for (int32_t j = 0; j < njobs; ++j) {
        const dtw_job &J = b->jobs[j];
        b->pad_base[j] = elems;
        elems += (J.offsets_host[J.p] - J.offsets_host[0]) + (int64_t)J.p * pad;
        if (J.query) {
            b->qpad_base[j] = elems;
            elems += J.qlen + pad;
        }
    }
    // device buffers: plain allocations for a batch that is run many times, the
    // stream-ordered pool for a pooled one
    auto dev_alloc = [&](void **p, size_t bytes) -> bool {
        if (b->pooled) return scratch_alloc(p, bytes, st) == DTW_OK;
        return cudaMalloc(p, bytes) == cudaSuccess;
    };
    auto h2d = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
        return b->pooled ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st)
                         : cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    if (!dev_alloc((void **)&b->d_padded, sizeof(float) * (size_t)std::max<int64_t>(elems, 1)) ||
        !dev_alloc((void **)&b->d_jobs, sizeof(BandArgs) * (size_t)njobs)) {
        set_error("device allocation for the batch failed");
        return fail(DTW_ENOMEM);
    }
    b->args.resize(njobs);
    for (int32_t j = 0; j < njobs; ++j) {
        const dtw_job &J = b->jobs[j];
        BandArgs A{};
        A.padded = b->d_padded + b->pad_base[j];
        A.offsets = J.offsets;
        A.qbase = J.query ? (b->qpad_base[j] - b->pad_base[j]) + b->PL : 0;
        A.qlen = J.query ? J.qlen : 0;
        A.p = J.p;
        A.n_pairs = J.query ? J.p : (int64_t)J.p * (J.p - 1) / 2;
        A.window = J.window;
        A.wpermille = J.window_permille;
        A.strict = (J.flags & DTW_BAND_STRICT) ? 1 : 0;
        A.src = J.query ? SRC_QUERY : SRC_TRIANGLE;
        A.out_mode = J.query ? OUT_ROW : ((J.flags & DTW_OUT_PACKED_UPPER) ? OUT_PACKED : OUT_FULL);
        A.out = J.out;
        A.G = 32;
        A.log2G = 5;
        A.PL = b->PL;
        A.PR = b->PR;
        b->args[j] = A;
    }
    DTWGB_CUDA(h2d(b->d_jobs, b->args.data(), sizeof(BandArgs) * (size_t)njobs));

    // ---- autotune the buckets that carry the work
    if (flags & DTW_BATCH_AUTOTUNE) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache_load();
        const std::string dev = device_key();
        for (int32_t j = 0; j < njobs; ++j) {  // staged data for the timing runs
            const dtw_job &J = b->jobs[j];
            int rc = launch_stage_set(J.values, J.offsets, J.p, b->PL, b->PR,
                                      b->d_padded + b->pad_base[j], st);
            if (!rc && J.query)
                rc = launch_stage_one(J.query, J.qlen, b->PL, b->PR, b->d_padded + b->qpad_base[j], st);
            if (rc) return fail(rc);
        }
        const size_t kSample = 1024, kFill = 16384;
        uint64_t *d_tmp = nullptr;
        unsigned long long *d_head = nullptr;
        float *d_bnd = nullptr;
        const int64_t bnd_elems = strip_bnd_stride(maxlen) * 152 * 8 * 4;
        cudaEvent_t e0, e1;
        if (cudaMalloc(&d_tmp, kFill * 2 * sizeof(uint64_t)) != cudaSuccess ||
            cudaMalloc(&d_head, sizeof(unsigned long long)) != cudaSuccess ||
            cudaMalloc(&d_bnd, sizeof(float) * (size_t)bnd_elems) != cudaSuccess ||
            cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            cudaFree(d_tmp);
            cudaFree(d_head);
            cudaFree(d_bnd);
            set_error("autotuner allocation failed");
            return fail(DTW_ENOMEM);
        }
        for (auto &kv : buckets) {
            if (bucket_cost[kv.first] < 0.002 * total_cost) continue;  // too little work to matter
            auto hit = g_tune.find({dev, kv.first});
            if (hit != g_tune.end()) {
                choice[kv.first] = hit->second;
                continue;
            }
            // candidates: the model's three cheapest families
            const PairInfo &R = infos[kv.second[kv.second.size() / 2]];
            std::vector<std::pair<double, Family>> cands;
            for (const Family &f : kFamilies) {
                const double c = family_cost(f, R.n, R.m, R.w);
                if (c < 1e299) cands.push_back({c, f});
            }
            std::sort(cands.begin(), cands.end(),
                      [](const std::pair<double, Family> &x, const std::pair<double, Family> &y) {
                          return x.first < y.first;
                      });
            if (cands.size() > 3) cands.resize(3);
            // up to kSample distinct pairs of the bucket, repeated until the timing
            // run fills the GPU as the real run does (repeats rewrite equal values)
            std::vector<uint64_t> sample;
            std::vector<PairInfo> sinfo;
            const size_t step = std::max<size_t>(1, kv.second.size() / kSample);
            for (size_t q = 0; q < kv.second.size() && sample.size() < kSample; q += step) {
                sample.push_back(items[kv.second[q]]);
                sinfo.push_back(infos[kv.second[q]]);
            }
            const size_t distinct = sample.size();
            while (sample.size() < kFill) {
                sample.push_back(sample[sample.size() % distinct]);
                sinfo.push_back(sinfo[sinfo.size() % distinct]);
            }
            double best = 1e300;
            Family bf = choice[kv.first];
            for (auto &c : cands) {
                const double ms = time_family(b, c.second, sample, sinfo, d_tmp, d_head, d_bnd,
                                              bnd_elems, st, e0, e1);
                if (ms >= 0 && ms < best) { best = ms; bf = c.second; }
            }
            choice[kv.first] = bf;
            tune_cache_store(dev, kv.first, bf);
            ++b->buckets_tuned;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(d_tmp);
        cudaFree(d_head);
        cudaFree(d_bnd);
        DTWGB_CUDA(cudaStreamSynchronize(st));
    }

    // ---- classes: exact shape per pair, cost-sorted queues
    std::map<ClassKey, size_t> cls_index;
    std::vector<std::vector<std::pair<float, uint64_t>>> cls_items;
    auto class_of = [&](const ClassKey &k) {
        auto it = cls_index.find(k);
        if (it != cls_index.end()) return it->second;
        const size_t id = b->classes.size();
        cls_index[k] = id;
        b->classes.push_back(ClassPlan());
        b->classes.back().key = k;
        cls_items.emplace_back();
        return id;
    };
    for (size_t i = 0; i < infos.size(); ++i) {
        const PairInfo &P = infos[i];
        b->pairs += 1;
        if (P.trivial) continue;  // placed below, into any class
        const Family f = choice[bucket_of(P.n, P.m, P.w)];
        const ClassKey k = class_key(f, P.n, P.w);
        const size_t c = class_of(k);
        const int64_t cells = band_cells_exact(P.n, P.m, P.w);
        b->cells += cells;
        b->classes[c].cells += cells;
        if (k.kind == 1) b->classes[c].maxlen = std::max(b->classes[c].maxlen, P.n);
        const float cost = (float)(k.kind == 0   ? cost_rotated(P.n, k.K, k.G, k.MT)
                                   : k.kind == 2 ? cost_tstrip(P.n, P.m, P.w, k.K)
                                   : k.kind == 3 ? cost_tworow(P.n, k.K / 2, k.G, k.MT)
                                                 : cost_strip(P.n, P.m, P.w, k.K));
        cls_items[c].push_back({cost, items[i]});
    }
    for (size_t i = 0; i < infos.size(); ++i)
        if (infos[i].trivial) {
            const size_t c = b->classes.empty() ? class_of(ClassKey{0, 4, 2, 1}) : 0;
            cls_items[c].push_back({0.f, items[i]});
        }
    const bool sorted = !(flags & DTW_BATCH_UNSORTED);
    size_t n_items_all = 0;
    for (size_t c = 0; c < b->classes.size(); ++c) {
        auto &v = cls_items[c];
        if (sorted)
            std::stable_sort(v.begin(), v.end(),
                             [](const std::pair<float, uint64_t> &x,
                                const std::pair<float, uint64_t> &y) { return x.first > y.first; });
        b->classes[c].items.resize(v.size());
        for (size_t i = 0; i < v.size(); ++i) b->classes[c].items[i] = v[i].second;
        std::vector<std::pair<float, uint64_t>>().swap(v);
        n_items_all += b->classes[c].items.size();
    }
    std::vector<uint64_t>().swap(items);
    std::vector<PairInfo>().swap(infos);

    const int nc = (int)b->classes.size();
    if (!dev_alloc((void **)&b->d_items, sizeof(uint64_t) * std::max<size_t>(n_items_all, 1)) ||
        !dev_alloc((void **)&b->d_heads, sizeof(unsigned long long) * std::max(nc, 1))) {
        set_error("device allocation for the batch queues failed");
        return fail(DTW_ENOMEM);
    }
    size_t off = 0;
    int64_t bnd_total = 0;
    for (ClassPlan &C : b->classes) {
        C.d_items = b->d_items + off;
        DTWGB_CUDA(h2d(C.d_items, C.items.data(), sizeof(uint64_t) * C.items.size()));
        off += C.items.size();
        if (C.key.kind == 1) {
            int rc = strip_warps(C.key.K, (int64_t)C.items.size(), &C.warps);
            if (rc) return fail(rc);
            C.bnd_stride = strip_bnd_stride(C.maxlen);
            bnd_total += C.bnd_stride * C.warps;
        }
    }
    if (bnd_total > 0) {
        if (!dev_alloc((void **)&b->d_bnd, sizeof(float) * (size_t)bnd_total)) {
            set_error("device allocation for strip buffers failed");
            return fail(DTW_ENOMEM);
        }
        int64_t boff = 0;
        for (ClassPlan &C : b->classes)
            if (C.key.kind == 1) {
                C.d_bnd = b->d_bnd + boff;
                boff += C.bnd_stride * C.warps;
            }
    }
    for (int c = 1; c < nc && c <= 8 && !b->pooled; ++c) {
        cudaStream_t s;
        DTWGB_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        b->side.push_back(s);
    }
    b->ev.resize(std::max(nc, 1));
    for (auto &e : b->ev) DTWGB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));

    if (flags & DTW_BATCH_GRAPH) {
        DTWGB_CUDA(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
        DTWGB_CUDA(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeRelaxed));
        int rc = enqueue(b, b->capture_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->capture_stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return fail(rc);
        }
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamEndCapture"));
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaGraphInstantiate"));
    }
    if (!b->pooled) DTWGB_CUDA(cudaStreamSynchronize(st));
    *out = b;
    return DTW_OK;
}

extern "C" int dtw_batch_run(dtw_batch *b, void *stream)
{
    clear_error();
    if (!b) { set_error("NULL batch"); return DTW_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    if (b->exec) {
        DTWGB_CUDA(cudaGraphLaunch(b->exec, st));
        return DTW_OK;
    }
    return enqueue(b, st);
}

extern "C" int dtw_batch_run_once(const dtw_job *jobs, int32_t njobs, uint32_t flags,
                                  void *stream)
{
    clear_error();
    if (flags & ~(uint32_t)DTW_BATCH_UNSORTED) {
        set_error("dtw_batch_run_once takes DTW_BATCH_UNSORTED only");
        return DTW_EINVAL;
    }
    dtw_batch *b = nullptr;
    int rc = dtw_batch_create(jobs, njobs, flags | DTW_BATCH_POOLED, stream, &b);
    if (rc) return rc;
    rc = enqueue(b, (cudaStream_t)stream);
    release(b);  // stream-ordered frees behind the run
    return rc;
}

extern "C" int dtw_batch_get_info(const dtw_batch *b, dtw_batch_info *info)
{
    clear_error();
    if (!b || !info) { set_error("NULL argument"); return DTW_EINVAL; }
    info->pairs = b->pairs;
    info->cells = b->cells;
    info->classes = (int32_t)b->classes.size();
    info->graph = b->exec ? 1 : 0;
    info->buckets_tuned = b->buckets_tuned;
    info->jobs = (int32_t)b->jobs.size();
    return DTW_OK;
}

extern "C" int dtw_batch_get_class(const dtw_batch *b, int32_t i, int32_t *kind, int32_t *K,
                                   int32_t *G, int64_t *items, int64_t *cells)
{
    clear_error();
    if (!b || i < 0 || i >= (int32_t)b->classes.size()) {
        set_error("class index %d out of range", i);
        return DTW_EINVAL;
    }
    const ClassPlan &C = b->classes[i];
    if (kind) *kind = C.key.kind;
    if (K) *K = C.key.K;
    if (G) *G = C.key.G;
    if (items) *items = (int64_t)C.items.size();
    if (cells) *cells = C.cells;
    return DTW_OK;
}

extern "C" void dtw_batch_destroy(dtw_batch *b) { release(b); }
