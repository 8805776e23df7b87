// Served form: a request engine with continuous batching.
//
// A worker thread owns a stream on the engine's device.  Requests are queued
// by cf_engine_submit (their host arrays copied).  Each loop iteration:
//   1. admission: queued requests are admitted in arrival order while a slot
//      is free and their device state (points, poses, one chunk of domains,
//      tuples and margins) fits in the HBM budget;
//   2. a round: every active request takes its next pose chunk; all chunks go
//      through one launch per query group (same finger count, slot bits and
//      binning method), one sampling launch and one launch per score group
//      (same k, K), exactly as a cf_batch does;
//   3. results: a compaction kernel gathers every request's accepted tuples
//      (pose, margin, point ids), in tuple order, into one contiguous run per
//      request; two copies bring the runs' extents and the runs themselves
//      back into page-locked memory, and they are appended to the requests; a
//      request that reached its grasp count or ran out of poses completes,
//      frees its device state and its slot, and the next round admits whoever
//      is waiting.
// Request arrays are copied at submission into page-locked blocks from a pool
// the engine keeps, so admission uploads are plain DMA.
// Tuple draws use the request's seed and the GLOBAL pose index (pose_base), so
// a request's result is independent of the rounds it shares.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "cf_internal.cuh"

using namespace cf;

namespace {

struct EngReq {
    uint64_t id = 0;
    cf_request req{};
    const cf_field *fd = nullptr;
    float *h_in = nullptr;  // page-locked: soa [6][n] then poses [n_poses][12]
    size_t h_in_bytes = 0;
    int limit = 0;  // poses this request may use
    int cap = 0;    // poses its device state holds (the largest chunk it may take)
    // device state
    void *d_block = nullptr;
    size_t bytes = 0;
    float *d_soa = nullptr, *d_poses = nullptr, *d_margin = nullptr;
    uint32_t *d_masks = nullptr, *d_counts = nullptr;
    int32_t *d_tuples = nullptr;
    uint8_t *d_fingers = nullptr, *d_accept = nullptr;
    // progress
    int pose_next = 0, chunk = 0;
    unsigned rec_off = 0, rec_cnt = 0;  // this round's accepted records in the engine's host buffer
    std::vector<int32_t> res_pose, res_tuples;
    std::vector<float> res_margin;
    double t_submit = 0, t_admit = 0, t_first_round = -1;
    int n_rounds = 0;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Page-locked host blocks in power-of-two size classes (>= 64 KiB), reused
// across requests.
struct PinnedPool {
    std::mutex mu;
    std::multimap<size_t, void *> free_blocks;
    std::vector<std::pair<void *, size_t>> all;
    static size_t size_class(size_t b) {
        size_t c = (size_t)1 << 16;
        while (c < b) c <<= 1;
        return c;
    }
    // allocates on `dev` without changing the calling thread's current device
    void *get(size_t bytes, int dev, size_t *cap) {
        const size_t c = size_class(bytes);
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = free_blocks.find(c);
            if (it != free_blocks.end()) {
                void *p = it->second;
                free_blocks.erase(it);
                *cap = c;
                return p;
            }
        }
        int old = 0;
        if (cudaGetDevice(&old) != cudaSuccess) return nullptr;
        void *p = nullptr;
        const bool sw = old != dev && cudaSetDevice(dev) == cudaSuccess;
        const cudaError_t err = cudaHostAlloc(&p, c, cudaHostAllocPortable);
        if (sw) cudaSetDevice(old);
        if (err != cudaSuccess) return nullptr;
        std::lock_guard<std::mutex> lk(mu);
        all.emplace_back(p, c);
        *cap = c;
        return p;
    }
    void put(void *p, size_t cap) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu);
        free_blocks.emplace(cap, p);
    }
    ~PinnedPool() {
        for (auto &b : all) cudaFreeHost(b.first);
    }
};

// One accepted tuple as the engine returns it.
struct AccRecord {
    int32_t pose;
    float margin;
    int32_t t[CF_MAX_K];
};

struct CompactDesc {
    const uint8_t *accept;
    const int32_t *tuples;
    const float *margin;
    int nt, T, k, pose_base;
};

constexpr int kCompactThreads = 256;
constexpr int kCompactWarps = kCompactThreads / 32;

// Block i gathers request i's accepted tuples, in tuple order, into one
// contiguous run of `out`: the run's start is reserved with one atomic on the
// round's cursor; the start and length are reported in off[i] / cnt[i].
__global__ void __launch_bounds__(kCompactThreads) k_compact_accepted(const CompactDesc *descs, AccRecord *out,
                                                                     unsigned *cursor, unsigned *off,
                                                                     unsigned *cnt) {
    __shared__ unsigned s_warp[kCompactWarps];
    __shared__ unsigned s_base;
    const CompactDesc d = descs[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned c = 0;
    for (int u = threadIdx.x; u < d.nt; u += kCompactThreads) c += d.accept[u] != 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) s_warp[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
        for (int w = 0; w < kCompactWarps; ++w) tot += s_warp[w];
        s_base = atomicAdd(cursor, tot);
        off[blockIdx.x] = s_base;
        cnt[blockIdx.x] = tot;
    }
    __syncthreads();
    unsigned run = s_base;
    for (int t0 = 0; t0 < d.nt; t0 += kCompactThreads) {
        const int u = t0 + threadIdx.x;
        const bool a = u < d.nt && d.accept[u] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, a);
        __syncthreads();  // the previous tile's counts have been read
        if (lane == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        unsigned before = 0, tile = 0;
        for (int w = 0; w < kCompactWarps; ++w) {
            const unsigned x = s_warp[w];
            before += w < warp ? x : 0u;
            tile += x;
        }
        if (a) {
            AccRecord r;
            r.pose = d.pose_base + u / d.T;
            r.margin = d.margin[u];
#pragma unroll
            for (int q = 0; q < CF_MAX_K; ++q) r.t[q] = q < d.k ? d.tuples[(size_t)u * d.k + q] : -1;
            out[run + before + __popc(bal & ((1u << lane) - 1u))] = r;
        }
        run += tile;
    }
}

size_t state_bytes(const cf_request &r, int F, int chunk) {
    const size_t W = (size_t)(r.n + 31) / 32, T = r.prm.n_tuples, k = r.prm.k;
    return align256(sizeof(float) * 6 * r.n) + align256(sizeof(float) * 12 * (size_t)r.n_poses) +
           align256(sizeof(uint32_t) * chunk * F * W) + align256(sizeof(uint32_t) * chunk * F) +
           align256(sizeof(int32_t) * chunk * T * k) + align256(chunk * T * k) + align256(sizeof(float) * chunk * T) +
           align256(chunk * T);
}

}  // namespace

struct cf_engine {
    cf_engine_params prm{};
    std::vector<const cf_field *> fields;
    std::vector<FieldGeom> geoms;
    int dev = 0;
    cudaStream_t st = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv, cv_idle;
    bool stop = false;
    std::deque<EngReq *> queue;
    std::vector<EngReq *> active;
    std::deque<cf_result> done;
    uint64_t next_id = 1;
    cf_engine_stats stats{};
    std::chrono::steady_clock::time_point t0;
    // round scratch (device): geoms | query descs | score descs | all descs | prefixes | counters |
    // compaction descs | cursor, offsets, counts
    void *d_round = nullptr;
    size_t round_bytes = 0;
    void *d_rec = nullptr;  // accepted records of a round (capacity: every tuple of the round)
    size_t rec_bytes = 0;
    AccRecord *h_rec = nullptr;  // page-locked copy of the used part
    size_t h_rec_bytes = 0;
    unsigned *h_meta = nullptr;  // page-locked: cursor, offsets [n], counts [n]
    size_t h_meta_bytes = 0;
    PinnedPool pinned;
    std::string worker_error;
    Tuning tune{4, 8, 0};  // launch shapes (the tuning at creation)

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void finish(cf_engine *e, EngReq *r, int status, bool partial) {
    cf_result res;
    memset(&res, 0, sizeof res);
    res.id = r->id;
    res.tag = r->req.tag;
    res.status = status;
    res.partial = partial ? 1 : 0;
    res.k = r->req.prm.k;
    res.n_accepted = (int32_t)r->res_margin.size();
    res.n_poses_used = r->pose_next;
    res.t_submit = r->t_submit;
    res.t_admit = r->t_admit;
    res.t_done = e->now();
    res.n_rounds = r->n_rounds;
    res.t_first_round = r->t_first_round >= 0 ? r->t_first_round : res.t_done;
    if (res.n_accepted > 0) {
        res.pose = (int32_t *)malloc(sizeof(int32_t) * res.n_accepted);
        res.tuples = (int32_t *)malloc(sizeof(int32_t) * res.n_accepted * res.k);
        res.margin = (float *)malloc(sizeof(float) * res.n_accepted);
        memcpy(res.pose, r->res_pose.data(), sizeof(int32_t) * res.n_accepted);
        memcpy(res.tuples, r->res_tuples.data(), sizeof(int32_t) * res.n_accepted * res.k);
        memcpy(res.margin, r->res_margin.data(), sizeof(float) * res.n_accepted);
    }
    if (r->d_block) cudaFreeAsync(r->d_block, e->st);
    e->pinned.put(r->h_in, r->h_in_bytes);  // its upload was followed by a stream wait
    std::lock_guard<std::mutex> lk(e->mu);
    if (r->d_block) e->stats.bytes_in_use -= (int64_t)r->bytes;
    e->done.push_back(res);
    e->stats.completed++;
    delete r;
}

// Allocate a request's device state and upload its points and poses.
int admit_one(cf_engine *e, EngReq *r) {
    const int F = r->fd->F;
    const cf_request &q = r->req;
    int rc = pool_alloc(&r->d_block, r->bytes, e->st, "alloc request");
    if (rc) return rc;
    char *p = (char *)r->d_block;
    const size_t W = (size_t)(q.n + 31) / 32, T = q.prm.n_tuples, k = q.prm.k, c = (size_t)r->cap;
    r->d_soa = (float *)p; p += align256(sizeof(float) * 6 * q.n);
    r->d_poses = (float *)p; p += align256(sizeof(float) * 12 * (size_t)q.n_poses);
    r->d_masks = (uint32_t *)p; p += align256(sizeof(uint32_t) * c * F * W);
    r->d_counts = (uint32_t *)p; p += align256(sizeof(uint32_t) * c * F);
    r->d_tuples = (int32_t *)p; p += align256(sizeof(int32_t) * c * T * k);
    r->d_fingers = (uint8_t *)p; p += align256(c * T * k);
    r->d_margin = (float *)p; p += align256(sizeof(float) * c * T);
    r->d_accept = (uint8_t *)p;
    if (q.n > 0) CF_TRY(cudaMemcpyAsync(r->d_soa, r->h_in, sizeof(float) * 6 * q.n, cudaMemcpyHostToDevice, e->st),
                        "upload points");
    if (q.n_poses > 0)
        CF_TRY(cudaMemcpyAsync(r->d_poses, r->h_in + 6 * (size_t)q.n, sizeof(float) * 12 * (size_t)q.n_poses,
                               cudaMemcpyHostToDevice, e->st), "upload poses");
    return CF_OK;
}

// The poses a request takes this round: pose_chunk, or, with adaptive chunks after its first
// round, the poses its acceptance so far says it still needs (25 % to spare; twice its last
// chunk while it has accepted nothing), at most chunk_pairs_max / n of them, kept between
// pose_chunk and its capacity.  Depends only on the request's own progress.
int next_chunk(const cf_engine *e, const EngReq *r) {
    const int left = r->limit - r->pose_next;
    long long c = e->prm.pose_chunk;
    if (r->pose_next > 0 && r->cap > e->prm.pose_chunk) {
        const long long got = (long long)r->res_margin.size(), need = (long long)r->req.n_grasps - got;
        if (got > 0)
            c = (long long)ceil(1.25 * (double)need * (double)r->pose_next / (double)got);
        else
            c = 2LL * r->chunk;
        if (e->prm.chunk_pairs_max > 0) c = std::min<long long>(c, e->prm.chunk_pairs_max / std::max(1, r->req.n));
        c = std::max<long long>(c, e->prm.pose_chunk);
    }
    return (int)std::max<long long>(1, std::min<long long>({c, (long long)r->cap, (long long)left}));
}

// One round over the active requests.  Returns CF_OK or an error code.
int run_round(cf_engine *e, std::vector<EngReq *> &act) {
    const int n = (int)act.size();
    const double t_start = e->now();
    for (EngReq *r : act) {
        if (r->t_first_round < 0) r->t_first_round = t_start;
        ++r->n_rounds;
    }
    std::vector<ScoreArgs> sargs(n);
    std::vector<cf_points> objs(n);
    for (int i = 0; i < n; ++i) {
        EngReq *r = act[i];
        const cf_request &q = r->req;
        r->chunk = next_chunk(e, r);
        objs[i] = cf_points{r->d_soa, r->d_soa + q.n, r->d_soa + 2 * q.n, r->d_soa + 3 * q.n, r->d_soa + 4 * q.n,
                            r->d_soa + 5 * q.n, q.n};
        int rc = fill_score_args(&objs[i], r->fd->F, r->d_masks, r->d_counts, r->chunk, &q.prm, r->d_tuples,
                                 r->d_fingers, r->d_margin, r->d_accept, &sargs[i]);
        if (rc) return rc;
        sargs[i].pose_base = (uint32_t)r->pose_next;
        sargs[i].refill = e->tune.score_refill;
        sargs[i].bpsm = e->tune.score_bpsm;
    }
    auto geom_of = [&](int i) {
        for (size_t f = 0; f < e->fields.size(); ++f)
            if (e->fields[f] == act[i]->fd) return (int)f;
        return 0;
    };
    std::vector<int> skeys;
    for (int i = 0; i < n; ++i) {
        const int sk = sargs[i].k * 100 + sargs[i].K;
        if (std::find(skeys.begin(), skeys.end(), sk) == skeys.end()) skeys.push_back(sk);
    }
    // every request's query chunk in one persistent launch (any hand)
    std::vector<QueryDesc> qd;
    int q_items = 0;
    for (int i = 0; i < n; ++i) {
        QueryDesc d;
        memset(&d, 0, sizeof d);
        d.obj = objs[i];
        d.poses = act[i]->d_poses + 12 * (size_t)act[i]->pose_next;
        d.P = act[i]->chunk;
        d.W = (objs[i].n + 31) / 32;
        d.masks = act[i]->d_masks;
        d.counts = act[i]->d_counts;
        d.table = act[i]->fd->d_table;
        d.geom = geom_of(i);
        d.block0 = q_items;
        q_items += query_blocks(d.P, e->tune.query_ppb);
        qd.push_back(d);
    }
    std::vector<ScoreArgs> sd;
    std::vector<long long> t0, pose0(n + 1, 0);
    std::vector<int> s_off, t_off, s_n;
    std::vector<long long> s_tuples;
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
        pose0[i + 1] = pose0[i] + act[i]->chunk;
        smem = std::max(smem, score_smem_bytes(sargs[i].F, sargs[i].W, sargs[i].T, sargs[i].k, true));
    }
    for (int key : skeys) {
        s_off.push_back((int)sd.size());
        t_off.push_back((int)t0.size());
        long long tuples = 0;
        for (int i = 0; i < n; ++i) {
            if (sargs[i].k * 100 + sargs[i].K != key) continue;
            t0.push_back(tuples);
            tuples += (long long)sargs[i].P * sargs[i].T;
            sd.push_back(sargs[i]);
        }
        t0.push_back(tuples);
        s_n.push_back((int)sd.size() - s_off.back());
        s_tuples.push_back(tuples);
    }
    // upload descriptors
    const size_t o_g = 0, o_q = align256(sizeof(FieldGeom) * e->geoms.size());
    const size_t o_s = align256(o_q + sizeof(QueryDesc) * qd.size());
    const size_t o_a = align256(o_s + sizeof(ScoreArgs) * sd.size());
    const size_t o_p = align256(o_a + sizeof(ScoreArgs) * n);
    const size_t o_t = align256(o_p + sizeof(long long) * pose0.size());
    const size_t o_w = align256(o_t + sizeof(long long) * t0.size());
    const size_t o_c = align256(o_w + 2 * sizeof(unsigned int));  // the query's item counter, zero
    const size_t o_m = align256(o_c + sizeof(CompactDesc) * n);
    const size_t meta_bytes = sizeof(unsigned) * (1 + 2 * (size_t)n);  // cursor, offsets, counts
    const size_t total = align256(o_m + meta_bytes);
    std::vector<CompactDesc> cd(n);
    size_t rec_need = 0;
    for (int i = 0; i < n; ++i) {
        EngReq *r = act[i];
        const int T = r->req.prm.n_tuples;
        cd[i] = CompactDesc{r->d_accept, r->d_tuples, r->d_margin, r->chunk * T, T, r->req.prm.k, r->pose_next};
        rec_need += (size_t)r->chunk * T;
    }
    rec_need *= sizeof(AccRecord);
    if (rec_need > e->rec_bytes) {
        if (e->d_rec) cudaFreeAsync(e->d_rec, e->st);
        e->d_rec = nullptr;
        e->rec_bytes = 0;
        int rc = pool_alloc(&e->d_rec, 2 * rec_need, e->st, "alloc round records");
        if (rc) return rc;
        e->rec_bytes = 2 * rec_need;
    }
    if (meta_bytes > e->h_meta_bytes) {
        if (e->h_meta) cudaFreeHost(e->h_meta);
        e->h_meta = nullptr;
        e->h_meta_bytes = 0;
        CF_TRY(cudaHostAlloc((void **)&e->h_meta, 2 * meta_bytes, cudaHostAllocDefault), "alloc round meta");
        e->h_meta_bytes = 2 * meta_bytes;
    }
    if (total > e->round_bytes) {
        if (e->d_round) cudaFreeAsync(e->d_round, e->st);
        e->d_round = nullptr;
        int rc = pool_alloc(&e->d_round, 2 * total, e->st, "alloc round");
        if (rc) return rc;
        e->round_bytes = 2 * total;
    }
    std::vector<char> img(total, 0);
    memcpy(img.data() + o_g, e->geoms.data(), sizeof(FieldGeom) * e->geoms.size());
    memcpy(img.data() + o_q, qd.data(), sizeof(QueryDesc) * qd.size());
    memcpy(img.data() + o_s, sd.data(), sizeof(ScoreArgs) * sd.size());
    memcpy(img.data() + o_a, sargs.data(), sizeof(ScoreArgs) * n);
    memcpy(img.data() + o_p, pose0.data(), sizeof(long long) * pose0.size());
    memcpy(img.data() + o_t, t0.data(), sizeof(long long) * t0.size());
    memcpy(img.data() + o_c, cd.data(), sizeof(CompactDesc) * n);  // the meta region stays zero: cursor = 0
    char *base = (char *)e->d_round;
    CF_TRY(cudaMemcpyAsync(base, img.data(), total, cudaMemcpyHostToDevice, e->st), "upload round");
    const FieldGeom *d_geoms = (const FieldGeom *)(base + o_g);
    unsigned int *d_work = (unsigned int *)(base + o_w);
    int launches = 0;
    CF_TRY(launch_query_batch((const QueryDesc *)(base + o_q), d_geoms, n, q_items, e->tune.query_ppb, d_work, e->st),
           "round query");
    ++launches;
    CF_TRY(launch_sample_batch((const ScoreArgs *)(base + o_a), (const long long *)(base + o_p), n, pose0[n], smem,
                               e->st), "round sample");
    ++launches;
    for (size_t g = 0; g < skeys.size(); ++g) {
        CF_TRY(launch_score_batch(sd[s_off[g]], (const ScoreArgs *)(base + o_s) + s_off[g],
                                  (const long long *)(base + o_t) + t_off[g], s_n[g], s_tuples[g], e->st),
               "round score");
        ++launches;
    }
    unsigned *d_meta = (unsigned *)(base + o_m);
    k_compact_accepted<<<n, kCompactThreads, 0, e->st>>>((const CompactDesc *)(base + o_c), (AccRecord *)e->d_rec,
                                                        d_meta, d_meta + 1, d_meta + 1 + n);
    CF_TRY(cudaGetLastError(), "round compaction");
    ++launches;
    CF_TRY(cudaMemcpyAsync(e->h_meta, d_meta, meta_bytes, cudaMemcpyDeviceToHost, e->st), "download round extents");
    const double t_launched = e->now();
    CF_TRY(cudaStreamSynchronize(e->st), "round");
    const size_t used = sizeof(AccRecord) * (size_t)e->h_meta[0];
    if (used > e->h_rec_bytes) {
        if (e->h_rec) cudaFreeHost(e->h_rec);
        e->h_rec = nullptr;
        e->h_rec_bytes = 0;
        CF_TRY(cudaHostAlloc((void **)&e->h_rec, 2 * used, cudaHostAllocDefault), "alloc round records (host)");
        e->h_rec_bytes = 2 * used;
    }
    if (used > 0)
        CF_TRY(cudaMemcpyAsync(e->h_rec, e->d_rec, used, cudaMemcpyDeviceToHost, e->st), "download accepted records");
    for (int i = 0; i < n; ++i) {
        act[i]->rec_off = e->h_meta[1 + i];
        act[i]->rec_cnt = e->h_meta[1 + n + i];
    }
    CF_TRY(cudaStreamSynchronize(e->st), "round");
    const double t_end = e->now();
    std::lock_guard<std::mutex> lk(e->mu);
    e->stats.rounds++;
    e->stats.launches += launches;
    e->stats.round_host_s += t_launched - t_start;
    e->stats.round_wait_s += t_end - t_launched;
    return CF_OK;
}

void worker_main(cf_engine *e) {
    cudaSetDevice(e->dev);
    for (;;) {
        std::vector<EngReq *> act;
        std::vector<EngReq *> rejected;
        {
            std::unique_lock<std::mutex> lk(e->mu);
            for (;;) {
                if (e->stop) return;
                // admission, in arrival order
                while (!e->queue.empty() && (int)e->active.size() < e->prm.max_active) {
                    EngReq *r = e->queue.front();
                    if ((int64_t)r->bytes > e->prm.hbm_budget_bytes) {  // can never fit
                        e->queue.pop_front();
                        rejected.push_back(r);
                        continue;
                    }
                    if (e->stats.bytes_in_use + (int64_t)r->bytes > e->prm.hbm_budget_bytes) break;
                    e->queue.pop_front();
                    e->stats.bytes_in_use += (int64_t)r->bytes;
                    e->stats.peak_bytes_in_use = std::max(e->stats.peak_bytes_in_use, e->stats.bytes_in_use);
                    r->t_admit = e->now();
                    e->active.push_back(r);
                    act.push_back(r);  // newly admitted: uploaded below
                }
                e->stats.peak_active = std::max(e->stats.peak_active, (int32_t)e->active.size());
                if (!e->active.empty() || !rejected.empty()) break;
                e->cv_idle.notify_all();
                e->cv.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
        for (EngReq *r : rejected) finish(e, r, CF_ENOMEM, false);
        rejected.clear();
        const double t_adm = e->now();
        for (EngReq *r : act) {
            const int arc = admit_one(e, r);
            if (arc != CF_OK) {  // the request ends with the error; its budget share is returned by finish
                cudaStreamSynchronize(e->st);  // no upload of its block may still be running
                {
                    std::lock_guard<std::mutex> lk(e->mu);
                    e->active.erase(std::find(e->active.begin(), e->active.end(), r));
                    if (!r->d_block) e->stats.bytes_in_use -= (int64_t)r->bytes;
                }
                finish(e, r, arc, false);
            }
        }
        if (!act.empty()) {
            const double dt = e->now() - t_adm;
            std::lock_guard<std::mutex> lk(e->mu);
            e->stats.admit_s += dt;
        }
        std::vector<EngReq *> round;
        {
            std::lock_guard<std::mutex> lk(e->mu);
            round = e->active;
        }
        if (round.empty()) continue;
        const int rc = run_round(e, round);
        std::vector<EngReq *> finished;
        for (EngReq *r : round) {
            bool done = rc != CF_OK;
            if (rc == CF_OK) {
                const int k = r->req.prm.k;
                const AccRecord *rec = e->h_rec + r->rec_off;
                for (unsigned a = 0; a < r->rec_cnt; ++a) {
                    r->res_pose.push_back(rec[a].pose);
                    r->res_margin.push_back(rec[a].margin);
                    for (int d = 0; d < k; ++d) r->res_tuples.push_back(rec[a].t[d]);
                }
                r->pose_next += r->chunk;
                done = (int)r->res_margin.size() >= r->req.n_grasps || r->pose_next >= r->limit;
            }
            if (done) finished.push_back(r);
        }
        {
            std::lock_guard<std::mutex> lk(e->mu);
            for (EngReq *r : finished) e->active.erase(std::find(e->active.begin(), e->active.end(), r));
        }
        for (EngReq *r : finished)
            finish(e, r, rc, rc == CF_OK && (int)r->res_margin.size() < r->req.n_grasps);
    }
}

}  // namespace

extern "C" int cf_engine_create(const cf_engine_params *prm, cf_engine **out) {
    if (!prm || !out) return fail(CF_EINVAL, "NULL argument");
    if (prm->n_fields < 1 || !prm->fields) return fail(CF_EINVAL, "no fields");
    if (prm->max_active < 1 || prm->pose_chunk < 1 || prm->pose_cap < 1 || prm->hbm_budget_bytes <= 0)
        return fail(CF_EINVAL, "max_active, pose_chunk, pose_cap and the budget must be positive");
    if (prm->reserve_bytes < 0) return fail(CF_EINVAL, "reserve_bytes must be >= 0");
    cf_engine *e = new cf_engine();
    e->prm = *prm;
    for (int i = 0; i < prm->n_fields; ++i) {
        if (!prm->fields[i] || prm->fields[i]->table_words == 0) {
            delete e;
            return fail(CF_EINVAL, "field %d is NULL or empty", i);
        }
        if (prm->fields[i]->geom.patches) {
            delete e;
            return fail(CF_EINVAL, "field %d is a patch field: the engine samples from finger domains", i);
        }
        e->fields.push_back(prm->fields[i]);
        e->geoms.push_back(prm->fields[i]->geom);
    }
    e->prm.fields = nullptr;
    CF_TRY(cudaGetDevice(&e->dev), "cudaGetDevice");
    e->tune = current_tuning();
    cudaError_t err = cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking);
    if (err != cudaSuccess) { delete e; return cuda_fail(err, "stream"); }
    if (prm->reserve_bytes > 0) {  // grow the pool now (it keeps what is freed), not while admitting requests
        void *p = nullptr;
        int rc = pool_alloc(&p, (size_t)prm->reserve_bytes, e->st, "reserve engine memory");
        if (rc == CF_OK) {
            err = cudaFreeAsync(p, e->st);
            if (err == cudaSuccess) err = cudaStreamSynchronize(e->st);
            if (err != cudaSuccess) rc = cuda_fail(err, "reserve engine memory");
        }
        if (rc != CF_OK) {
            cudaStreamDestroy(e->st);
            delete e;
            return rc;
        }
    }
    e->t0 = std::chrono::steady_clock::now();
    e->worker = std::thread(worker_main, e);
    *out = e;
    return CF_OK;
}

extern "C" int cf_engine_submit(cf_engine *e, const cf_request *q, uint64_t *id) {
    if (!e || !q) return fail(CF_EINVAL, "NULL argument");
    if (q->field < 0 || q->field >= (int)e->fields.size()) return fail(CF_EINVAL, "field %d out of range", q->field);
    if (q->n < 1 || !q->h_soa || q->n_poses < 1 || !q->h_poses) return fail(CF_EINVAL, "empty object or pose list");
    if (q->prm.tuples_given) return fail(CF_EINVAL, "requests sample their own tuples");
    if (q->prm.k < 1 || q->prm.k > CF_MAX_K || q->prm.n_edges < 3 || q->prm.n_edges > CF_MAX_EDGES ||
        q->prm.k * q->prm.n_edges > 32 || q->prm.n_tuples < 1 || q->n_grasps < 1)
        return fail(CF_EINVAL, "bad k / K / T / n_grasps");
    EngReq *r = new EngReq();
    r->req = *q;
    r->fd = e->fields[q->field];
    const size_t in_bytes = sizeof(float) * (6 * (size_t)q->n + 12 * (size_t)q->n_poses);
    r->h_in = (float *)e->pinned.get(in_bytes, e->dev, &r->h_in_bytes);
    if (!r->h_in) {
        delete r;
        return fail(CF_ENOMEM, "page-locked host memory for a request of %zu bytes", in_bytes);
    }
    memcpy(r->h_in, q->h_soa, sizeof(float) * 6 * (size_t)q->n);
    memcpy(r->h_in + 6 * (size_t)q->n, q->h_poses, sizeof(float) * 12 * (size_t)q->n_poses);
    r->req.h_soa = nullptr;
    r->req.h_poses = nullptr;
    r->limit = std::min(q->n_poses, e->prm.pose_cap);
    r->cap = std::max(1, std::min(r->limit, std::max(e->prm.pose_chunk, e->prm.pose_chunk_max)));
    r->bytes = state_bytes(*q, r->fd->F, r->cap);
    {
        std::lock_guard<std::mutex> lk(e->mu);
        r->id = e->next_id++;
        r->t_submit = e->now();
        e->queue.push_back(r);
        e->stats.submitted++;
    }
    e->cv.notify_all();
    if (id) *id = r->id;
    return CF_OK;
}

extern "C" int cf_engine_poll(cf_engine *e, cf_result *out, int32_t max, int32_t *n_done) {
    if (!e || !out || !n_done) return fail(CF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(e->mu);
    int n = 0;
    while (n < max && !e->done.empty()) {
        out[n++] = e->done.front();
        e->done.pop_front();
    }
    *n_done = n;
    return CF_OK;
}

extern "C" int cf_engine_result_free(cf_result *r) {
    if (!r) return CF_OK;
    free(r->pose);
    free(r->tuples);
    free(r->margin);
    r->pose = r->tuples = nullptr;
    r->margin = nullptr;
    return CF_OK;
}

extern "C" int cf_engine_get_stats(const cf_engine *ce, cf_engine_stats *out) {
    if (!ce || !out) return fail(CF_EINVAL, "NULL argument");
    cf_engine *e = const_cast<cf_engine *>(ce);
    std::lock_guard<std::mutex> lk(e->mu);
    *out = e->stats;
    out->queued = (int32_t)e->queue.size();
    out->active = (int32_t)e->active.size();
    return CF_OK;
}

extern "C" int cf_engine_drain(cf_engine *e, int32_t timeout_ms) {
    if (!e) return fail(CF_EINVAL, "NULL argument");
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    std::unique_lock<std::mutex> lk(e->mu);
    while (!e->queue.empty() || !e->active.empty()) {
        if (timeout_ms >= 0 && std::chrono::steady_clock::now() >= deadline)
            return fail(CF_ETIMEOUT, "engine still has %zu queued and %zu active requests", e->queue.size(),
                        e->active.size());
        e->cv_idle.wait_for(lk, std::chrono::milliseconds(2));
    }
    return CF_OK;
}

extern "C" int cf_engine_destroy(cf_engine *e) {
    if (!e) return CF_OK;
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->stop = true;
    }
    e->cv.notify_all();
    if (e->worker.joinable()) e->worker.join();
    for (EngReq *r : e->active) {
        if (r->d_block) cudaFreeAsync(r->d_block, e->st);
        delete r;
    }
    for (EngReq *r : e->queue) delete r;
    for (cf_result &r : e->done) cf_engine_result_free(&r);
    if (e->d_round) cudaFreeAsync(e->d_round, e->st);
    if (e->d_rec) cudaFreeAsync(e->d_rec, e->st);
    cudaStreamSynchronize(e->st);
    cudaStreamDestroy(e->st);
    if (e->h_rec) cudaFreeHost(e->h_rec);
    if (e->h_meta) cudaFreeHost(e->h_meta);
    delete e;  // the page-locked request blocks go with the pool
    return CF_OK;
}
