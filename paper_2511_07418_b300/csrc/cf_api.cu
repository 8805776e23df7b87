// Host side of the libcf C ABI: argument checks, field lifecycle, launches,
// the host-buffer request plan and the device status word / counters.
#include <limits.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "cf_internal.cuh"

using namespace cf;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
namespace cf {

thread_local std::string t_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? CF_ENOMEM : CF_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e),
                cudaGetErrorString(e));
}


// ---------------------------------------------------------------------------
// device status word and counters (one copy per device that loads libcf)
// ---------------------------------------------------------------------------
__device__ unsigned int g_status;
__device__ unsigned long long g_counters[4];

struct DevState {
    unsigned int *status = nullptr;
    unsigned long long *counters = nullptr;
};

std::mutex g_state_mu;
DevState g_state[64];

std::mutex g_tune_mu;
Tuning g_tune[64];
bool g_tune_set[64] = {};
constexpr Tuning kDefaultTuning{4, 8, 0};

int device_state(DevState *out) {
    int dev = 0;
    CF_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(CF_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_state_mu);
    DevState &s = g_state[dev];
    if (!s.status) {
        CF_TRY(cudaGetSymbolAddress((void **)&s.status, g_status), "cudaGetSymbolAddress(status)");
        CF_TRY(cudaGetSymbolAddress((void **)&s.counters, g_counters), "cudaGetSymbolAddress(counters)");
    }
    *out = s;
    return CF_OK;
}

}  // namespace cf

// ---------------------------------------------------------------------------
// device memory: one stream-ordered pool per device, owned by the library
// (allocations and frees are ordered on the caller's stream; the pool keeps
// freed memory for reuse instead of returning it to the CUDA driver)
// ---------------------------------------------------------------------------
namespace cf {

std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

int device_pool(cudaMemPool_t *out) {
    int dev = 0;
    CF_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(CF_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        CF_TRY(cudaMemPoolCreate(&g_pool[dev], &props), "cudaMemPoolCreate");
        uint64_t keep = UINT64_MAX;
        CF_TRY(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep), "pool attribute");
    }
    *out = g_pool[dev];
    return CF_OK;
}

int pool_alloc(void **p, size_t bytes, cudaStream_t st, const char *what) {
    cudaMemPool_t pool;
    int rc = device_pool(&pool);
    if (rc) return rc;
    CF_TRY(cudaMallocFromPoolAsync(p, bytes ? bytes : 1, pool, st), what);
    return CF_OK;
}

// Normal-bin candidate tables, computed once per distinct direction set.
struct CandEntry {
    std::vector<float> dirs;
    std::vector<uint32_t> table;
    int worst;
};
std::mutex g_cand_mu;
std::vector<CandEntry *> g_cand_cache;

const CandEntry *cached_candidates(const float *dirs, int B) {
    std::lock_guard<std::mutex> lk(g_cand_mu);
    for (const CandEntry *c : g_cand_cache)
        if ((int)c->dirs.size() == 3 * B && memcmp(c->dirs.data(), dirs, sizeof(float) * 3 * B) == 0) return c;
    CandEntry *c = new CandEntry();
    c->dirs.assign(dirs, dirs + 3 * B);
    c->table.resize(kCandCells);
    c->worst = build_bin_candidates(dirs, B, c->table.data());
    g_cand_cache.push_back(c);
    return c;
}

}  // namespace cf

// ---------------------------------------------------------------------------
// field
// ---------------------------------------------------------------------------

namespace {

void field_release(cf_field *fd) {
    if (!fd) return;
    if (fd->d_block) cudaFreeAsync(fd->d_block, fd->st);
    if (fd->d_table) cudaFreeAsync(fd->d_table, fd->st);
    if (fd->d_cand) cudaFreeAsync(fd->d_cand, fd->st);
    if (fd->d_rep) cudaFreeAsync(fd->d_rep, fd->st);
    if (fd->d_qs) cudaFreeAsync(fd->d_qs, fd->st);
    if (fd->d_prefix) cudaFreeAsync(fd->d_prefix, fd->st);
    if (fd->ev0) cudaEventDestroy(fd->ev0);
    if (fd->ev1) cudaEventDestroy(fd->ev1);
    delete fd;
}

int check_hand(const cf_hand_desc *h) {
    if (!h) return fail(CF_EINVAL, "hand is NULL");
    if (h->n_fingers < 1 || h->n_fingers > CF_MAX_FINGERS)
        return fail(CF_EINVAL, "n_fingers=%d not in [1,%d]", h->n_fingers, CF_MAX_FINGERS);
    if (h->n_joints < 1 || h->n_joints > CF_MAX_JOINTS)
        return fail(CF_EINVAL, "n_joints=%d not in [1,%d]", h->n_joints, CF_MAX_JOINTS);
    if (h->n_surf < 1 || h->n_surf > CF_MAX_SURF)
        return fail(CF_EINVAL, "n_surf=%d not in [1,%d]", h->n_surf, CF_MAX_SURF);
    if (!h->base || !h->axis || !h->offset || !h->surf_p || !h->surf_n || !h->surf_link)
        return fail(CF_EINVAL, "hand array pointer is NULL");
    for (int i = 0; i < h->n_fingers * h->n_surf; ++i)
        if (h->surf_link[i] < 0 || h->surf_link[i] >= h->n_joints)
            return fail(CF_EINVAL, "surf_link[%d]=%d not in [0,%d)", i, h->surf_link[i], h->n_joints);
    if ((h->lo != nullptr) != (h->hi != nullptr) || (h->lo != nullptr) != (h->radius != nullptr))
        return fail(CF_EINVAL, "lo, hi and radius must be given together");
    if (h->lo)
        for (int i = 0; i < h->n_fingers * h->n_joints; ++i) {
            if (!(h->lo[i] <= h->hi[i]) || !isfinite(h->lo[i]) || !isfinite(h->hi[i]))
                return fail(CF_EINVAL, "joint %d: limits [%g, %g] are not a finite interval", i, h->lo[i], h->hi[i]);
            if (!(h->radius[i] >= 0.f) || !isfinite(h->radius[i]))
                return fail(CF_EINVAL, "joint %d: radius %g must be finite and >= 0", i, h->radius[i]);
        }
    return CF_OK;
}

// Upload the normal-bin candidate table of fd's directions (stream-ordered).
int setup_candidates(cf_field *fd) {
    const CandEntry *c = cached_candidates(&fd->geom.dirs[0][0], fd->geom.B);
    fd->geom.use_cand = c->worst <= 4 ? 1 : 0;
    int rc = pool_alloc((void **)&fd->d_cand, sizeof(uint32_t) * kCandCells, fd->st, "alloc candidates");
    if (rc) return rc;
    CF_TRY(cudaMemcpyAsync(fd->d_cand, c->table.data(), sizeof(uint32_t) * kCandCells, cudaMemcpyHostToDevice, fd->st),
           "copy candidates");
    fd->geom.cand = fd->d_cand;
    return CF_OK;
}

// Table slots: one per finger, or (patch field, Sec. 4.4) one per (finger, link with surface points),
// fingers in order and links ascending.
int slot_map(cf_field *fd, const cf_hand_desc *hand, const cf_field_params *prm) {
    if (prm->patches != 0 && prm->patches != 1) return fail(CF_EINVAL, "patches=%d not in {0, 1}", prm->patches);
    if (prm->patches && prm->want_rep)
        return fail(CF_EINVAL, "patch fields keep no representative table (want_rep needs patches = 0)");
    FieldGeom &g = fd->geom;
    g.patches = prm->patches;
    memset(g.slot_of, -1, sizeof g.slot_of);
    memset(g.slot_finger, -1, sizeof g.slot_finger);
    memset(g.slot_link, -1, sizeof g.slot_link);
    const int F = hand->n_fingers, J = hand->n_joints, M = hand->n_surf;
    int ns = 0;
    for (int f = 0; f < F; ++f) {
        if (!g.patches) {
            for (int l = 0; l < J; ++l) g.slot_of[f][l] = (int8_t)f;
            g.slot_finger[f] = (int8_t)f;
            ++ns;
            continue;
        }
        for (int l = 0; l < J; ++l) {
            bool has = false;
            for (int m = 0; m < M && !has; ++m) has = hand->surf_link[(size_t)f * M + m] == l;
            if (!has) continue;
            if (ns == CF_MAX_SLOTS)
                return fail(CF_EINVAL, "the hand has more than %d (finger, link) patches", CF_MAX_SLOTS);
            g.slot_of[f][l] = (int8_t)ns;
            g.slot_finger[ns] = (int8_t)f;
            g.slot_link[ns] = (int8_t)l;
            ++ns;
        }
    }
    g.F = ns;
    return CF_OK;
}

int geom_from_params(cf_field *fd, const cf_field_params *prm) {
    if (!prm) return fail(CF_EINVAL, "params is NULL");
    if (!(prm->inv_h > 0.f) || !isfinite(prm->inv_h)) return fail(CF_EINVAL, "inv_h must be finite and > 0");
    if (prm->n_bins < 1 || prm->n_bins > CF_MAX_BINS)
        return fail(CF_EINVAL, "n_bins=%d not in [1,%d]", prm->n_bins, CF_MAX_BINS);
    if (!prm->bin_dirs) return fail(CF_EINVAL, "bin_dirs is NULL");
    FieldGeom &g = fd->geom;
    g.F = fd->F;
    g.B = prm->n_bins;
    g.inv_h = prm->inv_h;
    g.clamp = (float)(2097152.0 / (double)prm->inv_h);  // |x * inv_h| <= 2^21
    for (int b = 0; b < g.B; ++b)
        for (int c = 0; c < 3; ++c) g.dirs[b][c] = prm->bin_dirs[3 * b + c];
    if (!(prm->dilate_deg >= 0.f && prm->dilate_deg <= 180.f)) return fail(CF_EINVAL, "dilate_deg not in [0, 180]");
    g.dilate_deg = prm->dilate_deg;
    const double dcos = cos((double)prm->dilate_deg * (M_PI / 180.0));
    for (int b = 0; b < CF_MAX_BINS; ++b) g.dil[b] = 0u;
    for (int b = 0; b < g.B; ++b) {
        g.dil[b] = 1u << b;
        if (!(prm->dilate_deg > 0.f)) continue;
        for (int b2 = 0; b2 < g.B; ++b2) {
            const double d = (double)g.dirs[b][0] * g.dirs[b2][0] + (double)g.dirs[b][1] * g.dirs[b2][1] +
                             (double)g.dirs[b][2] * g.dirs[b2][2];
            if (d >= dcos) g.dil[b] |= 1u << b2;
        }
    }
    fd->B = g.B;
    return CF_OK;
}

}  // namespace

namespace cf {
// Page-locked buffers for cf_build's cell-bounds read-back (a copy into pageable memory goes through a
// driver staging buffer and completes later): taken and returned under a lock, allocated on first need
// and kept for the life of the process.
std::mutex g_bnd_mu;
std::vector<int *> g_bnd_free;
constexpr int kBoundsInts = 6 * CF_MAX_FINGERS;

struct BoundsBuffer {
    int *p = nullptr;
    BoundsBuffer() {
        {
            std::lock_guard<std::mutex> lk(g_bnd_mu);
            if (!g_bnd_free.empty()) {
                p = g_bnd_free.back();
                g_bnd_free.pop_back();
                return;
            }
        }
        if (cudaHostAlloc((void **)&p, sizeof(int) * kBoundsInts, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();  // the caller falls back to pageable memory
            p = nullptr;
        }
    }
    ~BoundsBuffer() {
        if (!p) return;
        std::lock_guard<std::mutex> lk(g_bnd_mu);
        g_bnd_free.push_back(p);
    }
};

cudaError_t launch_shape(const void *func, int threads, size_t smem, int *per_sm, int *sms) {
    struct Entry {
        int dev;
        const void *func;
        int threads;
        size_t smem;
        int per_sm, sms;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (const Entry &c : cache)
            if (c.dev == dev && c.func == func && c.threads == threads && c.smem == smem) {
                *per_sm = c.per_sm;
                *sms = c.sms;
                return cudaSuccess;
            }
    }
    Entry c{dev, func, threads, smem, 0, 0};
    if ((e = cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.per_sm, func, threads, smem)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    cache.push_back(c);
    *per_sm = c.per_sm;
    *sms = c.sms;
    return cudaSuccess;
}

Tuning current_tuning() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return kDefaultTuning;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune_set[dev] ? g_tune[dev] : kDefaultTuning;
}
}  // namespace cf

extern "C" int cf_build(const cf_hand_desc *hand, const cf_field_params *prm, const float *d_q, int32_t n_samples,
                        cf_stream stream, cf_field **out) {
    if (!out) return fail(CF_EINVAL, "out is NULL");
    int rc = check_hand(hand);
    if (rc) return rc;
    if (n_samples < 0) return fail(CF_EINVAL, "n_samples < 0");
    if (n_samples > 0 && !d_q) return fail(CF_EINVAL, "d_q is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    DevState ds;
    if ((rc = device_state(&ds))) return rc;

    cf_field *fd = new cf_field();
    const int F = hand->n_fingers, J = hand->n_joints, M = hand->n_surf;
    fd->F = F; fd->J = J; fd->M = M; fd->S = n_samples;
    fd->st = st;
    CF_TRY(cudaGetDevice(&fd->dev), "cudaGetDevice");
    if ((rc = geom_from_params(fd, prm)) || (rc = setup_candidates(fd))) { field_release(fd); return rc; }
    if ((rc = slot_map(fd, hand, prm))) { field_release(fd); return rc; }

    const bool want_rep = prm->want_rep != 0;
    if (want_rep && !hand->lo) { field_release(fd); return fail(CF_EINVAL, "want_rep needs the joint limits"); }
    if (want_rep && (uint64_t)n_samples * (uint64_t)M >= 0xffffffffull) {
        field_release(fd);
        return fail(CF_EINVAL, "want_rep: n_samples * n_surf = %lld does not fit 32 bits",
                    (long long)n_samples * M);
    }
    fd->has_limits = hand->lo != nullptr;

    // host staging of the hand block: base | axis | offset | surf (sorted by link) | lo | hi | radius |
    // link ranges | sorted position of each surface point | bounds init
    const size_t n_base = (size_t)F * 12, n_axis = (size_t)F * J * 3, n_surf = (size_t)F * M * 8;
    const size_t n_fj = (size_t)F * J, n_lb = (size_t)F * (J + 1), n_so = (size_t)F * M, n_bnd = (size_t)6 * F;
    const size_t bytes = sizeof(float) * (n_base + 2 * n_axis + n_surf + 3 * n_fj) + sizeof(int) * (n_lb + n_so + n_bnd);
    std::vector<char> stage(bytes, 0);
    float *h_base = (float *)stage.data(), *h_axis = h_base + n_base, *h_off = h_axis + n_axis, *h_surf = h_off + n_axis;
    float *h_lo = h_surf + n_surf, *h_hi = h_lo + n_fj, *h_rad = h_hi + n_fj;
    int *h_lb = (int *)(h_rad + n_fj), *h_so = h_lb + n_lb, *h_bnd = h_so + n_so;
    memcpy(h_base, hand->base, sizeof(float) * n_base);
    memcpy(h_axis, hand->axis, sizeof(float) * n_axis);
    memcpy(h_off, hand->offset, sizeof(float) * n_axis);
    if (hand->lo) {
        memcpy(h_lo, hand->lo, sizeof(float) * n_fj);
        memcpy(h_hi, hand->hi, sizeof(float) * n_fj);
        memcpy(h_rad, hand->radius, sizeof(float) * n_fj);
    }
    for (int f = 0; f < F; ++f) {
        std::vector<int> order(M);
        for (int m = 0; m < M; ++m) order[m] = m;
        const int32_t *lk = hand->surf_link + (size_t)f * M;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lk[a] < lk[b]; });
        for (int m = 0; m < M; ++m) {
            const int src = order[m];
            float *d = h_surf + ((size_t)f * M + m) * 8;
            for (int c = 0; c < 3; ++c) {
                d[c] = hand->surf_p[((size_t)f * M + src) * 3 + c];
                d[3 + c] = hand->surf_n[((size_t)f * M + src) * 3 + c];
            }
            d[6] = (float)lk[src];
            d[7] = (float)src;  // original index (exact: M <= CF_MAX_SURF)
            h_so[(size_t)f * M + src] = m;
        }
        for (int l = 0; l <= J; ++l) {
            int c = 0;
            for (int m = 0; m < M; ++m) c += lk[m] < l;
            h_lb[(size_t)f * (J + 1) + l] = c;
        }
        for (int c = 0; c < 3; ++c) { h_bnd[6 * f + c] = INT_MAX; h_bnd[6 * f + 3 + c] = INT_MIN; }
    }
    if ((rc = pool_alloc(&fd->d_block, bytes, st, "alloc hand block"))) { field_release(fd); return rc; }
    float *d_base = (float *)fd->d_block, *d_axis = d_base + n_base, *d_off = d_axis + n_axis, *d_surf = d_off + n_axis;
    float *d_lo = d_surf + n_surf, *d_hi = d_lo + n_fj, *d_rad = d_hi + n_fj;
    int *d_lb = (int *)(d_rad + n_fj), *d_so = d_lb + n_lb, *d_bounds = d_so + n_so;
    fd->hand = HandDev{F, J, M, d_base, d_axis, d_off, d_surf, d_lb, hand->lo ? d_lo : nullptr,
                       hand->lo ? d_hi : nullptr, d_rad, d_so};
    if (hand->lo) {
        fd->h_lo.assign(hand->lo, hand->lo + n_fj);
        fd->h_hi.assign(hand->hi, hand->hi + n_fj);
        fd->h_radius.assign(hand->radius, hand->radius + n_fj);
    }
    fd->h_offset.assign(hand->offset, hand->offset + n_axis);
    float *d_links = nullptr;
    auto bail = [&](cudaError_t err, const char *what) {
        if (d_links) cudaFreeAsync(d_links, st);
        field_release(fd);
        return cuda_fail(err, what);
    };
#define CF_STEP(call, what) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return bail(e_, what); } while (0)
    CF_STEP(cudaMemcpyAsync(fd->d_block, stage.data(), bytes, cudaMemcpyHostToDevice, st), "copy hand");
    CF_STEP(cudaEventCreate(&fd->ev0), "event");
    CF_STEP(cudaEventCreate(&fd->ev1), "event");
    CF_STEP(cudaEventRecord(fd->ev0, st), "event record");
    if (n_samples > 0) {
        if ((rc = pool_alloc((void **)&d_links, sizeof(float) * 12 * (size_t)F * J * n_samples, st, "alloc links"))) {
            field_release(fd);
            return rc;
        }
        CF_STEP(launch_fk_cell_bounds(fd->hand, d_q, n_samples, fd->geom.inv_h, fd->geom.clamp, d_bounds, d_links, st),
                "launch k_fk_cell_bounds");
    }
    std::vector<int> bnd(n_bnd);
    {
        BoundsBuffer hb;  // page-locked when it can be had
        int *dst = hb.p && n_bnd <= (size_t)kBoundsInts ? hb.p : bnd.data();
        CF_STEP(cudaMemcpyAsync(dst, d_bounds, sizeof(int) * n_bnd, cudaMemcpyDeviceToHost, st), "copy bounds");
        CF_STEP(cudaStreamSynchronize(st), "k_fk_cell_bounds");  // the table's size depends on these bounds
        if (dst != bnd.data()) memcpy(bnd.data(), dst, sizeof(int) * n_bnd);
    }

    // one box over all fingers' samples; per-finger tight bounds are kept for reporting
    FieldGeom &g = fd->geom;
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (int f = 0; f < F; ++f) {
        const int *b = &bnd[6 * f];
        if (b[0] > b[3]) {  // finger without samples
            for (int c = 0; c < 3; ++c) { g.flo[f][c] = 0; g.fdims[f][c] = 0; }
            continue;
        }
        for (int c = 0; c < 3; ++c) {
            if (b[c] <= -(1 << 20) || b[3 + c] >= (1 << 20)) {
                if (d_links) cudaFreeAsync(d_links, st);
                field_release(fd);
                return fail(CF_EINVAL, "finger %d cells span [%d,%d] on axis %d: beyond |k| < 2^20 (voxel too small "
                                       "or hand too large)", f, b[c], b[3 + c], c);
            }
            g.flo[f][c] = b[c];
            g.fdims[f][c] = b[3 + c] - b[c] + 1;
            lo[c] = std::min(lo[c], b[c]);
            hi[c] = std::max(hi[c], b[3 + c]);
        }
    }
    g.bits = slot_bits_for(g.B);
    g.fpw = 32 / g.bits;
    g.rw = record_stride((g.F + g.fpw - 1) / g.fpw);  // words per record (padded to aligned loads)
    int64_t words = 0;
    if (lo[0] <= hi[0]) {
        for (int c = 0; c < 3; ++c) { g.lo[c] = lo[c]; g.dims[c] = hi[c] - lo[c] + 1; }
        words = (int64_t)g.dims[0] * g.dims[1] * g.dims[2] * g.rw;
    } else {
        for (int c = 0; c < 3; ++c) { g.lo[c] = 0; g.dims[c] = 0; }
    }
    fd->table_words = words;
    if (words > 0) {
        if ((rc = pool_alloc((void **)&fd->d_table, sizeof(uint32_t) * (size_t)words, st, "alloc table"))) {
            if (d_links) cudaFreeAsync(d_links, st);
            field_release(fd);
            return rc;
        }
        CF_STEP(cudaMemsetAsync(fd->d_table, 0, sizeof(uint32_t) * (size_t)words, st), "memset table");
        CF_STEP(launch_fk_bin(fd->hand, h_lb, d_links, n_samples, fd->geom, fd->d_table, ds.status, st), "launch k_fk_bin");
    }
    int64_t rep_bytes = 0;
    if (want_rep) {
        // keep the joint samples (reverse lookup starts IK from them) and build the representative table:
        // count the codes (one more wait), size the hash at load <= 1/2, then pass 3
        const size_t qbytes = sizeof(float) * (size_t)F * J * n_samples;
        if (qbytes) {
            if ((rc = pool_alloc((void **)&fd->d_qs, qbytes, st, "alloc samples"))) {
                if (d_links) cudaFreeAsync(d_links, st);
                field_release(fd);
                return rc;
            }
            CF_STEP(cudaMemcpyAsync(fd->d_qs, d_q, qbytes, cudaMemcpyDeviceToDevice, st), "copy samples");
        }
        unsigned long long *d_cnt = nullptr;
        if ((rc = pool_alloc((void **)&d_cnt, sizeof(unsigned long long), st, "alloc count"))) {
            if (d_links) cudaFreeAsync(d_links, st);
            field_release(fd);
            return rc;
        }
        CF_STEP(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st), "memset count");
        CF_STEP(launch_popcount(fd->d_table, words, d_cnt, st), "launch k_popcount");
        unsigned long long n_codes = 0;
        CF_STEP(cudaMemcpyAsync(&n_codes, d_cnt, sizeof n_codes, cudaMemcpyDeviceToHost, st), "copy count");
        CF_STEP(cudaFreeAsync(d_cnt, st), "free count");
        CF_STEP(cudaStreamSynchronize(st), "k_popcount");
        int lg = 4;
        while ((1ull << lg) < 2 * n_codes) ++lg;
        if (lg > 31) {
            if (d_links) cudaFreeAsync(d_links, st);
            field_release(fd);
            return fail(CF_EINVAL, "%llu field codes: too many for the representative table", n_codes);
        }
        const size_t slots = (size_t)1 << lg;
        rep_bytes = (int64_t)(slots * (sizeof(unsigned long long) + sizeof(uint32_t)));
        if ((rc = pool_alloc(&fd->d_rep, (size_t)rep_bytes, st, "alloc representative table"))) {
            if (d_links) cudaFreeAsync(d_links, st);
            field_release(fd);
            return rc;
        }
        fd->rep = RepTable{(unsigned long long *)fd->d_rep, (uint32_t *)((char *)fd->d_rep + slots * 8), lg};
        CF_STEP(cudaMemsetAsync(fd->d_rep, 0xff, (size_t)rep_bytes, st), "memset representative table");
        CF_STEP(launch_fk_rep(fd->hand, d_links, n_samples, fd->geom, fd->rep, ds.status, st), "launch k_fk_rep");
        rep_bytes += (int64_t)qbytes;
    }
    if (d_links) CF_STEP(cudaFreeAsync(d_links, st), "free links");
    CF_STEP(cudaEventRecord(fd->ev1, st), "event record");
#undef CF_STEP
    fd->device_bytes = (int64_t)bytes + (int64_t)sizeof(uint32_t) * (words + kCandCells) + rep_bytes;
    *out = fd;
    return CF_OK;
}

extern "C" int cf_field_get_info(const cf_field *fd, cf_field_info *info) {
    if (!fd || !info) return fail(CF_EINVAL, "NULL argument");
    memset(info, 0, sizeof *info);
    info->n_fingers = fd->F;
    info->n_joints = fd->J;
    info->n_surf = fd->M;
    info->n_bins = fd->B;
    info->n_samples = fd->S;
    info->inv_h = fd->geom.inv_h;
    for (int c = 0; c < 3; ++c) {
        info->box_lo[c] = fd->geom.lo[c];
        info->box_dims[c] = fd->geom.dims[c];
    }
    info->bits_per_finger = fd->geom.bits;
    info->fingers_per_word = fd->geom.fpw;
    info->record_words = fd->geom.rw;
    for (int f = 0; f < fd->F; ++f)
        for (int c = 0; c < 3; ++c) {
            info->finger_lo[f][c] = fd->geom.flo[f][c];
            info->finger_dims[f][c] = fd->geom.fdims[f][c];
        }
    info->table_words = fd->table_words;
    info->device_bytes = fd->device_bytes;
    cf_field *mfd = const_cast<cf_field *>(fd);
    if (mfd->build_ms < 0.f && mfd->ev1) {
        CF_TRY(cudaEventSynchronize(mfd->ev1), "build event");
        cudaEventElapsedTime(&mfd->build_ms, mfd->ev0, mfd->ev1);
    }
    info->build_ms = fd->build_ms < 0.f ? 0.f : fd->build_ms;
    info->dilate_deg = fd->geom.dilate_deg;
    for (int b = 0; b < CF_MAX_BINS; ++b) info->dilation[b] = fd->geom.dil[b];
    info->n_slots = fd->geom.F;
    for (int sl = 0; sl < CF_MAX_SLOTS; ++sl) {
        info->slot_finger[sl] = sl < fd->geom.F ? fd->geom.slot_finger[sl] : -1;
        info->slot_link[sl] = sl < fd->geom.F ? fd->geom.slot_link[sl] : -1;
    }
    return CF_OK;
}

extern "C" int cf_merge_domains(const cf_field *fd, const uint32_t *d_slot_masks, int32_t n_poses, int32_t n_words,
                                uint32_t *d_group_masks, uint32_t *d_group_counts, cf_stream stream) {
    if (!fd) return fail(CF_EINVAL, "field is NULL");
    if (n_poses < 0 || n_words < 0) return fail(CF_EINVAL, "n_poses / n_words < 0");
    if (n_poses == 0) return CF_OK;
    if (!d_slot_masks || !d_group_masks || !d_group_counts) return fail(CF_EINVAL, "array pointer is NULL");
    CF_TRY(launch_merge_domains(fd->geom, fd->F, d_slot_masks, n_poses, n_words, d_group_masks, d_group_counts,
                                (cudaStream_t)stream),
           "launch k_merge_domains");
    return CF_OK;
}

extern "C" int cf_field_copy_table(const cf_field *fd, uint32_t *host_words, int64_t capacity_words) {
    if (!fd || (!host_words && fd->table_words > 0)) return fail(CF_EINVAL, "NULL argument");
    if (capacity_words < fd->table_words)
        return fail(CF_EINVAL, "capacity %lld < table_words %lld", (long long)capacity_words,
                    (long long)fd->table_words);
    if (fd->table_words == 0) return CF_OK;
    CF_TRY(cudaStreamSynchronize(fd->st), "field stream");
    CF_TRY(cudaMemcpy(host_words, fd->d_table, sizeof(uint32_t) * (size_t)fd->table_words, cudaMemcpyDeviceToHost),
           "copy table");
    return CF_OK;
}

extern "C" int cf_field_rep_slots(const cf_field *fd, int64_t *slots) {
    if (!fd || !slots) return fail(CF_EINVAL, "NULL argument");
    *slots = fd->d_rep ? ((int64_t)1 << fd->rep.log2_slots) : 0;
    return CF_OK;
}

extern "C" int cf_field_copy_rep(const cf_field *fd, uint64_t *host_keys, uint32_t *host_vals, int64_t capacity) {
    if (!fd) return fail(CF_EINVAL, "field is NULL");
    if (!fd->d_rep) return fail(CF_EINVAL, "the field was built without want_rep");
    const int64_t slots = (int64_t)1 << fd->rep.log2_slots;
    if (!host_keys || !host_vals) return fail(CF_EINVAL, "NULL argument");
    if (capacity < slots) return fail(CF_EINVAL, "capacity %lld < rep slots %lld", (long long)capacity, (long long)slots);
    CF_TRY(cudaStreamSynchronize(fd->st), "field stream");
    CF_TRY(cudaMemcpy(host_keys, fd->rep.keys, sizeof(uint64_t) * (size_t)slots, cudaMemcpyDeviceToHost), "copy rep keys");
    CF_TRY(cudaMemcpy(host_vals, fd->rep.vals, sizeof(uint32_t) * (size_t)slots, cudaMemcpyDeviceToHost), "copy rep vals");
    return CF_OK;
}

extern "C" int cf_field_destroy(cf_field *fd) {
    field_release(fd);
    return CF_OK;
}

namespace {
const char kMagic[8] = {'C', 'F', 'F', 'I', 'E', 'L', 'D', '5'};
}

extern "C" int cf_field_save(const cf_field *fd, const char *path) {
    if (!fd || !path) return fail(CF_EINVAL, "NULL argument");
    std::vector<uint32_t> tab((size_t)fd->table_words);
    int rc = cf_field_copy_table(fd, tab.data(), fd->table_words);
    if (rc) return rc;
    FILE *fp = fopen(path, "wb");
    if (!fp) return fail(CF_EIO, "cannot open %s for writing", path);
    const int32_t hdr[5] = {fd->F, fd->J, fd->M, fd->S, fd->B};
    bool ok = fwrite(kMagic, 1, 8, fp) == 8 && fwrite(hdr, sizeof hdr, 1, fp) == 1 &&
              fwrite(&fd->geom, sizeof fd->geom, 1, fp) == 1 &&
              fwrite(&fd->table_words, sizeof fd->table_words, 1, fp) == 1 &&
              (tab.empty() || fwrite(tab.data(), sizeof(uint32_t), tab.size(), fp) == tab.size());
    ok = (fclose(fp) == 0) && ok;
    return ok ? CF_OK : fail(CF_EIO, "write to %s failed", path);
}

extern "C" int cf_field_load(const char *path, cf_field **out) {
    if (!path || !out) return fail(CF_EINVAL, "NULL argument");
    FILE *fp = fopen(path, "rb");
    if (!fp) return fail(CF_EIO, "cannot open %s", path);
    char magic[8];
    int32_t hdr[5];
    cf_field tmp;
    bool ok = fread(magic, 1, 8, fp) == 8 && memcmp(magic, kMagic, 8) == 0 && fread(hdr, sizeof hdr, 1, fp) == 1 &&
              fread(&tmp.geom, sizeof tmp.geom, 1, fp) == 1 &&
              fread(&tmp.table_words, sizeof tmp.table_words, 1, fp) == 1 && tmp.table_words >= 0 &&
              hdr[0] >= 1 && hdr[0] <= CF_MAX_FINGERS && hdr[4] >= 1 && hdr[4] <= CF_MAX_BINS;
    std::vector<uint32_t> tab(ok ? (size_t)tmp.table_words : 0);
    ok = ok && (tab.empty() || fread(tab.data(), sizeof(uint32_t), tab.size(), fp) == tab.size());
    fclose(fp);
    if (!ok) return fail(CF_EIO, "%s is not a valid field file", path);
    cf_field *fd = new cf_field();
    fd->F = hdr[0]; fd->J = hdr[1]; fd->M = hdr[2]; fd->S = hdr[3]; fd->B = hdr[4];
    fd->geom = tmp.geom;
    fd->geom.cand = nullptr;
    fd->table_words = tmp.table_words;
    fd->st = nullptr;
    fd->build_ms = 0.f;
    cudaGetDevice(&fd->dev);
    if (int rc2 = setup_candidates(fd)) { field_release(fd); return rc2; }
    if (!tab.empty()) {
        if (int rc2 = pool_alloc((void **)&fd->d_table, sizeof(uint32_t) * tab.size(), nullptr, "alloc table")) {
            field_release(fd);
            return rc2;
        }
        cudaError_t e = cudaMemcpyAsync(fd->d_table, tab.data(), sizeof(uint32_t) * tab.size(), cudaMemcpyHostToDevice,
                                        nullptr);
        if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
        if (e != cudaSuccess) { field_release(fd); return cuda_fail(e, "copy table"); }
    }
    fd->device_bytes = (int64_t)sizeof(uint32_t) * (fd->table_words + kCandCells);
    *out = fd;
    return CF_OK;
}

// ---------------------------------------------------------------------------
// query
// ---------------------------------------------------------------------------
namespace cf {
int check_points(const cf_points *obj) {
    if (!obj) return fail(CF_EINVAL, "obj is NULL");
    if (obj->n < 0) return fail(CF_EINVAL, "obj->n < 0");
    if (obj->n > 0 && (!obj->px || !obj->py || !obj->pz || !obj->nx || !obj->ny || !obj->nz))
        return fail(CF_EINVAL, "obj array pointer is NULL");
    return CF_OK;
}
}  // namespace cf

extern "C" int cf_query_domains(const cf_field *fd, const cf_points *obj, const float *d_poses, int32_t n_poses,
                                uint32_t *d_masks, uint32_t *d_counts, cf_stream stream) {
    if (!fd) return fail(CF_EINVAL, "field is NULL");
    int rc = check_points(obj);
    if (rc) return rc;
    if (n_poses < 0) return fail(CF_EINVAL, "n_poses < 0");
    if (n_poses > 0 && (!d_poses || !d_counts)) return fail(CF_EINVAL, "poses / counts pointer is NULL");
    if (n_poses == 0) return CF_OK;
    if (fd->table_words == 0) {  // empty field: no hits anywhere
        CF_TRY(cudaMemsetAsync(d_counts, 0, sizeof(uint32_t) * (size_t)n_poses * fd->F, (cudaStream_t)stream),
               "memset counts");
        if (d_masks)
            CF_TRY(cudaMemsetAsync(d_masks, 0, sizeof(uint32_t) * (size_t)n_poses * fd->F * ((obj->n + 31) / 32),
                                   (cudaStream_t)stream), "memset masks");
        return CF_OK;
    }
    CF_TRY(launch_query(fd->geom, fd->d_table, *obj, d_poses, n_poses, d_masks, d_counts, current_tuning().query_ppb,
                        (cudaStream_t)stream),
           "launch k_query_domains");
    return CF_OK;
}

// ---------------------------------------------------------------------------
// sampling + scoring
// ---------------------------------------------------------------------------
namespace cf {

int fill_score_args(const cf_points *obj, int32_t F, const uint32_t *d_masks, const uint32_t *d_counts, int32_t P,
                    const cf_score_params *prm, int32_t *d_tuples, uint8_t *d_fingers, float *d_margin,
                    uint8_t *d_accept, ScoreArgs *a) {
    int rc = check_points(obj);
    if (rc) return rc;
    if (!prm) return fail(CF_EINVAL, "params is NULL");
    if (P < 0) return fail(CF_EINVAL, "n_poses < 0");
    if (prm->k < 1 || prm->k > CF_MAX_K) return fail(CF_EINVAL, "k=%d not in [1,%d]", prm->k, CF_MAX_K);
    if (prm->n_edges < 3 || prm->n_edges > CF_MAX_EDGES)
        return fail(CF_EINVAL, "n_edges=%d not in [3,%d]", prm->n_edges, CF_MAX_EDGES);
    if (prm->k * prm->n_edges > 32) return fail(CF_EINVAL, "k * n_edges = %d > 32", prm->k * prm->n_edges);
    if (prm->n_tuples < 1) return fail(CF_EINVAL, "n_tuples < 1");
    // the kernels index tuples with 32-bit counters
    if ((long long)P * prm->n_tuples >= (1LL << 32))
        return fail(CF_EINVAL, "n_poses * n_tuples = %lld >= 2^32", (long long)P * prm->n_tuples);
    if (!(prm->mu >= 0.f) || !isfinite(prm->mu)) return fail(CF_EINVAL, "mu must be finite and >= 0");
    if (!(prm->rho > 0.f) || !isfinite(prm->rho)) return fail(CF_EINVAL, "rho must be finite and > 0");
    if (P > 0 && (!d_tuples || !d_margin || !d_accept)) return fail(CF_EINVAL, "output pointer is NULL");
    const bool sampling = !prm->tuples_given;
    if (sampling) {
        if (F < 1 || F > CF_MAX_FINGERS) return fail(CF_EINVAL, "n_fingers=%d not in [1,%d]", F, CF_MAX_FINGERS);
        if (P > 0 && (!d_masks || !d_counts)) return fail(CF_EINVAL, "masks / counts pointer is NULL");
    }
    const int W = (obj->n + 31) / 32;
    const size_t smem = score_smem_bytes(sampling ? F : 0, W, prm->n_tuples, prm->k, sampling);
    int dev = 0, optin = 0;
    CF_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    CF_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "device attribute");
    if (smem + 1024 > (size_t)optin)
        return fail(CF_EINVAL, "a pose's domains and tuples need %zu B of shared memory (limit %d): reduce N or T",
                    smem, optin);
    DevState ds;
    if ((rc = device_state(&ds))) return rc;
    memset(a, 0, sizeof *a);
    a->px = obj->px; a->py = obj->py; a->pz = obj->pz;
    a->nx = obj->nx; a->ny = obj->ny; a->nz = obj->nz;
    a->N = obj->n; a->W = W; a->F = sampling ? F : 0; a->P = P;
    a->masks = d_masks; a->counts = d_counts;
    a->T = prm->n_tuples; a->k = prm->k; a->K = prm->n_edges;
    a->mu = prm->mu; a->eps = prm->eps;
    a->cx = prm->centroid[0]; a->cy = prm->centroid[1]; a->cz = prm->centroid[2];
    a->inv_rho = (float)(1.0 / (double)prm->rho);
    for (int m = 0; m < CF_MAX_EDGES; ++m) {
        const double th = 2.0 * M_PI * (double)m / (double)prm->n_edges;
        a->cs[m] = (float)cos(th);
        a->sn[m] = (float)sin(th);
    }
    a->seed_lo = (uint32_t)prm->seed;
    a->seed_hi = (uint32_t)(prm->seed >> 32);
    a->tuples_given = prm->tuples_given ? 1 : 0;
    a->tuples = d_tuples; a->fingers = d_fingers; a->margin = d_margin; a->accept = d_accept;
    a->status = ds.status;
    a->counters = ds.counters;
    const Tuning tu = current_tuning();
    a->refill = tu.score_refill;
    a->bpsm = tu.score_bpsm;
    return CF_OK;
}

}  // namespace cf

extern "C" int cf_score_tuples(const cf_points *obj, int32_t n_fingers, const uint32_t *d_masks,
                               const uint32_t *d_counts, int32_t n_poses, const cf_score_params *prm,
                               int32_t *d_tuples, uint8_t *d_fingers, float *d_margin, uint8_t *d_accept,
                               cf_stream stream) {
    ScoreArgs a;
    int rc = fill_score_args(obj, n_fingers, d_masks, d_counts, n_poses, prm, d_tuples, d_fingers, d_margin,
                             d_accept, &a);
    if (rc) return rc;
    if (n_poses == 0) return CF_OK;
    // the lane scorer takes tuples from per-block shared-memory counters: no global scratch
    CF_TRY(launch_score(a, (cudaStream_t)stream), "launch k_sample_tuples / k_score_lanes");
    return CF_OK;
}

namespace {
std::mutex g_beta_mu;
std::vector<std::pair<std::pair<int, int>, float *>> g_beta;  // (device, n_iter) -> device table

int momentum_table(int n_iter, const float **out) {
    int dev = 0;
    CF_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_beta_mu);
    for (auto &e : g_beta)
        if (e.first.first == dev && e.first.second == n_iter) { *out = e.second; return CF_OK; }
    std::vector<float> beta((size_t)std::max(n_iter, 1), 0.f);
    double t = 1.0;
    for (int it = 0; it < n_iter; ++it) {
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        beta[it] = (float)((t - 1.0) / tn);
        t = tn;
    }
    float *d = nullptr;
    CF_TRY(cudaMalloc((void **)&d, sizeof(float) * beta.size()), "alloc momentum table");
    cudaError_t e = cudaMemcpy(d, beta.data(), sizeof(float) * beta.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(d); return cuda_fail(e, "upload momentum table"); }
    g_beta.push_back({{dev, n_iter}, d});
    *out = d;
    return CF_OK;
}
}  // namespace

extern "C" int cf_score_gswo(const cf_points *obj, int32_t n_poses, const cf_score_params *prm, int32_t n_iter,
                             float eps_g, const int32_t *d_tuples, float *d_value, uint8_t *d_accept,
                             cf_stream stream) {
    int rc = check_points(obj);
    if (rc) return rc;
    if (!prm) return fail(CF_EINVAL, "params is NULL");
    if (n_poses < 0 || prm->n_tuples < 1) return fail(CF_EINVAL, "n_poses < 0 or n_tuples < 1");
    if (prm->k < 2 || prm->k > CF_MAX_K) return fail(CF_EINVAL, "k=%d not in [2,%d]", prm->k, CF_MAX_K);
    if (!(prm->mu >= 0.f) || !isfinite(prm->mu)) return fail(CF_EINVAL, "mu must be finite and >= 0");
    if (!(prm->rho > 0.f) || !isfinite(prm->rho)) return fail(CF_EINVAL, "rho must be finite and > 0");
    if (n_iter < 0 || n_iter > 1000000) return fail(CF_EINVAL, "n_iter=%d out of range", n_iter);
    if (!isfinite(eps_g)) return fail(CF_EINVAL, "eps_g must be finite");
    const long long n = (long long)n_poses * prm->n_tuples;
    if (n == 0) return CF_OK;
    if (!d_tuples || !d_value || !d_accept) return fail(CF_EINVAL, "array pointer is NULL");
    const float *pts[6] = {obj->px, obj->py, obj->pz, obj->nx, obj->ny, obj->nz};
    // FISTA momentum coefficients (t_k - 1) / t_{k+1}, t_1 = 1, computed in FP64 once per
    // (device, n_iter) and kept for the process
    const float *d_beta = nullptr;
    if ((rc = momentum_table(n_iter, &d_beta))) return rc;
    CF_TRY(launch_gswo(pts, obj->n, n, prm->k, prm->mu, prm->centroid, prm->rho, eps_g, n_iter, d_beta, d_tuples,
                       d_value, d_accept, (cudaStream_t)stream),
           "launch k_gswo");
    return CF_OK;
}

extern "C" int cf_optimize_tuples(const cf_points *obj, int32_t n_fingers, const uint32_t *d_masks, int32_t n_poses,
                                  const cf_score_params *prm, const cf_opt_params *opt, int32_t *d_tuples,
                                  const uint8_t *d_fingers, float *d_margin, uint8_t *d_accept, cf_stream stream) {
    if (!prm || !opt) return fail(CF_EINVAL, "NULL argument");
    if (!prm->tuples_given) return fail(CF_EINVAL, "cf_optimize_tuples needs tuples_given = 1 (tuples are in/out)");
    if (n_fingers < 1 || n_fingers > CF_MAX_FINGERS)
        return fail(CF_EINVAL, "n_fingers=%d not in [1,%d]", n_fingers, CF_MAX_FINGERS);
    if (opt->n_outer < 0 || opt->n_outer > 64) return fail(CF_EINVAL, "n_outer=%d not in [0,64]", opt->n_outer);
    if (opt->n_inner != 4 && opt->n_inner != 8 && opt->n_inner != 16)
        return fail(CF_EINVAL, "n_inner=%d not in {4, 8, 16}", opt->n_inner);
    if (!(opt->sigma >= 0.f) || !isfinite(opt->sigma)) return fail(CF_EINVAL, "sigma must be finite and >= 0");
    if (!(opt->zero_tol >= 0.f) || !isfinite(opt->zero_tol)) return fail(CF_EINVAL, "zero_tol must be >= 0");
    if (!(opt->min_gain >= 0.f && opt->min_gain < 1.f)) return fail(CF_EINVAL, "min_gain must be in [0, 1)");
    if (opt->warm_start != 0 && opt->warm_start != 1) return fail(CF_EINVAL, "warm_start not in {0, 1}");
    ScoreArgs a;
    int rc = fill_score_args(obj, n_fingers, d_masks, nullptr, n_poses, prm, d_tuples, const_cast<uint8_t *>(d_fingers),
                             d_margin, d_accept, &a);
    if (rc) return rc;
    if (n_poses == 0) return CF_OK;
    if (!d_masks || !d_fingers) return fail(CF_EINVAL, "masks / fingers pointer is NULL");
    a.F = n_fingers;
    a.masks = d_masks;
    cudaStream_t st = (cudaStream_t)stream;
    // scratch: the work counter, then the point boxes of the projections' pruning (one per mask
    // word, then one per chunk of 32 words), then the per-tuple state of the phases
    void *scratch = nullptr;
    const size_t box_off = 256,
                 box_bytes = sizeof(float) * 6 * ((size_t)std::max(a.W, 1) + (size_t)(a.W + 31) / 32),
                 state_off = box_off + (box_bytes + 255) / 256 * 256,
                 bytes = state_off + optimize_state_bytes((long long)n_poses * prm->n_tuples, opt->n_inner, prm->k,
                                                           opt->warm_start);
    if ((rc = pool_alloc(&scratch, bytes, st, "alloc optimisation scratch"))) return rc;
    unsigned int *work = (unsigned int *)scratch;
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        a.work = work;
        a.word_box = (float *)((char *)scratch + box_off);
        e = launch_optimize(a, opt->n_outer, opt->n_inner, opt->sigma, opt->zero_tol, opt->min_gain, opt->warm_start,
                            (char *)scratch + state_off, st);
    }
    cudaError_t e2 = cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "launch the Alg. 2 phases");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync(optimisation scratch)");
    return CF_OK;
}

extern "C" int cf_sample_tuples(const cf_points *obj, int32_t n_fingers, const uint32_t *d_masks,
                                const uint32_t *d_counts, int32_t n_poses, const cf_score_params *prm,
                                int32_t *d_tuples, uint8_t *d_fingers, cf_stream stream) {
    if (prm && prm->tuples_given) return fail(CF_EINVAL, "cf_sample_tuples needs tuples_given = 0");
    ScoreArgs a;
    int rc = fill_score_args(obj, n_fingers, d_masks, d_counts, n_poses, prm, d_tuples, d_fingers,
                             (float *)d_tuples, (uint8_t *)d_tuples, &a);
    if (rc) return rc;
    if (n_poses == 0) return CF_OK;
    CF_TRY(launch_sample(a, (cudaStream_t)stream), "launch k_sample_tuples");
    return CF_OK;
}

// ---------------------------------------------------------------------------
// scoring without allocation: the work counter lives in a static device array
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned int g_noalloc_scratch[CF_NOALLOC_SCRATCH_BYTES / sizeof(unsigned int)];

std::mutex g_noalloc_mu;
unsigned int *g_noalloc_addr[64] = {};  // device address of g_noalloc_scratch, per device

// Device address of the scratch array on the current device (looked up once
// per device; the host-side symbol is not a device address).
int noalloc_scratch(unsigned int **out) {
    int dev = 0;
    CF_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(CF_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        unsigned int *p = nullptr;
        CF_TRY(cudaGetSymbolAddress((void **)&p, g_noalloc_scratch), "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return CF_OK;
}

}  // namespace

extern "C" int cf_score_tuples_noalloc(const cf_points *obj, int32_t n_fingers, const uint32_t *d_masks,
                                       const uint32_t *d_counts, int32_t n_poses, const cf_score_params *prm,
                                       int32_t *d_tuples, uint8_t *d_fingers, float *d_margin, uint8_t *d_accept,
                                       cf_stream stream) {
    ScoreArgs a;
    int rc = fill_score_args(obj, n_fingers, d_masks, d_counts, n_poses, prm, d_tuples, d_fingers, d_margin,
                             d_accept, &a);
    if (rc) return rc;
    // global scratch of the scoring kernels: none today (sampling stages each pose's masks in shared
    // memory; the lane scorer hands out tuples from per-block shared-memory counters), so nothing is
    // cleared; a kernel that needs some takes it from the static array, within its size
    const size_t need = 0;
    if (need > (size_t)CF_NOALLOC_SCRATCH_BYTES)
        return fail(CF_EINVAL, "scratch need %zu B exceeds the %d B no-allocation scratch", need,
                    CF_NOALLOC_SCRATCH_BYTES);
    unsigned int *scratch = nullptr;
    if ((rc = noalloc_scratch(&scratch))) return rc;
    if (n_poses == 0) return CF_OK;
    a.work = scratch;
    CF_TRY(launch_score(a, (cudaStream_t)stream), "launch k_sample_tuples / k_score_tuples");
    return CF_OK;
}

// ---------------------------------------------------------------------------
// batch: many objects, one launch per kernel variant, replayed as a CUDA graph
// ---------------------------------------------------------------------------
struct cf_batch {
    int dev = 0;
    cudaStream_t st = nullptr;          // internal stream the graph runs on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *d_block = nullptr;            // descriptors, prefix sums, the query work counter
    QueryDesc *d_qdescs = nullptr;      // every object's query
    int n_q = 0, q_items = 0;
    unsigned int *d_qwork = nullptr;    // 2 words: the query kernel's item counter (left zero by each launch)
    struct SGroup { ScoreArgs launch; ScoreArgs *d_descs; long long *d_tuple0; int n; long long tuples; };
    std::vector<SGroup> sgroups;        // one scoring launch per (k, K)
    ScoreArgs *d_sdescs = nullptr;      // all items, for sampling
    long long *d_pose0 = nullptr;
    int n_items = 0;
    long long total_poses = 0;
    size_t sample_smem = 0;
    std::vector<FieldGeom> geoms;
    FieldGeom *d_geoms = nullptr;
    int launches = 0;
    int ppb = 4;                        // query poses per item (the tuning at creation)
};

extern "C" int cf_batch_create(const cf_batch_item *items, int32_t n_items, cf_batch **out) {
    if (!items || !out || n_items < 1) return fail(CF_EINVAL, "items / out NULL or n_items < 1");
    std::vector<ScoreArgs> sargs(n_items);
    std::vector<int> geom_of(n_items);
    cf_batch *b = new cf_batch();
    CF_TRY(cudaGetDevice(&b->dev), "cudaGetDevice");
    b->ppb = current_tuning().query_ppb;
    std::vector<const cf_field *> fields;
    for (int i = 0; i < n_items; ++i) {
        const cf_batch_item &it = items[i];
        if (!it.field) { delete b; return fail(CF_EINVAL, "item %d: field is NULL", i); }
        if (it.prm.tuples_given) { delete b; return fail(CF_EINVAL, "item %d: batches sample their own tuples", i); }
        if (it.field->table_words == 0) { delete b; return fail(CF_EINVAL, "item %d: empty field", i); }
        if (it.field->geom.patches) {
            delete b;
            return fail(CF_EINVAL, "item %d: a patch field's domains need cf_merge_domains before sampling", i);
        }
        int rc = check_points(&it.obj);
        if (!rc) rc = fill_score_args(&it.obj, it.field->F, it.d_masks, it.d_counts, it.n_poses, &it.prm, it.d_tuples,
                                      it.d_fingers, it.d_margin, it.d_accept, &sargs[i]);
        if (rc) { delete b; return fail(rc, "item %d: %s", i, t_err.c_str()); }
        if (it.n_poses > 0 && (!it.d_poses || !it.d_counts || !it.d_masks)) {
            delete b;
            return fail(CF_EINVAL, "item %d: poses / masks / counts NULL", i);
        }
        int gi = -1;
        for (size_t f = 0; f < fields.size(); ++f)
            if (fields[f] == it.field) gi = (int)f;
        if (gi < 0) {
            gi = (int)fields.size();
            fields.push_back(it.field);
            b->geoms.push_back(it.field->geom);
        }
        geom_of[i] = gi;
    }
    // the query: every object in one persistent launch, items = (object, block of ppb poses)
    std::vector<QueryDesc> qdesc_all;
    long long q_items = 0;
    for (int i = 0; i < n_items; ++i) {
        if (items[i].n_poses == 0) continue;
        QueryDesc d;
        memset(&d, 0, sizeof d);
        d.obj = items[i].obj;
        d.poses = items[i].d_poses;
        d.P = items[i].n_poses;
        d.W = (items[i].obj.n + 31) / 32;
        d.masks = items[i].d_masks;
        d.counts = items[i].d_counts;
        d.table = items[i].field->d_table;
        d.geom = geom_of[i];
        d.block0 = (int)q_items;
        q_items += query_blocks(d.P, b->ppb);
        qdesc_all.push_back(d);
    }
    if (q_items >= INT_MAX) { delete b; return fail(CF_EINVAL, "the batch holds >= 2^31 query items"); }
    b->n_q = (int)qdesc_all.size();
    b->q_items = (int)q_items;
    // sampling: one launch over every pose; scoring: one launch per (k, K) (the LP lane layout)
    std::vector<long long> pose0(n_items + 1, 0);
    size_t smem = 0;
    for (int i = 0; i < n_items; ++i) {
        pose0[i + 1] = pose0[i] + sargs[i].P;
        smem = std::max(smem, score_smem_bytes(sargs[i].F, sargs[i].W, sargs[i].T, sargs[i].k, true));
    }
    b->total_poses = pose0[n_items];
    b->sample_smem = smem;
    std::vector<int> skeys;
    for (int i = 0; i < n_items; ++i) {
        const int key = sargs[i].k * 100 + sargs[i].K;
        if (std::find(skeys.begin(), skeys.end(), key) == skeys.end()) skeys.push_back(key);
    }
    std::vector<ScoreArgs> sdesc_all;
    std::vector<long long> tuple0_all;
    std::vector<size_t> s_off, t_off;
    for (int key : skeys) {
        cf_batch::SGroup sg{};
        const size_t so = sdesc_all.size(), to = tuple0_all.size();
        long long tuples = 0;
        for (int i = 0; i < n_items; ++i) {
            if (sargs[i].k * 100 + sargs[i].K != key) continue;
            tuple0_all.push_back(tuples);
            tuples += (long long)sargs[i].P * sargs[i].T;
            sdesc_all.push_back(sargs[i]);
            sg.launch = sargs[i];
        }
        s_off.push_back(so);
        t_off.push_back(to);
        tuple0_all.push_back(tuples);
        sg.n = (int)(sdesc_all.size() - so);
        sg.tuples = tuples;
        if (tuples >= (1LL << 32)) { delete b; return fail(CF_EINVAL, "a score group holds >= 2^32 tuples"); }
        b->sgroups.push_back(sg);
    }
    // one device block: geoms | query descs | score descs (grouped) | sample descs (all) | pose0 | tuple0 | counter
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_geom = 0, o_q = al(o_geom + sizeof(FieldGeom) * b->geoms.size());
    const size_t o_s = al(o_q + sizeof(QueryDesc) * std::max<size_t>(1, qdesc_all.size()));
    const size_t o_sa = al(o_s + sizeof(ScoreArgs) * std::max<size_t>(1, sdesc_all.size()));
    const size_t o_p0 = al(o_sa + sizeof(ScoreArgs) * n_items);
    const size_t o_t0 = al(o_p0 + sizeof(long long) * pose0.size());
    const size_t o_w = al(o_t0 + sizeof(long long) * std::max<size_t>(1, tuple0_all.size()));
    const size_t total = al(o_w + 2 * sizeof(unsigned int));
    CF_TRY(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking), "stream");
    CF_TRY(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming), "event");
    CF_TRY(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming), "event");
    int rc = pool_alloc(&b->d_block, total, b->st, "alloc batch");
    if (rc) { cf_batch_destroy(b); return rc; }
    char *base = (char *)b->d_block;
    b->d_geoms = (FieldGeom *)(base + o_geom);
    b->d_qdescs = (QueryDesc *)(base + o_q);
    b->d_sdescs = (ScoreArgs *)(base + o_sa);
    b->d_pose0 = (long long *)(base + o_p0);
    b->d_qwork = (unsigned int *)(base + o_w);
    for (size_t g = 0; g < b->sgroups.size(); ++g) {
        b->sgroups[g].d_descs = (ScoreArgs *)(base + o_s) + s_off[g];
        b->sgroups[g].d_tuple0 = (long long *)(base + o_t0) + t_off[g];
    }
    std::vector<char> img(total, 0);  // the work counter starts at zero
    memcpy(img.data() + o_geom, b->geoms.data(), sizeof(FieldGeom) * b->geoms.size());
    if (!qdesc_all.empty()) memcpy(img.data() + o_q, qdesc_all.data(), sizeof(QueryDesc) * qdesc_all.size());
    if (!sdesc_all.empty()) memcpy(img.data() + o_s, sdesc_all.data(), sizeof(ScoreArgs) * sdesc_all.size());
    memcpy(img.data() + o_sa, sargs.data(), sizeof(ScoreArgs) * n_items);
    memcpy(img.data() + o_p0, pose0.data(), sizeof(long long) * pose0.size());
    memcpy(img.data() + o_t0, tuple0_all.data(), sizeof(long long) * tuple0_all.size());
    cudaError_t e = cudaMemcpyAsync(b->d_block, img.data(), total, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) { cf_batch_destroy(b); return cuda_fail(e, "upload batch"); }
    b->n_items = n_items;
    b->launches = (b->q_items > 0 ? 1 : 0) + (b->total_poses > 0 ? 1 : 0) + (int)b->sgroups.size();
    *out = b;
    return CF_OK;
}

namespace {
int batch_enqueue(cf_batch *b, cudaStream_t st) {
    if (b->q_items > 0)
        CF_TRY(launch_query_batch(b->d_qdescs, b->d_geoms, b->n_q, b->q_items, b->ppb, b->d_qwork, st), "batch query");
    if (b->total_poses > 0)
        CF_TRY(launch_sample_batch(b->d_sdescs, b->d_pose0, b->n_items, b->total_poses, b->sample_smem, st),
               "batch sample");
    for (const auto &sg : b->sgroups)
        if (sg.tuples > 0)
            CF_TRY(launch_score_batch(sg.launch, sg.d_descs, sg.d_tuple0, sg.n, sg.tuples, st), "batch score");
    return CF_OK;
}
}  // namespace

extern "C" int cf_batch_run(cf_batch *b, cf_stream stream) {
    if (!b) return fail(CF_EINVAL, "batch is NULL");
    cudaStream_t caller = (cudaStream_t)stream;
    CF_TRY(cudaEventRecord(b->ev_in, caller), "event record");
    CF_TRY(cudaStreamWaitEvent(b->st, b->ev_in, 0), "stream wait");
    if (!b->exec) {
        cudaGraph_t graph = nullptr;
        CF_TRY(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal), "begin capture");
        const int rc = batch_enqueue(b, b->st);
        const cudaError_t e = cudaStreamEndCapture(b->st, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "end capture");
        const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) { b->exec = nullptr; return cuda_fail(ei, "graph instantiate"); }
    }
    CF_TRY(cudaGraphLaunch(b->exec, b->st), "graph launch");
    CF_TRY(cudaEventRecord(b->ev_out, b->st), "event record");
    CF_TRY(cudaStreamWaitEvent(caller, b->ev_out, 0), "stream wait");
    return CF_OK;
}

extern "C" int cf_batch_launches(const cf_batch *b, int32_t *n_launches, int32_t *n_groups) {
    if (!b) return fail(CF_EINVAL, "batch is NULL");
    if (n_launches) *n_launches = b->launches;
    if (n_groups) *n_groups = (b->q_items > 0 ? 1 : 0) + (int)b->sgroups.size();
    return CF_OK;
}

extern "C" int cf_batch_destroy(cf_batch *b) {
    if (!b) return CF_OK;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->d_block) cudaFreeAsync(b->d_block, b->st);
    if (b->st) {
        cudaStreamSynchronize(b->st);
        cudaStreamDestroy(b->st);
    }
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    delete b;
    return CF_OK;
}

// ---------------------------------------------------------------------------
// object placement (Sec. 5.2) and preprocessing (Sec. 5.1)
// ---------------------------------------------------------------------------
namespace {
// exclusive set-bit prefix per table chunk, built on first use and kept with the field
int field_prefix(cf_field *fd) {
    if (fd->d_prefix || fd->table_words == 0) return CF_OK;
    const int n = (int)((fd->table_words + kChunkWords - 1) / kChunkWords);
    unsigned long long *d_counts = nullptr;
    int rc = pool_alloc((void **)&d_counts, sizeof(unsigned long long) * n, fd->st, "alloc chunk counts");
    if (rc) return rc;
    std::vector<unsigned long long> h(n + 1, 0);
    cudaError_t e = launch_chunk_counts(fd->d_table, fd->table_words, d_counts, fd->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data() + 1, d_counts, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, fd->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(fd->st);
    cudaFreeAsync(d_counts, fd->st);
    if (e != cudaSuccess) return cuda_fail(e, "chunk counts");
    for (int i = 0; i < n; ++i) h[i + 1] += h[i];
    if ((rc = pool_alloc((void **)&fd->d_prefix, sizeof(unsigned long long) * (n + 1), fd->st, "alloc prefix"))) return rc;
    CF_TRY(cudaMemcpyAsync(fd->d_prefix, h.data(), sizeof(unsigned long long) * (n + 1), cudaMemcpyHostToDevice, fd->st),
           "copy prefix");
    CF_TRY(cudaStreamSynchronize(fd->st), "prefix upload");
    fd->n_chunks = n;
    fd->n_codes = h[n];
    return CF_OK;
}
}  // namespace

extern "C" int cf_place(const cf_field *field, const cf_points *obj, int32_t n_poses, const cf_place_params *prm,
                        float *d_poses, cf_stream stream) {
    if (!prm) return fail(CF_EINVAL, "NULL argument");
    if (n_poses < 0) return fail(CF_EINVAL, "n_poses < 0");
    if (n_poses == 0) return CF_OK;
    if (!d_poses) return fail(CF_EINVAL, "poses pointer is NULL");
    PlaceArgs a;
    memset(&a, 0, sizeof a);
    a.P = n_poses;
    a.seed_lo = (uint32_t)prm->seed;
    a.seed_hi = (uint32_t)(prm->seed >> 32);
    a.pose_base = prm->pose_base;
    for (int c = 0; c < 3; ++c) {
        a.centroid[c] = prm->centroid[c];
        a.g[c] = prm->g[c];
        a.up[c] = prm->up[c];
    }
    a.d_lo = prm->d_lo;
    a.d_hi = prm->d_hi;
    a.poses = d_poses;
    const bool ex = prm->exhaustive != 0;
    if (ex) {
        if (!field) return fail(CF_EINVAL, "exhaustive placement needs the field");
        int rc = check_points(obj);
        if (rc) return rc;
        if (obj->n < 1) return fail(CF_EINVAL, "exhaustive placement needs object points");
        cf_field *fd = const_cast<cf_field *>(field);
        if ((rc = field_prefix(fd))) return rc;
        if (fd->n_codes == 0) return fail(CF_EINVAL, "the field holds no code");
        a.table = fd->d_table;
        a.prefix = fd->d_prefix;
        a.n_chunks = fd->n_chunks;
        a.n_codes = fd->n_codes;
        a.table_words = fd->table_words;
        a.g_field = fd->geom;
        a.obj = *obj;
    } else if (!(prm->d_hi >= prm->d_lo) || !isfinite(prm->d_lo) || !isfinite(prm->d_hi)) {
        return fail(CF_EINVAL, "d_lo / d_hi must be finite with d_lo <= d_hi");
    }
    CF_TRY(launch_place(a, ex, (cudaStream_t)stream), "launch placement");
    return CF_OK;
}

extern "C" int cf_concave_filter(const cf_points *obj, const cf_sdf *sdf, float side, float tau, uint8_t *d_keep,
                                 float *d_out, int32_t *d_n_out, cf_stream stream) {
    int rc = check_points(obj);
    if (rc) return rc;
    if (!sdf) return fail(CF_EINVAL, "sdf is NULL");
    if (!(side > 0.f) || !isfinite(side) || !(tau >= 0.f) || !isfinite(tau))
        return fail(CF_EINVAL, "side must be > 0 and tau >= 0");
    if (obj->n == 0) return CF_OK;
    if (!d_keep || !d_n_out) return fail(CF_EINVAL, "keep / n_out pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int *counts = nullptr;
    const int blocks = (obj->n + 1023) / 1024;
    if ((rc = pool_alloc((void **)&counts, sizeof(unsigned int) * blocks, st, "alloc block counts"))) return rc;
    cudaError_t e = launch_concave(*obj, sdf->g, side, tau, d_keep, counts, d_out, d_n_out, st);
    cudaError_t e2 = cudaFreeAsync(counts, st);
    if (e != cudaSuccess) return cuda_fail(e, "launch k_concave / k_compact");
    if (e2 != cudaSuccess) return cuda_fail(e2, "free block counts");
    return CF_OK;
}

// ---------------------------------------------------------------------------
// launch shapes and the autotuner
// ---------------------------------------------------------------------------
namespace {
bool tuning_valid(const cf_tuning *t) {
    const int p = t->query_poses_per_block, r = t->score_refill, s = t->score_blocks_per_sm;
    return p >= 1 && p <= kMaxPosesPerBlock && (r == 4 || r == 8 || r == 16) && s >= 0 && s <= 3;
}
}  // namespace

extern "C" int cf_get_tuning(cf_tuning *out) {
    if (!out) return fail(CF_EINVAL, "NULL argument");
    const Tuning t = current_tuning();
    out->query_poses_per_block = t.query_ppb;
    out->score_refill = t.score_refill;
    out->score_blocks_per_sm = t.score_bpsm;
    return CF_OK;
}

extern "C" int cf_set_tuning(const cf_tuning *t) {
    if (!t) return fail(CF_EINVAL, "NULL argument");
    if (!tuning_valid(t)) return fail(CF_EINVAL, "tuning out of range");
    int dev = 0;
    CF_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(CF_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[dev] = Tuning{t->query_poses_per_block, t->score_refill, t->score_blocks_per_sm};
    g_tune_set[dev] = true;
    return CF_OK;
}

extern "C" int cf_autotune(const cf_batch_item *items, int32_t n_items, int32_t reps, cf_tuning *out,
                           double *best_ms) {
    if (!items || n_items < 1) return fail(CF_EINVAL, "no items");
    if (reps < 1 || reps > 64) return fail(CF_EINVAL, "reps=%d not in [1,64]", reps);
    for (int i = 0; i < n_items; ++i) {
        if (!items[i].field || items[i].prm.tuples_given) return fail(CF_EINVAL, "item %d: no field or tuples given", i);
        if (items[i].field->geom.patches) return fail(CF_EINVAL, "item %d: patch fields are not tuned", i);
    }
    cf_tuning saved;
    int rc = cf_get_tuning(&saved);
    if (rc) return rc;
    cudaStream_t st = nullptr;
    CF_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // time one full pass of `phase` (0: queries, 1: sampling + scoring) under tuning t; median of reps
    auto run = [&](const cf_tuning &t, int phase, double *ms) -> int {
        int r = cf_set_tuning(&t);
        if (r) return r;
        std::vector<double> v;
        for (int rep = 0; rep < reps + 1; ++rep) {  // the first pass warms up
            CF_TRY(cudaEventRecord(e0, st), "event");
            for (int i = 0; i < n_items && !r; ++i) {
                const cf_batch_item &it = items[i];
                if (phase == 0)
                    r = cf_query_domains(it.field, &it.obj, it.d_poses, it.n_poses, it.d_masks, it.d_counts, st);
                else
                    r = cf_score_tuples(&it.obj, it.field->F, it.d_masks, it.d_counts, it.n_poses, &it.prm, it.d_tuples,
                                        it.d_fingers, it.d_margin, it.d_accept, st);
            }
            if (r) return r;
            CF_TRY(cudaEventRecord(e1, st), "event");
            CF_TRY(cudaEventSynchronize(e1), "autotune run");
            float f = 0.f;
            cudaEventElapsedTime(&f, e0, e1);
            if (rep > 0) v.push_back(f);
        }
        std::sort(v.begin(), v.end());
        *ms = v[v.size() / 2];
        return CF_OK;
    };
    cf_tuning best = saved;
    double bq = 1e300, bs = 1e300;
    // 4, 8, 16, and the largest count that lets each lane keep one (pose, slot) word: 32 / slots
    std::vector<int> ppbs = {4, 8, 16};
    for (int i = 0; i < n_items; ++i) {
        const int own = 32 / std::max(1, items[i].field->geom.F);
        if (own >= 2 && own <= kMaxPosesPerBlock && std::find(ppbs.begin(), ppbs.end(), own) == ppbs.end())
            ppbs.push_back(own);
    }
    for (int ppb : ppbs) {
        cf_tuning t = saved;
        t.query_poses_per_block = ppb;
        double ms = 0;
        if ((rc = run(t, 0, &ms))) break;
        if (ms < bq) { bq = ms; best.query_poses_per_block = ppb; }
    }
    for (int refill : {4, 8, 16}) {
        if (rc) break;
        for (int bpsm : {0, 1, 2}) {
            cf_tuning t = best;
            t.score_refill = refill;
            t.score_blocks_per_sm = bpsm;
            double ms = 0;
            if ((rc = run(t, 1, &ms))) break;
            if (ms < bs) { bs = ms; best.score_refill = refill; best.score_blocks_per_sm = bpsm; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (rc) {
        cf_set_tuning(&saved);
        return rc;
    }
    if ((rc = cf_set_tuning(&best))) return rc;
    if (out) *out = best;
    if (best_ms) { best_ms[0] = bq; best_ms[1] = bs; }
    return CF_OK;
}

// ---------------------------------------------------------------------------
// plan: one object request from host buffers
// ---------------------------------------------------------------------------
// A plan runs a request's query, sampling and scoring as one launch each; its
// inputs go up, and its results come back, on a second stream: the tuples while
// the scoring kernel runs, the margins and flags after it.  Or only the accepted
// tuples come back (cf_plan_run_host_accepted), gathered first on the device.

// Ordered gather of the accepted tuples into cf_grasp records, in chunks of kGatherChunk
// tuples: count per chunk, an exclusive scan of the counts (one block), then each chunk
// writes its records from its offset, in tuple order.
constexpr int kGatherChunk = 4096;
constexpr int kGatherThreads = 256;

__global__ void __launch_bounds__(kGatherThreads) k_count_accepted(const uint8_t *__restrict__ accept, size_t n,
                                                                   unsigned *__restrict__ cnt) {
    const size_t c0 = (size_t)blockIdx.x * kGatherChunk, c1 = c0 + kGatherChunk < n ? c0 + kGatherChunk : n;
    unsigned c = 0;
    for (size_t u = c0 + threadIdx.x; u < c1; u += kGatherThreads) c += accept[u] != 0;
    c = __reduce_add_sync(0xffffffffu, c);
    __shared__ unsigned s_w[kGatherThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < kGatherThreads / 32; ++w) t += s_w[w];
        cnt[blockIdx.x] = t;
    }
}

// In place: cnt[b] <- the sum of cnt[0 .. b) (one block).
__global__ void __launch_bounds__(1024) k_scan_counts(unsigned *cnt, int nb) {
    block_exclusive_scan_1024(cnt, nb, nullptr);
}

__global__ void __launch_bounds__(kGatherThreads) k_write_accepted(const uint8_t *__restrict__ accept,
                                                                   const int32_t *__restrict__ tuples,
                                                                   const float *__restrict__ margin, size_t n, int T,
                                                                   int k, const unsigned *__restrict__ off,
                                                                   cf_grasp *__restrict__ out) {
    __shared__ unsigned s_w[kGatherThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t c0 = (size_t)blockIdx.x * kGatherChunk, c1 = c0 + kGatherChunk < n ? c0 + kGatherChunk : n;
    unsigned run = off[blockIdx.x];
    for (size_t t0 = c0; t0 < c1; t0 += kGatherThreads) {
        const size_t u = t0 + threadIdx.x;
        const bool acc = u < c1 && accept[u] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, acc);
        __syncthreads();  // the previous tile's counts have been read
        if (lane == 0) s_w[warp] = __popc(bal);
        __syncthreads();
        unsigned before = 0, tile = 0;
        for (int w = 0; w < kGatherThreads / 32; ++w) {
            before += w < warp ? s_w[w] : 0u;
            tile += s_w[w];
        }
        if (acc) {
            cf_grasp g;
            g.pose = (int32_t)(u / (size_t)T);
            g.margin = margin[u];
#pragma unroll
            for (int q = 0; q < CF_MAX_K; ++q) g.point[q] = q < k ? tuples[u * k + q] : -1;
            out[run + before + __popc(bal & ((1u << lane) - 1u))] = g;
        }
        run += tile;
    }
}

constexpr int kPlanEvents = 2;  // tuples sampled; tuples scored

struct cf_plan {
    int n_max = 0, p_max = 0, T = 0, k = 0, F = 0;
    void *d_block = nullptr;
    float *d_soa = nullptr, *d_poses = nullptr, *d_margin = nullptr;
    uint32_t *d_masks = nullptr, *d_counts = nullptr;
    int32_t *d_tuples = nullptr;
    uint8_t *d_fingers = nullptr, *d_accept = nullptr;
    unsigned long long *d_n_acc = nullptr;  // accepted tuples of the request
    cf_grasp *d_grasps = nullptr;           // the gathered accepted tuples
    unsigned *d_chunk = nullptr;            // accepted tuples per gather chunk, then their offsets
    unsigned long long *h_n_acc = nullptr;  // page-locked copy
    cudaStream_t copy_st = nullptr;
    cudaEvent_t ev[kPlanEvents] = {};
    cudaEvent_t ev_in = nullptr;            // the request's inputs are on the device
};

extern "C" int cf_plan_create(int32_t n_fingers, int32_t n_max, int32_t p_max, const cf_score_params *prm,
                              cf_plan **out) {
    if (!prm || !out) return fail(CF_EINVAL, "NULL argument");
    if (n_fingers < 1 || n_fingers > CF_MAX_FINGERS) return fail(CF_EINVAL, "n_fingers=%d not in [1,%d]", n_fingers,
                                                                 CF_MAX_FINGERS);
    if (n_max < 1 || p_max < 1) return fail(CF_EINVAL, "n_max and p_max must be >= 1");
    if (prm->n_tuples < 1 || prm->k < 1 || prm->k > CF_MAX_K) return fail(CF_EINVAL, "bad T or k");
    cf_plan *pl = new cf_plan();
    pl->n_max = n_max; pl->p_max = p_max; pl->T = prm->n_tuples; pl->k = prm->k; pl->F = n_fingers;
    const size_t W = (size_t)(n_max + 31) / 32, P = (size_t)p_max, PT = P * pl->T;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_soa = al(sizeof(float) * 6 * n_max), b_pose = al(sizeof(float) * 12 * P),
                 b_mask = al(sizeof(uint32_t) * P * pl->F * W), b_cnt = al(sizeof(uint32_t) * P * pl->F),
                 b_tup = al(sizeof(int32_t) * PT * pl->k), b_fin = al(PT * pl->k), b_mar = al(sizeof(float) * PT),
                 b_acc = al(PT), b_nacc = 256, b_grasp = al(sizeof(cf_grasp) * PT),
                 b_chunk = al(sizeof(unsigned) * ((PT + kGatherChunk - 1) / kGatherChunk + 1));
    const size_t total = b_soa + b_pose + b_mask + b_cnt + b_tup + b_fin + b_mar + b_acc + b_nacc + b_grasp + b_chunk;
    cudaError_t e = cudaMalloc(&pl->d_block, total);
    if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaMalloc(plan)"); }
    auto undo = [&](cudaError_t err, const char *what) {
        cf_plan_destroy(pl);
        return cuda_fail(err, what);
    };
    if ((e = cudaMallocHost((void **)&pl->h_n_acc, sizeof(unsigned long long))) != cudaSuccess)
        return undo(e, "cudaMallocHost(plan)");
    if ((e = cudaStreamCreateWithFlags(&pl->copy_st, cudaStreamNonBlocking)) != cudaSuccess)
        return undo(e, "cudaStreamCreate(plan)");
    for (int c = 0; c < kPlanEvents; ++c)
        if ((e = cudaEventCreateWithFlags(&pl->ev[c], cudaEventDisableTiming)) != cudaSuccess)
            return undo(e, "cudaEventCreate(plan)");
    if ((e = cudaEventCreateWithFlags(&pl->ev_in, cudaEventDisableTiming)) != cudaSuccess)
        return undo(e, "cudaEventCreate(plan)");
    char *p = (char *)pl->d_block;
    pl->d_soa = (float *)p; p += b_soa;
    pl->d_poses = (float *)p; p += b_pose;
    pl->d_masks = (uint32_t *)p; p += b_mask;
    pl->d_counts = (uint32_t *)p; p += b_cnt;
    pl->d_tuples = (int32_t *)p; p += b_tup;
    pl->d_fingers = (uint8_t *)p; p += b_fin;
    pl->d_margin = (float *)p; p += b_mar;
    pl->d_accept = (uint8_t *)p; p += b_acc;
    pl->d_n_acc = (unsigned long long *)p; p += b_nacc;
    pl->d_grasps = (cf_grasp *)p; p += b_grasp;
    pl->d_chunk = (unsigned *)p;
    *out = pl;
    return CF_OK;
}

namespace {
// The request's inputs up, domains, sampling and scoring queued on `st`; the sampled tuples
// go back to h_tuples (when given) on the copy stream while the scoring kernel runs.
int plan_enqueue(cf_plan *pl, const cf_field *fd, const float *h_soa, int32_t n, const float *h_poses, int32_t n_poses,
                 const cf_score_params *prm, int32_t *h_tuples, cf_stream stream) {
    if (!pl || !fd || !prm || (n > 0 && !h_soa) || (n_poses > 0 && !h_poses)) return fail(CF_EINVAL, "NULL argument");
    if (fd->F > pl->F) return fail(CF_EINVAL, "field has %d fingers, plan holds %d", fd->F, pl->F);
    if (fd->geom.patches) return fail(CF_EINVAL, "a plan samples from finger domains: not a patch field");
    if (n < 0 || n > pl->n_max) return fail(CF_EINVAL, "n=%d not in [0,%d]", n, pl->n_max);
    if (n_poses < 0 || n_poses > pl->p_max) return fail(CF_EINVAL, "n_poses=%d not in [0,%d]", n_poses, pl->p_max);
    if (prm->n_tuples != pl->T || prm->k != pl->k) return fail(CF_EINVAL, "T / k differ from the plan's");
    if (prm->tuples_given) return fail(CF_EINVAL, "a plan samples its own tuples");
    cudaStream_t st = (cudaStream_t)stream;
    // the inputs go up on the copy stream, which holds no earlier work of the plan (each call ends by
    // waiting for both streams), so they overlap whatever the caller's stream is still running (the
    // field build); the query waits for them
    if (n > 0)
        CF_TRY(cudaMemcpyAsync(pl->d_soa, h_soa, sizeof(float) * 6 * n, cudaMemcpyHostToDevice, pl->copy_st),
               "H2D points");
    if (n_poses > 0)
        CF_TRY(cudaMemcpyAsync(pl->d_poses, h_poses, sizeof(float) * 12 * n_poses, cudaMemcpyHostToDevice,
                               pl->copy_st), "H2D poses");
    CF_TRY(cudaEventRecord(pl->ev_in, pl->copy_st), "event record");
    CF_TRY(cudaStreamWaitEvent(st, pl->ev_in, 0), "stream wait");
    CF_TRY(cudaMemsetAsync(pl->d_n_acc, 0, sizeof(unsigned long long), st), "memset accept count");
    cf_points obj{pl->d_soa, pl->d_soa + n, pl->d_soa + 2 * n, pl->d_soa + 3 * n, pl->d_soa + 4 * n,
                  pl->d_soa + 5 * n, n};
    const int F = fd->F, T = pl->T, k = pl->k;
    int rc = cf_query_domains(fd, &obj, pl->d_poses, n_poses, pl->d_masks, pl->d_counts, stream);
    if (rc) return rc;
    ScoreArgs a;
    rc = fill_score_args(&obj, F, pl->d_masks, pl->d_counts, n_poses, prm, pl->d_tuples, pl->d_fingers, pl->d_margin,
                         pl->d_accept, &a);
    if (rc) return rc;
    a.n_accept = pl->d_n_acc;
    const size_t pt = (size_t)n_poses * T;
    if (n_poses > 0) CF_TRY(launch_sample(a, st), "launch k_sample_tuples");
    CF_TRY(cudaEventRecord(pl->ev[0], st), "event record");
    CF_TRY(cudaStreamWaitEvent(pl->copy_st, pl->ev[0], 0), "stream wait");
    if (pt > 0 && h_tuples)
        CF_TRY(cudaMemcpyAsync(h_tuples, pl->d_tuples, sizeof(int32_t) * pt * k, cudaMemcpyDeviceToHost, pl->copy_st),
               "D2H tuples");
    if (n_poses > 0) {
        a.tuples_given = 1;  // sampled above
        CF_TRY(launch_score(a, st), "launch k_score_lanes");
    }
    return CF_OK;
}
}  // namespace

extern "C" int cf_plan_run_host(cf_plan *pl, const cf_field *fd, const float *h_soa, int32_t n, const float *h_poses,
                                int32_t n_poses, const cf_score_params *prm, int32_t *h_tuples, float *h_margin,
                                uint8_t *h_accept, int64_t *h_n_accepted, cf_stream stream) {
    // the tuples (most of the result bytes) go back while the scoring kernel runs; margins and flags follow
    int rc = plan_enqueue(pl, fd, h_soa, n, h_poses, n_poses, prm, h_tuples, stream);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t pt = (size_t)n_poses * pl->T;
    CF_TRY(cudaEventRecord(pl->ev[1], st), "event record");
    CF_TRY(cudaStreamWaitEvent(pl->copy_st, pl->ev[1], 0), "stream wait");
    if (pt > 0 && h_margin)
        CF_TRY(cudaMemcpyAsync(h_margin, pl->d_margin, sizeof(float) * pt, cudaMemcpyDeviceToHost, pl->copy_st),
               "D2H margin");
    if (pt > 0 && h_accept)
        CF_TRY(cudaMemcpyAsync(h_accept, pl->d_accept, pt, cudaMemcpyDeviceToHost, pl->copy_st), "D2H accept");
    CF_TRY(cudaMemcpyAsync(pl->h_n_acc, pl->d_n_acc, sizeof(unsigned long long), cudaMemcpyDeviceToHost, pl->copy_st),
           "D2H accept count");
    CF_TRY(cudaStreamSynchronize(pl->copy_st), "plan copies");
    CF_TRY(cudaStreamSynchronize(st), "plan run");
    if (h_n_accepted) *h_n_accepted = (int64_t)*pl->h_n_acc;
    return CF_OK;
}

extern "C" int cf_plan_run_host_accepted(cf_plan *pl, const cf_field *fd, const float *h_soa, int32_t n,
                                         const float *h_poses, int32_t n_poses, const cf_score_params *prm,
                                         cf_grasp *h_grasps, int64_t cap, int64_t *h_n_accepted, cf_stream stream) {
    if (cap < 0 || (cap > 0 && !h_grasps)) return fail(CF_EINVAL, "bad grasp buffer");
    int rc = plan_enqueue(pl, fd, h_soa, n, h_poses, n_poses, prm, nullptr, stream);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t pt = (size_t)n_poses * pl->T;
    const unsigned nb = (unsigned)((pt + kGatherChunk - 1) / kGatherChunk);
    if (nb > 0) {  // the accepted tuples gathered in order, on the device
        k_count_accepted<<<nb, kGatherThreads, 0, st>>>(pl->d_accept, pt, pl->d_chunk);
        CF_TRY(cudaGetLastError(), "launch k_count_accepted");
        k_scan_counts<<<1, 1024, 0, st>>>(pl->d_chunk, (int)nb);
        CF_TRY(cudaGetLastError(), "launch k_scan_counts");
        k_write_accepted<<<nb, kGatherThreads, 0, st>>>(pl->d_accept, pl->d_tuples, pl->d_margin, pt, pl->T, pl->k,
                                                        pl->d_chunk, pl->d_grasps);
        CF_TRY(cudaGetLastError(), "launch k_write_accepted");
    }
    CF_TRY(cudaMemcpyAsync(pl->h_n_acc, pl->d_n_acc, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st),
           "D2H accept count");
    CF_TRY(cudaStreamSynchronize(st), "plan run");
    const int64_t count = (int64_t)*pl->h_n_acc, m = count < cap ? count : cap;
    if (m > 0) {
        CF_TRY(cudaMemcpyAsync(h_grasps, pl->d_grasps, sizeof(cf_grasp) * (size_t)m, cudaMemcpyDeviceToHost, st),
               "D2H grasps");
        CF_TRY(cudaStreamSynchronize(st), "plan copies");
    }
    CF_TRY(cudaStreamSynchronize(pl->copy_st), "plan copies");
    if (h_n_accepted) *h_n_accepted = count;
    return CF_OK;
}

extern "C" int cf_plan_destroy(cf_plan *pl) {
    if (!pl) return CF_OK;
    if (pl->copy_st) cudaStreamSynchronize(pl->copy_st);
    for (int c = 0; c < kPlanEvents; ++c)
        if (pl->ev[c]) cudaEventDestroy(pl->ev[c]);
    if (pl->ev_in) cudaEventDestroy(pl->ev_in);
    if (pl->copy_st) cudaStreamDestroy(pl->copy_st);
    if (pl->h_n_acc) cudaFreeHost(pl->h_n_acc);
    if (pl->d_block) cudaFree(pl->d_block);
    delete pl;
    return CF_OK;
}

// ---------------------------------------------------------------------------
// reverse lookup + DLS IK (Sec. 5.5); object SDF grid and realization filter (Sec. 5.6)
// ---------------------------------------------------------------------------

extern "C" int cf_ik_dls(const cf_field *fd, const cf_points *obj, const float *d_poses, int32_t n_slots,
                         int32_t n_tuples, int32_t k, const int32_t *d_tuples, const uint8_t *d_fingers,
                         const uint8_t *d_accept, const cf_ik_params *prm, float *d_q, uint8_t *d_used,
                         float *d_contacts, int32_t *d_rtuples, float *d_resid, uint8_t *d_ok, cf_stream stream) {
    if (!fd || !prm) return fail(CF_EINVAL, "NULL argument");
    if (!fd->d_rep || !fd->d_qs || !fd->has_limits)
        return fail(CF_EINVAL, "the field needs joint limits and a representative table (want_rep)");
    int rc = check_points(obj);
    if (rc) return rc;
    if (n_slots < 0 || n_tuples < 1) return fail(CF_EINVAL, "n_slots < 0 or n_tuples < 1");
    if (k < 1 || k > CF_MAX_K || k > fd->F) return fail(CF_EINVAL, "k=%d not in [1,min(%d,F)]", k, CF_MAX_K);
    if (!(prm->lambda > 0.f) || !isfinite(prm->lambda)) return fail(CF_EINVAL, "lambda must be finite and > 0");
    if (!isfinite(prm->beta) || !isfinite(prm->tol_pos) || !isfinite(prm->tol_cos))
        return fail(CF_EINVAL, "beta / tolerances must be finite");
    if (prm->n_phase1 < 0 || prm->n_rounds < 0 || prm->n_phase2 < 0 || prm->n_phase1 > 4096 ||
        prm->n_rounds > 256 || prm->n_phase2 > 4096)
        return fail(CF_EINVAL, "iteration counts out of range");
    if (n_slots == 0) return CF_OK;
    if (!d_poses || !d_tuples || !d_fingers || !d_q || !d_used || !d_contacts || !d_rtuples || !d_resid || !d_ok)
        return fail(CF_EINVAL, "array pointer is NULL");
    DevState ds;
    if ((rc = device_state(&ds))) return rc;
    IkArgs a;
    memset(&a, 0, sizeof a);
    a.h = fd->hand;
    a.g = fd->geom;
    a.rep = fd->rep;
    a.qs = fd->d_qs;
    a.S = fd->S;
    a.obj = *obj;
    a.poses = d_poses;
    a.n = n_slots;
    a.T = n_tuples;
    a.k = k;
    a.tuples = d_tuples;
    a.fingers = d_fingers;
    a.accept = d_accept;
    a.beta = prm->beta;
    a.lambda = prm->lambda;
    a.tol_pos = prm->tol_pos;
    a.tol_cos = prm->tol_cos;
    a.n1 = prm->n_phase1;
    a.nr = prm->n_rounds;
    a.n2 = prm->n_phase2;
    a.q = d_q;
    a.used = d_used;
    const size_t nk = (size_t)n_slots * k;
    for (int i = 0; i < 6; ++i) a.cp[i] = d_contacts + i * nk;
    a.rtuples = d_rtuples;
    a.resid = d_resid;
    a.ok = d_ok;
    a.status = ds.status;
    // scratch: work list of accepted slots + its counter (stream-ordered)
    cudaStream_t st = (cudaStream_t)stream;
    void *scratch = nullptr;
    const size_t list_bytes = (sizeof(int) * (size_t)n_slots + 255) & ~(size_t)255;
    if ((rc = pool_alloc(&scratch, list_bytes + 256, st, "alloc IK work list"))) return rc;
    unsigned int *count = (unsigned int *)((char *)scratch + list_bytes);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = launch_ik(a, (int *)scratch, count, st);
    cudaError_t e2 = cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "launch k_ik_compact / k_ik_dls");
    if (e2 != cudaSuccess) return cuda_fail(e2, "free IK work list");
    return CF_OK;
}

extern "C" int cf_sdf_build(const cf_points *obj, const float lo[3], float h, const int32_t dims[3],
                            cf_stream stream, cf_sdf **out) {
    if (!out || !lo || !dims) return fail(CF_EINVAL, "NULL argument");
    int rc = check_points(obj);
    if (rc) return rc;
    if (!(h > 0.f) || !isfinite(h)) return fail(CF_EINVAL, "h must be finite and > 0");
    for (int c = 0; c < 3; ++c) {
        if (!isfinite(lo[c])) return fail(CF_EINVAL, "lo must be finite");
        if (dims[c] < 2 || dims[c] > 4096) return fail(CF_EINVAL, "dims[%d]=%d not in [2,4096]", c, dims[c]);
    }
    const int64_t nodes = (int64_t)dims[0] * dims[1] * dims[2];
    if (nodes > ((int64_t)1 << 31)) return fail(CF_EINVAL, "%lld grid nodes: too many", (long long)nodes);
    cf_sdf *s = new cf_sdf();
    s->st = (cudaStream_t)stream;
    cudaGetDevice(&s->dev);
    for (int c = 0; c < 3; ++c) { s->g.lo[c] = lo[c]; s->g.dims[c] = dims[c]; }
    s->g.h = h;
    s->g.inv_h = 1.f / h;
    s->nodes = nodes;
    if ((rc = pool_alloc((void **)&s->d_grid, sizeof(float) * (size_t)nodes, s->st, "alloc sdf grid"))) {
        delete s;
        return rc;
    }
    s->g.v = s->d_grid;
    cudaError_t e = launch_sdf(*obj, s->g, s->d_grid, s->st);
    if (e != cudaSuccess) {
        cudaFreeAsync(s->d_grid, s->st);
        delete s;
        return cuda_fail(e, "launch k_sdf_build");
    }
    *out = s;
    return CF_OK;
}

extern "C" int cf_sdf_copy(const cf_sdf *s, float *host, int64_t capacity) {
    if (!s || !host) return fail(CF_EINVAL, "NULL argument");
    if (capacity < s->nodes) return fail(CF_EINVAL, "capacity %lld < nodes %lld", (long long)capacity, (long long)s->nodes);
    CF_TRY(cudaStreamSynchronize(s->st), "sdf stream");
    CF_TRY(cudaMemcpy(host, s->d_grid, sizeof(float) * (size_t)s->nodes, cudaMemcpyDeviceToHost), "copy sdf");
    return CF_OK;
}

extern "C" int cf_sdf_destroy(cf_sdf *s) {
    if (!s) return CF_OK;
    if (s->d_grid) cudaFreeAsync(s->d_grid, s->st);
    delete s;
    return CF_OK;
}

extern "C" int cf_realize(const cf_field *fd, const cf_sdf *sdf, const float *d_poses, int32_t n_slots,
                          int32_t n_tuples, const cf_realize_params *prm, const uint8_t *d_gate_a,
                          const uint8_t *d_gate_b, float *d_q, const uint8_t *d_used, uint8_t *d_flags,
                          cf_stream stream) {
    if (!fd || !sdf || !prm) return fail(CF_EINVAL, "NULL argument");
    if (!fd->has_limits) return fail(CF_EINVAL, "the field's hand has no joint limits / radii");
    if (n_slots < 0 || n_tuples < 1) return fail(CF_EINVAL, "n_slots < 0 or n_tuples < 1");
    if (!(prm->axis_step > 0.f) || !isfinite(prm->axis_step)) return fail(CF_EINVAL, "axis_step must be > 0");
    if (!isfinite(prm->pen_margin)) return fail(CF_EINVAL, "pen_margin must be finite");
    if (n_slots == 0) return CF_OK;
    if (!d_poses || !d_q || !d_used || !d_flags) return fail(CF_EINVAL, "array pointer is NULL");
    RealizeArgs a;
    memset(&a, 0, sizeof a);
    a.h = fd->hand;
    a.sdf = sdf->g;
    a.poses = d_poses;
    a.n = n_slots;
    a.T = n_tuples;
    a.gate_a = d_gate_a;
    a.gate_b = d_gate_b;
    a.q = d_q;
    a.used = d_used;
    a.flags = d_flags;
    a.pen_margin = prm->pen_margin;
    a.seed_lo = (uint32_t)prm->seed;
    a.seed_hi = (uint32_t)(prm->seed >> 32);
    // capsules: links of positive radius and length, in (finger, link) order; axis samples at s / ns
    const int F = fd->F, J = fd->J;
    for (int f = 0; f < F; ++f)
        for (int j = 0; j < J; ++j) {
            const float *o = &fd->h_offset[3 * ((size_t)f * J + j)];
            const double len = sqrt((double)o[0] * o[0] + (double)o[1] * o[1] + (double)o[2] * o[2]);
            const float r = fd->h_radius[(size_t)f * J + j];
            if (!(r > 0.f) || !(len > 0.0)) {
                a.cap_of[f * J + j] = -1;
                continue;
            }
            const double ns = std::max(1.0, ceil(len / (double)prm->axis_step));
            if (ns > 32767.0) return fail(CF_EINVAL, "axis_step too small: %g samples on one link", ns);
            const int cid = a.n_caps++;
            a.cap_of[f * J + j] = (int8_t)cid;
            a.cap_f[cid] = (uint8_t)f;
            a.cap_ns[cid] = (int16_t)ns;
            a.cap_r[cid] = r;
        }
    for (int i = F * J; i < kMaxCapsules; ++i) a.cap_of[i] = -1;
    CF_TRY(launch_realize(a, (cudaStream_t)stream), "launch k_realize");
    return CF_OK;
}

// ---------------------------------------------------------------------------
// diagnostics
// ---------------------------------------------------------------------------
extern "C" const char *cf_last_error(void) { return t_err.c_str(); }

extern "C" int cf_device_status(uint32_t *status) {
    if (!status) return fail(CF_EINVAL, "NULL argument");
    DevState ds;
    int rc = device_state(&ds);
    if (rc) return rc;
    unsigned int v = 0;
    CF_TRY(cudaMemcpy(&v, ds.status, sizeof v, cudaMemcpyDeviceToHost), "read status");
    const unsigned int zero = 0;
    CF_TRY(cudaMemcpy(ds.status, &zero, sizeof zero, cudaMemcpyHostToDevice), "clear status");
    *status = v;
    return CF_OK;
}

extern "C" int cf_device_counters(uint64_t counters[4], int reset) {
    if (!counters) return fail(CF_EINVAL, "NULL argument");
    DevState ds;
    int rc = device_state(&ds);
    if (rc) return rc;
    unsigned long long v[4];
    CF_TRY(cudaMemcpy(v, ds.counters, sizeof v, cudaMemcpyDeviceToHost), "read counters");
    for (int i = 0; i < 4; ++i) counters[i] = v[i];
    if (reset) {
        const unsigned long long z[4] = {0, 0, 0, 0};
        CF_TRY(cudaMemcpy(ds.counters, z, sizeof z, cudaMemcpyHostToDevice), "reset counters");
    }
    return CF_OK;
}

extern "C" int cf_pool_usage(uint64_t usage[3], int reset_high) {
    if (!usage) return fail(CF_EINVAL, "NULL argument");
    cudaMemPool_t pool;
    int rc = device_pool(&pool);
    if (rc) return rc;
    unsigned long long used = 0, reserved = 0, high = 0;  // the attributes are 64-bit
    CF_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used), "pool used");
    CF_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved), "pool reserved");
    CF_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high), "pool high-water");
    usage[0] = used;
    usage[1] = reserved;
    usage[2] = high;
    if (reset_high) {
        unsigned long long zero = 0;  // the high-water mark restarts at the current use
        CF_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero), "reset pool high-water");
    }
    return CF_OK;
}

extern "C" int cf_place_static(const cf_palm_desc *palm, const cf_points *obj, int32_t n_poses, uint64_t seed,
                               uint32_t pose_base, float pen_margin, float *d_poses, int32_t *d_static_pt,
                               uint8_t *d_valid, cf_stream stream) {
    if (!palm) return fail(CF_EINVAL, "palm is NULL");
    int rc = check_points(obj);
    if (rc) return rc;
    if (n_poses < 0) return fail(CF_EINVAL, "n_poses < 0");
    if (n_poses > 0 && obj->n < 1) return fail(CF_EINVAL, "the object has no points");
    for (int c = 0; c < 3; ++c)
        if (!(palm->lo[c] < palm->hi[c]) || !isfinite(palm->lo[c]) || !isfinite(palm->hi[c]))
            return fail(CF_EINVAL, "palm box axis %d: [%g, %g] is not a finite interval", c, palm->lo[c], palm->hi[c]);
    if (!(pen_margin >= 0.f) || !isfinite(pen_margin)) return fail(CF_EINVAL, "pen_margin must be finite and >= 0");
    if (n_poses == 0) return CF_OK;
    if (!d_poses || !d_static_pt || !d_valid) return fail(CF_EINVAL, "output pointer is NULL");
    CF_TRY(launch_place_static(palm->lo, palm->hi, *obj, n_poses, (uint32_t)seed, (uint32_t)(seed >> 32), pose_base,
                               pen_margin, d_poses, d_static_pt, d_valid, (cudaStream_t)stream),
           "launch k_place_static");
    return CF_OK;
}

extern "C" int cf_append_contact(const int32_t *d_tuples, int32_t n_poses, int32_t n_tuples, int32_t k,
                                 const int32_t *d_first, const uint8_t *d_valid, int32_t *d_out, cf_stream stream) {
    if (n_poses < 0 || n_tuples < 1 || k < 1 || k + 1 > CF_MAX_K)
        return fail(CF_EINVAL, "n_poses >= 0, n_tuples >= 1 and 1 <= k < %d needed", CF_MAX_K);
    if (n_poses == 0) return CF_OK;
    if (!d_tuples || !d_first || !d_out) return fail(CF_EINVAL, "array pointer is NULL");
    CF_TRY(launch_append_contact(d_tuples, n_poses, n_tuples, k, d_first, d_valid, d_out, (cudaStream_t)stream),
           "launch k_append_contact");
    return CF_OK;
}

extern "C" int cf_sdf_box(const float *h_soa, int32_t n, float h, float margin, float lo[3], int32_t dims[3]) {
    if (!h_soa || !lo || !dims) return fail(CF_EINVAL, "NULL argument");
    if (n < 1) return fail(CF_EINVAL, "n < 1");
    if (!(h > 0.f) || !isfinite(h)) return fail(CF_EINVAL, "h must be finite and > 0");
    if (!(margin >= 0.f) || !isfinite(margin)) return fail(CF_EINVAL, "margin must be finite and >= 0");
    for (int c = 0; c < 3; ++c) {
        double mn = INFINITY, mx = -INFINITY;
        for (int i = 0; i < n; ++i) {
            const double v = h_soa[(size_t)c * n + i];
            if (!isfinite(v)) return fail(CF_EINVAL, "point %d is not finite", i);
            mn = v < mn ? v : mn;
            mx = v > mx ? v : mx;
        }
        const float l = (float)(mn - (double)margin);
        const double cells = ceil((mx + (double)margin - (double)l) / (double)h) + 1.0;
        if (cells > (double)(1 << 20)) return fail(CF_EINVAL, "axis %d needs %.0f nodes (> 2^20)", c, cells);
        lo[c] = l;
        dims[c] = (int32_t)cells;
    }
    return CF_OK;
}

