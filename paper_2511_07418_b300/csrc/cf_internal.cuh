// Internal declarations shared by the libcf translation units (device helpers,
// device-side views of the field, kernel launchers).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "cf.h"

namespace cf {

// ---------------------------------------------------------------------------
// device views
// ---------------------------------------------------------------------------

// Hand data copied to the device by cf_build.  Surface points are stored per
// finger sorted by link: surf[f][m] = (px, py, pz, nx, ny, nz, link, -), and
// link_begin[f][l] .. link_begin[f][l + 1] is link l's range.
struct HandDev {
    int F, J, M;
    const float *base;     // [F][12]
    const float *axis;     // [F][J][3]
    const float *offset;   // [F][J][3]
    const float *surf;     // [F][M][8]: p, n, link, original index (sorted by link)
    const int *link_begin; // [F][J + 1]
    const float *lo, *hi;  // [F][J] joint limits (NULL when not given)
    const float *radius;   // [F][J]
    const int *sorted_of;  // [F][M]: sorted position of original surface point m
};

// Representative hash: key = record word index * 32 + bit, value = min s*M + m.
constexpr unsigned long long kRepEmpty = ~0ull;
struct RepTable {
    unsigned long long *keys;
    uint32_t *vals;
    int log2_slots;
};

__device__ __forceinline__ unsigned rep_hash(unsigned long long key, int log2_slots) {
    return (unsigned)((key * 0x9E3779B97F4A7C15ull) >> (64 - log2_slots));
}

// value for key, or 0xffffffff when absent
__device__ __forceinline__ uint32_t rep_lookup(const RepTable &t, unsigned long long key) {
    const unsigned mask = (1u << t.log2_slots) - 1u;
    unsigned h = rep_hash(key, t.log2_slots);
    for (int probe = 0; probe <= (int)mask; ++probe, h = (h + 1) & mask) {
        const unsigned long long k = __ldg(t.keys + h);
        if (k == key) return __ldg(t.vals + h);
        if (k == kRepEmpty) return 0xffffffffu;
    }
    return 0xffffffffu;
}

// Normal-bin candidate table: a cube map of 6 faces x kCandG x kCandG cells
// over the unit sphere.  Each cell lists, ascending, every bin that can be the
// argmax for some direction in the cell (up to 4, 6 bits each, in bits 0..23;
// the count in bits 24..26), so evaluating only the listed bins gives exactly
// the full-scan result; a single listed bin needs no evaluation at all.
constexpr int kCandG = 32;
constexpr int kCandCells = 6 * kCandG * kCandG;

// Field geometry as the kernels need it (passed by value).  The table is one
// box of cells over all fingers; each cell owns a record of `rw` words and
// finger f's bin set sits at bit (f % fpw) * bits of word f / fpw.
struct FieldGeom {
    int F;                   // table slots (record rows of a query): the fingers, or the patches of a patch field
    int B;
    float inv_h;
    float clamp;             // |x| is clamped to this before the cell floor
    int lo[3];               // box: first cell
    int dims[3];             // box: cells per axis
    int bits, fpw, rw;       // bits per finger slot, slots per word, words per record
    int flo[CF_MAX_FINGERS][3], fdims[CF_MAX_FINGERS][3];  // tight per-finger bounds (reported only)
    float dirs[CF_MAX_BINS][3];
    uint32_t dil[CF_MAX_BINS];  // bins a query of bin b accepts: d_b . d_b' >= cos(dilate_deg) (bit b always)
    float dilate_deg;           // 0: no dilation
    int use_cand;            // 1: candidate table valid (every cell has <= 4 candidates)
    const uint32_t *cand;    // device [kCandCells]
    int patches;             // 1: one slot per (finger, link) patch (Sec. 4.4 fine-grained field)
    int8_t slot_of[CF_MAX_FINGERS][CF_MAX_JOINTS];  // slot of (finger, link); -1: a link without surface points
    int8_t slot_finger[CF_MAX_SLOTS], slot_link[CF_MAX_SLOTS];  // owner of each slot (link -1: every link)
};

inline int slot_bits_for(int B) { return B <= 8 ? 8 : (B <= 16 ? 16 : 32); }
// Words per cell record in the table: the words the slots need, ceil(slots / slots per word),
// rounded up to 1, 2, 4, 8 or 16 so a record is one or more aligned 16-byte loads (the extra
// words stay zero).
__host__ __device__ constexpr int record_stride(int words) {
    return words <= 2 ? words : (words <= 4 ? 4 : (words <= 8 ? 8 : 16));
}

// Host: fill the candidate table for the given directions; returns the largest
// per-cell candidate count.
int build_bin_candidates(const float *dirs, int B, uint32_t *table);

// In place, by one block of 1024 threads: v[b] <- v[0] + ... + v[b - 1] for b < nb (tiles of
// 1024 entries in turn, the running sum carried across them); *total (when given) <- the sum of
// all nb entries.  Every thread of the block must call it.
__device__ __forceinline__ void block_exclusive_scan_1024(unsigned *v, int nb, unsigned *total) {
    __shared__ unsigned s_w[32];
    __shared__ unsigned s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const unsigned x = b < nb ? v[b] : 0u;
        unsigned incl = x;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        unsigned before = s_carry;
        for (int w = 0; w < warp; ++w) before += s_w[w];
        if (b < nb) v[b] = before + incl - x;
        __syncthreads();  // every thread has read s_carry and s_w
        if (threadIdx.x == 1023) s_carry = before + incl;
        __syncthreads();
    }
    if (total && threadIdx.x == 0) *total = s_carry;
}

// bin of m from the cube-map candidate list (exactly the full-scan argmax)
__device__ __forceinline__ int bin_by_candidates(float mx, float my, float mz, const uint32_t *s_cand,
                                                 const float4 *s_dir) {
    const float ax = fabsf(mx), ay = fabsf(my), az = fabsf(mz);
    const bool xmaj = ax >= ay && ax >= az;
    const bool ymaj = !xmaj && ay >= az;
    const int face = xmaj ? (mx < 0.f ? 1 : 0) : (ymaj ? (my < 0.f ? 3 : 2) : (mz < 0.f ? 5 : 4));
    const float ma = xmaj ? my : mx;
    const float mb = (xmaj || ymaj) ? mz : my;
    // approximate reciprocal (relative error ~1e-7): the table's cells are enlarged by 1e-4 in u, v, so a
    // cell chosen from a slightly perturbed coordinate still lists the true bin
    const float inv = __fdividef(1.f, fmaxf(ax, fmaxf(ay, az)));
    // the cell of c = ma / major in [-1, 1] (up to the reciprocal's error): c * G/2 + G/2 + 1.5 * 2^23,
    // rounded toward zero, keeps the integer part in its low mantissa bits (an FMA, no conversion
    // instruction); the clamp keeps c = +-1 (and a non-finite normal) inside the table.  Near a cell
    // edge this may name the neighbouring cell, which lists the bin all the same (cells are enlarged by
    // 1e-4)
    const float sc = inv * (0.5f * kCandG);
    const int iu =
        min(max(__float_as_int(__fmaf_rz(ma, sc, 0.5f * kCandG + 12582912.0f)) - 0x4B400000, 0), kCandG - 1);
    const int iv =
        min(max(__float_as_int(__fmaf_rz(mb, sc, 0.5f * kCandG + 12582912.0f)) - 0x4B400000, 0), kCandG - 1);
    const uint32_t word = s_cand[(face * kCandG + iu) * kCandG + iv];
    const int cnt = (int)(word >> 24);
    // the first two candidates (ascending) without a branch: a one-candidate cell
    // compares its bin with itself; most cells have one or two
    const int b0 = (int)(word & 63u);
    const int b1 = cnt > 1 ? (int)((word >> 6) & 63u) : b0;
    const float4 d0 = s_dir[b0], d1 = s_dir[b1];
    float best = __fmaf_rn(d0.z, mz, __fmaf_rn(d0.y, my, __fmul_rn(d0.x, mx)));
    const float s1 = __fmaf_rn(d1.z, mz, __fmaf_rn(d1.y, my, __fmul_rn(d1.x, mx)));
    int bin = b0;
    if (s1 > best) { best = s1; bin = b1; }
    for (int c = 2; c < cnt; ++c) {  // rare
        const int b = (int)((word >> (6 * c)) & 63u);
        const float4 d = s_dir[b];
        const float sc = __fmaf_rn(d.z, mz, __fmaf_rn(d.y, my, __fmul_rn(d.x, mx)));
        if (sc > best) { best = sc; bin = b; }
    }
    return bin;
}

// ---------------------------------------------------------------------------
// decision arithmetic (single-rounding FMAs, component order x, y, z)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float xf_row(float r0, float r1, float r2, float t, float x, float y, float z) {
    return __fmaf_rn(r2, z, __fmaf_rn(r1, y, __fmaf_rn(r0, x, t)));
}

__device__ __forceinline__ float rot_row(float r0, float r1, float r2, float x, float y, float z) {
    return __fmaf_rn(r2, z, __fmaf_rn(r1, y, __fmul_rn(r0, x)));
}

// floor of the exact product x * inv_h for |x * inv_h| < 2^22: the product is
// added to 1.5 * 2^23 with one rounding toward -inf, which lands on the integer
// grid of the [2^23, 2^24) binade; the low mantissa bits are the floor.
__device__ __forceinline__ int cell_floor(float x, float inv_h, float clamp) {
    x = fminf(fmaxf(x, -clamp), clamp);
    float y = __fmaf_rd(x, inv_h, 12582912.0f);
    return __float_as_int(y) - 0x4B400000;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// ---------------------------------------------------------------------------
// launchers (return cudaError_t of the launch)
// ---------------------------------------------------------------------------
cudaError_t launch_fk_cell_bounds(const HandDev &h, const float *q, int S, float inv_h, float clamp,
                                  int *bounds, float *links, cudaStream_t st);
cudaError_t launch_fk_bin(const HandDev &h, const int *h_link_begin, const float *links, int S, const FieldGeom &g,
                          uint32_t *table, unsigned int *status, cudaStream_t st);
// ---- reverse lookup + DLS IK (Sec. 5.5), object SDF grid, realization (Sec. 5.6) ----
struct IkArgs {
    HandDev h;
    FieldGeom g;
    RepTable rep;
    const float *qs;  // field joint samples [F][J][S]
    int S;
    cf_points obj;
    const float *poses;
    int n, T, k;
    const int32_t *tuples;
    const uint8_t *fingers;
    const uint8_t *accept;
    float beta, lambda, tol_pos, tol_cos;
    int n1, nr, n2;
    float *q;
    uint8_t *used;
    float *cp[6];     // realised contacts, object frame: px py pz nx ny nz [n * k]
    int32_t *rtuples;
    float *resid;     // [n][k][2]: distance, cosine
    uint8_t *ok;
    unsigned int *status;
};

struct SdfGrid {
    const float *v;
    float lo[3];
    float h, inv_h;
    int dims[3];
};

// Trilinear object SDF at (x, y, z) (object frame); +inf outside the grid.
__device__ __forceinline__ float sdf_at(const SdfGrid &g, float x, float y, float z) {
    const float u = (x - g.lo[0]) * g.inv_h, v = (y - g.lo[1]) * g.inv_h, w = (z - g.lo[2]) * g.inv_h;
    const float fu = floorf(u), fv = floorf(v), fw = floorf(w);
    const int i = (int)fu, j = (int)fv, kk = (int)fw;
    if (!(fu >= 0.f && fv >= 0.f && fw >= 0.f) || i + 1 >= g.dims[0] || j + 1 >= g.dims[1] || kk + 1 >= g.dims[2])
        return INFINITY;  // outside the grid: farther from the object than its margin
    const float a = u - fu, b = v - fv, c = w - fw;
    const size_t sx = 1, sy = (size_t)g.dims[0], sz = (size_t)g.dims[0] * g.dims[1];
    const float *p = g.v + (size_t)kk * sz + (size_t)j * sy + i;
    const float v000 = __ldg(p), v100 = __ldg(p + sx), v010 = __ldg(p + sy), v110 = __ldg(p + sy + sx);
    const float v001 = __ldg(p + sz), v101 = __ldg(p + sz + sx), v011 = __ldg(p + sz + sy),
                v111 = __ldg(p + sz + sy + sx);
    const float x00 = fmaf(a, v100 - v000, v000), x10 = fmaf(a, v110 - v010, v010);
    const float x01 = fmaf(a, v101 - v001, v001), x11 = fmaf(a, v111 - v011, v011);
    const float y0 = fmaf(b, x10 - x00, x00), y1 = fmaf(b, x11 - x01, x01);
    return fmaf(c, y1 - y0, y0);
}

constexpr int kMaxCapsules = CF_MAX_FINGERS * CF_MAX_JOINTS;
struct RealizeArgs {
    HandDev h;
    SdfGrid sdf;
    const float *poses;
    int n, T;
    const uint8_t *gate_a, *gate_b;
    float *q;
    const uint8_t *used;
    uint8_t *flags;
    float pen_margin;
    uint32_t seed_lo, seed_hi;
    int n_caps;
    int8_t cap_of[kMaxCapsules];   // capsule id of (f, j), -1 when link j of finger f has none
    uint8_t cap_f[kMaxCapsules];
    int16_t cap_ns[kMaxCapsules];  // axis intervals: samples at s / ns, s = 0..ns
    float cap_r[kMaxCapsules];
};

cudaError_t launch_ik(const IkArgs &a, int *list, unsigned int *count, cudaStream_t st);
cudaError_t launch_sdf(const cf_points &obj, const SdfGrid &g, float *grid, cudaStream_t st);
cudaError_t launch_realize(const RealizeArgs &a, cudaStream_t st);

// ---- placement (Sec. 5.2) and object preprocessing (Sec. 5.1) ----
struct PlaceArgs {
    int P;
    uint32_t seed_lo, seed_hi, pose_base;
    float centroid[3];
    float g[3], up[3];  // canonical: anchor point and palm normal
    float d_lo, d_hi;   // canonical: offset range along up
    // exhaustive: the field's table, its chunk prefix counts and the object's points
    const uint32_t *table;
    const unsigned long long *prefix;  // [n_chunks + 1] exclusive prefix of set bits per chunk
    int n_chunks;
    unsigned long long n_codes;
    long long table_words;
    FieldGeom g_field;
    cf_points obj;
    float *poses;
};
constexpr int kChunkWords = 256;
cudaError_t launch_chunk_counts(const uint32_t *table, long long words, unsigned long long *counts, cudaStream_t st);
cudaError_t launch_place(const PlaceArgs &a, bool exhaustive, cudaStream_t st);
cudaError_t launch_place_static(const float lo[3], const float hi[3], const cf_points &obj, int P, uint32_t seed_lo,
                                uint32_t seed_hi, uint32_t pose_base, float pen_margin, float *poses, int32_t *static_pt,
                                uint8_t *valid, cudaStream_t st);
cudaError_t launch_append_contact(const int32_t *tuples, int P, int T, int k, const int32_t *first, const uint8_t *valid,
                                  int32_t *out, cudaStream_t st);
cudaError_t launch_concave(const cf_points &obj, const SdfGrid &sdf, float side, float tau, uint8_t *keep,
                           unsigned int *block_counts, float *out, int *n_out, cudaStream_t st);

cudaError_t launch_gswo(const float *const pts[6], int N, long long n, int k, float mu, const float c[3], float rho,
                        float eps, int n_iter, const float *beta, const int32_t *tuples, float *value, uint8_t *accept,
                        cudaStream_t st);
cudaError_t launch_popcount(const uint32_t *table, long long words, unsigned long long *count, cudaStream_t st);
cudaError_t launch_fk_rep(const HandDev &h, const float *links, int S, const FieldGeom &g, RepTable t,
                          unsigned int *status, cudaStream_t st);
cudaError_t launch_query(const FieldGeom &g, const uint32_t *table, const cf_points &obj, const float *poses,
                         int P, uint32_t *masks, uint32_t *counts, int ppb, cudaStream_t st);

// One object's domain query (the plain call uses one by value; a batch keeps an
// array of them in device memory, block0 = first grid block of the object).
struct QueryDesc {
    cf_points obj;
    const float *poses;
    int P, W;
    uint32_t *masks, *counts;
    const uint32_t *table;
    int geom;     // index into the batch's FieldGeom array
    int block0;   // first block of this object in the batch grid
};

// Every object of a batch in one persistent launch (any hand): items are
// (object, block of ppb poses), object d's first item is descs[d].block0
// (ascending).  d_work: 2 device words, zero before the first launch; each
// launch leaves them zero again.
cudaError_t launch_query_batch(const QueryDesc *d_descs, const FieldGeom *d_geoms, int n_desc, int total_items,
                               int ppb, unsigned int *d_work, cudaStream_t st);
int query_blocks(int P, int ppb);  // grid blocks one object of P poses needs at ppb poses per block
// Sec. 5.3 dependency-group merge: group_masks[i][f] = OR of slot_masks[i][s] over g.slot_finger[s] == f
// (n_fingers groups), group_counts its popcount.
cudaError_t launch_merge_domains(const FieldGeom &g, int n_fingers, const uint32_t *slot_masks, int P, int W,
                                 uint32_t *group_masks, uint32_t *group_counts, cudaStream_t st);
// The current device's SM count and the resident blocks per SM of kernel `func` at `threads` threads
// and `smem` dynamic shared bytes, queried once per (device, kernel, shape) and then served from a cache.
cudaError_t launch_shape(const void *func, int threads, size_t smem, int *per_sm, int *sms);
constexpr int kMaxPosesPerBlock = 16;

// Launch shapes picked by the autotuner (per device); results do not depend on them.
struct Tuning {
    int query_ppb;    // poses per query block: 4, 8 or 16
    int score_refill; // idle lanes of a scoring warp before they take new tuples together: 4, 8 or 16
    int score_bpsm;   // scoring blocks per SM (0: as many as fit)
};
Tuning current_tuning();

struct ScoreArgs {
    const float *px, *py, *pz, *nx, *ny, *nz;
    int N, W, F, P;
    const uint32_t *masks, *counts;
    int T, k, K;
    float mu, eps, cx, cy, cz, inv_rho;
    float cs[CF_MAX_EDGES], sn[CF_MAX_EDGES];
    uint32_t seed_lo, seed_hi;
    int tuples_given;
    uint32_t pose_base;  // added to the pose index in the tuple draws' counter
    int32_t *tuples;
    uint8_t *fingers;
    float *margin;
    uint8_t *accept;
    unsigned int *work;  // scratch: tuple work counter, zero at launch
    float *word_box;     // Alg. 2 scratch: per mask word, the bounding box of its 32 points [W][6] (lo xyz, hi xyz)
    unsigned int *status;          // device status word (CF_DEV_* bits)
    unsigned long long *counters;  // [0] pivots, [1] LPs, [2] tuples, [3] warm-started Alg. 2 candidates
    int refill;                    // idle lanes of a scoring warp before a group refill (launch-level)
    int bpsm;                      // scoring blocks per SM, 0 = as many as fit (launch-level)
    unsigned long long *n_accept;  // optional: accepted tuples of the launch are added here
};
// k_sample_tuples (unless tuples_given) then k_score_tuples
cudaError_t launch_score(const ScoreArgs &a, cudaStream_t st);
// k_sample_tuples only
cudaError_t launch_sample(const ScoreArgs &a, cudaStream_t st);
// batches: pose0 / tuple0 = [n_desc + 1] prefix sums (device); the score launch's
// work counter, status and counters come from `launch`, which also fixes k and K
cudaError_t launch_sample_batch(const ScoreArgs *d_descs, const long long *d_pose0, int n_desc, long long total_poses,
                                size_t smem, cudaStream_t st);
cudaError_t launch_score_batch(const ScoreArgs &launch, const ScoreArgs *d_descs, const long long *d_tuple0, int n_desc,
                               long long total_tuples, cudaStream_t st);
size_t score_smem_bytes(int F, int W, int T, int k, bool sampling);
// Alg. 2 contact optimisation of the tuples in place (a.tuples / a.fingers given; a.masks;
// margin / accept out; a.word_box: scratch for (W + ceil(W / 32)) point boxes); n_inner in
// {4, 8, 16}.  state: device scratch of optimize_state_bytes(P * T, n_inner, k, warm_start)
// bytes for the per-tuple state between the phases (k_opt_* kernels).
size_t optimize_state_bytes(long long n, int n_inner, int k, int warm);
cudaError_t launch_optimize(const ScoreArgs &a, int n_outer, int n_inner, float sigma, float zero_tol,
                            float min_gain, int warm_start, void *state, cudaStream_t st);

// ---------------------------------------------------------------------------
// host helpers shared by the ABI translation units
// ---------------------------------------------------------------------------
extern thread_local std::string t_err;
int fail(int code, const char *fmt, ...);                // sets the thread's error message, returns code
int cuda_fail(cudaError_t e, const char *what);
int pool_alloc(void **p, size_t bytes, cudaStream_t st, const char *what);  // library stream-ordered pool
int check_points(const cf_points *obj);
int fill_score_args(const cf_points *obj, int32_t F, const uint32_t *d_masks, const uint32_t *d_counts, int32_t P,
                    const cf_score_params *prm, int32_t *d_tuples, uint8_t *d_fingers, float *d_margin,
                    uint8_t *d_accept, ScoreArgs *a);

#define CF_TRY(call, what)                                     \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return ::cf::cuda_fail(e_, what); \
    } while (0)

}  // namespace cf

// the field handle of the ABI (opaque to callers)
struct cf_field {
    int dev = 0;
    cudaStream_t st = nullptr;  // device memory is freed on this stream
    int F = 0, J = 0, M = 0, S = 0, B = 0;
    cf::FieldGeom geom{};
    cf::HandDev hand{};
    void *d_block = nullptr;     // hand arrays + bounds scratch
    uint32_t *d_table = nullptr;
    uint32_t *d_cand = nullptr;  // normal-bin candidate table
    int64_t table_words = 0;
    int64_t device_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    float build_ms = -1.f;
    cf::RepTable rep{nullptr, nullptr, 0};  // reverse-lookup table (want_rep)
    void *d_rep = nullptr;
    float *d_qs = nullptr;                  // joint samples [F][J][S] (kept with the representative table)
    bool has_limits = false;
    std::vector<float> h_lo, h_hi, h_radius, h_offset;  // host copies for realization planning
    unsigned long long *d_prefix = nullptr;  // exclusive set-bit prefix per table chunk (exhaustive placement)
    int n_chunks = 0;
    unsigned long long n_codes = 0;
};

struct cf_sdf {
    int dev = 0;
    cudaStream_t st = nullptr;
    cf::SdfGrid g{};
    float *d_grid = nullptr;
    int64_t nodes = 0;
};
