// Tuple sampling + closure margin kernels (rows a4 + a5 of the hot path).
//
// Sec. 5.3: a k-contact grasp takes k contact domains of different fingers
// (independent dependency groups) chosen at random; Alg. 2 starts from
// (p_i, n_i) <- Random(D_i).  Eq. GSWO (Sec. 3.2) scores the contacts: with
// alpha_j = 1 for some j and friction forces inside the cones, minimise the
// resultant force and (weighted) torque; the problem splits into one convex
// subproblem per j.  Linearised here: each cone becomes its inscribed K-edge
// pyramid and the squared norm becomes the max-norm of [force ; torque / rho],
// so every subproblem is the LP
//     LP_j = min t  s.t.  -t <= (sum_im c_im w_im)_r <= t,  sum_m c_jm = 1,  c >= 0
// and the margin is min_j LP_j.
//
// k_sample_tuples: one block per pose stages the F mask rows in shared memory
// with per-32-word popcount prefixes; one thread per tuple draws its fingers
// and points (Philox4x32-10) and writes them out.
//
// k_score_tuples: persistent warps pull batches of tuples from a work counter;
// each warp solves its tuple's k LPs in the scaled bounded-variable form below
// (6 rows, kK + 6 columns, one column per lane), LP_{j+1} warm-started from
// LP_j's basis.  Pricing and the ratio test are single warp reductions
// (redux.sync) on order-preserving integer keys of the floats; the entering
// column reaches every lane through a per-warp shared buffer.  FP32 throughout.
#include <limits.h>

#include <string.h>

#include <algorithm>

#include "cf_internal.cuh"

namespace cf {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// sampling
// ---------------------------------------------------------------------------
constexpr int kSampleThreads = 128;

__device__ __forceinline__ int select_in_word(uint32_t v, uint32_t r) {
    int pos = 0;
    uint32_t c = __popc(v & 0xFFFFu);
    if (r >= c) { r -= c; v >>= 16; pos += 16; }
    c = __popc(v & 0xFFu);
    if (r >= c) { r -= c; v >>= 8; pos += 8; }
    c = __popc(v & 0xFu);
    if (r >= c) { r -= c; v >>= 4; pos += 4; }
    c = __popc(v & 0x3u);
    if (r >= c) { r -= c; v >>= 2; pos += 2; }
    c = v & 1u;
    if (r >= c) pos += 1;
    return pos;
}

// r-th set bit (ascending) of a staged mask row, -1 if the row has <= r bits.
__device__ __forceinline__ int select_in_row(const uint32_t *row, const uint32_t *gp, int W, int G, uint32_t r) {
    if (r >= gp[G]) return -1;
    int lo = 0, hi = G - 1;  // largest g with gp[g] <= r
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gp[mid] <= r) lo = mid; else hi = mid - 1;
    }
    uint32_t rr = r - gp[lo];
    const int wend = min(32 * lo + 32, W);
    for (int w = 32 * lo; w < wend; ++w) {
        const uint32_t v = row[w];
        const uint32_t c = __popc(v);
        if (rr < c) return 32 * w + select_in_word(v, rr);
        rr -= c;
    }
    return -1;
}

__device__ __forceinline__ uint32_t draw_word(const uint4 &a, const uint4 &b, int d) {
    switch (d) {
        case 0: return a.x;
        case 1: return a.y;
        case 2: return a.z;
        case 3: return a.w;
        case 4: return b.x;
        case 5: return b.y;
        case 6: return b.z;
        default: return b.w;
    }
}

// MULTI: block b samples pose b - pose0[d] of object d, pose0 = first block of
// each object (ascending); the object's arguments are copied to shared memory.
template <bool MULTI>
__global__ void __launch_bounds__(kSampleThreads) k_sample_tuples(const ScoreArgs a1, const ScoreArgs *descs,
                                                                  const long long *pose0, int n_desc) {
    extern __shared__ uint32_t s_dyn[];
    __shared__ uint32_t s_cnt[CF_MAX_FINGERS];
    __shared__ ScoreArgs s_args;
    __shared__ int s_i;
    if (MULTI) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = n_desc - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (pose0[mid] <= (long long)blockIdx.x) lo = mid; else hi = mid - 1;
            }
            s_args = descs[lo];
            s_i = (int)((long long)blockIdx.x - pose0[lo]);
        }
        __syncthreads();
    }
    const ScoreArgs &a = MULTI ? s_args : a1;
    const int F = a.F, W = a.W, T = a.T, k = a.k;
    const int G = (W + 31) / 32;
    uint32_t *s_mask = s_dyn;           // [F][W]
    uint32_t *s_gpre = s_mask + F * W;  // [F][G + 1]
    const int i = MULTI ? s_i : (int)blockIdx.x;
    if (threadIdx.x < F) s_cnt[threadIdx.x] = a.counts[(size_t)i * F + threadIdx.x];
    const uint32_t *src = a.masks + (size_t)i * F * W;
    for (int e = threadIdx.x; e < F * W; e += blockDim.x) s_mask[e] = src[e];
    __syncthreads();
    for (int e = threadIdx.x; e < F * G; e += blockDim.x) {
        const int f = e / G, g = e % G;
        const uint32_t *row = s_mask + f * W;
        uint32_t c = 0;
        const int wend = min(32 * g + 32, W);
        for (int w = 32 * g; w < wend; ++w) c += __popc(row[w]);
        s_gpre[f * (G + 1) + g + 1] = c;
    }
    __syncthreads();
    if (threadIdx.x < F) {
        uint32_t *gp = s_gpre + threadIdx.x * (G + 1);
        gp[0] = 0;
        for (int g = 1; g <= G; ++g) gp[g] += gp[g - 1];
    }
    __syncthreads();
    uint32_t pk0 = 0;  // non-empty fingers, 4 bits each, ascending
    int m = 0;
    for (int f = 0; f < F; ++f)
        if (s_cnt[f] > 0) pk0 |= (uint32_t)f << (4 * m++);
    const uint2 key = make_uint2(a.seed_lo, a.seed_hi);
    for (int tau = threadIdx.x; tau < T; tau += blockDim.x) {
        int32_t *gt = a.tuples + ((size_t)i * T + tau) * k;
        uint8_t *gf = a.fingers ? a.fingers + ((size_t)i * T + tau) * k : nullptr;
        if (m < k) {
            for (int d = 0; d < k; ++d) {
                gt[d] = -1;
                if (gf) gf[d] = 255;
            }
            continue;
        }
        const uint32_t pid = (uint32_t)i + a.pose_base;
        const uint4 u0 = philox4x32_10(make_uint4(pid, (uint32_t)tau, 0u, 0u), key);
        const uint4 u1 = philox4x32_10(make_uint4(pid, (uint32_t)tau, 1u, 0u), key);
        uint32_t pk = pk0;
        for (int d = 0; d < k; ++d) {  // partial Fisher-Yates over the non-empty fingers
            const int jj = d + (int)__umulhi(draw_word(u0, u1, d), (uint32_t)(m - d));
            const uint32_t fd = (pk >> (4 * d)) & 15u, fj = (pk >> (4 * jj)) & 15u;
            pk &= ~((15u << (4 * d)) | (15u << (4 * jj)));
            pk |= (fj << (4 * d)) | (fd << (4 * jj));
        }
        for (int d = 0; d < k; ++d) {
            const int f = (pk >> (4 * d)) & 15u;
            const uint32_t r = __umulhi(draw_word(u0, u1, k + d), s_cnt[f]);
            gt[d] = select_in_row(s_mask + f * W, s_gpre + f * (G + 1), W, G, r);
            if (gf) gf[d] = (uint8_t)f;
        }
    }
}

// ---------------------------------------------------------------------------
// scoring
// ---------------------------------------------------------------------------
constexpr int kScoreThreads = 256;
constexpr int kScoreWarps = kScoreThreads / 32;
constexpr int kMaxPivots = 64;        // per LP, after the two start pivots
constexpr int kDegenerateToBland = 16;
constexpr float kDTol = 1e-6f;        // reduced-cost tolerance
constexpr float kPTol = 1e-6f;        // smallest admissible pivot entry
constexpr float kZeroExit = 1e-7f;    // an LP this close to 0 ends the tuple (min over j)

// order-preserving map float -> unsigned (NaN above +inf)
__device__ __forceinline__ unsigned fkey(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Scaled LP.  For t > 0 put c = t c'; then LP_j = 1 / s_j with
//     s_j = max sum_m c'_jm  s.t.  -1 <= (sum_im c'_im w_im)_r <= 1 (r = 1..6),  c' >= 0,
// and LP_j = 0 exactly when s_j is unbounded.  With y = W c' kept as six
// variables boxed in [-1, 1], the LP has 6 equality rows W c' - y = 0 and
// kK + 6 columns, and c' = 0, y = 0 is a feasible start (no phase 1).  The j
// subproblems differ only in the objective, so LP_{j+1} starts from LP_j's
// optimal basis.  Bounded-variable primal simplex: Dantzig pricing, ratio test
// over the basic variables' bounds and the entering variable's own box (a bound
// flip), the largest pivot entry among degenerate rows (ratio 0) and the lowest
// row among other exact ties, Bland's rule after a run of degenerate pivots.
//
// Warp layout (NS slots per lane): the column with id c' = 0..kK-1 (contact
// c / K, edge c % K) is slot 0 of lane c; the y_r columns are slot 0 of lane
// kK + r when kK + 6 <= 32 (NS = 1), else slot 1 of lane r (id 32 + r).  Each
// slot holds the column's 6 tableau entries and its reduced cost.  Lane r < 6
// also holds row r's basic variable (id) and its value.
constexpr int kRows = 6;
constexpr unsigned kNoKey = 0xffffffffu;

template <int NS>
struct BoxLp {
    float T[NS][kRows + 1];  // rows 0..5 of the tableau, then the reduced cost
    int st[NS];              // 0 basic, 1 at lower bound, 2 at upper bound, 3 no column
    float v;                 // lane r < 6: value of row r's basic variable
    int beta;                // lane r < 6: id of row r's basic variable
};

template <int NS>
__device__ __forceinline__ int y_id(int r, int kK) { return NS == 1 ? kK + r : 32 + r; }

// Closure margin min_j LP_j of one tuple on the warp.  w = this lane's wrench
// column (lanes < kK).  Stops at the first unbounded s_j (margin 0).
template <int NS>
__device__ float closure_margin(const float (&w)[6], int k, int K, int lane, float *buf, unsigned long long &n_piv,
                                unsigned long long &n_lp, unsigned &flags) {
    const int kK = k * K;
    BoxLp<NS> s;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        const int id = 32 * q + lane;
        const bool isx = q == 0 && lane < kK;
        const int yr = NS == 1 ? lane - kK : (q == 1 ? lane : -1);
        const bool isy = yr >= 0 && yr < kRows;
#pragma unroll
        for (int r = 0; r < kRows; ++r) s.T[q][r] = isx ? -w[r] : (isy && r == yr ? 1.f : 0.f);
        s.T[q][kRows] = 0.f;
        s.st[q] = isx ? 1 : (isy ? 0 : 3);
        (void)id;
    }
    s.v = 0.f;
    s.beta = lane < kRows ? y_id<NS>(lane, kK) : -1;

    const unsigned kinf = fkey(INFINITY);
    const unsigned kzero = fkey(0.f);
    unsigned npv = 0;
    float best_s = 0.f;
    bool unbounded = false;
    for (int j = 0; j < k && !unbounded; ++j) {
        const int c0 = j * K, c1 = c0 + K;  // contact j's columns
        // reduced costs of the objective sum_m c'_jm at the current basis
        const unsigned inj =
            __ballot_sync(kFull, lane < kRows && s.beta >= c0 && s.beta < c1) & ((1u << kRows) - 1u);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int id = 32 * q + lane;
            float d = (id >= c0 && id < c1 && s.st[q] != 3) ? 1.f : 0.f;
#pragma unroll
            for (int r = 0; r < kRows; ++r)
                if (inj & (1u << r)) d -= s.T[q][r];
            s.T[q][kRows] = s.st[q] == 0 ? 0.f : d;
        }
        bool bland = false;
        int degenerate = 0, it = 0;
        for (; it < kMaxPivots; ++it) {
            // pricing: an at-lower column with d > 0 or an at-upper column with d < 0
            int e;
            float sc[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const float d = s.T[q][kRows];
                sc[q] = s.st[q] == 1 ? d : (s.st[q] == 2 ? -d : -INFINITY);
            }
            if (bland) {
                const unsigned b0 = __ballot_sync(kFull, sc[0] > kDTol);
                const unsigned b1 = NS > 1 ? __ballot_sync(kFull, sc[NS - 1] > kDTol) : 0u;
                e = b0 ? __ffs(b0) - 1 : (b1 ? 31 + __ffs(b1) : -1);
            } else {
                unsigned key = kNoKey;
#pragma unroll
                for (int q = 0; q < NS; ++q)
                    if (sc[q] > kDTol) key = min(key, (fkey(-sc[q]) & ~63u) | (unsigned)(32 * q + lane));
                const unsigned kmin = __reduce_min_sync(kFull, key);
                e = kmin == kNoKey ? -1 : (int)(kmin & 63u);
            }
            if (e < 0) break;
            // publish the entering column (and its direction: +1 up from lower, -1 down from upper)
            const int qe = e >> 5;
            if (lane == (e & 31)) {
                float c[kRows + 1];
                int ste = 0;
#pragma unroll
                for (int q = 0; q < NS; ++q)
                    if (q == qe) {
#pragma unroll
                        for (int r = 0; r <= kRows; ++r) c[r] = s.T[q][r];
                        ste = s.st[q];
                    }
                float4 *b4 = reinterpret_cast<float4 *>(buf);
                b4[0] = make_float4(c[0], c[1], c[2], c[3]);
                b4[1] = make_float4(c[4], c[5], c[6], ste == 1 ? 1.f : -1.f);
            }
            __syncwarp();
            const float4 c03 = reinterpret_cast<const float4 *>(buf)[0];
            const float4 c47 = reinterpret_cast<const float4 *>(buf)[1];
            const float col[kRows + 1] = {c03.x, c03.y, c03.z, c03.w, c47.x, c47.y, c47.z};
            const float dl = c47.w;
            const bool ey = e >= kK;  // entering a y (boxed, range 2)
            // ratio test: lane r < 6 -> row r; lane 6 -> the entering variable's own box
            const float mine = lane < kRows ? buf[lane] : 0.f;
            const float alpha = mine * dl;  // the basic variable of row lane moves by -alpha theta
            float theta = INFINITY;
            if (lane < kRows) {
                const bool bx = s.beta < kK;
                const float lo = bx ? 0.f : -1.f, hi = bx ? INFINITY : 1.f;
                if (alpha > kPTol) theta = __fdividef(fmaxf(s.v - lo, 0.f), alpha);
                else if (alpha < -kPTol) theta = __fdividef(fmaxf(hi - s.v, 0.f), -alpha);
            } else if (lane == kRows && ey) {
                theta = 2.f;
            }
            // degenerate rows (theta = 0) key below every positive ratio, by decreasing |pivot entry|
            const unsigned rk =
                (!bland && theta == 0.f) ? (~__float_as_uint(fabsf(alpha)) & 0x7fffffffu) : fkey(theta);
            const unsigned rmin = __reduce_min_sync(kFull, rk);
            if (rmin == kinf) {  // s_j unbounded: LP_j = 0
                unbounded = true;
                __syncwarp();
                break;
            }
            const bool tie = rk == rmin;
            unsigned cand;
            if (bland) {  // a bound flip first, then the lowest basic-variable id
                const unsigned bk = !tie ? kNoKey : (lane == kRows ? 0u : (unsigned)s.beta + 1u);
                const unsigned bmin = __reduce_min_sync(kFull, bk);
                cand = __ballot_sync(kFull, tie && bk == bmin);
            } else {
                cand = __ballot_sync(kFull, tie);
            }
            const int l = __ffs(cand) - 1;
            const float th = __shfl_sync(kFull, theta, l);
            degenerate = rmin <= kzero ? degenerate + 1 : 0;
            if (degenerate >= kDegenerateToBland) bland = true;
            ++npv;
            if (l == kRows) {  // bound flip: no basis change
                if (lane < kRows) s.v = __fmaf_rn(-alpha, th, s.v);
#pragma unroll
                for (int q = 0; q < NS; ++q)
                    if (q == qe && lane == (e & 31)) s.st[q] = 3 - s.st[q];
                __syncwarp();
                continue;
            }
            const int leave = __shfl_sync(kFull, s.beta, l);
            const float piv = __shfl_sync(kFull, mine, l);
            const bool to_lower = piv * dl > 0.f;  // the leaving variable stops at its lower bound
            const float xe0 = !ey ? 0.f : (dl > 0.f ? -1.f : 1.f);
            if (lane < kRows) {
                if (lane == l) {
                    s.v = xe0 + dl * th;
                    s.beta = e;
                } else {
                    s.v = __fmaf_rn(-alpha, th, s.v);
                }
            }
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const int id = 32 * q + lane;
                if (id == e) s.st[q] = 0;
                if (id == leave) s.st[q] = to_lower ? 1 : 2;
            }
            // tableau pivot on (row l, column e)
            const float inv = __fdividef(1.f, piv);  // fast reciprocal: |piv| > kPTol
            bool isl[kRows];
#pragma unroll
            for (int r = 0; r < kRows; ++r) isl[r] = r == l;
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                float tl = s.T[q][0];
#pragma unroll
                for (int r = 1; r < kRows; ++r) tl = isl[r] ? s.T[q][r] : tl;
                const float pa = __fmul_rn(tl, inv);
#pragma unroll
                for (int r = 0; r <= kRows; ++r) {
                    const float u = __fmaf_rn(-col[r], pa, s.T[q][r]);
                    s.T[q][r] = (r < kRows && isl[r]) ? pa : u;
                }
            }
            __syncwarp();  // every lane has read buf before it is written again
        }
        if (it == kMaxPivots) flags |= CF_DEV_LP_PIVOT_CAP;
        ++n_lp;
        if (!unbounded) {  // s_j = the sum of contact j's basic values (nonbasic c' sit at 0)
            float part = (lane < kRows && s.beta >= c0 && s.beta < c1) ? s.v : 0.f;
            part += __shfl_xor_sync(kFull, part, 4);
            part += __shfl_xor_sync(kFull, part, 2);
            part += __shfl_xor_sync(kFull, part, 1);
            best_s = fmaxf(best_s, __shfl_sync(kFull, part, 0));
            if (best_s >= 1.f / kZeroExit) break;
        }
    }
    n_piv += npv;
    if (unbounded) return 0.f;
    return best_s > 0.f ? __fdiv_rn(1.f, best_s) : INFINITY;
}

// MULTI: global tuple u belongs to object d with tuple0[d] <= u < tuple0[d + 1]
// (all objects of one launch share k and K); each warp keeps its current
// object's arguments in shared memory.
template <bool MULTI, int NS>
__global__ void __launch_bounds__(kScoreThreads, 3) k_score_tuples(const ScoreArgs a1, const ScoreArgs *descs,
                                                                    const long long *tuple0, int n_desc,
                                                                    unsigned total) {
    __shared__ __align__(16) float s_buf[kScoreWarps][16];
    __shared__ ScoreArgs s_obj[MULTI ? kScoreWarps : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = a1.k, K = a1.K, kK = k * K;
    const bool colA = lane < kK;
    const int ci = colA ? lane / K : 0, cm = colA ? lane % K : 0;
    float ec = a1.cs[cm] * a1.mu, es = a1.sn[cm] * a1.mu;
    float *buf = s_buf[warp];
    int cur = -1;
    long long cur0 = 0, cur1 = 0;
    unsigned long long n_piv = 0, n_lp = 0, n_tup = 0;
    unsigned flags = 0, n_acc = 0;

    for (;;) {
        unsigned u0 = 0;
        if (lane == 0) u0 = atomicAdd(a1.work, (unsigned)a1.batch);
        u0 = __shfl_sync(kFull, u0, 0);
        if (u0 >= total) break;
        const unsigned uend = min(u0 + (unsigned)a1.batch, total);
        for (unsigned ug = u0; ug < uend; ++ug) {
            unsigned u = ug;
            if (MULTI) {
                if ((long long)ug < cur0 || (long long)ug >= cur1) {  // switch object
                    int lo = 0, hi = n_desc - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (__ldg(tuple0 + mid) <= (long long)ug) lo = mid; else hi = mid - 1;
                    }
                    cur = lo;
                    cur0 = __ldg(tuple0 + lo);
                    cur1 = __ldg(tuple0 + lo + 1);
                    __syncwarp();
                    const int *src = reinterpret_cast<const int *>(descs + cur);
                    int *dst = reinterpret_cast<int *>(&s_obj[warp]);
                    for (int e = lane; e < (int)(sizeof(ScoreArgs) / sizeof(int)); e += 32) dst[e] = src[e];
                    __syncwarp();
                    ec = s_obj[warp].cs[cm] * s_obj[warp].mu;
                    es = s_obj[warp].sn[cm] * s_obj[warp].mu;
                }
                u = (unsigned)((long long)ug - cur0);
            }
            const ScoreArgs &a = MULTI ? s_obj[warp] : a1;
            const int32_t *st = a.tuples + (size_t)u * k;
            bool valid = true;
            for (int d = 0; d < k; ++d) {
                const int x = __ldg(st + d);
                valid = valid && x >= 0 && x < a.N;
            }
            float margin = INFINITY;
            if (valid) {
                float wv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (colA) {
                    const int x = __ldg(st + ci);
                    const float px = __ldg(a.px + x), py = __ldg(a.py + x), pz = __ldg(a.pz + x);
                    const float vx = -__ldg(a.nx + x), vy = -__ldg(a.ny + x), vz = -__ldg(a.nz + x);
                    // tangent basis of nu (Duff et al. 2017)
                    const float sgn = copysignf(1.f, vz);
                    const float aa = -1.f / (sgn + vz);
                    const float bb = vx * vy * aa;
                    const float xx = 1.f + sgn * vx * vx * aa, xy = sgn * bb, xz = -sgn * vx;
                    const float yx = bb, yy = sgn + vy * vy * aa, yz = -vy;
                    const float ex = vx + ec * xx + es * yx, ey = vy + ec * xy + es * yy, ez = vz + ec * xz + es * yz;
                    const float rx = px - a.cx, ry = py - a.cy, rz = pz - a.cz;
                    wv[0] = ex; wv[1] = ey; wv[2] = ez;
                    wv[3] = (ry * ez - rz * ey) * a.inv_rho;
                    wv[4] = (rz * ex - rx * ez) * a.inv_rho;
                    wv[5] = (rx * ey - ry * ex) * a.inv_rho;
                }
                margin = closure_margin<NS>(wv, k, K, lane, buf, n_piv, n_lp, flags);
                ++n_tup;
            }
            if (lane == 0) {
                a.margin[u] = margin;
                a.accept[u] = (uint8_t)(margin <= a.eps);
                n_acc += margin <= a.eps;
            }
        }
    }
    if (lane == 0) {
        atomicAdd(a1.counters + 0, n_piv);
        atomicAdd(a1.counters + 1, n_lp);
        atomicAdd(a1.counters + 2, n_tup);
        if (flags) atomicOr(a1.status, flags);
        if (a1.n_accept && n_acc) atomicAdd(a1.n_accept, (unsigned long long)n_acc);
    }
}

// ---------------------------------------------------------------------------
// Alg. 2: blockwise zeroth-order contact optimisation
// ---------------------------------------------------------------------------
constexpr int kOptThreads = 128;
constexpr int kOptWarps = kOptThreads / 32;

// Wrench column of this lane (contact ci = lane / K, edge cm) for point x.
__device__ __forceinline__ void wrench_column(const ScoreArgs &a, int x, float ec, float es, float (&wv)[6]) {
    const float px = __ldg(a.px + x), py = __ldg(a.py + x), pz = __ldg(a.pz + x);
    const float vx = -__ldg(a.nx + x), vy = -__ldg(a.ny + x), vz = -__ldg(a.nz + x);
    const float sgn = copysignf(1.f, vz);
    const float aa = -1.f / (sgn + vz);
    const float bb = vx * vy * aa;
    const float xx = 1.f + sgn * vx * vx * aa, xy = sgn * bb, xz = -sgn * vx;
    const float yx = bb, yy = sgn + vy * vy * aa, yz = -vy;
    const float ex = vx + ec * xx + es * yx, ey = vy + ec * xy + es * yy, ez = vz + ec * xz + es * yz;
    const float rx = px - a.cx, ry = py - a.cy, rz = pz - a.cz;
    wv[0] = ex; wv[1] = ey; wv[2] = ez;
    wv[3] = (ry * ez - rz * ey) * a.inv_rho;
    wv[4] = (rz * ex - rx * ez) * a.inv_rho;
    wv[5] = (rx * ey - ry * ex) * a.inv_rho;
}

// Closure margin of the tuple whose contact d is point id_d (min over j of LP_j,
// stopping at a zero), computed by the whole warp.
template <int NS>
__device__ __forceinline__ float tuple_margin(const ScoreArgs &a, int id0, int id1, int id2, int id3, int k, bool colA,
                                              int ci, float ec, float es, int lane, float *buf,
                                              unsigned long long &n_piv, unsigned long long &n_lp, unsigned &flags) {
    float wv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (colA) wrench_column(a, ci == 0 ? id0 : ci == 1 ? id1 : ci == 2 ? id2 : id3, ec, es, wv);
    return closure_margin<NS>(wv, k, a.K, lane, buf, n_piv, n_lp, flags);
}

struct OptArgs {
    int n_outer, n_inner;
    float sigma, zero_tol, min_gain;
};

// One warp per tuple (persistent warps, work counter).  Per outer iteration and
// contact i: NI Gaussian mutations of p_i in its tangent plane (Box-Muller on
// Philox4x32-10 words), each projected onto finger f_i's domain (the nearest
// object point whose mask bit is set; all lanes scan the mask words, then one
// warp reduction per candidate), then the candidates in order replace the best
// so far when their margin is lower by more than the relative min_gain (margins
// <= zero_tol count as 0), so the margin never increases.
template <int NI, int NS>
__global__ void __launch_bounds__(kOptThreads) k_optimize_tuples(const ScoreArgs a, const OptArgs o, unsigned total) {
    __shared__ __align__(16) float s_buf[kOptWarps][16];
    __shared__ float s_cand[kOptWarps][NI][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = a.k, K = a.K, kK = k * K, F = a.F, W = a.W;
    const bool colA = lane < kK;
    const int ci = colA ? lane / K : 0, cm = colA ? lane % K : 0;
    const float ec = a.cs[cm] * a.mu, es = a.sn[cm] * a.mu;
    float *buf = s_buf[warp];
    unsigned long long n_piv = 0, n_lp = 0, n_tup = 0;
    unsigned flags = 0;
    const uint2 key = make_uint2(a.seed_lo, a.seed_hi);
    const int blocks_per_draw = (NI + 1) / 2;
    for (;;) {
        unsigned u = 0;
        if (lane == 0) u = atomicAdd(a.work, 1u);
        u = __shfl_sync(kFull, u, 0);
        if (u >= total) break;
        const int pose = (int)(u / (unsigned)a.T), tau = (int)(u % (unsigned)a.T);
        int id[CF_MAX_K] = {0, 0, 0, 0}, fg[CF_MAX_K] = {0, 0, 0, 0};
        bool valid = true;
        for (int d = 0; d < k; ++d) {
            id[d] = __ldg(a.tuples + (size_t)u * k + d);
            fg[d] = (int)__ldg(a.fingers + (size_t)u * k + d);
            valid = valid && id[d] >= 0 && id[d] < a.N && fg[d] < F;
        }
        float J = INFINITY;
        if (valid) {
            J = tuple_margin<NS>(a, id[0], id[1], id[2], id[3], k, colA, ci, ec, es, lane, buf, n_piv, n_lp, flags);
            float Jc = J <= o.zero_tol ? 0.f : J;
            const uint32_t pid = (uint32_t)pose + a.pose_base;
            for (int it = 0; it < o.n_outer && Jc > 0.f; ++it) {
                for (int i = 0; i < k && Jc > 0.f; ++i) {
                    const int x0 = i == 0 ? id[0] : i == 1 ? id[1] : i == 2 ? id[2] : id[3];
                    const int fi = i == 0 ? fg[0] : i == 1 ? fg[1] : i == 2 ? fg[2] : fg[3];
                    // tangent basis of nu = -n at the current point (Duff et al. 2017); this
                    // and the mutated points use explicitly rounded FP32 operations, so the
                    // projection below (an index decision) is reproducible operation by operation
                    const float px = __ldg(a.px + x0), py = __ldg(a.py + x0), pz = __ldg(a.pz + x0);
                    const float vx = -__ldg(a.nx + x0), vy = -__ldg(a.ny + x0), vz = -__ldg(a.nz + x0);
                    const float sgn = copysignf(1.f, vz);
                    const float aa = __fdiv_rn(-1.f, __fadd_rn(sgn, vz));
                    const float bb = __fmul_rn(__fmul_rn(vx, vy), aa);
                    const float xx = __fadd_rn(1.f, __fmul_rn(__fmul_rn(__fmul_rn(sgn, vx), vx), aa));
                    const float xy = __fmul_rn(sgn, bb), xz = -__fmul_rn(sgn, vx);
                    const float yx = bb, yy = __fadd_rn(sgn, __fmul_rn(__fmul_rn(vy, vy), aa)), yz = -vy;
                    if (lane < NI) {  // candidate `lane`: one Box-Muller pair, FP64 then rounded to FP32
                        const int c = lane;
                        const uint4 w4 = philox4x32_10(
                            make_uint4(pid, (uint32_t)tau, (uint32_t)((it * k + i) * blocks_per_draw + c / 2), 0xA162u),
                            key);
                        const uint32_t w0 = (c & 1) ? w4.z : w4.x, w1 = (c & 1) ? w4.w : w4.y;
                        const double u1 = (double)((w0 >> 8) + 1u) * 5.9604644775390625e-8;  // (0, 1]
                        const double u2 = (double)(w1 >> 8) * 5.9604644775390625e-8;         // [0, 1)
                        const double r = sqrt(-2.0 * log(u1));
                        double sd, cd;
                        sincospi(2.0 * u2, &sd, &cd);
                        const float g1 = (float)(r * cd), g2 = (float)(r * sd);
                        const float sg = o.sigma;
                        s_cand[warp][c][0] = __fadd_rn(px, __fmul_rn(sg, __fadd_rn(__fmul_rn(g1, xx), __fmul_rn(g2, yx))));
                        s_cand[warp][c][1] = __fadd_rn(py, __fmul_rn(sg, __fadd_rn(__fmul_rn(g1, xy), __fmul_rn(g2, yy))));
                        s_cand[warp][c][2] = __fadd_rn(pz, __fmul_rn(sg, __fadd_rn(__fmul_rn(g1, xz), __fmul_rn(g2, yz))));
                    }
                    __syncwarp();
                    // projection onto the domain: lanes scan mask words lane, lane + 32, ...
                    float bd[NI];
                    int bi[NI];
#pragma unroll
                    for (int c = 0; c < NI; ++c) { bd[c] = INFINITY; bi[c] = INT_MAX; }
                    const uint32_t *row = a.masks + ((size_t)pose * F + fi) * W;
                    for (int w = lane; w < W; w += 32) {
                        uint32_t bits = __ldg(row + w);
                        while (bits) {
                            const int b = __ffs(bits) - 1;
                            bits &= bits - 1;
                            const int x = 32 * w + b;
                            const float qx = __ldg(a.px + x), qy = __ldg(a.py + x), qz = __ldg(a.pz + x);
#pragma unroll
                            for (int c = 0; c < NI; ++c) {
                                const float dx = __fsub_rn(qx, s_cand[warp][c][0]), dy = __fsub_rn(qy, s_cand[warp][c][1]),
                                            dz = __fsub_rn(qz, s_cand[warp][c][2]);
                                const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                                if (d2 < bd[c]) { bd[c] = d2; bi[c] = x; }
                            }
                        }
                    }
                    int cand_mine = -1;  // lane c < NI keeps candidate c's point
#pragma unroll
                    for (int c = 0; c < NI; ++c) {
                        const unsigned kd = fkey(bd[c]);
                        const unsigned kmin = __reduce_min_sync(kFull, kd);
                        const unsigned imin = __reduce_min_sync(kFull, kd == kmin ? (unsigned)bi[c] : 0xffffffffu);
                        if (lane == c) cand_mine = imin == 0xffffffffu ? -1 : (int)imin;
                    }
                    // candidates equal to the current point or to an earlier candidate cannot win
                    const unsigned same = __match_any_sync(kFull, lane < NI ? cand_mine : -2 - lane);
                    const bool skip = lane >= NI || cand_mine < 0 || cand_mine == x0 ||
                                      (same & ((1u << lane) - 1u)) != 0u;
                    const unsigned todo = __ballot_sync(kFull, !skip);
                    float best = Jc, bestJ = J;
                    int bestc = -1;
                    for (unsigned m = todo; m; m &= m - 1) {
                        const int c = __ffs(m) - 1;
                        const int xc = __shfl_sync(kFull, cand_mine, c);
                        const float Jt = tuple_margin<NS>(a, i == 0 ? xc : id[0], i == 1 ? xc : id[1],
                                                      i == 2 ? xc : id[2], i == 3 ? xc : id[3], k, colA, ci, ec, es,
                                                      lane, buf, n_piv, n_lp, flags);
                        const float Jtc = Jt <= o.zero_tol ? 0.f : Jt;
                        if (Jtc < (1.f - o.min_gain) * best) { best = Jtc; bestJ = Jt; bestc = xc; }
                    }
                    if (bestc >= 0) {
                        if (i == 0) id[0] = bestc; else if (i == 1) id[1] = bestc; else if (i == 2) id[2] = bestc; else id[3] = bestc;
                        Jc = best;
                        J = bestJ;
                    }
                }
            }
            ++n_tup;
        }
        if (lane == 0) {
            if (valid)
                for (int d = 0; d < k; ++d) a.tuples[(size_t)u * k + d] = id[d];
            a.margin[u] = J;
            a.accept[u] = (uint8_t)(J <= a.eps);
        }
        __syncwarp();
    }
    if (lane == 0) {
        atomicAdd(a.counters + 0, n_piv);
        atomicAdd(a.counters + 1, n_lp);
        atomicAdd(a.counters + 2, n_tup);
        if (flags) atomicOr(a.status, flags);
    }
}

}  // namespace

size_t score_smem_bytes(int F, int W, int T, int k, bool sampling) {
    (void)T;
    (void)k;
    const int G = (W + 31) / 32;
    return sampling ? sizeof(uint32_t) * ((size_t)F * W + (size_t)F * (G + 1)) : 0;
}

cudaError_t launch_sample(const ScoreArgs &a, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    const size_t smem = score_smem_bytes(a.F, a.W, a.T, a.k, true);
    if (smem > 48 * 1024) {
        cudaError_t err =
            cudaFuncSetAttribute(k_sample_tuples<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    k_sample_tuples<false><<<a.P, kSampleThreads, smem, st>>>(a, nullptr, nullptr, 0);
    return cudaGetLastError();
}

namespace {
// slots per lane of the scaled LP: kK + 6 columns fit one slot when kK <= 26
inline int lp_slots(int k, int K) { return k * K + kRows <= 32 ? 1 : 2; }

template <bool MULTI, int NS>
cudaError_t launch_score_grid(const ScoreArgs &a1, const ScoreArgs *descs, const long long *tuple0, int n_desc,
                              long long total, cudaStream_t st) {
    cudaError_t err;
    int dev = 0, sms = 0, per_sm = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_score_tuples<MULTI, NS>, kScoreThreads, 0)) !=
        cudaSuccess)
        return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (a1.batch < 1) return cudaErrorInvalidValue;
    if (a1.bpsm > 0) per_sm = std::min(per_sm, a1.bpsm);
    const long long warps_needed = (total + a1.batch - 1) / a1.batch;
    const int grid = (int)std::min<long long>((long long)sms * per_sm, (warps_needed + kScoreWarps - 1) / kScoreWarps);
    k_score_tuples<MULTI, NS><<<grid, kScoreThreads, 0, st>>>(a1, descs, tuple0, n_desc, (unsigned)total);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_score(const ScoreArgs &a, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    cudaError_t err;
    if (!a.tuples_given && (err = launch_sample(a, st)) != cudaSuccess) return err;
    return lp_slots(a.k, a.K) == 1 ? launch_score_grid<false, 1>(a, nullptr, nullptr, 0, (long long)a.P * a.T, st)
                                   : launch_score_grid<false, 2>(a, nullptr, nullptr, 0, (long long)a.P * a.T, st);
}

cudaError_t launch_optimize(const ScoreArgs &a, int n_outer, int n_inner, float sigma, float zero_tol,
                            float min_gain, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    const OptArgs o{n_outer, n_inner, sigma, zero_tol, min_gain};
    const long long total = (long long)a.P * a.T;
    cudaError_t err;
    int dev = 0, sms = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    const long long want = (total + kOptWarps - 1) / kOptWarps;
    const int grid = (int)std::min<long long>((long long)sms * 16, want);
    const bool one = lp_slots(a.k, a.K) == 1;
    switch (n_inner) {
#define CF_OPT(NI)                                                                                        \
    case NI:                                                                                              \
        if (one) k_optimize_tuples<NI, 1><<<grid, kOptThreads, 0, st>>>(a, o, (unsigned)total);           \
        else k_optimize_tuples<NI, 2><<<grid, kOptThreads, 0, st>>>(a, o, (unsigned)total);               \
        break;
        CF_OPT(4) CF_OPT(8) CF_OPT(16)
#undef CF_OPT
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_sample_batch(const ScoreArgs *d_descs, const long long *d_pose0, int n_desc, long long total_poses,
                                size_t smem, cudaStream_t st) {
    if (total_poses <= 0) return cudaSuccess;
    if (smem > 48 * 1024) {
        cudaError_t err =
            cudaFuncSetAttribute(k_sample_tuples<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    ScoreArgs dummy;
    memset(&dummy, 0, sizeof dummy);
    k_sample_tuples<true><<<(unsigned)total_poses, kSampleThreads, smem, st>>>(dummy, d_descs, d_pose0, n_desc);
    return cudaGetLastError();
}

cudaError_t launch_score_batch(const ScoreArgs &launch, const ScoreArgs *d_descs, const long long *d_tuple0, int n_desc,
                               long long total_tuples, cudaStream_t st) {
    if (total_tuples <= 0) return cudaSuccess;
    return lp_slots(launch.k, launch.K) == 1
               ? launch_score_grid<true, 1>(launch, d_descs, d_tuple0, n_desc, total_tuples, st)
               : launch_score_grid<true, 2>(launch, d_descs, d_tuple0, n_desc, total_tuples, st);
}

}  // namespace cf
