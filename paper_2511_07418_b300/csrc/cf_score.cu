// Tuple sampling + closure margin kernels (Sec. 5.3, Alg. 2 Random(D_i); Eq. GSWO, Sec. 3.2).
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
// k_sample_tuples: one block per pose builds popcount prefixes per 8-word
// group of its F mask rows in shared memory (reading the rows once, coalesced);
// one thread per tuple draws its fingers and points (Philox4x32-10), finds each
// point's group by binary search and its bit in the group's words, and writes
// them out.
//
// k_score_lanes: each lane scores its own tuples, the k LPs of a tuple in the
// scaled bounded-variable form below, solved by a revised simplex whose state
// (a 6 x 6 basis inverse and the simplex multipliers) lives in the lane's
// registers; LP_{j+1} starts from LP_j's basis.  The warp-per-LP form of the
// same simplex (closure_margin) scores the candidates of Alg. 2.  FP32
// throughout.
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

// words per prefix group of a mask row
constexpr int kGroupWords = 8;

// r-th set bit (ascending) of the mask row `row` (global memory), -1 if the row
// has <= r bits.  gp = exclusive prefix of the row's group popcounts (shared
// memory, G + 1 entries): a binary search finds the group, whose <= 8 words are
// loaded together and scanned.
__device__ __forceinline__ int select_in_row(const uint32_t *__restrict__ row, const uint32_t *gp, int W, int G,
                                             uint32_t r) {
    if (r >= gp[G]) return -1;
    int lo = 0, hi = G - 1;  // largest g with gp[g] <= r
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gp[mid] <= r) lo = mid; else hi = mid - 1;
    }
    uint32_t rr = r - gp[lo];
    const int wb = kGroupWords * lo, n = min(kGroupWords, W - wb);
    uint32_t v[kGroupWords];
#pragma unroll
    for (int q = 0; q < kGroupWords; ++q) v[q] = q < n ? __ldg(row + wb + q) : 0u;
    int out = -1;
#pragma unroll
    for (int q = 0; q < kGroupWords; ++q) {
        const uint32_t c = __popc(v[q]);
        if (out < 0 && rr < c) out = 32 * (wb + q) + select_in_word(v[q], rr);
        if (out < 0) rr -= c;
    }
    return out;
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
    const int G = (W + kGroupWords - 1) / kGroupWords;
    uint32_t *s_gpre = s_dyn;  // [F][G + 1]
    const int i = MULTI ? s_i : (int)blockIdx.x;
    if (threadIdx.x < F) s_cnt[threadIdx.x] = a.counts[(size_t)i * F + threadIdx.x];
    const uint32_t *src = a.masks + (size_t)i * F * W;
    // group sums straight from the masks (no staging): a warp takes 128 consecutive words of a row, four
    // independent coalesced loads per lane, and adds the popcounts in groups of kGroupWords lanes
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    constexpr int kLoads = 8;  // words per lane in flight
    const int CW = (W + 32 * kLoads - 1) / (32 * kLoads);
    for (int ch = warp; ch < F * CW; ch += nwarps) {
        const int f = ch / CW, w0 = (ch % CW) * 32 * kLoads;
        const uint32_t *row = src + (size_t)f * W;
        uint32_t v[kLoads];
#pragma unroll
        for (int q = 0; q < kLoads; ++q) {
            const int w = w0 + 32 * q + lane;
            v[q] = w < W ? __ldg(row + w) : 0u;
        }
#pragma unroll
        for (int q = 0; q < kLoads; ++q) {
            const int w = w0 + 32 * q + lane;
            uint32_t c = __popc(v[q]);
#pragma unroll
            for (int o = 1; o < kGroupWords; o <<= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (lane % kGroupWords == 0 && w < W) s_gpre[f * (G + 1) + 1 + w / kGroupWords] = c;
        }
    }
    __syncthreads();
    // exclusive prefix of the group sums per row: one warp per row, 32 groups per step
    for (int f = warp; f < F; f += nwarps) {
        uint32_t *gp = s_gpre + f * (G + 1);
        uint32_t carry = 0;
        for (int g0 = 0; g0 < G; g0 += 32) {
            const int g = g0 + lane;
            uint32_t v = g < G ? gp[1 + g] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            if (g < G) gp[1 + g] = v + carry;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
        if (lane == 0) gp[0] = 0;
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
            gt[d] = select_in_row(src + (size_t)f * W, s_gpre + f * (G + 1), W, G, r);
            if (gf) gf[d] = (uint8_t)f;
        }
    }
}

// ---------------------------------------------------------------------------
// scoring
// ---------------------------------------------------------------------------
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

// The feasible start c' = 0, y = 0 (every y_r basic, B = I) of the tuple whose
// wrench column on this lane is w (lanes < kK).
template <int NS>
__device__ __forceinline__ void lp_init_cold(BoxLp<NS> &s, const float (&w)[6], int kK, int lane) {
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
}

// Warm start with repair (Sec. 5.4, "A Free Lunch"): state s is an optimal
// basis of the current tuple; the trial tuple moves contact ci, whose new wrench
// column on this lane is w (lanes of contact ci).  Contact ci's columns get
// their new tableau B^-1 (-w); each of them that is basic is then swapped for
// its own new version by a pivot on its row (a column-replacement pivot), so
// the basis keeps its variables with contact ci's new columns; the basic values
// are recomputed from the nonbasic bounds (c' = 0, y = -1 or +1).  Returns false
// when a replacement pivot is too small (the new basis is near singular) or the
// recomputed basis is infeasible; s is then unusable and the caller starts cold.
template <int NS>
__device__ bool lp_warm_repair(BoxLp<NS> &s, const float (&w)[6], int ci, int k, int K, int lane, float *buf) {
    const int kK = k * K, c0 = ci * K, c1 = c0 + K;
    // stage B^-1 = [T(y_0) .. T(y_5)] as buf[r' * 6 + r]
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        const int yr = NS == 1 ? lane - kK : (q == 1 ? lane : -1);
        if (yr >= 0 && yr < kRows) {
#pragma unroll
            for (int r = 0; r < kRows; ++r) buf[yr * kRows + r] = s.T[q][r];
        }
    }
    __syncwarp();
    if (lane >= c0 && lane < c1) {  // slot 0 of lane c is column c
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int rr = 0; rr < kRows; ++rr) acc = __fmaf_rn(buf[rr * kRows + r], -w[rr], acc);
            s.T[0][r] = acc;
        }
    }
    __syncwarp();
    // column-replacement pivots on the rows whose basic variable is a column of contact ci
    unsigned rows = __ballot_sync(kFull, lane < kRows && s.beta >= c0 && s.beta < c1) & ((1u << kRows) - 1u);
    bool ok = true;
    while (rows) {
        const int l = __ffs(rows) - 1;
        rows &= rows - 1;
        const int e = __shfl_sync(kFull, s.beta, l);  // the variable (lane e, slot 0)
        if (lane == e) {
#pragma unroll
            for (int r = 0; r < kRows; ++r) buf[r] = s.T[0][r];
        }
        __syncwarp();
        float col[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) col[r] = buf[r];
        __syncwarp();
        float piv = col[0];
#pragma unroll
        for (int r = 1; r < kRows; ++r) piv = r == l ? col[r] : piv;
        if (!(fabsf(piv) > 1e-4f)) { ok = false; break; }  // warp-uniform
        const float inv = __frcp_rn(piv);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            float tl = s.T[q][0];
#pragma unroll
            for (int r = 1; r < kRows; ++r) tl = r == l ? s.T[q][r] : tl;
            const float pa = __fmul_rn(tl, inv);
#pragma unroll
            for (int r = 0; r < kRows; ++r) s.T[q][r] = r == l ? pa : __fmaf_rn(-col[r], pa, s.T[q][r]);
        }
    }
    if (!ok) return false;
    // basic values: B x_B = -N x_N, x_N = -1 / +1 for nonbasic y at the lower / upper bound, 0 for c'
    float contrib[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) contrib[r] = 0.f;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        const int yr = NS == 1 ? lane - kK : (q == 1 ? lane : -1);
        if (yr >= 0 && yr < kRows && s.st[q] != 0) {
            const float val = s.st[q] == 2 ? 1.f : -1.f;
#pragma unroll
            for (int r = 0; r < kRows; ++r) contrib[r] = __fmaf_rn(-s.T[q][r], val, contrib[r]);
        }
    }
    float vr = 0.f;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        float x = contrib[r];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        if (lane == r) vr = x;
    }
    bool feas = true;
    if (lane < kRows) {
        const bool bx = s.beta < kK;
        if (bx) { feas = vr >= -1e-6f; vr = fmaxf(vr, 0.f); }
        else { feas = vr >= -1.f - 1e-6f && vr <= 1.f + 1e-6f; vr = fminf(fmaxf(vr, -1.f), 1.f); }
        s.v = vr;
    }
    return __all_sync(kFull, feas);
}

// LP_j from the feasible state s: returns s_j (+inf when unbounded, i.e.
// LP_j = 0); s ends in its final basis.
template <int NS>
__device__ float lp_solve_one(BoxLp<NS> &s, int j, int k, int K, int lane, float *buf, unsigned long long &n_piv,
                              unsigned long long &n_lp, unsigned &flags) {
    const int kK = k * K;
    const unsigned kinf = fkey(INFINITY);
    const unsigned kzero = fkey(0.f);
    unsigned npv = 0;
    bool unbounded = false;
    {
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
    }
    ++n_lp;
    n_piv += npv;
    if (unbounded) return INFINITY;
    // s_j = the sum of contact j's basic values (nonbasic c' sit at 0)
    const int c0 = j * K, c1 = c0 + K;
    float part = (lane < kRows && s.beta >= c0 && s.beta < c1) ? s.v : 0.f;
    part += __shfl_xor_sync(kFull, part, 4);
    part += __shfl_xor_sync(kFull, part, 2);
    part += __shfl_xor_sync(kFull, part, 1);
    return __shfl_sync(kFull, part, 0);
}

// Closure margin min_j LP_j from the feasible state s (each LP_j starts from
// the basis the previous one ended in).  Stops at the first unbounded s_j
// (margin 0).  s ends in the last LP's final basis.
template <int NS>
__device__ float lp_solve_margin(BoxLp<NS> &s, int k, int K, int lane, float *buf, unsigned long long &n_piv,
                                 unsigned long long &n_lp, unsigned &flags) {
    float best_s = 0.f;
    for (int j = 0; j < k; ++j) {
        const float sj = lp_solve_one<NS>(s, j, k, K, lane, buf, n_piv, n_lp, flags);
        if (!(sj < INFINITY)) return 0.f;
        best_s = fmaxf(best_s, sj);
        if (best_s >= 1.f / kZeroExit) break;
    }
    return best_s > 0.f ? __fdiv_rn(1.f, best_s) : INFINITY;
}

// Closure margin min_j LP_j of one tuple on the warp, from the cold start.
template <int NS>
__device__ float closure_margin(const float (&w)[6], int k, int K, int lane, float *buf, unsigned long long &n_piv,
                                unsigned long long &n_lp, unsigned &flags) {
    BoxLp<NS> s;
    lp_init_cold<NS>(s, w, k * K, lane);
    return lp_solve_margin<NS>(s, k, K, lane, buf, n_piv, n_lp, flags);
}

// Bounding box of the (up to) 32 points of each mask word: warp per word.
__global__ void k_word_boxes(const float *__restrict__ px, const float *__restrict__ py, const float *__restrict__ pz,
                             int N, int W, float *__restrict__ box) {
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= W) return;
    const int x = 32 * w + lane;
    const bool ok = x < N;
    float v[3] = {ok ? __ldg(px + x) : 0.f, ok ? __ldg(py + x) : 0.f, ok ? __ldg(pz + x) : 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float lo = ok ? v[c] : INFINITY, hi = ok ? v[c] : -INFINITY;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(kFull, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(kFull, hi, o));
        }
        if (lane == 0) {
            box[6 * (size_t)w + c] = lo;
            box[6 * (size_t)w + 3 + c] = hi;
        }
    }
}

// ---------------------------------------------------------------------------
// Alg. 2: blockwise zeroth-order contact optimisation
// ---------------------------------------------------------------------------
// A warp's simplex state in shared memory: word w of lane l at p[w * 32 + l]
// (conflict-free), kStateWords(NS) words per lane.
template <int NS>
__host__ __device__ constexpr int state_words() { return NS * (kRows + 2) + 2; }

template <int NS>
__device__ __forceinline__ void state_store(float *p, int lane, const BoxLp<NS> &s) {
#pragma unroll
    for (int q = 0; q < NS; ++q) {
#pragma unroll
        for (int r = 0; r <= kRows; ++r) p[(q * (kRows + 2) + r) * 32 + lane] = s.T[q][r];
        p[(q * (kRows + 2) + kRows + 1) * 32 + lane] = __int_as_float(s.st[q]);
    }
    p[(NS * (kRows + 2)) * 32 + lane] = s.v;
    p[(NS * (kRows + 2) + 1) * 32 + lane] = __int_as_float(s.beta);
}

template <int NS>
__device__ __forceinline__ void state_load(const float *p, int lane, BoxLp<NS> &s) {
#pragma unroll
    for (int q = 0; q < NS; ++q) {
#pragma unroll
        for (int r = 0; r <= kRows; ++r) s.T[q][r] = p[(q * (kRows + 2) + r) * 32 + lane];
        s.st[q] = __float_as_int(p[(q * (kRows + 2) + kRows + 1) * 32 + lane]);
    }
    s.v = p[(NS * (kRows + 2)) * 32 + lane];
    s.beta = __float_as_int(p[(NS * (kRows + 2) + 1) * 32 + lane]);
}
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

struct OptArgs {
    int n_outer, n_inner;
    float sigma, zero_tol, min_gain;
    int warm_start;
};

// One warp per tuple (persistent warps, work counter).  Per outer iteration and
// contact i: NI Gaussian mutations of p_i in its tangent plane (Box-Muller on
// Philox4x32-10 words), each projected onto finger f_i's domain (the nearest
// object point whose mask bit is set; all lanes scan the mask words, then one
// warp reduction per candidate), then the candidates in order replace the best
// so far when their margin is lower by more than the relative min_gain (margins
// <= zero_tol count as 0), so the margin never increases.  The free lunch of
// Sec. 5.4: the current tuple's optimal basis of each LP_j stays in shared
// memory, and a candidate's LP_j starts from it, repaired for the moved
// contact (lp_warm_repair), whenever the repaired basis is feasible; else from
// the candidate's previous LP's basis, or c' = 0.  Three state buffers per
// warp: the current tuple's, the best candidate's so far, the trial's.
template <int NI, int NS>
__global__ void __launch_bounds__(kOptThreads) k_optimize_tuples(const ScoreArgs a, const OptArgs o, unsigned total) {
    __shared__ __align__(16) float s_buf[kOptWarps][kRows * kRows];  // entering column; B^-1 for warm starts
    __shared__ float s_cand[kOptWarps][NI][3];
    extern __shared__ float s_states[];  // [warp][3 buffers][k][state_words][32]
    constexpr int SW = state_words<NS>();
    float *const states = s_states + (size_t)(threadIdx.x >> 5) * 3 * a.k * SW * 32;
    auto slot = [&](int b, int j) { return states + ((size_t)b * a.k + j) * SW * 32; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = a.k, K = a.K, kK = k * K, F = a.F, W = a.W;
    const bool colA = lane < kK;
    const int ci = colA ? lane / K : 0, cm = colA ? lane % K : 0;
    const float ec = a.cs[cm] * a.mu, es = a.sn[cm] * a.mu;
    float *buf = s_buf[warp];
    unsigned long long n_piv = 0, n_lp = 0, n_tup = 0, n_warm = 0;
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
            // the current tuple's optimal basis of each LP_j: the warm starts of its candidates (Sec. 5.4)
            int b_cur = 0, b_best = 1, b_trial = 2, n_cur = 0, n_best = 0;
            {
                float wv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (colA) wrench_column(a, ci == 0 ? id[0] : ci == 1 ? id[1] : ci == 2 ? id[2] : id[3], ec, es, wv);
                BoxLp<NS> st;
                lp_init_cold<NS>(st, wv, kK, lane);
                float bs = 0.f;
                bool zero = false;
                for (int j = 0; j < k; ++j) {
                    const float sj = lp_solve_one<NS>(st, j, k, K, lane, buf, n_piv, n_lp, flags);
                    state_store<NS>(slot(b_cur, j), lane, st);
                    n_cur = j + 1;
                    if (!(sj < INFINITY)) { zero = true; break; }
                    bs = fmaxf(bs, sj);
                    if (bs >= 1.f / kZeroExit) break;
                }
                J = zero ? 0.f : (bs > 0.f ? __fdiv_rn(1.f, bs) : INFINITY);
            }
            float Jc = J <= o.zero_tol ? 0.f : J;
            const uint32_t pid = (uint32_t)pose + a.pose_base;
            for (int it = 0; it < o.n_outer && Jc > 0.f; ++it) {
                for (int i = 0; i < k && Jc > 0.f; ++i) {
                    const int x0 = i == 0 ? id[0] : i == 1 ? id[1] : i == 2 ? id[2] : id[3];
                    const int fi = i == 0 ? fg[0] : i == 1 ? fg[1] : i == 2 ? fg[2] : fg[3];
                    // tangent basis of nu = -n at the current point (Duff et al. 2017) and the mutated
                    // points in explicitly rounded FP32 operations (no contraction left to the compiler)
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
                    // exact pruning: the current point x0 lies in the domain, so every candidate q_c has a
                    // domain point within |q_c - p0| and its nearest lies within R = 2 max_c |q_c - p0| of
                    // p0; words whose box is farther than R from p0 hold none (R with slack for rounding;
                    // no pruning when x0's bit is not set, e.g. for given tuples outside the domain)
                    float rc = 0.f;
                    if (lane < NI) {
                        const float dx = s_cand[warp][lane][0] - px, dy = s_cand[warp][lane][1] - py,
                                    dz = s_cand[warp][lane][2] - pz;
                        rc = sqrtf(dx * dx + dy * dy + dz * dz);
                    }
                    rc = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(rc)));  // rc >= 0: bits order
                    const bool in_dom = (__ldg(row + (x0 >> 5)) >> (x0 & 31)) & 1u;
                    const float R = 2.f * rc * 1.0001f + 1e-6f;
                    const float R2 = in_dom ? R * R : INFINITY;
                    for (int w = lane; w < W; w += 32) {
                        uint32_t bits = __ldg(row + w);
                        if (bits && R2 < INFINITY) {
                            const float *bx = a.word_box + 6 * (size_t)w;
                            const float ex = fmaxf(fmaxf(__ldg(bx) - px, px - __ldg(bx + 3)), 0.f);
                            const float ey = fmaxf(fmaxf(__ldg(bx + 1) - py, py - __ldg(bx + 4)), 0.f);
                            const float ez = fmaxf(fmaxf(__ldg(bx + 2) - pz, pz - __ldg(bx + 5)), 0.f);
                            if (ex * ex + ey * ey + ez * ez > R2) bits = 0u;  // every point of the word is farther
                        }
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
                        // the trial tuple's wrench column on this lane (contact i moved to xc)
                        float wt[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                        if (colA)
                            wrench_column(a, ci == i ? xc : (ci == 0 ? id[0] : ci == 1 ? id[1] : ci == 2 ? id[2] : id[3]),
                                          ec, es, wt);
                        // each LP_j from the current tuple's optimal LP_j basis repaired for the moved contact
                        // (warm), else from this candidate's previous LP's basis, else from c' = 0
                        float bs = 0.f;
                        bool zero = false;
                        int nt = 0;
                        BoxLp<NS> chain;
                        for (int j = 0; j < k; ++j) {
                            BoxLp<NS> st;
                            bool warm = false;
                            if (o.warm_start && j < n_cur) {
                                state_load<NS>(slot(b_cur, j), lane, st);
                                warm = lp_warm_repair<NS>(st, wt, i, k, K, lane, buf);
                            }
                            if (warm) ++n_warm;
                            else if (j > 0) st = chain;
                            else lp_init_cold<NS>(st, wt, kK, lane);
                            const float sj = lp_solve_one<NS>(st, j, k, K, lane, buf, n_piv, n_lp, flags);
                            state_store<NS>(slot(b_trial, j), lane, st);
                            nt = j + 1;
                            chain = st;
                            if (!(sj < INFINITY)) { zero = true; break; }
                            bs = fmaxf(bs, sj);
                            if (bs >= 1.f / kZeroExit) break;
                        }
                        const float Jt = zero ? 0.f : (bs > 0.f ? __fdiv_rn(1.f, bs) : INFINITY);
                        const float Jtc = Jt <= o.zero_tol ? 0.f : Jt;
                        if (Jtc < (1.f - o.min_gain) * best) {
                            best = Jtc;
                            bestJ = Jt;
                            bestc = xc;
                            const int t = b_best; b_best = b_trial; b_trial = t;  // the trial's states: the best's
                            n_best = nt;
                        }
                    }
                    if (bestc >= 0) {
                        if (i == 0) id[0] = bestc; else if (i == 1) id[1] = bestc; else if (i == 2) id[2] = bestc; else id[3] = bestc;
                        Jc = best;
                        J = bestJ;
                        const int t = b_cur; b_cur = b_best; b_best = t;  // the winner's states: the current tuple's
                        n_cur = n_best;
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
        atomicAdd(a.counters + 3, n_warm);
        if (flags) atomicOr(a.status, flags);
    }
}

// ---------------------------------------------------------------------------
// Lane-per-tuple scoring
// ---------------------------------------------------------------------------
// Each lane solves its own tuple's k LPs (the scaled bounded form above) with a
// revised simplex.  The 6 x 6 basis inverse B^-1 (of the rows -W c' + y = 0,
// starting from the y basis, B = I), the basic values and the simplex
// multipliers pi = c_B B^-1 live in registers.  The columns are never stored:
// column (i, m) is w_im = [nu_i + ec_m x_i + es_m y_i ; t_nu + ec_m t_x + es_m t_y]
// (ec_m, es_m = mu cos, mu sin of edge m; t_* = r_i x (*) / rho), so the lane keeps
// the 18 numbers of each contact in its own stretch of shared memory, and
// pricing needs three 6-term dot products per contact, alpha_i, beta_i,
// gamma_i, after which d_im = [i = j] + alpha_i + ec_m beta_i + es_m gamma_i
// costs two FMAs.  d = -pi_r for y_r.  Dantzig pricing (the lowest id on
// ties; Bland after a run of degenerate pivots); the entering column is
// u = B^-1 a_e; the ratio test, bound flips and tie rules are those of the warp
// solver; a pivot updates B^-1, the basic values and pi in place.  Lanes run
// independently; lanes that finished a tuple take new ones together, when
// `refill` lanes of the warp wait (8 by default) or no lane is in an LP, so the
// tuple set-up mostly runs converged.  Each block scores a contiguous share of the tuples.
constexpr int kLaneThreads = 128;
constexpr float kDTolRel = 4e-6f;  // reduced-cost tolerance per unit of max |pi_r|
constexpr int kContactFloats = 20;                             // 18 used, padded to five float4
constexpr int kLaneStride = kContactFloats * CF_MAX_K + 4;     // 84 floats: stride / 4 odd, float4 loads conflict-free

// An object's arguments as a lane needs them (the kernel's own, or its object's descriptor).
struct LaneObj {
    const float *px, *py, *pz, *nx, *ny, *nz;
    float cx, cy, cz, inv_rho, mu, eps;
    int N;
    const int32_t *tuples;
    float *margin;
    uint8_t *accept;
};

__device__ __forceinline__ LaneObj lane_obj(const ScoreArgs &a) {
    return LaneObj{a.px, a.py, a.pz, a.nx, a.ny, a.nz, a.cx, a.cy, a.cz, a.inv_rho, a.mu, a.eps, a.N,
                   a.tuples, a.margin, a.accept};
}

// The contact's 18 numbers (nu, x, y, t_nu, t_x, t_y), rounded like wrench_column.
__device__ __forceinline__ void contact_frame(const LaneObj &a, int x, float *dst) {
    const float px = __ldg(a.px + x), py = __ldg(a.py + x), pz = __ldg(a.pz + x);
    const float vx = -__ldg(a.nx + x), vy = -__ldg(a.ny + x), vz = -__ldg(a.nz + x);
    const float sgn = copysignf(1.f, vz);
    const float aa = -__frcp_rn(sgn + vz);  // = -1 / (sgn + vz), correctly rounded
    const float bb = vx * vy * aa;
    const float xx = 1.f + sgn * vx * vx * aa, xy = sgn * bb, xz = -sgn * vx;
    const float yx = bb, yy = sgn + vy * vy * aa, yz = -vy;
    const float rx = px - a.cx, ry = py - a.cy, rz = pz - a.cz, ir = a.inv_rho;
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    d4[0] = make_float4(vx, vy, vz, xx);
    d4[1] = make_float4(xy, xz, yx, yy);
    d4[2] = make_float4(yz, (ry * vz - rz * vy) * ir, (rz * vx - rx * vz) * ir, (rx * vy - ry * vx) * ir);
    d4[3] = make_float4((ry * xz - rz * xy) * ir, (rz * xx - rx * xz) * ir, (rx * xy - ry * xx) * ir,
                        (ry * yz - rz * yy) * ir);
    d4[4] = make_float4((rz * yx - rx * yz) * ir, (rx * yy - ry * yx) * ir, 0.f, 0.f);
}

struct Frame {
    float v[18];
};

__device__ __forceinline__ Frame load_frame(const float *src) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    const float4 f0 = s4[0], f1 = s4[1], f2 = s4[2], f3 = s4[3], f4 = s4[4];
    return Frame{{f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w, f2.x, f2.y, f2.z, f2.w, f3.x, f3.y, f3.z, f3.w, f4.x,
                  f4.y}};
}

// KT: the edge count when known at compile time (0: a.K at run time, <= CF_MAX_EDGES).
// MULTI: global tuple u belongs to object d with tuple0[d] <= u < tuple0[d + 1]
// (all objects share k and K); a lane reads its object's arguments from descs[d].
template <int KT, bool MULTI>
__global__ void __launch_bounds__(kLaneThreads) k_score_lanes(const ScoreArgs a, const ScoreArgs *__restrict__ descs,
                                                              const long long *__restrict__ tuple0, int n_desc,
                                                              unsigned total) {
    __shared__ __align__(16) float s_c[kLaneThreads * kLaneStride];
    __shared__ unsigned s_next;
    const int tid = threadIdx.x, lane = tid & 31;
    const int k = a.k, K = KT > 0 ? KT : a.K, kK = k * K;
    constexpr int KM = KT > 0 ? KT : CF_MAX_EDGES;
    const int refill = min(max(a.refill, 1), 32);  // idle lanes before a group refill
    float *cf = s_c + tid * kLaneStride;
    float mu = a.mu;  // the lane's object's mu (edge m is mu (cos, sin) of its angle: a.cs[m], a.sn[m])
    const unsigned per = (total + gridDim.x - 1) / gridDim.x;
    const unsigned u_lo = min(total, blockIdx.x * per), u_hi = min(total, u_lo + per);
    if (tid == 0) s_next = u_lo;
    __syncthreads();

    constexpr int kIdle = 0, kInLp = 1, kDone = 2;
    int state = kIdle;
    unsigned u = 0;  // the lane's tuple within its object
    int od = 0;      // MULTI: the lane's object
    long long od_lo = 0, od_hi = -1;  // MULTI: its global tuple range [tuple0[od], tuple0[od + 1])
    float B[kRows][kRows], xb[kRows], pi[kRows];
    int beta[kRows];
    unsigned basic_x = 0;  // bit c: column c' basic
    unsigned ystat = 0;    // bit r: y_r basic; bit 8 + r: y_r nonbasic at its upper bound
    int j = 0, it = 0, degenerate = 0;
    bool bland = false, lp_start = false, unbounded = false;
    float best_s = 0.f;
    unsigned n_piv = 0, n_lp = 0, n_tup = 0, n_acc = 0, flags = 0;

    for (;;) {
        // ---- idle lanes take tuples together
        const unsigned idle = __ballot_sync(kFull, state == kIdle);
        const unsigned busy = __ballot_sync(kFull, state == kInLp);
        if (idle && (__popc(idle) >= refill || busy == 0)) {
            const int leader = __ffs(idle) - 1;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(&s_next, (unsigned)__popc(idle));
            base = __shfl_sync(kFull, base, leader);
            if (state == kIdle) {
                u = base + (unsigned)__popc(idle & ((1u << lane) - 1u));
                if (u >= u_hi) {
                    state = kDone;
                } else {
                    if (MULTI) {
                        // tuples come in ascending runs: search only when u leaves the lane's object
                        if ((long long)u < od_lo || (long long)u >= od_hi) {
                            int lo = 0, hi = n_desc - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi + 1) >> 1;
                                if (__ldg(tuple0 + mid) <= (long long)u) lo = mid; else hi = mid - 1;
                            }
                            od = lo;
                            od_lo = __ldg(tuple0 + lo);
                            od_hi = __ldg(tuple0 + lo + 1);
                        }
                        u = (unsigned)((long long)u - od_lo);
                    }
                    const LaneObj o = lane_obj(MULTI ? descs[od] : a);
                    if (MULTI) mu = o.mu;
                    const int32_t *tp = o.tuples + (size_t)u * k;
                    bool valid = true;
                    for (int d = 0; d < k; ++d) {
                        const int x = __ldg(tp + d);
                        valid = valid && x >= 0 && x < o.N;
                        if (valid) contact_frame(o, x, cf + kContactFloats * d);
                    }
                    if (!valid) {
                        o.margin[u] = INFINITY;
                        o.accept[u] = 0;
                    } else {
#pragma unroll
                        for (int r = 0; r < kRows; ++r) {
#pragma unroll
                            for (int c = 0; c < kRows; ++c) B[r][c] = r == c ? 1.f : 0.f;
                            xb[r] = 0.f;
                            beta[r] = kK + r;
                        }
                        basic_x = 0;
                        ystat = (1u << kRows) - 1u;
                        j = 0;
                        best_s = 0.f;
                        unbounded = false;
                        lp_start = true;
                        state = kInLp;
                    }
                }
            }
        }
        if (__all_sync(kFull, state == kDone)) break;
        if (state != kInLp) continue;

        const int c0 = j * K, c1 = c0 + K;  // contact j's columns
        if (lp_start) {
            // pi = c_B B^-1, c_B = 1 on the basic columns of contact j: 0 / 1 row weights through exact FMAs
            // (fma(1, b, acc) rounds like acc + b, fma(0, b, acc) = acc)
            float wr[kRows];
#pragma unroll
            for (int r = 0; r < kRows; ++r) wr[r] = (beta[r] >= c0 && beta[r] < c1) ? 1.f : 0.f;
#pragma unroll
            for (int c = 0; c < kRows; ++c) {
                float acc = 0.f;
#pragma unroll
                for (int r = 0; r < kRows; ++r) acc = __fmaf_rn(wr[r], B[r][c], acc);
                pi[c] = acc;
            }
            it = 0;
            degenerate = 0;
            bland = false;
            lp_start = false;
        }
        // ---- pricing.  d is a sum of terms of size up to |pi| |w| (|w| <= 1 + mu), so its rounding
        // error grows with |pi| (= the LP's objective at the optimum): the tolerance scales with it,
        // or rounding noise would keep letting columns that do not improve enter.
        int e = -1;
        float pmax = 0.f;
#pragma unroll
        for (int r = 0; r < kRows; ++r) pmax = fmaxf(pmax, fabsf(pi[r]));
        const float tol = __fmaf_rn(kDTolRel, pmax, kDTol);
        float best = tol, de = 0.f;
        // Dantzig pricing without the basic-column test: a basic column's reduced cost is zero up to
        // rounding, below tol, so it can only win by rounding noise; then, and in Bland mode, the
        // masked scan below redoes the choice
        bool masked = bland;
        if (!bland) {
            for (int i = 0; i < k; ++i) {
                const Frame f = load_frame(cf + kContactFloats * i);
                const float al = (i == j ? 1.f : 0.f) + pi[0] * f.v[0] + pi[1] * f.v[1] + pi[2] * f.v[2] +
                                 pi[3] * f.v[9] + pi[4] * f.v[10] + pi[5] * f.v[11];
                const float be = pi[0] * f.v[3] + pi[1] * f.v[4] + pi[2] * f.v[5] + pi[3] * f.v[12] +
                                 pi[4] * f.v[13] + pi[5] * f.v[14];
                const float ga = pi[0] * f.v[6] + pi[1] * f.v[7] + pi[2] * f.v[8] + pi[3] * f.v[15] +
                                 pi[4] * f.v[16] + pi[5] * f.v[17];
                const float bem = mu * be, gam = mu * ga;
                const int ci = i * K;
#pragma unroll
                for (int m = 0; m < KM; ++m) {
                    if (KT == 0 && m >= K) break;
                    const float d = __fmaf_rn(a.sn[m], gam, __fmaf_rn(a.cs[m], bem, al));
                    if (d > best) {
                        best = d;
                        e = ci + m;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const float sc = ((ystat >> (8 + r)) & 1u) ? pi[r] : -pi[r];
                if (!((ystat >> r) & 1u) && sc > best) {
                    best = sc;
                    e = kK + r;
                }
            }
            if (e >= 0 && e < kK && ((basic_x >> e) & 1u)) {
                masked = true;
                best = tol;
                e = -1;
            } else {
                de = (e >= kK && ((ystat >> (8 + e - kK)) & 1u)) ? -best : best;
            }
        }
        if (masked) for (int i = 0; i < k; ++i) {
            const Frame f = load_frame(cf + kContactFloats * i);
            const float al = (i == j ? 1.f : 0.f) + pi[0] * f.v[0] + pi[1] * f.v[1] + pi[2] * f.v[2] +
                             pi[3] * f.v[9] + pi[4] * f.v[10] + pi[5] * f.v[11];
            const float be = pi[0] * f.v[3] + pi[1] * f.v[4] + pi[2] * f.v[5] + pi[3] * f.v[12] + pi[4] * f.v[13] +
                             pi[5] * f.v[14];
            const float ga = pi[0] * f.v[6] + pi[1] * f.v[7] + pi[2] * f.v[8] + pi[3] * f.v[15] + pi[4] * f.v[16] +
                             pi[5] * f.v[17];
            const unsigned bx = basic_x >> (i * K);
            const float bem = mu * be, gam = mu * ga;
#pragma unroll
            for (int m = 0; m < KM; ++m) {
                if (KT == 0 && m >= K) break;
                const float d = __fmaf_rn(a.sn[m], gam, __fmaf_rn(a.cs[m], bem, al));
                const bool elig = !((bx >> m) & 1u) && d > (bland ? tol : best);
                if (elig && (!bland || e < 0)) {
                    best = bland ? best : d;
                    e = i * K + m;
                    de = d;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            if (!masked) break;
            const bool up = (ystat >> (8 + r)) & 1u;
            const float d = -pi[r];
            const float sc = up ? -d : d;
            const bool elig = !((ystat >> r) & 1u) && sc > (bland ? tol : best);
            if (elig && (!bland || e < 0)) {
                best = bland ? best : sc;
                e = kK + r;
                de = d;
            }
        }
        bool lp_end = e < 0;
        if (!lp_end && it == kMaxPivots) {
            flags |= CF_DEV_LP_PIVOT_CAP;
            lp_end = true;
        }
        if (!lp_end) {
            // ---- entering column u = B^-1 a_e (a = -w_e for c', the unit vector e_r for y_r)
            const bool ey = e >= kK;
            const int re = e - kK;
            float ae[kRows];
            float dl = 1.f;
            if (!ey) {
                const int ie = e / K, me = e - ie * K;
                const Frame f = load_frame(cf + kContactFloats * ie);
                const float cm = a.cs[me] * mu, sm = a.sn[me] * mu;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    ae[q] = -__fmaf_rn(sm, f.v[6 + q], __fmaf_rn(cm, f.v[3 + q], f.v[q]));
                    ae[3 + q] = -__fmaf_rn(sm, f.v[15 + q], __fmaf_rn(cm, f.v[12 + q], f.v[9 + q]));
                }
            } else {
#pragma unroll
                for (int c = 0; c < kRows; ++c) ae[c] = c == re ? 1.f : 0.f;
                dl = ((ystat >> (8 + re)) & 1u) ? -1.f : 1.f;
            }
            float uu[kRows];
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                float acc = 0.f;
#pragma unroll
                for (int c = 0; c < kRows; ++c) acc = __fmaf_rn(B[r][c], ae[c], acc);
                uu[r] = acc;
            }
            // ---- ratio test: the basic variable of row r moves by -dl u_r theta; the entering variable's own
            // box (y: width 2) is candidate kRows, preferred on equal ratios
            int l = ey ? kRows : -1;
            float th = ey ? 2.f : INFINITY, big = 0.f;
            int lbeta = INT_MAX;
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const float al = dl * uu[r];
                const bool bx = beta[r] < kK;
                const float lo = bx ? 0.f : -1.f, hi = bx ? INFINITY : 1.f;
                // rising basic variable (al > 0) meets its lower bound, a falling one its upper bound
                const float aa = fabsf(al);
                const float num = al > 0.f ? xb[r] - lo : hi - xb[r];
                const float t = aa > kPTol ? __fdividef(fmaxf(num, 0.f), aa) : INFINITY;
                bool take;
                if (t < th) take = true;
                else if (t > th || l == kRows || !(t < INFINITY)) take = false;
                else if (bland) take = beta[r] < lbeta;          // lowest basic-variable id
                else take = t == 0.f && aa > big;                 // degenerate: largest pivot entry
                if (take) {
                    th = t;
                    l = r;
                    big = aa;
                    lbeta = beta[r];
                }
            }
            if (l < 0) {  // s_j unbounded: LP_j = 0
                unbounded = true;
                lp_end = true;
            } else {
                degenerate = th == 0.f ? degenerate + 1 : 0;
                if (degenerate >= kDegenerateToBland) bland = true;
                ++it;
                ++n_piv;
                if (l == kRows) {  // bound flip
#pragma unroll
                    for (int r = 0; r < kRows; ++r) xb[r] = __fmaf_rn(-dl * uu[r], th, xb[r]);
                    ystat ^= 1u << (8 + re);
                } else {
                    float ul = 0.f;
                    int leave = 0;
#pragma unroll
                    for (int r = 0; r < kRows; ++r)
                        if (r == l) {
                            ul = uu[r];
                            leave = beta[r];
                        }
                    const float all = dl * ul;
                    const float xe = (!ey ? 0.f : (dl > 0.f ? -1.f : 1.f)) + dl * th;
#pragma unroll
                    for (int r = 0; r < kRows; ++r) {
                        xb[r] = r == l ? xe : __fmaf_rn(-dl * uu[r], th, xb[r]);
                        beta[r] = r == l ? e : beta[r];
                    }
                    if (leave < kK) {
                        basic_x &= ~(1u << leave);
                    } else {
                        ystat &= ~(1u << (leave - kK));
                        if (all < 0.f) ystat |= 1u << (8 + leave - kK);  // it rose to its upper bound
                    }
                    if (!ey) basic_x |= 1u << e;
                    else ystat = (ystat | (1u << re)) & ~(1u << (8 + re));
                    // B^-1: row l / u_l, other rows minus u_r times it; pi += d_e times the new row l
                    const float inv = __fdividef(1.f, ul);
                    // one-hot row weights: row l is read out with exact FMAs (one nonzero term) and
                    // rewritten as 0 * B + 1 * rowl, the other rows as 1 * B - u_r * rowl
                    float oh[kRows], keep[kRows], g[kRows];
#pragma unroll
                    for (int r = 0; r < kRows; ++r) {
                        oh[r] = r == l ? 1.f : 0.f;
                        keep[r] = r == l ? 0.f : 1.f;
                        g[r] = r == l ? -1.f : uu[r];
                    }
                    float rowl[kRows];
#pragma unroll
                    for (int c = 0; c < kRows; ++c) {
                        float v = 0.f;
#pragma unroll
                        for (int r = 0; r < kRows; ++r) v = __fmaf_rn(oh[r], B[r][c], v);
                        rowl[c] = __fmul_rn(v, inv);
                    }
#pragma unroll
                    for (int r = 0; r < kRows; ++r)
#pragma unroll
                        for (int c = 0; c < kRows; ++c)
                            B[r][c] = __fmaf_rn(-g[r], rowl[c], __fmul_rn(keep[r], B[r][c]));
#pragma unroll
                    for (int c = 0; c < kRows; ++c) pi[c] = __fmaf_rn(de, rowl[c], pi[c]);
                }
            }
        }
        if (lp_end) {
            ++n_lp;
            if (!unbounded) {
                float sj = 0.f;
#pragma unroll
                for (int r = 0; r < kRows; ++r) sj = __fmaf_rn((beta[r] >= c0 && beta[r] < c1) ? 1.f : 0.f, xb[r], sj);
                best_s = fmaxf(best_s, sj);
            }
            if (unbounded || best_s >= 1.f / kZeroExit || j + 1 == k) {
                const float margin = unbounded ? 0.f : (best_s > 0.f ? __frcp_rn(best_s) : INFINITY);
                float *mg = MULTI ? descs[od].margin : a.margin;
                uint8_t *ac = MULTI ? descs[od].accept : a.accept;
                const float eps = MULTI ? descs[od].eps : a.eps;
                mg[u] = margin;
                ac[u] = (uint8_t)(margin <= eps);
                n_acc += margin <= eps;
                ++n_tup;
                state = kIdle;
            } else {
                ++j;
                lp_start = true;
            }
        }
    }
    // every lane has left the loop together
    unsigned long long v0 = n_piv, v1 = n_lp, v2 = n_tup;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        v0 += __shfl_xor_sync(kFull, v0, o);
        v1 += __shfl_xor_sync(kFull, v1, o);
        v2 += __shfl_xor_sync(kFull, v2, o);
    }
    const unsigned acc_all = __reduce_add_sync(kFull, n_acc);
    const unsigned fl = __reduce_or_sync(kFull, flags);
    if (lane == 0) {
        atomicAdd(a.counters + 0, v0);
        atomicAdd(a.counters + 1, v1);
        atomicAdd(a.counters + 2, v2);
        if (fl) atomicOr(a.status, fl);
        if (a.n_accept && acc_all) atomicAdd(a.n_accept, (unsigned long long)acc_all);
    }
}

}  // namespace

size_t score_smem_bytes(int F, int W, int T, int k, bool sampling) {
    (void)T;
    (void)k;
    const int G = (W + kGroupWords - 1) / kGroupWords;
    return sampling ? sizeof(uint32_t) * (size_t)F * (G + 1) : 0;  // the group prefixes
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

}  // namespace

namespace {
template <int KT, bool MULTI>
cudaError_t launch_score_lanes_k(const ScoreArgs &a, const ScoreArgs *descs, const long long *tuple0, int n_desc,
                                 long long total, cudaStream_t st) {
    cudaError_t err;
    int sms = 0, per_sm = 0;
    if ((err = launch_shape((const void *)k_score_lanes<KT, MULTI>, kLaneThreads, 0, &per_sm, &sms)) != cudaSuccess)
        return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (a.bpsm > 0) per_sm = std::min(per_sm, a.bpsm);
    const int grid = (int)std::min<long long>((long long)sms * per_sm, (total + kLaneThreads - 1) / kLaneThreads);
    k_score_lanes<KT, MULTI><<<grid, kLaneThreads, 0, st>>>(a, descs, tuple0, n_desc, (unsigned)total);
    return cudaGetLastError();
}

template <bool MULTI>
cudaError_t launch_score_lanes(const ScoreArgs &a, const ScoreArgs *descs, const long long *tuple0, int n_desc,
                               long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    return a.K == 8 ? launch_score_lanes_k<8, MULTI>(a, descs, tuple0, n_desc, total, st)
                    : launch_score_lanes_k<0, MULTI>(a, descs, tuple0, n_desc, total, st);
}
}  // namespace

cudaError_t launch_score(const ScoreArgs &a, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    cudaError_t err;
    if (!a.tuples_given && (err = launch_sample(a, st)) != cudaSuccess) return err;
    return launch_score_lanes<false>(a, nullptr, nullptr, 0, (long long)a.P * a.T, st);
}

cudaError_t launch_optimize(const ScoreArgs &a, int n_outer, int n_inner, float sigma, float zero_tol,
                            float min_gain, int warm_start, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    const OptArgs o{n_outer, n_inner, sigma, zero_tol, min_gain, warm_start};
    const long long total = (long long)a.P * a.T;
    cudaError_t err;
    int dev = 0, sms = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    const long long want = (total + kOptWarps - 1) / kOptWarps;
    const int grid = (int)std::min<long long>((long long)sms * 16, want);
    if (!a.word_box) return cudaErrorInvalidValue;
    k_word_boxes<<<(unsigned)((a.W * 32 + 255) / 256), 256, 0, st>>>(a.px, a.py, a.pz, a.N, a.W, a.word_box);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const bool one = lp_slots(a.k, a.K) == 1;
    const size_t smem1 = (size_t)kOptWarps * 3 * a.k * state_words<1>() * 32 * sizeof(float);
    const size_t smem2 = (size_t)kOptWarps * 3 * a.k * state_words<2>() * 32 * sizeof(float);
    switch (n_inner) {
#define CF_OPT(NI)                                                                                        \
    case NI:                                                                                              \
        if (one) {                                                                                        \
            if ((err = cudaFuncSetAttribute(k_optimize_tuples<NI, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                            (int)smem1)) != cudaSuccess) return err;                      \
            k_optimize_tuples<NI, 1><<<grid, kOptThreads, smem1, st>>>(a, o, (unsigned)total);            \
        } else {                                                                                          \
            if ((err = cudaFuncSetAttribute(k_optimize_tuples<NI, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                            (int)smem2)) != cudaSuccess) return err;                      \
            k_optimize_tuples<NI, 2><<<grid, kOptThreads, smem2, st>>>(a, o, (unsigned)total);            \
        }                                                                                                 \
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
    if (total_tuples >= (1LL << 32)) return cudaErrorInvalidValue;
    return launch_score_lanes<true>(launch, d_descs, d_tuple0, n_desc, total_tuples, st);
}

}  // namespace cf
