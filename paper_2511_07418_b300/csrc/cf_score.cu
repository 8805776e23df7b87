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
// registers; LP_{j+1} starts from LP_j's basis.
//
// k_optimize_lanes (Alg. 2): one warp per tuple; the candidates' LPs run on the
// same lane simplex, one LP per lane, warm-started from the current tuple's
// optimal bases (Sec. 5.4, "A Free Lunch").  FP32 throughout.
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
constexpr int kRows = 6;

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

// Bounding box of each chunk of 32 mask words (1,024 points) from the word boxes:
// warp per chunk.  Chunk boxes follow the W word boxes.
__global__ void k_chunk_boxes(float *__restrict__ box, int W) {
    const int ch = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    const int n_ch = (W + 31) / 32;
    if (ch >= n_ch) return;
    const int w = 32 * ch + lane;
    const bool ok = w < W;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float lo = ok ? box[6 * (size_t)w + c] : INFINITY, hi = ok ? box[6 * (size_t)w + 3 + c] : -INFINITY;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(kFull, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(kFull, hi, o));
        }
        if (lane == 0) {
            box[6 * ((size_t)W + ch) + c] = lo;
            box[6 * ((size_t)W + ch) + 3 + c] = hi;
        }
    }
}

// ---------------------------------------------------------------------------
// Alg. 2: blockwise zeroth-order contact optimisation
// ---------------------------------------------------------------------------
constexpr int kOptThreads = 128;
constexpr int kOptWarps = kOptThreads / 32;

struct OptArgs {
    int n_outer, n_inner;
    float sigma, zero_tol, min_gain;
    int warm_start;
};

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
// u = B^-1 a_e; the ratio test takes the basic variables' bounds and the
// entering y's own box (a bound flip), with the tie rules above; a pivot
// updates B^-1, the basic values and pi in place.  Lanes run
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

// The contact's 18 numbers (nu, x, y, t_nu, t_x, t_y): nu = -n, its Duff et al. 2017 basis, the torques / rho.
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

// ---- the lane simplex: one LP per lane, state in registers
struct LaneLp {
    float B[kRows][kRows];  // B^-1
    float xb[kRows];        // basic values
    float pi[kRows];        // simplex multipliers c_B B^-1
    int beta[kRows];        // basic variable of each row (c' ids 0..kK-1, y_r id kK + r)
    unsigned basic_x;       // bit c: column c' basic
    unsigned ystat;         // bit r: y_r basic; bit 8 + r: y_r nonbasic at its upper bound
    int it, degenerate;     // pivots of the current LP; run of degenerate pivots
    bool bland;
};

// Contact d's frame (its 18 numbers) of a lane's LP.
struct OwnFrames {  // contiguous, kContactFloats apart
    const float *cf;
    __device__ __forceinline__ const float *operator()(int d) const { return cf + kContactFloats * d; }
};

// The feasible start c' = 0, y = 0: every y_r basic, B = I.
__device__ __forceinline__ void lane_lp_cold(LaneLp &s, int kK) {
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
#pragma unroll
        for (int c = 0; c < kRows; ++c) s.B[r][c] = r == c ? 1.f : 0.f;
        s.xb[r] = 0.f;
        s.beta[r] = kK + r;
    }
    s.basic_x = 0;
    s.ystat = (1u << kRows) - 1u;
}

// Start LP_j (objective: the sum of contact j's columns c0 .. c1 - 1) from the current basis.
__device__ __forceinline__ void lane_lp_begin(LaneLp &s, int c0, int c1) {
    // pi = c_B B^-1, c_B = 1 on the basic columns of contact j: 0 / 1 row weights through exact FMAs
    // (fma(1, b, acc) rounds like acc + b, fma(0, b, acc) = acc)
    float wr[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) wr[r] = (s.beta[r] >= c0 && s.beta[r] < c1) ? 1.f : 0.f;
#pragma unroll
    for (int c = 0; c < kRows; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int r = 0; r < kRows; ++r) acc = __fmaf_rn(wr[r], s.B[r][c], acc);
        s.pi[c] = acc;
    }
    s.it = 0;
    s.degenerate = 0;
    s.bland = false;
}

// Pricing of LP_j: the entering column (-1: optimal) and its reduced cost de.
template <int KT, class Frames>
__device__ __forceinline__ int lane_lp_price(const LaneLp &s, const Frames &fr, int k, int K, int j, float mu,
                                             const ScoreArgs &a, float &de) {
    constexpr int KM = KT > 0 ? KT : CF_MAX_EDGES;
    const int kK = k * K;
    // d is a sum of terms of size up to |pi| |w| (|w| <= 1 + mu), so its rounding error grows with |pi|
    // (= the LP's objective at the optimum): the tolerance scales with it, or rounding noise would keep
    // letting columns that do not improve enter.
    int e = -1;
    float pmax = 0.f;
#pragma unroll
    for (int r = 0; r < kRows; ++r) pmax = fmaxf(pmax, fabsf(s.pi[r]));
    const float tol = __fmaf_rn(kDTolRel, pmax, kDTol);
    float best = tol;
    de = 0.f;
    // Dantzig pricing without the basic-column test: a basic column's reduced cost is zero up to
    // rounding, below tol, so it can only win by rounding noise; then, and in Bland mode, the
    // masked scan below redoes the choice
    bool masked = s.bland;
    if (!s.bland) {
        for (int i = 0; i < k; ++i) {
            const Frame f = load_frame(fr(i));
            const float al = (i == j ? 1.f : 0.f) + s.pi[0] * f.v[0] + s.pi[1] * f.v[1] + s.pi[2] * f.v[2] +
                             s.pi[3] * f.v[9] + s.pi[4] * f.v[10] + s.pi[5] * f.v[11];
            const float be = s.pi[0] * f.v[3] + s.pi[1] * f.v[4] + s.pi[2] * f.v[5] + s.pi[3] * f.v[12] +
                             s.pi[4] * f.v[13] + s.pi[5] * f.v[14];
            const float ga = s.pi[0] * f.v[6] + s.pi[1] * f.v[7] + s.pi[2] * f.v[8] + s.pi[3] * f.v[15] +
                             s.pi[4] * f.v[16] + s.pi[5] * f.v[17];
            const int ci = i * K;
            if constexpr (KT > 0 && KT % 2 == 0) {
                // edges m and m + K/2 lie at angles theta_m and theta_m + pi, so the better of the
                // pair is al + mu |cs_m be + sn_m ga|, its sign naming the edge: K/2 evaluations
                constexpr int KH = KT / 2;
                float tm = -1.f;
                int mm = 0;
#pragma unroll
                for (int m = 0; m < KH; ++m) {
                    const float t = __fmaf_rn(a.sn[m], ga, __fmul_rn(a.cs[m], be));
                    if (fabsf(t) > tm) {
                        tm = fabsf(t);
                        mm = t >= 0.f ? m : m + KH;
                    }
                }
                const float d = __fmaf_rn(mu, tm, al);
                if (d > best) {
                    best = d;
                    e = ci + mm;
                }
            } else {
                const float bem = mu * be, gam = mu * ga;
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
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const float sc = ((s.ystat >> (8 + r)) & 1u) ? s.pi[r] : -s.pi[r];
            if (!((s.ystat >> r) & 1u) && sc > best) {
                best = sc;
                e = kK + r;
            }
        }
        if (e >= 0 && e < kK && ((s.basic_x >> e) & 1u)) {
            masked = true;
            best = tol;
            e = -1;
        } else {
            de = (e >= kK && ((s.ystat >> (8 + e - kK)) & 1u)) ? -best : best;
        }
    }
    if (masked) for (int i = 0; i < k; ++i) {
        const Frame f = load_frame(fr(i));
        const float al = (i == j ? 1.f : 0.f) + s.pi[0] * f.v[0] + s.pi[1] * f.v[1] + s.pi[2] * f.v[2] +
                         s.pi[3] * f.v[9] + s.pi[4] * f.v[10] + s.pi[5] * f.v[11];
        const float be = s.pi[0] * f.v[3] + s.pi[1] * f.v[4] + s.pi[2] * f.v[5] + s.pi[3] * f.v[12] +
                         s.pi[4] * f.v[13] + s.pi[5] * f.v[14];
        const float ga = s.pi[0] * f.v[6] + s.pi[1] * f.v[7] + s.pi[2] * f.v[8] + s.pi[3] * f.v[15] +
                         s.pi[4] * f.v[16] + s.pi[5] * f.v[17];
        const unsigned bx = s.basic_x >> (i * K);
        const float bem = mu * be, gam = mu * ga;
#pragma unroll
        for (int m = 0; m < KM; ++m) {
            if (KT == 0 && m >= K) break;
            const float d = __fmaf_rn(a.sn[m], gam, __fmaf_rn(a.cs[m], bem, al));
            const bool elig = !((bx >> m) & 1u) && d > (s.bland ? tol : best);
            if (elig && (!s.bland || e < 0)) {
                best = s.bland ? best : d;
                e = i * K + m;
                de = d;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        if (!masked) break;
        const bool up = (s.ystat >> (8 + r)) & 1u;
        const float d = -s.pi[r];
        const float sc = up ? -d : d;
        const bool elig = !((s.ystat >> r) & 1u) && sc > (s.bland ? tol : best);
        if (elig && (!s.bland || e < 0)) {
            best = s.bland ? best : sc;
            e = kK + r;
            de = d;
        }
    }
    return e;
}

// One pivot on entering column e (reduced cost de): ratio test, then a bound flip or a basis
// change (B^-1, basic values, pi updated in place).  Returns false when no bound limits the
// entering variable (s_j unbounded); counts the pivot in s.it.
template <int KT, class Frames>
__device__ __forceinline__ bool lane_lp_pivot(LaneLp &s, const Frames &fr, int e, float de, int K, int kK, float mu,
                                              const ScoreArgs &a) {
    // entering column u = B^-1 a_e (a = -w_e for c', the unit vector e_r for y_r)
    const bool ey = e >= kK;
    const int re = e - kK;
    float ae[kRows];
    float dl = 1.f;
    if (!ey) {
        const int ie = e / K, me = e - ie * K;
        const Frame f = load_frame(fr(ie));
        const float cm = a.cs[me] * mu, sm = a.sn[me] * mu;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            ae[q] = -__fmaf_rn(sm, f.v[6 + q], __fmaf_rn(cm, f.v[3 + q], f.v[q]));
            ae[3 + q] = -__fmaf_rn(sm, f.v[15 + q], __fmaf_rn(cm, f.v[12 + q], f.v[9 + q]));
        }
    } else {
#pragma unroll
        for (int c = 0; c < kRows; ++c) ae[c] = c == re ? 1.f : 0.f;
        dl = ((s.ystat >> (8 + re)) & 1u) ? -1.f : 1.f;
    }
    float uu[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < kRows; ++c) acc = __fmaf_rn(s.B[r][c], ae[c], acc);
        uu[r] = acc;
    }
    // ratio test: the basic variable of row r moves by -dl u_r theta; the entering variable's own
    // box (y: width 2) is candidate kRows, preferred on equal ratios
    int l = ey ? kRows : -1;
    float th = ey ? 2.f : INFINITY, big = 0.f;
    int lbeta = INT_MAX;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const float al = dl * uu[r];
        const bool bx = s.beta[r] < kK;
        const float lo = bx ? 0.f : -1.f, hi = bx ? INFINITY : 1.f;
        // rising basic variable (al > 0) meets its lower bound, a falling one its upper bound
        const float aa = fabsf(al);
        const float num = al > 0.f ? s.xb[r] - lo : hi - s.xb[r];
        const float t = aa > kPTol ? __fdividef(fmaxf(num, 0.f), aa) : INFINITY;
        bool take;
        if (t < th) take = true;
        else if (t > th || l == kRows || !(t < INFINITY)) take = false;
        else if (s.bland) take = s.beta[r] < lbeta;     // lowest basic-variable id
        else take = t == 0.f && aa > big;                // degenerate: largest pivot entry
        if (take) {
            th = t;
            l = r;
            big = aa;
            lbeta = s.beta[r];
        }
    }
    if (l < 0) return false;
    s.degenerate = th == 0.f ? s.degenerate + 1 : 0;
    if (s.degenerate >= kDegenerateToBland) s.bland = true;
    ++s.it;
    if (l == kRows) {  // bound flip
#pragma unroll
        for (int r = 0; r < kRows; ++r) s.xb[r] = __fmaf_rn(-dl * uu[r], th, s.xb[r]);
        s.ystat ^= 1u << (8 + re);
        return true;
    }
    float ul = 0.f;
    int leave = 0;
#pragma unroll
    for (int r = 0; r < kRows; ++r)
        if (r == l) {
            ul = uu[r];
            leave = s.beta[r];
        }
    const float all = dl * ul;
    const float xe = (!ey ? 0.f : (dl > 0.f ? -1.f : 1.f)) + dl * th;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        s.xb[r] = r == l ? xe : __fmaf_rn(-dl * uu[r], th, s.xb[r]);
        s.beta[r] = r == l ? e : s.beta[r];
    }
    if (leave < kK) {
        s.basic_x &= ~(1u << leave);
    } else {
        s.ystat &= ~(1u << (leave - kK));
        if (all < 0.f) s.ystat |= 1u << (8 + leave - kK);  // it rose to its upper bound
    }
    if (!ey) s.basic_x |= 1u << e;
    else s.ystat = (s.ystat | (1u << re)) & ~(1u << (8 + re));
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
        for (int r = 0; r < kRows; ++r) v = __fmaf_rn(oh[r], s.B[r][c], v);
        rowl[c] = __fmul_rn(v, inv);
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int c = 0; c < kRows; ++c) s.B[r][c] = __fmaf_rn(-g[r], rowl[c], __fmul_rn(keep[r], s.B[r][c]));
#pragma unroll
    for (int c = 0; c < kRows; ++c) s.pi[c] = __fmaf_rn(de, rowl[c], s.pi[c]);
    return true;
}

// s_j at the optimum: the sum of contact j's basic values (nonbasic c' sit at 0), as 0 / 1-weighted FMAs.
__device__ __forceinline__ float lane_lp_value(const LaneLp &s, int c0, int c1) {
    float sj = 0.f;
#pragma unroll
    for (int r = 0; r < kRows; ++r) sj = __fmaf_rn((s.beta[r] >= c0 && s.beta[r] < c1) ? 1.f : 0.f, s.xb[r], sj);
    return sj;
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
    LaneLp s;
    s.basic_x = 0u;
    s.ystat = 0u;
    const OwnFrames fr{cf};
    int j = 0;
    bool lp_start = false, unbounded = false;
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
                        lane_lp_cold(s, kK);
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
            lane_lp_begin(s, c0, c1);
            lp_start = false;
        }
        float de = 0.f;
        const int e = lane_lp_price<KT>(s, fr, k, K, j, mu, a, de);
        bool lp_end = e < 0;
        if (!lp_end && s.it == kMaxPivots) {
            flags |= CF_DEV_LP_PIVOT_CAP;
            lp_end = true;
        }
        if (!lp_end && !lane_lp_pivot<KT>(s, fr, e, de, K, kK, mu, a)) {  // s_j unbounded: LP_j = 0
            unbounded = true;
            lp_end = true;
        }
        if (lp_end) {
            ++n_lp;
            n_piv += (unsigned)s.it;
            if (!unbounded) best_s = fmaxf(best_s, lane_lp_value(s, c0, c1));
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

// Projection of Alg. 2: for each of the NI candidate points cand[c] (c < NI, x y z), the
// domain point nearest to it (mask bit set in row `row`), lowest index on ties; lane c
// returns candidate c's (-1 when the domain is empty).  Exact pruning: the current
// point x0 (p) lies in the domain, so candidate q_c's nearest domain point lies within
// r_c = |q_c - p| of q_c.  Chunks of 32 mask words, then the words of the chunks that
// remain (lane, lane + 32, ...), keep only the candidates whose r_c-ball reaches their
// point box, and a word left with none is skipped (radii with slack for rounding; no
// pruning when x0's bit is not set, e.g. for given tuples outside the domain).  A test of
// the word box against p alone was dropped: the balls already exclude every word it did.  The warp then takes each surviving word together, lane b
// on the word's point b, for the candidates the word can serve: point loads are
// coalesced and the candidate test is uniform across the warp.
template <int NI>
__device__ __forceinline__ int project_candidates(const ScoreArgs &a, const float *cand, const uint32_t *row, int x0,
                                                  float px, float py, float pz, int lane) {
    const int W = a.W;
    // candidates in registers up to 8 of them; more would cost the kernel a block per SM
    constexpr bool kCandRegs = NI <= 8;
    float bd[NI];
    int bi[NI];
    float cq[kCandRegs ? NI : 1][3];
#pragma unroll
    for (int c = 0; c < NI; ++c) {
        bd[c] = INFINITY;
        bi[c] = INT_MAX;
        if (kCandRegs) {
            cq[kCandRegs ? c : 0][0] = cand[3 * c];
            cq[kCandRegs ? c : 0][1] = cand[3 * c + 1];
            cq[kCandRegs ? c : 0][2] = cand[3 * c + 2];
        }
    }
    float rc = 0.f;
    if (lane < NI) {
        const float dx = cand[3 * lane] - px, dy = cand[3 * lane + 1] - py, dz = cand[3 * lane + 2] - pz;
        rc = sqrtf(dx * dx + dy * dy + dz * dz);
    }
    // each candidate's pruning radius r_c (squared, with slack)
    const float rs = rc * 1.0001f + 1e-6f;
    float r2c[NI];
#pragma unroll
    for (int c = 0; c < NI; ++c) r2c[c] = __shfl_sync(kFull, rs * rs, c);
    rc = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(rc)));  // rc >= 0: bits order
    const bool in_dom = (__ldg(row + (x0 >> 5)) >> (x0 & 31)) & 1u;
    // R bounds every candidate's nearest domain point from p (|q_c - p| + r_c <= 2 max r_c); finite
    // only when p lies in the domain, R2 gates the pruning below (kept in this form: the same test on a
    // bool costs the kernel a spill in its word loop)
    const float R = 2.f * rc * 1.0001f + 1e-6f;
    const float R2 = in_dom ? R * R : INFINITY;
    constexpr unsigned kAll = NI >= 32 ? 0xffffffffu : (1u << NI) - 1u;
    // chunks of 32 words (1,024 points) first: a chunk whose box no candidate's ball reaches is skipped
    const int n_ch = (W + 31) / 32;
    const float *chunk_box = a.word_box + 6 * (size_t)W;
    for (int c0 = 0; c0 < n_ch; c0 += 32) {
        // the candidates whose ball reaches this lane's chunk (a word's box lies inside its chunk's)
        unsigned ccm = c0 + lane < n_ch ? kAll : 0u;
        if (ccm && R2 < INFINITY) {
            const float *bx = chunk_box + 6 * (size_t)(c0 + lane);
            const float lx = __ldg(bx), ly = __ldg(bx + 1), lz = __ldg(bx + 2);
            const float hx = __ldg(bx + 3), hy = __ldg(bx + 4), hz = __ldg(bx + 5);
            ccm = 0u;
#pragma unroll
            for (int c = 0; c < NI; ++c) {
                const float *qc = kCandRegs ? cq[kCandRegs ? c : 0] : cand + 3 * c;
                const float fx = fmaxf(fmaxf(lx - qc[0], qc[0] - hx), 0.f);
                const float fy = fmaxf(fmaxf(ly - qc[1], qc[1] - hy), 0.f);
                const float fz = fmaxf(fmaxf(lz - qc[2], qc[2] - hz), 0.f);
                if (fx * fx + fy * fy + fz * fz <= r2c[c]) ccm |= 1u << c;
            }
        }
        for (unsigned chm = __ballot_sync(kFull, ccm != 0u); chm; chm &= chm - 1) {
            const int cb = __ffs(chm) - 1;
            const unsigned chunk_cm = __shfl_sync(kFull, ccm, cb);  // uniform across the warp
            const int w0 = 32 * (c0 + cb);
            const int w = w0 + lane;
            uint32_t bits = w < W ? __ldg(row + w) : 0u;
            unsigned cmask = chunk_cm;  // the candidates this word can serve
            if (bits && R2 < INFINITY) {
                const float *bx = a.word_box + 6 * (size_t)w;
                const float lx = __ldg(bx), ly = __ldg(bx + 1), lz = __ldg(bx + 2);
                const float hx = __ldg(bx + 3), hy = __ldg(bx + 4), hz = __ldg(bx + 5);
                {
                    cmask = 0u;
#pragma unroll
                    for (int c = 0; c < NI; ++c) {
                        if (!((chunk_cm >> c) & 1u)) continue;  // its ball misses the whole chunk
                        const float *qc = kCandRegs ? cq[kCandRegs ? c : 0] : cand + 3 * c;
                        const float r2 = r2c[c];
                        const float fx = fmaxf(fmaxf(lx - qc[0], qc[0] - hx), 0.f);
                        const float fy = fmaxf(fmaxf(ly - qc[1], qc[1] - hy), 0.f);
                        const float fz = fmaxf(fmaxf(lz - qc[2], qc[2] - hz), 0.f);
                        if (fx * fx + fy * fy + fz * fz <= r2) cmask |= 1u << c;
                    }
                    if (!cmask) bits = 0u;
                }
            }
            // each lane visits its points in ascending index order, as the (distance, index) reduction assumes
            for (unsigned need = __ballot_sync(kFull, bits != 0u); need; need &= need - 1) {
                const int b = __ffs(need) - 1;
                const uint32_t wb = __shfl_sync(kFull, bits, b);
                const unsigned wc = __shfl_sync(kFull, cmask, b);
                const int x = 32 * (w0 + b) + lane;
                if ((wb >> lane) & 1u) {
                    const float qx = __ldg(a.px + x), qy = __ldg(a.py + x), qz = __ldg(a.pz + x);
#pragma unroll
                    for (int c = 0; c < NI; ++c) {
                        if (!((wc >> c) & 1u)) continue;
                        const float *qc = kCandRegs ? cq[kCandRegs ? c : 0] : cand + 3 * c;
                        const float dx = __fsub_rn(qx, qc[0]), dy = __fsub_rn(qy, qc[1]), dz = __fsub_rn(qz, qc[2]);
                        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                        if (d2 < bd[c]) {
                            bd[c] = d2;
                            bi[c] = x;
                        }
                    }
                }
            }
        }
    }
    int mine = -1;
#pragma unroll
    for (int c = 0; c < NI; ++c) {
        const unsigned kd = fkey(bd[c]);
        const unsigned kmin = __reduce_min_sync(kFull, kd);
        const unsigned imin = __reduce_min_sync(kFull, kd == kmin ? (unsigned)bi[c] : 0xffffffffu);
        if (lane == c) mine = imin == 0xffffffffu ? -1 : (int)imin;
    }
    return mine;
}

// ---------------------------------------------------------------------------
// Alg. 2 on the lane simplex
// ---------------------------------------------------------------------------
// An LP_j's optimal basis as kept between solves: B^-1 (36 words), the basic values (6), the
// basic ids (6) and the status words basic_x, ystat.
constexpr int kBasisWords = 50;

// Warm start with repair (Sec. 5.4, "A Free Lunch"): s is an optimal basis of the
// current tuple's LP_j; the trial moves contact i to the frame fi.  Each basic
// column of contact i is swapped for its own new version by a column-replacement
// pivot on its row (B^-1 updated with u = B^-1 a_new), so the basis keeps its
// variables; the basic values are then recomputed from the nonbasic bounds
// (c' = 0, y = -1 or +1); with no basic column of contact i the basis and its
// values stand as they are.  False when a replacement pivot is below 1e-4 (a near
// singular basis) or the recomputed basis is infeasible beyond 1e-6.
__device__ __forceinline__ bool lane_lp_repair(LaneLp &s, const float *fi, int i, int K, int kK, float mu,
                                               const ScoreArgs &a) {
    const int c0 = i * K, c1 = c0 + K;
    unsigned rows = 0u;  // the rows whose basic variable is a column of contact i
#pragma unroll
    for (int r = 0; r < kRows; ++r)
        if (s.beta[r] >= c0 && s.beta[r] < c1) rows |= 1u << r;
    if (!rows) return true;  // B and the basic values stay as they are
    const Frame f = load_frame(fi);
    while (rows) {  // in ascending row order
        const int l = __ffs(rows) - 1;
        rows &= rows - 1;
        int me = 0;
#pragma unroll
        for (int r = 0; r < kRows; ++r)
            if (r == l) me = s.beta[r] - c0;
        const float cm = a.cs[me] * mu, sm = a.sn[me] * mu;
        float ae[kRows];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            ae[q] = -__fmaf_rn(sm, f.v[6 + q], __fmaf_rn(cm, f.v[3 + q], f.v[q]));
            ae[3 + q] = -__fmaf_rn(sm, f.v[15 + q], __fmaf_rn(cm, f.v[12 + q], f.v[9 + q]));
        }
        float uu[kRows], ul = 0.f;
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < kRows; ++c) acc = __fmaf_rn(s.B[r][c], ae[c], acc);
            uu[r] = acc;
            if (r == l) ul = acc;
        }
        if (!(fabsf(ul) > 1e-4f)) return false;
        const float inv = __frcp_rn(ul);
        // row l / u_l, the other rows minus u_r times it, with one-hot row weights (exact FMAs)
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
            for (int r = 0; r < kRows; ++r) v = __fmaf_rn(oh[r], s.B[r][c], v);
            rowl[c] = __fmul_rn(v, inv);
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r)
#pragma unroll
            for (int c = 0; c < kRows; ++c) s.B[r][c] = __fmaf_rn(-g[r], rowl[c], __fmul_rn(keep[r], s.B[r][c]));
    }
    // B x_B = -N x_N: x_B = -sum over the nonbasic y_r of x_r B^-1 e_r
    float wn[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
        wn[r] = ((s.ystat >> r) & 1u) ? 0.f : (((s.ystat >> (8 + r)) & 1u) ? -1.f : 1.f);
    bool feas = true;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        float x = 0.f;
#pragma unroll
        for (int c = 0; c < kRows; ++c) x = __fmaf_rn(wn[c], s.B[r][c], x);
        if (s.beta[r] < kK) {
            feas = feas && x >= -1e-6f;
            x = fmaxf(x, 0.f);
        } else {
            feas = feas && x >= -1.f - 1e-6f && x <= 1.f + 1e-6f;
            x = fminf(fmaxf(x, -1.f), 1.f);
        }
        s.xb[r] = x;
    }
    return feas;
}

// The closure margin of a tuple from its s_j (v[0..k-1]), taken in order j = 0 .. k - 1
// as k_score_lanes takes them: the first unbounded s_j gives 0, and a running
// maximum past 1 / kZeroExit ends the scan.
__device__ __forceinline__ float margin_from(const float *v, int k) {
    float bs = 0.f;
    for (int q = 0; q < k; ++q) {
        if (!(v[q] < INFINITY)) return 0.f;
        bs = fmaxf(bs, v[q]);
        if (bs >= 1.f / kZeroExit) break;
    }
    return bs > 0.f ? __fdiv_rn(1.f, bs) : INFINITY;
}

// ---------------------------------------------------------------------------
// Alg. 2 in phases: every tuple of the launch advances one step at a time
// ---------------------------------------------------------------------------
// Sec. 5.4, Alg. 2, with every tuple of the launch in lockstep.  First each
// tuple's own k LPs (from c' = 0; their optimal bases are kept) give its margin.
// Then each step (outer iteration it, contact i) is a projection kernel (a warp
// per tuple: n_in Gaussian mutations of p_i in its tangent plane, each projected
// onto finger f_i's domain), an LP-job kernel (a lane per LP_j of a candidate,
// warm-started from the tuple's optimal LP_j basis repaired for the moved
// contact -- "A Free Lunch" -- or from c' = 0; jobs handed out across the whole
// grid) and a selection kernel (a thread per tuple: the candidates, in order,
// replace the best so far when their margin is lower by more than the relative
// min_gain; margins <= zero_tol count as 0 and end the tuple).  With the warm
// start a fourth kernel replays the winners' LPs from the same starts, which
// gives back their optimal bases without storing every candidate's.  Each
// tuple's result depends only on the tuple.

// Per-tuple state between the phases (global memory).
struct OptPhaseState {
    float *J;        // [n] the tuple's margin (+inf: invalid tuple)
    uint8_t *live;   // [n] 1 while the tuple is optimised (valid, margin above zero_tol)
    float *base;     // word w of LP_j's optimal basis of tuple u at base[w * n * k + u * k + j]
    int *cand;       // [n][NI] the step's candidate points, by rank
    int *n_todo;     // [n] the step's candidates
    float *sres;     // [n][NI * k] s_j of job g * k + j (the tuple's own LPs: j)
    int *win;        // [n] the step's winning rank, -1 when none
    unsigned *jobs;    // the step's candidate LP jobs, u * 64 + g * 4 + j each, by tuple, then g, then j
    unsigned *n_jobs;  // their count
    unsigned *chunk;   // [n / kJobChunk + 1] jobs per chunk of kJobChunk tuples, then the chunks' offsets
};

// Idle lanes before a group refill in the LP jobs.  Alg. 2's LPs are short (3.7 pivots with the
// warm start, 7.1 cold, against 13 in the scorer) and a warm start loads and repairs a basis, so
// starts are taken in larger groups than the scorer's: at hand20, 12 gave 355 ms (8: 364, 16: 355,
// 24: 376) with the warm start and 358 ms cold (8: 358, 16: 365).
constexpr int kOptRefill = 12;
constexpr int kJobInit = 0;  // LP_j of the tuple itself, from c' = 0; its basis is kept
constexpr int kJobCand = 1;  // LP_j of candidate g, warm-started (counted in the device counters)
constexpr int kJobWin = 2;   // LP_j of the step's winner, replayed to keep its basis (not counted)

__device__ __forceinline__ void basis_store_g(float *base, size_t stride, size_t at, const LaneLp &s) {
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
#pragma unroll
        for (int c = 0; c < kRows; ++c) base[(size_t)(r * kRows + c) * stride + at] = s.B[r][c];
        base[(size_t)(36 + r) * stride + at] = s.xb[r];
        base[(size_t)(42 + r) * stride + at] = __int_as_float(s.beta[r]);
    }
    base[(size_t)48 * stride + at] = __uint_as_float(s.basic_x);
    base[(size_t)49 * stride + at] = __uint_as_float(s.ystat);
}

__device__ __forceinline__ void basis_load_g(LaneLp &s, const float *base, size_t stride, size_t at) {
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
#pragma unroll
        for (int c = 0; c < kRows; ++c) s.B[r][c] = base[(size_t)(r * kRows + c) * stride + at];
        s.xb[r] = base[(size_t)(36 + r) * stride + at];
        s.beta[r] = __float_as_int(base[(size_t)(42 + r) * stride + at]);
    }
    s.basic_x = __float_as_uint(base[(size_t)48 * stride + at]);
    s.ystat = __float_as_uint(base[(size_t)49 * stride + at]);
}

// LP jobs of one phase.  Candidates and the winners' replays: the job list written after the
// projection or the selection (descriptor u * 64 + g * 4 + j: tuple u, candidate g, LP j; its
// length is read on the device).  A tuple's own LPs: slots u * k + j in tuple order (the jobs
// write the bases, whose stores then stay sequential), a slot whose tuple is not live ending at
// once.  Lanes take jobs together, when `refill` of them wait or none is busy, from the
// block's contiguous share.  The contact frames live in the lane's stretch of shared memory.
template <int KT, int MODE>
__global__ void __launch_bounds__(kLaneThreads) k_opt_lp_jobs(const ScoreArgs a, const OptPhaseState ps, int NI,
                                                              int i_moved, int warm, unsigned n_slots) {
    __shared__ __align__(16) float s_c[kLaneThreads * kLaneStride];
    __shared__ unsigned s_next;
    const int tid = threadIdx.x, lane = tid & 31;
    const int k = a.k, K = KT > 0 ? KT : a.K, kK = k * K;
    const int SPT = NI * k;  // result slots per tuple
    const unsigned n_jobs = MODE != kJobInit ? *ps.n_jobs : n_slots;
    const size_t nk = (size_t)a.P * a.T * k;                     // the bases' word stride
    constexpr int refill = kOptRefill;
    const float mu = a.mu;
    const LaneObj ob = lane_obj(a);
    float *cf = s_c + tid * kLaneStride;
    const unsigned per = (n_jobs + gridDim.x - 1) / gridDim.x;
    const unsigned q_lo = min(n_jobs, blockIdx.x * per), q_hi = min(n_jobs, q_lo + per);
    if (tid == 0) s_next = q_lo;
    __syncthreads();
    constexpr int kIdle = 0, kInLp = 1, kDone = 2;
    int state = kIdle;
    LaneLp s;
    lane_lp_cold(s, kK);
    const OwnFrames fr{cf};
    unsigned u = 0;
    int j = 0, g = 0;
    unsigned long long n_piv = 0, n_lp = 0, n_warm = 0;
    unsigned flags = 0;
    for (;;) {
        const unsigned idle = __ballot_sync(kFull, state == kIdle);
        const unsigned busy = __ballot_sync(kFull, state == kInLp);
        if (idle && (__popc(idle) >= refill || busy == 0)) {
            const int leader = __ffs(idle) - 1;
            unsigned base_q = 0;
            if (lane == leader) base_q = atomicAdd(&s_next, (unsigned)__popc(idle));
            base_q = __shfl_sync(kFull, base_q, leader);
            if (state == kIdle) {
                const unsigned q = base_q + (unsigned)__popc(idle & ((1u << lane) - 1u));
                if (q >= q_hi) {
                    state = kDone;
                } else {
                    bool run = true;
                    if (MODE != kJobInit) {  // a listed job: every one runs
                        const unsigned dsc = ps.jobs[q];
                        u = dsc >> 6;
                        g = (int)((dsc >> 2) & 15u);
                        j = (int)(dsc & 3u);
                    } else {
                        u = q / (unsigned)k;
                        j = (int)(q - u * (unsigned)k);
                        g = 0;
                        run = ps.live[u] != 0;
                    }
                    if (run) {
                        for (int d = 0; d < k; ++d) {
                            int x = __ldg(a.tuples + (size_t)u * k + d);
                            if (MODE == kJobCand && d == i_moved) x = ps.cand[(size_t)u * NI + g];
                            contact_frame(ob, x, cf + kContactFloats * d);
                        }
                        bool ws = false;
                        if (MODE != kJobInit && warm) {
                            basis_load_g(s, ps.base, nk, (size_t)u * k + j);
                            ws = lane_lp_repair(s, cf + kContactFloats * i_moved, i_moved, K, kK, mu, a);
                        }
                        if (!ws) lane_lp_cold(s, kK);
                        if (MODE == kJobCand) n_warm += ws;
                        lane_lp_begin(s, j * K, j * K + K);
                        state = kInLp;
                    }
                }
            }
        }
        if (__all_sync(kFull, state == kDone)) break;
        if (state != kInLp) continue;
        float de = 0.f;
        const int e = lane_lp_price<KT>(s, fr, k, K, j, mu, a, de);
        bool end = e < 0, unb = false;
        if (!end && s.it == kMaxPivots) {
            flags |= CF_DEV_LP_PIVOT_CAP;
            end = true;
        }
        if (!end && !lane_lp_pivot<KT>(s, fr, e, de, K, kK, mu, a)) {
            unb = true;
            end = true;
        }
        if (end) {
            if (MODE != kJobWin) {
                ps.sres[(size_t)u * SPT + g * k + j] = unb ? INFINITY : lane_lp_value(s, j * K, j * K + K);
                ++n_lp;
                n_piv += (unsigned)s.it;
            }
            if (MODE != kJobCand && ps.base) basis_store_g(ps.base, nk, (size_t)u * k + j, s);
            state = kIdle;
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        n_piv += __shfl_xor_sync(kFull, n_piv, off);
        n_lp += __shfl_xor_sync(kFull, n_lp, off);
        n_warm += __shfl_xor_sync(kFull, n_warm, off);
    }
    flags = __reduce_or_sync(kFull, flags);
    if (lane == 0) {
        if (n_piv) atomicAdd(a.counters + 0, n_piv);
        if (n_lp) atomicAdd(a.counters + 1, n_lp);
        if (n_warm) atomicAdd(a.counters + 3, n_warm);
        if (flags) atomicOr(a.status, flags);
    }
}

// A thread per tuple: validity (points in range, fingers below F), the starting margin
// +inf, and the count of valid tuples.
__global__ void k_opt_begin(const ScoreArgs a, const OptPhaseState ps, unsigned n) {
    const unsigned u = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = false;
    if (u < n) {
        valid = true;
        for (int d = 0; d < a.k; ++d) {
            const int x = __ldg(a.tuples + (size_t)u * a.k + d);
            const int f = (int)__ldg(a.fingers + (size_t)u * a.k + d);
            valid = valid && x >= 0 && x < a.N && f < a.F;
        }
        ps.live[u] = valid ? 1 : 0;
        ps.J[u] = INFINITY;
        ps.win[u] = -1;
    }
    const unsigned c = __reduce_add_sync(kFull, valid ? 1u : 0u);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(a.counters + 2, (unsigned long long)c);
}

// A warp per live tuple: the NI mutations of contact i at outer iteration it (Box-Muller on
// Philox4x32-10 words at counter (pose, tau, (it k + i) ceil(n_in / 2) + c / 2, 0xA162), key seed),
// their projections onto finger f_i's
// domain, and the distinct candidates other than the current point, by rank.  Bounded to 7
// blocks per SM (72 registers): latency-bound scans gain more from warps than they lose to
// a few spilled words.
template <int NI>
__global__ void __launch_bounds__(kOptThreads, 7) k_opt_project(const ScoreArgs a, const OptArgs o, const OptPhaseState ps,
                                                             int it, int i, unsigned n) {
    __shared__ float s_xyz[kOptWarps][NI][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = a.k, F = a.F, W = a.W;
    const uint2 key = make_uint2(a.seed_lo, a.seed_hi);
    const int blocks_per_draw = (NI + 1) / 2;
    for (unsigned u = blockIdx.x * kOptWarps + warp; u < n; u += gridDim.x * kOptWarps) {
        if (!ps.live[u]) {
            if (lane == 0) ps.n_todo[u] = 0;
            continue;
        }
        const int pose = (int)(u / (unsigned)a.T), tau = (int)(u % (unsigned)a.T);
        const int x0 = __ldg(a.tuples + (size_t)u * k + i), fi = (int)__ldg(a.fingers + (size_t)u * k + i);
        // tangent basis of nu = -n at the current point (Duff et al. 2017) and the mutated points in
        // explicitly rounded FP32 operations
        const float px = __ldg(a.px + x0), py = __ldg(a.py + x0), pz = __ldg(a.pz + x0);
        const float vx = -__ldg(a.nx + x0), vy = -__ldg(a.ny + x0), vz = -__ldg(a.nz + x0);
        const float sgn = copysignf(1.f, vz);
        const float aa = __fdiv_rn(-1.f, __fadd_rn(sgn, vz));
        const float bb = __fmul_rn(__fmul_rn(vx, vy), aa);
        const float xx = __fadd_rn(1.f, __fmul_rn(__fmul_rn(__fmul_rn(sgn, vx), vx), aa));
        const float xy = __fmul_rn(sgn, bb), xz = -__fmul_rn(sgn, vx);
        const float yx = bb, yy = __fadd_rn(sgn, __fmul_rn(__fmul_rn(vy, vy), aa)), yz = -vy;
        if (lane < NI) {  // candidate `lane`: one Box-Muller pair in FP32 (u1, u2 exact; a few ulps)
            const uint32_t pid = (uint32_t)pose + a.pose_base;
            const uint4 w4 = philox4x32_10(
                make_uint4(pid, (uint32_t)tau, (uint32_t)((it * k + i) * blocks_per_draw + lane / 2), 0xA162u), key);
            const uint32_t w0 = (lane & 1) ? w4.z : w4.x, w1 = (lane & 1) ? w4.w : w4.y;
            const float u1 = (float)((w0 >> 8) + 1u) * 5.9604644775390625e-8f;  // (0, 1]
            const float u2 = (float)(w1 >> 8) * 5.9604644775390625e-8f;         // [0, 1)
            const float r = sqrtf(-2.f * logf(u1));
            float sd, cd;
            sincospif(2.f * u2, &sd, &cd);
            const float g1 = __fmul_rn(r, cd), g2 = __fmul_rn(r, sd);
            const float sg = o.sigma;
            s_xyz[warp][lane][0] = __fadd_rn(px, __fmul_rn(sg, __fadd_rn(__fmul_rn(g1, xx), __fmul_rn(g2, yx))));
            s_xyz[warp][lane][1] = __fadd_rn(py, __fmul_rn(sg, __fadd_rn(__fmul_rn(g1, xy), __fmul_rn(g2, yy))));
            s_xyz[warp][lane][2] = __fadd_rn(pz, __fmul_rn(sg, __fadd_rn(__fmul_rn(g1, xz), __fmul_rn(g2, yz))));
        }
        __syncwarp();
        const int cand_mine = project_candidates<NI>(a, &s_xyz[warp][0][0], a.masks + ((size_t)pose * F + fi) * W, x0,
                                                     px, py, pz, lane);
        // candidates equal to the current point or to an earlier candidate cannot win
        const unsigned same = __match_any_sync(kFull, lane < NI ? cand_mine : -2 - lane);
        const bool skip = lane >= NI || cand_mine < 0 || cand_mine == x0 || (same & ((1u << lane) - 1u)) != 0u;
        const unsigned todo = __ballot_sync(kFull, !skip);
        if (!skip) ps.cand[(size_t)u * NI + __popc(todo & ((1u << lane) - 1u))] = cand_mine;
        if (lane == 0) ps.n_todo[u] = __popc(todo);
        __syncwarp();
    }
}

// The step's candidate LP jobs, and then its winners' replays, as one list in tuple order, so that
// the lanes of a block read neighbouring tuples' bases (word-major rows: neighbouring tuples share
// sectors) and no lane takes a slot without work: the jobs per chunk of kJobChunk tuples, an
// exclusive scan of those counts (one block; it also writes the total), then every chunk writes its
// tuples' jobs from its offset.
constexpr int kJobChunk = 4096;
constexpr int kJobThreads = 256;

// Jobs of tuple u over k: the step's candidates (kJobCand), or 1 when its winner's LPs replay (kJobWin).
template <int MODE>
__device__ __forceinline__ unsigned listed_per_tuple(const OptPhaseState &ps, unsigned u) {
    return MODE == kJobCand ? (unsigned)ps.n_todo[u] : (ps.live[u] != 0 && ps.win[u] >= 0 ? 1u : 0u);
}

template <int MODE>
__global__ void __launch_bounds__(kJobThreads) k_job_counts(const OptPhaseState ps, unsigned n, int k) {
    __shared__ unsigned s_w[kJobThreads / 32];
    const unsigned c0 = blockIdx.x * kJobChunk, c1 = min(n, c0 + kJobChunk);
    unsigned c = 0;
    for (unsigned u = c0 + threadIdx.x; u < c1; u += kJobThreads) c += listed_per_tuple<MODE>(ps, u);
    c = __reduce_add_sync(kFull, c);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < kJobThreads / 32; ++w) t += s_w[w];
        ps.chunk[blockIdx.x] = t * (unsigned)k;
    }
}

__global__ void __launch_bounds__(1024) k_job_scan(const OptPhaseState ps, int nb) {
    block_exclusive_scan_1024(ps.chunk, nb, ps.n_jobs);
}

constexpr int kJobStage = 8192;  // jobs of one tile staged in shared memory for coalesced writes

template <int MODE>
__global__ void __launch_bounds__(kJobThreads) k_job_write(const OptPhaseState ps, unsigned n, int k) {
    __shared__ unsigned s_w[kJobThreads / 32];
    __shared__ unsigned s_jobs[kJobStage];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned c0 = blockIdx.x * kJobChunk, c1 = min(n, c0 + kJobChunk);
    unsigned run = ps.chunk[blockIdx.x];
    for (unsigned t0 = c0; t0 < c1; t0 += kJobThreads) {
        const unsigned u = t0 + threadIdx.x;
        const unsigned cnt = u < c1 ? listed_per_tuple<MODE>(ps, u) * (unsigned)k : 0u;
        unsigned incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += y;
        }
        __syncthreads();  // the previous tile's sums have been read
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        unsigned before = 0, tile = 0;
        for (int w = 0; w < kJobThreads / 32; ++w) {
            before += w < warp ? s_w[w] : 0u;
            tile += s_w[w];
        }
        const unsigned at = before + incl - cnt;  // within the tile
        if (tile <= (unsigned)kJobStage) {  // block-uniform: staged, then written out coalesced
            for (unsigned t = 0; t < cnt; ++t) s_jobs[at + t] = u * 64u + (t / (unsigned)k) * 4u + t % (unsigned)k;
            __syncthreads();
            for (unsigned q = threadIdx.x; q < tile; q += kJobThreads) ps.jobs[run + q] = s_jobs[q];
        } else {
            for (unsigned t = 0; t < cnt; ++t)
                ps.jobs[run + at + t] = u * 64u + (t / (unsigned)k) * 4u + t % (unsigned)k;
        }
        run += tile;
    }
}

// A thread per tuple.  init: the margin of the tuple's own LPs.  Otherwise the step's
// candidates, in order, replace the best so far when their margin is lower by more than
// the relative min_gain (margins <= zero_tol count as 0); the winner's point becomes
// contact i.  A tuple whose margin reaches zero_tol stops.
__global__ void k_opt_select(const ScoreArgs a, const OptArgs o, const OptPhaseState ps, int NI, int i, int init,
                             unsigned n) {
    const unsigned u = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = a.k;
    int win = -1;
    bool live = false;
    if (u < n && ps.live[u]) {
        const float *sr = ps.sres + (size_t)u * NI * k;
        float J = ps.J[u];
        if (init) {
            J = margin_from(sr, k);
        } else {
            const int n_todo = ps.n_todo[u];
            float best = J <= o.zero_tol ? 0.f : J;
            for (int g = 0; g < n_todo; ++g) {
                const float Jt = margin_from(sr + g * k, k);
                const float Jtc = Jt <= o.zero_tol ? 0.f : Jt;
                if (Jtc < (1.f - o.min_gain) * best) {
                    best = Jtc;
                    J = Jt;
                    win = g;
                }
            }
            if (win >= 0) a.tuples[(size_t)u * k + i] = ps.cand[(size_t)u * NI + win];
            ps.win[u] = win;
        }
        ps.J[u] = J;
        live = (J <= o.zero_tol ? 0.f : J) > 0.f;
        if (!live) ps.live[u] = 0;
    }
}

// A thread per tuple: the final margin and accept flag.
__global__ void k_opt_finish(const ScoreArgs a, const OptPhaseState ps, unsigned n) {
    const unsigned u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const float J = ps.J[u];
    a.margin[u] = J;
    a.accept[u] = (uint8_t)(J <= a.eps);
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

namespace {
size_t align256z(size_t x) { return (x + 255) & ~(size_t)255; }

// The phase state's arrays inside one scratch block (see optimize_state_bytes).
OptPhaseState phase_state(void *scratch, size_t n, int NI, int k, bool warm) {
    char *p = (char *)scratch;
    OptPhaseState ps;
    ps.J = (float *)p; p += align256z(sizeof(float) * n);
    ps.live = (uint8_t *)p; p += align256z(n);
    ps.win = (int *)p; p += align256z(sizeof(int) * n);
    ps.n_todo = (int *)p; p += align256z(sizeof(int) * n);
    ps.cand = (int *)p; p += align256z(sizeof(int) * n * NI);
    ps.sres = (float *)p; p += align256z(sizeof(float) * n * NI * k);
    ps.n_jobs = (unsigned *)p; p += 256;
    ps.chunk = (unsigned *)p; p += align256z(sizeof(unsigned) * (n / kJobChunk + 1));
    ps.jobs = (unsigned *)p; p += align256z(sizeof(unsigned) * n * NI * k);
    ps.base = warm ? (float *)p : nullptr;
    return ps;
}

// The LP jobs of the list the previous kernel wrote (its length is read on the device): a
// grid of as many blocks as fit at once, each taking a contiguous share.
template <int KT, int MODE>
cudaError_t launch_lp_jobs(const ScoreArgs &a, const OptPhaseState &ps, int NI, int i, int warm, unsigned n_slots,
                           cudaStream_t st) {
    int sms = 0, per_sm = 0;
    cudaError_t e = launch_shape((const void *)k_opt_lp_jobs<KT, MODE>, kLaneThreads, 0, &per_sm, &sms);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (a.bpsm > 0) per_sm = std::min(per_sm, a.bpsm);
    k_opt_lp_jobs<KT, MODE><<<sms * per_sm, kLaneThreads, 0, st>>>(a, ps, NI, i, warm, n_slots);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t lp_jobs(const ScoreArgs &a, const OptPhaseState &ps, int NI, int i, int warm, unsigned n_slots,
                    cudaStream_t st) {
    return a.K == 8 ? launch_lp_jobs<8, MODE>(a, ps, NI, i, warm, n_slots, st)
                    : launch_lp_jobs<0, MODE>(a, ps, NI, i, warm, n_slots, st);
}

template <int NI>
cudaError_t launch_project(const ScoreArgs &a, const OptArgs &o, const OptPhaseState &ps, int it, int i, unsigned n,
                           cudaStream_t st) {
    int sms = 0, per_sm = 0;
    cudaError_t e = launch_shape((const void *)k_opt_project<NI>, kOptThreads, 0, &per_sm, &sms);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = (int)std::min<long long>((long long)sms * per_sm, ((long long)n + kOptWarps - 1) / kOptWarps);
    k_opt_project<NI><<<grid, kOptThreads, 0, st>>>(a, o, ps, it, i, n);
    return cudaGetLastError();
}
}  // namespace

size_t optimize_state_bytes(long long n, int n_inner, int k, int warm) {
    const size_t N = (size_t)std::max<long long>(n, 1);
    return align256z(sizeof(float) * N) + align256z(N) + 2 * align256z(sizeof(int) * N) +
           align256z(sizeof(int) * N * n_inner) + align256z(sizeof(float) * N * n_inner * k) + 256 +
           align256z(sizeof(unsigned) * (N / kJobChunk + 1)) + align256z(sizeof(unsigned) * N * n_inner * k) + (warm ? sizeof(float) * (size_t)kBasisWords * N * k : 0);
}

cudaError_t launch_optimize(const ScoreArgs &a, int n_outer, int n_inner, float sigma, float zero_tol,
                            float min_gain, int warm_start, void *state, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    const long long total = (long long)a.P * a.T;
    if (!a.word_box || !state) return cudaErrorInvalidValue;
    if (total * n_inner * a.k >= (1LL << 32) || total >= (1LL << 26)) return cudaErrorInvalidValue;  // job descriptors
    if (n_inner != 4 && n_inner != 8 && n_inner != 16) return cudaErrorInvalidValue;
    const OptArgs o{n_outer, n_inner, sigma, zero_tol, min_gain, warm_start};
    const unsigned n = (unsigned)total;
    const int NI = n_inner, k = a.k;
    const OptPhaseState ps = phase_state(state, n, NI, k, warm_start != 0);
    cudaError_t err;
    k_word_boxes<<<(unsigned)((a.W * 32 + 255) / 256), 256, 0, st>>>(a.px, a.py, a.pz, a.N, a.W, a.word_box);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    k_chunk_boxes<<<(unsigned)(((a.W + 31) / 32 * 32 + 255) / 256), 256, 0, st>>>(a.word_box, a.W);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const unsigned tb = (n + 255) / 256;
    const unsigned nk = n * (unsigned)k;  // slots of the tuples' own LPs
    const unsigned nb = (n + kJobChunk - 1) / kJobChunk;  // chunks of the job lists
    k_opt_begin<<<tb, 256, 0, st>>>(a, ps, n);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // the tuples' own LPs, from c' = 0; their optimal bases seed the candidates
    if ((err = lp_jobs<kJobInit>(a, ps, NI, 0, warm_start, nk, st)) != cudaSuccess) return err;
    k_opt_select<<<tb, 256, 0, st>>>(a, o, ps, NI, 0, 1, n);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    for (int it = 0; it < n_outer; ++it) {
        for (int i = 0; i < k; ++i) {
            err = NI == 4 ? launch_project<4>(a, o, ps, it, i, n, st)
                          : (NI == 8 ? launch_project<8>(a, o, ps, it, i, n, st) : launch_project<16>(a, o, ps, it, i, n, st));
            if (err != cudaSuccess) return err;
            k_job_counts<kJobCand><<<nb, kJobThreads, 0, st>>>(ps, n, k);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            k_job_scan<<<1, 1024, 0, st>>>(ps, (int)nb);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            k_job_write<kJobCand><<<nb, kJobThreads, 0, st>>>(ps, n, k);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            if ((err = lp_jobs<kJobCand>(a, ps, NI, i, warm_start, 0, st)) != cudaSuccess) return err;
            k_opt_select<<<tb, 256, 0, st>>>(a, o, ps, NI, i, 0, n);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            // the winners' LPs again from the same starts: their optimal bases become the tuples'
            if (warm_start) {  // listed like the candidates': only the tuples with a winner replay
                k_job_counts<kJobWin><<<nb, kJobThreads, 0, st>>>(ps, n, k);
                if ((err = cudaGetLastError()) != cudaSuccess) return err;
                k_job_scan<<<1, 1024, 0, st>>>(ps, (int)nb);
                if ((err = cudaGetLastError()) != cudaSuccess) return err;
                k_job_write<kJobWin><<<nb, kJobThreads, 0, st>>>(ps, n, k);
                if ((err = cudaGetLastError()) != cudaSuccess) return err;
                if ((err = lp_jobs<kJobWin>(a, ps, NI, i, 1, 0, st)) != cudaSuccess) return err;
            }
        }
    }
    k_opt_finish<<<tb, 256, 0, st>>>(a, ps, n);
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
