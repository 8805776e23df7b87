// Tuple sampling + closure margin kernel (rows a4 + a5 of the hot path).
//
// Sec. 4.3: a k-contact grasp takes k contact domains of different fingers
// (independent dependency groups) chosen at random; Alg. 2 starts from
// (p_i, n_i) <- Random(D_i).  Eq. GSWO (Sec. 2.2) scores the contacts: with
// alpha_j = 1 for some j, friction forces inside the cones, minimise the
// resultant force and (weighted) torque; the problem splits into one convex
// subproblem per j.  Linearised here: each cone becomes its inscribed K-edge
// pyramid and the squared norm becomes the max-norm of [force ; torque / rho],
// so every subproblem is the LP
//     LP_j = min t  s.t.  -t <= (sum_im c_im w_im)_r <= t,  sum_m c_jm = 1,  c >= 0
// and the margin is min_j LP_j.
//
// Launch: persistent blocks of 8 warps pull poses from a work counter.  For a
// pose, the block stages the F mask rows in shared memory with per-32-word
// popcount prefixes, one thread per tuple draws its fingers and points
// (Philox4x32-10), then each warp solves the LPs of one tuple at a time.
//
// LP layout (one warp per LP): a dense tableau of 13 constraint rows plus the
// reduced-cost row.  Column c_im (i-major, c < k*K <= 32) lives in slot A of
// lane c; t lives in slot B of lane 0 and slack s_r in slot B of lane r + 1.
// Lane r (< 13) also holds row r's right-hand side and basic variable; lane
// 13 holds the objective's.  Two forced pivots give a feasible start (c_{j,m0}
// with the smallest max-norm wrench enters the equality row, then t enters the
// most violated row); Dantzig pricing follows, switching to Bland's rule after
// a run of degenerate pivots.  FP32 throughout.
#include "cf_internal.cuh"

namespace cf {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxPivots = 64;        // per LP, on top of the two start pivots
constexpr int kDegenerateToBland = 16;
constexpr float kDTol = 1e-6f;        // reduced-cost tolerance
constexpr float kPTol = 1e-6f;        // smallest admissible pivot entry
constexpr float kZeroExit = 1e-7f;    // an LP this close to 0 ends the tuple (min over j)
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void warp_argmin(float &v, int &idx) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ov = __shfl_xor_sync(kFull, v, off);
        const int oi = __shfl_xor_sync(kFull, idx, off);
        if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
}

// Broadcast the entering column e (slot A of lane e for e < 32, slot B of lane
// e - 32 otherwise) to every lane; mycol = its entry in row `lane`.
__device__ __forceinline__ void fetch_column(const float (&A)[14], const float (&B)[14], int e, int lane,
                                             float (&col)[14], float &mycol) {
    const bool slotB = e >= 32;
    const int owner = e & 31;
    mycol = 0.f;
#pragma unroll
    for (int r = 0; r < 14; ++r) {
        const float v = slotB ? B[r] : A[r];
        col[r] = __shfl_sync(kFull, v, owner);
        if (lane == r) mycol = col[r];
    }
}

#define CF_ROWS13(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

// Pivot on (row l, column e) given the broadcast entering column.
__device__ __forceinline__ void pivot(float (&A)[14], float (&B)[14], float &rhs, int &basis, float (&col)[14],
                                      float mycol, int l, int e, int lane) {
    const float pe = __shfl_sync(kFull, mycol, l);
    const float inv = __frcp_rn(pe);
    float pa = 0.f, pb = 0.f;
    switch (l) {
#define CF_GET(r) \
    case r: pa = A[r]; pb = B[r]; col[r] = 0.f; break;
        CF_ROWS13(CF_GET)
#undef CF_GET
        default: break;
    }
    pa = __fmul_rn(pa, inv);
    pb = __fmul_rn(pb, inv);
#pragma unroll
    for (int r = 0; r < 14; ++r) {
        A[r] = __fmaf_rn(-col[r], pa, A[r]);
        B[r] = __fmaf_rn(-col[r], pb, B[r]);
    }
    switch (l) {
#define CF_SET(r) \
    case r: A[r] = pa; B[r] = pb; break;
        CF_ROWS13(CF_SET)
#undef CF_SET
        default: break;
    }
    const float rl = __fmul_rn(__shfl_sync(kFull, rhs, l), inv);
    if (lane == l) {
        rhs = rl;
        basis = e;
    } else if (lane < 14) {
        rhs = __fmaf_rn(-mycol, rl, rhs);
    }
}

// One LP_j on the warp; returns max(t*, 0).  w = this lane's wrench column.
__device__ float solve_lp(const float (&w)[6], bool colA, int ci, int j, int lane, int &npiv, unsigned &flags) {
    float A[14], B[14], col[14], mycol;
    const bool inj = colA && ci == j;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        A[r] = colA ? w[r] : 0.f;
        A[6 + r] = colA ? -w[r] : 0.f;
    }
    A[12] = inj ? 1.f : 0.f;
    A[13] = colA ? 0.f : INFINITY;
#pragma unroll
    for (int r = 0; r < 12; ++r) B[r] = lane == 0 ? -1.f : (lane == r + 1 ? 1.f : 0.f);
    B[12] = 0.f;
    B[13] = lane == 0 ? 1.f : (lane < 13 ? 0.f : INFINITY);
    float rhs = lane == 12 ? 1.f : 0.f;
    int basis = lane < 12 ? 33 + lane : -1;

    // start 1: the edge of contact j with the smallest max-norm wrench enters the equality row
    float mw = INFINITY;
    if (inj) {
        mw = 0.f;
#pragma unroll
        for (int r = 0; r < 6; ++r) mw = fmaxf(mw, fabsf(w[r]));
    }
    int e1 = lane;
    warp_argmin(mw, e1);
    fetch_column(A, B, e1, lane, col, mycol);
    pivot(A, B, rhs, basis, col, mycol, 12, e1, lane);
    // start 2: t enters the most violated row -> every right-hand side >= 0
    float rv = lane < 12 ? rhs : INFINITY;
    int q = lane;
    warp_argmin(rv, q);
    fetch_column(A, B, 32, lane, col, mycol);
    pivot(A, B, rhs, basis, col, mycol, q, 32, lane);
    npiv = 2;

    bool bland = false;
    int degenerate = 0, it = 0;
    for (; it < kMaxPivots; ++it) {
        int e;
        if (bland) {
            const unsigned ba = __ballot_sync(kFull, A[13] < -kDTol);
            const unsigned bb = __ballot_sync(kFull, B[13] < -kDTol);
            e = ba ? __ffs(ba) - 1 : (bb ? 31 + __ffs(bb) : -1);
        } else {
            float dv;
            if (A[13] <= B[13]) { dv = A[13]; e = lane; } else { dv = B[13]; e = 32 + lane; }
            warp_argmin(dv, e);
            if (!(dv < -kDTol)) e = -1;
        }
        if (e < 0) break;
        fetch_column(A, B, e, lane, col, mycol);
        // ratio test over rows 0..12 (lane = row); ties: larger pivot entry (Dantzig) or lower basic index (Bland)
        float ratio = INFINITY, sec = 0.f;
        int l = lane;
        if (lane < 13 && mycol > kPTol) ratio = __fdividef(fmaxf(rhs, 0.f), mycol);
        sec = bland ? (float)basis : -mycol;
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) {
            const float orr = __shfl_xor_sync(kFull, ratio, off);
            const float os = __shfl_xor_sync(kFull, sec, off);
            const int ol = __shfl_xor_sync(kFull, l, off);
            if (orr < ratio || (orr == ratio && (os < sec || (os == sec && ol < l)))) { ratio = orr; sec = os; l = ol; }
        }
        ratio = __shfl_sync(kFull, ratio, 0);
        l = __shfl_sync(kFull, l, 0);
        if (!(ratio < INFINITY)) {
            flags |= CF_DEV_LP_UNBOUNDED;
            break;
        }
        degenerate = ratio == 0.f ? degenerate + 1 : 0;
        if (degenerate >= kDegenerateToBland) bland = true;
        pivot(A, B, rhs, basis, col, mycol, l, e, lane);
        ++npiv;
    }
    if (it == kMaxPivots) flags |= CF_DEV_LP_PIVOT_CAP;
    const float z = -__shfl_sync(kFull, rhs, 13);
    return fmaxf(z, 0.f);
}

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

__global__ void __launch_bounds__(kThreads) k_sample_score(ScoreArgs a) {
    extern __shared__ uint32_t s_dyn[];
    __shared__ float s_cs[CF_MAX_EDGES], s_sn[CF_MAX_EDGES];
    __shared__ uint32_t s_cnt[CF_MAX_FINGERS];
    __shared__ int s_pose, s_next;

    const int F = a.F, W = a.W, T = a.T, k = a.k, K = a.K, kK = k * K;
    const int G = (W + 31) / 32;
    const bool sampling = !a.tuples_given;
    uint32_t *s_mask = s_dyn;                                   // [F][W]
    uint32_t *s_gpre = s_mask + (sampling ? F * W : 0);         // [F][G + 1]
    int *s_tup = (int *)(s_gpre + (sampling ? F * (G + 1) : 0)); // [T][k]

    if (threadIdx.x < CF_MAX_EDGES) {
        s_cs[threadIdx.x] = a.cs[threadIdx.x];
        s_sn[threadIdx.x] = a.sn[threadIdx.x];
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool colA = lane < kK;
    const int ci = colA ? lane / K : 0, cm = colA ? lane % K : 0;
    unsigned long long n_piv = 0, n_lp = 0, n_tup = 0;
    unsigned flags = 0;

    for (;;) {
        if (threadIdx.x == 0) {
            s_pose = (int)atomicAdd(a.work, 1u);
            s_next = 0;
        }
        __syncthreads();
        const int i = s_pose;
        if (i >= a.P) break;

        // ---- stage the pose's domains and draw its tuples -----------------
        if (sampling) {
            if (threadIdx.x < F) s_cnt[threadIdx.x] = a.counts[(size_t)i * F + threadIdx.x];
            const uint32_t *src = a.masks + (size_t)i * F * W;
            for (int e = threadIdx.x; e < F * W; e += kThreads) s_mask[e] = src[e];
            __syncthreads();
            for (int e = threadIdx.x; e < F * G; e += kThreads) {
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
            for (int tau = threadIdx.x; tau < T; tau += kThreads) {
                uint32_t pk = 0;  // non-empty fingers, 4 bits each, ascending
                int m = 0;
                for (int f = 0; f < F; ++f)
                    if (s_cnt[f] > 0) pk |= (uint32_t)f << (4 * m++);
                int32_t *gt = a.tuples + ((size_t)i * T + tau) * k;
                uint8_t *gf = a.fingers ? a.fingers + ((size_t)i * T + tau) * k : nullptr;
                int *st = s_tup + tau * k;
                if (m < k) {
                    for (int d = 0; d < k; ++d) {
                        gt[d] = -1;
                        st[d] = -1;
                        if (gf) gf[d] = 255;
                    }
                    continue;
                }
                const uint2 key = make_uint2(a.seed_lo, a.seed_hi);
                const uint4 u0 = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)tau, 0u, 0u), key);
                const uint4 u1 = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)tau, 1u, 0u), key);
                for (int d = 0; d < k; ++d) {  // partial Fisher-Yates
                    const int jj = d + (int)__umulhi(draw_word(u0, u1, d), (uint32_t)(m - d));
                    const uint32_t fd = (pk >> (4 * d)) & 15u, fj = (pk >> (4 * jj)) & 15u;
                    pk &= ~((15u << (4 * d)) | (15u << (4 * jj)));
                    pk |= (fj << (4 * d)) | (fd << (4 * jj));
                }
                for (int d = 0; d < k; ++d) {
                    const int f = (pk >> (4 * d)) & 15u;
                    const uint32_t r = __umulhi(draw_word(u0, u1, k + d), s_cnt[f]);
                    const int x = select_in_row(s_mask + f * W, s_gpre + f * (G + 1), W, G, r);
                    gt[d] = x;
                    st[d] = x;
                    if (gf) gf[d] = (uint8_t)f;
                }
            }
        } else {
            for (int e = threadIdx.x; e < T * k; e += kThreads) s_tup[e] = a.tuples[(size_t)i * T * k + e];
        }
        __syncthreads();

        // ---- score: one warp per tuple ------------------------------------
        for (;;) {
            int tau = 0;
            if (lane == 0) tau = atomicAdd(&s_next, 1);
            tau = __shfl_sync(kFull, tau, 0);
            if (tau >= T) break;
            const int *st = s_tup + tau * k;
            bool valid = true;
            for (int d = 0; d < k; ++d) valid = valid && st[d] >= 0 && st[d] < a.N;
            float margin = INFINITY;
            if (valid) {
                float wv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (colA) {
                    const int x = st[ci];
                    const float px = __ldg(a.px + x), py = __ldg(a.py + x), pz = __ldg(a.pz + x);
                    const float vx = -__ldg(a.nx + x), vy = -__ldg(a.ny + x), vz = -__ldg(a.nz + x);
                    // tangent basis of nu (Duff et al. 2017)
                    const float sgn = copysignf(1.f, vz);
                    const float aa = -1.f / (sgn + vz);
                    const float bb = vx * vy * aa;
                    const float xx = 1.f + sgn * vx * vx * aa, xy = sgn * bb, xz = -sgn * vx;
                    const float yx = bb, yy = sgn + vy * vy * aa, yz = -vy;
                    const float c = s_cs[cm] * a.mu, s = s_sn[cm] * a.mu;
                    const float ex = vx + c * xx + s * yx, ey = vy + c * xy + s * yy, ez = vz + c * xz + s * yz;
                    const float rx = px - a.cx, ry = py - a.cy, rz = pz - a.cz;
                    wv[0] = ex; wv[1] = ey; wv[2] = ez;
                    wv[3] = (ry * ez - rz * ey) * a.inv_rho;
                    wv[4] = (rz * ex - rx * ez) * a.inv_rho;
                    wv[5] = (rx * ey - ry * ex) * a.inv_rho;
                }
                for (int j = 0; j < k; ++j) {
                    int np = 0;
                    const float tj = solve_lp(wv, colA, ci, j, lane, np, flags);
                    n_piv += np;
                    ++n_lp;
                    margin = fminf(margin, tj);
                    if (margin <= kZeroExit) break;
                }
                ++n_tup;
            }
            if (lane == 0) {
                const size_t u = (size_t)i * T + tau;
                a.margin[u] = margin;
                a.accept[u] = (uint8_t)(margin <= a.eps);
            }
        }
        __syncthreads();
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
    const int G = (W + 31) / 32;
    size_t b = sizeof(int) * (size_t)T * k;
    if (sampling) b += sizeof(uint32_t) * ((size_t)F * W + (size_t)F * (G + 1));
    return b;
}

cudaError_t launch_score(const ScoreArgs &a, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    const size_t smem = score_smem_bytes(a.F, a.W, a.T, a.k, !a.tuples_given);
    cudaError_t err;
    if (smem > 48 * 1024) {
        err = cudaFuncSetAttribute(k_sample_score, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    int dev = 0, sms = 0, per_sm = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sample_score, kThreads, smem)) != cudaSuccess)
        return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = min(a.P, sms * per_sm);
    k_sample_score<<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace cf
