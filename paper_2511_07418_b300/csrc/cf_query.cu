// Contact-domain query kernel (Def. Contact Surface Representation; Sec. 4.3 "Object Contact Query"; Sec. 5.3).
//
// Def. "Contact Surface Representation": an object contributes the vectors
// (p, -n) of its surface points; Sec. 4.2 defines the contact domain as the
// intersection of the hand's contact field with them, and Sec. 4.3 ("Object
// Contact Query") queries the field with the object's points: position part to
// find the box, normal part to test the box's normal set.  For a palm pose
// (R, t) (object -> palm) the query vector of object point x is
// (R p_x + t, -(R n_x)); it hits finger f iff the finger's table has a word at
// cell(R p_x + t) whose bit bin(-(R n_x)) is set.
//
// Launch: one block per ppb consecutive poses (4, 8 or 16, picked by the
// autotuner); each warp walks the mask words
// of the object (32 points per word, one point per lane, held in registers),
// and for each pose of the block transforms its point, loads the cell's record
// (the bin sets of all fingers, one vector load from the L2-resident table),
// bins the normal where the record is not empty and ballots the hits into the
// F mask words of that (pose, word).  When the block's poses x F fit in a warp,
// lane p * F + f keeps the word of (pose p, finger f) and stores it once per word
// index, adding its popcount to a register count; otherwise lanes 0..F-1 store
// each pose's words.  Counts are summed per (pose, finger) in shared memory.
// With theta-dilated bins (Sec. 4.3 leaf test -x^T n >= theta_hit) the query of
// bin b hits when the cell holds any bin b' with d_b . d_b' >= cos(theta).
//
// Binning: with the candidate table (see cf_bincand.cu) the normal's cube-map
// cell names at most 4 bins, evaluated in ascending order with the same FP32
// dot products and first-maximum rule as a full scan over the B directions,
// so the bin is identical to the full scan's.
#include <limits.h>
#include <string.h>

#include <algorithm>

#include "cf_internal.cuh"

namespace cf {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Offset of x's cell from the box origin lo, as unsigned: floor(x * inv_h) - lo
// (the same rounding as cell_floor) whenever |x * inv_h| < 2^22.  No clamp is
// needed here: beyond that range, and for inf / NaN, the sum lands outside the
// [2^23, 2^24) binade and the offset is >= 2^22 - lo or wraps below zero, so it
// exceeds every box the build admits (|cell| < 2^20) and the range test that
// follows rejects the point.  base = 0x4B400000 + lo.
__device__ __forceinline__ unsigned cell_offset(float x, float inv_h, unsigned base) {
    return __float_as_uint(__fmaf_rd(x, inv_h, 12582912.0f)) - base;
}

template <int RW>
__device__ __forceinline__ void load_record(const uint32_t *__restrict__ r, uint32_t (&rec)[RW]) {
    if (RW == 1) {
        rec[0] = __ldg(r);
    } else if (RW == 2) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(r));
        rec[0] = v.x;
        rec[1 % RW] = v.y;
    } else if (RW % 4 == 0) {
#pragma unroll
        for (int i = 0; i < RW / 4; ++i) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(r) + i);
            rec[(4 * i) % RW] = v.x;
            rec[(4 * i + 1) % RW] = v.y;
            rec[(4 * i + 2) % RW] = v.z;
            rec[(4 * i + 3) % RW] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < RW; ++i) rec[i] = __ldg(r + i);
    }
}

struct QueryArgs {
    FieldGeom g;               // geometry
    QueryDesc one;             // request
    int ppb;                   // poses per block (<= kMaxPosesPerBlock)
};

// Shared memory of one query block: its poses, per-(pose, finger) counts and
// the field's bin directions and dilation sets.
struct QuerySmem {
    __align__(16) float pose[kMaxPosesPerBlock][12];
    unsigned cnt[kMaxPosesPerBlock][CF_MAX_SLOTS];
    float4 dir[CF_MAX_BINS];
    uint32_t dil[CF_MAX_BINS];
};

// Poses i0 .. i0 + np - 1 of request D against field g, by the whole block
// (kThreads threads).  load_geom: stage g's directions, dilation sets and
// candidate table (s_cand, kCandCells words when CAND) before the poses.
// Ends with every thread past the block's last shared-memory read.
template <int F, int BITS, bool CAND>
__device__ __forceinline__ void query_poses(const FieldGeom &g, const QueryDesc &D, int i0, int np, QuerySmem &s,
                                            uint32_t *s_cand, bool load_geom) {
    const cf_points &obj = D.obj;
    const float *__restrict__ poses = D.poses;
    const int W = D.W;
    uint32_t *__restrict__ masks = D.masks;
    uint32_t *__restrict__ counts = D.counts;
    const uint32_t *__restrict__ table = D.table;
    for (int e = threadIdx.x; e < np * 12; e += kThreads) s.pose[e / 12][e % 12] = poses[(size_t)i0 * 12 + e];
    for (int e = threadIdx.x; e < kMaxPosesPerBlock * F; e += kThreads) s.cnt[e / F][e % F] = 0u;
    if (load_geom) {
        if (threadIdx.x < CF_MAX_BINS) s.dil[threadIdx.x] = g.dil[threadIdx.x];
        if (CAND) {
            for (int e = threadIdx.x; e < kCandCells; e += kThreads) s_cand[e] = __ldg(g.cand + e);
            if (threadIdx.x < g.B) s.dir[threadIdx.x] = make_float4(g.dirs[threadIdx.x][0], g.dirs[threadIdx.x][1],
                                                                    g.dirs[threadIdx.x][2], 0.f);
        }
    }
    __syncthreads();
    const bool dilated = g.dilate_deg > 0.f;  // block-uniform

    constexpr int FPW = 32 / BITS;
    constexpr int RW = record_stride((F + FPW - 1) / FPW);  // words per record (the table's stride)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = obj.n;
    const int B = g.B;
    const unsigned base_x = 0x4B400000u + (unsigned)g.lo[0], base_y = 0x4B400000u + (unsigned)g.lo[1],
                   base_z = 0x4B400000u + (unsigned)g.lo[2];
    // with ppb * F <= 32 each lane keeps one (pose, finger) word of the block's poses: one store per
    // word index and counts in registers
    const bool own = np * F <= 32;
    unsigned cnt = 0;
    for (int w = warp; w < W; w += kWarps) {
        uint32_t owned = 0u;
        const int x = 32 * w + lane;
        const bool valid = x < N;
        const float px = valid ? __ldg(obj.px + x) : 0.f, py = valid ? __ldg(obj.py + x) : 0.f,
                    pz = valid ? __ldg(obj.pz + x) : 0.f;
        const float nx = valid ? __ldg(obj.nx + x) : 0.f, ny = valid ? __ldg(obj.ny + x) : 0.f,
                    nz = valid ? __ldg(obj.nz + x) : 0.f;
        for (int pi = 0; pi < np; ++pi) {
            const float4 T0 = reinterpret_cast<const float4 *>(s.pose[pi])[0];
            const float4 T1 = reinterpret_cast<const float4 *>(s.pose[pi])[1];
            const float4 T2 = reinterpret_cast<const float4 *>(s.pose[pi])[2];
            const float qx = xf_row(T0.x, T0.y, T0.z, T0.w, px, py, pz);
            const float qy = xf_row(T1.x, T1.y, T1.z, T1.w, px, py, pz);
            const float qz = xf_row(T2.x, T2.y, T2.z, T2.w, px, py, pz);
            const unsigned ux = cell_offset(qx, g.inv_h, base_x);
            const unsigned uy = cell_offset(qy, g.inv_h, base_y);
            const unsigned uz = cell_offset(qz, g.inv_h, base_z);
            uint32_t rec[RW];
#pragma unroll
            for (int i = 0; i < RW; ++i) rec[i] = 0u;
            if (valid && ux < (unsigned)g.dims[0] && uy < (unsigned)g.dims[1] && uz < (unsigned)g.dims[2])
                load_record<RW>(table + (((size_t)uz * g.dims[1] + uy) * g.dims[0] + ux) * RW, rec);
            uint32_t occ = 0u;
#pragma unroll
            for (int i = 0; i < RW; ++i) occ |= rec[i];
            // an empty record hits no finger whatever the bin, so the normal is binned only where the
            // cell holds a bin (about 3 queries in 5; a warp whose 32 cells are all empty skips the
            // binning, the ballots and the count update)
            uint32_t mine = 0u;
            if (__any_sync(0xffffffffu, occ != 0u)) {
                int bin = 0;
                if (occ != 0u) {
                    // contact-surface normal -(R n): exact negation of the rotated normal
                    const float mx = -rot_row(T0.x, T0.y, T0.z, nx, ny, nz);
                    const float my = -rot_row(T1.x, T1.y, T1.z, nx, ny, nz);
                    const float mz = -rot_row(T2.x, T2.y, T2.z, nx, ny, nz);
                    if (CAND) {
                        bin = bin_by_candidates(mx, my, mz, s_cand, s.dir);
                    } else {
                        float best = -INFINITY;
#pragma unroll 4
                        for (int b = 0; b < B; ++b) {
                            const float sc = __fmaf_rn(g.dirs[b][2], mz,
                                                       __fmaf_rn(g.dirs[b][1], my, __fmul_rn(g.dirs[b][0], mx)));
                            if (sc > best) { best = sc; bin = b; }
                        }
                    }
                }
                const uint32_t dm = dilated ? s.dil[bin] : (1u << bin);  // the bins this query accepts
                const int lf = own ? lane - pi * F : lane;  // the finger whose word this lane keeps
                uint32_t dmf[FPW];  // the accepted bins at each finger's slot of a record word
#pragma unroll
                for (int q = 0; q < FPW; ++q) dmf[q] = dm << (q * BITS);
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    const bool hit = (rec[f / FPW] & dmf[f % FPW]) != 0u;
                    const uint32_t bal = __ballot_sync(0xffffffffu, hit);
                    if (lf == f) mine = bal;
                }
            }
            if (own) {
                owned |= mine;  // nonzero only on lane pi * F + f: this lane's (pose, finger) word
            } else if (lane < F) {
                if (masks) masks[((size_t)(i0 + pi) * F + lane) * W + w] = mine;
                if (mine) atomicAdd(&s.cnt[pi][lane], (unsigned)__popc(mine));
            }
        }
        if (own && lane < np * F) {  // lane = pose * F + finger
            if (masks) masks[((size_t)i0 * F + lane) * W + w] = owned;
            cnt += (unsigned)__popc(owned);
        }
    }
    if (own && lane < np * F && cnt) atomicAdd(&s.cnt[lane / F][lane % F], cnt);
    __syncthreads();
    for (int e = threadIdx.x; e < np * F; e += kThreads) counts[(size_t)(i0 + e / F) * F + e % F] = s.cnt[e / F][e % F];
    __syncthreads();
}

template <int F, int BITS, bool CAND>
__global__ void __launch_bounds__(kThreads, 5) k_query_domains(const QueryArgs a) {
    __shared__ QuerySmem s;
    __shared__ uint32_t s_cand[CAND ? kCandCells : 1];
    const int i0 = (int)blockIdx.x * a.ppb;
    query_poses<F, BITS, CAND>(a.g, a.one, i0, min(a.ppb, a.one.P - i0), s, s_cand, true);
}

// The binning method of a field: a full scan of <= 8 bins costs no more than the candidate lookup.
__host__ __device__ __forceinline__ bool use_candidates(const FieldGeom &g) {
    return g.bits > 8 && g.use_cand && g.B > 8;
}

template <int F, int BITS>
__device__ __forceinline__ void query_poses_any_cand(const FieldGeom &g, const QueryDesc &D, int i0, int np,
                                                     QuerySmem &s, uint32_t *s_cand, bool load_geom) {
    if (BITS > 8 && use_candidates(g)) query_poses<F, BITS, (BITS > 8)>(g, D, i0, np, s, s_cand, load_geom);
    else query_poses<F, BITS, false>(g, D, i0, np, s, s_cand, load_geom);
}

// One launch for every object of a batch, whatever its hand: a persistent grid
// whose blocks take (object, pose-block) items in order from a device work
// counter (work[0]; object d owns items descs[d].block0 .. descs[d + 1].block0 - 1)
// and run the query body specialised for the object's finger count and slot
// width, picked at run time.  A block re-stages the field's directions and
// candidate table only when its object's field changes.  The last block to
// finish returns both counters (work[0], work[1]) to zero for the next launch;
// nothing waits on another block.
__global__ void __launch_bounds__(kThreads, 4) k_query_batch(const QueryDesc *__restrict__ descs,
                                                             const FieldGeom *__restrict__ geoms, int n_desc,
                                                             int total_items, int ppb, unsigned int *work) {
    __shared__ QuerySmem s;
    __shared__ uint32_t s_cand[kCandCells];
    __shared__ FieldGeom s_geom;
    __shared__ QueryDesc s_desc;
    __shared__ int s_item, s_geom_idx;
    if (threadIdx.x == 0) s_geom_idx = -1;
    for (;;) {
        __syncthreads();  // the previous item's shared data is no longer read
        if (threadIdx.x == 0) {
            const int item = (int)atomicAdd(work, 1u);
            s_item = item;
            if (item < total_items) {
                int lo = 0, hi = n_desc - 1;  // last descriptor with block0 <= item
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (descs[mid].block0 <= item) lo = mid; else hi = mid - 1;
                }
                s_desc = descs[lo];
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item >= total_items) break;
        const bool new_geom = s_desc.geom != s_geom_idx;  // block-uniform
        if (new_geom) {
            const int *src = reinterpret_cast<const int *>(geoms + s_desc.geom);
            int *dst = reinterpret_cast<int *>(&s_geom);
            for (int e = threadIdx.x; e < (int)(sizeof(FieldGeom) / sizeof(int)); e += kThreads) dst[e] = src[e];
            __syncthreads();
            if (threadIdx.x == 0) s_geom_idx = s_desc.geom;
        }
        const int i0 = (item - s_desc.block0) * ppb;
        const int np = min(ppb, s_desc.P - i0);
#define CF_QB(FF)                                                                                   \
    case FF:                                                                                        \
        if (s_geom.bits == 8) query_poses_any_cand<FF, 8>(s_geom, s_desc, i0, np, s, s_cand, new_geom);        \
        else if (s_geom.bits == 16) query_poses_any_cand<FF, 16>(s_geom, s_desc, i0, np, s, s_cand, new_geom); \
        else query_poses_any_cand<FF, 32>(s_geom, s_desc, i0, np, s, s_cand, new_geom);                        \
        break;
        switch (s_geom.F) {
            CF_QB(1) CF_QB(2) CF_QB(3) CF_QB(4) CF_QB(5) CF_QB(6) CF_QB(7) CF_QB(8)
            CF_QB(9) CF_QB(10) CF_QB(11) CF_QB(12) CF_QB(13) CF_QB(14) CF_QB(15) CF_QB(16)
            default: break;
        }
#undef CF_QB
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(work + 1, 1u) == gridDim.x - 1) {  // every block has taken its last item
            atomicExch(work, 0u);
            atomicExch(work + 1, 0u);
        }
    }
}

template <int F, int BITS>
cudaError_t launch_fb(const QueryArgs &a, const FieldGeom &g, int grid, cudaStream_t st) {
    if (BITS > 8 && use_candidates(g))
        k_query_domains<F, BITS, (BITS > 8)><<<grid, kThreads, 0, st>>>(a);
    else
        k_query_domains<F, BITS, false><<<grid, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_any(const QueryArgs &a, const FieldGeom &g, int grid, cudaStream_t st) {
#define CF_QF(FF)                                                          \
    case FF:                                                               \
        switch (g.bits) {                                                  \
            case 8: return launch_fb<FF, 8>(a, g, grid, st);              \
            case 16: return launch_fb<FF, 16>(a, g, grid, st);            \
            case 32: return launch_fb<FF, 32>(a, g, grid, st);            \
            default: return cudaErrorInvalidValue;                         \
        }
    switch (g.F) {
        CF_QF(1) CF_QF(2) CF_QF(3) CF_QF(4) CF_QF(5) CF_QF(6) CF_QF(7) CF_QF(8)
        CF_QF(9) CF_QF(10) CF_QF(11) CF_QF(12) CF_QF(13) CF_QF(14) CF_QF(15) CF_QF(16)
        default: return cudaErrorInvalidValue;
    }
#undef CF_QF
}

// Sec. 5.3: merge the domains of one dependency group (a finger's patch slots).
// Block per (pose, finger): each thread ORs the group's slot rows word by word
// (coalesced over words) and the popcounts are summed in the block.
constexpr int kMergeThreads = 256;
__global__ void __launch_bounds__(kMergeThreads) k_merge_domains(const uint32_t *__restrict__ slot_masks, int S, int W,
                                                                 int F, uint32_t slot_set0, uint32_t slot_set1,
                                                                 uint32_t slot_set2, uint32_t slot_set3,
                                                                 uint32_t slot_set4, uint32_t slot_set5,
                                                                 uint32_t slot_set6, uint32_t slot_set7,
                                                                 uint32_t *__restrict__ group_masks,
                                                                 uint32_t *__restrict__ group_counts) {
    __shared__ unsigned s_cnt[kMergeThreads / 32];
    const int i = blockIdx.x / F, f = blockIdx.x - i * F;
    const uint32_t sets[8] = {slot_set0, slot_set1, slot_set2, slot_set3, slot_set4, slot_set5, slot_set6, slot_set7};
    const uint32_t mine = sets[f];  // slots of finger f
    const uint32_t *src = slot_masks + (size_t)i * S * W;
    uint32_t *dst = group_masks + ((size_t)i * F + f) * W;
    unsigned c = 0;
    for (int w = threadIdx.x; w < W; w += kMergeThreads) {
        uint32_t v = 0u;
        for (uint32_t m = mine; m; m &= m - 1) v |= __ldg(src + (size_t)(__ffs(m) - 1) * W + w);
        dst[w] = v;
        c += __popc(v);
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int j = 0; j < kMergeThreads / 32; ++j) t += s_cnt[j];
        group_counts[(size_t)i * F + f] = t;
    }
}

}  // namespace

cudaError_t launch_merge_domains(const FieldGeom &g, int n_fingers, const uint32_t *slot_masks, int P, int W,
                                 uint32_t *group_masks, uint32_t *group_counts, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (n_fingers < 1 || n_fingers > CF_MAX_FINGERS || g.F < 1 || g.F > CF_MAX_SLOTS) return cudaErrorInvalidValue;
    uint32_t sets[CF_MAX_FINGERS] = {};
    for (int s = 0; s < g.F; ++s) sets[(int)g.slot_finger[s]] |= 1u << s;
    const long long blocks = (long long)P * n_fingers;
    if (blocks > INT_MAX) return cudaErrorInvalidValue;
    k_merge_domains<<<(unsigned)blocks, kMergeThreads, 0, st>>>(slot_masks, g.F, W, n_fingers, sets[0], sets[1], sets[2],
                                                              sets[3], sets[4], sets[5], sets[6], sets[7], group_masks,
                                                              group_counts);
    return cudaGetLastError();
}

int query_blocks(int P, int ppb) { return (P + ppb - 1) / ppb; }

cudaError_t launch_query(const FieldGeom &g, const uint32_t *table, const cf_points &obj, const float *poses, int P,
                         uint32_t *masks, uint32_t *counts, int ppb, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (ppb < 1 || ppb > kMaxPosesPerBlock) return cudaErrorInvalidValue;
    QueryArgs a;
    memset(&a, 0, sizeof a);
    a.ppb = ppb;
    a.g = g;
    a.one.obj = obj;
    a.one.poses = poses;
    a.one.P = P;
    a.one.W = (obj.n + 31) / 32;
    a.one.masks = masks;
    a.one.counts = counts;
    a.one.table = table;
    return launch_any(a, g, query_blocks(P, ppb), st);
}

cudaError_t launch_query_batch(const QueryDesc *d_descs, const FieldGeom *d_geoms, int n_desc, int total_items,
                               int ppb, unsigned int *d_work, cudaStream_t st) {
    if (total_items <= 0) return cudaSuccess;
    if (ppb < 1 || ppb > kMaxPosesPerBlock || !d_work) return cudaErrorInvalidValue;
    int per_sm = 0, sms = 0;
    cudaError_t err = launch_shape((const void *)k_query_batch, kThreads, 0, &per_sm, &sms);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::min(total_items, sms * per_sm);
    k_query_batch<<<grid, kThreads, 0, st>>>(d_descs, d_geoms, n_desc, total_items, ppb, d_work);
    return cudaGetLastError();
}

}  // namespace cf
