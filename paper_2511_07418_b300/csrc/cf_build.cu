// Contact-field build kernels (Def. Contact Field; Sec. 4.3 "Implementation", Alg. 1).
//
// Def. "Contact Field (Point)" / "Contact Field (Hand)": the field of a hand is
// the set of contact vectors FK((p, n); i, q) of its surface points over the
// configuration space; Sec. 4.3 approximates it by randomly sampled q and
// Alg. 1 organises the samples in boxes of a grid cover, each box holding the
// normals that fall in it.  Here the grid cover is a dense per-finger table of
// voxels on one global lattice (cell k = floor(x * inv_h)) and a box's normal
// set is a B-bit word: bit b is set iff some sample in the cell has normal bin
// b (the fixed-direction normal index of Sec. 4.4 "Memory Consumption").
//
// The table is one box of cells over all fingers; a cell's record holds the
// bin sets of all fingers (finger f: bits (f % fpw) * bits .. of word f / fpw).
//
// k_fk_cell_bounds: thread per (finger, joint sample).  The kinematic chain is
// evaluated in FP32 with explicitly rounded operations (joint sin / cos from FP64,
// rounded once); each surface point is then transformed with single-rounding FP32
// FMAs (component order x, y, z).  Two passes: k_fk_cell_bounds evaluates the
// chain, stores the FP32 link frames ([F][J][12][S], coalesced over samples) and
// reduces the per-finger cell AABB (-> table extents); k_fk_bin, a persistent grid
// over (finger, point group, sample chunk) items, reads the frames back and sets
// each sample's bin in its cell word.  Most vectors repeat a code already set, so
// k_fk_bin reads the word first (an L1-cached read) and issues the atomicOr only
// when its bit is missing.  Bins come
// from the same cube-map candidate lists as the query when they are valid.
#include <limits.h>

#include <algorithm>

#include "cf_internal.cuh"

namespace cf {

namespace {

constexpr int kThreads = 256;

// Link frames of finger f for sample s: the chain base * prod_j [Trans(o_j) Rot(a_j, q_j)]
// in FP32 with explicitly rounded operations (no contraction left to the
// compiler), so every build evaluates it bit for bit the same way; the joint's
// sin and cos are CUDA's sincosf (a few ulps: the contact vectors move by ~1e-8 m,
// far inside the 1e-5 m band within which an FP64 evaluation counts a code uncertain).
template <int J>
__device__ __forceinline__ void link_frames(const HandDev &h, int f, const float *__restrict__ q, int S, int s,
                                            float R[J][9], float t[J][3]) {
    const float *b = h.base + 12 * f;
    float Rc[9] = {b[0], b[1], b[2], b[4], b[5], b[6], b[8], b[9], b[10]};
    float tc[3] = {b[3], b[7], b[11]};
#pragma unroll
    for (int j = 0; j < J; ++j) {
        if (j > 0) {
            const float *o = h.offset + 3 * (f * J + j - 1);
            const float o0 = o[0], o1 = o[1], o2 = o[2];
#pragma unroll
            for (int r = 0; r < 3; ++r)
                tc[r] = __fmaf_rn(Rc[3 * r + 2], o2, __fmaf_rn(Rc[3 * r + 1], o1, __fmaf_rn(Rc[3 * r], o0, tc[r])));
        }
        const float *a = h.axis + 3 * (f * J + j);
        const float ax = a[0], ay = a[1], az = a[2];
        float sq, cq;
        sincosf(q[((size_t)f * J + j) * S + s], &sq, &cq);
        const float v = __fsub_rn(1.f, cq);
        // axis-angle rotation (Rodrigues)
        const float xs = __fmul_rn(ax, sq), ys = __fmul_rn(ay, sq), zs = __fmul_rn(az, sq);
        const float xy = __fmul_rn(__fmul_rn(ax, ay), v), xz = __fmul_rn(__fmul_rn(ax, az), v),
                    yz = __fmul_rn(__fmul_rn(ay, az), v);
        const float Q[9] = {__fmaf_rn(__fmul_rn(ax, ax), v, cq), __fsub_rn(xy, zs), __fadd_rn(xz, ys),
                            __fadd_rn(xy, zs), __fmaf_rn(__fmul_rn(ay, ay), v, cq), __fsub_rn(yz, xs),
                            __fsub_rn(xz, ys), __fadd_rn(yz, xs), __fmaf_rn(__fmul_rn(az, az), v, cq)};
        float Rn[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Rn[3 * r + c] = __fmaf_rn(Rc[3 * r + 2], Q[6 + c], __fmaf_rn(Rc[3 * r + 1], Q[3 + c], __fmul_rn(Rc[3 * r], Q[c])));
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            Rc[e] = Rn[e];
            R[j][e] = Rn[e];
        }
        t[j][0] = tc[0];
        t[j][1] = tc[1];
        t[j][2] = tc[2];
    }
}

// Stage finger f's surface points and link ranges in shared memory.
__device__ __forceinline__ void stage_surface(const HandDev &h, int f, float *s_surf, int *s_lb) {
    const float *src = h.surf + (size_t)f * h.M * 8;
    for (int i = threadIdx.x; i < h.M * 8; i += blockDim.x) s_surf[i] = src[i];
    for (int i = threadIdx.x; i <= h.J; i += blockDim.x) s_lb[i] = h.link_begin[f * (h.J + 1) + i];
}

template <int J>
__global__ void __launch_bounds__(kThreads) k_fk_cell_bounds(HandDev h, const float *__restrict__ q, int S,
                                                             float inv_h, float clamp, int *bounds,
                                                             float *__restrict__ links) {
    extern __shared__ float s_surf[];
    __shared__ int s_lb[CF_MAX_JOINTS + 1];
    const int f = blockIdx.y;
    stage_surface(h, f, s_surf, s_lb);
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    int mn0 = INT_MAX, mn1 = INT_MAX, mn2 = INT_MAX, mx0 = INT_MIN, mx1 = INT_MIN, mx2 = INT_MIN;
    if (s < S) {
        float R[J][9], t[J][3];
        link_frames<J>(h, f, q, S, s, R, t);
#pragma unroll
        for (int l = 0; l < J; ++l) {
            float *lk = links + ((size_t)(f * J + l) * 12) * S + s;
#pragma unroll
            for (int e = 0; e < 9; ++e) lk[(size_t)e * S] = R[l][e];
#pragma unroll
            for (int e = 0; e < 3; ++e) lk[(size_t)(9 + e) * S] = t[l][e];
        }
#pragma unroll
        for (int l = 0; l < J; ++l) {
            for (int m = s_lb[l]; m < s_lb[l + 1]; ++m) {
                const float *sp = s_surf + 8 * m;
                const float x = xf_row(R[l][0], R[l][1], R[l][2], t[l][0], sp[0], sp[1], sp[2]);
                const float y = xf_row(R[l][3], R[l][4], R[l][5], t[l][1], sp[0], sp[1], sp[2]);
                const float z = xf_row(R[l][6], R[l][7], R[l][8], t[l][2], sp[0], sp[1], sp[2]);
                const int kx = cell_floor(x, inv_h, clamp), ky = cell_floor(y, inv_h, clamp),
                          kz = cell_floor(z, inv_h, clamp);
                mn0 = min(mn0, kx); mn1 = min(mn1, ky); mn2 = min(mn2, kz);
                mx0 = max(mx0, kx); mx1 = max(mx1, ky); mx2 = max(mx2, kz);
            }
        }
    }
    const unsigned full = 0xffffffffu;
    mn0 = __reduce_min_sync(full, mn0); mn1 = __reduce_min_sync(full, mn1); mn2 = __reduce_min_sync(full, mn2);
    mx0 = __reduce_max_sync(full, mx0); mx1 = __reduce_max_sync(full, mx1); mx2 = __reduce_max_sync(full, mx2);
    if ((threadIdx.x & 31) == 0 && mn0 != INT_MAX) {
        int *bf = bounds + 6 * f;
        atomicMin(bf + 0, mn0); atomicMin(bf + 1, mn1); atomicMin(bf + 2, mn2);
        atomicMax(bf + 3, mx0); atomicMax(bf + 4, mx1); atomicMax(bf + 5, mx2);
    }
}

// Work items of the binning pass: (finger, point group, chunk of kThreads samples), the
// chunk index fastest.  A point group is kGroupPts consecutive surface points of one
// link (a link's points are cut into groups; G = the most groups of any finger), so a
// thread loads one link frame per item.  A persistent grid walks the items with a
// static stride, which spreads them evenly over the SMs whatever the sample count.
constexpr int kGroupPts = 16;

// A plain (weak, L1-cached) read of a table word that other threads are setting bits
// in.  It returns the word as it was at some point of the pass: the table starts at
// zero and bits are only ever set, so a stale read shows a subset of the final bits
// and only costs an update that was not needed; a bit it shows is set for good.
// Inline PTX keeps the compiler from reasoning about the concurrent updates.
__device__ __forceinline__ uint32_t table_peek(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Offset of x's cell from the box origin, as floor(x * inv_h) - lo (the same
// rounding as cell_floor).  The binning pass needs no clamp: the bounds pass saw
// these exact coordinates and the box was accepted only if every cell satisfied
// |k| < 2^20, so no coordinate reached the clamp (|x * inv_h| = 2^21).
__device__ __forceinline__ unsigned bin_cell_offset(float x, float inv_h, unsigned base) {
    return __float_as_uint(__fmaf_rd(x, inv_h, 12582912.0f)) - base;
}

template <int J, bool CAND>
__global__ void __launch_bounds__(kThreads) k_fk_bin(HandDev h, const float *__restrict__ links, int S, FieldGeom g,
                                                     int G, uint32_t *table, unsigned int *status) {
    extern __shared__ float s_surf[];
    __shared__ int s_lb[CF_MAX_JOINTS + 1];
    __shared__ float4 s_dir[CF_MAX_BINS];
    __shared__ uint32_t s_cand[CAND ? kCandCells : 1];
    if (CAND) {
        for (int e = threadIdx.x; e < kCandCells; e += blockDim.x) s_cand[e] = __ldg(g.cand + e);
        if (threadIdx.x < g.B)
            s_dir[threadIdx.x] = make_float4(g.dirs[threadIdx.x][0], g.dirs[threadIdx.x][1], g.dirs[threadIdx.x][2], 0.f);
    }
    const int chunks = (S + kThreads - 1) / kThreads;
    const long long items = (long long)h.F * G * chunks;
    const unsigned base_x = 0x4B400000u + (unsigned)g.lo[0], base_y = 0x4B400000u + (unsigned)g.lo[1],
                   base_z = 0x4B400000u + (unsigned)g.lo[2];
    const unsigned dx = (unsigned)g.dims[0], dy = (unsigned)g.dims[1], dz = (unsigned)g.dims[2];
    constexpr int kBatch = 4;  // points transformed and binned together, then their table updates
    int cur_f = -1;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int chunk = (int)(it % chunks);
        const int fg = (int)(it / chunks);
        const int f = fg / G, grp = fg - f * G;
        if (f != cur_f) {  // block-uniform: stage the finger's surface points
            __syncthreads();
            stage_surface(h, f, s_surf, s_lb);
            __syncthreads();
            cur_f = f;
        }
        int l = -1, mb = 0, me = 0;  // the group's link and point range
        for (int ll = 0, acc = 0; ll < J; ++ll) {
            const int b0 = s_lb[ll], n = s_lb[ll + 1] - b0, ng = (n + kGroupPts - 1) / kGroupPts;
            if (grp >= acc && grp < acc + ng) {
                l = ll;
                mb = b0 + (grp - acc) * kGroupPts;
                me = min(mb + kGroupPts, b0 + n);
            }
            acc += ng;
        }
        const int s = chunk * kThreads + threadIdx.x;
        if (l < 0 || s >= S) continue;
        const int slot = g.slot_of[f][l];  // the finger's slot, or its link's patch slot
        uint32_t *tab = table + slot / g.fpw;
        const int shift = (slot % g.fpw) * g.bits;
        float Rl[9], tl[3];
        {
            const float *lk = links + ((size_t)(f * J + l) * 12) * S + s;
#pragma unroll
            for (int e = 0; e < 9; ++e) Rl[e] = __ldg(lk + (size_t)e * S);
#pragma unroll
            for (int e = 0; e < 3; ++e) tl[e] = __ldg(lk + (size_t)(9 + e) * S);
        }
        for (int m0 = mb; m0 < me; m0 += kBatch) {
            uint32_t *wp[kBatch];
            uint32_t bit[kBatch];
#pragma unroll
            for (int i = 0; i < kBatch; ++i) {
                wp[i] = nullptr;
                bit[i] = 0u;
                if (m0 + i >= me) continue;
                const float *sp = s_surf + 8 * (m0 + i);
                const float x = xf_row(Rl[0], Rl[1], Rl[2], tl[0], sp[0], sp[1], sp[2]);
                const float y = xf_row(Rl[3], Rl[4], Rl[5], tl[1], sp[0], sp[1], sp[2]);
                const float z = xf_row(Rl[6], Rl[7], Rl[8], tl[2], sp[0], sp[1], sp[2]);
                const float nx = rot_row(Rl[0], Rl[1], Rl[2], sp[3], sp[4], sp[5]);
                const float ny = rot_row(Rl[3], Rl[4], Rl[5], sp[3], sp[4], sp[5]);
                const float nz = rot_row(Rl[6], Rl[7], Rl[8], sp[3], sp[4], sp[5]);
                int bin = 0;
                if (CAND) {
                    bin = bin_by_candidates(nx, ny, nz, s_cand, s_dir);
                } else {
                    float best = -INFINITY;
                    for (int b = 0; b < g.B; ++b) {
                        const float sc =
                            __fmaf_rn(g.dirs[b][2], nz, __fmaf_rn(g.dirs[b][1], ny, __fmul_rn(g.dirs[b][0], nx)));
                        if (sc > best) { best = sc; bin = b; }
                    }
                }
                const unsigned ux = bin_cell_offset(x, g.inv_h, base_x);
                const unsigned uy = bin_cell_offset(y, g.inv_h, base_y);
                const unsigned uz = bin_cell_offset(z, g.inv_h, base_z);
                if (ux >= dx || uy >= dy || uz >= dz) {  // cannot happen: extents come from the same arithmetic
                    atomicOr(status, CF_DEV_BIN_RANGE);
                    continue;
                }
                wp[i] = tab + (((size_t)uz * dy + uy) * dx + ux) * g.rw;
                bit[i] = 1u << (shift + bin);
            }
            // most contact vectors repeat a code that is already set (65,536 samples give ~14 vectors per
            // distinct code on a 4-finger hand), so the word is read first and the update skipped when
            // its bit is there
            uint32_t cur[kBatch];
#pragma unroll
            for (int i = 0; i < kBatch; ++i) cur[i] = wp[i] ? table_peek(wp[i]) : 0xffffffffu;
#pragma unroll
            for (int i = 0; i < kBatch; ++i)  // (an empty slot of a batch tail has no word: wp == nullptr)
                if (wp[i] && !(cur[i] & bit[i])) atomicOr(wp[i], bit[i]);  // result unused: a reduction
        }
    }
}

}  // namespace

#define CF_J_DISPATCH(J, CALL)            \
    switch (J) {                          \
        case 1: { constexpr int JJ = 1; CALL; } break; \
        case 2: { constexpr int JJ = 2; CALL; } break; \
        case 3: { constexpr int JJ = 3; CALL; } break; \
        case 4: { constexpr int JJ = 4; CALL; } break; \
        case 5: { constexpr int JJ = 5; CALL; } break; \
        case 6: { constexpr int JJ = 6; CALL; } break; \
        case 7: { constexpr int JJ = 7; CALL; } break; \
        case 8: { constexpr int JJ = 8; CALL; } break; \
        default: return cudaErrorInvalidValue;         \
    }

__global__ void k_popcount(const uint32_t *__restrict__ table, long long words, unsigned long long *count) {
    unsigned long long c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < words; i += (long long)gridDim.x * blockDim.x)
        c += __popc(__ldg(table + i));
    c = __reduce_add_sync(0xffffffffu, (unsigned)c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// Pass 3 (reverse lookup): every contact vector offers s * M + m (original m)
// for its code; the table keeps the smallest.  Open addressing, linear probing.
template <int J>
__global__ void __launch_bounds__(kThreads) k_fk_rep(HandDev h, const float *__restrict__ links, int S, FieldGeom g,
                                                     RepTable t, unsigned int *status) {
    extern __shared__ float s_surf[];
    __shared__ int s_lb[CF_MAX_JOINTS + 1];
    const int f = blockIdx.y;
    stage_surface(h, f, s_surf, s_lb);
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    float R[J][9], tt[J][3];
#pragma unroll
    for (int l = 0; l < J; ++l) {
        const float *lk = links + ((size_t)(f * J + l) * 12) * S + s;
#pragma unroll
        for (int e = 0; e < 9; ++e) R[l][e] = __ldg(lk + (size_t)e * S);
#pragma unroll
        for (int e = 0; e < 3; ++e) tt[l][e] = __ldg(lk + (size_t)(9 + e) * S);
    }
    const unsigned mask = (1u << t.log2_slots) - 1u;
#pragma unroll
    for (int l = 0; l < J; ++l) {
        for (int m = s_lb[l]; m < s_lb[l + 1]; ++m) {
            const float *sp = s_surf + 8 * m;
            const float x = xf_row(R[l][0], R[l][1], R[l][2], tt[l][0], sp[0], sp[1], sp[2]);
            const float y = xf_row(R[l][3], R[l][4], R[l][5], tt[l][1], sp[0], sp[1], sp[2]);
            const float z = xf_row(R[l][6], R[l][7], R[l][8], tt[l][2], sp[0], sp[1], sp[2]);
            const float nx = rot_row(R[l][0], R[l][1], R[l][2], sp[3], sp[4], sp[5]);
            const float ny = rot_row(R[l][3], R[l][4], R[l][5], sp[3], sp[4], sp[5]);
            const float nz = rot_row(R[l][6], R[l][7], R[l][8], sp[3], sp[4], sp[5]);
            int bin = 0;
            float best = -INFINITY;
            for (int b = 0; b < g.B; ++b) {
                const float sc = __fmaf_rn(g.dirs[b][2], nz, __fmaf_rn(g.dirs[b][1], ny, __fmul_rn(g.dirs[b][0], nx)));
                if (sc > best) { best = sc; bin = b; }
            }
            const unsigned ux = (unsigned)(cell_floor(x, g.inv_h, g.clamp) - g.lo[0]);
            const unsigned uy = (unsigned)(cell_floor(y, g.inv_h, g.clamp) - g.lo[1]);
            const unsigned uz = (unsigned)(cell_floor(z, g.inv_h, g.clamp) - g.lo[2]);
            if (ux >= (unsigned)g.dims[0] || uy >= (unsigned)g.dims[1] || uz >= (unsigned)g.dims[2]) continue;
            const unsigned long long word = (((unsigned long long)uz * g.dims[1] + uy) * g.dims[0] + ux) * g.rw + f / g.fpw;
            const unsigned long long key = word * 32ull + (unsigned)((f % g.fpw) * g.bits + bin);
            const uint32_t val = (uint32_t)s * (uint32_t)h.M + (uint32_t)sp[7];
            unsigned hh = rep_hash(key, t.log2_slots);
            bool placed = false;
            for (int probe = 0; probe <= (int)mask; ++probe, hh = (hh + 1) & mask) {
                unsigned long long prev = __ldcg(t.keys + hh);
                if (prev == kRepEmpty) prev = atomicCAS(t.keys + hh, kRepEmpty, key);
                if (prev == kRepEmpty || prev == key) {
                    if (val < __ldcg(t.vals + hh)) atomicMin(t.vals + hh, val);  // most samples repeat a code
                    placed = true;
                    break;
                }
            }
            if (!placed) atomicOr(status, CF_DEV_REP_FULL);
        }
    }
}

cudaError_t launch_fk_cell_bounds(const HandDev &h, const float *q, int S, float inv_h, float clamp, int *bounds,
                                  float *links, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const dim3 grid((S + kThreads - 1) / kThreads, h.F);
    const size_t smem = sizeof(float) * 8 * h.M;
    CF_J_DISPATCH(h.J, (k_fk_cell_bounds<JJ><<<grid, kThreads, smem, st>>>(h, q, S, inv_h, clamp, bounds, links)));
    return cudaGetLastError();
}

template <int J, bool CAND>
static cudaError_t launch_fk_bin_t(const HandDev &h, const float *links, int S, const FieldGeom &g, int G,
                                   uint32_t *table, unsigned int *status, cudaStream_t st) {
    const size_t smem = sizeof(float) * 8 * h.M;
    int sms = 0, per_sm = 0;
    const cudaError_t err = launch_shape((const void *)k_fk_bin<J, CAND>, kThreads, smem, &per_sm, &sms);
    if (err != cudaSuccess) return err;
    const long long items = (long long)h.F * G * ((S + kThreads - 1) / kThreads);
    const int grid = (int)std::min<long long>(items, (long long)std::max(per_sm, 1) * sms);
    k_fk_bin<J, CAND><<<grid, kThreads, smem, st>>>(h, links, S, g, G, table, status);
    return cudaGetLastError();
}

cudaError_t launch_fk_bin(const HandDev &h, const int *h_link_begin, const float *links, int S, const FieldGeom &g,
                          uint32_t *table, unsigned int *status, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    int G = 0;  // the most point groups of any finger
    for (int f = 0; f < h.F; ++f) {
        int n = 0;
        for (int l = 0; l < h.J; ++l) {
            const int c = h_link_begin[f * (h.J + 1) + l + 1] - h_link_begin[f * (h.J + 1) + l];
            n += (c + kGroupPts - 1) / kGroupPts;
        }
        G = std::max(G, n);
    }
    if (G == 0) return cudaSuccess;
    if (g.use_cand && g.B > 8) {
        CF_J_DISPATCH(h.J, return (launch_fk_bin_t<JJ, true>(h, links, S, g, G, table, status, st)));
    } else {
        CF_J_DISPATCH(h.J, return (launch_fk_bin_t<JJ, false>(h, links, S, g, G, table, status, st)));
    }
    return cudaSuccess;
}

cudaError_t launch_popcount(const uint32_t *table, long long words, unsigned long long *count, cudaStream_t st) {
    if (words <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((words + kThreads - 1) / kThreads, 4096);
    k_popcount<<<(unsigned)blocks, kThreads, 0, st>>>(table, words, count);
    return cudaGetLastError();
}

cudaError_t launch_fk_rep(const HandDev &h, const float *links, int S, const FieldGeom &g, RepTable t,
                          unsigned int *status, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const dim3 grid((S + kThreads - 1) / kThreads, h.F);
    const size_t smem = sizeof(float) * 8 * h.M;
    CF_J_DISPATCH(h.J, (k_fk_rep<JJ><<<grid, kThreads, smem, st>>>(h, links, S, g, t, status)));
    return cudaGetLastError();
}

}  // namespace cf
