// Contact-domain query kernel (row a3 of the hot path).
//
// Def. "Contact Surface Representation": an object contributes the vectors
// (p, -n) of its surface points; Sec. 3.2 defines the contact domain as the
// intersection of the hand's contact field with them, and Sec. 3.3 ("Object
// Contact Query") queries the field with the object's points: position part to
// find the box, normal part to test the box's normal set.  For a palm pose
// (R, t) (object -> palm) the query vector of object point x is
// (R p_x + t, -(R n_x)); it hits finger f iff the finger's table has a word at
// cell(R p_x + t) whose bit bin(-(R n_x)) is set.
//
// Launch: one block per QP consecutive poses; each warp walks the mask words
// of the object (32 points per word, one point per lane, held in registers),
// and for each pose of the block transforms its point, bins the normal, looks
// the cell up in every finger's table (L1/L2-resident, read-only path) and
// ballots the hits into the F mask words of that (pose, word).  Counts are
// accumulated per (pose, finger) in shared memory.
#include "cf_internal.cuh"

namespace cf {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPosesPerBlock = 8;

template <int F, int BT>
__global__ void __launch_bounds__(kThreads) k_query_domains(FieldGeom g, const uint32_t *__restrict__ table,
                                                            cf_points obj, const float *__restrict__ poses, int P,
                                                            int W, uint32_t *__restrict__ masks,
                                                            uint32_t *__restrict__ counts) {
    __shared__ float s_pose[kPosesPerBlock][12];
    __shared__ unsigned s_cnt[kPosesPerBlock][F];
    const int i0 = blockIdx.x * kPosesPerBlock;
    const int np = min(kPosesPerBlock, P - i0);
    for (int e = threadIdx.x; e < np * 12; e += kThreads) s_pose[e / 12][e % 12] = poses[(size_t)i0 * 12 + e];
    for (int e = threadIdx.x; e < kPosesPerBlock * F; e += kThreads) s_cnt[e / F][e % F] = 0u;
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = obj.n;
    const int B = BT > 0 ? BT : g.B;
    for (int w = warp; w < W; w += kWarps) {
        const int x = 32 * w + lane;
        const bool valid = x < N;
        const float px = valid ? __ldg(obj.px + x) : 0.f, py = valid ? __ldg(obj.py + x) : 0.f,
                    pz = valid ? __ldg(obj.pz + x) : 0.f;
        const float nx = valid ? __ldg(obj.nx + x) : 0.f, ny = valid ? __ldg(obj.ny + x) : 0.f,
                    nz = valid ? __ldg(obj.nz + x) : 0.f;
        for (int pi = 0; pi < np; ++pi) {
            const float *T = s_pose[pi];
            const float qx = xf_row(T[0], T[1], T[2], T[3], px, py, pz);
            const float qy = xf_row(T[4], T[5], T[6], T[7], px, py, pz);
            const float qz = xf_row(T[8], T[9], T[10], T[11], px, py, pz);
            // contact-surface normal -(R n): exact negation of the rotated normal
            const float mx = -rot_row(T[0], T[1], T[2], nx, ny, nz);
            const float my = -rot_row(T[4], T[5], T[6], nx, ny, nz);
            const float mz = -rot_row(T[8], T[9], T[10], nx, ny, nz);
            int bin = 0;
            float best = -INFINITY;
#pragma unroll(BT > 0 ? BT : 4)
            for (int b = 0; b < B; ++b) {
                const float sc =
                    __fmaf_rn(g.dirs[b][2], mz, __fmaf_rn(g.dirs[b][1], my, __fmul_rn(g.dirs[b][0], mx)));
                if (sc > best) { best = sc; bin = b; }
            }
            const int kx = cell_floor(qx, g.inv_h, g.clamp);
            const int ky = cell_floor(qy, g.inv_h, g.clamp);
            const int kz = cell_floor(qz, g.inv_h, g.clamp);
            uint32_t mine = 0u;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const unsigned ux = (unsigned)(kx - g.lo[f][0]);
                const unsigned uy = (unsigned)(ky - g.lo[f][1]);
                const unsigned uz = (unsigned)(kz - g.lo[f][2]);
                bool hit = false;
                if (valid && ux < (unsigned)g.dims[f][0] && uy < (unsigned)g.dims[f][1] &&
                    uz < (unsigned)g.dims[f][2]) {
                    const uint32_t word =
                        __ldg(table + g.off[f] + ((size_t)uz * g.dims[f][1] + uy) * g.dims[f][0] + ux);
                    hit = (word >> bin) & 1u;
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, hit);
                if (lane == f) mine = bal;
            }
            if (lane < F) {
                if (masks) masks[((size_t)(i0 + pi) * F + lane) * W + w] = mine;
                atomicAdd(&s_cnt[pi][lane], (unsigned)__popc(mine));
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < np * F; e += kThreads) counts[(size_t)(i0 + e / F) * F + e % F] = s_cnt[e / F][e % F];
}

template <int F>
cudaError_t launch_f(const FieldGeom &g, const uint32_t *table, const cf_points &obj, const float *poses, int P,
                     uint32_t *masks, uint32_t *counts, cudaStream_t st) {
    const int W = (obj.n + 31) / 32;
    const int grid = (P + kPosesPerBlock - 1) / kPosesPerBlock;
    switch (g.B) {
        case 8: k_query_domains<F, 8><<<grid, kThreads, 0, st>>>(g, table, obj, poses, P, W, masks, counts); break;
        case 16: k_query_domains<F, 16><<<grid, kThreads, 0, st>>>(g, table, obj, poses, P, W, masks, counts); break;
        case 32: k_query_domains<F, 32><<<grid, kThreads, 0, st>>>(g, table, obj, poses, P, W, masks, counts); break;
        default: k_query_domains<F, 0><<<grid, kThreads, 0, st>>>(g, table, obj, poses, P, W, masks, counts); break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_query(const FieldGeom &g, const uint32_t *table, const cf_points &obj, const float *poses, int P,
                         uint32_t *masks, uint32_t *counts, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    switch (g.F) {
        case 1: return launch_f<1>(g, table, obj, poses, P, masks, counts, st);
        case 2: return launch_f<2>(g, table, obj, poses, P, masks, counts, st);
        case 3: return launch_f<3>(g, table, obj, poses, P, masks, counts, st);
        case 4: return launch_f<4>(g, table, obj, poses, P, masks, counts, st);
        case 5: return launch_f<5>(g, table, obj, poses, P, masks, counts, st);
        case 6: return launch_f<6>(g, table, obj, poses, P, masks, counts, st);
        case 7: return launch_f<7>(g, table, obj, poses, P, masks, counts, st);
        case 8: return launch_f<8>(g, table, obj, poses, P, masks, counts, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cf
