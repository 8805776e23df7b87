// Kinematics optimisation and post-processing (Sec. 5.5, Sec. 5.6).
//
// k_ik_dls (Sec. 5.5 "Kinematics Optimization"): for every contact of an
// accepted tuple, the reverse lookup finds the hand-surface sample that put
// the contact's (cell, normal bin) code into the field -- the smallest
// s * M + m over the samples that did, kept by the build's representative
// table -- and starts from that sample's joint vector q_s.  Damped least
// squares then moves the attached hand point p~ onto the object point p and
// p~ + beta n~ onto p + beta n (Eq. DLS of Sec. 5.5; n the inward contact
// normal, n~ the hand's outward normal):
//     dq = (J^T J + lambda I)^-1 J^T e,   q <- clamp(q + dq, lo, hi),
// J the 6 x J position Jacobian of the two points, column j = a_j x (x - o_j)
// for joints j up to the contact link (a_j, o_j the world axis and origin of
// joint j), 0 beyond it: the point form of Eq. (J_p - [p~]x J_r).  Fingers
// share no joint, so the multi-chain normal equations are block diagonal and
// each (tuple, contact) is solved on its own lane.  Phase II ("Finetuning"):
// rounds of projecting (p, n) onto the latest capsule of the contact link, then
// more DLS steps.  Success: |p~ - p| <= tol_pos and n~ . n >= tol_cos after a
// last projection.  The projection keeps the axis point nearest p and picks
// there the capsule normal that minimises the DLS objective: re-attaching the
// nearest surface point instead tilts the attached normal away from n every
// round on a curved link, and the rounds diverge.
//
// k_sdf_build: signed distance of the object's oriented point set on a
// regular grid, by brute force over all points (nearest point, sign of
// (x - p) . n of that point).
//
// k_realize (Sec. 5.6 "Postprocessing"): joints the IK left free get uniform
// random values in their limits (Philox4x32-10); the grasp is rejected when a
// link capsule's axis comes closer to the object surface than its radius less
// the penetration margin (trilinear SDF along the axis), or when capsules of two
// fingers intersect (segment-segment distance below the sum of radii).
#include <string.h>

#include "cf_internal.cuh"

namespace cf {

namespace {

constexpr int kIkThreads = 128;
constexpr int kRealizeWarps = 4;

// Joint axes / origins in the palm frame and the frame of link l (FP32 chain).
template <int J>
__device__ __forceinline__ void chain_fp32(const HandDev &h, int f, const float (&q)[J], int l, float (&ax)[J][3],
                                           float (&og)[J][3], float (&Rl)[9], float (&tl)[3]) {
    const float *b = h.base + 12 * f;
    float R[9] = {__ldg(b + 0), __ldg(b + 1), __ldg(b + 2), __ldg(b + 4), __ldg(b + 5),
                  __ldg(b + 6), __ldg(b + 8), __ldg(b + 9), __ldg(b + 10)};
    float t[3] = {__ldg(b + 3), __ldg(b + 7), __ldg(b + 11)};
#pragma unroll
    for (int j = 0; j < J; ++j) {
        if (j > 0) {
            const float *o = h.offset + 3 * (f * J + j - 1);
            const float o0 = __ldg(o), o1 = __ldg(o + 1), o2 = __ldg(o + 2);
#pragma unroll
            for (int r = 0; r < 3; ++r) t[r] = fmaf(R[3 * r + 2], o2, fmaf(R[3 * r + 1], o1, fmaf(R[3 * r], o0, t[r])));
        }
        const float *a = h.axis + 3 * (f * J + j);
        const float x = __ldg(a), y = __ldg(a + 1), z = __ldg(a + 2);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            ax[j][r] = R[3 * r] * x + R[3 * r + 1] * y + R[3 * r + 2] * z;
            og[j][r] = t[r];
        }
        float s, c;
        sincosf(q[j], &s, &c);
        const float v = 1.f - c;
        const float Q[9] = {c + x * x * v,     x * y * v - z * s, x * z * v + y * s,
                            y * x * v + z * s, c + y * y * v,     y * z * v - x * s,
                            z * x * v - y * s, z * y * v + x * s, c + z * z * v};
        float Rn[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
                Rn[3 * r + cc] = R[3 * r] * Q[cc] + R[3 * r + 1] * Q[3 + cc] + R[3 * r + 2] * Q[6 + cc];
#pragma unroll
        for (int e = 0; e < 9; ++e) R[e] = Rn[e];
        if (j == l) {
#pragma unroll
            for (int e = 0; e < 9; ++e) Rl[e] = R[e];
#pragma unroll
            for (int r = 0; r < 3; ++r) tl[r] = t[r];
        }
    }
}

// Capsule axes of finger f (palm frame): link j runs from the origin of its
// frame along offset_j; written to cap[cap_of[f * J + j]] as (start, vector).
template <int J>
__device__ __forceinline__ void chain_capsules(const HandDev &h, int f, const float (&q)[J], const int8_t *cap_of,
                                               float (*cap)[6]) {
    const float *b = h.base + 12 * f;
    float R[9] = {__ldg(b + 0), __ldg(b + 1), __ldg(b + 2), __ldg(b + 4), __ldg(b + 5),
                  __ldg(b + 6), __ldg(b + 8), __ldg(b + 9), __ldg(b + 10)};
    float t[3] = {__ldg(b + 3), __ldg(b + 7), __ldg(b + 11)};
#pragma unroll
    for (int j = 0; j < J; ++j) {
        if (j > 0) {
            const float *o = h.offset + 3 * (f * J + j - 1);
            const float o0 = __ldg(o), o1 = __ldg(o + 1), o2 = __ldg(o + 2);
#pragma unroll
            for (int r = 0; r < 3; ++r) t[r] = fmaf(R[3 * r + 2], o2, fmaf(R[3 * r + 1], o1, fmaf(R[3 * r], o0, t[r])));
        }
        const float *a = h.axis + 3 * (f * J + j);
        const float x = __ldg(a), y = __ldg(a + 1), z = __ldg(a + 2);
        float s, c;
        sincosf(q[j], &s, &c);
        const float v = 1.f - c;
        const float Q[9] = {c + x * x * v,     x * y * v - z * s, x * z * v + y * s,
                            y * x * v + z * s, c + y * y * v,     y * z * v - x * s,
                            z * x * v - y * s, z * y * v + x * s, c + z * z * v};
        float Rn[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
                Rn[3 * r + cc] = R[3 * r] * Q[cc] + R[3 * r + 1] * Q[3 + cc] + R[3 * r + 2] * Q[6 + cc];
#pragma unroll
        for (int e = 0; e < 9; ++e) R[e] = Rn[e];
        const int cid = cap_of[f * J + j];
        if (cid >= 0) {
            const float *o = h.offset + 3 * (f * J + j);
            const float o0 = __ldg(o), o1 = __ldg(o + 1), o2 = __ldg(o + 2);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cap[cid][r] = t[r];
                cap[cid][3 + r] = R[3 * r] * o0 + R[3 * r + 1] * o1 + R[3 * r + 2] * o2;
            }
        }
    }
}

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// One damped-least-squares step of finger f for the attached point pl / normal
// nl of link l towards (p, n).
template <int J>
__device__ __forceinline__ void dls_step(const IkArgs &a, int f, int l, const float (&pl)[3], const float (&nl)[3],
                                         const float (&p)[3], const float (&n)[3], float (&q)[J]) {
    float ax[J][3], og[J][3], R[9], t[3];
    chain_fp32<J>(a.h, f, q, l, ax, og, R, t);
    float x1[3], x2[3], e1[3], e2[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        x1[r] = t[r] + R[3 * r] * pl[0] + R[3 * r + 1] * pl[1] + R[3 * r + 2] * pl[2];
        const float nn = R[3 * r] * nl[0] + R[3 * r + 1] * nl[1] + R[3 * r + 2] * nl[2];
        x2[r] = x1[r] + a.beta * nn;
        e1[r] = p[r] - x1[r];
        e2[r] = (p[r] + a.beta * n[r]) - x2[r];
    }
    float c1[J][3], c2[J][3];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const float d1[3] = {x1[0] - og[j][0], x1[1] - og[j][1], x1[2] - og[j][2]};
        const float d2[3] = {x2[0] - og[j][0], x2[1] - og[j][1], x2[2] - og[j][2]};
        cross3(ax[j], d1, c1[j]);
        cross3(ax[j], d2, c2[j]);
        if (j > l) {
#pragma unroll
            for (int r = 0; r < 3; ++r) c1[j][r] = c2[j][r] = 0.f;
        }
    }
    // normal equations (J^T J + lambda I) dq = J^T e, Cholesky in registers
    float L[J][J], y[J], inv[J];
#pragma unroll
    for (int i = 0; i < J; ++i) {
        y[i] = c1[i][0] * e1[0] + c1[i][1] * e1[1] + c1[i][2] * e1[2] + c2[i][0] * e2[0] + c2[i][1] * e2[1] +
               c2[i][2] * e2[2];
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float s = c1[i][0] * c1[j][0] + c1[i][1] * c1[j][1] + c1[i][2] * c1[j][2] + c2[i][0] * c2[j][0] +
                      c2[i][1] * c2[j][1] + c2[i][2] * c2[j][2];
            if (i == j) s += a.lambda;
#pragma unroll
            for (int kk = 0; kk < j; ++kk) s -= L[i][kk] * L[j][kk];
            if (i == j) {
                L[i][i] = sqrtf(fmaxf(s, 1e-30f));
                inv[i] = 1.f / L[i][i];
            } else {
                L[i][j] = s * inv[j];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < J; ++i) {
#pragma unroll
        for (int kk = 0; kk < i; ++kk) y[i] -= L[i][kk] * y[kk];
        y[i] *= inv[i];
    }
#pragma unroll
    for (int i = J - 1; i >= 0; --i) {
#pragma unroll
        for (int kk = i + 1; kk < J; ++kk) y[i] -= L[kk][i] * y[kk];
        y[i] *= inv[i];
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const float lo = __ldg(a.h.lo + f * J + j), hi = __ldg(a.h.hi + f * J + j);
        q[j] = fminf(fmaxf(q[j] + y[j], lo), hi);
    }
}

// Phase II projection of the target (p, n) onto the capsule of link l: the
// axis point c nearest p, and there the outward capsule normal minimising the
// DLS objective |p~ - p|^2 + |p~ + beta n~ - p - beta n|^2 with p~ = c + r n~:
// the direction of w = (2r + beta)(p - c) + beta (r + beta) n, restricted to
// the normals the capsule has at c (perpendicular to the axis inside the
// segment, the outward hemisphere at an end).  Updates the attached point /
// normal (link frame) and returns the palm-frame point and normal.
template <int J>
__device__ __forceinline__ void project_capsule(const IkArgs &a, int f, int l, const float (&q)[J],
                                                const float (&p)[3], const float (&n)[3], float (&pl)[3],
                                                float (&nl)[3], float (&xw)[3], float (&nw)[3]) {
    float ax[J][3], og[J][3], R[9], t[3];
    chain_fp32<J>(a.h, f, q, l, ax, og, R, t);
    const float *o = a.h.offset + 3 * (f * J + l);
    const float o0 = __ldg(o), o1 = __ldg(o + 1), o2 = __ldg(o + 2);
    float bv[3], d[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        bv[r] = R[3 * r] * o0 + R[3 * r + 1] * o1 + R[3 * r + 2] * o2;
        d[r] = p[r] - t[r];
    }
    const float L2 = bv[0] * bv[0] + bv[1] * bv[1] + bv[2] * bv[2];
    float s = 0.f;
    if (L2 > 0.f) s = fminf(fmaxf((d[0] * bv[0] + d[1] * bv[1] + d[2] * bv[2]) / L2, 0.f), 1.f);
    const float rad = __ldg(a.h.radius + f * J + l);
    const float wa = 2.f * rad + a.beta, wb = a.beta * (rad + a.beta);
    float cpt[3], w[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        cpt[r] = t[r] + s * bv[r];
        w[r] = wa * (p[r] - cpt[r]) + wb * n[r];
    }
    if (L2 > 0.f) {
        const float il = 1.f / sqrtf(L2);
        const float u[3] = {bv[0] * il, bv[1] * il, bv[2] * il};
        const float wu = w[0] * u[0] + w[1] * u[1] + w[2] * u[2];
        if ((s > 0.f && s < 1.f) || (s <= 0.f && wu > 0.f) || (s >= 1.f && wu < 0.f)) {
#pragma unroll
            for (int r = 0; r < 3; ++r) w[r] -= wu * u[r];
        }
    }
    const float wn = sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (wn > 1e-12f) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            nw[r] = w[r] / wn;
            xw[r] = cpt[r] + rad * nw[r];
        }
        // back into the link frame: R^T (x - t), R^T n
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            pl[cc] = R[cc] * (xw[0] - t[0]) + R[3 + cc] * (xw[1] - t[1]) + R[6 + cc] * (xw[2] - t[2]);
            nl[cc] = R[cc] * nw[0] + R[3 + cc] * nw[1] + R[6 + cc] * nw[2];
        }
    } else {  // degenerate: keep the attached point
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            xw[r] = t[r] + R[3 * r] * pl[0] + R[3 * r + 1] * pl[1] + R[3 * r + 2] * pl[2];
            nw[r] = R[3 * r] * nl[0] + R[3 * r + 1] * nl[1] + R[3 * r + 2] * nl[2];
        }
    }
}

// Pass 1: accepted slots go to a work list (order irrelevant: every slot
// writes only its own outputs); the others get their "not attempted" outputs.
__global__ void __launch_bounds__(256) k_ik_compact(const IkArgs a, int *list, unsigned int *count) {
    const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = slot < a.n;
    const bool acc = in && (!a.accept || a.accept[slot]);
    const unsigned full = 0xffffffffu;
    const unsigned bal = __ballot_sync(full, acc);
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == 0 && bal) base = atomicAdd(count, (unsigned)__popc(bal));
    base = __shfl_sync(full, base, 0);
    if (acc) list[base + __popc(bal & ((1u << lane) - 1u))] = (int)slot;
    if (!in || acc) return;
    const int k = a.k, F = a.h.F, J = a.h.J;
    for (int c = 0; c < k; ++c) {
        const size_t e = (size_t)slot * k + c;
        a.rtuples[e] = -1;
        a.resid[2 * e] = INFINITY;
        a.resid[2 * e + 1] = -2.f;
        for (int i = 0; i < 6; ++i) a.cp[i][e] = 0.f;
    }
    a.ok[slot] = 0;
    for (int i = 0; i < F * J; ++i) {
        a.q[(size_t)slot * F * J + i] = 0.f;
        a.used[(size_t)slot * F * J + i] = 0;
    }
}

// Pass 2, lanes in groups of k: group g of warp w works on list entry
// w * (32 / k) + g, lane c of the group on its contact c.
template <int J>
__global__ void __launch_bounds__(kIkThreads) k_ik_dls(const IkArgs a, const int *__restrict__ list,
                                                       const unsigned int *__restrict__ count) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int k = a.k, G = 32 / k;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int grp = lane / k, c = lane - grp * k;
    const long long entry = gw * G + grp;
    const long long n_list = (long long)*count;
    if (gw * G >= n_list) return;  // warp-uniform: the whole warp is past the list
    const bool in_grp = grp < G && entry < n_list;
    const long long slot = in_grp ? (long long)__ldg(list + entry) : 0;
    const unsigned gmask = in_grp ? (((1u << k) - 1u) << (grp * k)) : 0u;
    const int F = a.h.F, M = a.h.M;

    int x = -1, f = 255;
    bool live = in_grp;
    if (live) {
        x = __ldg(a.tuples + slot * k + c);
        f = a.fingers ? (int)__ldg(a.fingers + slot * k + c) : 255;
        live = x >= 0 && x < a.obj.n && f < F;
    }
    unsigned fset = 0u;  // fingers of the group (for the rows no contact writes)
    bool dup = false;
    for (int cc = 0; cc < k; ++cc) {
        const int src = min(grp * k + cc, 31);
        const int ff = __shfl_sync(full, f, src);
        if (ff < F) fset |= 1u << ff;
        if (cc != c && ff == f) dup = true;
    }
    const unsigned vb = __ballot_sync(full, live && !dup);
    const bool gvalid = in_grp && (vb & gmask) == gmask;

    bool ok_c = false;
    float pos = INFINITY, cosv = -2.f;
    float xo[3] = {0.f, 0.f, 0.f}, no[3] = {0.f, 0.f, 0.f};
    // ---- setup: target vector, reverse lookup, starting sample ----
    int link = -1;                                            // contact link; joints beyond it stay free
    float pl[3] = {0.f, 0.f, 0.f}, nl[3] = {0.f, 0.f, 1.f};   // attached point / normal (link frame)
    float p[3] = {0.f, 0.f, 0.f}, n[3] = {0.f, 0.f, 0.f};     // target: the query's FP32 contact-surface vector
    float Tp[12];
    float q[J];
#pragma unroll
    for (int j = 0; j < J; ++j) q[j] = 0.f;
#pragma unroll
    for (int e = 0; e < 12; ++e) Tp[e] = 0.f;
    bool attempt = false;
    if (gvalid) {
        const float *T = a.poses + (size_t)(slot / a.T) * 12;
#pragma unroll
        for (int e = 0; e < 12; ++e) Tp[e] = __ldg(T + e);
        const float ox = __ldg(a.obj.px + x), oy = __ldg(a.obj.py + x), oz = __ldg(a.obj.pz + x);
        const float onx = __ldg(a.obj.nx + x), ony = __ldg(a.obj.ny + x), onz = __ldg(a.obj.nz + x);
        p[0] = xf_row(Tp[0], Tp[1], Tp[2], Tp[3], ox, oy, oz);
        p[1] = xf_row(Tp[4], Tp[5], Tp[6], Tp[7], ox, oy, oz);
        p[2] = xf_row(Tp[8], Tp[9], Tp[10], Tp[11], ox, oy, oz);
        n[0] = -rot_row(Tp[0], Tp[1], Tp[2], onx, ony, onz);
        n[1] = -rot_row(Tp[4], Tp[5], Tp[6], onx, ony, onz);
        n[2] = -rot_row(Tp[8], Tp[9], Tp[10], onx, ony, onz);
        // reverse lookup of the (cell, bin) code
        const FieldGeom &g = a.g;
        int bin = 0;
        float best = -INFINITY;
        for (int b = 0; b < g.B; ++b) {
            const float sc = __fmaf_rn(g.dirs[b][2], n[2], __fmaf_rn(g.dirs[b][1], n[1], __fmul_rn(g.dirs[b][0], n[0])));
            if (sc > best) { best = sc; bin = b; }
        }
        const unsigned ux = (unsigned)(cell_floor(p[0], g.inv_h, g.clamp) - g.lo[0]);
        const unsigned uy = (unsigned)(cell_floor(p[1], g.inv_h, g.clamp) - g.lo[1]);
        const unsigned uz = (unsigned)(cell_floor(p[2], g.inv_h, g.clamp) - g.lo[2]);
        uint32_t v = 0xffffffffu;
        if (ux < (unsigned)g.dims[0] && uy < (unsigned)g.dims[1] && uz < (unsigned)g.dims[2]) {
            const unsigned long long word =
                (((unsigned long long)uz * g.dims[1] + uy) * g.dims[0] + ux) * g.rw + f / g.fpw;
            const unsigned long long base = word * 32ull + (unsigned)((f % g.fpw) * g.bits);
            v = rep_lookup(a.rep, base + (unsigned)bin);
            // with dilated bins the hit may come from another accepted bin: the lowest one present
            for (uint32_t rest = g.dil[bin] & ~(1u << bin); v == 0xffffffffu && rest; rest &= rest - 1)
                v = rep_lookup(a.rep, base + (unsigned)(__ffs(rest) - 1));
        }
        attempt = v != 0xffffffffu;
        if (!attempt) {
            atomicOr(a.status, CF_DEV_REP_MISS);
#pragma unroll
            for (int j = 0; j < J; ++j) q[j] = __ldg(a.h.lo + f * J + j);
        } else {
            const int s = (int)(v / (uint32_t)M), m = (int)(v % (uint32_t)M);
#pragma unroll
            for (int j = 0; j < J; ++j) q[j] = __ldg(a.qs + ((size_t)f * J + j) * a.S + s);
            const float *sp = a.h.surf + ((size_t)f * M + __ldg(a.h.sorted_of + f * M + m)) * 8;
            pl[0] = __ldg(sp); pl[1] = __ldg(sp + 1); pl[2] = __ldg(sp + 2);
            nl[0] = __ldg(sp + 3); nl[1] = __ldg(sp + 4); nl[2] = __ldg(sp + 5);
            link = (int)__ldg(sp + 6);
        }
    }
    // ---- IK: one loop over the DLS steps with the Phase II projections in
    // between (a single inlined copy of each); the lanes that run it are
    // re-converged after every step, since their contacts sit on different links
    const unsigned ikmask = __ballot_sync(full, attempt);
    if (attempt) {
        const int n1 = a.n1, nr = a.nr, n2 = a.n2, total = n1 + nr * n2;
        float xw[3], nw[3];
        for (int it = 0; it <= total; ++it) {
            // projections due before DLS step `it` (after the last one when it == total)
            int nproj = 0;
            if (n2 > 0) {
                const int d = it - n1;
                nproj = (d >= 0 && d % n2 == 0 && d / n2 < nr) ? 1 : 0;
                if (it == total) nproj += 1;
            } else if (it == total) {
                nproj = nr + 1;
            }
            for (int pj = 0; pj < nproj; ++pj) project_capsule<J>(a, f, link, q, p, n, pl, nl, xw, nw);
            if (it == total) break;
            dls_step<J>(a, f, link, pl, nl, p, n, q);
            __syncwarp(ikmask);
        }
        const float dx = xw[0] - p[0], dy = xw[1] - p[1], dz = xw[2] - p[2];
        pos = sqrtf(dx * dx + dy * dy + dz * dz);
        cosv = nw[0] * n[0] + nw[1] * n[1] + nw[2] * n[2];
        ok_c = pos <= a.tol_pos && cosv >= a.tol_cos;
        // realised contact in the object frame: R^T (x - t); outward object normal -R^T n~
        const float d[3] = {xw[0] - Tp[3], xw[1] - Tp[7], xw[2] - Tp[11]};
        xo[0] = Tp[0] * d[0] + Tp[4] * d[1] + Tp[8] * d[2];
        xo[1] = Tp[1] * d[0] + Tp[5] * d[1] + Tp[9] * d[2];
        xo[2] = Tp[2] * d[0] + Tp[6] * d[1] + Tp[10] * d[2];
        no[0] = -(Tp[0] * nw[0] + Tp[4] * nw[1] + Tp[8] * nw[2]);
        no[1] = -(Tp[1] * nw[0] + Tp[5] * nw[1] + Tp[9] * nw[2]);
        no[2] = -(Tp[2] * nw[0] + Tp[6] * nw[1] + Tp[10] * nw[2]);
    }
    if (gvalid) {
        float *qo = a.q + ((size_t)slot * F + f) * J;
        uint8_t *uo = a.used + ((size_t)slot * F + f) * J;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            qo[j] = q[j];
            uo[j] = (uint8_t)(j <= link);
        }
    }
    const unsigned okb = __ballot_sync(full, ok_c);
    const bool gok = gvalid && (okb & gmask) == gmask;
    if (in_grp) {
        const size_t e = (size_t)slot * k + c;
        a.rtuples[e] = gok ? (int32_t)e : -1;
        a.resid[2 * e] = pos;
        a.resid[2 * e + 1] = cosv;
        a.cp[0][e] = xo[0]; a.cp[1][e] = xo[1]; a.cp[2][e] = xo[2];
        a.cp[3][e] = no[0]; a.cp[4][e] = no[1]; a.cp[5][e] = no[2];
        if (c == 0) {
            a.ok[slot] = (uint8_t)gok;
            for (int ff = 0; ff < F; ++ff) {
                if (gvalid && ((fset >> ff) & 1u)) continue;
                float *qo = a.q + ((size_t)slot * F + ff) * J;
                uint8_t *uo = a.used + ((size_t)slot * F + ff) * J;
                for (int j = 0; j < J; ++j) { qo[j] = 0.f; uo[j] = 0; }
            }
        }
    }
}

// ---- object SDF grid ---------------------------------------------------------
constexpr int kSdfThreads = 256;
constexpr int kSdfTile = 1024;

__global__ void __launch_bounds__(kSdfThreads) k_sdf_build(const cf_points obj, const SdfGrid g, float *grid) {
    __shared__ float s_p[6][kSdfTile];
    const long long nodes = (long long)g.dims[0] * g.dims[1] * g.dims[2];
    const long long id = (long long)blockIdx.x * kSdfThreads + threadIdx.x;
    const bool live = id < nodes;
    const int ix = live ? (int)(id % g.dims[0]) : 0;
    const int iy = live ? (int)((id / g.dims[0]) % g.dims[1]) : 0;
    const int iz = live ? (int)(id / ((long long)g.dims[0] * g.dims[1])) : 0;
    const float gx = fmaf((float)ix, g.h, g.lo[0]), gy = fmaf((float)iy, g.h, g.lo[1]),
                gz = fmaf((float)iz, g.h, g.lo[2]);
    float best = INFINITY, bsx = 0.f, bsy = 0.f, bsz = 0.f;
    for (int base = 0; base < obj.n; base += kSdfTile) {
        const int cnt = min(kSdfTile, obj.n - base);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt; e += kSdfThreads) {
            s_p[0][e] = __ldg(obj.px + base + e);
            s_p[1][e] = __ldg(obj.py + base + e);
            s_p[2][e] = __ldg(obj.pz + base + e);
            s_p[3][e] = __ldg(obj.nx + base + e);
            s_p[4][e] = __ldg(obj.ny + base + e);
            s_p[5][e] = __ldg(obj.nz + base + e);
        }
        __syncthreads();
        int bi = -1;
        for (int e = 0; e < cnt; ++e) {
            const float dx = gx - s_p[0][e], dy = gy - s_p[1][e], dz = gz - s_p[2][e];
            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (d2 < best) { best = d2; bi = e; }
        }
        if (bi >= 0) {  // sign of the nearest point so far: (x - p) . n
            const float dx = gx - s_p[0][bi], dy = gy - s_p[1][bi], dz = gz - s_p[2][bi];
            bsx = dx * s_p[3][bi];
            bsy = dy * s_p[4][bi];
            bsz = dz * s_p[5][bi];
        }
    }
    if (live) {
        const float side = bsx + bsy + bsz;
        grid[id] = side >= 0.f ? sqrtf(best) : -sqrtf(best);
    }
}

// ---- realization filter --------------------------------------------------------
// Distance between segments [p0, p0 + d1] and [q0, q0 + d2] (both of positive
// length): minimum of the convex quadratic |p0 + s d1 - q0 - t d2|^2 over the
// unit square -- the unconstrained s for the unconstrained t, clamped, then t
// for that s, clamped, and s again when t was clamped.
__device__ __forceinline__ float seg_seg_dist(const float *p0, const float *d1, const float *q0, const float *d2) {
    const float r[3] = {p0[0] - q0[0], p0[1] - q0[1], p0[2] - q0[2]};
    const float aa = d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2];
    const float ee = d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2];
    const float bb = d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2];
    const float cc = d1[0] * r[0] + d1[1] * r[1] + d1[2] * r[2];
    const float ff = d2[0] * r[0] + d2[1] * r[1] + d2[2] * r[2];
    const float den = aa * ee - bb * bb;
    float s = den > 1e-12f * aa * ee ? fminf(fmaxf((bb * ff - cc * ee) / den, 0.f), 1.f) : 0.f;
    float t = (bb * s + ff) / ee;
    if (t < 0.f) {
        t = 0.f;
        s = fminf(fmaxf(-cc / aa, 0.f), 1.f);
    } else if (t > 1.f) {
        t = 1.f;
        s = fminf(fmaxf((bb - cc) / aa, 0.f), 1.f);
    }
    const float dx = r[0] + s * d1[0] - t * d2[0], dy = r[1] + s * d1[1] - t * d2[1], dz = r[2] + s * d1[2] - t * d2[2];
    return sqrtf(dx * dx + dy * dy + dz * dz);
}

// One warp per tuple slot.
template <int J>
__global__ void __launch_bounds__(32 * kRealizeWarps) k_realize(const RealizeArgs a) {
    __shared__ float s_cap[kRealizeWarps][kMaxCapsules][6];  // axis start, axis vector (palm frame)
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long slot = (long long)blockIdx.x * kRealizeWarps + wib;
    if (slot >= a.n) return;  // warp-uniform
    const bool gate = (!a.gate_a || a.gate_a[slot]) && (!a.gate_b || a.gate_b[slot]);
    if (!gate) {
        if (lane == 0) a.flags[slot] = 1u;
        return;
    }
    const int F = a.h.F;
    float(*cap)[6] = s_cap[wib];
    if (lane < F) {
        const int f = lane;
        float q[J];
        float *qrow = a.q + ((size_t)slot * F + f) * J;
        const uint8_t *urow = a.used + ((size_t)slot * F + f) * J;
        uint4 rnd = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if ((j & 3) == 0)
                rnd = philox4x32_10(make_uint4((uint32_t)slot, (uint32_t)f, (uint32_t)(j >> 2), 0x7EA1u),
                                    make_uint2(a.seed_lo, a.seed_hi));
            if (urow[j]) {
                q[j] = qrow[j];
            } else {
                const uint32_t w = (j & 3) == 0 ? rnd.x : (j & 3) == 1 ? rnd.y : (j & 3) == 2 ? rnd.z : rnd.w;
                const float lo = __ldg(a.h.lo + f * J + j), hi = __ldg(a.h.hi + f * J + j);
                const float u = __fmul_rn((float)(w >> 8), 5.9604644775390625e-8f);  // exact: u24 * 2^-24
                q[j] = __fadd_rn(lo, __fmul_rn(u, __fsub_rn(hi, lo)));
                qrow[j] = q[j];
            }
        }
        chain_capsules<J>(a.h, f, q, a.cap_of, cap);
    }
    __syncwarp();
    const float *T = a.poses + (size_t)(slot / a.T) * 12;
    const float T0 = __ldg(T), T1 = __ldg(T + 1), T2 = __ldg(T + 2), T3 = __ldg(T + 3);
    const float T4 = __ldg(T + 4), T5 = __ldg(T + 5), T6 = __ldg(T + 6), T7 = __ldg(T + 7);
    const float T8 = __ldg(T + 8), T9 = __ldg(T + 9), T10 = __ldg(T + 10), T11 = __ldg(T + 11);
    bool pen = false;
    for (int cid = 0; cid < a.n_caps; ++cid) {
        const int ns = a.cap_ns[cid];
        const float thr = a.cap_r[cid] - a.pen_margin;
        for (int s = lane; s <= ns; s += 32) {
            const float fr = (float)s / (float)ns;
            const float x = fmaf(fr, cap[cid][3], cap[cid][0]) - T3;
            const float y = fmaf(fr, cap[cid][4], cap[cid][1]) - T7;
            const float z = fmaf(fr, cap[cid][5], cap[cid][2]) - T11;
            // palm -> object frame: R^T (x - t)
            const float ox = T0 * x + T4 * y + T8 * z, oy = T1 * x + T5 * y + T9 * z, oz = T2 * x + T6 * y + T10 * z;
            pen = pen || sdf_at(a.sdf, ox, oy, oz) < thr;
        }
    }
    bool col = false;
    const int nc = a.n_caps;
    for (int pidx = lane; pidx < nc * nc; pidx += 32) {
        const int c1 = pidx / nc, c2 = pidx - c1 * nc;
        if (c1 >= c2 || a.cap_f[c1] == a.cap_f[c2]) continue;
        const float d = seg_seg_dist(cap[c1], cap[c1] + 3, cap[c2], cap[c2] + 3);
        col = col || d < a.cap_r[c1] + a.cap_r[c2];
    }
    const bool anyp = __any_sync(full, pen), anyc = __any_sync(full, col);
    if (lane == 0) a.flags[slot] = (uint8_t)((anyp ? 2u : 0u) | (anyc ? 4u : 0u));
}

#define CF_KJ_DISPATCH(J, CALL)                         \
    switch (J) {                                        \
        case 1: { constexpr int JJ = 1; CALL; } break;  \
        case 2: { constexpr int JJ = 2; CALL; } break;  \
        case 3: { constexpr int JJ = 3; CALL; } break;  \
        case 4: { constexpr int JJ = 4; CALL; } break;  \
        case 5: { constexpr int JJ = 5; CALL; } break;  \
        case 6: { constexpr int JJ = 6; CALL; } break;  \
        case 7: { constexpr int JJ = 7; CALL; } break;  \
        case 8: { constexpr int JJ = 8; CALL; } break;  \
        default: return cudaErrorInvalidValue;          \
    }

}  // namespace

cudaError_t launch_ik(const IkArgs &a, int *list, unsigned int *count, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    k_ik_compact<<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(a, list, count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long G = 32 / a.k;
    const long long warps = (a.n + G - 1) / G;
    const long long blocks = (warps * 32 + kIkThreads - 1) / kIkThreads;
    CF_KJ_DISPATCH(a.h.J, (k_ik_dls<JJ><<<(unsigned)blocks, kIkThreads, 0, st>>>(a, list, count)));
    return cudaGetLastError();
}

cudaError_t launch_sdf(const cf_points &obj, const SdfGrid &g, float *grid, cudaStream_t st) {
    const long long nodes = (long long)g.dims[0] * g.dims[1] * g.dims[2];
    if (nodes <= 0) return cudaSuccess;
    k_sdf_build<<<(unsigned)((nodes + kSdfThreads - 1) / kSdfThreads), kSdfThreads, 0, st>>>(obj, g, grid);
    return cudaGetLastError();
}

cudaError_t launch_realize(const RealizeArgs &a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    const long long blocks = (a.n + kRealizeWarps - 1) / kRealizeWarps;
    CF_KJ_DISPATCH(a.h.J, (k_realize<JJ><<<(unsigned)blocks, 32 * kRealizeWarps, 0, st>>>(a)));
    return cudaGetLastError();
}

}  // namespace cf
