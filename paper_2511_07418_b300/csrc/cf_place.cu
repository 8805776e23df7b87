// Object placement (Sec. 5.2) and object preprocessing (Sec. 5.1).
//
// k_place_canonical: the object's centroid goes to g + d up with d uniform in
// [d_lo, d_hi] and the object turns by a uniform rotation about its centroid
// (Shoemake's quaternion from three uniforms) -- the "box region above the
// palm" of canonical placement.
//
// k_place_exhaustive: a uniformly random code of the hand's field (the r-th set
// bit of the table in table order: cell, then finger, then bin) gives a point
// (its cell's centre) and a normal (its bin direction d_b); a uniformly random
// object point x is aligned with it -- R takes the object's outward normal n_x
// to -d_b (so the contact-surface normal -R n_x is d_b) and then spins by a
// uniform angle about d_b -- and t puts R p_x on the cell centre.
//
// Both draw from Philox4x32-10 (counter (pose + pose_base, tag, 0, 0), key
// seed) and compute in FP64, rounding the pose to FP32.
//
// k_concave: a small cube of side s rests on the tangent plane outside each
// object point (centre p + (s/2) n, axes the Duff et al. 2017 basis of n and n);
// the point is concave -- removed -- when the object's SDF at the cube's centre
// or at a corner of its upper half (heights s/2 and s, lateral +-s/2) is below
// -tau: the surface closes in on the box.  The lower half is not sampled: a
// point-sampled SDF's sign is unreliable that close to the surface.  k_compact writes the kept points in their
// original order.
#include <math.h>

#include "cf_internal.cuh"

namespace cf {

namespace {

constexpr int kPlaceThreads = 128;
constexpr int kConcaveThreads = 1024;

__global__ void k_chunk_counts(const uint32_t *__restrict__ table, long long words, unsigned long long *counts) {
    __shared__ unsigned s[kChunkWords / 32];
    const long long w = (long long)blockIdx.x * kChunkWords + threadIdx.x;
    const unsigned c = w < words ? __popc(__ldg(table + w)) : 0u;
    const unsigned r = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < kChunkWords / 32; ++i) t += s[i];
        counts[blockIdx.x] = t;
    }
}

__device__ __forceinline__ double unit24(uint32_t w) { return (double)(w >> 8) * 5.9604644775390625e-8; }

// R = cos a I + sin a [k]x + (1 - cos a) k k^T (k unit)
__device__ __forceinline__ void rodrigues(const double k[3], double ang, double R[9]) {
    double s, c;
    sincos(ang, &s, &c);
    const double v = 1.0 - c;
    R[0] = c + k[0] * k[0] * v;        R[1] = k[0] * k[1] * v - k[2] * s; R[2] = k[0] * k[2] * v + k[1] * s;
    R[3] = k[1] * k[0] * v + k[2] * s; R[4] = c + k[1] * k[1] * v;        R[5] = k[1] * k[2] * v - k[0] * s;
    R[6] = k[2] * k[0] * v - k[1] * s; R[7] = k[2] * k[1] * v + k[0] * s; R[8] = c + k[2] * k[2] * v;
}

__device__ __forceinline__ void store_pose(float *out, const double R[9], const double t[3]) {
    for (int r = 0; r < 3; ++r) {
        out[4 * r] = (float)R[3 * r];
        out[4 * r + 1] = (float)R[3 * r + 1];
        out[4 * r + 2] = (float)R[3 * r + 2];
        out[4 * r + 3] = (float)t[r];
    }
}

__global__ void __launch_bounds__(kPlaceThreads) k_place_canonical(const PlaceArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.P) return;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i + a.pose_base, 0x91ACu, 0u, 0u), make_uint2(a.seed_lo, a.seed_hi));
    const double u1 = unit24(w.x), u2 = unit24(w.y), u3 = unit24(w.z), u4 = unit24(w.w);
    const double s1 = sqrt(1.0 - u1), s2 = sqrt(u1);
    double sa, ca, sb, cb;
    sincospi(2.0 * u2, &sa, &ca);
    sincospi(2.0 * u3, &sb, &cb);
    const double x = s1 * sa, y = s1 * ca, z = s2 * sb, qw = s2 * cb;  // unit quaternion (x, y, z, w)
    const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - z * qw),     2 * (x * z + y * qw),
                         2 * (x * y + z * qw),     1 - 2 * (x * x + z * z), 2 * (y * z - x * qw),
                         2 * (x * z - y * qw),     2 * (y * z + x * qw),     1 - 2 * (x * x + y * y)};
    const double d = (double)a.d_lo + u4 * ((double)a.d_hi - (double)a.d_lo);
    double t[3];
    for (int r = 0; r < 3; ++r) {
        const double rc = R[3 * r] * a.centroid[0] + R[3 * r + 1] * a.centroid[1] + R[3 * r + 2] * a.centroid[2];
        t[r] = (double)a.g[r] + d * (double)a.up[r] - rc;
    }
    store_pose(a.poses + 12 * (size_t)i, R, t);
}

__global__ void __launch_bounds__(kPlaceThreads) k_place_exhaustive(const PlaceArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.P) return;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i + a.pose_base, 0xE7A1u, 0u, 0u), make_uint2(a.seed_lo, a.seed_hi));
    // the r-th code in table order
    const unsigned long long r = ((unsigned long long)w.x * a.n_codes) >> 32;
    int lo = 0, hi = a.n_chunks - 1;  // last chunk with prefix <= r
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(a.prefix + mid) <= r) lo = mid; else hi = mid - 1;
    }
    unsigned long long rr = r - __ldg(a.prefix + lo);
    long long word = -1;
    int bit = 0;
    const long long w_end = min((long long)(lo + 1) * kChunkWords, a.table_words);
    for (long long wi = (long long)lo * kChunkWords; wi < w_end; ++wi) {
        const uint32_t v = __ldg(a.table + wi);
        const unsigned c = __popc(v);
        if (rr < c) {
            word = wi;
            bit = __fns(v, 0u, (int)rr + 1);
            break;
        }
        rr -= c;
    }
    if (word < 0) {  // cannot happen with consistent prefixes: leave an identity pose far away
        const double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, t[3] = {1e3, 1e3, 1e3};
        store_pose(a.poses + 12 * (size_t)i, R, t);
        return;
    }
    const FieldGeom &g = a.g_field;
    const long long cell = word / g.rw;
    const int sw = (int)(word % g.rw);
    const int bin = bit % g.bits;
    const long long ux = cell % g.dims[0], uy = (cell / g.dims[0]) % g.dims[1], uz = cell / ((long long)g.dims[0] * g.dims[1]);
    (void)sw;
    const double ih = (double)g.inv_h;
    const double pc[3] = {((double)(ux + g.lo[0]) + 0.5) / ih, ((double)(uy + g.lo[1]) + 0.5) / ih,
                          ((double)(uz + g.lo[2]) + 0.5) / ih};
    double dv[3] = {g.dirs[bin][0], g.dirs[bin][1], g.dirs[bin][2]};
    const double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    for (int c = 0; c < 3; ++c) dv[c] /= dn;
    // the object point
    const int x = (int)(((unsigned long long)w.y * (unsigned long long)a.obj.n) >> 32);
    double av[3] = {__ldg(a.obj.nx + x), __ldg(a.obj.ny + x), __ldg(a.obj.nz + x)};
    const double an = sqrt(av[0] * av[0] + av[1] * av[1] + av[2] * av[2]);
    for (int c = 0; c < 3; ++c) av[c] /= an;
    const double b[3] = {-dv[0], -dv[1], -dv[2]};
    // R_align: a -> b
    double v[3] = {av[1] * b[2] - av[2] * b[1], av[2] * b[0] - av[0] * b[2], av[0] * b[1] - av[1] * b[0]};
    const double s = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const double cdot = av[0] * b[0] + av[1] * b[1] + av[2] * b[2];
    double Ra[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (s > 1e-12) {
        for (int c = 0; c < 3; ++c) v[c] /= s;
        rodrigues(v, atan2(s, cdot), Ra);
    } else if (cdot < 0.0) {  // opposite: a half turn about any axis perpendicular to a
        const double e[3] = {fabs(av[0]) < 0.9 ? 1.0 : 0.0, fabs(av[0]) < 0.9 ? 0.0 : 1.0, 0.0};
        double k[3] = {av[1] * e[2] - av[2] * e[1], av[2] * e[0] - av[0] * e[2], av[0] * e[1] - av[1] * e[0]};
        const double kn = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        for (int c = 0; c < 3; ++c) k[c] /= kn;
        rodrigues(k, M_PI, Ra);
    }
    double Rs[9];
    rodrigues(dv, 2.0 * M_PI * unit24(w.z), Rs);
    double R[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) R[3 * r + c] = Rs[3 * r] * Ra[c] + Rs[3 * r + 1] * Ra[3 + c] + Rs[3 * r + 2] * Ra[6 + c];
    const double px[3] = {__ldg(a.obj.px + x), __ldg(a.obj.py + x), __ldg(a.obj.pz + x)};
    double t[3];
    for (int r = 0; r < 3; ++r) t[r] = pc[r] - (R[3 * r] * px[0] + R[3 * r + 1] * px[1] + R[3 * r + 2] * px[2]);
    store_pose(a.poses + 12 * (size_t)i, R, t);
}

// pass 1: keep flags and one count per block
__global__ void __launch_bounds__(kConcaveThreads) k_concave(const cf_points obj, const SdfGrid sdf, float side,
                                                             float tau, uint8_t *keep, unsigned int *block_counts) {
    __shared__ unsigned s_w[kConcaveThreads / 32];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    bool k = false;
    if (x < obj.n) {
        const float h = 0.5f * side;
        const float nx = __ldg(obj.nx + x), ny = __ldg(obj.ny + x), nz = __ldg(obj.nz + x);
        const float cx = fmaf(h, nx, __ldg(obj.px + x));
        const float cy = fmaf(h, ny, __ldg(obj.py + x));
        const float cz = fmaf(h, nz, __ldg(obj.pz + x));
        // the cube rests on the tangent plane: axes (t1, t2, n), t1, t2 the Duff et al. 2017 basis of n
        const float sgn = copysignf(1.f, nz);
        const float aa = -1.f / (sgn + nz);
        const float bb = nx * ny * aa;
        const float t1[3] = {1.f + sgn * nx * nx * aa, sgn * bb, -sgn * nx};
        const float t2[3] = {bb, sgn + ny * ny * aa, -ny};
        const float nv[3] = {nx, ny, nz};
        float m = sdf_at(sdf, cx, cy, cz);
        for (int c = 0; c < 8; ++c) {  // the upper half of the cube: heights s/2 and s above the tangent plane
            const float s1 = (c & 1) ? h : -h, s2 = (c & 2) ? h : -h, s3 = (c & 4) ? h : 0.f;
            m = fminf(m, sdf_at(sdf, cx + s1 * t1[0] + s2 * t2[0] + s3 * nv[0], cy + s1 * t1[1] + s2 * t2[1] + s3 * nv[1],
                                cz + s1 * t1[2] + s2 * t2[2] + s3 * nv[2]));
        }
        k = !(m < -tau);
        keep[x] = (uint8_t)k;
    }
    const unsigned b = __ballot_sync(0xffffffffu, k);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int i = 0; i < kConcaveThreads / 32; ++i) t += s_w[i];
        block_counts[blockIdx.x] = t;
    }
}

// pass 2: kept points in their original order (block offset = sum of the earlier blocks' counts)
__global__ void __launch_bounds__(kConcaveThreads) k_compact(const cf_points obj, const uint8_t *keep,
                                                             const unsigned int *block_counts, float *out,
                                                             int *n_out) {
    __shared__ unsigned s_w[kConcaveThreads / 32];
    __shared__ unsigned s_base;
    if (threadIdx.x == 0) {
        unsigned base = 0;
        for (unsigned b = 0; b < blockIdx.x; ++b) base += block_counts[b];
        s_base = base;
        if (blockIdx.x == gridDim.x - 1) *n_out = (int)(base + block_counts[blockIdx.x]);
    }
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const bool k = x < obj.n && keep[x];
    const unsigned b = __ballot_sync(0xffffffffu, k);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_w[warp] = __popc(b);
    __syncthreads();
    if (!k || !out) return;
    unsigned off = s_base;
    for (int i = 0; i < warp; ++i) off += s_w[i];
    off += __popc(b & ((1u << lane) - 1u));
    const size_t N = (size_t)obj.n;
    out[off] = __ldg(obj.px + x);
    out[N + off] = __ldg(obj.py + x);
    out[2 * N + off] = __ldg(obj.pz + x);
    out[3 * N + off] = __ldg(obj.nx + x);
    out[4 * N + off] = __ldg(obj.ny + x);
    out[5 * N + off] = __ldg(obj.nz + x);
}

// Static-link placement (Sec. 5.2): block per pose.  Thread 0 draws the pose in
// FP64 (rounded to FP32 in shared memory and in the output); then every thread
// tests its share of the object points against the palm box with the stored
// FP32 pose, and the block stops at the first penetrating point it sees.
constexpr int kStaticThreads = 256;
struct StaticArgs {
    float lo[3], hi[3];
    cf_points obj;
    int P;
    uint32_t seed_lo, seed_hi, pose_base;
    float pen_margin;
    float *poses;
    int32_t *static_pt;
    uint8_t *valid;
};

__global__ void __launch_bounds__(kStaticThreads) k_place_static(const StaticArgs a) {
    __shared__ float s_pose[12];
    __shared__ int s_hit;
    const int i = blockIdx.x;
    if (threadIdx.x == 0) {
        s_hit = 0;
        const uint4 w = philox4x32_10(make_uint4((uint32_t)i + a.pose_base, 0x57A7u, 0u, 0u),
                                      make_uint2(a.seed_lo, a.seed_hi));
        const int x = (int)(((unsigned long long)w.x * (unsigned long long)a.obj.n) >> 32);
        const double c[3] = {(double)a.lo[0] + unit24(w.y) * ((double)a.hi[0] - (double)a.lo[0]),
                             (double)a.lo[1] + unit24(w.z) * ((double)a.hi[1] - (double)a.lo[1]), (double)a.hi[2]};
        double av[3] = {__ldg(a.obj.nx + x), __ldg(a.obj.ny + x), __ldg(a.obj.nz + x)};
        const double an = sqrt(av[0] * av[0] + av[1] * av[1] + av[2] * av[2]);
        for (int k = 0; k < 3; ++k) av[k] /= an;
        // R_align: n_x -> -z
        double v[3] = {-av[1], av[0], 0.0};  // n_x x (-z)
        const double sv = sqrt(v[0] * v[0] + v[1] * v[1]);
        const double cdot = -av[2];
        double Ra[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        if (sv > 1e-12) {
            for (int k = 0; k < 3; ++k) v[k] /= sv;
            rodrigues(v, atan2(sv, cdot), Ra);
        } else if (cdot < 0.0) {  // n_x = +z: a half turn about n_x x e_x / |...| = (0, 1, 0)
            const double k2[3] = {0.0, 1.0, 0.0};
            rodrigues(k2, M_PI, Ra);
        }
        const double zk[3] = {0.0, 0.0, 1.0};
        double Rs[9];
        rodrigues(zk, 2.0 * M_PI * unit24(w.w), Rs);
        double R[9];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc)
                R[3 * r + cc] = Rs[3 * r] * Ra[cc] + Rs[3 * r + 1] * Ra[3 + cc] + Rs[3 * r + 2] * Ra[6 + cc];
        const double px[3] = {__ldg(a.obj.px + x), __ldg(a.obj.py + x), __ldg(a.obj.pz + x)};
        double t[3];
        for (int r = 0; r < 3; ++r) t[r] = c[r] - (R[3 * r] * px[0] + R[3 * r + 1] * px[1] + R[3 * r + 2] * px[2]);
        store_pose(s_pose, R, t);
        store_pose(a.poses + 12 * (size_t)i, R, t);
        a.static_pt[i] = x;
    }
    __syncthreads();
    const float top = a.hi[2] - a.pen_margin;
    for (int j0 = 0; j0 < a.obj.n; j0 += kStaticThreads) {
        const int j = j0 + threadIdx.x;
        bool pen = false;
        if (j < a.obj.n) {
            const float px = __ldg(a.obj.px + j), py = __ldg(a.obj.py + j), pz = __ldg(a.obj.pz + j);
            const float qx = xf_row(s_pose[0], s_pose[1], s_pose[2], s_pose[3], px, py, pz);
            const float qy = xf_row(s_pose[4], s_pose[5], s_pose[6], s_pose[7], px, py, pz);
            const float qz = xf_row(s_pose[8], s_pose[9], s_pose[10], s_pose[11], px, py, pz);
            pen = qx >= a.lo[0] && qx <= a.hi[0] && qy >= a.lo[1] && qy <= a.hi[1] && qz >= a.lo[2] && qz < top;
        }
        if (__any_sync(0xffffffffu, pen) && (threadIdx.x & 31) == 0) s_hit = 1;
        __syncthreads();
        if (s_hit) break;  // block-uniform
    }
    if (threadIdx.x == 0) a.valid[i] = (uint8_t)(s_hit == 0);
}

__global__ void k_append_contact(const int32_t *__restrict__ tuples, long long n, int T, int k,
                                 const int32_t *__restrict__ first, const uint8_t *__restrict__ valid,
                                 int32_t *__restrict__ out) {
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const long long i = u / T;
    const int32_t f0 = __ldg(first + i);
    bool ok = f0 >= 0 && (!valid || __ldg(valid + i) != 0);
    for (int d = 0; d < k; ++d) ok = ok && __ldg(tuples + u * k + d) >= 0;
    int32_t *o = out + u * (k + 1);
    o[0] = ok ? f0 : -1;
    for (int d = 0; d < k; ++d) o[1 + d] = ok ? __ldg(tuples + u * k + d) : -1;
}

}  // namespace

cudaError_t launch_chunk_counts(const uint32_t *table, long long words, unsigned long long *counts, cudaStream_t st) {
    if (words <= 0) return cudaSuccess;
    k_chunk_counts<<<(unsigned)((words + kChunkWords - 1) / kChunkWords), kChunkWords, 0, st>>>(table, words, counts);
    return cudaGetLastError();
}

cudaError_t launch_place(const PlaceArgs &a, bool exhaustive, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((a.P + kPlaceThreads - 1) / kPlaceThreads);
    if (exhaustive)
        k_place_exhaustive<<<grid, kPlaceThreads, 0, st>>>(a);
    else
        k_place_canonical<<<grid, kPlaceThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_concave(const cf_points &obj, const SdfGrid &sdf, float side, float tau, uint8_t *keep,
                           unsigned int *block_counts, float *out, int *n_out, cudaStream_t st) {
    if (obj.n <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((obj.n + kConcaveThreads - 1) / kConcaveThreads);
    k_concave<<<grid, kConcaveThreads, 0, st>>>(obj, sdf, side, tau, keep, block_counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_compact<<<grid, kConcaveThreads, 0, st>>>(obj, keep, block_counts, out, n_out);
    return cudaGetLastError();
}

cudaError_t launch_place_static(const float lo[3], const float hi[3], const cf_points &obj, int P, uint32_t seed_lo,
                                uint32_t seed_hi, uint32_t pose_base, float pen_margin, float *poses, int32_t *static_pt,
                                uint8_t *valid, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    StaticArgs a;
    for (int c = 0; c < 3; ++c) { a.lo[c] = lo[c]; a.hi[c] = hi[c]; }
    a.obj = obj;
    a.P = P;
    a.seed_lo = seed_lo;
    a.seed_hi = seed_hi;
    a.pose_base = pose_base;
    a.pen_margin = pen_margin;
    a.poses = poses;
    a.static_pt = static_pt;
    a.valid = valid;
    k_place_static<<<P, kStaticThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_append_contact(const int32_t *tuples, int P, int T, int k, const int32_t *first, const uint8_t *valid,
                                  int32_t *out, cudaStream_t st) {
    const long long n = (long long)P * T;
    if (n <= 0) return cudaSuccess;
    k_append_contact<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tuples, n, T, k, first, valid, out);
    return cudaGetLastError();
}

}  // namespace cf
