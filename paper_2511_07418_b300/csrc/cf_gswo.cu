// The paper's own grasp metric (Eq. GSWO, Sec. 3.2) with true quadratic
// friction cones: for each subproblem j (alpha_j = 1), minimise |A z|^2 over
// z = (alpha_i, bx_i, by_i)_i with |b_j| <= mu and |b_i| <= mu alpha_i (i != j),
// where column block i of A is [nu_i x_i y_i ; r_i x (nu_i, x_i, y_i) / rho],
// nu_i = -n_i, (x_i, y_i) its Duff et al. 2017 basis, r_i = p_i - c; the tuple's
// value is min_j.  Solved as the paper says, by projected gradient descent --
// here with Nesterov momentum (FISTA), a fixed number of steps of size
// 1 / (2 tr(A^T A)) from alpha = e_j, beta = 0.
//
// Launch: lanes in groups of k (32 / k tuples per warp); lane c of a group
// solves subproblem j = c of its tuple entirely in registers (Q = A^T A, the
// iterate, the momentum point); the group's minimum is a shuffle reduction.
#include "cf_internal.cuh"

namespace cf {

namespace {

constexpr int kGswoThreads = 128;

struct GswoArgs {
    const float *px, *py, *pz, *nx, *ny, *nz;
    int N;
    long long n;         // tuples
    int k;
    float mu, cx, cy, cz, inv_rho, eps;
    int n_iter;
    const float *beta;   // [n_iter] momentum coefficients (t_k - 1) / t_{k+1}, from the host in FP64
    const int32_t *tuples;
    float *value;
    uint8_t *accept;
};

// Projection of (a, b1, b2) onto |b| <= mu a, a >= 0, without branches: inside
// the cone the point stays, inside the polar cone it goes to 0, otherwise to
// a' = (a + mu s) / (1 + mu^2), b' = (mu a' / s) b.  inv1m = 1 / (1 + mu^2).  At
// mu = 0 the cone is the ray b = 0, a >= 0 (a frictionless contact, Eq. FSWO),
// so a point with b = 0 is inside only when a >= 0.
__device__ __forceinline__ void project_soc(float &a, float &b1, float &b2, float mu, float inv1m) {
    const float s2 = b1 * b1 + b2 * b2;
    const float s = sqrtf(s2);
    const bool inside = a >= 0.f && s <= mu * a, polar = mu * s <= -a;
    const float a2 = (a + mu * s) * inv1m;
    const float f = mu * a2 * rsqrtf(fmaxf(s2, 1e-30f));
    const float fa = inside ? a : (polar ? 0.f : a2);
    const float fb = inside ? 1.f : (polar ? 0.f : f);
    a = fa; b1 *= fb; b2 *= fb;
}

template <int K>
__global__ void __launch_bounds__(kGswoThreads) k_gswo(const GswoArgs g) {
    constexpr int V = 3 * K;
    constexpr int G = 32 / K;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int grp = lane / K, j = lane - grp * K;
    const long long u = warp * G + grp;
    const bool live = grp < G && u < g.n;
    bool valid = live;
    int ids[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        ids[i] = live ? __ldg(g.tuples + u * K + i) : 0;
        valid = valid && ids[i] >= 0 && ids[i] < g.N;
    }
    float J = INFINITY;
    if (valid) {
        // A column by column (6 rows), then Q = A^T A (upper triangle)
        float A[6][V];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int x = ids[i];
            const float vx = -__ldg(g.nx + x), vy = -__ldg(g.ny + x), vz = -__ldg(g.nz + x);
            const float sgn = copysignf(1.f, vz);
            const float aa = -1.f / (sgn + vz);
            const float bb = vx * vy * aa;
            const float d[3][3] = {{vx, vy, vz},
                                   {1.f + sgn * vx * vx * aa, sgn * bb, -sgn * vx},
                                   {bb, sgn + vy * vy * aa, -vy}};
            const float rx = __ldg(g.px + x) - g.cx, ry = __ldg(g.py + x) - g.cy, rz = __ldg(g.pz + x) - g.cz;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                A[0][3 * i + c] = d[c][0];
                A[1][3 * i + c] = d[c][1];
                A[2][3 * i + c] = d[c][2];
                A[3][3 * i + c] = (ry * d[c][2] - rz * d[c][1]) * g.inv_rho;
                A[4][3 * i + c] = (rz * d[c][0] - rx * d[c][2]) * g.inv_rho;
                A[5][3 * i + c] = (rx * d[c][1] - ry * d[c][0]) * g.inv_rho;
            }
        }
        float Q[V][V];
        float tr = 0.f;
#pragma unroll
        for (int a = 0; a < V; ++a)
#pragma unroll
            for (int b = a; b < V; ++b) {
                float s = 0.f;
#pragma unroll
                for (int r = 0; r < 6; ++r) s = fmaf(A[r][a], A[r][b], s);
                Q[a][b] = s;
                Q[b][a] = s;
                if (a == b) tr += s;
            }
        const float step2 = 2.f * (1.f / (2.f * tr));  // gradient 2 Q y times the step 1 / (2 tr)
        float z[V], y[V];
#pragma unroll
        for (int v = 0; v < V; ++v) z[v] = y[v] = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i)
            if (i == j) z[3 * i] = y[3 * i] = 1.f;
        const float mu = g.mu, inv1m = 1.f / (1.f + g.mu * g.mu);
        for (int it = 0; it < g.n_iter; ++it) {
            float zn[V];
#pragma unroll
            for (int a = 0; a < V; ++a) {
                float s = 0.f;
#pragma unroll
                for (int b = 0; b < V; ++b) s = fmaf(Q[a][b], y[b], s);
                zn[a] = y[a] - step2 * s;
            }
#pragma unroll
            for (int i = 0; i < K; ++i) {
                // contact j: alpha_j = 1, friction in the disc |b| <= mu; the others: the cone
                float a = zn[3 * i], b1 = zn[3 * i + 1], b2 = zn[3 * i + 2];
                project_soc(a, b1, b2, mu, inv1m);
                const float s2 = zn[3 * i + 1] * zn[3 * i + 1] + zn[3 * i + 2] * zn[3 * i + 2];
                const float fd = fminf(1.f, mu * rsqrtf(fmaxf(s2, 1e-30f)));
                const bool mine = i == j;
                zn[3 * i] = mine ? 1.f : a;
                zn[3 * i + 1] = mine ? zn[3 * i + 1] * fd : b1;
                zn[3 * i + 2] = mine ? zn[3 * i + 2] * fd : b2;
            }
            const float beta = __ldg(g.beta + it);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                y[v] = zn[v] + beta * (zn[v] - z[v]);
                z[v] = zn[v];
            }
        }
        // J_j = |A z|^2
        J = 0.f;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            float s = 0.f;
#pragma unroll
            for (int v = 0; v < V; ++v) s = fmaf(A[r][v], z[v], s);
            J = fmaf(s, s, J);
        }
    }
    // min over the group's subproblems
    float m = J;
#pragma unroll
    for (int c = 1; c < K; ++c) {
        const int src = min(grp * K + c, 31);
        const float o = __shfl_sync(full, J, src);
        if (j == 0) m = fminf(m, o);
    }
    if (live && j == 0) {
        g.value[u] = m;
        g.accept[u] = (uint8_t)(m <= g.eps);
    }
}

}  // namespace

cudaError_t launch_gswo(const float *const pts[6], int N, long long n, int k, float mu, const float c[3], float rho,
                        float eps, int n_iter, const float *beta, const int32_t *tuples, float *value, uint8_t *accept,
                        cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    GswoArgs g{pts[0], pts[1], pts[2], pts[3], pts[4], pts[5], N, n, k, mu, c[0], c[1], c[2], 1.f / rho, eps, n_iter,
               beta, tuples, value, accept};
    const long long per_warp = 32 / k;
    const long long warps = (n + per_warp - 1) / per_warp;
    const unsigned blocks = (unsigned)((warps * 32 + kGswoThreads - 1) / kGswoThreads);
    switch (k) {
        case 2: k_gswo<2><<<blocks, kGswoThreads, 0, st>>>(g); break;
        case 3: k_gswo<3><<<blocks, kGswoThreads, 0, st>>>(g); break;
        case 4: k_gswo<4><<<blocks, kGswoThreads, 0, st>>>(g); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace cf
