/*
 * CPU oracle for the Contact-Field grasp path (Lightning Grasp, arXiv 2511.07418).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct reference code that
 * the GPU library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load this file; the GPU library
 * shares no source, header, table or constant with it.
 *
 * What it computes (each function cites the passage it follows):
 *   - Philox4x32-10 counter-based generator (Salmon et al., SC'11), used to key
 *     the random choices of tuple sampling;
 *   - forward kinematics of a capsule-chain finger in FP64 (Sec. 3.1 notation,
 *     Def. "Contact Field (Point)": FK((p,n); i, q));
 *   - the sampled hand contact field as a SET of (finger, voxel cell, normal bin)
 *     codes (Sec. 4.3 "Implementation", Alg. 1, Def. "Contact Field (Hand)"),
 *     and the contact domain of an object pose as set membership of the
 *     object's contact-surface codes (p, -n) (Def. "Contact Surface
 *     Representation", Sec. 4.2 "Contact Interaction", Sec. 4.3 "Object Contact
 *     Query");
 *   - a literal brute-force existential check ("is there a field sample with the
 *     same code?") for tiny inputs;
 *   - random k-tuples of contacts from k distinct non-empty finger domains
 *     (Sec. 5.3 "Contact Domain Generation": randomly select k domains;
 *     Alg. 2 step "Random(D_i)");
 *   (the closure margin's linear programs are written out and solved in
 *   oracle/__init__.py with a library LP solver).
 *
 * Precision: kinematics, geometry and every integer decision (voxel cell,
 * normal bin, hence field codes, domain masks, reverse-lookup representatives
 * and contact codes) are FP64: the FP32 inputs are widened and the chain, the
 * transforms and the dot products are evaluated in double precision.  Beside
 * each FP64 decision the oracle keeps a tolerance band (tau metres on every
 * coordinate, bin_tol in cosine on the bin argmax) to flag the entries whose
 * decision could change under a perturbation that small: the "ambiguous"
 * entries, where a correct FP32 implementation may legitimately decide
 * otherwise.  An FP32 evaluation of the codes (orc_fk_links32 and the fmaf
 * helpers) is kept only as a diagnostic: no acceptance test relies on it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC 2011): 4x32-bit counter, 2x32-bit key, 10 rounds of    */
/* multiply-hi/lo S-boxes with a Weyl key schedule.                            */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod1;
        uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += ORC_PHILOX_W0;
        k1 += ORC_PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Forward kinematics (FP64).  Chain convention: frame_{-1} = base;           */
/* frame_j = frame_{j-1} * Trans(offset_{j-1}) * Rot(axis_j, q_j).            */
/* ------------------------------------------------------------------------ */
static void rot_axis_angle(const double a[3], double q, double R[9]) {
    /* Rodrigues: R = cos q I + sin q [a]x + (1 - cos q) a a^T */
    double c = cos(q), s = sin(q), v = 1.0 - c;
    R[0] = c + a[0] * a[0] * v;        R[1] = a[0] * a[1] * v - a[2] * s; R[2] = a[0] * a[2] * v + a[1] * s;
    R[3] = a[1] * a[0] * v + a[2] * s; R[4] = c + a[1] * a[1] * v;        R[5] = a[1] * a[2] * v - a[0] * s;
    R[6] = a[2] * a[0] * v - a[1] * s; R[7] = a[2] * a[1] * v + a[0] * s; R[8] = c + a[2] * a[2] * v;
}

static void matmul3(const double A[9], const double B[9], double C[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            C[3 * r + c] = A[3 * r + 0] * B[0 + c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

/* Link frames of one finger for one configuration q[J]:
 * Rout[J][9] (row-major), tout[J][3], both in the palm frame. */
void orc_fk_links(int J, const float *base12, const float *axis, const float *offset,
                  const double *q, double *Rout, double *tout) {
    double R[9] = {base12[0], base12[1], base12[2], base12[4], base12[5], base12[6],
                   base12[8], base12[9], base12[10]};
    double t[3] = {base12[3], base12[7], base12[11]};
    for (int j = 0; j < J; ++j) {
        if (j > 0) {
            const float *o = offset + 3 * (j - 1);
            double o0 = o[0], o1 = o[1], o2 = o[2];
            double t0 = t[0] + R[0] * o0 + R[1] * o1 + R[2] * o2;
            double t1 = t[1] + R[3] * o0 + R[4] * o1 + R[5] * o2;
            double t2 = t[2] + R[6] * o0 + R[7] * o1 + R[8] * o2;
            t[0] = t0; t[1] = t1; t[2] = t2;
        }
        double a[3] = {axis[3 * j + 0], axis[3 * j + 1], axis[3 * j + 2]};
        double Rj[9], Rn[9];
        rot_axis_angle(a, q[j], Rj);
        matmul3(R, Rj, Rn);
        memcpy(R, Rn, sizeof R);
        memcpy(Rout + 9 * j, R, sizeof R);
        memcpy(tout + 3 * j, t, sizeof t);
    }
}

/* Link frames in the decision precision: sin and cos of each joint angle in
 * FP64 rounded to FP32, then the same chain as orc_fk_links in FP32 with every
 * operation rounded (translation t + R o as nested fmaf in component order;
 * Rodrigues' Q = c I + s [a]x + v a a^T with v = 1 - c; R Q as nested fmaf). */
void orc_fk_links32(int J, const float *base12, const float *axis, const float *offset,
                    const double *q, float *Rout, float *tout) {
    float R[9] = {base12[0], base12[1], base12[2], base12[4], base12[5], base12[6],
                  base12[8], base12[9], base12[10]};
    float t[3] = {base12[3], base12[7], base12[11]};
    for (int j = 0; j < J; ++j) {
        if (j > 0) {
            const float *o = offset + 3 * (j - 1);
            for (int r = 0; r < 3; ++r)
                t[r] = fmaf(R[3 * r + 2], o[2], fmaf(R[3 * r + 1], o[1], fmaf(R[3 * r], o[0], t[r])));
        }
        const float ax = axis[3 * j + 0], ay = axis[3 * j + 1], az = axis[3 * j + 2];
        const float s = (float)sin(q[j]), c = (float)cos(q[j]);
        const float v = 1.0f - c;
        const float xs = ax * s, ys = ay * s, zs = az * s;
        const float xy = (ax * ay) * v, xz = (ax * az) * v, yz = (ay * az) * v;
        const float Q[9] = {fmaf(ax * ax, v, c), xy - zs, xz + ys,
                            xy + zs, fmaf(ay * ay, v, c), yz - xs,
                            xz - ys, yz + xs, fmaf(az * az, v, c)};
        float Rn[9];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc)
                Rn[3 * r + cc] = fmaf(R[3 * r + 2], Q[6 + cc], fmaf(R[3 * r + 1], Q[3 + cc], R[3 * r] * Q[cc]));
        memcpy(R, Rn, sizeof R);
        memcpy(Rout + 9 * j, R, sizeof R);
        memcpy(tout + 3 * j, t, sizeof t);
    }
}

/* ------------------------------------------------------------------------ */
/* FP32 decision arithmetic: single-rounding fmaf in component order x, y, z. */
/* ------------------------------------------------------------------------ */
static inline void xform_point32(const float R[9], const float t[3], const float p[3], float o[3]) {
    o[0] = fmaf(R[2], p[2], fmaf(R[1], p[1], fmaf(R[0], p[0], t[0])));
    o[1] = fmaf(R[5], p[2], fmaf(R[4], p[1], fmaf(R[3], p[0], t[1])));
    o[2] = fmaf(R[8], p[2], fmaf(R[7], p[1], fmaf(R[6], p[0], t[2])));
}

static inline void rotate32(const float R[9], const float n[3], float o[3]) {
    float m0 = R[0] * n[0], m1 = R[3] * n[0], m2 = R[6] * n[0];
    o[0] = fmaf(R[2], n[2], fmaf(R[1], n[1], m0));
    o[1] = fmaf(R[5], n[2], fmaf(R[4], n[1], m1));
    o[2] = fmaf(R[8], n[2], fmaf(R[7], n[1], m2));
}

/* cell index along one axis: floor of the exact real product x * inv_h */
static inline int64_t cell_axis(float x, float inv_h) {
    return (int64_t)floor((double)x * (double)inv_h);
}

/* normal bin: argmax_b d_b . m, first maximum wins (lowest index on ties) */
static inline int bin32(const float m[3], int B, const float *dirs) {
    int best_b = 0;
    float best = -INFINITY;
    for (int b = 0; b < B; ++b) {
        const float *d = dirs + 3 * b;
        float s = fmaf(d[2], m[2], fmaf(d[1], m[1], d[0] * m[0]));
        if (s > best) { best = s; best_b = b; }
    }
    return best_b;
}

/* Contact vectors of one (finger, sample): p32/n32 are the FP32 decision values
 * (orc_fk_links32 frames, fmaf transform), p64/n64 the FP64 values.
 * Any output pointer may be NULL. */
void orc_contact_vectors(int J, int M, const float *base12, const float *axis, const float *offset,
                         const float *surf_p, const float *surf_n, const int32_t *surf_link,
                         const double *q, float *p32, float *n32, double *p64, double *n64) {
    double R[8 * 9], t[8 * 3];
    orc_fk_links(J, base12, axis, offset, q, R, t);
    float Rf[8 * 9], tf[8 * 3];
    orc_fk_links32(J, base12, axis, offset, q, Rf, tf);
    for (int m = 0; m < M; ++m) {
        int l = surf_link[m];
        const float *ps = surf_p + 3 * m, *ns = surf_n + 3 * m;
        if (p32) xform_point32(Rf + 9 * l, tf + 3 * l, ps, p32 + 3 * m);
        if (n32) rotate32(Rf + 9 * l, ns, n32 + 3 * m);
        const double *Rl = R + 9 * l, *tl = t + 3 * l;
        for (int r = 0; r < 3; ++r) {
            if (p64) p64[3 * m + r] = tl[r] + Rl[3 * r] * ps[0] + Rl[3 * r + 1] * ps[1] + Rl[3 * r + 2] * ps[2];
            if (n64) n64[3 * m + r] = Rl[3 * r] * ns[0] + Rl[3 * r + 1] * ns[1] + Rl[3 * r + 2] * ns[2];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Field as a set of codes                                                    */
/* ------------------------------------------------------------------------ */
#define ORC_KOFF 32768
static inline int in_key_range(int64_t k) { return k > -ORC_KOFF && k < ORC_KOFF - 1; }

static inline uint64_t pack_key(int f, int64_t kx, int64_t ky, int64_t kz, int b) {
    return ((uint64_t)f << 56) | ((uint64_t)(kx + ORC_KOFF) << 40) | ((uint64_t)(ky + ORC_KOFF) << 24) |
           ((uint64_t)(kz + ORC_KOFF) << 8) | (uint64_t)b;
}

typedef struct {
    uint64_t *v;
    int64_t n, cap;
} keyvec;

static void kv_push(keyvec *kv, uint64_t key) {
    if (kv->n == kv->cap) {
        kv->cap = kv->cap ? 2 * kv->cap : 1024;
        kv->v = (uint64_t *)realloc(kv->v, (size_t)kv->cap * sizeof(uint64_t));
    }
    kv->v[kv->n++] = key;
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static void kv_sort_unique(keyvec *kv) {
    if (kv->n == 0) return;
    qsort(kv->v, (size_t)kv->n, sizeof(uint64_t), cmp_u64);
    int64_t w = 1;
    for (int64_t i = 1; i < kv->n; ++i)
        if (kv->v[i] != kv->v[w - 1]) kv->v[w++] = kv->v[i];
    kv->n = w;
}

static int kv_has(const keyvec *kv, uint64_t key) {
    int64_t lo = 0, hi = kv->n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (kv->v[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo < kv->n && kv->v[lo] == key;
}

typedef struct {
    int F, B;
    float inv_h;
    float *dirs;
    double tau, bin_tol;
    int with_band;
    keyvec *k32;   /* [F] FP32-decision codes of all samples */
    keyvec *k64;   /* [F] FP64-decision codes */
    keyvec *kpos;  /* [F] codes a sample could take within the band */
    keyvec *ksure; /* [F] codes of samples whose code is the same everywhere in the band */
    int64_t n_samples_out_of_range;
    uint32_t dil[64]; /* bins a query of bin b accepts (theta-dilated bins, Sec. 4.3 leaf test); bit b alone by default */
} orc_field;

/* does finger f's code set hold cell (kx, ky, kz) with any bin of `bins`? */
static int has_any_bin(const keyvec *kv, int f, int64_t kx, int64_t ky, int64_t kz, uint32_t bins) {
    for (; bins; bins &= bins - 1) {
        const int b = __builtin_ctz(bins);
        if (kv_has(kv, pack_key(f, kx, ky, kz, b))) return 1;
    }
    return 0;
}

/* candidate codes of a vector within the tolerance band (FP64) */
static int band_cells(double x, double tau, double inv_h, int64_t c[2]) {
    c[0] = (int64_t)floor((x - tau) * inv_h);
    c[1] = (int64_t)floor((x + tau) * inv_h);
    return c[0] == c[1] ? 1 : 2;
}

static int band_bins(const double m[3], int B, const float *dirs, double tol, int out[64]) {
    double best = -INFINITY;
    double s[256];
    for (int b = 0; b < B; ++b) {
        s[b] = dirs[3 * b] * m[0] + dirs[3 * b + 1] * m[1] + dirs[3 * b + 2] * m[2];
        if (s[b] > best) best = s[b];
    }
    int n = 0;
    for (int b = 0; b < B && n < 64; ++b)
        if (s[b] >= best - tol) out[n++] = b;
    return n;
}

/* FP64 cell index along one axis: floor(x * inv_h) of the FP64 coordinate */
static inline int64_t cell64(double x, float inv_h) { return (int64_t)floor(x * (double)inv_h); }

static int bin64(const double m[3], int B, const float *dirs) {
    int best_b = 0;
    double best = -INFINITY;
    for (int b = 0; b < B; ++b) {
        double s = dirs[3 * b] * m[0] + dirs[3 * b + 1] * m[1] + dirs[3 * b + 2] * m[2];
        if (s > best) { best = s; best_b = b; }
    }
    return best_b;
}

/* Build the sampled contact field of a hand (Sec. 4.3, Alg. 1 input: all
 * contact vectors FK((p,n); i, q_s) over sampled q_s), as code sets per finger.
 * q is [F][J][S] float32 (widened to FP64).  with_band != 0 also builds the
 * FP64 and tolerance-band sets used to count ambiguous entries. */
void *orc_field_create(int F, int J, int M, const float *base, const float *axis, const float *offset,
                       const float *surf_p, const float *surf_n, const int32_t *surf_link,
                       const float *q, int S, float inv_h, int B, const float *dirs,
                       int with_band, double tau, double bin_tol) {
    orc_field *fd = (orc_field *)calloc(1, sizeof(orc_field));
    fd->F = F; fd->B = B; fd->inv_h = inv_h;
    for (int b = 0; b < 64; ++b) fd->dil[b] = b < 32 ? 1u << b : 0u;
    fd->tau = tau; fd->bin_tol = bin_tol; fd->with_band = with_band;
    fd->dirs = (float *)malloc(sizeof(float) * 3 * B);
    memcpy(fd->dirs, dirs, sizeof(float) * 3 * B);
    fd->k32 = (keyvec *)calloc(F, sizeof(keyvec));
    fd->k64 = (keyvec *)calloc(F, sizeof(keyvec));
    fd->kpos = (keyvec *)calloc(F, sizeof(keyvec));
    fd->ksure = (keyvec *)calloc(F, sizeof(keyvec));
    int64_t oor = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : oor)
    for (int f = 0; f < F; ++f) {
        const float *bf = base + 12 * f, *af = axis + 3 * J * f, *of = offset + 3 * J * f;
        const float *spf = surf_p + 3 * M * f, *snf = surf_n + 3 * M * f;
        const int32_t *slf = surf_link + M * f;
        float *p32 = (float *)malloc(sizeof(float) * 3 * M), *n32 = (float *)malloc(sizeof(float) * 3 * M);
        double *p64 = (double *)malloc(sizeof(double) * 3 * M), *n64 = (double *)malloc(sizeof(double) * 3 * M);
        double qs[8];
        for (int s = 0; s < S; ++s) {
            for (int j = 0; j < J; ++j) qs[j] = (double)q[((size_t)f * J + j) * S + s];
            orc_contact_vectors(J, M, bf, af, of, spf, snf, slf, qs, p32, n32, p64, n64);
            for (int m = 0; m < M; ++m) {
                const double *pp = p64 + 3 * m, *nn = n64 + 3 * m;
                int64_t ex = cell64(pp[0], inv_h), ey = cell64(pp[1], inv_h), ez = cell64(pp[2], inv_h);
                if (!in_key_range(ex) || !in_key_range(ey) || !in_key_range(ez)) { ++oor; continue; }
                kv_push(&fd->k64[f], pack_key(f, ex, ey, ez, bin64(nn, B, dirs)));
                /* diagnostic: the same code decided in FP32 */
                int64_t kx = cell_axis(p32[3 * m], inv_h), ky = cell_axis(p32[3 * m + 1], inv_h),
                        kz = cell_axis(p32[3 * m + 2], inv_h);
                if (in_key_range(kx) && in_key_range(ky) && in_key_range(kz))
                    kv_push(&fd->k32[f], pack_key(f, kx, ky, kz, bin32(n32 + 3 * m, B, dirs)));
                if (!with_band) continue;
                int64_t cx[2], cy[2], cz[2];
                int nx = band_cells(pp[0], tau, inv_h, cx), ny = band_cells(pp[1], tau, inv_h, cy),
                    nz = band_cells(pp[2], tau, inv_h, cz);
                int bins[64];
                int nb = band_bins(nn, B, dirs, bin_tol, bins);
                for (int a = 0; a < nx; ++a)
                    for (int c = 0; c < ny; ++c)
                        for (int d = 0; d < nz; ++d)
                            for (int e = 0; e < nb; ++e)
                                kv_push(&fd->kpos[f], pack_key(f, cx[a], cy[c], cz[d], bins[e]));
                if (nx == 1 && ny == 1 && nz == 1 && nb == 1)
                    kv_push(&fd->ksure[f], pack_key(f, cx[0], cy[0], cz[0], bins[0]));
            }
        }
        kv_sort_unique(&fd->k32[f]);
        kv_sort_unique(&fd->k64[f]);
        kv_sort_unique(&fd->kpos[f]);
        kv_sort_unique(&fd->ksure[f]);
        free(p32); free(n32); free(p64); free(n64);
    }
    fd->n_samples_out_of_range = oor;
    return fd;
}

/* theta-dilated bins: a query of bin b hits when the cell holds any bin of dil[b] */
void orc_field_set_dilation(void *h, const uint32_t *dil) {
    orc_field *fd = (orc_field *)h;
    for (int b = 0; b < fd->B; ++b) fd->dil[b] = dil ? (dil[b] | (1u << b)) : (1u << b);
}

void orc_field_free(void *h) {
    orc_field *fd = (orc_field *)h;
    if (!fd) return;
    for (int f = 0; f < fd->F; ++f) {
        free(fd->k32[f].v); free(fd->k64[f].v); free(fd->kpos[f].v); free(fd->ksure[f].v);
    }
    free(fd->k32); free(fd->k64); free(fd->kpos); free(fd->ksure); free(fd->dirs);
    free(fd);
}

/* number of distinct (cell, bin) codes per finger (FP64 decisions) */
void orc_field_sizes(const void *h, int64_t *n_codes) {
    const orc_field *fd = (const orc_field *)h;
    for (int f = 0; f < fd->F; ++f) n_codes[f] = fd->k64[f].n;
}

/* copy one of finger f's sorted code sets: which = 0 FP32 decisions, 1 FP64
 * decisions, 2 codes some sample could take within the band (possible), 3 codes
 * of samples whose code is the same everywhere in the band (sure).  Sets 1-3
 * need with_band; returns the set's size, or -1 if it was not built. */
int64_t orc_field_code_set(const void *h, int f, int which, uint64_t *out, int64_t cap) {
    const orc_field *fd = (const orc_field *)h;
    const keyvec *kv = which == 0 ? &fd->k32[f] : which == 1 ? &fd->k64[f] : which == 2 ? &fd->kpos[f]
                     : which == 3 ? &fd->ksure[f] : NULL;
    if (!kv || (which >= 2 && !fd->with_band)) return -1;
    int64_t n = kv->n < cap ? kv->n : cap;
    if (n > 0) memcpy(out, kv->v, (size_t)n * sizeof(uint64_t));
    return kv->n;
}

/* Contact domains (Sec. 4.2: CF(H) intersected with S(O); Sec. 4.3 object
 * contact query).  For pose i = (R_i, t_i) (object -> palm) and object point x
 * with outward normal n_x, the contact-surface vector is (R p_x + t, -(R n_x))
 * (Def. "Contact Surface Representation" flips the normal), evaluated in FP64.
 * Bit x of masks[i][f] is set iff finger f's FP64 code set contains its FP64
 * (cell, bin) code (or, with theta-dilated bins, the cell with any accepted bin).
 * soa is [6][N] (px,py,pz,nx,ny,nz); poses [P][12] row-major (R | t).
 * masks [P][F][W] with W = ceil(N/32), bit (x & 31) of word x >> 5; counts are
 * the row popcounts.  Optional outputs (NULL to skip):
 *   amb    [P][F][N] uint8 (needs with_band): 1 if the decision is not the same
 *          everywhere within the tolerance band (tau metres on the query point
 *          and on the field samples, bin_tol in cosine);
 *   mask32 [P][F][W]: diagnostic, the decisions taken in FP32 on both sides. */
void orc_query_masks(const void *h, int N, const float *soa, int P, const float *poses,
                     uint32_t *masks, uint32_t *counts, uint8_t *amb, uint32_t *mask32) {
    const orc_field *fd = (const orc_field *)h;
    const int F = fd->F, B = fd->B, W = (N + 31) / 32;
    const float inv_h = fd->inv_h;
    const double tau = fd->tau;
    if (amb && !fd->with_band) amb = NULL;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < P; ++i) {
        const float *T = poses + 12 * i;
        const float R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
        const float t[3] = {T[3], T[7], T[11]};
        uint32_t *mrow = masks + (size_t)i * F * W;
        memset(mrow, 0, sizeof(uint32_t) * F * W);
        if (mask32) memset(mask32 + (size_t)i * F * W, 0, sizeof(uint32_t) * F * W);
        for (int x = 0; x < N; ++x) {
            const float p[3] = {soa[x], soa[N + x], soa[2 * N + x]};
            const float n[3] = {soa[3 * N + x], soa[4 * N + x], soa[5 * N + x]};
            double p64[3], m64[3];
            for (int r = 0; r < 3; ++r) {
                p64[r] = (double)t[r] + (double)R[3 * r] * p[0] + (double)R[3 * r + 1] * p[1] + (double)R[3 * r + 2] * p[2];
                m64[r] = -((double)R[3 * r] * n[0] + (double)R[3 * r + 1] * n[1] + (double)R[3 * r + 2] * n[2]);
            }
            const int64_t ex = cell64(p64[0], inv_h), ey = cell64(p64[1], inv_h), ez = cell64(p64[2], inv_h);
            const int b64 = bin64(m64, B, fd->dirs);
            const int ok64 = in_key_range(ex) && in_key_range(ey) && in_key_range(ez);
            for (int f = 0; f < F; ++f)
                if (ok64 && has_any_bin(&fd->k64[f], f, ex, ey, ez, fd->dil[b64]))
                    mrow[(size_t)f * W + (x >> 5)] |= 1u << (x & 31);
            if (mask32) {  /* diagnostic: FP32 decisions on both sides */
                float pq[3], nq[3];
                xform_point32(R, t, p, pq);
                rotate32(R, n, nq);
                const float mq[3] = {-nq[0], -nq[1], -nq[2]};
                const int64_t kx = cell_axis(pq[0], inv_h), ky = cell_axis(pq[1], inv_h), kz = cell_axis(pq[2], inv_h);
                const int ok = in_key_range(kx) && in_key_range(ky) && in_key_range(kz);
                const int b = bin32(mq, B, fd->dirs);
                for (int f = 0; f < F; ++f)
                    if (ok && has_any_bin(&fd->k32[f], f, kx, ky, kz, fd->dil[b]))
                        mask32[((size_t)i * F + f) * W + (x >> 5)] |= 1u << (x & 31);
            }
            if (!amb) continue;
            int64_t cx[2], cy[2], cz[2];
            int nx = band_cells(p64[0], tau, inv_h, cx), ny = band_cells(p64[1], tau, inv_h, cy),
                nz = band_cells(p64[2], tau, inv_h, cz);
            int bins[64];
            int nb = band_bins(m64, B, fd->dirs, fd->bin_tol, bins);
            for (int f = 0; f < F; ++f) {
                int possible = 0, sure = 1;
                for (int a = 0; a < nx; ++a)
                    for (int c = 0; c < ny; ++c)
                        for (int d = 0; d < nz; ++d)
                            for (int e = 0; e < nb; ++e) {
                                int rng_ok = in_key_range(cx[a]) && in_key_range(cy[c]) && in_key_range(cz[d]);
                                const uint32_t acc = fd->dil[bins[e]];
                                if (rng_ok && has_any_bin(&fd->kpos[f], f, cx[a], cy[c], cz[d], acc)) possible = 1;
                                if (!rng_ok || !has_any_bin(&fd->ksure[f], f, cx[a], cy[c], cz[d], acc)) sure = 0;
                            }
                amb[((size_t)i * F + f) * N + x] = (uint8_t)(possible != sure);
            }
        }
        for (int f = 0; f < F; ++f) {
            uint32_t c = 0;
            for (int w = 0; w < W; ++w) c += (uint32_t)__builtin_popcount(mrow[(size_t)f * W + w]);
            counts[(size_t)i * F + f] = c;
        }
    }
}

/* Literal existential check for tiny inputs: bit x of mask[i][f] is set iff
 * SOME field sample (s, m) of finger f has the same cell as the contact-surface
 * vector of point x under pose i and a bin that query accepts (the same bin, or
 * one of dil[bin] with theta-dilated bins; dil may be NULL).  No index, no
 * sorting. */
void orc_query_masks_brute(int F, int J, int M, const float *base, const float *axis, const float *offset,
                           const float *surf_p, const float *surf_n, const int32_t *surf_link,
                           const float *q, int S, float inv_h, int B, const float *dirs,
                           int N, const float *soa, int P, const float *poses, const uint32_t *dil,
                           uint32_t *masks) {
    const int W = (N + 31) / 32;
    memset(masks, 0, sizeof(uint32_t) * (size_t)P * F * W);
    if (M > 128 || J > 8) return;
    /* per (f, s, m) codes of the samples, recomputed from FK */
    int64_t *scode = (int64_t *)malloc(sizeof(int64_t) * 4 * (size_t)F * S * M);
    for (int f = 0; f < F; ++f) {
        double p64[3 * 128], n64[3 * 128];
        double qs[8];
        for (int s = 0; s < S; ++s) {
            for (int j = 0; j < J; ++j) qs[j] = (double)q[((size_t)f * J + j) * S + s];
            orc_contact_vectors(J, M, base + 12 * f, axis + 3 * J * f, offset + 3 * J * f, surf_p + 3 * M * f,
                                surf_n + 3 * M * f, surf_link + M * f, qs, NULL, NULL, p64, n64);
            for (int m = 0; m < M; ++m) {
                int64_t *c = scode + 4 * (((size_t)f * S + s) * M + m);
                c[0] = cell64(p64[3 * m], inv_h);
                c[1] = cell64(p64[3 * m + 1], inv_h);
                c[2] = cell64(p64[3 * m + 2], inv_h);
                c[3] = bin64(n64 + 3 * m, B, dirs);
            }
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < P; ++i) {
        const float *T = poses + 12 * i;
        const float R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
        const float t[3] = {T[3], T[7], T[11]};
        for (int x = 0; x < N; ++x) {
            const float p[3] = {soa[x], soa[N + x], soa[2 * N + x]};
            const float n[3] = {soa[3 * N + x], soa[4 * N + x], soa[5 * N + x]};
            double pq[3], mq[3];
            for (int r = 0; r < 3; ++r) {
                pq[r] = (double)t[r] + (double)R[3 * r] * p[0] + (double)R[3 * r + 1] * p[1] + (double)R[3 * r + 2] * p[2];
                mq[r] = -((double)R[3 * r] * n[0] + (double)R[3 * r + 1] * n[1] + (double)R[3 * r + 2] * n[2]);
            }
            int64_t qc[4] = {cell64(pq[0], inv_h), cell64(pq[1], inv_h), cell64(pq[2], inv_h), bin64(mq, B, dirs)};
            const uint32_t acc = dil ? (dil[qc[3]] | (1u << qc[3])) : (1u << qc[3]);
            for (int f = 0; f < F; ++f) {
                const int64_t *c = scode + 4 * (size_t)f * S * M;
                for (int64_t e = 0; e < (int64_t)S * M; ++e, c += 4) {
                    if (c[0] == qc[0] && c[1] == qc[1] && c[2] == qc[2] && ((acc >> c[3]) & 1u)) {
                        masks[((size_t)i * F + f) * W + (x >> 5)] |= 1u << (x & 31);
                        break;
                    }
                }
            }
        }
    }
    free(scode);
}

/* ------------------------------------------------------------------------ */
/* Tuple sampling (Sec. 5.3: randomly select k contact domains of distinct    */
/* fingers; Alg. 2: (p_i, n_i) <- Random(D_i)).                               */
/* Draw d of tuple (i, tau) is word (d mod 4) of Philox4x32-10 with counter   */
/* (i, tau, d div 4, 0) and key (seed lo, seed hi).  A uniform integer in     */
/* [0, m) is floor(u * m / 2^32).  Fingers: partial Fisher-Yates over the     */
/* non-empty fingers in ascending order with draws 0..k-1; point of chosen    */
/* finger d: the r-th set bit (ascending) of its mask row, r from draw k + d. */
/* Fewer than k non-empty fingers: tuple ids -1, finger ids 255.             */
/* ------------------------------------------------------------------------ */
static void tuple_draws(uint64_t seed, uint32_t i, uint32_t tau, int ndraw, uint32_t *u) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int blk = 0; 4 * blk < ndraw; ++blk) {
        uint32_t ctr[4] = {i, tau, (uint32_t)blk, 0u}, out[4];
        orc_philox4x32_10(ctr, key, out);
        for (int w = 0; w < 4 && 4 * blk + w < ndraw; ++w) u[4 * blk + w] = out[w];
    }
}

static int32_t select_set_bit(const uint32_t *row, int W, uint32_t r) {
    for (int w = 0; w < W; ++w) {
        uint32_t v = row[w];
        uint32_t c = (uint32_t)__builtin_popcount(v);
        if (r < c) {
            for (int b = 0; b < 32; ++b)
                if (v >> b & 1u) {
                    if (r == 0) return 32 * w + b;
                    --r;
                }
        }
        r -= c;
    }
    return -1;
}

void orc_sample_tuples(int P, int F, int N, const uint32_t *masks, const uint32_t *counts, int T, int k,
                       uint64_t seed, int32_t *tuples, uint8_t *fingers) {
    const int W = (N + 31) / 32;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < P; ++i) {
        int nonempty[32], m = 0;
        for (int f = 0; f < F; ++f)
            if (counts[(size_t)i * F + f] > 0) nonempty[m++] = f;
        for (int tau = 0; tau < T; ++tau) {
            int32_t *tp = tuples + ((size_t)i * T + tau) * k;
            uint8_t *fp = fingers + ((size_t)i * T + tau) * k;
            if (m < k) {
                for (int d = 0; d < k; ++d) { tp[d] = -1; fp[d] = 255; }
                continue;
            }
            uint32_t u[64];
            tuple_draws(seed, (uint32_t)i, (uint32_t)tau, 2 * k, u);
            int idx[32];
            memcpy(idx, nonempty, sizeof(int) * m);
            for (int d = 0; d < k; ++d) {
                int j = d + (int)(((uint64_t)u[d] * (uint64_t)(m - d)) >> 32);
                int tmp = idx[d]; idx[d] = idx[j]; idx[j] = tmp;
            }
            for (int d = 0; d < k; ++d) {
                int f = idx[d];
                uint32_t cnt = counts[(size_t)i * F + f];
                uint32_t r = (uint32_t)(((uint64_t)u[k + d] * (uint64_t)cnt) >> 32);
                tp[d] = select_set_bit(masks + ((size_t)i * F + f) * W, W, r);
                fp[d] = (uint8_t)f;
            }
        }
    }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* OpenMP threads of the following calls (for a single-core timing) */
void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Reverse lookup (Sec. 5.5 "Kinematics Optimization")                       */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; uint32_t val; } keyval;

static int cmp_keyval(const void *a, const void *b) {
    const keyval *x = (const keyval *)a, *y = (const keyval *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->val < y->val ? -1 : (x->val > y->val);
}

/* For every FP64 (cell, bin) code of finger f: the smallest s * M + m over the
 * field samples (joint sample s, surface point m in the caller's order) whose
 * contact vector has that code -- the sample the reverse lookup retrieves.
 * Writes up to cap (packed key, value) pairs sorted by key; returns the number
 * of distinct codes.  sure (optional, [cap]) flags the representatives no
 * perturbation within the band (tau metres, bin_tol in cosine) can change:
 * no sample with a smaller index takes the code anywhere in its band, and the
 * representative's own code is the same everywhere in its band. */
int64_t orc_rep_codes(int F, int J, int M, const float *base, const float *axis, const float *offset,
                      const float *surf_p, const float *surf_n, const int32_t *surf_link, const float *q, int S,
                      float inv_h, int B, const float *dirs, int f, double tau, double bin_tol,
                      uint64_t *keys, uint32_t *vals, uint8_t *sure, int64_t cap) {
    (void)F;
    const float *bf = base + 12 * f, *af = axis + 3 * J * f, *of = offset + 3 * J * f;
    const float *spf = surf_p + 3 * M * f, *snf = surf_n + 3 * M * f;
    const int32_t *slf = surf_link + M * f;
    keyval *kv = (keyval *)malloc(sizeof(keyval) * (size_t)S * M + 1);
    uint8_t *exact = (uint8_t *)malloc((size_t)S * M + 1); /* [s*M+m]: the sample's code is band-stable */
    int64_t pcap = 16 * (int64_t)S * M / 8 + 1024, np_ = 0; /* band codes of all samples (grown as needed) */
    keyval *pk = (keyval *)malloc(sizeof(keyval) * (size_t)pcap);
    double *p64 = (double *)malloc(sizeof(double) * 3 * M), *n64 = (double *)malloc(sizeof(double) * 3 * M);
    int64_t n = 0;
    double qs[8];
    for (int s = 0; s < S; ++s) {
        for (int j = 0; j < J; ++j) qs[j] = (double)q[((size_t)f * J + j) * S + s];
        orc_contact_vectors(J, M, bf, af, of, spf, snf, slf, qs, NULL, NULL, p64, n64);
        for (int m = 0; m < M; ++m) {
            const double *pp = p64 + 3 * m, *nn = n64 + 3 * m;
            const uint32_t val = (uint32_t)s * (uint32_t)M + (uint32_t)m;
            int64_t kx = cell64(pp[0], inv_h), ky = cell64(pp[1], inv_h), kz = cell64(pp[2], inv_h);
            exact[val] = 0;
            if (!in_key_range(kx) || !in_key_range(ky) || !in_key_range(kz)) continue;
            kv[n].key = pack_key(f, kx, ky, kz, bin64(nn, B, dirs));
            kv[n].val = val;
            ++n;
            if (!sure) continue;
            int64_t cx[2], cy[2], cz[2];
            int bins[64];
            const int nx = band_cells(pp[0], tau, inv_h, cx), ny = band_cells(pp[1], tau, inv_h, cy),
                      nz = band_cells(pp[2], tau, inv_h, cz), nb = band_bins(nn, B, dirs, bin_tol, bins);
            exact[val] = (uint8_t)(nx * ny * nz * nb == 1);
            for (int a = 0; a < nx; ++a)
                for (int c = 0; c < ny; ++c)
                    for (int d = 0; d < nz; ++d)
                        for (int e = 0; e < nb; ++e) {
                            if (!in_key_range(cx[a]) || !in_key_range(cy[c]) || !in_key_range(cz[d])) continue;
                            if (np_ == pcap) {
                                pcap *= 2;
                                pk = (keyval *)realloc(pk, sizeof(keyval) * (size_t)pcap);
                            }
                            pk[np_].key = pack_key(f, cx[a], cy[c], cz[d], bins[e]);
                            pk[np_].val = val;
                            ++np_;
                        }
        }
    }
    qsort(kv, (size_t)n, sizeof(keyval), cmp_keyval);
    if (sure) qsort(pk, (size_t)np_, sizeof(keyval), cmp_keyval);
    int64_t u = 0, ip = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (i > 0 && kv[i].key == kv[i - 1].key) continue;  /* first of each key = smallest value */
        if (u < cap) {
            keys[u] = kv[i].key;
            vals[u] = kv[i].val;
            if (sure) {
                while (ip < np_ && pk[ip].key < kv[i].key) ++ip;  /* first band entry of this key: its smallest value */
                sure[u] = (uint8_t)(ip < np_ && pk[ip].key == kv[i].key && pk[ip].val == kv[i].val && exact[kv[i].val]);
            }
        }
        ++u;
    }
    free(kv); free(pk); free(exact); free(p64); free(n64);
    return u;
}

/* FP64 (cell, bin) code of the contact-surface vector of point pt[i] under pose
 * pose[i] (the domain query's decision): out[i] = (kx, ky, kz, bin).  amb
 * (optional) flags the points whose code is not the same everywhere within the
 * band (tau metres, bin_tol in cosine). */
void orc_point_codes(int N, const float *soa, const float *poses, int n, const int32_t *pose_idx,
                     const int32_t *pt_idx, float inv_h, int B, const float *dirs, double tau, double bin_tol,
                     int64_t *out, uint8_t *amb) {
    for (int i = 0; i < n; ++i) {
        const float *T = poses + 12 * (size_t)pose_idx[i];
        const float R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
        const float t[3] = {T[3], T[7], T[11]};
        const int x = pt_idx[i];
        const float p[3] = {soa[x], soa[N + x], soa[2 * N + x]};
        const float nv[3] = {soa[3 * N + x], soa[4 * N + x], soa[5 * N + x]};
        double pq[3], mq[3];
        for (int r = 0; r < 3; ++r) {
            pq[r] = (double)t[r] + (double)R[3 * r] * p[0] + (double)R[3 * r + 1] * p[1] + (double)R[3 * r + 2] * p[2];
            mq[r] = -((double)R[3 * r] * nv[0] + (double)R[3 * r + 1] * nv[1] + (double)R[3 * r + 2] * nv[2]);
        }
        out[4 * i] = cell64(pq[0], inv_h);
        out[4 * i + 1] = cell64(pq[1], inv_h);
        out[4 * i + 2] = cell64(pq[2], inv_h);
        out[4 * i + 3] = bin64(mq, B, dirs);
        if (amb) {
            int64_t c[2];
            int bins[64];
            amb[i] = (uint8_t)(band_cells(pq[0], tau, inv_h, c) * band_cells(pq[1], tau, inv_h, c) *
                                   band_cells(pq[2], tau, inv_h, c) * band_bins(mq, B, dirs, bin_tol, bins) != 1);
        }
    }
}
