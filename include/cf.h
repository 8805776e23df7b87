/*
 * cf.h -- C ABI of libcf, the Contact-Field grasp hot path of Lightning Grasp
 * (Yin & Abbeel, arXiv 2511.07418) for one NVIDIA B300 (sm_103a).
 *
 * Three steps, each a call below:
 *   cf_build          sampled contact field of a hand: forward kinematics of the
 *                     hand surface over joint samples, binned into a voxel x
 *                     normal-bin bit table            (Def. Contact Field (Point),
 *                     Def. Contact Field (Hand), Sec. 4.3 Implementation, Alg. 1)
 *   cf_query_domains  contact domains of an object over many palm poses, as
 *                     per-finger bitmasks             (Def. Contact Surface
 *                     Representation, Sec. 4.2, Sec. 4.3 Object Contact Query)
 *   cf_score_tuples   random contact k-tuples from k distinct finger domains and
 *                     their linearised friction-cone closure margin
 *                                                     (Sec. 5.3, Alg. 2 Random(D_i),
 *                     Eq. GSWO of Sec. 3.2)
 * plus cf_plan_*, the same path driven from host buffers (one object request).
 *
 * Conventions
 *  - Every call returns CF_OK (0) or a CF_E* code; cf_last_error() gives a
 *    thread-local message.  Nothing throws across the ABI.
 *  - "d_" pointers are device pointers owned by the caller; libcf never frees
 *    them.  "host" pointers are read during the call only.
 *  - Handles (cf_field, cf_plan) are owned by the library and freed by their
 *    destroy call.
 *  - Work is queued on the caller's CUDA stream (cf_stream = cudaStream_t, NULL
 *    = legacy default stream).  cf_build waits once on that stream (for the
 *    table's extents) and returns with its last kernel queued;
 *    cf_plan_run_host and cf_plan_run_host_accepted synchronise the stream;
 *    the other calls do not.
 *  - Device memory the library owns comes from a per-device stream-ordered
 *    pool that keeps freed blocks for reuse.
 *  - Shapes are checked on the host (CF_EINVAL); a kernel that meets a
 *    condition it cannot honour (an LP that exceeds its pivot cap) sets a bit in
 *    a device status word read by cf_device_status().
 *  - Geometry is FP32, metres.  Row-major 3x4 rigid transforms [R | t].
 */
#ifndef CF_H
#define CF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CF_MAX_FINGERS 8
#define CF_MAX_SLOTS 16   /* table slots: one per finger, or one per (finger, link) patch */
#define CF_MAX_JOINTS 8
#define CF_MAX_SURF 256
#define CF_MAX_BINS 32
#define CF_MAX_K 4        /* contacts per tuple */
#define CF_MAX_EDGES 16   /* friction-pyramid edges; k * K <= 32 */

enum {
    CF_OK = 0,
    CF_EINVAL = 1,   /* bad argument / shape */
    CF_ENOMEM = 2,   /* device or host allocation failed */
    CF_ECUDA = 3,    /* a CUDA runtime call failed (message has the CUDA error) */
    CF_ETIMEOUT = 4, /* a bounded wait ran out (cf_engine_drain's host-side limit; no kernel waits) */
    CF_EBUSY = 5,    /* resource in use */
    CF_EDEVICE = 6,  /* device status word reported a kernel-side condition */
    CF_EIO = 7       /* file read / write failed */
};

/* device status bits (cf_device_status) */
#define CF_DEV_LP_PIVOT_CAP 0x1u   /* an LP stopped at its pivot cap; its margin is an upper bound */
#define CF_DEV_LP_UNBOUNDED 0x2u   /* reserved (the scaled LP reads an unbounded ratio test as margin 0) */
#define CF_DEV_REP_FULL 0x4u       /* the representative table had no free slot (cannot happen at load <= 1/2) */
#define CF_DEV_REP_MISS 0x8u       /* an IK contact's code has no representative (tuple not from this field) */
#define CF_DEV_BIN_RANGE 0x80000000u /* a build sample fell outside the table box (cannot happen) */

typedef void *cf_stream; /* cudaStream_t */

/* Hand: F fingers, each a serial chain of J revolute joints (host arrays).
 * frame_{-1} = base[f]; frame_j = frame_{j-1} * Trans(offset[f][j-1]) *
 * Rot(axis[f][j], q_j).  Surface point m of finger f lies on link
 * surf_link[f][m] at surf_p[f][m] with outward normal surf_n[f][m], both in that
 * link's frame (the hand-surface points of Def. Contact Field (Hand)). */
typedef struct cf_hand_desc {
    int32_t n_fingers;        /* F, 1..CF_MAX_FINGERS */
    int32_t n_joints;         /* J, 1..CF_MAX_JOINTS */
    int32_t n_surf;           /* M, 1..CF_MAX_SURF */
    const float *base;        /* [F][12] row-major (R | t), palm frame */
    const float *axis;        /* [F][J][3] unit joint axes */
    const float *offset;      /* [F][J][3] link vectors */
    const float *surf_p;      /* [F][M][3] */
    const float *surf_n;      /* [F][M][3] */
    const int32_t *surf_link; /* [F][M], 0..J-1 */
    const float *lo, *hi;     /* [F][J] joint limits (rad); NULL: the field cannot drive IK / realization */
    const float *radius;      /* [F][J] capsule radius of link j (0 for a zero-length link) */
} cf_hand_desc;

/* Field parameters.  Cells live on one global lattice: cell k covers
 * [k / inv_h, (k + 1) / inv_h) per axis, k = floor(x * inv_h) of the exact
 * product.  Normal bin of a unit vector v = argmax_b bin_dirs[b] . v (first
 * maximum), the fixed direction set of Sec. 4.4 "Memory Consumption". */
typedef struct cf_field_params {
    float inv_h;              /* 1 / voxel edge, cells per metre (> 0) */
    int32_t n_bins;           /* B, 1..CF_MAX_BINS */
    const float *bin_dirs;    /* host [B][3] */
    int32_t want_rep;         /* 1: also keep, per (cell, finger, bin) code, the smallest s * M + m of the
                                 samples that produced it (reverse lookup, Sec. 5.5) */
    float dilate_deg;         /* theta-dilated bins (the leaf test -x^T n >= theta_hit of Sec. 4.3): a query
                                 of bin b accepts every bin b' with d_b . d_b' >= cos(dilate_deg * (pi / 180))
                                 (FP64 on the host); 0 = the same bin only */
    int32_t patches;          /* 0: one table slot per finger; 1: the fine-grained field of Sec. 4.4 ("break
                                 down the whole hand surface into m patches, and compute the contact field for
                                 each patch"), a patch being the surface points of one link of one finger: one
                                 slot per (finger, link with surface points), fingers in order, links
                                 ascending, at most CF_MAX_SLOTS; the query then returns per-patch domains,
                                 which cf_merge_domains combines per finger.  Not with want_rep. */
} cf_field_params;

typedef struct cf_field cf_field;

/* Table layout: one box of cells covering every finger's samples.  Cell
 * (x, y, z) of the box (x fastest) owns a record of record_words uint32 words;
 * slot s's normal-bin set is bits [(s % fingers_per_word) * bits_per_finger,
 * + n_bins) of word s / fingers_per_word of the record.  Slot s holds the
 * samples of finger slot_finger[s] (link slot_link[s] in a patch field, -1:
 * every link). */
typedef struct cf_field_info {
    int32_t n_fingers, n_joints, n_surf, n_bins, n_samples;
    float inv_h;
    int32_t box_lo[3];                 /* first cell of the box, per axis */
    int32_t box_dims[3];               /* cells per axis (0 when the field is empty) */
    int32_t bits_per_finger;           /* 8, 16 or 32 */
    int32_t fingers_per_word;          /* 32 / bits_per_finger */
    int32_t record_words;              /* ceil(n_slots / fingers_per_word) rounded up to 1, 2, 4, 8 or 16
                                          (a record is whole aligned 16-byte loads; extra words are 0) */
    int32_t finger_lo[CF_MAX_FINGERS][3];   /* tight cell bounds of finger f's samples */
    int32_t finger_dims[CF_MAX_FINGERS][3]; /* (0 if the finger has no sample) */
    int64_t table_words;               /* total uint32 words of the bit table */
    int64_t device_bytes;              /* device memory held by the field */
    float build_ms;                    /* device time of the two build kernels */
    float dilate_deg;                  /* bin dilation of queries (0: none) */
    uint32_t dilation[CF_MAX_BINS];    /* bins accepted by a query of bin b */
    int32_t n_slots;                   /* table slots: n_fingers, or the patch count of a patch field */
    int32_t slot_finger[CF_MAX_SLOTS]; /* finger of slot s */
    int32_t slot_link[CF_MAX_SLOTS];   /* link of slot s in a patch field, -1 otherwise */
} cf_field_info;

/* Object surface points + outward unit normals, device SoA, N each. */
typedef struct cf_points {
    const float *px, *py, *pz;
    const float *nx, *ny, *nz;
    int32_t n;
} cf_points;

/* Tuple scoring parameters (Eq. GSWO, linearised). */
typedef struct cf_score_params {
    int32_t n_tuples;      /* T per pose, >= 1 */
    int32_t k;             /* contacts per tuple, 2..CF_MAX_K */
    int32_t n_edges;       /* K friction-pyramid edges, 3..CF_MAX_EDGES, k*K <= 32 */
    float mu;              /* friction coefficient >= 0 */
    float eps;             /* accept iff margin <= eps */
    float centroid[3];     /* torque reference point c (object frame) */
    float rho;             /* torque scale: torque rows are divided by rho (> 0) */
    uint64_t seed;         /* key of the tuple draws */
    int32_t tuples_given;  /* 1: d_tuples holds the tuples (sampling skipped) */
} cf_score_params;

/* ---- the contact field (Def. Contact Field; Sec. 4.3, Alg. 1) ------------ */

/* Def. Contact Field (Point) and (Hand), Sec. 4.3 "Implementation", Alg. 1.
 * Build the sampled contact field of `hand` from n_samples joint
 * configurations d_q [F][J][n_samples] (device, FP32, SoA per joint).
 * Every (finger, sample, surface point) contact vector is transformed to the
 * palm frame and sets bit bin(n) of its cell's word in the finger's table.
 * Two passes: cell bounds (the host reads them back: one wait on `stream`),
 * then binning, left queued on `stream`.
 * Errors: CF_EINVAL (shapes, NULLs, B or J out of range, cell bounds beyond
 * |k| < 2^20), CF_ENOMEM, CF_ECUDA.  *out is set only on success. */
int cf_build(const cf_hand_desc *hand, const cf_field_params *prm, const float *d_q, int32_t n_samples,
             cf_stream stream, cf_field **out);

/* Sizes, layout and build time of a field (waits for its build to finish). */
int cf_field_get_info(const cf_field *field, cf_field_info *info);

/* Copy the bit table (table_words uint32 words) to host memory. */
int cf_field_copy_table(const cf_field *field, uint32_t *host_words, int64_t capacity_words);

/* Representative table (want_rep): open-addressing hash of rep_slots slots;
 * key = record word index * 32 + bit (the code's position in the table,
 * ~0 for an empty slot), value = smallest sample * M + surface point (original
 * order) that set that bit.  *slots = 0 when the field has none. */
int cf_field_rep_slots(const cf_field *field, int64_t *slots);
int cf_field_copy_rep(const cf_field *field, uint64_t *host_keys, uint32_t *host_vals, int64_t capacity);

/* Frees the field.  Its device memory is released in order on the stream it was
 * built on (that stream must still exist); work that uses the field on other
 * streams must be finished, or ordered before that stream's current work,
 * when this is called. */
int cf_field_destroy(cf_field *field);

/* Raw save / load of a field (header + bin directions + table). */
int cf_field_save(const cf_field *field, const char *path);
int cf_field_load(const char *path, cf_field **out);

/* ---- contact domains (Sec. 4.3 Object Contact Query; Sec. 5.3) ---------- */

/* Def. Contact Surface Representation, Sec. 4.3 "Object Contact Query",
 * Sec. 5.3.  For every pose i (d_poses [P][12], object -> palm) and object point x, the
 * contact-surface vector (R p_x + t, -(R n_x)) is looked up in every slot of
 * the table (a finger, or a patch of a patch field): bit x of d_masks[i][s][W]
 * (W = ceil(N/32) words, bit x & 31 of word x >> 5) is set iff its cell holds
 * its normal bin in slot s.  Bits past N are 0.  d_counts[i][s] = popcount of
 * the row.  d_masks may be NULL (counts only).  Rows: n_slots per pose.
 * Errors: CF_EINVAL, CF_ECUDA (launch). Asynchronous on `stream`. */
int cf_query_domains(const cf_field *field, const cf_points *obj, const float *d_poses, int32_t n_poses,
                     uint32_t *d_masks, uint32_t *d_counts, cf_stream stream);

/* Sec. 5.3 "Contact Domain Generation": the domains of one dependency group (a
 * finger: the connected component of the kinematic tree once the static palm
 * is removed) are merged.  For a patch field (cf_field_params.patches),
 * d_group_masks[i][f][W] = OR over the slots s of finger f of
 * d_slot_masks[i][s][W] (as cf_query_domains wrote them, n_slots rows per
 * pose), and d_group_counts[i][f] its popcount: the per-finger domains that
 * cf_score_tuples samples from.  For a plain field the rows are copied.  n_words
 * = ceil(N/32) of the object queried.  Caller-owned device arrays, no
 * allocation.  Errors: CF_EINVAL, CF_ECUDA.  Asynchronous on `stream`. */
int cf_merge_domains(const cf_field *field, const uint32_t *d_slot_masks, int32_t n_poses, int32_t n_words,
                     uint32_t *d_group_masks, uint32_t *d_group_counts, cf_stream stream);

/* ---- tuple sampling and closure margin (Sec. 5.3; Alg. 2; Eq. GSWO) ----- */

/* Sec. 5.3 and Alg. 2 (Random(D_i)) for the tuples, Eq. GSWO (Sec. 3.2),
 * linearised, for the margin.  Per pose i and tuple tau (u = i*T + tau): unless prm->tuples_given, choose k
 * distinct fingers among those with d_counts[i][f] > 0 and one random point of
 * each domain (Philox4x32-10, key = seed, counter = (i, tau, draw/4, 0)); write
 * d_tuples [P][T][k] (point ids, -1 if fewer than k fingers are non-empty) and
 * d_fingers [P][T][k] (255 when invalid).  Then score every valid tuple:
 * margin = min over j of LP_j = min t s.t. |sum c_im w_im| <= t componentwise,
 * sum_m c_jm = 1, c >= 0, with w_im = [e_im ; (p_i - c) x e_im / rho] and
 * e_im = nu_i + mu (cos(2 pi m/K) x_i + sin(2 pi m/K) y_i), nu_i = -n_i,
 * (x_i, y_i) the Duff et al. 2017 basis of nu_i.  d_margin [P][T] (+inf when
 * invalid), d_accept [P][T] = margin <= eps.  d_masks / d_counts / d_fingers
 * may be NULL when tuples_given.  No global scratch: the scoring kernel
 * hands out tuples from per-block shared-memory counters.  Errors: CF_EINVAL,
 * CF_ECUDA (launch).  Asynchronous on `stream`. */
int cf_score_tuples(const cf_points *obj, int32_t n_fingers, const uint32_t *d_masks, const uint32_t *d_counts,
                    int32_t n_poses, const cf_score_params *prm, int32_t *d_tuples, uint8_t *d_fingers,
                    float *d_margin, uint8_t *d_accept, cf_stream stream);

/* Same computation and outputs as cf_score_tuples, but this call allocates no
 * device memory.  It is for callers that cannot allocate while scoring.  Some
 * have given a fixed budget of device memory to other work on the same GPU
 * (a robot controller or renderer sharing the device).  Some must not risk a
 * failed or blocking allocation in the middle of a control loop.  Some run
 * where the allocator belongs to another framework.  Unlike cf_score_tuples,
 * this entry point promises to allocate nothing, whichever scoring kernel the
 * library runs.  Global scratch, where a scoring kernel needs any, comes from a
 * library-wide device array of CF_NOALLOC_SCRATCH_BYTES bytes; every GPU that
 * loads libcf holds that array until the process exits.  The current kernels
 * need none (sampling stages each pose's masks in shared memory and the scorer
 * hands out tuples from per-block shared-memory counters), so today no call is
 * rejected for size and nothing is cleared; a call whose need exceeded the
 * array would be rejected with CF_EINVAL.  The first call on each device looks
 * up the array's device address.  Make that first call before any stream
 * capture.  Every call shares the array: calls whose work overlaps on the GPU
 * (different streams, or different host threads on one device) would race on
 * it and must be serialised by the caller.  The paper has no counterpart to this
 * entry point.  Errors: as cf_score_tuples, except CF_ENOMEM. */
#define CF_NOALLOC_SCRATCH_BYTES 256
int cf_score_tuples_noalloc(const cf_points *obj, int32_t n_fingers, const uint32_t *d_masks,
                            const uint32_t *d_counts, int32_t n_poses, const cf_score_params *prm, int32_t *d_tuples,
                            uint8_t *d_fingers, float *d_margin, uint8_t *d_accept, cf_stream stream);

/* Sampling step of cf_score_tuples on its own (Sec. 5.3, Alg. 2 Random(D_i)):
 * writes d_tuples / d_fingers exactly as cf_score_tuples would, scores
 * nothing.  prm->tuples_given must be 0; d_margin-style outputs are not used.
 * Errors: CF_EINVAL, CF_ECUDA.  Asynchronous on `stream`. */
int cf_sample_tuples(const cf_points *obj, int32_t n_fingers, const uint32_t *d_masks, const uint32_t *d_counts,
                     int32_t n_poses, const cf_score_params *prm, int32_t *d_tuples, uint8_t *d_fingers,
                     cf_stream stream);

/* ---- reverse lookup + damped-least-squares IK (Sec. 5.5) ---------------- */

typedef struct cf_ik_params {
    float beta;         /* lever of the normal target (m): p~ + beta n~ -> p + beta n */
    float lambda;       /* DLS damping (> 0) */
    int32_t n_phase1;   /* DLS steps from the representative sample */
    int32_t n_rounds;   /* Phase II rounds: project p onto the contact link's capsule, then n_phase2 steps */
    int32_t n_phase2;
    float tol_pos;      /* success: |p~ - p| <= tol_pos (m) ... */
    float tol_cos;      /* ... and n~ . n >= tol_cos, after a last projection */
} cf_ik_params;

/* Kinematics optimisation of tuple slots u = 0..n_slots-1 (pose u / n_tuples),
 * typically cf_score_tuples' outputs.  Slot u is attempted when d_accept[u]
 * (NULL: every slot) and its k contacts (point d_tuples[u][c] of finger
 * d_fingers[u][c]) are valid and of distinct fingers.  Contact c targets the
 * query's contact-surface vector p = R p_x + t, n = -(R n_x) of pose u / T.  The
 * reverse lookup reads the representative (sample s, surface point m) of the
 * contact's (cell, bin) code in finger f's table, and the IK starts from joint
 * sample s with p~, n~ = surface point m; then n_phase1 DLS steps
 * dq = (J^T J + lambda I)^-1 J^T e (e stacks p - p~ and p + beta n - (p~ + beta
 * n~); J their position Jacobians), q clamped to [lo, hi]; then the Phase II
 * rounds; then one last projection.  Fingers share no joint, so each contact is
 * solved on its own.  Outputs (device, caller-owned):
 *   d_q [n_slots][F][J]       joint values (rows of fingers without a contact: 0)
 *   d_used [n_slots][F][J]    1 for joints 0..(contact link) of contact fingers
 *   d_contacts [6][n_slots*k] realised contacts in the object frame (px py pz
 *                             nx ny nz; n = -R^T n~, the object's outward normal)
 *   d_rtuples [n_slots][k]    u*k + c when every contact of the slot succeeded, else -1
 *                             (pass with d_contacts to cf_score_tuples, tuples_given,
 *                             n_poses = n_slots, T = 1, to re-score the realised contacts)
 *   d_resid [n_slots][k][2]   |p~ - p| and n~ . n (inf / -2 when not attempted)
 *   d_ok [n_slots]            1 when every contact succeeded
 * The field must have been built with joint limits and want_rep.  A contact
 * whose code has no representative sets CF_DEV_REP_MISS and fails.
 * Errors: CF_EINVAL, CF_ECUDA.  Asynchronous on `stream`. */
int cf_ik_dls(const cf_field *field, const cf_points *obj, const float *d_poses, int32_t n_slots, int32_t n_tuples,
              int32_t k, const int32_t *d_tuples, const uint8_t *d_fingers, const uint8_t *d_accept,
              const cf_ik_params *prm, float *d_q, uint8_t *d_used, float *d_contacts, int32_t *d_rtuples,
              float *d_resid, uint8_t *d_ok, cf_stream stream);

/* ---- object SDF grid and the realization filter (Sec. 5.6) -------------- */

typedef struct cf_sdf cf_sdf;

/* The grid box that covers host points h_soa [6][n] (px, py, pz rows first)
 * with a margin: lo = min - margin (FP64, rounded to FP32), dims = ceil((max +
 * margin - lo) / h) + 1 per axis (h rounded to FP32 first).  Host only, no
 * device work.  Errors: CF_EINVAL (n < 1, h <= 0, margin < 0, non-finite
 * point, a box beyond 2^20 nodes per axis). */
int cf_sdf_box(const float *h_soa, int32_t n, float h, float margin, float lo[3], int32_t dims[3]);

/* Signed distance of the object's oriented point set on the grid
 * lo + (i, j, k) h, i < dims[0] ... (x fastest): distance to the nearest point
 * (first on ties), negative when (x - p) . n of that point is < 0.  Brute force
 * over all points.  The grid should extend past the object by more than the
 * largest capsule radius: lookups outside it count as far away.
 * Errors: CF_EINVAL, CF_ENOMEM, CF_ECUDA. */
int cf_sdf_build(const cf_points *obj, const float lo[3], float h, const int32_t dims[3], cf_stream stream,
                 cf_sdf **out);
int cf_sdf_copy(const cf_sdf *sdf, float *host, int64_t capacity);
int cf_sdf_destroy(cf_sdf *sdf);

typedef struct cf_realize_params {
    float pen_margin;   /* tolerated penetration depth (m) */
    float axis_step;    /* spacing of the samples along each capsule axis (m) */
    uint64_t seed;      /* key of the random joint values */
} cf_realize_params;

/* Post-processing of tuple slots u (pose u / n_tuples): when d_gate_a[u] and
 * d_gate_b[u] (NULL: 1), every joint with d_used == 0 gets a uniform value in
 * its limits, lo + (u24 * 2^-24) * (hi - lo) in FP32 with u24 the top 24 bits of
 * word j % 4 of Philox4x32-10(counter (u, f, j / 4, 0x7EA1), key seed), written
 * back to d_q.  Capsule links (radius > 0, length > 0) are then checked:
 * penetration when the trilinear SDF at a sample x_s = a + (s / ns)(b - a),
 * s = 0..ns, ns = ceil(length / axis_step), taken to the object frame, is below
 * radius - pen_margin; self-collision when capsules of two fingers are closer
 * than the sum of their radii.  d_flags[u] = 0 for a realised grasp, else bits
 * 1 (gated out), 2 (penetration), 4 (self-collision).
 * Errors: CF_EINVAL, CF_ECUDA.  Asynchronous on `stream`. */
int cf_realize(const cf_field *field, const cf_sdf *sdf, const float *d_poses, int32_t n_slots, int32_t n_tuples,
               const cf_realize_params *prm, const uint8_t *d_gate_a, const uint8_t *d_gate_b, float *d_q,
               const uint8_t *d_used, uint8_t *d_flags, cf_stream stream);

/* ---- Eq. GSWO with true friction cones (Sec. 3.2) ------------------------ */

/* The paper's own metric for given tuples d_tuples [P][T][k] (prm: T, k, mu,
 * centroid, rho; n_edges, eps and seed unused): contact i applies
 * f_i = alpha_i nu_i + bx_i x_i + by_i y_i (nu_i = -n_i, (x_i, y_i) the Duff et
 * al. 2017 basis of nu_i); J_j = min |sum f_i|^2 + |sum (p_i - c) x f_i|^2 / rho^2
 * s.t. alpha_j = 1, |b_j| <= mu, |b_i| <= mu alpha_i (i != j); d_value = min_j J_j,
 * d_accept = d_value <= eps_g.  Each J_j is the value after n_iter projected
 * gradient steps with Nesterov momentum (FISTA), step 1 / (2 tr(A^T A)), from
 * alpha = e_j, beta = 0 (an upper bound that tightens with n_iter).  Invalid
 * tuples (an id < 0) get +inf.  The first call with a given n_iter on a device
 * uploads its momentum table (synchronously, kept for the process).
 * Errors: CF_EINVAL, CF_ECUDA.  Asynchronous otherwise. */
int cf_score_gswo(const cf_points *obj, int32_t n_poses, const cf_score_params *prm, int32_t n_iter, float eps_g,
                  const int32_t *d_tuples, float *d_value, uint8_t *d_accept, cf_stream stream);

/* ---- Alg. 2: blockwise zeroth-order contact optimisation (Sec. 5.4) ------ */

typedef struct cf_opt_params {
    int32_t n_outer;    /* outer iterations n_o (0..64) */
    int32_t n_inner;    /* mutations per contact and iteration n_in: 4, 8 or 16 */
    float sigma;        /* standard deviation of each tangent-plane mutation component (m) */
    float zero_tol;     /* margins <= zero_tol count as 0 (a closed grasp): optimisation stops there */
    float min_gain;     /* a candidate replaces the best so far only when its margin is < (1 - min_gain) x best */
    int32_t warm_start; /* 1: a candidate's LP_j starts from the current tuple's optimal LP_j basis, its moved
                           contact's columns replaced by their new values (a column-replacement pivot where they
                           are basic), when that basis stays feasible (Sec. 5.4 "A Free Lunch"); 0: from
                           c' = 0.  Margins agree either way (each LP is solved to its optimum). */
} cf_opt_params;

/* Improves every valid tuple of d_tuples [P][T][k] in place (Sec. 5.4, Alg. 2;
 * prm->tuples_given must be 1; d_fingers [P][T][k] gives each contact's finger;
 * d_masks [P][n_fingers][ceil(N/32)] the domains the projections use).  For it = 0 ..
 * n_outer-1 and each contact i: with (x, y) the Duff et al. 2017 basis of
 * nu = -n_i, candidate c = 0 .. n_inner-1 mutates p_i by sigma (g1 x + g2 y), with
 * (g1, g2) the Box-Muller pair of Philox4x32-10 words (2 (c mod 2), 2 (c mod 2)
 * + 1) at counter (pose, tau, (it k + i) ceil(n_inner / 2) + c / 2, 0xA162), key
 * seed: u1 = (w >> 8 + 1) 2^-24, u2 = (w' >> 8) 2^-24, g = sqrt(-2 ln u1)
 * (cos, sin)(2 pi u2), in FP32.  Each mutation is projected onto finger f_i's domain at
 * the pose (the object point with its mask bit set nearest to it, lowest index
 * on ties).  Starting from the current point, the candidates in order replace
 * the best so far when their closure margin is below (1 - min_gain) x best
 * (margins <= zero_tol count as 0); contact i moves to the final best.  d_margin / d_accept receive the
 * final tuple's margin and margin <= eps.  Invalid tuples (an id outside [0, N) or a
 * finger >= n_fingers) are left unchanged with margin +inf.  Each tuple's result
 * depends only on the tuple (its pose index, tau, points and domains), not on how
 * the launch schedules tuples over warps.  Needs scratch from the library's pool
 * (word and chunk boxes of the points, and per tuple its candidates, their LP values and,
 * with warm_start, its k optimal LP bases: ~840 bytes per tuple at n_inner 8, k 3).  Errors: CF_EINVAL,
 * CF_ENOMEM, CF_ECUDA; device status CF_DEV_LP_PIVOT_CAP. */
int cf_optimize_tuples(const cf_points *obj, int32_t n_fingers, const uint32_t *d_masks, int32_t n_poses,
                       const cf_score_params *prm, const cf_opt_params *opt, int32_t *d_tuples,
                       const uint8_t *d_fingers, float *d_margin, uint8_t *d_accept, cf_stream stream);

/* ---- many objects in one graph launch (no paper counterpart) ------------ */

/* One object request of a batch: the same inputs and caller-owned outputs as
 * cf_query_domains + cf_score_tuples (prm.tuples_given must be 0). */
typedef struct cf_batch_item {
    const cf_field *field;
    cf_points obj;
    const float *d_poses;
    int32_t n_poses;
    cf_score_params prm;
    uint32_t *d_masks, *d_counts;
    int32_t *d_tuples;
    uint8_t *d_fingers;
    float *d_margin;
    uint8_t *d_accept;
} cf_batch_item;

typedef struct cf_batch cf_batch;

/* Plan a batch of objects (fields, hands, sizes and pose counts may differ).
 * A run is three persistent launches whatever the mix: the domain query of
 * every object (one grid whose blocks take (object, block of poses) items from
 * a device work counter and pick the kernel body for the object's hand at run
 * time), the tuple sampling of every pose, and the LP scoring of every tuple
 * (one scoring launch per distinct (k, K)).  No kernel waits on another block.
 * Results equal the per-object calls bit for bit.  The items' buffers are used
 * in place by every run.  The paper has no counterpart (its forward pass
 * handles one object).  Errors: CF_EINVAL, CF_ENOMEM, CF_ECUDA. */
int cf_batch_create(const cf_batch_item *items, int32_t n_items, cf_batch **out);

/* Run the batch after the work already queued on `stream`.  The first run
 * captures the launches into a CUDA graph; later runs replay it (one graph
 * launch).  Asynchronous. */
int cf_batch_run(cf_batch *batch, cf_stream stream);

/* Number of kernel launches one run performs and the number of launch groups. */
int cf_batch_launches(const cf_batch *batch, int32_t *n_launches, int32_t *n_groups);

int cf_batch_destroy(cf_batch *batch);

/* ---- object placement (Sec. 5.2) and preprocessing (Sec. 5.1) ------------ */

typedef struct cf_place_params {
    int32_t exhaustive;   /* 0: canonical placement, 1: exhaustive placement */
    float centroid[3];    /* canonical: the object's centroid (object frame) */
    float g[3], up[3];    /* canonical: anchor point and unit palm normal (palm frame) */
    float d_lo, d_hi;     /* canonical: offset of the centroid along up */
    uint64_t seed;        /* key of the draws */
    uint32_t pose_base;   /* added to the pose index in the draws' counter */
} cf_place_params;

/* Palm poses d_poses [n_poses][12] (object -> palm, row-major (R | t)), FP64
 * arithmetic rounded to FP32, from Philox4x32-10 words at counter (pose +
 * pose_base, tag, 0, 0), key seed; u = (w >> 8) 2^-24.
 * Canonical (tag 0x91AC): R = the unit quaternion (sqrt(1-u1) sin 2 pi u2,
 * sqrt(1-u1) cos 2 pi u2, sqrt(u1) sin 2 pi u3, sqrt(u1) cos 2 pi u3) (x, y, z, w;
 * Shoemake), t = g + (d_lo + u4 (d_hi - d_lo)) up - R centroid.
 * Exhaustive (tag 0xE7A1; needs `field` and `obj`): the r-th code of the field
 * in table order (cell, finger, bin), r = floor(w0 n_codes / 2^32), gives the
 * point c = (k + 1/2) / inv_h (its cell centre) and the normal d_b (its bin
 * direction); object point x = floor(w1 N / 2^32); R = Rot(d_b, 2 pi u2) R_align
 * with R_align the shortest rotation taking n_x to -d_b (a half turn about
 * (n_x x e) / |...| when opposite, e = e_x or e_y), t = c - R p_x.  The first
 * exhaustive call on a field counts its codes per table chunk (one wait).
 * Errors: CF_EINVAL, CF_ENOMEM, CF_ECUDA. */
int cf_place(const cf_field *field, const cf_points *obj, int32_t n_poses, const cf_place_params *prm,
             float *d_poses, cf_stream stream);

/* Static-link placement (Sec. 5.2, last paragraph): poses that put the object
 * against the palm, for grasps such as the power grasp.  The palm is the box
 * [lo, hi] of the palm frame; its top face z = hi[2] is the contact surface,
 * outward normal +z.  Pose i draws Philox4x32-10 words (w0..w3) at counter
 * (i + pose_base, 0x57A7, 0, 0), key seed: object point x = floor(w0 N / 2^32);
 * palm point c = (lo_x + u1 (hi_x - lo_x), lo_y + u2 (hi_y - lo_y), hi_z),
 * u = (w >> 8) 2^-24; R = Rot(+z, 2 pi u3) R_align with R_align the shortest
 * rotation taking n_x to -z (the object's outward normal at x faces into the
 * palm; a half turn about (n_x x e) / |...| when n_x = +z, e = e_x); t = c - R
 * p_x.  FP64, rounded to FP32 into d_poses [P][12].  d_static_pt[i] = x.
 * The penetration filter: d_valid[i] = 0 when some object point q = R p + t
 * (FP32, with the stored pose) lies inside the palm's xy rectangle with
 * lo_z <= q_z < hi_z - pen_margin (the placement "causes penetration"), else 1.
 * A valid pose's static contact (x, and the palm's force along -n_x) joins the
 * finger contacts through cf_append_contact.  Errors: CF_EINVAL, CF_ECUDA.
 * Asynchronous on `stream`. */
typedef struct cf_palm_desc {
    float lo[3], hi[3];  /* palm box, palm frame (lo < hi per axis) */
} cf_palm_desc;
int cf_place_static(const cf_palm_desc *palm, const cf_points *obj, int32_t n_poses, uint64_t seed,
                    uint32_t pose_base, float pen_margin, float *d_poses, int32_t *d_static_pt, uint8_t *d_valid,
                    cf_stream stream);

/* Tuples with one more contact in front: d_out[i][t] = (d_first[i],
 * d_tuples[i][t][0 .. k-1]) for [P][T][k] tuples, d_out [P][T][k+1]; a pose
 * whose d_first is < 0 or whose d_valid (may be NULL) is 0 gets an invalid
 * tuple (all -1), as does an invalid input tuple.  With cf_place_static this
 * scores the static contact with the sampled finger contacts (the "contact
 * vectors" that placement advances, Sec. 5.2).  Errors: CF_EINVAL, CF_ECUDA.
 * Asynchronous on `stream`. */
int cf_append_contact(const int32_t *d_tuples, int32_t n_poses, int32_t n_tuples, int32_t k, const int32_t *d_first,
                      const uint8_t *d_valid, int32_t *d_out, cf_stream stream);

/* Concave-point removal: point x is kept (d_keep[x] = 1) unless the object SDF
 * (trilinear, cf_sdf_build) is below -tau at the centre or at a corner of the
 * upper half of the cube of side `side` resting on the tangent plane outside x
 * (centre p_x + (side / 2) n_x, axes (t1, t2, n_x), t1, t2 the Duff et al. 2017
 * basis of n_x; samples at heights side/2 and side, lateral +-side/2).  The kept points
 * are written to d_out [6][n] (px..nz rows of stride n, original order; may be
 * NULL) and their number to *d_n_out (device).  Errors: CF_EINVAL, CF_ENOMEM,
 * CF_ECUDA.  Asynchronous. */
int cf_concave_filter(const cf_points *obj, const cf_sdf *sdf, float side, float tau, uint8_t *d_keep,
                      float *d_out, int32_t *d_n_out, cf_stream stream);

/* ---- launch shapes and the autotuner (no paper counterpart) ------------- */

/* Launch shapes of the query and scoring kernels on the current device.  The
 * results of every call are the same under any shape; only the time changes.
 * Batches and engines take the shapes current at their creation. */
typedef struct cf_tuning {
    int32_t query_poses_per_block;  /* poses per domain-query block, 1..16 (default 4); with poses x slots
                                       <= 32 each lane keeps one (pose, slot) mask word */
    int32_t score_refill;           /* scoring lanes of a warp that wait before they take new tuples together:
                                       4, 8 or 16 (default 8) */
    int32_t score_blocks_per_sm;    /* scoring blocks per SM: 1, 2, 3, or 0 = as many as fit (default 0) */
} cf_tuning;

int cf_get_tuning(cf_tuning *out);
int cf_set_tuning(const cf_tuning *tuning);

/* Autotuner: runs the items' query launches under every poses-per-block
 * candidate, then their sampling + scoring under every (refill, blocks per SM)
 * candidate, `reps` times each (median of the summed CUDA-event
 * times), keeps the fastest and makes it the device's tuning; *out (if not
 * NULL) receives it and best_ms[0..1] the query and scoring times it measured.
 * The items' output buffers are written by the trial runs.  Synchronous.
 * Errors: CF_EINVAL, CF_ENOMEM, CF_ECUDA. */
int cf_autotune(const cf_batch_item *items, int32_t n_items, int32_t reps, cf_tuning *out, double *best_ms);

/* ---- served form: continuous batching (no paper counterpart) ------------ */

typedef struct cf_engine cf_engine;

typedef struct cf_engine_params {
    const cf_field *const *fields;  /* resident hand fields (not owned; must outlive the engine) */
    int32_t n_fields;
    int64_t hbm_budget_bytes;       /* device memory the active requests may hold together */
    int32_t max_active;             /* requests processed concurrently (slots) */
    int32_t pose_chunk;             /* poses of each active request per round */
    int32_t pose_cap;               /* poses a request may use before it ends with a partial result */
    int32_t pose_chunk_max;         /* <= pose_chunk: every round takes pose_chunk poses.  Larger: after its
                                       first round a request takes the poses that its acceptance so far says
                                       it still needs (with 25 % to spare; twice its last chunk while it has
                                       none), between pose_chunk and pose_chunk_max; its device state (and
                                       budget share) is sized for min(pose_chunk_max, its pose limit).  The
                                       chunks depend only on the request's own results, so a result is still
                                       the same alone and in any mix. */
    int64_t chunk_pairs_max;        /* with adaptive chunks, a chunk above pose_chunk also keeps chunk x n
                                       (the query's point-pose pairs) <= chunk_pairs_max, so one large
                                       object's round stays short for the requests it shares it with
                                       (0: no limit) */
    int64_t reserve_bytes;          /* device memory the engine grows the library's pool by at creation
                                       (allocated and freed; the pool keeps freed memory), so the first
                                       requests do not wait while the pool grows; 0: none */
} cf_engine_params;

typedef struct cf_request {
    int32_t field;                  /* index into cf_engine_params.fields */
    const float *h_soa;             /* host [6][n] object points + outward normals (copied by submit) */
    int32_t n;
    const float *h_poses;           /* host [n_poses][12] candidate palm poses, used in order (copied) */
    int32_t n_poses;
    cf_score_params prm;            /* T, k, K, mu, eps, centroid, rho, seed (tuples_given = 0) */
    int32_t n_grasps;               /* the request ends once this many tuples are accepted */
    uint64_t tag;                   /* caller's label, returned with the result */
} cf_request;

typedef struct cf_result {
    uint64_t id, tag;
    int32_t status;                 /* CF_OK or the error that ended the request */
    int32_t partial;                /* 1: the pose cap (or the pose list) ran out first */
    int32_t k;
    int32_t n_accepted;             /* accepted tuples (all of the last round's chunk, may exceed n_grasps) */
    int32_t n_poses_used;
    double t_submit, t_admit, t_done;  /* seconds on the engine's clock */
    int32_t *pose;                  /* [n_accepted] pose index of each accepted tuple */
    int32_t *tuples;                /* [n_accepted][k] object point ids */
    float *margin;                  /* [n_accepted] closure margins */
    int32_t n_rounds;               /* rounds the request took part in */
    double t_first_round;           /* start of its first round (engine clock; t_done if none) */
} cf_result;

typedef struct cf_engine_stats {
    int64_t submitted, completed, rounds, launches;
    int32_t queued, active;
    int64_t bytes_in_use, peak_bytes_in_use;
    int32_t peak_active;
    /* cumulative worker seconds: admission uploads, round preparation and
     * launches on the host, waiting for the round's GPU work and result copies */
    double admit_s, round_host_s, round_wait_s;
} cf_engine_stats;

/* Start an engine: a worker thread on the current device admits queued
 * requests in arrival order while a slot is free and their device state fits
 * in the HBM budget, then runs rounds: every active request contributes its
 * next pose_chunk poses, and all of them go through the grouped query,
 * sampling and scoring launches together.  Requests that arrive while others
 * are on the GPU join at the next round.  Tuple draws are keyed by the
 * request's seed and global pose index, so a request's result does not depend
 * on what it shares rounds with.  Errors: CF_EINVAL, CF_ENOMEM, CF_ECUDA. */
int cf_engine_create(const cf_engine_params *prm, cf_engine **out);

/* Queue a request (copies its host arrays); never blocks on the GPU.  A
 * request whose device state alone exceeds the budget completes at once with
 * status CF_ENOMEM. */
int cf_engine_submit(cf_engine *eng, const cf_request *req, uint64_t *id);

/* Take up to max finished requests (non-blocking); free each with
 * cf_engine_result_free. */
int cf_engine_poll(cf_engine *eng, cf_result *out, int32_t max, int32_t *n_done);

int cf_engine_result_free(cf_result *res);

int cf_engine_get_stats(const cf_engine *eng, cf_engine_stats *out);

/* Wait (up to timeout_ms; < 0: no limit) until nothing is queued or active.
 * Returns CF_ETIMEOUT if work remains. */
int cf_engine_drain(cf_engine *eng, int32_t timeout_ms);

/* Stops the worker after the current round; unfinished requests are dropped. */
int cf_engine_destroy(cf_engine *eng);

/* ---- one object request from host buffers (no paper counterpart) -------- */

typedef struct cf_plan cf_plan;

/* Device buffers for objects of up to n_max points and p_max poses, fields of
 * up to n_fingers fingers, and prm's T and k.  Errors: CF_EINVAL, CF_ENOMEM. */
int cf_plan_create(int32_t n_fingers, int32_t n_max, int32_t p_max, const cf_score_params *prm, cf_plan **out);

/* One request against `field`: h_soa [6][n] (px..nz), h_poses [P][12] are copied to the device (on a
 * plan-owned stream, so the copies overlap work still queued on `stream`, such as the field build; the
 * host buffers must not change until the call returns), domains,
 * tuples and margins computed, results copied back: h_tuples [P][T][k],
 * h_margin [P][T], h_accept [P][T] (each may be NULL), *h_n_accepted (counted
 * on the device).  The tuples are copied back while the scoring kernel runs,
 * the margins and flags after it.  Host buffers should be page-locked
 * for full copy speed.  Synchronises `stream`. */
int cf_plan_run_host(cf_plan *plan, const cf_field *field, const float *h_soa, int32_t n, const float *h_poses,
                     int32_t n_poses,
                     const cf_score_params *prm, int32_t *h_tuples, float *h_margin, uint8_t *h_accept,
                     int64_t *h_n_accepted, cf_stream stream);

/* One accepted grasp as cf_plan_run_host_accepted returns it. */
typedef struct cf_grasp {
    int32_t pose;              /* pose index within the request */
    float margin;              /* its closure margin (<= eps) */
    int32_t point[CF_MAX_K];   /* its k object point ids (-1 beyond k) */
} cf_grasp;

/* As cf_plan_run_host, but only the accepted tuples come back: they are gathered on the device,
 * in (pose, tuple) order, into records (24 bytes each instead of 4k + 5 bytes per sampled tuple),
 * and h_grasps[0 .. min(count, cap)) receives them; *h_n_accepted is the full count (larger
 * than cap when h_grasps was too small).  The records are the tuples whose margin passes the
 * closure test (the output set of Alg. 1).  h_grasps is the caller's (page-locked, or the copy
 * is staged by the CUDA driver); cap = 0 with h_grasps NULL returns the count alone.  Synchronises
 * `stream`.  Errors: CF_EINVAL (as cf_plan_run_host; cap < 0; h_grasps NULL with cap > 0),
 * CF_ECUDA. */
int cf_plan_run_host_accepted(cf_plan *plan, const cf_field *field, const float *h_soa, int32_t n,
                              const float *h_poses, int32_t n_poses, const cf_score_params *prm, cf_grasp *h_grasps,
                              int64_t cap, int64_t *h_n_accepted, cf_stream stream);

int cf_plan_destroy(cf_plan *plan);

/* ---- diagnostics (no paper counterpart) --------------------------------- */

/* FP32 FMA throughput of the current device in TFLOP/s (2 flop per FMA),
 * measured by a kernel of independent FMA chains timed with CUDA events: the
 * denominator of the FP32-issue-bound rooflines.  Synchronous. */
int cf_fp32_peak(double *tflops);

const char *cf_last_error(void);

/* Read and clear the device status word (CF_DEV_* bits) of the current device. */
int cf_device_status(uint32_t *status);

/* Cumulative device counters of the current device since the last reset:
 * [0] LP pivots performed, [1] LPs solved, [2] tuples scored, [3] LPs of
 * cf_optimize_tuples' candidates that started from the current tuple's
 * optimal basis of the same LP, repaired for the moved contact (the warm
 * start of Sec. 5.4). */
int cf_device_counters(uint64_t counters[4], int reset);

/* Device memory of the library's stream-ordered pool on the current device,
 * from which every library-owned buffer (fields, batches, requests, temporary
 * work lists) is drawn: usage[0] bytes in use now, usage[1] bytes reserved
 * from the CUDA driver, usage[2] the largest use since the last reset.
 * reset_high != 0 restarts that high-water mark at the current use (after
 * reading it).  The first call on a device creates the pool.  Synchronous
 * with respect to nothing: allocations still queued on a stream count once
 * they run.  The paper has no counterpart.  Errors: CF_EINVAL, CF_ECUDA. */
int cf_pool_usage(uint64_t usage[3], int reset_high);

#ifdef __cplusplus
}
#endif
#endif /* CF_H */
