/*
 * srp.h -- C ABI of the GB300-native ray-traced solar radiation pressure
 * library (libsrp.so).
 *
 * The library evaluates the solar radiation pressure (SRP) force and torque on
 * a triangle-mesh spacecraft with articulated solar panels by casting one ray
 * per pixel of a projection window along the Sun direction, following first
 * hits (self-shadowing) and specular secondary rays, and propagates orbits
 * whose acceleration includes that force.
 *
 * Paper sections that define the operations (arxiv 2608.07307):
 *   Sec. 3, Eqs. 1-3   equations of motion y' = (v, a_g + a_SRP) integrated by an
 *                      explicit embedded Runge-Kutta 7(8);
 *   Sec. 4.3           per-pixel independent rays over a discretised image plane,
 *                      iterated secondary rays, on-GPU reduction of all pixel
 *                      contributions so only the final force is read back;
 *   Sec. 4.4.1-4.4.2   kinematic tree of rigid parts; each movable joint rotates
 *                      its subtree so the panel normal is as close as possible to
 *                      the Sun, clamped to the joint's admissible interval;
 *   Sec. 6.1           N x N projection window, levels of secondary reflections.
 *
 * Conventions shared by every entry point
 *   - Units: SI (m, s, N, N m, kg) and radians.  Body frame for srp_eval_batch.
 *   - Photons travel along d = -s, s the unit body-frame vector towards the Sun.
 *   - Ray r of an evaluation is pixel (i, j) = (r / N, r % N) of the window;
 *     i runs along the window's u axis, j along its v axis.
 *   - Quaternions are scalar first and rotate body axes into inertial axes
 *     (into LVLH axes for SRP_ATT_LVLH).
 *   - Pointers to per-call data may be host or device memory (the library asks
 *     the driver which); outputs are owned by the caller and written before the
 *     call returns.  Mesh descriptions must be host memory; the library copies
 *     them at load.
 *   - Calls are ordered on the context's CUDA stream and synchronous on return.
 *   - No C++ exception crosses the ABI.  Every call returns an srp_status; on
 *     failure srp_last_error() describes it.  A context is used by one host
 *     thread at a time.
 */
#ifndef SRP_H
#define SRP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct srp_ctx srp_ctx;
typedef int32_t srp_status;

#define SRP_OK 0
#define SRP_ERR_ARG (-1)     /* invalid argument (null pointer, bad size, bad id)        */
#define SRP_ERR_OOM (-2)     /* device or host allocation failed                         */
#define SRP_ERR_CUDA (-3)    /* a CUDA runtime call failed                               */
#define SRP_ERR_MESH (-4)    /* mesh rejected (indices, tree order, materials, degenerate) */
#define SRP_ERR_STACK (-5)   /* a traversal stack bound was reached (device flag)       */
#define SRP_ERR_TIMEOUT (-6) /* a bounded device-side wait gave up                       */
#define SRP_ERR_STEP (-7)    /* integrator: step size underflow or step budget exhausted  */
#define SRP_ERR_STATE (-8)   /* call out of order (e.g. no mesh loaded, context unusable) */

#define SRP_F32 0
#define SRP_F64 1

/* Limits of the library. */
#define SRP_MAX_PARTS 16
#define SRP_MAX_MATS 256
#define SRP_MAX_BOUNCES 4
#define SRP_MAX_N 8192

/*
 * Mesh description (Sec. 4.4.1).  Part 0 is the root (body frame); part p > 0
 * hangs from parent[p] < p.  A part with a non-zero axis is a movable joint:
 * its transform is the parent's composed with a rotation by its angle about
 * axis through pivot (rest body frame), so a joint moves its whole subtree.
 * Triangles are counter-clockwise seen from their front side; every triangle
 * has one part and a material per side.  A vertex may be used by one part only.
 */
typedef struct {
    int32_t n_verts;
    int32_t vertex_dtype;     /* SRP_F32 or SRP_F64                                    */
    const void *xyz;          /* [n_verts][3] rest pose, metres                         */
    int32_t n_tris;
    const int32_t *tri;       /* [n_tris][3] vertex indices                             */
    const int32_t *tri_part;  /* [n_tris]                                               */
    const int32_t *tri_mat;   /* [n_tris][2] material of the front, back side          */
    int32_t n_mats;
    const double *mat;        /* [n_mats][2] rho_s, rho_d; rho_s, rho_d >= 0, sum <= 1  */
    int32_t n_parts;
    const int32_t *parent;    /* [n_parts]; parent[0] = -1                              */
    const double *pivot;      /* [n_parts][3]                                           */
    const double *axis;       /* [n_parts][3] unit, or all zero for a rigid link        */
    const double *limits;     /* [n_parts][2] admissible angle interval lo <= hi (rad)  */
    const double *normal0;    /* [n_parts][3] rest front normal of a movable panel part */
    double c_ref[3];          /* torque reference point                                 */
    double mass;              /* kg (used by srp_propagate)                             */
} srp_mesh_desc;

/* How joint angles are chosen for each evaluation (Sec. 4.4.2). */
#define SRP_PANELS_TRACK 0        /* angle = argmax of n(theta) . s, clamped             */
#define SRP_PANELS_SET 1          /* angle = value from srp_set_panel_angles, clamped    */
#define SRP_PANELS_TRACK_OFFSET 2 /* angle = tracking angle + set value, clamped          */

typedef struct {
    int32_t N;           /* rays per side of the projection window, 1..SRP_MAX_N       */
    int32_t bounces;     /* specular secondary levels, 0..SRP_MAX_BOUNCES                */
    double P0;           /* radiation pressure at 1 AU, N/m^2 (e.g. 4.56e-6)             */
    double eps_rel;      /* secondary-ray self-hit threshold / window diagonal (1e-9)    */
    int32_t panel_mode;  /* SRP_PANELS_*                                                 */
    int32_t flags;       /* 0, or SRP_EVAL_COUNT to gather srp_eval_stats counters       */
    int32_t n_diffuse;   /* diffuse secondary rays per hit, 0..SRP_MAX_DIFFUSE (0: none;
                            see below)                                                   */
    uint32_t diffuse_seed; /* seed of the diffuse rays' sample stream                    */
} srp_eval_params;

/*
 * Diffuse secondary rays (Sec. 6.1: the paper's configuration traces 16 per
 * hit).  With n_diffuse = K > 0, the hit of every ray segment that has a next
 * level (segment k < bounces) also emits K rays of weight w rho_d / K (w the
 * segment's weight, rho_d that of the side hit) from the hit point, in
 * cosine-weighted directions about the normal of the lit side; each is traced
 * once (never onto the emitting triangle, t > eps) and deposits the full
 * per-hit law at its hit, spawning nothing further.  The emitter keeps its
 * analytic 2/3 rho_d recoil.  Sample q of segment k of ray r = i N + j uses
 * outputs 2c and 2c + 1 of the SplitMix64 stream seeded with diffuse_seed,
 * c = (r (bounces + 1) + k) K + q, as uniforms u1, u2 (top 53 bits): local
 * direction (sqrt(u1) cos 2 pi u2, sqrt(u1) sin 2 pi u2, sqrt(1 - u1)) in the
 * basis of Duff et al. around that normal.  The diffuse rays are traced with
 * FP64 decisions.  srp_eval_batch and srp_propagate take them;
 * srp_grad, srp_prop_grad and srp_propagate_batch need n_diffuse = 0.
 */
#define SRP_MAX_DIFFUSE 256

#define SRP_EVAL_COUNT 1  /* gather traversal counters (slower kernel variant)        */
#define SRP_EVAL_TIMING 2 /* time each phase with CUDA events on the context stream   */
/* Primary visibility by BVH traversal of every pixel's ray instead of the
 * default rasterisation.  All primary rays of an evaluation are parallel
 * (Sec. 4.3: one independent ray per pixel, all along d), so the default
 * projects each triangle into the window and applies the same FP32 test to the
 * pixel centres it covers, keeping per pixel the nearest certain hit and the
 * triangles the test could not settle (resolved in FP64 as after a traversal).
 * Both give the same hits and the same force bits; this flag is for testing
 * that and for meshes whose triangles each cover much of the window. */
#define SRP_EVAL_TRAVERSE 8
/* Test of the traversal's error path: every BVH walk is bounded at one step,
 * so any evaluation that walks the tree stops there and returns
 * SRP_ERR_STACK (a bounded loop that sets a device flag; nothing faults or
 * waits).  For tests only. */
#define SRP_EVAL_TEST_WALK_BOUND 16
/* Run every chunk of evaluations on one pipeline lane, in order, instead of
 * overlapping chunks on several lanes.  With SRP_EVAL_TIMING each phase's
 * time is then the GPU time of its own kernels (no other chunk runs beside
 * them), e.g. the trace kernel's duration per launch for a roofline.  Results
 * are the same bits either way. */
#define SRP_EVAL_SERIAL 32
/* Run the raster's second pass and the trace of each chunk as one persistent
 * launch over a device-side work queue: items (second pass over 128 small
 * triangles, over 4 chunks of large triangles, a block of 4 trace tiles) are
 * handed out in that order, and a trace item waits until its slot's second
 * pass is complete.  Every wait is bounded (2 s of device time); a wait that
 * gives up makes the call return SRP_ERR_TIMEOUT (its tiles contribute
 * nothing) and leaves the context usable.  Results are the same bits as
 * without the flag. */
#define SRP_EVAL_QUEUE 64
/* Test of the work queue's bounded wait: every trace item waits for a count
 * that is never reached, with a 2 ms bound, so the call returns
 * SRP_ERR_TIMEOUT.  Implies SRP_EVAL_QUEUE.  For tests only. */
#define SRP_EVAL_TEST_WAIT_TIMEOUT 128
/* Precision report (Sec. 4.3: the paper's shaders keep compensated (Kahan)
 * FP32 sums): the sums above the 32-ray tile, normally FP64, in compensated
 * FP32 (each addition's exact rounding error carried in a second FP32 word,
 * the Kahan-Babuska form) or in plain FP32.  Per-ray and per-tile sums are
 * FP32 in every mode; only the accumulation across tiles changes. */
#define SRP_EVAL_SUM_COMP32 256
#define SRP_EVAL_SUM_FP32 512

/* Counters of the last srp_eval_batch call (summed over its evaluations). */
typedef struct {
    int64_t evals;
    int64_t rays;             /* primary rays cast                                       */
    int64_t segments;         /* ray segments traced (primary + secondary)               */
    int64_t hits[SRP_MAX_BOUNCES + 1]; /* hits per segment level                         */
    int64_t refined;          /* rays re-traced in FP64 because an FP32 decision was within its error bound */
    int64_t nodes_visited;    /* BVH nodes fetched (SRP_EVAL_COUNT only)                  */
    int64_t tris_tested;      /* ray/triangle tests (SRP_EVAL_COUNT only)                 */
    int64_t box_tests;        /* ray/box slab tests (SRP_EVAL_COUNT only)                 */
    int64_t handoff_cause[4]; /* FP64 hand-offs by cause: primary edge, secondary edge,
                                 near tie in t, self-hit band (SRP_EVAL_COUNT only)       */
    int64_t launches;         /* kernels launched by the call                            */
    int64_t trace_launches;   /* of which FP32 trace kernels                             */
    /* GPU time per phase, milliseconds (SRP_EVAL_TIMING only), after the
     * paper's split of an evaluation into compute, transfer and reduction
     * (Sec. 8.2, Eq. 4): */
    double ms_geometry;       /* joint angles, posing, window bounds, refit              */
    double ms_trace;          /* FP32 trace: first hits, shading, bounces                */
    double ms_refine;         /* 0: the FP64 settling runs inside the trace and the rare FP64
                                 re-trace inside the reduction (kept for layout)           */
    double ms_reduce;         /* fixed-order FP64 reduction to force / torque            */
    double ms_transfer;       /* host <-> device copies made by the call                 */
    double ms_raster;         /* window frame and primary visibility by rasterisation    */
} srp_eval_stats;

/*
 * Create a context on CUDA device `device`.  cuda_stream is a cudaStream_t to
 * order work on, or NULL for a stream the context creates and owns.
 * Errors: SRP_ERR_ARG (out NULL), SRP_ERR_CUDA (no such device), SRP_ERR_OOM.
 */
srp_status srp_create(srp_ctx **out, int32_t device, void *cuda_stream);

/* Destroy a context and every mesh and buffer it holds.  NULL is a no-op. */
void srp_destroy(srp_ctx *ctx);

/* Message of the last failed call on ctx ("" when none); valid until the next call. */
const char *srp_last_error(const srp_ctx *ctx);

/*
 * Load a mesh: validate, copy to the device, build one LBVH per rigid part
 * (Morton codes of triangle centroids, radix sort, binary radix tree) and fit
 * its boxes to the rest pose.  mesh_id receives a handle >= 0.
 * Errors: SRP_ERR_ARG (NULL pointers, counts <= 0, limits exceeded),
 * SRP_ERR_MESH (index out of range, parent order, shared vertex, degenerate
 * triangle, material coefficients outside [0, 1] or summing above 1, a part
 * of 2^24 triangles or more).
 */
srp_status srp_mesh_load(srp_ctx *ctx, const srp_mesh_desc *desc, int32_t *mesh_id);

/* Release a mesh and its device memory. */
srp_status srp_mesh_free(srp_ctx *ctx, int32_t mesh_id);

/*
 * Joint angles (rad) used by SRP_PANELS_SET (as the angle) and
 * SRP_PANELS_TRACK_OFFSET (as an offset added to the tracking angle); one per
 * part, n == n_parts; entries of rigid parts are ignored.  Initially zero.
 * Errors: SRP_ERR_ARG (bad id, n mismatch, NULL).
 */
srp_status srp_set_panel_angles(srp_ctx *ctx, int32_t mesh_id, int32_t n, const double *rad);

/*
 * SRP force and torque for n Sun directions (Sec. 4.3, 4.4.2, 6.1).
 * For each direction k: joint angles per params->panel_mode; posed mesh; window
 * = tight bounds of the posed vertices on the basis (u, v) of the plane normal
 * to d; N x N rays from the pixel centres, 1 m in front of the nearest vertex;
 * first hit of each ray (two-sided, ties to the lowest triangle id); per hit
 * the absorbed + specular + Lambertian-diffuse momentum, with the specular beam
 * traced for `bounces` more levels (weight times rho_s; a secondary ray never
 * hits the triangle it leaves); sum of all pixels times P0 / dist^2 times the
 * pixel area.
 *   sun_dir_body [n][3]   unit vectors towards the Sun, body frame; with quat,
 *                         the Sun direction in the inertial frame instead
 *   quat         [n][4]   NULL, or the attitude per evaluation: scalar-first
 *                         quaternion body -> inertial (normalised here).  The
 *                         body-frame direction is then R(q)^T sun_dir and
 *                         `force` receives the SRP acceleration of the state,
 *                         R(q) F_body / mass (m/s^2, inertial frame; Sec. 3
 *                         Eq. 1), mass from the mesh description (must be > 0)
 *   sun_dist_au  [n]      Sun distance (AU); NULL means 1; a negative entry skips
 *                         that evaluation (force and torque 0, hit ids untouched)
 *   force        [n][3]   out, N (body frame), or m/s^2 (inertial) with quat
 *   torque       [n][3]   out, N m about c_ref, body frame
 *   hit_tri      [n][N*N][bounces+1] out, original triangle id per ray segment,
 *                         -1 when that segment missed or was not traced; NULL
 *                         to skip (debug output, large)
 * Errors: SRP_ERR_ARG, SRP_ERR_STATE (bad mesh id), SRP_ERR_STACK, SRP_ERR_CUDA.
 */
srp_status srp_eval_batch(srp_ctx *ctx, int32_t mesh_id, const srp_eval_params *params, int32_t n,
                          const double *sun_dir_body, const double *quat, const double *sun_dist_au, double *force,
                          double *torque, int32_t *hit_tri);

/* Counters of the last srp_eval_batch on ctx. */
srp_status srp_eval_stats_get(srp_ctx *ctx, srp_eval_stats *out);

/*
 * Replace the optical coefficients of a loaded mesh (the rho_s, rho_d per
 * material of Sec. 4.3's per-hit momentum law); the geometry and its
 * acceleration structure are kept.
 *   mat [n_mats][2] host or device, n_mats == the mesh's material count.
 * Errors: SRP_ERR_ARG (bad id, count mismatch, NULL), SRP_ERR_MESH (a
 * coefficient outside [0, 1] or rho_s + rho_d above 1).
 */
srp_status srp_set_materials(srp_ctx *ctx, int32_t mesh_id, int32_t n_mats, const double *mat);

/* ------------------------------------------------------------- gradients */
/*
 * Gradient of the SRP evaluation with its hit set frozen (reverse mode).
 *
 * For each direction k this runs srp_eval_batch's evaluation, recording every
 * ray segment's hit triangle and the four posed vertices that bound the window
 * (extreme along u and v).  Holding those fixed -- each segment meets the
 * plane of its recorded triangle, the window spans the recorded vertices --
 * force and torque are smooth in the optical coefficients, the joint angles,
 * the Sun direction and the Sun distance (Sec. 4.3 momentum law, Sec. 4.4.2
 * tracking and clamping, Sec. 6.1 window).  With the caller's cotangents the
 * call returns the derivatives of
 *     L = sum_k g_force[k] . F_k + g_torque[k] . T_k
 * with respect to
 *   g_sun    [n][3]  out: each sun_dir_body entry as given (before the
 *                    normalisation; so g_sun[k] . sun_dir_body[k] = 0);
 *   g_dist   [n]     out: each sun_dist_au entry (needs sun_dist_au; NULL skips);
 *   g_mat    [n_mats][2] out: each material's (rho_s, rho_d), summed over k;
 *   g_angle  [n_parts]   out: the joint parameter of each part, summed over k:
 *                    the commanded angle (SRP_PANELS_SET) or the offset added
 *                    to the tracking angle (SRP_PANELS_TRACK_OFFSET; for
 *                    SRP_PANELS_TRACK the offset at 0).  Zero for rigid parts
 *                    and for joints held at a limit of their interval.
 *   g_quat   [n][4]  out: each quat entry as given (before the normalisation;
 *                    so g_quat[k] . quat[k] = 0); needs quat.
 * With quat (as in srp_eval_batch: sun_dir in the inertial frame, the force
 * output the acceleration R(q) F_body / mass) the cotangent g_force is that of
 * the acceleration and g_sun that of the inertial direction; the attitude
 * enters twice, through the body-frame Sun direction and through the rotation
 * of the force, and g_quat holds both.
 * Sun tracking is differentiated: a tracking joint's angle moves with the Sun
 * direction, and with the angles of the joints above it.
 *   g_force, g_torque [n][3]  in: cotangents (host or device).
 *   force, torque     [n][3]  out (may be NULL): the evaluation itself, equal
 *                    to srp_eval_batch's.
 * Any of g_sun, g_dist, g_mat, g_angle, g_quat may be NULL.  An entry skipped with a
 * negative distance contributes nothing and gets zero gradients.  The result
 * is deterministic (every sum has a fixed order).
 * Errors: as srp_eval_batch; SRP_ERR_ARG when g_force or g_torque is NULL, or
 * g_quat is given without quat.
 */
srp_status srp_grad(srp_ctx *ctx, int32_t mesh_id, const srp_eval_params *params, int32_t n,
                    const double *sun_dir_body, const double *quat, const double *sun_dist_au, const double *g_force,
                    const double *g_torque, double *force, double *torque, double *g_sun, double *g_dist,
                    double *g_mat, double *g_angle, double *g_quat);

/* ---------------------------------------------------- SPAD interpolation */
/*
 * A SPAD table (Sec. 4.2, Sec. 6.1): the force and torque of srp_eval_batch at
 * 1 AU, precomputed for a grid of body-frame Sun directions and interpolated
 * bilinearly in (azimuth, elevation) wherever an SRP force is needed instead
 * of tracing rays.  Sample (i, j), 0 <= i < n_az, 0 <= j < n_el, is the
 * direction (cos el cos az, cos el sin az, sin el) with
 *     az = az0 + i 2 pi / n_az      (periodic: the full circle)
 *     el = el0 + j d_el
 * The paper's tables: n_az = 20, n_el = 10, d_el = pi / 10, from
 * (az0, el0) = (-pi, -pi/2), and shifted by 5 degrees on both axes.
 * Interpolation at a direction s (any length > 0): az = atan2(s_y, s_x),
 * el = atan2(s_z, hypot(s_x, s_y)); azimuth cells wrap from the last sample to
 * the first; beyond the first or last elevation row the row itself is used
 * (no extrapolation).  Force and torque scale as (1 AU / r)^2.
 * Table layout: [n_el][n_az][6] doubles, Fx Fy Fz (N) Tx Ty Tz (N m).
 */
typedef struct {
    int32_t n_az;  /* azimuth samples around the circle (1 .. 2^20)          */
    int32_t n_el;  /* elevation samples (1 .. 2^20); n_az n_el <= 2^24       */
    double az0;    /* first azimuth (rad)                                     */
    double el0;    /* first elevation (rad)                                   */
    double d_el;   /* elevation spacing (rad, > 0)                            */
} srp_spad_grid;

/*
 * Build a SPAD table: one srp_eval_batch evaluation (params: grid N, bounces,
 * P0, panel mode, flags) per sample direction at 1 AU.
 *   table  [n_el][n_az][6] out (host or device; caller-owned)
 * Errors: SRP_ERR_ARG (bad grid or params, NULL table), SRP_ERR_STATE (bad
 * mesh id), and those of srp_eval_batch.
 */
srp_status srp_spad_build(srp_ctx *ctx, int32_t mesh_id, const srp_eval_params *params, const srp_spad_grid *grid,
                          double *table);

/*
 * Interpolate a SPAD table at n body-frame Sun directions.
 *   table        [n_el][n_az][6] (host or device; read only)
 *   sun_dir_body [n][3], sun_dist_au [n] or NULL (= 1 AU; a negative
 *                distance gives zeros)
 *   force, torque [n][3] out (host or device)
 * Errors: SRP_ERR_ARG (bad grid, NULL pointer), SRP_ERR_CUDA.
 */
srp_status srp_spad_eval(srp_ctx *ctx, const srp_spad_grid *grid, const double *table, int32_t n,
                         const double *sun_dir_body, const double *sun_dist_au, double *force, double *torque);

/* ------------------------------------------------------------ propagation */
#define SRP_RKF78 0           /* Fehlberg 7(8) embedded pair, adaptive step      */
#define SRP_RK4 1             /* classical RK4, fixed step h0                    */
#define SRP_CENTRAL_EARTH 0
#define SRP_CENTRAL_SUN 1
#define SRP_ATT_LVLH 0        /* LVLH frame (z to nadir, y along minus the orbit normal)
                                 turned by the constant quaternion q (body -> LVLH)    */
#define SRP_ATT_INERTIAL 1    /* fixed quaternion q (body -> inertial)             */

typedef struct {
    int32_t method;        /* SRP_RKF78 or SRP_RK4                                        */
    int32_t central;       /* SRP_CENTRAL_EARTH or SRP_CENTRAL_SUN                         */
    int32_t j2;            /* Earth J2, pole along inertial z (Earth-centred only)         */
    int32_t sun3;          /* Sun as a third body (Earth-centred only)                     */
    int32_t srp;           /* ray-traced SRP acceleration on (1) or off (0)                */
    int32_t attitude;      /* SRP_ATT_LVLH or SRP_ATT_INERTIAL                             */
    double q[4];           /* attitude quaternion, scalar first (normalised by the library):
                              body -> inertial (SRP_ATT_INERTIAL) or body -> LVLH (SRP_ATT_LVLH;
                              (1, 0, 0, 0) keeps the body on the LVLH axes)                   */
    double epoch_mjd_tt;   /* epoch of t = 0, MJD in TT (Sun ephemeris)                     */
    double rtol;           /* RKF7(8) relative tolerance                                   */
    double atol_pos;       /* absolute tolerance on position components (m)                 */
    double atol_vel;       /* absolute tolerance on velocity components (m/s)               */
    double h0;             /* first step (RKF7(8)) or fixed step (RK4), s                   */
    double h_min;          /* step-size floor (RKF7(8)); below it: SRP_ERR_STEP              */
    double h_max;          /* step-size ceiling (RKF7(8)); 0 = none                          */
    int64_t max_steps;     /* accepted + rejected step budget per trajectory                */
    int32_t poll;          /* steps launched between completion checks (0 = 16)             */
    int32_t host_loop;     /* 0: graph-captured steps; 1: the same kernels issued stage by
                              stage with the host waiting for every stage's SRP result (the
                              pattern of a host integrator calling a GPU force model)       */
    srp_eval_params eval;  /* ray grid, bounces, P0, panel mode of every SRP evaluation     */
    const double *h_replay; /* NULL, or [n_traj][n_replay] step sizes (host or device): RKF7(8)
                               then takes exactly these steps, all accepted, no error control,
                               and ends after n_replay steps (t1 is ignored); this reproduces
                               another integrator's accepted steps                            */
    int64_t n_replay;
    const double *spad_table; /* NULL: trace rays in every stage; else a SPAD table for
                                 spad_grid ([n_el][n_az][6], host or device): the SRP force
                                 is its interpolant (srp_spad_eval) and eval is not used
                                 (srp_propagate only)                                      */
    srp_spad_grid spad_grid;
} srp_prop_params;

typedef struct {
    int64_t steps, rejects, evals; /* accepted steps, rejected steps, SRP evaluations          */
    double t;                      /* time reached (s)                                          */
    int32_t status;                /* SRP_OK or SRP_ERR_STEP                                    */
    int32_t reserved;
    double h_next;                 /* RKF7(8): the step size proposed after the last accepted
                                      step; passing it as h0 with t and y1 resumes the arc as the
                                      integrator would have continued it (RK4: h0)              */
} srp_prop_stats;

/*
 * Propagate n_traj trajectories of one mesh's spacecraft (Sec. 3, Eqs. 1-3):
 * y' = (v, a_g + a_SRP), a_SRP = R(q) F_body / mass with F_body the ray-traced
 * force of srp_eval_batch for the Sun direction in the body frame (zero inside
 * a cylindrical Earth shadow), integrated with RKF7(8) (adaptive: error norm
 * max_i |e_i| / (atol_i + rtol max(|y_i|, |y_new_i|)), accepted when <= 1,
 * next h = h clamp(0.9 err^(-1/8), 0.2, 5), the 7th-order solution kept) or RK4
 * (fixed step).  Every trajectory evaluates the SRP force in every stage; the
 * whole step (stage states, Sun directions, the SRP pipeline for all
 * trajectories, accelerations, step control) is captured once in a CUDA graph
 * and relaunched until every trajectory reached its end time.  With
 * params->spad_table the SRP force of every stage is the SPAD interpolant of
 * that table (Sec. 4.2) instead of a ray-traced evaluation: the step is then
 * the stage, acceleration and control kernels alone.
 *   y0     [n_traj][6]  initial position (m) and velocity (m/s), inertial
 *   t0_t1  [n_traj][2]  start and end time (s after the epoch)
 *   y1     [n_traj][6]  out: state at t1 (or where the trajectory stopped)
 *   stats  [n_traj]     out (may be NULL)
 *   h_log  [n_traj][h_cap] out (may be NULL): accepted step sizes, in order
 * Errors: SRP_ERR_ARG, SRP_ERR_STATE (bad mesh id), SRP_ERR_STEP (some
 * trajectory hit h_min or max_steps; its stats say which), SRP_ERR_STACK,
 * SRP_ERR_CUDA.
 */
srp_status srp_propagate(srp_ctx *ctx, int32_t mesh_id, const srp_prop_params *params, int32_t n_traj,
                         const double *y0, const double *t0_t1, double *y1, srp_prop_stats *stats, double *h_log,
                         int64_t h_cap);

/* ---------------------------------------------------- batched propagation */
/* One trajectory of a heterogeneous batch (srp_propagate_batch). */
typedef struct {
    int32_t mesh_id;        /* a loaded mesh                                                   */
    int32_t N;              /* rays per side of this trajectory's SRP evaluations               */
    int32_t bounces;        /* specular levels                                                  */
    int32_t panel_mode;     /* SRP_PANELS_*                                                     */
    const double *angles;   /* [n_parts] host: commanded angles / tracking offsets, or NULL for
                               the mesh's values (srp_set_panel_angles)                          */
    int32_t central;        /* SRP_CENTRAL_*                                                    */
    int32_t attitude;       /* SRP_ATT_*                                                        */
    double q[4];            /* attitude quaternion, scalar first (see srp_prop_params)          */
    double y0[6];           /* initial position (m) and velocity (m/s), inertial                */
    double t0, t1;          /* start and end time (s after the epoch)                           */
} srp_traj;

/*
 * Propagate a batch of trajectories that may differ in mesh, ray grid, bounce
 * count, joint law, central body and attitude (Sec. 3 Eqs. 1-3 with the
 * evaluation of srp_eval_batch in every stage), in persistent graph-captured
 * rounds.  Every integrator stage evaluates the SRP force of all running
 * trajectories in one pipeline: one launch per kernel covers the work items
 * (trajectory, tile) of every mesh and grid at once (each slot carries its own
 * mesh, grid, bounces, joint values and tile shape).  A round relaunches the
 * captured step until the furthest trajectory is likely done; when half of the
 * running trajectories have finished, the rest are compacted into fewer slots
 * and the step is captured again.  Results equal srp_propagate's for each
 * trajectory alone (same kernels; the per-slot sums do not depend on the batch).
 *   params  shared settings: method, j2, sun3, srp, epoch, tolerances, h0,
 *           h_min, h_max, max_steps, poll, eval.P0, eval.eps_rel; eval.flags may
 *           hold SRP_EVAL_AUTOTUNE (tune the tile shape of every new (mesh, N,
 *           bounces) key first, see srp_autotune) and SRP_EVAL_TRAVERSE (primary
 *           hits by traversal, as for srp_eval_batch).  Its central, attitude, q,
 *           eval.N, eval.bounces, eval.panel_mode, h_replay and host_loop are
 *           ignored: each srp_traj supplies its own.  spad_table must be NULL.
 *   traj    [n] host
 *   y1      [n][6] out; stats [n] out (may be NULL)
 * Errors: SRP_ERR_ARG (a bad field; its index in srp_last_error), SRP_ERR_STATE
 * (bad mesh id), SRP_ERR_STEP, SRP_ERR_STACK, SRP_ERR_OOM, SRP_ERR_CUDA.
 */
srp_status srp_propagate_batch(srp_ctx *ctx, const srp_prop_params *params, int32_t n, const srp_traj *traj,
                               double *y1, srp_prop_stats *stats);

#define SRP_EVAL_AUTOTUNE 4 /* srp_propagate_batch: autotune every new (mesh, N, bounces) key */

/*
 * Autotuner of the trace launch shape: times srp_eval_batch's pipeline on 8
 * fixed Sun directions (a Fibonacci sphere) with each trace tile shape
 * (4 x 8, 8 x 4, 16 x 2 and 32 x 1 pixels per warp), and keeps the fastest for
 * (mesh, params->N, params->bounces) in the context; later evaluations,
 * propagations and batches with that key use it.  Forces and hit decisions do
 * not depend on the tile shape; forces change only by the rounding of the
 * 32-ray FP32 tile sums (below 2e-6 relative).
 *   tile_w  out (may be NULL): the chosen tile width in pixels
 *   ms      out (may be NULL): [4] milliseconds per evaluation of each shape
 * Errors: as srp_eval_batch.
 */
srp_status srp_autotune(srp_ctx *ctx, int32_t mesh_id, const srp_eval_params *params, int32_t *tile_w, double *ms);

/*
 * Set the trace tile width (4, 8, 16 or 32 pixels; the tile is 32 pixels) for
 * (mesh, N, bounces) in the context, as srp_autotune would.  The default is 8.
 * Errors: SRP_ERR_ARG (bad id or width).
 */
srp_status srp_set_tile_shape(srp_ctx *ctx, int32_t mesh_id, int32_t N, int32_t bounces, int32_t tile_w);

/*
 * Discrete adjoint of an RK4 arc (Sec. 3, Eqs. 1-3, with the frozen-hit SRP
 * gradient of srp_grad in every stage).  Propagates like srp_propagate with
 * params->method == SRP_RK4 (fixed step h0, the last step shortened to land on
 * t1; every trajectory must take the same number of steps), then returns the
 * derivatives of
 *     L = sum_i g_y1[i] . y1[i]
 * with respect to the initial states, the optical coefficients, the joint
 * parameters (as srp_grad: commanded angle or offset from the tracking angle)
 * and the attitude quaternion params->q.  Each SRP evaluation keeps the hit set
 * and window vertices it had on the propagated arc, and each stage keeps its
 * lit / shadowed state; gravity (central body, J2, Sun), the Sun direction and
 * distance, the attitude (LVLH turned by q, or q) and the RK4 stage
 * combination are differentiated exactly.
 * Memory: the forward pass keeps the state every ckpt_every steps; the reverse
 * pass recomputes one segment at a time, recording its stage states and hit
 * ids (ckpt_every * 4 * n_traj * N^2 * (bounces + 1) int32 on the device),
 * then sweeps it backward, so each SRP evaluation is traced twice and
 * differentiated once.
 *   g_y1     [n_traj][6]  in: cotangent of the final state
 *   y1       [n_traj][6]  out (may be NULL): final state
 *   g_y0     [n_traj][6]  out (may be NULL)
 *   g_mat    [n_mats][2], g_angle [n_parts], g_q [4]: out (may be NULL), summed
 *                         over the trajectories; g_q is orthogonal to q
 *   stats    [n_traj]     out (may be NULL)
 * Errors: SRP_ERR_ARG (not RK4, step replay, a SPAD table, unequal step
 * counts, ckpt_every < 1), SRP_ERR_STEP (more than max_steps steps), SRP_ERR_OOM,
 * and those of srp_propagate.
 */
srp_status srp_prop_grad(srp_ctx *ctx, int32_t mesh_id, const srp_prop_params *params, int32_t n_traj,
                         const double *y0, const double *t0_t1, const double *g_y1, int32_t ckpt_every, double *y1,
                         double *g_y0, double *g_mat, double *g_angle, double *g_q, srp_prop_stats *stats);

/* Limits of srp_eval_noalloc. */
#define SRP_NOALLOC_MAX_N 1024    /* rays per window side                     */
#define SRP_NOALLOC_MAX_TRIS 4096 /* triangles (every ray tests every one)     */

/*
 * srp_eval_noalloc -- one SRP evaluation that allocates no memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they run, e.g. flight or real-time code
 * whose memory budget is fixed at start-up (an allocation could fail or stall
 * in mid-mission), or hosts whose memory only comes from their own pool.  It
 * needs no srp_ctx (creating one allocates) and calls no cudaMalloc, cudaFree
 * or allocating library routine.
 *
 * It computes the same force and torque as srp_eval_batch for one Sun
 * direction, for a mesh already posed by the caller (no joints), by testing
 * every ray against every triangle in FP64 (no BVH), so it is meant for small
 * meshes.  Its only scratch is a fixed array of 8 + 8 * SRP_NOALLOC_MAX_N^2 / 256
 * doubles (about 256 KiB) in the library's device globals, which every GPU that
 * loads the library holds until the process exits.
 *   tri_xyz  [n_tris][3][3] device, posed vertices (m), counter-clockwise front
 *   tri_mat  [n_tris][2]    device, material of the front, back side; every
 *                           index must lie in [0, n_mats): the kernel reads no
 *                           material for an index outside it, and a ray that
 *                           hits such a side makes force and torque NaN
 *   mat      [n_mats][2]    device, rho_s, rho_d
 *   sun_dir  [3] host, towards the Sun, body frame (normalised here)
 *   c_ref    [3] host, torque reference point
 *   force, torque  [3] device outputs (N, N m)
 *   cuda_stream    stream to launch on (NULL = legacy default stream)
 * Work runs on the current CUDA device and is asynchronous: synchronise the
 * stream before reading the outputs.  The first call on a device looks up the
 * scratch array's device address (kept once it succeeds; a failed lookup is
 * tried again on the next call); make that first call before any stream
 * capture.  A launch error left pending by earlier, unrelated work on the
 * calling thread is cleared, not reported.  All calls share the scratch array, which keeps
 * the last call's contents (each call rewrites all it reads), so calls whose
 * work overlaps on the GPU (other streams, other host threads) race.
 * Errors: SRP_ERR_ARG (null pointer, n_tris outside [1, SRP_NOALLOC_MAX_TRIS],
 * N outside [1, SRP_NOALLOC_MAX_N], bounces outside [0, SRP_MAX_BOUNCES], bad
 * distance / pressure / direction), SRP_ERR_CUDA (device lookup or launch).
 */
srp_status srp_eval_noalloc(const double *tri_xyz, const int32_t *tri_mat, int32_t n_tris, const double *mat,
                            int32_t n_mats, const double sun_dir[3], double sun_dist_au, const double c_ref[3],
                            int32_t N, int32_t bounces, double P0, double eps_rel, double *force, double *torque,
                            void *cuda_stream);

/* ------------------------------------------------------------ diagnostics */
/*
 * Cap on the library's device memory in this process (every context and
 * mesh), in bytes; 0 removes it.  An allocation that would exceed the cap
 * fails with SRP_ERR_OOM, as a full device would; the context stays usable.
 * srp_memory_usage reports the bytes the library holds and the cap.
 * Errors: SRP_ERR_ARG (NULL ctx or outputs).
 */
srp_status srp_set_memory_limit(srp_ctx *ctx, uint64_t bytes);
srp_status srp_memory_usage(srp_ctx *ctx, uint64_t *used, uint64_t *limit);

/*
 * The LSD radix sort of the BVH build (csrc/build.cu): sorts n (key, value)
 * pairs in place by the key bits [0, key_bits), key_bits rounded up to whole
 * bytes (8 bits per pass), stable (equal keys keep their input order).
 * keys [n], vals [n]: host or device.
 * Errors: SRP_ERR_ARG (n < 0, NULL arrays, key_bits outside 1..64),
 * SRP_ERR_OOM, SRP_ERR_CUDA.
 */
srp_status srp_sort_pairs(srp_ctx *ctx, int32_t n, uint64_t *keys, int32_t *vals, int32_t key_bits);

/*
 * Structural check of a mesh's acceleration structure as evaluations use it:
 * the mesh is posed for the body-frame Sun direction (tracking panels; NULL
 * for +z) and refit as in srp_eval_batch, then each part's 4-wide tree is
 * walked from its root on the device.
 *   report [SRP_CHECK_N] out (host):
 *     [0] leaf references (a correct tree has one per triangle: n_tris)
 *     [1] triangles referenced by no leaf or by more than one
 *     [2] child boxes not inside the box their parent holds for them (the
 *         root's not inside the part's root box)
 *     [3] leaf triangles with a vertex outside their leaf box
 *     [4] nodes reached
 *     [5] walks stopped by their bound
 *     [6] triangles of the mesh, [7] parts
 * Errors: SRP_ERR_ARG, SRP_ERR_STATE (bad mesh id), SRP_ERR_OOM, SRP_ERR_CUDA.
 */
#define SRP_CHECK_N 8
srp_status srp_mesh_check(srp_ctx *ctx, int32_t mesh_id, const double *sun_dir_body, int64_t *report);

#ifdef __cplusplus
}
#endif

#endif /* SRP_H */
