// srp_internal.cuh -- device data layout and kernel launchers of libsrp.
//
// Layout in HBM (one mesh):
//   * triangles are sorted part-major (static parts first, then parts whose
//     pose depends on a joint angle), then by coplanar group, then in Morton
//     order (one scale for all three axes of the part);
//   * each part has its own LBVH over its triangles, built as a binary radix
//     tree and collapsed to 4-wide nodes of 128 B (four child boxes as six
//     float4 in SoA order, four child refs, parent / slot / child count);
//     leaves are triangles;
//   * a triangle record is 48 B: three FP32 vertices + original id +
//     packed front/back material;
//   * FP64 copies of the vertices (rest pose for static parts, posed per slot
//     for dynamic parts) are read only by the FP64 refinement path;
//   * dynamic parts have one copy of their vertices / triangle records /
//     nodes per evaluation "slot", so S evaluations of a batch run at once.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/srp.h"
#include <utility>

// Programmatic dependent launch: a kernel of the evaluation and propagation
// chains is launched while its predecessor in the stream drains, which hides
// the launch gap between dependent kernels.  Every such kernel calls
// pdl_enter() first, in every thread: griddepcontrol.wait returns once the
// predecessor grid has completed and its writes are visible, so no kernel of
// the chain completes before its predecessor and nothing is read or written
// early.  No kernel signals its dependents before it exits (an early signal
// let waiting blocks hold SM slots that the concurrent lanes' kernels needed:
// 2-3% slower).  Launched without the attribute the wait does nothing.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... P, typename... A>
inline cudaError_t launch_chained(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                  A &&...args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}


namespace srp {

constexpr int kMaxParts = SRP_MAX_PARTS;
constexpr int kMaxMats = SRP_MAX_MATS;
constexpr int kMaxBounces = SRP_MAX_BOUNCES;
constexpr int kStack = 96;          // traversal stack entries (>= 3 x 4-wide tree depth + 1, checked at load)
constexpr int kNode4 = 8;           // float4 per 4-wide node
constexpr int kEmptyChild = (int)0x80000000;  // child ref of an unused slot (its box is empty)
constexpr int kTraceThreads = 256;  // 16 x 16 pixel tile per block
constexpr int kTile = 16;
constexpr double kStandoff = 1.0;   // ray origins start 1 m in front of the nearest vertex

// Device error flags (bits of SlotPose::flags / the context error word).
constexpr int kFlagStack = 1;
constexpr int kFlagTimeout = 2;  // a bounded device-side wait gave up (work queue)

// Rotation of the normalised scalar-first quaternion q, row-major.
__device__ __forceinline__ void quat_matrix(const double *q, double *Q)
{
    double w = q[0], x = q[1], yy = q[2], z = q[3];
    double qn = sqrt(w * w + x * x + yy * yy + z * z);
    w /= qn; x /= qn; yy /= qn; z /= qn;
    Q[0] = 1.0 - 2.0 * (yy * yy + z * z); Q[1] = 2.0 * (x * yy - w * z);       Q[2] = 2.0 * (x * z + w * yy);
    Q[3] = 2.0 * (x * yy + w * z);       Q[4] = 1.0 - 2.0 * (x * x + z * z);   Q[5] = 2.0 * (yy * z - w * x);
    Q[6] = 2.0 * (x * z - w * yy);       Q[7] = 2.0 * (yy * z + w * x);       Q[8] = 1.0 - 2.0 * (x * x + yy * yy);
}

// Cotangent g[4] of the quaternion q as given (before its normalisation) from
// the cotangent Qb[9] of its rotation matrix: the derivative of each entry of
// quat_matrix in the normalised components, then the projection of the
// normalisation (g is orthogonal to q).
__device__ __forceinline__ void quat_matrix_vjp(const double *q, const double *Qb, double *out)
{
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w0 = q[0] / qn, x = q[1] / qn, yy = q[2] / qn, z = q[3] / qn;
    double g[4];
    g[0] = -2 * z * Qb[1] + 2 * yy * Qb[2] + 2 * z * Qb[3] - 2 * x * Qb[5] - 2 * yy * Qb[6] + 2 * x * Qb[7];
    g[1] = 2 * yy * Qb[1] + 2 * z * Qb[2] + 2 * yy * Qb[3] - 4 * x * Qb[4] - 2 * w0 * Qb[5] + 2 * z * Qb[6] +
           2 * w0 * Qb[7] - 4 * x * Qb[8];
    g[2] = -4 * yy * Qb[0] + 2 * x * Qb[1] + 2 * w0 * Qb[2] + 2 * x * Qb[3] + 2 * z * Qb[5] - 2 * w0 * Qb[6] +
           2 * z * Qb[7] - 4 * yy * Qb[8];
    g[3] = -4 * z * Qb[0] - 2 * w0 * Qb[1] + 2 * x * Qb[2] + 2 * w0 * Qb[3] - 4 * z * Qb[4] + 2 * yy * Qb[5] +
           2 * x * Qb[6] + 2 * yy * Qb[7];
    double qh[4] = {w0, x, yy, z};
    double gd = g[0] * qh[0] + g[1] * qh[1] + g[2] * qh[2] + g[3] * qh[3];
    for (int k = 0; k < 4; k++) out[k] = (g[k] - gd * qh[k]) / qn;
}

// Static per-part description (host and device copies).
struct PartInfo {
    int parent;         // -1 for the root
    int movable;        // has its own joint
    int dynamic;        // pose depends on some joint angle (itself or an ancestor)
    int tri_begin;      // first sorted triangle of the part (global sorted index)
    int tri_count;
    int node_begin;     // first 4-wide node of the part within its node array
    int vert_begin;     // first vertex of the part (global, part-major re-indexed)
    int vert_count;
    int dyn_tri_off;    // offset of the part in the per-slot dynamic arrays (dynamic only)
    int dyn_node_off;
    int dyn_vert_off;
    int node_count;     // 4-wide nodes of the part (0 for a part of fewer than 2 triangles)
    double pivot[3], axis[3], lim[2], n0[3];
};

// Per-slot pose + window, written by the pose / vertex kernels.
struct SlotPose {
    double M[kMaxParts][9];   // part rotation (row-major), body = M x_rest + T
    double T[kMaxParts][3];
    double s[3];              // unit Sun direction, body frame
    double u[3], v[3], d[3];  // image-plane basis, d = -s
    unsigned long long wmin_bits[3];  // ordered-int encodings of min(u.x), min(v.x), min(d.x)
    unsigned long long wmax_bits[3];
    double scale;             // P0 / dist^2 (multiplied by the pixel area at the end)
    int eval;                 // evaluation index in the batch
    int flags;                // device error flags
    int skip;                 // evaluation skipped (negative Sun distance): every later kernel returns early
    unsigned free_mask;       // bit p: joint p is movable and its angle lies strictly inside its limits
    unsigned track_mask;      // bit p: joint p's angle follows the Sun (tracking, non-degenerate)
    double s_norm;            // length of the Sun direction as given
};

// Per-slot traversal view built from SlotPose by each trace block.
struct Frame {
    float org[3], du[3], dv[3], dir[3];  // FP32 ray generation: o = org + (i+.5) du + (j+.5) dv
    double umin, vmin, wmin, Du, Dv, L, eps;
};

struct MeshDev {
    int n_parts, n_tris, n_verts, n_mats;
    int n_static_tris, n_static_nodes, n_static_verts;
    int n_dyn_tris, n_dyn_nodes, n_dyn_verts;
    int max_depth;
    double pad;                 // absolute AABB padding (m)
    double R;                   // bound on |x| over all poses (m)
    double c_ref[3];
    PartInfo part[kMaxParts];
    int part_order[kMaxParts];  // layout position -> part id (static parts first)
    // device arrays
    double *rest64;        // [n_verts][3] rest pose FP64 (part-major)
    int *vert_part;        // [n_verts]
    int *tri_vidx;         // [n_tris][3] sorted triangles -> global vertex index
    int4 *tri_v4;          // [n_tris] the same, and (part << 24) | index within the part in .w
    int *tri_orig;         // [n_tris] sorted -> original triangle id
    int *tri_pos;          // [n_tris] original triangle id -> sorted position
    unsigned *tri_mat;     // [n_tris] sorted -> (front | back << 16)
    int *leaf_parent;      // [n_tris] sorted -> (parent 4-wide node (part-local) << 2) | slot, -1 for a
                           // single-leaf part
    float4 *tri_static;    // [n_static_tris][3]
    float4 *node_static;   // [n_static_nodes][kNode4]
    int2 *grp;             // [n_tris] sorted -> (part-local 4-wide ref of the subtree holding the triangle's
                           // coplanar group or kEmptyChild, FP32 bits of the group's deviation from its plane
                           // plus the posing error bound, metres)
    float2 *mat32;         // [n_mats] (rho_s, rho_d) FP32
    double *mat64;         // [n_mats][2]
    float root_box_static[kMaxParts][6];
};

// Per-slot dynamic storage (one block of arrays per concurrent evaluation).
struct SlotBufs {
    double *vert64;     // [S][n_dyn_verts][3] posed FP64
    float4 *vview;      // [S][n_verts] (u.x, v.x, d.x, 0) of every posed vertex, FP32 rounded from FP64
    double *vview64;    // [S][n_verts][3] the same projections in FP64 (settling uncertain primary decisions)
    float4 *tri;        // [S][n_dyn_tris][3]
    float4 *node;       // [S][n_dyn_nodes][kNode4]
    unsigned *counter;  // [S][n_dyn_nodes] refit arrival counters (the last arrival resets them)
    float *root_box;    // [S][kMaxParts][6]
};

// One evaluation slot of a launch: what is evaluated there.  A launch may mix
// meshes, grid sizes, bounce counts, joint laws and tile shapes (batched
// propagation); a single-mesh call fills every slot alike.
struct SlotDesc {
    const MeshDev *mesh;   // device copy of the slot's mesh
    SlotBufs sb;           // the slot's own dynamic storage (already offset to the slot)
    const double *angles;  // [n_parts] commanded angles / tracking offsets of the slot
    int N, nseg;           // rays per side; segments per ray (1 + bounces)
    int panel_mode;        // SRP_PANELS_*
    int tile_w;            // trace tile width in pixels (4, 8, 16 or 32); height 32 / tile_w
    int tiles_x, tiles;    // trace tiles across the window, in total
    int tile0;             // first flattened trace block of the slot (blocks of kTraceWarps tiles)
    int rast0;             // work queue: first second-pass raster item of the slot (128 triangles an item)
};

// Partial sums per block (FP64; integer counts are exact below 2^53):
//   0..2 force, 3..5 torque (unscaled), 6 rays sent to / done by the FP64 path,
//   7 segments traced, 8..12 hits per segment level, 13 nodes, 14 triangles,
//   15 box tests, 16..19 FP64 hand-offs by cause (primary edge, secondary
//   edge, near tie, self-hit band).
constexpr int kPart = 20;
constexpr int kCnt = kPart - 6;  // the integer counts (6..19) of a tile partial

// Arguments of the trace / refine kernels.  A trace warp covers one tile of
// kTileRays rays (4 x 8, 8 x 4, 16 x 2 or 32 x 1 pixels).
constexpr int kTileRays = 32;
constexpr int kTraceWarps = 4;  // trace tiles (warps) per block, sharing one context copy
inline int trace_blocks(int tiles) { return (tiles + kTraceWarps - 1) / kTraceWarps; }
constexpr int kRed1 = 64;  // first-level reduction blocks per slot

struct TraceArgs {
    const SlotDesc *sd;          // [S] what each slot evaluates
    int n_slots;                 // S
    int n_tiles;                 // trace blocks of the launch (sum over slots of ceil(tiles / kTraceWarps))
    SlotPose *pose;              // [S] (trace / refine OR their error flags into it)
    unsigned char *tctx;         // [S] per-slot traversal context (k_frame output)
    double eps_rel;
    size_t ray_stride;           // hits: [S][ray_stride][seg_stride]
    int seg_stride;
    int n_blocks_x;              // stride of the per-tile arrays: the largest tile count of a slot
    float *partials;             // [S][n_blocks_x][6] force and torque per tile (FP32 tile sums)
    unsigned *pcounts;           // [S][n_blocks_x][kCnt] counts 6..19 per tile
    double *partials1;           // [S][kRed1][kPart] first-level sums of the tile partials
    unsigned *red_ticket;        // [S] first-level blocks done (the last one adds their sums); reset by the frame kernel
    int *amb_list;               // [S][n_blocks_x][kTileRays] rays handed to the FP64 path, per tile
    int *amb_count;              // [S][n_blocks_x]
    int32_t *hits;               // [S][ray_stride][seg_stride] or null
    int count;                   // gather traversal counters
    // rasterised primary visibility (raster != 0); the pixel buffers are
    // cleared before each launch's raster passes
    int raster;
    int rast_tris;               // largest triangle count of a slot's mesh (raster grid width)
    unsigned long long *pix_key; // [S][ray_stride] nearest certain FP32 hit: t bits << 32 | 7 - (uncertain
                                 // triangles, at most kPixCand + 1) << 29 | part << 24 | tl; ~0 none
    unsigned *pix_cand;          // [S][ray_stride][kPixCand] the first kPixCand uncertain triangles
    int4 *big;                   // [big_cap] (slot, sorted triangle, chunk column, chunk row): chunks of large
                                 // triangles that can meet them
    unsigned *big_count;         // entries claimed in big (reset by k_frame)
    int2 *bigt;                  // [big_cap] (slot, sorted triangle) of the large triangles
    unsigned *bigt_count;        // entries claimed in bigt (reset by k_frame)
    int big_cap;
    int *rast_bad;               // [S] 1: a slot's list entry did not fit; every ray of it traverses
    // diffuse secondary rays (n_diffuse > 0; hits must then be recorded)
    int n_diffuse;
    unsigned diffuse_seed;
    double *dpart;               // [S][kDiffBlocks][6] unscaled force / torque of the diffuse rays
    struct DEmit *demit;         // [S][ray_stride][nseg - 1] emission records of the diffuse rays (dense)
    int *dcnt;                   // [S][ray_stride] emissions of each primary ray, then their exclusive prefix
    int *dtot;                   // [S] emissions of the slot
    int walk_limit_test;         // 1: every BVH walk is bounded at one step (tests of the bound's error path)
    int sum_mode;                // sums above the tile: 0 FP64, 1 compensated FP32, 2 plain FP32
    int ctx_parts, hpt_segs;     // most parts / segments over the launch's slots (the trace kernels' shared memory; 0: the maxima)
    // work queue (queue != 0): the raster's second pass and the trace as one
    // persistent launch; qstate = [head, abort, then per slot: second-pass
    // items done, large-triangle chunks done, chunks listed]
    int queue;
    int n_small_items;           // second-pass items over small triangles, all slots
    int wait_test;               // 1: every trace item's wait targets a count never reached (timeout tests)
    unsigned *qstate;
};
constexpr int kQHead = 0, kQAbort = 1, kQSlot = 2;  // qstate layout; 3 words per slot from kQSlot
constexpr int kQueueBlocksPerSM = 8;
inline size_t qstate_words(size_t slots) { return (size_t)kQSlot + 3 * slots; }
constexpr int kDiffBlocks = 64;  // k_diffuse blocks per slot (fixed: the sums have a fixed order)
// One hit that emits diffuse secondary rays: the FP64 point and lit-side
// normal from the replay of its ray's specular chain, the weight of one sample
// (w rho_d / K), the emitting triangle and the sample counter of sample 0.
struct DEmit {
    double x[3], nf[3], wd;
    int src, pad_;
    unsigned long long c0;
};
constexpr int kPixCand = 2;      // uncertain triangles kept per pixel (more: the ray traverses)
constexpr int kRastSmall = 64;   // largest pixel box one thread rasterises
constexpr int kRastChunk = 16;   // larger triangles: chunks of 16 x 16 pixels, one warp each
constexpr int kRastBigBlocksPerSM = 2;  // k_raster_big grid: blocks of 8 warps per SM and 8 slots, one listed chunk a warp
constexpr int kBigPerSlot = 65536;  // chunk-list entries reserved per slot
size_t trace_ctx_bytes();

// SPAD table (Sec. 4.2, Sec. 6.1): force and torque at 1 AU for a grid of body-frame Sun
// directions, [n_el][n_az][6] (srp_spad_grid gives the sample directions).
struct SpadDev {
    const double *table;  // device; null when the SRP force is ray-traced
    int n_az, n_el;
    double az0, el0, d_el;
};

// Bilinear interpolant of the SPAD table at body-frame direction s and Sun
// distance dist (AU; negative gives zeros): out = [F, T] scaled by 1/dist^2.
// Azimuth is periodic over n_az cells; elevation clamps to the outer rows.
__device__ __forceinline__ void spad_lookup(const SpadDev &g, const double *s, double dist, double out[6])
{
    if (dist < 0.0) {
        for (int k = 0; k < 6; k++) out[k] = 0.0;
        return;
    }
    const double az = atan2(s[1], s[0]);
    const double el = atan2(s[2], hypot(s[0], s[1]));
    double u = (az - g.az0) * (g.n_az * 0.15915494309189535);  // cells of 2 pi / n_az
    u -= floor(u / g.n_az) * g.n_az;                          // into [0, n_az]
    const int i0 = min((int)u, g.n_az - 1);
    const double fa = u - i0;
    const int i1 = i0 + 1 == g.n_az ? 0 : i0 + 1;
    const double v = (el - g.el0) / g.d_el;
    int j0 = 0, j1 = 0;
    double fe = 0.0;
    if (g.n_el > 1 && v > 0.0) {
        if (v >= g.n_el - 1) {
            j0 = j1 = g.n_el - 1;
        } else {
            j0 = (int)v;
            j1 = j0 + 1;
            fe = v - j0;
        }
    }
    const double w00 = (1.0 - fa) * (1.0 - fe), w01 = fa * (1.0 - fe), w10 = (1.0 - fa) * fe, w11 = fa * fe;
    const double *t00 = g.table + 6 * ((size_t)j0 * g.n_az + i0), *t01 = g.table + 6 * ((size_t)j0 * g.n_az + i1);
    const double *t10 = g.table + 6 * ((size_t)j1 * g.n_az + i0), *t11 = g.table + 6 * ((size_t)j1 * g.n_az + i1);
    const double r2 = 1.0 / (dist * dist);
    for (int k = 0; k < 6; k++)
        out[k] = (w00 * __ldg(t00 + k) + w01 * __ldg(t01 + k) + w10 * __ldg(t10 + k) + w11 * __ldg(t11 + k)) * r2;
}

// Propagation settings as seen by the device (from srp_prop_params).
struct PropDev {
    int method, central, j2, sun3, srp, attitude;
    double q[4];
    double epoch_mjd_tt, mass;
    double rtol, atol_pos, atol_vel, h0, h_min, h_max;
    long long max_steps;
    const double *h_replay;  // [n][n_replay] device, or null
    long long n_replay;
    SpadDev spad;            // SPAD table in place of the ray tracer, or spad.table null
};

// Per-trajectory integrator state (device).
struct PropState {
    double t, t1, h, hs;       // time, end time, proposed step, step of the current attempt
    double y[6];               // state (m, m/s), inertial
    double ys[6], ts;          // current stage state and time
    double k[13][6];           // stage derivatives
    double rsun[3];            // Sun position at the stage time
    double R[9];               // body -> inertial at the stage
    long long steps, rejects, evals, nlog;
    int done, status, shadow, pad_;
    int central, attitude;     // per-trajectory force model and attitude law
    double q[4], mass;         // attitude quaternion, spacecraft mass (kg)
    double Qm[9];              // rotation of the normalised q, row-major (fixed per trajectory)
    double rs_st[13][3];       // Sun position at every stage time of the current step
};

// One stage of an RK4 step, recorded for the reverse pass of the propagation adjoint.
struct StageRec {
    double ys[6], ts, hs;  // stage state and time, step size
    double R[9];           // body -> inertial at the stage
    double rsun[3];        // Sun position at the stage time
    double F[3];           // SRP force, body frame (N); zero when not lit
    int lit;               // the SRP evaluation ran (SRP on, not shadowed)
    int pad_;
};

// Reverse-pass state of one trajectory.
struct PropAdj {
    double lam[6];      // cotangent of the state at the current step boundary
    double ybar[4][6];  // cotangents of the current step's stage states
    double kbar[6];     // cotangent of the current stage derivative
    double qbar[4];     // attitude quaternion cotangent, summed over the arc
};

// ordered-int encoding of doubles for atomicMin/Max
__host__ __device__ inline unsigned long long dbl_to_ord(double x)
{
    unsigned long long b;
    memcpy(&b, &x, 8);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double ord_to_dbl(unsigned long long o)
{
    unsigned long long b = (o & 0x8000000000000000ull) ? (o & 0x7fffffffffffffffull) : ~o;
    double x;
    memcpy(&x, &b, 8);
    return x;
}

// ---------------------------------------------------------------- launchers
// build.cu
cudaError_t launch_morton(const double *rest64, const int *tri_vidx, const int *tri_part, const int *rank_of_part,
                          const int *tri_grp, const float *part_lo, const float *part_ext, int n_tris,
                          unsigned long long *keys, int *vals, cudaStream_t st);
cudaError_t radix_sort_pairs(unsigned long long *keys, int *vals, unsigned long long *keys_tmp, int *vals_tmp,
                             int n, int lo_bit, int hi_bit, int *scratch, size_t scratch_ints, cudaStream_t st);
size_t radix_sort_scratch_ints(int n);
cudaError_t launch_karras(const unsigned long long *keys, const int *part_tri_begin, const int *part_tri_count,
                          const int *part_node_begin, int n_parts_layout, int n_internal_total,
                          const int *node_part, int4 *node_refs, int *leaf_parent, cudaStream_t st);
cudaError_t launch_depth(const int4 *node_refs, const int *node_part_base, int n_nodes, int *depth, cudaStream_t st);

// pose.cu
cudaError_t launch_pose(const SlotDesc *sd, const double *sun_dirs, const double *sun_dist, double P0, int eval0,
                        int S, SlotPose *pose, cudaStream_t st);
cudaError_t launch_vertices(const SlotDesc *sd, SlotPose *pose, int S, int max_verts, cudaStream_t st);
// dynamic parts of every slot (max_dyn_tris: the largest count of a slot's mesh)
cudaError_t launch_refit(const SlotDesc *sd, const SlotPose *pose, int S, int max_dyn_tris, cudaStream_t st);
// static parts of one mesh at load
cudaError_t launch_refit_static(const MeshDev *mesh_d, const MeshDev &mh, float4 *node_static, float4 *tri_static,
                                unsigned *counter_static, float *root_static, cudaStream_t st);

// trace.cu
// Per-slot window frame and, when rasterising, the primary visibility passes.
// Raster-related launches of one launch_frame call of S slots (for launch counts).
int raster_launches(int S, bool queue);
cudaError_t launch_frame(const TraceArgs &a, int S, cudaStream_t st);
// The FP32 trace (after launch_frame on the same stream).
// The trace kernels' L1 / shared-memory split (once per process and device).
cudaError_t configure_trace_kernels();
cudaError_t launch_trace(const TraceArgs &a, int S, cudaStream_t st);
cudaError_t launch_reduce(const TraceArgs &a, int S, int eval0, double *force, double *torque, int *err_flags,
                          unsigned long long *stats_accum, cudaStream_t st);

// adjoint.cu: reverse sweep of one evaluation with the hit set frozen
struct AdjArgs {
    const SlotDesc *sd;          // [S]
    const SlotPose *pose;        // [S]
    const int32_t *hits;         // [S][ray_stride][seg_stride] original triangle ids recorded by the trace
    size_t ray_stride;
    int seg_stride;
    const double *sun_dirs;      // [n][3] as given (device)
    const double *sun_dist;      // [n] Sun distance (AU, device) when g_dist is wanted
    const double *g_force;       // [n][3] cotangent of the force (device)
    const double *g_torque;      // [n][3] cotangent of the torque (device)
    int panel_mode, n_mats, n_parts, eval0;
    int nb;                      // ray blocks per slot
    int width;                   // doubles per block partial (kAdjFixed + 2 n_mats + 6 n_parts)
    int *win_ids;                // [S][4] extreme vertices: argmin u, argmax u, argmin v, argmax v
    double *win_val;             // [S][kAdjWinBlocks][4] the window blocks' extreme projections
    int *win_pid;                // [S][kAdjWinBlocks][4] and their vertices
    int n_verts;                 // most vertices of the slots' meshes
    double *partials;            // [S][nb][width]
    double *partials2;           // [S][ceil(nb / kAdjSumRun)][width] runs of kAdjSumRun partials summed, when nb > 2 kAdjSumRun
    double *g_sun;               // [n][3] out
    double *g_dist;              // [n] out, or null
    double *g_eval;              // [n][2 n_mats + n_parts] out: per-evaluation coefficient and angle terms
};
constexpr int kAdjFixed = 14;    // dbar(3) ubar(3) vbar(3) umin umax vmin vmax, sum of the local loss
constexpr int kAdjWinBlocks = 32;  // most blocks a slot's window search uses
constexpr int kAdjSumRun = 32;     // ray-block partials one block of the first summing level adds
int adj_blocks(int S, size_t rays);
cudaError_t launch_adjoint(const AdjArgs &a, int S, cudaStream_t st);
cudaError_t launch_adj_sum(const double *g_eval, int n, int n_mats, int n_parts, double *g_mat, double *g_angle,
                           cudaStream_t st, bool accumulate = false);

// prop.cu
// cfg: null, or [n][8] per trajectory: central, attitude, q[4], mass, unused
cudaError_t launch_prop_init(PropState *S, int n, const double *y0, const double *t01, const PropDev &P,
                             const double *cfg, int *n_done, cudaStream_t st);
cudaError_t launch_prop_stage(PropState *S, int n, const PropDev &P, int stage, double *sun_dir, double *sun_dist,
                              cudaStream_t st);
cudaError_t launch_prop_accel(PropState *S, int n, const PropDev &P, int stage, const double *force, cudaStream_t st,
                              const double *sun_dir = nullptr, const double *sun_dist = nullptr);
// Structural check of slot 0's BVH (csrc/trace.cu, srp_mesh_check): per part a
// walk from the root; tri_seen[n_tris] counts the leaf references of each
// sorted triangle; report[8] (see srp_mesh_check) accumulates violations.
cudaError_t launch_bvh_check(const unsigned char *tctx, int n_parts, int *tri_seen, unsigned long long *report,
                             cudaStream_t st);
// A whole integrator step in one launch (no ray-traced SRP between the stages).
cudaError_t launch_prop_step(PropState *S, int n, const PropDev &P, double *sun_dir, double *sun_dist, int *n_done,
                             double *h_log, int64_t h_cap, cudaStream_t st);
// SPAD (csrc/spad.cu): the sample directions, [n_el][n_az][3]; the interpolant at n directions.
cudaError_t launch_spad_dirs(const SpadDev &g, double *dirs, cudaStream_t st);
cudaError_t launch_spad_eval(const SpadDev &g, int n, const double *dirs, const double *dist, double *force,
                             double *torque, cudaStream_t st);
// The acceleration of `stage`, then the next stage's state; after the last
// stage, step control and the next step's first stage (captured steps).
cudaError_t launch_prop_next(PropState *S, int n, const PropDev &P, int stage, const double *force, double *sun_dir,
                             double *sun_dist, int *n_done, double *h_log, int64_t h_cap, cudaStream_t st);
cudaError_t launch_prop_control(PropState *S, int n, const PropDev &P, int *n_done, double *h_log, int64_t h_cap,
                                cudaStream_t st);
// propagation adjoint (RK4): checkpoints, stage records, reverse stage sweep
cudaError_t launch_prop_ckpt(PropState *S, int n, double *buf, bool save, double h0, cudaStream_t st);
cudaError_t launch_prop_record(const PropState *S, int n, const double *sun, const double *dist, const double *force,
                               StageRec *rec, double *rec_sun, double *rec_dist, cudaStream_t st);
cudaError_t launch_adj_prop_in(int n, const PropDev &P, int stage, const StageRec *rec, PropAdj *A, double *g_force,
                               cudaStream_t st);
cudaError_t launch_adj_prop_out(int n, const PropDev &P, int stage, const StageRec *rec, PropAdj *A,
                                const double *g_sun, const double *g_dist, cudaStream_t st);
cudaError_t launch_adj_prop_step(int n, PropAdj *A, cudaStream_t st);
cudaError_t launch_adj_prop_qsum(int n, const PropAdj *A, double *out, cudaStream_t st);

// attitude.cu: evaluations given in the inertial frame with a body -> inertial
// quaternion per evaluation.  att_in: s_body = R(q)^T s_in (and, when g_in is
// given, g_body = R(q)^T g_in / mass); att_out: force = R(q) F_body / mass;
// att_grad: additionally g_sun = R g_sbody and the quaternion cotangent of
// L = g_acc . R F_body / mass + g_sbody . R^T s_in.
cudaError_t launch_att_in(int n, const double *q, const double *s_in, double *s_body, const double *g_in,
                          double *g_body, double mass, cudaStream_t st);
cudaError_t launch_att_out(int n, const double *q, const double *f_body, double *acc, double mass, cudaStream_t st);
cudaError_t launch_att_grad(int n, const double *q, const double *s_in, const double *f_body, const double *g_acc,
                            const double *g_sbody, double *g_sun, double *g_q, double mass, cudaStream_t st);

}  // namespace srp
