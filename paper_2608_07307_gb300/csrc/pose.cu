// pose.cu -- per-evaluation geometry update (Sec. 4.4.2) and window bounds.
//
//   k_pose      a warp per evaluation slot, a lane per part: joint angles (Sun tracking,
//               commanded, or tracking + offset; clamped), part transforms
//               composed down the kinematic tree (Sec. 4.4.1), image-plane
//               basis, window accumulators reset.
//   k_vertices  four vertices a thread, per slot: posed FP64 position of dynamic
//               vertices; FP64 projections on (u, v, d) reduced to the window
//               min / max (exact, order independent).
//   k_refit     one thread per triangle of the refitted parts: FP32 triangle
//               record from the posed FP64 vertices, leaf box, then bottom-up
//               refit of the 4-wide nodes: the last child to arrive at a node
//               (an acquire-release counter it resets) fits the parent.
#include <math.h>

#include "srp_internal.cuh"

namespace srp {

// Rotation by the angle whose cosine and sine are c, s about unit axis a.
__device__ inline void rot_axis_cs(const double *a, double c, double s, double *R)
{
    const double k = 1.0 - c;
    R[0] = c + k * a[0] * a[0];        R[1] = k * a[0] * a[1] - s * a[2]; R[2] = k * a[0] * a[2] + s * a[1];
    R[3] = k * a[1] * a[0] + s * a[2]; R[4] = c + k * a[1] * a[1];        R[5] = k * a[1] * a[2] - s * a[0];
    R[6] = k * a[2] * a[0] - s * a[1]; R[7] = k * a[2] * a[1] + s * a[0]; R[8] = c + k * a[2] * a[2];
}

constexpr double kPiPose = 3.14159265358979323846;

__global__ void __launch_bounds__(32) k_pose(const SlotDesc *sd, const double *sun_dirs, const double *sun_dist,
                                             double P0, int eval0, int S, SlotPose *pose)
{
    pdl_enter();
    // a warp per slot, a lane per part: the parts of one tree level are posed
    // together (their FP64 chains overlap), each reading its parent's transform
    // from shared memory
    const int slot = blockIdx.x, lane = threadIdx.x;
    if (slot >= S) return;
    __shared__ double sM[kMaxParts][9], sT[kMaxParts][3];
    SlotPose &P = pose[slot];
    const MeshDev *mesh = sd[slot].mesh;
    const double *angles = sd[slot].angles;
    const int panel_mode = sd[slot].panel_mode;
    const int e = eval0 + slot;
    double s[3] = {sun_dirs[3 * e], sun_dirs[3 * e + 1], sun_dirs[3 * e + 2]};
    const double sn = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    for (int k = 0; k < 3; k++) s[k] /= sn;
    const double dist = sun_dist ? sun_dist[e] : 1.0;
    const int skip = dist < 0.0 ? 1 : 0;  // a negative distance asks to skip this evaluation
    if (lane == 0) {
        P.eval = e;
        P.flags = 0;
        P.s_norm = sn;
        P.free_mask = 0;
        P.track_mask = 0;
        P.skip = skip;
    }
    if (skip) return;
    const int np = mesh->n_parts;
    const int p = lane;
    PartInfo pi{};
    if (p < np) pi = mesh->part[p];
    // depth of each part in the kinematic tree (parents precede children)
    const int par = (p < np && p > 0) ? pi.parent : -1;
    int depth = 0;
    for (int q = par, it = 0; it < kMaxParts && __any_sync(0xffffffffu, q >= 0); it++) {
        const int up = __shfl_sync(0xffffffffu, par, q >= 0 ? q : 0);
        if (q >= 0) depth++;
        q = q >= 0 ? up : -1;
    }
    const int levels = __reduce_max_sync(0xffffffffu, p < np ? depth : 0);
    bool track = false, freej = false;
    for (int L = 0; L <= levels; L++) {
        if (p < np && depth == L) {
            double *M = sM[p], *T = sT[p];
            if (p == 0) {
                for (int k = 0; k < 9; k++) M[k] = (k % 4 == 0) ? 1.0 : 0.0;
                T[0] = T[1] = T[2] = 0.0;
            } else {
                const double *Mq = sM[par], *Tq = sT[par];
                // cosine and sine of the joint angle: from the tracking direction itself
                // when the limits cannot clamp it (no FP64 transcendentals), else from the angle
                double th = 0.0, cth = 1.0, sth = 0.0;
                bool have_cs = false;
                if (pi.movable) {
                    if (panel_mode != SRP_PANELS_SET) {
                        // Sun in the parent's current frame: Mq^T s
                        double sl[3];
                        for (int k = 0; k < 3; k++) sl[k] = Mq[k] * s[0] + Mq[3 + k] * s[1] + Mq[6 + k] * s[2];
                        const double *a = pi.axis, *n0 = pi.n0;
                        const double na = n0[0] * a[0] + n0[1] * a[1] + n0[2] * a[2];
                        const double n[3] = {n0[0] - na * a[0], n0[1] - na * a[1], n0[2] - na * a[2]};
                        const double b[3] = {a[1] * n[2] - a[2] * n[1], a[2] * n[0] - a[0] * n[2], a[0] * n[1] - a[1] * n[0]};
                        const double x = n[0] * sl[0] + n[1] * sl[1] + n[2] * sl[2];
                        const double y = b[0] * sl[0] + b[1] * sl[1] + b[2] * sl[2];
                        track = !(x == 0.0 && y == 0.0);
                        const bool plain = panel_mode == SRP_PANELS_TRACK || !angles;
                        if (plain && pi.lim[0] <= -kPiPose && pi.lim[1] >= kPiPose && !(x < 0.0 && fabs(y) <= 1e-12 * -x)) {
                            // atan2(y, x) lies strictly inside (-pi, pi): never clamped, always free
                            const double r = sqrt(x * x + y * y);
                            if (r > 0.0) { cth = x / r; sth = y / r; }
                            have_cs = true;
                            freej = true;
                        }
                        th = (x == 0.0 && y == 0.0) ? 0.0 : (have_cs ? 0.0 : atan2(y, x));
                        if (panel_mode == SRP_PANELS_TRACK_OFFSET && angles) th += angles[p];
                    } else {
                        th = angles ? angles[p] : 0.0;
                    }
                    if (!have_cs) {
                        if (th > pi.lim[0] && th < pi.lim[1]) freej = true;
                        th = fmin(fmax(th, pi.lim[0]), pi.lim[1]);
                        sincos(th, &sth, &cth);
                    }
                }
                double R[9];
                if (pi.movable) rot_axis_cs(pi.axis, cth, sth, R);
                else for (int k = 0; k < 9; k++) R[k] = (k % 4 == 0) ? 1.0 : 0.0;
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++)
                        M[3 * i + j] = Mq[3 * i] * R[j] + Mq[3 * i + 1] * R[3 + j] + Mq[3 * i + 2] * R[6 + j];
                const double *pv = pi.pivot;
                double w[3];
                for (int i = 0; i < 3; i++) w[i] = pv[i] - (R[3 * i] * pv[0] + R[3 * i + 1] * pv[1] + R[3 * i + 2] * pv[2]);
                for (int i = 0; i < 3; i++) T[i] = Mq[3 * i] * w[0] + Mq[3 * i + 1] * w[1] + Mq[3 * i + 2] * w[2] + Tq[i];
            }
            for (int k = 0; k < 9; k++) P.M[p][k] = M[k];
            for (int k = 0; k < 3; k++) P.T[p][k] = T[k];
        }
        __syncwarp();
    }
    const unsigned track_mask = __ballot_sync(0xffffffffu, track);
    const unsigned free_mask = __ballot_sync(0xffffffffu, freej);
    if (lane != 0) return;
    P.track_mask = track_mask;
    P.free_mask = free_mask;
    // basis of the image plane around d = -s (Duff et al., JCGT 2017)
    double d[3] = {-s[0], -s[1], -s[2]};
    double sg = copysign(1.0, d[2]);
    double a = -1.0 / (sg + d[2]);
    double b = d[0] * d[1] * a;
    P.u[0] = 1.0 + sg * d[0] * d[0] * a; P.u[1] = sg * b; P.u[2] = -sg * d[0];
    P.v[0] = b; P.v[1] = sg + d[1] * d[1] * a; P.v[2] = -d[1];
    for (int k = 0; k < 3; k++) { P.d[k] = d[k]; P.s[k] = s[k]; }
    for (int k = 0; k < 3; k++) {
        P.wmin_bits[k] = dbl_to_ord(INFINITY);
        P.wmax_bits[k] = dbl_to_ord(-INFINITY);
    }
    P.scale = P0 / (dist * dist);
}

cudaError_t launch_pose(const SlotDesc *sd, const double *sun_dirs, const double *sun_dist, double P0, int eval0,
                        int S, SlotPose *pose, cudaStream_t st)
{
    return launch_chained(k_pose, dim3(S), dim3(32), 0, st, sd, sun_dirs, sun_dist, P0, eval0, S, pose);
}

// ------------------------------------------------------------- vertices
// vertices a thread: one for a launch of few slots (latency: one vertex's
// chain a thread), four for many (fewer blocks beside the other lanes' traces)
constexpr int kVertsPerThreadMany = 4;
constexpr int kManySlots = 4;

__device__ inline unsigned long long warp_min_u64(unsigned long long x)
{
    for (int o = 16; o; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y < x ? y : x;
    }
    return x;
}
__device__ inline unsigned long long warp_max_u64(unsigned long long x)
{
    for (int o = 16; o; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y > x ? y : x;
    }
    return x;
}

// vpt vertices a thread (strided by the block for coalescing).
// The window bounds are reduced as order-preserving integer images of the
// FP64 projections (exact, order independent, and off the slow FP64 pipe).
__global__ void __launch_bounds__(256) k_vertices(const SlotDesc *sd, SlotPose *pose, int vpt)
{
    pdl_enter();
    const int s = blockIdx.y;
    SlotPose &P = pose[s];
    const MeshDev *mesh = sd[s].mesh;
    const SlotBufs &slot = sd[s].sb;
    const int n_verts = mesh->n_verts;
    const int k0 = blockIdx.x * blockDim.x * vpt;
    if (P.skip || k0 >= n_verts) return;  // uniform over the block
    unsigned long long mn[3], mx[3];
    for (int c = 0; c < 3; c++) { mn[c] = ~0ull; mx[c] = 0ull; }
    const double *ax[3] = {P.u, P.v, P.d};
    for (int q = 0; q < vpt; q++) {
        const int k = k0 + q * blockDim.x + threadIdx.x;
        if (k >= n_verts) break;
        const int p = mesh->vert_part[k];
        const PartInfo &pi = mesh->part[p];
        double x[3] = {mesh->rest64[3 * k], mesh->rest64[3 * k + 1], mesh->rest64[3 * k + 2]};
        if (pi.dynamic) {
            const double *M = P.M[p], *T = P.T[p];
            double y[3];
            for (int i = 0; i < 3; i++) y[i] = M[3 * i] * x[0] + M[3 * i + 1] * x[1] + M[3 * i + 2] * x[2] + T[i];
            size_t o = (size_t)(k - pi.vert_begin + pi.dyn_vert_off) * 3;
            slot.vert64[o] = y[0]; slot.vert64[o + 1] = y[1]; slot.vert64[o + 2] = y[2];
            x[0] = y[0]; x[1] = y[1]; x[2] = y[2];
        }
        double pr[3];
        for (int c = 0; c < 3; c++) {
            pr[c] = ax[c][0] * x[0] + ax[c][1] * x[1] + ax[c][2] * x[2];
            const unsigned long long o = dbl_to_ord(pr[c]);
            mn[c] = o < mn[c] ? o : mn[c];
            mx[c] = o > mx[c] ? o : mx[c];
        }
        // view-frame position of the vertex for the primary-ray test, rounded once
        slot.vview[k] = make_float4((float)pr[0], (float)pr[1], (float)pr[2], 0.f);
        slot.vview64[3 * (size_t)k] = pr[0];
        slot.vview64[3 * (size_t)k + 1] = pr[1];
        slot.vview64[3 * (size_t)k + 2] = pr[2];
    }
    __shared__ unsigned long long smn[3][8], smx[3][8];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = 0; c < 3; c++) {
        const unsigned long long a = warp_min_u64(mn[c]), b = warp_max_u64(mx[c]);
        if (lane == 0) { smn[c][w] = a; smx[c][w] = b; }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int c = threadIdx.x;
        unsigned long long a = smn[c][0], b = smx[c][0];
        for (int i = 1; i < (int)(blockDim.x >> 5); i++) {
            a = smn[c][i] < a ? smn[c][i] : a;
            b = smx[c][i] > b ? smx[c][i] : b;
        }
        if (a <= b) {
            atomicMin(&P.wmin_bits[c], a);
            atomicMax(&P.wmax_bits[c], b);
        }
    }
}

cudaError_t launch_vertices(const SlotDesc *sd, SlotPose *pose, int S, int max_verts, cudaStream_t st)
{
    const int vpt = S >= kManySlots ? kVertsPerThreadMany : 1;
    const int per_block = 256 * vpt;
    dim3 grid((max_verts + per_block - 1) / per_block, S);
    return launch_chained(k_vertices, grid, dim3(256), 0, st, sd, pose, vpt);
}

// ---------------------------------------------------------------- refit
__device__ __forceinline__ unsigned atomic_add_acq_rel(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Thread per sorted triangle: the static parts of one mesh (sd == null, at
// load) or the dynamic parts of every slot's mesh.
__global__ void __launch_bounds__(256) k_refit(const SlotDesc *sd, const SlotPose *pose, const MeshDev *static_mesh,
                                               float4 *node_static, float4 *tri_static, unsigned *counter_static,
                                               float *root_static)
{
    int s = blockIdx.y;
    const int dyn = sd != nullptr;
    const MeshDev *mesh = dyn ? sd[s].mesh : static_mesh;
    const int t0 = dyn ? mesh->n_static_tris : 0, n = dyn ? mesh->n_dyn_tris : mesh->n_static_tris;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    if (dyn && pose[s].skip) return;  // no arrivals in a skipped slot: counter parities stay consistent
    SlotBufs slot{};
    if (dyn) slot = sd[s].sb;
    int t = t0 + idx;
    // part of this sorted triangle: parts are contiguous in sorted order
    int p = -1;
    for (int q = 0; q < mesh->n_parts; q++) {
        const PartInfo &pi = mesh->part[q];
        if (t >= pi.tri_begin && t < pi.tri_begin + pi.tri_count) p = q;
    }
    if (p < 0) return;
    const PartInfo &pi = mesh->part[p];
    float4 *nodes;
    float4 *tris;
    unsigned *cnt;
    float *root;
    int tl = t - pi.tri_begin;
    if (dyn) {
        nodes = slot.node + (size_t)pi.dyn_node_off * kNode4;
        tris = slot.tri + (size_t)pi.dyn_tri_off * 3;
        cnt = slot.counter + pi.dyn_node_off;
        root = slot.root_box + (size_t)p * 6;
    } else {
        nodes = node_static + (size_t)pi.node_begin * kNode4;
        tris = tri_static + (size_t)pi.tri_begin * 3;
        cnt = counter_static + pi.node_begin;
        root = root_static + p * 6;
    }
    // triangle record from FP64 vertices (posed for dynamic parts)
    float v[3][3];
    for (int c = 0; c < 3; c++) {
        int vi = mesh->tri_vidx[3 * t + c];
        const double *x;
        if (dyn) x = slot.vert64 + (size_t)(vi - pi.vert_begin + pi.dyn_vert_off) * 3;
        else x = mesh->rest64 + (size_t)vi * 3;
        v[c][0] = (float)x[0]; v[c][1] = (float)x[1]; v[c][2] = (float)x[2];
    }
    int orig = mesh->tri_orig[t];
    unsigned mt = mesh->tri_mat[t];
    float4 *rec = tris + (size_t)tl * 3;
    rec[0] = make_float4(v[0][0], v[0][1], v[0][2], __int_as_float(orig));
    rec[1] = make_float4(v[1][0], v[1][1], v[1][2], __uint_as_float(mt));
    rec[2] = make_float4(v[2][0], v[2][1], v[2][2], 0.f);
    float pad = (float)mesh->pad;
    float box[6];
    for (int k = 0; k < 3; k++) {
        box[k] = fminf(fminf(v[0][k], v[1][k]), v[2][k]) - pad;
        box[3 + k] = fmaxf(fmaxf(v[0][k], v[1][k]), v[2][k]) + pad;
    }
    // walk up the 4-wide tree: every child stores its box in its slot of the
    // parent; the last of the parent's children to arrive forms the parent's
    // box and resets the counter for the next refit
    int up = mesh->leaf_parent[t];  // (node << 2) | slot, or -1 for a one-triangle part
    for (int guard = 0; up >= 0; guard++) {
        if (guard > kStack + 4) return;  // cannot happen for a tree that passed the depth check
        const int node = up >> 2, slot = up & 3;
        float4 *nd = nodes + (size_t)node * kNode4;
        float *f = reinterpret_cast<float *>(nd);
        f[slot] = box[0];
        f[4 + slot] = box[3];
        f[8 + slot] = box[1];
        f[12 + slot] = box[4];
        f[16 + slot] = box[2];
        f[20 + slot] = box[5];
        const int4 meta = *reinterpret_cast<const int4 *>(nd + 7);  // parent, slot in it, children
        // release: the box above is visible to whoever arrives last; acquire: the
        // last arrival sees every sibling's box
        const unsigned old = atomic_add_acq_rel(cnt + node, 1u);
        if (old + 1u < (unsigned)meta.z) return;  // a sibling still has to arrive
        cnt[node] = 0u;
        float4 c[6];
        for (int k = 0; k < 6; k++) c[k] = __ldcg(nd + k);
        box[0] = fminf(fminf(c[0].x, c[0].y), fminf(c[0].z, c[0].w));
        box[3] = fmaxf(fmaxf(c[1].x, c[1].y), fmaxf(c[1].z, c[1].w));
        box[1] = fminf(fminf(c[2].x, c[2].y), fminf(c[2].z, c[2].w));
        box[4] = fmaxf(fmaxf(c[3].x, c[3].y), fmaxf(c[3].z, c[3].w));
        box[2] = fminf(fminf(c[4].x, c[4].y), fminf(c[4].z, c[4].w));
        box[5] = fmaxf(fmaxf(c[5].x, c[5].y), fmaxf(c[5].z, c[5].w));
        up = meta.x < 0 ? -1 : ((meta.x << 2) | meta.y);
    }
    for (int k = 0; k < 6; k++) root[k] = box[k];
}

cudaError_t launch_refit(const SlotDesc *sd, const SlotPose *pose, int S, int max_dyn_tris, cudaStream_t st)
{
    if (max_dyn_tris <= 0) return cudaSuccess;
    dim3 grid((max_dyn_tris + 255) / 256, S);
    k_refit<<<grid, 256, 0, st>>>(sd, pose, nullptr, nullptr, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_refit_static(const MeshDev *mesh_d, const MeshDev &mh, float4 *node_static, float4 *tri_static,
                                unsigned *counter_static, float *root_static, cudaStream_t st)
{
    if (mh.n_static_tris <= 0) return cudaSuccess;
    dim3 grid((mh.n_static_tris + 255) / 256, 1);
    k_refit<<<grid, 256, 0, st>>>(nullptr, nullptr, mesh_d, node_static, tri_static, counter_static, root_static);
    return cudaGetLastError();
}

}  // namespace srp
