// trace.cu -- ray generation, first-hit traversal, SRP shading, specular
// bounces and the force / torque reduction (Sec. 4.3, 6.1).
//
// k_trace (FP32 fast path).  One thread per pixel ray, 16 x 16 pixel tiles
// per block (a warp covers 8 x 4 pixels, so neighbouring rays walk the same
// nodes).  Per segment: stack traversal of each part's binary LBVH (64 B
// nodes fetched as four float4; child boxes slab-tested with the segment's
// current best t), watertight ray/triangle test in FP32 (Woop, Benthin and
// Wald, "Watertight ray/triangle intersection", JCGT 2(1), 2013).  Every FP32
// decision carries an error bound: when an edge function, the self-hit test
// or the nearest-hit comparison is within its bound, the ray is marked for the
// FP64 path and contributes nothing here.  Per hit: absorbed + specular +
// Lambertian momentum, torque about c_ref, specular ray of weight w rho_s.
// Per-ray sums in FP32 (at most 1 + bounces terms), per-thread and block sums
// in FP64 (warp shuffles, then shared memory), one FP64 partial per block.
//
// k_refine (FP64 path).  Re-traces the marked rays from the pixel definition
// with FP64 rays and vertices, the same BVH (boxes are padded well beyond the
// FP32 rounding of the ray) and the same watertight test in FP64.
//
// k_reduce.  Fixed-order FP64 sum of the block partials of one evaluation,
// scaled by P0 / dist^2 times the pixel area.  No atomics on data: results are
// bit-reproducible for a given launch shape.
#include <math.h>

#include "srp_internal.cuh"

namespace srp {

struct PartView {
    const float4 *node;
    const float4 *tri;
    const double *v64;   // v64[3 * (vi - vert_begin) + c]
    int root;            // 0, or ~0 for a one-triangle part
    int limit;           // bound on loop iterations of one part walk (2 n - 1 items)
    int tri_begin, vert_begin, pad_;
    float box[6];
};

struct BlockCtx {
    Frame fr;
    PartView part[kMaxParts];
    int n_parts, n_mats;
    double u[3], v[3], d[3];
    double c_ref[3];
    float cref32[3];
    float delta0;   // bound on the FP32 error of projected coordinates (m), primary segment
    float tau;      // band on t for near ties and the self-hit threshold (m)
    float pad;
};

__device__ __forceinline__ float pick(float x, float y, float z, int k) { return k == 0 ? x : (k == 1 ? y : z); }
__device__ __forceinline__ double pickd(double x, double y, double z, int k) { return k == 0 ? x : (k == 1 ? y : z); }

// Fill the block context of slot s (thread 0), materials (all threads).
__device__ void setup_block(BlockCtx &B, float2 *mat, const TraceArgs &a, int s)
{
    const MeshDev *m = a.mesh_d;
    if (threadIdx.x == 0) {
        const SlotPose &P = a.pose[s];
        double umin = ord_to_dbl(P.wmin_bits[0]), umax = ord_to_dbl(P.wmax_bits[0]);
        double vmin = ord_to_dbl(P.wmin_bits[1]), vmax = ord_to_dbl(P.wmax_bits[1]);
        double wmin = ord_to_dbl(P.wmin_bits[2]), wmax = ord_to_dbl(P.wmax_bits[2]);
        Frame &f = B.fr;
        f.umin = umin; f.vmin = vmin; f.wmin = wmin;
        f.Du = umax - umin; f.Dv = vmax - vmin;
        double Dw = wmax - wmin;
        f.L = sqrt(f.Du * f.Du + f.Dv * f.Dv + Dw * Dw);
        f.eps = a.eps_rel * f.L;
        double w0 = wmin - kStandoff;
        double omax = 0.0;
        for (int k = 0; k < 3; k++) {
            double o = umin * P.u[k] + vmin * P.v[k] + w0 * P.d[k];
            f.org[k] = (float)o;
            f.du[k] = (float)(f.Du / a.N * P.u[k]);
            f.dv[k] = (float)(f.Dv / a.N * P.v[k]);
            f.dir[k] = (float)P.d[k];
            B.u[k] = P.u[k]; B.v[k] = P.v[k]; B.d[k] = P.d[k];
            B.c_ref[k] = m->c_ref[k];
            B.cref32[k] = (float)m->c_ref[k];
            omax = fmax(omax, fabs(o));
        }
        // Magnitude bound of every coordinate and difference the FP32 path forms.
        double R = fmax(m->R, omax + f.Du + f.Dv) + f.L + 2.0 * kStandoff;
        B.delta0 = (float)(16.0 * 5.9604644775390625e-8 * R);
        B.tau = (float)(64.0 * 16.0 * 5.9604644775390625e-8 * R + 1e-6 * f.L);
        B.pad = (float)m->pad;
        B.n_parts = m->n_parts;
        B.n_mats = m->n_mats;
        for (int p = 0; p < m->n_parts; p++) {
            const PartInfo &pi = m->part[p];
            PartView &pv = B.part[p];
            pv.root = pi.tri_count > 1 ? 0 : ~0;
            pv.limit = 2 * pi.tri_count + 8;
            pv.tri_begin = pi.tri_begin;
            pv.vert_begin = pi.vert_begin;
            if (pi.dynamic) {
                pv.node = a.slot.node + ((size_t)s * m->n_dyn_nodes + pi.dyn_node_off) * 4;
                pv.tri = a.slot.tri + ((size_t)s * m->n_dyn_tris + pi.dyn_tri_off) * 3;
                pv.v64 = a.slot.vert64 + ((size_t)s * m->n_dyn_verts + pi.dyn_vert_off) * 3;
                const float *rb = a.slot.root_box + ((size_t)s * kMaxParts + p) * 6;
                for (int k = 0; k < 6; k++) pv.box[k] = rb[k];
            } else {
                pv.node = m->node_static + (size_t)pi.node_begin * 4;
                pv.tri = m->tri_static + (size_t)pi.tri_begin * 3;
                pv.v64 = m->rest64 + (size_t)pi.vert_begin * 3;
                for (int k = 0; k < 6; k++) pv.box[k] = m->root_box_static[p][k];
            }
        }
    }
    for (int i = threadIdx.x; i < m->n_mats; i += blockDim.x) mat[i] = m->mat32[i];
    __syncthreads();
}

// Slab test of one box; returns entry t or +inf.
__device__ __forceinline__ float box_enter(float lx, float hx, float ly, float hy, float lz, float hz, const float *inv,
                                           const float *oi, float tlo, float thi)
{
    float x0 = fmaf(lx, inv[0], -oi[0]), x1 = fmaf(hx, inv[0], -oi[0]);
    float y0 = fmaf(ly, inv[1], -oi[1]), y1 = fmaf(hy, inv[1], -oi[1]);
    float z0 = fmaf(lz, inv[2], -oi[2]), z1 = fmaf(hz, inv[2], -oi[2]);
    float tn = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), tlo));
    float tf = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), thi));
    return tn <= tf ? tn : INFINITY;
}

struct Ray32 {
    float o[3], d[3], inv[3], oi[3];
    float Sx, Sy, Sz;
    int kx, ky, kz;
};

__device__ __forceinline__ void ray_setup(Ray32 &r)
{
    for (int k = 0; k < 3; k++) {
        float dk = r.d[k];
        float ds = fabsf(dk) < 1e-20f ? copysignf(1e-20f, dk) : dk;
        r.inv[k] = 1.0f / ds;
        r.oi[k] = r.o[k] * r.inv[k];
    }
    float ax = fabsf(r.d[0]), ay = fabsf(r.d[1]), az = fabsf(r.d[2]);
    int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    float dz = pick(r.d[0], r.d[1], r.d[2], kz);
    if (dz < 0.f) { int t = kx; kx = ky; ky = t; }
    r.kx = kx; r.ky = ky; r.kz = kz;
    r.Sx = pick(r.d[0], r.d[1], r.d[2], kx) / dz;
    r.Sy = pick(r.d[0], r.d[1], r.d[2], ky) / dz;
    r.Sz = 1.0f / dz;
}

struct Best32 {
    float t;
    int part, tl;
};

// Nearest hit of one segment in FP32.  Returns false when some decision was
// within its error bound (the ray then goes to the FP64 path).
struct Counts {
    float nodes, tris, boxes;
    int flags;
};

template <bool COUNT>
__device__ bool nearest32(const BlockCtx &B, const Ray32 &r, float tlo, int skip, float delta, Best32 &best,
                          Counts &cn)
{
    best.t = INFINITY;
    best.part = -1;
    best.tl = -1;
    const float tau = B.tau;
    int stack[kStack];
    unsigned n_nodes = 0, n_tris = 0, n_boxes = 0;
    bool clean = true;
    for (int p = 0; p < B.n_parts; p++) {
        const PartView &pv = B.part[p];
        float thi = best.t + tau;
        if (box_enter(pv.box[0], pv.box[3], pv.box[1], pv.box[4], pv.box[2], pv.box[5], r.inv, r.oi, tlo - tau,
                      thi) == INFINITY)
            continue;
        int sp = 0, iters = 0;
        int ref = pv.root;
        while (true) {
            if (++iters > pv.limit) { clean = false; cn.flags |= kFlagStack; break; }
            if (ref >= 0) {
                const float4 *nd = pv.node + (size_t)ref * 4;
                float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
                int4 c = __ldg(reinterpret_cast<const int4 *>(nd + 3));
                float th = best.t + tau;
                float t0 = box_enter(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, r.inv, r.oi, tlo - tau, th);
                float t1 = box_enter(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, r.inv, r.oi, tlo - tau, th);
                if (COUNT) { n_nodes++; n_boxes += 2; }
                bool h0 = t0 != INFINITY, h1 = t1 != INFINITY;
                if (h0 && h1) {
                    int nr = t0 <= t1 ? c.x : c.y, fr = t0 <= t1 ? c.y : c.x;
                    if (sp >= kStack) { clean = false; cn.flags |= kFlagStack; break; }
                    stack[sp++] = fr;
                    ref = nr;
                    continue;
                } else if (h0) { ref = c.x; continue; }
                else if (h1) { ref = c.y; continue; }
            } else {
                int tl = ~ref;
                const float4 *tr = pv.tri + (size_t)tl * 3;
                float4 a = __ldg(tr), b = __ldg(tr + 1), c = __ldg(tr + 2);
                if (COUNT) n_tris++;
                if (__float_as_int(a.w) != skip) {
                    // watertight test, FP32, with error bounds
                    float A0 = a.x - r.o[0], A1 = a.y - r.o[1], A2 = a.z - r.o[2];
                    float B0 = b.x - r.o[0], B1 = b.y - r.o[1], B2 = b.z - r.o[2];
                    float C0 = c.x - r.o[0], C1 = c.y - r.o[1], C2 = c.z - r.o[2];
                    float Akz = pick(A0, A1, A2, r.kz), Bkz = pick(B0, B1, B2, r.kz), Ckz = pick(C0, C1, C2, r.kz);
                    float Ax = fmaf(-r.Sx, Akz, pick(A0, A1, A2, r.kx)), Ay = fmaf(-r.Sy, Akz, pick(A0, A1, A2, r.ky));
                    float Bx = fmaf(-r.Sx, Bkz, pick(B0, B1, B2, r.kx)), By = fmaf(-r.Sy, Bkz, pick(B0, B1, B2, r.ky));
                    float Cx = fmaf(-r.Sx, Ckz, pick(C0, C1, C2, r.kx)), Cy = fmaf(-r.Sy, Ckz, pick(C0, C1, C2, r.ky));
                    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
                    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
                    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
                    const float u4 = 4.0f * 5.9604645e-8f;
                    float eU = delta * (fabsf(Bx) + fabsf(By) + fabsf(Cx) + fabsf(Cy)) + u4 * (fabsf(Cx * By) + fabsf(Cy * Bx));
                    float eV = delta * (fabsf(Ax) + fabsf(Ay) + fabsf(Cx) + fabsf(Cy)) + u4 * (fabsf(Ax * Cy) + fabsf(Ay * Cx));
                    float eW = delta * (fabsf(Ax) + fabsf(Ay) + fabsf(Bx) + fabsf(By)) + u4 * (fabsf(Bx * Ay) + fabsf(By * Ax));
                    bool neg = (U < -eU) || (V < -eV) || (W < -eW);
                    bool pos = (U > eU) || (V > eV) || (W > eW);
                    if (!(neg && pos)) {
                        bool unsure = fabsf(U) <= eU || fabsf(V) <= eV || fabsf(W) <= eW;
                        float det = U + V + W;
                        float T = fmaf(U, r.Sz * Akz, fmaf(V, r.Sz * Bkz, W * (r.Sz * Ckz)));
                        float t = T / det;
                        if (unsure) {
                            // near an edge: matters unless the plane is clearly behind or beyond the best hit
                            bool far = (fabsf(det) > 1e-30f) && (t > best.t + tau || t < tlo - tau);
                            if (!far) clean = false;
                        } else {
                            if (fabsf(t - tlo) <= tau || fabsf(t - best.t) <= tau) clean = false;
                            if (t > tlo && t < best.t) { best.t = t; best.part = p; best.tl = tl; }
                        }
                    }
                }
            }
            if (sp == 0) break;
            ref = stack[--sp];
        }
    }
    if (COUNT) { cn.nodes += (float)n_nodes; cn.tris += (float)n_tris; cn.boxes += (float)n_boxes; }
    return clean;
}

__device__ inline double warp_sum(double x)
{
    for (int o = 16; o; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// Partial sums per block (FP64; integer counts are exact below 2^53):
//   0..2 force, 3..5 torque (unscaled), 6 rays sent to / done by the FP64 path,
//   7 segments traced, 8..12 hits per segment level, 13 nodes, 14 triangles,
//   15 box tests.
constexpr int kPart = 16;

// Block-wide FP64 sum of v[0..15] into out[0..15] (fixed order).
__device__ void block_sum16(const double *v, double *out)
{
    __shared__ double red[kPart][kTraceThreads / 32];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = 0; k < kPart; k++) {
        double x = warp_sum(v[k]);
        if (lane == 0) red[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < kPart) {
        double x = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) x += red[threadIdx.x][i];
        out[threadIdx.x] = x;
    }
    __syncthreads();
}

template <bool COUNT>
__global__ void __launch_bounds__(kTraceThreads) k_trace(TraceArgs a)
{
    __shared__ BlockCtx B;
    __shared__ float2 mat[kMaxMats];
    __shared__ int blk_flags;
    int s = blockIdx.y;
    if (threadIdx.x == 0) blk_flags = 0;
    setup_block(B, mat, a, s);
    const int N = a.N;
    int tiles_x = (N + kTile - 1) / kTile;
    int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int i = tx * kTile + (w & 1) * 8 + (lane & 7);
    int j = ty * kTile + (w >> 1) * 4 + (lane >> 3);
    double acc64[kPart];
    for (int k = 0; k < kPart; k++) acc64[k] = 0.0;
    if (i < N && j < N) {
        int ray = i * N + j;
        Ray32 r;
        for (int k = 0; k < 3; k++) {
            r.o[k] = fmaf((float)i + 0.5f, B.fr.du[k], fmaf((float)j + 0.5f, B.fr.dv[k], B.fr.org[k]));
            r.d[k] = B.fr.dir[k];
        }
        float wgt = 1.0f;
        int skip = -1;
        float acc[6] = {0, 0, 0, 0, 0, 0};
        int hits[kMaxBounces + 1];
        for (int k = 0; k <= kMaxBounces; k++) hits[k] = -1;
        bool clean = true;
        int nseg_done = 0;
        Counts cn = {0.f, 0.f, 0.f, 0};
        float delta = B.delta0;
        for (int seg = 0; seg < a.nseg; seg++) {
            ray_setup(r);
            Best32 h;
            float tlo = seg == 0 ? 0.0f : (float)B.fr.eps;
            nseg_done++;
            if (!nearest32<COUNT>(B, r, tlo, skip, delta, h, cn)) { clean = false; break; }
            if (h.part < 0) break;
            const float4 *tr = B.part[h.part].tri + (size_t)h.tl * 3;
            float4 a0 = __ldg(tr), a1 = __ldg(tr + 1), a2 = __ldg(tr + 2);
            int orig = __float_as_int(a0.w);
            unsigned mt = __float_as_uint(a1.w);
            hits[seg] = orig;
            float e1[3] = {a1.x - a0.x, a1.y - a0.y, a1.z - a0.z};
            float e2[3] = {a2.x - a0.x, a2.y - a0.y, a2.z - a0.z};
            float n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
            float il = rsqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            n[0] *= il; n[1] *= il; n[2] *= il;
            float dn = r.d[0] * n[0] + r.d[1] * n[1] + r.d[2] * n[2];
            int side = dn < 0.f ? 0 : 1;
            float sg = side ? -1.f : 1.f;
            float2 m = mat[side ? (mt >> 16) : (mt & 0xffffu)];
            float c = -sg * dn;
            // f = w [(1 - rho_s) d - 2 (rho_s c + rho_d / 3) n_f],  n_f = sg n
            float ka = wgt * (1.0f - m.x), kn = -2.0f * wgt * (m.x * c + m.y * (1.0f / 3.0f)) * sg;
            float F[3], hp[3], arm[3];
            for (int k = 0; k < 3; k++) {
                F[k] = ka * r.d[k] + kn * n[k];
                hp[k] = fmaf(h.t, r.d[k], r.o[k]);
                arm[k] = hp[k] - B.cref32[k];
            }
            acc[0] += F[0]; acc[1] += F[1]; acc[2] += F[2];
            acc[3] += arm[1] * F[2] - arm[2] * F[1];
            acc[4] += arm[2] * F[0] - arm[0] * F[2];
            acc[5] += arm[0] * F[1] - arm[1] * F[0];
            wgt *= m.x;
            if (seg + 1 >= a.nseg || wgt == 0.0f) break;
            for (int k = 0; k < 3; k++) {
                r.o[k] = hp[k];
                r.d[k] = r.d[k] - 2.0f * dn * n[k];
            }
            skip = orig;
            delta = delta * 4.0f;
        }
        if (cn.flags) atomicOr(&blk_flags, cn.flags);
        if (clean) {
            for (int k = 0; k < 6; k++) acc64[k] = (double)acc[k];
            acc64[7] = (double)nseg_done;
            for (int k = 0; k < a.nseg; k++) acc64[8 + k] = hits[k] >= 0 ? 1.0 : 0.0;
            if (a.hits) {
                int32_t *hp = a.hits + ((size_t)s * N * N + ray) * a.nseg;
                for (int k = 0; k < a.nseg; k++) hp[k] = hits[k];
            }
        } else {
            atomicOr(a.amb + (size_t)s * ((N * N + 31) / 32) + (ray >> 5), 1u << (ray & 31));
            acc64[6] = 1.0;
        }
        if (COUNT) { acc64[13] = cn.nodes; acc64[14] = cn.tris; acc64[15] = cn.boxes; }
    }
    __shared__ double out[kPart];
    block_sum16(acc64, out);
    if (threadIdx.x < kPart) a.partials[((size_t)s * a.n_blocks_x + blockIdx.x) * kPart + threadIdx.x] = out[threadIdx.x];
    if (threadIdx.x == 0 && blk_flags) atomicOr(&a.pose[s].flags, blk_flags);
}

// ------------------------------------------------------------- FP64 path
struct Ray64 {
    double o[3], d[3];
    double Sx, Sy, Sz;
    int kx, ky, kz;
};

__device__ void ray64_setup(Ray64 &r)
{
    double ax = fabs(r.d[0]), ay = fabs(r.d[1]), az = fabs(r.d[2]);
    int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    double dz = pickd(r.d[0], r.d[1], r.d[2], kz);
    if (dz < 0.0) { int t = kx; kx = ky; ky = t; }
    r.kx = kx; r.ky = ky; r.kz = kz;
    r.Sx = pickd(r.d[0], r.d[1], r.d[2], kx) / dz;
    r.Sy = pickd(r.d[0], r.d[1], r.d[2], ky) / dz;
    r.Sz = 1.0 / dz;
}

__device__ void tri_v64(const BlockCtx &B, const MeshDev *m, int p, int tl, double *v)
{
    const PartView &pv = B.part[p];
    int t = pv.tri_begin + tl;
    for (int c = 0; c < 3; c++) {
        int vi = m->tri_vidx[3 * t + c] - pv.vert_begin;
        for (int k = 0; k < 3; k++) v[3 * c + k] = pv.v64[3 * vi + k];
    }
}

// Nearest hit in FP64 (same BVH; boxes tested with the rounded ray, whose
// deviation from the FP64 ray is far below the box padding).
__device__ void nearest64(const BlockCtx &B, const MeshDev *m, const Ray64 &r, double tlo, int skip, double &bt,
                          int &bpart, int &btl, int &borig, int &flags)
{
    bt = INFINITY;
    bpart = -1; btl = -1; borig = 0x7fffffff;
    Ray32 q;
    for (int k = 0; k < 3; k++) { q.o[k] = (float)r.o[k]; q.d[k] = (float)r.d[k]; }
    ray_setup(q);
    const float slack = 4.0f * B.pad;
    int stack[kStack];
    for (int p = 0; p < B.n_parts; p++) {
        const PartView &pv = B.part[p];
        float thi = (float)bt + slack;
        if (box_enter(pv.box[0], pv.box[3], pv.box[1], pv.box[4], pv.box[2], pv.box[5], q.inv, q.oi,
                      (float)tlo - slack, thi) == INFINITY)
            continue;
        int sp = 0, ref = pv.root, iters = 0;
        while (true) {
            if (++iters > pv.limit) { flags |= kFlagStack; break; }
            if (ref >= 0) {
                const float4 *nd = pv.node + (size_t)ref * 4;
                float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
                int4 c = __ldg(reinterpret_cast<const int4 *>(nd + 3));
                float th = (float)bt + slack;
                float t0 = box_enter(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, q.inv, q.oi, (float)tlo - slack, th);
                float t1 = box_enter(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, q.inv, q.oi, (float)tlo - slack, th);
                bool h0 = t0 != INFINITY, h1 = t1 != INFINITY;
                if (h0 && h1) {
                    if (sp >= kStack) { flags |= kFlagStack; break; }
                    stack[sp++] = t0 <= t1 ? c.y : c.x;
                    ref = t0 <= t1 ? c.x : c.y;
                    continue;
                } else if (h0) { ref = c.x; continue; }
                else if (h1) { ref = c.y; continue; }
            } else {
                int tl = ~ref;
                int orig = __float_as_int(__ldg(pv.tri + (size_t)tl * 3).w);
                if (orig != skip) {
                    double v[9];
                    tri_v64(B, m, p, tl, v);
                    double A[3], Bv[3], C[3];
                    for (int k = 0; k < 3; k++) { A[k] = v[k] - r.o[k]; Bv[k] = v[3 + k] - r.o[k]; C[k] = v[6 + k] - r.o[k]; }
                    double Akz = pickd(A[0], A[1], A[2], r.kz), Bkz = pickd(Bv[0], Bv[1], Bv[2], r.kz),
                           Ckz = pickd(C[0], C[1], C[2], r.kz);
                    double Ax = pickd(A[0], A[1], A[2], r.kx) - r.Sx * Akz, Ay = pickd(A[0], A[1], A[2], r.ky) - r.Sy * Akz;
                    double Bx = pickd(Bv[0], Bv[1], Bv[2], r.kx) - r.Sx * Bkz, By = pickd(Bv[0], Bv[1], Bv[2], r.ky) - r.Sy * Bkz;
                    double Cx = pickd(C[0], C[1], C[2], r.kx) - r.Sx * Ckz, Cy = pickd(C[0], C[1], C[2], r.ky) - r.Sy * Ckz;
                    double U = __dsub_rn(__dmul_rn(Cx, By), __dmul_rn(Cy, Bx));
                    double V = __dsub_rn(__dmul_rn(Ax, Cy), __dmul_rn(Ay, Cx));
                    double W = __dsub_rn(__dmul_rn(Bx, Ay), __dmul_rn(By, Ax));
                    bool out = (U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0);
                    double det = U + V + W;
                    if (!out && det != 0.0) {
                        double T = U * (r.Sz * Akz) + V * (r.Sz * Bkz) + W * (r.Sz * Ckz);
                        double t = T / det;
                        if (t > tlo && (t < bt || (t == bt && orig < borig))) {
                            bt = t; bpart = p; btl = tl; borig = orig;
                        }
                    }
                }
            }
            if (sp == 0) break;
            ref = stack[--sp];
        }
    }
}

__global__ void __launch_bounds__(kTraceThreads) k_refine(TraceArgs a)
{
    __shared__ BlockCtx B;
    __shared__ float2 mat[kMaxMats];
    __shared__ int any, blk_flags;
    int s = blockIdx.y;
    const int N = a.N;
    size_t R = (size_t)N * N;
    size_t words = (R + 31) / 32;
    uint32_t *amb = a.amb + (size_t)s * words;
    size_t ray0 = (size_t)blockIdx.x * blockDim.x;
    if (threadIdx.x == 0) { any = 0; blk_flags = 0; }
    __syncthreads();
    size_t ray = ray0 + threadIdx.x;
    bool mine = false;
    if (ray < R) mine = (amb[ray >> 5] >> (ray & 31)) & 1u;
    if (mine) any = 1;
    __syncthreads();
    double acc[kPart];
    for (int k = 0; k < kPart; k++) acc[k] = 0.0;
    if (any) {
        setup_block(B, mat, a, s);
        const MeshDev *m = a.mesh_d;
        if (mine) {
            int i = (int)(ray / N), j = (int)(ray % N);
            Ray64 r;
            double uc = B.fr.umin + ((double)i + 0.5) * B.fr.Du / N;
            double vc = B.fr.vmin + ((double)j + 0.5) * B.fr.Dv / N;
            double w0 = B.fr.wmin - kStandoff;
            for (int k = 0; k < 3; k++) { r.o[k] = uc * B.u[k] + vc * B.v[k] + w0 * B.d[k]; r.d[k] = B.d[k]; }
            double wgt = 1.0;
            int skip = -1, nseg_done = 0, flags = 0;
            int32_t *hp = a.hits ? a.hits + ((size_t)s * R + ray) * a.nseg : nullptr;
            if (hp) for (int k = 0; k < a.nseg; k++) hp[k] = -1;
            for (int seg = 0; seg < a.nseg; seg++) {
                ray64_setup(r);
                double t;
                int hpart, htl, horig;
                nseg_done++;
                nearest64(B, m, r, seg == 0 ? 0.0 : B.fr.eps, skip, t, hpart, htl, horig, flags);
                if (hpart < 0) break;
                if (hp) hp[seg] = horig;
                acc[8 + seg] += 1.0;
                double v[9];
                tri_v64(B, m, hpart, htl, v);
                double e1[3], e2[3], n[3];
                for (int k = 0; k < 3; k++) { e1[k] = v[3 + k] - v[k]; e2[k] = v[6 + k] - v[k]; }
                n[0] = e1[1] * e2[2] - e1[2] * e2[1];
                n[1] = e1[2] * e2[0] - e1[0] * e2[2];
                n[2] = e1[0] * e2[1] - e1[1] * e2[0];
                double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
                for (int k = 0; k < 3; k++) n[k] /= nl;
                double dn = r.d[0] * n[0] + r.d[1] * n[1] + r.d[2] * n[2];
                int side = dn < 0.0 ? 0 : 1;
                double sg = side ? -1.0 : 1.0;
                unsigned mt = m->tri_mat[B.part[hpart].tri_begin + htl];
                int mi = side ? (int)(mt >> 16) : (int)(mt & 0xffffu);
                double rs = m->mat64[2 * mi], rd = m->mat64[2 * mi + 1];
                double c = -sg * dn;
                double F[3], x[3];
                for (int k = 0; k < 3; k++) F[k] = wgt * ((1.0 - rs) * r.d[k] - 2.0 * (rs * c + rd / 3.0) * sg * n[k]);
                for (int k = 0; k < 3; k++) x[k] = r.o[k] + t * r.d[k];
                double arm[3] = {x[0] - B.c_ref[0], x[1] - B.c_ref[1], x[2] - B.c_ref[2]};
                acc[0] += F[0]; acc[1] += F[1]; acc[2] += F[2];
                acc[3] += arm[1] * F[2] - arm[2] * F[1];
                acc[4] += arm[2] * F[0] - arm[0] * F[2];
                acc[5] += arm[0] * F[1] - arm[1] * F[0];
                wgt *= rs;
                if (seg + 1 >= a.nseg || wgt == 0.0) break;
                for (int k = 0; k < 3; k++) { r.d[k] = r.d[k] - 2.0 * dn * n[k]; r.o[k] = x[k]; }
                skip = horig;
            }
            acc[6] = 1.0;
            acc[7] = (double)nseg_done;
            if (flags) atomicOr(&blk_flags, flags);
        }
    }
    __syncthreads();
    // clear this block's mask words for the next use of the slot
    if (threadIdx.x < blockDim.x / 32) {
        size_t wi = (ray0 >> 5) + threadIdx.x;
        if (wi < words) amb[wi] = 0u;
    }
    __shared__ double out[kPart];
    block_sum16(acc, out);
    if (threadIdx.x < kPart)
        a.partials_ref[((size_t)s * a.n_blocks_ref + blockIdx.x) * kPart + threadIdx.x] = out[threadIdx.x];
    if (threadIdx.x == 0 && blk_flags) atomicOr(&a.pose[s].flags, blk_flags);
}

// ------------------------------------------------------------- reduce
// One block per slot: fixed-order sums of the trace and refine partials.
// stats_accum[16]: 0 evals, 1 rays, 2 refined rays, 3 segments,
// 4..8 hits per segment, 9 nodes, 10 triangles, 11 box tests.
__global__ void __launch_bounds__(256) k_reduce(TraceArgs a, int eval0, double *force, double *torque, int *err_flags,
                                                unsigned long long *stats_accum)
{
    int s = blockIdx.x;
    __shared__ double red[kPart][256];
    double acc[kPart], accr[kPart];
    for (int k = 0; k < kPart; k++) { acc[k] = 0.0; accr[k] = 0.0; }
    for (int b = threadIdx.x; b < a.n_blocks_x; b += blockDim.x)
        for (int k = 0; k < kPart; k++) acc[k] += a.partials[((size_t)s * a.n_blocks_x + b) * kPart + k];
    for (int b = threadIdx.x; b < a.n_blocks_ref; b += blockDim.x)
        for (int k = 0; k < kPart; k++) accr[k] += a.partials_ref[((size_t)s * a.n_blocks_ref + b) * kPart + k];
    // refined rays: their count is in the refine partials; the trace partial
    // counted the same rays as sent, so take the refine side for slot 6
    for (int k = 0; k < kPart; k++) red[k][threadIdx.x] = (k == 6) ? accr[k] : acc[k] + accr[k];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int k = 0; k < kPart; k++) red[k][threadIdx.x] += red[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const SlotPose &P = a.pose[s];
        double Du = ord_to_dbl(P.wmax_bits[0]) - ord_to_dbl(P.wmin_bits[0]);
        double Dv = ord_to_dbl(P.wmax_bits[1]) - ord_to_dbl(P.wmin_bits[1]);
        double sc = P.scale * (Du * Dv) / ((double)a.N * (double)a.N);
        int e = eval0 + s;
        for (int k = 0; k < 3; k++) {
            force[3 * e + k] = red[k][0] * sc;
            torque[3 * e + k] = red[3 + k][0] * sc;
        }
        if (P.flags) atomicOr(err_flags, P.flags);
        if (stats_accum) {
            atomicAdd(&stats_accum[0], 1ull);
            atomicAdd(&stats_accum[1], (unsigned long long)a.N * (unsigned long long)a.N);
            atomicAdd(&stats_accum[2], (unsigned long long)red[6][0]);
            atomicAdd(&stats_accum[3], (unsigned long long)red[7][0]);
            for (int k = 0; k < 5; k++) atomicAdd(&stats_accum[4 + k], (unsigned long long)red[8 + k][0]);
            for (int k = 0; k < 3; k++) atomicAdd(&stats_accum[9 + k], (unsigned long long)red[13 + k][0]);
        }
    }
}

// ------------------------------------------------------------ launchers
cudaError_t launch_trace(const TraceArgs &a, int S, cudaStream_t st)
{
    dim3 grid(a.n_blocks_x, S);
    if (a.count) k_trace<true><<<grid, kTraceThreads, 0, st>>>(a);
    else k_trace<false><<<grid, kTraceThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_refine(const TraceArgs &a, int S, cudaStream_t st)
{
    dim3 grid(a.n_blocks_ref, S);
    k_refine<<<grid, kTraceThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const TraceArgs &a, int S, int eval0, double *force, double *torque, int *err_flags,
                          unsigned long long *stats_accum, cudaStream_t st)
{
    k_reduce<<<S, 256, 0, st>>>(a, eval0, force, torque, err_flags, stats_accum);
    return cudaGetLastError();
}

}  // namespace srp
