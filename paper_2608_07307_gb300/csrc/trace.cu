// trace.cu -- ray generation, first-hit traversal, SRP shading, specular
// bounces and the force / torque reduction (Sec. 4.3, 6.1).
//
// k_frame.  Once per slot: the window (u, v bounds from the vertex pass), the
// FP32 ray generation, the error bounds of the FP32 decisions and the
// per-part traversal views, into a small context every trace block copies;
// in launches of few slots its extra blocks also clear the pixel keys
// (k_clear_keys otherwise).
//
// k_raster / k_raster_big / k_raster_chunks / k_raster_pass1 (primary visibility).  All primary
// rays of an evaluation are parallel, so each triangle applies the trace's own
// FP32 view-frame test (prim_test) to the pixel centres inside its projected
// box: pass 0 keeps the nearest certain hit per pixel (64-bit atomic minimum of
// depth bits and triangle), pass 1 lists the triangles whose decision there was
// uncertain against it.  Large projected triangles are rasterised in 16 x 16
// pixel chunks, a warp each, listing only the chunks that can meet them
// (k_raster_pass1: the second pass over both kinds in one launch).
//
// k_trace (FP32 fast path).  A block is four warps, each over a 32-pixel tile
// (8 x 4 by default; the shape is chosen per mesh, grid and bounce count by the
// autotuner), sharing one copy of the slot context.  The tiles of every slot of
// a launch form one flat grid, so one launch can trace different meshes, grid
// sizes and bounce counts.  The primary segment takes the raster's nearest
// certain hit and candidates (a pixel with too many candidates, or every pixel
// when rasterisation is off, traverses instead).  Every traversed segment walks
// each part's 4-wide BVH (128 B nodes: six float4 of child boxes in SoA order,
// the near and far planes picked by the ray's octant, and the child refs),
// parts in the order the ray enters their root boxes, with the watertight
// ray/triangle test (Woop, Benthin and Wald, "Watertight ray/triangle
// intersection", JCGT 2(1), 2013):
//   * primary rays share the direction d, so their test runs in the view frame
//     (u, v, d): per-vertex projections computed in FP64 and rounded once to
//     FP32, the ray is the line through the pixel centre (uc, vc) along the
//     third axis, and the watertight shear vanishes;
//   * secondary (specular) rays use the world-frame test with the shear; their
//     origin is rebuilt from the hit's barycentric weights, and they pass over
//     the subtree of their origin's coplanar group.
// Every FP32 decision carries an error bound: when an edge function, the
// nearest-hit comparison or the self-hit threshold is within its bound, the
// triangle is settled in FP64 at the end of the segment (resolve64); only a ray
// with too many such triangles is handed to the FP64 re-trace and contributes
// nothing here.  Per hit:
// absorbed + specular + Lambertian momentum, torque about c_ref, specular ray
// of weight w rho_s.  Per-ray sums in FP32 (at most 1 + bounces terms), tile
// sums by an FP32 butterfly and integer reductions, one partial per tile; the
// tile's handed-off rays go to its own list slot.
//
// resolve64 (FP64, inside k_trace).  When a segment had FP32 decisions within
// their bounds, its uncertain triangles and its nearest certain hit are tested
// again in FP64 against the exact ray of the segment (rare: ~0.5% of the rays
// of a 200k-triangle mesh at 1024^2).
//
// FP64 re-trace (in k_reduce1).  A ray whose uncertain triangles overflow the
// candidate list is re-traced from its pixel definition with FP64 rays and
// vertices, the same BVH (boxes padded well beyond the FP32 rounding of the
// ray; leaves pre-tested in FP32 with a bound, so only triangles not certainly
// missed are tested in FP64) and the same watertight test in FP64.
//
// k_reduce1 (+ k_reduce after diffuse rays).  Fixed-order FP64 sums: contiguous
// ranges of tile partials (and the re-traced rays of those tiles) per
// first-level block, then those per evaluation in block order, by the last
// first-level block of the evaluation to finish (an atomic ticket; without
// diffuse rays) or by k_reduce, scaled by P0 / dist^2 times the pixel area.  No
// atomics on data: results are bit-reproducible.
//
// k_diffuse (optional, Sec. 6.1's diffuse rays).  After the re-trace, a thread per
// (primary ray, sample) replays the ray's specular chain in FP64 through the recorded
// hit triangles and, at each hit with a next level, traces its sample of the K
// cosine-weighted diffuse rays (SplitMix64 stream) in FP32 with the same error bounds,
// settling the uncertain triangles in FP64 (settle64); its per-block FP64 sums are added
// by k_reduce in a fixed order.
//
// k_bvh_check (diagnostics).  One thread per part walks slot 0's 4-wide tree and counts
// leaf references, child boxes outside their parent's and triangles outside their leaf.
#include <math.h>
#include <stddef.h>

#include <algorithm>

#include "srp_internal.cuh"

namespace srp {

constexpr float kU = 5.9604645e-8f;  // unit roundoff of FP32, 2^-24

struct PartView {
    const float4 *node;
    const float4 *tri;   // world-frame triangle records
    const int4 *v4;      // vertex ids of the part's sorted triangles
    const double *v64;   // v64[3 * (vi - vert_begin) + c]
    int root;            // 0, or ~0 for a one-triangle part
    int limit;           // bound on loop iterations of one part walk (nodes + triangles)
    int tri_begin, vert_begin;
    float box[6];        // root box (filled when a block loads the context, from box_src)
    const float *box_src;  // the part's root box: the refit's output for a dynamic part
};

struct TraceCtx {
    // FP32 ray generation: o = org + (i+.5) du + (j+.5) dv; view-frame pixel centres
    float org[3], du[3], dv[3], dir[3];
    float umin32, vmin32, du32, dv32, w0_32;
    float rdu32, rdv32;    // 1 / du32, 1 / dv32 (the raster's conservative pixel boxes)
    float delta_p, tau_p;  // primary: bound on view-frame coordinate error, band on t
    float delta_s;         // secondary: origin-error term added per segment
    float R, L, pad, eps32;
    float cref32[3];
    int n_parts, n_mats;
    int skip;              // evaluation skipped: trace blocks only clear their hand-off count
    const float4 *vview;   // slot's view-frame vertices
    const double *vview64; // the same in FP64
    const float2 *mat32;
    const double *mat64;
    const unsigned *tri_mat;
    const int *tri_vidx;
    const int2 *grp;  // per sorted triangle: subtree of its coplanar group, deviation bound
    const int4 *tri_v4;    // vertex ids of the sorted triangles (the raster's first load)
    int n_tris;
    // FP64 window and basis for the FP64 path
    double umin, vmin, wmin, Du, Dv, Lw, eps;
    double rN;  // 1 / N when N is a power of two (dividing by N is then exactly this product), else 0
    double u[3], v[3], d[3], c_ref[3];
    PartView part[kMaxParts];
};

size_t trace_ctx_bytes() { return sizeof(TraceCtx); }

// The trace kernels' dynamic shared memory: the slot context up to the most
// parts of the launch's slots (16-byte rounded), then the per-thread hit
// columns of the most segments; sized per launch so that the blocks an SM runs
// fit the small shared-memory configuration the kernels ask for.
__host__ __device__ __forceinline__ int trace_parts_cap(int ctx_parts)
{
    return ctx_parts > 0 && ctx_parts < kMaxParts ? ctx_parts : kMaxParts;
}
__host__ __device__ __forceinline__ size_t trace_ctx_dyn_bytes(int ctx_parts)
{
    return (offsetof(TraceCtx, part) + (size_t)trace_parts_cap(ctx_parts) * sizeof(PartView) + 15) / 16 * 16;
}
__host__ __device__ __forceinline__ size_t trace_dyn_bytes(int ctx_parts, int hpt_segs)
{
    const int ns = hpt_segs > 0 && hpt_segs < kMaxBounces + 1 ? hpt_segs : kMaxBounces + 1;
    return trace_ctx_dyn_bytes(ctx_parts) + (size_t)ns * 128 * sizeof(int);
}

// x / N, as a product when N is a power of two (the same value, without an FP64 division)
__device__ __forceinline__ double pix64(double x, double rN, int N) { return rN != 0.0 ? x * rN : x / N; }

__device__ __forceinline__ float pick(float x, float y, float z, int k) { return k == 0 ? x : (k == 1 ? y : z); }
__device__ __forceinline__ double pickd(double x, double y, double z, int k) { return k == 0 ? x : (k == 1 ? y : z); }

// ------------------------------------------------------------- k_frame
__global__ void k_frame(TraceArgs a)
{
    pdl_enter();
    // every load first, then the arithmetic and the stores: a load placed after
    // a store it might alias waits for everything before it, and a chain of such
    // round trips, not the arithmetic, would set this kernel's duration
    const int s = blockIdx.x, lane = threadIdx.x;
    // launches of few slots: every block of the slot sets the pixel keys to all
    // ones (no hit, no candidate) for the raster
    if (a.raster && a.pix_key) {
        unsigned long long *key = a.pix_key + (size_t)s * a.ray_stride;
        const size_t stride = (size_t)gridDim.y * blockDim.x;
        for (size_t i = (size_t)blockIdx.y * blockDim.x + threadIdx.x; i < a.ray_stride; i += stride) key[i] = ~0ull;
    }
    if (blockIdx.y != 0 || lane >= 32) return;  // the context: one warp of the slot
    const SlotDesc &D = a.sd[s];
    const MeshDev *m = D.mesh;
    const SlotBufs sb = D.sb;
    const int N = D.N;
    const SlotPose &P = a.pose[s];
    const int skip = P.skip;
    const int np = m->n_parts;
    PartInfo pi{};
    if (lane < kMaxParts) pi = m->part[lane];
    const float *box_static = lane < kMaxParts ? m->root_box_static[lane] : nullptr;
    const int4 *tri_v4 = m->tri_v4;
    const int n_tris = m->n_tris;
    const float4 *node_static = m->node_static, *tri_static = m->tri_static;
    const double *rest64 = m->rest64;
    double wlo[3], whi[3], u3[3], v3[3], d3[3], cref[3], Rm = 0.0, pad = 0.0;
    int n_mats = 0;
    const float2 *mat32 = nullptr;
    const double *mat64 = nullptr;
    const unsigned *tri_mat = nullptr;
    const int *tri_vidx = nullptr;
    const int2 *grp = nullptr;
    if (lane == 0) {
        for (int k = 0; k < 3; k++) {
            wlo[k] = ord_to_dbl(P.wmin_bits[k]);
            whi[k] = ord_to_dbl(P.wmax_bits[k]);
            u3[k] = P.u[k]; v3[k] = P.v[k]; d3[k] = P.d[k];
            cref[k] = m->c_ref[k];
        }
        Rm = m->R;
        pad = m->pad;
        n_mats = m->n_mats;
        mat32 = m->mat32;
        mat64 = m->mat64;
        tri_mat = m->tri_mat;
        tri_vidx = m->tri_vidx;
        grp = m->grp;
    }
    TraceCtx &B = reinterpret_cast<TraceCtx *>(a.tctx)[s];
    if (lane == 0) {
        B.skip = skip;
        if (a.raster) {
            a.rast_bad[s] = 0;
            if (s == 0) { *a.big_count = 0u; *a.bigt_count = 0u; }
        }
        if (a.queue) {
            for (int k = 0; k < 3; k++) a.qstate[kQSlot + 3 * s + k] = 0u;
            if (s == 0) { a.qstate[kQHead] = 0u; a.qstate[kQAbort] = 0u; }
        }
        B.n_parts = np;
        if (a.red_ticket) a.red_ticket[s] = 0u;
    }
    if (skip) return;
    // the parts' traversal views, a lane each
    if (lane < np) {
        PartView &pv = B.part[lane];
        pv.root = pi.tri_count > 1 ? 0 : ~0;
        pv.limit = a.walk_limit_test ? 1 : pi.node_count + pi.tri_count + 8;
        pv.tri_begin = pi.tri_begin;
        pv.vert_begin = pi.vert_begin;
        pv.v4 = tri_v4 + pi.tri_begin;
        if (pi.dynamic) {
            pv.node = sb.node + (size_t)pi.dyn_node_off * kNode4;
            pv.tri = sb.tri + (size_t)pi.dyn_tri_off * 3;
            pv.v64 = sb.vert64 + (size_t)pi.dyn_vert_off * 3;
            pv.box_src = sb.root_box + (size_t)lane * 6;
        } else {
            pv.node = node_static + (size_t)pi.node_begin * kNode4;
            pv.tri = tri_static + (size_t)pi.tri_begin * 3;
            pv.v64 = rest64 + (size_t)pi.vert_begin * 3;
            pv.box_src = box_static;
        }
    }
    if (lane != 0) return;
    const double umin = wlo[0], umax = whi[0], vmin = wlo[1], vmax = whi[1], wmin = wlo[2], wmax = whi[2];
    const double Du = umax - umin, Dv = vmax - vmin, Dw = wmax - wmin;
    const double Lw = sqrt(Du * Du + Dv * Dv + Dw * Dw);
    const double eps = a.eps_rel * Lw;
    B.umin = umin; B.vmin = vmin; B.wmin = wmin;
    B.rN = (N & (N - 1)) == 0 ? 1.0 / N : 0.0;
    B.Du = Du; B.Dv = Dv;
    B.Lw = Lw;
    B.eps = eps;
    B.eps32 = (float)eps;
    const double w0 = wmin - kStandoff;
    for (int k = 0; k < 3; k++) {
        double o = umin * u3[k] + vmin * v3[k] + w0 * d3[k];
        B.org[k] = (float)o;
        B.du[k] = (float)(Du / N * u3[k]);
        B.dv[k] = (float)(Dv / N * v3[k]);
        B.dir[k] = (float)d3[k];
        B.u[k] = u3[k]; B.v[k] = v3[k]; B.d[k] = d3[k];
        B.c_ref[k] = cref[k];
        B.cref32[k] = (float)cref[k];
    }
    B.umin32 = (float)umin; B.vmin32 = (float)vmin;
    B.du32 = (float)(Du / N); B.dv32 = (float)(Dv / N);
    B.rdu32 = 1.0f / B.du32; B.rdv32 = 1.0f / B.dv32;
    B.w0_32 = (float)w0;
    const double u = 5.9604644775390625e-8;
    // Primary (view frame): vertex projections rounded once (|p| u/2), pixel
    // centres from rounded umin, du and one FMA, differences rounded; the bound
    // doubles that sum.
    const double Mw = fmax(fmax(fabs(umin), fabs(umax)), fmax(fabs(vmin), fabs(vmax)));
    const double Dm = fmax(Du, Dv);
    const float delta_p = (float)(2.0 * u * (3.0 * Mw + 2.0 * Dm));
    B.delta_p = delta_p;
    const double Wm = fmax(fabs(wmin), fabs(wmax)) + kStandoff;
    B.tau_p = (float)(16.0 * u * Wm + 32.0 * delta_p);
    // Secondary (world frame): the origin is rebuilt from the hit's barycentric
    // weights (error ~2 x the previous bound + rounding at |x| <= R, plus the
    // rounding of posed vertices); the per-triangle terms (subtraction, shear,
    // reflected direction) are added in the test from that triangle's distance.
    B.delta_s = (float)(6.0 * u * Rm);
    B.R = (float)Rm;
    B.L = (float)Lw;
    B.pad = (float)pad;
    B.n_mats = n_mats;
    B.vview = sb.vview;
    B.vview64 = sb.vview64;
    B.mat32 = mat32;
    B.mat64 = mat64;
    B.tri_mat = tri_mat;
    B.tri_vidx = tri_vidx;
    B.grp = grp;
    B.tri_v4 = tri_v4;
    B.n_tris = n_tris;
}

// Copy the slot context (header + the parts in use) into shared memory.
__device__ __forceinline__ void load_ctx(TraceCtx &B, const TraceArgs &a, int s)
{
    const TraceCtx *g = reinterpret_cast<const TraceCtx *>(a.tctx) + s;
    // the record up to its last used part view (the part count from the record itself)
    const int np = __ldg(&g->n_parts);
    const int words = (int)((offsetof(TraceCtx, part) + np * sizeof(PartView)) / 4);
    const int *src = reinterpret_cast<const int *>(g);
    int *dst = reinterpret_cast<int *>(&B);
    for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = __ldg(src + k);
    __syncthreads();
    // the root boxes, from where the refit (or the mesh load) left them: the
    // frame kernel that wrote the context did not wait for the refit
    for (int k = threadIdx.x; k < 6 * np; k += blockDim.x) B.part[k / 6].box[k % 6] = B.part[k / 6].box_src[k % 6];
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

// Slab test of one box given its near and far plane on each axis (the planes
// the ray meets first and last): no per-axis ordering needed.
__device__ __forceinline__ float box_enter_nf(float nx, float fx, float ny, float fy, float nz, float fz,
                                              const float *inv, const float *oi, float tlo, float thi)
{
    float tn = fmaxf(fmaxf(fmaf(nx, inv[0], -oi[0]), fmaf(ny, inv[1], -oi[1])), fmaxf(fmaf(nz, inv[2], -oi[2]), tlo));
    float tf = fminf(fminf(fmaf(fx, inv[0], -oi[0]), fmaf(fy, inv[1], -oi[1])), fminf(fmaf(fz, inv[2], -oi[2]), thi));
    return tn <= tf ? tn : INFINITY;
}

__device__ __forceinline__ void cswap(float &ta, int &ra, float &tb, int &rb)
{
    if (tb < ta) {
        float t = ta; ta = tb; tb = t;
        int r = ra; ra = rb; rb = r;
    }
}

// One 4-wide node: slab tests of its four child boxes (lo.x, hi.x, lo.y, hi.y,
// lo.z, hi.z in float4 0..5, one lane per child; child refs in float4 6).
// Bit k of oct is 1 where the ray runs backwards along axis k: the near plane is then
// the box's upper bound, so picking the float4 by address replaces the per-axis
// min/max of the slab test.  An unused slot's box (+inf, -inf) is entered at
// +inf and never hit.  Continues with the nearest child entered and pushes the
// others, farthest first.  Returns the number of children entered (0: pop the
// stack), -1 when the stack would overflow.
__device__ __forceinline__ int node4_step(const float4 *nd, const float *inv, const float *oi, int oct,
                                          float tlo, float thi, int &ref, int *stack, int &sp)
{
    const int ox = oct & 1, oy = (oct >> 1) & 1, oz = (oct >> 2) & 1;
    float4 nx = __ldg(nd + ox), fx = __ldg(nd + 1 - ox), ny = __ldg(nd + 2 + oy),
           fy = __ldg(nd + 3 - oy), nz = __ldg(nd + 4 + oz), fz = __ldg(nd + 5 - oz);
    int4 c = __ldg(reinterpret_cast<const int4 *>(nd + 6));
    float ta = box_enter_nf(nx.x, fx.x, ny.x, fy.x, nz.x, fz.x, inv, oi, tlo, thi);
    float tb = box_enter_nf(nx.y, fx.y, ny.y, fy.y, nz.y, fz.y, inv, oi, tlo, thi);
    float tc = box_enter_nf(nx.z, fx.z, ny.z, fy.z, nz.z, fz.z, inv, oi, tlo, thi);
    float td = box_enter_nf(nx.w, fx.w, ny.w, fy.w, nz.w, fz.w, inv, oi, tlo, thi);
    int ra = c.x, rb = c.y, rc = c.z, rd = c.w;
    cswap(ta, ra, tb, rb);
    cswap(tc, rc, td, rd);
    cswap(ta, ra, tc, rc);
    cswap(tb, rb, td, rd);
    cswap(tb, rb, tc, rc);
    if (ta == INFINITY) return 0;
    const int n = 1 + (tb != INFINITY) + (tc != INFINITY) + (td != INFINITY);
    if (sp + n - 1 > kStack) return -1;
    if (td != INFINITY) stack[sp++] = rd;
    if (tc != INFINITY) stack[sp++] = rc;
    if (tb != INFINITY) stack[sp++] = rb;
    ref = ra;
    return n;
}

struct Ray32 {
    float o[3], d[3], inv[3], oi[3];
    float Sx, Sy, Sz;
    // bits 0-2: 1 where the direction component is negative (the ray's octant);
    // bits 3-4, 5-6, 7-8: the axes kx, ky, kz of the watertight test (one
    // register instead of six)
    int code;
    __device__ __forceinline__ int kx() const { return (code >> 3) & 3; }
    __device__ __forceinline__ int ky() const { return (code >> 5) & 3; }
    __device__ __forceinline__ int kz() const { return (code >> 7) & 3; }
};

__device__ __forceinline__ void ray_setup(Ray32 &r)
{
    int oct = 0;
    for (int k = 0; k < 3; k++) {
        float dk = r.d[k];
        float ds = fabsf(dk) < 1e-20f ? copysignf(1e-20f, dk) : dk;
        r.inv[k] = 1.0f / ds;
        r.oi[k] = r.o[k] * r.inv[k];
        oct |= (r.inv[k] < 0.f ? 1 : 0) << k;
    }
    float ax = fabsf(r.d[0]), ay = fabsf(r.d[1]), az = fabsf(r.d[2]);
    int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    float dz = pick(r.d[0], r.d[1], r.d[2], kz);
    if (dz < 0.f) { int t = kx; kx = ky; ky = t; }
    r.code = oct | (kx << 3) | (ky << 5) | (kz << 7);
    r.Sx = pick(r.d[0], r.d[1], r.d[2], kx) / dz;
    r.Sy = pick(r.d[0], r.d[1], r.d[2], ky) / dz;
    r.Sz = 1.0f / dz;
}

// FP32 view-frame test of one triangle against the primary ray through pixel
// centre (uc, vc): the ray is the third axis, so the edge functions are 2-D
// cross products of the projected vertices (u, v, depth in a, b, c) relative
// to the centre.  Error bounds from the coordinate error delta of the rounded
// projections and centre, plus the rounding of the products.
struct Prim32 {
    float U, V, W, eU, eV, eW, det, T;
};

// The edge functions, determinant and scaled depth without the bounds.
__device__ __forceinline__ Prim32 prim_core(float4 a, float4 b, float4 c, float uc, float vc, float w0)
{
    Prim32 q;
    float Ax = a.x - uc, Ay = a.y - vc, Bx = b.x - uc, By = b.y - vc, Cx = c.x - uc, Cy = c.y - vc;
    q.U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    q.V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    q.W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    q.eU = q.eV = q.eW = 0.0f;
    q.det = q.U + q.V + q.W;
    q.T = fmaf(q.U, a.z - w0, fmaf(q.V, b.z - w0, q.W * (c.z - w0)));
    return q;
}

__device__ __forceinline__ Prim32 prim_test(float4 a, float4 b, float4 c, float uc, float vc, float delta, float w0)
{
    const float u4 = 4.0f * kU;
    Prim32 q;
    float Ax = a.x - uc, Ay = a.y - vc, Bx = b.x - uc, By = b.y - vc, Cx = c.x - uc, Cy = c.y - vc;
    q.U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    q.V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    q.W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    q.eU = delta * (fabsf(Bx) + fabsf(By) + fabsf(Cx) + fabsf(Cy)) + u4 * (fabsf(Cx * By) + fabsf(Cy * Bx));
    q.eV = delta * (fabsf(Ax) + fabsf(Ay) + fabsf(Cx) + fabsf(Cy)) + u4 * (fabsf(Ax * Cy) + fabsf(Ay * Cx));
    q.eW = delta * (fabsf(Ax) + fabsf(Ay) + fabsf(Bx) + fabsf(By)) + u4 * (fabsf(Bx * Ay) + fabsf(By * Ax));
    q.det = q.U + q.V + q.W;
    q.T = fmaf(q.U, a.z - w0, fmaf(q.V, b.z - w0, q.W * (c.z - w0)));
    return q;
}

struct Best32 {
    float t;
    int part, tl;
    float b1, b2;  // barycentric weights of the hit's second and third vertex
};

struct Counts {
    unsigned nodes, tris, boxes;
    unsigned why[4];  // uncertain FP32 decisions: primary edge, secondary edge, near tie, self-hit band
    int flags;
};

// Triangles whose FP32 decision was not certain, for the FP64 resolution at the
// end of the segment (part << 24 | part-local triangle).  The list lives in
// shared memory, one column per thread (entry c at id[c * kLaneStride]) of a
// block-wide array: a per-thread array indexed at run time would sit in local
// memory, and its traffic would compete with the node fetches in L1.
constexpr int kCand = 8;
constexpr int kLaneStride = 128;  // threads of the kernels that keep per-thread columns in shared memory
struct Cands {
    int n;
    int *id;
};

__device__ __forceinline__ bool push_cand(Cands &c, int p, int tl)
{
    if (c.n >= kCand) return false;
    c.id[c.n * kLaneStride] = (p << 24) | tl;
    c.n++;
    return true;
}

// Classify one candidate from its edge functions and depth.  Certain misses and
// certain hits are settled here (best keeps the nearest certain hit); a triangle
// whose decision is within its bound becomes a candidate of the FP64 resolution,
// and so does the best hit it displaces within the tie band.  Returns false when
// the candidate list overflows (the ray then goes to the FP64 re-trace).
template <bool COUNT>
__device__ __forceinline__ bool classify(float U, float V, float W, float eU, float eV, float eW, float T, float det,
                                         float tlo, float tau, int p, int tl, Best32 &best, bool primary, Counts &cn,
                                         Cands &cd)
{
    bool neg = (U < -eU) || (V < -eV) || (W < -eW);
    bool pos = (U > eU) || (V > eV) || (W > eW);
    if (neg && pos) return true;  // certainly outside
    bool unsure = fabsf(U) <= eU || fabsf(V) <= eV || fabsf(W) <= eW;
    float t = T / det;
    if (unsure) {
        // near an edge: matters unless the plane is certainly behind the origin or beyond the best hit
        bool far = (fabsf(det) > 1e-30f) && (t > best.t + tau || t < tlo - tau);
        if (far) return true;
        if (COUNT) cn.why[primary ? 0 : 1]++;
        return push_cand(cd, p, tl);
    }
    bool amb = false;
    if (fabsf(t - tlo) <= tau) { amb = true; if (COUNT) cn.why[3]++; }
    else if (fabsf(t - best.t) <= tau) { amb = true; if (COUNT) cn.why[2]++; }
    if (amb && !push_cand(cd, p, tl)) return false;
    if (t > tlo && t < best.t) {
        if (amb && best.part >= 0 && !push_cand(cd, best.part, best.tl)) return false;
        float id = 1.0f / det;
        best.t = t; best.part = p; best.tl = tl; best.b1 = V * id; best.b2 = W * id;
    }
    return true;
}

// Nearest hit of one segment in FP32.  `primary`: the view-frame test at pixel
// centre (uc, vc); otherwise the world-frame test.  Triangles whose decision
// was within its error bound are collected in cd (settled in FP64 afterwards);
// returns false when they overflow the list or a walk bound is reached (the ray
// then goes to the FP64 re-trace).  A secondary ray leaving the plane of its
// origin's coplanar group passes the group's subtree (ref gskip of part gpart)
// by: none of its triangles can be hit beyond the origin.
template <bool COUNT, bool PRIMARY>
__device__ __forceinline__ bool nearest32(const TraceCtx &B, const Ray32 &r, float uc, float vc, float tlo, int skip,
                                          int gpart, int gskip, float delta, float tau, Best32 &best, Counts &cn,
                                          Cands &cd)
{
    best.t = INFINITY;
    best.part = -1;
    best.tl = -1;
    cd.n = 0;
    int stack[kStack];
    unsigned n_nodes = 0, n_tris = 0, n_boxes = 0;
    bool clean = true;
    const float u4 = 4.0f * kU;
    // parts in the order the ray enters their root boxes: a near hit then culls
    // the parts behind it at their root
    float te[kMaxParts];
    int po[kMaxParts], np = 0;
    for (int p = 0; p < B.n_parts; p++) {
        const PartView &pv = B.part[p];
        if (p == gpart && pv.root == gskip) continue;  // the whole part is the origin's plane
        float t = box_enter(pv.box[0], pv.box[3], pv.box[1], pv.box[4], pv.box[2], pv.box[5], r.inv, r.oi, tlo - tau,
                            INFINITY);
        if (t == INFINITY) continue;
        int k = np++;
        while (k > 0 && te[k - 1] > t) { te[k] = te[k - 1]; po[k] = po[k - 1]; k--; }
        te[k] = t;
        po[k] = p;
    }
    for (int q = 0; q < np; q++) {
        if (te[q] > best.t + tau) break;  // this part and every later one start beyond the best hit
        const int p = po[q];
        const PartView &pv = B.part[p];
        const int gs = p == gpart ? gskip : kEmptyChild;
        int sp = 0, iters = 0;
        int ref = pv.root;
        while (true) {
            if (++iters > pv.limit) { clean = false; cn.flags |= kFlagStack; break; }
            if (ref >= 0) {
                if (ref != gs) {
                    const int n = node4_step(pv.node + (size_t)ref * kNode4, r.inv, r.oi, r.code, tlo - tau,
                                             best.t + tau, ref, stack, sp);
                    if (COUNT) { n_nodes++; n_boxes += 4; }
                    if (n < 0) { clean = false; cn.flags |= kFlagStack; break; }
                    if (n > 0) continue;
                }
            } else {
                int tl = ~ref;
                if (COUNT) n_tris++;
                if (PRIMARY) {
                    int4 vi = __ldg(pv.v4 + tl);
                    const Prim32 q = prim_test(__ldg(B.vview + vi.x), __ldg(B.vview + vi.y), __ldg(B.vview + vi.z), uc,
                                               vc, delta, B.w0_32);
                    if (!classify<COUNT>(q.U, q.V, q.W, q.eU, q.eV, q.eW, q.T, q.det, tlo, tau, p, tl, best, true, cn,
                                         cd)) {
                        clean = false;
                        sp = 0;
                    }
                } else {
                    const float4 *tr = pv.tri + (size_t)tl * 3;
                    float4 a = __ldg(tr), b = __ldg(tr + 1), c = __ldg(tr + 2);
                    if (__float_as_int(a.w) != skip) {
                        float A0 = a.x - r.o[0], A1 = a.y - r.o[1], A2 = a.z - r.o[2];
                        float B0 = b.x - r.o[0], B1 = b.y - r.o[1], B2 = b.z - r.o[2];
                        float C0 = c.x - r.o[0], C1 = c.y - r.o[1], C2 = c.z - r.o[2];
                        float Akz = pick(A0, A1, A2, r.kz()), Bkz = pick(B0, B1, B2, r.kz()), Ckz = pick(C0, C1, C2, r.kz());
                        float Ax = fmaf(-r.Sx, Akz, pick(A0, A1, A2, r.kx())), Ay = fmaf(-r.Sy, Akz, pick(A0, A1, A2, r.ky()));
                        float Bx = fmaf(-r.Sx, Bkz, pick(B0, B1, B2, r.kx())), By = fmaf(-r.Sy, Bkz, pick(B0, B1, B2, r.ky()));
                        float Cx = fmaf(-r.Sx, Ckz, pick(C0, C1, C2, r.kx())), Cy = fmaf(-r.Sy, Ckz, pick(C0, C1, C2, r.ky()));
                        float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
                        float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
                        float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
                        // coordinate error: origin error (delta) + subtraction, shear and
                        // reflected-direction rounding, growing with this triangle's distance
                        const float mxy = fmaxf(fmaxf(fabsf(Ax), fabsf(Bx)), fabsf(Cx)), myy = fmaxf(fmaxf(fabsf(Ay), fabsf(By)), fabsf(Cy));
                        float dz = fmaxf(fmaxf(fabsf(Akz), fabsf(Bkz)), fabsf(Ckz)) + mxy + myy;
                        float dc = fmaf(16.0f * kU, dz, delta);
                        // the common case first: with M the largest |x|, |y| of the three
                        // vertices, every edge function's bound below is at most
                        // 4 M dc + 2 M^2 u4 (the factor covers this sum's own rounding);
                        // an edge function beyond it on each side is a certain miss, as
                        // classify would find with the exact bounds
                        const float Mv = fmaxf(mxy, myy);
                        if (Mv > 1e-18f) {
                            const float Eb = fmaf(dc, 4.0f * Mv, (2.0f * u4) * Mv * Mv) * 1.001f;
                            if (fminf(fminf(U, V), W) < -Eb && fmaxf(fmaxf(U, V), W) > Eb) {
                                if (sp == 0) break;
                                ref = stack[--sp];
                                continue;
                            }
                        }
                        float eU = dc * (fabsf(Bx) + fabsf(By) + fabsf(Cx) + fabsf(Cy)) + u4 * (fabsf(Cx * By) + fabsf(Cy * Bx));
                        float eV = dc * (fabsf(Ax) + fabsf(Ay) + fabsf(Cx) + fabsf(Cy)) + u4 * (fabsf(Ax * Cy) + fabsf(Ay * Cx));
                        float eW = dc * (fabsf(Ax) + fabsf(Ay) + fabsf(Bx) + fabsf(By)) + u4 * (fabsf(Bx * Ay) + fabsf(By * Ax));
                        float det = U + V + W;
                        float T = fmaf(U, r.Sz * Akz, fmaf(V, r.Sz * Bkz, W * (r.Sz * Ckz)));
                        if (!classify<COUNT>(U, V, W, eU, eV, eW, T, det, tlo, tau, p, tl, best, false, cn, cd)) { clean = false; sp = 0; }
                    }
                }
            }
            // a handed-off ray (overflow) is re-traced from scratch: its stack was emptied
            if (sp == 0) break;
            ref = stack[--sp];
        }
    }
    if (COUNT) { cn.nodes += n_nodes; cn.tris += n_tris; cn.boxes += n_boxes; }
    return clean;
}

// The primary segment's traversal (a pixel whose raster result is not usable:
// too many uncertain candidates, or rasterisation off): rare, so kept out of
// line, where its registers do not weigh on the rest of the trace kernel.
struct Near32 {
    Best32 b;
    Counts cn;
    int cand_n;
    int ok;
};

template <bool COUNT>
__device__ __noinline__ Near32 nearest32_primary(const TraceCtx &B, const Ray32 r, float uc, float vc, float delta,
                                                 float tau, Counts cn, Cands cd)
{
    Near32 o;
    o.ok = nearest32<COUNT, true>(B, r, uc, vc, 0.0f, -1, -1, kEmptyChild, delta, tau, o.b, cn, cd) ? 1 : 0;
    o.cn = cn;
    o.cand_n = cd.n;
    return o;
}

// Compensated FP32 sums (the Kahan-Babuska form of compensated summation):
// the value is hi + lo, lo collecting the exact rounding error of every
// addition into hi (Knuth's TwoSum), so the sum keeps about twice FP32's
// precision without FP64 arithmetic.
struct Comp32 {
    float hi, lo;
};
__device__ __forceinline__ void comp_add(Comp32 &c, float x)
{
    const float s = __fadd_rn(c.hi, x);
    const float bp = __fsub_rn(s, c.hi);
    const float e = __fadd_rn(__fsub_rn(c.hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    c.hi = s;
    c.lo = __fadd_rn(c.lo, e);
}
__device__ __forceinline__ void comp_merge(Comp32 &c, const Comp32 &d)
{
    comp_add(c, d.hi);
    c.lo = __fadd_rn(c.lo, d.lo);
}
__device__ __forceinline__ float comp_value(const Comp32 &c) { return __fadd_rn(c.hi, c.lo); }

__device__ inline double warp_sum(double x)
{
    for (int o = 16; o; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// Block-wide FP64 sum of v[0..kPart) into out[0..kPart) (fixed order).
__device__ void block_sum(const double *v, double *out)
{
    __shared__ double red[kPart][32];
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

// Slot of flattened trace block g: the last slot whose first block is <= g.
__device__ __forceinline__ int slot_of_block(const SlotDesc *sd, int S, int g)
{
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&sd[mid].tile0) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __noinline__ Best32 resolve64(const TraceCtx &B, int N, int i, int j, int seg, const int *hpt, int skip,
                                         Cands cd, Best32 best);

// One warp per block, one 32-pixel tile (tile_w x 32 / tile_w) per block; the
// blocks of all slots form one flat grid.  Latency bound: 32 warps per SM at
// the kernel's 64 registers (no spills).
// ------------------------------------------------------------- raster
// Primary visibility by rasterisation.  Every primary ray of an evaluation runs
// along the same direction d from its pixel centre, so the nearest hit of a
// pixel is the nearest triangle whose view-frame projection covers the centre:
// each triangle visits the pixel centres of its projected box and applies the
// very test the traversal would (prim_test).  Pass 0 keeps, per pixel, the
// nearest certain hit (64-bit atomic minimum of depth bits and triangle).
// Pass 1 lists the pixel's triangles the FP32 test could not settle against
// that minimum: uncertain edge decisions not certainly beyond it, and certain
// hits within its depth band (what the traversal sends to its FP64
// resolution).  The trace then settles those candidates in FP64 exactly as
// after a traversal; a pixel with more than kPixCand of them traverses.

struct RastView {
    const float4 *vview;
    float umin32, vmin32, du32, dv32, rdu32, rdv32, w0, delta, tau;
    int N;
};

__device__ __forceinline__ RastView rast_view(const TraceArgs &a, int s)
{
    const TraceCtx *g = reinterpret_cast<const TraceCtx *>(a.tctx) + s;
    RastView V;
    V.vview = g->vview;
    V.umin32 = g->umin32; V.vmin32 = g->vmin32; V.du32 = g->du32; V.dv32 = g->dv32;
    V.rdu32 = g->rdu32; V.rdv32 = g->rdv32;
    V.w0 = g->w0_32; V.delta = g->delta_p; V.tau = g->tau_p;
    V.N = a.sd[s].N;
    return V;
}

// Pixels whose centre lies within the triangle's projected box widened by a
// hundredth of a pixel plus 64 delta: every other centre is outside the exact
// projection by more than the coordinate error, so the pixel cannot be hit.
__device__ __forceinline__ bool rast_box(const RastView &V, float4 a, float4 b, float4 c, int &i0, int &i1, int &j0,
                                         int &j1)
{
    const float mu = 0.01f * V.du32 + 64.0f * V.delta, mv = 0.01f * V.dv32 + 64.0f * V.delta;
    const float lim = (float)V.N + 1.0f;
    // products with the reciprocal pixel sizes: their rounding (~1e-4 pixel at
    // N = 1024) is far inside the hundredth of a pixel the box is widened by
    float ulo = (fminf(fminf(a.x, b.x), c.x) - mu - V.umin32) * V.rdu32 - 0.5f;
    float uhi = (fmaxf(fmaxf(a.x, b.x), c.x) + mu - V.umin32) * V.rdu32 - 0.5f;
    float vlo = (fminf(fminf(a.y, b.y), c.y) - mv - V.vmin32) * V.rdv32 - 0.5f;
    float vhi = (fmaxf(fmaxf(a.y, b.y), c.y) + mv - V.vmin32) * V.rdv32 - 0.5f;
    ulo = fminf(fmaxf(ulo, -1.0f), lim); uhi = fminf(fmaxf(uhi, -1.0f), lim);
    vlo = fminf(fmaxf(vlo, -1.0f), lim); vhi = fminf(fmaxf(vhi, -1.0f), lim);
    i0 = max((int)ceilf(ulo), 0); i1 = min((int)floorf(uhi), V.N - 1);
    j0 = max((int)ceilf(vlo), 0); j1 = min((int)floorf(vhi), V.N - 1);
    return i0 <= i1 && j0 <= j1;
}

// Can pixel centres [ib, ie] x [jb, je] meet the projected triangle?  False
// only when all four corners lie more than a pixel outside one edge line.
__device__ __forceinline__ bool chunk_meets(const RastView &V, float4 a, float4 b, float4 c, int ib, int ie, int jb,
                                            int je)
{
    const float u0 = fmaf((float)ib + 0.5f, V.du32, V.umin32), u1 = fmaf((float)ie + 0.5f, V.du32, V.umin32);
    const float v0 = fmaf((float)jb + 0.5f, V.dv32, V.vmin32), v1 = fmaf((float)je + 0.5f, V.dv32, V.vmin32);
    const float area = (b.x - a.x) * (c.y - a.y) - (b.y - a.y) * (c.x - a.x);
    const float pix = V.du32 + V.dv32;
    if (!(fabsf(area) > 1e-3f * pix * pix)) return true;  // sliver: keep every chunk
    const float sg = area > 0.0f ? 1.0f : -1.0f;
    const float px[3] = {a.x, b.x, c.x}, py[3] = {a.y, b.y, c.y};
    for (int e = 0; e < 3; e++) {
        const int f = e == 2 ? 0 : e + 1;
        const float ex = px[f] - px[e], ey = py[f] - py[e];
        const float m = pix * (fabsf(ex) + fabsf(ey));
        // edge function, positive inside: sg ((q - p) x (x - p))
        const float e00 = sg * (ex * (v0 - py[e]) - ey * (u0 - px[e]));
        const float e01 = sg * (ex * (v1 - py[e]) - ey * (u0 - px[e]));
        const float e10 = sg * (ex * (v0 - py[e]) - ey * (u1 - px[e]));
        const float e11 = sg * (ex * (v1 - py[e]) - ey * (u1 - px[e]));
        if (fmaxf(fmaxf(e00, e01), fmaxf(e10, e11)) < -m) return false;
    }
    return true;
}

// An upper bound, over the pixel centres [i0, i1] x [j0, j1], of the error
// bounds prim_test forms for the triangle: every coordinate relative to a
// centre is at most xm (u) or ym (v) in size, and FP32 rounding is monotone.
__device__ __forceinline__ float rast_bound(const RastView &V, float4 a, float4 b, float4 c, int i0, int i1, int j0,
                                            int j1)
{
    const float u0 = fmaf((float)i0 + 0.5f, V.du32, V.umin32), u1 = fmaf((float)i1 + 0.5f, V.du32, V.umin32);
    const float v0 = fmaf((float)j0 + 0.5f, V.dv32, V.vmin32), v1 = fmaf((float)j1 + 0.5f, V.dv32, V.vmin32);
    const float xm = fmaxf(fmaxf(fmaxf(fabsf(a.x - u0), fabsf(a.x - u1)), fmaxf(fabsf(b.x - u0), fabsf(b.x - u1))),
                           fmaxf(fabsf(c.x - u0), fabsf(c.x - u1)));
    const float ym = fmaxf(fmaxf(fmaxf(fabsf(a.y - v0), fabsf(a.y - v1)), fmaxf(fabsf(b.y - v0), fabsf(b.y - v1))),
                           fmaxf(fabsf(c.y - v0), fabsf(c.y - v1)));
    return (V.delta * (2.0f * xm + 2.0f * ym) + 4.0f * kU * (2.0f * xm * ym)) * 1.001f;
}

// The pixel key (one 64-bit word per pixel): the nearest certain hit's depth
// bits in the high word; in the low word a 3-bit field (bits 29-31) holding 7
// minus the number of uncertain candidates pass 1 listed (saturating at 4:
// more than kPixCand, the ray then traverses) and the hit as part << 24 |
// part-local triangle (bits 0-27).  All ones: no certain hit, no candidate.
// Pass 0 writes its keys with the field at 7, so the 64-bit minimum orders by
// depth, then triangle; pass 1 only lowers the field.
static_assert(kMaxParts <= 16, "the pixel key holds the part in 4 bits");
constexpr unsigned kKeyId = 0x0fffffffu;
constexpr unsigned kKeyField = 29;
__device__ __forceinline__ bool key_none(unsigned long long k) { return (unsigned)(k >> 32) == 0xffffffffu; }
__device__ __forceinline__ unsigned key_cands(unsigned long long k) { return 7u - ((unsigned)(k >> kKeyField) & 7u); }

// One (triangle, pixel centre) pair.  E bounds the pair's error bounds: a
// decision certain against E is certain against them, so the exact bounds are
// formed only near an edge; the decisions are those of prim_test.
template <int PASS>
__device__ __forceinline__ void rast_pixel(const RastView &V, unsigned long long *key, unsigned *cand, int i, int j,
                                           float4 a, float4 b, float4 c, unsigned id, float E)
{
    const float uc = fmaf((float)i + 0.5f, V.du32, V.umin32);
    const float vc = fmaf((float)j + 0.5f, V.dv32, V.vmin32);
    Prim32 q = prim_core(a, b, c, uc, vc, V.w0);
    if (((q.U < -E) || (q.V < -E) || (q.W < -E)) && ((q.U > E) || (q.V > E) || (q.W > E))) return;
    bool unsure = false;
    if (!(fabsf(q.U) > E && fabsf(q.V) > E && fabsf(q.W) > E)) {
        q = prim_test(a, b, c, uc, vc, V.delta, V.w0);
        const bool neg = (q.U < -q.eU) || (q.V < -q.eV) || (q.W < -q.eW);
        const bool pos = (q.U > q.eU) || (q.V > q.eV) || (q.W > q.eW);
        if (neg && pos) return;  // certainly outside
        unsure = fabsf(q.U) <= q.eU || fabsf(q.V) <= q.eV || fabsf(q.W) <= q.eW;
    }
    const float t = q.T / q.det;
    const size_t px = (size_t)i * V.N + j;
    if (PASS == 0) {
        // primary rays start at the window (tlo = 0); t > 0 orders as its bits
        if (!unsure && t > 0.0f)
            atomicMin(key + px, ((unsigned long long)__float_as_uint(t) << 32) | (7u << kKeyField) | id);
        return;
    }
    // (other pass-1 threads may lower this key's candidate field meanwhile:
    // depth and triangle stay as pass 0 left them)
    const unsigned long long k = key[px];
    const float tmin = key_none(k) ? INFINITY : __uint_as_float((unsigned)(k >> 32));
    bool take;
    if (unsure) take = !(fabsf(q.det) > 1e-30f && (t > tmin + V.tau || t < -V.tau));
    else take = fabsf(t) <= V.tau || (((unsigned)k & kKeyId) != id && fabsf(t - tmin) <= V.tau);
    if (take) {
        // claim a candidate slot by lowering the key's field; every failed
        // compare-and-swap means another thread's succeeded, and the loop is
        // bounded all the same: past the bound the field is cleared, which
        // sends the ray to the traversal (always correct)
        unsigned long long old = k;
        int slot = kPixCand;
        for (int it = 0; it < 64; it++) {
            const unsigned f = (unsigned)(old >> kKeyField) & 7u;
            if (7u - f >= (unsigned)kPixCand + 1u) break;  // saturated: the ray traverses
            const unsigned long long seen = atomicCAS(key + px, old, old - (1ull << kKeyField));
            if (seen == old) { slot = (int)(7u - f); break; }
            old = seen;
            if (it == 63) atomicAnd(key + px, ~(7ull << kKeyField));
        }
        if (slot < kPixCand) cand[px * kPixCand + slot] = id;
    }
}

__device__ __forceinline__ int part_of_sorted(const MeshDev *m, int t)
{
    int p = 0;
    for (int q = 0; q < m->n_parts; q++)
        if (t >= m->part[q].tri_begin && t < m->part[q].tri_begin + m->part[q].tri_count) p = q;
    return p;
}

// Thread per (slot, sorted triangle): small projected boxes in place; larger
// ones are listed for k_raster_chunks, which lists their 16 x 16-pixel chunks
// that can meet them for k_raster_big (pass 0 lists, pass 1 reuses the lists).
template <int PASS>
__device__ __forceinline__ void raster_tri(const TraceArgs &a, int s, int t)
{
    const TraceCtx *g = reinterpret_cast<const TraceCtx *>(a.tctx) + s;
    // the slot's context in one round of loads (nothing read from the mesh record)
    const int skip = g->skip, n_tris = g->n_tris;
    const int4 *tv4 = g->tri_v4;
    const RastView V = rast_view(a, s);
    if (skip || t >= n_tris) return;
    if (!(V.du32 > 0.0f && V.dv32 > 0.0f)) {
        if (PASS == 0 && t == 0) a.rast_bad[s] = 1;
        return;
    }
    const int4 vi = __ldg(tv4 + t);
    const float4 A = __ldg(V.vview + vi.x), B = __ldg(V.vview + vi.y), C = __ldg(V.vview + vi.z);
    int i0, i1, j0, j1;
    if (!rast_box(V, A, B, C, i0, i1, j0, j1)) return;
    const int w = i1 - i0 + 1, h = j1 - j0 + 1;
    if (w * h > kRastSmall) {
        if (PASS == 0) {
            // listed for k_raster_chunks, which lists its chunks
            const unsigned at = atomicAdd(a.bigt_count, 1u);
            if (at >= (unsigned)a.big_cap) {
                a.rast_bad[s] = 1;
                return;
            }
            a.bigt[at] = make_int2(s, t);
        }
        return;
    }
    const unsigned id = (unsigned)vi.w;  // (part << 24) | index within the part
    const size_t off = (size_t)s * a.ray_stride;
    const float eb = rast_bound(V, A, B, C, i0, i1, j0, j1);
    for (int i = i0; i <= i1; i++)
        for (int j = j0; j <= j1; j++)
            rast_pixel<PASS>(V, a.pix_key + off, a.pix_cand + off * kPixCand, i, j, A, B, C, id, eb);
}

template <int PASS>
__global__ void __launch_bounds__(128) k_raster(TraceArgs a)
{
    pdl_enter();
    raster_tri<PASS>(a, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x);
}

// Warp per listed large triangle: its 16 x 16-pixel chunks that can meet it,
// tested a chunk per lane and appended with one atomic per warp pass.
__global__ void __launch_bounds__(256) k_raster_chunks(TraceArgs a)
{
    pdl_enter();
    const unsigned n = min(__ldcg(a.bigt_count), (unsigned)a.big_cap);
    const unsigned lane = threadIdx.x & 31u, nw = gridDim.x * (blockDim.x >> 5);
    for (unsigned e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < n; e += nw) {
        const int2 E = a.bigt[e];
        const int s = E.x, t = E.y;
        const TraceCtx *g = reinterpret_cast<const TraceCtx *>(a.tctx) + s;
        const int4 *tv4 = g->tri_v4;
        const RastView V = rast_view(a, s);
        const int4 vi = __ldg(tv4 + t);
        const float4 A = __ldg(V.vview + vi.x), B = __ldg(V.vview + vi.y), C = __ldg(V.vview + vi.z);
        int i0, i1, j0, j1;
        if (!rast_box(V, A, B, C, i0, i1, j0, j1)) continue;
        const int cw = (i1 - i0 + kRastChunk) / kRastChunk, ch = (j1 - j0 + kRastChunk) / kRastChunk;
        for (int k0 = 0; k0 < cw * ch; k0 += 32) {
            const int k = k0 + (int)lane;
            bool meets = false;
            if (k < cw * ch) {
                const int ib = i0 + (k % cw) * kRastChunk, jb = j0 + (k / cw) * kRastChunk;
                meets = chunk_meets(V, A, B, C, ib, min(ib + kRastChunk - 1, i1), jb, min(jb + kRastChunk - 1, j1));
            }
            const unsigned bal = __ballot_sync(0xffffffffu, meets);
            if (!bal) continue;
            unsigned at = 0u;
            if (lane == 0) at = atomicAdd(a.big_count, (unsigned)__popc(bal));
            at = __shfl_sync(0xffffffffu, at, 0);
            const unsigned cnt = (unsigned)__popc(bal);
            const unsigned room = at < (unsigned)a.big_cap ? (unsigned)a.big_cap - at : 0u;
            if (cnt > room) {
                // the list is full: the slot's pixels traverse instead; the part of this
                // warp's range below the capacity is filled with placeholders (slot -1)
                // so that every entry a reader sees was written
                const unsigned idx = at + __popc(bal & ((1u << lane) - 1u));
                if (meets && idx < (unsigned)a.big_cap) a.big[idx] = make_int4(-1, 0, 0, 0);
                if (lane == 0) a.rast_bad[s] = 1;
                break;
            }
            if (meets) a.big[at + __popc(bal & ((1u << lane) - 1u))] = make_int4(s, t, k % cw, k / cw);
            if (a.queue && lane == 0) atomicAdd(a.qstate + kQSlot + 3 * s + 2, cnt);
        }
    }
}

// One listed chunk of a large triangle, by the calling warp.  Returns the
// entry's slot, or -1 for a placeholder of a full list.
template <int PASS>
__device__ __forceinline__ int raster_big_entry(const TraceArgs &a, unsigned e, unsigned lane)
{
    const int4 E = a.big[e];
    const int s = E.x, t = E.y;
    if (s < 0) return -1;
    const TraceCtx *g = reinterpret_cast<const TraceCtx *>(a.tctx) + s;
    const int4 *tv4 = g->tri_v4;
    const RastView V = rast_view(a, s);
    const int4 vi = __ldg(tv4 + t);
    const float4 A = __ldg(V.vview + vi.x), B = __ldg(V.vview + vi.y), C = __ldg(V.vview + vi.z);
    int i0, i1, j0, j1;
    if (!rast_box(V, A, B, C, i0, i1, j0, j1)) return s;
    const int ib = i0 + E.z * kRastChunk, jb = j0 + E.w * kRastChunk;
    const int ie = min(ib + kRastChunk - 1, i1), je = min(jb + kRastChunk - 1, j1);
    const unsigned id = (unsigned)vi.w;  // (part << 24) | index within the part
    const size_t off = (size_t)s * a.ray_stride;
    const float eb = rast_bound(V, A, B, C, ib, ie, jb, je);
    for (int q = (int)lane; q < kRastChunk * kRastChunk; q += 32) {
        const int i = ib + q / kRastChunk, j = jb + q % kRastChunk;
        if (i <= ie && j <= je)
            rast_pixel<PASS>(V, a.pix_key + off, a.pix_cand + off * kPixCand, i, j, A, B, C, id, eb);
    }
    return s;
}

// Warp per listed chunk of a large triangle (grid-stride over the list).
template <int PASS>
__global__ void __launch_bounds__(256) k_raster_big(TraceArgs a)
{
    pdl_enter();
    const unsigned n = min(__ldcg(a.big_count), (unsigned)a.big_cap);
    const unsigned lane = threadIdx.x & 31u, nw = gridDim.x * (blockDim.x >> 5);
    for (unsigned e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < n; e += nw) raster_big_entry<PASS>(a, e, lane);
}

// The second raster pass in one launch: blocks below nbig take listed chunks
// of large triangles (a warp per chunk, grid-stride over the list), the rest a
// small triangle per thread (per_slot blocks a slot).
__global__ void __launch_bounds__(128) k_raster_pass1(TraceArgs a, int nbig, int per_slot)
{
    pdl_enter();
    if ((int)blockIdx.x < nbig) {
        const unsigned n = min(__ldcg(a.big_count), (unsigned)a.big_cap);
        const unsigned lane = threadIdx.x & 31u, nw = (unsigned)nbig * (blockDim.x >> 5);
        for (unsigned e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < n; e += nw) raster_big_entry<1>(a, e, lane);
        return;
    }
    const int b = (int)blockIdx.x - nbig;
    raster_tri<1>(a, b / per_slot, (b % per_slot) * (int)blockDim.x + (int)threadIdx.x);
}

// A block is kTraceWarps warps over consecutive tiles of one slot, sharing
// one copy of the slot's context; a warp past the slot's last tile idles.
// The trace of flattened block vb (kTraceWarps tiles of one slot).  B, s_cand
// and s_hpt are the block's shared context copy and per-thread columns (entry k
// of thread x at [k * kLaneStride + x]): the candidates of the FP64 resolution,
// and each segment's hit as (part, triangle) for the FP64 replay of the
// specular chain and the hit record.  QUEUE: run inside the work queue, where
// this SM may hold stale L1 copies of pixel keys another SM's second raster
// pass has changed since, so the raster's results are read from L2.
template <bool COUNT, bool HITS, bool QUEUE>
__device__ __forceinline__ void trace_block(const TraceArgs &a, int vb, TraceCtx &B, int *s_cand, int *s_hpt)
{
    static_assert(kTileRays * kTraceWarps == kLaneStride, "per-thread shared columns assume 128 threads");
    const int s = slot_of_block(a.sd, a.n_slots, vb);
    const SlotDesc &D = a.sd[s];
    const int tile_id = (vb - D.tile0) * kTraceWarps + (int)(threadIdx.x >> 5);
    load_ctx(B, a, s);
    __syncthreads();
    if (tile_id >= D.tiles) return;
    const int N = D.N, nseg = D.nseg;
    const int lane = threadIdx.x & 31;
    if (B.skip) {
        if (lane == 0) a.amb_count[(size_t)s * a.n_blocks_x + tile_id] = 0;
        return;
    }
    const int tw = D.tile_w, lw = __ffs(tw) - 1;
    const int i = (tile_id % D.tiles_x) * tw + (lane & (tw - 1));
    const int j = (tile_id / D.tiles_x) * (kTileRays >> lw) + (lane >> lw);
    // per-ray results: force / torque in FP32 (at most 1 + bounces terms); counts
    // as scalars (a hand-off flag, the segments traced, a bit per segment hit)
    float fac[6] = {0, 0, 0, 0, 0, 0};
    unsigned c_handoff = 0u, c_segs = 0u, c_hitbits = 0u;
    bool handoff = false;
    int flags = 0;
    const int ray = i * N + j;
    int *hpt = s_hpt + threadIdx.x;
    Counts cn = {0u, 0u, 0u, {0u, 0u, 0u, 0u}, 0};
    if (i < N && j < N) {
        Ray32 r;
        for (int k = 0; k < 3; k++) r.d[k] = B.dir[k];
        const float uc = fmaf((float)i + 0.5f, B.du32, B.umin32);
        const float vc = fmaf((float)j + 0.5f, B.dv32, B.vmin32);
        float wgt = 1.0f;
        int skip = -1, gpart = -1, gskip = kEmptyChild;
        float acc[6] = {0, 0, 0, 0, 0, 0};
        unsigned hitbits = 0u;
        bool clean = true;
        int nseg_done = 0;
        Cands cd;
        cd.n = 0;
        cd.id = s_cand + threadIdx.x;
        float delta = B.delta_p, tau = B.tau_p;
        // rasterised primary visibility of this pixel
        bool rast = false;
        unsigned long long pk = ~0ull;
        if (a.raster) {
            const size_t px = (size_t)s * a.ray_stride + ray;
            pk = QUEUE ? __ldcg(a.pix_key + px) : __ldcs(a.pix_key + px);
            const unsigned pn = key_cands(pk);
            rast = pn <= (unsigned)kPixCand && !a.rast_bad[s];
            if (rast) {
                cd.n = (int)pn;
                for (int c = 0; c < (int)pn; c++)
                    cd.id[c * kLaneStride] = (int)(QUEUE ? __ldcg(a.pix_cand + px * kPixCand + c) : a.pix_cand[px * kPixCand + c]);
                if (COUNT) cn.why[0] += pn;
            }
        }
        for (int seg = 0; seg < nseg; seg++) {
            Best32 h;
            float tlo = seg == 0 ? 0.0f : B.eps32;
            nseg_done++;
            if (seg == 0 && !rast)  // a traversed primary segment starts at its pixel on the window
                for (int k = 0; k < 3; k++) r.o[k] = fmaf((float)i + 0.5f, B.du[k], fmaf((float)j + 0.5f, B.dv[k], B.org[k]));
            if (seg > 0 || !rast) ray_setup(r);  // the raster's primary segment needs no ray frame
            if (seg == 0 && rast) {
                // the raster's nearest certain hit; its barycentric weights as the traversal forms them
                h.t = INFINITY;
                h.part = -1;
                h.tl = -1;
                if (!key_none(pk)) {
                    const unsigned id = (unsigned)pk & kKeyId;
                    h.part = (int)(id >> 24);
                    h.tl = (int)(id & 0xffffffu);
                    const int4 vi = __ldg(B.part[h.part].v4 + h.tl);
                    const Prim32 q = prim_core(__ldg(B.vview + vi.x), __ldg(B.vview + vi.y), __ldg(B.vview + vi.z), uc,
                                               vc, B.w0_32);
                    const float id32 = 1.0f / q.det;
                    h.t = q.T * id32;  // not used past this point; the weights are the traversal's
                    h.b1 = q.V * id32;
                    h.b2 = q.W * id32;
                }
            } else {
                bool ok;
                if (seg == 0) {
                    const Near32 o = nearest32_primary<COUNT>(B, r, uc, vc, delta, tau, cn, cd);
                    h = o.b;
                    cn = o.cn;
                    cd.n = o.cand_n;
                    ok = o.ok != 0;
                } else {
                    ok = nearest32<COUNT, false>(B, r, uc, vc, tlo, skip, gpart, gskip, delta, tau, h, cn, cd);
                }
                if (!ok) {
                    clean = false;
                    break;
                }
            }
            if (cd.n > 0) h = resolve64(B, N, i, j, seg, hpt, skip, cd, h);  // rare: settle in FP64
            if (h.part < 0) break;
            hpt[seg * kLaneStride] = (h.part << 24) | h.tl;
            const float4 *tr = B.part[h.part].tri + (size_t)h.tl * 3;
            float4 a0 = __ldg(tr), a1 = __ldg(tr + 1), a2 = __ldg(tr + 2);
            int orig = __float_as_int(a0.w);
            unsigned mt = __float_as_uint(a1.w);
            hitbits |= 1u << seg;
            float e1[3] = {a1.x - a0.x, a1.y - a0.y, a1.z - a0.z};
            float e2[3] = {a2.x - a0.x, a2.y - a0.y, a2.z - a0.z};
            float n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
            float il = rsqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            n[0] *= il; n[1] *= il; n[2] *= il;
            float dn = r.d[0] * n[0] + r.d[1] * n[1] + r.d[2] * n[2];
            int side = dn < 0.f ? 0 : 1;
            float sg = side ? -1.f : 1.f;
            float2 m = __ldg(B.mat32 + (side ? (mt >> 16) : (mt & 0xffffu)));
            float c = -sg * dn;
            // f = w [(1 - rho_s) d - 2 (rho_s c + rho_d / 3) n_f],  n_f = sg n
            float ka = wgt * (1.0f - m.x), kn = -2.0f * wgt * (m.x * c + m.y * (1.0f / 3.0f)) * sg;
            float F[3], hp[3], arm[3];
            const float a0v[3] = {a0.x, a0.y, a0.z};
            for (int k = 0; k < 3; k++) {
                F[k] = ka * r.d[k] + kn * n[k];
                // hit point from the barycentric weights on the hit triangle: its error
                // is that of the test, not that of a long FP32 ray
                hp[k] = fmaf(h.b1, e1[k], fmaf(h.b2, e2[k], a0v[k]));
                arm[k] = hp[k] - B.cref32[k];
            }
            acc[0] += F[0]; acc[1] += F[1]; acc[2] += F[2];
            acc[3] += arm[1] * F[2] - arm[2] * F[1];
            acc[4] += arm[2] * F[0] - arm[0] * F[2];
            acc[5] += arm[0] * F[1] - arm[1] * F[0];
            wgt *= m.x;
            if (seg + 1 >= nseg || wgt == 0.0f) break;
            for (int k = 0; k < 3; k++) {
                r.o[k] = hp[k];
                r.d[k] = r.d[k] - 2.0f * dn * n[k];
            }
            skip = orig;
            // the reflected ray leaves the hit triangle's plane at |dn|: its coplanar group can
            // only be met within dev / |dn| of the origin, inside the self-hit distance eps
            const int2 g = __ldg(B.grp + B.part[h.part].tri_begin + h.tl);
            gpart = h.part;
            gskip = fabsf(dn) * B.eps32 > 16.0f * __int_as_float(g.y) ? g.x : kEmptyChild;
            // next segment: world-frame test; the origin error grows with the previous bound
            delta = B.delta_s + 2.0f * delta;
            tau = 64.0f * delta + 32.0f * kU * (B.R + B.L);
        }
        flags = cn.flags;
        if (clean) {
            for (int k = 0; k < 6; k++) fac[k] = acc[k];
            c_segs = nseg_done;
            c_hitbits = hitbits;
            if (HITS) {
                int32_t *hq = a.hits + ((size_t)s * a.ray_stride + ray) * a.seg_stride;
                for (int k = 0; k < nseg; k++) {
                    int o = -1;
                    if ((hitbits >> k) & 1u) {
                        const int hk = hpt[k * kLaneStride];
                        o = __float_as_int(__ldg(B.part[hk >> 24].tri + (size_t)(hk & 0xffffff) * 3).w);
                    }
                    hq[k] = o;
                }
            }
        } else {
            handoff = true;
            c_handoff = 1u;
        }
    }
    // tile-ordered list of the rays handed to the FP64 path
    const size_t tile = (size_t)s * a.n_blocks_x + tile_id;
    unsigned bal = __ballot_sync(0xffffffffu, handoff);
    if (handoff) a.amb_list[tile * kTileRays + __popc(bal & ((1u << lane) - 1u))] = ray;
    // tile sums, one partial per tile: force and torque by a fixed FP32
    // butterfly over the 32 rays (FP64 shuffles would occupy GB300's slow FP64
    // pipe), counts by integer reductions; every sum above the tile is FP64
    for (int k = 0; k < 6; k++) {
        float x = fac[k];
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) a.partials[tile * 6 + k] = x;
    }
    // counts 0..6 always (hand-offs, segments, hits per segment level); the
    // traversal counters only in the counting variant
#pragma unroll
    for (int k = 0; k < (COUNT ? kCnt : 7); k++) {
        unsigned v;
        if (k == 0) v = c_handoff;
        else if (k == 1) v = c_segs;
        else if (k <= 2 + kMaxBounces) v = (c_hitbits >> (k - 2)) & 1u;
        else if (k == 7) v = cn.nodes;
        else if (k == 8) v = cn.tris;
        else if (k == 9) v = cn.boxes;
        else v = cn.why[k - 10];
        const unsigned x = __reduce_add_sync(0xffffffffu, v);
        if (lane == 0) a.pcounts[tile * kCnt + k] = x;
    }
    int fl = __reduce_or_sync(0xffffffffu, flags);
    if (lane == 0) {
        a.amb_count[tile] = __popc(bal);
        if (fl) atomicOr(&a.pose[s].flags, fl);
    }
}

template <bool COUNT, bool HITS>
__global__ void __launch_bounds__(kTileRays * kTraceWarps, 32 / kTraceWarps) k_trace(TraceArgs a)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char s_dyn[];
    TraceCtx &B = *reinterpret_cast<TraceCtx *>(s_dyn);
    int *s_hpt = reinterpret_cast<int *>(s_dyn + trace_ctx_dyn_bytes(a.ctx_parts));
    __shared__ int s_cand[kCand * kLaneStride];
    trace_block<COUNT, HITS, false>(a, blockIdx.x, B, s_cand, s_hpt);
}

// ------------------------------------------------------------- work queue
// The raster's second pass and the trace of a launch's slots as one persistent
// kernel over a queue of work items, handed out in this order: the second pass
// over small triangles (slot-major, 128 triangles an item), over the listed
// chunks of large triangles (kTraceWarps chunks an item, a warp each), then the
// trace blocks (kTraceWarps tiles an item).  A trace item of slot s may start
// once every second-pass item of slot s has finished, which its block waits for
// on the slot's completion counters.  Items are handed out in order and
// second-pass items never wait, so the items a trace item waits for are held by
// running blocks and every wait ends; each is bounded all the same (device
// time): past the bound the block sets the slot's timeout flag and the queue's
// abort flag (later waits give up at once), writes an empty result for its
// tiles and goes on, and the call reports SRP_ERR_TIMEOUT.
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long kQueueWaitNs = 2000000000ull;  // 2 s of device time
constexpr unsigned long long kQueueTestWaitNs = 2000000ull; // 2 ms when a test makes the wait run out
constexpr int kQueueBatch = 4;  // consecutive items a block claims at once

// Slot of second-pass item it: the last slot whose first item is <= it.
__device__ __forceinline__ int slot_of_rast_item(const SlotDesc *sd, int S, unsigned it)
{
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if ((unsigned)__ldg(&sd[mid].rast0) <= it) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Wait (thread 0 of a block) until slot s's second raster pass is complete; 1
// when it is, 0 when the wait gave up.
__device__ int queue_wait(const TraceArgs &a, int s)
{
    const unsigned *q = a.qstate + kQSlot + 3 * s;
    const unsigned need_small = (unsigned)((a.sd[s].mesh->n_tris + 127) / 128) + (a.wait_test ? 1u : 0u);
    const unsigned need_big = ld_acquire(q + 2);  // final: counted by the chunk listing, an earlier launch
    const unsigned long long limit = a.wait_test ? kQueueTestWaitNs : kQueueWaitNs;
    const unsigned long long t0 = global_ns();
    unsigned ns = 32;
    while (true) {
        if (ld_acquire(q) >= need_small && ld_acquire(q + 1) >= need_big) return 1;
        if (ld_acquire(a.qstate + kQAbort)) break;
        if (global_ns() - t0 > limit) {
            atomicExch(a.qstate + kQAbort, 1u);
            break;
        }
        __nanosleep(ns);
        if (ns < 1024) ns *= 2;
    }
    atomicOr(&a.pose[s].flags, kFlagTimeout);
    return 0;
}

// An empty result for trace block vb (its wait gave up): no force, no counts,
// no hand-offs.
__device__ void trace_block_empty(const TraceArgs &a, int vb)
{
    const int s = slot_of_block(a.sd, a.n_slots, vb);
    const SlotDesc &D = a.sd[s];
    const int tile_id = (vb - D.tile0) * kTraceWarps + (int)(threadIdx.x >> 5);
    if (tile_id >= D.tiles || (threadIdx.x & 31) != 0) return;
    const size_t tile = (size_t)s * a.n_blocks_x + tile_id;
    for (int k = 0; k < 6; k++) a.partials[tile * 6 + k] = 0.0f;
    for (int k = 0; k < kCnt; k++) a.pcounts[tile * kCnt + k] = 0u;
    a.amb_count[tile] = 0;
}

template <bool COUNT, bool HITS>
__global__ void __launch_bounds__(kTileRays * kTraceWarps, 32 / kTraceWarps) k_queue(TraceArgs a)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char s_dyn[];
    TraceCtx &B = *reinterpret_cast<TraceCtx *>(s_dyn);
    int *s_hpt = reinterpret_cast<int *>(s_dyn + trace_ctx_dyn_bytes(a.ctx_parts));
    __shared__ int s_cand[kCand * kLaneStride];
    __shared__ unsigned s_item;
    __shared__ int s_ok, s_ready;  // s_ready: a slot whose second pass this block has seen complete
    const unsigned lane = threadIdx.x & 31u;
    const unsigned n_small = (unsigned)a.n_small_items;
    const unsigned n_big_e = min(ld_acquire(a.big_count), (unsigned)a.big_cap);
    const unsigned n_big = (n_big_e + kTraceWarps - 1) / kTraceWarps;
    const unsigned total = n_small + n_big + (unsigned)a.n_tiles;
    if (threadIdx.x == 0) s_ready = -1;
    for (;;) {
        __syncthreads();  // every warp is done with the previous item and its shared state
        if (threadIdx.x == 0) s_item = atomicAdd(a.qstate + kQHead, (unsigned)kQueueBatch);
        __syncthreads();
        const unsigned it0 = s_item;
        if (it0 >= total) break;
        const unsigned it1 = min(it0 + (unsigned)kQueueBatch, total);
        for (unsigned it = it0; it < it1; it++) {
        if (it > it0) __syncthreads();
        if (it < n_small) {
            const int s = slot_of_rast_item(a.sd, a.n_slots, it);
            raster_tri<1>(a, s, (int)(it - (unsigned)a.sd[s].rast0) * 128 + (int)threadIdx.x);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(a.qstate + kQSlot + 3 * s, 1u);
            }
        } else if (it < n_small + n_big) {
            const unsigned e = (it - n_small) * kTraceWarps + (threadIdx.x >> 5);
            if (e < n_big_e) {
                const int s = raster_big_entry<1>(a, e, lane);
                __syncwarp();
                if (lane == 0 && s >= 0) {
                    __threadfence();
                    atomicAdd(a.qstate + kQSlot + 3 * s + 1, 1u);
                }
            }
        } else {
            const int vb = (int)(it - n_small - n_big);
            if (threadIdx.x == 0) {
                const int s = slot_of_block(a.sd, a.n_slots, vb);
                s_ok = s == s_ready ? 1 : queue_wait(a, s);
                if (s_ok) s_ready = s;
            }
            __syncthreads();
            if (s_ok) trace_block<COUNT, HITS, true>(a, vb, B, s_cand, s_hpt);
            else trace_block_empty(a, vb);
        }
        }
    }
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
    const double rz = 1.0 / dz;
    r.Sx = pickd(r.d[0], r.d[1], r.d[2], kx) * rz;
    r.Sy = pickd(r.d[0], r.d[1], r.d[2], ky) * rz;
    r.Sz = rz;
}

__device__ void tri_v64(const TraceCtx &B, int p, int tl, double *v)
{
    const PartView &pv = B.part[p];
    int t = pv.tri_begin + tl;
    for (int c = 0; c < 3; c++) {
        int vi = B.tri_vidx[3 * t + c] - pv.vert_begin;
        for (int k = 0; k < 3; k++) v[3 * c + k] = pv.v64[3 * vi + k];
    }
}

// FP64 watertight edge functions and scaled depth of triangle v against ray r.
__device__ __forceinline__ void wt64(const Ray64 &r, const double *v, double &U, double &V, double &W, double &det,
                                     double &T)
{
    double A[3], Bv[3], C[3];
    for (int k = 0; k < 3; k++) { A[k] = v[k] - r.o[k]; Bv[k] = v[3 + k] - r.o[k]; C[k] = v[6 + k] - r.o[k]; }
    double Akz = pickd(A[0], A[1], A[2], r.kz), Bkz = pickd(Bv[0], Bv[1], Bv[2], r.kz), Ckz = pickd(C[0], C[1], C[2], r.kz);
    double Ax = pickd(A[0], A[1], A[2], r.kx) - r.Sx * Akz, Ay = pickd(A[0], A[1], A[2], r.ky) - r.Sy * Akz;
    double Bx = pickd(Bv[0], Bv[1], Bv[2], r.kx) - r.Sx * Bkz, By = pickd(Bv[0], Bv[1], Bv[2], r.ky) - r.Sy * Bkz;
    double Cx = pickd(C[0], C[1], C[2], r.kx) - r.Sx * Ckz, Cy = pickd(C[0], C[1], C[2], r.ky) - r.Sy * Ckz;
    U = __dsub_rn(__dmul_rn(Cx, By), __dmul_rn(Cy, Bx));
    V = __dsub_rn(__dmul_rn(Ax, Cy), __dmul_rn(Ay, Cx));
    W = __dsub_rn(__dmul_rn(Bx, Ay), __dmul_rn(By, Ax));
    det = U + V + W;
    T = U * (r.Sz * Akz) + V * (r.Sz * Bkz) + W * (r.Sz * Ckz);
}

// Settle one segment's uncertain FP32 decisions in FP64: the FP64 test of each
// candidate and of the nearest certain FP32 hit against the segment's exact
// ray; the nearest t above the self-hit threshold wins, equal t goes to the
// lowest original triangle id (the rule of the FP64 re-trace).  Every other
// triangle was certainly missed, certainly farther, or culled beyond the
// certain hit plus its band.  Primary segments are tested in the view frame
// (the ray is the line through the FP64 pixel centre along d; vertex
// projections computed once per evaluation in FP64); a specular segment's ray
// is the FP64 chain through the earlier segments' hit triangles, tested with
// the FP64 watertight test.  FP64 is slow on this GPU: no square roots, one
// division per candidate, barycentric weights for the winner only.
// hpt: this thread's column of the block's hit records (segment s at hpt[s * kLaneStride]).
__device__ __noinline__ Best32 resolve64(const TraceCtx &B, int N, int i, int j, int seg, const int *hpt, int skip,
                                         Cands cd, Best32 best)
{
    double bt = INFINITY, bU = 0.0, bV = 0.0, bW = 0.0;
    int bp = -1, btl = -1, bo = 0x7fffffff;
    const double uc = B.umin + pix64(((double)i + 0.5) * B.Du, B.rN, N);
    const double vc = B.vmin + pix64(((double)j + 0.5) * B.Dv, B.rN, N);
    const double w0 = B.wmin - kStandoff;
    Ray64 r;
    double tlo = 0.0;
    if (seg > 0) {
        for (int k = 0; k < 3; k++) { r.o[k] = uc * B.u[k] + vc * B.v[k] + w0 * B.d[k]; r.d[k] = B.d[k]; }
        double v[9];
        for (int s = 0; s < seg; s++) {
            // hit point on the plane of the segment's triangle, then the specular direction
            const int hs = hpt[s * kLaneStride];
            tri_v64(B, hs >> 24, hs & 0xffffff, v);
            double e1[3], e2[3], m[3], ao[3];
            for (int k = 0; k < 3; k++) { e1[k] = v[3 + k] - v[k]; e2[k] = v[6 + k] - v[k]; ao[k] = v[k] - r.o[k]; }
            m[0] = e1[1] * e2[2] - e1[2] * e2[1];
            m[1] = e1[2] * e2[0] - e1[0] * e2[2];
            m[2] = e1[0] * e2[1] - e1[1] * e2[0];
            double dm = r.d[0] * m[0] + r.d[1] * m[1] + r.d[2] * m[2];
            double t = (ao[0] * m[0] + ao[1] * m[1] + ao[2] * m[2]) / dm;
            double f = 2.0 * dm / (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
            for (int k = 0; k < 3; k++) { r.o[k] = r.o[k] + t * r.d[k]; r.d[k] = r.d[k] - f * m[k]; }
        }
        ray64_setup(r);
        tlo = B.eps;
    }
    for (int c = 0; c <= cd.n; c++) {
        int p, tl;
        if (c < cd.n) { const int id = cd.id[c * kLaneStride]; p = id >> 24; tl = id & 0xffffff; }
        else if (best.part >= 0) { p = best.part; tl = best.tl; }
        else break;
        const PartView &pv = B.part[p];
        int orig = __float_as_int(__ldg(pv.tri + (size_t)tl * 3).w);
        if (orig == skip) continue;
        double U, V, W, det, T;
        if (seg == 0) {
            int4 vi = __ldg(pv.v4 + tl);
            const double *a = B.vview64 + 3 * (size_t)vi.x, *b = B.vview64 + 3 * (size_t)vi.y,
                         *q = B.vview64 + 3 * (size_t)vi.z;
            double Ax = a[0] - uc, Ay = a[1] - vc, Bx = b[0] - uc, By = b[1] - vc, Cx = q[0] - uc, Cy = q[1] - vc;
            U = __dsub_rn(__dmul_rn(Cx, By), __dmul_rn(Cy, Bx));
            V = __dsub_rn(__dmul_rn(Ax, Cy), __dmul_rn(Ay, Cx));
            W = __dsub_rn(__dmul_rn(Bx, Ay), __dmul_rn(By, Ax));
            det = U + V + W;
            T = U * (a[2] - w0) + V * (b[2] - w0) + W * (q[2] - w0);
        } else {
            double v[9];
            tri_v64(B, p, tl, v);
            wt64(r, v, U, V, W, det, T);
        }
        bool out = (U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0);
        if (out || det == 0.0) continue;
        double t = T / det;
        if (t > tlo && (t < bt || (t == bt && orig < bo))) {
            bt = t; bp = p; btl = tl; bo = orig; bU = det; bV = V; bW = W;
        }
    }
    best.t = (float)bt;
    best.part = bp;
    best.tl = btl;
    best.b1 = bp >= 0 ? (float)(bV / bU) : 0.f;
    best.b2 = bp >= 0 ? (float)(bW / bU) : 0.f;
    return best;
}

// True when the FP32 world-frame test shows the triangle certainly misses the
// ray: some edge function certainly negative and another certainly positive,
// with the per-triangle error bound of the secondary-ray test.
__device__ __forceinline__ bool outside32(const Ray32 &r, float4 a, float4 b, float4 c, float delta)
{
    const float u4 = 4.0f * kU;
    float A0 = a.x - r.o[0], A1 = a.y - r.o[1], A2 = a.z - r.o[2];
    float B0 = b.x - r.o[0], B1 = b.y - r.o[1], B2 = b.z - r.o[2];
    float C0 = c.x - r.o[0], C1 = c.y - r.o[1], C2 = c.z - r.o[2];
    float Akz = pick(A0, A1, A2, r.kz()), Bkz = pick(B0, B1, B2, r.kz()), Ckz = pick(C0, C1, C2, r.kz());
    float Ax = fmaf(-r.Sx, Akz, pick(A0, A1, A2, r.kx())), Ay = fmaf(-r.Sy, Akz, pick(A0, A1, A2, r.ky()));
    float Bx = fmaf(-r.Sx, Bkz, pick(B0, B1, B2, r.kx())), By = fmaf(-r.Sy, Bkz, pick(B0, B1, B2, r.ky()));
    float Cx = fmaf(-r.Sx, Ckz, pick(C0, C1, C2, r.kx())), Cy = fmaf(-r.Sy, Ckz, pick(C0, C1, C2, r.ky()));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    float dz = fmaxf(fmaxf(fabsf(Akz), fabsf(Bkz)), fabsf(Ckz)) + fmaxf(fmaxf(fabsf(Ax), fabsf(Bx)), fabsf(Cx)) +
               fmaxf(fmaxf(fabsf(Ay), fabsf(By)), fabsf(Cy));
    float dc = fmaf(16.0f * kU, dz, delta);
    float eU = dc * (fabsf(Bx) + fabsf(By) + fabsf(Cx) + fabsf(Cy)) + u4 * (fabsf(Cx * By) + fabsf(Cy * Bx));
    float eV = dc * (fabsf(Ax) + fabsf(Ay) + fabsf(Cx) + fabsf(Cy)) + u4 * (fabsf(Ax * Cy) + fabsf(Ay * Cx));
    float eW = dc * (fabsf(Ax) + fabsf(Ay) + fabsf(Bx) + fabsf(By)) + u4 * (fabsf(Bx * Ay) + fabsf(By * Ax));
    bool neg = (U < -eU) || (V < -eV) || (W < -eW);
    bool pos = (U > eU) || (V > eV) || (W > eW);
    return neg && pos;
}

// Nearest hit in FP64 (same BVH; boxes tested with the rounded ray, whose
// deviation from the FP64 ray is far below the box padding).
__device__ void nearest64(const TraceCtx &B, const Ray64 &r, double tlo, int skip, double &bt, int &bpart, int &btl,
                          int &borig, int &flags)
{
    bt = INFINITY;
    bpart = -1; btl = -1; borig = 0x7fffffff;
    Ray32 q;
    for (int k = 0; k < 3; k++) { q.o[k] = (float)r.o[k]; q.d[k] = (float)r.d[k]; }
    ray_setup(q);
    const float slack = 4.0f * B.pad;
    // bound on the coordinate error of the rounded ray and FP32 vertices, for the
    // FP32 pre-test that skips triangles the ray certainly misses
    float omax = fmaxf(fmaxf(fabsf(q.o[0]), fabsf(q.o[1])), fabsf(q.o[2]));
    const float dq = 2.0f * kU * (omax + B.R);
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
                const int n = node4_step(pv.node + (size_t)ref * kNode4, q.inv, q.oi, q.code, (float)tlo - slack,
                                         (float)bt + slack, ref, stack, sp);
                if (n < 0) { flags |= kFlagStack; break; }
                if (n > 0) continue;
            } else {
                int tl = ~ref;
                const float4 *tr = pv.tri + (size_t)tl * 3;
                float4 fa = __ldg(tr), fb = __ldg(tr + 1), fc = __ldg(tr + 2);
                int orig = __float_as_int(fa.w);
                if (orig != skip && !outside32(q, fa, fb, fc, dq)) {
                    double v[9];
                    tri_v64(B, p, tl, v);
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

// Re-trace of one handed-off ray, FP64 from the pixel definition; adds to acc.
__device__ void refine_ray(const TraceCtx &B, const TraceArgs &a, int s, int ray, double *acc, int &flags)
{
    const int N = a.sd[s].N, nseg = a.sd[s].nseg;
    int i = ray / N, j = ray % N;
    Ray64 r;
    double uc = B.umin + pix64(((double)i + 0.5) * B.Du, B.rN, N);
    double vc = B.vmin + pix64(((double)j + 0.5) * B.Dv, B.rN, N);
    double w0 = B.wmin - kStandoff;
    for (int k = 0; k < 3; k++) { r.o[k] = uc * B.u[k] + vc * B.v[k] + w0 * B.d[k]; r.d[k] = B.d[k]; }
    double wgt = 1.0;
    int skip = -1, nseg_done = 0;
    int32_t *hp = a.hits ? a.hits + ((size_t)s * a.ray_stride + ray) * a.seg_stride : nullptr;
    if (hp) for (int k = 0; k < nseg; k++) hp[k] = -1;
    for (int seg = 0; seg < nseg; seg++) {
        ray64_setup(r);
        double t;
        int hpart, htl, horig;
        nseg_done++;
        nearest64(B, r, seg == 0 ? 0.0 : B.eps, skip, t, hpart, htl, horig, flags);
        if (hpart < 0) break;
        if (hp) hp[seg] = horig;
        acc[8 + seg] += 1.0;
        double v[9];
        tri_v64(B, hpart, htl, v);
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
        unsigned mt = B.tri_mat[B.part[hpart].tri_begin + htl];
        int mi = side ? (int)(mt >> 16) : (int)(mt & 0xffffu);
        double rs = B.mat64[2 * mi], rd = B.mat64[2 * mi + 1];
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
        if (seg + 1 >= nseg || wgt == 0.0) break;
        for (int k = 0; k < 3; k++) { r.d[k] = r.d[k] - 2.0 * dn * n[k]; r.o[k] = x[k]; }
        skip = horig;
    }
    acc[6] += 1.0;
    acc[7] += (double)nseg_done;
}

// ------------------------------------------------------- diffuse rays
// SplitMix64 output number c of the stream seeded with `seed` (Steele, Lea &
// Flood, OOPSLA 2014): the state after c + 1 golden-ratio increments, mixed.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long c)
{
    unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Cosine-weighted direction about the unit normal nf for sample counter c:
// uniforms from outputs 2c and 2c + 1 (top 53 bits), a uniform point of the
// unit disc lifted to the hemisphere (Malley's method), in the orthonormal
// basis of Duff et al. (JCGT 2017) around nf.
__device__ __forceinline__ void diffuse_dir(unsigned long long seed, unsigned long long c, const double *nf, double *w)
{
    const double u1 = (double)(splitmix64_at(seed, 2ull * c) >> 11) * 0x1.0p-53;
    const double u2 = (double)(splitmix64_at(seed, 2ull * c + 1ull) >> 11) * 0x1.0p-53;
    double sp, cp;
    sincospi(2.0 * u2, &sp, &cp);  // the angle 2 pi u2, reduced exactly (2 u2 is exact)
    const double rr = sqrt(u1), lz = sqrt(1.0 - u1);
    const double sign = copysign(1.0, nf[2]);
    const double a = -1.0 / (sign + nf[2]);
    const double b = nf[0] * nf[1] * a;
    const double t1[3] = {1.0 + sign * nf[0] * nf[0] * a, sign * b, -sign * nf[0]};
    const double t2[3] = {b, sign + nf[1] * nf[1] * a, -nf[1]};
    for (int k = 0; k < 3; k++) w[k] = rr * cp * t1[k] + rr * sp * t2[k] + lz * nf[k];
}

// Unit normal of a triangle from its FP64 vertices (v0 v1 v2 row-major).
__device__ __forceinline__ void tri_normal64(const double *v, double *n)
{
    double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]}, e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double il = 1.0 / sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int k = 0; k < 3; k++) n[k] *= il;
}

// Settle an FP32 traversal's result in FP64: the FP64 watertight test of each
// uncertain candidate and of the nearest certain FP32 hit against the exact
// ray; the nearest t above tlo wins, equal t to the lowest original id.  Every
// other triangle was certainly missed, certainly farther, or culled beyond
// the certain hit plus its band.
__device__ void settle64(const TraceCtx &B, const Ray64 &r, double tlo, int skip, const Cands &cd, const Best32 &best,
                         double &bt, int &bp, int &btl)
{
    bt = INFINITY;
    bp = -1;
    btl = -1;
    int bo = 0x7fffffff;
    for (int c = 0; c <= cd.n; c++) {
        int p, tl;
        if (c < cd.n) { const int id = cd.id[c * kLaneStride]; p = id >> 24; tl = id & 0xffffff; }
        else if (best.part >= 0) { p = best.part; tl = best.tl; }
        else break;
        const int orig = __float_as_int(__ldg(B.part[p].tri + (size_t)tl * 3).w);
        if (orig == skip) continue;
        double v[9], U, V, W, det, T;
        tri_v64(B, p, tl, v);
        wt64(r, v, U, V, W, det, T);
        const bool out = (U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0);
        if (out || det == 0.0) continue;
        const double t = T / det;
        if (t > tlo && (t < bt || (t == bt && orig < bo))) { bt = t; bp = p; btl = tl; bo = orig; }
    }
}

// One diffuse sample (counter c) leaving hit point x of triangle `src` about
// the lit side's normal nf with weight wd: traced in FP32 with error-bounded
// decisions (as a secondary segment of the trace, the origin error being the
// rounding of the FP64 point), the uncertain ones settled in FP64; the FP64
// traversal when the candidate list overflows.  Its per-hit force and torque
// about c_ref are added to acc.
__device__ __forceinline__ void diffuse_sample(const TraceCtx &B, unsigned long long seed, unsigned long long c,
                                               const double *x, const double *nf, int src, double wd, double *acc,
                                               int &flags, int *cand_col)
{
    Ray64 r;
    diffuse_dir(seed, c, nf, r.d);
    for (int e = 0; e < 3; e++) r.o[e] = x[e];
    ray64_setup(r);
    double t;
    int p, tl;
    {
        Ray32 q;
        for (int e = 0; e < 3; e++) { q.o[e] = (float)r.o[e]; q.d[e] = (float)r.d[e]; }
        ray_setup(q);
        const float delta = 2.0f * B.delta_s;
        const float tau = 64.0f * delta + 32.0f * kU * (B.R + B.L);
        Best32 b;
        Counts cn = {0u, 0u, 0u, {0u, 0u, 0u, 0u}, 0};
        Cands cd;
        cd.n = 0;
        cd.id = cand_col;
        if (nearest32<false, false>(B, q, 0.0f, 0.0f, B.eps32, src, -1, kEmptyChild, delta, tau, b, cn, cd)) {
            if (cd.n == 0) {
                // every FP32 decision was certain: the FP32 nearest hit is the FP64 one,
                // and its FP32 distance places the hit point for the torque arm
                p = b.part;
                tl = b.tl;
                t = (double)b.t;
            } else {
                settle64(B, r, B.eps, src, cd, b, t, p, tl);
            }
        } else {
            int orig;
            nearest64(B, r, B.eps, src, t, p, tl, orig, flags);
        }
        flags |= cn.flags;  // a walk bound is an error, as in the trace
    }
    if (p < 0) return;
    double v[9], n[3];
    tri_v64(B, p, tl, v);
    tri_normal64(v, n);
    const double dn = r.d[0] * n[0] + r.d[1] * n[1] + r.d[2] * n[2];
    const int side = dn < 0.0 ? 0 : 1;
    const double sg = side ? -1.0 : 1.0;
    const unsigned mt = B.tri_mat[B.part[p].tri_begin + tl];
    const int mi = side ? (int)(mt >> 16) : (int)(mt & 0xffffu);
    const double rs = B.mat64[2 * mi], rd = B.mat64[2 * mi + 1];
    const double cs = -sg * dn;
    double F[3], arm[3];
    for (int e = 0; e < 3; e++) {
        F[e] = wd * ((1.0 - rs) * r.d[e] - 2.0 * (rs * cs + rd / 3.0) * sg * n[e]);
        arm[e] = x[e] + t * r.d[e] - B.c_ref[e];
    }
    acc[0] += F[0]; acc[1] += F[1]; acc[2] += F[2];
    acc[3] += arm[1] * F[2] - arm[2] * F[1];
    acc[4] += arm[2] * F[0] - arm[0] * F[2];
    acc[5] += arm[0] * F[1] - arm[1] * F[0];
}

// Diffuse secondary rays of every ray of slot s (grid: kDiffBlocks x slots; a
// thread per (primary ray, sample q) work item in turn, so the K lanes of one
// ray share its control flow).  The ray's segments are replayed in FP64
// through the triangles the trace recorded (hit point on the triangle's
// plane, specular direction), and at each hit of a segment with a next level
// sample q of the K rays of weight w rho_d / K, cosine-distributed about the
// lit side's normal, is traced with the FP64 traversal and deposits the
// per-hit law at its hit.  Sums per block in a fixed order: the result is
// reproducible.
// Diffuse rays, step 1: a thread per primary ray replays its specular chain in
// FP64 through the recorded hit triangles and writes one record per hit that
// emits (a segment with a next level, rho_d > 0) to the ray's slots of the
// dense array, and the number of records.
__global__ void __launch_bounds__(kLaneStride) k_demit(TraceArgs a)
{
    pdl_enter();
    __shared__ TraceCtx B;
    const int s = blockIdx.y;
    load_ctx(B, a, s);
    __syncthreads();
    const SlotDesc &D = a.sd[s];
    const int N = D.N, nseg = D.nseg, K = a.n_diffuse;
    const size_t R = (size_t)N * N;
    int *cnt = a.dcnt + (size_t)s * a.ray_stride;
    for (size_t ray = (size_t)blockIdx.x * blockDim.x + threadIdx.x; ray < R; ray += (size_t)gridDim.x * blockDim.x) {
        int ne = 0;
        if (!B.skip) {
            const int *tri_pos = D.mesh->tri_pos;
            const int32_t *hq = a.hits + ((size_t)s * a.ray_stride + ray) * a.seg_stride;
            DEmit *out = a.demit + ((size_t)s * a.ray_stride + ray) * (size_t)(nseg - 1);
            const int i = (int)(ray / N), j = (int)(ray % N);
            const double uc = B.umin + pix64(((double)i + 0.5) * B.Du, B.rN, N);
            const double vc = B.vmin + pix64(((double)j + 0.5) * B.Dv, B.rN, N);
            const double w0 = B.wmin - kStandoff;
            double o[3], d[3];
            for (int k = 0; k < 3; k++) { o[k] = uc * B.u[k] + vc * B.v[k] + w0 * B.d[k]; d[k] = B.d[k]; }
            double wgt = 1.0;
            for (int k = 0; k + 1 < nseg; k++) {
                const int h = hq[k];
                if (h < 0) break;
                const int t = __ldg(tri_pos + h);
                const int p = part_of_sorted(D.mesh, t);
                const int tl = t - B.part[p].tri_begin;
                double v[9], n[3];
                tri_v64(B, p, tl, v);
                tri_normal64(v, n);
                // hit point on the triangle's plane
                const double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
                const double th = ((v[0] - o[0]) * n[0] + (v[1] - o[1]) * n[1] + (v[2] - o[2]) * n[2]) / dn;
                double x[3];
                for (int c = 0; c < 3; c++) x[c] = o[c] + th * d[c];
                const int side = dn < 0.0 ? 0 : 1;
                const double sg = side ? -1.0 : 1.0;
                const unsigned mt = B.tri_mat[B.part[p].tri_begin + tl];
                const int mi = side ? (int)(mt >> 16) : (int)(mt & 0xffffu);
                const double rs = B.mat64[2 * mi], rd = B.mat64[2 * mi + 1];
                if (rd > 0.0) {
                    DEmit &e = out[ne++];
                    for (int c = 0; c < 3; c++) { e.x[c] = x[c]; e.nf[c] = sg * n[c]; }
                    e.wd = wgt * rd / K;
                    e.src = h;
                    e.c0 = ((unsigned long long)ray * (unsigned long long)nseg + (unsigned long long)k) *
                           (unsigned long long)K;
                }
                wgt *= rs;
                if (wgt == 0.0) break;
                for (int c = 0; c < 3; c++) { d[c] = d[c] - 2.0 * dn * n[c]; o[c] = x[c]; }
            }
        }
        cnt[ray] = ne;
    }
}

// Diffuse rays, step 2: a block per slot turns the per-ray record counts into
// their exclusive prefix (each thread a contiguous range, then the block's
// ranges in order) and the slot's total.
__global__ void __launch_bounds__(1024) k_dscan(TraceArgs a)
{
    pdl_enter();
    __shared__ int part[1024];
    const int s = blockIdx.x;
    const size_t R = (size_t)a.sd[s].N * a.sd[s].N;
    int *cnt = a.dcnt + (size_t)s * a.ray_stride;
    const size_t per = (R + blockDim.x - 1) / blockDim.x;
    const size_t r0 = min(R, per * threadIdx.x), r1 = min(R, r0 + per);
    int sum = 0;
    for (size_t r = r0; r < r1; r++) sum += cnt[r];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {  // inclusive scan of the ranges' sums
        const int v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - sum;
    for (size_t r = r0; r < r1; r++) {
        const int c = cnt[r];
        cnt[r] = run;
        run += c;
    }
    if (threadIdx.x == blockDim.x - 1) a.dtot[s] = part[threadIdx.x];
}

// Diffuse rays, step 3: a thread per (record, sample) work item, items in the
// order of the records (ray-major), each record's K samples consecutive; the
// record of item e K + q is found by binary search over the prefix.
__global__ void __launch_bounds__(kLaneStride) k_diffuse(TraceArgs a)
{
    pdl_enter();
    __shared__ TraceCtx B;
    __shared__ double red[4][6];
    __shared__ int s_cand[kCand * kLaneStride];  // per-thread candidate columns (see Cands)
    const int s = blockIdx.y;
    load_ctx(B, a, s);
    __syncthreads();
    double acc[6] = {0, 0, 0, 0, 0, 0};
    if (!B.skip) {
        const SlotDesc &D = a.sd[s];
        const int N = D.N, nseg = D.nseg, K = a.n_diffuse;
        const size_t R = (size_t)N * N;
        const int *off = a.dcnt + (size_t)s * a.ray_stride;
        const DEmit *rec = a.demit + (size_t)s * a.ray_stride * (size_t)(nseg - 1);
        int flags = 0;
        const size_t items = (size_t)a.dtot[s] * (size_t)K;
        for (size_t it = (size_t)blockIdx.x * blockDim.x + threadIdx.x; it < items; it += (size_t)gridDim.x * blockDim.x) {
            const int e = (int)(it / K);
            const int q = (int)(it - (size_t)e * K);
            // the last ray whose first record is <= e
            size_t lo = 0, hi = R - 1;
            while (lo < hi) {
                const size_t mid = (lo + hi + 1) >> 1;
                if (__ldg(off + mid) <= e) lo = mid; else hi = mid - 1;
            }
            const DEmit &E = rec[lo * (size_t)(nseg - 1) + (size_t)(e - __ldg(off + lo))];
            diffuse_sample(B, (unsigned long long)a.diffuse_seed, E.c0 + (unsigned long long)q, E.x, E.nf, E.src, E.wd,
                           acc, flags, s_cand + threadIdx.x);
        }
        if (flags) atomicOr(&a.pose[s].flags, flags);
    }
    // block sum in a fixed order: warps by shuffles, then the four warps in turn
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = 0; k < 6; k++) {
        const double x = warp_sum(acc[k]);
        if (lane == 0) red[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        a.dpart[((size_t)s * kDiffBlocks + blockIdx.x) * 6 + k] = ((red[0][k] + red[1][k]) + red[2][k]) + red[3][k];
    }
}

// ------------------------------------------------------------- reduce
// First level: block b of slot s sums tiles [b * chunk, (b + 1) * chunk), and
// re-traces in FP64 the rays its tiles handed off (a walk bound, or more
// uncertain triangles than the candidate list holds; rare: the traversal
// context is loaded only when the block has any).  Each thread takes a fixed,
// strided set of tiles in order, so the sums are reproducible.
__device__ void final_reduce(const TraceArgs &a, int s, int eval0, double *force, double *torque, int *err_flags,
                             unsigned long long *stats_accum, bool cg);

__global__ void __launch_bounds__(256) k_reduce1(TraceArgs a, int eval0, double *force, double *torque,
                                                 int *err_flags, unsigned long long *stats_accum, int fuse)
{
    pdl_enter();
    const int s = blockIdx.y, b = blockIdx.x;
    if (a.pose[s].skip) {  // uniform over the block
        // a skipped evaluation outputs zero force and torque
        if (fuse && b == 0 && threadIdx.x < 6) (threadIdx.x < 3 ? force : torque)[3 * (eval0 + s) + threadIdx.x % 3] = 0.0;
        return;
    }
    const int nt = a.sd[s].tiles;
    const int chunk = (nt + kRed1 - 1) / kRed1;
    const int t0 = b * chunk, t1 = min(t0 + chunk, nt);
    const size_t base = (size_t)s * a.n_blocks_x;
    double f[6] = {0, 0, 0, 0, 0, 0};
    Comp32 f32[6];  // the FP32 sum modes
    for (int k = 0; k < 6; k++) f32[k] = Comp32{0.0f, 0.0f};
    const int mode = a.sum_mode;
    // counts of one block (at most 512 tiles of 32 rays) fit 32 bits
    unsigned c[kCnt];
    for (int k = 0; k < kCnt; k++) c[k] = 0u;
    const int kc = a.count ? kCnt : 7;  // the trace writes the traversal counters only when counting
    int mine = 0;
    for (int t = t0 + (int)threadIdx.x; t < t1; t += blockDim.x) {
        for (int k = 0; k < 6; k++) {
            const float p = a.partials[(base + t) * 6 + k];
            if (mode == 0) f[k] += (double)p;
            else if (mode == 1) comp_add(f32[k], p);
            else f32[k].hi = __fadd_rn(f32[k].hi, p);
        }
        // count 0: the tile's hand-off flags; the re-trace below counts the rays it does
        for (int k = 1; k < kc; k++) c[k] += a.pcounts[(base + t) * kCnt + k];
        mine |= a.amb_count[base + t];
    }
    __shared__ TraceCtx B;
    __shared__ int blk_flags;
    if (__syncthreads_or(mine)) {
        if (threadIdx.x == 0) blk_flags = 0;
        load_ctx(B, a, s);
        __syncthreads();
        int flags = 0;
        double acc[kPart];
        for (int k = 0; k < kPart; k++) acc[k] = 0.0;
        for (int t = t0 + (int)threadIdx.x; t < t1; t += blockDim.x) {
            const int n = a.amb_count[base + t];
            for (int q = 0; q < n; q++) refine_ray(B, a, s, a.amb_list[(base + t) * kTileRays + q], acc, flags);
        }
        for (int k = 0; k < 6; k++) {
            if (mode == 0) f[k] += acc[k];
            else if (mode == 1) comp_add(f32[k], (float)acc[k]);
            else f32[k].hi = __fadd_rn(f32[k].hi, (float)acc[k]);
        }
        for (int k = 0; k < kCnt; k++) c[k] += (unsigned)acc[6 + k];
        if (flags) atomicOr(&blk_flags, flags);
        __syncthreads();
        if (threadIdx.x == 0 && blk_flags) atomicOr(&a.pose[s].flags, blk_flags);
    }
    // block sums in a fixed order: FP64 for force and torque (or the FP32
    // modes' sums, threads in turn by one thread), integers for counts
    __shared__ double rf[6][8];
    __shared__ unsigned long long rc[kCnt][8];
    __shared__ Comp32 r32[6][256];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (mode == 0) {
        for (int k = 0; k < 6; k++) {
            const double x = warp_sum(f[k]);
            if (lane == 0) rf[k][w] = x;
        }
    } else {
        for (int k = 0; k < 6; k++) r32[k][threadIdx.x] = f32[k];
    }
    for (int k = 0; k < kCnt; k++) {
        // only the live counts (kc is uniform over the launch)
        unsigned x = c[k];
        if (k < kc)
            for (int o = 16; o; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) rc[k][w] = x;
    }
    __syncthreads();
    const int nw = (int)(blockDim.x >> 5);
    double *out = a.partials1 + ((size_t)s * kRed1 + b) * kPart;
    if (threadIdx.x < 6) {
        if (mode == 0) {
            double x = 0.0;
            for (int q = 0; q < nw; q++) x += rf[threadIdx.x][q];
            out[threadIdx.x] = x;
        } else {
            Comp32 x{0.0f, 0.0f};
            for (int q = 0; q < (int)blockDim.x; q++) {
                if (mode == 1) comp_merge(x, r32[threadIdx.x][q]);
                else x.hi = __fadd_rn(x.hi, r32[threadIdx.x][q].hi);
            }
            out[threadIdx.x] = (double)comp_value(x);  // an FP32 value, exact in FP64
        }
    } else if (threadIdx.x < kPart) {
        unsigned long long x = 0ull;
        for (int q = 0; q < nw; q++) x += rc[threadIdx.x - 6][q];
        out[threadIdx.x] = (double)x;
    }
    if (!fuse) return;
    // the last of the slot's blocks to finish adds the first-level sums, in
    // block order whichever block that is (the second level, without a launch)
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&a.red_ticket[s], 1u) == (unsigned)(kRed1 - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    final_reduce(a, s, eval0, force, torque, err_flags, stats_accum, true);
}

// The second level for slot s: its kRed1 first-level sums added in block order
// (FP64; the FP32 modes add them again in FP32), the diffuse blocks' sums, the
// pixel-area scale, the stores.  Threads below kRed1 of the calling block hold
// the sums (whole warps); `cg` reads what other blocks of the same launch wrote
// through L2.  stats_accum[16]: 0 evals, 1 rays, 2 refined rays, 3 segments,
// 4..8 hits per segment, 9 nodes, 10 triangles, 11 box tests, 12..15 hand-offs
// by cause.
__device__ void final_reduce(const TraceArgs &a, int s, int eval0, double *force, double *torque, int *err_flags,
                             unsigned long long *stats_accum, bool cg)
{
    // what the last step needs, loaded before the sums (a load is not moved across the barriers)
    const SlotPose &P = a.pose[s];
    double Du = 0.0, Dv = 0.0, scale = 0.0;
    int N = 0, pflags = 0;
    if (threadIdx.x == 0) {
        Du = ord_to_dbl(P.wmax_bits[0]) - ord_to_dbl(P.wmin_bits[0]);
        Dv = ord_to_dbl(P.wmax_bits[1]) - ord_to_dbl(P.wmin_bits[1]);
        scale = P.scale;
        pflags = cg ? __ldcg(&P.flags) : P.flags;
        N = a.sd[s].N;
    }
    __shared__ double red2[kPart][kRed1 / 32];
    __shared__ double red[kPart];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < kRed1) {
        const double *src = a.partials1 + ((size_t)s * kRed1 + threadIdx.x) * kPart;
        for (int k = 0; k < kPart; k++) {
            const double x = warp_sum(cg ? __ldcg(src + k) : src[k]);
            if (lane == 0) red2[k][w] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x < kPart) {
        double x = 0.0;
        for (int q = 0; q < kRed1 / 32; q++) x += red2[threadIdx.x][q];
        red[threadIdx.x] = x;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (a.sum_mode != 0) {
        // the FP32 modes: the first-level sums again, in order, in FP32
        for (int k = 0; k < 6; k++) {
            Comp32 x{0.0f, 0.0f};
            for (int b = 0; b < kRed1; b++) {
                const double *src = a.partials1 + ((size_t)s * kRed1 + b) * kPart + k;
                const float p = (float)(cg ? __ldcg(src) : *src);
                if (a.sum_mode == 1) comp_add(x, p);
                else x.hi = __fadd_rn(x.hi, p);
            }
            if (a.n_diffuse > 0)
                for (int b = 0; b < kDiffBlocks; b++) {
                    const float p = (float)a.dpart[((size_t)s * kDiffBlocks + b) * 6 + k];
                    if (a.sum_mode == 1) comp_add(x, p);
                    else x.hi = __fadd_rn(x.hi, p);
                }
            red[k] = (double)comp_value(x);
        }
    } else if (a.n_diffuse > 0) {
        for (int b = 0; b < kDiffBlocks; b++)
            for (int k = 0; k < 6; k++) red[k] += a.dpart[((size_t)s * kDiffBlocks + b) * 6 + k];
    }
    const double sc = scale * (Du * Dv) / ((double)N * (double)N);
    const int e = eval0 + s;
    for (int k = 0; k < 3; k++) {
        force[3 * e + k] = red[k] * sc;
        torque[3 * e + k] = red[3 + k] * sc;
    }
    if (pflags) atomicOr(err_flags, pflags);
    if (stats_accum) {
        atomicAdd(&stats_accum[0], 1ull);
        atomicAdd(&stats_accum[1], (unsigned long long)N * (unsigned long long)N);
        atomicAdd(&stats_accum[2], (unsigned long long)red[6]);
        atomicAdd(&stats_accum[3], (unsigned long long)red[7]);
        for (int k = 0; k < 5; k++) atomicAdd(&stats_accum[4 + k], (unsigned long long)red[8 + k]);
        for (int k = 0; k < 3; k++) atomicAdd(&stats_accum[9 + k], (unsigned long long)red[13 + k]);
        for (int k = 0; k < 4; k++) atomicAdd(&stats_accum[12 + k], (unsigned long long)red[16 + k]);
    }
}

// The second level as its own launch (after the diffuse rays), a block per slot.
__global__ void __launch_bounds__(kRed1) k_reduce(TraceArgs a, int eval0, double *force, double *torque, int *err_flags,
                                                unsigned long long *stats_accum)
{
    pdl_enter();
    const int s = blockIdx.x;
    if (a.pose[s].skip) {
        // a skipped evaluation outputs zero force and torque
        if (threadIdx.x < 6) (threadIdx.x < 3 ? force : torque)[3 * (eval0 + s) + threadIdx.x % 3] = 0.0;
        return;
    }
    final_reduce(a, s, eval0, force, torque, err_flags, stats_accum, false);
}

// ------------------------------------------------------------ BVH check
// One thread per part walks the part's 4-wide tree of slot 0 from the root:
// every child box of a reached node must lie inside the box its parent holds
// for that node (the root's inside the part's root box), every leaf
// triangle's three vertices inside its leaf box; each leaf reference is
// counted per triangle.  report: [0] leaf references, [2] child boxes outside
// the parent's, [3] leaf triangles outside their box, [4] nodes reached,
// [5] walks stopped by their bound ([1], [6], [7] are filled on the host).
__global__ void k_bvh_check(const unsigned char *tctx, int *tri_seen, unsigned long long *report)
{
    const TraceCtx &B = *reinterpret_cast<const TraceCtx *>(tctx);
    const PartView &pv = B.part[blockIdx.x];
    if (threadIdx.x != 0) return;
    unsigned long long refs = 0, outside_box = 0, outside_tri = 0, nodes = 0, bound = 0;
    auto inside = [](const float *in, const float *out) {
        return in[0] >= out[0] && in[1] <= out[1] && in[2] >= out[2] && in[3] <= out[3] && in[4] >= out[4] &&
               in[5] <= out[5];
    };
    auto tri_inside = [&](int tl, const float *bx) {
        const float4 *tr = pv.tri + (size_t)tl * 3;
        bool ok = true;
        for (int c = 0; c < 3; c++) {
            const float4 v = tr[c];
            ok = ok && v.x >= bx[0] && v.x <= bx[1] && v.y >= bx[2] && v.y <= bx[3] && v.z >= bx[4] && v.z <= bx[5];
        }
        atomicAdd(tri_seen + pv.tri_begin + tl, 1);
        refs++;
        if (!ok) outside_tri++;
    };
    const float *bs = pv.box_src;
    const float root_box[6] = {bs[0], bs[3], bs[1], bs[4], bs[2], bs[5]};
    if (pv.root < 0) {
        tri_inside(~pv.root, root_box);
    } else {
        // stack of (node, parent slot box) pairs: the box is re-read from the parent node
        constexpr int kCheckStack = 256;
        int st_node[kCheckStack], st_par[kCheckStack];
        int sp = 0, iters = 0;
        st_node[sp] = pv.root;
        st_par[sp] = -1;
        sp++;
        const int limit = pv.limit;
        while (sp > 0) {
            if (++iters > limit) { bound++; break; }
            sp--;
            const int nd = st_node[sp], par = st_par[sp];
            float pbox[6];
            if (par < 0) {
                for (int k = 0; k < 6; k++) pbox[k] = root_box[k];
            } else {
                const float4 *pn = pv.node + (size_t)(par >> 2) * kNode4;
                const int c = par & 3;
                for (int k = 0; k < 6; k++) pbox[k] = reinterpret_cast<const float *>(pn + k)[c];
            }
            const float4 *n = pv.node + (size_t)nd * kNode4;
            const int4 refs4 = *reinterpret_cast<const int4 *>(n + 6);
            const int rf[4] = {refs4.x, refs4.y, refs4.z, refs4.w};
            nodes++;
            for (int c = 0; c < 4; c++) {
                if (rf[c] == kEmptyChild) continue;
                float bx[6];
                for (int k = 0; k < 6; k++) bx[k] = reinterpret_cast<const float *>(n + k)[c];
                if (!inside(bx, pbox)) outside_box++;
                if (rf[c] >= 0) {
                    if (sp >= kCheckStack) { bound++; continue; }
                    st_node[sp] = rf[c];
                    st_par[sp] = nd * 4 + c;
                    sp++;
                } else {
                    tri_inside(~rf[c], bx);
                }
            }
        }
    }
    atomicAdd(report + 0, refs);
    atomicAdd(report + 2, outside_box);
    atomicAdd(report + 3, outside_tri);
    atomicAdd(report + 4, nodes);
    atomicAdd(report + 5, bound);
}

cudaError_t launch_bvh_check(const unsigned char *tctx, int n_parts, int *tri_seen, unsigned long long *report,
                             cudaStream_t st)
{
    k_bvh_check<<<n_parts, 32, 0, st>>>(tctx, tri_seen, report);
    return cudaGetLastError();
}

// ------------------------------------------------------------ launchers
// All-ones pixel keys (no hit, no candidate) before the first raster pass.
__global__ void __launch_bounds__(256) k_clear_keys(unsigned long long *key, size_t n)
{
    pdl_enter();
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        key[i] = ~0ull;
}

static int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return std::max(1, sms);
}

// Launch shapes by batch: a launch of few slots (a propagation stage) is
// latency-bound, so the frame kernel clears the pixel keys and the second
// raster pass is one launch; with many slots the launches overlap other lanes'
// traces, where a separate clear and separate second-pass launches measured faster.
constexpr int kFewSlots = 4;

int raster_launches(int S, bool queue)
{
    if (S < kFewSlots) return queue ? 3 : 4;  // first pass, chunk listing, chunks; the merged second pass
    return queue ? 4 : 6;                     // key clear, first pass, listing, chunks; two second-pass launches
}

cudaError_t launch_frame(const TraceArgs &a, int S, cudaStream_t st)
{
    const int sms = device_sms();
    const bool raster = a.raster && a.rast_tris > 0 && a.n_tiles > 0;
    const bool few = S < kFewSlots;
    TraceArgs f = a;
    if (!raster || !few) f.pix_key = nullptr;
    cudaError_t e;
    if (raster && few) {
        // the frame kernel's blocks beyond the context's warp clear the pixel keys
        const size_t per = (size_t)256 * 4;  // keys a block clears in one sweep of four
        const int ky = (int)std::max<size_t>(1, std::min((a.ray_stride + per - 1) / per,
                                                         (size_t)(sms * 4 + S - 1) / (size_t)S));
        e = launch_chained(k_frame, dim3(S, ky), dim3(256), 0, st, f);
    } else {
        e = launch_chained(k_frame, dim3(S, 1), dim3(32), 0, st, f);
    }
    if (e != cudaSuccess || !raster) return e;
    if (!few) {
        const size_t px = (size_t)S * a.ray_stride;
        const size_t kb = std::min((px + 255) / 256, (size_t)sms * 8);
        e = launch_chained(k_clear_keys, dim3((unsigned)std::max<size_t>(1, kb)), dim3(256), 0, st, a.pix_key, px);
        if (e != cudaSuccess) return e;
    }
    const dim3 grid((a.rast_tris + 127) / 128, S);
    // the chunk lists grow with the slots: a grid of the device's size per eight
    // slots, not of the lists' capacity
    const int big_blocks = sms * kRastBigBlocksPerSM * std::max(1, (S + 7) / 8);
    if ((e = launch_chained(k_raster<0>, grid, dim3(128), 0, st, a)) != cudaSuccess) return e;
    if ((e = launch_chained(k_raster_chunks, dim3(std::max(1, big_blocks / 4)), dim3(256), 0, st, a)) != cudaSuccess)
        return e;
    if ((e = launch_chained(k_raster_big<0>, dim3(big_blocks), dim3(256), 0, st, a)) != cudaSuccess) return e;
    if (a.queue) return cudaSuccess;  // the work queue runs the second pass with the trace
    if (few) {
        // the second pass over large triangles' chunks and small triangles: one launch
        const int nbig = 2 * big_blocks, per_slot = (int)grid.x;
        const unsigned blocks = (unsigned)nbig + (unsigned)per_slot * (unsigned)S;
        return launch_chained(k_raster_pass1, dim3(blocks), dim3(128), 0, st, a, nbig, per_slot);
    }
    if ((e = launch_chained(k_raster<1>, grid, dim3(128), 0, st, a)) != cudaSuccess) return e;
    return launch_chained(k_raster_big<1>, dim3(big_blocks), dim3(256), 0, st, a);
}

// The trace kernels' split of the SM's 256 KB between L1 and shared memory:
// a request for a small shared-memory configuration, so that L1 keeps most of
// the SM's memory for the hot tree nodes and the traversal stacks.  The
// driver's default had been 132 KB of shared memory (L1 124 KB); with this
// request and the context and hit columns sized per launch (7.4 KB a block of
// the headline workload) it takes 100 KB for the eight blocks the registers
// allow (L1 156 KB, L1 hit rate 68 -> 74%).  A percentage of the largest
// shared-memory configuration (228 KB); the driver rounds it up to a
// configuration that holds the blocks.
constexpr int kTraceCarveoutPct = 27;

cudaError_t configure_trace_kernels()
{
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, kTraceCarveoutPct);
    };
    set((const void *)k_trace<false, false>);
    set((const void *)k_trace<false, true>);
    set((const void *)k_trace<true, false>);
    set((const void *)k_trace<true, true>);
    set((const void *)k_queue<false, false>);
    set((const void *)k_queue<false, true>);
    set((const void *)k_queue<true, false>);
    set((const void *)k_queue<true, true>);
    return e;
}

cudaError_t launch_trace(const TraceArgs &a, int S, cudaStream_t st)
{
    (void)S;
    if (a.n_tiles <= 0) return cudaSuccess;
    // the hit records and the traversal counters are separate kernel variants:
    // code a launch never runs still costs registers in the others
    const dim3 g(a.n_tiles), b(kTileRays * kTraceWarps);
    const size_t dyn = trace_dyn_bytes(a.ctx_parts, a.hpt_segs);
    if (a.queue) {
        // persistent: as many blocks as fit on the device at once
        const dim3 gq(device_sms() * kQueueBlocksPerSM);
        if (a.count) return launch_chained(a.hits ? k_queue<true, true> : k_queue<true, false>, gq, b, dyn, st, a);
        return launch_chained(a.hits ? k_queue<false, true> : k_queue<false, false>, gq, b, dyn, st, a);
    }
    if (a.count) return launch_chained(a.hits ? k_trace<true, true> : k_trace<true, false>, g, b, dyn, st, a);
    return launch_chained(a.hits ? k_trace<false, true> : k_trace<false, false>, g, b, dyn, st, a);
}

cudaError_t launch_reduce(const TraceArgs &a, int S, int eval0, double *force, double *torque, int *err_flags,
                          unsigned long long *stats_accum, cudaStream_t st)
{
    // without diffuse rays the last first-level block of a slot does the second level
    const int fuse = (a.n_diffuse <= 0 && a.red_ticket) ? 1 : 0;
    cudaError_t e = launch_chained(k_reduce1, dim3(kRed1, S), dim3(256), 0, st, a, eval0, force, torque, err_flags,
                                   stats_accum, fuse);
    if (e != cudaSuccess || fuse) return e;
    // diffuse secondaries after the FP64 re-trace (which records the hits of the rays it takes)
    if (a.n_diffuse > 0) {
        if ((e = launch_chained(k_demit, dim3(kDiffBlocks, S), dim3(kLaneStride), 0, st, a)) != cudaSuccess) return e;
        if ((e = launch_chained(k_dscan, dim3(S), dim3(1024), 0, st, a)) != cudaSuccess) return e;
        if ((e = launch_chained(k_diffuse, dim3(kDiffBlocks, S), dim3(kLaneStride), 0, st, a)) != cudaSuccess) return e;
    }
    return launch_chained(k_reduce, dim3(S), dim3(kRed1), 0, st, a, eval0, force, torque, err_flags, stats_accum);
}

}  // namespace srp
