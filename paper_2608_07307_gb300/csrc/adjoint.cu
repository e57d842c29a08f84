// adjoint.cu -- reverse-mode derivative of one SRP evaluation with the hit set
// frozen: each ray segment meets the plane of the triangle the trace recorded
// for it, and the window spans the four vertices that were extreme, so the
// force and torque are smooth functions of the optical coefficients, the joint
// angles (hence the joint offsets and, through Sun tracking, the Sun
// direction), the Sun direction and the Sun distance (Sec. 4.3, 4.4.2, 6.1).
//
//   k_adj_window  blocks per slot over the posed vertices, extreme along u and v
//                 (k_adj_window_merge: the blocks' extremes in block order)
//                 (lowest vertex index among equal projections).
//   k_adj_rays    grid-stride over the rays of every slot: per ray, the
//                 segments are replayed forward in FP32 from the recorded hits,
//                 then swept backward; cotangents of the ray direction, the
//                 basis, the window bounds and the local loss stay in
//                 registers; per-coefficient and per-part terms are summed
//                 over the warp for each distinct key (fixed butterfly) and
//                 added by one lane into the warp's own shared-memory row.
//                 Every sum has a fixed order: the result is deterministic.
//   k_adj_finish  one block per slot: the block partials are added in block
//                 order, then one thread chains window -> vertices, basis ->
//                 direction, joint rotations -> angles, Sun tracking ->
//                 direction, normalisation -> the direction as given.
//   k_adj_sum     coefficient and angle gradients summed over the batch in
//                 evaluation order.
//
// Scalar loss per evaluation: L = g_F . F + g_T . T, F = scale * A_pix * sum f,
// per segment f = w [(1 - rho_s) d - 2 (rho_s c + rho_d / 3) n_f],
// T = scale * A_pix * sum (x - c_ref) x f.
#include <math.h>

#include <algorithm>

#include "srp_internal.cuh"

namespace srp {

namespace {

constexpr int kAdjThreads = 256;
constexpr int kAdjWarps = kAdjThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

struct V3 {
    double x, y, z;
};
__device__ inline V3 v3(double x, double y, double z) { return {x, y, z}; }
__device__ inline V3 ld3(const double *p) { return {p[0], p[1], p[2]}; }
__device__ inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ inline V3 &operator+=(V3 &a, V3 b) { a.x += b.x; a.y += b.y; a.z += b.z; return a; }
__device__ inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
__device__ inline V3 mat_mul(const double *M, V3 x)
{
    return {M[0] * x.x + M[1] * x.y + M[2] * x.z, M[3] * x.x + M[4] * x.y + M[5] * x.z,
            M[6] * x.x + M[7] * x.y + M[8] * x.z};
}
__device__ inline V3 mat_tmul(const double *M, V3 x)
{
    return {M[0] * x.x + M[3] * x.y + M[6] * x.z, M[1] * x.x + M[4] * x.y + M[7] * x.z,
            M[2] * x.x + M[5] * x.y + M[8] * x.z};
}

__device__ inline double wsum(double x)
{
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// posed FP64 position of (re-indexed) vertex v of a slot
__device__ inline V3 vertex(const MeshDev &m, const SlotBufs &sb, int v)
{
    const PartInfo &pi = m.part[m.vert_part[v]];
    if (!pi.dynamic) return ld3(m.rest64 + 3 * (size_t)v);
    return ld3(sb.vert64 + (size_t)(v - pi.vert_begin + pi.dyn_vert_off) * 3);
}

// Add val[0..n) of the lanes holding `key` (>= 0) into row[key * n ..], for
// every distinct key in the warp: masked butterfly sums, one writer (lane 0).
template <int n>
__device__ inline void warp_scatter(int key, const double *val, double *row)
{
    unsigned todo = __ballot_sync(kFull, key >= 0);
    while (todo) {
        int k = __shfl_sync(kFull, key, __ffs(todo) - 1);
        bool mine = key == k;
        double sum[n];
#pragma unroll
        for (int c = 0; c < n; c++) sum[c] = wsum(mine ? val[c] : 0.0);
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int c = 0; c < n; c++) row[k * n + c] += sum[c];
        }
        todo &= ~__ballot_sync(kFull, mine);
    }
}

// ------------------------------------------------------------- window
__global__ void __launch_bounds__(kAdjThreads) k_adj_window(AdjArgs a)
{
    const int s = blockIdx.y, b = blockIdx.x, G = gridDim.x;
    const SlotPose &P = a.pose[s];
    if (P.skip) return;
    const MeshDev &m = *a.sd[s].mesh;
    const SlotBufs &sb = a.sd[s].sb;
    V3 u = ld3(P.u), v = ld3(P.v);
    double best[4] = {INFINITY, -INFINITY, INFINITY, -INFINITY};
    int id[4] = {-1, -1, -1, -1};
    for (int k = b * blockDim.x + threadIdx.x; k < m.n_verts; k += G * blockDim.x) {  // ascending k per thread
        V3 x = vertex(m, sb, k);
        double pu = dot(u, x), pv = dot(v, x);
        if (pu < best[0]) { best[0] = pu; id[0] = k; }
        if (pu > best[1]) { best[1] = pu; id[1] = k; }
        if (pv < best[2]) { best[2] = pv; id[2] = k; }
        if (pv > best[3]) { best[3] = pv; id[3] = k; }
    }
    __shared__ double sv[4][kAdjThreads];
    __shared__ int si[4][kAdjThreads];
    for (int c = 0; c < 4; c++) { sv[c][threadIdx.x] = best[c]; si[c][threadIdx.x] = id[c]; }
    __syncthreads();
    for (int h = kAdjThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            for (int c = 0; c < 4; c++) {
                double b0 = sv[c][threadIdx.x], b1 = sv[c][threadIdx.x + h];
                int i0 = si[c][threadIdx.x], i1 = si[c][threadIdx.x + h];
                bool take = (c & 1) ? (b1 > b0) : (b1 < b0);
                if (i1 >= 0 && (i0 < 0 || take || (b1 == b0 && i1 < i0))) {
                    sv[c][threadIdx.x] = b1;
                    si[c][threadIdx.x] = i1;
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) {
        const size_t o = ((size_t)s * G + b) * 4 + threadIdx.x;
        a.win_val[o] = sv[threadIdx.x][0];
        a.win_pid[o] = si[threadIdx.x][0];
    }
}

// The blocks' extremes of a slot merged in block order: the extreme value, the
// lowest vertex id among equal values (the single-block search's result).
__global__ void k_adj_window_merge(AdjArgs a, int G)
{
    const int s = blockIdx.x, c = threadIdx.x;
    if (a.pose[s].skip || c >= 4) return;
    double best = (c & 1) ? -INFINITY : INFINITY;
    int id = -1;
    for (int b = 0; b < G; b++) {
        const size_t o = ((size_t)s * G + b) * 4 + c;
        const double v = a.win_val[o];
        const int i = a.win_pid[o];
        const bool take = (c & 1) ? (v > best) : (v < best);
        if (i >= 0 && (id < 0 || take || (v == best && i < id))) {
            best = v;
            id = i;
        }
    }
    a.win_ids[4 * s + c] = id;
}

// --------------------------------------------------------------- rays
// Per-ray arithmetic is FP32 (GB300's FP64 rate is a small fraction of its
// FP32 rate; a ray's terms are O(1) with relative rounding ~1e-7), sums over
// rays are FP64 from the warp level up.
struct F3 {
    float x, y, z;
};
__device__ inline F3 f3(float x, float y, float z) { return {x, y, z}; }
__device__ inline F3 f3(V3 a) { return {(float)a.x, (float)a.y, (float)a.z}; }
__device__ inline F3 operator+(F3 a, F3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ inline F3 operator-(F3 a, F3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ inline F3 operator*(float s, F3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ inline F3 &operator+=(F3 &a, F3 b) { a.x += b.x; a.y += b.y; a.z += b.z; return a; }
__device__ inline float dot(F3 a, F3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline F3 cross(F3 a, F3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }

__device__ inline float wsumf(float x)
{
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// FP32 copy of a posed vertex
__device__ inline F3 vertex32(const MeshDev &m, const SlotBufs &sb, int v) { return f3(vertex(m, sb, v)); }

// warp_scatter with FP32 lane values and FP64 accumulation
template <int n>
__device__ inline void warp_scatter32(int key, const float *val, double *row)
{
    unsigned todo = __ballot_sync(kFull, key >= 0);
    while (todo) {
        int k = __shfl_sync(kFull, key, __ffs(todo) - 1);
        bool mine = key == k;
        float sum[n];
#pragma unroll
        for (int c = 0; c < n; c++) sum[c] = wsumf(mine ? val[c] : 0.0f);
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int c = 0; c < n; c++) row[k * n + c] += (double)sum[c];
        }
        todo &= ~__ballot_sync(kFull, mine);
    }
}

__global__ void __launch_bounds__(kAdjThreads) k_adj_rays(AdjArgs a)
{
    const int s = blockIdx.y;
    const SlotPose &P = a.pose[s];
    if (P.skip) return;
    const MeshDev &m = *a.sd[s].mesh;
    const SlotBufs &sb = a.sd[s].sb;
    const int e = a.eval0 + s, N = a.sd[s].N, nseg = a.sd[s].nseg;
    const int W = a.width, nm2 = 2 * a.n_mats;
    extern __shared__ double sh[];  // [kAdjWarps][W]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *row = sh + (size_t)warp * W;
    for (int k = lane; k < W; k += 32) row[k] = 0.0;
    __syncwarp();
    __shared__ double win[4];
    if (threadIdx.x < 4) {
        int vi = a.win_ids[4 * s + threadIdx.x];
        V3 x = vertex(m, sb, vi);
        win[threadIdx.x] = dot(threadIdx.x < 2 ? ld3(P.u) : ld3(P.v), x);
    }
    __syncthreads();
    const F3 u = f3(ld3(P.u)), v = f3(ld3(P.v)), d0 = f3(ld3(P.d)), cref = f3(ld3(m.c_ref));
    const F3 gF = f3(ld3(a.g_force + 3 * (size_t)e)), gT = f3(ld3(a.g_torque + 3 * (size_t)e));
    const float umin = (float)win[0], vmin = (float)win[2];
    const float Du = (float)((win[1] - win[0]) / N), Dv = (float)((win[3] - win[2]) / N);
    const size_t R = (size_t)N * N;
    F3 acc_d = f3(0, 0, 0), acc_u = f3(0, 0, 0), acc_v = f3(0, 0, 0);
    float acc_w[4] = {0, 0, 0, 0}, acc_l = 0.0f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of iterations (warp_scatter needs the whole warp)
    const size_t iters = (R + stride - 1) / stride;
    for (size_t it = 0; it < iters; it++) {
        const size_t ray = it * stride + (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        const bool live = ray < R;
        int tri[kMaxBounces + 1];
        int nh = 0;
        if (live) {
            const int32_t *hq = a.hits + ((size_t)s * a.ray_stride + ray) * a.seg_stride;
            for (int k = 0; k < nseg; k++) {
                int h = hq[k];
                if (h < 0) break;
                tri[nh++] = m.tri_pos[h];
            }
        }
        const int i = live ? (int)(ray / N) : 0, j = live ? (int)(ray % N) : 0;
        const float al = (i + 0.5f) / N, be = (j + 0.5f) / N;
        const float uc = fmaf(i + 0.5f, Du, umin), vc = fmaf(j + 0.5f, Dv, vmin);
        // forward replay: origin, direction and weight entering each segment
        F3 so[kMaxBounces + 1], sd[kMaxBounces + 1];
        float sw[kMaxBounces + 1];
        {
            F3 o = uc * u + vc * v, d = d0;
            float w = 1.0f;
            for (int k = 0; k < nh; k++) {
                so[k] = o; sd[k] = d; sw[k] = w;
                int4 tv = m.tri_v4[tri[k]];
                F3 A = vertex32(m, sb, tv.x), B = vertex32(m, sb, tv.y), C = vertex32(m, sb, tv.z);
                F3 n = cross(B - A, C - A);
                n = rsqrtf(dot(n, n)) * n;
                float dn = dot(d, n);
                float t = dot(n, A - o) / dn;
                F3 x = o + t * d;
                unsigned mp = m.tri_mat[tri[k]];
                int mi = dn < 0.0f ? (int)(mp & 0xffffu) : (int)(mp >> 16);
                w *= m.mat32[mi].x;
                d = d - (2.0f * dn) * n;
                o = x;
            }
        }
        // backward sweep, uniform over the warp
        F3 ob = f3(0, 0, 0), db = f3(0, 0, 0);
        float wb = 0.0f;
        for (int k = nseg - 1; k >= 0; k--) {
            const bool act = k < nh;
            int mkey = -1, pkey = -1;
            float mval[2] = {0.0f, 0.0f}, pval[6] = {0, 0, 0, 0, 0, 0};
            if (act) {
                const F3 o = so[k], d = sd[k];
                const float w = sw[k];
                const int4 tv = m.tri_v4[tri[k]];
                const F3 A = vertex32(m, sb, tv.x), B = vertex32(m, sb, tv.y),
                         C = vertex32(m, sb, tv.z);
                const F3 e1 = B - A, e2 = C - A, mr = cross(e1, e2);
                const float il = rsqrtf(dot(mr, mr));
                const F3 n = il * mr;
                const float dn = dot(d, n);
                const F3 ao = A - o;
                const float t = dot(n, ao) / dn;
                const F3 x = o + t * d;
                const unsigned mp = m.tri_mat[tri[k]];
                const bool front = dn < 0.0f;
                const int mi = front ? (int)(mp & 0xffffu) : (int)(mp >> 16);
                const float2 rho = m.mat32[mi];
                const float rs = rho.x, rd = rho.y;
                const float sg = front ? 1.0f : -1.0f;
                const F3 nf = sg * n;
                const float c = -dot(nf, d);
                const float kq = rs * c + rd * (1.0f / 3.0f);
                const F3 q = (1.0f - rs) * d - (2.0f * kq) * nf;
                const F3 f = w * q;
                const F3 r = x - cref;
                acc_l += dot(gF, f) + dot(gT, cross(r, f));
                // cotangents
                const F3 fb = gF + cross(gT, r);
                const F3 xb = cross(f, gT) + ob;      // ob: cotangent of the next segment's origin (= x)
                float wl = dot(fb, q);                // cotangent of w
                const F3 qb = w * fb;
                float rsb = dot(qb, -1.0f * d - (2.0f * c) * nf);
                float rdb = -(2.0f / 3.0f) * dot(qb, nf);
                F3 dbl = (1.0f - rs) * qb;            // cotangent of d (this segment)
                const float cb = -2.0f * rs * dot(qb, nf);
                F3 nfb = (-2.0f * kq) * qb;
                float dnb = 0.0f;
                F3 nb = f3(0, 0, 0);
                if (k + 1 < nh) {                     // the next segment's d' = d - 2 dn n and w' = w rho_s
                    rsb += wb * w;
                    wl += wb * rs;
                    dbl += db;
                    dnb += -2.0f * dot(db, n);
                    nb += (-2.0f * dn) * db;
                }
                nfb += (-cb) * d;                     // c = -nf . d
                dbl += (-cb) * nf;
                nb += sg * nfb;
                F3 obl = xb;                          // x = o + t d
                const float tb = dot(xb, d);
                dbl += t * xb;
                const float naob = tb / dn;           // t = (n . ao) / dn
                dnb += -tb * t / dn;
                nb += naob * ao;
                F3 Ab = naob * n;
                obl += (-naob) * n;
                dbl += dnb * n;                       // dn = d . n
                nb += dnb * d;
                const F3 mb = il * (nb - dot(nb, n) * n);
                const F3 e1b = cross(e2, mb), e2b = cross(mb, e1);
                Ab += -1.0f * (e1b + e2b);
                mkey = mi;
                mval[0] = rsb;
                mval[1] = rdb;
                const int pp = m.vert_part[tv.x];
                if (m.part[pp].dynamic) {
                    pkey = pp;
                    const F3 G = Ab + e1b + e2b, Mm = cross(A, Ab) + cross(B, e1b) + cross(C, e2b);
                    pval[0] = G.x; pval[1] = G.y; pval[2] = G.z;
                    pval[3] = Mm.x; pval[4] = Mm.y; pval[5] = Mm.z;
                }
                ob = obl;
                db = dbl;
                wb = wl;
            }
            warp_scatter32<2>(mkey, mval, row + kAdjFixed);
            warp_scatter32<6>(pkey, pval, row + kAdjFixed + nm2);
        }
        if (nh > 0) {
            // primary origin o = uc u + vc v (its component along d does not move the hit point)
            acc_d += db;
            acc_u += uc * ob;
            acc_v += vc * ob;
            const float ucb = dot(u, ob), vcb = dot(v, ob);
            acc_w[0] += (1.0f - al) * ucb;
            acc_w[1] += al * ucb;
            acc_w[2] += (1.0f - be) * vcb;
            acc_w[3] += be * vcb;
        }
    }
    float fix[kAdjFixed] = {acc_d.x, acc_d.y, acc_d.z, acc_u.x, acc_u.y, acc_u.z, acc_v.x, acc_v.y, acc_v.z,
                            acc_w[0], acc_w[1], acc_w[2], acc_w[3], acc_l};
#pragma unroll
    for (int c = 0; c < kAdjFixed; c++) {
        double x = wsum((double)fix[c]);
        if (lane == 0) row[c] += x;
    }
    __syncthreads();
    double *out = a.partials + ((size_t)s * a.nb + blockIdx.x) * W;
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
        double x = 0.0;
        for (int w = 0; w < kAdjWarps; w++) x += sh[(size_t)w * W + k];
        out[k] = x;
    }
}

// -------------------------------------------------------------- finish
// The column sums of runs of kAdjSumRun ray-block partials, a block per (run,
// slot): the first of two fixed-order levels when a slot has many ray blocks
// (one evaluation a launch), so that no single thread adds hundreds of FP64
// values in a row.
__global__ void __launch_bounds__(128) k_adj_finish_sum(AdjArgs a)
{
    const int s = blockIdx.y, g = blockIdx.x, G = gridDim.x, W = a.width;
    if (a.pose[s].skip) return;
    const int b0 = g * kAdjSumRun, b1 = min(b0 + kAdjSumRun, a.nb);
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
        double x = 0.0;
        for (int b = b0; b < b1; b++) x += a.partials[((size_t)s * a.nb + b) * W + k];
        a.partials2[((size_t)s * G + g) * W + k] = x;
    }
}

__global__ void __launch_bounds__(128) k_adj_finish(AdjArgs a, int runs)
{
    const int s = blockIdx.x;
    const SlotPose &P = a.pose[s];
    const MeshDev &m = *a.sd[s].mesh;
    const SlotBufs &sb = a.sd[s].sb;
    const int e = a.eval0 + s, W = a.width, nm2 = 2 * a.n_mats, np = a.n_parts;
    double *ge = a.g_eval + (size_t)e * (nm2 + np);
    if (P.skip) {
        for (int k = threadIdx.x; k < nm2 + np; k += blockDim.x) ge[k] = 0.0;
        if (threadIdx.x < 3) a.g_sun[3 * (size_t)e + threadIdx.x] = 0.0;
        if (threadIdx.x == 0 && a.g_dist) a.g_dist[e] = 0.0;
        return;
    }
    extern __shared__ double tot[];  // [W]
    // the ray blocks' partials in block order, directly or as the runs' sums in run order
    const double *src = runs > 0 ? a.partials2 : a.partials;
    const int cnt = runs > 0 ? runs : a.nb;
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
        double x = 0.0;
        for (int b = 0; b < cnt; b++) x += src[((size_t)s * cnt + b) * W + k];
        tot[k] = x;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int N = a.sd[s].N;
    const int *ids = a.win_ids + 4 * s;
    V3 X[4];
    for (int c = 0; c < 4; c++) X[c] = vertex(m, sb, ids[c]);
    V3 u = ld3(P.u), v = ld3(P.v), d = ld3(P.d), sh = ld3(P.s);
    const double umin = dot(u, X[0]), umax = dot(u, X[1]), vmin = dot(v, X[2]), vmax = dot(v, X[3]);
    const double area = (umax - umin) * (vmax - vmin) / ((double)N * N);
    const double sc = P.scale * area;
    const double Lsum = tot[13], L = sc * Lsum;
    V3 db = sc * v3(tot[0], tot[1], tot[2]);
    V3 ub = sc * v3(tot[3], tot[4], tot[5]);
    V3 vb = sc * v3(tot[6], tot[7], tot[8]);
    double wb[4] = {sc * tot[9], sc * tot[10], sc * tot[11], sc * tot[12]};
    // pixel area: A_pix = (umax - umin)(vmax - vmin) / N^2
    const double kA = P.scale * Lsum / ((double)N * N);
    wb[0] -= kA * (vmax - vmin);
    wb[1] += kA * (vmax - vmin);
    wb[2] -= kA * (umax - umin);
    wb[3] += kA * (umax - umin);
    // part accumulators: G = sum of vertex cotangents, M = sum of x cross cotangent
    double G[kMaxParts][3], Mx[kMaxParts][3];
    for (int p = 0; p < np; p++)
        for (int c = 0; c < 3; c++) {
            G[p][c] = sc * tot[kAdjFixed + nm2 + 6 * p + c];
            Mx[p][c] = sc * tot[kAdjFixed + nm2 + 6 * p + 3 + c];
        }
    // window bounds: umin = u . X0, umax = u . X1, vmin = v . X2, vmax = v . X3
    for (int c = 0; c < 4; c++) {
        const V3 ax = c < 2 ? u : v;
        if (c < 2) ub += wb[c] * X[c]; else vb += wb[c] * X[c];
        const int p = m.vert_part[ids[c]];
        if (m.part[p].dynamic) {
            const V3 g = wb[c] * ax, mm = cross(X[c], g);
            G[p][0] += g.x; G[p][1] += g.y; G[p][2] += g.z;
            Mx[p][0] += mm.x; Mx[p][1] += mm.y; Mx[p][2] += mm.z;
        }
    }
    // joint angles: a rotation d theta of joint q moves every vertex of its
    // subtree by (a_q x (x - p_q)) d theta, a_q and p_q the axis and pivot in
    // the body frame, so dL/dtheta_q = a_q . sum over the subtree (M - p_q x G)
    double thb[kMaxParts];
    for (int q = 0; q < np; q++) {
        thb[q] = 0.0;
        const PartInfo &pq = m.part[q];
        if (!pq.movable) continue;
        const int par = pq.parent;
        const V3 aw = mat_mul(P.M[par], ld3(pq.axis));
        const V3 pw = mat_mul(P.M[par], ld3(pq.pivot)) + ld3(P.T[par]);
        V3 Gs = v3(0, 0, 0), Ms = v3(0, 0, 0);
        for (int p = 0; p < np; p++) {
            int x = p;
            while (x > q) x = m.part[x].parent;
            if (x != q) continue;
            Gs += v3(G[p][0], G[p][1], G[p][2]);
            Ms += v3(Mx[p][0], Mx[p][1], Mx[p][2]);
        }
        thb[q] = dot(aw, Ms - cross(pw, Gs));
    }
    // Sun tracking, children first: theta_q = atan2(b . s', n . s') (+ offset),
    // s' = M_parent^T s; s' also turns with every movable ancestor of q
    V3 shb = v3(0, 0, 0);
    for (int q = np - 1; q >= 1; q--) {
        const PartInfo &pq = m.part[q];
        const bool free = (P.free_mask >> q) & 1u;
        ge[nm2 + q] = free ? thb[q] : 0.0;
        if (!free || !((P.track_mask >> q) & 1u) || a.panel_mode == SRP_PANELS_SET) continue;
        const int par = pq.parent;
        const V3 ax = ld3(pq.axis), n0 = ld3(pq.n0);
        const V3 nn = n0 - dot(n0, ax) * ax;
        const V3 bb = cross(ax, nn);
        const V3 sl = mat_tmul(P.M[par], sh);
        const double x = dot(nn, sl), y = dot(bb, sl), den = x * x + y * y;
        const V3 slb = (thb[q] / den) * (x * bb - y * nn);
        const V3 g = mat_mul(P.M[par], slb);  // cotangent of s through s'
        shb += g;
        for (int an = par; an > 0; an = m.part[an].parent) {
            const PartInfo &pa = m.part[an];
            if (!pa.movable || !((P.free_mask >> an) & 1u)) continue;
            const V3 aw = mat_mul(P.M[pa.parent], ld3(pa.axis));
            thb[an] += -dot(g, cross(aw, sh));
        }
    }
    ge[nm2 + 0] = 0.0;
    for (int k = 0; k < nm2; k++) ge[k] = sc * tot[kAdjFixed + k];
    // basis (u, v) of the plane normal to d (Duff et al., JCGT 2017), differentiated
    {
        const double sg = copysign(1.0, d.z);
        const double aa = -1.0 / (sg + d.z);
        const double bbv = sg * ub.y + vb.x;              // cotangent of b = dx dy a
        const double ab = sg * d.x * d.x * ub.x + d.y * d.y * vb.y + bbv * d.x * d.y;
        db.x += 2.0 * sg * d.x * aa * ub.x - sg * ub.z + bbv * d.y * aa;
        db.y += 2.0 * d.y * aa * vb.y - vb.z + bbv * d.x * aa;
        db.z += ab * aa * aa;
    }
    // d = -s_hat, s_hat = s / |s|
    shb += -1.0 * db;
    const V3 gs = (1.0 / P.s_norm) * (shb - dot(shb, sh) * sh);
    a.g_sun[3 * (size_t)e] = gs.x;
    a.g_sun[3 * (size_t)e + 1] = gs.y;
    a.g_sun[3 * (size_t)e + 2] = gs.z;
    if (a.g_dist) a.g_dist[e] = -2.0 * L / a.sun_dist[e];  // pressure P0 / dist^2
}

__global__ void k_adj_sum(const double *g_eval, int n, int width, double *g_mat, int nm2, double *g_angle, int accumulate)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= width) return;
    double x = 0.0;
    for (int e = 0; e < n; e++) x += g_eval[(size_t)e * width + k];
    double *dst = k < nm2 ? (g_mat ? g_mat + k : nullptr) : (g_angle ? g_angle + (k - nm2) : nullptr);
    if (dst) *dst = accumulate ? *dst + x : x;
}

}  // namespace

int adj_blocks(int S, size_t rays)
{
    // about four blocks per SM over the S evaluations of a chunk
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
        sms = 1;
    size_t need = (rays + kAdjThreads - 1) / kAdjThreads;
    size_t cap = (size_t)std::max(1, 4 * sms / std::max(S, 1));
    return (int)std::max<size_t>(1, std::min(need, cap));
}

cudaError_t launch_adjoint(const AdjArgs &a, int S, cudaStream_t st)
{
    // the window search over the vertices: several blocks a slot (four vertices
    // a thread), merged in block order
    const int G = std::max(1, std::min(kAdjWinBlocks, (a.n_verts + 4 * kAdjThreads - 1) / (4 * kAdjThreads)));
    k_adj_window<<<dim3(G, S), kAdjThreads, 0, st>>>(a);
    k_adj_window_merge<<<S, 32, 0, st>>>(a, G);
    size_t smem = sizeof(double) * (size_t)kAdjWarps * a.width;
    k_adj_rays<<<dim3(a.nb, S), kAdjThreads, smem, st>>>(a);
    const int runs = a.nb > 2 * kAdjSumRun && a.partials2 ? (a.nb + kAdjSumRun - 1) / kAdjSumRun : 0;
    if (runs > 0) k_adj_finish_sum<<<dim3(runs, S), 128, 0, st>>>(a);
    k_adj_finish<<<S, 128, sizeof(double) * a.width, st>>>(a, runs);
    return cudaGetLastError();
}

cudaError_t launch_adj_sum(const double *g_eval, int n, int n_mats, int n_parts, double *g_mat, double *g_angle,
                           cudaStream_t st, bool accumulate)
{
    int width = 2 * n_mats + n_parts;
    k_adj_sum<<<(width + 127) / 128, 128, 0, st>>>(g_eval, n, width, g_mat, 2 * n_mats, g_angle, accumulate ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace srp
