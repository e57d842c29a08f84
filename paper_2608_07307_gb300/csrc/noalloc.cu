// noalloc.cu -- srp_eval_noalloc: an SRP evaluation that allocates no memory.
//
// For callers that cannot allocate device memory at run time: flight or
// real-time software whose memory is fixed at start-up (an allocation could
// fail or stall mid-mission), or a host that only hands out memory through its
// own pool.  The caller passes every input and output; the only scratch is the
// file-scope array below, reserved when the library is loaded.
//
// It is a variant of the FP64 re-trace kernel of trace.cu without the BVH:
// each ray is tested against every triangle (small meshes only), in FP64, so
// its hits agree with the main path, whose FP32 decisions are either exact or
// handed to that same FP64 path.  The paper has no counterpart.
#include <math.h>

#include <mutex>

#include "srp_internal.cuh"

namespace srp {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = SRP_NOALLOC_MAX_N * SRP_NOALLOC_MAX_N / kNaThreads;
constexpr int kNaTile = 128;  // triangles staged in shared memory per pass

// Scratch shared by every call on a device: [0..7] window bounds (umin umax
// vmin vmax wmin wmax), [8 ..] one 8-double partial sum per trace block.
// 8 + 4096 * 8 doubles = 262 208 bytes, held by each GPU that loads the library.
constexpr int kNaScratch = 8 + kNaMaxBlocks * 8;
static __device__ __align__(256) double g_na_scratch[kNaScratch];

struct NaArgs {
    const double *xyz;     // [n_tris][9] posed vertices
    const int32_t *tmat;   // [n_tris][2]
    const double *mat;     // [n_mats][2]
    int n_tris, n_mats, N, nseg;
    double u[3], v[3], d[3];
    double c_ref[3];
    double eps_rel, scale;
};

__global__ void __launch_bounds__(kNaThreads) k_na_window(NaArgs a, double *scratch)
{
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = threadIdx.x; k < 3 * a.n_tris; k += blockDim.x) {
        const double *x = a.xyz + 3 * (size_t)k;
        const double *ax[3] = {a.u, a.v, a.d};
        for (int c = 0; c < 3; c++) {
            double p = ax[c][0] * x[0] + ax[c][1] * x[1] + ax[c][2] * x[2];
            mn[c] = fmin(mn[c], p);
            mx[c] = fmax(mx[c], p);
        }
    }
    __shared__ double smn[3][kNaThreads], smx[3][kNaThreads];
    for (int c = 0; c < 3; c++) { smn[c][threadIdx.x] = mn[c]; smx[c][threadIdx.x] = mx[c]; }
    __syncthreads();
    for (int h = kNaThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int c = 0; c < 3; c++) {
                smn[c][threadIdx.x] = fmin(smn[c][threadIdx.x], smn[c][threadIdx.x + h]);
                smx[c][threadIdx.x] = fmax(smx[c][threadIdx.x], smx[c][threadIdx.x + h]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; c++) { scratch[2 * c] = smn[c][0]; scratch[2 * c + 1] = smx[c][0]; }
}

__device__ __forceinline__ double pk(const double *x, int k) { return k == 0 ? x[0] : (k == 1 ? x[1] : x[2]); }

__global__ void __launch_bounds__(kNaThreads) k_na_trace(NaArgs a, double *scratch)
{
    __shared__ double tv[kNaTile][9];
    __shared__ int tid_[kNaTile];
    const double umin = scratch[0], umax = scratch[1], vmin = scratch[2], vmax = scratch[3];
    const double wmin = scratch[4], wmax = scratch[5];
    const double Du = umax - umin, Dv = vmax - vmin, Dw = wmax - wmin;
    const double eps = a.eps_rel * sqrt(Du * Du + Dv * Dv + Dw * Dw);
    const size_t R = (size_t)a.N * a.N;
    size_t ray = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool live = ray < R;
    double o[3], dir[3], w = 1.0, acc[6] = {0, 0, 0, 0, 0, 0};
    int skip = -1;
    if (live) {
        int i = (int)(ray / a.N), j = (int)(ray % a.N);
        double uc = umin + ((double)i + 0.5) * Du / a.N, vc = vmin + ((double)j + 0.5) * Dv / a.N;
        double w0 = wmin - kStandoff;
        for (int k = 0; k < 3; k++) { o[k] = uc * a.u[k] + vc * a.v[k] + w0 * a.d[k]; dir[k] = a.d[k]; }
    }
    for (int seg = 0; seg < a.nseg; seg++) {
        // watertight set-up of this segment's ray (FP64)
        int kx = 0, ky = 1, kz = 2;
        double Sx = 0, Sy = 0, Sz = 1;
        if (live) {
            double ax = fabs(dir[0]), ay = fabs(dir[1]), az = fabs(dir[2]);
            kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
            kx = kz == 2 ? 0 : kz + 1;
            ky = kx == 2 ? 0 : kx + 1;
            if (pk(dir, kz) < 0.0) { int t = kx; kx = ky; ky = t; }
            Sx = pk(dir, kx) / pk(dir, kz);
            Sy = pk(dir, ky) / pk(dir, kz);
            Sz = 1.0 / pk(dir, kz);
        }
        double bt = INFINITY;
        int best = -1;
        for (int t0 = 0; t0 < a.n_tris; t0 += kNaTile) {
            __syncthreads();
            for (int q = threadIdx.x; q < kNaTile * 9; q += blockDim.x) {
                int t = t0 + q / 9;
                tv[q / 9][q % 9] = t < a.n_tris ? a.xyz[9 * (size_t)t + q % 9] : 0.0;
            }
            for (int q = threadIdx.x; q < kNaTile; q += blockDim.x) tid_[q] = t0 + q;
            __syncthreads();
            if (!live) continue;
            int nt = min(kNaTile, a.n_tris - t0);
            for (int q = 0; q < nt; q++) {
                int t = tid_[q];
                if (t == skip) continue;
                double A[3], B[3], C[3];
                for (int k = 0; k < 3; k++) { A[k] = tv[q][k] - o[k]; B[k] = tv[q][3 + k] - o[k]; C[k] = tv[q][6 + k] - o[k]; }
                double Ax = pk(A, kx) - Sx * pk(A, kz), Ay = pk(A, ky) - Sy * pk(A, kz);
                double Bx = pk(B, kx) - Sx * pk(B, kz), By = pk(B, ky) - Sy * pk(B, kz);
                double Cx = pk(C, kx) - Sx * pk(C, kz), Cy = pk(C, ky) - Sy * pk(C, kz);
                double U = __dsub_rn(__dmul_rn(Cx, By), __dmul_rn(Cy, Bx));
                double V = __dsub_rn(__dmul_rn(Ax, Cy), __dmul_rn(Ay, Cx));
                double W = __dsub_rn(__dmul_rn(Bx, Ay), __dmul_rn(By, Ax));
                if ((U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0)) continue;
                double det = U + V + W;
                if (det == 0.0) continue;
                double T = U * (Sz * pk(A, kz)) + V * (Sz * pk(B, kz)) + W * (Sz * pk(C, kz));
                double tt = T / det;
                if (tt > (seg == 0 ? 0.0 : eps) && tt < bt) { bt = tt; best = t; }
            }
        }
        if (!live) continue;
        if (best < 0) { live = false; continue; }
        const double *x = a.xyz + 9 * (size_t)best;
        double e1[3] = {x[3] - x[0], x[4] - x[1], x[5] - x[2]}, e2[3] = {x[6] - x[0], x[7] - x[1], x[8] - x[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int k = 0; k < 3; k++) n[k] /= nl;
        double dn = dir[0] * n[0] + dir[1] * n[1] + dir[2] * n[2];
        int side = dn < 0.0 ? 0 : 1;
        double sg = side ? -1.0 : 1.0;
        int mi = a.tmat[2 * best + side];
        if (mi < 0 || mi >= a.n_mats) {
            // a material index the caller left out of range: no read of mat; the
            // result becomes NaN so the caller sees it
            for (int k = 0; k < 6; k++) acc[k] += NAN;
            live = false;
            continue;
        }
        double rs = a.mat[2 * mi], rd = a.mat[2 * mi + 1];
        double c = -sg * dn, F[3], hp[3];
        for (int k = 0; k < 3; k++) {
            F[k] = w * ((1.0 - rs) * dir[k] - 2.0 * (rs * c + rd / 3.0) * sg * n[k]);
            hp[k] = o[k] + bt * dir[k];
        }
        double arm[3] = {hp[0] - a.c_ref[0], hp[1] - a.c_ref[1], hp[2] - a.c_ref[2]};
        acc[0] += F[0]; acc[1] += F[1]; acc[2] += F[2];
        acc[3] += arm[1] * F[2] - arm[2] * F[1];
        acc[4] += arm[2] * F[0] - arm[0] * F[2];
        acc[5] += arm[0] * F[1] - arm[1] * F[0];
        w *= rs;
        if (w == 0.0) { live = false; continue; }
        for (int k = 0; k < 3; k++) { dir[k] = dir[k] - 2.0 * dn * n[k]; o[k] = hp[k]; }
        skip = best;
    }
    // block sum in fixed order, one 8-double partial per block
    __shared__ double red[6][kNaThreads];
    for (int k = 0; k < 6; k++) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int h = kNaThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int k = 0; k < 6; k++) red[k][threadIdx.x] += red[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 8) scratch[8 + 8 * (size_t)blockIdx.x + threadIdx.x] = threadIdx.x < 6 ? red[threadIdx.x][0] : 0.0;
}

__global__ void __launch_bounds__(kNaThreads) k_na_reduce(NaArgs a, int nblocks, const double *scratch, double *force,
                                                          double *torque)
{
    __shared__ double red[6][kNaThreads];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 6; k++) acc[k] += scratch[8 + 8 * (size_t)b + k];
    for (int k = 0; k < 6; k++) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int h = kNaThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int k = 0; k < 6; k++) red[k][threadIdx.x] += red[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double Du = scratch[1] - scratch[0], Dv = scratch[3] - scratch[2];
        double sc = a.scale * Du * Dv / ((double)a.N * (double)a.N);
        for (int k = 0; k < 3; k++) { force[k] = red[k][0] * sc; torque[k] = red[3 + k][0] * sc; }
    }
}

// Device address of the scratch array per device.  Only a successful lookup
// is kept; a failed one is tried again on the next call.
constexpr int kNaMaxDevices = 64;
double *g_na_ptr[kNaMaxDevices];
std::mutex g_na_mu[kNaMaxDevices];

double *na_scratch(int dev)
{
    std::lock_guard<std::mutex> lk(g_na_mu[dev]);
    if (!g_na_ptr[dev]) {
        double *p = nullptr;
        if (cudaGetSymbolAddress((void **)&p, g_na_scratch) == cudaSuccess) g_na_ptr[dev] = p;
    }
    return g_na_ptr[dev];
}

}  // namespace
}  // namespace srp

using namespace srp;

extern "C" srp_status srp_eval_noalloc(const double *tri_xyz, const int32_t *tri_mat, int32_t n_tris,
                                       const double *mat, int32_t n_mats, const double sun_dir[3], double sun_dist_au,
                                       const double c_ref[3], int32_t N, int32_t bounces, double P0, double eps_rel,
                                       double *force, double *torque, void *cuda_stream)
{
    if (!tri_xyz || !tri_mat || !mat || !sun_dir || !c_ref || !force || !torque) return SRP_ERR_ARG;
    if (n_tris < 1 || n_tris > SRP_NOALLOC_MAX_TRIS || n_mats < 1 || n_mats > SRP_MAX_MATS) return SRP_ERR_ARG;
    if (N < 1 || N > SRP_NOALLOC_MAX_N || bounces < 0 || bounces > SRP_MAX_BOUNCES) return SRP_ERR_ARG;
    if (!(sun_dist_au > 0.0) || !(P0 >= 0.0) || !(eps_rel >= 0.0)) return SRP_ERR_ARG;
    double sn = sqrt(sun_dir[0] * sun_dir[0] + sun_dir[1] * sun_dir[1] + sun_dir[2] * sun_dir[2]);
    if (!(sn > 0.0)) return SRP_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return SRP_ERR_CUDA;
    double *scratch = na_scratch(dev);
    if (!scratch) return SRP_ERR_CUDA;
    NaArgs a{};
    a.xyz = tri_xyz; a.tmat = tri_mat; a.mat = mat;
    a.n_tris = n_tris; a.n_mats = n_mats; a.N = N; a.nseg = bounces + 1;
    double s[3] = {sun_dir[0] / sn, sun_dir[1] / sn, sun_dir[2] / sn};
    double d[3] = {-s[0], -s[1], -s[2]};
    double sg = copysign(1.0, d[2]), aa = -1.0 / (sg + d[2]), b = d[0] * d[1] * aa;
    a.u[0] = 1.0 + sg * d[0] * d[0] * aa; a.u[1] = sg * b; a.u[2] = -sg * d[0];
    a.v[0] = b; a.v[1] = sg + d[1] * d[1] * aa; a.v[2] = -d[1];
    for (int k = 0; k < 3; k++) { a.d[k] = d[k]; a.c_ref[k] = c_ref[k]; }
    a.eps_rel = eps_rel;
    a.scale = P0 / (sun_dist_au * sun_dist_au);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int nblocks = (int)(((size_t)N * N + kNaThreads - 1) / kNaThreads);
    // A launch error left pending by earlier, unrelated work on this thread is
    // cleared here so that it is not reported as this call's failure (an error
    // that poisons the context makes the launches below fail as well).
    (void)cudaGetLastError();
    k_na_window<<<1, kNaThreads, 0, st>>>(a, scratch);
    if (cudaPeekAtLastError() != cudaSuccess) return SRP_ERR_CUDA;
    k_na_trace<<<nblocks, kNaThreads, 0, st>>>(a, scratch);
    if (cudaPeekAtLastError() != cudaSuccess) return SRP_ERR_CUDA;
    k_na_reduce<<<1, kNaThreads, 0, st>>>(a, nblocks, scratch, force, torque);
    if (cudaPeekAtLastError() != cudaSuccess) return SRP_ERR_CUDA;
    return SRP_OK;
}
