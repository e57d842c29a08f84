// SPAD interpolation model (Sec. 4.2, Sec. 6.1): the sample directions of a
// table and its bilinear interpolant at arbitrary body-frame directions.  The
// table itself is built by the evaluation pipeline (srp_spad_build) and read
// inside propagation by k_prop_accel through spad_lookup.
#include "srp_internal.cuh"

namespace srp {

// Sample (i, j) of the grid: direction (cos el cos az, cos el sin az, sin el),
// az = az0 + i 2 pi / n_az, el = el0 + j d_el; one thread per sample.
__global__ void k_spad_dirs(SpadDev g, double *dirs)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n_az * g.n_el) return;
    const int i = k % g.n_az, j = k / g.n_az;
    const double az = g.az0 + i * (6.283185307179586 / g.n_az);
    const double el = g.el0 + j * g.d_el;
    double sa, ca, se, ce;
    sincos(az, &sa, &ca);
    sincos(el, &se, &ce);
    dirs[3 * k] = ce * ca;
    dirs[3 * k + 1] = ce * sa;
    dirs[3 * k + 2] = se;
}

// The interpolant at n directions; dist null means 1 AU.
__global__ void k_spad_eval(SpadDev g, int n, const double *dirs, const double *dist, double *force, double *torque)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double s[3] = {dirs[3 * k], dirs[3 * k + 1], dirs[3 * k + 2]};
    double o[6];
    spad_lookup(g, s, dist ? dist[k] : 1.0, o);
    for (int c = 0; c < 3; c++) {
        force[3 * k + c] = o[c];
        torque[3 * k + c] = o[3 + c];
    }
}

cudaError_t launch_spad_dirs(const SpadDev &g, double *dirs, cudaStream_t st)
{
    const int n = g.n_az * g.n_el;
    k_spad_dirs<<<(n + 127) / 128, 128, 0, st>>>(g, dirs);
    return cudaGetLastError();
}

cudaError_t launch_spad_eval(const SpadDev &g, int n, const double *dirs, const double *dist, double *force,
                             double *torque, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_spad_eval<<<(n + 127) / 128, 128, 0, st>>>(g, n, dirs, dist, force, torque);
    return cudaGetLastError();
}

}  // namespace srp
