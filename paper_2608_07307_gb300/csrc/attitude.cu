// attitude.cu -- SRP acceleration in the inertial frame (Sec. 3, Eq. 1: the
// perturbing acceleration of the equations of motion) for evaluations given as
// an inertial Sun direction and a body -> inertial attitude quaternion per
// evaluation.
//
// The ray tracer works in the body frame.  Around it:
//   att_in    s_body = R(q)^T s_in               (FP64, one thread per evaluation)
//   att_out   a = R(q) F_body / m                (the acceleration of the state)
//   att_grad  the reverse of both: with the body-frame gradient g_sbody of the
//             evaluation (the frozen-hit adjoint) and the cotangent g_a of the
//             acceleration,
//                 g_sun = R g_sbody,
//                 dL/dR = g_a F_body^T / m + s_in g_sbody^T,
//             and the quaternion cotangent through quat_matrix_vjp.
// q is normalised before use; its cotangent is that of q as given.
#include <math.h>

#include "srp_internal.cuh"

namespace srp {
namespace {

__global__ void k_att_in(int n, const double *q, const double *s_in, double *s_body, const double *g_in,
                         double *g_body, double inv_mass)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double R[9];
    quat_matrix(q + 4 * (size_t)k, R);
    const double *s = s_in + 3 * (size_t)k;
    for (int c = 0; c < 3; c++) s_body[3 * (size_t)k + c] = R[c] * s[0] + R[3 + c] * s[1] + R[6 + c] * s[2];
    if (g_in) {
        const double *g = g_in + 3 * (size_t)k;
        for (int c = 0; c < 3; c++)
            g_body[3 * (size_t)k + c] = (R[c] * g[0] + R[3 + c] * g[1] + R[6 + c] * g[2]) * inv_mass;
    }
}

__global__ void k_att_out(int n, const double *q, const double *f_body, double *acc, double inv_mass)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double R[9];
    quat_matrix(q + 4 * (size_t)k, R);
    const double *f = f_body + 3 * (size_t)k;
    double a[3];
    for (int r = 0; r < 3; r++) a[r] = (R[3 * r] * f[0] + R[3 * r + 1] * f[1] + R[3 * r + 2] * f[2]) * inv_mass;
    for (int r = 0; r < 3; r++) acc[3 * (size_t)k + r] = a[r];
}

__global__ void k_att_grad(int n, const double *q, const double *s_in, const double *f_body, const double *g_acc,
                           const double *g_sbody, double *g_sun, double *g_q, double inv_mass)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double *qk = q + 4 * (size_t)k;
    double R[9];
    quat_matrix(qk, R);
    const double *s = s_in + 3 * (size_t)k, *f = f_body + 3 * (size_t)k, *ga = g_acc + 3 * (size_t)k;
    const double *gb = g_sbody + 3 * (size_t)k;
    double Rb[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) Rb[3 * r + c] = ga[r] * f[c] * inv_mass + s[r] * gb[c];
    if (g_sun)
        for (int r = 0; r < 3; r++) g_sun[3 * (size_t)k + r] = R[3 * r] * gb[0] + R[3 * r + 1] * gb[1] + R[3 * r + 2] * gb[2];
    if (g_q) quat_matrix_vjp(qk, Rb, g_q + 4 * (size_t)k);
}

}  // namespace

cudaError_t launch_att_in(int n, const double *q, const double *s_in, double *s_body, const double *g_in,
                          double *g_body, double mass, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_att_in<<<(n + 127) / 128, 128, 0, st>>>(n, q, s_in, s_body, g_in, g_body, 1.0 / mass);
    return cudaGetLastError();
}

cudaError_t launch_att_out(int n, const double *q, const double *f_body, double *acc, double mass, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_att_out<<<(n + 127) / 128, 128, 0, st>>>(n, q, f_body, acc, 1.0 / mass);
    return cudaGetLastError();
}

cudaError_t launch_att_grad(int n, const double *q, const double *s_in, const double *f_body, const double *g_acc,
                            const double *g_sbody, double *g_sun, double *g_q, double mass, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_att_grad<<<(n + 127) / 128, 128, 0, st>>>(n, q, s_in, f_body, g_acc, g_sbody, g_sun, g_q, 1.0 / mass);
    return cudaGetLastError();
}

}  // namespace srp
