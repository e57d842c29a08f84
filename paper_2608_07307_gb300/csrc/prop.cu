// prop.cu -- orbit propagation with the ray-traced SRP force in every stage
// (Sec. 3, Eqs. 1-3: y = (x, v), y' = (v, a_g + a_SRP), integrated with an
// explicit embedded Runge-Kutta 7(8) pair that evaluates the SRP acceleration
// several times per step).
//
// One step is a fixed sequence of kernels, captured once in a CUDA graph and
// relaunched: for each stage, k_prop_stage forms the stage state and the Sun
// direction in the body frame, the SRP evaluation pipeline runs for every
// trajectory, k_prop_accel forms the stage derivative; k_prop_control then
// accepts or rejects the step and picks the next step size.  All state lives
// on the device; the host only relaunches the graph and polls a done counter.
//
// Integrators: Fehlberg's 7(8) pair (13 stages, NASA TR R-287, 1968),
// propagating the 7th-order solution, error norm
// max_i |e_i| / (atol_i + rtol max(|y_i|, |y_new_i|)), next h = h clamp(0.9
// err^(-1/8), 0.2, 5); or classical RK4 with a fixed step.  Forces: central
// point mass, optional Earth J2 (z = pole) and the Sun as a third body from the
// low-precision solar coordinates of Montenbruck & Gill (Satellite Orbits,
// Sec. 3.3.2), SRP zero inside a cylindrical Earth shadow; attitude LVLH (body
// z to nadir, body y along minus the orbit normal) or a fixed quaternion.
#include <math.h>

#include "srp_internal.cuh"

namespace srp {

namespace {

constexpr double kMuEarth = 3.986004418e14;
constexpr double kREarth = 6378137.0;
constexpr double kJ2 = 1.08262668e-3;
constexpr double kMuSun = 1.32712440018e20;
constexpr double kAU = 1.495978707e11;
constexpr double kPi = 3.14159265358979323846;

// Fehlberg 7(8): nodes, stage weights (lower triangle), 7th / 8th order weights.
__constant__ double cC[13] = {0.0,       2.0 / 27.0, 1.0 / 9.0, 1.0 / 6.0, 5.0 / 12.0, 0.5, 5.0 / 6.0,
                              1.0 / 6.0, 2.0 / 3.0,  1.0 / 3.0, 1.0,       0.0,        1.0};
__constant__ double cA[13][12] = {
    {0},
    {2.0 / 27.0},
    {1.0 / 36.0, 1.0 / 12.0},
    {1.0 / 24.0, 0.0, 1.0 / 8.0},
    {5.0 / 12.0, 0.0, -25.0 / 16.0, 25.0 / 16.0},
    {1.0 / 20.0, 0.0, 0.0, 1.0 / 4.0, 1.0 / 5.0},
    {-25.0 / 108.0, 0.0, 0.0, 125.0 / 108.0, -65.0 / 27.0, 125.0 / 54.0},
    {31.0 / 300.0, 0.0, 0.0, 0.0, 61.0 / 225.0, -2.0 / 9.0, 13.0 / 900.0},
    {2.0, 0.0, 0.0, -53.0 / 6.0, 704.0 / 45.0, -107.0 / 9.0, 67.0 / 90.0, 3.0},
    {-91.0 / 108.0, 0.0, 0.0, 23.0 / 108.0, -976.0 / 135.0, 311.0 / 54.0, -19.0 / 60.0, 17.0 / 6.0, -1.0 / 12.0},
    {2383.0 / 4100.0, 0.0, 0.0, -341.0 / 164.0, 4496.0 / 1025.0, -301.0 / 82.0, 2133.0 / 4100.0, 45.0 / 82.0,
     45.0 / 164.0, 18.0 / 41.0},
    {3.0 / 205.0, 0.0, 0.0, 0.0, 0.0, -6.0 / 41.0, -3.0 / 205.0, -3.0 / 41.0, 3.0 / 41.0, 6.0 / 41.0, 0.0},
    {-1777.0 / 4100.0, 0.0, 0.0, -341.0 / 164.0, 4496.0 / 1025.0, -289.0 / 82.0, 2193.0 / 4100.0, 51.0 / 82.0,
     33.0 / 164.0, 12.0 / 41.0, 0.0, 1.0},
};
__constant__ double cB7[13] = {41.0 / 840.0, 0.0, 0.0, 0.0, 0.0, 34.0 / 105.0, 9.0 / 35.0, 9.0 / 35.0, 9.0 / 280.0,
                               9.0 / 280.0, 41.0 / 840.0, 0.0, 0.0};
__constant__ double cB8[13] = {0.0, 0.0, 0.0, 0.0, 0.0, 34.0 / 105.0, 9.0 / 35.0, 9.0 / 35.0, 9.0 / 280.0,
                               9.0 / 280.0, 0.0, 41.0 / 840.0, 41.0 / 840.0};
// classical RK4
__constant__ double cC4[4] = {0.0, 0.5, 0.5, 1.0};
__constant__ double cB4[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

__device__ void sun_pos(double mjd_tt, double *r)
{
    const double deg = kPi / 180.0;
    double T = (mjd_tt - 51544.5) / 36525.0;
    double M = fmod(357.5256 + 35999.049 * T, 360.0) * deg;
    double lam = 282.94 * deg + M + (6892.0 * sin(M) + 72.0 * sin(2.0 * M)) * (deg / 3600.0);
    double rr = 149.619e9 - 2.499e9 * cos(M) - 0.021e9 * cos(2.0 * M);
    double ce = cos(23.43929111 * deg), se = sin(23.43929111 * deg);
    r[0] = rr * cos(lam);
    r[1] = rr * sin(lam) * ce;
    r[2] = rr * sin(lam) * se;
}

// body -> inertial rotation, row-major
__device__ void body_to_inertial(const PropDev &P, const double *y, double *R)
{
    if (P.attitude == 1) {
        double w = P.q[0], x = P.q[1], yy = P.q[2], z = P.q[3];
        double qn = sqrt(w * w + x * x + yy * yy + z * z);
        w /= qn; x /= qn; yy /= qn; z /= qn;
        R[0] = 1.0 - 2.0 * (yy * yy + z * z); R[1] = 2.0 * (x * yy - w * z);       R[2] = 2.0 * (x * z + w * yy);
        R[3] = 2.0 * (x * yy + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z);   R[5] = 2.0 * (yy * z - w * x);
        R[6] = 2.0 * (x * z - w * yy);       R[7] = 2.0 * (yy * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + yy * yy);
        return;
    }
    double rn = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
    double h[3] = {y[1] * y[5] - y[2] * y[4], y[2] * y[3] - y[0] * y[5], y[0] * y[4] - y[1] * y[3]};
    double hn = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    double zb[3] = {-y[0] / rn, -y[1] / rn, -y[2] / rn};
    double yb[3] = {-h[0] / hn, -h[1] / hn, -h[2] / hn};
    double xb[3] = {yb[1] * zb[2] - yb[2] * zb[1], yb[2] * zb[0] - yb[0] * zb[2], yb[0] * zb[1] - yb[1] * zb[0]};
    for (int k = 0; k < 3; k++) { R[3 * k] = xb[k]; R[3 * k + 1] = yb[k]; R[3 * k + 2] = zb[k]; }
}

// Gravity of the configured bodies at (t, y).
__device__ void gravity(const PropDev &P, double t, const double *y, const double *rs, double *a)
{
    double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2], r = sqrt(r2);
    double mu = P.central == 1 ? kMuSun : kMuEarth;
    for (int k = 0; k < 3; k++) a[k] = -mu * y[k] / (r2 * r);
    if (P.central == 0 && P.j2) {
        double z2 = y[2] * y[2] / r2;
        double f = -1.5 * kJ2 * kMuEarth * kREarth * kREarth / (r2 * r2 * r);
        a[0] += f * y[0] * (1.0 - 5.0 * z2);
        a[1] += f * y[1] * (1.0 - 5.0 * z2);
        a[2] += f * y[2] * (3.0 - 5.0 * z2);
    }
    if (P.central == 0 && P.sun3) {
        double d[3] = {rs[0] - y[0], rs[1] - y[1], rs[2] - y[2]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double sn = sqrt(rs[0] * rs[0] + rs[1] * rs[1] + rs[2] * rs[2]);
        double d3 = dn * dn * dn, s3 = sn * sn * sn;
        for (int k = 0; k < 3; k++) a[k] += kMuSun * (d[k] / d3 - rs[k] / s3);
    }
}

__global__ void k_prop_init(PropState *S, int n, const double *y0, const double *t01, double h0, int *n_done)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PropState &X = S[i];
    for (int k = 0; k < 6; k++) X.y[k] = y0[6 * i + k];
    X.t = t01[2 * i];
    X.t1 = t01[2 * i + 1];
    X.h = h0;
    X.hs = h0;
    X.done = X.t1 <= X.t ? 1 : 0;
    X.status = 0;
    X.steps = X.rejects = X.evals = 0;
    X.nlog = 0;
    X.shadow = 0;
    for (int j = 0; j < 13; j++)
        for (int k = 0; k < 6; k++) X.k[j][k] = 0.0;
    if (X.done) atomicAdd(n_done, 1);
}

// Stage state, Sun direction (body frame) and distance for the SRP call.
__global__ void k_prop_stage(PropState *S, int n, PropDev P, int stage, double *sun_dir, double *sun_dist)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PropState &X = S[i];
    const int rk4 = P.method == 1;
    double h = X.h;
    if (!X.done) {
        if (P.n_replay > 0) {
            h = X.steps < P.n_replay ? P.h_replay[(size_t)i * P.n_replay + X.steps] : 0.0;
        } else if (X.t + h >= X.t1) {
            h = X.t1 - X.t;  // land exactly on t1
        }
        X.hs = h;
    }
    double c = rk4 ? cC4[stage] : cC[stage];
    for (int k = 0; k < 6; k++) {
        double acc = 0.0;
        if (rk4) {
            if (stage > 0) acc = 0.5 * X.k[stage - 1][k] * (stage == 3 ? 2.0 : 1.0);
        } else {
            for (int j = 0; j < stage; j++) acc += cA[stage][j] * X.k[j][k];
        }
        X.ys[k] = X.y[k] + X.hs * acc;
    }
    X.ts = X.t + c * X.hs;
    // Sun direction and distance
    double rs[3] = {0.0, 0.0, 0.0}, sv[3];
    if (P.central == 0) sun_pos(P.epoch_mjd_tt + X.ts / 86400.0, rs);
    for (int k = 0; k < 3; k++) { X.rsun[k] = rs[k]; sv[k] = rs[k] - X.ys[k]; }
    double sd = sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
    for (int k = 0; k < 3; k++) sv[k] /= sd;
    // cylindrical Earth shadow
    X.shadow = 0;
    if (P.central == 0) {
        double rsn = sqrt(rs[0] * rs[0] + rs[1] * rs[1] + rs[2] * rs[2]);
        double e[3] = {rs[0] / rsn, rs[1] / rsn, rs[2] / rsn};
        double pr = X.ys[0] * e[0] + X.ys[1] * e[1] + X.ys[2] * e[2];
        double q[3] = {X.ys[0] - pr * e[0], X.ys[1] - pr * e[1], X.ys[2] - pr * e[2]};
        if (pr < 0.0 && sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) < kREarth) X.shadow = 1;
    }
    double R[9];
    body_to_inertial(P, X.ys, R);
    for (int k = 0; k < 9; k++) X.R[k] = R[k];
    for (int k = 0; k < 3; k++) sun_dir[3 * i + k] = R[k] * sv[0] + R[3 + k] * sv[1] + R[6 + k] * sv[2];
    // finished and shadowed trajectories skip their SRP evaluation (negative distance)
    sun_dist[i] = (X.done || X.shadow || !P.srp) ? -1.0 : sd / kAU;
}

__global__ void k_prop_accel(PropState *S, int n, PropDev P, int stage, const double *force)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PropState &X = S[i];
    double a[3];
    gravity(P, X.ts, X.ys, X.rsun, a);
    if (P.srp && !X.shadow) {
        const double *F = force + 3 * i;
        for (int k = 0; k < 3; k++) a[k] += (X.R[3 * k] * F[0] + X.R[3 * k + 1] * F[1] + X.R[3 * k + 2] * F[2]) / P.mass;
    }
    for (int k = 0; k < 3; k++) { X.k[stage][k] = X.ys[3 + k]; X.k[stage][3 + k] = a[k]; }
    if (!X.done) X.evals++;
}

__global__ void k_prop_control(PropState *S, int n, PropDev P, int *n_done, double *h_log, int64_t h_cap)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PropState &X = S[i];
    if (X.done) return;
    const double h = X.hs;
    if (P.n_replay > 0) {
        // replay: take the given step, 7th-order solution, no error control
        for (int k = 0; k < 6; k++) {
            double s7 = 0.0;
            for (int j = 0; j < 13; j++) s7 += cB7[j] * X.k[j][k];
            X.y[k] = X.y[k] + h * s7;
        }
        X.t += h;
        if (h_log && X.nlog < h_cap) h_log[(size_t)i * h_cap + X.nlog] = h;
        X.nlog++;
        X.steps++;
        if (X.steps >= P.n_replay) { X.done = 1; atomicAdd(n_done, 1); }
        return;
    }
    const bool last = X.t + X.h >= X.t1;
    bool accept = true;
    double yn[6];
    double fac = 1.0;
    if (P.method == 1) {
        for (int k = 0; k < 6; k++) {
            double acc = 0.0;
            for (int j = 0; j < 4; j++) acc += cB4[j] * X.k[j][k];
            yn[k] = X.y[k] + h * acc;
        }
    } else {
        double e = 0.0;
        for (int k = 0; k < 6; k++) {
            double s7 = 0.0, s8 = 0.0;
            for (int j = 0; j < 13; j++) { s7 += cB7[j] * X.k[j][k]; s8 += cB8[j] * X.k[j][k]; }
            yn[k] = X.y[k] + h * s7;
            double sc = (k < 3 ? P.atol_pos : P.atol_vel) + P.rtol * fmax(fabs(X.y[k]), fabs(yn[k]));
            e = fmax(e, fabs(h * (s7 - s8)) / sc);
        }
        fac = e == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(e, -1.0 / 8.0)));
        accept = e <= 1.0;
    }
    if (accept) {
        for (int k = 0; k < 6; k++) X.y[k] = yn[k];
        // fixed steps snap onto t1 when they land within 1e-9 of a step of it
        X.t = (last || (P.method == 1 && X.t1 - (X.t + h) < 1e-9 * P.h0)) ? X.t1 : X.t + h;
        if (h_log && X.nlog < h_cap) h_log[(size_t)i * h_cap + X.nlog] = h;
        X.nlog++;
        X.steps++;
    } else {
        X.rejects++;
    }
    if (P.method == 0) {
        double hn = X.hs * fac;
        if (P.h_max > 0.0) hn = fmin(hn, P.h_max);
        if (X.t < X.t1 && hn < P.h_min) { X.status = SRP_ERR_STEP; X.done = 1; }
        X.h = hn;
    }
    if (X.t >= X.t1) X.done = 1;
    if (X.steps + X.rejects > P.max_steps && !X.done) { X.status = SRP_ERR_STEP; X.done = 1; }
    if (X.done) atomicAdd(n_done, 1);
}

}  // namespace

cudaError_t launch_prop_init(PropState *S, int n, const double *y0, const double *t01, double h0, int *n_done,
                             cudaStream_t st)
{
    k_prop_init<<<(n + 63) / 64, 64, 0, st>>>(S, n, y0, t01, h0, n_done);
    return cudaGetLastError();
}
cudaError_t launch_prop_stage(PropState *S, int n, const PropDev &P, int stage, double *sun_dir, double *sun_dist,
                              cudaStream_t st)
{
    k_prop_stage<<<(n + 63) / 64, 64, 0, st>>>(S, n, P, stage, sun_dir, sun_dist);
    return cudaGetLastError();
}
cudaError_t launch_prop_accel(PropState *S, int n, const PropDev &P, int stage, const double *force, cudaStream_t st)
{
    k_prop_accel<<<(n + 63) / 64, 64, 0, st>>>(S, n, P, stage, force);
    return cudaGetLastError();
}
cudaError_t launch_prop_control(PropState *S, int n, const PropDev &P, int *n_done, double *h_log, int64_t h_cap,
                                cudaStream_t st)
{
    k_prop_control<<<(n + 63) / 64, 64, 0, st>>>(S, n, P, n_done, h_log, h_cap);
    return cudaGetLastError();
}

}  // namespace srp
