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
// k_prop_stage runs a warp per trajectory: at the first stage of a step, lanes
// compute the Sun positions of all stages (their times are fixed with the step
// size), lanes 0-5 form the stage state.  Without ray tracing between the
// stages (a SPAD table, read by spad_lookup in the acceleration, or SRP off)
// the whole step is one kernel, k_prop_step, built from the same parts.
//
// Integrators: Fehlberg's 7(8) pair (13 stages, NASA TR R-287, 1968),
// propagating the 7th-order solution, error norm
// max_i |e_i| / (atol_i + rtol max(|y_i|, |y_new_i|)), next h = h clamp(0.9
// err^(-1/8), 0.2, 5); or classical RK4 with a fixed step.  Forces: central
// point mass, optional Earth J2 (z = pole) and the Sun as a third body from the
// low-precision solar coordinates of Montenbruck & Gill (Satellite Orbits,
// Sec. 3.3.2), SRP zero inside a cylindrical Earth shadow; attitude: the LVLH
// frame (z to nadir, y along minus the orbit normal) turned by a constant
// quaternion, or a fixed inertial quaternion.
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
    // two FP64 sincos calls (slow on this GPU's FP64 pipe); the double angle by identity
    double sM, cM;
    sincos(M, &sM, &cM);
    const double s2M = 2.0 * sM * cM, c2M = (cM - sM) * (cM + sM);
    double lam = 282.94 * deg + M + (6892.0 * sM + 72.0 * s2M) * (deg / 3600.0);
    double rr = 149.619e9 - 2.499e9 * cM - 0.021e9 * c2M;
    const double ce = 0.9174820620768958, se = 0.3977771559141214;  // cos, sin of the obliquity 23.43929111 deg
    double sl, cl;
    sincos(lam, &sl, &cl);
    r[0] = rr * cl;
    r[1] = rr * sl * ce;
    r[2] = rr * sl * se;
}

// LVLH frame at y: columns x_b = y_b x z_b, y_b = -orbit normal, z_b = nadir
__device__ void lvlh_matrix(const double *y, double *L)
{
    const double irn = -1.0 / sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
    double h[3] = {y[1] * y[5] - y[2] * y[4], y[2] * y[3] - y[0] * y[5], y[0] * y[4] - y[1] * y[3]};
    const double ihn = -1.0 / sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    double zb[3] = {y[0] * irn, y[1] * irn, y[2] * irn};
    double yb[3] = {h[0] * ihn, h[1] * ihn, h[2] * ihn};
    double xb[3] = {yb[1] * zb[2] - yb[2] * zb[1], yb[2] * zb[0] - yb[0] * zb[2], yb[0] * zb[1] - yb[1] * zb[0]};
    for (int k = 0; k < 3; k++) { L[3 * k] = xb[k]; L[3 * k + 1] = yb[k]; L[3 * k + 2] = zb[k]; }
}

// body -> inertial rotation, row-major: Q (inertial attitude) or LVLH(y) Q
// (the LVLH frame turned by the constant quaternion whose rotation is Q)
__device__ void body_to_inertial(int attitude, const double *Q, const double *y, double *R)
{
    if (attitude == 1) {
        for (int k = 0; k < 9; k++) R[k] = Q[k];
        return;
    }
    double L[9];
    lvlh_matrix(y, L);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) R[3 * i + j] = L[3 * i] * Q[j] + L[3 * i + 1] * Q[3 + j] + L[3 * i + 2] * Q[6 + j];
}

// Gravity of the configured bodies at (t, y).
__device__ void gravity(const PropDev &P, int central, const double *y, const double *rs, double *a)
{
    double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2], r = sqrt(r2);
    double mu = central == 1 ? kMuSun : kMuEarth;
    const double ir3 = 1.0 / (r2 * r);
    for (int k = 0; k < 3; k++) a[k] = -mu * y[k] * ir3;
    if (central == 0 && P.j2) {
        const double ir2 = 1.0 / r2;
        double z2 = y[2] * y[2] * ir2;
        double f = -1.5 * kJ2 * kMuEarth * kREarth * kREarth * (ir3 * ir2);
        a[0] += f * y[0] * (1.0 - 5.0 * z2);
        a[1] += f * y[1] * (1.0 - 5.0 * z2);
        a[2] += f * y[2] * (3.0 - 5.0 * z2);
    }
    if (central == 0 && P.sun3) {
        double d[3] = {rs[0] - y[0], rs[1] - y[1], rs[2] - y[2]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double sn = sqrt(rs[0] * rs[0] + rs[1] * rs[1] + rs[2] * rs[2]);
        const double id3 = 1.0 / (dn * dn * dn), is3 = 1.0 / (sn * sn * sn);
        for (int k = 0; k < 3; k++) a[k] += kMuSun * (d[k] * id3 - rs[k] * is3);
    }
}

// cfg (null: P's values for every trajectory): [n][8] central, attitude, q[4], mass, unused
__global__ void k_prop_init(PropState *S, int n, const double *y0, const double *t01, PropDev P, const double *cfg,
                            int *n_done)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PropState &X = S[i];
    const double h0 = P.h0;
    if (cfg) {
        const double *c = cfg + 8 * (size_t)i;
        X.central = (int)c[0];
        X.attitude = (int)c[1];
        for (int k = 0; k < 4; k++) X.q[k] = c[2 + k];
        X.mass = c[6];
    } else {
        X.central = P.central;
        X.attitude = P.attitude;
        for (int k = 0; k < 4; k++) X.q[k] = P.q[k];
        X.mass = P.mass;
    }
    quat_matrix(X.q, X.Qm);
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

// Lane 0's part of a stage: time, Sun direction in the body frame and
// distance (negative to skip the SRP call), shadow, attitude.
__device__ __forceinline__ void stage_tail(PropState &X, int i, const PropDev &P, int stage, double *sun_dir,
                                           double *sun_dist)
{
    const int rk4 = P.method == 1;
    X.ts = X.t + (rk4 ? cC4[stage] : cC[stage]) * X.hs;
    // Sun direction and distance
    double rs[3] = {0.0, 0.0, 0.0}, sv[3];
    if (X.central == 0)
        for (int k = 0; k < 3; k++) rs[k] = X.rs_st[stage][k];
    for (int k = 0; k < 3; k++) { X.rsun[k] = rs[k]; sv[k] = rs[k] - X.ys[k]; }
    double sd = sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
    for (int k = 0; k < 3; k++) sv[k] /= sd;
    // cylindrical Earth shadow
    X.shadow = 0;
    if (X.central == 0) {
        const double irsn = 1.0 / sqrt(rs[0] * rs[0] + rs[1] * rs[1] + rs[2] * rs[2]);
        double e[3] = {rs[0] * irsn, rs[1] * irsn, rs[2] * irsn};
        double pr = X.ys[0] * e[0] + X.ys[1] * e[1] + X.ys[2] * e[2];
        double q[3] = {X.ys[0] - pr * e[0], X.ys[1] - pr * e[1], X.ys[2] - pr * e[2]};
        if (pr < 0.0 && q[0] * q[0] + q[1] * q[1] + q[2] * q[2] < kREarth * kREarth) X.shadow = 1;
    }
    double R[9];
    body_to_inertial(X.attitude, X.Qm, X.ys, R);
    for (int k = 0; k < 9; k++) X.R[k] = R[k];
    for (int k = 0; k < 3; k++) sun_dir[3 * i + k] = R[k] * sv[0] + R[3 + k] * sv[1] + R[6 + k] * sv[2];
    // finished and shadowed trajectories skip their SRP evaluation (negative distance)
    sun_dist[i] = (X.done || X.shadow || !P.srp) ? -1.0 : sd / kAU;
}

// Stage state, Sun direction (body frame) and distance for the SRP call; a
// warp per trajectory.  At the first stage of a step, once the step size is
// fixed, every stage time is known: lanes compute the Sun positions of all
// stages at once.  Lanes 0-5 form the six components of the stage state; lane
// 0 the rest.
__device__ __forceinline__ void stage_body(PropState &X, int i, const PropDev &P, int stage, int lane, double *sun_dir,
                                           double *sun_dist)
{
    const int rk4 = P.method == 1;
    if (stage == 0) {
        if (lane == 0 && !X.done) {
            double h = X.h;
            if (P.n_replay > 0) {
                h = X.steps < P.n_replay ? P.h_replay[(size_t)i * P.n_replay + X.steps] : 0.0;
            } else if (X.t + h >= X.t1) {
                h = X.t1 - X.t;  // land exactly on t1
            }
            X.hs = h;
        }
        __syncwarp();
        if (lane < (rk4 ? 4 : 13) && X.central == 0) {
            const double ts = X.t + (rk4 ? cC4[lane] : cC[lane]) * X.hs;
            double rs[3];
            sun_pos(P.epoch_mjd_tt + ts / 86400.0, rs);
            for (int k = 0; k < 3; k++) X.rs_st[lane][k] = rs[k];
        }
    }
    if (lane < 6) {
        const int k = lane;
        double acc = 0.0;
        if (rk4) {
            if (stage > 0) acc = 0.5 * X.k[stage - 1][k] * (stage == 3 ? 2.0 : 1.0);
        } else {
            for (int j = 0; j < stage; j++) acc += cA[stage][j] * X.k[j][k];
        }
        X.ys[k] = X.y[k] + X.hs * acc;
    }
    __syncwarp();
    if (lane != 0) return;
    stage_tail(X, i, P, stage, sun_dir, sun_dist);
}

__global__ void k_prop_stage(PropState *S, int n, PropDev P, int stage, double *sun_dir, double *sun_dist)
{
    pdl_enter();
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;  // whole warps (blocks are multiples of 32 threads)
    stage_body(S[i], i, P, stage, threadIdx.x & 31, sun_dir, sun_dist);
}

// Stage derivative: gravity plus the SRP force (traced, or the SPAD interpolant).
__device__ __forceinline__ void accel_body(PropState &X, int i, const PropDev &P, int stage, const double *force,
                                           const double *sun_dir, const double *sun_dist)
{
    double a[3];
    gravity(P, X.central, X.ys, X.rsun, a);
    if (P.srp && !X.shadow) {
        double Fs[6];
        const double *F = force + 3 * i;
        if (P.spad.table) {
            // SPAD interpolation (Sec. 4.2) at this stage's body-frame Sun direction
            spad_lookup(P.spad, sun_dir + 3 * i, sun_dist[i], Fs);
            F = Fs;
        }
        const double im = 1.0 / X.mass;
        for (int k = 0; k < 3; k++) a[k] += (X.R[3 * k] * F[0] + X.R[3 * k + 1] * F[1] + X.R[3 * k + 2] * F[2]) * im;
    }
    for (int k = 0; k < 3; k++) { X.k[stage][k] = X.ys[3 + k]; X.k[stage][3 + k] = a[k]; }
    if (!X.done) X.evals++;
}

__global__ void k_prop_accel(PropState *S, int n, PropDev P, int stage, const double *force, const double *sun_dir,
                             const double *sun_dist)
{
    pdl_enter();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    accel_body(S[i], i, P, stage, force, sun_dir, sun_dist);
}

// Step control: accept or reject, next step size, completion.
__device__ __forceinline__ void control_body(PropState &X, int i, const PropDev &P, int *n_done, double *h_log,
                                             int64_t h_cap)
{
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

__global__ void k_prop_control(PropState *S, int n, PropDev P, int *n_done, double *h_log, int64_t h_cap)
{
    pdl_enter();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    control_body(S[i], i, P, n_done, h_log, h_cap);
}

// The stage derivative of `stage` and, in the same launch, the state of the
// next stage; after the last stage, step control and the first stage of the
// next step (which the captured step then starts from).  A warp per trajectory.
__global__ void k_prop_next(PropState *S, int n, PropDev P, int stage, const double *force, double *sun_dir,
                            double *sun_dist, int *n_done, double *h_log, int64_t h_cap)
{
    pdl_enter();
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;  // whole warps
    PropState &X = S[i];
    const int nst = P.method == 1 ? 4 : 13;
    if (lane == 0) accel_body(X, i, P, stage, force, sun_dir, sun_dist);
    __syncwarp();
    if (stage + 1 < nst) {
        stage_body(X, i, P, stage + 1, lane, sun_dir, sun_dist);
        return;
    }
    if (lane == 0) control_body(X, i, P, n_done, h_log, h_cap);
    __syncwarp();
    stage_body(X, i, P, 0, lane, sun_dir, sun_dist);
}

// A whole step in one launch when no ray-traced evaluation sits between the
// stages (SPAD table or SRP off): the stage, acceleration and control parts of
// the kernels above, in their order, a warp per trajectory.
__global__ void k_prop_step(PropState *S, int n, PropDev P, double *sun_dir, double *sun_dist, int *n_done,
                            double *h_log, int64_t h_cap)
{
    pdl_enter();
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;  // whole warps
    PropState &X = S[i];
    const int nst = P.method == 1 ? 4 : 13;
    for (int stage = 0; stage < nst; stage++) {
        stage_body(X, i, P, stage, lane, sun_dir, sun_dist);
        __syncwarp();
        if (lane == 0) accel_body(X, i, P, stage, nullptr, sun_dir, sun_dist);
        __syncwarp();
    }
    if (lane == 0) control_body(X, i, P, n_done, h_log, h_cap);
}


// ------------------------------------------------------------------ adjoint
// Discrete adjoint of the RK4 step y' = y + h sum_i b_i k_i, k_i = f(t_i, y_i),
// y_i = y + h a_{i,i-1} k_{i-1}: with lam the cotangent of y',
//   kbar_i = h b_i lam + h a_{i+1,i} ybar_{i+1},   ybar_i = (df/dy_i)^T kbar_i,
//   lam_before = lam + sum_i ybar_i,
// and the SRP part of df/dy_i, d f / d(parameters) through the frozen-hit
// adjoint of the evaluation (adjoint.cu).  Stages run 3, 2, 1, 0.

__device__ inline void save_ckpt(const PropState &X, double *b)
{
    b[0] = X.t;
    for (int k = 0; k < 6; k++) b[1 + k] = X.y[k];
}

__global__ void k_prop_ckpt(PropState *S, int n, double *buf, int save, double h0)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PropState &X = S[i];
    double *b = buf + 7 * (size_t)i;
    if (save) {
        save_ckpt(X, b);
        return;
    }
    X.t = b[0];
    for (int k = 0; k < 6; k++) X.y[k] = b[1 + k];
    X.h = X.hs = h0;  // a fixed-step arc always proposes h0
    X.done = X.t >= X.t1 ? 1 : 0;
    X.status = 0;
}

__global__ void k_prop_record(const PropState *S, int n, const double *sun, const double *dist, const double *force,
                              StageRec *rec, double *rec_sun, double *rec_dist)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const PropState &X = S[i];
    StageRec &r = rec[i];
    for (int k = 0; k < 6; k++) r.ys[k] = X.ys[k];
    r.ts = X.ts;
    r.hs = X.hs;
    for (int k = 0; k < 9; k++) r.R[k] = X.R[k];
    for (int k = 0; k < 3; k++) r.rsun[k] = X.rsun[k];
    r.lit = dist[i] >= 0.0 ? 1 : 0;
    for (int k = 0; k < 3; k++) {
        r.F[k] = r.lit ? force[3 * i + k] : 0.0;
        rec_sun[3 * i + k] = sun[3 * i + k];
    }
    rec_dist[i] = dist[i];
}

// kbar of this stage, and the cotangent of the body-frame SRP force
__global__ void k_adj_prop_in(int n, PropDev P, int stage, const StageRec *rec, PropAdj *A, double *g_force)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const StageRec &r = rec[i];
    PropAdj &X = A[i];
    const double h = r.hs;
    const double anext = stage == 2 ? 1.0 : 0.5;  // a_{stage+1, stage}
    for (int k = 0; k < 6; k++)
        X.kbar[k] = h * cB4[stage] * X.lam[k] + (stage < 3 ? h * anext * X.ybar[stage + 1][k] : 0.0);
    const double *ab = X.kbar + 3;
    for (int k = 0; k < 3; k++)
        g_force[3 * i + k] = r.lit ? (r.R[k] * ab[0] + r.R[3 + k] * ab[1] + r.R[6 + k] * ab[2]) / P.mass : 0.0;
}

// (df/dy)^T kbar at this stage: gravity, SRP through the Sun direction,
// distance and attitude; attitude quaternion cotangent
__global__ void k_adj_prop_out(int n, PropDev P, int stage, const StageRec *rec, PropAdj *A, const double *g_sun,
                               const double *g_dist)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const StageRec &r = rec[i];
    PropAdj &X = A[i];
    const double *y = r.ys, *ab = X.kbar + 3;
    double rb[3] = {0, 0, 0}, vb[3] = {X.kbar[0], X.kbar[1], X.kbar[2]};  // x' = v
    // central body: J = -mu (I / r^3 - 3 r r^T / r^5), symmetric
    {
        double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2], rn = sqrt(r2);
        double mu = P.central == 1 ? kMuSun : kMuEarth;
        double ra = y[0] * ab[0] + y[1] * ab[1] + y[2] * ab[2];
        // one reciprocal instead of a division per term (GB300's FP64 divisions are long chains)
        const double ir3 = 1.0 / (r2 * rn), ir5 = ir3 / r2;
        for (int k = 0; k < 3; k++) rb[k] += -mu * (ab[k] * ir3 - 3.0 * y[k] * ra * ir5);
    }
    if (P.central == 0 && P.j2) {
        double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
        const double ir2 = 1.0 / r2;
        double z2 = y[2] * y[2] * ir2;
        double f = -1.5 * kJ2 * kMuEarth * kREarth * kREarth / (r2 * r2 * sqrt(r2));
        double g[3] = {y[0] * (1.0 - 5.0 * z2), y[1] * (1.0 - 5.0 * z2), y[2] * (3.0 - 5.0 * z2)};
        double fb = ab[0] * g[0] + ab[1] * g[1] + ab[2] * g[2];
        rb[0] += f * ab[0] * (1.0 - 5.0 * z2);
        rb[1] += f * ab[1] * (1.0 - 5.0 * z2);
        rb[2] += f * ab[2] * (3.0 - 5.0 * z2);
        double z2b = -5.0 * f * (ab[0] * y[0] + ab[1] * y[1] + ab[2] * y[2]);
        rb[2] += z2b * 2.0 * y[2] * ir2;
        double r2b = -z2b * y[2] * y[2] * (ir2 * ir2) + fb * (-2.5) * f * ir2;
        for (int k = 0; k < 3; k++) rb[k] += 2.0 * r2b * y[k];
    }
    if (P.central == 0 && P.sun3) {
        double d[3] = {r.rsun[0] - y[0], r.rsun[1] - y[1], r.rsun[2] - y[2]};
        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], dn = sqrt(d2);
        double da = d[0] * ab[0] + d[1] * ab[1] + d[2] * ab[2];
        const double id3 = 1.0 / (d2 * dn), id5 = id3 / d2;
        for (int k = 0; k < 3; k++) rb[k] += -kMuSun * (ab[k] * id3 - 3.0 * d[k] * da * id5);
    }
    if (r.lit) {
        // a_SRP = R F / m, s_body = R^T s_hat, s_hat = w / |w|, w = r_sun - r, dist = |w| / AU
        const double *R = r.R, *gs = g_sun + 3 * i;
        double Rb[9];
        const double im = 1.0 / P.mass;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) Rb[3 * a + b] = ab[a] * r.F[b] * im;
        double w[3] = {r.rsun[0] - y[0], r.rsun[1] - y[1], r.rsun[2] - y[2]};
        double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        const double iwn = 1.0 / wn;
        double sh[3] = {w[0] * iwn, w[1] * iwn, w[2] * iwn};
        double shb[3];
        for (int a = 0; a < 3; a++) {
            shb[a] = R[3 * a] * gs[0] + R[3 * a + 1] * gs[1] + R[3 * a + 2] * gs[2];
            for (int b = 0; b < 3; b++) Rb[3 * a + b] += sh[a] * gs[b];
        }
        double sd = shb[0] * sh[0] + shb[1] * sh[1] + shb[2] * sh[2];
        for (int k = 0; k < 3; k++) {
            double wb = (shb[k] - sd * sh[k]) * iwn + g_dist[i] * sh[k] * (1.0 / kAU);
            rb[k] -= wb;
        }
        // attitude: R = Q(q) or R = L(y) Q(q)
        double Q[9], L[9], Qb[9];
        quat_matrix(P.q, Q);
        if (P.attitude == 1) {
            for (int k = 0; k < 9; k++) Qb[k] = Rb[k];
        } else {
            lvlh_matrix(y, L);
            double Lb[9];
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    double x = 0.0, z = 0.0;
                    for (int c = 0; c < 3; c++) {
                        x += L[3 * c + a] * Rb[3 * c + b];  // Qb = L^T Rb
                        z += Rb[3 * a + c] * Q[3 * b + c];  // Lb = Rb Q^T
                    }
                    Qb[3 * a + b] = x;
                    Lb[3 * a + b] = z;
                }
            // L = [x_b y_b z_b]: x_b = y_b x z_b, y_b = -h / |h|, h = r x v, z_b = -r / |r|
            double yb[3] = {L[1], L[4], L[7]}, zb[3] = {L[2], L[5], L[8]};
            double xbb[3] = {Lb[0], Lb[3], Lb[6]}, ybb[3] = {Lb[1], Lb[4], Lb[7]}, zbb[3] = {Lb[2], Lb[5], Lb[8]};
            ybb[0] += zb[1] * xbb[2] - zb[2] * xbb[1];
            ybb[1] += zb[2] * xbb[0] - zb[0] * xbb[2];
            ybb[2] += zb[0] * xbb[1] - zb[1] * xbb[0];
            zbb[0] += xbb[1] * yb[2] - xbb[2] * yb[1];
            zbb[1] += xbb[2] * yb[0] - xbb[0] * yb[2];
            zbb[2] += xbb[0] * yb[1] - xbb[1] * yb[0];
            const double *v = y + 3;
            double hv[3] = {y[1] * v[2] - y[2] * v[1], y[2] * v[0] - y[0] * v[2], y[0] * v[1] - y[1] * v[0]};
            double hn = sqrt(hv[0] * hv[0] + hv[1] * hv[1] + hv[2] * hv[2]);
            const double ihn = 1.0 / hn;
            double hh[3] = {hv[0] * ihn, hv[1] * ihn, hv[2] * ihn};
            double yd = ybb[0] * hh[0] + ybb[1] * hh[1] + ybb[2] * hh[2];
            double hb[3];
            for (int k = 0; k < 3; k++) hb[k] = -(ybb[k] - yd * hh[k]) * ihn;
            rb[0] += v[1] * hb[2] - v[2] * hb[1];
            rb[1] += v[2] * hb[0] - v[0] * hb[2];
            rb[2] += v[0] * hb[1] - v[1] * hb[0];
            vb[0] += hb[1] * y[2] - hb[2] * y[1];
            vb[1] += hb[2] * y[0] - hb[0] * y[2];
            vb[2] += hb[0] * y[1] - hb[1] * y[0];
            double rn = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
            const double irn = 1.0 / rn;
            double rh[3] = {y[0] * irn, y[1] * irn, y[2] * irn};
            double zd = zbb[0] * rh[0] + zbb[1] * rh[1] + zbb[2] * rh[2];
            for (int k = 0; k < 3; k++) rb[k] += -(zbb[k] - zd * rh[k]) * irn;
        }
        // Q of the normalised quaternion, differentiated
        double g[4];
        quat_matrix_vjp(P.q, Qb, g);
        for (int k = 0; k < 4; k++) X.qbar[k] += g[k];
    }
    for (int k = 0; k < 3; k++) { X.ybar[stage][k] = rb[k]; X.ybar[stage][3 + k] = vb[k]; }
}

// attitude quaternion cotangent summed over the trajectories, in order
__global__ void k_adj_prop_qsum(int n, const PropAdj *A, double *out)
{
    if (threadIdx.x >= 4) return;
    double x = 0.0;
    for (int i = 0; i < n; i++) x += A[i].qbar[threadIdx.x];
    out[threadIdx.x] = x;
}

__global__ void k_adj_prop_step(int n, PropAdj *A)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PropAdj &X = A[i];
    for (int k = 0; k < 6; k++) X.lam[k] += X.ybar[0][k] + X.ybar[1][k] + X.ybar[2][k] + X.ybar[3][k];
}

}  // namespace

cudaError_t launch_prop_init(PropState *S, int n, const double *y0, const double *t01, const PropDev &P,
                             const double *cfg, int *n_done, cudaStream_t st)
{
    k_prop_init<<<(n + 63) / 64, 64, 0, st>>>(S, n, y0, t01, P, cfg, n_done);
    return cudaGetLastError();
}
cudaError_t launch_prop_stage(PropState *S, int n, const PropDev &P, int stage, double *sun_dir, double *sun_dist,
                              cudaStream_t st)
{
    return launch_chained(k_prop_stage, dim3((n + 3) / 4), dim3(128), 0, st, S, n, P, stage, sun_dir, sun_dist);  // a warp per trajectory
}
cudaError_t launch_prop_accel(PropState *S, int n, const PropDev &P, int stage, const double *force, cudaStream_t st,
                              const double *sun_dir, const double *sun_dist)
{
    return launch_chained(k_prop_accel, dim3((n + 63) / 64), dim3(64), 0, st, S, n, P, stage, force, sun_dir, sun_dist);
}
cudaError_t launch_prop_next(PropState *S, int n, const PropDev &P, int stage, const double *force, double *sun_dir,
                             double *sun_dist, int *n_done, double *h_log, int64_t h_cap, cudaStream_t st)
{
    return launch_chained(k_prop_next, dim3((n + 3) / 4), dim3(128), 0, st, S, n, P, stage, force, sun_dir, sun_dist,
                          n_done, h_log, h_cap);
}
cudaError_t launch_prop_step(PropState *S, int n, const PropDev &P, double *sun_dir, double *sun_dist, int *n_done,
                             double *h_log, int64_t h_cap, cudaStream_t st)
{
    return launch_chained(k_prop_step, dim3((n + 3) / 4), dim3(128), 0, st, S, n, P, sun_dir, sun_dist, n_done, h_log, h_cap);
}
cudaError_t launch_prop_control(PropState *S, int n, const PropDev &P, int *n_done, double *h_log, int64_t h_cap,
                                cudaStream_t st)
{
    return launch_chained(k_prop_control, dim3((n + 63) / 64), dim3(64), 0, st, S, n, P, n_done, h_log, h_cap);
}

cudaError_t launch_prop_ckpt(PropState *S, int n, double *buf, bool save, double h0, cudaStream_t st)
{
    k_prop_ckpt<<<(n + 63) / 64, 64, 0, st>>>(S, n, buf, save ? 1 : 0, h0);
    return cudaGetLastError();
}
cudaError_t launch_prop_record(const PropState *S, int n, const double *sun, const double *dist, const double *force,
                               StageRec *rec, double *rec_sun, double *rec_dist, cudaStream_t st)
{
    k_prop_record<<<(n + 63) / 64, 64, 0, st>>>(S, n, sun, dist, force, rec, rec_sun, rec_dist);
    return cudaGetLastError();
}
cudaError_t launch_adj_prop_in(int n, const PropDev &P, int stage, const StageRec *rec, PropAdj *A, double *g_force,
                               cudaStream_t st)
{
    k_adj_prop_in<<<(n + 63) / 64, 64, 0, st>>>(n, P, stage, rec, A, g_force);
    return cudaGetLastError();
}
cudaError_t launch_adj_prop_out(int n, const PropDev &P, int stage, const StageRec *rec, PropAdj *A,
                                const double *g_sun, const double *g_dist, cudaStream_t st)
{
    k_adj_prop_out<<<(n + 63) / 64, 64, 0, st>>>(n, P, stage, rec, A, g_sun, g_dist);
    return cudaGetLastError();
}
cudaError_t launch_adj_prop_qsum(int n, const PropAdj *A, double *out, cudaStream_t st)
{
    k_adj_prop_qsum<<<1, 32, 0, st>>>(n, A, out);
    return cudaGetLastError();
}
cudaError_t launch_adj_prop_step(int n, PropAdj *A, cudaStream_t st)
{
    k_adj_prop_step<<<(n + 63) / 64, 64, 0, st>>>(n, A);
    return cudaGetLastError();
}

}  // namespace srp
