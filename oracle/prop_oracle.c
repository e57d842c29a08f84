/*
 * prop_oracle.c -- double-precision reference orbit propagation with
 * ray-traced SRP (TEST INFRASTRUCTURE ONLY; see srp_oracle.c).
 *
 * Sec. 3, Eqs. 1-3: the state y = (x, v) obeys y' = (v, a_g + a_SRP); the
 * paper integrates it with an explicit embedded Runge-Kutta 7(8) scheme that
 * evaluates the SRP acceleration several times per step.
 * Readings (the paper names "RK78" and cites a 1980 embedded family, but
 * prints no tableau, tolerances or force constants):
 *   - the embedded pair is Fehlberg's 7(8) (13 stages, NASA TR R-287, 1968),
 *     propagating the 7th-order solution; error norm
 *       err = max_i |e_i| / (atol_i + rtol max(|y_i|, |y_new_i|)),
 *     step accepted when err <= 1, next h = h clamp(0.9 err^(-1/8), 0.2, 5);
 *   - classical RK4 for fixed-step arcs;
 *   - gravity: central body point mass; optional Earth J2 (z = pole) and Sun
 *     as a third body with the low-precision analytic solar coordinates of
 *     Montenbruck & Gill (Satellite Orbits, Sec. 3.3.2);
 *   - SRP: the force of srp_oracle.c for the Sun direction in the body frame
 *     (or the SPAD interpolant of spad_oracle.c when a table is given),
 *     rotated to inertial and divided by the mass; zero inside a cylindrical
 *     Earth shadow;
 *   - attitude: the LVLH frame (z to nadir, y along minus the orbit normal)
 *     turned by a constant quaternion q (body -> LVLH; identity by default),
 *     or a fixed inertial quaternion q (body -> inertial); q scalar first.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "srp_oracle.h"

#define MU_EARTH 3.986004418e14
#define R_EARTH 6378137.0
#define J2_EARTH 1.08262668e-3
#define MU_SUN 1.32712440018e20
#define AU 1.495978707e11
#define PI 3.14159265358979323846

typedef struct {
    int32_t central;     /* 0 Earth, 1 Sun                                      */
    int32_t j2, sun3;    /* Earth J2, Sun third body (Earth-centred only)       */
    int32_t srp;         /* include ray-traced SRP                              */
    int32_t attitude;    /* 0 LVLH, 1 fixed inertial quaternion                 */
    double q[4];         /* body -> inertial, scalar first                      */
    double epoch_mjd_tt; /* t = 0                                               */
    double mass;         /* kg                                                  */
    int32_t N, bounces;  /* SRP ray grid and specular levels                    */
    double P0, eps_rel;
    int32_t method;      /* 0 RKF7(8) adaptive, 1 RK4 fixed step h0            */
    double rtol, atol_pos, atol_vel, h0, h_min, h_max;
    int64_t max_steps;
    const double *spad_table; /* NULL: trace rays; else the SPAD table (spad_oracle.c) */
    int32_t spad_n_az, spad_n_el;
    double spad_az0, spad_el0, spad_d_el;
    int32_t track;            /* joint mode of every evaluation (Sec. 4.4.2): 1 Sun tracking,
                                 2 tracking + angles[] offsets, 0 commanded angles[] */
    const double *angles;     /* [n_parts] offsets (2) or commanded angles (0)  */
} orc_prop;

/* Fehlberg 7(8) coefficients (NASA TR R-287, Table X). */
static const double RK_C[13] = {0.0, 2.0 / 27, 1.0 / 9, 1.0 / 6, 5.0 / 12, 1.0 / 2, 5.0 / 6, 1.0 / 6, 2.0 / 3, 1.0 / 3,
                                1.0, 0.0, 1.0};
static const double RK_A[13][12] = {
    {0},
    {2.0 / 27},
    {1.0 / 36, 1.0 / 12},
    {1.0 / 24, 0, 1.0 / 8},
    {5.0 / 12, 0, -25.0 / 16, 25.0 / 16},
    {1.0 / 20, 0, 0, 1.0 / 4, 1.0 / 5},
    {-25.0 / 108, 0, 0, 125.0 / 108, -65.0 / 27, 125.0 / 54},
    {31.0 / 300, 0, 0, 0, 61.0 / 225, -2.0 / 9, 13.0 / 900},
    {2.0, 0, 0, -53.0 / 6, 704.0 / 45, -107.0 / 9, 67.0 / 90, 3.0},
    {-91.0 / 108, 0, 0, 23.0 / 108, -976.0 / 135, 311.0 / 54, -19.0 / 60, 17.0 / 6, -1.0 / 12},
    {2383.0 / 4100, 0, 0, -341.0 / 164, 4496.0 / 1025, -301.0 / 82, 2133.0 / 4100, 45.0 / 82, 45.0 / 164, 18.0 / 41},
    {3.0 / 205, 0, 0, 0, 0, -6.0 / 41, -3.0 / 205, -3.0 / 41, 3.0 / 41, 6.0 / 41, 0},
    {-1777.0 / 4100, 0, 0, -341.0 / 164, 4496.0 / 1025, -289.0 / 82, 2193.0 / 4100, 51.0 / 82, 33.0 / 164, 12.0 / 41,
     0, 1.0},
};
static const double RK_B7[13] = {41.0 / 840, 0, 0, 0, 0, 34.0 / 105, 9.0 / 35, 9.0 / 35, 9.0 / 280, 9.0 / 280,
                                 41.0 / 840, 0, 0};
static const double RK_B8[13] = {0, 0, 0, 0, 0, 34.0 / 105, 9.0 / 35, 9.0 / 35, 9.0 / 280, 9.0 / 280, 0, 41.0 / 840,
                                 41.0 / 840};

/* Export the tableau so tests can check it against the order conditions. */
void orc_rkf78_tableau(double *c, double *a, double *b7, double *b8)
{
    for (int i = 0; i < 13; i++) {
        c[i] = RK_C[i]; b7[i] = RK_B7[i]; b8[i] = RK_B8[i];
        for (int j = 0; j < 13; j++) a[13 * i + j] = (j < i) ? RK_A[i][j] : 0.0;
    }
}

/* Geocentric equatorial Sun position (m) at MJD (TT): Montenbruck & Gill,
 * Sec. 3.3.2, mean anomaly / ecliptic longitude series, obliquity 23.43929111 deg. */
void orc_sun_position(double mjd_tt, double r[3])
{
    const double deg = PI / 180.0;
    double T = (mjd_tt - 51544.5) / 36525.0;
    double M = fmod(357.5256 + 35999.049 * T, 360.0) * deg;
    double L = (282.9400 * deg) + M + (6892.0 * sin(M) + 72.0 * sin(2.0 * M)) / 3600.0 * deg;
    double dist = (149.619e9 - 2.499e9 * cos(M) - 0.021e9 * cos(2.0 * M));
    double eps = 23.43929111 * deg;
    r[0] = dist * cos(L);
    r[1] = dist * sin(L) * cos(eps);
    r[2] = dist * sin(L) * sin(eps);
}

/* Body -> inertial rotation (row-major) for state y at time t. */
void orc_attitude(const orc_prop *pp, const double y[6], double R[9])
{
    double Q[9];
    {
        double w = pp->q[0], x = pp->q[1], yy = pp->q[2], z = pp->q[3];
        double n = sqrt(w * w + x * x + yy * yy + z * z);
        w /= n; x /= n; yy /= n; z /= n;
        Q[0] = 1 - 2 * (yy * yy + z * z); Q[1] = 2 * (x * yy - w * z);     Q[2] = 2 * (x * z + w * yy);
        Q[3] = 2 * (x * yy + w * z);     Q[4] = 1 - 2 * (x * x + z * z);  Q[5] = 2 * (yy * z - w * x);
        Q[6] = 2 * (x * z - w * yy);     Q[7] = 2 * (yy * z + w * x);     Q[8] = 1 - 2 * (x * x + yy * yy);
    }
    if (pp->attitude == 1) {
        memcpy(R, Q, sizeof Q);
        return;
    }
    const double *r = y, *v = y + 3;
    double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double h[3] = {r[1] * v[2] - r[2] * v[1], r[2] * v[0] - r[0] * v[2], r[0] * v[1] - r[1] * v[0]};
    double hn = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    double zb[3], yb[3], xb[3];
    for (int k = 0; k < 3; k++) { zb[k] = -r[k] / rn; yb[k] = -h[k] / hn; }
    xb[0] = yb[1] * zb[2] - yb[2] * zb[1];
    xb[1] = yb[2] * zb[0] - yb[0] * zb[2];
    xb[2] = yb[0] * zb[1] - yb[1] * zb[0];
    double L[9];
    for (int k = 0; k < 3; k++) { L[3 * k] = xb[k]; L[3 * k + 1] = yb[k]; L[3 * k + 2] = zb[k]; }
    /* body -> LVLH -> inertial */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) R[3 * i + j] = L[3 * i] * Q[j] + L[3 * i + 1] * Q[3 + j] + L[3 * i + 2] * Q[6 + j];
}

/*
 * Acceleration a(t, y) = a_g + a_SRP (Eq. 1).  aux (may be NULL) receives
 * [0..2] Sun direction in the body frame, [3] Sun distance (AU), [4] shadow
 * flag, [5..7] SRP force in the body frame (N).
 */
/* Gravity of the configured bodies; rs receives the Sun position (Earth-centred). */
static void gravity(const orc_prop *pp, double t, const double *r, double a[3], double rs[3])
{
    double rn2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], rn = sqrt(rn2);
    double mu = pp->central == 1 ? MU_SUN : MU_EARTH;
    for (int k = 0; k < 3; k++) a[k] = -mu * r[k] / (rn2 * rn);
    rs[0] = rs[1] = rs[2] = 0.0;
    if (pp->central == 0 && (pp->sun3 || pp->srp)) orc_sun_position(pp->epoch_mjd_tt + t / 86400.0, rs);
    if (pp->central == 0 && pp->j2) {
        double z2 = r[2] * r[2] / rn2;
        double k = -1.5 * J2_EARTH * MU_EARTH * R_EARTH * R_EARTH / (rn2 * rn2 * rn);
        a[0] += k * r[0] * (1.0 - 5.0 * z2);
        a[1] += k * r[1] * (1.0 - 5.0 * z2);
        a[2] += k * r[2] * (3.0 - 5.0 * z2);
    }
    if (pp->central == 0 && pp->sun3) {
        double dr[3] = {rs[0] - r[0], rs[1] - r[1], rs[2] - r[2]};
        double d3 = pow(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2], 1.5);
        double s3 = pow(rs[0] * rs[0] + rs[1] * rs[1] + rs[2] * rs[2], 1.5);
        for (int k = 0; k < 3; k++) a[k] += MU_SUN * (dr[k] / d3 - rs[k] / s3);
    }
}

/* Sun direction (inertial, unit), distance (AU) and the shadow test. */
static int sun_geometry(const orc_prop *pp, const double *r, const double rs[3], double sv[3], double *dist_au)
{
    if (pp->central == 1) { for (int k = 0; k < 3; k++) sv[k] = -r[k]; }
    else { for (int k = 0; k < 3; k++) sv[k] = rs[k] - r[k]; }
    double sd = sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
    for (int k = 0; k < 3; k++) sv[k] /= sd;
    *dist_au = sd / AU;
    if (pp->central == 0) {
        /* cylindrical Earth shadow (Montenbruck & Gill, Sec. 3.4.2) */
        double rsn = sqrt(rs[0] * rs[0] + rs[1] * rs[1] + rs[2] * rs[2]);
        double e[3] = {rs[0] / rsn, rs[1] / rsn, rs[2] / rsn};
        double pr = r[0] * e[0] + r[1] * e[1] + r[2] * e[2];
        double perp[3] = {r[0] - pr * e[0], r[1] - pr * e[1], r[2] - pr * e[2]};
        if (pr < 0.0 && sqrt(perp[0] * perp[0] + perp[1] * perp[1] + perp[2] * perp[2]) < R_EARTH) return 1;
    }
    return 0;
}

int orc_accel(const orc_mesh *mesh, const orc_prop *pp, double t, const double y[6], double a[3], double *aux)
{
    const double *r = y;
    double rs[3];
    gravity(pp, t, r, a, rs);
    if (aux) memset(aux, 0, 8 * sizeof(double));
    if (!pp->srp) return 0;
    /* unit vector spacecraft -> Sun and distance */
    double sv[3], dist;
    if (sun_geometry(pp, r, rs, sv, &dist)) {
        if (aux) aux[4] = 1.0;
        return 0;
    }
    double R[9], sb[3];
    orc_attitude(pp, y, R);
    for (int k = 0; k < 3; k++) sb[k] = R[k] * sv[0] + R[3 + k] * sv[1] + R[6 + k] * sv[2];
    double Fb[3];
    if (pp->spad_table) {
        /* interpolated force (Sec. 4.2): the table replaces the ray tracer */
        double out[6];
        int rc = orc_spad_interp(pp->spad_n_az, pp->spad_n_el, pp->spad_az0, pp->spad_el0, pp->spad_d_el,
                                 pp->spad_table, sb, dist, out);
        if (rc) return rc;
        for (int k = 0; k < 3; k++) Fb[k] = out[k];
    } else {
        orc_params ep = {pp->N, pp->bounces, pp->P0, dist, pp->eps_rel, pp->track, pp->angles};
        double acc[6] = {0, 0, 0, 0, 0, 0}, scale = 0.0;
        int rc = orc_eval_range(mesh, &ep, sb, 0, (int64_t)pp->N * pp->N, acc, &scale, NULL, NULL, NULL, NULL, NULL);
        if (rc) return rc;
        for (int k = 0; k < 3; k++) Fb[k] = acc[k] * scale;
    }
    for (int k = 0; k < 3; k++) a[k] += (R[3 * k] * Fb[0] + R[3 * k + 1] * Fb[1] + R[3 * k + 2] * Fb[2]) / pp->mass;
    if (aux) { aux[0] = sb[0]; aux[1] = sb[1]; aux[2] = sb[2]; aux[3] = dist; aux[5] = Fb[0]; aux[6] = Fb[1]; aux[7] = Fb[2]; }
    return 0;
}

static int deriv(const orc_mesh *mesh, const orc_prop *pp, double t, const double y[6], double f[6], int64_t *evals)
{
    double a[3];
    int rc = orc_accel(mesh, pp, t, y, a, NULL);
    if (evals) (*evals)++;
    f[0] = y[3]; f[1] = y[4]; f[2] = y[5];
    f[3] = a[0]; f[4] = a[1]; f[5] = a[2];
    return rc;
}

/* One RKF7(8) step: y_new (7th order) and the embedded error estimate. */
static int rkf78_step(const orc_mesh *mesh, const orc_prop *pp, double t, const double y[6], double h, double yn[6],
                      double err[6], int64_t *evals)
{
    double k[13][6], ys[6];
    for (int s = 0; s < 13; s++) {
        for (int i = 0; i < 6; i++) {
            double acc = 0.0;
            for (int j = 0; j < s; j++) acc += RK_A[s][j] * k[j][i];
            ys[i] = y[i] + h * acc;
        }
        int rc = deriv(mesh, pp, t + RK_C[s] * h, ys, k[s], evals);
        if (rc) return rc;
    }
    for (int i = 0; i < 6; i++) {
        double s7 = 0.0, s8 = 0.0;
        for (int j = 0; j < 13; j++) { s7 += RK_B7[j] * k[j][i]; s8 += RK_B8[j] * k[j][i]; }
        yn[i] = y[i] + h * s7;
        err[i] = h * (s7 - s8);
    }
    return 0;
}

static int rk4_step(const orc_mesh *mesh, const orc_prop *pp, double t, const double y[6], double h, double yn[6],
                    int64_t *evals)
{
    double k1[6], k2[6], k3[6], k4[6], ys[6];
    int rc = deriv(mesh, pp, t, y, k1, evals);
    for (int i = 0; i < 6; i++) ys[i] = y[i] + 0.5 * h * k1[i];
    rc |= deriv(mesh, pp, t + 0.5 * h, ys, k2, evals);
    for (int i = 0; i < 6; i++) ys[i] = y[i] + 0.5 * h * k2[i];
    rc |= deriv(mesh, pp, t + 0.5 * h, ys, k3, evals);
    for (int i = 0; i < 6; i++) ys[i] = y[i] + h * k3[i];
    rc |= deriv(mesh, pp, t + h, ys, k4, evals);
    for (int i = 0; i < 6; i++) yn[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    return rc;
}

/*
 * Propagate y0 from t0 to t1 (seconds from the epoch).
 * stats[0..2] (may be NULL): accepted steps, rejected steps, acceleration evaluations.
 * h_log (may be NULL): accepted step sizes, up to h_cap entries.
 * h_replay (may be NULL): when given (RKF7(8) only), the step sizes are taken
 *   from it in order with no error control: a replay of another integrator's
 *   accepted steps.
 * Returns 0, -1 for bad arguments, -7 when max_steps or h_min is hit.
 */
int orc_propagate(const orc_mesh *mesh, const orc_prop *pp, double t0, double t1, const double y0[6], double y1[6],
                  int64_t *stats, double *h_log, int64_t h_cap, const double *h_replay, int64_t n_replay)
{
    if (!pp || !y0 || !y1 || t1 < t0) return -1;
    double y[6], yn[6], err[6];
    memcpy(y, y0, sizeof y);
    double t = t0;
    int64_t acc_steps = 0, rej = 0, evals = 0;
    int rc = 0;
    if (pp->method == 1) {
        while (t < t1 && rc == 0) {
            double h = pp->h0;
            if (t + h > t1) h = t1 - t;
            rc = rk4_step(mesh, pp, t, y, h, yn, &evals);
            memcpy(y, yn, sizeof y);
            t = (t + h > t1 || t1 - (t + h) < 1e-9 * pp->h0) ? t1 : t + h;
            if (h_log && acc_steps < h_cap) h_log[acc_steps] = h;
            acc_steps++;
            if (acc_steps > pp->max_steps) { rc = -7; break; }
        }
    } else if (h_replay) {
        for (int64_t s = 0; s < n_replay && rc == 0; s++) {
            double h = h_replay[s];
            rc = rkf78_step(mesh, pp, t, y, h, yn, err, &evals);
            memcpy(y, yn, sizeof y);
            t += h;
            acc_steps++;
        }
    } else {
        double h = pp->h0;
        while (t < t1 && rc == 0) {
            int last = 0;
            if (t + h >= t1) { h = t1 - t; last = 1; }
            rc = rkf78_step(mesh, pp, t, y, h, yn, err, &evals);
            if (rc) break;
            double e = 0.0;
            for (int i = 0; i < 6; i++) {
                double sc = (i < 3 ? pp->atol_pos : pp->atol_vel) + pp->rtol * fmax(fabs(y[i]), fabs(yn[i]));
                double q = fabs(err[i]) / sc;
                if (q > e) e = q;
            }
            double fac = e == 0.0 ? 5.0 : 0.9 * pow(e, -1.0 / 8.0);
            if (fac < 0.2) fac = 0.2;
            if (fac > 5.0) fac = 5.0;
            if (e <= 1.0) {
                memcpy(y, yn, sizeof y);
                t = last ? t1 : t + h;
                if (h_log && acc_steps < h_cap) h_log[acc_steps] = h;
                acc_steps++;
            } else {
                rej++;
            }
            if (t >= t1) break;
            h = h * fac;
            if (pp->h_max > 0.0 && h > pp->h_max) h = pp->h_max;
            if (h < pp->h_min || acc_steps + rej > pp->max_steps) { rc = -7; break; }
        }
    }
    memcpy(y1, y, sizeof y);
    if (stats) { stats[0] = acc_steps; stats[1] = rej; stats[2] = evals; }
    return rc;
}

/* ------------------------------------------------- frozen-hit RK4 arcs */
int orc_window_ids(const orc_mesh *m, const orc_params *p, const double s[3], int32_t ids[4]);
int orc_eval_frozen(const orc_mesh *m, const orc_params *p, const double s_raw[3], int64_t r0, int64_t r1,
                    const int32_t *hits, const int32_t ids[4], double *acc, double *scale);

/*
 * A fixed-step RK4 arc (the step loop of orc_propagate with method 1) whose
 * SRP evaluations are either traced and recorded (record = 1) or replaced by
 * the frozen-hit function F_H of frozen_oracle.c using those records
 * (record = 0).  Stage k = 4 * step + stage keeps:
 *   hits [k][N*N][bounces+1]  triangle ids, ids [k][4] window vertices,
 *   lit  [k]                  1 when SRP was evaluated (not shadowed, SRP on).
 * The frozen arc takes the lit flags from the record (the shadow boundary is
 * part of the frozen combinatorial state).  track / angles: joint mode of
 * every evaluation (1 tracking, 2 tracking + offsets, 0 commanded).
 * Returns 0, or -1 for bad arguments / a record too small (cap stages).
 */
int orc_rk4_arc(const orc_mesh *mesh, const orc_prop *pp, int32_t track, const double *angles, double t0, double t1,
                const double y0[6], int32_t record, int32_t *hits, int32_t *ids, int32_t *lit, int64_t cap,
                double y1[6], int64_t *n_steps)
{
    if (!pp || !y0 || !y1 || t1 < t0 || pp->method != 1 || !(pp->h0 > 0.0)) return -1;
    if (pp->srp && (!mesh || !hits || !ids || !lit)) return -1;
    if (pp->spad_table) return ORC_ERR_ARG; /* frozen-hit arcs trace rays; no SPAD table */
    const int64_t rays = (int64_t)pp->N * pp->N, nseg = pp->bounces + 1;
    double y[6], k[4][6], ys[6];
    memcpy(y, y0, sizeof y);
    double t = t0;
    int64_t step = 0;
    static const double C4[4] = {0.0, 0.5, 0.5, 1.0}, A4[4] = {0.0, 0.5, 0.5, 1.0};
    while (t < t1) {
        double h = pp->h0;
        if (t + h > t1) h = t1 - t;
        for (int sg = 0; sg < 4; sg++) {
            for (int i = 0; i < 6; i++) ys[i] = sg == 0 ? y[i] : y[i] + A4[sg] * h * k[sg - 1][i];
            double ts = t + C4[sg] * h, a[3], rs[3];
            gravity(pp, ts, ys, a, rs);
            if (pp->srp) {
                int64_t kk = 4 * step + sg;
                if (kk >= cap) return -1;
                double sv[3], dist;
                int shadow = sun_geometry(pp, ys, rs, sv, &dist);
                if (record) lit[kk] = !shadow;
                if (lit[kk]) {
                    double R[9], sb[3];
                    orc_attitude(pp, ys, R);
                    for (int c = 0; c < 3; c++) sb[c] = R[c] * sv[0] + R[3 + c] * sv[1] + R[6 + c] * sv[2];
                    orc_params ep = {pp->N, pp->bounces, pp->P0, dist, pp->eps_rel, track, angles};
                    double acc[6] = {0, 0, 0, 0, 0, 0}, scale = 0.0;
                    int32_t *hk = hits + kk * rays * nseg, *ik = ids + 4 * kk;
                    int rc;
                    if (record) {
                        rc = orc_eval_range(mesh, &ep, sb, 0, rays, acc, &scale, NULL, NULL, hk, NULL, NULL);
                        if (!rc) rc = orc_window_ids(mesh, &ep, sb, ik);
                    } else {
                        rc = orc_eval_frozen(mesh, &ep, sb, 0, rays, hk, ik, acc, &scale);
                    }
                    if (rc) return -1;
                    double Fb[3] = {acc[0] * scale, acc[1] * scale, acc[2] * scale};
                    for (int c = 0; c < 3; c++)
                        a[c] += (R[3 * c] * Fb[0] + R[3 * c + 1] * Fb[1] + R[3 * c + 2] * Fb[2]) / pp->mass;
                }
            }
            for (int i = 0; i < 3; i++) { k[sg][i] = ys[3 + i]; k[sg][3 + i] = a[i]; }
        }
        for (int i = 0; i < 6; i++) y[i] = y[i] + h / 6.0 * (k[0][i] + 2.0 * k[1][i] + 2.0 * k[2][i] + k[3][i]);
        t = (t + h > t1 || t1 - (t + h) < 1e-9 * pp->h0) ? t1 : t + h;
        step++;
    }
    memcpy(y1, y, sizeof y);
    if (n_steps) *n_steps = step;
    return 0;
}
