/*
 * spad_oracle.c -- double-precision reference of the SPAD interpolation model
 * (TEST INFRASTRUCTURE ONLY; see srp_oracle.c).
 *
 * Sec. 4.2 (interpolation-based SRP) and Sec. 6.1 (the two tables): instead of tracing rays in
 * every integrator stage, the SRP force is read from a table precomputed by
 * the ray tracer over a grid of Sun directions in the body frame (azimuth x
 * elevation), interpolated bilinearly.  The paper fixes the grid only by its
 * sample counts and first sample (20 azimuths x 10 elevations from -180 deg,
 * -90 deg; the shifted set from -175 deg, -85 deg), says the first set holds
 * samples at 0 deg elevation and the shifted one does not, and names the
 * scheme bilinear.  Readings:
 *   - azimuth az = atan2(s_y, s_x), elevation el = atan2(s_z, hypot(s_x, s_y));
 *     the grid direction of (az, el) is (cos el cos az, cos el sin az, sin el);
 *   - azimuth samples az_i = az0 + i 2 pi / n_az (periodic: the cell after
 *     the last sample wraps to the first);  elevation samples
 *     el_j = el0 + j d_el, j < n_el (the paper's sets: d_el = 180 deg / 10,
 *     the only spacing that both puts a sample at 0 deg from -90 deg and none
 *     from -85 deg);
 *   - outside [el_0, el_{n_el-1}] the elevation clamps to the edge row;
 *   - the table holds force (N) and torque (N m) at 1 AU, [n_el][n_az][6];
 *     an interpolated entry scales as (1 AU / r)^2 like the traced force.
 */
#include <math.h>
#include <stdint.h>

#include "srp_oracle.h"

#define PI 3.14159265358979323846

/* Grid direction of sample (i, j). */
int orc_spad_dir(int32_t n_az, double az0, double el0, double d_el, int32_t i, int32_t j, double s[3])
{
    if (n_az < 1) return ORC_ERR_ARG;
    double az = az0 + i * (2.0 * PI / n_az);
    double el = el0 + j * d_el;
    s[0] = cos(el) * cos(az);
    s[1] = cos(el) * sin(az);
    s[2] = sin(el);
    return ORC_OK;
}

/* Bilinear interpolation of the table at body-frame direction s (unit or
 * not; only its direction is used) and Sun distance dist_au (> 0; a negative
 * distance gives zeros).  out = [F (3), T (3)]. */
int orc_spad_interp(int32_t n_az, int32_t n_el, double az0, double el0, double d_el, const double *table,
                    const double s[3], double dist_au, double out[6])
{
    if (n_az < 1 || n_el < 1 || !(d_el > 0.0)) return ORC_ERR_ARG;
    for (int k = 0; k < 6; k++) out[k] = 0.0;
    if (dist_au < 0.0) return ORC_OK;
    double az = atan2(s[1], s[0]);
    double el = atan2(s[2], hypot(s[0], s[1]));
    /* azimuth cell: u in sample units from az0, periodic */
    double u = (az - az0) / (2.0 * PI / n_az);
    double iu = floor(u);
    double fa = u - iu;
    int64_t i0 = (int64_t)iu % n_az;
    if (i0 < 0) i0 += n_az;
    int64_t i1 = (i0 + 1) % n_az;
    /* elevation cell, clamped to the table's rows */
    double v = (el - el0) / d_el;
    int64_t j0, j1;
    double fe;
    if (n_el == 1 || v <= 0.0) { j0 = j1 = 0; fe = 0.0; }
    else if (v >= n_el - 1) { j0 = j1 = n_el - 1; fe = 0.0; }
    else { double jv = floor(v); j0 = (int64_t)jv; j1 = j0 + 1; fe = v - jv; }
    const double *t00 = table + 6 * (j0 * n_az + i0), *t01 = table + 6 * (j0 * n_az + i1);
    const double *t10 = table + 6 * (j1 * n_az + i0), *t11 = table + 6 * (j1 * n_az + i1);
    double sc = 1.0 / (dist_au * dist_au);
    for (int k = 0; k < 6; k++) {
        double lo = (1.0 - fa) * t00[k] + fa * t01[k];
        double hi = (1.0 - fa) * t10[k] + fa * t11[k];
        out[k] = ((1.0 - fe) * lo + fe * hi) * sc;
    }
    return ORC_OK;
}
