/*
 * frozen_oracle.c -- the frozen-hit SRP function F_H of the FP64 oracle, the
 * object whose central finite differences are the reference gradient
 * (TEST INFRASTRUCTURE ONLY; same rules as srp_oracle.c).
 *
 * Ray-traced SRP (Sec. 4.3) is piecewise smooth: as a parameter moves, a ray
 * keeps hitting the same triangles until it crosses an edge.  F_H is the force
 * and torque with that combinatorial state held fixed:
 *   - every segment of every ray hits the triangle recorded for it at the base
 *     point, at the intersection of the ray with that triangle's plane (no
 *     inside test, no search, no self-hit threshold);
 *   - the window bounds are the projections of the four vertices that were
 *     extreme at the base point (argmin / argmax along u and v);
 *   - a segment is shaded only if it and every earlier segment of its ray were
 *     recorded as hits.
 * Everything else (tracking angle, clamp, posing, basis, pixel centres, force
 * law, specular direction, weights, pressure scaling) is the evaluation of
 * srp_oracle.c.  F_H is smooth in the optical coefficients, the joint angle
 * offsets, the (unnormalised) Sun direction and the Sun distance, and equals
 * the traced result at the base point.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "srp_oracle.h"

int orc_pose(const orc_mesh *m, const double s[3], int32_t track, const double *angles_in, double *angles_out,
             double *xyz_out);
void orc_onb(const double n[3], double b1[3], double b2[3]);

static double fdot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void fcross(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/*
 * The window's extreme vertices for Sun direction s (unit): ids[0..3] =
 * argmin u.x, argmax u.x, argmin v.x, argmax v.x over the posed vertices that
 * some triangle references; among equal projections the lowest vertex index.
 */
int orc_window_ids(const orc_mesh *m, const orc_params *p, const double s[3], int32_t ids[4])
{
    if (!m || !p || !s || !ids || m->n_tris <= 0) return ORC_ERR_ARG;
    int nv = m->n_verts;
    double *xyz = (double *)malloc(sizeof(double) * 3 * (size_t)nv);
    char *used = (char *)calloc((size_t)nv, 1);
    if (!xyz || !used) { free(xyz); free(used); return ORC_ERR_ARG; }
    int rc = orc_pose(m, s, p->track, p->angles, NULL, xyz);
    if (rc == ORC_OK) {
        double d[3] = {-s[0], -s[1], -s[2]}, u[3], v[3];
        orc_onb(d, u, v);
        for (int t = 0; t < m->n_tris; t++)
            for (int k = 0; k < 3; k++) used[m->tri[3 * t + k]] = 1;
        double best[4] = {INFINITY, -INFINITY, INFINITY, -INFINITY};
        for (int k = 0; k < 4; k++) ids[k] = -1;
        for (int i = 0; i < nv; i++) {
            if (!used[i]) continue;
            double pu = fdot(u, xyz + 3 * i), pv = fdot(v, xyz + 3 * i);
            if (pu < best[0]) { best[0] = pu; ids[0] = i; }
            if (pu > best[1]) { best[1] = pu; ids[1] = i; }
            if (pv < best[2]) { best[2] = pv; ids[2] = i; }
            if (pv > best[3]) { best[3] = pv; ids[3] = i; }
        }
    }
    free(xyz); free(used);
    return rc;
}

/*
 * F_H for rays [r0, r1).
 *   s_raw[3]  Sun direction, body frame, any positive length (normalised here)
 *   hits      [(r1 - r0)][bounces + 1] recorded triangle ids, -1 = none
 *   ids[4]    recorded extreme vertices (orc_window_ids)
 *   acc[6]    += unscaled force / torque sums, in ray order
 *   scale     out: P0 / dist_au^2 * pixel area
 * Per segment, with n the unit normal of the recorded triangle, the hit point
 * is x = o + t d with t = n.(A - o) / n.d, and the deposit is the force law of
 * srp_oracle.c: f = w [(1 - rho_s) d - 2 (rho_s c + rho_d / 3) n_f].
 */
int orc_eval_frozen(const orc_mesh *m, const orc_params *p, const double s_raw[3], int64_t r0, int64_t r1,
                    const int32_t *hits, const int32_t ids[4], double *acc, double *scale)
{
    if (!m || !p || !s_raw || !hits || !ids || !acc || p->N <= 0 || p->bounces < 0 || r0 < 0 || r1 < r0 ||
        r1 > (int64_t)p->N * p->N)
        return ORC_ERR_ARG;
    for (int k = 0; k < 4; k++)
        if (ids[k] < 0 || ids[k] >= m->n_verts) return ORC_ERR_ARG;
    double sn = sqrt(fdot(s_raw, s_raw));
    if (!(sn > 0.0)) return ORC_ERR_ARG;
    double s[3] = {s_raw[0] / sn, s_raw[1] / sn, s_raw[2] / sn};
    double *xyz = (double *)malloc(sizeof(double) * 3 * (size_t)(m->n_verts > 0 ? m->n_verts : 1));
    if (!xyz) return ORC_ERR_ARG;
    int rc = orc_pose(m, s, p->track, p->angles, NULL, xyz);
    if (rc != ORC_OK) { free(xyz); return rc; }
    double d0[3] = {-s[0], -s[1], -s[2]}, u[3], v[3];
    orc_onb(d0, u, v);
    double umin = fdot(u, xyz + 3 * ids[0]), umax = fdot(u, xyz + 3 * ids[1]);
    double vmin = fdot(v, xyz + 3 * ids[2]), vmax = fdot(v, xyz + 3 * ids[3]);
    int N = p->N, nseg = p->bounces + 1;
    if (scale) *scale = p->P0 / (p->dist_au * p->dist_au) * (umax - umin) * (vmax - vmin) / ((double)N * (double)N);
    for (int64_t r = r0; r < r1; r++) {
        const int32_t *hr = hits + (r - r0) * nseg;
        int64_t i = r / N, j = r % N;
        double uc = umin + ((double)i + 0.5) * (umax - umin) / N;
        double vc = vmin + ((double)j + 0.5) * (vmax - vmin) / N;
        double o[3], d[3], w = 1.0;
        for (int c = 0; c < 3; c++) { o[c] = uc * u[c] + vc * v[c]; d[c] = d0[c]; }
        for (int k = 0; k < nseg; k++) {
            int32_t h = hr[k];
            if (h < 0 || h >= m->n_tris) break;
            const int32_t *f = m->tri + 3 * h;
            const double *A = xyz + 3 * f[0], *B = xyz + 3 * f[1], *C = xyz + 3 * f[2];
            double e1[3], e2[3], n[3], nf[3], x[3], arm[3], F[3], Tq[3], ao[3];
            for (int c = 0; c < 3; c++) { e1[c] = B[c] - A[c]; e2[c] = C[c] - A[c]; ao[c] = A[c] - o[c]; }
            fcross(e1, e2, n);
            double nl = sqrt(fdot(n, n));
            for (int c = 0; c < 3; c++) n[c] /= nl;
            double dn = fdot(d, n);
            double t = fdot(n, ao) / dn;
            for (int c = 0; c < 3; c++) x[c] = o[c] + t * d[c];
            int side = dn < 0.0 ? 0 : 1;
            for (int c = 0; c < 3; c++) nf[c] = side ? -n[c] : n[c];
            int mi = m->tri_mat[2 * h + side];
            double rs = m->mat[2 * mi], rd = m->mat[2 * mi + 1];
            double cs = -fdot(nf, d);
            for (int c = 0; c < 3; c++) F[c] = w * ((1.0 - rs) * d[c] - 2.0 * (rs * cs + rd / 3.0) * nf[c]);
            for (int c = 0; c < 3; c++) arm[c] = x[c] - m->c_ref[c];
            fcross(arm, F, Tq);
            for (int c = 0; c < 3; c++) { acc[c] += F[c]; acc[3 + c] += Tq[c]; }
            w *= rs;
            if (k + 1 >= nseg) break;
            for (int c = 0; c < 3; c++) { d[c] = d[c] - 2.0 * dn * n[c]; o[c] = x[c]; }
        }
    }
    free(xyz);
    return ORC_OK;
}
