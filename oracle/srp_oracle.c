/*
 * srp_oracle.c -- double-precision reference ("oracle") for ray-traced solar
 * radiation pressure (SRP) on an articulated triangle-mesh spacecraft.
 *
 * TEST INFRASTRUCTURE ONLY.  It is loaded by tests/, by __graft_entry__.smoke()
 * and by bench.py's CPU-baseline and reference legs.  The library in
 * paper_2608_07307_gb300/ never includes, links or calls anything here, and
 * this file shares no code, header or constant table with it.
 *
 * Plain, slow and single-threaded on purpose: every ray is tested against
 * every triangle (no acceleration structure), everything is FP64, sums run in
 * ray order.  A caller that wants more cores shards the ray range over
 * processes and adds the partial sums in a fixed order.
 *
 * What it computes, by paper section:
 *   Sec. 1      ray tracing on a triangle mesh gives self-shadowing and
 *               multiple reflections.
 *   Sec. 4.3    one ray per pixel of a discretised image plane; secondary rays
 *               are iterated; all pixel contributions are aggregated into one
 *               force.
 *   Sec. 6.1    the image plane is an N x N projection window; the number of
 *               secondary reflection levels is a parameter.
 *   Sec. 4.4.1  the spacecraft is a rooted tree of rigid parts; a rotation at a
 *               joint moves the whole subtree; joints carry pivot, axis and
 *               admissible interval.
 *   Sec. 4.4.2  for each movable joint: take the subtree, find its panel
 *               normal, rotate so that normal is as close as possible to the
 *               Sun direction, clamp to the limits, transform the subtree.
 * Readings where the paper is silent (it prints no force law, window, basis,
 * tie rule or self-hit rule):
 *   - force law per hit: absorbed + specular + Lambertian-diffuse momentum
 *     transfer of a flat facet (the law of the Cannonball / N-plate models the
 *     paper compares against, Sec. 1), with diffusely reflected light leaving
 *     the body and specular light traced as a secondary ray;
 *   - window: tight bounds of the projections of all posed vertices on an
 *     orthonormal basis (u, v) of the plane normal to the ray direction d = -s,
 *     built with the branchless construction of Duff et al. (JCGT 2017);
 *     pixel centres; ray origins 1 m in front of the nearest vertex;
 *   - hits are two-sided; the nearest t > eps wins; equal t goes to the lowest
 *     triangle id; a secondary ray never hits the triangle it left;
 *     edges count as inside.
 *   - tracking angle: theta = atan2(b . s', n . s') with n the rest panel
 *     normal made orthogonal to the axis a, b = a x n, s' the Sun direction in
 *     the parent part's frame; theta = 0 when both are zero; then clamp.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "srp_oracle.h"

/* Per-evaluation geometry shared by all rays of one Sun direction. */
typedef struct {
    const orc_mesh *m;
    const double *xyz;       /* posed vertices                                  */
    double d[3], u[3], v[3]; /* ray direction and image-plane basis             */
    double umin, umax, vmin, vmax, wmin, wmax;
    double L, eps;
    int32_t N, bounces;
    int32_t n_diffuse;       /* diffuse secondary rays per hit                  */
    uint64_t seed;           /* their sample stream                             */
} orc_scene;

/* ---------------------------------------------------------------- vectors */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static void sub3(const double *a, const double *b, double *c) { c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2]; }
static void matvec(const double *R, const double *x, double *y)
{
    for (int i = 0; i < 3; i++) y[i] = R[3 * i] * x[0] + R[3 * i + 1] * x[1] + R[3 * i + 2] * x[2];
}
static void mattvec(const double *R, const double *x, double *y)
{
    for (int i = 0; i < 3; i++) y[i] = R[i] * x[0] + R[3 + i] * x[1] + R[6 + i] * x[2];
}
static void matmul(const double *A, const double *B, double *C)
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

/* Rotation by angle th about unit axis a (Rodrigues' formula), row-major. */
void orc_rotation(const double a[3], double th, double R[9])
{
    double c = cos(th), s = sin(th), k = 1.0 - c;
    R[0] = c + k * a[0] * a[0];        R[1] = k * a[0] * a[1] - s * a[2]; R[2] = k * a[0] * a[2] + s * a[1];
    R[3] = k * a[1] * a[0] + s * a[2]; R[4] = c + k * a[1] * a[1];        R[5] = k * a[1] * a[2] - s * a[0];
    R[6] = k * a[2] * a[0] - s * a[1]; R[7] = k * a[2] * a[1] + s * a[0]; R[8] = c + k * a[2] * a[2];
}

/* Orthonormal basis (b1, b2) completing unit vector n: the branchless
 * construction of Duff, Burgess, Christensen, Hery, Kensler, Liani, Villemin,
 * "Building an Orthonormal Basis, Revisited", JCGT 6(1), 2017. */
void orc_onb(const double n[3], double b1[3], double b2[3])
{
    double sign = copysign(1.0, n[2]);
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sign * n[0] * n[0] * a; b1[1] = sign * b; b1[2] = -sign * n[0];
    b2[0] = b; b2[1] = sign + n[1] * n[1] * a; b2[2] = -n[1];
}

/* ------------------------------------------------------------ Sec. 4.4 pose */
/*
 * Joint angles and posed vertices for Sun direction s (body frame, unit).
 * Sec. 4.4.1: parts form a rooted tree; the transform of a part is its
 * parent's transform composed with its own joint rotation about its pivot, so
 * a joint moves its whole subtree.  Sec. 4.4.2: for a movable joint the angle
 * brings the panel normal as close as possible to s (step 3), then is clamped
 * to the joint's interval (step 4); the transform is applied to every vertex of
 * the subtree (step 5).  A commanded angle (track == 0) is clamped the same way;
 * track == 2 adds angles_in[p] to the tracking angle before the clamp.
 * Returns ORC_ERR_MESH when a vertex is shared by two parts or the part order
 * is not topological.
 */
int orc_pose(const orc_mesh *m, const double s[3], int32_t track, const double *angles_in, double *angles_out,
             double *xyz_out)
{
    int np = m->n_parts;
    double *M = (double *)malloc(sizeof(double) * 9 * (size_t)np);
    double *T = (double *)malloc(sizeof(double) * 3 * (size_t)np);
    int32_t *vpart = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m->n_verts > 0 ? m->n_verts : 1));
    if (!M || !T || !vpart) { free(M); free(T); free(vpart); return ORC_ERR_ARG; }
    int rc = ORC_OK;
    for (int p = 0; p < np; p++) {
        double th = 0.0;
        const double *a = m->axis + 3 * p;
        int q = m->parent[p];
        if (q >= p || (p == 0 && q != -1) || (p > 0 && q < 0)) { rc = ORC_ERR_MESH; break; }
        int movable = (p > 0) && (a[0] != 0.0 || a[1] != 0.0 || a[2] != 0.0);
        if (movable) {
            if (track) {
                double sl[3], n[3], b[3];
                mattvec(M + 9 * q, s, sl); /* Sun in the parent's current frame */
                const double *n0 = m->normal0 + 3 * p;
                double na = dot3(n0, a);
                for (int k = 0; k < 3; k++) n[k] = n0[k] - na * a[k];
                cross3(a, n, b);
                double x = dot3(n, sl), y = dot3(b, sl);
                th = (x == 0.0 && y == 0.0) ? 0.0 : atan2(y, x);
                if (track == 2 && angles_in) th += angles_in[p]; /* offset from the tracking angle */
            } else {
                th = angles_in ? angles_in[p] : 0.0;
            }
            double lo = m->limits[2 * p], hi = m->limits[2 * p + 1];
            if (th < lo) th = lo;
            if (th > hi) th = hi;
        }
        if (angles_out) angles_out[p] = th;
        if (p == 0) {
            for (int k = 0; k < 9; k++) M[k] = (k % 4 == 0) ? 1.0 : 0.0;
            T[0] = T[1] = T[2] = 0.0;
            continue;
        }
        double R[9], Rp[3], tmp[3];
        if (movable) orc_rotation(a, th, R);
        else for (int k = 0; k < 9; k++) R[k] = (k % 4 == 0) ? 1.0 : 0.0;
        matmul(M + 9 * q, R, M + 9 * p);
        const double *pv = m->pivot + 3 * p;
        matvec(R, pv, Rp);
        sub3(pv, Rp, tmp);               /* x -> pivot + R (x - pivot) = R x + (pivot - R pivot) */
        matvec(M + 9 * q, tmp, T + 3 * p);
        for (int k = 0; k < 3; k++) T[3 * p + k] += T[3 * q + k];
    }
    if (rc == ORC_OK && xyz_out) {
        for (int i = 0; i < m->n_verts; i++) vpart[i] = -1;
        for (int t = 0; t < m->n_tris && rc == ORC_OK; t++)
            for (int k = 0; k < 3; k++) {
                int vi = m->tri[3 * t + k], pp = m->tri_part[t];
                if (vi < 0 || vi >= m->n_verts || pp < 0 || pp >= np) { rc = ORC_ERR_MESH; break; }
                if (vpart[vi] >= 0 && vpart[vi] != pp) { rc = ORC_ERR_MESH; break; }
                vpart[vi] = pp;
            }
        for (int i = 0; i < m->n_verts && rc == ORC_OK; i++) {
            int pp = vpart[i] < 0 ? 0 : vpart[i];
            double y[3];
            matvec(M + 9 * pp, m->xyz + 3 * i, y);
            for (int k = 0; k < 3; k++) xyz_out[3 * i + k] = y[k] + T[3 * pp + k];
        }
    }
    free(M); free(T); free(vpart);
    return rc;
}

/* ------------------------------------------------ Sec. 4.3 / 6.1 the window */
/* Build the per-direction scene: d = -s, basis (u, v), window bounds over every
 * vertex referenced by a triangle, window diagonal L and self-hit threshold. */
static int scene_setup(orc_scene *sc, const orc_mesh *m, const double *xyz, const double s[3], int32_t N,
                       int32_t bounces, double eps_rel)
{
    sc->m = m; sc->xyz = xyz; sc->N = N; sc->bounces = bounces;
    sc->n_diffuse = 0; sc->seed = 0;
    for (int k = 0; k < 3; k++) sc->d[k] = -s[k];
    orc_onb(sc->d, sc->u, sc->v);
    sc->umin = sc->vmin = sc->wmin = INFINITY;
    sc->umax = sc->vmax = sc->wmax = -INFINITY;
    for (int t = 0; t < m->n_tris; t++)
        for (int k = 0; k < 3; k++) {
            const double *x = xyz + 3 * m->tri[3 * t + k];
            double pu = dot3(sc->u, x), pv = dot3(sc->v, x), pw = dot3(sc->d, x);
            if (pu < sc->umin) sc->umin = pu;
            if (pu > sc->umax) sc->umax = pu;
            if (pv < sc->vmin) sc->vmin = pv;
            if (pv > sc->vmax) sc->vmax = pv;
            if (pw < sc->wmin) sc->wmin = pw;
            if (pw > sc->wmax) sc->wmax = pw;
        }
    if (m->n_tris == 0) { sc->umin = sc->umax = sc->vmin = sc->vmax = sc->wmin = sc->wmax = 0.0; }
    double du = sc->umax - sc->umin, dv = sc->vmax - sc->vmin, dw = sc->wmax - sc->wmin;
    sc->L = sqrt(du * du + dv * dv + dw * dw);
    sc->eps = eps_rel * sc->L;
    return ORC_OK;
}

/* Origin of primary ray r: pixel (i, j) = (r / N, r % N), centre of its cell. */
static void ray_origin(const orc_scene *sc, int64_t r, double o[3])
{
    int64_t i = r / sc->N, j = r % sc->N;
    double uc = sc->umin + ((double)i + 0.5) * (sc->umax - sc->umin) / sc->N;
    double vc = sc->vmin + ((double)j + 0.5) * (sc->vmax - sc->vmin) / sc->N;
    double w0 = sc->wmin - ORC_STANDOFF;
    for (int k = 0; k < 3; k++) o[k] = uc * sc->u[k] + vc * sc->v[k] + w0 * sc->d[k];
}

/* Two-sided Moller-Trumbore ray/triangle test (Moller & Trumbore, JGT 1997),
 * edges inclusive.  Returns 1 and the ray parameter when the line hits. */
static int mt_test(const double *o, const double *d, const double *v0, const double *v1, const double *v2, double *t)
{
    double e1[3], e2[3], p[3], q[3], sv[3];
    sub3(v1, v0, e1); sub3(v2, v0, e2);
    cross3(d, e2, p);
    double det = dot3(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    sub3(o, v0, sv);
    double bu = dot3(sv, p) * inv;
    if (bu < 0.0 || bu > 1.0) return 0;
    cross3(sv, e1, q);
    double bv = dot3(d, q) * inv;
    if (bv < 0.0 || bu + bv > 1.0) return 0;
    *t = dot3(e2, q) * inv;
    return 1;
}

/* Nearest hit along (o, d) over every triangle except `skip`: t > eps, ties to
 * the lowest id (triangles are visited in id order and only a strictly
 * smaller t replaces the current best). */
static int32_t nearest_hit(const orc_scene *sc, const double *o, const double *d, int32_t skip, double *tbest)
{
    const orc_mesh *m = sc->m;
    int32_t best = -1;
    double bt = INFINITY;
    for (int32_t t = 0; t < m->n_tris; t++) {
        if (t == skip) continue;
        const int32_t *f = m->tri + 3 * t;
        double tt;
        if (!mt_test(o, d, sc->xyz + 3 * f[0], sc->xyz + 3 * f[1], sc->xyz + 3 * f[2], &tt)) continue;
        if (tt > sc->eps && tt < bt) { bt = tt; best = t; }
    }
    *tbest = bt;
    return best;
}

/* Distance from the origin of the plane to segment (a, b) in that plane. */
static double seg_dist2d(const double *a, const double *b)
{
    double ex = b[0] - a[0], ey = b[1] - a[1];
    double ll = ex * ex + ey * ey, h = 0.0;
    if (ll > 0.0) {
        h = -(a[0] * ex + a[1] * ey) / ll;
        if (h < 0.0) h = 0.0;
        if (h > 1.0) h = 1.0;
    }
    double px = a[0] + h * ex, py = a[1] + h * ey;
    return sqrt(px * px + py * py);
}

/*
 * Edge proximity of one ray segment (test classification only, not part of the
 * SRP definition): the smallest distance, measured in the plane normal to the
 * ray, from the ray to the boundary of any triangle the ray reaches no later
 * than its hit (plus tol).  Zero when another triangle ties the hit in t within
 * tol, or a containing triangle sits within tol of the self-hit threshold.
 */
static double edge_distance(const orc_scene *sc, const double *o, const double *d, int32_t skip, int32_t hit,
                            double thit, double tol)
{
    const orc_mesh *m = sc->m;
    double b1[3], b2[3];
    orc_onb(d, b1, b2);
    double best = INFINITY;
    for (int32_t t = 0; t < m->n_tris; t++) {
        if (t == skip) continue;
        const int32_t *f = m->tri + 3 * t;
        const double *v0 = sc->xyz + 3 * f[0], *v1 = sc->xyz + 3 * f[1], *v2 = sc->xyz + 3 * f[2];
        double e1[3], e2[3], n[3], w[3];
        sub3(v1, v0, e1); sub3(v2, v0, e2); cross3(e1, e2, n);
        double nn = sqrt(dot3(n, n)), den = dot3(n, d);
        int relevant;
        double tp = 0.0;
        if (fabs(den) <= 1e-12 * nn) {
            relevant = 1;
        } else {
            sub3(v0, o, w);
            tp = dot3(n, w) / den;
            relevant = tp > sc->eps - tol && (hit < 0 || tp <= thit + tol);
        }
        if (!relevant) continue;
        double P[3][2];
        const double *vs[3] = {v0, v1, v2};
        for (int k = 0; k < 3; k++) {
            double r[3];
            sub3(vs[k], o, r);
            P[k][0] = dot3(r, b1);
            P[k][1] = dot3(r, b2);
        }
        double dist = seg_dist2d(P[0], P[1]);
        double d2 = seg_dist2d(P[1], P[2]);
        double d3 = seg_dist2d(P[2], P[0]);
        if (d2 < dist) dist = d2;
        if (d3 < dist) dist = d3;
        if (dist < best) best = dist;
        double tt;
        if (t != hit && mt_test(o, d, v0, v1, v2, &tt)) {
            if ((hit >= 0 && fabs(tt - thit) <= tol) || fabs(tt - sc->eps) <= tol) best = 0.0;
        }
    }
    return best;
}

/* ---------------------------------------------- diffuse secondary rays */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output number c (from 0) of
 * the sequence seeded with `seed`: the state after c + 1 increments of the
 * golden-ratio constant, mixed. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Diffuse sample q of segment k of primary ray r (nseg segments, K samples):
 * two uniforms in [0, 1) from outputs 2c and 2c + 1, c = (r nseg + k) K + q
 * (top 53 bits), then a cosine-weighted direction about the unit normal nf
 * (Malley's method: a uniform point of the unit disc lifted to the
 * hemisphere), in the basis of Duff et al. around nf. */
void orc_diffuse_dir(uint64_t seed, uint64_t c, const double nf[3], double w[3])
{
    double u1 = (double)(orc_splitmix64(seed, 2 * c) >> 11) * 0x1.0p-53;
    double u2 = (double)(orc_splitmix64(seed, 2 * c + 1) >> 11) * 0x1.0p-53;
    double rr = sqrt(u1), ph = 2.0 * 3.14159265358979323846 * u2;
    double lx = rr * cos(ph), ly = rr * sin(ph), lz = sqrt(1.0 - u1);
    double t1[3], t2[3];
    orc_onb(nf, t1, t2);
    for (int k = 0; k < 3; k++) w[k] = lx * t1[k] + ly * t2[k] + lz * nf[k];
}

/*
 * Diffuse secondaries of one hit (reading of Sec. 6.1's diffuse rays): the
 * light the facet reflects diffusely, w rho_d, leaves as K rays of weight
 * w rho_d / K, cosine-distributed about nf, from the hit point x; each is
 * traced once (never the emitting triangle, t > eps) and deposits at its hit
 * the full per-hit law along its own direction; it spawns nothing further.
 * The emitter's own recoil stays the analytic 2/3 rho_d term of the law.
 */
static void diffuse_hits(const orc_scene *sc, int64_t r, int k, const double x[3], const double nf[3], int32_t src,
                         double wd, double *acc)
{
    const orc_mesh *m = sc->m;
    int nseg = sc->bounces + 1;
    for (int q = 0; q < sc->n_diffuse; q++) {
        uint64_t c = ((uint64_t)r * (uint64_t)nseg + (uint64_t)k) * (uint64_t)sc->n_diffuse + (uint64_t)q;
        double w[3], th;
        orc_diffuse_dir(sc->seed, c, nf, w);
        int32_t h = nearest_hit(sc, x, w, src, &th);
        if (h < 0) continue;
        const int32_t *f = m->tri + 3 * h;
        const double *v0 = sc->xyz + 3 * f[0], *v1 = sc->xyz + 3 * f[1], *v2 = sc->xyz + 3 * f[2];
        double e1[3], e2[3], n[3], nf2[3], x2[3], arm[3], F[3], Tq[3];
        sub3(v1, v0, e1); sub3(v2, v0, e2); cross3(e1, e2, n);
        double nl = sqrt(dot3(n, n));
        for (int c3 = 0; c3 < 3; c3++) n[c3] /= nl;
        int side = dot3(w, n) < 0.0 ? 0 : 1;
        for (int c3 = 0; c3 < 3; c3++) nf2[c3] = side ? -n[c3] : n[c3];
        int mi = m->tri_mat[2 * h + side];
        double rs = m->mat[2 * mi], rd = m->mat[2 * mi + 1];
        double cs = -dot3(nf2, w);
        for (int c3 = 0; c3 < 3; c3++) F[c3] = wd * ((1.0 - rs) * w[c3] - 2.0 * (rs * cs + rd / 3.0) * nf2[c3]);
        for (int c3 = 0; c3 < 3; c3++) x2[c3] = x[c3] + th * w[c3];
        sub3(x2, m->c_ref, arm);
        cross3(arm, F, Tq);
        for (int c3 = 0; c3 < 3; c3++) { acc[c3] += F[c3]; acc[3 + c3] += Tq[c3]; }
    }
}

/*
 * Trace primary ray r and its specular secondaries (Sec. 4.3: secondary rays
 * are handled iteratively).  Per hit, with n_f the unit facet normal turned
 * towards the incoming ray, c = -n_f . d and (rho_s, rho_d) of the side hit,
 * the momentum deposited per unit beam weight is
 *     f = w [ (1 - rho_s) d  -  2 (rho_s c + rho_d / 3) n_f ],
 * (absorbed + Lambertian incidence along d; specular and diffuse reflection
 * recoil along -n_f), torque (x_hit - c_ref) x f.  The specular beam leaves
 * with direction d - 2 (d . n) n and weight w rho_s; segment k+1 is traced
 * only if segment k hit, k < bounces, and the new weight is non-zero.  With
 * n_diffuse > 0, every hit of a segment k < bounces also emits its diffuse
 * secondaries (diffuse_hits) before the specular ray goes on.
 * acc[0..5] += (f, tau) summed over the segments (not yet scaled by P dA).
 */
static void trace_ray(const orc_scene *sc, int64_t r, double *acc, int32_t *hits, double *edge, int64_t *nhit)
{
    const orc_mesh *m = sc->m;
    double o[3], d[3], w = 1.0;
    int32_t src = -1;
    ray_origin(sc, r, o);
    for (int k = 0; k < 3; k++) d[k] = sc->d[k];
    int nseg = sc->bounces + 1;
    for (int k = 0; k < nseg; k++) { if (hits) hits[k] = -1; if (edge) edge[k] = INFINITY; }
    for (int k = 0; k < nseg; k++) {
        double th;
        int32_t h = nearest_hit(sc, o, d, src, &th);
        if (hits) hits[k] = h;
        if (edge) edge[k] = edge_distance(sc, o, d, src, h, th, 1e-6 * sc->L);
        if (h < 0) break;
        if (nhit) nhit[k]++;
        const int32_t *f = m->tri + 3 * h;
        const double *v0 = sc->xyz + 3 * f[0], *v1 = sc->xyz + 3 * f[1], *v2 = sc->xyz + 3 * f[2];
        double e1[3], e2[3], n[3], nf[3], x[3], arm[3], F[3], Tq[3];
        sub3(v1, v0, e1); sub3(v2, v0, e2); cross3(e1, e2, n);
        double nl = sqrt(dot3(n, n));
        for (int c = 0; c < 3; c++) n[c] /= nl;
        int side = dot3(d, n) < 0.0 ? 0 : 1; /* 0: front face hit */
        for (int c = 0; c < 3; c++) nf[c] = side ? -n[c] : n[c];
        int mi = m->tri_mat[2 * h + side];
        double rs = m->mat[2 * mi], rd = m->mat[2 * mi + 1];
        double cs = -dot3(nf, d);
        for (int c = 0; c < 3; c++) F[c] = w * ((1.0 - rs) * d[c] - 2.0 * (rs * cs + rd / 3.0) * nf[c]);
        for (int c = 0; c < 3; c++) x[c] = o[c] + th * d[c];
        sub3(x, m->c_ref, arm);
        cross3(arm, F, Tq);
        for (int c = 0; c < 3; c++) { acc[c] += F[c]; acc[3 + c] += Tq[c]; }
        if (k + 1 < nseg && sc->n_diffuse > 0 && rd > 0.0) diffuse_hits(sc, r, k, x, nf, h, w * rd / sc->n_diffuse, acc);
        w *= rs;
        if (k + 1 >= nseg || w == 0.0) break;
        double dn = dot3(d, n);
        for (int c = 0; c < 3; c++) { d[c] = d[c] - 2.0 * dn * n[c]; o[c] = x[c]; }
        src = h;
    }
}

/*
 * Evaluate rays [r0, r1) of one Sun direction.
 *   s[3]      Sun direction, body frame, unit (photons travel along -s).
 *   acc[6]    += unscaled force / torque sums of those rays, in ray order.
 *   scale[1]  out: P0 / dist_au^2 * dA, the factor turning acc into N and N m.
 *   win[8]    out (may be NULL): umin umax vmin vmax wmin wmax L eps.
 *   angles    out (may be NULL): joint angles [n_parts].
 *   hits      out (may be NULL): [(r1-r0)][bounces+1] triangle id, -1 = none.
 *   edge      out (may be NULL): [(r1-r0)][bounces+1] edge proximity, metres.
 *   nhit      out (may be NULL): [bounces+1] += number of hits per segment.
 */
int orc_eval_range(const orc_mesh *m, const orc_params *p, const double s[3], int64_t r0, int64_t r1, double *acc,
                   double *scale, double *win, double *angles, int32_t *hits, double *edge, int64_t *nhit)
{
    if (!m || !p || !s || !acc || p->N <= 0 || p->bounces < 0 || r0 < 0 || r1 < r0 ||
        r1 > (int64_t)p->N * p->N || p->dist_au <= 0.0)
        return ORC_ERR_ARG;
    double *xyz = (double *)malloc(sizeof(double) * 3 * (size_t)(m->n_verts > 0 ? m->n_verts : 1));
    if (!xyz) return ORC_ERR_ARG;
    int rc = orc_pose(m, s, p->track, p->angles, angles, xyz);
    if (rc != ORC_OK) { free(xyz); return rc; }
    orc_scene sc;
    scene_setup(&sc, m, xyz, s, p->N, p->bounces, p->eps_rel);
    sc.n_diffuse = p->n_diffuse > 0 ? p->n_diffuse : 0;
    sc.seed = p->diffuse_seed;
    if (win) {
        win[0] = sc.umin; win[1] = sc.umax; win[2] = sc.vmin; win[3] = sc.vmax;
        win[4] = sc.wmin; win[5] = sc.wmax; win[6] = sc.L; win[7] = sc.eps;
    }
    double dA = (sc.umax - sc.umin) * (sc.vmax - sc.vmin) / ((double)p->N * (double)p->N);
    if (scale) *scale = p->P0 / (p->dist_au * p->dist_au) * dA;
    int nseg = p->bounces + 1;
    for (int64_t r = r0; r < r1; r++) {
        trace_ray(&sc, r, acc, hits ? hits + (r - r0) * nseg : NULL, edge ? edge + (r - r0) * nseg : NULL, nhit);
    }
    free(xyz);
    return ORC_OK;
}

/* Trace an explicit list of primary rays (for sampled checks at full size). */
int orc_eval_rays(const orc_mesh *m, const orc_params *p, const double s[3], int64_t n, const int64_t *rays,
                  double *contrib /*[n][6] unscaled*/, int32_t *hits, double *edge)
{
    if (!m || !p || !s || n < 0 || p->N <= 0 || p->bounces < 0 || p->dist_au <= 0.0) return ORC_ERR_ARG;
    double *xyz = (double *)malloc(sizeof(double) * 3 * (size_t)(m->n_verts > 0 ? m->n_verts : 1));
    if (!xyz) return ORC_ERR_ARG;
    int rc = orc_pose(m, s, p->track, p->angles, NULL, xyz);
    if (rc != ORC_OK) { free(xyz); return rc; }
    orc_scene sc;
    scene_setup(&sc, m, xyz, s, p->N, p->bounces, p->eps_rel);
    sc.n_diffuse = p->n_diffuse > 0 ? p->n_diffuse : 0;
    sc.seed = p->diffuse_seed;
    int nseg = p->bounces + 1;
    for (int64_t q = 0; q < n; q++) {
        if (rays[q] < 0 || rays[q] >= (int64_t)p->N * p->N) { free(xyz); return ORC_ERR_ARG; }
        double a[6] = {0, 0, 0, 0, 0, 0};
        trace_ray(&sc, rays[q], a, hits ? hits + q * nseg : NULL, edge ? edge + q * nseg : NULL, NULL);
        if (contrib) memcpy(contrib + 6 * q, a, sizeof a);
    }
    free(xyz);
    return ORC_OK;
}
