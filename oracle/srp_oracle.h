/*
 * srp_oracle.h -- types of the FP64 reference oracle (TEST INFRASTRUCTURE ONLY).
 * Shared by the oracle's own translation units; nothing outside oracle/ includes it.
 */
#ifndef SRP_ORACLE_H
#define SRP_ORACLE_H
#include <stdint.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_MESH (-2)

/* Distance (m) between the ray origins' plane and the nearest vertex. */
#define ORC_STANDOFF 1.0

typedef struct {
    int32_t n_verts;
    const double *xyz;       /* [n_verts][3] rest pose, body frame, metres      */
    int32_t n_tris;
    const int32_t *tri;      /* [n_tris][3], counter-clockwise seen from front  */
    const int32_t *tri_part; /* [n_tris] rigid part of each triangle            */
    const int32_t *tri_mat;  /* [n_tris][2] material of the front, back side    */
    int32_t n_mats;
    const double *mat;       /* [n_mats][2] rho_s, rho_d (rho_a = 1 - both)     */
    int32_t n_parts;
    const int32_t *parent;   /* [n_parts]; -1 for the root; parent index < own  */
    const double *pivot;     /* [n_parts][3] joint pivot, rest body frame       */
    const double *axis;      /* [n_parts][3] unit joint axis; zero = rigid link */
    const double *limits;    /* [n_parts][2] admissible interval lo, hi (rad)   */
    const double *normal0;   /* [n_parts][3] rest front normal of the panel     */
    double c_ref[3];         /* torque reference point                          */
} orc_mesh;

typedef struct {
    int32_t N;               /* rays per side of the projection window          */
    int32_t bounces;         /* levels of specular secondary rays               */
    double P0;               /* radiation pressure at 1 AU, N/m^2               */
    double dist_au;          /* Sun distance, AU (pressure scales as 1/r^2)     */
    double eps_rel;          /* self-hit threshold, relative to window diagonal */
    int32_t track;           /* 1: Sun tracking; 0: angles[]; 2: tracking + angles[] */
    const double *angles;    /* [n_parts] commanded angles (0) or offsets (2)   */
    int32_t n_diffuse;       /* diffuse secondary rays per hit (0: none)        */
    uint32_t diffuse_seed;   /* seed of their SplitMix64 sample stream          */
} orc_params;


int orc_eval_range(const orc_mesh *m, const orc_params *p, const double s[3], int64_t r0, int64_t r1, double *acc,
                   double *scale, double *win, double *angles, int32_t *hits, double *edge, int64_t *nhit);

int orc_spad_interp(int32_t n_az, int32_t n_el, double az0, double el0, double d_el, const double *table,
                    const double s[3], double dist_au, double out[6]);

#endif
