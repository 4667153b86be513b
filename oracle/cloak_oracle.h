/*
 * cloak_oracle.h -- plain CPU FP64 oracle for ray tracing through the
 * non-magnetic uniaxial cylindrical cloaks of Halimeh & Wegener,
 * "Photorealistic ray tracing of free-space invisibility cloaks made of
 * uniaxial dielectrics" (arXiv:1209.6038).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, literal statement of
 * the method that the CUDA renderer is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * renderer never calls it and shares no code, header or constant table with it.
 *
 * Units: c0 = omega = 1 (vacuum |k| = |v| = 1).  Cylinder axis = +z.
 * Cloak shell: R1 <= r <= R2, |z| <= H/2; metal core r <= R1, |z| <= H/2.
 *
 * Every function states the passage it follows (Sect., Eq.).
 */
#ifndef CLOAK_ORACLE_H
#define CLOAK_ORACLE_H

#include <stdint.h>

/* Arithmetic type of the oracle: FP64.  Built with -DORC_REAL_KIND=1 (long double) or 2 (_Float128) the
   same source runs in extended precision (test infrastructure for rays FP64 cannot determine); the
   structures, the records, orc_uniform, the rays of orc_trace_rays and the image of orc_render stay FP64
   in every build. */
#ifndef ORC_REAL_KIND
#define ORC_REAL_KIND 0
#endif
#if ORC_REAL_KIND == 0
typedef double orc_real;
#elif ORC_REAL_KIND == 1
typedef long double orc_real;
#else
typedef _Float128 orc_real;
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORC_RADIAL = 0,        /* Eq. 14: optic axis along r-hat */
    ORC_AZIMUTHAL = 1,     /* Eq. 15: optic axis along theta-hat */
    ORC_TEST_CONST = 100   /* homogeneous uniaxial test medium (Eq. 1, fixed c-hat), no metal core */
};
enum { ORC_ORDINARY = 0, ORC_EXTRAORDINARY = 1 };
enum { ORC_RK4 = 0, ORC_DP45 = 1 };

enum {
    ORC_MISSED = 0,           /* camera ray never meets the cylinder */
    ORC_EXITED = 1,           /* passed through the cloak and left it */
    ORC_HIT_METAL_EXITED = 2, /* mirrored at r = R1 at least once, then left */
    ORC_NO_TRANSMISSION = 3,  /* chosen mode has no propagating refracted wave at entry */
    ORC_TIR = 4,              /* total internal reflection at the exit face */
    ORC_STEP_LIMIT = 5,       /* max_steps reached or step size underflow */
    ORC_SINGULAR = 6,         /* reached r <= R1 in a mode that has no mirror rule */
    ORC_METAL_CAP = 7         /* mirrored off a metal end disc (r <= R1) from outside */
};

typedef struct {
    int variant;
    double R1, R2, H;          /* inner radius a, outer radius b, height */
    double eps_o_test, eps_e_test, c_test[3];
    uint64_t scene_seed;       /* seed of the procedural room */
    double analyzer[3];        /* axis of a linear polariser in front of the camera (the paper's
                                  "polarization goggles"); all zero: none */
    int form;                  /* ray equations: 0 Fermat form (Eq. 2 / Eq. 8, state (x, v)),
                                  1 Hamiltonian form (state (x, k), k = M v) */
} orc_cloak;

typedef struct {
    int kind;                  /* ORC_RK4 or ORC_DP45 */
    double h_or_tol;           /* fixed step (RK4) or tolerance (DP45) */
    long max_steps;            /* step attempts per ray before ORC_STEP_LIMIT */
} orc_integrator;

typedef struct {
    double eye[3], target[3], up[3];
    double hfov_deg;           /* horizontal field of view */
    int width, height;
} orc_camera;

/* 80-byte per-sample record */
typedef struct {
    double exit_pos[3];        /* start of the final vacuum ray */
    double exit_dir[3];        /* direction of the final vacuum ray (unit) */
    double tof;                /* time spent inside the cloak (t of Eq. 2 / Eq. 8) */
    double weight;             /* T_in * T_out of Eq. 12 (physical direction), 1 for misses */
    int32_t tile_id;           /* room tile hit by the final vacuum ray, -1 if none */
    int32_t status;
    int32_t steps;             /* integrator step attempts */
    int32_t mode;              /* polarization mode traced */
} orc_record;

/* ---- counter-based random numbers (splitmix64, Steele/Lea/Flood 2014) ---- */
uint64_t orc_splitmix64(uint64_t z);
double orc_uniform(uint64_t seed, uint64_t pixel, uint32_t sample, uint32_t dim);

/* ---- material (Eq. 1, 7, 14, 15) ---- */
void orc_permittivity(const orc_cloak *c, const orc_real x[3], orc_real eps[9],
                      orc_real *eps_o, orc_real *eps_e, orc_real chat[3]);
void orc_aux_matrix(const orc_cloak *c, const orc_real x[3], orc_real M[9], orc_real dM[27]);
void orc_aux_inverse(const orc_cloak *c, const orc_real x[3], orc_real Minv[9]);
void orc_eq8_accel(const orc_real Minv[9], const orc_real dM[27], const orc_real v[3], orc_real a[3]);
void orc_eq2_accel(orc_real n, const orc_real gradn[3], const orc_real v[3], orc_real a[3]);
void orc_rhs(const orc_cloak *c, int mode, const orc_real y[6], orc_real dy[6]);

/* ---- interface (Sect. 3, Eqs. 9-12) ---- */
int orc_refract_into(const orc_cloak *c, int mode, const orc_real x[3], const orc_real nhat[3],
                     const orc_real kt[3], orc_real k[3], orc_real v[3]);
void orc_mode_fields(const orc_cloak *c, int mode, const orc_real x[3], const orc_real k[3],
                     orc_real D[3], orc_real E[3], orc_real H[3]);
int orc_transmission_in(const orc_cloak *c, const orc_real x[3], const orc_real nhat[3],
                        const orc_real d[3], orc_real out[8]);
/* out[0] transmitted flux fraction, out[1], out[2] reflected into o / e, out[3] fraction of the
   transmitted flux that passes the analyser c->analyzer (1 without one); under total internal
   reflection out[0] = 0 and out[1] + out[2] = 1 */
int orc_transmission_out(const orc_cloak *c, int mode, const orc_real x[3], const orc_real nhat[3],
                         const orc_real k[3], orc_real out[4]);

/* First-order reflections of one camera sample traced in `mode` (the paper keeps first-order reflections,
   Sect. 4): vac = room light the outer surface reflects into the camera at the entry point (weight =
   reflectance, the same for both modes), refl[m'] = room light that enters the cloak, travels as mode m',
   reflects at the far face of the camera-backward ray into `mode` and leaves towards the camera (exit
   point and direction of the m' ray, time of flight of both legs, weight = camera-side Eq. 12 factor x
   reflection coefficient x entry Eq. 12 factor of m').  Returns 0 for rays that never enter the shell. */
int orc_trace_reflections(const orc_cloak *c, const orc_integrator *in, int mode, const orc_real o[3],
                          const orc_real d[3], orc_record *vac, orc_record refl[2]);

/* Hamiltonian form of the ray equations, state (x, k), k = M v: dx/dt = M^-1 k,
   dk/dt = (1/2) v^T (d_i M) v (the comparison system of Sect. 4's closing remark) */
void orc_rhs_hamiltonian(const orc_cloak *c, int mode, const orc_real y[6], orc_real dy[6]);

/* ---- integrator steps (Sect. 4: RK4; Dormand-Prince 5(4) adaptive) ---- */
void orc_rk4_step(const orc_cloak *c, int mode, const orc_real y[6], orc_real h, orc_real out[6]);
void orc_dp45_step(const orc_cloak *c, int mode, const orc_real y[6], orc_real h,
                   orc_real out[6], orc_real err[6]);

/* ---- whole-ray tracing ---- */
int orc_trace_ray(const orc_cloak *c, const orc_integrator *in, int mode,
                  const orc_real o[3], const orc_real d[3], orc_record *rec,
                  orc_real *path, long path_cap, long *path_len);
void orc_trace_rays(const orc_cloak *c, const orc_integrator *in, int mode,
                    const double *rays, long n, orc_record *recs, int nthreads);

/* ---- camera, room, render ---- */
void orc_camera_ray(const orc_camera *cam, int i, int j, int s, int spp, uint64_t seed,
                    orc_real o[3], orc_real d[3]);
int orc_shade(const orc_cloak *c, const orc_real p[3], const orc_real d[3], orc_real rgb[3]);
void orc_render(const orc_cloak *c, const orc_integrator *in, const orc_camera *cam,
                int mode, int spp, uint64_t seed, const int64_t *pixels, long npix,
                double *rgba, orc_record *recs, int nthreads);

/* ---- time-of-flight difference images (Sect. 4, after Ref. [10]) ---- */
/* distance from p along the unit direction d to the room of orc_shade (INFINITY if none) */
orc_real orc_room_distance(const orc_cloak *c, const orc_real p[3], const orc_real d[3]);
/* time of flight (c0 = 1) of the light a camera sample (o, d, its record) receives from the room, minus
   the time from the room point the same camera ray sees without the cylinder; 0 for rays that miss the
   cylinder and for records that carry no light */
orc_real orc_tof_difference(const orc_cloak *c, const orc_real o[3], const orc_real d[3], const orc_record *rec);

#ifdef __cplusplus
}
#endif
#endif
