/*
 * cloak_oracle.c -- plain CPU FP64 oracle (TEST INFRASTRUCTURE ONLY).
 *
 * A slow, literal statement of the method of Halimeh & Wegener,
 * arXiv:1209.6038, used to check the CUDA renderer.  It follows the paper's
 * steps in its own notation: the Cartesian permittivity tensor of Eq. 14 / 15,
 * the auxiliary matrix of Eq. 7 from the principal-frame inverse permittivity, the equations of
 * motion Eq. 2 and Eq. 8 written term by term, the Sect. 3 interface through
 * Eqs. 9-11 (angle of refraction found by bisection), the transmission
 * coefficients of Eq. 12 from a 4x4 field-continuity solve, and classical
 * fourth-order Runge-Kutta (Sect. 4).  No blocking, fusion or algebraic
 * simplification beyond what those formulas state.
 *
 * Readings where the paper is silent are marked "Reading:".
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1 /* _Float128 in <tgmath.h> (extended-precision build) */
#include "cloak_oracle.h"

#include <complex.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Arithmetic type.  The oracle is FP64 (orc_real = double).  The same source also builds in extended
   precision (cloak_oracle.h: ORC_REAL_KIND 1 = long double, 2 = _Float128) to settle what FP64 cannot determine:
   <tgmath.h> makes sqrt, sin, fabs, ... follow the argument type, complex arguments included. */
typedef orc_real real;
#if ORC_REAL_KIND == 0
typedef _Complex double cplx;
#define R_PI 3.141592653589793
#elif ORC_REAL_KIND == 1
typedef _Complex long double cplx;
#define R_PI 3.14159265358979323846264338327950288L
#else
typedef _Complex _Float128 cplx;
#define R_PI 3.14159265358979323846264338327950288f128
#endif
/* ORC_STATE_F64 (extended-precision builds only): the integrated state and every stage point are rounded
   to FP64 -- the right-hand sides and all other arithmetic stay exact -- to measure how far FP64 states
   alone move a ray, i.e. what an FP64 integrator can determine at best. */
#ifndef ORC_STATE_F64
#define ORC_STATE_F64 0
#endif
static void store_state(real y[6], const real y1[6]) {
    for (int i = 0; i < 6; ++i) y[i] = ORC_STATE_F64 ? (real)(double)y1[i] : y1[i];
}
/* exact ratios of the Dormand-Prince tableau evaluated in the arithmetic type */
#define R(x) ((real)(x))
static cplx csqrt_r(cplx z) { return sqrt(z); }
static real cabs_r(cplx z) { return fabs(z); }

/* ------------------------------------------------------------------ */
/* small linear algebra                                                */
/* ------------------------------------------------------------------ */
static real dot3(const real a[3], const real b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const real a[3], const real b[3], real o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static real norm3(const real a[3]) { return sqrt(dot3(a, a)); }
/* a vector of the (FP64) input structures in the arithmetic type */
static void vec_in(const double a[3], real o[3]) { o[0] = a[0]; o[1] = a[1]; o[2] = a[2]; }
static void matvec3(const real A[9], const real x[3], real y[3]) {
    for (int i = 0; i < 3; ++i) y[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
}
/* some unit vector perpendicular to n */
static void any_perp(const real n[3], real t[3]) {
    real ax[3] = {1.0, 0.0, 0.0};
    if (fabs(n[0]) > 0.9) { ax[0] = 0.0; ax[1] = 1.0; }
    cross3(n, ax, t);
    real l = norm3(t);
    for (int i = 0; i < 3; ++i) t[i] /= l;
}

static cplx cdot3(const cplx a[3], const cplx b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void ccross3(const cplx a[3], const cplx b[3], cplx o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static real cnorm2(const cplx a[3]) {
    return creal(a[0] * conj(a[0]) + a[1] * conj(a[1]) + a[2] * conj(a[2]));
}
/* normal component of the time-averaged Poynting vector, n . Re(E x H*) (factor 1/2 dropped) */
static real normal_flux(const real n[3], const cplx E[3], const cplx H[3]) {
    cplx Hc[3] = {conj(H[0]), conj(H[1]), conj(H[2])}, S[3];
    ccross3(E, Hc, S);
    return n[0] * creal(S[0]) + n[1] * creal(S[1]) + n[2] * creal(S[2]);
}
/* Gaussian elimination with partial pivoting, 4x4 complex, in place; returns 0 if singular */
static int solve4(cplx A[4][4], cplx b[4], cplx x[4]) {
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (cabs_r(A[r][col]) > cabs_r(A[piv][col])) piv = r;
        if (cabs_r(A[piv][col]) == 0.0) return 0;
        if (piv != col) {
            for (int k = 0; k < 4; ++k) { cplx t = A[col][k]; A[col][k] = A[piv][k]; A[piv][k] = t; }
            cplx t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        for (int r = col + 1; r < 4; ++r) {
            cplx f = A[r][col] / A[col][col];
            for (int k = col; k < 4; ++k) A[r][k] -= f * A[col][k];
            b[r] -= f * b[col];
        }
    }
    for (int r = 3; r >= 0; --r) {
        cplx s = b[r];
        for (int k = r + 1; k < 4; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
    return 1;
}

/* ------------------------------------------------------------------ */
/* splitmix64 (Steele, Lea & Flood, OOPSLA 2014), counter-based use     */
/* ------------------------------------------------------------------ */
uint64_t orc_splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
/* Reading: uniform in [0,1) from the top 53 bits of a hash chain over
   (seed, pixel, sample, dimension). */
double orc_uniform(uint64_t seed, uint64_t pixel, uint32_t sample, uint32_t dim) {
    uint64_t h = orc_splitmix64(seed);
    h = orc_splitmix64(h ^ pixel);
    h = orc_splitmix64(h ^ (((uint64_t)sample << 8) | (uint64_t)dim));
    return (double)(h >> 11) * 0x1.0p-53;
}

/* ------------------------------------------------------------------ */
/* material: Eq. 14 / Eq. 15 in cylindrical components                 */
/* ------------------------------------------------------------------ */
/* Cylindrical components (eps'_r, eps'_theta, eps'_z) at radius r and their
   r-derivatives.  a = R1, b = R2. */
static void cyl_eps(const orc_cloak *c, real r, real e[3], real de[3]) {
    real a = c->R1, b = c->R2;
    real K = (b / (b - a)) * (b / (b - a));
    real q = (r - a) / r;
    real er = q * q * K;                      /* ((r-a)/r)^2 (b/(b-a))^2 */
    real der = 2.0 * q * (a / (r * r)) * K;   /* d/dr of the above */
    e[0] = er;
    de[0] = der;
    e[1] = K; /* eps'_theta = (b/(b-a))^2 in both Eq. 14 and Eq. 15 */
    de[1] = 0.0;
    if (c->variant == ORC_RADIAL) { e[2] = K; de[2] = 0.0; }   /* Eq. 14 */
    else { e[2] = er; de[2] = der; }                            /* Eq. 15 */
}
static void cyl_basis(const real x[3], real *r, real rh[3], real th[3]) {
    *r = hypot(x[0], x[1]);
    rh[0] = x[0] / *r; rh[1] = x[1] / *r; rh[2] = 0.0;
    th[0] = -x[1] / *r; th[1] = x[0] / *r; th[2] = 0.0;
}

/* Cartesian permittivity tensor (Eq. 1 rotated to the lab frame), with the
   ordinary/extraordinary values and the optic axis c-hat. */
void orc_permittivity(const orc_cloak *c, const real x[3], real eps[9], real *eps_o, real *eps_e,
                      real chat[3]) {
    if (c->variant == ORC_TEST_CONST) {
        real ct[3];
        vec_in(c->c_test, ct);
        real l = norm3(ct);
        for (int i = 0; i < 3; ++i) chat[i] = ct[i] / l;
        *eps_o = c->eps_o_test;
        *eps_e = c->eps_e_test;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                eps[3 * i + j] = (i == j ? *eps_o : 0.0) + (*eps_e - *eps_o) * chat[i] * chat[j];
        return;
    }
    real r, rh[3], th[3], zh[3] = {0, 0, 1}, e[3], de[3];
    cyl_basis(x, &r, rh, th);
    cyl_eps(c, r, e, de);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            eps[3 * i + j] = e[0] * rh[i] * rh[j] + e[1] * th[i] * th[j] + e[2] * zh[i] * zh[j];
    if (c->variant == ORC_RADIAL) {          /* optic axis r-hat: eps_e = eps'_r, eps_o = eps'_theta = eps'_z */
        *eps_e = e[0]; *eps_o = e[1];
        for (int i = 0; i < 3; ++i) chat[i] = rh[i];
    } else {                                 /* optic axis theta-hat: eps_e = eps'_theta, eps_o = eps'_r = eps'_z */
        *eps_e = e[1]; *eps_o = e[0];
        for (int i = 0; i < 3; ++i) chat[i] = th[i];
    }
}

/* Inverse permittivity in the lab frame.  eps is diagonal in its own frame
   (Eq. 1; the cylindrical frame of Eq. 14 / 15), so its inverse is the sum of
   the reciprocal principal values times the projectors -- no numerical
   inversion (which would lose ~eps_max/eps_min of relative precision near
   r = R1, where one principal value tends to zero). */
static void inv_permittivity(const orc_cloak *c, const real x[3], real ie[9]) {
    if (c->variant == ORC_TEST_CONST) {
        real ct[3], ch[3];
        vec_in(c->c_test, ct);
        real l = norm3(ct);
        for (int i = 0; i < 3; ++i) ch[i] = ct[i] / l;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                ie[3 * i + j] = (i == j ? 1.0 / c->eps_o_test : 0.0) +
                                (1.0 / c->eps_e_test - 1.0 / c->eps_o_test) * ch[i] * ch[j];
        return;
    }
    real r, rh[3], th[3], zh[3] = {0, 0, 1}, e[3], de[3];
    cyl_basis(x, &r, rh, th);
    cyl_eps(c, r, e, de);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            ie[3 * i + j] = rh[i] * rh[j] / e[0] + th[i] * th[j] / e[1] + zh[i] * zh[j] / e[2];
}

/* Eq. 7: M = n_o^2 n_e^2 eps^{-1} and its Cartesian gradient.
   dM[9*k + 3*i + j] = d M_ij / d x_k. */
void orc_aux_matrix(const orc_cloak *c, const real x[3], real M[9], real dM[27]) {
    real eps[9], eo, ee, ch[3], ie[9];
    orc_permittivity(c, x, eps, &eo, &ee, ch);
    inv_permittivity(c, x, ie);
    real P = eo * ee; /* n_o^2 n_e^2 */
    for (int i = 0; i < 9; ++i) M[i] = P * ie[i];
    if (c->variant == ORC_TEST_CONST) {
        memset(dM, 0, 27 * sizeof(real));
        return;
    }
    real r, rh[3], th[3], zh[3] = {0, 0, 1}, e[3], de[3];
    cyl_basis(x, &r, rh, th);
    cyl_eps(c, r, e, de);
    real deo, dee; /* d eps_o / dr, d eps_e / dr */
    if (c->variant == ORC_RADIAL) { dee = de[0]; deo = de[1]; }
    else { dee = de[1]; deo = de[0]; }
    for (int k = 0; k < 3; ++k) {
        /* derivatives of the basis along x_k: d rh = th_k th / r, d th = -th_k rh / r, d zh = 0 */
        real drh[3], dth[3];
        for (int i = 0; i < 3; ++i) { drh[i] = th[k] * th[i] / r; dth[i] = -th[k] * rh[i] / r; }
        real die[9]; /* d(eps^{-1}) / dx_k */
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                die[3 * i + j] = -de[0] / (e[0] * e[0]) * rh[k] * rh[i] * rh[j] +
                                 (drh[i] * rh[j] + rh[i] * drh[j]) / e[0] -
                                 de[1] / (e[1] * e[1]) * rh[k] * th[i] * th[j] +
                                 (dth[i] * th[j] + th[i] * dth[j]) / e[1] -
                                 de[2] / (e[2] * e[2]) * rh[k] * zh[i] * zh[j];
        real dP = (deo * ee + eo * dee) * rh[k];
        for (int i = 0; i < 9; ++i) dM[9 * k + i] = dP * ie[i] + P * die[i];
    }
}

/* Eq. 7 inverted: M^{-1} = eps / (n_o^2 n_e^2). */
void orc_aux_inverse(const orc_cloak *c, const real x[3], real Mi[9]) {
    real eps[9], eo, ee, ch[3];
    orc_permittivity(c, x, eps, &eo, &ee, ch);
    for (int i = 0; i < 9; ++i) Mi[i] = eps[i] / (eo * ee);
}

/* Eq. 8: dv/dt = (1/2) M^{-1} [ v (grad M) v - 2 ((grad M) . v) v ].
   Reading: component i of "v (grad M) v" is v^T (d_i M) v; "((grad M) . v) v"
   is sum_l v_l (d_l M) v. */
void orc_eq8_accel(const real Mi[9], const real dM[27], const real v[3], real a[3]) {
    real g[3], h[3], w[3];
    for (int i = 0; i < 3; ++i) {
        real s = 0.0;
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) s += v[j] * dM[9 * i + 3 * j + k] * v[k];
        g[i] = s;
    }
    for (int j = 0; j < 3; ++j) {
        real s = 0.0;
        for (int l = 0; l < 3; ++l)
            for (int k = 0; k < 3; ++k) s += v[l] * dM[9 * l + 3 * j + k] * v[k];
        h[j] = s;
    }
    for (int i = 0; i < 3; ++i) w[i] = g[i] - 2.0 * h[i];
    matvec3(Mi, w, a);
    for (int i = 0; i < 3; ++i) a[i] *= 0.5;
}

/* Eq. 2: dv/dt = ( |v|^2 grad n - 2 (grad n . v) v ) / n. */
void orc_eq2_accel(real n, const real gn[3], const real v[3], real a[3]) {
    real vv = dot3(v, v), gv = dot3(gn, v);
    for (int i = 0; i < 3; ++i) a[i] = (vv * gn[i] - 2.0 * gv * v[i]) / n;
}

/* right-hand side of the first-order system y = (x, v): dx/dt = v, dv/dt = Eq. 2 (o) or Eq. 8 (e) */
void orc_rhs(const orc_cloak *c, int mode, const real y[6], real dy[6]) {
    const real *x = y, *v = y + 3;
    dy[0] = v[0]; dy[1] = v[1]; dy[2] = v[2];
    if (mode == ORC_EXTRAORDINARY) {
        real M[9], dM[27], Mi[9];
        orc_aux_matrix(c, x, M, dM);
        orc_aux_inverse(c, x, Mi);
        orc_eq8_accel(Mi, dM, v, dy + 3);
    } else {
        real gn[3] = {0, 0, 0}, n;
        if (c->variant == ORC_TEST_CONST) {
            n = sqrt(c->eps_o_test);
        } else {
            real r, rh[3], th[3], e[3], de[3];
            cyl_basis(x, &r, rh, th);
            cyl_eps(c, r, e, de);
            real eo = (c->variant == ORC_RADIAL) ? e[1] : e[0];
            real deo = (c->variant == ORC_RADIAL) ? de[1] : de[0];
            n = sqrt(eo);                       /* n_o = sqrt(eps_o) */
            for (int i = 0; i < 3; ++i) gn[i] = deo / (2.0 * n) * rh[i];
        }
        orc_eq2_accel(n, gn, v, dy + 3);
    }
}

/* ------------------------------------------------------------------ */
/* Sect. 3: refraction into the medium (Eqs. 9-11)                      */
/* ------------------------------------------------------------------ */
/* Eq. 9 with Eq. 10: index seen by the extraordinary wave whose wave vector
   makes angle phi with -n-hat inside the plane of incidence (unit tangent t).
   Eq. 10 gives the angle of D_e with c-hat through its sine; only its sine and
   cosine squared enter Eq. 9, so the arcsin is not taken. */
static real eq9_index(real no, real ne, const real ch[3], const real t[3], const real n[3], real phi) {
    real s = dot3(ch, t) * sin(phi) - dot3(ch, n) * cos(phi);
    real s2 = s * s, c2 = 1.0 - s2;
    return no * ne / sqrt(no * no * c2 + ne * ne * s2);
}

/* The propagating wave of `mode` inside the medium at face point x (outward
   normal n) whose tangential wave vector is kt, travelling inward.
   Returns 1 with k and v = M^{-1} k (Eq. 6), or 0 if the mode has no real
   angle of refraction in [0, pi/2] (evanescent). */
int orc_refract_into(const orc_cloak *c, int mode, const real x[3], const real n[3], const real kt[3],
                     real k[3], real v[3]) {
    real eps[9], eo, ee, ch[3];
    orc_permittivity(c, x, eps, &eo, &ee, ch);
    real no = sqrt(eo), ne = sqrt(ee);
    real st = norm3(kt); /* n_i sin(phi_i), left side of Eq. 11 */
    real t[3];
    if (st > 0.0) for (int i = 0; i < 3; ++i) t[i] = kt[i] / st;
    else any_perp(n, t);
    if (mode == ORC_ORDINARY) {
        real s = st / no; /* Eq. 11: n_o sin(phi_o) = n_i sin(phi_i) */
        if (s > 1.0) return 0;
        real phi = asin(s);
        for (int i = 0; i < 3; ++i) k[i] = no * (t[i] * sin(phi) - n[i] * cos(phi)); /* |k_o| = n_o */
        for (int i = 0; i < 3; ++i) v[i] = k[i] / eo; /* Eq. 6 with M = n_o^2 I */
        return 1;
    }
    /* Eq. 11 for the extraordinary wave: n(phi) sin(phi) = st, root in [0, pi/2] by bisection */
    real phi;
    if (st == 0.0) {
        phi = 0.0;
    } else {
        real hi = 0.5 * R_PI, lo = 0.0;
        if (eq9_index(no, ne, ch, t, n, hi) * sin(hi) - st < 0.0) return 0;
        for (int it = 0; it < 400; ++it) {
            real mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (eq9_index(no, ne, ch, t, n, mid) * sin(mid) - st < 0.0) lo = mid;
            else hi = mid;
        }
        phi = 0.5 * (lo + hi);
    }
    real nn = eq9_index(no, ne, ch, t, n, phi); /* |k_e| = n(phi_e) */
    for (int i = 0; i < 3; ++i) k[i] = nn * (t[i] * sin(phi) - n[i] * cos(phi));
    real Mi[9];
    orc_aux_inverse(c, x, Mi);
    matvec3(Mi, k, v); /* Eq. 6 */
    return 1;
}

/* Wave vector (possibly complex) of the inward wave of `mode` with tangential kt.
   Propagating: Eqs. 9-11 (above).  Evanescent -- Reading: the paper is silent;
   the normal component q solves the dispersion relation |k|^2 = eps_o (o) or
   k^T M^{-1} k = 1 (e) with the branch that decays into the medium. */
static void inward_wave(const orc_cloak *c, int mode, const real x[3], const real n[3], const real kt[3],
                        cplx k[3]) {
    real kr[3], vr[3];
    if (orc_refract_into(c, mode, x, n, kt, kr, vr)) {
        for (int i = 0; i < 3; ++i) k[i] = kr[i];
        return;
    }
    real eps[9], eo, ee, ch[3];
    orc_permittivity(c, x, eps, &eo, &ee, ch);
    cplx q;
    if (mode == ORC_ORDINARY) {
        q = -csqrt_r((cplx)(eo - dot3(kt, kt)));
    } else {
        real Mi[9], Mn[3], Mk[3];
        orc_aux_inverse(c, x, Mi);
        matvec3(Mi, n, Mn);
        matvec3(Mi, kt, Mk);
        real A = dot3(n, Mn), B = dot3(n, Mk), C = dot3(kt, Mk) - 1.0;
        q = (-B - csqrt_r((cplx)(B * B - A * C))) / A;
    }
    for (int i = 0; i < 3; ++i) k[i] = kt[i] + q * n[i];
}

/* Field directions of a plane wave of `mode` in the medium (Sect. 3):
   D_o is perpendicular to the ordinary main section, D_e lies in the
   extraordinary main section and is perpendicular to k; E = eps^{-1} D,
   H = k x E (mu = 1, omega = c0 = 1).
   Reading: when k is parallel to c-hat the two modes are degenerate and
   D_o is taken along z-hat x k (x-hat x k if that vanishes too). */
static void mode_fields(int mode, const cplx k[3], const real ie[9], const real ch[3], cplx E[3], cplx H[3]) {
    cplx c3[3] = {ch[0], ch[1], ch[2]}, Do[3], D[3];
    ccross3(c3, k, Do);
    if (cnorm2(Do) < 1e-20 * cnorm2(k)) {
        cplx z3[3] = {0, 0, 1};
        ccross3(z3, k, Do);
        if (cnorm2(Do) < 1e-20 * cnorm2(k)) {
            cplx x3[3] = {1, 0, 0};
            ccross3(x3, k, Do);
        }
        if (mode == ORC_EXTRAORDINARY) ccross3(k, Do, D);
        else for (int i = 0; i < 3; ++i) D[i] = Do[i];
    } else if (mode == ORC_ORDINARY) {
        for (int i = 0; i < 3; ++i) D[i] = Do[i];
    } else {
        cplx kk = cdot3(k, k), ck = cdot3(c3, k);
        for (int i = 0; i < 3; ++i) D[i] = kk * c3[i] - ck * k[i];
    }
    for (int i = 0; i < 3; ++i) E[i] = ie[3 * i] * D[0] + ie[3 * i + 1] * D[1] + ie[3 * i + 2] * D[2];
    ccross3(k, E, H);
}

/* Field directions (D, E, H) of a propagating wave of `mode` with real wave
   vector k at point x (for tests of the Sect. 3 / Sect. 5 field rules). */
void orc_mode_fields(const orc_cloak *c, int mode, const real x[3], const real k[3], real D[3], real E[3],
                     real H[3]) {
    real eps[9], eo, ee, ch[3];
    orc_permittivity(c, x, eps, &eo, &ee, ch);
    cplx ck[3] = {k[0], k[1], k[2]}, cE[3], cH[3];
    real ie[9];
    inv_permittivity(c, x, ie);
    mode_fields(mode, ck, ie, ch, cE, cH);
    for (int i = 0; i < 3; ++i) { E[i] = creal(cE[i]); H[i] = creal(cH[i]); }
    matvec3(eps, E, D);
}

/* s and p unit polarisations of a real vacuum wave k at a face with normal n */
static void vacuum_basis(const real k[3], const real n[3], real s[3], real p[3]) {
    cross3(k, n, s);
    real l = norm3(s);
    if (l < 1e-12) any_perp(n, s);
    else for (int i = 0; i < 3; ++i) s[i] /= l;
    cross3(s, k, p);
}

/* Eq. 12 at a vacuum -> medium face.  Incident unit vacuum direction d
   (d . n < 0), outward normal n, face point x.  out = {T_o^s, T_o^p, T_e^s,
   T_e^p, R^s, R^p, T_o (unpolarised), T_e (unpolarised)}. */
static int vacuum_face(const orc_cloak *c, const real x[3], const real n[3], const real d[3], const real *e3,
                       real out[9]);
int orc_transmission_in(const orc_cloak *c, const real x[3], const real n[3], const real d[3], real out[8]) {
    real o9[9];
    if (!vacuum_face(c, x, n, d, NULL, o9)) return 0;
    for (int i = 0; i < 8; ++i) out[i] = o9[i];
    return 1;
}

/* The solve of orc_transmission_in; with e3 (a unit incident polarisation across d) also out[8] = the
   reflectance of that incident wave. */
static int vacuum_face(const orc_cloak *c, const real x[3], const real n[3], const real d[3], const real *e3,
                       real out[9]) {
    real eps[9], eo, ee, ch[3];
    orc_permittivity(c, x, eps, &eo, &ee, ch);
    real dn = dot3(d, n), kt[3], kr[3];
    for (int i = 0; i < 3; ++i) { kt[i] = d[i] - dn * n[i]; kr[i] = d[i] - 2.0 * dn * n[i]; }
    cplx ko[3], ke[3], Eo[3], Ho[3], Ee[3], He[3];
    inward_wave(c, ORC_ORDINARY, x, n, kt, ko);
    inward_wave(c, ORC_EXTRAORDINARY, x, n, kt, ke);
    real ie[9];
    inv_permittivity(c, x, ie);
    mode_fields(ORC_ORDINARY, ko, ie, ch, Eo, Ho);
    mode_fields(ORC_EXTRAORDINARY, ke, ie, ch, Ee, He);
    real s[3], pi[3], pr[3];
    vacuum_basis(d, n, s, pi);
    cross3(s, kr, pr); /* reflected wave: same s, p = s x k_r */
    real t1[3], t2[3];
    for (int i = 0; i < 3; ++i) t1[i] = s[i];
    cross3(n, s, t2);
    cplx ckr[3] = {kr[0], kr[1], kr[2]}, cd[3] = {d[0], d[1], d[2]};
    cplx Ers[3] = {s[0], s[1], s[2]}, Erp[3] = {pr[0], pr[1], pr[2]}, Hrs[3], Hrp[3];
    ccross3(ckr, Ers, Hrs);
    ccross3(ckr, Erp, Hrp);
    out[8] = 0.0;
    for (int pol = 0; pol < (e3 ? 3 : 2); ++pol) {
        cplx Ei[3], Hi[3];
        for (int i = 0; i < 3; ++i) Ei[i] = pol == 0 ? s[i] : pol == 1 ? pi[i] : e3[i];
        ccross3(cd, Ei, Hi);
        /* tangential continuity of E and H: incident + reflected = transmitted */
        const cplx *cols_E[4] = {Ers, Erp, Eo, Ee}, *cols_H[4] = {Hrs, Hrp, Ho, He};
        real sign[4] = {1, 1, -1, -1};
        cplx A[4][4], b[4], u[4];
        for (int col = 0; col < 4; ++col) {
            cplx t1c[3] = {t1[0], t1[1], t1[2]}, t2c[3] = {t2[0], t2[1], t2[2]};
            A[0][col] = sign[col] * cdot3(cols_E[col], t1c);
            A[1][col] = sign[col] * cdot3(cols_E[col], t2c);
            A[2][col] = sign[col] * cdot3(cols_H[col], t1c);
            A[3][col] = sign[col] * cdot3(cols_H[col], t2c);
        }
        cplx t1c[3] = {t1[0], t1[1], t1[2]}, t2c[3] = {t2[0], t2[1], t2[2]};
        b[0] = -cdot3(Ei, t1c); b[1] = -cdot3(Ei, t2c);
        b[2] = -cdot3(Hi, t1c); b[3] = -cdot3(Hi, t2c);
        if (!solve4(A, b, u)) return 0;
        real fi = fabs(normal_flux(n, Ei, Hi));
        real To = cabs_r(u[2]) * cabs_r(u[2]) * fabs(normal_flux(n, Eo, Ho)) / fi;
        real Te = cabs_r(u[3]) * cabs_r(u[3]) * fabs(normal_flux(n, Ee, He)) / fi;
        cplx Er[3], Hr[3];
        for (int i = 0; i < 3; ++i) { Er[i] = u[0] * Ers[i] + u[1] * Erp[i]; Hr[i] = u[0] * Hrs[i] + u[1] * Hrp[i]; }
        real R = fabs(normal_flux(n, Er, Hr)) / fi;
        if (pol == 2) { out[8] = R; break; }
        out[0 + pol] = To;
        out[2 + pol] = Te;
        out[4 + pol] = R;
    }
    out[6] = 0.5 * (out[0] + out[1]); /* unpolarised light: mean over s and p */
    out[7] = 0.5 * (out[2] + out[3]);
    return 1;
}

/* Eq. 12 at a medium -> vacuum face (Sect. 3, last paragraph): incident
   wave of `mode` with real wave vector k, one refracted vacuum wave and two
   reflected waves (o and e) in the medium.  out = {T, R_o, R_e, polariser fraction of the transmitted
   wave}.  Under total internal reflection (|k_t| > 1) T = 0 and R_o + R_e = 1. */
int orc_transmission_out(const orc_cloak *c, int mode, const real x[3], const real n[3], const real k[3],
                         real out[4]) {
    real eps[9], eo, ee, ch[3];
    orc_permittivity(c, x, eps, &eo, &ee, ch);
    real kn = dot3(k, n), kt[3];
    for (int i = 0; i < 3; ++i) kt[i] = k[i] - kn * n[i];
    real kt2 = dot3(kt, kt);
    out[0] = out[1] = out[2] = out[3] = 0.0;
    /* vacuum side: propagating wave, or under total internal reflection (|k_t| > 1) the evanescent wave
       that decays away from the face (k_n = i sqrt(|k_t|^2 - 1)); it carries no flux */
    const int tir = kt2 > 1.0;
    cplx ckv[3];
    for (int i = 0; i < 3; ++i) ckv[i] = kt[i] + (tir ? I * sqrt(kt2 - 1.0) : sqrt(1.0 - kt2)) * n[i];
    real s[3];
    cross3(kt, n, s); /* s perpendicular to the plane of incidence; p = s x k */
    {
        real l = norm3(s);
        if (l < 1e-12) any_perp(n, s);
        else for (int i = 0; i < 3; ++i) s[i] /= l;
    }
    real kv[3] = {creal(ckv[0]), creal(ckv[1]), creal(ckv[2])};
    cplx Es[3] = {s[0], s[1], s[2]}, Ep[3], Hs[3], Hp[3];
    ccross3(Es, ckv, Ep);
    ccross3(ckv, Es, Hs);
    ccross3(ckv, Ep, Hp);
    cplx kro[3], kre[3], Ero[3], Hro[3], Ere[3], Hre[3], ck[3] = {k[0], k[1], k[2]}, Em[3], Hm[3];
    inward_wave(c, ORC_ORDINARY, x, n, kt, kro);
    inward_wave(c, ORC_EXTRAORDINARY, x, n, kt, kre);
    real ie[9];
    inv_permittivity(c, x, ie);
    mode_fields(ORC_ORDINARY, kro, ie, ch, Ero, Hro);
    mode_fields(ORC_EXTRAORDINARY, kre, ie, ch, Ere, Hre);
    mode_fields(mode, ck, ie, ch, Em, Hm);
    real t1[3], t2[3];
    for (int i = 0; i < 3; ++i) t1[i] = s[i];
    cross3(n, s, t2);
    cplx t1c[3] = {t1[0], t1[1], t1[2]}, t2c[3] = {t2[0], t2[1], t2[2]};
    /* tangential continuity: incident + reflected (medium side) = transmitted (vacuum side) */
    const cplx *cols_E[4] = {Es, Ep, Ero, Ere}, *cols_H[4] = {Hs, Hp, Hro, Hre};
    real sign[4] = {1, 1, -1, -1};
    cplx A[4][4], b[4], u[4];
    for (int col = 0; col < 4; ++col) {
        A[0][col] = sign[col] * cdot3(cols_E[col], t1c);
        A[1][col] = sign[col] * cdot3(cols_E[col], t2c);
        A[2][col] = sign[col] * cdot3(cols_H[col], t1c);
        A[3][col] = sign[col] * cdot3(cols_H[col], t2c);
    }
    b[0] = cdot3(Em, t1c); b[1] = cdot3(Em, t2c);
    b[2] = cdot3(Hm, t1c); b[3] = cdot3(Hm, t2c);
    if (!solve4(A, b, u)) return 0;
    real fi = fabs(normal_flux(n, Em, Hm));
    cplx Et[3], Ht[3];
    for (int i = 0; i < 3; ++i) { Et[i] = u[0] * Es[i] + u[1] * Ep[i]; Ht[i] = u[0] * Hs[i] + u[1] * Hp[i]; }
    out[0] = tir ? 0.0 : fabs(normal_flux(n, Et, Ht)) / fi;
    out[1] = cabs_r(u[2]) * cabs_r(u[2]) * fabs(normal_flux(n, Ero, Hro)) / fi;
    out[2] = cabs_r(u[3]) * cabs_r(u[3]) * fabs(normal_flux(n, Ere, Hre)) / fi;
    if (tir) return 1; /* nothing reaches the camera-side polariser */
    /* linear polariser in front of the camera: it passes the field component along its axis, taken
       across the transmitted vacuum wave (Malus's law, |E . a|^2 / |E|^2) */
    out[3] = 1.0;
    real av[3];
    vec_in(c->analyzer, av);
    real an = dot3(av, av);
    if (an > 0.0) {
        real a[3], ak = dot3(av, kv);
        for (int i = 0; i < 3; ++i) a[i] = av[i] - ak * kv[i];
        real al = sqrt(dot3(a, a));
        cplx ea = 0.0, ee2 = 0.0;
        for (int i = 0; i < 3; ++i) {
            ea += Et[i] * (a[i] / al);
            ee2 += Et[i] * conj(Et[i]);
        }
        out[3] = al > 0.0 && creal(ee2) > 0.0 ? creal(ea * conj(ea)) / creal(ee2) : 0.0;
    }
    return 1;
}

/* ------------------------------------------------------------------ */
/* integrators                                                          */
/* ------------------------------------------------------------------ */
/* classical fourth-order Runge-Kutta (Sect. 4) */
/* right-hand side of the cloak's formulation (Fermat: orc_rhs; Hamiltonian: orc_rhs_hamiltonian) */
/* ORC_MIXED_F32 (extended-precision builds only): a model of where FP32 enters a mixed-precision
   integrator.  Outside the band r < R1 + ORC_F32_BAND the stage point's z and velocity are FP32 numbers (x
   and y stay exact) and the right-hand side is rounded to FP32; inside the band the stage point is an FP64
   state.  Everything else stays exact, so the distance of the result from the exact run measures how far
   FP32 right-hand sides alone move a ray -- what such an integrator can determine at best. */
#ifndef ORC_MIXED_F32
#define ORC_MIXED_F32 0
#endif
#define ORC_F32_BAND 0.02
static void rhs_of(const orc_cloak *c, int mode, const real y[6], real dy[6]) {
    real ys[6];
    store_state(ys, y);  /* ORC_STATE_F64: every stage point the right-hand side is evaluated at is an FP64 state */
    int f32 = 0;
    if (ORC_MIXED_F32) {
        f32 = !(hypot(y[0], y[1]) < c->R1 + ORC_F32_BAND);
        for (int i = 0; i < 6; ++i)
            ys[i] = f32 ? (i < 2 ? y[i] : (real)(float)y[i]) : (real)(double)y[i];
    }
    if (c->form) orc_rhs_hamiltonian(c, mode, ys, dy);
    else orc_rhs(c, mode, ys, dy);
    if (f32)
        for (int i = 3; i < 6; ++i) dy[i] = (real)(float)dy[i];
}

void orc_rk4_step(const orc_cloak *c, int mode, const real y[6], real h, real out[6]) {
    real k1[6], k2[6], k3[6], k4[6], t[6];
    rhs_of(c, mode, y, k1);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + 0.5 * h * k1[i];
    rhs_of(c, mode, t, k2);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + 0.5 * h * k2[i];
    rhs_of(c, mode, t, k3);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + h * k3[i];
    rhs_of(c, mode, t, k4);
    for (int i = 0; i < 6; ++i) out[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* Dormand & Prince (1980) 5(4) pair: out = fifth-order solution, err = its
   difference from the embedded fourth-order solution. */
void orc_dp45_step(const orc_cloak *c, int mode, const real y[6], real h, real out[6], real err[6]) {
    static const real a[7][6] = {
        {0, 0, 0, 0, 0, 0},
        {R(1) / 5, 0, 0, 0, 0, 0},
        {R(3) / 40, R(9) / 40, 0, 0, 0, 0},
        {R(44) / 45, -R(56) / 15, R(32) / 9, 0, 0, 0},
        {R(19372) / 6561, -R(25360) / 2187, R(64448) / 6561, -R(212) / 729, 0, 0},
        {R(9017) / 3168, -R(355) / 33, R(46732) / 5247, R(49) / 176, -R(5103) / 18656, 0},
        {R(35) / 384, 0, R(500) / 1113, R(125) / 192, -R(2187) / 6784, R(11) / 84}};
    static const real b5[7] = {R(35) / 384, 0, R(500) / 1113, R(125) / 192, -R(2187) / 6784, R(11) / 84, 0};
    static const real b4[7] = {R(5179) / 57600, 0, R(7571) / 16695, R(393) / 640, -R(92097) / 339200,
                                 R(187) / 2100, R(1) / 40};
    real k[7][6], t[6];
    rhs_of(c, mode, y, k[0]);
    for (int s = 1; s < 7; ++s) {
        for (int i = 0; i < 6; ++i) {
            real acc = 0.0;
            for (int j = 0; j < s; ++j) acc += a[s][j] * k[j][i];
            t[i] = y[i] + h * acc;
        }
        rhs_of(c, mode, t, k[s]);
    }
    for (int i = 0; i < 6; ++i) {
        real s5 = 0.0, s4 = 0.0;
        for (int j = 0; j < 7; ++j) { s5 += b5[j] * k[j][i]; s4 += b4[j] * k[j][i]; }
        out[i] = y[i] + h * s5;
        err[i] = h * (s5 - s4);
    }
}

static void step_solution(const orc_cloak *c, const orc_integrator *in, int mode, const real y[6], real h,
                          real out[6]) {
    if (in->kind == ORC_RK4) orc_rk4_step(c, mode, y, h, out);
    else { real e[6]; orc_dp45_step(c, mode, y, h, out, e); }
}

/* ------------------------------------------------------------------ */
/* geometry                                                             */
/* ------------------------------------------------------------------ */
/* event functions: positive once the surface has been crossed */
enum { EV_LATERAL = 0, EV_TOP = 1, EV_BOTTOM = 2, EV_METAL = 3 };
static real event_value(const orc_cloak *c, int ev, const real y[6]) {
    switch (ev) {
    case EV_LATERAL: return hypot(y[0], y[1]) - c->R2;
    case EV_TOP: return y[2] - 0.5 * c->H;
    case EV_BOTTOM: return -y[2] - 0.5 * c->H;
    default: return c->R1 - hypot(y[0], y[1]);
    }
}

/* Reading (the paper is silent): the crossing inside a step y_n -> y_{n+1} is
   the s in (0, h] at which one step of size s of the same integrator from
   y_n lands on the surface, namely the root that bisection of [0, h]
   converges to (this selects one root when a coarse step crosses the
   surface more than once).  The returned s is on the far side (exits) or the
   near side (metal). */
static real crossing(const orc_cloak *c, const orc_integrator *in, int mode, const real y[6], real h, int ev) {
    real lo = 0.0, hi = h, t[6];
    for (int it = 0; it < 400; ++it) {
        real mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        step_solution(c, in, mode, y, mid, t);
        if (event_value(c, ev, t) > 0.0) hi = mid;
        else lo = mid;
    }
    return ev == EV_METAL ? lo : hi;
}

/* first entry of the ray o + s d into the finite cylinder r <= R2, |z| <= H/2 */
static int hit_cylinder(const orc_cloak *c, const real o[3], const real d[3], real p[3], real n[3],
                        int *face) {
    real best = INFINITY;
    *face = -1;
    real A = d[0] * d[0] + d[1] * d[1], B = o[0] * d[0] + o[1] * d[1],
           C = o[0] * o[0] + o[1] * o[1] - c->R2 * c->R2;
    if (A > 0.0) {
        real disc = B * B - A * C;
        if (disc >= 0.0) {
            real s = (-B - sqrt(disc)) / A; /* nearer root: where the ray enters the infinite cylinder */
            if (s > 0.0 && fabs(o[2] + s * d[2]) <= 0.5 * c->H) { best = s; *face = EV_LATERAL; }
        }
    }
    for (int cap = 0; cap < 2; ++cap) {
        real zc = cap == 0 ? 0.5 * c->H : -0.5 * c->H;
        if (d[2] == 0.0) continue;
        if ((cap == 0 && d[2] >= 0.0) || (cap == 1 && d[2] <= 0.0)) continue; /* must approach from outside */
        real s = (zc - o[2]) / d[2];
        real px = o[0] + s * d[0], py = o[1] + s * d[1];
        if (s > 0.0 && px * px + py * py <= c->R2 * c->R2 && s < best) { best = s; *face = cap == 0 ? EV_TOP : EV_BOTTOM; }
    }
    if (*face < 0) return 0;
    for (int i = 0; i < 3; ++i) p[i] = o[i] + best * d[i];
    if (*face == EV_LATERAL) {
        real r = hypot(p[0], p[1]);
        n[0] = p[0] / r; n[1] = p[1] / r; n[2] = 0.0;
    } else {
        n[0] = n[1] = 0.0;
        n[2] = *face == EV_TOP ? 1.0 : -1.0;
    }
    return 1;
}

static void face_normal(int ev, const real x[3], real n[3]) {
    if (ev == EV_LATERAL) {
        real r = hypot(x[0], x[1]);
        n[0] = x[0] / r; n[1] = x[1] / r; n[2] = 0.0;
    } else {
        n[0] = n[1] = 0.0;
        n[2] = ev == EV_TOP ? 1.0 : -1.0;
    }
}

/* wave vector of the mode from the ray velocity: k = M v (Eq. 6) */
static void wave_vector(const orc_cloak *c, int mode, const real x[3], const real v[3], real k[3]) {
    if (mode == ORC_EXTRAORDINARY) {
        real M[9], dM[27];
        orc_aux_matrix(c, x, M, dM);
        matvec3(M, v, k);
    } else {
        real eps[9], eo, ee, ch[3];
        orc_permittivity(c, x, eps, &eo, &ee, ch);
        for (int i = 0; i < 3; ++i) k[i] = eo * v[i];
    }
}

/* ------------------------------------------------------------------ */
/* procedural room (stands in for the missing scene of the paper)       */
/* ------------------------------------------------------------------ */
/* Reading: axis-aligned box x, y in [-10, 10], z in [-H/2, -H/2 + 10];
   walls and floor checkered with 8 tiles per unit, per-tile tint from
   splitmix64(scene seed, face, i, j); constant ceiling. */
int orc_shade(const orc_cloak *c, const real p[3], const real d[3], real rgb[3]) {
    const real L = 10.0, z0 = -0.5 * c->H, z1 = z0 + 10.0;
    real best = INFINITY, s;
    int face = -1;
    if (d[0] > 0.0) { s = (L - p[0]) / d[0]; if (s < best) { best = s; face = 0; } }
    else if (d[0] < 0.0) { s = (-L - p[0]) / d[0]; if (s < best) { best = s; face = 1; } }
    if (d[1] > 0.0) { s = (L - p[1]) / d[1]; if (s < best) { best = s; face = 2; } }
    else if (d[1] < 0.0) { s = (-L - p[1]) / d[1]; if (s < best) { best = s; face = 3; } }
    if (d[2] < 0.0) { s = (z0 - p[2]) / d[2]; if (s < best) { best = s; face = 4; } }
    else if (d[2] > 0.0) { s = (z1 - p[2]) / d[2]; if (s < best) { best = s; face = 5; } }
    if (face < 0) { rgb[0] = rgb[1] = rgb[2] = 0.0; return -1; }
    if (face == 5) { rgb[0] = 0.55; rgb[1] = 0.55; rgb[2] = 0.6; return 5 << 20; }
    real q[3];
    for (int i = 0; i < 3; ++i) q[i] = p[i] + best * d[i];
    real u, v;
    int nu = 160, nv;
    if (face <= 1) { u = q[1] + L; v = q[2] - z0; nv = 80; }
    else if (face <= 3) { u = q[0] + L; v = q[2] - z0; nv = 80; }
    else { u = q[0] + L; v = q[1] + L; nv = 160; }
    int i = (int)floor(u * 8.0), j = (int)floor(v * 8.0);
    if (i < 0) i = 0;
    if (i > nu - 1) i = nu - 1;
    if (j < 0) j = 0;
    if (j > nv - 1) j = nv - 1;
    uint64_t h = orc_splitmix64(c->scene_seed);
    h = orc_splitmix64(h ^ (uint64_t)face);
    h = orc_splitmix64(h ^ (uint64_t)i);
    h = orc_splitmix64(h ^ (uint64_t)j);
    real base = ((i + j) & 1) ? 0.25 : 0.85;
    for (int ch = 0; ch < 3; ++ch) rgb[ch] = base * (0.6 + 0.4 * (real)((h >> (8 * ch)) & 255u) / 255.0);
    return (face << 20) | (i << 10) | j;
}

/* ------------------------------------------------------------------ */
/* time-of-flight difference (Sect. 4; TOF images of Ref. [10])         */
/* ------------------------------------------------------------------ */
real orc_room_distance(const orc_cloak *c, const real p[3], const real d[3]) {
    /* nearest of the six planes of the room box that the ray moves towards */
    const real L = 10.0, z0 = -0.5 * c->H, z1 = z0 + 10.0;
    real best = INFINITY;
    const real lo[3] = {-L, -L, z0}, hi[3] = {L, L, z1};
    for (int a = 0; a < 3; ++a) {
        real s = INFINITY;
        if (d[a] > 0.0) s = (hi[a] - p[a]) / d[a];
        else if (d[a] < 0.0) s = (lo[a] - p[a]) / d[a];
        if (s < best) best = s;
    }
    return best;
}

static real dist3(const real a[3], const real b[3]) {
    return sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
}

real orc_tof_difference(const orc_cloak *c, const real o[3], const real d[3], const orc_record *rec) {
    /* with c0 = 1 a time of flight is a vacuum path length, plus the time t spent inside the cloak */
    const real t_ref = orc_room_distance(c, o, d);
    const real xp[3] = {rec->exit_pos[0], rec->exit_pos[1], rec->exit_pos[2]};
    const real xd[3] = {rec->exit_dir[0], rec->exit_dir[1], rec->exit_dir[2]};
    real t;
    if (rec->status == ORC_METAL_CAP) {
        t = dist3(xp, o) + orc_room_distance(c, xp, xd);
    } else if (rec->status == ORC_EXITED || rec->status == ORC_HIT_METAL_EXITED) {
        real p[3], n[3];
        int face;
        if (!hit_cylinder(c, o, d, p, n, &face)) return 0.0;
        t = dist3(p, o) + rec->tof + orc_room_distance(c, xp, xd);
    } else {
        return 0.0;
    }
    return t - t_ref;
}

/* ------------------------------------------------------------------ */
/* one ray: entry split, integration, exit refraction, shading          */
/* ------------------------------------------------------------------ */
static void path_push(real *path, long cap, long *len, real t, const real y[6]) {
    if (!path || *len >= cap) { if (len) ++*len; return; }
    real *p = path + 7 * (*len);
    p[0] = t;
    for (int i = 0; i < 6; ++i) p[1 + i] = y[i];
    ++*len;
}

static void finish_vacuum(const orc_cloak *c, const real p[3], const real d[3], orc_record *rec) {
    real rgb[3];
    for (int i = 0; i < 3; ++i) { rec->exit_pos[i] = p[i]; rec->exit_dir[i] = d[i]; }
    rec->tile_id = orc_shade(c, p, d, rgb);
}

/* Integration inside the cloak from state y (Fermat (x, v) or Hamiltonian (x, k)) at time *t until the
   ray crosses a face: returns ORC_EXITED with y on the crossing and *ev_hit the face, or ORC_STEP_LIMIT /
   ORC_SINGULAR.  The metal cylinder mirrors radial ordinary rays (*metal set). */
static int integrate_inside(const orc_cloak *c, const orc_integrator *in, int mode, real y[6], real *t,
                            int *steps, int *metal, int *ev_hit, real *path, long path_cap, long *plen) {
    real y1[6];
    real h = in->kind == ORC_RK4 ? in->h_or_tol : 1e-3, tol = in->h_or_tol;
    const int nev = c->R1 > 0.0 ? 4 : 3;
    for (;;) {
        if (*steps >= in->max_steps || (in->kind == ORC_DP45 && h < 1e-14)) return ORC_STEP_LIMIT;
        real fac = 1.0;
        if (in->kind == ORC_RK4) {
            orc_rk4_step(c, mode, y, h, y1);
            ++*steps;
        } else {
            real e[6];
            orc_dp45_step(c, mode, y, h, y1, e);
            ++*steps;
            /* error norm: max_i |e_i| / (tol + tol max(|y_i|, |y1_i|)) */
            real err = 0.0;
            int bad = 0;
            for (int i = 0; i < 6; ++i) {
                real sc = tol + tol * fmax(fabs(y[i]), fabs(y1[i]));
                real q = fabs(e[i]) / sc;
                if (q != q) bad = 1;
                else if (q > err) err = q;
            }
            if (bad) err = NAN;
            if (!(err <= 1.0)) {
                h *= isfinite(err) ? fmax(0.2, 0.9 * pow(err, -0.2)) : 0.2;
                continue;
            }
            fac = err == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2)));
        }
        /* Reading: a DP5(4) step whose end points both lie outside the metal cylinder while its
           chord passes inside r < R1 is retried with the step shortened to the chord's closest
           approach.  (Sect. 4: all radial ordinary rays reach the metal; they travel on straight
           lines, along which the error estimate vanishes and the step grows without bound.) */
        if (in->kind == ORC_DP45 && c->R1 > 0.0 && event_value(c, EV_METAL, y1) <= 0.0) {
            real dx = y1[0] - y[0], dy = y1[1] - y[1], dd = dx * dx + dy * dy;
            if (dd > 0.0) {
                real sc = -(y[0] * dx + y[1] * dy) / dd;
                real mx = y[0] + sc * dx, my = y[1] + sc * dy;
                if (sc > 0.0 && sc < 1.0 && mx * mx + my * my < c->R1 * c->R1) {
                    h *= sc;
                    continue;
                }
            }
        }
        /* surfaces crossed by this step; the earliest crossing wins */
        int hit = -1;
        real s_hit = INFINITY;
        for (int ev = 0; ev < nev; ++ev) {
            if (event_value(c, ev, y1) > 0.0) {
                real sx = crossing(c, in, mode, y, h, ev);
                if (sx < s_hit) { s_hit = sx; hit = ev; }
            }
        }
        if (hit < 0) {
            store_state(y, y1);
            *t += h;
            h *= fac;
            path_push(path, path_cap, plen, *t, y);
            continue;
        }
        step_solution(c, in, mode, y, s_hit, y1);
        store_state(y, y1);
        *t += s_hit;
        h *= fac;
        path_push(path, path_cap, plen, *t, y);
        if (hit == EV_METAL) {
            if (c->variant == ORC_RADIAL && mode == ORC_ORDINARY) {
                /* Sect. 4: c-hat parallel to the metal normal, single mirror ray with equal angles */
                real nm[3], r = hypot(y[0], y[1]);
                nm[0] = y[0] / r; nm[1] = y[1] / r; nm[2] = 0.0;
                real vn = dot3(y + 3, nm);
                for (int i = 0; i < 3; ++i) y[3 + i] -= 2.0 * vn * nm[i];
                *metal = 1;
                path_push(path, path_cap, plen, *t, y);
                continue;
            }
            return ORC_SINGULAR;
        }
        *ev_hit = hit;
        return ORC_EXITED;
    }
}

/* Wave vector of the mode from the state's second half (Fermat: ray velocity, k = M v; Hamiltonian: k). */
static void state_wave_vector(const orc_cloak *c, int mode, const real y[6], real k[3]) {
    if (c->form)
        for (int i = 0; i < 3; ++i) k[i] = y[3 + i];
    else
        wave_vector(c, mode, y, y + 3, k);
}

/* What a camera-backward ray reaches inside: entry data and the state on the far face. */
typedef struct {
    int status;           /* ORC_* so far; ORC_EXITED: y is on face `ev` (crossed, not yet refracted) */
    real x_in[3], n_in[3], k0[3];
    real y[6], t;
    int ev, steps, metal;
} inner_path;

/* Entry split and integration of `mode` from the camera ray (o, d) to the far face. */
static void trace_to_far_face(const orc_cloak *c, const orc_integrator *in, int mode, const real o[3],
                              const real d[3], const real p[3], const real n[3], inner_path *ip,
                              real *path, long path_cap, long *plen) {
    real dn = dot3(d, n), kt[3], v0[3];
    for (int i = 0; i < 3; ++i) kt[i] = d[i] - dn * n[i];
    ip->t = 0.0;
    ip->steps = 0;
    ip->metal = 0;
    ip->ev = -1;
    for (int i = 0; i < 3; ++i) { ip->x_in[i] = p[i]; ip->n_in[i] = n[i]; }
    if (!orc_refract_into(c, mode, p, n, kt, ip->k0, v0)) {
        ip->status = ORC_NO_TRANSMISSION;
        return;
    }
    /* state (x, v) of the Fermat form or (x, k) of the Hamiltonian form */
    for (int i = 0; i < 3; ++i) { ip->y[i] = p[i]; ip->y[3 + i] = c->form ? ip->k0[i] : v0[i]; }
    path_push(path, path_cap, plen, 0.0, ip->y);
    ip->status = integrate_inside(c, in, mode, ip->y, &ip->t, &ip->steps, &ip->metal, &ip->ev, path, path_cap, plen);
    (void)o;
}

int orc_trace_ray(const orc_cloak *c, const orc_integrator *in, int mode, const real o[3], const real d[3],
                  orc_record *rec, real *path, long path_cap, long *path_len) {
    memset(rec, 0, sizeof(*rec));
    rec->mode = mode;
    rec->tile_id = -1;
    long plen = 0;
    if (path_len) *path_len = 0;
    real p[3], n[3];
    int face;
    /* unpolarised room light through a linear polariser: half of it */
    real av[3];
    vec_in(c->analyzer, av);
    const real vac = dot3(av, av) > 0.0 ? 0.5 : 1.0;
    if (!hit_cylinder(c, o, d, p, n, &face)) {
        rec->status = ORC_MISSED;
        rec->weight = vac;
        finish_vacuum(c, o, d, rec);
        return rec->status;
    }
    if (face != EV_LATERAL && c->R1 > 0.0 && hypot(p[0], p[1]) <= c->R1) {
        /* metal end disc seen from outside: mirror, reflectance 1 */
        real dr[3], dn = dot3(d, n);
        for (int i = 0; i < 3; ++i) dr[i] = d[i] - 2.0 * dn * n[i];
        rec->status = ORC_METAL_CAP;
        rec->weight = vac;
        finish_vacuum(c, p, dr, rec);
        return rec->status;
    }
    /* entry real refraction (Sect. 3), then the integration to the far face */
    inner_path ip;
    trace_to_far_face(c, in, mode, o, d, p, n, &ip, path, path_cap, &plen);
    if (path_len) *path_len = plen;
    rec->steps = ip.steps;
    rec->tof = ip.t;
    if (ip.status != ORC_EXITED) {
        rec->status = ip.status;
        const real *x = ip.status == ORC_NO_TRANSMISSION ? p : ip.y;
        for (int i = 0; i < 3; ++i) { rec->exit_pos[i] = x[i]; rec->exit_dir[i] = d[i]; }
        if (ip.status == ORC_NO_TRANSMISSION) rec->tof = 0.0;
        return rec->status;
    }
    /* exit refraction (Sect. 3): keep k_t, vacuum k_n = +sqrt(1 - |k_t|^2) */
    real xo[3] = {ip.y[0], ip.y[1], ip.y[2]}, no[3], kx[3], ktx[3];
    face_normal(ip.ev, xo, no);
    state_wave_vector(c, mode, ip.y, kx);
    real kn = dot3(kx, no);
    for (int i = 0; i < 3; ++i) ktx[i] = kx[i] - kn * no[i];
    real kt2 = dot3(ktx, ktx);
    if (kt2 > 1.0) {
        rec->status = ORC_TIR;
        for (int i = 0; i < 3; ++i) { rec->exit_pos[i] = xo[i]; rec->exit_dir[i] = d[i]; }
        return rec->status;
    }
    real dout[3];
    for (int i = 0; i < 3; ++i) dout[i] = ktx[i] + sqrt(1.0 - kt2) * no[i];
    /* Eq. 12 along the physical direction of light: from the room into the
       cloak at the exit point, and out of the cloak towards the camera at the
       entry point.  Unpolarised source: mean over s and p. */
    real Tin[8], Tout[4], mdout[3], mk0[3];
    for (int i = 0; i < 3; ++i) { mdout[i] = -dout[i]; mk0[i] = -ip.k0[i]; }
    real w = 0.0;
    if (orc_transmission_in(c, xo, no, mdout, Tin) && orc_transmission_out(c, mode, ip.x_in, ip.n_in, mk0, Tout))
        w = (mode == ORC_ORDINARY ? Tin[6] : Tin[7]) * Tout[0] * Tout[3];
    rec->weight = w;
    rec->status = ip.metal ? ORC_HIT_METAL_EXITED : ORC_EXITED;
    finish_vacuum(c, xo, dout, rec);
    return rec->status;
}

/* ------------------------------------------------------------------ */
/* first-order reflections (Sect. 3 last paragraphs, Sect. 4)          */
/* ------------------------------------------------------------------ */
/* Fraction of unpolarised room light that the outer surface at x (normal n) reflects into the camera ray
   d, through the camera's polariser if one is set.  Reading (reciprocity of the lossless, reciprocal
   interface): the light arriving along d after the reflection is what, run backwards, a vacuum wave
   incident along d reflects; so the fraction is the mean over the camera-side polarisations e (s and p,
   or the polariser's axis across d alone) of the backward reflectance R(e), halved behind a polariser. */
static real vacuum_reflection(const orc_cloak *c, const real x[3], const real n[3], const real d[3]) {
    real T[8];
    if (!orc_transmission_in(c, x, n, d, T)) return 0.0;
    real av[3];
    vec_in(c->analyzer, av);
    const real an = dot3(av, av);
    if (!(an > 0.0)) return 0.5 * (T[4] + T[5]);
    /* backward reflectance for the incident polarisation along the polariser's axis across d: the
       reflected fields of the s and p solutions superposed with the axis' s and p components */
    real a[3], ad = dot3(av, d);
    for (int i = 0; i < 3; ++i) a[i] = av[i] - ad * d[i];
    const real al = norm3(a);
    if (!(al > 0.0)) return 0.0;
    for (int i = 0; i < 3; ++i) a[i] /= al;
    real o9[9];
    if (!vacuum_face(c, x, n, d, a, o9)) return 0.0;
    return 0.5 * o9[8];
}

int orc_trace_reflections(const orc_cloak *c, const orc_integrator *in, int mode, const real o[3],
                          const real d[3], orc_record *vacrec, orc_record refl[2]) {
    memset(vacrec, 0, sizeof(*vacrec));
    memset(refl, 0, 2 * sizeof(orc_record));
    vacrec->tile_id = refl[0].tile_id = refl[1].tile_id = -1;
    vacrec->status = refl[0].status = refl[1].status = ORC_MISSED;
    refl[0].mode = ORC_ORDINARY;
    refl[1].mode = ORC_EXTRAORDINARY;
    vacrec->mode = -1;
    real p[3], n[3];
    int face;
    if (!hit_cylinder(c, o, d, p, n, &face)) return 0;
    if (face != EV_LATERAL && c->R1 > 0.0 && hypot(p[0], p[1]) <= c->R1) {
        vacrec->status = refl[0].status = refl[1].status = ORC_METAL_CAP;
        return 0;
    }
    /* (R0) the outer surface reflects room light into the camera (the same for both modes) */
    {
        real dr[3], dn = dot3(d, n);
        for (int i = 0; i < 3; ++i) dr[i] = d[i] - 2.0 * dn * n[i];
        vacrec->status = ORC_EXITED;
        vacrec->weight = vacuum_reflection(c, p, n, d);
        finish_vacuum(c, p, dr, vacrec);
    }
    /* (R1) the mode reaches the far face and, run backwards, reflects there into o' and e' */
    inner_path ip;
    trace_to_far_face(c, in, mode, o, d, p, n, &ip, NULL, 0, NULL);
    if (ip.status != ORC_EXITED) {
        refl[0].status = refl[1].status = ip.status;
        return 1;
    }
    real x1[3] = {ip.y[0], ip.y[1], ip.y[2]}, n1[3], k1[3], kt[3];
    face_normal(ip.ev, x1, n1);
    state_wave_vector(c, mode, ip.y, k1);
    const real kn = dot3(k1, n1);
    for (int i = 0; i < 3; ++i) kt[i] = k1[i] - kn * n1[i];
    /* camera-side factor: Eq. 12 out of the cloak at the entry point, through the polariser */
    real Tout0[4], mk0[3], R1[4];
    for (int i = 0; i < 3; ++i) mk0[i] = -ip.k0[i];
    const real wcam = orc_transmission_out(c, mode, ip.x_in, ip.n_in, mk0, Tout0) ? Tout0[0] * Tout0[3] : 0.0;
    if (!orc_transmission_out(c, mode, x1, n1, k1, R1)) R1[1] = R1[2] = 0.0;
    for (int m2 = 0; m2 < 2; ++m2) {
        orc_record *r = refl + m2;
        r->mode = m2;
        real kr[3], vr[3];
        if (!(R1[1 + m2] > 0.0) || !orc_refract_into(c, m2, x1, n1, kt, kr, vr)) {
            r->status = ORC_NO_TRANSMISSION; /* the reflected mode does not propagate */
            for (int i = 0; i < 3; ++i) { r->exit_pos[i] = x1[i]; r->exit_dir[i] = d[i]; }
            continue;
        }
        real y[6] = {x1[0], x1[1], x1[2], 0, 0, 0}, t = ip.t;
        for (int i = 0; i < 3; ++i) y[3 + i] = c->form ? kr[i] : vr[i];
        int steps = 0, metal = ip.metal, ev = -1;
        const int st = integrate_inside(c, in, m2, y, &t, &steps, &metal, &ev, NULL, 0, NULL);
        r->steps = steps;
        r->tof = t;
        if (st != ORC_EXITED) {
            r->status = st;
            for (int i = 0; i < 3; ++i) { r->exit_pos[i] = y[i]; r->exit_dir[i] = d[i]; }
            continue;
        }
        /* refraction out at the reflected ray's own exit, no further reflection (first order) */
        real xo[3] = {y[0], y[1], y[2]}, no[3], kx[3], ktx[3];
        face_normal(ev, xo, no);
        state_wave_vector(c, m2, y, kx);
        const real kn2 = dot3(kx, no);
        for (int i = 0; i < 3; ++i) ktx[i] = kx[i] - kn2 * no[i];
        const real kt2 = dot3(ktx, ktx);
        if (kt2 > 1.0) {
            r->status = ORC_TIR;
            for (int i = 0; i < 3; ++i) { r->exit_pos[i] = xo[i]; r->exit_dir[i] = d[i]; }
            continue;
        }
        real dout[3], mdout[3], Tin[8];
        for (int i = 0; i < 3; ++i) { dout[i] = ktx[i] + sqrt(1.0 - kt2) * no[i]; mdout[i] = -dout[i]; }
        const real tin = orc_transmission_in(c, xo, no, mdout, Tin) ? (m2 == ORC_ORDINARY ? Tin[6] : Tin[7]) : 0.0;
        r->weight = wcam * R1[1 + m2] * tin;
        r->status = metal ? ORC_HIT_METAL_EXITED : ORC_EXITED;
        finish_vacuum(c, xo, dout, r);
    }
    return 1;
}

/* The ray equations in Hamiltonian form (the comparison system of Sect. 4's closing remark): state
   (x, k) with k = M v (Eq. 7; M = eps_o I for the ordinary ray), H = (k^T M^-1 k - 1) / 2,
   dx/dt = dH/dk = M^-1 k, dk/dt = -dH/dx = -(1/2) k^T (d_i M^-1) k = (1/2) v^T (d_i M) v with v = M^-1 k
   (d M^-1 = -M^-1 (d M) M^-1, M symmetric). */
void orc_rhs_hamiltonian(const orc_cloak *c, int mode, const real y[6], real dy[6]) {
    const real *x = y, *k = y + 3;
    real M[9], dM[27], Mi[9];
    if (mode == ORC_EXTRAORDINARY) {
        orc_aux_matrix(c, x, M, dM);
        orc_aux_inverse(c, x, Mi);
    } else {
        real eo = c->eps_o_test, g[3] = {0, 0, 0};
        if (c->variant != ORC_TEST_CONST) {
            real r, rh[3], th[3], e[3], de[3];
            cyl_basis(x, &r, rh, th);
            cyl_eps(c, r, e, de);
            eo = (c->variant == ORC_RADIAL) ? e[1] : e[0];
            real deo = (c->variant == ORC_RADIAL) ? de[1] : de[0];
            for (int i = 0; i < 3; ++i) g[i] = deo * rh[i];
        }
        memset(M, 0, sizeof(M));
        memset(Mi, 0, sizeof(Mi));
        memset(dM, 0, sizeof(dM));
        for (int i = 0; i < 3; ++i) {
            M[4 * i] = eo;
            Mi[4 * i] = 1.0 / eo;
            for (int d = 0; d < 3; ++d) dM[9 * d + 4 * i] = g[d];
        }
    }
    real v[3];
    matvec3(Mi, k, v);
    for (int i = 0; i < 3; ++i) dy[i] = v[i];
    for (int d = 0; d < 3; ++d) {
        real s = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) s += v[i] * dM[9 * d + 3 * i + j] * v[j];
        dy[3 + d] = 0.5 * s;
    }
}

void orc_trace_rays(const orc_cloak *c, const orc_integrator *in, int mode, const double *rays, long n,
                    orc_record *recs, int nthreads) {
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads)
    for (long i = 0; i < n; ++i) {
        real r[6];
        for (int k = 0; k < 6; ++k) r[k] = rays[6 * i + k];
        orc_trace_ray(c, in, mode, r, r + 3, recs + i, NULL, 0, NULL);
    }
}

/* ------------------------------------------------------------------ */
/* camera and render                                                    */
/* ------------------------------------------------------------------ */
/* Pinhole camera; horizontal field of view; row 0 at the top.  One sample per
   pixel goes through the pixel centre; more samples are jittered with
   orc_uniform(seed, pixel, sample, 0 / 1). */
void orc_camera_ray(const orc_camera *cam, int i, int j, int s, int spp, uint64_t seed, real o[3], real d[3]) {
    real w[3], u[3], v[3];
    for (int k = 0; k < 3; ++k) w[k] = cam->target[k] - cam->eye[k];
    real l = norm3(w);
    for (int k = 0; k < 3; ++k) w[k] /= l;
    real up[3];
    vec_in(cam->up, up);
    cross3(w, up, u);
    l = norm3(u);
    for (int k = 0; k < 3; ++k) u[k] /= l;
    cross3(u, w, v);
    real tx = tan(0.5 * cam->hfov_deg * R_PI / 180.0);
    real ty = tx * (real)cam->height / (real)cam->width;
    real xi1 = 0.5, xi2 = 0.5;
    if (spp > 1) {
        uint64_t pix = (uint64_t)j * (uint64_t)cam->width + (uint64_t)i;
        xi1 = orc_uniform(seed, pix, (uint32_t)s, 0);
        xi2 = orc_uniform(seed, pix, (uint32_t)s, 1);
    }
    real px = (2.0 * (i + xi1) / cam->width - 1.0) * tx;
    real py = (1.0 - 2.0 * (j + xi2) / cam->height) * ty;
    for (int k = 0; k < 3; ++k) d[k] = w[k] + px * u[k] + py * v[k];
    l = norm3(d);
    for (int k = 0; k < 3; ++k) { d[k] /= l; o[k] = cam->eye[k]; }
}

void orc_render(const orc_cloak *c, const orc_integrator *in, const orc_camera *cam, int mode, int spp,
                uint64_t seed, const int64_t *pixels, long npix, double *rgba, orc_record *recs, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    long total = pixels ? npix : (long)cam->width * cam->height;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (long idx = 0; idx < total; ++idx) {
        long pix = pixels ? (long)pixels[idx] : idx;
        int i = (int)(pix % cam->width), j = (int)(pix / cam->width);
        real acc[4] = {0, 0, 0, 0};
        for (int s = 0; s < spp; ++s) {
            real o[3], d[3], rgb[3];
            orc_record rec;
            orc_camera_ray(cam, i, j, s, spp, seed, o, d);
            orc_trace_ray(c, in, mode, o, d, &rec, NULL, 0, NULL);
            if (rec.tile_id >= 0) {
                real xp[3] = {rec.exit_pos[0], rec.exit_pos[1], rec.exit_pos[2]};
                real xd[3] = {rec.exit_dir[0], rec.exit_dir[1], rec.exit_dir[2]};
                orc_shade(c, xp, xd, rgb);
            }
            else rgb[0] = rgb[1] = rgb[2] = 0.0;
            for (int k = 0; k < 3; ++k) acc[k] += rec.weight * rgb[k];
            acc[3] += rec.weight;
            if (recs) recs[idx * spp + s] = rec;
        }
        if (rgba)
            for (int k = 0; k < 4; ++k) rgba[4 * idx + k] = acc[k] / spp;
    }
}
