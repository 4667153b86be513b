// trace.cuh -- one camera/test ray through the cloak in FP64 (Sect. 4 pipeline):
// cylinder entry, Sect. 3 double refraction into the chosen mode, integration of
// Eq. 2 / Eq. 8 (RK4 at fixed h, or Dormand-Prince 5(4)), crossing of the exit face,
// the metal mirror at r = R1 for radial ordinary rays, exit refraction, Eq. 12
// weights along the physical direction of light, and the room lookup.
#pragma once

#include "physics.cuh"

namespace ck {

__device__ __forceinline__ void set_vec(double *dst, const double *src) {
    dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2];
}

// Time-of-flight difference of one camera sample (TOF images, Sect. 4 after Ref. [10]); c0 = 1, so a time
// of flight is a vacuum path length plus the time t spent inside the cloak.  The light the sample
// receives travels from the room point its final vacuum ray reaches, back along that ray, through the
// cloak and to the camera; subtracted is the time from the room point the straight camera ray reaches.
// Rays that miss the cylinder give 0, as do records that carry no light.
__device__ __forceinline__ double tof_difference(const Params &p, const double o[3], const double d[3],
                                                 const cloak_record &rec) {
    int face;
    const double t_ref = room_distance(p, o, d, face);
    double t, pt[3], n[3];
    if (rec.status == CLOAK_RAY_METAL_CAP) {
        for (int i = 0; i < 3; ++i) pt[i] = rec.exit_pos[i];
        t = 0.0;
    } else if (rec.status == CLOAK_RAY_EXITED || rec.status == CLOAK_RAY_HIT_METAL_EXITED) {
        if (cylinder_entry(p, o, d, pt, n) < 0) return 0.0;
        t = rec.tof;
    } else {
        return 0.0;
    }
    const double dx = pt[0] - o[0], dy = pt[1] - o[1], dz = pt[2] - o[2];
    t += sqrt(dx * dx + dy * dy + dz * dz) + room_distance(p, rec.exit_pos, rec.exit_dir, face);
    return t - t_ref;
}

// Entry part: returns true when the ray continues into the medium with state y (x, v).
// Otherwise rec and rgb are final.
template <int MODE>
__device__ __forceinline__ bool enter(const Params &p, const double o[3], const double d[3], cloak_record &rec,
                                      float rgb[3], double y[6], double k0[3], double n_in[3], double mat_in[5]) {
    rec.mode = MODE;
    rec.tile_id = -1;
    rec.steps = 0;
    rec.tof = 0.0;
    rec.weight = 0.0;
    rgb[0] = rgb[1] = rgb[2] = 0.f;
    double pt[3];
    int face = cylinder_entry(p, o, d, pt, n_in);
    // unpolarised room light through the camera's polariser: half of it
    const double vac = p.analyzer ? 0.5 : 1.0;
    if (face < 0) {
        rec.status = CLOAK_RAY_MISSED;
        rec.weight = vac;
        set_vec(rec.exit_pos, o);
        set_vec(rec.exit_dir, d);
        rec.tile_id = room_hit(p, o, d, rgb);
        return false;
    }
    if (face != EV_LAT && p.R1 > 0.0 && hypot(pt[0], pt[1]) <= p.R1) {  // metal end disc: mirror
        double dr[3], dn = dot3(d, n_in);
        for (int i = 0; i < 3; ++i) dr[i] = d[i] - 2.0 * dn * n_in[i];
        rec.status = CLOAK_RAY_METAL_CAP;
        rec.weight = vac;
        set_vec(rec.exit_pos, pt);
        set_vec(rec.exit_dir, dr);
        rec.tile_id = room_hit(p, pt, dr, rgb);
        return false;
    }
    double eo, ee, c[3];
    local_material(p, pt, eo, ee, c);
    double dn = dot3(d, n_in), kt[3], v0[3];
    for (int i = 0; i < 3; ++i) kt[i] = d[i] - dn * n_in[i];
    if (!refract_in(MODE, eo, ee, c, n_in, kt, k0, v0)) {
        rec.status = CLOAK_RAY_NO_TRANSMISSION;
        set_vec(rec.exit_pos, pt);
        set_vec(rec.exit_dir, d);
        return false;
    }
    mat_in[0] = eo; mat_in[1] = ee; mat_in[2] = c[0]; mat_in[3] = c[1]; mat_in[4] = c[2];
    y[0] = pt[0]; y[1] = pt[1]; y[2] = pt[2];
    // the state's second half: ray velocity (Fermat form) or wave vector (Hamiltonian form)
    const double *w = p.formulation ? k0 : v0;
    y[3] = w[0]; y[4] = w[1]; y[5] = w[2];
    return true;
}

// Exit part: refraction into vacuum at the crossed face, Eq. 12 weights, room lookup.
template <int MODE>
__device__ __forceinline__ void leave(const Params &p, int ev, const double y[6], const double d_cam[3],
                                      const double k0[3], const double n_in[3], const double mat_in[5], bool metal,
                                      double t, int steps, cloak_record &rec, float rgb[3]) {
    double x[3] = {y[0], y[1], y[2]}, n[3], eo, ee, c[3], k[3];
    face_normal(ev, x, n);
    local_material(p, x, eo, ee, c);
    if (p.formulation) set_vec(k, y + 3);
    else wave_from_velocity(MODE, eo, ee, c, y + 3, k);
    double kn = dot3(k, n), kt[3];
    for (int i = 0; i < 3; ++i) kt[i] = k[i] - kn * n[i];
    double kt2 = dot3(kt, kt);
    rec.steps = steps;
    rec.tof = t;
    set_vec(rec.exit_pos, x);
    if (kt2 > 1.0) {
        rec.status = CLOAK_RAY_TIR;
        set_vec(rec.exit_dir, d_cam);
        return;
    }
    double qn = sqrt(1.0 - kt2), dout[3], mdout[3], mk0[3];
    for (int i = 0; i < 3; ++i) {
        dout[i] = fma(qn, n[i], kt[i]);
        mdout[i] = -dout[i];
        mk0[i] = -k0[i];
    }
    // light enters from the room at this face and leaves towards the camera at the entry face
    double tin = transmission_in(MODE, eo, ee, c, n, mdout);
    double cin[3] = {mat_in[2], mat_in[3], mat_in[4]};
    double tout = transmission_out(MODE, mat_in[0], mat_in[1], cin, n_in, mk0, analyzer_axis(p));
    rec.weight = tin * tout;
    rec.status = metal ? CLOAK_RAY_HIT_METAL_EXITED : CLOAK_RAY_EXITED;
    set_vec(rec.exit_dir, dout);
    rec.tile_id = room_hit(p, x, dout, rgb);
}

// Whole ray, FP64.  rgb receives the room colour (0 when there is none).
template <int VAR, int MODE, int INTEG>
__device__ void trace_ray(const Params &p, const double o[3], const double d[3], cloak_record &rec, float rgb[3]) {
    double y[6], k0[3], n_in[3], mat_in[5];
    if (!enter<MODE>(p, o, d, rec, rgb, y, k0, n_in, mat_in)) return;
    double t = 0.0, h = INTEG == I_RK4 ? p.h_or_tol : 1e-3, tol = p.h_or_tol;
    int steps = 0;
    bool metal = false, have_k1 = false;
    const int nev = p.R1 > 0.0 ? 4 : 3;
    double k1[6];
    for (;;) {
        if (steps >= p.max_steps || (INTEG == I_DP45 && h < 1e-14)) {
            rec.status = CLOAK_RAY_STEP_LIMIT;
            break;
        }
        double y1[6], fac = 1.0, k7[6];
        if (INTEG == I_RK4) {
            rk4_step<VAR, MODE>(p, y, h, y1);
            ++steps;
        } else {
            if (!have_k1) { rhs<VAR, MODE>(p, y, k1); have_k1 = true; }
            double e6[6];
            dp45_step<VAR, MODE>(p, y, k1, h, y1, e6, k7);
            ++steps;
            if (!dp_control(y, y1, e6, tol, fac)) {
                h *= fmin(fac, 1.0);
                continue;
            }
        }
        if (INTEG == I_DP45 && nev == 4 && event_g(p, EV_METAL, y1) <= 0.0) {
            double sc = metal_chord(y[0], y[1], y1[0], y1[1], p.R1sq);
            if (sc > 0.0) {
                h *= sc;
                continue;
            }
        }
        int evh = -1;
        double sh = 1e300;
        for (int ev = 0; ev < nev; ++ev) {
            double g1 = event_g(p, ev, y1);
            if (g1 > 0.0) {
                double s = crossing<VAR, MODE, INTEG>(p, y, k1, h, g1, ev);
                if (s < sh) { sh = s; evh = ev; }
            }
        }
        if (evh < 0) {
#pragma unroll
            for (int i = 0; i < 6; ++i) y[i] = y1[i];
            t += h;
            h *= fac;
            if (INTEG == I_DP45) {
#pragma unroll
                for (int i = 0; i < 6; ++i) k1[i] = k7[i];  // first stage of the next step (FSAL)
            }
            continue;
        }
        flow<VAR, MODE, INTEG>(p, y, k1, sh, y1);
#pragma unroll
        for (int i = 0; i < 6; ++i) y[i] = y1[i];
        t += sh;
        h *= fac;
        have_k1 = false;
        if (evh == EV_METAL) {
            if (VAR == V_RADIAL && MODE == M_ORD) {  // Sect. 4: single mirror ray, c-hat along the metal normal
                double r = hypot(y[0], y[1]), nm0 = y[0] / r, nm1 = y[1] / r;
                double vn = y[3] * nm0 + y[4] * nm1;
                y[3] -= 2.0 * vn * nm0;
                y[4] -= 2.0 * vn * nm1;
                metal = true;
                continue;
            }
            rec.status = CLOAK_RAY_SINGULAR;
            break;
        }
        leave<MODE>(p, evh, y, d, k0, n_in, mat_in, metal, t, steps, rec, rgb);
        return;
    }
    // STEP_LIMIT or SINGULAR
    rec.steps = steps;
    rec.tof = t;
    rec.exit_pos[0] = y[0]; rec.exit_pos[1] = y[1]; rec.exit_pos[2] = y[2];
    set_vec(rec.exit_dir, d);
}

}  // namespace ck
