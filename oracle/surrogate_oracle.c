/*
 * surrogate_oracle.c -- plain FP64 statement of the learned surrogate (see
 * surrogate_oracle.h).  TEST INFRASTRUCTURE ONLY.
 *
 * Plain loops, one sample at a time, no blocking or reordering: the reader can
 * check every formula by eye.
 */
#include "surrogate_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

double orc_gelu(double x) {
    const double c = sqrt(2.0 / PI);
    return 0.5 * x * (1.0 + tanh(c * (x + 0.044715 * x * x * x)));
}

/* d/dx of 0.5 x (1 + tanh(u)), u = c (x + 0.044715 x^3):
 * 0.5 (1 + tanh u) + 0.5 x (1 - tanh^2 u) c (1 + 3 * 0.044715 x^2) */
double orc_gelu_grad(double x) {
    const double c = sqrt(2.0 / PI);
    double u = c * (x + 0.044715 * x * x * x);
    double th = tanh(u);
    return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th * th) * c * (1.0 + 3.0 * 0.044715 * x * x);
}

long orc_mlp_nparams(int nl, const int *dims) {
    long n = 0;
    for (int l = 0; l < nl; ++l) n += (long)dims[l + 1] * dims[l] + dims[l + 1];
    return n;
}

static int max_width(int nl, const int *dims) {
    int w = 0;
    for (int l = 0; l <= nl; ++l)
        if (dims[l] > w) w = dims[l];
    return w;
}

/* one sample through the network; z[l] and a[l] receive the pre-activation of layer l
 * and the input of layer l (a[0] = x), each max-width long */
static void forward_one(int nl, const int *dims, const double *params, const double *x, double *z, double *a,
                        double *y) {
    int w = max_width(nl, dims);
    for (int i = 0; i < dims[0]; ++i) a[i] = x[i];
    const double *p = params;
    for (int l = 0; l < nl; ++l) {
        const double *W = p, *b = p + (long)dims[l + 1] * dims[l];
        const double *in = a + (long)l * w;
        double *zl = z + (long)l * w;
        for (int o = 0; o < dims[l + 1]; ++o) {
            double s = b[o];
            for (int i = 0; i < dims[l]; ++i) s += W[(long)o * dims[l] + i] * in[i];
            zl[o] = s;
        }
        if (l < nl - 1) {
            double *next = a + (long)(l + 1) * w;
            for (int o = 0; o < dims[l + 1]; ++o) next[o] = orc_gelu(zl[o]);
        } else {
            for (int o = 0; o < dims[l + 1]; ++o) y[o] = zl[o];
        }
        p += (long)dims[l + 1] * dims[l] + dims[l + 1];
    }
}

void orc_mlp_forward(int nl, const int *dims, const double *params, long n, const double *x, double *y) {
    if (nl <= 0) return;
    int w = max_width(nl, dims);
    double *z = malloc(sizeof(double) * (size_t)w * nl);
    double *a = malloc(sizeof(double) * (size_t)w * nl);
    for (long s = 0; s < n; ++s) forward_one(nl, dims, params, x + s * dims[0], z, a, y + s * dims[nl]);
    free(z);
    free(a);
}

void orc_mlp_backward(int nl, const int *dims, const double *params, long n, const double *x, const double *dy,
                      double *grad) {
    if (nl <= 0) return;
    int w = max_width(nl, dims);
    long np = orc_mlp_nparams(nl, dims);
    double *z = malloc(sizeof(double) * (size_t)w * nl);
    double *a = malloc(sizeof(double) * (size_t)w * nl);
    double *y = malloc(sizeof(double) * (size_t)dims[nl]);
    double *delta = malloc(sizeof(double) * (size_t)w);
    double *prev = malloc(sizeof(double) * (size_t)w);
    long *off = malloc(sizeof(long) * (size_t)nl);
    long o_acc = 0;
    for (int l = 0; l < nl; ++l) {
        off[l] = o_acc;
        o_acc += (long)dims[l + 1] * dims[l] + dims[l + 1];
    }
    memset(grad, 0, sizeof(double) * (size_t)np);
    for (long s = 0; s < n; ++s) {
        forward_one(nl, dims, params, x + s * dims[0], z, a, y);
        /* the output layer is affine: dL/dz of the last layer is dy */
        for (int o = 0; o < dims[nl]; ++o) delta[o] = dy[s * dims[nl] + o];
        for (int l = nl - 1; l >= 0; --l) {
            const double *W = params + off[l];
            double *gW = grad + off[l], *gb = grad + off[l] + (long)dims[l + 1] * dims[l];
            const double *in = a + (long)l * w;
            for (int o = 0; o < dims[l + 1]; ++o) {
                gb[o] += delta[o];
                for (int i = 0; i < dims[l]; ++i) gW[(long)o * dims[l] + i] += delta[o] * in[i];
            }
            if (l == 0) break;
            /* back through W_l, then through the GELU of layer l-1 */
            const double *zp = z + (long)(l - 1) * w;
            for (int i = 0; i < dims[l]; ++i) {
                double s2 = 0.0;
                for (int o = 0; o < dims[l + 1]; ++o) s2 += W[(long)o * dims[l] + i] * delta[o];
                prev[i] = s2 * orc_gelu_grad(zp[i]);
            }
            for (int i = 0; i < dims[l]; ++i) delta[i] = prev[i];
        }
    }
    free(z);
    free(a);
    free(y);
    free(delta);
    free(prev);
    free(off);
}

double orc_sur_loss(int stage, long n, const double *y, const double *t, const double *mask, double *dy) {
    static const double wgt[4] = {1.0, 1.0, 1.0, 0.1};
    double L = 0.0;
    for (long i = 0; i < n * ORC_SUR_OUT; ++i) dy[i] = 0.0;
    for (long i = 0; i < n; ++i) {
        const double *yi = y + i * ORC_SUR_OUT, *ti = t + i * ORC_SUR_OUT;
        double *di = dy + i * ORC_SUR_OUT;
        if (stage == 1) {
            for (int j = 0; j < 4; ++j) {
                double e = yi[j] - ti[j];
                L += mask[i] * wgt[j] * e * e / (double)n;
                di[j] = 2.0 * mask[i] * wgt[j] * e / (double)n;
            }
        } else {
            double e = yi[4] - ti[4];
            L += fabs(e) / (double)n;
            di[4] = (e > 0.0 ? 1.0 : (e < 0.0 ? -1.0 : 0.0)) / (double)n;
        }
    }
    return L;
}

void orc_adam_step(long n, double *p, const double *g, double *m, double *v, long step, double lr, double beta1,
                   double beta2, double eps) {
    double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
    for (long i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* local frame of the lateral surface at azimuth phi */
static void frame(double phi, double rh[3], double th[3]) {
    rh[0] = cos(phi); rh[1] = sin(phi); rh[2] = 0.0;
    th[0] = -sin(phi); th[1] = cos(phi); th[2] = 0.0;
}

static double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

void orc_sur_sample(uint64_t seed, uint64_t i, double R2, double H, double P[3], double d[3], int *mode,
                    int *variant) {
    const uint32_t stream = 0x53555200u;
    double u0 = orc_uniform(seed, i, stream, 0), u1 = orc_uniform(seed, i, stream, 1);
    double u2 = orc_uniform(seed, i, stream, 2), u3 = orc_uniform(seed, i, stream, 3);
    double u4 = orc_uniform(seed, i, stream, 4);
    double phi = 2.0 * PI * u1, rh[3], th[3];
    frame(phi, rh, th);
    P[0] = R2 * rh[0]; P[1] = R2 * rh[1]; P[2] = (u0 - 0.5) * H;
    /* cosine-weighted hemisphere about -r-hat: a uniform point of the unit disc lifted onto it */
    double rho = sqrt(u2), ang = 2.0 * PI * u3;
    double dr = -sqrt(1.0 - u2), dt = rho * cos(ang), dz = rho * sin(ang);
    for (int k = 0; k < 3; ++k) d[k] = dr * rh[k] + dt * th[k];
    d[2] = dz;
    int bits = (int)(u4 * 4.0);
    *mode = bits & 1;
    *variant = bits >> 1;
}

/* azimuth in [0, 2 pi) and the local direction components (d_r, d_theta, d_z) */
static double entry_local(const double P[3], const double d[3], double *dr, double *dt, double *dz) {
    double phi = atan2(P[1], P[0]);
    if (phi < 0.0) phi += 2.0 * PI;
    double rh[3], th[3];
    frame(phi, rh, th);
    *dr = dot(d, rh);
    *dt = dot(d, th);
    *dz = d[2];
    return phi;
}

void orc_sur_features(double R1, double R2, double H, int variant, int mode, const double P[3], const double d[3],
                      double x[7]) {
    double dr, dt, dz;
    double phi = entry_local(P, d, &dr, &dt, &dz);
    x[0] = P[2] / (0.5 * H);
    x[1] = phi / PI - 1.0;
    x[2] = asin(dz) / (0.5 * PI);
    x[3] = atan2(dt, -dr) / (0.5 * PI);
    x[4] = 2.0 * mode - 1.0;
    x[5] = 2.0 * variant - 1.0;
    x[6] = R1 / R2;
}

int orc_sur_targets(double R2, double H, const double P[3], const double d[3], const orc_record *rec, double t[4]) {
    if (rec->status != ORC_EXITED && rec->status != ORC_HIT_METAL_EXITED) return 0;
    double re = hypot(rec->exit_pos[0], rec->exit_pos[1]);
    if (fabs(re - R2) > 1e-9 * R2 || !(fabs(rec->exit_pos[2]) < 0.5 * H)) return 0;
    double dr, dt, dz;
    double phi = entry_local(P, d, &dr, &dt, &dz);
    double beta = atan2(dt, -dr);
    double psi = atan2(rec->exit_pos[1], rec->exit_pos[0]) - (phi + PI - 2.0 * beta);
    t[0] = (rec->exit_pos[2] - P[2]) / (2.0 * R2);
    t[1] = cos(psi);
    t[2] = sin(psi);
    t[3] = rec->tof / 4.0;
    return 1;
}

void orc_sur_reconstruct(double R2, double H, const double P[3], const double d[3], const double y[4],
                         double exit_pos[3], double exit_dir[3], double *tof) {
    double dr, dt, dz;
    double phi = entry_local(P, d, &dr, &dt, &dz);
    double beta = atan2(dt, -dr);
    double phe = phi + PI - 2.0 * beta + atan2(y[2], y[1]);
    double rh[3], th[3];
    frame(phe, rh, th);
    exit_pos[0] = R2 * rh[0];
    exit_pos[1] = R2 * rh[1];
    exit_pos[2] = P[2] + y[0] * 2.0 * R2;
    /* k_z and L_z conserved, radial component outward */
    for (int k = 0; k < 3; ++k) exit_dir[k] = -dr * rh[k] + dt * th[k];
    exit_dir[2] = dz;
    *tof = 4.0 * y[3];
}
