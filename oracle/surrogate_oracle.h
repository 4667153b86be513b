/*
 * surrogate_oracle.h -- plain CPU FP64 statement of the learned surrogate of the
 * cloak ray tracer: a small multilayer perceptron that maps the state of a ray
 * entering the lateral surface r = R2 to its exit from that surface.
 *
 * TEST INFRASTRUCTURE ONLY, like cloak_oracle.h: only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  The CUDA path
 * shares no code, header or constant table with it.
 *
 * The paper has no surrogate; what it fixes, and what this file relies on, is
 * the symmetry of both media (Eqs. 14, 15): invariance under rotation about the
 * axis and under translation along it.  Hence k_z and L_z = (x cross k)_z are
 * conserved from the entry face to the exit face (Sect. 2 equations of motion,
 * Sect. 3 tangential continuity), and for a ray that enters and leaves through
 * the lateral surface the vacuum exit direction follows from the exit azimuth
 * alone: in the local (r, theta, z) frame it is the entry direction with the
 * sign of its radial component flipped.
 *
 * Network: n_in -> hidden ... -> n_out, GELU (tanh form) after every hidden
 * layer, affine output.  Parameters are stored per layer as W_l (row-major,
 * dims[l+1] x dims[l]) followed by b_l (dims[l+1]).
 */
#ifndef SURROGATE_ORACLE_H
#define SURROGATE_ORACLE_H

#include <stdint.h>

#include "cloak_oracle.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SUR_IN = 7, ORC_SUR_OUT = 5 };

/* GELU, tanh form: 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))), and its derivative */
double orc_gelu(double x);
double orc_gelu_grad(double x);

/* number of parameters of the network with nl layers and widths dims[0..nl] */
long orc_mlp_nparams(int nl, const int *dims);

/* y[n x dims[nl]] = network(x[n x dims[0]]) */
void orc_mlp_forward(int nl, const int *dims, const double *params, long n, const double *x, double *y);

/* grad (layout of params) = d/dparams of sum_i sum_j dy[i][j] * y[i][j] (back-propagation) */
void orc_mlp_backward(int nl, const int *dims, const double *params, long n, const double *x,
                      const double *dy, double *grad);

/* Training loss of the surrogate and its gradient with respect to the outputs.
 * stage 1: mean over samples of mask_i * sum_{j<4} w_j (y_ij - t_ij)^2, w = (1, 1, 1, 0.1)
 * stage 2: mean over samples of |y_i4 - t_i4|   (confidence head, L1)
 * y, t: n x 5; dy receives n x 5. */
double orc_sur_loss(int stage, long n, const double *y, const double *t, const double *mask, double *dy);

/* One Adam step (Kingma & Ba 2015) with bias correction; step counts from 1. */
void orc_adam_step(long n, double *p, const double *g, double *m, double *v, long step, double lr,
                   double beta1, double beta2, double eps);

/* Training ray number i of a seeded set: entry point uniform on the lateral surface
 * (z ~ U(-H/2, H/2), phi ~ U(0, 2 pi)), direction cosine-weighted about the inward
 * normal, polarization mode and variant uniform.  Random numbers are
 * orc_uniform(seed, i, 0x53555200, dim) for dim = 0..4. */
void orc_sur_sample(uint64_t seed, uint64_t i, double R2, double H, double P[3], double d[3], int *mode,
                    int *variant);

/* The 7 network inputs of a ray entering at P (on r = R2) with vacuum direction d:
 * z/(H/2), phi/pi - 1, asin(d_z)/(pi/2), atan2(d_theta, -d_r)/(pi/2), 2 mode - 1,
 * 2 variant - 1, R1/R2. */
void orc_sur_features(double R1, double R2, double H, int variant, int mode, const double P[3], const double d[3],
                      double x[7]);

/* Regression targets of a traced ray (outputs 0..3): (exit z - entry z) / (2 R2), cos psi,
 * sin psi, tof/4, psi = exit azimuth - (entry azimuth + pi - 2 beta) (the azimuth the straight
 * line would reach).  All four are functions of the direction angles, mode and variant alone:
 * the media are invariant under translation along the axis and rotation about it.  Returns 1
 * if the ray left through the lateral surface (the targets are defined), else 0. */
int orc_sur_targets(double R2, double H, const double P[3], const double d[3], const orc_record *rec,
                    double t[4]);

/* Exit of a ray from predicted outputs y[0..3]: point on r = R2, vacuum direction by the
 * conservation of k_z and L_z, time of flight. */
void orc_sur_reconstruct(double R2, double H, const double P[3], const double d[3], const double y[4],
                         double exit_pos[3], double exit_dir[3], double *tof);

#ifdef __cplusplus
}
#endif
#endif
