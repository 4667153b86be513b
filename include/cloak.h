/*
 * cloak.h -- C ABI of the GB300 (sm_103a) renderer for light rays through the
 * non-magnetic uniaxial cylindrical invisibility cloaks of Halimeh & Wegener,
 * "Photorealistic ray tracing of free-space invisibility cloaks made of
 * uniaxial dielectrics" (arXiv:1209.6038).
 *
 * Conventions (all entry points):
 *   - Units c0 = omega = 1: a vacuum ray has |k| = |v| = 1, time t is the
 *     integration variable of Eq. 2 / Eq. 8 and also the time of flight.
 *   - The cylinder axis is +z.  The cloak shell is R1 <= r <= R2,
 *     |z| <= height/2; a metal cylinder fills r <= R1, |z| <= height/2.
 *   - Device buffers are allocated and owned by the caller; the library
 *     writes them asynchronously on the caller's CUDA stream (`cuda_stream`
 *     is a cudaStream_t passed as void*, NULL = legacy default stream).
 *   - The library owns only the handle and its internal scratch memory.
 *   - Every call returns CLOAK_OK or an error code and never aborts; the
 *     reason of the last failure on the calling thread is returned by
 *     cloak_last_error().  Argument errors are detected before any launch;
 *     launch errors are reported as CLOAK_ECUDA.
 *   - A handle is not thread-safe: serialise calls on one handle.
 */
#ifndef CLOAK_H
#define CLOAK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cloak cloak_t; /* opaque handle */

/* cloak variants */
enum {
    CLOAK_RADIAL = 0,                /* Eq. 14: optic axis along r-hat (Sect. 4) */
    CLOAK_AZIMUTHAL = 1,             /* Eq. 15: optic axis along theta-hat (Sect. 4) */
    CLOAK_TEST_UNIAXIAL_CONST = 100  /* homogeneous uniaxial medium of Eq. 1 with a fixed optic axis
                                        filling r <= R2 (requires R1 = 0); for interface tests */
};
/* polarization mode traced through the medium (Sect. 2) */
enum { CLOAK_POL_ORDINARY = 0, CLOAK_POL_EXTRAORDINARY = 1 };
/* integrators for Eq. 2 / Eq. 8 */
enum {
    CLOAK_RK4 = 0,  /* classical fourth-order Runge-Kutta at a fixed step h in t (Sect. 4) */
    CLOAK_DP45 = 1  /* Dormand-Prince 5(4), adaptive, tolerance tol */
};
/* arithmetic of the integrator */
enum {
    CLOAK_FP64 = 0,  /* all of the path in FP64 */
    CLOAK_MIXED = 1,   /* RK stepping in FP32 (right-hand sides, stage combinations, step control) with
                          float-float state accumulation; whole steps in FP64 where r < R1 + 0.02; entry
                          and exit interface solves in FP64 (wavefront schedule only) */
    CLOAK_MIXED_FF = 2, /* as CLOAK_MIXED with the steps of the band in double-float (pairs of FP32
                          numbers, ~48 significant bits) instead of FP64 */
    CLOAK_SURROGATE = 3 /* learned surrogate (see cloak_surrogate_train) for rays that enter through the
                          lateral surface and whose predicted error passes the gate; the FP64 integrator
                          for all others (wavefront schedule: cloak_render, cloak_render_records,
                          cloak_render_batch) */
};
/* kernel schedule */
enum {
    CLOAK_SCHED_PLAIN = 0,     /* one thread per pixel, whole path in one kernel (FP64 comparator) */
    CLOAK_SCHED_WAVEFRONT = 1  /* camera/entry, compacted integration and exit/shade stages */
};
/* return codes */
enum { CLOAK_OK = 0, CLOAK_EINVAL = 1, CLOAK_ENOMEM = 2, CLOAK_ECUDA = 3, CLOAK_ETIMEOUT = 4, CLOAK_ESTATE = 5 };
/* per-ray status in cloak_record.status */
enum {
    CLOAK_RAY_MISSED = 0,           /* the camera ray never meets the cylinder */
    CLOAK_RAY_EXITED = 1,           /* went through the cloak and left it */
    CLOAK_RAY_HIT_METAL_EXITED = 2, /* mirrored at r = R1 (radial ordinary rays, Sect. 4), then left */
    CLOAK_RAY_NO_TRANSMISSION = 3,  /* the chosen mode is evanescent at the entry face */
    CLOAK_RAY_TIR = 4,              /* total internal reflection at the exit face (weight 0) */
    CLOAK_RAY_STEP_LIMIT = 5,       /* max_steps reached or adaptive step below 1e-14 */
    CLOAK_RAY_SINGULAR = 6,         /* reached r = R1 in a mode without a mirror rule */
    CLOAK_RAY_METAL_CAP = 7         /* mirrored off a metal end disc (r <= R1) from outside */
};

/* 80-byte per-ray (per-sample) result */
typedef struct cloak_record {
    double exit_pos[3]; /* start point of the final vacuum ray */
    double exit_dir[3]; /* unit direction of the final vacuum ray */
    double tof;         /* time spent inside the cloak */
    double weight;      /* T_in * T_out from Eq. 12 along the physical direction of light
                           (unpolarised source); 1 for rays that miss or hit a metal disc */
    int32_t tile_id;    /* (face << 20) | (i << 10) | j of the room tile hit, -1 for none */
    int32_t status;     /* CLOAK_RAY_* */
    int32_t steps;      /* integrator step attempts */
    int32_t mode;       /* CLOAK_POL_* traced */
} cloak_record;

/* Create a cloak.  variant: CLOAK_RADIAL / CLOAK_AZIMUTHAL (Eqs. 14, 15 with
 * a = R1, b = R2; needs 0 < R1 < R2) or CLOAK_TEST_UNIAXIAL_CONST (needs
 * R1 = 0).  height > 0.  Defaults: camera at (5,0,0) looking at the origin,
 * 60 deg horizontal field of view, 128x96; RK4 with h = 1e-3, FP64,
 * max_steps = 1e6; plain schedule; room seed 0.
 * Returns NULL on error (see cloak_last_error()).  Needs a current CUDA device. */
cloak_t *cloak_create(int variant, double R1, double R2, double height);
/* Release the handle and its scratch memory (synchronises the device). NULL is ignored. */
void cloak_destroy(cloak_t *h);
/* Message of the last failed call on this thread ("" if none).  Owned by the library. */
const char *cloak_last_error(void);

/* Pinhole camera: eye, look-at target, up vector (host arrays of 3 doubles),
 * horizontal field of view in degrees (0 < hfov < 180), image size in pixels
 * (width, height >= 1, width*height <= 2^31 - 1).  Row 0 is the top row. */
int cloak_camera_set(cloak_t *h, const double eye[3], const double target[3], const double up[3], double hfov_deg,
                     int width, int height);
/* Integrator (Sect. 4 and its adaptive form): kind CLOAK_RK4 with h_or_tol = step h > 0, or CLOAK_DP45
 * with h_or_tol = tolerance > 0 (error norm max_i |err_i| / (tol + tol max(|y_i|, |y_i'|)), safety 0.9,
 * step factor in [0.2, 5], initial step 1e-3).  precision CLOAK_FP64, CLOAK_MIXED, CLOAK_MIXED_FF or
 * CLOAK_SURROGATE.
 * max_steps >= 1 bounds the step attempts of one ray. */
int cloak_set_integrator(cloak_t *h, int kind, double h_or_tol, int precision, long max_steps);
/* Medium of CLOAK_TEST_UNIAXIAL_CONST (Eq. 1): eps_o, eps_e > 0, optic axis c_hat (host, 3 doubles,
 * nonzero; normalised internally).  CLOAK_ESTATE for other variants. */
int cloak_set_test_medium(cloak_t *h, double eps_o, double eps_e, const double c_hat[3]);
/* Seed of the procedural room that stands in for the paper's scenery (checkered walls and floor,
 * 8 tiles per unit, box x,y in [-10,10], z in [-height/2, -height/2 + 10]). */
int cloak_set_scene_seed(cloak_t *h, unsigned long long seed);
/* Ray equations: CLOAK_FORM_FERMAT (default: Eq. 2 for ordinary, Eq. 8 for extraordinary rays, state
 * (x, v)) or CLOAK_FORM_HAMILTONIAN (the comparison system of Sect. 4's closing remark: state (x, k) with
 * k = M v, dx/dt = M^-1 k, dk/dt = -(1/2) k^T (grad M^-1) k; the same integrator, crossings and
 * interfaces).  The Hamiltonian form needs a radial or azimuthal handle and FP64 (precision CLOAK_FP64 or
 * CLOAK_SURROGATE); CLOAK_ESTATE otherwise. */
enum { CLOAK_FORM_FERMAT = 0, CLOAK_FORM_HAMILTONIAN = 1 };
int cloak_set_formulation(cloak_t *h, int formulation);
/* Linear polariser in front of the camera (the paper's "polarization goggles"): CLOAK_ANALYZER_NONE,
 * CLOAK_ANALYZER_RIGHT (axis along the camera's right vector) or CLOAK_ANALYZER_UP (its up vector).  With
 * one, a ray's weight is multiplied by the fraction of the vacuum wave leaving the cloak towards the
 * camera that passes it (Malus's law, the axis taken across the wave); a ray that never enters the cloak
 * keeps half of the unpolarised room light.  Applies to cloak_render, cloak_render_records,
 * cloak_render_batch and cloak_render_noalloc; cloak_trace_rays has no camera and ignores it. */
enum { CLOAK_ANALYZER_NONE = 0, CLOAK_ANALYZER_RIGHT = 1, CLOAK_ANALYZER_UP = 2 };
int cloak_set_analyzer(cloak_t *h, int analyzer);
/* Kernel schedule (CLOAK_SCHED_*).  packet: threads per block of the persistent integration kernel
 * (32, 64, 96 or 128; 0 = the precision's default: 128 for CLOAK_FP64, 64 for CLOAK_MIXED and
 * CLOAK_MIXED_FF).  steps_per_round: reserved (0): lanes refill one by one from
 * the queue, there are no compaction rounds. */
int cloak_set_schedule(cloak_t *h, int schedule, int packet, int steps_per_round);
/* Step-schedule knobs of the wavefront and batched integration (the paper has no counterpart; images and
 * records do not depend on them, only the time does): long_ray_blocks (0..64, default 4) blocks of the
 * persistent kernel, each on an SM of its own, take the slowest rays first -- those passing closest to
 * the axis; reserve_per_thread (1..8, default 1) rays are reserved for them per thread; cost_scale
 * (1..16, default 4) sets the resolution of the sort's cost buckets, bucket = cost_scale x -log2 |L_z|
 * (64 buckets).  CLOAK_EINVAL outside these ranges.  Until this call is made on a handle, CLOAK_MIXED and
 * CLOAK_MIXED_FF use their own defaults (16, 4, 3): the slow near-axis rays weigh more in their shorter
 * steps.  The autotuner (autotune.py) searches them. */
int cloak_set_schedule_tuning(cloak_t *h, int long_ray_blocks, int reserve_per_thread, double cost_scale);

/* Per-stage device timing (CUDA events on the call's stream).  on != 0 enables it for later calls.
 * cloak_stage_times waits for the last cloak_render / cloak_render_records call on this handle and
 * writes its stage durations in milliseconds: ms[0] camera rays + entry refraction, ms[1] integration
 * of Eq. 2 / Eq. 8 (the whole kernel on the plain schedule), ms[2] exit refraction + Eq. 12 weights +
 * room lookup, ms[3] per-pixel resolve (0 where a stage does not exist).  CLOAK_ESTATE if timing was
 * off or nothing was rendered since it was enabled. */
int cloak_set_stage_timing(cloak_t *h, int on);
int cloak_stage_times(cloak_t *h, float ms[4]);

/* Render one image of the chosen polarization (Sect. 4): dev_rgba is float4[width*height]
 * (bytes >= 16*width*height), RGB = mean over the spp samples of weight * colour, A = mean weight.
 * spp >= 1; one sample goes through the pixel centre, more samples are jittered from
 * splitmix64(seed, pixel, sample, dim).  polarization: CLOAK_POL_*. */
int cloak_render(cloak_t *h, int polarization, int spp, unsigned long long seed, void *dev_rgba, size_t bytes,
                 void *cuda_stream);
/* As cloak_render, but writes one cloak_record per sample: dev_records is
 * cloak_record[width*height*spp] (sample s of pixel p at p*spp + s). */
int cloak_render_records(cloak_t *h, int polarization, int spp, unsigned long long seed, void *dev_records,
                         size_t bytes, void *cuda_stream);
/* Trace n >= 0 arbitrary rays without a camera: dev_rays is double[n][6] (origin xyz, unit direction
 * xyz; origins outside the cylinder), dev_records is cloak_record[n].  Both device memory. */
int cloak_trace_rays(cloak_t *h, int polarization, const double *dev_rays, long n, void *dev_records,
                     void *cuda_stream);
/* Right-hand side of the ray equations at n >= 0 states, as the integrators evaluate it.  Fermat form
 * (default): state (x, v), result (v, dv/dt) of Eq. 8 (extraordinary) or Eq. 2 (ordinary) with the
 * Eq. 7 matrix of Eq. 14 / 15; Hamiltonian form (cloak_set_formulation): state (x, k), result
 * (M^-1 k, -1/2 k^T (grad M^-1) k).  dev_y and dev_dy are double[n][6] device memory; states must lie
 * inside the shell (R1 < r).  Radial and azimuthal handles only (CLOAK_ESTATE otherwise). */
int cloak_eval_rhs(cloak_t *h, int polarization, const double *dev_y, long n, double *dev_dy, void *cuda_stream);

/* One view of a batched render: medium (CLOAK_RADIAL or CLOAK_AZIMUTHAL, with the handle's R1, R2 and
 * height), traced polarization, pinhole camera (as cloak_camera_set) and its output, a caller-owned
 * device buffer of float4[width*height]. */
typedef struct cloak_view {
    int variant;
    int polarization;
    double eye[3], target[3], up[3];
    double hfov_deg;
    int width, height;
    void *dev_rgba;
} cloak_view;

/* Batched render (many views in one pass, Sect. 4 per ray): one camera/entry kernel over the samples
 * of all views, one device queue of entering rays ordered by expected cost and medium, ONE persistent
 * integration kernel for the rays of every view, one exit kernel and one resolve kernel writing every
 * view's image.  The launch sequence is captured in a CUDA graph the first time a batch (views, spp,
 * seed, integrator, precision, packet) is seen and replayed on later identical calls.  The handle's
 * variant must be CLOAK_RADIAL or CLOAK_AZIMUTHAL; integrator, precision and packet come from the
 * handle.  With CLOAK_SURROGATE (a trained network of the handle's geometry) the network and its gate
 * run on the whole queue before the sort and the integrator takes the rays the gate leaves; with a
 * network of another geometry every ray is integrated.  views: host array of nviews >= 1 entries (read
 * during the call); total samples sum(width*height*spp) <= 2^31 - 1.  Scratch: about 128 bytes per
 * sample, owned by the handle (plus the network's inference buffers, 208 bytes per sample).
 * Every view's output is written on cuda_stream.  With stage timing on, cloak_stage_times reports the
 * stages of the last batch (events recorded inside the graph). */
int cloak_render_batch(cloak_t *h, const cloak_view *views, int nviews, int spp, unsigned long long seed,
                       void *cuda_stream);

/* BF16 tensor-core GEMM of the learned surrogate (tcgen05 with a TMEM accumulator, operands staged by
 * TMA with 128-byte swizzle): C = A B^T with A[M x K] and B[N x K] row-major BF16 device arrays
 * (16-byte aligned) and C[M x N] row-major FP32.  M % 128 == 0; N % 16 == 0 with 16 <= N <= 256;
 * K % 64 == 0.  Synchronises cuda_stream; CLOAK_ETIMEOUT if a bounded wait inside the kernel expired.
 * The paper has no counterpart: it serves the learned surrogate of the exit state. */
int cloak_mlp_gemm(const void *dev_a, const void *dev_b, float *dev_c, int M, int N, int K, void *cuda_stream);

/* Bounded waits of the tensor-core kernels (the surrogate's GEMMs and fused forward pass; the paper has no
 * counterpart).  Every mbarrier wait of those kernels polls at most a bounded number of times; when a wait
 * that the kernel's progress depends on runs out, the kernel sets its error flag, lets the MMAs and copies
 * it has in flight complete (those waits keep the default bound), frees its TMEM and returns:
 * cloak_mlp_gemm, cloak_surrogate_forward, _step and _train then return CLOAK_ETIMEOUT, and a
 * CLOAK_SURROGATE render leaves every ray to the FP64 integrator (the image is the integrator's).
 * polls: the bound for all later launches in this process (default 2^22 polls, 0 restores it).  A small
 * bound makes the waits run out on purpose -- this is how the timeout path is tested.  CLOAK_EINVAL
 * outside [0, 2^32 - 1]. */
int cloak_set_wait_limit(long long polls);

/* FMA throughput microbenchmark (the measured denominators of the ALU rooflines; the paper has no
 * counterpart).  Launches `blocks` x `threads` threads (threads a multiple of 32 in [32, 256]), each
 * running 8 independent fused multiply-add chains for 8 x iters steps, in FP64 (precision CLOAK_FP64)
 * or FP32 (CLOAK_MIXED) on cuda_stream, and returns at once; *flops (host) receives the floating-point
 * operations the launch performs (2 per FMA).  The caller times the launch (CUDA events on the same
 * stream).  dev_sink: device memory of blocks x threads elements of the chosen type (never written in
 * practice; it keeps the chains live).  CLOAK_EINVAL on bad arguments, CLOAK_ECUDA if the launch fails. */
int cloak_fma_peak(int precision, int blocks, int threads, long long iters, void *dev_sink, double *flops,
                   void *cuda_stream);

/* Allocation-free render.  The paper has no counterpart: this is a service for callers that may not
 * allocate device memory -- processes whose device memory is owned entirely by another allocator
 * (a framework's caching pool), latency-critical render loops that cannot afford the device-wide
 * synchronisation of cudaMalloc / cudaFree, or programs that must not grow their footprint after
 * start-up.  It renders exactly like cloak_render on the wavefront schedule (the handle's camera,
 * integrator and precision), but its queue and per-sample buffer live in one fixed device array
 * inside the library (128 MiB + 4 KiB, held on every GPU that loads the library until the process
 * exits) instead of handle scratch, and it calls no cudaMalloc, cudaFree or allocating routine.
 * Limit: width*height*spp <= 1048576 samples, else CLOAK_EINVAL before any launch.  The caller still
 * passes the output (dev_rgba, float4[width*height], bytes >= 16*width*height).  The first call on a
 * device resolves the array's device address (cudaGetSymbolAddress) and caches it for the life of the
 * process; make that first call before any stream capture, and do not use this entry point again on a
 * device after cudaDeviceReset (the cached address belongs to the old context).  Stage timing
 * (cloak_set_stage_timing) does not cover this call.  All calls share the array, which keeps the last
 * call's contents: calls whose GPU work overlaps (other streams, other threads, other handles) race on it
 * and must be serialised. */
int cloak_render_noalloc(cloak_t *h, int polarization, int spp, unsigned long long seed, void *dev_rgba,
                         size_t bytes, void *cuda_stream);

/* Panels of the paper's figures (Figs. 1, 2), with the handle's camera and room, written on cuda_stream
 * into dev_rgba (float4[width*height], bytes >= 16*width*height; RGB = mean over samples of weight x room
 * colour, A = mean weight):
 *   CLOAK_PANEL_ROOM         (a) the room without the cylinder
 *   CLOAK_PANEL_METAL        (b) the bare metal cylinder of radius R1 and height H (a mirror, reflectance 1)
 *   CLOAK_PANEL_UNPOLARIZED  (c) the cloak in unpolarised light: per sample the sum of the ordinary and the
 *                            extraordinary contribution (each weighted by its Eq. 12 factors), a ray that
 *                            never enters the shell counted once.  Both polarisations run in one batched
 *                            render (radial or azimuthal handle; the handle's integrator and precision).
 * The paper's images show the cylinder axis horizontal, here it is vertical (+z): its "vertical" goggles
 * (d), across the cylinder axis, are CLOAK_PANEL_POLARIZER_RIGHT at elevation 0; its "horizontal" ones (e)
 * are CLOAK_PANEL_POLARIZER_UP.
 *   CLOAK_PANEL_TOF          time-of-flight difference image (Sect. 4, the TOF images of its Ref. [10]):
 *                            per sample, the time (c0 = 1: vacuum path lengths plus the time of flight
 *                            inside the cloak) the light takes from the room point the sample sees to the
 *                            camera, minus the time from the room point the straight camera ray sees
 *                            without the cylinder.  Per pixel float4: x = intensity-weighted mean over
 *                            the samples of both polarizations (a ray that never enters the shell counted
 *                            once), y = of the ordinary and z = of the extraordinary light alone,
 *                            w = summed weight (mean over samples); 0 where no light arrives.  The
 *                            weights include the handle's camera polariser (cloak_set_analyzer). */
enum {
    CLOAK_PANEL_ROOM = 0, CLOAK_PANEL_METAL = 1, CLOAK_PANEL_UNPOLARIZED = 2,
    CLOAK_PANEL_POLARIZER_RIGHT = 3, /* (d): as (c) seen through a linear polariser along the camera's right vector */
    CLOAK_PANEL_POLARIZER_UP = 4,    /* (e): ... along the camera's up vector */
    CLOAK_PANEL_TOF = 5              /* time-of-flight difference image (see above) */
};
/* First-order reflections (Sect. 4: the paper keeps them and omits higher orders) in the panels
 * CLOAK_PANEL_UNPOLARIZED and CLOAK_PANEL_POLARIZER_*: on = 1 adds, per sample that enters the shell,
 * (a) room light that the outer surface reflects into the camera (by reciprocity, the mean over the
 * camera-side polarisations of the reflectance of a vacuum wave along the camera ray; counted once), and
 * (b) for each traced polarization, light that travelled inside as the ordinary or the extraordinary wave
 * and reflected at the camera-backward ray's far face into the traced wave (Sect. 3's double reflection;
 * reflection coefficients of the 4x4 field solve, also under total internal reflection), each reflected
 * ray traced through the cloak to its own exit and refracted out without further reflection.  The
 * reflected rays run through a second queue and integration launch after the batched render.  on = 0
 * (default): refraction only.  The TOF panel, cloak_render and the records ignore it. */
int cloak_set_reflections(cloak_t *h, int on);
int cloak_render_panel(cloak_t *h, int panel, int spp, unsigned long long seed, void *dev_rgba, size_t bytes,
                       void *cuda_stream);

/* ---- learned surrogate of the exit state (the paper has none) -------------------------------------
 * A multilayer perceptron 7 -> 256 -> 256 -> 256 -> 256 -> 5 (GELU, tanh form; BF16 operands, FP32
 * accumulation on the tensor cores; FP16 inference on request, cloak_surrogate_set_precision) maps a
 * ray entering the lateral surface r = R2 -- entry height and
 * azimuth, the two angles of its vacuum direction in the local (r, theta, z) frame, polarization bit,
 * variant bit, R1/R2 -- to its exit through r = R2: exit height, cos and sin of the exit azimuth's
 * departure from the straight line's, time of flight, and a confidence output (predicted log10 of its
 * own exit error: the larger of the exit-direction angle and the exit-point distance / R2).  The exit
 * direction follows from the exit azimuth because both media conserve k_z and L_z (rotation and
 * translation symmetry of Eqs. 14, 15).  The model belongs to the handle; its geometry is the handle's
 * at training time, and renders of another geometry integrate every ray (outside the support). */

/* Train the handle's surrogate on n_rays rays that the handle's integrator traces (FP64 or mixed as
 * set; both variants and polarizations, entry points uniform on the lateral surface, directions
 * cosine-weighted about the inward normal, splitmix64 stream of `seed`).  Stage 1: `epochs` passes of
 * Adam on the regression outputs (masked squared error; lateral exits only); stage 2: epochs / 3 passes
 * on the confidence output alone (L1 against the stage-1 model's log10 exit error; 0 for rays that do
 * not leave laterally).  n_rays in [19456, 2^31 - 1].  Allocates about 170 bytes per ray for the
 * duration of the call; synchronises cuda_stream. */
int cloak_surrogate_train(cloak_t *h, long n_rays, unsigned long long seed, int epochs, void *cuda_stream);
/* Checkpoint: the FP32 weights, the Adam moments, the geometry, the gate and the training summary as a
 * flat binary file with a header ("CKSURR01").  load replaces the handle's surrogate. */
int cloak_surrogate_save(cloak_t *h, const char *path);
int cloak_surrogate_load(cloak_t *h, const char *path);
/* Gate of CLOAK_SURROGATE renders: a ray keeps the surrogate's exit when its predicted log10 error is
 * <= max_log10_err (default -3) and its predicted exit height is inside the cylinder. */
int cloak_surrogate_set_gate(cloak_t *h, double max_log10_err);
/* Training summary (host, 8 doubles): final stage-1 loss, final stage-2 loss, lateral-exit fraction of
 * the training rays, rays, seconds in total, seconds tracing the training rays, optimiser steps, batch
 * size.  CLOAK_ESTATE without a trained surrogate. */
int cloak_surrogate_info(cloak_t *h, double info[8]);
/* Operand precision of the surrogate's inference (renders with CLOAK_SURROGATE and
 * cloak_surrogate_forward): fp16 = 0, the default, evaluates the network with BF16 weights, input pairs
 * and activations like its training; fp16 = 1 in FP16 (weights, input pairs and activations: 11
 * significant bits instead of 8, slightly faster).  In both the accumulation is FP32 and the hidden
 * layers' bias and GELU are computed in half-precision pairs.  The setting belongs to the handle's network
 * (kept across cloak_surrogate_load); a handle without a surrogate gets one with seeded weights first.
 * The paper has no counterpart. */
int cloak_surrogate_set_precision(cloak_t *h, int fp16);
/* Device timing of the last cloak_surrogate_train (host, 4 doubles): milliseconds per optimizer step of
 * stage 1 (batch gather, forward, loss, backward and Adam over one batch, as the training replays it in a
 * CUDA graph; CUDA events around the stage), the same for stage 2, the algorithmic tensor-core flops of a
 * stage-1 step (2 x the multiply-adds of the forward, backward-data and weight-gradient GEMMs without
 * padding), and the batch size.  CLOAK_ESTATE if the handle's surrogate was not trained here. */
int cloak_surrogate_train_timing(cloak_t *h, double out[4]);
/* Parameters as one flat FP32 host vector of n = 200709 values (per layer: W_l, out x in row-major,
 * then b_l).  set = 0 copies them into host; set = 1 loads host into the network and clears the Adam
 * state.  A handle without a surrogate gets one with seeded initial weights first. */
int cloak_surrogate_params(cloak_t *h, float *host, long n, int set);
/* Network outputs for n input rows: dev_x FP32 [n x 7] (device), dev_y FP32 [n x 5] (device).
 * Synchronises cuda_stream. */
int cloak_surrogate_forward(cloak_t *h, const float *dev_x, long n, float *dev_y, void *cuda_stream);
/* One training step on a given batch: dev_x FP32 [n x 7], dev_t FP32 [n x 8] (targets of outputs 0..3,
 * confidence target, mask, two unused), n % 128 == 0.  stage 1 or 2 selects the loss (see train).
 * host_grad (nullable): receives the gradient of the mean loss, flat layout of cloak_surrogate_params.
 * lr > 0 also applies one Adam step (beta 0.9 / 0.999, eps 1e-8) with that learning rate.
 * Synchronises cuda_stream. */
int cloak_surrogate_step(cloak_t *h, const float *dev_x, const float *dev_t, long n, int stage, double lr,
                         float *host_grad, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* CLOAK_H */
