// surrogate.h -- the learned surrogate of the integrator (internal).
//
// A multilayer perceptron 7 -> 256 -> 256 -> 256 -> 256 -> 5 (GELU, tanh form, after each hidden layer)
// maps a ray entering the lateral surface r = R2 to its exit from that surface.  Inputs (7): entry
// height and azimuth, the two angles of the vacuum direction in the local (r, theta, z) frame,
// polarization and variant bits, R1/R2.  Outputs (5): exit height, cos and sin of the exit azimuth's
// departure from the straight line's, time of flight, and a confidence head (predicted log10 of the
// surrogate's own exit error).  The exit direction is not predicted: both media are invariant under
// rotation about the axis and translation along it, so k_z and L_z are conserved and the vacuum exit
// direction follows from the exit azimuth.
//
// Weights are BF16 with FP32 accumulation on the tensor cores (mlp_tc.cuh); FP32 master weights and
// Adam moments train on rays that the integrator itself traces.  The paper has no surrogate.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

#include "cloak.h"
#include "mlp_tc.cuh"
#include "physics.cuh"

namespace ck {

struct Queue;

constexpr int SUR_L = 5;
constexpr int SUR_IN = 7, SUR_OUT = 5, SUR_W = 256;
constexpr int SUR_TSTRIDE = 8;  // per-sample target record: t0..t3, conf target, mask, spare x2
constexpr int SUR_XSTRIDE = 8;  // per-sample feature record: x0..x6, spare
constexpr unsigned int SUR_STREAM = 0x53555200u;  // random stream id of the training set

// real and padded dimensions of layer l (W_l: out x in)
struct SurDims {
    int in, out;   // real
    int kin;       // K of the forward GEMM (in rounded up to 64)
    int nout;      // N of the forward GEMM (out rounded up to 16)
    int mw;        // rows of the weight-gradient GEMM (out rounded up to 128)
    int kb;        // K of the input-gradient GEMM (out rounded up to 64)
};
__host__ __device__ inline SurDims sur_dims(int l) {
    const int in = l == 0 ? SUR_IN : SUR_W, out = l == SUR_L - 1 ? SUR_OUT : SUR_W;
    SurDims d;
    d.in = in; d.out = out;
    d.kin = (in + 63) / 64 * 64;
    d.nout = (out + 15) / 16 * 16;
    d.mw = (out + 127) / 128 * 128;
    d.kb = (out + 63) / 64 * 64;
    return d;
}

struct SurNet {
    // parameters, FP32 master copies (W: mw x kin, zero outside out x in; b: mw)
    float *W[SUR_L], *b[SUR_L];
    float *mW[SUR_L], *vW[SUR_L], *mb[SUR_L], *vb[SUR_L];  // Adam moments
    float *gW[SUR_L], *gb[SUR_L];                          // gradients
    __nv_bfloat16 *Wb[SUR_L];   // nout x kin, B operand of the forward GEMM
    __nv_bfloat16 *WTb[SUR_L];  // kin x kb, B operand of the input-gradient GEMM
    __half *Wh[SUR_L];          // nout x kin in half precision: B operand of the fused inference kernel
    __half *bh[SUR_L];          // the biases in half precision (the fused kernel's hidden layers)
    CUtensorMap tWb[SUR_L], tWTb[SUR_L], tWh[SUR_L];
    char *arena;          // one allocation for all of the above
    size_t grad_bytes;    // the gradients are contiguous from gW[0]
    char *grad_begin;
    long long adam_step;
    double R1, R2, H;     // geometry of the training rays
    float gate;           // inference: rays whose predicted log10 error exceeds this are integrated
    int trained;
    double info[8];       // final stage-1 loss, final stage-2 loss, lateral fraction, rays, seconds, ...
    double train_ms[2];   // device time per optimizer step of stage 1 and stage 2 of the last training
    unsigned int *err;    // device GEMM error flag
    // inference scratch: inputs, outputs and gate flags for inf_rows rows (a multiple of 128); the
    // hidden activations never leave the SM (mlp_fused.cu)
    long long inf_rows;
    char *inf_arena;
    uint16_t *X;  // input pairs (hi, lo), n x 64, BF16 or FP16 as the inference precision is
    int inf_f16;  // inference operands: 0 = BF16 (the training precision, default), 1 = FP16
    float *Y;
    unsigned char *elig;
};

// lifetime and parameters (surrogate.cu)
SurNet *sur_create(double R1, double R2, double H, unsigned long long seed, const char **why);
void sur_destroy(SurNet *s);
cudaError_t sur_refresh_bf16(SurNet *s, cudaStream_t st);  // Wb / WTb / Wh / bh from the FP32 masters
// forward pass of n rows of X (input pairs, n x 64) into Y (FP32, n x 16); n % 128 == 0;
// m_count: optional device row count (rows at or beyond it are skipped tile by tile)
cudaError_t sur_forward(SurNet *s, long long n, const unsigned int *m_count, cudaStream_t st);
// the same as one persistent tcgen05 kernel (mlp_fused.cu)
cudaError_t launch_mlp_fused(SurNet *s, long long n, const unsigned int *m_count, cudaStream_t st);
cudaError_t mlp_fused_prepare();  // one-time setup on the current device (call before capturing a forward pass)
cudaError_t sur_ensure_inference(SurNet *s, long long rows);

// training data (kernels_batch.cu): n seeded rays through entry, the any-medium integrator and exit;
// writes X_all (n x SUR_XSTRIDE) and T_all (n x SUR_TSTRIDE).  q: a queue of capacity n.
cudaError_t launch_sur_data(const Params &p, long long n, unsigned long long seed, const Queue &q, float *X_all,
                            float *T_all, cudaStream_t st);

// render hooks (kernels_surrogate.cu): features of the queued rays, and the gate that finishes the
// confident ones and removes them from the integration
cudaError_t launch_sur_features(const Params &p, int mode, int spp, unsigned long long seed, const Queue &q,
                                SurNet *s, cudaStream_t st);
cudaError_t launch_sur_gate(const Params &p, int mode, int spp, unsigned long long seed, const Queue &q, SurNet *s,
                            float4 *samples, cloak_record *recs, cudaStream_t st);
// confidence targets of the training set from the current predictions Y of rows [i0, i0 + n)
cudaError_t launch_sur_conf_targets(double R2, double H, unsigned long long seed, long long i0, long long n,
                                    const float *Y, float *T_all, cudaStream_t st);

// C ABI back ends (surrogate.cu); CLOAK_* return codes, `why` receives the error text
// polls of the tensor-core kernels' bounded waits that decide a timeout (0 restores the default)
unsigned int wait_limit();
void set_wait_limit(unsigned int polls);
long long sur_nparams();  // flat FP32 parameter vector: per layer W_l (out x in, row-major), then b_l
cudaError_t sur_get_params(SurNet *s, float *host);
cudaError_t sur_set_params(SurNet *s, const float *host);  // also clears the Adam state
int sur_forward_rows(SurNet *s, const float *dev_x, long long n, float *dev_y, cudaStream_t st, std::string &why);
int sur_batch_grad(SurNet *s, const float *dev_x, const float *dev_t, long long n, int stage, double lr,
                   float *host_grad, cudaStream_t st, std::string &why);
int sur_train(SurNet *s, const Params &p, long long n, unsigned long long seed, int epochs, cudaStream_t st,
              std::string &why);
int sur_save(SurNet *s, const char *path, std::string &why);
int sur_load(SurNet *s, const char *path, std::string &why);

struct ViewDev;
struct SurRenderCtx {
    SurNet *s;
    Params p;
    int mode, spp;
    unsigned long long seed;
    float4 *samples;
    cloak_record *recs;
    long long cap;
    // batched render: the device view table (mode, variant and camera ray per queued ray); null for one image
    const ViewDev *views = nullptr;
    int nviews = 0;
};
cudaError_t sur_render_hook(void *ctx, const Queue &q, cudaStream_t st);  // a WfHook function
cudaError_t launch_sur_features_batch(const Params &p, const ViewDev *views, int nviews, int spp,
                                      unsigned long long seed, const Queue &q, SurNet *s, cudaStream_t st);
cudaError_t launch_sur_gate_batch(const Params &p, const ViewDev *views, int nviews, int spp, unsigned long long seed,
                                  const Queue &q, SurNet *s, float4 *samples, cudaStream_t st);

}  // namespace ck
