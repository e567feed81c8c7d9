// Internal interface between the C-ABI layer (api.cu) and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sdfnn {

constexpr int kMaxHidden = 4;
constexpr int kMaxLevels = 8;

// Device view of one prepared network (all pointers are device memory).
struct NetView {
    int in_dim, width, n_hidden;
    const float* w0;               // [width][in_dim], folded by omega0
    const float* b0;               // [width], folded
    const float* wt[kMaxHidden];   // FP32 hidden weights, transposed: wt[i][k * width + n] = W_i[n][k], folded
    const float* bh[kMaxHidden];   // [width], folded
    const float* wout;             // [width]
    float bout;
    const uint8_t* wbf;            // 16-bit hidden weights in the 128-byte-swizzled K-major layout
    const uint8_t* wbf_lo;         // 16-bit rounding of (weight - head), same layout, or NULL
    uint32_t wbf_layer_bytes;      // bytes per hidden layer in wbf
    int rows_pad;                  // rows per 128-byte K block in wbf (max(width, 128), zero padded)
    int op_f16;                    // tensor-core operand type of wbf: 1 = IEEE half, 0 = bfloat16
    // E4M3 networks (op_fp8 = 1): wbf holds the hidden weights as E4M3 bytes
    // (128-element K blocks) scaled by q_w[l]; wout_q the output row as a head
    // (W bytes, scaled by q_o) and a remainder (W bytes, scaled by 16 q_o);
    // q_g[l] is the scale of the tangents stored after layer l (0 = input layer).
    int op_fp8;
    float q_w[kMaxHidden];
    float q_g[kMaxHidden + 1];
    float q_o;
    const uint8_t* wout_q;
};

// The per-unit FP32 parameters of a width-64 network that the trace kernel
// reads for every ray and step, carried in the launch parameters so that the
// kernel loads them through the constant cache instead of shared memory (a
// float4 that all lanes load from one shared address costs extra shared-memory
// wavefronts; a uniform constant load does not).  Layer 0 on
// unit pairs p = (2p, 2p+1): w0[2p] = (w_x0, w_x1, w_y0, w_y1) and
// w0[2p+1] = (w_z0, w_z1, b_0, b_1), the bias holding w_t * time when the
// time is one scalar for all rays; bl = bias of the last hidden layer and
// wo = the output weights, four units per float4.  Filled by the host for
// width-64 networks only.
constexpr int kConstWidth = 64;
struct TraceConsts {
    float4 w0[kConstWidth];
    float4 bl[kConstWidth / 4];
    float4 wo[kConstWidth / 4];
};

// One level of Alg. 1 as launched.
struct LevelArgs {
    TraceConsts k;    // width-64 networks (see TraceConsts)
    NetView net;
    float d;          // t = f(p) - d
    float scale;      // step = scale * t
    int cap;          // iteration cap of this level
    int is_last;      // last level: the hit decision is taken here
    float time;       // 4th network input of every ray when ray_time is NULL
    const float* ray_time;  // 4th network input per ray (n floats, 4-input networks), or NULL
    int tiles;        // ray tiles per CTA of the tensor-core kernel (0: the launcher's choice)
    float eps, box_lo, box_hi;
    // rays and outputs (SoA, n items)
    const float* orig;
    const float* dir;
    int64_t n;
    float* out_pos;
    float* out_t;
    uint8_t* out_hit;
    uint16_t* out_iters;
    // work lists: level 0 reads rays 0..n-1 directly; later levels read in_list[0..*in_count)
    const int32_t* in_list;
    const unsigned long long* in_count;
    int32_t* out_list;              // NULL on the last level
    unsigned long long* out_count;
    unsigned long long* grab;       // work counter, zero at launch
    int* status;
};

// Gradient / normal-mapping launch.
struct GradArgs {
    NetView net;
    float time;                     // 4th network input of every point when pt_time is NULL
    const float* pt_time;           // 4th network input per point (n floats, 4-input networks), or NULL
    const float* pts;               // SoA (3, n)
    int64_t n;
    const int32_t* list;            // NULL: points 0..n-1; else list[0..*count)
    const unsigned long long* count;
    float* out;                     // SoA (3, n)
    int normalize;                  // 1: unit normal (0 where |g| < 1e-12)
    unsigned long long* grab;       // tile counter, zero at launch
    int* status;
    // training forward of the tensor-core path (the kernel's TRAIN variant): the
    // pre-activations saved for the backward, f written beside grad f
    float* save_a0;                 // [n][width] A_0
    float* save_a;                  // A_l, hidden layers 1..k (layout: rec_a in grad_tc.cuh)
    uint2* save_h;                  // (H_l^x, H_l^y | H_l^z, 0) in the operand type (layout: rec_h)
    int64_t save_np;                // points of the record layout: n rounded up to 64
    float* out_f;                   // (n)
    const float* out_bias;          // device address of b_out
};

// Kernel launchers (return cudaError_t of the launch).
cudaError_t launch_trace_level_simt(const LevelArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_grad_simt(const GradArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_trace_level_tc(const LevelArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_grad_tc(const GradArgs& a, int num_sms, cudaStream_t s);
int trace_tiles_max(const NetView& net);  // largest `tiles` the tensor-core trace kernel accepts for net
bool tc_trace_supported(int width, int n_hidden);
// Measured throughput of the tensor-core kernels' sine on all SMs (sines per second).
cudaError_t measure_sine_rate(int num_sms, cudaStream_t s, double* sines_per_s);
// The kernels' sine and cosine at x[0..n): variant 0 = FP32 path, 1 = tensor-core paths.
cudaError_t launch_sine_eval(int variant, const float* x, int64_t n, float* out_sin, float* out_cos, int num_sms,
                             cudaStream_t s);
bool tc_trace_split(int width, int n_hidden);  // head+remainder operands in the trace kernel
bool tc_grad_supported(int width, int n_hidden);

// ---------------------------------------------------------------------------
// training path (FP32)
// ---------------------------------------------------------------------------
// Parameter vector theta: the folded parameters of Eq. 2 in the order of the
// SDFN file (W_0 [w][in], b_0, then per hidden layer W_i [w][w], b_i, then
// w_out [w], b_out), FP32.
struct TrainShape {
    int in_dim, width, n_hidden;
    int64_t off_w0, off_b0, off_w[kMaxHidden], off_b[kMaxHidden], off_wout, off_bout, count;
};
TrainShape train_shape(int in_dim, int width, int n_hidden);

// Workspace of one forward / backward pair over n points.
struct TrainWork {
    // FP32 SIMT path
    float* wt;                     // [k][w][w] transposed hidden weights
    float* z0;                     // [n][w] layer-0 pre-activations A_0 (both paths)
    float* z;                      // [k][n][4][w] per hidden layer: A_i and the tangent pre-images W_i G_{i-1}
    float* d;                      // [k][n][4][w] their adjoints (backward)
    unsigned long long* counters;  // [4] tile counters
    // tensor-core path
    uint8_t* wbf;                  // [k] 16-bit W_l images (K-major, 128-byte swizzle, rows padded to 128)
    uint8_t* wbft;                 // [k] 16-bit W_l^T images, same layout
    float* qa;                     // A_l records (rec_a layout)
    uint2* qh;                     // H_l^x, H_l^y | H_l^z, 0 as 16-bit operand-type values (rec_h layout)
    uint8_t* dtile;                // [k][n_halves][w * 256] 16-bit (dA_l, dH_l) tiles
    int64_t n_halves;              // 2 ceil(n / 64): half-tiles of 32 points, in pairs
};
size_t train_workspace_bytes(const TrainShape& sh, int64_t n);
TrainWork train_work(const TrainShape& sh, int64_t n, void* ws);
size_t train_tc_workspace_bytes(const TrainShape& sh, int64_t n);
TrainWork train_tc_work(const TrainShape& sh, int64_t n, void* ws);

struct TrainArgs {
    TrainShape sh;
    const float* theta;
    const float* pts;      // SoA (3, n)
    const float* pt_time;  // (n) or NULL (4-input networks)
    int64_t n;
    float* out_f;          // forward: (n)
    float* out_grad;       // forward: SoA (3, n)
    const float* d_f;      // backward: dL/df (n)
    const float* d_grad;   // backward: dL/d(grad f) SoA (3, n)
    TrainWork w;
    float* d_theta;        // backward: accumulated dL/dtheta
    int* status;           // device status word (bounded waits of the tensor-core kernels)
};
cudaError_t launch_train_forward(const TrainArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_train_backward(const TrainArgs& a, int num_sms, cudaStream_t s);
// Tensor-core training (16-bit operands: f16 = IEEE half, else bfloat16; FP32 accumulation).
cudaError_t launch_train_forward_tc(const TrainArgs& a, bool f16, int num_sms, cudaStream_t s);
cudaError_t launch_train_backward_tc(const TrainArgs& a, bool f16, int num_sms, cudaStream_t s);
cudaError_t launch_fit_loss(const float* f, const float* grad, const float* tf, const float* tgrad,
                            const uint8_t* near, int64_t n, float lam_n, float lam_e, float* d_f, float* d_grad,
                            double* sums, unsigned long long* n_near, double* out, int num_sms, cudaStream_t s);
cudaError_t launch_adam(float* theta, const float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                        float beta2, float eps, int step, int num_sms, cudaStream_t s);

// A bounded wait on a barrier nothing signals, with the given budget: must
// latch kStatusTimeout in *status and return.
cudaError_t launch_wait_timeout_selftest(int* status, unsigned long long budget_ns, cudaStream_t s);

// Builds list[] of the indices with mask[i] != 0 (order unspecified), zeroes
// out[.][i] where mask[i] == 0 (out may be NULL: nothing is zeroed), and
// counts into *count (zero at launch).
cudaError_t launch_mask_compact(const uint8_t* mask, int64_t n, int32_t* list, unsigned long long* count,
                                float* out, int num_sms, cudaStream_t s);

}  // namespace sdfnn
