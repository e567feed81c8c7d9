/*
 * sdfnn.h - C ABI of the GB300 (sm_103a) renderer for nested neural SDFs.
 *
 * Implements the rendering hot path of da Silva et al., "Neural Implicit
 * Mapping via Nested Neighborhoods" (CVPR 2023):
 *   - multiscale sphere tracing of a nested sequence f_1 |> ... |> f_m (Sec. 4, Alg. 1),
 *   - analytic gradients of sine MLPs (Sec. 5.1, Eqs. 3-4, Alg. 2),
 *   - neural normal mapping N(p) = grad f(p) on a coarse surface (Sec. 5).
 *
 * Conventions shared by every call:
 *   - Point and ray arrays are structure-of-arrays float32: element c of item
 *     i lives at ptr[c * n + i] (c = 0, 1, 2 for x, y, z).
 *   - Buffers passed to sdf_trace_multiscale, sdf_normals and sdf_normal_map
 *     are caller-owned DEVICE memory (cudaMalloc / torch CUDA tensors) on the
 *     device the networks were loaded on.  Host pointers are rejected with
 *     SDF_ERR_ARG before any kernel runs.  sdf_render_host and
 *     sdf_frame_queue_submit are the calls that take host memory.
 *   - Calls are asynchronous on `cuda_stream` (a cudaStream_t; NULL means the
 *     legacy default stream).  Argument errors are returned immediately.
 *     Errors a kernel detects on the device (a bounded wait that expired:
 *     SDF_ERR_TIMEOUT) are latched in a per-device status word and returned
 *     by sdf_sync_status.
 *   - n == 0 is valid and launches nothing.
 *   - Per-call scratch (work counters, ray queues, compaction lists, the
 *     host-frame buffers of sdf_render_host) comes from a stream-ordered
 *     memory pool of the library on each device, which keeps the memory it
 *     has reserved for later calls (up to the largest call's need).
 *   - Every non-OK return sets a thread-local message (sdf_last_error).
 *
 * Network files ("SDFN", little-endian):
 *   offset 0  char[4] "SDFN"       offset 16 u32 n_hidden k
 *   offset 4  u32 version = 1      offset 20 f32 omega0 (layer-0 sine frequency)
 *   offset 8  u32 in_dim (3 or 4)  offset 24 f32 omega  (hidden sine frequency)
 *   offset 12 u32 width w          offset 28 u32 flags  (bit 0: weights already folded)
 *   offset 32 f32 W_0[w][in_dim], b_0[w], then k times (W_i[w][w], b_i[w]),
 *             then W_out[w], b_out: the MLP of Eq. 2 with k + 1 sine layers
 *             of width w, written (w, k) in Sec. 6.
 */
#ifndef SDFNN_H
#define SDFNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdf_net *sdf_net_t; /* opaque, owned by the library until sdf_net_free */

enum {
    SDF_OK = 0,
    SDF_ERR_ARG = -1,         /* NULL / host pointer, bad size, inconsistent parameters */
    SDF_ERR_FILE = -2,        /* file cannot be read */
    SDF_ERR_FORMAT = -3,      /* not a valid SDFN image */
    SDF_ERR_CUDA = -4,        /* a CUDA runtime call failed */
    SDF_ERR_NONFINITE = -5,   /* NaN or Inf in the network parameters */
    SDF_ERR_TIMEOUT = -6,     /* a kernel's bounded wait expired (device status word) */
    SDF_ERR_UNSUPPORTED = -7  /* shape / precision combination this build does not run */
};

/* Arithmetic of the hidden w x w layers.  Layer 0, the output layer, the
 * sine/cosine epilogues, the ray state and the step update are FP32 in all
 * modes. */
enum {
    SDF_FP32 = 0, /* SIMT FP32 contractions (the plain comparison path) */
    SDF_BF16 = 1, /* tcgen05 tensor-core contractions, bfloat16 operands, FP32 accumulation */
    SDF_FP8 = 2,  /* tcgen05 kind::f8f6f4 contractions with E4M3 operands, FP32 accumulation, for
                     sdf_normals / sdf_normal_map(_timed) of width 128 or 256 networks and
                     for tracing with width 256 networks (SDF_ERR_UNSUPPORTED at load for
                     width 64, and when tracing with width 128).  Hidden weights are
                     stored as W_l * 448 / max|W_l|; the sine activations as 256 sin; the
                     tangents of Alg. 2 with per-layer scales fixed at load from their
                     largest value on a 7^3 grid over [-1, 1]^3 (mapped to 64, leaving 7x
                     headroom before the conversion saturates at 448); w_out as an E4M3
                     head plus a remainder.  E4M3 keeps 3 mantissa bits: normals are
                     accurate to a few degrees and hit points to ~1e-2, not to SDF_BF16's
                     bounds. */
    SDF_FP16 = 3  /* tcgen05 tensor-core contractions, IEEE half operands, FP32 accumulation:
                     same tensor rate as SDF_BF16 with 3 more mantissa bits; the sine
                     activations lie in [-1, 1] and need no wider exponent range */
};

/* Load a network and prepare it on `device`: fold the sine frequencies into
 * the weights (layer 0 by omega0, hidden layers by omega), compute the
 * Lipschitz bound L = prod_i ||W_i||_2 * ||W_out||_2 in FP64 (sin is
 * 1-Lipschitz, so 1/L is a step that never crosses the zero set), and upload
 * FP32 parameters plus, for SDF_BF16 / SDF_FP16, the hidden matrices rounded
 * to bfloat16 / half (nearest even) in the tensor-core operand layout.
 * Supported shapes: in_dim 3 or 4, width 64, 128 or 256, 1 <= n_hidden <= 4.
 * Errors: SDF_ERR_ARG (NULL out / bad precision / bad device), SDF_ERR_FILE,
 * SDF_ERR_FORMAT, SDF_ERR_NONFINITE, SDF_ERR_UNSUPPORTED, SDF_ERR_CUDA.
 * On error *out is set to NULL and nothing is leaked. */
int sdf_net_load(const char *path, int precision, int device, sdf_net_t *out);
int sdf_net_load_mem(const void *bytes, size_t n_bytes, int precision, int device, sdf_net_t *out);

/* Shape and Lipschitz bound of a loaded network (any out pointer may be NULL). */
int sdf_net_info(sdf_net_t net, int *in_dim, int *width, int *n_hidden, double *lipschitz);

/* Time coordinate fed as the 4th input of 4-D networks by sdf_normals and
 * sdf_normal_map (Sec. 3.2 families of neural SDFs).  Ignored for 3-D nets. */
int sdf_net_set_time(sdf_net_t net, float time);

/* Frees the network and its device memory.  NULL is a no-op.  The caller
 * must not free a network while work that uses it is still in flight. */
void sdf_net_free(sdf_net_t net);

/* Parameters of Alg. 1 for a nested sequence f_1 |> ... |> f_m. */
typedef struct {
    int n_levels;              /* m >= 1 (at most 8) */
    const sdf_net_t *nets;     /* m networks, same device, same in_dim */
    const float *delta;        /* m thresholds delta_j (Eq. 1); delta_m is used only when final_mode == 1 */
    const int *max_iters;      /* m iteration caps (>= 0); the paper fixes iteration counts (Sec. 6) */
    float eps;                 /* epsilon of Alg. 1 (> 0) */
    const float *step_scale;   /* m step scales s_j, or NULL for s_j = 1/L_j */
    float box_min, box_max;    /* rays are clipped to the cube [box_min, box_max]^3 */
    int final_mode;            /* 0: trace S_m (Alg. 1); 1: stop on the delta_m shell of f_m */
    float time;                /* 4th input of 4-D networks, the same for every ray */
    const float *ray_time;     /* device, (n) float32: the 4th input of each ray, overriding `time`
                                  (frames of an animation traced together, Sec. 3.2); NULL for none.
                                  4-D networks only (SDF_ERR_ARG otherwise). */
} sdf_trace_params;

/* Multiscale sphere tracing (Sec. 4, Alg. 1) of n rays.
 *   orig, dir : device, SoA (3, n) float32; dir must be unit length.
 *   out_pos   : device, SoA (3, n) float32, end point of each ray.
 *   out_t     : device, (n) float32, distance travelled from orig to out_pos.
 *   out_hit   : device, (n) uint8, 1 = hit, 0 = miss.
 *   out_iters : device, (n) uint16 total steps over all levels, or NULL.
 * Per ray: start where the ray enters the cube (or at orig if inside; a ray
 * that misses the cube is a miss with no evaluation); for each level j run
 *     t = f_j(p) - d_j ;  p += s_j * t * dir
 * (d_j = delta_j, or 0 on the last level with final_mode 0) while t > eps
 * and fewer than max_iters[j] steps were taken, the step taken before the
 * test as in Alg. 1.  A point outside the cube widened by 1e-3 ends the ray
 * as a miss.  Hit iff the last level ended with t <= eps.
 * Errors: SDF_ERR_ARG (NULL or host pointers, n < 0, m out of range, eps <= 0,
 * negative caps, delta_j <= 0 for a level that uses it, mixed devices or
 * in_dim), SDF_ERR_UNSUPPORTED, SDF_ERR_CUDA. */
int sdf_trace_multiscale(const sdf_trace_params *params, const float *orig, const float *dir, int64_t n,
                         float *out_pos, float *out_t, uint8_t *out_hit, uint16_t *out_iters,
                         void *cuda_stream);

/* Analytic gradient grad f(p) (Sec. 5.1, Eqs. 3-4, Alg. 2) at n points.
 *   pts      : device, SoA (3, n) float32.
 *   out_grad : device, SoA (3, n) float32, unnormalised gradient (x, y, z).
 * Errors: SDF_ERR_ARG, SDF_ERR_CUDA. */
int sdf_normals(sdf_net_t net, const float *pts, int64_t n, float *out_grad, void *cuda_stream);

/* Neural normal mapping (Sec. 5): N(p) = grad f(p) / |grad f(p)| of the fine
 * network at points of a coarser surface (end points of a coarse trace, or
 * mesh vertices).
 *   pts        : device, SoA (3, n) float32.
 *   mask       : device, (n) uint8 (0 = skip) or NULL for all points.
 *   out_normal : device, SoA (3, n) float32; (0, 0, 0) where the mask is 0
 *                or |grad f| < 1e-12.
 * Errors: SDF_ERR_ARG, SDF_ERR_CUDA. */
int sdf_normal_map(sdf_net_t fine, const float *pts, const uint8_t *mask, int64_t n, float *out_normal,
                   void *cuda_stream);

/* sdf_normal_map of a 4-D network with a time per point: the 4th input of
 * point i is pt_time[i] (device, (n) float32, not NULL).  The gradient is
 * the spatial one (x, y, z), as for a 3-D network at that time.
 * Errors: as sdf_normal_map; SDF_ERR_ARG for a 3-input network. */
int sdf_normal_map_timed(sdf_net_t fine, const float *pts, const float *pt_time, const uint8_t *mask, int64_t n,
                         float *out_normal, void *cuda_stream);

/* One frame end to end from HOST memory: sdf_trace_multiscale of the rays
 * orig/dir, then sdf_normal_map(fine) on the hits; hit, end point and normal
 * come back to host memory.  Two ways, chosen per call:
 *   - every buffer page-locked and mapped into the device's address space
 *     (cudaHostAlloc, cudaHostRegister, pinned torch tensors; the whole
 *     range is checked with cudaPointerGetAttributes): the kernels read the
 *     rays and write the normals in host memory themselves (over NVLink-C2C on
 *     Grace systems), one trace covers all rays, and the copy engine brings
 *     back the end points and hit flags while the normals are computed;
 *   - otherwise: frames of 2^18 rays and more are split into 2 or 4 chunks
 *     whose copies in, kernels and copies out run on three streams of the
 *     library, so the transfers of one chunk overlap the kernels of another.
 * Both give the same bytes as the device calls.  Device buffers come from
 * the library's pool on `cuda_stream`, which waits for the whole frame.
 * orig, dir: host (3, n); out_pos, out_normal: host (3, n); out_hit: host
 * (n).  params->ray_time must be NULL.  Calls on one device are serialised.
 * Returns after the results are in host memory (the stream is synchronised).
 * Errors: as sdf_trace_multiscale and sdf_normal_map. */
int sdf_render_host(const sdf_trace_params *params, sdf_net_t fine, const float *orig, const float *dir,
                    int64_t n, float *out_pos, uint8_t *out_hit, float *out_normal, void *cuda_stream);

/* Multiscale sphere tracing that allocates no device memory.
 *
 * The paper has no counterpart: this is a convenience of the library.
 * sdf_trace_multiscale takes the scratch it needs (work counters and the
 * ray queues between levels) from the stream-ordered allocator on every
 * call.  Some callers cannot allow that: render loops that forbid device
 * allocation once they are running, or hosts whose device memory is owned
 * by an allocator of their own.  This entry point has the same arguments,
 * semantics and errors, but its scratch is one static device array inside
 * the library (16 MB, present on every device that loads the library until
 * the process exits).
 *   - n may not exceed 2,097,152 rays (one 1920 x 1080 frame fits); a larger
 *     n returns SDF_ERR_ARG before anything is launched.
 *   - The first call on a device looks up the array's device address with
 *     that device current (cudaGetSymbolAddress); make that first call
 *     before capturing any stream.
 *   - Every call uses the same array: it zeroes the counters at its start,
 *     and calls whose work overlaps on the GPU (other streams, other host
 *     threads) race on it and corrupt each other's results.  Serialise them.
 *   - Device-side timeouts of these launches are latched in a status word
 *     inside the array; sdf_sync_status reads and clears it together with
 *     the library's per-device status word, so a timed-out call is reported
 *     as SDF_ERR_TIMEOUT by the next sdf_sync_status on that device. */
int sdf_trace_multiscale_noalloc(const sdf_trace_params *params, const float *orig, const float *dir, int64_t n,
                                 float *out_pos, float *out_t, uint8_t *out_hit, uint16_t *out_iters,
                                 void *cuda_stream);

/* Frame-batch plans.
 *
 * The paper renders animations of 4-D networks frame by frame (Sec. 3.2,
 * Sec. 6).  A plan renders a whole batch of frames - any mix of
 * resolutions, each ray carrying its frame's time - as one unit: all
 * levels of Alg. 1 over every ray of the batch (the level queues mix rays
 * of all frames, so small frames never leave the GPU idle) followed by the
 * normal mapping of the hits, captured once into a CUDA graph and replayed
 * by sdf_plan_launch.  The buffers are fixed when the plan is made: write
 * the next batch's rays into the same orig / dir / ray_time and launch
 * again.
 *
 * sdf_plan_create(params, fine, batch, autotune, stream, &plan)
 *   params   : as for sdf_trace_multiscale, copied; params->ray_time must
 *              be NULL or equal to batch->ray_time.  The networks are not
 *              copied: keep them alive while the plan exists.
 *   fine     : network of the normal-mapping stage, or NULL with
 *              batch->out_normal NULL (trace only).
 *   batch    : the device buffers (all on the networks' device):
 *              orig, dir (3, n); ray_time (n) or NULL; out_pos (3, n);
 *              out_t (n); out_hit (n); out_iters (n) or NULL;
 *              out_normal (3, n) or NULL.  The normals are those of
 *              sdf_normal_map(_timed) with out_hit as the mask.
 *   autotune : nonzero: before capturing, time every tile count (ray tiles
 *              per CTA) of each tensor-core level on these buffers and keep
 *              the fastest; the outputs are overwritten meanwhile and the
 *              stream is synchronised.  0: the library's default counts.
 *              The tile count changes the speed only: every ray's
 *              arithmetic, and so every output bit, is the same.
 *   stream   : stream of the autotuning runs (capture uses a private one).
 *   The plan owns its scratch (device memory for the level queues and the
 *   normal-map compaction: 8 * n + 12 * n bytes at most, from cudaMalloc).
 * sdf_plan_launch: enqueues the graph on `stream`; device-side errors are
 *   latched in the status word read by sdf_sync_status.  Launches of one plan
 *   share its scratch, so launches on different streams must not overlap.
 * sdf_plan_info: tile count per level (max_levels entries, 0 = default for
 *   SIMT levels) and the number of graph nodes; either pointer may be NULL.
 * sdf_plan_free: NULL is a no-op; no launch of the plan may be in flight.
 * Errors: as sdf_trace_multiscale and sdf_normal_map, SDF_ERR_CUDA for a
 * failed capture or instantiation; on error *plan is NULL. */
typedef struct sdf_plan *sdf_plan_t;

typedef struct {
    const float *orig, *dir;
    const float *ray_time;
    int64_t n;
    float *out_pos;
    float *out_t;
    uint8_t *out_hit;
    uint16_t *out_iters;
    float *out_normal;
} sdf_frame_batch;

int sdf_plan_create(const sdf_trace_params *params, sdf_net_t fine, const sdf_frame_batch *batch, int autotune,
                    void *cuda_stream, sdf_plan_t *plan);
int sdf_plan_launch(sdf_plan_t plan, void *cuda_stream);
int sdf_plan_info(sdf_plan_t plan, int *tiles, int max_levels, int64_t *n_graph_nodes);
void sdf_plan_free(sdf_plan_t plan);

/* Frame queues: host frames rendered back to back.
 *
 * The paper renders image after image (its frame rates, Tab. 3; its
 * animations, Sec. 6).  sdf_render_host does one frame per call and returns
 * with the results in host memory, so each call pays for its own copies.  A
 * queue keeps `depth` frames in flight instead: every slot holds device
 * copies of one frame's rays and results and a plan (one CUDA graph: all
 * levels of Alg. 1, then sdf_normal_map of the fine network at the hits),
 * and while frame k's graph runs, the rays of frame k + 1 are copied in and
 * the results of frame k - 1 copied out on two copy streams of the queue;
 * consecutive frames alternate between two compute streams, so a frame's
 * kernels may start while the previous frame's last rays are still traced.
 * The results are the bytes sdf_trace_multiscale + sdf_normal_map give.
 *
 * sdf_frame_queue_create(params, fine, n, depth, &queue)
 *   params : as for sdf_trace_multiscale (copied; ray_time must be NULL).
 *            The networks are not copied: keep them and `fine` alive while
 *            the queue exists.
 *   fine   : the normal-mapping network (not NULL).
 *   n      : rays per frame (1 .. 2^31 - 1), the same for every frame.
 *   depth  : frames in flight, 1 .. 4 (2 overlaps copies and kernels).
 *   The queue owns per slot 4 * 12n + 4n + n bytes of device memory
 *   (cudaMalloc) plus the plan's scratch.
 * sdf_frame_queue_submit(queue, orig, dir, out_pos, out_hit, out_normal, &ticket)
 *   Enqueues one frame: host orig, dir (3, n); host out_pos (3, n), out_hit
 *   (n), out_normal (3, n) receive the end points, hit flags and unit
 *   normals ((0,0,0) at misses).  Returns at once with the frame's ticket
 *   (0, 1, 2, ... in submission order; `ticket` may be NULL), after waiting
 *   for the frame that last used the slot when `depth` frames are in flight.
 *   The host buffers must stay valid, and the outputs untouched, until the
 *   frame is waited for.  Page-locked host memory lets the copies overlap the
 *   kernels; pageable memory gives the same bytes with less overlap.
 * sdf_frame_queue_wait(queue, ticket)
 *   Returns when frame `ticket` and every earlier frame are in host memory
 *   (ticket < 0: every frame submitted); a device-side timeout of any frame
 *   since the last check (the status word of sdf_sync_status) is returned
 *   as SDF_ERR_TIMEOUT.  A ticket not yet issued is SDF_ERR_ARG.
 * sdf_frame_queue_free: waits for the frames in flight, then frees; NULL is
 *   a no-op.
 * A queue is used by one host thread at a time.
 * Errors: as sdf_plan_create; SDF_ERR_ARG for a bad n, depth or NULL
 * buffer; SDF_ERR_CUDA for a failed copy, launch or wait. */
typedef struct sdf_frame_queue *sdf_frame_queue_t;

int sdf_frame_queue_create(const sdf_trace_params *params, sdf_net_t fine, int64_t n, int depth,
                           sdf_frame_queue_t *queue);
int sdf_frame_queue_submit(sdf_frame_queue_t queue, const float *orig, const float *dir, float *out_pos,
                           uint8_t *out_hit, float *out_normal, int64_t *ticket);
int sdf_frame_queue_wait(sdf_frame_queue_t queue, int64_t ticket);
void sdf_frame_queue_free(sdf_frame_queue_t queue);

/* Training.
 *
 * The paper fits every network of a sequence with an external framework
 * (Sec. 2, Sec. 3.3).  These calls make that fitting native: the forward
 * pass of Eq. 2 together with the tangents of Alg. 2, the fitting objective,
 * the backward pass through both (the direction and Eikonal terms depend on
 * grad f, so their parameter gradients are second derivatives of f) and an
 * Adam step.
 *
 * precision: SDF_FP32 runs every contraction on the CUDA cores in FP32.
 * SDF_BF16 (or SDF_FP16) runs the hidden-layer contractions on the tensor
 * cores with 16-bit operands and FP32 accumulation: the forward W_l X_{l-1}
 * over the value and the three tangent streams, the adjoint W_l^T (dA_l, dH_l)
 * and the weight gradient sum (dA_l, dH_l) (P_{l-1}, G_{l-1})^T; layer 0, the
 * output layer, the sines and every elementwise step stay FP32.  The weights
 * are rounded from theta at every forward call.  SDF_FP8: SDF_ERR_UNSUPPORTED.
 *
 * theta: device float32, the folded parameters (the frequencies multiplied
 * in) in the order of the SDFN file - W_0 [w][in_dim], b_0, then for each
 * hidden layer W_i [w][w], b_i, then w_out [w], b_out - 16-byte aligned.  An
 * SDFN file with flags bit 0 set stores exactly this vector.
 * Shapes: in_dim 3 or 4, width 64, 128 or 256, 1 <= n_hidden <= 4
 * (SDF_ERR_UNSUPPORTED otherwise).
 *
 * sdf_train_shape_info: the length of theta and the workspace bytes the
 *   forward / backward pair needs for n points at that precision (either
 *   pointer may be NULL).  FP32: (1 + 8k) w floats per point; 16-bit:
 *   (1 + 5k) w floats per point plus two 16-bit copies of the hidden weights.
 * sdf_train_forward: f (n) and the unnormalised grad f (3, n) at pts (3, n)
 *   (pt_time (n) for 4-input networks, else NULL); saves the layers'
 *   pre-activations in `workspace` (device, 256-byte aligned, of the size
 *   above) for the backward.
 * sdf_train_backward: ADDS dL/dtheta to d_theta (16-byte aligned, like theta) given d_f = dL/df (n) and
 *   d_grad = dL/d(grad f) (3, n), from the workspace of the forward call made
 *   with the same theta, points and n (zero d_theta first for a fresh
 *   gradient).  Points are independent: chunks of a batch may be run one
 *   after another into the same d_theta.
 * sdf_fit_loss: the objective over n points
 *     L = mean |f - g| + lam_n mean_near (1 - cos(grad f, grad g)) + lam_e mean | |grad f| - 1 |
 *   (g, grad g: target_f (n), target_grad (3, n); near (n) uint8 marks the
 *   points of the direction term, whose mean over no point is 0).  Writes
 *   d_f, d_grad (the inputs of sdf_train_backward) and loss (device, 4
 *   doubles: the three means and L).  Subgradients: sign(0) = 0; points
 *   with grad f = 0 contribute no gradient to the direction and Eikonal terms.
 * sdf_adam_step: one Adam update of `count` parameters in place (m, v: the
 *   moment estimates, zero before step 1; step counts from 1).
 * Errors: SDF_ERR_ARG (NULL / host pointers, bad sizes, misalignment),
 * SDF_ERR_UNSUPPORTED, SDF_ERR_CUDA. */
int sdf_train_shape_info(int precision, int in_dim, int width, int n_hidden, int64_t n, int64_t *param_count,
                         int64_t *workspace_bytes);
int sdf_train_forward(int precision, int in_dim, int width, int n_hidden, const float *theta, const float *pts,
                      const float *pt_time, int64_t n, float *out_f, float *out_grad, void *workspace,
                      void *cuda_stream);
int sdf_train_backward(int precision, int in_dim, int width, int n_hidden, const float *theta, const float *pts,
                       const float *pt_time, int64_t n, const float *d_f, const float *d_grad, void *workspace,
                       float *d_theta, void *cuda_stream);
int sdf_fit_loss(const float *f, const float *grad, const float *target_f, const float *target_grad,
                 const uint8_t *near, int64_t n, float lam_n, float lam_e, float *d_f, float *d_grad, double *loss,
                 void *cuda_stream);
int sdf_adam_step(float *theta, const float *grad, float *m, float *v, int64_t count, float lr, float beta1,
                  float beta2, float eps, int step, void *cuda_stream);

/* Synchronises the stream, then returns and clears the status word of the
 * current device (SDF_OK, or the first device-side error since the last call). */
int sdf_sync_status(void *cuda_stream);

/* Self-test of the device-side failure detection: launches a kernel whose
 * bounded wait (the same loop the library's kernels use around every
 * mbarrier) waits on a barrier that nothing signals, with a limit of
 * budget_us microseconds (1 .. 10^7).  Returns SDF_OK when the wait expired,
 * the kernel returned and sdf_sync_status reported (and cleared)
 * SDF_ERR_TIMEOUT; the device stays usable.  The paper has no counterpart.
 * Errors: SDF_ERR_ARG, SDF_ERR_CUDA (also when the expiry was not reported),
 * or a status already pending on the device before the call. */
int sdf_selftest_wait_timeout(int device, int64_t budget_us, void *cuda_stream);

/* Self-test of the timeout reporting of sdf_trace_multiscale_noalloc (the
 * paper has no counterpart): the bounded wait of sdf_selftest_wait_timeout,
 * latching into the status word of the allocation-free entry point's static
 * array instead of the library's per-device word.  Returns SDF_OK when the
 * wait expired and sdf_sync_status reported (and cleared) SDF_ERR_TIMEOUT
 * from that array.  Sets the array up on `device` like the entry point's
 * first call does (allocates nothing).
 * Errors: SDF_ERR_ARG, SDF_ERR_CUDA, or a status already pending. */
int sdf_selftest_noalloc_timeout(int device, int64_t budget_us, void *cuda_stream);

/* Step a1 on the host, for the training calls: the folded parameter vector
 * theta (Eq. 2 with the sine frequencies multiplied in: W_0, b_0 by omega0,
 * the hidden W_i, b_i by omega, the output row unchanged; FP64 products
 * rounded to FP32) of an SDFN image, in the file's order.  Host memory only;
 * no device is touched.
 *   theta    : host float32 buffer of `capacity` entries, or NULL to query.
 *   count, in_dim, width, n_hidden : outputs (each may be NULL).
 * Errors: SDF_ERR_ARG (NULL bytes, capacity below the parameter count),
 * SDF_ERR_FORMAT, SDF_ERR_NONFINITE. */
int sdf_theta_from_image(const void *bytes, size_t n_bytes, float *theta, int64_t capacity, int64_t *count,
                         int *in_dim, int *width, int *n_hidden);

/* Accuracy helper: the sine and cosine the kernels use for the sine layers of
 * Eq. 2 and the cosines of Alg. 2, at given arguments (the paper does not
 * discuss their accuracy).
 *   variant 0 : the FP32 (SDF_FP32) kernels' functions: reduction of x by the
 *               nearest multiple of 2 pi (a two-float split of 2 pi), then the
 *               hardware approximation on [-pi, pi];
 *   variant 1 : the tensor-core kernels' functions (SDF_BF16, SDF_FP16,
 *               SDF_FP8): the hardware approximation applied to x directly.
 *   x, out_sin, out_cos : device, (n) float32.
 * A NaN in out_sin marks an argument at which the trace kernels' own sine
 * would differ from the value written (it never should).
 * Errors: SDF_ERR_ARG, SDF_ERR_CUDA. */
int sdf_eval_sine(int variant, const float *x, int64_t n, float *out_sin, float *out_cos, void *cuda_stream);

/* Measurement helper: the throughput, in sines per second on all SMs, of the
 * hardware sine the tensor-core kernels use (independent chains of
 * sin(x) * c + d, timed with CUDA events on `cuda_stream`, which is
 * synchronised).  It is the ALU roof of the sine-bound trace kernel.
 * Errors: SDF_ERR_ARG, SDF_ERR_CUDA. */
int sdf_measure_sine_rate(int device, double *sines_per_s, void *cuda_stream);

/* Thread-local message describing the last non-OK return of this thread. */
const char *sdf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SDFNN_H */
