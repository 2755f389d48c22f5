/*
 * disk.h -- C ABI of libdisk.so: spatially varying filtering with a sparse
 * kernel complex (DISK, "Differentiable Sparse Kernel Complex for Efficient
 * Spatially-Variant Convolution", arXiv 2512.04556), GB300 (sm_103a) native.
 *
 * General rules for every entry point
 *   - Status: 0 (DISK_OK) on success, a negative DISK_ERR_* code otherwise;
 *     disk_error_string() names it.  Arguments are validated before any work
 *     is queued; on an error nothing is launched and outputs are untouched.
 *   - Pointers prefixed d_ are device pointers on the current CUDA device;
 *     all other pointers are host pointers.  Every buffer is caller-owned;
 *     the library owns only disk_basis handles, a status word per device and
 *     per-call scratch, which it takes stream-ordered from its own memory
 *     pool on the current device (freed memory stays mapped for the next
 *     call) and returns on the same stream.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream; no entry point
 *     synchronises the device except disk_basis_* (host<->device uploads),
 *     the autotuners and disk_device_status.
 *   - Images are interleaved H x W x C (C = 3 or 4), row pitch in BYTES,
 *     element type DISK_F32 (float) or DISK_F16 (IEEE half).  Arithmetic is
 *     FP32 throughout; FP16 is a storage type only (inputs widened exactly,
 *     outputs rounded to nearest even).
 *   - Offsets are in pixels, (dx, dy) = (column, row) direction.  A tap at a
 *     fractional offset is sampled bilinearly with texel centres at integer
 *     coordinates; image filtering clamps coordinates to the edge, impulse
 *     synthesis treats everything outside its canvas as zero.
 */
#ifndef DISK_H
#define DISK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DISK_OK = 0,
  DISK_ERR_INVALID_ARG = -1,  /* bad shape, pitch, pointer, enum or value   */
  DISK_ERR_BAD_FILE = -2,     /* basis file missing, truncated or corrupt   */
  DISK_ERR_UNSUPPORTED = -3,  /* valid request outside the built limits     */
  DISK_ERR_CUDA = -4,         /* a CUDA runtime call failed                 */
  DISK_ERR_OOM = -5,          /* device or host allocation failed           */
  DISK_ERR_TIMEOUT = -6       /* a bounded device-side wait expired         */
};

enum { DISK_F32 = 0, DISK_F16 = 1 };

/* Library limits (validated at every entry point). */
#define DISK_MAX_DIMS 2          /* kernel-space dimensions of a basis       */
#define DISK_MAX_NODES_AXIS 64   /* basis nodes per kernel-space axis        */
#define DISK_MAX_LAYERS 16       /* sparse layers L                          */
#define DISK_MAX_TAPS 64         /* taps per layer T                         */
#define DISK_MAX_REACH 40.0f     /* largest |dx|, |dy| of any basis tap, px   */

/* Library version, major*10000 + minor*100 + patch. */
int disk_version(void);

/* Human-readable name of a status code (static string, never NULL). */
const char *disk_error_string(int status);

/* Detail of the last failure on the calling thread (never NULL; valid until
 * the thread's next failing call). */
const char *disk_last_error_message(void);

/* ---------------------------------------------------------------------------
 * Basis of pre-optimised complexes (Sec. 4.3, Eq. 8).
 *
 * A basis samples a 1-D or 2-D kernel space at nodes p_1 < ... < p_n per
 * axis (Eq. 8 orders them increasingly); node k holds one complex
 * f_k = {(o_{k,l,i}, w_{k,l,i})}: L layers of T taps (Eq. 2, Eq. 5).
 * theta layout: float [B][L][T][3] = (dx, dy, w), B = n_nodes[0] (1-D) or
 * n_nodes[0] * n_nodes[1] (2-D, node (a, b) at index a * n_nodes[1] + b, axis
 * 0 driven by map 0).  The handle keeps a host copy and a device copy on the
 * device current at creation; it is immutable and may be shared by
 * concurrent calls on any stream of that device.
 * ------------------------------------------------------------------------- */
typedef struct disk_basis disk_basis;

/* Build a basis from host arrays.  node_vals holds n_nodes[0] values for
 * axis 0 followed (2-D) by n_nodes[1] values for axis 1, each strictly
 * increasing.  Every value must be finite and every |dx|, |dy| at most
 * DISK_MAX_REACH.  Uploads synchronously.  *out receives a new handle. */
int disk_basis_from_arrays(int dims, const int *n_nodes, const float *node_vals,
                           int L, int T, const float *theta, disk_basis **out);

/* Read a basis file (format: 8-byte magic "DISKBAS1", then little-endian
 * uint32 version=1, dims, L, T, n_nodes[2] (n_nodes[1]=1 for 1-D), float32
 * node values, float32 theta, and a trailing uint64 FNV-1a hash of all
 * preceding bytes).  DISK_ERR_BAD_FILE on any mismatch. */
int disk_basis_load(const char *path, disk_basis **out);

/* Write the basis in the format disk_basis_load reads. */
int disk_basis_save(const disk_basis *basis, const char *path);

/* Shape of a basis; any output pointer may be NULL. */
int disk_basis_info(const disk_basis *basis, int *dims, int *n_nodes2, int *L,
                    int *T);

/* Release a handle (NULL is a no-op).  The caller ensures no queued call
 * still uses it. */
void disk_basis_free(disk_basis *basis);

/* ---------------------------------------------------------------------------
 * Spatially varying filter (Sec. 4.3 Eq. 9 + Sec. 3.2 Eq. 3).
 *
 * For every output pixel x, alpha(x) are the linear (1-D) or bilinear (2-D)
 * interpolation weights of the map value(s) p(x) between the bracketing
 * nodes (p clamped to the node range; a non-finite p acts as the first
 * node), the pixel's complex is sum_k alpha_k(x) f_k applied to offsets and
 * weights alike (Eq. 9), and the L layers are applied in cascade (Eq. 3):
 *   I_l[x] = sum_i w_{l,i}(x) * bilinear(I_{l-1}, x + o_{l,i}(x)),
 * every layer using the parameters interpolated at its own output pixel.
 *
 * d_in / d_out: H x W x C images of type dtype with row pitches in bytes
 *   (multiples of the element size, at least W*C*elem).  d_in and d_out must
 *   not overlap.
 * d_maps: float [dims][H][W], dense, raw parameter values.
 * Limits: 1 <= H, W <= 32768; C in {3, 4}.
 * Intermediate layers are stored in FP32 whatever the image precision, C
 *   floats per pixel, rows padded to 16 bytes; arithmetic and accumulation
 *   are FP32.  The output is rounded to the image's precision (FP16 round to
 *   nearest even).
 * Scratch: two intermediate buffers (one for L = 2, none for L = 1) of
 *   about H * W * (C == 4 ? 16 : 12) bytes, plus, for the rotated variant,
 *   an H * W * 8-byte (cos, sin) plane, from the library's memory pool,
 *   freed on the stream.
 * Tile configuration: the one disk_sv_filter_autotune recorded for this
 *   frame shape, else 32 x 16 tiles.  Layers after the first have their tile
 *   copied by the tensor-memory accelerator; a copy that does not complete
 *   within its bounded wait is reported by disk_device_status. */
int disk_sv_filter(const disk_basis *basis, const void *d_in, size_t in_pitch,
                   void *d_out, size_t out_pitch, int H, int W, int C,
                   int dtype, const float *d_maps, void *stream);

/* ---------------------------------------------------------------------------
 * Gradient of the spatially varying filter with respect to its input image
 * (transpose of Eq. 3 with the Eq. 9 per-pixel complex):
 *   d_grad_in = A_1^T A_2^T ... A_L^T d_grad_out,
 * A_l the layer-l operator of disk_sv_filter on the same maps, basis and
 * clamp-to-edge border (a corner clamped onto the border pixel sends its
 * share back to that pixel).  The filter is linear in the image, so the
 * result does not depend on the image itself.
 * d_grad_out: H x W x C of type dtype (pitch in bytes); d_grad_in: H x W x C
 *   float (pitch in bytes, at least W * C * 4).  Other arguments as
 *   disk_sv_filter.  Scratch: two FP32 RGBA planes (2 * H * W * 16 bytes)
 *   from the library's memory pool.  Accumulation uses floating-point atomics, so the
 *   last bits of the result vary from run to run. */
int disk_sv_filter_backward_image(const disk_basis *basis, const void *d_grad_out,
                                  size_t gout_pitch, float *d_grad_in,
                                  size_t gin_pitch, int H, int W, int C, int dtype,
                                  const float *d_maps, void *stream);

/* Full backward of the spatially varying filter for training (gradients with
 * respect to the tap weights and fractional offsets of the basis, and the
 * input image), for the loss L = <d_grad_out, F(d_in)>:
 *   d_grad_theta [B][L][T][3] (float, overwritten): dL/d theta_k -- each
 *     pixel's tap gradient (d/dw = sum_c g_c s_c, d/d(dx,dy) = w sum_c g_c
 *     ds_c/d(dx,dy), s the bilinear sample of the layer input) passed to node
 *     k with the pixel's Eq. 9 weight alpha_k, summed over pixels;
 *   d_grad_in (float H x W x C, may be NULL): as disk_sv_filter_backward_image.
 * The layer inputs are recomputed from d_in by the forward kernels (nothing
 * is stored by the forward call).  At an exact integer offset the derivative
 * is the one-sided one of the floor convention.  Floating-point atomics: the
 * last bits vary from run to run.  Scratch: (L-1) activation planes in the
 * image's precision plus two FP32 RGBA planes, from the library's memory pool. */
int disk_sv_filter_backward(const disk_basis *basis, const void *d_in, size_t in_pitch,
                            const void *d_grad_out, size_t gout_pitch, float *d_grad_in,
                            size_t gin_pitch, float *d_grad_theta, int H, int W, int C,
                            int dtype, const float *d_maps, void *stream);

/* ---------------------------------------------------------------------------
 * disk_sv_filter without any allocation.  The paper has no counterpart: this
 * is a deployment variant of disk_sv_filter.
 *
 * Some callers cannot allocate device memory at all: a plug-in inside a host
 * application that owns the whole device-memory budget, a real-time loop that
 * forbids allocation after start-up so that its latency stays bounded, or
 * code that runs where the allocator may not be re-entered.  This entry point
 * runs disk_sv_filter's own code path (argument checks, the per-layer tile
 * record of disk_sv_filter_autotune, tensor-memory-accelerator copies, FP32
 * intermediates) and so returns disk_sv_filter's results bit for bit, with
 * the same arguments, layouts and status codes, but calls no cudaMalloc,
 * cudaFree or other allocating routine: the two intermediate planes live in
 * one fixed 32 MiB array built into the library, which every device that
 * loads the library holds until the process exits.
 * Limit: H * W <= 1048576 pixels; larger images return DISK_ERR_UNSUPPORTED
 *   before any work is queued.
 * First call on a device: it looks up the array's device address on the
 *   current device (once per device, then cached), so make that first call
 *   before capturing a stream into a CUDA graph.
 * Shared state: every call on a device uses the same array.  The array keeps
 *   the last call's contents; each layer overwrites every pixel it later
 *   reads, so nothing has to start at zero.  Calls that overlap on the GPU
 *   (different streams without ordering between them) race on the array and
 *   give undefined results: order them on one stream or with events. */
int disk_sv_filter_noalloc(const disk_basis *basis, const void *d_in,
                           size_t in_pitch, void *d_out, size_t out_pitch, int H,
                           int W, int C, int dtype, const float *d_maps,
                           void *stream);

/* Tile autotuner of disk_sv_filter: runs the filter on these buffers with
 * each built tile configuration (2 or 4 pixels per thread: 32 x 16 or
 * 32 x 32 output tiles), times every layer of each (the best tile depends
 * on the layer's halo), then times every adjacent pair of layers fused into
 * one launch -- the layer-fused form of the cascade (Sec. 3.2 Eq. 3): a
 * 32 x 16 tile stages the first layer's source on the tile grown by both
 * layers' halos, computes the first layer on the tile grown by the second
 * layer's halo into shared memory and the second layer from there, so the
 * intermediate between them never leaves the chip, at the price of
 * recomputing the first layer on the grown region -- and records, in the
 * basis handle for this (H, W, C, dtype), the fastest cover of the layers by
 * single layers and fused pairs; later disk_sv_filter calls with that shape
 * use it (without a record: 32 x 16 single layers).  Writes d_out.
 * Synchronises the stream (do not call while capturing a graph).  chosen
 * (may be NULL; int[L]) receives every layer's code: 2 or 4 (pixels per
 * thread of a single-layer launch), 8 (first layer of a fused pair, 32 x 16
 * tiles) followed by 0 (second layer of that pair). */
int disk_sv_filter_autotune(const disk_basis *basis, const void *d_in, size_t in_pitch,
                            void *d_out, size_t out_pitch, int H, int W, int C,
                            int dtype, const float *d_maps, int *chosen, void *stream);

/* Spatially varying filter with a per-pixel rotation of the complex
 * (Sec. 5.3: the rotational-bokeh and radial-motion effects are driven by a
 * blur strength and a local blur angle).  Computes what disk_sv_filter
 * computes, except that after the Eq. 9 blend every tap offset of output
 * pixel x is turned by angle[x] (radians; x to the right, y down):
 *   (dx, dy) -> (dx cos a - dy sin a, dx sin a + dy cos a).
 * Turning every offset of every layer turns the impulse response (Eq. 10) of
 * a shift-invariant complex by the same angle, so a basis over blur strength
 * (and, for 2-D bases, shape) plus an angle map replaces a basis grid over
 * the angle.  d_angle: float32 [H][W], device, caller-owned; a non-finite
 * angle acts as 0.  Other arguments as disk_sv_filter.  The shared-memory
 * halo of layer l comes from its largest Euclidean tap length (a turned tap
 * keeps its length); DISK_ERR_UNSUPPORTED if that halo does not fit.
 * Tile choice: recorded by disk_sv_filter_rotated_autotune (separately from
 * the plain filter's), else 32 x 16. */
int disk_sv_filter_rotated(const disk_basis *basis, const void *d_in, size_t in_pitch,
                           void *d_out, size_t out_pitch, int H, int W, int C, int dtype,
                           const float *d_maps, const float *d_angle, void *stream);

/* Tile autotuner of disk_sv_filter_rotated (as disk_sv_filter_autotune). */
int disk_sv_filter_rotated_autotune(const disk_basis *basis, const void *d_in,
                                    size_t in_pitch, void *d_out, size_t out_pitch, int H,
                                    int W, int C, int dtype, const float *d_maps,
                                    const float *d_angle, int *chosen, void *stream);

/* Filters n_frames frames that live in host memory (the deployment form of
 * disk_sv_filter: a video or burst whose frames arrive on the host).  Frame
 * i: image h_in[i] (H x W x C, rows packed, dtype as disk_sv_filter), maps
 * h_maps[i] (dims x H x W float32) -> h_out[i] (same layout as h_in[i]).
 * The host-to-device copies of one frame and the device-to-host copy of
 * another overlap the filtering of a third: two device slots alternate,
 * copies run on two streams the call creates, the filter on `stream`, all
 * ordered by events.  Host buffers should be page-locked (cudaHostAlloc or
 * cudaHostRegister) for the copies to be asynchronous; every buffer must
 * stay valid, and h_out untouched, until `stream` has completed (the call
 * returns once the work is queued).  Output equals disk_sv_filter on the
 * same frame with the same tile record.  Not capturable into a CUDA graph
 * (it creates streams).  Ownership: all buffers caller-owned; the slots come
 * from the library's pool. */
int disk_sv_filter_frames(const disk_basis *basis, const void *const *h_in,
                          void *const *h_out, const float *const *h_maps, int n_frames,
                          int H, int W, int C, int dtype, void *stream);

/* Device-side status of the current device: reads and clears the status
 * word that the library's kernels set when a bounded wait gives up (a
 * tile copy into shared memory that did not complete; the kernel then
 * returns without computing its tile).  Synchronises `stream` first.
 * Returns DISK_OK, or DISK_ERR_TIMEOUT if any kernel gave up since the last
 * call (outputs written since then are then incomplete). */
int disk_device_status(void *stream);

/* Self-test of the bounded waits (failure detection without a GPU fault):
 * launches one block that arms a tile-copy barrier no copy will complete and
 * waits at most `iterations` polls (1 .. 2^24), then records
 * DISK_ERR_TIMEOUT in the device status word exactly as a layer kernel whose
 * copy did not land would; a following disk_device_status reports it.
 * Asynchronous on `stream`. */
int disk_selftest_bounded_wait(long long iterations, void *stream);

/* Records every layer's launch choice for disk_sv_filter at this (H, W, C,
 * dtype) in the basis handle: choice int[L] with the codes that
 * disk_sv_filter_autotune reports (2 or 4; 8 followed by 0 for a fused
 * pair).  DISK_ERR_INVALID_ARG for other codes or an 8 not followed by 0;
 * DISK_ERR_UNSUPPORTED where a tile or pair does not fit shared memory. */
int disk_sv_filter_set_layers(const disk_basis *basis, int H, int W, int C, int dtype,
                              const int *choice);

/* Records one tile configuration (pixels per thread: 2 or 4) for every
 * layer, for this (H, W, C, dtype), in the basis handle. */
int disk_sv_filter_set_tile(const disk_basis *basis, int H, int W, int C, int dtype,
                            int pix);

/* ---------------------------------------------------------------------------
 * Dense spatially varying convolution (Sec. 3.1 Eq. 1 per pixel), the
 * reference DISK approximates and its speed baseline:
 *   out[x] = sum_m K_x[m] * I[clamp(x - m)],  K_x = sum_k alpha_k(x) D_k,
 * with the same alpha(x) as disk_sv_filter over the dense node kernels D_k.
 * The x - m indexing is true convolution, which is what a fitted complex
 * reproduces (its impulse response is its gather stencil reflected).
 * d_lut: float [B][Kd][Kd] node kernels (Kd odd, centre (Kd-1)/2, Kd <= 85),
 *   node order as for a basis.  Other arguments as disk_sv_filter.  No
 *   scratch. */
int disk_dense_sv(int dims, const int *n_nodes, const float *node_vals,
                  const float *d_lut, int Kd, const void *d_in, size_t in_pitch,
                  void *d_out, size_t out_pitch, int H, int W, int C,
                  int dtype, const float *d_maps, void *stream);

/* ---------------------------------------------------------------------------
 * Impulse-response synthesis (Sec. 4.4 Eq. 10; the composite of Eq. 4).
 *
 * For each of `batch` shift-invariant complexes d_theta [batch][L][T][3]
 * (pixels), the response to a unit impulse at the centre of a zero-padded
 * plane (nothing is truncated), cropped to K x K about the centre, into
 * d_out [batch][K][K] (float).  K odd, 1 <= K <= 257.  max_reach (<= 256)
 * bounds every |dx|, |dy| of d_theta and sizes the canvases; a complex with a
 * tap beyond it (or a non-finite value) gets NaN in every output element.
 * Scratch: 2 * batch canvases of side 2 * ((K-1)/2 + L*(ceil(max_reach)+1)
 * + 1) + 1 floats from the library's memory pool. */
int disk_synth_kernel(const float *d_theta, int batch, int L, int T, int K,
                      float max_reach, float *d_out, void *stream);

/* ---------------------------------------------------------------------------
 * Differentiable fit (Sec. 4.1 Eq. 4-5): for each of `batch` dense targets,
 * the complex theta minimising the loss between its impulse response
 * (Eq. 10) and the target, by Adam (beta 0.9/0.999, eps 1e-8) with the
 * learning rate decayed linearly from lr0 to lr1 over `steps` (Sec. 5.1).
 *
 * d_targets: the batch's targets packed back to back, target b a float
 *   [K_b][K_b] block (K_b = sizes[b], odd, <= 257, centre (K_b-1)/2).
 * sizes: host int[batch].
 * loss: DISK_LOSS_MSE = sum over the plane of (K_syn - K_tgt)^2 / K^2 with
 *   the target zero-padded; DISK_LOSS_CHARB = sum of (sqrt(d^2 + eps^2) - eps)
 *   / K^2 (Charbonnier, Eq. 11; eps > 0).
 * init: DISK_INIT_GIVEN (d_theta_io holds the start), DISK_INIT_IR (Eq. 6,
 *   ring step matching the target's second moment), DISK_INIT_SS (Sec. 4.2:
 *   layer 1 from dart throwing over the target's non-zero pixels with the
 *   Eq. 7 radius, SplitMix64 seeded with `seed`; later layers Eq. 6 rings),
 *   DISK_INIT_RAND (offsets uniform in +-(K-1)/(2L), SplitMix64).
 * Offsets are optimised in units of s_b = max(1, (K_b-1)/2) and clamped to
 * |o| <= s_b per axis (from the start, whatever the init); weights are raw.
 * d_theta_io: float [batch][L][T][3] (pixels): start (GIVEN) and result.
 * d_final_loss: float [batch], loss at the result (may be NULL).
 * d_loss_hist: float [batch][steps+1], loss before every step and after the
 *   last (may be NULL).
 * Limits: L * T <= 512.  Launches: a plan upload (per-target offsets carried
 * in kernel parameters, one launch per 512 targets), one init kernel (unless
 * GIVEN) and one persistent kernel, one CTA per target, largest targets
 * first.  Never synchronises, so a call can be captured in a CUDA graph.
 * Scratch:
 * (L+3) canvases of side 2*max((K_b-1)/2, (L+1)*(ceil(s_b)+1))+3 per target
 * from the library's memory pool. */
enum { DISK_LOSS_MSE = 0, DISK_LOSS_CHARB = 1 };
enum { DISK_INIT_GIVEN = 0, DISK_INIT_IR = 1, DISK_INIT_SS = 2, DISK_INIT_RAND = 3 };

int disk_fit(const float *d_targets, const int *sizes, int batch, int L, int T,
             int steps, float lr0, float lr1, int init, int loss, float eps,
             uint64_t seed, float *d_theta_io, float *d_final_loss,
             float *d_loss_hist, void *stream);

/* Checkpointed form of disk_fit (same optimisation, Sec. 4.1 Eq. 4-5 with
 * the Sec. 5.1 schedule): runs steps step0 .. step0+steps-1 of a fit whose
 * learning rate decays linearly from lr0 to lr1 over total_steps steps, with
 * the optimiser's state carried in d_state, so that a fit can be stopped,
 * saved and continued.
 * d_state: float [batch][3][L*T*3], per target the optimised variables (the
 *   offsets in units of s_b, clamped to [-1, 1], and the raw weights, in the
 *   [L][T][3] order of theta), then Adam's first and second moments in the
 *   same order.  step0 == 0: the start is built as disk_fit builds it for
 *   `init` and `seed` (DISK_INIT_GIVEN: from d_theta_io; moments zero) and
 *   d_state's contents are ignored; step0 > 0: the state is read from d_state
 *   (offsets clamped again, an identity on any state this call wrote), and
 *   d_theta_io's contents, init and seed are ignored.  On return d_state holds
 *   the state after the call's last step and d_theta_io the corresponding
 *   complex (pixels).
 * d_loss_hist: float [batch][steps+1], loss before each step of this call and
 *   after its last (may be NULL).  d_final_loss as disk_fit.
 * A fit of n steps split into calls [0, k) and [k, n) returns, bit for bit,
 * what one disk_fit of n steps with the same init and seed returns, as long
 * as both run in the same launch configuration (disk_fit_set_config).
 * DISK_ERR_INVALID_ARG for a null d_state, a bad init, or unless
 * 0 <= step0 <= step0 + steps <= total_steps <= 10^6.  Other arguments,
 * limits, launches and scratch as disk_fit (the init kernel only when
 * step0 == 0 and init is not DISK_INIT_GIVEN). */
int disk_fit_resume(const float *d_targets, const int *sizes, int batch, int L, int T,
                    int step0, int steps, int total_steps, float lr0, float lr1,
                    int init, int loss, float eps, uint64_t seed, float *d_state,
                    float *d_theta_io, float *d_final_loss, float *d_loss_hist,
                    void *stream);

/* Launch-configuration autotuner of disk_fit: times the persistent fit kernel
 * in each built configuration -- 256, 512 or 1024 threads per CTA, and one
 * CTA or a thread-block cluster of 2 or 4 CTAs (on as many SMs) per target --
 * for a few steps each from the sparse-sampling initialisation (seed 0) on
 * this batch, and
 * records the fastest for every later disk_fit with the same L, T and largest
 * target size (in 32-pixel buckets); without a recorded choice disk_fit uses
 * 512 threads, one CTA per target.  Synchronises the stream (do not call
 * while capturing a graph).  *chosen_config (may be NULL) receives the
 * choice as threads * 16 + CTAs per target. */
int disk_fit_autotune(const float *d_targets, const int *sizes, int batch, int L,
                      int T, int loss, float eps, int *chosen_config, void *stream);

/* Records a launch configuration (threads * 16 + CTAs per target, one of
 * those disk_fit_autotune tries) for disk_fit calls with this L, T and
 * largest target size kmax.  DISK_ERR_INVALID_ARG for any other value. */
int disk_fit_set_config(int L, int T, int kmax, int config);

/* One evaluation of the fit objective and its gradient (the hand-written
 * backward of the cascade: d/dw, d/ddx, d/ddy of every tap, through the
 * adjoint of each layer), at d_theta [batch][L][T][3] (pixels, offsets
 * clamped to |o| <= s_b as in disk_fit), into d_loss [batch] and
 * d_grad [batch][L][T][3] (pixel units).  Other arguments as disk_fit.  At an
 * exact integer offset the derivative is the one-sided one of the floor
 * convention (fraction in [0, 1)). */
int disk_fit_loss_grad(const float *d_targets, const int *sizes, int batch, int L,
                       int T, int loss, float eps, const float *d_theta,
                       float *d_loss, float *d_grad, void *stream);

/* ---------------------------------------------------------------------------
 * Learned initializer of the fit.  The paper initialises with Eq. 6 / Eq. 7;
 * this network (a project addition) predicts a complex from the target so
 * that the Eq. 4 fit starts closer to its optimum.  A multilayer perceptron:
 * input the target area-resampled to side x side and scaled to a maximum of
 * 1 (disk_downsample_targets), `depth` ReLU hidden layers of width `hidden`,
 * linear output of L*T*3 values (offsets in units of the target half-width
 * max(1, (K-1)/2), weights raw).  Parameters: a flat float array, for each
 * layer W [n_in][n_out] row-major then b [n_out].  FP32 throughout.
 * ------------------------------------------------------------------------- */

/* Number of parameters (-1 for an invalid shape). */
long long disk_mlp_param_count(int n_in, int hidden, int depth, int n_out);

/* He-uniform weights U(+-sqrt(6 / n_in)) from SplitMix64 at counter
 * seed + element index, zero biases. */
int disk_mlp_init(float *d_params, int n_in, int hidden, int depth, int n_out,
                  uint64_t seed, void *stream);

/* d_y [batch][n_out] = network(d_x [batch][n_in]).  Scratch: two
 * [batch][hidden] planes. */
int disk_mlp_forward(const float *d_params, int n_in, int hidden, int depth,
                     int n_out, const float *d_x, int batch, float *d_y,
                     void *stream);

/* One training step on a batch: mean squared error between network(d_x)
 * and d_target [batch][n_out] into *d_loss (device float), its gradient by
 * the hand-written backward pass, and one Adam update (beta 0.9 / 0.999,
 * eps 1e-8, step counted from 1) of d_params with moments d_m, d_v (same
 * size, caller-zeroed before the first step). */
int disk_mlp_train_step(float *d_params, float *d_m, float *d_v, int step,
                        float lr, int n_in, int hidden, int depth, int n_out,
                        const float *d_x, const float *d_target, int batch,
                        float *d_loss, void *stream);

/* The two halves of disk_mlp_train_step, for data-parallel training (each
 * rank computes the gradient of its own batch, the ranks average the
 * gradients with one all-reduce, every rank applies the same update):
 * disk_mlp_grad writes the loss of the batch (mean squared error, device
 * float) and its gradient d_grad (one float per parameter, layout of the
 * parameters); disk_mlp_adam applies one Adam update with that gradient
 * (as disk_mlp_train_step; step counted from 1). */
int disk_mlp_grad(const float *d_params, int n_in, int hidden, int depth, int n_out,
                  const float *d_x, const float *d_target, int batch, float *d_grad,
                  float *d_loss, void *stream);
int disk_mlp_adam(float *d_params, float *d_m, float *d_v, const float *d_grad, int step,
                  float lr, int n_in, int hidden, int depth, int n_out, void *stream);

/* Area resampling of `batch` packed targets (as for disk_fit; sizes host
 * int[batch], <= 4096) to d_out [batch][side][side], each scaled to a
 * maximum of 1: output cell (j, i) averages the input pixels it overlaps,
 * weighted by overlap area.  Copies the small size table from pageable host
 * memory (not capturable in a graph). */
int disk_downsample_targets(const float *d_targets, const int *sizes, int batch,
                            int side, float *d_out, void *stream);

/* The learned start of the fit, every step on the device.  The paper starts
 * the Eq. 4 fit from Eq. 6 rings or Eq. 7 sparse samples (Sec. 4.1-4.2);
 * this project adds the network above and uses the fitted loss to judge it:
 *   1. each target is area-resampled to side x side (disk_downsample_targets);
 *   2. the network (d_params, n_in = side * side, `hidden`, `depth`,
 *      n_out = L * T * 3) maps it to network units;
 *   3. network units -> pixels: offsets clamped to [-1, 1] and multiplied by
 *      the half-width s_b = max(1, (K_b - 1) / 2), weights divided by T;
 *   4. the Eq. 6 start is built as disk_fit does for DISK_INIT_IR;
 *   5. the loss (`loss`, `eps` as in disk_fit) of both starts is evaluated,
 *      and per target the network start is kept if its loss is <= the Eq. 6
 *      start's (a NaN loss keeps the Eq. 6 start).
 * d_targets, sizes, batch, L, T: as disk_fit (sizes odd, <= 257).
 * d_theta_out: float [batch][L][T][3] (pixels, device, caller-owned): the
 *   chosen start, ready for disk_fit with DISK_INIT_GIVEN.
 * d_used_network: int [batch] (device, may be NULL): 1 where the network
 *   start was kept, else 0.
 * Scratch: batch * (side^2 + 4 L T 3 + 3) floats from the library's memory
 * pool.  Copies a small per-target table from pageable host memory (not
 * capturable in a graph).  Errors: DISK_ERR_INVALID_ARG for null pointers,
 * bad shapes or even sizes; otherwise those of the steps it runs. */
int disk_learned_init(const float *d_targets, const int *sizes, int batch, int L, int T,
                      const float *d_params, int side, int hidden, int depth, int loss,
                      float eps, float *d_theta_out, int *d_used_network, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DISK_H */
