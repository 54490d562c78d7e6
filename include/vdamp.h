/*
 * vdamp.h -- C ABI of the GB300 VDAMP library.
 *
 * VDAMP (variable-density approximate message passing, Algorithm 1 of
 * Millard, Hess, Mailhe and Tanner, "An approximate message passing algorithm
 * for rapid parameter-free compressed sensing MRI") reconstructs an image x0
 * from y = Phi x0 + eps (Eq. 1) with Phi = M_Omega F (Sec. 1): F the unitary
 * 2D DFT, M_Omega a Bernoulli variable-density row selection.  Every step of
 * the iteration runs in this library's CUDA kernels (sm_103a); there is no
 * CPU fallback.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex arrays are interleaved float32 (re, im) pairs, i.e. complex64.
 * - Image and k-space arrays are [batch][ny][nx] row-major; k-space is
 *   unshifted (DC at index 0, signed frequency i for i < n/2, else i - n).
 *   F and F^H are unitary (1/sqrt(ny nx) each way).
 * - Psi is an orthonormal periodic 2D wavelet transform with `levels` = s
 *   scales: a[n] = sum_k h[k] x[(2n+k) mod L], d[n] = sum_k g[k] x[(2n+k) mod L],
 *   g[k] = (-1)^k h[len-1-k], h the minimum-phase Daubechies filter
 *   (Haar: 2 taps, DB4: 8 taps, 4 vanishing moments).
 * - Wavelet coefficients are "packed": [batch][ny*nx] complex, the 1 + 3s
 *   subbands of Eq. 6 stored one after another in the order
 *   A_s, H_s, V_s, D_s, H_{s-1}, V_{s-1}, D_{s-1}, ..., H_1, V_1, D_1
 *   (H high-pass along x, V along y, D along both), each row-major with
 *   (ny >> j) x (nx >> j) entries at level j.  B = 1 + 3s.
 * - Per-iteration outputs tau, thr, alpha are double [batch][iters][B]:
 *   tau is the colored noise estimate of Algorithm 1 line 5, thr the
 *   absolute soft threshold theta_b = lambda_b tau_b (same units as |r|) of
 *   the SURE-tuned denoiser (Sec. 3), alpha the subband-mean derivative of
 *   line 7.
 * - "device" pointers must be CUDA device (or managed) memory of the current
 *   device; "host" pointers ordinary CPU memory.  The caller owns every
 *   buffer it passes; the plan owns its own workspace.
 * - Calls that take a stream are asynchronous on it (NULL = legacy default
 *   stream); they return VDAMP_EINVAL without launching anything when an
 *   argument is invalid.  Errors met inside kernels (a non-finite tau or
 *   alpha) are recorded in the plan and read with vdamp_device_status().
 * - A plan may be used by one host thread at a time.
 */
#ifndef VDAMP_H
#define VDAMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VDAMP_OK = 0,
    VDAMP_EINVAL = 1,    /* invalid argument; nothing was launched          */
    VDAMP_ENOMEM = 2,    /* a device or host allocation failed              */
    VDAMP_ECUDA = 3,     /* a CUDA runtime call failed (see last_error)     */
    VDAMP_ENUMERIC = 4,  /* tau or alpha became non-finite during a solve   */
    VDAMP_ETIMEOUT = 5   /* a bounded device wait ran out                   */
} vdamp_status;

typedef enum { VDAMP_HAAR = 1, VDAMP_DB4 = 4 } vdamp_wavelet;

typedef struct vdamp_plan vdamp_plan;

/* Thread-local text of the last error raised by any call on this thread. */
const char* vdamp_last_error(void);

/*
 * Create a plan for ny x nx slices with wavelet `wavelet` at `levels` scales
 * (Algorithm 1 "Require": Psi; line 1: S = |Phi Psi^H|^2 is tabulated here
 * from its 1 + 3s unique columns, Sec. 2).  Sizes: ny and nx divisible by
 * 2^levels, of the form 2^a 3^b 5^c, 8 <= n <= 1024; 1 <= levels <= 6;
 * 1 <= max_batch; 1 <= max_iters <= 100000 (the most iterations any solve on
 * the plan may run; it sizes the plan's staging of the per-iteration outputs
 * of vdamp_solve_host and vdamp_solve_batched).  Finest subbands above 32768
 * coefficients (ny nx > 131072, e.g. 512 x 512) always take the split SURE
 * search (tuning entry 7 >= 4).  Allocates the device workspace for up to
 * max_batch slices on the current device (the input staging of the host and
 * descriptor entry points on their first call).  On success *out holds the plan; on failure *out is
 * NULL and the status says why.
 */
vdamp_status vdamp_plan_create(vdamp_plan** out, int ny, int nx, int wavelet, int levels,
                               int max_iters, int max_batch);

/* Release the plan and its device memory (waits for its work to finish). */
vdamp_status vdamp_plan_destroy(vdamp_plan* plan);

/* Number of subbands B = 1 + 3 levels, or -1 for a NULL plan. */
int vdamp_num_subbands(const vdamp_plan* plan);

/* Bytes of device workspace the plan holds. */
size_t vdamp_workspace_bytes(const vdamp_plan* plan);

/* Option switches.
 *   VDAMP_OPT_GRAPH (default 1): replay solves from a cached CUDA graph;
 *     0 launches every kernel directly.
 *   VDAMP_OPT_KERNEL_TIMING (default 0): launch directly and bracket every
 *     kernel with CUDA events on its stream; read with vdamp_kernel_times().
 *   VDAMP_OPT_FUSED (default 0): run vdamp_solve as one persistent launch in
 *     which a thread-block cluster iterates each slice (when the device can
 *     hold such a cluster); 0 runs one kernel per step of the iteration.
 *     Both give the same results up to the order of the tau partial sums.
 *   VDAMP_OPT_OVERLAP (default 1): in vdamp_solve (and the batched and
 *     grouped solves), search the three finest subbands on a second stream of
 *     the plan while the coarser scales of Psi, their search and the coarser
 *     scales of the next Psi^H run (with the split search, and with the pruned
 *     one when the finest subbands are its one-CTA subbands); with the split
 *     search the subbands of every scale below the coarsest likewise, each
 *     scale on a stream of its own; 0 keeps one stream.  The same kernels
 *     with the same arguments: identical results. */
enum { VDAMP_OPT_GRAPH = 1, VDAMP_OPT_KERNEL_TIMING = 2, VDAMP_OPT_FUSED = 3, VDAMP_OPT_OVERLAP = 4 };
vdamp_status vdamp_plan_set_option(vdamp_plan* plan, int option, int value);

/* Kernel kinds reported by vdamp_kernel_times. */
enum {
    VDAMP_KERNEL_IDWT = 0,      /* one synthesis scale of Psi^H (+ line 8 / line 6 prologue) */
    VDAMP_KERNEL_FFT_ROWS = 1,  /* row pass of F or F^H */
    VDAMP_KERNEL_COL_PASS = 2,  /* column pass of F and F^H with lines 3-5 fused */
    VDAMP_KERNEL_DWT = 3,       /* one analysis scale of Psi (+ r~ of line 4) */
    VDAMP_KERNEL_SURE = 4,      /* SURE threshold, alpha, tau (lines 5-7) */
    VDAMP_KERNEL_OTHER = 5,     /* line-8 write-out, sigma upload */
    VDAMP_KERNEL_FUSED = 6,     /* the persistent cluster solve (all steps) */
    VDAMP_KERNEL_KINDS = 7
};

/* With VDAMP_OPT_KERNEL_TIMING on: wait for the timed launches, then add up
 * their event-measured durations per kind since the last call.  ms and
 * counts hold VDAMP_KERNEL_KINDS entries each (milliseconds, launches). */
vdamp_status vdamp_kernel_times(vdamp_plan* plan, double* ms, int* counts);

/* Number of kernel launches (graph kernel nodes included) made by the last
 * solve/iterate/transform call on this plan. */
int vdamp_last_launch_count(const vdamp_plan* plan);

/*
 * Launch shapes of a plan ("tuning"), int[VDAMP_TUNING_LEN]:
 *   [0] columns per CTA of the column pass: 2, 4, 8 or 16 (dividing nx)
 *   [1] rows per CTA of the row pass: 1, 2, 4 or 8
 *   [2] synthesis (Psi^H) tile side in pixels: 16, 32 or 64
 *   [3] analysis (Psi) tile side in coefficients: 16 or 32
 *   [4], [5] radix plan of the transform along y and x: 0 = radix 8 first,
 *            1 = radix 4 only, 2 = radix 8 with the radices 3 and 5 first
 *   [6] 1: the scales s .. 2 of Psi (and of Psi^H) in one launch, one
 *       thread-block cluster per slice, scale 1 in its own launch, while
 *       batch x cluster size <= the SM count; 2: any batch, the coarse
 *       scales (from the first whose synthesis output is at most 128 x 128)
 *       in one launch, a cluster of up to 4 CTAs per slice, the finer
 *       scales in their own launches; 0: one launch per scale
 *   [7] parts per subband of the SURE threshold search (Algorithm 1 lines
 *       6-7): 1 = one CTA per subband bounds SURE per bucket of magnitudes,
 *       sorts only the candidate buckets and searches them (subbands with
 *       too many candidates take the full sort in a second, one-wave kernel);
 *       2, 4 or 8 = subbands above 2048 coefficients split over up to that
 *       many CTAs (a sort and a search launch); 0 = 8 while the CTAs of the
 *       split (batch x the parts of all subbands) fit on the SMs at once,
 *       else 1
 * Every tuning computes the same method; tunings differ in FP32 summation
 * order only (the tau partial sums depend on [0], the DFT on [4], [5], the
 * FP32 candidate sums of the SURE search on [7]).
 * get copies the current tuning out; set validates and applies one
 * (VDAMP_EINVAL for an unsupported value, nothing changed) and drops the
 * plan's cached graphs.
 */
#define VDAMP_TUNING_LEN 8
vdamp_status vdamp_plan_get_tuning(const vdamp_plan* plan, int* tuning);
vdamp_status vdamp_plan_set_tuning(vdamp_plan* plan, const int* tuning);

/*
 * Autotuner: times a solve of max(trials, 2) iterations (Algorithm 1 lines
 * 3-8 and the return line) of `batch` synthetic slices, captured in one CUDA
 * graph as vdamp_solve captures it (side streams included), per candidate on
 * `stream` and keeps, one parameter after another (coordinate descent over
 * the tuning above, starting from the current one), the fastest shape.  Blocks until done; allocates and frees
 * its own temporary device buffers (about 6 batch ny nx complex values).
 * Writes the chosen tuning to `tuning` (int[VDAMP_TUNING_LEN]) if not NULL.
 */
vdamp_status vdamp_plan_autotune(vdamp_plan* plan, int batch, int trials, int* tuning,
                                 void* stream);

/*
 * One group of same-size slices for vdamp_solve_groups: the arguments of
 * vdamp_solve for a cold start (r_tilde0 = NULL), without the optional
 * outputs.  Each group has its own plan (the plan's size fixes the slices').
 */
typedef struct {
    vdamp_plan* plan;
    int batch;
    const float* y;          /* device [batch][ny][nx] complex64 */
    const uint8_t* mask;     /* device [batch][ny][nx] */
    const float* density;    /* device [batch][ny][nx] */
    const float* sigma;      /* host [batch] */
    int iters;
    float* x_hat;            /* device [batch][ny][nx] complex64 out */
    double* tau;             /* device [batch][iters][B] out */
    double* thr;
    double* alpha;
} vdamp_group;

/*
 * Mixed-size batched VDAMP: solves `count` groups (1 <= count <= 64, each
 * with a distinct plan) as ONE CUDA graph launch on `stream`, in which every
 * group's kernels run on a branch of their own, so that groups of different
 * slice sizes overlap on the GPU.  The graph is cached per argument set (the
 * sigma values are uploaded before each launch).  Results are identical to
 * solving each group with vdamp_solve.  Errors met inside kernels are
 * recorded per plan (vdamp_device_status).  With graphs off on the first
 * plan, or kernel timing on any, the groups run one after another.
 */
vdamp_status vdamp_solve_groups(const vdamp_group* groups, int count, void* stream);

/* ======================================================================
 * Learned per-subband denoiser (operations).  A 5-layer network of 3x3
 * convolutions per subband index b stands in for the soft threshold:
 *   f(r) = r - sqrt(tau_b) n_b(r / sqrt(tau_b), 0.1 ln tau_b),
 * n_b: conv 3->32, ReLU, 3 x (conv 32->32, ReLU), conv 32->2, zero padding
 * at the subband border.  The paper only anticipates such a denoiser (its
 * concluding section); these operations are the building blocks of its
 * inference, its Monte-Carlo divergence and its training.
 *
 * Images: the network runs on a list of n_img images, given as a device
 * int array [n_img][9] = (off, h, w, tile0, src_off, src_pitch, band, slice,
 * ctile0): image i has h x w pixels stored densely in the activation arrays
 * from pixel `off` on; its 128-pixel tiles (elementwise operations) are
 * tile0 .. tile0 + ceil(h w / 128) - 1 and its convolution tiles ctile0 ..
 * ctile0 + ceil(w / Wb) ceil(h / R) - 1 (blocks of R = floor(128 / (Wb + 2))
 * rows and Wb = min(w, 30) columns; both ascending with i; total_tiles /
 * conv_tiles_total = the sums over images); src_off and
 * src_pitch locate its top-left coefficient and row pitch in packed complex
 * arrays (r, w0, f); band selects the weight set; slice selects tau.
 * Activations are BF16 [pixel][C] with C = 16 or 32 channels.  Weights are
 * FP32 [bands][cout][9][cin] (tap t = 3 (dy + 1) + (dx + 1)), packed by
 * vdamp_cnn_pack_weights into BF16 operand images [bands][cout_pad x 9
 * cin_pad] for the tensor cores.  Calls are asynchronous on `stream`;
 * VDAMP_EINVAL (nothing launched) for invalid arguments.
 * ==================================================================== */

/* 3x3 convolution of every image (zero padding), BF16 x BF16 -> FP32 on the
 * tensor cores; mirror = 1 negates the tap offsets (transposed convolution).
 * max_w: the largest image width (>= 1; it sizes the shared-memory halo). 
 * mode 0: out = relu(acc + bias) BF16 [pixel][cout_pad]
 * mode 1: out = acc * (mask > 0)  BF16, mask BF16 [pixel][cout_pad]
 * mode 2: out = acc + bias        FP32 [pixel][cout_store]
 * mode 3: out = acc               FP32 [pixel][cout_store]
 * bias FP32 [bands][cout_pad].  status: device int set to 1 if a bounded
 * wait for the tensor cores ran out (the outputs are then incomplete). */
vdamp_status vdamp_cnn_conv3x3(const void* in, int cin_pad, const void* wimg, int cout_pad,
                               const float* bias, const void* mask, void* out, int mode,
                               int mirror, int cout_store, const int* images, int n_img,
                               int conv_tiles_total, int max_w, int* status, void* stream);

/* Failure detection of the convolution's bounded waits.  Each tile's
 * tensor-core result is awaited on an mbarrier for at most `polls` polls
 * (default vdamp_cnn_default_wait_limit(), about 1.7e7); when that runs out
 * the kernel sets its status to 1, gives the operations still in flight one
 * more wait of the default length, frees its tensor memory and returns, so
 * the context stays usable.  vdamp_cnn_set_wait_limit sets the first limit
 * for convolutions launched afterwards by this process (0 gives up at once,
 * which is how the tests exercise this path) and returns the old one in
 * *previous (may be NULL).  vdamp_cnn_status waits for `stream`, reads and
 * clears a status word written by vdamp_cnn_conv3x3 and returns VDAMP_OK or
 * VDAMP_ETIMEOUT. */
vdamp_status vdamp_cnn_set_wait_limit(unsigned polls, unsigned* previous);
unsigned vdamp_cnn_default_wait_limit(void);
vdamp_status vdamp_cnn_status(int* status, void* stream);

/* FP32 weights [bands][cout][9][cin] -> BF16 operand images; transpose = 1
 * packs the transposed convolution (cin outputs from cout inputs) used for
 * the gradient with respect to the layer input (with mirror = 1). */
vdamp_status vdamp_cnn_pack_weights(const float* w, int bands, int cin, int cout, int cin_pad,
                                    int cout_pad, int transpose, void* img, void* stream);

/* Weight and bias gradients of a convolution: dw[band][co][tap][ci] +=
 * sum_p x[p + offset(tap)][ci] dy[p][co], db[band][co] += sum_p dy[p][co]
 * (FP32; band < 32).  Each CTA's sums over its tiles are stored as records and
 * then added per band in record order, so the result does not depend on the
 * order in which CTAs run.  The records live in a device buffer the library
 * grows on demand and keeps (about total_tiles (9 cin cout + cout) floats);
 * calls that overlap on the GPU share it and must not run concurrently. */
vdamp_status vdamp_cnn_wgrad(const void* x, int cin, int cin_pad, const void* dy, int cout,
                             int cout_pad, const int* images, int n_img, int total_tiles,
                             float* dw, float* db, void* stream);

/* Input planes: x[p] = (Re r / sqrt(tau), Im r / sqrt(tau), 0.1 ln tau, 0...)
 * BF16 [pixel][16], r packed complex64, tau double [slices][B]. */
vdamp_status vdamp_cnn_input(const float* r, const double* tau, int B, const int* images,
                             int n_img, int total_tiles, void* x, void* stream);

/* Hutchinson probe: t0[p] = (eta_re, eta_im, 0...) BF16 [pixel][16], eta
 * Rademacher from splitmix64 (Steele, Lea and Flood 2014) of
 * seed + golden_gamma (2 key + c + 1), key = the packed index of the
 * coefficient, c = 0 (re) or 1 (im), sign from bit 0. */
vdamp_status vdamp_cnn_probe(unsigned long long seed, const int* images, int n_img,
                             int total_tiles, void* t0, void* stream);

/* Residual output and its statistics: f = r - sqrt(tau) n written at the
 * images' packed positions (f may be NULL), and per image i
 *   sums[2 i]     += sum |f - r|^2
 *   sums[2 i + 1] += sum eta . (J_n eta)  (jn = the network's JVP output for
 *                    the probe of `seed`, FP32 [pixel][2]; NULL: 0)
 * n FP32 [pixel][2]; sums double, accumulated with atomics. */
vdamp_status vdamp_cnn_output(const float* r, const double* tau, int B, const int* images,
                              int n_img, int total_tiles, const float* n, const float* jn,
                              unsigned long long seed, float* f, double* sums, void* stream);

/* Training loss sum |f - w0|^2 * inv_count over the images (added to *loss,
 * double) and its gradient with respect to n, BF16 [pixel][16] (channels 0,
 * 1: -2 sqrt(tau) (f - w0) inv_count). */
vdamp_status vdamp_cnn_loss(const float* r, const float* w0, const double* tau, int B,
                            const int* images, int n_img, int total_tiles, const float* n,
                            float inv_count, void* dn, double* loss, void* stream);

/* Adam (Kingma and Ba) on n FP32 parameters, step >= 1 (bias corrected). */
vdamp_status vdamp_cnn_adam(float* p, const float* g, float* m, float* v, size_t n, float lr,
                            float beta1, float beta2, float eps, int step, void* stream);

/* Onsager step of the learned denoiser (Algorithm 1 lines 6-8) per subband
 * image i (subband b = band, slice s): with N_b = h w, div = 2 N_b - probe
 * and SURE_cnn = sum |f - r|^2 - N_b tau + tau div (sums from
 * vdamp_cnn_output), the network is used when SURE_cnn < sure_soft[s][b]
 * (the soft threshold's minimum SURE, vdamp_last_sure) and 0 <= div / (2 N_b)
 * < 1; then w_hat = f and alpha = div / (2 N_b), else w_hat = soft(r, thr)
 * and alpha = alpha_soft.  Writes r~ = (w_hat - alpha r) / (1 - alpha) and
 * (if not NULL) w_hat at the images' packed positions, use_out[i] (1 = the
 * network) and alpha_out[i].  f may be NULL (soft everywhere).  tau, thr,
 * alpha_soft, sure_soft: double [slices][B]. */
vdamp_status vdamp_cnn_onsager(const float* r, const float* f, const double* tau,
                               const double* thr, const double* alpha_soft,
                               const double* sure_soft, int B, const double* sums,
                               const int* images, int n_img, int total_tiles, float* r_tilde,
                               float* w_hat, int* use_out, double* alpha_out, void* stream);

/* Diagnostics of the one-CTA-per-subband threshold search (tuning entry 7 =
 * 1, chosen automatically for many slices): it bounds SURE per bucket of
 * magnitudes and sorts only the buckets that can hold the minimiser; a
 * subband whose candidates do not fit its tables (heavy ties, degenerate
 * data) is solved by the full sort and search instead.  Waits for `stream`
 * and writes to *count how many subbands took that path since the plan was
 * created (Sec. 3's minimiser either way). */
vdamp_status vdamp_sure_fallback_count(vdamp_plan* plan, int* count, void* stream);

/* Minimum SURE value of each subband at the last threshold search (solve
 * or iterate) of this plan: double [batch][B], copied to `out` (device or
 * host) asynchronously on `stream`. */
vdamp_status vdamp_last_sure(vdamp_plan* plan, int batch, double* out, void* stream);

/*
 * VDAMP solve, Algorithm 1 lines 1-10 with the SURE soft threshold of Sec. 3,
 * on `batch` independent slices (1 <= batch <= max_batch).
 *   y         device  [batch][ny][nx] complex64  measurements (ignored off the mask)
 *   mask      device  [batch][ny][nx] uint8      1 where the frequency is sampled
 *   density   device  [batch][ny][nx] float32    sampling probability p; 0 < p <= 1
 *                                                wherever mask = 1 (P of Algorithm 1)
 *   sigma     host    [batch] float32            noise level sigma_eps (Eq. 1), >= 0
 *   iters     number of iterations, 1 <= iters <= max_iters of the plan
 *   r_tilde0  device  [batch][ny*nx] complex64 packed, or NULL: starting r~_0
 *                     (NULL = 0 as in line 1; non-NULL resumes a stopped run)
 *   k0        index of the first iteration: 0 for a cold start, the number of
 *             iterations already run when resuming (Algorithm 1 does not
 *             depend on k, so k0 changes no result; vdamp_device_status
 *             reports iteration numbers k0 + k)
 *   x_hat     device  [batch][ny][nx] complex64 out: the return line applied to
 *                     the last denoiser output
 *   tau, thr, alpha  device  [batch][iters][B] double out (see conventions)
 *   r_tilde_out      device  [batch][ny*nx] complex64 out or NULL: r~ after the
 *                     last iteration (line 8), the state to resume from
 *   x_hat_iters      device  [iters][batch][ny][nx] complex64 out or NULL: the
 *                     return line applied to every w_hat_k (NMSE curves)
 * Asynchronous on `stream` (a cudaStream_t).  A solve that hits a non-finite
 * tau or alpha finishes its launches and records VDAMP_ENUMERIC for
 * vdamp_device_status().
 */
vdamp_status vdamp_solve(vdamp_plan* plan, int batch, const float* y, const uint8_t* mask,
                         const float* density, const float* sigma, int iters,
                         const float* r_tilde0, int k0, float* x_hat, double* tau, double* thr,
                         double* alpha, float* r_tilde_out, float* x_hat_iters, void* stream);

/*
 * The same solve on HOST buffers (same shapes as vdamp_solve; r_tilde0 may be
 * NULL).  Copies inputs to the plan's device staging, solves on `stream`,
 * copies x_hat, tau, thr and alpha back and waits.  Returns VDAMP_ENUMERIC
 * if the solve met a non-finite tau or alpha.
 */
vdamp_status vdamp_solve_host(vdamp_plan* plan, int batch, const float* y, const uint8_t* mask,
                              const float* density, const float* sigma, int iters,
                              const float* r_tilde0, int k0, float* x_hat, double* tau,
                              double* thr, double* alpha, void* stream);

/*
 * One slice of vdamp_solve_batched: the arguments of vdamp_solve for a single
 * slice of the plan's size, each in its own device buffers.
 */
typedef struct {
    const float* y;          /* device [ny][nx] complex64 measurements (ignored off the mask) */
    const uint8_t* mask;     /* device [ny][nx] uint8, 1 where sampled */
    const float* density;    /* device [ny][nx] float32 p, 0 < p <= 1 on the mask */
    float sigma;             /* noise level sigma_eps >= 0 (Eq. 1) */
    int iters;               /* iterations, 1 <= iters <= max_iters */
    const float* r_tilde0;   /* device [ny*nx] packed complex64 to resume from, or NULL */
    int k0;                  /* index of the first iteration (0 with r_tilde0 = NULL) */
    float* x_hat;            /* device [ny][nx] complex64 out (return line) */
    double* tau;             /* device [iters][B] out */
    double* thr;             /* device [iters][B] out */
    double* alpha;           /* device [iters][B] out */
} vdamp_slice_desc;

/*
 * Batched VDAMP from slice descriptors (Algorithm 1 per slice, as vdamp_solve):
 * `count` slices of the plan's size whose buffers lie anywhere in device
 * memory.  Slices that share (iters, k0, cold start or not) are solved
 * together, up to max_batch at a time, as one vdamp_solve on the plan's
 * staging: a kernel gathers their inputs into it and another scatters x_hat,
 * tau, thr and alpha back, so each slice's results equal those of vdamp_solve
 * on that slice.  Asynchronous on `stream`; VDAMP_EINVAL (nothing launched)
 * for an invalid descriptor; non-finite tau or alpha is recorded for
 * vdamp_device_status as in vdamp_solve.  Slices already contiguous in
 * memory are solved faster by vdamp_solve (no gather or scatter).
 */
vdamp_status vdamp_solve_batched(vdamp_plan* plan, const vdamp_slice_desc* slices, int count,
                                 void* stream);

/*
 * One pass of Algorithm 1 lines 3-8 from an explicit r~_k (device buffers as
 * in vdamp_solve):
 *   z_k = y - Phi Psi^H r~_k;  r_k = r~_k + Psi Phi^H P^{-1} z_k;
 *   tau_k (line 5); w_hat_k, theta_k (line 6, Sec. 3); alpha_k (line 7);
 *   r~_{k+1} = (w_hat_k - alpha_k r_k) / (1 - alpha_k) (line 8).
 * Outputs: r (packed r_k), tau/thr/alpha [batch][B], r_tilde_next (packed).
 */
vdamp_status vdamp_iterate(vdamp_plan* plan, int batch, const float* r_tilde, const float* y,
                           const uint8_t* mask, const float* density, const float* sigma,
                           float* r, double* tau, double* thr, double* alpha,
                           float* r_tilde_next, void* stream);

/*
 * Return line of Algorithm 1 for packed coefficients w (device):
 *   x_hat = Psi^H w + Phi^H (y - Phi Psi^H w).
 */
vdamp_status vdamp_final_estimate(vdamp_plan* plan, int batch, const float* w, const float* y,
                                  const uint8_t* mask, float* x_hat, void* stream);

/* Transforms on their own (device buffers, [batch] slices):
 *   vdamp_psi:    packed w = Psi x        (x image, [batch][ny][nx])
 *   vdamp_psi_h:  image  x = Psi^H w
 *   vdamp_fft2:   out = F in (inverse = 0) or F^H in (inverse = 1), unitary.
 * in and out must not overlap. */
vdamp_status vdamp_psi(vdamp_plan* plan, int batch, const float* x, float* w, void* stream);
vdamp_status vdamp_psi_h(vdamp_plan* plan, int batch, const float* w, float* x, void* stream);
vdamp_status vdamp_fft2(vdamp_plan* plan, int batch, const float* in, float* out, int inverse,
                        void* stream);

/*
 * Wait for the plan's last call on `stream` and report what its kernels
 * recorded: VDAMP_OK, or VDAMP_ENUMERIC with *iter (may be NULL) set to the
 * first iteration whose tau or alpha was non-finite.  Clears the record.
 */
vdamp_status vdamp_device_status(vdamp_plan* plan, int* iter, void* stream);

/* ---- host-only helpers (no GPU needed) ----------------------------------- */

/* The plan's analysis low-pass filter h for `wavelet`, derived in double by
 * Daubechies' spectral factorisation.  h must hold 8 doubles; *len gets the
 * tap count (2 or 8). */
vdamp_status vdamp_wavelet_filter(int wavelet, double* h, int* len);

/*
 * The 1D factors of S = |Phi Psi^H|^2 (Algorithm 1 line 1) along an axis of
 * length n: out[(2(j-1) + t) * n + k], j = 1..levels, t = 0 for the level-j
 * scaling atom and t = 1 for the level-j wavelet atom, is |F_n psi|^2 at
 * frequency k.  Column b of S is the outer product of the y and x factors of
 * its subband (A_s: scaling/scaling; H_j: scaling along y, wavelet along x;
 * V_j: wavelet/scaling; D_j: wavelet/wavelet).  out holds 2*levels*n doubles.
 */
vdamp_status vdamp_subband_spectra(int wavelet, int levels, int n, double* out);

/* ---- measurement of the machine ------------------------------------------ */

/*
 * Peak fused multiply-add throughput of the current GPU in FP32 (precision =
 * 32) or FP64 (64), in TFLOP/s (2 FLOP per FMA), from `iters` rounds of a
 * kernel of independent FMA chains (4 resident CTAs of 256 threads per SM,
 * 8 chains of 16 FMAs per thread and round): the denominator of the ALU
 * roofline of the transforms.  The paper has no counterpart; this measures
 * the machine, not the method.  Blocks until done (one warm-up launch, then
 * the fastest of three, timed with CUDA events on `stream`); *ms (may be
 * NULL) gets that launch's milliseconds.
 */
vdamp_status vdamp_fma_peak(int precision, int iters, double* tflops, double* ms, void* stream);

/* ---- no device allocation ------------------------------------------------ */

/* Largest ny or nx that vdamp_tau_estimate_noalloc accepts. */
#define VDAMP_NOALLOC_MAX_SIDE 1024

/*
 * The paper has no counterpart to this entry point: it is a service of the
 * library, not a step of the method.  It computes the same per-subband noise
 * estimate tau that a solve reports, tau_b = sum_i S[i,b] w_i ((w_i - 1)|z_i|^2
 * + sigma^2) with w = 1/p on the mask, from a k-space residual z, for callers
 * that cannot allocate device memory: code running inside a fixed device
 * memory pool or budget, hosts without an allocator, or tools that must not
 * disturb a caching allocator they share with other code.
 *
 * It needs no plan and calls no cudaMalloc, cudaFree or other allocating
 * routine.  Its device scratch (the S tables and per-block partial sums, about
 * 175 KB) is one fixed array inside the library that every GPU which loads
 * the library keeps until the process exits.  Limits: 8 <= ny, nx <=
 * VDAMP_NOALLOC_MAX_SIDE, of the form 2^a 3^b 5^c, divisible by 2^levels,
 * 1 <= levels <= 6; larger sizes return VDAMP_EINVAL with a message.
 *   z        device [ny][nx] complex64 residual (only entries with mask = 1 are read)
 *   mask     device [ny][nx] uint8;  density device [ny][nx] float32 (p, > 0 on the mask)
 *   sigma    noise level sigma_eps >= 0
 *   tau      device out [1 + 3 levels] double, subbands in packed order
 * Asynchronous on `stream`: the S tables are filled on the device by a kernel
 * of this call (from the filter taps, passed by value), so no host buffer is
 * read after the call returns.  The first call on each device looks up the
 * scratch address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  All calls share the one scratch
 * array and each overwrites it: calls that overlap on the GPU (different
 * streams, no ordering between them) race and give wrong results; calls on
 * one stream are ordered and correct.  Every partial sum is written before it
 * is read, so nothing needs clearing between calls.  A CUDA error already
 * pending when the call starts is returned as VDAMP_ECUDA with its text, and
 * nothing is launched.
 */
vdamp_status vdamp_tau_estimate_noalloc(int ny, int nx, int wavelet, int levels, const float* z,
                                        const uint8_t* mask, const float* density, float sigma,
                                        double* tau, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* VDAMP_H */
