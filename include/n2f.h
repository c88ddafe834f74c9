/*
 * n2f.h -- C ABI of the GB300 (sm_103a) Noise2Fast library.
 *
 * Noise2Fast (Lequyer, Philip, Sharma & Pelletier, arXiv 2108.10209) denoises ONE noisy image
 * x in R^{m x n} into f_theta(x) ~ s of the same size (Theoretical Background, Eq. 1-2) using
 * only that image: checkerboard downsampling into four sub-images (Eq. 6-7 and the Methods'
 * primed "left" equations), a small CNN (Methods, first paragraph: 3x3 conv + ReLU layers,
 * then 1x1 conv + sigmoid) trained with BCE and Adam (lr 0.001, batch size 1) on the four
 * input/target pairs of the Methods table, full-image validation after every epoch, and the
 * stopping rule: stop once 100 epochs pass without a better validation MSE and output the
 * average of the last 100 validation outputs (Methods, validation paragraph). The method is
 * blind: no noise parameter is passed.
 *
 * Conventions
 *   - Every entry point returns N2F_OK (0) or a negative N2F_E* code; n2f_strerror() gives
 *     text, including the CUDA error message of the last N2F_EDEVICE on this thread.
 *   - Images are row-major float32, H rows by W columns. "Host" pointers are ordinary CPU
 *     memory; "device" pointers are CUDA global memory on the context's device.
 *   - Nothing here takes or returns a PyTorch type. A stream is passed as a cudaStream_t
 *     cast to void* (NULL = the legacy default stream).
 *   - The library owns every device buffer it allocates (through the allocator in
 *     n2f_config, cudaMalloc when none is given) and frees it when a job is collected,
 *     cancelled or its context is destroyed.
 *   - Thread safety: n2f_submit / n2f_poll / n2f_wait / n2f_result / n2f_cancel may be called
 *     from any thread on the same context. Trainer and op-level calls are not thread-safe
 *     per object.
 */
#ifndef N2F_H
#define N2F_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------------------------ */
#define N2F_OK 0
#define N2F_EINVAL (-1)     /* NULL pointer, H or W < 2 or H*W >= 2^31, non-finite pixel, bad
                               struct_size/enum */
#define N2F_ETOOBIG (-2)    /* the job can never fit the context's HBM budget */
#define N2F_EAGAIN (-3)     /* result not ready yet */
#define N2F_ENOENT (-4)     /* unknown or already collected job */
#define N2F_ETIMEDOUT (-5)  /* a wait ran out of time */
#define N2F_ENONFINITE (-6) /* training diverged: a non-finite validation score */
#define N2F_EDEVICE (-7)    /* CUDA error (message kept for n2f_strerror) */
#define N2F_ENOMEM (-8)     /* an allocation failed */
#define N2F_ECANCELED (-9)  /* the job was cancelled */
#define N2F_ENOTSUP (-10)   /* a combination this build does not provide */

/* ---- enumerations ----------------------------------------------------------------------- */
enum n2f_precision {
  N2F_FP32 = 0, /* activations, weights, gradients and results in float32 (plain form); the
                   tensor-core GEMMs multiply two power-of-two-scaled fp16 parts of every
                   float32 operand (about 22 significant bits per product) */
  N2F_BF16 = 1  /* GEMM operands and stored activations in bfloat16, FP32 accumulation,
                   FP32 master weights, Adam and loss; FP64 validation-MSE reduction */
};
enum n2f_loss { N2F_LOSS_BCE = 0, N2F_LOSS_MSE = 1 };
enum n2f_widths {
  N2F_WIDTHS_PLIT = 0, /* 32,32,64,64,128,128,256,256: the Methods text read literally */
  N2F_WIDTHS_W64 = 1   /* eight 64-channel layers */
};
enum n2f_engine {
  N2F_ENGINE_AUTO = 0, /* tensor-core kernels where built for the precision, else SIMT */
  N2F_ENGINE_SIMT = 1, /* CUDA-core implicit-GEMM kernels (the FP32 reference kernels) */
  N2F_ENGINE_TC = 2    /* tcgen05/TMEM implicit-GEMM kernels for the C_in >= 32 layers */
};
enum n2f_job_state {
  N2F_QUEUED = 0, N2F_RUNNING = 1, N2F_DONE = 2, N2F_FAILED = 3, N2F_CANCELED = 4
};

/* ---- configuration ---------------------------------------------------------------------- */
typedef void* (*n2f_alloc_fn)(size_t bytes, void* user); /* device memory; NULL on failure */
typedef void (*n2f_free_fn)(void* ptr, size_t bytes, void* user);

/* Kernel classes the context can time with CUDA events on their launching stream. */
enum n2f_kernel_class {
  N2F_K_NONE = 0,
  N2F_K_CONV_FWD = 1,   /* 3x3 forward layers with C_in >= 8 (training and validation) */
  N2F_K_CONV_DGRAD = 2, /* 3x3 input-gradient layers */
  N2F_K_CONV_WGRAD = 3, /* 3x3 weight-gradient layers with C_in >= 8 (incl. their reduce) */
  N2F_K_FIRST = 4,      /* the one-channel first layer, forward */
  N2F_K_HEAD = 5,       /* the 1x1 + sigmoid head, training and validation */
  N2F_K_ADAM = 6,       /* Adam + operand packing */
  N2F_K_CONV = 7        /* forward and dgrad 3x3 layers with C_in >= 8 (one kernel template) */
};

typedef struct {
  uint32_t struct_size;      /* sizeof(n2f_config) */
  int device;                /* CUDA device ordinal */
  uint64_t hbm_budget_bytes; /* admission budget for resident job state; 0 = 150 GB */
  uint32_t max_slots;        /* jobs resident at once; 0 = 64 */
  uint32_t lookahead;        /* epochs enqueued ahead of the stop check; 0 = 2 */
  n2f_alloc_fn alloc;        /* optional device allocator (e.g. a framework's caching one) */
  n2f_free_fn free;
  void* alloc_user;
  int32_t profile_kernel;    /* enum n2f_kernel_class timed per launch (events), 0 = off */
  int32_t use_graphs;        /* 1: each job's epoch is captured once as a CUDA graph and
                                replayed (default); 0: kernels are launched one by one. */
  uint32_t group_size;       /* > 1: jobs admitted together with identical parameters (stopping
                                rule, not fixed steps) run in lockstep groups of up to this many
                                on one stream, the tensor-core forward and dgrad of each layer
                                as ONE persistent launch over all members' tiles, each member
                                with its own weights, size and stop flag; the group's epoch is
                                one CUDA graph. A member's result is ready when every member of
                                its group has stopped. Grouped jobs are not kernel-timed.
                                0 or 1: every job alone (default). */
  int32_t autotune;          /* 1: before a job's first epoch, the launch choices that leave
                                results unchanged (pipeline stages, CTAs per SM) are timed for
                                each of its conv shapes not seen before in this process and the
                                fastest kept; 0: fixed choices (default). */
  uint32_t profile_every;    /* with profile_kernel: the launches of every profile_every-th
                                epoch of a job are timed (its epoch graph is captured twice,
                                with and without the event records); 0 or 1: every epoch. */
} n2f_config;

enum n2f_downsample { N2F_DOWN_CHECKER = 0, N2F_DOWN_QUAD = 1 };

/* Per-image parameters. Defaults (n2f_params_default) follow the Methods section; the Adam
 * moments and epsilon are Kingma & Ba's defaults (the paper cites Adam without them). */
typedef struct {
  uint32_t struct_size; /* sizeof(n2f_params) */
  /* Adam's step size and constants, held in double like the method's own values: the kernels
   * take beta, 1 - beta (formed in double), lr and eps rounded once to float32, and the bias
   * corrections 1 - beta^t come from powers of the double beta. */
  double lr;            /* 1e-3 */
  double beta1, beta2;  /* 0.9, 0.999 */
  double eps;           /* 1e-8 */
  uint32_t patience;    /* 100 */
  uint32_t max_epochs;  /* safety cap, 0 = none */
  int32_t fixed_steps;  /* -1: stopping rule; k >= 0: k steps (pairs cycled), one validation */
  uint64_t seed;        /* SplitMix64 seed of the initial weights */
  int32_t precision;    /* enum n2f_precision */
  int32_t loss;         /* enum n2f_loss */
  int32_t widths;       /* enum n2f_widths */
  int32_t incl_best;    /* 0: the window is the 100 epochs after the best (the reading used) */
  int32_t engine;       /* enum n2f_engine */
  /* Input channels C_0 (1..4; 0 means 1) and the predicted channel 0..C_0-1. Fig. 2a's caption:
   * the network input may be multi-channel, its output is always one channel, and an RGB
   * image is denoised one channel per network. With C_0 > 1 the submitted image is C_0 planes
   * of H*W floats; every plane is downsampled alike, each pair's input is all C_0 planes of one
   * sub-image and its target the predicted plane of the paired sub-image, and validation
   * compares with that plane of the image. The result is one H*W plane. */
  int32_t channels;
  int32_t target_channel;
  /* Ablation Study variants (not the method; for comparisons on synthetic data):
   * downsample = N2F_DOWN_QUAD replaces the checkerboard sub-images by the four images of the
   * 2x2 blocks' top-left, top-right, bottom-right and bottom-left pixels (floor(H/2) x
   * floor(W/2)), trained on the pairs TL->TR, TR->BR, BR->BL, BL->TL (a reading: the paper
   * names the four images, not the pairs). exact = 1 takes the clean (ground-truth) plane of the
   * predicted channel as one more plane after the input planes and trains on the targets
   * x_tgt - (s_tgt - s_in), removing the signal-difference term of the Theoretical Background. */
  int32_t downsample;   /* enum n2f_downsample */
  int32_t exact;
  /* overlap = 1: a job that runs alone (not in a lockstep group, stopping rule) validates each
   * epoch's weights on a second stream while the next epoch trains: the weights and packed
   * copies are snapshot at the epoch boundary (one device copy) and the validation reads the
   * snapshot, so the validation scores, the stop epoch and the result are bit-identical to
   * overlap = 0. The epoch after the stop has then already run; its steps are discarded (Adam
   * state counters restored, the weights not used again). Costs one more set of validation
   * activations (2 x 256 x H x W elements) and the snapshot (theta and the forward weight
   * copies: about twice the weight count in floats with the tensor-core engine). A job in a
   * lockstep group validates in line with its group. 0: each validation runs in line after its
   * epoch (default). */
  int32_t overlap;
} n2f_params;

typedef struct {
  uint32_t struct_size;  /* sizeof(n2f_status) */
  int32_t state;         /* enum n2f_job_state */
  int32_t error;         /* N2F_E* when FAILED */
  uint32_t epoch;        /* epochs completed */
  uint32_t steps;        /* Adam steps taken */
  uint32_t since;        /* epochs since the best */
  uint32_t stopped;      /* 1: the stopping rule fired, 2: max_epochs reached */
  uint32_t H, W;
  double best_mse;       /* best validation MSE */
  double last_mse;       /* validation MSE of the last epoch */
  double last_loss;      /* training loss of the last step */
  double device_ms;      /* GPU time from admission (input upload) to the result copied out */
  double compute_ms;     /* GPU time from the input being resident to the result being ready */
  double latency_ms;     /* host time from n2f_submit to DONE */
  double t_start_ms;     /* device timestamps of admission and completion, relative to the */
  double t_done_ms;      /* context's creation (CUDA events), for makespan measurements    */
} n2f_status;

typedef struct n2f_ctx n2f_ctx;
typedef uint64_t n2f_job;

void n2f_config_default(n2f_config* cfg);
void n2f_params_default(n2f_params* p);
const char* n2f_strerror(int code);

/* ---- job API (the serving boundary) ----------------------------------------------------- */
/* Creates a context on cfg->device with a scheduler thread. cfg may be NULL (defaults). */
int n2f_create(n2f_ctx** out, const n2f_config* cfg);
/* Stops the scheduler, cancels unfinished jobs and frees everything. */
void n2f_destroy(n2f_ctx* ctx);
/* Queues one H x W image (host memory, copied before return) for the whole method (Methods,
 * "Noise2Fast Implementation Details"); with p->channels = C_0 > 1, C_0 planes of H x W. p may
 * be NULL (defaults).
 * Errors: EINVAL (NULL, H or W < 2, H*W >= 2^31, non-finite pixel, bad params), ETOOBIG. */
int n2f_submit(n2f_ctx* ctx, const float* image, int H, int W, const n2f_params* p, n2f_job* out);
/* Same, for an image already in device memory (this context's device). The library copies it
 * on the job's own stream when the job is admitted, which can be any time after the call, with
 * no ordering against the caller's streams: the work that wrote the image must be finished
 * before the call (its stream synchronised), and the image must stay valid and unchanged until
 * the job is DONE, FAILED or CANCELED. Pixels are not checked for finiteness here. */
int n2f_submit_device(n2f_ctx* ctx, const float* dimage, int H, int W, const n2f_params* p,
                      n2f_job* out);
/* Same, for a 16-bit microscope image, normalised on the device as value / 65535 (one plane:
 * EINVAL when p->channels > 1). */
int n2f_submit_u16(n2f_ctx* ctx, const uint16_t* image, int H, int W, const n2f_params* p,
                   n2f_job* out);
/* Device bytes a job of this size and parameters holds while it is admitted: the amount the
 * scheduler counts against n2f_config.hbm_budget_bytes (weights, Adam moments, the training
 * activations of the larger sub-image, the validation buffers, the output sum and history).
 * Touches no device. EINVAL for a NULL bytes pointer, bad params or image size; ENOTSUP for a
 * combination this build does not provide. */
int n2f_job_bytes(int H, int W, const n2f_params* p, uint64_t* bytes);
/* Status snapshot; never blocks. */
int n2f_poll(n2f_ctx* ctx, n2f_job job, n2f_status* st);
/* Blocks until the job is DONE/FAILED/CANCELED or timeout_ms passes (< 0: no limit). */
int n2f_wait(n2f_ctx* ctx, n2f_job job, int timeout_ms);
/* Copies the H*W denoised floats (the averaged output of the stopping rule, Methods) to host
 * memory and releases the job.
 * EAGAIN while queued or running. A FAILED or CANCELED job is released too and its error
 * code (ENONFINITE, EDEVICE, ECANCELED, ...) is returned instead of an image. */
int n2f_result(n2f_ctx* ctx, n2f_job job, float* out, size_t out_elems);
/* Same, into device memory (the copy is complete when the call returns). */
int n2f_result_device(n2f_ctx* ctx, n2f_job job, float* dout, size_t out_elems);
/* Cancels a queued or running job; its resources are freed by the scheduler. */
int n2f_cancel(n2f_ctx* ctx, n2f_job job);
/* The job's validation history (Methods, validation paragraph: one full-image MSE per epoch,
 * the scores the stopping rule decides on), kept on the device while the job runs and copied
 * out with its result: the scores of epochs first..epoch, oldest first, at most N2F_HIST_CAP
 * (the latest ones). *n_out receives the count and *first_epoch (may be NULL) the 1-based
 * epoch of out[0]; out may be NULL to query the count. Available once the job is DONE and
 * until its result is collected; EAGAIN while it is queued or running, ENOENT for an unknown
 * or collected job, EINVAL if cap is below the count or the job did not finish (FAILED,
 * CANCELED). A fixed-step job takes no scores under the rule: count 0. */
int n2f_history(n2f_ctx* ctx, n2f_job job, double* out, size_t cap, size_t* n_out,
                uint32_t* first_epoch);

typedef struct {
  uint32_t struct_size;
  uint64_t kernel_launches; /* kernels this context has launched */
  uint64_t bytes_resident;  /* device bytes held by admitted jobs */
  uint32_t jobs_queued, jobs_running, jobs_done;
  /* the profiled kernel class (n2f_config.profile_kernel), over finished jobs: */
  uint64_t prof_launches;   /* launches timed */
  double prof_ms;           /* summed event-timed duration */
  double prof_flops;        /* algorithmic floating-point operations of those launches */
  double prof_bytes;        /* algorithmic DRAM bytes of those launches */
} n2f_ctx_stats;
int n2f_stats(n2f_ctx* ctx, n2f_ctx_stats* st);

/* ---- trainer API: one job's device state, stepped by the caller (parity tests) ----------
 * A trainer runs on the caller's stream; calls enqueue work and return. Exports synchronise
 * the stream and return values converted to float64 in the layouts of the CPU oracle:
 * NCHW maps, weights [C_out][C_in][3][3], the flat parameter order of n2f_param_count.
 * Errors: n2f_trainer_create returns EINVAL for a NULL out or image, bad params, H or W < 2,
 * H*W >= 2^31 or a non-finite pixel, all checked before any device work, and ENOMEM / EDEVICE when the device
 * state cannot be made; every call returns EINVAL for a NULL trainer and EDEVICE for a failed
 * CUDA call. n2f_trainer_run (max_epochs <= 0: no limit) runs epochs in blocks of four and
 * reads the device state after each block: it stops once the rule has fired or at least
 * max_epochs epochs ran (params.max_epochs is the exact cap on the device), and returns
 * ETIMEDOUT if a kernel's bounded wait ran out; n2f_trainer_status then reports FAILED with
 * that error (ENONFINITE for a non-finite validation score). */
typedef struct n2f_trainer n2f_trainer;
int n2f_trainer_create(n2f_trainer** out, const float* image, int H, int W, const n2f_params* p,
                       void* stream);          /* image: host memory, p->channels planes */
void n2f_trainer_destroy(n2f_trainer* tr);
int n2f_trainer_step(n2f_trainer* tr, int pair); /* one Adam step on pair 0..3 (Methods table) */
int n2f_trainer_validate(n2f_trainer* tr); /* full-image forward + MSE + stop rule (Methods,
                                              validation paragraph) */
int n2f_trainer_epoch(n2f_trainer* tr);    /* four steps in table order + validate (Methods) */
int n2f_trainer_run(n2f_trainer* tr, int max_epochs); /* epochs until the rule fires or cap */
int n2f_trainer_finish(n2f_trainer* tr); /* the output image on the device: the mean of the
                                            averaging window (Methods, last sentence of the
                                            validation paragraph), or the fixed-step run's
                                            validation output */
/* Sets the parameters (the flat order of n2f_param_count, rounded to float32) and repacks the
 * kernels' weight copies; EINVAL unless n equals n2f_param_count. Synchronises the stream. */
int n2f_trainer_set_theta(n2f_trainer* tr, const double* theta, size_t n);
enum n2f_export {
  N2F_X_THETA = 0, N2F_X_GRAD = 1, N2F_X_ADAM_M = 2, N2F_X_ADAM_V = 3, /* flat */
  N2F_X_ACT = 4,    /* post-ReLU map of layer 1..8 from the last step, C*h*w */
  N2F_X_DELTA = 5,  /* dL/d(pre-activation) of layer 1..8 from the last step, C*h*w */
  N2F_X_DZ = 7,     /* dL/dz of the last step, h*w */
  N2F_X_PAIR = 8,   /* sub-image 0..3 = up_e, up_o, lf_e, lf_o (all input planes) */
  N2F_X_VAL = 9,    /* last validation output, H*W */
  N2F_X_SUM = 10,   /* running output sum, H*W */
  N2F_X_OUT = 11,   /* output image (after n2f_trainer_finish), H*W */
  N2F_X_HIST = 12,  /* validation scores (FP64 MSE, Methods' validation paragraph) of the last
                       min(epoch, N2F_HIST_CAP) epochs under the stopping rule, oldest first */
  N2F_X_VBEST = 13  /* validation output of the best epoch, H*W */
};
/* Epochs of validation scores each job keeps on the device (a ring; older epochs are
 * overwritten). */
#define N2F_HIST_CAP 4096
/* Returns the number of values through *n_out; out may be NULL to query the size. EINVAL for an
 * unknown `what`, a layer index outside 1..8 or a pair outside 0..3, or cap below the size. */
int n2f_trainer_export(n2f_trainer* tr, int what, int index, double* out, size_t cap,
                       size_t* n_out);
int n2f_trainer_status(n2f_trainer* tr, n2f_status* st);
/* Loads one part of the job's state from host doubles (rounded to float32), the inverse of
 * n2f_trainer_export for: N2F_X_THETA (then the kernels' weight copies are repacked, as by
 * n2f_trainer_set_theta), N2F_X_ADAM_M, N2F_X_ADAM_V (flat, n2f_param_count values),
 * N2F_X_SUM and N2F_X_VBEST (H*W). With n2f_trainer_set_progress it puts a trainer in any
 * state the method passes through (Methods: Adam moments, the stopping rule's best score and
 * count, the running output sum), so that an epoch can be compared with another
 * implementation's epoch from the same state. index is unused (0). EINVAL for another `what`
 * or n not equal to the size. Synchronises the stream. */
int n2f_trainer_import(n2f_trainer* tr, int what, int index, const double* in, size_t n);
/* Sets the step and stopping-rule counters: t Adam steps taken (bias corrections 1 - beta^t),
 * `epoch` epochs validated, `since` epochs since the best, `best` the best validation score
 * (+inf: none yet); the job is marked running. Validation scores recorded before keep their
 * places in the N2F_X_HIST ring. EINVAL in fixed-step mode or for since > epoch.
 * Synchronises the stream. */
int n2f_trainer_set_progress(n2f_trainer* tr, uint32_t t, uint32_t epoch, uint32_t since,
                             double best);
uint64_t n2f_trainer_launches(const n2f_trainer* tr);

/* Number of parameters of the network (n2f_widths). */
size_t n2f_param_count(int widths);

/* ---- op-level entry points (device pointers, caller's stream; parity of single kernels) --
 * "CG layout": channel-grouped maps, act[g][y][x][k] with g = c / G, k = c % G and
 * G = 4 (float32) or 8 (bfloat16), i.e. one 16-byte group per pixel and group. */

/* Checkerboard gather (Eq. 6-7 and the Methods' "left" equations; odd images read as the
 * order-preserving compaction of the pixels with i+j odd). x: H*W floats; up_e/up_o:
 * H*(W/2); lf_e/lf_o: (H/2)*W. Exact copies. */
int n2f_checker_gather(const float* x, int H, int W, float* up_e, float* up_o, float* lf_e,
                       float* lf_o, void* stream);

/* Maximum projection of a Z-stack (Methods, fluorescence microscopy: the slices of a volume are
 * denoised as independent images and max projected along Z). vol: Z planes of H*W floats,
 * contiguous, device memory; out: H*W floats, device memory, caller-owned; may not overlap vol.
 * out[y*W + x] = max over z of vol[z*H*W + y*W + x], exact. Runs on `stream` (0: default) and
 * returns without waiting. N2F_EINVAL for a NULL pointer or Z, H or W < 1; N2F_EDEVICE if the
 * launch fails. */
int n2f_max_project(const float* vol, int Z, int H, int W, float* out, void* stream);
/* NCHW float32 <-> CG layout of the given precision (C a multiple of G); device pointers, runs on
 * `stream` without waiting. N2F_EINVAL for a NULL pointer, a precision other than N2F_FP32 or
 * N2F_BF16, C not a positive multiple of G, or H or W < 1.
 * The convolution entry points below return N2F_EINVAL in the same cases (C_in and C_out
 * positive multiples of 8, an engine outside enum n2f_engine, a mode other than 0 or 1) and
 * N2F_ENOTSUP when N2F_ENGINE_TC is asked for channel counts it is not built for. */
int n2f_pack_cg(const float* nchw, int C, int H, int W, int precision, void* cg, void* stream);
int n2f_unpack_cg(const void* cg, int C, int H, int W, int precision, float* nchw, void* stream);
/* One 3x3 convolution layer with zero "same" padding (Methods; Fig. 2a):
 *   forward (mode 0):  out = ReLU(conv(in, w) + b)
 *   dgrad   (mode 1):  out = conv^T(in, w) * [mask > 0]   (in = dL/d pre-activation of this
 *                      layer, mask = the layer's input activation, out has C_in channels)
 * in/out/mask in CG layout of `precision`; w: float32 [C_out][C_in][3][3] (device), b: C_out.
 * C_in, C_out in {32, 64, 128, 256} for the tensor-core engine; multiples of G for SIMT.
 * Tensor-core engine, N2F_FP32: the call first finds the largest |w| and |in| (the power-of-two
 * scales of their two fp16 parts); accuracy about 2^-22 per product at any float32 magnitude.
 * Allocates a small workspace (cudaMallocAsync), synchronises the stream; N2F_ETIMEDOUT if a
 * kernel wait ran out. */
int n2f_conv3x3(int mode, int engine, int precision, const void* in, int cin, int cout, int H,
                int W, const float* w, const float* b, const void* mask, void* out,
                void* stream);
/* Weight/bias gradient of one 3x3 layer: dw[C_out][C_in][3][3] and db[C_out] (float32,
 * overwritten) from dout (CG, C_out channels) and in (CG, C_in channels). Tensor-core engine,
 * N2F_FP32: scales from the largest |dout| and |in|, as for n2f_conv3x3. Allocates its
 * partial-sum workspace (cudaMallocAsync), synchronises the stream; N2F_ETIMEDOUT if a kernel
 * wait ran out. */
int n2f_conv3x3_wgrad(int engine, int precision, const void* dout, const void* in, int cin,
                      int cout, int H, int W, float* dw, float* db, void* stream);

/* Allocation-free variant of n2f_conv3x3_wgrad (same arguments, same results up to the
 * summation order of the pixel splits). The paper has no counterpart: this exists for callers
 * that cannot allocate device memory when they need a weight gradient -- a process whose device
 * memory is wholly reserved by another allocator (a framework's caching pool or a fixed arena),
 * where a cudaMalloc would fail or fragment it, or a latency-bound loop that must not block on
 * the CUDA allocator. The partial-sum workspace is a fixed 16 MiB device array compiled into the
 * library: every GPU the library is loaded on holds it until the process exits, and nothing is
 * allocated or freed per call (no cudaMalloc / cudaFree / cudaMallocAsync).
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *    that device current; make that first call before any stream capture on that device.
 *  - All calls share the one array and it keeps the last call's contents: calls that can overlap
 *    on the GPU (different streams, or several host threads) race and must be serialised.
 *  - The address is looked up once per device and kept: after cudaDeviceReset on a device the
 *    cached address is stale, so a process that resets a device must not call this entry point
 *    on that device again.
 *  - A layer needs 9*C_in*C_out + C_out + 64 floats (one split of the pixel sum) of the
 *    4 Mi-float array, less 64 floats the library keeps for its error and magnitude words;
 *    larger layers return N2F_ETOOBIG. Layers that leave room use several splits.
 *    Synchronises the stream; N2F_ETIMEDOUT if a kernel wait ran out. */
int n2f_conv3x3_wgrad_noalloc(int engine, int precision, const void* dout, const void* in, int cin,
                              int cout, int H, int W, float* dw, float* db, void* stream);

/* ---- checked build ----------------------------------------------------------------------
 * libn2f_checked.so (paper_2108_10209_gb300/build.py --checked: the same sources compiled with
 * N2F_CHECKED) tests the global-memory indexes its kernels compute against the extent of the
 * tensor each one addresses, known from the launch shapes and the workspace sizes: an index out
 * of range is counted and that access skipped, so nothing traps and the context stays usable.
 * n2f_check_status reports the count since the last clear on the current device and the first
 * failing site as file * 100000 + line (file 1 kernels_basic.cu, 2 kernels_simt.cu,
 * 3 conv_tc.cu, 4 wgrad_tc.cu; 0: none); clear != 0 zeroes the counts afterwards. Synchronises
 * the device. N2F_ENOTSUP in the normal build (libn2f.so), whose kernels carry no checks;
 * N2F_EINVAL for a NULL pointer; N2F_EDEVICE if the counts cannot be read. */
int n2f_check_status(uint64_t* failures, int* first_site, int clear);

/* ---- diagnostics ------------------------------------------------------------------------
 * One 128 x N tile of D = A * B^T (K-step by K-step) through the tcgen05 tensor cores, with the
 * operands given as ready shared-memory images (no swizzle) and the descriptor strides the
 * convolution kernels rely on: lbo = byte distance of core matrices adjacent along K, sbo =
 * along M (A) or N (B); kstep = byte advance of the start address per MMA (K = 16 bf16 or
 * 8 tf32 elements). tf32 = 0: bf16 operands; a_mn / b_mn = 1: MN-major images.
 * A, B: device; D: device float32 [128][N] row-major. N in 16..256 step 16, images <= 100 KB
 * each. Synchronises the stream; ETIMEDOUT if the MMA completion never arrived. */
int n2f_umma_gemm(int tf32, int N, int K, int a_mn, int b_mn, const void* A, size_t a_bytes,
                  uint32_t a_lbo, uint32_t a_sbo, uint32_t a_kstep, const void* B, size_t b_bytes,
                  uint32_t b_lbo, uint32_t b_sbo, uint32_t b_kstep, float* D, void* stream);

/* Failure-detection check: one kernel waits on a barrier that nothing ever completes, with the
 * bounded wait every tensor-core kernel uses (here limit_ms, 1..10000). The wait gives up after
 * the limit, the kernel records the time-out and returns, and the context stays usable: the
 * call returns N2F_ETIMEDOUT (the expected result) after about limit_ms, N2F_OK never.
 * N2F_EINVAL for a limit out of range. Synchronises the stream. */
int n2f_wait_probe(uint32_t limit_ms, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* N2F_H */
