/*
 * FP64 CPU oracle for Noise2Fast (Lequyer et al., arXiv 2108.10209).
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously correct restatement of the
 * paper's per-image procedure that the CUDA library is checked against. Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the library never does,
 * and the two share no source, header, table or helper.
 *
 * Conventions
 *   - Every value is double precision. Images and activation maps are planes in NCHW order
 *     (channel, row, column), row-major, batch size one.
 *   - 3x3 weights are [C_out][C_in][ky][kx] with ky, kx = 0..2 meaning offsets -1..+1;
 *     "same" zero padding (an f: R^{m x n} -> R^{m x n} map, Eq. 2).
 *   - OpenMP splits only the outermost loop over independent output elements, and every
 *     output element is accumulated by one thread in the fixed order written in the loop
 *     nest, so the results do not depend on the number of threads.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py against a
 * closed form, an invariant, a library special case (float64 torch) or finite differences.
 * The paper's own end-to-end quality numbers (Table 1, BSD68) cannot be reproduced without
 * its datasets, so end-to-end denoising quality is "parity unpinned" against the paper;
 * it is pinned only relatively (GPU vs oracle, and the trained net beating the noisy input).
 */
#ifndef N2F_ORACLE_H
#define N2F_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_LAYERS 8 /* eight 3x3 conv + ReLU layers, then a 1x1 conv + sigmoid head */

/* ---- Weight initialisation (the paper leaves it unstated) --------------------------------
 * SplitMix64 (Steele, Lea & Flood 2014): output k (k = 0, 1, ...) of the generator seeded with
 * `seed` is mix(seed + (k+1) * 0x9E3779B97F4A7C15). */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t k);

/* Number of parameters of the network with the given eight layer widths and C_0 input channels
 * (Fig. 2a caption: inputs can be multi-channel; the output is always one channel).
 * Flat order: for l = 1..8: W_l[C_l][C_{l-1}][3][3], b_l[C_l]; then head w[C_8], b.
 * orc_param_count is the one-channel case. */
size_t orc_param_count_c(const int widths[ORC_LAYERS], int c0);
size_t orc_param_count(const int widths[ORC_LAYERS]);

/* theta[i] = float( (2u_i - 1) / sqrt(fan_in) ), u_i = (splitmix64_at(seed, i) >> 11) * 2^-53,
 * fan_in = 9 C_in for the 3x3 layers and C_8 for the head (weights and biases alike). */
void orc_init_params_c(const int widths[ORC_LAYERS], int c0, uint64_t seed, double* theta);
void orc_init_params(const int widths[ORC_LAYERS], uint64_t seed, double* theta);

/* ---- Checkerboard downsampling (Theoretical Background Eq. 6-7; Methods, "up" and "left") --
 * Reading of the odd formulas: the pixel set with i+j odd, compacted in order, i.e.
 *   up_e(i,j) = x(i, 2j + (i mod 2)),      up_o(i,j) = x(i, 2j + 1 - (i mod 2)),  H x floor(W/2)
 *   lf_e(i,j) = x(2i + (j mod 2), j),      lf_o(i,j) = x(2i + 1 - (j mod 2), j),  floor(H/2) x W  */
void orc_checker(const double* x, int H, int W, double* up_e, double* up_o, double* lf_e,
                 double* lf_o);

/* Ablation Study, "Quad": 2x2 blocks -> the images of their top-left, top-right, bottom-left
 * and bottom-right pixels, floor(H/2) x floor(W/2) each:
 *   tl(i,j) = x(2i, 2j), tr(i,j) = x(2i, 2j+1), bl(i,j) = x(2i+1, 2j), br(i,j) = x(2i+1, 2j+1) */
void orc_quad(const double* x, int H, int W, double* tl, double* tr, double* bl, double* br);

/* ---- Network pieces (Methods, first paragraph; Fig. 2a) ---------------------------------- */
/* out[o] = b[o] + sum_c sum_ky sum_kx w[o][c][ky][kx] * in[c](y+ky-1, x+kx-1), then ReLU if relu. */
void orc_conv3x3_fwd(const double* in, int cin, int h, int w, const double* wt, const double* b,
                     int cout, int relu, double* out);
/* din[c](y,x) = sum_o sum_ky sum_kx w[o][c][ky][kx] * dout[o](y-ky+1, x-kx+1)  (no ReLU mask). */
void orc_conv3x3_dgrad(const double* dout, int cout, int h, int w, const double* wt, int cin,
                       double* din);
/* dw[o][c][ky][kx] = sum_{y,x} dout[o](y,x) * in[c](y+ky-1, x+kx-1);  db[o] = sum dout[o].
 * Sums run over pixels in raster order. */
void orc_conv3x3_wgrad(const double* dout, int cout, int h, int w, const double* in, int cin,
                       double* dw, double* db);
/* z(p) = b + sum_c w[c] a[c](p)  (the final 1x1 convolution, before the sigmoid). */
void orc_head_fwd(const double* a, int c, int npx, const double* w, double b, double* z);
double orc_sigmoid(double z);

/* Training loss (Methods: binary cross-entropy between the network output and the target).
 * BCE(s, y), s = sigmoid(z), with each log term clamped at -100 (bounded for the unclipped
 * targets y outside [0, 1]); logs evaluated in logit space. dL/dz = (s - y)/P away from the
 * clamps. loss_kind 1 is the MSE alternative the paper mentions: L = (1/P) sum (s - y)^2. */
double orc_loss(const double* z, const double* y, int npx, int loss_kind, double* dz);

/* Adam (Kingma & Ba, Algorithm 1), step t >= 1, no weight decay. */
void orc_adam(double* theta, const double* g, double* m, double* v, size_t n, long t, double lr,
              double beta1, double beta2, double eps);

/* ---- Stopping rule (Methods: 100 epochs without improvement, average the last 100) ------- */
typedef struct {
  double best;   /* best validation score so far (+inf before the first epoch) */
  int since;     /* epochs since the best */
  int epoch;     /* epochs completed */
  int stopped;   /* 1 once the rule fired */
} orc_stop_state;
void orc_stop_init(orc_stop_state* s);
/* Threads the oracle's parallel loops use (1 without OpenMP). */
int orc_threads(void);
/* Feed one validation score. Returns 1 when it is a new best (the running output sum restarts),
 * 0 otherwise (the output of this epoch joins the sum). Sets ->stopped when `since` reaches
 * `patience` (or patience-1 when incl_best, the reading whose window contains the best epoch). */
int orc_stop_update(orc_stop_state* s, double score, int patience, int incl_best);

/* ---- Whole procedure ---------------------------------------------------------------------- */
typedef struct {
  int widths[ORC_LAYERS];
  double lr, beta1, beta2, eps; /* 1e-3, 0.9, 0.999, 1e-8 */
  int patience;                 /* 100 */
  int max_epochs;               /* 0 = no cap */
  int fixed_steps;              /* < 0: stopping rule; >= 0: that many steps, then one validation */
  int loss_kind;                /* 0 = BCE, 1 = MSE */
  int incl_best;                /* 0 = window is the 100 epochs after the best */
  uint64_t seed;
  int channels;                 /* input channels C_0 (0 or 1: a grayscale image) */
  int target;                   /* the predicted channel, 0 .. C_0 - 1 (Fig. 2a caption: an RGB
                                   image is denoised one output channel per network) */
  int downsample;               /* 0 = checkerboard (the method); 1 = the Ablation Study's Quad */
  int exact;                    /* 1 = the Ablation Study's Exact: the job's image carries the
                                   clean target plane after the C_0 input planes, and each
                                   target becomes x_tgt - (s_tgt - s_in) */
} orc_params;

typedef struct orc_job orc_job;

/* A job owns the image (C_0 planes of H x W, plus the clean plane for Exact), the four training
 * pairs, theta, Adam moments and the stop state. Each pair's input is all C_0 channels of one
 * sub-image, its target the predicted channel of the paired sub-image; validation compares
 * with that channel of x. Pairs: checkerboard up_e->up_o, up_o->up_e, lf_e->lf_o, lf_o->lf_e
 * (Methods table); Quad TL->TR, TR->BR, BR->BL, BL->TL (the reading taken: once round the
 * 2x2 block through adjacent pixels). */
orc_job* orc_job_new(const double* x, int H, int W, const orc_params* p);
/* Replace theta (n = orc_param_count values). */
void orc_job_set_theta(orc_job* j, const double* theta);
/* One Adam step on pair k (0..3, in the pair order above).
 * Returns the training loss before the update. Keeps activations, deltas and grads for inspection. */
double orc_job_step(orc_job* j, int pair);
/* Full-image validation forward; writes V (H*W) if v != NULL; returns mean((V - x)^2). */
double orc_job_validate(orc_job* j, double* v);
/* One epoch = four steps + validation + stop-rule bookkeeping. Returns the validation score. */
double orc_job_epoch(orc_job* j);
/* Run to completion (stop rule or fixed steps); out gets H*W values. */
void orc_job_run(orc_job* j, double* out);

enum {
  ORC_THETA = 0, ORC_GRAD = 1, ORC_ADAM_M = 2, ORC_ADAM_V = 3, /* flat, orc_param_count values */
  ORC_ACT = 4,   /* layer l = 1..8 post-ReLU activation of the last training step, C_l*h*w */
  ORC_DELTA = 5, /* layer l = 1..8 gradient of the loss w.r.t. the pre-activation, C_l*h*w */
  ORC_Z = 6,     /* head logits of the last training step, h*w */
  ORC_DZ = 7,    /* dL/dz of the last training step, h*w */
  ORC_PAIR_IN = 8, ORC_PAIR_TGT = 9, /* input / target sub-image of pair `layer` */
  ORC_SUM = 10,  /* running output sum S, H*W */
  ORC_VBEST = 11 /* validation output of the best epoch, H*W */
};
/* Copies the requested array into out; returns the number of values (0 if unknown). */
size_t orc_job_get(const orc_job* j, int what, int layer, double* out);
/* Scalars: step count t, epoch, since, stopped, capped, best, last loss, pair dims. */
void orc_job_info(const orc_job* j, long* t, int* epoch, int* since, int* stopped, int* capped,
                  double* best, double* last_loss, int dims[4]);
void orc_job_free(orc_job* j);

/* Forward pass of the whole network on an arbitrary h x w image of C_0 channels (planes):
 * writes V = sigmoid(z) (h*w) and z if non-NULL. orc_net_forward is the one-channel case. */
void orc_net_forward_c(const int widths[ORC_LAYERS], int c0, const double* theta,
                       const double* img, int h, int w, double* v, double* z);
void orc_net_forward(const int widths[ORC_LAYERS], const double* theta, const double* img, int h,
                     int w, double* v, double* z);

/* ---- Volumes (Methods, fluorescence microscopy: a Z-stack is denoised slice by slice, each
 * slice an independent image, and the denoised slices are max projected along Z) ----------
 * out[y][x] = max over z of vol[z][y][x]; vol is Z planes of H x W. */
void orc_max_project(const double* vol, int Z, int H, int W, double* out);

#ifdef __cplusplus
}
#endif
#endif
