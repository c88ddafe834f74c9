/*
 * FP64 CPU oracle for Noise2Fast (arXiv 2108.10209) -- TEST INFRASTRUCTURE ONLY.
 *
 * Written from the paper's Methods section ("Noise2Fast Implementation Details") and the
 * Theoretical Background (Eq. 6-7). Each function states the passage it follows; the readings
 * taken where the paper is silent or garbled are listed in oracle.h and in the design notes.
 * No blocking, fusion or reordering beyond the definitions: every output element is a plain
 * sum accumulated in the order the loop nest shows.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
int omp_get_max_threads(void); /* OpenMP runtime library routine */
#endif

/* Threads the parallel loops use (OpenMP over independent outputs only), for reporting. */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), counter form.                                */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Methods, first paragraph: two 32-channel 3x3 conv+ReLU, repeated three more times with the
 * width doubled each time, then 1x1 conv + sigmoid. Widths are a parameter (see oracle.h); the
 * first layer sees c0 input channels (Fig. 2a caption: inputs may be multi-channel). */
size_t orc_param_count_c(const int widths[ORC_LAYERS], int c0) {
  size_t n = 0;
  int cin = c0;
  for (int l = 0; l < ORC_LAYERS; ++l) {
    n += (size_t)widths[l] * cin * 9 + widths[l];
    cin = widths[l];
  }
  return n + (size_t)cin + 1;
}

size_t orc_param_count(const int widths[ORC_LAYERS]) { return orc_param_count_c(widths, 1); }

/* Offsets of W_l and b_l (l = 0..7) and of the head (index 8) in the flat vector. */
static void param_offsets(const int widths[ORC_LAYERS], int c0, size_t ow[ORC_LAYERS + 1],
                          size_t ob[ORC_LAYERS + 1]) {
  size_t n = 0;
  int cin = c0;
  for (int l = 0; l < ORC_LAYERS; ++l) {
    ow[l] = n;
    n += (size_t)widths[l] * cin * 9;
    ob[l] = n;
    n += widths[l];
    cin = widths[l];
  }
  ow[ORC_LAYERS] = n;
  ob[ORC_LAYERS] = n + cin;
}

void orc_init_params_c(const int widths[ORC_LAYERS], int c0, uint64_t seed, double* theta) {
  size_t k = 0;
  int cin = c0;
  for (int l = 0; l <= ORC_LAYERS; ++l) {
    const int head = (l == ORC_LAYERS);
    const int cout = head ? 1 : widths[l];
    const int fan_in = head ? cin : cin * 9;
    const size_t nw = head ? (size_t)cin : (size_t)cout * cin * 9;
    const double bound = 1.0 / sqrt((double)fan_in);
    for (size_t i = 0; i < nw + (size_t)cout; ++i, ++k) {
      const double u = (double)(orc_splitmix64_at(seed, k) >> 11) * 0x1.0p-53;
      theta[k] = (double)(float)((2.0 * u - 1.0) * bound);
    }
    if (!head) cin = widths[l];
  }
}

void orc_init_params(const int widths[ORC_LAYERS], uint64_t seed, double* theta) {
  orc_init_params_c(widths, 1, seed, theta);
}

/* ------------------------------------------------------------------------------------------ */
/* Checkerboard downsampling, Eq. 6-7 ("up") and the Methods' primed equations ("left").       */
void orc_checker(const double* x, int H, int W, double* up_e, double* up_o, double* lf_e,
                 double* lf_o) {
  const int hw = W / 2, hh = H / 2;
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < hw; ++j) {
      up_e[i * hw + j] = x[i * W + 2 * j + (i % 2)];
      up_o[i * hw + j] = x[i * W + 2 * j + 1 - (i % 2)];
    }
  for (int i = 0; i < hh; ++i)
    for (int j = 0; j < W; ++j) {
      lf_e[i * W + j] = x[(2 * i + (j % 2)) * W + j];
      lf_o[i * W + j] = x[(2 * i + 1 - (j % 2)) * W + j];
    }
}

/* Ablation Study, "Quad": the image cut into 2x2 blocks and four images made of the blocks'
 * top-left, top-right, bottom-left and bottom-right pixels, floor(H/2) x floor(W/2) each.    */
void orc_quad(const double* x, int H, int W, double* tl, double* tr, double* bl, double* br) {
  const int hh = H / 2, hw = W / 2;
  for (int i = 0; i < hh; ++i)
    for (int j = 0; j < hw; ++j) {
      tl[i * hw + j] = x[(2 * i) * W + 2 * j];
      tr[i * hw + j] = x[(2 * i) * W + 2 * j + 1];
      bl[i * hw + j] = x[(2 * i + 1) * W + 2 * j];
      br[i * hw + j] = x[(2 * i + 1) * W + 2 * j + 1];
    }
}

/* ------------------------------------------------------------------------------------------ */
/* 3x3 convolution with zero "same" padding, forward.                                         */
void orc_conv3x3_fwd(const double* in, int cin, int h, int w, const double* wt, const double* b,
                     int cout, int relu, double* out) {
  const size_t hw = (size_t)h * w;
#pragma omp parallel for schedule(dynamic, 1)
  for (int o = 0; o < cout; ++o) {
    double* op = out + (size_t)o * hw;
    for (size_t i = 0; i < hw; ++i) op[i] = b[o];
    for (int c = 0; c < cin; ++c) {
      const double* ip = in + (size_t)c * hw;
      for (int ky = 0; ky < 3; ++ky)
        for (int kx = 0; kx < 3; ++kx) {
          const double wv = wt[((size_t)o * cin + c) * 9 + ky * 3 + kx];
          const int dy = ky - 1, dx = kx - 1;
          const int x0 = dx < 0 ? 1 : 0, x1 = dx > 0 ? w - 1 : w;
          for (int y = 0; y < h; ++y) {
            const int yy = y + dy;
            if (yy < 0 || yy >= h) continue;
            double* orow = op + (size_t)y * w;
            const double* irow = ip + (size_t)yy * w + dx;
            for (int x = x0; x < x1; ++x) orow[x] += wv * irow[x];
          }
        }
    }
    if (relu)
      for (size_t i = 0; i < hw; ++i) op[i] = op[i] > 0.0 ? op[i] : 0.0;
  }
}

/* Gradient w.r.t. the input: correlation with the 180-degree-rotated, transposed kernel.     */
void orc_conv3x3_dgrad(const double* dout, int cout, int h, int w, const double* wt, int cin,
                       double* din) {
  const size_t hw = (size_t)h * w;
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < cin; ++c) {
    double* dp = din + (size_t)c * hw;
    for (size_t i = 0; i < hw; ++i) dp[i] = 0.0;
    for (int o = 0; o < cout; ++o) {
      const double* gp = dout + (size_t)o * hw;
      for (int ky = 0; ky < 3; ++ky)
        for (int kx = 0; kx < 3; ++kx) {
          const double wv = wt[((size_t)o * cin + c) * 9 + ky * 3 + kx];
          const int dy = ky - 1, dx = kx - 1;
          /* din(y,x) += w * dout(y-dy, x-dx) */
          const int x0 = dx > 0 ? 1 : 0, x1 = dx < 0 ? w - 1 : w;
          for (int y = 0; y < h; ++y) {
            const int yy = y - dy;
            if (yy < 0 || yy >= h) continue;
            double* drow = dp + (size_t)y * w;
            const double* grow = gp + (size_t)yy * w - dx;
            for (int x = x0; x < x1; ++x) drow[x] += wv * grow[x];
          }
        }
    }
  }
}

/* Gradient w.r.t. the weights and biases; each sum runs over pixels in raster order.       */
void orc_conv3x3_wgrad(const double* dout, int cout, int h, int w, const double* in, int cin,
                       double* dw, double* db) {
  const size_t hw = (size_t)h * w;
#pragma omp parallel for schedule(dynamic, 1)
  for (int oc = 0; oc < cout * cin; ++oc) {
    const int o = oc / cin, c = oc % cin;
    const double* gp = dout + (size_t)o * hw;
    const double* ip = in + (size_t)c * hw;
    for (int ky = 0; ky < 3; ++ky)
      for (int kx = 0; kx < 3; ++kx) {
        const int dy = ky - 1, dx = kx - 1;
        double s = 0.0;
        for (int y = 0; y < h; ++y) {
          const int yy = y + dy;
          if (yy < 0 || yy >= h) continue;
          for (int x = 0; x < w; ++x) {
            const int xx = x + dx;
            if (xx < 0 || xx >= w) continue;
            s += gp[(size_t)y * w + x] * ip[(size_t)yy * w + xx];
          }
        }
        dw[((size_t)o * cin + c) * 9 + ky * 3 + kx] = s;
      }
  }
  for (int o = 0; o < cout; ++o) {
    double s = 0.0;
    for (size_t i = 0; i < hw; ++i) s += dout[(size_t)o * hw + i];
    db[o] = s;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Head: 1x1 convolution to one channel (sigmoid applied by the callers).                     */
void orc_head_fwd(const double* a, int c, int npx, const double* w, double b, double* z) {
#pragma omp parallel for schedule(static)
  for (int p = 0; p < npx; ++p) {
    double s = b;
    for (int k = 0; k < c; ++k) s += w[k] * a[(size_t)k * npx + p];
    z[p] = s;
  }
}

double orc_sigmoid(double z) {
  if (z >= 0.0) return 1.0 / (1.0 + exp(-z));
  const double e = exp(z);
  return e / (1.0 + e);
}

static double softplus(double z) { return (z > 0.0 ? z : 0.0) + log1p(exp(-fabs(z))); }

/* Methods: BCE loss between the target and the network output (batch size 1, mean over pixels).
 * The noisy targets are not clipped (Compared Methods, Self2Self paragraph), so y may leave
 * [0, 1], where -[y log s + (1-y) log(1-s)] is unbounded below as s -> 0 or 1. The loss is the
 * usual library definition of BCE, with each log term clamped at -100, and the logs are taken
 * in logit space (log s = -softplus(-z), log(1-s) = -softplus(z)):
 *   L = (1/P) sum -y max(log s, -100) - (1-y) max(log(1-s), -100)
 *   dL/dz = (s - y)/P where neither clamp is active; otherwise the unclamped terms' derivatives,
 *   -y (1-s) [log s > -100] + (1-y) s [log(1-s) > -100], over P.
 * loss_kind 1 is the MSE alternative the paper mentions: L = (1/P) sum (s-y)^2. */
double orc_loss(const double* z, const double* y, int npx, int loss_kind, double* dz) {
  double L = 0.0;
  for (int p = 0; p < npx; ++p) {
    const double s = orc_sigmoid(z[p]);
    if (loss_kind == 0) {
      const double lp = -softplus(-z[p]), lq = -softplus(z[p]);
      const int m1 = lp > -100.0, m2 = lq > -100.0;
      L += -y[p] * (m1 ? lp : -100.0) - (1.0 - y[p]) * (m2 ? lq : -100.0);
      if (dz) {
        double g;
        if (m1 && m2)
          g = s - y[p];
        else
          g = (m1 ? -y[p] * (1.0 - s) : 0.0) + (m2 ? (1.0 - y[p]) * s : 0.0);
        dz[p] = g / npx;
      }
    } else {
      L += (s - y[p]) * (s - y[p]);
      if (dz) dz[p] = 2.0 * (s - y[p]) * s * (1.0 - s) / npx;
    }
  }
  return L / npx;
}

/* Kingma & Ba, Algorithm 1 (bias-corrected moments), as cited by the Methods for Adam.        */
void orc_adam(double* theta, const double* g, double* m, double* v, size_t n, long t, double lr,
              double beta1, double beta2, double eps) {
  const double bc1 = 1.0 - pow(beta1, (double)t), bc2 = 1.0 - pow(beta2, (double)t);
  for (size_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    const double mh = m[i] / bc1, vh = v[i] / bc2;
    theta[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Methods, validation paragraph: stop once one hundred epochs pass without improving the best
 * validation score; the output is the average of the last one hundred validation outputs,
 * which are exactly the outputs of the epochs after the best one.                             */
void orc_stop_init(orc_stop_state* s) {
  s->best = INFINITY;
  s->since = 0;
  s->epoch = 0;
  s->stopped = 0;
}

int orc_stop_update(orc_stop_state* s, double score, int patience, int incl_best) {
  int improved = 0;
  s->epoch += 1;
  if (score < s->best) {
    s->best = score;
    s->since = 0;
    improved = 1;
  } else {
    s->since += 1;
  }
  if (s->since >= (incl_best ? patience - 1 : patience)) s->stopped = 1;
  return improved;
}

/* ------------------------------------------------------------------------------------------ */
struct orc_job {
  orc_params p;
  int H, W;
  int c0, tc; /* input channels, target channel */
  double* x;  /* c0 planes of H*W */
  int ph[4], pw[4];
  double* pin[4]; /* pair inputs */
  double* ptg[4]; /* pair targets (channel tc of the paired sub-image, table order) */
  double* ptx[4]; /* Exact ablation: the adjusted targets (owned) */
  double* sub[4]; /* up_e, up_o, lf_e, lf_o; c0 planes each */
  size_t np;
  double *theta, *grad, *m, *v;
  long t;
  size_t ow[ORC_LAYERS + 1], ob[ORC_LAYERS + 1];
  int cin[ORC_LAYERS];
  /* last training step */
  int lh, lw;
  double* act[ORC_LAYERS];
  double* delta[ORC_LAYERS];
  double *z, *dz;
  double last_loss;
  /* stop rule and output averaging */
  orc_stop_state st;
  int capped;
  double *S, *Vbest, *V;
};

static double* dalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

orc_job* orc_job_new(const double* x, int H, int W, const orc_params* p) {
  orc_job* j = (orc_job*)calloc(1, sizeof(orc_job));
  j->p = *p;
  j->H = H;
  j->W = W;
  j->c0 = p->channels > 0 ? p->channels : 1;
  j->tc = p->target;
  const size_t N = (size_t)H * W;
  /* x holds the C_0 input planes and, for the Exact ablation, the clean target plane after them */
  const int nplanes = j->c0 + (p->exact ? 1 : 0);
  j->x = dalloc((size_t)nplanes * N);
  memcpy(j->x, x, sizeof(double) * nplanes * N);
  const int quad = p->downsample == 1;
  for (int k = 0; k < 4; ++k) {
    j->ph[k] = quad ? H / 2 : (k < 2 ? H : H / 2);
    j->pw[k] = quad ? W / 2 : (k < 2 ? W / 2 : W);
  }
  size_t P[4];
  for (int k = 0; k < 4; ++k) {
    P[k] = (size_t)j->ph[k] * j->pw[k];
    j->sub[k] = dalloc((size_t)nplanes * P[k]);
  }
  /* every plane is downsampled the same way. Checkerboard: sub = up_e, up_o, lf_e, lf_o and the
   * Methods table's pairs k -> k^1. Quad (the reading taken: the pairs go once round the 2x2
   * block through horizontally and vertically adjacent pixels): sub = TL, TR, BR, BL and the
   * pairs k -> k+1 mod 4, i.e. TL->TR, TR->BR, BR->BL, BL->TL. */
  int tgt_of[4];
  for (int c = 0; c < nplanes; ++c) {
    const double* xc = j->x + c * N;
    if (quad)
      orc_quad(xc, H, W, j->sub[0] + c * P[0], j->sub[1] + c * P[1], j->sub[3] + c * P[3],
               j->sub[2] + c * P[2]);
    else
      orc_checker(xc, H, W, j->sub[0] + c * P[0], j->sub[1] + c * P[1], j->sub[2] + c * P[2],
                  j->sub[3] + c * P[3]);
  }
  for (int k = 0; k < 4; ++k) tgt_of[k] = quad ? (k + 1) % 4 : k ^ 1;
  /* the target is the predicted channel of the paired sub-image (Fig. 2a caption: one output
   * channel per network). Exact ablation: the signal difference s_tgt - s_in (the s_odd - s_even
   * term of the Theoretical Background) is subtracted using the clean plane,
   * target = x_tgt - (s_tgt - s_in). */
  for (int k = 0; k < 4; ++k) {
    const int g = tgt_of[k];
    j->pin[k] = j->sub[k];
    j->ptg[k] = j->sub[g] + (size_t)j->tc * P[g];
    if (p->exact) {
      j->ptx[k] = dalloc(P[k]);
      const double* sg = j->sub[g] + (size_t)j->c0 * P[g];
      const double* sk = j->sub[k] + (size_t)j->c0 * P[k];
      for (size_t i = 0; i < P[k]; ++i) j->ptx[k][i] = j->ptg[k][i] - (sg[i] - sk[i]);
      j->ptg[k] = j->ptx[k];
    }
  }
  j->np = orc_param_count_c(p->widths, j->c0);
  j->theta = dalloc(j->np);
  j->grad = dalloc(j->np);
  j->m = dalloc(j->np);
  j->v = dalloc(j->np);
  orc_init_params_c(p->widths, j->c0, p->seed, j->theta);
  param_offsets(p->widths, j->c0, j->ow, j->ob);
  int cin = j->c0;
  size_t maxpx = 0;
  for (int k = 0; k < 4; ++k)
    if ((size_t)j->ph[k] * j->pw[k] > maxpx) maxpx = (size_t)j->ph[k] * j->pw[k];
  for (int l = 0; l < ORC_LAYERS; ++l) {
    j->cin[l] = cin;
    j->act[l] = dalloc((size_t)p->widths[l] * maxpx);
    j->delta[l] = dalloc((size_t)p->widths[l] * maxpx);
    cin = p->widths[l];
  }
  j->z = dalloc(maxpx);
  j->dz = dalloc(maxpx);
  j->S = dalloc((size_t)H * W);
  j->Vbest = dalloc((size_t)H * W);
  j->V = dalloc((size_t)H * W);
  orc_stop_init(&j->st);
  return j;
}

void orc_job_set_theta(orc_job* j, const double* theta) {
  memcpy(j->theta, theta, sizeof(double) * j->np);
}

/* Forward through the eight conv layers, keeping every post-ReLU map in act[]. */
static void forward_layers(const int widths[ORC_LAYERS], int c0, const double* theta,
                           const size_t* ow, const size_t* ob, const double* img, int h, int w,
                           double** act) {
  const double* in = img;
  int cin = c0;
  for (int l = 0; l < ORC_LAYERS; ++l) {
    orc_conv3x3_fwd(in, cin, h, w, theta + ow[l], theta + ob[l], widths[l], 1, act[l]);
    in = act[l];
    cin = widths[l];
  }
}

double orc_job_step(orc_job* j, int pair) {
  const int h = j->ph[pair], w = j->pw[pair];
  const int npx = h * w;
  const int* wd = j->p.widths;
  j->lh = h;
  j->lw = w;
  forward_layers(wd, j->c0, j->theta, j->ow, j->ob, j->pin[pair], h, w, j->act);
  const int c8 = wd[ORC_LAYERS - 1];
  const double* w9 = j->theta + j->ow[ORC_LAYERS];
  orc_head_fwd(j->act[ORC_LAYERS - 1], c8, npx, w9, j->theta[j->ob[ORC_LAYERS]], j->z);
  j->last_loss = orc_loss(j->z, j->ptg[pair], npx, j->p.loss_kind, j->dz);

  /* backward: head */
  double* g = j->grad;
  memset(g, 0, sizeof(double) * j->np);
  {
    const double* a8 = j->act[ORC_LAYERS - 1];
    double* gw9 = g + j->ow[ORC_LAYERS];
    for (int c = 0; c < c8; ++c) {
      double s = 0.0;
      for (int p = 0; p < npx; ++p) s += j->dz[p] * a8[(size_t)c * npx + p];
      gw9[c] = s;
    }
    double s = 0.0;
    for (int p = 0; p < npx; ++p) s += j->dz[p];
    g[j->ob[ORC_LAYERS]] = s;
    double* d8 = j->delta[ORC_LAYERS - 1];
    for (int c = 0; c < c8; ++c)
      for (int p = 0; p < npx; ++p) {
        const size_t i = (size_t)c * npx + p;
        d8[i] = a8[i] > 0.0 ? j->dz[p] * w9[c] : 0.0;
      }
  }
  /* backward: conv layers 8..1 */
  for (int l = ORC_LAYERS - 1; l >= 0; --l) {
    const double* in = l > 0 ? j->act[l - 1] : j->pin[pair];
    const int cin = j->cin[l], cout = wd[l];
    orc_conv3x3_wgrad(j->delta[l], cout, h, w, in, cin, g + j->ow[l], g + j->ob[l]);
    if (l > 0) {
      double* dprev = j->delta[l - 1];
      orc_conv3x3_dgrad(j->delta[l], cout, h, w, j->theta + j->ow[l], cin, dprev);
      const double* aprev = j->act[l - 1];
      const size_t n = (size_t)cin * npx;
      for (size_t i = 0; i < n; ++i)
        if (!(aprev[i] > 0.0)) dprev[i] = 0.0;
    }
  }
  j->t += 1;
  orc_adam(j->theta, g, j->m, j->v, j->np, j->t, j->p.lr, j->p.beta1, j->p.beta2, j->p.eps);
  return j->last_loss;
}

void orc_net_forward_c(const int widths[ORC_LAYERS], int c0, const double* theta,
                       const double* img, int h, int w, double* v, double* z) {
  size_t ow[ORC_LAYERS + 1], ob[ORC_LAYERS + 1];
  param_offsets(widths, c0, ow, ob);
  const size_t npx = (size_t)h * w;
  double* act[ORC_LAYERS];
  for (int l = 0; l < ORC_LAYERS; ++l) act[l] = dalloc((size_t)widths[l] * npx);
  forward_layers(widths, c0, theta, ow, ob, img, h, w, act);
  double* zz = dalloc(npx);
  orc_head_fwd(act[ORC_LAYERS - 1], widths[ORC_LAYERS - 1], (int)npx, theta + ow[ORC_LAYERS],
               theta[ob[ORC_LAYERS]], zz);
  for (size_t p = 0; p < npx; ++p) {
    if (v) v[p] = orc_sigmoid(zz[p]);
    if (z) z[p] = zz[p];
  }
  free(zz);
  for (int l = 0; l < ORC_LAYERS; ++l) free(act[l]);
}

void orc_net_forward(const int widths[ORC_LAYERS], const double* theta, const double* img, int h,
                     int w, double* v, double* z) {
  orc_net_forward_c(widths, 1, theta, img, h, w, v, z);
}

/* Methods: after each epoch, run the full noisy image through the network and take the MSE
 * between that output and the noisy image itself (its predicted channel). */
double orc_job_validate(orc_job* j, double* v) {
  const size_t n = (size_t)j->H * j->W;
  orc_net_forward_c(j->p.widths, j->c0, j->theta, j->x, j->H, j->W, j->V, NULL);
  const double* y = j->x + (size_t)j->tc * n;
  double s = 0.0;
  for (size_t i = 0; i < n; ++i) s += (j->V[i] - y[i]) * (j->V[i] - y[i]);
  if (v) memcpy(v, j->V, sizeof(double) * n);
  return s / (double)n;
}

double orc_job_epoch(orc_job* j) {
  for (int k = 0; k < 4; ++k) orc_job_step(j, k);
  const double s = orc_job_validate(j, NULL);
  const size_t n = (size_t)j->H * j->W;
  const int improved = orc_stop_update(&j->st, s, j->p.patience, j->p.incl_best);
  if (improved) {
    memcpy(j->Vbest, j->V, sizeof(double) * n);
    for (size_t i = 0; i < n; ++i) j->S[i] = j->p.incl_best ? j->V[i] : 0.0;
  } else {
    for (size_t i = 0; i < n; ++i) j->S[i] += j->V[i];
  }
  return s;
}

void orc_job_run(orc_job* j, double* out) {
  const size_t n = (size_t)j->H * j->W;
  if (j->p.fixed_steps >= 0) {
    for (int k = 0; k < j->p.fixed_steps; ++k) orc_job_step(j, k % 4);
    orc_job_validate(j, out);
    return;
  }
  while (!j->st.stopped) {
    orc_job_epoch(j);
    if (!j->st.stopped && j->p.max_epochs > 0 && j->st.epoch >= j->p.max_epochs) {
      j->capped = 1;
      break;
    }
  }
  if (j->st.stopped) {
    for (size_t i = 0; i < n; ++i) out[i] = j->S[i] / j->p.patience;
  } else {
    /* cap reached before the rule fired: average what the window holds so far */
    const int cnt = j->st.since + (j->p.incl_best ? 1 : 0);
    for (size_t i = 0; i < n; ++i) out[i] = cnt > 0 ? j->S[i] / cnt : j->Vbest[i];
  }
}

size_t orc_job_get(const orc_job* j, int what, int layer, double* out) {
  size_t n = 0;
  const double* src = NULL;
  const size_t lpx = (size_t)j->lh * j->lw;
  switch (what) {
    case ORC_THETA: src = j->theta; n = j->np; break;
    case ORC_GRAD: src = j->grad; n = j->np; break;
    case ORC_ADAM_M: src = j->m; n = j->np; break;
    case ORC_ADAM_V: src = j->v; n = j->np; break;
    case ORC_ACT:
      if (layer < 1 || layer > ORC_LAYERS) return 0;
      src = j->act[layer - 1]; n = (size_t)j->p.widths[layer - 1] * lpx; break;
    case ORC_DELTA:
      if (layer < 1 || layer > ORC_LAYERS) return 0;
      src = j->delta[layer - 1]; n = (size_t)j->p.widths[layer - 1] * lpx; break;
    case ORC_Z: src = j->z; n = lpx; break;
    case ORC_DZ: src = j->dz; n = lpx; break;
    case ORC_PAIR_IN:
      if (layer < 0 || layer > 3) return 0;
      src = j->pin[layer]; n = (size_t)j->c0 * j->ph[layer] * j->pw[layer]; break;
    case ORC_PAIR_TGT:
      if (layer < 0 || layer > 3) return 0;
      src = j->ptg[layer]; n = (size_t)j->ph[layer] * j->pw[layer]; break;
    case ORC_SUM: src = j->S; n = (size_t)j->H * j->W; break;
    case ORC_VBEST: src = j->Vbest; n = (size_t)j->H * j->W; break;
    default: return 0;
  }
  if (out) memcpy(out, src, sizeof(double) * n);
  return n;
}

void orc_job_info(const orc_job* j, long* t, int* epoch, int* since, int* stopped, int* capped,
                  double* best, double* last_loss, int dims[4]) {
  if (t) *t = j->t;
  if (epoch) *epoch = j->st.epoch;
  if (since) *since = j->st.since;
  if (stopped) *stopped = j->st.stopped;
  if (capped) *capped = j->capped;
  if (best) *best = j->st.best;
  if (last_loss) *last_loss = j->last_loss;
  if (dims) {
    dims[0] = j->ph[0]; dims[1] = j->pw[0]; dims[2] = j->ph[2]; dims[3] = j->pw[2];
  }
}

void orc_job_free(orc_job* j) {
  if (!j) return;
  free(j->x);
  for (int k = 0; k < 4; ++k) {
    free(j->sub[k]);
    free(j->ptx[k]);
  }
  free(j->theta); free(j->grad); free(j->m); free(j->v);
  for (int l = 0; l < ORC_LAYERS; ++l) { free(j->act[l]); free(j->delta[l]); }
  free(j->z); free(j->dz); free(j->S); free(j->Vbest); free(j->V);
  free(j);
}

/* Maximum intensity projection along Z of the independently denoised slices. */
void orc_max_project(const double* vol, int Z, int H, int W, double* out) {
  const size_t n = (size_t)H * W;
  for (size_t p = 0; p < n; ++p) {
    double m = vol[p];
    for (int z = 1; z < Z; ++z)
      if (vol[(size_t)z * n + p] > m) m = vol[(size_t)z * n + p];
    out[p] = m;
  }
}
