// C ABI of the library: defaults, the trainer API, op-level entry points and the job
// scheduler (admission by HBM budget, epochs enqueued ahead of a device-side stop flag,
// several jobs resident at once on their own streams).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "trainer.h"

using namespace n2f;

#define CKR(expr)                                            \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return set_cuda_error(_e, #expr); \
  } while (0)

extern "C" {

void n2f_config_default(n2f_config* c) {
  memset(c, 0, sizeof(*c));
  c->struct_size = sizeof(n2f_config);
  c->device = 0;
  c->hbm_budget_bytes = 150ull << 30;
  c->max_slots = 64;
  c->lookahead = 2;
  c->use_graphs = 1;
}

void n2f_params_default(n2f_params* p) {
  memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(n2f_params);
  p->lr = 1e-3;
  p->beta1 = 0.9;
  p->beta2 = 0.999;
  p->eps = 1e-8;
  p->patience = 100;
  p->max_epochs = 0;
  p->fixed_steps = -1;
  p->seed = 0;
  p->precision = N2F_FP32;
  p->loss = N2F_LOSS_BCE;
  p->widths = N2F_WIDTHS_PLIT;
  p->incl_best = 0;
  p->engine = N2F_ENGINE_AUTO;
  p->channels = 1;
  p->target_channel = 0;
  p->downsample = N2F_DOWN_CHECKER;
  p->exact = 0;
  p->overlap = 0;
}

const char* n2f_strerror(int code) {
  switch (code) {
    case N2F_OK: return "ok";
    case N2F_EINVAL: return "invalid argument";
    case N2F_ETOOBIG: return "job can never fit the HBM budget";
    case N2F_EAGAIN: return "result not ready";
    case N2F_ENOENT: return "unknown or collected job";
    case N2F_ETIMEDOUT: return "wait timed out";
    case N2F_ENONFINITE: return "training diverged (non-finite validation score)";
    case N2F_EDEVICE: return tl_error.empty() ? "CUDA error" : tl_error.c_str();
    case N2F_ENOMEM: return tl_error.empty() ? "out of memory" : tl_error.c_str();
    case N2F_ECANCELED: return "job cancelled";
    case N2F_ENOTSUP: return "not supported by this build";
    default: return "unknown error";
  }
}

size_t n2f_param_count(int widths) {
  NetShape s;
  s.init(widths);
  return s.count;
}

}  // extern "C"

static int check_params(const n2f_params* p) {
  if (!p || p->struct_size != sizeof(n2f_params)) return N2F_EINVAL;
  if (p->precision != N2F_FP32 && p->precision != N2F_BF16) return N2F_EINVAL;
  if (p->loss != N2F_LOSS_BCE && p->loss != N2F_LOSS_MSE) return N2F_EINVAL;
  if (p->widths != N2F_WIDTHS_PLIT && p->widths != N2F_WIDTHS_W64) return N2F_EINVAL;
  if (p->engine < N2F_ENGINE_AUTO || p->engine > N2F_ENGINE_TC) return N2F_EINVAL;
  if (!(p->lr > 0.0 && p->lr < 1e30) || !(p->beta1 >= 0.0 && p->beta1 < 1.0) ||
      !(p->beta2 >= 0.0 && p->beta2 < 1.0) || !(p->eps > 0.0 && p->eps < 1e30))
    return N2F_EINVAL;
  if (p->fixed_steps < 0 && p->patience < 1) return N2F_EINVAL;
  if (p->incl_best && p->patience < 2) return N2F_EINVAL;
  if (p->channels < 0 || p->channels > kMaxC0) return N2F_EINVAL;
  if (p->target_channel < 0 || p->target_channel >= std::max(1, (int)p->channels))
    return N2F_EINVAL;
  if (p->downsample != N2F_DOWN_CHECKER && p->downsample != N2F_DOWN_QUAD) return N2F_EINVAL;
  if (p->exact != 0 && p->exact != 1) return N2F_EINVAL;
  if (p->overlap != 0 && p->overlap != 1) return N2F_EINVAL;
  return N2F_OK;
}

// planes of a job's image: the input channels, then the clean plane for the Exact ablation
static size_t planes(const n2f_params* p) {
  return (size_t)std::max(1, (int)p->channels) + (p->exact ? 1 : 0);
}

static int check_image(int H, int W) {
  if (H < 2 || W < 2) return N2F_EINVAL;
  if ((size_t)H * W >= ((size_t)1 << 31)) return N2F_EINVAL;  // pixel indices are 32-bit ints
  return N2F_OK;
}

// ------------------------------------------------------------------------------------------
// Trainer API
struct n2f_trainer {
  Trainer t;
  bool own_stream;
};

extern "C" int n2f_trainer_create(n2f_trainer** out, const float* image, int H, int W,
                                  const n2f_params* p, void* stream) {
  if (!out || !image) return N2F_EINVAL;
  n2f_params def;
  n2f_params_default(&def);
  if (!p) p = &def;
  int rc = check_params(p);
  if (rc) return rc;
  if ((rc = check_image(H, W))) return rc;
  for (size_t i = 0; i < planes(p) * H * W; ++i)
    if (!isfinite(image[i])) return N2F_EINVAL;
  n2f_trainer* tr = new n2f_trainer();
  tr->own_stream = false;
  if ((rc = trainer_configure(&tr->t, H, W, p, 1))) {
    delete tr;
    return rc;
  }
  Allocator al;
  if ((rc = trainer_init(&tr->t, al, (cudaStream_t)stream, 0))) {
    delete tr;
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(tr->t.x, image, sizeof(float) * planes(p) * H * W,
                                  cudaMemcpyHostToDevice, tr->t.st);
  if (e != cudaSuccess) {
    trainer_release(&tr->t);
    delete tr;
    return set_cuda_error(e, "image upload");
  }
  if ((rc = trainer_start(&tr->t, 0))) {
    trainer_release(&tr->t);
    delete tr;
    return rc;
  }
  *out = tr;
  return N2F_OK;
}

extern "C" void n2f_trainer_destroy(n2f_trainer* tr) {
  if (!tr) return;
  cudaStreamSynchronize(tr->t.st);
  trainer_release(&tr->t);
  delete tr;
}

extern "C" int n2f_trainer_step(n2f_trainer* tr, int pair) {
  if (!tr || pair < 0 || pair > 3) return N2F_EINVAL;
  return trainer_step(&tr->t, pair);
}

extern "C" int n2f_trainer_validate(n2f_trainer* tr) {
  if (!tr) return N2F_EINVAL;
  return trainer_validate(&tr->t);
}

extern "C" int n2f_trainer_epoch(n2f_trainer* tr) {
  if (!tr) return N2F_EINVAL;
  return trainer_epoch(&tr->t);
}

extern "C" int n2f_trainer_run(n2f_trainer* tr, int max_epochs) {
  if (!tr) return N2F_EINVAL;
  Trainer* t = &tr->t;
  if (t->fixed_mode) {
    for (int k = 0; k < t->prm.fixed_steps; ++k) {
      int rc = trainer_step(t, k % 4);
      if (rc) return rc;
    }
    int rc = trainer_validate(t);
    if (rc) return rc;
    return trainer_finish(t);
  }
  DevState s;
  for (int e = 0; max_epochs <= 0 || e < max_epochs; e += 4) {
    for (int k = 0; k < 4; ++k) {
      int rc = trainer_epoch(t);
      if (rc) return rc;
    }
    int rc = trainer_read_state(t, &s);
    if (rc) return rc;
    if (s.kerr) {
      tl_error = "a device wait ran out of time";
      return N2F_ETIMEDOUT;
    }
    if (s.stopped) break;
  }
  return trainer_finish(t);
}

extern "C" int n2f_trainer_finish(n2f_trainer* tr) {
  if (!tr) return N2F_EINVAL;
  return trainer_finish(&tr->t);
}

extern "C" int n2f_trainer_set_theta(n2f_trainer* tr, const double* theta, size_t n) {
  if (!tr || !theta || n != tr->t.net.count) return N2F_EINVAL;
  std::vector<float> f(n);
  for (size_t i = 0; i < n; ++i) f[i] = (float)theta[i];
  CKR(cudaMemcpyAsync(tr->t.theta, f.data(), n * sizeof(float), cudaMemcpyHostToDevice,
                      tr->t.st));
  CKR(cudaStreamSynchronize(tr->t.st));
  return trainer_repack(&tr->t);
}

// Copies a device float array, or a CG map converted to NCHW, into host doubles.
static int export_floats(cudaStream_t st, const float* d, size_t n, double* out) {
  std::vector<float> h(n);
  CKR(cudaMemcpyAsync(h.data(), d, n * sizeof(float), cudaMemcpyDeviceToHost, st));
  CKR(cudaStreamSynchronize(st));
  for (size_t i = 0; i < n; ++i) out[i] = h[i];
  return N2F_OK;
}

static int export_cg(Trainer* t, const void* cg, int C, int h, int w, double* out) {
  const size_t n = (size_t)C * h * w;
  float* tmp = nullptr;
  CKR(cudaMallocAsync((void**)&tmp, n * sizeof(float), t->st));
  cudaError_t e = launch_unpack_cg(cg, C, h, w, t->bf16, tmp, t->st);
  int rc = e == cudaSuccess ? export_floats(t->st, tmp, n, out) : set_cuda_error(e, "unpack");
  cudaFreeAsync(tmp, t->st);
  cudaStreamSynchronize(t->st);
  return rc;
}

// The ring holds the score of epoch e at (e - 1) % kHistCap: writes the last min(end, kHistCap)
// of epochs 1..end oldest first.
static void hist_unroll(const double* ring, int end, double* out) {
  const int n = std::min(end, kHistCap);
  for (int k = 0; k < n; ++k) {
    const int e = end - n + 1 + k;  // 1-based epoch
    out[k] = ring[(e - 1) % kHistCap];
  }
}

extern "C" int n2f_trainer_export(n2f_trainer* tr, int what, int index, double* out, size_t cap,
                                  size_t* n_out) {
  if (!tr) return N2F_EINVAL;
  int hist_end = 0;
  Trainer* t = &tr->t;
  const int h = t->ph[t->last_pair], w = t->pw[t->last_pair];
  size_t n = 0;
  switch (what) {
    case N2F_X_THETA: case N2F_X_GRAD: case N2F_X_ADAM_M: case N2F_X_ADAM_V: n = t->net.count; break;
    case N2F_X_ACT: case N2F_X_DELTA:
      if (index < 1 || index > kLayers) return N2F_EINVAL;
      n = (size_t)t->net.widths[index - 1] * h * w;
      break;
    case N2F_X_DZ: n = (size_t)h * w; break;
    case N2F_X_PAIR:
      if (index < 0 || index > 3) return N2F_EINVAL;
      n = (size_t)t->net.c0 * t->ph[index] * t->pw[index];
      break;
    case N2F_X_VAL: case N2F_X_SUM: case N2F_X_OUT: case N2F_X_VBEST: n = t->N; break;
    case N2F_X_HIST: {
      DevState s;
      const int rc = trainer_read_state(t, &s);
      if (rc) return rc;
      n = (size_t)std::min(s.epoch, kHistCap);
      hist_end = s.epoch;
      break;
    }
    default: return N2F_EINVAL;
  }
  if (n_out) *n_out = n;
  if (!out) return N2F_OK;
  if (cap < n) return N2F_EINVAL;
  switch (what) {
    case N2F_X_THETA: return export_floats(t->st, t->theta, n, out);
    case N2F_X_GRAD: return export_floats(t->st, t->grad, n, out);
    case N2F_X_ADAM_M: return export_floats(t->st, t->m, n, out);
    case N2F_X_ADAM_V: return export_floats(t->st, t->v, n, out);
    case N2F_X_ACT: return export_cg(t, t->act[index - 1], t->net.widths[index - 1], h, w, out);
    case N2F_X_DELTA: return export_cg(t, t->dkeep[index - 1], t->net.widths[index - 1], h, w, out);
    case N2F_X_DZ: return export_floats(t->st, t->dz, n, out);
    case N2F_X_PAIR: return export_floats(t->st, t->sub[index], n, out);
    case N2F_X_VAL: return export_floats(t->st, t->V, n, out);
    case N2F_X_SUM: return export_floats(t->st, t->S, n, out);
    case N2F_X_OUT: return export_floats(t->st, t->out, n, out);
    case N2F_X_VBEST: return export_floats(t->st, t->Vbest, n, out);
    case N2F_X_HIST: {
      std::vector<double> ring(kHistCap);
      CKR(cudaMemcpyAsync(ring.data(), t->hist, kHistCap * sizeof(double), cudaMemcpyDeviceToHost,
                          t->st));
      CKR(cudaStreamSynchronize(t->st));
      hist_unroll(ring.data(), hist_end, out);
      return N2F_OK;
    }
  }
  return N2F_EINVAL;
}

static int import_floats(cudaStream_t st, float* d, const double* in, size_t n) {
  std::vector<float> f(n);
  for (size_t i = 0; i < n; ++i) f[i] = (float)in[i];
  CKR(cudaMemcpyAsync(d, f.data(), n * sizeof(float), cudaMemcpyHostToDevice, st));
  CKR(cudaStreamSynchronize(st));
  return N2F_OK;
}

extern "C" int n2f_trainer_import(n2f_trainer* tr, int what, int index, const double* in,
                                  size_t n) {
  (void)index;
  if (!tr || !in) return N2F_EINVAL;
  Trainer* t = &tr->t;
  switch (what) {
    case N2F_X_THETA: return n2f_trainer_set_theta(tr, in, n);
    case N2F_X_ADAM_M: case N2F_X_ADAM_V:
      if (n != t->net.count) return N2F_EINVAL;
      return import_floats(t->st, what == N2F_X_ADAM_M ? t->m : t->v, in, n);
    case N2F_X_SUM: case N2F_X_VBEST:
      if (n != t->N) return N2F_EINVAL;
      return import_floats(t->st, what == N2F_X_SUM ? t->S : t->Vbest, in, n);
  }
  return N2F_EINVAL;
}

extern "C" int n2f_trainer_set_progress(n2f_trainer* tr, uint32_t steps, uint32_t epoch,
                                        uint32_t since, double best) {
  if (!tr) return N2F_EINVAL;
  Trainer* t = &tr->t;
  if (t->fixed_mode || since > epoch || epoch > (uint32_t)INT32_MAX || steps > (uint32_t)INT32_MAX)
    return N2F_EINVAL;
  DevState s;
  int rc = trainer_read_state(t, &s);
  if (rc) return rc;
  s.t = (int)steps;
  // beta^t by repeated products, as the step kernel forms it one step at a time
  s.b1t = 1.0;
  s.b2t = 1.0;
  for (uint32_t k = 0; k < steps; ++k) {
    s.b1t *= t->prm.beta1;
    s.b2t *= t->prm.beta2;
  }
  s.bc1 = (float)(1.0 - s.b1t);
  s.bc2 = (float)(1.0 - s.b2t);
  s.epoch = (int)epoch;
  s.since = (int)since;
  s.best = best;
  s.stopped = 0;
  s.decision = -1;
  CKR(cudaMemcpyAsync(t->state, &s, sizeof(DevState), cudaMemcpyHostToDevice, t->st));
  CKR(cudaStreamSynchronize(t->st));
  return N2F_OK;
}

extern "C" int n2f_trainer_status(n2f_trainer* tr, n2f_status* st) {
  if (!tr || !st || st->struct_size != sizeof(n2f_status)) return N2F_EINVAL;
  DevState s;
  int rc = trainer_read_state(&tr->t, &s);
  if (rc) return rc;
  fill_status(&tr->t, s, st);
  st->state = s.stopped ? N2F_DONE : N2F_RUNNING;
  st->error = s.kerr ? N2F_ETIMEDOUT : (s.stopped == 3 ? N2F_ENONFINITE : N2F_OK);
  if (s.stopped == 3 || s.kerr) st->state = N2F_FAILED;
  return N2F_OK;
}

extern "C" uint64_t n2f_trainer_launches(const n2f_trainer* tr) { return tr ? tr->t.launches : 0; }

// ------------------------------------------------------------------------------------------
// Op-level entry points
extern "C" int n2f_checker_gather(const float* x, int H, int W, float* up_e, float* up_o,
                                  float* lf_e, float* lf_o, void* stream) {
  if (!x || !up_e || !up_o || !lf_e || !lf_o || check_image(H, W)) return N2F_EINVAL;
  CKR(launch_gather(x, H, W, up_e, up_o, lf_e, lf_o, (cudaStream_t)stream));
  return N2F_OK;
}

extern "C" int n2f_max_project(const float* vol, int Z, int H, int W, float* out, void* stream) {
  if (!vol || !out || Z < 1 || H < 1 || W < 1) return N2F_EINVAL;
  CKR(launch_max_project(vol, Z, (size_t)H * W, out, (cudaStream_t)stream));
  return N2F_OK;
}

// the op-level entry points take one of the two precision forms and one of the engines by value
static bool valid_form(int precision) { return precision == N2F_FP32 || precision == N2F_BF16; }
static bool valid_engine(int engine) {
  return engine >= N2F_ENGINE_AUTO && engine <= N2F_ENGINE_TC;
}

extern "C" int n2f_pack_cg(const float* nchw, int C, int H, int W, int precision, void* cg,
                           void* stream) {
  const int G = precision == N2F_BF16 ? 8 : 4;
  if (!valid_form(precision) || !nchw || !cg || C < G || C % G || H < 1 || W < 1)
    return N2F_EINVAL;
  CKR(launch_pack_cg(nchw, C, H, W, precision == N2F_BF16, cg, (cudaStream_t)stream));
  return N2F_OK;
}

extern "C" int n2f_unpack_cg(const void* cg, int C, int H, int W, int precision, float* nchw,
                             void* stream) {
  const int G = precision == N2F_BF16 ? 8 : 4;
  if (!valid_form(precision) || !nchw || !cg || C < G || C % G || H < 1 || W < 1)
    return N2F_EINVAL;
  CKR(launch_unpack_cg(cg, C, H, W, precision == N2F_BF16, nchw, (cudaStream_t)stream));
  return N2F_OK;
}

static int resolve_engine(int engine, int cin, int cout) {
  if (engine == N2F_ENGINE_SIMT) return N2F_ENGINE_SIMT;
  const bool tc = tc_supported(cin, cout);
  if (engine == N2F_ENGINE_TC) return tc ? N2F_ENGINE_TC : -1;
  return tc ? N2F_ENGINE_TC : N2F_ENGINE_SIMT;
}

extern "C" int n2f_conv3x3(int mode, int engine, int precision, const void* in, int cin, int cout,
                           int H, int W, const float* w, const float* b, const void* mask,
                           void* out, void* stream) {
  if (!in || !out || !w || (mode == 0 && !b) || (mode == 1 && !mask) || H < 1 || W < 1 ||
      cin % 8 || cout % 8 || cin < 8 || cout < 8 || (mode != 0 && mode != 1) ||
      !valid_form(precision) || !valid_engine(engine))
    return N2F_EINVAL;
  const int bf16 = precision == N2F_BF16;
  const int eng = resolve_engine(engine, cin, cout);
  if (eng < 0) return N2F_ENOTSUP;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nw = (size_t)cin * cout * 9;
  char* buf = nullptr;
  const size_t bytes = 2 * nw * sizeof(float) + 4 * nw * 2 + 4096 + 256;
  CKR(cudaMallocAsync((void**)&buf, bytes, st));
  float* fwd = (float*)buf;
  float* dgr = fwd + nw;
  char* tc0 = (char*)(dgr + nw);
  void *tcf = nullptr, *tcd = nullptr, *tcf_lo = nullptr, *tcd_lo = nullptr;
  const bool tc = eng == N2F_ENGINE_TC;
  if (tc) {  // 16-bit copies: bf16, or the float32 form's fp16 hi and lo parts
    tcf = tc0;
    tcd = tc0 + nw * 2;
    if (!bf16) {
      tcf_lo = tc0 + 2 * nw * 2;
      tcd_lo = tc0 + 3 * nw * 2;
    }
  }
  int* err = (int*)(tc0 + 4 * nw * 2);
  // float32 form: the largest weight and the largest input value set the operand scales
  unsigned* wmax = (unsigned*)(err + 1);
  unsigned* imax = wmax + 1;
  const ConvScales sc{imax, wmax, nullptr};
  const size_t n_in = (size_t)(mode == 0 ? cin : cout) * H * W;
  cudaError_t e = cudaMemsetAsync(err, 0, 4 * sizeof(int), st);
  if (e == cudaSuccess)
    e = launch_pack_layer(w, cin, cout, fwd, dgr, tcf, tcd, tcf_lo, tcd_lo, bf16, wmax, st);
  if (e == cudaSuccess && tc && !bf16) e = launch_absmax(in, n_in, 0, imax, nullptr, st);
  if (e == cudaSuccess) {
    if (mode == 0) {
      e = tc ? launch_conv_tc(0, bf16, in, cin, cout, H, W, tcf, tcf_lo, b, nullptr, out, sc,
                              nullptr, err, st)
             : launch_conv_simt(0, bf16, in, cin, cout, H, W, fwd, b, nullptr, out, nullptr, st);
    } else {
      // dgrad: `in` has C_out channels, `out` and `mask` have C_in
      e = tc ? launch_conv_tc(1, bf16, in, cout, cin, H, W, tcd, tcd_lo, nullptr, mask, out, sc,
                              nullptr, err, st)
             : launch_conv_simt(1, bf16, in, cout, cin, H, W, dgr, nullptr, mask, out, nullptr,
                                st);
    }
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return set_cuda_error(e, "n2f_conv3x3");
  return herr ? N2F_ETIMEDOUT : N2F_OK;
}

extern "C" int n2f_conv3x3_wgrad(int engine, int precision, const void* dout, const void* in,
                                 int cin, int cout, int H, int W, float* dw, float* db,
                                 void* stream) {
  if (!dout || !in || !dw || !db || H < 1 || W < 1 || cin % 8 || cout % 8 || cin < 8 ||
      cout < 8 || !valid_form(precision) || !valid_engine(engine))
    return N2F_EINVAL;
  const int bf16 = precision == N2F_BF16;
  int eng = resolve_engine(engine, cin, cout);
  if (eng == N2F_ENGINE_TC && !tc_wgrad_supported(cin, cout, bf16))
    eng = engine == N2F_ENGINE_TC ? -1 : N2F_ENGINE_SIMT;
  if (eng < 0) return N2F_ENOTSUP;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t cap = (size_t)16 << 20;
  float* part = nullptr;
  CKR(cudaMallocAsync((void**)&part, cap * sizeof(float) + 256, st));
  int* err = (int*)(part + cap);
  unsigned* dmax = (unsigned*)(err + 1);  // float32 form: operand scales
  unsigned* xmax = dmax + 1;
  const bool tc = eng == N2F_ENGINE_TC;
  cudaError_t e = cudaMemsetAsync(err, 0, 4 * sizeof(int), st);
  if (e == cudaSuccess && tc && !bf16)
    e = launch_absmax(dout, (size_t)cout * H * W, 0, dmax, nullptr, st);
  if (e == cudaSuccess && tc && !bf16) e = launch_absmax(in, (size_t)cin * H * W, 0, xmax, nullptr, st);
  if (e == cudaSuccess)
    e = tc ? launch_wgrad_tc(bf16, dout, in, cin, cout, H, W, dmax, xmax, part, cap, dw, db,
                             nullptr, err, st)
           : launch_wgrad_simt(bf16, dout, in, cin, cout, H, W, part, cap, dw, db, nullptr, st);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(part, st);
  if (e != cudaSuccess) return set_cuda_error(e, "n2f_conv3x3_wgrad");
  return herr ? N2F_ETIMEDOUT : N2F_OK;
}

extern "C" int n2f_check_status(uint64_t* failures, int* first_site, int clear) {
  if (!failures || !first_site) return N2F_EINVAL;
#ifndef N2F_CHECKED
  (void)clear;
  return N2F_ENOTSUP;
#else
  CKR(cudaDeviceSynchronize());
  int (*const readers[4])(unsigned long long*, int*, int) = {check_read_basic, check_read_simt,
                                                            check_read_conv, check_read_wgrad};
  uint64_t total = 0;
  int site = 0;
  for (int k = 0; k < 4; ++k) {
    unsigned long long f = 0;
    int line = 0;
    if (readers[k](&f, &line, clear)) return set_cuda_error(cudaGetLastError(), "n2f_check_status");
    total += f;
    if (f && !site) site = (k + 1) * 100000 + line;
  }
  *failures = total;
  *first_site = site;
  return N2F_OK;
#endif
}

// ------------------------------------------------------------------------------------------
// Job scheduler
namespace {

using Clock = std::chrono::steady_clock;

struct Group;

struct Job {
  n2f_job id = 0;
  Group* grp = nullptr;  // lockstep group (nullptr: the job runs alone)
  int H = 0, W = 0;
  n2f_params prm;
  int src_kind = 0;  // 0 host f32, 1 device f32, 2 host u16
  float* pin_in = nullptr;
  uint16_t* pin_u16 = nullptr;
  const float* dev_in = nullptr;
  float* pin_out = nullptr;
  double* pin_hist = nullptr;  // the device history ring, copied out with the result
  std::atomic<int> state{N2F_QUEUED};
  int error = 0;
  bool cancel = false;
  Trainer tr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_start = nullptr, ev_in = nullptr, ev_out = nullptr, ev_done = nullptr;
  KTimer kt;
  // ring of host mirrors of the device state, one per epoch in flight
  DevState* hst = nullptr;
  cudaEvent_t ev_ep[8] = {};
  int ring = 0;
  uint64_t ep_enq = 0, ep_seen = 0;
  bool finishing = false, result_enq = false;
  DevState last;
  Clock::time_point t_submit, t_done;
  double device_ms = 0, compute_ms = 0, t0_ms = 0, t1_ms = 0;
};

// Jobs stepped in lockstep (n2f_config.group_size): one stream, one epoch graph, the grouped
// tensor-core launches; each member keeps its own state ring for the host's epoch reads.
struct Group {
  std::vector<Job*> m;
  TrainerGroup tg;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_ep[8] = {};
  int ring = 0;
  uint64_t ep_enq = 0, ep_seen = 0;
  bool finishing = false, results = false;
  int fail_rc = 0;    // set when the group failed: every member then finishes with it
  int remaining = 0;  // references: unfinished members (+ one while the worker sets it up)
};

void group_unref(Group* g) {
  if (--g->remaining > 0) return;
  if (g->st) cudaStreamSynchronize(g->st);
  group_release(&g->tg);
  for (int k = 0; k < 8; ++k)
    if (g->ev_ep[k]) cudaEventDestroy(g->ev_ep[k]);
  if (g->st) cudaStreamDestroy(g->st);
  delete g;
}

// Jobs that may share a group: everything that shapes the kernels and the schedule is equal,
// the image size included -- members of different sizes run their per-member kernels for
// different times, and the group's epoch waits for the largest at every join.
bool same_group_key(const Job* a, const Job* b) {
  const n2f_params &p = a->prm, &q = b->prm;
  return a->H == b->H && a->W == b->W &&
         p.precision == q.precision && p.widths == q.widths && p.engine == q.engine &&
         p.loss == q.loss && p.channels == q.channels && p.downsample == q.downsample &&
         p.exact == q.exact && p.fixed_steps < 0 && q.fixed_steps < 0 &&
         a->src_kind != 2 && b->src_kind != 2;
}

}  // namespace

struct n2f_ctx {
  n2f_config cfg;
  Allocator al;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> queue;
  std::vector<Job*> active;
  std::unordered_map<n2f_job, Job*> jobs;
  bool stop = false;
  uint64_t next_id = 1;
  uint64_t launches = 0;
  size_t bytes_resident = 0;
  uint32_t n_done = 0;
  cudaEvent_t ev_ref = nullptr;
  KTimer prof;  // totals of the profiled kernel class over finished jobs
};

static void free_job_host(Job* j) {
  if (j->pin_in) cudaFreeHost(j->pin_in);
  if (j->pin_u16) cudaFreeHost(j->pin_u16);
  if (j->pin_out) cudaFreeHost(j->pin_out);
  if (j->hst) cudaFreeHost(j->hst);
  if (j->pin_hist) cudaFreeHost(j->pin_hist);
  j->pin_hist = nullptr;
  j->pin_in = nullptr;
  j->pin_u16 = nullptr;
  j->pin_out = nullptr;
  j->hst = nullptr;
}

static void release_device(n2f_ctx* c, Job* j) {
  if (j->st) cudaStreamSynchronize(j->st);
  trainer_release(&j->tr);
  j->kt.destroy();
  for (int k = 0; k < 8; ++k)
    if (j->ev_ep[k]) cudaEventDestroy(j->ev_ep[k]), j->ev_ep[k] = nullptr;
  for (cudaEvent_t* e : {&j->ev_start, &j->ev_in, &j->ev_out, &j->ev_done})
    if (*e) cudaEventDestroy(*e), *e = nullptr;
  if (Group* g = j->grp) {
    j->st = nullptr;  // the group's stream
    j->grp = nullptr;
    group_unref(g);
  }
  if (j->st) cudaStreamDestroy(j->st), j->st = nullptr;
  std::lock_guard<std::mutex> g(c->mu);
  c->bytes_resident -= j->bytes;
}

static void finish_job(n2f_ctx* c, Job* j, int state, int err) {
  j->t_done = Clock::now();
  j->error = err;
  release_device(c, j);
  {
    std::lock_guard<std::mutex> g(c->mu);
    j->state.store(state);
    c->active.erase(std::remove(c->active.begin(), c->active.end(), j), c->active.end());
    c->n_done += 1;
  }
  c->cv_done.notify_all();
}

// Creates the device state of a job and enqueues upload, gather and initialisation.
static int admit(n2f_ctx* c, Job* j) {
  LaunchScope ls(&c->launches);
  if (j->grp)
    j->st = j->grp->st;
  else
    CKR(cudaStreamCreateWithFlags(&j->st, cudaStreamNonBlocking));
  CKR(cudaEventCreate(&j->ev_start));
  CKR(cudaEventCreate(&j->ev_in));
  CKR(cudaEventCreate(&j->ev_out));
  CKR(cudaEventCreate(&j->ev_done));
  j->kt.kind = j->grp ? N2F_K_NONE : c->cfg.profile_kernel;
  if (j->kt.kind != N2F_K_NONE) j->tr.kt = &j->kt;
  j->tr.profile_every = std::max<uint32_t>(1, c->cfg.profile_every);
  j->ring = (int)std::min<uint32_t>(8, std::max<uint32_t>(2, c->cfg.lookahead + 1));
  for (int k = 0; k < j->ring; ++k) CKR(cudaEventCreateWithFlags(&j->ev_ep[k], cudaEventDisableTiming));
  CKR(cudaMallocHost((void**)&j->hst, sizeof(DevState) * j->ring));
  CKR(cudaMallocHost((void**)&j->pin_out, sizeof(float) * (size_t)j->H * j->W));
  CKR(cudaMallocHost((void**)&j->pin_hist, sizeof(double) * kHistCap));
  int rc = trainer_init(&j->tr, c->al, j->st, j->src_kind == 2);
  if (rc) return rc;
  CKR(cudaEventRecord(j->ev_start, j->st));
  const size_t n = (size_t)j->H * j->W, nin = planes(&j->prm) * n;
  if (j->src_kind == 0)
    CKR(cudaMemcpyAsync(j->tr.x, j->pin_in, nin * sizeof(float), cudaMemcpyHostToDevice, j->st));
  else if (j->src_kind == 1)
    CKR(cudaMemcpyAsync(j->tr.x, j->dev_in, nin * sizeof(float), cudaMemcpyDeviceToDevice, j->st));
  else
    CKR(cudaMemcpyAsync(j->tr.in_u16, j->pin_u16, n * sizeof(uint16_t), cudaMemcpyHostToDevice,
                        j->st));
  CKR(cudaEventRecord(j->ev_in, j->st));
  rc = trainer_start(&j->tr, j->src_kind == 2);
  if (rc) return rc;
  if (c->cfg.autotune && (rc = trainer_autotune(&j->tr))) return rc;
  if (j->tr.fixed_mode) {
    for (int k = 0; k < j->prm.fixed_steps; ++k)
      if ((rc = trainer_step(&j->tr, k % 4))) return rc;
    if ((rc = trainer_validate(&j->tr))) return rc;
    j->finishing = true;
  }
  return N2F_OK;
}

// Advances a lockstep group without blocking (called through its first member).
static bool group_progress(n2f_ctx* c, Group* g) {
  bool did = false;
  int rc = 0;
  // members finish themselves (in their own progress calls) once the group has failed
  auto fail_all = [&](int err) { g->fail_rc = err; };
  while (!g->finishing && g->ep_seen < g->ep_enq) {
    const int slot = (int)(g->ep_seen % g->ring);
    const cudaError_t q = cudaEventQuery(g->ev_ep[slot]);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) {
      set_cuda_error(q, "group epoch");
      fail_all(N2F_EDEVICE);
      return true;
    }
    int stopped = 0, kerr = 0;
    for (Job* j : g->m) {
      {
        std::lock_guard<std::mutex> lk(c->mu);
        j->last = j->hst[slot];
      }
      stopped += j->last.stopped != 0;
      kerr |= j->last.kerr;
    }
    g->ep_seen += 1;
    did = true;
    if (kerr) {
      tl_error = "a device wait ran out of time";
      fail_all(N2F_ETIMEDOUT);
      return true;
    }
    if (stopped == (int)g->m.size()) g->finishing = true;
  }
  const uint32_t la = std::max<uint32_t>(1, c->cfg.lookahead);
  while (!g->finishing && g->ep_enq - g->ep_seen < la) {
    if ((rc = !c->cfg.use_graphs ? group_epoch(&g->tg) : group_epoch_graph(&g->tg))) break;
    const int slot = (int)(g->ep_enq % g->ring);
    cudaError_t e = cudaSuccess;
    for (Job* j : g->m)
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&j->hst[slot], j->tr.state, sizeof(DevState), cudaMemcpyDeviceToHost,
                            g->st);
    if (e == cudaSuccess) e = cudaEventRecord(g->ev_ep[slot], g->st);
    if (e != cudaSuccess) {
      rc = set_cuda_error(e, "group epoch enqueue");
      break;
    }
    g->ep_enq += 1;
    did = true;
  }
  if (rc) {
    fail_all(rc);
    return true;
  }
  if (g->finishing && !g->results) {
    // each member enqueues its result on its own stream, after the group's last epoch
    cudaError_t e = cudaEventRecord(g->tg.ev_fork, g->st);
    for (Job* j : g->m)
      if (e == cudaSuccess) e = cudaStreamWaitEvent(j->st, g->tg.ev_fork, 0);
    if (e != cudaSuccess) {
      fail_all(set_cuda_error(e, "group results"));
      return true;
    }
    for (Job* j : g->m) j->finishing = true;
    g->results = true;
    did = true;
  }
  return did;
}

// Advances one running job without blocking. Returns true if it enqueued or finished work.
static bool progress(n2f_ctx* c, Job* j) {
  LaunchScope ls(&c->launches);
  bool did = false;
  int rc = 0;
  if (j->grp && j->grp->fail_rc) {
    finish_job(c, j, N2F_FAILED, j->grp->fail_rc);
    return true;
  }
  if (j->grp && !j->result_enq) {
    // a group member: epochs are the group's; a cancelled member finishes with its group
    if (j == j->grp->m[0] && group_progress(c, j->grp)) return true;
    if (!j->finishing) return false;
  }
  if (j->cancel && !j->grp) {
    finish_job(c, j, N2F_CANCELED, N2F_ECANCELED);
    return true;
  }
  if (!j->finishing) {
    while (j->ep_seen < j->ep_enq) {
      const int slot = (int)(j->ep_seen % j->ring);
      const cudaError_t q = cudaEventQuery(j->ev_ep[slot]);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        set_cuda_error(q, "epoch");
        finish_job(c, j, N2F_FAILED, N2F_EDEVICE);
        return true;
      }
      {
        std::lock_guard<std::mutex> g(c->mu);
        j->last = j->hst[slot];
      }
      j->ep_seen += 1;
      did = true;
      if (j->last.kerr) {
        tl_error = "a device wait ran out of time";
        finish_job(c, j, N2F_FAILED, N2F_ETIMEDOUT);
        return true;
      }
      if (j->last.stopped) {
        j->finishing = true;
        break;
      }
    }
    const uint32_t la = std::max<uint32_t>(1, c->cfg.lookahead);
    while (!j->finishing && j->ep_enq - j->ep_seen < la) {
      // epochs replay a captured graph (timed launches keep event-record nodes in it)
      if ((rc = !c->cfg.use_graphs ? trainer_epoch_job(&j->tr) : trainer_epoch_graph(&j->tr)))
        break;
      const int slot = (int)(j->ep_enq % j->ring);
      cudaError_t e = cudaMemcpyAsync(&j->hst[slot], j->tr.state, sizeof(DevState),
                                      cudaMemcpyDeviceToHost, j->st);
      if (e == cudaSuccess) e = cudaEventRecord(j->ev_ep[slot], j->st);
      if (e != cudaSuccess) {
        rc = set_cuda_error(e, "epoch enqueue");
        break;
      }
      j->ep_enq += 1;
      did = true;
    }
    if (rc) {
      finish_job(c, j, N2F_FAILED, rc);
      return true;
    }
  }
  if (j->finishing && !j->result_enq) {
    rc = trainer_finish(&j->tr);
    cudaError_t e = cudaSuccess;
    if (!rc) {
      e = cudaEventRecord(j->ev_out, j->st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(j->pin_out, j->tr.out, sizeof(float) * j->tr.N, cudaMemcpyDeviceToHost,
                          j->st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&j->hst[0], j->tr.state, sizeof(DevState),
                                                cudaMemcpyDeviceToHost, j->st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(j->pin_hist, j->tr.hist, sizeof(double) * kHistCap,
                                                cudaMemcpyDeviceToHost, j->st);
      if (e == cudaSuccess) e = cudaEventRecord(j->ev_done, j->st);
      if (e != cudaSuccess) rc = set_cuda_error(e, "result enqueue");
    }
    if (rc) {
      finish_job(c, j, N2F_FAILED, rc);
      return true;
    }
    j->result_enq = true;
    did = true;
  }
  if (j->result_enq) {
    const cudaError_t q = cudaEventQuery(j->ev_done);
    if (q == cudaErrorNotReady) return did;
    if (q != cudaSuccess) {
      set_cuda_error(q, "result");
      finish_job(c, j, N2F_FAILED, N2F_EDEVICE);
      return true;
    }
    {
      std::lock_guard<std::mutex> g(c->mu);
      j->last = j->hst[0];
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, j->ev_start, j->ev_done);
    j->device_ms = ms;
    cudaEventElapsedTime(&ms, j->ev_in, j->ev_out);
    j->compute_ms = ms;
    if (j->tr.kt) {
      // validations that ran: one per epoch under the stop rule, one in fixed-step mode
      const uint64_t vals = j->tr.fixed_mode ? j->tr.vals_enqueued : (uint64_t)j->last.epoch;
      j->kt.harvest((uint64_t)j->last.t, vals);
      std::lock_guard<std::mutex> g(c->mu);
      c->prof.launches += j->kt.launches;
      c->prof.ms += j->kt.ms;
      c->prof.flops += j->kt.flops;
      c->prof.bytes += j->kt.bytes;
    }
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, c->ev_ref, j->ev_start);
    cudaEventElapsedTime(&b, c->ev_ref, j->ev_done);
    j->t0_ms = a;
    j->t1_ms = b;
    const bool bad = j->last.stopped == 3 || j->last.kerr;
    if (j->cancel)
      finish_job(c, j, N2F_CANCELED, N2F_ECANCELED);
    else
      finish_job(c, j, bad ? N2F_FAILED : N2F_DONE,
                 j->last.kerr ? N2F_ETIMEDOUT : (bad ? N2F_ENONFINITE : N2F_OK));
    return true;
  }
  return did;
}

static void worker_main(n2f_ctx* c) {
  cudaSetDevice(c->cfg.device);
  for (;;) {
    std::vector<Job*> to_admit;
    {
      std::unique_lock<std::mutex> lk(c->mu);
      if (c->active.empty() && c->queue.empty())
        c->cv_work.wait(lk, [&] { return c->stop || !c->queue.empty(); });
      if (c->stop) break;
      while (!c->queue.empty() && c->active.size() + to_admit.size() < c->cfg.max_slots) {
        Job* j = c->queue.front();
        if (j->cancel) {
          c->queue.pop_front();
          j->state.store(N2F_CANCELED);
          j->error = N2F_ECANCELED;
          c->cv_done.notify_all();
          continue;
        }
        if (c->bytes_resident + j->bytes > c->cfg.hbm_budget_bytes) break;  // FIFO admission
        c->queue.pop_front();
        c->bytes_resident += j->bytes;
        to_admit.push_back(j);
      }
    }
    // lockstep groups of jobs admitted together with the same key
    std::vector<Group*> groups;
    if (c->cfg.group_size > 1) {
      std::vector<bool> used(to_admit.size(), false);
      for (size_t a = 0; a < to_admit.size(); ++a) {
        if (used[a] || !same_group_key(to_admit[a], to_admit[a])) continue;
        std::vector<Job*> mem{to_admit[a]};
        for (size_t b = a + 1; b < to_admit.size() && mem.size() < c->cfg.group_size; ++b)
          if (!used[b] && same_group_key(to_admit[a], to_admit[b])) {
            mem.push_back(to_admit[b]);
            used[b] = true;
          }
        if (mem.size() < 2) continue;
        used[a] = true;
        Group* g = new Group();
        g->m = mem;
        g->remaining = (int)mem.size() + 1;  // + the set-up reference
        g->ring = (int)std::min<uint32_t>(8, std::max<uint32_t>(2, c->cfg.lookahead + 1));
        for (Job* j : mem) j->grp = g;
        groups.push_back(g);
      }
    }
    for (Group* g : groups) {
      cudaError_t e = cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking);
      for (int k = 0; k < g->ring && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&g->ev_ep[k], cudaEventDisableTiming);
      if (e != cudaSuccess) {  // run the members alone instead
        for (Job* j : g->m) j->grp = nullptr;
        g->remaining = 1;
        group_unref(g);
      }
    }
    groups.erase(std::remove_if(groups.begin(), groups.end(),
                                [](Group* g) { return g->m.empty() || g->m[0]->grp != g; }),
                 groups.end());
    for (Job* j : to_admit) {
      {
        std::lock_guard<std::mutex> g(c->mu);
        c->active.push_back(j);
      }
      j->state.store(N2F_RUNNING);
      int rc = admit(c, j);
      if (rc) finish_job(c, j, N2F_FAILED, rc);
    }
    for (Group* g : groups) {
      // members that failed at admission left the group; the rest get the grouped tables
      std::vector<Job*> ok;
      for (Job* j : g->m)
        if (j->grp == g) ok.push_back(j);
      g->m = ok;
      if (!ok.empty()) {
        for (Job* j : ok) g->tg.ts.push_back(&j->tr);
        const int rc = group_init(&g->tg, c->al, g->st);
        if (rc) g->fail_rc = rc;
        else
          for (Job* j : ok) j->st = j->tr.st;  // the member's own stream (owned by the group)
      }
      group_unref(g);  // the set-up reference
    }
    std::vector<Job*> act;
    {
      std::lock_guard<std::mutex> g(c->mu);
      act = c->active;
    }
    bool any = false;
    for (Job* j : act) any |= progress(c, j);
    if (!any && !act.empty()) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

extern "C" int n2f_create(n2f_ctx** out, const n2f_config* cfg) {
  if (!out) return N2F_EINVAL;
  n2f_config def;
  n2f_config_default(&def);
  if (!cfg) cfg = &def;
  if (cfg->struct_size != sizeof(n2f_config)) return N2F_EINVAL;
  int ndev = 0;
  CKR(cudaGetDeviceCount(&ndev));
  if (cfg->device < 0 || cfg->device >= ndev) return N2F_EINVAL;
  CKR(cudaSetDevice(cfg->device));
  n2f_ctx* c = new n2f_ctx();
  c->cfg = *cfg;
  if (c->cfg.use_graphs < 0) c->cfg.use_graphs = 1;
  if (!c->cfg.hbm_budget_bytes) c->cfg.hbm_budget_bytes = 150ull << 30;
  if (!c->cfg.max_slots) c->cfg.max_slots = 64;
  if (!c->cfg.lookahead) c->cfg.lookahead = 2;
  c->al.alloc = cfg->alloc;
  c->al.free = cfg->free;
  c->al.user = cfg->alloc_user;
  cudaError_t e = cudaEventCreate(&c->ev_ref);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_ref, 0);
  if (e == cudaSuccess) e = cudaEventSynchronize(c->ev_ref);
  if (e != cudaSuccess) {
    delete c;
    return set_cuda_error(e, "n2f_create");
  }
  c->worker = std::thread(worker_main, c);
  *out = c;
  return N2F_OK;
}

extern "C" void n2f_destroy(n2f_ctx* c) {
  if (!c) return;
  {
    std::lock_guard<std::mutex> g(c->mu);
    c->stop = true;
  }
  c->cv_work.notify_all();
  if (c->worker.joinable()) c->worker.join();
  for (Job* j : c->active) {
    release_device(c, j);
    j->state.store(N2F_CANCELED);
  }
  for (auto& kv : c->jobs) {
    free_job_host(kv.second);
    delete kv.second;
  }
  if (c->ev_ref) cudaEventDestroy(c->ev_ref);
  delete c;
}

static int submit_common(n2f_ctx* c, int kind, const void* image, int H, int W,
                         const n2f_params* p, n2f_job* out) {
  if (!c || !image || !out) return N2F_EINVAL;
  n2f_params def;
  n2f_params_default(&def);
  if (!p) p = &def;
  int rc = check_params(p);
  if (rc) return rc;
  if ((rc = check_image(H, W))) return rc;
  if (kind == 2 && planes(p) != 1) return N2F_EINVAL;  // 16-bit input: one plane, no clean plane
  const size_t n = (size_t)H * W * planes(p);
  if (kind == 0) {
    const float* f = (const float*)image;
    for (size_t i = 0; i < n; ++i)
      if (!isfinite(f[i])) return N2F_EINVAL;
  }
  Job* j = new Job();
  j->H = H;
  j->W = W;
  j->prm = *p;
  j->src_kind = kind;
  if ((rc = trainer_configure(&j->tr, H, W, p, 0))) {
    delete j;
    return rc;
  }
  j->bytes = trainer_bytes(H, W, p, 0);
  if (j->bytes > c->cfg.hbm_budget_bytes) {
    delete j;
    return N2F_ETOOBIG;
  }
  cudaError_t e = cudaSuccess;
  if (kind == 0) {
    e = cudaMallocHost((void**)&j->pin_in, n * sizeof(float));
    if (e == cudaSuccess) memcpy(j->pin_in, image, n * sizeof(float));
  } else if (kind == 2) {
    e = cudaMallocHost((void**)&j->pin_u16, n * sizeof(uint16_t));
    if (e == cudaSuccess) memcpy(j->pin_u16, image, n * sizeof(uint16_t));
  } else {
    j->dev_in = (const float*)image;
  }
  if (e != cudaSuccess) {
    free_job_host(j);
    delete j;
    return set_cuda_error(e, "pinned staging");
  }
  j->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> g(c->mu);
    j->id = c->next_id++;
    c->jobs[j->id] = j;
    c->queue.push_back(j);
  }
  c->cv_work.notify_all();
  *out = j->id;
  return N2F_OK;
}

extern "C" int n2f_submit(n2f_ctx* c, const float* image, int H, int W, const n2f_params* p,
                          n2f_job* out) {
  return submit_common(c, 0, image, H, W, p, out);
}
extern "C" int n2f_submit_device(n2f_ctx* c, const float* dimage, int H, int W,
                                 const n2f_params* p, n2f_job* out) {
  return submit_common(c, 1, dimage, H, W, p, out);
}
extern "C" int n2f_submit_u16(n2f_ctx* c, const uint16_t* image, int H, int W,
                              const n2f_params* p, n2f_job* out) {
  return submit_common(c, 2, image, H, W, p, out);
}

extern "C" int n2f_job_bytes(int H, int W, const n2f_params* p, uint64_t* bytes) {
  if (!bytes) return N2F_EINVAL;
  n2f_params def;
  n2f_params_default(&def);
  if (!p) p = &def;
  int rc = check_params(p);
  if (rc) return rc;
  if ((rc = check_image(H, W))) return rc;
  Trainer t;
  if ((rc = trainer_configure(&t, H, W, p, 0))) return rc;
  *bytes = trainer_bytes(H, W, p, 0);
  return N2F_OK;
}

static Job* find(n2f_ctx* c, n2f_job id) {
  auto it = c->jobs.find(id);
  return it == c->jobs.end() ? nullptr : it->second;
}

extern "C" int n2f_poll(n2f_ctx* c, n2f_job id, n2f_status* st) {
  if (!c || !st || st->struct_size != sizeof(n2f_status)) return N2F_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  Job* j = find(c, id);
  if (!j) return N2F_ENOENT;
  const uint32_t ss = st->struct_size;
  memset(st, 0, sizeof(*st));
  st->struct_size = ss;
  st->state = j->state.load();
  st->error = j->error;
  fill_status(&j->tr, j->last, st);
  st->H = (uint32_t)j->H;
  st->W = (uint32_t)j->W;
  st->device_ms = j->device_ms;
  st->compute_ms = j->compute_ms;
  st->t_start_ms = j->t0_ms;
  st->t_done_ms = j->t1_ms;
  if (st->state >= N2F_DONE)
    st->latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
  return N2F_OK;
}

extern "C" int n2f_wait(n2f_ctx* c, n2f_job id, int timeout_ms) {
  if (!c) return N2F_EINVAL;
  std::unique_lock<std::mutex> lk(c->mu);
  Job* j = find(c, id);
  if (!j) return N2F_ENOENT;
  auto done = [&] { return j->state.load() >= N2F_DONE; };
  if (timeout_ms < 0)
    c->cv_done.wait(lk, done);
  else if (!c->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
    return N2F_ETIMEDOUT;
  return N2F_OK;
}

static int take_result(n2f_ctx* c, n2f_job id, float* out, size_t n, bool device) {
  if (!c || !out) return N2F_EINVAL;
  Job* j;
  {
    std::lock_guard<std::mutex> g(c->mu);
    j = find(c, id);
    if (!j) return N2F_ENOENT;
    const int s = j->state.load();
    if (s < N2F_DONE) return N2F_EAGAIN;
    if (s != N2F_DONE) {
      const int err = j->error ? j->error : N2F_EDEVICE;
      c->jobs.erase(id);
      free_job_host(j);
      delete j;
      return err;
    }
    if (n < (size_t)j->H * j->W) return N2F_EINVAL;
  }
  const size_t bytes = sizeof(float) * (size_t)j->H * j->W;
  if (device) {
    CKR(cudaMemcpy(out, j->pin_out, bytes, cudaMemcpyHostToDevice));
  } else {
    memcpy(out, j->pin_out, bytes);
  }
  std::lock_guard<std::mutex> g(c->mu);
  c->jobs.erase(id);
  free_job_host(j);
  delete j;
  return N2F_OK;
}

extern "C" int n2f_result(n2f_ctx* c, n2f_job id, float* out, size_t out_elems) {
  return take_result(c, id, out, out_elems, false);
}
extern "C" int n2f_result_device(n2f_ctx* c, n2f_job id, float* dout, size_t out_elems) {
  return take_result(c, id, dout, out_elems, true);
}

extern "C" int n2f_history(n2f_ctx* c, n2f_job id, double* out, size_t cap, size_t* n_out,
                           uint32_t* first_epoch) {
  if (!c || !n_out) return N2F_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  Job* j = find(c, id);
  if (!j) return N2F_ENOENT;
  const int s = j->state.load();
  if (s < N2F_DONE) return N2F_EAGAIN;
  if (s != N2F_DONE || !j->pin_hist) return N2F_EINVAL;
  const int end = j->prm.fixed_steps >= 0 ? 0 : j->last.epoch;
  const size_t n = (size_t)std::min(end, kHistCap);
  *n_out = n;
  if (first_epoch) *first_epoch = (uint32_t)(end - (int)n + 1);
  if (!out) return N2F_OK;
  if (cap < n) return N2F_EINVAL;
  hist_unroll(j->pin_hist, end, out);
  return N2F_OK;
}

extern "C" int n2f_cancel(n2f_ctx* c, n2f_job id) {
  if (!c) return N2F_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  Job* j = find(c, id);
  if (!j) return N2F_ENOENT;
  if (j->state.load() >= N2F_DONE) return N2F_OK;
  j->cancel = true;
  c->cv_work.notify_all();
  return N2F_OK;
}

extern "C" int n2f_stats(n2f_ctx* c, n2f_ctx_stats* st) {
  if (!c || !st || st->struct_size != sizeof(n2f_ctx_stats)) return N2F_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  st->kernel_launches = c->launches;
  st->bytes_resident = c->bytes_resident;
  st->jobs_queued = (uint32_t)c->queue.size();
  st->jobs_running = (uint32_t)c->active.size();
  st->jobs_done = c->n_done;
  st->prof_launches = c->prof.launches;
  st->prof_ms = c->prof.ms;
  st->prof_flops = c->prof.flops;
  st->prof_bytes = c->prof.bytes;
  return N2F_OK;
}
