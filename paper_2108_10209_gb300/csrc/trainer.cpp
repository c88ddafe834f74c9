// Step executor: one job's device state and the kernel sequence of a training step, a
// validation pass and an epoch (Methods, "Noise2Fast Implementation Details").
#include "trainer.h"

#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

namespace n2f {

thread_local std::string tl_error;

int set_cuda_error(cudaError_t e, const char* where) {
  tl_error = std::string(where) + ": " + cudaGetErrorString(e);
  return N2F_EDEVICE;
}

void NetShape::init(int which, int channels) {
  for (int l = 0; l < kLayers; ++l) {
    static const int plit[kLayers] = {32, 32, 64, 64, 128, 128, 256, 256};
    widths[l] = which == N2F_WIDTHS_W64 ? 64 : plit[l];
  }
  c0 = channels > 0 ? channels : 1;
  size_t n = 0;
  int cin = c0;
  for (int l = 0; l < kLayers; ++l) {
    w_off[l] = n;
    n += (size_t)widths[l] * cin * 9;
    b_off[l] = n;
    n += widths[l];
    cin = widths[l];
  }
  w_off[kLayers] = n;
  b_off[kLayers] = n + cin;
  count = n + cin + 1;
}

void* dev_alloc(const Allocator& a, size_t bytes) {
  if (a.alloc) return a.alloc(bytes, a.user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(const Allocator& a, void* p, size_t bytes) {
  if (!p) return;
  if (a.free)
    a.free(p, bytes, a.user);
  else
    cudaFree(p);
}

cudaEvent_t KTimer::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void KTimer::harvest(uint64_t steps_done, uint64_t vals_done) {
  for (const Pair& p : pending) {
    const bool counted = p.val ? p.seq < vals_done : p.seq < steps_done;
    float t = 0.f;
    if (counted && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      ms += t;
      flops += p.flops;
      bytes += p.bytes;
      launches += 1;
    }
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  cudaGetLastError();
  pending.clear();
}

void KTimer::destroy() {
  for (const Pair& p : pending) {
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
  pool.clear();
}

namespace {

// Brackets one launch of kernel class `kind` with events when the trainer times that class.
// While an epoch is being captured the events become event-record nodes of the graph.
struct Timed {
  Trainer* t = nullptr;
  KTimer* kt = nullptr;
  cudaStream_t st;
  KTimer::Pair p;
  Timed(Trainer* tr, int kind, double flops, double bytes, int val) : st(tr->st) {
    if (!tr->kt || !tr->timing_on) return;
    const bool conv = tr->kt->kind == N2F_K_CONV && (kind == N2F_K_CONV_FWD || kind == N2F_K_CONV_DGRAD);
    if (tr->kt->kind != kind && !conv) return;
    t = tr;
    kt = tr->kt;
    p.a = kt->get();
    p.b = nullptr;
    p.flops = flops;
    p.bytes = bytes;
    p.val = val;
    p.seq = val ? t->vals_enqueued : t->steps_enqueued;
    if (t->capturing)
      cudaEventRecordWithFlags(p.a, st, cudaEventRecordExternal);
    else
      cudaEventRecord(p.a, st);
  }
  ~Timed() {
    if (!kt) return;
    p.b = kt->get();
    if (t->capturing) {
      cudaEventRecordWithFlags(p.b, st, cudaEventRecordExternal);
      Trainer::TimedNode n;
      n.a = p.a;
      n.b = p.b;
      n.flops = p.flops;
      n.bytes = p.bytes;
      n.val = p.val;
      n.k = (int)(p.seq - (p.val ? t->cap_vals0 : t->cap_steps0));
      t->tnodes.push_back(n);
    } else {
      cudaEventRecord(p.b, st);
      kt->pending.push_back(p);
    }
  }
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Carver {
  size_t off = 0;
  char* base = nullptr;
  template <typename T>
  T* take(size_t elems) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += elems * sizeof(T);
    return p;
  }
};

}  // namespace

static int layer_engine(const Trainer* t, int l) {
  if (l == 0) return N2F_ENGINE_SIMT;
  const int e = t->prm.engine;
  const bool tc = tc_supported(t->net.cin(l), t->net.widths[l]);
  if (e == N2F_ENGINE_SIMT) return N2F_ENGINE_SIMT;
  if (e == N2F_ENGINE_TC) return tc ? N2F_ENGINE_TC : -1;
  return tc ? N2F_ENGINE_TC : N2F_ENGINE_SIMT;
}

// The job validates beside the next epoch's training (stopping-rule jobs only).
static bool overlapped(const Trainer* t) { return t->prm.overlap && !t->fixed_mode; }

// Carves every buffer out of one slab; with base == nullptr it only measures.
static size_t layout(Trainer* t, char* base) {
  Carver c;
  c.base = base;
  const NetShape& net = t->net;
  const size_t es = t->bf16 ? 2 : 4;
  const size_t np = (size_t)t->nplanes;
  t->x = c.take<float>(np * t->N);
  for (int k = 0; k < 4; ++k) t->sub[k] = c.take<float>(np * t->ph[k] * t->pw[k]);
  for (int k = 0; k < 4; ++k) t->tx[k] = c.take<float>(t->prm.exact ? (size_t)t->ph[k] * t->pw[k] : 0);
  // theta and every weight copy a forward pass reads form one contiguous range: the snapshot
  // that an overlapped validation reads
  memset(&t->pa, 0, sizeof(t->pa));
  t->snap_off = align_up(c.off, 256);
  t->theta = c.take<float>(net.count);
  bool any_tc = false;
  for (int l = 0; l < kLayers; ++l) {
    const size_t nw = (size_t)net.widths[l] * net.cin(l) * 9;
    // the CUDA-core copies only for the layers that run on the CUDA cores (the first layer
    // always): the packing kernels skip a copy that is not there
    const bool tc = l > 0 && t->engine[l] == N2F_ENGINE_TC;
    t->pa.fwd[l] = tc ? nullptr : c.take<float>(nw);
    if (tc) {
      any_tc = true;
      // 16-bit elements: bf16, or the float32 form's fp16 hi and lo parts
      t->pa.tcf[l] = c.take<uint16_t>(nw);
      if (!t->bf16) t->pa.tcf_lo[l] = c.take<uint16_t>(nw);
    }
  }
  t->snap_bytes = c.off - t->snap_off;
  for (int l = 1; l < kLayers; ++l) {
    const size_t nw = (size_t)net.widths[l] * net.cin(l) * 9;
    const bool tc = t->engine[l] == N2F_ENGINE_TC;
    t->pa.dgr[l] = tc ? nullptr : c.take<float>(nw);
    if (tc) {
      t->pa.tcd[l] = c.take<uint16_t>(nw);
      if (!t->bf16) t->pa.tcd_lo[l] = c.take<uint16_t>(nw);
    }
  }
  t->grad = c.take<float>(net.count);
  t->m = c.take<float>(net.count);
  t->v = c.take<float>(net.count);
  t->sw = !t->bf16 && any_tc ? c.take<ScaleWords>(1) : nullptr;
  t->pa.sw = t->sw;
  // activations / deltas (training) alias the validation ping-pong buffers, unless the two run
  // at the same time (overlap)
  const bool ovl = overlapped(t);
  const size_t Cmax = net.cmax(), Csum = net.csum();
  const size_t train_elems = Csum * t->maxP + (t->keep_deltas ? Csum : 2 * Cmax) * t->maxP;
  const size_t val_elems = 2 * Cmax * t->N;
  char* region = c.take<char>((ovl ? train_elems : std::max(train_elems, val_elems)) * es);
  char* vregion = ovl ? c.take<char>(val_elems * es) : region;
  char* vsnap = c.take<char>(ovl ? t->snap_bytes : 0);
  DevState* ssave = c.take<DevState>(ovl ? 1 : 0);
  if (base && ovl) {
    t->vsnap = vsnap;
    t->state_save = ssave;
    // the snapshot's copies sit at the same offsets from vsnap as the live ones from snap_off
    auto rebase = [&](auto* p) -> decltype(p) {
      return p ? reinterpret_cast<decltype(p)>(vsnap + (reinterpret_cast<char*>(p) -
                                                        (base + t->snap_off)))
               : nullptr;
    };
    t->vpa = t->pa;
    t->vpa.theta = rebase(t->theta);
    for (int l = 0; l < kLayers; ++l) {
      t->vpa.fwd[l] = rebase(t->pa.fwd[l]);
      t->vpa.tcf[l] = rebase(t->pa.tcf[l]);
      t->vpa.tcf_lo[l] = rebase(t->pa.tcf_lo[l]);
      t->vpa.dgr[l] = nullptr;
      t->vpa.tcd[l] = t->vpa.tcd_lo[l] = nullptr;
    }
  }
  if (base) {
    size_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
      t->act[l] = region + o * es;
      o += (size_t)net.widths[l] * t->maxP;
    }
    if (t->keep_deltas) {
      for (int l = 0; l < kLayers; ++l) {
        t->dkeep[l] = region + o * es;
        o += (size_t)net.widths[l] * t->maxP;
      }
      t->dl[0] = t->dl[1] = nullptr;
    } else {
      t->dl[0] = region + o * es;
      t->dl[1] = region + (o + Cmax * t->maxP) * es;
    }
    t->vb[0] = vregion;
    t->vb[1] = vregion + Cmax * t->N * es;
  }
  t->dz = c.take<float>(t->maxP);
  t->V = c.take<float>(t->N);
  t->S = c.take<float>(t->N);
  t->Vbest = c.take<float>(t->N);
  t->out = c.take<float>(t->N);
  t->nblk_max = (int)((std::max(t->maxP, t->N) + 255) / 256);
  t->lpart = c.take<double>(t->nblk_max);
  t->mpart = c.take<double>(t->nblk_max);
  t->hpart = c.take<float>((size_t)t->nblk_max * (Cmax + 1));
  t->wpart_cap = (size_t)16 << 20;
  t->wpart = c.take<float>(t->wpart_cap);
  t->state = c.take<DevState>(1);
  t->hist = c.take<double>(kHistCap);
  t->in_u16 = c.take<uint16_t>(t->want_u16 ? t->N : 0);
  return align_up(c.off, 256);
}

size_t trainer_bytes(int H, int W, const n2f_params* p, int keep_deltas) {
  Trainer t;
  if (trainer_configure(&t, H, W, p, keep_deltas) != N2F_OK) return 0;
  return layout(&t, nullptr);
}

int trainer_configure(Trainer* t, int H, int W, const n2f_params* p, int keep_deltas) {
  t->prm = *p;
  t->H = H;
  t->W = W;
  t->N = (size_t)H * W;
  const bool quad = p->downsample == N2F_DOWN_QUAD;
  for (int k = 0; k < 4; ++k) {
    t->ph[k] = quad ? H / 2 : (k < 2 ? H : H / 2);
    t->pw[k] = quad ? W / 2 : (k < 2 ? W / 2 : W);
    // checkerboard: the Methods table's pairs k -> k^1; Quad: once round the 2x2 block
    t->tgt_of[k] = quad ? (k + 1) % 4 : k ^ 1;
  }
  t->maxP = 0;
  for (int k = 0; k < 4; ++k) t->maxP = std::max(t->maxP, (size_t)t->ph[k] * t->pw[k]);
  t->net.init(p->widths, p->channels);
  t->nplanes = t->net.c0 + (p->exact ? 1 : 0);
  t->bf16 = p->precision == N2F_BF16;
  t->keep_deltas = keep_deltas;
  t->fixed_mode = p->fixed_steps >= 0;
  for (int l = 0; l < kLayers; ++l) {
    t->engine[l] = layer_engine(t, l);
    if (t->engine[l] < 0) return N2F_ENOTSUP;
    t->wg_engine[l] = t->engine[l] == N2F_ENGINE_TC &&
                              tc_wgrad_supported(t->net.cin(l), t->net.widths[l], t->bf16)
                          ? N2F_ENGINE_TC
                          : N2F_ENGINE_SIMT;
  }
  return N2F_OK;
}

int trainer_init(Trainer* t, const Allocator& al, cudaStream_t st, int want_u16) {
  for (int l = 0; l < kLayers; ++l)
    if (t->engine[l] == N2F_ENGINE_TC) {
      const cudaError_t e = tc_prepare();
      if (e != cudaSuccess) return set_cuda_error(e, "tensor-core kernel set-up");
      break;
    }
  t->al = al;
  t->st = st;
  t->want_u16 = want_u16;
  t->slab_bytes = layout(t, nullptr);
  t->slab = (char*)dev_alloc(al, t->slab_bytes);
  if (!t->slab) {
    tl_error = "device allocation of the job state failed";
    return N2F_ENOMEM;
  }
  layout(t, t->slab);
  PackArgs& pa = t->pa;
  pa.theta = t->theta;
  for (int l = 0; l < kLayers; ++l) pa.widths[l] = t->net.widths[l];
  pa.c0 = t->net.c0;
  for (int l = 0; l <= kLayers; ++l) {
    pa.w_off[l] = t->net.w_off[l];
    pa.b_off[l] = t->net.b_off[l];
  }
  pa.count = t->net.count;
  pa.tc_bf16 = t->bf16;
  if (overlapped(t)) {
    PackArgs v = pa;  // the shape fields; the pointers into the snapshot come from layout
    v.theta = t->vpa.theta;
    for (int l = 0; l < kLayers; ++l) {
      v.fwd[l] = t->vpa.fwd[l];
      v.tcf[l] = t->vpa.tcf[l];
      v.tcf_lo[l] = t->vpa.tcf_lo[l];
      v.dgr[l] = nullptr;
      v.tcd[l] = v.tcd_lo[l] = nullptr;
    }
    t->vpa = v;
    cudaError_t e = cudaStreamCreateWithFlags(&t->vst, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->ev_vfork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->ev_vjoin, cudaEventDisableTiming);
    if (e != cudaSuccess) return set_cuda_error(e, "validation stream");
  }
  return N2F_OK;
}

void trainer_release(Trainer* t) {
  if (t->epoch_exec) cudaGraphExecDestroy(t->epoch_exec);
  t->epoch_exec = nullptr;
  if (t->epoch_graph) cudaGraphDestroy(t->epoch_graph);
  t->epoch_graph = nullptr;
  if (t->epoch_exec_plain) cudaGraphExecDestroy(t->epoch_exec_plain);
  t->epoch_exec_plain = nullptr;
  if (t->epoch_graph_plain) cudaGraphDestroy(t->epoch_graph_plain);
  t->epoch_graph_plain = nullptr;
  for (Trainer::TimedNode& n : t->tnodes) {
    if (t->kt) {
      t->kt->pool.push_back(n.a);
      t->kt->pool.push_back(n.b);
    }
  }
  t->tnodes.clear();
  if (t->vst) cudaStreamSynchronize(t->vst), cudaStreamDestroy(t->vst);
  if (t->ev_vfork) cudaEventDestroy(t->ev_vfork);
  if (t->ev_vjoin) cudaEventDestroy(t->ev_vjoin);
  t->vst = nullptr;
  t->ev_vfork = t->ev_vjoin = nullptr;
  if (t->slab) dev_free(t->al, t->slab, t->slab_bytes);
  t->slab = nullptr;
}

#define CK(expr)                                            \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return set_cuda_error(_e, #expr); \
  } while (0)

// Image already in t->x (or t->in_u16): gather, initial weights, packed copies, state.
int trainer_start(Trainer* t, int from_u16) {
  LaunchScope ls(&t->launches);
  cudaStream_t st = t->st;
  if (from_u16) CK(launch_u16_to_f32(t->in_u16, t->x, t->N, st));
  // every plane is downsampled the same way
  for (int c = 0; c < t->nplanes; ++c) {
    size_t P[4];
    for (int k = 0; k < 4; ++k) P[k] = (size_t)c * t->ph[k] * t->pw[k];
    const float* xc = t->x + (size_t)c * t->N;
    if (t->prm.downsample == N2F_DOWN_QUAD)
      CK(launch_gather_quad(xc, t->H, t->W, t->sub[0] + P[0], t->sub[1] + P[1], t->sub[2] + P[2],
                            t->sub[3] + P[3], st));
    else
      CK(launch_gather(xc, t->H, t->W, t->sub[0] + P[0], t->sub[1] + P[1], t->sub[2] + P[2],
                       t->sub[3] + P[3], st));
  }
  if (t->prm.exact) {
    // targets x_tgt - (s_tgt - s_in): the clean plane is the last plane of every sub-image
    for (int k = 0; k < 4; ++k) {
      const int g = t->tgt_of[k];
      const size_t Pg = (size_t)t->ph[g] * t->pw[g], Pk = (size_t)t->ph[k] * t->pw[k];
      CK(launch_exact_target(t->sub[g] + (size_t)t->prm.target_channel * Pg,
                             t->sub[g] + (size_t)t->net.c0 * Pg, t->sub[k] + (size_t)t->net.c0 * Pk,
                             Pk, t->tx[k], st));
    }
  }
  CK(launch_init_params(t->theta, t->net, t->prm.seed, st));
  CK(cudaMemsetAsync(t->m, 0, t->net.count * sizeof(float), st));
  CK(cudaMemsetAsync(t->v, 0, t->net.count * sizeof(float), st));
  CK(cudaMemsetAsync(t->grad, 0, t->net.count * sizeof(float), st));
  CK(cudaMemsetAsync(t->S, 0, t->N * sizeof(float), st));
  CK(cudaMemsetAsync(t->Vbest, 0, t->N * sizeof(float), st));
  CK(cudaMemsetAsync(t->V, 0, t->N * sizeof(float), st));
  // all-ones bytes: the history ring starts as NaN (no score recorded)
  CK(cudaMemsetAsync(t->hist, 0xff, kHistCap * sizeof(double), st));
  DevState s;
  memset(&s, 0, sizeof(s));
  s.best = INFINITY;
  s.patience = (int)t->prm.patience;
  s.max_epochs = (int)t->prm.max_epochs;
  s.incl_best = t->prm.incl_best;
  s.b1t = 1.0;
  s.b2t = 1.0;
  s.bc1 = s.bc2 = 1.f;
  s.decision = -1;
  t->hstate_init = s;
  CK(cudaMemcpyAsync(t->state, &t->hstate_init, sizeof(DevState), cudaMemcpyHostToDevice, st));
  if (t->sw) CK(cudaMemsetAsync(t->sw, 0, sizeof(ScaleWords), st));
  CK(launch_adam(t->pa, t->grad, t->m, t->v, AdamConsts{}, t->state, 0, st));
  return N2F_OK;
}

int trainer_repack(Trainer* t) {
  LaunchScope ls(&t->launches);
  // the largest weights are collected afresh for the new parameters
  if (t->sw) CK(cudaMemsetAsync(t->sw->wnew, 0, sizeof(t->sw->wnew), t->st));
  CK(launch_adam(t->pa, t->grad, t->m, t->v, AdamConsts{}, t->state, 0, t->st));
  return N2F_OK;
}

// Magnitude words of the float32 form (all null in the bf16 form). One forward pass uses one
// set: the training step's act[] with w[], or the validation's vact[] with w[] (in line) or
// vw[] (reading the weight snapshot). The forward of layer l reads act[l - 1] and the weights,
// raises act[l]; the dgrad of layer l reads delta[l] and the weights, raises delta[l - 1].
struct FwdWords {
  unsigned* act = nullptr;
  const unsigned* w = nullptr;
};
static FwdWords train_words(const Trainer* t) {
  FwdWords f;
  if (t->sw) {
    f.act = t->sw->act;
    f.w = t->sw->w;
  }
  return f;
}
static FwdWords val_words(const Trainer* t, bool snap) {
  FwdWords f;
  if (t->sw) {
    f.act = t->sw->vact;
    f.w = snap ? t->sw->vw : t->sw->w;
  }
  return f;
}
static ConvScales fwd_scales(FwdWords f, int l) {
  ConvScales s;
  if (f.act) {
    s.in = &f.act[l - 1];
    s.w = &f.w[l];
    s.out = &f.act[l];
  }
  return s;
}
static ConvScales dgrad_scales(const Trainer* t, int l) {
  ConvScales s;
  if (t->sw) {
    s.in = &t->sw->delta[l];
    s.w = &t->sw->w[l];
    s.out = &t->sw->delta[l - 1];
  }
  return s;
}

// Forward of layer l with the weights of `wp` (the live ones, or the validation's snapshot).
static int conv_layer(Trainer* t, int l, const void* in, void* out, int H, int W,
                      const int* skip, int val, const PackArgs& wp, FwdWords fw) {
  const int cin = t->net.cin(l), cout = t->net.widths[l];
  const float* b = wp.theta + t->net.b_off[l];
  const double P = (double)H * W, es = t->bf16 ? 2.0 : 4.0;
  Timed tm(t, l == 0 ? N2F_K_FIRST : N2F_K_CONV_FWD, 2.0 * P * 9 * cin * cout,
           l == 0 ? P * 4.0 + P * cout * es : P * (cin + cout) * es, val);
  if (l == 0) {
    CK(launch_conv1_fwd((const float*)in, cin, H, W, wp.fwd[0], b, cout, t->bf16, out,
                        fw.act ? &fw.act[0] : nullptr, skip, t->st));
  } else if (t->engine[l] == N2F_ENGINE_TC) {
    CK(launch_conv_tc(0, t->bf16, in, cin, cout, H, W, wp.tcf[l], wp.tcf_lo[l], b, nullptr, out,
                      fwd_scales(fw, l), skip, &t->state->kerr, t->st));
  } else {
    CK(launch_conv_simt(0, t->bf16, in, cin, cout, H, W, wp.fwd[l], b, nullptr, out, skip,
                        t->st));
    if (fw.act) CK(launch_absmax(out, (size_t)cout * H * W, 0, &fw.act[l], skip, t->st));
  }
  return N2F_OK;
}

// ---- one training step, in pieces (the grouped executor replaces the tensor-core forward and
// dgrad launches by one launch over all its jobs and calls the rest per job) ----------------

static const int* step_skip(const Trainer* t) { return t->fixed_mode ? nullptr : &t->state->stopped; }

// delta (dL/d pre-activation) of layer m (0-based) in the training step
static void* delta_of(const Trainer* t, int m) {
  return t->keep_deltas ? t->dkeep[m] : t->dl[(kLayers - 1 - m) & 1];
}

static int step_forward(Trainer* t, int pair, int l) {
  const void* in = l == 0 ? (const void*)t->sub[pair] : t->act[l - 1];
  return conv_layer(t, l, in, t->act[l], t->ph[pair], t->pw[pair], step_skip(t), 0, t->pa,
                    train_words(t));
}

static int step_head(Trainer* t, int pair) {
  const int h = t->ph[pair], w = t->pw[pair];
  const int npx = h * w;
  const NetShape& net = t->net;
  const int* skip = step_skip(t);
  // Methods table: even <-> odd of the same kind (Quad: the next image round the block); the
  // target is the predicted channel (Exact: with the signal difference removed)
  const int g = t->tgt_of[pair];
  const float* tgt = t->prm.exact ? t->tx[pair]
                                  : t->sub[g] + (size_t)t->prm.target_channel * t->ph[g] * t->pw[g];
  t->last_pair = pair;
  const int C8 = net.widths[kLayers - 1];
  int nblk = 0;
  const double es = t->bf16 ? 2.0 : 4.0;
  {
    Timed tm(t, N2F_K_HEAD, 2.0 * npx * C8, (double)npx * C8 * 2 * es + npx * 8.0, 0);
    CK(launch_head_train(t->act[kLayers - 1], C8, npx, t->theta + net.w_off[kLayers],
                         t->theta + net.b_off[kLayers], tgt, t->prm.loss, t->bf16, t->dz,
                         delta_of(t, kLayers - 1), t->sw ? &t->sw->delta[kLayers - 1] : nullptr,
                         t->lpart, t->hpart, &nblk, skip, t->st));
  }
  CK(launch_step_finish(t->hpart, t->lpart, nblk, C8, npx, t->grad + net.w_off[kLayers],
                        t->grad + net.b_off[kLayers], t->state, t->prm.beta1, t->prm.beta2,
                        t->st));
  return N2F_OK;
}

static int step_wgrad(Trainer* t, int pair, int l) {
  const int h = t->ph[pair], w = t->pw[pair];
  const int npx = h * w;
  const NetShape& net = t->net;
  const int* skip = step_skip(t);
  const int cin = net.cin(l), cout = net.widths[l];
  float* gw = t->grad + net.w_off[l];
  float* gb = t->grad + net.b_off[l];
  const void* dcur = delta_of(t, l);
  if (l == 0) {
    CK(launch_conv1_wgrad(dcur, t->sub[pair], cin, h, w, cout, t->bf16, t->wpart, t->wpart_cap,
                          gw, gb, skip, t->st));
    return N2F_OK;
  }
  const double es = t->bf16 ? 2.0 : 4.0;
  Timed tm(t, N2F_K_CONV_WGRAD, 2.0 * npx * 9 * cin * cout, (double)npx * (cin + cout) * es, 0);
  if (t->wg_engine[l] == N2F_ENGINE_TC)
    CK(launch_wgrad_tc(t->bf16, dcur, t->act[l - 1], cin, cout, h, w,
                       t->sw ? &t->sw->delta[l] : nullptr, t->sw ? &t->sw->act[l - 1] : nullptr,
                       t->wpart, t->wpart_cap, gw, gb, skip, &t->state->kerr, t->st));
  else
    CK(launch_wgrad_simt(t->bf16, dcur, t->act[l - 1], cin, cout, h, w, t->wpart, t->wpart_cap,
                         gw, gb, skip, t->st));
  return N2F_OK;
}

static int step_dgrad(Trainer* t, int pair, int l) {
  const int h = t->ph[pair], w = t->pw[pair];
  const NetShape& net = t->net;
  const int cin = net.cin(l), cout = net.widths[l];
  const double es = t->bf16 ? 2.0 : 4.0;
  Timed tm(t, N2F_K_CONV_DGRAD, 2.0 * h * w * 9 * cin * cout, (double)h * w * (cin * 2 + cout) * es,
           0);
  if (t->engine[l] == N2F_ENGINE_TC)
    CK(launch_conv_tc(1, t->bf16, delta_of(t, l), cout, cin, h, w, t->pa.tcd[l], t->pa.tcd_lo[l],
                      nullptr, t->act[l - 1], delta_of(t, l - 1), dgrad_scales(t, l), step_skip(t),
                      &t->state->kerr, t->st));
  else {
    CK(launch_conv_simt(1, t->bf16, delta_of(t, l), cout, cin, h, w, t->pa.dgr[l], nullptr,
                        t->act[l - 1], delta_of(t, l - 1), step_skip(t), t->st));
    if (t->sw)
      CK(launch_absmax(delta_of(t, l - 1), (size_t)cin * h * w, 0, &t->sw->delta[l - 1],
                       step_skip(t), t->st));
  }
  return N2F_OK;
}

static int step_adam(Trainer* t) {
  Timed tm(t, N2F_K_ADAM, 0.0, (double)t->net.count * 4.0 * 9, 0);
  CK(launch_adam(t->pa, t->grad, t->m, t->v,
                 adam_consts(t->prm.lr, t->prm.beta1, t->prm.beta2, t->prm.eps), t->state, 1,
                 t->st));
  return N2F_OK;
}

int trainer_step(Trainer* t, int pair) {
  LaunchScope ls(&t->launches);
  int rc;
  for (int l = 0; l < kLayers; ++l)
    if ((rc = step_forward(t, pair, l))) return rc;
  if ((rc = step_head(t, pair))) return rc;
  for (int l = kLayers - 1; l >= 0; --l) {
    if ((rc = step_wgrad(t, pair, l))) return rc;
    if (l > 0 && (rc = step_dgrad(t, pair, l))) return rc;
  }
  if ((rc = step_adam(t))) return rc;
  t->steps_enqueued += 1;
  return N2F_OK;
}

// validation forward of layer l: x -> vb[0] -> vb[1] -> ...; snap: with the weight snapshot
static int val_forward(Trainer* t, int l, bool snap) {
  const void* in = l == 0 ? (const void*)t->x : t->vb[(l - 1) & 1];
  return conv_layer(t, l, in, t->vb[l & 1], t->H, t->W, step_skip(t), 1, snap ? t->vpa : t->pa,
                    val_words(t, snap));
}

// the validation's magnitude words start afresh
static int val_begin(Trainer* t) {
  if (t->sw) CK(cudaMemsetAsync(t->sw->vact, 0, sizeof(t->sw->vact), t->st));
  return N2F_OK;
}

static int val_finish(Trainer* t, bool snap) {
  const NetShape& net = t->net;
  const float* th = snap ? t->vpa.theta : t->theta;
  const int* skip = step_skip(t);
  int nblk = 0;
  {
    const double es = t->bf16 ? 2.0 : 4.0, C8 = net.widths[kLayers - 1];
    Timed tm(t, N2F_K_HEAD, 2.0 * t->N * C8, (double)t->N * (C8 * es + 8.0), 1);
    CK(launch_head_val(t->vb[(kLayers - 1) & 1], net.widths[kLayers - 1], (int)t->N,
                       th + net.w_off[kLayers], th + net.b_off[kLayers],
                       t->x + (size_t)t->prm.target_channel * t->N, t->bf16, t->V, t->mpart,
                       &nblk, skip, t->st));
  }
  CK(launch_val_decide(t->mpart, nblk, t->N, t->state, t->fixed_mode, t->hist, t->st));
  if (!t->fixed_mode) CK(launch_val_accum(t->V, t->S, t->Vbest, t->N, t->state, t->st));
  t->vals_enqueued += 1;
  return N2F_OK;
}

static int validate(Trainer* t, bool snap) {
  LaunchScope ls(&t->launches);
  int rc;
  if ((rc = val_begin(t))) return rc;
  for (int l = 0; l < kLayers; ++l)
    if ((rc = val_forward(t, l, snap))) return rc;
  return val_finish(t, snap);
}

int trainer_validate(Trainer* t) { return validate(t, false); }

// ---- lockstep group -----------------------------------------------------------------------

int group_init(TrainerGroup* g, const Allocator& al, cudaStream_t st) {
  g->al = al;
  g->st = st;
  const int n = (int)g->ts.size();
  if (n < 1) return N2F_EINVAL;
  const Trainer* t0 = g->ts[0];
  const size_t js = conv_job_size();
  // table layout: [layer][kind][mode] blocks of n entries; kinds 0/1 the pairs' two shapes,
  // kind 2 the validation; mode 1 (dgrad) only for the training kinds
  size_t off = 0;
  for (int l = 0; l < kLayers; ++l) {
    g->grouped[l] = l > 0 && t0->engine[l] == N2F_ENGINE_TC;
    for (int k = 0; k < 3; ++k)
      for (int m = 0; m < 2; ++m) {
        g->toff[l][k][m] = off;
        g->ntiles[l][k][m] = 0;
        if (g->grouped[l] && !(m == 1 && k == 2)) off += (size_t)n * js;
      }
  }
  g->tbl_bytes = off ? off : js;
  g->tbl = (char*)dev_alloc(al, g->tbl_bytes);
  if (!g->tbl) {
    tl_error = "device allocation of the group tables failed";
    return N2F_ENOMEM;
  }
  std::vector<char> host(g->tbl_bytes);
  std::vector<ConvGroupEntry> e(n);
  for (int l = 1; l < kLayers; ++l) {
    if (!g->grouped[l]) continue;
    const int cin = t0->net.cin(l), cout = t0->net.widths[l];
    for (int k = 0; k < 3; ++k)
      for (int m = 0; m < 2; ++m) {
        if (m == 1 && k == 2) continue;
        for (int i = 0; i < n; ++i) {
          Trainer* t = g->ts[i];
          const int pk = k == 0 ? 0 : 2;  // a pair of this kind
          ConvGroupEntry& q = e[i];
          q.H = k == 2 ? t->H : t->ph[pk];
          q.W = k == 2 ? t->W : t->pw[pk];
          q.skip = step_skip(t);
          if (m == 0) {
            q.in = k == 2 ? t->vb[(l - 1) & 1] : t->act[l - 1];
            q.out = k == 2 ? t->vb[l & 1] : t->act[l];
            q.w_hi = t->pa.tcf[l];
            q.w_lo = t->pa.tcf_lo[l];
            q.bias = t->theta + t->net.b_off[l];
            q.mask = nullptr;
            q.sc = fwd_scales(k == 2 ? val_words(t, false) : train_words(t), l);
          } else {
            q.in = delta_of(t, l);
            q.out = delta_of(t, l - 1);
            q.w_hi = t->pa.tcd[l];
            q.w_lo = t->pa.tcd_lo[l];
            q.bias = nullptr;
            q.mask = t->act[l - 1];
            q.sc = dgrad_scales(t, l);
          }
        }
        long nt = 0;
        const cudaError_t r = m == 0 ? conv_group_table(0, t0->bf16, cin, cout, e.data(), n,
                                                        host.data() + g->toff[l][k][m], &nt)
                                     : conv_group_table(1, t0->bf16, cout, cin, e.data(), n,
                                                        host.data() + g->toff[l][k][m], &nt);
        if (r != cudaSuccess) return set_cuda_error(r, "group table");
        g->ntiles[l][k][m] = nt;
      }
  }
  CK(cudaMemcpyAsync(g->tbl, host.data(), g->tbl_bytes, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  CK(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
  g->mst.assign(n, nullptr);
  g->ev_join.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    CK(cudaStreamCreateWithFlags(&g->mst[i], cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&g->ev_join[i], cudaEventDisableTiming));
    g->ts[i]->st = g->mst[i];
  }
  return N2F_OK;
}

// per-member phases: the member streams start after everything enqueued on the group stream
static int fork(TrainerGroup* g) {
  CK(cudaEventRecord(g->ev_fork, g->st));
  for (cudaStream_t s : g->mst) CK(cudaStreamWaitEvent(s, g->ev_fork, 0));
  return N2F_OK;
}

// ... and the group stream continues after everything enqueued on the member streams
static int join(TrainerGroup* g) {
  for (size_t i = 0; i < g->mst.size(); ++i) {
    CK(cudaEventRecord(g->ev_join[i], g->mst[i]));
    CK(cudaStreamWaitEvent(g->st, g->ev_join[i], 0));
  }
  return N2F_OK;
}

void group_release(TrainerGroup* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  g->exec = nullptr;
  g->graph = nullptr;
  if (g->tbl) dev_free(g->al, g->tbl, g->tbl_bytes);
  g->tbl = nullptr;
  for (cudaStream_t s : g->mst)
    if (s) cudaStreamSynchronize(s), cudaStreamDestroy(s);
  for (cudaEvent_t e : g->ev_join)
    if (e) cudaEventDestroy(e);
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  g->mst.clear();
  g->ev_join.clear();
  g->ev_fork = nullptr;
}

static int group_conv(TrainerGroup* g, int l, int k, int m) {
  const Trainer* t0 = g->ts[0];
  const int cin = t0->net.cin(l), cout = t0->net.widths[l];
  CK(launch_conv_tc_grouped(m, t0->bf16, m == 0 ? cin : cout, m == 0 ? cout : cin,
                            g->tbl + g->toff[l][k][m], (int)g->ts.size(), g->ntiles[l][k][m],
                            &g->ts[0]->state->kerr, g->st));
  return N2F_OK;
}

int group_step(TrainerGroup* g, int pair) {
  LaunchScope ls(&g->launches);
  const int kind = pair < 2 ? 0 : 1;
  int rc;
  for (int l = 0; l < kLayers; ++l) {
    if (g->grouped[l]) {
      if ((rc = group_conv(g, l, kind, 0))) return rc;
    } else {
      if ((rc = fork(g))) return rc;
      for (Trainer* t : g->ts)
        if ((rc = step_forward(t, pair, l))) return rc;
      if ((rc = join(g))) return rc;
    }
  }
  if ((rc = fork(g))) return rc;
  for (Trainer* t : g->ts)
    if ((rc = step_head(t, pair))) return rc;
  if ((rc = join(g))) return rc;
  // layer l's weight gradients (member streams) overlap its grouped dgrad (group stream); they
  // are joined before the next dgrad overwrites the delta buffer they read
  for (int l = kLayers - 1; l >= 0; --l) {
    if ((rc = fork(g))) return rc;
    for (Trainer* t : g->ts)
      if ((rc = step_wgrad(t, pair, l))) return rc;
    if (l > 0 && g->grouped[l]) {
      if ((rc = group_conv(g, l, kind, 1))) return rc;
    } else if (l > 0) {
      for (Trainer* t : g->ts)
        if ((rc = step_dgrad(t, pair, l))) return rc;
    }
    if ((rc = join(g))) return rc;
  }
  if ((rc = fork(g))) return rc;
  for (Trainer* t : g->ts) {
    if ((rc = step_adam(t))) return rc;
    t->steps_enqueued += 1;
  }
  return join(g);
}

int group_validate(TrainerGroup* g) {
  LaunchScope ls(&g->launches);
  int rc;
  for (Trainer* t : g->ts)
    if (t->sw) CK(cudaMemsetAsync(t->sw->vact, 0, sizeof(t->sw->vact), g->st));
  for (int l = 0; l < kLayers; ++l) {
    if (g->grouped[l]) {
      if ((rc = group_conv(g, l, 2, 0))) return rc;
    } else {
      if ((rc = fork(g))) return rc;
      for (Trainer* t : g->ts)
        if ((rc = val_forward(t, l, false))) return rc;
      if ((rc = join(g))) return rc;
    }
  }
  if ((rc = fork(g))) return rc;
  for (Trainer* t : g->ts)
    if ((rc = val_finish(t, false))) return rc;
  return join(g);
}

int group_epoch(TrainerGroup* g) {
  int rc;
  for (int k = 0; k < 4; ++k)
    if ((rc = group_step(g, k))) return rc;
  return group_validate(g);
}

int group_epoch_graph(TrainerGroup* g) {
  if (!g->exec) {
    uint64_t counted = 0;
    cudaGraph_t gr = nullptr;
    {
      LaunchScope ls(&counted);
      cudaError_t e = cudaStreamBeginCapture(g->st, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return set_cuda_error(e, "group graph capture");
      const int rc = group_epoch(g);
      e = cudaStreamEndCapture(g->st, &gr);
      if (rc) {
        if (gr) cudaGraphDestroy(gr);
        return rc;
      }
      if (e != cudaSuccess) return set_cuda_error(e, "group graph capture");
    }
    const cudaError_t e = cudaGraphInstantiate(&g->exec, gr, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(gr);
      return set_cuda_error(e, "group graph instantiate");
    }
    g->graph = gr;
    g->epoch_kernels = counted;
    for (Trainer* t : g->ts) {  // the capture advanced the counters once
      t->steps_enqueued -= 4;
      t->vals_enqueued -= 1;
    }
  }
  CK(cudaGraphLaunch(g->exec, g->st));
  for (Trainer* t : g->ts) {
    t->steps_enqueued += 4;
    t->vals_enqueued += 1;
  }
  g->launches += g->epoch_kernels;
  count_launch((int)g->epoch_kernels);
  return N2F_OK;
}


// Tunes every tensor-core conv shape of the job (training pairs' two shapes and the full image,
// forward and dgrad) on its own buffers, before its first epoch: the buffers written here are
// all rewritten by the epochs.
int trainer_autotune(Trainer* t) {
  for (int l = 1; l < kLayers; ++l) {
    if (t->engine[l] != N2F_ENGINE_TC) continue;
    const int cin = t->net.cin(l), cout = t->net.widths[l];
    const float* b = t->theta + t->net.b_off[l];
    for (int k = 0; k < 3; ++k) {
      const int h = k == 2 ? t->H : t->ph[k == 0 ? 0 : 2];
      const int w = k == 2 ? t->W : t->pw[k == 0 ? 0 : 2];
      const void* in = k == 2 ? t->vb[(l - 1) & 1] : t->act[l - 1];
      void* out = k == 2 ? t->vb[l & 1] : t->act[l];
      CK(conv_tc_autotune(0, t->bf16, in, cin, cout, h, w, t->pa.tcf[l], t->pa.tcf_lo[l], b,
                          nullptr, out, fwd_scales(k == 2 ? val_words(t, false) : train_words(t), l),
                          &t->state->kerr, t->st));
      if (k == 2) continue;
      CK(conv_tc_autotune(1, t->bf16, delta_of(t, l), cout, cin, h, w, t->pa.tcd[l],
                          t->pa.tcd_lo[l], nullptr, t->act[l - 1], delta_of(t, l - 1),
                          dgrad_scales(t, l), &t->state->kerr, t->st));
    }
  }
  return N2F_OK;
}

int trainer_epoch(Trainer* t) {
  for (int k = 0; k < 4; ++k) {
    int rc = trainer_step(t, k);
    if (rc) return rc;
  }
  return trainer_validate(t);
}

// Overlapped epoch: the previous epoch's validation runs on vst, reading a snapshot of the
// weights that epoch left, beside this epoch's four steps on st; the streams join before the
// epoch ends. The validation's buffers, magnitude words and weight copies are its own, so the
// two share only the job state, in which they write different fields (the steps: t, the bias
// corrections and the loss; the validation: the stop-rule fields). If the validation stops the
// job the steps beside it are discarded (k_step_restore) and the job's final state equals the
// in-line schedule's.
static int epoch_overlapped(Trainer* t) {
  int rc;
  const bool val = t->val_pending;
  if (val) {
    LaunchScope ls(&t->launches);
    CK(cudaMemcpyAsync(t->vsnap, t->slab + t->snap_off, t->snap_bytes, cudaMemcpyDeviceToDevice,
                       t->st));
    if (t->sw)
      CK(cudaMemcpyAsync(t->sw->vw, t->sw->w, sizeof(t->sw->w), cudaMemcpyDeviceToDevice, t->st));
    CK(cudaMemcpyAsync(t->state_save, t->state, sizeof(DevState), cudaMemcpyDeviceToDevice,
                       t->st));
    CK(cudaEventRecord(t->ev_vfork, t->st));
    CK(cudaStreamWaitEvent(t->vst, t->ev_vfork, 0));
    cudaStream_t main = t->st;
    t->st = t->vst;  // every launch of the validation goes to vst
    rc = validate(t, true);
    t->st = main;
    if (rc) return rc;
    CK(cudaEventRecord(t->ev_vjoin, t->vst));
  }
  for (int k = 0; k < 4; ++k)
    if ((rc = trainer_step(t, k))) return rc;
  t->val_pending = true;
  if (val) {
    LaunchScope ls(&t->launches);
    CK(cudaStreamWaitEvent(t->st, t->ev_vjoin, 0));
    CK(launch_step_restore(t->state, t->state_save, t->st));
  }
  return N2F_OK;
}

// Whether the launches of the next epoch are timed (kt set): every profile_every-th epoch.
static bool timed_epoch(const Trainer* t) {
  return t->profile_every <= 1 || (t->steps_enqueued / 4) % t->profile_every == 0;
}

static int epoch_job(Trainer* t) {
  return overlapped(t) ? epoch_overlapped(t) : trainer_epoch(t);
}

int trainer_epoch_job(Trainer* t) {
  t->timing_on = !t->kt || timed_epoch(t);
  const int rc = epoch_job(t);
  t->timing_on = true;
  return rc;
}

namespace {

// Finds the event-record nodes of the captured epoch that belong to timed launches.
int bind_timed_nodes(Trainer* t, cudaGraph_t g) {
  if (t->tnodes.empty()) return N2F_OK;
  size_t n = 0;
  CK(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  CK(cudaGraphGetNodes(g, nodes.data(), &n));
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    CK(cudaGraphNodeGetType(nd, &ty));
    if (ty != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t ev = nullptr;
    CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
    for (Trainer::TimedNode& tn : t->tnodes) {
      if (tn.a == ev) tn.na = nd;
      if (tn.b == ev) tn.nb = nd;
    }
  }
  for (const Trainer::TimedNode& tn : t->tnodes)
    if (!tn.na || !tn.nb) return set_cuda_error(cudaErrorInvalidValue, "timed graph nodes");
  return N2F_OK;
}

}  // namespace

// Captures one epoch (with the timed launches' event records, or without any) and
// instantiates it; the enqueue counters are left as they were.
static int capture_epoch(Trainer* t, bool timed, cudaGraph_t* gout, cudaGraphExec_t* xout,
                         uint64_t* kernels) {
  uint64_t counted = 0;
  cudaGraph_t g = nullptr;
  {
    LaunchScope ls(&counted);
    if (timed) t->tnodes.clear();
    t->cap_steps0 = t->steps_enqueued;
    t->cap_vals0 = t->vals_enqueued;
    t->capturing = true;
    t->timing_on = timed;
    cudaError_t e = cudaStreamBeginCapture(t->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      t->capturing = false;
      t->timing_on = true;
      return set_cuda_error(e, "epoch graph capture");
    }
    const int rc = epoch_job(t);
    e = cudaStreamEndCapture(t->st, &g);
    t->capturing = false;
    t->timing_on = true;
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return set_cuda_error(e, "epoch graph capture");
  }
  int rc = timed ? bind_timed_nodes(t, g) : N2F_OK;
  if (rc) {
    cudaGraphDestroy(g);
    return rc;
  }
  const cudaError_t e = cudaGraphInstantiate(xout, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return set_cuda_error(e, "epoch graph instantiate");
  }
  *gout = g;  // kept: the timed nodes are addressed through it
  *kernels = counted;
  // the captured calls advanced the enqueue counters once; the launch is the epoch
  t->steps_enqueued -= 4;
  t->vals_enqueued -= 1;
  return N2F_OK;
}

int trainer_epoch_graph(Trainer* t) {
  // an overlapped job's first epoch has no validation beside it: it runs as it is
  if (overlapped(t) && !t->val_pending) return trainer_epoch_job(t);
  // a profiled job replays the graph with event records on its timed epochs only
  const bool timed = !t->kt || timed_epoch(t);
  cudaGraph_t* g = timed ? &t->epoch_graph : &t->epoch_graph_plain;
  cudaGraphExec_t* x = timed ? &t->epoch_exec : &t->epoch_exec_plain;
  if (!*x) {
    const int rc = capture_epoch(t, timed && t->kt, g, x, &t->epoch_kernels);
    if (rc) return rc;
  }
  if (timed && t->kt) {
    // every replay records into its own events, harvested when the job's steps are known
    for (const Trainer::TimedNode& tn : t->tnodes) {
      KTimer::Pair p;
      p.a = t->kt->get();
      p.b = t->kt->get();
      p.flops = tn.flops;
      p.bytes = tn.bytes;
      p.val = tn.val;
      p.seq = tn.val ? t->vals_enqueued + tn.k : t->steps_enqueued + tn.k;
      CK(cudaGraphExecEventRecordNodeSetEvent(*x, tn.na, p.a));
      CK(cudaGraphExecEventRecordNodeSetEvent(*x, tn.nb, p.b));
      t->kt->pending.push_back(p);
    }
  }
  CK(cudaGraphLaunch(*x, t->st));
  t->steps_enqueued += 4;
  t->vals_enqueued += 1;
  t->launches += t->epoch_kernels;
  count_launch((int)t->epoch_kernels);
  return N2F_OK;
}

int trainer_finish(Trainer* t) {
  LaunchScope ls(&t->launches);
  CK(launch_result(t->V, t->S, t->Vbest, t->out, t->N, t->state, t->fixed_mode, t->st));
  return N2F_OK;
}

int trainer_read_state(Trainer* t, DevState* s) {
  CK(cudaMemcpyAsync(s, t->state, sizeof(DevState), cudaMemcpyDeviceToHost, t->st));
  CK(cudaStreamSynchronize(t->st));
  return N2F_OK;
}

void fill_status(const Trainer* t, const DevState& s, n2f_status* st) {
  st->epoch = (uint32_t)s.epoch;
  st->steps = (uint32_t)s.t;
  st->since = (uint32_t)s.since;
  st->stopped = (uint32_t)(s.stopped == 3 ? 0 : s.stopped);
  st->H = (uint32_t)t->H;
  st->W = (uint32_t)t->W;
  st->best_mse = s.best;
  st->last_mse = s.last_mse;
  st->last_loss = s.loss;
}

}  // namespace n2f
