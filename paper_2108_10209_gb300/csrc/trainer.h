// Step executor of one Noise2Fast job (host side).
#pragma once
#include <string>
#include <vector>

#include "n2f_internal.h"

namespace n2f {

extern thread_local std::string tl_error;
int set_cuda_error(cudaError_t e, const char* where);

struct Allocator {
  n2f_alloc_fn alloc = nullptr;
  n2f_free_fn free = nullptr;
  void* user = nullptr;
};
void* dev_alloc(const Allocator& a, size_t bytes);
void dev_free(const Allocator& a, void* p, size_t bytes);

// Counts the kernels enqueued while it is alive into *dst, and into the enclosing scope's
// counter as well when scopes nest (a context counting around a trainer).
struct LaunchScope {
  uint64_t* prev;
  uint64_t* dst;
  uint64_t start;
  explicit LaunchScope(uint64_t* d) : prev(tl_launch_counter), dst(d), start(*d) {
    tl_launch_counter = d;
  }
  ~LaunchScope() {
    if (prev && prev != dst) *prev += *dst - start;
    tl_launch_counter = prev;
  }
};

// Times the launches of one kernel class with CUDA events on the launching stream.
struct KTimer {
  struct Pair {
    cudaEvent_t a, b;
    double flops, bytes;
    int val;  // 0: part of training step `seq`, 1: part of validation `seq`
    uint64_t seq;
  };
  int kind = N2F_K_NONE;
  std::vector<cudaEvent_t> pool;
  std::vector<Pair> pending;
  uint64_t launches = 0;
  double ms = 0, flops = 0, bytes = 0;
  cudaEvent_t get();
  // Adds the finished pairs that belong to steps < steps_done and validations < vals_done
  // (launches of epochs enqueued after the stop returned at once and are not counted).
  void harvest(uint64_t steps_done, uint64_t vals_done);
  void destroy();
};

struct Trainer {
  NetShape net;
  n2f_params prm;
  int H = 0, W = 0;
  size_t N = 0;
  int ph[4], pw[4];  // sub-image sizes: up (H x W/2) twice, left (H/2 x W) twice; Quad H/2 x W/2
  int tgt_of[4];     // pair k trains sub-image k -> sub-image tgt_of[k]
  int nplanes = 1;   // planes of x and of every sub-image: input channels (+ the clean plane)
  float* tx[4] = {nullptr, nullptr, nullptr, nullptr};  // Exact: the adjusted targets
  size_t maxP = 0;
  int bf16 = 0, keep_deltas = 0, fixed_mode = 0, want_u16 = 0;
  int engine[kLayers];     // forward / dgrad kernels of layer l
  int wg_engine[kLayers];  // weight-gradient kernel of layer l
  cudaStream_t st = nullptr;
  Allocator al;
  char* slab = nullptr;
  size_t slab_bytes = 0;
  uint64_t launches = 0;
  // device buffers (views into the slab)
  float *x = nullptr, *sub[4] = {nullptr, nullptr, nullptr, nullptr};
  float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  PackArgs pa;
  void* act[kLayers] = {};
  void* dkeep[kLayers] = {};
  void* dl[2] = {};
  void* vb[2] = {};
  float *dz = nullptr, *V = nullptr, *S = nullptr, *Vbest = nullptr, *out = nullptr;
  double *lpart = nullptr, *mpart = nullptr;
  float* hpart = nullptr;
  float* wpart = nullptr;
  size_t wpart_cap = 0;
  int nblk_max = 0;
  DevState* state = nullptr;
  double* hist = nullptr;    // validation scores by epoch, a ring of kHistCap
  ScaleWords* sw = nullptr;  // float32 form: tensor magnitudes for the fp16 operand scales
  uint16_t* in_u16 = nullptr;
  DevState hstate_init;
  int last_pair = 0;
  uint64_t steps_enqueued = 0, vals_enqueued = 0;
  KTimer* kt = nullptr;  // optional kernel-class timer (owned by the caller)
  // one epoch captured as a CUDA graph (everything it mutates lives in device memory)
  cudaGraph_t epoch_graph = nullptr;
  cudaGraphExec_t epoch_exec = nullptr;
  // a profiled job (kt) with profile_every > 1 also replays an epoch captured without the
  // timed launches' event records on its untimed epochs
  cudaGraph_t epoch_graph_plain = nullptr;
  cudaGraphExec_t epoch_exec_plain = nullptr;
  uint32_t profile_every = 1;
  bool timing_on = true;       // Timed brackets launches (cleared for untimed epochs)
  uint64_t epoch_kernels = 0;  // kernels in one captured epoch
  // Timed launches inside the captured epoch: their event-record nodes get fresh events before
  // every replay, so a profiled job still replays graphs. `k` is the step within the epoch
  // (or 0 for the validation), `a`/`b` the nodes' events while capturing.
  struct TimedNode {
    cudaGraphNode_t na = nullptr, nb = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    double flops = 0, bytes = 0;
    int val = 0, k = 0;
  };
  bool capturing = false;
  uint64_t cap_steps0 = 0, cap_vals0 = 0;
  std::vector<TimedNode> tnodes;
  // Overlapped validation (prm.overlap): the validation buffers do not alias the training
  // ones; at each epoch boundary theta and the forward weight copies (one contiguous range of
  // the slab, snap_off / snap_bytes) are copied to vsnap, and the previous epoch's validation
  // runs on vst from that copy (vpa) while the epoch trains on st. DevState's step counters
  // are saved in state_save at the boundary and put back if that validation stopped the job.
  cudaStream_t vst = nullptr;
  cudaEvent_t ev_vfork = nullptr, ev_vjoin = nullptr;
  char* vsnap = nullptr;
  size_t snap_off = 0, snap_bytes = 0;
  PackArgs vpa;
  DevState* state_save = nullptr;
  bool val_pending = false;  // an epoch has trained whose validation has not been enqueued
};

int trainer_configure(Trainer* t, int H, int W, const n2f_params* p, int keep_deltas);
size_t trainer_bytes(int H, int W, const n2f_params* p, int keep_deltas);
int trainer_init(Trainer* t, const Allocator& al, cudaStream_t st, int want_u16);
void trainer_release(Trainer* t);
int trainer_start(Trainer* t, int from_u16);
int trainer_repack(Trainer* t);
int trainer_step(Trainer* t, int pair);
int trainer_validate(Trainer* t);
int trainer_epoch(Trainer* t);
// Tunes the job's conv launch choices (see conv_tc_autotune) before its first epoch.
int trainer_autotune(Trainer* t);
// A job's epoch: trainer_epoch, or with prm.overlap the previous epoch's validation on a
// second stream beside this epoch's four steps (the first epoch trains only).
int trainer_epoch_job(Trainer* t);
// Same as trainer_epoch_job, replaying a CUDA graph of the epoch captured on first use.
int trainer_epoch_graph(Trainer* t);
int trainer_finish(Trainer* t);

// Jobs of identical parameters stepped in lockstep on one stream: the tensor-core forward and
// dgrad of every layer run as one grouped launch over all members' tiles (each member with its
// own weights, image size and stop flag); the other kernels run per member on the member's
// own stream. Members must be trainer_init'ed on the group's stream without kept deltas;
// group_init moves each member to its own stream.
struct TrainerGroup {
  std::vector<Trainer*> ts;
  cudaStream_t st = nullptr;
  Allocator al;
  char* tbl = nullptr;  // grouped-launch tables, device memory
  size_t tbl_bytes = 0;
  size_t toff[kLayers][3][2];  // [layer][pair shape 0/1, validation 2][forward, dgrad]
  long ntiles[kLayers][3][2];
  bool grouped[kLayers];
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t epoch_kernels = 0, launches = 0;
  // per-member work forks from the group stream onto one stream per member and joins back,
  // so members' kernels overlap each other (and a layer's weight gradients its grouped dgrad)
  std::vector<cudaStream_t> mst;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
};
int group_init(TrainerGroup* g, const Allocator& al, cudaStream_t st);
void group_release(TrainerGroup* g);
int group_step(TrainerGroup* g, int pair);
int group_validate(TrainerGroup* g);
int group_epoch(TrainerGroup* g);
int group_epoch_graph(TrainerGroup* g);
int trainer_read_state(Trainer* t, DevState* s);
void fill_status(const Trainer* t, const DevState& s, n2f_status* st);

}  // namespace n2f
