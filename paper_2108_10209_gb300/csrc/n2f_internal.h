// Internal declarations of the sm_103a Noise2Fast library (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/n2f.h"

namespace n2f {

constexpr int kLayers = 8;  // eight 3x3 conv + ReLU layers, then the 1x1 + sigmoid head

// Flat parameter vector in the canonical order: for l = 1..8: W_l[C_out][C_in][3][3], b_l;
// then head w[C_8], b. Kernels read weights from packed copies (see Packing), never from it.
struct NetShape {
  int widths[kLayers];
  int c0 = 1;  // input channels of the first layer
  size_t w_off[kLayers + 1], b_off[kLayers + 1], count;
  int cin(int l) const { return l == 0 ? c0 : widths[l - 1]; }
  int cmax() const {
    int m = 0;
    for (int l = 0; l < kLayers; ++l) m = widths[l] > m ? widths[l] : m;
    return m;
  }
  int csum() const {
    int s = 0;
    for (int l = 0; l < kLayers; ++l) s += widths[l];
    return s;
  }
  void init(int which, int channels = 1);
};

// Device-resident per-job scalars (updated only by kernels, so CUDA graphs can replay epochs).
struct DevState {
  double best;      // best validation MSE (+inf before the first epoch)
  double last_mse;  // MSE of the last validation
  double loss;      // training loss of the last step
  int since;        // epochs since the best
  int epoch;        // validations done under the stop rule
  int stopped;      // 0 running, 1 rule fired, 2 max_epochs reached, 3 non-finite
  int t;            // Adam steps taken
  int decision;     // last validation: 1 new best, 0 joins the window, -1 ignored
  int patience, max_epochs, incl_best;
  float bc1, bc2;   // Adam bias corrections 1 - beta^t of the current step
  double b1t, b2t;  // beta1^t, beta2^t
  int kerr;         // first error a kernel reported (a wait that ran out of time), 0 = none
  int pad;
};

// Largest magnitudes (float bits of |v|, raised by atomicMax in the kernels that write the
// tensor) of the tensors that the float32 form's tensor-core kernels split into two fp16 parts;
// each consumer derives its power-of-two operand scale from them (tc_common.cuh, f16_scale).
// The Adam kernel clears `act` and `delta` after every step, so a word bounds the tensor's
// current contents (it may also cover an earlier pass: still a bound, never too small).
struct ScaleWords {
  unsigned act[kLayers];       // act[m]: output of layer m in the training forward
  unsigned delta[kLayers];     // delta[m]: masked gradient at layer m's pre-activation
  unsigned wnew[2][kLayers];   // weights after an Adam step, by the step's parity
  unsigned w[kLayers];         // the weights that the packed tensor-core copies were made from
  // the validation forward's own words (cleared when a validation starts), so that training
  // and validation scales never mix and the two may run at the same time
  unsigned vact[kLayers];      // vact[m]: output of layer m in the validation forward
  unsigned vw[kLayers];        // w[] as of the weight snapshot a concurrent validation reads
};

// Packed weight copies written by the init/Adam kernels, one per layer l = 0..7:
//   fwd : [C_in/8][9][8][C_out] f32 (tap = 3*ky + kx; layer 1: [C_out][9]) -- SIMT forward
//   dgr : [C_out/8][9][8][C_in] f32, tap rotated to 8 - tap                -- SIMT dgrad
//   tcf/tcd : the same two matrices in the tensor-core operand order (tc_layout.cuh), bf16,
//             or in the float32 form fp16 hi parts of the scaled weights with the fp16
//             residuals in tcf_lo/tcd_lo (written by k_pack_tc after the Adam kernel; the
//             CUDA-core copies fwd/dgr exist only for the layers that run on the CUDA cores)
struct PackArgs {
  float* theta;
  float* fwd[kLayers];
  float* dgr[kLayers];
  void* tcf[kLayers];
  void* tcd[kLayers];
  void* tcf_lo[kLayers];
  void* tcd_lo[kLayers];
  ScaleWords* sw;  // float32 form with tensor-core layers; nullptr otherwise
  int widths[kLayers];
  int c0;       // input channels of the first layer
  unsigned long long w_off[kLayers + 1], b_off[kLayers + 1];
  unsigned long long count;
  int tc_bf16;  // tensor-core copies in bf16 (1) or f32 (0); tcf[l] == nullptr: none
};

// ---- kernel launchers (kernels_*.cu); all enqueue on `st` and return cudaError_t ----------
cudaError_t launch_gather_quad(const float* x, int H, int W, float* tl, float* tr, float* br,
                               float* bl, cudaStream_t st);
cudaError_t launch_exact_target(const float* xt, const float* s_tgt, const float* s_in, size_t n,
                                float* out, cudaStream_t st);
cudaError_t launch_max_project(const float* vol, int Z, size_t n, float* out, cudaStream_t st);
cudaError_t launch_gather(const float* x, int H, int W, float* ue, float* uo, float* le, float* lo,
                          cudaStream_t st);
cudaError_t launch_u16_to_f32(const uint16_t* in, float* out, size_t n, cudaStream_t st);
cudaError_t launch_init_params(float* theta, const NetShape& net, uint64_t seed, cudaStream_t st);
// Adam's constants as the float32 kernel uses them: beta, 1 - beta formed in double, lr, eps.
struct AdamConsts {
  float lr, b1, omb1, b2, omb2, eps;
};
AdamConsts adam_consts(double lr, double b1, double b2, double eps);
// Adam step (update = 1) or a plain repack (update = 0), then the tensor-core copies
// (k_pack_tc: bf16, or the float32 form's fp16 parts). With update = 0 the caller clears
// pa.sw->wnew first.
cudaError_t launch_adam(const PackArgs& pa, const float* grad, float* m, float* v,
                        const AdamConsts& k, const DevState* state, int update, cudaStream_t st);
// One canonical weight tensor into its operand copies. Float32 form: wmax (device word, zeroed
// by the caller) receives the tensor's largest magnitude and the fp16 parts are scaled by it.
cudaError_t launch_pack_layer(const float* w, int cin, int cout, float* fwd, float* dgr, void* tcf,
                              void* tcd, void* tcf_lo, void* tcd_lo, int tc_bf16, unsigned* wmax,
                              cudaStream_t st);
// *out = max(*out, largest |x[i]|) as float bits, x float32 (bf16 = 0) or bf16.
cudaError_t launch_absmax(const void* x, size_t n, int bf16, unsigned* out, const int* skip,
                          cudaStream_t st);
cudaError_t launch_pack_cg(const float* nchw, int C, int H, int W, int bf16, void* cg,
                           cudaStream_t st);
cudaError_t launch_unpack_cg(const void* cg, int C, int H, int W, int bf16, float* nchw,
                             cudaStream_t st);
cudaError_t launch_unpack_cg_f64(const void* cg, int C, int H, int W, int bf16, double* out,
                                 cudaStream_t st);

// First layer (C_in = 1): image plane -> CG map with bias + ReLU.
constexpr int kMaxC0 = 4;  // input channels the first-layer kernels take
// amax (may be null): receives the output's largest magnitude (float32 form).
cudaError_t launch_conv1_fwd(const float* img /*[C0][H][W]*/, int C0, int H, int W,
                             const float* w /*[C][C0][9]*/, const float* b, int C, int bf16,
                             void* out, unsigned* amax, const int* skip, cudaStream_t st);
// First layer weight gradient: partials then ordered reduce into grad (canonical order).
cudaError_t launch_conv1_wgrad(const void* dout, const float* img, int C0, int H, int W, int C,
                               int bf16, float* part, size_t part_cap, float* gw, float* gb,
                               const int* skip, cudaStream_t st);

// SIMT implicit-GEMM 3x3 layers (C_in, C_out multiples of 8).
// mode 0: out = ReLU(conv(in, wk) + b);  mode 1: out = conv(in, wk) * [mask > 0]
// wk: [C_in/8][9][8][C_out] f32 (for dgrad: the rotated transpose, "C_out" = layer C_in)
cudaError_t launch_conv_simt(int mode, int bf16, const void* in, int cin, int cout, int H, int W,
                             const float* wk, const float* b, const void* mask, void* out,
                             const int* skip, cudaStream_t st);
// SIMT weight gradient: dW[o][c][ky][kx] (canonical order) and db[o] from CG maps.
cudaError_t launch_wgrad_simt(int bf16, const void* dout, const void* in, int cin, int cout, int H,
                              int W, float* part, size_t part_cap, float* gw, float* gb,
                              const int* skip, cudaStream_t st);

// Tensor-core (tcgen05) kernels; return cudaErrorNotSupported when a shape is not covered.
cudaError_t tc_prepare();  // once per process, before any launch or capture
cudaError_t conv_tc_prepare();   // the forward / dgrad kernels' part of tc_prepare
cudaError_t wgrad_tc_prepare();  // the weight-gradient kernels' part
bool tc_supported(int cin, int cout);
bool tc_wgrad_supported(int cin, int cout, int bf16);
// mode 0 forward (bias + ReLU), 1 dgrad (ReLU mask); w_hi/w_lo: packed operand copies
// (tc_layout.cuh), w_lo only in the float32 form. err: device error word.
// Float32 form: the operands are split into two fp16 parts scaled by powers of two derived from
// the largest magnitudes `sc.in` (the A operand tensor) and `sc.w` (the weights the packed copies
// were made from); `sc.out`, if not null, receives the output's largest magnitude. The bf16 form
// ignores all three.
struct ConvScales {
  const unsigned* in = nullptr;
  const unsigned* w = nullptr;
  unsigned* out = nullptr;
};
// Times the launch choices that leave results unchanged (pipeline stages, CTAs per SM) for one
// conv shape on the given buffers (their contents are overwritten) and caches the fastest for
// every later launch of that (mode, precision, C_in, C_out, H, W) in this process.
cudaError_t conv_tc_autotune(int mode, int bf16, const void* in, int cin, int cout, int H, int W,
                             const void* w_hi, const void* w_lo, const float* b, const void* mask,
                             void* out, ConvScales sc, int* err, cudaStream_t st);
// Grouped forward / dgrad: one persistent launch over the tiles of n images of the same layer
// shape, each with its own input, weights, bias or mask and output. The table (conv_job_size()
// bytes per image, 128-byte aligned) is filled on the host by conv_group_table and copied to
// device memory before the launch.
struct ConvGroupEntry {
  const void* in;
  int H, W;
  const void* w_hi;
  const void* w_lo;
  const float* bias;
  const void* mask;
  void* out;
  const int* skip;
  ConvScales sc;
};
size_t conv_job_size();
cudaError_t conv_group_table(int mode, int bf16, int cin, int cout, const ConvGroupEntry* e,
                             int n, void* table, long* ntiles);
cudaError_t launch_conv_tc_grouped(int mode, int bf16, int cin, int cout, const void* dtable,
                                   int n, long ntiles, int* err, cudaStream_t st);
cudaError_t launch_conv_tc(int mode, int bf16, const void* in, int cin, int cout, int H, int W,
                           const void* w_hi, const void* w_lo, const float* b, const void* mask,
                           void* out, ConvScales sc, const int* skip, int* err, cudaStream_t st);
// dmax / xmax: largest magnitudes of dout and in (float32 form; ignored by the bf16 form).
cudaError_t launch_wgrad_tc(int bf16, const void* dout, const void* in, int cin, int cout, int H,
                            int W, const unsigned* dmax, const unsigned* xmax, float* part,
                            size_t part_cap, float* gw, float* gb, const int* skip, int* err,
                            cudaStream_t st);
size_t tc_weight_elems(int cin, int cout);  // elements of one packed tensor-core weight copy

// Head (1x1 conv + sigmoid), training: z, loss partials, dL/dz, delta_8, head-grad partials;
// dmax (may be null) receives delta_8's largest magnitude.
cudaError_t launch_head_train(const void* a8, int C, int npx, const float* w9, const float* b9,
                              const float* tgt, int loss_kind, int bf16, float* dz, void* d8,
                              unsigned* dmax, double* loss_part, float* hpart, int* nblk_out,
                              const int* skip, cudaStream_t st);
// Sums head-grad and loss partials in a fixed order, advances the Adam step counter (one launch).
cudaError_t launch_step_finish(const float* hpart, const double* loss_part, int nblk, int C,
                               int npx, float* gw9, float* gb9, DevState* state, double b1,
                               double b2, cudaStream_t st);
// Head, validation: V = sigmoid(z), FP64 partial sums of (V - x)^2.
cudaError_t launch_head_val(const void* a8, int C, int npx, const float* w9, const float* b9,
                            const float* x, int bf16, float* V, double* mse_part, int* nblk_out,
                            const int* skip, cudaStream_t st);
// Stop rule: reduce the MSE partials (fixed order), update best/since/epoch/stopped, and
// record the score in the history ring (kHistCap doubles; may be null) at (epoch - 1) % kHistCap.
constexpr int kHistCap = N2F_HIST_CAP;
cudaError_t launch_val_decide(const double* mse_part, int nblk, size_t npx, DevState* state,
                              int fixed_mode, double* hist, cudaStream_t st);
// Output averaging: S = 0 / V (new best) or S += V; Vbest = V on a new best.
cudaError_t launch_val_accum(const float* V, float* S, float* Vbest, size_t n,
                             const DevState* state, cudaStream_t st);
// Result: S / patience, S / count, Vbest or V (fixed-step mode).
cudaError_t launch_result(const float* V, const float* S, const float* Vbest, float* out, size_t n,
                          const DevState* state, int fixed_mode, cudaStream_t st);
// Puts DevState's step counters back from `saved` if the job has stopped (overlapped
// validation: the epoch that ran beside the deciding validation is discarded).
cudaError_t launch_step_restore(DevState* state, const DevState* saved, cudaStream_t st);

// Checked builds (N2F_CHECKED, checked.cuh): each kernel file's count of indexes found outside
// their tensor and the first such source line, on the current device (clear != 0: zero them
// afterwards); the normal build reports zeros.
int check_read_basic(unsigned long long* fails, int* line, int clear);
int check_read_simt(unsigned long long* fails, int* line, int clear);
int check_read_conv(unsigned long long* fails, int* line, int clear);
int check_read_wgrad(unsigned long long* fails, int* line, int clear);

// Count of kernel launches made by this thread's current owner (see LaunchCounter).
extern thread_local uint64_t* tl_launch_counter;
inline void count_launch(int n = 1) {
  if (tl_launch_counter) *tl_launch_counter += (uint64_t)n;
}

}  // namespace n2f
