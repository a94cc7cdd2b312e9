/*
 * gfflow.h -- C ABI of the GB300 flow-based sampler for lattice phi^4 theory
 * (method of Tomiya & Terasaki, "GomalizingFlow.jl", arXiv:2208.08903).
 *
 * Conventions for every call
 *   - Fields are [B][V] row-major, V = L^nd sites, site index
 *     n = x + L*(y + L*z) (x fastest), periodic boundaries in every axis.
 *   - Pointers named d_* / "device" are device memory owned by the caller;
 *     "host" pointers are host memory owned by the caller.  The library owns
 *     only what gf_flow_create allocates (the device copy of the weights).
 *   - Every compute call is asynchronous on the given stream and launches
 *     only this library's kernels.  Argument errors return GF_EINVAL before
 *     anything is launched; a failed launch returns GF_ECUDA.  Errors a kernel
 *     detects (a bounded wait that ran out, a corrupt schedule) are recorded
 *     in a device status word read by gf_device_status; no call traps.
 *   - Random numbers: Philox4x64-10 (Salmon et al., SC'11), keyed by the
 *     caller's seed, one counter sub-space per purpose, so results do not
 *     depend on launch shape or batching.
 */
#ifndef GFFLOW_H
#define GFFLOW_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GF_OK = 0,
    GF_EINVAL = -1,        /* bad argument (null pointer, size, shape)            */
    GF_ENOMEM = -2,        /* device allocation failed (gf_flow_create only)      */
    GF_ECUDA = -3,         /* a CUDA runtime call or launch failed                */
    GF_EUNSUPPORTED = -4,  /* valid request this build has no kernel for          */
    GF_ETIMEOUT = -5,      /* reported through gf_device_status                   */
    GF_EDEVICE = -6        /* reported through gf_device_status                   */
} gf_status;

typedef enum {
    GF_PREC_FP32 = 0,             /* FP32 convolutions, FP64 sums                  */
    GF_PREC_BF16CONV_FP64RED = 1  /* tensor-core convolutions with FP32
                                     accumulation; log-det, z^2 and action sums
                                     to FP64 accuracy (FP32 pairs per thread,
                                     FP64 across the block).  Two kernels:
                                     3D, L=16, C=32: conv2 (the dominant one)
                                     with BF16 operands (h1, W2), conv1 and
                                     conv3 on the tensor cores with FP16
                                     operands (the masked field, W1; h2, W3),
                                     so |field| and |h2| must stay below 65504
                                     (a non-finite s or t records GF_EDEVICE);
                                     other shapes (see gf_flow_tensor_core_
                                     supported): conv2 with BF16 operands (h1,
                                     W2) on the tensor cores, conv1 and conv3 in
                                     FP32 from the FP32 field and weights and
                                     the BF16 h2                                  */
} gf_precision;

/* Flow shape (paper Sec. 3, model parameters: n_layers, hidden_sizes =
 * [c_hidden1, c_hidden2], kernel_size, inC=1, outC=2, use_final_tanh,
 * use_bn=false).  The same network as gf_flow_shape_ex with n_hidden = 2 (see
 * there for what is supported); L even (the checkerboard is a bipartition). */
typedef struct {
    int32_t nd, L, n_layers, c_hidden1, c_hidden2, ksize, use_final_tanh;
    double leaky_slope;   /* LeakyReLU slope after conv1 and conv2 */
} gf_flow_shape;

/* The general s/t network of the paper's model section (Sec. 3, model
 * parameters hidden_sizes and kernel_size): n_hidden convolutions of widths
 * hidden[0..n_hidden-1], each followed by LeakyReLU, then the head conv(-> 2)
 * (channel 0 = s, tanh when use_final_tanh; channel 1 = t).  Every
 * convolution is periodic with ksize^nd taps (ksize odd, circular padding
 * (ksize-1)/2), taps ordered (kz,ky,kx) resp. (ky,kx), kx fastest, offset
 * k - (ksize-1)/2.  Canonical weights per layer: for each convolution j =
 * 0..n_hidden, W_j[c_out][c_in][T] then b_j[c_out] (c_in of the first is 1,
 * c_out of the head 2).  n_hidden = 2, ksize = 3 is the layout of
 * gf_flow_shape.
 * Supported: nd in {2,3}; L even, L^nd <= 65536; 0 <= n_hidden <=
 * GF_MAX_HIDDEN; widths 1..256; ksize in {1,3,5,7}.  Two equal hidden widths in
 * {8,16,24,32} with ksize 3 run on the slice-cached kernels (the tensor-core
 * precision for the shapes gf_flow_tensor_core_supported accepts);
 * every other network runs on a whole-lattice FP32 kernel that needs
 * 4 (V + 2 V Cp) bytes of shared memory per block, Cp = the widest hidden
 * layer rounded up to odd, at most 227 KB (else GF_EUNSUPPORTED); those flows
 * support sampling and log q only (training and the unfused form return
 * GF_EUNSUPPORTED). */
#define GF_MAX_HIDDEN 8
typedef struct {
    int32_t nd, L, n_layers;
    int32_t n_hidden;
    int32_t hidden[GF_MAX_HIDDEN];
    int32_t ksize, use_final_tanh;
    double leaky_slope;   /* LeakyReLU slope after every hidden convolution */
} gf_flow_shape_ex;

/* phi^4 couplings (paper Sec. 1, action S[phi] and potential V[phi]):
 * S = sum_n [ sum_mu phi(n)(2 phi(n) - phi(n+mu) - phi(n-mu)) + m2 phi^2 + lam phi^4 ]. */
typedef struct { double m2, lam; } gf_phi4;

typedef struct gf_flow gf_flow;   /* opaque; owns the device copy of the weights */

/* MH chain state.  Lives in DEVICE memory (caller-allocated, 48 bytes,
 * 8-byte aligned) so successive calls continue one chain without a host
 * round trip.  Initialise with logw_cur=0, idx_cur=0, n_acc=0, step=0. */
typedef struct {
    double   logw_cur;   /* log weight of the current state                   */
    int64_t  idx_cur;    /* global proposal index of the current state        */
    int64_t  n_acc;      /* accepted proposals among steps 1..step-1          */
    int64_t  step;       /* proposals consumed so far (global step counter)   */
    uint64_t seed, stream_id;   /* Philox key of this chain's uniforms        */
} gf_mh_state;

/* ---------------------------------------------------------------------- */
/* Flow object                                                             */
/* ---------------------------------------------------------------------- */

/* Copies host FP64 weights (canonical layout, one block per layer in the
 * order the layers act on the prior sample; for gf_flow_shape: W1[c1][1][T] b1[c1]
 * W2[c2][c1][T] b2[c2] W3[2][c2][T] b3[2], T = 3^nd taps ordered
 * (kz,ky,kx) resp. (ky,kx), offset k-1; conv3 channel 0 is s, 1 is t) to the
 * device in the kernels' layouts.  Synchronises `stream` before returning.
 * *out is set only on GF_OK; release with gf_flow_destroy. */
gf_status gf_flow_create(const gf_flow_shape* shape, const double* weights_host,
                         gf_precision prec, cudaStream_t stream, gf_flow** out);
/* The same for the general network (any hidden_sizes list, odd kernel size;
 * canonical weights as described at gf_flow_shape_ex).  GF_PREC_BF16CONV_FP64RED
 * is supported only where gf_flow_create supports it. */
gf_status gf_flow_create_ex(const gf_flow_shape_ex* shape, const double* weights_host,
                            gf_precision prec, cudaStream_t stream, gf_flow** out);
/* 1 when gf_flow_create_ex accepts GF_PREC_BF16CONV_FP64RED for `shape`, else 0
 * (host only, no device work; a null or invalid shape gives 0).  Convolutions
 * go on the tensor cores where the hidden width makes conv2 a dense
 * contraction (paper Sec. 1, the coupling layers' convolutional networks):
 * two equal hidden widths of 8, 16, 24 or 32 (24 padded to 32 with zero
 * weights), ksize 3, and either 3D L=16 with width 32 (its own kernel) or a
 * lattice whose padded activations (about 2 Cp (L+2)^nd bytes, Cp = 8, 16 or
 * 32), weights and field fit one block's 227 KB of shared memory: 2D L <= 32
 * with any of the widths, 2D L = 64 and 3D L = 12, 16 with widths 8 and 16,
 * 3D L = 8 with any. */
int32_t gf_flow_tensor_core_supported(const gf_flow_shape_ex* shape);
gf_status gf_flow_destroy(gf_flow* flow);
/* Number of canonical parameters. */
int64_t   gf_flow_n_params(const gf_flow* flow);
/* Replaces the weights from a DEVICE FP32 array in canonical layout
 * (asynchronous on `stream`). */
gf_status gf_flow_set_weights_device(gf_flow* flow, const float* d_weights, cudaStream_t stream);
/* Copies the current FP32 canonical weights into d_weights_out [n_params]. */
gf_status gf_flow_get_weights_device(const gf_flow* flow, float* d_weights_out, cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* Sampling: phi = F^{-1}(z) with log q, S and log w (paper Sec. 1: prior  */
/* sample, untrivialising map, Jacobian, model density P^(ML)).            */
/* ---------------------------------------------------------------------- */

/* For b < B: z_b is d_z_in[b] when d_z_in != NULL, else drawn in-kernel from
 * philox(key=(seed,0), ctr=(counter0+b, j, 0, 1)) for sites 4j..4j+3 (FP32
 * Box-Muller).  Layer l (0-based) keeps sites with (x+y+z)%2 == l%2 fixed
 * and maps the others by x -> x*exp(s)+t, s=tanh(conv-net(fixed sites)).
 * Writes d_phi_out[b] (FP32), d_logq_out[b] = log r(z_b) - sum s (FP64).
 * d_z_out (nullable) receives z.  When phi4 != NULL, d_S_out and
 * d_logw_out (each nullable) receive S(phi_b) and -S - log q (FP64);
 * when phi4 == NULL both must be NULL. */
gf_status gf_flow_sample(const gf_flow* flow, const gf_phi4* phi4, int64_t B,
                         uint64_t seed, uint64_t counter0, const float* d_z_in,
                         float* d_z_out, float* d_phi_out, double* d_logq_out,
                         double* d_S_out, double* d_logw_out, cudaStream_t stream);

/* Trivialising direction z = F(phi) (paper Sec. 1, F_theta and its
 * bijectivity): layers in reverse order, x -> (x - t)*exp(-s).
 * d_logq_out[b] = log r(z_b) - sum s.  d_z_out nullable. */
gf_status gf_flow_logq(const gf_flow* flow, int64_t B, const float* d_phi_in,
                       float* d_z_out, double* d_logq_out, cudaStream_t stream);

/* The same function as gf_flow_sample computed the plain way: one kernel per
 * convolution (conv1, conv2, conv3 + affine update) per layer with every
 * activation written to and read back from device memory, then one kernel
 * for log r, S, log q and log w.  FP32 throughout except the FP64 sums.  It
 * is the comparison point for the fused kernels (same results within the
 * FP32 tolerance).  d_workspace: >= gf_unfused_workspace_bytes(flow, B)
 * bytes of device memory, 256-byte aligned, owned by the caller. */
size_t gf_unfused_workspace_bytes(const gf_flow* flow, int64_t B);
gf_status gf_flow_sample_unfused(const gf_flow* flow, const gf_phi4* phi4, int64_t B,
                                 uint64_t seed, uint64_t counter0, const float* d_z_in,
                                 float* d_z_out, float* d_phi_out, double* d_logq_out,
                                 double* d_S_out, double* d_logw_out, void* d_workspace,
                                 size_t workspace_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* Action (paper Sec. 1)                                                    */
/* ---------------------------------------------------------------------- */

/* d_S_out[b] = S(phi_b) in FP64 for d_phi [B][L^nd], FP32 (phi_is_fp64=0)
 * or FP64 (phi_is_fp64=1).  Each site term is formed in FP64. */
gf_status gf_phi4_action(int32_t nd, int32_t L, const gf_phi4* phi4, int64_t B,
                         const void* d_phi, int32_t phi_is_fp64, double* d_S_out,
                         cudaStream_t stream);
/* d_F_out = dS/dphi = 2 sum_mu (2phi - phi(n+mu) - phi(n-mu)) + 2 m2 phi
 * + 4 lam phi^3, FP64 in and out ([B][V]). */
gf_status gf_phi4_force(int32_t nd, int32_t L, const gf_phi4* phi4, int64_t B,
                        const double* d_phi, double* d_F_out, cudaStream_t stream);

/* Vector-Jacobian product for FP32 fields: d_gphi_out[b][n] = d_gS[b] *
 * dS/dphi_b(n), each product formed in FP64 and rounded once to FP32.  With
 * d_gS[b] = dLoss/dS_b it gives dLoss/dphi for a loss built on S (the
 * reverse-KL loss of Sec. 1 uses d_gS[b] = 1/B). */
gf_status gf_phi4_action_vjp(int32_t nd, int32_t L, const gf_phi4* phi4, int64_t B,
                             const float* d_phi, const double* d_gS, float* d_gphi_out,
                             cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* Metropolis-Hastings independence chain (paper Sec. 1: flow proposals   */
/* corrected by the MH test with the Jacobian)                             */
/* ---------------------------------------------------------------------- */

/* Bytes of device workspace gf_mh_chain needs for n proposals. */
size_t gf_mh_chain_workspace_bytes(int64_t n);

/* Consumes proposals k = 0..n-1 with log weights d_logw[k] (FP64, log p -
 * log q).  Global step g = state.step + k: g == 0 is accepted
 * unconditionally; otherwise accept iff (d_logw[k] - log u_g) > logw_cur
 * (w_k / w_cur > u_g, the proposal-only term formed first in FP64),
 * u_g = (2*(w>>12)+1)*2^-53, w = word 0 of philox(key=(seed, stream_id),
 * ctr=(g, 0, 0, 2)).  Writes d_chain_idx_out[k] = global index of the state
 * after step g and d_acc_out[k] in {0,1} (each nullable); updates
 * *d_state in place.  d_workspace: >= gf_mh_chain_workspace_bytes(n) bytes
 * of device memory, 8-byte aligned, owned by the caller, free after the
 * call's work on `stream` completes. */
gf_status gf_mh_chain(gf_mh_state* d_state, int64_t n, const double* d_logw,
                      int64_t* d_chain_idx_out, uint8_t* d_acc_out,
                      void* d_workspace, size_t workspace_bytes, cudaStream_t stream);

/* Largest n accepted by gf_mh_chain_noalloc (1 MiB of device scratch). */
#define GF_MH_NOALLOC_MAX_N 131072

/* Same chain as gf_mh_chain, for callers that cannot allocate device memory
 * where they run the chain: for example a serving loop that owns a fixed
 * memory budget handed out by its own allocator, or a latency-critical
 * thread that must not risk the device-wide synchronisation a cudaMalloc can
 * cause.  The paper has no counterpart; this is an interface convenience.
 *
 * The per-proposal scratch (one 8-byte key per proposal) lives in a fixed
 * device array inside the library (GF_MH_NOALLOC_MAX_N entries = 1 MiB,
 * held on every device that loads the library until the process exits).  The caller still passes the state,
 * log weights and outputs (same meaning as for gf_mh_chain).  No memory is
 * allocated.  Every call made outside stream capture looks up the array's
 * device address (cudaGetSymbolAddress) with that device current, so a device
 * reset or a new primary context is followed; a call being captured into a
 * graph reuses the last address, so make one call on the device before
 * capturing.  n > GF_MH_NOALLOC_MAX_N returns GF_EINVAL.
 * Every call on a device shares the one array and leaves its contents
 * behind; each call writes every entry it reads before reading it, so
 * nothing needs clearing, but calls that overlap on the GPU (different
 * streams, no ordering between them) race on it and must not be issued. */
gf_status gf_mh_chain_noalloc(gf_mh_state* d_state, int64_t n, const double* d_logw,
                              int64_t* d_chain_idx_out, uint8_t* d_acc_out,
                              cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* HMC comparison sampler (paper Sec. 2.2: HMC for the same theory)        */
/* ---------------------------------------------------------------------- */

/* One trajectory per chain, FP64.  H = 1/2 sum pi^2 + S; momenta from
 * philox(key=(seed,0), ctr=(chain, traj_index, j, 3)) (FP64 Box-Muller);
 * leapfrog: half kick, n_steps x (drift eps, kick eps) with the last kick
 * halved; accept iff -dH > log u, u from ctr=(chain, traj_index, 0, 4).
 * d_phi [n_chains][V] is updated in place (restored on reject);
 * d_dH_out, d_acc_out nullable.  Supported: V <= 4096. */
gf_status gf_hmc_trajectory(int32_t nd, int32_t L, const gf_phi4* phi4, int64_t n_chains,
                            double* d_phi, int32_t n_steps, double eps, uint64_t seed,
                            uint64_t traj_index, double* d_dH_out, uint8_t* d_acc_out,
                            cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* Reverse-KL self-training (paper Sec. 1, shifted reverse KL divergence;  */
/* Sec. 3, training loop with Adam)                                        */
/* ---------------------------------------------------------------------- */

/* Bytes of device workspace gf_flow_train_step needs for batch B. */
size_t gf_train_workspace_bytes(const gf_flow* flow, int64_t B);

/* loss = (1/B) sum_b [log q(phi_b) + S(phi_b)], phi_b = F^{-1}(z_b), z_b as
 * in gf_flow_sample.  Writes *d_loss_out (FP64 device scalar) and, when
 * d_grad_out != NULL, dloss/dtheta in canonical order (FP32 [n_params]).
 * When lr > 0 also applies one Adam step (Kingma & Ba; bias-corrected,
 * 1-based step adam_t) to the flow's weights using the caller's FP32 moment
 * buffers d_adam_m, d_adam_v [n_params].  d_workspace as for gf_mh_chain. */
gf_status gf_flow_train_step(gf_flow* flow, const gf_phi4* phi4, int64_t B, uint64_t seed,
                             uint64_t counter0, const float* d_z_in, double* d_loss_out,
                             float* d_grad_out, float lr, float beta1, float beta2,
                             float adam_eps, float* d_adam_m, float* d_adam_v,
                             int64_t adam_t, void* d_workspace, size_t workspace_bytes,
                             cudaStream_t stream);

/* One Adam step (Kingma & Ba; bias-corrected, 1-based step adam_t) on the
 * flow's weights with a gradient supplied by the caller: d_grad [n_params]
 * FP32 in canonical order (for example the average over data-parallel ranks
 * of gf_flow_train_step's gradients, or gf_flow_backward's), moments
 * d_adam_m, d_adam_v [n_params] FP32 updated in place.  The same update
 * gf_flow_train_step applies when lr > 0 (Sec. 3: opt = Adam).  Any flow,
 * including general networks. */
gf_status gf_flow_adam_step(gf_flow* flow, const float* d_grad, float lr, float beta1, float beta2,
                            float adam_eps, float* d_adam_m, float* d_adam_v, int64_t adam_t,
                            cudaStream_t stream);

/* The training step in two halves, for a loss assembled by the caller
 * (e.g. through torch.autograd).  Both take the workspace of
 * gf_train_workspace_bytes(flow, B).
 *
 * Forward half: phi_b = F^{-1}(z_b) and log q(phi_b) = log r(z_b) - log det
 * (Sec. 1), z_b as in gf_flow_sample.  Writes d_phi_out [B][V] FP32 and
 * d_logq_out [B] FP64, and keeps every layer's input in the workspace. */
gf_status gf_flow_forward_train(const gf_flow* flow, int64_t B, uint64_t seed, uint64_t counter0,
                                const float* d_z_in, float* d_phi_out, double* d_logq_out,
                                void* d_workspace, size_t workspace_bytes, cudaStream_t stream);
/* Backward half: given dLoss/dphi (d_gphi [B][V] FP32, NULL = 0) and
 * dLoss/dlog q (d_glogq [B] FP64, NULL = 0), writes dLoss/dtheta to
 * d_grad_out [n_params] FP32 in canonical order.  The workspace must hold the
 * state left by the latest gf_flow_forward_train with the same B and the
 * same weights; it is overwritten (a second backward needs a new forward).
 * With d_gphi = dS/dphi / B and d_glogq = 1/B it equals the gradient of
 * gf_flow_train_step up to FP32 rounding order. */
gf_status gf_flow_backward(const gf_flow* flow, int64_t B, const float* d_gphi, const double* d_glogq,
                           float* d_grad_out, void* d_workspace, size_t workspace_bytes,
                           cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* Observables of the chain (Sec. 1: expectation values as chain averages, */
/* the autocorrelation time tau_ac and N_indep = N_conf / (2 tau_ac);      */
/* Sec. 3: condensate, zero-momentum two-point function, ESS)              */
/* ---------------------------------------------------------------------- */

#define GF_OBS_MAX_L 4096

/* Per configuration of d_phi [B][L^nd] FP32: d_M_out[b] = (1/V) sum_n
 * phi_b(n) (the magnetisation; the condensate is the chain average of |M|)
 * and d_C_out[b][t], t < L: (1/V) sum_tau Phi_b(tau) Phi_b(tau + t mod L),
 * Phi_b(tau) = sum of phi_b over the sites whose outermost coordinate (y in
 * 2D, z in 3D) is tau -- the zero-momentum two-point function of one
 * configuration.  FP64 outputs; either may be NULL (not both).  L <=
 * GF_OBS_MAX_L. */
gf_status gf_observables(int32_t nd, int32_t L, int64_t B, const float* d_phi, double* d_M_out,
                         double* d_C_out, cudaStream_t stream);

/* The chain's series of a per-proposal observable: d_out[k][j] =
 * d_values[(d_chain_idx[k] - idx0) * width + j] for k < n, j < width, where
 * d_chain_idx is gf_mh_chain's output and row r of d_values belongs to
 * proposal idx0 + r (n_values rows).  An index outside the rows writes NaN
 * and records GF_EINVAL in the device status word. */
gf_status gf_chain_gather(int64_t n, const int64_t* d_chain_idx, int64_t idx0, int64_t n_values,
                          const double* d_values, int32_t width, double* d_out, cudaStream_t stream);

/* Autocorrelation of the series d_y [n] FP64: d_gamma_out[t] = 1/(n-t)
 * sum_{k<n-t} (y_k - ybar)(y_{k+t} - ybar) for t = 0..t_max (t_max < n),
 * and d_tau_out[4] = {tau_int, W, error, ybar}: tau_int = 1/2 +
 * sum_{t=1}^{W} Gamma(t)/Gamma(0) with the automatic window of Madras and
 * Sokal (the smallest W >= 1 with W >= c_window * tau_int(W), else t_max),
 * error = tau_int sqrt((4W+2)/n).  A constant series gives {1/2, 0, 0, y0}.
 * N_indep = n / (2 tau_int). */
gf_status gf_autocorr(int64_t n, const double* d_y, int32_t t_max, double c_window,
                      double* d_gamma_out, double* d_tau_out, cudaStream_t stream);

/* Effective sample size fraction of the importance weights w = exp(logw)
 * of d_logw [n]: *d_ess_out = (sum w)^2 / (n sum w^2), 0 when n == 0 or all
 * weights vanish.  FP64. */
gf_status gf_ess(int64_t n, const double* d_logw, double* d_ess_out, cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* Measurement (no counterpart in the paper: the roofline denominators of   */
/* this library's FP32 and FP64 kernels)                                   */
/* ---------------------------------------------------------------------- */

/* Measured multiply-add throughput of the current device: kind 0 = FP32
 * FFMA, 1 = FP64 DFMA, 2 = packed FP32x2 FMA (fma.rn.f32x2), 2 FLOP per
 * FP32/FP64 multiply-add, from eight independent multiply-add chains per
 * thread on 4 x 256 threads per SM for `iters` iterations, timed with CUDA
 * events on `stream` (synchronises it).  *flops_per_s_out in FLOP/s.
 * iters < 8 or another kind returns GF_EINVAL. */
gf_status gf_alu_peak(int32_t kind, int64_t iters, double* flops_per_s_out, cudaStream_t stream);

/* ---------------------------------------------------------------------- */
/* Status                                                                  */
/* ---------------------------------------------------------------------- */

/* Test hook for the failure path of the tensor-core kernels (the bounded
 * mbarrier waits between their roles; both GF_PREC_BF16CONV_FP64RED kernels).
 * spins > 0: in launches made after the call (process-wide), each block's (or
 * block half's) first conv2 issuer, before its first MMA, waits up to `spins`
 * polls for a barrier completion that never comes; the wait then gives up as
 * any pipeline wait does when its limit runs out: it records GF_ETIMEOUT in
 * the device status word and raises the block's abort flag; every other role
 * leaves its loops, the block waits for its queued tensor-core work and weight
 * copies, frees its tensor memory and returns.  The outputs of such a launch are undefined.  spins = 0 turns the
 * hook off; spins < 0 or above 2^21 returns GF_EINVAL.  Not for production
 * use. */
gf_status gf_set_bf16_stall_test(int64_t spins);

/* Returns in *status_out the status word that kernels launched on `stream`
 * record errors in (0 = no error, else a negative gf_status) and clears it:
 * after the work already queued on `stream`, one atomic exchange on the device
 * reads and zeroes it, then the call waits for `stream`.  Without a slot set
 * for `stream` (gf_set_stream_status_slot) the word is process-wide: it holds
 * the first error of any kernel of this library on any stream since it was
 * last cleared, so with work in flight on several streams an error cannot be
 * attributed to one of them (use per-stream slots for that). */
gf_status gf_device_status(cudaStream_t stream, int32_t* status_out);
/* Per-stream error attribution (for example one stream per request in a
 * serving loop): kernels launched on `stream` after this call record their
 * device-detected errors (first error wins) in *d_slot -- 4 bytes of device
 * memory owned by the caller, zeroed by the caller, alive while associated --
 * instead of the process-wide word, and gf_device_status(stream) reads and
 * clears that slot.  d_slot = NULL removes the association.  Host-side only;
 * thread-safe. */
gf_status gf_set_stream_status_slot(cudaStream_t stream, int32_t* d_slot);
/* Human-readable name of a status code (static string). */
const char* gf_status_string(int32_t status);

#ifdef __cplusplus
}
#endif
#endif /* GFFLOW_H */
