/*
 * gf_oracle.h -- plain FP64 CPU oracle of the flow-based sampler for lattice
 * phi^4 theory (Tomiya & Terasaki, GomalizingFlow.jl, arXiv:2208.08903).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference arm may call this library.  It shares
 * no source, header, table or helper with the CUDA library and never calls it.
 *
 * Every routine is the direct definition from the paper, in FP64, with plain
 * loops and explicit modular neighbour indexing:
 *   - action S[phi]              : Sec. 1, the phi^4 action and potential V[phi]
 *   - target density exp(-S)/Z   : Sec. 1, the QFT probability density
 *   - prior, iid N(0,1) per site : Sec. 1 (trivial distribution) and Sec. 3
 *                                   (prior = Normal{Float32}(0, 1))
 *   - affine coupling layers     : Sec. 1, the even/odd coupling map and the
 *                                   composition of N_tri layers
 *   - log-det / model density    : Sec. 1, the Jacobian of F^{-1} and P^(ML)
 *   - reverse (shifted) KL loss  : Sec. 1, the shifted reverse KL divergence
 *   - Metropolis-Hastings test   : Sec. 1, the flow proposals corrected by the
 *                                   MH test with the Jacobian
 *   - HMC                        : Sec. 2.2 (HMC for the same theory)
 *   - chain observables          : Sec. 1 (chain averages, tau_ac, N_indep)
 *                                   and Sec. 3 (condensate, zero-momentum
 *                                   two-point function, ESS)
 *
 * Readings where the paper is silent (sign convention, parity order, tap
 * order, activation, uniform construction, MH tie rule, leapfrog form) are
 * listed in the design notes; the ones that fix arithmetic are repeated at the
 * routine that implements them.
 *
 * Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written here from that definition.
 *
 * Parity status: the action, force, PRNG, prior, MH rule, HMC integrator,
 * single coupling layer, layer composition, log-det and loss gradient are
 * pinned by the CPU tests (closed forms, library routines, brute force,
 * invariants).  Flow outputs for random weights have no paper values: they
 * are pinned only through those invariants.
 */
#ifndef GF_ORACLE_H
#define GF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Flow shape (Sec. 3, model parameters n_layers, hidden_sizes, kernel_size,
 * inC = 1, outC = 2, use_final_tanh).  Each coupling layer's net is the chain
 * conv(1 -> hidden[0]) LReLU ... conv(hidden[n_hidden-2] -> hidden[n_hidden-1])
 * LReLU conv(hidden[n_hidden-1] -> 2), every convolution periodic with
 * ksize^nd taps (ksize odd, circular padding (ksize-1)/2).  n_hidden = 0 is a
 * single conv(1 -> 2). */
#define GFO_MAX_HIDDEN 8
typedef struct {
    int32_t nd;            /* 2 or 3 */
    int32_t L;             /* sites per axis */
    int32_t n_layers;
    int32_t n_hidden;      /* number of hidden convolutions, 0..GFO_MAX_HIDDEN */
    int32_t hidden[GFO_MAX_HIDDEN];   /* their output widths */
    int32_t ksize;         /* taps per axis, odd */
    int32_t use_final_tanh;
    double  leaky_slope;   /* LeakyReLU slope after every hidden convolution */
} gfo_shape;

/* Rounding points for the BF16-emulation mode (bit flags, 0 = pure FP64).
 * "conv1" is the first convolution, "conv3" the head (the last), "conv2"
 * every convolution in between; h1 is the first hidden activation, h2 every
 * later one (the names of the two-hidden-layer net). */
enum {
    GFO_BF16_H1 = 1,   /* round h1 (after LeakyReLU) to bf16 */
    GFO_BF16_W2 = 2,   /* round conv2 weights to bf16 */
    GFO_BF16_H2 = 4,   /* round h2 (after LeakyReLU) to bf16 */
    GFO_BF16_W3 = 8,   /* round conv3 (head) weights to bf16 */
    GFO_BF16_W1 = 16,  /* round conv1 weights to bf16 */
    GFO_F32_IO  = 32,  /* round the prior sample z to fp32 (the paper's Float32 prior) */
    GFO_BF16_X1 = 64,  /* round conv1's input (the masked field) to bf16 */
    /* Model of an FP32-accumulating device, used only to measure how far two
     * computations that differ at the FP32 level drift apart through the bf16
     * roundings: every convolution is summed in FP32 (sequentially, bias
     * first, each product rounded to FP32 before it is added) and the field
     * is rounded to FP32 after every affine update.  Sums over the lattice
     * (log-det, z^2, action) stay FP64. */
    GFO_F32_ACC = 128,
    /* With GFO_F32_ACC, for the same experiment: each prior sample drawn in
     * the sampler (not a given z) is multiplied by (1 + e), e uniform in
     * +-2^-20 (the relative bound to which an FP32 Box-Muller prior is tested
     * against this oracle's), from philox(key=(seed, 1), ctr=(counter0+b, n,
     * 0, 5)) word 0, before the FP32 rounding. */
    GFO_Z_JITTER = 256,
    /* FP16 (IEEE binary16, round to nearest even, subnormals kept, overflow to
     * infinity) instead of bf16 at four rounding points: conv1's input and
     * weights, the later hidden activations (h2) and the head's weights (the
     * tensor-core precision mode rounds those to FP16, the dominant
     * convolution's operands h1 and W2 to bf16). */
    GFO_F16_X1 = 512,
    GFO_F16_W1 = 1024,
    GFO_F16_H2 = 2048,
    GFO_F16_W3 = 4096
};

typedef struct {
    double   logw_cur;
    int64_t  idx_cur, n_acc, step;
    uint64_t seed, stream_id;
} gfo_mh_state;

/* Philox4x64-10: out = philox(key, ctr). */
void gfo_philox4x64_10(const uint64_t key[2], const uint64_t ctr[4], uint64_t out[4]);

/* Prior z[b][n], b < B, from (seed, counter0); rounds to fp32 when f32 != 0. */
void gfo_prior(int64_t V, int64_t B, uint64_t seed, uint64_t counter0, int32_t f32, double* z);

/* log r(z) = -1/2 sum z^2 - (V/2) ln(2 pi), per configuration. */
void gfo_log_prior(int64_t V, int64_t B, const double* z, double* logr);

/* phi^4 action and its gradient (force) for B configurations [B][V]. */
void gfo_action(int32_t nd, int32_t L, double m2, double lam, int64_t B, const double* phi, double* S);
void gfo_force(int32_t nd, int32_t L, double m2, double lam, int64_t B, const double* phi, double* F);

/* One coupling network evaluation on a single configuration: given the masked
 * input y[V] of layer `layer`, writes s[V] (after tanh if enabled) and t[V]. */
int gfo_coupling_net(const gfo_shape* sh, const double* w, int32_t layer, int32_t bf16_mask,
                     const double* y, double* s, double* t);

/* Sampling direction: phi = F^{-1}(z).  z_in nullable (then drawn from
 * (seed, counter0)); outputs nullable except phi_out and logq_out. */
int gfo_flow_sample(const gfo_shape* sh, const double* w, int32_t bf16_mask, double m2, double lam,
                    int64_t B, uint64_t seed, uint64_t counter0, const double* z_in,
                    double* z_out, double* phi_out, double* logq_out, double* S_out,
                    double* logw_out, int32_t nthreads);

/* Trivialising direction: z = F(phi) and log q(phi). */
int gfo_flow_logq(const gfo_shape* sh, const double* w, int32_t bf16_mask, int64_t B,
                  const double* phi, double* z_out, double* logq_out, int32_t nthreads);

/* MH: uniforms log u_k for steps step0 .. step0+n-1 of stream (seed, stream_id). */
void gfo_mh_logu(uint64_t seed, uint64_t stream_id, int64_t step0, int64_t n, double* logu);
/* MH decisions given log u: step 0 accepts, step k > 0 accepts iff
 * (logw[k] - logu[k]) > logw_cur (logu[k] is ignored on global step 0). */
void gfo_mh_scan(gfo_mh_state* st, int64_t n, const double* logw, const double* logu,
                 int64_t* chain_idx, uint8_t* acc);
/* MH chain with its own uniforms (gfo_mh_logu + gfo_mh_scan). */
void gfo_mh_chain(gfo_mh_state* st, int64_t n, const double* logw, int64_t* chain_idx, uint8_t* acc);

/* HMC: one trajectory per chain, phi [n_chains][V] updated in place. */
void gfo_hmc_trajectory(int32_t nd, int32_t L, double m2, double lam, int64_t n_chains,
                        double* phi, int32_t n_steps, double eps, uint64_t seed,
                        uint64_t traj_index, double* dH_out, uint8_t* acc_out,
                        int32_t nthreads);
/* Leapfrog only (no momentum draw, no accept): phi, pi updated in place,
 * returns H(end) - H(start).  Used by the reversibility and O(eps^2) pins. */
double gfo_leapfrog(int32_t nd, int32_t L, double m2, double lam, double* phi, double* pi,
                    int32_t n_steps, double eps);
/* Momenta for (chain, traj) as the trajectory routine draws them. */
void gfo_hmc_momenta(int64_t V, uint64_t seed, uint64_t chain, uint64_t traj, double* pi);

/* Reverse-KL loss L = (1/B) sum_b [log q_b + S_b] for given z [B][V] and its
 * gradient w.r.t. every canonical weight (hand-derived reverse pass). */
int gfo_flow_loss_grad(const gfo_shape* sh, const double* w, double m2, double lam, int64_t B,
                       const double* z, double* loss_out, double* grad_out, int32_t nthreads);

/* Adam (Kingma & Ba), in place; t is the 1-based step count. */
void gfo_adam(int64_t n, double* theta, const double* g, double* m, double* v, int64_t t,
              double lr, double beta1, double beta2, double eps);

/* Chain observables (Sec. 1: chain averages and tau_ac; Sec. 3: condensate,
 * zero-momentum two-point function, ESS).  Per configuration:
 * M[b] = mean of phi; C[b][t] = (1/V) sum_tau Phi(tau) Phi(tau+t), Phi(tau) =
 * sum of phi over the slice at outermost coordinate tau.  Outputs nullable. */
void gfo_observables(int32_t nd, int32_t L, int64_t B, const double* phi, double* M, double* C);
/* Gamma(t), t = 0..t_max, of the series y (mean subtracted, 1/(n-t) normalised). */
void gfo_autocorr(int64_t n, const double* y, int32_t t_max, double* gamma);
/* out = {tau_int, W, error}: Madras-Sokal automatic window with constant c. */
void gfo_tau_int(int64_t n, const double* gamma, int32_t t_max, double c, double out[3]);
/* ESS fraction (sum w)^2 / (n sum w^2) of w = exp(logw). */
double gfo_ess(int64_t n, const double* logw);

#ifdef __cplusplus
}
#endif
#endif
