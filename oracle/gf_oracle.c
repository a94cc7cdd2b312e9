/*
 * gf_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see
 * gf_oracle.h for the scope and the paper sections each routine follows).
 *
 * Deliberately slow and literal: direct periodic cross-correlation with a
 * neighbour table, the action with both neighbour terms, a serial MH loop and
 * a textbook leapfrog.  OpenMP (when enabled) only splits independent
 * configurations / chains across threads.
 */
#include "gf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon et al., SC'11): two 64x64->128 multiplies per round,
 * Weyl key schedule, ten rounds.                                            */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL
#define PHILOX_W1 0xBB67AE8584CAA73BULL

void gfo_philox4x64_10(const uint64_t key[2], const uint64_t ctr[4], uint64_t out[4]) {
    uint64_t k0 = key[0], k1 = key[1];
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Stream tags in the last counter word (reading: the paper does not specify
 * its generator; each random purpose gets its own counter sub-space). */
enum { TAG_PRIOR = 1, TAG_MH = 2, TAG_HMC_P = 3, TAG_HMC_U = 4, TAG_Z_JITTER = 5 };

/* Uniform in (0,1) with 23 random bits: (2k+1) * 2^-24, exact in fp32. */
static double u24(uint64_t w) { return (double)(2 * (w >> 41) + 1) * 0x1p-24; }
/* Uniform in (0,1) with 52 random bits: (2k+1) * 2^-53, exact in fp64. */
static double u53(uint64_t w) { return (double)(2 * (w >> 12) + 1) * 0x1p-53; }

static const double TWO_PI = 6.283185307179586476925286766559;

void gfo_prior(int64_t V, int64_t B, uint64_t seed, uint64_t counter0, int32_t f32, double* z) {
    /* Sites 4j..4j+3 of configuration b use philox(key=(seed,0),
     * ctr=(counter0+b, j, 0, TAG_PRIOR)); words (0,1) and (2,3) feed two
     * Box-Muller pairs (cos, sin) in that order. */
    for (int64_t b = 0; b < B; ++b) {
        for (int64_t j = 0; 4 * j < V; ++j) {
            uint64_t key[2] = {seed, 0};
            uint64_t ctr[4] = {counter0 + (uint64_t)b, (uint64_t)j, 0, TAG_PRIOR};
            uint64_t w[4];
            gfo_philox4x64_10(key, ctr, w);
            double zz[4];
            for (int p = 0; p < 2; ++p) {
                double r = sqrt(-2.0 * log(u24(w[2 * p])));
                double th = TWO_PI * u24(w[2 * p + 1]);
                zz[2 * p] = r * cos(th);
                zz[2 * p + 1] = r * sin(th);
            }
            for (int q = 0; q < 4 && 4 * j + q < V; ++q) {
                double v = zz[q];
                if (f32) v = (double)(float)v;
                z[b * V + 4 * j + q] = v;
            }
        }
    }
}

void gfo_log_prior(int64_t V, int64_t B, const double* z, double* logr) {
    for (int64_t b = 0; b < B; ++b) {
        double s = 0.0;
        for (int64_t n = 0; n < V; ++n) s += z[b * V + n] * z[b * V + n];
        logr[b] = -0.5 * s - 0.5 * (double)V * log(TWO_PI);
    }
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry: site index n = x + L*(y + L*z) (x fastest).            */
/* ------------------------------------------------------------------------ */
static int64_t ipow(int64_t a, int e) { int64_t r = 1; while (e--) r *= a; return r; }

static void coords(int nd, int L, int64_t n, int c[3]) {
    c[0] = c[1] = c[2] = 0;
    for (int a = 0; a < nd; ++a) { c[a] = (int)(n % L); n /= L; }   /* c[0]=x, c[1]=y, c[2]=z */
}
static int64_t site(int nd, int L, const int c[3]) {
    int64_t n = 0;
    for (int a = nd - 1; a >= 0; --a) n = n * L + (((c[a] % L) + L) % L);
    return n;
}
static int parity(int nd, int L, int64_t n) {
    int c[3]; coords(nd, L, n, c);
    return (c[0] + c[1] + c[2]) & 1;
}
/* nbr[n*T + t] = index of n + delta(t) for a K^nd-tap stencil; taps ordered
 * (kz,ky,kx) / (ky,kx) with kx fastest, delta = k - (K-1)/2 along each axis. */
static int64_t* make_nbr(int nd, int L, int K) {
    int64_t V = ipow(L, nd); int T = (int)ipow(K, nd);
    const int h = (K - 1) / 2;
    int64_t* nbr = (int64_t*)malloc(sizeof(int64_t) * V * T);
    for (int64_t n = 0; n < V; ++n) {
        int c[3]; coords(nd, L, n, c);
        for (int t = 0; t < T; ++t) {
            int k[3] = {0, 0, 0}; int tt = t;
            for (int a = 0; a < nd; ++a) { k[a] = tt % K; tt /= K; } /* k[0]=kx (fastest) */
            int d[3] = {c[0] + k[0] - h, c[1] + k[1] - h, c[2] + k[2] - h};
            nbr[n * T + t] = site(nd, L, d);
        }
    }
    return nbr;
}

/* phi^4 action (Sec. 1): S = sum_n [ -phi(n) Lap phi(n) + m2 phi^2 + lam phi^4 ],
 * Lap phi(n) = sum_mu [phi(n+mu) + phi(n-mu) - 2 phi(n)], periodic.
 * Reading: the printed summand phi(n_o) d^2 phi(n_o) uses the summation index n. */
static double action_one(int nd, int L, double m2, double lam, const double* phi) {
    int64_t V = ipow(L, nd);
    double S = 0.0;
    for (int64_t n = 0; n < V; ++n) {
        int c[3]; coords(nd, L, n, c);
        double p = phi[n], lap = 0.0;
        for (int mu = 0; mu < nd; ++mu) {
            int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
            cp[mu] += 1; cm[mu] -= 1;
            lap += phi[site(nd, L, cp)] + phi[site(nd, L, cm)] - 2.0 * p;
        }
        S += -p * lap + m2 * p * p + lam * p * p * p * p;
    }
    return S;
}

void gfo_action(int32_t nd, int32_t L, double m2, double lam, int64_t B, const double* phi, double* S) {
    int64_t V = ipow(L, nd);
    for (int64_t b = 0; b < B; ++b) S[b] = action_one(nd, L, m2, lam, phi + b * V);
}

/* dS/dphi(n) = 2 sum_mu (2 phi(n) - phi(n+mu) - phi(n-mu)) + 2 m2 phi + 4 lam phi^3 */
static void force_one(int nd, int L, double m2, double lam, const double* phi, double* F) {
    int64_t V = ipow(L, nd);
    for (int64_t n = 0; n < V; ++n) {
        int c[3]; coords(nd, L, n, c);
        double p = phi[n], k = 0.0;
        for (int mu = 0; mu < nd; ++mu) {
            int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
            cp[mu] += 1; cm[mu] -= 1;
            k += 2.0 * p - phi[site(nd, L, cp)] - phi[site(nd, L, cm)];
        }
        F[n] = 2.0 * k + 2.0 * m2 * p + 4.0 * lam * p * p * p;
    }
}

void gfo_force(int32_t nd, int32_t L, double m2, double lam, int64_t B, const double* phi, double* F) {
    int64_t V = ipow(L, nd);
    for (int64_t b = 0; b < B; ++b) force_one(nd, L, m2, lam, phi + b * V, F + b * V);
}

/* ------------------------------------------------------------------------ */
/* Coupling network (Sec. 1: s, t are the output of a convolutional network */
/* of the fixed sites; Sec. 3: hidden_sizes, kernel_size, inC = 1, outC = 2): */
/* conv 0 .. conv n_hidden, periodic K^nd cross-correlation                  */
/* out[n][o] = b[o] + sum_{i,t} W[o][i][t] in[nbr(n,t)][i].                  */
/* ------------------------------------------------------------------------ */
static double bf16_round(double x) {
    /* Round to the nearest value with 8 significant bits, ties to even. */
    if (x == 0.0 || !isfinite(x)) return x;
    int e; double m = frexp(x, &e);               /* x = m * 2^e, 0.5 <= |m| < 1 */
    double r = nearbyint(ldexp(m, 8));            /* default mode: ties to even */
    return ldexp(r, e - 8);
}

/* Round to the nearest IEEE binary16 value, ties to even: 11 significant bits
 * for |x| >= 2^-14, multiples of 2^-24 below (subnormals), infinity from
 * 65520 (half-way between the largest finite value 65504 and 2^16) up. */
static double f16_round(double x) {
    if (x == 0.0 || !isfinite(x)) return x;
    if (fabs(x) >= 65520.0) return copysign(INFINITY, x);
    int e; frexp(x, &e);                          /* |x| in [2^(e-1), 2^e) */
    int q = e - 11;                               /* quantum of 11 significant bits */
    if (q < -24) q = -24;
    return ldexp(nearbyint(ldexp(x, -q)), q);     /* default mode: ties to even */
}

static double lrelu(double v, double a) { return v > 0.0 ? v : a * v; }

static int n_taps(const gfo_shape* sh) { return (int)ipow(sh->ksize, sh->nd); }
/* input / output channels of convolution j (0 .. n_hidden) */
static int conv_cin(const gfo_shape* sh, int j) { return j == 0 ? 1 : sh->hidden[j - 1]; }
static int conv_cout(const gfo_shape* sh, int j) { return j == sh->n_hidden ? 2 : sh->hidden[j]; }

/* Canonical per-layer block: for j = 0..n_hidden, W_j[cout][cin][T] then b_j[cout]. */
typedef struct {
    const double* W[GFO_MAX_HIDDEN + 1];
    const double* b[GFO_MAX_HIDDEN + 1];
} layer_w;

static int64_t layer_size(const gfo_shape* sh) {
    int64_t T = n_taps(sh), n = 0;
    for (int j = 0; j <= sh->n_hidden; ++j)
        n += (int64_t)conv_cout(sh, j) * conv_cin(sh, j) * T + conv_cout(sh, j);
    return n;
}

static layer_w layer_ptrs(const gfo_shape* sh, const double* w, int layer) {
    int64_t T = n_taps(sh);
    const double* p = w + layer * layer_size(sh);
    layer_w lw;
    for (int j = 0; j <= sh->n_hidden; ++j) {
        lw.W[j] = p; p += (int64_t)conv_cout(sh, j) * conv_cin(sh, j) * T;
        lw.b[j] = p; p += conv_cout(sh, j);
    }
    return lw;
}

/* Periodic cross-correlation: in [V][Cin] -> out [V][Cout], W [Cout][Cin][T].
 * f32acc: the sum is carried in FP32 (GFO_F32_ACC), else in FP64. */
static void conv(int64_t V, int T, const int64_t* nbr, int Cin, int Cout,
                 const double* W, const double* b, int round_w, int f32acc,
                 const double* in, double* out) {
    /* bf16 weights: every weight rounded once up front (the same values the
     * products below would see if each were rounded where it is read) */
    const int64_t nw = (int64_t)Cout * Cin * T;
    double* Wr = NULL;
    if (round_w) {                    /* 1: bf16, 2: FP16 */
        Wr = (double*)malloc(sizeof(double) * (nw > 0 ? nw : 1));
        for (int64_t k = 0; k < nw; ++k) Wr[k] = round_w == 2 ? f16_round(W[k]) : bf16_round(W[k]);
        W = Wr;
    }
    for (int64_t n = 0; n < V; ++n) {
        for (int o = 0; o < Cout; ++o) {
            double acc = b[o];
            float facc = (float)b[o];
            for (int i = 0; i < Cin; ++i) {
                for (int t = 0; t < T; ++t) {
                    const double wv = W[((int64_t)o * Cin + i) * T + t];
                    const double prod = wv * in[nbr[n * T + t] * Cin + i];
                    if (f32acc) facc = facc + (float)prod;
                    else acc += prod;
                }
            }
            out[n * Cout + o] = f32acc ? (double)facc : acc;
        }
    }
    free(Wr);
}

/* Network intermediates of one layer on one configuration: for hidden
 * convolution j, pre[j] = its output before the activation, post[j] = after. */
typedef struct {
    double *yin, *spre, *s, *t;
    double *pre[GFO_MAX_HIDDEN], *post[GFO_MAX_HIDDEN];
} net_buf;

static net_buf net_alloc(const gfo_shape* sh, int64_t V) {
    net_buf nb;
    nb.yin = (double*)malloc(sizeof(double) * V);
    for (int j = 0; j < sh->n_hidden; ++j) {
        nb.pre[j] = (double*)malloc(sizeof(double) * V * sh->hidden[j]);
        nb.post[j] = (double*)malloc(sizeof(double) * V * sh->hidden[j]);
    }
    nb.spre = (double*)malloc(sizeof(double) * V * 2);
    nb.s = (double*)malloc(sizeof(double) * V);
    nb.t = (double*)malloc(sizeof(double) * V);
    return nb;
}
static void net_free(const gfo_shape* sh, net_buf* nb) {
    free(nb->yin);
    for (int j = 0; j < sh->n_hidden; ++j) { free(nb->pre[j]); free(nb->post[j]); }
    free(nb->spre); free(nb->s); free(nb->t);
}

/* s, t = net(y) where y is the layer input with its updated (active) sites zeroed.
 * Readings: LeakyReLU after every hidden convolution, none after the head;
 * tanh on channel 0 (s) only when use_final_tanh; channel 1 is t. */
static void net_forward(const gfo_shape* sh, layer_w lw, int32_t bf16, int64_t V, int T,
                        const int64_t* nbr, const double* y, net_buf* nb) {
    if (bf16 & (GFO_BF16_X1 | GFO_F16_X1)) {  /* the tensor-core mode's conv1 reads a rounded field */
        for (int64_t n = 0; n < V; ++n) nb->yin[n] = (bf16 & GFO_F16_X1) ? f16_round(y[n]) : bf16_round(y[n]);
        y = nb->yin;
    }
    const int f32acc = (bf16 & GFO_F32_ACC) != 0;
    const double* in = y;
    for (int j = 0; j <= sh->n_hidden; ++j) {
        const int cin = conv_cin(sh, j), cout = conv_cout(sh, j);
        const int head = j == sh->n_hidden;
        const int round_w = head ? ((bf16 & GFO_F16_W3) ? 2 : (bf16 & GFO_BF16_W3) ? 1 : 0)
                          : j == 0 ? ((bf16 & GFO_F16_W1) ? 2 : (bf16 & GFO_BF16_W1) ? 1 : 0)
                                   : ((bf16 & GFO_BF16_W2) ? 1 : 0);
        double* out = head ? nb->spre : nb->pre[j];
        conv(V, T, nbr, cin, cout, lw.W[j], lw.b[j], round_w, f32acc, in, out);
        if (head) break;
        const int round_h = j == 0 ? ((bf16 & GFO_BF16_H1) ? 1 : 0)
                                   : ((bf16 & GFO_F16_H2) ? 2 : (bf16 & GFO_BF16_H2) ? 1 : 0);
        for (int64_t k = 0; k < V * cout; ++k) {
            nb->post[j][k] = lrelu(nb->pre[j][k], sh->leaky_slope);
            if (round_h == 1) nb->post[j][k] = bf16_round(nb->post[j][k]);
            else if (round_h == 2) nb->post[j][k] = f16_round(nb->post[j][k]);
        }
        in = nb->post[j];
    }
    for (int64_t n = 0; n < V; ++n) {
        nb->s[n] = sh->use_final_tanh ? tanh(nb->spre[2 * n]) : nb->spre[2 * n];
        nb->t[n] = nb->spre[2 * n + 1];
    }
}

static int shape_ok(const gfo_shape* sh) {
    if (!sh || (sh->nd != 2 && sh->nd != 3) || sh->L < 1 || sh->n_layers < 0) return 0;
    if (sh->n_hidden < 0 || sh->n_hidden > GFO_MAX_HIDDEN) return 0;
    if (sh->ksize < 1 || (sh->ksize & 1) == 0) return 0;
    for (int j = 0; j < sh->n_hidden; ++j) if (sh->hidden[j] < 1) return 0;
    return 1;
}

int gfo_coupling_net(const gfo_shape* sh, const double* w, int32_t layer, int32_t bf16_mask,
                     const double* y, double* s, double* t) {
    if (!shape_ok(sh) || layer < 0 || layer >= sh->n_layers) return -1;
    int64_t V = ipow(sh->L, sh->nd); int T = n_taps(sh);
    int64_t* nbr = make_nbr(sh->nd, sh->L, sh->ksize);
    net_buf nb = net_alloc(sh, V);
    net_forward(sh, layer_ptrs(sh, w, layer), bf16_mask, V, T, nbr, y, &nb);
    memcpy(s, nb.s, sizeof(double) * V);
    memcpy(t, nb.t, sizeof(double) * V);
    net_free(sh, &nb); free(nbr);
    return 0;
}

/* Sampling direction for one configuration (Sec. 1, coupling layer and its
 * composition).  Reading: layer l (0-based, in application order) keeps the
 * sites with parity (x+y+z) mod 2 == l mod 2 fixed and maps the others by
 * x -> x * exp(s) + t, s and t computed from the fixed sites only; the
 * log-det of dphi/dz is the sum of s over the updated sites. */
static void sample_one(const gfo_shape* sh, const double* w, int32_t bf16, int64_t V, int T,
                       const int64_t* nbr, const int* par, const double* z, double* x,
                       double* logdet_out, net_buf* nb, double* y) {
    memcpy(x, z, sizeof(double) * V);
    double logdet = 0.0;
    for (int l = 0; l < sh->n_layers; ++l) {
        int frozen = l & 1;
        for (int64_t n = 0; n < V; ++n) y[n] = (par[n] == frozen) ? x[n] : 0.0;
        net_forward(sh, layer_ptrs(sh, w, l), bf16, V, T, nbr, y, nb);
        for (int64_t n = 0; n < V; ++n) {
            if (par[n] != frozen) {
                x[n] = x[n] * exp(nb->s[n]) + nb->t[n];
                if (bf16 & GFO_F32_ACC) x[n] = (double)(float)x[n];
                logdet += nb->s[n];
            }
        }
    }
    *logdet_out = logdet;
}

int gfo_flow_sample(const gfo_shape* sh, const double* w, int32_t bf16_mask, double m2, double lam,
                    int64_t B, uint64_t seed, uint64_t counter0, const double* z_in,
                    double* z_out, double* phi_out, double* logq_out, double* S_out,
                    double* logw_out, int32_t nthreads) {
    if (!shape_ok(sh) || B < 0 || !phi_out || !logq_out) return -1;
    int64_t V = ipow(sh->L, sh->nd); int T = n_taps(sh);
    int64_t* nbr = make_nbr(sh->nd, sh->L, sh->ksize);
    int* par = (int*)malloc(sizeof(int) * V);
    for (int64_t n = 0; n < V; ++n) par[n] = parity(sh->nd, sh->L, n);
    double* zall = (double*)malloc(sizeof(double) * (B > 0 ? B : 1) * V);
    if (z_in) memcpy(zall, z_in, sizeof(double) * B * V);
    else {
        gfo_prior(V, B, seed, counter0, 0, zall);
        if (bf16_mask & GFO_Z_JITTER) {         /* tolerance experiment only (see header) */
            for (int64_t b = 0; b < B; ++b)
                for (int64_t n = 0; n < V; ++n) {
                    uint64_t key[2] = {seed, 1};
                    uint64_t ctr[4] = {counter0 + (uint64_t)b, (uint64_t)n, 0, TAG_Z_JITTER};
                    uint64_t w[4];
                    gfo_philox4x64_10(key, ctr, w);
                    const double e = (2.0 * u53(w[0]) - 1.0) * 0x1p-20;
                    zall[b * V + n] *= 1.0 + e;
                }
        }
        if (bf16_mask & GFO_F32_IO)
            for (int64_t k = 0; k < B * V; ++k) zall[k] = (double)(float)zall[k];
    }
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
    {
        net_buf nb = net_alloc(sh, V);
        double* y = (double*)malloc(sizeof(double) * V);
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < B; ++b) {
            const double* z = zall + b * V;
            double* x = phi_out + b * V;
            double logdet, logr, S;
            sample_one(sh, w, bf16_mask, V, T, nbr, par, z, x, &logdet, &nb, y);
            gfo_log_prior(V, 1, z, &logr);
            S = action_one(sh->nd, sh->L, m2, lam, x);
            logq_out[b] = logr - logdet;                 /* log q = log r(z) - log|det dphi/dz| */
            if (S_out) S_out[b] = S;
            if (logw_out) logw_out[b] = -S - logq_out[b]; /* log p - log q, p = exp(-S) unnormalised */
        }
        net_free(sh, &nb); free(y);
    }
    if (z_out) memcpy(z_out, zall, sizeof(double) * B * V);
    free(zall); free(par); free(nbr);
    return 0;
}

int gfo_flow_logq(const gfo_shape* sh, const double* w, int32_t bf16_mask, int64_t B,
                  const double* phi, double* z_out, double* logq_out, int32_t nthreads) {
    if (!shape_ok(sh) || B < 0 || !phi || !logq_out) return -1;
    int64_t V = ipow(sh->L, sh->nd); int T = n_taps(sh);
    int64_t* nbr = make_nbr(sh->nd, sh->L, sh->ksize);
    int* par = (int*)malloc(sizeof(int) * V);
    for (int64_t n = 0; n < V; ++n) par[n] = parity(sh->nd, sh->L, n);
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
    {
        net_buf nb = net_alloc(sh, V);
        double* y = (double*)malloc(sizeof(double) * V);
        double* x = (double*)malloc(sizeof(double) * V);
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < B; ++b) {
            memcpy(x, phi + b * V, sizeof(double) * V);
            double logdet = 0.0, logr;
            /* Layers in reverse order; each inverts x = (x - t) * exp(-s) on its
             * updated sites, with s, t from the fixed sites (unchanged by the layer). */
            for (int l = sh->n_layers - 1; l >= 0; --l) {
                int frozen = l & 1;
                for (int64_t n = 0; n < V; ++n) y[n] = (par[n] == frozen) ? x[n] : 0.0;
                net_forward(sh, layer_ptrs(sh, w, l), bf16_mask, V, T, nbr, y, &nb);
                for (int64_t n = 0; n < V; ++n) {
                    if (par[n] != frozen) {
                        x[n] = (x[n] - nb.t[n]) * exp(-nb.s[n]);
                        logdet += nb.s[n];
                    }
                }
            }
            gfo_log_prior(V, 1, x, &logr);
            logq_out[b] = logr - logdet;
            if (z_out) memcpy(z_out + b * V, x, sizeof(double) * V);
        }
        net_free(sh, &nb); free(y); free(x);
    }
    free(par); free(nbr);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Metropolis-Hastings independence chain (Sec. 1: flow proposals made exact */
/* by the MH test with the Jacobian).  Readings: accept proposal k when      */
/* w_k / w_cur > u_k, evaluated as (log w_k - log u_k) > log w_cur in FP64   */
/* (strict, ties reject; the proposal-only term is formed first), with       */
/* log w = log p - log q = -S - log q; the very first proposal of a chain is */
/* accepted unconditionally; u_k from philox(key=(seed, stream_id),          */
/* ctr=(step, 0, 0, TAG_MH)) word 0.                                         */
/* ------------------------------------------------------------------------ */
void gfo_mh_logu(uint64_t seed, uint64_t stream_id, int64_t step0, int64_t n, double* logu) {
    for (int64_t k = 0; k < n; ++k) {
        uint64_t key[2] = {seed, stream_id};
        uint64_t ctr[4] = {(uint64_t)(step0 + k), 0, 0, TAG_MH};
        uint64_t w[4];
        gfo_philox4x64_10(key, ctr, w);
        logu[k] = log(u53(w[0]));
    }
}

void gfo_mh_scan(gfo_mh_state* st, int64_t n, const double* logw, const double* logu,
                 int64_t* chain_idx, uint8_t* acc) {
    for (int64_t k = 0; k < n; ++k) {
        int64_t g = st->step;
        int a;
        if (g == 0) a = 1;
        else a = (logw[k] - logu[k]) > st->logw_cur;
        if (a) {
            st->logw_cur = logw[k];
            st->idx_cur = g;
            if (g > 0) st->n_acc += 1;
        }
        if (chain_idx) chain_idx[k] = st->idx_cur;
        if (acc) acc[k] = (uint8_t)a;
        st->step = g + 1;
    }
}

void gfo_mh_chain(gfo_mh_state* st, int64_t n, const double* logw, int64_t* chain_idx, uint8_t* acc) {
    double* logu = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
    gfo_mh_logu(st->seed, st->stream_id, st->step, n, logu);
    gfo_mh_scan(st, n, logw, logu, chain_idx, acc);
    free(logu);
}

/* ------------------------------------------------------------------------ */
/* HMC (Sec. 2.2) with H = 1/2 sum pi^2 + S.  Leapfrog: half kick, then       */
/* n_steps x (drift, kick) with the last kick halved; accept iff             */
/* -dH > log u.  Momenta: FP64 Box-Muller from philox(key=(seed,0),          */
/* ctr=(chain, traj, j, TAG_HMC_P)); u from ctr=(chain, traj, 0, TAG_HMC_U). */
/* ------------------------------------------------------------------------ */
void gfo_hmc_momenta(int64_t V, uint64_t seed, uint64_t chain, uint64_t traj, double* pi) {
    for (int64_t j = 0; 4 * j < V; ++j) {
        uint64_t key[2] = {seed, 0};
        uint64_t ctr[4] = {chain, traj, (uint64_t)j, TAG_HMC_P};
        uint64_t w[4];
        gfo_philox4x64_10(key, ctr, w);
        double pp[4];
        for (int p = 0; p < 2; ++p) {
            double r = sqrt(-2.0 * log(u53(w[2 * p])));
            double th = TWO_PI * u53(w[2 * p + 1]);
            pp[2 * p] = r * cos(th);
            pp[2 * p + 1] = r * sin(th);
        }
        for (int q = 0; q < 4 && 4 * j + q < V; ++q) pi[4 * j + q] = pp[q];
    }
}

static double kinetic(int64_t V, const double* pi) {
    double k = 0.0;
    for (int64_t n = 0; n < V; ++n) k += 0.5 * pi[n] * pi[n];
    return k;
}

double gfo_leapfrog(int32_t nd, int32_t L, double m2, double lam, double* phi, double* pi,
                    int32_t n_steps, double eps) {
    int64_t V = ipow(L, nd);
    double* F = (double*)malloc(sizeof(double) * V);
    double H0 = kinetic(V, pi) + action_one(nd, L, m2, lam, phi);
    force_one(nd, L, m2, lam, phi, F);
    for (int64_t n = 0; n < V; ++n) pi[n] -= 0.5 * eps * F[n];
    for (int i = 1; i <= n_steps; ++i) {
        for (int64_t n = 0; n < V; ++n) phi[n] += eps * pi[n];
        force_one(nd, L, m2, lam, phi, F);
        double h = (i < n_steps) ? eps : 0.5 * eps;
        for (int64_t n = 0; n < V; ++n) pi[n] -= h * F[n];
    }
    double H1 = kinetic(V, pi) + action_one(nd, L, m2, lam, phi);
    free(F);
    return H1 - H0;
}

void gfo_hmc_trajectory(int32_t nd, int32_t L, double m2, double lam, int64_t n_chains,
                        double* phi, int32_t n_steps, double eps, uint64_t seed,
                        uint64_t traj_index, double* dH_out, uint8_t* acc_out,
                        int32_t nthreads) {
    int64_t V = ipow(L, nd);
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
    {
        double* pi = (double*)malloc(sizeof(double) * V);
        double* old = (double*)malloc(sizeof(double) * V);
#pragma omp for schedule(dynamic, 1)
        for (int64_t c = 0; c < n_chains; ++c) {
            double* p = phi + c * V;
            memcpy(old, p, sizeof(double) * V);
            gfo_hmc_momenta(V, seed, (uint64_t)c, traj_index, pi);
            double dH = gfo_leapfrog(nd, L, m2, lam, p, pi, n_steps, eps);
            uint64_t key[2] = {seed, 0};
            uint64_t ctr[4] = {(uint64_t)c, traj_index, 0, TAG_HMC_U};
            uint64_t w[4];
            gfo_philox4x64_10(key, ctr, w);
            int a = (-dH) > log(u53(w[0]));
            if (!a) memcpy(p, old, sizeof(double) * V);
            if (dH_out) dH_out[c] = dH;
            if (acc_out) acc_out[c] = (uint8_t)a;
        }
        free(pi); free(old);
    }
}

/* ------------------------------------------------------------------------ */
/* Reverse-KL loss and its gradient (Sec. 1, shifted reverse KL divergence):  */
/* L = (1/B) sum_b [log q(phi_b) + S(phi_b)], phi_b = F^{-1}(z_b), z fixed.  */
/* The reverse pass is the chain rule written out by hand, layer by layer.   */
/* ------------------------------------------------------------------------ */

/* Adjoint of out = conv(in): gin += W^T gout (scatter form), gW += gout (x) in, gb += gout. */
static void conv_backward(int64_t V, int T, const int64_t* nbr, int Cin, int Cout,
                          const double* W, const double* in, const double* gout,
                          double* gin, double* gW, double* gb) {
    for (int64_t n = 0; n < V; ++n) {
        for (int o = 0; o < Cout; ++o) {
            double g = gout[n * Cout + o];
            if (g == 0.0) continue;
            gb[o] += g;
            for (int i = 0; i < Cin; ++i) {
                for (int t = 0; t < T; ++t) {
                    int64_t m = nbr[n * T + t];
                    gW[((int64_t)o * Cin + i) * T + t] += g * in[m * Cin + i];
                    if (gin) gin[m * Cin + i] += W[((int64_t)o * Cin + i) * T + t] * g;
                }
            }
        }
    }
}

int gfo_flow_loss_grad(const gfo_shape* sh, const double* w, double m2, double lam, int64_t B,
                       const double* z, double* loss_out, double* grad_out, int32_t nthreads) {
    if (!shape_ok(sh) || B <= 0 || !z || !loss_out || !grad_out) return -1;
    int64_t V = ipow(sh->L, sh->nd); int T = n_taps(sh);
    int64_t P = layer_size(sh) * sh->n_layers;
    int64_t* nbr = make_nbr(sh->nd, sh->L, sh->ksize);
    int* par = (int*)malloc(sizeof(int) * V);
    for (int64_t n = 0; n < V; ++n) par[n] = parity(sh->nd, sh->L, n);
    double* loss_b = (double*)malloc(sizeof(double) * B);
    if (nthreads < 1) nthreads = 1;
    double* gpart = (double*)calloc((size_t)nthreads * P, sizeof(double));
#pragma omp parallel num_threads(nthreads)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* G = gpart + (int64_t)tid * P;
        net_buf nb = net_alloc(sh, V);
        double* xs = (double*)malloc(sizeof(double) * V * (sh->n_layers + 1)); /* x_l, l=0..N */
        double* y = (double*)malloc(sizeof(double) * V);
        double* gx = (double*)malloc(sizeof(double) * V);
        double* gy = (double*)malloc(sizeof(double) * V);
        double* g3 = (double*)malloc(sizeof(double) * V * 2);
        int cmax = 1;
        for (int j = 0; j < sh->n_hidden; ++j) if (sh->hidden[j] > cmax) cmax = sh->hidden[j];
        double* gA = (double*)malloc(sizeof(double) * V * cmax);   /* adjoint of a hidden activation */
        double* gB = (double*)malloc(sizeof(double) * V * cmax);
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < B; ++b) {
            /* forward, keeping each layer input x_l */
            memcpy(xs, z + b * V, sizeof(double) * V);
            double logdet = 0.0;
            for (int l = 0; l < sh->n_layers; ++l) {
                const double* xi = xs + (int64_t)l * V;
                double* xo = xs + (int64_t)(l + 1) * V;
                int frozen = l & 1;
                for (int64_t n = 0; n < V; ++n) y[n] = (par[n] == frozen) ? xi[n] : 0.0;
                net_forward(sh, layer_ptrs(sh, w, l), 0, V, T, nbr, y, &nb);
                for (int64_t n = 0; n < V; ++n) {
                    if (par[n] != frozen) { xo[n] = xi[n] * exp(nb.s[n]) + nb.t[n]; logdet += nb.s[n]; }
                    else xo[n] = xi[n];
                }
            }
            const double* phi = xs + (int64_t)sh->n_layers * V;
            double logr;
            gfo_log_prior(V, 1, z + b * V, &logr);
            loss_b[b] = (logr - logdet) + action_one(sh->nd, sh->L, m2, lam, phi);

            /* reverse pass: dL_b/dphi = force, dL_b/dlogdet = -1 */
            force_one(sh->nd, sh->L, m2, lam, phi, gx);
            for (int l = sh->n_layers - 1; l >= 0; --l) {
                const double* xi = xs + (int64_t)l * V;
                layer_w lw = layer_ptrs(sh, w, l);
                /* gradient blocks of this layer, in the canonical layout */
                double* gW[GFO_MAX_HIDDEN + 1];
                double* gb[GFO_MAX_HIDDEN + 1];
                {
                    double* q = G + (int64_t)l * layer_size(sh);
                    for (int j = 0; j <= sh->n_hidden; ++j) {
                        gW[j] = q; q += (int64_t)conv_cout(sh, j) * conv_cin(sh, j) * T;
                        gb[j] = q; q += conv_cout(sh, j);
                    }
                }
                int frozen = l & 1;
                for (int64_t n = 0; n < V; ++n) y[n] = (par[n] == frozen) ? xi[n] : 0.0;
                net_forward(sh, lw, 0, V, T, nbr, y, &nb);
                for (int64_t n = 0; n < V; ++n) {
                    if (par[n] != frozen) {
                        double e = exp(nb.s[n]);
                        double gs = gx[n] * xi[n] * e - 1.0;     /* d/ds of x*e^s + t, and of -logdet */
                        double gspre = sh->use_final_tanh ? gs * (1.0 - nb.s[n] * nb.s[n]) : gs;
                        g3[2 * n] = gspre;
                        g3[2 * n + 1] = gx[n];                     /* d/dt */
                        gx[n] = gx[n] * e;                          /* d/dx_in at updated sites */
                    } else {
                        g3[2 * n] = 0.0; g3[2 * n + 1] = 0.0;
                    }
                }
                /* back through the convolutions, head first: gout is the adjoint of
                 * convolution j's output (pre-activation), gin that of its input */
                const double* gout = g3;
                for (int j = sh->n_hidden; j >= 0; --j) {
                    const int cin = conv_cin(sh, j), cout = conv_cout(sh, j);
                    const double* in = j == 0 ? y : nb.post[j - 1];
                    double* gin = j == 0 ? gy : (gout == gA ? gB : gA);
                    memset(gin, 0, sizeof(double) * V * cin);
                    conv_backward(V, T, nbr, cin, cout, lw.W[j], in, gout, gin, gW[j], gb[j]);
                    if (j > 0)               /* through the LeakyReLU of hidden j-1 */
                        for (int64_t k = 0; k < V * cin; ++k)
                            gin[k] *= (nb.pre[j - 1][k] > 0.0) ? 1.0 : sh->leaky_slope;
                    gout = gin;
                }
                for (int64_t n = 0; n < V; ++n)
                    if (par[n] == frozen) gx[n] += gy[n];          /* y = x on fixed sites only */
            }
        }
        net_free(sh, &nb); free(xs); free(y); free(gx); free(gy); free(g3); free(gA); free(gB);
    }
    double loss = 0.0;
    for (int64_t b = 0; b < B; ++b) loss += loss_b[b];
    *loss_out = loss / (double)B;
    for (int64_t p = 0; p < P; ++p) {
        double s = 0.0;
        for (int t = 0; t < nthreads; ++t) s += gpart[(int64_t)t * P + p];
        grad_out[p] = s / (double)B;
    }
    free(gpart); free(loss_b); free(par); free(nbr);
    return 0;
}

void gfo_adam(int64_t n, double* theta, const double* g, double* m, double* v, int64_t t,
              double lr, double beta1, double beta2, double eps) {
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        theta[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Observables of the Markov chain (Sec. 1: expectation values as chain     */
/* averages, the autocorrelation time tau_ac with N_indep = N_conf/(2 tau); */
/* Sec. 3: condensate, zero-momentum two-point function, ESS).              */
/* ------------------------------------------------------------------------ */

/* Per configuration b: M[b] = (1/V) sum_n phi(n) and, for t = 0..L-1,
 * C[b][t] = (1/V) sum_tau Phi(tau) Phi(tau + t mod L), where Phi(tau) is the
 * sum of phi over the sites whose outermost coordinate (y in 2D, z in 3D) is
 * tau.  Either output may be NULL. */
void gfo_observables(int32_t nd, int32_t L, int64_t B, const double* phi, double* M, double* C) {
    int64_t V = ipow(L, nd);
    double* Phi = (double*)malloc(sizeof(double) * L);
    for (int64_t b = 0; b < B; ++b) {
        const double* p = phi + b * V;
        double m = 0.0;
        for (int tau = 0; tau < L; ++tau) Phi[tau] = 0.0;
        for (int64_t n = 0; n < V; ++n) {
            int c[3]; coords(nd, L, n, c);
            Phi[c[nd - 1]] += p[n];
            m += p[n];
        }
        if (M) M[b] = m / (double)V;
        if (C) {
            for (int t = 0; t < L; ++t) {
                double acc = 0.0;
                for (int tau = 0; tau < L; ++tau) acc += Phi[tau] * Phi[(tau + t) % L];
                C[b * L + t] = acc / (double)V;
            }
        }
    }
    free(Phi);
}

/* Gamma(t) = 1/(n-t) sum_{k=0}^{n-t-1} (y_k - ybar)(y_{k+t} - ybar) for
 * t = 0..t_max (t_max < n), ybar the mean of y.  Evaluated on d_k = y_k - y_0
 * (the same deviations from the mean), so that a constant series gives
 * exactly zero. */
void gfo_autocorr(int64_t n, const double* y, int32_t t_max, double* gamma) {
    double dbar = 0.0;
    for (int64_t k = 0; k < n; ++k) dbar += y[k] - y[0];
    dbar /= (double)n;
    for (int32_t t = 0; t <= t_max; ++t) {
        double acc = 0.0;
        for (int64_t k = 0; k + t < n; ++k) acc += ((y[k] - y[0]) - dbar) * ((y[k + t] - y[0]) - dbar);
        gamma[t] = acc / (double)(n - t);
    }
}

/* Integrated autocorrelation time with the automatic window of Madras and
 * Sokal: tau(W) = 1/2 + sum_{t=1}^{W} Gamma(t)/Gamma(0); W is the smallest
 * W >= 1 with W >= c * tau(W), else t_max.  out = {tau(W), W, tau(W) *
 * sqrt((4W + 2)/n)} (the last is their error estimate).  A constant series
 * (Gamma(0) = 0) gives {1/2, 0, 0}. */
void gfo_tau_int(int64_t n, const double* gamma, int32_t t_max, double c, double out[3]) {
    if (!(gamma[0] > 0.0)) { out[0] = 0.5; out[1] = 0.0; out[2] = 0.0; return; }
    double tau = 0.5;
    int32_t W = t_max;
    for (int32_t w = 1; w <= t_max; ++w) {
        tau += gamma[w] / gamma[0];
        if ((double)w >= c * tau) { W = w; break; }
    }
    out[0] = tau;
    out[1] = (double)W;
    out[2] = tau * sqrt((4.0 * W + 2.0) / (double)n);
}

/* Effective sample size fraction of importance weights w_k = exp(logw_k):
 * (sum w)^2 / (n sum w^2), evaluated with the largest log w factored out.
 * Returns 0 when n == 0 or every weight is zero. */
double gfo_ess(int64_t n, const double* logw) {
    if (n <= 0) return 0.0;
    double mx = -INFINITY;
    for (int64_t k = 0; k < n; ++k) if (logw[k] > mx) mx = logw[k];
    if (!(mx > -INFINITY)) return 0.0;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        const double w = exp(logw[k] - mx);
        s1 += w;
        s2 += w * w;
    }
    return s1 * s1 / ((double)n * s2);
}
