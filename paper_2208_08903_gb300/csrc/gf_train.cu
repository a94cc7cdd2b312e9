// gf_train.cu -- reverse-KL self-training step of the coupling stack.
//
// Paper arXiv:2208.08903 Sec. 1 (shifted reverse Kullback-Leibler divergence
// as the training objective) and Sec. 3 (training loop: sample z from the
// prior, gradient of the loss, Adam update).  Loss per configuration:
// log q(phi) + S(phi) = log r(z) - sum_l sum_{updated} s + S(F^{-1}(z)),
// differentiated by a hand-written reverse pass:
//   forward  : layer-wise batched kernels, saving only each layer's input x_l
//   backward : per layer (last first) recompute h1, h2, s from x_l, then
//              affine adjoint -> conv3^T -> LReLU' -> conv2^T -> LReLU'
//              -> conv1^T onto the fixed sites, and the weight gradients.
// Activations go through HBM in a channel-chunk-major layout,
// [B][C/4][V][4] FP32 (chunk width min(C, 4)), so that lanes working on
// consecutive sites load consecutive 16-byte words; the step is bound by FP32
// FMA throughput and the extra traffic is a few percent of its time.  Weight
// gradients: each CTA accumulates its configurations in registers and
// writes a partial; a second kernel sums the partials in a fixed order
// (deterministic, no atomics).
#include <algorithm>
#include <cstring>

#include "gf_flow.cuh"

namespace gf {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int wrapi(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }
__device__ __forceinline__ float lrelu(float v, float a) { return v > 0.f ? v : a * v; }

template <int ND>
__device__ __forceinline__ void tap_delta(int t, int& ds, int& dy, int& dx) {
    if (ND == 3) { ds = t / 9 - 1; dy = (t / 3) % 3 - 1; dx = t % 3 - 1; }
    else { ds = t / 3 - 1; dy = 0; dx = t % 3 - 1; }
}

// Site n + delta(t) on the periodic lattice (n = x + L*(y + L*z)).
template <int ND>
__device__ __forceinline__ int nbr(int n, int t, int L) {
    int ds, dy, dx;
    tap_delta<ND>(t, ds, dy, dx);
    const int x = n % L;
    if (ND == 3) {
        const int y = (n / L) % L, z = n / (L * L);
        return (wrapi(z + ds, L) * L + wrapi(y + dy, L)) * L + wrapi(x + dx, L);
    }
    const int y = n / L;
    return wrapi(y + ds, L) * L + wrapi(x + dx, L);
}

template <int ND>
__device__ __forceinline__ int parity(int n, int L) {
    const int x = n % L, y = (n / L) % L;
    return (ND == 3 ? (x + y + n / (L * L)) : (x + y)) & 1;
}

// Element (b, n, c) of a C-channel activation tensor: chunk width W = min(C, 4),
// offset ((b * (C / W) + c / W) * V + n) * W + c % W.  This returns the start of
// chunk c / W (c a multiple of W).
__device__ __forceinline__ int64_t chunk_at(int64_t b, int n, int c, int C, int V) {
    const int W = C < 4 ? C : 4;
    return ((b * (C / W) + c / W) * (int64_t)V + n) * W;
}

// ------------------------------------------------------------------ prior
__global__ void k_prior(int V, int64_t B, uint64_t seed, uint64_t counter0, const float* __restrict__ zin,
                        float* __restrict__ z) {
    const int64_t groups = (int64_t)B * ((V + 3) / 4);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = g / ((V + 3) / 4);
        const int j = (int)(g - b * ((V + 3) / 4));
        if (zin) {
            for (int q = 0; q < 4 && 4 * j + q < V; ++q) z[b * V + 4 * j + q] = zin[b * V + 4 * j + q];
            continue;
        }
        const u64x4 w = philox4x64_10(seed, 0ull, u64x4{counter0 + (uint64_t)b, (uint64_t)j, 0ull, TAG_PRIOR});
        float zz[4];
        normals4_f32(w, zz);
        for (int q = 0; q < 4 && 4 * j + q < V; ++q) z[b * V + 4 * j + q] = zz[q];
    }
}

// ------------------------------------------------------------------ generic periodic conv
// out(b, n, co..co+8) = epi( sum_t sum_ci W[t][ci][co] * in'(b, nbr(n,t), ci) )
// in' = in, or in masked to sites of parity `mask` (mask >= 0).
// mode 0: + bias, LeakyReLU.  mode 1: * LReLU'(ref(b, n, co)) (ref = post-activation).
// Warp task = (configuration, 128 sites, 8 output channels); lane owns sites
// lane + 32k (k < 4).  The conv's weights [T][Cin][Cout] are staged in shared
// memory once per CTA (warp-uniform broadcast reads).
struct ConvArgs {
    const float* in; int Cin; int mask;
    const float* W; const float* bias; int Cout;
    float* out; const float* ref; int mode; float slope;
    int L, V; int64_t B;
};

template <int ND, int VEC, bool MASKED>
__global__ void __launch_bounds__(kThreads) k_conv(const ConvArgs a) {
    extern __shared__ __align__(16) float wsm[];
    const int T = ND == 3 ? 27 : 9;
    {
        const int n4 = T * a.Cin * a.Cout / 4;
        for (int i = threadIdx.x; i < n4; i += blockDim.x)
            reinterpret_cast<float4*>(wsm)[i] = __ldg(reinterpret_cast<const float4*>(a.W) + i);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int nblk = (a.V + 127) >> 7, ngrp = a.Cout >> 3;
    const int64_t tasks = a.B * nblk * ngrp;
    const int64_t cstride = (int64_t)a.V * VEC;            // floats between input chunks
    for (int64_t task = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; task < tasks;
         task += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int g = (int)(task % ngrp);
        const int64_t rest = task / ngrp;
        const int blk = (int)(rest % nblk);
        const int64_t b = rest / nblk;
        const int co = g << 3;
        int n[4];
        bool valid[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            n[k] = (blk << 7) + lane + 32 * k;
            valid[k] = n[k] < a.V;
            if (!valid[k]) n[k] = a.V - 1;
        }
        float acc[4][8];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[k][c] = (a.mode == 0) ? __ldg(a.bias + co + c) : 0.f;
        const float* inb = a.in + chunk_at(b, 0, 0, a.Cin, a.V);
        for (int t = 0; t < T; ++t) {
            int m[4];
            float msk[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                m[k] = nbr<ND>(n[k], t, a.L);
                msk[k] = (!MASKED || parity<ND>(m[k], a.L) == a.mask) ? 1.f : 0.f;
            }
            const float* Wt = wsm + t * a.Cin * a.Cout + co;
            for (int c0 = 0; c0 < a.Cin; c0 += VEC) {
                float hv[4][VEC];
                const float* pc = inb + (int64_t)(c0 / VEC) * cstride;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float* p = pc + (int64_t)m[k] * VEC;
                    if (VEC == 4) {
                        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
                        hv[k][0] = v.x; hv[k][VEC > 1 ? 1 : 0] = v.y;
                        hv[k][VEC > 2 ? 2 : 0] = v.z; hv[k][VEC > 3 ? 3 : 0] = v.w;
                    } else if (VEC == 2) {
                        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
                        hv[k][0] = v.x; hv[k][VEC > 1 ? 1 : 0] = v.y;
                    } else {
                        hv[k][0] = __ldg(p);
                    }
                    if constexpr (MASKED) {
#pragma unroll
                        for (int q = 0; q < VEC; ++q) hv[k][q] *= msk[k];
                    }
                }
#pragma unroll
                for (int q = 0; q < VEC; ++q) {
                    const float* wp = Wt + (c0 + q) * a.Cout;
                    const float4 wa = *reinterpret_cast<const float4*>(wp);
                    const float4 wb = *reinterpret_cast<const float4*>(wp + 4);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float h = hv[k][q];
                        acc[k][0] = fmaf(h, wa.x, acc[k][0]); acc[k][1] = fmaf(h, wa.y, acc[k][1]);
                        acc[k][2] = fmaf(h, wa.z, acc[k][2]); acc[k][3] = fmaf(h, wa.w, acc[k][3]);
                        acc[k][4] = fmaf(h, wb.x, acc[k][4]); acc[k][5] = fmaf(h, wb.y, acc[k][5]);
                        acc[k][6] = fmaf(h, wb.z, acc[k][6]); acc[k][7] = fmaf(h, wb.w, acc[k][7]);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!valid[k]) continue;
            float* o0 = a.out + chunk_at(b, n[k], co, a.Cout, a.V);
            float* o1 = a.out + chunk_at(b, n[k], co + 4, a.Cout, a.V);
            float r[8];
            if (a.mode == 0) {
#pragma unroll
                for (int c = 0; c < 8; ++c) r[c] = lrelu(acc[k][c], a.slope);
            } else {
                const float4 q0 = __ldg(reinterpret_cast<const float4*>(a.ref + chunk_at(b, n[k], co, a.Cout, a.V)));
                const float4 q1 = __ldg(reinterpret_cast<const float4*>(a.ref + chunk_at(b, n[k], co + 4, a.Cout, a.V)));
                const float rv[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
                for (int c = 0; c < 8; ++c) r[c] = acc[k][c] * (rv[c] > 0.f ? 1.f : a.slope);
            }
            *reinterpret_cast<float4*>(o0) = make_float4(r[0], r[1], r[2], r[3]);
            *reinterpret_cast<float4*>(o1) = make_float4(r[4], r[5], r[6], r[7]);
        }
    }
}

// ------------------------------------------------------------------ conv3 + affine (forward)
// One CTA per configuration: (s, t) at the updated sites, x_out = x_in*e^s + t
// there, x_out = x_in on fixed sites; s saved for the reverse pass;
// logdet[b] += sum s (FP64, fixed-order block reduction) unless logdet is null.
template <int ND>
__global__ void __launch_bounds__(kThreads) k_couple_fwd(const float* __restrict__ h2, int C2,
                                                        const float* __restrict__ W3, const float* __restrict__ b3,
                                                        int use_tanh, int frozen, int L, int V, int64_t B,
                                                        const float* __restrict__ xin, float* __restrict__ xout,
                                                        float* __restrict__ s_save, double* __restrict__ logdet) {
    __shared__ double red[32];
    const int T = ND == 3 ? 27 : 9;
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        double ld = 0.0;
        for (int n = threadIdx.x; n < V; n += blockDim.x) {
            const float xv = xin[b * V + n];
            if (parity<ND>(n, L) == frozen) { xout[b * V + n] = xv; s_save[b * V + n] = 0.f; continue; }
            float ps = __ldg(b3), pt = __ldg(b3 + 1);
            for (int t = 0; t < T; ++t) {
                const int m = nbr<ND>(n, t, L);
                const float* wp = W3 + (int64_t)t * C2 * 2;
                for (int c = 0; c < C2; c += 4) {
                    const float4 h = __ldg(reinterpret_cast<const float4*>(h2 + chunk_at(b, m, c, C2, V)));
                    const float4 w01 = __ldg(reinterpret_cast<const float4*>(wp + 2 * c));
                    const float4 w23 = __ldg(reinterpret_cast<const float4*>(wp + 2 * c + 4));
                    ps = fmaf(h.x, w01.x, ps); pt = fmaf(h.x, w01.y, pt);
                    ps = fmaf(h.y, w01.z, ps); pt = fmaf(h.y, w01.w, pt);
                    ps = fmaf(h.z, w23.x, ps); pt = fmaf(h.z, w23.y, pt);
                    ps = fmaf(h.w, w23.z, ps); pt = fmaf(h.w, w23.w, pt);
                }
            }
            const float s = use_tanh ? tanhf(ps) : ps;
            xout[b * V + n] = fmaf(xv, expf(s), pt);
            s_save[b * V + n] = s;
            ld += (double)s;
        }
        if (logdet) {                                   // uniform over the block
            const double tot = block_sum(ld, red);
            if (threadIdx.x == 0) logdet[b] += tot;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ affine adjoint
// At updated sites: g3 = (dL/ds_pre, dL/dt), gx <- gx*e^s.  Fixed sites: g3 = 0.
template <int ND>
__global__ void k_couple_bwd(int frozen, int use_tanh, int L, int V, int64_t B, const float* __restrict__ xin,
                             const float* __restrict__ s_save, const double* __restrict__ glq, float glq_const,
                             float* __restrict__ gx, float* __restrict__ g3) {
    const int64_t total = B * (int64_t)V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(i % V);
        float2 o = make_float2(0.f, 0.f);
        if (parity<ND>(n, L) != frozen) {
            const float s = s_save[i], e = expf(s), g = gx[i];
            // d/ds of x*e^s, and of log q = log r - logdet (dLoss/dlog q per configuration)
            const float gq = glq ? (float)glq[i / V] : glq_const;
            const float gs = g * xin[i] * e - gq;
            o.x = use_tanh ? gs * (1.f - s * s) : gs;
            o.y = g;
            gx[i] = g * e;
        }
        reinterpret_cast<float2*>(g3)[i] = o;
    }
}

// ------------------------------------------------------------------ conv1^T onto fixed sites
// gx[b][n] += sum_t sum_c W1b[t][c] * gh1[b][nbr(n,t)][c] at sites of parity `frozen`.
template <int ND>
__global__ void k_conv1_bwd(const float* __restrict__ gh1, int C1, const float* __restrict__ W1b, int frozen,
                            int L, int V, int64_t B, float* __restrict__ gx) {
    const int T = ND == 3 ? 27 : 9;
    const int64_t total = B * (int64_t)V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(i % V);
        if (parity<ND>(n, L) != frozen) continue;
        const int64_t b = i / V;
        float acc = 0.f;
        for (int t = 0; t < T; ++t) {
            const int m = nbr<ND>(n, t, L);
            const float* wp = W1b + (int64_t)t * C1;
            for (int c = 0; c < C1; c += 4) {
                const float4 h = __ldg(reinterpret_cast<const float4*>(gh1 + chunk_at(b, m, c, C1, V)));
                const float4 w = __ldg(reinterpret_cast<const float4*>(wp + c));
                acc = fmaf(h.x, w.x, acc); acc = fmaf(h.y, w.y, acc);
                acc = fmaf(h.z, w.z, acc); acc = fmaf(h.w, w.w, acc);
            }
        }
        gx[i] += acc;
    }
}

// ------------------------------------------------------------------ weight gradients
// partial[cta][t][i][o] = sum over this CTA's configurations and all sites of
//   gout[b][n][o] * in'[b][nbr(n,t)][i];  tap t == T is the bias (in' = 1, i = 0).
// Thread task = (t, IB input channels, OB output channels).
struct WgArgs {
    const float* in; int Cin; int mask;
    const float* gout; int Cout;
    float* partial; int L, V; int64_t B;
};

template <int ND, int IB, int OB>
__global__ void k_wgrad(const WgArgs a, int nsplit) {
    // Thread = (task, split): the nsplit lanes of a task (adjacent lanes of one
    // warp) take every nsplit-th site and are combined by a fixed shuffle tree.
    const int T = ND == 3 ? 27 : 9;
    const int nic = a.Cin / IB, noc = a.Cout / OB;
    const int tasks = (T + 1) * nic * noc;
    const int task = threadIdx.x / nsplit, split = threadIdx.x % nsplit;
    const bool active = task < tasks;
    const int oc = active ? task % noc : 0;
    const int ic = active ? (task / noc) % nic : 0;
    const int t = active ? task / (noc * nic) : 0;
    const bool bias = t == T;
    float acc[IB][OB];
#pragma unroll
    for (int i = 0; i < IB; ++i)
#pragma unroll
        for (int o = 0; o < OB; ++o) acc[i][o] = 0.f;
    if (active && !(bias && ic != 0)) {
        for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
            for (int n = split; n < a.V; n += nsplit) {
                float iv[IB];
                if (bias) {
#pragma unroll
                    for (int i = 0; i < IB; ++i) iv[i] = (i == 0) ? 1.f : 0.f;
                } else {
                    const int m = nbr<ND>(n, t, a.L);
                    const float mk = (a.mask < 0 || parity<ND>(m, a.L) == a.mask) ? 1.f : 0.f;
                    const float* p = a.in + chunk_at(b, m, ic * IB, a.Cin, a.V);
                    if (IB == 4) {
                        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
                        iv[0] = v.x * mk; iv[IB > 1 ? 1 : 0] = v.y * mk;
                        iv[IB > 2 ? 2 : 0] = v.z * mk; iv[IB > 3 ? 3 : 0] = v.w * mk;
                    } else {
                        iv[0] = __ldg(p) * mk;
                    }
                }
                float gv[OB];
                const float* q = a.gout + chunk_at(b, n, oc * OB, a.Cout, a.V);
                if (OB == 8) {
                    const float4 g0 = __ldg(reinterpret_cast<const float4*>(q));
                    const float4 g1 = __ldg(reinterpret_cast<const float4*>(a.gout + chunk_at(b, n, oc * OB + 4, a.Cout, a.V)));
                    gv[0] = g0.x; gv[1 % OB] = g0.y; gv[2 % OB] = g0.z; gv[3 % OB] = g0.w;
                    gv[4 % OB] = g1.x; gv[5 % OB] = g1.y; gv[6 % OB] = g1.z; gv[7 % OB] = g1.w;
                } else {
                    const float2 g0 = __ldg(reinterpret_cast<const float2*>(q));
                    gv[0] = g0.x; gv[1 % OB] = g0.y;
                }
#pragma unroll
                for (int i = 0; i < IB; ++i)
#pragma unroll
                    for (int o = 0; o < OB; ++o) acc[i][o] = fmaf(iv[i], gv[o], acc[i][o]);
            }
        }
    }
    // combine the nsplit lanes of each task (fixed order: deterministic)
    for (int off = 1; off < nsplit; off <<= 1)
#pragma unroll
        for (int i = 0; i < IB; ++i)
#pragma unroll
            for (int o = 0; o < OB; ++o) acc[i][o] += __shfl_xor_sync(0xffffffffu, acc[i][o], off);
    if (active && split == 0) {
        float* P = a.partial + (int64_t)blockIdx.x * (T + 1) * a.Cin * a.Cout;
#pragma unroll
        for (int i = 0; i < IB; ++i)
#pragma unroll
            for (int o = 0; o < OB; ++o)
                P[((int64_t)t * a.Cin + ic * IB + i) * a.Cout + oc * OB + o] = acc[i][o];
    }
}

// Weight gradient of a C -> C convolution (conv2), tiled through shared memory.
// A work unit is G consecutive slices (outermost axis) of one configuration:
// its gout rows and its input rows plus one halo slice on each side are staged
// site-major ([site][C], bank-conflict-free for the 8 input / 8 output chunks a
// warp reads per site), then thread (tap t, input chunk ic, 8 outputs oc)
// accumulates over the unit's sites from shared memory.  Tap t == T is the bias.
template <int ND>
__global__ void __launch_bounds__(1024) k_wgrad_tiled(const WgArgs a, int G) {
    extern __shared__ __align__(16) float sm[];
    const int T = ND == 3 ? 27 : 9;
    const int L = a.L, V = a.V, C = a.Cin, CO = a.Cout;
    const int S = V / L;                                   // sites per slice
    const int nic = C / 4, noc = CO / 8;
    const int tasks = (T + 1) * nic * noc;
    const int task = threadIdx.x;
    const bool active = task < tasks;
    const int oc = active ? task % noc : 0;
    const int ic = active ? (task / noc) % nic : 0;
    const int t = active ? task / (noc * nic) : T;
    const bool bias = t == T;
    int ds = 0, dy = 0, dx = 0;
    if (!bias) tap_delta<ND>(t, ds, dy, dx);
    float* g_s = sm;                                       // [G*S][CO]
    float* x_s = sm + (size_t)G * S * CO;                  // [(G+2)*S][C]
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[i][o] = 0.f;
    const int units_per_cfg = L / G;
    const int64_t units = a.B * units_per_cfg;
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int64_t b = u / units_per_cfg;
        const int s0 = (int)(u % units_per_cfg) * G;
        __syncthreads();
        // stage gout for slices s0 .. s0+G-1 and the input for s0-1 .. s0+G
        for (int e = threadIdx.x; e < G * S * (CO / 4); e += blockDim.x) {
            const int site = e / (CO / 4), c4 = e % (CO / 4);
            const int n = s0 * S + site;
            *reinterpret_cast<float4*>(g_s + (size_t)site * CO + c4 * 4) =
                __ldg(reinterpret_cast<const float4*>(a.gout + chunk_at(b, n, c4 * 4, CO, V)));
        }
        for (int e = threadIdx.x; e < (G + 2) * S * (C / 4); e += blockDim.x) {
            const int site = e / (C / 4), c4 = e % (C / 4);
            const int sl = s0 - 1 + site / S;
            const int n = ((sl % L + L) % L) * S + site % S;
            *reinterpret_cast<float4*>(x_s + (size_t)site * C + c4 * 4) =
                __ldg(reinterpret_cast<const float4*>(a.in + chunk_at(b, n, c4 * 4, C, V)));
        }
        __syncthreads();
        if (active && !(bias && ic != 0)) {
            for (int r = 0; r < G * S; ++r) {
                const int j = r % S, rs = r / S;               // slice offset within the unit, in-slice site
                const float4 g0 = *reinterpret_cast<const float4*>(g_s + (size_t)r * CO + oc * 8);
                const float4 g1 = *reinterpret_cast<const float4*>(g_s + (size_t)r * CO + oc * 8 + 4);
                const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
                float iv[4];
                if (bias) {
                    iv[0] = 1.f; iv[1] = iv[2] = iv[3] = 0.f;
                } else {
                    int j2;
                    if (ND == 3) {
                        const int y = j / L, x = j - y * L;
                        j2 = wrapi(y + dy, L) * L + wrapi(x + dx, L);
                    } else {
                        j2 = wrapi(j + dx, L);
                    }
                    const float4 v = *reinterpret_cast<const float4*>(x_s + (size_t)((rs + 1 + ds) * S + j2) * C + ic * 4);
                    iv[0] = v.x; iv[1] = v.y; iv[2] = v.z; iv[3] = v.w;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int o = 0; o < 8; ++o) acc[i][o] = fmaf(iv[i], gv[o], acc[i][o]);
            }
        }
    }
    if (active) {
        float* P = a.partial + (int64_t)blockIdx.x * (T + 1) * C * CO;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int o = 0; o < 8; ++o)
                P[((int64_t)t * C + ic * 4 + i) * CO + oc * 8 + o] = acc[i][o];
    }
}

// Weight gradient of the two thin convolutions, tiled through shared memory:
// conv3 (C -> 2, unmasked input) and conv1 (1 -> C, input masked to the fixed
// sites).  A work unit is G consecutive slices of one configuration; its gout
// rows and its input rows plus one halo slice on each side are staged in
// shared memory (input [site][Cin], gout [site][Cout]).  conv3: thread = input
// channel ci and row group; conv1: thread = output channel and row group.  A
// thread walks its rows (an x-row of a slice) along x with a sliding window of
// the 3 (2D) or 9 (3D) input rows' values at x-1, x, x+1, so every input value
// is loaded once per row and feeds all taps: per site 1 (2D) or 3 (3D) input
// loads and one gout load feed 18 / 54 (conv3) or 9 / 27 (conv1) FMAs.  The
// row groups' sums are combined in a fixed order in shared memory (the bias is
// tap T); per-CTA partials as k_wgrad.
template <int ND>
__global__ void __launch_bounds__(512) k_wgrad_thin(const WgArgs a, int G) {
    extern __shared__ __align__(16) float sm[];
    constexpr int T = ND == 3 ? 27 : 9, NR = ND == 3 ? 9 : 3;   // taps, input rows per output row
    const int L = a.L, V = a.V, CI = a.Cin, CO = a.Cout;
    const int S = V / L;
    const bool conv3 = CO == 2;                           // else conv1 (CI == 1)
    const int nch = conv3 ? CI : CO;                      // channels one row group covers
    const int ngrp = blockDim.x / nch;
    const int ch = threadIdx.x % nch, grp = threadIdx.x / nch;
    const bool active = grp < ngrp;
    // row pitches: 4 extra floats for 16-byte chunked rows, so the staging
    // stores of consecutive sites fall in distinct bank groups
    const int PI = CI % 4 == 0 ? CI + 4 : CI, PO = CO % 4 == 0 ? CO + 4 : CO;
    float* g_s = sm;                                       // [G*S][PO]
    float* x_s = g_s + (size_t)G * S * PO;                 // [(G+2)*S][PI]
    float* red = sm;                                       // [ngrp][nch][(T+1)*2], after the units
    constexpr int NA = (T + 1) * 2;
    float acc[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) acc[i] = 0.f;
    const int rows_per_slice = ND == 3 ? L : 1;
    const int units_per_cfg = L / G;
    const int64_t units = a.B * units_per_cfg;
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int64_t b = u / units_per_cfg;
        const int s0 = (int)(u % units_per_cfg) * G;
        __syncthreads();
        // staging: 16-byte chunk loads (4 channels of one site) where the
        // channel count allows, consecutive threads on consecutive sites
        if (CO % 4 == 0) {
            const int nc = CO / 4;
            for (int e = threadIdx.x; e < G * S * nc; e += blockDim.x) {
                const int c4 = e / (G * S), site = e % (G * S);
                const float4 v = __ldg(reinterpret_cast<const float4*>(a.gout + chunk_at(b, s0 * S + site, 4 * c4, CO, V)));
                *reinterpret_cast<float4*>(g_s + (size_t)site * PO + 4 * c4) = v;
            }
        } else {
            for (int e = threadIdx.x; e < G * S * CO; e += blockDim.x) {
                const int site = e / CO, c = e % CO, w = CO < 4 ? CO : 4;
                g_s[(size_t)site * PO + c] = __ldg(a.gout + chunk_at(b, s0 * S + site, c - c % w, CO, V) + c % w);
            }
        }
        if (CI % 4 == 0) {
            const int nc = CI / 4, nsite = (G + 2) * S;
            for (int e = threadIdx.x; e < nsite * nc; e += blockDim.x) {
                const int c4 = e / nsite, site = e % nsite;
                const int sl = s0 - 1 + site / S;
                const int n = ((sl % L + L) % L) * S + site % S;
                const float4 v = __ldg(reinterpret_cast<const float4*>(a.in + chunk_at(b, n, 4 * c4, CI, V)));
                *reinterpret_cast<float4*>(x_s + (size_t)site * PI + 4 * c4) = v;     // (inputs with CI > 1 are unmasked)
            }
        } else {
            for (int e = threadIdx.x; e < (G + 2) * S * CI; e += blockDim.x) {
                const int site = e / CI, c = e % CI, w = CI < 4 ? CI : 4;
                const int sl = s0 - 1 + site / S;
                const int n = ((sl % L + L) % L) * S + site % S;
                float v = __ldg(a.in + chunk_at(b, n, c - c % w, CI, V) + c % w);
                if (a.mask >= 0 && parity<ND>(n, L) != a.mask) v = 0.f;
                x_s[(size_t)site * PI + c] = v;
            }
        }
        __syncthreads();
        if (!active) continue;
        const int cin = conv3 ? ch : 0;
        for (int row = grp; row < G * rows_per_slice; row += ngrp) {
            const int rs = row / rows_per_slice, y = row % rows_per_slice;
            // input row k = (ds, dy) of output row (rs, y): slice rs + 1 + ds, row y + dy
            int base[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const int ds = (ND == 3 ? k / 3 : k) - 1, dy = ND == 3 ? k % 3 - 1 : 0;
                base[k] = (rs + 1 + ds) * S + (ND == 3 ? wrapi(y + dy, L) * L : 0);
            }
            const int gbase = rs * S + (ND == 3 ? y * L : 0);
            float wm[NR], w0[NR], wp[NR];                  // window at x-1, x, x+1
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                wm[k] = x_s[(size_t)(base[k] + L - 1) * PI + cin];
                w0[k] = x_s[(size_t)base[k] * PI + cin];
            }
            for (int x = 0; x < L; ++x) {
                const int xp = x + 1 == L ? 0 : x + 1;
#pragma unroll
                for (int k = 0; k < NR; ++k) wp[k] = x_s[(size_t)(base[k] + xp) * PI + cin];
                float g0, g1 = 0.f;
                if (conv3) {
                    const float2 gg = *reinterpret_cast<const float2*>(g_s + (size_t)(gbase + x) * PO);
                    g0 = gg.x;
                    g1 = gg.y;
                } else {
                    g0 = g_s[(size_t)(gbase + x) * PO + ch];
                }
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    // taps (k, dx = -1, 0, +1) = tap index 3k + dxi
                    acc[(3 * k + 0) * 2] = fmaf(wm[k], g0, acc[(3 * k + 0) * 2]);
                    acc[(3 * k + 1) * 2] = fmaf(w0[k], g0, acc[(3 * k + 1) * 2]);
                    acc[(3 * k + 2) * 2] = fmaf(wp[k], g0, acc[(3 * k + 2) * 2]);
                    if (conv3) {
                        acc[(3 * k + 0) * 2 + 1] = fmaf(wm[k], g1, acc[(3 * k + 0) * 2 + 1]);
                        acc[(3 * k + 1) * 2 + 1] = fmaf(w0[k], g1, acc[(3 * k + 1) * 2 + 1]);
                        acc[(3 * k + 2) * 2 + 1] = fmaf(wp[k], g1, acc[(3 * k + 2) * 2 + 1]);
                    }
                    wm[k] = w0[k];
                    w0[k] = wp[k];
                }
                acc[T * 2] += g0;                          // bias
                acc[T * 2 + 1] += g1;
            }
        }
    }
    // combine the row groups in a fixed order, then one partial per CTA
    __syncthreads();
    if (active)
#pragma unroll
        for (int i = 0; i < NA; ++i) red[((size_t)grp * nch + ch) * NA + i] = acc[i];
    __syncthreads();
    float* P = a.partial + (int64_t)blockIdx.x * (T + 1) * CI * CO;
    for (int e = threadIdx.x; e < nch * NA; e += blockDim.x) {
        const int c = e / NA, i = e % NA;
        float sum = 0.f;
        for (int g = 0; g < ngrp; ++g) sum += red[((size_t)g * nch + c) * NA + i];
        const int t = i >> 1, o = i & 1;
        if (conv3) P[((int64_t)t * CI + c) * 2 + o] = (t == T && c != 0) ? 0.f : sum;
        else if (o == 0) P[(int64_t)t * CO + c] = sum;
    }
}

// Weight gradient of the C -> C convolution (conv2) for C = 32 as a GEMM over
// the sites: dW[(t, i)][o] = sum_n x(n + delta(t))[i] g(n)[o].  A work unit is G
// slices of one configuration, staged in shared memory with a row pitch of 36
// floats (input slices with one halo slice on each side, gout slices); each
// thread owns an 8 x 8 tile (8 input channels of one tap x 8 output channels),
// so per site two 16-byte input loads and two 16-byte gout loads (both shared
// by the lanes of the same tap / channel group) feed 64 FMAs.  In 2D the CTA's
// two thread halves take alternate sites of a unit and are added in a fixed
// order at the end.  The bias gradient rides on the threads of tap 0, input
// group 0.  Per-CTA partials in k_wgrad's layout (tap T = bias).
template <int ND>
__global__ void __launch_bounds__(ND == 3 ? 448 : 288, ND == 3 ? 1 : 2) k_wgrad_c32(const WgArgs a, int G) {
    extern __shared__ __align__(16) float sm[];
    constexpr int T = ND == 3 ? 27 : 9, C = 32, P = 36;
    constexpr int TILES = T * 4 * 4;                  // (tap, input group) x output group
    constexpr int HALVES = ND == 3 ? 1 : 2;
    const int L = a.L, V = a.V, S = V / L;
    const int half = threadIdx.x / TILES, r = threadIdx.x % TILES;
    const bool active = half < HALVES;
    const int ar = r >> 2, og = r & 3;               // A row group (tap, input group), output group
    const int t = ar >> 2, ig = ar & 3;
    int ds, dy, dx;
    tap_delta<ND>(t, ds, dy, dx);
    float* x_s = sm;                                   // [(G+2)*S][P]
    float* g_s = sm + (size_t)(G + 2) * S * P;         // [G*S][P]
    float acc[8][8], accb[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        accb[i] = 0.f;
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[i][o] = 0.f;
    }
    const bool does_bias = ar == 0;
    const int units_per_cfg = L / G;
    const int64_t units = a.B * units_per_cfg;
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int64_t b = u / units_per_cfg;
        const int s0 = (int)(u % units_per_cfg) * G;
        __syncthreads();
        const int nsx = (G + 2) * S;
        for (int e = threadIdx.x; e < nsx * 8; e += blockDim.x) {
            const int c4 = e / nsx, site = e % nsx;
            const int sl = s0 - 1 + site / S;
            const int n = ((sl % L + L) % L) * S + site % S;
            *reinterpret_cast<float4*>(x_s + (size_t)site * P + 4 * c4) =
                __ldg(reinterpret_cast<const float4*>(a.in + chunk_at(b, n, 4 * c4, C, V)));
        }
        const int nsg = G * S;
        for (int e = threadIdx.x; e < nsg * 8; e += blockDim.x) {
            const int c4 = e / nsg, site = e % nsg;
            *reinterpret_cast<float4*>(g_s + (size_t)site * P + 4 * c4) =
                __ldg(reinterpret_cast<const float4*>(a.gout + chunk_at(b, s0 * S + site, 4 * c4, C, V)));
        }
        __syncthreads();
        if (!active) continue;
        // sites of the unit as (slice rs, row y, column x); the 2D halves take
        // alternate columns, the tap's shifted column is a wrap of x + dx
        const int rows = ND == 3 ? L : 1;
        for (int rr = 0; rr < G * rows; ++rr) {
            const int rs = ND == 3 ? rr / L : rr, y = ND == 3 ? rr - rs * L : 0;
            const int in_row = (rs + 1 + ds) * S + (ND == 3 ? wrapi(y + dy, L) * L : 0);
            const int g_row = rs * S + y * L;
            for (int x = half; x < L; x += HALVES) {
            const int j2 = wrapi(x + dx, L);
            const float* ap = x_s + (size_t)(in_row + j2) * P + ig * 8;
            const float* bp = g_s + (size_t)(g_row + x) * P + og * 8;
            const float4 a0 = *reinterpret_cast<const float4*>(ap);
            const float4 a1 = *reinterpret_cast<const float4*>(ap + 4);
            const float4 b0 = *reinterpret_cast<const float4*>(bp);
            const float4 b1 = *reinterpret_cast<const float4*>(bp + 4);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int o = 0; o < 8; ++o) acc[i][o] = fmaf(av[i], bv[o], acc[i][o]);
            if (does_bias)
#pragma unroll
                for (int o = 0; o < 8; ++o) accb[o] += bv[o];
            }
        }
    }
    // combine the halves (2D) in a fixed order through shared memory, then write
    __syncthreads();
    float* Pt = a.partial + (int64_t)blockIdx.x * (T + 1) * C * C;
    if (HALVES == 2) {
        float* red = sm;                               // [TILES][72]
        if (active && half == 1) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int o = 0; o < 8; ++o) red[(size_t)r * 72 + i * 8 + o] = acc[i][o];
#pragma unroll
            for (int o = 0; o < 8; ++o) red[(size_t)r * 72 + 64 + o] = accb[o];
        }
        __syncthreads();
        if (active && half == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int o = 0; o < 8; ++o) acc[i][o] += red[(size_t)r * 72 + i * 8 + o];
#pragma unroll
            for (int o = 0; o < 8; ++o) accb[o] += red[(size_t)r * 72 + 64 + o];
        }
    }
    if (active && half == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int o = 0; o < 8; ++o) Pt[((int64_t)t * C + ig * 8 + i) * C + og * 8 + o] = acc[i][o];
        if (does_bias)
#pragma unroll
            for (int o = 0; o < 8; ++o) Pt[((int64_t)T * C + 0) * C + og * 8 + o] = accb[o];
    }
}

// grad (canonical, for one conv of one layer): W[o][i][t] and b[o], scaled by 1/B.
__global__ void __launch_bounds__(256) k_wgrad_reduce(const float* __restrict__ partial, int nparts, int T, int Cin,
                                                      int Cout, float scale, float* __restrict__ gW,
                                                      float* __restrict__ gb) {
    // block = 32 outputs (lane); its 8 warps sum interleaved eighths of the
    // partials, combined in warp order (fixed: deterministic)
    __shared__ float part[8][32];
    const int per = (T + 1) * Cin * Cout;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (p < per)
        for (int k = wid; k < nparts; k += 8) s += partial[(int64_t)k * per + p];
    part[wid][lane] = s;
    __syncthreads();
    if (wid == 0 && p < per) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += part[w][lane];
        const int o = p % Cout, i = (p / Cout) % Cin, tt = p / (Cout * Cin);
        if (tt < T) gW[((int64_t)o * Cin + i) * T + tt] = t * scale;
        else if (i == 0) gb[o] = t * scale;
    }
}

// ------------------------------------------------------------------ loss, force
// loss_b = log r(z_b) - logdet_b + S(phi_b); gx = dS/dphi (FP64 terms, FP32 out).
template <int ND>
__global__ void __launch_bounds__(kThreads) k_loss_force(const float* __restrict__ z, const float* __restrict__ phi,
                                                        const double* __restrict__ logdet, double m2, double lam,
                                                        int L, int V, int64_t B, double* __restrict__ loss_b,
                                                        float* __restrict__ gx) {
    __shared__ double red[32];
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        const float* p = phi + b * V;
        double acc = 0.0, z2 = 0.0;
        for (int n = threadIdx.x; n < V; n += blockDim.x) {
            const double c = p[n];
            acc += c * lap_minus(p, n, ND, L) + m2 * c * c + lam * c * c * c * c;
            gx[b * V + n] = (float)phi4_force_site(p, n, ND, L, m2, lam);
            const double zz = z[b * V + n];
            z2 += zz * zz;
        }
        const double S = block_sum(acc, red);
        const double Z2 = block_sum(z2, red);
        if (threadIdx.x == 0) loss_b[b] = (-0.5 * Z2 - 0.5 * (double)V * LOG_2PI) - logdet[b] + S;
        __syncthreads();
    }
}

__global__ void k_mean(const double* __restrict__ v, int64_t n, double* __restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = s / (double)n;
}

// ------------------------------------------------------------------ unfused sampler epilogue
// log r(z), S(phi) (FP64 site terms), log q = log r - logdet, log w = -S - log q.
template <int ND>
__global__ void __launch_bounds__(kThreads) k_finish(const float* __restrict__ z, const float* __restrict__ phi,
                                                    const double* __restrict__ logdet, int has_phi4, double m2,
                                                    double lam, int L, int V, int64_t B, float* __restrict__ phi_out,
                                                    float* __restrict__ z_out, double* __restrict__ logq,
                                                    double* __restrict__ S_out, double* __restrict__ logw) {
    __shared__ double red[32];
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        const float* p = phi + b * V;
        double acc = 0.0, z2 = 0.0;
        for (int n = threadIdx.x; n < V; n += blockDim.x) {
            const double c = p[n];
            if (has_phi4) {
                double k = 0.0;
                for (int mu = 0; mu < ND; ++mu) {
                    const int t_plus = (mu == 0) ? (ND == 3 ? 14 : 5) : (mu == 1) ? (ND == 3 ? 16 : 7) : 22;
                    const int t_minus = (ND == 3 ? 26 : 8) - t_plus;
                    k += 2.0 * c - (double)p[nbr<ND>(n, t_plus, L)] - (double)p[nbr<ND>(n, t_minus, L)];
                }
                acc += c * k + m2 * c * c + lam * c * c * c * c;
            }
            const double zz = z[b * V + n];
            z2 += zz * zz;
            phi_out[b * V + n] = p[n];
            if (z_out) z_out[b * V + n] = z[b * V + n];
        }
        const double S = block_sum(acc, red);
        const double Z2 = block_sum(z2, red);
        if (threadIdx.x == 0) {
            const double lq = (-0.5 * Z2 - 0.5 * (double)V * LOG_2PI) - logdet[b];
            logq[b] = lq;
            if (has_phi4 && S_out) S_out[b] = S;
            if (has_phi4 && logw) logw[b] = -S - lq;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ weights for the reverse pass
// Transposed + tap-flipped copies: Wb[t][o][i] = W[o][i][T-1-t] (delta(T-1-t) = -delta(t)).
__global__ void k_pack_bwd(const float* __restrict__ canon, int64_t cstride, int n_layers, int T, int C1, int C2,
                           float* __restrict__ out, int64_t ostride) {
    const int64_t total = (int64_t)n_layers * ostride;
    const int64_t n1 = (int64_t)T * C1, n2 = (int64_t)T * C2 * C1, n3 = (int64_t)T * 2 * C2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / ostride);
        int64_t r = i - l * ostride;
        const float* W = canon + l * cstride;
        float v = 0.f;
        if (r < n1) {                                    // W1b[t][c] = W1[c][0][T-1-t]
            const int t = (int)(r / C1), c = (int)(r % C1);
            v = W[(int64_t)c * T + (T - 1 - t)];
        } else if ((r -= n1) < n2) {                     // W2b[t][o][i] = W2[o][i][T-1-t]
            const int t = (int)(r / ((int64_t)C2 * C1));
            const int o = (int)((r / C1) % C2), ii = (int)(r % C1);
            v = W[n1 + C1 + ((int64_t)o * C1 + ii) * T + (T - 1 - t)];
        } else if ((r -= n2) < n3) {                     // W3b[t][o][i] = W3[o][i][T-1-t]
            const int t = (int)(r / (2 * C2));
            const int o = (int)((r / C2) % 2), ii = (int)(r % C2);
            v = W[n1 + C1 + n2 + C2 + ((int64_t)o * C2 + ii) * T + (T - 1 - t)];
        }
        out[i] = v;
    }
}

// ------------------------------------------------------------------ Adam (Kingma & Ba)
__global__ void k_adam(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ------------------------------------------------------------------ workspace
struct TrainWs {
    float *xs, *h1, *h2, *s, *gx, *g3, *gh2, *gh1, *wb, *partial, *grad;
    double *logdet, *loss_b;
    size_t bytes;
};

int wgrad_grid() { return num_sms() * 2; }

TrainWs carve(const gf_flow* f, int64_t B, char* base) {
    TrainWs w;
    std::memset(&w, 0, sizeof(w));
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += (bytes + 255) & ~size_t(255);
        return p;
    };
    const int64_t BV = B * (int64_t)f->V;
    const int N = f->shape.n_layers, C = std::max(f->C1, f->C2);
    const int64_t obstride = (int64_t)f->T * f->C1 + (int64_t)f->T * f->C2 * f->C1 + 2LL * f->T * f->C2;
    w.xs = (float*)take(sizeof(float) * BV * (N + 1));
    w.h1 = (float*)take(sizeof(float) * BV * f->C1);
    w.h2 = (float*)take(sizeof(float) * BV * f->C2);
    w.s = (float*)take(sizeof(float) * BV);
    w.gx = (float*)take(sizeof(float) * BV);
    w.g3 = (float*)take(sizeof(float) * BV * 2);
    w.gh2 = (float*)take(sizeof(float) * BV * f->C2);
    w.gh1 = (float*)take(sizeof(float) * BV * f->C1);
    w.wb = (float*)take(sizeof(float) * obstride * std::max(N, 1));
    w.partial = (float*)take(sizeof(float) * (size_t)wgrad_grid() * (f->T + 1) * C * C);
    w.grad = (float*)take(sizeof(float) * std::max<int64_t>(f->n_params, 1));
    w.logdet = (double*)take(sizeof(double) * std::max<int64_t>(B, 1));
    w.loss_b = (double*)take(sizeof(double) * std::max<int64_t>(B, 1));
    w.bytes = off;
    return w;
}

int64_t grid1d(int64_t n) { return std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)num_sms() * 16)); }

template <int ND>
gf_status conv(const ConvArgs& a, cudaStream_t st) {
    const int64_t warps = a.B * ((a.V + 127) / 128) * (a.Cout / 8);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, (int64_t)num_sms() * 8));
    const int T = ND == 3 ? 27 : 9;
    const size_t smem = (size_t)T * a.Cin * a.Cout * sizeof(float);
    auto go = [&](auto kern) -> bool {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return false;
        kern<<<(unsigned)grid, kThreads, smem, st>>>(a);
        return true;
    };
    bool ok;
    if (a.mask >= 0) {      // masked input (conv1 of a coupling): parity test per neighbour
        if (a.Cin % 4 == 0) ok = go(k_conv<ND, 4, true>);
        else if (a.Cin % 2 == 0) ok = go(k_conv<ND, 2, true>);
        else ok = go(k_conv<ND, 1, true>);
    } else {
        if (a.Cin % 4 == 0) ok = go(k_conv<ND, 4, false>);
        else if (a.Cin % 2 == 0) ok = go(k_conv<ND, 2, false>);
        else ok = go(k_conv<ND, 1, false>);
    }
    if (!ok) return GF_ECUDA;
    GF_CHECK_LAUNCH();
    return GF_OK;
}

// conv1 + LReLU and conv2 + LReLU of layer l on x_l (FP32, activations in the workspace).
template <int ND>
gf_status net_fwd(const gf_flow* f, int l, const float* xl, int64_t B, const TrainWs& w, cudaStream_t st) {
    const PackedOffsets po = packed_offsets(f->T, f->C1, f->C2);
    const float slope = (float)f->shape.leaky_slope;
    const float* P = f->d_packed + (int64_t)l * f->packed_stride;
    ConvArgs c1{xl, 1, l & 1, P + po.W1, P + po.b1, f->C1, w.h1, nullptr, 0, slope, f->shape.L, f->V, B};
    gf_status s = conv<ND>(c1, st);
    if (s != GF_OK) return s;
    ConvArgs c2{w.h1, f->C1, -1, P + po.W2, P + po.b2, f->C2, w.h2, nullptr, 0, slope, f->shape.L, f->V, B};
    return conv<ND>(c2, st);
}

template <int ND>
gf_status wgrad(const WgArgs& a, float* gW, float* gbias, float scale, cudaStream_t st) {
    const int T = ND == 3 ? 27 : 9;
    const int grid = (int)std::min<int64_t>(a.B, wgrad_grid());
    // lanes per task: enough threads per CTA for the small (conv1, conv3) gradients
    auto launch = [&](auto kern, int tasks) {
        int nsplit = 1;
        while (nsplit < 8 && tasks * nsplit * 2 <= 512) nsplit *= 2;
        const int threads = (tasks * nsplit + 31) / 32 * 32;
        kern<<<grid, threads, 0, st>>>(a, nsplit);
    };
    if (a.Cin == 1 || a.Cout == 2) {
        // thin convolutions: shared-memory tiled, one thread per (tap, channel);
        // G = the largest divisor of L whose staged rows fit in 96 KB
        const int S = a.V / a.L;
        const int nch = a.Cout == 2 ? a.Cin : a.Cout;
        const int ngrp = std::max(1, 512 / nch);
        const size_t red = (size_t)ngrp * nch * (T + 1) * 2 * sizeof(float);
        int G = a.L;
        const int PI = a.Cin % 4 == 0 ? a.Cin + 4 : a.Cin, PO = a.Cout % 4 == 0 ? a.Cout + 4 : a.Cout;
        auto staged = [&](int g) { return (size_t)(g * S * PO + (g + 2) * S * PI) * sizeof(float); };
        while (G > 1 && (staged(G) > 112 * 1024 || a.L % G != 0)) --G;
        auto bytes = [&](int g) { return std::max(staged(g), red); };   // the group sums reuse the staging area
        if (cudaFuncSetAttribute(k_wgrad_thin<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes(G)) != cudaSuccess)
            return GF_ECUDA;
        k_wgrad_thin<ND><<<grid, ngrp * nch, bytes(G), st>>>(a, G);
    } else {
        // C -> C (unmasked input): shared-memory tiled; G = the largest divisor of
        // L whose staged rows fit in 96 KB, else 1
        if (a.mask >= 0) return GF_EINVAL;
        if (a.Cin == 32 && a.Cout == 32) {
            const int S = a.V / a.L;
            auto bytes = [&](int g) { return (size_t)((g + 2) * S + g * S) * 36 * sizeof(float); };
            int G = a.L;
            while (G > 1 && (bytes(G) > 100 * 1024 || a.L % G != 0)) --G;
            const size_t smem = std::max(bytes(G), (size_t)(T * 16) * 72 * sizeof(float));
            const int threads = ND == 3 ? 448 : 288;
            if (cudaFuncSetAttribute(k_wgrad_c32<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
                return GF_ECUDA;
            k_wgrad_c32<ND><<<grid, threads, smem, st>>>(a, G);
            GF_CHECK_LAUNCH();
            const int per = (T + 1) * a.Cin * a.Cout;
            k_wgrad_reduce<<<(per + 31) / 32, 256, 0, st>>>(a.partial, grid, T, a.Cin, a.Cout, scale, gW, gbias);
            GF_CHECK_LAUNCH();
            return GF_OK;
        }
        const int S = a.V / a.L;
        int G = a.L;
        auto bytes = [&](int g) { return (size_t)(g * S * a.Cout + (g + 2) * S * a.Cin) * sizeof(float); };
        while (G > 1 && (bytes(G) > 96 * 1024 || a.L % G != 0)) --G;
        const int threads = ((T + 1) * (a.Cin / 4) * (a.Cout / 8) + 31) / 32 * 32;
        if (cudaFuncSetAttribute(k_wgrad_tiled<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes(G)) != cudaSuccess)
            return GF_ECUDA;
        k_wgrad_tiled<ND><<<grid, threads, bytes(G), st>>>(a, G);
    }
    GF_CHECK_LAUNCH();
    const int per = (T + 1) * a.Cin * a.Cout;
    k_wgrad_reduce<<<(per + 31) / 32, 256, 0, st>>>(a.partial, grid, T, a.Cin, a.Cout, scale, gW, gbias);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

// Forward pass of training: z -> x_1 .. x_N saved in the workspace, logdet per
// configuration.  Leaves the last layer's h1 / h2 / s in the workspace.
template <int ND>
gf_status forward_pass(const gf_flow* f, int64_t B, uint64_t seed, uint64_t counter0, const float* z_in,
                       const TrainWs& w, cudaStream_t st) {
    const int L = f->shape.L, V = f->V, N = f->shape.n_layers, T = f->T;
    const int C1 = f->C1, C2 = f->C2;
    const int64_t BV = B * (int64_t)V;
    const float slope = (float)f->shape.leaky_slope;
    const PackedOffsets po = packed_offsets(T, C1, C2);
    if (fp32_c32_supported(f)) {
        // one fused launch: z (or the prior) -> every layer's input x_l and the
        // log-det, with the FP32 weights (log q goes to a scratch buffer)
        return launch_flow_fp32_c32(f, false, nullptr, B, seed, counter0, z_in, w.xs, nullptr,
                                    w.xs + (int64_t)N * BV, w.loss_b, nullptr, nullptr, st, w.xs, BV, w.logdet);
    }
    k_prior<<<(unsigned)grid1d(BV / 4 + 1), kThreads, 0, st>>>(V, B, seed, counter0, z_in, w.xs);
    GF_CHECK_LAUNCH();
    if (cudaMemsetAsync(w.logdet, 0, sizeof(double) * B, st) != cudaSuccess) return GF_ECUDA;
    const unsigned cfg_grid = (unsigned)std::min<int64_t>(B, (int64_t)num_sms() * 8);
    for (int l = 0; l < N; ++l) {
        const float* xl = w.xs + (int64_t)l * BV;
        gf_status s = net_fwd<ND>(f, l, xl, B, w, st);
        if (s != GF_OK) return s;
        const float* P = f->d_packed + (int64_t)l * f->packed_stride;
        k_couple_fwd<ND><<<cfg_grid, kThreads, 0, st>>>(w.h2, C2, P + po.W3, P + po.b3, f->shape.use_final_tanh,
                                                       l & 1, L, V, B, xl, w.xs + (int64_t)(l + 1) * BV, w.s,
                                                       w.logdet);
        GF_CHECK_LAUNCH();
    }
    return GF_OK;
}

// Reverse pass: with w.gx = dLoss/dphi seeded and dLoss/dlog q = glq[b] (or
// glq_const when glq is null), writes dLoss/dtheta * scale to grad (canonical
// order).  Needs the x_l saved by forward_pass with the same weights.
template <int ND>
gf_status reverse_pass(const gf_flow* f, int64_t B, const double* glq, float glq_const, float scale, float* grad,
                       const TrainWs& w, cudaStream_t st) {
    const int L = f->shape.L, V = f->V, N = f->shape.n_layers, T = f->T;
    const int C1 = f->C1, C2 = f->C2;
    const int64_t BV = B * (int64_t)V;
    const float slope = (float)f->shape.leaky_slope;
    const int use_tanh = f->shape.use_final_tanh;
    const PackedOffsets po = packed_offsets(T, C1, C2);
    const int64_t obstride = (int64_t)T * C1 + (int64_t)T * C2 * C1 + 2LL * T * C2;
    if (N > 0) {
        k_pack_bwd<<<(unsigned)grid1d(obstride * N), kThreads, 0, st>>>(f->d_canon, f->canon_stride, N, T, C1, C2,
                                                                        w.wb, obstride);
        GF_CHECK_LAUNCH();
    }
    const unsigned cfg_grid = (unsigned)std::min<int64_t>(B, (int64_t)num_sms() * 8);
    for (int l = N - 1; l >= 0; --l) {
        const float* xl = w.xs + (int64_t)l * BV;
        const float* P = f->d_packed + (int64_t)l * f->packed_stride;
        const float* Wb = w.wb + (int64_t)l * obstride;
        float* G = grad + (int64_t)l * f->canon_stride;
        float* gW1 = G;
        float* gb1 = gW1 + (int64_t)C1 * T;
        float* gW2 = gb1 + C1;
        float* gb2 = gW2 + (int64_t)C2 * C1 * T;
        float* gW3 = gb2 + C2;
        float* gb3 = gW3 + 2LL * C2 * T;
        gf_status s;
        if (fp32_c32_recompute_supported(f)) {                          // h1, h2, s in one launch
            if ((s = launch_c32_recompute(f, l, B, xl, w.h1, w.h2, w.s, st)) != GF_OK) return s;
        } else {
            if ((s = net_fwd<ND>(f, l, xl, B, w, st)) != GF_OK) return s;   // recompute h1, h2
            k_couple_fwd<ND><<<cfg_grid, kThreads, 0, st>>>(w.h2, C2, P + po.W3, P + po.b3, use_tanh, l & 1, L, V,
                                                           B, xl, w.g3 /* scratch for x_out */, w.s, nullptr);
            GF_CHECK_LAUNCH();
        }
        k_couple_bwd<ND><<<(unsigned)grid1d(BV), kThreads, 0, st>>>(l & 1, use_tanh, L, V, B, xl, w.s, glq,
                                                                   glq_const, w.gx, w.g3);
        GF_CHECK_LAUNCH();
        // The data gradients (gh2, gh1, gx) stay on `st`; each weight gradient
        // runs on the flow's side stream as soon as its inputs exist and
        // overlaps the next data gradient.  The side stream only reads
        // activations and writes G and the partial sums; the next layer (which
        // rewrites the activations) and the caller wait for it.
        if (cudaEventRecord(f->ev_fork[0], st) != cudaSuccess || cudaStreamWaitEvent(f->side, f->ev_fork[0], 0) != cudaSuccess)
            return GF_ECUDA;
        WgArgs a3{w.h2, C2, -1, w.g3, 2, w.partial, L, V, B};
        if ((s = wgrad<ND>(a3, gW3, gb3, scale, f->side)) != GF_OK) return s;
        ConvArgs d3{w.g3, 2, -1, Wb + (int64_t)T * C1 + (int64_t)T * C2 * C1, nullptr, C2, w.gh2, w.h2, 1, slope, L, V, B};
        if ((s = conv<ND>(d3, st)) != GF_OK) return s;                // gh2 * LReLU'
        if (cudaEventRecord(f->ev_fork[1], st) != cudaSuccess || cudaStreamWaitEvent(f->side, f->ev_fork[1], 0) != cudaSuccess)
            return GF_ECUDA;
        WgArgs a2{w.h1, C1, -1, w.gh2, C2, w.partial, L, V, B};
        if ((s = wgrad<ND>(a2, gW2, gb2, scale, f->side)) != GF_OK) return s;
        ConvArgs d2{w.gh2, C2, -1, Wb + (int64_t)T * C1, nullptr, C1, w.gh1, w.h1, 1, slope, L, V, B};
        if ((s = conv<ND>(d2, st)) != GF_OK) return s;                // gh1 * LReLU'
        if (cudaEventRecord(f->ev_fork[2], st) != cudaSuccess || cudaStreamWaitEvent(f->side, f->ev_fork[2], 0) != cudaSuccess)
            return GF_ECUDA;
        WgArgs a1{xl, 1, l & 1, w.gh1, C1, w.partial, L, V, B};
        if ((s = wgrad<ND>(a1, gW1, gb1, scale, f->side)) != GF_OK) return s;
        k_conv1_bwd<ND><<<(unsigned)grid1d(BV), kThreads, 0, st>>>(w.gh1, C1, Wb, l & 1, L, V, B, w.gx);
        GF_CHECK_LAUNCH();
        if (cudaEventRecord(f->ev_join, f->side) != cudaSuccess || cudaStreamWaitEvent(st, f->ev_join, 0) != cudaSuccess)
            return GF_ECUDA;
    }
    return GF_OK;
}

template <int ND>
gf_status train_step(gf_flow* f, const gf_phi4* phi4, int64_t B, uint64_t seed, uint64_t counter0,
                     const float* z_in, double* loss_out, float* grad_out, float lr, float beta1,
                     float beta2, float adam_eps, float* adam_m, float* adam_v, int64_t adam_t,
                     const TrainWs& w, cudaStream_t st) {
    const int L = f->shape.L, V = f->V, N = f->shape.n_layers;
    const int64_t BV = B * (int64_t)V;
    float* grad = grad_out ? grad_out : w.grad;
    gf_status s = forward_pass<ND>(f, B, seed, counter0, z_in, w, st);
    if (s != GF_OK) return s;
    const unsigned cfg_grid = (unsigned)std::min<int64_t>(B, (int64_t)num_sms() * 8);
    // per-configuration loss log r - logdet + S and the seed dS/dphi; the loss
    // is the mean, so every configuration's gradient is scaled by 1/B
    k_loss_force<ND><<<cfg_grid, kThreads, 0, st>>>(w.xs, w.xs + (int64_t)N * BV, w.logdet, phi4->m2, phi4->lam,
                                                    L, V, B, w.loss_b, w.gx);
    GF_CHECK_LAUNCH();
    k_mean<<<1, kThreads, 0, st>>>(w.loss_b, B, loss_out);
    GF_CHECK_LAUNCH();
    if ((s = reverse_pass<ND>(f, B, nullptr, 1.0f, 1.0f / (float)B, grad, w, st)) != GF_OK) return s;
    if (lr > 0.f) {
        const float c1 = 1.f - powf(beta1, (float)adam_t), c2 = 1.f - powf(beta2, (float)adam_t);
        k_adam<<<(unsigned)grid1d(f->n_params), kThreads, 0, st>>>(f->n_params, f->d_canon, grad, adam_m, adam_v,
                                                                    lr, beta1, beta2, adam_eps, c1, c2);
        GF_CHECK_LAUNCH();
        return repack_weights(f, st);
    }
    return GF_OK;
}

// Forward half for autograd: phi = x_N and log q = log r(z) - logdet.
template <int ND>
gf_status forward_train(const gf_flow* f, int64_t B, uint64_t seed, uint64_t counter0, const float* z_in,
                        float* phi_out, double* logq_out, const TrainWs& w, cudaStream_t st) {
    gf_status s = forward_pass<ND>(f, B, seed, counter0, z_in, w, st);
    if (s != GF_OK) return s;
    const int64_t BV = B * (int64_t)f->V;
    const unsigned cfg_grid = (unsigned)std::min<int64_t>(B, (int64_t)num_sms() * 8);
    k_finish<ND><<<cfg_grid, kThreads, 0, st>>>(w.xs, w.xs + (int64_t)f->shape.n_layers * BV, w.logdet, 0, 0.0,
                                               0.0, f->shape.L, f->V, B, phi_out, nullptr, logq_out, nullptr,
                                               nullptr);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

// Backward half: gx <- dLoss/dphi (zero when null), then the reverse pass.
template <int ND>
gf_status backward(const gf_flow* f, int64_t B, const float* gphi, const double* glogq, float* grad,
                   const TrainWs& w, cudaStream_t st) {
    const size_t bytes = sizeof(float) * (size_t)B * f->V;
    const cudaError_t e = gphi ? cudaMemcpyAsync(w.gx, gphi, bytes, cudaMemcpyDeviceToDevice, st)
                               : cudaMemsetAsync(w.gx, 0, bytes, st);
    if (e != cudaSuccess) return GF_ECUDA;
    return reverse_pass<ND>(f, B, glogq, 0.0f, 1.0f, grad, w, st);
}

// Unfused FP32 sampler: one kernel per convolution, activations through HBM.
// Workspace: z, two x buffers, h1, h2, s [B][V](x C), logdet [B].
struct PlainWs { float *z, *xa, *xb, *h1, *h2, *s; double* logdet; size_t bytes; };

PlainWs carve_plain(const gf_flow* f, int64_t B, char* base) {
    PlainWs w;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += (bytes + 255) & ~size_t(255);
        return p;
    };
    const int64_t BV = B * (int64_t)f->V;
    w.z = (float*)take(sizeof(float) * BV);
    w.xa = (float*)take(sizeof(float) * BV);
    w.xb = (float*)take(sizeof(float) * BV);
    w.h1 = (float*)take(sizeof(float) * BV * f->C1);
    w.h2 = (float*)take(sizeof(float) * BV * f->C2);
    w.s = (float*)take(sizeof(float) * BV);
    w.logdet = (double*)take(sizeof(double) * std::max<int64_t>(B, 1));
    w.bytes = off;
    return w;
}

template <int ND>
gf_status sample_unfused(const gf_flow* f, const gf_phi4* phi4, int64_t B, uint64_t seed, uint64_t counter0,
                         const float* z_in, float* z_out, float* phi_out, double* logq, double* S_out,
                         double* logw, const PlainWs& w, cudaStream_t st) {
    const int L = f->shape.L, V = f->V, N = f->shape.n_layers;
    const int C1 = f->C1, C2 = f->C2;
    const int64_t BV = B * (int64_t)V;
    const float slope = (float)f->shape.leaky_slope;
    const PackedOffsets po = packed_offsets(f->T, C1, C2);
    k_prior<<<(unsigned)grid1d(BV / 4 + 1), kThreads, 0, st>>>(V, B, seed, counter0, z_in, w.z);
    GF_CHECK_LAUNCH();
    if (cudaMemsetAsync(w.logdet, 0, sizeof(double) * B, st) != cudaSuccess) return GF_ECUDA;
    const unsigned cfg_grid = (unsigned)std::min<int64_t>(B, (int64_t)num_sms() * 8);
    const float* xin = w.z;
    float* bufs[2] = {w.xa, w.xb};
    for (int l = 0; l < N; ++l) {
        const float* P = f->d_packed + (int64_t)l * f->packed_stride;
        ConvArgs c1{xin, 1, l & 1, P + po.W1, P + po.b1, C1, w.h1, nullptr, 0, slope, L, V, B};
        gf_status s = conv<ND>(c1, st);
        if (s != GF_OK) return s;
        ConvArgs c2{w.h1, C1, -1, P + po.W2, P + po.b2, C2, w.h2, nullptr, 0, slope, L, V, B};
        if ((s = conv<ND>(c2, st)) != GF_OK) return s;
        float* xout = bufs[l & 1];
        k_couple_fwd<ND><<<cfg_grid, kThreads, 0, st>>>(w.h2, C2, P + po.W3, P + po.b3, f->shape.use_final_tanh,
                                                       l & 1, L, V, B, xin, xout, w.s, w.logdet);
        GF_CHECK_LAUNCH();
        xin = xout;
    }
    k_finish<ND><<<cfg_grid, kThreads, 0, st>>>(w.z, xin, w.logdet, phi4 != nullptr, phi4 ? phi4->m2 : 0.0,
                                               phi4 ? phi4->lam : 0.0, L, V, B, phi_out, z_out, logq, S_out, logw);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

}  // namespace
}  // namespace gf

using namespace gf;

extern "C" {

size_t gf_train_workspace_bytes(const gf_flow* flow, int64_t B) {
    if (!flow || B < 0 || flow->variant) return 0;
    return carve(flow, B, nullptr).bytes;
}

gf_status gf_flow_train_step(gf_flow* flow, const gf_phi4* phi4, int64_t B, uint64_t seed,
                             uint64_t counter0, const float* d_z_in, double* d_loss_out,
                             float* d_grad_out, float lr, float beta1, float beta2,
                             float adam_eps, float* d_adam_m, float* d_adam_v,
                             int64_t adam_t, void* d_workspace, size_t workspace_bytes,
                             cudaStream_t stream) {
    if (!flow || !phi4 || B <= 0 || !d_loss_out) return GF_EINVAL;
    if (flow->variant) return GF_EUNSUPPORTED;
    if (!(lr >= 0.f)) return GF_EINVAL;
    if (lr > 0.f && (!d_adam_m || !d_adam_v || adam_t < 1)) return GF_EINVAL;
    const TrainWs w = carve(flow, B, static_cast<char*>(d_workspace));
    if (!d_workspace || workspace_bytes < w.bytes) return GF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_workspace) & 255) != 0) return GF_EINVAL;
    if (flow->shape.nd == 3)
        return train_step<3>(flow, phi4, B, seed, counter0, d_z_in, d_loss_out, d_grad_out, lr, beta1, beta2,
                             adam_eps, d_adam_m, d_adam_v, adam_t, w, stream);
    return train_step<2>(flow, phi4, B, seed, counter0, d_z_in, d_loss_out, d_grad_out, lr, beta1, beta2,
                         adam_eps, d_adam_m, d_adam_v, adam_t, w, stream);
}

gf_status gf_flow_forward_train(const gf_flow* flow, int64_t B, uint64_t seed, uint64_t counter0,
                                const float* d_z_in, float* d_phi_out, double* d_logq_out, void* d_workspace,
                                size_t workspace_bytes, cudaStream_t stream) {
    if (!flow || B <= 0 || !d_phi_out || !d_logq_out) return GF_EINVAL;
    if (flow->variant) return GF_EUNSUPPORTED;
    const TrainWs w = carve(flow, B, static_cast<char*>(d_workspace));
    if (!d_workspace || workspace_bytes < w.bytes) return GF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_workspace) & 255) != 0) return GF_EINVAL;
    if (flow->shape.nd == 3)
        return forward_train<3>(flow, B, seed, counter0, d_z_in, d_phi_out, d_logq_out, w, stream);
    return forward_train<2>(flow, B, seed, counter0, d_z_in, d_phi_out, d_logq_out, w, stream);
}

gf_status gf_flow_backward(const gf_flow* flow, int64_t B, const float* d_gphi, const double* d_glogq,
                           float* d_grad_out, void* d_workspace, size_t workspace_bytes, cudaStream_t stream) {
    if (!flow || B <= 0 || !d_grad_out) return GF_EINVAL;
    if (flow->variant) return GF_EUNSUPPORTED;
    const TrainWs w = carve(flow, B, static_cast<char*>(d_workspace));
    if (!d_workspace || workspace_bytes < w.bytes) return GF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_workspace) & 255) != 0) return GF_EINVAL;
    if (flow->shape.nd == 3) return backward<3>(flow, B, d_gphi, d_glogq, d_grad_out, w, stream);
    return backward<2>(flow, B, d_gphi, d_glogq, d_grad_out, w, stream);
}

gf_status gf_flow_adam_step(gf_flow* flow, const float* d_grad, float lr, float beta1, float beta2,
                            float adam_eps, float* d_adam_m, float* d_adam_v, int64_t adam_t,
                            cudaStream_t stream) {
    if (!flow || !d_grad || !d_adam_m || !d_adam_v || adam_t < 1 || !(lr >= 0.f)) return GF_EINVAL;
    if (flow->n_params == 0) return GF_OK;
    const float c1 = 1.f - powf(beta1, (float)adam_t), c2 = 1.f - powf(beta2, (float)adam_t);
    k_adam<<<(unsigned)grid1d(flow->n_params), kThreads, 0, stream>>>(flow->n_params, flow->d_canon, d_grad,
                                                                       d_adam_m, d_adam_v, lr, beta1, beta2,
                                                                       adam_eps, c1, c2);
    GF_CHECK_LAUNCH();
    if (flow->variant) return repack_variant(flow, stream);
    return repack_weights(flow, stream);
}

size_t gf_unfused_workspace_bytes(const gf_flow* flow, int64_t B) {
    if (!flow || B < 0 || flow->variant) return 0;
    return carve_plain(flow, B, nullptr).bytes;
}

gf_status gf_flow_sample_unfused(const gf_flow* flow, const gf_phi4* phi4, int64_t B, uint64_t seed,
                                 uint64_t counter0, const float* d_z_in, float* d_z_out, float* d_phi_out,
                                 double* d_logq_out, double* d_S_out, double* d_logw_out, void* d_workspace,
                                 size_t workspace_bytes, cudaStream_t stream) {
    if (!flow || B < 0 || (B > 0 && (!d_phi_out || !d_logq_out))) return GF_EINVAL;
    if (!phi4 && (d_S_out || d_logw_out)) return GF_EINVAL;
    if (flow->variant) return GF_EUNSUPPORTED;
    if (B == 0) return GF_OK;
    const PlainWs w = carve_plain(flow, B, static_cast<char*>(d_workspace));
    if (!d_workspace || workspace_bytes < w.bytes) return GF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_workspace) & 255) != 0) return GF_EINVAL;
    if (flow->shape.nd == 3)
        return sample_unfused<3>(flow, phi4, B, seed, counter0, d_z_in, d_z_out, d_phi_out, d_logq_out, d_S_out,
                                 d_logw_out, w, stream);
    return sample_unfused<2>(flow, phi4, B, seed, counter0, d_z_in, d_z_out, d_phi_out, d_logq_out, d_S_out,
                             d_logw_out, w, stream);
}

}  // extern "C"
