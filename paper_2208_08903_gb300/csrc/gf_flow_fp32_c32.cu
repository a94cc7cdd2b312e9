// gf_flow_fp32_c32.cu -- fused FP32 coupling-stack kernel for 3D L=16 with
// hidden width 32 (the paper's network form, Sec. 3, at the 3D workload's
// size), both directions.  Paper Sec. 1: prior, even/odd affine coupling
// layers x -> x*exp(s) + t, log-det = sum of s, log q = log r - log det, the
// action and log w = -S - log q.
//
// One CTA per configuration (persistent grid-stride loop), 256 threads.  The
// layer's packed weights (conv2: 110.6 KB) are staged in shared memory, so
// every weight read is a broadcast shared-memory load; the field stays in
// shared memory through all layers.  conv2 (95 % of the FLOPs) runs as a
// sequence of 18 steps per layer over the z-slices zs = 15, 0, 1, ..., 15, 0:
// step k computes h1 of slice zs (conv1 + LeakyReLU, 256 sites x 32 channels,
// one shared-memory slice) and adds its contributions to the conv2 outputs of
// slices k (tap plane dz = -1), k-1 (dz = 0) and k-2 (dz = +1).  Those three
// output slices live in registers (a ring of three 4-site x 8-channel tiles
// per thread: 96 accumulators), so each h1 slice is read once per layer and
// no h2 ring is stored; the 48 (source, output) slice pairs of a layer are
// each computed exactly once (the first and last steps feed only the wrapped
// outputs).  When output slice k-2 is complete it becomes h2 (LeakyReLU) in
// one shared slice, and its conv3 contributions to the s, t accumulators of
// the updated sites of slices k-3, k-2, k-1 are added at once; after step 17
// every s, t is complete and the affine update runs.  Per conv2 weight/input
// read: 4 h1 loads (one per site) and 2 broadcast 16-byte weight loads per
// tap plane feed 32 FMAs per plane, issued as 16 packed FP32-pair FMAs
// (fma.rn.f32x2: same rounding, half the issue slots).
//
// 2D L=32 with hidden width 32 (the 2D training workload's flow) uses the same
// plan with slabs of 16 rows instead of z-slices: per layer two steps, each
// computing h1 of the slab's 16 rows plus one halo row on each side (18 rows,
// 12.5 % extra conv1 work), conv2 of the 16 rows from that buffer (a thread
// holds 8 sites x 8 channels: 8 h1 loads and 2 broadcast weight loads feed 64
// FMAs, issued as 32 packed FP32-pair FMAs), h2 of the slab, and its conv3
// contributions to the s, t accumulators of rows -1 .. 16 of the slab.
#include <algorithm>
#include <cstring>

#include "gf_f32x2.cuh"
#include "gf_flow.cuh"

namespace gf {

namespace {

constexpr int kThr = 256;
constexpr int kL = 16, kS = 256, kV = 4096, kC = 32, kCP = 33;   // CP: row pitch of h1 / h2 (conflict-free)
constexpr int kT = 27;
// shared memory (floats)
constexpr int kOffX = 0;
constexpr int kOffH1 = kOffX + kV;
constexpr int kOffH2 = kOffH1 + kS * kCP;
constexpr int kOffST = kOffH2 + kS * kCP;             // [16 slices][128 updated sites][2]
constexpr int kOffRed = kOffST + kL * 128 * 2;        // 32 FF
constexpr int kOffW = kOffRed + 64;                   // the layer's packed weights (16-byte aligned)
static_assert((kOffW * 4) % 16 == 0, "weight block alignment");

struct C32Args {
    const float* W;            // packed weights (layer stride `stride`)
    int64_t stride;
    PackedOffsets off;
    int n_layers;
    float slope;
    int use_tanh, has_phi4;
    FF c2d_ff, lam_ff;
    int64_t B;
    uint64_t seed, counter0;
    const float* z_in;
    float* z_out;
    const float* phi_in;
    float* phi_out;
    double* logq_out;
    double* S_out;
    double* logw_out;
    // training forward pass (nullable): the field after layers 1 .. N-1 of
    // configuration b at xs_out + layer * xs_stride + b * V, and its log-det
    float* xs_out;
    int64_t xs_stride;
    double* logdet_out;
};

__device__ __forceinline__ float lrelu(float v, float a) { return v > 0.f ? v : a * v; }

// conv1 + LeakyReLU of slice zs into h1[s][kCP]: thread = site, 32 channels.
// The net input is the field at the fixed sites (parity `frozen`), zero elsewhere.
__device__ __forceinline__ void conv1_slice(const float* __restrict__ x, const float* __restrict__ W1,
                                            const float* __restrict__ b1, float* __restrict__ h1, int zs,
                                            int frozen, float slope) {
    const int s = threadIdx.x, y = s >> 4, xc = s & 15;
    float acc[kC];
#pragma unroll
    for (int c = 0; c < kC; c += 4) {
        const float4 b = *reinterpret_cast<const float4*>(b1 + c);
        acc[c] = b.x; acc[c + 1] = b.y; acc[c + 2] = b.z; acc[c + 3] = b.w;
    }
    int t = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        const int z = (zs + dz) & 15;
        for (int dy = -1; dy <= 1; ++dy) {
            const int yy = (y + dy) & 15;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx, ++t) {
                const int xx = (xc + dx) & 15;
                const float xv = (((xx + yy + z) & 1) == frozen) ? x[(z << 8) | (yy << 4) | xx] : 0.f;
                const float* w = W1 + t * kC;
#pragma unroll
                for (int c = 0; c < kC; c += 4) {
                    const float4 wv = *reinterpret_cast<const float4*>(w + c);
                    acc[c] = fmaf(xv, wv.x, acc[c]);
                    acc[c + 1] = fmaf(xv, wv.y, acc[c + 1]);
                    acc[c + 2] = fmaf(xv, wv.z, acc[c + 2]);
                    acc[c + 3] = fmaf(xv, wv.w, acc[c + 3]);
                }
            }
        }
    }
    float* row = h1 + s * kCP;
#pragma unroll
    for (int c = 0; c < kC; ++c) row[c] = lrelu(acc[c], slope);
}

// Accumulator ring: a[r][k][p] = channels co8 + 2p, co8 + 2p + 1 of site k of
// the output slice held in ring slot r, as a packed FP32 pair: conv2 runs as
// fma.rn.f32x2 (two output channels per instruction, the same rounding as two
// fmaf), which halves the issue slots of the FMA stream.
struct Ring {
    f32x2 a[3][4][4];
};

// one input channel of one tap plane: a[R][k][.] += h[k] * (w[co8 .. co8 + 7])
template <int R>
__device__ __forceinline__ void ring_fma(Ring& g, const f32x2 (&hh)[4], const float* __restrict__ w) {
    const ulonglong2 u = *reinterpret_cast<const ulonglong2*>(w);
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(w + 4);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        g.a[R][k][0] = f2_fma(hh[k], u.x, g.a[R][k][0]);
        g.a[R][k][1] = f2_fma(hh[k], u.y, g.a[R][k][1]);
        g.a[R][k][2] = f2_fma(hh[k], v.x, g.a[R][k][2]);
        g.a[R][k][3] = f2_fma(hh[k], v.y, g.a[R][k][3]);
    }
}

// conv2 contributions of h1 slice zs to the output slices in ring slots RM
// (tap plane dz = -1), R0 (dz = 0) and RP (dz = +1); PM / P0 / PP say which of
// the three exist at this step.
template <int RM, int R0, int RP, bool PM, bool P0, bool PP>
__device__ __forceinline__ void conv2_step(Ring& g, const float* __restrict__ h1, const float* __restrict__ W2,
                                           const int (&ys)[4], const int (&xs)[4], int co8) {
#pragma unroll 1
    for (int tp = 0; tp < 9; ++tp) {
        const int dy = tp / 3 - 1, dx = tp % 3 - 1;
        int base[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) base[k] = ((((ys[k] + dy) & 15) << 4) | ((xs[k] + dx) & 15)) * kCP;
        // weights of tap (dz, dy, dx): W2[(tap * 32 + ci) * 32 + co]
        const float* wm = W2 + (size_t)(0 * 9 + tp) * kC * kC + co8;
        const float* w0 = W2 + (size_t)(1 * 9 + tp) * kC * kC + co8;
        const float* wp = W2 + (size_t)(2 * 9 + tp) * kC * kC + co8;
#pragma unroll 4
        for (int ci = 0; ci < kC; ++ci) {
            f32x2 hh[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) hh[k] = f2_splat(h1[base[k] + ci]);
            if (PM) ring_fma<RM>(g, hh, wm + ci * kC);
            if (P0) ring_fma<R0>(g, hh, w0 + ci * kC);
            if (PP) ring_fma<RP>(g, hh, wp + ci * kC);
        }
    }
}

template <int R>
__device__ __forceinline__ void ring_init(Ring& g, const float* __restrict__ b2, int co8) {
    const ulonglong2 u = *reinterpret_cast<const ulonglong2*>(b2 + co8);
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(b2 + co8 + 4);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        g.a[R][k][0] = u.x; g.a[R][k][1] = u.y; g.a[R][k][2] = v.x; g.a[R][k][3] = v.y;
    }
}

// h2 = LeakyReLU(conv2) of the output slice in ring slot R -> h2[s][kCP].
template <int R>
__device__ __forceinline__ void ring_store(const Ring& g, float* __restrict__ h2, const int (&ss)[4], int co8,
                                           float slope) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float* row = h2 + ss[k] * kCP + co8;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            row[2 * p] = lrelu(f2_lo(g.a[R][k][p]), slope);
            row[2 * p + 1] = lrelu(f2_hi(g.a[R][k][p]), slope);
        }
    }
}

// conv3 contributions of h2 slice zo to the s, t accumulators of the updated
// sites of slices zo - 1 (tap plane dz = +1), zo (dz = 0), zo + 1 (dz = -1).
__device__ __forceinline__ void conv3_from(const float* __restrict__ h2, const float* __restrict__ W3,
                                           float* __restrict__ st, int zo, int frozen) {
    const int pa = frozen ^ 1;                       // parity of the updated sites
    for (int it = threadIdx.x; it < 3 * 128; it += kThr) {
        const int j = it >> 7, a = it & 127;         // j = 0, 1, 2: target slice zo - 1, zo, zo + 1
        const int zc = (zo + j - 1) & 15, dz = 1 - j;  // h2 slice zo = zc + dz
        const int y = a >> 3, xc = 2 * (a & 7) + ((pa ^ zc ^ y) & 1);
        float ps = 0.f, pt = 0.f;
        for (int tp = 0; tp < 9; ++tp) {
            const int dy = tp / 3 - 1, dx = tp % 3 - 1;
            const float* row = h2 + ((((y + dy) & 15) << 4) | ((xc + dx) & 15)) * kCP;
            const float* w = W3 + (size_t)(((dz + 1) * 9 + tp) * kC) * 2;
#pragma unroll 8
            for (int ci = 0; ci < kC; ++ci) {
                const float2 wv = *reinterpret_cast<const float2*>(w + 2 * ci);
                ps = fmaf(row[ci], wv.x, ps);
                pt = fmaf(row[ci], wv.y, pt);
            }
        }
        float* o = st + ((zc << 7) | a) * 2;
        o[0] += ps;
        o[1] += pt;
    }
}

template <int K>
__device__ __forceinline__ void step(Ring& g, float* sm, const float* Wl, const C32Args& a, int frozen,
                                     const int (&ys)[4], const int (&xs)[4], const int (&ss)[4], int co8) {
    constexpr int zs = (K + 15) & 15;
    // ring slots: output slice o lives in slot o % 3
    constexpr int RM = K % 3, R0 = (K + 2) % 3, RP = (K + 1) % 3;
    constexpr bool PM = K <= 15, P0 = K >= 1 && K <= 16, PP = K >= 2;
    const float* x = sm + kOffX;
    float* h1 = sm + kOffH1;
    float* h2 = sm + kOffH2;
    float* st = sm + kOffST;
    conv1_slice(x, Wl + a.off.W1, Wl + a.off.b1, h1, zs, frozen, a.slope);
    __syncthreads();
    if (PM) ring_init<RM>(g, Wl + a.off.b2, co8);
    conv2_step<RM, R0, RP, PM, P0, PP>(g, h1, Wl + a.off.W2, ys, xs, co8);
    if (PP) {                                        // output slice K-2 is complete
        ring_store<RP>(g, h2, ss, co8, a.slope);
        __syncthreads();
        conv3_from(h2, Wl + a.off.W3, st, K - 2, frozen);
    }
    __syncthreads();
}

template <bool INVERSE>
__global__ void __launch_bounds__(kThr, 1) flow_fp32_c32_kernel(const C32Args a) {
    extern __shared__ __align__(16) float sm[];
    float* x = sm + kOffX;
    float* st = sm + kOffST;
    FF* red = reinterpret_cast<FF*>(sm + kOffRed);
    float* Wl = sm + kOffW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // conv2 tile of this thread: channels co8..co8+7 of sites 128 h + lane + 32 k
    const int co8 = (warp & 3) * 8, half = warp >> 2;
    int ys[4], xs[4], ss[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ss[k] = 128 * half + lane + 32 * k;
        ys[k] = ss[k] >> 4;
        xs[k] = ss[k] & 15;
    }
    const int nstage = (int)(a.stride / 4);

    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        FF sumz2{0.f, 0.f};
        if (!INVERSE) {
            if (a.z_in) {
                for (int n = tid; n < kV; n += kThr) {
                    const float v = __ldg(a.z_in + b * kV + n);
                    x[n] = v;
                    const float p = v * v;
                    ff_add(sumz2, FF{p, fmaf(v, v, -p)});
                }
            } else {
                for (int j = tid; 4 * j < kV; j += kThr) {
                    const u64x4 w = philox4x64_10(a.seed, 0ull,
                                                  u64x4{a.counter0 + (uint64_t)b, (uint64_t)j, 0ull, TAG_PRIOR});
                    float zz[4];
                    normals4_f32(w, zz);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        x[4 * j + q] = zz[q];
                        const float p = zz[q] * zz[q];
                        ff_add(sumz2, FF{p, fmaf(zz[q], zz[q], -p)});
                    }
                }
            }
            __syncthreads();
            if (a.z_out)
                for (int n = tid; n < kV; n += kThr) a.z_out[b * kV + n] = x[n];
        } else {
            for (int n = tid; n < kV; n += kThr) x[n] = __ldg(a.phi_in + b * kV + n);
        }

        FF logdet{0.f, 0.f};
        for (int li = 0; li < a.n_layers; ++li) {
            const int l = INVERSE ? a.n_layers - 1 - li : li;
            const int frozen = l & 1;
            __syncthreads();                          // previous layer done with the weights and st
            if (a.xs_out && li > 0)                   // the field after li layers (training)
                for (int n = tid; n < kV; n += kThr) a.xs_out[li * a.xs_stride + b * kV + n] = x[n];
            const float4* src = reinterpret_cast<const float4*>(a.W + (size_t)l * a.stride);
            float4* dst = reinterpret_cast<float4*>(Wl);
            for (int i = tid; i < nstage; i += kThr) dst[i] = __ldg(src + i);
            for (int i = tid; i < kL * 128 * 2; i += kThr) st[i] = 0.f;
            __syncthreads();
            Ring g;
            step<0>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<1>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<2>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<3>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<4>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<5>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<6>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<7>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<8>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<9>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<10>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<11>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<12>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<13>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<14>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<15>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<16>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            step<17>(g, sm, Wl, a, frozen, ys, xs, ss, co8);
            // every s, t is complete: affine update of the updated sites
            const float bs = Wl[a.off.b3], bt = Wl[a.off.b3 + 1];
            const int pa = frozen ^ 1;
            for (int i = tid; i < kL * 128; i += kThr) {
                const int zc = i >> 7, ai = i & 127, y = ai >> 3;
                const int xc = 2 * (ai & 7) + ((pa ^ zc ^ y) & 1);
                const float spre = st[2 * i] + bs, tt = st[2 * i + 1] + bt;
                const float s = a.use_tanh ? tanhf(spre) : spre;
                float& xv = x[(zc << 8) | (y << 4) | xc];
                if (!INVERSE) xv = fmaf(xv, expf(s), tt);
                else xv = (xv - tt) * expf(-s);
                ff_add(logdet, s);
            }
        }
        __syncthreads();

        if (INVERSE) {
            for (int n = tid; n < kV; n += kThr) {
                const float v = x[n];
                const float p = v * v;
                ff_add(sumz2, FF{p, fmaf(v, v, -p)});
                if (a.z_out) a.z_out[b * kV + n] = v;
            }
        } else {
            for (int n = tid; n < kV; n += kThr) a.phi_out[b * kV + n] = x[n];
        }
        const double ld = block_sum_ff(logdet, red);
        const double z2 = block_sum_ff(sumz2, red);
        double S = 0.0;
        if (!INVERSE && a.has_phi4) S = block_sum_ff(action_part<3>(x, kL, kV, a.c2d_ff, a.lam_ff), red);
        if (tid == 0) {
            if (a.logdet_out) a.logdet_out[b] = ld;
            const double logr = -0.5 * z2 - 0.5 * (double)kV * LOG_2PI;
            const double logq = logr - ld;
            a.logq_out[b] = logq;
            if (!INVERSE && a.has_phi4) {
                if (a.S_out) a.S_out[b] = S;
                if (a.logw_out) a.logw_out[b] = -S - logq;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ 2D L=32, C=32
// 2D slab conv2 (packed FP32 pairs as in the 3D ring): acc[k][p] holds
// channels co8 + 2p, co8 + 2p + 1 of site k; init from the bias, then one tap:
// sites k at hb + k * kstride (h1 rows of pitch kCP), weights wt[ci * 32 + co8 ..].
__device__ __forceinline__ void slab_init(f32x2 (&acc)[8][4], const float* __restrict__ b2, int co8) {
    const ulonglong2 u = *reinterpret_cast<const ulonglong2*>(b2 + co8);
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(b2 + co8 + 4);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        acc[k][0] = u.x; acc[k][1] = u.y; acc[k][2] = v.x; acc[k][3] = v.y;
    }
}
__device__ __forceinline__ void slab_tap(f32x2 (&acc)[8][4], const float* __restrict__ hb, int kstride,
                                         const float* __restrict__ wt) {
#pragma unroll 4
    for (int ci = 0; ci < kC; ++ci) {
        const ulonglong2 u = *reinterpret_cast<const ulonglong2*>(wt + ci * kC);
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(wt + ci * kC + 4);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const f32x2 hh = f2_splat(hb[k * kstride + ci]);
            acc[k][0] = f2_fma(hh, u.x, acc[k][0]);
            acc[k][1] = f2_fma(hh, u.y, acc[k][1]);
            acc[k][2] = f2_fma(hh, v.x, acc[k][2]);
            acc[k][3] = f2_fma(hh, v.y, acc[k][3]);
        }
    }
}
__device__ __forceinline__ float slab_out(const f32x2 (&acc)[8][4], int k, int j) {
    return (j & 1) ? f2_hi(acc[k][j >> 1]) : f2_lo(acc[k][j >> 1]);
}

namespace d2 {
constexpr int L = 32, V = 1024, T = 9, ROWS = 16, HROWS = ROWS + 2;
constexpr int kOffX = 0;
constexpr int kOffH1 = kOffX + V;                          // [18 rows][32][kCP]
constexpr int kOffH2 = kOffH1 + HROWS * L * kCP;           // [16 rows][32][kCP]
constexpr int kOffST = kOffH2 + ROWS * L * kCP;            // [32 rows][16 updated sites][2]
constexpr int kOffRed = kOffST + L * 16 * 2;
constexpr int kOffW = kOffRed + 64;
static_assert((kOffW * 4) % 16 == 0, "weight block alignment");
}  // namespace d2

template <bool INVERSE>
__global__ void __launch_bounds__(kThr, 1) flow_fp32_c32_2d_kernel(const C32Args a) {
    extern __shared__ __align__(16) float sm[];
    float* x = sm + d2::kOffX;
    float* h1 = sm + d2::kOffH1;
    float* h2 = sm + d2::kOffH2;
    float* st = sm + d2::kOffST;
    FF* red = reinterpret_cast<FF*>(sm + d2::kOffRed);
    float* Wl = sm + d2::kOffW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int co8 = (warp & 3) * 8, half = warp >> 2;
    const int nstage = (int)(a.stride / 4);

    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        FF sumz2{0.f, 0.f};
        if (!INVERSE) {
            if (a.z_in) {
                for (int n = tid; n < d2::V; n += kThr) {
                    const float v = __ldg(a.z_in + b * d2::V + n);
                    x[n] = v;
                    const float p = v * v;
                    ff_add(sumz2, FF{p, fmaf(v, v, -p)});
                }
            } else {
                for (int j = tid; 4 * j < d2::V; j += kThr) {
                    const u64x4 w = philox4x64_10(a.seed, 0ull,
                                                  u64x4{a.counter0 + (uint64_t)b, (uint64_t)j, 0ull, TAG_PRIOR});
                    float zz[4];
                    normals4_f32(w, zz);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        x[4 * j + q] = zz[q];
                        const float p = zz[q] * zz[q];
                        ff_add(sumz2, FF{p, fmaf(zz[q], zz[q], -p)});
                    }
                }
            }
            __syncthreads();
            if (a.z_out)
                for (int n = tid; n < d2::V; n += kThr) a.z_out[b * d2::V + n] = x[n];
        } else {
            for (int n = tid; n < d2::V; n += kThr) x[n] = __ldg(a.phi_in + b * d2::V + n);
        }

        FF logdet{0.f, 0.f};
        for (int li = 0; li < a.n_layers; ++li) {
            const int l = INVERSE ? a.n_layers - 1 - li : li;
            const int frozen = l & 1, pa = frozen ^ 1;
            __syncthreads();
            if (a.xs_out && li > 0)                   // the field after li layers (training)
                for (int n = tid; n < d2::V; n += kThr) a.xs_out[li * a.xs_stride + b * d2::V + n] = x[n];
            const float4* src = reinterpret_cast<const float4*>(a.W + (size_t)l * a.stride);
            float4* dst = reinterpret_cast<float4*>(Wl);
            for (int i = tid; i < nstage; i += kThr) dst[i] = __ldg(src + i);
            for (int i = tid; i < d2::L * 16 * 2; i += kThr) st[i] = 0.f;
            __syncthreads();
            const float* W1 = Wl + a.off.W1;
            const float* b1 = Wl + a.off.b1;
            const float* W2 = Wl + a.off.W2;
            const float* b2 = Wl + a.off.b2;
            const float* W3 = Wl + a.off.W3;
            for (int slab = 0; slab < 2; ++slab) {
                const int r0 = slab * d2::ROWS;
                // conv1 + LeakyReLU of rows r0-1 .. r0+16 (thread = site)
                for (int i = tid; i < d2::HROWS * d2::L; i += kThr) {
                    const int hr = i >> 5, xc = i & 31, y = (r0 - 1 + hr) & 31;
                    float acc[kC];
#pragma unroll
                    for (int c = 0; c < kC; c += 4) {
                        const float4 bb = *reinterpret_cast<const float4*>(b1 + c);
                        acc[c] = bb.x; acc[c + 1] = bb.y; acc[c + 2] = bb.z; acc[c + 3] = bb.w;
                    }
#pragma unroll 1
                    for (int t = 0; t < d2::T; ++t) {
                        const int yy = (y + t / 3 - 1) & 31, xx = (xc + t % 3 - 1) & 31;
                        const float xv = (((xx + yy) & 1) == frozen) ? x[(yy << 5) | xx] : 0.f;
#pragma unroll
                        for (int c = 0; c < kC; c += 4) {
                            const float4 wv = *reinterpret_cast<const float4*>(W1 + t * kC + c);
                            acc[c] = fmaf(xv, wv.x, acc[c]);
                            acc[c + 1] = fmaf(xv, wv.y, acc[c + 1]);
                            acc[c + 2] = fmaf(xv, wv.z, acc[c + 2]);
                            acc[c + 3] = fmaf(xv, wv.w, acc[c + 3]);
                        }
                    }
                    float* row = h1 + i * kCP;
#pragma unroll
                    for (int c = 0; c < kC; ++c) row[c] = lrelu(acc[c], a.slope);
                }
                __syncthreads();
                // conv2 of the 16 rows: sites 256 half + lane + 32 k (row = k + 8 half), channels co8..co8+7
                {
                    f32x2 acc[8][4];
                    slab_init(acc, b2, co8);
#pragma unroll 1
                    for (int t = 0; t < d2::T; ++t) {
                        const int dy = t / 3 - 1, dx = t % 3 - 1;
                        const int xs = (lane + dx) & 31;
                        const float* hb = h1 + ((8 * half + dy + 1) * d2::L + xs) * kCP;   // row k: + k * d2::L * kCP
                        slab_tap(acc, hb, d2::L * kCP, W2 + (size_t)t * kC * kC + co8);
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        float* row = h2 + ((8 * half + k) * d2::L + lane) * kCP + co8;
#pragma unroll
                        for (int j = 0; j < 8; ++j) row[j] = lrelu(slab_out(acc, k, j), a.slope);
                    }
                }
                __syncthreads();
                // conv3 contributions of h2 rows r0 .. r0+15 to rows r0-1 .. r0+16 (updated sites)
                for (int it = tid; it < d2::HROWS * 16; it += kThr) {
                    const int tr = it >> 4, kx = it & 15;           // target row r0 - 1 + tr
                    const int y = (r0 - 1 + tr) & 31;
                    const int xc = 2 * kx + ((pa ^ y) & 1);
                    float ps = 0.f, pt = 0.f;
                    for (int dy = -1; dy <= 1; ++dy) {
                        const int hr = tr - 1 + dy;                  // h2 row index in the slab
                        if (hr < 0 || hr >= d2::ROWS) continue;
                        for (int dx = -1; dx <= 1; ++dx) {
                            const float* row = h2 + (hr * d2::L + ((xc + dx) & 31)) * kCP;
                            const float* w = W3 + (size_t)((dy + 1) * 3 + dx + 1) * kC * 2;
#pragma unroll 8
                            for (int ci = 0; ci < kC; ++ci) {
                                const float2 wv = *reinterpret_cast<const float2*>(w + 2 * ci);
                                ps = fmaf(row[ci], wv.x, ps);
                                pt = fmaf(row[ci], wv.y, pt);
                            }
                        }
                    }
                    float* o = st + ((y << 4) | kx) * 2;
                    o[0] += ps;
                    o[1] += pt;
                }
                __syncthreads();
            }
            const float bs = Wl[a.off.b3], bt = Wl[a.off.b3 + 1];
            for (int i = tid; i < d2::L * 16; i += kThr) {
                const int y = i >> 4, xc = 2 * (i & 15) + ((pa ^ y) & 1);
                const float spre = st[2 * i] + bs, tt = st[2 * i + 1] + bt;
                const float s = a.use_tanh ? tanhf(spre) : spre;
                float& xv = x[(y << 5) | xc];
                if (!INVERSE) xv = fmaf(xv, expf(s), tt);
                else xv = (xv - tt) * expf(-s);
                ff_add(logdet, s);
            }
        }
        __syncthreads();

        if (INVERSE) {
            for (int n = tid; n < d2::V; n += kThr) {
                const float v = x[n];
                const float p = v * v;
                ff_add(sumz2, FF{p, fmaf(v, v, -p)});
                if (a.z_out) a.z_out[b * d2::V + n] = v;
            }
        } else {
            for (int n = tid; n < d2::V; n += kThr) a.phi_out[b * d2::V + n] = x[n];
        }
        const double ld = block_sum_ff(logdet, red);
        const double z2 = block_sum_ff(sumz2, red);
        double S = 0.0;
        if (!INVERSE && a.has_phi4) S = block_sum_ff(action_part<2>(x, d2::L, d2::V, a.c2d_ff, a.lam_ff), red);
        if (tid == 0) {
            if (a.logdet_out) a.logdet_out[b] = ld;
            const double logr = -0.5 * z2 - 0.5 * (double)d2::V * LOG_2PI;
            const double logq = logr - ld;
            a.logq_out[b] = logq;
            if (!INVERSE && a.has_phi4) {
                if (a.S_out) a.S_out[b] = S;
                if (a.logw_out) a.logw_out[b] = -S - logq;
            }
        }
        __syncthreads();
    }
}

// One coupling layer's network recomputed for the training reverse pass (2D
// L=32, width 32): from the layer input x_l of each configuration, h1 and h2
// (after LeakyReLU) in the channel-chunk-major activation layout of the
// training workspace ([b][c/4][V][4]) and s at the updated sites (after the
// tanh; 0 at the fixed sites), with the same slab plan as the sampler.
__global__ void __launch_bounds__(kThr, 1) c32_2d_recompute_kernel(const C32Args a, int layer, const float* __restrict__ xl,
                                                                  float* __restrict__ h1_out, float* __restrict__ h2_out,
                                                                  float* __restrict__ s_out) {
    extern __shared__ __align__(16) float sm[];
    float* x = sm + d2::kOffX;
    float* h1 = sm + d2::kOffH1;
    float* h2 = sm + d2::kOffH2;
    float* st = sm + d2::kOffST;
    float* Wl = sm + d2::kOffW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int co8 = (warp & 3) * 8, half = warp >> 2;
    const int frozen = layer & 1, pa = frozen ^ 1;
    constexpr int V = d2::V, L = d2::L;
    {
        const float4* src = reinterpret_cast<const float4*>(a.W + (size_t)layer * a.stride);
        float4* dst = reinterpret_cast<float4*>(Wl);
        for (int i = tid; i < (int)(a.stride / 4); i += kThr) dst[i] = __ldg(src + i);
    }
    const float* W1 = Wl + a.off.W1;
    const float* b1 = Wl + a.off.b1;
    const float* W2 = Wl + a.off.W2;
    const float* b2 = Wl + a.off.b2;
    const float* W3 = Wl + a.off.W3;
    // chunk-major activation layout: element (b, n, c) at ((b*8 + c/4)*V + n)*4 + c%4
    const auto chunk = [](int64_t b, int n, int c4) { return ((b * 8 + c4) * (int64_t)V + n) * 4; };
    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        __syncthreads();
        for (int n = tid; n < V; n += kThr) x[n] = __ldg(xl + b * V + n);
        for (int i = tid; i < L * 16 * 2; i += kThr) st[i] = 0.f;
        __syncthreads();
        for (int slab = 0; slab < 2; ++slab) {
            const int r0 = slab * d2::ROWS;
            for (int i = tid; i < d2::HROWS * L; i += kThr) {
                const int hr = i >> 5, xc = i & 31, y = (r0 - 1 + hr) & 31;
                float acc[kC];
#pragma unroll
                for (int c = 0; c < kC; c += 4) {
                    const float4 bb = *reinterpret_cast<const float4*>(b1 + c);
                    acc[c] = bb.x; acc[c + 1] = bb.y; acc[c + 2] = bb.z; acc[c + 3] = bb.w;
                }
#pragma unroll 1
                for (int t = 0; t < d2::T; ++t) {
                    const int yy = (y + t / 3 - 1) & 31, xx = (xc + t % 3 - 1) & 31;
                    const float xv = (((xx + yy) & 1) == frozen) ? x[(yy << 5) | xx] : 0.f;
#pragma unroll
                    for (int c = 0; c < kC; c += 4) {
                        const float4 wv = *reinterpret_cast<const float4*>(W1 + t * kC + c);
                        acc[c] = fmaf(xv, wv.x, acc[c]);
                        acc[c + 1] = fmaf(xv, wv.y, acc[c + 1]);
                        acc[c + 2] = fmaf(xv, wv.z, acc[c + 2]);
                        acc[c + 3] = fmaf(xv, wv.w, acc[c + 3]);
                    }
                }
                float* row = h1 + i * kCP;
#pragma unroll
                for (int c = 0; c < kC; ++c) row[c] = lrelu(acc[c], a.slope);
            }
            __syncthreads();
            // h1 of the slab's 16 rows to the workspace
            for (int e = tid; e < d2::ROWS * L * 8; e += kThr) {
                const int c4 = e / (d2::ROWS * L), site = e % (d2::ROWS * L);
                const float* rw = h1 + (L + site) * kCP + 4 * c4;
                *reinterpret_cast<float4*>(h1_out + chunk(b, (r0 << 5) + site, c4)) = make_float4(rw[0], rw[1], rw[2], rw[3]);
            }
            {
                f32x2 acc[8][4];
                slab_init(acc, b2, co8);
#pragma unroll 1
                for (int t = 0; t < d2::T; ++t) {
                    const int dy = t / 3 - 1, dx = t % 3 - 1;
                    const int xs = (lane + dx) & 31;
                    const float* hb = h1 + ((8 * half + dy + 1) * L + xs) * kCP;
                    slab_tap(acc, hb, L * kCP, W2 + (size_t)t * kC * kC + co8);
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    float o[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) o[j] = lrelu(slab_out(acc, k, j), a.slope);
                    float* row = h2 + ((8 * half + k) * L + lane) * kCP + co8;
#pragma unroll
                    for (int j = 0; j < 8; ++j) row[j] = o[j];
                    const int n = ((r0 + 8 * half + k) << 5) | lane;
                    *reinterpret_cast<float4*>(h2_out + chunk(b, n, co8 / 4)) = make_float4(o[0], o[1], o[2], o[3]);
                    *reinterpret_cast<float4*>(h2_out + chunk(b, n, co8 / 4 + 1)) = make_float4(o[4], o[5], o[6], o[7]);
                }
            }
            __syncthreads();
            for (int it = tid; it < d2::HROWS * 16; it += kThr) {
                const int tr = it >> 4, kx = it & 15;
                const int y = (r0 - 1 + tr) & 31;
                const int xc = 2 * kx + ((pa ^ y) & 1);
                float ps = 0.f, pt = 0.f;
                for (int dy = -1; dy <= 1; ++dy) {
                    const int hr = tr - 1 + dy;
                    if (hr < 0 || hr >= d2::ROWS) continue;
                    for (int dx = -1; dx <= 1; ++dx) {
                        const float* row = h2 + (hr * L + ((xc + dx) & 31)) * kCP;
                        const float* w = W3 + (size_t)((dy + 1) * 3 + dx + 1) * kC * 2;
#pragma unroll 8
                        for (int ci = 0; ci < kC; ++ci) {
                            const float2 wv = *reinterpret_cast<const float2*>(w + 2 * ci);
                            ps = fmaf(row[ci], wv.x, ps);
                            pt = fmaf(row[ci], wv.y, pt);
                        }
                    }
                }
                float* o = st + ((y << 4) | kx) * 2;
                o[0] += ps;
                o[1] += pt;
            }
            __syncthreads();
        }
        const float bs = Wl[a.off.b3];
        for (int n = tid; n < V; n += kThr) {
            const int y = n >> 5, xc = n & 31;
            float sv = 0.f;
            if (((xc + y) & 1) == pa) {
                const float spre = st[((y << 4) | (xc >> 1)) * 2] + bs;
                sv = a.use_tanh ? tanhf(spre) : spre;
            }
            s_out[b * V + n] = sv;
        }
    }
}

}  // namespace

bool fp32_c32_recompute_supported(const gf_flow* f) {
    return !f->variant && f->C1 == kC && f->C2 == kC && f->shape.nd == 2 && f->shape.L == d2::L && f->T == d2::T;
}

gf_status launch_c32_recompute(const gf_flow* f, int layer, int64_t B, const float* xl, float* h1_out, float* h2_out,
                               float* s_out, cudaStream_t stream) {
    C32Args a;
    std::memset(&a, 0, sizeof(a));
    a.W = f->d_packed;
    a.stride = f->packed_stride;
    a.off = packed_offsets(f->T, f->C1, f->C2);
    a.n_layers = f->shape.n_layers;
    a.slope = (float)f->shape.leaky_slope;
    a.use_tanh = f->shape.use_final_tanh;
    a.B = B;
    const size_t smem = (size_t)(d2::kOffW + f->packed_stride) * 4;
    if (cudaFuncSetAttribute(c32_2d_recompute_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return GF_ECUDA;
    const int64_t grid = std::min<int64_t>(B, (int64_t)num_sms());
    if (grid <= 0) return GF_OK;
    c32_2d_recompute_kernel<<<(unsigned)grid, kThr, smem, stream>>>(a, layer, xl, h1_out, h2_out, s_out);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

bool fp32_c32_supported(const gf_flow* f) {
    if (f->variant || f->C1 != kC || f->C2 != kC) return false;
    return (f->shape.nd == 3 && f->shape.L == kL && f->T == kT) || (f->shape.nd == 2 && f->shape.L == d2::L && f->T == d2::T);
}

size_t fp32_c32_smem(const gf_flow* f) {
    return (size_t)((f->shape.nd == 3 ? kOffW : d2::kOffW) + f->packed_stride) * 4;
}

gf_status launch_flow_fp32_c32(const gf_flow* f, bool inverse, const gf_phi4* phi4, int64_t B, uint64_t seed,
                               uint64_t counter0, const float* z_in, float* z_out, const float* phi_in,
                               float* phi_out, double* logq_out, double* S_out, double* logw_out,
                               cudaStream_t stream, float* xs_out, int64_t xs_stride, double* logdet_out) {
    C32Args a;
    std::memset(&a, 0, sizeof(a));
    a.W = f->d_packed;
    a.stride = f->packed_stride;
    a.off = packed_offsets(f->T, f->C1, f->C2);
    a.n_layers = f->shape.n_layers;
    a.slope = (float)f->shape.leaky_slope;
    a.use_tanh = f->shape.use_final_tanh;
    a.has_phi4 = phi4 != nullptr;
    ff_split(2.0 * f->shape.nd + (phi4 ? phi4->m2 : 0.0), &a.c2d_ff.hi, &a.c2d_ff.lo);
    ff_split(phi4 ? phi4->lam : 0.0, &a.lam_ff.hi, &a.lam_ff.lo);
    a.B = B; a.seed = seed; a.counter0 = counter0;
    a.z_in = z_in; a.z_out = z_out; a.phi_in = phi_in; a.phi_out = phi_out;
    a.logq_out = logq_out; a.S_out = S_out; a.logw_out = logw_out;
    a.xs_out = xs_out; a.xs_stride = xs_stride; a.logdet_out = logdet_out;
    const size_t smem = fp32_c32_smem(f);
    auto kern = f->shape.nd == 3 ? (inverse ? flow_fp32_c32_kernel<true> : flow_fp32_c32_kernel<false>)
                                 : (inverse ? flow_fp32_c32_2d_kernel<true> : flow_fp32_c32_2d_kernel<false>);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GF_ECUDA;
    const int64_t grid = std::min<int64_t>(B, (int64_t)num_sms());
    if (grid <= 0) return GF_OK;
    kern<<<(unsigned)grid, kThr, smem, stream>>>(a);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

}  // namespace gf
