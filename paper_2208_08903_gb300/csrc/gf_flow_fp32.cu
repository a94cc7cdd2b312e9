// gf_flow_fp32.cu -- fused FP32 coupling-stack kernel (both directions).
//
// Paper (arXiv:2208.08903) Sec. 1: prior sample, even/odd affine coupling
// layers x -> x*exp(s) + t with (s, t) a convolutional net of the fixed
// sites, composition of N_tri layers, Jacobian via the sum of s, model density
// log q = log r - log|det|, and the phi^4 action for log w = -S - log q.
//
// One CTA owns one configuration at a time (persistent grid-stride loop):
// the field x stays in shared memory through every layer, the hidden
// activations h1/h2 live in a slot cache of slices (see gf_flow.cuh), the
// log-det, sum z^2 and action are summed to FP64 accuracy (FP32 pairs per
// thread, see gf_common.cuh, then across the block).  Nothing but the inputs
// and the per-configuration results touches global memory: weights are read
// through the read-only path (L1/L2), or, when every layer's packed weights
// fit beside the activations (small flows such as the paper's 2D L=8 example),
// staged once per CTA in shared memory.
#include <algorithm>
#include <cstring>

#include "gf_flow.cuh"

namespace gf {

namespace {

constexpr int kThreads = 256;

struct FlowArgs {
    const float* W;            // packed weights
    const Phase* sched;
    int n_phases;
    int64_t stride;
    PackedOffsets off;
    int L, S, V, C1, C2, n_layers, R;
    float slope;
    int use_tanh;
    int has_phi4;
    double m2, lam;
    FF c2d_ff, lam_ff;       // 2 nd + m2 and lam as FP32 pairs
    int64_t B;
    uint64_t seed, counter0;
    const float* z_in;
    float* z_out;
    const float* phi_in;
    float* phi_out;
    double* logq_out;
    double* S_out;
    double* logw_out;
};

// Tap t -> offsets (ds along the slice axis, dy, dx in the slice).
template <int ND>
__device__ __forceinline__ void tap_delta(int t, int& ds, int& dy, int& dx) {
    if (ND == 3) { ds = t / 9 - 1; dy = (t / 3) % 3 - 1; dx = t % 3 - 1; }
    else { ds = t / 3 - 1; dy = 0; dx = t % 3 - 1; }
}

__device__ __forceinline__ int wrap(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// In-slice site j = y*L + x (3D) or x (2D), shifted by (dy, dx) periodically.
template <int ND>
__device__ __forceinline__ int shift_in_slice(int j, int dy, int dx, int L) {
    if (ND == 3) {
        int y = j / L, x = j - y * L;
        return wrap(y + dy, L) * L + wrap(x + dx, L);
    }
    return wrap(j + dx, L);
}
template <int ND>
__device__ __forceinline__ int coord_sum_in_slice(int j, int L) {
    if (ND == 3) { int y = j / L; return y + (j - y * L); }
    return j;
}

// Swizzled float4 chunk of a site row of C floats (conflict-free LDS.128
// when consecutive lanes read consecutive sites): xor with the site index for
// a power-of-two number of chunks, a rotation otherwise (ROT: C = 24).  ROT is
// a template parameter so the power-of-two kernels carry no division.
template <bool ROT>
__device__ __forceinline__ int swz(int chunk, int j, int C) {
    const int n = C >> 2;
    if constexpr (ROT) return (chunk + j) % n;
    else return chunk ^ (j & (n - 1));
}

__device__ __forceinline__ float lrelu(float v, float a) { return v > 0.f ? v : a * v; }

// Weight reads: through the read-only cache from global memory, or plain loads
// when the whole flow's packed weights were staged in shared memory (WS).
template <bool WS>
__device__ __forceinline__ float4 ldw4(const float* p) {
    if (WS) return *reinterpret_cast<const float4*>(p);
    return __ldg(reinterpret_cast<const float4*>(p));
}
template <bool WS>
__device__ __forceinline__ float ldw(const float* p) {
    if (WS) return *p;
    return __ldg(p);
}

// ---------------------------------------------------------------- conv1
template <int ND, bool WS, bool ROT>
__device__ void phase_h1(const FlowArgs& a, const float* __restrict__ Wl, const Phase& ph,
                         const float* x, float* h1, int frozen) {
    const int L = a.L, S = a.S, C1 = a.C1, T = (ND == 3) ? 27 : 9;
    const int nf = ph.n * S, items = nf * (C1 >> 3);
    const float* W1 = Wl + a.off.W1;
    const float* b1 = Wl + a.off.b1;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int g = it / nf, f = it - g * nf;
        const int r = f / S, j = f - r * S;
        const int sl = wrap(ph.s0 + r, L);
        const int co = g << 3;
        float acc[8];
        const float4 bb0 = ldw4<WS>(b1 + co);
        const float4 bb1 = ldw4<WS>(b1 + co + 4);
        acc[0] = bb0.x; acc[1] = bb0.y; acc[2] = bb0.z; acc[3] = bb0.w;
        acc[4] = bb1.x; acc[5] = bb1.y; acc[6] = bb1.z; acc[7] = bb1.w;
        for (int t = 0; t < T; ++t) {
            int ds, dy, dx;
            tap_delta<ND>(t, ds, dy, dx);
            const int sl2 = wrap(sl + ds, L);
            const int j2 = shift_in_slice<ND>(j, dy, dx, L);
            const int par = (sl2 + coord_sum_in_slice<ND>(j2, L)) & 1;
            const float xv = (par == frozen) ? x[sl2 * S + j2] : 0.f;
            const float4 w0 = ldw4<WS>(W1 + t * C1 + co);
            const float4 w1 = ldw4<WS>(W1 + t * C1 + co + 4);
            acc[0] = fmaf(xv, w0.x, acc[0]); acc[1] = fmaf(xv, w0.y, acc[1]);
            acc[2] = fmaf(xv, w0.z, acc[2]); acc[3] = fmaf(xv, w0.w, acc[3]);
            acc[4] = fmaf(xv, w1.x, acc[4]); acc[5] = fmaf(xv, w1.y, acc[5]);
            acc[6] = fmaf(xv, w1.z, acc[6]); acc[7] = fmaf(xv, w1.w, acc[7]);
        }
        float* row = h1 + ((size_t)ph.out[r] * S + j) * C1;
        const float4 o0 = make_float4(lrelu(acc[0], a.slope), lrelu(acc[1], a.slope),
                                      lrelu(acc[2], a.slope), lrelu(acc[3], a.slope));
        const float4 o1 = make_float4(lrelu(acc[4], a.slope), lrelu(acc[5], a.slope),
                                      lrelu(acc[6], a.slope), lrelu(acc[7], a.slope));
        *reinterpret_cast<float4*>(row + (swz<ROT>(co >> 2, j, C1) << 2)) = o0;
        *reinterpret_cast<float4*>(row + (swz<ROT>((co >> 2) + 1, j, C1) << 2)) = o1;
    }
}

// ---------------------------------------------------------------- conv2
// Warp task = 128 consecutive chunk sites x 8 output channels; lane i owns
// sites i, i+32, i+64, i+96 (register tile 4 x 8), weights are warp-uniform.
template <int ND, bool WS, bool ROT>
__device__ void phase_h2(const FlowArgs& a, const float* __restrict__ Wl, const Phase& ph,
                         const float* h1, float* h2) {
    const int L = a.L, S = a.S, C1 = a.C1, C2 = a.C2, T = (ND == 3) ? 27 : 9;
    const int nf = ph.n * S, nblk = (nf + 127) >> 7, ngrp = C2 >> 3;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const float* W2 = Wl + a.off.W2;
    const float* b2 = Wl + a.off.b2;
    const size_t slot_sz = (size_t)S * C1;
    for (int task = warp; task < nblk * ngrp; task += nwarps) {
        const int blk = task % nblk, g = task / nblk, co = g << 3;
        int rr[4], jj[4];
        bool valid[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int f = (blk << 7) + lane + 32 * k;
            valid[k] = f < nf;
            if (!valid[k]) f = nf - 1;
            rr[k] = f / S;
            jj[k] = f - rr[k] * S;
        }
        float acc[4][8];
        {
            const float4 bb0 = ldw4<WS>(b2 + co);
            const float4 bb1 = ldw4<WS>(b2 + co + 4);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                acc[k][0] = bb0.x; acc[k][1] = bb0.y; acc[k][2] = bb0.z; acc[k][3] = bb0.w;
                acc[k][4] = bb1.x; acc[k][5] = bb1.y; acc[k][6] = bb1.z; acc[k][7] = bb1.w;
            }
        }
        for (int t = 0; t < T; ++t) {
            int ds, dy, dx;
            tap_delta<ND>(t, ds, dy, dx);
            const float* row[4];
            int key[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j2 = shift_in_slice<ND>(jj[k], dy, dx, L);
                row[k] = h1 + ph.in[rr[k] + 1 + ds] * slot_sz + (size_t)j2 * C1;
                key[k] = j2;
            }
            const float* Wt = W2 + (size_t)t * C1 * C2 + co;
            for (int c4 = 0; c4 < (C1 >> 2); ++c4) {
                float4 hv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    hv[k] = *reinterpret_cast<const float4*>(row[k] + (swz<ROT>(c4, key[k], C1) << 2));
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const float* wp = Wt + (size_t)(4 * c4 + cc) * C2;
                    const float4 wa = ldw4<WS>(wp);
                    const float4 wb = ldw4<WS>(wp + 4);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float h = cc == 0 ? hv[k].x : cc == 1 ? hv[k].y : cc == 2 ? hv[k].z : hv[k].w;
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
            float* orow = h2 + ((size_t)ph.out[rr[k]] * S + jj[k]) * C2;
            const float4 o0 = make_float4(lrelu(acc[k][0], a.slope), lrelu(acc[k][1], a.slope),
                                          lrelu(acc[k][2], a.slope), lrelu(acc[k][3], a.slope));
            const float4 o1 = make_float4(lrelu(acc[k][4], a.slope), lrelu(acc[k][5], a.slope),
                                          lrelu(acc[k][6], a.slope), lrelu(acc[k][7], a.slope));
            *reinterpret_cast<float4*>(orow + (swz<ROT>(co >> 2, jj[k], C2) << 2)) = o0;
            *reinterpret_cast<float4*>(orow + (swz<ROT>((co >> 2) + 1, jj[k], C2) << 2)) = o1;
        }
    }
}

// ---------------------------------------------------------------- conv3 + affine update
// (s, t) at the updated sites only; `tps` lanes share a site, each summing
// C2/tps channels, combined with xor-shuffles.
template <int ND, bool INVERSE, bool WS, bool ROT>
__device__ void phase_c3(const FlowArgs& a, const float* __restrict__ Wl, const Phase& ph,
                         const float* h2, float* x, int frozen, FF& logdet) {
    const int L = a.L, S = a.S, C2 = a.C2, T = (ND == 3) ? 27 : 9;
    const int half = S >> 1, nact = ph.n * half;
    int tps = 1;
    while (tps * 2 <= (C2 >> 2) && (C2 >> 2) % (tps * 2) == 0 && nact * tps * 2 <= (int)blockDim.x) tps *= 2;
    const int nchunk = (C2 >> 2) / tps;
    const int total = nact * tps;
    const float* W3 = Wl + a.off.W3;
    const float bs = ldw<WS>(Wl + a.off.b3), bt = ldw<WS>(Wl + a.off.b3 + 1);
    const size_t slot_sz = (size_t)S * C2;
    const int iters = (total + blockDim.x - 1) / blockDim.x;
    for (int i = 0; i < iters; ++i) {
        const int it = i * blockDim.x + threadIdx.x;
        const bool valid = it < total;
        const int ai = valid ? it / tps : 0, rk = it % tps;
        const int r = ai / half, aa = ai - r * half;
        const int sl = wrap(ph.s0 + r, L);
        int j;
        if (ND == 3) {
            const int hl = L >> 1, y = aa / hl, k = aa - y * hl;
            j = y * L + 2 * k + ((frozen ^ 1 ^ sl ^ y) & 1);
        } else {
            j = 2 * aa + ((frozen ^ 1 ^ sl) & 1);
        }
        float ps = 0.f, pt = 0.f;
        if (valid) {
            for (int t = 0; t < T; ++t) {
                int ds, dy, dx;
                tap_delta<ND>(t, ds, dy, dx);
                const int j2 = shift_in_slice<ND>(j, dy, dx, L);
                const float* row = h2 + ph.in[r + 1 + ds] * slot_sz + (size_t)j2 * C2;

                const float* Wt = W3 + (size_t)t * C2 * 2;
                for (int c = 0; c < nchunk; ++c) {
                    const int c4 = rk * nchunk + c;
                    const float4 hv = *reinterpret_cast<const float4*>(row + (swz<ROT>(c4, j2, C2) << 2));
                    const float4 w01 = ldw4<WS>(Wt + 8 * c4);
                    const float4 w23 = ldw4<WS>(Wt + 8 * c4 + 4);
                    ps = fmaf(hv.x, w01.x, ps); pt = fmaf(hv.x, w01.y, pt);
                    ps = fmaf(hv.y, w01.z, ps); pt = fmaf(hv.y, w01.w, pt);
                    ps = fmaf(hv.z, w23.x, ps); pt = fmaf(hv.z, w23.y, pt);
                    ps = fmaf(hv.w, w23.z, ps); pt = fmaf(hv.w, w23.w, pt);
                }
            }
        }
        for (int o = 1; o < tps; o <<= 1) {
            ps += __shfl_xor_sync(0xffffffffu, ps, o);
            pt += __shfl_xor_sync(0xffffffffu, pt, o);
        }
        if (valid && rk == 0) {
            const float spre = ps + bs, tt = pt + bt;
            const float s = a.use_tanh ? tanhf(spre) : spre;
            float& xv = x[sl * S + j];
            if (!INVERSE) xv = fmaf(xv, expf(s), tt);
            else xv = (xv - tt) * expf(-s);
            ff_add(logdet, s);
        }
    }
}

template <int ND, bool INVERSE, bool WS, bool ROT>
__global__ void __launch_bounds__(kThreads) flow_fp32_kernel(const FlowArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int V = a.V;
    const int Vpad = (V + 3) & ~3;
    float* x = reinterpret_cast<float*>(smem_raw);
    float* h1 = x + Vpad;
    float* h2 = h1 + (size_t)a.R * a.S * a.C1;
    double* red = reinterpret_cast<double*>(h2 + (size_t)a.R * a.S * a.C2);   // 32 doubles
    Phase* ph = reinterpret_cast<Phase*>(red + 32);
    // optional copy of every layer's packed weights (16-byte aligned after the phase header)
    float* wsm = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(ph) + ((sizeof(Phase) + 15) & ~size_t(15)));
    if (WS) {
        const float4* src = reinterpret_cast<const float4*>(a.W);
        float4* dst = reinterpret_cast<float4*>(wsm);
        const int64_t n4 = (int64_t)a.n_layers * a.stride / 4;
        for (int64_t i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = __ldg(src + i);
        __syncthreads();
    }
    const float* Wbase = WS ? wsm : a.W;

    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        FF sumz2{0.f, 0.f};                        // sum z^2: each square exactly as a pair
        if (!INVERSE) {
            if (a.z_in) {
                for (int n = threadIdx.x; n < V; n += blockDim.x) {
                    const float v = __ldg(a.z_in + b * V + n);
                    x[n] = v;
                    const float p = v * v;
                    ff_add(sumz2, FF{p, fmaf(v, v, -p)});
                }
            } else {
                for (int j = threadIdx.x; 4 * j < V; j += blockDim.x) {
                    const u64x4 w = philox4x64_10(a.seed, 0ull,
                                                  u64x4{a.counter0 + (uint64_t)b, (uint64_t)j, 0ull, TAG_PRIOR});
                    float zz[4];
                    normals4_f32(w, zz);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (4 * j + q < V) {
                            x[4 * j + q] = zz[q];
                            const float p = zz[q] * zz[q];
                            ff_add(sumz2, FF{p, fmaf(zz[q], zz[q], -p)});
                        }
                    }
                }
            }
            __syncthreads();
            if (a.z_out)
                for (int n = threadIdx.x; n < V; n += blockDim.x) a.z_out[b * V + n] = x[n];
        } else {
            for (int n = threadIdx.x; n < V; n += blockDim.x) x[n] = __ldg(a.phi_in + b * V + n);
        }
        __syncthreads();

        FF logdet{0.f, 0.f};
        for (int li = 0; li < a.n_layers; ++li) {
            const int l = INVERSE ? a.n_layers - 1 - li : li;
            const int frozen = l & 1;
            const float* Wl = Wbase + (size_t)l * a.stride;
            for (int p = 0; p < a.n_phases; ++p) {
                if (threadIdx.x < (int)(sizeof(Phase) / 4))
                    reinterpret_cast<uint32_t*>(ph)[threadIdx.x] =
                        __ldg(reinterpret_cast<const uint32_t*>(a.sched + p) + threadIdx.x);
                __syncthreads();
                if (ph->type == PH_H1) phase_h1<ND, WS, ROT>(a, Wl, *ph, x, h1, frozen);
                else if (ph->type == PH_H2) phase_h2<ND, WS, ROT>(a, Wl, *ph, h1, h2);
                else phase_c3<ND, INVERSE, WS, ROT>(a, Wl, *ph, h2, x, frozen, logdet);
                __syncthreads();
            }
        }

        if (INVERSE) {
            for (int n = threadIdx.x; n < V; n += blockDim.x) {
                const float v = x[n];
                const float p = v * v;
                ff_add(sumz2, FF{p, fmaf(v, v, -p)});
                if (a.z_out) a.z_out[b * V + n] = v;
            }
        } else {
            for (int n = threadIdx.x; n < V; n += blockDim.x) a.phi_out[b * V + n] = x[n];
        }
        FF* red_ff = reinterpret_cast<FF*>(red);
        const double ld = block_sum_ff(logdet, red_ff);
        const double z2 = block_sum_ff(sumz2, red_ff);
        double S = 0.0;
        if (!INVERSE && a.has_phi4) S = block_sum_ff(action_part<ND>(x, a.L, V, a.c2d_ff, a.lam_ff), red_ff);
        if (threadIdx.x == 0) {
            const double logr = -0.5 * z2 - 0.5 * (double)V * LOG_2PI;
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

template <int ND, bool INV, bool WS>
gf_status launch_t(const gf_flow* f, const FlowArgs& a, cudaStream_t stream) {
    const int n1 = f->C1 >> 2, n2 = f->C2 >> 2;      // float4 chunks per row (C1 == C2 here)
    const bool rot = (n1 & (n1 - 1)) != 0 || (n2 & (n2 - 1)) != 0;
    auto kern = rot ? flow_fp32_kernel<ND, INV, WS, true> : flow_fp32_kernel<ND, INV, WS, false>;
    static int configured_bytes[2] = {0, 0};   // per-instantiation attribute cache
    (void)configured_bytes;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)f->smem_bytes) != cudaSuccess)
        return GF_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, f->smem_bytes) !=
            cudaSuccess || per_sm < 1)
        return GF_ECUDA;
    const int64_t grid = std::min<int64_t>(a.B, (int64_t)num_sms() * per_sm);
    if (grid <= 0) return GF_OK;
    kern<<<(unsigned)grid, kThreads, f->smem_bytes, stream>>>(a);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

}  // namespace

size_t flow_fp32_smem(const gf_flow* f, int R) {
    const size_t Vpad = (f->V + 3) & ~3;
    return Vpad * 4 + (size_t)R * f->S * (f->C1 + f->C2) * 4 + 32 * 8 + ((sizeof(Phase) + 15) & ~size_t(15));
}

gf_status flow_fp32_configure(gf_flow* f) {
    constexpr size_t kBudget = 227 * 1024;
    const int L = f->shape.L;
    if (L <= MAX_PHASE_SLICES && flow_fp32_smem(f, L) <= kBudget) {
        f->full = true; f->G = L; f->R = L;
    } else {
        int G = std::min(MAX_PHASE_SLICES, L - 3);
        while (G >= 1 && flow_fp32_smem(f, G + 2) > kBudget) --G;
        if (G < 1) return GF_EUNSUPPORTED;
        f->full = false; f->G = G; f->R = G + 2;
    }
    f->smem_bytes = flow_fp32_smem(f, f->R);
    // small flows: keep every layer's packed weights in shared memory as well
    const size_t wbytes = (size_t)f->shape.n_layers * (size_t)f->packed_stride * 4;
    f->wsmem = f->smem_bytes + wbytes <= kBudget && wbytes > 0;
    if (f->wsmem) f->smem_bytes += wbytes;
    return GF_OK;
}

gf_status launch_flow_fp32(const gf_flow* f, bool inverse, const gf_phi4* phi4, int64_t B,
                           uint64_t seed, uint64_t counter0, const float* z_in, float* z_out,
                           const float* phi_in, float* phi_out, double* logq_out,
                           double* S_out, double* logw_out, cudaStream_t stream) {
    if (fp32_c32_supported(f))
        return launch_flow_fp32_c32(f, inverse, phi4, B, seed, counter0, z_in, z_out, phi_in, phi_out, logq_out,
                                    S_out, logw_out, stream);
    FlowArgs a;
    std::memset(&a, 0, sizeof(a));
    a.W = f->d_packed;
    a.sched = f->d_sched;
    a.n_phases = f->n_phases;
    a.stride = f->packed_stride;
    a.off = packed_offsets(f->T, f->C1, f->C2);
    a.L = f->shape.L; a.S = f->S; a.V = f->V; a.C1 = f->C1; a.C2 = f->C2;
    a.n_layers = f->shape.n_layers; a.R = f->R;
    a.slope = (float)f->shape.leaky_slope;
    a.use_tanh = f->shape.use_final_tanh;
    a.has_phi4 = phi4 != nullptr;
    a.m2 = phi4 ? phi4->m2 : 0.0;
    a.lam = phi4 ? phi4->lam : 0.0;
    ff_split(2.0 * f->shape.nd + a.m2, &a.c2d_ff.hi, &a.c2d_ff.lo);
    ff_split(a.lam, &a.lam_ff.hi, &a.lam_ff.lo);
    a.B = B; a.seed = seed; a.counter0 = counter0;
    a.z_in = z_in; a.z_out = z_out; a.phi_in = phi_in; a.phi_out = phi_out;
    a.logq_out = logq_out; a.S_out = S_out; a.logw_out = logw_out;
    if (f->wsmem) {
        if (f->shape.nd == 3)
            return inverse ? launch_t<3, true, true>(f, a, stream) : launch_t<3, false, true>(f, a, stream);
        return inverse ? launch_t<2, true, true>(f, a, stream) : launch_t<2, false, true>(f, a, stream);
    }
    if (f->shape.nd == 3)
        return inverse ? launch_t<3, true, false>(f, a, stream) : launch_t<3, false, false>(f, a, stream);
    return inverse ? launch_t<2, true, false>(f, a, stream) : launch_t<2, false, false>(f, a, stream);
}

}  // namespace gf
