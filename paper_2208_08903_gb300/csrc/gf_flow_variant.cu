// gf_flow_variant.cu -- fused FP32 coupling-stack kernel for the general s/t
// network of the paper's model section (Sec. 3, model parameters
// hidden_sizes and kernel_size): any list of up to GF_MAX_HIDDEN hidden
// convolutions of any width (LeakyReLU after each), an odd kernel size
// (k^nd taps, circular padding (k-1)/2), then the head conv(-> 2) giving s
// (tanh when use_final_tanh) and t.  The coupling layers, log-det, log q, the
// action and log w are those of Sec. 1, as in gf_flow_fp32.cu.
//
// One CTA owns one configuration at a time (persistent grid-stride loop).
// The whole lattice stays in shared memory through every layer: the field x
// and two ping-pong activation buffers [V][Cp], Cp = the widest hidden layer
// rounded up to an odd number of floats, so that lanes reading consecutive
// sites' rows hit distinct banks.  A thread computes up to 8 output channels
// of one site; consecutive lanes take consecutive sites of the same channel
// group, so every weight load is warp-uniform (one broadcast transaction per
// warp, through L1/L2).  Supported while x and both buffers fit in the
// 227 KB of shared memory (gf_flow_create_ex returns GF_EUNSUPPORTED
// otherwise); the paper's example network keeps the slice-cached kernels.
#include <algorithm>
#include <cstring>

#include "gf_flow.cuh"

namespace gf {

namespace {

struct VarArgs {
    const float* W;                        // packed weights, layer stride `stride`
    int64_t stride;
    int32_t woff[GF_MAX_HIDDEN + 1];       // conv j: W[t][cin][cop] (layer-relative)
    int32_t boff[GF_MAX_HIDDEN + 1];       // conv j: bias[cop]
    int32_t cin[GF_MAX_HIDDEN + 1], cout[GF_MAX_HIDDEN + 1], cop[GF_MAX_HIDDEN + 1];
    int nh, K, L, V, Cp, n_layers;
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
};

// v mod L for |v| < 2L + 8 (offsets are at most (k-1)/2 <= 3 from a site).
__device__ __forceinline__ int wrapv(int v, int L) {
    while (v < 0) v += L;
    while (v >= L) v -= L;
    return v;
}
__device__ __forceinline__ float lrelu(float v, float a) { return v > 0.f ? v : a * v; }

// Site n -> coordinates (x fastest).
template <int ND>
__device__ __forceinline__ void site_xyz(int n, int L, int& xc, int& yc, int& zc) {
    xc = n % L;
    yc = (n / L) % L;
    zc = ND == 3 ? n / (L * L) : 0;
}

// conv j >= 1 of the hidden chain: out = LReLU(conv_j(in)), rows of Cp floats.
// conv 0 (j == 0) reads the masked field instead: x at sites of parity
// `frozen`, zero elsewhere (one input channel).
template <int ND, bool FIRST>
__device__ void hidden_conv(const VarArgs& a, const float* __restrict__ Wl, int j, const float* x,
                            int frozen, const float* in, float* out) {
    const int cin = FIRST ? 1 : a.cin[j], cout = a.cout[j], cop = a.cop[j];
    const int ngrp = (cop + 7) >> 3, V = a.V, L = a.L, K = a.K, h = (K - 1) >> 1, Cp = a.Cp;
    const float* W = Wl + a.woff[j];
    const float* bias = Wl + a.boff[j];
    for (int it = threadIdx.x; it < V * ngrp; it += blockDim.x) {
        const int g = it / V, n = it - g * V, co = g << 3;
        const bool eight = co + 4 < cop;
        float acc[8];
        {
            const float4 b0 = __ldg(reinterpret_cast<const float4*>(bias + co));
            const float4 b1 = eight ? __ldg(reinterpret_cast<const float4*>(bias + co + 4)) : make_float4(0.f, 0.f, 0.f, 0.f);
            acc[0] = b0.x; acc[1] = b0.y; acc[2] = b0.z; acc[3] = b0.w;
            acc[4] = b1.x; acc[5] = b1.y; acc[6] = b1.z; acc[7] = b1.w;
        }
        int xc, yc, zc;
        site_xyz<ND>(n, L, xc, yc, zc);
        int t = 0;
        for (int kz = 0; kz < (ND == 3 ? K : 1); ++kz) {
            const int zz = ND == 3 ? wrapv(zc + kz - h, L) : 0;
            for (int ky = 0; ky < K; ++ky) {
                const int yy = wrapv(yc + ky - h, L);
                const int rowbase = (zz * L + yy) * L;
                for (int kx = 0; kx < K; ++kx, ++t) {
                    const int xx = wrapv(xc + kx - h, L);
                    const int m = rowbase + xx;
                    for (int ci = 0; ci < cin; ++ci) {
                        float v;
                        if (FIRST) v = (((xx + yy + zz) & 1) == frozen) ? x[m] : 0.f;
                        else v = in[m * Cp + ci];
                        const float* wp = W + ((size_t)t * cin + ci) * cop + co;
                        const float4 w0 = __ldg(reinterpret_cast<const float4*>(wp));
                        acc[0] = fmaf(v, w0.x, acc[0]); acc[1] = fmaf(v, w0.y, acc[1]);
                        acc[2] = fmaf(v, w0.z, acc[2]); acc[3] = fmaf(v, w0.w, acc[3]);
                        if (eight) {
                            const float4 w1 = __ldg(reinterpret_cast<const float4*>(wp + 4));
                            acc[4] = fmaf(v, w1.x, acc[4]); acc[5] = fmaf(v, w1.y, acc[5]);
                            acc[6] = fmaf(v, w1.z, acc[6]); acc[7] = fmaf(v, w1.w, acc[7]);
                        }
                    }
                }
            }
        }
        float* orow = out + (size_t)n * Cp + co;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (co + q < cout) orow[q] = lrelu(acc[q], a.slope);
    }
}

// Head conv(-> s, t) at the updated sites of this layer and the affine
// update of x there (x * e^s + t, or (x - t) e^-s inverting), log-det += s.
// Its input is the last hidden activation, or the masked field when the net
// has no hidden layer (the head then reads only fixed sites, which this
// layer does not change).
template <int ND, bool INVERSE>
__device__ void head_conv(const VarArgs& a, const float* __restrict__ Wl, const float* in, float* x,
                          int frozen, FF& logdet) {
    const int j = a.nh, cin = a.nh == 0 ? 1 : a.cin[j];
    const int V = a.V, L = a.L, K = a.K, h = (K - 1) >> 1, Cp = a.Cp, half = L >> 1;
    const float* W = Wl + a.woff[j];                  // [T][cin][4]: (s, t, 0, 0)
    const float bs = __ldg(Wl + a.boff[j]), bt = __ldg(Wl + a.boff[j] + 1);
    const int pa = frozen ^ 1;                        // parity of the updated sites
    for (int ai = threadIdx.x; ai < (V >> 1); ai += blockDim.x) {
        const int r = ai / half, k = ai - r * half;  // row r = y + L z, k-th updated site in it
        const int yc = r % L, zc = ND == 3 ? r / L : 0;
        const int xc = 2 * k + ((pa ^ yc ^ zc) & 1);
        const int n = (zc * L + yc) * L + xc;
        float ps = bs, pt = bt;
        int t = 0;
        for (int kz = 0; kz < (ND == 3 ? K : 1); ++kz) {
            const int zz = ND == 3 ? wrapv(zc + kz - h, L) : 0;
            for (int ky = 0; ky < K; ++ky) {
                const int yy = wrapv(yc + ky - h, L);
                const int rowbase = (zz * L + yy) * L;
                for (int kx = 0; kx < K; ++kx, ++t) {
                    const int xx = wrapv(xc + kx - h, L);
                    const int m = rowbase + xx;
                    for (int ci = 0; ci < cin; ++ci) {
                        float v;
                        if (a.nh == 0) v = (((xx + yy + zz) & 1) == frozen) ? x[m] : 0.f;
                        else v = in[m * Cp + ci];
                        const float2 w = __ldg(reinterpret_cast<const float2*>(W + ((size_t)t * cin + ci) * 4));
                        ps = fmaf(v, w.x, ps);
                        pt = fmaf(v, w.y, pt);
                    }
                }
            }
        }
        const float s = a.use_tanh ? tanhf(ps) : ps;
        float& xv = x[n];
        if (!INVERSE) xv = fmaf(xv, expf(s), pt);
        else xv = (xv - pt) * expf(-s);
        ff_add(logdet, s);
    }
}

template <int ND, bool INVERSE>
__global__ void __launch_bounds__(256) flow_variant_kernel(const VarArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int V = a.V;
    const int Vpad = (V + 3) & ~3;
    float* x = reinterpret_cast<float*>(smem_raw);
    float* bufA = x + Vpad;
    float* bufB = bufA + (size_t)V * a.Cp;
    FF* red = reinterpret_cast<FF*>(x + (((size_t)Vpad + 2 * (size_t)V * a.Cp + 1) & ~size_t(1)));

    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        FF sumz2{0.f, 0.f};
        if (!INVERSE) {
            if (a.z_in) {
                for (int n = threadIdx.x; n < V; n += blockDim.x) {
                    const float v = __ldg(a.z_in + b * V + n);
                    x[n] = v;
                    const float p = v * v;
                    ff_add(sumz2, FF{p, fmaf(v, v, -p)});
                }
            } else {
                for (int jq = threadIdx.x; 4 * jq < V; jq += blockDim.x) {
                    const u64x4 w = philox4x64_10(a.seed, 0ull,
                                                  u64x4{a.counter0 + (uint64_t)b, (uint64_t)jq, 0ull, TAG_PRIOR});
                    float zz[4];
                    normals4_f32(w, zz);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (4 * jq + q < V) {
                            x[4 * jq + q] = zz[q];
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
            const float* Wl = a.W + (size_t)l * a.stride;
            float* cur = bufA;
            float* nxt = bufB;
            if (a.nh > 0) {
                hidden_conv<ND, true>(a, Wl, 0, x, frozen, nullptr, cur);
                __syncthreads();
                for (int j = 1; j < a.nh; ++j) {
                    hidden_conv<ND, false>(a, Wl, j, x, frozen, cur, nxt);
                    __syncthreads();
                    float* tmp = cur; cur = nxt; nxt = tmp;
                }
            }
            head_conv<ND, INVERSE>(a, Wl, cur, x, frozen, logdet);
            __syncthreads();
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
        const double ld = block_sum_ff(logdet, red);
        const double z2 = block_sum_ff(sumz2, red);
        double S = 0.0;
        if (!INVERSE && a.has_phi4) S = block_sum_ff(action_part<ND>(x, a.L, V, a.c2d_ff, a.lam_ff), red);
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

// Canonical FP32 weights -> variant packed layout.  Canonical per layer, for
// each conv j: W_j[o][i][t] then b_j[o]; packed: W_j[t][i][cop] at woff[j]
// (o fastest, zero-padded to cop) and b_j[cop] at boff[j].
struct VarRepack {
    int32_t coff[GF_MAX_HIDDEN + 2];       // canonical start of conv j in a layer (j = nh+1: end)
    int32_t woff[GF_MAX_HIDDEN + 1], boff[GF_MAX_HIDDEN + 1];
    int32_t cin[GF_MAX_HIDDEN + 1], cout[GF_MAX_HIDDEN + 1], cop[GF_MAX_HIDDEN + 1];
    int nh, T, n_layers;
    int64_t cstride, pstride;
};

__global__ void repack_variant_kernel(const float* __restrict__ canon, float* __restrict__ packed, const VarRepack r) {
    const int64_t total = (int64_t)r.n_layers * r.cstride;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / r.cstride);
        const int q = (int)(i - (int64_t)l * r.cstride);
        int j = 0;
        while (j < r.nh && q >= r.coff[j + 1]) ++j;
        const int k = q - r.coff[j];
        const int nw = r.cout[j] * r.cin[j] * r.T;
        float* P = packed + (int64_t)l * r.pstride;
        if (k < nw) {
            const int o = k / (r.cin[j] * r.T), ci = (k / r.T) % r.cin[j], t = k % r.T;
            P[r.woff[j] + ((int64_t)t * r.cin[j] + ci) * r.cop[j] + o] = canon[i];
        } else {
            P[r.boff[j] + (k - nw)] = canon[i];
        }
    }
}

VarRepack repack_plan(const gf_flow* f) {
    VarRepack r;
    std::memset(&r, 0, sizeof(r));
    r.nh = f->n_hidden;
    r.T = f->T;
    r.n_layers = f->shape.n_layers;
    r.cstride = f->canon_stride;
    r.pstride = f->vstride;
    int32_t c = 0;
    for (int j = 0; j <= f->n_hidden; ++j) {
        r.coff[j] = c;
        r.cin[j] = f->vcin[j];
        r.cout[j] = f->vcout[j];
        r.cop[j] = f->vcop[j];
        r.woff[j] = f->vwoff[j];
        r.boff[j] = f->vboff[j];
        c += r.cout[j] * r.cin[j] * r.T + r.cout[j];
    }
    r.coff[f->n_hidden + 1] = c;
    return r;
}

template <int ND, bool INV>
gf_status launch_v(const gf_flow* f, const VarArgs& a, cudaStream_t stream) {
    auto kern = flow_variant_kernel<ND, INV>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f->smem_bytes) != cudaSuccess)
        return GF_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, f->vthreads, f->smem_bytes) != cudaSuccess ||
        per_sm < 1)
        return GF_ECUDA;
    const int64_t grid = std::min<int64_t>(a.B, (int64_t)num_sms() * per_sm);
    if (grid <= 0) return GF_OK;
    kern<<<(unsigned)grid, f->vthreads, f->smem_bytes, stream>>>(a);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

}  // namespace

// Plans the variant network: packed offsets, shared-memory size and block size.
gf_status variant_configure(gf_flow* f) {
    constexpr size_t kBudget = 227 * 1024;
    const int nh = f->n_hidden;
    int cmax = 1;
    int64_t off = 0;
    for (int j = 0; j <= nh; ++j) {
        f->vcin[j] = j == 0 ? 1 : f->hidden[j - 1];
        f->vcout[j] = j == nh ? 2 : f->hidden[j];
        f->vcop[j] = (f->vcout[j] + 3) & ~3;
        f->vwoff[j] = (int32_t)off;
        off += (int64_t)f->T * f->vcin[j] * f->vcop[j];
        f->vboff[j] = (int32_t)off;
        off += f->vcop[j];
        if (j < nh) cmax = std::max(cmax, f->hidden[j]);
    }
    f->vstride = (off + 3) & ~int64_t(3);
    f->Cp = nh == 0 ? 1 : (cmax | 1);
    const size_t Vpad = (f->V + 3) & ~3;
    const size_t floats = ((Vpad + 2 * (size_t)f->V * f->Cp + 1) & ~size_t(1)) + 2 * 32;
    f->smem_bytes = floats * 4;
    if (f->smem_bytes > kBudget) return GF_EUNSUPPORTED;
    // threads: enough for the widest conv's (site, channel-group) items, 64..256
    int items = f->V / 2;
    for (int j = 0; j < nh; ++j) items = std::max(items, f->V * ((f->vcop[j] + 7) / 8));
    f->vthreads = std::max(64, std::min(256, (items + 31) & ~31));
    return GF_OK;
}

gf_status repack_variant(gf_flow* f, cudaStream_t stream) {
    const VarRepack r = repack_plan(f);
    const int64_t total = f->n_params;
    if (total == 0) return GF_OK;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 4096);
    repack_variant_kernel<<<grid, 256, 0, stream>>>(f->d_canon, f->d_vpacked, r);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

gf_status launch_flow_variant(const gf_flow* f, bool inverse, const gf_phi4* phi4, int64_t B,
                              uint64_t seed, uint64_t counter0, const float* z_in, float* z_out,
                              const float* phi_in, float* phi_out, double* logq_out,
                              double* S_out, double* logw_out, cudaStream_t stream) {
    VarArgs a;
    std::memset(&a, 0, sizeof(a));
    a.W = f->d_vpacked;
    a.stride = f->vstride;
    for (int j = 0; j <= f->n_hidden; ++j) {
        a.woff[j] = f->vwoff[j];
        a.boff[j] = f->vboff[j];
        a.cin[j] = f->vcin[j];
        a.cout[j] = f->vcout[j];
        a.cop[j] = f->vcop[j];
    }
    a.nh = f->n_hidden;
    a.K = f->K;
    a.L = f->shape.L;
    a.V = f->V;
    a.Cp = f->Cp;
    a.n_layers = f->shape.n_layers;
    a.slope = (float)f->shape.leaky_slope;
    a.use_tanh = f->shape.use_final_tanh;
    a.has_phi4 = phi4 != nullptr;
    ff_split(2.0 * f->shape.nd + (phi4 ? phi4->m2 : 0.0), &a.c2d_ff.hi, &a.c2d_ff.lo);
    ff_split(phi4 ? phi4->lam : 0.0, &a.lam_ff.hi, &a.lam_ff.lo);
    a.B = B;
    a.seed = seed;
    a.counter0 = counter0;
    a.z_in = z_in; a.z_out = z_out; a.phi_in = phi_in; a.phi_out = phi_out;
    a.logq_out = logq_out; a.S_out = S_out; a.logw_out = logw_out;
    if (f->shape.nd == 3)
        return inverse ? launch_v<3, true>(f, a, stream) : launch_v<3, false>(f, a, stream);
    return inverse ? launch_v<2, true>(f, a, stream) : launch_v<2, false>(f, a, stream);
}

}  // namespace gf
