// gf_observables.cu -- observables of the flow / MH chain on the device
// (paper arXiv:2208.08903 Sec. 1: expectation values as chain averages, the
// autocorrelation time tau_ac with N_indep = N_conf / (2 tau_ac); Sec. 3: the
// condensate, the zero-momentum two-point function and the effective sample
// size of the analysis tools).
//
//  - per configuration: M = mean of phi and C(t) = (1/V) sum_tau Phi(tau)
//    Phi(tau + t), Phi(tau) = sum of phi over the slice at outermost
//    coordinate tau (V/L contiguous sites).  Threads accumulate in FP32 pairs
//    (error-free transformations), so the kernel reads each field once with
//    little FP64 work.  FP32 fields of 2D L = 16, 32, 64 and 3D L = 8, 16 are
//    streamed through shared memory by bulk copies; other shapes read global
//    memory directly (a warp per configuration or a block per configuration).
//  - chain gather: the chain's series O[chain_idx[k]] of a per-proposal
//    observable.
//  - Gamma(t) of a series (one CTA per lag, fixed-order FP64 reduction), then
//    the Madras-Sokal automatic window for tau_int in one thread.
//  - ESS fraction (sum w)^2 / (n sum w^2) of w = exp(log w), the largest
//    log w factored out.
#include <algorithm>
#include <cmath>

#include "gf_async.cuh"
#include "gf_common.cuh"

namespace gf {
namespace {

constexpr int kObsThreads = 256;
constexpr int kRedThreads = 1024;

// One CTA per configuration (grid-stride).  Dynamic shared memory: L pairs.
// Each warp sums whole slices: every lane first issues up to four 16-byte loads,
// then adds them into its FP32 pair; the warp reduces the pairs the same way.
// M and C(t) are formed from the slice pairs in pair arithmetic too and widened
// to FP64 once per output, so FP64 instructions are a few per configuration.
__global__ void __launch_bounds__(kObsThreads) obs_kernel(int L, int64_t V, int64_t B, double inv_v,
                                                         const float* __restrict__ phi, double* __restrict__ M,
                                                         double* __restrict__ C) {
    extern __shared__ FF Phi[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t S = V / L;
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        const float* p = phi + b * V;
        const bool vec = (S % 4 == 0) && ((reinterpret_cast<uintptr_t>(p) & 15) == 0);
        for (int tau = wid; tau < L; tau += nw) {
            const float* q = p + (int64_t)tau * S;
            FF acc{0.f, 0.f};
            if (vec) {
                const float4* q4 = reinterpret_cast<const float4*>(q);
                const int64_t S4 = S / 4;
                for (int64_t i0 = lane; i0 < S4; i0 += 4 * 32) {
                    float4 v[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (i0 + 32 * k < S4) v[k] = __ldg(q4 + i0 + 32 * k);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (i0 + 32 * k < S4) {
                            ff_add(acc, v[k].x);
                            ff_add(acc, v[k].y);
                            ff_add(acc, v[k].z);
                            ff_add(acc, v[k].w);
                        }
                }
            } else {
                for (int64_t i = lane; i < S; i += 32) ff_add(acc, __ldg(q + i));
            }
            acc = warp_sum_ff(acc);
            if (lane == 0) Phi[tau] = acc;
        }
        __syncthreads();
        if (M && threadIdx.x == 0) {
            FF m{0.f, 0.f};
            for (int tau = 0; tau < L; ++tau) ff_add(m, Phi[tau]);
            M[b] = ff_to_double(m) * inv_v;
        }
        if (C) {
            for (int t = threadIdx.x; t < L; t += blockDim.x) {
                FF acc{0.f, 0.f};
                for (int tau = 0, u = t; tau < L; ++tau, u = (u + 1 == L) ? 0 : u + 1) ff_fma(acc, Phi[tau], Phi[u]);
                C[b * L + t] = ff_to_double(acc) * inv_v;
            }
        }
        __syncthreads();
    }
}

// One warp per configuration (grid-stride over configurations), for slices of
// a multiple of 128 sites and L <= kObsWarpMaxL: lane l reads 16-byte pieces
// l, l + 32, ... of the field in batches of eight loads, so every lane sees the
// same slice at the same step.  Each lane sums its part of a slice with a
// compensated sum (Knuth's TwoSum into hi, the exact rounding errors added
// into lo: seven FP32 operations per site) and, at the slice's end, leaves the
// pair in the warp's table (dynamic shared memory, [L][32] pairs, lane index
// xor-swizzled by the slice so stores and the column reads below are free of
// bank conflicts).  Lane tau then adds up the 32 pairs of slice tau in pair
// arithmetic; M and C(t) follow from the L slice sums, as pairs, widened to
// FP64 once per output.  No CTA barrier is needed.  1/V comes from the host.
constexpr int kObsWarpMaxL = 64;
__global__ void __launch_bounds__(kObsThreads) obs_warp_kernel(int L, int64_t V, int64_t B, double inv_v,
                                                              const float* __restrict__ phi,
                                                              double* __restrict__ M, double* __restrict__ C) {
    extern __shared__ FF tab_all[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    FF* tab = tab_all + (size_t)wid * L * 32;
    const int64_t S4 = V / L / 4;                 // 16-byte pieces per slice, a multiple of 32
    const int per = (int)(S4 / 32);               // batches of 32 pieces per slice
    const int nk = L * per;                       // pieces per lane
    for (int64_t b = (int64_t)blockIdx.x * wpb + wid; b < B; b += (int64_t)gridDim.x * wpb) {
        const float4* q4 = reinterpret_cast<const float4*>(phi + b * V) + lane;
        float hi = 0.f, lo = 0.f;
        for (int k0 = 0; k0 < nk; k0 += 8) {
            float4 v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (k0 + j < nk) v[j] = __ldg(q4 + (int64_t)32 * (k0 + j));
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (k0 + j < nk) {
                    const float c[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float s = hi + c[q];
                        const float bp = s - hi;
                        lo += (hi - (s - bp)) + (c[q] - bp);
                        hi = s;
                    }
                    if ((k0 + j + 1) % per == 0) {             // end of slice (k0 + j) / per
                        const int tau = (k0 + j) / per;
                        tab[tau * 32 + ((lane ^ tau) & 31)] = FF{hi, lo};
                        hi = 0.f;
                        lo = 0.f;
                    }
                }
            }
        }
        __syncwarp();
        for (int tau = lane; tau < L; tau += 32) {
            FF acc{0.f, 0.f};
            for (int i = 0; i < 32; ++i) ff_add(acc, tab[tau * 32 + ((i ^ tau) & 31)]);
            tab[tau * 32 + ((0 ^ tau) & 31)] = acc;     // the slice sum, in lane 0's entry
        }
        __syncwarp();
        const auto slice = [&](int tau) -> FF { return tab[tau * 32 + (tau & 31)]; };
        if (M && lane == 0) {
            FF m{0.f, 0.f};
            for (int tau = 0; tau < L; ++tau) ff_add(m, slice(tau));
            M[b] = ff_to_double(m) * inv_v;
        }
        if (C) {
            for (int t = lane; t < L; t += 32) {
                FF a{0.f, 0.f};
                for (int tau = 0, u = t; tau < L; ++tau, u = (u + 1 == L) ? 0 : u + 1) ff_fma(a, slice(tau), slice(u));
                C[b * L + t] = ff_to_double(a) * inv_v;
            }
        }
        __syncwarp();
    }
}

// Streaming form: a block of 128 threads owns a ring of shared-memory buffers
// that bulk copies fill with whole configurations (BulkRing), so the next
// configurations arrive while the current one is summed.  The TPS = 128 / L
// consecutive threads of slice tau each sum every TPS-th 4-site chunk of it
// with a compensated sum (TwoSum into hi, the exact rounding errors into lo:
// seven FP32 operations per site), combine their pairs by shuffles and leave
// Phi(tau) in shared memory; after one block barrier threads t < L form C(t)
// and thread L forms M, in pair arithmetic widened to FP64 once per output.
// Phi is double-buffered, so one barrier per configuration suffices.
constexpr int kOsThreads = 128;
constexpr long long kOsWaitLimit = 1ll << 24;     // bounded wait for a configuration's bulk copy

template <int ND, int L>
__global__ void __launch_bounds__(kOsThreads) obs_stream_kernel(int64_t B, double inv_v,
                                                                const float* __restrict__ phi,
                                                                double* __restrict__ M_out,
                                                                double* __restrict__ C_out,
                                                                int32_t* __restrict__ status) {
    constexpr int V = ND == 3 ? L * L * L : L * L;
    constexpr int NBUF = ring_depth<V * 4>();
    constexpr int CPS = V / L / 4;                          // chunks per slice
    constexpr int TPS = kOsThreads / L;                     // threads per slice
    constexpr int PER = CPS >= TPS ? CPS / TPS : 1;         // chunks per thread
    static_assert((L & (L - 1)) == 0 && L >= 8 && L <= 64 && TPS <= 32, "streaming lattice");
    static_assert(CPS % TPS == 0 || TPS % CPS == 0, "slice split");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + NBUF * V * 4);  // [NBUF]
    FF* Phi = reinterpret_cast<FF*>(full + NBUF);                          // [2][L]
    int* abort_s = reinterpret_cast<int*>(Phi + 2 * L);
    const int tid = threadIdx.x, tau = tid / TPS, sub = tid % TPS;
    const BulkRing<NBUF> ring(smem_raw, full, phi, V * 4, B);
    if (tid == 0) {
        *abort_s = 0;
        ring.start();
    }
    __syncthreads();
    int64_t k = 0;
    for (; k < ring.count; ++k) {
        const int64_t b = blockIdx.x + k * gridDim.x;
        const float4* p4 = static_cast<const float4*>(ring.data(k));
        float hi = 0.f, lo = 0.f;
        if (!ring.wait(k, kOsWaitLimit)) {
            set_status(status, GF_ETIMEOUT);
            *abort_s = 1;
        } else if (CPS >= TPS || sub < CPS) {
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const float4 v = p4[tau * CPS + sub + TPS * j];
                const float c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float s = hi + c[q], bp = s - hi;
                    lo += (hi - (s - bp)) + (c[q] - bp);
                    hi = s;
                }
            }
        }
        FF a{hi, lo};
#pragma unroll
        for (int o = TPS / 2; o > 0; o >>= 1)
            ff_add(a, FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)});
        FF* ph = Phi + (k & 1) * L;
        if (sub == 0) ph[tau] = a;
        __syncthreads();
        if (*abort_s) break;                    // block-uniform
        if (tid == 0) ring.refill(k);           // every thread has read this buffer
        if (tid < L) {
            if (C_out) {
                FF c{0.f, 0.f};
#pragma unroll 4
                for (int u = 0; u < L; ++u) ff_fma(c, ph[u], ph[(u + tid) & (L - 1)]);
                C_out[b * L + tid] = ff_to_double(c) * inv_v;
            }
        } else if (tid == L && M_out) {
            FF m{0.f, 0.f};
#pragma unroll 4
            for (int u = 0; u < L; ++u) ff_add(m, ph[u]);
            M_out[b] = ff_to_double(m) * inv_v;
        }
    }
    if (tid == 0) ring.drain(k, kOsWaitLimit);
}

template <int ND, int L>
void launch_obs_stream(int64_t B, double inv_v, const float* phi, double* M, double* C, cudaStream_t stream,
                       bool* ok) {
    constexpr int V = ND == 3 ? L * L * L : L * L;
    constexpr int NBUF = ring_depth<V * 4>();
    const size_t smem = (size_t)NBUF * V * 4 + NBUF * 8 + 2 * L * sizeof(FF) + 16;
    auto kern = obs_stream_kernel<ND, L>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kOsThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t grid = std::min<int64_t>(B, (int64_t)num_sms() * per_sm);
    kern<<<(unsigned)grid, kOsThreads, smem, stream>>>(B, inv_v, phi, M, C, status_word(stream));
    *ok = true;
}

// The streaming kernel for FP32 fields of 2D L = 16, 32, 64 and 3D L = 8, 16
// that start on a 16-byte boundary; false when the shape or the alignment does
// not qualify.
bool launch_obs_stream_if(int nd, int L, int64_t B, double inv_v, const float* phi, double* M, double* C,
                          cudaStream_t stream) {
    if ((reinterpret_cast<uintptr_t>(phi) & 15) != 0) return false;
    bool ok = false;
    if (nd == 2 && L == 16) launch_obs_stream<2, 16>(B, inv_v, phi, M, C, stream, &ok);
    else if (nd == 2 && L == 32) launch_obs_stream<2, 32>(B, inv_v, phi, M, C, stream, &ok);
    else if (nd == 2 && L == 64) launch_obs_stream<2, 64>(B, inv_v, phi, M, C, stream, &ok);
    else if (nd == 3 && L == 8) launch_obs_stream<3, 8>(B, inv_v, phi, M, C, stream, &ok);
    else if (nd == 3 && L == 16) launch_obs_stream<3, 16>(B, inv_v, phi, M, C, stream, &ok);
    return ok;
}

// out[k][j] = values[(chain_idx[k] - idx0) * width + j]; an index outside
// [0, n_values) writes NaN and records GF_EINVAL in the status word.
__global__ void gather_kernel(int64_t n, const int64_t* __restrict__ chain_idx, int64_t idx0, int64_t n_values,
                              const double* __restrict__ values, int width, double* __restrict__ out,
                              int32_t* status) {
    const int64_t total = n * width;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / width;
        const int j = (int)(i - k * width);
        const int64_t r = chain_idx[k] - idx0;
        if (r < 0 || r >= n_values) {
            out[i] = __longlong_as_double(0x7ff8000000000000ll);
            set_status(status, GF_EINVAL);
        } else {
            out[i] = values[r * width + j];
        }
    }
}

// dbar = mean of (y_k - y_0), one block, fixed order.  Stored in out[3].
__global__ void __launch_bounds__(kRedThreads) mean_dev_kernel(int64_t n, const double* __restrict__ y,
                                                              double* __restrict__ out) {
    __shared__ double red[32];
    const double y0 = y[0];
    double acc = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) acc += y[k] - y0;
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[3] = acc / (double)n;
}

// Gamma(t) for t = blockIdx.x (grid-stride over lags).
__global__ void __launch_bounds__(kObsThreads) gamma_kernel(int64_t n, const double* __restrict__ y, int t_max,
                                                           const double* __restrict__ stats,
                                                           double* __restrict__ gamma) {
    __shared__ double red[32];
    const double y0 = y[0], dbar = stats[3];
    for (int t = blockIdx.x; t <= t_max; t += gridDim.x) {
        double acc = 0.0;
        for (int64_t k = threadIdx.x; k + t < n; k += blockDim.x)
            acc += ((y[k] - y0) - dbar) * ((y[k + t] - y0) - dbar);
        acc = block_sum(acc, red);
        if (threadIdx.x == 0) gamma[t] = acc / (double)(n - t);
        __syncthreads();
    }
}

// Madras-Sokal window and the summary {tau, W, error, mean}; one thread.
__global__ void window_kernel(int64_t n, const double* __restrict__ y, const double* __restrict__ gamma, int t_max,
                              double c, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double mean = y[0] + out[3];
    if (!(gamma[0] > 0.0)) {
        out[0] = 0.5; out[1] = 0.0; out[2] = 0.0; out[3] = mean;
        return;
    }
    double tau = 0.5;
    int W = t_max;
    for (int w = 1; w <= t_max; ++w) {
        tau += gamma[w] / gamma[0];
        if ((double)w >= c * tau) { W = w; break; }
    }
    out[0] = tau;
    out[1] = (double)W;
    out[2] = tau * sqrt((4.0 * W + 2.0) / (double)n);
    out[3] = mean;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ESS fraction in one block: max, then sum w and sum w^2 in a fixed order.
__global__ void __launch_bounds__(kRedThreads) ess_kernel(int64_t n, const double* __restrict__ logw,
                                                         double* __restrict__ out) {
    __shared__ double red[32];
    __shared__ double mx_s;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double mx = -INFINITY;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) mx = fmax(mx, logw[k]);
    mx = warp_max(mx);
    if (lane == 0) red[wid] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = -INFINITY;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, red[i]);
        mx_s = m;
    }
    __syncthreads();
    mx = mx_s;
    if (!(mx > -INFINITY)) {                       // n == 0 or all weights zero
        if (threadIdx.x == 0) *out = 0.0;
        return;
    }
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        const double w = exp(logw[k] - mx);
        s1 += w;
        s2 += w * w;
    }
    s1 = block_sum(s1, red);
    s2 = block_sum(s2, red);
    if (threadIdx.x == 0) *out = s1 * s1 / ((double)n * s2);
}

int64_t ipow(int64_t a, int e) {
    int64_t r = 1;
    while (e-- > 0) r *= a;
    return r;
}

}  // namespace
}  // namespace gf

using namespace gf;

extern "C" {

gf_status gf_observables(int32_t nd, int32_t L, int64_t B, const float* d_phi, double* d_M_out, double* d_C_out,
                         cudaStream_t stream) {
    if ((nd != 2 && nd != 3) || L < 1 || L > GF_OBS_MAX_L || B < 0) return GF_EINVAL;
    if (B > 0 && (!d_phi || (!d_M_out && !d_C_out))) return GF_EINVAL;
    if (B == 0) return GF_OK;
    const int64_t V = ipow(L, nd);
    const int64_t S = V / L;
    if (launch_obs_stream_if(nd, L, B, 1.0 / (double)V, d_phi, d_M_out, d_C_out, stream)) {
        // streaming kernel launched
    } else if (S % 128 == 0 && L <= kObsWarpMaxL && (reinterpret_cast<uintptr_t>(d_phi) & 15) == 0) {
        // warps per block: each warp's table is L x 32 pairs; at most 48 KB per block
        const int wpb = (int)std::max<int64_t>(1, std::min<int64_t>(kObsThreads / 32, 49152 / (256 * (int64_t)L)));
        const size_t smem = (size_t)wpb * L * 32 * sizeof(FF);
        const unsigned grid = (unsigned)std::min<int64_t>((B + wpb - 1) / wpb, (int64_t)num_sms() * 16);
        obs_warp_kernel<<<grid, 32 * wpb, smem, stream>>>(L, V, B, 1.0 / (double)V, d_phi, d_M_out, d_C_out);
    } else {
        const size_t smem = sizeof(FF) * (size_t)L;
        const unsigned grid = (unsigned)std::min<int64_t>(B, (int64_t)num_sms() * 8);
        obs_kernel<<<grid, kObsThreads, smem, stream>>>(L, V, B, 1.0 / (double)V, d_phi, d_M_out, d_C_out);
    }
    GF_CHECK_LAUNCH();
    return GF_OK;
}

gf_status gf_chain_gather(int64_t n, const int64_t* d_chain_idx, int64_t idx0, int64_t n_values,
                          const double* d_values, int32_t width, double* d_out, cudaStream_t stream) {
    if (n < 0 || width < 1 || n_values < 0) return GF_EINVAL;
    if (n > 0 && (!d_chain_idx || !d_values || !d_out)) return GF_EINVAL;
    if (n == 0) return GF_OK;
    const int64_t total = n * width;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, num_sms() * 16LL));
    gather_kernel<<<grid, 256, 0, stream>>>(n, d_chain_idx, idx0, n_values, d_values, width, d_out, status_word(stream));
    GF_CHECK_LAUNCH();
    return GF_OK;
}

gf_status gf_autocorr(int64_t n, const double* d_y, int32_t t_max, double c_window, double* d_gamma_out,
                      double* d_tau_out, cudaStream_t stream) {
    if (n < 1 || t_max < 0 || t_max >= n || !(c_window > 0.0)) return GF_EINVAL;
    if (!d_y || !d_gamma_out || !d_tau_out) return GF_EINVAL;
    mean_dev_kernel<<<1, kRedThreads, 0, stream>>>(n, d_y, d_tau_out);
    GF_CHECK_LAUNCH();
    const unsigned grid = (unsigned)std::min<int64_t>((int64_t)t_max + 1, (int64_t)num_sms() * 8);
    gamma_kernel<<<grid, kObsThreads, 0, stream>>>(n, d_y, t_max, d_tau_out, d_gamma_out);
    GF_CHECK_LAUNCH();
    window_kernel<<<1, 32, 0, stream>>>(n, d_y, d_gamma_out, t_max, c_window, d_tau_out);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

gf_status gf_ess(int64_t n, const double* d_logw, double* d_ess_out, cudaStream_t stream) {
    if (n < 0 || !d_ess_out || (n > 0 && !d_logw)) return GF_EINVAL;
    ess_kernel<<<1, kRedThreads, 0, stream>>>(n, d_logw, d_ess_out);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

}  // extern "C"
