// gf_common.cuh -- device helpers shared by the sampler's kernels:
// Philox4x64-10 (Salmon et al., SC'11), uniform/normal conversions, FP64
// block reductions, the device status word and host launch utilities.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gfflow.h"

namespace gf {

// ---------------------------------------------------------------------------
// Device status word: kernels that can detect an error receive its address
// and record the first error (atomicCAS from 0); gf_device_status reads and
// clears it.  (The word itself is defined in gf_api.cu; no relocatable
// device code is needed.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int32_t* word, int32_t code) {
    atomicCAS(reinterpret_cast<int*>(word), 0, code);
}
int32_t* status_word();   // host: device address of the process-wide status word
// host: where kernels launched on `stream` record errors (the stream's slot
// from gf_set_stream_status_slot, else the process-wide word)
int32_t* status_word(cudaStream_t stream);

// ---------------------------------------------------------------------------
// Philox4x64-10: ten rounds of two 64x64->128 multiplies with a Weyl key
// schedule.  Counter sub-spaces (last counter word) per random purpose.
// ---------------------------------------------------------------------------
enum : uint64_t { TAG_PRIOR = 1, TAG_MH = 2, TAG_HMC_P = 3, TAG_HMC_U = 4 };

struct u64x4 { uint64_t x, y, z, w; };

__device__ __forceinline__ u64x4 philox4x64_10(uint64_t k0, uint64_t k1, u64x4 c) {
    constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    constexpr uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        const uint64_t hi0 = __umul64hi(M0, c.x), lo0 = M0 * c.x;
        const uint64_t hi1 = __umul64hi(M1, c.z), lo1 = M1 * c.z;
        c = u64x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    }
    return c;
}

// (2k+1) * 2^-24 with k the top 23 bits: exact in FP32, in (0,1).
__device__ __forceinline__ float u24f(uint64_t w) {
    return (float)(2u * (uint32_t)(w >> 41) + 1u) * 0x1p-24f;
}
// (2k+1) * 2^-53 with k the top 52 bits: exact in FP64, in (0,1).
__device__ __forceinline__ double u53(uint64_t w) {
    return (double)(2ull * (w >> 12) + 1ull) * 0x1p-53;
}

// Four FP32 standard normals (two Box-Muller pairs, cos then sin) from one block.
__device__ __forceinline__ void normals4_f32(u64x4 w, float out[4]) {
    float r0 = sqrtf(-2.0f * logf(u24f(w.x)));
    float r1 = sqrtf(-2.0f * logf(u24f(w.z)));
    float s0, c0, s1, c1;
    sincospif(2.0f * u24f(w.y), &s0, &c0);
    sincospif(2.0f * u24f(w.w), &s1, &c1);
    out[0] = r0 * c0; out[1] = r0 * s0; out[2] = r1 * c1; out[3] = r1 * s1;
}

// Four FP64 standard normals.
__device__ __forceinline__ void normals4_f64(u64x4 w, double out[4]) {
    double r0 = sqrt(-2.0 * log(u53(w.x)));
    double r1 = sqrt(-2.0 * log(u53(w.z)));
    double s0, c0, s1, c1;
    sincospi(2.0 * u53(w.y), &s0, &c0);
    sincospi(2.0 * u53(w.w), &s1, &c1);
    out[0] = r0 * c0; out[1] = r0 * s0; out[2] = r1 * c1; out[3] = r1 * s1;
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide FP64 sum; `scratch` holds >= 32 doubles; result valid in all
// threads.  Contains __syncthreads(): call from uniform control flow.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < nw; ++i) r += scratch[i];   // fixed order: deterministic
    return r;
}

// Unevaluated sum hi + lo of two FP32 numbers ("double-float"): Knuth's
// TwoSum gives the exact rounding error of an addition, Dekker's Fast2Sum
// renormalises the pair and an FMA gives the exact error of a product, so sums
// and products keep about 2^-48 relative accuracy with FP32 instructions only.
// FP64 instructions are slow on this GPU (about one lane per SM clock).
struct FF { float hi, lo; };
__device__ __forceinline__ void ff_add(FF& a, float b) {
    const float s = a.hi + b;
    const float bp = s - a.hi;
    const float e = (a.hi - (s - bp)) + (b - bp);   // s + e == a.hi + b exactly
    const float lo = a.lo + e;
    a.hi = s + lo;
    a.lo = lo - (a.hi - s);
}
__device__ __forceinline__ void ff_add(FF& a, const FF& b) {
    const float s = a.hi + b.hi;
    const float bp = s - a.hi;
    const float e = (a.hi - (s - bp)) + (b.hi - bp);
    const float lo = e + (a.lo + b.lo);
    a.hi = s + lo;
    a.lo = lo - (a.hi - s);
}
// x * y for pairs: the head product exactly (FMA residual), the cross terms in
// FP32 (their rounding is about 2^-48 of the product).
__device__ __forceinline__ FF ff_mul(const FF& x, const FF& y) {
    const float p = x.hi * y.hi;
    const float e = fmaf(x.hi, y.hi, -p) + (x.hi * y.lo + x.lo * y.hi);
    const float s = p + e;
    return FF{s, e - (s - p)};
}
// acc += x * y
__device__ __forceinline__ void ff_fma(FF& acc, const FF& x, const FF& y) {
    const float p = x.hi * y.hi;
    const float e = fmaf(x.hi, y.hi, -p) + (x.hi * y.lo + x.lo * y.hi);
    ff_add(acc, FF{p, e});
}
__device__ __forceinline__ double ff_to_double(const FF& a) { return (double)a.hi + (double)a.lo; }
// Butterfly sum of the lanes' pairs (fixed order).
__device__ __forceinline__ FF warp_sum_ff(FF a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const FF b{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
        ff_add(a, b);
    }
    return a;
}
// Block sum of the threads' pairs in a fixed order, widened to FP64 (valid in
// every thread); scratch holds 32 pairs.
__device__ __forceinline__ double block_sum_ff(FF v, FF* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum_ff(v);
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    FF r = lane < nw ? scratch[lane] : FF{0.f, 0.f};
    r = warp_sum_ff(r);
    __syncthreads();
    return ff_to_double(r);
}
// Host: the pair nearest a double (hi = nearest float, lo = nearest float of the rest).
inline void ff_split(double d, float* hi, float* lo) {
    *hi = (float)d;
    *lo = (float)(d - (double)*hi);
}

constexpr double LOG_2PI = 1.8378770664093454835606594728112;

// Periodic neighbour wrap for |offset| <= L.
__device__ __forceinline__ int wrap_site(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// The 2 nd periodic neighbours of site n = x + L (y + L z) (x fastest).
struct SiteNbrs {
    int xp, xm, yp, ym, zp, zm;
};
__device__ __forceinline__ SiteNbrs site_nbrs(int n, int nd, int L) {
    const int xc = n % L, yc = (n / L) % L;
    SiteNbrs b;
    b.xp = n - xc + wrap_site(xc + 1, L);
    b.xm = n - xc + wrap_site(xc - 1, L);
    b.yp = n + (wrap_site(yc + 1, L) - yc) * L;
    b.ym = n + (wrap_site(yc - 1, L) - yc) * L;
    b.zp = b.zm = n;
    if (nd == 3) {
        const int zc = n / (L * L), LL = L * L;
        b.zp = n + (wrap_site(zc + 1, L) - zc) * LL;
        b.zm = n + (wrap_site(zc - 1, L) - zc) * LL;
    }
    return b;
}
// The same for L = 2^lg with bit operations only.
__device__ __forceinline__ SiteNbrs site_nbrs_pow2(int n, int nd, int lg) {
    const int m = (1 << lg) - 1;
    const int xc = n & m, yc = (n >> lg) & m;
    SiteNbrs b;
    b.xp = n - xc + ((xc + 1) & m);
    b.xm = n - xc + ((xc - 1) & m);
    b.yp = n + ((((yc + 1) & m) - yc) << lg);
    b.ym = n + ((((yc - 1) & m) - yc) << lg);
    b.zp = b.zm = n;
    if (nd == 3) {
        const int zc = n >> (2 * lg);
        b.zp = n + ((((zc + 1) & m) - zc) << (2 * lg));
        b.zm = n + ((((zc - 1) & m) - zc) << (2 * lg));
    }
    return b;
}

// Sum over mu of (2 phi(n) - phi(n+mu) - phi(n-mu)), i.e. minus the lattice
// Laplacian of the paper's action (Sec. 1), in FP64 on a periodic lattice;
// fields of any element type (widened exactly).
template <typename T>
__device__ __forceinline__ double lap_minus_at(const T* p, int n, int nd, const SiteNbrs& b) {
    const double c = (double)p[n];
    double k = 2.0 * c - (double)p[b.xp] - (double)p[b.xm];
    k += 2.0 * c - (double)p[b.yp] - (double)p[b.ym];
    if (nd == 3) k += 2.0 * c - (double)p[b.zp] - (double)p[b.zm];
    return k;
}
template <typename T>
__device__ __forceinline__ double lap_minus(const T* p, int n, int nd, int L) {
    return lap_minus_at(p, n, nd, site_nbrs(n, nd, L));
}

// The force dS/dphi(n) = 2 sum_mu (2 phi - phi(n+mu) - phi(n-mu)) + 2 m2 phi
// + 4 lam phi^3 in FP64: the one definition used by gf_phi4_force, the action
// VJP, the HMC kicks and the training reverse pass's seed.
template <typename T>
__device__ __forceinline__ double phi4_force_at(const T* p, int n, int nd, const SiteNbrs& b, double m2, double lam) {
    const double c = (double)p[n];
    return 2.0 * lap_minus_at(p, n, nd, b) + 2.0 * m2 * c + 4.0 * lam * c * c * c;
}
template <typename T>
__device__ __forceinline__ double phi4_force_site(const T* p, int n, int nd, int L, double m2, double lam) {
    return phi4_force_at(p, n, nd, site_nbrs(n, nd, L), m2, lam);
}

// phi^4 action (paper Sec. 1) of one configuration held in shared memory,
// this thread's share of the sites (n = t0, += stride; by default the
// thread's index in the block and the block size), in the
// forward-hop arrangement (equal to the two-neighbour form summed over the
// periodic lattice): phi^2 (c2d + lam phi^2) - 2 phi sum_mu phi(n + mu),
// c2d = 2 nd + m2, in FP32 pairs (phi^2 exact, products and sums to about
// 2^-48).  Used by the fused coupling-stack kernels' epilogues.
template <int ND>
__device__ FF action_part(const float* x, int L, int V, const FF& c2d, const FF& lam, int t0 = threadIdx.x,
                          int stride = blockDim.x) {
    FF acc{0.f, 0.f};
    for (int n = t0; n < V; n += stride) {
        const int xc = n % L, yc = (n / L) % L, zc = n / (L * L);
        FF hop{x[n - xc + (xc + 1 == L ? 0 : xc + 1)], 0.f};
        ff_add(hop, x[n + ((yc + 1 == L ? 0 : yc + 1) - yc) * L]);
        if (ND == 3) ff_add(hop, x[n + ((zc + 1 == L ? 0 : zc + 1) - zc) * L * L]);
        const float c = x[n], cp = c * c;
        const FF qq{cp, fmaf(c, c, -cp)};
        FF inner = ff_mul(lam, qq);
        ff_add(inner, c2d);
        ff_add(acc, ff_mul(qq, inner));
        ff_add(acc, ff_mul(FF{-2.f * c, 0.f}, hop));
    }
    return acc;
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
int num_sms();   // cached multiprocessor count of the current device

}  // namespace gf

#define GF_CHECK_LAUNCH()                                          \
    do {                                                           \
        if (cudaGetLastError() != cudaSuccess) return GF_ECUDA;    \
    } while (0)
