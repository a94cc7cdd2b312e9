// gf_action.cu -- standalone phi^4 action and force (paper arXiv:2208.08903
// Sec. 1: S = sum_n [-phi(n) Lap phi(n) + m2 phi^2 + lam phi^4], periodic
// lattice Laplacian).
//
// FP32 fields of the common lattices (2D L = 16, 32, 64; 3D L = 8, 16) take
// the streaming kernel: a CTA of 128 threads owns a ring of shared-memory
// buffers that bulk copies (cp.async.bulk) fill with whole configurations, so
// the next configurations arrive while the current one is summed.  S enters the
// Metropolis-Hastings log weights, so it needs FP64 accuracy, and FP64
// instructions are slow on GB300 (about 1/75 of the FP32 rate): the sums run
// in FP32 with error-free transformations (below) and only the final
// per-configuration value is formed in FP64.  Other lattices and FP64 fields
// stage one configuration at a time and form each site term in FP32 pairs
// (FP32 fields) or FP64.
#include <cfloat>
#include <algorithm>

#include "gf_async.cuh"
#include "gf_common.cuh"

namespace gf {
namespace {

constexpr int kActThreads = 256;

__device__ __forceinline__ int wrapi(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

template <typename T>
__device__ __forceinline__ void stage(const T* __restrict__ g, T* s, int V) {
    // 16-byte vector path when the configuration is 16-byte aligned.
    constexpr int per = 16 / sizeof(T);
    if ((reinterpret_cast<uintptr_t>(g) & 15) == 0 && V % per == 0) {
        const int4* g4 = reinterpret_cast<const int4*>(g);
        int4* s4 = reinterpret_cast<int4*>(s);
        for (int i = threadIdx.x; i < V / per; i += blockDim.x) s4[i] = __ldg(g4 + i);
    } else {
        for (int i = threadIdx.x; i < V; i += blockDim.x) s[i] = g[i];
    }
}

// Site term in the forward-hop arrangement (equal to the two-neighbour form of
// the action summed over the lattice): (2d + m2) phi^2 + lam phi^4
// - 2 phi(n) sum_mu phi(n + mu).  It needs d neighbour reads and about half the
// FP64 operations of the two-neighbour form; FP64 issue rate, not HBM, bounds
// this kernel on GB300.
template <typename T>
__device__ __forceinline__ double site_term_fwd(const T* p, int n, int nd, int L, double c2d, double lam) {
    const int xc = n % L, yc = (n / L) % L;
    double hop = (double)p[n - xc + wrapi(xc + 1, L)] + (double)p[n + (wrapi(yc + 1, L) - yc) * L];
    if (nd == 3) {
        const int zc = n / (L * L);
        hop += (double)p[n + (wrapi(zc + 1, L) - zc) * L * L];
    }
    const double c = (double)p[n], q = c * c;
    return fma(q, fma(lam, q, c2d), -2.0 * c * hop);
}

// The same site term for an FP32 field in FP32 pairs, added to acc: phi^2
// exactly (FMA residual), the products and sums to about 2^-48.
// LC > 0: the lattice size as a compile-time constant (the index arithmetic,
// which otherwise dominates, becomes shifts and masks for powers of two).
template <int LC>
__device__ __forceinline__ void site_term_ff(FF& acc, const float* p, int n, int nd, int L_rt, const FF& c2d,
                                             const FF& lam) {
    const int L = LC > 0 ? LC : L_rt;
    const int xc = n % L, yc = (n / L) % L;
    FF hop{p[n - xc + wrapi(xc + 1, L)], 0.f};
    ff_add(hop, p[n + (wrapi(yc + 1, L) - yc) * L]);
    if (nd == 3) {
        const int zc = n / (L * L);
        ff_add(hop, p[n + (wrapi(zc + 1, L) - zc) * L * L]);
    }
    const float c = p[n], cp = c * c;
    const FF qq{cp, fmaf(c, c, -cp)};
    FF inner = ff_mul(lam, qq);
    ff_add(inner, c2d);
    ff_add(acc, ff_mul(qq, inner));
    ff_add(acc, ff_mul(FF{-2.f * c, 0.f}, hop));
}

template <typename T, int LC = 0>
__global__ void __launch_bounds__(kActThreads) action_kernel(int nd, int L, int V, double m2, double lam,
                                                             FF c2d_ff, FF lam_ff, int64_t B,
                                                             const T* __restrict__ phi, double* __restrict__ S_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* p = reinterpret_cast<T*>(smem_raw);
    double* red = reinterpret_cast<double*>(smem_raw + (((size_t)V * sizeof(T) + 15) & ~size_t(15)));
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        stage(phi + b * V, p, V);
        __syncthreads();
        double S;
        if constexpr (sizeof(T) == 4) {
            FF a{0.f, 0.f};
            for (int n = threadIdx.x; n < V; n += blockDim.x) site_term_ff<LC>(a, p, n, nd, L, c2d_ff, lam_ff);
            S = block_sum_ff(a, reinterpret_cast<FF*>(red));
        } else {
            const double c2d = 2.0 * nd + m2;
            double acc = 0.0;
            for (int n = threadIdx.x; n < V; n += blockDim.x) acc += site_term_fwd(p, n, nd, L, c2d, lam);
            S = block_sum(acc, red);
        }
        if (threadIdx.x == 0) S_out[b] = S;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Streaming action of FP32 fields.
//
// With the forward-hop arrangement S = c2d A + lam B - 2 H, where
// A = sum phi^2, B = sum phi^4, H = sum_n phi(n) sum_mu phi(n + mu) and
// c2d = 2 nd + m2, each thread accumulates its share of A, B and H in
// (hi, lo) FP32 pairs.  Every term t = u * v is a product of FP32 numbers and
// is added with Dekker's Fast2Sum: s = hi + t, z = s - hi is exact whenever
// |hi| >= |t|, and fma(u, v, -z) = (t - z) + (u v - t) is the part of the exact
// product that s misses, rounded once; it goes to lo.  That takes five FP32
// operations per term instead of the eight of a general two-sum.  The
// condition |hi| >= |t| is made to hold by starting hi at a power of two
// sigma >= every term (M = max |phi| of the configuration, from a first pass
// over the staged field): A and B only grow from sigma_A >= M^2 and
// sigma_B >= M^4; H, whose terms have either sign, starts at
// sigma_H >= (16 nd + 1) M^2 and is folded into a pair accumulator (and reset)
// after every 2 x 4 sites, so its 8 nd terms never move hi outside
// [sigma_H / 2, 2 sigma_H] and hi - sigma_H is exact.  A - sigma_A and
// B - sigma_B are exact because sigma is a power of two no smaller than any
// term and hi stays below 2^24 sigma.
//
// The B term also needs the cross term 2 q qe of c^4 = (q + qe)^2 (q = fl(c c),
// qe its FMA residual; qe^2 ~ 2^-48 q^2 is dropped), collected in plain FP32.
//
// The biased H accumulator keeps about 2^-47 sigma_H per fold.  When the
// field has a few sites far larger than the rest, sigma_H is large next to the
// typical product and that is not enough: after the block sum, a
// configuration whose estimated H error, 2^-44.5 sigma_H sqrt(V / 8), exceeds
// 1e-13 max(|S|, 1) is summed again from global memory with a general pair
// sum per site (site_term_ff, as the non-streaming kernel does).
//
// Per configuration there is one block barrier: before it every thread
// leaves its share of S (pairs combined with c2d, lam and -2) in shared memory
// and forms M of the next configuration; after it one warp, in turn, adds up
// the 128 shares and writes S while the others start the next configuration.
// ---------------------------------------------------------------------------
constexpr int kAsThreads = 128;               // a block sums one configuration at a time
constexpr int kAsWarps = kAsThreads / 32;
constexpr long long kAsWaitLimit = 1ll << 24;     // bounded wait for a configuration's bulk copy

// Smallest power of two >= x for finite x >= 0 (0 -> 0); inf and NaN unchanged.
__device__ __forceinline__ float pow2_ceil(float x) {
    const uint32_t b = __float_as_uint(x);
    if (b >= 0x7f800000u) return x;
    return __uint_as_float((b + 0x7fffffu) & 0xff800000u);
}

// hi + lo += u * v for |hi| >= |u v| (see above).
__device__ __forceinline__ void f2s_prod(float& hi, float& lo, float u, float v) {
    const float s = hi + u * v, z = s - hi;
    lo += fmaf(u, v, -z);
    hi = s;
}

// max |phi| over this thread's chunks of a staged configuration
template <int NCH, int ITER>
__device__ __forceinline__ float chunk_absmax(const float4* p4) {
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < ITER; ++i) {
        const int kc = i * kAsThreads + threadIdx.x;
        if (NCH % kAsThreads == 0 || kc < NCH) {
            const float4 v = p4[kc];
            m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    return m;
}

template <int ND, int L>
__global__ void __launch_bounds__(kAsThreads) action_stream_kernel(int64_t B, const float* __restrict__ phi,
                                                                   double* __restrict__ S_out, FF c2d_ff,
                                                                   FF lam_ff, int32_t* __restrict__ status) {
    constexpr int V = ND == 3 ? L * L * L : L * L;
    constexpr int NBUF = ring_depth<V * 4>();
    constexpr int CPR = L / 4;                  // 4-site chunks per lattice row (x direction)
    constexpr int NCH = V / 4;                  // chunks per configuration
    constexpr int ITER = (NCH + kAsThreads - 1) / kAsThreads;
    static_assert(L >= 8 && (L & (L - 1)) == 0 && 32 % CPR == 0 && NCH % 32 == 0, "streaming lattice");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + NBUF * V * 4);   // [NBUF]
    FF* part = reinterpret_cast<FF*>(full + NBUF);                          // [2][kAsThreads]
    float* wmax = reinterpret_cast<float*>(part + 2 * kAsThreads);          // [2][kAsWarps]
    int* abort_s = reinterpret_cast<int*>(wmax + 2 * kAsWarps);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const BulkRing<NBUF> ring(smem_raw, full, phi, V * 4, B);
    if (tid == 0) {
        *abort_s = 0;
        ring.start();
    }
    __syncthreads();
    // M of local configuration 0; the loop below forms M of configuration
    // k + 1 before the one barrier of configuration k
    if (ring.count > 0) {
        float m = 0.f;
        if (ring.wait(0, kAsWaitLimit)) {
            m = chunk_absmax<NCH, ITER>(static_cast<const float4*>(ring.data(0)));
        } else {
            set_status(status, GF_ETIMEOUT);
            *abort_s = 1;
        }
        if (lane == 0) wmax[warp] = m;
    }
    __syncthreads();
    int64_t k = 0;
    for (; k < ring.count; ++k) {
        if (*abort_s) break;                    // set before the last barrier: block-uniform
        const int64_t b = blockIdx.x + k * gridDim.x;
        const int slot = (int)(k & 1);
        const float* p = static_cast<const float*>(ring.data(k));
        const float4* p4 = reinterpret_cast<const float4*>(p);
        float M = wmax[slot * kAsWarps];
#pragma unroll
        for (int w = 1; w < kAsWarps; ++w) M = fmaxf(M, wmax[slot * kAsWarps + w]);
        const float M2 = M * M;
        const float sA = pow2_ceil(M2), sB = pow2_ceil(M2 * M2), sH = pow2_ceil((16.f * ND + 1.f) * M2);

        // A, B and H of this thread's chunks (see above); xB collects q qe,
        // the cross term of c^4 = (q + qe)^2 (qe^2 ~ 2^-48 q^2 is dropped)
        float aA = sA, lA = 0.f, aB = sB, lB = 0.f, xB = 0.f, aH = sH, lH = 0.f;
        FF hsum{0.f, 0.f};
        // chunk kc = i * 128 + tid lies in row r = i * RI + r0 (RI = 128 / CPR rows
        // per step); its y and z neighbours are the same chunk of the next row
        // and of the next plane, wrapping at the lattice edge
        constexpr int RI = kAsThreads / CPR;
        const int r0 = tid / CPR;
#pragma unroll
        for (int i = 0; i < ITER; ++i) {
            const int kc = i * kAsThreads + tid;
            if (NCH % kAsThreads == 0 || kc < NCH) {
                const int r = i * RI + r0;
                const float4 c4 = p4[kc];
                // x neighbour of the chunk's last site: first site of the next chunk of the row
                const float xn = __shfl_sync(0xffffffffu, c4.x, (lane & ~(CPR - 1)) | ((lane + 1) & (CPR - 1)));
                int ky, kz = 0;
                if constexpr (ND == 2) {
                    ky = r == L - 1 ? kc - (L - 1) * CPR : kc + CPR;
                } else {
                    static_assert(RI % L == 0, "the y coordinate of a thread's chunks is fixed");
                    ky = (r & (L - 1)) == L - 1 ? kc - (L - 1) * CPR : kc + CPR;
                    kz = r / L == L - 1 ? kc - (L - 1) * L * CPR : kc + L * CPR;
                }
                const float4 y4 = p4[ky];
                const float4 z4 = ND == 3 ? p4[kz] : y4;
                const float cs[4] = {c4.x, c4.y, c4.z, c4.w}, xs[4] = {c4.y, c4.z, c4.w, xn};
                const float ys[4] = {y4.x, y4.y, y4.z, y4.w}, zs[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float c = cs[j], q = c * c;
                    {
                        const float s = aA + q, z = s - aA;
                        lA += fmaf(c, c, -z);
                        aA = s;
                    }
                    {
                        const float qe = fmaf(c, c, -q), s = aB + q * q, z = s - aB;
                        lB += fmaf(q, q, -z);
                        xB = fmaf(q, qe, xB);
                        aB = s;
                    }
                    f2s_prod(aH, lH, c, xs[j]);
                    f2s_prod(aH, lH, c, ys[j]);
                    if constexpr (ND == 3) f2s_prod(aH, lH, c, zs[j]);
                }
            }
            if ((i & 1) || i == ITER - 1) {     // fold H (hi - sigma_H is exact) and restart it
                ff_add(hsum, FF{aH - sH, lH});
                aH = sH;
                lH = 0.f;
            }
        }
        // this thread's share of S = c2d A + lam B - 2 H
        FF t = ff_mul(c2d_ff, FF{aA - sA, lA});
        ff_add(t, ff_mul(lam_ff, FF{aB - sB, fmaf(2.f, xB, lB)}));
        ff_add(t, FF{-2.f * hsum.hi, -2.f * hsum.lo});
        part[slot * kAsThreads + tid] = t;
        // M of the next configuration (its copy was issued NBUF configurations ago)
        if (k + 1 < ring.count) {
            float m = 0.f;
            if (ring.wait(k + 1, kAsWaitLimit)) {
                m = chunk_absmax<NCH, ITER>(static_cast<const float4*>(ring.data(k + 1)));
            } else {
                set_status(status, GF_ETIMEOUT);
                *abort_s = 1;
            }
            if (lane == 0) wmax[(slot ^ 1) * kAsWarps + warp] = m;
        }
        __syncthreads();
        if (tid == 0) ring.refill(k);           // every thread has read this buffer
        // one warp (in turn) sums the 128 shares and writes S
        if (warp == (int)(k & (kAsWarps - 1))) {
            const FF* pk = part + slot * kAsThreads;
            FF tot = pk[lane];
#pragma unroll
            for (int w = 1; w < kAsWarps; ++w) ff_add(tot, pk[lane + 32 * w]);
            tot = warp_sum_ff(tot);
            // statistical size of the biased H error against the tolerance:
            // 2^-44.5 sqrt(V/8) sigma_H <= 1e-13 max(|S|, 1), else (or NaN) the
            // warp sums the configuration again from global memory, a general
            // pair sum per site
            const float h_err = sH * (0.42044820f * sqrtf((float)(V / 8)));
            if (!(h_err <= fmaxf(fabsf(tot.hi), 1.f))) {
                const float* g = phi + b * V;
                FF a{0.f, 0.f};
                for (int n = lane; n < V; n += 32) site_term_ff<L>(a, g, n, ND, L, c2d_ff, lam_ff);
                tot = warp_sum_ff(a);
            }
            if (lane == 0) S_out[b] = ff_to_double(tot);
        }
    }
    if (tid == 0) ring.drain(k, kAsWaitLimit);
}

__global__ void __launch_bounds__(kActThreads) force_kernel(int nd, int L, int V, double m2, double lam,
                                                            int64_t B, const double* __restrict__ phi,
                                                            double* __restrict__ F) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* p = reinterpret_cast<double*>(smem_raw);
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        stage(phi + b * V, p, V);
        __syncthreads();
        for (int n = threadIdx.x; n < V; n += blockDim.x) F[b * V + n] = phi4_force_site(p, n, nd, L, m2, lam);
        __syncthreads();
    }
}

// Vector-Jacobian product of the action for FP32 fields: gphi = gS[b] dS/dphi,
// formed in FP64 from the exactly widened field, rounded once to FP32.
__global__ void __launch_bounds__(kActThreads) action_vjp_kernel(int nd, int L, int V, double m2, double lam,
                                                                 int64_t B, const float* __restrict__ phi,
                                                                 const double* __restrict__ gS,
                                                                 float* __restrict__ gphi) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* p = reinterpret_cast<float*>(smem_raw);
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        stage(phi + b * V, p, V);
        __syncthreads();
        const double g = gS[b];
        for (int n = threadIdx.x; n < V; n += blockDim.x)
            gphi[b * V + n] = (float)(g * phi4_force_site(p, n, nd, L, m2, lam));
        __syncthreads();
    }
}

bool lattice_ok(int nd, int L) {
    if (nd != 2 && nd != 3) return false;
    if (L < 1) return false;
    int64_t V = 1;
    for (int i = 0; i < nd; ++i) V *= L;
    return V <= 16384;
}

template <typename K>
int64_t grid_for(K kern, size_t smem, int64_t B) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kActThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return std::min<int64_t>(B, (int64_t)num_sms() * per_sm);
}

template <int ND, int L>
void launch_stream(int64_t B, const float* phi, double* S, FF c2d, FF lam, cudaStream_t stream, bool* ok) {
    constexpr int V = ND == 3 ? L * L * L : L * L;
    constexpr int NBUF = ring_depth<V * 4>();
    const size_t smem = (size_t)NBUF * V * 4 + NBUF * 8 + 2 * kAsThreads * 8 + 2 * kAsWarps * 4 + 16;
    auto k = action_stream_kernel<ND, L>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kAsThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t grid = std::min<int64_t>(B, (int64_t)num_sms() * per_sm);
    k<<<(unsigned)grid, kAsThreads, smem, stream>>>(B, phi, S, c2d, lam, status_word(stream));
    *ok = true;
}

// The streaming kernel for FP32 fields of 2D L = 16, 32, 64 and 3D L = 8, 16
// whose configurations start on 16-byte boundaries (the bulk copies need
// that); false when the lattice or the alignment does not qualify.
bool launch_action_stream(int nd, int L, int64_t B, const float* phi, double* S, FF c2d, FF lam,
                          cudaStream_t stream) {
    if ((reinterpret_cast<uintptr_t>(phi) & 15) != 0) return false;
    bool ok = false;
    if (nd == 2 && L == 16) launch_stream<2, 16>(B, phi, S, c2d, lam, stream, &ok);
    else if (nd == 2 && L == 32) launch_stream<2, 32>(B, phi, S, c2d, lam, stream, &ok);
    else if (nd == 2 && L == 64) launch_stream<2, 64>(B, phi, S, c2d, lam, stream, &ok);
    else if (nd == 3 && L == 8) launch_stream<3, 8>(B, phi, S, c2d, lam, stream, &ok);
    else if (nd == 3 && L == 16) launch_stream<3, 16>(B, phi, S, c2d, lam, stream, &ok);
    return ok;
}

}  // namespace
}  // namespace gf

using namespace gf;

extern "C" {

gf_status gf_phi4_action(int32_t nd, int32_t L, const gf_phi4* phi4, int64_t B,
                         const void* d_phi, int32_t phi_is_fp64, double* d_S_out,
                         cudaStream_t stream) {
    if (!phi4 || !lattice_ok(nd, L) || B < 0 || (B > 0 && (!d_phi || !d_S_out))) return GF_EINVAL;
    if (phi_is_fp64 != 0 && phi_is_fp64 != 1) return GF_EINVAL;
    if (B == 0) return GF_OK;
    int V = 1;
    for (int i = 0; i < nd; ++i) V *= L;
    const size_t esz = phi_is_fp64 ? 8 : 4;
    FF c2d_ff, lam_ff;
    ff_split(2.0 * nd + phi4->m2, &c2d_ff.hi, &c2d_ff.lo);
    ff_split(phi4->lam, &lam_ff.hi, &lam_ff.lo);
    const size_t smem = (((size_t)V * esz + 15) & ~size_t(15)) + 32 * sizeof(double);
    if (phi_is_fp64) {
        auto k = action_kernel<double>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return GF_ECUDA;
        k<<<(unsigned)grid_for(k, smem, B), kActThreads, smem, stream>>>(
            nd, L, V, phi4->m2, phi4->lam, c2d_ff, lam_ff, B, static_cast<const double*>(d_phi), d_S_out);
    } else if (launch_action_stream(nd, L, B, static_cast<const float*>(d_phi), d_S_out, c2d_ff, lam_ff,
                                    stream)) {
        // streaming kernel launched
    } else {
        auto k = (nd == 3 && L == 16) ? action_kernel<float, 16> : action_kernel<float>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return GF_ECUDA;
        k<<<(unsigned)grid_for(k, smem, B), kActThreads, smem, stream>>>(
            nd, L, V, phi4->m2, phi4->lam, c2d_ff, lam_ff, B, static_cast<const float*>(d_phi), d_S_out);
    }
    GF_CHECK_LAUNCH();
    return GF_OK;
}

gf_status gf_phi4_force(int32_t nd, int32_t L, const gf_phi4* phi4, int64_t B,
                        const double* d_phi, double* d_F_out, cudaStream_t stream) {
    if (!phi4 || !lattice_ok(nd, L) || B < 0 || (B > 0 && (!d_phi || !d_F_out))) return GF_EINVAL;
    if (B == 0) return GF_OK;
    int V = 1;
    for (int i = 0; i < nd; ++i) V *= L;
    const size_t smem = (size_t)V * 8;
    if (cudaFuncSetAttribute(force_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GF_ECUDA;
    force_kernel<<<(unsigned)grid_for(force_kernel, smem, B), kActThreads, smem, stream>>>(
        nd, L, V, phi4->m2, phi4->lam, B, d_phi, d_F_out);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

gf_status gf_phi4_action_vjp(int32_t nd, int32_t L, const gf_phi4* phi4, int64_t B, const float* d_phi,
                             const double* d_gS, float* d_gphi_out, cudaStream_t stream) {
    if (!phi4 || !lattice_ok(nd, L) || B < 0 || (B > 0 && (!d_phi || !d_gS || !d_gphi_out))) return GF_EINVAL;
    if (B == 0) return GF_OK;
    int V = 1;
    for (int i = 0; i < nd; ++i) V *= L;
    const size_t smem = (size_t)V * 4;
    if (cudaFuncSetAttribute(action_vjp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return GF_ECUDA;
    action_vjp_kernel<<<(unsigned)grid_for(action_vjp_kernel, smem, B), kActThreads, smem, stream>>>(
        nd, L, V, phi4->m2, phi4->lam, B, d_phi, d_gS, d_gphi_out);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

}  // extern "C"
