// gf_action.cu -- standalone phi^4 action and force (paper arXiv:2208.08903
// Sec. 1: S = sum_n [-phi(n) Lap phi(n) + m2 phi^2 + lam phi^4], periodic
// lattice Laplacian).
//
// Each CTA stages one configuration at a time in shared memory with 16-byte
// loads (grid-stride over configurations), evaluates the site terms from shared
// memory and reduces them in a fixed order.  S enters the Metropolis-Hastings
// log weights, so it needs FP64 accuracy; for FP32 fields the site terms and the
// per-thread sums are formed in FP32 pairs (about 2^-48 relative), because FP64
// instructions are slow on GB300 (the FP64 form was FP64-bound at 2 % of HBM);
// FP64 fields keep FP64 arithmetic.
#include <algorithm>

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
