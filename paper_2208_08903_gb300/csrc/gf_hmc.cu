// gf_hmc.cu -- FP64 HMC trajectories for lattice phi^4 (the comparison
// sampler of paper arXiv:2208.08903 Sec. 2.2, for the same action).
//
// One CTA per chain.  The field lives in shared memory for the whole
// trajectory (the force needs neighbours); each thread keeps the momenta of
// its own sites (n = tid + k*blockDim) in registers.  HBM is touched once at
// the start (phi) and once at the end (phi on accept, dH, accept flag).
#include <algorithm>

#include "gf_common.cuh"

namespace gf {
namespace {

constexpr int kHmcThreads = 256;
constexpr int kMaxSitesPerThread = 16;    // V <= 4096

// POW2: L = 2^lg, neighbour indices by bit operations instead of runtime
// divisions.
template <bool POW2>
__global__ void __launch_bounds__(kHmcThreads) hmc_kernel(int nd, int L, int lg, int V, double m2, double lam,
                                                          int64_t n_chains, double* __restrict__ phi_g,
                                                          int n_steps, double eps, uint64_t seed,
                                                          uint64_t traj, double* __restrict__ dH_out,
                                                          uint8_t* __restrict__ acc_out) {
    const auto nbrs = [&](int n) { return POW2 ? site_nbrs_pow2(n, nd, lg) : site_nbrs(n, nd, L); };
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* p = reinterpret_cast<double*>(smem_raw);
    double* red = p + V;
    const int nper = (V + blockDim.x - 1) / blockDim.x;
    for (int64_t c = blockIdx.x; c < n_chains; c += gridDim.x) {
        double* g = phi_g + c * V;
        for (int n = threadIdx.x; n < V; n += blockDim.x) p[n] = g[n];
        // momenta: sites 4j..4j+3 from one Philox block (FP64 Box-Muller)
        double pi[kMaxSitesPerThread];
#pragma unroll
        for (int k = 0; k < kMaxSitesPerThread; ++k) {
            pi[k] = 0.0;
            const int n = threadIdx.x + k * blockDim.x;
            if (k < nper && n < V) {
                const u64x4 w = philox4x64_10(seed, 0ull, u64x4{(uint64_t)c, traj, (uint64_t)(n >> 2), TAG_HMC_P});
                double nn[4];
                normals4_f64(w, nn);
                pi[k] = nn[n & 3];
            }
        }
        __syncthreads();
        auto energy = [&](void) -> double {
            double h = 0.0;
#pragma unroll
            for (int k = 0; k < kMaxSitesPerThread; ++k) {
                const int n = threadIdx.x + k * blockDim.x;
                if (k < nper && n < V) {
                    const double f = p[n], f2 = f * f;
                    h += 0.5 * pi[k] * pi[k] + f * lap_minus_at(p, n, nd, nbrs(n)) + m2 * f2 + lam * f2 * f2;
                }
            }
            return block_sum(h, red);
        };
        auto kick = [&](double h) {
#pragma unroll
            for (int k = 0; k < kMaxSitesPerThread; ++k) {
                const int n = threadIdx.x + k * blockDim.x;
                if (k < nper && n < V) pi[k] -= h * phi4_force_at(p, n, nd, nbrs(n), m2, lam);
            }
        };
        const double H0 = energy();
        kick(0.5 * eps);
        for (int i = 1; i <= n_steps; ++i) {
            __syncthreads();     // all kicks read p before it moves
#pragma unroll
            for (int k = 0; k < kMaxSitesPerThread; ++k) {
                const int n = threadIdx.x + k * blockDim.x;
                if (k < nper && n < V) p[n] += eps * pi[k];
            }
            __syncthreads();
            kick(i < n_steps ? eps : 0.5 * eps);
        }
        __syncthreads();
        const double dH = energy() - H0;
        const u64x4 w = philox4x64_10(seed, 0ull, u64x4{(uint64_t)c, traj, 0ull, TAG_HMC_U});
        const bool acc = (-dH) > log(u53(w.x));
        if (acc)
            for (int n = threadIdx.x; n < V; n += blockDim.x) g[n] = p[n];
        if (threadIdx.x == 0) {
            if (dH_out) dH_out[c] = dH;
            if (acc_out) acc_out[c] = acc ? 1 : 0;
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace gf

using namespace gf;

extern "C" gf_status gf_hmc_trajectory(int32_t nd, int32_t L, const gf_phi4* phi4, int64_t n_chains,
                                       double* d_phi, int32_t n_steps, double eps, uint64_t seed,
                                       uint64_t traj_index, double* d_dH_out, uint8_t* d_acc_out,
                                       cudaStream_t stream) {
    if (!phi4 || (nd != 2 && nd != 3) || L < 1 || n_chains < 0 || n_steps < 1 || !(eps == eps))
        return GF_EINVAL;
    int64_t V = 1;
    for (int i = 0; i < nd; ++i) V *= L;
    if (V > (int64_t)kHmcThreads * kMaxSitesPerThread) return GF_EUNSUPPORTED;
    if (n_chains == 0) return GF_OK;
    if (!d_phi) return GF_EINVAL;
    const size_t smem = (size_t)V * 8 + 32 * 8;
    int lg = 0;
    while ((1 << lg) < L) ++lg;
    const bool pow2 = (1 << lg) == L;
    auto kern = pow2 ? hmc_kernel<true> : hmc_kernel<false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GF_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kHmcThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t grid = std::min<int64_t>(n_chains, (int64_t)num_sms() * per_sm);
    kern<<<(unsigned)grid, kHmcThreads, smem, stream>>>(nd, L, lg, (int)V, phi4->m2, phi4->lam, n_chains, d_phi,
                                                        n_steps, eps, seed, traj_index, d_dH_out, d_acc_out);
    GF_CHECK_LAUNCH();
    return GF_OK;
}
