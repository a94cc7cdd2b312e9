// gf_mh.cu -- Metropolis-Hastings independence chain over flow proposals
// (paper arXiv:2208.08903 Sec. 1: proposals from the flow corrected by the
// MH test with the Jacobian; acceptance min(1, w'/w), w = p/q).
//
// Two kernels on the caller's stream:
//  1. mh_logu_kernel: log u_g for every step in parallel (Philox word 0 of
//     ctr = (g, 0, 0, TAG_MH), key = (seed, stream_id)) into the workspace;
//  2. mh_scan_kernel: one warp walks the proposals in chunks of 32.  Within
//     a chunk every lane tests its proposal against the current state; the
//     first lane that accepts is the chain's next accept (all earlier lanes
//     rejected against the same state), the state moves there and the lanes
//     after it are re-tested.  A chunk costs 1 + (accepts in it) rounds of
//     ballot instead of 32 dependent steps.  The state stays in device memory.
#include <algorithm>
#include <mutex>

#include "gf_common.cuh"

namespace gf {

__global__ void mh_logu_kernel(const gf_mh_state* __restrict__ st, int64_t n, double* __restrict__ logu) {
    const int64_t step0 = st->step;
    const uint64_t seed = st->seed, stream_id = st->stream_id;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const u64x4 w = philox4x64_10(seed, stream_id, u64x4{(uint64_t)(step0 + k), 0ull, 0ull, TAG_MH});
        logu[k] = log(u53(w.x));
    }
}

__global__ void __launch_bounds__(32) mh_scan_kernel(gf_mh_state* __restrict__ st, int64_t n,
                                                     const double* __restrict__ logw,
                                                     const double* __restrict__ logu,
                                                     int64_t* __restrict__ chain_idx,
                                                     uint8_t* __restrict__ acc_out) {
    constexpr int kChunks = 8;                 // 256 proposals loaded per round trip to memory
    const int lane = threadIdx.x;
    double cur = st->logw_cur;
    int64_t idx = st->idx_cur, nacc = st->n_acc;
    const int64_t g0 = st->step;
    for (int64_t blk = 0; blk < n; blk += 32 * kChunks) {
        double lwv[kChunks], luv[kChunks];
#pragma unroll
        for (int c = 0; c < kChunks; ++c) {
            const int64_t k = blk + 32 * c + lane;
            lwv[c] = k < n ? __ldg(logw + k) : 0.0;
            luv[c] = k < n ? __ldg(logu + k) : 0.0;
        }
#pragma unroll
        for (int c = 0; c < kChunks; ++c) {
            const int64_t base = blk + 32 * c;
            if (base >= n) break;
            const int64_t k = base + lane;
            const bool valid = k < n;
            const double lw = lwv[c], lu = luv[c];
            const int64_t g = g0 + k;
            const int64_t idx_before = idx;
            unsigned remaining = __ballot_sync(0xffffffffu, valid);
            unsigned accm = 0u;
            while (remaining) {
                const bool mine = (remaining >> lane) & 1u;
                const bool test = mine && (g == 0 || (lw - cur) > lu);
                const unsigned m = __ballot_sync(0xffffffffu, test);
                if (m == 0u) break;
                const int j = __ffs(m) - 1;
                accm |= 1u << j;
                cur = __shfl_sync(0xffffffffu, lw, j);
                idx = g0 + base + j;
                remaining &= (j == 31) ? 0u : ~((2u << j) - 1u);
            }
            // state after this lane's step: the last accept at or before it
            const unsigned le = (lane == 31) ? accm : (accm & ((2u << lane) - 1u));
            if (valid) {
                if (chain_idx) chain_idx[k] = le ? (g0 + base + (31 - __clz(le))) : idx_before;
                if (acc_out) acc_out[k] = (uint8_t)((accm >> lane) & 1u);
            }
            int cnt = __popc(accm);
            if (g0 + base == 0 && (accm & 1u)) cnt -= 1;   // step 0 is not counted
            nacc += cnt;
        }
    }
    if (lane == 0) {
        st->logw_cur = cur;
        st->idx_cur = idx;
        st->n_acc = nacc;
        st->step = g0 + n;
    }
}

gf_status mh_launch(gf_mh_state* d_state, int64_t n, const double* d_logw, int64_t* d_idx,
                    uint8_t* d_acc, double* d_logu, cudaStream_t stream) {
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
    mh_logu_kernel<<<(unsigned)blocks, 256, 0, stream>>>(d_state, n, d_logu);
    GF_CHECK_LAUNCH();
    mh_scan_kernel<<<1, 32, 0, stream>>>(d_state, n, d_logw, d_logu, d_idx, d_acc);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant: log u goes to a fixed device array owned by the
// library instead of caller workspace.  Host code cannot use the array's
// name as a device address, so its address is looked up once per device.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_mh_noalloc_logu[GF_MH_NOALLOC_MAX_N];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

gf_status noalloc_scratch(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GF_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return GF_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_mh_noalloc_logu) != cudaSuccess || p == nullptr) return GF_ECUDA;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return GF_OK;
}
}  // namespace

}  // namespace gf

using namespace gf;

extern "C" {

size_t gf_mh_chain_workspace_bytes(int64_t n) { return n > 0 ? (size_t)n * sizeof(double) : 0; }

gf_status gf_mh_chain(gf_mh_state* d_state, int64_t n, const double* d_logw,
                      int64_t* d_chain_idx_out, uint8_t* d_acc_out,
                      void* d_workspace, size_t workspace_bytes, cudaStream_t stream) {
    if (!d_state || n < 0) return GF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_state) & 7) != 0) return GF_EINVAL;
    if (n == 0) return GF_OK;
    if (!d_logw || !d_workspace || workspace_bytes < gf_mh_chain_workspace_bytes(n)) return GF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_workspace) & 7) != 0) return GF_EINVAL;
    return mh_launch(d_state, n, d_logw, d_chain_idx_out, d_acc_out,
                     static_cast<double*>(d_workspace), stream);
}

gf_status gf_mh_chain_noalloc(gf_mh_state* d_state, int64_t n, const double* d_logw,
                              int64_t* d_chain_idx_out, uint8_t* d_acc_out, cudaStream_t stream) {
    if (!d_state || n < 0) return GF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_state) & 7) != 0) return GF_EINVAL;
    if (n > GF_MH_NOALLOC_MAX_N) return GF_EINVAL;
    if (n == 0) return GF_OK;
    if (!d_logw) return GF_EINVAL;
    double* scratch = nullptr;
    const gf_status st = noalloc_scratch(&scratch);
    if (st != GF_OK) return st;
    return mh_launch(d_state, n, d_logw, d_chain_idx_out, d_acc_out, scratch, stream);
}

}  // extern "C"
