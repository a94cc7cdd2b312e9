// gf_mh.cu -- Metropolis-Hastings independence chain over flow proposals
// (paper arXiv:2208.08903 Sec. 1: proposals from the flow corrected by the
// MH test with the Jacobian; acceptance min(1, w'/w), w = p/q).
//
// Two kernels on the caller's stream:
//  1. mh_prep_kernel: in parallel for every step g, u_g from Philox word 0 of
//     ctr = (g, 0, 0, TAG_MH), key = (seed, stream_id), and the proposal-only
//     part of the test, a_k = log w_k - log u_g (FP64), stored as an
//     order-preserving int64 key in the workspace;
//  2. mh_scan_kernel: one warp walks the proposals in chunks of 32.  Proposal
//     k is accepted iff a_k > log w_cur (w_k / w_cur > u); every lane tests its
//     key against the current state's key (integer compares only), the first
//     lane that accepts is the chain's next accept (all earlier lanes rejected
//     against the same state), the state moves there and the lanes after it
//     are re-tested.  A chunk costs 1 + (accepts in it) ballot rounds instead
//     of 32 dependent steps.  The state stays in device memory.
#include <algorithm>
#include <mutex>

#include "gf_common.cuh"

namespace gf {

// Order-preserving map of doubles to int64 (x < y <=> key(x) < key(y) for
// non-NaN x, y; -0 and +0 map to the same key).  `nan_key` is returned for NaN.
__device__ __forceinline__ int64_t order_key(double x, int64_t nan_key) {
    if (x != x) return nan_key;
    int64_t b = __double_as_longlong(x);
    if (b == INT64_MIN) b = 0;                              // -0 -> +0
    return b >= 0 ? b : (b ^ INT64_MAX);
}

__global__ void mh_prep_kernel(const gf_mh_state* __restrict__ st, int64_t n, const double* __restrict__ logw,
                               int64_t* __restrict__ key_a) {
    const int64_t step0 = st->step;
    const uint64_t seed = st->seed, stream_id = st->stream_id;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const u64x4 w = philox4x64_10(seed, stream_id, u64x4{(uint64_t)(step0 + k), 0ull, 0ull, TAG_MH});
        key_a[k] = order_key(logw[k] - log(u53(w.x)), INT64_MIN);      // NaN never accepts
    }
}

__global__ void __launch_bounds__(32) mh_scan_kernel(gf_mh_state* __restrict__ st, int64_t n,
                                                     const double* __restrict__ logw,
                                                     const int64_t* __restrict__ key_a,
                                                     int64_t* __restrict__ chain_idx,
                                                     uint8_t* __restrict__ acc_out) {
    constexpr int kChunks = 8;                 // 256 proposals loaded per round trip to memory
    const int lane = threadIdx.x;
    double cur = st->logw_cur;
    int64_t cur_key = order_key(cur, INT64_MAX);           // a NaN state accepts nothing more
    int64_t idx = st->idx_cur, nacc = st->n_acc;
    const int64_t g0 = st->step;
    for (int64_t blk = 0; blk < n; blk += 32 * kChunks) {
        double lwv[kChunks];
        int64_t kav[kChunks];
#pragma unroll
        for (int c = 0; c < kChunks; ++c) {
            const int64_t k = blk + 32 * c + lane;
            lwv[c] = k < n ? __ldg(logw + k) : 0.0;
            kav[c] = k < n ? __ldg(key_a + k) : INT64_MIN;
        }
#pragma unroll
        for (int c = 0; c < kChunks; ++c) {
            const int64_t base = blk + 32 * c;
            if (base >= n) break;
            const int64_t k = base + lane;
            const bool valid = k < n;
            const int64_t ka = kav[c];
            const bool first = (g0 + k) == 0;
            const int64_t idx_before = idx;
            unsigned remaining = __ballot_sync(0xffffffffu, valid);
            unsigned accm = 0u;
            while (remaining) {
                const bool mine = (remaining >> lane) & 1u;
                const bool test = mine && (first || ka > cur_key);
                const unsigned m = __ballot_sync(0xffffffffu, test);
                if (m == 0u) break;
                const int j = __ffs(m) - 1;
                accm |= 1u << j;
                cur = __shfl_sync(0xffffffffu, lwv[c], j);
                cur_key = order_key(cur, INT64_MAX);
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
                    uint8_t* d_acc, int64_t* d_keys, cudaStream_t stream) {
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
    mh_prep_kernel<<<(unsigned)blocks, 256, 0, stream>>>(d_state, n, d_logw, d_keys);
    GF_CHECK_LAUNCH();
    mh_scan_kernel<<<1, 32, 0, stream>>>(d_state, n, d_logw, d_keys, d_idx, d_acc);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant: log u goes to a fixed device array owned by the
// library instead of caller workspace.  Host code cannot use the array's
// name as a device address, so its address is looked up on every call made
// outside stream capture (a device reset or a new primary context can move
// it) and cached per device; a call being captured into a graph uses the
// cached address (looked up first if there is none).
// ---------------------------------------------------------------------------
static __device__ __align__(256) int64_t g_mh_noalloc_keys[GF_MH_NOALLOC_MAX_N];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
int64_t* g_noalloc_ptr[kMaxDevices] = {};

gf_status noalloc_scratch(cudaStream_t stream, int64_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GF_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return GF_EUNSUPPORTED;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return GF_ECUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr || cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_mh_noalloc_keys) != cudaSuccess || p == nullptr) return GF_ECUDA;
        g_noalloc_ptr[dev] = static_cast<int64_t*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return GF_OK;
}
}  // namespace

}  // namespace gf

using namespace gf;

extern "C" {

size_t gf_mh_chain_workspace_bytes(int64_t n) { return n > 0 ? (size_t)n * sizeof(int64_t) : 0; }

gf_status gf_mh_chain(gf_mh_state* d_state, int64_t n, const double* d_logw,
                      int64_t* d_chain_idx_out, uint8_t* d_acc_out,
                      void* d_workspace, size_t workspace_bytes, cudaStream_t stream) {
    if (!d_state || n < 0) return GF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_state) & 7) != 0) return GF_EINVAL;
    if (n == 0) return GF_OK;
    if (!d_logw || !d_workspace || workspace_bytes < gf_mh_chain_workspace_bytes(n)) return GF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_workspace) & 7) != 0) return GF_EINVAL;
    return mh_launch(d_state, n, d_logw, d_chain_idx_out, d_acc_out,
                     static_cast<int64_t*>(d_workspace), stream);
}

gf_status gf_mh_chain_noalloc(gf_mh_state* d_state, int64_t n, const double* d_logw,
                              int64_t* d_chain_idx_out, uint8_t* d_acc_out, cudaStream_t stream) {
    if (!d_state || n < 0) return GF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_state) & 7) != 0) return GF_EINVAL;
    if (n > GF_MH_NOALLOC_MAX_N) return GF_EINVAL;
    if (n == 0) return GF_OK;
    if (!d_logw) return GF_EINVAL;
    int64_t* scratch = nullptr;
    const gf_status st = noalloc_scratch(stream, &scratch);
    if (st != GF_OK) return st;
    return mh_launch(d_state, n, d_logw, d_chain_idx_out, d_acc_out, scratch, stream);
}

}  // extern "C"
