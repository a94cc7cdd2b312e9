// gf_async.cuh -- PTX wrappers for shared-memory mbarriers and bulk
// (cp.async.bulk) copies, used by the kernels that stage their inputs
// asynchronously.
#pragma once

#include <cstdint>

namespace gf {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy, tensor core) accesses.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Arrival that also announces `bytes` of bulk-copy data for the current phase.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Bulk copy global -> shared (16-byte aligned, size a multiple of 16), completing on bar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ uint64_t mbar_arrive(uint64_t* bar) {
    uint64_t state;
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(smem_u32(bar)) : "memory");
    return state;
}

// Ring depth for records of BYTES bytes: about 16 KB in flight per block.
template <int BYTES>
__host__ __device__ constexpr int ring_depth() { return BYTES >= 8192 ? 2 : (BYTES >= 4096 ? 4 : 8); }

// A ring of NBUF shared-memory buffers that bulk copies fill with this block's
// share of a batch of equal-sized records (records blockIdx.x,
// blockIdx.x + gridDim.x, ...; the k-th of them is "local record k"), so
// later records arrive while earlier ones are read.  Thread 0 issues the
// copies; every thread waits on a record's barrier before reading it.  The
// source records and `bytes` must be multiples of 16 bytes, 16-byte aligned.
// Lives in registers, built the same way by every thread of the block.
template <int NBUF>
struct BulkRing {
    unsigned char* buf;            // NBUF x bytes of shared memory
    uint64_t* full;                // NBUF mbarriers
    const unsigned char* src;      // record 0 of the batch
    uint32_t bytes;
    int64_t count;                 // records of this block

    __device__ BulkRing(void* shared_buf, uint64_t* bars, const void* records, uint32_t record_bytes,
                        int64_t n_records)
        : buf(static_cast<unsigned char*>(shared_buf)), full(bars), src(static_cast<const unsigned char*>(records)),
          bytes(record_bytes),
          count(n_records > (int64_t)blockIdx.x ? (n_records - 1 - (int64_t)blockIdx.x) / gridDim.x + 1 : 0) {}

    __device__ const void* data(int64_t k) const { return buf + (size_t)(k % NBUF) * bytes; }

    __device__ void issue(int64_t k) const {
        if (k >= count) return;
        const int s = (int)(k % NBUF);
        mbar_expect_tx(&full[s], bytes);
        bulk_g2s(buf + (size_t)s * bytes, src + (size_t)(blockIdx.x + k * gridDim.x) * bytes, bytes, &full[s]);
    }
    // thread 0, before a __syncthreads: barriers and the first NBUF copies
    __device__ void start() const {
        for (int s = 0; s < NBUF; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
        for (int s = 0; s < NBUF; ++s) issue(s);
    }
    // bounded wait for local record k; false when the limit ran out
    __device__ bool wait(int64_t k, long long limit) const {
        const uint32_t parity = (uint32_t)((k / NBUF) & 1);
        for (long long spins = 0; !mbar_try_wait(&full[k % NBUF], parity);)
            if (++spins > limit) return false;
        return true;
    }
    // thread 0, once every thread is done reading local record k: reuse its
    // buffer for record k + NBUF
    __device__ void refill(int64_t k) const {
        fence_proxy_async();
        issue(k + NBUF);
    }
    // thread 0, when leaving with records 0..k-1 consumed: bounded waits for
    // the copies still in flight (records k .. k+NBUF-1), so none lands after
    // the block has exited
    __device__ void drain(int64_t k, long long limit) const {
        for (int64_t j = k; j < k + NBUF && j < count; ++j) wait(j, limit);
    }
};

}  // namespace gf
