// gf_flow_bf16.cu -- fused coupling stack with conv2 and conv3 on the
// 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// TMEM), for 3D lattices with L = 16 and hidden width 32.
//
// Paper arXiv:2208.08903 Sec. 1 (affine coupling layers, Jacobian, model
// density, action); precision split of this variant: conv2 and conv3 operands
// (h1, h2 and their weights) in BF16 with FP32 accumulation, conv1 and the
// affine update in FP32, the field x in FP32, and log-det, sum z^2, S, log q,
// log w in FP64.
//
// Per CTA one configuration at a time (persistent).  Within a layer the
// lattice is walked along z one 256-site slice at a time:
//   conv1 (FFMA, only the 13/14 taps that reach fixed sites) -> h1 slice (BF16)
//   conv2 as an implicit GEMM on the tensor cores -> h2 slice (BF16)
//   conv3 as an implicit GEMM (N = 16, rows s and t) -> affine update of x
// Implicit GEMM: per z-slice two M = 128 tiles (8 y-rows x 16 x); K = the 9
// (dz,dy) taps x 32 channels in steps of 16; the three dx weight sets are
// stacked along N (conv2: N = 96, conv3: N = 32), so one instruction yields
// the three dx partial sums.  Activations are stored channel-
// group major ([4][288 sites][8 ch], 288 = 18 y-rows with one periodic halo row
// on each side), so each 8-site core matrix is 128 contiguous bytes and a
// (dz,dy) shift is only a different start address.  The periodic x-shift is
// not gathered: three accumulators P_dx (dx = -1, 0, +1) stay in TMEM and the
// epilogues form out(x) = sum_dx P_dx(x + dx) with width-16 shuffles (one
// x-row = one half-warp = 16 TMEM lanes).
// Warp-specialised pipeline within a layer (mbarriers only, no CTA barrier):
// producer warps run conv1 on the FMA pipes up to four slices ahead (four h1
// slots); one thread of warp 0 queues conv2 of slice u (into one of two TMEM
// buffers) and then conv3 of slice u-2 (two TMEM buffers) on the tensor cores;
// four epilogue warps turn conv2 accumulators into h2 (three slots) and conv3
// accumulators into the affine update of x.  conv1 reads only fixed sites of
// x and the update writes only the other parity, so x needs no ordering within
// a layer; the CTA meets at a barrier between layers.
#include <algorithm>
#include <cstring>

#include <cuda_bf16.h>

#include "gf_flow.cuh"

namespace gf {

namespace {

constexpr int kThreads = 512;
constexpr int kL = 16, kS = 256, kC = 32, kT = 27;
constexpr int kHaloSites = 18 * 16;                    // y = -1 .. 16
constexpr int kCgStride = kHaloSites * 16;             // bytes between channel groups
constexpr int kSlotBytes = 4 * kCgStride;              // [cg][site][8] bf16 = 18432
// conv2 B operand per (dz,dy) tap pair: the three dx weight sets stacked along N
// (N = 96: row dxi*32 + o); conv3 B: rows dxi*8 + {s, t, 6 zeros} for dxi < 3 and
// 8 zero rows (N = 32).  Layout [tap9][kg][n][8] bf16 (K-major core matrices).
constexpr int kW2Bytes = 9 * 4 * 96 * 16;              // 55296
constexpr int kW3Bytes = 9 * 4 * 32 * 16;              // 18432
// FP32 part of a layer block (floats): W1s[t][c], b1[c], b2[c], b3[2], pad
constexpr int kF_W1 = 0, kF_b1 = kT * kC, kF_b2 = kF_b1 + kC, kF_b3 = kF_b2 + kC;
constexpr int kF_N = (kF_b3 + 2 + 3) & ~3;
constexpr int kLayerBytes = kW2Bytes + kW3Bytes + kF_N * 4;
constexpr int kTmem3 = 192;                             // conv3 accumulators (2 tiles x 32 columns)
constexpr int kTmem2B = 256;                            // second conv2 buffer (2 tiles x 96 columns)
constexpr int kTmemCols = 512;
constexpr long long kWaitLimit = 1ll << 22;             // bounded mbarrier wait (iterations)
constexpr int kProdWarp0 = 4, kProdWarps = 8, kProdThreads = kProdWarps * 32;   // conv1 producers
constexpr int kEpiWarp0 = 12, kEpiThreads = 4 * 32;                            // epilogue warps 12..15

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(dst)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (BF16 in, FP32 accumulate).
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}
// 32 lanes x 16 consecutive FP32 columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr) : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// 32 lanes x 2 consecutive FP32 columns.
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float& a, float& b) {
    uint32_t r0, r1;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr) : "memory");
    a = __uint_as_float(r0);
    b = __uint_as_float(r1);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// core matrix = 8 rows x 16 bytes contiguous; LBO = byte distance between
// core matrices adjacent in K, SBO = between 8-row groups.  The start address
// occupies the low 14 bits (in 16-byte units): adding (bytes >> 4) to a
// descriptor moves its start; every shared address here is below 256 KB, so
// the field never carries into LBO.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;              // descriptor version for tcgen05
    return d;                            // base offset 0, swizzle mode 0 (none)
}
// Instruction descriptors: D = F32, A = B = BF16, both K-major, M = 128, N = 96 / 32.
constexpr uint32_t kIdesc96 = (1u << 4) | (1u << 7) | (1u << 10) | ((96u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdesc32 = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

struct Bf16Args {
    const unsigned char* Wl;   // per-layer blocks of kLayerBytes
    int n_layers;
    float slope;
    int use_tanh, has_phi4;
    double m2, lam;
    int64_t B;
    uint64_t seed, counter0;
    const float* z_in; float* z_out; const float* phi_in; float* phi_out;
    double* logq_out; double* S_out; double* logw_out;
    int32_t* status;
};

__device__ __forceinline__ int wrap16(int v) { return v & 15; }

// halo-row site index of interior (y, x), y in -1..16
__device__ __forceinline__ int hsite(int y, int x) { return (y + 1) * 16 + x; }

// Stores 8 channels (one channel group) of a site in BF16, plus the periodic
// halo copy when the row is y = 0 or y = 15.
__device__ __forceinline__ void store8(unsigned char* slot, int cg, int y, int x, const float* v) {
    __align__(16) __nv_bfloat162 p[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const uint4 w = *reinterpret_cast<const uint4*>(p);
    unsigned char* base = slot + (size_t)cg * kCgStride;
    *reinterpret_cast<uint4*>(base + hsite(y, x) * 16) = w;
    if (y == 0) *reinterpret_cast<uint4*>(base + hsite(16, x) * 16) = w;
    if (y == 15) *reinterpret_cast<uint4*>(base + hsite(-1, x) * 16) = w;
}

// Virtual slice v (may lie outside 0..L-1 by the wrap-around recomputation)
// -> lattice slice v mod L; h1 slot v mod 4, h2 slot v mod 3.
__device__ __forceinline__ int slice_of(int v) { return v & 15; }
__device__ __forceinline__ int h1_slot(int v) { return (v + 16) & 3; }
__device__ __forceinline__ int h2_slot(int v) { return (v + 15) % 3; }

// The taps of conv1 that reach fixed sites from an output site of parity p are
// those whose offset parity (|dz|+|dy|+|dx|) mod 2 equals NEED = frozen ^ p; the
// tap set is chosen at compile time, so the loop has no branches.  Two sites
// (rows y and y + 8, same parity) share each tap's weight loads.
template <int NEED>
__device__ __forceinline__ void conv1_taps2(float (&acc)[2][8], const float* wf, const float* x, const int (&zr)[3],
                                            const int (&yr)[2][3], const int (&xc)[2][3], int cg) {
#pragma unroll
    for (int t = 0; t < kT; ++t) {
        const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
        if (((dz + dy + dx + 1) & 1) != NEED) continue;                     // resolved at compile time
        const float x0 = x[zr[dz] + yr[0][dy] + xc[0][dx]];
        const float x1 = x[zr[dz] + yr[1][dy] + xc[1][dx]];
        const float4 w0 = *reinterpret_cast<const float4*>(wf + kF_W1 + t * kC + cg * 8);
        const float4 w1 = *reinterpret_cast<const float4*>(wf + kF_W1 + t * kC + cg * 8 + 4);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            acc[0][c] = fmaf(x0, w[c], acc[0][c]);
            acc[1][c] = fmaf(x1, w[c], acc[1][c]);
        }
    }
}

// conv1 + LReLU of virtual slice v into its h1 slot (BF16).  512 work items:
// (channel group, site parity class, 64 site pairs) spread over the producer
// threads (ptid < kProdThreads); a warp holds sites of one parity, so all its
// lanes take the same 13 or 14 taps.  Neighbouring lanes alternate between
// rows y and y+1, which keeps the 16-byte stores free of bank conflicts.
__device__ __forceinline__ void conv1_slice(unsigned char* h1, int v, const float* wf, const float* x, int frozen,
                                            float slope, int ptid) {
    const int z = slice_of(v);
    unsigned char* slot = h1 + (size_t)h1_slot(v) * kSlotBytes;
#pragma unroll 1
    for (int it = ptid; it < kS * 2; it += kProdThreads) {
        const int cg = it >> 7, rest = it & 127, pcls = rest >> 6, k = rest & 63;
        int ys[2], xs[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            ys[q] = 2 * (k >> 4) + (k & 1) + 8 * q;
            xs[q] = 2 * ((k >> 1) & 7) + ((pcls ^ z ^ ys[q]) & 1);        // parity pcls
        }
        int zr[3], yr[2][3], xc[2][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            zr[d] = wrap16(z + d - 1) << 8;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                yr[q][d] = wrap16(ys[q] + d - 1) << 4;
                xc[q][d] = wrap16(xs[q] + d - 1);
            }
        }
        const float4 b0 = *reinterpret_cast<const float4*>(wf + kF_b1 + cg * 8);
        const float4 b1 = *reinterpret_cast<const float4*>(wf + kF_b1 + cg * 8 + 4);
        float acc[2][8];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            acc[q][0] = b0.x; acc[q][1] = b0.y; acc[q][2] = b0.z; acc[q][3] = b0.w;
            acc[q][4] = b1.x; acc[q][5] = b1.y; acc[q][6] = b1.z; acc[q][7] = b1.w;
        }
        if ((frozen ^ pcls) & 1) conv1_taps2<1>(acc, wf, x, zr, yr, xc, cg);
        else conv1_taps2<0>(acc, wf, x, zr, yr, xc, cg);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[q][c] = acc[q][c] > 0.f ? acc[q][c] : slope * acc[q][c];
            store8(slot, cg, ys[q], xs[q], acc[q]);
        }
    }
}

// One elected thread: an implicit-GEMM convolution of a slice: for each of the
// 2 M-tiles, 9 (dz,dy) taps x 2 K-steps of tcgen05.mma, each producing the three
// dx partial sums at once (B holds the dx weight sets stacked along N).
// a_slot[dzi] = A descriptors of the three input slices; b0 = B descriptor of
// tap pair 0, K-step 0; tap pair p, K-step k adds p * b_tap + k * b_k (16-byte units).
__device__ __forceinline__ void issue_conv(const uint64_t (&a_slot)[3], uint64_t b0, uint32_t b_tap, uint32_t b_k,
                                           uint32_t d0, uint32_t d_tile, uint32_t idesc) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const uint32_t d = d0 + (uint32_t)mt * d_tile;
#pragma unroll
        for (int dzi = 0; dzi < 3; ++dzi) {
#pragma unroll
            for (int dyi = 0; dyi < 3; ++dyi) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const uint64_t ad = a_slot[dzi] + (uint64_t)((2 * k * kCgStride + (mt * 8 + dyi) * 256) >> 4);
                    const uint64_t bd = b0 + (uint64_t)((dzi * 3 + dyi) * b_tap + k * b_k);
                    mma_bf16(d, ad, bd, idesc, (dzi | dyi | k) ? 1u : 0u);
                }
            }
        }
    }
}

// conv2 epilogue, one (tile mt, TMEM lane quarter q, channel half hf) part:
// out(x) = sum_dx P_dx(x + dx) + b2, LReLU, BF16 into the h2 slot of v.
__device__ __forceinline__ void conv2_epilogue_part(unsigned char* h2, uint32_t tmem, int v, const float* wf,
                                                    float slope, int mt, int q, int hf, int lane) {
    const int y = mt * 8 + q * 2 + (lane >> 4), xx = lane & 15;
    float pm[16], p0[16], pp[16];
    const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hf * 16);
    tmem_ld16(base + (uint32_t)((mt * 3 + 0) * 32), pm);
    tmem_ld16(base + (uint32_t)((mt * 3 + 1) * 32), p0);
    tmem_ld16(base + (uint32_t)((mt * 3 + 2) * 32), pp);
    tmem_ld_wait();
    const int src_m = (lane & 16) | ((xx + 15) & 15);   // x - 1
    const int src_p = (lane & 16) | ((xx + 1) & 15);    // x + 1
    unsigned char* slot = h2 + (size_t)h2_slot(v) * kSlotBytes;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const float4 bA = *reinterpret_cast<const float4*>(wf + kF_b2 + hf * 16 + g * 8);
        const float4 bB = *reinterpret_cast<const float4*>(wf + kF_b2 + hf * 16 + g * 8 + 4);
        const float bias[8] = {bA.x, bA.y, bA.z, bA.w, bB.x, bB.y, bB.z, bB.w};
        float o[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int ch = g * 8 + c;
            const float s = p0[ch] + __shfl_sync(0xffffffffu, pm[ch], src_m) +
                            __shfl_sync(0xffffffffu, pp[ch], src_p) + bias[c];
            o[c] = s > 0.f ? s : slope * s;
        }
        store8(slot, hf * 2 + g, y, xx, o);
    }
}

// conv3 epilogue of slice z, tile mt, lane quarter q: (s, t) = sum_dx P3_dx(x + dx)
// + b3 for every site; the updated sites apply the affine map and accumulate
// the log-det.  tmem3 = the conv3 accumulator buffer (2 tiles x 32 columns).
__device__ __forceinline__ void conv3_epilogue_part(uint32_t tmem3, int z, const float* wf, float* x, int frozen,
                                                    int use_tanh, bool inverse, double& logdet, int mt, int q,
                                                    int lane) {
    const int y = mt * 8 + q * 2 + (lane >> 4), xx = lane & 15;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    float sm, tm, s0, t0, sp, tp;
    tmem_ld2(tmem3 + lane_base + (uint32_t)(mt * 32 + 0), sm, tm);
    tmem_ld2(tmem3 + lane_base + (uint32_t)(mt * 32 + 8), s0, t0);
    tmem_ld2(tmem3 + lane_base + (uint32_t)(mt * 32 + 16), sp, tp);
    tmem_ld_wait();
    const int src_m = (lane & 16) | ((xx + 15) & 15);
    const int src_p = (lane & 16) | ((xx + 1) & 15);
    const float spre = s0 + __shfl_sync(0xffffffffu, sm, src_m) + __shfl_sync(0xffffffffu, sp, src_p) + wf[kF_b3];
    const float tt = t0 + __shfl_sync(0xffffffffu, tm, src_m) + __shfl_sync(0xffffffffu, tp, src_p) + wf[kF_b3 + 1];
    if (((z + y + xx) & 1) != frozen) {
        const float s = use_tanh ? tanhf(spre) : spre;
        float& xv = x[(z * 16 + y) * 16 + xx];
        if (!inverse) xv = fmaf(xv, expf(s), tt);
        else xv = (xv - tt) * expf(-s);
        logdet += (double)s;
    }
}

// Bounded wait for completion number `n` (0-based) of an mbarrier: parity of
// n.  Returns false (and raises the CTA's abort flag, recording GF_ETIMEOUT)
// when the limit runs out, or at once when another thread already aborted.
// Every waiter is at most one completion behind the barrier (the pipeline's
// dependencies guarantee it), so the parity identifies the completion.
__device__ __forceinline__ bool wait_n(uint64_t* bar, int n, volatile int* abort_flag, int32_t* status) {
    long long spins = 0;
    while (!mbar_try_wait(bar, (uint32_t)n & 1u)) {
        if (*abort_flag) return false;
        if (++spins > kWaitLimit) { *abort_flag = 1; set_status(status, GF_ETIMEOUT); return false; }
    }
    return true;
}
__device__ __forceinline__ uint64_t mbar_arrive(uint64_t* bar) {
    uint64_t state;
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(smem_u32(bar)) : "memory");
    return state;
}

// Per layer and CTA: 20 conv1 slices (virtual v = -2..17), 18 conv2 slices
// (u = -1..16) and 16 conv3 slices (w = 0..15).  With seq = the CTA's running
// layer count, the global numbers c = 20 seq + v + 2, g2 = 18 seq + u + 1 and
// g3 = 16 seq + w index the barrier completions:
//   h1 slot c % 4 (barrier bar_h1[c % 4], completion c / 4),
//   conv2 TMEM buffer g2 & 1 (bar_m2 / bar_t2 completion g2 >> 1), h2 slot g2 % 3
//   (bar_h2, completion g2 / 3), conv3 TMEM buffer g3 & 1 (bar_m3 / bar_t3, g3 >> 1).
constexpr int kConv1PerLayer = 20, kConv2PerLayer = 18, kConv3PerLayer = kL;

// Warp roles: warp 0 (one lane) issues every tcgen05.mma; warps 4..11 compute
// conv1 (FFMA) into the h1 slots; warps 12..15 (TMEM lane quarter = warp & 3)
// run the conv2 and conv3 epilogues.  They synchronise through mbarriers only,
// so the tensor cores, the FMA pipes and the epilogues overlap; the CTA meets
// at a barrier only between layers.
template <bool INVERSE>
__global__ void __launch_bounds__(kThreads, 1) flow_bf16_kernel(const Bf16Args a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* w2s = smem;                                                 // kW2Bytes
    unsigned char* w3s = smem + kW2Bytes;                                      // kW3Bytes
    float* wf = reinterpret_cast<float*>(smem + kW2Bytes + kW3Bytes);          // kF_N floats
    unsigned char* h1 = smem + kLayerBytes;                                    // 4 slots
    unsigned char* h2 = h1 + 4 * kSlotBytes;                                   // 3 slots
    float* x = reinterpret_cast<float*>(h2 + 3 * kSlotBytes);                  // 4096 floats
    double* red = reinterpret_cast<double*>(x + 4096);                         // 32
    uint64_t* bar_h1 = reinterpret_cast<uint64_t*>(red + 32);  // 4: h1 slot written (producers)
    uint64_t* bar_h2 = bar_h1 + 4;                             // 3: h2 slot written (epilogue)
    uint64_t* bar_m2 = bar_h2 + 3;                             // 2: conv2 MMAs done (commit)
    uint64_t* bar_m3 = bar_m2 + 2;                             // 2: conv3 MMAs done (commit)
    uint64_t* bar_t2 = bar_m3 + 2;                             // 2: conv2 TMEM buffer drained
    uint64_t* bar_t3 = bar_t2 + 2;                             // 2: conv3 TMEM buffer drained
    uint64_t* bar_fin = bar_t3 + 2;                            // 1: every queued MMA done (exit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_fin + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int V = 4096;
    if (warp == 0) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(bar_h1 + i, kProdThreads);
        for (int i = 0; i < 3; ++i) mbar_init(bar_h2 + i, kEpiThreads);
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar_m2 + i, 1);
            mbar_init(bar_m3 + i, 1);
            mbar_init(bar_t2 + i, kEpiThreads);
            mbar_init(bar_t3 + i, kEpiThreads);
        }
        mbar_init(bar_fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    // conv2 buffers at columns 0 and 256 (2 tiles x 96), conv3 buffers at 192 and 448 (2 tiles x 32)
    const auto t2buf = [tmem](int b) { return tmem + (b ? kTmem2B : 0u); };
    const auto t3buf = [tmem](int b) { return tmem + (uint32_t)kTmem3 + (b ? kTmem2B : 0u); };

    // A descriptors of every h1 / h2 slot (LBO = channel-group stride, SBO = 8 sites);
    // B: conv2 LBO = 96 rows x 16 B between K groups, conv3 LBO = 32 rows x 16 B, SBO = 128.
    const uint64_t a1_0 = smem_desc(smem_u32(h1), kCgStride, 128);
    const uint64_t a2_0 = smem_desc(smem_u32(h2), kCgStride, 128);
    const auto a1 = [a1_0](int slot) { return a1_0 + (uint64_t)(slot * (kSlotBytes >> 4)); };
    const auto a2 = [a2_0](int slot) { return a2_0 + (uint64_t)(slot * (kSlotBytes >> 4)); };
    const uint64_t b2d = smem_desc(smem_u32(w2s), 96 * 16, 128);
    const uint64_t b3d = smem_desc(smem_u32(w3s), 32 * 16, 128);

    int seq = 0;                                   // layers processed by this CTA so far
    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        double sumz2 = 0.0;
        if (!INVERSE) {
            if (a.z_in) {
                for (int n = tid; n < V; n += kThreads) {
                    const float v = __ldg(a.z_in + b * V + n);
                    x[n] = v;
                    sumz2 += (double)v * v;
                }
            } else {
                for (int j = tid; 4 * j < V; j += kThreads) {
                    const u64x4 w = philox4x64_10(a.seed, 0ull,
                                                  u64x4{a.counter0 + (uint64_t)b, (uint64_t)j, 0ull, TAG_PRIOR});
                    float zz[4];
                    normals4_f32(w, zz);
#pragma unroll
                    for (int q = 0; q < 4; ++q) { x[4 * j + q] = zz[q]; sumz2 += (double)zz[q] * zz[q]; }
                }
            }
            __syncthreads();
            if (a.z_out)
                for (int n = tid; n < V; n += kThreads) a.z_out[b * V + n] = x[n];
        } else {
            for (int n = tid; n < V; n += kThreads) x[n] = __ldg(a.phi_in + b * V + n);
        }
        __syncthreads();

        double logdet = 0.0;
        for (int li = 0; li < a.n_layers; ++li, ++seq) {
            const int l = INVERSE ? a.n_layers - 1 - li : li;
            const int frozen = l & 1;
            {   // stage this layer's weights (W2, W3 already in the MMA operand layouts)
                const uint4* src = reinterpret_cast<const uint4*>(a.Wl + (size_t)l * kLayerBytes);
                uint4* dst = reinterpret_cast<uint4*>(smem);
                for (int i = tid; i < kLayerBytes / 16; i += kThreads) dst[i] = __ldg(src + i);
            }
            fence_proxy_async();
            __syncthreads();
            const int c0 = seq * kConv1PerLayer, g20 = seq * kConv2PerLayer, g30 = seq * kConv3PerLayer;

            if (warp == 0) {
                // ---------------- tensor-core issue (one thread)
                if (lane == 0) {
                    auto wait_h1 = [&](int v) {
                        const int c = c0 + v + 2;
                        return wait_n(bar_h1 + (c & 3), c >> 2, abort_flag, a.status);
                    };
                    auto wait_h2 = [&](int u) {
                        const int g = g20 + u + 1;
                        return wait_n(bar_h2 + g % 3, g / 3, abort_flag, a.status);
                    };
                    auto issue3 = [&](int w) {
                        const int g3 = g30 + w;
                        if (g3 >= 2 && !wait_n(bar_t3 + (g3 & 1), (g3 - 2) >> 1, abort_flag, a.status)) return;
                        fence_after_sync();
                        const uint64_t as[3] = {a2(h2_slot(w - 1)), a2(h2_slot(w)), a2(h2_slot(w + 1))};
                        issue_conv(as, b3d, (4 * 32 * 16) >> 4, (2 * 32 * 16) >> 4, t3buf(g3 & 1), 32, kIdesc32);
                        mma_commit(bar_m3 + (g3 & 1));
                    };
                    for (int u = -1; u <= kL && !*abort_flag; ++u) {
                        if (u == -1) {
                            if (!wait_h1(-2) || !wait_h1(-1) || !wait_h1(0)) break;
                        } else if (!wait_h1(u + 1)) {
                            break;
                        }
                        const int g2 = g20 + u + 1;
                        if (g2 >= 2 && !wait_n(bar_t2 + (g2 & 1), (g2 - 2) >> 1, abort_flag, a.status)) break;
                        fence_after_sync();
                        const uint64_t as[3] = {a1(h1_slot(u - 1)), a1(h1_slot(u)), a1(h1_slot(u + 1))};
                        issue_conv(as, b2d, (4 * 96 * 16) >> 4, (2 * 96 * 16) >> 4, t2buf(g2 & 1), 96, kIdesc96);
                        mma_commit(bar_m2 + (g2 & 1));
                        if (u >= 2) {                    // conv3 of slice u - 2 reads h2[u-3 .. u-1]
                            if (u == 2 && (!wait_h2(-1) || !wait_h2(0))) break;
                            if (!wait_h2(u - 1)) break;
                            issue3(u - 2);
                        }
                    }
                    // the loop issued conv3 of slices 0 .. L-2; slice L-1 reads h2[L-2 .. L]
                    if (!*abort_flag && wait_h2(kL)) issue3(kL - 1);
                }
                __syncwarp();
            } else if (warp >= kProdWarp0 && warp < kProdWarp0 + kProdWarps) {
                // ---------------- conv1 producers
                const int ptid = tid - kProdWarp0 * 32;
                for (int v = -2; v <= kL + 1 && !*abort_flag; ++v) {
                    if (v >= 2) {                        // slot of h1[v-4] is free once conv2 of slice v-3 is done
                        const int g2 = g20 + v - 2;
                        if (!wait_n(bar_m2 + (g2 & 1), g2 >> 1, abort_flag, a.status)) break;
                    }
                    conv1_slice(h1, v, wf, x, frozen, a.slope, ptid);
                    fence_proxy_async();
                    mbar_arrive(bar_h1 + ((c0 + v + 2) & 3));
                }
            } else if (warp >= kEpiWarp0) {
                // ---------------- epilogues (TMEM lane quarter q)
                const int q = warp & 3;
                auto epi3 = [&](int w) {
                    const int g3 = g30 + w;
                    if (!wait_n(bar_m3 + (g3 & 1), g3 >> 1, abort_flag, a.status)) return false;
                    fence_after_sync();
                    for (int mt = 0; mt < 2; ++mt)
                        conv3_epilogue_part(t3buf(g3 & 1), slice_of(w), wf, x, frozen, a.use_tanh, INVERSE, logdet,
                                            mt, q, lane);
                    fence_before_sync();
                    mbar_arrive(bar_t3 + (g3 & 1));
                    return true;
                };
                for (int u = -1; u <= kL && !*abort_flag; ++u) {
                    const int g2 = g20 + u + 1;
                    if (u >= 2) {                        // h2 slot of u held h2[u-3], last read by conv3 of u-2
                        const int g3 = g30 + u - 2;
                        if (!wait_n(bar_m3 + (g3 & 1), g3 >> 1, abort_flag, a.status)) break;
                    }
                    if (!wait_n(bar_m2 + (g2 & 1), g2 >> 1, abort_flag, a.status)) break;
                    fence_after_sync();
                    for (int mt = 0; mt < 2; ++mt)
                        for (int hf = 0; hf < 2; ++hf)
                            conv2_epilogue_part(h2, t2buf(g2 & 1), u, wf, a.slope, mt, q, hf, lane);
                    fence_before_sync();
                    mbar_arrive(bar_t2 + (g2 & 1));
                    fence_proxy_async();
                    mbar_arrive(bar_h2 + g2 % 3);
                    if (u >= 2 && !epi3(u - 2)) break;
                }
                if (!*abort_flag) epi3(kL - 1);     // the loop handled conv3 of slices 0 .. L-2
            }
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
            if (*abort_flag) break;
        }
        if (*abort_flag) break;

        if (INVERSE) {
            for (int n = tid; n < V; n += kThreads) {
                const float v = x[n];
                sumz2 += (double)v * v;
                if (a.z_out) a.z_out[b * V + n] = v;
            }
        } else {
            for (int n = tid; n < V; n += kThreads) a.phi_out[b * V + n] = x[n];
        }
        const double ld = block_sum(logdet, red);
        const double z2 = block_sum(sumz2, red);
        double S = 0.0;
        if (!INVERSE && a.has_phi4) {
            // forward-hop arrangement of the action: (2d + m2) phi^2 + lam phi^4 - 2 phi sum_mu phi(n + mu)
            const double c2d = 6.0 + a.m2;
            double acc = 0.0;
            for (int n = tid; n < V; n += kThreads) {
                const int xc = n & 15, yc = (n >> 4) & 15, zc = n >> 8;
                const double hop = (double)x[(n & ~15) | wrap16(xc + 1)] +
                                   (double)x[(zc << 8) | (wrap16(yc + 1) << 4) | xc] +
                                   (double)x[(wrap16(zc + 1) << 8) | (yc << 4) | xc];
                const double c = x[n], qq = c * c;
                acc += fma(qq, fma(a.lam, qq, c2d), -2.0 * c * hop);
            }
            S = block_sum(acc, red);
        }
        if (tid == 0) {
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
    if (tid == 0) {
        // after an abort some MMAs may still be queued: wait (bounded) until all
        // of this thread's tensor-core work is done before TMEM is freed
        mma_commit(bar_fin);
        for (long long spins = 0; !mbar_try_wait(bar_fin, 0u) && spins < kWaitLimit; ++spins) {}
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(tmem, kTmemCols);
    }
}

constexpr size_t kSmemBytes = (size_t)kLayerBytes + 7 * (size_t)kSlotBytes + 4096 * 4 + 32 * 8 +
                              16 * 8 + 4 + 4;

// canonical FP32 -> per-layer block: W2 [tap9][kg][dxi*32 + o][8] bf16,
// W3 [tap9][kg][dxi*8 + j][8] bf16 (j = 0: s, 1: t, else 0; rows 24..31 zero),
// then FP32 W1s[t][c], b1, b2, b3.
__global__ void repack_bf16_kernel(const float* __restrict__ canon, int64_t cstride, int n_layers,
                                   unsigned char* __restrict__ out) {
    constexpr int n2 = 9 * 4 * 96 * 8, n3 = 9 * 4 * 32 * 8;
    const int64_t per = n2 + n3 + kF_N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per * n_layers;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / per);
        const int64_t r = i - l * per;
        const float* W = canon + l * cstride;
        const float* W1 = W;                    // [c][0][t]
        const float* b1 = W1 + kC * kT;
        const float* W2 = b1 + kC;              // [o][i][t]
        const float* b2 = W2 + kC * kC * kT;
        const float* W3 = b2 + kC;              // [o][i][t]
        const float* b3 = W3 + 2 * kC * kT;
        unsigned char* blk = out + (size_t)l * kLayerBytes;
        if (r < n2) {
            const int e = (int)(r & 7), row = (int)((r >> 3) % 96), kg = (int)((r / 768) & 3), tp = (int)(r / 3072);
            const int dxi = row >> 5, o = row & 31, t = tp * 3 + dxi;
            const float v = W2[((int64_t)o * kC + kg * 8 + e) * kT + t];
            reinterpret_cast<__nv_bfloat16*>(blk)[r] = __float2bfloat16_rn(v);
        } else if (r < n2 + n3) {
            const int r3 = (int)(r - n2);
            const int e = r3 & 7, row = (r3 >> 3) & 31, kg = (r3 >> 8) & 3, tp = r3 >> 10;
            const int dxi = row >> 3, j = row & 7, t = tp * 3 + dxi;
            const float v = (dxi < 3 && j < 2) ? W3[((int64_t)j * kC + kg * 8 + e) * kT + t] : 0.f;
            reinterpret_cast<__nv_bfloat16*>(blk + kW2Bytes)[r3] = __float2bfloat16_rn(v);
        } else {
            const int f = (int)(r - n2 - n3);
            float v = 0.f;
            if (f < kF_b1) v = W1[(f % kC) * kT + f / kC];
            else if (f < kF_b2) v = b1[f - kF_b1];
            else if (f < kF_b3) v = b2[f - kF_b2];
            else if (f < kF_b3 + 2) v = b3[f - kF_b3];
            reinterpret_cast<float*>(blk + kW2Bytes + kW3Bytes)[f] = v;
        }
    }
}

}  // namespace

bool bf16_supported(const gf_flow_shape* s) {
    return s && s->nd == 3 && s->L == kL && s->c_hidden1 == kC && s->c_hidden2 == kC && s->ksize == 3;
}

gf_status bf16_configure(gf_flow* f) {
    if (!bf16_supported(&f->shape)) return GF_EUNSUPPORTED;
    f->smem_bytes_bf16 = kSmemBytes;
    if (cudaMalloc(&f->d_bf16, (size_t)kLayerBytes * std::max(1, f->shape.n_layers)) != cudaSuccess)
        return GF_ENOMEM;
    return GF_OK;
}

gf_status repack_bf16(gf_flow* f, cudaStream_t stream) {
    const int64_t total = (int64_t)(9 * 4 * 96 * 8 + 9 * 4 * 32 * 8 + kF_N) * f->shape.n_layers;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 4096);
    if (total == 0) return GF_OK;
    repack_bf16_kernel<<<grid, 256, 0, stream>>>(f->d_canon, f->canon_stride, f->shape.n_layers,
                                                 static_cast<unsigned char*>(f->d_bf16));
    GF_CHECK_LAUNCH();
    return GF_OK;
}

gf_status launch_flow_bf16(const gf_flow* f, bool inverse, const gf_phi4* phi4, int64_t B,
                           uint64_t seed, uint64_t counter0, const float* z_in, float* z_out,
                           const float* phi_in, float* phi_out, double* logq_out,
                           double* S_out, double* logw_out, cudaStream_t stream) {
    Bf16Args a;
    std::memset(&a, 0, sizeof(a));
    a.Wl = static_cast<const unsigned char*>(f->d_bf16);
    a.n_layers = f->shape.n_layers;
    a.slope = (float)f->shape.leaky_slope;
    a.use_tanh = f->shape.use_final_tanh;
    a.has_phi4 = phi4 != nullptr;
    a.m2 = phi4 ? phi4->m2 : 0.0;
    a.lam = phi4 ? phi4->lam : 0.0;
    a.B = B; a.seed = seed; a.counter0 = counter0;
    a.z_in = z_in; a.z_out = z_out; a.phi_in = phi_in; a.phi_out = phi_out;
    a.logq_out = logq_out; a.S_out = S_out; a.logw_out = logw_out;
    a.status = status_word();
    if (!a.status) return GF_ECUDA;
    auto kern = inverse ? flow_bf16_kernel<true> : flow_bf16_kernel<false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess)
        return GF_ECUDA;
    const int64_t grid = std::min<int64_t>(B, (int64_t)num_sms());
    kern<<<(unsigned)grid, kThreads, kSmemBytes, stream>>>(a);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

}  // namespace gf
