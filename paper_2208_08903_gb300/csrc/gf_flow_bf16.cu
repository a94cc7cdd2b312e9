// gf_flow_bf16.cu -- fused coupling stack with conv1, conv2 and conv3 on the
// 5th-generation tensor cores (tcgen05, 16-bit operands, FP32 accumulation in
// TMEM), for 3D lattices with L = 16 and hidden width 32.
//
// Paper arXiv:2208.08903 Sec. 1 (affine coupling layers, Jacobian, model
// density, action); precision split of this variant: conv2 (95 % of the
// FLOPs) reads BF16 operands (h1 and W2); conv1 and conv3 read FP16 operands
// (the masked field and W1; h2 and W3) at the same tensor-core rate, because
// the BF16 rounding of those weights moved log w the most (on a trained 3D
// flow it cost a fifth of the MH acceptance); every convolution accumulates
// in FP32; the field x and the affine update stay FP32; each thread sums its
// log-det terms, z^2 and action terms in FP32 pairs (about 2^-48 relative, with
// no FP64 instruction per site), and the block sums, log q and log w are FP64.
//
// Per CTA one configuration at a time (persistent).  Within a layer the
// lattice is walked along z one 256-site slice at a time:
//   conv1: per parity tile (M = 128 sites of one parity, K = the 13 or 14 taps
//   that reach fixed sites, padded to 16, N = 32) -> h1 slice (BF16)
//   conv2 as an implicit GEMM -> h2 slice (FP16)
//   conv3 as an implicit GEMM (rows s and t) -> affine update of x
// Implicit GEMM: per z-slice two M = 128 tiles (8 y-rows x 16 x); K = the 9
// (dz,dy) taps x 32 channels in steps of 16; the three dx weight sets are
// stacked along N (conv2: N = 96; conv3: N = 32 with its three dz parts
// stacked too), so one instruction yields the three dx partial sums.
// Activations are stored channel-group major ([4][288 sites][8 ch], 288 = 18
// y-rows with one periodic halo row on each side), so each 8-site core matrix
// is 128 contiguous bytes and a (dz,dy) shift is only a different start
// address.  The periodic x-shift is not gathered: the epilogues form
// out(x) = sum_dx P_dx(x + dx) with width-16 shuffles (one x-row = one
// half-warp = 16 TMEM lanes).
// Warp-specialised pipeline (mbarriers only, no CTA barrier):
// eight conv1 worker warps gather each slice's conv1 operand (the field at the
// live taps, FP16) two slices ahead and turn the conv1 accumulators into h1
// (four h1 slots); four single threads, one per sub-partition, queue the
// tensor-core work: conv2 of M-tile 0, conv2 of M-tile 1 (one TMEM buffer per
// M-tile), the conv3 batches (once h2[u] exists, one batch with every
// contribution of h2[u]: the three dz parts stacked along N, so each h2 tile is
// read from shared memory three times instead of nine; three TMEM batch
// regions) and conv1; eight epilogue warps turn conv2 accumulators into h2
// (three slots) and, from three batch regions, the conv3 result into the affine
// update of x.  An issuing thread stalls behind its own queued MMAs, so each
// kind of work has its own issuer and none waits for another's backlog.  conv1 reads only fixed sites
// of x and the update writes only the other parity, so x needs no ordering
// within a layer.  Layers follow one another without a CTA barrier: each layer
// walks the slices from a start rotated by 4, so its first conv1 slices read
// field slices that the previous layer finished early; four checkpoint barriers
// per layer tell the conv1 workers which slices the previous layer has updated,
// and the workers stage the next layer's weights (bulk copies for W2 and W3) as
// soon as the previous layer's last conv2 / conv3 has finished.
#include <algorithm>
#include <atomic>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gf_async.cuh"
#include "gf_flow.cuh"
#include "gf_tcgen05.cuh"

namespace gf {

namespace {

constexpr int kThreads = 20 * 32;                      // 4 MMA-issuing, 8 epilogue, 8 conv1 warps
constexpr int kL = 16, kC = 32, kT = 27;
constexpr int kHaloSites = 18 * 16;                    // y = -1 .. 16
constexpr int kCgStride = kHaloSites * 16;             // bytes between channel groups
constexpr int kSlotBytes = 4 * kCgStride;              // [cg][site][8] bf16 = 18432
// conv2 B operand per (dz,dy) tap pair: the three dx weight sets stacked along N
// (N = 96: row dxi*32 + o), layout [tap9][kg][n][8] bf16 (K-major core matrices).
// conv3 B operand per dy tap: the three dz parts and three dx weight sets of s
// and t stacked along N (N = 32: row d*8 + dxi*2 + {0: s, 1: t}, rows 6, 7, 14,
// 15, 22..31 zero), layout [dy3][kg][n][8] bf16.
constexpr int kW2Bytes = 9 * 4 * 96 * 16;              // 55296
constexpr int kW3Bytes = 3 * 4 * 32 * 16;              // 6144
// The field x in shared memory, [z][y][x] (rows of 16 floats).  Column x of row y
// is stored at x ^ xswz(y): a warp of conv1 gathers reads four consecutive rows at
// one column parity each, and the swizzle puts those rows in four distinct
// (bank half, parity) classes, so the gathers are free of bank conflicts.
constexpr int kXRow = 16, kXSlice = 16 * kXRow, kXFloats = 16 * kXSlice;
__device__ __forceinline__ int xswz(int y) { return (y >> 1) & 1; }
// conv1 B operands: for each tap set (NEED = 0, 1: the 13 or 14 taps that reach
// fixed sites from a site of one parity, in tap order, padded to K = 16 with
// zeros), W1 as [need][kg][32 rows][8] bf16.
constexpr int kW1Bytes = 2 * 2 * 32 * 16;              // 2048
// FP32 part of a layer block (floats): b1[c], b2[c], b3[2], pad
constexpr int kF_b1 = 0, kF_b2 = kC, kF_b3 = 2 * kC;
constexpr int kF_N = (kF_b3 + 2 + 3) & ~3;
constexpr int kLayerBytes = kW2Bytes + kW3Bytes + kW1Bytes + kF_N * 4;
static_assert(kLayerBytes % 16 == 0, "layer block staged in 16-byte pieces");
// TMEM columns: conv2 accumulators of tile 0 at 0 and tile 1 at 96 (N = 96 each);
// three conv3 batch regions at 192 + 64 r (2 tiles x N = 32); two conv1
// accumulators at 384 + 64 b (2 parity tiles x N = 32)
constexpr int kTmemC3 = 192;
constexpr int kTmemC1 = 384;
// conv1 A operands, double-buffered: [buffer][tile][kg][128 rows][8] bf16
constexpr int kIm2colBufBytes = 2 * 2 * 128 * 16, kIm2colBytes = 2 * kIm2colBufBytes;
constexpr int kTmemCols = 512;
constexpr long long kWaitLimit = 1ll << 22;             // bounded mbarrier wait (iterations)
// Failure-path test of the next launches (gf_set_bf16_stall_test): 0 = off.
std::atomic<long long> g_stall_spins{0};
// Warp w runs on sub-partition w % 4 and may read TMEM lane quarter w % 4.
// One lane each of warps 0, 17, 18 and 19 (sub-partitions 0..3) issues conv2 of
// M-tile 0, conv2 of M-tile 1, the conv3 batches and conv1; warps 1..8 are the
// conv2/conv3 epilogue (e = w - 1); warps 9..16 are the conv1 workers (tile =
// (w - 9) >> 2, TMEM lane quarter w & 3), which build conv1's A operand and
// turn its accumulator into h1.
constexpr int kMmaWarp = 0;                                     // conv2 of M-tile 0; owns TMEM
constexpr int kEpiWarps = 8, kEpiThreads = kEpiWarps * 32;      // warps 1..8
constexpr int kC1Warp0 = 9, kProdThreads = 8 * 32;              // warps 9..16
constexpr int kMma2Warp = 17;                                   // conv2 of M-tile 1
constexpr int kMma3Warp = 18;                                   // conv3 batches
constexpr int kMma1Warp = 19;                                   // conv1
constexpr int kIssuers = 4;

// Instruction descriptors: D = F32, A = B = BF16 (conv2), both K-major, M = 128, N = 96.
constexpr uint32_t kIdesc96 = (1u << 4) | (1u << 7) | (1u << 10) | ((96u >> 3) << 17) | ((128u >> 4) << 24);
// D = F32, A = B = FP16 (conv1 and conv3), K-major, M = 128, N = 32.
constexpr uint32_t kIdesc32h = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

struct Bf16Args {
    const unsigned char* Wl;   // per-layer blocks of kLayerBytes
    int n_layers;
    float slope;
    int use_tanh, has_phi4;
    double m2, lam;
    float c2d_hi, c2d_lo, lam_hi, lam_lo;   // 2d + m2 and lam as FP32 pairs
    int64_t B;
    uint64_t seed, counter0;
    const float* z_in; float* z_out; const float* phi_in; float* phi_out;
    double* logq_out; double* S_out; double* logw_out;
    int32_t* status;
    long long stall_spins;     // > 0: failure-path test (see gf_set_bf16_stall_test)
};

__device__ __forceinline__ int wrap16(int v) { return v & 15; }

// halo-row site index of interior (y, x), y in -1..16
__device__ __forceinline__ int hsite(int y, int x) { return (y + 1) * 16 + x; }

// Stores 8 channels (one channel group) of a site in BF16 (h1, conv2's A
// operand) or FP16 (h2, conv3's A operand), plus the periodic halo copy when
// the row is y = 0 or y = 15.
template <bool F16>
__device__ __forceinline__ void store8(unsigned char* slot, int cg, int y, int x, const float* v) {
    uint4 w;
    if (F16) {
        __align__(16) __half2 p[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) p[i] = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
        w = *reinterpret_cast<const uint4*>(p);
    } else {
        __align__(16) __nv_bfloat162 p[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w = *reinterpret_cast<const uint4*>(p);
    }
    unsigned char* base = slot + (size_t)cg * kCgStride;
    *reinterpret_cast<uint4*>(base + hsite(y, x) * 16) = w;
    if (y == 0) *reinterpret_cast<uint4*>(base + hsite(16, x) * 16) = w;
    if (y == 15) *reinterpret_cast<uint4*>(base + hsite(-1, x) * 16) = w;
}

// Virtual slice v of a layer (may lie outside 0..L-1 by the wrap-around
// recomputation) is lattice slice (v + R) mod L for the layer's rotation R; its
// h1 slot is v mod 4, its h2 slot v mod 3 (the same in every layer, as a layer
// has 20 conv1 and 18 conv2 slices).
__device__ __forceinline__ int h1_slot(int v) { return (v + 16) & 3; }
__device__ __forceinline__ int h2_slot(int v) { return (v + 15) % 3; }

// conv1 tap sets: from an output site of parity p, the taps reaching fixed sites
// are those whose offset parity (|dz|+|dy|+|dx|) mod 2 equals NEED = frozen ^ p.
// tap_of(need, k) = the k-th such tap in tap order, or -1 past the end.
__host__ __device__ constexpr int tap_of(int need, int k) {
    int n = 0;
    for (int t = 0; t < kT; ++t) {
        if (((t / 9 + (t / 3) % 3 + t % 3 + 1) & 1) != need) continue;
        if (n == k) return t;
        ++n;
    }
    return -1;
}

// conv1's bias rides in the last two K columns (A = 1, B = b1 split into an FP16
// head and an FP16 remainder, so the FP32 accumulator adds b1 to about 2^-22);
// every tap set has at most 14 live taps.
constexpr int kBiasK = 14;
static_assert(tap_of(0, kBiasK) < 0 && tap_of(1, kBiasK) < 0, "conv1 bias columns must be padding");

// conv1 A operand row of one site: the masked field at its 13 or 14 live taps
// (FP16), zero-padded, then the two bias columns (1.0), stored as the row's two
// 16-byte core-matrix pieces.  yr[dy] = row offset, ys[dy] = that row's column
// swizzle, xc[dx] = column.
template <int NEED>
__device__ __forceinline__ void im2col_row(unsigned char* a_tile, int r, const float* x, const int (&zr)[3],
                                           const int (&yr)[3], const int (&ys)[3], const int (&xc)[3]) {
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int t = tap_of(NEED, k);
        v[k] = k >= kBiasK ? 1.f
                           : (t < 0 ? 0.f : x[zr[t / 9] + yr[(t / 3) % 3] + (xc[t % 3] ^ ys[(t / 3) % 3])]);
    }
#pragma unroll
    for (int kg = 0; kg < 2; ++kg) {
        __align__(16) __half2 p[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) p[i] = __floats2half2_rn(v[kg * 8 + 2 * i], v[kg * 8 + 2 * i + 1]);
        *reinterpret_cast<uint4*>(a_tile + kg * 2048 + r * 16) = *reinterpret_cast<const uint4*>(p);
    }
}

// One elected thread: conv2 of one M-tile (mt) of a slice as an implicit GEMM:
// 9 (dz,dy) taps x 2 K-steps of tcgen05.mma, each producing the three dx
// partial sums at once (B holds the dx weight sets stacked along N = 96).
// a_slot[dzi] = A descriptors of the three input slices; b0 = B descriptor of
// tap pair 0, K-step 0; tap pair p, K-step k adds p * b_tap + k * b_k (16-byte units).
__device__ __forceinline__ void issue_conv2_tile(const uint64_t (&a_slot)[3], uint64_t b0, uint32_t d, int mt) {
    constexpr uint32_t b_tap = (4 * 96 * 16) >> 4, b_k = (2 * 96 * 16) >> 4;
#pragma unroll
    for (int dzi = 0; dzi < 3; ++dzi) {
#pragma unroll
        for (int dyi = 0; dyi < 3; ++dyi) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const uint64_t ad = desc_add(a_slot[dzi], (uint32_t)((2 * k * kCgStride + (mt * 8 + dyi) * 256) >> 4));
                const uint64_t bd = desc_add(b0, (uint32_t)((dzi * 3 + dyi) * b_tap + k * b_k));
                mma_bf16(d, ad, bd, kIdesc96, (dzi | dyi | k) ? 1u : 0u);
            }
        }
    }
}

// One elected thread: every conv3 contribution of one h2 slice (A descriptor a)
// into a fresh batch region: 2 M-tiles x 3 dy taps x 2 K-steps with N = 32, the
// three dz parts (for the slices after, at and before the h2 slice) and the dx
// weight sets stacked along N.
__device__ __forceinline__ void issue_conv3_batch(uint64_t a, uint64_t b0, uint32_t region) {
    constexpr uint32_t b_tap = (4 * 32 * 16) >> 4, b_k = (2 * 32 * 16) >> 4;
#pragma unroll
    for (int dyi = 0; dyi < 3; ++dyi) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const uint64_t ad = desc_add(a, (uint32_t)((2 * k * kCgStride + (mt * 8 + dyi) * 256) >> 4));
                const uint64_t bd = desc_add(b0, (uint32_t)(dyi * b_tap + k * b_k));
                mma_bf16(region + (uint32_t)mt * 32, ad, bd, kIdesc32h, (dyi | k) ? 1u : 0u);
            }
        }
    }
}

// conv2 epilogue of one M-tile mt, TMEM lane quarter q, channel half hf:
// load the three dx partial sums (16 channels each) of the tile's TMEM buffer,
// then out(x) = sum_dx P_dx(x + dx) + b2, LReLU, BF16 into the h2 slot of v.
struct Conv2Parts { float pm[16], p0[16], pp[16]; };
__device__ __forceinline__ void conv2_epi_load(Conv2Parts& P, uint32_t tile_buf, int q, int hf) {
    const uint32_t base = tile_buf + ((uint32_t)(q * 32) << 16) + (uint32_t)(hf * 16);
    tmem_ld16(base + 0u, P.pm);
    tmem_ld16(base + 32u, P.p0);
    tmem_ld16(base + 64u, P.pp);
    tmem_ld_wait();
}
__device__ __forceinline__ void conv2_epi_store(const Conv2Parts& P, unsigned char* h2, int v, const float (&b2)[16],
                                                float slope, int mt, int q, int hf, int lane) {
    const int y = mt * 8 + q * 2 + (lane >> 4), xx = lane & 15;
    const int src_m = (lane & 16) | ((xx + 15) & 15);   // x - 1
    const int src_p = (lane & 16) | ((xx + 1) & 15);    // x + 1
    unsigned char* slot = h2 + (size_t)h2_slot(v) * kSlotBytes;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        float o[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int ch = g * 8 + c;
            const float s = P.p0[ch] + __shfl_sync(0xffffffffu, P.pm[ch], src_m) +
                            __shfl_sync(0xffffffffu, P.pp[ch], src_p) + b2[ch];
            o[c] = s > 0.f ? s : slope * s;
        }
        store8<true>(slot, hf * 2 + g, y, xx, o);
    }
}

// conv3 epilogue of slice z, tile mt, lane quarter q.  The slice's (s, t)
// partial sums lie in three batch regions: part 0 (dz = -1) in columns 0..5 of
// the batch before it, part 1 in columns 8..13 of its own batch, part 2 in
// columns 16..21 of the batch after it (columns 2*dxi + {0: s, 1: t}).
// load: the three 8-column pieces; finish: (s, t) = sum_dx P_dx(x + dx) + b3 and,
// at the updated sites, the affine map and the log-det.
__device__ __forceinline__ void conv3_epi_load(float (&p)[3][8], uint32_t rm, uint32_t r0, uint32_t rp, int mt,
                                               int q) {
    const uint32_t lane_base = ((uint32_t)(q * 32) << 16) + (uint32_t)(mt * 32);
    tmem_ld8(rm + lane_base + 0u, p[0]);
    tmem_ld8(r0 + lane_base + 8u, p[1]);
    tmem_ld8(rp + lane_base + 16u, p[2]);
    tmem_ld_wait();
}
__device__ __forceinline__ void conv3_epi_finish(const float (&p)[3][8], int z, float b3s, float b3t, float* x,
                                                 int frozen, int use_tanh, bool inverse, FF& logdet, int mt,
                                                 int q, int lane, float& chk) {
    const int y = mt * 8 + q * 2 + (lane >> 4), xx = lane & 15;
    float st[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) st[i] = p[0][i] + p[1][i] + p[2][i];
    const int src_m = (lane & 16) | ((xx + 15) & 15);
    const int src_p = (lane & 16) | ((xx + 1) & 15);
    const float spre = st[2] + __shfl_sync(0xffffffffu, st[0], src_m) + __shfl_sync(0xffffffffu, st[4], src_p) +
                       b3s;
    const float tt = st[3] + __shfl_sync(0xffffffffu, st[1], src_m) + __shfl_sync(0xffffffffu, st[5], src_p) + b3t;
    if (((z + y + xx) & 1) != frozen) {
        // FP16 operands of conv1 / conv3 overflow beyond 65504: a non-finite s
        // or t (from a field or h2 value out of that range) turns chk into NaN
        // (0 * inf and 0 * NaN are NaN); it is reported once per configuration
        chk = fmaf(spre, 0.f, fmaf(tt, 0.f, chk));
        const float s = use_tanh ? tanhf(spre) : spre;
        float& xv = x[(z * 16 + y) * kXRow + (xx ^ xswz(y))];
        if (!inverse) xv = fmaf(xv, expf(s), tt);
        else xv = (xv - tt) * expf(-s);
        ff_add(logdet, s);
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
        ++spins;
        if ((spins & 63) == 0 && *abort_flag) return false;      // another thread gave up
        if (spins > kWaitLimit) { *abort_flag = 1; set_status(status, GF_ETIMEOUT); return false; }
    }
    return true;
}
// Bounded wait that ignores the abort flag (teardown: work already issued must
// finish before its shared memory or TMEM is released).
__device__ __forceinline__ void drain_wait(uint64_t* bar, int n) {
    for (long long spins = 0; !mbar_try_wait(bar, (uint32_t)n & 1u) && spins < kWaitLimit; ++spins) {}
}

// Per layer and CTA: 20 conv1 slices (virtual v = -2..17), 18 conv2 slices
// (u = -1..16), 18 conv3 batches and 16 conv3 slices (w = 0..15).  Batch u is
// queued once h2[u] exists and computes every conv3 contribution of h2[u] (to
// slices u+1, u and u-1, stacked along N) into its own TMEM region, so slice w
// is complete after batch w+1; a region is released once the last existing
// slice that reads it has been drained.  With seq = the CTA's running layer
// count, the global numbers c = 20 seq + v + 2 and g2 = gb = 18 seq + u + 1
// index the barrier completions:
//   h1 slot: bar_h1[c % 4], completion c / 4;
//   conv2 of tile t: bar_m2[2 t + (g2 & 1)] completion g2 >> 1; its TMEM drained:
//   bar_t2[t] completion g2; h2 written: bar_h2[g2 % 3], completion g2 / 3;
//   conv3 batch gb: bar_m3[gb & 1], completion gb >> 1; its region gb % 3
//   released: bar_t3[gb % 3], completion gb / 3;
//   once per layer (completion seq): W2 and biases staged bar_w2, W3 staged
//   bar_w3, field slices <= 5 / 9 / 13 / 15 updated bar_x[0..3].
constexpr int kConv1PerLayer = 20, kConv2PerLayer = 18;

// Warp roles: four issuing threads (warps 0, 17, 18, 19); warps 1..8 run the
// conv2 and conv3 epilogues (e = w - 1: M-tile or channel half e >> 2, TMEM lane
// quarter w & 3); warps 9..16 build conv1's operands and turn its accumulators
// into the h1 slots.  They synchronise through mbarriers only, so the tensor
// cores and the epilogues overlap; the CTA meets at a barrier only between
// configurations.
template <bool INVERSE>
__global__ void __launch_bounds__(kThreads, 1) flow_bf16_kernel(const Bf16Args a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* w2s = smem;                                                 // kW2Bytes
    unsigned char* w3s = smem + kW2Bytes;                                      // kW3Bytes
    unsigned char* w1s = smem + kW2Bytes + kW3Bytes;                           // kW1Bytes
    float* wf = reinterpret_cast<float*>(smem + kW2Bytes + kW3Bytes + kW1Bytes);  // kF_N floats
    unsigned char* h1 = smem + kLayerBytes;                                    // 4 slots
    unsigned char* h2 = h1 + 4 * kSlotBytes;                                   // 3 slots
    float* x = reinterpret_cast<float*>(h2 + 3 * kSlotBytes);                  // kXFloats (padded rows)
    unsigned char* im2col = reinterpret_cast<unsigned char*>(x + kXFloats);  // kIm2colBytes
    double* red = reinterpret_cast<double*>(im2col + kIm2colBytes);            // 32
    uint64_t* bar_h1 = reinterpret_cast<uint64_t*>(red + 32);  // 4: h1 slot written (producers)
    uint64_t* bar_h2 = bar_h1 + 4;                             // 3: h2 slot written (epilogue)
    uint64_t* bar_m2 = bar_h2 + 3;                             // 4: conv2 of a tile done (commit)
    uint64_t* bar_m3 = bar_m2 + 4;                             // 2: conv3 batch done (commit)
    uint64_t* bar_t2 = bar_m3 + 2;                             // 2: conv2 tile buffer drained
    uint64_t* bar_t3 = bar_t2 + 2;                             // 3: conv3 batch region released
    uint64_t* bar_b1 = bar_t3 + 3;                             // 2: conv1 A operand built (workers)
    uint64_t* bar_c1 = bar_b1 + 2;                             // 2: conv1 MMAs done (commit)
    uint64_t* bar_fin = bar_c1 + 2;                            // 1: every queued MMA done (exit)
    uint64_t* bar_w2 = bar_fin + 1;                            // 1: a layer's W2 and biases staged
    uint64_t* bar_w3 = bar_w2 + 1;                             // 1: a layer's W3 staged
    uint64_t* bar_x = bar_w3 + 1;                              // 4: a layer's field slices <= 5, 9, 13, 15 updated
    uint64_t* bar_stall = bar_x + 4;                           // 1: never completed (failure-path test)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_stall + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int V = 4096;
    if (warp == kMmaWarp) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(bar_h1 + i, kProdThreads);
        for (int i = 0; i < 3; ++i) mbar_init(bar_h2 + i, kEpiThreads);
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar_m3 + i, 1);
            mbar_init(bar_t2 + i, kEpiThreads);
        }
        for (int i = 0; i < 4; ++i) mbar_init(bar_m2 + i, 1);
        for (int i = 0; i < 3; ++i) mbar_init(bar_t3 + i, kEpiThreads);
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar_b1 + i, kProdThreads);
            mbar_init(bar_c1 + i, 1);
        }
        mbar_init(bar_fin, kIssuers);                          // one commit per issuing thread
        mbar_init(bar_w2, 1);                                  // expect_tx by the staging thread
        mbar_init(bar_w3, 1);
        for (int i = 0; i < 4; ++i) mbar_init(bar_x + i, kEpiThreads);
        mbar_init(bar_stall, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const auto t2tile = [tmem](int t) { return tmem + (uint32_t)(t * 96); };
    const auto t3reg = [tmem](int r) { return tmem + (uint32_t)(kTmemC3 + (r % 3) * 64); };
    const auto xi = [](int n) { return (n >> 4) * kXRow + ((n & 15) ^ xswz(n >> 4)); };   // site -> x index

    // A descriptors of every h1 / h2 slot (LBO = channel-group stride, SBO = 8 sites);
    // B: conv2 LBO = 96 rows x 16 B between K groups, conv3 LBO = 32 rows x 16 B, SBO = 128.
    const uint64_t a1_0 = smem_desc(smem_u32(h1), kCgStride, 128);
    const uint64_t a2_0 = smem_desc(smem_u32(h2), kCgStride, 128);
    const auto a1 = [a1_0](int slot) { return desc_add(a1_0, (uint32_t)(slot * (kSlotBytes >> 4))); };
    const auto a2 = [a2_0](int slot) { return desc_add(a2_0, (uint32_t)(slot * (kSlotBytes >> 4))); };
    const uint64_t b2d = smem_desc(smem_u32(w2s), 96 * 16, 128);
    const uint64_t b3d = smem_desc(smem_u32(w3s), 32 * 16, 128);
    const uint64_t b1d = smem_desc(smem_u32(w1s), 32 * 16, 128);               // + need * 64
    const uint64_t a1c = smem_desc(smem_u32(im2col), 128 * 16, 128);           // + (buffer, tile)

    int seq = 0;                                   // layers processed by this CTA so far
    int last_w2 = -1, last_w3 = -1;                // staging thread: completions its last copies bring
    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        FF sumz2{0.f, 0.f};                        // sum z^2: each square exactly as a pair
        if (!INVERSE) {
            if (a.z_in) {
                for (int n = tid; n < V; n += kThreads) {
                    const float v = __ldg(a.z_in + b * V + n);
                    x[xi(n)] = v;
                    const float p = v * v;
                    ff_add(sumz2, FF{p, fmaf(v, v, -p)});
                }
            } else {
                for (int j = tid; 4 * j < V; j += kThreads) {
                    const u64x4 w = philox4x64_10(a.seed, 0ull,
                                                  u64x4{a.counter0 + (uint64_t)b, (uint64_t)j, 0ull, TAG_PRIOR});
                    float zz[4];
                    normals4_f32(w, zz);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        x[xi(4 * j + q)] = zz[q];
                        const float p = zz[q] * zz[q];
                        ff_add(sumz2, FF{p, fmaf(zz[q], zz[q], -p)});
                    }
                }
            }
            __syncthreads();
            if (a.z_out)
                for (int n = tid; n < V; n += kThreads) a.z_out[b * V + n] = x[xi(n)];
        } else {
            for (int n = tid; n < V; n += kThreads) x[xi(n)] = __ldg(a.phi_in + b * V + n);
        }
        __syncthreads();

        FF logdet{0.f, 0.f};                       // this thread's sum of s over its updated sites
        float chk = 0.f;                           // NaN once a non-finite s or t was seen
        const int seq0 = seq, nl = a.n_layers;
        // Layers are pipelined into one another (no CTA barrier between them): layer li
        // (global number s = seq0 + li) walks the lattice slices in the order R + v with
        // R = 4 li (mod 16), so the first slices of layer li need only field slices that
        // layer li-1 finished early, and its conv1 overlaps layer li-1's last conv2 and
        // conv3 work.  The conv1 workers stage each layer's weights: the conv1 B operand
        // after their last drain of layer li-1, W2 and the FP32 biases once layer li-1's
        // last conv2 is done (bar_w2), W3 once its last conv3 batch is done (bar_w3).
        const auto lay = [&](int li) { return INVERSE ? nl - 1 - li : li; };
        const auto rot = [](int li) { return (4 * li) & 15; };
        if (warp == kMmaWarp || warp == kMma2Warp) {
            // ---------------- conv2 of M-tile t (one thread): slice u needs h1 of u-1..u+1
            // and the tile's TMEM buffer drained by the epilogue of u-1
            if (lane == 0) {
                const int t = warp == kMma2Warp;
                bool ok = true;
                if (a.stall_spins > 0 && seq0 == 0 && t == 0) {
                    // failure-path test: a wait for a completion that never comes runs
                    // out long after every MMA issued so far has finished
                    for (long long spins = 0; !mbar_try_wait(bar_stall, 0u); ++spins)
                        if (spins > a.stall_spins) {
                            *abort_flag = 1;
                            set_status(a.status, GF_ETIMEOUT);
                            ok = false;
                            break;
                        }
                }
                for (int li = 0; li < nl && ok; ++li) {
                    const int s = seq0 + li, c0 = s * kConv1PerLayer, g20 = s * kConv2PerLayer;
                    ok = wait_n(bar_w2, s, abort_flag, a.status);          // this layer's W2 staged
                    for (int u = -1; u <= kL && ok; ++u) {
                        for (int v = (u == -1 ? -2 : u + 1); v <= u + 1 && ok; ++v) {
                            const int c = c0 + v + 2;
                            ok = wait_n(bar_h1 + (c & 3), c >> 2, abort_flag, a.status);
                        }
                        const int g2 = g20 + u + 1;
                        if (!ok || (g2 >= 1 && !(ok = wait_n(bar_t2 + t, g2 - 1, abort_flag, a.status)))) break;
                        fence_after_sync();
                        const uint64_t as[3] = {a1(h1_slot(u - 1)), a1(h1_slot(u)), a1(h1_slot(u + 1))};
                        issue_conv2_tile(as, b2d, t2tile(t), t);
                        mma_commit(bar_m2 + 2 * t + (g2 & 1));
                    }
                }
            }
            __syncwarp();
        } else if (warp == kMma3Warp) {
            // ---------------- conv3 batch ub (one thread): every contribution of h2[ub]; needs
            // h2[ub] written and its batch region free (batch ub-3's readers drained)
            if (lane == 0) {
                bool ok = true;
                for (int li = 0; li < nl && ok; ++li) {
                    const int s = seq0 + li, g20 = s * kConv2PerLayer;
                    ok = wait_n(bar_w3, s, abort_flag, a.status);          // this layer's W3 staged
                    for (int ub = -1; ub <= kL && ok; ++ub) {
                        const int gh = g20 + ub + 1;
                        ok = wait_n(bar_h2 + gh % 3, gh / 3, abort_flag, a.status) &&
                             (gh < 3 || wait_n(bar_t3 + gh % 3, (gh - 3) / 3, abort_flag, a.status));
                        if (!ok) break;
                        fence_after_sync();
                        issue_conv3_batch(a2(h2_slot(ub)), b3d, t3reg(gh));
                        mma_commit(bar_m3 + (gh & 1));
                    }
                }
            }
            __syncwarp();
        } else if (warp == kMma1Warp) {
            // ---------------- conv1 of virtual slice v (one thread): one MMA (K = 16) per
            // parity tile, B = the tile's tap set, into buffer b = c & 1 of the A operand
            // and of the accumulator, once the workers have built the A operand (they
            // build slice v only after draining conv1 of slice v-2)
            if (lane == 0) {
                bool ok = true;
                for (int li = 0; li < nl && ok; ++li) {
                    const int s = seq0 + li, c0 = s * kConv1PerLayer, frozen = lay(li) & 1;
                    for (int v = -2; v <= kL + 1; ++v) {
                        const int c = c0 + v + 2, b = c & 1;
                        if (!(ok = wait_n(bar_b1 + b, c >> 1, abort_flag, a.status))) break;
                        fence_after_sync();
#pragma unroll
                        for (int pc = 0; pc < 2; ++pc)
                            mma_bf16(tmem + (uint32_t)(kTmemC1 + 64 * b + 32 * pc),
                                     desc_add(a1c, (uint32_t)((b * kIm2colBufBytes + pc * 4096) >> 4)),
                                     desc_add(b1d, (uint32_t)(((frozen ^ pc) & 1) * 64)), kIdesc32h, 0u);
                        mma_commit(bar_c1 + b);
                    }
                }
            }
            __syncwarp();
        } else if (warp >= kC1Warp0 && warp < kC1Warp0 + 8) {
            // ---------------- conv1 workers: thread = row r of parity tile pc.  Two A
            // operand buffers and two accumulators (b = c & 1): the A operand of slice
            // v+2 is built as soon as conv1 of slice v has been drained.  Row r holds
            // site (y, 2 xh + parity) with lanes 0-3 / 4-7 on rows 2j / 2j+1 (opposite
            // parities), so each 8-lane phase of the 16-byte h1 stores covers 8
            // distinct bank groups.
            const int wt = tid - kC1Warp0 * 32;                   // 0..255
            const int pc = (warp - kC1Warp0) >> 2, r = ((warp & 3) << 5) | lane;
            const int y = ((r >> 4) << 1) | ((r >> 2) & 1), xh = (((r >> 3) & 1) << 2) | (r & 3);
            const uint32_t t1lane = (uint32_t)((warp & 3) * 32) << 16;
            // layer l's block: W2 with the FP32 biases and W3 arrive by bulk copies issued by
            // one thread (completion on bar_w2 / bar_w3 by byte count); the conv1 B operand
            // (2 KB) by one 16-byte copy per thread of the first 128
            const auto stage_w2 = [&](int l) {
                const unsigned char* blk = a.Wl + (size_t)l * kLayerBytes;
                ++last_w2;                                // bar_w2 completes once per staged layer
                mbar_expect_tx(bar_w2, (uint32_t)(kW2Bytes + kF_N * 4));
                bulk_g2s(w2s, blk, (uint32_t)kW2Bytes, bar_w2);
                bulk_g2s(wf, blk + kW2Bytes + kW3Bytes + kW1Bytes, (uint32_t)(kF_N * 4), bar_w2);
            };
            const auto stage_w3 = [&](int l) {
                ++last_w3;
                mbar_expect_tx(bar_w3, (uint32_t)kW3Bytes);
                bulk_g2s(w3s, a.Wl + (size_t)l * kLayerBytes + kW2Bytes, (uint32_t)kW3Bytes, bar_w3);
            };
            const auto stage_w1 = [&](int l) {
                if (wt < kW1Bytes / 16)
                    reinterpret_cast<uint4*>(w1s)[wt] =
                        __ldg(reinterpret_cast<const uint4*>(a.Wl + (size_t)l * kLayerBytes + kW2Bytes + kW3Bytes) + wt);
            };
            int xseen = 0, kx = 0;                                 // slices of layer li-1 known updated
            bool ok = true;
            for (int li = 0; li < nl && ok; ++li) {
                const int s = seq0 + li, c0 = s * kConv1PerLayer, g20 = s * kConv2PerLayer, l = lay(li);
                const int need = ((l & 1) ^ pc) & 1, R = rot(li);
                if (li == 0 && wt == 0) {                          // the first layer's W2 and W3
                    stage_w2(l);
                    stage_w3(l);
                }
                stage_w1(l);                                       // (conv1 of layer li-1 drained)
                xseen = li == 0 ? kL : 0;
                kx = 0;
                auto build = [&](int v) {                          // A operand of slice v, then signal it
                    const int c = c0 + v + 2;
                    // slices R+v-1 .. R+v+1 were slices v+3 .. v+5 (mod 16) of layer li-1
                    // (v >= 10 reaches its last two): wait until its epilogue has updated them,
                    // at four checkpoints per layer (slices 5, 9, 13, 15; the last one, which
                    // comes after layer li's first conv2, is first needed at v = 9)
                    while (xseen <= (v + 5 < kL - 1 ? v + 5 : kL - 1) && ok) {
                        ok = wait_n(bar_x + kx, s - 1, abort_flag, a.status);
                        xseen = (kx == 3 ? kL - 1 : 5 + 4 * kx) + 1;
                        ++kx;
                    }
                    const int z = (v + R) & 15;
                    const int xs = 2 * xh + ((pc ^ z ^ y) & 1);
                    int zr[3], yr[3], ys[3], xc[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        zr[d] = wrap16(z + d - 1) * kXSlice;
                        yr[d] = wrap16(y + d - 1) * kXRow;
                        ys[d] = xswz(wrap16(y + d - 1));
                        xc[d] = wrap16(xs + d - 1);
                    }
                    unsigned char* a_tile = im2col + (c & 1) * kIm2colBufBytes + pc * 4096;
                    if (need) im2col_row<1>(a_tile, r, x, zr, yr, ys, xc);
                    else im2col_row<0>(a_tile, r, x, zr, yr, ys, xc);
                    fence_proxy_async();
                    mbar_arrive(bar_b1 + (c & 1));
                };
                build(-2);
                build(-1);
                for (int v = -2; v <= kL + 1 && ok; ++v) {
                    const int c = c0 + v + 2;
                    if (!(ok = wait_n(bar_c1 + (c & 1), c >> 1, abort_flag, a.status))) break;
                    fence_after_sync();
                    float d[32];
                    const uint32_t acc = tmem + (uint32_t)(kTmemC1 + 64 * (c & 1) + 32 * pc) + t1lane;
                    tmem_ld16(acc, *reinterpret_cast<float(*)[16]>(d));
                    tmem_ld16(acc + 16u, *reinterpret_cast<float(*)[16]>(d + 16));
                    tmem_ld_wait();
                    fence_before_sync();
                    // its arrival also says this accumulator (and A buffer) may be reused
                    if (v + 2 <= kL + 1) build(v + 2);
                    if (!ok) break;
                    // the h1 slot of v last held h1 of v-4 (or of slice v+16 of the previous
                    // layer): wait until the last conv2 that read it is done (both tiles)
                    const int g2 = v >= 2 ? g20 + v - 2 : (li > 0 ? g20 - kConv2PerLayer + (v + 17 < 16 ? v + 17 : 16) + 1 : -1);
                    if (g2 >= 0 && !(ok = wait_n(bar_m2 + (g2 & 1), g2 >> 1, abort_flag, a.status) &&
                                          wait_n(bar_m2 + 2 + (g2 & 1), g2 >> 1, abort_flag, a.status)))
                        break;
                    const int z = (v + R) & 15;
                    const int xs = 2 * xh + ((pc ^ z ^ y) & 1);
                    unsigned char* slot = h1 + (size_t)h1_slot(v) * kSlotBytes;
#pragma unroll
                    for (int cg = 0; cg < 4; ++cg) {
                        float o[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float hv = d[cg * 8 + i];             // b1 is in the MMA
                            o[i] = hv > 0.f ? hv : a.slope * hv;
                        }
                        store8<false>(slot, cg, y, xs, o);
                    }
                    fence_proxy_async();
                    mbar_arrive(bar_h1 + (c & 3));
                    if (li > 0 && v == -1 && wt == 0) {
                        stage_w2(l);                     // layer li-1's last conv2 is done (waited above)
                    } else if (li > 0 && v == 2 && wt == 0) {
                        const int gb = g20 - 1;          // layer li-1's last conv3 batch
                        if (!(ok = wait_n(bar_m3 + (gb & 1), gb >> 1, abort_flag, a.status))) break;
                        stage_w3(l);
                    }
                }
            }
        } else if (warp >= 1 && warp <= kEpiWarps) {
            // ---------------- epilogues.  conv2: lane quarter q, channel half hf of each
            // tile in turn; conv3: tile mt, lane quarter q.  Iteration u of layer li first
            // finishes the conv3 slice two batches behind (u-3 of layer li, or the last two
            // slices of layer li-1 at u = -1, 0), then turns conv2 of slice u into h2.
            // After the last layer, two more iterations finish its last two slices.
            const int e = warp - 1;                  // 0..7: quarters 1, 2, 3, 0, 1, 2, 3, 0
            const int q = warp & 3, hf = e >> 2, mt = e >> 2;
            float b2[16];                            // this thread's conv2 biases, conv3 biases
            float b3s = 0.f, b3t = 0.f, b3s_p = 0.f, b3t_p = 0.f;   // of layer li and of li-1
            bool ok = true;
            for (int li = 0; li <= nl && ok; ++li) {
                const int s = seq0 + li, g20 = s * kConv2PerLayer;
                for (int u = -1; u <= (li < nl ? kL : 0) && ok; ++u) {
                    const int g2 = g20 + u + 1;
                    // batch g2-2 done: the conv3 slice below is complete and the h2 slot of u
                    // (last read by batch g2-3) is free
                    const bool tail = u <= 0 && li > 0, own = u >= 3;
                    if (li > 0 || u >= 1) {
                        const int gb = g2 - 2;
                        if (!(ok = wait_n(bar_m3 + (gb & 1), gb >> 1, abort_flag, a.status))) break;
                        fence_after_sync();
                    }
                    if (tail || own) {
                        // slice w of layer lj (global conv3 numbers gw = g20 of lj + w + 1)
                        const int lj = tail ? li - 1 : li, w = tail ? kL - 1 + u : u - 3;
                        const int gj = (seq0 + lj) * kConv2PerLayer + w + 1;
                        float p[3][8];
                        conv3_epi_load(p, t3reg(gj - 1), t3reg(gj), t3reg(gj + 1), mt, q);
                        fence_before_sync();
                        mbar_arrive(bar_t3 + (gj - 1) % 3);   // slice w is the last reader of batch w-1
                        if (w == kL - 1) { mbar_arrive(bar_t3 + gj % 3); mbar_arrive(bar_t3 + (gj + 1) % 3); }
                        // layer li's biases replace li-1's at u = -1, after its slice 14
                        const bool prev = u == 0 && li < nl;
                        conv3_epi_finish(p, (w + rot(lj)) & 15, prev ? b3s_p : b3s, prev ? b3t_p : b3t, x,
                                         lay(lj) & 1, a.use_tanh, INVERSE, logdet, mt, q, lane, chk);
                        if (w == kL - 1 || (w >= 5 && (w & 3) == 1))   // checkpoint: slices <= w updated
                            mbar_arrive(bar_x + (w == kL - 1 ? 3 : (w - 5) >> 2));
                    }
                    if (li == nl) continue;
                    if (u == -1) {                                 // this layer's biases (W2 staged)
                        if (!(ok = wait_n(bar_w2, s, abort_flag, a.status))) break;
                        b3s_p = b3s; b3t_p = b3t;
#pragma unroll
                        for (int c = 0; c < 16; ++c) b2[c] = wf[kF_b2 + hf * 16 + c];
                        b3s = wf[kF_b3]; b3t = wf[kF_b3 + 1];
                    }
                    for (int t = 0; t < 2; ++t) {
                        if (!(ok = wait_n(bar_m2 + 2 * t + (g2 & 1), g2 >> 1, abort_flag, a.status))) break;
                        fence_after_sync();
                        Conv2Parts P;
                        conv2_epi_load(P, t2tile(t), q, hf);
                        fence_before_sync();
                        mbar_arrive(bar_t2 + t);         // the tile's TMEM buffer may be refilled
                        conv2_epi_store(P, h2, u, b2, a.slope, t, q, hf, lane);
                    }
                    if (!ok) break;
                    fence_proxy_async();
                    mbar_arrive(bar_h2 + g2 % 3);
                }
            }
        }
        seq = seq0 + nl;
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (*abort_flag) break;

        if (INVERSE) {
            for (int n = tid; n < V; n += kThreads) {
                const float v = x[xi(n)];
                const float p = v * v;
                ff_add(sumz2, FF{p, fmaf(v, v, -p)});
                if (a.z_out) a.z_out[b * V + n] = v;
            }
        } else {
            for (int n = tid; n < V; n += kThreads) a.phi_out[b * V + n] = x[xi(n)];
        }
        FF* red_ff = reinterpret_cast<FF*>(red);
        if (chk != chk) set_status(a.status, GF_EDEVICE);
        const double ld = block_sum_ff(logdet, red_ff);
        const double z2 = block_sum_ff(sumz2, red_ff);
        double S = 0.0;
        if (!INVERSE && a.has_phi4) {
            // forward-hop arrangement of the action, per site
            // phi^2 (c2d + lam phi^2) - 2 phi sum_mu phi(n + mu), c2d = 2d + m2, in FP32 pairs
            // (phi^2 exact, products and sums to about 2^-48), widened to FP64 per thread
            const FF c2d{a.c2d_hi, a.c2d_lo}, lam{a.lam_hi, a.lam_lo};
            FF acc{0.f, 0.f};
            for (int n = tid; n < V; n += kThreads) {
                const int xc = n & 15, yc = (n >> 4) & 15, zc = n >> 8;
                FF hop{x[xi((n & ~15) | wrap16(xc + 1))], 0.f};
                ff_add(hop, x[xi((zc << 8) | (wrap16(yc + 1) << 4) | xc)]);
                ff_add(hop, x[xi((wrap16(zc + 1) << 8) | (yc << 4) | xc)]);
                const float c = x[xi(n)], cp = c * c;
                const FF qq{cp, fmaf(c, c, -cp)};
                FF inner = ff_mul(lam, qq);
                ff_add(inner, c2d);
                const FF pot = ff_mul(qq, inner);
                const FF kin = ff_mul(FF{-2.f * c, 0.f}, hop);
                ff_add(acc, pot);
                ff_add(acc, kin);
            }
            S = block_sum_ff(acc, red_ff);
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
    // after an abort some MMAs may still be queued and a weight copy may still be
    // writing shared memory: every issuing thread commits, and TMEM is freed only
    // once all their tensor-core work is done; the staging thread waits for the
    // completions its last W2 / W3 copies bring (bounded waits, abort flag ignored)
    if ((warp == kMma2Warp || warp == kMma3Warp || warp == kMma1Warp) && lane == 0) mma_commit(bar_fin);
    if (warp == kMmaWarp && lane == 0) {
        mma_commit(bar_fin);
        drain_wait(bar_fin, 0);
    }
    if (warp == kC1Warp0 && lane == 0) {           // the staging thread (worker wt == 0)
        if (last_w2 >= 0) drain_wait(bar_w2, last_w2);
        if (last_w3 >= 0) drain_wait(bar_w3, last_w3);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == kMmaWarp) {
        fence_after_sync();
        tmem_dealloc(tmem, kTmemCols);
    }
}

constexpr size_t kSmemBytes = (size_t)kLayerBytes + 7 * (size_t)kSlotBytes + (size_t)kXFloats * 4 + kIm2colBytes +
                              32 * 8 + 32 * 8 + 4 + 4;
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");

// canonical FP32 -> per-layer block: W2 [tap9][kg][dxi*32 + o][8] bf16,
// W3 [dy3][kg][d*8 + dxi*2 + j][8] fp16 (tap (d, dy, dxi); j = 0: s, 1: t; rows
// with (row & 7) >= 6 or row >= 24 zero),
// then W1 as the two conv1 B operands [need][kg][o][8] fp16 (tap_of order; K
// columns 14 and 15 hold b1's FP16 head and remainder), then FP32 b1, b2, b3.
__global__ void repack_bf16_kernel(const float* __restrict__ canon, int64_t cstride, int n_layers,
                                   unsigned char* __restrict__ out) {
    constexpr int n2 = 9 * 4 * 96 * 8, n3 = 3 * 4 * 32 * 8, n1 = 2 * 2 * 32 * 8;
    const int64_t per = n2 + n3 + n1 + kF_N;
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
            const int e = r3 & 7, row = (r3 >> 3) & 31, kg = (r3 >> 8) & 3, dyi = r3 >> 10;
            const int d = row >> 3, rr = row & 7, dxi = rr >> 1, j = rr & 1;
            const bool live = d < 3 && rr < 6;
            const int t = live ? d * 9 + dyi * 3 + dxi : 0;
            const float v = live ? W3[((int64_t)j * kC + kg * 8 + e) * kT + t] : 0.f;
            reinterpret_cast<__half*>(blk + kW2Bytes)[r3] = __float2half_rn(v);
        } else if (r < n2 + n3 + n1) {
            const int r1 = (int)(r - n2 - n3);
            const int e = r1 & 7, o = (r1 >> 3) & 31, kg = (r1 >> 8) & 1, need = r1 >> 9;
            const int k = kg * 8 + e, t = tap_of(need, k);
            const float bh = __half2float(__float2half_rn(b1[o]));
            const float v = k == kBiasK ? b1[o] : k == kBiasK + 1 ? b1[o] - bh : t < 0 ? 0.f : W1[(int64_t)o * kT + t];
            reinterpret_cast<__half*>(blk + kW2Bytes + kW3Bytes)[r1] = __float2half_rn(v);
        } else {
            const int f = (int)(r - n2 - n3 - n1);
            float v = 0.f;
            if (f < kF_b2) v = b1[f - kF_b1];
            else if (f < kF_b3) v = b2[f - kF_b2];
            else if (f < kF_b3 + 2) v = b3[f - kF_b3];
            reinterpret_cast<float*>(blk + kW2Bytes + kW3Bytes + kW1Bytes)[f] = v;
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
    const int64_t total = (int64_t)(9 * 4 * 96 * 8 + 3 * 4 * 32 * 8 + 2 * 2 * 32 * 8 + kF_N) * f->shape.n_layers;
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
    ff_split(6.0 + a.m2, &a.c2d_hi, &a.c2d_lo);
    ff_split(a.lam, &a.lam_hi, &a.lam_lo);
    a.B = B; a.seed = seed; a.counter0 = counter0;
    a.z_in = z_in; a.z_out = z_out; a.phi_in = phi_in; a.phi_out = phi_out;
    a.logq_out = logq_out; a.S_out = S_out; a.logw_out = logw_out;
    a.status = status_word(stream);
    a.stall_spins = g_stall_spins.load(std::memory_order_relaxed);
    if (!a.status) return GF_ECUDA;
    auto kern = inverse ? flow_bf16_kernel<true> : flow_bf16_kernel<false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess)
        return GF_ECUDA;
    const int64_t grid = std::min<int64_t>(B, (int64_t)num_sms());
    kern<<<(unsigned)grid, kThreads, kSmemBytes, stream>>>(a);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

long long bf16_stall_spins() { return g_stall_spins.load(std::memory_order_relaxed); }

}  // namespace gf

extern "C" gf_status gf_set_bf16_stall_test(int64_t spins) {
    if (spins < 0 || spins > gf::kWaitLimit / 2) return GF_EINVAL;
    gf::g_stall_spins.store((long long)spins, std::memory_order_relaxed);
    return GF_OK;
}
