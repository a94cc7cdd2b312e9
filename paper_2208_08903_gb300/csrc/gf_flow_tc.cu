// gf_flow_tc.cu -- fused coupling stack with conv2 and the conv3 head on the
// tensor cores (tcgen05, 16-bit operands, FP32 accumulation in TMEM) for the
// lattice shapes other than 3D L=16 with hidden width 32 (which has its own
// kernel): 2D and 3D, even L, two equal hidden widths of 8, 16, 24 or 32
// channels (24 padded to 32 with zero weights), kernel size 3, while the
// lattice's activations fit in shared memory.
//
// Paper arXiv:2208.08903 Sec. 1 (checkerboard affine coupling layers, their
// Jacobian, the model density and the action).  Precision: conv2, the dense
// contraction (C x C x 3^d per site), reads BF16 h1 and W2; the conv3 head
// reads FP16 h2 and W3 (FP16 keeps three more mantissa bits of the small head
// weights, whose BF16 rounding moved log w the most in the 3D kernel's
// experiments); both accumulate in FP32.  conv1 (one input channel, about half
// of its taps live) runs on the FP32 pipe from the FP32 field and weights; the
// affine update is FP32; log-det and z^2 are summed per thread in FP32 pairs
// (about 2^-48 relative) and across the block in FP64, as are log q, the
// action and log w.  |h2| must stay below 65504: a non-finite s or t records
// GF_EDEVICE.
//
// Persistent grid of one CTA per SM (the runtime places one CTA of a tcgen05
// kernel on an SM); a CTA runs one configuration at a time, or, where two
// copies of the shared-memory plan fit (2D lattices up to L = 32, small 3D
// lattices), two, one per half of its warps, each half with its own shared
// memory, TMEM columns and barriers (see flow_tc_kernel).  The activations
// live in a zero-padded copy of the lattice, one halo layer per axis holding
// the periodic images: P = L + 2 positions per axis, x fastest, stored
// channel-group major [Cp/8][position][8 channels] so that 8 consecutive
// positions of one channel group are one 128-byte core matrix of the
// K-major canonical layout.  A convolution is then an implicit GEMM whose A
// operand for taps (dz,dy,*) is the same array started (dy-1) P + (dz-1) P^2
// positions later, K = the 3^(d-1) (dz,dy) pairs x Cp channels in steps of
// 16 (width 8: two (dz,dy) pairs per step), and whose three x-taps are
// stacked along N (conv2: N = 3 Cp, 32 for width 8; head: N = 16, columns
// 2 dx + (s, t)): each row's column block dx is the partial
// sum of tap dx at the row's own position, and the epilogue adds block 0 of
// the row to the left, block 1 and block 2 of the row to the right.  The 128
// rows of a tile are 16 core matrices of 8 consecutive positions, each 6
// positions after the previous one, so rows 1..6 of every 8 are outputs (96
// per tile, positions on the halo dropped) whose x-neighbours are in the same
// 8 TMEM lanes (width-8 shuffles).  Per layer, with a barrier of the
// configuration's warps between the phases:
//   conv1 (all warps): h1 = LReLU(W1 * masked x + b1) at every site, BF16, at
//     its padded position and at its periodic images;
//   conv2 (two issuing threads on different sub-partitions, alternate tiles):
//     two groups of four epilogue warps (one warp per TMEM lane quarter) take
//     the same alternate tiles, each through its own ring of TMEM
//     accumulators, and turn them into
//     h2 = LReLU(acc + b2) in FP16, released from TMEM at once and written
//     over h1 in place once every tile that reads those positions (up to
//     ceil(p0 / 96) tiles on, p0 = 1 + P (+ P^2) the largest tap offset) has
//     completed;
//   halo (all warps): the periodic images of h2;
//   conv3 (the issuing threads, the epilogue groups): (s, t) for every tile;
//     at the updated sites s = tanh(s + b_s), x <- x e^s + t (or the
//     inverse), log-det += s.
// Each layer's weights arrive by bulk copies (cp.async.bulk): W2 for the next
// layer once this layer's conv2 has completed, W3 once its conv3 has, the
// FP32 part (W1, b1, b2, b3) one layer ahead into a second buffer.  Every wait
// on an mbarrier is bounded: a wait that runs out records GF_ETIMEOUT, raises
// the CTA's abort flag, and the CTA leaves after draining its queued MMAs and
// copies.
#include <algorithm>
#include <cstring>
#include <mutex>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gf_async.cuh"
#include "gf_flow.cuh"
#include "gf_tcgen05.cuh"

namespace gf {

namespace {

constexpr int kTcThreads = 384;           // warps 0, 1: MMA issue (warp 0 owns TMEM); warps 4..11: two epilogue groups
constexpr int kTcM = 128;                 // rows per tile (TMEM lanes)
constexpr int kTcOut = 96;                // output positions per tile (6 of every 8 rows)
constexpr int kTcRing = 8;                // TMEM accumulators per epilogue group (at most)
constexpr int kTcMaxTiles = 64;           // tiles per layer (one completion barrier each)
constexpr long long kTcWaitLimit = 1ll << 22;
constexpr int kSmemPerCTA = 232448;       // 227 KB opt-in maximum per CTA

// n / d as (n * m) >> k, exact for 0 <= n < 2^24 and 1 <= d < 2^12
// (m = ceil(2^k / d) with k = 24 + ceil(log2 d): the round-up reciprocal of
// Granlund and Montgomery, which fits 32 bits here).
struct FastDiv {
    uint32_t m;
    int k;
};
FastDiv make_fastdiv(uint32_t d) {
    int s = 0;
    while ((1u << s) < d) ++s;
    const int k = 24 + s;
    return FastDiv{(uint32_t)(((1ull << k) + d - 1) / d), k};
}
__device__ __forceinline__ int fdiv(int n, const FastDiv& f) {
    return (int)(((uint64_t)(uint32_t)n * f.m) >> f.k);
}

struct TcGeom {
    int nd, L, V, P, C, Cp, T;
    int p_first;          // padded position of site (0, ..., 0) = 1 + P (+ P^2); also the largest tap offset
    int n_tiles;          // tiles covering the positions p_first .. L p_first, 96 each
    int npos;             // positions held per channel group (multiple of 8)
    int r_lag;            // tiles after a tile that read its outputs' positions: ceil(p_first / 96)
    int npad;             // P^nd: positions of the padded lattice
    int nbuf2, nbuf3, tmem_cols;   // TMEM accumulators per epilogue group: conv2 (3 Cp columns), conv3 (16); set at launch
    FastDiv fd_half, fd_Lh, fd_L, fd_P, fd_PP;
    uint32_t w2_bytes, w3_bytes, wf_bytes, layer_bytes;   // layer block: W2 | W3 | FP32 part
    int wf_W1, wf_b1, wf_b2, wf_b3;                        // float offsets in the FP32 part
    uint32_t off_act, off_w2, off_w3, off_wf, off_x, off_red, off_bar, smem_need;
    uint32_t half_bytes;   // shared memory of one half (smem_need rounded up to 1 KB)
};

struct TcArgs {
    TcGeom g;
    const unsigned char* Wl;   // per-layer blocks (layer_bytes each)
    int n_layers;
    float slope;
    int use_tanh, has_phi4;
    FF c2d_ff, lam_ff;
    int64_t B;
    uint64_t seed, counter0;
    const float* z_in; float* z_out; const float* phi_in; float* phi_out;
    double* logq_out; double* S_out; double* logw_out;
    int32_t* status;
    long long stall_spins;     // > 0: failure-path test (gf_set_bf16_stall_test)
};

__device__ __forceinline__ int wrapc(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// conv2's N, the TMEM columns of one accumulator: the three x-taps of CP
// channels (width 8: 24, padded to 32, a multiple of 16)
template <int CP>
__host__ __device__ constexpr int tc_n2() { return CP == 8 ? 32 : 3 * CP; }

// Width 8: the (dz, dy) tap (dz 3 + dy in 3D, dy in 2D) in half kh of
// K-step k (issue_tile_c8), or -1 for the repeated tap's zero weights.
__host__ __device__ inline int tc8_tap(int nd, int k, int kh) {
    const int ta = nd == 3 ? (k < 4 ? 2 * k : 7) : k;
    if (kh == 0 && ta == (nd == 3 ? 7 : 1) && k == (nd == 3 ? 4 : 1)) return -1;
    return ta + kh;
}
__device__ __forceinline__ float lrelu_tc(float v, float a) { return v > 0.f ? v : a * v; }

// Bounded wait for completion number n (0-based) of an mbarrier (phase parity
// n & 1; every waiter has seen completion n - 1 already, so the parity names
// completion n).  False when the limit ran out (the CTA's abort flag is raised
// and GF_ETIMEOUT recorded) or another thread already gave up.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, int64_t n, volatile int* abort_flag, int32_t* status) {
    long long spins = 0;
    while (!mbar_try_wait(bar, (uint32_t)(n & 1))) {
        ++spins;
        if ((spins & 63) == 0 && *abort_flag) return false;
        if (spins > kTcWaitLimit) {
            *abort_flag = 1;
            set_status(status, GF_ETIMEOUT);
            return false;
        }
    }
    return true;
}
// Bounded wait ignoring the abort flag (teardown: issued work must finish
// before its shared memory or TMEM is released).
__device__ __forceinline__ void tc_drain(uint64_t* bar, int64_t n) {
    for (long long spins = 0; !mbar_try_wait(bar, (uint32_t)(n & 1)) && spins < kTcWaitLimit; ++spins) {}
}

__device__ __forceinline__ uint4 pack_bf16x8(const float* v) {
    __align__(16) __nv_bfloat162 p[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    return *reinterpret_cast<const uint4*>(p);
}
__device__ __forceinline__ uint4 pack_f16x8(const float* v) {
    __align__(16) __half2 p[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) p[i] = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
    return *reinterpret_cast<const uint4*>(p);
}

// Padded coordinates (px, py, pz) of position p (row stride P, plane stride
// PP); pz = 1 in 2D.
template <int ND>
__device__ __forceinline__ void pos_xyz(int p, int P, int PP, FastDiv fdP, FastDiv fdPP, int& px, int& py, int& pz) {
    int rem = p;
    pz = 1;
    if (ND == 3) {
        pz = fdiv(p, fdPP);
        rem = p - pz * PP;
    }
    py = fdiv(rem, fdP);
    px = rem - py * P;
}

// conv1: h1 = LReLU(W1 * (x at the frozen sites) + b1) for every site, all
// channels per thread, BF16, at the site's padded position and its periodic
// images.  Sites are ordered (parity, site), so a warp holds one site parity
// and the live taps (those that reach frozen sites) are the same for the
// whole warp; the weight loads are broadcasts.  A thread takes NS sites of
// one parity (j and j + V/(2 NS)), so each weight load feeds NS sites.  Site
// j of parity q (rows y + L z in order, x fastest in a row): x = 2 (j mod
// L/2) + ((q + y + z) mod 2).
template <int ND, int CP, int NS>
__device__ void tc_conv1(const TcGeom& g, const float* wf, const float* x, int frozen, float slope,
                         unsigned char* act, int t0, int nthr) {
    constexpr int NKG = CP / 8;
    const int L = g.L, half = g.V >> 1, per = half / NS, Lh = L >> 1, P = g.P, npos = g.npos;
    const float* W1 = wf + g.wf_W1;
    const float* b1 = wf + g.wf_b1;
    for (int it = t0; it < 2 * per; it += nthr) {
        const int q = it >= per ? 1 : 0, j0 = it - q * per;
        int xc[NS], yc[NS], zc[NS], xs[NS][3], ys[NS][3], zs[NS][3];
#pragma unroll
        for (int n = 0; n < NS; ++n) {
            const int j = j0 + n * per;
            const int r = fdiv(j, g.fd_Lh), xh = j - r * Lh;
            zc[n] = ND == 3 ? fdiv(r, g.fd_L) : 0;
            yc[n] = r - zc[n] * L;
            xc[n] = 2 * xh + ((q ^ yc[n] ^ zc[n]) & 1);
            xs[n][0] = wrapc(xc[n] - 1, L); xs[n][1] = xc[n]; xs[n][2] = wrapc(xc[n] + 1, L);
            ys[n][0] = wrapc(yc[n] - 1, L) * L; ys[n][1] = yc[n] * L; ys[n][2] = wrapc(yc[n] + 1, L) * L;
            zs[n][0] = zs[n][1] = zs[n][2] = 0;
            if (ND == 3) {
                zs[n][0] = wrapc(zc[n] - 1, L) * L * L;
                zs[n][1] = zc[n] * L * L;
                zs[n][2] = wrapc(zc[n] + 1, L) * L * L;
            }
        }
        float acc[NS][CP];
#pragma unroll
        for (int c4 = 0; c4 < CP / 4; ++c4) {
            const float4 b = *reinterpret_cast<const float4*>(b1 + 4 * c4);
#pragma unroll
            for (int n = 0; n < NS; ++n) {
                acc[n][4 * c4] = b.x; acc[n][4 * c4 + 1] = b.y; acc[n][4 * c4 + 2] = b.z; acc[n][4 * c4 + 3] = b.w;
            }
        }
#pragma unroll
        for (int dz = 0; dz < (ND == 3 ? 3 : 1); ++dz) {
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    // parity of the tap offset; the neighbour's parity is q ^ po
                    const int po = ND == 3 ? ((dx + dy + dz + 1) & 1) : ((dx + dy) & 1);
                    if ((q ^ po) != frozen) continue;
                    const int t = ND == 3 ? (dz * 3 + dy) * 3 + dx : dy * 3 + dx;
                    float v[NS];
#pragma unroll
                    for (int n = 0; n < NS; ++n) v[n] = x[zs[n][dz] + ys[n][dy] + xs[n][dx]];
                    const float4* w = reinterpret_cast<const float4*>(W1 + t * CP);
#pragma unroll
                    for (int c4 = 0; c4 < CP / 4; ++c4) {
                        const float4 ww = w[c4];
#pragma unroll
                        for (int n = 0; n < NS; ++n) {
                            acc[n][4 * c4] = fmaf(v[n], ww.x, acc[n][4 * c4]);
                            acc[n][4 * c4 + 1] = fmaf(v[n], ww.y, acc[n][4 * c4 + 1]);
                            acc[n][4 * c4 + 2] = fmaf(v[n], ww.z, acc[n][4 * c4 + 2]);
                            acc[n][4 * c4 + 3] = fmaf(v[n], ww.w, acc[n][4 * c4 + 3]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int n = 0; n < NS; ++n) {
#pragma unroll
            for (int c = 0; c < CP; ++c) acc[n][c] = lrelu_tc(acc[n][c], slope);
            // padded coordinates of the site and of its periodic images (a site on
            // the first or last row of an axis is also the halo beyond the other end)
            int xo[2], yo[2], zo[2], nx = 1, ny = 1, nz = 1;
            xo[0] = xc[n] + 1;
            if (xc[n] == 0) xo[nx++] = L + 1; else if (xc[n] == L - 1) xo[nx++] = 0;
            yo[0] = (yc[n] + 1) * P;
            if (yc[n] == 0) yo[ny++] = (L + 1) * P; else if (yc[n] == L - 1) yo[ny++] = 0;
            zo[0] = ND == 3 ? (zc[n] + 1) * P * P : 0;
            if (ND == 3) {
                if (zc[n] == 0) zo[nz++] = (L + 1) * P * P; else if (zc[n] == L - 1) zo[nz++] = 0;
            }
#pragma unroll
            for (int kg = 0; kg < NKG; ++kg) {
                const uint4 w = pack_bf16x8(acc[n] + 8 * kg);
                unsigned char* base = act + (size_t)kg * npos * 16;
                for (int iz = 0; iz < nz; ++iz)
                    for (int iy = 0; iy < ny; ++iy)
                        for (int ix = 0; ix < nx; ++ix)
                            *reinterpret_cast<uint4*>(base + (size_t)(xo[ix] + yo[iy] + zo[iz]) * 16) = w;
            }
        }
    }
}

// The periodic images: every halo position of the padded lattice (one of
// its coordinates 0 or L + 1) takes the value of the interior position it
// is an image of.  The halo is enumerated face by face (3D: the two z faces
// of P^2 positions, the two y faces of L P, the two x faces of L^2; 2D: the
// two y rows of P, the two x columns of L), so no thread visits the interior.
template <int ND, int CP>
__device__ void tc_halo(const TcGeom& g, unsigned char* act, int t0, int nthr) {
    constexpr int NKG = CP / 8;
    const int L = g.L, P = g.P, npos = g.npos, PP = P * P, LL = L * L, LP = L * P;
    const int nhalo = ND == 3 ? PP * P - LL * L : PP - LL;
    for (int i = t0; i < nhalo; i += nthr) {
        int px, py, pz = 1;
        if (ND == 3) {
            if (i < 2 * PP) {                       // z faces
                const int f = i >= PP, rem = i - f * PP;
                pz = f ? L + 1 : 0;
                py = fdiv(rem, g.fd_P);
                px = rem - py * P;
            } else if (i < 2 * PP + 2 * LP) {       // y faces, 1 <= z <= L
                const int j = i - 2 * PP, f = j >= LP, rem = j - f * LP, t = fdiv(rem, g.fd_P);
                py = f ? L + 1 : 0;
                pz = 1 + t;
                px = rem - t * P;
            } else {                                // x faces, 1 <= y, z <= L
                const int k = i - 2 * PP - 2 * LP, f = k >= LL, rem = k - f * LL, t = fdiv(rem, g.fd_L);
                px = f ? L + 1 : 0;
                pz = 1 + t;
                py = 1 + rem - t * L;
            }
        } else {
            if (i < 2 * P) {                        // y rows
                const int f = i >= P;
                px = i - f * P;
                py = f ? L + 1 : 0;
            } else {                                // x columns, 1 <= y <= L
                const int k = i - 2 * P, f = k >= L;
                py = 1 + k - f * L;
                px = f ? L + 1 : 0;
            }
        }
        const int p = px + py * P + (ND == 3 ? pz * PP : 0);
        const int sx = px == 0 ? L : (px == L + 1 ? 1 : px);
        const int sy = py == 0 ? L : (py == L + 1 ? 1 : py);
        const int sz = ND == 3 ? (pz == 0 ? L : (pz == L + 1 ? 1 : pz)) : 0;
        const int src = sx + sy * P + sz * P * P;
#pragma unroll
        for (int kg = 0; kg < NKG; ++kg)
            *reinterpret_cast<uint4*>(act + ((size_t)kg * npos + p) * 16) =
                *reinterpret_cast<const uint4*>(act + ((size_t)kg * npos + src) * 16);
    }
}

// One issuing thread: a convolution's tile as an implicit GEMM with the three
// x-taps stacked along N: for each (dz, dy) and K-step of 16 channels one MMA
// whose column block dx holds the partial sum of tap (dz, dy, dx) at the row's
// own position; the epilogue adds block dx of the row one position to the
// left / right.  Rows: 16 core matrices of 8 positions, each 6 positions after
// the previous one (SBO = 96 bytes), so row 8 g + r is position
// first + 6 g + r and every row with r in 1..6 finds both x-neighbours in its
// own 8 rows.  a0 / b0: descriptors of the activations and of the weights'
// first block; P, PP: the padded row and plane strides; a_ks, b_tap, b_ks:
// descriptor steps (16-byte units).  Everything arrives by value (registers):
// the issuing thread is latency-bound, and values read from the kernel's
// parameters would be read again after every tcgen05 statement.
template <int ND, int CP>
__device__ __forceinline__ void issue_tile(int first, int P, int PP, uint32_t d, uint64_t a0, uint64_t b0,
                                           uint32_t a_ks, uint32_t b_tap, uint32_t b_ks, uint32_t idesc) {
#pragma unroll
    for (int dz = 0; dz < (ND == 3 ? 3 : 1); ++dz) {
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const int tp = (ND == 3 ? dz * 3 : 0) + dy;
            const uint64_t arow = desc_add(a0, (uint32_t)(first + (dy - 1) * P + (ND == 3 ? (dz - 1) * PP : 0)));
#pragma unroll
            for (int ks = 0; ks < CP / 16; ++ks) {
                const uint64_t ad = desc_add(arow, (uint32_t)ks * a_ks);
                const uint64_t bd = desc_add(b0, (uint32_t)tp * b_tap + (uint32_t)ks * b_ks);
                mma_bf16(d, ad, bd, idesc, (tp | ks) ? 1u : 0u);
            }
        }
    }
}

// Width 8: one K-step of 16 takes the 8 channels of two (dz, dy) taps; the
// descriptor's K-direction core-matrix stride (LBO) is the distance between
// the two taps' positions: P within a z-plane (aP), P^2 - 2P from (dz, 2) to
// (dz + 1, 0) (aQ).  The 3^(d-1) taps pair as (0,1) (2,3) (4,5) (6,7) (7,8)
// in 3D and (0,1) (1,2) in 2D; the repeated tap (7, resp. 1) has zero
// weights in the second pair that holds it (tc8_tap).
template <int ND>
__device__ __forceinline__ void issue_tile_c8(int first, int P, int PP, uint32_t d, uint64_t aP, uint64_t aQ,
                                              uint64_t b0, uint32_t b_ks, uint32_t idesc) {
    constexpr int NKS = ND == 3 ? 5 : 2;
#pragma unroll
    for (int k = 0; k < NKS; ++k) {
        const int ta = ND == 3 ? (k < 4 ? 2 * k : 7) : k;   // first tap of the pair
        const int dz = ND == 3 ? ta / 3 : 1, dy = ND == 3 ? ta % 3 : ta;
        const uint64_t ad = desc_add((ND == 3 && k == 1) ? aQ : aP, (uint32_t)(first + (dy - 1) * P + (dz - 1) * PP));
        mma_bf16(d, ad, desc_add(b0, (uint32_t)k * b_ks), idesc, k ? 1u : 0u);
    }
}

// H halves of 12 warps each run one configuration at a time on their own
// shared memory, TMEM columns and barriers (bar.sync 1 + half between
// their phases), so that one half's CUDA-core phases overlap the other's
// tensor-core phases: the runtime places a single CTA of a tcgen05 kernel
// on an SM.
template <int ND, int CP, bool INVERSE, int H>
__global__ void __launch_bounds__(kTcThreads * H, 1) flow_tc_kernel(const TcArgs a) {
    constexpr int NKG = CP / 8;
    constexpr int N2 = tc_n2<CP>();
    extern __shared__ __align__(1024) unsigned char smem_all[];
    const TcGeom& g = a.g;
    const int h = H == 1 ? 0 : (int)(threadIdx.x / kTcThreads);
    unsigned char* smem = smem_all + (size_t)h * g.half_bytes;
    unsigned char* act = smem + g.off_act;
    unsigned char* w2s = smem + g.off_w2;
    unsigned char* w3s = smem + g.off_w3;
    float* wfs = reinterpret_cast<float*>(smem + g.off_wf);
    float* x = reinterpret_cast<float*>(smem + g.off_x);
    FF* red = reinterpret_cast<FF*>(smem + g.off_red);
    // TMEM accumulator rings, one per epilogue group: full = the tile's MMAs
    // done (commit), empty = its accumulator drained (the group's 128 threads)
    uint64_t* full2 = reinterpret_cast<uint64_t*>(smem + g.off_bar);   // [2][kTcRing]
    uint64_t* empty2 = full2 + 2 * kTcRing;
    uint64_t* full3 = empty2 + 2 * kTcRing;
    uint64_t* empty3 = full3 + 2 * kTcRing;
    uint64_t* done2 = empty3 + 2 * kTcRing;                              // [kTcMaxTiles]: conv2 tile done, once a layer
    uint64_t* bar_w2 = done2 + kTcMaxTiles;                              // a layer's W2 staged
    uint64_t* bar_w3 = bar_w2 + 1;                                       // a layer's W3 staged
    uint64_t* bar_wf = bar_w3 + 1;                                       // 2: a layer's FP32 part staged
    uint64_t* bar_fin = bar_wf + 2;                                      // every queued MMA done (exit)
    uint64_t* bar_stall = bar_fin + 1;                                   // never completed (failure-path test)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_stall + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = (int)threadIdx.x - h * kTcThreads, lane = tid & 31, warp = tid >> 5;   // within the half
    // geometry in registers (the tcgen05 statements' memory clobbers would
    // otherwise make every use read the kernel parameters again)
    const int V = g.V, L = g.L, npos = g.npos, nt = g.n_tiles, P = g.P, PP = g.P * g.P, p_first = g.p_first;
    const int nb2 = g.nbuf2, nb3 = g.nbuf3, r_lag = g.r_lag;
    const FastDiv fdP = g.fd_P, fdPP = g.fd_PP;
    const uint32_t a_ks = 2u * (uint32_t)npos;
    const int wf_floats = (int)(g.wf_bytes >> 2);
    const int64_t b0 = (int64_t)blockIdx.x * H + h, bstride = (int64_t)gridDim.x * H;
    const int64_t n_cfg = a.B > b0 ? (a.B - 1 - b0) / bstride + 1 : 0;
    const int64_t total_steps = n_cfg * a.n_layers;   // this half's layer applications
    int64_t w2_issued = -1, w3_issued = -1, wf_issued = -1;   // thread 0: the last staged steps
    // epilogue warps: group eg (0: warps 4..7, 1: warps 8..11) takes the tiles
    // t = eg (mod 2) through its own TMEM ring; warp w reads lane quarter w mod 4
    const int eg = warp >= 4 ? (warp - 4) >> 2 : -1, q = warp & 3;

    const auto block_of = [&](int64_t step) {
        const int li = (int)(step % a.n_layers);
        return a.Wl + (size_t)(INVERSE ? a.n_layers - 1 - li : li) * g.layer_bytes;
    };
    const auto stage = [&](int64_t step, void* dst, uint32_t off, uint32_t bytes, uint64_t* bar) {
        fence_proxy_async();
        mbar_expect_tx(bar, bytes);
        bulk_g2s(dst, block_of(step) + off, bytes, bar);
    };
    const auto stage_w2 = [&](int64_t step) { stage(step, w2s, 0, g.w2_bytes, bar_w2); w2_issued = step; };
    const auto stage_w3 = [&](int64_t step) { stage(step, w3s, g.w2_bytes, g.w3_bytes, bar_w3); w3_issued = step; };
    const auto stage_wf = [&](int64_t step) {
        stage(step, wfs + (int)(step & 1) * wf_floats, g.w2_bytes + g.w3_bytes, g.wf_bytes, bar_wf + (step & 1));
        wf_issued = step;
    };

    // one allocation for the CTA (warp 0 of half 0); half h uses columns
    // h * tmem_cols .. (h + 1) * tmem_cols
    uint32_t* tmem_slot0 = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(tmem_slot) - h * g.half_bytes);
    if (threadIdx.x < 32) {
        tmem_alloc(tmem_slot0, (uint32_t)(g.tmem_cols * H));
        tmem_relinquish();
    }
    const auto half_sync = [&]() {
        if (H == 1) __syncthreads();
        else asm volatile("bar.sync %0, %1;" :: "r"(1 + h), "r"(kTcThreads) : "memory");
    };
    // FP64-accurate sum over the half's threads (fixed order)
    const auto half_sum = [&](FF v) {
        v = warp_sum_ff(v);
        if (lane == 0) red[warp] = v;
        half_sync();
        FF r = lane < kTcThreads / 32 ? red[lane] : FF{0.f, 0.f};
        r = warp_sum_ff(r);
        half_sync();
        return ff_to_double(r);
    };
    if (tid == 0) {
        for (int i = 0; i < 2 * kTcRing; ++i) {
            mbar_init(full2 + i, 1);
            mbar_init(empty2 + i, 4 * 32);
            mbar_init(full3 + i, 1);
            mbar_init(empty3 + i, 4 * 32);
        }
        for (int i = 0; i < kTcMaxTiles; ++i) mbar_init(done2 + i, 1);
        mbar_init(bar_w2, 1);
        mbar_init(bar_w3, 1);
        mbar_init(bar_wf, 1);
        mbar_init(bar_wf + 1, 1);
        mbar_init(bar_fin, 2);                 // one commit per issuing thread
        mbar_init(bar_stall, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    // positions past the padded lattice feed only dropped rows of the last
    // tiles; zero them once so every MMA reads finite numbers
    for (int i = tid; i < NKG * npos; i += kTcThreads)
        reinterpret_cast<uint4*>(act)[i] = make_uint4(0u, 0u, 0u, 0u);
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (tid == 0 && total_steps > 0) {
        stage_w2(0);
        stage_w3(0);
        stage_wf(0);
    }
    const uint32_t tmem = *tmem_slot0 + (uint32_t)(h * g.tmem_cols);
    // D = F32, K-major A and B, M = 128: conv2 BF16 with N = 3 CP, conv3 FP16 with N = 16
    const uint32_t idesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N2 >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);
    const uint32_t idesc3 = (1u << 4) | ((16u >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
    const uint64_t a0 = smem_desc(smem_u32(act), (uint32_t)npos * 16u, 6u * 16u);
    // width 8: the two tap-pair strides (issue_tile_c8)
    const uint64_t aP = smem_desc(smem_u32(act), (uint32_t)P * 16u, 6u * 16u);
    const uint64_t aQ = smem_desc(smem_u32(act), (uint32_t)(PP - 2 * P) * 16u, 6u * 16u);
    // [tp][kg][dx CP + c][8] bf16 (width 8: [pair][tap][dx 8 + c][8], N = 32)
    const uint64_t b2d = smem_desc(smem_u32(w2s), (uint32_t)N2 * 16u, 128u);
    // [tp][kg][2 dx + j][8] fp16 (width 8: [pair][tap][2 dx + j][8])
    const uint64_t b3d = smem_desc(smem_u32(w3s), 16u * 16u, 128u);
    // this thread's row of a tile: position first + 6 (row >> 3) + (row & 7),
    // an output when row & 7 is in 1..6
    const int row = 32 * q + lane, roff = 6 * (row >> 3) + (row & 7);
    const bool rvalid = (row & 7) >= 1 && (row & 7) <= 6;

    int64_t step = 0;
    // the next accumulator of this thread's ring (issuing thread r: ring r;
    // epilogue group g: ring g) and how often it has been filled before
    int i2 = 0, i3 = 0;
    int64_t k2 = 0, k3 = 0;
    for (int64_t b = b0; b < a.B; b += bstride) {
        // prior sample (sampling) or the given field (inverting)
        FF sumz2{0.f, 0.f};
        if (!INVERSE) {
            if (a.z_in) {
                for (int n = tid; n < V; n += kTcThreads) {
                    const float v = __ldg(a.z_in + b * V + n);
                    x[n] = v;
                    const float p = v * v;
                    ff_add(sumz2, FF{p, fmaf(v, v, -p)});
                }
            } else {
                for (int jq = tid; 4 * jq < V; jq += kTcThreads) {
                    const u64x4 w = philox4x64_10(a.seed, 0ull,
                                                  u64x4{a.counter0 + (uint64_t)b, (uint64_t)jq, 0ull, TAG_PRIOR});
                    float zz[4];
                    normals4_f32(w, zz);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        x[4 * jq + k] = zz[k];
                        const float p = zz[k] * zz[k];
                        ff_add(sumz2, FF{p, fmaf(zz[k], zz[k], -p)});
                    }
                }
            }
            half_sync();
            if (a.z_out)
                for (int n = tid; n < V; n += kTcThreads) a.z_out[b * V + n] = x[n];
        } else {
            for (int n = tid; n < V; n += kTcThreads) x[n] = __ldg(a.phi_in + b * V + n);
        }
        half_sync();

        FF logdet{0.f, 0.f};
        for (int li = 0; li < a.n_layers; ++li, ++step) {
            const int l = INVERSE ? a.n_layers - 1 - li : li;
            const int frozen = l & 1;
            const float* wf = wfs + (int)(step & 1) * wf_floats;

            // ---- conv1 -> h1 (BF16, padded, with periodic images)
            if (tc_wait(bar_wf + (step & 1), step >> 1, abort_flag, a.status)) {
                if (tid == 0 && step + 1 < total_steps) stage_wf(step + 1);
                tc_conv1<ND, CP, H == 1 ? 2 : 1>(g, wf, x, frozen, a.slope, act, tid, kTcThreads);
            }
            fence_proxy_async();
            half_sync();
            if (*abort_flag) break;

            // ---- conv2 on the tensor cores; the epilogue writes h2 (FP16) over h1 in place
            if (warp < 2) {
                // issuing thread r (lane 0 of warp r, sub-partition r): tiles t = r (mod 2) into ring r
                bool go = lane == 0;
                if (go && a.stall_spins > 0 && step == 0 && warp == 0) {
                    // failure-path test: a wait for a completion that never comes,
                    // before this half's first MMA
                    for (long long spins = 0; !mbar_try_wait(bar_stall, 0u); ++spins)
                        if (spins > a.stall_spins) {
                            *abort_flag = 1;
                            set_status(a.status, GF_ETIMEOUT);
                            go = false;
                            break;
                        }
                }
                if (go && tc_wait(bar_w2, step, abort_flag, a.status)) {
                    fence_after_sync();
                    for (int t = warp; t < nt; t += 2) {
                        if (k2 >= 1) {
                            if (!tc_wait(empty2 + warp * kTcRing + i2, k2 - 1, abort_flag, a.status)) break;
                            fence_after_sync();
                        }
                        const uint32_t d2 = tmem + (uint32_t)((warp * nb2 + i2) * N2);
                        if constexpr (CP == 8)
                            issue_tile_c8<ND>(p_first - 1 + kTcOut * t, P, PP, d2, aP, aQ, b2d, 2u * N2, idesc2);
                        else
                            issue_tile<ND, CP>(p_first - 1 + kTcOut * t, P, PP, d2, a0, b2d, a_ks,
                                               (uint32_t)(NKG * N2), (uint32_t)(2 * N2), idesc2);
                        mma_commit(full2 + warp * kTcRing + i2);
                        mma_commit(done2 + t);
                        if (++i2 == nb2) { i2 = 0; ++k2; }
                    }
                }
                __syncwarp();
            } else if (eg >= 0) {
                const float* b2 = wf + g.wf_b2;
                int dwaited = 0;           // tiles whose completion this thread has seen (done2)
                bool ok = true;
                for (int t = eg; t < nt && ok; t += 2) {
                    if (!(ok = tc_wait(full2 + eg * kTcRing + i2, k2, abort_flag, a.status))) break;
                    fence_after_sync();
                    // out = D_0(left) + D_1 + D_2(right) + b2, 16 channels at a time, LeakyReLU
                    const uint32_t tcol = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((eg * nb2 + i2) * N2);
                    float out[CP];
                    if constexpr (CP == 8) {
                        // columns dx 8 + c; 24..31 are the zero padding of N
                        float v01[16], v2p[16];
                        tmem_ld16(tcol, v01);
                        tmem_ld16(tcol + 16, v2p);
                        tmem_ld_wait();
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const float left = __shfl_up_sync(0xffffffffu, v01[c], 1, 8);
                            const float right = __shfl_down_sync(0xffffffffu, v2p[c], 1, 8);
                            out[c] = lrelu_tc(left + v01[8 + c] + right + b2[c], a.slope);
                        }
                    }
#pragma unroll
                    for (int h = 0; h < CP / 16; ++h) {
                        float v0[16], v1[16], v2[16];
                        tmem_ld16(tcol + h * 16, v0);
                        tmem_ld16(tcol + CP + h * 16, v1);
                        tmem_ld16(tcol + 2 * CP + h * 16, v2);
                        tmem_ld_wait();
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            const float left = __shfl_up_sync(0xffffffffu, v0[c], 1, 8);
                            const float right = __shfl_down_sync(0xffffffffu, v2[c], 1, 8);
                            out[h * 16 + c] = lrelu_tc(left + v1[c] + right + b2[h * 16 + c], a.slope);
                        }
                    }
                    fence_before_sync();
                    mbar_arrive(empty2 + eg * kTcRing + i2);
                    if (++i2 == nb2) { i2 = 0; ++k2; }
                    // h2 of tile t may overwrite h1 once tiles t .. t + r_lag are done
                    const int need = t + r_lag < nt ? t + r_lag : nt - 1;
                    while (ok && dwaited <= need) {
                        ok = tc_wait(done2 + dwaited, step, abort_flag, a.status);
                        ++dwaited;
                    }
                    if (!ok) break;
                    const int p = p_first - 1 + kTcOut * t + roff;
                    int px, py, pz;
                    pos_xyz<ND>(p, P, PP, fdP, fdPP, px, py, pz);
                    if (rvalid && px >= 1 && px <= L && py >= 1 && py <= L && pz >= 1 && pz <= L) {
#pragma unroll
                        for (int kg = 0; kg < NKG; ++kg)
                            *reinterpret_cast<uint4*>(act + ((size_t)kg * npos + p) * 16) = pack_f16x8(out + kg * 8);
                    }
                }
            }
            fence_before_sync();
            half_sync();
            if (*abort_flag) break;
            fence_after_sync();
            // every conv2 MMA of this layer has completed: the next layer's W2 may land
            if (tid == 0 && step + 1 < total_steps) stage_w2(step + 1);

            // ---- periodic images of h2
            tc_halo<ND, CP>(g, act, tid, kTcThreads);
            fence_proxy_async();
            half_sync();

            // ---- conv3 (s, t) on the tensor cores; the epilogue updates the other parity
            if (warp < 2) {
                if (lane == 0 && tc_wait(bar_w3, step, abort_flag, a.status)) {
                    fence_after_sync();
                    for (int t = warp; t < nt; t += 2) {
                        if (k3 >= 1) {
                            if (!tc_wait(empty3 + warp * kTcRing + i3, k3 - 1, abort_flag, a.status)) break;
                            fence_after_sync();
                        }
                        const uint32_t d3 = tmem + (uint32_t)((warp * nb3 + i3) * 16);
                        if constexpr (CP == 8)
                            issue_tile_c8<ND>(p_first - 1 + kTcOut * t, P, PP, d3, aP, aQ, b3d, 2u * 16u, idesc3);
                        else
                            issue_tile<ND, CP>(p_first - 1 + kTcOut * t, P, PP, d3, a0, b3d, a_ks,
                                               (uint32_t)(NKG * 16), (uint32_t)(2 * 16), idesc3);
                        mma_commit(full3 + warp * kTcRing + i3);
                        if (++i3 == nb3) { i3 = 0; ++k3; }
                    }
                }
                __syncwarp();
            } else if (eg >= 0) {
                const float bs = wf[g.wf_b3], bt = wf[g.wf_b3 + 1];
                const int pa = frozen ^ 1;
                bool ok = true;
                for (int t = eg; t < nt && ok; t += 2) {
                    if (!(ok = tc_wait(full3 + eg * kTcRing + i3, k3, abort_flag, a.status))) break;
                    fence_after_sync();
                    float v[8];
                    tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((eg * nb3 + i3) * 16), v);
                    tmem_ld_wait();
                    fence_before_sync();
                    mbar_arrive(empty3 + eg * kTcRing + i3);
                    if (++i3 == nb3) { i3 = 0; ++k3; }
                    // columns 2 dx + j: j = 0 s, 1 t of tap dx at the row's own position
                    const float sl = __shfl_up_sync(0xffffffffu, v[0], 1, 8);
                    const float tl = __shfl_up_sync(0xffffffffu, v[1], 1, 8);
                    const float sr = __shfl_down_sync(0xffffffffu, v[4], 1, 8);
                    const float tr = __shfl_down_sync(0xffffffffu, v[5], 1, 8);
                    const int p = p_first - 1 + kTcOut * t + roff;
                    int px, py, pz;
                    pos_xyz<ND>(p, P, PP, fdP, fdPP, px, py, pz);
                    // parity of the site (px - 1, py - 1, pz - 1)
                    const int par = ND == 3 ? ((px + py + pz + 1) & 1) : ((px + py) & 1);
                    if (rvalid && px >= 1 && px <= L && py >= 1 && py <= L && pz >= 1 && pz <= L && par == pa) {
                        const float s0 = sl + v[2] + sr + bs;
                        const float s = a.use_tanh ? tanhf(s0) : s0;
                        const float tt = tl + v[3] + tr + bt;
                        if (!isfinite(s) || !isfinite(tt)) set_status(a.status, GF_EDEVICE);
                        float& xv = x[((ND == 3 ? (pz - 1) * L : 0) + (py - 1)) * L + (px - 1)];
                        if (!INVERSE) xv = fmaf(xv, expf(s), tt);
                        else xv = (xv - tt) * expf(-s);
                        ff_add(logdet, s);
                    }
                }
            }
            fence_before_sync();
            half_sync();
            if (*abort_flag) break;
            fence_after_sync();
            // every conv3 MMA of this layer has completed: the next layer's W3 may land
            if (tid == 0 && step + 1 < total_steps) stage_w3(step + 1);
        }
        if (*abort_flag) break;

        if (INVERSE) {
            for (int n = tid; n < V; n += kTcThreads) {
                const float v = x[n];
                const float p = v * v;
                ff_add(sumz2, FF{p, fmaf(v, v, -p)});
                if (a.z_out) a.z_out[b * V + n] = v;
            }
        } else {
            for (int n = tid; n < V; n += kTcThreads) a.phi_out[b * V + n] = x[n];
        }
        const double ld = half_sum(logdet);
        const double z2 = half_sum(sumz2);
        double S = 0.0;
        if (!INVERSE && a.has_phi4) S = half_sum(action_part<ND>(x, L, V, a.c2d_ff, a.lam_ff, tid, kTcThreads));
        if (tid == 0) {
            const double logr = -0.5 * z2 - 0.5 * (double)V * LOG_2PI;
            const double logq = logr - ld;
            a.logq_out[b] = logq;
            if (!INVERSE && a.has_phi4) {
                if (a.S_out) a.S_out[b] = S;
                if (a.logw_out) a.logw_out[b] = -S - logq;
            }
        }
        half_sync();
    }
    // teardown: copies still landing and MMAs still queued (only after an
    // abort) finish before their shared memory and TMEM are released
    if (warp < 2 && lane == 0) mma_commit(bar_fin);
    if (tid == 0) {
        if (w2_issued >= 0) tc_drain(bar_w2, w2_issued);
        if (w3_issued >= 0) tc_drain(bar_w3, w3_issued);
        if (wf_issued >= 0) tc_drain(bar_wf + (wf_issued & 1), wf_issued >> 1);
        tc_drain(bar_fin, 0);
    }
    fence_before_sync();
    __syncthreads();                             // both halves
    if (threadIdx.x < 32) {
        fence_after_sync();
        tmem_dealloc(*tmem_slot0, (uint32_t)(g.tmem_cols * H));
    }
}

// canonical FP32 -> per-layer block: W2 as [tp][kg][dx CP + c][8] bf16 (tap
// (tp, dx) with tp = (dz, dy); K-major core matrices; channels >= C zero), W3
// as [tp][kg][2 dx + j][8] fp16 (j = 0: s, 1: t; rows 6..15 zero), then FP32
// W1 [tap][Cp], b1 [Cp], b2 [Cp], b3 [2], zero padding.  Width 8: W2 as
// [k][kh][dx 8 + c][8] (rows 24..31 zero) and W3 as [k][kh][2 dx + j][8], tp =
// tc8_tap(k, kh) (zero weights where it is -1).
__global__ void repack_tc_kernel(const float* __restrict__ canon, int64_t cstride, int n_layers, TcGeom g,
                                 unsigned char* __restrict__ out) {
    const int T = g.T, C = g.C, CP = g.Cp, NKG = CP / 8, N2 = 3 * CP;
    const int64_t n2 = g.w2_bytes / 2, n3 = g.w3_bytes / 2, nf = g.wf_bytes / 4, per = n2 + n3 + nf;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per * n_layers;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / per);
        const int64_t r = i - l * per;
        const float* W1 = canon + l * cstride;      // [c][0][t]
        const float* b1 = W1 + (int64_t)C * T;
        const float* W2 = b1 + C;                   // [o][i][t]
        const float* b2 = W2 + (int64_t)C * C * T;
        const float* W3 = b2 + C;                   // [o][i][t], o = 0: s, 1: t
        const float* b3 = W3 + 2LL * C * T;
        unsigned char* blk = out + (size_t)l * g.layer_bytes;
        if (CP == 8 && r < n2) {
            const int e = (int)(r & 7), n = (int)((r >> 3) & 31), kh = (int)((r >> 8) & 1), k = (int)(r >> 9);
            const int tp = tc8_tap(g.nd, k, kh), dx = n >> 3, c = n & 7;
            const float v = (tp >= 0 && n < 24 && c < C && e < C) ? W2[((int64_t)c * C + e) * T + tp * 3 + dx] : 0.f;
            reinterpret_cast<__nv_bfloat16*>(blk)[r] = __float2bfloat16_rn(v);
        } else if (CP == 8 && r < n2 + n3) {
            const int r3 = (int)(r - n2);
            const int e = r3 & 7, n = (r3 >> 3) & 15, kh = (r3 >> 7) & 1, k = r3 >> 8;
            const int tp = tc8_tap(g.nd, k, kh), dx = n >> 1, j = n & 1;
            const float v = (tp >= 0 && n < 6 && e < C) ? W3[((int64_t)j * C + e) * T + tp * 3 + dx] : 0.f;
            reinterpret_cast<__half*>(blk + g.w2_bytes)[r3] = __float2half_rn(v);
        } else if (r < n2) {
            const int e = (int)(r & 7), n = (int)((r >> 3) % N2), kg = (int)((r / (8 * N2)) % NKG);
            const int tp = (int)(r / (8 * N2 * NKG)), dx = n / CP, c = n % CP, ic = kg * 8 + e;
            const int t = tp * 3 + dx;
            const float v = (c < C && ic < C) ? W2[((int64_t)c * C + ic) * T + t] : 0.f;
            reinterpret_cast<__nv_bfloat16*>(blk)[r] = __float2bfloat16_rn(v);
        } else if (r < n2 + n3) {
            const int r3 = (int)(r - n2);
            const int e = r3 & 7, n = (r3 >> 3) & 15, kg = (r3 >> 7) % NKG, tp = r3 / (128 * NKG), ic = kg * 8 + e;
            const int dx = n >> 1, j = n & 1, t = tp * 3 + dx;
            const float v = (n < 6 && ic < C) ? W3[((int64_t)j * C + ic) * T + t] : 0.f;
            reinterpret_cast<__half*>(blk + g.w2_bytes)[r3] = __float2half_rn(v);
        } else {
            const int f = (int)(r - n2 - n3);
            float v = 0.f;
            if (f < g.wf_b1) {
                const int t = f / CP, c = f % CP;
                if (c < C) v = W1[(int64_t)c * T + t];
            } else if (f < g.wf_b2) {
                const int c = f - g.wf_b1;
                if (c < C) v = b1[c];
            } else if (f < g.wf_b3) {
                const int c = f - g.wf_b2;
                if (c < C) v = b2[c];
            } else if (f < g.wf_b3 + 2) {
                v = b3[f - g.wf_b3];
            }
            reinterpret_cast<float*>(blk + g.w2_bytes + g.w3_bytes)[f] = v;
        }
    }
}

// Geometry and shared-memory plan of a shape; false when this kernel does not
// take it (the TMEM rings are chosen at launch).
bool tc_plan(const gf_flow_shape& s, TcGeom& g) {
    std::memset(&g, 0, sizeof(g));
    if (s.nd != 2 && s.nd != 3) return false;
    if (s.ksize != 3 || s.c_hidden1 != s.c_hidden2) return false;
    const int C = s.c_hidden1;
    // width 24 runs as 32 with zero weights and biases in the padding
    // channels, whose activations are then LReLU(0) = 0
    if (C < 8 || C > 32 || C % 8 != 0) return false;
    if (s.nd == 3 && s.L == 16 && C == 32) return false;   // the dedicated 3D L=16 kernel
    if (s.L < 4 || (s.L & 1)) return false;
    g.nd = s.nd;
    g.L = s.L;
    g.C = C;
    g.Cp = C == 8 ? 8 : (C <= 16 ? 16 : 32);
    g.V = 1;
    for (int i = 0; i < s.nd; ++i) g.V *= s.L;
    if (g.V % 64 != 0 || g.V > 65536) return false;        // V/2 a multiple of 32: parity-uniform warps
    g.P = s.L + 2;
    g.T = s.nd == 3 ? 27 : 9;
    g.npad = s.nd == 3 ? g.P * g.P * g.P : g.P * g.P;
    g.p_first = s.nd == 3 ? 1 + g.P + g.P * g.P : 1 + g.P;
    const int p_last = g.p_first * s.L;
    g.n_tiles = (p_last - g.p_first + 1 + kTcOut - 1) / kTcOut;
    if (g.n_tiles > kTcMaxTiles) return false;
    // tile t reads positions 96 t .. 96 t + 96 + 2 p_first - 1 (rows first .. first + 97, taps +-(p_first - 1))
    g.npos = (2 * g.p_first + g.n_tiles * kTcOut + 7) & ~7;
    if (g.npos > 16383) return false;                      // descriptor LBO field (16-byte units)
    g.r_lag = (g.p_first + kTcOut - 1) / kTcOut;
    g.fd_half = make_fastdiv((uint32_t)(g.V / 2));
    g.fd_Lh = make_fastdiv((uint32_t)(s.L / 2));
    g.fd_L = make_fastdiv((uint32_t)s.L);
    g.fd_P = make_fastdiv((uint32_t)g.P);
    g.fd_PP = make_fastdiv((uint32_t)(g.P * g.P));
    if (g.V / 2 >= 4096 || g.npos * 4 >= (1 << 24)) return false;   // FastDiv ranges
    const int NKG = g.Cp / 8;
    if (g.Cp == 8) {
        const int nks = s.nd == 3 ? 5 : 2;                 // K-steps of two taps (issue_tile_c8)
        g.w2_bytes = (uint32_t)(nks * 2 * tc_n2<8>() * 16);
        g.w3_bytes = (uint32_t)(nks * 2 * 16 * 16);
    } else {
        g.w2_bytes = (uint32_t)(g.T / 3 * NKG * 3 * g.Cp * 16);
        g.w3_bytes = (uint32_t)(g.T / 3 * NKG * 16 * 16);
    }
    g.wf_W1 = 0;
    g.wf_b1 = g.T * g.Cp;
    g.wf_b2 = g.wf_b1 + g.Cp;
    g.wf_b3 = g.wf_b2 + g.Cp;
    g.wf_bytes = (uint32_t)(((g.wf_b3 + 2 + 3) & ~3) * 4);
    g.layer_bytes = g.w2_bytes + g.w3_bytes + g.wf_bytes;
    g.off_act = 0;
    g.off_w2 = (uint32_t)NKG * g.npos * 16;
    g.off_w3 = g.off_w2 + g.w2_bytes;
    g.off_wf = g.off_w3 + g.w3_bytes;
    g.off_x = g.off_wf + 2 * g.wf_bytes;
    g.off_red = g.off_x + (uint32_t)((g.V * 4 + 15) & ~15);
    g.off_bar = g.off_red + 32 * 8;
    g.smem_need = g.off_bar + (8 * kTcRing + kTcMaxTiles + 6) * 8 + 16;
    g.half_bytes = (g.smem_need + 1023) & ~1023u;
    return g.smem_need <= (uint32_t)kSmemPerCTA;
}

template <int ND, int CP, bool INV, int H>
gf_status launch_tc(TcArgs& a, cudaStream_t stream) {
    auto kern = flow_tc_kernel<ND, CP, INV, H>;
    TcGeom& g = a.g;
    const size_t smem = (size_t)H * g.half_bytes;
    if (smem > (size_t)kSmemPerCTA) return GF_EUNSUPPORTED;
    // once per device and instantiation: the shared-memory limit, and the
    // check that the runtime places one CTA of this tcgen05 kernel per SM (its
    // H halves share the SM's 512 TMEM columns, each needing two conv2
    // accumulators of tc_n2 columns, one per epilogue group)
    static std::mutex mu;
    static int checked[64] = {0};   // 0: not yet, 1: ok, -1: more than one CTA per SM
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return GF_EUNSUPPORTED;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (checked[dev] == 0) {
            int per_sm = 0;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemPerCTA) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTcThreads * H, kSmemPerCTA / 2) !=
                    cudaSuccess ||
                per_sm < 1)
                return GF_ECUDA;
            checked[dev] = per_sm > 1 ? -1 : 1;
        }
        if (checked[dev] < 0) return GF_EUNSUPPORTED;
    }
    g.tmem_cols = 512 / H;
    g.nbuf2 = std::min(kTcRing, g.tmem_cols / (2 * tc_n2<CP>()));
    g.nbuf3 = std::min(kTcRing, g.tmem_cols / (2 * 16));
    if (g.nbuf2 < 1 || g.nbuf3 < 1) return GF_EUNSUPPORTED;
    // the conv2 schedule needs r_lag <= 2 nbuf2 (+ 1 when r_lag is odd): an
    // epilogue group holding tile t's store waits for tile t + r_lag's MMAs,
    // whose accumulator is the one tile t + r_lag - 2 nbuf2 used, drained only
    // by a group that has reached that tile (the same group when r_lag is
    // even, which has drained up to t; the other, up to t + 1, when odd)
    if (g.r_lag > 2 * g.nbuf2 + (g.r_lag & 1)) return GF_EUNSUPPORTED;
    const int64_t grid = std::min<int64_t>((a.B + H - 1) / H, (int64_t)num_sms());
    if (grid <= 0) return GF_OK;
    kern<<<(unsigned)grid, kTcThreads * H, smem, stream>>>(a);
    GF_CHECK_LAUNCH();
    return GF_OK;
}

}  // namespace

bool tc_supported(const gf_flow_shape* s) {
    TcGeom g;
    return s && tc_plan(*s, g);
}

gf_status tc_configure(gf_flow* f) {
    TcGeom g;
    if (!tc_plan(f->shape, g)) return GF_EUNSUPPORTED;
    f->tc = true;
    if (cudaMalloc(&f->d_bf16, (size_t)g.layer_bytes * std::max(1, f->shape.n_layers)) != cudaSuccess)
        return GF_ENOMEM;
    return GF_OK;
}

gf_status repack_tc(gf_flow* f, cudaStream_t stream) {
    TcGeom g;
    if (!tc_plan(f->shape, g)) return GF_EUNSUPPORTED;
    const int64_t total = (int64_t)(g.w2_bytes / 2 + g.w3_bytes / 2 + g.wf_bytes / 4) * f->shape.n_layers;
    if (total == 0) return GF_OK;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 4096);
    repack_tc_kernel<<<grid, 256, 0, stream>>>(f->d_canon, f->canon_stride, f->shape.n_layers, g,
                                               static_cast<unsigned char*>(f->d_bf16));
    GF_CHECK_LAUNCH();
    return GF_OK;
}

gf_status launch_flow_tc(const gf_flow* f, bool inverse, const gf_phi4* phi4, int64_t B,
                         uint64_t seed, uint64_t counter0, const float* z_in, float* z_out,
                         const float* phi_in, float* phi_out, double* logq_out,
                         double* S_out, double* logw_out, cudaStream_t stream) {
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    if (!tc_plan(f->shape, a.g)) return GF_EUNSUPPORTED;
    a.Wl = static_cast<const unsigned char*>(f->d_bf16);
    a.n_layers = f->shape.n_layers;
    a.slope = (float)f->shape.leaky_slope;
    a.use_tanh = f->shape.use_final_tanh;
    a.has_phi4 = phi4 != nullptr;
    ff_split(2.0 * f->shape.nd + (phi4 ? phi4->m2 : 0.0), &a.c2d_ff.hi, &a.c2d_ff.lo);
    ff_split(phi4 ? phi4->lam : 0.0, &a.lam_ff.hi, &a.lam_ff.lo);
    a.B = B;
    a.seed = seed;
    a.counter0 = counter0;
    a.z_in = z_in; a.z_out = z_out; a.phi_in = phi_in; a.phi_out = phi_out;
    a.logq_out = logq_out; a.S_out = S_out; a.logw_out = logw_out;
    a.status = status_word(stream);
    a.stall_spins = bf16_stall_spins();
    if (!a.status) return GF_ECUDA;
    const bool c32 = a.g.Cp == 32, c8 = a.g.Cp == 8;
    // two configurations per CTA where two halves' shared memory fits (every
    // 2D lattice but the largest; 3D L = 8 with widths 8, 16 and L = 12 with 8)
    const bool two = 2 * (size_t)a.g.half_bytes <= (size_t)kSmemPerCTA && B > num_sms();
    if (f->shape.nd == 3) {
        if (c32) return inverse ? launch_tc<3, 32, true, 1>(a, stream) : launch_tc<3, 32, false, 1>(a, stream);
        if (c8) {
            if (two) return inverse ? launch_tc<3, 8, true, 2>(a, stream) : launch_tc<3, 8, false, 2>(a, stream);
            return inverse ? launch_tc<3, 8, true, 1>(a, stream) : launch_tc<3, 8, false, 1>(a, stream);
        }
        if (two) return inverse ? launch_tc<3, 16, true, 2>(a, stream) : launch_tc<3, 16, false, 2>(a, stream);
        return inverse ? launch_tc<3, 16, true, 1>(a, stream) : launch_tc<3, 16, false, 1>(a, stream);
    }
    if (c8) {
        if (two) return inverse ? launch_tc<2, 8, true, 2>(a, stream) : launch_tc<2, 8, false, 2>(a, stream);
        return inverse ? launch_tc<2, 8, true, 1>(a, stream) : launch_tc<2, 8, false, 1>(a, stream);
    }
    if (c32) {
        if (two) return inverse ? launch_tc<2, 32, true, 2>(a, stream) : launch_tc<2, 32, false, 2>(a, stream);
        return inverse ? launch_tc<2, 32, true, 1>(a, stream) : launch_tc<2, 32, false, 1>(a, stream);
    }
    if (two) return inverse ? launch_tc<2, 16, true, 2>(a, stream) : launch_tc<2, 16, false, 2>(a, stream);
    return inverse ? launch_tc<2, 16, true, 1>(a, stream) : launch_tc<2, 16, false, 1>(a, stream);
}

}  // namespace gf
