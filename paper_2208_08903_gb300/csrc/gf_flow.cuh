// gf_flow.cuh -- internal representation of a flow object and the slice
// schedule shared by the fused coupling-stack kernels.
#pragma once

#include <cstdint>
#include <vector>

#include "gf_common.cuh"

namespace gf {

// A lattice is processed as L "slices" along its outermost axis (z in 3D,
// y in 2D), each of S = L^(nd-1) sites.  Hidden activations h1 / h2 live in
// shared memory in R "slots" of one slice each; a phase computes one kind of
// result for n consecutive slices s0 .. s0+n-1 (mod L):
//   PH_H1: h1 = LReLU(conv1(masked x))     -> slots out[0..n)
//   PH_H2: h2 = LReLU(conv2(h1))           <- h1 of slices s0-1 .. s0+n in in[0..n+2)
//                                          -> slots out[0..n)
//   PH_C3: (s,t) = conv3(h2) at the updated sites, affine update of x
//                                          <- h2 of slices s0-1 .. s0+n in in[0..n+2)
constexpr int PH_H1 = 0, PH_H2 = 1, PH_C3 = 2;
constexpr int MAX_PHASE_SLICES = 62;

struct Phase {
    uint8_t type, n;
    uint16_t s0;
    uint8_t in[MAX_PHASE_SLICES + 2];
    uint8_t out[MAX_PHASE_SLICES + 2];
};

// Builds the per-layer phase list.  full: all L slices resident (R = L).
// Otherwise an LRU slot cache of R = G + 2 slots per tensor, results produced
// G slices at a time, the two wrap-around slices recomputed at the end.
std::vector<Phase> build_schedule(int L, int G, bool full);

}  // namespace gf

struct gf_flow {
    gf_flow_shape shape;
    gf_precision prec;
    int device;
    int V, S, T, C1, C2;
    int64_t n_params;       // canonical parameter count
    int64_t canon_stride;   // canonical floats per layer
    int64_t packed_stride;  // packed floats per layer (multiple of 4)
    float* d_canon;         // FP32 canonical weights [n_params]
    float* d_packed;        // per-layer packed FP32 weights
    gf::Phase* d_sched;
    int n_phases;
    int G;                  // slices per phase (RING) or L (FULL)
    int R;                  // slots per hidden tensor
    bool full;
    size_t smem_bytes;
    bool wsmem;             // FP32 kernel keeps all packed weights in shared memory
    // BF16 tensor-core path: the 3D L=16, C=32 kernel (gf_flow_bf16.cu) or,
    // when tc is set, the kernel for other shapes (gf_flow_tc.cu)
    void* d_bf16;           // per-layer weight blocks of the tensor-core kernel
    size_t smem_bytes_bf16;
    bool tc;
    // General s/t network (gf_flow_create_ex with hidden_sizes other than two
    // equal widths in {8,16,32}, or a kernel size other than 3): whole-lattice
    // FP32 kernel of gf_flow_variant.cu
    bool variant;
    int n_hidden;
    int hidden[GF_MAX_HIDDEN];
    int K;                  // taps per axis
    float* d_vpacked;       // per layer: conv j weights [t][cin][cop], bias [cop]
    int64_t vstride;        // packed floats per layer
    int32_t vwoff[GF_MAX_HIDDEN + 1], vboff[GF_MAX_HIDDEN + 1];
    int32_t vcin[GF_MAX_HIDDEN + 1], vcout[GF_MAX_HIDDEN + 1], vcop[GF_MAX_HIDDEN + 1];
    int Cp;                 // shared-memory row width of the hidden activations (odd)
    int vthreads;
    // reverse pass: the weight gradients of a layer run on `side`, forked from
    // and joined back into the caller's stream with these events
    cudaStream_t side;
    cudaEvent_t ev_fork[3], ev_join;
};

namespace gf {
// Packed layout per layer (floats, from the layer's base):
//   W1p[T][C1], b1[C1], W2p[T][C1][C2], b2[C2], W3p[T][C2][2], b3[2], pad
struct PackedOffsets {
    int64_t W1, b1, W2, b2, W3, b3, stride;
};
PackedOffsets packed_offsets(int T, int C1, int C2);

gf_status repack_weights(gf_flow* f, cudaStream_t stream);  // d_canon -> d_packed (+ bf16)

gf_status launch_flow_fp32(const gf_flow* f, bool inverse, const gf_phi4* phi4, int64_t B,
                           uint64_t seed, uint64_t counter0, const float* z_in, float* z_out,
                           const float* phi_in, float* phi_out, double* logq_out,
                           double* S_out, double* logw_out, cudaStream_t stream);
gf_status flow_fp32_configure(gf_flow* f);   // chooses FULL/RING, G, smem

// 3D L=16, hidden 32, FP32 (gf_flow_fp32_c32.cu)
bool fp32_c32_supported(const gf_flow* f);
// xs_out / logdet_out (training forward pass, nullable): the field after
// layers 1..N-1 at xs_out + layer * xs_stride + b * V, and the log-det.
gf_status launch_flow_fp32_c32(const gf_flow* f, bool inverse, const gf_phi4* phi4, int64_t B, uint64_t seed,
                               uint64_t counter0, const float* z_in, float* z_out, const float* phi_in,
                               float* phi_out, double* logq_out, double* S_out, double* logw_out,
                               cudaStream_t stream, float* xs_out = nullptr, int64_t xs_stride = 0,
                               double* logdet_out = nullptr);

// The training reverse pass's recompute of one layer's network (2D L=32,
// width 32): h1, h2 (chunk-major workspace layout) and s from x_l.
bool fp32_c32_recompute_supported(const gf_flow* f);
gf_status launch_c32_recompute(const gf_flow* f, int layer, int64_t B, const float* xl, float* h1_out, float* h2_out,
                               float* s_out, cudaStream_t stream);

// Polls of the failure-path test hook of the tensor-core kernels
// (gf_set_bf16_stall_test; 0 = off).
long long bf16_stall_spins();

// Tensor-core kernel for the shapes other than 3D L=16, C=32 (gf_flow_tc.cu)
bool tc_supported(const gf_flow_shape* s);
gf_status tc_configure(gf_flow* f);          // allocates the weight blocks
gf_status repack_tc(gf_flow* f, cudaStream_t stream);
gf_status launch_flow_tc(const gf_flow* f, bool inverse, const gf_phi4* phi4, int64_t B,
                         uint64_t seed, uint64_t counter0, const float* z_in, float* z_out,
                         const float* phi_in, float* phi_out, double* logq_out,
                         double* S_out, double* logw_out, cudaStream_t stream);

// General network (gf_flow_variant.cu)
gf_status variant_configure(gf_flow* f);     // packed offsets, smem, threads (host only)
gf_status repack_variant(gf_flow* f, cudaStream_t stream);
gf_status launch_flow_variant(const gf_flow* f, bool inverse, const gf_phi4* phi4, int64_t B,
                              uint64_t seed, uint64_t counter0, const float* z_in, float* z_out,
                              const float* phi_in, float* phi_out, double* logq_out,
                              double* S_out, double* logw_out, cudaStream_t stream);

}  // namespace gf
