// gf_api.cu -- C-ABI entry points of the flow object (create / destroy /
// weights / sample / logq / status), the slice schedule builder and the
// weight repacking kernel.  Declarations and contracts: include/gfflow.h.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "gf_flow.cuh"

namespace gf {

namespace {
__device__ int32_t g_status = 0;
__device__ int32_t g_status_read = 0;     // gf_device_status's copy of the exchanged word

std::mutex g_slot_mu;
std::unordered_map<cudaStream_t, int32_t*> g_stream_slot;   // gf_set_stream_status_slot
std::mutex g_read_mu;                                        // one gf_device_status at a time

__global__ void status_exchange_kernel(int32_t* word, int32_t* out) {
    *out = atomicExch(reinterpret_cast<int*>(word), 0);
}
}  // namespace

int32_t* status_word() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
    return static_cast<int32_t*>(p);
}

int32_t* status_word(cudaStream_t stream) {
    {
        std::lock_guard<std::mutex> lk(g_slot_mu);
        auto it = g_stream_slot.find(stream);
        if (it != g_stream_slot.end()) return it->second;
    }
    return status_word();
}

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

PackedOffsets packed_offsets(int T, int C1, int C2) {
    PackedOffsets o;
    o.W1 = 0;
    o.b1 = o.W1 + (int64_t)T * C1;
    o.W2 = o.b1 + C1;
    o.b2 = o.W2 + (int64_t)T * C1 * C2;
    o.W3 = o.b2 + C2;
    o.b3 = o.W3 + (int64_t)T * C2 * 2;
    o.stride = (o.b3 + 2 + 7) & ~int64_t(7);   // 32-byte aligned layer blocks
    return o;
}

// ---------------------------------------------------------------------------
// Slice schedule (see gf_flow.cuh).
// ---------------------------------------------------------------------------
namespace {

struct SlotCache {
    std::vector<int> slice;   // slice held by each slot, -1 = empty
    std::vector<long> used;   // last-use tick
    long tick = 0;
    explicit SlotCache(int R) : slice(R, -1), used(R, -1) {}
    int find(int s) const {
        for (size_t i = 0; i < slice.size(); ++i) if (slice[i] == s) return (int)i;
        return -1;
    }
    void touch(int slot) { used[slot] = ++tick; }
    // slot for a new slice, never evicting a slice listed in `keep`
    int alloc(int s, const std::vector<int>& keep) {
        int best = -1;
        for (size_t i = 0; i < slice.size(); ++i) {
            if (slice[i] >= 0 && std::find(keep.begin(), keep.end(), slice[i]) != keep.end()) continue;
            if (best < 0 || slice[i] < 0 && slice[best] >= 0 ||
                ((slice[i] < 0) == (slice[best] < 0) && used[i] < used[best]))
                best = (int)i;
        }
        if (best >= 0) { slice[best] = s; touch(best); }
        return best;
    }
};

int wrapL(int v, int L) { return ((v % L) + L) % L; }

}  // namespace

std::vector<Phase> build_schedule(int L, int G, bool full) {
    std::vector<Phase> out;
    auto blank = [](int type, int s0, int n) {
        Phase p;
        std::memset(&p, 0, sizeof(p));
        p.type = (uint8_t)type; p.s0 = (uint16_t)s0; p.n = (uint8_t)n;
        return p;
    };
    if (full) {
        Phase h1 = blank(PH_H1, 0, L), h2 = blank(PH_H2, 0, L), c3 = blank(PH_C3, 0, L);
        for (int r = 0; r < L; ++r) { h1.out[r] = h2.out[r] = (uint8_t)r; }
        for (int r = 0; r < L + 2; ++r) h2.in[r] = c3.in[r] = (uint8_t)wrapL(r - 1, L);
        out.push_back(h1); out.push_back(h2); out.push_back(c3);
        return out;
    }
    const int R = G + 2;
    SlotCache c1(R), c2(R);
    for (int a = 0; a < L; a += G) {
        const int n = std::min(G, L - a);
        std::vector<int> need2;
        for (int s = a - 1; s <= a + n; ++s) need2.push_back(wrapL(s, L));
        std::vector<int> miss2;
        for (int s : need2) if (c2.find(s) < 0) miss2.push_back(s);
        // runs of at most G consecutive slices (miss2 is consecutive mod L)
        for (size_t i0 = 0; i0 < miss2.size(); i0 += G) {
            const int m = (int)std::min<size_t>(G, miss2.size() - i0);
            const int r0 = miss2[i0];
            std::vector<int> need1;
            for (int s = r0 - 1; s <= r0 + m; ++s) need1.push_back(wrapL(s, L));
            std::vector<int> miss1;
            for (int s : need1) if (c1.find(s) < 0) miss1.push_back(s);
            for (size_t k0 = 0; k0 < miss1.size(); k0 += G) {
                const int mm = (int)std::min<size_t>(G, miss1.size() - k0);
                Phase p = blank(PH_H1, miss1[k0], mm);
                for (int q = 0; q < mm; ++q) p.out[q] = (uint8_t)c1.alloc(miss1[k0 + q], need1);
                out.push_back(p);
            }
            Phase p = blank(PH_H2, r0, m);
            for (int q = 0; q < m + 2; ++q) {
                const int slot = c1.find(need1[q]);
                c1.touch(slot);
                p.in[q] = (uint8_t)slot;
            }
            for (int q = 0; q < m; ++q) p.out[q] = (uint8_t)c2.alloc(wrapL(r0 + q, L), need2);
            out.push_back(p);
        }
        Phase p = blank(PH_C3, a, n);
        for (int q = 0; q < n + 2; ++q) {
            const int slot = c2.find(need2[q]);
            c2.touch(slot);
            p.in[q] = (uint8_t)slot;
        }
        out.push_back(p);
    }
    return out;
}

// ---------------------------------------------------------------------------
// Canonical FP32 [layer][W1 b1 W2 b2 W3 b3] -> packed per-layer layouts.
// ---------------------------------------------------------------------------
__global__ void repack_kernel(const float* __restrict__ canon, float* __restrict__ packed,
                              int n_layers, int T, int C1, int C2, int64_t cstride,
                              PackedOffsets o) {
    const int64_t total = (int64_t)n_layers * cstride;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / cstride);
        int64_t r = i - l * cstride;
        float* P = packed + l * o.stride;
        const float v = canon[i];
        if (r < (int64_t)C1 * T) {                       // W1[c][0][t]
            const int c = (int)(r / T), t = (int)(r % T);
            P[o.W1 + t * C1 + c] = v; continue;
        }
        r -= (int64_t)C1 * T;
        if (r < C1) { P[o.b1 + r] = v; continue; }
        r -= C1;
        if (r < (int64_t)C2 * C1 * T) {                  // W2[o][i][t]
            const int oc = (int)(r / ((int64_t)C1 * T));
            const int ic = (int)((r / T) % C1), t = (int)(r % T);
            P[o.W2 + ((int64_t)t * C1 + ic) * C2 + oc] = v; continue;
        }
        r -= (int64_t)C2 * C1 * T;
        if (r < C2) { P[o.b2 + r] = v; continue; }
        r -= C2;
        if (r < (int64_t)2 * C2 * T) {                   // W3[o][i][t]
            const int oc = (int)(r / ((int64_t)C2 * T));
            const int ic = (int)((r / T) % C2), t = (int)(r % T);
            P[o.W3 + ((int64_t)t * C2 + ic) * 2 + oc] = v; continue;
        }
        r -= (int64_t)2 * C2 * T;
        P[o.b3 + r] = v;
    }
}

gf_status repack_bf16(gf_flow* f, cudaStream_t stream);   // gf_flow_bf16.cu

gf_status repack_weights(gf_flow* f, cudaStream_t stream) {
    const PackedOffsets o = packed_offsets(f->T, f->C1, f->C2);
    const int64_t total = f->n_params;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 4096);
    repack_kernel<<<grid, 256, 0, stream>>>(f->d_canon, f->d_packed, f->shape.n_layers, f->T,
                                            f->C1, f->C2, f->canon_stride, o);
    GF_CHECK_LAUNCH();
    if (f->prec == GF_PREC_BF16CONV_FP64RED) return f->tc ? repack_tc(f, stream) : repack_bf16(f, stream);
    return GF_OK;
}

bool bf16_supported(const gf_flow_shape* s);          // gf_flow_bf16.cu
gf_status bf16_configure(gf_flow* f);                 // gf_flow_bf16.cu
gf_status launch_flow_bf16(const gf_flow* f, bool inverse, const gf_phi4* phi4, int64_t B,
                           uint64_t seed, uint64_t counter0, const float* z_in, float* z_out,
                           const float* phi_in, float* phi_out, double* logq_out,
                           double* S_out, double* logw_out, cudaStream_t stream);

}  // namespace gf

using namespace gf;

namespace {

bool shape_ex_valid(const gf_flow_shape_ex* s) {
    if (!s) return false;
    if (s->nd != 2 && s->nd != 3) return false;
    if (s->ksize < 1 || s->ksize > 7 || (s->ksize & 1) == 0) return false;
    if (s->L < 2 || (s->L & 1)) return false;
    int64_t V = 1;
    for (int i = 0; i < s->nd; ++i) V *= s->L;
    if (V > 65536) return false;
    if (s->n_layers < 0 || s->n_layers > 4096) return false;
    if (s->n_hidden < 0 || s->n_hidden > GF_MAX_HIDDEN) return false;
    for (int j = 0; j < s->n_hidden; ++j)
        if (s->hidden[j] < 1 || s->hidden[j] > 256) return false;
    if (!(s->leaky_slope == s->leaky_slope)) return false;
    return true;
}

// The paper's example network form on the slice-cached kernels: two equal
// hidden widths in {8, 16, 24, 32}, 3 taps per axis.
bool default_net(const gf_flow_shape_ex* s) {
    if (s->n_hidden != 2 || s->ksize != 3 || s->hidden[0] != s->hidden[1]) return false;
    const int c = s->hidden[0];
    return c == 8 || c == 16 || c == 24 || c == 32;
}

void free_flow(gf_flow* f) {
    if (!f) return;
    cudaFree(f->d_vpacked);
    cudaFree(f->d_canon);
    cudaFree(f->d_packed);
    cudaFree(f->d_sched);
    cudaFree(f->d_bf16);
    for (cudaEvent_t e : f->ev_fork)
        if (e) cudaEventDestroy(e);
    if (f->ev_join) cudaEventDestroy(f->ev_join);
    if (f->side) cudaStreamDestroy(f->side);
    delete f;
}

}  // namespace

extern "C" {

const char* gf_status_string(int32_t s) {
    switch (s) {
        case GF_OK: return "GF_OK";
        case GF_EINVAL: return "GF_EINVAL";
        case GF_ENOMEM: return "GF_ENOMEM";
        case GF_ECUDA: return "GF_ECUDA";
        case GF_EUNSUPPORTED: return "GF_EUNSUPPORTED";
        case GF_ETIMEOUT: return "GF_ETIMEOUT";
        case GF_EDEVICE: return "GF_EDEVICE";
        default: return "GF_UNKNOWN";
    }
}

gf_status gf_flow_create(const gf_flow_shape* shape, const double* weights_host,
                         gf_precision prec, cudaStream_t stream, gf_flow** out) {
    if (!shape) return GF_EINVAL;
    gf_flow_shape_ex ex;
    std::memset(&ex, 0, sizeof(ex));
    ex.nd = shape->nd;
    ex.L = shape->L;
    ex.n_layers = shape->n_layers;
    ex.n_hidden = 2;
    ex.hidden[0] = shape->c_hidden1;
    ex.hidden[1] = shape->c_hidden2;
    ex.ksize = shape->ksize;
    ex.use_final_tanh = shape->use_final_tanh;
    ex.leaky_slope = shape->leaky_slope;
    return gf_flow_create_ex(&ex, weights_host, prec, stream, out);
}

gf_status gf_flow_create_ex(const gf_flow_shape_ex* shape, const double* weights_host,
                            gf_precision prec, cudaStream_t stream, gf_flow** out) {
    if (!out || !weights_host || !shape_ex_valid(shape)) return GF_EINVAL;
    if (prec != GF_PREC_FP32 && prec != GF_PREC_BF16CONV_FP64RED) return GF_EINVAL;
    const bool dflt = default_net(shape);
    gf_flow_shape legacy;
    std::memset(&legacy, 0, sizeof(legacy));
    legacy.nd = shape->nd;
    legacy.L = shape->L;
    legacy.n_layers = shape->n_layers;
    legacy.c_hidden1 = shape->n_hidden > 0 ? shape->hidden[0] : 0;
    legacy.c_hidden2 = shape->n_hidden > 1 ? shape->hidden[1] : 0;
    legacy.ksize = shape->ksize;
    legacy.use_final_tanh = shape->use_final_tanh;
    legacy.leaky_slope = shape->leaky_slope;
    if (prec == GF_PREC_BF16CONV_FP64RED && (!dflt || !(bf16_supported(&legacy) || tc_supported(&legacy))))
        return GF_EUNSUPPORTED;

    gf_flow* f = new gf_flow;
    std::memset(f, 0, sizeof(*f));
    f->shape = legacy;
    f->prec = prec;
    cudaGetDevice(&f->device);
    f->V = 1;
    for (int i = 0; i < shape->nd; ++i) f->V *= shape->L;
    f->S = f->V / shape->L;
    f->K = shape->ksize;
    f->T = 1;
    for (int i = 0; i < shape->nd; ++i) f->T *= f->K;
    f->n_hidden = shape->n_hidden;
    for (int j = 0; j < shape->n_hidden; ++j) f->hidden[j] = shape->hidden[j];
    f->variant = !dflt;
    gf_status st;
    if (f->variant) {
        f->canon_stride = 0;
        for (int j = 0; j <= f->n_hidden; ++j) {
            const int64_t ci = j == 0 ? 1 : f->hidden[j - 1], co = j == f->n_hidden ? 2 : f->hidden[j];
            f->canon_stride += co * ci * f->T + co;
        }
        f->n_params = f->canon_stride * shape->n_layers;
        st = variant_configure(f);
        if (st != GF_OK) { free_flow(f); return st; }
        std::vector<float> w32((size_t)std::max<int64_t>(f->n_params, 1));
        for (int64_t i = 0; i < f->n_params; ++i) w32[i] = (float)weights_host[i];
        const size_t pbytes = sizeof(float) * (size_t)std::max<int64_t>(1, f->vstride * shape->n_layers);
        if (cudaMalloc(&f->d_canon, sizeof(float) * w32.size()) != cudaSuccess ||
            cudaMalloc(&f->d_vpacked, pbytes) != cudaSuccess) {
            free_flow(f);
            return GF_ENOMEM;
        }
        if (cudaMemcpyAsync(f->d_canon, w32.data(), sizeof(float) * w32.size(), cudaMemcpyHostToDevice,
                            stream) != cudaSuccess ||
            cudaMemsetAsync(f->d_vpacked, 0, pbytes, stream) != cudaSuccess) {
            free_flow(f);
            return GF_ECUDA;
        }
        st = repack_variant(f, stream);
        if (st != GF_OK) { free_flow(f); return st; }
        if (cudaStreamSynchronize(stream) != cudaSuccess) { free_flow(f); return GF_ECUDA; }
        *out = f;
        return GF_OK;
    }

    f->C1 = shape->hidden[0];
    f->C2 = shape->hidden[1];
    f->canon_stride = (int64_t)f->C1 * f->T + f->C1 + (int64_t)f->C2 * f->C1 * f->T + f->C2 +
                      2LL * f->C2 * f->T + 2;
    f->n_params = f->canon_stride * shape->n_layers;
    f->packed_stride = packed_offsets(f->T, f->C1, f->C2).stride;

    st = flow_fp32_configure(f);
    if (st != GF_OK) { free_flow(f); return st; }
    if (prec == GF_PREC_BF16CONV_FP64RED) {
        st = bf16_supported(&f->shape) ? bf16_configure(f) : tc_configure(f);
        if (st != GF_OK) { free_flow(f); return st; }
    }
    std::vector<Phase> sched = build_schedule(shape->L, f->G, f->full);
    f->n_phases = (int)sched.size();

    std::vector<float> w32((size_t)std::max<int64_t>(f->n_params, 1));
    for (int64_t i = 0; i < f->n_params; ++i) w32[i] = (float)weights_host[i];

    // side stream and events of the training reverse pass
    if (cudaStreamCreateWithFlags(&f->side, cudaStreamNonBlocking) != cudaSuccess) { free_flow(f); return GF_ECUDA; }
    for (cudaEvent_t& e : f->ev_fork)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { free_flow(f); return GF_ECUDA; }
    if (cudaEventCreateWithFlags(&f->ev_join, cudaEventDisableTiming) != cudaSuccess) { free_flow(f); return GF_ECUDA; }
    if (cudaMalloc(&f->d_canon, sizeof(float) * w32.size()) != cudaSuccess ||
        cudaMalloc(&f->d_packed, sizeof(float) * std::max<int64_t>(1, f->packed_stride * shape->n_layers)) != cudaSuccess ||
        cudaMalloc(&f->d_sched, sizeof(Phase) * sched.size()) != cudaSuccess) {
        free_flow(f);
        return GF_ENOMEM;
    }
    if (cudaMemcpyAsync(f->d_canon, w32.data(), sizeof(float) * w32.size(),
                        cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(f->d_sched, sched.data(), sizeof(Phase) * sched.size(),
                        cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemsetAsync(f->d_packed, 0, sizeof(float) * std::max<int64_t>(1, f->packed_stride * shape->n_layers),
                        stream) != cudaSuccess) {
        free_flow(f);
        return GF_ECUDA;
    }
    if (f->n_params > 0) {
        st = repack_weights(f, stream);
        if (st != GF_OK) { free_flow(f); return st; }
    }
    if (cudaStreamSynchronize(stream) != cudaSuccess) { free_flow(f); return GF_ECUDA; }
    *out = f;
    return GF_OK;
}

int32_t gf_flow_tensor_core_supported(const gf_flow_shape_ex* shape) {
    if (!shape_ex_valid(shape) || !default_net(shape)) return 0;
    gf_flow_shape s;
    std::memset(&s, 0, sizeof(s));
    s.nd = shape->nd;
    s.L = shape->L;
    s.n_layers = shape->n_layers;
    s.c_hidden1 = shape->hidden[0];
    s.c_hidden2 = shape->hidden[1];
    s.ksize = shape->ksize;
    s.use_final_tanh = shape->use_final_tanh;
    s.leaky_slope = shape->leaky_slope;
    return (bf16_supported(&s) || tc_supported(&s)) ? 1 : 0;
}

gf_status gf_flow_destroy(gf_flow* flow) {
    if (!flow) return GF_EINVAL;
    free_flow(flow);
    return GF_OK;
}

int64_t gf_flow_n_params(const gf_flow* flow) { return flow ? flow->n_params : -1; }

gf_status gf_flow_set_weights_device(gf_flow* flow, const float* d_weights, cudaStream_t stream) {
    if (!flow || !d_weights) return GF_EINVAL;
    if (flow->n_params == 0) return GF_OK;
    if (cudaMemcpyAsync(flow->d_canon, d_weights, sizeof(float) * flow->n_params,
                        cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
        return GF_ECUDA;
    if (flow->variant) return repack_variant(flow, stream);
    return repack_weights(flow, stream);
}

gf_status gf_flow_get_weights_device(const gf_flow* flow, float* d_weights_out, cudaStream_t stream) {
    if (!flow || !d_weights_out) return GF_EINVAL;
    if (flow->n_params == 0) return GF_OK;
    if (cudaMemcpyAsync(d_weights_out, flow->d_canon, sizeof(float) * flow->n_params,
                        cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
        return GF_ECUDA;
    return GF_OK;
}

gf_status gf_flow_sample(const gf_flow* flow, const gf_phi4* phi4, int64_t B,
                         uint64_t seed, uint64_t counter0, const float* d_z_in,
                         float* d_z_out, float* d_phi_out, double* d_logq_out,
                         double* d_S_out, double* d_logw_out, cudaStream_t stream) {
    if (!flow || B < 0 || (B > 0 && (!d_phi_out || !d_logq_out))) return GF_EINVAL;
    if (!phi4 && (d_S_out || d_logw_out)) return GF_EINVAL;
    if (B == 0) return GF_OK;
    if (flow->variant)
        return launch_flow_variant(flow, false, phi4, B, seed, counter0, d_z_in, d_z_out, nullptr,
                                   d_phi_out, d_logq_out, d_S_out, d_logw_out, stream);
    if (flow->prec == GF_PREC_BF16CONV_FP64RED && flow->tc)
        return launch_flow_tc(flow, false, phi4, B, seed, counter0, d_z_in, d_z_out, nullptr,
                              d_phi_out, d_logq_out, d_S_out, d_logw_out, stream);
    if (flow->prec == GF_PREC_BF16CONV_FP64RED)
        return launch_flow_bf16(flow, false, phi4, B, seed, counter0, d_z_in, d_z_out, nullptr,
                                d_phi_out, d_logq_out, d_S_out, d_logw_out, stream);
    return launch_flow_fp32(flow, false, phi4, B, seed, counter0, d_z_in, d_z_out, nullptr,
                            d_phi_out, d_logq_out, d_S_out, d_logw_out, stream);
}

gf_status gf_flow_logq(const gf_flow* flow, int64_t B, const float* d_phi_in,
                       float* d_z_out, double* d_logq_out, cudaStream_t stream) {
    if (!flow || B < 0 || (B > 0 && (!d_phi_in || !d_logq_out))) return GF_EINVAL;
    if (B == 0) return GF_OK;
    if (flow->variant)
        return launch_flow_variant(flow, true, nullptr, B, 0, 0, nullptr, d_z_out, d_phi_in, nullptr,
                                   d_logq_out, nullptr, nullptr, stream);
    if (flow->prec == GF_PREC_BF16CONV_FP64RED && flow->tc)
        return launch_flow_tc(flow, true, nullptr, B, 0, 0, nullptr, d_z_out, d_phi_in, nullptr,
                              d_logq_out, nullptr, nullptr, stream);
    if (flow->prec == GF_PREC_BF16CONV_FP64RED)
        return launch_flow_bf16(flow, true, nullptr, B, 0, 0, nullptr, d_z_out, d_phi_in, nullptr,
                                d_logq_out, nullptr, nullptr, stream);
    return launch_flow_fp32(flow, true, nullptr, B, 0, 0, nullptr, d_z_out, d_phi_in, nullptr,
                            d_logq_out, nullptr, nullptr, stream);
}

gf_status gf_device_status(cudaStream_t stream, int32_t* status_out) {
    if (!status_out) return GF_EINVAL;
    std::lock_guard<std::mutex> lk(g_read_mu);
    int32_t* word = status_word(stream);
    void* outp = nullptr;
    if (!word || cudaGetSymbolAddress(&outp, g_status_read) != cudaSuccess) return GF_ECUDA;
    // read and clear in one atomic exchange on the device, after the stream's work
    status_exchange_kernel<<<1, 1, 0, stream>>>(word, static_cast<int32_t*>(outp));
    if (cudaGetLastError() != cudaSuccess) return GF_ECUDA;
    int32_t v = 0;
    if (cudaMemcpyAsync(&v, outp, sizeof(v), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return GF_ECUDA;
    *status_out = v;
    return GF_OK;
}

gf_status gf_set_stream_status_slot(cudaStream_t stream, int32_t* d_slot) {
    std::lock_guard<std::mutex> lk(g_slot_mu);
    if (d_slot) g_stream_slot[stream] = d_slot;
    else g_stream_slot.erase(stream);
    return GF_OK;
}

}  // extern "C"
