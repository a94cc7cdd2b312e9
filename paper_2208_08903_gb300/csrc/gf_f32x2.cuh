// gf_f32x2.cuh -- packed FP32 pairs (two FP32 lanes in one 64-bit register)
// for the sm_100+ fma.rn.f32x2 instruction.  One packed FMA does the work of
// two FP32 FMAs in one issue slot; the FP32 pipe's FLOP rate is the same, so
// FMA-dominated kernels that are short of issue slots gain.  Each lane rounds
// exactly like fmaf (round to nearest even), so results are bit-identical.
#pragma once

#include <cstdint>

namespace gf {

typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 f2_make(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f32x2 f2_splat(float v) { return f2_make(v, v); }
__device__ __forceinline__ float f2_lo(f32x2 v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2_hi(f32x2 v) { return __uint_as_float((uint32_t)(v >> 32)); }
// a * b + c in both lanes
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

}  // namespace gf
