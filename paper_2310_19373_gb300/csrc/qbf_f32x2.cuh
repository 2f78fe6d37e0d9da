// qbf_f32x2.cuh -- packed FP32 helpers of the FP32-pipe walks: a 64-bit
// register holds two FP32 values (lo, hi) that one add.rn.f32x2 moves
// together.  All values the walks keep are integers below 2^24 in magnitude,
// so every add is exact.
#pragma once

namespace qbf {
namespace f32x2 {

typedef unsigned long long u64;

__device__ __forceinline__ u64 add(u64 a, u64 b)
{
    u64 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ u64 sub(u64 a, u64 b)
{
    u64 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ u64 pack(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack(u64 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ float min3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ u64 splat(float k) { return pack(k, k); }

}  // namespace f32x2
}  // namespace qbf
