// lat_pairs.cuh -- two-site arithmetic for the step kernels. FP32 sites travel
// as packed f32x2 register pairs so that one add/sub/mul/fma instruction of the
// sm_100 family updates two lattice sites; FP64 uses two scalar doubles.
#pragma once

#include <cuda_runtime.h>

namespace lat {

struct F2 {
    unsigned long long v;
};
struct D2 {
    double x, y;
};
__device__ __forceinline__ F2 mk2(float lo, float hi)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void un2(F2 a, float& lo, float& hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v)); }
__device__ __forceinline__ float lo2(F2 a) { float l, h; un2(a, l, h); return l; }
__device__ __forceinline__ float hi2(F2 a) { float l, h; un2(a, l, h); return h; }
__device__ __forceinline__ F2 add2(F2 a, F2 b) { F2 r; asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v)); return r; }
__device__ __forceinline__ F2 sub2(F2 a, F2 b) { F2 r; asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v)); return r; }
__device__ __forceinline__ F2 mul2(F2 a, F2 b) { F2 r; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v)); return r; }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c)
{
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ D2 mk2(double lo, double hi) { return D2{lo, hi}; }
__device__ __forceinline__ double lo2(D2 a) { return a.x; }
__device__ __forceinline__ double hi2(D2 a) { return a.y; }
__device__ __forceinline__ D2 add2(D2 a, D2 b) { return D2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ D2 sub2(D2 a, D2 b) { return D2{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ D2 mul2(D2 a, D2 b) { return D2{a.x * b.x, a.y * b.y}; }
__device__ __forceinline__ D2 fma2(D2 a, D2 b, D2 c) { return D2{fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)}; }

// A 16-byte vector of one row: NP pairs (4 floats or 2 doubles).
template <typename T>
struct PK;
template <>
struct PK<float> {
    typedef F2 P;
    static constexpr int NP = 2;
    static __device__ __forceinline__ void ld(const void* p, P (&v)[2])
    {
        const ulonglong2 q = *reinterpret_cast<const ulonglong2*>(p);
        v[0].v = q.x; v[1].v = q.y;
    }
    static __device__ __forceinline__ void st(void* p, const P (&v)[2])
    {
        *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(v[0].v, v[1].v);
    }
    // a global store not read again soon: evict first from the caches
    static __device__ __forceinline__ void st_stream(void* p, const P (&v)[2])
    {
        __stcs(reinterpret_cast<ulonglong2*>(p), make_ulonglong2(v[0].v, v[1].v));
    }
};
template <>
struct PK<double> {
    typedef D2 P;
    static constexpr int NP = 1;
    static __device__ __forceinline__ void ld(const void* p, P (&v)[1])
    {
        const double2 q = *reinterpret_cast<const double2*>(p);
        v[0].x = q.x; v[0].y = q.y;
    }
    static __device__ __forceinline__ void st(void* p, const P (&v)[1])
    {
        *reinterpret_cast<double2*>(p) = make_double2(v[0].x, v[0].y);
    }
    static __device__ __forceinline__ void st_stream(void* p, const P (&v)[1])
    {
        __stcs(reinterpret_cast<double2*>(p), make_double2(v[0].x, v[0].y));
    }
};

} // namespace lat
