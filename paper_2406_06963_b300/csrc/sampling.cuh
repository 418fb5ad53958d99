// Ray-direction sampling on the device (Section 3.1 cone-jittered shadow
// rays, Section 3.2 cosine-weighted AO rays).
//
// Every floating-point operation here is an explicitly rounded intrinsic
// (__fmul_rn, __fadd_rn, __fdiv_rn, __fsqrt_rn), so that no multiply-add
// contraction happens and each written operation rounds once in binary32.
// The sequence of operations is a written specification that an
// independent host implementation can follow to get identical bits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dhr {

// pcg4d: Jarzynski & Olano, "Hash Functions for GPU Rendering", JCGT 2020.
__device__ __forceinline__ uint4 pcg4d(uint4 v) {
    v.x = v.x * 1664525u + 1013904223u;
    v.y = v.y * 1664525u + 1013904223u;
    v.z = v.z * 1664525u + 1013904223u;
    v.w = v.w * 1664525u + 1013904223u;
    v.x += v.y * v.w;
    v.y += v.z * v.x;
    v.z += v.x * v.y;
    v.w += v.y * v.z;
    v.x ^= v.x >> 16;
    v.y ^= v.y >> 16;
    v.z ^= v.z >> 16;
    v.w ^= v.w >> 16;
    v.x += v.y * v.w;
    v.y += v.z * v.x;
    v.z += v.x * v.y;
    v.w += v.y * v.z;
    return v;
}

// top 24 bits -> exact float in [0, 1)
__device__ __forceinline__ float unit24(uint32_t h) {
    return __uint2float_rn(h >> 8) * (1.0f / 16777216.0f);
}

enum RayType : uint32_t { kShadowRay = 0u, kAoRay = 1u };

// Uniform point on the unit disk by rejection.  Input words of call c:
// (px, py, frame ^ seed, type << 24 | (sample & 0xFFFF) << 8 | c); each call
// gives candidates (u0, u1) and (u2, u3), x = 2u - 1 (exact); accepted when
// x*x + y*y < 1 in binary32; after 8 rejections the centre is used.
__device__ __forceinline__ float2 disk_point(uint32_t px, uint32_t py, uint32_t frame, uint32_t seed,
                                             uint32_t type, uint32_t sample) {
    const uint32_t stream = (type << 24) | ((sample & 0xFFFFu) << 8);
#pragma unroll 1
    for (uint32_t call = 0; call < 4; ++call) {
        uint4 h = pcg4d(make_uint4(px, py, frame ^ seed, stream | call));
        float x = __fsub_rn(__fmul_rn(2.0f, unit24(h.x)), 1.0f);
        float y = __fsub_rn(__fmul_rn(2.0f, unit24(h.y)), 1.0f);
        if (__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)) < 1.0f) return make_float2(x, y);
        x = __fsub_rn(__fmul_rn(2.0f, unit24(h.z)), 1.0f);
        y = __fsub_rn(__fmul_rn(2.0f, unit24(h.w)), 1.0f);
        if (__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)) < 1.0f) return make_float2(x, y);
    }
    return make_float2(0.0f, 0.0f);
}

// Branch-free orthonormal basis (T, B) around unit n: Duff et al.,
// "Building an Orthonormal Basis, Revisited", JCGT 2017.
__device__ __forceinline__ void onb(float3 n, float3& T, float3& B) {
    const float sgn = copysignf(1.0f, n.z);
    const float a = __fdiv_rn(-1.0f, __fadd_rn(sgn, n.z));
    const float b = __fmul_rn(__fmul_rn(n.x, n.y), a);
    T = make_float3(__fadd_rn(1.0f, __fmul_rn(__fmul_rn(__fmul_rn(sgn, n.x), n.x), a)),
                    __fmul_rn(sgn, b), -__fmul_rn(sgn, n.x));
    B = make_float3(b, __fadd_rn(sgn, __fmul_rn(__fmul_rn(n.y, n.y), a)), -n.y);
}

// Cosine-weighted direction about n (Malley): d = (x T + y B) + z n with
// z = sqrt(max(0, 1 - (x*x + y*y))).
__device__ __forceinline__ float3 ao_direction(float3 n, float2 xy) {
    float3 T, B;
    onb(n, T, B);
    const float s = __fadd_rn(__fmul_rn(xy.x, xy.x), __fmul_rn(xy.y, xy.y));
    const float z = __fsqrt_rn(fmaxf(__fsub_rn(1.0f, s), 0.0f));
    return make_float3(
        __fadd_rn(__fadd_rn(__fmul_rn(xy.x, T.x), __fmul_rn(xy.y, B.x)), __fmul_rn(z, n.x)),
        __fadd_rn(__fadd_rn(__fmul_rn(xy.x, T.y), __fmul_rn(xy.y, B.y)), __fmul_rn(z, n.y)),
        __fadd_rn(__fadd_rn(__fmul_rn(xy.x, T.z), __fmul_rn(xy.y, B.z)), __fmul_rn(z, n.z)));
}

// Direction toward a directional light jittered inside its cone (tangent
// disk form): q = l + tan_theta (x T_l + y B_l), d = q / |q|, where
// |q| = sqrt((qx*qx + qy*qy) + qz*qz).
__device__ __forceinline__ float3 cone_direction(float3 l, float tan_theta, float2 xy) {
    float3 T, B;
    onb(l, T, B);
    const float3 q = make_float3(
        __fadd_rn(l.x, __fmul_rn(tan_theta, __fadd_rn(__fmul_rn(xy.x, T.x), __fmul_rn(xy.y, B.x)))),
        __fadd_rn(l.y, __fmul_rn(tan_theta, __fadd_rn(__fmul_rn(xy.x, T.y), __fmul_rn(xy.y, B.y)))),
        __fadd_rn(l.z, __fmul_rn(tan_theta, __fadd_rn(__fmul_rn(xy.x, T.z), __fmul_rn(xy.y, B.z)))));
    const float len = __fsqrt_rn(
        __fadd_rn(__fadd_rn(__fmul_rn(q.x, q.x), __fmul_rn(q.y, q.y)), __fmul_rn(q.z, q.z)));
    return make_float3(__fdiv_rn(q.x, len), __fdiv_rn(q.y, len), __fdiv_rn(q.z, len));
}

}  // namespace dhr
