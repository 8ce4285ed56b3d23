// Device math for the batched rigid-body step: float3 algebra, quaternions
// (x, y, z, w; Hamilton product), rotation matrices and symmetric 3x3
// inverse-inertia tensors.  FP32 throughout.
//
// The library is compiled with automatic multiply-add contraction off, and
// every fused multiply-add here is written out (fmaf).  The rounding of each
// operation is therefore fixed by this source, not by how the compiler
// inlines it into a kernel: the plain and batched kernels, and every launch
// shape, produce bit-identical results.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define MSD __device__ __forceinline__

MSD float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
MSD float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
MSD float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
MSD float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
MSD float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
// a + b * s, one rounding per component
MSD float3 madd(float3 a, float3 b, float s) { return f3(fmaf(b.x, s, a.x), fmaf(b.y, s, a.y), fmaf(b.z, s, a.z)); }
MSD float dot(float3 a, float3 b) { return fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)); }
MSD float3 cross(float3 a, float3 b) {
    return f3(fmaf(a.y, b.z, -(a.z * b.y)), fmaf(a.z, b.x, -(a.x * b.z)), fmaf(a.x, b.y, -(a.y * b.x)));
}
MSD float len(float3 a) { return sqrtf(dot(a, a)); }
MSD float comp(float3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
MSD float3 axis3(int i) { return f3(i == 0 ? 1.f : 0.f, i == 1 ? 1.f : 0.f, i == 2 ? 1.f : 0.f); }
MSD float3 with_comp(float3 a, int i, float s) {
    if (i == 0) a.x = s; else if (i == 1) a.y = s; else a.z = s;
    return a;
}
MSD float clampf(float x, float lo, float hi) { return x < lo ? lo : (x > hi ? hi : x); }
MSD float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }
MSD float4 f4(float3 a, float w) { return make_float4(a.x, a.y, a.z, w); }

MSD float4 qmul(float4 a, float4 b) {
    // (a_v, a_w)(b_v, b_w) = (a_w b_v + b_w a_v + a_v x b_v, a_w b_w - a_v.b_v)
    float3 av = xyz(a), bv = xyz(b);
    float3 c = cross(av, bv);
    float3 r = f3(fmaf(a.w, bv.x, fmaf(b.w, av.x, c.x)), fmaf(a.w, bv.y, fmaf(b.w, av.y, c.y)),
                  fmaf(a.w, bv.z, fmaf(b.w, av.z, c.z)));
    return make_float4(r.x, r.y, r.z, fmaf(a.w, b.w, -dot(av, bv)));
}
MSD float4 qconj(float4 a) { return make_float4(-a.x, -a.y, -a.z, a.w); }
MSD float4 qnormalize(float4 a) {
    float n = sqrtf(fmaf(a.w, a.w, fmaf(a.z, a.z, fmaf(a.y, a.y, a.x * a.x))));
    return make_float4(a.x / n, a.y / n, a.z / n, a.w / n);
}

// rotation matrix of a unit quaternion, row major
struct M3 { float m[9]; };
MSD M3 qmat(float4 q) {
    M3 R;
    float x = q.x, y = q.y, z = q.z, w = q.w;
    float xx = x * x, yy = y * y, zz = z * z;
    R.m[0] = 1.f - 2.f * (yy + zz); R.m[1] = 2.f * fmaf(x, y, -(z * w)); R.m[2] = 2.f * fmaf(x, z, y * w);
    R.m[3] = 2.f * fmaf(x, y, z * w); R.m[4] = 1.f - 2.f * (xx + zz); R.m[5] = 2.f * fmaf(y, z, -(x * w));
    R.m[6] = 2.f * fmaf(x, z, -(y * w)); R.m[7] = 2.f * fmaf(y, z, x * w); R.m[8] = 1.f - 2.f * (xx + yy);
    return R;
}
MSD float3 mv(const M3& R, float3 a) {
    return f3(fmaf(R.m[2], a.z, fmaf(R.m[1], a.y, R.m[0] * a.x)),
              fmaf(R.m[5], a.z, fmaf(R.m[4], a.y, R.m[3] * a.x)),
              fmaf(R.m[8], a.z, fmaf(R.m[7], a.y, R.m[6] * a.x)));
}
MSD float3 mtv(const M3& R, float3 a) {
    return f3(fmaf(R.m[6], a.z, fmaf(R.m[3], a.y, R.m[0] * a.x)),
              fmaf(R.m[7], a.z, fmaf(R.m[4], a.y, R.m[1] * a.x)),
              fmaf(R.m[8], a.z, fmaf(R.m[5], a.y, R.m[2] * a.x)));
}
MSD float3 mcol(const M3& R, int j) { return f3(R.m[j], R.m[3 + j], R.m[6 + j]); }
MSD float3 qrot(float4 q, float3 a) { M3 R = qmat(q); return mv(R, a); }

// symmetric 3x3 stored (xx, xy, xz, yy, yz, zz)
struct S3 { float xx, xy, xz, yy, yz, zz; };
MSD float3 smv(const S3& I, float3 v) {
    return f3(fmaf(I.xz, v.z, fmaf(I.xy, v.y, I.xx * v.x)),
              fmaf(I.yz, v.z, fmaf(I.yy, v.y, I.xy * v.x)),
              fmaf(I.zz, v.z, fmaf(I.yz, v.y, I.xz * v.x)));
}
// R diag(d) R^T
MSD S3 rdrt(const M3& R, float3 d) {
    float dd[3] = {d.x, d.y, d.z};
    float o[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            float acc = (R.m[3 * i] * dd[0]) * R.m[3 * j];
            acc = fmaf(R.m[3 * i + 1] * dd[1], R.m[3 * j + 1], acc);
            acc = fmaf(R.m[3 * i + 2] * dd[2], R.m[3 * j + 2], acc);
            o[3 * i + j] = acc;
        }
    S3 s;
    s.xx = o[0]; s.xy = o[1]; s.xz = o[2]; s.yy = o[4]; s.yz = o[5]; s.zz = o[8];
    return s;
}

// Axis used to build a basis orthogonal to a unit vector: the first index
// whose |component| is within 0.1 of the smallest one.  Near a coordinate
// axis it never flips between nearly equal tiny components; for a vector in
// a coordinate plane it picks the axis normal to that plane.
MSD int basis_axis(float3 a) {
    float c0 = fabsf(a.x), c1 = fabsf(a.y), c2 = fabsf(a.z);
    float mn = fminf(c0, fminf(c1, c2));
    if (c0 <= mn + 0.1f) return 0;
    if (c1 <= mn + 0.1f) return 1;
    return 2;
}

// wrap an angle in [-2 pi, 2 pi] (twice an atan2) to (-pi, pi]
MSD float wrap_pi(float x) {
    const float PI = 3.14159265358979323846f;
    if (x > PI) x -= 2.f * PI;
    if (x <= -PI) x += 2.f * PI;
    return x;
}
