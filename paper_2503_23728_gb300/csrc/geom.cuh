// geom.cuh -- device helpers shared by the descriptor and adjoint kernels:
// pair vectors under the minimum-image convention, the cosine cutoff and the
// Gaussian factors of the symmetry functions (internal).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace pimd {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
// Raise a kernel's dynamic shared-memory limit once (before any graph capture
// records the launch).
template <typename K>
inline void set_smem(K kernel, size_t bytes, size_t& done)
{
    if (bytes > done) {
        cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        done = bytes;
    }
}

// Gaussian factor exp(-eta x2). FAST (BF16 network path, whose tolerance is
// 1e-2): exp2(-(eta log2 e) x2) on the special-function unit; otherwise the
// accurate expf / exp.
template <bool FAST>
__device__ __forceinline__ float gauss(float eta, float eta_l2, float x2)
{
    if (FAST) return exp2f(-eta_l2 * x2);
    return expf(-eta * x2);
}
// The 32 radial Gaussians exp2(-eta' (r - r_mu)^2) of evenly spaced centres,
// in groups of 8: exact at the group's first centre, then g_(c+1) = g_c R_c
// with R_c = 2^(eta' (2 t_c dr - dr^2)) and R_(c+1) = R_c 2^(-2 eta' dr^2)
// (t_c = r - r_mu[c]; 2 exponentials and 14 products per group instead of 8
// exponentials; ~8 roundings of relative error). A group whose first value
// underflows (eta' t_0^2 > 149) leaves its members at 0 although the last
// one is 2^(-eta' (t_0 - 7 dr)^2); for the 32 centres over 0.5 .. 5.5 A that
// is below 2^-39 of the peak value 1.
template <typename DP>
__device__ __forceinline__ void radial_gauss32(const DP& dp, float r, float (&g)[32])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float t0 = r - dp.r_mu[8 * q];
        float e = exp2f(-dp.eta_R_l2 * t0 * t0);
        float R = exp2f(dp.eta_R_l2 * (2.0f * t0 * dp.r_delta - dp.r_delta * dp.r_delta));
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            g[8 * q + c] = e;
            e *= R;
            R *= dp.rec_k;
        }
    }
}

template <bool FAST>
__device__ __forceinline__ double gauss(double eta, double eta_l2, double x2)
{
    (void)eta_l2;
    return exp(-eta * x2);
}
__device__ __forceinline__ float f_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double f_sqrt(double v) { return sqrt(v); }

// Behler cosine cutoff fc(r) and its slope, from sincospi(r / rc)
__device__ __forceinline__ void cutoff(float r, float rc, float pi_over_rc, float& fc, float& dfc)
{
    if (r < rc) {
        float s, c;
        sincospif(r / rc, &s, &c);
        fc = 0.5f * (c + 1.0f);
        dfc = -0.5f * pi_over_rc * s;
    } else {
        fc = 0.0f;
        dfc = 0.0f;
    }
}
__device__ __forceinline__ void cutoff(double r, double rc, double pi_over_rc, double& fc, double& dfc)
{
    if (r < rc) {
        double s, c;
        sincospi(r / rc, &s, &c);
        fc = 0.5 * (c + 1.0);
        dfc = -0.5 * pi_over_rc * s;
    } else {
        fc = 0.0;
        dfc = 0.0;
    }
}

// Minimum-image pair vector x_j - x_i in the working precision. FP32: the
// difference is formed error-free (TwoSum: s + e = x_j - x_i exactly), shifted
// by k = rint(s / L) boxes (s - k L_hi is exact for |k| <= 1 by Sterbenz) and
// rounded once, so wrapped pairs are as accurate as unwrapped ones.
__device__ __forceinline__ float pair_axis(float xi, float xj, float L, float invL, float Llo, bool per)
{
    const float a = xj, b = -xi;
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    float e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
    float t = s;
    if (per) {
        const float k = rintf(__fmul_rn(s, invL));
        t = __fmaf_rn(-k, L, s);
        e = __fmaf_rn(-k, Llo, e);
    }
    return __fadd_rn(t, e);
}
template <typename V4>
__device__ __forceinline__ void pair_vec(const Rep& rp, const V4& xi, const V4& xj, float& dx, float& dy, float& dz)
{
    const bool per = rp.periodic != 0;
    dx = pair_axis(xi.x, xj.x, rp.Lf[0], rp.invLf[0], rp.Llo[0], per);
    dy = pair_axis(xi.y, xj.y, rp.Lf[1], rp.invLf[1], rp.Llo[1], per);
    dz = pair_axis(xi.z, xj.z, rp.Lf[2], rp.invLf[2], rp.Llo[2], per);
}
template <typename V4>
__device__ __forceinline__ void pair_vec(const Rep& rp, const V4& xi, const V4& xj, double& dx, double& dy,
                                         double& dz)
{
    dx = xj.x - xi.x;
    dy = xj.y - xi.y;
    dz = xj.z - xi.z;
    if (rp.periodic) {
        dx = __dsub_rn(dx, __dmul_rn(rp.L[0], rint(dx / rp.L[0])));
        dy = __dsub_rn(dy, __dmul_rn(rp.L[1], rint(dy / rp.L[1])));
        dz = __dsub_rn(dz, __dmul_rn(rp.L[2], rint(dz / rp.L[2])));
    }
}

// FP32 box of a replica in registers (invL = 0 for free clusters: no shift)
struct Box {
    float L[3], invL[3];
};
__device__ __forceinline__ Box box_of(const Rep& rp)
{
    Box b;
    for (int a = 0; a < 3; ++a) {
        b.L[a] = rp.Lf[a];
        b.invL[a] = rp.periodic ? rp.invLf[a] : 0.0f;
    }
    return b;
}
__device__ __forceinline__ float box_len(const Box& b, int a) { return b.L[a]; }
__device__ __forceinline__ float box_inv(const Box& b, int a) { return b.invL[a]; }
__device__ __forceinline__ float box_len(const Rep& r, int a) { return r.Lf[a]; }
__device__ __forceinline__ float box_inv(const Rep& r, int a) { return r.periodic ? r.invLf[a] : 0.0f; }

// BF16-path geometry of one neighbour (the path's bar is 1e-2 on the forces):
// minimum-image pair vector with one rounding per component, the distance
// and its inverse from the reciprocal square root, and the cutoff and its
// slope from the special-function sine and cosine of pi r / r_c (absolute
// error ~1e-6). The exact FP32 path keeps the error-free forms above.
// BX: Box (registers) or Rep (fields read where they are used)
template <typename BX>
__device__ __forceinline__ void geo_fast(const BX& bx, const float4& xi, const float4& xj, float rc,
                                         float pi_over_rc, float& dx, float& dy, float& dz, float& r, float& ir,
                                         float& fc, float& dfc)
{
    dx = xj.x - xi.x;
    dy = xj.y - xi.y;
    dz = xj.z - xi.z;
    dx = fmaf(-rintf(dx * box_inv(bx, 0)), box_len(bx, 0), dx);
    dy = fmaf(-rintf(dy * box_inv(bx, 1)), box_len(bx, 1), dy);
    dz = fmaf(-rintf(dz * box_inv(bx, 2)), box_len(bx, 2), dz);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    ir = rsqrtf(r2);
    r = r2 * ir;
    float s, c;
    __sincosf(r * pi_over_rc, &s, &c);
    const bool in = r < rc;
    fc = in ? fmaf(0.5f, c, 0.5f) : 0.0f;
    dfc = in ? -0.5f * pi_over_rc * s : 0.0f;
}

__device__ __forceinline__ float3 as_f32(const float4& v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 as_f32(const Dbl4& v)
{
    return make_float3(__double2float_rn(v.x), __double2float_rn(v.y), __double2float_rn(v.z));
}

template <typename V4, typename Real>
__device__ __forceinline__ V4 make4(Real a, Real b, Real c, Real d)
{
    V4 v;
    v.x = a; v.y = b; v.z = c; v.w = d;
    return v;
}

}  // namespace pimd
