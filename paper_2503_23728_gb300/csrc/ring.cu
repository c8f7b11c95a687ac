// ring.cu -- FP64 ring-polymer kernels: initial state, normal-mode <-> bead
// transforms, the OBABO step in normal-mode space (exact free-ring-polymer A,
// PILE-L O with Philox4x32-10 noise), and the finite-P estimators.
//
// Work decomposition: a block owns T = blockDim / P (atom, dimension)
// entries of one replica and all P modes of each, so every P-point transform
// is a shared-memory matrix-vector product spread over T * P threads.
#include <cuda_runtime.h>
#include <cstdint>

#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace pimd {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 multiplies
// with Weyl key increments; one standard normal per counter by Box-Muller on
// two 53-bit uniforms in (0, 1].
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ double normal_dev(unsigned long long seed, unsigned idx, unsigned step, unsigned rep,
                                             unsigned stream)
{
    const uint4 w = philox10(make_uint4(idx, step, rep, stream), make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
    const double u1 = ((double)(w.x >> 5) * 67108864.0 + (double)(w.y >> 6) + 1.0) * (1.0 / 9007199254740992.0);
    const double u2 = ((double)(w.z >> 5) * 67108864.0 + (double)(w.w >> 6) + 1.0) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// FP32 paths: the same deviate from the same counter with FP32 arithmetic.
// The first uniform is the 53-bit one rounded to FP32 (not truncated, so the
// log keeps its relative accuracy down to u1 ~ 2^-29); log, cos and sqrt
// in FP32 (deviates within ~1e-7 relative of the FP64 ones). FP64 runs at a
// small fraction of the FP32 rate on this GPU, and the FP32 force path's own
// rounding is larger than this.
__device__ __forceinline__ float normal_dev_f(unsigned long long seed, unsigned idx, unsigned step, unsigned rep,
                                              unsigned stream)
{
    const uint4 w = philox10(make_uint4(idx, step, rep, stream), make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
    const float u1 = fmaf(__uint2float_rn(w.x >> 5), 7.450580596923828125e-9f,              // 2^-27
                          __uint2float_rn((w.y >> 6) + 1u) * 1.1102230246251565e-16f);   // 2^-53
    const float u2 = fmaf(__uint2float_rn(w.z >> 5), 7.450580596923828125e-9f,
                          __uint2float_rn((w.w >> 6) + 1u) * 1.1102230246251565e-16f);
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// bead coordinate j from the ring-polymer coordinates of one (atom, dim):
// FP64 paths sum all P terms in FP64; FP32 paths keep the mode-0 term (the
// absolute position) in FP64 and sum the other modes, deviations of tenths of
// an Angstrom, in FP32 (rounding far below one FP32 ulp of the position)
template <typename Real>
__device__ __forceinline__ double to_bead(const double* __restrict__ C, const float* Cf,
                                          const double* sq, const float* sqf, int P, int stride)
{
    if constexpr (std::is_same<Real, float>::value) {
        float a = 0.0f;
        if ((P & 3) == 0 && (reinterpret_cast<uintptr_t>(Cf) & 15) == 0) {
            // the row as 16-byte loads (a quarter of the load instructions),
            // the same order of multiply-adds
            const float4* C4 = reinterpret_cast<const float4*>(Cf);
            for (int k4 = 0; k4 < (P >> 2); ++k4) {
                const float4 c = __ldg(C4 + k4);
                const float* q = sqf + (size_t)(4 * k4) * stride;
                if (k4 > 0) a = fmaf(c.x, q[0], a);
                a = fmaf(c.y, q[stride], a);
                a = fmaf(c.z, q[2 * stride], a);
                a = fmaf(c.w, q[3 * stride], a);
            }
        } else {
            for (int k = 1; k < P; ++k) a = fmaf(Cf[k], sqf[k * stride], a);
        }
        return fma(C[0], sq[0], (double)a);
    }
    double acc = 0.0;
    for (int k = 0; k < P; ++k) acc = fma(C[k], sq[k * stride], acc);
    return acc;
}

// FP32 transform staged per block in shared memory ([P][P + 1], the padding
// keeps the rows a warp touches in distinct banks) when P is at most
// RP_STAGE_P; larger P read the global copy. Returns the rows to use. The
// ring finish stages it (a thread reads a column); the ring start reads its
// row from global memory (one row per thread, cached), which measured faster
// than staging there.
constexpr int RP_STAGE_P = 64;

__device__ __forceinline__ const float* stage_cmatf(const float* __restrict__ cmatf, int P, float* buf, int& ld)
{
    if (P > RP_STAGE_P) {
        ld = P;
        return cmatf;
    }
    ld = P + 1;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        const int j = e / P;
        buf[j * (P + 1) + (e - j * P)] = cmatf[e];
    }
    return buf;   // visible after the caller's next __syncthreads
}

template <typename Real>
__device__ __forceinline__ Real& comp(Vec4<Real>& v, int d)
{
    return reinterpret_cast<Real*>(&v)[d];
}

// ---------------------------------------------------------------------------
// initial state: q_nm(k=0) = sqrt(P) x0, other modes 0; p_nm ~ N(0, m k_B T_P)
// with Philox stream 1, step 0. One thread per state entry.
// ---------------------------------------------------------------------------
__global__ void rp_init_kernel(const Rep* __restrict__ reps, const BeadSys* __restrict__ bsys,
                               const int* __restrict__ ba_sys, const Mode* __restrict__ modes,
                               const double* __restrict__ mass,
                               const double* __restrict__ x0, int B, double* __restrict__ q, double* __restrict__ p)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 3 * B) return;
    const int b = g / 3, dd = g - 3 * b;
    const BeadSys sy = bsys[ba_sys[b]];
    const Rep& rp = reps[sy.rep];
    const int i = b - sy.ba0;
    const int k = sy.bead;
    const unsigned local = (unsigned)((k * rp.noise_N + rp.noise_atom0 + i) * 3 + dd);
    const Mode md = modes[rp.mode0 + k];
    const double m = mass[rp.atom0 + i] * md.mfac;
    // all beads at x0: q_0 = P x0 / (column sum of mode 0), other modes 0
    q[g] = (k == 0) ? (double)rp.P / md.cs * x0[3 * (size_t)(rp.atom0 + i) + dd] : 0.0;
    p[g] = sqrt(m * rp.kT_md) * normal_dev(rp.seed, local, 0u, (unsigned)sy.rep, 1u);
}

void launch_rp_init(const Dev& d, cudaStream_t st)
{
    rp_init_kernel<<<(3 * d.B + 255) / 256, 256, 0, st>>>(d.reps, d.bsys, d.ba_sys, d.modes, d.mass, d.x0, d.B, d.q,
                                                          d.p);
}

// ---------------------------------------------------------------------------
// block geometry: block -> (replica, first of T entries); thread -> (mode kk,
// entry le) with the entry fastest, so that a warp touches consecutive
// entries of one mode: the state [mode][atom][dim] and the bead records are
// read and written in contiguous runs. Per-entry vectors over the modes sit
// in shared memory as [mode][entry] (index kk * T + le).
// ---------------------------------------------------------------------------
struct RpThread {
    int r, e, kk, le, T, N, P, i, dd;
    bool active;
};

__device__ __forceinline__ RpThread rp_thread(const int2* __restrict__ blocks, const Rep* __restrict__ reps)
{
    RpThread t;
    const int2 bl = blocks[blockIdx.x];
    t.r = bl.x;
    const Rep& rp = reps[t.r];
    t.N = rp.N;
    t.P = rp.P;
    t.T = blockDim.x / t.P;
    t.kk = threadIdx.x / t.T;
    t.le = threadIdx.x - t.kk * t.T;
    t.e = bl.y + t.le;
    t.active = t.kk < t.P && t.e < 3 * t.N;
    t.i = t.e / 3;
    t.dd = t.e - 3 * t.i;
    return t;
}

// normal-mode -> bead positions for all beads (no dynamics)
template <typename Real>
__global__ void beads_kernel(const int2* __restrict__ blocks, const Rep* __restrict__ reps,
                             const double* __restrict__ cmat, const float* __restrict__ cmatf,
                             const double* __restrict__ q, Vec4<Real>* __restrict__ x)
{
    extern __shared__ double sq[];
    float* sqf = reinterpret_cast<float*>(sq + blockDim.x);
    const RpThread t = rp_thread(blocks, reps);
    const Rep& rp = reps[t.r];
    if (t.active) {
        const double qv = q[3 * ((size_t)rp.ba0 + (size_t)t.kk * t.N + t.i) + t.dd];
        sq[t.kk * t.T + t.le] = qv;
        sqf[t.kk * t.T + t.le] = (float)qv;
    }
    __syncthreads();
    if (!t.active) return;
    const int j = t.kk;
    const double acc = to_bead<Real>(cmat + rp.cmat + (size_t)j * t.P, cmatf + rp.cmat + (size_t)j * t.P,
                                     sq + t.le, sqf + t.le, t.P, t.T);
    comp<Real>(x[rp.ba0 + (size_t)j * t.N + t.i], t.dd) = (Real)acc;
}

// free ring-polymer step of mode k over hA: centroid drift, or the rotation
// (cw, sw) of the scaled phase plane that the host computed for the chosen
// propagator (exact or Cayley)
// (m: the coordinate's mass, im: its inverse)
__device__ __forceinline__ void free_rp(int k, const Mode& md, double m, double im, double hA, double& pv,
                                        double& qv)
{
    // explicit roundings, so that every kernel that takes this step (ring
    // start, fused ring finish + start) produces the same bits
    if (k == 0) {
        qv = fma(__dmul_rn(pv, hA), im, qv);
    } else {
        const double pn = fma(md.cw, pv, -__dmul_rn(__dmul_rn(m, md.wsw), qv));
        qv = fma(__dmul_rn(md.sw_w, im), pv, __dmul_rn(md.cw, qv));
        pv = pn;
    }
}

// PILE-L O sub-step with the host's (c1, c2) for its duration; returns the
// kinetic-energy change (smkT = sqrt(m k_B T_P) of the coordinate, im = 1/m).
// The momentum update is FP64 on every path. The FP32 paths form the heat
// increment and its block sums in FP32 (this GPU runs FP64 at 2 lanes per SM
// per clock): with a = sigma xi the noise kick, pn - pv = (c1 - 1) pv + a and
// pn + pv = (c1 + 1) pv + a, each term of which is FP32-accurate.
template <typename Real>
using HeatT = typename std::conditional<std::is_same<Real, float>::value, float, double>::type;

template <typename Real>
__device__ __forceinline__ HeatT<Real> pile_o(const Rep& rp, const Mode& md, double smkT, double im, unsigned local,
                                              unsigned step, unsigned rep, unsigned stream, double& pv)
{
    if constexpr (std::is_same<Real, float>::value) {
        const float xi = normal_dev_f(rp.seed, local, step, rep, stream);
        const double sig = __dmul_rn(smkT, md.c2);
        const double pn = fma(md.c1, pv, __dmul_rn(sig, (double)xi));
        const float pvf = (float)pv, a = (float)sig * xi;
        const float dK = 0.5f * (float)im * (fmaf(md.c1m1, pvf, a) * fmaf(md.c1p1, pvf, a));
        pv = pn;
        return dK;
    } else {
        const double xi = normal_dev(rp.seed, local, step, rep, stream);
        const double pn = fma(md.c1, pv, __dmul_rn(__dmul_rn(smkT, md.c2), xi));
        const double dK = __dmul_rn(__dmul_rn(fma(pn, pn, -__dmul_rn(pv, pv)), 0.5), im);
        pv = pn;
        return dK;
    }
}

// OBABO: O(dt/2) B(dt/2) A(dt); BAOAB: B(dt/2) A(dt/2) O(dt) A(dt/2); on each
// mode, then the new bead positions
template <typename Real>
__global__ void __launch_bounds__(256, std::is_same<Real, float>::value ? 5 : 4) rp_start_kernel(const int2* __restrict__ blocks, const Rep* __restrict__ reps,
                                const double* __restrict__ cmat, const float* __restrict__ cmatf,
                                const Mode* __restrict__ modes,
                                const double* __restrict__ mass, const double2* __restrict__ minv,
                                const unsigned long long* __restrict__ stepp, double hdt, double kick, int unit_mfac, int thermostat, int baoab, double* __restrict__ q, double* __restrict__ p,
                                const double* __restrict__ fnm, Vec4<Real>* __restrict__ x,
                                double* __restrict__ qlo, Vec4<Real>* __restrict__ f, double* __restrict__ W,
                                double* __restrict__ V, double* __restrict__ Q, int ordered_heat,
                                unsigned long long* __restrict__ stepc)
{
    extern __shared__ double sq[];
    float* sqf = reinterpret_cast<float*>(sq + blockDim.x);
    __shared__ double red[32];
    const RpThread t = rp_thread(blocks, reps);
    const Rep& rp = reps[t.r];
    HeatT<Real> dK = 0;
    if (t.active) {
        const int k = t.kk;
        const size_t g = 3 * ((size_t)rp.ba0 + (size_t)k * t.N + t.i) + t.dd;
        const Mode md = modes[rp.mode0 + k];
        const double2 mi = minv[rp.atom0 + t.i];
        // mass factors of the ring coordinate (all 1 for normal modes)
        const double ma = mass[rp.atom0 + t.i];
        const double m = unit_mfac ? ma : ma * md.mfac, im = unit_mfac ? mi.x : mi.x * md.imf,
                     smkT = unit_mfac ? mi.y : mi.y * md.smf;
        double pv = p[g], qv = q[g];
        const unsigned local = (unsigned)((k * rp.noise_N + rp.noise_atom0 + t.i) * 3 + t.dd);
        if (baoab) {
            pv = fma(kick, fnm[g], pv);   // B: one rounding, as in the fused boundary kernel
            free_rp(k, md, m, im, hdt, pv, qv);
            if (thermostat) dK = pile_o<Real>(rp, md, smkT, im, local, (unsigned)(*stepp), (unsigned)t.r, 2u, pv);
            free_rp(k, md, m, im, hdt, pv, qv);
        } else {
            if (thermostat) dK = pile_o<Real>(rp, md, smkT, im, local, (unsigned)(*stepp), (unsigned)t.r, 2u, pv);
            pv = fma(kick, fnm[g], pv);   // B: one rounding, as in the fused boundary kernel
            free_rp(k, md, m, im, 2.0 * hdt, pv, qv);
        }
        p[g] = pv;
        q[g] = qv;
        sq[k * t.T + t.le] = qv;
        sqf[k * t.T + t.le] = (float)qv;
    }
    // thermostat heat: block partial, summed per replica in block order later
    dK = warp_sum(dK);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)dK;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        s = thermostat ? s * MVV2E : 0.0;
        qlo[blockIdx.x] = s;
        if (!ordered_heat && thermostat) atomicAdd(&Q[t.r], s);
        if (blockIdx.x == 0) *stepc = *stepp;   // the step the ring finish will read
    }
    if (!t.active) return;
    const int j = t.kk;
    const double acc = to_bead<Real>(cmat + rp.cmat + (size_t)j * t.P, cmatf + rp.cmat + (size_t)j * t.P,
                                     sq + t.le, sqf + t.le, t.P, t.T);
    comp<Real>(x[rp.ba0 + (size_t)j * t.N + t.i], t.dd) = (Real)acc;
    // clear the force record of this bead-atom and, once per bead, its virial
    // and energy, for the force evaluation that follows
    if (t.dd == 0) {
        Vec4<Real> z;
        z.x = z.y = z.z = z.w = (Real)0;
        f[rp.ba0 + (size_t)j * t.N + t.i] = z;
        if (t.i == 0) {
            const int bs = rp.bs0 + j;
#pragma unroll
            for (int a = 0; a < 9; ++a) W[(size_t)bs * 9 + a] = 0.0;
            V[bs] = 0.0;
        }
    }
}

// f_nm = C^T f; if do_step: B(dt/2), then O(dt/2) for OBABO, and the step
// ends here: block 0 advances the step counter that the next ring start
// reads (this kernel reads the copy that the ring start made, plus offset:
// the steps of a multi-step launch since that ring start), and each block
// adds its thermostat heat to Q (FP64 atomics) unless the heat is summed in
// a fixed order afterwards (deterministic mode).
template <typename Real>
__global__ void rp_finish_kernel(const int2* __restrict__ blocks, const Rep* __restrict__ reps,
                                 const double* __restrict__ cmat, const float* __restrict__ cmatf,
                                 const Mode* __restrict__ modes,
                                 const double* __restrict__ mass, const double2* __restrict__ minv,
                                 const unsigned long long* stepp, int offset, double kick, int unit_mfac, int thermostat, int do_step, const Vec4<Real>* __restrict__ f,
                                 double* __restrict__ p, double* __restrict__ fnm, double* __restrict__ qhi,
                                 DevErr* __restrict__ err, double* __restrict__ Q, int ordered_heat,
                                 unsigned long long* stepw)
{
    extern __shared__ double sf[];
    float* sff = reinterpret_cast<float*>(sf + blockDim.x);
    __shared__ double red[32];
    const RpThread t = rp_thread(blocks, reps);
    const Rep& rp = reps[t.r];
    int ldc = t.P;
    const float* Cfs = cmatf + rp.cmat;
    if constexpr (std::is_same<Real, float>::value) Cfs = stage_cmatf(Cfs, t.P, sff + blockDim.x, ldc);
    if (t.active) {
        const Vec4<Real> fv = f[rp.ba0 + (size_t)t.kk * t.N + t.i];
        const Real fc = t.dd == 0 ? fv.x : (t.dd == 1 ? fv.y : fv.z);   // selects, no local array
        if constexpr (std::is_same<Real, float>::value)
            sff[t.kk * t.T + t.le] = fc;
        else
            sf[t.kk * t.T + t.le] = (double)fc;
    }
    __syncthreads();
    HeatT<Real> dK = 0;
    if (t.active) {
        const int k = t.kk;
        double fn = 0.0;
        if constexpr (std::is_same<Real, float>::value) {
            // FP32 forces: their normal-mode components summed in FP32
            float a = 0.0f;
            for (int j = 0; j < t.P; ++j) a = fmaf(Cfs[j * ldc + k], sff[j * t.T + t.le], a);
            fn = (double)a;
        } else {
            for (int j = 0; j < t.P; ++j) fn = fma(cmat[rp.cmat + (size_t)j * t.P + k], sf[j * t.T + t.le], fn);
        }
        const size_t g = 3 * ((size_t)rp.ba0 + (size_t)k * t.N + t.i) + t.dd;
        fnm[g] = fn;
        if (!isfinite(fn)) atomicOr(&err->flags, ERR_NONFINITE);
        if (do_step) {
            const Mode md = modes[rp.mode0 + k];
            const double2 mi = minv[rp.atom0 + t.i];
            double pv = fma(kick, fn, p[g]);
            if (thermostat) {
                const unsigned local = (unsigned)((k * rp.noise_N + rp.noise_atom0 + t.i) * 3 + t.dd);
                const double smkT = unit_mfac ? mi.y : mi.y * md.smf, im = unit_mfac ? mi.x : mi.x * md.imf;
                dK = pile_o<Real>(rp, md, smkT, im, local, (unsigned)(*stepp + (unsigned long long)offset), (unsigned)t.r,
                                  3u, pv);
            }
            p[g] = pv;
        }
    }
    dK = warp_sum(dK);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)dK;
    __syncthreads();
    if (!do_step) return;   // block-uniform
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        s = thermostat ? s * MVV2E : 0.0;
        qhi[blockIdx.x] = s;
        if (!ordered_heat && thermostat) atomicAdd(&Q[t.r], s);
        if (blockIdx.x == 0) *stepw = *stepp + (unsigned long long)offset + 1ull;   // no block of this kernel reads stepw
    }
}

// deterministic mode: thermostat heat of both O halves added per replica in a
// fixed order (one block per replica) after the ring finish
__global__ void heat_sum_kernel(double* __restrict__ Q, const double* __restrict__ qlo,
                                const double* __restrict__ qhi, const int* __restrict__ rep_blk0)
{
    __shared__ double red[8];
    const int r = blockIdx.x;
    double s = 0.0;
    for (int b = rep_blk0[r] + threadIdx.x; b < rep_blk0[r + 1]; b += blockDim.x) s += qlo[b] + qhi[b];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        Q[r] += t;
    }
}

// Inside a multi-step launch, the ring finish of step j and the ring start
// of step j + 1 (nothing runs between them) as one kernel: every coordinate
// does the finish's f_nm = C^T f, B(dt/2) and (OBABO) O(dt/2), then the
// start's O / B / A in the same registers, with the same operations in the
// same order as the two kernels, so the state is bit-identical. Noise
// counters: the call's first ring start copied the step counter to stepc;
// this boundary ends step stepc + offset. The heat of the finish half goes
// to qhi, that of the start half to qlo (the other lo half than the one the
// step being finished used, for the ordered sums).
template <typename Real>
__global__ void __launch_bounds__(256, 4) rp_finish_start_kernel(
    const int2* __restrict__ blocks, const Rep* __restrict__ reps, const double* __restrict__ cmat,
    const float* __restrict__ cmatf, const Mode* __restrict__ modes, const double* __restrict__ mass,
    const double2* __restrict__ minv, const unsigned long long* __restrict__ stepc, int offset, double hdt,
    double kick, int unit_mfac, int thermostat, int baoab, double* __restrict__ q, double* __restrict__ p,
    double* __restrict__ fnm, Vec4<Real>* __restrict__ x, Vec4<Real>* __restrict__ f, double* __restrict__ W,
    double* __restrict__ V, double* __restrict__ qhi, double* __restrict__ qlo, DevErr* __restrict__ err,
    double* __restrict__ Q, int ordered_heat)
{
    extern __shared__ double sbuf[];   // forces, then positions: [T P] doubles, [T P] floats, staged C
    double* sv = sbuf;
    float* svf = reinterpret_cast<float*>(sbuf + blockDim.x);
    __shared__ double red[2][32];
    const RpThread t = rp_thread(blocks, reps);
    const Rep& rp = reps[t.r];
    int ldc = t.P;
    const float* Cfs = cmatf + rp.cmat;
    if constexpr (std::is_same<Real, float>::value) Cfs = stage_cmatf(Cfs, t.P, svf + blockDim.x, ldc);
    if (t.active) {
        const Vec4<Real> fv = f[rp.ba0 + (size_t)t.kk * t.N + t.i];
        const Real fc = t.dd == 0 ? fv.x : (t.dd == 1 ? fv.y : fv.z);
        if constexpr (std::is_same<Real, float>::value)
            svf[t.kk * t.T + t.le] = fc;
        else
            sv[t.kk * t.T + t.le] = (double)fc;
    }
    __syncthreads();
    HeatT<Real> dK1 = 0, dK2 = 0;
    double qv = 0.0;
    const unsigned long long s0 = *stepc + (unsigned long long)offset;
    if (t.active) {
        const int k = t.kk;
        double fn = 0.0;
        if constexpr (std::is_same<Real, float>::value) {
            float a = 0.0f;
            for (int j = 0; j < t.P; ++j) a = fmaf(Cfs[j * ldc + k], svf[j * t.T + t.le], a);
            fn = (double)a;
        } else {
            for (int j = 0; j < t.P; ++j) fn = fma(cmat[rp.cmat + (size_t)j * t.P + k], sv[j * t.T + t.le], fn);
        }
        const size_t g = 3 * ((size_t)rp.ba0 + (size_t)k * t.N + t.i) + t.dd;
        fnm[g] = fn;
        if (!isfinite(fn)) atomicOr(&err->flags, ERR_NONFINITE);
        const Mode md = modes[rp.mode0 + k];
        const double2 mi = minv[rp.atom0 + t.i];
        const double ma = mass[rp.atom0 + t.i];
        const double m = unit_mfac ? ma : ma * md.mfac, im = unit_mfac ? mi.x : mi.x * md.imf,
                     smkT = unit_mfac ? mi.y : mi.y * md.smf;
        const unsigned local = (unsigned)((k * rp.noise_N + rp.noise_atom0 + t.i) * 3 + t.dd);
        // the finish of step s0: B(dt/2), then O(dt/2) for OBABO
        double pv = fma(kick, fn, p[g]);
        if (thermostat && !baoab) dK1 = pile_o<Real>(rp, md, smkT, im, local, (unsigned)s0, (unsigned)t.r, 3u, pv);
        // the start of step s0 + 1
        qv = q[g];
        const unsigned s1 = (unsigned)(s0 + 1ull);
        if (baoab) {
            pv = fma(kick, fn, pv);
            free_rp(k, md, m, im, hdt, pv, qv);
            if (thermostat) dK2 = pile_o<Real>(rp, md, smkT, im, local, s1, (unsigned)t.r, 2u, pv);
            free_rp(k, md, m, im, hdt, pv, qv);
        } else {
            if (thermostat) dK2 = pile_o<Real>(rp, md, smkT, im, local, s1, (unsigned)t.r, 2u, pv);
            pv = fma(kick, fn, pv);
            free_rp(k, md, m, im, 2.0 * hdt, pv, qv);
        }
        p[g] = pv;
        q[g] = qv;
    }
    dK1 = warp_sum(dK1);
    dK2 = warp_sum(dK2);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = (double)dK1;
        red[1][threadIdx.x >> 5] = (double)dK2;
    }
    __syncthreads();   // the forces in shared memory are read; the positions may overwrite them
    if (t.active) {
        sv[t.kk * t.T + t.le] = qv;
        svf[t.kk * t.T + t.le] = (float)qv;
    }
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        a = (thermostat && !baoab) ? a * MVV2E : 0.0;
        b = thermostat ? b * MVV2E : 0.0;
        qhi[blockIdx.x] = a;
        qlo[blockIdx.x] = b;
        if (!ordered_heat && thermostat) {
            if (!baoab) atomicAdd(&Q[t.r], a);
            atomicAdd(&Q[t.r], b);
        }
    }
    __syncthreads();
    if (!t.active) return;
    const int j = t.kk;
    const double acc = to_bead<Real>(cmat + rp.cmat + (size_t)j * t.P, cmatf + rp.cmat + (size_t)j * t.P,
                                     sv + t.le, svf + t.le, t.P, t.T);
    comp<Real>(x[rp.ba0 + (size_t)j * t.N + t.i], t.dd) = (Real)acc;
    if (t.dd == 0) {
        Vec4<Real> z;
        z.x = z.y = z.z = z.w = (Real)0;
        f[rp.ba0 + (size_t)j * t.N + t.i] = z;
        if (t.i == 0) {
            const int bs = rp.bs0 + j;
#pragma unroll
            for (int a = 0; a < 9; ++a) W[(size_t)bs * 9 + a] = 0.0;
            V[bs] = 0.0;
        }
    }
}

// heat partials: [lo 0][hi][lo 1], each n_rp_blocks. A ring start writes a
// lo half (the start of step j of a multi-step launch writes lo (j & 1)), the
// ring finish the hi half; the ordered sum after a finish adds the lo half of
// the same step.
static double* heat_lo(const Dev& d, int lo) { return d.qpart + (size_t)(lo ? 2 : 0) * d.n_rp_blocks; }
static double* heat_hi(const Dev& d) { return d.qpart + (size_t)d.n_rp_blocks; }

void launch_heat_sum(const Dev& d, int lo, cudaStream_t st)
{
    heat_sum_kernel<<<d.R, 256, 0, st>>>(d.Q, heat_lo(d, lo), heat_hi(d), d.rep_blk0);
}

static size_t rp_smem(const Dev& d) { return (size_t)d.rp_threads * (sizeof(double) + sizeof(float)); }

// ring finish: the per-entry vectors plus, on the FP32 paths, the staged
// transform of the largest P <= RP_STAGE_P among the replicas
static size_t rp_step_smem(const Dev& d)
{
    const size_t stage = d.precision == 0 ? 0 : (size_t)d.rp_stage_P * (d.rp_stage_P + 1) * sizeof(float);
    return rp_smem(d) + stage;
}

void launch_beads(const Dev& d, cudaStream_t st)
{
    if (d.precision == 0)
        beads_kernel<double><<<d.n_rp_blocks, d.rp_threads, rp_smem(d), st>>>(d.rp_blocks, d.reps, d.cmat, d.cmatf, d.q,
                                                                                (Dbl4*)d.x);
    else
        beads_kernel<float><<<d.n_rp_blocks, d.rp_threads, rp_smem(d), st>>>(d.rp_blocks, d.reps, d.cmat, d.cmatf, d.q,
                                                                               (float4*)d.x);
}

void launch_rp_start(const Dev& d, cudaStream_t st, int lo)
{
    if (d.precision == 0)
        rp_start_kernel<double><<<d.n_rp_blocks, d.rp_threads, rp_smem(d), st>>>(
            d.rp_blocks, d.reps, d.cmat, d.cmatf, d.modes, d.mass, d.minv, d.step, 0.5 * d.dt, 0.5 * d.dt * INV_MVV2E, d.unit_mfac, d.thermostat, d.splitting, d.q, d.p, d.fnm,
            (Dbl4*)d.x, heat_lo(d, lo), (Dbl4*)d.f, d.W, d.V, d.Q, d.deterministic, d.step_cur);
    else
        rp_start_kernel<float><<<d.n_rp_blocks, d.rp_threads, rp_smem(d), st>>>(
            d.rp_blocks, d.reps, d.cmat, d.cmatf, d.modes, d.mass, d.minv, d.step, 0.5 * d.dt, 0.5 * d.dt * INV_MVV2E, d.unit_mfac, d.thermostat, d.splitting, d.q, d.p, d.fnm,
            (float4*)d.x, heat_lo(d, lo), (float4*)d.f, d.W, d.V, d.Q, d.deterministic, d.step_cur);
}

void launch_rp_finish(const Dev& d, bool do_step, cudaStream_t st, int offset)
{
    if (d.precision == 0)
        rp_finish_kernel<double><<<d.n_rp_blocks, d.rp_threads, rp_step_smem(d), st>>>(
            d.rp_blocks, d.reps, d.cmat, d.cmatf, d.modes, d.mass, d.minv, d.step_cur, offset, 0.5 * d.dt * INV_MVV2E, d.unit_mfac, d.thermostat && !d.splitting,
            do_step ? 1 : 0, (const Dbl4*)d.f, d.p, d.fnm, heat_hi(d), d.err, d.Q, d.deterministic, d.step);
    else
        rp_finish_kernel<float><<<d.n_rp_blocks, d.rp_threads, rp_step_smem(d), st>>>(
            d.rp_blocks, d.reps, d.cmat, d.cmatf, d.modes, d.mass, d.minv, d.step_cur, offset, 0.5 * d.dt * INV_MVV2E, d.unit_mfac, d.thermostat && !d.splitting,
            do_step ? 1 : 0, (const float4*)d.f, d.p, d.fnm, heat_hi(d), d.err, d.Q, d.deterministic, d.step);
}

void launch_rp_finish_start(const Dev& d, int offset, int lo, cudaStream_t st)
{
    if (d.precision == 0)
        rp_finish_start_kernel<double><<<d.n_rp_blocks, d.rp_threads, rp_step_smem(d), st>>>(
            d.rp_blocks, d.reps, d.cmat, d.cmatf, d.modes, d.mass, d.minv, d.step_cur, offset, 0.5 * d.dt,
            0.5 * d.dt * INV_MVV2E, d.unit_mfac, d.thermostat, d.splitting, d.q, d.p, d.fnm, (Dbl4*)d.x, (Dbl4*)d.f,
            d.W, d.V, heat_hi(d), heat_lo(d, lo), d.err, d.Q, d.deterministic);
    else
        rp_finish_start_kernel<float><<<d.n_rp_blocks, d.rp_threads, rp_step_smem(d), st>>>(
            d.rp_blocks, d.reps, d.cmat, d.cmatf, d.modes, d.mass, d.minv, d.step_cur, offset, 0.5 * d.dt,
            0.5 * d.dt * INV_MVV2E, d.unit_mfac, d.thermostat, d.splitting, d.q, d.p, d.fnm, (float4*)d.x,
            (float4*)d.f, d.W, d.V, heat_hi(d), heat_lo(d, lo), d.err, d.Q, d.deterministic);
}


// ---------------------------------------------------------------------------
// a8: estimators in normal-mode space, one block per replica (FP64).
//   spring = sum_k 1/2 m omega_k^2 q_k^2     (= bead-space spring energy)
//   sum_k (x_k - centroid) . f_k = sum_{k>0} q_k f_nm,k
//   kinetic = sum p^2 / 2m
// record: V_mean K_prim K_cv E_tot W[9] H_cons Q_thermo T_kin nbr_mean nbr_max
// ---------------------------------------------------------------------------
__global__ void estimators_kernel(const Rep* __restrict__ reps, const Mode* __restrict__ modes,
                                  const double* __restrict__ mass, const double* __restrict__ q,
                                  const double* __restrict__ p, const double* __restrict__ fnm,
                                  const double* __restrict__ V, const double* __restrict__ Wv,
                                  const double* __restrict__ Q, const int* __restrict__ nnb,
                                  double* __restrict__ est)
{
    __shared__ double red[4][32];
    __shared__ int redm[32];
    const int r = blockIdx.x;
    const Rep& rp = reps[r];
    const int N = rp.N, P = rp.P;
    double spring = 0.0, cv = 0.0, kin = 0.0, nsum = 0.0;
    int nmax = 0;
    // per (atom, dimension): spring sum_k 1/2 m_k w_k^2 q_k^2, kinetic
    // sum_k p_k^2 / 2 m_k, and sum_j (x_j - centroid) f_j = sum_k q_k fnm_k
    // - centroid * total force (the transform is x = C q, fnm = C^T f)
    for (int e = threadIdx.x; e < 3 * N; e += blockDim.x) {
        const int i = e / 3;
        const double m0 = mass[rp.atom0 + i];
        double qf = 0.0, xc = 0.0;
        for (int k = 0; k < P; ++k) {
            const size_t g = 3 * ((size_t)rp.ba0 + (size_t)k * N) + e;
            const Mode& md = modes[rp.mode0 + k];
            const double m = m0 * md.mfac;
            spring += 0.5 * m * md.w * md.w * q[g] * q[g];
            kin += p[g] * p[g] / (2.0 * m);
            qf += q[g] * fnm[g];
            xc += md.cs * q[g];
        }
        cv += qf - (xc / P) * modes[rp.mode0].ft * fnm[3 * (size_t)rp.ba0 + e];
    }
    for (int b = threadIdx.x; b < N * P; b += blockDim.x) {
        const int c = nnb[rp.ba0 + b];
        nsum += c;
        nmax = max(nmax, c);
    }
    double vals[4] = {spring, cv, kin, nsum};
    for (int a = 0; a < 4; ++a) {
        double v = warp_sum(vals[a]);
        if ((threadIdx.x & 31) == 0) red[a][threadIdx.x >> 5] = v;
    }
    for (int o = 16; o >= 1; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    if ((threadIdx.x & 31) == 0) redm[threadIdx.x >> 5] = nmax;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double tot[4] = {0, 0, 0, 0};
    int mx = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        for (int a = 0; a < 4; ++a) tot[a] += red[a][w];
        mx = max(mx, redm[w]);
    }
    const double spring_eV = tot[0] * MVV2E, kin_eV = tot[2] * MVV2E;
    const double beta = 1.0 / (rp.kT_md * MVV2E / P);   // 1 / (k_B T)
    double Vsum = 0.0;
    for (int k = 0; k < P; ++k) Vsum += V[rp.bs0 + k];
    double* o = est + (size_t)r * EST_STRIDE;
    const double Vbar = Vsum / P;
    const double K_prim = 3.0 * N * P / (2.0 * beta) - spring_eV / P;
    const double K_cv = 3.0 * N / (2.0 * beta) - tot[1] / (2.0 * P);
    o[0] = Vbar;
    o[1] = K_prim;
    o[2] = K_cv;
    o[3] = K_cv + Vbar;
    for (int a = 0; a < 9; ++a) {
        double w = 0.0;
        for (int k = 0; k < P; ++k) w += Wv[9 * (size_t)(rp.bs0 + k) + a];
        o[4 + a] = w / P;
    }
    o[13] = kin_eV + spring_eV + Vsum - Q[r];
    o[14] = Q[r];
    o[15] = 2.0 * kin_eV / (3.0 * N * P * KB);
    o[16] = tot[3] / ((double)N * P);
    o[17] = (double)mx;
}

void launch_estimators(const Dev& d, cudaStream_t st)
{
    estimators_kernel<<<d.R, 256, 0, st>>>(d.reps, d.modes, d.mass, d.q, d.p, d.fnm, d.V, d.W, d.Q, d.nnb, d.est);
}

}  // namespace pimd
