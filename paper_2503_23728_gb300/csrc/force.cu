// force.cu -- neighbour lists, symmetry-function descriptors, the network on
// CUDA cores and the hand-written adjoint (forces and virial as the gradient
// of the per-atom energies). One warp per bead-atom for the neighbour-bound
// parts; bead-atoms are batched over all beads of all replicas.
#include <cuda_runtime.h>

#include <type_traits>

#include "common.cuh"
#include "geom.cuh"
#include "kernels.h"

namespace pimd {

// ---------------------------------------------------------------------------
// a3: descriptors. Warp per bead-atom. Neighbour records (unit vector, r,
// A_eta = exp(-eta r^2) fc) in shared memory; radial channels accumulated
// per lane over its neighbours, angular channels over the unordered
// neighbour pairs, then 32-way transposed warp reductions.
//
// Pair schedule. The unordered pairs of n neighbours are (j, k = j + d mod n)
// for diagonals d = 1..D, D = (n-1)/2, plus the half diagonal d = n/2, j < n/2
// when n is even. For n >= band_min the diagonals are cut into bands of R <=
// rmax; cell (band, j) is one lane's run of R pairs with j fixed in
// registers, so each pair loads only k's record, and 32 consecutive cells
// (one warp step) touch consecutive k (conflict-free shared loads). Small n
// use a flat walk over all pairs instead.
// ---------------------------------------------------------------------------
constexpr int RMAX_CAP = 16;   // largest band length (staging capacity)
// band_min >= rmax + 32 keeps the k of lanes in one step distinct (host enforces)

struct PairWalk {
    int n, j, d, t, npairs;
    __device__ __forceinline__ void init(int n_, int start)
    {
        n = n_;
        npairs = n * (n - 1) / 2;
        t = start;
        if (n > 1) {
            d = 1 + start / n;
            j = start - (d - 1) * n;
        } else {
            d = 1;
            j = 0;
        }
    }
    __device__ __forceinline__ bool valid() const { return t < npairs; }
    __device__ __forceinline__ int k() const
    {
        int kk = j + d;
        return kk >= n ? kk - n : kk;
    }
    __device__ __forceinline__ void advance(int by)
    {
        t += by;
        j += by;
        while (j >= n) {
            j -= n;
            ++d;
        }
    }
};

// this lane's cell of the band schedule; cells c = band * n + j advance by 32
// per warp step (n >= 33 here, so j wraps at most once per step)
struct BandCell {
    int j, dlo, len, band;
    bool act;
    __device__ __forceinline__ void start(int lane, int n, int D, int R, int NB)
    {
        band = 0;
        j = lane;
        set(D, R, NB);
    }
    __device__ __forceinline__ void next(int n, int D, int R, int NB)
    {
        j += 32;
        if (j >= n) {
            j -= n;
            ++band;
        }
        set(D, R, NB);
    }
    __device__ __forceinline__ void set(int D, int R, int NB)
    {
        act = band < NB;
        dlo = 1 + band * R;
        len = act ? min(D - dlo + 1, R) : 0;
        if (!act) j = 0;
    }
};

__device__ __forceinline__ void band_geometry(int n, int rmax, int& D, int& NB, int& R, int& ncell)
{
    D = (n - 1) >> 1;
    NB = (D + rmax - 1) / rmax;
    R = (D + NB - 1) / NB;
    ncell = NB * n;
}

// forward contribution of pair (j, k): ga[q*4+e] += (1 + lambda c)^zeta B_e,
// q = zeta_index * 2 + lambda_index. FP64: 32 scalar FMAs. FP32: packed
// FP32x2 over lambda = (+1, -1): g2[z*4+e] = (ga[(2z)*4+e], ga[(2z+1)*4+e]).
template <typename Real> struct FwdAcc;
template <> struct FwdAcc<double> {
    double g[NA];
};
template <> struct FwdAcc<float> {
    float2 g[16];
};

__device__ __forceinline__ void acc_zero(FwdAcc<double>& a)
{
#pragma unroll
    for (int c = 0; c < NA; ++c) a.g[c] = 0.0;
}
__device__ __forceinline__ void acc_zero(FwdAcc<float>& a)
{
#pragma unroll
    for (int c = 0; c < 16; ++c) a.g[c] = make_float2(0.0f, 0.0f);
}
__device__ __forceinline__ void acc_out(const FwdAcc<double>& a, double (&ga)[NA])
{
#pragma unroll
    for (int c = 0; c < NA; ++c) ga[c] = a.g[c];
}
__device__ __forceinline__ void acc_out(const FwdAcc<float>& a, float (&ga)[NA])
{
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            ga[(2 * z) * 4 + e] = a.g[z * 4 + e].x;
            ga[(2 * z + 1) * 4 + e] = a.g[z * 4 + e].y;
        }
}

__device__ __forceinline__ void fwd_pair(const Dbl4& uj, const Dbl4& aj, const Dbl4& uk, const Dbl4& ak,
                                         FwdAcc<double>& acc)
{
    const double c = uj.x * uk.x + uj.y * uk.y + uj.z * uk.z;
    const double Bv[4] = {aj.x * ak.x, aj.y * ak.y, aj.z * ak.z, aj.w * ak.w};
    const double xp = 1.0 + c, xm = 1.0 - c;
    const double xp2 = xp * xp, xm2 = xm * xm;
    const double xp4 = xp2 * xp2, xm4 = xm2 * xm2;
    const double Pq[8] = {xp, xm, xp2, xm2, xp4, xm4, xp4 * xp4, xm4 * xm4};
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc.g[q * 4 + e] += Pq[q] * Bv[e];
}

__device__ __forceinline__ void fwd_pair(const float4& uj, const float4& aj, const float4& uk, const float4& ak,
                                         FwdAcc<float>& acc)
{
    const float c = fmaf(uj.x, uk.x, fmaf(uj.y, uk.y, uj.z * uk.z));
    const float Bv[4] = {aj.x * ak.x, aj.y * ak.y, aj.z * ak.z, aj.w * ak.w};
    // X_n = ((1 + c)^n, (1 - c)^n)
    const float2 X1 = __ffma2_rn(make_float2(c, c), make_float2(1.0f, -1.0f), make_float2(1.0f, 1.0f));
    const float2 X2 = __fmul2_rn(X1, X1);
    const float2 X4 = __fmul2_rn(X2, X2);
    const float2 X8 = __fmul2_rn(X4, X4);
    const float2 Xz[4] = {X1, X2, X4, X8};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float2 Bb = make_float2(Bv[e], Bv[e]);
#pragma unroll
        for (int z = 0; z < 4; ++z) acc.g[z * 4 + e] = __ffma2_rn(Xz[z], Bb, acc.g[z * 4 + e]);
    }
}

template <typename Real, bool FAST>
__global__ void __launch_bounds__(256, 4) desc_fwd_kernel(
    const Vec4<Real>* __restrict__ x, const int* __restrict__ ba_sys, const BeadSys* __restrict__ bsys,
    const Rep* __restrict__ reps, const int* __restrict__ nbr, const int* __restrict__ nnb, int maxnb, int B,
    DescParams<Real> dp, Sched sc, Real* __restrict__ G)
{
    using V4 = Vec4<Real>;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int wib = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    V4* U = reinterpret_cast<V4*>(smem_raw) + (size_t)wib * 2 * maxnb;
    V4* A = U + maxnb;
    const int b = blockIdx.x * (blockDim.x >> 5) + wib;
    if (b >= B) return;
    const BeadSys sy = bsys[ba_sys[b]];
    const Rep& rp = reps[sy.rep];
    const int n = min(nnb[b], maxnb);
    const V4 xi = x[b];

    Real gr[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) gr[c] = Real(0);
    for (int s = (int)lane; s < n; s += 32) {
        const int j = nbr[(size_t)b * maxnb + s];
        const V4 xj = x[sy.ba0 + j];
        Real dx, dy, dz;
        pair_vec(rp, xi, xj, dx, dy, dz);
        const Real r2 = dx * dx + dy * dy + dz * dz;
        const Real r = f_sqrt(r2);
        const Real ir = Real(1) / r;
        Real fc, dfc;
        cutoff(r, dp.rc, dp.pi_over_rc, fc, dfc);
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            const Real t = r - dp.r_mu[c];
            gr[c] += gauss<FAST>(dp.eta_R, dp.eta_R_l2, t * t) * fc;
        }
        U[s] = make4<V4, Real>(dx * ir, dy * ir, dz * ir, r);
        A[s] = make4<V4, Real>(gauss<FAST>(dp.eta_A[0], dp.eta_A_l2[0], r2) * fc,
                               gauss<FAST>(dp.eta_A[1], dp.eta_A_l2[1], r2) * fc,
                               gauss<FAST>(dp.eta_A[2], dp.eta_A_l2[2], r2) * fc,
                               gauss<FAST>(dp.eta_A[3], dp.eta_A_l2[3], r2) * fc);
    }
    const Real Gr = transpose_reduce32(gr, lane);
    __syncwarp();

    FwdAcc<Real> acc;
    acc_zero(acc);
    if (n >= sc.band_min) {
        int D, NB, R, ncell;
        band_geometry(n, sc.rmax, D, NB, R, ncell);
        BandCell cl;
        cl.start((int)lane, n, D, R, NB);
        for (int c0 = 0; c0 < ncell; c0 += 32, cl.next(n, D, R, NB)) {
            const V4 uj = U[cl.j], aj = A[cl.j];
#pragma unroll 2
            for (int r = 0; r < cl.len; ++r) {
                int k = cl.j + cl.dlo + r;
                k = k >= n ? k - n : k;
                fwd_pair(uj, aj, U[k], A[k], acc);
            }
        }
        if ((n & 1) == 0) {
            const int h = n >> 1;
            for (int j = (int)lane; j < h; j += 32) fwd_pair(U[j], A[j], U[j + h], A[j + h], acc);
        }
    } else {
        PairWalk w;
        w.init(n, (int)lane);
        for (; w.valid(); w.advance(32)) {
            const int k = w.k();
            fwd_pair(U[w.j], A[w.j], U[k], A[k], acc);
        }
    }
    Real ga[NA];
    acc_out(acc, ga);
    Real Ga = transpose_reduce32(ga, lane);
    // 2^(1 - zeta) for zeta = 1, 2, 4, 8 (channel zeta index = lane / 8)
    const int zi = (int)lane >> 3;
    Ga *= (zi == 0) ? Real(1) : (zi == 1) ? Real(0.5) : (zi == 2) ? Real(0.125) : Real(0.0078125);
    G[(size_t)b * ND + lane] = Gr;
    G[(size_t)b * ND + NR + lane] = Ga;
}

// ---------------------------------------------------------------------------
// Descriptors for small clusters: every replica has at most 33 atoms, so n <= 32
// neighbours. Half a warp per bead-atom (two per warp): lanes l and l + 16 of
// the half take the neighbours' radial terms and weights, and the unordered
// pairs are walked over the half's 16 lanes. The arithmetic is that of
// desc_fwd_kernel. A whole warp per atom would leave the lanes beyond n idle
// in the neighbour phase; these clusters have 5-23 neighbours.
// ---------------------------------------------------------------------------
constexpr int SMALL_SL = 32;    // neighbour slots per atom
constexpr int SMALL_ATOMS = 16; // bead-atoms per 256-thread block

// Sums over the 16 lanes of a half warp of 32 per-lane values: lane l of the
// half ends with the totals of values 2l (v[0]) and 2l + 1 (v[1]).
__device__ __forceinline__ void half_reduce32(float (&v)[32], int hl)
{
#pragma unroll
    for (int o = 8, n = 32; o >= 1; o >>= 1, n >>= 1) {
        const bool upper = (hl & o) != 0;
#pragma unroll
        for (int q = 0; q < n / 2; ++q) {
            const float send = upper ? v[q] : v[q + n / 2];
            const float keep = upper ? v[q + n / 2] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
}

template <bool FAST>
__global__ void __launch_bounds__(256) desc_fwd_small_kernel(
    const float4* __restrict__ x, const int* __restrict__ ba_sys, const BeadSys* __restrict__ bsys,
    const Rep* __restrict__ reps, const int* __restrict__ nbr, const int* __restrict__ nnb, int maxnb, int B,
    DescParams<float> dp, float* __restrict__ G)
{
    __shared__ float4 U[SMALL_ATOMS][SMALL_SL], A[SMALL_ATOMS][SMALL_SL];
    const int hw = threadIdx.x >> 4;
    const int hl = threadIdx.x & 15;
    const int b = blockIdx.x * SMALL_ATOMS + hw;
    // no early return: the two halves of a warp meet in the shuffles
    const bool live = b < B;
    int n = 0;
    BeadSys sy{0, 0, 0, 0};
    float4 xi = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (live) {
        sy = bsys[ba_sys[b]];
        n = min(nnb[b], min(maxnb, SMALL_SL));
        xi = x[b];
    }
    const Rep& rp = reps[sy.rep];

    // radial sums; on the BF16 path with evenly spaced centres the product
    // recurrence of radial_gauss32 runs on centre pairs (c, c + 16), packed
    const bool packed = FAST && dp.r_even;
    float2 gr2[NR / 2];
#pragma unroll
    for (int c = 0; c < NR / 2; ++c) gr2[c] = make_float2(0.0f, 0.0f);
    for (int sl = hl; sl < n; sl += 16) {
        const int j = nbr[(size_t)b * maxnb + sl];
        const float4 xj = x[sy.ba0 + j];
        float dx, dy, dz;
        pair_vec(rp, xi, xj, dx, dy, dz);
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float r = sqrtf(r2);
        const float ir = 1.0f / r;
        float fc, dfc;
        cutoff(r, dp.rc, dp.pi_over_rc, fc, dfc);
        if (packed) {
            const float2 rho = make_float2(dp.rec_k, dp.rec_k);
            const float dd = dp.r_delta * dp.r_delta;
#pragma unroll
            for (int qp = 0; qp < 2; ++qp) {
                const float ta = r - dp.r_mu[8 * qp], tb = r - dp.r_mu[8 * qp + 16];
                float2 e2 = make_float2(exp2f(-dp.eta_R_l2 * ta * ta) * fc, exp2f(-dp.eta_R_l2 * tb * tb) * fc);
                float2 R2 = make_float2(exp2f(dp.eta_R_l2 * fmaf(2.0f * ta, dp.r_delta, -dd)),
                                        exp2f(dp.eta_R_l2 * fmaf(2.0f * tb, dp.r_delta, -dd)));
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    gr2[8 * qp + k] = __fadd2_rn(gr2[8 * qp + k], e2);
                    if (k < 7) {
                        e2 = __fmul2_rn(e2, R2);
                        R2 = __fmul2_rn(R2, rho);
                    }
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                const float t = r - dp.r_mu[c];
                const float g = gauss<FAST>(dp.eta_R, dp.eta_R_l2, t * t) * fc;
                float2& slot = gr2[8 * ((c >> 3) & 1) + (c & 7)];
                if (c < 16) slot.x += g;
                else slot.y += g;
            }
        }
        U[hw][sl] = make_float4(dx * ir, dy * ir, dz * ir, r);
        A[hw][sl] = make_float4(gauss<FAST>(dp.eta_A[0], dp.eta_A_l2[0], r2) * fc,
                                gauss<FAST>(dp.eta_A[1], dp.eta_A_l2[1], r2) * fc,
                                gauss<FAST>(dp.eta_A[2], dp.eta_A_l2[2], r2) * fc,
                                gauss<FAST>(dp.eta_A[3], dp.eta_A_l2[3], r2) * fc);
    }
    float gr[NR];
#pragma unroll
    for (int qp = 0; qp < 2; ++qp)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            gr[8 * qp + k] = gr2[8 * qp + k].x;
            gr[8 * qp + k + 16] = gr2[8 * qp + k].y;
        }
    half_reduce32(gr, hl);
    __syncwarp();

    FwdAcc<float> acc;
    acc_zero(acc);
    PairWalk w;
    w.init(n, hl);
    for (; w.valid(); w.advance(16)) {
        const int k = w.k();
        fwd_pair(U[hw][w.j], A[hw][w.j], U[hw][k], A[hw][k], acc);
    }
    float ga[NA];
    acc_out(acc, ga);
    half_reduce32(ga, hl);
    if (live) {
        // channels 2 hl and 2 hl + 1; 2^(1 - zeta) for zeta = 1, 2, 4, 8 (zeta index = channel / 8)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int ch = 2 * hl + k;
            const int zi = ch >> 3;
            const float sc = zi == 0 ? 1.0f : zi == 1 ? 0.5f : zi == 2 ? 0.125f : 0.0078125f;
            G[(size_t)b * ND + ch] = gr[k];
            G[(size_t)b * ND + NR + ch] = ga[k] * sc;
        }
    }
}

template <typename Real>
static int desc_warps(int maxnb)
{
    // shared memory per warp: U, A records
    const size_t per = (size_t)2 * maxnb * sizeof(Vec4<Real>);
    int w = 8;
    while (w > 1 && per * w > 200 * 1024) w >>= 1;
    return w;
}

template <bool FAST>
static void run_desc_f32(const Dev& d, const void* dpv, cudaStream_t st)
{
    const int w = desc_warps<float>(d.maxnb);
    const size_t sm = (size_t)w * 2 * d.maxnb * sizeof(float4);
    { static size_t done = 0; set_smem(desc_fwd_kernel<float, FAST>, sm, done); }
    desc_fwd_kernel<float, FAST><<<(d.B + w - 1) / w, 32 * w, sm, st>>>(
        (const float4*)d.x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, d.B,
        *(const DescParams<float>*)dpv, d.sched, (float*)d.G);
}

void launch_descriptors(const Dev& d, const void* dpv, cudaStream_t st)
{
    if (d.precision != 0 && d.sched.ang && d.mom) {
        launch_descriptors_moment(d, dpv, st);
        return;
    }
    if (d.precision == 0) {
        const int w = desc_warps<double>(d.maxnb);
        const size_t sm = (size_t)w * 2 * d.maxnb * sizeof(Dbl4);
        { static size_t done = 0; set_smem(desc_fwd_kernel<double, false>, sm, done); }
        desc_fwd_kernel<double, false><<<(d.B + w - 1) / w, 32 * w, sm, st>>>(
            (const Dbl4*)d.x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, d.B,
            *(const DescParams<double>*)dpv, d.sched, (double*)d.G);
    } else if (d.max_N <= SMALL_SL + 1) {
        if (d.precision == 2)
            desc_fwd_small_kernel<true><<<(d.B + SMALL_ATOMS - 1) / SMALL_ATOMS, 256, 0, st>>>(
                (const float4*)d.x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, d.B,
                *(const DescParams<float>*)dpv, (float*)d.G);
        else
            desc_fwd_small_kernel<false><<<(d.B + SMALL_ATOMS - 1) / SMALL_ATOMS, 256, 0, st>>>(
                (const float4*)d.x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, d.B,
                *(const DescParams<float>*)dpv, (float*)d.G);
    } else if (d.precision == 2) {
        run_desc_f32<true>(d, dpv, st);
    } else {
        run_desc_f32<false>(d, dpv, st);
    }
}

// ---------------------------------------------------------------------------
// a5: adjoint. With g = dE_i/dG_i from the network, accumulate per neighbour
//   dE/dA_eta(j) = sum_k sum_(zeta,lambda) g'_(zeta,lambda,eta) (1+lambda c)^zeta A_eta(k)
//   w_j = sum_k dE/dc_jk u_k,   s_j = sum_k dE/dc_jk c_jk
// over the neighbour pairs (g' = 2^(1-zeta) g), then
//   v_j = dE_i/dr_ij = [dE/dr_radial + sum_eta dE/dA_eta dA_eta/dr] u_j + (w_j - s_j u_j) / r_j
// and scatter F_j -= v_j, F_i += v_j, W -= r_ij (x) v_j.
//
// In the band schedule the j-side sums stay in registers for the lane's run,
// and the k-side sums ride down the lanes as a shuffle carry: lane L at step
// r and lane L-1 at step r+1 handle the same k. A carry is added into k's
// shared-memory accumulator when its chain ends: at the band's last step
// (all lanes, distinct k), or earlier at lane 0 / the first lane of a new
// band, whose finished carries are parked in a small staging area and
// added after the run.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_add_vec(float4* f, float ax, float ay, float az)
{
    atomicAdd(f, make_float4(ax, ay, az, 0.0f));
}
__device__ __forceinline__ void atomic_add_vec(Dbl4* f, double ax, double ay, double az)
{
    atomicAdd(&f->x, ax);
    atomicAdd(&f->y, ay);
    atomicAdd(&f->z, az);
}

// adjoint contribution of pair (j, k): jd / kd += (dE/dA(.)[4], w[3], s).
// Coefficients g'_nu = 2^(1-zeta) g_(32+nu); FP32 packs them over lambda:
// g2[z*4+e] = (g'_((2z)*4+e), g'_((2z+1)*4+e)).
template <typename Real> struct AdjCoef;
template <> struct AdjCoef<double> {
    double g[NA];
};
template <> struct AdjCoef<float> {
    float2 g[16];
};

__device__ __forceinline__ double zeta_scale(int zi) { return zi == 0 ? 1.0 : zi == 1 ? 0.5 : zi == 2 ? 0.125 : 0.0078125; }

__device__ __forceinline__ void coef_load(AdjCoef<double>& a, const double* gs)
{
#pragma unroll
    for (int nu = 0; nu < NA; ++nu) a.g[nu] = gs[NR + nu] * zeta_scale(nu >> 3);
}
__device__ __forceinline__ void coef_load(AdjCoef<float>& a, const float* gs)
{
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float sc = (float)zeta_scale(z);
            a.g[z * 4 + e] = make_float2(gs[NR + (2 * z) * 4 + e] * sc, gs[NR + (2 * z + 1) * 4 + e] * sc);
        }
}

__device__ __forceinline__ void adj_pair(const AdjCoef<double>& cf, const Dbl4& uj, const Dbl4& aj, const Dbl4& uk,
                                         const Dbl4& ak, double (&jd)[8], double (&kd)[8])
{
    const double c = uj.x * uk.x + uj.y * uk.y + uj.z * uk.z;
    const double Bv[4] = {aj.x * ak.x, aj.y * ak.y, aj.z * ak.z, aj.w * ak.w};
    const double xp = 1.0 + c, xm = 1.0 - c;
    const double xp2 = xp * xp, xm2 = xm * xm;
    const double xp3 = xp2 * xp, xm3 = xm2 * xm;
    const double xp4 = xp2 * xp2, xm4 = xm2 * xm2;
    const double xp7 = xp4 * xp3, xm7 = xm4 * xm3;
    const double Pq[8] = {xp, xm, xp2, xm2, xp4, xm4, xp4 * xp4, xm4 * xm4};
    double H[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        H[q] = cf.g[q * 4] * Bv[0];
#pragma unroll
        for (int e = 1; e < 4; ++e) H[q] += cf.g[q * 4 + e] * Bv[e];
    }
    // dE/dc = sum_q zeta lambda (1 + lambda c)^(zeta - 1) H_q
    double dEdc = H[0] - H[1];
    dEdc += 2.0 * (xp * H[2] - xm * H[3]);
    dEdc += 4.0 * (xp3 * H[4] - xm3 * H[5]);
    dEdc += 8.0 * (xp7 * H[6] - xm7 * H[7]);
    double K[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        K[e] = cf.g[e] * Pq[0];
#pragma unroll
        for (int q = 1; q < 8; ++q) K[e] += cf.g[q * 4 + e] * Pq[q];
    }
    jd[0] += K[0] * ak.x; jd[1] += K[1] * ak.y; jd[2] += K[2] * ak.z; jd[3] += K[3] * ak.w;
    kd[0] += K[0] * aj.x; kd[1] += K[1] * aj.y; kd[2] += K[2] * aj.z; kd[3] += K[3] * aj.w;
    jd[4] += dEdc * uk.x; jd[5] += dEdc * uk.y; jd[6] += dEdc * uk.z; jd[7] += dEdc * c;
    kd[4] += dEdc * uj.x; kd[5] += dEdc * uj.y; kd[6] += dEdc * uj.z; kd[7] += dEdc * c;
}

__device__ __forceinline__ void adj_pair(const AdjCoef<float>& cf, const float4& uj, const float4& aj,
                                         const float4& uk, const float4& ak, float (&jd)[8], float (&kd)[8])
{
    const float c = fmaf(uj.x, uk.x, fmaf(uj.y, uk.y, uj.z * uk.z));
    const float Bv[4] = {aj.x * ak.x, aj.y * ak.y, aj.z * ak.z, aj.w * ak.w};
    // X_n = ((1 + c)^n, (1 - c)^n)
    const float2 X1 = __ffma2_rn(make_float2(c, c), make_float2(1.0f, -1.0f), make_float2(1.0f, 1.0f));
    const float2 X2 = __fmul2_rn(X1, X1);
    const float2 X3 = __fmul2_rn(X2, X1);
    const float2 X4 = __fmul2_rn(X2, X2);
    const float2 X7 = __fmul2_rn(X4, X3);
    const float2 X8 = __fmul2_rn(X4, X4);
    // per eta channel e, with D_zeta = zeta X_(zeta-1) (the c-derivative of X_zeta):
    //   K_e = sum_z (g'_(z,+,e) xp^zeta + g'_(z,-,e) xm^zeta)
    //   M_e = sum_z zeta (g'_(z,+,e) xp^(zeta-1) - g'_(z,-,e) xm^(zeta-1)),  dE/dc = sum_e B_e M_e
    const float2 D2 = __fmul2_rn(X1, make_float2(2.0f, 2.0f));
    const float2 D4 = __fmul2_rn(X3, make_float2(4.0f, 4.0f));
    const float2 D8 = __fmul2_rn(X7, make_float2(8.0f, 8.0f));
    float K[4];
    float dEdc = 0.0f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float2 k2 = __fmul2_rn(cf.g[e], X1);
        k2 = __ffma2_rn(cf.g[4 + e], X2, k2);
        k2 = __ffma2_rn(cf.g[8 + e], X4, k2);
        k2 = __ffma2_rn(cf.g[12 + e], X8, k2);
        K[e] = k2.x + k2.y;
        float2 m2 = __ffma2_rn(cf.g[4 + e], D2, cf.g[e]);
        m2 = __ffma2_rn(cf.g[8 + e], D4, m2);
        m2 = __ffma2_rn(cf.g[12 + e], D8, m2);
        dEdc = fmaf(Bv[e], m2.x - m2.y, dEdc);
    }
    jd[0] += K[0] * ak.x; jd[1] += K[1] * ak.y; jd[2] += K[2] * ak.z; jd[3] += K[3] * ak.w;
    kd[0] += K[0] * aj.x; kd[1] += K[1] * aj.y; kd[2] += K[2] * aj.z; kd[3] += K[3] * aj.w;
    jd[4] += dEdc * uk.x; jd[5] += dEdc * uk.y; jd[6] += dEdc * uk.z; jd[7] += dEdc * c;
    kd[4] += dEdc * uj.x; kd[5] += dEdc * uj.y; kd[6] += dEdc * uj.z; kd[7] += dEdc * c;
}

template <typename Real, typename V4>
__device__ __forceinline__ void acc_rmw(V4* ACC0, V4* ACC1, int s, const Real (&v)[8])
{
    V4 a = ACC0[s];
    a.x += v[0]; a.y += v[1]; a.z += v[2]; a.w += v[3];
    ACC0[s] = a;
    V4 b = ACC1[s];
    b.x += v[4]; b.y += v[5]; b.z += v[6]; b.w += v[7];
    ACC1[s] = b;
}

template <typename Real, bool FAST>
__global__ void __launch_bounds__(256) desc_adj_kernel(
    const Vec4<Real>* __restrict__ x, const int* __restrict__ ba_sys, const BeadSys* __restrict__ bsys,
    const Rep* __restrict__ reps, const int* __restrict__ nbr, const int* __restrict__ nnb, int maxnb, int B,
    DescParams<Real> dp, Sched sc, const Real* __restrict__ dEdG, Vec4<Real>* __restrict__ f,
    Real* __restrict__ wbuf, int det, Vec4<Real>* __restrict__ vbuf)
{
    using V4 = Vec4<Real>;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int wib = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const unsigned lane = lane_id();
    // per warp: U, A, DA, ACC0 (dE/dA), ACC1 (w, s) records; staging [2][RMAX_CAP][2];
    // radial dE/dr and g
    V4* U = reinterpret_cast<V4*>(smem_raw) + (size_t)wib * (5 * maxnb + 4 * RMAX_CAP);
    V4* A = U + maxnb;
    V4* DA = A + maxnb;
    V4* ACC0 = DA + maxnb;
    V4* ACC1 = ACC0 + maxnb;
    V4* STG = ACC1 + maxnb;   // [2 buffers][RMAX_CAP][2 records]
    Real* RAD = reinterpret_cast<Real*>(reinterpret_cast<V4*>(smem_raw) + (size_t)nw * (5 * maxnb + 4 * RMAX_CAP)) +
                (size_t)wib * (maxnb + ND);
    Real* gs = RAD + maxnb;
    const int b = blockIdx.x * nw + wib;
    if (b >= B) return;
    const BeadSys sy = bsys[ba_sys[b]];
    const Rep& rp = reps[sy.rep];
    const int n = min(nnb[b], maxnb);
    const V4 xi = x[b];
    gs[lane] = dEdG[(size_t)b * ND + lane];
    gs[NR + lane] = dEdG[(size_t)b * ND + NR + lane];
    __syncwarp();

    for (int s = (int)lane; s < n; s += 32) {
        const int j = nbr[(size_t)b * maxnb + s];
        const V4 xj = x[sy.ba0 + j];
        Real dx, dy, dz;
        pair_vec(rp, xi, xj, dx, dy, dz);
        const Real r2 = dx * dx + dy * dy + dz * dz;
        const Real r = f_sqrt(r2);
        const Real ir = Real(1) / r;
        Real fc, dfc;
        cutoff(r, dp.rc, dp.pi_over_rc, fc, dfc);
        Real dEdr = Real(0);
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            const Real t = r - dp.r_mu[c];
            const Real e = gauss<FAST>(dp.eta_R, dp.eta_R_l2, t * t);
            dEdr += gs[c] * e * (Real(-2) * dp.eta_R * t * fc + dfc);
        }
        Real a[4], da[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const Real ex = gauss<FAST>(dp.eta_A[e], dp.eta_A_l2[e], r2);
            a[e] = ex * fc;
            da[e] = ex * (Real(-2) * dp.eta_A[e] * r * fc + dfc);
        }
        U[s] = make4<V4, Real>(dx * ir, dy * ir, dz * ir, r);
        A[s] = make4<V4, Real>(a[0], a[1], a[2], a[3]);
        DA[s] = make4<V4, Real>(da[0], da[1], da[2], da[3]);
        ACC0[s] = make4<V4, Real>(Real(0), Real(0), Real(0), Real(0));
        ACC1[s] = make4<V4, Real>(Real(0), Real(0), Real(0), Real(0));
        RAD[s] = dEdr;
    }
    __syncwarp();

    // angular coefficients g'_nu = 2^(1-zeta) g_(32+nu)
    AdjCoef<Real> gp;
    coef_load(gp, gs);
    if (n >= sc.band_min) {
        int D, NB, R, ncell;
        band_geometry(n, sc.rmax, D, NB, R, ncell);
        BandCell cl;
        cl.start((int)lane, n, D, R, NB);
        for (int c0 = 0; c0 < ncell; c0 += 32, cl.next(n, D, R, NB)) {
            const int band_up = __shfl_down_sync(0xffffffffu, cl.band, 1);
            const int band_dn = __shfl_up_sync(0xffffffffu, cl.band, 1);
            const bool recv = cl.act && lane < 31 && band_up == cl.band;   // carry arrives from lane + 1
            const bool pass = cl.act && lane > 0 && band_dn == cl.band;    // carry leaves to lane - 1
            const int nst = __reduce_max_sync(0xffffffffu, (unsigned)cl.len);
            // exit lanes: lane 0 (buffer 0) and the first lane of a second band (buffer 1)
            const int sbuf = lane == 0 ? 0 : 1;
            const V4 uj = U[cl.j], aj = A[cl.j];
            Real jd[8], kd[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) jd[q] = kd[q] = Real(0);
#pragma unroll 2
            for (int r = 0; r < nst; ++r) {
                const bool valid = r < cl.len;
                if (valid) {
                    int k = cl.j + cl.dlo + r;
                    k = k >= n ? k - n : k;
                    adj_pair(gp, uj, aj, U[k], A[k], jd, kd);
                    if (!pass && r < cl.len - 1) {
                        V4* st = STG + (size_t)(sbuf * RMAX_CAP + r) * 2;
                        st[0] = make4<V4, Real>(kd[0], kd[1], kd[2], kd[3]);
                        st[1] = make4<V4, Real>(kd[4], kd[5], kd[6], kd[7]);
                    }
                }
                const bool shift = r < cl.len - 1;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const Real nk = __shfl_down_sync(0xffffffffu, kd[q], 1);
                    if (shift) kd[q] = recv ? nk : Real(0);
                }
            }
            __syncwarp();
            // j-side sums, distinct j per lane
            if (cl.act) acc_rmw(ACC0, ACC1, cl.j, jd);
            __syncwarp();
            // chains ending at the band's last step, distinct k per lane
            if (cl.act && cl.len > 0) {
                int k = cl.j + cl.dlo + cl.len - 1;
                acc_rmw(ACC0, ACC1, k >= n ? k - n : k, kd);
            }
            __syncwarp();
            // parked chains of lane 0 (buffer 0) and of the first lane of the second band (buffer 1)
            const unsigned seams = __ballot_sync(0xffffffffu, cl.act && lane > 0 && !pass);
            const int sl = seams ? __ffs(seams) - 1 : 0;
            const int j0 = __shfl_sync(0xffffffffu, cl.j, 0), d0 = __shfl_sync(0xffffffffu, cl.dlo, 0);
            const int l0 = __shfl_sync(0xffffffffu, cl.len, 0);
            const int js = __shfl_sync(0xffffffffu, cl.j, sl), ds = __shfl_sync(0xffffffffu, cl.dlo, sl);
            const int ls = seams ? __shfl_sync(0xffffffffu, cl.len, sl) : 0;
            const int rr = (int)(lane & 15);
            const int buf = (int)(lane >> 4);
            const int jb = buf ? js : j0, db = buf ? ds : d0, lb = buf ? ls : l0;
            if (rr < lb - 1) {
                const V4* st = STG + (size_t)(buf * RMAX_CAP + rr) * 2;
                const Real v[8] = {st[0].x, st[0].y, st[0].z, st[0].w, st[1].x, st[1].y, st[1].z, st[1].w};
                int k = jb + db + rr;
                acc_rmw(ACC0, ACC1, k >= n ? k - n : k, v);
            }
            __syncwarp();
        }
        if ((n & 1) == 0) {
            const int h = n >> 1;
            for (int j0 = 0; j0 < h; j0 += 32) {
                const int j = j0 + (int)lane;
                Real jd[8], kd[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) jd[q] = kd[q] = Real(0);
                if (j < h) adj_pair(gp, U[j], A[j], U[j + h], A[j + h], jd, kd);
                if (j < h) acc_rmw(ACC0, ACC1, j, jd);
                __syncwarp();
                if (j < h) acc_rmw(ACC0, ACC1, j + h, kd);
                __syncwarp();
            }
        }
    } else if (det || !sc.small_atomics) {
        // ordered pairs, j-side sums only: every unordered pair is evaluated
        // twice, and each lane owns its j's accumulators (fixed order, no
        // atomics; shared-memory float atomics cost ~4x more per pair)
        for (int j0 = 0; j0 < n; j0 += 32) {
            const int j = j0 + (int)lane;
            if (j < n) {
                const V4 uj = U[j], aj = A[j];
                Real jd[8], kd[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) jd[q] = kd[q] = Real(0);
                for (int k = 0; k < n; ++k)
                    if (k != j) adj_pair(gp, uj, aj, U[k], A[k], jd, kd);
                acc_rmw(ACC0, ACC1, j, jd);
            }
        }
    } else {
        PairWalk w;
        w.init(n, (int)lane);
        for (; w.valid(); w.advance(32)) {
            const int j = w.j, k = w.k();
            Real jd[8], kd[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) jd[q] = kd[q] = Real(0);
            adj_pair(gp, U[j], A[j], U[k], A[k], jd, kd);
            Real* a0j = reinterpret_cast<Real*>(&ACC0[j]);
            Real* a1j = reinterpret_cast<Real*>(&ACC1[j]);
            Real* a0k = reinterpret_cast<Real*>(&ACC0[k]);
            Real* a1k = reinterpret_cast<Real*>(&ACC1[k]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                atomicAdd(a0j + q, jd[q]);
                atomicAdd(a1j + q, jd[4 + q]);
                atomicAdd(a0k + q, kd[q]);
                atomicAdd(a1k + q, kd[4 + q]);
            }
        }
    }
    __syncwarp();

    Real fi[3] = {Real(0), Real(0), Real(0)};
    Real wl[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) wl[q] = Real(0);
    for (int s = (int)lane; s < n; s += 32) {
        const int j = nbr[(size_t)b * maxnb + s];
        const V4 u = U[s], da = DA[s], a0 = ACC0[s], a1 = ACC1[s];
        const Real dEdr = RAD[s] + a0.x * da.x + a0.y * da.y + a0.z * da.z + a0.w * da.w;
        const Real ir = Real(1) / u.w;
        const Real v[3] = {dEdr * u.x + (a1.x - a1.w * u.x) * ir, dEdr * u.y + (a1.y - a1.w * u.y) * ir,
                           dEdr * u.z + (a1.z - a1.w * u.z) * ir};
        if (det)
            vbuf[(size_t)b * maxnb + s] = make4<V4, Real>(v[0], v[1], v[2], Real(0));
        else
            atomic_add_vec(&f[sy.ba0 + j], -v[0], -v[1], -v[2]);
        const Real d3[3] = {u.x * u.w, u.y * u.w, u.z * u.w};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            fi[a] += v[a];
#pragma unroll
            for (int c = 0; c < 3; ++c) wl[3 * a + c] -= d3[a] * v[c];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) fi[a] = warp_sum(fi[a]);
#pragma unroll
    for (int q = 0; q < 9; ++q) wl[q] = warp_sum(wl[q]);
    if (lane == 0) {
        if (det)
            f[b] = make4<V4, Real>(fi[0], fi[1], fi[2], Real(0));   // gathered later
        else
            atomic_add_vec(&f[b], fi[0], fi[1], fi[2]);
    }
    if (lane < 9) {
        Real mine = wl[0];
#pragma unroll
        for (int q = 1; q < 9; ++q)
            if ((int)lane == q) mine = wl[q];
        wbuf[(size_t)b * 9 + lane] = mine;   // per bead-atom virial, reduced per bead in FP64
    }
}

// Deterministic force gather: F_b = (sum of b's own pair vectors) - sum over
// neighbours j of the pair vector j stored for b (b's slot in j's sorted
// list, found by bisection). Fixed order, no atomics. Warp per bead-atom.
template <typename Real>
__global__ void __launch_bounds__(256) force_gather_kernel(const int* __restrict__ ba_sys,
                                                           const BeadSys* __restrict__ bsys,
                                                           const int* __restrict__ nbr, const int* __restrict__ nnb,
                                                           int maxnb, int B, const Vec4<Real>* __restrict__ vbuf,
                                                           Vec4<Real>* __restrict__ f)
{
    using V4 = Vec4<Real>;
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = lane_id();
    if (b >= B) return;
    const BeadSys sy = bsys[ba_sys[b]];
    const int il = b - sy.ba0;
    const int n = min(nnb[b], maxnb);
    Real acc[3] = {Real(0), Real(0), Real(0)};
    for (int s = (int)lane; s < n; s += 32) {
        const int jg = sy.ba0 + nbr[(size_t)b * maxnb + s];
        const int* L = nbr + (size_t)jg * maxnb;
        int lo = 0, hi = min(nnb[jg], maxnb);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (L[mid] < il) lo = mid + 1;
            else hi = mid;
        }
        const V4 v = vbuf[(size_t)jg * maxnb + lo];
        acc[0] += v.x;
        acc[1] += v.y;
        acc[2] += v.z;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[a] = warp_sum(acc[a]);
    if (lane == 0) {
        V4 v = f[b];
        v.x -= acc[0];
        v.y -= acc[1];
        v.z -= acc[2];
        f[b] = v;
    }
}

void launch_force_gather(const Dev& d, cudaStream_t st)
{
    const int blocks = (int)(((size_t)d.B * 32 + 255) / 256);
    if (d.precision == 0)
        force_gather_kernel<double><<<blocks, 256, 0, st>>>(d.ba_sys, d.bsys, d.nbr, d.nnb, d.maxnb, d.B,
                                                            (const Dbl4*)d.vbuf, (Dbl4*)d.f);
    else
        force_gather_kernel<float><<<blocks, 256, 0, st>>>(d.ba_sys, d.bsys, d.nbr, d.nnb, d.maxnb, d.B,
                                                           (const float4*)d.vbuf, (float4*)d.f);
}

template <typename Real>
static size_t adj_smem_per_warp(int maxnb)
{
    return (size_t)(5 * maxnb + 4 * RMAX_CAP) * sizeof(Vec4<Real>) + (size_t)(maxnb + ND) * sizeof(Real);
}

template <typename Real>
static int adj_warps(int maxnb)
{
    const size_t per = adj_smem_per_warp<Real>(maxnb);
    int w = 8;
    while (w > 1 && per * w > 200 * 1024) w >>= 1;
    return w;
}

template <bool FAST>
static void run_adj_f32(const Dev& d, const void* dpv, cudaStream_t st)
{
    const int w = adj_warps<float>(d.maxnb);
    const size_t sm = (size_t)w * adj_smem_per_warp<float>(d.maxnb);
    { static size_t done = 0; set_smem(desc_adj_kernel<float, FAST>, sm, done); }
    desc_adj_kernel<float, FAST><<<(d.B + w - 1) / w, 32 * w, sm, st>>>(
        (const float4*)d.x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, d.B,
        *(const DescParams<float>*)dpv, d.sched, (const float*)d.dEdG, (float4*)d.f, (float*)d.wbuf,
        d.deterministic, (float4*)d.vbuf);
}

// ---------------------------------------------------------------------------
// Adjoint for small clusters: every replica has at most 33 atoms, so n <= 32
// neighbours. Half a warp per bead-atom (two per warp); lane l of the half
// owns neighbour slots l and l + 16. The unordered pairs are walked along
// the diagonals (p, p + d mod n), d = 1 .. n/2 (for even n the last one only
// from p < n/2): each slot adds its own side of the pair in registers and
// hands the other side to slot p + d through shared memory, which every
// slot receives from exactly one sender per diagonal (no atomics). The pair
// arithmetic is that of desc_adj_kernel. A whole warp per atom would leave
// the lanes beyond n idle; these clusters have 5-23 neighbours.
// ---------------------------------------------------------------------------

constexpr int SMALL_ADJ_ATOMS = 8;   // bead-atoms per 128-thread block (shared memory under 48 KB)

template <bool FAST>
__global__ void __launch_bounds__(32 * SMALL_ADJ_ATOMS / 2) desc_adj_small_kernel(
    const float4* __restrict__ x, const int* __restrict__ ba_sys, const BeadSys* __restrict__ bsys,
    const Rep* __restrict__ reps, const int* __restrict__ nbr, const int* __restrict__ nnb, int maxnb, int B,
    DescParams<float> dp, const float* __restrict__ dEdG, float4* __restrict__ f, float* __restrict__ wbuf,
    int det, float4* __restrict__ vbuf)
{
    __shared__ float4 U[SMALL_ADJ_ATOMS][SMALL_SL], A[SMALL_ADJ_ATOMS][SMALL_SL], DA[SMALL_ADJ_ATOMS][SMALL_SL];
    __shared__ float4 KD[SMALL_ADJ_ATOMS][SMALL_SL][2];   // the other side of a pair, per receiving slot
    __shared__ float4 RGs[SMALL_ADJ_ATOMS][16];
    __shared__ float RAD[SMALL_ADJ_ATOMS][SMALL_SL];
    __shared__ float gsh[SMALL_ADJ_ATOMS][ND];
    const int hw = threadIdx.x >> 4;
    const int hl = threadIdx.x & 15;
    const unsigned hmask = 0xffffu << (16 * (hw & 1));
    const int b = blockIdx.x * SMALL_ADJ_ATOMS + hw;
    // no early return: the two halves of a warp meet in __syncwarp
    const bool live = b < B;
    int n = 0;
    BeadSys sy{0, 0, 0, 0};
    float4 xi = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (live) {
        sy = bsys[ba_sys[b]];
        n = min(nnb[b], min(maxnb, SMALL_SL));
        xi = x[b];
#pragma unroll
        for (int q = 0; q < ND / 16; ++q) gsh[hw][hl + 16 * q] = dEdG[(size_t)b * ND + hl + 16 * q];
    }
    const Rep& rp = reps[sy.rep];
    // BF16 path, evenly spaced centres: (gs_c, gs_(c+16), gs_c r_c, gs_(c+16) r_(c+16))
    // for the product recurrence of the radial sums
    const bool packed = FAST && dp.r_even;
    if (packed && live) {
        const int c = (hl >> 3) * 8 + (hl & 7);   // 0..7, 8..15
        const float ga = dEdG[(size_t)b * ND + c], gb = dEdG[(size_t)b * ND + c + 16];
        RGs[hw][hl] = make_float4(ga, gb, ga * dp.r_mu[c], gb * dp.r_mu[c + 16]);
    }
    __syncwarp();

    for (int sl = hl; sl < n; sl += 16) {
        const int j = nbr[(size_t)b * maxnb + sl];
        const float4 xj = x[sy.ba0 + j];
        float dx, dy, dz;
        pair_vec(rp, xi, xj, dx, dy, dz);
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float r = sqrtf(r2);
        const float ir = 1.0f / r;
        float fc, dfc;
        cutoff(r, dp.rc, dp.pi_over_rc, fc, dfc);
        float dEdr = 0.0f;
        if (packed) {
            // sum_c gs_c g_c (-2 eta (r - r_c) fc + dfc) = (-2 eta r fc + dfc) s1 + 2 eta fc s2,
            // s1 = sum gs_c g_c, s2 = sum gs_c r_c g_c; g_c by the recurrence of radial_gauss32
            // on the centre pairs (c, c + 16)
            float2 a1 = make_float2(0.0f, 0.0f), a2 = a1;
            const float2 rho = make_float2(dp.rec_k, dp.rec_k);
            const float dd = dp.r_delta * dp.r_delta;
#pragma unroll
            for (int qp = 0; qp < 2; ++qp) {
                const float ta = r - dp.r_mu[8 * qp], tb = r - dp.r_mu[8 * qp + 16];
                float2 e2 = make_float2(exp2f(-dp.eta_R_l2 * ta * ta), exp2f(-dp.eta_R_l2 * tb * tb));
                float2 R2 = make_float2(exp2f(dp.eta_R_l2 * fmaf(2.0f * ta, dp.r_delta, -dd)),
                                        exp2f(dp.eta_R_l2 * fmaf(2.0f * tb, dp.r_delta, -dd)));
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float4 g = RGs[hw][qp * 8 + k];
                    a1 = __ffma2_rn(e2, make_float2(g.x, g.y), a1);
                    a2 = __ffma2_rn(e2, make_float2(g.z, g.w), a2);
                    if (k < 7) {
                        e2 = __fmul2_rn(e2, R2);
                        R2 = __fmul2_rn(R2, rho);
                    }
                }
            }
            dEdr = (a1.x + a1.y) * fmaf(-2.0f * dp.eta_R * r, fc, dfc) + 2.0f * dp.eta_R * fc * (a2.x + a2.y);
        } else {
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                const float t = r - dp.r_mu[c];
                const float e = gauss<FAST>(dp.eta_R, dp.eta_R_l2, t * t);
                dEdr += gsh[hw][c] * e * (-2.0f * dp.eta_R * t * fc + dfc);
            }
        }
        float a[4], da[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float ex = gauss<FAST>(dp.eta_A[e], dp.eta_A_l2[e], r2);
            a[e] = ex * fc;
            da[e] = ex * (-2.0f * dp.eta_A[e] * r * fc + dfc);
        }
        U[hw][sl] = make_float4(dx * ir, dy * ir, dz * ir, r);
        A[hw][sl] = make_float4(a[0], a[1], a[2], a[3]);
        DA[hw][sl] = make_float4(da[0], da[1], da[2], da[3]);
        RAD[hw][sl] = dEdr;
    }
    __syncwarp();

    AdjCoef<float> gp;
    coef_load(gp, gsh[hw]);
    float jd[2][8];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int q = 0; q < 8; ++q) jd[rr][q] = 0.0f;
    for (int d = 1; 2 * d <= n; ++d) {   // uniform within the half
        const bool last = 2 * d == n;    // even n: pairs (p, p + n/2) from p < n/2 only
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int sp = hl + 16 * rr;
            if (sp < n && (!last || sp < d)) {
                int sq = sp + d;
                sq = sq >= n ? sq - n : sq;
                float kd[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) kd[q] = 0.0f;
                adj_pair(gp, U[hw][sp], A[hw][sp], U[hw][sq], A[hw][sq], jd[rr], kd);
                KD[hw][sq][0] = make_float4(kd[0], kd[1], kd[2], kd[3]);
                KD[hw][sq][1] = make_float4(kd[4], kd[5], kd[6], kd[7]);
            }
        }
        __syncwarp(hmask);
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int sp = hl + 16 * rr;
            if (sp < n && (!last || sp >= d)) {
                const float4 k0 = KD[hw][sp][0], k1 = KD[hw][sp][1];
                jd[rr][0] += k0.x; jd[rr][1] += k0.y; jd[rr][2] += k0.z; jd[rr][3] += k0.w;
                jd[rr][4] += k1.x; jd[rr][5] += k1.y; jd[rr][6] += k1.z; jd[rr][7] += k1.w;
            }
        }
        __syncwarp(hmask);
    }
    float red[12];   // force on the centre (3), virial (9)
#pragma unroll
    for (int q = 0; q < 12; ++q) red[q] = 0.0f;
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
        const int sj = hl + 16 * jj;
        if (sj < n) {
            const float4 uj = U[hw][sj];
            const float4 da = DA[hw][sj];
            const float dEdr = RAD[hw][sj] + jd[jj][0] * da.x + jd[jj][1] * da.y + jd[jj][2] * da.z + jd[jj][3] * da.w;
            const float ir = 1.0f / uj.w;
            const float v[3] = {dEdr * uj.x + (jd[jj][4] - jd[jj][7] * uj.x) * ir,
                                dEdr * uj.y + (jd[jj][5] - jd[jj][7] * uj.y) * ir,
                                dEdr * uj.z + (jd[jj][6] - jd[jj][7] * uj.z) * ir};
            if (det)
                vbuf[(size_t)b * maxnb + sj] = make_float4(v[0], v[1], v[2], 0.0f);
            else
                atomic_add_vec(&f[sy.ba0 + nbr[(size_t)b * maxnb + sj]], -v[0], -v[1], -v[2]);
            const float d3[3] = {uj.x * uj.w, uj.y * uj.w, uj.z * uj.w};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                red[a] += v[a];
#pragma unroll
                for (int c = 0; c < 3; ++c) red[3 + 3 * a + c] -= d3[a] * v[c];
            }
        }
    }
    // sums over the 16 lanes of the half
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1)
#pragma unroll
        for (int q = 0; q < 12; ++q) red[q] += __shfl_xor_sync(0xffffffffu, red[q], o);
    if (live && hl == 0) {
        if (det)
            f[b] = make_float4(red[0], red[1], red[2], 0.0f);   // gathered later
        else
            atomic_add_vec(&f[b], red[0], red[1], red[2]);
    }
    if (live && hl < 9) {
        float mine = red[3];
#pragma unroll
        for (int q = 1; q < 9; ++q)
            if (hl == q) mine = red[3 + q];
        wbuf[(size_t)b * 9 + hl] = mine;
    }
}

template <bool FAST>
static void run_adj_small(const Dev& d, const void* dpv, cudaStream_t st)
{
    desc_adj_small_kernel<FAST><<<(d.B + SMALL_ADJ_ATOMS - 1) / SMALL_ADJ_ATOMS, 16 * SMALL_ADJ_ATOMS, 0, st>>>(
        (const float4*)d.x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, d.B, *(const DescParams<float>*)dpv,
        (const float*)d.dEdG, (float4*)d.f, (float*)d.wbuf, d.deterministic, (float4*)d.vbuf);
}

bool adjoint_sums_energy(const Dev& d, const void* dpv)
{
    return d.precision != 0 && d.sched.ang && d.mom && moment_adjoint_sums_energy(d, dpv);
}

void launch_adjoint(const Dev& d, const void* dpv, cudaStream_t st)
{
    if (d.precision != 0 && d.sched.ang && d.mom) {
        launch_adjoint_moment(d, dpv, st);
        return;
    }
    if (d.precision == 0) {
        const int w = adj_warps<double>(d.maxnb);
        const size_t sm = (size_t)w * adj_smem_per_warp<double>(d.maxnb);
        { static size_t done = 0; set_smem(desc_adj_kernel<double, false>, sm, done); }
        desc_adj_kernel<double, false><<<(d.B + w - 1) / w, 32 * w, sm, st>>>(
            (const Dbl4*)d.x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, d.B,
            *(const DescParams<double>*)dpv, d.sched, (const double*)d.dEdG, (Dbl4*)d.f, (double*)d.wbuf,
            d.deterministic, (Dbl4*)d.vbuf);
    } else if (d.max_N <= SMALL_SL + 1) {
        if (d.precision == 2) run_adj_small<true>(d, dpv, st);
        else run_adj_small<false>(d, dpv, st);
    } else if (d.precision == 2) {
        run_adj_f32<true>(d, dpv, st);
    } else {
        run_adj_f32<false>(d, dpv, st);
    }
}

// ---------------------------------------------------------------------------
// a4 on CUDA cores: per-element network forward and input gradient for a
// tile of TM rows of one element. Activations of every layer stay in shared
// memory, k-major ([feature][row]), so that a thread's rows are contiguous;
// weight chunks of 32 along K pass through two shared-memory buffers; each
// thread holds an RT x CT block of the layer's output in registers.
// ---------------------------------------------------------------------------
size_t blob_elems(int n_hidden, const int* widths)
{
    size_t o = 0;
    int prev = ND;
    for (int l = 0; l < n_hidden; ++l) {
        o += (size_t)widths[l] * prev + widths[l];
        prev = widths[l];
    }
    return o + prev + 1 + 2 * ND + 2;
}

constexpr int KC_WIDE = 32;   // K chunk of the weights staged per step (one CTA per SM)
constexpr int KC_PAIR = 8;    // the same for two CTAs per SM (less shared memory)
constexpr size_t PAIR_SMEM_MAX = 113 * 1024;   // two CTAs per SM: 228 KB less 1 KB reserved per CTA
constexpr int APAD = 4;  // row padding of the k-major activation tiles (keeps 16-byte alignment)

// N consecutive values at p (16-byte aligned when N * sizeof(Real) >= 16)
template <typename Real, int N>
__device__ __forceinline__ void ld_vec(const Real* __restrict__ p, Real (&v)[N])
{
    if constexpr (sizeof(Real) == 4 && N % 4 == 0) {
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            const float4 x = reinterpret_cast<const float4*>(p)[q];
            v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
        }
    } else if constexpr (N % 2 == 0) {
        using V2 = typename std::conditional<sizeof(Real) == 4, float2, double2>::type;
#pragma unroll
        for (int q = 0; q < N / 2; ++q) {
            const V2 x = reinterpret_cast<const V2*>(p)[q];
            v[2 * q] = x.x; v[2 * q + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) v[q] = p[q];
    }
}

template <typename Real, int N>
__device__ __forceinline__ void st_vec(Real* __restrict__ p, const Real (&v)[N])
{
    if constexpr (sizeof(Real) == 4 && N % 4 == 0) {
#pragma unroll
        for (int q = 0; q < N / 4; ++q)
            reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) p[q] = v[q];
    }
}

// Column m of thread tx in a tile product: groups of 4 consecutive columns,
// the threads' groups side by side (16 threads x 4 columns = 64), so that a
// 16-byte load by the 16 column threads reads 256 contiguous bytes.
__device__ __forceinline__ int tile_col(int tx, int m) { return (m >> 2) * 64 + tx * 4 + (m & 3); }

// Register-blocked tile product out[TM][NOUT] = A[TM][K] Bmat[K][NOUT] with
// A stored k-major in shared memory (A(r, k) = At[k * lda + r]) and
// Bmat(k, o) = W[o * ldw + k] when transB (forward: W is [out][in]), else
// W[k * ldw + o] (backward). 256 threads as 16 row groups x 16 column
// groups: thread (ty, tx) owns the contiguous rows ty RT .. and the columns
// tile_col(tx, m), so per k it loads RT + CT values as 16-byte vectors and
// issues RT x CT multiply-adds. The weights pass through two shared-memory buffers
// of KC rows: while a chunk is multiplied, each thread holds its share of
// the next chunk in registers and stores it into the other buffer after, so
// the global loads overlap the arithmetic (one barrier per chunk).
template <typename Real, int RT, int CT, bool transB, int KC>
__device__ __forceinline__ void tile_gemm(const Real* __restrict__ At, int lda, int K, const Real* __restrict__ W,
                                          int ldw, Real* __restrict__ Bs, Real (&acc)[RT][CT])
{
    constexpr int NOUT = 16 * CT;
    constexpr int ldb = NOUT + APAD;
    constexpr int PER = KC * NOUT / 256;   // chunk elements per thread
    static_assert(PER * 256 == KC * NOUT, "chunk split over the threads");
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int m = 0; m < CT; ++m) acc[i][m] = Real(0);
    Real pre[PER];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + 256 * q;
            if (transB) {
                const int o = e / KC, kk = e - o * KC;
                pre[q] = W[(size_t)o * ldw + k0 + kk];
            } else {
                const int kk = e / NOUT, o = e - kk * NOUT;
                pre[q] = W[(size_t)(k0 + kk) * ldw + o];
            }
        }
    };
    auto stash = [&](Real* buf) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + 256 * q;
            if (transB) {
                const int o = e / KC, kk = e - o * KC;
                buf[kk * ldb + o] = pre[q];
            } else {
                const int kk = e / NOUT, o = e - kk * NOUT;
                buf[kk * ldb + o] = pre[q];
            }
        }
    };
    __syncthreads();   // earlier readers of the buffers and of At's producers are done
    fetch(0);
    stash(Bs);
    __syncthreads();
    int cur = 0;
    for (int k0 = 0; k0 < K; k0 += KC) {
        const bool more = k0 + KC < K;
        if (more) fetch(k0 + KC);
        const Real* B0 = Bs + cur * KC * ldb;
#pragma unroll 4
        for (int kk = 0; kk < KC; ++kk) {
            Real a[RT], b[CT];
            ld_vec<Real, RT>(At + (size_t)(k0 + kk) * lda + ty * RT, a);
#pragma unroll
            for (int g = 0; g < CT / 4; ++g) {
                Real b4[4];
                ld_vec<Real, 4>(B0 + kk * ldb + g * 64 + tx * 4, b4);
#pragma unroll
                for (int j = 0; j < 4; ++j) b[4 * g + j] = b4[j];
            }
#pragma unroll
            for (int i = 0; i < RT; ++i)
#pragma unroll
                for (int m = 0; m < CT; ++m) acc[i][m] = fma(a[i], b[m], acc[i][m]);
        }
        if (more) stash(Bs + (cur ^ 1) * KC * ldb);
        __syncthreads();
        cur ^= 1;
    }
}

__device__ __forceinline__ float f_tanh(float v) { return tanhf(v); }
__device__ __forceinline__ double f_tanh(double v) { return tanh(v); }

// PAIR: two CTAs per SM. The weights then pass in chunks of KC_PAIR rows and
// the input tile h_0 shares the buffer of the last hidden layer (h_0 is read
// only by layer 1, whose reads end at the product's last barrier, before any
// layer writes its output), which brings a 64-row tile of width 128 to
// 110 KB of shared memory.
template <typename Real, int RT, int CT, bool PAIR>
struct FpTile {
    static constexpr int TM = RT * 16;
    static constexpr int Wd = CT * 16;          // hidden width
    static constexpr int lda = TM + APAD;       // activations are k-major: [feature][row]
    static constexpr int BW = (Wd > ND ? Wd : ND) + APAD;
    static constexpr int KC = PAIR ? KC_PAIR : KC_WIDE;
    static size_t smem(int n_hidden)
    {
        const size_t h0 = PAIR ? 0 : (size_t)ND * lda;
        return sizeof(Real) * (h0 + (size_t)n_hidden * Wd * lda + (size_t)2 * KC * BW + TM);
    }
};

template <typename Real, int RT, int CT, bool PAIR>
__global__ void __launch_bounds__(256, PAIR ? 2 : 1) mlp_fp_kernel(
    const Real* __restrict__ G, const int* __restrict__ perm, const int* __restrict__ tile_type,
    const Real* __restrict__ wts, size_t blob, int n_hidden, Real* __restrict__ Eatom, Real* __restrict__ dEdG)
{
    using Tl = FpTile<Real, RT, CT, PAIR>;
    constexpr int TM = Tl::TM, Wd = Tl::Wd, lda = Tl::lda, BW = Tl::BW, KC = Tl::KC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real* base = reinterpret_cast<Real*>(smem_raw);
    Real* Hl = PAIR ? base : base + ND * lda;                 // [n_hidden][Wd][lda]
    Real* H0 = PAIR ? Hl + (size_t)(n_hidden - 1) * Wd * lda : base;   // [ND][lda]
    Real* Bs = Hl + (size_t)n_hidden * Wd * lda;              // [2][KC][BW]
    Real* yv = Bs + 2 * KC * BW;                              // [TM]
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int row0 = blockIdx.x * TM;
    const int type = tile_type[row0 / TILE_ROWS];
    const Real* P = wts + (size_t)type * blob;
    // blob pieces
    const Real* Wl[MAX_LAYERS];
    const Real* bl[MAX_LAYERS];
    size_t off = 0;
    int prev = ND;
    for (int l = 0; l < n_hidden; ++l) {
        Wl[l] = P + off; off += (size_t)Wd * prev;
        bl[l] = P + off; off += Wd;
        prev = Wd;
    }
    const Real* w_out = P + off; off += Wd;
    const Real b_out = P[off]; off += 1;
    const Real* mu = P + off; off += ND;
    const Real* sigma = P + off; off += ND;
    const Real s_E = P[off], e_Z = P[off + 1];

    // h_0 = (G - mu) / sigma, stored k-major
    for (int e = tid; e < TM * ND; e += 256) {
        const int r = e / ND, c = e - r * ND;
        const int ba = perm[row0 + r];
        H0[c * lda + r] = ba >= 0 ? (G[(size_t)ba * ND + c] - mu[c]) / sigma[c] : Real(0);
    }
    // forward through the hidden layers
    for (int l = 0; l < n_hidden; ++l) {
        const Real* Ain = (l == 0) ? H0 : Hl + (size_t)(l - 1) * Wd * lda;
        const int K = (l == 0) ? ND : Wd;
        Real acc[RT][CT];
        tile_gemm<Real, RT, CT, true, KC>(Ain, lda, K, Wl[l], K, Bs, acc);
        Real* Hout = Hl + (size_t)l * Wd * lda;
#pragma unroll
        for (int m = 0; m < CT; ++m) {
            const int o = tile_col(tx, m);
            const Real bo = bl[l][o];
            Real v[RT];
#pragma unroll
            for (int i = 0; i < RT; ++i) v[i] = f_tanh(acc[i][m] + bo);
            st_vec<Real, RT>(Hout + (size_t)o * lda + ty * RT, v);
        }
    }
    __syncthreads();
    Real* HL = Hl + (size_t)(n_hidden - 1) * Wd * lda;
    // output layer: y = w_out . h_L + b_out, 256 / TM threads per row
    {
        constexpr int TPR = 256 / TM;   // threads per row (a power of two)
        const int r = tid / TPR, part = tid - r * TPR;
        Real y = Real(0);
        for (int k = part; k < Wd; k += TPR) y += w_out[k] * HL[k * lda + r];
#pragma unroll
        for (int o = TPR / 2; o >= 1; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
        if (part == 0) {
            y += b_out;
            yv[r] = y;
            const int ba = perm[row0 + r];
            if (ba >= 0) Eatom[ba] = s_E * y + e_Z;
        }
    }
    __syncthreads();
    // dE/da_L = s_E w_out (1 - h_L^2), written over h_L
    for (int e = tid; e < TM * Wd; e += 256) {
        const int k = e / TM, r = e - k * TM;
        const Real h = HL[k * lda + r];
        HL[k * lda + r] = s_E * w_out[k] * (Real(1) - h * h);
    }
    // backward: dE/dh_{l-1} = W_l^T dE/da_l, times tanh' of layer l-1
    for (int l = n_hidden - 1; l >= 0; --l) {
        const Real* Ga = Hl + (size_t)l * Wd * lda;
        if (l > 0) {
            Real acc[RT][CT];
            tile_gemm<Real, RT, CT, false, KC>(Ga, lda, Wd, Wl[l], Wd, Bs, acc);
            Real* Hp = Hl + (size_t)(l - 1) * Wd * lda;
#pragma unroll
            for (int m = 0; m < CT; ++m) {
                const int k = tile_col(tx, m);
                Real h[RT];
                ld_vec<Real, RT>(Hp + (size_t)k * lda + ty * RT, h);
#pragma unroll
                for (int i = 0; i < RT; ++i) h[i] = acc[i][m] * (Real(1) - h[i] * h[i]);
                st_vec<Real, RT>(Hp + (size_t)k * lda + ty * RT, h);
            }
        } else {
            constexpr int C0 = ND / 16;
            Real acc[RT][C0];
            tile_gemm<Real, RT, C0, false, KC>(Ga, lda, Wd, Wl[0], ND, Bs, acc);
            static_assert(C0 == 4, "one group of 4 descriptor columns per thread");
            Real is[C0];
#pragma unroll
            for (int m = 0; m < C0; ++m) is[m] = Real(1) / sigma[tile_col(tx, m)];
#pragma unroll
            for (int i = 0; i < RT; ++i) {
                const int ba = perm[row0 + ty * RT + i];
                if (ba < 0) continue;
                Real v[C0];
#pragma unroll
                for (int m = 0; m < C0; ++m) v[m] = acc[i][m] * is[m];
                st_vec<Real, C0>(dEdG + (size_t)ba * ND + tx * C0, v);
            }
        }
    }
}

template <typename Real, int RT, int CT, bool PAIR>
static void run_mlp_fp(const Dev& d, cudaStream_t st)
{
    using Tl = FpTile<Real, RT, CT, PAIR>;
    const size_t sm = Tl::smem(d.n_hidden);
    static size_t done = 0;
    set_smem(mlp_fp_kernel<Real, RT, CT, PAIR>, sm, done);
    mlp_fp_kernel<Real, RT, CT, PAIR><<<d.rows_pad / Tl::TM, 256, sm, st>>>(
        (const Real*)d.G, d.perm, d.tile_type, (const Real*)d.wts, d.blob, d.n_hidden, (Real*)d.Eatom,
        (Real*)d.dEdG);
}

template <typename Real, int CT>
static void dispatch_rows(const Dev& d, cudaStream_t st)
{
    // 64-row tiles two per SM when they fit in half the shared memory (width
    // 128 in FP32), else the largest row tile that fits in ~200 KB, one per SM
    if (FpTile<Real, 4, CT, true>::smem(d.n_hidden) <= PAIR_SMEM_MAX)
        run_mlp_fp<Real, 4, CT, true>(d, st);
    else if (FpTile<Real, 4, CT, false>::smem(d.n_hidden) <= 200 * 1024)
        run_mlp_fp<Real, 4, CT, false>(d, st);
    else if (FpTile<Real, 2, CT, false>::smem(d.n_hidden) <= 200 * 1024)
        run_mlp_fp<Real, 2, CT, false>(d, st);
    else
        run_mlp_fp<Real, 1, CT, false>(d, st);
}

void launch_network_fp(const Dev& d, cudaStream_t st)
{
    if (d.precision == 0) {
        switch (d.width) {
            case 64: dispatch_rows<double, 4>(d, st); break;
            case 128: dispatch_rows<double, 8>(d, st); break;
            default: dispatch_rows<double, 16>(d, st); break;
        }
    } else {
        switch (d.width) {
            case 64: dispatch_rows<float, 4>(d, st); break;
            case 128: dispatch_rows<float, 8>(d, st); break;
            default: dispatch_rows<float, 16>(d, st); break;
        }
    }
}

// ---------------------------------------------------------------------------
// a6: per-bead energy V_k = sum_i E_i, FP64 sum in a fixed order (one warp
// per bead).
// ---------------------------------------------------------------------------
// (hi, lo) += v with Knuth's TwoSum: hi + lo holds the running sum of FP32
// terms to ~2^-48 relative, on the FP32 pipes (FP64 runs at 2 lanes per SM
// per clock on this GPU, which made the FP64 butterflies of many small beads
// the cost of the whole reduction)
__device__ __forceinline__ void df_add(float& hi, float& lo, float v)
{
    const float s = __fadd_rn(hi, v);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(v, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

template <typename Real>
__global__ void __launch_bounds__(256) energy_reduce_kernel(const Real* __restrict__ Eatom,
                                                            const Real* __restrict__ wbuf,
                                                            const BeadSys* __restrict__ bsys, int S, int wpb,
                                                            int lpb, double* __restrict__ V,
                                                            double* __restrict__ Wv)
{
    // The energy and the 9 virial entries of a bead summed over its atoms in
    // a fixed order: atoms strided over the bead's lanes, a fixed butterfly
    // within the bead's lanes, the warps' partials in warp order. Large
    // beads take wpb warps (8 / wpb beads per 256-thread block); small ones
    // share a warp, lpb lanes each (a power of two <= 32; lpb = 32 when
    // wpb > 1). FP64 terms in FP64; FP32 terms as double-float pairs,
    // rounded to FP64 at the end.
    __shared__ double part[8][10][2];
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int gl = (int)lane & (lpb - 1);
    const int s = (blockIdx.x * (8 / wpb) + w / wpb) * (32 / lpb) + (int)lane / lpb, sub = w % wpb;
    const bool live = s < S;
    const BeadSys sy = live ? bsys[s] : BeadSys{0, 0, 0, 0};
    double hi[10], lo[10];
    if constexpr (std::is_same<Real, double>::value) {
#pragma unroll
        for (int q = 0; q < 10; ++q) hi[q] = lo[q] = 0.0;
        for (int i = sub * lpb + gl; i < sy.N; i += lpb * wpb) {
            const size_t b = (size_t)(sy.ba0 + i);
            hi[0] += Eatom[b];
#pragma unroll
            for (int q = 0; q < 9; ++q) hi[1 + q] += wbuf[b * 9 + q];
        }
        for (int o = lpb >> 1; o >= 1; o >>= 1)
#pragma unroll
            for (int q = 0; q < 10; ++q) {
                // both partners add in the same order (lower lane's value first)
                const double oh = __shfl_xor_sync(0xffffffffu, hi[q], o);
                hi[q] = ((int)lane & o) ? oh + hi[q] : hi[q] + oh;
            }
    } else {
        float fh[10], fl[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) fh[q] = fl[q] = 0.0f;
        for (int i = sub * lpb + gl; i < sy.N; i += lpb * wpb) {
            const size_t b = (size_t)(sy.ba0 + i);
            df_add(fh[0], fl[0], (float)Eatom[b]);
#pragma unroll
            for (int q = 0; q < 9; ++q) df_add(fh[1 + q], fl[1 + q], (float)wbuf[b * 9 + q]);
        }
        for (int o = lpb >> 1; o >= 1; o >>= 1)
#pragma unroll
            for (int q = 0; q < 10; ++q) {
                const float oh = __shfl_xor_sync(0xffffffffu, fh[q], o);
                const float ol = __shfl_xor_sync(0xffffffffu, fl[q], o);
                // both partners add in the same order (lower lane's pair first)
                const bool upper = (lane & o) != 0;
                float h = upper ? oh : fh[q], l = upper ? ol : fl[q];
                df_add(h, l, upper ? fh[q] : oh);
                l = __fadd_rn(l, upper ? fl[q] : ol);
                fh[q] = h;
                fl[q] = l;
            }
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            hi[q] = (double)fh[q];
            lo[q] = (double)fl[q];
        }
    }
    if (wpb > 1) {
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 10; ++q) {
                part[w][q][0] = hi[q];
                part[w][q][1] = lo[q];
            }
        }
        __syncthreads();
        if (sub != 0 || !live) return;
        if (lane < 10) {
            double h = 0.0, l = 0.0;
            for (int t = 0; t < wpb; ++t) {
                h += part[w + t][lane][0];
                l += part[w + t][lane][1];
            }
            const double tot = h + l;
            if (lane == 0) V[s] = tot;
            else Wv[(size_t)s * 9 + lane - 1] = tot;
        }
        return;
    }
    if (!live || gl != 0) return;
    V[s] = hi[0] + lo[0];
#pragma unroll
    for (int q = 1; q < 10; ++q) Wv[(size_t)s * 9 + q - 1] = hi[q] + lo[q];
}

void launch_energy_reduce(const Dev& d, cudaStream_t st)
{
    // warps per bead from the largest bead: one up to 64 atoms, up to 8;
    // beads of at most 64 atoms share a warp, about 4 atoms per lane
    const int wpb = d.max_N <= 64 ? 1 : d.max_N <= 256 ? 2 : d.max_N <= 1024 ? 4 : 8;
    int lpb = 32;
    if (wpb == 1)
        while (lpb > 4 && 4 * (lpb / 2) >= d.max_N) lpb >>= 1;
    const int bpb = 8 / wpb * (32 / lpb);
    const int blocks = (d.S + bpb - 1) / bpb;
    if (d.precision == 0)
        energy_reduce_kernel<double><<<blocks, 256, 0, st>>>((const double*)d.Eatom, (const double*)d.wbuf, d.bsys, d.S,
                                                             wpb, lpb, d.V, d.W);
    else
        energy_reduce_kernel<float><<<blocks, 256, 0, st>>>((const float*)d.Eatom, (const float*)d.wbuf, d.bsys, d.S,
                                                            wpb, lpb, d.V, d.W);
}

// ---------------------------------------------------------------------------
// harmonic test potential V = sum_i 1/2 m_i omega^2 |x_i|^2 (Sec. S1)
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void harmonic_kernel(const Vec4<Real>* __restrict__ x, const int* __restrict__ ba_sys,
                                const BeadSys* __restrict__ bsys, const Rep* __restrict__ reps,
                                const double* __restrict__ mass, int B, double omega, Real* __restrict__ Eatom,
                                Vec4<Real>* __restrict__ f, Real* __restrict__ wbuf)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int s = ba_sys[b];
    const BeadSys sy = bsys[s];
    const Rep& rp = reps[sy.rep];
    const double m = mass[rp.atom0 + (b - sy.ba0) % sy.N];
    const double k = m * omega * omega * MVV2E;
    const double p[3] = {(double)x[b].x, (double)x[b].y, (double)x[b].z};
    Eatom[b] = (Real)(0.5 * k * (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]));
    Vec4<Real> fv;
    fv.x = (Real)(-k * p[0]);
    fv.y = (Real)(-k * p[1]);
    fv.z = (Real)(-k * p[2]);
    fv.w = Real(0);
    f[b] = fv;
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) wbuf[(size_t)b * 9 + 3 * a + c] = (Real)(-k * p[a] * p[c]);
}

void launch_harmonic(const Dev& d, cudaStream_t st)
{
    const int blocks = (d.B + 255) / 256;
    if (d.precision == 0)
        harmonic_kernel<double><<<blocks, 256, 0, st>>>((const Dbl4*)d.x, d.ba_sys, d.bsys, d.reps, d.mass, d.B,
                                                        d.omega_harm, (double*)d.Eatom, (Dbl4*)d.f, (double*)d.wbuf);
    else
        harmonic_kernel<float><<<blocks, 256, 0, st>>>((const float4*)d.x, d.ba_sys, d.bsys, d.reps, d.mass, d.B,
                                                       d.omega_harm, (float*)d.Eatom, (float4*)d.f, (float*)d.wbuf);
}

// ---------------------------------------------------------------------------
// boundary conversions (FP64 [B][3] <-> internal 4-wide records)
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void pack_kernel(const double* __restrict__ x3, Vec4<Real>* __restrict__ x, int B)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    Vec4<Real> v = x[b];
    v.x = (Real)x3[3 * (size_t)b];
    v.y = (Real)x3[3 * (size_t)b + 1];
    v.z = (Real)x3[3 * (size_t)b + 2];
    x[b] = v;
}

void launch_pack_positions(const Dev& d, const double* x3, cudaStream_t st)
{
    const int blocks = (d.B + 255) / 256;
    if (d.precision == 0)
        pack_kernel<double><<<blocks, 256, 0, st>>>(x3, (Dbl4*)d.x, d.B);
    else
        pack_kernel<float><<<blocks, 256, 0, st>>>(x3, (float4*)d.x, d.B);
}

// external bead forces [B][3] FP64 into the force records
void launch_pack_forces(const Dev& d, const double* f3, cudaStream_t st)
{
    const int blocks = (d.B + 255) / 256;
    if (d.precision == 0)
        pack_kernel<double><<<blocks, 256, 0, st>>>(f3, (Dbl4*)d.f, d.B);
    else
        pack_kernel<float><<<blocks, 256, 0, st>>>(f3, (float4*)d.f, d.B);
}

template <typename Real>
__global__ void unpack_kernel(const Vec4<Real>* __restrict__ f, const Vec4<Real>* __restrict__ x,
                              const double* __restrict__ V, const double* __restrict__ Wv, int B, int S,
                              double* __restrict__ f3, double* __restrict__ e, double* __restrict__ vir,
                              double* __restrict__ x3)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B) {
        if (f3) {
            const Vec4<Real> v = f[i];
            f3[3 * (size_t)i] = v.x;
            f3[3 * (size_t)i + 1] = v.y;
            f3[3 * (size_t)i + 2] = v.z;
        }
        if (x3) {
            const Vec4<Real> v = x[i];
            x3[3 * (size_t)i] = v.x;
            x3[3 * (size_t)i + 1] = v.y;
            x3[3 * (size_t)i + 2] = v.z;
        }
    }
    if (i < S) {
        if (e) e[i] = V[i];
        if (vir)
            for (int q = 0; q < 9; ++q) vir[9 * (size_t)i + q] = Wv[9 * (size_t)i + q];
    }
}

void launch_unpack(const Dev& d, double* f3, double* e, double* vir, double* x3, cudaStream_t st)
{
    const int n = d.B > d.S ? d.B : d.S;
    const int blocks = (n + 255) / 256;
    if (d.precision == 0)
        unpack_kernel<double><<<blocks, 256, 0, st>>>((const Dbl4*)d.f, (const Dbl4*)d.x, d.V, d.W, d.B, d.S, f3, e,
                                                      vir, x3);
    else
        unpack_kernel<float><<<blocks, 256, 0, st>>>((const float4*)d.f, (const float4*)d.x, d.V, d.W, d.B, d.S, f3,
                                                     e, vir, x3);
}

template <typename Real>
__global__ void desc_out_kernel(const Real* __restrict__ G, double* __restrict__ out, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)G[i];
}

void launch_descriptors_out(const Dev& d, double* G, cudaStream_t st)
{
    const size_t n = (size_t)d.B * ND;
    const int blocks = (int)((n + 255) / 256);
    if (d.precision == 0)
        desc_out_kernel<double><<<blocks, 256, 0, st>>>((const double*)d.G, G, n);
    else
        desc_out_kernel<float><<<blocks, 256, 0, st>>>((const float*)d.G, G, n);
}

}  // namespace pimd
