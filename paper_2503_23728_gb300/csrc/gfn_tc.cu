// gfn_tc.cu -- the graph-field-network force head (Sec. 2.2) with its dense
// layers on the 5th-gen tensor cores (tcgen05.mma kind::f16, BF16 operands,
// FP32 accumulators in tensor memory); the same equations as gfn.cu.
//
// Every kernel works on tiles of 128 rows, one row per thread and per
// tensor-memory lane: the neighbour slots of one bead-atom (edge kernels) or
// 128 bead-atoms (node update). Thread 0 streams each layer's BF16 weight
// image ([out][in], K-major core-matrix layout) into one shared buffer with a
// bulk copy and issues the MMAs; the threads stage the A operand (rows
// rounded to BF16) and run the epilogues from tensor memory. Edge states e
// and node states n stay FP32 in the workspace; messages are summed over the
// rows of a tile by transposed shuffles. Every wait on an mbarrier is
// bounded (ERR_TIMEOUT, then the tensor memory is released).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "common.cuh"
#include "geom.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace pimd {

namespace {

constexpr int TR = 128;   // rows per tile = threads per CTA

__device__ __forceinline__ uint32_t bf2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

__device__ __forceinline__ float silu_f(float v) { return v / (1.0f + __expf(-v)); }

// 8 FP32 values -> one 16-byte chunk of row r, columns k0..k0+7, of a
// [TR][K] BF16 operand in the core-matrix layout
__device__ __forceinline__ void put8(unsigned char* A, int r, int k0, int K, const float (&v)[8])
{
    *reinterpret_cast<uint4*>(A + 2 * cm_index(r, k0, K)) =
        make_uint4(bf2(v[0], v[1]), bf2(v[2], v[3]), bf2(v[4], v[5]), bf2(v[6], v[7]));
}

// 16 per-lane values: lanes c and c + 16 end with the warp sum of v[c]
__device__ __forceinline__ float tr_reduce16(float (&v)[16], unsigned lane)
{
#pragma unroll
    for (int o = 8, n = 16; o >= 1; o >>= 1, n >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < n / 2; ++q) {
            const float send = upper ? v[q] : v[q + n / 2];
            const float keep = upper ? v[q + n / 2] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// CTA scaffolding shared by the kernels: two mbarriers (weights, MMA), the
// tensor-memory allocation, phase counters and the bounded waits
struct Tc {
    uint32_t bar_w, bar_mma, tmem;
    uint32_t wph = 0, mph = 0;
    int issued_w = 0;   // weight copies issued
    int mmas = 0;       // MMA groups committed
    bool ok = true;
};

__device__ __forceinline__ void tc_begin(Tc& t, uint64_t* bars, uint32_t* tslot, uint32_t cols)
{
    t.bar_w = smem_u32(&bars[0]);
    t.bar_mma = smem_u32(&bars[1]);
    if (threadIdx.x == 0) {
        mbar_init(t.bar_w, 1);
        mbar_init(t.bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    t.tmem = *tslot;
}

__device__ __forceinline__ void tc_load_w(Tc& t, unsigned char* WB, const unsigned char* src, uint32_t bytes)
{
    if (threadIdx.x == 0) {
        bulk_load(smem_u32(WB), src, bytes, t.bar_w);
        ++t.issued_w;
    }
}

// D = A W^T for an A of TR x K and the N x K weight image in WB; all threads
// return after the MMA has completed (or a wait gave up: t.ok false)
__device__ __forceinline__ void tc_gemm(Tc& t, const unsigned char* A, const unsigned char* WB, int N, int K)
{
    fence_proxy();
    fence_before();
    __syncthreads();
    fence_after();
    bool good = true;
    if (threadIdx.x == 0) {
        good = mbar_wait(t.bar_w, t.wph & 1u);
        if (good) {
            fence_after();
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(WB);
            const uint32_t sbo = (uint32_t)(K / 8) * 128u;
            const uint32_t idesc = make_idesc(TR, N);
            for (int ks = 0; ks < K / 16; ++ks)
                mma_f16(t.tmem, make_desc(a0 + ks * 256u, 128u, sbo), make_desc(b0 + ks * 256u, 128u, sbo), idesc,
                        ks > 0 ? 1u : 0u);
            mma_commit(t.bar_mma);
            ++t.mmas;
        }
    }
    ++t.wph;
    good = mbar_wait(t.bar_mma, t.mph & 1u) && good;
    ++t.mph;
    t.ok = __syncthreads_and(good ? 1 : 0) != 0 && t.ok;
    fence_after();
}

__device__ __forceinline__ void tc_end(Tc& t, uint32_t cols, DevErr* err)
{
    if (!t.ok && threadIdx.x == 0) {
        // let the last copy and MMA finish (bounded) before the memory goes
        atomicOr(&err->flags, ERR_TIMEOUT);
        if (t.issued_w > 0) mbar_wait(t.bar_w, (uint32_t)(t.issued_w - 1) & 1u);
        if (t.mmas > 0) mbar_wait(t.bar_mma, (uint32_t)(t.mmas - 1) & 1u);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t.tmem), "r"(cols) : "memory");
}

template <int F>
__host__ __device__ constexpr uint32_t tcols() { return F < 32 ? 32u : (uint32_t)F; }

// thread row r of the tile: its tensor-memory lane base
__device__ __forceinline__ uint32_t lane_base(const Tc& t) { return t.tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16); }

}  // namespace

// e^(0) = W_e rho(r) + b_e on the rows of one bead-atom, n^(0) = emb
template <int F>
__global__ void __launch_bounds__(TR, 2) gfn_tc_init_kernel(
    const float4* __restrict__ x, const int* __restrict__ ba_sys, const BeadSys* __restrict__ bsys,
    const Rep* __restrict__ reps, const int* __restrict__ atype, const int* __restrict__ nbr,
    const int* __restrict__ nnb, int maxnb, GfnParams gp, const float* __restrict__ W,
    const unsigned char* __restrict__ Wtc, float* __restrict__ nf, float* __restrict__ ef,
    float* __restrict__ Eatom, DevErr* __restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A = sm;                       // [TR][NR] BF16
    unsigned char* WB = A + TR * NR * 2;         // [F][NR] BF16
    uint64_t* bars = reinterpret_cast<uint64_t*>(WB + F * NR * 2);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
    Tc t;
    tc_begin(t, bars, tslot, tcols<F>());
    const int b = blockIdx.x, row = threadIdx.x;
    const BeadSys sy = bsys[ba_sys[b]];
    const Rep rp = reps[sy.rep];
    const int n = min(nnb[b], maxnb);
    const float4 xi = x[b];
    {
        const int ty = atype[rp.atom0 + (b - sy.ba0)];
        for (int c = row; c < F; c += TR) nf[(size_t)b * F + c] = W[gp.o_emb + (size_t)ty * F + c];
        if (row == 0) Eatom[b] = 0.0f;
    }
    float* eb = ef + (size_t)b * maxnb * F;
    for (int t0 = 0; t0 < n && t.ok; t0 += TR) {
        tc_load_w(t, WB, Wtc + gp.t_We, (uint32_t)(F * NR * 2));
        const int s = t0 + row;
        const bool act = s < n;
        float rho[NR];
        if (act) {
            float dx, dy, dz;
            pair_vec(rp, xi, x[sy.ba0 + nbr[(size_t)b * maxnb + s]], dx, dy, dz);
            const float r = sqrtf(dx * dx + dy * dy + dz * dz);
            float fc, dfc;
            cutoff(r, gp.rc, gp.pi_over_rc, fc, dfc);
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const float tt = r - gp.r_mu[k];
                rho[k] = __expf(-gp.eta_R * tt * tt) * fc;
            }
        } else {
#pragma unroll
            for (int k = 0; k < NR; ++k) rho[k] = 0.0f;
        }
#pragma unroll
        for (int k0 = 0; k0 < NR; k0 += 8) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = rho[k0 + q];
            put8(A, row, k0, NR, v);
        }
        tc_gemm(t, A, WB, F, NR);
        if (!t.ok) break;
        for (int c0 = 0; c0 < F; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base(t) + (uint32_t)c0, v);
            if (act) {
                float4* dst = reinterpret_cast<float4*>(eb + (size_t)s * F + c0);
                const float4* bb = reinterpret_cast<const float4*>(W + gp.o_be + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 bv = bb[q];
                    dst[q] = make_float4(v[4 * q] + bv.x, v[4 * q + 1] + bv.y, v[4 * q + 2] + bv.z, v[4 * q + 3] + bv.w);
                }
            }
        }
    }
    tc_end(t, tcols<F>(), err);
}

// iteration l on the rows of one bead-atom: m_i = sum_rows SiLU(W_m e + b_m);
// e += W_a2 SiLU(W_a1 (n_i + n_j) + b_a1) + b_a2. One A buffer (e, then
// n_i + n_j, then the hidden layer), so three CTAs share an SM; rows are
// staged and the residual is added by whole warps on contiguous rows.
template <int F>
__global__ void __launch_bounds__(TR, 3) gfn_tc_iter_kernel(
    const int* __restrict__ ba_sys, const BeadSys* __restrict__ bsys, const int* __restrict__ nbr,
    const int* __restrict__ nnb, int maxnb, GfnParams gp, int l, const float* __restrict__ W,
    const unsigned char* __restrict__ Wtc, const float* __restrict__ nf, float* __restrict__ mf,
    float* __restrict__ ef, DevErr* __restrict__ err)
{
    constexpr int CPR = F / 8;                   // 16-byte BF16 chunks per row
    constexpr int HC = F / 4;                    // columns of the FP32 staging of D per pass
    constexpr int HCS = HC + 4;                  // its row stride (floats): 16-byte stores conflict-free
    static_assert(TR * HCS * 4 <= TR * F * 2, "the FP32 staging of D fits the A buffer");
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A = sm;                       // [TR][F] BF16; also [TR][HCS] FP32
    unsigned char* WB = A + TR * F * 2;          // [F][F] BF16
    float* msum = reinterpret_cast<float*>(WB + F * F * 2);   // [4][F]
    int* jrow = reinterpret_cast<int*>(msum + 4 * F);          // [TR] neighbour of each row, -1 beyond the list
    uint64_t* bars = reinterpret_cast<uint64_t*>(jrow + TR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
    Tc t;
    tc_begin(t, bars, tslot, tcols<F>());
    const int b = blockIdx.x, row = threadIdx.x, warp = row >> 5;
    const unsigned lane = lane_id();
    const BeadSys sy = bsys[ba_sys[b]];
    const int n = min(nnb[b], maxnb);
    const unsigned* o = gp.o_it[l];
    const uint32_t wbytes = (uint32_t)(F * F * 2);
    float* eb = ef + (size_t)b * maxnb * F;
    const float* ni = nf + (size_t)b * F;
    for (int c = row; c < 4 * F; c += TR) msum[c] = 0.0f;
    for (int t0 = 0; t0 < n && t.ok; t0 += TR) {
        tc_load_w(t, WB, Wtc + gp.t_it[l][0], wbytes);
        const int s = t0 + row;
        const bool act = s < n;
        jrow[row] = act ? nbr[(size_t)b * maxnb + s] : -1;
        __syncthreads();
        // A = e rows (a warp stages its 32 rows, consecutive lanes on consecutive chunks)
        for (int q = (int)lane; q < 32 * CPR; q += 32) {
            const int r = 32 * warp + q / CPR, k0 = 8 * (q % CPR);
            float v[8];
            if (jrow[r] >= 0) {
                const float4* src = reinterpret_cast<const float4*>(eb + (size_t)(t0 + r) * F + k0);
                const float4 p0 = src[0], p1 = src[1];
                v[0] = p0.x; v[1] = p0.y; v[2] = p0.z; v[3] = p0.w; v[4] = p1.x; v[5] = p1.y; v[6] = p1.z; v[7] = p1.w;
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = 0.0f;
            }
            put8(A, r, k0, F, v);
        }
        // messages
        tc_gemm(t, A, WB, F, F);
        if (!t.ok) break;
        tc_load_w(t, WB, Wtc + gp.t_it[l][1], wbytes);
        for (int c0 = 0; c0 < F; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base(t) + (uint32_t)c0, v);
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = act ? silu_f(v[u] + W[o[1] + c0 + u]) : 0.0f;
            const float tot = tr_reduce16(v, lane);
            if (lane < 16) msum[warp * F + c0 + lane] += tot;
        }
        // A = n_i + n_j (the message MMA has read A)
        for (int q = (int)lane; q < 32 * CPR; q += 32) {
            const int r = 32 * warp + q / CPR, k0 = 8 * (q % CPR);
            const int j = jrow[r];
            float v[8];
            if (j >= 0) {
                const float4* a = reinterpret_cast<const float4*>(ni + k0);
                const float4* c = reinterpret_cast<const float4*>(nf + (size_t)(sy.ba0 + j) * F + k0);
                const float4 a0 = a[0], a1 = a[1], c0 = c[0], c1 = c[1];
                v[0] = a0.x + c0.x; v[1] = a0.y + c0.y; v[2] = a0.z + c0.z; v[3] = a0.w + c0.w;
                v[4] = a1.x + c1.x; v[5] = a1.y + c1.y; v[6] = a1.z + c1.z; v[7] = a1.w + c1.w;
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = 0.0f;
            }
            put8(A, r, k0, F, v);
        }
        // edge update, first layer
        tc_gemm(t, A, WB, F, F);
        if (!t.ok) break;
        tc_load_w(t, WB, Wtc + gp.t_it[l][2], wbytes);
        for (int c0 = 0; c0 < F; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base(t) + (uint32_t)c0, v);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float w8[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) w8[u] = silu_f(v[8 * h + u] + W[o[7] + c0 + 8 * h + u]);
                put8(A, row, c0 + 8 * h, F, w8);
            }
        }
        // edge update, second layer: e += W_a2 h + b_a2, through an FP32 staging
        // of HC columns at a time so that whole warps update contiguous rows
        tc_gemm(t, A, WB, F, F);
        if (!t.ok) break;
        float* D = reinterpret_cast<float*>(A);   // [TR][HCS], the hidden layer has been read
        for (int h0 = 0; h0 < F; h0 += HC) {
            for (int c0 = h0; c0 < h0 + HC; c0 += 16) {
                float v[16];
                tmem_ld16(lane_base(t) + (uint32_t)c0, v);
#pragma unroll
                for (int u = 0; u < 16; u += 4)
                    *reinterpret_cast<float4*>(D + row * HCS + (c0 - h0) + u) =
                        make_float4(v[u] + W[o[9] + c0 + u], v[u + 1] + W[o[9] + c0 + u + 1],
                                    v[u + 2] + W[o[9] + c0 + u + 2], v[u + 3] + W[o[9] + c0 + u + 3]);
            }
            __syncthreads();
            for (int q = (int)lane; q < 32 * HC / 4; q += 32) {
                const int r = 32 * warp + q / (HC / 4), c4 = q % (HC / 4);
                if (jrow[r] >= 0) {
                    float4* dst = reinterpret_cast<float4*>(eb + (size_t)(t0 + r) * F + h0) + c4;
                    const float4 cur = *dst, add = reinterpret_cast<const float4*>(D + r * HCS)[c4];
                    *dst = make_float4(cur.x + add.x, cur.y + add.y, cur.z + add.z, cur.w + add.w);
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int c = row; c < F; c += TR) mf[(size_t)b * F + c] = msum[c] + msum[F + c] + msum[2 * F + c] + msum[3 * F + c];
    tc_end(t, tcols<F>(), err);
}

// node update of 128 bead-atoms: n += W_v2 SiLU(W_v1 [n; m] + b_v1) + b_v2
template <int F>
__global__ void __launch_bounds__(TR, 1) gfn_tc_node_kernel(int B, GfnParams gp, int l, const float* __restrict__ W,
                                                            const unsigned char* __restrict__ Wtc,
                                                            float* __restrict__ nf, const float* __restrict__ mf,
                                                            DevErr* __restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A = sm;                       // [TR][2F] BF16, later [TR][F]
    unsigned char* WB = A + TR * 2 * F * 2;      // [F][2F] BF16, later [F][F]
    uint64_t* bars = reinterpret_cast<uint64_t*>(WB + F * 2 * F * 2);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
    Tc t;
    tc_begin(t, bars, tslot, tcols<F>());
    const int row = threadIdx.x, a = blockIdx.x * TR + row;
    const bool act = a < B;
    const unsigned* o = gp.o_it[l];
    tc_load_w(t, WB, Wtc + gp.t_it[l][3], (uint32_t)(F * 2 * F * 2));
    for (int k0 = 0; k0 < 2 * F; k0 += 8) {
        float v[8];
        if (act) {
            const float* src = k0 < F ? nf + (size_t)a * F + k0 : mf + (size_t)a * F + k0 - F;
            const float4 p0 = reinterpret_cast<const float4*>(src)[0], p1 = reinterpret_cast<const float4*>(src)[1];
            v[0] = p0.x; v[1] = p0.y; v[2] = p0.z; v[3] = p0.w; v[4] = p1.x; v[5] = p1.y; v[6] = p1.z; v[7] = p1.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = 0.0f;
        }
        put8(A, row, k0, 2 * F, v);
    }
    tc_gemm(t, A, WB, F, 2 * F);
    if (t.ok) {
        tc_load_w(t, WB, Wtc + gp.t_it[l][4], (uint32_t)(F * F * 2));
        for (int c0 = 0; c0 < F; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base(t) + (uint32_t)c0, v);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float w8[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) w8[q] = silu_f(v[8 * h + q] + W[o[3] + c0 + 8 * h + q]);
                put8(A, row, c0 + 8 * h, F, w8);
            }
        }
        tc_gemm(t, A, WB, F, F);
    }
    if (t.ok) {
        for (int c0 = 0; c0 < F; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base(t) + (uint32_t)c0, v);
            if (act) {
                float4* dst = reinterpret_cast<float4*>(nf + (size_t)a * F + c0);
                const float4* bb = reinterpret_cast<const float4*>(W + o[5] + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 cur = dst[q], bv = bb[q];
                    dst[q] = make_float4(cur.x + v[4 * q] + bv.x, cur.y + v[4 * q + 1] + bv.y,
                                         cur.z + v[4 * q + 2] + bv.z, cur.w + v[4 * q + 3] + bv.w);
                }
            }
        }
    }
    tc_end(t, tcols<F>(), err);
}

// force readout on the rows of one bead-atom: phi = w_f2 . SiLU(W_f1 e + b_f1)
// + b_f2, F_ij = s_F fc phi (x_i - x_j) / r, summed per atom with the virial
template <int F>
__global__ void __launch_bounds__(TR, 2) gfn_tc_force_kernel(
    const float4* __restrict__ x, const int* __restrict__ ba_sys, const BeadSys* __restrict__ bsys,
    const Rep* __restrict__ reps, const int* __restrict__ nbr, const int* __restrict__ nnb, int maxnb,
    GfnParams gp, const float* __restrict__ W, const unsigned char* __restrict__ Wtc, const float* __restrict__ ef,
    float4* __restrict__ f, float* __restrict__ wbuf, DevErr* __restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A = sm;                       // [TR][F] BF16
    unsigned char* WB = A + TR * F * 2;          // [F][F] BF16
    float* red = reinterpret_cast<float*>(WB + F * F * 2);   // [4][16]
    uint64_t* bars = reinterpret_cast<uint64_t*>(red + 64);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
    Tc t;
    tc_begin(t, bars, tslot, tcols<F>());
    const int b = blockIdx.x, row = threadIdx.x, warp = row >> 5;
    const unsigned lane = lane_id();
    const BeadSys sy = bsys[ba_sys[b]];
    const Rep rp = reps[sy.rep];
    const int n = min(nnb[b], maxnb);
    const float4 xi = x[b];
    const float* eb = ef + (size_t)b * maxnb * F;
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
    for (int t0 = 0; t0 < n && t.ok; t0 += TR) {
        tc_load_w(t, WB, Wtc + gp.t_Wf1, (uint32_t)(F * F * 2));
        const int s = t0 + row;
        const bool act = s < n;
        // a warp stages its 32 rows, consecutive lanes on consecutive chunks
        for (int q = (int)lane; q < 32 * (F / 8); q += 32) {
            const int r = 32 * warp + q / (F / 8), k0 = 8 * (q % (F / 8));
            float v[8];
            if (t0 + r < n) {
                const float4 p0 = reinterpret_cast<const float4*>(eb + (size_t)(t0 + r) * F + k0)[0];
                const float4 p1 = reinterpret_cast<const float4*>(eb + (size_t)(t0 + r) * F + k0)[1];
                v[0] = p0.x; v[1] = p0.y; v[2] = p0.z; v[3] = p0.w; v[4] = p1.x; v[5] = p1.y; v[6] = p1.z; v[7] = p1.w;
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = 0.0f;
            }
            put8(A, r, k0, F, v);
        }
        tc_gemm(t, A, WB, F, F);
        if (!t.ok) break;
        float phi = gp.b_f2;
        for (int c0 = 0; c0 < F; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base(t) + (uint32_t)c0, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) phi = fmaf(W[gp.o_wf2 + c0 + q], silu_f(v[q] + W[gp.o_bf1 + c0 + q]), phi);
        }
        if (act) {
            const int j = nbr[(size_t)b * maxnb + s];
            float dx, dy, dz;
            pair_vec(rp, xi, x[sy.ba0 + j], dx, dy, dz);
            const float r = sqrtf(dx * dx + dy * dy + dz * dz);
            float fc, dfc;
            cutoff(r, gp.rc, gp.pi_over_rc, fc, dfc);
            const float sc = gp.s_F * fc * phi / r;
            const float d3[3] = {dx, dy, dz};
            const float Fij[3] = {-sc * dx, -sc * dy, -sc * dz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                acc[a] += Fij[a];
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[3 + 3 * a + c] -= 0.5f * d3[a] * Fij[c];
            }
        }
    }
    const float tot = tr_reduce16(acc, lane);
    if (lane < 16) red[warp * 16 + lane] = tot;
    __syncthreads();
    if (row < 12) {
        const float sum = red[row] + red[16 + row] + red[32 + row] + red[48 + row];
        if (row >= 3) wbuf[(size_t)b * 9 + row - 3] = sum;
        else reinterpret_cast<float*>(&f[b])[row] = sum;
    }
    if (row == 3) reinterpret_cast<float*>(&f[b])[3] = 0.0f;
    tc_end(t, tcols<F>(), err);
}

namespace {

// (the input layer's tiles are small: its shared memory is padded so that
// at most four CTAs share an SM's tensor memory)
template <int F>
size_t init_smem() { return 48 * 1024; }
template <int F>
size_t iter_smem() { return (size_t)TR * F * 2 + (size_t)F * F * 2 + 4 * F * 4 + TR * 4 + 64; }
template <int F>
size_t node_smem() { return (size_t)TR * 2 * F * 2 + (size_t)F * 2 * F * 2 + 64; }
template <int F>
size_t force_smem() { return (size_t)TR * F * 2 + (size_t)F * F * 2 + 64 * 4 + 64; }

template <int F>
void run_gfn_tc(const Dev& d, cudaStream_t st)
{
    const GfnParams& gp = d.gfn;
    const float* W = d.gfn_w;
    const unsigned char* Wt = d.gfn_wtc;
    {
        static size_t d0 = 0, d1 = 0, d2 = 0, d3 = 0;
        set_smem(gfn_tc_init_kernel<F>, init_smem<F>(), d0);
        set_smem(gfn_tc_iter_kernel<F>, iter_smem<F>(), d1);
        set_smem(gfn_tc_node_kernel<F>, node_smem<F>(), d2);
        set_smem(gfn_tc_force_kernel<F>, force_smem<F>(), d3);
    }
    const float4* x = (const float4*)d.x;
    gfn_tc_init_kernel<F><<<d.B, TR, init_smem<F>(), st>>>(x, d.ba_sys, d.bsys, d.reps, d.atype, d.nbr, d.nnb,
                                                            d.maxnb, gp, W, Wt, d.gfn_n, d.gfn_e, (float*)d.Eatom,
                                                            d.err);
    for (int l = 0; l < gp.L; ++l) {
        gfn_tc_iter_kernel<F><<<d.B, TR, iter_smem<F>(), st>>>(d.ba_sys, d.bsys, d.nbr, d.nnb, d.maxnb, gp, l, W, Wt,
                                                                d.gfn_n, d.gfn_m, d.gfn_e, d.err);
        gfn_tc_node_kernel<F><<<(d.B + TR - 1) / TR, TR, node_smem<F>(), st>>>(d.B, gp, l, W, Wt, d.gfn_n, d.gfn_m,
                                                                               d.err);
    }
    gfn_tc_force_kernel<F><<<d.B, TR, force_smem<F>(), st>>>(x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, gp,
                                                              W, Wt, d.gfn_e, (float4*)d.f, (float*)d.wbuf, d.err);
}

}  // namespace

void launch_gfn_tc(const Dev& d, cudaStream_t st)
{
    if (d.gfn.F == 64)
        run_gfn_tc<64>(d, st);
    else
        run_gfn_tc<128>(d, st);
}

// bytes of the BF16 images: W_e [F][32]; per iteration W_m, W_a1, W_a2 [F][F],
// W_v1 [F][2F], W_v2 [F][F]; W_f1 [F][F]
size_t gfn_tc_image_bytes(int F, int L)
{
    const size_t FF = (size_t)F * F;
    return 2 * ((size_t)F * NR + (size_t)L * (3 * FF + 2 * FF + FF) + FF);
}

}  // namespace pimd
