// mlp_tc.cu -- per-element network forward and input gradient on the 5th-gen
// tensor cores (tcgen05.mma kind::f16, BF16 x BF16 -> FP32 accumulators in
// tensor memory), for tiles of 128 bead-atoms of one element.
//
// One CTA of 256 threads per tile. Thread 0 issues the bulk weight copies
// (cp.async.bulk, double-buffered, completion on mbarriers) and the MMAs
// (completion through tcgen05.commit on an mbarrier); all 8 warps run the
// epilogues, warp w reading TMEM lanes 32 (w % 4).. and half of the columns.
// Operands sit in shared memory in the no-swizzle K-major canonical layout:
// 8-row x 16-byte core matrices, adjacent along K at 128 B (leading byte
// offset), adjacent along M/N at (K / 8) * 128 B (stride byte offset).
//
// Layers: forward h_l = tanh(W_l h_{l-1} + b_l) (accumulator a_l in TMEM,
// h_l stored as BF16 for the next layer and for tanh'), y = w_out . h_L
// (FP32 epilogue), then backward dE/da_L = s_E w_out (1 - h_L^2),
// dE/dh_{l-1} = W_l^T dE/da_l on the tensor cores with pre-transposed
// weight images, and dE/dG = dE/dh_0 / sigma.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace pimd {

namespace {

constexpr int TC_THREADS = 256;

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

__device__ __forceinline__ float2 unpack_bf16(uint32_t u)
{
    __nv_bfloat162 h;
    memcpy(&h, &u, 4);
    return __bfloat1622float2(h);
}

// tanh on the special-function unit (tanh.approx.f32, relative error ~2^-11):
// the activations are rounded to BF16 (2^-9) right after, so the accurate
// library tanh would not change the result beyond that rounding
__device__ __forceinline__ float tanh_f(float v)
{
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// byte sizes / offsets of the weight images of one element type:
// forward images W_l [W][in_l], then backward images W_l^T [in_l][W]
__host__ __device__ __forceinline__ size_t img_bytes(int n, int k) { return (size_t)n * k * 2; }

__host__ __device__ __forceinline__ size_t img_offset(int W, int L, int phase)
{
    // phase 0..L-1: forward layer phase+1; phase L..2L-1: backward layer 2L-phase
    size_t o = 0;
    for (int p = 0; p < phase; ++p) {
        const int l = p < L ? p + 1 : 2 * L - p;
        const int in = l == 1 ? ND : W;
        o += img_bytes(W, in);
    }
    return o;
}

}  // namespace

template <int W, int L, bool DB>
__global__ void __launch_bounds__(TC_THREADS, 1) mlp_tc_kernel(
    const float* __restrict__ G, const int* __restrict__ perm, const int* __restrict__ tile_type,
    const unsigned char* __restrict__ wimg, size_t img_per_type, const float* __restrict__ wvec,
    size_t vec_per_type, float* __restrict__ Eatom, float* __restrict__ dEdG, DevErr* __restrict__ err)
{
    constexpr int M = 128;
    constexpr int A0_B = M * ND * 2;
    constexpr int H_B = M * W * 2;
    constexpr int WB_B = W * W * 2 > W * ND * 2 ? W * W * 2 : W * ND * 2;
    constexpr int TCOLS = W < 64 ? 64 : W;   // TMEM columns (power of two >= 32)
    constexpr int NPH = 2 * L;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A0 = sm;
    unsigned char* Hs = A0 + A0_B;                 // h_1 .. h_{L-1} (h_L is not kept)
    unsigned char* GA = Hs + (L > 1 ? (L - 1) : 1) * H_B;
    unsigned char* WB0 = GA + H_B;
    unsigned char* WB1 = WB0 + (DB ? WB_B : 0);
    uint64_t* bars = reinterpret_cast<uint64_t*>(WB1 + WB_B);   // [0] mma, [1] wbuf0, [2] wbuf1
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
    float* ysum = reinterpret_cast<float*>(tslot + 4);          // [2][128]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, hsel = warp >> 2;
    const int row = 32 * q + lane;                              // TMEM lane / tile row of this thread
    const int row0 = blockIdx.x * M;
    const int type = tile_type[row0 / TILE_ROWS];
    const unsigned char* img = wimg + (size_t)type * img_per_type;
    const float* vec = wvec + (size_t)type * vec_per_type;
    const float* b_l = vec;                    // [L][W]
    const float* w_out = vec + L * W;          // [W]
    const float* mu = w_out + W;               // [64]
    const float* sigma = mu + ND;              // [64]
    const float b_out = sigma[ND], s_E = sigma[ND + 1], e_Z = sigma[ND + 2];

    const uint32_t bar_mma = smem_u32(&bars[0]);
    const uint32_t bar_w[2] = {smem_u32(&bars[1]), smem_u32(&bars[2])};
    if (tid == 0) {
        mbar_init(bar_mma, 1);
        mbar_init(bar_w[0], 1);
        mbar_init(bar_w[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    // weight loads: phase p uses buffer p % 2 (double-buffered) or buffer 0
    bool w_issued[NPH];
#pragma unroll
    for (int p = 0; p < NPH; ++p) w_issued[p] = false;
    auto issue_w = [&](int p) {
        const int l = p < L ? p + 1 : 2 * L - p;
        const int in = l == 1 ? ND : W;
        const int buf = DB ? (p & 1) : 0;
        bulk_load(smem_u32(buf ? WB1 : WB0), img + img_offset(W, L, p), (uint32_t)img_bytes(W, in), bar_w[buf]);
    };
    if (tid == 0) {
        issue_w(0);
        w_issued[0] = true;
        if (DB && NPH > 1) {
            issue_w(1);
            w_issued[1] = true;
        }
    }

    // h_0 = (G - mu) / sigma in BF16: thread -> (row tid % 128, 32 columns)
    {
        const int r = tid & (M - 1), c0 = (tid >> 7) * 32;
        const int ba = perm[row0 + r];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = c0 + 8 * g + j;
                v[j] = ba >= 0 ? (G[(size_t)ba * ND + c] - mu[c]) / sigma[c] : 0.0f;
            }
            uint4 pk = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                  pack_bf16(v[6], v[7]));
            *reinterpret_cast<uint4*>(A0 + 2 * cm_index(r, c0 + 8 * g, ND)) = pk;
        }
    }
    fence_proxy();
    __syncthreads();

    bool ok = true;
    float y_part = 0.0f;
    for (int p = 0; p < NPH && ok; ++p) {
        const bool fwd = p < L;
        const int l = fwd ? p + 1 : 2 * L - p;             // layer of this phase
        const int K = fwd ? (l == 1 ? ND : W) : W;          // reduction length
        const int N = fwd ? W : (l == 1 ? ND : W);          // output columns
        const unsigned char* Aop = fwd ? (l == 1 ? A0 : Hs + (size_t)(l - 2) * H_B) : GA;
        const int buf = DB ? (p & 1) : 0;
        const uint32_t wpar = DB ? ((p >> 1) & 1) : (p & 1);
        // ---- MMA issue
        bool good = true;
        if (tid == 0) {
            good = mbar_wait(bar_w[buf], wpar);
            if (good) {
                fence_after();
                const uint32_t a0 = smem_u32(Aop), b0 = smem_u32(buf ? WB1 : WB0);
                const uint32_t sbo = (uint32_t)(K / 8) * 128u;
                const uint32_t idesc = make_idesc(M, N);
                for (int ks = 0; ks < K / 16; ++ks) {
                    const uint64_t ad = make_desc(a0 + ks * 256u, 128u, sbo);
                    const uint64_t bd = make_desc(b0 + ks * 256u, 128u, sbo);
                    mma_f16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
                }
                mma_commit(bar_mma);
            }
        }
        good = mbar_wait(bar_mma, p & 1) && good;
        ok = __syncthreads_and(good ? 1 : 0) != 0;
        if (!ok) break;
        fence_after();
        // ---- the weight buffer of this phase is free: prefetch
        if (tid == 0) {
            const int nxt = DB ? p + 2 : p + 1;
            if (nxt < NPH) {
                issue_w(nxt);
                w_issued[nxt] = true;
            }
        }
        // ---- epilogue over this thread's row and column half
        const int cbeg = hsel * (N / 2), cend = cbeg + N / 2;
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
            if (fwd) {
                float h[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) h[j] = tanh_f(v[j] + b_l[(l - 1) * W + c0 + j]);
                if (l < L) {
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        uint4 pk = make_uint4(pack_bf16(h[8 * g], h[8 * g + 1]), pack_bf16(h[8 * g + 2], h[8 * g + 3]),
                                              pack_bf16(h[8 * g + 4], h[8 * g + 5]),
                                              pack_bf16(h[8 * g + 6], h[8 * g + 7]));
                        *reinterpret_cast<uint4*>(Hs + (size_t)(l - 1) * H_B + 2 * cm_index(row, c0 + 8 * g, W)) = pk;
                    }
                } else {
                    float ga[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float wo = w_out[c0 + j];
                        y_part += wo * h[j];
                        ga[j] = s_E * wo * (1.0f - h[j] * h[j]);
                    }
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        uint4 pk = make_uint4(pack_bf16(ga[8 * g], ga[8 * g + 1]), pack_bf16(ga[8 * g + 2], ga[8 * g + 3]),
                                              pack_bf16(ga[8 * g + 4], ga[8 * g + 5]),
                                              pack_bf16(ga[8 * g + 6], ga[8 * g + 7]));
                        *reinterpret_cast<uint4*>(GA + 2 * cm_index(row, c0 + 8 * g, W)) = pk;
                    }
                }
            } else if (l > 1) {
                // dE/da_{l-1} = (W_l^T dE/da_l) * (1 - h_{l-1}^2)
                const unsigned char* Hp = Hs + (size_t)(l - 2) * H_B;
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const uint4 hv = *reinterpret_cast<const uint4*>(Hp + 2 * cm_index(row, c0 + 8 * g, W));
                    const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
                    float o[8];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const float2 hh = unpack_bf16(hw[t]);
                        o[2 * t] = v[8 * g + 2 * t] * (1.0f - hh.x * hh.x);
                        o[2 * t + 1] = v[8 * g + 2 * t + 1] * (1.0f - hh.y * hh.y);
                    }
                    uint4 pk = make_uint4(pack_bf16(o[0], o[1]), pack_bf16(o[2], o[3]), pack_bf16(o[4], o[5]),
                                          pack_bf16(o[6], o[7]));
                    *reinterpret_cast<uint4*>(GA + 2 * cm_index(row, c0 + 8 * g, W)) = pk;
                }
            } else {
                const int ba = perm[row0 + row];
                if (ba >= 0) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4) {
                        float4 o = make_float4(v[j] / sigma[c0 + j], v[j + 1] / sigma[c0 + j + 1],
                                               v[j + 2] / sigma[c0 + j + 2], v[j + 3] / sigma[c0 + j + 3]);
                        *reinterpret_cast<float4*>(dEdG + (size_t)ba * ND + c0 + j) = o;
                    }
                }
            }
        }
        if (fwd && l == L) ysum[hsel * M + row] = y_part;
        fence_proxy();
        fence_before();
        __syncthreads();
        fence_after();
        if (fwd && l == L && hsel == 0) {
            const int ba = perm[row0 + row];
            if (ba >= 0) Eatom[ba] = s_E * (ysum[row] + ysum[M + row] + b_out) + e_Z;
        }
    }
    if (!ok) {
        // a wait gave up: report, let issued copies land, then release TMEM
        if (tid == 0) {
            atomicOr(&err->flags, ERR_TIMEOUT);
            for (int p = 0; p < NPH; ++p)
                if (w_issued[p]) {
                    const int buf = DB ? (p & 1) : 0;
                    mbar_wait(bar_w[buf], DB ? ((p >> 1) & 1) : (p & 1));
                }
            mbar_wait(bar_mma, 0);
        }
        __syncthreads();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Network for widths 64 / 128 with two tiles resident per SM: the hidden
// activations h_1 .. h_(L-1) are parked in tensor memory (packed BF16 pairs
// next to the accumulator) for the backward pass, so shared memory holds only
// the descriptor tile, one activation / gradient tile and one weight buffer
// (80 KB at width 128) and tensor memory 256 columns per CTA. While one CTA
// waits on its MMA or its weight copy, the other runs its epilogue.
// ---------------------------------------------------------------------------
template <int W, int L>
__host__ __device__ constexpr int park_cols() { return (W < 64 ? 64 : W) + (L - 1) * (W / 2); }

// threads of the parked kernel: NT / 128 warps per tensor-memory lane
// quadrant, each taking that share of a phase's columns in the epilogues.
// 512 threads and 256 tensor-memory columns per tile, two tiles per SM; a
// narrow network whose parked columns fit in 128 runs 256 threads and 128
// columns per tile, four tiles per SM.
template <int W, int L>
__host__ __device__ constexpr int park_threads() { return (W == 64 && park_cols<W, L>() <= 128) ? 256 : 512; }

template <int W, int L>
__global__ void __launch_bounds__(park_threads<W, L>(), park_threads<W, L>() == 512 ? 2 : 4) mlp_tc_park_kernel(
    const float* __restrict__ G, const int* __restrict__ perm, const int* __restrict__ tile_type,
    const unsigned char* __restrict__ wimg, size_t img_per_type, const float* __restrict__ wvec,
    size_t vec_per_type, float* __restrict__ Eatom, float* __restrict__ dEdG, DevErr* __restrict__ err, int tile0)
{
    constexpr int M = 128;
    constexpr int A0_B = M * ND * 2;
    constexpr int H_B = M * W * 2;
    constexpr int WB_B = W * W * 2 > W * ND * 2 ? W * W * 2 : W * ND * 2;
    constexpr int PARK_THREADS = park_threads<W, L>();
    constexpr int PARK_NH = PARK_THREADS / 128;   // column groups per row
    constexpr int TACC = W < 64 ? 64 : W;       // accumulator columns
    constexpr int TALLOC = PARK_THREADS == 512 ? 256 : 128;   // per CTA: the SM's 512 columns over 2 or 4 CTAs
    static_assert(park_cols<W, L>() <= TALLOC, "parked activations exceed tensor memory");
    static_assert((W / PARK_NH) % 16 == 0 && (ND / PARK_NH) % 16 == 0, "column groups of whole 16-column chunks");
    constexpr int NPH = 2 * L;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A0 = sm;
    unsigned char* ACT = A0 + A0_B;              // h_(l-1) as the next A operand, later dE/da_l
    unsigned char* WB = ACT + H_B;
    uint64_t* bars = reinterpret_cast<uint64_t*>(WB + WB_B);   // [0] mma, [1] weights
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
    float* ysum = reinterpret_cast<float*>(tslot + 4);          // [PARK_NH][128]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, hsel = warp >> 2;
    const int row = 32 * q + lane;
    const int row0 = (tile0 + blockIdx.x) * M;   // tiles tile0 .. of the launch
    const int type = tile_type[row0 / TILE_ROWS];
    const unsigned char* img = wimg + (size_t)type * img_per_type;
    const float* vec = wvec + (size_t)type * vec_per_type;
    const float* w_out = vec + L * W;
    const float* mu = w_out + W;
    const float* sigma = mu + ND;
    const float b_out = sigma[ND], s_E = sigma[ND + 1], e_Z = sigma[ND + 2];
    // the element's vectors in shared memory: biases, output weights, mu and
    // 1 / sigma (the epilogues read them in every 16-column chunk)
    float* sb = ysum + PARK_NH * M;   // [L][W]
    float* swo = sb + L * W;
    float* smu = swo + W;
    float* sis = smu + ND;
    for (int i = threadIdx.x; i < L * W + W + ND; i += blockDim.x) sb[i] = vec[i];
    for (int i = threadIdx.x; i < ND; i += blockDim.x) sis[i] = 1.0f / sigma[i];

    const uint32_t bar_mma = smem_u32(&bars[0]);
    const uint32_t bar_w = smem_u32(&bars[1]);
    if (tid == 0) {
        mbar_init(bar_mma, 1);
        mbar_init(bar_w, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TALLOC)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);

    int issued = 0;   // weight copies issued (phase p uses parity p & 1)
    auto issue_w = [&](int p) {
        const int l = p < L ? p + 1 : 2 * L - p;
        const int in = l == 1 ? ND : W;
        bulk_load(smem_u32(WB), img + img_offset(W, L, p), (uint32_t)img_bytes(W, in), bar_w);
    };
    if (tid == 0) {
        issue_w(0);
        issued = 1;
    }

    // h_0 = (G - mu) / sigma in BF16: thread -> (row tid % 128, CPT columns),
    // the row's FP32 values as 16-byte loads
    {
        constexpr int CPT = ND / PARK_NH;
        const int r = tid & (M - 1), c0 = (tid >> 7) * CPT;
        const int ba = perm[row0 + r];
        float4 gv[CPT / 4];
        const float4* grow = reinterpret_cast<const float4*>(G + (size_t)(ba >= 0 ? ba : 0) * ND + c0);
#pragma unroll
        for (int g = 0; g < CPT / 4; ++g) gv[g] = ba >= 0 ? grow[g] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int g = 0; g < CPT / 8; ++g) {
            float v[8];
            const float gg[8] = {gv[2 * g].x, gv[2 * g].y, gv[2 * g].z, gv[2 * g].w,
                                 gv[2 * g + 1].x, gv[2 * g + 1].y, gv[2 * g + 1].z, gv[2 * g + 1].w};
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const int c = c0 + 8 * g + jj;
                v[jj] = ba >= 0 ? (gg[jj] - smu[c]) * sis[c] : 0.0f;
            }
            uint4 pk = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                  pack_bf16(v[6], v[7]));
            *reinterpret_cast<uint4*>(A0 + 2 * cm_index(r, c0 + 8 * g, ND)) = pk;
        }
    }
    fence_proxy();
    __syncthreads();

    bool ok = true;
    float y_part = 0.0f;
    int p_fail = -1;
    for (int p = 0; p < NPH && ok; ++p) {
        const bool fwd = p < L;
        const int l = fwd ? p + 1 : 2 * L - p;
        const int K = fwd ? (l == 1 ? ND : W) : W;
        const int N = fwd ? W : (l == 1 ? ND : W);
        const unsigned char* Aop = (fwd && l == 1) ? A0 : ACT;
        p_fail = p;
        bool good = true;
        if (tid == 0) {
            good = mbar_wait(bar_w, (uint32_t)(p & 1));
            if (good) {
                fence_after();
                const uint32_t a0 = smem_u32(Aop), b0 = smem_u32(WB);
                const uint32_t sbo = (uint32_t)(K / 8) * 128u;
                const uint32_t idesc = make_idesc(M, N);
                for (int ks = 0; ks < K / 16; ++ks) {
                    const uint64_t ad = make_desc(a0 + ks * 256u, 128u, sbo);
                    const uint64_t bd = make_desc(b0 + ks * 256u, 128u, sbo);
                    mma_f16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
                }
                mma_commit(bar_mma);
            }
        }
        good = mbar_wait(bar_mma, (uint32_t)(p & 1)) && good;
        ok = __syncthreads_and(good ? 1 : 0) != 0;
        if (!ok) break;
        fence_after();
        // the MMA has read the weights and the A tile: next weights, then the epilogue
        if (tid == 0 && p + 1 < NPH) {
            issue_w(p + 1);
            issued = p + 2;
        }
        const int cbeg = hsel * (N / PARK_NH), cend = cbeg + N / PARK_NH;
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base + (uint32_t)c0, v);
            if (fwd) {
                float h[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) h[j] = tanh_f(v[j] + sb[(l - 1) * W + c0 + j]);
                if (l < L) {
                    uint32_t pk[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) pk[t] = pack_bf16(h[2 * t], h[2 * t + 1]);
#pragma unroll
                    for (int g = 0; g < 2; ++g)
                        *reinterpret_cast<uint4*>(ACT + 2 * cm_index(row, c0 + 8 * g, W)) =
                            make_uint4(pk[4 * g], pk[4 * g + 1], pk[4 * g + 2], pk[4 * g + 3]);
                    // parked for the backward: tanh' = 1 - h^2 from the FP32 h,
                    // rounded once (from a BF16 h it loses its digits where
                    // the unit saturates)
                    uint32_t dk[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        dk[t] = pack_bf16(1.0f - h[2 * t] * h[2 * t], 1.0f - h[2 * t + 1] * h[2 * t + 1]);
                    tmem_st8(lane_base + (uint32_t)(TACC + (l - 1) * (W / 2) + (c0 >> 1)), dk);
                } else {
                    float ga[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float wo = swo[c0 + j];
                        y_part += wo * h[j];
                        ga[j] = s_E * wo * (1.0f - h[j] * h[j]);
                    }
#pragma unroll
                    for (int g = 0; g < 2; ++g)
                        *reinterpret_cast<uint4*>(ACT + 2 * cm_index(row, c0 + 8 * g, W)) =
                            make_uint4(pack_bf16(ga[8 * g], ga[8 * g + 1]), pack_bf16(ga[8 * g + 2], ga[8 * g + 3]),
                                       pack_bf16(ga[8 * g + 4], ga[8 * g + 5]), pack_bf16(ga[8 * g + 6], ga[8 * g + 7]));
                }
            } else if (l > 1) {
                // dE/da_(l-1) = (W_l^T dE/da_l) * (1 - h_(l-1)^2), the derivative from its parking place
                uint32_t hw[8];
                tmem_ld8(lane_base + (uint32_t)(TACC + (l - 2) * (W / 2) + (c0 >> 1)), hw);
                uint32_t pk[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float2 dd = unpack_bf16(hw[t]);
                    pk[t] = pack_bf16(v[2 * t] * dd.x, v[2 * t + 1] * dd.y);
                }
#pragma unroll
                for (int g = 0; g < 2; ++g)
                    *reinterpret_cast<uint4*>(ACT + 2 * cm_index(row, c0 + 8 * g, W)) =
                        make_uint4(pk[4 * g], pk[4 * g + 1], pk[4 * g + 2], pk[4 * g + 3]);
            } else {
                const int ba = perm[row0 + row];
                if (ba >= 0) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4) {
                        float4 o = make_float4(v[j] * sis[c0 + j], v[j + 1] * sis[c0 + j + 1],
                                               v[j + 2] * sis[c0 + j + 2], v[j + 3] * sis[c0 + j + 3]);
                        *reinterpret_cast<float4*>(dEdG + (size_t)ba * ND + c0 + j) = o;
                    }
                }
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        if (fwd && l == L) ysum[hsel * M + row] = y_part;
        fence_proxy();
        fence_before();
        __syncthreads();
        fence_after();
        if (fwd && l == L && hsel == 0) {
            const int ba = perm[row0 + row];
            float ys = 0.0f;
#pragma unroll
            for (int h = 0; h < PARK_NH; ++h) ys += ysum[h * M + row];
            if (ba >= 0) Eatom[ba] = s_E * (ys + b_out) + e_Z;
        }
    }
    if (!ok) {
        // a wait gave up: report, let the last issued copy and an MMA still in
        // flight finish (bounded), then release TMEM
        if (tid == 0) {
            atomicOr(&err->flags, ERR_TIMEOUT);
            if (issued > 0) mbar_wait(bar_w, (uint32_t)((issued - 1) & 1));
            if (p_fail >= 0) mbar_wait(bar_mma, (uint32_t)(p_fail & 1));
        }
        __syncthreads();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TALLOC) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Wide network (hidden width 256): weights stream through shared memory in
// K-chunks of 64 (double-buffered bulk copies; a tcgen05.commit per chunk
// releases its buffer), one activation buffer serves as the next layer's A
// operand, and hidden activations needed again by the backward pass
// (h_1 .. h_{L-2}) are parked in tensor memory as packed BF16 next to the
// 256-column accumulator (512 TMEM columns).
// ---------------------------------------------------------------------------
namespace {

constexpr int WW = 256;          // hidden width of the wide kernel
constexpr int KCH = 64;          // K elements per weight chunk

__host__ __device__ __forceinline__ int wide_phase_layer(int L, int p) { return p < L ? p + 1 : 2 * L - p; }
__host__ __device__ __forceinline__ int wide_phase_K(int L, int p)
{
    return (p < L && wide_phase_layer(L, p) == 1) ? ND : WW;
}
__host__ __device__ __forceinline__ int wide_phase_N(int L, int p)
{
    return (p >= L && wide_phase_layer(L, p) == 1) ? ND : WW;
}
// chunks of all phases, in issue order
__host__ __device__ __forceinline__ int wide_nchunks(int L)
{
    int g = 0;
    for (int p = 0; p < 2 * L; ++p) g += wide_phase_K(L, p) / KCH;
    return g;
}
// byte offset of chunk g in one type's image, and its phase's N
__host__ __device__ __forceinline__ size_t wide_chunk_offset(int L, int g, int* Nout)
{
    size_t o = 0;
    int gg = 0;
    for (int p = 0; p < 2 * L; ++p) {
        const int nch = wide_phase_K(L, p) / KCH, N = wide_phase_N(L, p);
        for (int c = 0; c < nch; ++c, ++gg) {
            if (gg == g) {
                if (Nout) *Nout = N;
                return o;
            }
            o += (size_t)N * KCH * 2;
        }
    }
    if (Nout) *Nout = 0;
    return o;
}


}  // namespace

template <int L>
__global__ void __launch_bounds__(TC_THREADS, 1) mlp_tc_wide_kernel(
    const float* __restrict__ G, const int* __restrict__ perm, const int* __restrict__ tile_type,
    const unsigned char* __restrict__ wimg, size_t img_per_type, const float* __restrict__ wvec,
    size_t vec_per_type, float* __restrict__ Eatom, float* __restrict__ dEdG, DevErr* __restrict__ err)
{
    constexpr int M = 128;
    constexpr int A0_B = M * ND * 2;          // 16 KB
    constexpr int ACT_B = M * WW * 2;         // 64 KB
    constexpr int WB_B = WW * KCH * 2;        // 32 KB per chunk buffer
    constexpr int NCH = (L == 1 ? 1 : 1 + 4 * (L - 1)) + 4 * L;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A0 = sm;
    unsigned char* ACT = A0 + A0_B;
    unsigned char* GA = ACT + ACT_B;
    unsigned char* WB[2] = {GA + ACT_B, GA + ACT_B + WB_B};
    uint64_t* bars = reinterpret_cast<uint64_t*>(GA + ACT_B + 2 * WB_B);   // mma, wload[2], wfree[2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 6);
    float* ysum = reinterpret_cast<float*>(tslot + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, hsel = warp >> 2;
    const int row = 32 * q + lane;
    const int row0 = blockIdx.x * M;
    const int type = tile_type[row0 / TILE_ROWS];
    const unsigned char* img = wimg + (size_t)type * img_per_type;
    const float* vec = wvec + (size_t)type * vec_per_type;
    const float* w_out = vec + L * WW;
    const float* mu = w_out + WW;
    const float* sigma = mu + ND;
    const float b_out = sigma[ND], s_E = sigma[ND + 1], e_Z = sigma[ND + 2];
    // the element's vectors in shared memory: biases, output weights, mu and
    // 1 / sigma (the epilogues read them in every 16-column chunk)
    float* sb = ysum + 2 * M;   // [L][WW]
    float* swo = sb + L * WW;
    float* smu = swo + WW;
    float* sis = smu + ND;
    for (int i = threadIdx.x; i < L * WW + WW + ND; i += blockDim.x) sb[i] = vec[i];
    for (int i = threadIdx.x; i < ND; i += blockDim.x) sis[i] = 1.0f / sigma[i];

    const uint32_t bar_mma = smem_u32(&bars[0]);
    const uint32_t bar_ld[2] = {smem_u32(&bars[1]), smem_u32(&bars[2])};
    const uint32_t bar_free[2] = {smem_u32(&bars[3]), smem_u32(&bars[4])};
    if (tid == 0) {
        mbar_init(bar_mma, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar_ld[i], 1);
            mbar_init(bar_free[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);

    int issued = 0;   // chunks whose bulk copy thread 0 has started
    auto load_chunk = [&](int g) {
        int N = 0;
        const size_t off = wide_chunk_offset(L, g, &N);
        bulk_load(smem_u32(WB[g & 1]), img + off, (uint32_t)(N * KCH * 2), bar_ld[g & 1]);
    };
    if (tid == 0) {
        load_chunk(0);
        issued = 1;
        if (NCH > 1) {
            load_chunk(1);
            issued = 2;
        }
    }

    // h_0 = (G - mu) / sigma in BF16
    {
        const int r = tid & (M - 1), c0 = (tid >> 7) * 32;
        const int ba = perm[row0 + r];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = c0 + 8 * g + j;
                v[j] = ba >= 0 ? (G[(size_t)ba * ND + c] - smu[c]) * sis[c] : 0.0f;
            }
            uint4 pk = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                  pack_bf16(v[6], v[7]));
            *reinterpret_cast<uint4*>(A0 + 2 * cm_index(r, c0 + 8 * g, ND)) = pk;
        }
    }
    fence_proxy();
    __syncthreads();

    bool ok = true;
    float y_part = 0.0f;
    int g0 = 0;   // first chunk of the current phase
    for (int p = 0; p < 2 * L && ok; ++p) {
        const bool fwd = p < L;
        const int l = wide_phase_layer(L, p);
        const int K = wide_phase_K(L, p), N = wide_phase_N(L, p);
        const int nch = K / KCH;
        const unsigned char* Aop = fwd ? (l == 1 ? A0 : ACT) : GA;
        bool good = true;
        if (tid == 0) {
            const uint32_t a0 = smem_u32(Aop);
            const uint32_t sbo_a = (uint32_t)(K / 8) * 128u;
            const uint32_t idesc = make_idesc(M, N);
            for (int c = 0; c < nch && good; ++c) {
                const int g = g0 + c;
                good = mbar_wait(bar_ld[g & 1], (uint32_t)((g >> 1) & 1));
                if (!good) break;
                fence_after();
                const uint32_t b0 = smem_u32(WB[g & 1]);
                for (int ks = 0; ks < KCH / 16; ++ks) {
                    const uint64_t ad = make_desc(a0 + (uint32_t)c * 1024u + ks * 256u, 128u, sbo_a);
                    const uint64_t bd = make_desc(b0 + ks * 256u, 128u, 1024u);
                    mma_f16(tmem, ad, bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                }
                mma_commit(bar_free[g & 1]);
                // buffer of chunk g-1 is reused for chunk g+1 once chunk g-1's MMAs are done
                if (g >= 1 && g + 1 < NCH && issued == g + 1) {
                    good = mbar_wait(bar_free[(g + 1) & 1], (uint32_t)(((g - 1) >> 1) & 1));
                    if (good) {
                        load_chunk(g + 1);
                        issued = g + 2;
                    }
                }
            }
            if (good) mma_commit(bar_mma);
        }
        good = mbar_wait(bar_mma, (uint32_t)(p & 1)) && good;
        ok = __syncthreads_and(good ? 1 : 0) != 0;
        if (!ok) break;
        fence_after();
        g0 += nch;
        const int cbeg = hsel * (N / 2), cend = cbeg + N / 2;
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base + (uint32_t)c0, v);
            if (fwd) {
                float h[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) h[j] = tanh_f(v[j] + sb[(l - 1) * WW + c0 + j]);
                if (l < L) {
                    uint32_t pk[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) pk[t] = pack_bf16(h[2 * t], h[2 * t + 1]);
#pragma unroll
                    for (int g = 0; g < 2; ++g)
                        *reinterpret_cast<uint4*>(ACT + 2 * cm_index(row, c0 + 8 * g, WW)) =
                            make_uint4(pk[4 * g], pk[4 * g + 1], pk[4 * g + 2], pk[4 * g + 3]);
                    if (l <= L - 2) {
                        // parked for the backward: tanh' = 1 - h^2 from the FP32 h
                        uint32_t dk[8];
#pragma unroll
                        for (int t = 0; t < 8; ++t)
                            dk[t] = pack_bf16(1.0f - h[2 * t] * h[2 * t], 1.0f - h[2 * t + 1] * h[2 * t + 1]);
                        tmem_st8(lane_base + 256u + 128u * (uint32_t)(l - 1) + (uint32_t)(c0 >> 1), dk);
                    }
                } else {
                    float ga[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float wo = swo[c0 + j];
                        y_part += wo * h[j];
                        ga[j] = s_E * wo * (1.0f - h[j] * h[j]);
                    }
#pragma unroll
                    for (int g = 0; g < 2; ++g)
                        *reinterpret_cast<uint4*>(GA + 2 * cm_index(row, c0 + 8 * g, WW)) =
                            make_uint4(pack_bf16(ga[8 * g], ga[8 * g + 1]), pack_bf16(ga[8 * g + 2], ga[8 * g + 3]),
                                       pack_bf16(ga[8 * g + 4], ga[8 * g + 5]), pack_bf16(ga[8 * g + 6], ga[8 * g + 7]));
                }
            } else if (l > 1) {
                // tanh'(a_{l-1}): h_{L-1} is still in ACT (BF16 h); earlier
                // layers parked 1 - h^2 in TMEM
                uint32_t hw[8];
                const bool from_act = l - 1 == L - 1;
                if (from_act) {
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        const uint4 u = *reinterpret_cast<const uint4*>(ACT + 2 * cm_index(row, c0 + 8 * g, WW));
                        hw[4 * g] = u.x; hw[4 * g + 1] = u.y; hw[4 * g + 2] = u.z; hw[4 * g + 3] = u.w;
                    }
                } else {
                    tmem_ld8(lane_base + 256u + 128u * (uint32_t)(l - 2) + (uint32_t)(c0 >> 1), hw);
                }
                uint32_t pk[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float2 hh = unpack_bf16(hw[t]);
                    const float2 dd = from_act ? make_float2(1.0f - hh.x * hh.x, 1.0f - hh.y * hh.y) : hh;
                    pk[t] = pack_bf16(v[2 * t] * dd.x, v[2 * t + 1] * dd.y);
                }
#pragma unroll
                for (int g = 0; g < 2; ++g)
                    *reinterpret_cast<uint4*>(GA + 2 * cm_index(row, c0 + 8 * g, WW)) =
                        make_uint4(pk[4 * g], pk[4 * g + 1], pk[4 * g + 2], pk[4 * g + 3]);
            } else {
                const int ba = perm[row0 + row];
                if (ba >= 0) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4) {
                        float4 o = make_float4(v[j] * sis[c0 + j], v[j + 1] * sis[c0 + j + 1],
                                               v[j + 2] * sis[c0 + j + 2], v[j + 3] * sis[c0 + j + 3]);
                        *reinterpret_cast<float4*>(dEdG + (size_t)ba * ND + c0 + j) = o;
                    }
                }
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        if (fwd && l == L) ysum[hsel * M + row] = y_part;
        fence_proxy();
        fence_before();
        __syncthreads();
        fence_after();
        if (fwd && l == L && hsel == 0) {
            const int ba = perm[row0 + row];
            if (ba >= 0) Eatom[ba] = s_E * (ysum[row] + ysum[M + row] + b_out) + e_Z;
        }
    }
    if (!ok) {
        // a wait gave up: report, let started copies land, then release TMEM
        if (tid == 0) {
            atomicOr(&err->flags, ERR_TIMEOUT);
            for (int g = (issued > 2 ? issued - 2 : 0); g < issued; ++g)
                mbar_wait(bar_ld[g & 1], (uint32_t)((g >> 1) & 1));
        }
        __syncthreads();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static size_t tc_smem(int W, int L, bool db)
{
    const size_t A0_B = 128 * ND * 2, H_B = (size_t)128 * W * 2;
    const size_t WB_B = (size_t)W * (W > ND ? W : ND) * 2;
    return A0_B + (L > 1 ? (L - 1) : 1) * H_B + H_B + (db ? 2 : 1) * WB_B + 64 + 2 * 128 * 4 + 1024;
}

static size_t tc_wide_smem()
{
    return (size_t)128 * ND * 2 + 2 * (size_t)128 * WW * 2 + 2 * (size_t)WW * KCH * 2 + 64 + 2 * 128 * 4 +
           (size_t)(MAX_LAYERS * WW + WW + 2 * ND) * 4 + 1024;
}

bool network_tc_supported(int width, int n_hidden)
{
    if (n_hidden < 1 || n_hidden > MAX_LAYERS) return false;
    if (width == WW) return tc_wide_smem() <= 227 * 1024;
    if (width != 64 && width != 128) return false;
    return tc_smem(width, n_hidden, false) <= 227 * 1024;
}

size_t tc_weight_bytes(int width, int n_hidden)
{
    if (width == WW) return wide_chunk_offset(n_hidden, wide_nchunks(n_hidden), nullptr);
    return img_offset(width, n_hidden, 2 * n_hidden);
}

// weight images (BF16, core-matrix layout) and FP32 epilogue vectors of one type
void prepare_tc_weights(const Dev& d, int /*type*/, const double* blob, void* host_img, float* host_vec)
{
    const int W = d.width, L = d.n_hidden;
    unsigned char* img = static_cast<unsigned char*>(host_img);
    // blob pieces
    const double* Wl[MAX_LAYERS];
    const double* bl[MAX_LAYERS];
    size_t off = 0;
    int prev = ND;
    for (int l = 0; l < L; ++l) {
        Wl[l] = blob + off; off += (size_t)W * prev;
        bl[l] = blob + off; off += W;
        prev = W;
    }
    const double* w_out = blob + off; off += W;
    const double b_out = blob[off]; off += 1;
    const double* mu = blob + off; off += ND;
    const double* sigma = blob + off; off += ND;
    const double s_E = blob[off], e_Z = blob[off + 1];
    if (W == WW) {
        // chunked images: per phase, K-chunks of 64, each [N][64] core-matrix layout
        int g = 0;
        for (int p = 0; p < 2 * L; ++p) {
            const int l = wide_phase_layer(L, p), K = wide_phase_K(L, p), N = wide_phase_N(L, p);
            const int in = l == 1 ? ND : W;
            const double* Wm = Wl[l - 1];   // [W][in]
            for (int c = 0; c < K / KCH; ++c, ++g) {
                int Nc = 0;
                __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(img + wide_chunk_offset(L, g, &Nc));
                for (int n = 0; n < N; ++n)
                    for (int kk = 0; kk < KCH; ++kk) {
                        const int k = c * KCH + kk;
                        const double v = p < L ? Wm[(size_t)n * in + k] : Wm[(size_t)k * in + n];
                        dst[cm_index(n, kk, KCH)] = __float2bfloat16_rn((float)v);
                    }
            }
        }
    }
    for (int p = 0; p < 2 * L && W != WW; ++p) {
        const int l = p < L ? p + 1 : 2 * L - p;
        const int in = l == 1 ? ND : W;
        __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(img + img_offset(W, L, p));
        const double* Wm = Wl[l - 1];   // [W][in]
        if (p < L) {
            for (int n = 0; n < W; ++n)
                for (int k = 0; k < in; ++k) dst[cm_index(n, k, in)] = __float2bfloat16_rn((float)Wm[(size_t)n * in + k]);
        } else {
            for (int n = 0; n < in; ++n)
                for (int k = 0; k < W; ++k) dst[cm_index(n, k, W)] = __float2bfloat16_rn((float)Wm[(size_t)k * in + n]);
        }
    }
    float* v = host_vec;
    for (int l = 0; l < L; ++l)
        for (int c = 0; c < W; ++c) *v++ = (float)bl[l][c];
    for (int c = 0; c < W; ++c) *v++ = (float)w_out[c];
    for (int c = 0; c < ND; ++c) *v++ = (float)mu[c];
    for (int c = 0; c < ND; ++c) *v++ = (float)sigma[c];
    *v++ = (float)b_out;
    *v++ = (float)s_E;
    *v++ = (float)e_Z;
    *v++ = 0.0f;
}

template <int W, int L>
static size_t park_smem()
{
    const size_t WB_B = (size_t)W * (W > ND ? W : ND) * 2;
    return (size_t)128 * ND * 2 + (size_t)128 * W * 2 + WB_B + 64 + (size_t)(park_threads<W, L>() / 128) * 128 * 4 +
           (size_t)(L * W + W + 2 * ND) * 4 + 1024;
}

template <int W, int L>
static bool run_tc_park(const Dev& d, int t0, int nt, cudaStream_t st, bool urgent = false)
{
    if constexpr (park_cols<W, L>() <= 256) {
        if (nt <= 0) return true;
        const size_t sm = park_smem<W, L>();
        static size_t done = 0;
        if (sm > done) {
            cudaFuncSetAttribute(mlp_tc_park_kernel<W, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            done = sm;
        }
        if (urgent) {
            // the highest stream priority of the device for this launch: its
            // blocks are placed before those of concurrent kernels
            int least = 0, greatest = 0;
            cudaDeviceGetStreamPriorityRange(&least, &greatest);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributePriority;
            at[0].val.priority = greatest;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(nt);
            cfg.blockDim = dim3(park_threads<W, L>());
            cfg.dynamicSmemBytes = sm;
            cfg.stream = st;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            cudaLaunchKernelEx(&cfg, mlp_tc_park_kernel<W, L>, (const float*)d.G, (const int*)d.perm,
                               (const int*)d.tile_type, (const unsigned char*)d.wtc, d.wtc_bytes_per_type,
                               (const float*)d.wtc_vec, d.wtc_vec_per_type, (float*)d.Eatom, (float*)d.dEdG, d.err,
                               t0);
            return true;
        }
        mlp_tc_park_kernel<W, L><<<nt, park_threads<W, L>(), sm, st>>>(
            (const float*)d.G, d.perm, d.tile_type, (const unsigned char*)d.wtc, d.wtc_bytes_per_type, d.wtc_vec,
            d.wtc_vec_per_type, (float*)d.Eatom, (float*)d.dEdG, d.err, t0);
        return true;
    }
    return false;
}

template <int W, int L>
static void run_tc(const Dev& d, cudaStream_t st)
{
    if (run_tc_park<W, L>(d, 0, d.rows_pad / 128, st)) return;
    const bool db = tc_smem(W, L, true) <= 227 * 1024;
    const size_t sm = tc_smem(W, L, db);
    static size_t done[2] = {0, 0};
    if (db) {
        if (sm > done[1]) {
            cudaFuncSetAttribute(mlp_tc_kernel<W, L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            done[1] = sm;
        }
        mlp_tc_kernel<W, L, true><<<d.rows_pad / 128, TC_THREADS, sm, st>>>(
            (const float*)d.G, d.perm, d.tile_type, (const unsigned char*)d.wtc, d.wtc_bytes_per_type, d.wtc_vec,
            d.wtc_vec_per_type, (float*)d.Eatom, (float*)d.dEdG, d.err);
    } else {
        if (sm > done[0]) {
            cudaFuncSetAttribute(mlp_tc_kernel<W, L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            done[0] = sm;
        }
        mlp_tc_kernel<W, L, false><<<d.rows_pad / 128, TC_THREADS, sm, st>>>(
            (const float*)d.G, d.perm, d.tile_type, (const unsigned char*)d.wtc, d.wtc_bytes_per_type, d.wtc_vec,
            d.wtc_vec_per_type, (float*)d.Eatom, (float*)d.dEdG, d.err);
    }
}

template <int L>
static void run_tc_wide(const Dev& d, cudaStream_t st)
{
    const size_t sm = tc_wide_smem();
    static size_t done = 0;
    if (sm > done) {
        cudaFuncSetAttribute(mlp_tc_wide_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        done = sm;
    }
    mlp_tc_wide_kernel<L><<<d.rows_pad / 128, TC_THREADS, sm, st>>>(
        (const float*)d.G, d.perm, d.tile_type, (const unsigned char*)d.wtc, d.wtc_bytes_per_type, d.wtc_vec,
        d.wtc_vec_per_type, (float*)d.Eatom, (float*)d.dEdG, d.err);
}

// Whether launch_network_tiles can run this configuration's network (widths
// 64 / 128 with the hidden activations parked in tensor memory).
bool network_tiles_available(const Dev& d)
{
    if (d.precision != 2 || d.rows_pad == 0) return false;
    if (d.width == 64) return 64 + (d.n_hidden - 1) * 32 <= 256;
    if (d.width == 128) return 128 + (d.n_hidden - 1) * 64 <= 256;
    return false;
}

// The tiles t0 .. t0+nt-1 only (widths 64 / 128 with parked activations);
// false when the configuration uses another network kernel.
bool launch_network_tiles(const Dev& d, int t0, int nt, cudaStream_t st, bool urgent)
{
    if (d.width == 64) {
        switch (d.n_hidden) {
            case 1: return run_tc_park<64, 1>(d, t0, nt, st, urgent);
            case 2: return run_tc_park<64, 2>(d, t0, nt, st, urgent);
            case 3: return run_tc_park<64, 3>(d, t0, nt, st, urgent);
            default: return run_tc_park<64, 4>(d, t0, nt, st, urgent);
        }
    }
    if (d.width == 128) {
        switch (d.n_hidden) {
            case 1: return run_tc_park<128, 1>(d, t0, nt, st, urgent);
            case 2: return run_tc_park<128, 2>(d, t0, nt, st, urgent);
            case 3: return run_tc_park<128, 3>(d, t0, nt, st, urgent);
            default: return run_tc_park<128, 4>(d, t0, nt, st, urgent);
        }
    }
    return false;
}

void launch_network_tc(const Dev& d, cudaStream_t st)
{
    if (d.rows_pad == 0) return;
    if (d.width == WW) {
        switch (d.n_hidden) {
            case 1: run_tc_wide<1>(d, st); break;
            case 2: run_tc_wide<2>(d, st); break;
            case 3: run_tc_wide<3>(d, st); break;
            default: run_tc_wide<4>(d, st); break;
        }
        return;
    }
    if (d.width == 64) {
        switch (d.n_hidden) {
            case 1: run_tc<64, 1>(d, st); break;
            case 2: run_tc<64, 2>(d, st); break;
            case 3: run_tc<64, 3>(d, st); break;
            default: run_tc<64, 4>(d, st); break;
        }
    } else {
        switch (d.n_hidden) {
            case 1: run_tc<128, 1>(d, st); break;
            case 2: run_tc<128, 2>(d, st); break;
            case 3: run_tc<128, 3>(d, st); break;
            default: run_tc<128, 4>(d, st); break;
        }
    }
}

// ---------------------------------------------------------------------------
// Self-test of the bounded waits: one thread initialises an mbarrier that
// nothing arrives on and waits on it with mbar_wait, exactly as the network
// kernels wait on their MMA and copy barriers; the bound expires after
// ~WAIT_CYCLES and the kernel records the timeout and returns.
// ---------------------------------------------------------------------------
__device__ int g_wait_selftest;

__global__ void wait_selftest_kernel(long long cycles)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const long long t0 = clock64();
    bool done = false;
    while (!(done = mbar_try(b, 0u))) {
        if (clock64() - t0 > cycles) break;
    }
    g_wait_selftest = done ? 0 : 1;
}

int run_wait_selftest(cudaStream_t st, long long cycles, int* timed_out)
{
    wait_selftest_kernel<<<1, 1, 0, st>>>(cycles);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(timed_out, g_wait_selftest, sizeof(int), 0,
                                                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace pimd
