// gfn.cu -- graph-field-network force head (Sec. 2.2): forces read out
// directly from edge representations, no energy and no adjoint.
//
//   m_i^(l)    = sum_j SiLU(W_m e_ij^(l) + b_m)
//   n_i^(l+1)  = n_i^(l) + W_v2 SiLU(W_v1 [n_i^(l); m_i^(l)] + b_v1) + b_v2
//   e_ij^(l+1) = e_ij^(l) + W_a2 SiLU(W_a1 (n_i^(l) + n_j^(l)) + b_a1) + b_a2
//   F_ij       = s_F fc(r_ij) (x_i - x_j) / r_ij (w_f2 . SiLU(W_f1 e_ij^(L) + b_f1) + b_f2)
//
// with n_i^(0) an element embedding and e_ij^(0) = W_e rho(r_ij) + b_e over
// the 32 radial functions of the descriptors. FP32 throughout.
//
// Work decomposition: a CTA of 128 threads per bead-atom takes its directed
// edges (neighbour slots) 32 rows at a time; every dense layer is a 32 x F
// tile product X W^T with X in shared memory and W^T streamed through shared
// memory in chunks of 32 rows of K (weights are stored transposed, [K][F]),
// thread (row group, column group) accumulating a 4 x F/16 block. The
// segmented sum m_i stays in the CTA; the edge state e (slots x F) lives in
// the workspace between iterations. Node updates run as 32-atom tiles.
#include <cuda_runtime.h>

#include "common.cuh"
#include "geom.cuh"
#include "kernels.h"

namespace pimd {

namespace {

constexpr int GR = 32;     // rows per tile
constexpr int GT = 128;    // threads per CTA: 8 row groups x 16 column groups
constexpr int GKC = 32;    // K rows of W^T per shared-memory chunk

__device__ __forceinline__ float silu(float v) { return v / (1.0f + expf(-v)); }

// acc[r][c] += sum_k X[4 rg + r][k] W^T[k][CPT cg + c] over k < K (K a multiple
// of GKC); X: shared [GR][ldx]; WT: global [K][F]; Ws: shared [GKC][F]
template <int F>
__device__ __forceinline__ void tile_gemm(const float* __restrict__ Xs, int ldx, int K,
                                          const float* __restrict__ WT, float* __restrict__ Ws,
                                          float (&acc)[4][F / 16])
{
    constexpr int CPT = F / 16;
    const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;
    for (int k0 = 0; k0 < K; k0 += GKC) {
        __syncthreads();   // the previous chunk (and the writers of X) are done
        const float4* src = reinterpret_cast<const float4*>(WT + (size_t)k0 * F);
        for (int q = tid; q < GKC * F / 4; q += GT) reinterpret_cast<float4*>(Ws)[q] = __ldg(src + q);
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GKC; ++kk) {
            float xv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) xv[r] = Xs[(4 * rg + r) * ldx + k0 + kk];
            float wv[CPT];
#pragma unroll
            for (int c4 = 0; c4 < CPT / 2; ++c4) {
                const float2 w2 = reinterpret_cast<const float2*>(Ws + kk * F + cg * CPT)[c4];
                wv[2 * c4] = w2.x;
                wv[2 * c4 + 1] = w2.y;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < CPT; ++c) acc[r][c] = fmaf(xv[r], wv[c], acc[r][c]);
        }
    }
}

template <int F>
__device__ __forceinline__ void zero(float (&acc)[4][F / 16])
{
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < F / 16; ++c) acc[r][c] = 0.0f;
}

// one tile's pair geometry: r, fc, r_ij = x_j - x_i (FP32 pair rule of the
// descriptors) and the neighbour index; rows beyond the list are marked j = -1
struct TileGeo {
    float r[GR], fc[GR], d[GR][3];
    int j[GR];
};

}  // namespace

// MODE 0: n^(0) and e^(0); MODE 1: iteration l (messages, edge update);
// MODE 2: force readout, forces and per-atom virial
template <int F, int MODE>
__global__ void __launch_bounds__(GT) gfn_edge_kernel(
    const float4* __restrict__ x, const int* __restrict__ ba_sys, const BeadSys* __restrict__ bsys,
    const Rep* __restrict__ reps, const int* __restrict__ atype, const int* __restrict__ nbr,
    const int* __restrict__ nnb, int maxnb, GfnParams gp, int l, const float* __restrict__ W,
    float* __restrict__ nf, float* __restrict__ mf, float* __restrict__ ef, float4* __restrict__ f,
    float* __restrict__ wbuf, float* __restrict__ Eatom)
{
    constexpr int CPT = F / 16;
    extern __shared__ __align__(16) float smf[];
    float* Xs = smf;                 // [GR][F] (MODE 0: [GR][NR])
    float* Hs = Xs + GR * F;         // [GR][F]
    float* Ws = Hs + GR * F;         // [GKC][F]
    float* red = Ws + GKC * F;       // [8][F] or [8][12]
    __shared__ TileGeo geo;
    const int b = blockIdx.x;
    const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;
    const BeadSys sy = bsys[ba_sys[b]];
    const Rep rp = reps[sy.rep];
    const int n = min(nnb[b], maxnb);
    const float4 xi = x[b];
    float* eb = ef + (size_t)b * maxnb * F;

    if (MODE == 0) {
        const int t = atype[rp.atom0 + (b - sy.ba0)];
        for (int c = tid; c < F; c += GT) nf[(size_t)b * F + c] = W[gp.o_emb + (size_t)t * F + c];
        if (tid == 0) Eatom[b] = 0.0f;
    }
    float msum[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) msum[c] = 0.0f;
    float fi[3] = {0.0f, 0.0f, 0.0f}, wl[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) wl[q] = 0.0f;

    for (int t0 = 0; t0 < n; t0 += GR) {
        const int rows = min(GR, n - t0);
        __syncthreads();   // the previous tile's readers of geo / X / H are done
        if (tid < GR) {
            if (tid < rows) {
                const int j = nbr[(size_t)b * maxnb + t0 + tid];
                float dx, dy, dz;
                pair_vec(rp, xi, x[sy.ba0 + j], dx, dy, dz);
                const float r = sqrtf(dx * dx + dy * dy + dz * dz);
                float fc, dfc;
                cutoff(r, gp.rc, gp.pi_over_rc, fc, dfc);
                geo.r[tid] = r;
                geo.fc[tid] = fc;
                geo.d[tid][0] = dx;
                geo.d[tid][1] = dy;
                geo.d[tid][2] = dz;
                geo.j[tid] = j;
            } else {
                geo.r[tid] = 0.0f;
                geo.fc[tid] = 0.0f;
                geo.d[tid][0] = geo.d[tid][1] = geo.d[tid][2] = 0.0f;
                geo.j[tid] = -1;
            }
        }
        __syncthreads();
        float acc[4][CPT];
        if (MODE == 0) {
            // rho(r) of the tile's rows, then e^(0) = W_e rho + b_e
            for (int q = tid; q < GR * NR; q += GT) {
                const int row = q / NR, k = q % NR;
                const float tt = geo.r[row] - gp.r_mu[k];
                Xs[q] = row < rows ? expf(-gp.eta_R * tt * tt) * geo.fc[row] : 0.0f;
            }
            zero<F>(acc);
            tile_gemm<F>(Xs, NR, NR, W + gp.o_We, Ws, acc);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = 4 * rg + r;
                if (row < rows)
#pragma unroll
                    for (int c = 0; c < CPT; ++c)
                        eb[(size_t)(t0 + row) * F + cg * CPT + c] = acc[r][c] + W[gp.o_be + cg * CPT + c];
            }
        } else if (MODE == 1) {
            const unsigned* o = gp.o_it[l];
            // messages: SiLU(W_m e + b_m) summed over the rows
            for (int q = tid; q < GR * F / 4; q += GT) {
                const int row = q / (F / 4);
                reinterpret_cast<float4*>(Xs)[q] =
                    row < rows ? reinterpret_cast<const float4*>(eb + (size_t)t0 * F)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            zero<F>(acc);
            tile_gemm<F>(Xs, F, F, W + o[0], Ws, acc);
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (4 * rg + r < rows)
#pragma unroll
                    for (int c = 0; c < CPT; ++c) msum[c] += silu(acc[r][c] + W[o[1] + cg * CPT + c]);
            // edge update from the pre-update node states: e += W_a2 SiLU(W_a1 (n_i + n_j) + b_a1) + b_a2
            __syncthreads();   // X is rewritten below
            for (int q = tid; q < GR * F / 4; q += GT) {
                const int row = q / (F / 4), c4 = q % (F / 4);
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (row < rows) {
                    const float4 a = reinterpret_cast<const float4*>(nf + (size_t)b * F)[c4];
                    const float4 bb = reinterpret_cast<const float4*>(nf + (size_t)(sy.ba0 + geo.j[row]) * F)[c4];
                    v = make_float4(a.x + bb.x, a.y + bb.y, a.z + bb.z, a.w + bb.w);
                }
                reinterpret_cast<float4*>(Xs)[q] = v;
            }
            zero<F>(acc);
            tile_gemm<F>(Xs, F, F, W + o[6], Ws, acc);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < CPT; ++c)
                    Hs[(4 * rg + r) * F + cg * CPT + c] = silu(acc[r][c] + W[o[7] + cg * CPT + c]);
            zero<F>(acc);
            tile_gemm<F>(Hs, F, F, W + o[8], Ws, acc);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = 4 * rg + r;
                if (row < rows)
#pragma unroll
                    for (int c = 0; c < CPT; ++c)
                        eb[(size_t)(t0 + row) * F + cg * CPT + c] += acc[r][c] + W[o[9] + cg * CPT + c];
            }
        } else {
            // readout phi_f(e) per row, then F_ij = s_F fc phi (x_i - x_j) / r
            for (int q = tid; q < GR * F / 4; q += GT) {
                const int row = q / (F / 4);
                reinterpret_cast<float4*>(Xs)[q] =
                    row < rows ? reinterpret_cast<const float4*>(eb + (size_t)t0 * F)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            zero<F>(acc);
            tile_gemm<F>(Xs, F, F, W + gp.o_Wf1, Ws, acc);
            float ph[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float s = 0.0f;
#pragma unroll
                for (int c = 0; c < CPT; ++c)
                    s = fmaf(W[gp.o_wf2 + cg * CPT + c], silu(acc[r][c] + W[gp.o_bf1 + cg * CPT + c]), s);
                // the 16 column groups of a row group share one half-warp
#pragma unroll
                for (int o = 8; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                ph[r] = s + gp.b_f2;
            }
            if (cg == 0) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int row = 4 * rg + r;
                    if (row < rows) {
                        const float rr = geo.r[row];
                        const float sc = gp.s_F * geo.fc[row] * ph[r] / rr;
                        const float d3[3] = {geo.d[row][0], geo.d[row][1], geo.d[row][2]};
                        const float Fij[3] = {-sc * d3[0], -sc * d3[1], -sc * d3[2]};
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            fi[a] += Fij[a];
#pragma unroll
                            for (int c = 0; c < 3; ++c) wl[3 * a + c] -= 0.5f * d3[a] * Fij[c];
                        }
                    }
                }
            }
        }
    }
    if (MODE == 1) {
        // m_i: column sums over the 8 row groups
        __syncthreads();
#pragma unroll
        for (int c = 0; c < CPT; ++c) red[rg * F + cg * CPT + c] = msum[c];
        __syncthreads();
        for (int c = tid; c < F; c += GT) {
            float s = 0.0f;
#pragma unroll
            for (int g = 0; g < 8; ++g) s += red[g * F + c];
            mf[(size_t)b * F + c] = s;
        }
    } else if (MODE == 2) {
        __syncthreads();
        if (cg == 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) red[rg * 12 + a] = fi[a];
#pragma unroll
            for (int q = 0; q < 9; ++q) red[rg * 12 + 3 + q] = wl[q];
        }
        __syncthreads();
        if (tid < 12) {
            float s = 0.0f;
#pragma unroll
            for (int g = 0; g < 8; ++g) s += red[g * 12 + tid];
            red[8 * 12 + tid] = s;
        }
        __syncthreads();
        if (tid == 0) f[b] = make_float4(red[96], red[97], red[98], 0.0f);
        if (tid < 9) wbuf[(size_t)b * 9 + tid] = red[99 + tid];
    }
}

// node update of 32 bead-atoms: n += W_v2 SiLU(W_v1 [n; m] + b_v1) + b_v2
template <int F>
__global__ void __launch_bounds__(GT) gfn_node_kernel(int B, GfnParams gp, int l, const float* __restrict__ W,
                                                      float* __restrict__ nf, const float* __restrict__ mf)
{
    constexpr int CPT = F / 16;
    extern __shared__ __align__(16) float smf[];
    float* Xs = smf;                  // [GR][2F]
    float* Hs = Xs + GR * 2 * F;      // [GR][F]
    float* Ws = Hs + GR * F;          // [GKC][F]
    const int a0 = blockIdx.x * GR;
    const int rows = min(GR, B - a0);
    const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;
    const unsigned* o = gp.o_it[l];
    for (int q = tid; q < GR * 2 * F / 4; q += GT) {
        const int row = q / (2 * F / 4), c4 = q % (2 * F / 4);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < rows)
            v = c4 < F / 4 ? reinterpret_cast<const float4*>(nf + (size_t)(a0 + row) * F)[c4]
                           : reinterpret_cast<const float4*>(mf + (size_t)(a0 + row) * F)[c4 - F / 4];
        reinterpret_cast<float4*>(Xs)[q] = v;
    }
    float acc[4][CPT];
    zero<F>(acc);
    tile_gemm<F>(Xs, 2 * F, 2 * F, W + o[2], Ws, acc);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < CPT; ++c) Hs[(4 * rg + r) * F + cg * CPT + c] = silu(acc[r][c] + W[o[3] + cg * CPT + c]);
    zero<F>(acc);
    tile_gemm<F>(Hs, F, F, W + o[4], Ws, acc);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int row = 4 * rg + r;
        if (row < rows)
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int col = cg * CPT + c;
                // this row's n was read into X before the first product
                nf[(size_t)(a0 + row) * F + col] = Xs[row * 2 * F + col] + acc[r][c] + W[o[5] + col];
            }
    }
}

namespace {

template <int F>
size_t edge_smem() { return sizeof(float) * (2 * GR * F + GKC * F + 8 * F); }
template <int F>
size_t node_smem() { return sizeof(float) * (3 * GR * F + GKC * F); }

template <int F>
void run_gfn(const Dev& d, cudaStream_t st)
{
    const GfnParams& gp = d.gfn;
    const float* W = d.gfn_w;
    const size_t se = edge_smem<F>(), sn = node_smem<F>();
    {
        static size_t d0 = 0, d1 = 0, d2 = 0, d3 = 0;
        set_smem(gfn_edge_kernel<F, 0>, se, d0);
        set_smem(gfn_edge_kernel<F, 1>, se, d1);
        set_smem(gfn_edge_kernel<F, 2>, se, d2);
        set_smem(gfn_node_kernel<F>, sn, d3);
    }
    const float4* x = (const float4*)d.x;
    gfn_edge_kernel<F, 0><<<d.B, GT, se, st>>>(x, d.ba_sys, d.bsys, d.reps, d.atype, d.nbr, d.nnb, d.maxnb, gp, 0, W,
                                               d.gfn_n, d.gfn_m, d.gfn_e, (float4*)d.f, (float*)d.wbuf,
                                               (float*)d.Eatom);
    for (int l = 0; l < gp.L; ++l) {
        gfn_edge_kernel<F, 1><<<d.B, GT, se, st>>>(x, d.ba_sys, d.bsys, d.reps, d.atype, d.nbr, d.nnb, d.maxnb, gp, l,
                                                   W, d.gfn_n, d.gfn_m, d.gfn_e, (float4*)d.f, (float*)d.wbuf,
                                                   (float*)d.Eatom);
        gfn_node_kernel<F><<<(d.B + GR - 1) / GR, GT, sn, st>>>(d.B, gp, l, W, d.gfn_n, d.gfn_m);
    }
    gfn_edge_kernel<F, 2><<<d.B, GT, se, st>>>(x, d.ba_sys, d.bsys, d.reps, d.atype, d.nbr, d.nnb, d.maxnb, gp, 0, W,
                                               d.gfn_n, d.gfn_m, d.gfn_e, (float4*)d.f, (float*)d.wbuf,
                                               (float*)d.Eatom);
}

}  // namespace

void launch_gfn(const Dev& d, cudaStream_t st)
{
    switch (d.gfn.F) {
    case 32: run_gfn<32>(d, st); break;
    case 64: run_gfn<64>(d, st); break;
    default: run_gfn<128>(d, st); break;
    }
}

int gfn_kernels_per_eval(int L) { return 2 + 2 * L; }

}  // namespace pimd
