// nbr.cu -- a2: neighbour lists under the exact FP32 rule
//   d = x_j - x_i, d -= L rint(d / L) (FP32 box), r2 = (dx dx + dy dy) + dz dz
//   without contraction, j in N(i) iff r2 < (float)(r_c^2),
// stored per bead-atom as ascending atom indices within its bead.
//
// Periodic beads whose box holds >= 3 cells of edge >= r_c per side use cell
// lists: one block per bead bins its atoms (shared-memory counting sort),
// then one warp per bead-atom applies the rule to the 27 stencil cells and
// sorts what passes. Other beads (gas phase, small boxes) scan all atoms of
// the bead in ascending order, which yields sorted lists directly.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace pimd {

namespace {

__device__ __forceinline__ float3 pos_f32(const float4& v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 pos_f32(const Dbl4& v)
{
    return make_float3(__double2float_rn(v.x), __double2float_rn(v.y), __double2float_rn(v.z));
}

// the inclusion rule on FP32 positions
__device__ __forceinline__ bool within(const Rep& rp, const float3& xi, const float3& xj, float rc2)
{
    float dx = __fsub_rn(xj.x, xi.x), dy = __fsub_rn(xj.y, xi.y), dz = __fsub_rn(xj.z, xi.z);
    if (rp.periodic) {
        dx = __fsub_rn(dx, __fmul_rn(rp.Lf[0], rintf(__fmul_rn(dx, rp.invLf[0]))));
        dy = __fsub_rn(dy, __fmul_rn(rp.Lf[1], rintf(__fmul_rn(dy, rp.invLf[1]))));
        dz = __fsub_rn(dz, __fmul_rn(rp.Lf[2], rintf(__fmul_rn(dz, rp.invLf[2]))));
    }
    const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    return r2 < rc2;
}

// cell coordinate along one axis of a periodic box (wrapped fractional coordinate)
__device__ __forceinline__ int cell_axis(float x, float invL, int nc)
{
    float s = __fmul_rn(x, invL);
    s = s - floorf(s);
    int c = (int)(s * (float)nc);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__device__ __forceinline__ int3 cell_of(const Rep& rp, const float3& p)
{
    return make_int3(cell_axis(p.x, rp.invLf[0], rp.nc[0]), cell_axis(p.y, rp.invLf[1], rp.nc[1]),
                     cell_axis(p.z, rp.invLf[2], rp.nc[2]));
}

}  // namespace

// one block per bead using cells: counting sort of its atoms into cells
template <typename V4>
__global__ void cell_build_kernel(const V4* __restrict__ x, const BeadSys* __restrict__ bsys,
                                  const Rep* __restrict__ reps, const int* __restrict__ cell_bs,
                                  int* __restrict__ cell_start, int* __restrict__ cell_cnt,
                                  int* __restrict__ cell_atoms)
{
    extern __shared__ int sh[];   // [ncells] counters, then [ncells] fill offsets
    const BeadSys sy = bsys[cell_bs[blockIdx.x]];
    const Rep& rp = reps[sy.rep];
    const int nc = rp.ncells;
    int* cnt = sh;
    int* off = sh + nc;
    const int cbase = rp.cell0 + sy.bead * nc;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) cnt[c] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < sy.N; i += blockDim.x) {
        const int3 c = cell_of(rp, pos_f32(x[sy.ba0 + i]));
        atomicAdd(&cnt[(c.x * rp.nc[1] + c.y) * rp.nc[2] + c.z], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int c = 0; c < nc; ++c) {
            off[c] = acc;
            cell_start[cbase + c] = sy.ba0 + acc;
            cell_cnt[cbase + c] = cnt[c];
            acc += cnt[c];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < sy.N; i += blockDim.x) {
        const int3 c = cell_of(rp, pos_f32(x[sy.ba0 + i]));
        const int pos = atomicAdd(&off[(c.x * rp.nc[1] + c.y) * rp.nc[2] + c.z], 1);
        cell_atoms[sy.ba0 + pos] = i;
    }
}

// Neighbours of bead-atom il (FP32 position xi) with rule radius r2cut, in
// ascending order into out[0 .. cap); returns the count (may exceed cap).
// Beads without cells scan all their atoms; beads with cells scan the 27
// stencil cells and order what passes: through a bitmap over the bead's atom
// indices when the bead has at most 32 x NBR_BM_WORDS atoms (BM: the warp's
// shared bitmap), else by a bitonic sort (L: the warp's shared sort buffer).
constexpr int NBR_BM_WORDS = 512;   // bitmap words per warp: beads of up to 16,384 atoms

template <typename V4>
__device__ int scan_list(const V4* __restrict__ x, const BeadSys& sy, const Rep& rp, int il, const float3& xi,
                         const int* __restrict__ cell_start, const int* __restrict__ cell_cnt,
                         const int* __restrict__ cell_atoms, float r2cut, int* __restrict__ out, int cap, int* L,
                         unsigned* BM, unsigned lane)
{
    int cnt = 0;
    if (rp.ncells == 0) {
        // four chunks of 32 atoms per round: their positions are loaded
        // together, then tested and stored in ascending order
        constexpr int KS = 4;
        for (int j0 = 0; j0 < sy.N; j0 += 32 * KS) {
            float3 pj[KS];
#pragma unroll
            for (int k = 0; k < KS; ++k) {
                const int j = j0 + 32 * k + (int)lane;
                pj[k] = j < sy.N ? pos_f32(x[sy.ba0 + j]) : xi;
            }
#pragma unroll
            for (int k = 0; k < KS; ++k) {
                if (j0 + 32 * k >= sy.N) break;   // warp-uniform
                const int j = j0 + 32 * k + (int)lane;
                const bool in = j < sy.N && j != il && within(rp, xi, pj[k], r2cut);
                const unsigned m = __ballot_sync(0xffffffffu, in);
                const int pos = cnt + __popc(m & ((1u << lane) - 1u));
                if (in && pos < cap) out[pos] = j;
                cnt += __popc(m);
            }
        }
    } else {
        const int3 ci = cell_of(rp, xi);
        const int cbase = rp.cell0 + sy.bead * rp.ncells;
        // lane s < 27 holds stencil cell s; an inclusive scan of the counts
        // flattens the 27 cells into one candidate list
        int st = 0, ct = 0;
        if (lane < 27) {
            int cx = ci.x + (int)lane / 9 - 1, cy = ci.y + ((int)lane / 3) % 3 - 1, cz = ci.z + (int)lane % 3 - 1;
            cx += cx < 0 ? rp.nc[0] : (cx >= rp.nc[0] ? -rp.nc[0] : 0);
            cy += cy < 0 ? rp.nc[1] : (cy >= rp.nc[1] ? -rp.nc[1] : 0);
            cz += cz < 0 ? rp.nc[2] : (cz >= rp.nc[2] ? -rp.nc[2] : 0);
            const int cell = cbase + (cx * rp.nc[1] + cy) * rp.nc[2] + cz;
            st = cell_start[cell];
            ct = cell_cnt[cell];
        }
        int incl = ct;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int words = (sy.N + 31) >> 5;
        const bool use_bm = words <= NBR_BM_WORDS;
        if (use_bm) {
            for (int w = (int)lane; w < words; w += 32) BM[w] = 0u;
            __syncwarp();
        }
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + (int)lane;
            // stencil cell of candidate t: first s with incl[s] > t
            int lo = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
                if (v <= t) lo += step;
            }
            const int sc = lo > 26 ? 26 : lo;
            const int base = __shfl_sync(0xffffffffu, st, sc);
            const int before = __shfl_sync(0xffffffffu, incl - ct, sc);
            bool in = false;
            int j = -1;
            if (t < total) {
                j = cell_atoms[base + (t - before)];
                in = j != il && within(rp, xi, pos_f32(x[sy.ba0 + j]), r2cut);
            }
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (use_bm) {
                if (in) atomicOr(&BM[j >> 5], 1u << (j & 31));
            } else {
                const int pos = cnt + __popc(m & ((1u << lane) - 1u));
                if (in && pos < cap) L[pos] = j;
            }
            cnt += __popc(m);
        }
        __syncwarp();
        if (use_bm) {
            // ascending order: 32 bitmap words at a time, lane -> word, the
            // words' set bits placed by a prefix sum of their counts
            int base = 0;
            for (int w0 = 0; w0 < words; w0 += 32) {
                const int w = w0 + (int)lane;
                unsigned wv = w < words ? BM[w] : 0u;
                const int pc = __popc(wv);
                int inc = pc;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, inc, o);
                    if ((int)lane >= o) inc += v;
                }
                int pos = base + inc - pc;
                while (wv) {
                    const int bit = __ffs(wv) - 1;
                    if (pos < cap) out[pos] = (w << 5) + bit;
                    ++pos;
                    wv &= wv - 1u;
                }
                base += __shfl_sync(0xffffffffu, inc, 31);
            }
            return cnt;
        }
        // ascending order: bitonic sort over the next power of two, padded
        const int m = cnt < cap ? cnt : cap;
        int n2 = 1;
        while (n2 < m) n2 <<= 1;
        for (int t = m + (int)lane; t < n2; t += 32) L[t] = 0x7fffffff;
        __syncwarp();
        for (int k = 2; k <= n2; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int t = (int)lane; t < n2; t += 32) {
                    const int p = t ^ jj;
                    if (p > t) {
                        const int a = L[t], c = L[p];
                        const bool up = (t & k) == 0;
                        if ((a > c) == up) {
                            L[t] = c;
                            L[p] = a;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (int t = (int)lane; t < m; t += 32) out[t] = L[t];
    }
    return cnt;
}

// Verlet candidates: a pair's distance changes by at most the sum of its two
// atoms' displacements, so a bead's candidates stay complete while the two
// largest displacements (FP32 positions, since the last build) sum to less
// than 0.98 skin; block per bead, top-two reduction.
__device__ __forceinline__ void top2_merge(float& a1, float& a2, float b1, float b2)
{
    // (a1 >= a2), (b1 >= b2) -> the two largest of the four
    const float hi = fmaxf(a1, b1), lo = fminf(a1, b1);
    a2 = fmaxf(lo, fmaxf(a2, b2));
    a1 = hi;
}

template <typename V4>
__global__ void skin_check_kernel(const V4* __restrict__ x, const BeadSys* __restrict__ bsys,
                                  const Rep* __restrict__ reps, const float4* __restrict__ xref,
                                  int* __restrict__ rebuild)
{
    __shared__ float red[2][32];
    const BeadSys sy = bsys[blockIdx.x];
    const Rep& rp = reps[sy.rep];
    float m1 = 0.0f, m2 = 0.0f;
    for (int i = threadIdx.x; i < sy.N; i += blockDim.x) {
        const float3 p = pos_f32(x[sy.ba0 + i]);
        const float4 r = xref[sy.ba0 + i];
        const float dx = p.x - r.x, dy = p.y - r.y, dz = p.z - r.z;
        const float d = sqrtf(dx * dx + dy * dy + dz * dz);   // +inf after a reset of the references
        top2_merge(m1, m2, d, 0.0f);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const float b1 = __shfl_xor_sync(0xffffffffu, m1, o), b2 = __shfl_xor_sync(0xffffffffu, m2, o);
        top2_merge(m1, m2, b1, b2);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = m1;
        red[1][threadIdx.x >> 5] = m2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a1 = red[0][0], a2 = red[1][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) top2_merge(a1, a2, red[0][w], red[1][w]);
        rebuild[blockIdx.x] = (rp.skin > 0.0f && !(a1 + a2 < 0.98f * rp.skin)) ? 1 : 0;
    }
}

// warp per bead-atom. With a skin: rebuild the candidates (r < r_c + skin)
// when the bead is flagged, then keep the candidates the exact rule accepts,
// in their ascending order, so the list equals a full scan; without a skin,
// or when the candidates overflowed their slots, scan directly.
template <typename V4>
__global__ void __launch_bounds__(256) nbr_kernel(const V4* __restrict__ x, const int* __restrict__ ba_sys,
                                                  const BeadSys* __restrict__ bsys, const Rep* __restrict__ reps,
                                                  const int* __restrict__ cell_start, const int* __restrict__ cell_cnt,
                                                  const int* __restrict__ cell_atoms, float rc2, int maxnb, int B,
                                                  int* __restrict__ nbr, int* __restrict__ nnb,
                                                  DevErr* __restrict__ err, int* __restrict__ cand,
                                                  int* __restrict__ ncand, float4* __restrict__ xref,
                                                  const int* __restrict__ rebuild, int maxcand, int b0,
                                                  const int4* __restrict__ ba_info)
{
    __shared__ int lst[8][PIMD_SORT_CAP];
    __shared__ unsigned bmap[8][NBR_BM_WORDS];
    const int wib = threadIdx.x >> 5;
    const int b = b0 + blockIdx.x * (blockDim.x >> 5) + wib;   // bead-atoms b0 .. B-1
    const unsigned lane = lane_id();
    if (b >= B) return;
    // the bead-atom's record in one load (bead-system, first bead-atom,
    // atoms, replica) and its candidate count alongside, so that the
    // replica record and the rebuild flag form the second round of loads
    int bs;
    BeadSys sy;
    int nc0 = 0;
    if (ba_info) {
        const int4 bi = ba_info[b];
        if (maxcand > 0) nc0 = ncand[b];
        bs = bi.x;
        sy.ba0 = bi.y;
        sy.N = bi.z;
        sy.rep = bi.w;
    } else {
        bs = ba_sys[b];
        sy = bsys[bs];
        if (maxcand > 0) nc0 = ncand[b];
    }
    const Rep& rp = reps[sy.rep];
    if (ba_info) sy.bead = bs - rp.bs0;
    const int il = b - sy.ba0;
    const float3 xi = pos_f32(x[b]);
    int* out = nbr + (size_t)b * maxnb;
    int cnt;
    if (rp.skin > 0.0f && maxcand > 0) {
        int* cl = cand + (size_t)b * maxcand;
        int nc = nc0;
        if (rebuild[bs]) {
            nc = scan_list(x, sy, rp, il, xi, cell_start, cell_cnt, cell_atoms, rp.rcs2, cl, maxcand, lst[wib], bmap[wib], lane);
            if (lane == 0) {
                ncand[b] = nc;
                xref[b] = make_float4(xi.x, xi.y, xi.z, 0.0f);
            }
            __syncwarp();   // the candidates written by all lanes are read by all lanes below
        }
        if (nc <= maxcand) {
            // groups of four chunks of 32: the group's candidate indices
            // first, then their positions (independent loads), then the rule
            constexpr int KC = 4;
            cnt = 0;
            for (int g0 = 0; g0 < nc; g0 += 32 * KC) {
                int jv[KC];
                float3 pv[KC];
#pragma unroll
                for (int k = 0; k < KC; ++k) {
                    const int t = g0 + 32 * k + (int)lane;
                    jv[k] = t < nc ? cl[t] : -1;
                }
#pragma unroll
                for (int k = 0; k < KC; ++k) pv[k] = jv[k] >= 0 ? pos_f32(x[sy.ba0 + jv[k]]) : xi;
#pragma unroll
                for (int k = 0; k < KC; ++k) {
                    if (g0 + 32 * k >= nc) break;   // warp-uniform
                    const bool in = jv[k] >= 0 && within(rp, xi, pv[k], rc2);
                    const unsigned m = __ballot_sync(0xffffffffu, in);
                    const int pos = cnt + __popc(m & ((1u << lane) - 1u));
                    if (in && pos < maxnb) out[pos] = jv[k];
                    cnt += __popc(m);
                }
            }
        } else {
            cnt = scan_list(x, sy, rp, il, xi, cell_start, cell_cnt, cell_atoms, rc2, out, maxnb, lst[wib], bmap[wib], lane);
        }
    } else {
        cnt = scan_list(x, sy, rp, il, xi, cell_start, cell_cnt, cell_atoms, rc2, out, maxnb, lst[wib], bmap[wib], lane);
    }
    if (lane == 0) {
        nnb[b] = cnt;
        if (cnt > maxnb) {
            atomicOr(&err->flags, ERR_NBR_OVERFLOW);
            atomicMax(&err->max_nbr, cnt);
        }
    }
}

// Every bead of at most 32 atoms, no cells and no candidates: one warp per
// bead, lane = atom i; the bead's positions are shuffled to all lanes and
// each lane tests j = 0 .. N-1 in order with the same rule, so the lists are
// the full scan's (ascending, j = i skipped).
template <typename V4>
__global__ void __launch_bounds__(256) nbr_small_kernel(const V4* __restrict__ x, const BeadSys* __restrict__ bsys,
                                                        const Rep* __restrict__ reps, float rc2, int maxnb, int S,
                                                        int* __restrict__ nbr, int* __restrict__ nnb,
                                                        DevErr* __restrict__ err)
{
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= S) return;   // warp-uniform
    const unsigned lane = lane_id();
    const BeadSys sy = bsys[s];
    const Rep& rp = reps[sy.rep];
    const int n = sy.N;   // <= 32
    const bool me = (int)lane < n;
    const float3 xi = me ? pos_f32(x[sy.ba0 + lane]) : make_float3(0.0f, 0.0f, 0.0f);
    int* out = nbr + (size_t)(sy.ba0 + (me ? (int)lane : 0)) * maxnb;
    int cnt = 0;
    for (int j = 0; j < n; ++j) {
        const float3 xj = make_float3(__shfl_sync(0xffffffffu, xi.x, j), __shfl_sync(0xffffffffu, xi.y, j),
                                      __shfl_sync(0xffffffffu, xi.z, j));
        if (me && j != (int)lane && within(rp, xi, xj, rc2)) {
            if (cnt < maxnb) out[cnt] = j;
            ++cnt;
        }
    }
    if (me) {
        nnb[sy.ba0 + lane] = cnt;
        if (cnt > maxnb) {
            atomicOr(&err->flags, ERR_NBR_OVERFLOW);
            atomicMax(&err->max_nbr, cnt);
        }
    }
}

// cell lists and the Verlet check of every bead (before any list range)
void launch_neighbour_prep(const Dev& d, cudaStream_t st)
{
    if (d.precision == 0) {
        if (d.n_cell_bs)
            cell_build_kernel<Dbl4><<<d.n_cell_bs, 256, 2 * d.max_cells * sizeof(int), st>>>(
                (const Dbl4*)d.x, d.bsys, d.reps, d.cell_bs, d.cell_start, d.cell_cnt, d.cell_atoms);
        if (d.maxcand)
            skin_check_kernel<Dbl4><<<d.S, 1024, 0, st>>>((const Dbl4*)d.x, d.bsys, d.reps, d.xref, d.rebuild);
    } else {
        if (d.n_cell_bs)
            cell_build_kernel<float4><<<d.n_cell_bs, 256, 2 * d.max_cells * sizeof(int), st>>>(
                (const float4*)d.x, d.bsys, d.reps, d.cell_bs, d.cell_start, d.cell_cnt, d.cell_atoms);
        if (d.maxcand)
            skin_check_kernel<float4><<<d.S, 1024, 0, st>>>((const float4*)d.x, d.bsys, d.reps, d.xref, d.rebuild);
    }
}

// the lists of bead-atoms b0 .. b1-1 (after launch_neighbour_prep); ranges
// made of whole beads may run concurrently
void launch_neighbour_lists(const Dev& d, int b0, int b1, cudaStream_t st)
{
    if (b1 <= b0) return;
    const int threads = 256;
    const int blocks = (int)(((size_t)(b1 - b0) * 32 + threads - 1) / threads);
    const float rc2 = (float)(d.rc * d.rc);
    if (d.precision == 0)
        nbr_kernel<Dbl4><<<blocks, threads, 0, st>>>((const Dbl4*)d.x, d.ba_sys, d.bsys, d.reps, d.cell_start,
                                                     d.cell_cnt, d.cell_atoms, rc2, d.maxnb, b1, d.nbr, d.nnb, d.err,
                                                     d.cand, d.ncand, d.xref, d.rebuild, d.maxcand, b0, d.ba_info);
    else
        nbr_kernel<float4><<<blocks, threads, 0, st>>>((const float4*)d.x, d.ba_sys, d.bsys, d.reps, d.cell_start,
                                                       d.cell_cnt, d.cell_atoms, rc2, d.maxnb, b1, d.nbr, d.nnb,
                                                       d.err, d.cand, d.ncand, d.xref, d.rebuild, d.maxcand, b0, d.ba_info);
}

void launch_neighbours(const Dev& d, cudaStream_t st)
{
    if (d.max_N <= 32 && d.n_cell_bs == 0 && d.maxcand == 0) {
        // only small beads: a warp per bead instead of a warp per bead-atom
        const float rc2 = (float)(d.rc * d.rc);
        const int blocks = (d.S + 7) / 8;
        if (d.precision == 0)
            nbr_small_kernel<Dbl4><<<blocks, 256, 0, st>>>((const Dbl4*)d.x, d.bsys, d.reps, rc2, d.maxnb, d.S,
                                                           d.nbr, d.nnb, d.err);
        else
            nbr_small_kernel<float4><<<blocks, 256, 0, st>>>((const float4*)d.x, d.bsys, d.reps, rc2, d.maxnb, d.S,
                                                             d.nbr, d.nnb, d.err);
        return;
    }
    launch_neighbour_prep(d, st);
    launch_neighbour_lists(d, 0, d.B, st);
}

}  // namespace pimd
