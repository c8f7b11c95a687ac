// analysis.cu -- structural analysis of the bead configurations on the GPU:
// radial-distribution pair counts per element pair and the proton-transfer
// coordinate v = d(O_bond, H) - d(O_nearest other, H) (Sec. 3.2, Figs. 8, 9,
// 11). Both decide integers (histogram bins) from floating point, so both
// use the FP32 pair rule of the neighbour lists (positions rounded to FP32,
// minimum image in FP32, r2 = (dx dx + dy dy) + dz dz without contraction)
// and bin edges formed in FP64 and rounded to FP32.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "common.cuh"
#include "kernels.h"

namespace pimd {

__device__ __forceinline__ float3 pos32(const float4& v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 pos32(const Dbl4& v)
{
    return make_float3(__double2float_rn(v.x), __double2float_rn(v.y), __double2float_rn(v.z));
}

// squared minimum-image distance by the FP32 rule (no contraction)
__device__ __forceinline__ float rule_r2(const float3& a, const float3& b, const Rep& rp)
{
    float t[3] = {__fsub_rn(b.x, a.x), __fsub_rn(b.y, a.y), __fsub_rn(b.z, a.z)};
    if (rp.periodic) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float k = rintf(__fmul_rn(t[d], rp.invLf[d]));
            t[d] = __fsub_rn(t[d], __fmul_rn(rp.Lf[d], k));
        }
    }
    float r2 = __fmul_rn(t[0], t[0]);
    r2 = __fadd_rn(r2, __fmul_rn(t[1], t[1]));
    r2 = __fadd_rn(r2, __fmul_rn(t[2], t[2]));
    return r2;
}

// bin k with e[k] <= v < e[k+1], given e[0] <= v < e[n]; k0 is a guess
__device__ __forceinline__ int find_bin(const float* e, int n, float v, int k0)
{
    int k = min(max(k0, 0), n - 1);
    while (k > 0 && v < e[k]) --k;
    while (k < n - 1 && !(v < e[k + 1])) ++k;
    return k;
}

// ---------------------------------------------------------------------------
// RDF pair counts: grid (atom tiles, beads of the replica). Atom i pairs with
// j = i + d mod N for d = 1 .. (N-1)/2, and d = N/2 for i < N/2 when N is
// even: every unordered pair once, the same work per thread. Counts gather
// in a shared-memory histogram, then go to the caller's array.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(256) rdf_kernel(const Vec4<Real>* __restrict__ x, const Rep* __restrict__ reps,
                                                  const int* __restrict__ atype, int rep, int n_types, BinEdges edges,
                                                  int n_bins, float inv_dr, unsigned long long* __restrict__ counts)
{
    extern __shared__ unsigned int hist[];
    float* e = reinterpret_cast<float*>(hist + (size_t)n_types * (n_types + 1) / 2 * n_bins);
    const Rep& rp = reps[rep];
    const int N = rp.N;
    const int nh = n_types * (n_types + 1) / 2 * n_bins;
    for (int q = threadIdx.x; q < nh; q += blockDim.x) hist[q] = 0u;
    for (int q = threadIdx.x; q <= n_bins; q += blockDim.x) e[q] = edges.e[q];
    __syncthreads();
    const Vec4<Real>* xb = x + rp.ba0 + (size_t)blockIdx.y * N;
    const int* ty = atype + rp.atom0;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const float3 pi = pos32(xb[i]);
        const int ti = ty[i];
        const float emax = e[n_bins];
        const int D = (N - 1) / 2;
        const int dmax = ((N & 1) == 0 && i < N / 2) ? N / 2 : D;
        for (int d = 1; d <= dmax; ++d) {
            int j = i + d;
            j = j >= N ? j - N : j;
            const float r2 = rule_r2(pi, pos32(xb[j]), rp);
            if (r2 < emax) {
                const int k = find_bin(e, n_bins, r2, (int)(sqrtf(r2) * inv_dr));
                const int tj = ty[j];
                const int ta = min(ti, tj), tb = max(ti, tj);
                const int p = ta * (2 * n_types - ta - 1) / 2 + tb;
                atomicAdd(&hist[p * n_bins + k], 1u);
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nh; q += blockDim.x)
        if (hist[q]) atomicAdd(&counts[q], (unsigned long long)hist[q]);
}

size_t rdf_smem_bytes(int n_types, int n_bins)
{
    return sizeof(unsigned int) * (size_t)n_types * (n_types + 1) / 2 * n_bins + sizeof(float) * (n_bins + 1);
}

void launch_rdf(const Dev& d, int rep, int P, int N, const BinEdges& edges, int n_bins, float inv_dr,
                unsigned long long* counts, cudaStream_t st)
{
    const dim3 grid((N + 255) / 256, P);
    const size_t sm = rdf_smem_bytes(d.n_types, n_bins);
    if (d.precision == 0) {
        cudaFuncSetAttribute((const void*)rdf_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        rdf_kernel<double><<<grid, 256, sm, st>>>((const Dbl4*)d.x, d.reps, d.atype, rep, d.n_types, edges, n_bins,
                                                  inv_dr, counts);
    } else {
        cudaFuncSetAttribute((const void*)rdf_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        rdf_kernel<float><<<grid, 256, sm, st>>>((const float4*)d.x, d.reps, d.atype, rep, d.n_types, edges, n_bins,
                                                 inv_dr, counts);
    }
}

// ---------------------------------------------------------------------------
// proton-transfer coordinate: thread per (atom, bead); protons (bond >= 0)
// scan the acceptors (element type t_acc) for the nearest one other than
// their bonding atom. v goes to v_out [P][N] (NaN for other atoms) and into
// the histogram over [e_0, e_n).
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(256) pt_kernel(const Vec4<Real>* __restrict__ x, const Rep* __restrict__ reps,
                                                 const int* __restrict__ atype, int rep, const int* __restrict__ bond,
                                                 int t_acc, BinEdges edges, int n_bins, float inv_w,
                                                 float* __restrict__ v_out, unsigned long long* __restrict__ hist_out)
{
    extern __shared__ unsigned int hist[];
    float* e = reinterpret_cast<float*>(hist + n_bins);
    const Rep& rp = reps[rep];
    const int N = rp.N;
    for (int q = threadIdx.x; q < n_bins; q += blockDim.x) hist[q] = 0u;
    for (int q = threadIdx.x; q <= n_bins; q += blockDim.x) e[q] = edges.e[q];
    __syncthreads();
    const Vec4<Real>* xb = x + rp.ba0 + (size_t)blockIdx.y * N;
    const int* ty = atype + rp.atom0;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h < N) {
        float v = __int_as_float(0x7fc00000);   // NaN
        const int ob = bond[h];
        if (ob >= 0 && ob < N) {
            const float3 ph = pos32(xb[h]);
            const float db = sqrtf(rule_r2(ph, pos32(xb[ob]), rp));
            float dn = __int_as_float(0x7f800000);   // +inf
            for (int j = 0; j < N; ++j) {
                if (j == ob || j == h || ty[j] != t_acc) continue;
                dn = fminf(dn, sqrtf(rule_r2(ph, pos32(xb[j]), rp)));
            }
            if (dn < __int_as_float(0x7f800000)) {
                v = __fsub_rn(db, dn);
                if (hist_out && v >= e[0] && v < e[n_bins])
                    atomicAdd(&hist[find_bin(e, n_bins, v, (int)floorf(__fmul_rn(v - e[0], inv_w)))], 1u);
            }
        }
        if (v_out) v_out[(size_t)blockIdx.y * N + h] = v;
    }
    __syncthreads();
    if (hist_out)
        for (int q = threadIdx.x; q < n_bins; q += blockDim.x)
            if (hist[q]) atomicAdd(&hist_out[q], (unsigned long long)hist[q]);
}

void launch_pt(const Dev& d, int rep, int P, int N, const int* bond, int t_acc, const BinEdges& edges, int n_bins,
               float inv_w, float* v_out, unsigned long long* hist, cudaStream_t st)
{
    const dim3 grid((N + 255) / 256, P);
    const size_t sm = sizeof(unsigned int) * n_bins + sizeof(float) * (n_bins + 1);
    if (d.precision == 0) {
        cudaFuncSetAttribute((const void*)pt_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        pt_kernel<double><<<grid, 256, sm, st>>>((const Dbl4*)d.x, d.reps, d.atype, rep, bond, t_acc, edges, n_bins,
                                                 inv_w, v_out, hist);
    } else {
        cudaFuncSetAttribute((const void*)pt_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        pt_kernel<float><<<grid, 256, sm, st>>>((const float4*)d.x, d.reps, d.atype, rep, bond, t_acc, edges, n_bins,
                                                inv_w, v_out, hist);
    }
}

// g(r) per element pair from pair counts summed over n_configs bead
// configurations: counts / (n_configs pairs_p shell_k / volume), shell_k =
// 4/3 pi ((k+1)^3 - k^3) dr^3; thread per (pair, bin)
__global__ void rdf_gr_kernel(const unsigned long long* __restrict__ counts, RdfNorm nm, int n_pairs, int n_bins,
                              double* __restrict__ g)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_pairs * n_bins) return;
    const int p = q / n_bins, k = q - p * n_bins;
    const double r0 = k * nm.dr, r1 = (k + 1) * nm.dr;
    const double shell = 4.0 / 3.0 * CUDART_PI * (r1 * r1 * r1 - r0 * r0 * r0);
    const double ideal = nm.n_configs * nm.pairs[p] * shell / nm.volume;
    g[q] = ideal > 0.0 ? (double)counts[q] / ideal : 0.0;
}

void launch_rdf_gr(const unsigned long long* counts, const RdfNorm& nm, int n_pairs, int n_bins, double* g,
                   cudaStream_t st)
{
    const int n = n_pairs * n_bins;
    rdf_gr_kernel<<<(n + 127) / 128, 128, 0, st>>>(counts, nm, n_pairs, n_bins, g);
}

}  // namespace pimd
