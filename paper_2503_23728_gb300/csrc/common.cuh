// common.cuh -- device-side types shared by the PIMD kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pimd {

// physical constants (CODATA 2018)
constexpr double KB = 8.617333262e-5;          // eV / K
constexpr double HBAR = 0.6582119569;          // eV fs
constexpr double MVV2E = 103.64269652680505;   // eV per amu A^2 fs^-2

constexpr int NR = 32;    // radial channels
constexpr int NA = 32;    // angular channels
constexpr int ND = 64;    // descriptor length
constexpr int MAX_LAYERS = 4;
constexpr int TILE_ROWS = 128;     // network rows per tensor-core tile; element groups pad to it
#define PIMD_SORT_CAP 256          // neighbour-list sort buffer per warp (>= max_neighbours)

// device error word
enum : unsigned { ERR_NBR_OVERFLOW = 1u, ERR_NONFINITE = 2u, ERR_TIMEOUT = 4u, ERR_METAD_FULL = 8u };
struct DevErr {
    unsigned flags;
    int max_nbr;
    int pad[2];
};

// FP64 position / force record (x, y, z, w); w of positions carries the
// element type as an integer bit pattern
struct __align__(32) Dbl4 {
    double x, y, z, w;
};

template <typename Real> struct Vec4T;
template <> struct Vec4T<float> { using type = float4; };
template <> struct Vec4T<double> { using type = Dbl4; };
template <typename Real> using Vec4 = typename Vec4T<Real>::type;

// one ring polymer (replica)
struct Rep {
    int N, P;
    int ba0;          // bead-atom index of (bead 0, atom 0); state index base / 3
    int bs0;          // bead-system index of bead 0
    int atom0;        // index into per-atom arrays (mass, type)
    int cmat;         // offset of this P's normal-mode matrix C[P][P] (doubles)
    int mode0;        // offset of this replica's per-mode records
    int periodic;
    double L[3], invL[3];
    float Lf[3], invLf[3];   // FP32 box for the exact neighbour rule
    float Llo[3];            // L - Lf, for error-free FP32 pair vectors
    double kT_md;            // k_B T_P in amu A^2 / fs^2
    unsigned long long seed;
    int nc[3];               // cells per side (cell lists), 0 = scan all atoms
    int ncells;              // nc[0] nc[1] nc[2], 0 without cells
    int cell0;               // first cell of bead 0; bead k owns cell0 + k ncells ..
    float skin;              // Verlet skin of the candidate lists, A (0 = rebuild every step)
    float rcs2;              // (float)((r_c + skin)^2), candidate radius squared
    // noise counters index atoms as atom noise_atom0 + i of a system of
    // noise_N atoms (a shard of a larger ring polymer draws that system's
    // deviates); 0 and N for a whole system
    int noise_atom0, noise_N;
};

// one bead of one replica: N atoms starting at bead-atom index ba0
struct BeadSys {
    int ba0, N, rep, bead;
};

// per normal mode of a replica
struct Mode {
    double w, cw, sw, c1, c2;
    double mfac;   // mass of this ring coordinate / atom mass (normal modes 1; staging k/(k-1))
    double cs;     // sum over beads of the transform column: centroid = sum_k cs_k q_k / P
    double ft;     // total bead force = ft * (C^T f)_0 (normal modes sqrt(P), staging 1)
    // derived on the host so that the FP64 kernels divide and take roots
    // only in the random deviates: sw / w, w sw, sqrt(mfac), 1 / mfac
    double sw_w, wsw, smf, imf;
    // c1 - 1 and c1 + 1 in FP32 (from FP64), for the FP32 paths' heat terms
    float c1m1, c1p1;
};

constexpr double INV_MVV2E = 1.0 / MVV2E;

// pair schedule of the descriptor / adjoint kernels (chosen by the tuner)
struct Sched {
    int rmax;            // band length cap (<= 16)
    int band_min;        // neighbours needed for the band schedule (>= rmax + 32)
    int small_atomics;   // below band_min: 1 = flat walk with shared atomics,
                         // 0 = ordered pairs (each pair twice, no atomics)
    int ang;             // angular terms: 0 = pair sums, 1 = moment tensors (FP32 only)
    int adj_wide;        // BF16 moment adjoint: 0 = 12 warps per SM (166 registers),
                         // 1 = 16 warps per SM (128 registers)
};

// metadynamics: CV definition and bias parameters (by value to the kernels)
struct MetadParams {
    int cv;              // 0 none, 1 distance combination, 2 XRD intensity
    int n_terms;
    int ti[8], tj[8];
    double tc[8];
    double Q;            // XRD scattering vector magnitude, 1/A
    double f_type[8];    // XRD scattering factor per element type
    double h0, sigma, gamma;
    int stride, max_hills;
};

// symmetry-function parameters in the working precision
template <typename Real>
struct DescParams {
    Real rc, pi_over_rc, eta_R;
    Real r_mu[NR];
    Real eta_A[4];
    Real eta_R_l2, eta_A_l2[4];   // widths times log2(e) (FP32 exponentials use exp2)
    // evenly spaced radial centres (r_mu[c] = r_mu[0] + c r_delta): the BF16
    // path forms the Gaussians of a group of 8 centres by a product recurrence
    int r_even;
    Real r_delta;
    Real rec_k;    // 2^(-2 eta_R log2(e) r_delta^2), the ratio of successive ratios
};

// graph-field-network head: sizes, radial basis, scalars and the offsets
// (floats) of its FP32 parameters in the device weight buffer; matrices are
// stored transposed ([in][out]) for the tile products
constexpr int GFN_MAX_ITERS = 8;
struct GfnParams {
    int F, L;
    float rc, pi_over_rc, eta_R, s_F, b_f2;
    float r_mu[NR];
    unsigned o_emb, o_We, o_be, o_Wf1, o_bf1, o_wf2;
    unsigned o_it[GFN_MAX_ITERS][10];   // W_m^T, b_m, W_v1^T, b_v1, W_v2^T, b_v2, W_a1^T, b_a1, W_a2^T, b_a2
    // tensor-core path: byte offsets of the BF16 weight images ([out][in],
    // K-major core-matrix layout) in the image buffer
    unsigned t_We, t_Wf1;
    unsigned t_it[GFN_MAX_ITERS][5];    // W_m, W_a1, W_a2, W_v1, W_v2
};

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Reduce 32 per-lane values so that lane c ends with the sum over lanes of
// v[c] (31 shuffles): recursive halving of the channel set.
template <typename Real>
__device__ __forceinline__ Real transpose_reduce32(Real (&v)[32], unsigned lane)
{
#pragma unroll
    for (int o = 16, n = 32; o >= 1; o >>= 1, n >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < n / 2; ++q) {
            Real send = upper ? v[q] : v[q + n / 2];
            Real keep = upper ? v[q + n / 2] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

template <typename Real>
__device__ __forceinline__ Real warp_sum(Real v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace pimd
