// moment.cu -- angular symmetry functions and their adjoint through moment
// tensors, O(n) per atom in the neighbour count n (FP32 working precision).
//
// The G5 functions (Behler's angular functions without the r_jk term) have
// an exponent that splits over the two neighbours, exp(-eta (r_ij^2 + r_ik^2))
// fc(r_ij) fc(r_ik) = b_eta(j) b_eta(k) with b_eta(j) = exp(-eta r_ij^2)
// fc(r_ij), and for integer zeta the angle term is a polynomial of the
// cosine c_jk = u_j . u_k of the unit vectors. The multinomial theorem gives
//   (1 + lambda u_j . u_k)^zeta = sum_{a+b+c <= zeta} w_zeta(a,b,c) lambda^(a+b+c) m_abc(u_j) m_abc(u_k),
//   m_abc(u) = u_x^a u_y^b u_z^c,   w_zeta(a,b,c) = zeta! / ((zeta-a-b-c)! a! b! c!),
// so with the moments M_eta,abc = sum_j b_eta(j) m_abc(u_j) over all
// neighbours of the atom,
//   sum_{j,k} (1 + lambda c_jk)^zeta b_eta(j) b_eta(k) = sum_abc w_zeta lambda^(a+b+c) M_eta,abc^2.
// The sum over unordered pairs j < k is half of the sum over j != k, and the
// j = k terms have c = 1, so
//   G_(zeta,lambda,eta) = sum_abc 2^-zeta w_zeta(a,b,c) lambda^(a+b+c) M_eta,abc^2
//                         - [lambda = +1] sum_j b_eta(j)^2,
// the same value as the pair sum up to rounding. zeta <= 8 needs the 165
// monomials of degree <= 8; per neighbour that is 165 x 4 multiply-adds
// instead of ~n/2 pair evaluations.
//
// Adjoint: with D_nu = dE/dG_nu from the network,
//   Q_eta,abc = dE/dM_eta,abc = 2 M_eta,abc sum_zeta 2^-zeta w_zeta (D_(zeta,+,eta) + (-1)^(a+b+c) D_(zeta,-,eta)),
//   dE/db_eta(j) = sum_abc Q_eta,abc m_abc(u_j) - 2 b_eta(j) sum_zeta D_(zeta,+,eta),
//   dE/du_j      = sum_eta b_eta(j) sum_abc Q_eta,abc grad m_abc(u_j),
// and the chain rule through u = r / |r| and b_eta(r) gives dE_i/dr_ij.
#include <cuda_runtime.h>

#include "common.cuh"
#include "geom.cuh"
#include "kernels.h"

namespace pimd {

constexpr int MDEG = 8;           // largest zeta
constexpr int NMONO = 165;        // monomials u_x^a u_y^b u_z^c with a + b + c <= 8
constexpr int MSLOT = 6;          // per lane: monomial m = lane + 32 * slot
constexpr int MLAST = NMONO - 32 * (MSLOT - 1);   // lanes holding a monomial in the last slot

// Monomial order ("chain order"): c outer, b middle, a inner. Per slot and
// lane: cf[z] = 2^-zeta_z w_zeta_z(a,b,c) (0 where a+b+c > zeta_z or for the
// padding beyond m = 164), sg = (-1)^(a+b+c).
struct MonoTab {
    float cf[MSLOT][4][32];
    float sg[MSLOT][32];
};

constexpr double cfact(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

constexpr MonoTab make_mono_tab()
{
    MonoTab t{};
    const int zetas[4] = {1, 2, 4, 8};
    int m = 0;
    for (int c = 0; c <= MDEG; ++c)
        for (int b = 0; b <= MDEG - c; ++b)
            for (int a = 0; a <= MDEG - b - c; ++a, ++m) {
                const int s = a + b + c;
                for (int z = 0; z < 4; ++z) {
                    const int ze = zetas[z];
                    t.cf[m / 32][z][m % 32] =
                        s > ze ? 0.0f
                               : (float)(cfact(ze) / (cfact(ze - s) * cfact(a) * cfact(b) * cfact(c)) /
                                         (double)(1 << ze));
                }
                t.sg[m / 32][m % 32] = (s & 1) ? -1.0f : 1.0f;
            }
    return t;
}

__device__ const MonoTab g_mono = make_mono_tab();

// chain-order index of u_x^a u_y^b u_z^c: the monomials with z-degree below c
// (tetrahedral numbers), those with z-degree c and y-degree below b, then a.
// Closed form, so that it folds to a constant in the unrolled loops.
__host__ __device__ constexpr int tet(int n) { return n * (n + 1) * (n + 2) / 6; }
__host__ __device__ constexpr int mono_index(int a, int b, int c)
{
    return tet(MDEG + 1) - tet(MDEG + 1 - c) + b * (MDEG + 1 - c) - b * (b - 1) / 2 + a;
}
static_assert(mono_index(0, 0, MDEG) == NMONO - 1, "monomial count");
static_assert(mono_index(MDEG, 0, 0) == MDEG, "chain order");

// shared memory of the forward kernel, per warp: monomials of 32 neighbours
// (row stride 165 floats: odd, so the 32 rows written in one step hit distinct
// banks) and their weights b_eta
constexpr int FWD_WARP_FLOATS = 32 * NMONO + 32 * 4;
constexpr int FWD_WARPS = 1;
constexpr int MBLK = 4;   // neighbours per partial sum of the moments

// s += v by Kahan's compensated summation on both halves; nc carries minus
// the low-order part lost so far (the squared moments of the descriptors
// would otherwise double the relative rounding error of a plain FP32 sum)
__device__ __forceinline__ void kahan_add(float2& s, float2& nc, const float2 v)
{
    const float2 y = __fadd2_rn(v, nc);
    const float2 t = __fadd2_rn(s, y);
    nc = __fadd2_rn(__ffma2_rn(t, make_float2(-1.0f, -1.0f), s), y);
    s = t;
}

// Store the moments (lane slots) for the adjoint, and form G: per lane its
// monomials' share of sum_abc 2^-zeta w lambda^s M^2, packed over lambda =
// (+1, -1), then the 32-channel transposed reduction; the j = k terms
// (1 + lambda)^zeta 2^-zeta sum_j b^2 = sum_j b^2 leave the lambda = +1
// channels. Lane = channel nu = (zeta_index * 2 + lambda_index) * 4 + eta_index.
__device__ __forceinline__ void finish_moments(const float2 (&acc)[MSLOT][2], const float (&diag)[4], float Gr,
                                               unsigned lane, int b, float* __restrict__ G,
                                               float4* __restrict__ Mout)
{
    if (Mout != nullptr) {
        // the last slot's lanes past the 165th monomial hold nothing (the
        // adjoints read only the 165); streaming (evict-first) stores, so the
        // moments do not push the lists and positions the adjoint reads out
        // of L2
#pragma unroll
        for (int k = 0; k < MSLOT; ++k)
            if (k < MSLOT - 1 || lane < (unsigned)MLAST)
                __stcs(&Mout[((size_t)b * MSLOT + k) * 32 + lane],
                       make_float4(acc[k][0].x, acc[k][0].y, acc[k][1].x, acc[k][1].y));
    }

    // per lane: its monomials' share of sum_abc 2^-zeta w lambda^s M^2, packed
    // over lambda = (+1, -1); then the 32-channel transposed reduction
    float2 S[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) S[q] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < MSLOT; ++k) {
        const float sg = g_mono.sg[k][lane];
        const float mm[4] = {acc[k][0].x * acc[k][0].x, acc[k][0].y * acc[k][0].y, acc[k][1].x * acc[k][1].x,
                             acc[k][1].y * acc[k][1].y};
#pragma unroll
        for (int z = 0; z < 4; ++z) {
            const float cz = g_mono.cf[k][z][lane];
            const float2 c2 = make_float2(cz, cz * sg);
#pragma unroll
            for (int e = 0; e < 4; ++e) S[z * 4 + e] = __ffma2_rn(c2, make_float2(mm[e], mm[e]), S[z * 4 + e]);
        }
    }
    float ga[NA];
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            ga[(2 * z) * 4 + e] = S[z * 4 + e].x;
            ga[(2 * z + 1) * 4 + e] = S[z * 4 + e].y;
        }
    float Ga = transpose_reduce32(ga, lane);
    // lane = channel nu = (zeta_index * 2 + lambda_index) * 4 + eta_index:
    // remove the j = k terms, (1 + lambda)^zeta 2^-zeta sum_j b^2 = sum_j b^2 for lambda = +1
    const int e = (int)lane & 3;
    const float dge = e == 0 ? diag[0] : e == 1 ? diag[1] : e == 2 ? diag[2] : diag[3];
    if ((lane & 4u) == 0) Ga -= dge;
    G[(size_t)b * ND + lane] = Gr;
    G[(size_t)b * ND + NR + lane] = Ga;
}

// ---------------------------------------------------------------------------
// forward: warp per bead-atom. Neighbours are taken 32 at a time: each lane
// forms its neighbour's geometry, radial terms, weights b_eta and the 165
// monomials (into shared memory); then each lane accumulates the moments of
// its own monomials m = lane + 32 slot over the 32 neighbours (broadcast
// weights, conflict-free monomial loads). Moments go to Mout for the adjoint.
// ---------------------------------------------------------------------------
template <bool FAST>
__global__ void __launch_bounds__(32 * FWD_WARPS) desc_mom_fwd_kernel(
    const float4* __restrict__ x, const int* __restrict__ ba_sys, const BeadSys* __restrict__ bsys,
    const Rep* __restrict__ reps, const int* __restrict__ nbr, const int* __restrict__ nnb, int maxnb, int B,
    DescParams<float> dp, float* __restrict__ G, float4* __restrict__ Mout)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wib = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    float* MONO = reinterpret_cast<float*>(smem_raw) + (size_t)wib * FWD_WARP_FLOATS;
    float4* BW = reinterpret_cast<float4*>(MONO + 32 * NMONO);
    const int b = blockIdx.x * FWD_WARPS + wib;
    if (b >= B) return;
    const BeadSys sy = bsys[ba_sys[b]];
    const Rep& rp = reps[sy.rep];
    const int n = min(nnb[b], maxnb);
    const float4 xi = x[b];

    float gr[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) gr[c] = 0.0f;
    float dg[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // sum_j b_eta(j)^2 (this lane's neighbours)
    float2 acc[MSLOT][2];                      // moments (eta 0,1) and (eta 2,3)
    float2 cmp[MSLOT][2];                      // their compensation terms (FP32 path)
#pragma unroll
    for (int k = 0; k < MSLOT; ++k) acc[k][0] = acc[k][1] = cmp[k][0] = cmp[k][1] = make_float2(0.0f, 0.0f);

    for (int s0 = 0; s0 < n; s0 += 32) {
        const int s = s0 + (int)lane;
        if (s < n) {
            const int j = nbr[(size_t)b * maxnb + s];
            const float4 xj = x[sy.ba0 + j];
            float dx, dy, dz;
            pair_vec(rp, xi, xj, dx, dy, dz);
            const float r2 = dx * dx + dy * dy + dz * dz;
            const float r = sqrtf(r2);
            const float ir = 1.0f / r;
            float fc, dfc;
            cutoff(r, dp.rc, dp.pi_over_rc, fc, dfc);
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                const float t = r - dp.r_mu[c];
                gr[c] += gauss<FAST>(dp.eta_R, dp.eta_R_l2, t * t) * fc;
            }
            float bw[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                bw[e] = gauss<FAST>(dp.eta_A[e], dp.eta_A_l2[e], r2) * fc;
                dg[e] = fmaf(bw[e], bw[e], dg[e]);
            }
            BW[lane] = make_float4(bw[0], bw[1], bw[2], bw[3]);
            float px[MDEG + 1], py[MDEG + 1], pz[MDEG + 1];
            px[0] = py[0] = pz[0] = 1.0f;
            px[1] = dx * ir;
            py[1] = dy * ir;
            pz[1] = dz * ir;
#pragma unroll
            for (int a = 2; a <= MDEG; ++a) {
                px[a] = px[a - 1] * px[1];
                py[a] = py[a - 1] * py[1];
                pz[a] = pz[a - 1] * pz[1];
            }
            float* row = MONO + (size_t)lane * NMONO;
            int m = 0;
#pragma unroll
            for (int c = 0; c <= MDEG; ++c)
#pragma unroll
                for (int bb = 0; bb <= MDEG - c; ++bb) {
                    const float base = py[bb] * pz[c];
#pragma unroll
                    for (int a = 0; a <= MDEG - bb - c; ++a) row[m + a] = base * px[a];
                    m += MDEG - bb - c + 1;
                }
        }
        __syncwarp();
        const int cnt = min(32, n - s0);
        const float* col = MONO + lane;
        // blocks of MBLK neighbours are summed into a small partial first,
        // then added to the running moments (compensated on the FP32 path)
        for (int j0 = 0; j0 < cnt; j0 += MBLK) {
            float2 part[MSLOT][2];
#pragma unroll
            for (int k = 0; k < MSLOT; ++k) part[k][0] = part[k][1] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int q = 0; q < MBLK; ++q) {
                const int jj = j0 + q;
                if (jj < cnt) {
                    const float4 w4 = BW[jj];
                    const float2 w01 = make_float2(w4.x, w4.y), w23 = make_float2(w4.z, w4.w);
                    const float* rowj = col + (size_t)jj * NMONO;
#pragma unroll
                    for (int k = 0; k < MSLOT - 1; ++k) {
                        const float mv = rowj[32 * k];
                        const float2 m2 = make_float2(mv, mv);
                        part[k][0] = __ffma2_rn(w01, m2, part[k][0]);
                        part[k][1] = __ffma2_rn(w23, m2, part[k][1]);
                    }
                    if (lane < (unsigned)MLAST) {
                        const float mv = rowj[32 * (MSLOT - 1)];
                        const float2 m2 = make_float2(mv, mv);
                        part[MSLOT - 1][0] = __ffma2_rn(w01, m2, part[MSLOT - 1][0]);
                        part[MSLOT - 1][1] = __ffma2_rn(w23, m2, part[MSLOT - 1][1]);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < MSLOT; ++k)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (FAST)
                        acc[k][h] = __fadd2_rn(acc[k][h], part[k][h]);
                    else
                        kahan_add(acc[k][h], cmp[k][h], part[k][h]);
                }
        }
        __syncwarp();
    }
    if (!FAST) {
#pragma unroll
        for (int k = 0; k < MSLOT; ++k) {
            acc[k][0] = __fadd2_rn(acc[k][0], cmp[k][0]);
            acc[k][1] = __fadd2_rn(acc[k][1], cmp[k][1]);
        }
    }
    const float Gr = transpose_reduce32(gr, lane);
    float diag[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) diag[e] = warp_sum(dg[e]);
    finish_moments(acc, diag, Gr, lane, b, G, Mout);
}

// ---------------------------------------------------------------------------
// Reduced basis (BF16 network path). On the unit sphere x^2 = 1 - y^2 - z^2,
// so m_abc = m_(a-2)bc - m_(a-2)(b+2)c - m_(a-2)b(c+2): every polynomial of
// degree <= 8 in u equals one in the 81 monomials with a in {0, 1}, and
// the moments of all 165 monomials follow from those 81 by that recurrence
// (a = 2 .. 8 in turn). The adjoint needs only the tangential gradient of
// sum Q m(u), which the restricted polynomial shares, so it folds Q onto the
// 81 by the transposed recurrence. Differences cancel in the recurrence, so
// the exact FP32 path keeps the 165-monomial form.
// ---------------------------------------------------------------------------
constexpr int NRED = 81;

struct alignas(16) RedTab {
    short up[7][32][4];           // level a = 2..8: (m_abc, m_(a-2)bc, m_(a-2)(b+2)c, m_(a-2)b(c+2)), -1 idle
    // the same entries in 5 slots per lane over 4 rounds: levels a and a + 1
    // both read level a - 2 and a - 1 only, so they share a round (slots
    // 0-1: a = 2, 3; slot 2: a = 4, 5; slot 3: a = 6, 7; slot 4: a = 8)
    short upr[5][32][4];
    short down[7][2][32][4];      // level a = 8..2: target m_(a-2)BC and sources (a,B,C), (a,B-2,C), (a,B,C-2)
};

constexpr RedTab make_red_tab()
{
    RedTab t{};
    for (int L = 0; L < 7; ++L) {
        const int a = L + 2;
        int q = 0;
        for (int i = 0; i < 32; ++i)
            for (int k = 0; k < 4; ++k) t.up[L][i][k] = -1;
        for (int c = 0; c <= MDEG - a; ++c)
            for (int b = 0; b <= MDEG - a - c; ++b, ++q) {
                t.up[L][q][0] = (short)mono_index(a, b, c);
                t.up[L][q][1] = (short)mono_index(a - 2, b, c);
                t.up[L][q][2] = (short)mono_index(a - 2, b + 2, c);
                t.up[L][q][3] = (short)mono_index(a - 2, b, c + 2);
            }
    }
    {
        int q[4] = {0, 0, 0, 0};   // entries placed per round
        const int first_slot[4] = {0, 2, 3, 4};
        for (int sl = 0; sl < 5; ++sl)
            for (int i = 0; i < 32; ++i)
                for (int k = 0; k < 4; ++k) t.upr[sl][i][k] = -1;
        for (int L = 0; L < 7; ++L) {
            const int rd = L / 2;
            for (int i = 0; i < 32; ++i) {
                if (t.up[L][i][0] < 0) continue;
                const int pos = q[rd]++;
                const int sl = first_slot[rd] + pos / 32;
                for (int k = 0; k < 4; ++k) t.upr[sl][pos % 32][k] = t.up[L][i][k];
            }
        }
    }
    for (int L = 0; L < 7; ++L) {
        const int a = MDEG - L;   // 8 .. 2
        for (int h = 0; h < 2; ++h)
            for (int i = 0; i < 32; ++i)
                for (int k = 0; k < 4; ++k) t.down[L][h][i][k] = -1;
        int q = 0;
        for (int C = 0; C <= MDEG - a + 2; ++C)
            for (int B = 0; B <= MDEG - a + 2 - C; ++B, ++q) {
                short* e = t.down[L][q / 32][q % 32];
                e[0] = (short)mono_index(a - 2, B, C);
                if (a + B + C <= MDEG) e[1] = (short)mono_index(a, B, C);
                if (B >= 2) e[2] = (short)mono_index(a, B - 2, C);
                if (C >= 2) e[3] = (short)mono_index(a, B, C - 2);
            }
    }
    return t;
}

__device__ const RedTab g_red = make_red_tab();

// reduced-basis forward (BF16 path). The x-degree rides on the weights:
// M_eta,1bc = sum_j (b_eta(j) u_x,j) u_y,j^b u_z,j^c, so per neighbour the
// warp stores the 45 products u_y^b u_z^c (b + c <= 8; row stride 45, odd,
// so the 32 rows written in one step hit distinct banks) and the weights
// b_eta and b_eta u_x. Each half-warp then owns the 45 products (3 slots of
// 16 lanes) and half of the neighbours: half h reads row t + 16 h in step
// t, and 16 x 45 = 16 (mod 32) puts the two halves' loads in complementary
// banks, so each load and each weight broadcast serves two neighbours. The
// halves are added at the end, and the 165 moments are rebuilt in shared
// memory by the recurrence and finished as in the full forward.
constexpr int NBASE = 45;                    // u_y^b u_z^c, b + c <= MDEG
constexpr int BSLOT = 3;                     // base slots of 16 lanes per half-warp
constexpr int BLAST = NBASE - 16 * (BSLOT - 1);   // half-warp lanes holding a base in the last slot
constexpr int FWDR_WPAD = 34;                // weight float4 per warp and kind: neighbour j at j + 2 (j / 16)
constexpr int FWDR_WARP_FLOATS = 32 * NBASE + 2 * 4 * FWDR_WPAD;
constexpr int FWDR_WARPS = 1;   // one-warp CTAs: a finished warp frees its slot at once
static_assert(32 * NBASE >= 4 * NMONO, "moment table reuses the product rows");
static_assert((16 * NBASE) % 32 == 16, "half-warps read complementary banks");
static_assert((32 * NBASE) % 4 == 0, "weights 16-byte aligned");

// chain-order index of u_x^a u_y^b u_z^c for base slot q (c outer, b inner,
// the order of a row), a = 0, 1; -1 beyond the 45 or where a + b + c > MDEG
struct BaseTab {
    short full[2][16 * BSLOT];
};
constexpr BaseTab make_base_tab()
{
    BaseTab t{};
    for (int q = 0; q < 16 * BSLOT; ++q) t.full[0][q] = t.full[1][q] = -1;
    int q = 0;
    for (int c = 0; c <= MDEG; ++c)
        for (int b = 0; b <= MDEG - c; ++b, ++q) {
            t.full[0][q] = (short)mono_index(0, b, c);
            if (b + c < MDEG) t.full[1][q] = (short)mono_index(1, b, c);
        }
    return t;
}
__device__ const BaseTab g_base = make_base_tab();

template <bool FAST>
__global__ void __launch_bounds__(32 * FWDR_WARPS, 20) desc_mom_fwd_red_kernel(
    const float4* __restrict__ x, const int* __restrict__ ba_sys, const BeadSys* __restrict__ bsys,
    const Rep* __restrict__ reps, const int* __restrict__ nbr, const int* __restrict__ nnb, int maxnb, int B,
    DescParams<float> dp, float* __restrict__ G, float4* __restrict__ Mout, int b0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wib = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    float* ROW = reinterpret_cast<float*>(smem_raw) + (size_t)wib * FWDR_WARP_FLOATS;
    float4* W0 = reinterpret_cast<float4*>(ROW + 32 * NBASE);   // b_eta
    float4* W1 = W0 + FWDR_WPAD;                                 // b_eta u_x
    const int b = b0 + blockIdx.x * FWDR_WARPS + wib;   // bead-atoms b0 .. B-1
    if (b >= B) return;
    const BeadSys sy = bsys[ba_sys[b]];
    const Rep& rp = reps[sy.rep];
    const Box bx = box_of(rp);   // read once, not in every chunk
    const int n = min(nnb[b], maxnb);
    const float4 xi = x[b];
    const unsigned hl = lane & 15u;    // base lane within the half-warp
    const int hh = (int)(lane >> 4);   // half-warp

    // radial sums; evenly spaced centres on the fast path keep channels c and
    // c + 16 in one register pair (gr2[8 qp + k] = channels 8 qp + k, 8 qp + k + 16)
    float2 gr2[NR / 2];
#pragma unroll
    for (int c = 0; c < NR / 2; ++c) gr2[c] = make_float2(0.0f, 0.0f);
    const bool packed = FAST && dp.r_even;
    float dg[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    // acc[k][0..1]: moments of (0, b, c), widths (0, 1) and (2, 3); acc[k][2..3]: (1, b, c)
    float2 acc[BSLOT][4];
#pragma unroll
    for (int k = 0; k < BSLOT; ++k)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[k][v] = make_float2(0.0f, 0.0f);

    // the next chunk's neighbour position is loaded while this chunk computes
    float4 xnext = ((int)lane < n) ? x[sy.ba0 + nbr[(size_t)b * maxnb + lane]] : xi;
    for (int s0 = 0; s0 < n; s0 += 32) {
        const int s = s0 + (int)lane;
        const float4 xj = xnext;
        if (s + 32 < n) xnext = x[sy.ba0 + nbr[(size_t)b * maxnb + s + 32]];
        // the chunk's cnt neighbours split between the halves: lane l < hc
        // (hc = ceil(cnt / 2)) writes row l, lane l >= hc row 16 + l - hc; for
        // odd cnt, lane cnt writes the zero-weight row that half 1 reads last
        const int cnt = min(32, n - s0);
        const int hc = (cnt + 1) >> 1;
        const int rl = (int)lane < hc ? (int)lane : 16 + (int)lane - hc;
        const bool wr = (int)lane <= cnt;
        float bw[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        float ux = 0.0f, uy = 0.0f, uz = 0.0f;
        if (s < n) {
            float dx, dy, dz, r, r2, ir, fc, dfc;
            if (FAST) {
                geo_fast(bx, xi, xj, dp.rc, dp.pi_over_rc, dx, dy, dz, r, ir, fc, dfc);
                r2 = r * r;
            } else {
                pair_vec(rp, xi, xj, dx, dy, dz);
                r2 = dx * dx + dy * dy + dz * dz;
                r = sqrtf(r2);
                ir = 1.0f / r;
                cutoff(r, dp.rc, dp.pi_over_rc, fc, dfc);
            }
            if (packed) {
                // product recurrence of radial_gauss32 on two groups at once
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
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                bw[e] = gauss<FAST>(dp.eta_A[e], dp.eta_A_l2[e], r2) * fc;
                dg[e] = fmaf(bw[e], bw[e], dg[e]);
            }
            ux = dx * ir;
            uy = dy * ir;
            uz = dz * ir;
        }
        if (wr) {
            const int pw = rl + 2 * (rl >> 4);
            W0[pw] = make_float4(bw[0], bw[1], bw[2], bw[3]);
            W1[pw] = make_float4(bw[0] * ux, bw[1] * ux, bw[2] * ux, bw[3] * ux);
            float py[MDEG + 1], pz[MDEG + 1];
            py[0] = pz[0] = 1.0f;
            py[1] = uy;
            pz[1] = uz;
#pragma unroll
            for (int a = 2; a <= MDEG; ++a) {
                py[a] = py[a - 1] * py[1];
                pz[a] = pz[a - 1] * pz[1];
            }
            float* row = ROW + (size_t)rl * NBASE;
            int q = 0;
#pragma unroll
            for (int c = 0; c <= MDEG; ++c)
#pragma unroll
                for (int bb = 0; bb <= MDEG - c; ++bb) row[q++] = py[bb] * pz[c];
        }
        __syncwarp();
        // step t: half hh takes row t + 16 hh
        const int steps = hc;
        const float* col = ROW + (size_t)(16 * hh) * NBASE + hl;
        const float4* w0p = W0 + 18 * hh;
        const float4* w1p = W1 + 18 * hh;
        int t = 0;
        for (; t + 4 <= steps; t += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 a4 = w0p[t + u], c4 = w1p[t + u];
                const float2 w01 = make_float2(a4.x, a4.y), w23 = make_float2(a4.z, a4.w);
                const float2 x01 = make_float2(c4.x, c4.y), x23 = make_float2(c4.z, c4.w);
                const float* rowj = col + (size_t)(t + u) * NBASE;
#pragma unroll
                for (int k = 0; k < BSLOT; ++k) {
                    if (k < BSLOT - 1 || hl < (unsigned)BLAST) {
                        const float mv = rowj[16 * k];
                        const float2 m2 = make_float2(mv, mv);
                        acc[k][0] = __ffma2_rn(w01, m2, acc[k][0]);
                        acc[k][1] = __ffma2_rn(w23, m2, acc[k][1]);
                        acc[k][2] = __ffma2_rn(x01, m2, acc[k][2]);
                        acc[k][3] = __ffma2_rn(x23, m2, acc[k][3]);
                    }
                }
            }
        }
        for (; t < steps; ++t) {
            const float4 a4 = w0p[t], c4 = w1p[t];
            const float2 w01 = make_float2(a4.x, a4.y), w23 = make_float2(a4.z, a4.w);
            const float2 x01 = make_float2(c4.x, c4.y), x23 = make_float2(c4.z, c4.w);
            const float* rowj = col + (size_t)t * NBASE;
#pragma unroll
            for (int k = 0; k < BSLOT; ++k) {
                if (k < BSLOT - 1 || hl < (unsigned)BLAST) {
                    const float mv = rowj[16 * k];
                    const float2 m2 = make_float2(mv, mv);
                    acc[k][0] = __ffma2_rn(w01, m2, acc[k][0]);
                    acc[k][1] = __ffma2_rn(w23, m2, acc[k][1]);
                    acc[k][2] = __ffma2_rn(x01, m2, acc[k][2]);
                    acc[k][3] = __ffma2_rn(x23, m2, acc[k][3]);
                }
            }
        }
        __syncwarp();
    }
    float gr[NR];
#pragma unroll
    for (int qp = 0; qp < 2; ++qp)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            gr[8 * qp + k] = gr2[8 * qp + k].x;
            gr[8 * qp + k + 16] = gr2[8 * qp + k].y;
        }
    const float Gr = transpose_reduce32(gr, lane);
    float diag[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) diag[e] = warp_sum(dg[e]);

    // the recurrence's table entries, loaded before the sums they wait for
    short4 ue[5];
#pragma unroll
    for (int sl = 0; sl < 5; ++sl) ue[sl] = *reinterpret_cast<const short4*>(g_red.upr[sl][lane]);
    // the two halves' sums; then half 0 stores the moments of (0, b, c) and
    // half 1 those of (1, b, c) (rows of the last chunk are no longer needed)
    float4* T = reinterpret_cast<float4*>(ROW);
#pragma unroll
    for (int k = 0; k < BSLOT; ++k) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            acc[k][v].x += __shfl_xor_sync(0xffffffffu, acc[k][v].x, 16);
            acc[k][v].y += __shfl_xor_sync(0xffffffffu, acc[k][v].y, 16);
        }
        const int mf = g_base.full[hh][16 * k + hl];
        const float2 lo = hh ? acc[k][2] : acc[k][0];
        const float2 hi = hh ? acc[k][3] : acc[k][1];
        if (mf >= 0) T[mf] = make_float4(lo.x, lo.y, hi.x, hi.y);
    }
    __syncwarp();
#pragma unroll
    for (int sl = 0; sl < 5; ++sl) {
        const short4 e = ue[sl];
        if (e.x >= 0) {
            const float4 a0 = T[e.y], a1 = T[e.z], a2 = T[e.w];
            T[e.x] = make_float4(a0.x - a1.x - a2.x, a0.y - a1.y - a2.y, a0.z - a1.z - a2.z, a0.w - a1.w - a2.w);
        }
        if (sl != 0) __syncwarp();   // slots 0 and 1 form one round
    }
    float2 full[MSLOT][2];
#pragma unroll
    for (int k = 0; k < MSLOT; ++k) {
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (k < MSLOT - 1 || lane < (unsigned)MLAST) v = T[lane + 32 * k];
        full[k][0] = make_float2(v.x, v.y);
        full[k][1] = make_float2(v.z, v.w);
    }
    finish_moments(full, diag, Gr, lane, b, G, Mout);
}

// ---------------------------------------------------------------------------
// adjoint: warp per bead-atom. The warp forms Q = dE/dM (lane-owned
// monomials, into shared memory), then each lane takes one neighbour and
// evaluates the polynomials sum_abc Q_eta,abc m_abc(u) and their gradient by
// nested Horner recurrences (x innermost, then y, then z) with broadcast
// loads of Q.
// ---------------------------------------------------------------------------
constexpr int ADJ_WARP_BYTES = NMONO * 16 + ND * 4 + NR * 4;   // Q, dE/dG, radial dE/dG x r_mu
constexpr int ADJ_WARPS = 1;

template <bool FAST>
__global__ void __launch_bounds__(32 * ADJ_WARPS, FAST ? 20 : 12) desc_mom_adj_kernel(
    const float4* __restrict__ x, const int* __restrict__ ba_sys, const BeadSys* __restrict__ bsys,
    const Rep* __restrict__ reps, const int* __restrict__ nbr, const int* __restrict__ nnb, int maxnb, int B,
    DescParams<float> dp, const float4* __restrict__ Min, const float* __restrict__ dEdG,
    float4* __restrict__ f, float* __restrict__ wbuf, int det, float4* __restrict__ vbuf)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wib = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    float4* Q = reinterpret_cast<float4*>(smem_raw + (size_t)wib * ADJ_WARP_BYTES);
    float* gs = reinterpret_cast<float*>(Q + NMONO);
    const int b = blockIdx.x * ADJ_WARPS + wib;
    if (b >= B) return;
    const BeadSys sy = bsys[ba_sys[b]];
    const Rep& rp = reps[sy.rep];
    const int n = min(nnb[b], maxnb);
    const float4 xi = x[b];
    gs[lane] = dEdG[(size_t)b * ND + lane];
    gs[NR + lane] = dEdG[(size_t)b * ND + NR + lane];
    gs[ND + lane] = gs[lane] * dp.r_mu[lane];
    __syncwarp();

    // D(zeta,+,eta) +- D(zeta,-,eta) and sum_zeta D(zeta,+,eta)
    float Dp[16], Dm[16], dsum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float dplus = gs[NR + (2 * z) * 4 + e], dminus = gs[NR + (2 * z + 1) * 4 + e];
            Dp[z * 4 + e] = dplus + dminus;
            Dm[z * 4 + e] = dplus - dminus;
            dsum[e] += dplus;
        }
#pragma unroll
    for (int k = 0; k < MSLOT; ++k) {
        const int m = (int)lane + 32 * k;
        if (k < MSLOT - 1 || lane < (unsigned)MLAST) {
            const float4 M = Min[((size_t)b * MSLOT + k) * 32 + lane];
            const bool odd = g_mono.sg[k][lane] < 0.0f;
            float F[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int z = 0; z < 4; ++z) {
                const float cz = g_mono.cf[k][z][lane];
#pragma unroll
                for (int e = 0; e < 4; ++e) F[e] = fmaf(cz, odd ? Dm[z * 4 + e] : Dp[z * 4 + e], F[e]);
            }
            Q[m] = make_float4(2.0f * M.x * F[0], 2.0f * M.y * F[1], 2.0f * M.z * F[2], 2.0f * M.w * F[3]);
        }
    }
    __syncwarp();
    if (FAST) {
        // reduced basis: fold Q onto the monomials with a in {0, 1} by the
        // transposed recurrence, a = 8 .. 2 (sources at level a, targets at a - 2)
#pragma unroll 1
        for (int L = 0; L < 7; ++L) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const short* e = g_red.down[L][h][lane];
                if (e[0] >= 0) {
                    float4 t = Q[e[0]];
                    if (e[1] >= 0) {
                        const float4 u = Q[e[1]];
                        t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
                    }
                    if (e[2] >= 0) {
                        const float4 u = Q[e[2]];
                        t.x -= u.x; t.y -= u.y; t.z -= u.z; t.w -= u.w;
                    }
                    if (e[3] >= 0) {
                        const float4 u = Q[e[3]];
                        t.x -= u.x; t.y -= u.y; t.z -= u.z; t.w -= u.w;
                    }
                    Q[e[0]] = t;
                }
            }
            __syncwarp();
        }
    }

    float fi[3] = {0.0f, 0.0f, 0.0f};
    float wl[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) wl[q] = 0.0f;
    for (int s = (int)lane; s < n; s += 32) {
        const int j = nbr[(size_t)b * maxnb + s];
        const float4 xj = x[sy.ba0 + j];
        float dx, dy, dz;
        pair_vec(rp, xi, xj, dx, dy, dz);
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float r = sqrtf(r2);
        const float ir = 1.0f / r;
        float fc, dfc;
        cutoff(r, dp.rc, dp.pi_over_rc, fc, dfc);
        float dEdr = 0.0f;
        if (FAST && dp.r_even) {
            // sum_c gs_c g_c (-2 eta_R (r - r_mu_c) fc + dfc)
            //   = (-2 eta_R r fc + dfc) sum_c gs_c g_c + 2 eta_R fc sum_c gs_c r_mu_c g_c
            float g[NR];
            radial_gauss32(dp, r, g);
            float s1 = 0.0f, s2 = 0.0f;
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                s1 = fmaf(gs[c], g[c], s1);
                s2 = fmaf(gs[ND + c], g[c], s2);
            }
            dEdr = s1 * (-2.0f * dp.eta_R * r * fc + dfc) + 2.0f * dp.eta_R * fc * s2;
        } else {
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                const float t = r - dp.r_mu[c];
                const float ex = gauss<FAST>(dp.eta_R, dp.eta_R_l2, t * t);
                dEdr += gs[c] * ex * (-2.0f * dp.eta_R * t * fc + dfc);
            }
        }
        float bw[4], dbw[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float ex = gauss<FAST>(dp.eta_A[e], dp.eta_A_l2[e], r2);
            bw[e] = ex * fc;
            dbw[e] = ex * (-2.0f * dp.eta_A[e] * r * fc + dfc);
        }
        const float ux = dx * ir, uy = dy * ir, uz = dz * ir;
        const float2 X2 = make_float2(ux, ux), Y2 = make_float2(uy, uy), Z2 = make_float2(uz, uz);
        // P_eta(u) = sum_abc Q_eta,abc u_x^a u_y^b u_z^c and its gradient by
        // nested Horner recurrences (a, then b, then c, each descending);
        // float2 pairs hold (eta 0, eta 1) and (eta 2, eta 3)
        float2 V0, V1, VX0, VX1, VY0, VY1, VZ0, VZ1;
#pragma unroll
        for (int c = MDEG; c >= 0; --c) {
            float2 S0, S1, SX0, SX1, SY0, SY1;
#pragma unroll
            for (int bb = MDEG - c; bb >= 0; --bb) {
                // x-degree of the chain: up to 8, or 1 in the reduced basis
                const int A = (FAST && MDEG - bb - c > 1) ? 1 : MDEG - bb - c;
                const int m0 = mono_index(0, bb, c);
                float4 q = Q[m0 + A];
                float2 R0 = make_float2(q.x, q.y), R1 = make_float2(q.z, q.w);
                float2 RX0 = make_float2(0.0f, 0.0f), RX1 = RX0;
#pragma unroll
                for (int a = A - 1; a >= 0; --a) {
                    q = Q[m0 + a];
                    if (a == A - 1) {
                        RX0 = R0;
                        RX1 = R1;
                    } else {
                        RX0 = __ffma2_rn(RX0, X2, R0);
                        RX1 = __ffma2_rn(RX1, X2, R1);
                    }
                    R0 = __ffma2_rn(R0, X2, make_float2(q.x, q.y));
                    R1 = __ffma2_rn(R1, X2, make_float2(q.z, q.w));
                }
                if (bb == MDEG - c) {
                    S0 = R0; S1 = R1; SX0 = RX0; SX1 = RX1;
                    SY0 = SY1 = make_float2(0.0f, 0.0f);
                } else {
                    if (bb == MDEG - c - 1) {
                        SY0 = S0;
                        SY1 = S1;
                    } else {
                        SY0 = __ffma2_rn(SY0, Y2, S0);
                        SY1 = __ffma2_rn(SY1, Y2, S1);
                    }
                    S0 = __ffma2_rn(S0, Y2, R0);
                    S1 = __ffma2_rn(S1, Y2, R1);
                    SX0 = __ffma2_rn(SX0, Y2, RX0);
                    SX1 = __ffma2_rn(SX1, Y2, RX1);
                }
            }
            if (c == MDEG) {
                V0 = S0; V1 = S1; VX0 = SX0; VX1 = SX1; VY0 = SY0; VY1 = SY1;
                VZ0 = VZ1 = make_float2(0.0f, 0.0f);
            } else {
                if (c == MDEG - 1) {
                    VZ0 = V0;
                    VZ1 = V1;
                } else {
                    VZ0 = __ffma2_rn(VZ0, Z2, V0);
                    VZ1 = __ffma2_rn(VZ1, Z2, V1);
                }
                V0 = __ffma2_rn(V0, Z2, S0);
                V1 = __ffma2_rn(V1, Z2, S1);
                VX0 = __ffma2_rn(VX0, Z2, SX0);
                VX1 = __ffma2_rn(VX1, Z2, SX1);
                VY0 = __ffma2_rn(VY0, Z2, SY0);
                VY1 = __ffma2_rn(VY1, Z2, SY1);
            }
        }
        const float V[4] = {V0.x, V0.y, V1.x, V1.y};
#pragma unroll
        for (int e = 0; e < 4; ++e) dEdr = fmaf(V[e] - 2.0f * bw[e] * dsum[e], dbw[e], dEdr);
        const float gx = bw[0] * VX0.x + bw[1] * VX0.y + bw[2] * VX1.x + bw[3] * VX1.y;
        const float gy = bw[0] * VY0.x + bw[1] * VY0.y + bw[2] * VY1.x + bw[3] * VY1.y;
        const float gz = bw[0] * VZ0.x + bw[1] * VZ0.y + bw[2] * VZ1.x + bw[3] * VZ1.y;
        const float gu = gx * ux + gy * uy + gz * uz;
        const float v[3] = {dEdr * ux + (gx - gu * ux) * ir, dEdr * uy + (gy - gu * uy) * ir,
                            dEdr * uz + (gz - gu * uz) * ir};
        if (det)
            vbuf[(size_t)b * maxnb + s] = make_float4(v[0], v[1], v[2], 0.0f);
        else
            atomicAdd(&f[sy.ba0 + j], make_float4(-v[0], -v[1], -v[2], 0.0f));
        const float d3[3] = {dx, dy, dz};
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
            f[b] = make_float4(fi[0], fi[1], fi[2], 0.0f);   // gathered later
        else
            atomicAdd(&f[b], make_float4(fi[0], fi[1], fi[2], 0.0f));
    }
    if (lane < 9) {
        float mine = wl[0];
#pragma unroll
        for (int q = 1; q < 9; ++q)
            if ((int)lane == q) mine = wl[q];
        wbuf[(size_t)b * 9 + lane] = mine;
    }
}

// ---------------------------------------------------------------------------
// BF16-path adjoint (reduced basis, evenly spaced radial centres). The same
// sums as desc_mom_adj_kernel<true>, arranged for the GB300 pipes:
//  * per-atom set-up in one level: with s = a + b + c the coefficient
//    2^-zeta w_zeta(a,b,c) = [zeta! / (zeta - s)!] 2^-zeta / (a! b! c!), so
//    Q_abc = M_abc Phi(s) 2 / (a! b! c!) with Phi_eta(s) = sum_zeta
//    [zeta! / (zeta - s)!] 2^-zeta D^(+/-)_(zeta,eta) (9 values per eta); the
//    fold onto the 81 monomials with a in {0, 1} (x^2 = 1 - y^2 - z^2 on
//    the sphere) is the sparse matrix R^T, x^(2k) -> (1 - y^2 - z^2)^k
//    expanded by the trinomial theorem (483 terms), applied in one pass from
//    a table that spreads the terms evenly over the lanes (at most 16 each);
//  * while more than 32 neighbours remain each lane evaluates two of them in
//    lockstep, so that every shared-memory broadcast of a coefficient float4
//    of the compact 81-entry table feeds the Horner steps of both; the next
//    round's neighbour positions are loaded while the current round computes;
//  * the monomial index functions are closed forms: left as loops, the
//    compiler does not always fold them inside the unrolled Horner steps
//    and computes them at run time (3x the instructions);
//  * the radial sums sum_c gs_c g_c and sum_c gs_c r_mu_c g_c run the
//    product recurrence of radial_gauss32 on two groups of 8 centres at
//    once (packed FP32x2), with (gs, gs r_mu) of both groups in one float4;
//  * geometry and cutoff from geo_fast; the 12 per-atom sums (force on the
//    centre, virial) in one transposed warp reduction.
// ---------------------------------------------------------------------------
constexpr int ADJF_WARPS = 1;   // one-warp CTAs: a finished warp frees its slot at once
constexpr int ADJF_RG = 16;   // float4 per warp: (gs_a, gs_b, gs_a r_a, gs_b r_b) for centre pairs (c, c + 16)
constexpr int FOLD_MAX = 16;  // fold terms per lane

// compact index of the reduced monomial u_x^a u_y^b u_z^c (a <= 1), chain
// order: z-level cc holds 2 (MDEG - cc) + 1 of them, so the levels below c hold
// c (2 MDEG + 2 - c); within the level two per y-degree (closed form, folds to
// a constant in the unrolled loops)
__host__ __device__ constexpr int red_index(int a, int b, int c)
{
    return c * (2 * MDEG + 2 - c) + 2 * b + a;
}
static_assert(red_index(0, 0, MDEG) == NRED - 1, "reduced monomial count");

struct FoldTab {
    // per lane and term: bits 0-7 source monomial (chain order), 8-15 compact
    // target, bit 16 last term of its target, bits 24-31 signed coefficient
    unsigned ent[FOLD_MAX][32];
    // per slot and lane: 2 / (a! b! c!) and the degree s of monomial lane + 32 slot
    float w[MSLOT][32];
    int deg[MSLOT][32];
    // Phi coefficients [zeta! / (zeta - s)!] 2^-zeta (0 for s > zeta), [zeta index][s]
    float cphi[4][MDEG + 1];
};

constexpr FoldTab make_fold_tab()
{
    FoldTab t{};
    // terms of each target: full (a, b, c) -> (a % 2, b + 2i, c + 2j), k = a / 2,
    // coefficient (-1)^(i+j) k! / (i! j! (k-i-j)!)
    int tgt_cnt[NRED] = {};
    int src[NRED][16] = {};
    int cof[NRED][16] = {};
    for (int c = 0; c <= MDEG; ++c)
        for (int b = 0; b <= MDEG - c; ++b)
            for (int a = 0; a <= MDEG - b - c; ++a) {
                const int k = a / 2;
                for (int i = 0; i <= k; ++i)
                    for (int j = 0; j <= k - i; ++j) {
                        const int tg = red_index(a % 2, b + 2 * i, c + 2 * j);
                        const int co = (((i + j) & 1) ? -1 : 1) *
                                       (int)(cfact(k) / (cfact(i) * cfact(j) * cfact(k - i - j)));
                        src[tg][tgt_cnt[tg]] = mono_index(a, b, c);
                        cof[tg][tgt_cnt[tg]] = co;
                        ++tgt_cnt[tg];
                    }
            }
    // longest-processing-time assignment of the targets to the lanes
    int load[32] = {};
    bool done[NRED] = {};
    int lane_terms[32][FOLD_MAX][3] = {};   // (source, target, coefficient)
    for (int q = 0; q < NRED; ++q) {
        int best = -1;
        for (int tg = 0; tg < NRED; ++tg)
            if (!done[tg] && (best < 0 || tgt_cnt[tg] > tgt_cnt[best])) best = tg;
        done[best] = true;
        int ln = 0;
        for (int l = 1; l < 32; ++l)
            if (load[l] < load[ln]) ln = l;
        for (int e = 0; e < tgt_cnt[best]; ++e) {
            lane_terms[ln][load[ln] + e][0] = src[best][e];
            lane_terms[ln][load[ln] + e][1] = best;
            lane_terms[ln][load[ln] + e][2] = cof[best][e];
        }
        load[ln] += tgt_cnt[best];
    }
    for (int l = 0; l < 32; ++l)
        for (int e = 0; e < FOLD_MAX; ++e) {
            if (e < load[l]) {
                const bool last = e + 1 == load[l] || lane_terms[l][e + 1][1] != lane_terms[l][e][1];
                t.ent[e][l] = (unsigned)lane_terms[l][e][0] | ((unsigned)lane_terms[l][e][1] << 8) |
                              (last ? 0x10000u : 0u) | ((unsigned)(lane_terms[l][e][2] & 0xff) << 24);
            } else {
                t.ent[e][l] = 0u;   // coefficient 0, no store
            }
        }
    int m = 0;
    for (int c = 0; c <= MDEG; ++c)
        for (int b = 0; b <= MDEG - c; ++b)
            for (int a = 0; a <= MDEG - b - c; ++a, ++m) {
                t.w[m / 32][m % 32] = (float)(2.0 / (cfact(a) * cfact(b) * cfact(c)));
                t.deg[m / 32][m % 32] = a + b + c;
            }
    const int zetas[4] = {1, 2, 4, 8};
    for (int z = 0; z < 4; ++z)
        for (int sd = 0; sd <= MDEG; ++sd)
            t.cphi[z][sd] = sd > zetas[z] ? 0.0f
                                          : (float)(cfact(zetas[z]) / cfact(zetas[z] - sd) / (double)(1 << zetas[z]));
    return t;
}

__device__ const FoldTab g_fold = make_fold_tab();

template <int NB>
__device__ __forceinline__ void adj_fast_eval(const Box& bx, const DescParams<float>& dp, const float4& xi,
                                              const float4 (&xj)[NB], const bool (&valid)[NB],
                                              const float4* __restrict__ Q, const float4* __restrict__ RG,
                                              const float (&dsum)[4], float (&v)[NB][3], float (&d)[NB][3])
{
    float r[NB], ir[NB], fc[NB], dfc[NB];
    float2 X2[NB], Y2[NB], Z2[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        float dx, dy, dz;
        geo_fast(bx, xi, xj[t], dp.rc, dp.pi_over_rc, dx, dy, dz, r[t], ir[t], fc[t], dfc[t]);
        if (!valid[t]) {   // an idle slot: a unit vector with zero weights gives v = 0
            dx = 1.0f;
            dy = dz = 0.0f;
            r[t] = ir[t] = 1.0f;
            fc[t] = dfc[t] = 0.0f;
        }
        X2[t] = make_float2(dx * ir[t], dx * ir[t]);
        Y2[t] = make_float2(dy * ir[t], dy * ir[t]);
        Z2[t] = make_float2(dz * ir[t], dz * ir[t]);
    }

    // radial sums; centres c and c + 16 share a register pair
    float2 a1[NB], a2[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t) a1[t] = a2[t] = make_float2(0.0f, 0.0f);
    const float2 rho = make_float2(dp.rec_k, dp.rec_k);
    const float dd = dp.r_delta * dp.r_delta;
#pragma unroll
    for (int qp = 0; qp < 2; ++qp) {
        float2 e2[NB], R2[NB];
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            const float ta = r[t] - dp.r_mu[8 * qp], tb = r[t] - dp.r_mu[8 * qp + 16];
            e2[t] = make_float2(exp2f(-dp.eta_R_l2 * ta * ta), exp2f(-dp.eta_R_l2 * tb * tb));
            R2[t] = make_float2(exp2f(dp.eta_R_l2 * fmaf(2.0f * ta, dp.r_delta, -dd)),
                                exp2f(dp.eta_R_l2 * fmaf(2.0f * tb, dp.r_delta, -dd)));
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4 g = RG[qp * 8 + k];
#pragma unroll
            for (int t = 0; t < NB; ++t) {
                a1[t] = __ffma2_rn(e2[t], make_float2(g.x, g.y), a1[t]);
                a2[t] = __ffma2_rn(e2[t], make_float2(g.z, g.w), a2[t]);
                if (k < 7) {
                    e2[t] = __fmul2_rn(e2[t], R2[t]);
                    R2[t] = __fmul2_rn(R2[t], rho);
                }
            }
        }
    }
    float dEdr[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t)
        dEdr[t] = (a1[t].x + a1[t].y) * fmaf(-2.0f * dp.eta_R * r[t], fc[t], dfc[t]) +
                  2.0f * dp.eta_R * fc[t] * (a2[t].x + a2[t].y);

    // P_eta(u) = sum Q_eta,abc u_x^a u_y^b u_z^c (a <= 1) and its gradient:
    // Horner in y within each z-level (x-degree 1 folded in first), then in z
    float2 V[NB][2], VX[NB][2], VY[NB][2], VZ[NB][2];
#pragma unroll
    for (int c = MDEG; c >= 0; --c) {
        float2 S[NB][2], SX[NB][2], SY[NB][2];
#pragma unroll
        for (int bb = MDEG - c; bb >= 0; --bb) {
            const int m0 = red_index(0, bb, c);
            const float4 q0 = Q[m0];
            const float2 p0 = make_float2(q0.x, q0.y), p1 = make_float2(q0.z, q0.w);
            if (bb == MDEG - c) {   // degree 8: no x term
#pragma unroll
                for (int t = 0; t < NB; ++t) {
                    S[t][0] = p0;
                    S[t][1] = p1;
                }
            } else {
                const float4 q1 = Q[m0 + 1];
                const float2 w0 = make_float2(q1.x, q1.y), w1 = make_float2(q1.z, q1.w);
#pragma unroll
                for (int t = 0; t < NB; ++t) {
                    const float2 R0 = __ffma2_rn(w0, X2[t], p0), R1 = __ffma2_rn(w1, X2[t], p1);
                    if (bb == MDEG - c - 1) {
                        SY[t][0] = S[t][0];
                        SY[t][1] = S[t][1];
                        SX[t][0] = w0;
                        SX[t][1] = w1;
                    } else {
                        SY[t][0] = __ffma2_rn(SY[t][0], Y2[t], S[t][0]);
                        SY[t][1] = __ffma2_rn(SY[t][1], Y2[t], S[t][1]);
                        SX[t][0] = __ffma2_rn(SX[t][0], Y2[t], w0);
                        SX[t][1] = __ffma2_rn(SX[t][1], Y2[t], w1);
                    }
                    S[t][0] = __ffma2_rn(S[t][0], Y2[t], R0);
                    S[t][1] = __ffma2_rn(S[t][1], Y2[t], R1);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < NB; ++t)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (c == MDEG) {
                    V[t][h] = S[t][h];
                } else if (c == MDEG - 1) {
                    VZ[t][h] = V[t][h];
                    V[t][h] = __ffma2_rn(V[t][h], Z2[t], S[t][h]);
                    VX[t][h] = SX[t][h];
                    VY[t][h] = SY[t][h];
                } else {
                    VZ[t][h] = __ffma2_rn(VZ[t][h], Z2[t], V[t][h]);
                    V[t][h] = __ffma2_rn(V[t][h], Z2[t], S[t][h]);
                    VX[t][h] = __ffma2_rn(VX[t][h], Z2[t], SX[t][h]);
                    VY[t][h] = __ffma2_rn(VY[t][h], Z2[t], SY[t][h]);
                }
            }
    }

#pragma unroll
    for (int t = 0; t < NB; ++t) {
        float bw[4], dbw[4];
        const float r2 = r[t] * r[t];
        const float sl = fmaf(-2.0f * r[t], fc[t], 0.0f);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float ex = exp2f(-dp.eta_A_l2[e] * r2);
            bw[e] = ex * fc[t];
            dbw[e] = ex * fmaf(dp.eta_A[e], sl, dfc[t]);
        }
        const float Vv[4] = {V[t][0].x, V[t][0].y, V[t][1].x, V[t][1].y};
        float de = dEdr[t];
#pragma unroll
        for (int e = 0; e < 4; ++e) de = fmaf(fmaf(-2.0f * bw[e], dsum[e], Vv[e]), dbw[e], de);
        const float gx = bw[0] * VX[t][0].x + bw[1] * VX[t][0].y + bw[2] * VX[t][1].x + bw[3] * VX[t][1].y;
        const float gy = bw[0] * VY[t][0].x + bw[1] * VY[t][0].y + bw[2] * VY[t][1].x + bw[3] * VY[t][1].y;
        const float gz = bw[0] * VZ[t][0].x + bw[1] * VZ[t][0].y + bw[2] * VZ[t][1].x + bw[3] * VZ[t][1].y;
        const float ux = X2[t].x, uy = Y2[t].x, uz = Z2[t].x;
        const float gu = gx * ux + gy * uy + gz * uz;
        v[t][0] = de * ux + (gx - gu * ux) * ir[t];
        v[t][1] = de * uy + (gy - gu * uy) * ir[t];
        v[t][2] = de * uz + (gz - gu * uz) * ir[t];
        d[t][0] = ux * r[t];   // the pair vector, for the virial
        d[t][1] = uy * r[t];
        d[t][2] = uz * r[t];
    }
}

// asynchronous 16-byte copy global -> shared (LDGSTS); completion by
// cp_async_wait_all in the issuing thread, then __syncwarp for the warp
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

constexpr int ADJF_WARP_BYTES = NMONO * 16 + NRED * 16 + (MDEG + 1) * 16 + ADJF_RG * 16 + NA * 4;

// MINB: resident warps per SM that the register budget must allow (12: 166
// registers; 14 gives a 128-register build, which the hardware then runs at
// 16 warps per SM); which one is faster depends on the workload (tuned).
template <int MINB>
__global__ void __launch_bounds__(32 * ADJF_WARPS, MINB) desc_mom_adj_fast_kernel(
    const float4* __restrict__ x, const int* __restrict__ ba_sys, const BeadSys* __restrict__ bsys,
    const Rep* __restrict__ reps, const int* __restrict__ nbr, const int* __restrict__ nnb, int maxnb, int B,
    DescParams<float> dp, const float4* __restrict__ Min, const float* __restrict__ dEdG,
    float4* __restrict__ f, float* __restrict__ wbuf, int det, float4* __restrict__ vbuf,
    const float* __restrict__ Eatom, double* __restrict__ V, double* __restrict__ Wv, int b0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wib = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    float4* Qf = reinterpret_cast<float4*>(smem_raw + (size_t)wib * ADJF_WARP_BYTES);   // chain order, 165
    float4* Qr = Qf + NMONO;                                                             // compact, 81
    float4* Phi = Qr + NRED;                                                             // [s], over eta
    float4* RG = Phi + (MDEG + 1);
    float* gA = reinterpret_cast<float*>(RG + ADJF_RG);
    const int b = b0 + blockIdx.x * ADJF_WARPS + wib;   // bead-atoms b0 .. B-1
    if (b >= B) return;

    // loads that depend only on b first: moments (copied asynchronously into
    // the full table, scaled in place below), dE/dG, position, count
#pragma unroll
    for (int k = 0; k < MSLOT; ++k)
        if (k < MSLOT - 1 || lane < (unsigned)MLAST)
            cp_async16(&Qf[lane + 32 * k], &Min[((size_t)b * MSLOT + k) * 32 + lane]);
    cp_async_commit();
    const float gR = dEdG[(size_t)b * ND + lane];
    const float gAn = dEdG[(size_t)b * ND + NR + lane];
    const int n = min(nnb[b], maxnb);
    const float4 xi = x[b];
    const int* __restrict__ nb = nbr + (size_t)b * maxnb;
    const int bs = ba_sys[b];
    const BeadSys sy = bsys[bs];
    // the first round's neighbours
    int ja = 0, jb = 0;
    float4 xa = xi, xb = xi;
    if ((int)lane < n) {
        ja = nb[lane];
        xa = x[sy.ba0 + ja];
    }
    if (n > 32 && 32 + (int)lane < n) {
        jb = nb[32 + lane];
        xb = x[sy.ba0 + jb];
    }
    const Box bx = box_of(reps[sy.rep]);

    {
        const int q = (int)lane >> 3, k = (int)lane & 7;
        float* rg = reinterpret_cast<float*>(RG) + ((q & 1) * 8 + k) * 4 + (q >> 1);
        rg[0] = gR;
        rg[2] = gR * dp.r_mu[lane];
        gA[lane] = gAn;
    }
    __syncwarp();
    // Phi_eta(s): lane (s = lane / 4, eta = lane % 4) for s < 8, then s = 8
    {
        const int sd = (int)lane >> 2, e = (int)lane & 3;
        const int li = sd & 1;   // D^+ = D(+) + D(-) for even s, D^- = D(+) - D(-) for odd s
        float ph = 0.0f;
#pragma unroll
        for (int z = 0; z < 4; ++z) {
            const float dd = li ? gA[(2 * z) * 4 + e] - gA[(2 * z + 1) * 4 + e]
                                : gA[(2 * z) * 4 + e] + gA[(2 * z + 1) * 4 + e];
            ph = fmaf(g_fold.cphi[z][sd], dd, ph);
        }
        reinterpret_cast<float*>(Phi)[lane] = ph;
        if (lane < 4)
            reinterpret_cast<float*>(Phi)[32 + lane] = g_fold.cphi[3][MDEG] * (gA[6 * 4 + lane] + gA[7 * 4 + lane]);
    }
    float dsum[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) dsum[e] = gA[e] + gA[8 + e] + gA[16 + e] + gA[24 + e];
    cp_async_wait_all();
    __syncwarp();
    // Q_abc = M_abc Phi(s) 2 / (a! b! c!)
#pragma unroll
    for (int k = 0; k < MSLOT; ++k) {
        if (k < MSLOT - 1 || lane < (unsigned)MLAST) {
            const float4 ph = Phi[g_fold.deg[k][lane]];
            const float w = g_fold.w[k][lane];
            const float4 M = Qf[lane + 32 * k];
            Qf[lane + 32 * k] = make_float4(M.x * ph.x * w, M.y * ph.y * w, M.z * ph.z * w, M.w * ph.w * w);
        }
    }
    __syncwarp();
    // fold onto the compact reduced table, one pass
    {
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int e = 0; e < FOLD_MAX; ++e) {
            const unsigned w = g_fold.ent[e][lane];
            const float cf = (float)((int)w >> 24);
            const float4 q = Qf[w & 0xffu];
            acc.x = fmaf(cf, q.x, acc.x);
            acc.y = fmaf(cf, q.y, acc.y);
            acc.z = fmaf(cf, q.z, acc.z);
            acc.w = fmaf(cf, q.w, acc.w);
            if (w & 0x10000u) {
                Qr[(w >> 8) & 0xffu] = acc;
                acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
    }
    __syncwarp();

    float red[16];   // force on the centre (3), virial (9), padding
#pragma unroll
    for (int q = 0; q < 16; ++q) red[q] = 0.0f;
    int s0 = 0;
    while (s0 < n) {
        // keeps the coefficient loads inside the round: hoisted out of the
        // loop they would hold the 81 float4 in registers
        asm volatile("" ::: "memory");
        const bool paired = n - s0 > 32;        // warp-uniform
        const int s1 = s0 + (paired ? 64 : 32);
        const int sA = s0 + (int)lane, sB = sA + 32;
        const float4 ca = xa, cb = xb;
        const int ka = ja, kb = jb;
        // the next round's neighbours
        if (s1 + (int)lane < n) {
            ja = nb[s1 + lane];
            xa = x[sy.ba0 + ja];
        }
        if (n - s1 > 32 && s1 + 32 + (int)lane < n) {
            jb = nb[s1 + 32 + lane];
            xb = x[sy.ba0 + jb];
        }
        float v[2][3], dv[2][3];
        bool ok[2];
        if (paired) {
            const float4 xx[2] = {ca, cb};
            const bool vv[2] = {sA < n, sB < n};
            adj_fast_eval<2>(bx, dp, xi, xx, vv, Qr, RG, dsum, v, dv);
            ok[0] = vv[0];
            ok[1] = vv[1];
        } else {
            const float4 xx[1] = {ca};
            const bool vv[1] = {sA < n};
            float v1[1][3], d1[1][3];
            adj_fast_eval<1>(bx, dp, xi, xx, vv, Qr, RG, dsum, v1, d1);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                v[0][a] = v1[0][a];
                dv[0][a] = d1[0][a];
                v[1][a] = dv[1][a] = 0.0f;
            }
            ok[0] = vv[0];
            ok[1] = false;
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (!ok[t]) continue;
            const int sl = t == 0 ? sA : sB;
            const int j = t == 0 ? ka : kb;
            if (det)
                vbuf[(size_t)b * maxnb + sl] = make_float4(v[t][0], v[t][1], v[t][2], 0.0f);
            else
                atomicAdd(&f[sy.ba0 + j], make_float4(-v[t][0], -v[t][1], -v[t][2], 0.0f));
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                red[a] += v[t][a];
#pragma unroll
                for (int c = 0; c < 3; ++c) red[3 + 3 * a + c] -= dv[t][a] * v[t][c];
            }
        }
        s0 = s1;
    }
    // lanes 2q and 2q + 1 end with the sum of value q
#pragma unroll
    for (int o = 16, cnt = 16; o >= 2; o >>= 1, cnt >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < cnt / 2; ++q) {
            const float send = upper ? red[q] : red[q + cnt / 2];
            const float keep = upper ? red[q + cnt / 2] : red[q];
            red[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    const float tot = red[0] + __shfl_xor_sync(0xffffffffu, red[0], 1);
    const int vi = (int)(lane >> 1);
    if ((lane & 1) == 0) {
        if (vi < 3) {
            if (det)
                reinterpret_cast<float*>(&f[b])[vi] = tot;   // gathered later
            else
                atomicAdd(reinterpret_cast<float*>(&f[b]) + vi, tot);
        } else if (vi < 12) {
            // deterministic mode: per-atom virials, summed in a fixed order
            // later; otherwise straight into the bead's FP64 sums
            if (det)
                wbuf[(size_t)b * 9 + (vi - 3)] = tot;
            else
                atomicAdd(&Wv[(size_t)bs * 9 + (vi - 3)], (double)tot);
        } else if (vi == 12 && !det) {
            atomicAdd(&V[bs], (double)Eatom[b]);
        }
    }
}

size_t moment_elems_per_atom() { return (size_t)MSLOT * 32; }   // float4 per bead-atom

template <bool FAST>
static void run_fwd(const Dev& d, const void* dpv, cudaStream_t st)
{
    const size_t sm = (size_t)FWD_WARPS * FWD_WARP_FLOATS * sizeof(float);
    { static size_t done = 0; set_smem(desc_mom_fwd_kernel<FAST>, sm, done); }
    desc_mom_fwd_kernel<FAST><<<(d.B + FWD_WARPS - 1) / FWD_WARPS, 32 * FWD_WARPS, sm, st>>>(
        (const float4*)d.x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, d.B,
        *(const DescParams<float>*)dpv, (float*)d.G, (float4*)d.mom);
}

template <bool FAST>
static void run_adj(const Dev& d, const void* dpv, cudaStream_t st)
{
    const size_t sm = (size_t)ADJ_WARPS * ADJ_WARP_BYTES;
    desc_mom_adj_kernel<FAST><<<(d.B + ADJ_WARPS - 1) / ADJ_WARPS, 32 * ADJ_WARPS, sm, st>>>(
        (const float4*)d.x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, d.B,
        *(const DescParams<float>*)dpv, (const float4*)d.mom, (const float*)d.dEdG, (float4*)d.f,
        (float*)d.wbuf, d.deterministic, (float4*)d.vbuf);
}

static void run_fwd_red(const Dev& d, const void* dpv, int b0, int b1, cudaStream_t st)
{
    if (b1 <= b0) return;
    const size_t sm = (size_t)FWDR_WARPS * FWDR_WARP_FLOATS * sizeof(float);
    { static size_t done = 0; set_smem(desc_mom_fwd_red_kernel<true>, sm, done); }
    desc_mom_fwd_red_kernel<true><<<(b1 - b0 + FWDR_WARPS - 1) / FWDR_WARPS, 32 * FWDR_WARPS, sm, st>>>(
        (const float4*)d.x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, b1,
        *(const DescParams<float>*)dpv, (float*)d.G, (float4*)d.mom, b0);
}

void launch_descriptors_moment(const Dev& d, const void* dpv, cudaStream_t st)
{
    if (d.precision == 2)
        run_fwd_red(d, dpv, 0, d.B, st);
    else
        run_fwd<false>(d, dpv, st);
}

static void run_adj_fast(const Dev& d, const void* dpv, int b0, int b1, cudaStream_t st)
{
    if (b1 <= b0) return;
    const size_t sm = (size_t)ADJF_WARPS * ADJF_WARP_BYTES;
    const int grid = (b1 - b0 + ADJF_WARPS - 1) / ADJF_WARPS;
    if (d.sched.adj_wide)
        desc_mom_adj_fast_kernel<14><<<grid, 32 * ADJF_WARPS, sm, st>>>(
            (const float4*)d.x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, b1,
            *(const DescParams<float>*)dpv, (const float4*)d.mom, (const float*)d.dEdG, (float4*)d.f,
            (float*)d.wbuf, d.deterministic, (float4*)d.vbuf, (const float*)d.Eatom, d.V, d.W, b0);
    else
        desc_mom_adj_fast_kernel<12><<<grid, 32 * ADJF_WARPS, sm, st>>>(
            (const float4*)d.x, d.ba_sys, d.bsys, d.reps, d.nbr, d.nnb, d.maxnb, b1,
            *(const DescParams<float>*)dpv, (const float4*)d.mom, (const float*)d.dEdG, (float4*)d.f,
            (float*)d.wbuf, d.deterministic, (float4*)d.vbuf, (const float*)d.Eatom, d.V, d.W, b0);
}

// The BF16 moment path (reduced-basis forward, fast adjoint) on the bead-atoms
// b0 .. b1-1 only: the two halves of a step's beads can then run as
// overlapping branches of the step's graph.
bool moment_fast_path(const Dev& d, const void* dpv)
{
    return d.precision == 2 && d.sched.ang && d.mom && ((const DescParams<float>*)dpv)->r_even;
}
void launch_descriptors_range(const Dev& d, const void* dpv, int b0, int b1, cudaStream_t st)
{
    run_fwd_red(d, dpv, b0, b1, st);
}
void launch_adjoint_range(const Dev& d, const void* dpv, int b0, int b1, cudaStream_t st)
{
    run_adj_fast(d, dpv, b0, b1, st);
}

bool moment_adjoint_sums_energy(const Dev& d, const void* dpv)
{
    return d.precision == 2 && !d.deterministic && ((const DescParams<float>*)dpv)->r_even;
}

void launch_adjoint_moment(const Dev& d, const void* dpv, cudaStream_t st)
{
    if (d.precision == 2) {
        if (((const DescParams<float>*)dpv)->r_even)
            run_adj_fast(d, dpv, 0, d.B, st);
        else
            run_adj<true>(d, dpv, st);
    } else {
        run_adj<false>(d, dpv, st);
    }
}

}  // namespace pimd
