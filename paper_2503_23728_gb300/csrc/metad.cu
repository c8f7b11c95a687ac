// metad.cu -- well-tempered metadynamics on a collective variable of every
// bead (Sec. 2.5): the CV and its gradient per bead, the Gaussian bias and
// its force, and the deposition of hills.
//
// CVs (Secs. S2-S3):
//   distances:  s = sum_t c_t |x_(j_t) - x_(i_t)|   (the dimer's proton-transfer CV)
//   XRD:        s = (1/N) sum_i sum_j f_i f_j sin(Q R_ij) / (Q R_ij), i = j terms f_i^2
// Bias: V(s) = sum_k h_k exp(-(s - s_k)^2 / (2 sigma^2)) on every bead; hills
// go down after the force evaluation of step n when (n + 1) % stride == 0,
// one per bead at its CV with height (h0 / P) exp(-V(s_k) / (k_B T (gamma-1))).
#include <cuda_runtime.h>
#include <math_constants.h>

#include "common.cuh"
#include "geom.cuh"
#include "kernels.h"
#include "pimd.h"

namespace pimd {

// ---------------------------------------------------------------------------
// distance-combination CV: one thread per bead-system
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void cv_dist_kernel(const Vec4<Real>* __restrict__ x, const BeadSys* __restrict__ bsys,
                               const Rep* __restrict__ reps, int S, MetadParams mp, Vec4<Real>* __restrict__ grad,
                               double* __restrict__ cvpart, double* __restrict__ virpart, int ntile)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    const BeadSys sy = bsys[k];
    const Rep& rp = reps[sy.rep];
    double s = 0.0, vir[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = 0; t < mp.n_terms; ++t) {
        const int i = mp.ti[t], j = mp.tj[t];
        Real r[3];
        pair_vec(rp, x[sy.ba0 + i], x[sy.ba0 + j], r[0], r[1], r[2]);
        const double rx = (double)r[0], ry = (double)r[1], rz = (double)r[2];
        const double d = sqrt(rx * rx + ry * ry + rz * rz);
        s += mp.tc[t] * d;
        const double g[3] = {mp.tc[t] * rx / d, mp.tc[t] * ry / d, mp.tc[t] * rz / d};
        Vec4<Real>& gj = grad[sy.ba0 + j];
        Vec4<Real>& gi = grad[sy.ba0 + i];
        gj.x += (Real)g[0]; gj.y += (Real)g[1]; gj.z += (Real)g[2];
        gi.x -= (Real)g[0]; gi.y -= (Real)g[1]; gi.z -= (Real)g[2];
        const double rv[3] = {rx, ry, rz};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) vir[3 * a + b] += rv[a] * g[b];
    }
    cvpart[(size_t)k * ntile] = s;
#pragma unroll
    for (int q = 0; q < 9; ++q) virpart[((size_t)k * ntile) * 9 + q] = vir[q];
}

// ---------------------------------------------------------------------------
// XRD CV: grid (atom tiles x row slices, bead-systems); thread per atom i
// sums its row j != i over one of MD_SLICES slices (no atomics: every pair is
// seen from both ends), giving
//   N s = sum_i [f_i^2 + sum_(j != i) f_i f_j sinc(Q R_ij)],
//   ds/dx_i = (2/N) sum_(j != i) f_i f_j Q sinc'(Q R_ij) (x_i - x_j) / R_ij,
// and the pair virial (halved, each pair twice). Gradients go to per-slice
// buffers and block sums (FP64) to per-(tile, slice) partials; the bias
// kernels add both in a fixed order.
// ---------------------------------------------------------------------------
// sin and cos of y >= 0. FP32: Cody-Waite reduction y - 2 pi k with 2 pi
// split into a float head and the float of the remainder (k = rint(y / 2 pi)
// stays small here: Q R < 100), then the special-function unit on
// [-pi, pi] (absolute error ~5e-7, far inside the CV's use as a bias
// coordinate). FP64: the accurate library routine.
constexpr float TWO_PI_HI = 6.28318548202514648f;                    // float(2 pi)
constexpr float TWO_PI_LO = (float)(6.283185307179586477 - 6.28318548202514648);
__device__ __forceinline__ void sincos_r(float y, float& s, float& c)
{
    const float k = rintf(y * (1.0f / 6.283185307179586f));
    float t = fmaf(-k, TWO_PI_HI, y);
    t = fmaf(-k, TWO_PI_LO, t);
    s = __sinf(t);
    c = __cosf(t);
}
__device__ __forceinline__ void sincos_r(double y, double& s, double& c) { sincos(y, &s, &c); }

// plain minimum-image difference (the CV needs no error-free pair vector)
__device__ __forceinline__ void xrd_pair(const Rep& rp, const float4& a, const float4& b, float (&r)[3])
{
    r[0] = b.x - a.x; r[1] = b.y - a.y; r[2] = b.z - a.z;
    if (rp.periodic) {
#pragma unroll
        for (int d = 0; d < 3; ++d) r[d] = fmaf(-rp.Lf[d], rintf(r[d] * rp.invLf[d]), r[d]);
    }
}
__device__ __forceinline__ void xrd_pair(const Rep& rp, const Dbl4& a, const Dbl4& b, double (&r)[3])
{
    pair_vec(rp, a, b, r[0], r[1], r[2]);
}
__device__ __forceinline__ float xrd_rcp(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double xrd_rcp(double v) { return 1.0 / v; }

template <typename Real>
__global__ void __launch_bounds__(128) cv_xrd_kernel(const Vec4<Real>* __restrict__ x,
                                                     const BeadSys* __restrict__ bsys, const Rep* __restrict__ reps,
                                                     const int* __restrict__ atype, MetadParams mp,
                                                     Vec4<Real>* __restrict__ grad, double* __restrict__ cvpart,
                                                     double* __restrict__ virpart, int ntile, int B)
{
    __shared__ double red[10][4];
    const int k = blockIdx.y;
    const BeadSys sy = bsys[k];
    const Rep& rp = reps[sy.rep];
    const int N = sy.N;
    const int tile = blockIdx.x / MD_SLICES, slice = blockIdx.x - tile * MD_SLICES;
    const int i = tile * blockDim.x + threadIdx.x;
    const int jper = (N + MD_SLICES - 1) / MD_SLICES;
    const int jlo = slice * jper, jhi = min(N, jlo + jper);
    const Real Q = (Real)mp.Q;
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};   // N s share, then the 9 virial entries
    if (i < N) {
        const Vec4<Real> xi = x[sy.ba0 + i];
        const Real fi = (Real)mp.f_type[atype[rp.atom0 + i]];
        Real srow = Real(0), g[3] = {Real(0), Real(0), Real(0)}, vir[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) vir[q] = Real(0);
        const Real c0 = Real(2) * Q * Q / (Real)N;   // c = c0 f_i f_j (y cos y - sin y) / y^3
        for (int j = jlo; j < jhi; ++j) {
            if (j == i) continue;
            Real r[3];
            xrd_pair(rp, xi, x[sy.ba0 + j], r);
            const Real R2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            const Real R = f_sqrt(R2);
            const Real y = Q * R;
            Real sn, cs;
            sincos_r(y, sn, cs);
            const Real iy = xrd_rcp(y);
            const Real ff = fi * (Real)mp.f_type[atype[rp.atom0 + j]];
            const Real sc = sn * iy;                      // sinc(QR)
            srow += ff * sc;
            // ds/dr_ij = c r_ij, c = 2 f_i f_j Q sinc'(QR) / (N R) = c0 f_i f_j (cos y - sinc y) / y^2
            const Real c = c0 * ff * (cs - sc) * iy * iy;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                g[a] -= c * r[a];
#pragma unroll
                for (int b = a; b < 3; ++b) vir[3 * a + b] += r[a] * c * r[b];
            }
        }
        vir[3] = vir[1];
        vir[6] = vir[2];
        vir[7] = vir[5];
        grad[(size_t)slice * B + sy.ba0 + i] = make4<Vec4<Real>, Real>(g[0], g[1], g[2], Real(0));
        acc[0] = (slice == 0 ? (double)fi * (double)fi : 0.0) + (double)srow;
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[1 + q] = 0.5 * (double)vir[q];
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) acc[q] = warp_sum(acc[q]);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < 10; ++q) red[q][w] = acc[q];
    __syncthreads();
    if (threadIdx.x < 10) {
        const double v = red[threadIdx.x][0] + red[threadIdx.x][1] + red[threadIdx.x][2] + red[threadIdx.x][3];
        if (threadIdx.x == 0)
            cvpart[(size_t)k * ntile + blockIdx.x] = v;
        else
            virpart[((size_t)k * ntile + blockIdx.x) * 9 + threadIdx.x - 1] = v;   // ntile counts (tile, slice)
    }
}

// ---------------------------------------------------------------------------
// bias: one block per replica, thread per bead. s from the tile partials
// (fixed order), V(s) and dV/ds over the replica's hills, the bias energy
// and virial into the bead's V and W, then (deposition steps only) one hill
// per bead.
// ---------------------------------------------------------------------------
__global__ void bias_kernel(const Rep* __restrict__ reps, const BeadSys* __restrict__ bsys, MetadParams mp,
                            const double* __restrict__ cvpart, const double* __restrict__ virpart, int ntile,
                            double2* __restrict__ hills, int* __restrict__ nhill, double* __restrict__ cv,
                            double* __restrict__ vb, double* __restrict__ dvds, double* __restrict__ V,
                            double* __restrict__ W, const unsigned long long* __restrict__ stepp, int offset,
                            int deposit, DevErr* __restrict__ err)
{
    // stepp: the step counter copy made by the ring start of the current
    // launch; offset: the steps of a multi-step launch since that start
    const int r = blockIdx.x;
    const Rep& rp = reps[r];
    const int k = threadIdx.x;
    const int n = nhill[r];
    const double2* H = hills + (size_t)r * mp.max_hills;
    double s = 0.0, v = 0.0;
    if (k < rp.P) {
        const int bs = rp.bs0 + k;
        const int ntl = mp.cv == PIMD_CV_XRD ? ntile : 1;
        for (int t = 0; t < ntl; ++t) s += cvpart[(size_t)bs * ntile + t];
        if (mp.cv == PIMD_CV_XRD) s /= (double)bsys[bs].N;
        double dv = 0.0;
        const double is2 = 1.0 / (mp.sigma * mp.sigma);
        for (int h = 0; h < n; ++h) {
            const double u = s - H[h].x;
            const double g = H[h].y * exp(-0.5 * u * u * is2);
            v += g;
            dv -= g * u * is2;
        }
        cv[bs] = s;
        vb[bs] = v;
        dvds[bs] = dv;
        V[bs] += v;
        for (int q = 0; q < 9; ++q) {
            double w = 0.0;
            for (int t = 0; t < ntl; ++t) w += virpart[((size_t)bs * ntile + t) * 9 + q];
            W[(size_t)bs * 9 + q] -= dv * w;
        }
    }
    if (!deposit || ((*stepp + (unsigned long long)offset + 1ull) % (unsigned long long)mp.stride) != 0ull) return;
    __syncthreads();   // every bead has read the hills before any is added
    if (n + rp.P > mp.max_hills) {
        if (k == 0) atomicOr(&err->flags, ERR_METAD_FULL);
        return;
    }
    if (k < rp.P) {
        const double kT = rp.kT_md * MVV2E / rp.P;   // k_B T of the physical temperature, eV
        const double h = mp.h0 / rp.P * exp(-v / (kT * (mp.gamma - 1.0)));
        hills[(size_t)r * mp.max_hills + n + k] = make_double2(s, h);
    }
    __syncthreads();
    if (k == 0) nhill[r] = n + rp.P;
}

// f_b -= dV/ds ds/dx_b for every bead-atom (gradient slices added in order)
template <typename Real>
__global__ void bias_force_kernel(const int* __restrict__ ba_sys, const Vec4<Real>* __restrict__ grad,
                                  const double* __restrict__ dvds, Vec4<Real>* __restrict__ f, int B, int nslice)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const Real dv = (Real)dvds[ba_sys[b]];
    Vec4<Real> g = grad[b];
    for (int q = 1; q < nslice; ++q) {
        const Vec4<Real> h = grad[(size_t)q * B + b];
        g.x += h.x; g.y += h.y; g.z += h.z;
    }
    Vec4<Real> v = f[b];
    v.x -= dv * g.x;
    v.y -= dv * g.y;
    v.z -= dv * g.z;
    f[b] = v;
}

int metad_tiles(int max_N) { return (max_N + 127) / 128 * MD_SLICES; }

void launch_metad(const Dev& d, bool deposit, cudaStream_t st, int step_offset)
{
    const MetadParams& mp = d.metad;
    const int ntile = metad_tiles(d.max_N);
    const size_t v4 = d.precision == 0 ? sizeof(Dbl4) : sizeof(float4);
    const int nslice = mp.cv == PIMD_CV_XRD ? MD_SLICES : 1;
    if (mp.cv == PIMD_CV_DISTANCES) {
        cudaMemsetAsync(d.md_grad, 0, v4 * d.B, st);
        if (d.precision == 0)
            cv_dist_kernel<double><<<(d.S + 127) / 128, 128, 0, st>>>((const Dbl4*)d.x, d.bsys, d.reps, d.S, mp,
                                                                      (Dbl4*)d.md_grad, d.md_cvpart, d.md_virpart,
                                                                      ntile);
        else
            cv_dist_kernel<float><<<(d.S + 127) / 128, 128, 0, st>>>((const float4*)d.x, d.bsys, d.reps, d.S, mp,
                                                                     (float4*)d.md_grad, d.md_cvpart, d.md_virpart,
                                                                     ntile);
    } else {
        const dim3 grid(ntile, d.S);
        if (d.precision == 0)
            cv_xrd_kernel<double><<<grid, 128, 0, st>>>((const Dbl4*)d.x, d.bsys, d.reps, d.atype, mp,
                                                        (Dbl4*)d.md_grad, d.md_cvpart, d.md_virpart, ntile, d.B);
        else
            cv_xrd_kernel<float><<<grid, 128, 0, st>>>((const float4*)d.x, d.bsys, d.reps, d.atype, mp,
                                                       (float4*)d.md_grad, d.md_cvpart, d.md_virpart, ntile, d.B);
    }
    bias_kernel<<<d.R, d.max_P, 0, st>>>(d.reps, d.bsys, mp, d.md_cvpart, d.md_virpart, ntile, d.md_hills,
                                         d.md_nhill, d.md_cv, d.md_vb, d.md_dvds, d.V, d.W, d.step_cur,
                                         step_offset, deposit ? 1 : 0, d.err);
    if (d.precision == 0)
        bias_force_kernel<double><<<(d.B + 255) / 256, 256, 0, st>>>(d.ba_sys, (const Dbl4*)d.md_grad, d.md_dvds,
                                                                     (Dbl4*)d.f, d.B, nslice);
    else
        bias_force_kernel<float><<<(d.B + 255) / 256, 256, 0, st>>>(d.ba_sys, (const float4*)d.md_grad, d.md_dvds,
                                                                    (float4*)d.f, d.B, nslice);
}

// ---------------------------------------------------------------------------
// free-energy surfaces (Sec. 2.5)
// ---------------------------------------------------------------------------
// One sample of the bead-resolved CV histogram of the path-integral FES: the
// replica's P beads (CVs and biases of the last force evaluation) with the
// weight w = exp(sum_k V_b(s_k) / (k_B T P) - shift) that undoes the bias on
// the ring polymer's configurational weight. One thread, beads in order, so
// every sum has a fixed order.
__global__ void cv_hist_kernel(const double* __restrict__ cv, const double* __restrict__ vb, int bs0, int P,
                               double kTP, double s_min, double inv_ds, int n_bins, double shift,
                               double* __restrict__ hist, double* __restrict__ wsum)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double v = 0.0;
    for (int k = 0; k < P; ++k) v += vb[bs0 + k];
    const double w = exp(v / kTP - shift);
    for (int k = 0; k < P; ++k) {
        const double tb = (cv[bs0 + k] - s_min) * inv_ds;
        if (tb >= 0.0 && tb < (double)n_bins) hist[(size_t)k * n_bins + (int)floor(tb)] += w;
    }
    *wsum += w;
}

// F_k(s_b) = -k_B T ln(hist[k][b] / (wsum ds)) and the path-integral
// F(s_b) = -k_B T ln((1/P) sum_k hist[k][b] / (wsum ds)); thread per bin
__global__ void pi_fes_kernel(const double* __restrict__ hist, const double* __restrict__ wsum, int P, int n_bins,
                              double ds, double kT, double* __restrict__ F, double* __restrict__ Fk)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bins) return;
    const double ws = *wsum;
    double tot = 0.0;
    for (int k = 0; k < P; ++k) {
        const double h = hist[(size_t)k * n_bins + b];
        tot += h;
        if (Fk) Fk[(size_t)k * n_bins + b] = h > 0.0 ? -kT * log(h / (ws * ds)) : CUDART_INF;
    }
    F[b] = tot > 0.0 ? -kT * log(tot / (P * ws * ds)) : CUDART_INF;
}

// F(s) = -(gamma / (gamma - 1)) V(s) over the replica's hills; thread per s
__global__ void metad_fes_kernel(const double2* __restrict__ hills, const int* __restrict__ nhill, double sigma,
                                 double gamma, const double* __restrict__ s, int n, double* __restrict__ F)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nh = *nhill;
    double v = 0.0;
    for (int h = 0; h < nh; ++h) {
        const double u = s[i] - hills[h].x;
        v += hills[h].y * exp(-0.5 * u * u / (sigma * sigma));
    }
    F[i] = -(gamma / (gamma - 1.0)) * v;
}

void launch_cv_hist(const Dev& d, int replica, int bs0, int P, double kTP, double s_min, double inv_ds, int n_bins,
                    double shift, double* hist, double* wsum, cudaStream_t st)
{
    (void)replica;
    cv_hist_kernel<<<1, 32, 0, st>>>(d.md_cv, d.md_vb, bs0, P, kTP, s_min, inv_ds, n_bins, shift, hist, wsum);
}

void launch_pi_fes(const double* hist, const double* wsum, int P, int n_bins, double ds, double kT, double* F,
                   double* Fk, cudaStream_t st)
{
    pi_fes_kernel<<<(n_bins + 127) / 128, 128, 0, st>>>(hist, wsum, P, n_bins, ds, kT, F, Fk);
}

void launch_metad_fes(const Dev& d, int replica, const double* s, int n, double* F, cudaStream_t st)
{
    metad_fes_kernel<<<(n + 127) / 128, 128, 0, st>>>(d.md_hills + (size_t)replica * d.metad.max_hills,
                                                       d.md_nhill + replica, d.metad.sigma, d.metad.gamma, s, n, F);
}

}  // namespace pimd
