// noalloc.cu -- descriptor evaluation whose scratch memory is a fixed,
// file-scope device array instead of a caller workspace.
//
// For callers that cannot allocate device memory at all (hosts that reserve
// the whole device for their own pool, plug-in environments that forbid
// cudaMalloc after start-up, code that must not touch an allocator). The
// caller still passes the positions and the output array. Nothing here
// calls cudaMalloc, cudaFree or an allocating library routine.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/pimd.h"
#include "common.cuh"
#include "kernels.h"

using namespace pimd;

namespace {

constexpr int MAXA = PIMD_NOALLOC_MAX_ATOMS;
constexpr int MAXNB = PIMD_NOALLOC_MAX_NEIGHBOURS;

// carve of the static array (bytes, 256-aligned pieces)
constexpr size_t al(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t OFF_REP = 0;
constexpr size_t OFF_BS = OFF_REP + al(sizeof(Rep));
constexpr size_t OFF_BASYS = OFF_BS + al(sizeof(BeadSys));
constexpr size_t OFF_X = OFF_BASYS + al(sizeof(int) * MAXA);
constexpr size_t OFF_NBR = OFF_X + al(sizeof(float4) * MAXA);
constexpr size_t OFF_NNB = OFF_NBR + al(sizeof(int) * (size_t)MAXA * MAXNB);
constexpr size_t OFF_G = OFF_NNB + al(sizeof(int) * MAXA);
constexpr size_t OFF_ERR = OFF_G + al(sizeof(float) * (size_t)MAXA * ND);
constexpr size_t SCRATCH_BYTES = OFF_ERR + al(sizeof(DevErr));

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

std::mutex g_mu;
void* g_addr[256] = {};   // device address of g_noalloc_scratch, per device ordinal

// message for pimd_last_error(NULL)
int fail(int code, const std::string& m)
{
    pimd::set_thread_error(m);
    return code;
}

int scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PIMD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= 256) return fail(PIMD_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        // host code only holds a stand-in for the symbol: ask the runtime for
        // its address on the current device
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(PIMD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PIMD_OK;
}

}  // namespace

extern "C" int pimd_descriptors_noalloc(const double* x_dev, int n_atoms, const double* box, double cutoff_A,
                                        double eta_R, const double* r_mu, const double* eta_A, double* G_dev,
                                        void* stream)
{
    if (!x_dev || !G_dev || !r_mu || !eta_A) return fail(PIMD_ERR_INVALID_ARG, "NULL argument");
    if (n_atoms < 1 || n_atoms > MAXA)
        return fail(PIMD_ERR_INVALID_ARG, "n_atoms must be 1.." + std::to_string(MAXA) +
                                              " (size of the static scratch array), got " + std::to_string(n_atoms));
    if (!(cutoff_A > 0.0)) return fail(PIMD_ERR_INVALID_ARG, "cutoff_A must be > 0");
    const bool per = box && (box[0] != 0.0 || box[1] != 0.0 || box[2] != 0.0);
    if (per)
        for (int a = 0; a < 3; ++a)
            if (!(box[a] >= 2.0 * cutoff_A)) return fail(PIMD_ERR_INVALID_ARG, "periodic box shorter than twice the cutoff");
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    unsigned char* w = static_cast<unsigned char*>(base);
    cudaStream_t st = (cudaStream_t)stream;

    Rep rp;
    std::memset(&rp, 0, sizeof(rp));
    rp.N = n_atoms;
    rp.P = 1;
    rp.periodic = per ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        rp.L[a] = per ? box[a] : 0.0;
        rp.invL[a] = per ? 1.0 / box[a] : 0.0;
        rp.Lf[a] = (float)rp.L[a];
        rp.invLf[a] = (float)rp.invL[a];
        rp.Llo[a] = (float)(rp.L[a] - (double)rp.Lf[a]);
    }
    BeadSys bs = {0, n_atoms, 0, 0};
    DescParams<float> dp{};   // r_even = 0: the FP32 path's exact radial Gaussians
    dp.rc = (float)cutoff_A;
    dp.pi_over_rc = (float)(M_PI / cutoff_A);
    dp.eta_R = (float)eta_R;
    for (int q = 0; q < NR; ++q) dp.r_mu[q] = (float)r_mu[q];
    for (int q = 0; q < 4; ++q) dp.eta_A[q] = (float)eta_A[q];
    dp.eta_R_l2 = (float)(eta_R * M_LOG2E);
    for (int q = 0; q < 4; ++q) dp.eta_A_l2[q] = (float)(eta_A[q] * M_LOG2E);

    Dev d;
    d.R = 1; d.S = 1; d.B = n_atoms; d.NA = n_atoms;
    d.max_N = n_atoms;
    d.maxnb = MAXNB;
    d.precision = PIMD_FP32;
    d.rc = cutoff_A;
    d.reps = reinterpret_cast<Rep*>(w + OFF_REP);
    d.bsys = reinterpret_cast<BeadSys*>(w + OFF_BS);
    d.ba_sys = reinterpret_cast<int*>(w + OFF_BASYS);
    d.x = w + OFF_X;
    d.nbr = reinterpret_cast<int*>(w + OFF_NBR);
    d.nnb = reinterpret_cast<int*>(w + OFF_NNB);
    d.G = w + OFF_G;
    d.err = reinterpret_cast<DevErr*>(w + OFF_ERR);

    cudaError_t e = cudaMemcpyAsync(d.reps, &rp, sizeof(Rep), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.bsys, &bs, sizeof(BeadSys), cudaMemcpyHostToDevice, st);
    // the array keeps the previous call's contents: reset what must start at zero
    if (e == cudaSuccess) e = cudaMemsetAsync(d.ba_sys, 0, sizeof(int) * n_atoms, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.x, 0, sizeof(float4) * n_atoms, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.err, 0, sizeof(DevErr), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PIMD_ERR_CUDA, std::string("set-up copies: ") + cudaGetErrorString(e));
    }
    launch_pack_positions(d, x_dev, st);
    launch_neighbours(d, st);
    launch_descriptors(d, &dp, st);
    launch_descriptors_out(d, G_dev, st);
    DevErr h;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d.err, sizeof(DevErr), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PIMD_ERR_CUDA, std::string("descriptor launch: ") + cudaGetErrorString(e));
    }
    if (h.flags & ERR_NBR_OVERFLOW)
        return fail(PIMD_ERR_NBR_OVERFLOW, "an atom has " + std::to_string(h.max_nbr) + " neighbours, more than the " +
                                               std::to_string(MAXNB) + " slots of the static scratch array");
    return PIMD_OK;
}
