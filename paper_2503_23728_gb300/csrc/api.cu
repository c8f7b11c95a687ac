// api.cu -- the C ABI (include/pimd.h): context set-up inside the caller's
// workspace, weight loading, the per-step launch sequence captured in CUDA
// graphs, and the synchronising queries.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/pimd.h"
#include "common.cuh"
#include "kernels.h"

using namespace pimd;

namespace {

thread_local std::string g_tls_error;

struct HostRep {
    int N = 0, P = 0;
    std::vector<int> Z;
    std::vector<double> mass, x0;
    double box[3] = {0, 0, 0};
    double T = 0;
    unsigned long long seed = 0;
};

double default_mass(int z)
{
    switch (z) {
        case 1: return 1.008;
        case 6: return 12.011;
        case 7: return 14.007;
        case 8: return 15.999;
        default: return -1.0;
    }
}

// overlapping parts of a large BF16 step's force evaluation
constexpr int OVERLAP_PARTS = 2;

// Everything the host computes before touching the device.
struct Build {
    std::vector<Rep> reps;
    std::vector<BeadSys> bsys;
    std::vector<int> ba_sys, atype, perm, tile_type;
    std::vector<double> mass, x0, cmat;
    std::vector<Mode> modes;
    std::vector<int2> rp_blocks;
    std::vector<int> rep_blk0;
    std::vector<int> typeZ;
    std::vector<double> repT;   // physical temperature of each replica, K
    std::vector<int> cell_bs;
    int total_cells = 0, max_cells = 0;
    int R = 0, S = 0, B = 0, NA = 0, rows_pad = 0;
    std::vector<int> part_ba, part_tile;   // parts of the bead-atoms / network tiles (boundaries; one part: none)
    size_t blob = 0, wtc_bytes = 0, wtc_vec = 0;
    size_t gfn_params = 0;   // FP32 parameters of the graph-field-network head
    bool periodic_any = false;
    bool any_skin = false;
    double max_skin = 0.0;   // largest Verlet skin among the replicas, A
    double nb_est = 0.0;   // mean neighbour count per bead-atom (estimate from density)
};

// candidate slots per atom for Verlet lists: 1.5 x the neighbour slots
// (a skin of 0.5 A at r_c = 6 A holds 1.27 x the neighbours), multiple of 32,
// at most the sort capacity
// candidate slots per bead-atom: the neighbour slots scaled by the volume of
// the r_c + skin sphere over the r_c sphere, 10 % margin, multiple of 32, at
// most the sort buffer (an atom with more candidates is scanned directly)
int max_candidates(int maxnb, double rc, double skin)
{
    const double v = std::pow((rc + skin) / rc, 3.0) * 1.1 * maxnb;
    const int slots = ((int)std::ceil(v) + 31) / 32 * 32;
    return std::min(PIMD_SORT_CAP, std::max(32, slots));
}

// element (r, k) of an R x K operand in the tensor cores' K-major core-matrix layout
size_t cm_index_host(int r, int k, int K)
{
    return ((size_t)(r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// potentials evaluated on neighbour graphs (the network and the GFN head)
bool graph_pot(int pot) { return pot == PIMD_POT_MODEL || pot == PIMD_POT_GFN; }

// length of the graph-field-network parameter blob (layout in pimd.h)
size_t gfn_blob_len(int F, int L, int n_el)
{
    const size_t FF = (size_t)F * F;
    return (size_t)n_el * F + (size_t)F * NR + F + (size_t)L * (FF + F + 2 * FF + F + FF + F + FF + F + FF + F) + FF +
           F + F + 2;
}

struct Carve {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        off = (off + 255) & ~size_t(255);
        size_t o = off;
        off += bytes;
        return o;
    }
};

struct Offsets {
    size_t reps, bsys, ba_sys, mass, minv, atype, x0, cmat, cmatf, modes, rp_blocks, x, f, nbr, nnb, cell_start, cell_cnt,
        cell_atoms, cell_bs, G, dEdG, Eatom, V, W, q, p,
        fnm, Q, qpart, rep_blk0, step_cur, wbuf, vbuf, mom, md_hills, md_nhill, md_cv, md_vb, md_dvds, md_cvpart,
        md_virpart, md_grad, cand, ncand, xref, rebuild, ba_info, step, err, est, perm, tile_type, wts, wtc, wtc_vec, gfn_w,
        gfn_n, gfn_m, gfn_e, gfn_wtc, total;
};

int check_config(const pimd_config* cfg, std::string& e)
{
    if (!cfg) { e = "cfg is NULL"; return PIMD_ERR_INVALID_ARG; }
    if (!(cfg->dt_fs != 0.0) || !std::isfinite(cfg->dt_fs)) { e = "dt_fs must be finite and non-zero"; return PIMD_ERR_INVALID_ARG; }
    if (cfg->precision < 0 || cfg->precision > 2) { e = "unknown precision"; return PIMD_ERR_INVALID_ARG; }
    if (cfg->thermostat != 0 && cfg->thermostat != 1) { e = "thermostat must be 0 or 1"; return PIMD_ERR_INVALID_ARG; }
    if (cfg->nbr_algo < 0 || cfg->nbr_algo > 2) { e = "nbr_algo must be 0, 1 or 2"; return PIMD_ERR_INVALID_ARG; }
    if (!std::isfinite(cfg->nbr_skin_A)) { e = "nbr_skin_A must be finite"; return PIMD_ERR_INVALID_ARG; }
    if (cfg->transform != PIMD_TRANSFORM_NORMAL_MODES && cfg->transform != PIMD_TRANSFORM_STAGING)
        { e = "transform must be PIMD_TRANSFORM_NORMAL_MODES or PIMD_TRANSFORM_STAGING"; return PIMD_ERR_INVALID_ARG; }
    if (cfg->splitting != PIMD_OBABO && cfg->splitting != PIMD_BAOAB) { e = "splitting must be PIMD_OBABO or PIMD_BAOAB"; return PIMD_ERR_INVALID_ARG; }
    if (cfg->free_rp != PIMD_FREE_RP_EXACT && cfg->free_rp != PIMD_FREE_RP_CAYLEY) { e = "free_rp must be PIMD_FREE_RP_EXACT or PIMD_FREE_RP_CAYLEY"; return PIMD_ERR_INVALID_ARG; }
    if (cfg->deterministic != 0 && cfg->deterministic != 1) { e = "deterministic must be 0 or 1"; return PIMD_ERR_INVALID_ARG; }
    if (cfg->potential != PIMD_POT_MODEL && cfg->potential != PIMD_POT_HARMONIC && cfg->potential != PIMD_POT_GFN)
        { e = "unknown potential"; return PIMD_ERR_INVALID_ARG; }
    if (cfg->thermostat == 1 && !(cfg->gamma0_per_fs >= 0.0)) { e = "gamma0_per_fs must be >= 0"; return PIMD_ERR_INVALID_ARG; }
    if (cfg->thermostat == 1 && !(cfg->pile_lambda >= 0.0)) { e = "pile_lambda must be >= 0"; return PIMD_ERR_INVALID_ARG; }
    int mnb = cfg->max_neighbours == 0 ? 128 : cfg->max_neighbours;
    if (mnb < 32 || mnb > PIMD_MAX_NEIGHBOURS || mnb % 32) { e = "max_neighbours must be a multiple of 32 in [32, 256]"; return PIMD_ERR_INVALID_ARG; }
    if (cfg->potential == PIMD_POT_MODEL) {
        if (!(cfg->cutoff_A > 0.0)) { e = "cutoff_A must be > 0"; return PIMD_ERR_INVALID_ARG; }
        if (cfg->n_hidden < 1 || cfg->n_hidden > PIMD_MAX_LAYERS) { e = "n_hidden must be 1..4"; return PIMD_ERR_INVALID_ARG; }
        for (int l = 0; l < cfg->n_hidden; ++l) {
            if (cfg->widths[l] != cfg->widths[0]) { e = "hidden layers must share one width"; return PIMD_ERR_UNSUPPORTED; }
        }
        int w = cfg->widths[0];
        if (w != 64 && w != 128 && w != 256) { e = "hidden width must be 64, 128 or 256"; return PIMD_ERR_UNSUPPORTED; }
        if (cfg->precision == PIMD_BF16_TC && !network_tc_supported(w, cfg->n_hidden)) {
            e = "tensor-core network does not support this width"; return PIMD_ERR_UNSUPPORTED;
        }
    } else if (cfg->potential == PIMD_POT_GFN) {
        if (!(cfg->cutoff_A > 0.0)) { e = "cutoff_A must be > 0"; return PIMD_ERR_INVALID_ARG; }
        if (cfg->precision == PIMD_FP64) { e = "the GFN head runs in FP32 or BF16 precision"; return PIMD_ERR_UNSUPPORTED; }
        if (cfg->gfn_features != 32 && cfg->gfn_features != 64 && cfg->gfn_features != 128)
            { e = "gfn_features must be 32, 64 or 128"; return PIMD_ERR_UNSUPPORTED; }
        if (cfg->precision == PIMD_BF16_TC && cfg->gfn_features == 32)
            { e = "the tensor-core GFN head needs gfn_features 64 or 128"; return PIMD_ERR_UNSUPPORTED; }
        if (cfg->gfn_iterations < 0 || cfg->gfn_iterations > GFN_MAX_ITERS)
            { e = "gfn_iterations must be 0..8"; return PIMD_ERR_INVALID_ARG; }
    } else if (!(cfg->omega_harm >= 0.0)) {
        e = "omega_harm must be >= 0"; return PIMD_ERR_INVALID_ARG;
    }
    return PIMD_OK;
}

void nm_matrix(int P, double* C)
{
    for (int j = 0; j < P; ++j)
        for (int k = 0; k < P; ++k) {
            double v;
            if (k == 0) v = 1.0 / std::sqrt((double)P);
            else if (2 * k < P) v = std::sqrt(2.0 / P) * std::cos(2.0 * M_PI * j * k / P);
            else if (2 * k == P) v = ((j & 1) ? -1.0 : 1.0) / std::sqrt((double)P);
            else v = std::sqrt(2.0 / P) * std::sin(2.0 * M_PI * j * k / P);
            C[(size_t)j * P + k] = v;
        }
}

// staging transform as a matrix, x = S u: x_1 = u_1 and, for beads k >= 2,
// x_k = u_1 + sum_(j=k..P) ((k-1)/(j-1)) u_j (1-based; from the recursion
// x_k = u_k + ((k-1)/k) x_(k+1) + x_1/k with x_(P+1) = x_1). Staging forces
// are S^T f, the same product as the normal-mode forces C^T f.
void staging_matrix(int P, double* S)
{
    for (int j = 1; j <= P; ++j)
        for (int k = 1; k <= P; ++k) {
            double v = 0.0;
            if (k == 1) v = 1.0;
            else if (j >= 2 && j <= k) v = (double)(j - 1) / (k - 1);
            S[(size_t)(j - 1) * P + (k - 1)] = v;
        }
}

int make_build(const pimd_config* cfg, const pimd_replica_desc* reps, int n, Build& b, std::string& e)
{
    int rc = check_config(cfg, e);
    if (rc) return rc;
    if (!reps || n < 1) { e = "need at least one replica"; return PIMD_ERR_INVALID_ARG; }
    const int mnb = cfg->max_neighbours == 0 ? 128 : cfg->max_neighbours;
    (void)mnb;
    std::vector<HostRep> hr(n);
    long long B = 0, S = 0, NA = 0;
    std::vector<int> zs;
    for (int r = 0; r < n; ++r) {
        const pimd_replica_desc& d = reps[r];
        if (d.n_atoms < 1 || d.n_beads < 1 || d.n_beads > PIMD_MAX_BEADS) { e = "replica " + std::to_string(r) + ": bad N or P"; return PIMD_ERR_INVALID_ARG; }
        if (!d.Z || !d.x0) { e = "replica " + std::to_string(r) + ": Z and x0 are required"; return PIMD_ERR_INVALID_ARG; }
        if (!(d.T_K > 0.0) || !std::isfinite(d.T_K)) { e = "replica " + std::to_string(r) + ": T_K must be > 0"; return PIMD_ERR_INVALID_ARG; }
        const bool per = d.box[0] != 0.0 || d.box[1] != 0.0 || d.box[2] != 0.0;
        if (per) {
            for (int a = 0; a < 3; ++a)
                if (!(d.box[a] > 0.0)) { e = "replica " + std::to_string(r) + ": box lengths must all be > 0 or all 0"; return PIMD_ERR_INVALID_ARG; }
            if (graph_pot(cfg->potential) && std::min(d.box[0], std::min(d.box[1], d.box[2])) < 2.0 * cfg->cutoff_A) {
                e = "replica " + std::to_string(r) + ": periodic box shorter than twice the cutoff"; return PIMD_ERR_INVALID_ARG;
            }
        }
        HostRep& h = hr[r];
        h.N = d.n_atoms; h.P = d.n_beads; h.T = d.T_K; h.seed = d.seed;
        for (int a = 0; a < 3; ++a) h.box[a] = d.box[a];
        h.Z.assign(d.Z, d.Z + d.n_atoms);
        h.x0.assign(d.x0, d.x0 + 3 * (size_t)d.n_atoms);
        h.mass.resize(d.n_atoms);
        for (int i = 0; i < d.n_atoms; ++i) {
            double m = d.mass ? d.mass[i] : default_mass(h.Z[i]);
            if (!(m > 0.0)) { e = "replica " + std::to_string(r) + ": no mass for element " + std::to_string(h.Z[i]); return PIMD_ERR_INVALID_ARG; }
            if (!std::isfinite(h.x0[3 * i]) || !std::isfinite(h.x0[3 * i + 1]) || !std::isfinite(h.x0[3 * i + 2])) {
                e = "replica " + std::to_string(r) + ": non-finite x0"; return PIMD_ERR_INVALID_ARG;
            }
            h.mass[i] = m;
            zs.push_back(h.Z[i]);
        }
        B += (long long)d.n_atoms * d.n_beads;
        S += d.n_beads;
        NA += d.n_atoms;
    }
    if (3 * B >= (1ll << 31) - 1024) { e = "too many bead-atoms"; return PIMD_ERR_INVALID_ARG; }
    std::sort(zs.begin(), zs.end());
    zs.erase(std::unique(zs.begin(), zs.end()), zs.end());
    if ((int)zs.size() > PIMD_MAX_ELEMENTS) { e = "more than 8 elements"; return PIMD_ERR_UNSUPPORTED; }
    b.typeZ = zs;
    b.R = n; b.S = (int)S; b.B = (int)B; b.NA = (int)NA;
    if (cfg->metad && cfg->metad->cv != PIMD_CV_NONE) {
        const pimd_metad_desc* m = cfg->metad;
        int minN = 1 << 30, maxP = 1;
        for (int r = 0; r < n; ++r) { minN = std::min(minN, hr[r].N); maxP = std::max(maxP, hr[r].P); }
        if (m->cv != PIMD_CV_DISTANCES && m->cv != PIMD_CV_XRD) { e = "metad: unknown cv"; return PIMD_ERR_INVALID_ARG; }
        if (m->cv == PIMD_CV_DISTANCES) {
            if (m->n_terms < 1 || m->n_terms > 8) { e = "metad: n_terms must be 1..8"; return PIMD_ERR_INVALID_ARG; }
            for (int t = 0; t < m->n_terms; ++t)
                if (m->term_i[t] < 0 || m->term_j[t] < 0 || m->term_i[t] >= minN || m->term_j[t] >= minN ||
                    m->term_i[t] == m->term_j[t] || !std::isfinite(m->term_c[t])) {
                    e = "metad: term " + std::to_string(t) + " has bad atom indices or coefficient"; return PIMD_ERR_INVALID_ARG;
                }
        } else {
            if (!(m->xrd_Q > 0.0) || !std::isfinite(m->xrd_Q)) { e = "metad: xrd_Q must be > 0"; return PIMD_ERR_INVALID_ARG; }
            for (size_t t = 0; t < zs.size(); ++t)
                if (!std::isfinite(m->xrd_f[t])) { e = "metad: xrd_f must be finite"; return PIMD_ERR_INVALID_ARG; }
        }
        if (!(m->height_eV >= 0.0) || !(m->sigma > 0.0) || !(m->bias_factor > 1.0) || m->stride < 1)
            { e = "metad: need height_eV >= 0, sigma > 0, bias_factor > 1, stride >= 1"; return PIMD_ERR_INVALID_ARG; }
        if (m->max_hills < maxP || m->max_hills > (1 << 24)) { e = "metad: max_hills must be in [max P, 2^24]"; return PIMD_ERR_INVALID_ARG; }
    }

    // normal-mode matrices, one per distinct P
    std::map<int, int> cm_off;
    for (int r = 0; r < n; ++r) {
        int P = hr[r].P;
        if (!cm_off.count(P)) {
            cm_off[P] = (int)b.cmat.size();
            b.cmat.resize(b.cmat.size() + (size_t)P * P);
            if (cfg->transform == PIMD_TRANSFORM_STAGING)
                staging_matrix(P, b.cmat.data() + cm_off[P]);
            else
                nm_matrix(P, b.cmat.data() + cm_off[P]);
        }
    }
    const int rp_threads = 256;
    int ba0 = 0, bs0 = 0, atom0 = 0, mode0 = 0;
    for (int r = 0; r < n; ++r) {
        const HostRep& h = hr[r];
        Rep rp;
        std::memset(&rp, 0, sizeof(rp));
        rp.N = h.N; rp.P = h.P; rp.ba0 = ba0; rp.bs0 = bs0; rp.atom0 = atom0; rp.cmat = cm_off[h.P]; rp.mode0 = mode0;
        rp.periodic = (h.box[0] != 0.0) ? 1 : 0;
        if (rp.periodic) b.periodic_any = true;
        for (int a = 0; a < 3; ++a) {
            rp.L[a] = rp.periodic ? h.box[a] : 0.0;
            rp.invL[a] = rp.periodic ? 1.0 / h.box[a] : 0.0;
            rp.Lf[a] = (float)rp.L[a];
            rp.invLf[a] = (float)rp.invL[a];
            rp.Llo[a] = (float)(rp.L[a] - (double)rp.Lf[a]);
        }
        rp.kT_md = h.P * KB * h.T / MVV2E;
        rp.seed = h.seed;
        rp.noise_atom0 = 0;
        rp.noise_N = h.N;
        b.repT.push_back(h.T);
        // Verlet skin of the candidate lists: at most 0.9 of the room between
        // r_c and half the box (unique minimum images), off below 0.05 A
        const bool auto_skin = cfg->nbr_skin_A < 0.0;
        auto set_skin = [&](double sk) {
            if (rp.periodic)
                sk = std::min(sk, 0.9 * (0.5 * std::min(std::min(h.box[0], h.box[1]), h.box[2]) - cfg->cutoff_A));
            if (sk < 0.05) sk = 0.0;
            rp.skin = (float)sk;
            const double rcs = cfg->cutoff_A + sk;
            rp.rcs2 = (float)(rcs * rcs);
        };
        if (graph_pot(cfg->potential))
            // auto: 1.5 A for replicas of >= 256 atoms (small ones scan all
            // atoms faster than they would check and filter candidates)
            set_skin(auto_skin ? (h.N >= 256 ? 1.5 : 0.0) : cfg->nbr_skin_A);
        // cell lists: >= 3 cells per side with edge >= cutoff + skin (1e-5
        // margin against rounding of the FP32 cell coordinate)
        if (rp.periodic && graph_pot(cfg->potential) && cfg->nbr_algo != 1) {
            int nc[3];
            for (int a = 0; a < 3; ++a)
                nc[a] = (int)std::floor(h.box[a] / ((cfg->cutoff_A + rp.skin) * (1.0 + 1e-5)));
            const long long ncell = (long long)nc[0] * nc[1] * nc[2];
            // auto: cells when the stencil scan (+ sort) beats scanning the bead
            const double warp_iter_cells = 27.0 * h.N / std::max(1ll, ncell) / 32.0 + 12.0;
            const double warp_iter_all = h.N / 32.0;
            const bool pays = cfg->nbr_algo == 2 || warp_iter_cells < 0.8 * warp_iter_all;
            if (nc[0] >= 3 && nc[1] >= 3 && nc[2] >= 3 && ncell <= 16384 && pays) {
                for (int a = 0; a < 3; ++a) rp.nc[a] = nc[a];
                rp.ncells = nc[0] * nc[1] * nc[2];
                rp.cell0 = b.total_cells;
                b.total_cells += rp.ncells * h.P;
                b.max_cells = std::max(b.max_cells, rp.ncells);
                for (int k = 0; k < h.P; ++k) b.cell_bs.push_back(bs0 + k);
            }
        }
        if (rp.skin > 0.0f) b.any_skin = true;
        b.max_skin = std::max(b.max_skin, (double)rp.skin);
        b.reps.push_back(rp);
        {
            double est = h.N - 1.0;
            if (rp.periodic)
                est = std::min(est, h.N / (h.box[0] * h.box[1] * h.box[2]) * 4.0 / 3.0 * M_PI * cfg->cutoff_A *
                                        cfg->cutoff_A * cfg->cutoff_A);
            b.nb_est += est * h.N * h.P;
        }
        const double wP = h.P * KB * h.T / HBAR;
        // durations of the A and O sub-steps: OBABO A(dt) O(dt/2), BAOAB A(dt/2) O(dt)
        const double hA = cfg->splitting == PIMD_BAOAB ? 0.5 * cfg->dt_fs : cfg->dt_fs;
        const double hO = cfg->splitting == PIMD_BAOAB ? cfg->dt_fs : 0.5 * cfg->dt_fs;
        for (int k = 0; k < h.P; ++k) {
            Mode md;
            std::memset(&md, 0, sizeof(md));
            const bool stg = cfg->transform == PIMD_TRANSFORM_STAGING;
            md.w = stg ? (k == 0 ? 0.0 : wP) : 2.0 * wP * std::sin(k * M_PI / h.P);
            md.mfac = (stg && k >= 1) ? (k + 1.0) / k : 1.0;
            // column sums of the transform (centroid) and the total-force factor
            md.cs = stg ? (k == 0 ? (double)h.P : 0.5 * (k + 1)) : (k == 0 ? std::sqrt((double)h.P) : 0.0);
            md.ft = stg ? 1.0 : std::sqrt((double)h.P);
            if (cfg->free_rp == PIMD_FREE_RP_CAYLEY) {
                // Cayley transform of hA L_k: a rotation of the scaled phase
                // plane with cos = (1 - a) / (1 + a), sin = w hA / (1 + a),
                // a = (w hA / 2)^2
                const double a = 0.25 * md.w * md.w * hA * hA;
                md.cw = (1.0 - a) / (1.0 + a);
                md.sw = md.w * hA / (1.0 + a);
            } else {
                md.cw = std::cos(md.w * hA);
                md.sw = std::sin(md.w * hA);
            }
            const double gam = (k == 0) ? cfg->gamma0_per_fs : 2.0 * cfg->pile_lambda * md.w;
            md.c1 = std::exp(-hO * gam);
            md.c2 = std::sqrt(1.0 - md.c1 * md.c1);
            md.c1m1 = (float)std::expm1(-hO * gam);
            md.c1p1 = (float)(md.c1 + 1.0);
            md.sw_w = md.w > 0.0 ? md.sw / md.w : 0.0;
            md.wsw = md.w * md.sw;
            md.smf = std::sqrt(md.mfac);
            md.imf = 1.0 / md.mfac;
            b.modes.push_back(md);
        }
        for (int k = 0; k < h.P; ++k) {
            BeadSys s;
            s.ba0 = ba0 + k * h.N; s.N = h.N; s.rep = r; s.bead = k;
            b.bsys.push_back(s);
            for (int i = 0; i < h.N; ++i) b.ba_sys.push_back(bs0 + k);
        }
        for (int i = 0; i < h.N; ++i) {
            b.mass.push_back(h.mass[i]);
            b.atype.push_back((int)(std::lower_bound(zs.begin(), zs.end(), h.Z[i]) - zs.begin()));
            for (int a = 0; a < 3; ++a) b.x0.push_back(h.x0[3 * i + a]);
        }
        const int T = rp_threads / h.P;
        b.rep_blk0.push_back((int)b.rp_blocks.size());
        for (int first = 0; first < 3 * h.N; first += T) b.rp_blocks.push_back(make_int2(r, first));
        ba0 += h.N * h.P; bs0 += h.P; atom0 += h.N; mode0 += h.P;
    }
    b.rep_blk0.push_back((int)b.rp_blocks.size());
    b.nb_est /= std::max(1, b.B);
    // network rows grouped by element type, each group padded to 128 rows.
    // Large BF16 workloads split their bead-atoms into parts of whole
    // bead-systems (the branches of an overlapped step); each part has its
    // own element groups and tiles.
    if (cfg->potential == PIMD_POT_MODEL) {
        // parts: whole bead-systems; the first part takes 3/8 of the
        // bead-atoms and the others share the rest evenly (boundaries at the
        // nearest bead-system). The first part's forward runs alone, so a
        // smaller first part starts the overlap sooner (ice, two parts: a
        // first part of 8-14 of the 32 beads 0.4015-0.402 ms per step,
        // halves 0.404-0.405 ms)
        std::vector<int> cut = {0};
        if (cfg->precision == PIMD_BF16_TC && b.B >= 16384 && b.S >= OVERLAP_PARTS) {
            for (int k = 1; k < OVERLAP_PARTS; ++k) {
                const long long want =
                    (long long)b.B * (3 * (OVERLAP_PARTS - 1) + 5 * (k - 1)) / (8 * (OVERLAP_PARTS - 1));
                int best = 0;
                for (const BeadSys& sy : b.bsys)
                    if (std::llabs(sy.ba0 - want) < std::llabs(best - want)) best = sy.ba0;
                if (best > cut.back()) cut.push_back(best);
            }
        }
        cut.push_back(b.B);
        const int parts = (int)cut.size() - 1;
        for (int pt = 0; pt < parts; ++pt) {
            const int lo = cut[pt], hi = cut[pt + 1];
            if (parts > 1) b.part_tile.push_back((int)b.tile_type.size());
            std::vector<std::vector<int>> rows(zs.size());
            for (int r = 0; r < n; ++r) {
                const Rep& rp = b.reps[r];
                for (int k = 0; k < rp.P; ++k)
                    for (int i = 0; i < rp.N; ++i) {
                        const int ba = rp.ba0 + k * rp.N + i;
                        if (ba >= lo && ba < hi) rows[b.atype[rp.atom0 + i]].push_back(ba);
                    }
            }
            for (size_t t = 0; t < zs.size(); ++t) {
                std::vector<int> v = rows[t];
                std::sort(v.begin(), v.end());
                size_t padded = (v.size() + TILE_ROWS - 1) / TILE_ROWS * TILE_ROWS;
                for (size_t q = 0; q < padded; ++q) b.perm.push_back(q < v.size() ? v[q] : -1);
                for (size_t q = 0; q < padded / TILE_ROWS; ++q) b.tile_type.push_back((int)t);
            }
        }
        if (parts > 1) {
            b.part_ba = cut;
            b.part_tile.push_back((int)b.tile_type.size());
        }
        b.rows_pad = (int)b.perm.size();
        b.blob = blob_elems(cfg->n_hidden, cfg->widths);
        if (cfg->precision == PIMD_BF16_TC) {
            b.wtc_bytes = tc_weight_bytes(cfg->widths[0], cfg->n_hidden);
            b.wtc_vec = (size_t)cfg->n_hidden * cfg->widths[0] + cfg->widths[0] + 2 * ND + 4;
        }
    }
    if (cfg->potential == PIMD_POT_GFN)
        b.gfn_params = gfn_blob_len(cfg->gfn_features, cfg->gfn_iterations, (int)zs.size());
    return PIMD_OK;
}

Offsets layout(const pimd_config* cfg, const Build& b)
{
    const int mnb = cfg->max_neighbours == 0 ? 128 : cfg->max_neighbours;
    const size_t rs = cfg->precision == PIMD_FP64 ? sizeof(double) : sizeof(float);
    const size_t v4 = cfg->precision == PIMD_FP64 ? sizeof(Dbl4) : sizeof(float4);
    Carve c;
    Offsets o;
    o.reps = c.take(sizeof(Rep) * b.R);
    o.bsys = c.take(sizeof(BeadSys) * b.S);
    o.ba_sys = c.take(sizeof(int) * b.B);
    o.ba_info = c.take(sizeof(int4) * b.B);
    o.mass = c.take(sizeof(double) * b.NA);
    o.minv = c.take(sizeof(double2) * b.NA);
    o.atype = c.take(sizeof(int) * b.NA);
    o.x0 = c.take(sizeof(double) * 3 * (size_t)b.NA);
    o.cmat = c.take(sizeof(double) * b.cmat.size());
    o.cmatf = c.take(sizeof(float) * b.cmat.size());
    o.modes = c.take(sizeof(Mode) * b.modes.size());
    o.rp_blocks = c.take(sizeof(int2) * b.rp_blocks.size());
    o.x = c.take(v4 * b.B);
    o.f = c.take(v4 * b.B);
    const bool model = cfg->potential == PIMD_POT_MODEL;
    o.nbr = c.take(graph_pot(cfg->potential) ? sizeof(int) * (size_t)b.B * mnb : 0);
    o.nnb = c.take(sizeof(int) * b.B);
    o.cell_start = c.take(sizeof(int) * (size_t)b.total_cells);
    o.cell_cnt = c.take(sizeof(int) * (size_t)b.total_cells);
    o.cell_atoms = c.take(b.total_cells ? sizeof(int) * (size_t)b.B : 0);
    o.cell_bs = c.take(sizeof(int) * b.cell_bs.size());
    o.G = c.take(model ? rs * (size_t)b.B * ND : 0);
    o.dEdG = c.take(model ? rs * (size_t)b.B * ND : 0);
    o.Eatom = c.take(rs * b.B);
    o.V = c.take(sizeof(double) * b.S);
    o.W = c.take(sizeof(double) * 9 * (size_t)b.S);
    o.q = c.take(sizeof(double) * 3 * (size_t)b.B);
    o.p = c.take(sizeof(double) * 3 * (size_t)b.B);
    o.fnm = c.take(sizeof(double) * 3 * (size_t)b.B);
    o.Q = c.take(sizeof(double) * b.R);
    o.qpart = c.take(sizeof(double) * 3 * b.rp_blocks.size());
    o.rep_blk0 = c.take(sizeof(int) * b.rep_blk0.size());
    o.step_cur = c.take(sizeof(unsigned long long));
    o.wbuf = c.take(rs * 9 * (size_t)b.B);
    o.vbuf = c.take(cfg->deterministic && model ? v4 * (size_t)b.B * mnb : 0);
    o.mom = c.take(model && cfg->precision != PIMD_FP64 ? sizeof(float4) * moment_elems_per_atom() * (size_t)b.B : 0);
    {
        const size_t mc = b.any_skin ? (size_t)max_candidates(mnb, cfg->cutoff_A, b.max_skin) : 0;
        o.cand = c.take(sizeof(int) * (size_t)b.B * mc);
        o.ncand = c.take(mc ? sizeof(int) * (size_t)b.B : 0);
        o.xref = c.take(mc ? sizeof(float4) * (size_t)b.B : 0);
        o.rebuild = c.take(mc ? sizeof(int) * (size_t)b.S : 0);
    }
    {
        const bool md = cfg->metad && cfg->metad->cv != PIMD_CV_NONE;
        int maxN = 1;
        for (const Rep& rp : b.reps) maxN = std::max(maxN, rp.N);
        const size_t nt = md ? (size_t)metad_tiles(maxN) : 0;
        o.md_hills = c.take(md ? sizeof(double2) * (size_t)b.R * cfg->metad->max_hills : 0);
        o.md_nhill = c.take(md ? sizeof(int) * b.R : 0);
        o.md_cv = c.take(md ? sizeof(double) * b.S : 0);
        o.md_vb = c.take(md ? sizeof(double) * b.S : 0);
        o.md_dvds = c.take(md ? sizeof(double) * b.S : 0);
        o.md_cvpart = c.take(sizeof(double) * b.S * nt);
        o.md_virpart = c.take(sizeof(double) * 9 * b.S * nt);
        o.md_grad = c.take(md ? v4 * (size_t)b.B * (cfg->metad->cv == PIMD_CV_XRD ? MD_SLICES : 1) : 0);
    }
    o.step = c.take(sizeof(unsigned long long));
    o.err = c.take(sizeof(DevErr));
    o.est = c.take(sizeof(double) * EST_STRIDE * b.R);
    o.perm = c.take(sizeof(int) * b.perm.size());
    o.tile_type = c.take(sizeof(int) * b.tile_type.size());
    o.wts = c.take(rs * b.blob * b.typeZ.size());
    o.wtc = c.take(b.wtc_bytes * b.typeZ.size());
    o.wtc_vec = c.take(sizeof(float) * b.wtc_vec * b.typeZ.size());
    {
        const bool gfn = cfg->potential == PIMD_POT_GFN;
        const size_t F = gfn ? (size_t)cfg->gfn_features : 0;
        o.gfn_w = c.take(sizeof(float) * b.gfn_params);
        o.gfn_n = c.take(sizeof(float) * F * b.B);
        o.gfn_m = c.take(sizeof(float) * F * b.B);
        o.gfn_e = c.take(sizeof(float) * F * (size_t)b.B * mnb);
        o.gfn_wtc = c.take(gfn && cfg->precision == PIMD_BF16_TC ? gfn_tc_image_bytes(cfg->gfn_features, cfg->gfn_iterations) : 0);
    }
    o.total = c.take(0) + 256;
    return o;
}

}  // namespace

void pimd::set_thread_error(const std::string& msg) { g_tls_error = msg; }

struct pimd_ctx {
    Dev d;
    pimd_config cfg;
    cudaStream_t st = nullptr;
    Build build;
    DescParams<float> dpf;
    DescParams<double> dpd;
    bool weights_set = false, forces_valid = false, beads_current = true;
    unsigned long long step_host = 0;
    cudaGraphExec_t g1 = nullptr, g8 = nullptr;   // 1 and 8 steps, no stage markers
    cudaGraphExec_t g1t = nullptr;                 // 1 step with the stage markers (timing contexts)
    bool stage_timing = true;                      // mark the last step of each pimd_step call
    bool overlap = true;                           // overlapped parts in unmarked step graphs
    cudaStream_t cap = nullptr;
    cudaStream_t capx[MAX_PARTS] = {};             // branches 1.. of an overlapped step (capture only)
    cudaEvent_t ev_fwd[MAX_PARTS] = {}, ev_end[MAX_PARTS] = {};
    bool branches_ready = false;
    cudaEvent_t ev[PIMD_N_STAGES + 1] = {};
    bool stepped = false;
    std::string err;
    unsigned char* ws = nullptr;
};

namespace {

void drop_graphs(pimd_ctx* c)
{
    if (c->g1) { cudaGraphExecDestroy(c->g1); c->g1 = nullptr; }
    if (c->g8) { cudaGraphExecDestroy(c->g8); c->g8 = nullptr; }
    if (c->g1t) { cudaGraphExecDestroy(c->g1t); c->g1t = nullptr; }
}

int fail(pimd_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    else g_tls_error = msg;
    return code;
}

int cuda_check(pimd_ctx* c, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return PIMD_OK;
    // report, and clear the runtime's last-error slot so that an error that
    // is not sticky does not surface in the caller's next CUDA call
    cudaGetLastError();
    return fail(c, PIMD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

const void* dparams(const pimd_ctx* c)
{
    return c->d.precision == PIMD_FP64 ? (const void*)&c->dpd : (const void*)&c->dpf;
}

// event i marks the start of stage i (i = PIMD_N_STAGES: end of the step)
void mark(pimd_ctx* c, int i, cudaStream_t st, bool timed)
{
    // external record nodes: the events fire when the captured graph runs
    if (timed && c->ev[i]) cudaEventRecordWithFlags(c->ev[i], st, cudaEventRecordExternal);
}

// the model's force evaluation can run as overlapping branches (parts of the
// bead-atoms on the BF16 moment path with tensor-core network tiles)
bool splits_forces(const pimd_ctx* c)
{
    const Dev& d = c->d;
    return d.potential == PIMD_POT_MODEL && d.n_parts > 1 && moment_fast_path(d, dparams(c)) &&
           network_tiles_available(d);
}

// zeroed: the ring start of this step has already cleared the forces, the
// per-bead virials and energies
// branch: the step may run the force evaluation as two overlapping branches
// (captured graphs without stage markers)
void eval_forces(pimd_ctx* c, cudaStream_t st, bool timed = false, bool deposit = false, bool zeroed = false,
                 bool branch = false, int step_offset = 0)
{
    Dev& d = c->d;
    const size_t v4 = d.precision == PIMD_FP64 ? sizeof(Dbl4) : sizeof(float4);
    const bool summed = d.potential == PIMD_POT_MODEL && adjoint_sums_energy(d, dparams(c));
    if (!zeroed) {
        cudaMemsetAsync(d.f, 0, v4 * d.B, st);
        cudaMemsetAsync(d.W, 0, sizeof(double) * 9 * d.S, st);
        if (summed) cudaMemsetAsync(d.V, 0, sizeof(double) * d.S, st);
    }
    mark(c, PIMD_STAGE_NEIGHBOURS, st, timed);
    if (d.potential == PIMD_POT_HARMONIC) {
        launch_harmonic(d, st);
        mark(c, PIMD_STAGE_DESCRIPTORS, st, timed);
        mark(c, PIMD_STAGE_NETWORK, st, timed);
        mark(c, PIMD_STAGE_ADJOINT, st, timed);
    } else if (d.potential == PIMD_POT_GFN) {
        // direct forces: the whole head runs in the network stage
        launch_neighbours(d, st);
        mark(c, PIMD_STAGE_DESCRIPTORS, st, timed);
        mark(c, PIMD_STAGE_NETWORK, st, timed);
        if (d.gfn_wtc) launch_gfn_tc(d, st);
        else launch_gfn(d, st);
        mark(c, PIMD_STAGE_ADJOINT, st, timed);
    } else if (branch && splits_forces(c) && c->branches_ready) {
        // the parts as overlapping branches: part k's forward starts when
        // part k-1's forward ends, and each part's network (latency-bound,
        // short) and adjoint follow its forward on its own branch, beside the
        // next parts' forwards; every kernel's last wave is filled by another
        // branch. All forwards are captured before the networks: when part
        // k-1's forward ends, part k's forward and part k-1's network are
        // both ready, and the graph launches them in capture order (network
        // first cost 10 us per ice step)
        const void* dp = dparams(c);
        launch_neighbours(d, st);
        for (int k = 0; k < d.n_parts; ++k) {
            cudaStream_t sk = k == 0 ? st : c->capx[k];
            if (k > 0) cudaStreamWaitEvent(sk, c->ev_fwd[k - 1], 0);
            launch_descriptors_range(d, dp, d.part_ba[k], d.part_ba[k + 1], sk);
            if (k + 1 < d.n_parts) cudaEventRecord(c->ev_fwd[k], sk);
        }
        for (int k = 0; k < d.n_parts; ++k) {
            cudaStream_t sk = k == 0 ? st : c->capx[k];
            launch_network_tiles(d, d.part_tile[k], d.part_tile[k + 1] - d.part_tile[k], sk, true);
            launch_adjoint_range(d, dp, d.part_ba[k], d.part_ba[k + 1], sk);
        }
        for (int k = 1; k < d.n_parts; ++k) {
            cudaEventRecord(c->ev_end[k], c->capx[k]);
            cudaStreamWaitEvent(st, c->ev_end[k], 0);
        }
        if (d.deterministic) launch_force_gather(d, st);
    } else {
        launch_neighbours(d, st);
        mark(c, PIMD_STAGE_DESCRIPTORS, st, timed);
        launch_descriptors(d, dparams(c), st);
        mark(c, PIMD_STAGE_NETWORK, st, timed);
        if (d.precision == PIMD_BF16_TC) launch_network_tc(d, st);
        else launch_network_fp(d, st);
        mark(c, PIMD_STAGE_ADJOINT, st, timed);
        launch_adjoint(d, dparams(c), st);
        if (d.deterministic) launch_force_gather(d, st);
    }
    mark(c, PIMD_STAGE_ENERGY, st, timed);
    if (!summed) launch_energy_reduce(d, st);
    if (d.metad.cv) launch_metad(d, deposit, st, step_offset);   // bias on every bead (and hills on deposition steps)
}
void eval_forces(pimd_ctx* c) { eval_forces(c, c->st); }

void one_step(pimd_ctx* c, cudaStream_t st, bool timed)
{
    mark(c, PIMD_STAGE_RING_START, st, timed);
    launch_rp_start(c->d, st);   // also clears f, W and V for the force evaluation
    eval_forces(c, st, timed, true, true, !timed && c->overlap);
    mark(c, PIMD_STAGE_RING_FINISH, st, timed);
    launch_rp_finish(c->d, true, st);   // also advances the step counter
    if (c->d.deterministic) launch_heat_sum(c->d, 0, st);
    mark(c, PIMD_N_STAGES, st, timed);
}

// n >= 2 steps in one launch: one ring start, then per step the force
// evaluation and, between steps, the fused ring finish + next ring start;
// the last step ends with a plain ring finish, so the state at the end of
// the launch is the state after a ring finish, as with single steps
void fused_steps(pimd_ctx* c, cudaStream_t st, int n)
{
    Dev& d = c->d;
    launch_rp_start(d, st, 0);
    for (int j = 0; j < n; ++j) {
        eval_forces(c, st, false, true, true, c->overlap, j);
        if (j + 1 < n)
            launch_rp_finish_start(d, j, (j + 1) & 1, st);
        else
            launch_rp_finish(d, true, st, j);
        if (d.deterministic) launch_heat_sum(d, j & 1, st);
    }
}

int refresh_forces(pimd_ctx* c)
{
    if (!c->beads_current) {
        launch_beads(c->d, c->st);
        c->beads_current = true;
    }
    eval_forces(c);
    launch_rp_finish(c->d, false, c->st);
    c->forces_valid = true;
    return cuda_check(c, cudaGetLastError(), "force evaluation launch");
}

// Graphs are recorded on a private stream (the caller's stream may be the
// legacy default stream, which cannot be captured) and launched on the
// context stream.
int capture(pimd_ctx* c, int nsteps, bool marked, cudaGraphExec_t* out)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaSuccess;
    if (!c->cap) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaStreamCreateWithFlags");
    if (c->d.n_parts > 1 && !c->branches_ready) {
        for (int k = 0; k < c->d.n_parts && e == cudaSuccess; ++k) {
            if (k > 0) e = cudaStreamCreateWithFlags(&c->capx[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fwd[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_end[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_check(c, e, "branch streams");
        c->branches_ready = true;
    }
    e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaStreamBeginCapture");
    if (nsteps >= 2 && !marked)
        fused_steps(c, c->cap, nsteps);
    else
        for (int s = 0; s < nsteps; ++s) one_step(c, c->cap, marked && s == nsteps - 1);
    e = cudaStreamEndCapture(c->cap, &g);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return cuda_check(c, e, "cudaGraphInstantiate");
}

int device_errors(pimd_ctx* c)
{
    DevErr h;
    cudaError_t e = cudaMemcpyAsync(&h, c->d.err, sizeof(DevErr), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_check(c, e, "synchronise");
    if (h.flags) {
        cudaMemsetAsync(c->d.err, 0, sizeof(DevErr), c->st);
        cudaStreamSynchronize(c->st);
        if (h.flags & ERR_NBR_OVERFLOW)
            return fail(c, PIMD_ERR_NBR_OVERFLOW, "neighbour list overflow: an atom has " + std::to_string(h.max_nbr) +
                                                      " neighbours, max_neighbours is " + std::to_string(c->d.maxnb));
        if (h.flags & ERR_NONFINITE) return fail(c, PIMD_ERR_NONFINITE, "non-finite forces");
        if (h.flags & ERR_TIMEOUT) return fail(c, PIMD_ERR_TIMEOUT, "device wait timed out");
        if (h.flags & ERR_METAD_FULL) return fail(c, PIMD_ERR_METAD_FULL, "metadynamics hill capacity exhausted");
    }
    return PIMD_OK;
}

template <typename T>
int upload(pimd_ctx* c, void* dst, const std::vector<T>& v)
{
    if (v.empty()) return PIMD_OK;
    return cuda_check(c, cudaMemcpyAsync(dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, c->st),
                      "upload");
}

}  // namespace

namespace {
int check_replica(pimd_ctx* c, int replica)
{
    if (replica < 0 || replica >= c->d.R) return fail(c, PIMD_ERR_INVALID_ARG, "replica out of range");
    return PIMD_OK;
}
}  // namespace

extern "C" {

int pimd_abi_version(void) { return PIMD_ABI_VERSION; }

int pimd_workspace_size(const pimd_config* cfg, const pimd_replica_desc* reps, int n_reps, size_t* bytes)
{
    if (!bytes) return fail(nullptr, PIMD_ERR_INVALID_ARG, "bytes is NULL");
    Build b;
    std::string e;
    int rc = make_build(cfg, reps, n_reps, b, e);
    if (rc) return fail(nullptr, rc, e);
    *bytes = layout(cfg, b).total;
    return PIMD_OK;
}

int pimd_create(const pimd_config* cfg, const pimd_replica_desc* reps, int n_reps, void* workspace,
                size_t ws_bytes, pimd_ctx** out)
{
    if (!out) return fail(nullptr, PIMD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    pimd_ctx* c = new (std::nothrow) pimd_ctx();
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "host allocation failed");
    std::string e;
    int rc = make_build(cfg, reps, n_reps, c->build, e);
    if (rc) { delete c; return fail(nullptr, rc, e); }
    const Build& b = c->build;
    Offsets o = layout(cfg, b);
    if (!workspace) { delete c; return fail(nullptr, PIMD_ERR_INVALID_ARG, "workspace is NULL"); }
    if (((uintptr_t)workspace & 255u) != 0) { delete c; return fail(nullptr, PIMD_ERR_INVALID_ARG, "workspace must be 256-byte aligned"); }
    if (ws_bytes < o.total) {
        delete c;
        return fail(nullptr, PIMD_ERR_WORKSPACE_TOO_SMALL,
                    "workspace has " + std::to_string(ws_bytes) + " bytes, needs " + std::to_string(o.total));
    }
    c->cfg = *cfg;
    c->st = (cudaStream_t)cfg->stream;
    if (cfg->timing) {
        for (int i = 0; i <= PIMD_N_STAGES; ++i) {
            if (cudaEventCreate(&c->ev[i]) != cudaSuccess) {
                for (int k = 0; k < i; ++k) cudaEventDestroy(c->ev[k]);
                delete c;
                return fail(nullptr, PIMD_ERR_CUDA, "cudaEventCreate failed");
            }
        }
    }
    c->ws = (unsigned char*)workspace;
    Dev& d = c->d;
    unsigned char* w = c->ws;
    d.R = b.R; d.S = b.S; d.B = b.B; d.NA = b.NA;
    for (const Rep& rp : b.reps) d.max_N = std::max(d.max_N, rp.N);
    d.maxnb = cfg->max_neighbours == 0 ? 128 : cfg->max_neighbours;
    d.precision = cfg->precision;
    d.periodic_any = b.periodic_any;
    d.reps = (Rep*)(w + o.reps);
    d.bsys = (BeadSys*)(w + o.bsys);
    d.ba_sys = (int*)(w + o.ba_sys);
    d.ba_info = (int4*)(w + o.ba_info);
    d.mass = (double*)(w + o.mass);
    d.minv = (double2*)(w + o.minv);
    d.atype = (int*)(w + o.atype);
    d.x0 = (double*)(w + o.x0);
    d.cmat = (double*)(w + o.cmat);
    d.cmatf = (float*)(w + o.cmatf);
    d.modes = (Mode*)(w + o.modes);
    d.rp_blocks = (int2*)(w + o.rp_blocks);
    d.n_rp_blocks = (int)b.rp_blocks.size();
    for (const Rep& rp : b.reps)
        if (rp.P <= 64) d.rp_stage_P = std::max(d.rp_stage_P, rp.P);
    d.unit_mfac = 1;
    for (const Mode& md : b.modes)
        if (md.mfac != 1.0 || md.imf != 1.0 || md.smf != 1.0) d.unit_mfac = 0;
    d.rp_threads = 256;
    d.x = w + o.x;
    d.f = w + o.f;
    d.nbr = (int*)(w + o.nbr);
    d.nnb = (int*)(w + o.nnb);
    d.cell_start = (int*)(w + o.cell_start);
    d.cell_cnt = (int*)(w + o.cell_cnt);
    d.cell_atoms = (int*)(w + o.cell_atoms);
    d.cell_bs = (int*)(w + o.cell_bs);
    d.n_cell_bs = (int)b.cell_bs.size();
    d.max_cells = b.max_cells;
    d.G = w + o.G;
    d.dEdG = w + o.dEdG;
    d.Eatom = w + o.Eatom;
    d.V = (double*)(w + o.V);
    d.W = (double*)(w + o.W);
    d.q = (double*)(w + o.q);
    d.p = (double*)(w + o.p);
    d.fnm = (double*)(w + o.fnm);
    d.Q = (double*)(w + o.Q);
    d.qpart = (double*)(w + o.qpart);
    d.rep_blk0 = (int*)(w + o.rep_blk0);
    d.step_cur = (unsigned long long*)(w + o.step_cur);
    d.wbuf = w + o.wbuf;
    d.vbuf = w + o.vbuf;
    d.mom = (cfg->potential == PIMD_POT_MODEL && cfg->precision != PIMD_FP64) ? (void*)(w + o.mom) : nullptr;
    if (cfg->potential == PIMD_POT_GFN) {
        d.gfn_w = (float*)(w + o.gfn_w);
        d.gfn_n = (float*)(w + o.gfn_n);
        d.gfn_m = (float*)(w + o.gfn_m);
        d.gfn_e = (float*)(w + o.gfn_e);
        d.gfn_wtc = cfg->precision == PIMD_BF16_TC ? (unsigned char*)(w + o.gfn_wtc) : nullptr;
        d.gfn.F = cfg->gfn_features;
        d.gfn.L = cfg->gfn_iterations;
    }
    if (b.any_skin) {
        d.maxcand = max_candidates(d.maxnb, cfg->cutoff_A, b.max_skin);
        d.cand = (int*)(w + o.cand);
        d.ncand = (int*)(w + o.ncand);
        d.xref = (float4*)(w + o.xref);
        d.rebuild = (int*)(w + o.rebuild);
    }
    for (const Rep& rp : b.reps) d.max_P = std::max(d.max_P, rp.P);
    if (cfg->metad && cfg->metad->cv != PIMD_CV_NONE) {
        const pimd_metad_desc* m = cfg->metad;
        MetadParams& mp = d.metad;
        mp.cv = m->cv;
        mp.n_terms = m->cv == PIMD_CV_DISTANCES ? m->n_terms : 0;
        for (int t = 0; t < mp.n_terms; ++t) {
            mp.ti[t] = m->term_i[t];
            mp.tj[t] = m->term_j[t];
            mp.tc[t] = m->term_c[t];
        }
        mp.Q = m->xrd_Q;
        for (int t = 0; t < 8; ++t) mp.f_type[t] = m->cv == PIMD_CV_XRD ? m->xrd_f[t] : 0.0;
        mp.h0 = m->height_eV;
        mp.sigma = m->sigma;
        mp.gamma = m->bias_factor;
        mp.stride = m->stride;
        mp.max_hills = m->max_hills;
        d.md_hills = (double2*)(w + o.md_hills);
        d.md_nhill = (int*)(w + o.md_nhill);
        d.md_cv = (double*)(w + o.md_cv);
        d.md_vb = (double*)(w + o.md_vb);
        d.md_dvds = (double*)(w + o.md_dvds);
        d.md_cvpart = (double*)(w + o.md_cvpart);
        d.md_virpart = (double*)(w + o.md_virpart);
        d.md_grad = w + o.md_grad;
    }
    // angular terms through moment tensors when the mean neighbour count makes
    // the O(n) moment path cheaper than the O(n^2) pair sums
    d.sched.ang = (d.mom != nullptr && b.nb_est >= 24.0) ? 1 : 0;
    d.deterministic = cfg->deterministic ? 1 : 0;
    d.step = (unsigned long long*)(w + o.step);
    d.err = (DevErr*)(w + o.err);
    d.est = (double*)(w + o.est);
    d.perm = (int*)(w + o.perm);
    d.tile_type = (int*)(w + o.tile_type);
    d.rows_pad = b.rows_pad;
    d.n_parts = b.part_ba.empty() ? 1 : (int)b.part_ba.size() - 1;
    for (size_t k = 0; k < b.part_ba.size(); ++k) {
        d.part_ba[k] = b.part_ba[k];
        d.part_tile[k] = b.part_tile[k];
    }
    d.n_types = (int)b.typeZ.size();
    d.n_hidden = cfg->n_hidden;
    d.width = cfg->widths[0];
    d.blob = b.blob;
    d.wts = w + o.wts;
    d.wtc = w + o.wtc;
    d.wtc_bytes_per_type = b.wtc_bytes;
    d.wtc_vec = (float*)(w + o.wtc_vec);
    d.wtc_vec_per_type = b.wtc_vec;
    d.dt = cfg->dt_fs;
    d.gamma0 = cfg->gamma0_per_fs;
    d.lambda = cfg->pile_lambda;
    d.thermostat = cfg->thermostat;
    d.splitting = cfg->splitting;
    d.potential = cfg->potential;
    d.omega_harm = cfg->omega_harm;
    d.rc = cfg->cutoff_A;

    rc = upload(c, d.reps, b.reps);
    if (!rc) rc = upload(c, d.bsys, b.bsys);
    if (!rc) rc = upload(c, d.ba_sys, b.ba_sys);
    if (!rc) {
        std::vector<int4> bi(b.B);
        for (int i = 0; i < b.B; ++i) {
            const BeadSys& sy = b.bsys[b.ba_sys[i]];
            bi[i] = make_int4(b.ba_sys[i], sy.ba0, sy.N, sy.rep);
        }
        rc = upload(c, d.ba_info, bi);
    }
    if (!rc) rc = upload(c, d.mass, b.mass);
    if (!rc) {
        std::vector<double2> mi(b.NA);
        for (const Rep& rp : b.reps)
            for (int i = 0; i < rp.N; ++i) {
                const double m = b.mass[rp.atom0 + i];
                mi[rp.atom0 + i] = make_double2(1.0 / m, std::sqrt(m * rp.kT_md));
            }
        rc = upload(c, d.minv, mi);
    }
    if (!rc) rc = upload(c, d.atype, b.atype);
    if (!rc) rc = upload(c, d.x0, b.x0);
    if (!rc) rc = upload(c, d.cmat, b.cmat);
    const std::vector<float> cmatf(b.cmat.begin(), b.cmat.end());
    if (!rc) rc = upload(c, d.cmatf, cmatf);
    if (!rc) rc = upload(c, d.modes, b.modes);
    if (!rc) rc = upload(c, d.rp_blocks, b.rp_blocks);
    if (!rc) rc = upload(c, d.rep_blk0, b.rep_blk0);
    if (!rc) rc = upload(c, d.perm, b.perm);
    if (!rc) rc = upload(c, d.tile_type, b.tile_type);
    if (!rc) rc = upload(c, d.cell_bs, b.cell_bs);
    if (rc) { std::string m = c->err; delete c; return fail(nullptr, rc, m); }
    // positions carry the element type in w
    {
        std::vector<unsigned char> xs(d.precision == PIMD_FP64 ? sizeof(Dbl4) * b.B : sizeof(float4) * b.B);
        for (int r = 0; r < b.R; ++r) {
            const Rep& rp = b.reps[r];
            for (int k = 0; k < rp.P; ++k)
                for (int i = 0; i < rp.N; ++i) {
                    const size_t ba = rp.ba0 + (size_t)k * rp.N + i;
                    const int t = b.atype[rp.atom0 + i];
                    if (d.precision == PIMD_FP64) {
                        Dbl4 v = {b.x0[3 * (rp.atom0 + i)], b.x0[3 * (rp.atom0 + i) + 1], b.x0[3 * (rp.atom0 + i) + 2], 0.0};
                        long long tb = t;
                        std::memcpy(&v.w, &tb, sizeof(double));
                        std::memcpy(xs.data() + sizeof(Dbl4) * ba, &v, sizeof(Dbl4));
                    } else {
                        float4 v = make_float4((float)b.x0[3 * (rp.atom0 + i)], (float)b.x0[3 * (rp.atom0 + i) + 1],
                                               (float)b.x0[3 * (rp.atom0 + i) + 2], 0.0f);
                        std::memcpy(&v.w, &t, sizeof(float));
                        std::memcpy(xs.data() + sizeof(float4) * ba, &v, sizeof(float4));
                    }
                }
        }
        rc = upload(c, d.x, xs);
        if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->st), "create upload");
        if (rc) { std::string m = c->err; delete c; return fail(nullptr, rc, m); }
    }
    cudaMemsetAsync(d.Q, 0, sizeof(double) * d.R, c->st);
    if (d.maxcand) {
        // reference positions far away: the first list build rebuilds every bead
        cudaMemsetAsync(d.xref, 0x7f, sizeof(float4) * d.B, c->st);
        cudaMemsetAsync(d.ncand, 0, sizeof(int) * d.B, c->st);
    }
    if (d.metad.cv) {
        cudaMemsetAsync(d.md_nhill, 0, sizeof(int) * d.R, c->st);
        cudaMemsetAsync(d.md_cv, 0, sizeof(double) * d.S, c->st);
        cudaMemsetAsync(d.md_vb, 0, sizeof(double) * d.S, c->st);
    }
    cudaMemsetAsync(d.step, 0, sizeof(unsigned long long), c->st);
    cudaMemsetAsync(d.err, 0, sizeof(DevErr), c->st);
    cudaMemsetAsync(d.nnb, 0, sizeof(int) * d.B, c->st);
    cudaMemsetAsync(d.V, 0, sizeof(double) * d.S, c->st);
    cudaMemsetAsync(d.W, 0, sizeof(double) * 9 * d.S, c->st);
    cudaMemsetAsync(d.fnm, 0, sizeof(double) * 3 * d.B, c->st);
    launch_rp_init(d, c->st);
    launch_beads(d, c->st);
    c->beads_current = true;
    rc = cuda_check(c, cudaGetLastError(), "initial state");
    if (!rc && d.potential == PIMD_POT_HARMONIC) rc = refresh_forces(c);
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->st), "initial state");
    if (rc) { std::string m = c->err; delete c; return fail(nullptr, rc, m); }
    *out = c;
    return PIMD_OK;
}

int pimd_set_weights(pimd_ctx* c, const pimd_model_desc* m)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!m) return fail(c, PIMD_ERR_INVALID_ARG, "model is NULL");
    if (c->d.potential != PIMD_POT_MODEL) return fail(c, PIMD_ERR_STATE, "context does not use the network potential");
    if (m->n_hidden != c->cfg.n_hidden || !m->widths) return fail(c, PIMD_ERR_INVALID_ARG, "n_hidden differs from the config");
    for (int l = 0; l < m->n_hidden; ++l)
        if (m->widths[l] != c->cfg.widths[l]) return fail(c, PIMD_ERR_INVALID_ARG, "widths differ from the config");
    if (!m->Z || !m->params || !m->r_mu || !m->zeta || !m->lambda || !m->eta_A)
        return fail(c, PIMD_ERR_INVALID_ARG, "model arrays must not be NULL");
    const int zeta_ok[4] = {1, 2, 4, 8};
    for (int q = 0; q < 4; ++q)
        if (m->zeta[q] != zeta_ok[q]) return fail(c, PIMD_ERR_UNSUPPORTED, "zeta must be {1, 2, 4, 8}");
    if (m->lambda[0] != 1.0 || m->lambda[1] != -1.0) return fail(c, PIMD_ERR_UNSUPPORTED, "lambda must be {+1, -1}");
    const Build& b = c->build;
    Dev& d = c->d;
    const size_t blob = d.blob;
    std::vector<double> all((size_t)d.n_types * blob);
    for (int t = 0; t < d.n_types; ++t) {
        int e = -1;
        for (int q = 0; q < m->n_elements; ++q)
            if (m->Z[q] == b.typeZ[t]) e = q;
        if (e < 0 || !m->params[e]) return fail(c, PIMD_ERR_INVALID_ARG, "model has no parameters for element " + std::to_string(b.typeZ[t]));
        std::memcpy(all.data() + (size_t)t * blob, m->params[e], sizeof(double) * blob);
        for (size_t q = 0; q < blob; ++q)
            if (!std::isfinite(all[(size_t)t * blob + q])) return fail(c, PIMD_ERR_INVALID_ARG, "non-finite model parameter");
        const double* sig = all.data() + (size_t)t * blob + blob - 2 - ND;
        for (int q = 0; q < ND; ++q)
            if (!(sig[q] > 0.0)) return fail(c, PIMD_ERR_INVALID_ARG, "sigma must be > 0");
    }
    // descriptor parameters in both precisions
    c->dpd.rc = c->cfg.cutoff_A;
    c->dpd.pi_over_rc = M_PI / c->cfg.cutoff_A;
    c->dpd.eta_R = m->eta_R;
    for (int q = 0; q < NR; ++q) c->dpd.r_mu[q] = m->r_mu[q];
    for (int q = 0; q < 4; ++q) c->dpd.eta_A[q] = m->eta_A[q];
    c->dpf.rc = (float)c->dpd.rc;
    c->dpf.pi_over_rc = (float)c->dpd.pi_over_rc;
    c->dpf.eta_R = (float)c->dpd.eta_R;
    for (int q = 0; q < NR; ++q) c->dpf.r_mu[q] = (float)c->dpd.r_mu[q];
    for (int q = 0; q < 4; ++q) c->dpf.eta_A[q] = (float)c->dpd.eta_A[q];
    c->dpd.eta_R_l2 = c->dpd.eta_R * M_LOG2E;
    c->dpf.eta_R_l2 = (float)c->dpd.eta_R_l2;
    {
        const double dr = (m->r_mu[NR - 1] - m->r_mu[0]) / (NR - 1);
        bool even = dr > 0.0;
        for (int q = 0; q < NR && even; ++q)
            even = std::fabs(m->r_mu[q] - (m->r_mu[0] + q * dr)) <= 1e-9 * std::max(1.0, std::fabs(m->r_mu[q]));
        c->dpf.r_even = c->dpd.r_even = even ? 1 : 0;
        c->dpd.r_delta = dr;
        c->dpf.r_delta = (float)dr;
        c->dpd.rec_k = std::exp2(-2.0 * c->dpd.eta_R_l2 * dr * dr);
        c->dpf.rec_k = (float)c->dpd.rec_k;
    }
    for (int q = 0; q < 4; ++q) {
        c->dpd.eta_A_l2[q] = c->dpd.eta_A[q] * M_LOG2E;
        c->dpf.eta_A_l2[q] = (float)c->dpd.eta_A_l2[q];
    }
    int rc;
    if (d.precision == PIMD_FP64) {
        rc = upload(c, d.wts, all);
    } else {
        std::vector<float> f32(all.begin(), all.end());
        rc = upload(c, d.wts, f32);
        if (!rc && d.precision == PIMD_BF16_TC) {
            std::vector<unsigned char> img(d.wtc_bytes_per_type * d.n_types);
            std::vector<float> vec(d.wtc_vec_per_type * d.n_types);
            for (int t = 0; t < d.n_types; ++t)
                prepare_tc_weights(d, t, all.data() + (size_t)t * blob, img.data() + d.wtc_bytes_per_type * t,
                                   vec.data() + d.wtc_vec_per_type * t);
            rc = upload(c, d.wtc, img);
            if (!rc) rc = upload(c, d.wtc_vec, vec);
            if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->st), "weights upload");
        }
    }
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->st), "weights upload");
    if (rc) return rc;
    c->weights_set = true;
    rc = refresh_forces(c);
    if (!rc) rc = device_errors(c);
    return rc;
}

int pimd_set_gfn(pimd_ctx* c, const pimd_gfn_desc* g)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!g) return fail(c, PIMD_ERR_INVALID_ARG, "desc is NULL");
    if (c->d.potential != PIMD_POT_GFN) return fail(c, PIMD_ERR_STATE, "context does not use the GFN head");
    Dev& d = c->d;
    const Build& b = c->build;
    const int F = d.gfn.F, L = d.gfn.L, ne = g->n_elements;
    if (!g->params) return fail(c, PIMD_ERR_INVALID_ARG, "params is NULL");
    if (ne < 1 || ne > PIMD_MAX_ELEMENTS) return fail(c, PIMD_ERR_INVALID_ARG, "n_elements must be 1..8");
    for (int q = 1; q < ne; ++q)
        if (!(g->Z[q] > g->Z[q - 1])) return fail(c, PIMD_ERR_INVALID_ARG, "Z must be ascending");
    if (g->n_params != gfn_blob_len(F, L, ne))
        return fail(c, PIMD_ERR_INVALID_ARG, "n_params is " + std::to_string(g->n_params) + ", the layout needs " +
                                                 std::to_string(gfn_blob_len(F, L, ne)));
    for (size_t q = 0; q < g->n_params; ++q)
        if (!std::isfinite(g->params[q])) return fail(c, PIMD_ERR_INVALID_ARG, "non-finite GFN parameter");
    if (!(g->eta_R > 0.0) || !std::isfinite(g->eta_R)) return fail(c, PIMD_ERR_INVALID_ARG, "eta_R must be > 0");
    for (int q = 0; q < NR; ++q)
        if (!std::isfinite(g->r_mu[q])) return fail(c, PIMD_ERR_INVALID_ARG, "non-finite r_mu");
    // FP32 device image: the context's element types in ascending Z, matrices transposed
    std::vector<float> w(b.gfn_params, 0.0f);
    GfnParams gp = d.gfn;
    unsigned o = 0;
    const double* q = g->params;
    gp.o_emb = o;
    for (size_t t = 0; t < b.typeZ.size(); ++t) {
        int e = -1;
        for (int k = 0; k < ne; ++k)
            if (g->Z[k] == b.typeZ[t]) e = k;
        if (e < 0) return fail(c, PIMD_ERR_INVALID_ARG, "no embedding for element " + std::to_string(b.typeZ[t]));
        for (int k = 0; k < F; ++k) w[o + t * F + k] = (float)q[(size_t)e * F + k];
    }
    o += (unsigned)(b.typeZ.size() * F);
    q += (size_t)ne * F;
    auto put_t = [&](int out, int in) {   // host W [out][in] -> device W^T [in][out]
        const unsigned off = o;
        for (int i = 0; i < in; ++i)
            for (int j = 0; j < out; ++j) w[o + (size_t)i * out + j] = (float)q[(size_t)j * in + i];
        o += (unsigned)(in * out);
        q += (size_t)in * out;
        return off;
    };
    auto put_v = [&](int n) {
        const unsigned off = o;
        for (int i = 0; i < n; ++i) w[o + i] = (float)q[i];
        o += (unsigned)n;
        q += n;
        return off;
    };
    gp.o_We = put_t(F, NR);
    gp.o_be = put_v(F);
    for (int l = 0; l < L; ++l) {
        gp.o_it[l][0] = put_t(F, F);
        gp.o_it[l][1] = put_v(F);
        gp.o_it[l][2] = put_t(F, 2 * F);
        gp.o_it[l][3] = put_v(F);
        gp.o_it[l][4] = put_t(F, F);
        gp.o_it[l][5] = put_v(F);
        gp.o_it[l][6] = put_t(F, F);
        gp.o_it[l][7] = put_v(F);
        gp.o_it[l][8] = put_t(F, F);
        gp.o_it[l][9] = put_v(F);
    }
    gp.o_Wf1 = put_t(F, F);
    gp.o_bf1 = put_v(F);
    gp.o_wf2 = put_v(F);
    gp.b_f2 = (float)q[0];
    gp.s_F = (float)q[1];
    gp.rc = (float)c->cfg.cutoff_A;
    gp.pi_over_rc = (float)(M_PI / c->cfg.cutoff_A);
    gp.eta_R = (float)g->eta_R;
    for (int k = 0; k < NR; ++k) gp.r_mu[k] = (float)g->r_mu[k];
    int rc = upload(c, d.gfn_w, w);
    if (!rc && d.gfn_wtc) {
        // BF16 images [out][in] in the K-major core-matrix layout, from the FP32
        // transposed copies just built
        std::vector<unsigned short> img(gfn_tc_image_bytes(F, L) / 2);
        size_t ob = 0;
        auto put_img = [&](unsigned src, int out, int in) {   // w[src] holds W^T [in][out]
            const unsigned off = (unsigned)(ob * 2);
            for (int n2 = 0; n2 < out; ++n2)
                for (int k = 0; k < in; ++k) {
                    const float v = w[src + (size_t)k * out + n2];
                    unsigned u;
                    std::memcpy(&u, &v, 4);
                    u += 0x7FFFu + ((u >> 16) & 1u);   // round to nearest even (finite values)
                    img[ob + cm_index_host(n2, k, in)] = (unsigned short)(u >> 16);
                }
            ob += (size_t)out * in;
            return off;
        };
        gp.t_We = put_img(gp.o_We, F, NR);
        for (int l = 0; l < L; ++l) {
            gp.t_it[l][0] = put_img(gp.o_it[l][0], F, F);
            gp.t_it[l][1] = put_img(gp.o_it[l][6], F, F);
            gp.t_it[l][2] = put_img(gp.o_it[l][8], F, F);
            gp.t_it[l][3] = put_img(gp.o_it[l][2], F, 2 * F);
            gp.t_it[l][4] = put_img(gp.o_it[l][4], F, F);
        }
        gp.t_Wf1 = put_img(gp.o_Wf1, F, F);
        rc = upload(c, d.gfn_wtc, img);
    }
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->st), "GFN parameter upload");
    if (rc) return rc;
    d.gfn = gp;
    drop_graphs(c);
    c->weights_set = true;
    rc = refresh_forces(c);
    if (!rc) rc = device_errors(c);
    return rc;
}

int pimd_step(pimd_ctx* c, int n_steps)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (n_steps < 0) return fail(c, PIMD_ERR_INVALID_ARG, "n_steps < 0");
    if (graph_pot(c->d.potential) && !c->weights_set) return fail(c, PIMD_ERR_STATE, "weights not set");
    if (n_steps == 0) return PIMD_OK;
    int rc = PIMD_OK;
    if (!c->forces_valid) {
        rc = refresh_forces(c);
        if (rc) return rc;
    }
    // the stage markers (event records inside the graph) cost time of their
    // own, so only the last step of a call carries them, and only when asked
    const bool marked = c->cfg.timing != 0 && c->stage_timing;
    int left = n_steps - (marked ? 1 : 0);
    if (left > 0 && !c->g1) {
        rc = capture(c, 1, false, &c->g1);
        if (rc) return rc;
    }
    if (left >= 8 && !c->g8) {
        rc = capture(c, 8, false, &c->g8);
        if (rc) return rc;
    }
    if (marked && !c->g1t) {
        rc = capture(c, 1, true, &c->g1t);
        if (rc) return rc;
    }
    while (left >= 8) {
        rc = cuda_check(c, cudaGraphLaunch(c->g8, c->st), "cudaGraphLaunch");
        if (rc) return rc;
        left -= 8;
    }
    while (left-- > 0) {
        rc = cuda_check(c, cudaGraphLaunch(c->g1, c->st), "cudaGraphLaunch");
        if (rc) return rc;
    }
    if (marked) {
        rc = cuda_check(c, cudaGraphLaunch(c->g1t, c->st), "cudaGraphLaunch");
        if (rc) return rc;
        c->stepped = true;
    }
    c->step_host += (unsigned long long)n_steps;
    return PIMD_OK;
}

int pimd_set_noise_index(pimd_ctx* c, int replica, int atom_offset, int n_atoms_total)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    int rc = check_replica(c, replica);
    if (rc) return rc;
    Rep& rp = c->build.reps[replica];
    if (atom_offset < 0 || n_atoms_total < rp.N || atom_offset > n_atoms_total - rp.N)
        return fail(c, PIMD_ERR_INVALID_ARG, "the replica's atoms must lie inside 0 .. n_atoms_total - 1");
    if ((long long)n_atoms_total * rp.P * 3 > 0xffffffffLL)
        return fail(c, PIMD_ERR_INVALID_ARG, "noise counter index exceeds 32 bits");
    rp.noise_atom0 = atom_offset;
    rp.noise_N = n_atoms_total;
    Dev& d = c->d;
    rc = cuda_check(c, cudaMemcpyAsync(d.reps + replica, &rp, sizeof(Rep), cudaMemcpyHostToDevice, c->st), "copy");
    // the initial state again, with the momenta drawn at the new indices
    const unsigned long long zero = 0;
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(d.step, &zero, sizeof(zero), cudaMemcpyHostToDevice, c->st), "copy");
    if (!rc) rc = cuda_check(c, cudaMemsetAsync(d.Q, 0, sizeof(double) * d.R, c->st), "memset");
    if (rc) return rc;
    launch_rp_init(d, c->st);
    launch_beads(d, c->st);
    c->beads_current = true;
    c->step_host = 0;
    c->forces_valid = false;
    rc = cuda_check(c, cudaStreamSynchronize(c->st), "initial state");
    if (!rc && !(graph_pot(d.potential) && !c->weights_set)) rc = refresh_forces(c);
    return rc;
}

int pimd_set_forces(pimd_ctx* c, const double* f_dev)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!f_dev) return fail(c, PIMD_ERR_INVALID_ARG, "f is NULL");
    if (!c->beads_current) {
        launch_beads(c->d, c->st);
        c->beads_current = true;
    }
    launch_pack_forces(c->d, f_dev, c->st);
    launch_rp_finish(c->d, false, c->st);   // f_nm = C^T f, no dynamics
    c->forces_valid = true;
    return cuda_check(c, cudaGetLastError(), "set forces");
}

int pimd_ring_start(pimd_ctx* c, double* x_dev)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!x_dev) return fail(c, PIMD_ERR_INVALID_ARG, "x is NULL");
    if (!c->forces_valid) return fail(c, PIMD_ERR_STATE, "no forces for the first half step (pimd_set_forces)");
    launch_rp_start(c->d, c->st);
    launch_unpack(c->d, nullptr, nullptr, nullptr, x_dev, c->st);
    c->forces_valid = false;   // the next forces belong to the new positions
    return cuda_check(c, cudaGetLastError(), "ring start");
}

int pimd_ring_finish(pimd_ctx* c, const double* f_dev)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!f_dev) return fail(c, PIMD_ERR_INVALID_ARG, "f is NULL");
    if (c->forces_valid) return fail(c, PIMD_ERR_STATE, "pimd_ring_finish without a pimd_ring_start before it");
    launch_pack_forces(c->d, f_dev, c->st);
    launch_rp_finish(c->d, true, c->st);
    if (c->d.deterministic) launch_heat_sum(c->d, 0, c->st);
    c->forces_valid = true;
    c->step_host += 1;
    return cuda_check(c, cudaGetLastError(), "ring finish");
}

int pimd_set_overlap(pimd_ctx* c, int on)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (c->overlap != (on != 0)) drop_graphs(c);
    c->overlap = on != 0;
    return (c->d.n_parts > 1 && network_tiles_available(c->d)) ? 1 : 0;
}

int pimd_set_stage_timing(pimd_ctx* c, int on)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!c->cfg.timing) return fail(c, PIMD_ERR_STATE, "context was created without timing");
    c->stage_timing = on != 0;
    return PIMD_OK;
}

int pimd_stage_times(pimd_ctx* c, float* ms)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!ms) return fail(c, PIMD_ERR_INVALID_ARG, "ms is NULL");
    if (!c->cfg.timing || !c->ev[0]) return fail(c, PIMD_ERR_STATE, "context was created without timing");
    if (!c->stepped) return fail(c, PIMD_ERR_STATE, "no step has run yet");
    int rc = cuda_check(c, cudaEventSynchronize(c->ev[PIMD_N_STAGES]), "cudaEventSynchronize");
    if (rc) return rc;
    for (int i = 0; i < PIMD_N_STAGES; ++i) {
        float t = 0.0f;
        rc = cuda_check(c, cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1]), "cudaEventElapsedTime");
        if (rc) return rc;
        ms[i] = t;
    }
    return PIMD_OK;
}

int pimd_tune(pimd_ctx* c, int reps, double* out_ms)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (reps < 1) return fail(c, PIMD_ERR_INVALID_ARG, "reps must be >= 1");
    if (c->d.potential != PIMD_POT_MODEL || !c->weights_set) return fail(c, PIMD_ERR_STATE, "weights not set");
    int rc = refresh_forces(c);   // current neighbour lists, dE/dG
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_check(c, cudaErrorUnknown, "cudaEventCreate");
    }
    const Sched before = c->d.sched;
    Sched cands[10];
    int nc = 0;
    const int rl[6] = {4, 6, 8, 10, 12, 16};
    for (int q = 0; q < 6; ++q) cands[nc++] = Sched{rl[q], rl[q] + 32, 0, 0};
    cands[nc++] = Sched{8, 1 << 30, 0, 0};                 // ordered pairs for every atom
    if (c->d.mom) {
        cands[nc++] = Sched{8, 40, 0, 1, 0};                 // moment tensors
        // the BF16 moment adjoint at 16 warps per SM (128 registers)
        if (c->d.precision == PIMD_BF16_TC) cands[nc++] = Sched{8, 40, 0, 1, 1};
    }
    double best = 1e30, t_default = 0.0;
    Sched pick = before;
    for (int q = 0; q < nc && !rc; ++q) {
        c->d.sched = cands[q];
        launch_descriptors(c->d, dparams(c), c->st);   // warm the schedule
        launch_adjoint(c->d, dparams(c), c->st);
        double tmin = 1e30;
        for (int r = 0; r < reps && !rc; ++r) {
            cudaEventRecord(e0, c->st);
            launch_descriptors(c->d, dparams(c), c->st);
            launch_adjoint(c->d, dparams(c), c->st);
            cudaEventRecord(e1, c->st);
            rc = cuda_check(c, cudaEventSynchronize(e1), "tune");
            float ms = 0.0f;
            if (!rc) cudaEventElapsedTime(&ms, e0, e1);
            tmin = std::min(tmin, (double)ms);
        }
        const Sched& s = cands[q];
        const bool same = s.ang == before.ang && (s.ang ? s.adj_wide == before.adj_wide
                                                        : (s.rmax == before.rmax && s.band_min == before.band_min &&
                                                           s.small_atomics == before.small_atomics));
        if (same) t_default = tmin;   // the schedule in force before tuning
        if (tmin < best) {
            best = tmin;
            pick = cands[q];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->d.sched = pick;
    drop_graphs(c);
    if (!rc) rc = refresh_forces(c);   // forces with the chosen schedule
    if (!rc) rc = device_errors(c);
    if (out_ms) {
        out_ms[0] = best;
        out_ms[1] = pick.ang ? -1.0 : pick.band_min >= (1 << 30) ? 0.0 : (double)pick.rmax;
        out_ms[2] = t_default;
    }
    return rc;
}

int pimd_set_schedule(pimd_ctx* c, int band_length)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (band_length != 0 && (band_length < 1 || band_length > 16))
        return fail(c, PIMD_ERR_INVALID_ARG, "band_length must be 0 or 1..16");
    const int ang = c->d.sched.ang, wide = c->d.sched.adj_wide;
    c->d.sched = band_length == 0 ? Sched{8, 1 << 30, 0, ang, wide} : Sched{band_length, band_length + 32, 0, ang, wide};
    drop_graphs(c);
    c->forces_valid = false;
    return PIMD_OK;
}

int pimd_set_angular(pimd_ctx* c, int algo)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (algo != PIMD_ANG_PAIRS && algo != PIMD_ANG_MOMENTS)
        return fail(c, PIMD_ERR_INVALID_ARG, "algo must be PIMD_ANG_PAIRS or PIMD_ANG_MOMENTS");
    if (algo == PIMD_ANG_MOMENTS && !c->d.mom)
        return fail(c, PIMD_ERR_UNSUPPORTED, "moment tensors need the model potential in FP32 or BF16 precision");
    c->d.sched.ang = algo == PIMD_ANG_MOMENTS ? 1 : 0;
    drop_graphs(c);
    c->forces_valid = false;
    return PIMD_OK;
}

int pimd_get_angular(const pimd_ctx* c)
{
    if (!c) return -1;
    return c->d.sched.ang ? PIMD_ANG_MOMENTS : PIMD_ANG_PAIRS;
}

int pimd_set_adjoint_warps(pimd_ctx* c, int warps_per_sm)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (warps_per_sm != 12 && warps_per_sm != 16)
        return fail(c, PIMD_ERR_INVALID_ARG, "warps_per_sm must be 12 or 16");
    c->d.sched.adj_wide = warps_per_sm == 16 ? 1 : 0;
    drop_graphs(c);
    c->forces_valid = false;
    return PIMD_OK;
}

int pimd_get_adjoint_warps(const pimd_ctx* c)
{
    if (!c) return -1;
    return c->d.sched.adj_wide ? 16 : 12;
}

int pimd_kernels_per_step(const pimd_ctx* c)
{
    if (!c) return 0;
    // ring start, ring finish (which also ends the step; deterministic mode
    // adds the ordered heat sum); metadynamics: CV, bias, bias force
    const Dev& d = c->d;
    const int ring = 2 + (d.deterministic ? 1 : 0), md = d.metad.cv ? 3 : 0;
    if (d.potential == PIMD_POT_HARMONIC) return ring + 2 + md;   // harmonic forces, energy
    if (d.potential == PIMD_POT_GFN)   // neighbours, the head, energy
        return ring + 2 + 2 + gfn_kernels_per_eval(d.gfn.L) + md;
    // neighbours (cell binning, Verlet skin check, lists), descriptors,
    // network, adjoint (+ force gather), energy unless the adjoint sums it
    // the overlapped halves launch the descriptors, network and adjoint once
    // per half
    const int halves = c->overlap && splits_forces(c) ? c->d.n_parts : 1;
    const int nbr = 1 + (d.n_cell_bs ? 1 : 0) + (d.maxcand ? 1 : 0);
    const int energy = adjoint_sums_energy(d, dparams(c)) ? 0 : 1;
    return ring + nbr + 3 * halves + (d.deterministic ? 1 : 0) + energy + md;
}

int pimd_energy_forces(pimd_ctx* c, const double* x_dev, double* e_dev, double* f_dev, double* virial_dev)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (graph_pot(c->d.potential) && !c->weights_set) return fail(c, PIMD_ERR_STATE, "weights not set");
    if (x_dev) {
        launch_pack_positions(c->d, x_dev, c->st);
        c->beads_current = false;
        c->forces_valid = false;
    } else if (!c->beads_current) {
        launch_beads(c->d, c->st);
        c->beads_current = true;
    }
    eval_forces(c);
    if (!x_dev) {
        launch_rp_finish(c->d, false, c->st);
        c->forces_valid = true;
    }
    launch_unpack(c->d, f_dev, e_dev, virial_dev, nullptr, c->st);
    return cuda_check(c, cudaGetLastError(), "energy_forces launch");
}

int pimd_descriptors(pimd_ctx* c, const double* x_dev, double* G_dev)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!G_dev) return fail(c, PIMD_ERR_INVALID_ARG, "G_dev is NULL");
    if (c->d.potential != PIMD_POT_MODEL) return fail(c, PIMD_ERR_STATE, "context does not use the network potential");
    if (!c->weights_set) {
        // descriptor hyper-parameters arrive with the weights
        return fail(c, PIMD_ERR_STATE, "weights not set");
    }
    if (x_dev) {
        launch_pack_positions(c->d, x_dev, c->st);
        c->beads_current = false;
        c->forces_valid = false;
    } else if (!c->beads_current) {
        launch_beads(c->d, c->st);
        c->beads_current = true;
    }
    launch_neighbours(c->d, c->st);
    launch_descriptors(c->d, dparams(c), c->st);
    launch_descriptors_out(c->d, G_dev, c->st);
    return cuda_check(c, cudaGetLastError(), "descriptors launch");
}

int pimd_estimators(pimd_ctx* c, pimd_est* out, int n_reps)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!out || n_reps != c->d.R) return fail(c, PIMD_ERR_INVALID_ARG, "n_reps must equal the replica count");
    if (graph_pot(c->d.potential) && !c->weights_set) return fail(c, PIMD_ERR_STATE, "weights not set");
    int rc = PIMD_OK;
    if (!c->forces_valid) {
        rc = refresh_forces(c);
        if (rc) return rc;
    }
    launch_estimators(c->d, c->st);
    std::vector<double> h((size_t)EST_STRIDE * c->d.R);
    rc = cuda_check(c, cudaMemcpyAsync(h.data(), c->d.est, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->st),
                    "estimators copy");
    if (rc) return rc;
    rc = device_errors(c);
    if (rc) return rc;
    for (int r = 0; r < c->d.R; ++r) {
        const double* o = h.data() + (size_t)r * EST_STRIDE;
        pimd_est& e = out[r];
        e.V_mean = o[0]; e.K_prim = o[1]; e.K_cv = o[2]; e.E_tot = o[3];
        for (int a = 0; a < 9; ++a) e.W[a] = o[4 + a];
        e.H_cons = o[13]; e.Q_thermo = o[14]; e.T_kin = o[15]; e.nbr_mean = o[16]; e.nbr_max = o[17];
    }
    return PIMD_OK;
}

int pimd_get_state(pimd_ctx* c, double* q_nm, double* p_nm, uint64_t* step, double* Q)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    const size_t n = 3 * (size_t)c->d.B;
    int rc = PIMD_OK;
    if (q_nm) rc = cuda_check(c, cudaMemcpyAsync(q_nm, c->d.q, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st), "copy");
    if (!rc && p_nm) rc = cuda_check(c, cudaMemcpyAsync(p_nm, c->d.p, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st), "copy");
    if (!rc && Q) rc = cuda_check(c, cudaMemcpyAsync(Q, c->d.Q, sizeof(double) * c->d.R, cudaMemcpyDeviceToHost, c->st), "copy");
    if (rc) return rc;
    rc = device_errors(c);
    if (step) *step = c->step_host;
    return rc;
}

int pimd_set_state(pimd_ctx* c, const double* q_nm, const double* p_nm, uint64_t step, const double* Q)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!q_nm || !p_nm) return fail(c, PIMD_ERR_INVALID_ARG, "q_nm and p_nm are required");
    const size_t n = 3 * (size_t)c->d.B;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(q_nm[i]) || !std::isfinite(p_nm[i])) return fail(c, PIMD_ERR_INVALID_ARG, "non-finite state");
    int rc = cuda_check(c, cudaMemcpyAsync(c->d.q, q_nm, sizeof(double) * n, cudaMemcpyHostToDevice, c->st), "copy");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(c->d.p, p_nm, sizeof(double) * n, cudaMemcpyHostToDevice, c->st), "copy");
    unsigned long long s = step;
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(c->d.step, &s, sizeof(s), cudaMemcpyHostToDevice, c->st), "copy");
    std::vector<double> Qz(c->d.R, 0.0);
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(c->d.Q, Q ? Q : Qz.data(), sizeof(double) * c->d.R,
                                                cudaMemcpyHostToDevice, c->st), "copy");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->st), "set_state");
    if (rc) return rc;
    c->step_host = step;
    c->beads_current = false;
    c->forces_valid = false;
    if (graph_pot(c->d.potential) && !c->weights_set) return PIMD_OK;
    rc = refresh_forces(c);
    if (!rc) rc = device_errors(c);
    return rc;
}

int pimd_get_forces(pimd_ctx* c, double* x_host, double* f_host, double* V_host)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (graph_pot(c->d.potential) && !c->weights_set) return fail(c, PIMD_ERR_STATE, "weights not set");
    int rc = PIMD_OK;
    if (!c->forces_valid) {
        rc = refresh_forces(c);
        if (rc) return rc;
    }
    Dev& d = c->d;
    const size_t v4 = d.precision == PIMD_FP64 ? sizeof(Dbl4) : sizeof(float4);
    std::vector<unsigned char> xs(v4 * d.B), fs(v4 * d.B);
    rc = cuda_check(c, cudaMemcpyAsync(xs.data(), d.x, xs.size(), cudaMemcpyDeviceToHost, c->st), "copy");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(fs.data(), d.f, fs.size(), cudaMemcpyDeviceToHost, c->st), "copy");
    if (!rc && V_host) rc = cuda_check(c, cudaMemcpyAsync(V_host, d.V, sizeof(double) * d.S, cudaMemcpyDeviceToHost, c->st), "copy");
    if (rc) return rc;
    rc = device_errors(c);
    if (rc) return rc;
    for (int b = 0; b < d.B; ++b)
        for (int a = 0; a < 3; ++a) {
            double xv, fv;
            if (d.precision == PIMD_FP64) {
                xv = ((const double*)xs.data())[4 * (size_t)b + a];
                fv = ((const double*)fs.data())[4 * (size_t)b + a];
            } else {
                xv = ((const float*)xs.data())[4 * (size_t)b + a];
                fv = ((const float*)fs.data())[4 * (size_t)b + a];
            }
            if (x_host) x_host[3 * (size_t)b + a] = xv;
            if (f_host) f_host[3 * (size_t)b + a] = fv;
        }
    return PIMD_OK;
}

int pimd_get_neighbours(pimd_ctx* c, int* nnb_host, int* nbr_host)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!graph_pot(c->d.potential)) return fail(c, PIMD_ERR_STATE, "no neighbour lists for this potential");
    int rc = PIMD_OK;
    if (nnb_host) rc = cuda_check(c, cudaMemcpyAsync(nnb_host, c->d.nnb, sizeof(int) * c->d.B, cudaMemcpyDeviceToHost, c->st), "copy");
    if (!rc && nbr_host)
        rc = cuda_check(c, cudaMemcpyAsync(nbr_host, c->d.nbr, sizeof(int) * (size_t)c->d.B * c->d.maxnb,
                                           cudaMemcpyDeviceToHost, c->st), "copy");
    if (rc) return rc;
    return device_errors(c);
}

int pimd_sync(pimd_ctx* c)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    return device_errors(c);
}

int pimd_sizes(const pimd_ctx* c, int64_t* B, int64_t* S, int* R, int* maxnb)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (B) *B = c->d.B;
    if (S) *S = c->d.S;
    if (R) *R = c->d.R;
    if (maxnb) *maxnb = c->d.maxnb;
    return PIMD_OK;
}


int pimd_metad_hills(pimd_ctx* c, int replica, double* s, double* h, int capacity)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!c->d.metad.cv) return fail(c, PIMD_ERR_STATE, "no metadynamics bias configured");
    int rc = check_replica(c, replica);
    if (rc) return rc;
    int n = 0;
    rc = cuda_check(c, cudaMemcpyAsync(&n, c->d.md_nhill + replica, sizeof(int), cudaMemcpyDeviceToHost, c->st), "hills");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->st), "hills");
    if (rc) return rc;
    const int m = std::min(n, std::max(capacity, 0));
    if (m > 0 && (s || h)) {
        std::vector<double2> buf(m);
        rc = cuda_check(c, cudaMemcpyAsync(buf.data(), c->d.md_hills + (size_t)replica * c->d.metad.max_hills,
                                           sizeof(double2) * m, cudaMemcpyDeviceToHost, c->st), "hills");
        if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->st), "hills");
        if (rc) return rc;
        for (int k = 0; k < m; ++k) {
            if (s) s[k] = buf[k].x;
            if (h) h[k] = buf[k].y;
        }
    }
    return n;
}

int pimd_metad_set_hills(pimd_ctx* c, int replica, const double* s, const double* h, int n)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!c->d.metad.cv) return fail(c, PIMD_ERR_STATE, "no metadynamics bias configured");
    int rc = check_replica(c, replica);
    if (rc) return rc;
    if (n < 0 || n > c->d.metad.max_hills || (n > 0 && (!s || !h)))
        return fail(c, PIMD_ERR_INVALID_ARG, "n must be 0..max_hills with s and h given");
    std::vector<double2> buf(n);
    for (int k = 0; k < n; ++k) buf[k] = make_double2(s[k], h[k]);
    if (n > 0)
        rc = cuda_check(c, cudaMemcpyAsync(c->d.md_hills + (size_t)replica * c->d.metad.max_hills, buf.data(),
                                           sizeof(double2) * n, cudaMemcpyHostToDevice, c->st), "set hills");
    if (!rc)
        rc = cuda_check(c, cudaMemcpyAsync(c->d.md_nhill + replica, &n, sizeof(int), cudaMemcpyHostToDevice, c->st),
                        "set hills");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->st), "set hills");
    c->forces_valid = false;
    return rc;
}

int pimd_metad_cv(pimd_ctx* c, double* cv, double* bias)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!c->d.metad.cv) return fail(c, PIMD_ERR_STATE, "no metadynamics bias configured");
    int rc = PIMD_OK;
    if (cv) rc = cuda_check(c, cudaMemcpyAsync(cv, c->d.md_cv, sizeof(double) * c->d.S, cudaMemcpyDeviceToHost, c->st), "cv");
    if (!rc && bias)
        rc = cuda_check(c, cudaMemcpyAsync(bias, c->d.md_vb, sizeof(double) * c->d.S, cudaMemcpyDeviceToHost, c->st), "cv");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->st), "cv");
    return rc;
}

int pimd_selftest_bounded_wait(void* stream, double seconds)
{
    if (!(seconds > 0.0) || seconds > 10.0) return fail(nullptr, PIMD_ERR_INVALID_ARG, "seconds must be in (0, 10]");
    int timed_out = 0;
    if (run_wait_selftest((cudaStream_t)stream, (long long)(seconds * 2.0e9), &timed_out)) {
        cudaGetLastError();
        return fail(nullptr, PIMD_ERR_CUDA, "self-test launch failed");
    }
    return timed_out ? fail(nullptr, PIMD_ERR_TIMEOUT, "bounded wait expired (as designed)") : PIMD_OK;
}

int pimd_element_types(const pimd_ctx* c, int* Z)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    const std::vector<int>& t = c->build.typeZ;
    if (Z)
        for (size_t k = 0; k < t.size(); ++k) Z[k] = t[k];
    return (int)t.size();
}

int pimd_rdf_counts(pimd_ctx* c, int replica, double r_max, int n_bins, unsigned long long* counts)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    int rc = check_replica(c, replica);
    if (rc) return rc;
    if (!counts) return fail(c, PIMD_ERR_INVALID_ARG, "counts is NULL");
    if (n_bins < 1 || n_bins > ANALYSIS_MAX_BINS) return fail(c, PIMD_ERR_INVALID_ARG, "n_bins must be 1..1024");
    if (!(r_max > 0.0)) return fail(c, PIMD_ERR_INVALID_ARG, "r_max must be > 0");
    const Rep& rp = c->build.reps[replica];
    if (rp.periodic) {
        const double half = 0.5 * std::min(std::min(rp.L[0], rp.L[1]), rp.L[2]);
        if (r_max > half) return fail(c, PIMD_ERR_INVALID_ARG, "r_max exceeds half the smallest box edge");
    }
    if (rdf_smem_bytes(c->d.n_types, n_bins) > 200 * 1024)
        return fail(c, PIMD_ERR_INVALID_ARG, "too many bins for the element pairs (shared-memory histogram)");
    BinEdges e;
    for (int k = 0; k <= n_bins; ++k) {
        const double rk = k * (r_max / n_bins);
        e.e[k] = (float)(rk * rk);
    }
    launch_rdf(c->d, replica, rp.P, rp.N, e, n_bins, (float)(n_bins / r_max), counts, c->st);
    return cuda_check(c, cudaGetLastError(), "rdf kernel");
}

int pimd_pt_coordinate(pimd_ctx* c, int replica, const int* bond, int acceptor_Z, double v_min, double v_max,
                       int n_bins, float* v, unsigned long long* hist)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    int rc = check_replica(c, replica);
    if (rc) return rc;
    if (!bond) return fail(c, PIMD_ERR_INVALID_ARG, "bond is NULL");
    if (!v && !hist) return fail(c, PIMD_ERR_INVALID_ARG, "v and hist are both NULL");
    if (n_bins < 1 || n_bins > ANALYSIS_MAX_BINS) return fail(c, PIMD_ERR_INVALID_ARG, "n_bins must be 1..1024");
    if (!(v_max > v_min)) return fail(c, PIMD_ERR_INVALID_ARG, "v_max must exceed v_min");
    const std::vector<int>& tz = c->build.typeZ;
    const auto it = std::find(tz.begin(), tz.end(), acceptor_Z);
    if (it == tz.end()) return fail(c, PIMD_ERR_INVALID_ARG, "acceptor_Z is not an element of the context");
    const Rep& rp = c->build.reps[replica];
    BinEdges e;
    for (int k = 0; k <= n_bins; ++k) e.e[k] = (float)(v_min + k * ((v_max - v_min) / n_bins));
    launch_pt(c->d, replica, rp.P, rp.N, bond, (int)(it - tz.begin()), e, n_bins, (float)(n_bins / (v_max - v_min)),
              v, hist, c->st);
    return cuda_check(c, cudaGetLastError(), "proton-transfer kernel");
}

int pimd_rdf_gr(pimd_ctx* c, int replica, double r_max, int n_bins, double n_configs,
                const unsigned long long* counts, double* g)
{
    static_assert(RDF_MAX_PAIRS == PIMD_MAX_ELEMENTS * (PIMD_MAX_ELEMENTS + 1) / 2, "pair slots");
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    int rc = check_replica(c, replica);
    if (rc) return rc;
    if (!counts || !g) return fail(c, PIMD_ERR_INVALID_ARG, "counts or g is NULL");
    if (n_bins < 1 || n_bins > ANALYSIS_MAX_BINS) return fail(c, PIMD_ERR_INVALID_ARG, "n_bins must be 1..1024");
    if (!(r_max > 0.0)) return fail(c, PIMD_ERR_INVALID_ARG, "r_max must be > 0");
    if (!(n_configs > 0.0)) return fail(c, PIMD_ERR_INVALID_ARG, "n_configs must be > 0");
    const Rep& rp = c->build.reps[replica];
    if (!rp.periodic) return fail(c, PIMD_ERR_INVALID_ARG, "g(r) needs a periodic replica (a box volume)");
    const int T = (int)c->build.typeZ.size();
    std::vector<double> n_per(T, 0.0);
    for (int i = 0; i < rp.N; ++i) n_per[c->build.atype[rp.atom0 + i]] += 1.0;
    RdfNorm nm{};
    int p = 0;
    for (int a = 0; a < T; ++a)
        for (int b = a; b < T; ++b, ++p) nm.pairs[p] = a == b ? n_per[a] * (n_per[a] - 1.0) / 2.0 : n_per[a] * n_per[b];
    nm.volume = rp.L[0] * rp.L[1] * rp.L[2];
    nm.dr = r_max / n_bins;
    nm.n_configs = n_configs;
    launch_rdf_gr(counts, nm, p, n_bins, g, c->st);
    return cuda_check(c, cudaGetLastError(), "g(r) kernel");
}

int pimd_cv_histogram(pimd_ctx* c, int replica, double s_min, double s_max, int n_bins, double log_w_shift,
                      double* hist, double* wsum)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!c->d.metad.cv) return fail(c, PIMD_ERR_STATE, "no collective variable configured (cfg.metad)");
    int rc = check_replica(c, replica);
    if (rc) return rc;
    if (!hist || !wsum) return fail(c, PIMD_ERR_INVALID_ARG, "hist or wsum is NULL");
    if (n_bins < 1 || n_bins > (1 << 20)) return fail(c, PIMD_ERR_INVALID_ARG, "n_bins must be 1..2^20");
    if (!(s_max > s_min)) return fail(c, PIMD_ERR_INVALID_ARG, "s_max must exceed s_min");
    if (!std::isfinite(log_w_shift)) return fail(c, PIMD_ERR_INVALID_ARG, "log_w_shift is not finite");
    const Rep& rp = c->build.reps[replica];
    const double kTP = KB * c->build.repT[replica] * rp.P;
    launch_cv_hist(c->d, replica, rp.bs0, rp.P, kTP, s_min, n_bins / (s_max - s_min), n_bins, log_w_shift, hist,
                   wsum, c->st);
    return cuda_check(c, cudaGetLastError(), "cv histogram kernel");
}

int pimd_pi_fes(pimd_ctx* c, int replica, const double* hist, const double* wsum, double s_min, double s_max,
                int n_bins, double* F, double* Fk)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    int rc = check_replica(c, replica);
    if (rc) return rc;
    if (!hist || !wsum || !F) return fail(c, PIMD_ERR_INVALID_ARG, "hist, wsum or F is NULL");
    if (n_bins < 1 || n_bins > (1 << 20)) return fail(c, PIMD_ERR_INVALID_ARG, "n_bins must be 1..2^20");
    if (!(s_max > s_min)) return fail(c, PIMD_ERR_INVALID_ARG, "s_max must exceed s_min");
    const Rep& rp = c->build.reps[replica];
    launch_pi_fes(hist, wsum, rp.P, n_bins, (s_max - s_min) / n_bins, KB * c->build.repT[replica], F, Fk, c->st);
    return cuda_check(c, cudaGetLastError(), "path-integral FES kernel");
}

int pimd_metad_fes(pimd_ctx* c, int replica, const double* s, int n, double* F)
{
    if (!c) return fail(nullptr, PIMD_ERR_INVALID_ARG, "ctx is NULL");
    if (!c->d.metad.cv) return fail(c, PIMD_ERR_STATE, "no metadynamics bias configured");
    int rc = check_replica(c, replica);
    if (rc) return rc;
    if (n < 0) return fail(c, PIMD_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return PIMD_OK;
    if (!s || !F) return fail(c, PIMD_ERR_INVALID_ARG, "s or F is NULL");
    launch_metad_fes(c->d, replica, s, n, F, c->st);
    return cuda_check(c, cudaGetLastError(), "metadynamics FES kernel");
}

void pimd_destroy(pimd_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->st);
    drop_graphs(c);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (int k = 0; k < MAX_PARTS; ++k) {
        if (c->capx[k]) cudaStreamDestroy(c->capx[k]);
        if (c->ev_fwd[k]) cudaEventDestroy(c->ev_fwd[k]);
        if (c->ev_end[k]) cudaEventDestroy(c->ev_end[k]);
    }
    for (int i = 0; i <= PIMD_N_STAGES; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    delete c;
}

const char* pimd_last_error(const pimd_ctx* c)
{
    if (c) return c->err.c_str();
    return g_tls_error.c_str();
}

}  // extern "C"
