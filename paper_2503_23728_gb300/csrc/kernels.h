// kernels.h -- host-side declarations of the kernel launchers (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "common.cuh"

namespace pimd {

// Device pointers and sizes of one context (all inside the caller's workspace).
constexpr int MAX_PARTS = 4;   // overlapping parts of a step's force evaluation

struct Dev {
    int R = 0, S = 0, B = 0, NA = 0;   // replicas, bead-systems, bead-atoms, atoms
    int max_N = 0;                     // largest replica
    int maxnb = 128;
    int precision = 1;                 // 0 FP64, 1 FP32, 2 BF16 tensor cores
    bool periodic_any = false;

    Rep* reps = nullptr;
    BeadSys* bsys = nullptr;
    int* ba_sys = nullptr;             // [B] bead-system of each bead-atom
    int4* ba_info = nullptr;           // [B] (bead-system, its first bead-atom, its atoms, replica)
    double* mass = nullptr;            // [NA]
    double2* minv = nullptr;           // [NA] (1 / m, sqrt(m k_B T_P) of the atom's replica)
    int* atype = nullptr;              // [NA] element type index
    double* x0 = nullptr;              // [NA][3]
    double* cmat = nullptr;            // normal-mode matrices
    float* cmatf = nullptr;            // the same in FP32 (FP32 paths)
    Mode* modes = nullptr;             // [sum P]
    int2* rp_blocks = nullptr;         // (replica, first entry) per ring-polymer block
    int n_rp_blocks = 0;
    int rp_threads = 256;
    int rp_stage_P = 0;                // largest P <= 64 among the replicas (transform rows staged per block)
    int unit_mfac = 0;                 // every ring coordinate has the atom's mass (normal modes): skip the factors

    void* x = nullptr;                 // Vec4<Real>[B] positions (w = type)
    void* f = nullptr;                 // Vec4<Real>[B] forces
    int* nbr = nullptr;                // [B][maxnb]
    int* nnb = nullptr;                // [B]
    int* cell_start = nullptr;         // per cell: first slot in cell_atoms
    int* cell_cnt = nullptr;           // per cell: atom count
    int* cell_atoms = nullptr;         // [B] atoms of each bead grouped by cell
    int* cell_bs = nullptr;            // beads that use cell lists
    int* cand = nullptr;               // [B][maxcand] Verlet candidate lists (r < r_c + skin)
    int* ncand = nullptr;              // [B]
    float4* xref = nullptr;            // [B] FP32 positions at the last candidate build
    int* rebuild = nullptr;            // [S] 1: rebuild this bead's candidates now
    int maxcand = 0;                   // 0: no replica uses a skin
    int n_cell_bs = 0, max_cells = 0;
    void* G = nullptr;                 // Real[B][64]
    void* dEdG = nullptr;              // Real[B][64]
    void* Eatom = nullptr;             // Real[B]
    double* V = nullptr;               // [S]
    double* W = nullptr;               // [S][9]
    double* q = nullptr;               // [3B] normal-mode positions
    double* p = nullptr;               // [3B] normal-mode momenta
    double* fnm = nullptr;             // [3B] normal-mode forces
    double* Q = nullptr;               // [R] thermostat heat
    double* qpart = nullptr;           // [3][n_rp_blocks] thermostat heat per block: start half (two buffers), finish half
    int* rep_blk0 = nullptr;           // [R + 1] first ring-polymer block of each replica
    unsigned long long* step_cur = nullptr;   // the step being taken (copied by the ring start for the ring finish)
    void* wbuf = nullptr;              // Real[B][9] per bead-atom virial
    void* vbuf = nullptr;              // Vec4<Real>[B][maxnb] pair vectors (deterministic mode)
    void* mom = nullptr;               // float4[B][6][32] angular moments (moment path, FP32)
    int max_P = 1;                     // largest bead count

    // metadynamics (md_* in the workspace when metad.cv != 0)
    MetadParams metad = {};
    double2* md_hills = nullptr;       // [R][max_hills] (centre, height)
    int* md_nhill = nullptr;           // [R]
    double* md_cv = nullptr;           // [S] CV of each bead at the last evaluation
    double* md_vb = nullptr;           // [S] bias
    double* md_dvds = nullptr;         // [S] dV/ds
    double* md_cvpart = nullptr;       // [S][tiles] CV partial sums
    double* md_virpart = nullptr;      // [S][tiles][9] pair-virial partial sums
    void* md_grad = nullptr;           // Vec4<Real>[B] ds/dx
    int deterministic = 0;
    unsigned long long* step = nullptr;
    DevErr* err = nullptr;
    double* est = nullptr;             // [R][EST_STRIDE]

    // graph-field-network head (potential PIMD_POT_GFN)
    GfnParams gfn = {};
    float* gfn_w = nullptr;            // FP32 parameters (layout in GfnParams)
    float* gfn_n = nullptr;            // [B][F] node representations
    float* gfn_m = nullptr;            // [B][F] messages
    float* gfn_e = nullptr;            // [B][maxnb][F] edge representations
    unsigned char* gfn_wtc = nullptr;  // BF16 weight images (tensor-core path)

    // network
    int n_types = 0, n_hidden = 0, width = 0;
    size_t blob = 0;                   // elements per type blob
    void* wts = nullptr;               // Real[n_types][blob]
    int* perm = nullptr;               // [rows_pad] bead-atom of each network row, -1 pad
    int* tile_type = nullptr;          // [rows_pad / 128]
    int rows_pad = 0;
    // two halves of the bead-atoms (whole bead-systems) for overlapping
    // parts of the step's force evaluation run as overlapping graph branches:
    // part k owns bead-atoms [part_ba[k], part_ba[k + 1]) and network tiles
    // [part_tile[k], part_tile[k + 1]); n_parts = 1: one branch
    int n_parts = 1;
    int part_ba[MAX_PARTS + 1] = {};
    int part_tile[MAX_PARTS + 1] = {};
    void* wtc = nullptr;               // tensor-core weight images
    size_t wtc_bytes_per_type = 0;
    float* wtc_vec = nullptr;          // FP32 vectors for the tensor-core epilogues
    size_t wtc_vec_per_type = 0;

    Sched sched = {8, 40, 0};          // pair schedule (band length 8, bands for n >= 40)

    // integrator
    double dt = 0.5, gamma0 = 0.0, lambda = 1.0;
    int thermostat = 1;
    int splitting = 0;                 // 0 OBABO, 1 BAOAB
    int potential = 0;
    double omega_harm = 0.0;
    double rc = 6.0;
};

constexpr int EST_STRIDE = 24;

// histogram bin edges passed by value to the analysis kernels
constexpr int ANALYSIS_MAX_BINS = 1024;
struct BinEdges {
    float e[ANALYSIS_MAX_BINS + 1];
};

size_t blob_elems(int n_hidden, const int* widths);

// force evaluation pieces
void launch_neighbours(const Dev& d, cudaStream_t st);
void launch_neighbour_prep(const Dev& d, cudaStream_t st);
void launch_neighbour_lists(const Dev& d, int b0, int b1, cudaStream_t st);
void launch_descriptors(const Dev& d, const void* dp, cudaStream_t st);
void launch_network_fp(const Dev& d, cudaStream_t st);
void launch_network_tc(const Dev& d, cudaStream_t st);
// halves of a step's bead-atoms as overlapping branches (BF16 moment path)
bool moment_fast_path(const Dev& d, const void* dp);
void launch_descriptors_range(const Dev& d, const void* dp, int b0, int b1, cudaStream_t st);
void launch_adjoint_range(const Dev& d, const void* dp, int b0, int b1, cudaStream_t st);
// urgent: the network's blocks at the highest stream priority
bool launch_network_tiles(const Dev& d, int t0, int nt, cudaStream_t st, bool urgent = false);
bool network_tiles_available(const Dev& d);
void launch_adjoint(const Dev& d, const void* dp, cudaStream_t st);
// true when the adjoint kernel also sums the per-bead energies V and virials
// W (FP64 atomics; V and W zeroed before): the energy reduction is skipped
bool adjoint_sums_energy(const Dev& d, const void* dp);
bool moment_adjoint_sums_energy(const Dev& d, const void* dp);
void launch_gfn(const Dev& d, cudaStream_t st);
void launch_gfn_tc(const Dev& d, cudaStream_t st);
size_t gfn_tc_image_bytes(int F, int L);
int gfn_kernels_per_eval(int L);
void launch_descriptors_moment(const Dev& d, const void* dp, cudaStream_t st);
void launch_adjoint_moment(const Dev& d, const void* dp, cudaStream_t st);
size_t moment_elems_per_atom();        // float4 moments per bead-atom
void launch_energy_reduce(const Dev& d, cudaStream_t st);
void launch_force_gather(const Dev& d, cudaStream_t st);
void launch_harmonic(const Dev& d, cudaStream_t st);
void launch_pack_positions(const Dev& d, const double* x3, cudaStream_t st);
void launch_pack_forces(const Dev& d, const double* f3, cudaStream_t st);
void launch_unpack(const Dev& d, double* f3, double* e, double* vir, double* x3, cudaStream_t st);
void launch_descriptors_out(const Dev& d, double* G, cudaStream_t st);
bool network_tc_supported(int width, int n_hidden);
size_t tc_weight_bytes(int width, int n_hidden);
void prepare_tc_weights(const Dev& d, int type, const double* blob, void* host_img, float* host_vec);

// metadynamics
constexpr int MD_SLICES = 8;           // XRD CV: row slices per atom tile (gradient buffers)
int metad_tiles(int max_N);            // partial sums per bead-system (tiles x slices)
void launch_metad(const Dev& d, bool deposit, cudaStream_t st, int step_offset = 0);

// structural analysis
size_t rdf_smem_bytes(int n_types, int n_bins);
void launch_rdf(const Dev& d, int rep, int P, int N, const BinEdges& edges, int n_bins, float inv_dr,
                unsigned long long* counts, cudaStream_t st);
// normalisation of RDF counts: ideal-gas pairs per element pair, box volume,
// shell width, number of configurations summed
constexpr int RDF_MAX_PAIRS = 36;   // element pairs of up to 8 types
struct RdfNorm {
    double pairs[RDF_MAX_PAIRS];
    double volume, dr, n_configs;
};
void launch_rdf_gr(const unsigned long long* counts, const RdfNorm& nm, int n_pairs, int n_bins, double* g,
                   cudaStream_t st);
void launch_cv_hist(const Dev& d, int replica, int bs0, int P, double kTP, double s_min, double inv_ds, int n_bins,
                    double shift, double* hist, double* wsum, cudaStream_t st);
void launch_pi_fes(const double* hist, const double* wsum, int P, int n_bins, double ds, double kT, double* F,
                   double* Fk, cudaStream_t st);
void launch_metad_fes(const Dev& d, int replica, const double* s, int n, double* F, cudaStream_t st);
void launch_pt(const Dev& d, int rep, int P, int N, const int* bond, int t_acc, const BinEdges& edges, int n_bins,
               float inv_w, float* v_out, unsigned long long* hist, cudaStream_t st);

// bounded-wait self-test (mlp_tc.cu): 0 on success, *timed_out = 1 when the bound expired
int run_wait_selftest(cudaStream_t st, long long cycles, int* timed_out);

// message returned by pimd_last_error(NULL) on this thread
void set_thread_error(const std::string& msg);

// ring polymer
void launch_rp_init(const Dev& d, cudaStream_t st);
void launch_beads(const Dev& d, cudaStream_t st);
// lo: which of the two start-half heat buffers (0 / 1) a ring start writes and
// an ordered heat sum reads; offset: steps since the call's first ring start
void launch_rp_start(const Dev& d, cudaStream_t st, int lo = 0);
void launch_rp_finish(const Dev& d, bool do_step, cudaStream_t st, int offset = 0);
void launch_rp_finish_start(const Dev& d, int offset, int lo, cudaStream_t st);
void launch_heat_sum(const Dev& d, int lo, cudaStream_t st);
void launch_estimators(const Dev& d, cudaStream_t st);

}  // namespace pimd
