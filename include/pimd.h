/*
 * pimd.h -- C ABI of the GB300 path-integral molecular dynamics library with a
 * symmetry-function neural-network potential.
 *
 * The library advances ring polymers (paper Sec. 2.1: effective Hamiltonian
 * with P beads per atom, normal-mode transformation, H_eff = H_p + U) whose
 * potential U is a per-element network on radial/angular symmetry functions
 * (the descriptor-based energy model of Sec. 1, ref. [17]); forces are the
 * analytic gradient of that energy (Sec. 2.2). One context holds any number
 * of independent replicas with their own N, P, temperature and seed (the
 * multi-trajectory mode of Sec. 2.3), all advanced by the same launches.
 *
 * Conventions
 *   units: Angstrom, fs, amu, eV, K.
 *   ring polymer: i-PI form, beta_P = beta / P, omega_P = P k_B T / hbar,
 *   sampled at T_P = P T (equivalent to Sec. 2.1 after dividing by P).
 *   bead-atom order: replica-major, then bead, then atom.
 *   normal-mode state: per replica [P][N][3] FP64, replicas concatenated.
 *
 * Memory ownership
 *   The library never allocates device memory. The caller passes one device
 *   workspace to pimd_create (size from pimd_workspace_size) and keeps it
 *   alive until pimd_destroy. Host arrays passed in are copied before the
 *   call returns. Device pointers passed to pimd_energy_forces /
 *   pimd_descriptors are caller-owned and used stream-ordered on the
 *   context's stream.
 *
 * Errors
 *   Every call returns a pimd_status. Argument and state errors leave the
 *   context unchanged. Errors detected on the device (non-finite forces,
 *   neighbour overflow) are reported at the next synchronising call
 *   (pimd_sync, pimd_estimators, pimd_get_state, pimd_get_forces). A CUDA
 *   error is sticky: destroy the context. Nothing here throws or exits.
 */
#ifndef PIMD_H
#define PIMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIMD_ABI_VERSION 3
#define PIMD_N_RADIAL 32
#define PIMD_N_ANGULAR 32
#define PIMD_N_DESC 64
#define PIMD_MAX_ELEMENTS 8
#define PIMD_MAX_LAYERS 4
#define PIMD_MAX_WIDTH 256
#define PIMD_MAX_BEADS 256
#define PIMD_MAX_NEIGHBOURS 256

typedef enum {
    PIMD_OK = 0,
    PIMD_ERR_INVALID_ARG = -1,
    PIMD_ERR_STATE = -2,
    PIMD_ERR_WORKSPACE_TOO_SMALL = -3,
    PIMD_ERR_CUDA = -4,
    PIMD_ERR_NONFINITE = -5,
    PIMD_ERR_TIMEOUT = -6,
    PIMD_ERR_NBR_OVERFLOW = -7,
    PIMD_ERR_UNSUPPORTED = -8,
    PIMD_ERR_METAD_FULL = -9
} pimd_status;

/* arithmetic of the force evaluation */
typedef enum {
    PIMD_FP64 = 0,     /* descriptors, network, adjoint all FP64                    */
    PIMD_FP32 = 1,     /* FP32 descriptors/adjoint, FP32 network on CUDA cores      */
    PIMD_BF16_TC = 2   /* FP32 descriptors/adjoint, BF16 network on tcgen05 tensor
                          cores with FP32 accumulation in tensor memory            */
} pimd_precision;

/* how the angular symmetry functions and their adjoint are evaluated */
typedef enum {
    PIMD_ANG_PAIRS = 0,   /* sums over the unordered neighbour pairs, O(n^2) per atom */
    PIMD_ANG_MOMENTS = 1  /* moment tensors of degree <= 8, O(n) per atom (FP32 and
                             BF16 precision; same values up to rounding)           */
} pimd_angular;

/* order of the sub-steps of one time step dt (O: PILE-L thermostat, B: force
 * kick, A: free ring-polymer evolution, all in normal-mode space) */
typedef enum {
    PIMD_OBABO = 0,   /* O(dt/2) B(dt/2) A(dt) [forces] B(dt/2) O(dt/2); noise
                         streams 2 and 3                                       */
    PIMD_BAOAB = 1    /* B(dt/2) A(dt/2) O(dt) A(dt/2) [forces] B(dt/2); noise
                         stream 2                                              */
} pimd_splitting;

/* coordinates of the ring-polymer state (pimd_get_state / pimd_set_state) */
typedef enum {
    PIMD_TRANSFORM_NORMAL_MODES = 0,  /* orthogonal normal modes, mass m, frequencies
                                         omega_k = 2 omega_P sin(k pi / P)        */
    PIMD_TRANSFORM_STAGING = 1        /* staging u_1 = x_1, u_k = x_k - ((k-1) x_(k+1)
                                         + x_1) / k, masses k/(k-1) m (k >= 2), all
                                         at omega_P; u_1 drifts freely           */
} pimd_transform;

/* free ring-polymer step of each internal mode k over a time h */
typedef enum {
    PIMD_FREE_RP_EXACT = 0,   /* exp(h L_k): rotation by omega_k h            */
    PIMD_FREE_RP_CAYLEY = 1   /* Cayley transform (1 - h L_k/2)^-1 (1 + h L_k/2):
                                 rotation by 2 atan(omega_k h / 2), stable for
                                 any omega_k h                                 */
} pimd_free_rp;

typedef enum {
    PIMD_POT_MODEL = 0,     /* symmetry-function network (set by pimd_set_weights)  */
    PIMD_POT_HARMONIC = 1,  /* V = sum_i 1/2 m_i omega^2 |x_i|^2 (Sec. S1 test case) */
    PIMD_POT_GFN = 2        /* graph-field-network force head (Sec. 2.2, set by
                               pimd_set_gfn): forces read out directly from edge
                               representations, no energy (per-bead V = 0, so
                               the energy estimators carry only the ring-polymer
                               terms); FP32 (CUDA cores) or BF16 precision
                               (tensor cores, F = 64 or 128)                     */
} pimd_potential;

/* ---- well-tempered metadynamics (Sec. 2.5) --------------------------------
 * A bias V(s) = sum_k h_k exp(-(s - s_k)^2 / (2 sigma^2)) on a collective
 * variable s of every bead; each replica keeps its own hills. Hills go down
 * after the force evaluation of step n when (n + 1) % stride == 0: one per
 * bead at its CV, height (h0 / P) exp(-V(s_k) / (k_B T (gamma - 1))) with
 * the bias before the deposition, T the replica's physical temperature.
 * They act from the next force evaluation on. The bias enters each bead's
 * potential, forces and virial (and so the estimators).                     */
enum {
    PIMD_CV_NONE = 0,
    PIMD_CV_DISTANCES = 1,   /* s = sum_t c_t |x_(j_t) - x_(i_t)| (minimum image);
                                e.g. the dimer's proton-transfer CV (Sec. 3.1)  */
    PIMD_CV_XRD = 2          /* s = (1/N) sum_i sum_j f_i f_j sin(Q R_ij) / (Q R_ij),
                                i = j terms f_i^2 (Sec. S3)                      */
};

typedef struct {
    int cv;                  /* PIMD_CV_*                                       */
    int n_terms;             /* DISTANCES: 1..8 terms                           */
    int term_i[8], term_j[8];/* DISTANCES: replica-local atom indices           */
    double term_c[8];        /* DISTANCES: coefficients                         */
    double xrd_Q;            /* XRD: |Q| = 4 pi sin(theta) / lambda, 1/A        */
    double xrd_f[PIMD_MAX_ELEMENTS]; /* XRD: scattering factor of each element
                                in ascending-Z order (pimd_element_types)      */
    double height_eV;        /* h0 >= 0 (0: the CV of every bead, no bias)      */
    double sigma;            /* Gaussian width > 0, CV units                    */
    double bias_factor;      /* gamma > 1                                       */
    int stride;              /* steps between depositions >= 1                  */
    int max_hills;           /* hill capacity per replica (a deposition adds P);
                                a deposition that does not fit sets
                                PIMD_ERR_METAD_FULL at the next sync            */
} pimd_metad_desc;

typedef struct {
    double dt_fs;            /* time step                                          */
    double gamma0_per_fs;    /* PILE-L centroid friction 1/tau_0                   */
    double pile_lambda;      /* internal-mode friction gamma_k = 2 lambda omega_k  */
    double cutoff_A;         /* symmetry-function cutoff r_c (graph edges)         */
    int precision;           /* pimd_precision                                     */
    int thermostat;          /* 0 = NVE, 1 = PILE-L                                */
    int potential;           /* pimd_potential                                     */
    int max_neighbours;      /* neighbour slots per atom, multiple of 32, <= 256;
                                0 selects 128                                      */
    double omega_harm;       /* 1/fs, PIMD_POT_HARMONIC only                       */
    int n_hidden;            /* network hidden layers (1..4)                       */
    int widths[PIMD_MAX_LAYERS]; /* hidden widths, each a multiple of 32, <= 256   */
    void* stream;            /* cudaStream_t for all work; NULL = default stream   */
    int timing;              /* nonzero: record CUDA events around every stage of
                                a step (see pimd_stage_times)                      */
    int nbr_algo;            /* 0: cell lists where a periodic box holds >= 3
                                cells of edge >= cutoff per side and the stencil
                                scan is cheaper than scanning the bead, else all
                                pairs; 1: all pairs; 2: cells wherever the box
                                allows. Same lists in every case.                 */
    int deterministic;       /* 1: forces summed in a fixed order (pair vectors
                                stored, then gathered per atom; small neighbour
                                counts use ordered pairs), so runs and resumed
                                runs are bit-identical. Costs B*max_neighbours
                                records of workspace and one more kernel.
                                0: atomic force accumulation (faster).           */
    int splitting;           /* pimd_splitting: order of the step's sub-steps    */
    int free_rp;             /* pimd_free_rp: free ring-polymer propagator       */
    const pimd_metad_desc* metad; /* NULL: no bias. Read during pimd_workspace_size
                                and pimd_create only.                          */
    double nbr_skin_A;       /* Verlet skin of the neighbour candidates: each
                                bead keeps the atoms within r_c + skin, rebuilt
                                when the two largest atom displacements since the
                                last build add up to 0.98 skin; every step filters
                                them with the exact rule, so the lists equal a
                                full rebuild. < 0: 1.5 A for replicas of >= 256
                                atoms (reduced to 0.9 of the room between r_c
                                and half the box, off below 0.05 A), none for
                                smaller ones; 0: rebuild every step.           */
    int transform;           /* pimd_transform: ring-polymer coordinates       */
    int gfn_features;        /* PIMD_POT_GFN: feature width F of node and edge
                                representations: 32, 64 or 128                */
    int gfn_iterations;      /* PIMD_POT_GFN: message-passing iterations L, 0..8 */
} pimd_config;

/* stages of one step, in launch order (pimd_stage_times) */
enum {
    PIMD_STAGE_RING_START = 0,   /* O B A in normal-mode space + beads           */
    PIMD_STAGE_NEIGHBOURS = 1,   /* neighbour lists                              */
    PIMD_STAGE_DESCRIPTORS = 2,  /* radial + angular symmetry functions          */
    PIMD_STAGE_NETWORK = 3,      /* per-element network forward + input gradient */
    PIMD_STAGE_ADJOINT = 4,      /* forces and virial                            */
    PIMD_STAGE_ENERGY = 5,       /* per-bead energies                            */
    PIMD_STAGE_RING_FINISH = 6,  /* C^T f, B O, step counter                     */
    PIMD_N_STAGES = 7
};

typedef struct {
    int n_atoms;             /* N >= 1                                             */
    int n_beads;             /* P, 1..256                                          */
    const int* Z;            /* host [N] element numbers                           */
    const double* x0;        /* host [N][3] initial positions (all beads start here) */
    const double* mass;      /* host [N] amu, or NULL for standard masses of H C N O */
    double box[3];           /* orthorhombic periodic box; all 0 = non-periodic.
                                Periodic boxes need min(box) >= 2 cutoff            */
    double T_K;              /* physical temperature                               */
    uint64_t seed;           /* Philox key of this replica's noise                 */
} pimd_replica_desc;

/* Per-element network on the descriptor G (64 = 32 radial + 32 angular):
 *   h_0 = (G - mu) / sigma,  h_l = tanh(W_l h_{l-1} + b_l),
 *   E_i = s_E (w_out . h_L + b_out) + e_Z.
 * params[e] is element Z[e]'s flat FP64 host blob in this order:
 *   for each hidden layer l: W_l [h_l][h_{l-1}] row-major, b_l [h_l];
 *   w_out [h_L]; b_out; mu [64]; sigma [64]; s_E; e_Z.
 * Descriptors (cutoff fc(r) = (cos(pi r / r_c) + 1) / 2 for r < r_c):
 *   G[mu]      = sum_j exp(-eta_R (r_ij - r_mu[mu])^2) fc(r_ij),    mu < 32
 *   G[32 + nu] = 2^(1-zeta) sum_{j<k} (1 + lambda cos theta_jik)^zeta
 *                exp(-eta_A (r_ij^2 + r_ik^2)) fc(r_ij) fc(r_ik)
 *   with nu = (zeta_index * 2 + lambda_index) * 4 + eta_index; zeta must be
 *   {1, 2, 4, 8} and lambda {+1, -1} in that order.                        */
typedef struct {
    int n_elements;
    const int* Z;                 /* [n_elements]                                  */
    int n_hidden;                 /* must equal pimd_config.n_hidden               */
    const int* widths;            /* [n_hidden], must equal pimd_config.widths     */
    const double* const* params;  /* [n_elements] host blobs (layout above)        */
    double eta_R;
    const double* r_mu;           /* [32]                                          */
    const int* zeta;              /* [4]                                           */
    const double* lambda;         /* [2]                                           */
    const double* eta_A;          /* [4]                                           */
} pimd_model_desc;

/* per-replica estimators (finite-P ensemble averages of Sec. 2.1), eV */
typedef struct {
    double V_mean;     /* (1/P) sum_k V_k                                          */
    double K_prim;     /* primitive kinetic-energy estimator                       */
    double K_cv;       /* centroid-virial kinetic-energy estimator                 */
    double E_tot;      /* K_cv + V_mean                                            */
    double W[9];       /* bead-averaged virial tensor, W_ab = sum_i x_a f_b form    */
    double H_cons;     /* ring-polymer Hamiltonian minus thermostat heat           */
    double Q_thermo;   /* kinetic energy added by all thermostat steps             */
    double T_kin;      /* ring-polymer kinetic temperature (expect P T), K         */
    double nbr_mean;   /* mean neighbours per bead-atom at the last evaluation     */
    double nbr_max;    /* largest neighbour count at the last evaluation           */
} pimd_est;

typedef struct pimd_ctx pimd_ctx;

/* Device workspace bytes needed for this configuration and replica set.
 * Errors: INVALID_ARG for NULL pointers or inconsistent sizes.            */
int pimd_workspace_size(const pimd_config* cfg, const pimd_replica_desc* reps, int n_reps,
                        size_t* bytes);

/* Create a context. Initial state (Sec. 2.1 ring polymer): every bead at x0,
 * normal-mode momenta drawn from N(0, m k_B T_P) with Philox stream 1.
 * `workspace` is a caller-owned device buffer of >= pimd_workspace_size bytes,
 * aligned to 256 bytes. Errors: INVALID_ARG, WORKSPACE_TOO_SMALL, CUDA.      */
int pimd_create(const pimd_config* cfg, const pimd_replica_desc* reps, int n_reps,
                void* workspace, size_t ws_bytes, pimd_ctx** out);

/* Load the network (FP64 host parameters, converted to the working precision)
 * and evaluate forces at the current state. Every element present in the
 * replicas must be in the model. Errors: INVALID_ARG (shape mismatch, missing
 * element, unsupported zeta/lambda), STATE (potential is not PIMD_POT_MODEL). */
int pimd_set_weights(pimd_ctx* ctx, const pimd_model_desc* model);

/* Advance all replicas by n_steps of OBABO in normal-mode space:
 * O(dt/2) B(dt/2) A(dt) [forces] B(dt/2) O(dt/2) with exact free-ring-polymer
 * A and PILE-L O (Philox counter: index, step, replica, stream 2 / 3).
 * Runs of 8 steps are one graph launch whose inner step boundaries fuse the
 * ring finish with the next ring start (the same bits as separate kernels);
 * the state after the call is the state after the last step's ring finish.
 * Asynchronous on the context stream. Errors: STATE if weights are missing. */
int pimd_step(pimd_ctx* ctx, int n_steps);

/* ---- graph-field-network force head (Sec. 2.2) ----------------------------
 * With F features and L iterations (pimd_config.gfn_features / _iterations)
 * and SiLU activations:
 *   n_i^(0) = emb[Z_i],  e_ij^(0) = W_e rho(r_ij) + b_e,
 *     rho_mu(r) = exp(-eta_R (r - r_mu)^2) fc(r), mu = 0..31, fc the cosine
 *     cutoff at pimd_config.cutoff_A;
 *   for l = 0 .. L-1:
 *     m_i     = sum_{j in N(i)} SiLU(W_m e_ij + b_m)
 *     n_i'    = n_i + W_v2 SiLU(W_v1 [n_i; m_i] + b_v1) + b_v2
 *     e_ij'   = e_ij + W_a2 SiLU(W_a1 (n_i + n_j) + b_a1) + b_a2   (pre-update n)
 *   F_i = sum_{j in N(i)} s_F fc(r_ij) (x_i - x_j) / r_ij (w_f2 . SiLU(W_f1 e_ij^(L) + b_f1) + b_f2),
 *   virial W = 1/2 sum_i sum_j (x_i - x_j) (x) F_ij.
 * params: FP64 host blob, row-major matrices (y = W x): emb [n_el][F];
 * W_e [F][32], b_e [F]; per iteration W_m [F][F], b_m [F], W_v1 [F][2F],
 * b_v1 [F], W_v2 [F][F], b_v2 [F], W_a1 [F][F], b_a1 [F], W_a2 [F][F],
 * b_a2 [F]; then W_f1 [F][F], b_f1 [F], w_f2 [F], b_f2, s_F.                */
typedef struct {
    int n_elements;                  /* element types, 1..PIMD_MAX_ELEMENTS        */
    int Z[PIMD_MAX_ELEMENTS];        /* their atomic numbers, ascending (rows of emb) */
    const double* params;            /* host, copied during the call               */
    size_t n_params;                 /* length of params (checked against F, L)    */
    double r_mu[32];                 /* radial centres, A                          */
    double eta_R;                    /* radial width, 1/A^2                        */
} pimd_gfn_desc;

/* Set the graph-field-network parameters (converted to FP32 on the device).
 * Errors: STATE (potential is not PIMD_POT_GFN), INVALID_ARG (NULL arrays,
 * wrong n_params, Z not ascending or missing an element of the replicas,
 * non-finite parameters).                                                   */
int pimd_set_gfn(pimd_ctx* ctx, const pimd_gfn_desc* g);

/* Potential energy, forces and virial of arbitrary bead positions, without
 * touching the dynamical state. x_dev: device [B][3] FP64 positions in
 * bead-atom order (B = sum_r N_r P_r), or NULL for the current beads.
 * e_dev: device [S] FP64 per-bead energies V_k (S = sum_r P_r), may be NULL.
 * f_dev: device [B][3] FP64 forces -dV_k/dx, may be NULL.
 * virial_dev: device [S][9] FP64 per-bead virials, may be NULL.
 * Stream-ordered; returns without synchronising.                            */
int pimd_energy_forces(pimd_ctx* ctx, const double* x_dev, double* e_dev, double* f_dev,
                       double* virial_dev);

/* Raw descriptors G (before normalisation) of arbitrary bead positions:
 * x_dev as in pimd_energy_forces (NULL = current beads); G_dev: device
 * [B][64] FP64. Stream-ordered.                                             */
int pimd_descriptors(pimd_ctx* ctx, const double* x_dev, double* G_dev);

/* Synchronise and fill out_host[0..n_reps) with each replica's estimators.
 * Errors: INVALID_ARG if n_reps differs from the context's count; device
 * errors (NONFINITE, NBR_OVERFLOW) detected since the last sync.             */
int pimd_estimators(pimd_ctx* ctx, pimd_est* out_host, int n_reps);

/* Checkpoint / resume. Host arrays of 3 sum_r P_r N_r doubles each (normal-
 * mode positions and momenta), the step counter and the accumulated
 * thermostat heat per replica ([n_reps]). set_state recomputes forces; a
 * resumed run is bit-identical to an uninterrupted one. get_state syncs.    */
int pimd_get_state(pimd_ctx* ctx, double* q_nm, double* p_nm, uint64_t* step, double* Q_thermo);
int pimd_set_state(pimd_ctx* ctx, const double* q_nm, const double* p_nm, uint64_t step,
                   const double* Q_thermo);

/* Current bead positions [B][3], forces [B][3] and per-bead energies [S]
 * copied to host arrays (any may be NULL). Synchronises.                     */
int pimd_get_forces(pimd_ctx* ctx, double* x_host, double* f_host, double* V_host);

/* Neighbour lists of the last force evaluation: nnb_host [B] counts and
 * nbr_host [B][max_neighbours] atom indices within each bead (ascending).
 * Synchronises.                                                             */
int pimd_get_neighbours(pimd_ctx* ctx, int* nnb_host, int* nbr_host);

/* Device time (ms) of each stage of the last step of the most recent
 * pimd_step call that ran with stage timing on, measured with CUDA events
 * recorded inside the step's graph on the context stream (requires
 * cfg.timing). ms: host [PIMD_N_STAGES]. Synchronises. Errors: STATE without
 * timing or before the first marked step.                                   */
int pimd_stage_times(pimd_ctx* ctx, float* ms);

/* ---- ring-polymer step with forces from elsewhere (bead-sharded runs) -----
 * The OBABO step cut at its force evaluation (Sec. 2.1: the beads of a ring
 * polymer interact only through the springs of the ring-polymer step, so
 * the forces of different beads can be evaluated apart). A run whose beads
 * are spread over several GPUs gives each GPU a context holding all beads of
 * a slice of the atoms (typically PIMD_POT_HARMONIC with omega_harm = 0, so
 * that it evaluates no forces of its own) and advances it with:
 *   pimd_set_forces(ctx, f)    bead forces of the current positions, once
 *                              before the first step (and after set_state);
 *   pimd_ring_start(ctx, x)    first half: OBABO O(dt/2) B(dt/2) A(dt)
 *                              (BAOAB: B A O A) with the current forces, then
 *                              the new bead positions into x;
 *   pimd_ring_finish(ctx, f)   second half: B(dt/2) with the forces f of
 *                              those positions, then O(dt/2); the step ends.
 * x, f: device FP64 [sum P][N][3] in the context's (replica, bead, atom)
 * order; f is rounded to the working precision like the library's own
 * forces. pimd_set_noise_index makes replica `replica` draw its thermostat
 * noise as atoms atom_offset .. of a system of n_atoms_total atoms, so that
 * slices of one system reproduce the whole system's trajectory, and resets
 * the replica's initial state (all beads at x0, momenta drawn at the new
 * indices, step 0, no heat): call it right after pimd_create. Energies are
 * not part of external forces, so the estimators of such a context hold the
 * ring-polymer terms only. Context stream, no synchronisation except in
 * pimd_set_noise_index. Errors: INVALID_ARG, STATE (start without forces,
 * finish without a start). The paper has no counterpart of the split; it is
 * the decomposition of its Sec. 2.1 step.                                   */
int pimd_set_noise_index(pimd_ctx* ctx, int replica, int atom_offset, int n_atoms_total);
int pimd_set_forces(pimd_ctx* ctx, const double* f);
int pimd_ring_start(pimd_ctx* ctx, double* x);
int pimd_ring_finish(pimd_ctx* ctx, const double* f);

/* Overlapped parts (default on). Contexts of at least 16,384 bead-atoms on
 * the BF16 path with networks of width 64 or 128 (whose hidden activations
 * fit in tensor memory) split their bead-atoms into two parts of whole
 * beads, the first with about 3/8 of the bead-atoms; a step then runs the
 * first part's network and adjoint beside the second part's descriptors and
 * network (two branches of the step's graph), so the network's short
 * latency-bound launches and the last waves of every kernel are filled with
 * the other part's work. Results are the same either way (every
 * bead-atom's arithmetic is unchanged). Steps that carry the stage markers
 * always run the parts one after the other. Returns 1 when the context has
 * parts, 0 when it runs one branch anyway, < 0 on error. The paper has no
 * counterpart (a scheduling choice).                                       */
int pimd_set_overlap(pimd_ctx* ctx, int on);

/* Stage timing on (default for cfg.timing contexts) or off. The event
 * records that time the stages are nodes of the step's graph and cost some
 * microseconds each, so with timing on only the last step of each pimd_step
 * call carries them, and with it off no step does (the step then runs as
 * fast as without cfg.timing). Errors: STATE without cfg.timing. The paper
 * has no counterpart (instrumentation).                                     */
int pimd_set_stage_timing(pimd_ctx* ctx, int on);

/* Autotuner. Times the descriptor + adjoint kernels on the context's current
 * configuration for each candidate (pair sums with band length 4..16 of the
 * shuffle-carry schedule, ordered pairs, and -- in FP32 / BF16 precision --
 * moment tensors, in BF16 with the adjoint at 12 and at 16 warps per SM)
 * and keeps the fastest; the per-step graphs are re-recorded
 * at the next pimd_step. reps: timed repetitions per candidate (>= 1).
 * out_ms: host [3] or NULL -> best time (ms, descriptors + adjoint), the
 * choice (band length, 0 = ordered pairs, -1 = moment tensors), time of the
 * schedule in force before the call. Synchronises. Errors: STATE before
 * weights set.                                                              */
int pimd_tune(pimd_ctx* ctx, int reps, double* out_ms);

/* Set the pair schedule directly: band_length 1..16 (shuffle-carry bands for
 * atoms with >= band_length + 32 neighbours, ordered pairs below), or 0 for
 * ordered pairs everywhere. Errors: INVALID_ARG for other lengths.          */
int pimd_set_schedule(pimd_ctx* ctx, int band_length);

/* Choose how the angular terms are evaluated (pimd_angular). The default is
 * PIMD_ANG_MOMENTS in FP32 / BF16 precision when the mean neighbour count
 * estimated from the replicas' densities is >= 24, else PIMD_ANG_PAIRS; the
 * pair schedule of pimd_set_schedule applies to PIMD_ANG_PAIRS only.
 * Errors: INVALID_ARG (unknown algo), UNSUPPORTED (moments in FP64 or
 * without the model potential).                                             */
int pimd_set_angular(pimd_ctx* ctx, int algo);

/* The angular evaluation in force (pimd_angular), -1 for a NULL ctx.       */
int pimd_get_angular(const pimd_ctx* ctx);

/* Residency of the BF16 moment-tensor adjoint (the force kernel of the
 * BF16_TC path with moment tensors; no counterpart in the paper, a launch
 * configuration): 12 warps per SM (166 registers per thread) or 16 (a
 * 128-register build). Same arithmetic per bead-atom either way; which is
 * faster depends on the workload, so pimd_tune times both. The per-step
 * graphs are re-recorded at the next pimd_step. Errors: INVALID_ARG
 * (warps_per_sm not 12 or 16). pimd_get_adjoint_warps: the setting in force
 * (12 or 16), -1 for a NULL ctx.                                            */
int pimd_set_adjoint_warps(pimd_ctx* ctx, int warps_per_sm);
int pimd_get_adjoint_warps(const pimd_ctx* ctx);

/* Number of kernels one single-step launch runs (memset nodes not counted).
 * Inside multi-step launches the ring finish of a step and the ring start of
 * the next are one kernel, one fewer per inner step boundary.               */
int pimd_kernels_per_step(const pimd_ctx* ctx);

/* Block until all queued work is done; report device-side errors.          */
int pimd_sync(pimd_ctx* ctx);

/* Sizes of the context: bead-atoms B, bead-systems S, replicas R, slots.  */
int pimd_sizes(const pimd_ctx* ctx, int64_t* B, int64_t* S, int* R, int* max_neighbours);

void pimd_destroy(pimd_ctx* ctx);

/* Message of the last failed call on ctx (NULL ctx: the calling thread's
 * last failure outside a context). Never NULL.                              */
const char* pimd_last_error(const pimd_ctx* ctx);

int pimd_abi_version(void);

/* ---- metadynamics state (contexts created with cfg.metad) ---------------
 * pimd_metad_hills: copies up to capacity hills of the replica (centres s,
 * heights h, host arrays or NULL) and returns the number of hills (>= 0) or
 * an error (< 0; STATE without a bias). pimd_metad_set_hills replaces them
 * (checkpoint / resume; n <= max_hills). pimd_metad_cv: CV and bias of every
 * bead-system at the last force evaluation, host [S] arrays or NULL.
 * All three synchronise the context stream.                                */
int pimd_metad_hills(pimd_ctx* ctx, int replica, double* s, double* h, int capacity);
int pimd_metad_set_hills(pimd_ctx* ctx, int replica, const double* s, const double* h, int n);
int pimd_metad_cv(pimd_ctx* ctx, double* cv, double* bias);

/* ---- self-test of the bounded waits -----------------------------------------
 * The paper has no counterpart. Every spin wait in the library's kernels
 * (tensor-core MMA and copy barriers) gives up after about a second of GPU
 * clock, records PIMD_ERR_TIMEOUT and returns, so a stalled pipeline never
 * hangs the GPU. This call runs one such wait on an mbarrier that nothing
 * completes, bounded by `seconds` of SM clock (2 GHz nominal, 0 < seconds <=
 * 10), on `stream` (NULL = default), and returns PIMD_ERR_TIMEOUT when the
 * bound expired (the expected outcome) or PIMD_OK if the barrier completed.
 * Synchronises the stream. No context is involved.                         */
int pimd_selftest_bounded_wait(void* stream, double seconds);

/* ---- structural analysis of the bead configurations (Sec. 3.2) ------------
 * Both calls read the bead positions of the last force evaluation (after
 * pimd_step, pimd_energy_forces or pimd_create) of one replica, run on the
 * context stream and return without synchronising. Bins are decided in FP32
 * by the neighbour-list rule: positions rounded to FP32, minimum image in
 * FP32, r2 = (dx dx + dy dy) + dz dz without contraction; bin edges are
 * formed in FP64 and rounded to FP32, so counts are reproducible exactly.  */

/* Element numbers of the context's types in type order (ascending Z).
 * Z: host [PIMD_MAX_ELEMENTS] or NULL. Returns the number of types.       */
int pimd_element_types(const pimd_ctx* ctx, int* Z);

/* Radial-distribution pair counts (Figs. 8, 9): for every bead of the
 * replica and every pair i < j with r2 < ((n_bins) dr)^2, dr = r_max/n_bins,
 * counts[p][k] += 1 where e_k <= r2 < e_(k+1), e_k = (float)((k dr)^2), and
 * p = a (2T - a - 1) / 2 + b for the pair's types a <= b (T types).
 * counts: device [T (T + 1) / 2][n_bins] uint64, added to (the caller zeroes
 * it); g(r) follows by dividing by the ideal-gas pair count of each shell.
 * Errors: INVALID_ARG (replica, n_bins outside 1..1024, r_max <= 0 or above
 * half the smallest box edge, histogram larger than 200 KB).              */
int pimd_rdf_counts(pimd_ctx* ctx, int replica, double r_max, int n_bins, unsigned long long* counts);

/* Proton-transfer coordinate (Fig. 11): for every atom h with bond[h] >= 0
 * (the replica-local index of its bonding atom), v = d(bond, h) - the
 * smallest d(j, h) over the atoms j of element acceptor_Z other than the
 * bonding atom, sqrtf of the rule's r2, difference in FP32. bond: device
 * [N] int. v: device [P][N] float or NULL (NaN where undefined). hist:
 * device [n_bins] uint64 or NULL, += 1 where e_k <= v < e_(k+1), e_k =
 * (float)(v_min + k (v_max - v_min) / n_bins). Errors: INVALID_ARG.        */
int pimd_pt_coordinate(pimd_ctx* ctx, int replica, const int* bond, int acceptor_Z, double v_min, double v_max,
                       int n_bins, float* v, unsigned long long* hist);

/* g(r) of every element pair of a periodic replica (Figs. 8, 9) from pair
 * counts of pimd_rdf_counts summed over n_configs bead configurations (one
 * pimd_rdf_counts call adds P of them): g[p][k] = counts[p][k] /
 * (n_configs n_pairs_p shell_k / V), shell_k = 4/3 pi ((k+1)^3 - k^3) dr^3,
 * dr = r_max / n_bins, V the box volume, n_pairs_p = n_a n_b for types a != b
 * and n_a (n_a - 1) / 2 for a = b (the replica's atoms of each type).
 * counts: device [T (T + 1) / 2][n_bins] uint64; g: device, same shape,
 * FP64. Context stream, no synchronisation. Errors: INVALID_ARG (replica,
 * NULL pointers, n_bins outside 1..1024, r_max or n_configs <= 0, a
 * non-periodic replica).                                                    */
int pimd_rdf_gr(pimd_ctx* ctx, int replica, double r_max, int n_bins, double n_configs,
                const unsigned long long* counts, double* g);

/* ---- free-energy surfaces (Sec. 2.5) ---------------------------------------
 * Path-integral reweighting: the quantum free energy along the CV is
 * F(s) = -k_B T ln[(1/P) sum_k <delta(S(r^(k)) - s)>], the bead-resolved CV
 * distributions averaged over the beads. Contexts created with cfg.metad
 * evaluate the CV of every bead in each force evaluation (a zero-height,
 * never-depositing bias, h0 = 0, gives the CV without biasing).
 *
 * pimd_cv_histogram adds the replica's current configuration (the P CVs and
 * biases of the last force evaluation) as one sample: weight w = exp(sum_k
 * V_b(s_k) / (k_B T P) - log_w_shift), which removes the bias V_b from the
 * ring polymer's configurational weight (w = exp(-log_w_shift) when no hill
 * has been deposited); hist[k][b] += w for bead k's bin b = floor((s_k -
 * s_min) n_bins / (s_max - s_min)), counted only for 0 <= b < n_bins, and
 * *wsum += w for every sample. The beads are summed in order by one thread,
 * so the result does not depend on the run. hist: device [P][n_bins] FP64,
 * wsum: device [1] FP64, both accumulated (the caller zeroes them). A
 * constant log_w_shift keeps w in range over long runs and cancels in F.
 *
 * pimd_pi_fes turns such a histogram into F_k(s_b) = -k_B T ln(hist[k][b] /
 * (wsum ds)) for every bead and the path-integral F(s_b) = -k_B T ln((1/P)
 * sum_k hist[k][b] / (wsum ds)) = -k_B T ln[(1/P) sum_k exp(-F_k(s_b)/k_B T)],
 * ds = (s_max - s_min) / n_bins, T the replica's temperature, in eV; +inf in
 * empty bins. F: device [n_bins]; Fk: device [P][n_bins] or NULL.
 *
 * pimd_metad_fes gives F(s) = -(gamma / (gamma - 1)) V(s) from the
 * replica's hills (the converged well-tempered bias), s and F device [n].
 *
 * All three run on the context stream without synchronising. Errors: STATE
 * (no CV / bias configured; histogram and metad FES), INVALID_ARG.         */
int pimd_cv_histogram(pimd_ctx* ctx, int replica, double s_min, double s_max, int n_bins, double log_w_shift,
                      double* hist, double* wsum);
int pimd_pi_fes(pimd_ctx* ctx, int replica, const double* hist, const double* wsum, double s_min, double s_max,
                int n_bins, double* F, double* Fk);
int pimd_metad_fes(pimd_ctx* ctx, int replica, const double* s, int n, double* F);

/* ---- descriptors without any device allocation ------------------------------
 * The paper has no counterpart to this call. It serves callers that cannot
 * allocate device memory at all -- a host engine that reserves the whole GPU
 * for its own memory pool, a plug-in host that forbids cudaMalloc after
 * start-up -- and so cannot provide the workspace pimd_create needs.
 *
 * Computes the raw descriptors G (same definitions and FP32 arithmetic as
 * pimd_descriptors) of one configuration. x_dev: device [n_atoms][3] FP64
 * positions; box: host [3] (all 0 = non-periodic), may be NULL; r_mu: host
 * [32]; eta_A: host [4]; G_dev: device [n_atoms][64] FP64 output; stream:
 * cudaStream_t or NULL. Blocks until the result is written.
 *
 * Scratch (FP32 positions, neighbour lists, descriptors) lives in one static
 * device array of about 3.2 MB inside this library, held on every GPU that
 * loads the library until the process exits. It limits n_atoms to
 * PIMD_NOALLOC_MAX_ATOMS and neighbours per atom to PIMD_NOALLOC_MAX_NEIGHBOURS;
 * larger inputs fail with INVALID_ARG, overfull neighbour lists with
 * NBR_OVERFLOW. No cudaMalloc, cudaFree or allocating library routine runs.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current): make that first call
 * before any stream capture. All calls share the one array, so calls that
 * overlap on the GPU (other threads, other streams) race with each other;
 * serialise them. Error text: pimd_last_error(NULL).                        */
#define PIMD_NOALLOC_MAX_ATOMS 4096
#define PIMD_NOALLOC_MAX_NEIGHBOURS 128
int pimd_descriptors_noalloc(const double* x_dev, int n_atoms, const double* box, double cutoff_A,
                             double eta_R, const double* r_mu, const double* eta_A, double* G_dev,
                             void* stream);

#ifdef __cplusplus
}
#endif
#endif
