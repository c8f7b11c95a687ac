/*
 * oracle.h -- FP64 CPU oracle for path-integral MD with a symmetry-function
 * neural-network potential.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * cpu_baseline / reference legs may load this library. It shares no code with
 * the CUDA path: it is a plain, slow restatement of the method's definitions
 * (paper Sec. 2.1 Eqs. for H_eff, H_p, U and the estimator; BPNN descriptors
 * of ref. [17] cited in Sec. 1; energy-derived forces of Sec. 2.2) written for
 * a reader to check against the paper by eye. Also: the step cut at its
 * force evaluation (bead-sharded runs), the path-integral free energy of
 * Sec. 2.5 from bead-resolved CV histograms, and g(r) (Figs. 8, 9).
 *
 * Units: Angstrom, fs, amu, eV, K.
 */
#ifndef PIMD_ORACLE_H
#define PIMD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_NR 32          /* radial channels                                  */
#define OR_NA 32          /* angular channels (4 zeta x 2 lambda x 4 eta)     */
#define OR_ND 64          /* descriptor length                                */
#define OR_MAX_ELEM 8
#define OR_MAX_LAYERS 8

/* Symmetry-function network. params[e] is element e's flat FP64 blob:
 * for l in hidden layers: W_l [h_l][h_{l-1}] row-major, b_l [h_l];
 * then w_out [h_L], b_out, mu [64], sigma [64], s_E, e_Z. */
typedef struct {
    int n_elem;
    int Z[OR_MAX_ELEM];
    int n_hidden;
    int width[OR_MAX_LAYERS];
    const double* params[OR_MAX_ELEM];
    double rc;
    double eta_R;
    double r_mu[OR_NR];
    int zeta[4];
    double lambda[2];
    double eta_A[4];
} or_model;

/* Well-tempered metadynamics on one collective variable of every bead
 * (Sec. 2.5; CVs of Secs. S2-S3). State (hills) lives in the struct.      */
typedef struct {
    int cv;                  /* 1 = sum_t c_t d(i_t, j_t), 2 = XRD intensity  */
    int n_terms;             /* cv 1: terms (<= 8)                           */
    int ti[8], tj[8];
    double tc[8];
    double Q;                /* cv 2: scattering vector magnitude, 1/A       */
    const double* f_atom;    /* cv 2: [N] atomic scattering factors           */
    double h0;               /* initial Gaussian height, eV                  */
    double sigma;            /* Gaussian width (standard deviation), CV units */
    double gamma;            /* bias factor (> 1)                            */
    int stride;              /* steps between depositions                    */
    int max_hills;
    double* hill_s;          /* [max_hills] centres                          */
    double* hill_h;          /* [max_hills] heights, eV                      */
    int n_hills;
    double* cv_last;         /* [P] CV of each bead at the last evaluation   */
    double* vb_last;         /* [P] bias of each bead at the last evaluation */
} or_metad;

/* One ring-polymer system and its integrator settings. */
typedef struct {
    int N, P;
    const int* Z;            /* [N]                                          */
    const double* mass;      /* [N] amu                                      */
    double box[3];           /* 0 = non-periodic                             */
    double T;                /* physical temperature, K                      */
    uint64_t seed;
    int replica;             /* replica index (enters the noise counter)     */
    double dt;               /* fs                                           */
    double gamma0;           /* centroid friction, 1/fs                      */
    double pile_lambda;      /* PILE-L scaling of internal-mode friction     */
    int thermostat;          /* 0 = NVE, 1 = PILE-L                          */
    int potential;           /* 0 = network, 1 = harmonic 0.5 m w^2 |x|^2    */
    double omega_harm;       /* 1/fs                                         */
    int maxnb;               /* neighbour slots per atom                     */
    int splitting;           /* 0 = OBABO, 1 = BAOAB                         */
    int free_rp;             /* free ring-polymer step: 0 = exact, 1 = Cayley */
    or_metad* metad;         /* NULL = no bias                               */
    int transform;           /* ring coordinates: 0 = normal modes, 1 = staging */
} or_sys;

/* estimator record, all eV except T_kin (K) */
typedef struct {
    double V_mean, K_prim, K_cv, E_tot;
    double W[9];
    double H_cons, Q_thermo, T_kin;
} or_est;

/* --- symmetry-function potential for one configuration ------------------ */
int  or_neighbours(int n, const double* x, const double* box, double rc, int maxnb,
                   int* nbr, int* nnb);
void or_descriptors(const or_model* m, int n, const double* x, const double* box,
                    const int* nbr, const int* nnb, int maxnb, double* G);
double or_mlp(const or_model* m, int z, const double* G, double* dEdG);
int  or_energy_forces(const or_model* m, int n, const int* Z, const double* x,
                      const double* box, int maxnb, double* E_atom, double* F, double* W);
int  or_energy_forces_batch(const or_model* m, int nconf, int n, const int* Z,
                            const double* x, const double* box, int maxnb,
                            double* E_atom, double* F, double* W);

/* --- ring polymer ---------------------------------------------------------- */
void or_nm_matrix(int P, double* C);
void or_nm_freqs(int P, double omega_P, double* wk);
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_normal(uint64_t seed, uint32_t index, uint32_t step, uint32_t replica, uint32_t stream);
int  or_init(const or_sys* s, const double* x0, double* q_nm, double* p_nm);
/* one free ring-polymer step of a single mode (w = 0: free drift) over time
 * h; free_rp 0 = exact, 1 = Cayley; p in amu A/fs, q in A                  */
void or_free_rp_step(int free_rp, double m, double w, double h, double* p, double* q);
/* staging coordinates of one (atom, dimension): u <-> bead positions x [P] */
void or_staging_to_beads(int P, const double* u, double* x);
void or_beads_to_staging(int P, const double* x, double* u);
/* -dPhi/du from bead forces f = -dPhi/dx [P] */
void or_staging_forces(int P, const double* f, double* Fu);
int  or_forces(const or_sys* s, const or_model* m, const double* q_nm,
               double* xb, double* f, double* V, double* W);
int  or_step(const or_sys* s, const or_model* m, int nsteps, uint64_t* step,
             double* q_nm, double* p_nm, double* f, double* V, double* W, double* Q_thermo);
/* the two halves of one step for atoms lo .. hi-1 with caller-supplied bead
 * forces (the sharded form of or_step) */
void or_ring_start(const or_sys* s, uint64_t step, int lo, int hi, double* q_nm, double* p_nm, const double* f,
                   double* xb, double* Q);
void or_ring_finish(const or_sys* s, uint64_t step, int lo, int hi, double* p_nm, const double* f, double* Q);
void or_estimators(const or_sys* s, const double* q_nm, const double* p_nm,
                   const double* f, const double* V, const double* W, double Q_thermo,
                   or_est* out);
/* --- collective variables and the metadynamics bias ----------------------- */
double or_cv(const or_metad* md, int n, const double* x, const double* box, double* grad, double* vir);
double or_metad_bias(const or_metad* md, double s, double* dVds);
void or_metad_deposit(or_metad* md, int P, double T);

/* --- structural analysis (RDF pair counts, proton-transfer coordinate) ---- */
void or_rdf_counts(int n, const double* x, const double* box, const int* type, int n_types,
                   double r_max, int n_bins, unsigned long long* counts);
void or_pt_coordinate(int n, const double* x, const double* box, const int* bond, const int* acceptor,
                      double v_min, double v_max, int n_bins, float* v, unsigned long long* hist);
/* g(r) of each element pair from pair counts summed over n_configs bead
 * configurations: counts[p][k] / (n_configs pairs_p shell_k / volume) */
void or_rdf_gr(int n_types, const int* n_per_type, double volume, double r_max, int n_bins,
               double n_configs, const unsigned long long* counts, double* g);

/* --- free-energy surfaces (Sec. 2.5) --------------------------------------- */
/* one sample of the bead-resolved CV histogram of the path-integral FES */
void or_cv_histogram(int P, const double* s, const double* vb, double T, double s_min, double inv_ds,
                     int n_bins, double log_w_shift, double* hist, double* wsum);
/* F_k(s) and the path-integral F(s) from that histogram */
void or_pi_fes(int P, int n_bins, const double* hist, double wsum, double ds, double T, double* F, double* Fk);
/* F(s) = -(gamma / (gamma - 1)) V(s) of a converged well-tempered bias */
void or_metad_fes(const or_metad* md, int n, const double* s, double* F);

void or_set_threads(int n);
int  or_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
