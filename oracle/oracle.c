/*
 * oracle.c -- FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Every routine follows a definition literally, in the order the method
 * states it: no blocking, fusion or reordering beyond the definition.
 *   - ring-polymer Hamiltonian, normal modes, estimator: paper Sec. 2.1;
 *   - descriptor + per-element network energy and its gradient (forces as
 *     -dE/dx of an energy model): Sec. 1 (BPNN, ref. [17]) and Sec. 2.2;
 *   - thermostat: PILE-L named in Tables of Sec. S2/S3 (Ceriotti et al. 2010);
 *   - noise: Philox4x32-10 (Salmon et al., SC'11) + Box-Muller.
 * Compile with -O2 -ffp-contract=off (no fast-math): the neighbour rule is an
 * exact FP32 computation that must not be contracted into FMAs.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#else
static int omp_in_parallel(void) { return 0; }
#endif

/* physical constants (CODATA 2018) */
static const double KB = 8.617333262e-5;          /* eV / K                  */
static const double HBAR = 0.6582119569;          /* eV fs                   */
static const double MVV2E = 103.64269652680505;   /* eV per amu A^2 fs^-2    */

static int g_threads = 0;

void or_set_threads(int n) { g_threads = n; }

int or_get_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* neighbour rule: FP32, no contraction, fixed operation order               */
/* ------------------------------------------------------------------------ */
typedef struct {
    int periodic;
    float L32[3], inv32[3];
} box32;

static box32 make_box32(const double* box)
{
    box32 b;
    b.periodic = box != NULL && box[0] > 0.0;
    for (int d = 0; d < 3; ++d) {
        b.L32[d] = b.periodic ? (float)box[d] : 0.0f;
        b.inv32[d] = b.periodic ? (float)(1.0 / box[d]) : 0.0f;
    }
    return b;
}

/* squared minimum-image distance of atoms i and j by the FP32 rule:
 * x32 = (float)x, t = x32_j - x32_i, t -= L32 rint(t invL32), then
 * r2 = (tx tx + ty ty) + tz tz, every operation rounded on its own */
static float r2_f32(const double* x, int i, int j, const box32* b)
{
    float dd[3];
    for (int d = 0; d < 3; ++d) {
        float t = (float)x[3 * j + d] - (float)x[3 * i + d];
        if (b->periodic) {
            float k = rintf(t * b->inv32[d]);
            float s = b->L32[d] * k;
            t = t - s;
        }
        dd[d] = t;
    }
    float r2 = dd[0] * dd[0];
    float yy = dd[1] * dd[1];
    float zz = dd[2] * dd[2];
    r2 = r2 + yy;
    r2 = r2 + zz;
    return r2;
}

int or_neighbours(int n, const double* x, const double* box, double rc, int maxnb,
                  int* nbr, int* nnb)
{
    box32 b = make_box32(box);
    float rc2 = (float)(rc * rc);
    int worst = 0;
#pragma omp parallel for num_threads(or_get_threads()) reduction(max : worst) if (!omp_in_parallel())
    for (int i = 0; i < n; ++i) {
        int cnt = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            float r2 = r2_f32(x, i, j, &b);
            if (r2 < rc2) {
                if (cnt < maxnb) nbr[(size_t)i * maxnb + cnt] = j;
                ++cnt;
            }
        }
        nnb[i] = cnt;
        if (cnt > worst) worst = cnt;
    }
    return worst;
}

/* ------------------------------------------------------------------------ */
/* geometry and symmetry functions                                          */
/* ------------------------------------------------------------------------ */
static void min_image(const double* xi, const double* xj, const double* box, double* d)
{
    for (int a = 0; a < 3; ++a) {
        d[a] = xj[a] - xi[a];
        if (box != NULL && box[0] > 0.0) d[a] -= box[a] * nearbyint(d[a] / box[a]);
    }
}

/* Behler cosine cutoff and its derivative */
static double cutoff_fn(double r, double rc) { return r < rc ? 0.5 * (cos(M_PI * r / rc) + 1.0) : 0.0; }
static double cutoff_dr(double r, double rc) { return r < rc ? -0.5 * M_PI / rc * sin(M_PI * r / rc) : 0.0; }

static double ipow(double b, int e)
{
    double p = 1.0;
    for (int k = 0; k < e; ++k) p *= b;
    return p;
}

/* angular channel nu = (zeta_index * 2 + lambda_index) * 4 + eta_index */
static void channel(const or_model* m, int nu, int* zeta, double* lambda, double* eta)
{
    *zeta = m->zeta[nu / 8];
    *lambda = m->lambda[(nu / 4) % 2];
    *eta = m->eta_A[nu % 4];
}

/* G2_mu = sum_j exp(-eta_R (r_ij - r_mu)^2) fc(r_ij)
 * G5_nu = 2^(1-zeta) sum_{j<k} (1 + lambda cos theta_jik)^zeta
 *                       exp(-eta (r_ij^2 + r_ik^2)) fc(r_ij) fc(r_ik)        */
static void descriptor_atom(const or_model* m, const double* x, const double* box, int i,
                            const int* nb, int cnt, double* G)
{
    for (int c = 0; c < OR_ND; ++c) G[c] = 0.0;
    for (int s = 0; s < cnt; ++s) {
        double d[3];
        min_image(x + 3 * i, x + 3 * nb[s], box, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int mu = 0; mu < OR_NR; ++mu) {
            double t = r - m->r_mu[mu];
            G[mu] += exp(-m->eta_R * t * t) * cutoff_fn(r, m->rc);
        }
    }
    for (int s = 0; s < cnt; ++s) {
        for (int t = s + 1; t < cnt; ++t) {
            double dj[3], dk[3];
            min_image(x + 3 * i, x + 3 * nb[s], box, dj);
            min_image(x + 3 * i, x + 3 * nb[t], box, dk);
            double rj = sqrt(dj[0] * dj[0] + dj[1] * dj[1] + dj[2] * dj[2]);
            double rk = sqrt(dk[0] * dk[0] + dk[1] * dk[1] + dk[2] * dk[2]);
            double cth = (dj[0] * dk[0] + dj[1] * dk[1] + dj[2] * dk[2]) / (rj * rk);
            for (int nu = 0; nu < OR_NA; ++nu) {
                int zeta;
                double lam, eta;
                channel(m, nu, &zeta, &lam, &eta);
                G[OR_NR + nu] += pow(2.0, 1 - zeta) * ipow(1.0 + lam * cth, zeta) *
                                 exp(-eta * (rj * rj + rk * rk)) *
                                 cutoff_fn(rj, m->rc) * cutoff_fn(rk, m->rc);
            }
        }
    }
}

void or_descriptors(const or_model* m, int n, const double* x, const double* box,
                    const int* nbr, const int* nnb, int maxnb, double* G)
{
#pragma omp parallel for num_threads(or_get_threads()) schedule(dynamic, 4) if (!omp_in_parallel())
    for (int i = 0; i < n; ++i)
        descriptor_atom(m, x, box, i, nbr + (size_t)i * maxnb, nnb[i], G + (size_t)i * OR_ND);
}

/* ------------------------------------------------------------------------ */
/* per-element network: E = s_E (w_out . h_L + b_out) + e_Z,                 */
/* h_l = tanh(W_l h_{l-1} + b_l), h_0 = (G - mu) / sigma; returns E and      */
/* dE/dG by back-propagation through the same layers.                        */
/* ------------------------------------------------------------------------ */
static int elem_index(const or_model* m, int z)
{
    for (int e = 0; e < m->n_elem; ++e)
        if (m->Z[e] == z) return e;
    return -1;
}

double or_mlp(const or_model* m, int z, const double* G, double* dEdG)
{
    int e = elem_index(m, z);
    const double* p = m->params[e];
    int L = m->n_hidden;
    /* locate the blob's pieces */
    const double* W[OR_MAX_LAYERS];
    const double* b[OR_MAX_LAYERS];
    int prev = OR_ND, off = 0;
    for (int l = 0; l < L; ++l) {
        W[l] = p + off; off += m->width[l] * prev;
        b[l] = p + off; off += m->width[l];
        prev = m->width[l];
    }
    const double* w_out = p + off; off += prev;
    double b_out = p[off]; off += 1;
    const double* mu = p + off; off += OR_ND;
    const double* sigma = p + off; off += OR_ND;
    double s_E = p[off];
    double e_Z = p[off + 1];

    /* forward, keeping every layer's output */
    double* h[OR_MAX_LAYERS + 1];
    int width_in[OR_MAX_LAYERS + 1];
    width_in[0] = OR_ND;
    h[0] = malloc(sizeof(double) * OR_ND);
    for (int c = 0; c < OR_ND; ++c) h[0][c] = (G[c] - mu[c]) / sigma[c];
    for (int l = 0; l < L; ++l) {
        int nin = width_in[l], nout = m->width[l];
        h[l + 1] = malloc(sizeof(double) * nout);
        width_in[l + 1] = nout;
        for (int o = 0; o < nout; ++o) {
            double a = b[l][o];
            for (int k = 0; k < nin; ++k) a += W[l][(size_t)o * nin + k] * h[l][k];
            h[l + 1][o] = tanh(a);
        }
    }
    double y = b_out;
    for (int k = 0; k < width_in[L]; ++k) y += w_out[k] * h[L][k];
    double E = s_E * y + e_Z;

    if (dEdG != NULL) {
        /* backward: dE/dh_L = s_E w_out; dE/da_l = dE/dh_l (1 - h_l^2);
           dE/dh_{l-1} = W_l^T dE/da_l */
        double* gh = malloc(sizeof(double) * width_in[L]);
        for (int k = 0; k < width_in[L]; ++k) gh[k] = s_E * w_out[k];
        for (int l = L - 1; l >= 0; --l) {
            int nin = width_in[l], nout = m->width[l];
            double* gprev = malloc(sizeof(double) * nin);
            for (int k = 0; k < nin; ++k) gprev[k] = 0.0;
            for (int o = 0; o < nout; ++o) {
                double ga = gh[o] * (1.0 - h[l + 1][o] * h[l + 1][o]);
                for (int k = 0; k < nin; ++k) gprev[k] += W[l][(size_t)o * nin + k] * ga;
            }
            free(gh);
            gh = gprev;
        }
        for (int c = 0; c < OR_ND; ++c) dEdG[c] = gh[c] / sigma[c];
        free(gh);
    }
    for (int l = 0; l <= L; ++l) free(h[l]);
    return E;
}

/* ------------------------------------------------------------------------ */
/* forces: chain rule of E_i(G_i(r_ij)) onto the pair vectors r_ij           */
/* v_s = dE_i / d r_{i j_s}; then F_j -= v_s, F_i += v_s,                    */
/* W_ab -= r_ij,a v_s,b (virial of the per-atom energy)                      */
/* ------------------------------------------------------------------------ */
static void pair_gradients(const or_model* m, const double* x, const double* box, int i,
                           const int* nb, int cnt, const double* g, double* v)
{
    for (int s = 0; s < 3 * cnt; ++s) v[s] = 0.0;
    double rc = m->rc;
    for (int s = 0; s < cnt; ++s) {
        double d[3];
        min_image(x + 3 * i, x + 3 * nb[s], box, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double dEdr = 0.0;
        for (int mu = 0; mu < OR_NR; ++mu) {
            double t = r - m->r_mu[mu];
            double ex = exp(-m->eta_R * t * t);
            dEdr += g[mu] * ex * (-2.0 * m->eta_R * t * cutoff_fn(r, rc) + cutoff_dr(r, rc));
        }
        for (int a = 0; a < 3; ++a) v[3 * s + a] += dEdr * d[a] / r;
    }
    for (int s = 0; s < cnt; ++s) {
        for (int t = s + 1; t < cnt; ++t) {
            double dj[3], dk[3], uj[3], uk[3];
            min_image(x + 3 * i, x + 3 * nb[s], box, dj);
            min_image(x + 3 * i, x + 3 * nb[t], box, dk);
            double rj = sqrt(dj[0] * dj[0] + dj[1] * dj[1] + dj[2] * dj[2]);
            double rk = sqrt(dk[0] * dk[0] + dk[1] * dk[1] + dk[2] * dk[2]);
            for (int a = 0; a < 3; ++a) { uj[a] = dj[a] / rj; uk[a] = dk[a] / rk; }
            double cth = uj[0] * uk[0] + uj[1] * uk[1] + uj[2] * uk[2];
            double fj = cutoff_fn(rj, rc), fk = cutoff_fn(rk, rc);
            double dfj = cutoff_dr(rj, rc), dfk = cutoff_dr(rk, rc);
            for (int nu = 0; nu < OR_NA; ++nu) {
                int zeta;
                double lam, eta;
                channel(m, nu, &zeta, &lam, &eta);
                double pre = pow(2.0, 1 - zeta);
                double ang = ipow(1.0 + lam * cth, zeta);
                double dang = zeta * lam * ipow(1.0 + lam * cth, zeta - 1);
                double ex = exp(-eta * (rj * rj + rk * rk));
                double T_c = pre * dang * ex * fj * fk;                        /* dT/dcos   */
                double T_rj = pre * ang * ex * fk * (-2.0 * eta * rj * fj + dfj); /* dT/dr_ij */
                double T_rk = pre * ang * ex * fj * (-2.0 * eta * rk * fk + dfk); /* dT/dr_ik */
                for (int a = 0; a < 3; ++a) {
                    /* d cos / d r_ij = (u_k - cos u_j) / r_ij, and symmetrically */
                    v[3 * s + a] += g[OR_NR + nu] * (T_rj * uj[a] + T_c * (uk[a] - cth * uj[a]) / rj);
                    v[3 * t + a] += g[OR_NR + nu] * (T_rk * uk[a] + T_c * (uj[a] - cth * uk[a]) / rk);
                }
            }
        }
    }
}

int or_energy_forces(const or_model* m, int n, const int* Z, const double* x,
                     const double* box, int maxnb, double* E_atom, double* F, double* W)
{
    int* nbr = malloc(sizeof(int) * (size_t)n * maxnb);
    int* nnb = malloc(sizeof(int) * (size_t)n);
    double* v = malloc(sizeof(double) * (size_t)n * maxnb * 3);
    int worst = or_neighbours(n, x, box, m->rc, maxnb, nbr, nnb);
    if (worst > maxnb) {
        free(nbr); free(nnb); free(v);
        return -worst;
    }
    int bad = 0;
#pragma omp parallel for num_threads(or_get_threads()) schedule(dynamic, 4) reduction(| : bad) if (!omp_in_parallel())
    for (int i = 0; i < n; ++i) {
        double G[OR_ND], g[OR_ND];
        const int* nb = nbr + (size_t)i * maxnb;
        if (elem_index(m, Z[i]) < 0) { bad = 1; continue; }
        descriptor_atom(m, x, box, i, nb, nnb[i], G);
        E_atom[i] = or_mlp(m, Z[i], G, g);
        pair_gradients(m, x, box, i, nb, nnb[i], g, v + (size_t)i * maxnb * 3);
    }
    if (bad) {
        free(nbr); free(nnb); free(v);
        return -1;
    }
    for (int k = 0; k < 3 * n; ++k) F[k] = 0.0;
    for (int k = 0; k < 9; ++k) W[k] = 0.0;
    for (int i = 0; i < n; ++i) {
        for (int s = 0; s < nnb[i]; ++s) {
            int j = nbr[(size_t)i * maxnb + s];
            const double* vs = v + ((size_t)i * maxnb + s) * 3;
            double d[3];
            min_image(x + 3 * i, x + 3 * j, box, d);
            for (int a = 0; a < 3; ++a) {
                F[3 * j + a] -= vs[a];
                F[3 * i + a] += vs[a];
                for (int b2 = 0; b2 < 3; ++b2) W[3 * a + b2] -= d[a] * vs[b2];
            }
        }
    }
    free(nbr); free(nnb); free(v);
    return worst;
}

int or_energy_forces_batch(const or_model* m, int nconf, int n, const int* Z,
                           const double* x, const double* box, int maxnb,
                           double* E_atom, double* F, double* W)
{
    int worst = 0;
    for (int c = 0; c < nconf; ++c) {
        int r = or_energy_forces(m, n, Z, x + (size_t)c * n * 3, box, maxnb,
                                 E_atom + (size_t)c * n, F + (size_t)c * n * 3, W + 9 * c);
        if (r < 0) return r;
        if (r > worst) worst = r;
    }
    return worst;
}

/* ------------------------------------------------------------------------ */
/* normal modes of the cyclic ring polymer                                   */
/* C[j][k]: bead j, mode k;  q_bead = C q_nm;  C^T C = I                      */
/* ------------------------------------------------------------------------ */
void or_nm_matrix(int P, double* C)
{
    for (int j = 0; j < P; ++j) {
        for (int k = 0; k < P; ++k) {
            double v;
            if (k == 0)
                v = 1.0 / sqrt((double)P);
            else if (2 * k < P)
                v = sqrt(2.0 / P) * cos(2.0 * M_PI * j * k / P);
            else if (2 * k == P)
                v = ((j % 2) ? -1.0 : 1.0) / sqrt((double)P);
            else
                v = sqrt(2.0 / P) * sin(2.0 * M_PI * j * k / P);
            C[j * P + k] = v;
        }
    }
}

/* free ring-polymer mode frequencies omega_k = 2 omega_P sin(k pi / P) */
void or_nm_freqs(int P, double omega_P, double* wk)
{
    for (int k = 0; k < P; ++k) wk[k] = 2.0 * omega_P * sin(k * M_PI / P);
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 and Box-Muller                                              */
/* ------------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c[0], &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c[2], &hi1, &lo1);
        uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    for (int a = 0; a < 4; ++a) out[a] = c[a];
}

/* one standard normal: counter (index, step, replica, stream), key = seed;
 * two 53-bit uniforms in (0, 1] from word pairs, then Box-Muller */
double or_normal(uint64_t seed, uint32_t index, uint32_t step, uint32_t replica, uint32_t stream)
{
    uint32_t ctr[4] = {index, step, replica, stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    double u1 = ((double)(w[0] >> 5) * 67108864.0 + (double)(w[1] >> 6) + 1.0) / 9007199254740992.0;
    double u2 = ((double)(w[2] >> 5) * 67108864.0 + (double)(w[3] >> 6) + 1.0) / 9007199254740992.0;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* ------------------------------------------------------------------------ */
/* ring-polymer dynamics in normal-mode space (state layout [P][N][3])       */
/* i-PI convention: beta_P = beta / P, omega_P = P k_B T / hbar               */
/* ------------------------------------------------------------------------ */
static double omega_P_of(const or_sys* s) { return s->P * KB * s->T / HBAR; }
static double kT_P_md(const or_sys* s) { return s->P * KB * s->T / MVV2E; }

/* ---- staging coordinates (Tuckerman's staging transformation) ------------
 * For one (atom, dimension), beads x_1 .. x_P (x_(P+1) = x_1, array index
 * k - 1):
 *   u_1 = x_1,  u_k = x_k - ((k - 1) x_(k+1) + x_1) / k   (k = 2 .. P)
 * and back, from k = P down to 2: x_k = u_k + ((k - 1)/k) x_(k+1) + x_1 / k.
 * The spring energy sum_k 1/2 m w_P^2 (x_k - x_(k+1))^2 becomes
 * sum_(k>=2) 1/2 m_k' w_P^2 u_k^2 with m_k' = k / (k - 1) m, so with these
 * masses every u_k (k >= 2) oscillates at w_P and u_1 moves freely.
 * Forces: -dPhi/du_1 = sum_j f_j, -dPhi/du_2 = f_2,
 * -dPhi/du_k = f_k + ((k - 2)/(k - 1)) (-dPhi/du_(k-1)) for k >= 3.        */
void or_staging_to_beads(int P, const double* u, double* x)
{
    x[0] = u[0];
    double next = x[0];   /* x_(k+1), starting with x_(P+1) = x_1 */
    for (int k = P; k >= 2; --k) {
        x[k - 1] = u[k - 1] + ((double)(k - 1) / k) * next + x[0] / k;
        next = x[k - 1];
    }
}

void or_beads_to_staging(int P, const double* x, double* u)
{
    u[0] = x[0];
    for (int k = 2; k <= P; ++k) {
        double xn = (k == P) ? x[0] : x[k];
        u[k - 1] = x[k - 1] - ((k - 1) * xn + x[0]) / k;
    }
}

void or_staging_forces(int P, const double* f, double* Fu)
{
    double s = 0.0;
    for (int j = 0; j < P; ++j) s += f[j];
    Fu[0] = s;
    if (P >= 2) Fu[1] = f[1];
    for (int k = 3; k <= P; ++k) Fu[k - 1] = f[k - 1] + ((double)(k - 2) / (k - 1)) * Fu[k - 2];
}

/* mass of ring coordinate k (0-based) of atom i, and its free frequency */
static double mode_mass(const or_sys* s, int k, int i)
{
    return (s->transform == 1 && k >= 1) ? s->mass[i] * (k + 1.0) / k : s->mass[i];
}
static void mode_freqs(const or_sys* s, double* wk)
{
    if (s->transform == 1) {
        for (int k = 0; k < s->P; ++k) wk[k] = k == 0 ? 0.0 : omega_P_of(s);
    } else {
        or_nm_freqs(s->P, omega_P_of(s), wk);
    }
}

int or_init(const or_sys* s, const double* x0, double* q_nm, double* p_nm)
{
    int N = s->N, P = s->P;
    double kT = kT_P_md(s);
    for (int k = 0; k < P; ++k)
        for (int i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) {
                size_t g = ((size_t)k * N + i) * 3 + d;
                if (s->transform == 1)
                    q_nm[g] = (k == 0) ? x0[3 * i + d] : 0.0;   /* all beads at x0 */
                else
                    q_nm[g] = (k == 0) ? sqrt((double)P) * x0[3 * i + d] : 0.0;
                p_nm[g] = sqrt(mode_mass(s, k, i) * kT) *
                          or_normal(s->seed, (uint32_t)g, 0u, (uint32_t)s->replica, 1u);
            }
    return 0;
}

static void to_beads(const or_sys* s, const double* C, const double* q_nm, double* xb)
{
    int N = s->N, P = s->P;
    if (s->transform == 1) {
        double* u = malloc(sizeof(double) * P);
        double* x = malloc(sizeof(double) * P);
        for (int i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) {
                for (int k = 0; k < P; ++k) u[k] = q_nm[((size_t)k * N + i) * 3 + d];
                or_staging_to_beads(P, u, x);
                for (int j = 0; j < P; ++j) xb[((size_t)j * N + i) * 3 + d] = x[j];
            }
        free(u);
        free(x);
        return;
    }
    for (int j = 0; j < P; ++j)
        for (int i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) {
                double acc = 0.0;
                for (int k = 0; k < P; ++k) acc += C[j * P + k] * q_nm[((size_t)k * N + i) * 3 + d];
                xb[((size_t)j * N + i) * 3 + d] = acc;
            }
}

/* ------------------------------------------------------------------------ */
/* collective variables and well-tempered metadynamics (Sec. 2.5)            */
/* ------------------------------------------------------------------------ */
static double sinc(double y) { return sin(y) / y; }
static double dsinc(double y) { return (y * cos(y) - sin(y)) / (y * y); }

/* CV of one configuration. cv 1: s = sum_t c_t |r_(i_t j_t)|; cv 2 (XRD
 * intensity, Sec. S3): s = (1/N) sum_i sum_j f_i f_j sin(Q R_ij) / (Q R_ij)
 * with the i = j terms f_i^2. R_ij are minimum-image distances. grad
 * [n][3] = ds/dx (may be NULL); vir [9] = sum over the pairs of r_ij (x)
 * ds/dr_ij, r_ij = x_j - x_i (may be NULL). */
double or_cv(const or_metad* md, int n, const double* x, const double* box, double* grad, double* vir)
{
    if (grad) memset(grad, 0, sizeof(double) * 3 * n);
    if (vir) memset(vir, 0, sizeof(double) * 9);
    double s = 0.0;
    if (md->cv == 1) {
        for (int t = 0; t < md->n_terms; ++t) {
            int i = md->ti[t], j = md->tj[t];
            double r[3];
            min_image(x + 3 * i, x + 3 * j, box, r);
            double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            s += md->tc[t] * d;
            for (int a = 0; a < 3; ++a) {
                double g = md->tc[t] * r[a] / d;   /* ds/dr_ij */
                if (grad) {
                    grad[3 * j + a] += g;
                    grad[3 * i + a] -= g;
                }
                if (vir)
                    for (int b = 0; b < 3; ++b) vir[3 * b + a] += r[b] * g;
            }
        }
        return s;
    }
    for (int i = 0; i < n; ++i) s += md->f_atom[i] * md->f_atom[i];
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double r[3];
            min_image(x + 3 * i, x + 3 * j, box, r);
            double R = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            double ff = md->f_atom[i] * md->f_atom[j];
            s += 2.0 * ff * sinc(md->Q * R);
            double c = 2.0 * ff * md->Q * dsinc(md->Q * R) / (n * R);   /* ds/dr_ij = c r_ij */
            for (int a = 0; a < 3; ++a) {
                if (grad) {
                    grad[3 * j + a] += c * r[a];
                    grad[3 * i + a] -= c * r[a];
                }
                if (vir)
                    for (int b = 0; b < 3; ++b) vir[3 * b + a] += r[b] * c * r[a];
            }
        }
    return s / n;
}

/* V(s) = sum_k h_k exp(-(s - s_k)^2 / (2 sigma^2)) and dV/ds */
double or_metad_bias(const or_metad* md, double s, double* dVds)
{
    double v = 0.0, dv = 0.0;
    for (int k = 0; k < md->n_hills; ++k) {
        double u = s - md->hill_s[k];
        double g = md->hill_h[k] * exp(-0.5 * u * u / (md->sigma * md->sigma));
        v += g;
        dv -= g * u / (md->sigma * md->sigma);
    }
    if (dVds) *dVds = dv;
    return v;
}

/* one deposition: a hill at every bead's CV of the last evaluation, height
 * (h0 / P) exp(-V(s_k) / (k_B T (gamma - 1))) with the bias before this
 * deposition (the well-tempered rule of Sec. 2.5, shared over the P beads) */
void or_metad_deposit(or_metad* md, int P, double T)
{
    if (md->n_hills + P > md->max_hills) return;
    int base = md->n_hills;
    for (int k = 0; k < P; ++k) {
        md->hill_s[base + k] = md->cv_last[k];
        md->hill_h[base + k] = md->h0 / P * exp(-md->vb_last[k] / (KB * T * (md->gamma - 1.0)));
    }
    md->n_hills += P;
}

/* bias of every bead: V_k += V(s_k), f_k -= dV/ds ds/dx, W_k -= dV/ds vir */
static void add_bias(const or_sys* s, const double* xb, double* f, double* V, double* W)
{
    int N = s->N, P = s->P;
    double* g = malloc(sizeof(double) * 3 * N);
    for (int j = 0; j < P; ++j) {
        double vir[9], dv;
        double cv = or_cv(s->metad, N, xb + (size_t)j * N * 3, s->box, g, vir);
        double vb = or_metad_bias(s->metad, cv, &dv);
        s->metad->cv_last[j] = cv;
        s->metad->vb_last[j] = vb;
        V[j] += vb;
        for (int q = 0; q < 3 * N; ++q) f[(size_t)j * N * 3 + q] -= dv * g[q];
        for (int q = 0; q < 9; ++q) W[9 * j + q] -= dv * vir[q];
    }
    free(g);
}

int or_forces(const or_sys* s, const or_model* m, const double* q_nm,
              double* xb, double* f, double* V, double* W)
{
    int N = s->N, P = s->P;
    double* C = malloc(sizeof(double) * P * P);
    or_nm_matrix(P, C);
    to_beads(s, C, q_nm, xb);
    free(C);
    if (s->potential == 1) {
        for (int j = 0; j < P; ++j) {
            double v = 0.0;
            for (int i = 0; i < N; ++i)
                for (int d = 0; d < 3; ++d) {
                    size_t g = ((size_t)j * N + i) * 3 + d;
                    double k = s->mass[i] * s->omega_harm * s->omega_harm * MVV2E; /* eV/A^2 */
                    v += 0.5 * k * xb[g] * xb[g];
                    f[g] = -k * xb[g];
                }
            V[j] = v;
            for (int a = 0; a < 3; ++a)
                for (int b2 = 0; b2 < 3; ++b2) {
                    double w = 0.0;
                    for (int i = 0; i < N; ++i)
                        w += xb[((size_t)j * N + i) * 3 + a] * f[((size_t)j * N + i) * 3 + b2];
                    W[9 * j + 3 * a + b2] = w;
                }
        }
        if (s->metad != NULL) add_bias(s, xb, f, V, W);
        return 0;
    }
    double* E = malloc(sizeof(double) * N);
    int rc = 0;
    for (int j = 0; j < P && rc >= 0; ++j) {
        int r = or_energy_forces(m, N, s->Z, xb + (size_t)j * N * 3, s->box, s->maxnb, E,
                                 f + (size_t)j * N * 3, W + 9 * j);
        if (r < 0) { rc = r; break; }
        double v = 0.0;
        for (int i = 0; i < N; ++i) v += E[i];
        V[j] = v;
    }
    free(E);
    if (rc >= 0 && s->metad != NULL) add_bias(s, xb, f, V, W);
    return rc;
}

/* O: p <- c1 p + sqrt(m k_B T_P) c2 xi over time h (PILE-L friction
 * gamma_0 on the centroid, 2 lambda omega_k on internal modes) */
static void step_O(const or_sys* s, const double* wk, double h, uint32_t step, uint32_t stream,
                   double* p_nm, double* Q)
{
    int N = s->N, P = s->P;
    double kT = kT_P_md(s), dq = 0.0;
    for (int k = 0; k < P; ++k) {
        double gam = (k == 0) ? s->gamma0 : 2.0 * s->pile_lambda * wk[k];
        double c1 = exp(-h * gam);
        double c2 = sqrt(1.0 - c1 * c1);
        for (int i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) {
                size_t g = ((size_t)k * N + i) * 3 + d;
                double xi = or_normal(s->seed, (uint32_t)g, step, (uint32_t)s->replica, stream);
                double mk = mode_mass(s, k, i);
                double pn = c1 * p_nm[g] + sqrt(mk * kT) * c2 * xi;
                dq += (pn * pn - p_nm[g] * p_nm[g]) / (2.0 * mk);
                p_nm[g] = pn;
            }
    }
    *Q += dq * MVV2E;
}

/* B: p_nm += dt/2 C^T f */
static void step_B(const or_sys* s, const double* C, const double* f, double* p_nm)
{
    int N = s->N, P = s->P;
    if (s->transform == 1) {
        double* fb = malloc(sizeof(double) * P);
        double* Fu = malloc(sizeof(double) * P);
        for (int i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) {
                for (int j = 0; j < P; ++j) fb[j] = f[((size_t)j * N + i) * 3 + d];
                or_staging_forces(P, fb, Fu);
                for (int k = 0; k < P; ++k) p_nm[((size_t)k * N + i) * 3 + d] += 0.5 * s->dt * Fu[k] / MVV2E;
            }
        free(fb);
        free(Fu);
        return;
    }
    for (int k = 0; k < P; ++k)
        for (int i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) {
                double fn = 0.0;
                for (int j = 0; j < P; ++j) fn += C[j * P + k] * f[((size_t)j * N + i) * 3 + d];
                p_nm[((size_t)k * N + i) * 3 + d] += 0.5 * s->dt * fn / MVV2E;
            }
}

/* A: free ring-polymer evolution of each normal mode over time h. Mode k
 * obeys d/dt (p, q) = L (p, q) with L = [[0, -m w_k^2], [1/m, 0]].
 * exact:  (p, q) <- exp(h L) (p, q);
 * Cayley: (p, q) <- (I - h L / 2)^-1 (I + h L / 2) (p, q), the Cayley
 *         transform of h L (stable for any w_k h). The centroid (w_0 = 0)
 *         drifts freely either way. */
void or_free_rp_step(int free_rp, double m, double w, double h, double* p, double* q)
{
    double p0 = *p, q0 = *q;
    if (w == 0.0) {
        *q = q0 + p0 * h / m;
    } else if (free_rp == 1) {
        /* M+ = I + h L / 2, M- = I - h L / 2, inverse of M- by the 2x2 rule */
        double ap[2][2] = {{1.0, -0.5 * h * m * w * w}, {0.5 * h / m, 1.0}};
        double am[2][2] = {{1.0, 0.5 * h * m * w * w}, {-0.5 * h / m, 1.0}};
        double det = am[0][0] * am[1][1] - am[0][1] * am[1][0];
        double inv[2][2] = {{am[1][1] / det, -am[0][1] / det}, {-am[1][0] / det, am[0][0] / det}};
        double u0 = ap[0][0] * p0 + ap[0][1] * q0, u1 = ap[1][0] * p0 + ap[1][1] * q0;
        *p = inv[0][0] * u0 + inv[0][1] * u1;
        *q = inv[1][0] * u0 + inv[1][1] * u1;
    } else {
        double cw = cos(w * h), sw = sin(w * h);
        *p = cw * p0 - m * w * sw * q0;
        *q = sw / (m * w) * p0 + cw * q0;
    }
}

static void step_A(const or_sys* s, const double* wk, double h, double* q_nm, double* p_nm)
{
    int N = s->N, P = s->P;
    for (int k = 0; k < P; ++k)
        for (int i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) {
                size_t g = ((size_t)k * N + i) * 3 + d;
                or_free_rp_step(s->free_rp, mode_mass(s, k, i), k == 0 ? 0.0 : wk[k], h, &p_nm[g], &q_nm[g]);
            }
}

/* one step, OBABO: O(dt/2) B(dt/2) A(dt) [forces] B(dt/2) O(dt/2), the noise
 * of step n with counter step n, streams 2 (first O) and 3 (second O);
 * BAOAB: B(dt/2) A(dt/2) O(dt) A(dt/2) [forces] B(dt/2), noise stream 2 */
int or_step(const or_sys* s, const or_model* m, int nsteps, uint64_t* step,
            double* q_nm, double* p_nm, double* f, double* V, double* W, double* Q_thermo)
{
    int N = s->N, P = s->P;
    double* C = malloc(sizeof(double) * P * P);
    double* wk = malloc(sizeof(double) * P);
    double* xb = malloc(sizeof(double) * (size_t)P * N * 3);
    or_nm_matrix(P, C);
    mode_freqs(s, wk);
    int rc = 0;
    for (int n = 0; n < nsteps; ++n) {
        uint32_t st = (uint32_t)(*step);
        if (s->splitting == 1) {
            step_B(s, C, f, p_nm);
            step_A(s, wk, 0.5 * s->dt, q_nm, p_nm);
            if (s->thermostat) step_O(s, wk, s->dt, st, 2u, p_nm, Q_thermo);
            step_A(s, wk, 0.5 * s->dt, q_nm, p_nm);
        } else {
            if (s->thermostat) step_O(s, wk, 0.5 * s->dt, st, 2u, p_nm, Q_thermo);
            step_B(s, C, f, p_nm);
            step_A(s, wk, s->dt, q_nm, p_nm);
        }
        rc = or_forces(s, m, q_nm, xb, f, V, W);
        if (rc < 0) break;
        /* hills go down after the force evaluation of step n when (n + 1) is a
           multiple of the stride; they act from the next evaluation on */
        if (s->metad != NULL && ((uint64_t)st + 1) % (uint64_t)s->metad->stride == 0)
            or_metad_deposit(s->metad, P, s->T);
        step_B(s, C, f, p_nm);
        if (s->thermostat && s->splitting != 1) step_O(s, wk, 0.5 * s->dt, st, 3u, p_nm, Q_thermo);
        *step += 1;
    }
    free(C); free(wk); free(xb);
    return rc;
}

/* The two halves of one step for the atoms lo .. hi-1 only, with the bead
 * forces supplied by the caller: the same splitting as or_step (Sec. 2.1),
 * cut at the force evaluation, so that atoms can be advanced in separate
 * shards once every bead's forces are known. Every coordinate (mode, atom,
 * dim) gets exactly the operations of or_step, in the same order, with the
 * same noise counters (global indices). Arrays are the full [P][N][3].
 *   start:  OBABO: O(dt/2, stream 2), B(dt/2) with f, A(dt);
 *           BAOAB: B(dt/2) with f, A(dt/2), O(dt, stream 2), A(dt/2);
 *           then the bead positions xb of the range.
 *   finish: B(dt/2) with the new forces f, then O(dt/2, stream 3) (OBABO).
 * The heat of the range's O steps is added to *Q.                           */
static void range_O(const or_sys* s, const double* wk, double h, uint32_t step, uint32_t stream, int lo, int hi,
                    double* p_nm, double* Q)
{
    int N = s->N, P = s->P;
    double kT = kT_P_md(s), dq = 0.0;
    for (int k = 0; k < P; ++k) {
        double gam = (k == 0) ? s->gamma0 : 2.0 * s->pile_lambda * wk[k];
        double c1 = exp(-h * gam);
        double c2 = sqrt(1.0 - c1 * c1);
        for (int i = lo; i < hi; ++i)
            for (int d = 0; d < 3; ++d) {
                size_t g = ((size_t)k * N + i) * 3 + d;
                double xi = or_normal(s->seed, (uint32_t)g, step, (uint32_t)s->replica, stream);
                double mk = mode_mass(s, k, i);
                double pn = c1 * p_nm[g] + sqrt(mk * kT) * c2 * xi;
                dq += (pn * pn - p_nm[g] * p_nm[g]) / (2.0 * mk);
                p_nm[g] = pn;
            }
    }
    *Q += dq * MVV2E;
}

static void range_B(const or_sys* s, const double* C, const double* f, int lo, int hi, double* p_nm)
{
    int N = s->N, P = s->P;
    if (s->transform == 1) {
        double* fb = malloc(sizeof(double) * P);
        double* Fu = malloc(sizeof(double) * P);
        for (int i = lo; i < hi; ++i)
            for (int d = 0; d < 3; ++d) {
                for (int j = 0; j < P; ++j) fb[j] = f[((size_t)j * N + i) * 3 + d];
                or_staging_forces(P, fb, Fu);
                for (int k = 0; k < P; ++k) p_nm[((size_t)k * N + i) * 3 + d] += 0.5 * s->dt * Fu[k] / MVV2E;
            }
        free(fb);
        free(Fu);
        return;
    }
    for (int k = 0; k < P; ++k)
        for (int i = lo; i < hi; ++i)
            for (int d = 0; d < 3; ++d) {
                double fn = 0.0;
                for (int j = 0; j < P; ++j) fn += C[j * P + k] * f[((size_t)j * N + i) * 3 + d];
                p_nm[((size_t)k * N + i) * 3 + d] += 0.5 * s->dt * fn / MVV2E;
            }
}

static void range_A(const or_sys* s, const double* wk, double h, int lo, int hi, double* q_nm, double* p_nm)
{
    int N = s->N, P = s->P;
    for (int k = 0; k < P; ++k)
        for (int i = lo; i < hi; ++i)
            for (int d = 0; d < 3; ++d) {
                size_t g = ((size_t)k * N + i) * 3 + d;
                or_free_rp_step(s->free_rp, mode_mass(s, k, i), k == 0 ? 0.0 : wk[k], h, &p_nm[g], &q_nm[g]);
            }
}

void or_ring_start(const or_sys* s, uint64_t step, int lo, int hi, double* q_nm, double* p_nm, const double* f,
                   double* xb, double* Q)
{
    int N = s->N, P = s->P;
    double* C = malloc(sizeof(double) * P * P);
    double* wk = malloc(sizeof(double) * P);
    or_nm_matrix(P, C);
    mode_freqs(s, wk);
    uint32_t st = (uint32_t)step;
    if (s->splitting == 1) {
        range_B(s, C, f, lo, hi, p_nm);
        range_A(s, wk, 0.5 * s->dt, lo, hi, q_nm, p_nm);
        if (s->thermostat) range_O(s, wk, s->dt, st, 2u, lo, hi, p_nm, Q);
        range_A(s, wk, 0.5 * s->dt, lo, hi, q_nm, p_nm);
    } else {
        if (s->thermostat) range_O(s, wk, 0.5 * s->dt, st, 2u, lo, hi, p_nm, Q);
        range_B(s, C, f, lo, hi, p_nm);
        range_A(s, wk, s->dt, lo, hi, q_nm, p_nm);
    }
    /* bead positions of the range (the transform of to_beads, per atom) */
    double* u = malloc(sizeof(double) * P);
    double* x = malloc(sizeof(double) * P);
    for (int i = lo; i < hi; ++i)
        for (int d = 0; d < 3; ++d) {
            for (int k = 0; k < P; ++k) u[k] = q_nm[((size_t)k * N + i) * 3 + d];
            if (s->transform == 1) {
                or_staging_to_beads(P, u, x);
            } else {
                for (int j = 0; j < P; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < P; ++k) acc += C[j * P + k] * u[k];
                    x[j] = acc;
                }
            }
            for (int j = 0; j < P; ++j) xb[((size_t)j * N + i) * 3 + d] = x[j];
        }
    free(u); free(x); free(C); free(wk);
}

void or_ring_finish(const or_sys* s, uint64_t step, int lo, int hi, double* p_nm, const double* f, double* Q)
{
    int P = s->P;
    double* C = malloc(sizeof(double) * P * P);
    double* wk = malloc(sizeof(double) * P);
    or_nm_matrix(P, C);
    mode_freqs(s, wk);
    range_B(s, C, f, lo, hi, p_nm);
    if (s->thermostat && s->splitting != 1) range_O(s, wk, 0.5 * s->dt, (uint32_t)step, 3u, lo, hi, p_nm, Q);
    free(C); free(wk);
}

/* ------------------------------------------------------------------------ */
/* estimators of the finite-P ensemble average                               */
/* ------------------------------------------------------------------------ */
void or_estimators(const or_sys* s, const double* q_nm, const double* p_nm,
                   const double* f, const double* V, const double* W, double Q_thermo,
                   or_est* out)
{
    int N = s->N, P = s->P;
    double beta = 1.0 / (KB * s->T);
    double wP = omega_P_of(s);
    double* C = malloc(sizeof(double) * P * P);
    double* xb = malloc(sizeof(double) * (size_t)P * N * 3);
    or_nm_matrix(P, C);
    to_beads(s, C, q_nm, xb);

    double Vbar = 0.0;
    for (int j = 0; j < P; ++j) Vbar += V[j];
    Vbar /= P;

    double spring = 0.0; /* sum_k sum_i 1/2 m omega_P^2 |q^k - q^{k+1}|^2, eV */
    for (int j = 0; j < P; ++j) {
        int jn = (j + 1) % P;
        for (int i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) {
                double dq = xb[((size_t)j * N + i) * 3 + d] - xb[((size_t)jn * N + i) * 3 + d];
                spring += 0.5 * s->mass[i] * wP * wP * dq * dq * MVV2E;
            }
    }
    double K_prim = 3.0 * N * P / (2.0 * beta) - spring / P;

    double cv = 0.0; /* sum_k sum_i (q_i^k - centroid_i) . f_i^k */
    for (int i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) {
            double cen = 0.0;
            for (int j = 0; j < P; ++j) cen += xb[((size_t)j * N + i) * 3 + d];
            cen /= P;
            for (int j = 0; j < P; ++j) {
                size_t g = ((size_t)j * N + i) * 3 + d;
                cv += (xb[g] - cen) * f[g];
            }
        }
    double K_cv = 3.0 * N / (2.0 * beta) - cv / (2.0 * P);

    double kin = 0.0; /* sum p^2 / 2m over all ring coordinates, eV */
    for (int k = 0; k < P; ++k)
        for (int i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) {
                double p = p_nm[((size_t)k * N + i) * 3 + d];
                kin += p * p / (2.0 * mode_mass(s, k, i)) * MVV2E;
            }
    double H_P = kin + spring;
    for (int j = 0; j < P; ++j) H_P += V[j];

    out->V_mean = Vbar;
    out->K_prim = K_prim;
    out->K_cv = K_cv;
    out->E_tot = K_cv + Vbar;
    for (int a = 0; a < 9; ++a) {
        double w = 0.0;
        for (int j = 0; j < P; ++j) w += W[9 * j + a];
        out->W[a] = w / P;
    }
    out->H_cons = H_P - Q_thermo;
    out->Q_thermo = Q_thermo;
    out->T_kin = 2.0 * kin / (3.0 * N * P * KB);
    free(C); free(xb);
}

/* ------------------------------------------------------------------------ */
/* structural analysis of bead configurations (Sec. 3.2, Figs. 8, 9, 11)     */
/* ------------------------------------------------------------------------ */
/* Pair counts of the radial distribution function. Element types a <= b
 * index the pair p = a (2T - a - 1) / 2 + b. A pair i < j at squared FP32
 * distance r2 (rule of r2_f32) lies in bin k when e_k <= r2 < e_(k+1), with
 * edges e_k = (float)((k r_max / n_bins)^2) formed in FP64; pairs with r2 >=
 * e_(n_bins) are not counted. counts[p][k] += the number of such pairs.     */
void or_rdf_counts(int n, const double* x, const double* box, const int* type, int n_types,
                   double r_max, int n_bins, unsigned long long* counts)
{
    box32 b = make_box32(box);
    float* e = malloc(sizeof(float) * (n_bins + 1));
    for (int k = 0; k <= n_bins; ++k) {
        double rk = k * (r_max / n_bins);
        e[k] = (float)(rk * rk);
    }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            float r2 = r2_f32(x, i, j, &b);
            if (!(r2 < e[n_bins])) continue;
            int k = 0;
            while (!(r2 < e[k + 1])) ++k;   /* plain scan of the edges */
            int ta = type[i] < type[j] ? type[i] : type[j];
            int tb = type[i] < type[j] ? type[j] : type[i];
            int pidx = ta * (2 * n_types - ta - 1) / 2 + tb;
            counts[(size_t)pidx * n_bins + k] += 1ull;
        }
    free(e);
}

/* Proton-transfer coordinate (Sec. 3.2, Fig. 11): for every proton h
 * (bond[h] >= 0, the index of its bonding oxygen), v = d(O_bond, h) -
 * min over the other acceptors O of d(O, h), acceptors being the atoms with
 * acceptor[j] != 0. Distances sqrtf(r2_f32) and the difference in FP32
 * (NaN for non-protons or without another acceptor). hist[k] += 1 when
 * e_k <= v < e_(k+1), e_k = (float)(v_min + k (v_max - v_min) / n_bins)
 * formed in FP64 (values outside [e_0, e_(n_bins)) are not counted).        */
void or_pt_coordinate(int n, const double* x, const double* box, const int* bond, const int* acceptor,
                      double v_min, double v_max, int n_bins, float* v, unsigned long long* hist)
{
    box32 b = make_box32(box);
    float* e = malloc(sizeof(float) * (n_bins + 1));
    for (int k = 0; k <= n_bins; ++k) e[k] = (float)(v_min + k * ((v_max - v_min) / n_bins));
    for (int h = 0; h < n; ++h) {
        v[h] = NAN;
        if (bond[h] < 0) continue;
        float db = sqrtf(r2_f32(x, h, bond[h], &b));
        float dn = INFINITY;
        for (int j = 0; j < n; ++j) {
            if (j == bond[h] || j == h || !acceptor[j]) continue;
            float d = sqrtf(r2_f32(x, h, j, &b));
            if (d < dn) dn = d;
        }
        if (dn == INFINITY) continue;
        float vv = db - dn;
        v[h] = vv;
        if (hist != NULL && vv >= e[0] && vv < e[n_bins]) {
            int k = 0;
            while (!(vv < e[k + 1])) ++k;
            hist[k] += 1ull;
        }
    }
    free(e);
}

/* g(r) per element pair (Figs. 8, 9): the pair counts of the shell
 * [k dr, (k + 1) dr), dr = r_max / n_bins, summed over n_configs bead
 * configurations, divided by the ideal-gas expectation
 * n_configs n_pairs shell_k / volume, shell_k = 4/3 pi ((k+1)^3 - k^3) dr^3,
 * n_pairs = n_a n_b (a != b) or n_a (n_a - 1) / 2 (a = b). Pair p of types
 * a <= b is p = a (2T - a - 1) / 2 + b, as in or_rdf_counts.              */
void or_rdf_gr(int n_types, const int* n_per_type, double volume, double r_max, int n_bins,
               double n_configs, const unsigned long long* counts, double* g)
{
    double dr = r_max / n_bins;
    int p = 0;
    for (int a = 0; a < n_types; ++a)
        for (int b = a; b < n_types; ++b, ++p) {
            double na = n_per_type[a], nb = n_per_type[b];
            double pairs = (a == b) ? na * (na - 1.0) / 2.0 : na * nb;
            for (int k = 0; k < n_bins; ++k) {
                double r0 = k * dr, r1 = (k + 1) * dr;
                double shell = 4.0 / 3.0 * M_PI * (r1 * r1 * r1 - r0 * r0 * r0);
                double ideal = n_configs * pairs * shell / volume;
                g[(size_t)p * n_bins + k] = ideal > 0.0 ? (double)counts[(size_t)p * n_bins + k] / ideal : 0.0;
            }
        }
}

/* Path-integral reweighting of Sec. 2.5, one sample of the bead-resolved
 * CV histogram. Under a bias V_b acting on every bead's CV the ring
 * polymer's configurational weight carries exp(-beta_P sum_k V_b(s_k)),
 * beta_P = 1 / (k_B T P) the ring polymer's inverse temperature; the sample
 * enters with the inverse factor w = exp(beta_P sum_k V_b(s_k) - shift)
 * (w = exp(-shift) without a bias). Bead k's CV falls in bin
 * b = floor((s_k - s_min) inv_ds), inv_ds = n_bins / (s_max - s_min), and
 * is counted when 0 <= b < n_bins: hist[k][b] += w. Every sample adds w to
 * *wsum, binned or not (the normalisation of the probability density).    */
void or_cv_histogram(int P, const double* s, const double* vb, double T, double s_min, double inv_ds,
                     int n_bins, double log_w_shift, double* hist, double* wsum)
{
    double v = 0.0;
    for (int k = 0; k < P; ++k) v += vb[k];
    double w = exp(v / (KB * T * P) - log_w_shift);
    for (int k = 0; k < P; ++k) {
        double t = (s[k] - s_min) * inv_ds;
        if (t >= 0.0 && t < (double)n_bins) hist[(size_t)k * n_bins + (int)floor(t)] += w;
    }
    *wsum += w;
}

/* Sec. 2.5: each bead's free energy F_k(s) = -k_B T ln p_k(s), p_k the
 * probability density of bead k's CV (histogram / (wsum ds)), and the
 * path-integral free energy F(s) = -k_B T ln[(1/P) sum_k p_k(s)], which is
 * -k_B T ln[(1/P) sum_k exp(-F_k(s) / k_B T)]. T is the physical
 * temperature; empty bins give +inf. Fk may be NULL.                       */
void or_pi_fes(int P, int n_bins, const double* hist, double wsum, double ds, double T, double* F, double* Fk)
{
    double kT = KB * T;
    for (int b = 0; b < n_bins; ++b) {
        double tot = 0.0;
        for (int k = 0; k < P; ++k) {
            double h = hist[(size_t)k * n_bins + b];
            tot += h;
            if (Fk) Fk[(size_t)k * n_bins + b] = h > 0.0 ? -kT * log(h / (wsum * ds)) : INFINITY;
        }
        F[b] = tot > 0.0 ? -kT * log(tot / (P * wsum * ds)) : INFINITY;
    }
}

/* Sec. 2.5: the converged well-tempered bias is V(s) = -(1 - 1/gamma) F(s)
 * up to a constant, so F(s) = -(gamma / (gamma - 1)) V(s).                 */
void or_metad_fes(const or_metad* md, int n, const double* s, double* F)
{
    for (int i = 0; i < n; ++i) F[i] = -(md->gamma / (md->gamma - 1.0)) * or_metad_bias(md, s[i], NULL);
}
