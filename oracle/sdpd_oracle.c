/*
 * sdpd_oracle.c -- plain FP64 CPU reference of the SDPD-DEM per-timestep
 * interaction step of Tsuzuki, "DEMocritus" (arXiv 2002.03120).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  The GPU library shares no
 * code, header, table or helper with it; the two meet only through arrays of
 * plain numbers produced by the seeded case generators.
 *
 * The code follows the paper's algorithms in their order:
 *   Algorithm 1  compute_total_processes: per step, velver = 1, 2:
 *                neighbour list -> density -> pressure -> pressure smoothing
 *                -> compute_force -> update
 *   Algorithm 2  compute_force: fluid -> fpi_action -> fpi_reaction -> rigid
 * and the equations of Section 2 (Eqs. govern, FijC, FijD, FijR, FijT, kernel,
 * F, compdens, prtcpres, dem_fnij .. deminputF, lubri, F_fpi_PG, F_fpi_DG,
 * beta, F_fpi_DG_reac, fvfdef, newton1, newton2).
 *
 * Where the paper is silent or garbled the reading taken is noted inline as
 * "reading:".  Everything is double precision; build with -ffp-contract=off so
 * that no multiply-add is fused behind the reader's back.
 *
 * Parity pins: every function here is checked by the CPU test-suite against a
 * closed form, an invariant or brute force (tests/test_oracle_*.py).  The
 * viscometer-with-solids and dam-break trajectories have no printed data to
 * compare with: their absolute values are "parity unpinned"; only invariants
 * (momentum balance, no escape) are checked for them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

enum { T_FLUID = 0, T_RIGID = 1, T_INNER_WALL = 2, T_OUTER_WALL = 3 };

/* Input parameters of one instance (Table 1 of the paper, plus the readings'
 * constants).  Field order is mirrored by oracle/__init__.py. */
typedef struct {
    double dx, r_c, dt;               /* initial spacing, kernel radius h, time step */
    double rho0, p0, alpha, beta_p;   /* Eq. prtcpres */
    double eta, xi, kBT;              /* Section 2.1 */
    double coeff_c, coeff_d, coeff_r, coeff_t; /* force switches (Coeff_f*ij) */
    double origin[3], box[3];
    double g[3];                      /* uniform acceleration (gravity) */
    double body_amp;                  /* reverse-Poiseuille forcing amplitude (accel.) */
    double artvis_alpha, artvis_e;    /* collision-method constants */
    double kn, restitution, nu_p, E_p, mu_fric; /* Section 2.2 */
    double lub_gap_min;               /* lubrication gap floor, fraction of d */
    double eps_min;                   /* lower clamp of the fluid volume fraction */
    int periodic[3];
    int body_axis, split_axis;        /* forcing direction, splitting direction */
    int pressure_filter, clamp_negative_p, artvis, dem_law;
    int density_reinit;               /* 1: Shepard density reinitialisation (reading B5) */
    uint64_t seed;
} orc_params;

typedef struct {
    orc_params P;
    int inst;
    int n;
    int K;                            /* contact-history slots per rigid particle */
    long long step;
    double *x, *v, *w;                /* [n][3] */
    int *type;
    double *R, *m, *I, *lever;
    double *d, *rho, *p;              /* number density, mass density, pressure */
    /* neighbour lists (CSR, all j != i with r_ij < h) */
    int *nb_off, *nb;
    long nb_len, nb_cap;
    /* force components, [n][3] each */
    double *F_sdpd, *F_pg, *F_dg, *F_rxn, *F_dem, *F_lub, *F_ext, *F;
    double *N_sdpd, *N_dem, *N;
    /* per-particle fluid-particle interaction quantities (rigid entries only) */
    double *eps, *Ssum, *vf;          /* vf is [n][3] */
    /* contact history: K slots per particle, partner code and delta_t */
    int *hist_n, *hist_partner;
    double *hist_delta;
    int *new_n, *new_partner;
    double *new_delta;
    int overflow;
    unsigned char *only;   /* if set: forces only for particles with only[i] != 0 */
} orc_sim;

/* ------------------------------------------------------------------ */
/* Kernel function: Lucy kernel, Eq. kernel, and F(r) = -W'(r)/r, Eq. F */
double orc_W(double r, double h)
{
    if (r >= h) return 0.0;
    double q = r / h;
    double omq = 1.0 - q;
    return 105.0 / (16.0 * ORC_PI * h * h * h) * (1.0 + 3.0 * q) * omq * omq * omq;
}

double orc_Fk(double r, double h)
{
    if (r >= h) return 0.0;
    double q = r / h;
    double omq = 1.0 - q;
    return 315.0 / (4.0 * ORC_PI * h * h * h * h * h) * omq * omq;
}

/* Normalisation of the kernel coefficient (Section 3.3, compute_particle_dens).
 * reading: C_n = 1 / (dx^3 * sum over a perfect cubic lattice of W, self
 * included), so that a perfect lattice has number density exactly 1/dx^3. */
double orc_kernel_norm(double dx, double h)
{
    int nmax = (int)ceil(h / dx) + 1;
    double s = 0.0;
    for (int a = -nmax; a <= nmax; ++a)
        for (int b = -nmax; b <= nmax; ++b)
            for (int c = -nmax; c <= nmax; ++c) {
                double r = sqrt((double)(a * a + b * b + c * c)) * dx;
                s += orc_W(r, h);
            }
    return 1.0 / (dx * dx * dx * s);
}

/* Equation of state, Eq. prtcpres. */
double orc_eos(double rho, double rho0, double p0, double alpha, double beta_p)
{
    return p0 * pow(rho / rho0, alpha) - beta_p;
}

/* ------------------------------------------------------------------ */
/* Counter-based random numbers.  The paper draws its Wiener increments with
 * MT19937-64 (Section 3.3); this oracle and the GPU path both draw them from
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), keyed per pair so the
 * matrix dW_ij is the same for (i,j) and (j,i), as the paper requires. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Six standard normals for the unordered pair {gi, gj} at time step `step`:
 * two Philox blocks (last counter word 0 and 1), uniforms
 * U = ((u >> 9) + 0.5) * 2^-23 (24 significant bits: exact in float and
 * double), Box-Muller on (U0,U1), (U2,U3), (U4,U5). */
void orc_pair_normals(uint64_t seed, int inst, uint32_t gi, uint32_t gj,
                      long long step, double z[6])
{
    uint32_t lo = gi < gj ? gi : gj, hi = gi < gj ? gj : gi;
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) ^ (uint32_t)inst };
    uint32_t u[8];
    for (uint32_t blk = 0; blk < 2; ++blk) {
        uint32_t ctr[4] = { lo, hi, (uint32_t)step, blk };
        orc_philox4x32_10(ctr, key, u + 4 * blk);
    }
    double U[6];
    for (int k = 0; k < 6; ++k)
        U[k] = ((double)(u[k] >> 9) + 0.5) * (1.0 / 8388608.0);
    for (int k = 0; k < 3; ++k) {
        double rad = sqrt(-2.0 * log(U[2 * k]));
        double ang = 2.0 * ORC_PI * U[2 * k + 1];
        z[2 * k] = rad * cos(ang);
        z[2 * k + 1] = rad * sin(ang);
    }
}

/* Random impulse direction term of Eq. FijT.  dW_ij has iid N(0, dt) entries;
 * only its symmetric part enters (reading of Eq. reldWij: the missing
 * transpose and identity restored, dWbar^S = (dW + dW^T)/2 - tr[dW]/3 * 1).
 * The symmetric part of a 3x3 iid-normal matrix has N(0,1) diagonal and
 * N(0,1/2) off-diagonal entries; it is drawn directly from the six normals:
 *   S_xx = z0, S_yy = z1, S_zz = z2, S_xy = z3/sqrt2, S_xz = z4/sqrt2,
 *   S_yz = z5/sqrt2.
 * Returns out = (sa * (S - trS/3) + sb * trS/3) . e  (unit-variance S). */
void orc_noise_vector(const double z[6], double sa, double sb, const double e[3], double out[3])
{
    const double is2 = 1.0 / sqrt(2.0);
    double S[3][3];
    S[0][0] = z[0]; S[1][1] = z[1]; S[2][2] = z[2];
    S[0][1] = S[1][0] = z[3] * is2;
    S[0][2] = S[2][0] = z[4] * is2;
    S[1][2] = S[2][1] = z[5] * is2;
    double tr3 = (S[0][0] + S[1][1] + S[2][2]) / 3.0;
    for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int b = 0; b < 3; ++b) {
            double dev = S[a][b] - (a == b ? tr3 : 0.0);
            double m = sa * dev + (a == b ? sb * tr3 : 0.0);
            acc += m * e[b];
        }
        out[a] = acc;
    }
}

/* ------------------------------------------------------------------ */
/* Drag, Eqs. F_fpi_DG, beta, C_D, Re_p.
 * reading (sign): F^DG acts on the rigid particle along (v_f - v_s); the
 * printed (v_i - v_f) would accelerate the slip.
 * reading (singularities): beta V_s/(1-eps) is evaluated in closed form so the
 * (1-eps) factor cancels and C_D*Re_p replaces C_D:
 *   eps <= 0.8 (Ergun):  [150 mu (1-eps)/(eps d^2) + 1.75 rho |dv| / d] V_s dv
 *   eps >  0.8 (Wen-Yu): 3/4 (C_D Re_p) mu eps^-2.65 / d^2 * V_s dv
 *   C_D Re_p = 24 (1 + 0.15 Re_p^0.687) for Re_p <= 1000, else 0.44 Re_p.
 * dv = v_f - v_s, Re_p = rho d eps |dv| / mu.  Writes the force into out. */
void orc_drag_force(double eps, double d, double rho, double mu, double Vs,
                    const double dv[3], double out[3])
{
    double mag = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    double coef;
    if (eps <= 0.8) {
        coef = 150.0 * mu * (1.0 - eps) / (eps * d * d) + 1.75 * rho * mag / d;
    } else {
        double Re = rho * d * eps * mag / mu;
        double CDRe = (Re <= 1000.0) ? 24.0 * (1.0 + 0.15 * pow(Re, 0.687)) : 0.44 * Re;
        coef = 0.75 * CDRe * mu * pow(eps, -2.65) / (d * d);
    }
    for (int k = 0; k < 3; ++k) out[k] = coef * Vs * dv[k];
}

/* DEM coefficients, Section 2.2.
 * law 0: Eqs. deminputA..F as printed (Hertz constant used in the linear law).
 * law 1 (reading for the SI configurations): linear spring kn given, damping
 *   from a restitution coefficient e: c = 2 zeta sqrt(m* k),
 *   zeta = -ln e / sqrt(pi^2 + ln^2 e);  kt = kn / (2 (1 + nu)).
 * mj <= 0 or Rj <= 0 denotes a wall plane (infinite mass / radius).
 * out = {kn, kt, cn, ct}. */
void orc_dem_coeffs(const orc_params *P, double Ri, double Rj, double mi, double mj, double out[4])
{
    double mstar = (mj > 0.0) ? mi * mj / (mi + mj) : mi;
    double kn, kt, cn, ct;
    if (P->dem_law == 0) {
        double D = (1.0 - P->nu_p * P->nu_p) / (P->E_p * ORC_PI);
        double Reff = (Rj > 0.0) ? Ri * Rj / (Ri + Rj) : Ri;
        kn = 4.0 / (3.0 * ORC_PI) * (1.0 / (D + D)) * sqrt(Reff);
        kt = kn / (2.0 * (1.0 + P->nu_p));
        cn = 2.0 * sqrt(2.0 * mstar * kn);
        ct = 2.0 * sqrt(2.0 * mstar * kt);
    } else {
        double le = log(P->restitution);
        double zeta = -le / sqrt(ORC_PI * ORC_PI + le * le);
        kn = P->kn;
        kt = kn / (2.0 * (1.0 + P->nu_p));
        cn = 2.0 * zeta * sqrt(mstar * kn);
        ct = 2.0 * zeta * sqrt(mstar * kt);
    }
    out[0] = kn; out[1] = kt; out[2] = cn; out[3] = ct;
}

/* ------------------------------------------------------------------ */
static double min_image(double d, double L, int periodic)
{
    if (!periodic) return d;
    if (d > 0.5 * L) return d - L;
    if (d < -0.5 * L) return d + L;
    return d;
}

/* r_ij = r_i - r_j with the minimum-image convention on periodic axes
 * (equivalent to the paper's halo copies, Section 2.5, for boxes at least
 * two kernel radii wide); returns r^2 = (x*x + y*y) + z*z. */
static double pair_vec(const orc_params *P, const double *xi, const double *xj, double r[3])
{
    for (int a = 0; a < 3; ++a)
        r[a] = min_image(xi[a] - xj[a], P->box[a], P->periodic[a]);
    return (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2];
}

static void cross(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static int is_mobile(int t) { return t == T_FLUID || t == T_RIGID; }

/* ------------------------------------------------------------------ */
orc_sim *orc_create(const orc_params *P, int inst, int n, const double *x, const double *v,
                    const double *w, const int *type, const double *R, const double *m, int K)
{
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->P = *P;
    s->inst = inst;
    s->n = n;
    s->K = K;
    size_t n3 = (size_t)n * 3;
    s->x = (double *)malloc(n3 * sizeof(double));
    s->v = (double *)malloc(n3 * sizeof(double));
    s->w = (double *)malloc(n3 * sizeof(double));
    memcpy(s->x, x, n3 * sizeof(double));
    memcpy(s->v, v, n3 * sizeof(double));
    memcpy(s->w, w, n3 * sizeof(double));
    s->type = (int *)malloc((size_t)n * sizeof(int));
    memcpy(s->type, type, (size_t)n * sizeof(int));
    s->R = (double *)malloc((size_t)n * sizeof(double));
    s->m = (double *)malloc((size_t)n * sizeof(double));
    s->I = (double *)malloc((size_t)n * sizeof(double));
    s->lever = (double *)malloc((size_t)n * sizeof(double));
    memcpy(s->R, R, (size_t)n * sizeof(double));
    memcpy(s->m, m, (size_t)n * sizeof(double));
    for (int i = 0; i < n; ++i) {
        /* Eq. newton2 needs an inertia (Table 1 --iner, no value printed).
         * reading: solid-sphere inertia 2/5 m a^2 with a = R for rigid
         * particles and a = dx/2 for fluid particles; the torque lever of
         * Section 2.6 is R (rigid) or dx/2 (fluid). */
        double a = (s->type[i] == T_RIGID) ? s->R[i] : 0.5 * P->dx;
        s->I[i] = 0.4 * s->m[i] * a * a;
        s->lever[i] = a;
    }
    s->d = (double *)calloc((size_t)n, sizeof(double));
    s->rho = (double *)calloc((size_t)n, sizeof(double));
    s->p = (double *)calloc((size_t)n, sizeof(double));
    s->nb_off = (int *)calloc((size_t)n + 1, sizeof(int));
    s->nb_cap = 0;
    s->nb = NULL;
    double **comp[] = { &s->F_sdpd, &s->F_pg, &s->F_dg, &s->F_rxn, &s->F_dem, &s->F_lub,
                        &s->F_ext, &s->F, &s->N_sdpd, &s->N_dem, &s->N, &s->vf };
    for (size_t k = 0; k < sizeof(comp) / sizeof(comp[0]); ++k)
        *comp[k] = (double *)calloc(n3, sizeof(double));
    s->eps = (double *)calloc((size_t)n, sizeof(double));
    s->Ssum = (double *)calloc((size_t)n, sizeof(double));
    s->hist_n = (int *)calloc((size_t)n, sizeof(int));
    s->hist_partner = (int *)calloc((size_t)n * K + 1, sizeof(int));
    s->hist_delta = (double *)calloc((size_t)n * K * 3 + 1, sizeof(double));
    s->new_n = (int *)calloc((size_t)n, sizeof(int));
    s->new_partner = (int *)calloc((size_t)n * K + 1, sizeof(int));
    s->new_delta = (double *)calloc((size_t)n * K * 3 + 1, sizeof(double));
    return s;
}

/* Restrict the force evaluation to the particles with mask[i] != 0 (a
 * sample; every other stage still runs for all).  mask = NULL: all. */
void orc_set_sample(orc_sim *s, const unsigned char *mask)
{
    free(s->only);
    s->only = NULL;
    if (mask) {
        s->only = (unsigned char *)malloc((size_t)(s->n > 0 ? s->n : 1));
        memcpy(s->only, mask, (size_t)s->n);
    }
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->only);
    void *ptrs[] = { s->x, s->v, s->w, s->type, s->R, s->m, s->I, s->lever, s->d, s->rho, s->p,
                     s->nb_off, s->nb, s->F_sdpd, s->F_pg, s->F_dg, s->F_rxn, s->F_dem, s->F_lub,
                     s->F_ext, s->F, s->N_sdpd, s->N_dem, s->N, s->vf, s->eps, s->Ssum,
                     s->hist_n, s->hist_partner, s->hist_delta, s->new_n, s->new_partner,
                     s->new_delta };
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    free(s);
}

void orc_set_step(orc_sim *s, long long step) { s->step = step; }
long long orc_get_step(const orc_sim *s) { return s->step; }

void orc_set_state(orc_sim *s, const double *x, const double *v, const double *w)
{
    size_t n3 = (size_t)s->n * 3;
    if (x) memcpy(s->x, x, n3 * sizeof(double));
    if (v) memcpy(s->v, v, n3 * sizeof(double));
    if (w) memcpy(s->w, w, n3 * sizeof(double));
}

/* Test hook: impose number densities d and pressures p (either may be NULL)
 * in place of those of orc_density, e.g. a hydrostatic field on a perfect
 * lattice; rho follows as m_f d.  The force routines read them as they are. */
void orc_set_fields(orc_sim *s, const double *d, const double *p)
{
    const double mf = s->P.rho0 * s->P.dx * s->P.dx * s->P.dx;
    for (int i = 0; i < s->n; ++i) {
        if (d) { s->d[i] = d[i]; s->rho[i] = mf * d[i]; }
        if (p) s->p[i] = p[i];
    }
}

void orc_get_state(const orc_sim *s, double *x, double *v, double *w, double *F, double *N,
                   double *d, double *p)
{
    size_t n3 = (size_t)s->n * 3;
    if (x) memcpy(x, s->x, n3 * sizeof(double));
    if (v) memcpy(v, s->v, n3 * sizeof(double));
    if (w) memcpy(w, s->w, n3 * sizeof(double));
    if (F) memcpy(F, s->F, n3 * sizeof(double));
    if (N) memcpy(N, s->N, n3 * sizeof(double));
    if (d) memcpy(d, s->d, (size_t)s->n * sizeof(double));
    if (p) memcpy(p, s->p, (size_t)s->n * sizeof(double));
}

/* Component forces: which = 0 sdpd, 1 pg, 2 dg, 3 rxn, 4 dem, 5 lub, 6 ext,
 * 7 N_sdpd, 8 N_dem, 9 fluid velocity v_f seen by rigid particles. */
void orc_get_component(const orc_sim *s, int which, double *out)
{
    double *src[] = { s->F_sdpd, s->F_pg, s->F_dg, s->F_rxn, s->F_dem, s->F_lub, s->F_ext,
                      s->N_sdpd, s->N_dem, s->vf };
    memcpy(out, src[which], (size_t)s->n * 3 * sizeof(double));
}

void orc_get_fpi(const orc_sim *s, double *eps, double *Ssum)
{
    if (eps) memcpy(eps, s->eps, (size_t)s->n * sizeof(double));
    if (Ssum) memcpy(Ssum, s->Ssum, (size_t)s->n * sizeof(double));
}

/* Contact history access (rigid particles): partner codes and delta_t. */
void orc_get_history(const orc_sim *s, int *counts, int *partner, double *delta)
{
    memcpy(counts, s->hist_n, (size_t)s->n * sizeof(int));
    memcpy(partner, s->hist_partner, (size_t)s->n * s->K * sizeof(int));
    memcpy(delta, s->hist_delta, (size_t)s->n * s->K * 3 * sizeof(double));
}

void orc_set_history(orc_sim *s, const int *counts, const int *partner, const double *delta)
{
    memcpy(s->hist_n, counts, (size_t)s->n * sizeof(int));
    memcpy(s->hist_partner, partner, (size_t)s->n * s->K * sizeof(int));
    memcpy(s->hist_delta, delta, (size_t)s->n * s->K * 3 * sizeof(double));
}

/* ------------------------------------------------------------------ */
/* compute_neighbor_list (Section 3.2, Algorithm 1): background grid with one
 * head particle per cell and a linked list through the particles (Grest et
 * al.); every particle then collects the j != i with r_ij < h from the
 * surrounding cells.  Grid cells are at least h wide. */
int orc_neighbors(orc_sim *s)
{
    const orc_params *P = &s->P;
    int n = s->n;
    double lo[3], cs[3];
    int nc[3];
    for (int a = 0; a < 3; ++a) {
        if (P->periodic[a]) {
            lo[a] = P->origin[a];
            nc[a] = (int)floor(P->box[a] / P->r_c);
            if (nc[a] < 1) nc[a] = 1;
            cs[a] = P->box[a] / nc[a];
        } else {
            double mn = 1e300, mx = -1e300;
            for (int i = 0; i < n; ++i) {
                if (s->x[3 * i + a] < mn) mn = s->x[3 * i + a];
                if (s->x[3 * i + a] > mx) mx = s->x[3 * i + a];
            }
            if (n == 0) { mn = 0; mx = 0; }
            lo[a] = mn;
            cs[a] = P->r_c;
            nc[a] = (int)floor((mx - mn) / cs[a]) + 1;
        }
    }
    long ncell = (long)nc[0] * nc[1] * nc[2];
    int *head = (int *)malloc((size_t)ncell * sizeof(int));
    int *link = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    int *cell_of = (int *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(int));
    for (long c = 0; c < ncell; ++c) head[c] = -1;
    for (int i = n - 1; i >= 0; --i) {
        int cc[3];
        for (int a = 0; a < 3; ++a) {
            int k = (int)floor((s->x[3 * i + a] - lo[a]) / cs[a]);
            if (k < 0) k = 0;
            if (k >= nc[a]) k = nc[a] - 1;
            cc[a] = k;
            cell_of[3 * i + a] = k;
        }
        long c = ((long)cc[2] * nc[1] + cc[1]) * nc[0] + cc[0];
        link[i] = head[c];
        head[c] = i;
    }
    /* two passes over the particles, each owning its own list: count, then
     * (after a prefix sum of the counts) fill; the lists are the same as
     * one sequential pass would append, at any number of threads */
    const double rc2 = P->r_c * P->r_c;
    int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            long tot = 0;
            for (int i = 0; i < n; ++i) { s->nb_off[i] = (int)tot; tot += cnt[i]; }
            s->nb_len = tot;
            if (tot > s->nb_cap) {
                s->nb_cap = tot;
                s->nb = (int *)realloc(s->nb, (size_t)s->nb_cap * sizeof(int));
            }
        }
#pragma omp parallel for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            /* distinct neighbour cells (a small periodic grid may wrap onto itself) */
            long cells[27];
            int ncl = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dxo = -1; dxo <= 1; ++dxo) {
                        int off[3] = { dxo, dy, dz };
                        int cc[3];
                        int ok = 1;
                        for (int a = 0; a < 3; ++a) {
                            int k = cell_of[3 * i + a] + off[a];
                            if (P->periodic[a]) {
                                k = ((k % nc[a]) + nc[a]) % nc[a];
                            } else if (k < 0 || k >= nc[a]) {
                                ok = 0;
                            }
                            cc[a] = k;
                        }
                        if (!ok) continue;
                        long c = ((long)cc[2] * nc[1] + cc[1]) * nc[0] + cc[0];
                        int dup = 0;
                        for (int q = 0; q < ncl; ++q) if (cells[q] == c) dup = 1;
                        if (!dup) cells[ncl++] = c;
                    }
            int m = 0;
            int *out = pass ? s->nb + s->nb_off[i] : NULL;
            for (int q = 0; q < ncl; ++q) {
                for (int j = head[cells[q]]; j >= 0; j = link[j]) {
                    if (j == i) continue;
                    double r[3];
                    double r2 = pair_vec(P, s->x + 3 * i, s->x + 3 * j, r);
                    if (r2 < rc2) {
                        if (out) out[m] = j;
                        ++m;
                    }
                }
            }
            if (!pass) cnt[i] = m;
        }
    }
    free(cnt);
    s->nb_off[n] = (int)s->nb_len;
    free(head);
    free(link);
    free(cell_of);
    return 0;
}

/* Brute-force O(N^2) neighbour pairs (i<j) with r_ij < h, for pinning the
 * cell search.  Returns the number of pairs (writes at most cap). */
long orc_pairs_brute(const orc_params *P, int n, const double *x, long cap, int *ij)
{
    long cnt = 0;
    const double rc2 = P->r_c * P->r_c;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double r[3];
            if (pair_vec(P, x + 3 * i, x + 3 * j, r) < rc2) {
                if (cnt < cap) { ij[2 * cnt] = i; ij[2 * cnt + 1] = j; }
                ++cnt;
            }
        }
    return cnt;
}

/* Pairs (i<j) found by the last orc_neighbors call. */
long orc_get_pairs(const orc_sim *s, long cap, int *ij)
{
    long cnt = 0;
    for (int i = 0; i < s->n; ++i)
        for (int k = s->nb_off[i]; k < s->nb_off[i + 1]; ++k) {
            int j = s->nb[k];
            if (j > i) {
                if (cnt < cap) { ij[2 * cnt] = i; ij[2 * cnt + 1] = j; }
                ++cnt;
            }
        }
    return cnt;
}

/* ------------------------------------------------------------------ */
/* compute_particle_dens + compute_particle_pres (Algorithm 1; Eqs. compdens,
 * prtcpres).
 * reading: the pair forces need a number density (units 1/m^3), so
 *   d_i = C_n * sum_j W(r_ij)   (self term included, all particle types),
 *   rho_i = m_f d_i with m_f = rho0 dx^3,  p_i from Eq. prtcpres.
 * Outer-wall particles are not updated (Section 2.5): d = 1/dx^3.
 * Negative pressures are set to zero when clamp_negative_p is on (Section
 * 2.5, free surfaces). */
void orc_density(orc_sim *s)
{
    const orc_params *P = &s->P;
    const double h = P->r_c;
    const double Cn = orc_kernel_norm(P->dx, h);
    const double mf = P->rho0 * P->dx * P->dx * P->dx;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < s->n; ++i) {
        double di;
        if (s->type[i] == T_OUTER_WALL) {
            di = 1.0 / (P->dx * P->dx * P->dx);
        } else {
            double sum = orc_W(0.0, h);
            for (int k = s->nb_off[i]; k < s->nb_off[i + 1]; ++k) {
                int j = s->nb[k];
                double r[3];
                double r2 = pair_vec(P, s->x + 3 * i, s->x + 3 * j, r);
                sum += orc_W(sqrt(r2), h);
            }
            di = Cn * sum;
        }
        s->d[i] = di;
        s->rho[i] = mf * di;
        double pi = orc_eos(s->rho[i], P->rho0, P->p0, P->alpha, P->beta_p);
        if (P->clamp_negative_p && pi < 0.0) pi = 0.0;
        s->p[i] = pi;
    }
}

/* Density reinitialisation (Section 2.1 and the text under Algorithm 1,
 * after Colagrossi and Landrini 2003).  reading B5: the zeroth-order (Shepard)
 * form applied to the summation density at every evaluation,
 *   d~_i = (W(0) + sum_j W_ij) / (W(0)/d_i + sum_j W_ij/d_j),
 * i.e. the W-weighted harmonic mean of the densities around i; outer-wall
 * particles keep theirs.  Pressure follows from the EOS again. */
void orc_reinit(orc_sim *s)
{
    const orc_params *P = &s->P;
    if (!P->density_reinit) return;
    const double h = P->r_c;
    const double mf = P->rho0 * P->dx * P->dx * P->dx;
    double *dn = (double *)malloc((size_t)(s->n > 0 ? s->n : 1) * sizeof(double));
    #pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < s->n; ++i) {
        if (s->type[i] == T_OUTER_WALL) { dn[i] = s->d[i]; continue; }
        double w0 = orc_W(0.0, h);
        double num = w0, den = w0 / s->d[i];
        for (int k = s->nb_off[i]; k < s->nb_off[i + 1]; ++k) {
            int j = s->nb[k];
            double r[3];
            double r2 = pair_vec(P, s->x + 3 * i, s->x + 3 * j, r);
            double W = orc_W(sqrt(r2), h);
            num += W;
            den += W / s->d[j];
        }
        dn[i] = num / den;
    }
    for (int i = 0; i < s->n; ++i) {
        s->d[i] = dn[i];
        s->rho[i] = mf * dn[i];
        double pi = orc_eos(s->rho[i], P->rho0, P->p0, P->alpha, P->beta_p);
        if (P->clamp_negative_p && pi < 0.0) pi = 0.0;
        s->p[i] = pi;
    }
    free(dn);
}

/* smoothe_particle_pres (Algorithm 1): pressure filter (Imoto 2019).
 * reading: Shepard average over the density neighbour set, self included,
 *   p~_i = (p_i W(0) + sum_j p_j W_ij) / (W(0) + sum_j W_ij);
 * outer-wall particles keep their pressure. */
void orc_filter(orc_sim *s)
{
    const orc_params *P = &s->P;
    if (!P->pressure_filter) return;
    const double h = P->r_c;
    double *pn = (double *)malloc((size_t)(s->n > 0 ? s->n : 1) * sizeof(double));
    #pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < s->n; ++i) {
        if (s->type[i] == T_OUTER_WALL) { pn[i] = s->p[i]; continue; }
        double w0 = orc_W(0.0, h);
        double num = s->p[i] * w0, den = w0;
        for (int k = s->nb_off[i]; k < s->nb_off[i + 1]; ++k) {
            int j = s->nb[k];
            double r[3];
            double r2 = pair_vec(P, s->x + 3 * i, s->x + 3 * j, r);
            double W = orc_W(sqrt(r2), h);
            num += s->p[j] * W;
            den += W;
        }
        pn[i] = num / den;
    }
    memcpy(s->p, pn, (size_t)s->n * sizeof(double));
    free(pn);
}

/* ------------------------------------------------------------------ */
/* The SDPD pair force of Eqs. FijC, FijD, FijR, FijT on particle i from j,
 * with the number densities of the reading above in place of rho.
 * with_rt selects whether the rotational and random parts are included
 * (they are not for pairs that involve a rigid particle, Section 2.4).
 * Writes the conservative + dissipative part into fcd and the total into f. */
static void sdpd_pair(const orc_sim *s, int i, int j, const double r[3], double rr,
                      int with_rt, double fcd[3], double f[3])
{
    const orc_params *P = &s->P;
    const double h = P->r_c;
    double e[3] = { r[0] / rr, r[1] / rr, r[2] / rr };
    double Fij = orc_Fk(rr, h);
    double di = s->d[i], dj = s->d[j];
    /* Eq. FijC */
    double pc = s->p[i] / (di * di) + s->p[j] / (dj * dj);
    double fc[3];
    for (int a = 0; a < 3; ++a) fc[a] = P->coeff_c * pc * Fij * r[a];
    /* gamma^a, gamma^b (Section 2.1) */
    double ga = (20.0 * P->eta / 3.0 - 4.0 * P->xi) * Fij / (di * dj);
    double gb = (17.0 * P->xi - 40.0 * P->eta / 3.0) * Fij / (di * dj);
    /* Eq. FijD */
    double vij[3];
    for (int a = 0; a < 3; ++a) vij[a] = s->v[3 * i + a] - s->v[3 * j + a];
    double ev = dot(e, vij);
    double fd[3];
    for (int a = 0; a < 3; ++a)
        fd[a] = P->coeff_d * (-ga * (vij[a] + e[a] * ev / 3.0) - 2.0 * gb / 3.0 * e[a] * ev);
    for (int a = 0; a < 3; ++a) { fcd[a] = fc[a] + fd[a]; f[a] = fcd[a]; }
    if (!with_rt) return;
    /* Eq. FijR */
    double half_r[3] = { 0.5 * r[0], 0.5 * r[1], 0.5 * r[2] };
    double wsum[3];
    for (int a = 0; a < 3; ++a) wsum[a] = s->w[3 * i + a] + s->w[3 * j + a];
    double rxw[3];
    cross(half_r, wsum, rxw);
    for (int a = 0; a < 3; ++a) f[a] += P->coeff_r * (-ga * rxw[a]);
    /* Eq. FijT: sigma^{a,b} = 2 sqrt(kBT gamma^{a,b}); dW_ij = sqrt(dt) Z so
     * (sigma dW . e)/dt = (sigma Z . e)/sqrt(dt). */
    if (P->coeff_t != 0.0 && P->kBT > 0.0) {
        double sa = 2.0 * sqrt(P->kBT * ga);
        double sb = 2.0 * sqrt(P->kBT * gb);
        double z[6];
        orc_pair_normals(P->seed, s->inst, (uint32_t)i, (uint32_t)j, s->step, z);
        double nv[3];
        orc_noise_vector(z, sa, sb, e, nv);
        double isdt = 1.0 / sqrt(P->dt);
        for (int a = 0; a < 3; ++a) f[a] += P->coeff_t * nv[a] * isdt;
    }
}

/* compute_fluid (Algorithm 2): SDPD forces on fluid particles from all their
 * neighbours (rigid neighbours included: single-pressure hypothesis,
 * Section 2.4), and the pressure-gradient force on rigid particles.
 * reading (Eq. F_fpi_PG, dimensionally garbled as printed): the force on a
 * fluid particle of volume 1/d_s, scaled to the sphere volume,
 *   F^PG_s = V_s d_s sum_{fluid j} (F^C_sj + F^D_sj).
 * Torque (Section 2.6): N_i += (-l_i e_ij) x F_ij with l_i the lever. */
static void compute_fluid(orc_sim *s)
{
    const orc_params *P = &s->P;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < s->n; ++i) {
        if (s->only && !s->only[i]) continue;
        double *Fs = s->F_sdpd + 3 * i, *Ns = s->N_sdpd + 3 * i, *Fp = s->F_pg + 3 * i;
        int ti = s->type[i];
        if (ti != T_FLUID && ti != T_RIGID) continue;
        double pg[3] = { 0, 0, 0 }, npg[3] = { 0, 0, 0 };
        for (int k = s->nb_off[i]; k < s->nb_off[i + 1]; ++k) {
            int j = s->nb[k];
            int tj = s->type[j];
            double r[3];
            double r2 = pair_vec(P, s->x + 3 * i, s->x + 3 * j, r);
            double rr = sqrt(r2);
            double e[3] = { r[0] / rr, r[1] / rr, r[2] / rr };
            double lev[3] = { -s->lever[i] * e[0], -s->lever[i] * e[1], -s->lever[i] * e[2] };
            double fcd[3], f[3], tq[3];
            if (ti == T_FLUID) {
                int with_rt = (tj != T_RIGID);
                sdpd_pair(s, i, j, r, rr, with_rt, fcd, f);
                for (int a = 0; a < 3; ++a) Fs[a] += f[a];
                cross(lev, f, tq);
                for (int a = 0; a < 3; ++a) Ns[a] += tq[a];
            } else if (tj == T_FLUID) {
                sdpd_pair(s, i, j, r, rr, 0, fcd, f);
                for (int a = 0; a < 3; ++a) pg[a] += fcd[a];
                cross(lev, fcd, tq);
                for (int a = 0; a < 3; ++a) npg[a] += tq[a];
            }
        }
        if (ti == T_RIGID) {
            double Vs = 4.0 / 3.0 * ORC_PI * s->R[i] * s->R[i] * s->R[i];
            double scale = Vs * s->d[i];
            for (int a = 0; a < 3; ++a) {
                Fp[a] = scale * pg[a];
                Ns[a] += scale * npg[a];
            }
        }
    }
}

/* compute_fpi_action (Algorithm 2): fluid volume fraction (Eq. fvfdef) and
 * drag (Eqs. F_fpi_DG, beta) on every rigid particle.
 * reading: eps_s = |V_f - sum_k V_k| / V_f over the rigid particles k within
 * h of s, s included (V_f = 4/3 pi h^3), clamped to [eps_min, 1]; v_f is the
 * W-weighted mean velocity of the fluid neighbours, v_f = U_s / S_s with
 * S_s = sum_{fluid j} W_sj; no fluid neighbour -> no drag. */
static void compute_fpi_action(orc_sim *s)
{
    const orc_params *P = &s->P;
    const double h = P->r_c;
    const double Vf = 4.0 / 3.0 * ORC_PI * h * h * h;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < s->n; ++i) {
        if (s->type[i] != T_RIGID) continue;
        double Vsum = 4.0 / 3.0 * ORC_PI * s->R[i] * s->R[i] * s->R[i];
        double S = 0.0, U[3] = { 0, 0, 0 };
        for (int k = s->nb_off[i]; k < s->nb_off[i + 1]; ++k) {
            int j = s->nb[k];
            double r[3];
            double rr = sqrt(pair_vec(P, s->x + 3 * i, s->x + 3 * j, r));
            if (s->type[j] == T_RIGID) {
                Vsum += 4.0 / 3.0 * ORC_PI * s->R[j] * s->R[j] * s->R[j];
            } else if (s->type[j] == T_FLUID) {
                double W = orc_W(rr, h);
                S += W;
                for (int a = 0; a < 3; ++a) U[a] += W * s->v[3 * j + a];
            }
        }
        double eps = fabs(Vf - Vsum) / Vf;
        if (eps > 1.0) eps = 1.0;
        if (eps < P->eps_min) eps = P->eps_min;
        s->eps[i] = eps;
        s->Ssum[i] = S;
        double *Fd = s->F_dg + 3 * i;
        if (S > 0.0) {
            double dv[3];
            for (int a = 0; a < 3; ++a) {
                s->vf[3 * i + a] = U[a] / S;
                dv[a] = s->vf[3 * i + a] - s->v[3 * i + a];
            }
            double Vs = 4.0 / 3.0 * ORC_PI * s->R[i] * s->R[i] * s->R[i];
            orc_drag_force(eps, 2.0 * s->R[i], P->rho0, P->eta, Vs, dv, Fd);
        } else {
            Fd[0] = Fd[1] = Fd[2] = 0.0;
        }
    }
}

/* compute_fpi_reaction (Algorithm 2; Eq. F_fpi_DG_reac).
 * reading: weights normalised per rigid particle so momentum is exchanged
 * exactly:  F^RXN_j = - sum_{rigid s, r_sj < h} F^DG_s W_sj / S_s. */
static void compute_fpi_reaction(orc_sim *s)
{
    const orc_params *P = &s->P;
    const double h = P->r_c;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int j = 0; j < s->n; ++j) {
        if (s->type[j] != T_FLUID) continue;
        if (s->only && !s->only[j]) continue;
        for (int k = s->nb_off[j]; k < s->nb_off[j + 1]; ++k) {
            int i = s->nb[k];
            if (s->type[i] != T_RIGID || !(s->Ssum[i] > 0.0)) continue;
            double r[3];
            double rr = sqrt(pair_vec(P, s->x + 3 * j, s->x + 3 * i, r));
            double W = orc_W(rr, h);
            for (int a = 0; a < 3; ++a) s->F_rxn[3 * j + a] -= s->F_dg[3 * i + a] * W / s->Ssum[i];
        }
    }
}

/* Tangential contact history lookup. */
static int hist_find(const orc_sim *s, int i, int partner, double out[3])
{
    for (int k = 0; k < s->hist_n[i]; ++k)
        if (s->hist_partner[i * s->K + k] == partner) {
            for (int a = 0; a < 3; ++a) out[a] = s->hist_delta[((size_t)i * s->K + k) * 3 + a];
            return 1;
        }
    out[0] = out[1] = out[2] = 0.0;
    return 0;
}

static void hist_push(orc_sim *s, int i, int partner, const double delta[3])
{
    int k = s->new_n[i];
    if (k >= s->K) { s->overflow = 1; return; }
    s->new_partner[i * s->K + k] = partner;
    for (int a = 0; a < 3; ++a) s->new_delta[((size_t)i * s->K + k) * 3 + a] = delta[a];
    s->new_n[i] = k + 1;
}

/* One DEM contact on rigid particle i (Eqs. dem_fnij .. slideref).
 * n points from the partner to i; overlap = L - (R_i + R_j) < 0.
 * reading (tangential velocity): the relative velocity of the two surface
 * points, v_t = v_ij - (v_ij.n) n - (R_i w_i + R_j w_j) x n, for the n of
 * the paper (from j to i); the printed "+ (...) x n" belongs to the opposite
 * orientation of n.
 * reading (history, Eq. tandispn): both velocity-Verlet evaluations use
 * delta^n; the update delta^{n+1} = |delta^n| t + v_t dt is committed from
 * the second evaluation, capped at mu |F_n| / k_t while sliding.
 * The torque is (-R_i n) x F. */
static void dem_contact(orc_sim *s, int i, int partner, const double n[3], double overlap,
                        const double vij[3], const double wsumR[3], const double coef[4],
                        int commit)
{
    const orc_params *P = &s->P;
    double kn = coef[0], kt = coef[1], cn = coef[2], ct = coef[3];
    double vn_s = dot(vij, n);
    double Fn[3];
    for (int a = 0; a < 3; ++a) Fn[a] = -kn * overlap * n[a] - cn * vn_s * n[a];
    double wxn[3];
    cross(wsumR, n, wxn);
    double vt[3];
    for (int a = 0; a < 3; ++a) vt[a] = vij[a] - vn_s * n[a] - wxn[a];
    double dlt[3];
    hist_find(s, i, partner, dlt);
    double vtm = sqrt(dot(vt, vt));
    double dm = sqrt(dot(dlt, dlt));
    double t[3] = { 0, 0, 0 };
    if (vtm > 0.0) {
        for (int a = 0; a < 3; ++a) t[a] = vt[a] / vtm;
    } else if (dm > 0.0) {
        for (int a = 0; a < 3; ++a) t[a] = dlt[a] / dm;
    }
    double Ft[3];
    for (int a = 0; a < 3; ++a) Ft[a] = -kt * dlt[a] - ct * vt[a];
    double Fnm = sqrt(dot(Fn, Fn));
    double Ftm = sqrt(dot(Ft, Ft));
    if (Ftm >= P->mu_fric * Fnm) {
        for (int a = 0; a < 3; ++a) Ft[a] = -P->mu_fric * Fnm * t[a];
    }
    double F[3], lev[3], tq[3];
    for (int a = 0; a < 3; ++a) {
        F[a] = Fn[a] + Ft[a];
        lev[a] = -s->R[i] * n[a];
    }
    cross(lev, F, tq);
    for (int a = 0; a < 3; ++a) {
        s->F_dem[3 * i + a] += F[a];
        s->N_dem[3 * i + a] += tq[a];
    }
    if (commit) {
        double dn[3];
        for (int a = 0; a < 3; ++a) dn[a] = dm * t[a] + vt[a] * P->dt;
        double dnm = sqrt(dot(dn, dn));
        double cap = (kt > 0.0) ? P->mu_fric * Fnm / kt : 0.0;
        if (dnm > cap && dnm > 0.0) {
            double sc = cap / dnm;
            for (int a = 0; a < 3; ++a) dn[a] *= sc;
        }
        hist_push(s, i, partner, dn);
    }
}

#define ORC_PLANE_BASE (-16)

/* compute_rigid (Algorithm 2): DEM between rigid particles (Section 2.2),
 * lubrication (Eq. lubri) and contact with the wall planes.
 * reading (lubrication): d = R_i + R_j; applied for 0 < gap = L - d and
 * L < h, gap floored at lub_gap_min * d; vector (v_j - v_i) as printed.
 * reading (walls): rigid particles touch the planes bounding the domain on
 * non-periodic axes, treated as a partner of infinite mass at rest. */
static void compute_rigid(orc_sim *s, int velver)
{
    const orc_params *P = &s->P;
    int commit = (velver == 2);
    if (commit)
        for (int i = 0; i < s->n; ++i) s->new_n[i] = 0;
    int nr = 0;
    int *rig = (int *)malloc((size_t)(s->n > 0 ? s->n : 1) * sizeof(int));
    for (int i = 0; i < s->n; ++i)
        if (s->type[i] == T_RIGID) rig[nr++] = i;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int ri = 0; ri < nr; ++ri) {
        const int i = rig[ri];
        if (s->only && !s->only[i]) continue;
        for (int rj = 0; rj < nr; ++rj) {
            const int j = rig[rj];
            if (j == i) continue;
            double r[3];
            double L = sqrt(pair_vec(P, s->x + 3 * i, s->x + 3 * j, r));
            double dsum = s->R[i] + s->R[j];
            double vij[3];
            for (int a = 0; a < 3; ++a) vij[a] = s->v[3 * i + a] - s->v[3 * j + a];
            if (L < dsum) {
                double n[3] = { r[0] / L, r[1] / L, r[2] / L };
                double wsumR[3];
                for (int a = 0; a < 3; ++a)
                    wsumR[a] = s->R[i] * s->w[3 * i + a] + s->R[j] * s->w[3 * j + a];
                double coef[4];
                orc_dem_coeffs(P, s->R[i], s->R[j], s->m[i], s->m[j], coef);
                dem_contact(s, i, j, n, L - dsum, vij, wsumR, coef, commit);
            } else if (L < P->r_c) {
                double gap = L - dsum;
                double gmin = P->lub_gap_min * dsum;
                if (gap < gmin) gap = gmin;
                double c = 3.0 * ORC_PI * P->eta * dsum * dsum / (8.0 * gap);
                for (int a = 0; a < 3; ++a) s->F_lub[3 * i + a] += c * (-vij[a]);
            }
        }
        for (int a = 0; a < 3; ++a) {
            if (P->periodic[a]) continue;
            for (int side = 0; side < 2; ++side) {
                double L = side == 0 ? s->x[3 * i + a] - P->origin[a]
                                     : (P->origin[a] + P->box[a]) - s->x[3 * i + a];
                if (!(L < s->R[i])) continue;
                double n[3] = { 0, 0, 0 };
                n[a] = side == 0 ? 1.0 : -1.0;
                double vij[3], wsumR[3];
                for (int b = 0; b < 3; ++b) {
                    vij[b] = s->v[3 * i + b];
                    wsumR[b] = s->R[i] * s->w[3 * i + b];
                }
                double coef[4];
                orc_dem_coeffs(P, s->R[i], 0.0, s->m[i], 0.0, coef);
                dem_contact(s, i, ORC_PLANE_BASE + 2 * a + side, n, L - s->R[i], vij, wsumR,
                            coef, commit);
            }
        }
    }
    free(rig);
    if (commit) {
        int *tn = s->hist_n; s->hist_n = s->new_n; s->new_n = tn;
        int *tp = s->hist_partner; s->hist_partner = s->new_partner; s->new_partner = tp;
        double *td = s->hist_delta; s->hist_delta = s->new_delta; s->new_delta = td;
    }
}

/* External acceleration of Eq. govern: uniform g plus, for the reverse
 * Poiseuille flow (Section 4.1), +body_amp along body_axis in the lower half
 * of the split_axis extent and -body_amp in the upper half. */
static void external_accel(const orc_params *P, const double *x, double a[3])
{
    for (int k = 0; k < 3; ++k) a[k] = P->g[k];
    if (P->body_amp != 0.0) {
        double rel = x[P->split_axis] - P->origin[P->split_axis];
        double sgn = (rel < 0.5 * P->box[P->split_axis]) ? 1.0 : -1.0;
        a[P->body_axis] += sgn * P->body_amp;
    }
}

/* compute_force (Algorithm 2) and the total force of Section 2.6. */
void orc_forces(orc_sim *s, int velver)
{
    size_t n3 = (size_t)s->n * 3;
    double *arrs[] = { s->F_sdpd, s->F_pg, s->F_dg, s->F_rxn, s->F_dem, s->F_lub, s->F_ext,
                       s->F, s->N_sdpd, s->N_dem, s->N, s->vf };
    for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); ++k) memset(arrs[k], 0, n3 * sizeof(double));
    memset(s->eps, 0, (size_t)s->n * sizeof(double));
    memset(s->Ssum, 0, (size_t)s->n * sizeof(double));
    compute_fluid(s);
    compute_fpi_action(s);
    compute_fpi_reaction(s);
    compute_rigid(s, velver);
    for (int i = 0; i < s->n; ++i) {
        if (!is_mobile(s->type[i])) continue;
        double a[3];
        external_accel(&s->P, s->x + 3 * i, a);
        for (int k = 0; k < 3; ++k) {
            s->F_ext[3 * i + k] = s->m[i] * a[k];
            s->F[3 * i + k] = s->F_sdpd[3 * i + k] + s->F_pg[3 * i + k] + s->F_dg[3 * i + k]
                            + s->F_rxn[3 * i + k] + s->F_dem[3 * i + k] + s->F_lub[3 * i + k]
                            + s->F_ext[3 * i + k];
            s->N[3 * i + k] = s->N_sdpd[3 * i + k] + s->N_dem[3 * i + k];
        }
    }
}

/* Boundary treatment after the drift (Section 2.5): periodic wrap, and on wall
 * axes the mirror reflection with reversal of the normal velocity. */
static void boundary(const orc_params *P, double *x, double *v)
{
    for (int a = 0; a < 3; ++a) {
        double lo = P->origin[a], hi = P->origin[a] + P->box[a];
        if (P->periodic[a]) {
            if (x[a] < lo) x[a] += P->box[a];
            else if (x[a] >= hi) x[a] -= P->box[a];
        } else {
            if (x[a] < lo) { x[a] = lo + (lo - x[a]); v[a] = -v[a]; }
            else if (x[a] > hi) { x[a] = hi - (x[a] - hi); v[a] = -v[a]; }
        }
    }
}

/* update(velver) (Algorithm 1; Eqs. newton1, newton2, velocity Verlet).
 * reading: velver 1 = half kick with F(x^n) then drift; velver 2 = half kick
 * with F(x^{n+1}).  Wall particles never move. */
void orc_update(orc_sim *s, int velver)
{
    const orc_params *P = &s->P;
    const double hdt = 0.5 * P->dt;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < s->n; ++i) {
        if (!is_mobile(s->type[i])) continue;
        for (int a = 0; a < 3; ++a) {
            s->v[3 * i + a] = s->v[3 * i + a] + hdt * (s->F[3 * i + a] / s->m[i]);
            s->w[3 * i + a] = s->w[3 * i + a] + hdt * (s->N[3 * i + a] / s->I[i]);
        }
        if (velver == 1) {
            for (int a = 0; a < 3; ++a) s->x[3 * i + a] = s->x[3 * i + a] + P->dt * s->v[3 * i + a];
            boundary(P, s->x + 3 * i, s->v + 3 * i);
        }
    }
}

/* Artificial viscosity by the collision method (Shakibaeinia & Jin; Section
 * 4.4, --enable_artvis).  reading: after the second kick, every pair of
 * mobile particles closer than artvis_alpha*dx that approaches
 * (v_ij . e_ij < 0) exchanges momentum as an inelastic collision with
 * restitution artvis_e; all corrections use the pre-correction velocities. */
void orc_artvis(orc_sim *s)
{
    const orc_params *P = &s->P;
    if (!P->artvis) return;
    size_t n3 = (size_t)s->n * 3;
    double *dv = (double *)calloc(n3 + 1, sizeof(double));
    double rlim = P->artvis_alpha * P->dx;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < s->n; ++i) {
        if (!is_mobile(s->type[i])) continue;
        for (int k = s->nb_off[i]; k < s->nb_off[i + 1]; ++k) {
            int j = s->nb[k];
            if (!is_mobile(s->type[j])) continue;
            double r[3];
            double rr = sqrt(pair_vec(P, s->x + 3 * i, s->x + 3 * j, r));
            if (!(rr < rlim)) continue;
            double e[3] = { r[0] / rr, r[1] / rr, r[2] / rr };
            double vij[3];
            for (int a = 0; a < 3; ++a) vij[a] = s->v[3 * i + a] - s->v[3 * j + a];
            double ve = dot(vij, e);
            if (!(ve < 0.0)) continue;
            double c = -(1.0 + P->artvis_e) * s->m[j] / (s->m[i] + s->m[j]) * ve;
            for (int a = 0; a < 3; ++a) dv[3 * i + a] += c * e[a];
        }
    }
    for (size_t k = 0; k < n3; ++k) s->v[k] += dv[k];
    free(dv);
}

/* One velocity-Verlet evaluation (the body of Algorithm 1 for one velver). */
int orc_substep(orc_sim *s, int velver)
{
    orc_neighbors(s);
    orc_density(s);
    orc_reinit(s);
    orc_filter(s);
    orc_forces(s, velver);
    orc_update(s, velver);
    if (velver == 2) orc_artvis(s);
    return s->overflow ? 1 : 0;
}

/* Algorithm 1: nsteps full steps. */
int orc_run(orc_sim *s, long long nsteps)
{
    for (long long k = 0; k < nsteps; ++k) {
        for (int velver = 1; velver <= 2; ++velver)
            if (orc_substep(s, velver)) return 1;
        s->step += 1;
    }
    return 0;
}

/* Evaluate the forces of one velver at the current state without moving
 * anything: neighbours, density, pressure, filter, compute_force. */
int orc_evaluate(orc_sim *s, int velver)
{
    orc_neighbors(s);
    orc_density(s);
    orc_reinit(s);
    orc_filter(s);
    orc_forces(s, velver);
    return s->overflow ? 1 : 0;
}

/* Reverse-Poiseuille viscometer read-out (Section 4.1, Eqs. poiseuanasol,
 * poiseuave): mean velocity along body_axis of the fluid particles binned by
 * their split_axis coordinate, and the apparent viscosity from the mean speed
 * of the two counter-flowing halves,  mu = rho0 a D^2 / (12 V), D = half box. */
void orc_profile(const orc_sim *s, int nbins, double *profile, double *mu_app)
{
    const orc_params *P = &s->P;
    double *cnt = (double *)calloc((size_t)nbins, sizeof(double));
    for (int b = 0; b < nbins; ++b) profile[b] = 0.0;
    double vsum[2] = { 0, 0 }, ncnt[2] = { 0, 0 };
    int ax = P->split_axis, fa = P->body_axis;
    for (int i = 0; i < s->n; ++i) {
        if (s->type[i] != T_FLUID) continue;
        double rel = s->x[3 * i + ax] - P->origin[ax];
        int b = (int)floor(rel / P->box[ax] * nbins);
        if (b < 0) b = 0;
        if (b >= nbins) b = nbins - 1;
        profile[b] += s->v[3 * i + fa];
        cnt[b] += 1.0;
        int half = (rel < 0.5 * P->box[ax]) ? 0 : 1;
        vsum[half] += (half == 0 ? 1.0 : -1.0) * s->v[3 * i + fa];
        ncnt[half] += 1.0;
    }
    for (int b = 0; b < nbins; ++b) profile[b] = cnt[b] > 0 ? profile[b] / cnt[b] : 0.0;
    double V = 0.5 * (vsum[0] / (ncnt[0] > 0 ? ncnt[0] : 1) + vsum[1] / (ncnt[1] > 0 ? ncnt[1] : 1));
    double D = 0.5 * P->box[ax];
    *mu_app = P->rho0 * P->body_amp * D * D / (12.0 * V);
    free(cnt);
}

int orc_overflow(const orc_sim *s) { return s->overflow; }
int orc_n_neighbors(const orc_sim *s, int i) { return s->nb_off[i + 1] - s->nb_off[i]; }

/* Threads of the per-particle loops (OpenMP, when the oracle was built with
 * it): every particle owns its sums and its list, so the results do not
 * depend on the count.  n <= 0 leaves it unchanged; returns the count in
 * use (1 without OpenMP). */
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
