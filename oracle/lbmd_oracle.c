/*
 * lbmd_oracle.c -- plain FP64 CPU oracle for the fluctuating D3Q19 lattice
 * Boltzmann fluid with dissipative point-particle coupling, variants A, B and C,
 * of Tretyakov & Duenweg, "An improved dissipative coupling scheme for a
 * system of Molecular Dynamics particles interacting with a Lattice Boltzmann
 * fluid" (arXiv:1610.02733).
 *
 * TEST INFRASTRUCTURE.  This file is the correctness authority for the GPU
 * library and nothing else: only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header, table or
 * helper with the CUDA path.  It is deliberately slow and written to be read
 * against the paper: one node or one particle at a time, in index order, every
 * quantity in double precision.
 *
 * Units: lattice units throughout, a = 1 and tau_LB = 1, so the MD step is
 * dt = 1/m with m = tau_LB/dt the integer time-scale ratio (Sec. 3).
 *
 * Where the paper defers to its references (the MRT collision operator, the
 * stochastic collision operator and the forcing term Delta'_i), the standard
 * moment-space formulation of the fluctuating lattice Boltzmann method is
 * used: orthogonal 19-mode basis, relaxation factors per mode group, noise of
 * variance mu rho b_k (1 - gamma_k^2) on the non-conserved modes, and Guo's
 * forcing in moment space (the functions below say which at each place).
 *
 * Parity pins (tests/test_oracle_*.py) tie each function below to something
 * other than itself; none of them is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "lbmd_oracle.h"

#define Q 19

/* ------------------------------------------------------------------------ */
/* D3Q19 velocity set, Sec. 2 and Fig. 1(a): the rest vector, the 6 nearest  */
/* and the 12 next-nearest neighbours of a simple cubic lattice.             */
/* ------------------------------------------------------------------------ */
static const int C[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

/* Lattice weights: 1/3 for the rest vector, 1/18 for |c|^2 = 1, 1/36 for
 * |c|^2 = 2; they give the isotropy c_s^2 = 1/3. */
static double weight(int i) {
    int c2 = C[i][0] * C[i][0] + C[i][1] * C[i][1] + C[i][2] * C[i][2];
    if (c2 == 0) return 1.0 / 3.0;
    if (c2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* Mode basis e_k(c) of the MRT collision operator (Sec. 2).  Row 0 gives the
 * mass density of Eq. (1), rows 1-3 the momentum density of Eq. (2); rows 4-9
 * span the stress (4 = trace/bulk, 5-9 = traceless shear); rows 10-18 are the
 * kinetic "ghost" modes.  The rows are orthogonal with respect to the lattice
 * weights. */
static double mode_value(int k, int cx, int cy, int cz) {
    double x = cx, y = cy, z = cz;
    double c2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return c2 - 1.0;
    case 5: return 3.0 * x * x - c2;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return x * z;
    case 9: return y * z;
    case 10: return (3.0 * c2 - 5.0) * x;
    case 11: return (3.0 * c2 - 5.0) * y;
    case 12: return (3.0 * c2 - 5.0) * z;
    case 13: return (y * y - z * z) * x;
    case 14: return (z * z - x * x) * y;
    case 15: return (x * x - y * y) * z;
    case 16: return 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
    case 17: return (2.0 * c2 - 3.0) * (3.0 * x * x - c2);
    case 18: return (2.0 * c2 - 3.0) * (y * y - z * z);
    }
    return 0.0;
}

struct orc_state {
    orc_params p;
    int64_t n_nodes;
    double w[Q];
    double e[Q][Q]; /* e[k][i] = e_k(c_i) */
    double b[Q];    /* b_k = sum_i w_i e_k(c_i)^2 */
    double gam[Q];  /* relaxation factor per mode; 0-3 unused (conserved) */
    double *f;      /* post-stream populations f*_i, [i][z][y][x] */
    double *f_tmp;  /* streaming target */
    double *rho;    /* rho* of f*, per node */
    double *jst;    /* j* of f*, 3 per node */
    double *jacc;   /* momentum density handed over since the last LB step */
    int64_t np, cap_p;
    double *pos, *vel, *mass, *fcons, *fc;
    int64_t nb, cap_b;
    int64_t *bond;
    double *bond_k, *bond_r0;
    int *bond_kind;       /* ORC_BOND_HARMONIC or ORC_BOND_FENE per bond */
    double lj_eps, lj_sigma, lj_rc; /* Lennard-Jones between all particles; off when lj_rc = 0 */
    int fcons_valid;
    uint64_t lb_step, md_step;
    int sub_done;
};

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11, */
/* "Parallel random numbers: as easy as 1, 2, 3").  Not from the paper: it   */
/* is the common source of every random number in both the oracle and the   */
/* GPU path, so that the two see the same noise.                             */
/* ------------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
    uint64_t prod = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(prod >> 32);
    *lo = (uint32_t)prod;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(M0, x0, &hi0, &lo0);
        mulhilo32(M1, x2, &hi1, &lo1);
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 32 random bits -> zero-mean, unit-variance uniform number:
 * u = (x + 1/2) 2^-32 in (0,1), xi = sqrt(12) (u - 1/2).  Used for the
 * random force on the particles. */
double orc_uniform_unit(uint32_t x) {
    double u = ((double)x + 0.5) * (1.0 / 4294967296.0);
    return sqrt(12.0) * (u - 0.5);
}

/* 16 random bits -> zero-mean, unit-variance uniform number on 65536 levels:
 * u = (h + 1/2) 2^-16, xi = sqrt(12) (u - 1/2).  The fluid noise takes two
 * such variates from each 32-bit Philox word (low half first). */
double orc_uniform_unit16(uint32_t h) {
    double u = ((double)(h & 0xffffu) + 0.5) * (1.0 / 65536.0);
    return sqrt(12.0) * (u - 0.5);
}

/* Two 32-bit Philox words -> two independent standard normal variates by the
 * Box-Muller transform (Box & Muller, Ann. Math. Stat. 29 (1958) 610): the
 * top 24 bits of each word give u = (h + 1/2) 2^-24 in (0, 1), and with
 * r = sqrt(-2 ln u1) the pair is (r cos 2 pi u2, r sin 2 pi u2).  Used for
 * every noise term when the Gaussian option is selected. */
void orc_box_muller(uint32_t w1, uint32_t w2, double out[2]) {
    const double two_pi = 6.283185307179586476925286766559;
    double u1 = ((double)(w1 >> 8) + 0.5) * (1.0 / 16777216.0);
    double u2 = ((double)(w2 >> 8) + 0.5) * (1.0 / 16777216.0);
    double r = sqrt(-2.0 * log(u1));
    out[0] = r * cos(two_pi * u2);
    out[1] = r * sin(two_pi * u2);
}

static void key_of(const orc_state *s, uint32_t key[2]) {
    key[0] = (uint32_t)(s->p.seed & 0xffffffffu);
    key[1] = (uint32_t)(s->p.seed >> 32);
}

/* ------------------------------------------------------------------------ */
/* Set-up                                                                    */
/* ------------------------------------------------------------------------ */
void orc_d3q19(int32_t c_out[Q * 3], double w_out[Q]) {
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) c_out[3 * i + a] = C[i][a];
        w_out[i] = weight(i);
    }
}

void orc_modes(double e_out[Q * Q], double b_out[Q]) {
    for (int k = 0; k < Q; ++k) {
        double bk = 0.0;
        for (int i = 0; i < Q; ++i) {
            double ek = mode_value(k, C[i][0], C[i][1], C[i][2]);
            e_out[k * Q + i] = ek;
            bk += weight(i) * ek * ek;
        }
        b_out[k] = bk;
    }
}

static void compute_moments(orc_state *s) {
    /* every node on its own (a timing build may spread the loop over threads) */
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < s->n_nodes; ++r) {
        double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
        for (int i = 0; i < Q; ++i) {
            double fi = s->f[i * s->n_nodes + r];
            rho += fi;
            jx += fi * C[i][0];
            jy += fi * C[i][1];
            jz += fi * C[i][2];
        }
        s->rho[r] = rho;
        s->jst[3 * r + 0] = jx;
        s->jst[3 * r + 1] = jy;
        s->jst[3 * r + 2] = jz;
    }
}

orc_state *orc_create(const orc_params *p) {
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->n_sub < 1) return NULL;
    if (p->variant < 0 || p->variant > 2) return NULL;
    if (p->integrator != 0 && p->integrator != 1) return NULL;
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->p = *p;
    s->n_nodes = (int64_t)p->nx * p->ny * p->nz;
    for (int i = 0; i < Q; ++i) s->w[i] = weight(i);
    for (int k = 0; k < Q; ++k) {
        double bk = 0.0;
        for (int i = 0; i < Q; ++i) {
            s->e[k][i] = mode_value(k, C[i][0], C[i][1], C[i][2]);
            bk += s->w[i] * s->e[k][i] * s->e[k][i];
        }
        s->b[k] = bk;
    }
    /* Relaxation factors (Sec. 2): the shear rate sets the viscosity,
     * nu = (1 + g_s) / (6 (1 - g_s)); the bulk rate sets
     * nu_b = (1 + g_b) / (9 (1 - g_b)); ghost modes relax with gamma_ghost. */
    double gs = (6.0 * p->nu - 1.0) / (6.0 * p->nu + 1.0);
    double gb = p->nu_bulk < 0.0 ? 0.0 : (9.0 * p->nu_bulk - 1.0) / (9.0 * p->nu_bulk + 1.0);
    for (int k = 0; k < Q; ++k) s->gam[k] = 0.0;
    s->gam[4] = gb;
    for (int k = 5; k <= 9; ++k) s->gam[k] = gs;
    for (int k = 10; k < Q; ++k) s->gam[k] = p->gamma_ghost;

    int64_t n = s->n_nodes;
    s->f = (double *)malloc(sizeof(double) * Q * n);
    s->f_tmp = (double *)malloc(sizeof(double) * Q * n);
    s->rho = (double *)malloc(sizeof(double) * n);
    s->jst = (double *)malloc(sizeof(double) * 3 * n);
    s->jacc = (double *)calloc(3 * n, sizeof(double));
    if (!s->f || !s->f_tmp || !s->rho || !s->jst || !s->jacc) {
        orc_destroy(s);
        return NULL;
    }
    /* Fluid initially at rest with density rho0: f_i = w_i rho0. */
    for (int i = 0; i < Q; ++i)
        for (int64_t r = 0; r < n; ++r) s->f[i * n + r] = s->w[i] * p->rho0;
    compute_moments(s);
    return s;
}

void orc_destroy(orc_state *s) {
    if (!s) return;
    free(s->f); free(s->f_tmp); free(s->rho); free(s->jst); free(s->jacc);
    free(s->pos); free(s->vel); free(s->mass); free(s->fcons); free(s->fc);
    free(s->bond); free(s->bond_k); free(s->bond_r0); free(s->bond_kind);
    free(s);
}

/* ------------------------------------------------------------------------ */
/* LB collision at one node: Sec. 2 (MRT relaxation in moment space, thermal */
/* noise of the stochastic collision operator) plus the forcing term         */
/* Delta'_i of Sec. 3 for the force density F.  Returns post-collision f'.   */
/* ------------------------------------------------------------------------ */
void orc_collide_node(const orc_state *s, const double f[Q], const double F[3],
                      uint32_t node, uint32_t lb_step, double fout[Q]) {
    /* Hydrodynamic moments, Eqs. (1) and (2). */
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += f[i] * C[i][a];
    }
    /* Streaming velocity entering the equilibrium and Delta'_i: half of the
     * force density's momentum is counted (second-order forcing). */
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];

    double m[Q];
    for (int k = 0; k < Q; ++k) {
        m[k] = 0.0;
        for (int i = 0; i < Q; ++i) m[k] += s->e[k][i] * f[i];
    }
    /* Equilibrium values of the stress modes; ghost equilibria vanish. */
    double meq[Q];
    for (int k = 0; k < Q; ++k) meq[k] = 0.0;
    meq[4] = rho * uu;
    meq[5] = rho * (3.0 * u[0] * u[0] - uu);
    meq[6] = rho * (u[1] * u[1] - u[2] * u[2]);
    meq[7] = rho * u[0] * u[1];
    meq[8] = rho * u[0] * u[2];
    meq[9] = rho * u[1] * u[2];

    double mp[Q];
    /* Mass is conserved; momentum changes by exactly F * tau_LB. */
    mp[0] = rho;
    for (int a = 0; a < 3; ++a) mp[1 + a] = j[a] + F[a];
    /* MRT relaxation of every non-conserved mode. */
    for (int k = 4; k < Q; ++k) mp[k] = meq[k] + s->gam[k] * (m[k] - meq[k]);
    /* Forcing term Delta'_i in moment space: linear in F, depends on u. */
    double gb = s->gam[4], gs = s->gam[5];
    mp[4] += (1.0 + gb) * uF;
    mp[5] += (1.0 + gs) * (3.0 * u[0] * F[0] - uF);
    mp[6] += (1.0 + gs) * (u[1] * F[1] - u[2] * F[2]);
    mp[7] += (1.0 + gs) * 0.5 * (u[0] * F[1] + u[1] * F[0]);
    mp[8] += (1.0 + gs) * 0.5 * (u[0] * F[2] + u[2] * F[0]);
    mp[9] += (1.0 + gs) * 0.5 * (u[1] * F[2] + u[2] * F[1]);
    /* Thermal noise: mode k gets variance mu rho b_k (1 - gamma_k^2) with
     * mu = kT / (a^3 c_s^2) = 3 kT, which keeps its equilibrium variance
     * mu rho b_k stationary (fluctuation-dissipation in the fluid). */
    if (s->p.kT > 0.0) {
        uint32_t key[2], ctr[4], out[4];
        double xi[16];
        key_of(s, key);
        if (s->p.noise == 1) {
            /* normal variates: four Philox calls, two Box-Muller pairs each */
            for (uint32_t q = 0; q < 4; ++q) {
                ctr[0] = node; ctr[1] = lb_step; ctr[2] = 0u; ctr[3] = q;
                orc_philox4x32_10(ctr, key, out);
                orc_box_muller(out[0], out[1], xi + 4 * q);
                orc_box_muller(out[2], out[3], xi + 4 * q + 2);
            }
        } else {
            for (uint32_t q = 0; q < 2; ++q) {
                ctr[0] = node; ctr[1] = lb_step; ctr[2] = 0u; ctr[3] = q;
                orc_philox4x32_10(ctr, key, out);
                for (int t = 0; t < 4; ++t) {
                    xi[8 * q + 2 * t] = orc_uniform_unit16(out[t] & 0xffffu);
                    xi[8 * q + 2 * t + 1] = orc_uniform_unit16(out[t] >> 16);
                }
            }
        }
        double mu = 3.0 * s->p.kT;
        for (int k = 4; k < Q; ++k)
            mp[k] += sqrt(mu * rho * s->b[k] * (1.0 - s->gam[k] * s->gam[k])) * xi[k - 4];
    }
    /* Back to populations: f'_i = w_i sum_k e_k(c_i) m'_k / b_k. */
    for (int i = 0; i < Q; ++i) {
        double acc = 0.0;
        for (int k = 0; k < Q; ++k) acc += s->e[k][i] * mp[k] / s->b[k];
        fout[i] = s->w[i] * acc;
    }
}

static int64_t wrap(int64_t x, int64_t L) {
    x %= L;
    return x < 0 ? x + L : x;
}

static int64_t node_index(const orc_state *s, int64_t x, int64_t y, int64_t z) {
    return wrap(x, s->p.nx) + (int64_t)s->p.nx * (wrap(y, s->p.ny) + (int64_t)s->p.ny * wrap(z, s->p.nz));
}

/* Full LB update, Eq. (3): collide every node with the force density
 * F = J_acc / tau_LB + g (the total momentum handed over by the particles
 * since the last LB step, Sec. 3, plus a uniform body force), then stream
 * f'_i(r) to r + c_i.  Afterwards J_acc restarts from zero. */
int orc_lb_step(orc_state *s) {
    if (s->sub_done != s->p.n_sub) return ORC_ERR_SEQUENCE;
    int64_t n = s->n_nodes;
    /* every node collides on its own and pushes to distinct targets (a timing
     * build may spread the planes over threads; the results do not change) */
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < s->p.nz; ++z)
        for (int64_t y = 0; y < s->p.ny; ++y)
            for (int64_t x = 0; x < s->p.nx; ++x) {
                int64_t r = node_index(s, x, y, z);
                double fin[Q], fout[Q], F[3];
                for (int i = 0; i < Q; ++i) fin[i] = s->f[i * n + r];
                for (int a = 0; a < 3; ++a) F[a] = s->jacc[3 * r + a] + s->p.body_force[a];
                orc_collide_node(s, fin, F, (uint32_t)r, (uint32_t)s->lb_step, fout);
                for (int i = 0; i < Q; ++i) {
                    int64_t t = node_index(s, x + C[i][0], y + C[i][1], z + C[i][2]);
                    s->f_tmp[i * n + t] = fout[i];
                }
            }
    double *tmp = s->f; s->f = s->f_tmp; s->f_tmp = tmp;
    compute_moments(s);
    memset(s->jacc, 0, sizeof(double) * 3 * n);
    s->lb_step += 1;
    s->sub_done = 0;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Particles                                                                 */
/* ------------------------------------------------------------------------ */
static double wrap_pos(double x, double L) {
    x -= L * floor(x / L);
    if (x >= L) x -= L; /* a tiny negative x can round up to exactly L */
    return x;
}

/* Trilinear weights of Eq. (5): the eight lattice sites r_k at the corners of
 * the unit cube that contains R; corner k = ox + 2 oy + 4 oz has weight
 * delta_k = prod_a (o_a ? d_a : 1 - d_a), d = R - floor(R). */
void orc_trilinear(const orc_state *s, const double R[3], int64_t corner[8], double delta[8]) {
    double base[3], d[3];
    for (int a = 0; a < 3; ++a) {
        base[a] = floor(R[a]);
        d[a] = R[a] - base[a];
    }
    for (int k = 0; k < 8; ++k) {
        int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
        double wk = 1.0;
        for (int a = 0; a < 3; ++a) wk *= o[a] ? d[a] : 1.0 - d[a];
        delta[k] = wk;
        corner[k] = node_index(s, (int64_t)base[0] + o[0], (int64_t)base[1] + o[1], (int64_t)base[2] + o[2]);
    }
}

/* Momentum density at node r as seen by the particles.  Variant A: the value
 * of the last LB update (Sec. 3, "variant A").  Variant B: that value plus
 * every transfer made since, so the node velocities follow each MD step.
 * Variant C: the momentum of the populations, which every MD step updates
 * (orc_forcing_update). */
static void node_momentum_seen(const orc_state *s, int64_t r, double jout[3]) {
    for (int a = 0; a < 3; ++a) {
        jout[a] = s->jst[3 * r + a];
        if (s->p.variant == 1) jout[a] += s->jacc[3 * r + a];
    }
}

/* Minimum-image separation d = R_j - R_i and its length squared. */
static double separation(const orc_state *s, int64_t i, int64_t j, double d[3]) {
    double L[3] = {s->p.nx, s->p.ny, s->p.nz}, r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        d[a] = s->pos[3 * j + a] - s->pos[3 * i + a];
        d[a] -= L[a] * round(d[a] / L[a]);
        r2 += d[a] * d[a];
    }
    return r2;
}

/* Bond b of length r: magnitude g with force g d on the first particle and
 * -g d on the second (d from the first to the second), and the energy.
 *   harmonic  U = (k/2)(r - r0)^2,                 g = k (r - r0) / r
 *   FENE      U = -(k/2) R0^2 ln(1 - (r/R0)^2),     g = k / (1 - (r/R0)^2)
 * (the finitely extensible springs of the Kremer-Grest chains, Sec. 4; R0 is
 * stored in bond_r0).  A FENE bond stretched to r >= R0 has infinite energy:
 * NaN force. */
static double bond_force(const orc_state *s, int64_t b, double r2, double *energy) {
    double k = s->bond_k[b], r0 = s->bond_r0[b];
    if (s->bond_kind[b] == ORC_BOND_FENE) {
        double x = r2 / (r0 * r0);
        if (!(x < 1.0)) {
            if (energy) *energy = INFINITY;
            return NAN;
        }
        if (energy) *energy = -0.5 * k * r0 * r0 * log(1.0 - x);
        return k / (1.0 - x);
    }
    double r = sqrt(r2);
    if (energy) *energy = 0.5 * k * (r - r0) * (r - r0);
    if (r == 0.0) return 0.0;
    return k * (r - r0) / r;
}

/* Lennard-Jones pair at distance^2 r2 < rc^2 (Sec. 4: the Kremer-Grest
 * monomers, cut off at rc): U = 4 eps ((sigma/r)^12 - (sigma/r)^6) - U_c with
 * the shift U_c making U(rc) = 0; magnitude g with force g d on the first
 * particle (d from the first to the second), g = -24 eps (2 t^2 - t) / r^2,
 * t = (sigma/r)^6. */
static double lj_force(const orc_state *s, double r2, double *energy) {
    double t = pow(s->lj_sigma * s->lj_sigma / r2, 3.0);
    if (energy) {
        double tc = pow(s->lj_sigma * s->lj_sigma / (s->lj_rc * s->lj_rc), 3.0);
        *energy = 4.0 * s->lj_eps * (t * t - t) - 4.0 * s->lj_eps * (tc * tc - tc);
    }
    return -24.0 * s->lj_eps * (2.0 * t * t - t) / r2;
}

/* Conservative force F^cons of Eq. (4) on every particle at the current
 * positions: bonds (harmonic or FENE) in bond order, then Lennard-Jones over
 * every pair i < j within the cut-off (bonded pairs included: all monomers
 * interact, Sec. 4).  Each pair's force is added to both particles with
 * opposite signs, so the total is zero up to rounding.  energy (if not NULL)
 * receives the harmonic, FENE and LJ potential energies. */
static void compute_conservative_forces(orc_state *s, double energy[3]) {
    for (int64_t q = 0; q < 3 * s->np; ++q) s->fcons[q] = 0.0;
    if (energy) energy[0] = energy[1] = energy[2] = 0.0;
    for (int64_t b = 0; b < s->nb; ++b) {
        int64_t i = s->bond[2 * b], j = s->bond[2 * b + 1];
        double d[3], u;
        double g = bond_force(s, b, separation(s, i, j, d), &u);
        for (int a = 0; a < 3; ++a) {
            s->fcons[3 * i + a] += g * d[a];
            s->fcons[3 * j + a] -= g * d[a];
        }
        if (energy) energy[s->bond_kind[b] == ORC_BOND_FENE ? 1 : 0] += u;
    }
    if (s->lj_rc > 0.0) {
        double rc2 = s->lj_rc * s->lj_rc;
        for (int64_t i = 0; i < s->np; ++i)
            for (int64_t j = i + 1; j < s->np; ++j) {
                double d[3], u;
                double r2 = separation(s, i, j, d);
                if (!(r2 < rc2)) continue;
                double g = lj_force(s, r2, &u);
                for (int a = 0; a < 3; ++a) {
                    s->fcons[3 * i + a] += g * d[a];
                    s->fcons[3 * j + a] -= g * d[a];
                }
                if (energy) energy[2] += u;
            }
    }
    s->fcons_valid = 1;
}

/* Variant C (Sec. 4): after every MD step the populations themselves take
 * the momentum transfer F = J_acc of that step through the forcing part
 * Delta'_i of the collision operator alone -- no relaxation, no noise, no
 * streaming.  In moment space (the forcing of orc_collide_node): mass
 * unchanged, momentum + F, stress modes + (1 + gamma) times the symmetric
 * products of u and F with the local streaming velocity u = (j + F/2)/rho of
 * the current populations, ghost modes unchanged.  The node moments are then
 * recomputed from the populations and J_acc restarts from zero. */
static void orc_forcing_update(orc_state *s) {
    int64_t n = s->n_nodes;
    double gb = s->gam[4], gs = s->gam[5];
    for (int64_t r = 0; r < n; ++r) {
        const double *F = s->jacc + 3 * r;
        if (F[0] == 0.0 && F[1] == 0.0 && F[2] == 0.0) continue;
        double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            double fi = s->f[i * n + r];
            rho += fi;
            for (int a = 0; a < 3; ++a) j[a] += fi * C[i][a];
        }
        double u[3];
        for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;
        double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
        double dm[Q];
        for (int k = 0; k < Q; ++k) dm[k] = 0.0;
        for (int a = 0; a < 3; ++a) dm[1 + a] = F[a];
        dm[4] = (1.0 + gb) * uF;
        dm[5] = (1.0 + gs) * (3.0 * u[0] * F[0] - uF);
        dm[6] = (1.0 + gs) * (u[1] * F[1] - u[2] * F[2]);
        dm[7] = (1.0 + gs) * 0.5 * (u[0] * F[1] + u[1] * F[0]);
        dm[8] = (1.0 + gs) * 0.5 * (u[0] * F[2] + u[2] * F[0]);
        dm[9] = (1.0 + gs) * 0.5 * (u[1] * F[2] + u[2] * F[1]);
        for (int i = 0; i < Q; ++i) {
            double acc = 0.0;
            for (int k = 0; k < Q; ++k) acc += s->e[k][i] * dm[k] / s->b[k];
            s->f[i * n + r] += s->w[i] * acc;
        }
    }
    compute_moments(s);
    memset(s->jacc, 0, sizeof(double) * 3 * n);
}

/* Coupling force of Eq. (4) on every particle at its current position and
 * velocity: the node velocities as they stand (Eq. (5)), the random force of
 * MD step md_step; fills s->fc and the interpolation corners and weights.
 * Every particle reads the nodes before any transfer of the step is made. */
static void coupling_forces(orc_state *s, double dt, int64_t *corner, double *delta) {
    uint32_t key[2];
    key_of(s, key);
    double amp = sqrt(2.0 * s->p.zeta * s->p.kT / dt);
    for (int64_t p = 0; p < s->np; ++p) {
        int64_t *ck = corner + 8 * p;
        double *dk = delta + 8 * p;
        orc_trilinear(s, s->pos + 3 * p, ck, dk);
        double uR[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 8; ++k) {
            double jn[3];
            node_momentum_seen(s, ck[k], jn);
            for (int a = 0; a < 3; ++a) uR[a] += dk[k] * jn[a] / s->rho[ck[k]];
        }
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)s->md_step, 1u, 0u}, out[4];
        orc_philox4x32_10(ctr, key, out);
        double xi[4];
        if (s->p.noise == 1) {
            orc_box_muller(out[0], out[1], xi);
            orc_box_muller(out[2], out[3], xi + 2);
        } else {
            for (int a = 0; a < 3; ++a) xi[a] = orc_uniform_unit(out[a]);
        }
        for (int a = 0; a < 3; ++a) {
            double frand = s->p.kT > 0.0 ? amp * xi[a] : 0.0;
            s->fc[3 * p + a] = -s->p.zeta * (s->vel[3 * p + a] - uR[a]) + frand;
        }
    }
}

/* One MD step of length dt = tau_LB / m for every particle (Sec. 3).
 * integrator 0 (the reading of Eq. (6): R, v and F_rand of the beginning of
 * the step):
 *   1. noise, then friction with the node velocities as they stand
 *      (Eqs. (4), (5)) at R, v of the start of the step: F_c, and
 *      Delta P = dt F_c (Eq. (6));
 *   2. velocity Verlet with F_c held fixed over the step (half kick, drift,
 *      conservative forces at the new positions, half kick);
 *   3. Newton's third law: node r_k around the start position receives
 *      Delta j_k = -delta_k Delta P / a^3 (Eqs. (7), (8)).
 * integrator 1 (velocity Verlet with the forces evaluated where an MD code
 * evaluates them, after the drift):
 *   1. half kick with the previous step's F_c and F_cons, drift;
 *   2. F_cons at the new positions; F_c from the half-step velocity and the
 *      node velocities interpolated at the new position;
 *   3. half kick with F_c + F_cons;
 *   4. transfer -delta_k dt F_c around the new position.
 *   The particle takes dt F_c in two halves (this step and the next), the
 *   fluid in full now: fluid + particle momentum + dt/2 sum F_c is conserved.
 * In both, every particle reads the nodes before any transfer of this step
 * is added. */
int orc_md_substep(orc_state *s) {
    if (s->sub_done >= s->p.n_sub) return ORC_ERR_SEQUENCE;
    int64_t np = s->np;
    double dt = 1.0 / (double)s->p.n_sub;
    if (np > 0) {
        if (!s->fcons_valid) compute_conservative_forces(s, NULL);
        int64_t *corner = (int64_t *)malloc(sizeof(int64_t) * 8 * np);
        double *delta = (double *)malloc(sizeof(double) * 8 * np);
        if (!corner || !delta) {
            free(corner); free(delta);
            return ORC_ERR_OOM;
        }
        double L[3] = {s->p.nx, s->p.ny, s->p.nz};
        if (s->p.integrator == 0) {
            coupling_forces(s, dt, corner, delta);
            for (int64_t p = 0; p < np; ++p) {
                double hm = 0.5 * dt / s->mass[p];
                for (int a = 0; a < 3; ++a) {
                    s->vel[3 * p + a] += hm * (s->fcons[3 * p + a] + s->fc[3 * p + a]);
                    s->pos[3 * p + a] = wrap_pos(s->pos[3 * p + a] + dt * s->vel[3 * p + a], L[a]);
                }
            }
            compute_conservative_forces(s, NULL);
        } else {
            for (int64_t p = 0; p < np; ++p) {
                double hm = 0.5 * dt / s->mass[p];
                for (int a = 0; a < 3; ++a) {
                    s->vel[3 * p + a] += hm * (s->fcons[3 * p + a] + s->fc[3 * p + a]);
                    s->pos[3 * p + a] = wrap_pos(s->pos[3 * p + a] + dt * s->vel[3 * p + a], L[a]);
                }
            }
            compute_conservative_forces(s, NULL);
            coupling_forces(s, dt, corner, delta);
        }
        for (int64_t p = 0; p < np; ++p) {
            double hm = 0.5 * dt / s->mass[p];
            for (int a = 0; a < 3; ++a) s->vel[3 * p + a] += hm * (s->fcons[3 * p + a] + s->fc[3 * p + a]);
        }
        /* Momentum handed to the fluid, particle by particle in id order. */
        for (int64_t p = 0; p < np; ++p)
            for (int k = 0; k < 8; ++k)
                for (int a = 0; a < 3; ++a)
                    s->jacc[3 * corner[8 * p + k] + a] -= delta[8 * p + k] * (dt * s->fc[3 * p + a]);
        free(corner); free(delta);
    }
    if (s->p.variant == 2) orc_forcing_update(s);
    s->md_step += 1;
    s->sub_done += 1;
    return ORC_OK;
}

int orc_add_particles(orc_state *s, int64_t n, const double *pos, const double *vel, const double *mass) {
    if (n < 0) return ORC_ERR_ARG;
    int64_t need = s->np + n;
    if (need > s->cap_p) {
        int64_t cap = need > 2 * s->cap_p ? need : 2 * s->cap_p;
        double **arrs[5] = {&s->pos, &s->vel, &s->mass, &s->fcons, &s->fc};
        int width[5] = {3, 3, 1, 3, 3};
        for (int t = 0; t < 5; ++t) {
            double *na = (double *)realloc(*arrs[t], sizeof(double) * width[t] * (cap > 0 ? cap : 1));
            if (!na) return ORC_ERR_OOM;
            *arrs[t] = na;
        }
        s->cap_p = cap;
    }
    double L[3] = {s->p.nx, s->p.ny, s->p.nz};
    for (int64_t q = 0; q < n; ++q) {
        int64_t p = s->np + q;
        for (int a = 0; a < 3; ++a) {
            s->pos[3 * p + a] = wrap_pos(pos[3 * q + a], L[a]);
            s->vel[3 * p + a] = vel[3 * q + a];
            s->fcons[3 * p + a] = 0.0;
            s->fc[3 * p + a] = 0.0;
        }
        s->mass[p] = mass ? mass[q] : 1.0;
    }
    s->np = need;
    s->fcons_valid = 0;
    return ORC_OK;
}

static int add_bonds_of_kind(orc_state *s, int64_t nb, const int64_t *pairs, double k, double r0, int kind) {
    if (nb < 0) return ORC_ERR_ARG;
    for (int64_t q = 0; q < 2 * nb; ++q)
        if (pairs[q] < 0 || pairs[q] >= s->np) return ORC_ERR_ARG;
    int64_t need = s->nb + nb;
    if (need > s->cap_b) {
        int64_t cap = need > 2 * s->cap_b ? need : 2 * s->cap_b;
        int64_t *nbnd = (int64_t *)realloc(s->bond, sizeof(int64_t) * 2 * cap);
        if (!nbnd) return ORC_ERR_OOM;
        s->bond = nbnd;
        double *nk = (double *)realloc(s->bond_k, sizeof(double) * cap);
        if (!nk) return ORC_ERR_OOM;
        s->bond_k = nk;
        double *nr = (double *)realloc(s->bond_r0, sizeof(double) * cap);
        if (!nr) return ORC_ERR_OOM;
        s->bond_r0 = nr;
        int *nkind = (int *)realloc(s->bond_kind, sizeof(int) * cap);
        if (!nkind) return ORC_ERR_OOM;
        s->bond_kind = nkind;
        s->cap_b = cap;
    }
    for (int64_t q = 0; q < nb; ++q) {
        s->bond[2 * (s->nb + q)] = pairs[2 * q];
        s->bond[2 * (s->nb + q) + 1] = pairs[2 * q + 1];
        s->bond_k[s->nb + q] = k;
        s->bond_r0[s->nb + q] = r0;
        s->bond_kind[s->nb + q] = kind;
    }
    s->nb = need;
    s->fcons_valid = 0;
    return ORC_OK;
}

int orc_add_bonds(orc_state *s, int64_t nb, const int64_t *pairs, double k, double r0) {
    return add_bonds_of_kind(s, nb, pairs, k, r0, ORC_BOND_HARMONIC);
}

int orc_add_fene_bonds(orc_state *s, int64_t nb, const int64_t *pairs, double k, double R0) {
    if (!(R0 > 0.0)) return ORC_ERR_ARG;
    return add_bonds_of_kind(s, nb, pairs, k, R0, ORC_BOND_FENE);
}

int orc_set_lj(orc_state *s, double eps, double sigma, double rc) {
    if (!(eps >= 0.0) || !(sigma > 0.0) || !(rc >= 0.0)) return ORC_ERR_ARG;
    s->lj_eps = eps;
    s->lj_sigma = sigma;
    s->lj_rc = rc;
    s->fcons_valid = 0;
    return ORC_OK;
}

/* Conservative forces (3 np) at the current positions and the potential
 * energies [harmonic, FENE, LJ]. */
void orc_conservative_forces(orc_state *s, double *forces, double energy[3]) {
    compute_conservative_forces(s, energy);
    if (forces) memcpy(forces, s->fcons, sizeof(double) * 3 * s->np);
}

/* ------------------------------------------------------------------------ */
/* Observables and accessors                                                 */
/* ------------------------------------------------------------------------ */
/* out: [0] total mass, [1..3] fluid momentum incl. the pending transfer
 * J_acc, [4..6] particle momentum, [7] particle kinetic temperature
 * (sum m v^2)/(3 N), [8] particle kinetic energy, [9] lb_step, [10] md_step. */
void orc_observables(const orc_state *s, double out[11]) {
    double mass = 0.0, pf[3] = {0.0, 0.0, 0.0}, pp[3] = {0.0, 0.0, 0.0}, mv2 = 0.0;
    for (int64_t r = 0; r < s->n_nodes; ++r) {
        mass += s->rho[r];
        for (int a = 0; a < 3; ++a) pf[a] += s->jst[3 * r + a] + s->jacc[3 * r + a];
    }
    for (int64_t p = 0; p < s->np; ++p)
        for (int a = 0; a < 3; ++a) {
            pp[a] += s->mass[p] * s->vel[3 * p + a];
            mv2 += s->mass[p] * s->vel[3 * p + a] * s->vel[3 * p + a];
        }
    out[0] = mass;
    for (int a = 0; a < 3; ++a) { out[1 + a] = pf[a]; out[4 + a] = pp[a]; }
    out[7] = s->np > 0 ? mv2 / (3.0 * (double)s->np) : 0.0;
    out[8] = 0.5 * mv2;
    out[9] = (double)s->lb_step;
    out[10] = (double)s->md_step;
}

void orc_get_populations(const orc_state *s, double *out) {
    memcpy(out, s->f, sizeof(double) * Q * s->n_nodes);
}

void orc_set_populations(orc_state *s, const double *in) {
    memcpy(s->f, in, sizeof(double) * Q * s->n_nodes);
    compute_moments(s);
}

void orc_get_jacc(const orc_state *s, double *out) { memcpy(out, s->jacc, sizeof(double) * 3 * s->n_nodes); }

void orc_set_jacc(orc_state *s, const double *in) { memcpy(s->jacc, in, sizeof(double) * 3 * s->n_nodes); }

/* (rho*, j seen by the particles) per node: 4 values per node. */
void orc_get_node_field(const orc_state *s, double *out) {
    for (int64_t r = 0; r < s->n_nodes; ++r) {
        double jn[3];
        node_momentum_seen(s, r, jn);
        out[4 * r] = s->rho[r];
        for (int a = 0; a < 3; ++a) out[4 * r + 1 + a] = jn[a];
    }
}

void orc_get_particles(const orc_state *s, double *pos, double *vel) {
    if (pos) memcpy(pos, s->pos, sizeof(double) * 3 * s->np);
    if (vel) memcpy(vel, s->vel, sizeof(double) * 3 * s->np);
}

void orc_set_particles(orc_state *s, const double *pos, const double *vel) {
    double L[3] = {s->p.nx, s->p.ny, s->p.nz};
    for (int64_t p = 0; p < s->np; ++p)
        for (int a = 0; a < 3; ++a) {
            if (pos) s->pos[3 * p + a] = wrap_pos(pos[3 * p + a], L[a]);
            if (vel) s->vel[3 * p + a] = vel[3 * p + a];
        }
    if (pos) s->fcons_valid = 0;
}

/* Coupling force F_c of each particle's last MD step, 3 per particle. */
void orc_get_coupling_forces(const orc_state *s, double *out) { memcpy(out, s->fc, sizeof(double) * 3 * s->np); }

void orc_counters(const orc_state *s, int64_t out[3]) {
    out[0] = (int64_t)s->lb_step;
    out[1] = (int64_t)s->md_step;
    out[2] = s->sub_done;
}

void orc_set_counters(orc_state *s, int64_t lb_step, int64_t md_step) {
    s->lb_step = (uint64_t)lb_step;
    s->md_step = (uint64_t)md_step;
}

int64_t orc_num_particles(const orc_state *s) { return s->np; }

/* ------------------------------------------------------------------------ */
/* Reduced-precision population storage (an extension of the method, not in */
/* the paper): the stored deviation of a population from its rest value is  */
/* rounded onto a binary floating-point grid with p significand bits and    */
/* minimum normal exponent emin (FP16: p = 11, emin = -14; BF16: p = 8,     */
/* emin = -126), written out from the definition of such a grid.  Finite    */
/* range assumed (the deviations are far below the largest finite value).   */
/* ------------------------------------------------------------------------ */

/* x rounded onto the grid: to nearest, ties to the even neighbour
 * (stochastic = 0), or stochastically with 16 random bits r (stochastic = 1):
 * away from zero when r < 2^16 frac, frac = the distance of |x| above the
 * grid value below it in units of the grid step there. */
double orc_round_storage(double x, int p, int emin, uint32_t r, int stochastic) {
    if (x == 0.0) return x;
    double a = fabs(x);
    int e;
    frexp(a, &e); /* a = m 2^e, 1/2 <= m < 1: the leading bit has exponent e - 1 */
    int E = e - 1 < emin ? emin : e - 1;
    double step = ldexp(1.0, E - (p - 1)); /* spacing of the grid around a */
    double q = a / step;                   /* exact: step is a power of two */
    double lo = floor(q), frac = q - lo;
    int up;
    if (stochastic)
        up = (double)(r & 0xffffu) < frac * 65536.0;
    else
        up = frac > 0.5 || (frac == 0.5 && fmod(lo, 2.0) == 1.0);
    double y = (lo + (double)up) * step;
    return x < 0.0 ? -y : y;
}

/* The 16 random bits of population i of node `node`'s post-collision state
 * in LB step `lb_step`: Philox4x32-10 under the seed, counter (node, lb_step,
 * 2, i / 8), word (i / 2) mod 4, low half for even i. */
void orc_sr_bits(uint64_t seed, uint32_t node, uint32_t lb_step, uint32_t out[Q]) {
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t ctr[4], w[4];
    for (int i = 0; i < Q; ++i) {
        if (i % 8 == 0) {
            ctr[0] = node; ctr[1] = lb_step; ctr[2] = 2u; ctr[3] = (uint32_t)(i / 8);
            orc_philox4x32_10(ctr, key, w);
        }
        uint32_t word = w[(i / 2) % 4];
        out[i] = (i % 2 == 0) ? (word & 0xffffu) : (word >> 16);
    }
}

/* Vector forms for the tests. */
void orc_round_storage_n(int64_t n, const double *x, int p, int emin, const uint32_t *r, int stochastic,
                         double *out) {
    for (int64_t k = 0; k < n; ++k) out[k] = orc_round_storage(x[k], p, emin, r ? r[k] : 0u, stochastic);
}
void orc_sr_bits_n(uint64_t seed, int64_t n, const uint32_t *nodes, uint32_t lb_step, uint32_t *out) {
    for (int64_t k = 0; k < n; ++k) orc_sr_bits(seed, nodes[k], lb_step, out + Q * k);
}
