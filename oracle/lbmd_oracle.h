/*
 * lbmd_oracle.h -- interface of the FP64 CPU oracle (test infrastructure).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * use this interface.  The GPU library has its own header (include/lbmd.h)
 * and shares nothing with this one.
 */
#ifndef LBMD_ORACLE_H
#define LBMD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_OOM = -3, ORC_ERR_SEQUENCE = -4 };
enum { ORC_BOND_HARMONIC = 0, ORC_BOND_FENE = 1 };

typedef struct orc_params {
    int32_t nx, ny, nz;   /* periodic lattice, nodes per axis, a = 1 */
    int32_t n_sub;        /* m = tau_LB / dt, MD steps per LB step */
    int32_t variant;      /* 0 = variant A, 1 = variant B (Sec. 3), 2 = variant C (Sec. 4) */
    int32_t integrator;   /* 0: coupling force from R, v at the start of the MD step (Eq. (6)),
                             held over both half-kicks; 1: from the half-step velocity after the
                             drift, at the new position (see orc_md_substep) */
    double rho0;          /* initial fluid density */
    double nu;            /* kinematic shear viscosity */
    double nu_bulk;       /* bulk viscosity; < 0 selects gamma_bulk = 0 */
    double gamma_ghost;   /* relaxation factor of the ghost modes */
    double kT;            /* temperature; 0 switches every noise term off */
    double zeta;          /* particle friction coefficient of Eq. (4) */
    double body_force[3]; /* uniform force density on the fluid */
    uint64_t seed;        /* Philox key */
    int32_t noise;        /* 0: uniform variates sqrt(12) (u - 1/2); 1: normal variates (Box-Muller) */
} orc_params;

typedef struct orc_state orc_state;

orc_state *orc_create(const orc_params *p);
void orc_destroy(orc_state *s);

int orc_add_particles(orc_state *s, int64_t n, const double *pos, const double *vel, const double *mass);
int orc_add_bonds(orc_state *s, int64_t nb, const int64_t *pairs, double k, double r0);
int orc_add_fene_bonds(orc_state *s, int64_t nb, const int64_t *pairs, double k, double R0);
int orc_set_lj(orc_state *s, double eps, double sigma, double rc);
void orc_conservative_forces(orc_state *s, double *forces, double energy[3]);
int orc_md_substep(orc_state *s);
int orc_lb_step(orc_state *s);
void orc_observables(const orc_state *s, double out[11]);

void orc_get_populations(const orc_state *s, double *out);
void orc_set_populations(orc_state *s, const double *in);
void orc_get_jacc(const orc_state *s, double *out);
void orc_set_jacc(orc_state *s, const double *in);
void orc_get_node_field(const orc_state *s, double *out);
void orc_get_particles(const orc_state *s, double *pos, double *vel);
void orc_set_particles(orc_state *s, const double *pos, const double *vel);
void orc_get_coupling_forces(const orc_state *s, double *out);
void orc_counters(const orc_state *s, int64_t out[3]);
void orc_set_counters(orc_state *s, int64_t lb_step, int64_t md_step);
int64_t orc_num_particles(const orc_state *s);

/* Building blocks, exposed so the tests can pin each one on its own. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform_unit(uint32_t x);
double orc_uniform_unit16(uint32_t h);
void orc_box_muller(uint32_t w1, uint32_t w2, double out[2]);
void orc_d3q19(int32_t c_out[19 * 3], double w_out[19]);
void orc_modes(double e_out[19 * 19], double b_out[19]);
void orc_collide_node(const orc_state *s, const double f[19], const double F[3], uint32_t node, uint32_t lb_step,
                      double fout[19]);
void orc_trilinear(const orc_state *s, const double R[3], int64_t corner[8], double delta[8]);

/* Reduced-precision storage of the populations (not part of the paper's
 * method): rounding onto a binary grid (p significand bits, minimum normal
 * exponent emin) to nearest or stochastically with 16 random bits, and the
 * random bits of each population of a node's post-collision state. */
double orc_round_storage(double x, int p, int emin, uint32_t r, int stochastic);
void orc_sr_bits(uint64_t seed, uint32_t node, uint32_t lb_step, uint32_t out[19]);
void orc_round_storage_n(int64_t n, const double *x, int p, int emin, const uint32_t *r, int stochastic,
                         double *out);
void orc_sr_bits_n(uint64_t seed, int64_t n, const uint32_t *nodes, uint32_t lb_step, uint32_t *out);

/* Forward-mode derivative (tangent) of the oracle's step for the mean
 * particle drag along x, ideal particles of mass 1 (lbmd_tangent.c). */
typedef struct tan_state tan_state;
tan_state *tan_create(const orc_params *p);
void tan_destroy(tan_state *t);
int tan_set_particles(tan_state *t, int64_t np, const double *pos, const double *vel, const double *dpos,
                      double dzeta);
int tan_md_substep(tan_state *t);
int tan_lb_step(tan_state *t);
void tan_drag(const tan_state *t, double out[2]);
void tan_get_populations(const tan_state *t, double *val, double *der);
void tan_get_particles(const tan_state *t, double *pos, double *vel, double *dpos, double *dvel);

#ifdef __cplusplus
}
#endif
#endif
