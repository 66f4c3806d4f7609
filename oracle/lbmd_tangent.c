/*
 * lbmd_tangent.c -- forward-mode derivative (tangent) of the FP64 oracle's
 * coupled LB/MD step, for the mean particle drag along x.
 *
 * TEST INFRASTRUCTURE, like lbmd_oracle.c: it checks the GPU library's
 * hand-written adjoint and is used by nothing else.
 *
 * The state of lbmd_oracle.c (populations, node moments, pending transfers,
 * particle positions and velocities) is carried as dual numbers (value,
 * derivative along one direction of the inputs: the friction coefficient
 * zeta of Eq. (4) and the initial particle positions).  Every step below is
 * the oracle's algorithm (Sec. 2 collision and streaming, Sec. 3 MD step,
 * Eqs. (4)-(8)) written once more, operation for operation in the same order,
 * with each arithmetic operation replaced by its dual counterpart: the value
 * parts therefore equal the oracle's results bit for bit, and the derivative
 * parts are the exact derivative of the computed map.  Random numbers are the
 * oracle's (same Philox counters): they are constants of the map, and only
 * the noise amplitudes depend on the inputs (sqrt(rho) in the fluid,
 * sqrt(zeta) on the particles).
 *
 * The floor() of the trilinear interpolation (Eq. (5)) has derivative zero;
 * the map is piecewise smooth, with kinks where a particle crosses a cell
 * face.
 *
 * Observable: S = sum over MD steps and particles of the coupling force
 * F_x (Eq. (4)); its mean over steps and particles is the drag the particles
 * feel along x.  Ideal particles of mass 1, no bonds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "lbmd_oracle.h"

#define Q 19

typedef struct {
    double v, d;
} dual;

static dual mk(double v, double d) {
    dual r;
    r.v = v;
    r.d = d;
    return r;
}
static dual cst(double v) { return mk(v, 0.0); }
static dual add(dual a, dual b) { return mk(a.v + b.v, a.d + b.d); }
static dual sub(dual a, dual b) { return mk(a.v - b.v, a.d - b.d); }
static dual mul(dual a, dual b) { return mk(a.v * b.v, a.d * b.v + a.v * b.d); }
static dual scl(double c, dual a) { return mk(c * a.v, c * a.d); }
static dual divd(dual a, dual b) {
    double q = a.v / b.v;
    return mk(q, (a.d - q * b.d) / b.v);
}
static dual divc(dual a, double c) { return mk(a.v / c, a.d / c); }
static dual sqrtd(dual a) {
    double s = sqrt(a.v);
    return mk(s, s > 0.0 ? 0.5 * a.d / s : 0.0);
}

struct tan_state {
    orc_params p;
    int64_t n;
    int32_t c[Q * 3];
    double w[Q], e[Q * Q], b[Q], gam[Q];
    dual *f, *f_tmp, *rho, *jst, *jacc;
    int64_t np;
    dual *pos, *vel;
    dual zeta;
    dual drag; /* S and its derivative */
    uint64_t lb_step, md_step;
};

typedef struct tan_state tan_state;

static int64_t wrap_i(int64_t x, int64_t L) {
    x %= L;
    return x < 0 ? x + L : x;
}

static int64_t node_at(const tan_state *t, int64_t x, int64_t y, int64_t z) {
    return wrap_i(x, t->p.nx) + (int64_t)t->p.nx * (wrap_i(y, t->p.ny) + (int64_t)t->p.ny * wrap_i(z, t->p.nz));
}

/* Eqs. (1), (2) at every node, in the oracle's summation order. */
static void moments(tan_state *t) {
    for (int64_t r = 0; r < t->n; ++r) {
        dual rho = cst(0.0), jx = cst(0.0), jy = cst(0.0), jz = cst(0.0);
        for (int i = 0; i < Q; ++i) {
            dual fi = t->f[i * t->n + r];
            rho = add(rho, fi);
            jx = add(jx, scl((double)t->c[3 * i + 0], fi));
            jy = add(jy, scl((double)t->c[3 * i + 1], fi));
            jz = add(jz, scl((double)t->c[3 * i + 2], fi));
        }
        t->rho[r] = rho;
        t->jst[3 * r + 0] = jx;
        t->jst[3 * r + 1] = jy;
        t->jst[3 * r + 2] = jz;
    }
}

tan_state *tan_create(const orc_params *p) {
    /* the tangent follows integrator 0 only */
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->n_sub < 1 || (p->variant != 0 && p->variant != 1) ||
        p->integrator != 0)
        return NULL;
    tan_state *t = (tan_state *)calloc(1, sizeof(tan_state));
    if (!t) return NULL;
    t->p = *p;
    t->n = (int64_t)p->nx * p->ny * p->nz;
    orc_d3q19(t->c, t->w);
    orc_modes(t->e, t->b);
    /* relaxation factors as in the oracle (Sec. 2) */
    double gs = (6.0 * p->nu - 1.0) / (6.0 * p->nu + 1.0);
    double gb = p->nu_bulk < 0.0 ? 0.0 : (9.0 * p->nu_bulk - 1.0) / (9.0 * p->nu_bulk + 1.0);
    for (int k = 0; k < Q; ++k) t->gam[k] = 0.0;
    t->gam[4] = gb;
    for (int k = 5; k <= 9; ++k) t->gam[k] = gs;
    for (int k = 10; k < Q; ++k) t->gam[k] = p->gamma_ghost;
    int64_t n = t->n;
    t->f = (dual *)calloc(Q * n, sizeof(dual));
    t->f_tmp = (dual *)calloc(Q * n, sizeof(dual));
    t->rho = (dual *)calloc(n, sizeof(dual));
    t->jst = (dual *)calloc(3 * n, sizeof(dual));
    t->jacc = (dual *)calloc(3 * n, sizeof(dual));
    if (!t->f || !t->f_tmp || !t->rho || !t->jst || !t->jacc) {
        free(t->f); free(t->f_tmp); free(t->rho); free(t->jst); free(t->jacc); free(t);
        return NULL;
    }
    for (int i = 0; i < Q; ++i)
        for (int64_t r = 0; r < n; ++r) t->f[i * n + r] = cst(t->w[i] * p->rho0);
    moments(t);
    t->zeta = cst(p->zeta);
    return t;
}

void tan_destroy(tan_state *t) {
    if (!t) return;
    free(t->f); free(t->f_tmp); free(t->rho); free(t->jst); free(t->jacc); free(t->pos); free(t->vel);
    free(t);
}

/* Particles of mass 1; dpos: derivative of the initial positions (3n, or
 * NULL for zero); dzeta: derivative of zeta.  Clears the accumulated drag. */
int tan_set_particles(tan_state *t, int64_t np, const double *pos, const double *vel, const double *dpos,
                      double dzeta) {
    free(t->pos);
    free(t->vel);
    t->pos = (dual *)calloc(3 * (np > 0 ? np : 1), sizeof(dual));
    t->vel = (dual *)calloc(3 * (np > 0 ? np : 1), sizeof(dual));
    if (!t->pos || !t->vel) return ORC_ERR_OOM;
    t->np = np;
    double L[3] = {t->p.nx, t->p.ny, t->p.nz};
    for (int64_t q = 0; q < 3 * np; ++q) {
        double x = pos[q], Lq = L[q % 3];
        x -= Lq * floor(x / Lq); /* the oracle's wrap of an added position */
        if (x >= Lq) x -= Lq;
        t->pos[q] = mk(x, dpos ? dpos[q] : 0.0);
        t->vel[q] = cst(vel[q]);
    }
    t->zeta = mk(t->p.zeta, dzeta);
    t->drag = cst(0.0);
    return ORC_OK;
}

/* Sec. 2 collision (MRT, noise, forcing) at one node, in dual numbers. */
static void collide(const tan_state *t, const dual f[Q], const dual F[3], uint32_t node, uint32_t step,
                    dual fout[Q]) {
    dual rho = cst(0.0), j[3] = {cst(0.0), cst(0.0), cst(0.0)};
    for (int i = 0; i < Q; ++i) {
        rho = add(rho, f[i]);
        for (int a = 0; a < 3; ++a) j[a] = add(j[a], scl((double)t->c[3 * i + a], f[i]));
    }
    dual u[3];
    for (int a = 0; a < 3; ++a) u[a] = divd(add(j[a], scl(0.5, F[a])), rho);
    dual uu = add(add(mul(u[0], u[0]), mul(u[1], u[1])), mul(u[2], u[2]));
    dual uF = add(add(mul(u[0], F[0]), mul(u[1], F[1])), mul(u[2], F[2]));
    dual m[Q];
    for (int k = 0; k < Q; ++k) {
        m[k] = cst(0.0);
        for (int i = 0; i < Q; ++i) m[k] = add(m[k], scl(t->e[k * Q + i], f[i]));
    }
    dual meq[Q];
    for (int k = 0; k < Q; ++k) meq[k] = cst(0.0);
    meq[4] = mul(rho, uu);
    meq[5] = mul(rho, sub(mul(scl(3.0, u[0]), u[0]), uu));
    meq[6] = mul(rho, sub(mul(u[1], u[1]), mul(u[2], u[2])));
    meq[7] = mul(mul(rho, u[0]), u[1]);
    meq[8] = mul(mul(rho, u[0]), u[2]);
    meq[9] = mul(mul(rho, u[1]), u[2]);
    dual mp[Q];
    mp[0] = rho;
    for (int a = 0; a < 3; ++a) mp[1 + a] = add(j[a], F[a]);
    for (int k = 4; k < Q; ++k) mp[k] = add(meq[k], scl(t->gam[k], sub(m[k], meq[k])));
    double gb = t->gam[4], gs = t->gam[5];
    mp[4] = add(mp[4], scl(1.0 + gb, uF));
    mp[5] = add(mp[5], scl(1.0 + gs, sub(mul(scl(3.0, u[0]), F[0]), uF)));
    mp[6] = add(mp[6], scl(1.0 + gs, sub(mul(u[1], F[1]), mul(u[2], F[2]))));
    mp[7] = add(mp[7], scl((1.0 + gs) * 0.5, add(mul(u[0], F[1]), mul(u[1], F[0]))));
    mp[8] = add(mp[8], scl((1.0 + gs) * 0.5, add(mul(u[0], F[2]), mul(u[2], F[0]))));
    mp[9] = add(mp[9], scl((1.0 + gs) * 0.5, add(mul(u[1], F[2]), mul(u[2], F[1]))));
    if (t->p.kT > 0.0) {
        uint32_t key[2] = {(uint32_t)(t->p.seed & 0xffffffffu), (uint32_t)(t->p.seed >> 32)}, ctr[4], out[4];
        double xi[16];
        for (uint32_t q = 0; q < 2; ++q) {
            ctr[0] = node; ctr[1] = step; ctr[2] = 0u; ctr[3] = q;
            orc_philox4x32_10(ctr, key, out);
            for (int s = 0; s < 4; ++s) {
                xi[8 * q + 2 * s] = orc_uniform_unit16(out[s] & 0xffffu);
                xi[8 * q + 2 * s + 1] = orc_uniform_unit16(out[s] >> 16);
            }
        }
        double mu = 3.0 * t->p.kT;
        for (int k = 4; k < Q; ++k) {
            dual var = scl(1.0 - t->gam[k] * t->gam[k], scl(t->b[k], scl(mu, rho)));
            mp[k] = add(mp[k], scl(xi[k - 4], sqrtd(var)));
        }
    }
    for (int i = 0; i < Q; ++i) {
        dual acc = cst(0.0);
        for (int k = 0; k < Q; ++k) acc = add(acc, divc(scl(t->e[k * Q + i], mp[k]), t->b[k]));
        fout[i] = scl(t->w[i], acc);
    }
}

/* One LB step, Eq. (3): collide with F = J_acc + g, stream, new moments. */
int tan_lb_step(tan_state *t) {
    int64_t n = t->n;
    for (int64_t z = 0; z < t->p.nz; ++z)
        for (int64_t y = 0; y < t->p.ny; ++y)
            for (int64_t x = 0; x < t->p.nx; ++x) {
                int64_t r = node_at(t, x, y, z);
                dual fin[Q], fo[Q], F[3];
                for (int i = 0; i < Q; ++i) fin[i] = t->f[i * n + r];
                for (int a = 0; a < 3; ++a) F[a] = add(t->jacc[3 * r + a], cst(t->p.body_force[a]));
                collide(t, fin, F, (uint32_t)r, (uint32_t)t->lb_step, fo);
                for (int i = 0; i < Q; ++i)
                    t->f_tmp[i * n + node_at(t, x + t->c[3 * i], y + t->c[3 * i + 1], z + t->c[3 * i + 2])] = fo[i];
            }
    dual *tmp = t->f;
    t->f = t->f_tmp;
    t->f_tmp = tmp;
    moments(t);
    memset(t->jacc, 0, sizeof(dual) * 3 * n);
    t->lb_step += 1;
    return ORC_OK;
}

/* One MD step (Sec. 3, Eqs. (4)-(8)) for every particle, and the drag sum. */
int tan_md_substep(tan_state *t) {
    int64_t np = t->np;
    double dt = 1.0 / (double)t->p.n_sub;
    double L[3] = {t->p.nx, t->p.ny, t->p.nz};
    if (np > 0) {
        int64_t *corner = (int64_t *)malloc(sizeof(int64_t) * 8 * np);
        dual *delta = (dual *)malloc(sizeof(dual) * 8 * np);
        dual *dP = (dual *)malloc(sizeof(dual) * 3 * np);
        dual *fc = (dual *)malloc(sizeof(dual) * 3 * np);
        if (!corner || !delta || !dP || !fc) {
            free(corner); free(delta); free(dP); free(fc);
            return ORC_ERR_OOM;
        }
        uint32_t key[2] = {(uint32_t)(t->p.seed & 0xffffffffu), (uint32_t)(t->p.seed >> 32)};
        dual amp = sqrtd(divc(scl(t->p.kT, scl(2.0, t->zeta)), dt));
        for (int64_t p = 0; p < np; ++p) {
            /* trilinear corners and weights of Eq. (5) */
            dual d[3];
            double base[3];
            for (int a = 0; a < 3; ++a) {
                base[a] = floor(t->pos[3 * p + a].v);
                d[a] = sub(t->pos[3 * p + a], cst(base[a]));
            }
            for (int k = 0; k < 8; ++k) {
                int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
                dual wk = cst(1.0);
                for (int a = 0; a < 3; ++a) wk = mul(wk, o[a] ? d[a] : sub(cst(1.0), d[a]));
                delta[8 * p + k] = wk;
                corner[8 * p + k] =
                    node_at(t, (int64_t)base[0] + o[0], (int64_t)base[1] + o[1], (int64_t)base[2] + o[2]);
            }
            dual uR[3] = {cst(0.0), cst(0.0), cst(0.0)};
            for (int k = 0; k < 8; ++k) {
                int64_t r = corner[8 * p + k];
                for (int a = 0; a < 3; ++a) {
                    dual jn = t->jst[3 * r + a];
                    if (t->p.variant == 1) jn = add(jn, t->jacc[3 * r + a]);
                    uR[a] = add(uR[a], divd(mul(delta[8 * p + k], jn), t->rho[r]));
                }
            }
            uint32_t ctr[4] = {(uint32_t)p, (uint32_t)t->md_step, 1u, 0u}, out[4];
            orc_philox4x32_10(ctr, key, out);
            for (int a = 0; a < 3; ++a) {
                dual frand = t->p.kT > 0.0 ? scl(orc_uniform_unit(out[a]), amp) : cst(0.0);
                dual f = add(mul(scl(-1.0, t->zeta), sub(t->vel[3 * p + a], uR[a])), frand);
                fc[3 * p + a] = f;
                dP[3 * p + a] = scl(dt, f);
            }
            t->drag = add(t->drag, fc[3 * p + 0]);
        }
        /* velocity Verlet with the coupling force held over the step (mass 1) */
        double hm = 0.5 * dt / 1.0;
        for (int64_t p = 0; p < np; ++p)
            for (int a = 0; a < 3; ++a) {
                t->vel[3 * p + a] = add(t->vel[3 * p + a], scl(hm, add(cst(0.0), fc[3 * p + a])));
                dual x = add(t->pos[3 * p + a], scl(dt, t->vel[3 * p + a]));
                double xv = x.v - L[a] * floor(x.v / L[a]); /* periodic wrap: derivative 1 */
                if (xv >= L[a]) xv -= L[a];
                t->pos[3 * p + a] = mk(xv, x.d);
            }
        for (int64_t p = 0; p < np; ++p)
            for (int a = 0; a < 3; ++a)
                t->vel[3 * p + a] = add(t->vel[3 * p + a], scl(hm, add(cst(0.0), fc[3 * p + a])));
        /* Eqs. (7), (8): transfers in particle id order */
        for (int64_t p = 0; p < np; ++p)
            for (int k = 0; k < 8; ++k)
                for (int a = 0; a < 3; ++a) {
                    int64_t r = corner[8 * p + k];
                    t->jacc[3 * r + a] = sub(t->jacc[3 * r + a], mul(delta[8 * p + k], dP[3 * p + a]));
                }
        free(corner); free(delta); free(dP); free(fc);
    }
    t->md_step += 1;
    return ORC_OK;
}

/* out[0] = S, out[1] = dS (sum of F_x over steps and particles). */
void tan_drag(const tan_state *t, double out[2]) {
    out[0] = t->drag.v;
    out[1] = t->drag.d;
}

/* Values and derivatives of the state (for the tests): populations 19 n,
 * positions and velocities 3 np each. */
void tan_get_populations(const tan_state *t, double *val, double *der) {
    for (int64_t q = 0; q < Q * t->n; ++q) {
        val[q] = t->f[q].v;
        der[q] = t->f[q].d;
    }
}

void tan_get_particles(const tan_state *t, double *pos, double *vel, double *dpos, double *dvel) {
    for (int64_t q = 0; q < 3 * t->np; ++q) {
        pos[q] = t->pos[q].v;
        vel[q] = t->vel[q].v;
        dpos[q] = t->pos[q].d;
        dvel[q] = t->vel[q].d;
    }
}
