/*
 * FP64 CPU oracle for the plane-strain lattice Boltzmann method of
 * arXiv:2301.00228 (Schlueter, Yan, Faust, Mueller & Mueller).
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow reference for the CUDA library.
 * It is loaded by the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark, and by nothing else.  It shares no code with the CUDA path.
 *
 * Every time step runs the blocks of the algorithm summary (Fig. 3) in the
 * paper's order, one full-lattice pass per block, no fusion:
 *   1. moments phi, psi of both population sets           Eq. interpretation
 *   2. acceleration at interior points                     Eq. navier
 *   3. acceleration at Neumann / Dirichlet points          Eq. acc_neumann,
 *                                                          Eq. acc_dirichlet
 *   4. explicit Newmark integration of u                   Eq. integration
 *   5. boundary phi, psi from finite differences of the
 *      new u, boundary populations reset                   Eq. psi_phi_at_bound,
 *                                                          Eq. correction-f
 *   6. LBE into interior points, with the time-averaged
 *      state for boundary sources                          Eq. LBE, Eq. LBE_mod
 *   7. every l-th step, synchronisation                    Sec. 3.2
 *
 * Readings where the paper is silent, garbled or inconsistent:
 *   R1  c_s = sqrt(mu/rho) (the text after Eq. wave-navier prints lambda;
 *       Sec. 4 states c_s/c_d = 1/sqrt(3), true for mu only at lambda = mu).
 *   R2  Fig. 3 initialises phi with the curl; phi is the divergence,
 *       Eq. phi-psi.
 *   R3  The interior acceleration is c_d^2 grad(phi) - c_s^2 curl(psi e_z)
 *       (Eq. navier); Fig. 3 drops the curl.
 *   R4  Finite differences are central where both neighbours exist (or wrap
 *       periodically) and one-sided three-point (second order) otherwise;
 *       the paper only states "second order accurate" (Sec. 3.1.2).
 *   R5  The segment length l_kr that Sec. 3.1.1 defines multiplies each
 *       stress term in Eq. acc_neumann (the printed sum omits it).
 *   R6  Rectangle cells: the square of side dh around a boundary point
 *       clipped to the body; faces towards each existing neighbour.
 *   R7  J(x_k, t) in Eq. correction-f is the first moment of the populations
 *       stored at x_k at time t.  Boundary points receive no LBE output, so
 *       their populations are only ever set by Eq. correction-f.
 *   R8  Eq. LBE_mod: with bc_feq_mode 0 the equilibrium is evaluated from the
 *       moments of the averaged state f-hat; with mode 1 from f(x_k, t) as
 *       printed.
 *   R9  With du/dt(x,0) given, the first moments start at J_phi = -v and
 *       J_psi = (-v_y, v_x), from d(phi)/dt = -div J_phi (the zeroth-moment
 *       balance of the LBE) and d(phi)/dt = div v.  All inputs at rest give
 *       J = 0.  (A discrete travelling plane wave started this way stays a
 *       pure travelling wave; the tests pin it so.)
 *   R10 tau = dt/2 in both Eq. LBE and Eq. LBE_mod (so dt/tau = 1/tau = 2).
 *   R11 The Newmark update is used as printed: beta = 0 and gamma = 0 (the
 *       velocity takes the acceleration at t only).  It is first order, and
 *       modes whose acceleration feeds back on u (boundary points) grow by
 *       about 1 + (omega dt)^2 / 4 per step, which is why small a_phi (the
 *       paper's a_{0,phi} = 0.9999, Sec. 4) is needed for stability.
 *   R12 Boundary data may vary in time as u*(t) = s_D(t) u*, F(t) = s_N(t) F
 *       with a ramp-then-hold factor s(t) = min(t, t_hold) / t_ramp (s = 1
 *       without a schedule; Sec. 4 ramps the traction of its tension and
 *       shear examples this way).  R13 says at which times they are taken.
 *   R14 General geometry (Sec. 3 preprocessing, not detailed in the paper):
 *       points are interior (0), Neumann (1), Dirichlet (2) or void (3, not
 *       in the body).  A body point with a neighbour outside the body (void,
 *       or past a non-periodic edge) is a boundary point.  Its cell is the
 *       square of side dh around it clipped to the body, given as data: the
 *       area V_C and the length in the body of each side (E, N, W, S).  A
 *       side facing a body neighbour r is shared with r's cell and carries
 *       (sigma_k + sigma_r)/2; a side facing no body neighbour that still
 *       lies partly in the body carries sigma_k (so a uniform stress is in
 *       equilibrium); the rest of the cell boundary is dC_ext, whose force F
 *       is supplied per point.  Without cell data the cells of R6 are used.
 *       Differences (R4) are central where both neighbours are in the body,
 *       otherwise one-sided towards the body; a body point without such a
 *       stencil makes the geometry invalid.  A boundary point streams into
 *       every interior neighbour (Eq. LBE_mod).
 *   R13 The Neumann force enters the acceleration at t with its value at t
 *       (like the stresses, Eq. acc_neumann); the Dirichlet target is
 *       u*(t + dt), the displacement the point must have after the step
 *       (Eq. acc_dirichlet lands u(t + dt) on it).
 *   R15 Eq. correction-f takes J(x_k, t) without saying which populations it
 *       is the moment of.  bc_j_mode 0 (default, R7): those stored at x_k.
 *       bc_j_mode 1: Sec. 3.1.2 says boundary points "can only partially be
 *       updated via the LBE"; J is then the first moment of that partial
 *       update, the populations the plain LBE (Eq. LBE, from f(., t))
 *       streams into x_k from its body neighbours, with f(x_k, t) kept for
 *       the directions whose source lies outside the body.
 *   R16 Cells of the plate with a circular hole (Sec. 4): the square of
 *       side dh around a boundary point, clipped to the body rectangle,
 *       minus the disk.  Its area and side lengths are computed here by
 *       Green's theorem along the clipped boundary (ora_clip_rect); the
 *       external faces on the outer edges carry the edge traction, the hole
 *       is traction-free.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D2Q5 lattice directions e_alpha; the velocities are c^alpha = c e_alpha
 * with c = dh/dt (Sec. 3, velocity set). */
static const int EX[5] = {0, 1, 0, -1, 0};
static const int EY[5] = {0, 0, 1, 0, -1};

struct ora_lattice {
    ora_params p;
    double cd, cs, a_phi, a_psi, a0_psi, dt, c;
    uint8_t* type;        /* [ny*nx]: 0 interior, 1 Neumann, 2 Dirichlet, 3 void */
    double* bc;           /* [ny*nx*2] */
    double* cell;         /* [ny*nx*5]: V_C and side lengths E, N, W, S of boundary cells */
    double* f[2][5];      /* populations at t: set 0 = phi, set 1 = psi */
    double* fn[2][5];     /* populations at t + dt */
    double* fc[2][5];     /* post-collision populations */
    double *ux, *uy, *vx, *vy;      /* u, du/dt at t */
    double *ux1, *uy1, *vx1, *vy1;  /* u, du/dt at t + dt */
    double* s[2];         /* phi, psi at t */
    double *ax, *ay;      /* acceleration at t */
    double load_rate[2];  /* 1 / t_ramp of the Neumann [0] and Dirichlet [1] data; 0 = constant */
    double load_hold[2];  /* t_hold: the factor stays at t_hold / t_ramp from there on */
    int64_t steps;
    int initialised;
};

static int32_t g_threads = 1;

void ora_set_threads(int32_t n) { g_threads = n > 0 ? n : 1; }
int32_t ora_get_threads(void) { return g_threads; }

static long at(const ora_lattice* L, int i, int j) { return (long)j * L->p.nx + i; }

/* Weights a_0, a of one population set (Eq. feq, Eq. feq_req). */
static double w0_of(const ora_lattice* L, int set) { return set == 0 ? L->p.a0_phi : L->a0_psi; }
static double w_of(const ora_lattice* L, int set) { return set == 0 ? L->a_phi : L->a_psi; }

/* Neighbour of (i,j) in direction (di,dj); 0 if it lies outside the body
 * (past a non-periodic edge, or void). */
static int neighbour(const ora_lattice* L, int i, int j, int di, int dj, int* oi, int* oj) {
    int ni = i + di, nj = j + dj;
    if (ni < 0 || ni >= L->p.nx) {
        if (!L->p.periodic_x) return 0;
        ni = (ni + L->p.nx) % L->p.nx;
    }
    if (nj < 0 || nj >= L->p.ny) {
        if (!L->p.periodic_y) return 0;
        nj = (nj + L->p.ny) % L->p.ny;
    }
    if (L->type[at(L, ni, nj)] == 3) return 0;
    *oi = ni;
    *oj = nj;
    return 1;
}

static int is_void(const ora_lattice* L, long k) { return L->type[k] == 3; }

/* A body point is a boundary lattice point when one of its four neighbours
 * lies outside the body (reading R14). */
static int is_boundary(const ora_lattice* L, int i, int j) {
    if (is_void(L, at(L, i, j))) return 0;
    int oi, oj;
    for (int a = 1; a < 5; ++a)
        if (!neighbour(L, i, j, EX[a], EY[a], &oi, &oj)) return 1;
    return 0;
}

/* Second-order finite difference of g along (dx, dy) at (i, j) (readings R4,
 * R14): central if both neighbours are in the body, else one-sided
 * three-point towards the body.  Returns 0 and sets *ok = 0 when neither is
 * possible. */
static double fd1(const ora_lattice* L, const double* g, int i, int j, int dx, int dy, int* ok) {
    double h = L->p.dh;
    int pi, pj, mi, mj, qi, qj;
    int hp = neighbour(L, i, j, dx, dy, &pi, &pj);
    int hm = neighbour(L, i, j, -dx, -dy, &mi, &mj);
    if (ok) *ok = 1;
    if (hp && hm) return (g[at(L, pi, pj)] - g[at(L, mi, mj)]) / (2.0 * h);
    if (hp && neighbour(L, pi, pj, dx, dy, &qi, &qj))
        return (-3.0 * g[at(L, i, j)] + 4.0 * g[at(L, pi, pj)] - g[at(L, qi, qj)]) / (2.0 * h);
    if (hm && neighbour(L, mi, mj, -dx, -dy, &qi, &qj))
        return (3.0 * g[at(L, i, j)] - 4.0 * g[at(L, mi, mj)] + g[at(L, qi, qj)]) / (2.0 * h);
    if (ok) *ok = 0;
    return 0.0;
}

static double d_dx(const ora_lattice* L, const double* g, int i, int j) { return fd1(L, g, i, j, 1, 0, NULL); }
static double d_dy(const ora_lattice* L, const double* g, int i, int j) { return fd1(L, g, i, j, 0, 1, NULL); }

/* Divergence and curl of u by finite differences (Eq. phi-psi). */
static double fd_div(const ora_lattice* L, const double* ux, const double* uy, int i, int j) {
    return d_dx(L, ux, i, j) + d_dy(L, uy, i, j);
}
static double fd_curl(const ora_lattice* L, const double* ux, const double* uy, int i, int j) {
    return d_dx(L, uy, i, j) - d_dy(L, ux, i, j);
}

/* Cauchy stress by finite differences of Eq. strain inserted in Eq. hooke:
 * sig = {sigma_xx, sigma_yy, sigma_xy}. */
static void stress(const ora_lattice* L, const double* ux, const double* uy, int i, int j, double sig[3]) {
    double exx = d_dx(L, ux, i, j);
    double eyy = d_dy(L, uy, i, j);
    double exy = 0.5 * (d_dy(L, ux, i, j) + d_dx(L, uy, i, j));
    double tr = exx + eyy;
    sig[0] = L->p.lambda * tr + 2.0 * L->p.mu * exx;
    sig[1] = L->p.lambda * tr + 2.0 * L->p.mu * eyy;
    sig[2] = 2.0 * L->p.mu * exy;
}

/* Equilibrium of Eq. feq for direction alpha, given s and J = sum c^alpha f^alpha. */
static double f_eq(const ora_lattice* L, int set, int alpha, double s, double jx, double jy) {
    const double b = 1.0; /* Eq. feq_req */
    if (alpha == 0) return w0_of(L, set) * s;
    double cax = L->c * EX[alpha], cay = L->c * EY[alpha];
    return w_of(L, set) * s + b * (cax * jx + cay * jy) / (2.0 * L->c * L->c);
}

/* Zeroth and first moments of five populations (Eq. interpretation, Eq. feq). */
static void moments(const ora_lattice* L, const double g[5], double* s, double* jx, double* jy) {
    double m0 = 0.0, mx = 0.0, my = 0.0;
    for (int a = 0; a < 5; ++a) {
        m0 += g[a];
        mx += L->c * EX[a] * g[a];
        my += L->c * EY[a] * g[a];
    }
    *s = m0;
    *jx = mx;
    *jy = my;
}

static void gather(double* const fs[5], long k, double g[5]) {
    for (int a = 0; a < 5; ++a) g[a] = fs[a][k];
}

/* ---------------------------------------------------------------- create */

static double* alloc0(long n) { return (double*)calloc((size_t)n, sizeof(double)); }

ora_lattice* ora_create(const ora_params* p, const uint8_t* node_type, const double* bc_value) {
    return ora_create_cells(p, node_type, bc_value, NULL);
}

ora_lattice* ora_create_cells(const ora_params* p, const uint8_t* node_type, const double* bc_value,
                              const double* cell) {
    if (!p || p->nx < 3 || p->ny < 3) return NULL;
    if (!(p->mu > 0.0) || !(p->rho > 0.0) || !(p->lambda + 2.0 * p->mu > 0.0) || !(p->dh > 0.0)) return NULL;
    if (!(p->a0_phi >= 0.0 && p->a0_phi < 1.0)) return NULL;
    if (p->bc_feq_mode != 0 && p->bc_feq_mode != 1) return NULL;
    if (p->bc_j_mode != 0 && p->bc_j_mode != 1) return NULL;
    if (p->sync_every < 0) return NULL;
    ora_lattice* L = (ora_lattice*)calloc(1, sizeof(ora_lattice));
    if (!L) return NULL;
    L->p = *p;
    /* Wave speeds after Eq. wave-navier (reading R1). */
    L->cd = sqrt((p->lambda + 2.0 * p->mu) / p->rho);
    L->cs = sqrt(p->mu / p->rho);
    /* Eq. feq_req: a_0 + 4a = 1; Eq. conditions-parameters for a_psi, dt. */
    L->a_phi = (1.0 - p->a0_phi) / 4.0;
    L->a_psi = (L->cs * L->cs) / (L->cd * L->cd) * L->a_phi;
    L->a0_psi = 1.0 - 4.0 * L->a_psi;
    L->dt = p->dh / L->cd * sqrt(2.0 * L->a_phi);
    L->c = p->dh / L->dt;
    long n = (long)p->nx * p->ny;
    L->type = (uint8_t*)calloc((size_t)n, 1);
    L->bc = alloc0(2 * n);
    L->cell = alloc0(5 * n);
    for (int set = 0; set < 2; ++set) {
        for (int a = 0; a < 5; ++a) {
            L->f[set][a] = alloc0(n);
            L->fn[set][a] = alloc0(n);
            L->fc[set][a] = alloc0(n);
        }
        L->s[set] = alloc0(n);
    }
    L->ux = alloc0(n); L->uy = alloc0(n); L->vx = alloc0(n); L->vy = alloc0(n);
    L->ux1 = alloc0(n); L->uy1 = alloc0(n); L->vx1 = alloc0(n); L->vy1 = alloc0(n);
    L->ax = alloc0(n); L->ay = alloc0(n);
    /* Node types first (void points change who is a boundary point). */
    for (long k = 0; k < n; ++k) {
        uint8_t t = node_type ? node_type[k] : 0;
        if (t > 3) {
            ora_destroy(L);
            return NULL;
        }
        L->type[k] = t;
    }
    for (int j = 0; j < p->ny; ++j) {
        for (int i = 0; i < p->nx; ++i) {
            long k = at(L, i, j);
            uint8_t t = L->type[k];
            if (t == 3) continue;
            int bnd = is_boundary(L, i, j), okx, oky;
            fd1(L, L->ux, i, j, 1, 0, &okx);
            fd1(L, L->ux, i, j, 0, 1, &oky);
            if ((bnd && t == 0) || (!bnd && t != 0) || !okx || !oky) {
                ora_destroy(L);
                return NULL;
            }
            if (!bnd) continue;
            if (bc_value) {
                L->bc[2 * k] = bc_value[2 * k];
                L->bc[2 * k + 1] = bc_value[2 * k + 1];
            }
            double* cd = L->cell + 5 * k;
            if (t != 1) continue;  /* only Neumann points use a cell */
            if (cell) {
                for (int q = 0; q < 5; ++q) cd[q] = cell[5 * k + q];
                int okc = isfinite(cd[0]) && cd[0] > 0.0;
                for (int q = 1; q < 5; ++q) okc = okc && isfinite(cd[q]) && cd[q] >= 0.0;
                if (!okc) {
                    ora_destroy(L);
                    return NULL;
                }
            } else {
                /* Reading R6: the square of side dh clipped to the rectangle. */
                double half = 0.5 * p->dh;
                int ti, tj;
                int has_e = neighbour(L, i, j, 1, 0, &ti, &tj), has_n = neighbour(L, i, j, 0, 1, &ti, &tj);
                int has_w = neighbour(L, i, j, -1, 0, &ti, &tj), has_s = neighbour(L, i, j, 0, -1, &ti, &tj);
                double wx = (has_w ? half : 0.0) + (has_e ? half : 0.0);
                double wy = (has_s ? half : 0.0) + (has_n ? half : 0.0);
                cd[0] = wx * wy;
                cd[1] = has_e ? wy : 0.0;
                cd[2] = has_n ? wx : 0.0;
                cd[3] = has_w ? wy : 0.0;
                cd[4] = has_s ? wx : 0.0;
            }
        }
    }
    return L;
}

void ora_destroy(ora_lattice* L) {
    if (!L) return;
    free(L->type);
    free(L->bc);
    free(L->cell);
    for (int set = 0; set < 2; ++set) {
        for (int a = 0; a < 5; ++a) {
            free(L->f[set][a]);
            free(L->fn[set][a]);
            free(L->fc[set][a]);
        }
        free(L->s[set]);
    }
    free(L->ux); free(L->uy); free(L->vx); free(L->vy);
    free(L->ux1); free(L->uy1); free(L->vx1); free(L->vy1);
    free(L->ax); free(L->ay);
    free(L);
}

void ora_constants(const ora_lattice* L, double out[6]) {
    out[0] = L->cd;
    out[1] = L->cs;
    out[2] = L->a_phi;
    out[3] = L->a_psi;
    out[4] = L->a0_psi;
    out[5] = L->dt;
}

int64_t ora_steps_done(const ora_lattice* L) { return L->steps; }

/* ------------------------------------------------------------------ init */

int ora_init(ora_lattice* L, const double* ux0, const double* uy0, const double* vx0, const double* vy0) {
    int nx = L->p.nx, ny = L->p.ny;
    long n = (long)nx * ny;
    for (long k = 0; k < n; ++k) {
        if (!isfinite(ux0[k]) || !isfinite(uy0[k])) return -1;
        if (vx0 && (!isfinite(vx0[k]) || !isfinite(vy0[k]))) return -1;
    }
    memcpy(L->ux, ux0, (size_t)n * sizeof(double));
    memcpy(L->uy, uy0, (size_t)n * sizeof(double));
    if (vx0) {
        memcpy(L->vx, vx0, (size_t)n * sizeof(double));
        memcpy(L->vy, vy0, (size_t)n * sizeof(double));
    } else {
        memset(L->vx, 0, (size_t)n * sizeof(double));
        memset(L->vy, 0, (size_t)n * sizeof(double));
    }
    for (long k = 0; k < n; ++k)  /* void points hold no state */
        if (is_void(L, k)) L->ux[k] = L->uy[k] = L->vx[k] = L->vy[k] = 0.0;
    /* Fig. 3, initialisation: phi = div u, psi = curl u by finite differences,
     * then f = f_eq (Eq. feq); first moments from reading R9. */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = at(L, i, j);
            if (is_void(L, k)) continue;  /* void points hold no state */
            double phi = fd_div(L, L->ux, L->uy, i, j);
            double psi = fd_curl(L, L->ux, L->uy, i, j);
            double jphi_x = -L->vx[k], jphi_y = -L->vy[k];
            double jpsi_x = -L->vy[k], jpsi_y = L->vx[k];
            for (int a = 0; a < 5; ++a) {
                L->f[0][a][k] = f_eq(L, 0, a, phi, jphi_x, jphi_y);
                L->f[1][a][k] = f_eq(L, 1, a, psi, jpsi_x, jpsi_y);
            }
        }
    }
    L->steps = 0;
    L->initialised = 1;
    return 0;
}

/* ---------------------------------------------------------- accelerations */

/* Interior points: Eq. navier with finite differences (reading R3). */
static void accel_interior(const ora_lattice* L, int i, int j, double* ax, double* ay) {
    double dphi_dx = d_dx(L, L->s[0], i, j), dphi_dy = d_dy(L, L->s[0], i, j);
    double dpsi_dx = d_dx(L, L->s[1], i, j), dpsi_dy = d_dy(L, L->s[1], i, j);
    double cd2 = L->cd * L->cd, cs2 = L->cs * L->cs;
    /* curl(psi e_z) = (d psi/dy, -d psi/dx) */
    *ax = cd2 * dphi_dx - cs2 * dpsi_dy;
    *ay = cd2 * dphi_dy + cs2 * dpsi_dx;
}

/* Time factor of the boundary data of one kind (0 Neumann, 1 Dirichlet) at
 * time t (reading R12). */
static double load_factor(const ora_lattice* L, int kind, double t) {
    if (!(L->load_rate[kind] > 0.0)) return 1.0;
    return L->load_rate[kind] * fmin(t, L->load_hold[kind]);
}

int ora_set_load(ora_lattice* L, int32_t kind, double t_ramp, double t_hold) {
    if (!L || (kind != 1 && kind != 2) || !(t_ramp >= 0.0) || !isfinite(t_ramp) || !(t_hold > 0.0)) return -1;
    L->load_rate[kind - 1] = t_ramp > 0.0 ? 1.0 / t_ramp : 0.0;
    L->load_hold[kind - 1] = t_hold;
    return 0;
}

/* Neumann points: momentum balance of the boundary cell, Eq.
 * contBalanceOfMomentum simplified to Eq. acc_neumann (readings R5, R6, R14). */
static void accel_neumann(const ora_lattice* L, int i, int j, double* ax, double* ay) {
    long k = at(L, i, j);
    const double* cd = L->cell + 5 * k;   /* V_C, side lengths E, N, W, S */
    double vol = cd[0];
    double sk[3];
    stress(L, L->ux, L->uy, i, j, sk);
    /* External part: integral of t* over dC_ext, supplied per point, at t
     * (readings R12, R13). */
    double sn = load_factor(L, 0, (double)L->steps * L->dt);
    double fx = sn * L->bc[2 * k], fy = sn * L->bc[2 * k + 1];
    /* Internal part: one side per direction, normal n_kr = e_alpha, length
     * l_kr; stress (sigma_k + sigma_r)/2 towards a body neighbour r, sigma_k
     * on a side with no body neighbour that lies partly in the body. */
    for (int a = 1; a < 5; ++a) {
        int ri, rj;
        double len = cd[a];
        int has = neighbour(L, i, j, EX[a], EY[a], &ri, &rj);
        if (!has && !(len > 0.0)) continue;
        double sr[3];
        if (has) stress(L, L->ux, L->uy, ri, rj, sr);
        else for (int q = 0; q < 3; ++q) sr[q] = sk[q];
        double sxx = 0.5 * (sk[0] + sr[0]);
        double syy = 0.5 * (sk[1] + sr[1]);
        double sxy = 0.5 * (sk[2] + sr[2]);
        double nx_ = (double)EX[a], ny_ = (double)EY[a];
        fx += (sxx * nx_ + sxy * ny_) * len;
        fy += (sxy * nx_ + syy * ny_) * len;
    }
    *ax = fx / (L->p.rho * vol);
    *ay = fy / (L->p.rho * vol);
}

/* Dirichlet points: Eq. acc_dirichlet with the target u*(t + dt) (readings
 * R12, R13). */
static void accel_dirichlet(const ora_lattice* L, int i, int j, double* ax, double* ay) {
    long k = at(L, i, j);
    double dt = L->dt;
    double s = load_factor(L, 1, (double)(L->steps + 1) * dt);
    *ax = 2.0 / (dt * dt) * (s * L->bc[2 * k] - L->ux[k]) - 2.0 / dt * L->vx[k];
    *ay = 2.0 / (dt * dt) * (s * L->bc[2 * k + 1] - L->uy[k]) - 2.0 / dt * L->vy[k];
}

/* Moments phi, psi of the current populations (Eq. interpretation). */
static void compute_moments(ora_lattice* L) {
    int nx = L->p.nx, ny = L->p.ny;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = at(L, i, j);
            for (int set = 0; set < 2; ++set) {
                double g[5], s, jx, jy;
                gather(L->f[set], k, g);
                moments(L, g, &s, &jx, &jy);
                L->s[set][k] = s;
            }
        }
    }
}

static void compute_accelerations(ora_lattice* L) {
    int nx = L->p.nx, ny = L->p.ny;
    /* Fig. 3: interior first ... */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            if (L->type[at(L, i, j)] == 0) accel_interior(L, i, j, &L->ax[at(L, i, j)], &L->ay[at(L, i, j)]);
    /* ... then boundary points. */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = at(L, i, j);
            if (L->type[k] == 1) accel_neumann(L, i, j, &L->ax[k], &L->ay[k]);
            else if (L->type[k] == 2) accel_dirichlet(L, i, j, &L->ax[k], &L->ay[k]);
        }
    }
}

/* -------------------------------------------------------------- one step */

static void swap_ptr(double** a, double** b) {
    double* t = *a;
    *a = *b;
    *b = t;
}

/* Sec. 3.2: phi, psi from finite differences of u everywhere, then the
 * populations from Eq. correction-f with the current first moments. */
static void synchronise(ora_lattice* L) {
    int nx = L->p.nx, ny = L->p.ny;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = at(L, i, j);
            if (is_void(L, k)) continue;
            double snew[2];
            snew[0] = fd_div(L, L->ux, L->uy, i, j);
            snew[1] = fd_curl(L, L->ux, L->uy, i, j);
            for (int set = 0; set < 2; ++set) {
                double g[5], s, jx, jy;
                gather(L->f[set], k, g);
                moments(L, g, &s, &jx, &jy);
                for (int a = 0; a < 5; ++a) L->fn[set][a][k] = f_eq(L, set, a, snew[set], jx, jy);
            }
        }
    }
    for (int set = 0; set < 2; ++set)
        for (int a = 0; a < 5; ++a) swap_ptr(&L->f[set][a], &L->fn[set][a]);
}

/* Reading R15, bc_j_mode 1: the populations the plain LBE (Eq. LBE, tau =
 * dt/2, from f(., t)) streams into the boundary point (i, j): direction alpha
 * comes from the body neighbour at x - c^alpha dt after its collision; a
 * direction whose source lies outside the body keeps f^alpha(x, t). */
static void partial_stream(const ora_lattice* L, int set, int i, int j, double g[5]) {
    long k = at(L, i, j);
    double fk[5], s, jx, jy;
    gather(L->f[set], k, fk);
    moments(L, fk, &s, &jx, &jy);
    g[0] = fk[0] - 2.0 * (fk[0] - f_eq(L, set, 0, s, jx, jy));  /* the point's own rest population */
    for (int a = 1; a < 5; ++a) {
        int si, sj;
        if (!neighbour(L, i, j, -EX[a], -EY[a], &si, &sj)) {
            g[a] = fk[a];
            continue;
        }
        double fs[5], ss, sx, sy;
        gather(L->f[set], at(L, si, sj), fs);
        moments(L, fs, &ss, &sx, &sy);
        g[a] = fs[a] - 2.0 * (fs[a] - f_eq(L, set, a, ss, sx, sy));
    }
}

static void one_step(ora_lattice* L) {
    int nx = L->p.nx, ny = L->p.ny;
    double dt = L->dt;

    /* Block 1: moments at t. */
    compute_moments(L);

    /* Blocks 2-3: accelerations at t. */
    compute_accelerations(L);

    /* Block 4: Newmark, Eq. integration, at every point. */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = at(L, i, j);
            L->ux1[k] = L->ux[k] + dt * L->vx[k] + dt * dt / 2.0 * L->ax[k];
            L->uy1[k] = L->uy[k] + dt * L->vy[k] + dt * dt / 2.0 * L->ay[k];
            L->vx1[k] = L->vx[k] + dt * L->ax[k];
            L->vy1[k] = L->vy[k] + dt * L->ay[k];
        }
    }

    /* Block 5: boundary phi, psi from the new u (Eq. psi_phi_at_bound) and
     * boundary populations from Eq. correction-f (reading R7). */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = at(L, i, j);
            if (L->type[k] == 0 || is_void(L, k)) continue;
            double snew[2];
            snew[0] = fd_div(L, L->ux1, L->uy1, i, j);
            snew[1] = fd_curl(L, L->ux1, L->uy1, i, j);
            for (int set = 0; set < 2; ++set) {
                double g[5], s, jx, jy;
                if (L->p.bc_j_mode == 1) partial_stream(L, set, i, j, g);
                else gather(L->f[set], k, g);
                moments(L, g, &s, &jx, &jy);
                for (int a = 0; a < 5; ++a) L->fn[set][a][k] = f_eq(L, set, a, snew[set], jx, jy);
            }
        }
    }

    /* Block 6a: collision at every source point.  Boundary sources collide the
     * time-averaged state f-tilde (Eq. LBE_mod); all others collide f(x,t)
     * (Eq. LBE).  tau = dt/2 (reading R10). */
    const double dt_over_tau = 2.0;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = at(L, i, j);
            if (is_void(L, k)) continue;  /* no state, never a source */
            int bnd = L->type[k] != 0;
            for (int set = 0; set < 2; ++set) {
                double fold[5], fhat[5], s, jx, jy;
                gather(L->f[set], k, fold);
                for (int a = 0; a < 5; ++a)
                    fhat[a] = bnd ? 0.5 * (L->fn[set][a][k] + fold[a]) : fold[a];
                if (bnd && L->p.bc_feq_mode == 1) moments(L, fold, &s, &jx, &jy);
                else moments(L, fhat, &s, &jx, &jy);
                for (int a = 0; a < 5; ++a) {
                    double feq = f_eq(L, set, a, s, jx, jy);
                    L->fc[set][a][k] = fhat[a] - dt_over_tau * (fhat[a] - feq);
                }
            }
        }
    }

    /* Block 6b: streaming into interior points only; boundary points keep the
     * values of block 5. */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = at(L, i, j);
            if (L->type[k] != 0) continue;
            for (int a = 0; a < 5; ++a) {
                int si = i, sj = j;
                neighbour(L, i, j, -EX[a], -EY[a], &si, &sj); /* interior: always exists */
                long ks = at(L, si, sj);
                L->fn[0][a][k] = L->fc[0][a][ks];
                L->fn[1][a][k] = L->fc[1][a][ks];
            }
        }
    }

    /* t -> t + dt */
    for (int set = 0; set < 2; ++set)
        for (int a = 0; a < 5; ++a) swap_ptr(&L->f[set][a], &L->fn[set][a]);
    swap_ptr(&L->ux, &L->ux1);
    swap_ptr(&L->uy, &L->uy1);
    swap_ptr(&L->vx, &L->vx1);
    swap_ptr(&L->vy, &L->vy1);
    L->steps += 1;

    /* Block 7: synchronisation every l-th step (Sec. 3.2). */
    if (L->p.sync_every > 0 && L->steps % L->p.sync_every == 0) synchronise(L);
}

int ora_step(ora_lattice* L, int64_t n) {
    if (!L->initialised || n < 0) return -1;
    for (int64_t t = 0; t < n; ++t) one_step(L);
    return 0;
}

int ora_sync(ora_lattice* L) {
    if (!L->initialised) return -1;
    synchronise(L);
    return 0;
}

/* ------------------------------------------------------------------ read */

int ora_read(ora_lattice* L, int32_t field, double* dst) {
    int nx = L->p.nx, ny = L->p.ny;
    long n = (long)nx * ny;
    switch (field) {
    case ORA_UX: memcpy(dst, L->ux, (size_t)n * sizeof(double)); return 0;
    case ORA_UY: memcpy(dst, L->uy, (size_t)n * sizeof(double)); return 0;
    case ORA_VX: memcpy(dst, L->vx, (size_t)n * sizeof(double)); return 0;
    case ORA_VY: memcpy(dst, L->vy, (size_t)n * sizeof(double)); return 0;
    case ORA_PHI:
    case ORA_PSI: {
        compute_moments(L);
        memcpy(dst, L->s[field == ORA_PHI ? 0 : 1], (size_t)n * sizeof(double));
        return 0;
    }
    case ORA_F_PHI:
    case ORA_F_PSI: {
        int set = field == ORA_F_PHI ? 0 : 1;
        for (int a = 0; a < 5; ++a) memcpy(dst + a * n, L->f[set][a], (size_t)n * sizeof(double));
        return 0;
    }
    case ORA_ERR: {
        /* Consistency error e(x,t) of Sec. 4. */
        compute_moments(L);
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                long k = at(L, i, j);
                if (is_void(L, k)) {
                    dst[k] = 0.0;
                    continue;
                }
                double d_psi = L->s[1][k] - fd_curl(L, L->ux, L->uy, i, j);
                double d_phi = L->s[0][k] - fd_div(L, L->ux, L->uy, i, j);
                dst[k] = sqrt(d_psi * d_psi + d_phi * d_phi);
            }
        }
        return 0;
    }
    case ORA_AX:
    case ORA_AY: {
        compute_moments(L);
        compute_accelerations(L);
        memcpy(dst, field == ORA_AX ? L->ax : L->ay, (size_t)n * sizeof(double));
        return 0;
    }
    case ORA_EKIN:
    case ORA_ESTRAIN: {
        /* Energy densities per unit area, 0 at void points: rho |v|^2 / 2, and
         * half the double contraction of the stress (Eq. hooke) with the
         * strain (Eq. strain), both from the finite differences of u. */
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                long k = at(L, i, j);
                if (is_void(L, k)) {
                    dst[k] = 0.0;
                    continue;
                }
                if (field == ORA_EKIN) {
                    dst[k] = 0.5 * L->p.rho * (L->vx[k] * L->vx[k] + L->vy[k] * L->vy[k]);
                    continue;
                }
                double sig[3];
                stress(L, L->ux, L->uy, i, j, sig);
                double exx = d_dx(L, L->ux, i, j);
                double eyy = d_dy(L, L->uy, i, j);
                double exy = 0.5 * (d_dy(L, L->ux, i, j) + d_dx(L, L->uy, i, j));
                dst[k] = 0.5 * (sig[0] * exx + sig[1] * eyy + 2.0 * sig[2] * exy);
            }
        }
        return 0;
    }
    default: return -1;
    }
}

/* ------------------------------------------------------------ state rows */

static double* row_plane(const ora_lattice* L, int q) {
    if (q < 10) return L->f[q / 5][q % 5];
    double* u[4] = {L->ux, L->uy, L->vx, L->vy};
    return u[q - 10];
}

int ora_get_rows(const ora_lattice* L, int32_t row0, int32_t rows, double* dst) {
    if (!L->initialised || row0 < 0 || rows < 0 || row0 + rows > L->p.ny) return -1;
    long blk = (long)rows * L->p.nx;
    for (int q = 0; q < 14; ++q)
        memcpy(dst + q * blk, row_plane(L, q) + (long)row0 * L->p.nx, (size_t)blk * sizeof(double));
    return 0;
}

int ora_set_rows(ora_lattice* L, int32_t row0, int32_t rows, const double* src) {
    if (!L->initialised || row0 < 0 || rows < 0 || row0 + rows > L->p.ny) return -1;
    long blk = (long)rows * L->p.nx;
    for (int q = 0; q < 14; ++q)
        memcpy(row_plane(L, q) + (long)row0 * L->p.nx, src + q * blk, (size_t)blk * sizeof(double));
    return 0;
}

/* ------------------------------------------------------ rectangle helper */

int ora_rect_bc(int32_t nx, int32_t ny, int32_t periodic_x, int32_t periodic_y, double dh,
                const int32_t edge_type[4], const double edge_value[8], uint8_t* node_type,
                double* bc_value) {
    if (nx < 3 || ny < 3 || !(dh > 0.0)) return -1;
    /* edges: 0 bottom (j = 0), 1 right (i = nx-1), 2 top (j = ny-1), 3 left (i = 0) */
    for (int e = 0; e < 4; ++e) {
        int active = (e == 0 || e == 2) ? !periodic_y : !periodic_x;
        if (active && edge_type[e] != 1 && edge_type[e] != 2) return -1;
    }
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = (long)j * nx + i;
            int on[4];
            on[0] = !periodic_y && j == 0;
            on[1] = !periodic_x && i == nx - 1;
            on[2] = !periodic_y && j == ny - 1;
            on[3] = !periodic_x && i == 0;
            int n_on = on[0] + on[1] + on[2] + on[3];
            node_type[k] = 0;
            bc_value[2 * k] = 0.0;
            bc_value[2 * k + 1] = 0.0;
            if (n_on == 0) continue;
            int n_dir = 0;
            for (int e = 0; e < 4; ++e) n_dir += on[e] && edge_type[e] == 2;
            if (n_dir > 0) {
                /* Dirichlet dominates; the mean of the prescribed u* at a
                 * Dirichlet-Dirichlet corner. */
                node_type[k] = 2;
                for (int e = 0; e < 4; ++e) {
                    if (on[e] && edge_type[e] == 2) {
                        bc_value[2 * k] += edge_value[2 * e] / n_dir;
                        bc_value[2 * k + 1] += edge_value[2 * e + 1] / n_dir;
                    }
                }
            } else {
                /* Neumann: F = sum over the external faces of t* times the face
                 * length; an edge point has one face of length dh, a corner two
                 * of length dh/2. */
                node_type[k] = 1;
                double len = n_on == 1 ? dh : 0.5 * dh;
                for (int e = 0; e < 4; ++e) {
                    if (on[e]) {
                        bc_value[2 * k] += edge_value[2 * e] * len;
                        bc_value[2 * k + 1] += edge_value[2 * e + 1] * len;
                    }
                }
            }
        }
    }
    return 0;
}

/* ------------------------------------------- plate with a circular hole */

#define ORA_PI 3.14159265358979323846

/* Contribution (x dy - y dx) / 2 of the straight segment p -> q to the area
 * of the region on its left (Green's theorem). */
static double green_segment(double px, double py, double qx, double qy) {
    return 0.5 * (px * qy - py * qx);
}

/* The same for the arc of the circle of radius r from angle t1 down to t0
 * (clockwise, t1 > t0), whose end points are p1 (at t1) and p0 (at t0): the
 * chord p1 -> p0, less the circular segment between arc and chord, of area
 * r^2 (dt - sin dt) / 2, which the clockwise arc leaves on its right. */
static double green_arc_cw(double r, double t0, double t1, double p0x, double p0y, double p1x, double p1y) {
    double dt = t1 - t0;
    return green_segment(p1x, p1y, p0x, p0y) - 0.5 * r * r * (dt - sin(dt));
}

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Reading R16: the region A = S minus the open disk D, S = [x0, x1] x
 * [y0, y1].  Its area is (1/2) times the integral of x dy - y dx around its
 * boundary, which consists of the parts of the sides of S outside D,
 * traversed counter-clockwise, and the arcs of the circle inside S,
 * traversed clockwise (A lies outside the circle).  The pieces need not be
 * joined into loops: the integral is a sum over them. */
void ora_clip_rect(double x0, double x1, double y0, double y1, double cx, double cy, double r, double out[5]) {
    /* coordinates relative to the rectangle's centre (the area does not
     * depend on the origin, and small coordinates keep the sums exact) */
    const double xm = 0.5 * (x0 + x1), ym = 0.5 * (y0 + y1);
    x0 -= xm; x1 -= xm; cx -= xm;
    y0 -= ym; y1 -= ym; cy -= ym;
    /* sides in counter-clockwise order: S (y = y0), E (x = x1), N (y = y1),
     * W (x = x0); out[] lists them E, N, W, S */
    const double P[4][2] = {{x0, y0}, {x1, y0}, {x1, y1}, {x0, y1}};
    const int slot[4] = {4, 1, 2, 3};
    double area = 0.0;
    for (int q = 1; q < 5; ++q) out[q] = 0.0;
    for (int e = 0; e < 4; ++e) {
        double ax = P[e][0], ay = P[e][1], bx = P[(e + 1) % 4][0], by = P[(e + 1) % 4][1];
        double dx = bx - ax, dy = by - ay, len = sqrt(dx * dx + dy * dy);
        if (!(len > 0.0)) continue;
        /* |a + t (b - a) - c|^2 < r^2 for t in (t_in, t_out): a quadratic in t */
        double ex = ax - cx, ey = ay - cy;
        double qa = dx * dx + dy * dy, qb = 2.0 * (ex * dx + ey * dy), qc = ex * ex + ey * ey - r * r;
        double disc = qb * qb - 4.0 * qa * qc;
        double pieces[2][2];
        int np = 0;
        if (r > 0.0 && disc > 0.0) {
            double sq = sqrt(disc);
            double t_in = (-qb - sq) / (2.0 * qa), t_out = (-qb + sq) / (2.0 * qa);
            if (t_in > 0.0) { pieces[np][0] = 0.0; pieces[np][1] = fmin(t_in, 1.0); ++np; }
            if (t_out < 1.0) { pieces[np][0] = fmax(t_out, 0.0); pieces[np][1] = 1.0; ++np; }
        } else {
            pieces[0][0] = 0.0;
            pieces[0][1] = 1.0;
            np = 1;
        }
        for (int m = 0; m < np; ++m) {
            double s0 = pieces[m][0], s1 = pieces[m][1];
            if (!(s1 > s0)) continue;
            area += green_segment(ax + s0 * dx, ay + s0 * dy, ax + s1 * dx, ay + s1 * dy);
            out[slot[e]] += (s1 - s0) * len;
        }
    }
    if (r > 0.0) {
        /* angles where the circle crosses the four lines of the sides */
        double th[9];
        int n = 0;
        const double lines_x[2] = {x0, x1}, lines_y[2] = {y0, y1};
        for (int m = 0; m < 2; ++m) {
            double u = (lines_x[m] - cx) / r;
            if (fabs(u) < 1.0) {
                double t = acos(u);
                th[n++] = t;
                th[n++] = 2.0 * ORA_PI - t;
            }
            double v = (lines_y[m] - cy) / r;
            if (fabs(v) < 1.0) {
                double t = asin(v);
                th[n++] = t < 0.0 ? t + 2.0 * ORA_PI : t;
                th[n++] = ORA_PI - t;
            }
        }
        if (n == 0) {
            /* no crossing: the whole circle lies inside S or outside it */
            if (cx + r > x0 && cx + r < x1 && cy > y0 && cy < y1) area -= ORA_PI * r * r;
        } else {
            qsort(th, (size_t)n, sizeof(double), cmp_double);
            th[n] = th[0] + 2.0 * ORA_PI;
            for (int m = 0; m < n; ++m) {
                double t0 = th[m], t1 = th[m + 1];
                if (!(t1 > t0)) continue;
                /* between two crossings the arc lies on one side of every
                 * line; it may still touch a side where it is tangent to it,
                 * so it counts as inside if any of three points along it lies
                 * strictly inside */
                int inside = 0;
                for (int q = 1; q <= 3; ++q) {
                    double tq = t0 + 0.25 * q * (t1 - t0);
                    double mx = cx + r * cos(tq), my = cy + r * sin(tq);
                    inside = inside || (mx > x0 && mx < x1 && my > y0 && my < y1);
                }
                if (inside)
                    area += green_arc_cw(r, t0, t1, cx + r * cos(t0), cy + r * sin(t0), cx + r * cos(t1),
                                         cy + r * sin(t1));
            }
        }
    }
    out[0] = area;
}

int ora_disk_cells(int32_t nx, int32_t ny, double dh, double cx, double cy, double r,
                   const int32_t edge_type[4], const double edge_value[8],
                   uint8_t* node_type, double* bc_value, double* cell) {
    if (nx < 3 || ny < 3 || !(dh > 0.0) || !(r >= 0.0) || !isfinite(r) || !isfinite(cx) || !isfinite(cy))
        return -1;
    for (int e = 0; e < 4; ++e)
        if (edge_type[e] != 1 && edge_type[e] != 2) return -1;
    long n = (long)nx * ny;
    double Lx = (nx - 1) * dh, Ly = (ny - 1) * dh, h2 = 0.5 * dh;
    /* void points: strictly inside the circle */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double x = i * dh - cx, y = j * dh - cy;
            node_type[(long)j * nx + i] = (x * x + y * y < r * r) ? 3 : 0;
        }
    for (long k = 0; k < 2 * n; ++k) bc_value[k] = 0.0;
    for (long k = 0; k < 5 * n; ++k) cell[k] = 0.0;
    const int DI[4] = {1, 0, -1, 0}, DJ[4] = {0, 1, 0, -1};
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = (long)j * nx + i;
            if (node_type[k] == 3) continue;
            int bnd = 0;
            for (int d = 0; d < 4; ++d) {
                int ni = i + DI[d], nj = j + DJ[d];
                if (ni < 0 || ni >= nx || nj < 0 || nj >= ny || node_type[(long)nj * nx + ni] == 3) bnd = 1;
            }
            if (!bnd) continue;
            /* outer edges the point lies on: bottom, right, top, left */
            int on[4] = {j == 0, i == nx - 1, j == ny - 1, i == 0};
            int n_dir = 0;
            for (int e = 0; e < 4; ++e) n_dir += on[e] && edge_type[e] == 2;
            if (n_dir > 0) {
                node_type[k] = 2;
                for (int e = 0; e < 4; ++e)
                    if (on[e] && edge_type[e] == 2) {
                        bc_value[2 * k] += edge_value[2 * e] / n_dir;
                        bc_value[2 * k + 1] += edge_value[2 * e + 1] / n_dir;
                    }
                continue;
            }
            node_type[k] = 1;
            double x = i * dh, y = j * dh;
            double sx0 = fmax(x - h2, 0.0), sx1 = fmin(x + h2, Lx);
            double sy0 = fmax(y - h2, 0.0), sy1 = fmin(y + h2, Ly);
            double c[5];
            ora_clip_rect(sx0, sx1, sy0, sy1, cx, cy, r, c);
            double* cd = cell + 5 * k;
            cd[0] = c[0];
            /* sides of the square inside the body rectangle; the sides of the
             * clipped square on an outer edge are external faces instead */
            int inside[4] = {x + h2 <= Lx, y + h2 <= Ly, x - h2 >= 0.0, y - h2 >= 0.0};
            for (int q = 0; q < 4; ++q) cd[1 + q] = inside[q] ? c[1 + q] : 0.0;
            /* external faces on the outer edges: E face on the right edge,
             * N on the top, W on the left, S on the bottom */
            const int edge_of_side[4] = {1, 2, 3, 0};
            for (int q = 0; q < 4; ++q) {
                if (inside[q]) continue;
                int e = edge_of_side[q];
                bc_value[2 * k] += edge_value[2 * e] * c[1 + q];
                bc_value[2 * k + 1] += edge_value[2 * e + 1] * c[1 + q];
            }
        }
    }
    return 0;
}
