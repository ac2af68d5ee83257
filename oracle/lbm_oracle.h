/*
 * FP64 CPU oracle for the plane-strain lattice Boltzmann method of
 * Schlueter, Yan, Faust, Mueller & Mueller, "A Lattice Boltzmann Method for
 * Elastic Solids Under Plane Strain Deformation" (arXiv:2301.00228).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and lbm_oracle.c are the plain,
 * slow reference that the CUDA library is checked against.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark load the
 * compiled oracle.  It shares no code, header, table or constant with the
 * CUDA library, and it never reads anything the CUDA library produced.
 *
 * The interface mirrors the problem statement of Sec. 2 and the algorithm
 * summary of Fig. 3: create a rectangular lattice with material constants
 * and boundary data, initialise from u(x,0) and du/dt(x,0), advance n time
 * steps, read fields.  All arrays are row-major [ny][nx] with x fastest.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ora_params {
    int32_t nx, ny;          /* lattice points along x and y (each >= 3)   */
    double lambda, mu, rho;  /* Lame constants and density, Sec. 2        */
    double dh;               /* lattice spacing Delta h                    */
    double a0_phi;           /* rest weight a_{0,phi}, Eq. feq_req; the
                                examples of Sec. 4 use 0.9999              */
    int32_t periodic_x;      /* 1: x wraps, no boundary points along x     */
    int32_t periodic_y;
    int32_t bc_feq_mode;     /* equilibrium in the modified LBE, Eq. LBE_mod:
                                0 = moments of the averaged state f-hat,
                                1 = moments of f(x_k, t)                   */
    int32_t sync_every;      /* periodic synchronisation interval l of
                                Sec. 3.2; 0 disables it                    */
    int32_t bc_j_mode;       /* first moment J(x_k, t) in Eq. correction-f:
                                0 = of the populations stored at x_k,
                                1 = of the populations the LBE streams into
                                x_k from its body neighbours, the stored
                                ones kept for directions from outside the
                                body (reading R15)                          */
} ora_params;

typedef struct ora_lattice ora_lattice;

/* node_type[ny][nx]: 0 interior, 1 Neumann, 2 Dirichlet.  Non-zero exactly on
 * the outer ring of non-periodic directions (see ora_create_cells for void
 * points).  bc_value[ny][nx][2]: prescribed
 * displacement u* at Dirichlet points, integrated external force
 * F = int_{dC_ext} t* da at Neumann points (Eq. acc_neumann), ignored at
 * interior points.  Returns NULL on invalid input. */
ora_lattice* ora_create(const ora_params* p, const uint8_t* node_type,
                        const double* bc_value);

/* As ora_create for a general geometry (reading R14): node_type may also
 * hold 3 (void, not in the body); cell[ny][nx][5] gives, at boundary
 * points, the cell area V_C and the length in the body of the cell's sides
 * towards E, N, W, S (NULL: the clipped squares of a rectangle, R6). */
ora_lattice* ora_create_cells(const ora_params* p, const uint8_t* node_type,
                              const double* bc_value, const double* cell);
void ora_destroy(ora_lattice* L);

/* Derived constants of Eq. conditions-parameters: c_d, c_s, a_phi, a_psi,
 * a_{0,psi}, Delta t. */
void ora_constants(const ora_lattice* L, double out[6]);

/* Initialisation block of Fig. 3.  v0 may be NULL (body at rest). */
int ora_init(ora_lattice* L, const double* ux0, const double* uy0,
             const double* vx0, const double* vy0);

/* Time-dependent boundary data (readings R12, R13): the values of one kind
 * (1 Neumann forces, 2 Dirichlet targets) are multiplied by
 * s(t) = min(t, t_hold) / t_ramp; t_ramp = 0 restores constant data.  The
 * Neumann force at step n uses t = n dt, the Dirichlet target t = (n+1) dt.
 * t_hold may be +infinity (a ramp without hold).  Returns -1 on bad input. */
int ora_set_load(ora_lattice* L, int32_t kind, double t_ramp, double t_hold);

/* Time loop of Fig. 3, n iterations. */
int ora_step(ora_lattice* L, int64_t n);

/* Periodic synchronisation of Sec. 3.2, applied to the current state. */
int ora_sync(ora_lattice* L);

/* Field ids for ora_read. */
enum {
    ORA_UX = 0, ORA_UY = 1, ORA_VX = 2, ORA_VY = 3,
    ORA_PHI = 4, ORA_PSI = 5,
    ORA_F_PHI = 6, ORA_F_PSI = 7,   /* 5 planes each, alpha-major          */
    ORA_ERR = 8,                    /* consistency error e of Sec. 4       */
    ORA_AX = 9, ORA_AY = 10,        /* acceleration the next step would use */
    ORA_EKIN = 11,                  /* kinetic energy density rho |v|^2 / 2  */
    ORA_ESTRAIN = 12                /* strain energy density sigma : eps / 2 (Eq. hooke,
                                       Eq. strain by the finite differences of Sec. 3.1.2) */
};
/* Copies a field into dst (nx*ny doubles, 5*nx*ny for population sets). */
int ora_read(ora_lattice* L, int32_t field, double* dst);
int64_t ora_steps_done(const ora_lattice* L);

/* Rectangle boundary helper.  edge order: bottom (y=0), right (x=nx-1),
 * top (y=ny-1), left (x=0).  edge_type: 1 Neumann, 2 Dirichlet (ignored for
 * periodic directions).  edge_value[e][2]: u* for Dirichlet edges, traction
 * t* (force per unit length) for Neumann edges.  Corner readings: Dirichlet
 * dominates Neumann; two Dirichlet edges give the mean u*; two Neumann edges
 * add both external half faces. */
int ora_rect_bc(int32_t nx, int32_t ny, int32_t periodic_x, int32_t periodic_y,
                double dh, const int32_t edge_type[4],
                const double edge_value[8], uint8_t* node_type,
                double* bc_value);

/* A rectangle of lattice points (point (i, j) at (i dh, j dh), body
 * [0, (nx-1) dh] x [0, (ny-1) dh]) with a traction-free circular hole of
 * centre (cx, cy) and radius r (reading R14; the plate with a hole of
 * Sec. 4).  Points strictly inside the circle are void (3); a body point with
 * a neighbour outside the body is a boundary point: Dirichlet (2) on a
 * Dirichlet outer edge (corner rules of ora_rect_bc), Neumann (1) otherwise.
 * bc_value[ny][nx][2]: u* at Dirichlet points; at Neumann points the outer
 * edges' traction t* times the length of the cell's faces on those edges
 * outside the hole (the hole itself is traction-free).  cell[ny][nx][5]: at
 * Neumann points the area of the cell (the square of side dh around the
 * point, clipped to the body rectangle, minus the disk) and the lengths of
 * its sides towards E, N, W, S that lie inside the body rectangle, outside
 * the disk; zero elsewhere.  Returns -1 on bad input. */
int ora_disk_cells(int32_t nx, int32_t ny, double dh, double cx, double cy, double r,
                   const int32_t edge_type[4], const double edge_value[8],
                   uint8_t* node_type, double* bc_value, double* cell);

/* The part of the rectangle [x0, x1] x [y0, y1] outside the open disk of
 * centre (cx, cy) and radius r: out[0] its area, out[1..4] the lengths of the
 * rectangle's sides x = x1, y = y1, x = x0, y = y0 outside the disk. */
void ora_clip_rect(double x0, double x1, double y0, double y1, double cx, double cy, double r,
                   double out[5]);

/* State rows for a domain decomposition test: rows [row0, row0 + rows) of
 * the current state, as 14 blocks of rows x nx doubles in the order
 * f_phi^0..4, f_psi^0..4, u_x, u_y, v_x, v_y.  get copies out, set copies in
 * (the lattice must be initialised).  Return -1 on a bad row range. */
int ora_get_rows(const ora_lattice* L, int32_t row0, int32_t rows, double* dst);
int ora_set_rows(ora_lattice* L, int32_t row0, int32_t rows, const double* src);

void ora_set_threads(int32_t n);
int32_t ora_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
