/*
 * lbps.h -- C ABI of the GB300 plane-strain lattice Boltzmann solver.
 *
 * Method: Schlueter, Yan, Faust, Mueller & Mueller, "A Lattice Boltzmann
 * Method for Elastic Solids Under Plane Strain Deformation",
 * arXiv:2301.00228.  The calls follow the paper's statement of the problem
 * (Sec. 2: a body with Dirichlet data u* and Neumann data t* on its edges)
 * and its algorithm summary (Fig. 3: build the lattice, initialise, run the
 * time loop, read fields).  Every time step runs on the GPU in hand-written
 * sm_103a CUDA kernels; nothing here falls back to the host.
 *
 * Conventions
 *   - Host arrays are row-major [ny][nx], x fastest, FP64 unless stated.
 *   - The caller owns every buffer it passes; the library copies what it
 *     needs during the call and keeps no pointer to caller host memory.
 *   - Device memory: lbps_create either allocates it (device_mem == NULL)
 *     or lives in a caller-provided device block of lbps_state_bytes()
 *     bytes that must outlive the lattice (e.g. a torch tensor).
 *   - Every call returns LBPS_OK (0) or a negative LBPS_ERR_* code.  No call
 *     aborts, prints or throws.  lbps_strerror() names the code.
 *   - Work is enqueued on params.cuda_stream (a cudaStream_t; NULL means
 *     the legacy default stream).  Calls that take host buffers synchronise
 *     the stream before returning; *_async / *_device calls do not.
 *   - Units are the caller's; the configurations used by the tests take
 *     lattice units (dh = 1).
 */
#ifndef LBPS_H
#define LBPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBPS_OK 0
#define LBPS_ERR_INVALID (-1)   /* bad argument, size, mask or parameter      */
#define LBPS_ERR_OOM (-2)       /* device allocation failed / block too small */
#define LBPS_ERR_CUDA (-3)      /* a CUDA runtime call or launch failed       */
#define LBPS_ERR_NONFINITE (-4) /* the state became non-finite (instability)  */
#define LBPS_ERR_TIMEOUT (-5)   /* reserved: no kernel waits on the device, so
                                   no call returns it                        */
#define LBPS_ERR_STATE (-6)     /* call out of order (e.g. step before init)  */

/* Node types of the boundary mask (Sec. 2, Fig. 1). */
#define LBPS_INTERIOR 0
#define LBPS_NEUMANN 1          /* traction t* prescribed: Eq. acc_neumann    */
#define LBPS_DIRICHLET 2        /* displacement u* prescribed: Eq. acc_dirichlet */
#define LBPS_VOID 3             /* not in the body (lbps_create_cells only)    */

/* Storage of the populations (Eq. interpretation).  u and du/dt are FP64 in
 * every format.  The 16-bit formats store, per set, the conserved moments
 * f^0, Jx = f^1 - f^3, Jy = f^2 - f^4 in FP32 and the two pair sums'
 * deviations from equilibrium (Eq. feq), Nx = f^1 + f^3 - 2 (a/a_0) f^0 and
 * Ny = f^2 + f^4 - 2 (a/a_0) f^0, in 16 bits a value multiplied by
 * 2^scale_exp; with a0_phi >= 0.999 (slow waves) BF16 and FP16 round them stochastically,
 * with random bits hashed from the value and its position (deterministic, so
 * results do not depend on launch shape, batching or resumes), otherwise to
 * nearest; arithmetic is FP32.  32 bytes per point per state copy instead of
 * 40 (FP32).  They reject lattices 3 points wide along a non-periodic axis
 * (LBPS_ERR_INVALID). */
#define LBPS_STORAGE_F32 0      /* FP32 populations, FP32 arithmetic          */
#define LBPS_STORAGE_F64 1      /* FP64 populations, FP64 arithmetic          */
#define LBPS_STORAGE_BF16 2     /* FP32 moments + bfloat16 Nx, Ny             */
#define LBPS_STORAGE_F16 3      /* FP32 moments + IEEE half Nx, Ny            */
#define LBPS_STORAGE_BFP13 4    /* FP32 moments + Nx, Ny of each set in one
                                   32-bit block-floating-point word: a shared
                                   4-bit exponent E and two sign + 13-bit
                                   magnitudes m, value m 2^(E-13) (bits 31..28
                                   E, 27 sign of Nx, 26..14 m of Nx, 13 sign of
                                   Ny, 12..0 m of Ny; E = 15 with m = 8191:
                                   infinity).  Rounded to nearest (ties to
                                   even), never stochastically.  The boundary
                                   reset takes one more launch per step.      */

/* Fields for lbps_read / lbps_read_device. */
#define LBPS_UX 0               /* displacement u_x                            */
#define LBPS_UY 1
#define LBPS_VX 2               /* velocity du_x/dt                            */
#define LBPS_VY 3
#define LBPS_PHI 4              /* dilatation phi = sum_alpha f_phi^alpha      */
#define LBPS_PSI 5              /* rotation psi = sum_alpha f_psi^alpha        */
#define LBPS_F_PHI 6            /* the 5 phi populations, [5][ny][nx]          */
#define LBPS_F_PSI 7            /* the 5 psi populations, [5][ny][nx]          */
#define LBPS_CONSISTENCY 8      /* error measure e(x,t) of Sec. 4              */
#define LBPS_KINETIC_ENERGY 9   /* rho |du/dt|^2 / 2 per unit area (0 at void points) */
#define LBPS_STRAIN_ENERGY 10   /* sigma : eps / 2 = lambda tr(eps)^2 / 2 + mu eps : eps
                                   (Eq. hooke, eps by the finite differences of
                                   Sec. 3.1.2; 0 at void points)              */

typedef struct lbps_params {
    int32_t nx, ny;             /* lattice points along x, y; each >= 3       */
    double lambda, mu, rho;     /* Lame constants, density (Sec. 2);
                                   mu > 0, rho > 0, lambda + 2 mu > 0          */
    double dh;                  /* lattice spacing Delta h > 0 (Sec. 3)       */
    double a0_phi;              /* rest weight a_{0,phi} in [0, 1) of Eq. feq;
                                   the paper's examples use 0.9999 (Sec. 4)   */
    int32_t periodic_x;         /* 1: x wraps around, no boundary along x     */
    int32_t periodic_y;
    int32_t bc_feq_mode;        /* Eq. LBE_mod equilibrium: 0 = moments of the
                                   averaged state f-hat, 1 = moments of
                                   f(x_k, t)                                   */
    int32_t sync_every;         /* l of Sec. 3.2 (0 = no synchronisation)     */
    int32_t storage;            /* LBPS_STORAGE_*                              */
    int32_t pop_scale_exp;      /* 16-bit storage: the exponent e of 2^e that
                                   Nx, Ny are stored times, |e| <= 100; 0 =
                                   chosen by each init so that the size of J
                                   the initial state and boundary values imply
                                   lands near 2^10 (Nx, Ny are smaller; half's
                                   limit is 65504).  Ignored for FP32 / FP64.  */
    void* cuda_stream;          /* cudaStream_t for all work of this lattice  */
    int32_t bc_j_mode;          /* J(x_k, t) of Eq. correction-f (Sec. 3.1.2):
                                   0 = first moment of the populations stored
                                   at the boundary point; 1 = of the
                                   populations the LBE (Eq. LBE, from f(., t))
                                   streams into it from its body neighbours,
                                   its own stored ones kept for directions
                                   coming from outside the body (the paper's
                                   boundary points "can only partially be
                                   updated via the LBE")                      */
} lbps_params;

typedef struct lbps_lattice lbps_lattice; /* opaque, library-owned */

/* Name of an error code (static string). */
const char* lbps_strerror(int code);

/* Rectangle helper (Sec. 2, Fig. 1; boundary cells of Sec. 3.1.1).
 * Fills node_type[ny][nx] and bc_value[ny][nx][2] for a rectangle whose four
 * edges (order: bottom y=0, right x=nx-1, top y=ny-1, left x=0) are each
 * Neumann or Dirichlet.  edge_value[2e], [2e+1]: u* of a Dirichlet edge, or
 * traction t* (force per unit length) of a Neumann edge, which is integrated
 * over each boundary cell's external faces (Eq. acc_neumann): dh at an edge
 * point, dh/2 per edge at a corner.  At corners Dirichlet dominates; two
 * Dirichlet edges give the mean u*.  Edges of periodic directions are
 * ignored.  Returns LBPS_ERR_INVALID for sides < 3 or an edge type other
 * than 1 or 2 on a non-periodic edge. */
int lbps_rect_bc(int32_t nx, int32_t ny, int32_t periodic_x, int32_t periodic_y, double dh,
                 const int32_t edge_type[4], const double edge_value[8],
                 uint8_t* node_type, double* bc_value);

/* Device bytes that lbps_create needs for this lattice (two state copies,
 * each with its boundary mirror and boundary-cell stresses, the boundary
 * table and reduction scratch). */
int lbps_state_bytes(const lbps_params* params, size_t* bytes);

/* Build the lattice (Fig. 3, preprocessing).
 * node_type[ny][nx]: LBPS_INTERIOR inside, LBPS_NEUMANN or LBPS_DIRICHLET on
 * the outer ring of every non-periodic direction (exactly there), or NULL for
 * a fully periodic lattice.  bc_value[ny][nx][2]: u* at Dirichlet points, the
 * integrated external force F = int_{dC_ext} t* da at Neumann points (Eq.
 * acc_neumann); NULL means zero.  device_mem: NULL to let the library
 * allocate, or a device block of at least lbps_state_bytes() bytes, 256-byte
 * aligned, owned by the caller.  On success *out owns the lattice. */
int lbps_create(const lbps_params* params, const uint8_t* node_type, const double* bc_value,
                void* device_mem, size_t device_bytes, lbps_lattice** out);

/* General geometry (Sec. 3 preprocessing, Sec. 4 plate with a hole; the
 * paper does not detail its cells, this is the library's reading):
 * node_type may also hold LBPS_VOID (points outside the body, e.g. inside a
 * hole).  A body point with a neighbour outside the body is a boundary point
 * and must be Neumann or Dirichlet; all others interior.  cell[ny][nx][5]
 * (may be NULL) gives at Neumann points the cell of side dh around the point
 * clipped to the body: its area V_C and the length in the body of its sides
 * towards E, N, W, S; NULL uses the square clipped at missing neighbours.
 * A side towards a body neighbour carries the averaged stress of Eq.
 * acc_neumann, a side towards none that lies partly in the body the point's
 * own stress (a uniform stress is then in equilibrium); bc_value gives the
 * force on the rest of the cell boundary.  Differences are central where both
 * neighbours are in the body, otherwise one-sided three-point towards it;
 * LBPS_ERR_INVALID if a body point has no such stencil along x or y, if the
 * node types do not match the body, or, with 16-bit storage, if a point has
 * boundary neighbours on both sides along an axis.  The interior kernel then
 * reads one byte of node type per point.  device_bytes: at least
 * lbps_state_bytes_cells.  Otherwise as lbps_create. */
int lbps_state_bytes_cells(const lbps_params* params, const uint8_t* node_type, const double* cell,
                           size_t* bytes);
int lbps_create_cells(const lbps_params* params, const uint8_t* node_type, const double* bc_value,
                      const double* cell, void* device_mem, size_t device_bytes, lbps_lattice** out);

/* Plate with a circular hole (Sec. 4, third example; Sec. 3 preprocessing:
 * the cell of a boundary point is the square of side dh around it "modified
 * to match the boundary geometry", which gives V_C, the face lengths l_kr and
 * the external boundary of Eq. acc_neumann).  Fills the inputs of
 * lbps_create_cells for an nx x ny rectangle of lattice points (point (i, j)
 * at (i dh, j dh); body [0, (nx-1) dh] x [0, (ny-1) dh]) with a traction-free
 * hole, the open disk of centre (cx, cy) and radius r (caller's length
 * units):
 *   node_type[ny][nx]: LBPS_VOID strictly inside the circle; a body point
 *     with a neighbour outside the body is LBPS_DIRICHLET if it lies on a
 *     Dirichlet outer edge (corner rules of lbps_rect_bc), else
 *     LBPS_NEUMANN; all others LBPS_INTERIOR;
 *   cell[ny][nx][5] at Neumann points: the area of the square around the
 *     point clipped to the body rectangle, minus the disk, and the lengths of
 *     its sides towards E, N, W, S that lie inside the body rectangle,
 *     outside the disk (sides on an outer edge are external faces: 0);
 *     zero elsewhere;
 *   bc_value[ny][nx][2]: u* at Dirichlet points (mean of the Dirichlet edges
 *     through the point); at Neumann points the traction t* of each outer
 *     edge (edge_type/edge_value as lbps_rect_bc, no periodic axes) times the
 *     length of the cell's face on that edge outside the disk; the hole
 *     itself carries no traction.
 * Host only, no device work.  The caller owns all arrays.  LBPS_ERR_INVALID
 * for sides < 3, dh <= 0, r < 0, non-finite input or an edge type other
 * than LBPS_NEUMANN / LBPS_DIRICHLET.  Whether the geometry is valid for the
 * method (a difference stencil at every body point) is checked by
 * lbps_create_cells. */
int lbps_disk_cells(int32_t nx, int32_t ny, double dh, double cx, double cy, double r,
                    const int32_t edge_type[4], const double edge_value[8], uint8_t* node_type,
                    double* bc_value, double* cell);

/* Initialisation (Fig. 3; Sec. 3 before Eq. integration): u(x,0), du/dt(x,0)
 * from host arrays [ny][nx]; phi, psi by finite differences of u; the
 * populations at equilibrium (Eq. feq).  vx0/vy0 may both be NULL (body at
 * rest); otherwise the first moments start at J_phi = -v, J_psi = (-v_y, v_x).
 * The input is copied into the state copy that is not current and checked
 * there on the device: non-finite input is rejected with LBPS_ERR_INVALID
 * and leaves the lattice as it was.  Synchronises.  With
 * 16-bit storage and pop_scale_exp 0, the storage scale is chosen here from a
 * device reduction over the initial state (lbps_scale_exp reports it). */
int lbps_init(lbps_lattice* lat, const double* ux0, const double* uy0,
              const double* vx0, const double* vy0);

/* As lbps_init with device arrays [ny][nx]; asynchronous, no finiteness check
 * (except that an automatic 16-bit scale choice waits for its reduction). */
int lbps_init_device(lbps_lattice* lat, const double* d_ux0, const double* d_uy0,
                     const double* d_vx0, const double* d_vy0);

/* Time loop of Fig. 3, n iterations: accelerations (Eq. navier,
 * acc_neumann, acc_dirichlet), Newmark (Eq. integration), boundary reset
 * (Eq. psi_phi_at_bound, correction-f), LBE with the averaged boundary state
 * (Eq. LBE, LBE_mod), and every sync_every-th step the synchronisation of
 * Sec. 3.2.  Enqueues the work, then waits for the stream and returns
 * LBPS_ERR_NONFINITE if any update produced a non-finite value. */
int lbps_step(lbps_lattice* lat, int64_t n);

/* As lbps_step without the final wait and check (use lbps_check later). */
int lbps_step_async(lbps_lattice* lat, int64_t n);

/* Waits for the stream; LBPS_ERR_NONFINITE if the state went non-finite
 * since the last initialisation. */
int lbps_check(lbps_lattice* lat);

/* Periodic synchronisation of Sec. 3.2 applied now to the current state. */
int lbps_sync(lbps_lattice* lat);

/* Copy a field to host memory as FP64 [ny][nx] (populations: [5][ny][nx]).
 * count is the capacity of dst in doubles.  Synchronises. */
int lbps_read(lbps_lattice* lat, int32_t field, double* dst, size_t count);

/* As lbps_read into device memory; asynchronous. */
int lbps_read_device(lbps_lattice* lat, int32_t field, double* d_dst, size_t count);

/* FP64 reductions over the lattice for one scalar field (LBPS_UX ..
 * LBPS_PSI, LBPS_CONSISTENCY .. LBPS_STRAIN_ENERGY): out[0] = sum (x - ref)^2,
 * out[1] = sum ref^2, out[2] = sum x, out[3] = max |x|.  d_ref is a device
 * array [ny][nx] or NULL (ref = 0).  Deterministic order.  Synchronises. */
int lbps_norms(lbps_lattice* lat, int32_t field, const double* d_ref, double out[4]);

/* Energy of the current state in FP64 on the device (a diagnostic; the paper
 * states the material law, Eq. hooke, and the strain, Eq. strain, but
 * reports no energy): out[0] = kinetic, out[1] = strain, out[2] = their sum,
 * each the sum over the body points of the density (LBPS_KINETIC_ENERGY,
 * LBPS_STRAIN_ENERGY) times dh^2, per unit thickness.  Every body point
 * counts one square of side dh; boundary cells are not clipped.  Waits for
 * the lattice's stream. */
int lbps_energy(lbps_lattice* lat, double out[3]);

/* lbps_norms without any allocation.  The paper has no counterpart: this is
 * a service routine for callers that cannot call cudaMalloc or cudaFree,
 * such as a serving loop that keeps all device memory in its own pool under a
 * fixed budget (an allocation behind its back breaks that accounting or
 * fails), or a latency-sensitive loop that must not stall on cudaFree, which
 * waits for the device.
 * Computes out[0] = sum (x - ref)^2, out[1] = sum ref^2, out[2] = sum x,
 * out[3] = max |x| over d_x[0..n) and d_ref[0..n) (device FP64 arrays the
 * caller owns; d_ref may be NULL for ref = 0), on cuda_stream (NULL = legacy
 * default stream), then waits for that stream and writes out (host).
 * Scratch: a fixed device array inside the library (2 MiB + 32 B per device
 * that loads it, held until the process exits), so n may be at most
 * LBPS_NOALLOC_MAX_POINTS; larger n returns LBPS_ERR_INVALID before any
 * device work.  Each call looks up the array's address on the current device.
 * The call ends by copying into the caller's host memory and waiting for the
 * stream, so it returns LBPS_ERR_INVALID, before any device work, when
 * cuda_stream is capturing.  All calls on a device share the array: calls
 * whose work overlaps on the GPU (other streams, other threads) race and must
 * be serialised by the caller.  out[3] is NaN if any x is NaN.
 * Each call overwrites every scratch slot it reads, so nothing in it needs
 * clearing between calls.  Calls no cudaMalloc, cudaFree or other allocating
 * routine. */
#define LBPS_NOALLOC_MAX_BLOCKS 65536
#define LBPS_NOALLOC_MAX_POINTS ((size_t)LBPS_NOALLOC_MAX_BLOCKS * 4096)
int lbps_norms_noalloc(const double* d_x, const double* d_ref, size_t n, void* cuda_stream, double out[4]);

/* ---- Batches: many lattices of different sizes, materials and edges
 * advanced together.  Each time step is two launches: a persistent grid
 * whose warps take tasks from one work list (strips of the interior of every
 * lattice, and groups of 32 boundary points for the Newmark pass), then the
 * boundary reset over the boundary points of every lattice (the same
 * per-point arithmetic as lbps_step, so every lattice gets the same bits as
 * when stepped alone).
 * Blocks of k steps (k even; 2 unless set or tuned) are captured once into
 * a CUDA graph and replayed.  The paper has no counterpart; this serves many
 * solves at once. */
typedef struct lbps_batch lbps_batch; /* opaque, library-owned */

/* lats[count]: distinct, initialised lattices, all of one storage format,
 * with sync_every == 0.  The batch keeps the pointers (not the lattices): destroy
 * the batch before any of its lattices.  cuda_stream: stream for the batch's
 * work (NULL: a blocking stream of the batch's own, ordered with the legacy
 * default stream).  Allocates a small device block for descriptors and work
 * lists (cudaMalloc). */
int lbps_batch_create(lbps_lattice* const* lats, int32_t count, void* cuda_stream, lbps_batch** out);

/* Advance every lattice of the batch by n steps (asynchronous; the work is
 * ordered after work queued on each lattice's stream, and later work on those
 * streams is ordered after it).  A lattice stepped on its own meanwhile is
 * picked up where it is. */
int lbps_batch_step(lbps_batch* b, int64_t n);

/* Waits; LBPS_ERR_NONFINITE if any lattice of the batch went non-finite. */
int lbps_batch_check(lbps_batch* b);

/* Launch shape of the batch's interior kernel (as lbps_set_tuning;
 * rows_per_warp 8..4096).  Results do not depend on it.  Defaults: 5, 16
 * (the batched kernel keeps each lattice's parameters in registers, so the
 * 6-blocks-per-SM variants spill there). */
int lbps_batch_set_tuning(lbps_batch* b, int32_t variant, int32_t rows_per_warp);

/* Steps per replayed CUDA graph: k even, 2..64 (LBPS_ERR_INVALID
 * otherwise).  lbps_batch_step(n) replays floor(n / k) graphs of k steps,
 * then pairs, then launches a last odd step directly.  Results do not depend
 * on it.  lbps_batch_graph_steps returns the current k. */
int lbps_batch_set_graph_steps(lbps_batch* b, int32_t k);
int lbps_batch_graph_steps(const lbps_batch* b);

/* Two time steps per sweep for every lattice of the batch (on != 0) or one
 * (0, the default), as lbps_set_step_pairs does for one lattice: each pair
 * of steps is four launches, a persistent kernel that advances the points at
 * least 3 from every edge of every lattice by two steps and runs the first
 * step on the points 1..3 from the edges and its boundary Newmark pass into
 * each lattice's scratch copy, the first step's reset, a persistent kernel
 * for the second step on the points 1..2 from the edges and its Newmark pass,
 * and the second step's reset.  Every lattice gets the same bits as when it
 * takes two steps per sweep on its own.  Turning it on calls
 * lbps_set_step_pairs(lat, 1) for every lattice (a scratch state copy each;
 * its error code if that fails) and returns LBPS_ERR_INVALID, changing
 * nothing, if a lattice is not a rectangle without periodic axes and at least
 * 16 points a side.  lbps_batch_step then runs n / 2 pairs and an odd last
 * step as a single step; no CUDA graph (the launches are few per pair).
 * lbps_batch_step_pairs returns 1 if on, 0 if off. */
int lbps_batch_set_step_pairs(lbps_batch* b, int32_t on);
int lbps_batch_step_pairs(const lbps_batch* b);

/* Autotuner: times one step for each launch shape (variants 0, 1, 2, 4, 5,
 * 6 x rows 8, 16, 32, 64, 128), repeats times each, keeps the fastest; then,
 * for that shape, times graphs of k = 2, 4, 8, 16, 32 steps (a longer graph
 * must be 1 % faster per step) and keeps the fastest k.  ms_per_step is the
 * time per step replayed from that graph.  Leaves every lattice's state
 * unchanged (a step is a pure function of the copy it reads; the timed steps
 * only rewrite the same next state, and the step counters are put back). */
int lbps_batch_tune(lbps_batch* b, int32_t repeats, int32_t* variant, int32_t* rows_per_warp,
                    double* ms_per_step);

/* cudaError_t of the batch's last failing CUDA call (0 if none). */
int lbps_batch_last_cuda_error(const lbps_batch* b);

void lbps_batch_destroy(lbps_batch* b);

/* Derived constants (Eq. conditions-parameters): out[0] c_d, out[1] c_s,
 * out[2] a_phi, out[3] a_psi, out[4] a_{0,psi}, out[5] Delta t; and the
 * number of completed time steps. */
int lbps_info(const lbps_lattice* lat, double out[6], int64_t* steps_done);

/* Checkpoint / resume (not in the paper).  A saved state is a small header
 * (sizes, storage format, step count, 16-bit scale, a 64-bit fingerprint of
 * the parameters and boundary description) and the raw current state copy:
 * the populations in the storage format and u, du/dt, so a lattice that
 * loads it continues bit-for-bit where the saved one was.  The parameters,
 * boundary data and load schedule are the lattice's own and are not saved:
 * load into a lattice created the same way (same parameters, node types,
 * boundary values and cells; the load schedule is not checked).
 *   lbps_state_size: bytes of a saved state.
 *   lbps_state_save: copies it into dst (host or device memory, at least
 *     lbps_state_size bytes); synchronises.  LBPS_ERR_STATE before init.
 *   lbps_state_load: restores it (the lattice counts as initialised); returns
 *     LBPS_ERR_INVALID if the header does not match this lattice (sizes,
 *     storage format, or the fingerprint of parameters and boundary
 *     description) or bytes is short.  Synchronises. */
int lbps_state_size(const lbps_lattice* lat, size_t* bytes);
int lbps_state_save(lbps_lattice* lat, void* dst, size_t bytes);
int lbps_state_load(lbps_lattice* lat, const void* src, size_t bytes);

/* Time-dependent boundary data (Sec. 4: the tension example ramps its
 * traction linearly to 0.005 mu at t = L/c_s and holds it; the shear example
 * ramps without end).  The values of one kind (kind = LBPS_NEUMANN: the
 * forces F, LBPS_DIRICHLET: the targets u*) given to lbps_create are
 * multiplied by s(t) = min(t, t_hold) / t_ramp, with t = n dt after n steps:
 * the Neumann force of a step is taken at its start t_n, the Dirichlet
 * target at its end t_{n+1} (the displacement the point lands on).
 * t_ramp = 0 restores constant data; t_hold may be +infinity.  The step
 * count n is kept on the device (reset by init, advanced by every step of
 * lbps_step or a batch).  LBPS_ERR_INVALID for another kind, t_ramp < 0 or
 * not finite, or t_hold <= 0.  The paper gives no more general schedule. */
int lbps_set_load(lbps_lattice* lat, int32_t kind, double t_ramp, double t_hold);

/* The exponent e of the 16-bit storage scale in use (Nx, Ny are stored
 * times 2^e; fixed by pop_scale_exp or chosen by the last init); 0 for FP32
 * and FP64 storage.  The paper stores populations in full precision; the
 * compressed formats are this library's. */
int lbps_scale_exp(const lbps_lattice* lat, int32_t* exp);

/* The value codec of a 16-bit storage format (storage = LBPS_STORAGE_BF16,
 * _F16 or _BFP13) on n values in caller-owned device arrays d_x (FP32) and
 * d_code (n 16-bit slots), enqueued on cuda_stream (NULL = legacy default
 * stream), not waited for.  encode = 1 writes the codes of d_x as the time
 * step rounds stored pair sums (d_x already multiplied by 2^e); encode = 0
 * writes into d_x the values of d_code.  BF16, FP16: d_code[i] is the code
 * of d_x[i], rounded to nearest (ties to even) with stochastic = 0, else
 * stochastically with the random bits hashed from d_x[i] and the key
 * 4 i + key0 (a point at plane offset i, slot key0 of 0..3, on a lattice with
 * no row offset).  BFP13: the values pair up, (d_x[2i], d_x[2i+1]) = (Nx, Ny)
 * in the 32-bit word d_code[2i] | d_code[2i+1] << 16 (n even, d_x 8-byte
 * and d_code 4-byte aligned; key0 and stochastic are not used).  Non-finite values and overflow give the format's
 * infinity.  Lets a caller read or reproduce stored sums.  LBPS_ERR_INVALID
 * for another storage, n < 0, a BFP13 call breaking those conditions, a null
 * array with n > 0, or encode or stochastic not 0 or 1; LBPS_ERR_CUDA if the
 * launch fails. */
int lbps_codec16(int32_t storage, int32_t encode, float* d_x, uint16_t* d_code, int64_t n, uint32_t key0,
                 int32_t stochastic, void* cuda_stream);

/* The CUDA runtime error code (a cudaError_t value) of the most recent
 * step, check or initialisation of this lattice that returned
 * LBPS_ERR_CUDA; 0 if none. */
int lbps_last_cuda_error(const lbps_lattice* lat);

/* Diagnostics of a checked build (compiled with LBPS_CHECKED): every device
 * access of the time-loop kernels is checked for alignment and against the
 * device blocks of the live lattices (at most 1024), and the first violation
 * since the library was loaded is recorded instead of performed.  Returns 1
 * and out[0] = source line, out[1] = address of that first violation (0, 0
 * if none) in a checked build; returns 0 and zeros in a normal build.  Waits
 * for the device. */
int lbps_check_report(uint64_t out[2]);

/* Launch shape of the interior kernel (performance only; results are
 * bit-identical for every setting).  variant 0..3 selects the register budget
 * (0: 6 blocks of 128 threads per SM, 1: 5, 2: 4, 3: 8) with u, du/dt loaded
 * two rows ahead; 4..7 the same budgets loading them one row ahead.
 * rows_per_warp (1..4096) is the number of rows each warp marches over.
 * Defaults: variant 0 (variant 2 for FP64 storage, which needs more
 * registers, and 4 for BFP13, whose codec does); 32 rows, or 16 or 8 on lattices too small to give the
 * interior kernel 16384 warps at 32 (below about 4096^2); 16 rows from
 * 640000 to 2000000 points and 4 rows below 640000 (measured best). */
int lbps_set_tuning(lbps_lattice* lat, int32_t variant, int32_t rows_per_warp);

/* Steps per CUDA graph of lbps_step: k even, 2..64 (LBPS_ERR_INVALID
 * otherwise; default 32).  lbps_step captures k consecutive steps once per
 * starting state copy and replays them; what is left of n (or a block a
 * synchronisation would split) runs as pairs from a 2-step graph or as
 * direct launches.  Results do not depend on it; a larger k saves launch
 * time on small lattices. */
int lbps_set_graph_steps(lbps_lattice* lat, int32_t k);

/* Two time steps per sweep of the interior (on != 0) or one (0, the default).
 * Applies to rectangles without periodic axes and at least 16 points a side
 * (other lattices keep single steps): the points at least 3 from every edge
 * advance two steps in one pass of a kernel that reads the state once and
 * writes it once; the boundary rules and the points up to 3 from the edges
 * run step by step through a scratch state copy, beside it.  The kernel
 * integrates u, du/dt of its points over both steps in one composed Newmark
 * update (Eq. integration applied twice, the sums of the two accelerations
 * taken in the populations' arithmetic type): the populations are the same
 * bits as single steps between synchronisations, u and du/dt the same up to
 * rounding.  Allocates the scratch copy (cudaMalloc, the
 * size of one state copy; LBPS_ERR_OOM if that fails) and frees it when
 * turned off or at lbps_destroy.  A synchronisation point that falls between
 * the two steps of a pair makes that pair two single steps.  With
 * lbps_profile on, the events of each pair bracket the two-step kernel only.
 * Below 12 x 2^20 points (and without per-kernel timing or synchronisation)
 * the pairs run as a batch of this one lattice (lbps_batch_set_step_pairs:
 * four launches a pair), from there on as the two-step kernel beside a chain
 * of boundary and frame launches on a second stream of greatest priority;
 * both give the same bits.  It pays from about 1700^2 points (FP32: 8192^2
 * 75.1 against 43.2 GLUPS; 4096^2 68.8 against 41.9; 2048^2 46.3 against
 * 37.1; 1536^2 32.5 against 33.6). */
int lbps_set_step_pairs(lbps_lattice* lat, int32_t on);

/* 1 if lbps_step takes two steps per sweep on this lattice (turned on and
 * applicable), else 0. */
int lbps_step_pairs(const lbps_lattice* lat);

/* Per-kernel timing for roofline reports.  enable != 0 starts recording CUDA
 * events on the lattice's stream around the interior kernel of every step
 * and around the boundary reset after it (the boundary Newmark pass runs on
 * a second stream beside the interior kernel and is not timed); 0 stops.
 * lbps_profile_read waits for the stream and returns, since recording
 * started: out[0] total milliseconds in the bulk (interior) kernel, out[1]
 * its launches, out[2] total milliseconds in the timed boundary passes,
 * out[3] their number (one per step; two if the second stream could not be
 * created, the Newmark pass then running, timed, on the lattice's stream);
 * then clears the record. */
int lbps_profile(lbps_lattice* lat, int32_t enable);
int lbps_profile_read(lbps_lattice* lat, double out[4]);

/* ---- Domain decomposition (not in the paper, whose only remark on
 * parallelism is that it is easy with most LBMs, Sec. 1).  A large lattice
 * split into slabs of rows, each a lattice of its own with a few ghost rows
 * beyond each cut, exchanges those rows with its neighbours after every
 * step; see paper_2301_00228_gb300/slab.py for the plan.
 *   lbps_halo_bytes: bytes of `rows` rows of the current state: every
 *     population plane (storage layout) and u_x, u_y, v_x, v_y, plane after
 *     plane, rows x (nx rounded up to 32) elements each.
 *   lbps_halo_pack: rows [row0, row0 + rows) of the current state into d_buf
 *     (device memory, 16-byte aligned, at least lbps_halo_bytes bytes, owned
 *     by the caller); asynchronous on the lattice's stream.
 *   lbps_halo_unpack: the same rows from d_buf into the current state, then
 *     recomputes what the state carries besides them (boundary stresses and
 *     the boundary mirror); asynchronous.
 * LBPS_ERR_INVALID for a bad row range, a short or misaligned buffer;
 * LBPS_ERR_STATE before init. */
int lbps_halo_bytes(const lbps_lattice* lat, int32_t rows, size_t* bytes);
int lbps_halo_pack(lbps_lattice* lat, int32_t row0, int32_t rows, void* d_buf, size_t bytes);
int lbps_halo_unpack(lbps_lattice* lat, int32_t row0, int32_t rows, const void* d_buf, size_t bytes);

/* The lattice is rows [row0, row0 + ny) of a larger one (a slab): the 16-bit
 * formats' stochastic rounding then draws its random bits from the global
 * position, so a slab rounds its rows as the whole lattice does.  Call before
 * lbps_init.  No effect for FP32 / FP64 storage. */
int lbps_set_origin(lbps_lattice* lat, int64_t row0);

/* Switch the stream used by later calls. */
int lbps_set_stream(lbps_lattice* lat, void* cuda_stream);

/* Release the lattice and any device memory the library allocated. */
void lbps_destroy(lbps_lattice* lat);

#ifdef __cplusplus
}
#endif
#endif /* LBPS_H */
