// CUDA kernels of the plane-strain lattice Boltzmann time loop
// (arXiv:2301.00228, algorithm summary of Fig. 3), sm_103a.
//
// One time step is two launches on the same stream:
//   boundary_kernel  one thread per boundary point: acceleration by Eq.
//                    acc_neumann / acc_dirichlet, Newmark (Eq. integration),
//                    phi, psi from differences of the new u (Eq.
//                    psi_phi_at_bound; the new u of the few stencil points is
//                    recomputed locally), populations by Eq. correction-f.
//                    Writes u, du/dt and the populations of boundary points
//                    of copy B.
//   bulk_kernel      every other point: interior acceleration (Eq. navier),
//                    Newmark, and the pull form of the LBE (Eq. LBE) with the
//                    time-averaged state of boundary sources (Eq. LBE_mod),
//                    which it reads from copy B.  Memory-bound stencil: reads
//                    copy A once, writes copy B once.
// Copies A (time t) and B (time t + dt) swap after each step.
#include "lbps_launch.h"

namespace lbps {

namespace {

enum {
    FLD_UX = 0, FLD_UY = 1, FLD_VX = 2, FLD_VY = 3, FLD_PHI = 4, FLD_PSI = 5,
    FLD_FPHI = 6, FLD_FPSI = 7, FLD_CONS = 8
};

template <typename T>
__device__ __forceinline__ T ld(const T* p) { return LBPS_LDG(p); }

// Sum of the five populations of one set at pitched offset p.
template <typename T>
__device__ __forceinline__ T moment0(const T* __restrict__ f, size_t plane, size_t p, int set) {
    const T* b = f + (size_t)set * 5 * plane + p;
    return sum5(ld(b), ld(b + plane), ld(b + 2 * plane), ld(b + 3 * plane), ld(b + 4 * plane));
}

// Equilibrium of Eq. feq for s and the lattice first moment Jbar = J / c
// (c cancels: c^alpha . J / (2 c^2) = e_alpha . Jbar / 2), written to plane
// set of copy V at offset p.
template <typename T>
__device__ __forceinline__ void store_feq(T* __restrict__ f, size_t plane, size_t p, int set, double a0,
                                          double a, double s, double jx, double jy) {
    T* b = f + (size_t)set * 5 * plane + p;
    double as = a * s;
    LBPS_ST(&b[0], (T)(a0 * s));
    LBPS_ST(&b[plane], (T)(as + 0.5 * jx));
    LBPS_ST(&b[2 * plane], (T)(as + 0.5 * jy));
    LBPS_ST(&b[3 * plane], (T)(as - 0.5 * jx));
    LBPS_ST(&b[4 * plane], (T)(as - 0.5 * jy));
}

// ------------------------------------------------------------------ init

// Fig. 3 initialisation: phi = div u, psi = curl u by finite differences of
// u(x, 0) (already copied into copy A), populations at equilibrium.
template <typename T>
__global__ void init_kernel(Geo g, Consts c, View<T> A) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const double* ux = A.u;
    const double* uy = A.u + g.plane;
    size_t p = (size_t)j * g.px + i;
    double phi = ddx(ux, g.px, i, j, g, c.inv2h) + ddy(uy, g.px, i, j, g, c.inv2h);
    double psi = ddx(uy, g.px, i, j, g, c.inv2h) - ddy(ux, g.px, i, j, g, c.inv2h);
    double vx = LBPS_LD(&A.u[2 * g.plane + p]), vy = LBPS_LD(&A.u[3 * g.plane + p]);
    // First moments from du/dt (J_phi = -v, J_psi = (-v_y, v_x)), in lattice
    // units Jbar = J dt / dh.
    double q = c.dt / c.dh;
    store_feq(A.f, g.plane, p, 0, c.a0[0], c.a[0], phi, -vx * q, -vy * q);
    store_feq(A.f, g.plane, p, 1, c.a0[1], c.a[1], psi, -vy * q, vx * q);
}

// ------------------------------------------------------------- boundary

// Cauchy stress from differences of u (Eq. strain in Eq. hooke): s = {xx, yy, xy}.
__device__ inline void stress_at(const Geo& g, const Consts& c, const double* ux, const double* uy, int i,
                                 int j, double s[3]) {
    double exx = ddx(ux, g.px, i, j, g, c.inv2h);
    double eyy = ddy(uy, g.px, i, j, g, c.inv2h);
    double exy = 0.5 * (ddy(ux, g.px, i, j, g, c.inv2h) + ddx(uy, g.px, i, j, g, c.inv2h));
    double tr = exx + eyy;
    s[0] = c.lam * tr + 2.0 * c.mu * exx;
    s[1] = c.lam * tr + 2.0 * c.mu * eyy;
    s[2] = 2.0 * c.mu * exy;
}

// Eq. acc_neumann for the boundary cell of (i, j): the square of side dh
// clipped to the rectangle; one face per existing neighbour r with normal
// pointing to r, length l_kr, stress (sigma_k + sigma_r)/2; external force
// F = int t* da supplied per point.  The stresses come from the stress pass:
// sig0[b] at boundary point b, sig1[b] at its interior neighbour.
__device__ inline void accel_neumann(const Geo& g, const Consts& c, const double* __restrict__ sig, int nb, int b,
                                     int i, int j, double fx, double fy, double& ax, double& ay) {
    const int DX[4] = {1, 0, -1, 0};
    const int DY[4] = {0, 1, 0, -1};
    bool has[4];
    has[0] = g.periodic_x || i < g.nx - 1;
    has[1] = g.periodic_y || j < g.ny - 1;
    has[2] = g.periodic_x || i > 0;
    has[3] = g.periodic_y || j > 0;
    double half = 0.5 * c.dh;
    double wx = (has[0] ? half : 0.0) + (has[2] ? half : 0.0);
    double wy = (has[1] ? half : 0.0) + (has[3] ? half : 0.0);
    double sk[3];
    for (int q = 0; q < 3; ++q) sk[q] = LBPS_LD(&sig[(size_t)b * 3 + q]);
    for (int d = 0; d < 4; ++d) {
        if (!has[d]) continue;
        int ri = wrap(i + DX[d], g.nx), rj = wrap(j + DY[d], g.ny);
        size_t slot = is_boundary(ri, rj, g) ? (size_t)perim_index(ri, rj, g) : (size_t)nb + b;
        double sr[3];
        for (int q = 0; q < 3; ++q) sr[q] = LBPS_LD(&sig[slot * 3 + q]);
        double sxx = 0.5 * (sk[0] + sr[0]);
        double syy = 0.5 * (sk[1] + sr[1]);
        double sxy = 0.5 * (sk[2] + sr[2]);
        double len = DX[d] != 0 ? wy : wx;
        fx += (sxx * DX[d] + sxy * DY[d]) * len;
        fy += (sxy * DX[d] + syy * DY[d]) * len;
    }
    // 1 / (rho V_C): V_C = wx wy is dh^2, dh^2/2 or dh^2/4 (exact powers of two)
    double inv_m = c.inv_rho_dh2 * ((has[0] && has[2]) ? 1.0 : 2.0) * ((has[1] && has[3]) ? 1.0 : 2.0);
    ax = fx * inv_m;
    ay = fy * inv_m;
}

// Value streamed out of a boundary source (Eq. LBE_mod).  f-hat is the mean
// of the stored (A) and reset (B) populations of the source; the
// equilibrium is taken from f-hat (mode 0) or from f(x_k, t) (mode 1).
// ALPHA is the direction of travel (1..4), OPP its reverse.
template <int ALPHA, int OPP, typename T>
__device__ inline T stream_from_boundary(const T* __restrict__ fa, const T* __restrict__ fb, size_t plane,
                                         const KC<T>& k, int set, int mode) {
    T a5[5], h5[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        a5[q] = ld(fa + q * plane);
        h5[q] = mul_rn((T)0.5, add_rn(a5[q], LBPS_LD(&fb[q * plane])));
    }
    if (mode == 0) {
        T sh = sum5(h5[0], h5[1], h5[2], h5[3], h5[4]);
        return fma_rn(k.two_a[set], sh, -h5[OPP]);  // 2 f_eq(f-hat) - f-hat = 2 a s-hat - f-hat^opp
    }
    T sa = sum5(a5[0], a5[1], a5[2], a5[3], a5[4]);
    T ej = sub_rn(a5[ALPHA], a5[OPP]);              // e_alpha . Jbar(x_k, t)
    return sub_rn(add_rn(mul_rn(k.two_a[set], sa), ej), h5[ALPHA]);
}

// Direction (1..4, D2Q5 numbering) from boundary point (i, j) towards its one
// interior neighbour, or 0 when it has none (corners, and points whose inward
// neighbour is itself on the boundary).
__device__ inline int inward_dir(int i, int j, const Geo& g) {
    bool l = !g.periodic_x && i == 0, r = !g.periodic_x && i == g.nx - 1;
    bool b = !g.periodic_y && j == 0, t = !g.periodic_y && j == g.ny - 1;
    if ((l || r) && (b || t)) return 0;  // corner
    if (l) return 1;                      // +x
    if (r) return 3;                      // -x
    if (b) return 2;                      // +y
    return 4;                             // -y (t)
}

// The boundary work of a step runs in three passes over the perimeter list,
// each one thread per boundary point b at (i, j):
//   stress   sigma at b and at its interior neighbour (for Eq. acc_neumann);
//   newmark  acceleration of b (Eq. acc_neumann or Eq. acc_dirichlet) and
//            u(t + dt) at b;
//   (the interior kernel runs here: u(t + dt) at every interior point)
//   reset    phi, psi from differences of u(t + dt) (Eq. psi_phi_at_bound),
//            populations by Eq. correction-f, and the value b streams into its
//            interior neighbour (Eq. LBE_mod), written over the population the
//            interior kernel put there.

__device__ inline void boundary_stress(const Geo& g, const Consts& c, const double* ux, const double* uy,
                                       const BNode* __restrict__ bn, int nb, double* __restrict__ sig, int b) {
    int i = LBPS_LD(&bn[b].i), j = LBPS_LD(&bn[b].j);
    double s[3];
    stress_at(g, c, ux, uy, i, j, s);
    for (int q = 0; q < 3; ++q) LBPS_ST(&sig[(size_t)b * 3 + q], s[q]);
    const int dir = inward_dir(i, j, g);
    if (dir != 0) {
        const int DX[5] = {0, 1, 0, -1, 0};
        const int DY[5] = {0, 0, 1, 0, -1};
        stress_at(g, c, ux, uy, i + DX[dir], j + DY[dir], s);
        for (int q = 0; q < 3; ++q) LBPS_ST(&sig[((size_t)nb + b) * 3 + q], s[q]);
    }
}

template <typename T>
__device__ inline void boundary_newmark(const Geo& g, const Consts& c, const KC<T>& k, const View<T>& A,
                                        const View<T>& B, const BNode* __restrict__ bn, int nb,
                                        const double* __restrict__ sig, int b) {
    int i = LBPS_LD(&bn[b].i), j = LBPS_LD(&bn[b].j);
    const int btype = LBPS_LD(&bn[b].type);
    const double bx = LBPS_LD(&bn[b].bx), by = LBPS_LD(&bn[b].by);
    size_t p = (size_t)j * g.px + i;
    const double* ux = A.u;
    const double* uy = A.u + g.plane;
    const double* vx = A.u + 2 * g.plane;
    const double* vy = A.u + 3 * g.plane;
    double ax, ay;
    if (btype == DIRICHLET) {
        ax = c.two_dt2 * (bx - LBPS_LD(&ux[p])) - c.two_dt * LBPS_LD(&vx[p]);
        ay = c.two_dt2 * (by - LBPS_LD(&uy[p])) - c.two_dt * LBPS_LD(&vy[p]);
    } else {
        accel_neumann(g, c, sig, nb, b, i, j, bx, by, ax, ay);
    }
    double ux1, uy1, vx1, vy1;
    newmark(LBPS_LD(&ux[p]), LBPS_LD(&vx[p]), ax, c, ux1, vx1);
    newmark(LBPS_LD(&uy[p]), LBPS_LD(&vy[p]), ay, c, uy1, vy1);
    LBPS_ST(&B.u[p], ux1);
    LBPS_ST(&B.u[g.plane + p], uy1);
    LBPS_ST(&B.u[2 * g.plane + p], vx1);
    LBPS_ST(&B.u[3 * g.plane + p], vy1);
}

template <typename T>
__device__ inline bool boundary_reset(const Geo& g, const Consts& c, const KC<T>& k, const View<T>& A,
                                      const View<T>& B, const BNode* __restrict__ bn, int b) {
    int i = LBPS_LD(&bn[b].i), j = LBPS_LD(&bn[b].j);
    size_t p = (size_t)j * g.px + i;
    const double* ux1 = B.u;
    const double* uy1 = B.u + g.plane;
    // Eq. psi_phi_at_bound: differences of u(t + dt) at (i, j).
    Sten sx = stencil(i, g.nx, g.periodic_x), sy = stencil(j, g.ny, g.periodic_y);
    double dux_dx = 0.0, duy_dx = 0.0, dux_dy = 0.0, duy_dy = 0.0;
    for (int q = 0; q < sx.n; ++q) {
        size_t o = (size_t)j * g.px + wrap(i + sx.d[q], g.nx);
        dux_dx = fma_rn(sx.w[q], LBPS_LD(&ux1[o]), dux_dx);
        duy_dx = fma_rn(sx.w[q], LBPS_LD(&uy1[o]), duy_dx);
    }
    for (int q = 0; q < sy.n; ++q) {
        size_t o = (size_t)wrap(j + sy.d[q], g.ny) * g.px + i;
        dux_dy = fma_rn(sy.w[q], LBPS_LD(&ux1[o]), dux_dy);
        duy_dy = fma_rn(sy.w[q], LBPS_LD(&uy1[o]), duy_dy);
    }
    double phi = mul_rn(dux_dx, c.inv2h) + mul_rn(duy_dy, c.inv2h);
    double psi = mul_rn(duy_dx, c.inv2h) - mul_rn(dux_dy, c.inv2h);
    // Eq. correction-f with J(x_k, t) of the stored populations, then the value
    // this point streams into its interior neighbour (Eq. LBE_mod): population
    // dir of that neighbour, replacing what the interior kernel wrote there.
    const int dir = inward_dir(i, j, g);
    const int DX[5] = {0, 1, 0, -1, 0};
    const int DY[5] = {0, 0, 1, 0, -1};
    const size_t pin = dir ? (size_t)(j + DY[dir]) * g.px + (i + DX[dir]) : p;
#pragma unroll
    for (int set = 0; set < 2; ++set) {
        const T* fa = A.f + (size_t)set * 5 * g.plane + p;
        const T* fb = B.f + (size_t)set * 5 * g.plane + p;
        double jx = (double)ld(fa + g.plane) - (double)ld(fa + 3 * g.plane);
        double jy = (double)ld(fa + 2 * g.plane) - (double)ld(fa + 4 * g.plane);
        store_feq(B.f, g.plane, p, set, c.a0[set], c.a[set], set == 0 ? phi : psi, jx, jy);
        T v = (T)0;
        switch (dir) {
        case 1: v = stream_from_boundary<1, 3>(fa, fb, g.plane, k, set, c.bc_feq_mode); break;
        case 2: v = stream_from_boundary<2, 4>(fa, fb, g.plane, k, set, c.bc_feq_mode); break;
        case 3: v = stream_from_boundary<3, 1>(fa, fb, g.plane, k, set, c.bc_feq_mode); break;
        case 4: v = stream_from_boundary<4, 2>(fa, fb, g.plane, k, set, c.bc_feq_mode); break;
        default: break;
        }
        if (dir != 0) LBPS_ST(&B.f[((size_t)set * 5 + dir) * g.plane + pin], v);
    }
    return !isfinite((T)phi + (T)psi);
}

template <typename T>
__global__ void __launch_bounds__(128) boundary_stress_kernel(Geo g, Consts c, View<T> A,
                                                              const BNode* __restrict__ bn, int nb, double* sig) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) boundary_stress(g, c, A.u, A.u + g.plane, bn, nb, sig, b);
}

template <typename T>
__global__ void __launch_bounds__(128) boundary_newmark_kernel(Geo g, Consts c, KC<T> k, View<T> A, View<T> B,
                                                               const BNode* __restrict__ bn, int nb,
                                                               const double* __restrict__ sig) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) boundary_newmark(g, c, k, A, B, bn, nb, sig, b);
}

template <typename T>
__global__ void __launch_bounds__(128) boundary_reset_kernel(Geo g, Consts c, KC<T> k, View<T> A, View<T> B,
                                                             const BNode* __restrict__ bn, int nb, unsigned* flag) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb && boundary_reset(g, c, k, A, B, bn, b)) atomicOr(flag, 1u);
}

// ---------------------------------------------------------------- bulk

// Bulk kernel: each warp owns a strip of kStripCols output columns and marches
// along y over kRowsPerWarp rows.  Lane l holds column xs - 1 + l, so lanes 0
// and 31 are halo lanes whose values reach their neighbours by shuffles; the
// rows above and below stay in registers, and the populations are prefetched
// two rows ahead.  Every lattice point's 14 words are read once per launch
// (plus the two halo columns and two halo rows of each strip).
constexpr int kStripCols = 30;
constexpr int kWarpsPerBlock = 4;

template <typename T>
__device__ __forceinline__ void load_row(const T* __restrict__ F, size_t plane, size_t p, bool ok, T (&f)[2][5]) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int q = 0; q < 5; ++q) f[s][q] = ok ? ld(F + (size_t)(s * 5 + q) * plane + p) : (T)0;
}

__device__ __forceinline__ void load_uv(const double* __restrict__ U, size_t plane, size_t p, bool ok,
                                        double (&u)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = ok ? ld(U + (size_t)q * plane + p) : 0.0;
}

// One warp's strip: output columns [xs, xs + kStripCols) of rows [j0, j1).
// Returns true in lanes that produced a non-finite value.  All 32 lanes of
// the warp must call it together (warp shuffles).
template <typename T>
__device__ __forceinline__ bool bulk_strip(const Geo& g, const Consts& c, const KC<T>& k, const View<T>& A,
                                           const View<T>& B, int xs, int j0, int j1) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int xl = xs - 1 + lane;
    const bool col_ok = g.periodic_x ? (xl <= g.nx) : (xl >= 0 && xl < g.nx);
    const int col = col_ok ? wrap(xl, g.nx) : 0;
    const bool out_lane = lane >= 1 && lane <= kStripCols && xl < g.nx &&
                          (g.periodic_x || (xl > 0 && xl < g.nx - 1));
    const size_t P = g.plane;

    auto row_ok = [&](int j) { return g.periodic_y || (j >= 0 && j < g.ny); };
    auto row_of = [&](int j) { return g.periodic_y ? wrap(j, g.ny) : j; };
    // Offsets are formed only for rows inside the lattice (rows outside are
    // clamped; their loads are masked), so no address ever leaves the planes
    // even where a masked load is issued unconditionally.
    auto at = [&](int j) { return (size_t)min(max(row_of(j), 0), g.ny - 1) * (size_t)g.px + (size_t)col; };

    T Ps[2], Pf4[2];                          // row j - 1: moment and f^4
    T Cf[2][5], Cs[2], Cm[2];                 // row j
    T Nf[2][5];                               // row j + 1
    T Qf[2][5];                               // row j + 2 (in flight)
    double Cu[4], Nu[4];
    {
        T t[2][5];
        load_row(A.f, P, at(j0 - 1), col_ok && row_ok(j0 - 1), t);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            Ps[s] = sum5(t[s][0], t[s][1], t[s][2], t[s][3], t[s][4]);
            Pf4[s] = t[s][4];
        }
    }
    load_row(A.f, P, at(j0), col_ok, Cf);
    load_row(A.f, P, at(j0 + 1), col_ok && row_ok(j0 + 1), Nf);
    load_uv(A.u, P, at(j0), out_lane, Cu);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        Cm[s] = add_rn(add_rn(Cf[s][1], Cf[s][2]), add_rn(Cf[s][3], Cf[s][4]));
        Cs[s] = add_rn(Cf[s][0], Cm[s]);
    }
    bool bad = false;
    for (int j = j0; j < j1; ++j) {
        // prefetch: populations two rows ahead, u and du/dt one row ahead
        load_row(A.f, P, at(j + 2), col_ok && row_ok(j + 2) && j + 2 <= j1, Qf);
        load_uv(A.u, P, at(j + 1), out_lane && j + 1 < j1, Nu);
        T Nm[2], Ns[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            Nm[s] = add_rn(add_rn(Nf[s][1], Nf[s][2]), add_rn(Nf[s][3], Nf[s][4]));
            Ns[s] = add_rn(Nf[s][0], Nm[s]);
        }
        const bool row_interior = g.periodic_y || (j > 0 && j < g.ny - 1);
        if (row_interior) {  // warp-uniform
            T sW[2], sE[2], out[2][5];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                sW[s] = __shfl_up_sync(FULL, Cs[s], 1);
                sE[s] = __shfl_down_sync(FULL, Cs[s], 1);
                T f3W = __shfl_up_sync(FULL, Cf[s][3], 1);
                T f1E = __shfl_down_sync(FULL, Cf[s][1], 1);
                // rest population: 2 a0 s - f0 = f0 + (2 a0 m - 8 a f0)
                out[s][0] = add_rn(Cf[s][0], fma_rn(k.two_a0[s], Cm[s], -mul_rn(k.eight_a[s], Cf[s][0])));
                // moving populations: f^alpha(x) = 2 a s(x - e_alpha) - f^opp(x - e_alpha)
                // (for sources on the boundary the reset pass overwrites them)
                out[s][1] = fma_rn(k.two_a[s], sW[s], -f3W);
                out[s][3] = fma_rn(k.two_a[s], sE[s], -f1E);
                out[s][2] = fma_rn(k.two_a[s], Ps[s], -Pf4[s]);
                out[s][4] = fma_rn(k.two_a[s], Ns[s], -Nf[s][2]);
            }
            if (out_lane) {
                double ax, ay;
                accel_interior<T>(sW[0], sE[0], Ps[0], Ns[0], sW[1], sE[1], Ps[1], Ns[1], k, ax, ay);
                double u1[4];
                newmark(Cu[0], Cu[2], ax, c, u1[0], u1[2]);
                newmark(Cu[1], Cu[3], ay, c, u1[1], u1[3]);
                const size_t p = at(j);
#pragma unroll
                for (int s = 0; s < 2; ++s)
#pragma unroll
                    for (int q = 0; q < 5; ++q) LBPS_ST(&B.f[(size_t)(s * 5 + q) * P + p], out[s][q]);
#pragma unroll
                for (int q = 0; q < 4; ++q) LBPS_ST(&B.u[(size_t)q * P + p], u1[q]);
                bad |= !isfinite(out[0][0] + out[1][0]);
            }
        }
        // shift the row window
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            Ps[s] = Cs[s];
            Pf4[s] = Cf[s][4];
            Cs[s] = Ns[s];
            Cm[s] = Nm[s];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                Cf[s][q] = Nf[s][q];
                Nf[s][q] = Qf[s][q];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) Cu[q] = Nu[q];
    }
    return bad;
}

template <typename T, int MINB>
__global__ void __launch_bounds__(128, MINB) bulk_kernel(Geo g, Consts c, KC<T> k, View<T> A, View<T> B,
                                                   unsigned* flag, int rows_per_warp) {
    const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int xs = warp * kStripCols;
    if (xs >= g.nx) return;  // whole warp
    const int j0 = blockIdx.y * rows_per_warp;
    const int j1 = min(j0 + rows_per_warp, g.ny);
    bool bad = bulk_strip(g, c, k, A, B, xs, j0, j1);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// --------------------------------------------------------------- batches

// The three boundary passes over the boundary points of every lattice in the
// batch (one thread per point).
template <typename T>
__global__ void __launch_bounds__(128) boundary_batch_kernel(const DomDesc<T>* __restrict__ dd,
                                                             const BndTask* __restrict__ tasks, int ntasks,
                                                             int parity, int pass) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntasks) return;
    const BndTask tk = tasks[t];
    const DomDesc<T>& d = dd[tk.dom];
    const int a = d.cur ^ parity;
    if (pass == 0)
        boundary_stress(d.g, d.c, d.v[a].u, d.v[a].u + d.g.plane, d.bn, d.nb, d.sig, tk.b);
    else if (pass == 1)
        boundary_newmark(d.g, d.c, d.k, d.v[a], d.v[a ^ 1], d.bn, d.nb, d.sig, tk.b);
    else if (boundary_reset(d.g, d.c, d.k, d.v[a], d.v[a ^ 1], d.bn, tk.b))
        atomicOr(d.flag, 1u);
}

// One warp per strip task of every lattice in the batch.
template <typename T, int MINB>
__global__ void __launch_bounds__(128, MINB) bulk_batch_kernel(const DomDesc<T>* __restrict__ dd,
                                                               const BulkTask* __restrict__ tasks, int ntasks,
                                                               int parity) {
    // Each warp copies its lattice's descriptor into shared memory, from where
    // the strip code reloads fields as it needs them (instead of holding them
    // in registers).
    __shared__ DomDesc<T> sd[kWarpsPerBlock];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * kWarpsPerBlock + wid;
    if (w >= ntasks) return;  // whole warp
    const BulkTask tk = tasks[w];
    {
        const unsigned* src = reinterpret_cast<const unsigned*>(dd + tk.dom);
        unsigned* dst = reinterpret_cast<unsigned*>(sd + wid);
        for (int q = lane; q < (int)(sizeof(DomDesc<T>) / 4); q += 32) dst[q] = src[q];
        __syncwarp();
    }
    const DomDesc<T>& d = sd[wid];
    const int a = d.cur ^ parity;
    bool bad = bulk_strip(d.g, d.c, d.k, d.v[a], d.v[a ^ 1], tk.xs, tk.j0, tk.j1);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(d.flag, 1u);
}

// ------------------------------------------------------------------ sync

// Sec. 3.2: phi, psi from differences of u at every point, populations by
// Eq. correction-f with the current first moments.  In place.
template <typename T>
__global__ void sync_kernel(Geo g, Consts c, View<T> A) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const double* ux = A.u;
    const double* uy = A.u + g.plane;
    size_t p = (size_t)j * g.px + i;
    double s[2];
    s[0] = ddx(ux, g.px, i, j, g, c.inv2h) + ddy(uy, g.px, i, j, g, c.inv2h);
    s[1] = ddx(uy, g.px, i, j, g, c.inv2h) - ddy(ux, g.px, i, j, g, c.inv2h);
    for (int set = 0; set < 2; ++set) {
        const T* fa = A.f + (size_t)set * 5 * g.plane + p;
        double jx = (double)fa[g.plane] - (double)fa[3 * g.plane];
        double jy = (double)fa[2 * g.plane] - (double)fa[4 * g.plane];
        store_feq(A.f, g.plane, p, set, c.a0[set], c.a[set], s[set], jx, jy);
    }
}

// ---------------------------------------------------------------- fields

template <typename T>
__device__ inline double moment0_fp64(const T* f, size_t plane, size_t p, int set) {
    const T* b = f + (size_t)set * 5 * plane + p;
    return (double)b[0] + (((double)b[plane] + (double)b[2 * plane]) + ((double)b[3 * plane] + (double)b[4 * plane]));
}

// Scalar field value at (i, j).
template <typename T>
__device__ inline double field_value(const Geo& g, const Consts& c, const View<T>& A, int field, int i, int j) {
    size_t p = (size_t)j * g.px + i;
    switch (field) {
    case FLD_UX: case FLD_UY: case FLD_VX: case FLD_VY: return A.u[(size_t)field * g.plane + p];
    case FLD_PHI: return moment0_fp64(A.f, g.plane, p, 0);
    case FLD_PSI: return moment0_fp64(A.f, g.plane, p, 1);
    default: {
        // consistency error e(x, t) of Sec. 4
        const double* ux = A.u;
        const double* uy = A.u + g.plane;
        double div = ddx(ux, g.px, i, j, g, c.inv2h) + ddy(uy, g.px, i, j, g, c.inv2h);
        double curl = ddx(uy, g.px, i, j, g, c.inv2h) - ddy(ux, g.px, i, j, g, c.inv2h);
        double e1 = moment0_fp64(A.f, g.plane, p, 1) - curl;
        double e0 = moment0_fp64(A.f, g.plane, p, 0) - div;
        return sqrt(e1 * e1 + e0 * e0);
    }
    }
}

// Dense FP64 copy of rows [j0, j0 + rows) of a field.  Population fields
// write 5 consecutive [rows][nx] blocks.
template <typename T>
__global__ void extract_kernel(Geo g, Consts c, View<T> A, int field, int j0, int rows, double* dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int jr = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || jr >= rows) return;
    int j = j0 + jr;
    size_t d = (size_t)jr * g.nx + i;
    if (field == FLD_FPHI || field == FLD_FPSI) {
        int set = field == FLD_FPHI ? 0 : 1;
        size_t p = (size_t)j * g.px + i;
        size_t blk = (size_t)rows * g.nx;
        for (int q = 0; q < 5; ++q) dst[q * blk + d] = (double)A.f[((size_t)set * 5 + q) * g.plane + p];
        return;
    }
    dst[d] = field_value(g, c, A, field, i, j);
}

// --------------------------------------------------------------- norms

constexpr int kNormThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kNormThreads) norms_partial_kernel(Geo g, Consts c, View<T> A, int field,
                                                                     const double* __restrict__ ref,
                                                                     double* partials) {
    __shared__ double sh[4][kNormThreads];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, mx = 0.0;
    size_t n = (size_t)g.nx * g.ny;
    for (size_t d = (size_t)blockIdx.x * blockDim.x + threadIdx.x; d < n; d += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(d % g.nx), j = (int)(d / g.nx);
        double x = field_value(g, c, A, field, i, j);
        double r = ref ? ref[d] : 0.0;
        double e = x - r;
        s0 += e * e;
        s1 += r * r;
        s2 += x;
        mx = fmax(mx, fabs(x));
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    sh[2][threadIdx.x] = s2;
    sh[3][threadIdx.x] = mx;
    __syncthreads();
    for (int w = kNormThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) partials[(size_t)blockIdx.x * 4 + q] = sh[q][0];
}

__global__ void __launch_bounds__(kNormThreads) norms_final_kernel(const double* partials, int nblk, double* out) {
    __shared__ double sh[4][kNormThreads];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += kNormThreads) {
        s[0] += partials[(size_t)b * 4];
        s[1] += partials[(size_t)b * 4 + 1];
        s[2] += partials[(size_t)b * 4 + 2];
        s[3] = fmax(s[3], partials[(size_t)b * 4 + 3]);
    }
    for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = kNormThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) out[q] = sh[q][0];
}

dim3 grid2d(int nx, int ny, dim3 blk) { return dim3((nx + blk.x - 1) / blk.x, (ny + blk.y - 1) / blk.y); }

}  // namespace

// ------------------------------------------------------------- launchers

template <typename T>
cudaError_t launch_boundary_batch(const DomDesc<T>* dd, const BndTask* tasks, int ntasks, int parity, int pass_lo,
                                  int pass_hi, cudaStream_t st) {
    if (ntasks > 0)
        for (int pass = pass_lo; pass < pass_hi; ++pass)
            boundary_batch_kernel<T><<<(ntasks + 127) / 128, 128, 0, st>>>(dd, tasks, ntasks, parity, pass);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bulk_batch(const DomDesc<T>* dd, const BulkTask* tasks, int ntasks, int parity, int variant,
                              cudaStream_t st) {
    if (ntasks <= 0) return cudaGetLastError();
    dim3 grid((ntasks + kWarpsPerBlock - 1) / kWarpsPerBlock), blk(32 * kWarpsPerBlock);
    switch (variant) {
    case 0: bulk_batch_kernel<T, 6><<<grid, blk, 0, st>>>(dd, tasks, ntasks, parity); break;
    case 1: bulk_batch_kernel<T, 5><<<grid, blk, 0, st>>>(dd, tasks, ntasks, parity); break;
    case 2: bulk_batch_kernel<T, 4><<<grid, blk, 0, st>>>(dd, tasks, ntasks, parity); break;
    default: bulk_batch_kernel<T, 8><<<grid, blk, 0, st>>>(dd, tasks, ntasks, parity); break;
    }
    return cudaGetLastError();
}

cudaError_t set_check_range(const void* base, size_t bytes, cudaStream_t st) {
#ifdef LBPS_CHECKED
    const char* lo = static_cast<const char*>(base);
    const char* hi = lo + bytes;
    unsigned long long zero = 0;
    cudaError_t e = cudaMemcpyToSymbolAsync(g_chk_lo, &lo, sizeof(lo), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_chk_hi, &hi, sizeof(hi), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_chk_line, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_chk_addr, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
#else
    (void)base;
    (void)bytes;
    (void)st;
    return cudaSuccess;
#endif
}

int check_report(unsigned long long out[2]) {
#ifdef LBPS_CHECKED
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    if (cudaMemcpyFromSymbol(&out[0], g_chk_line, sizeof(out[0])) != cudaSuccess) return -1;
    if (cudaMemcpyFromSymbol(&out[1], g_chk_addr, sizeof(out[1])) != cudaSuccess) return -1;
    return 1;
#else
    out[0] = out[1] = 0;
    return 0;
#endif
}

template <typename T>
cudaError_t launch_init(const Geo& g, const Consts& c, const KC<T>&, View<T> A, const double*, const double*,
                        const double*, const double*, cudaStream_t st) {
    dim3 blk(32, 8);
    init_kernel<T><<<grid2d(g.nx, g.ny, blk), blk, 0, st>>>(g, c, A);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_boundary(const Geo& g, const Consts& c, const KC<T>& k, View<T> A, View<T> B, const BNode* bn,
                            int nb, double* sig, unsigned* flag, cudaStream_t st, int pass_lo, int pass_hi) {
    if (nb > 0) {
        const int blocks = (nb + 127) / 128;
        for (int pass = pass_lo; pass < pass_hi; ++pass) {
            if (pass == 0) boundary_stress_kernel<T><<<blocks, 128, 0, st>>>(g, c, A, bn, nb, sig);
            if (pass == 1) boundary_newmark_kernel<T><<<blocks, 128, 0, st>>>(g, c, k, A, B, bn, nb, sig);
            if (pass == 2) boundary_reset_kernel<T><<<blocks, 128, 0, st>>>(g, c, k, A, B, bn, nb, flag);
        }
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bulk(const Geo& g, const Consts& c, const KC<T>& k, View<T> A, View<T> B, unsigned* flag,
                        cudaStream_t st, const Tuning& tu) {
    int warps = (g.nx + kStripCols - 1) / kStripCols;
    dim3 grid((warps + kWarpsPerBlock - 1) / kWarpsPerBlock, (g.ny + tu.rows_per_warp - 1) / tu.rows_per_warp);
    dim3 blk(32 * kWarpsPerBlock);
    switch (tu.variant) {
    case 0: bulk_kernel<T, 6><<<grid, blk, 0, st>>>(g, c, k, A, B, flag, tu.rows_per_warp); break;
    case 1: bulk_kernel<T, 5><<<grid, blk, 0, st>>>(g, c, k, A, B, flag, tu.rows_per_warp); break;
    case 2: bulk_kernel<T, 4><<<grid, blk, 0, st>>>(g, c, k, A, B, flag, tu.rows_per_warp); break;
    default: bulk_kernel<T, 8><<<grid, blk, 0, st>>>(g, c, k, A, B, flag, tu.rows_per_warp); break;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sync(const Geo& g, const Consts& c, const KC<T>&, View<T> A, cudaStream_t st) {
    dim3 blk(32, 8);
    sync_kernel<T><<<grid2d(g.nx, g.ny, blk), blk, 0, st>>>(g, c, A);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extract_rows(const Geo& g, const Consts& c, View<T> A, int field, int j0, int rows, double* dst,
                                cudaStream_t st) {
    dim3 blk(32, 8);
    extract_kernel<T><<<grid2d(g.nx, rows, blk), blk, 0, st>>>(g, c, A, field, j0, rows, dst);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extract(const Geo& g, const Consts& c, View<T> A, int field, double* dst, cudaStream_t st) {
    return launch_extract_rows<T>(g, c, A, field, 0, g.ny, dst, st);
}

template <typename T>
cudaError_t launch_norms(const Geo& g, const Consts& c, View<T> A, int field, const double* ref, double* partials,
                         double* out4, cudaStream_t st) {
    size_t n = (size_t)g.nx * g.ny;
    int nblk = (int)((n + kNormThreads - 1) / kNormThreads);
    if (nblk > kNormBlocks) nblk = kNormBlocks;
    norms_partial_kernel<T><<<nblk, kNormThreads, 0, st>>>(g, c, A, field, ref, partials);
    norms_final_kernel<<<1, kNormThreads, 0, st>>>(partials, nblk, out4);
    return cudaGetLastError();
}

#define LBPS_INSTANTIATE(T)                                                                                   \
    template cudaError_t launch_init<T>(const Geo&, const Consts&, const KC<T>&, View<T>, const double*,      \
                                        const double*, const double*, const double*, cudaStream_t);          \
    template cudaError_t launch_boundary<T>(const Geo&, const Consts&, const KC<T>&, View<T>, View<T>,        \
                                            const BNode*, int, double*, unsigned*, cudaStream_t, int, int);   \
    template cudaError_t launch_bulk<T>(const Geo&, const Consts&, const KC<T>&, View<T>, View<T>, unsigned*, \
                                        cudaStream_t, const Tuning&);                                         \
    template cudaError_t launch_sync<T>(const Geo&, const Consts&, const KC<T>&, View<T>, cudaStream_t);     \
    template cudaError_t launch_extract<T>(const Geo&, const Consts&, View<T>, int, double*, cudaStream_t);  \
    template cudaError_t launch_extract_rows<T>(const Geo&, const Consts&, View<T>, int, int, int, double*,   \
                                                cudaStream_t);                                                \
    template cudaError_t launch_norms<T>(const Geo&, const Consts&, View<T>, int, const double*, double*,    \
                                         double*, cudaStream_t);

LBPS_INSTANTIATE(float)
LBPS_INSTANTIATE(double)

template cudaError_t launch_boundary_batch<float>(const DomDesc<float>*, const BndTask*, int, int, int, int,
                                                  cudaStream_t);
template cudaError_t launch_boundary_batch<double>(const DomDesc<double>*, const BndTask*, int, int, int, int,
                                                   cudaStream_t);
template cudaError_t launch_bulk_batch<float>(const DomDesc<float>*, const BulkTask*, int, int, int, cudaStream_t);
template cudaError_t launch_bulk_batch<double>(const DomDesc<double>*, const BulkTask*, int, int, int, cudaStream_t);

}  // namespace lbps
